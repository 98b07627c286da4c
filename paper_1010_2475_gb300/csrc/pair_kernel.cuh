// All-pairs interaction kernel of the MMVM cross term (Appendix A.2).
//
// For a target j and a source j' the moment equations need the velocity jet
// of the source's Gaussian of core sqrt(2) lambda at the separation
// s = x^j - x^{j'} (eq:Fullint with b = s, eq:FinalCrossI/II), contracted with
// the source moments:  W_c[gamma] = sum_m M^{j'}_m D^{m+gamma} V_00,c(s; sqrt2 lambda).
// V_00 = grad-perp psi with the stream function psi of that Gaussian, so both
// components follow from one scalar correlation
//     Psi[beta] = sum_m a_m D^{m+beta} psi(b),   1 <= |beta| <= BMAX,
//     W_1[gamma] = -Psi[gamma + e2],  W_2[gamma] = Psi[gamma + e1],
// in units where c = 2 lambda^2 = 1: b = s / sqrt(c), a_m = M_m c^{-|m|/2}
// (the finish kernel undoes the scaling).
//
// Only the edge columns beta1 in {0, 1} (two per order) are contracted with
// the jet.  Since Lap psi = e^{-x}/pi and D_1^2 = Lap - D_2^2,
//     Psi[beta] = R[beta] - Psi[beta - 2 e1 + 2 e2]   (beta1 >= 2),
//     R[beta]   = sum_m a_m D^{m + beta - 2 e1} (e^{-x}/pi),
// and the Gaussian jet is a product of Hermite functions, so R is a separable
// double sum (over m2, then m1).  The kernel accumulates the edge columns and
// R in the same column layout as Psi; the finish kernel applies the
// recursion to the sums over all sources (in FP64).  Per pair this costs
// 2 x BMAX x K multiply-adds for the edges and K + (M+1) per Laplacian column
// group instead of K x |beta| for a full contraction.
//
// The jet D^alpha psi(b) is built one order at a time (1 <= |alpha| <= NJ =
// M + BMAX) and each order is added into the edge columns before the next
// order is formed, so only one order of the jet is live in registers; only
// the entries alpha1 <= M + 1 are formed.
//
// Jet of one order n (every step is exact):
//  * psi is radial, psi = Psi(|b|^2) with Psi' = (1 - e^{-x})/(4 pi x), so the
//    holomorphic edge is  d^n psi / dz^n = (1/4pi) (-1)^{n-1} zbar^n I_{n-1}(x),
//    I_k(x) = int_0^1 t^k e^{-xt} dt (x = |b|^2, z = b1 + i b2);
//  * Lap psi = e^{-x}/pi, whose Cartesian jet e_(a,b) = h_a(b1) h_b(b2) is a
//    product of Hermite functions h_k(t) = d^k/dt^k e^{-t^2} (1/pi folded in);
//  * with c_a = D_1^a D_2^{n-a} psi the Laplacian gives c_{a+2} = e_(a,n-2-a) - c_a,
//    i.e. c_a = (-1)^{floor(a/2)} c_{a mod 2} + chi_a with chi_0 = chi_1 = 0,
//    chi_{a+2} = e_(a,n-2-a) - chi_a;
//  * expanding d/dz = (D_1 - i D_2)/2 then fixes the two seeds:
//    c_0 + i c_1 = 2 i^n [ d^n psi/dz^n - 2^{-n} sum_a C(n,a) (-i)^{n-a} chi_a ].
// I_k is formed by the upward recurrence I_k = (k I_{k-1} - e^{-x})/x where it
// is stable (k <= x) and downward from a Kummer series at the top order
// otherwise; for x >= table_x(P) (well beyond the near field, and the self
// pair, which is moved far away) the edge zbar^n I_{n-1} itself is run upward
// in complex arithmetic so that nothing under- or overflows at large |b|.
//
// FP32 mode carries the separation as an exact pair b = b_hi + b_lo (the
// records hold zeta as (hi, lo) floats).  The Gaussian factors are sensitive
// to it (a relative error e in b moves e^{-x} by ~2 x e), so x = |b|^2 and
// e^{-x} are formed from the exact square, 1/x and the powers of zbar use the
// two-term value, and the Hermite functions get the first-order Taylor
// correction h_k(b) = h_k(b_hi) + b_lo h_{k+1}(b_hi).
#pragma once

#include "common.cuh"

namespace mmvm {

constexpr double kInvPi = 0.31830988618379067154;
constexpr double kInv4Pi = 0.07957747154594766788;

// 1/i, correctly rounded (compile-time), for the Kummer series below: the
// loop index is a run-time value, and a table read is cheaper than a
// correctly rounded reciprocal at run time.
struct RecipTable {
  float f[128];
  double d[128];
};
constexpr RecipTable make_recip_table() {
  RecipTable t{};
  for (int i = 1; i < 128; ++i) {
    t.f[i] = 1.0f / (float)i;
    t.d[i] = 1.0 / (double)i;
  }
  return t;
}
static __constant__ RecipTable kRecip = make_recip_table();

template <typename T> __device__ __forceinline__ T recip_of(int i);
template <> __device__ __forceinline__ float recip_of<float>(int i) { return kRecip.f[i]; }
template <> __device__ __forceinline__ double recip_of<double>(int i) { return kRecip.d[i]; }

// Terms of the FP32 Kummer series at order P: the smallest KN with
// prod_{j=1}^{KN} P / (P + 1 + j) below 2^-26, so that the terms dropped are
// below FP32 rounding of the sum for every x <= P (the series is only used
// there, or for x < 1).
constexpr int kummer_terms(int P) {
  double t = 1.0;
  int k = 0;
  while (t >= 1.0 / 67108864.0 && k < 120) {
    ++k;
    t *= (double)(P > 0 ? P : 1) / (double)(P + 1 + k);
  }
  return k + 1;
}
// Coefficients of the FP32 Horner form in y = x / Ps (Ps = max(P, 1)):
// d_k = Ps^k / ((P+1)(P+2)...(P+k+1)), all in (0, 1/(P+1)] and far inside the
// FP32 range (the unscaled 1 / ((P+1)...(P+k+1)) underflows it).
template <int P>
struct KummerCoef {
  static constexpr int KN = kummer_terms(P);
  static constexpr int PS = P > 0 ? P : 1;
  float c[KN];
  constexpr KummerCoef() : c() {
    double v = 1.0;
    for (int k = 0; k < KN; ++k) {
      v = v * (k > 0 ? (double)PS : 1.0) / (double)(P + 1 + k);
      c[k] = (float)v;
    }
  }
};

// sum_{k>=0} x^k / ((P+1)(P+2)...(P+k+1)) so that I_P(x) = e^{-x} * sum (x < P).
// FP32: a fixed Horner form (every coefficient positive, so it is as
// accurate as the term-by-term sum; no data-dependent trip count that would
// split the lanes of a warp).
template <int P, typename T>
__device__ __forceinline__ T kummer_sum(T x) {
  constexpr bool f32 = std::is_same<T, float>::value;
  if constexpr (f32) {
    constexpr KummerCoef<P> kc{};
    const T y = x * T(1.0 / KummerCoef<P>::PS);
    T s = T(kc.c[KummerCoef<P>::KN - 1]);
    static_for_down<0, KummerCoef<P>::KN - 1>([&](auto ic) {
      constexpr int k = decltype(ic)::value;
      s = fma(s, y, T(kc.c[k]));
    });
    return s;
  }
  const T eps = f32 ? T(2e-8) : T(5e-18);
  constexpr int kmax = f32 ? 48 : 80;
  static_assert(P + kmax < 128, "reciprocal table too short");
  T term = T(1.0 / (P + 1));
  T s = term;
#pragma unroll 1
  for (int k = 1; k < kmax; ++k) {
    term = term * x * recip_of<T>(P + 1 + k);
    s += term;
    if (term <= eps * s) break;
  }
  return s;
}

// Largest x = |b|^2 at which the edge takes the table form zbar^n I_{n-1}(x)
// up to n = P + 1 in FP32: there I_P(x) ~ P! / x^(P+1) stays above 1e-35 and
// |zbar|^(P+1) below 1e30, inside the normal FP32 range (I_17(300) ~ 1e-30,
// I_23(200) ~ 1e-33).  In FP32 the two forms agree to ~2e-6 of |w_n| at
// n = 18 over 20 <= x <= 400.
__host__ __device__ constexpr float table_x(int P) { return P <= 17 ? 300.f : 200.f; }

// Outputs of one order slice: Psi[beta] with LO <= |beta| <= HI, i.e. the
// columns [B0, B1).  They need the jet orders LO .. HI + M only.  PART 1
// accumulates only the edge columns (the jet), PART 2 only the Laplacian
// columns (Hermite functions, no jet), PART 0 both.
template <int M, typename T, int LO, int HI, int PART = 0>
struct PairNear {
  static constexpr int K = n_moments(M);
  static constexpr int NB = n_beta(M);
  static constexpr int NJ = HI + M;                // highest jet order of the slice
  static constexpr int NLO = LO;                    // lowest jet order of the slice
  static constexpr int BMAX = bmax_of(M);
  static constexpr int B0 = tri(LO) - 1;
  static constexpr int B1 = tri(HI + 1) - 1;
  static constexpr int NBL = B1 - B0;
  static constexpr int HN = NJ >= 2 ? NJ - 1 : 1;  // Hermite functions h_0..h_{NJ-2}
  // orders |gamma| = |beta| - 2 of the Laplacian columns of the slice
  static constexpr int GLO = LO > 2 ? LO - 2 : 0;
  static constexpr int GHI = HI - 2;
  static_assert(LO >= 1 && HI <= bmax_of(M) && LO <= HI, "bad order slice");

  // Add one source's contribution (moments a[K], separation b in c = 1 units)
  // to this slice acc[NBL] of Psi.  wmask = 0 removes the pair exactly (it is
  // used for the self pair, whose separation the caller moves far away).
  __device__ __forceinline__ static void run(T b1, T b2, T l1, T l2, T wmask,
                                             const T (&a)[K], T (&acc)[NBL]) {
    // squares (b_hi + b_lo)^2 = s_d + q_d + 2 b_hi b_lo (q_d: rounding of s_d)
    const T s1 = b1 * b1;
    const T s2 = b2 * b2;
    const T q1 = fma(b1, b1, -s1);
    const T q2 = fma(b2, b2, -s2);
    const T sl1 = q1 + T(2) * b1 * l1;
    const T sl2 = q2 + T(2) * b2 * l2;
    // x = xh + xl (TwoSum of the two squares plus the small corrections)
    const T xh = s1 + s2;
    const T bv = xh - s1;
    const T xl = ((s1 - (xh - bv)) + (s2 - bv)) + (sl1 + sl2);
    const T x = xh;
    // e^{-b_hi^2} per axis (the Hermite tables are built at b_hi) ...
    const T eh1 = dexp(-s1) * (T(1) - q1);
    const T eh2 = dexp(-s2) * (T(1) - q2);
    // ... and e^{-x} at the full separation
    const T E = eh1 * (T(1) - T(2) * b1 * l1) * (eh2 * (T(1) - T(2) * b2 * l2));
    // Hermite functions at b_hi, one order beyond what is used, then the
    // first-order correction to b = b_hi + b_lo: hx[k] = h_k(b1)/pi, hy[k] = h_k(b2)
    T hx[HN + 1], hy[HN + 1];
    hx[0] = eh1 * T(kInvPi);
    hy[0] = eh2;
    hx[1] = T(-2) * b1 * hx[0];
    hy[1] = T(-2) * b2 * hy[0];
    static_for<1, HN>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      hx[k + 1] = T(-2) * b1 * hx[k] - T(2 * k) * hx[k - 1];
      hy[k + 1] = T(-2) * b2 * hy[k] - T(2 * k) * hy[k - 1];
    });
    static_for<0, HN>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      hx[k] = fma(l1, hx[k + 1], hx[k]);
      hy[k] = fma(l2, hy[k + 1], hy[k]);
    });

    if constexpr (PART != 2) {
    // The holomorphic edge w_n = zbar^n I_{n-1}(x) is formed one order at a
    // time inside the order loop (only the current order is live): for
    // x < table_x(P) from the table I_k and the running power zbar^n, beyond
    // by the recursion w_{n+1} = (n zbar w_n - E zbar^{n+1}) / x, which
    // neither under- nor overflows at large |b|.  Near pairs lie below the
    // threshold, so the lanes of a warp agree and the per-order test does
    // not split the warp.
    constexpr int P = NJ - 1;
    const bool small = x < T(table_x(P));
    const T rxh = T(1) / x;  // inf at x == 0: those entries are replaced below
    const T rx = rxh * (T(1) - xl * rxh);
    T I[P + 1];
    if (small) {
      I[0] = (T(1) - E) * rx;
      static_for<1, P + 1>([&](auto nc) {
        constexpr int k = decltype(nc)::value;
        I[k] = (T(k) * I[k - 1] - E) * rx;
      });
      if (x < T(P) || x < T(1)) {
        T Id = E * kummer_sum<P, T>(x);
        static_for_down<1, P + 1>([&](auto nc) {
          constexpr int k = decltype(nc)::value;
          if (T(k) > x) I[k] = Id;
          Id = (fma(x, Id, xl * Id) + E) * T(1.0 / k);
        });
        if (x < T(1)) I[0] = Id;
      }
    }
    const T c1 = b1 + l1, c2 = b2 + l2;
    T zr = c1, zi = -c2;            // zbar^n (table form)
    T qr = E * c1, qi = -E * c2;    // E zbar^n (recursion)
    T wr = c1 * ((T(1) - E) * rx);  // w_n (recursion)
    T wi = -c2 * ((T(1) - E) * rx);
    // This pair's edge columns are summed apart from the running sums and
    // added to them once the last jet order feeding them is done (order k
    // takes jet orders k .. k + M): the terms of one pair cancel strongly,
    // and every other column of the order inherits the edges' rounding
    // through the recursion.
    T pe[2 * (HI - LO + 1)];
#pragma unroll
    for (int i = 0; i < 2 * (HI - LO + 1); ++i) pe[i] = T(0);
    static_for<1, NJ + 1>([&](auto nc) {
      constexpr int n = decltype(nc)::value;
      T w_r, w_i;
      if (small) {
        if constexpr (n > 1) {  // (zr + i zi) * ((b1 + l1) - i (b2 + l2)), two-term
          const T tr = fma(zr, b1, fma(zi, b2, fma(zr, l1, zi * l2)));
          const T ti = fma(zi, b1, fma(-zr, b2, fma(zi, l1, -zr * l2)));
          zr = tr;
          zi = ti;
        }
        w_r = zr * I[n - 1];
        w_i = zi * I[n - 1];
      } else {
        if constexpr (n > 1) {  // order n from order n - 1
          const T tr = qr * b1 + qi * b2;
          const T ti = qi * b1 - qr * b2;
          qr = tr;
          qi = ti;
          const T pr = fma(wr, b1, fma(wi, b2, fma(wr, l1, wi * l2)));
          const T pi = fma(wi, b1, fma(-wr, b2, fma(wi, l1, -wr * l2)));
          wr = (T(n - 1) * pr - qr) * rx;
          wi = (T(n - 1) * pi - qi) * rx;
        }
        w_r = wr;
        w_i = wi;
      }
      if constexpr (n >= NLO) {
      const T f = T(((n - 1) & 1) ? -kInv4Pi : kInv4Pi) * wmask;
      w_r *= f;
      w_i *= f;
      T chi[n + 1];
      chi[0] = T(0);
      chi[1] = T(0);
      T pr = T(0), pi = T(0);
      static_for<2, n + 1>([&](auto ac) {
        constexpr int aa = decltype(ac)::value;
        chi[aa] = hx[aa - 2] * hy[n - aa] - chi[aa - 2];
        constexpr T wgt = T(binom_d(n, aa) * pow2_neg(n));
        constexpr int r = (n - aa) & 3;  // (-i)^r
        if constexpr (r == 0) pr += wgt * chi[aa];
        if constexpr (r == 1) pi -= wgt * chi[aa];
        if constexpr (r == 2) pr -= wgt * chi[aa];
        if constexpr (r == 3) pi += wgt * chi[aa];
      });
      const T dr = w_r - pr;
      const T di = w_i - pi;
      T c0, c1;  // 2 i^n (dr + i di)
      if constexpr ((n & 3) == 0) { c0 = T(2) * dr;  c1 = T(2) * di; }
      if constexpr ((n & 3) == 1) { c0 = T(-2) * di; c1 = T(2) * dr; }
      if constexpr ((n & 3) == 2) { c0 = T(-2) * dr; c1 = T(-2) * di; }
      if constexpr ((n & 3) == 3) { c0 = T(2) * di;  c1 = T(-2) * dr; }
      // Cartesian entries alpha = (aa, n - aa) for aa <= M + 1: the edge
      // columns beta1 = aa - m1 in {0, 1} need no others
      constexpr int AMAX = n < M + 1 ? n : M + 1;
      static_for<0, AMAX + 1>([&](auto ac) {
        constexpr int aa = decltype(ac)::value;
        constexpr T s = ((aa >> 1) & 1) ? T(-1) : T(1);
        T ca;
        if constexpr (aa < 2) ca = s * ((aa & 1) ? c1 : c0);
        else ca = s * ((aa & 1) ? c1 : c0) + chi[aa];
        static_for<0, 2>([&](auto bc) {
          constexpr int bb1 = decltype(bc)::value;
          constexpr int m1 = aa - bb1;
          if constexpr (m1 >= 0 && m1 <= M) {
            static_for<0, M - m1 + 1>([&](auto m2c) {
              constexpr int m2 = decltype(m2c)::value;
              constexpr int bb2 = n - aa - m2;
              constexpr int bn = bb1 + bb2;
              if constexpr (bb2 >= 0 && bn >= LO && bn <= HI) {
                constexpr int e = 2 * (bn - LO) + bb1;
                pe[e] = fma(a[mcol(m1, m2)], ca, pe[e]);
              }
            });
          }
        });
      });
      constexpr int kd = n - M;  // edge order completed by this jet order
      if constexpr (kd >= LO && kd <= HI) {
        acc[bcol(0, kd) - B0] += pe[2 * (kd - LO)];
        acc[bcol(1, kd - 1) - B0] += pe[2 * (kd - LO) + 1];
      }
      }  // n >= NLO
    });
    }  // PART != 2
    // Laplacian columns (beta1 >= 2): R[beta] = sum_m a_m e_(m + beta - 2 e1),
    // taken one gamma2 = beta2 at a time as sum_m1 hx[m1 + gamma1] T[m1] with
    // T[m1] = sum_m2 a_(m1, m2) hy[m2 + gamma2] (the Gaussian jet is separable).
    if constexpr (GHI >= 0 && PART != 1) {
      static_for<0, GHI + 1>([&](auto g2c) {
        constexpr int g2 = decltype(g2c)::value;
        T tq[M + 1];
        static_for<0, M + 1>([&](auto m1c) {
          constexpr int m1 = decltype(m1c)::value;
          T sacc = T(0);
          static_for<0, M - m1 + 1>([&](auto m2c) {
            constexpr int m2 = decltype(m2c)::value;
            sacc = fma(a[mcol(m1, m2)], hy[m2 + g2], sacc);
          });
          tq[m1] = sacc;
        });
        static_for<(GLO > g2 ? GLO - g2 : 0), GHI - g2 + 1>([&](auto g1c) {
          constexpr int g1 = decltype(g1c)::value;
          constexpr int col = bcol(g1 + 2, g2) - B0;
          T sacc = T(0);
          static_for<0, M + 1>([&](auto m1c) {
            constexpr int m1 = decltype(m1c)::value;
            sacc = fma(hx[m1 + g1], tq[m1], sacc);
          });
          acc[col] += sacc;  // one rounding against the running sum per pair
        });
      });
    }
  }
};

// Far-field pair (x >= x_far(M) for every pair of the tile): the Gaussian part
// of the jet is below FP32 rounding, psi is the point-vortex stream function
// (1/4pi) ln|b|^2, and with u = 1/z its Cartesian jet is
//   D_1^a D_2^{n-a} psi = Re((-i)^a omega_n),  omega_n = -(-i)^n (n-1)! u^n / (2 pi),
// so the correlation collapses onto the source's complex multipoles
//   A'_n = sum_{|m| = n} a_m (-i)^{m1 + n}                (written by prep)
//   Y[nb] = sum_{n'=0}^{M} A'_{n'} rho_{n'+nb},  rho_n = (n-1)! u^n,
//   Psi[beta] += -Re((-i)^{beta1 + |beta|} Y[|beta|]) / (2 pi).
// Y is accumulated per target; fold_far adds it into the Psi slice.
// Only the multipole orders LO <= nb <= HI of the slice are formed (Y[nb - LO]).
// The sums above for NA multipole terms: Y[nb] += sum_{n < NA} A_n rho_{n+nb}(b)
// for LO <= nb <= HI, u = 1/b with b = (b1 + i b2) + (l1 + i l2) (hi and lo
// parts; u to first order in the lo part).  A single source passes its A'_n
// (NA = M + 1); a whole far tile passes its expansion B_j about the tile
// centre (NA = m2p_terms(M), see common.cuh).
template <int NA, typename T, int LO, int HI>
struct FarSums {
  static constexpr int NQ = HI + NA - 1;  // highest rho order
  static constexpr int NY = HI - LO + 1;

  __device__ __forceinline__ static void run(T b1, T b2, T l1, T l2, const T* af, T (&yr)[NY],
                                             T (&yi)[NY]) {
    const T inv = T(1) / (b1 * b1 + b2 * b2);
    T ur = b1 * inv, ui = -b2 * inv;  // 1 / z_hi
    // u = 1/(z_hi + l) = uh (1 - l uh) to first order in the low part l = l1 + i l2
    const T tr = l1 * ur - l2 * ui, ti = l1 * ui + l2 * ur;
    const T nr = ur - (ur * tr - ui * ti), ni = ui - (ur * ti + ui * tr);
    ur = nr;
    ui = ni;
    T ar[NA], ai[NA];
#pragma unroll
    for (int n = 0; n < NA; ++n) {
      ar[n] = af[2 * n];
      ai[n] = af[2 * n + 1];
    }
    // rho_q = (q-1)! u^q, one order at a time; Y[nb] += A_{q-nb} rho_q
    T rr = ur, ri = ui;
    static_for<1, NQ + 1>([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      if constexpr (q > 1) {
        const T pr = ur * rr - ui * ri;
        const T pi = ur * ri + ui * rr;
        rr = T(q - 1) * pr;
        ri = T(q - 1) * pi;
      }
      static_for<0, NA>([&](auto nc) {
        constexpr int n = decltype(nc)::value;
        constexpr int nb = q - n;
        if constexpr (nb >= LO && nb <= HI) {
          yr[nb - LO] = fma(ar[n], rr, fma(-ai[n], ri, yr[nb - LO]));
          yi[nb - LO] = fma(ar[n], ri, fma(ai[n], rr, yi[nb - LO]));
        }
      });
    });
  }
};

template <int M, typename T, int LO, int HI>
struct PairFar : FarSums<M + 1, T, LO, HI> {};

// Psi[beta] += -Re((-i)^{beta1+|beta|} Y[|beta|]) / (2 pi) over the edge
// columns beta1 in {0, 1} of the slice (acc indexed from column B0).  The
// point-vortex stream function is harmonic, so its Laplacian columns
// (beta1 >= 2) get nothing: the finish recovers them by the recursion.
template <int M, typename T, int LO, int HI>
__device__ __forceinline__ void fold_far(const T (&yr)[HI - LO + 1], const T (&yi)[HI - LO + 1],
                                         T* acc) {
  using PN = PairNear<M, T, LO, HI>;
  constexpr T s = T(1.0 / (2.0 * 3.14159265358979323846));
  static_for<LO, HI + 1>([&](auto nbc) {
    constexpr int nb = decltype(nbc)::value;
    static_for<0, 2>([&](auto b1c) {
      constexpr int bb1 = decltype(b1c)::value;
      if constexpr (bb1 <= nb) {
        constexpr int bb2 = nb - bb1;
        constexpr int col = bcol(bb1, bb2) - PN::B0;
        constexpr int r = (bb1 + nb) & 3;
        if constexpr (r == 0) acc[col] -= s * yr[nb - LO];
        if constexpr (r == 1) acc[col] -= s * yi[nb - LO];
        if constexpr (r == 2) acc[col] += s * yr[nb - LO];
        if constexpr (r == 3) acc[col] += s * yi[nb - LO];
      }
    });
  });
}

}  // namespace mmvm
