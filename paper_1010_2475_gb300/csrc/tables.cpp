// Host generation of the FP64 finish tables (see tables.h for the formulas).
#include "tables.h"

#include <algorithm>
#include <map>
#include <tuple>

#include "common.cuh"

namespace mmvm {

namespace {

long double factl(int n) {
  long double r = 1.0L;
  for (int i = 2; i <= n; ++i) r *= (long double)i;
  return r;
}
long double binoml(int n, int k) {
  if (k < 0 || k > n) return 0.0L;
  long double r = 1.0L;
  for (int i = 1; i <= k; ++i) r = r * (long double)(n - k + i) / (long double)i;
  return r;
}
long double pow4l(int e) {
  long double r = 1.0L;
  if (e >= 0)
    for (int i = 0; i < e; ++i) r *= 4.0L;
  else
    for (int i = 0; i < -e; ++i) r *= 0.25L;
  return r;
}

}  // namespace

FinishTables build_finish_tables(int M, bool entries) {
  FinishTables t;
  t.M = M;
  t.K = n_moments(M);
  t.NB = n_beta(M);
  t.NJ = jet_order(M);
  t.k_off.assign(t.K + 1, 0);
  for (int kn = 0, kcol = 0; entries && kn <= M; ++kn) {
    for (int k2 = 0; k2 <= kn; ++k2, ++kcol) {
      const int k1 = kn - k2;
      std::map<std::pair<int, int>, long double> acc;  // (l col, beta col) -> coef
      for (int ln = 0; ln <= M; ++ln) {
        for (int l2 = 0; l2 <= ln; ++l2) {
          const int l1 = ln - l2;
          const int lcol = mcol(l1, l2);
          const long double sgn = ((kn + ln) & 1) ? -1.0L : 1.0L;
          if (k1 >= 1) {  // Gamma^I, eq:FinalSingleI
            for (int i = 0; i <= (l1 < k1 - 1 ? l1 : k1 - 1); ++i)
              for (int q = 0; q <= (l2 < k2 ? l2 : k2); ++q) {
                const long double v = -sgn * binoml(l1, i) * binoml(l2, q) *
                                      pow4l(i + q + 1 - kn) /
                                      (factl(k1 - i - 1) * factl(k2 - q));
                const int b1 = k1 + l1 - 2 * i - 1, b2 = k2 + l2 - 2 * q + 1;
                acc[{lcol, bcol(b1, b2)}] += v;
              }
          }
          if (k2 >= 1) {  // Gamma^II, eq:FinalSingleII
            for (int i = 0; i <= (l1 < k1 ? l1 : k1); ++i)
              for (int q = 0; q <= (l2 < k2 - 1 ? l2 : k2 - 1); ++q) {
                const long double v = sgn * binoml(l1, i) * binoml(l2, q) *
                                      pow4l(i + q + 1 - kn) /
                                      (factl(k1 - i) * factl(k2 - q - 1));
                const int b1 = k1 + l1 - 2 * i + 1, b2 = k2 + l2 - 2 * q - 1;
                acc[{lcol, bcol(b1, b2)}] += v;
              }
          }
        }
      }
      for (auto& kv : acc) {
        if (kv.second == 0.0L) continue;
        t.e_l.push_back(kv.first.first);
        t.e_b.push_back(kv.first.second);
        t.e_c.push_back((double)kv.second);
      }
      t.k_off[kcol + 1] = (int)t.e_l.size();
    }
  }
  // psi0 (jet of the Gaussian-vortex stream function at the origin, c = 1)
  t.psi0.assign(tri(t.NJ + 1), 0.0);
  const long double inv4pi = 0.0795774715459476678844418816862571810L;
  for (int n = 2; n <= t.NJ; n += 2) {
    for (int a2 = 0; a2 <= n; a2 += 2) {
      const int p = (n - a2) / 2, q = a2 / 2;
      const long double r = factl(2 * p) / factl(p) * (factl(2 * q) / factl(q));
      const long double s = ((p + q) & 1) ? -1.0L : 1.0L;
      t.psi0[tri(n) + a2] = (double)(-inv4pi * s * r / (long double)(p + q));
    }
  }
  return t;
}

SeparableTables build_separable_tables(int M) {
  SeparableTables t;
  t.binom.assign((size_t)(M + 1) * (M + 1), 0.0);
  t.g.assign((size_t)M + 1, 0.0);
  for (int a = 0; a <= M; ++a) {
    for (int b = 0; b <= a; ++b) t.binom[(size_t)a * (M + 1) + b] = (double)binoml(a, b);
    t.g[a] = (double)(pow4l(-a) / factl(a));
  }
  const size_t W = (size_t)M + 1;
  t.cg.assign(W * W * W, 0.0);
  for (int l = 0; l <= M; ++l)
    for (int k = 0; k <= M; ++k)
      for (int q = 0; q <= std::min(l, k); ++q)
        t.cg[((size_t)l * W + k) * W + q] = t.binom[(size_t)l * W + q] * t.g[k - q];
  return t;
}

}  // namespace mmvm
