// Per-particle kernels of the MMVM right-hand side (FP64):
//  * prep:   core spreading lambda(t)^2 = lambda_0^2 + 4 nu t (eq:phi00) at the
//            stage time, c = 2 lambda^2, and the source records
//            (zeta = x / sqrt(c), a_m = M_m c^{-|m|/2}) for the pair kernel;
//  * finish: sum of the pair partials over source chunks, the Laplacian
//            recursion that turns them into the correlation Psi, the self pair from
//            the jet at the origin, the centroid velocity (eq:xjdot_Final, self
//            pair excluded), the moment equation (eq:Final_CrossCoef with the
//            (i,q) sums of eq:FinalSingleI/II folded into tables) including the
//            transport term C (eq:last_termsimp), and optionally the classic
//            RK4 stage combination;
//  * advance_time: t += dt after the fourth stage.
#include "particle_kernels.h"

#include <algorithm>

#include "common.cuh"

namespace mmvm {

__device__ __forceinline__ double stage_c(const double* t_dev, const double* dt_dev,
                                          double cs, double lam0sq, double four_nu) {
  const double t = *t_dev + cs * (dt_dev ? *dt_dev : 0.0);
  return 2.0 * (lam0sq + four_nu * t);
}

// The source record of one particle (centre xj, moments mj): zeta = x / sqrt(c)
// (FP32: exact (hi, lo) pair), a_m = M_m c^{-|m|/2} and, for FP32 records,
// the far-field multipoles A'_n = sum_{|m|=n} a_m (-i)^{m1+n}.
template <typename T>
__device__ __forceinline__ void make_record(T* __restrict__ r, const double* __restrict__ xj,
                                            const double* __restrict__ mj, int M, int K, int R,
                                            double irc) {
  const double z1 = xj[0] * irc;
  const double z2 = xj[1] * irc;
  int h;
  if constexpr (sizeof(T) == 4) {
    const float h1 = (float)z1, h2 = (float)z2;
    r[0] = h1;
    r[1] = h2;
    r[2] = (float)(z1 - (double)h1);
    r[3] = (float)(z2 - (double)h2);
    h = 4;
  } else {
    r[0] = (T)z1;
    r[1] = (T)z2;
    h = 2;
  }
  double sc = 1.0;
  int col = 0;
  for (int s = 0; s <= M; ++s) {
    double fr = 0.0, fi = 0.0;  // A'_s
    for (int k2 = 0; k2 <= s; ++k2, ++col) {
      const double a = mj[col] * sc;
      r[h + col] = (T)a;
      switch ((s - k2 + s) & 3) {  // (-i)^{m1 + s}, m1 = s - k2
        case 0: fr += a; break;
        case 1: fi -= a; break;
        case 2: fr -= a; break;
        default: fi += a; break;
      }
    }
    if constexpr (sizeof(T) == 4) {
      r[h + K + 2 * s] = (T)fr;
      r[h + K + 2 * s + 1] = (T)fi;
    }
    sc *= irc;
  }
  for (int q = h + K + rec_far<T>(M); q < R; ++q) r[q] = T(0);
}

// Sorted position p holds particle perm[p] (perm == null: identity).  Every
// warp (kGroup consecutive positions) writes the bounding box of its hi-part
// centres at the head of its group record in gdata (if given; records of GL
// floats, see gdata_len).
template <typename T>
__global__ void prep_kernel(int n, int M, int K, int R, const int* __restrict__ perm,
                            const double* __restrict__ x, const double* __restrict__ mom,
                            const double* t_dev, const double* dt_dev, double cs, double lam0sq,
                            double four_nu, T* __restrict__ rec, float* __restrict__ gdata,
                            int GL) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = p < n;
  float lo1 = 3.4e38f, hi1 = -3.4e38f, lo2 = 3.4e38f, hi2 = -3.4e38f;
  if (valid) {
    const int j = perm ? perm[p] : p;
    const double c = stage_c(t_dev, dt_dev, cs, lam0sq, four_nu);
    T* r = rec + (size_t)p * R;
    make_record<T>(r, x + 2 * j, mom + (size_t)j * K, M, K, R, 1.0 / sqrt(c));
    if constexpr (sizeof(T) == 4) {
      lo1 = hi1 = r[0];
      lo2 = hi2 = r[1];
    }
  }
  if (gdata) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo1 = fminf(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
      hi1 = fmaxf(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
      lo2 = fminf(lo2, __shfl_xor_sync(0xffffffffu, lo2, o));
      hi2 = fmaxf(hi2, __shfl_xor_sync(0xffffffffu, hi2, o));
    }
    if ((threadIdx.x & 31) == 0 && valid)
      *reinterpret_cast<float4*>(gdata + (size_t)(p / kGroup) * GL) =
          make_float4(lo1, hi1, lo2, hi2);
  }
}

// Expansion of every group of kGroup FP32 records about its centre (the
// centre of its hi-part box; see m2p_order in common.cuh): one warp per group,
// lane s adds its A'_n delta_s^k / k! into B_{n+k}, then a warp sum; the
// radius is the largest |delta_s|.  Slots past n (or, in a batch, past their
// instance's n) do not count.
template <int M>
__global__ void group_multipole_kernel(int n, const float* __restrict__ rec,
                                       float* __restrict__ gdata,
                                       const BatchInst* __restrict__ inst,
                                       const int* __restrict__ slot_inst,
                                       const int* __restrict__ n_slots) {
  constexpr int K = n_moments(M), R = rec_len<float>(M), P = m2p_order(M);
  constexpr int NA = m2p_terms(M), GL = gdata_len(M), H = Rec<float>::HDR;
  const int total = n_slots ? *n_slots : n;
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g * kGroup < total; g += nwarps) {
    const int p = g * kGroup + lane;
    bool valid = p < total;
    if (valid && inst) {
      const BatchInst& I = inst[slot_inst[g]];
      valid = p - I.slot0 < I.n;
    }
    float* gd = gdata + (size_t)g * GL;
    const float4 box = *reinterpret_cast<const float4*>(gd);
    const float cx = 0.5f * (box.x + box.y), cy = 0.5f * (box.z + box.w);
    float dr = 0.f, di = 0.f, ar[M + 1], ai[M + 1];
#pragma unroll
    for (int q = 0; q <= M; ++q) {
      ar[q] = 0.f;
      ai[q] = 0.f;
    }
    if (valid) {
      const float* r = rec + (size_t)p * R;
      dr = (r[0] - cx) + r[2];
      di = (r[1] - cy) + r[3];
#pragma unroll
      for (int q = 0; q <= M; ++q) {
        ar[q] = r[H + K + 2 * q];
        ai[q] = r[H + K + 2 * q + 1];
      }
    }
    float br[NA], bi[NA];
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      br[j] = 0.f;
      bi[j] = 0.f;
    }
    float er = 1.f, ei = 0.f;  // delta^k / k!
    static_for<0, P + 1>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      if constexpr (k > 0) {
        const float tr = (er * dr - ei * di) * (1.f / k);
        ei = (er * di + ei * dr) * (1.f / k);
        er = tr;
      }
      static_for<0, M + 1>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        br[q + k] = fmaf(ar[q], er, fmaf(-ai[q], ei, br[q + k]));
        bi[q + k] = fmaf(ar[q], ei, fmaf(ai[q], er, bi[q + k]));
      });
    });
    float rad2 = dr * dr + di * di;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rad2 = fmaxf(rad2, __shfl_xor_sync(0xffffffffu, rad2, o));
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        br[j] += __shfl_xor_sync(0xffffffffu, br[j], o);
        bi[j] += __shfl_xor_sync(0xffffffffu, bi[j], o);
      }
    }
    if (lane == 0) {
      *reinterpret_cast<float4*>(gd + 4) = make_float4(cx, cy, sqrtf(rad2), 0.f);
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        gd[8 + 2 * j] = br[j];
        gd[9 + 2 * j] = bi[j];
      }
    }
  }
}

// Shared-memory layout per block: for each of TB targets, Psi[NB], a[K], X[2],
// M_00 (read before any in-place stage write), then the powers c^{-s/2}.
// The block handles sorted positions j0 .. j0 + TB - 1 (those below A.n); all
// its threads call this, and it ends with the block's last writes to shared
// memory behind no barrier (a caller that loops must add one).
__device__ __forceinline__ void finish_block(const FinishArgs& A, int j0, double* sm) {
  const int TB = A.targets_per_block;
  const int NB = A.NB, K = A.K, M = A.M;
  double* psi = sm;                       // TB * NB
  double* at = psi + TB * NB;             // TB * K
  double* X = at + TB * K;                // TB * 2
  double* m00s = X + TB * 2;              // TB
  double* cpow = m00s + TB;               // c^{-s/2}, s = 0..2M+2
  const double c = stage_c(A.t_dev, A.dt_dev, A.cs, A.lam0sq, A.four_nu);
  for (int s = threadIdx.x; s <= 2 * M + 2; s += blockDim.x) cpow[s] = pow(c, -0.5 * s);
  __syncthreads();
  // 1. Psi_excl = sum over source chunks (fixed order), scaled moments
  for (int idx = threadIdx.x; idx < TB * NB; idx += blockDim.x) {
    const int tt = idx / NB, b = idx % NB, j = j0 + tt;
    double v = 0.0;
    if (j < A.n && A.partial) {
      for (int ch = 0; ch < A.nchunks; ++ch) v += A.partial[((size_t)ch * NB + b) * A.n + j];
      if (A.fpart) {  // far field of the list form: edge columns only
        int bn = 1;
        while (tri(bn + 1) - 1 <= b) ++bn;
        const int b1 = bn - (b + 1 - tri(bn));
        if (b1 <= 1) {
          const int e = 2 * (bn - 1) + b1;
          for (int ch = 0; ch < A.nfar; ++ch) v += A.fpart[((size_t)ch * A.n_edge + e) * A.n + j];
        }
      }
    }
    psi[idx] = v;
  }
  __syncthreads();
  // 1b. the pair kernels leave Psi itself only in the edge columns beta1 <= 1;
  //     a column beta1 >= 2 holds R[beta] = sum_m a_m D^{m + beta - 2 e1} Lap psi.
  //     D_1^2 = Lap - D_2^2 gives Psi[beta] = R[beta] - Psi[beta - 2 e1 + 2 e2],
  //     taken per order in increasing beta1.
  const int BM = bmax_of(M);
  for (int idx = threadIdx.x; idx < TB * BM; idx += blockDim.x) {
    const int tt = idx / BM, k = idx % BM + 1;
    double* ps = psi + tt * NB;
    for (int b1 = 2; b1 <= k; ++b1) ps[bcol(b1, k - b1)] -= ps[bcol(b1 - 2, k - b1 + 2)];
  }
  for (int idx = threadIdx.x; idx < TB * K; idx += blockDim.x) {
    const int tt = idx / K, m = idx % K, p = j0 + tt;
    int s = 0;
    while ((s + 1) * (s + 2) / 2 <= m) ++s;  // total order of column m
    const int j = p < A.n ? (A.perm ? A.perm[p] : p) : 0;
    const double mv = (p < A.n) ? A.Min[(size_t)j * K + m] : 0.0;
    at[idx] = mv * cpow[s];
    if (m == 0) m00s[tt] = (p < A.n) ? mv : 1.0;
  }
  __syncthreads();
  // 2. centroid sums X_c = sum_m (-1)^{|m|} a_m What_c[m], What_1[m] = -Psi[m+e2],
  //    What_2[m] = Psi[m+e1]  (eq:xjdot_Final in c = 1 units, self pair excluded)
  for (int idx = threadIdx.x; idx < TB * 2; idx += blockDim.x) {
    const int tt = idx >> 1, comp = idx & 1;
    double acc = 0.0;
    int col = 0;
    for (int s = 0; s <= M; ++s) {
      const double sg = (s & 1) ? -1.0 : 1.0;
      for (int m2 = 0; m2 <= s; ++m2, ++col) {
        const int m1 = s - m2;
        const double a = at[tt * K + col];
        if (comp == 0) acc -= sg * a * psi[tt * NB + bcol(m1, m2 + 1)];
        else acc += sg * a * psi[tt * NB + bcol(m1 + 1, m2)];
      }
    }
    X[idx] = acc;
  }
  __syncthreads();
  // 3. add the self pair: Psi_self[beta] = sum_m a_m psi0[m + beta]
  for (int idx = threadIdx.x; idx < TB * NB; idx += blockDim.x) {
    const int tt = idx / NB, b = idx % NB;
    int bn = 1;
    while (tri(bn + 1) - 1 <= b) ++bn;
    const int b2 = b + 1 - tri(bn), b1 = bn - b2;
    double acc = 0.0;
    int col = 0;
    for (int s = 0; s <= M; ++s) {
      for (int m2 = 0; m2 <= s; ++m2, ++col) {
        const int a1 = s - m2 + b1, a2 = m2 + b2;
        if ((a1 | a2) & 1) continue;  // psi0 vanishes at odd indices
        acc += at[tt * K + col] * A.psi0[tri(a1 + a2) + a2];
      }
    }
    psi[idx] += acc;
  }
  __syncthreads();
  // 4. moment equation and centroid velocity per (target, k)
  for (int idx = threadIdx.x; idx < TB * K; idx += blockDim.x) {
    const int tt = idx / K, k = idx % K, p = j0 + tt;
    if (p >= A.n) continue;
    const int j = A.perm ? A.perm[p] : p;
    int kn = 0;
    while ((kn + 1) * (kn + 2) / 2 <= k) ++kn;
    const int k2 = k - tri(kn), k1 = kn - k2;
    const double* a = at + tt * K;
    const double* ps = psi + tt * NB;
    double R = 0.0;
    for (int e = A.k_off[k]; e < A.k_off[k + 1]; ++e) R += A.e_c[e] * a[A.e_l[e]] * ps[A.e_b[e]];
    const double m00 = m00s[tt];
    double ctr = 0.0;
    if (k1 >= 1) ctr += X[2 * tt] * a[mcol(k1 - 1, k2)];
    if (k2 >= 1) ctr += X[2 * tt + 1] * a[mcol(k1, k2 - 1)];
    const double dm = (R + ctr / m00) / (cpow[kn] * c);  // c^{|k|/2 - 1}
    const size_t o = (size_t)j * K + k;
    if (A.mode == 0) {
      A.out_dM[o] = dm;
    } else {
      const double h = *A.dt_dev;
      const double base = A.y_M[o];
      if (A.mode == 1) { A.ys_M[o] = base + 0.5 * h * dm; A.sum_M[o] = base + h / 6.0 * dm; }
      if (A.mode == 2) { A.ys_M[o] = base + 0.5 * h * dm; A.sum_M[o] += h / 3.0 * dm; }
      if (A.mode == 3) { A.ys_M[o] = base + h * dm;       A.sum_M[o] += h / 3.0 * dm; }
      if (A.mode == 4) { A.y_M[o] = A.sum_M[o] + h / 6.0 * dm; }
    }
  }
  // 5. centroid velocity xdot_c = c^{-1/2} X_c / M_00 and its stage update
  for (int idx = threadIdx.x; idx < TB * 2; idx += blockDim.x) {
    const int tt = idx >> 1, comp = idx & 1, p = j0 + tt;
    if (p >= A.n) continue;
    const int j = A.perm ? A.perm[p] : p;
    const double dx = X[idx] * cpow[1] / m00s[tt];
    const size_t ox = (size_t)j * 2 + comp;
    if (A.mode == 0) {
      A.out_dx[ox] = dx;
    } else {
      const double h = *A.dt_dev;
      const double base = A.y_x[ox];
      if (A.mode == 1) { A.ys_x[ox] = base + 0.5 * h * dx; A.sum_x[ox] = base + h / 6.0 * dx; }
      if (A.mode == 2) { A.ys_x[ox] = base + 0.5 * h * dx; A.sum_x[ox] += h / 3.0 * dx; }
      if (A.mode == 3) { A.ys_x[ox] = base + h * dx;       A.sum_x[ox] += h / 3.0 * dx; }
      if (A.mode == 4) { A.y_x[ox] = A.sum_x[ox] + h / 6.0 * dx; }
    }
  }
}

__global__ void finish_kernel(FinishArgs A) {
  extern __shared__ double sm[];
  finish_block(A, blockIdx.x * A.targets_per_block, sm);  // sorted positions
}

__global__ void advance_time_kernel(double* t_dev, const double* dt_dev) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *t_dev += *dt_dev;
}

// Non-finite / zero-circulation scan of a state (flags[0]: non-finite,
// flags[1]: zero circulation); used after set_state and on demand.
__global__ void scan_state_kernel(int n, int K, const double* __restrict__ x,
                                  const double* __restrict__ mom, int* flags) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  bool bad = !isfinite(x[2 * j]) || !isfinite(x[2 * j + 1]);
  for (int m = 0; m < K; ++m) bad |= !isfinite(mom[(size_t)j * K + m]);
  if (bad) atomicOr(flags, 1);
  if (mom[(size_t)j * K] == 0.0) atomicOr(flags + 1, 1);
}

// ------------------------------------------------------------------ batches
// Offsets of the state blocks of one instance (see BatchInst).
__device__ __forceinline__ const double* inst_stage_x(const BatchInst& I, int K, int src) {
  return I.state + (src ? (size_t)I.n * (2 + K) : 0);
}
__device__ __forceinline__ const double* inst_stage_m(const BatchInst& I, int K, int src) {
  return inst_stage_x(I, K, src) + 2 * (size_t)I.n;
}

// Records of every instance of a batch of one order: slot p belongs to
// instance slot_inst[p / kGroup]; padding slots past an instance's n are not
// written (no kernel reads them).  src = 0 reads the step-start state y,
// src = 1 the stage state ys; the core is taken at t + cs dt of each instance.
// With perm_local, sorted slot p holds local particle perm_local[p]; with
// gdata, every warp (one group of kGroup slots: the loop keeps warps aligned
// to groups and n_slots is a multiple of kGroup) writes its group's box at
// the head of the group's record (GL floats).
template <typename T>
__global__ void prep_batch_kernel(int M, int K, int R, const BatchInst* __restrict__ inst,
                                  const int* __restrict__ slot_inst,
                                  const int* __restrict__ n_slots, int src, double cs,
                                  const int* __restrict__ perm_local, T* __restrict__ rec,
                                  float* __restrict__ gdata, int GL) {
  const int total = *n_slots;
  for (int base = blockIdx.x * blockDim.x; base < total; base += gridDim.x * blockDim.x) {
    const int p = base + threadIdx.x;  // whole warps are in or out of range
    if (p >= total) continue;
    const BatchInst& I = inst[slot_inst[p / kGroup]];
    const int j = p - I.slot0;
    float lo1 = 3.4e38f, hi1 = -3.4e38f, lo2 = 3.4e38f, hi2 = -3.4e38f;
    if (j < I.n) {
      const int jj = perm_local ? perm_local[p] : j;
      const double c = 2.0 * (I.lam0sq + I.four_nu * (I.t + cs * I.dt));
      T* r = rec + (size_t)p * R;
      make_record<T>(r, inst_stage_x(I, K, src) + 2 * jj, inst_stage_m(I, K, src) + (size_t)jj * K,
                     M, K, R, 1.0 / sqrt(c));
      if constexpr (sizeof(T) == 4) {
        lo1 = hi1 = r[0];
        lo2 = hi2 = r[1];
      }
    }
    if (gdata) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo1 = fminf(lo1, __shfl_xor_sync(0xffffffffu, lo1, o));
        hi1 = fmaxf(hi1, __shfl_xor_sync(0xffffffffu, hi1, o));
        lo2 = fminf(lo2, __shfl_xor_sync(0xffffffffu, lo2, o));
        hi2 = fmaxf(hi2, __shfl_xor_sync(0xffffffffu, hi2, o));
      }
      if ((threadIdx.x & 31) == 0)
        *reinterpret_cast<float4*>(gdata + (size_t)(p / kGroup) * GL) =
            make_float4(lo1, hi1, lo2, hi2);
    }
  }
}

// Finish of every instance of a batch: item (instance, first target) per
// block of TB targets; blocks loop over the items.
__global__ void finish_batch_kernel(BatchFinishArgs B) {
  extern __shared__ double sm[];
  const int total = *B.n_items;
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int2 w = B.items[it];
    const BatchInst& I = B.inst[w.x];
    const size_t blk = (size_t)I.n * (2 + B.K);
    FinishArgs A;
    A.n = I.n;
    A.M = B.M;
    A.K = B.K;
    A.NB = B.NB;
    A.nchunks = I.n > 1 ? I.chunks : 0;
    A.targets_per_block = B.targets_per_block;
    A.partial = I.n > 1 ? B.partial + I.part_off : nullptr;
    A.perm = B.perm_local ? B.perm_local + I.slot0 : nullptr;
    A.Min = inst_stage_m(I, B.K, B.src);
    A.k_off = B.k_off;
    A.e_l = B.e_l;
    A.e_b = B.e_b;
    A.e_c = B.e_c;
    A.psi0 = B.psi0;
    A.lam0sq = I.lam0sq;
    A.four_nu = I.four_nu;
    A.t_dev = &I.t;
    A.dt_dev = &I.dt;
    A.cs = B.cs;
    A.mode = B.mode;
    A.y_x = I.state;
    A.y_M = I.state + 2 * (size_t)I.n;
    A.ys_x = I.state + blk;
    A.ys_M = I.state + blk + 2 * (size_t)I.n;
    A.sum_x = I.state + 2 * blk;
    A.sum_M = I.state + 2 * blk + 2 * (size_t)I.n;
    finish_block(A, w.y, sm);
    __syncthreads();  // shared memory is reused by the next item
  }
}

__global__ void advance_batch_kernel(BatchInst* __restrict__ inst, const int* __restrict__ n_inst) {
  const int total = *n_inst;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
    inst[i].t += inst[i].dt;
}

// flags[i] = 1 if the step-start state of instance i holds a non-finite value,
// else 0; one block per instance (blocks loop over the instances).
__global__ void scan_batch_kernel(int K, const BatchInst* __restrict__ inst,
                                  const int* __restrict__ n_inst, int* __restrict__ flags) {
  const int total = *n_inst;
  for (int i = blockIdx.x; i < total; i += gridDim.x) {
    const BatchInst& I = inst[i];
    const size_t len = (size_t)I.n * (2 + K);
    bool bad = false;
    for (size_t q = threadIdx.x; q < len; q += blockDim.x) bad |= !isfinite(I.state[q]);
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) flags[i] = bad ? 1 : 0;
  }
}

cudaError_t launch_scan_batch(int M, const BatchInst* inst, const int* n_inst, int max_inst,
                              int* flags, cudaStream_t st) {
  scan_batch_kernel<<<std::max(1, std::min(max_inst, 1024)), 256, 0, st>>>(n_moments(M), inst,
                                                                          n_inst, flags);
  return cudaGetLastError();
}

cudaError_t launch_prep_batch(int precision, int M, const BatchInst* inst, const int* slot_inst,
                              const int* n_slots, int max_slots, int src, double cs,
                              const int* perm_local, void* rec, void* gbox, cudaStream_t st) {
  const int K = n_moments(M);
  const int threads = 128, blocks = std::max(1, std::min((max_slots + threads - 1) / threads, 4096));
  if (precision == 1) {
    prep_batch_kernel<float><<<blocks, threads, 0, st>>>(M, K, rec_len<float>(M), inst, slot_inst,
                                                         n_slots, src, cs, perm_local,
                                                         (float*)rec, (float*)gbox,
                                                         gdata_len(M));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !gbox) return e;
    return launch_group_multipole(M, 0, rec, gbox, inst, slot_inst, n_slots, max_slots, st);
  }
  prep_batch_kernel<double><<<blocks, threads, 0, st>>>(M, K, rec_len<double>(M), inst, slot_inst,
                                                        n_slots, src, cs, perm_local,
                                                        (double*)rec, nullptr, 0);
  return cudaGetLastError();
}

size_t finish_smem_bytes(int M, int targets_per_block) {
  const int K = n_moments(M), NB = n_beta(M);
  return sizeof(double) * ((size_t)targets_per_block * (NB + K + 3) + 2 * M + 3);
}

cudaError_t launch_finish_batch(const BatchFinishArgs& B, int grid, cudaStream_t st) {
  const size_t smem = finish_smem_bytes(B.M, B.targets_per_block);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(finish_batch_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  finish_batch_kernel<<<std::max(1, grid), 128, smem, st>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_advance_batch(BatchInst* inst, const int* n_inst, int max_inst,
                                 cudaStream_t st) {
  advance_batch_kernel<<<std::max(1, (max_inst + 127) / 128), 128, 0, st>>>(inst, n_inst);
  return cudaGetLastError();
}

cudaError_t launch_group_multipole(int M, int n, const void* rec, void* gdata,
                                   const BatchInst* inst, const int* slot_inst,
                                   const int* n_slots, int max_slots, cudaStream_t st) {
  const int groups = (max_slots + kGroup - 1) / kGroup;
  const int threads = 128, blocks = std::max(1, std::min((groups * 32 + threads - 1) / threads, 4096));
  const float* r = static_cast<const float*>(rec);
  float* g = static_cast<float*>(gdata);
  switch (M) {
#define MMVM_GM_CASE(m)                                                                  \
  case m:                                                                                \
    group_multipole_kernel<m><<<blocks, threads, 0, st>>>(n, r, g, inst, slot_inst, n_slots); \
    break;
    MMVM_GM_CASE(0) MMVM_GM_CASE(1) MMVM_GM_CASE(2) MMVM_GM_CASE(3) MMVM_GM_CASE(4)
    MMVM_GM_CASE(5) MMVM_GM_CASE(6) MMVM_GM_CASE(7) MMVM_GM_CASE(8)
#undef MMVM_GM_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_prep(int precision, int n, int M, const int* perm, const double* x,
                        const double* mom, const double* t_dev, const double* dt_dev, double cs,
                        double lam0sq, double four_nu, void* rec, void* gbox, cudaStream_t st) {
  const int K = n_moments(M);
  const int threads = 128, blocks = (n + threads - 1) / threads;
  if (precision == 1) {
    prep_kernel<float><<<blocks, threads, 0, st>>>(n, M, K, rec_len<float>(M), perm, x, mom,
                                                   t_dev, dt_dev, cs, lam0sq, four_nu,
                                                   (float*)rec, (float*)gbox, gdata_len(M));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !gbox) return e;
    return launch_group_multipole(M, n, rec, gbox, nullptr, nullptr, nullptr, n, st);
  }
  prep_kernel<double><<<blocks, threads, 0, st>>>(n, M, K, rec_len<double>(M), perm, x, mom,
                                                  t_dev, dt_dev, cs, lam0sq, four_nu,
                                                  (double*)rec, nullptr, 0);
  return cudaGetLastError();
}

cudaError_t launch_finish(const FinishArgs& A, cudaStream_t st) {
  const int TB = A.targets_per_block;
  const size_t smem = sizeof(double) * ((size_t)TB * (A.NB + A.K + 3) + 2 * A.M + 3);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(finish_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int blocks = (A.n + TB - 1) / TB;
  finish_kernel<<<blocks, 128, smem, st>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_advance_time(double* t_dev, const double* dt_dev, cudaStream_t st) {
  advance_time_kernel<<<1, 32, 0, st>>>(t_dev, dt_dev);
  return cudaGetLastError();
}

cudaError_t launch_scan(int n, int K, const double* x, const double* mom, int* flags,
                        cudaStream_t st) {
  scan_state_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, K, x, mom, flags);
  return cudaGetLastError();
}

}  // namespace mmvm
