// Single particle at high order: the self term of the moment equation
// (eq:moment_evolutionFinish, the (i,q) double sums of eq:FinalSingleI/II)
// without a table of (k, l, i, q) terms, whose size grows like M^6 (about
// 1e9 terms at M = 60).
//
// In units c = 2 lambda^2 = 1 (a_m = M_m c^{-|m|/2}) the equation reads
//   dM_k/dt = c^{|k|/2-1} R_k,
//   R_k = sum_l a_l sum_{i,q} coef(k,l,i,q) Psi[beta(k,l,i,q)],
//   Psi[beta] = sum_m a_m psi0[m + beta]           (the jet of the self pair),
// and with g(j) = 4^{-j} / j! every coefficient factors into an x part and a
// y part (4^{i+q+1-|k|} / ((k1-1-i)! (k2-q)!) = g(k1-1-i) g(k2-q), and the
// same with the Gamma^II factorials):
//   Gamma^I : -(-1)^{|k|} X1(k1,l1,i) Y1(k2,l2,q),
//             X1 = (-1)^{l1} C(l1,i) g(k1-1-i),  Y1 = (-1)^{l2} C(l2,q) g(k2-q),
//             beta = (k1+l1-2i-1, k2+l2-2q+1)
//   Gamma^II: +(-1)^{|k|} X2(k1,l1,i) Y2(k2,l2,q),
//             X2 = (-1)^{l1} C(l1,i) g(k1-i),    Y2 = (-1)^{l2} C(l2,q) g(k2-1-q),
//             beta = (k1+l1-2i+1, k2+l2-2q-1)
// with beta1 depending only on (k1, l1, i) and beta2 only on (k2, l2, q).
// So the sums are taken one index at a time:
//   pass 1  U[k2, l2, b1] = sum_q  C(l2,q) g(k2(-1)-q) Psi[b1, beta2(k2,l2,q)]
//   pass 2  V[k2, l1, b1] = sum_l2 (-1)^{l2} a_{l1,l2} U[k2, l2, b1]     (l1 + l2 <= M)
//   pass 3  R_k = (-1)^{|k|} sum_l1 (-1)^{l1} sum_i C(l1,i) g(k1(-1)-i)
//                 (-V^I[k2, l1, beta1] + V^II[k2, l1, beta1])
// for about 4.6e7 multiply-adds at M = 60 instead of about 1e9 (the products
// C g come from a host table, so each term is one multiply-add).  Every factor
// g is at most 1, so the intermediate sums stay far inside the FP64 range
// (the jet psi0 reaches ~1e190 at order 3M = 180; binomials ~1e17).  Only
// terms with |beta| <= 2M exist (|k|, |l| <= M); pass 1 skips the rest.
// A lone particle does not move (eq:xjdot_Final has no other particle), so
// dx/dt = 0.  Everything is FP64.
#include <algorithm>

#include "common.cuh"
#include "particle_kernels.h"

namespace mmvm {

namespace {

__device__ __forceinline__ double stage_c_high(const SelfHighArgs& A) {
  const double t = *A.t_dev + A.cs * (A.dt_dev ? *A.dt_dev : 0.0);
  return 2.0 * (A.lam0sq + A.four_nu * t);
}

__device__ __forceinline__ int order_of_col(int col) {  // total order of column col
  int s = 0;
  while (tri(s + 1) <= col) ++s;
  return s;
}

// a_m = M_m c^{-|m|/2}
__global__ void self_scale_kernel(SelfHighArgs A) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= A.K) return;
  const double c = stage_c_high(A);
  A.at[m] = A.Min[m] * pow(c, -0.5 * order_of_col(m));
}

// Psi[beta] = sum_m a_m psi0[m + beta] for 1 <= |beta| <= 2M (psi0 vanishes at
// odd indices, so only m of the parity of beta contribute).
__global__ void self_psi_kernel(SelfHighArgs A) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= A.NB) return;
  const int bn = order_of_col(b + 1);  // bcol(b1, b2) = tri(|beta|) + b2 - 1
  const int b2 = b + 1 - tri(bn), b1 = bn - b2;
  double acc = 0.0;
  for (int m1 = b1 & 1; m1 <= A.M; m1 += 2)
    for (int m2 = b2 & 1; m1 + m2 <= A.M; m2 += 2) {
      const int a1 = m1 + b1, a2 = m2 + b2;
      acc = fma(A.at[mcol(m1, m2)], A.psi0[tri(a1 + a2) + a2], acc);
    }
  A.Psi[b] = acc;
}

// pass 1: U1[k2][l2][b1] (Gamma^I), U2[k2][l2][b1] (Gamma^II)
__global__ void self_pass1_kernel(SelfHighArgs A) {
  const int M = A.M, W = 2 * M + 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (M + 1) * (M + 1) * W) return;
  const int b1 = idx % W, l2 = (idx / W) % (M + 1), k2 = idx / (W * (M + 1));
  // C(l2, q) g(k2 - q) and C(l2, q) g(k2 - 1 - q), q = 0, 1, ...
  const double* c1 = A.cg + ((size_t)l2 * (M + 1) + k2) * (M + 1);
  double u1 = 0.0, u2 = 0.0;
  for (int q = 0; q <= min(l2, k2); ++q) {
    const int bb2 = k2 + l2 - 2 * q + 1;
    if (b1 + bb2 <= 2 * M) u1 = fma(c1[q], A.Psi[bcol(b1, bb2)], u1);
  }
  if (k2 >= 1) {
    const double* c2 = c1 - (M + 1);
    for (int q = 0; q <= min(l2, k2 - 1); ++q) {
      const int bb2 = k2 + l2 - 2 * q - 1;
      if (b1 + bb2 <= 2 * M && b1 + bb2 >= 1) u2 = fma(c2[q], A.Psi[bcol(b1, bb2)], u2);
    }
  }
  A.U1[idx] = u1;
  A.U2[idx] = u2;
}

// pass 2: V[k2][l1][b1] = sum_{l2 <= M - l1} (-1)^{l2} a_{l1,l2} U[k2][l2][b1]
__global__ void self_pass2_kernel(SelfHighArgs A) {
  const int M = A.M, W = 2 * M + 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (M + 1) * (M + 1) * W) return;
  const int b1 = idx % W, l1 = (idx / W) % (M + 1), k2 = idx / (W * (M + 1));
  const double* u1 = A.U1 + (size_t)k2 * (M + 1) * W + b1;
  const double* u2 = A.U2 + (size_t)k2 * (M + 1) * W + b1;
  double v1 = 0.0, v2 = 0.0;
  for (int l2 = 0; l1 + l2 <= M; ++l2) {
    const double a = (l2 & 1) ? -A.at[mcol(l1, l2)] : A.at[mcol(l1, l2)];
    v1 = fma(a, u1[(size_t)l2 * W], v1);
    v2 = fma(a, u2[(size_t)l2 * W], v2);
  }
  A.V1[idx] = v1;
  A.V2[idx] = v2;
}

// pass 3 and the finish: one warp per moment row k; lanes split l1, then a
// warp sum.  R_k, dM_k = c^{|k|/2-1} R_k, the RK4 stage.
__global__ void self_pass3_kernel(SelfHighArgs A) {
  const int M = A.M, W = 2 * M + 1;
  const int lane = threadIdx.x & 31;
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (blockIdx.x == 0 && threadIdx.x < 2) {  // the centre does not move
    const int c = threadIdx.x;
    if (A.mode == 0) A.out_dx[c] = 0.0;
    if (A.mode == 1) { A.ys_x[c] = A.y_x[c]; A.sum_x[c] = A.y_x[c]; }
    if (A.mode == 2 || A.mode == 3) A.ys_x[c] = A.y_x[c];
    if (A.mode == 4) A.y_x[c] = A.sum_x[c];
  }
  if (k >= A.K) return;  // whole warps
  const int kn = order_of_col(k);
  const int k2 = k - tri(kn), k1 = kn - k2;
  const double* v1 = A.V1 + (size_t)k2 * (M + 1) * W;
  const double* v2 = A.V2 + (size_t)k2 * (M + 1) * W;
  double r = 0.0;
  for (int l1 = lane; l1 <= M; l1 += 32) {
    // C(l1, i) g(k1 - i) and C(l1, i) g(k1 - 1 - i), i = 0, 1, ...
    const double* cb = A.cg + ((size_t)l1 * (M + 1) + k1) * (M + 1);
    double s = 0.0;
    if (k1 >= 1) {
      const double* ca = cb - (M + 1);
      for (int i = 0; i <= min(l1, k1 - 1); ++i)
        s = fma(-ca[i], v1[(size_t)l1 * W + k1 + l1 - 2 * i - 1], s);
    }
    if (k2 >= 1)
      for (int i = 0; i <= min(l1, k1); ++i) {
        const int bb1 = k1 + l1 - 2 * i + 1;
        if (bb1 < W) s = fma(cb[i], v2[(size_t)l1 * W + bb1], s);
      }
    r += (l1 & 1) ? -s : s;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  if (lane != 0) return;
  if (kn & 1) r = -r;  // (-1)^{|k|}
  const double c = stage_c_high(A);
  const double dm = r * pow(c, 0.5 * kn - 1.0);
  if (A.mode == 0) {
    A.out_dM[k] = dm;
    return;
  }
  const double h = *A.dt_dev;
  const double base = A.y_M[k];
  if (A.mode == 1) { A.ys_M[k] = base + 0.5 * h * dm; A.sum_M[k] = base + h / 6.0 * dm; }
  if (A.mode == 2) { A.ys_M[k] = base + 0.5 * h * dm; A.sum_M[k] += h / 3.0 * dm; }
  if (A.mode == 3) { A.ys_M[k] = base + h * dm;       A.sum_M[k] += h / 3.0 * dm; }
  if (A.mode == 4) { A.y_M[k] = A.sum_M[k] + h / 6.0 * dm; }
}

}  // namespace

size_t self_high_scratch_doubles(int M) {
  const size_t P = (size_t)(M + 1) * (M + 1) * (2 * M + 1);
  return (size_t)n_moments(M) + (size_t)n_beta(M) + 4 * P;
}

cudaError_t launch_self_high(SelfHighArgs A, double* scratch, cudaStream_t st) {
  const int M = A.M;
  const size_t P = (size_t)(M + 1) * (M + 1) * (2 * M + 1);
  A.at = scratch;
  A.Psi = A.at + A.K;
  A.U1 = A.Psi + A.NB;
  A.U2 = A.U1 + P;
  A.V1 = A.U2 + P;
  A.V2 = A.V1 + P;
  const int T = 128;
  self_scale_kernel<<<(A.K + T - 1) / T, T, 0, st>>>(A);
  self_psi_kernel<<<(A.NB + T - 1) / T, T, 0, st>>>(A);
  self_pass1_kernel<<<(int)((P + T - 1) / T), T, 0, st>>>(A);
  self_pass2_kernel<<<(int)((P + T - 1) / T), T, 0, st>>>(A);
  self_pass3_kernel<<<(A.K * 32 + T - 1) / T, T, 0, st>>>(A);
  return cudaGetLastError();
}

}  // namespace mmvm
