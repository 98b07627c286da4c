// Shared compile-time index helpers and small device utilities of the MMVM
// kernels.  Index conventions (c = 2 lambda^2, zeta = x / sqrt(c)):
//  * moment column of (k1, k2):  mcol = q(k1+k2) + k2, q(s) = s(s+1)/2;
//  * stream-function correlation Psi[beta] for 1 <= |beta| <= BMAX, column
//    bcol = q(b1+b2) + b2 - 1 (beta = 0 is never needed);
//  * BMAX = 2M covers the velocity jet W[gamma], |gamma| <= 2M-1, that the
//    moment equations need (eq:FinalCrossI/II) and the |m| <= M entries of
//    the centroid equation (eq:xjdot_Final); for M = 0 it is 1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace mmvm {

__host__ __device__ constexpr int tri(int n) { return n * (n + 1) / 2; }
__host__ __device__ constexpr int n_moments(int M) { return tri(M + 1); }
__host__ __device__ constexpr int mcol(int k1, int k2) { return tri(k1 + k2) + k2; }
__host__ __device__ constexpr int bmax_of(int M) { return M == 0 ? 1 : 2 * M; }
__host__ __device__ constexpr int n_beta(int M) { return tri(bmax_of(M) + 1) - 1; }
__host__ __device__ constexpr int bcol(int b1, int b2) { return tri(b1 + b2) + b2 - 1; }
// Highest order of the stream-function jet a pair needs: |m + beta| <= M + BMAX.
__host__ __device__ constexpr int jet_order(int M) { return M + bmax_of(M); }

__host__ __device__ constexpr double binom_d(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}
__host__ __device__ constexpr double pow2_neg(int n) {
  double r = 1.0;
  for (int i = 0; i < n; ++i) r *= 0.5;
  return r;
}

// Source record: FP32 mode stores zeta split into (hi, lo) floats so that
// differences of nearby centres are exact; FP64 stores zeta directly.
template <typename T> struct Rec;
template <> struct Rec<float> {
  static constexpr int HDR = 4;  // zh1, zh2, zl1, zl2
};
template <> struct Rec<double> {
  static constexpr int HDR = 2;  // z1, z2
};
__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }
// FP32 records also carry the far-field moments A'_n (n = 0..M, complex).
template <typename T>
__host__ __device__ constexpr int rec_far(int M) {
  return sizeof(T) == 4 ? 2 * (M + 1) : 0;
}
template <typename T>
__host__ __device__ constexpr int rec_len(int M) {
  // pad to 16 bytes so a record (and a tile of records) can be bulk-copied
  return round_up(Rec<T>::HDR + n_moments(M) + rec_far<T>(M), 16 / (int)sizeof(T));
}

// Particles per spatial group: the source tile of the pair kernel and the
// unit of the bounding boxes used for the far-field test.
constexpr int kGroup = 32;

// One instance (an independent simulation) of a batch of one order.
//  * state: FP64 blocks y_x (n x 2), y_M (n x K), ys_x, ys_M (RK4 stage
//    state), sum_x, sum_M (RK4 running sum), one after another;
//  * records: n, starting at record slot0 of the batch (slot0 is a multiple
//    of kGroup, so every group of kGroup slots belongs to one instance);
//  * sources split into `chunks` chunks of chunk_len (a multiple of kGroup);
//    partial sums [chunk][beta][target] start part_off doubles into the
//    batch's partials;
//  * core lambda^2 = lam0sq + four_nu t; step size dt; t is advanced on the
//    device after every step.
struct BatchInst {
  double* state;
  int n;
  int slot0;
  int chunk_len;
  int chunks;
  long long part_off;
  double lam0sq;
  double four_nu;
  double t;
  double dt;
};

// Far-field threshold on x = |b|^2 (c = 1 units) per order M: beyond it the
// Gaussian part of every jet entry of order <= 3M is below 2^-25 of the
// largest entry of that order (measured against the FP64 oracle's jet over
// all directions; 6 units of margin added), so a tile pair whose bounding
// boxes are this far apart uses the point-vortex jet.
__host__ __device__ constexpr float x_far(int M) {
  return M <= 0 ? 20.f : M == 1 ? 32.f : M == 2 ? 40.f : M == 3 ? 50.f : M == 4 ? 58.f
       : M == 5 ? 66.f : M == 6 ? 74.f : M == 7 ? 80.f : 88.f;
}

// Far source tiles seen from far enough away are summed through one
// multipole expansion about the tile's centre instead of source by source.
// With u = 1/w, w = target - centre, delta_s = source - centre and
// rho_q(w) = (q-1)! u^q, the shift rho_q(w - delta) = sum_k delta^k/k!
// rho_{q+k}(w) turns the per-source sums sum_n A'_{s,n} rho_{n+nb} into
// sum_j B_j rho_{j+nb}(w), B_j = sum_s sum_{n+k=j} A'_{s,n} delta_s^k / k!.
// Truncating k at m2p_order(M) leaves sum_{k>P} C(q+k-1,k) theta^k below
// 2e-9 for every jet order q <= 3M when the tile radius is at most theta =
// 0.1 of the distance from the target group's box to the tile centre.
__host__ __device__ constexpr int m2p_order(int M) {
  return M <= 0 ? 8 : M == 1 ? 10 : M == 2 ? 12 : M == 3 ? 14 : M == 4 ? 15
       : M == 5 ? 17 : M == 6 ? 18 : M == 7 ? 19 : 21;
}
__host__ __device__ constexpr int m2p_terms(int M) { return M + m2p_order(M) + 1; }
constexpr float kM2PTheta2 = 0.01f;  // theta^2
// Per group of kGroup records (FP32 far field): (min z1, max z1, min z2,
// max z2) of the hi parts, (centre z1, centre z2, radius, 0), then
// Re/Im B_j for j < m2p_terms(M); padded to whole float4s.
__host__ __device__ constexpr int gdata_len(int M) { return round_up(8 + 2 * m2p_terms(M), 4); }

// Binary tree over G groups of kGroup sorted records (the far field of the
// list form): level L has ceil(G / 2^L) nodes, node i of level L >= 1 holds
// nodes 2i and 2i+1 of level L-1, the top level one node; the node records
// of levels 1.. are stored one level after another.
__host__ __device__ inline int tree_levels(int G) {
  int L = 0;
  while ((G + (1 << L) - 1) >> L > 1) ++L;
  return L;  // index of the top level (0 if G == 1)
}
__host__ __device__ inline int tree_level_nodes(int G, int L) { return (G + (1 << L) - 1) >> L; }
// Offset (in nodes) of level L >= 1 in the node storage.
__host__ __device__ inline long long tree_level_offset(int G, int L) {
  long long off = 0;
  for (int l = 1; l < L; ++l) off += tree_level_nodes(G, l);
  return off;
}

// Compile-time loop: f(std::integral_constant<int, i>) for i in [B, E).
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}
// Descending: i = E-1 down to B.
template <int B, int E, typename F>
__device__ __forceinline__ void static_for_down(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, E - 1>{});
    static_for_down<B, E - 1>(f);
  }
}

__device__ __forceinline__ float dexp(float v) { return expf(v); }
__device__ __forceinline__ double dexp(double v) { return exp(v); }

}  // namespace mmvm
