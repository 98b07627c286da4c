// Diagnostics of a state on the GPU (FP64): the reconstructed vorticity
//   omega(p) = sum_j sum_{|k|<=M} M^j_k D^k phi_00(p - x^j; lambda)
// (eq:vorticity_decomposition; phi_00 = exp(-|x|^2/lambda^2) / (pi lambda^2)),
// with D^k phi_00(x) = (-1/lambda)^{|k|} H_{k1}(t1) H_{k2}(t2) phi_00(x),
// t = x / lambda and H_n the physicists' Hermite polynomials
// (H_{n+1} = 2 t H_n - 2 n H_{n-1}), and the ring sums of the nonaxisymmetric
// enstrophy (eq:nonaxi_enstrophy): per ring of a polar grid, the sum over its
// angles of (omega - ring mean)^2.
//
// One thread per point; the particles pass through shared memory in tiles.
// A particle farther than (sqrt(2M+1) + 6) lambda from the point is skipped:
// every Hermite function of order <= M is below e^-36 of its peak there.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "particle_kernels.h"

namespace mmvm {

namespace {

constexpr int kMaxOrderDiag = 64;

__global__ void vorticity_kernel(int n, int M, int K, int tile, const double* __restrict__ x,
                                 const double* __restrict__ mom, const double* t_dev,
                                 double lam0sq, double four_nu, int npts,
                                 const double* __restrict__ pts, double* __restrict__ out) {
  extern __shared__ double sh[];  // tile x (2 + K)
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const double lam2 = lam0sq + four_nu * (t_dev ? *t_dev : 0.0);
  const double lam = sqrt(lam2), il = 1.0 / lam;
  const double rc = sqrt(2.0 * M + 1.0) + 6.0;
  const double cut2 = rc * rc;
  const double px = p < npts ? pts[2 * p] : 0.0, py = p < npts ? pts[2 * p + 1] : 0.0;
  double hx[kMaxOrderDiag + 1], hy[kMaxOrderDiag + 1];
  double acc = 0.0;
  const int W = 2 + K;
  for (int j0 = 0; j0 < n; j0 += tile) {
    const int cnt = min(tile, n - j0);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * W; i += blockDim.x) {
      const int jj = i / W, c = i % W;
      sh[i] = c < 2 ? x[2 * (size_t)(j0 + jj) + c] : mom[(size_t)(j0 + jj) * K + (c - 2)];
    }
    __syncthreads();
    if (p >= npts) continue;
    for (int jj = 0; jj < cnt; ++jj) {
      const double* r = sh + jj * W;
      const double t1 = (px - r[0]) * il, t2 = (py - r[1]) * il;
      const double r2 = t1 * t1 + t2 * t2;
      if (r2 > cut2) continue;
      hx[0] = 1.0;
      hy[0] = 1.0;
      if (M >= 1) {
        hx[1] = 2.0 * t1;
        hy[1] = 2.0 * t2;
      }
      for (int q = 1; q < M; ++q) {
        hx[q + 1] = 2.0 * t1 * hx[q] - 2.0 * q * hx[q - 1];
        hy[q + 1] = 2.0 * t2 * hy[q] - 2.0 * q * hy[q - 1];
      }
      const double* mk = r + 2;
      double sum = 0.0, sc = 1.0;  // sc = (-1/lambda)^s
      int col = 0;
      for (int s = 0; s <= M; ++s) {
        double part = 0.0;
        for (int k2 = 0; k2 <= s; ++k2, ++col) part = fma(mk[col], hx[s - k2] * hy[k2], part);
        sum = fma(sc, part, sum);
        sc *= -il;
      }
      acc = fma(sum, exp(-r2), acc);
    }
  }
  if (p < npts) out[p] = acc * (il * il) * 0.31830988618379067154;  // / (pi lambda^2)
}

// One block per ring of ntheta values: sum over the ring of (v - mean)^2.
__global__ void ring_deviation_kernel(int ntheta, const double* __restrict__ v,
                                      double* __restrict__ ring) {
  __shared__ double red[32];
  const double* w = v + (size_t)blockIdx.x * ntheta;
  auto block_sum = [&](double a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    __syncthreads();  // red is free
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
  };
  double a = 0.0;
  for (int i = threadIdx.x; i < ntheta; i += blockDim.x) a += w[i];
  const double mean = block_sum(a) / ntheta;
  double d = 0.0;
  for (int i = threadIdx.x; i < ntheta; i += blockDim.x) d += (w[i] - mean) * (w[i] - mean);
  const double tot = block_sum(d);
  if (threadIdx.x == 0) ring[blockIdx.x] = tot;
}

}  // namespace

int diag_max_order() { return kMaxOrderDiag; }

// Nodes and weights of n-point Gauss-Legendre quadrature on [-1, 1]: Newton's
// method on P_n (three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1})
// from the usual cosine start, w = 2 / ((1 - x^2) P_n'(x)^2).
void gauss_legendre(int n, std::vector<double>& xs, std::vector<double>& ws) {
  xs.assign(n, 0.0);
  ws.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      const double pn = n == 0 ? 1.0 : p1, pm = n == 0 ? 0.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
      const double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    xs[i] = -z;
    xs[n - 1 - i] = z;
    ws[i] = ws[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

cudaError_t launch_vorticity(int n, int M, const double* x, const double* mom, const double* t_dev,
                             double lam0sq, double four_nu, int npts, const double* pts,
                             double* out, cudaStream_t st) {
  if (M < 0 || M > kMaxOrderDiag) return cudaErrorInvalidValue;
  const int K = n_moments(M);
  const int tile = std::max(1, std::min(64, 6144 / (2 + K)));
  const size_t smem = (size_t)tile * (2 + K) * sizeof(double);
  const int threads = 128;
  vorticity_kernel<<<std::max(1, (npts + threads - 1) / threads), threads, smem, st>>>(
      n, M, K, tile, x, mom, t_dev, lam0sq, four_nu, npts, pts, out);
  return cudaGetLastError();
}

cudaError_t launch_ring_deviation(int nr, int ntheta, const double* v, double* ring,
                                  cudaStream_t st) {
  ring_deviation_kernel<<<std::max(1, nr), 256, 0, st>>>(ntheta, v, ring);
  return cudaGetLastError();
}

}  // namespace mmvm
