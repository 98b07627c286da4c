// Launchers of the per-particle MMVM kernels (see particle_kernels.cu).
#pragma once

#include <cuda_runtime.h>

namespace mmvm {

struct FinishArgs {
  int n = 0, M = 0, K = 0, NB = 0;
  int nchunks = 0;                  // number of pair partials (0: single particle)
  int targets_per_block = 1;
  const double* partial = nullptr;  // [nchunks][NB][n] by sorted position
  const int* perm = nullptr;        // sorted position -> particle (null: identity)
  const double* Min = nullptr;      // stage moments (n x K)
  const int* k_off = nullptr;       // finish tables (tables.h)
  const int* e_l = nullptr;
  const int* e_b = nullptr;
  const double* e_c = nullptr;
  const double* psi0 = nullptr;
  double lam0sq = 0, four_nu = 0;   // lambda^2 = lam0sq + four_nu * t
  const double* t_dev = nullptr;    // step start time
  const double* dt_dev = nullptr;   // step size (null: 0)
  double cs = 0;                    // stage time = t + cs * dt
  int mode = 0;                     // 0: RHS to out_*, 1..4: RK4 stage s
  double* out_dx = nullptr;
  double* out_dM = nullptr;
  double* y_x = nullptr;            // step-start state
  double* y_M = nullptr;
  double* ys_x = nullptr;           // next stage state
  double* ys_M = nullptr;
  double* sum_x = nullptr;          // RK4 running sum
  double* sum_M = nullptr;
};

cudaError_t launch_prep(int precision, int n, int M, const int* perm, const double* x,
                        const double* mom, const double* t_dev, const double* dt_dev, double cs,
                        double lam0sq, double four_nu, void* rec, void* gbox, cudaStream_t st);
// Spatial order: perm[p] = particle at sorted position p (Morton order of the
// centres, ties by index).  temp_bytes() sizes the scratch for n particles.
size_t spatial_order_temp_bytes(int n);
cudaError_t launch_spatial_order(int n, const double* x, void* temp, size_t temp_bytes,
                                 int* perm, cudaStream_t st);
cudaError_t launch_finish(const FinishArgs& A, cudaStream_t st);
cudaError_t launch_advance_time(double* t_dev, const double* dt_dev, cudaStream_t st);
cudaError_t launch_scan(int n, int K, const double* x, const double* mom, int* flags,
                        cudaStream_t st);

}  // namespace mmvm
