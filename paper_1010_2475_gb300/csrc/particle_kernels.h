// Launchers of the per-particle MMVM kernels (see particle_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

namespace mmvm {

struct FinishArgs {
  int n = 0, M = 0, K = 0, NB = 0;
  int nchunks = 0;                  // number of pair partials (0: single particle)
  int targets_per_block = 1;
  const double* partial = nullptr;  // [nchunks][NB][n] by sorted position
  const double* fpart = nullptr;    // far-field blocks [nfar][n_edge][n] (list form; nullable):
  int nfar = 0, n_edge = 0;         // edge column e = 2 (|beta| - 1) + beta1, beta1 <= 1
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

// Finish of a batch of one order (see BatchInst): items (instance, first
// target) of targets_per_block targets each; src selects the stage input
// (0: y, 1: ys); mode 1..4 is the RK4 stage (mode 0 is not used by batches).
struct BatchFinishArgs {
  int M = 0, K = 0, NB = 0;
  int targets_per_block = 1;
  const BatchInst* inst = nullptr;
  const int2* items = nullptr;
  const int* n_items = nullptr;     // device count of items
  const double* partial = nullptr;  // the batch's partials (BatchInst::part_off)
  const int* perm_local = nullptr;  // batch order (null: identity)
  const int* k_off = nullptr;       // finish tables of the order (tables.h)
  const int* e_l = nullptr;
  const int* e_b = nullptr;
  const double* e_c = nullptr;
  const double* psi0 = nullptr;
  int src = 0;
  double cs = 0;
  int mode = 1;
};

// perm_local (nullable): sorted slot -> local particle index (batch order);
// gbox (nullable, FP32 records only): group records as for launch_prep.
cudaError_t launch_prep_batch(int precision, int M, const BatchInst* inst, const int* slot_inst,
                              const int* n_slots, int max_slots, int src, double cs,
                              const int* perm_local, void* rec, void* gbox, cudaStream_t st);
// Spatial order of every instance of a batch (per-instance Morton keys in
// the instance's own bounding box, one stable 64-bit radix sort over the
// batch): perm_local[p] = the local particle at sorted slot p.
size_t batch_order_temp_bytes(int slot_cap);
cudaError_t launch_batch_order(int slot_cap, const int* n_slots, const BatchInst* inst,
                               const int* n_inst, int inst_cap, const int* slot_inst, void* ibox,
                               unsigned long long* kin, unsigned long long* kout, int* iin,
                               int* iout, void* temp, size_t temp_bytes, int* perm_local,
                               cudaStream_t st);
size_t finish_smem_bytes(int M, int targets_per_block);
// flags[i] = 1 if instance i's step-start state holds a non-finite value.
cudaError_t launch_scan_batch(int M, const BatchInst* inst, const int* n_inst, int max_inst,
                              int* flags, cudaStream_t st);
cudaError_t launch_finish_batch(const BatchFinishArgs& B, int grid, cudaStream_t st);
cudaError_t launch_advance_batch(BatchInst* inst, const int* n_inst, int max_inst,
                                 cudaStream_t st);

// Single particle, separable evaluation of the self term (self_high.cu).
struct SelfHighArgs {
  int M = 0, K = 0, NB = 0;
  const double* Min = nullptr;    // stage moments (K)
  const double* psi0 = nullptr;   // jet at the origin, |alpha| <= 3M (tables.h)
  const double* binom = nullptr;  // (M+1) x (M+1): C(l, q)
  const double* g = nullptr;      // M+1: g(j) = 4^{-j} / j!
  const double* cg = nullptr;     // (M+1)^3: C(l, q) g(k - q) at ((l (M+1) + k) (M+1) + q)
  double* at = nullptr;           // scratch (set by the launcher)
  double* Psi = nullptr;
  double *U1 = nullptr, *U2 = nullptr, *V1 = nullptr, *V2 = nullptr;
  double lam0sq = 0, four_nu = 0;
  const double* t_dev = nullptr;
  const double* dt_dev = nullptr;
  double cs = 0;
  int mode = 0;  // 0: RHS to out_*, 1..4: RK4 stage
  double *out_dx = nullptr, *out_dM = nullptr;
  double *y_x = nullptr, *y_M = nullptr, *ys_x = nullptr, *ys_M = nullptr;
  double *sum_x = nullptr, *sum_M = nullptr;
};
size_t self_high_scratch_doubles(int M);
cudaError_t launch_self_high(SelfHighArgs A, double* scratch, cudaStream_t st);  // 5 launches

// Records of the n particles (sorted position p holds particle perm[p]).  For
// FP32 records with gbox non-null also the group records (gdata_len(M)
// floats per group of kGroup: box, centre, radius, expansion; two launches).
// Diagnostics (diagnostics.cu): omega at npts points (device, interleaved
// x, y) of the state (x, mom) at the core of time *t_dev; the ring sums of
// squared deviations from the ring mean of v (nr rings of ntheta values).
int diag_max_order();
cudaError_t launch_vorticity(int n, int M, const double* x, const double* mom, const double* t_dev,
                             double lam0sq, double four_nu, int npts, const double* pts,
                             double* out, cudaStream_t st);
cudaError_t launch_ring_deviation(int nr, int ntheta, const double* v, double* ring,
                                  cudaStream_t st);
void gauss_legendre(int n, std::vector<double>& xs, std::vector<double>& ws);

// Adaptive Dormand-Prince steps (dopri.cu): out = y + h sum_j w_j k_j over
// the stage derivatives ks ([count][L], L = n (2 + K), x part first), and the
// max-norm error of a step into err_bits (the bits of a non-negative double).
struct DPCoef {
  double w[7];
  int count;
};
cudaError_t launch_dp_combine(int n, int K, const double* y_x, const double* y_M,
                              const double* ks, const DPCoef& c, const double* h_dev,
                              double* out_x, double* out_M, cudaStream_t st);
cudaError_t launch_dp_error(int n, int K, const double* y_x, const double* y_M,
                            const double* y5_x, const double* y5_M, const double* ks,
                            const DPCoef& c, const double* h_dev, double rtol, double atol,
                            unsigned long long* err_bits, cudaStream_t st);

cudaError_t launch_prep(int precision, int n, int M, const int* perm, const double* x,
                        const double* mom, const double* t_dev, const double* dt_dev, double cs,
                        double lam0sq, double four_nu, void* rec, void* gbox, cudaStream_t st);
// Centre, radius and expansion of every group (after the boxes are written);
// in a batch (inst non-null) n_slots and slot_inst give the slots, else n.
cudaError_t launch_group_multipole(int M, int n, const void* rec, void* gdata,
                                   const BatchInst* inst, const int* slot_inst,
                                   const int* n_slots, int max_slots, cudaStream_t st);
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
