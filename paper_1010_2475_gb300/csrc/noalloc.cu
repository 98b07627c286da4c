// Right-hand side without any device allocation (mmvm_rhs_noalloc).
//
// Some callers cannot call cudaMalloc: an application that hands all device
// memory to its own pool or works under a fixed memory budget, code on a
// latency-critical path where cudaMalloc/cudaFree would synchronise the
// device, or a plugin whose host forbids allocation once it is running.  This
// entry point takes the caller's device buffers for inputs and outputs and
// keeps everything else it needs (coefficient tables, source records,
// per-chunk partial sums) in one file-scope __device__ array of fixed size,
// which every GPU that loads the library holds until the process exits.
//
// Limits: n <= kMaxN particles, order <= kMaxOrder.  Every call shares the
// array: the tables of the last order used stay resident, and records and
// partials are rewritten in full by each call, so nothing needs clearing.
// Calls whose work overlaps on the GPU (on different streams, or from
// different host threads) race on the array and must be serialised by the
// caller.  The first call on a device looks up the array's device address
// (and uploads the tables of its order, as does the first call after a change
// of order, which also waits for the device); make such calls before any
// stream capture.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mmvm.h"
#include "common.cuh"
#include "pair_registry.h"
#include "particle_kernels.h"
#include "tables.h"

namespace mmvm {
void set_last_error(const char* msg);  // api.cu: message for mmvm_last_error()
}

namespace {

constexpr int kMaxN = 4096;
constexpr int kMaxOrder = 8;
constexpr int kChunks = 2;
// tables region: k_off, e_l, e_b (int) and e_c, psi0 (double), sized for order 8
constexpr size_t kTableBytes = 1u << 20;
// largest record: FP64 order 8, 48 doubles = 384 bytes (FP32: 68 floats)
constexpr size_t kRecBytes = (size_t)kMaxN * 384;
constexpr size_t kPartialBytes = (size_t)kChunks * 152 * kMaxN * 8;  // NB <= 152 at order 8
constexpr size_t kScratchBytes = kTableBytes + 256 + kRecBytes + kPartialBytes;

static_assert(kScratchBytes == 12583168, "the documented size of the scratch array");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceScratch {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_scratch on this device
  int tables_order = -1;          // order whose tables are resident
  int off_koff = 0, off_el = 0, off_eb = 0, off_ec = 0, off_psi0 = 0;
};
std::mutex g_mu;
DeviceScratch g_dev[64];

__global__ void set_time_kernel(double* t_dev, double t) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *t_dev = t;
}

int set_err(int code, const std::string& m) {
  mmvm::set_last_error(m.c_str());
  return code;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" int mmvm_rhs_noalloc(const mmvm_config* cfg, int64_t n, double t, const double* d_x,
                                const double* d_moments, double* d_dxdt, double* d_dMdt,
                                void* stream) {
  using namespace mmvm;
  if (!cfg || !d_x || !d_moments || !d_dxdt || !d_dMdt)
    return set_err(MMVM_E_INVALID_ARG, "null argument");
  if (cfg->order < 0 || cfg->order > kMaxOrder)
    return set_err(MMVM_E_UNSUPPORTED, "mmvm_rhs_noalloc: order must be 0..8");
  if (n < 1 || n > kMaxN)
    return set_err(MMVM_E_UNSUPPORTED, "mmvm_rhs_noalloc: n must be 1..4096 (fixed scratch)");
  if (cfg->precision != MMVM_FP64 && cfg->precision != MMVM_MIXED_FP32)
    return set_err(MMVM_E_INVALID_ARG, "unknown precision");
  if (!(cfg->lambda0 > 0.0) || !(cfg->nu >= 0.0) || !std::isfinite(t) ||
      cfg->lambda0 * cfg->lambda0 + 4.0 * cfg->nu * t <= 0.0)
    return set_err(MMVM_E_INVALID_ARG, "bad lambda0, nu or t");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int M = cfg->order, prec = cfg->precision;
  const int K = n_moments(M), NB = n_beta(M);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64)
    return set_err(MMVM_E_DEVICE, std::string("cudaGetDevice: ") + cudaGetErrorString(e));

  std::lock_guard<std::mutex> lk(g_mu);
  DeviceScratch& ds = g_dev[dev];
  if (!ds.ready) {  // once per device, with that device current
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess)
      return set_err(MMVM_E_DEVICE, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    ds.base = static_cast<unsigned char*>(p);
    ds.ready = true;
  }
  if (ds.tables_order != M) {  // upload the finish tables of this order
    if (ds.tables_order >= 0) {  // earlier calls may still read the old tables
      e = cudaDeviceSynchronize();
      if (e != cudaSuccess)
        return set_err(MMVM_E_DEVICE, std::string("synchronize: ") + cudaGetErrorString(e));
    }
    FinishTables T = build_finish_tables(M);
    size_t off = 0;
    ds.off_koff = (int)off;
    off = align256(off + T.k_off.size() * sizeof(int));
    ds.off_el = (int)off;
    off = align256(off + T.e_l.size() * sizeof(int));
    ds.off_eb = (int)off;
    off = align256(off + T.e_b.size() * sizeof(int));
    ds.off_ec = (int)off;
    off = align256(off + T.e_c.size() * sizeof(double));
    ds.off_psi0 = (int)off;
    off = align256(off + T.psi0.size() * sizeof(double));
    if (off > kTableBytes) return set_err(MMVM_E_UNSUPPORTED, "tables exceed the fixed scratch");
    struct Up {
      int off;
      const void* src;
      size_t bytes;
    } ups[] = {{ds.off_koff, T.k_off.data(), T.k_off.size() * sizeof(int)},
               {ds.off_el, T.e_l.data(), T.e_l.size() * sizeof(int)},
               {ds.off_eb, T.e_b.data(), T.e_b.size() * sizeof(int)},
               {ds.off_ec, T.e_c.data(), T.e_c.size() * sizeof(double)},
               {ds.off_psi0, T.psi0.data(), T.psi0.size() * sizeof(double)}};
    for (const Up& u : ups) {
      if (!u.bytes) continue;
      e = cudaMemcpyAsync(ds.base + u.off, u.src, u.bytes, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess)
        return set_err(MMVM_E_DEVICE, std::string("table upload: ") + cudaGetErrorString(e));
    }
    e = cudaStreamSynchronize(st);  // the host vectors go out of scope here
    if (e != cudaSuccess)
      return set_err(MMVM_E_DEVICE, std::string("table upload: ") + cudaGetErrorString(e));
    ds.tables_order = M;
  }
  unsigned char* base = ds.base;
  double* t_dev = reinterpret_cast<double*>(base + kTableBytes);
  unsigned char* rec = base + kTableBytes + 256;
  double* partial = reinterpret_cast<double*>(rec + kRecBytes);
  set_time_kernel<<<1, 32, 0, st>>>(t_dev, t);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return set_err(MMVM_E_DEVICE, std::string("launch: ") + cudaGetErrorString(e));
  const double lam0sq = cfg->lambda0 * cfg->lambda0, four_nu = 4.0 * cfg->nu;
  const int chunks = n > 1 ? (n >= 2 * kGroup * 4 ? kChunks : 1) : 0;
  if (n > 1) {
    PairEntry pe = pair_entry(M, prec, 0);
    if (pe.M != M) return set_err(MMVM_E_UNSUPPORTED, "pair kernel variant not compiled");
    if ((size_t)n * pe.rec_len * pe.elem_bytes > kRecBytes)
      return set_err(MMVM_E_UNSUPPORTED, "records exceed the fixed scratch");
    if ((e = pair_prepare(pe, kGroup)) != cudaSuccess ||
        (e = launch_prep(prec, (int)n, M, nullptr, d_x, d_moments, t_dev, nullptr, 0.0, lam0sq,
                         four_nu, rec, nullptr, st)) != cudaSuccess ||
        (e = pair_launch(pe, rec, (int)n, chunks, kGroup, nullptr, partial, 0, st)) != cudaSuccess)
      return set_err(MMVM_E_DEVICE, std::string("launch: ") + cudaGetErrorString(e));
  }
  FinishArgs A;
  A.n = (int)n;
  A.M = M;
  A.K = K;
  A.NB = NB;
  A.nchunks = chunks;
  A.targets_per_block = std::max(1, 128 / (((K + 31) / 32) * 32));  // as for a context
  A.partial = n > 1 ? partial : nullptr;
  A.Min = d_moments;
  A.k_off = reinterpret_cast<const int*>(base + ds.off_koff);
  A.e_l = reinterpret_cast<const int*>(base + ds.off_el);
  A.e_b = reinterpret_cast<const int*>(base + ds.off_eb);
  A.e_c = reinterpret_cast<const double*>(base + ds.off_ec);
  A.psi0 = reinterpret_cast<const double*>(base + ds.off_psi0);
  A.lam0sq = lam0sq;
  A.four_nu = four_nu;
  A.t_dev = t_dev;
  A.dt_dev = nullptr;
  A.cs = 0.0;
  A.mode = 0;
  A.out_dx = d_dxdt;
  A.out_dM = d_dMdt;
  if ((e = launch_finish(A, st)) != cudaSuccess)
    return set_err(MMVM_E_DEVICE, std::string("finish: ") + cudaGetErrorString(e));
  return MMVM_OK;
}
