// C-ABI of the MMVM library (declarations and contracts in include/mmvm.h).
//
// One right-hand-side evaluation is three launches on the context stream:
//   prep   (core size at the stage time, FP32/FP64 source records),
//   pair   (all-pairs stream-function correlation, skipped for n == 1),
//   finish (FP64: chunk sum, self pair, centroid, moment equation, RK4 stage).
// An RK4 step is four evaluations plus a one-thread time advance; the step is
// captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>
#include <vector>

#include "../../include/mmvm.h"
#include "common.cuh"
#include "pair_registry.h"
#include "particle_kernels.h"
#include "tables.h"

namespace {

// Highest order whose finish uses the (k, l, beta) coefficient tables.
constexpr int kMaxOrderTables = 16;

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? MMVM_E_OOM : MMVM_E_DEVICE;
}

#define MMVM_CK(expr)                                  \
  do {                                                 \
    cudaError_t e_ = (expr);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr); \
  } while (0)

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t cap = 0;  // elements
  cudaError_t ensure(size_t n) {
    if (n <= cap && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) cap = n;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

}  // namespace

namespace mmvm {
// Record the calling thread's last error message (for other files of the library).
void set_last_error(const char* msg) { g_err = msg ? msg : ""; }
}  // namespace mmvm

struct mmvm_ctx {
  mmvm_config cfg{};
  int M = 0, K = 0, NB = 0;
  int64_t n = 0;
  cudaStream_t own = nullptr, st = nullptr;
  DevBuf<double> x, m, xs, ms, xsum, msum, rdx, rdm, scal, partial;
  DevBuf<unsigned char> rec, order_tmp;
  DevBuf<int> flags, k_off, e_l, e_b, perm;
  DevBuf<float> gbox;  // group records (gdata_len(M) floats per kGroup sorted positions)
  // cumulative work of the all-pairs kernel: near pairs, far pairs source by
  // source, tile expansions evaluated, pairs those expansions covered
  DevBuf<unsigned long long> counts;
  bool far = false;    // FP32 and not MMVM_FLAG_NO_FAR_FIELD: sort + far-field tiles
  bool high = false;   // single particle through the separable self term (self_high.cu)
  DevBuf<double> sbinom, sg, scg, sscr;  // its factor tables and scratch
  DevBuf<double> dpts, dval, dring;  // diagnostics: points, values, ring sums
  DevBuf<double> dk;                  // adaptive steps: 7 stage derivatives
  DevBuf<unsigned long long> derr;    // adaptive steps: error of the step (bits)
  int order_launches = 0;  // kernels launched by one spatial ordering
  DevBuf<double> e_c, psi0;
  mmvm::PairEntry pe;
  // interaction-list form of the all-pairs kernels (FP32 with the far field):
  // near lists (G x G entries, G counts), far-field partials (lfar blocks of
  // the edge columns), list segments of the near partials, device error flag
  bool list = false;
  mmvm::ListEntry le;
  int lseg = 1, lfar = 1;
  DevBuf<int2> lent;
  DevBuf<int> lcnt, errf;
  DevBuf<double> fpart;
  // far field of the list form through the tree over the groups (walked from
  // the lc-th level, tfar nodes there = far blocks), else the flat far kernel
  bool tree = false;
  DevBuf<float> tnodes;
  int lc = 0, tfar = 1;
  int S = 32;            // sources per shared-memory tile
  int chunks = 1;        // source chunks of the pair kernel
  int finish_tb = 1;     // targets per finish block
  bool graph_ok = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int64_t launches = 0;
  double last_dt = NAN;  // dt currently held in dt_dev
  // optional pair-kernel timing: one event pair per RK stage (slot 4: rhs)
  bool timing = false;
  cudaEvent_t ev[5][2] = {};
  bool ev_pending[5] = {};
  // list form: marks between its kernels (after list build + tree, after the
  // far kernel, after each near kernel) and their summed times since the last
  // mmvm_pair_time_parts call
  static constexpr int kMarks = 2 + mmvm::kMaxListSlices;
  cudaEvent_t evm[5][kMarks] = {};
  bool evm_pending[5] = {};
  double parts_ms[kMarks] = {};
  int64_t parts_count = 0;

  double* t_dev() { return scal.p; }
  double* dt_dev() { return scal.p + 1; }

  void drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    gexec = nullptr;
    graph = nullptr;
    graph_ok = false;
  }
};

namespace {

// Source chunks of an all-pairs launch over n records with tpc targets per
// CTA and per_sm resident CTAs per SM.
int chunks_for(int64_t n, int tpc, int per_sm, int device, int S) {
  if (n <= 1) return 0;
  int dev_sms = 0;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, device);
  per_sm = std::max(per_sm, 1);
  const int64_t tiles = (n + tpc - 1) / tpc;
  const int64_t slots = (int64_t)std::max(dev_sms, 1) * per_sm;
  // ~48 waves of CTAs, chunks no shorter than 4 tiles of sources: target
  // tiles differ a lot in cost (near vs far tiles), and many small CTAs let
  // the block scheduler even out the SMs (measured at N = 65536, M = 6 with
  // 256 targets per CTA: 3 chunks 257 ms, 12 chunks 231 ms, 24 chunks 219 ms,
  // 48 chunks 217 ms per launch)
  int64_t ch = (48 * slots + tiles - 1) / tiles;
  if (const char* f = std::getenv("MMVM_CHUNKS")) ch = std::atoi(f);  // measurement override
  const int64_t max_ch = std::max<int64_t>(1, n / (4 * S));
  ch = std::min(std::max<int64_t>(ch, 1), max_ch);
  return (int)ch;
}

// Shape of the list form for n records: list segments per target group
// (enough CTAs of the near kernels for ~20 waves) and source ranges of the
// far kernel (~8 waves of warps, at least 16 source groups per warp).
void list_shape(const mmvm_ctx* c, const mmvm::ListEntry& e, int64_t n, int* lseg, int* lfar) {
  int dev_sms = 0;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->cfg.device);
  dev_sms = std::max(dev_sms, 1);
  const int64_t G = (n + mmvm::kGroup - 1) / mmvm::kGroup;
  const int occ = std::max(1, mmvm::list_occupancy(e));
  int64_t seg = (20 * (int64_t)dev_sms * occ + G - 1) / G;
  if (const char* f = std::getenv("MMVM_LIST_SEGMENTS")) seg = std::atoi(f);  // measurement override
  *lseg = (int)std::min<int64_t>(std::max<int64_t>(seg, 1), 16);
  int focc = 0;
  if (e.far.far_occupancy(&focc) != cudaSuccess) {
    cudaGetLastError();
    focc = 1;
  }
  const int64_t warp_slots = (int64_t)dev_sms * std::max(focc, 1) * 4;
  int64_t far = (8 * warp_slots + G - 1) / G;
  far = std::min<int64_t>(far, std::max<int64_t>(1, G / 16));
  if (const char* f = std::getenv("MMVM_FAR_RANGES")) far = std::atoi(f);  // measurement override
  *lfar = (int)std::min<int64_t>(std::max<int64_t>(far, 1), 64);
}

// Kernels one all-pairs evaluation launches (without prep and ordering).
int pair_launches(const mmvm_ctx* c) {
  if (!c->list) return c->pe.nslices;
  const int G = (int)((c->n + mmvm::kGroup - 1) / mmvm::kGroup);
  return 1 + (c->tree ? mmvm::tree_levels(G) + 1 : 1) + c->le.nslices;
}

int choose_chunks(const mmvm_ctx* c, int64_t n) {
  const int per_sm = c->pe.nslices ? mmvm::pair_occupancy(c->pe, c->S) : 1;
  return chunks_for(n, c->pe.tpc, per_sm, c->cfg.device, c->S);
}

// Chunks a variant is timed on by the autotuner (the partial buffer always
// holds at least this many).
constexpr int kTuneChunks = 8;

// Process-wide autotuning results: (device, M, precision, far, log2 n) -> variant.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_tuned;
std::map<std::tuple<int, int, int, int, int>, int> g_tuned_tree;  // list form: tree far field

int ilog2(int64_t v) {
  int r = 0;
  while (v > 1) {
    v >>= 1;
    ++r;
  }
  return r;
}

int ensure_buffers(mmvm_ctx* c, int64_t n) {
  const size_t K = c->K;
  bool realloc = false;
  auto grow = [&](auto& b, size_t cnt) -> cudaError_t {
    if (cnt > b.cap || !b.p) realloc = true;
    return b.ensure(cnt);
  };
  MMVM_CK(grow(c->x, 2 * n));
  MMVM_CK(grow(c->m, K * n));
  MMVM_CK(grow(c->xs, 2 * n));
  MMVM_CK(grow(c->ms, K * n));
  MMVM_CK(grow(c->xsum, 2 * n));
  MMVM_CK(grow(c->msum, K * n));
  MMVM_CK(grow(c->rdx, 2 * n));
  MMVM_CK(grow(c->rdm, K * n));
  if (n > 1) {
    c->chunks = choose_chunks(c, n);
    MMVM_CK(grow(c->rec, (size_t)n * c->pe.rec_len * c->pe.elem_bytes));
    MMVM_CK(grow(c->partial, (size_t)std::max(c->chunks, kTuneChunks) * c->NB * n));
    if (c->far) {
      const size_t G = (size_t)((n + mmvm::kGroup - 1) / mmvm::kGroup);
      MMVM_CK(grow(c->lent, G * G));
      MMVM_CK(grow(c->lcnt, G));
      if (!c->errf.p) {
        MMVM_CK(c->errf.ensure(1));
        MMVM_CK(cudaMemset(c->errf.p, 0, sizeof(int)));
      }
      MMVM_CK(grow(c->perm, (size_t)n));
      MMVM_CK(grow(c->gbox, (size_t)mmvm::gdata_len(c->M) *
                                ((n + mmvm::kGroup - 1) / mmvm::kGroup)));
      MMVM_CK(grow(c->order_tmp, mmvm::spatial_order_temp_bytes((int)n)));
      if (realloc) {
        // count the kernels one ordering launches (the sort's are the library's)
        cudaGraph_t g = nullptr;
        MMVM_CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
        cudaError_t e1 = mmvm::launch_spatial_order((int)n, c->x.p, c->order_tmp.p,
                                                    c->order_tmp.cap, c->perm.p, c->st);
        cudaError_t e2 = cudaStreamEndCapture(c->st, &g);
        if (e1 != cudaSuccess) return cuda_fail(e1, "spatial order");
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture(order)");
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(g, nodes.data(), &nn);
        int kn = 0;
        for (auto nd : nodes) {
          cudaGraphNodeType ty;
          cudaGraphNodeGetType(nd, &ty);
          if (ty == cudaGraphNodeTypeKernel) ++kn;
        }
        c->order_launches = kn;
        cudaGraphDestroy(g);
      }
    }
  } else {
    c->chunks = 0;
  }
  if (realloc) c->drop_graph();
  return MMVM_OK;
}

// One RHS evaluation: mode 0 writes (rdx, rdm); modes 1..4 are RK4 stages.
// out_dx / out_dM (mode 0 only): where the RHS goes (null: the context's own
// rdx / rdm).
int enqueue_rhs(mmvm_ctx* c, int mode, const double* xin, const double* min_, double cs,
                const double* dt_dev, double* out_dx = nullptr, double* out_dM = nullptr) {
  const int n = (int)c->n;
  if (!out_dx) out_dx = c->rdx.p;
  if (!out_dM) out_dM = c->rdm.p;
  const double lam0sq = c->cfg.lambda0 * c->cfg.lambda0;
  const double four_nu = 4.0 * c->cfg.nu;
  const int* perm = (n > 1 && c->far) ? c->perm.p : nullptr;
  if (n > 1) {
    if (c->far && (mode == 0 || mode == 1)) {  // order from the step-start centres
      MMVM_CK(mmvm::launch_spatial_order(n, xin, c->order_tmp.p, c->order_tmp.cap, c->perm.p,
                                         c->st));
      c->launches += c->order_launches;
    }
    MMVM_CK(mmvm::launch_prep(c->cfg.precision, n, c->M, perm, xin, min_, c->t_dev(), dt_dev,
                              cs, lam0sq, four_nu, c->rec.p, c->far ? c->gbox.p : nullptr,
                              c->st));
    const int slot = mode == 0 ? 4 : mode - 1;
    if (c->timing) MMVM_CK(cudaEventRecord(c->ev[slot][0], c->st));
    if (c->list) {
      MMVM_CK(mmvm::list_launch(c->le, reinterpret_cast<const float*>(c->rec.p), n, c->gbox.p,
                                c->lent.p, c->lcnt.p, c->lseg, c->partial.p, c->lfar, c->fpart.p,
                                c->tree ? c->tnodes.p : nullptr, c->lc, c->counts.p, c->errf.p,
                                c->st, c->timing ? c->evm[slot] : nullptr));
      if (c->timing) c->evm_pending[slot] = true;
    } else {
      MMVM_CK(mmvm::pair_launch(c->pe, c->rec.p, n, c->chunks, c->S,
                                c->far ? c->gbox.p : nullptr, c->partial.p, 0, c->st,
                                c->counts.p));
    }
    if (c->timing) {
      MMVM_CK(cudaEventRecord(c->ev[slot][1], c->st));
      c->ev_pending[slot] = true;
    }
    c->launches += (c->far ? 2 : 1) + pair_launches(c);
  }
  if (c->high) {  // n == 1: separable self term, dx/dt = 0
    mmvm::SelfHighArgs H;
    H.M = c->M;
    H.K = c->K;
    H.NB = c->NB;
    H.Min = min_;
    H.psi0 = c->psi0.p;
    H.binom = c->sbinom.p;
    H.g = c->sg.p;
    H.cg = c->scg.p;
    H.lam0sq = lam0sq;
    H.four_nu = four_nu;
    H.t_dev = c->t_dev();
    H.dt_dev = dt_dev;
    H.cs = cs;
    H.mode = mode;
    H.out_dx = out_dx;
    H.out_dM = out_dM;
    H.y_x = c->x.p;
    H.y_M = c->m.p;
    H.ys_x = c->xs.p;
    H.ys_M = c->ms.p;
    H.sum_x = c->xsum.p;
    H.sum_M = c->msum.p;
    MMVM_CK(mmvm::launch_self_high(H, c->sscr.p, c->st));
    c->launches += 5;
    return MMVM_OK;
  }
  mmvm::FinishArgs A;
  A.n = n;
  A.M = c->M;
  A.K = c->K;
  A.NB = c->NB;
  A.nchunks = n > 1 ? (c->list ? c->lseg : c->chunks) : 0;
  if (n > 1 && c->list) {
    A.fpart = c->fpart.p;
    A.nfar = c->tree ? c->tfar : c->lfar;
    A.n_edge = c->le.far.n_edge;
  }
  A.targets_per_block = c->finish_tb;
  A.partial = n > 1 ? c->partial.p : nullptr;
  A.perm = perm;
  A.Min = min_;
  A.k_off = c->k_off.p;
  A.e_l = c->e_l.p;
  A.e_b = c->e_b.p;
  A.e_c = c->e_c.p;
  A.psi0 = c->psi0.p;
  A.lam0sq = lam0sq;
  A.four_nu = four_nu;
  A.t_dev = c->t_dev();
  A.dt_dev = dt_dev;
  A.cs = cs;
  A.mode = mode;
  A.out_dx = out_dx;
  A.out_dM = out_dM;
  A.y_x = c->x.p;
  A.y_M = c->m.p;
  A.ys_x = c->xs.p;
  A.ys_M = c->ms.p;
  A.sum_x = c->xsum.p;
  A.sum_M = c->msum.p;
  MMVM_CK(mmvm::launch_finish(A, c->st));
  c->launches += 1;
  return MMVM_OK;
}

int enqueue_step(mmvm_ctx* c) {
  int rc;
  double* dt = c->dt_dev();
  if ((rc = enqueue_rhs(c, 1, c->x.p, c->m.p, 0.0, dt))) return rc;
  if ((rc = enqueue_rhs(c, 2, c->xs.p, c->ms.p, 0.5, dt))) return rc;
  if ((rc = enqueue_rhs(c, 3, c->xs.p, c->ms.p, 0.5, dt))) return rc;
  if ((rc = enqueue_rhs(c, 4, c->xs.p, c->ms.p, 1.0, dt))) return rc;
  MMVM_CK(mmvm::launch_advance_time(c->t_dev(), dt, c->st));
  c->launches += 1;
  return MMVM_OK;
}

// Time one launch of variant e over the first gy of its `chunks` source
// chunks on the context's current records (after one untimed launch);
// *per_pair = milliseconds per pair evaluated.
static cudaError_t time_pair_variant(mmvm_ctx* c, const mmvm::PairEntry& e, int n, int chunks,
                                     int gy, cudaEvent_t e0, cudaEvent_t e1, double* per_pair) {
  const int chunk_len = mmvm::round_up((n + chunks - 1) / chunks, c->S);
  const void* gb = c->far ? c->gbox.p : nullptr;
  cudaError_t r = mmvm::pair_launch(e, c->rec.p, n, chunks, c->S, gb, c->partial.p, gy, c->st);
  if (r == cudaSuccess) r = cudaEventRecord(e0, c->st);
  if (r == cudaSuccess)
    r = mmvm::pair_launch(e, c->rec.p, n, chunks, c->S, gb, c->partial.p, gy, c->st);
  if (r == cudaSuccess) r = cudaEventRecord(e1, c->st);
  if (r == cudaSuccess) r = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (r == cudaSuccess) r = cudaEventElapsedTime(&ms, e0, e1);
  if (r != cudaSuccess) return r;
  const double pairs = (double)n * std::min((double)gy * chunk_len, (double)n);
  *per_pair = ms / pairs;
  if (const char* vb = std::getenv("MMVM_TUNE_VERBOSE"))
    if (std::atoi(vb))
      std::fprintf(stderr, "[mmvm tune] M=%d prec=%d n=%d variant %d (slices=%d TPC=%d MINB=%d "
                   "SYNC=%d), %d of %d chunks: %.3f ms, %.3e pairs/s\n", c->M, c->cfg.precision,
                   n, e.variant, e.nslices, e.tpc, e.minb, e.sync, gy, chunks, ms,
                   pairs / (ms * 1e-3));
  return cudaSuccess;
}

// Make the list buffers hold list variant e's shape for n records; the
// shape goes to *lseg / *lfar.
static int ensure_list_buffers(mmvm_ctx* c, const mmvm::ListEntry& e, int n, int* lseg,
                               int* lfar) {
  list_shape(c, e, n, lseg, lfar);
  const size_t tn = (size_t)mmvm::tree_nodes((n + mmvm::kGroup - 1) / mmvm::kGroup) *
                    mmvm::gdata_len(c->M);
  if (tn > c->tnodes.cap || !c->tnodes.p) {
    MMVM_CK(c->tnodes.ensure(std::max<size_t>(tn, 1)));
    c->drop_graph();
  }
  const size_t part = (size_t)*lseg * c->NB * n;
  const size_t fp = (size_t)*lfar * e.far.n_edge * n;
  if (part > c->partial.cap || fp > c->fpart.cap || !c->fpart.p) {
    MMVM_CK(c->partial.ensure(std::max(part, c->partial.cap)));
    MMVM_CK(c->fpart.ensure(std::max(fp, c->fpart.cap)));
    c->drop_graph();
  }
  return MMVM_OK;
}

// Time one launch of list variant e on the context's current records (after
// one untimed launch); *per_pair = milliseconds per pair.
static int time_list_variant(mmvm_ctx* c, const mmvm::ListEntry& e, int n, bool tree,
                             cudaEvent_t e0, cudaEvent_t e1, double* per_pair) {
  int lseg = 1, lfar = 1;
  int rc = ensure_list_buffers(c, e, n, &lseg, &lfar);
  if (rc) return rc;
  const float* rec = reinterpret_cast<const float*>(c->rec.p);
  int tfar = 1;
  const int lc = mmvm::tree_chunk_level((n + mmvm::kGroup - 1) / mmvm::kGroup, lfar, &tfar);
  float* tr = tree ? c->tnodes.p : nullptr;
  MMVM_CK(mmvm::list_launch(e, rec, n, c->gbox.p, c->lent.p, c->lcnt.p, lseg, c->partial.p, lfar,
                            c->fpart.p, tr, lc, nullptr, c->errf.p, c->st));
  MMVM_CK(cudaEventRecord(e0, c->st));
  MMVM_CK(mmvm::list_launch(e, rec, n, c->gbox.p, c->lent.p, c->lcnt.p, lseg, c->partial.p, lfar,
                            c->fpart.p, tr, lc, nullptr, c->errf.p, c->st));
  MMVM_CK(cudaEventRecord(e1, c->st));
  MMVM_CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  MMVM_CK(cudaEventElapsedTime(&ms, e0, e1));
  *per_pair = ms / ((double)n * n);
  if (const char* vb = std::getenv("MMVM_TUNE_VERBOSE"))
    if (std::atoi(vb))
      std::fprintf(stderr, "[mmvm tune] M=%d n=%d list variant %d (near kernels=%d, segments=%d, "
                   "far %s, far blocks=%d): %.3f ms, %.3e pairs/s\n", c->M, n, e.variant,
                   e.nslices, lseg, tree ? "tree" : "flat", tree ? tfar : lfar, ms,
                   (double)n * n / (ms * 1e-3));
  return MMVM_OK;
}

// Pick the all-pairs variant for this (order, precision, size class): time
// each compiled variant of the direct form on the current records (every
// target tile against the first kTuneChunks source chunks of the variant's
// own chunking), then time the variants within 10 % of the best on their
// full launch, and (FP32 with the far field) every variant of the list form
// on its full launch, and keep the fastest per pair.  Variant numbers
// 0 .. nv-1 are the direct form, nv .. nv+nl-1 the list form.
// MMVM_PAIR_VARIANT=<v> forces a variant, MMVM_AUTOTUNE=0 keeps variant 0.
// Runs outside any stream capture (from set_state).
int tune_pair(mmvm_ctx* c) {
  const int n = (int)c->n;
  const int nv = mmvm::pair_variant_count(c->M, c->cfg.precision);
  const int nl = c->far ? mmvm::list_variant_count(c->M) : 0;
  if (n <= 1 || nv + nl <= 1) return MMVM_OK;
  const auto key = std::make_tuple(c->cfg.device, c->M, c->cfg.precision, c->far ? 1 : 0,
                                   ilog2(n));
  int choice = -1, tree_choice = -1;
  if (const char* f = std::getenv("MMVM_PAIR_VARIANT")) choice = std::atoi(f);
  if (choice < 0) {
    if (const char* a = std::getenv("MMVM_AUTOTUNE"))
      if (std::atoi(a) == 0) choice = 0;
  }
  if (choice < 0) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) choice = it->second;
  }
  if (choice < 0) {
    // records of the current state
    const double lam0sq = c->cfg.lambda0 * c->cfg.lambda0, four_nu = 4.0 * c->cfg.nu;
    const int* perm = c->far ? c->perm.p : nullptr;
    if (c->far)
      MMVM_CK(mmvm::launch_spatial_order(n, c->x.p, c->order_tmp.p, c->order_tmp.cap, c->perm.p,
                                         c->st));
    MMVM_CK(mmvm::launch_prep(c->cfg.precision, n, c->M, perm, c->x.p, c->m.p, c->t_dev(),
                              nullptr, 0.0, lam0sq, four_nu, c->rec.p,
                              c->far ? c->gbox.p : nullptr, c->st));
    cudaEvent_t e0, e1;
    MMVM_CK(cudaEventCreate(&e0));
    MMVM_CK(cudaEventCreate(&e1));
    // stage 1: every variant on the first kTuneChunks chunks of its own
    // production chunking (many waves of CTAs, so the tail does not decide)
    struct Cand {
      int v, chunks;
      double per_pair;
    };
    std::vector<Cand> cands;
    double best = 1e300;
    for (int v = 0; v < nv; ++v) {
      mmvm::PairEntry e = mmvm::pair_entry(c->M, c->cfg.precision, v);
      if (e.M != c->M) continue;
      if (mmvm::pair_prepare(e, c->S) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      const int per_sm = mmvm::pair_occupancy(e, c->S);
      if (per_sm < 1) continue;
      const int chunks = std::max(1, chunks_for(n, e.tpc, per_sm, c->cfg.device, c->S));
      double per_pair = 0.0;
      MMVM_CK(time_pair_variant(c, e, n, chunks, std::min(chunks, kTuneChunks), e0, e1,
                                &per_pair));
      cands.push_back({v, chunks, per_pair});
      best = std::min(best, per_pair);
    }
    // stage 2: the variants within 10 % of the best, on their full launch
    choice = 0;
    double best_full = 1e300;
    int close = 0;
    for (const Cand& k : cands) close += k.per_pair <= 1.1 * best ? 1 : 0;
    for (const Cand& k : cands) {
      if ((close > 1 || nl > 0) && k.per_pair > 1.1 * best) continue;
      double per_pair = k.per_pair;
      if (close > 1 || nl > 0) {
        mmvm::PairEntry e = mmvm::pair_entry(c->M, c->cfg.precision, k.v);
        MMVM_CK(mmvm::pair_prepare(e, c->S));
        if ((size_t)k.chunks * c->NB * n > c->partial.cap) {
          MMVM_CK(c->partial.ensure((size_t)k.chunks * c->NB * n));
          c->drop_graph();
        }
        MMVM_CK(time_pair_variant(c, e, n, k.chunks, k.chunks, e0, e1, &per_pair));
      }
      if (per_pair < best_full) {
        best_full = per_pair;
        choice = k.v;
      }
    }
    // the list form, every variant on its full launch
    for (int v = 0; v < nl; ++v) {
      mmvm::ListEntry e = mmvm::list_entry(c->M, v);
      if (e.M != c->M) continue;
      if (mmvm::list_prepare(e) != cudaSuccess || mmvm::list_occupancy(e) < 1) {
        cudaGetLastError();
        continue;
      }
      double per_pair = 0.0;
      int rc = time_list_variant(c, e, n, false, e0, e1, &per_pair);
      if (rc) return rc;
      if (per_pair < best_full) {
        best_full = per_pair;
        choice = nv + v;
      }
    }
    // the far field of the best list variant through the tree
    tree_choice = 0;
    if (choice >= nv) {
      mmvm::ListEntry e = mmvm::list_entry(c->M, choice - nv);
      double per_pair = 0.0;
      int rc = time_list_variant(c, e, n, true, e0, e1, &per_pair);
      if (rc) return rc;
      if (per_pair < best_full) {
        best_full = per_pair;
        tree_choice = 1;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = choice;
    g_tuned_tree[key] = tree_choice;
  }
  if (tree_choice < 0) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned_tree.find(key);
    tree_choice = it != g_tuned_tree.end() ? it->second : 1;
  }
  if (const char* f = std::getenv("MMVM_FAR_TREE")) tree_choice = std::atoi(f) != 0;
  if (choice >= nv) {  // list form
    if (choice >= nv + nl) return fail(MMVM_E_INVALID_ARG, "MMVM_PAIR_VARIANT out of range");
    mmvm::ListEntry e = mmvm::list_entry(c->M, choice - nv);
    if (e.M != c->M) return fail(MMVM_E_INVALID_ARG, "MMVM_PAIR_VARIANT out of range");
    MMVM_CK(mmvm::list_prepare(e));
    int lseg = 1, lfar = 1;
    int rc = ensure_list_buffers(c, e, n, &lseg, &lfar);
    if (rc) return rc;
    int tfar = 1;
    const int lc = mmvm::tree_chunk_level((n + mmvm::kGroup - 1) / mmvm::kGroup, lfar, &tfar);
    if (!c->list || e.variant != c->le.variant || lseg != c->lseg || lfar != c->lfar ||
        c->tree != (tree_choice != 0) || lc != c->lc)
      c->drop_graph();
    c->le = e;
    c->list = true;
    c->lseg = lseg;
    c->lfar = lfar;
    c->tree = tree_choice != 0;
    c->lc = lc;
    c->tfar = tfar;
    return MMVM_OK;
  }
  if (c->list) c->drop_graph();
  c->list = false;
  mmvm::PairEntry e = mmvm::pair_entry(c->M, c->cfg.precision, choice);
  if (e.M != c->M) return fail(MMVM_E_INVALID_ARG, "MMVM_PAIR_VARIANT out of range");
  if (e.variant != c->pe.variant || !c->pe.nslices) {
    MMVM_CK(mmvm::pair_prepare(e, c->S));
    c->pe = e;
    c->drop_graph();
  }
  const int ch = choose_chunks(c, n);
  if ((size_t)ch * c->NB * n > c->partial.cap) {
    MMVM_CK(c->partial.ensure((size_t)ch * c->NB * n));
    c->drop_graph();
  }
  if (ch != c->chunks) c->drop_graph();
  c->chunks = ch;
  return MMVM_OK;
}

// The device error flag of the list kernels (a bulk copy not completed
// within the wait limit); call after the context stream is synchronised.
int check_device_flag(mmvm_ctx* c) {
  if (!c->errf.p) return MMVM_OK;
  int h = 0;
  MMVM_CK(cudaMemcpy(&h, c->errf.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    cudaMemset(c->errf.p, 0, sizeof(int));
    return fail(MMVM_E_TIMEOUT, "a shared-memory stage of the all-pairs kernel did not arrive "
                                "within the wait limit; the results of the evaluation are invalid");
  }
  return MMVM_OK;
}

int check_host_state(const mmvm_ctx* c, int64_t n, const double* x, const double* mom) {
  for (int64_t j = 0; j < n; ++j) {
    if (!std::isfinite(x[2 * j]) || !std::isfinite(x[2 * j + 1]))
      return fail(MMVM_E_NUMERIC, "non-finite position at particle " + std::to_string(j));
    for (int k = 0; k < c->K; ++k)
      if (!std::isfinite(mom[j * c->K + k]))
        return fail(MMVM_E_NUMERIC, "non-finite moment at particle " + std::to_string(j));
    if (mom[j * c->K] == 0.0)
      return fail(MMVM_E_ZERO_CIRCULATION,
                  "M[0,0] == 0 at particle " + std::to_string(j) + " (eq:mass)");
  }
  return MMVM_OK;
}

}  // namespace

extern "C" {

const char* mmvm_last_error(void) { return g_err.c_str(); }

const char* mmvm_last_error_string(void) { return g_err.c_str(); }

int32_t mmvm_num_moments(int32_t order) { return order < 0 ? 0 : mmvm::n_moments(order); }

int64_t mmvm_num_particles(const mmvm_ctx* c) { return c ? c->n : 0; }

int64_t mmvm_launch_count(const mmvm_ctx* c) { return c ? c->launches : 0; }

int mmvm_create(const mmvm_config* cfg, mmvm_ctx** out) {
  g_err.clear();
  if (!cfg || !out) return fail(MMVM_E_INVALID_ARG, "null config or output handle");
  *out = nullptr;
  if (cfg->order < 0) return fail(MMVM_E_INVALID_ARG, "order must be >= 0");
  if (cfg->order > MMVM_MAX_ORDER_SINGLE)
    return fail(MMVM_E_UNSUPPORTED, "order above MMVM_MAX_ORDER_SINGLE");
  if (cfg->precision != MMVM_FP64 && cfg->precision != MMVM_MIXED_FP32)
    return fail(MMVM_E_INVALID_ARG, "unknown precision");
  if (!(cfg->lambda0 > 0.0) || !std::isfinite(cfg->lambda0))
    return fail(MMVM_E_INVALID_ARG, "lambda0 must be positive and finite");
  if (!(cfg->nu >= 0.0) || !std::isfinite(cfg->nu))
    return fail(MMVM_E_INVALID_ARG, "nu must be >= 0 and finite");
  if (cfg->flags & ~(MMVM_FLAG_NO_FAR_FIELD | MMVM_FLAG_SEPARABLE_SELF))
    return fail(MMVM_E_INVALID_ARG, "unknown flag bits");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (cfg->device < 0 || cfg->device >= ndev)
    return fail(MMVM_E_INVALID_ARG, "device ordinal out of range");
  e = cudaSetDevice(cfg->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");

  mmvm_ctx* c = new mmvm_ctx();
  c->cfg = *cfg;
  c->far = cfg->precision == MMVM_MIXED_FP32 && !(cfg->flags & MMVM_FLAG_NO_FAR_FIELD);
  c->M = cfg->order;
  c->K = mmvm::n_moments(c->M);
  c->NB = mmvm::n_beta(c->M);
  if (c->M <= MMVM_MAX_ORDER_PAIRS) {
    c->pe = mmvm::pair_entry(c->M, cfg->precision, 0);
    if (c->pe.M != c->M) {
      delete c;
      return fail(MMVM_E_UNSUPPORTED, "pair kernel variant not compiled");
    }
  }
  const int K = c->K;
  c->finish_tb = std::max(1, 128 / (((K + 31) / 32) * 32));
  c->S = mmvm::kGroup;
  auto bail = [&](int rc) {
    mmvm_destroy(c);
    return rc;
  };
  if ((e = cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(cuda_fail(e, "cudaStreamCreate"));
  c->st = c->own;
  // above this order the (k, l, beta) entries are too many: single particles
  // take the separable path, which needs only psi0 and two small tables
  c->high = c->M > kMaxOrderTables || (cfg->flags & MMVM_FLAG_SEPARABLE_SELF);
  mmvm::FinishTables T = mmvm::build_finish_tables(c->M, c->M <= kMaxOrderTables);
  if (c->high) {
    mmvm::SeparableTables ST = mmvm::build_separable_tables(c->M);
    if ((e = c->sbinom.ensure(ST.binom.size())) != cudaSuccess ||
        (e = c->sg.ensure(ST.g.size())) != cudaSuccess ||
        (e = c->scg.ensure(ST.cg.size())) != cudaSuccess ||
        (e = c->sscr.ensure(mmvm::self_high_scratch_doubles(c->M))) != cudaSuccess ||
        (e = cudaMemcpy(c->sbinom.p, ST.binom.data(), ST.binom.size() * sizeof(double),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(c->sg.p, ST.g.data(), ST.g.size() * sizeof(double),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(c->scg.p, ST.cg.data(), ST.cg.size() * sizeof(double),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(cuda_fail(e, "separable tables"));
  }
  if ((e = c->k_off.ensure(T.k_off.size())) != cudaSuccess ||
      (e = c->e_l.ensure(T.e_l.size())) != cudaSuccess ||
      (e = c->e_b.ensure(T.e_b.size())) != cudaSuccess ||
      (e = c->e_c.ensure(T.e_c.size())) != cudaSuccess ||
      (e = c->psi0.ensure(T.psi0.size())) != cudaSuccess ||
      (e = c->scal.ensure(2)) != cudaSuccess || (e = c->flags.ensure(2)) != cudaSuccess ||
      (e = c->counts.ensure(4)) != cudaSuccess)
    return bail(cuda_fail(e, "cudaMalloc(tables)"));
  auto up = [&](void* d, const void* h, size_t bytes) {
    return bytes ? cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
  };
  if ((e = up(c->k_off.p, T.k_off.data(), T.k_off.size() * sizeof(int))) != cudaSuccess ||
      (e = up(c->e_l.p, T.e_l.data(), T.e_l.size() * sizeof(int))) != cudaSuccess ||
      (e = up(c->e_b.p, T.e_b.data(), T.e_b.size() * sizeof(int))) != cudaSuccess ||
      (e = up(c->e_c.p, T.e_c.data(), T.e_c.size() * sizeof(double))) != cudaSuccess ||
      (e = up(c->psi0.p, T.psi0.data(), T.psi0.size() * sizeof(double))) != cudaSuccess ||
      (e = cudaMemset(c->scal.p, 0, 2 * sizeof(double))) != cudaSuccess ||
      (e = cudaMemset(c->counts.p, 0, 4 * sizeof(unsigned long long))) != cudaSuccess)
    return bail(cuda_fail(e, "cudaMemcpy(tables)"));
  if (c->pe.nslices && (e = mmvm::pair_prepare(c->pe, c->S)) != cudaSuccess)
    return bail(cuda_fail(e, "pair kernel shared-memory limit"));
  *out = c;
  return MMVM_OK;
}

void mmvm_destroy(mmvm_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->cfg.device);
  if (c->st) cudaStreamSynchronize(c->st);
  c->drop_graph();
  for (auto& pr : c->ev)
    for (auto& e : pr)
      if (e) cudaEventDestroy(e);
  for (auto& pr : c->evm)
    for (auto& e : pr)
      if (e) cudaEventDestroy(e);
  for (auto* b : {&c->x, &c->m, &c->xs, &c->ms, &c->xsum, &c->msum, &c->rdx, &c->rdm, &c->scal,
                  &c->partial, &c->e_c, &c->psi0, &c->sbinom, &c->sg, &c->scg, &c->sscr, &c->dpts, &c->dval, &c->dring, &c->dk,
                  &c->fpart})
    b->release();
  c->tnodes.release();
  c->lent.release();
  c->lcnt.release();
  c->errf.release();
  c->rec.release();
  c->counts.release();
  c->derr.release();
  c->order_tmp.release();
  c->perm.release();
  c->gbox.release();
  c->flags.release();
  c->k_off.release();
  c->e_l.release();
  c->e_b.release();
  if (c->own) cudaStreamDestroy(c->own);
  delete c;
}

int mmvm_set_stream(mmvm_ctx* c, void* stream) {
  if (!c) return fail(MMVM_E_INVALID_ARG, "null context");
  c->st = stream ? (cudaStream_t)stream : c->own;
  c->drop_graph();
  return MMVM_OK;
}

int mmvm_synchronize(mmvm_ctx* c) {
  if (!c) return fail(MMVM_E_INVALID_ARG, "null context");
  MMVM_CK(cudaSetDevice(c->cfg.device));
  MMVM_CK(cudaStreamSynchronize(c->st));
  return check_device_flag(c);
}

static int set_state_common(mmvm_ctx* c, int64_t n, const double* x, const double* mom,
                            double t, cudaMemcpyKind kind) {
  if (!c || !x || !mom) return fail(MMVM_E_INVALID_ARG, "null argument");
  if (n < 1 || n > (int64_t)1 << 30) return fail(MMVM_E_INVALID_ARG, "n out of range");
  if (!std::isfinite(t)) return fail(MMVM_E_INVALID_ARG, "t must be finite");
  if (n > 1 && c->M > MMVM_MAX_ORDER_PAIRS)
    return fail(MMVM_E_UNSUPPORTED, "order above MMVM_MAX_ORDER_PAIRS for n > 1");
  if (n > 1 && c->high)
    return fail(MMVM_E_UNSUPPORTED, "the separable self-term path serves one particle only");
  if (c->cfg.lambda0 * c->cfg.lambda0 + 4.0 * c->cfg.nu * t <= 0.0)
    return fail(MMVM_E_INVALID_ARG, "lambda(t)^2 <= 0");
  MMVM_CK(cudaSetDevice(c->cfg.device));
  if (kind == cudaMemcpyHostToDevice) {
    int rc = check_host_state(c, n, x, mom);
    if (rc) return rc;
  }
  MMVM_CK(cudaStreamSynchronize(c->st));
  c->n = n;
  int rc = ensure_buffers(c, n);
  if (rc) return rc;
  MMVM_CK(cudaMemcpyAsync(c->x.p, x, sizeof(double) * 2 * n, kind, c->st));
  MMVM_CK(cudaMemcpyAsync(c->m.p, mom, sizeof(double) * c->K * n, kind, c->st));
  static thread_local double t_host;
  t_host = t;
  MMVM_CK(cudaMemcpyAsync(c->t_dev(), &t_host, sizeof(double), cudaMemcpyHostToDevice, c->st));
  rc = tune_pair(c);
  if (rc) return rc;
  MMVM_CK(cudaStreamSynchronize(c->st));
  return MMVM_OK;
}

int mmvm_set_state(mmvm_ctx* c, int64_t n, const double* x, const double* mom, double t) {
  g_err.clear();
  return set_state_common(c, n, x, mom, t, cudaMemcpyHostToDevice);
}

int mmvm_set_state_device(mmvm_ctx* c, int64_t n, const double* x, const double* mom,
                          double t) {
  g_err.clear();
  return set_state_common(c, n, x, mom, t, cudaMemcpyDeviceToDevice);
}

int mmvm_get_state(mmvm_ctx* c, double* x, double* mom, double* t) {
  if (!c) return fail(MMVM_E_INVALID_ARG, "null context");
  if (c->n < 1) return fail(MMVM_E_INVALID_ARG, "no state loaded");
  MMVM_CK(cudaSetDevice(c->cfg.device));
  if (x) MMVM_CK(cudaMemcpyAsync(x, c->x.p, sizeof(double) * 2 * c->n, cudaMemcpyDeviceToHost, c->st));
  if (mom)
    MMVM_CK(cudaMemcpyAsync(mom, c->m.p, sizeof(double) * c->K * c->n, cudaMemcpyDeviceToHost, c->st));
  if (t) MMVM_CK(cudaMemcpyAsync(t, c->t_dev(), sizeof(double), cudaMemcpyDeviceToHost, c->st));
  MMVM_CK(cudaStreamSynchronize(c->st));
  return check_device_flag(c);
}

int mmvm_get_state_device(mmvm_ctx* c, double* d_x, double* d_mom) {
  if (!c || !d_x || !d_mom) return fail(MMVM_E_INVALID_ARG, "null argument");
  if (c->n < 1) return fail(MMVM_E_INVALID_ARG, "no state loaded");
  MMVM_CK(cudaSetDevice(c->cfg.device));
  MMVM_CK(cudaMemcpyAsync(d_x, c->x.p, sizeof(double) * 2 * c->n, cudaMemcpyDeviceToDevice, c->st));
  MMVM_CK(cudaMemcpyAsync(d_mom, c->m.p, sizeof(double) * c->K * c->n, cudaMemcpyDeviceToDevice, c->st));
  return MMVM_OK;
}

int mmvm_rhs_device(mmvm_ctx* c, double* d_dx, double* d_dM) {
  if (!c || !d_dx || !d_dM) return fail(MMVM_E_INVALID_ARG, "null argument");
  if (c->n < 1) return fail(MMVM_E_INVALID_ARG, "no state loaded");
  MMVM_CK(cudaSetDevice(c->cfg.device));
  int rc = enqueue_rhs(c, 0, c->x.p, c->m.p, 0.0, nullptr);
  if (rc) return rc;
  MMVM_CK(cudaMemcpyAsync(d_dx, c->rdx.p, sizeof(double) * 2 * c->n, cudaMemcpyDeviceToDevice, c->st));
  MMVM_CK(cudaMemcpyAsync(d_dM, c->rdm.p, sizeof(double) * c->K * c->n, cudaMemcpyDeviceToDevice, c->st));
  return MMVM_OK;
}

int mmvm_rhs(mmvm_ctx* c, double* dx, double* dM) {
  if (!c || !dx || !dM) return fail(MMVM_E_INVALID_ARG, "null argument");
  if (c->n < 1) return fail(MMVM_E_INVALID_ARG, "no state loaded");
  MMVM_CK(cudaSetDevice(c->cfg.device));
  int rc = enqueue_rhs(c, 0, c->x.p, c->m.p, 0.0, nullptr);
  if (rc) return rc;
  MMVM_CK(cudaMemcpyAsync(dx, c->rdx.p, sizeof(double) * 2 * c->n, cudaMemcpyDeviceToHost, c->st));
  MMVM_CK(cudaMemcpyAsync(dM, c->rdm.p, sizeof(double) * c->K * c->n, cudaMemcpyDeviceToHost, c->st));
  MMVM_CK(cudaStreamSynchronize(c->st));
  return check_device_flag(c);
}

int mmvm_step(mmvm_ctx* c, double dt, int64_t nsteps) {
  if (!c) return fail(MMVM_E_INVALID_ARG, "null context");
  if (c->n < 1) return fail(MMVM_E_INVALID_ARG, "no state loaded");
  if (!std::isfinite(dt) || nsteps < 0) return fail(MMVM_E_INVALID_ARG, "bad dt or nsteps");
  if (nsteps == 0) return MMVM_OK;
  MMVM_CK(cudaSetDevice(c->cfg.device));
  if (!(dt == c->last_dt)) {
    static thread_local double dt_host;
    dt_host = dt;
    MMVM_CK(cudaMemcpyAsync(c->dt_dev(), &dt_host, sizeof(double), cudaMemcpyHostToDevice, c->st));
    MMVM_CK(cudaStreamSynchronize(c->st));
    c->last_dt = dt;
  }
  if (c->timing) {
    // Timed steps are launched directly (events captured inside a graph
    // cannot be read back for elapsed time); the kernels are the same.
    for (int64_t s = 0; s < nsteps; ++s) {
      int rc = enqueue_step(c);
      if (rc) return rc;
    }
    return MMVM_OK;
  }
  if (!c->graph_ok) {
    MMVM_CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
    const int64_t before = c->launches;
    int rc = enqueue_step(c);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->st, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    c->launches = before;  // captured launches are counted on replay
    c->graph = g;
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    if (e != cudaSuccess) {
      c->drop_graph();
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    c->graph_ok = true;
  }
  const int per_step =
      (c->n > 1 ? 4 * ((c->far ? 2 : 1) + pair_launches(c) + 1) + (c->far ? c->order_launches : 0)
                : (c->high ? 20 : 4)) +
      1;
  for (int64_t s = 0; s < nsteps; ++s) {
    MMVM_CK(cudaGraphLaunch(c->gexec, c->st));
    c->launches += per_step;
  }
  return MMVM_OK;
}

int mmvm_integrate(mmvm_ctx* c, double t_end, double h0, double rtol, double atol,
                   int64_t max_steps, int64_t* accepted, int64_t* rejected) {
  // Dormand-Prince 5(4): nodes, stage weights, 5th-order weights minus 4th-order
  static const double kC[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
  static const double kA[7][6] = {
      {0, 0, 0, 0, 0, 0},
      {1.0 / 5, 0, 0, 0, 0, 0},
      {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
      {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
      {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
      {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
      {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
  static const double kB5[7] = {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784,
                                11.0 / 84, 0.0};
  static const double kB4[7] = {5179.0 / 57600, 0.0, 7571.0 / 16695, 393.0 / 640,
                                -92097.0 / 339200, 187.0 / 2100, 1.0 / 40};
  if (!c) return fail(MMVM_E_INVALID_ARG, "null context");
  if (c->n < 1) return fail(MMVM_E_INVALID_ARG, "no state loaded");
  if (!std::isfinite(t_end) || !(h0 > 0.0) || !std::isfinite(h0) || !(rtol >= 0.0) ||
      !(atol >= 0.0) || !(rtol + atol > 0.0) || max_steps < 1)
    return fail(MMVM_E_INVALID_ARG, "bad t_end, h0, tolerances or max_steps");
  int64_t acc_n = 0, rej_n = 0;
  if (accepted) *accepted = 0;
  if (rejected) *rejected = 0;
  MMVM_CK(cudaSetDevice(c->cfg.device));
  double t = 0.0;
  MMVM_CK(cudaMemcpyAsync(&t, c->t_dev(), sizeof(double), cudaMemcpyDeviceToHost, c->st));
  MMVM_CK(cudaStreamSynchronize(c->st));
  if (t_end < t) return fail(MMVM_E_INVALID_ARG, "t_end before the current time");
  if (t_end == t) return MMVM_OK;
  if (c->cfg.lambda0 * c->cfg.lambda0 + 4.0 * c->cfg.nu * t_end <= 0.0)
    return fail(MMVM_E_INVALID_ARG, "lambda(t_end)^2 <= 0");
  const int n = (int)c->n, K = c->K;
  const size_t L = (size_t)n * (2 + K);
  MMVM_CK(c->dk.ensure(7 * L));
  MMVM_CK(c->derr.ensure(1));
  c->last_dt = NAN;  // dt_dev holds the step size from here on
  double* dt = c->dt_dev();
  auto kx = [&](int s) { return c->dk.p + s * L; };
  auto km = [&](int s) { return c->dk.p + s * L + 2 * (size_t)n; };
  static thread_local double h_host;
  double h = h0;
  h_host = h;
  MMVM_CK(cudaMemcpyAsync(dt, &h_host, sizeof(double), cudaMemcpyHostToDevice, c->st));
  int rc = enqueue_rhs(c, 0, c->x.p, c->m.p, 0.0, dt, kx(0), km(0));  // k1 = f(t, y)
  if (rc) return rc;
  while (t < t_end && acc_n + rej_n < max_steps) {
    const bool last = t + h >= t_end;
    if (last) h = t_end - t;
    h_host = h;
    MMVM_CK(cudaMemcpyAsync(dt, &h_host, sizeof(double), cudaMemcpyHostToDevice, c->st));
    for (int s = 1; s < 7; ++s) {
      mmvm::DPCoef co{};
      for (int j = 0; j < s; ++j) co.w[j] = kA[s][j];
      co.count = s;
      double* ox = s == 6 ? c->xsum.p : c->xs.p;  // stage 7 is the 5th-order solution
      double* om = s == 6 ? c->msum.p : c->ms.p;
      MMVM_CK(mmvm::launch_dp_combine(n, K, c->x.p, c->m.p, c->dk.p, co, dt, ox, om, c->st));
      if ((rc = enqueue_rhs(c, 0, ox, om, kC[s], dt, kx(s), km(s)))) return rc;
      c->launches += 1;
    }
    mmvm::DPCoef ec{};
    for (int j = 0; j < 7; ++j) ec.w[j] = kB5[j] - kB4[j];
    ec.count = 7;
    MMVM_CK(mmvm::launch_dp_error(n, K, c->x.p, c->m.p, c->xsum.p, c->msum.p, c->dk.p, ec, dt,
                                  rtol, atol, c->derr.p, c->st));
    unsigned long long bits = 0;
    MMVM_CK(cudaMemcpyAsync(&bits, c->derr.p, sizeof(bits), cudaMemcpyDeviceToHost, c->st));
    MMVM_CK(cudaStreamSynchronize(c->st));
    c->launches += 1;
    double err;
    std::memcpy(&err, &bits, sizeof(err));
    if (!std::isfinite(err)) {
      if (accepted) *accepted = acc_n;
      if (rejected) *rejected = rej_n;
      return fail(MMVM_E_NUMERIC, "non-finite error estimate at t = " + std::to_string(t));
    }
    const double fac = err > 0.0 ? 0.9 * std::pow(err, -0.2) : 5.0;
    if (err <= 1.0) {
      MMVM_CK(cudaMemcpyAsync(c->x.p, c->xsum.p, 2 * (size_t)n * sizeof(double),
                              cudaMemcpyDeviceToDevice, c->st));
      MMVM_CK(cudaMemcpyAsync(c->m.p, c->msum.p, (size_t)K * n * sizeof(double),
                              cudaMemcpyDeviceToDevice, c->st));
      MMVM_CK(cudaMemcpyAsync(kx(0), kx(6), L * sizeof(double), cudaMemcpyDeviceToDevice,
                              c->st));  // first same as last
      if (last) {
        t = t_end;
        static thread_local double t_host;
        t_host = t;
        MMVM_CK(cudaMemcpyAsync(c->t_dev(), &t_host, sizeof(double), cudaMemcpyHostToDevice,
                                c->st));
        MMVM_CK(cudaStreamSynchronize(c->st));
      } else {
        t = t + h;  // the device adds the same two doubles
        MMVM_CK(mmvm::launch_advance_time(c->t_dev(), dt, c->st));
        c->launches += 1;
      }
      ++acc_n;
      h = h * std::min(5.0, std::max(0.2, fac));
    } else {
      ++rej_n;
      h = h * std::min(1.0, std::max(0.2, fac));
    }
  }
  MMVM_CK(cudaStreamSynchronize(c->st));
  if (accepted) *accepted = acc_n;
  if (rejected) *rejected = rej_n;
  if (t < t_end)
    return fail(MMVM_E_TIMEOUT, "step limit reached at t = " + std::to_string(t));
  return MMVM_OK;
}

int mmvm_vorticity(mmvm_ctx* c, int64_t npts, const double* pts, double* omega) {
  if (!c || (npts > 0 && (!pts || !omega))) return fail(MMVM_E_INVALID_ARG, "null argument");
  if (npts < 0 || npts > (int64_t)1 << 28) return fail(MMVM_E_INVALID_ARG, "npts out of range");
  if (c->n < 1) return fail(MMVM_E_INVALID_ARG, "no state loaded");
  if (c->M > mmvm::diag_max_order())
    return fail(MMVM_E_UNSUPPORTED, "order above the diagnostics limit (64)");
  if (npts == 0) return MMVM_OK;
  MMVM_CK(cudaSetDevice(c->cfg.device));
  MMVM_CK(c->dpts.ensure(2 * (size_t)npts));
  MMVM_CK(c->dval.ensure((size_t)npts));
  MMVM_CK(cudaMemcpyAsync(c->dpts.p, pts, 2 * (size_t)npts * sizeof(double),
                          cudaMemcpyHostToDevice, c->st));
  MMVM_CK(mmvm::launch_vorticity((int)c->n, c->M, c->x.p, c->m.p, c->t_dev(),
                                 c->cfg.lambda0 * c->cfg.lambda0, 4.0 * c->cfg.nu, (int)npts,
                                 c->dpts.p, c->dval.p, c->st));
  MMVM_CK(cudaMemcpyAsync(omega, c->dval.p, (size_t)npts * sizeof(double),
                          cudaMemcpyDeviceToHost, c->st));
  MMVM_CK(cudaStreamSynchronize(c->st));
  c->launches += 1;
  return MMVM_OK;
}

int mmvm_nonaxi_enstrophy(mmvm_ctx* c, double cx, double cy, double r_max, int32_t nr,
                          int32_t ntheta, double* E) {
  if (!c || !E) return fail(MMVM_E_INVALID_ARG, "null argument");
  if (!(r_max > 0.0) || !std::isfinite(r_max) || !std::isfinite(cx) || !std::isfinite(cy) ||
      nr < 1 || nr > 4096 || ntheta < 4 || ntheta > 65536)
    return fail(MMVM_E_INVALID_ARG, "bad polar grid");
  if (c->n < 1) return fail(MMVM_E_INVALID_ARG, "no state loaded");
  if (c->M > mmvm::diag_max_order())
    return fail(MMVM_E_UNSUPPORTED, "order above the diagnostics limit (64)");
  std::vector<double> xg, wg;
  mmvm::gauss_legendre(nr, xg, wg);
  const size_t np = (size_t)nr * ntheta;
  std::vector<double> pts(2 * np);
  const double two_pi = 6.28318530717958647692;
  for (int i = 0; i < nr; ++i) {
    const double r = 0.5 * r_max * (xg[i] + 1.0);
    for (int l = 0; l < ntheta; ++l) {
      const double th = two_pi * l / ntheta;
      pts[2 * ((size_t)i * ntheta + l)] = cx + r * std::cos(th);
      pts[2 * ((size_t)i * ntheta + l) + 1] = cy + r * std::sin(th);
    }
  }
  MMVM_CK(cudaSetDevice(c->cfg.device));
  MMVM_CK(c->dpts.ensure(2 * np));
  MMVM_CK(c->dval.ensure(np));
  MMVM_CK(c->dring.ensure((size_t)nr));
  MMVM_CK(cudaMemcpyAsync(c->dpts.p, pts.data(), 2 * np * sizeof(double), cudaMemcpyHostToDevice,
                          c->st));
  MMVM_CK(mmvm::launch_vorticity((int)c->n, c->M, c->x.p, c->m.p, c->t_dev(),
                                 c->cfg.lambda0 * c->cfg.lambda0, 4.0 * c->cfg.nu, (int)np,
                                 c->dpts.p, c->dval.p, c->st));
  MMVM_CK(mmvm::launch_ring_deviation(nr, ntheta, c->dval.p, c->dring.p, c->st));
  std::vector<double> ring(nr);
  MMVM_CK(cudaMemcpyAsync(ring.data(), c->dring.p, nr * sizeof(double), cudaMemcpyDeviceToHost,
                          c->st));
  MMVM_CK(cudaStreamSynchronize(c->st));
  c->launches += 2;
  double e = 0.0;  // sum over rings of (r dr weight) x (angle sum) x (2 pi / ntheta)
  for (int i = 0; i < nr; ++i) {
    const double r = 0.5 * r_max * (xg[i] + 1.0);
    e += 0.5 * r_max * wg[i] * r * ring[i];
  }
  *E = e * two_pi / ntheta;
  return MMVM_OK;
}

int mmvm_pair_work(mmvm_ctx* c, int64_t* out) {
  if (!c || !out) return fail(MMVM_E_INVALID_ARG, "null argument");
  MMVM_CK(cudaSetDevice(c->cfg.device));
  unsigned long long h[4] = {0, 0, 0, 0};
  MMVM_CK(cudaMemcpyAsync(h, c->counts.p, sizeof(h), cudaMemcpyDeviceToHost, c->st));
  MMVM_CK(cudaStreamSynchronize(c->st));
  for (int i = 0; i < 4; ++i) out[i] = (int64_t)h[i];
  return MMVM_OK;
}

int mmvm_pair_counts(mmvm_ctx* c, int64_t* near_pairs, int64_t* far_pairs) {
  if (!near_pairs || !far_pairs) return fail(MMVM_E_INVALID_ARG, "null argument");
  int64_t w[4];
  const int rc = mmvm_pair_work(c, w);
  if (rc) return rc;
  *near_pairs = w[0];
  *far_pairs = w[1] + w[3];
  return MMVM_OK;
}

int mmvm_pair_variant_counts(int32_t order, int32_t precision, int32_t* direct, int32_t* list) {
  if (!direct || !list) return fail(MMVM_E_INVALID_ARG, "null argument");
  if (order < 0 || order > MMVM_MAX_ORDER_PAIRS ||
      (precision != MMVM_FP64 && precision != MMVM_MIXED_FP32))
    return fail(MMVM_E_INVALID_ARG, "order or precision out of range");
  *direct = mmvm::pair_variant_count(order, precision);
  *list = precision == MMVM_MIXED_FP32 ? mmvm::list_variant_count(order) : 0;
  return MMVM_OK;
}

int mmvm_pair_config(const mmvm_ctx* c, int32_t* out) {
  if (!c || !out) return fail(MMVM_E_INVALID_ARG, "null argument");
  if (c->list) {
    out[0] = mmvm::pair_variant_count(c->M, c->cfg.precision) + c->le.variant;
    out[1] = c->le.nslices + 2;
    out[2] = c->le.slices[0].warps * 32;
    out[3] = mmvm::list_occupancy(c->le);
    out[4] = 1;
    out[5] = c->lseg;
    out[6] = c->tree ? 2 : 1;
    out[7] = c->tree ? c->tfar : c->lfar;
    return MMVM_OK;
  }
  out[0] = c->pe.variant;
  out[1] = c->pe.nslices;
  out[2] = c->pe.tpc;
  out[3] = c->pe.minb;
  out[4] = c->pe.sync;
  out[5] = c->chunks;
  out[6] = 0;
  out[7] = 0;
  return MMVM_OK;
}

int mmvm_enable_timing(mmvm_ctx* c, int on) {
  if (!c) return fail(MMVM_E_INVALID_ARG, "null context");
  MMVM_CK(cudaSetDevice(c->cfg.device));
  if (on && !c->ev[0][0]) {
    for (auto& pr : c->ev)
      for (auto& e : pr) MMVM_CK(cudaEventCreate(&e));
    for (auto& pr : c->evm)
      for (auto& e : pr) MMVM_CK(cudaEventCreate(&e));
  }
  if (c->timing != (on != 0)) c->drop_graph();  // re-capture with or without events
  c->timing = on != 0;
  for (bool& p : c->ev_pending) p = false;
  for (bool& p : c->evm_pending) p = false;
  return MMVM_OK;
}

int mmvm_pair_time(mmvm_ctx* c, double* ms, int64_t* count) {
  if (!c || !ms || !count) return fail(MMVM_E_INVALID_ARG, "null argument");
  *ms = 0.0;
  *count = 0;
  if (!c->timing) return MMVM_OK;
  MMVM_CK(cudaSetDevice(c->cfg.device));
  MMVM_CK(cudaStreamSynchronize(c->st));
  for (int s = 0; s < 5; ++s) {
    if (!c->ev_pending[s]) continue;
    float e = 0.f;
    MMVM_CK(cudaEventElapsedTime(&e, c->ev[s][0], c->ev[s][1]));
    *ms += e;
    *count += 1;
    c->ev_pending[s] = false;
    if (c->evm_pending[s] && c->list) {
      cudaEvent_t prev = c->ev[s][0];
      for (int k = 0; k < 2 + c->le.nslices; ++k) {
        float p = 0.f;
        MMVM_CK(cudaEventElapsedTime(&p, prev, c->evm[s][k]));
        c->parts_ms[k] += p;
        prev = c->evm[s][k];
      }
      c->parts_count += 1;
    }
    c->evm_pending[s] = false;
  }
  return MMVM_OK;
}

int mmvm_pair_time_parts(mmvm_ctx* c, double* ms, int32_t max_parts, int32_t* nparts,
                         int64_t* count) {
  if (!c || !ms || !nparts || !count) return fail(MMVM_E_INVALID_ARG, "null argument");
  const int np = c->list ? 2 + c->le.nslices : 0;
  *nparts = np;
  *count = c->parts_count;
  for (int k = 0; k < std::min<int>(np, max_parts); ++k) ms[k] = c->parts_ms[k];
  for (double& v : c->parts_ms) v = 0.0;
  c->parts_count = 0;
  return MMVM_OK;
}

}  // extern "C"
