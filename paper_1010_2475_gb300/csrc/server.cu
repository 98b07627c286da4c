// Serving: one request loop runs many independent MMVM simulations (different
// particle counts, orders, viscosities, core sizes, step sizes and step
// counts) on one GPU at once.
//
// * Continuous batching.  Requests wait in a FIFO queue and are admitted
//   while their device footprint (state, source records, partial sums, work
//   lists) fits the server's HBM budget; admitted state stays resident on the
//   device until the simulation ends, and a finished simulation frees its
//   footprint for the next request at once.
// * Batches.  Admitted simulations of one order and one size class (n up to
//   256, 1024, 4096, larger) form a batch: its records, partials and work
//   lists live in buffers of the batch, and one tick of the batch is one RK4
//   step of all its simulations: per stage three launches for the whole batch
//   (records; the persistent all-pairs kernel working through a list of
//   (simulation, target tile, source chunk) items; the FP64 finish), then the
//   time advance and a divergence scan.  A tick is a CUDA graph, captured
//   once and replayed; the kernels read the sizes of the batch from device
//   memory, so a change of members only re-uploads the work lists.
// * Batches tick independently, each on its own stream: a cheap batch (low
//   order, small n) is not held back by an expensive one, and the GPU runs
//   the ticks of different batches at the same time.  Members join and leave
//   a batch between its ticks.
// * The split of a simulation's pairs into items and its spatial order
//   depend on its own state only, and every item is summed in a fixed order,
//   so a simulation's result does not depend on the rest of its batch.
// * FP32 batches use the far-field path of the all-pairs kernel, with a
//   Morton order of each simulation's centres in its own bounding box.
// * The all-pairs variant of each order is chosen once per process by timing
//   every compiled variant on the first batch of that order.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/mmvm.h"
#include "common.cuh"
#include "pair_registry.h"
#include "particle_kernels.h"
#include "tables.h"

namespace mmvm {
void set_last_error(const char* msg);
}

namespace {

using Clock = std::chrono::steady_clock;
using mmvm::BatchInst;
using mmvm::kGroup;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

int fail(int code, const std::string& m) {
  mmvm::set_last_error(m.c_str());
  return code;
}

constexpr int kMaxOrderServed = 16;  // the batched finish uses the (k, l, beta) tables
constexpr int kChunkTarget = 1024;   // sources per chunk (items of similar cost)
constexpr int kMaxChunks = 16;
constexpr int kStages = 4;
constexpr int kCountHdr = 4;  // n_slots, n_pair_items, n_finish_items, n_inst
constexpr int kCounters = kStages * mmvm::kMaxSlices;

int chunks_for(int64_t n) {
  if (n <= 1) return 0;
  return (int)std::min<int64_t>((n + kChunkTarget - 1) / kChunkTarget, kMaxChunks);
}

int chunk_len_for(int64_t n, int chunks) {
  return mmvm::round_up((int)((n + chunks - 1) / chunks), kGroup);
}

int finish_tb(int K) { return std::max(1, 128 / (((K + 31) / 32) * 32)); }

int size_class(int64_t n) { return n <= 256 ? 0 : n <= 1024 ? 1 : n <= 4096 ? 2 : 3; }

size_t rec_bytes(int M, int precision) {
  return precision == MMVM_MIXED_FP32 ? (size_t)mmvm::rec_len<float>(M) * 4
                                      : (size_t)mmvm::rec_len<double>(M) * 8;
}

// Device bytes one simulation holds while admitted.
uint64_t footprint(int M, int precision, int64_t n) {
  const int K = mmvm::n_moments(M), NB = mmvm::n_beta(M);
  const uint64_t slots = (uint64_t)mmvm::round_up((int)n, kGroup);
  const uint64_t state = 6ull * n * (2 + K) * 8;
  const uint64_t recs = slots * rec_bytes(M, precision);
  const uint64_t part = (uint64_t)chunks_for(n) * NB * n * 8;
  const uint64_t items = (slots / 32 + 1) * (uint64_t)std::max(chunks_for(n), 1) * 16 +
                         (uint64_t)n * 8 + slots / kGroup * 4 + sizeof(BatchInst);
  // spatial order and far field of FP32 batches: sorted index, keys and
  // values twice, group records, the simulation's box
  const uint64_t order = precision == MMVM_MIXED_FP32
                             ? slots * 28 + slots / kGroup * 4 * mmvm::gdata_len(M) + 32
                             : 0;
  return state + recs + part + items + order;
}

template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t cap = 0;
  // at least n elements (contents are not kept); *grown is set on reallocation
  cudaError_t ensure(size_t n, bool* grown) {
    if (p && n <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t want = std::max<size_t>(n + n / 4, 64);
    cudaError_t e = cudaMalloc(&p, want * sizeof(T));
    if (e == cudaSuccess) cap = want;
    *grown = true;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

struct Request {
  uint64_t ticket = 0;
  int order = 0;
  int64_t n = 0;
  double lam0 = 0, nu = 0, t0 = 0, dt = 0;
  int64_t nsteps = 0;
  std::vector<double> x, m;  // the input, then the result
  int status = MMVM_PENDING;
  std::string err;
  int64_t steps_done = 0;
  double t = 0;
  uint64_t fp = 0;
  Clock::time_point t_submit, t_admit, t_done;
  double* d_state = nullptr;  // worker thread only
};

// Every admitted simulation of one order and size class.
struct Batch {
  int M = 0, K = 0, NB = 0, tb = 1;
  mmvm::PairEntry pe;  // pe.M == -1: no pair kernel (orders above the pair limit: n == 1 only)
  bool far = false;
  std::vector<Request*> members;   // in the work lists
  std::vector<Request*> incoming;  // admitted, state on its way, joining at the next tick
  bool dirty = true;
  bool tuned = false;
  DBuf<int> k_off, e_l, e_b;
  DBuf<double> e_c, psi0;
  DBuf<unsigned char> rec;
  DBuf<double> partial;
  DBuf<BatchInst> inst;
  DBuf<int> slot_inst;
  DBuf<int4> pitems;
  DBuf<int2> fitems;
  DBuf<int> counts;  // kCountHdr sizes, then the item counters
  DBuf<int> bad;     // per simulation: non-finite state after the tick
  DBuf<float> gbox;  // far field: group records (gdata_len(M) floats per kGroup slots)
  DBuf<int> perm, iin, iout;
  DBuf<unsigned long long> kin, kout;
  DBuf<double> ibox;
  DBuf<unsigned char> sort_tmp;
  std::vector<int> bad_host;
  int slot_cap = 0;  // slots every slot-sized buffer holds
  int inst_cap = 0;  // simulations every per-simulation buffer holds
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr, ev0 = nullptr, ev1 = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graph_valid = false;
  bool in_flight = false;
  int grid = 1;               // persistent CTAs of the pair kernel
  int64_t pairs_per_rhs = 0;  // sum of n^2 over the members
  void release() {
    for (auto* b : {&k_off, &e_l, &e_b, &slot_inst, &counts, &bad, &perm, &iin, &iout})
      b->release();
    e_c.release();
    psi0.release();
    rec.release();
    partial.release();
    inst.release();
    pitems.release();
    fitems.release();
    gbox.release();
    kin.release();
    kout.release();
    ibox.release();
    sort_tmp.release();
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    for (cudaEvent_t* ev : {&done, &ev0, &ev1})
      if (*ev) cudaEventDestroy(*ev);
    done = ev0 = ev1 = nullptr;
    if (st) cudaStreamDestroy(st);
    st = nullptr;
  }
};

std::mutex g_batch_tune_mu;
std::map<std::tuple<int, int, int>, int> g_batch_tuned;  // (device, order, precision) -> variant

}  // namespace

struct mmvm_server {
  mmvm_server_config cfg{};
  uint64_t budget = 0;
  int sms = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  bool broken = false;
  std::string broken_msg;
  uint64_t fp_used = 0, fp_peak = 0;
  int64_t n_active = 0, submitted = 0, completed = 0, failed = 0, ticks = 0, max_batch = 0;
  int64_t max_active = 0;
  double pair_interactions = 0, busy_ms = 0;
  std::thread worker;
  // worker-thread state
  cudaStream_t up = nullptr;       // uploads of admitted state
  cudaEvent_t up_done = nullptr;   // after the latest upload
  std::map<int, Batch> batches;    // key: order * 4 + size class
  int in_flight = 0;
  Clock::time_point busy_since;
};

namespace {

void finish_request(mmvm_server* s, Request* r, int status, const std::string& err) {
  // caller holds s->mu
  r->status = status;
  r->err = err;
  r->t_done = Clock::now();
  s->fp_used -= r->fp;
  s->n_active -= 1;
  if (status == MMVM_OK)
    s->completed += 1;
  else
    s->failed += 1;
}

cudaError_t upload_tables(Batch& b) {
  mmvm::FinishTables T = mmvm::build_finish_tables(b.M);
  bool g = false;
  cudaError_t e;
  if ((e = b.k_off.ensure(T.k_off.size(), &g)) != cudaSuccess ||
      (e = b.e_l.ensure(std::max<size_t>(T.e_l.size(), 1), &g)) != cudaSuccess ||
      (e = b.e_b.ensure(std::max<size_t>(T.e_b.size(), 1), &g)) != cudaSuccess ||
      (e = b.e_c.ensure(std::max<size_t>(T.e_c.size(), 1), &g)) != cudaSuccess ||
      (e = b.psi0.ensure(T.psi0.size(), &g)) != cudaSuccess)
    return e;
  auto up = [&](void* d, const void* h, size_t bytes) {
    return bytes ? cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, b.st) : cudaSuccess;
  };
  if ((e = up(b.k_off.p, T.k_off.data(), T.k_off.size() * sizeof(int))) != cudaSuccess ||
      (e = up(b.e_l.p, T.e_l.data(), T.e_l.size() * sizeof(int))) != cudaSuccess ||
      (e = up(b.e_b.p, T.e_b.data(), T.e_b.size() * sizeof(int))) != cudaSuccess ||
      (e = up(b.e_c.p, T.e_c.data(), T.e_c.size() * sizeof(double))) != cudaSuccess ||
      (e = up(b.psi0.p, T.psi0.data(), T.psi0.size() * sizeof(double))) != cudaSuccess)
    return e;
  return cudaStreamSynchronize(b.st);  // the host tables go out of scope
}

// Grow every slot-sized and per-simulation buffer to hold `slots` slots and
// `ninst` simulations (with room to spare).
cudaError_t ensure_caps(Batch& b, int slots, int ninst, bool* grown) {
  cudaError_t e = cudaSuccess;
  const int eb = b.pe.M >= 0 ? b.pe.elem_bytes : 8;
  const int R = b.pe.M >= 0 ? b.pe.rec_len : mmvm::rec_len<double>(b.M);
  if (slots > b.slot_cap || !b.rec.p) {
    const int cap = mmvm::round_up(std::max(slots + slots / 4, kGroup), kGroup);
    bool g = false;
    if ((e = b.rec.ensure((size_t)cap * R * eb, &g)) != cudaSuccess ||
        (e = b.slot_inst.ensure(cap / kGroup, &g)) != cudaSuccess)
      return e;
    if (b.far) {
      const size_t sb = mmvm::batch_order_temp_bytes(cap);
      if ((e = b.gbox.ensure((size_t)mmvm::gdata_len(b.M) * (cap / kGroup), &g)) != cudaSuccess ||
          (e = b.perm.ensure(cap, &g)) != cudaSuccess ||
          (e = b.iin.ensure(cap, &g)) != cudaSuccess ||
          (e = b.iout.ensure(cap, &g)) != cudaSuccess ||
          (e = b.kin.ensure(cap, &g)) != cudaSuccess ||
          (e = b.kout.ensure(cap, &g)) != cudaSuccess ||
          (e = b.sort_tmp.ensure(sb, &g)) != cudaSuccess)
        return e;
    }
    b.slot_cap = cap;
    *grown = true;
  }
  if (ninst > b.inst_cap || !b.inst.p) {
    const int cap = std::max(ninst + ninst / 4, 8);
    bool g = false;
    if ((e = b.inst.ensure(cap, &g)) != cudaSuccess || (e = b.bad.ensure(cap, &g)) != cudaSuccess)
      return e;
    if (b.far && (e = b.ibox.ensure((size_t)4 * cap, &g)) != cudaSuccess) return e;
    b.inst_cap = cap;
    *grown = true;
  }
  return e;
}

// Work lists and descriptors of a batch for its current members.
cudaError_t rebuild(Batch& b, bool* grown) {
  std::vector<BatchInst> inst;
  std::vector<int> slot_inst;
  std::vector<std::pair<int64_t, int4>> pit;
  std::vector<int2> fit;
  int slots = 0;
  long long part = 0;
  b.pairs_per_rhs = 0;
  const int tpc = b.pe.M >= 0 ? b.pe.tpc : 0;
  for (size_t i = 0; i < b.members.size(); ++i) {
    Request* r = b.members[i];
    const int n = (int)r->n;
    BatchInst I{};
    I.state = r->d_state;
    I.n = n;
    I.slot0 = slots;
    I.chunks = chunks_for(n);
    I.chunk_len = I.chunks ? chunk_len_for(n, I.chunks) : 0;
    I.part_off = part;
    I.lam0sq = r->lam0 * r->lam0;
    I.four_nu = 4.0 * r->nu;
    I.t = r->t;
    I.dt = r->dt;
    inst.push_back(I);
    const int nsl = mmvm::round_up(n, kGroup);
    for (int g = 0; g < nsl / kGroup; ++g) slot_inst.push_back((int)i);
    slots += nsl;
    part += (long long)I.chunks * b.NB * n;
    b.pairs_per_rhs += (int64_t)n * n;
    if (n > 1 && tpc > 0) {
      for (int t0 = 0; t0 < n; t0 += tpc)
        for (int ch = 0; ch < I.chunks; ++ch) {
          const int c0 = ch * I.chunk_len, c1 = std::min(n, c0 + I.chunk_len);
          const int64_t cost = (int64_t)std::min(tpc, n - t0) * std::max(0, c1 - c0);
          pit.push_back({cost, make_int4((int)i, t0, ch, 0)});
        }
    }
    for (int f = 0; f < n; f += b.tb) fit.push_back(make_int2((int)i, f));
  }
  // costliest items first, so the persistent CTAs finish together
  std::stable_sort(pit.begin(), pit.end(),
                   [](const std::pair<int64_t, int4>& a, const std::pair<int64_t, int4>& c) {
                     return a.first > c.first;
                   });
  std::vector<int4> pitems(pit.size());
  for (size_t i = 0; i < pit.size(); ++i) pitems[i] = pit[i].second;
  cudaError_t e;
  if ((e = ensure_caps(b, slots, (int)inst.size(), grown)) != cudaSuccess ||
      (e = b.partial.ensure((size_t)std::max<long long>(part, 1), grown)) != cudaSuccess ||
      (e = b.pitems.ensure(std::max<size_t>(pitems.size(), 1), grown)) != cudaSuccess ||
      (e = b.fitems.ensure(std::max<size_t>(fit.size(), 1), grown)) != cudaSuccess ||
      (e = b.counts.ensure(kCountHdr + kCounters, grown)) != cudaSuccess)
    return e;
  const int hdr[kCountHdr] = {slots, (int)pitems.size(), (int)fit.size(), (int)inst.size()};
  auto up = [&](void* d, const void* h, size_t bytes) {
    return bytes ? cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, b.st) : cudaSuccess;
  };
  if ((e = up(b.inst.p, inst.data(), inst.size() * sizeof(BatchInst))) != cudaSuccess ||
      (e = up(b.slot_inst.p, slot_inst.data(), slot_inst.size() * sizeof(int))) != cudaSuccess ||
      (e = up(b.pitems.p, pitems.data(), pitems.size() * sizeof(int4))) != cudaSuccess ||
      (e = up(b.fitems.p, fit.data(), fit.size() * sizeof(int2))) != cudaSuccess ||
      (e = up(b.counts.p, hdr, sizeof(hdr))) != cudaSuccess)
    return e;
  e = cudaStreamSynchronize(b.st);  // the host vectors go out of scope
  b.dirty = false;
  return e;
}

// Persistent CTAs of the batch's pair kernel (queried outside any capture).
int pair_grid(const mmvm_server* s, const Batch& b) {
  const int per_sm = std::max(1, mmvm::pair_batch_occupancy(b.pe, kGroup));
  return s->sms * per_sm;
}

// One RK4 step of a batch on its stream (captured into its tick graph).
cudaError_t enqueue_batch_step(const mmvm_server* s, Batch& b) {
  cudaError_t e;
  const int prec = s->cfg.precision;
  cudaStream_t st = b.st;
  int* counters = b.counts.p + kCountHdr;
  if ((e = cudaMemsetAsync(counters, 0, kCounters * sizeof(int), st)) != cudaSuccess) return e;
  const bool pairs = b.pe.M >= 0;
  const bool far = pairs && b.far;
  if (far && (e = mmvm::launch_batch_order(b.slot_cap, b.counts.p, b.inst.p, b.counts.p + 3,
                                           b.inst_cap, b.slot_inst.p, b.ibox.p, b.kin.p, b.kout.p,
                                           b.iin.p, b.iout.p, b.sort_tmp.p, b.sort_tmp.cap,
                                           b.perm.p, st)) != cudaSuccess)
    return e;
  static const double cs[kStages] = {0.0, 0.5, 0.5, 1.0};
  const int fgrid = std::max(1, std::min(s->sms * 4, (b.slot_cap + b.tb - 1) / b.tb));
  for (int stage = 1; stage <= kStages; ++stage) {
    const int src = stage == 1 ? 0 : 1;
    if (pairs) {
      if ((e = mmvm::launch_prep_batch(prec, b.M, b.inst.p, b.slot_inst.p, b.counts.p,
                                       b.slot_cap, src, cs[stage - 1], far ? b.perm.p : nullptr,
                                       b.rec.p, far ? b.gbox.p : nullptr, st)) != cudaSuccess)
        return e;
      if ((e = mmvm::pair_launch_batch(b.pe, b.rec.p, b.inst.p, b.pitems.p, b.counts.p + 1,
                                       counters + (stage - 1) * mmvm::kMaxSlices, b.grid, kGroup,
                                       far ? b.gbox.p : nullptr, b.partial.p, st)) != cudaSuccess)
        return e;
    }
    mmvm::BatchFinishArgs B;
    B.M = b.M;
    B.K = b.K;
    B.NB = b.NB;
    B.targets_per_block = b.tb;
    B.inst = b.inst.p;
    B.items = b.fitems.p;
    B.n_items = b.counts.p + 2;
    B.partial = b.partial.p;
    B.perm_local = far ? b.perm.p : nullptr;
    B.k_off = b.k_off.p;
    B.e_l = b.e_l.p;
    B.e_b = b.e_b.p;
    B.e_c = b.e_c.p;
    B.psi0 = b.psi0.p;
    B.src = src;
    B.cs = cs[stage - 1];
    B.mode = stage;
    if ((e = mmvm::launch_finish_batch(B, fgrid, st)) != cudaSuccess) return e;
  }
  if ((e = mmvm::launch_advance_batch(b.inst.p, b.counts.p + 3, b.inst_cap, st)) != cudaSuccess)
    return e;
  // divergence check: a simulation whose state left the finite range stops
  return mmvm::launch_scan_batch(b.M, b.inst.p, b.counts.p + 3, b.inst_cap, b.bad.p, st);
}

cudaError_t capture_batch(const mmvm_server* s, Batch& b) {
  if (b.exec) {
    cudaGraphExecDestroy(b.exec);
    b.exec = nullptr;
  }
  cudaError_t e = cudaStreamBeginCapture(b.st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t ee = enqueue_batch_step(s, b);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b.st, &g);
  if (ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return ee;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&b.exec, g, 0);
  cudaGraphDestroy(g);
  if (e == cudaSuccess) b.graph_valid = true;
  return e;
}

// Time every compiled variant of a batch's order on its first members
// (stage-1 records) and keep the fastest, once per (device, order, precision).
cudaError_t tune_batch(const mmvm_server* s, Batch& b) {
  b.tuned = true;
  const int nv = mmvm::pair_variant_count(b.M, s->cfg.precision);
  if (nv < 1) return cudaSuccess;
  const auto key = std::make_tuple(s->cfg.device, b.M, s->cfg.precision);
  int choice = -1;
  if (const char* f = std::getenv("MMVM_PAIR_VARIANT")) choice = std::atoi(f);
  if (choice < 0)
    if (const char* a = std::getenv("MMVM_AUTOTUNE"))
      if (std::atoi(a) == 0) choice = 0;
  if (choice < 0) {
    std::lock_guard<std::mutex> lk(g_batch_tune_mu);
    auto it = g_batch_tuned.find(key);
    if (it != g_batch_tuned.end()) choice = it->second;
  }
  cudaError_t e;
  if (choice < 0 && nv > 1) {
    double best = 1e300;
    choice = 0;
    for (int v = 0; v < nv; ++v) {
      mmvm::PairEntry pe = mmvm::pair_entry(b.M, s->cfg.precision, v);
      if (pe.M != b.M || !pe.uniform_tpc) continue;  // items are pe.tpc targets wide
      if ((e = mmvm::pair_prepare(pe, kGroup)) != cudaSuccess) return e;
      b.pe = pe;
      bool grown = false;
      if ((e = rebuild(b, &grown)) != cudaSuccess) return e;
      if ((e = mmvm::launch_prep_batch(s->cfg.precision, b.M, b.inst.p, b.slot_inst.p,
                                       b.counts.p, b.slot_cap, 0, 0.0, nullptr, b.rec.p, nullptr,
                                       b.st)) != cudaSuccess)
        return e;
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {
        int* counters = b.counts.p + kCountHdr;
        if ((e = cudaMemsetAsync(counters, 0, kCounters * sizeof(int), b.st)) != cudaSuccess)
          return e;
        if ((e = cudaEventRecord(b.ev0, b.st)) != cudaSuccess) return e;
        if ((e = mmvm::pair_launch_batch(pe, b.rec.p, b.inst.p, b.pitems.p, b.counts.p + 1,
                                         counters, pair_grid(s, b), kGroup, nullptr, b.partial.p,
                                         b.st)) != cudaSuccess)
          return e;
        if ((e = cudaEventRecord(b.ev1, b.st)) != cudaSuccess) return e;
        if ((e = cudaEventSynchronize(b.ev1)) != cudaSuccess) return e;
        if ((e = cudaEventElapsedTime(&ms, b.ev0, b.ev1)) != cudaSuccess) return e;
      }
      if (const char* vb = std::getenv("MMVM_TUNE_VERBOSE"))
        if (std::atoi(vb))
          std::fprintf(stderr, "[mmvm serve tune] M=%d variant %d: %.3f ms for %lld pairs\n",
                       b.M, v, ms, (long long)b.pairs_per_rhs);
      if (ms < best) {
        best = ms;
        choice = v;
      }
    }
    std::lock_guard<std::mutex> lk(g_batch_tune_mu);
    g_batch_tuned[key] = choice;
  }
  if (choice < 0) choice = 0;
  mmvm::PairEntry pe = mmvm::pair_entry(b.M, s->cfg.precision, choice);
  if (pe.M != b.M || !pe.uniform_tpc) pe = mmvm::pair_entry(b.M, s->cfg.precision, 0);
  if ((e = mmvm::pair_prepare(pe, kGroup)) != cudaSuccess) return e;
  b.pe = pe;
  b.dirty = true;
  b.graph_valid = false;
  return cudaSuccess;
}

Batch& batch_of(mmvm_server* s, int M, int64_t n, cudaError_t* e) {
  const int key = M * 4 + size_class(n);
  auto it = s->batches.find(key);
  if (it != s->batches.end()) return it->second;
  Batch& b = s->batches[key];
  b.M = M;
  b.K = mmvm::n_moments(M);
  b.NB = mmvm::n_beta(M);
  b.tb = finish_tb(b.K);
  b.pe = mmvm::PairEntry();
  if (M <= MMVM_MAX_ORDER_PAIRS) {
    b.pe = mmvm::pair_entry(M, s->cfg.precision, 0);
    if (b.pe.M == M) *e = mmvm::pair_prepare(b.pe, kGroup);
  }
  b.far = s->cfg.precision == MMVM_MIXED_FP32 && !(s->cfg.flags & MMVM_FLAG_NO_FAR_FIELD);
  if (*e == cudaSuccess) *e = cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking);
  if (*e == cudaSuccess) *e = cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming);
  if (*e == cudaSuccess) *e = cudaEventCreate(&b.ev0);
  if (*e == cudaSuccess) *e = cudaEventCreate(&b.ev1);
  if (*e == cudaSuccess) *e = upload_tables(b);
  return b;
}

void fail_everything(mmvm_server* s, const std::string& msg) {
  std::lock_guard<std::mutex> lk(s->mu);
  s->broken = true;
  s->broken_msg = msg;
  for (auto& kv : s->batches) {
    for (Request* r : kv.second.members) finish_request(s, r, MMVM_E_DEVICE, msg);
    for (Request* r : kv.second.incoming) finish_request(s, r, MMVM_E_DEVICE, msg);
    kv.second.members.clear();
    kv.second.incoming.clear();
  }
  for (Request* r : s->queue) {
    r->status = MMVM_E_DEVICE;
    r->err = msg;
    r->t_done = Clock::now();
    s->failed += 1;
  }
  s->queue.clear();
  s->cv.notify_all();
}

// Bookkeeping after a batch's tick: advance every member, retire the ones
// that are done or diverged (state back to the host, device state freed).
cudaError_t complete_tick(mmvm_server* s, Batch& b) {
  cudaError_t e;
  const size_t nm = b.members.size();
  b.bad_host.assign(nm, 0);
  if (nm && (e = cudaMemcpyAsync(b.bad_host.data(), b.bad.p, nm * sizeof(int),
                                 cudaMemcpyDeviceToHost, b.st)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(b.st)) != cudaSuccess) return e;
  // the members that are done or diverged: their state copies are queued
  // together and waited for once
  std::vector<Request*> keep;
  std::vector<size_t> done;
  for (size_t i = 0; i < nm; ++i) {
    Request* r = b.members[i];
    r->steps_done += 1;
    r->t = r->t + r->dt;  // the device does the same addition
    if (r->steps_done < r->nsteps && !b.bad_host[i]) {
      keep.push_back(r);
      continue;
    }
    done.push_back(i);
    e = cudaMemcpyAsync(r->x.data(), r->d_state, r->x.size() * sizeof(double),
                        cudaMemcpyDeviceToHost, b.st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(r->m.data(), r->d_state + 2 * r->n, r->m.size() * sizeof(double),
                          cudaMemcpyDeviceToHost, b.st);
    if (e != cudaSuccess) return e;
  }
  if (!done.empty() && (e = cudaStreamSynchronize(b.st)) != cudaSuccess) return e;
  for (size_t i : done) {
    Request* r = b.members[i];
    cudaFreeAsync(r->d_state, b.st);
    r->d_state = nullptr;
    int status = MMVM_OK;
    std::string msg;
    if (b.bad_host[i]) {
      status = MMVM_E_NUMERIC;
      msg = "the state left the finite range at step " + std::to_string(r->steps_done);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    finish_request(s, r, status, msg);
  }
  if (keep.size() != nm) {
    b.members.swap(keep);
    b.dirty = true;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->ticks += 1;
  s->pair_interactions += 4.0 * (double)b.pairs_per_rhs;
  s->max_batch = std::max(s->max_batch, (int64_t)nm);
  return cudaSuccess;
}

// Start the next tick of an idle batch (new members join first).
cudaError_t launch_tick(mmvm_server* s, Batch& b) {
  cudaError_t e;
  if (!b.incoming.empty()) {
    // the state of newcomers is uploaded on the upload stream
    if ((e = cudaStreamWaitEvent(b.st, s->up_done, 0)) != cudaSuccess) return e;
    for (Request* r : b.incoming) b.members.push_back(r);
    b.incoming.clear();
    b.dirty = true;
  }
  if (b.members.empty()) return cudaSuccess;
  if (!b.tuned && b.pe.M >= 0 && (e = tune_batch(s, b)) != cudaSuccess) return e;
  if (b.dirty) {
    bool grown = false;
    if ((e = rebuild(b, &grown)) != cudaSuccess) return e;
    if (grown) b.graph_valid = false;
  }
  if (!b.graph_valid) {
    if (b.pe.M >= 0) b.grid = pair_grid(s, b);
    if ((e = capture_batch(s, b)) != cudaSuccess) return e;
  }
  if ((e = cudaGraphLaunch(b.exec, b.st)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(b.done, b.st)) != cudaSuccess) return e;
  b.in_flight = true;
  if (s->in_flight++ == 0) s->busy_since = Clock::now();
  return cudaSuccess;
}

void worker_main(mmvm_server* s) {
  if (cudaSetDevice(s->cfg.device) != cudaSuccess) {
    fail_everything(s, "cudaSetDevice failed in the server thread");
    return;
  }
  for (;;) {
    std::vector<Request*> admitted;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop) break;
      while (!s->queue.empty() && s->n_active < s->cfg.max_active) {
        Request* r = s->queue.front();
        if (s->n_active > 0 && s->fp_used + r->fp > s->budget) break;  // FIFO: wait for room
        s->queue.pop_front();
        s->fp_used += r->fp;
        s->fp_peak = std::max(s->fp_peak, s->fp_used);
        s->n_active += 1;
        s->max_active = std::max(s->max_active, s->n_active);
        r->t_admit = Clock::now();
        admitted.push_back(r);
      }
      if (s->n_active == 0 && s->in_flight == 0) {
        s->cv.wait_for(lk, std::chrono::milliseconds(20));
        continue;
      }
    }
    bool progress = !admitted.empty();
    // newcomers: device state on the upload stream (stream-ordered allocation)
    for (Request* r : admitted) {
      if (r->nsteps == 0) {  // nothing to integrate: the input is the result
        std::lock_guard<std::mutex> lk(s->mu);
        finish_request(s, r, MMVM_OK, "");
        continue;
      }
      const int K = mmvm::n_moments(r->order);
      cudaError_t e =
          cudaMallocAsync(&r->d_state, 6 * (size_t)r->n * (2 + K) * sizeof(double), s->up);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->d_state, r->x.data(), r->x.size() * sizeof(double),
                            cudaMemcpyHostToDevice, s->up);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->d_state + 2 * r->n, r->m.data(), r->m.size() * sizeof(double),
                            cudaMemcpyHostToDevice, s->up);
      if (e != cudaSuccess) {
        if (r->d_state) cudaFreeAsync(r->d_state, s->up);
        r->d_state = nullptr;
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(s->mu);
        finish_request(s, r, e == cudaErrorMemoryAllocation ? MMVM_E_OOM : MMVM_E_DEVICE,
                       std::string("admission: ") + cudaGetErrorString(e));
        continue;
      }
      cudaError_t eb = cudaSuccess;
      Batch& b = batch_of(s, r->order, r->n, &eb);
      if (eb != cudaSuccess) {
        fail_everything(s, std::string("batch set-up: ") + cudaGetErrorString(eb));
        return;
      }
      b.incoming.push_back(r);
    }
    if (!admitted.empty() && cudaEventRecord(s->up_done, s->up) != cudaSuccess) {
      fail_everything(s, "upload event failed");
      return;
    }
    // finished ticks, then new ticks of every idle batch
    for (auto& kv : s->batches) {
      Batch& b = kv.second;
      cudaError_t e = cudaSuccess;
      if (b.in_flight) {
        const cudaError_t q = cudaEventQuery(b.done);
        if (q == cudaErrorNotReady) continue;
        b.in_flight = false;
        if (--s->in_flight == 0) {
          std::lock_guard<std::mutex> lk(s->mu);
          s->busy_ms += ms_between(s->busy_since, Clock::now());
        }
        e = q == cudaSuccess ? complete_tick(s, b) : q;
        progress = true;
      }
      if (e == cudaSuccess && !b.in_flight && (!b.members.empty() || !b.incoming.empty())) {
        e = launch_tick(s, b);
        progress = true;
      }
      if (e != cudaSuccess) {
        fail_everything(s, std::string("tick: ") + cudaGetErrorString(e));
        return;
      }
    }
    s->cv.notify_all();
    if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

}  // namespace

extern "C" {

int mmvm_request_footprint(int32_t order, int32_t precision, int64_t n, uint64_t* bytes) {
  if (!bytes) return fail(MMVM_E_INVALID_ARG, "null argument");
  if (order < 0 || order > MMVM_MAX_ORDER_SINGLE || n < 1)
    return fail(MMVM_E_INVALID_ARG, "order or n out of range");
  if (precision != MMVM_FP64 && precision != MMVM_MIXED_FP32)
    return fail(MMVM_E_INVALID_ARG, "unknown precision");
  *bytes = footprint(order, precision, n);
  return MMVM_OK;
}

int mmvm_server_create(const mmvm_server_config* cfg, mmvm_server** out) {
  if (!cfg || !out) return fail(MMVM_E_INVALID_ARG, "null argument");
  *out = nullptr;
  if (cfg->precision != MMVM_FP64 && cfg->precision != MMVM_MIXED_FP32)
    return fail(MMVM_E_INVALID_ARG, "unknown precision");
  if (cfg->max_active < 0) return fail(MMVM_E_INVALID_ARG, "max_active must be >= 0");
  if (cfg->flags & ~MMVM_FLAG_NO_FAR_FIELD) return fail(MMVM_E_INVALID_ARG, "unknown flag bits");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return fail(MMVM_E_DEVICE, cudaGetErrorString(e));
  if (cfg->device < 0 || cfg->device >= ndev)
    return fail(MMVM_E_INVALID_ARG, "device ordinal out of range");
  if ((e = cudaSetDevice(cfg->device)) != cudaSuccess)
    return fail(MMVM_E_DEVICE, cudaGetErrorString(e));
  mmvm_server* s = new mmvm_server();
  s->cfg = *cfg;
  if (s->cfg.max_active == 0) s->cfg.max_active = 256;
  size_t free_b = 0, total_b = 0;
  if ((e = cudaMemGetInfo(&free_b, &total_b)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, cfg->device)) !=
          cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&s->up, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&s->up_done, cudaEventDisableTiming)) != cudaSuccess) {
    if (s->up) cudaStreamDestroy(s->up);
    if (s->up_done) cudaEventDestroy(s->up_done);
    delete s;
    return fail(MMVM_E_DEVICE, cudaGetErrorString(e));
  }
  s->budget = cfg->hbm_budget_bytes ? cfg->hbm_budget_bytes : free_b / 2;
  s->worker = std::thread(worker_main, s);
  *out = s;
  return MMVM_OK;
}

void mmvm_server_destroy(mmvm_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->cfg.device);
  for (auto& kv : s->batches)
    if (kv.second.st) cudaStreamSynchronize(kv.second.st);
  cudaStreamSynchronize(s->up);
  for (auto& kv : s->batches) {
    for (Request* r : kv.second.members)
      if (r->d_state) cudaFree(r->d_state);
    for (Request* r : kv.second.incoming)
      if (r->d_state) cudaFree(r->d_state);
    kv.second.release();
  }
  cudaEventDestroy(s->up_done);
  cudaStreamDestroy(s->up);
  for (auto& kv : s->all) delete kv.second;
  delete s;
}

int mmvm_submit(mmvm_server* s, const mmvm_request* q, uint64_t* ticket) {
  if (!s || !q || !ticket) return fail(MMVM_E_INVALID_ARG, "null argument");
  if (q->order < 0 || q->order > kMaxOrderServed)
    return fail(MMVM_E_UNSUPPORTED, "order above 16 (the server's finish tables)");
  if (q->n < 1 || q->n > (1 << 20)) return fail(MMVM_E_INVALID_ARG, "n must be 1 .. 2^20");
  if (q->n > 1 && q->order > MMVM_MAX_ORDER_PAIRS)
    return fail(MMVM_E_UNSUPPORTED, "order above MMVM_MAX_ORDER_PAIRS for n > 1");
  if (!q->x || !q->moments) return fail(MMVM_E_INVALID_ARG, "null state");
  if (!(q->lambda0 > 0.0) || !std::isfinite(q->lambda0))
    return fail(MMVM_E_INVALID_ARG, "lambda0 must be positive and finite");
  if (!(q->nu >= 0.0) || !std::isfinite(q->nu))
    return fail(MMVM_E_INVALID_ARG, "nu must be >= 0 and finite");
  if (!std::isfinite(q->t0) || !std::isfinite(q->dt) || q->nsteps < 0)
    return fail(MMVM_E_INVALID_ARG, "t0 and dt must be finite and nsteps >= 0");
  if (q->lambda0 * q->lambda0 + 4.0 * q->nu * q->t0 <= 0.0 ||
      q->lambda0 * q->lambda0 + 4.0 * q->nu * (q->t0 + q->nsteps * q->dt) <= 0.0)
    return fail(MMVM_E_INVALID_ARG, "lambda^2 must stay positive over the run");
  const int K = mmvm::n_moments(q->order);
  for (int64_t j = 0; j < q->n; ++j) {
    if (!std::isfinite(q->x[2 * j]) || !std::isfinite(q->x[2 * j + 1]))
      return fail(MMVM_E_NUMERIC, "non-finite position at particle " + std::to_string(j));
    for (int k = 0; k < K; ++k)
      if (!std::isfinite(q->moments[j * K + k]))
        return fail(MMVM_E_NUMERIC, "non-finite moment at particle " + std::to_string(j));
    if (q->moments[j * K] == 0.0)
      return fail(MMVM_E_ZERO_CIRCULATION,
                  "M[0,0] == 0 at particle " + std::to_string(j) + " (eq:mass)");
  }
  const uint64_t fp = footprint(q->order, s->cfg.precision, q->n);
  if (fp > s->budget)
    return fail(MMVM_E_OOM, "request footprint " + std::to_string(fp) +
                                " bytes exceeds the server's HBM budget " +
                                std::to_string(s->budget));
  Request* r = new Request();
  r->order = q->order;
  r->n = q->n;
  r->lam0 = q->lambda0;
  r->nu = q->nu;
  r->t0 = q->t0;
  r->t = q->t0;
  r->dt = q->dt;
  r->nsteps = q->nsteps;
  r->x.assign(q->x, q->x + 2 * q->n);
  r->m.assign(q->moments, q->moments + (size_t)K * q->n);
  r->fp = fp;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->broken) {
      delete r;
      return fail(MMVM_E_DEVICE, "server stopped after a device error: " + s->broken_msg);
    }
    r->ticket = s->next_ticket++;
    s->all[r->ticket] = r;
    s->queue.push_back(r);
    s->submitted += 1;
    *ticket = r->ticket;
  }
  s->cv.notify_all();
  return MMVM_OK;
}

int mmvm_poll(mmvm_server* s, uint64_t ticket, double* x_out, double* moments_out,
              mmvm_result* res) {
  if (!s) return fail(MMVM_E_INVALID_ARG, "null server");
  Request* r = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return fail(MMVM_E_INVALID_ARG, "unknown ticket");
    r = it->second;
    if (res) {
      res->status = r->status;
      res->order = r->order;
      res->n = r->n;
      res->steps_done = r->steps_done;
      res->t = r->t;
      const auto now = Clock::now();
      const bool admitted = r->t_admit.time_since_epoch().count() != 0;
      res->queue_ms = ms_between(r->t_submit, admitted ? r->t_admit : now);
      res->latency_ms =
          ms_between(r->t_submit, r->status == MMVM_PENDING ? now : r->t_done);
    }
    if (r->status == MMVM_PENDING) return MMVM_PENDING;
    s->all.erase(it);
  }
  const int status = r->status;
  if (status == MMVM_OK) {
    if (x_out) std::memcpy(x_out, r->x.data(), r->x.size() * sizeof(double));
    if (moments_out) std::memcpy(moments_out, r->m.data(), r->m.size() * sizeof(double));
  } else {
    mmvm::set_last_error(r->err.c_str());
  }
  delete r;
  return status;
}

int mmvm_server_stats(mmvm_server* s, mmvm_server_counters* out) {
  if (!s || !out) return fail(MMVM_E_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->queued = (int64_t)s->queue.size();
  out->active = s->n_active;
  out->ticks = s->ticks;
  out->max_batch = s->max_batch;
  out->max_active = s->max_active;
  out->pair_interactions = s->pair_interactions;
  out->busy_ms = s->busy_ms;
  out->footprint_bytes = s->fp_used;
  out->peak_footprint_bytes = s->fp_peak;
  out->budget_bytes = s->budget;
  return s->broken ? fail(MMVM_E_DEVICE, s->broken_msg) : MMVM_OK;
}

}  // extern "C"
