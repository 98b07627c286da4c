// Serving: one request loop runs many independent MMVM simulations (different
// particle counts, orders, viscosities, core sizes, step sizes and step
// counts) on one GPU at once.
//
// * Continuous batching.  Requests wait in a FIFO queue and are admitted
//   between steps while their device footprint (state, source records,
//   partial sums) fits the server's HBM budget; a finished simulation leaves
//   at the end of the step in which it completes and frees its footprint for
//   the next one.  Admitted state stays resident on the device until then.
// * One tick = one RK4 step of every admitted simulation.  Simulations of one
//   order form a batch: its records, partials and work lists live in buffers
//   of the batch, and each RK4 stage is three launches for the whole batch
//   (records, the persistent all-pairs kernel working through a list of
//   (simulation, target tile, source chunk) items, the FP64 finish).  Batches
//   of different orders run on their own streams, so their work overlaps.
//   The tick is captured once as a CUDA graph and replayed; the kernels read
//   the sizes of the batch from device memory, so admitting or retiring a
//   simulation only re-uploads the work lists (the graph is captured again
//   only when a buffer grows or an order appears or disappears).
// * The way a simulation's pairs are split into items depends on its own
//   size only, and every item is summed in a fixed order, so a simulation's
//   result does not depend on what else is in the batch.
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

constexpr int kChunkTarget = 1024;  // sources per chunk (items of similar cost)
constexpr int kMaxChunks = 16;
constexpr int kStages = 4;

int chunks_for(int64_t n) {
  if (n <= 1) return 0;
  return (int)std::min<int64_t>((n + kChunkTarget - 1) / kChunkTarget, kMaxChunks);
}

int chunk_len_for(int64_t n, int chunks) {
  return mmvm::round_up((int)((n + chunks - 1) / chunks), kGroup);
}

int finish_tb(int K) { return std::max(1, 128 / (((K + 31) / 32) * 32)); }

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
  return state + recs + part + items;
}

template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t cap = 0;
  // grow to at least n elements (contents are not kept); true if reallocated
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

// Every admitted simulation of one order.
struct Batch {
  int M = 0, K = 0, NB = 0, tb = 1;
  mmvm::PairEntry pe;  // pe.M == -1: no pair kernel (orders above the pair limit: n == 1 only)
  std::vector<Request*> members;
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
  DBuf<int> counts;  // n_slots, n_pair_items, n_finish_items, n_inst, then the item counters
  DBuf<int> bad;     // per instance: non-finite state after the tick
  std::vector<int> bad_host;
  int slot_cap = 0;  // slots the prep grid covers
  cudaStream_t side = nullptr;
  int64_t pairs_per_rhs = 0;  // sum of n^2
  void release() {
    k_off.release();
    e_l.release();
    e_b.release();
    e_c.release();
    psi0.release();
    rec.release();
    partial.release();
    inst.release();
    slot_inst.release();
    pitems.release();
    fitems.release();
    counts.release();
    bad.release();
    if (side) cudaStreamDestroy(side);
    side = nullptr;
  }
};

constexpr int kCountHdr = 4;
constexpr int kCounters = kStages * mmvm::kMaxSlices;

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
  double pair_interactions = 0, busy_ms = 0;
  std::thread worker;
  // worker-thread state
  cudaStream_t st = nullptr;
  cudaEvent_t fork = nullptr, ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> join;
  std::map<int, Batch> batches;
  cudaGraphExec_t exec = nullptr;
  bool graph_valid = false;
  std::vector<int> graph_orders;
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

cudaError_t upload_tables(Batch& b, cudaStream_t st) {
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
    return bytes ? cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
  };
  if ((e = up(b.k_off.p, T.k_off.data(), T.k_off.size() * sizeof(int))) != cudaSuccess ||
      (e = up(b.e_l.p, T.e_l.data(), T.e_l.size() * sizeof(int))) != cudaSuccess ||
      (e = up(b.e_b.p, T.e_b.data(), T.e_b.size() * sizeof(int))) != cudaSuccess ||
      (e = up(b.e_c.p, T.e_c.data(), T.e_c.size() * sizeof(double))) != cudaSuccess ||
      (e = up(b.psi0.p, T.psi0.data(), T.psi0.size() * sizeof(double))) != cudaSuccess)
    return e;
  return cudaStreamSynchronize(st);  // the host tables go out of scope
}

// Work lists and descriptors of a batch for the current members.
cudaError_t rebuild(mmvm_server* s, Batch& b, bool* grown) {
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
  const int eb = b.pe.M >= 0 ? b.pe.elem_bytes : 8;
  const int R = b.pe.M >= 0 ? b.pe.rec_len : mmvm::rec_len<double>(b.M);
  if ((e = b.rec.ensure((size_t)std::max(slots, kGroup) * R * eb, grown)) != cudaSuccess ||
      (e = b.partial.ensure((size_t)std::max<long long>(part, 1), grown)) != cudaSuccess ||
      (e = b.inst.ensure(std::max<size_t>(inst.size(), 1), grown)) != cudaSuccess ||
      (e = b.slot_inst.ensure(std::max<size_t>(slot_inst.size(), 1), grown)) != cudaSuccess ||
      (e = b.pitems.ensure(std::max<size_t>(pitems.size(), 1), grown)) != cudaSuccess ||
      (e = b.fitems.ensure(std::max<size_t>(fit.size(), 1), grown)) != cudaSuccess ||
      (e = b.counts.ensure(kCountHdr + kCounters, grown)) != cudaSuccess ||
      (e = b.bad.ensure(std::max<size_t>(inst.size(), 1), grown)) != cudaSuccess)
    return e;
  const int slot_cap = (int)(b.rec.cap / ((size_t)R * eb));
  if (slot_cap != b.slot_cap) {
    b.slot_cap = slot_cap;
    *grown = true;
  }
  const int hdr[kCountHdr] = {slots, (int)pitems.size(), (int)fit.size(), (int)inst.size()};
  auto up = [&](void* d, const void* h, size_t bytes) {
    return bytes ? cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s->st) : cudaSuccess;
  };
  if ((e = up(b.inst.p, inst.data(), inst.size() * sizeof(BatchInst))) != cudaSuccess ||
      (e = up(b.slot_inst.p, slot_inst.data(), slot_inst.size() * sizeof(int))) != cudaSuccess ||
      (e = up(b.pitems.p, pitems.data(), pitems.size() * sizeof(int4))) != cudaSuccess ||
      (e = up(b.fitems.p, fit.data(), fit.size() * sizeof(int2))) != cudaSuccess ||
      (e = up(b.counts.p, hdr, sizeof(hdr))) != cudaSuccess)
    return e;
  // pageable sources: the copies are complete before the vectors go
  e = cudaStreamSynchronize(s->st);
  b.dirty = false;
  return e;
}

int pair_grid(mmvm_server* s, const Batch& b) {
  const int per_sm = std::max(1, mmvm::pair_batch_occupancy(b.pe, kGroup));
  return s->sms * per_sm;
}

// One RK4 step of a batch on stream st (captured into the tick graph).
cudaError_t enqueue_batch_step(mmvm_server* s, Batch& b, cudaStream_t st) {
  cudaError_t e;
  const int prec = s->cfg.precision;
  int* counters = b.counts.p + kCountHdr;
  if ((e = cudaMemsetAsync(counters, 0, kCounters * sizeof(int), st)) != cudaSuccess) return e;
  static const double cs[kStages] = {0.0, 0.5, 0.5, 1.0};
  const int fgrid = std::max(1, std::min(s->sms * 4, (b.slot_cap + b.tb - 1) / b.tb));
  for (int stage = 1; stage <= kStages; ++stage) {
    const int src = stage == 1 ? 0 : 1;
    if (b.pe.M >= 0) {
      if ((e = mmvm::launch_prep_batch(prec, b.M, b.inst.p, b.slot_inst.p, b.counts.p,
                                       b.slot_cap, src, cs[stage - 1], b.rec.p, st)) !=
          cudaSuccess)
        return e;
      if ((e = mmvm::pair_launch_batch(b.pe, b.rec.p, b.inst.p, b.pitems.p, b.counts.p + 1,
                                       counters + (stage - 1) * mmvm::kMaxSlices,
                                       pair_grid(s, b), kGroup, b.partial.p, st)) != cudaSuccess)
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
  if ((e = mmvm::launch_advance_batch(b.inst.p, b.counts.p + 3, (int)b.inst.cap, st)) !=
      cudaSuccess)
    return e;
  // divergence check: a simulation whose state left the finite range stops
  return mmvm::launch_scan_batch(b.M, b.inst.p, b.counts.p + 3, (int)b.inst.cap, b.bad.p, st);
}

cudaError_t capture_tick(mmvm_server* s) {
  if (s->exec) {
    cudaGraphExecDestroy(s->exec);
    s->exec = nullptr;
  }
  s->graph_orders.clear();
  cudaError_t e = cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t ee = cudaEventRecord(s->fork, s->st);
  size_t gi = 0;
  for (auto& kv : s->batches) {
    Batch& b = kv.second;
    if (b.members.empty() || ee != cudaSuccess) continue;
    if (gi >= s->join.size()) {
      cudaEvent_t ev;
      ee = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (ee != cudaSuccess) break;
      s->join.push_back(ev);
    }
    if ((ee = cudaStreamWaitEvent(b.side, s->fork, 0)) != cudaSuccess) break;
    if ((ee = enqueue_batch_step(s, b, b.side)) != cudaSuccess) break;
    if ((ee = cudaEventRecord(s->join[gi], b.side)) != cudaSuccess) break;
    if ((ee = cudaStreamWaitEvent(s->st, s->join[gi], 0)) != cudaSuccess) break;
    s->graph_orders.push_back(kv.first);
    ++gi;
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(s->st, &g);
  if (ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return ee;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&s->exec, g, 0);
  cudaGraphDestroy(g);
  if (e == cudaSuccess) s->graph_valid = true;
  return e;
}

// Time every compiled variant of a batch on its first members (stage-1
// records) and keep the fastest, once per (device, order, precision).
cudaError_t tune_batch(mmvm_server* s, Batch& b) {
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
      if (pe.M != b.M) continue;
      if ((e = mmvm::pair_prepare(pe, kGroup)) != cudaSuccess) return e;
      b.pe = pe;
      bool grown = false;
      if ((e = rebuild(s, b, &grown)) != cudaSuccess) return e;
      if ((e = mmvm::launch_prep_batch(s->cfg.precision, b.M, b.inst.p, b.slot_inst.p,
                                       b.counts.p, b.slot_cap, 0, 0.0, b.rec.p, s->st)) !=
          cudaSuccess)
        return e;
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {
        int* counters = b.counts.p + kCountHdr;
        if ((e = cudaMemsetAsync(counters, 0, kCounters * sizeof(int), s->st)) != cudaSuccess)
          return e;
        if ((e = cudaEventRecord(s->ev0, s->st)) != cudaSuccess) return e;
        if ((e = mmvm::pair_launch_batch(pe, b.rec.p, b.inst.p, b.pitems.p, b.counts.p + 1,
                                         counters, pair_grid(s, b), kGroup, b.partial.p,
                                         s->st)) != cudaSuccess)
          return e;
        if ((e = cudaEventRecord(s->ev1, s->st)) != cudaSuccess) return e;
        if ((e = cudaEventSynchronize(s->ev1)) != cudaSuccess) return e;
        if ((e = cudaEventElapsedTime(&ms, s->ev0, s->ev1)) != cudaSuccess) return e;
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
  if (pe.M != b.M) pe = mmvm::pair_entry(b.M, s->cfg.precision, 0);
  if ((e = mmvm::pair_prepare(pe, kGroup)) != cudaSuccess) return e;
  b.pe = pe;
  b.dirty = true;
  s->graph_valid = false;
  return cudaSuccess;
}

Batch& batch_of(mmvm_server* s, int M, cudaError_t* e) {
  auto it = s->batches.find(M);
  if (it != s->batches.end()) return it->second;
  Batch& b = s->batches[M];
  b.M = M;
  b.K = mmvm::n_moments(M);
  b.NB = mmvm::n_beta(M);
  b.tb = finish_tb(b.K);
  b.pe = mmvm::PairEntry();
  if (M <= MMVM_MAX_ORDER_PAIRS) {
    b.pe = mmvm::pair_entry(M, s->cfg.precision, 0);
    if (b.pe.M == M) *e = mmvm::pair_prepare(b.pe, kGroup);
  }
  if (*e == cudaSuccess) *e = cudaStreamCreateWithFlags(&b.side, cudaStreamNonBlocking);
  if (*e == cudaSuccess) *e = upload_tables(b, s->st);
  return b;
}

void fail_everything(mmvm_server* s, const std::string& msg) {
  std::lock_guard<std::mutex> lk(s->mu);
  s->broken = true;
  s->broken_msg = msg;
  for (auto& kv : s->batches) {
    for (Request* r : kv.second.members) finish_request(s, r, MMVM_E_DEVICE, msg);
    kv.second.members.clear();
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
      while (!s->queue.empty() && s->n_active + (int64_t)admitted.size() < s->cfg.max_active) {
        Request* r = s->queue.front();
        const bool idle = s->n_active == 0 && admitted.empty();
        if (!idle && s->fp_used + r->fp > s->budget) break;  // FIFO: wait for room
        s->queue.pop_front();
        s->fp_used += r->fp;
        s->fp_peak = std::max(s->fp_peak, s->fp_used);
        s->n_active += 1;
        r->t_admit = Clock::now();
        admitted.push_back(r);
      }
      if (s->n_active == 0) {
        s->cv.wait_for(lk, std::chrono::milliseconds(20));
        continue;
      }
    }
    // device state of the newcomers (step-start block y = (x, M))
    for (Request* r : admitted) {
      const int K = mmvm::n_moments(r->order);
      cudaError_t e = cudaMalloc(&r->d_state, 6 * (size_t)r->n * (2 + K) * sizeof(double));
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->d_state, r->x.data(), r->x.size() * sizeof(double),
                            cudaMemcpyHostToDevice, s->st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->d_state + 2 * r->n, r->m.data(), r->m.size() * sizeof(double),
                            cudaMemcpyHostToDevice, s->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
      if (e != cudaSuccess) {
        if (r->d_state) cudaFree(r->d_state);
        r->d_state = nullptr;
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(s->mu);
        finish_request(s, r, e == cudaErrorMemoryAllocation ? MMVM_E_OOM : MMVM_E_DEVICE,
                       std::string("admission: ") + cudaGetErrorString(e));
        s->cv.notify_all();
        continue;
      }
      if (r->nsteps == 0) {  // nothing to integrate
        cudaFree(r->d_state);
        r->d_state = nullptr;
        std::lock_guard<std::mutex> lk(s->mu);
        finish_request(s, r, MMVM_OK, "");
        s->cv.notify_all();
        continue;
      }
      cudaError_t eb = cudaSuccess;
      Batch& b = batch_of(s, r->order, &eb);
      if (eb != cudaSuccess) {
        fail_everything(s, std::string("batch set-up: ") + cudaGetErrorString(eb));
        return;
      }
      b.members.push_back(r);
      b.dirty = true;
    }
    // work lists; a new order or a grown buffer needs a new graph
    std::vector<int> orders;
    cudaError_t e = cudaSuccess;
    for (auto& kv : s->batches) {
      Batch& b = kv.second;
      if (b.members.empty()) continue;
      orders.push_back(kv.first);
      if (!b.tuned && b.pe.M >= 0) e = tune_batch(s, b);
      if (e != cudaSuccess) break;
      if (b.dirty) {
        bool grown = false;
        e = rebuild(s, b, &grown);
        if (grown) s->graph_valid = false;
      }
      if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess && orders.empty()) continue;
    if (e == cudaSuccess && (!s->graph_valid || orders != s->graph_orders)) e = capture_tick(s);
    const auto t0 = Clock::now();
    if (e == cudaSuccess) e = cudaGraphLaunch(s->exec, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    const auto t1 = Clock::now();
    if (e != cudaSuccess) {
      fail_everything(s, std::string("tick: ") + cudaGetErrorString(e));
      return;
    }
    // bookkeeping and retirement
    int64_t in_tick = 0;
    double pi = 0;
    for (auto& kv : s->batches) {
      Batch& b = kv.second;
      if (b.members.empty()) continue;
      in_tick += (int64_t)b.members.size();
      pi += 4.0 * (double)b.pairs_per_rhs;
      b.bad_host.assign(b.members.size(), 0);
      cudaError_t ce0 = cudaMemcpy(b.bad_host.data(), b.bad.p, b.members.size() * sizeof(int),
                                   cudaMemcpyDeviceToHost);
      if (ce0 != cudaSuccess) {
        fail_everything(s, std::string("divergence flags: ") + cudaGetErrorString(ce0));
        return;
      }
      std::vector<Request*> keep;
      for (size_t i = 0; i < b.members.size(); ++i) {
        Request* r = b.members[i];
        r->steps_done += 1;
        r->t = r->t + r->dt;  // the device does the same addition
        if (r->steps_done < r->nsteps && !b.bad_host[i]) {
          keep.push_back(r);
          continue;
        }
        cudaError_t ce = cudaMemcpy(r->x.data(), r->d_state, r->x.size() * sizeof(double),
                                    cudaMemcpyDeviceToHost);
        if (ce == cudaSuccess)
          ce = cudaMemcpy(r->m.data(), r->d_state + 2 * r->n, r->m.size() * sizeof(double),
                          cudaMemcpyDeviceToHost);
        cudaFree(r->d_state);
        r->d_state = nullptr;
        int status = MMVM_OK;
        std::string msg;
        if (ce != cudaSuccess) {
          status = MMVM_E_DEVICE;
          msg = std::string("result copy: ") + cudaGetErrorString(ce);
        } else {
          for (double v : r->x)
            if (!std::isfinite(v)) status = MMVM_E_NUMERIC;
          for (double v : r->m)
            if (!std::isfinite(v)) status = MMVM_E_NUMERIC;
          if (status != MMVM_OK) msg = "non-finite value in the state";
        }
        std::lock_guard<std::mutex> lk(s->mu);
        finish_request(s, r, status, msg);
      }
      if (keep.size() != b.members.size()) {
        b.members.swap(keep);
        b.dirty = true;
      }
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->ticks += 1;
      s->pair_interactions += pi;
      s->busy_ms += ms_between(t0, t1);
      s->max_batch = std::max(s->max_batch, in_tick);
    }
    s->cv.notify_all();
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
  if (cfg->flags != 0) return fail(MMVM_E_INVALID_ARG, "unknown flag bits");
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
      (e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreate(&s->ev0)) != cudaSuccess ||
      (e = cudaEventCreate(&s->ev1)) != cudaSuccess) {
    if (s->st) cudaStreamDestroy(s->st);
    if (s->fork) cudaEventDestroy(s->fork);
    if (s->ev0) cudaEventDestroy(s->ev0);
    if (s->ev1) cudaEventDestroy(s->ev1);
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
  cudaStreamSynchronize(s->st);
  for (auto& kv : s->batches) {
    for (Request* r : kv.second.members)
      if (r->d_state) cudaFree(r->d_state);
    kv.second.release();
  }
  if (s->exec) cudaGraphExecDestroy(s->exec);
  for (cudaEvent_t ev : s->join) cudaEventDestroy(ev);
  cudaEventDestroy(s->fork);
  cudaEventDestroy(s->ev0);
  cudaEventDestroy(s->ev1);
  cudaStreamDestroy(s->st);
  for (auto& kv : s->all) delete kv.second;
  delete s;
}

int mmvm_submit(mmvm_server* s, const mmvm_request* q, uint64_t* ticket) {
  if (!s || !q || !ticket) return fail(MMVM_E_INVALID_ARG, "null argument");
  if (q->order < 0 || q->order > MMVM_MAX_ORDER_SINGLE)
    return fail(MMVM_E_UNSUPPORTED, "order above MMVM_MAX_ORDER_SINGLE");
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
  out->pair_interactions = s->pair_interactions;
  out->busy_ms = s->busy_ms;
  out->footprint_bytes = s->fp_used;
  out->peak_footprint_bytes = s->fp_peak;
  out->budget_bytes = s->budget;
  return s->broken ? fail(MMVM_E_DEVICE, s->broken_msg) : MMVM_OK;
}

}  // extern "C"
