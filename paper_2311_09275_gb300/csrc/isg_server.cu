// isg_server.cu -- continuous-batching annealing server.
//
// A native worker thread owns the server's non-blocking streams.  Requests wait in a
// queue until a slot is free and their device state fits the memory budget;
// then their state is allocated and they join the active set.  Every
// iteration runs one chunk of sweeps for all active requests with the
// persistent unit kernels (torus replica words, graph replica words and CSR
// replica quads, the three kinds on concurrent streams; one CTA per unit,
// longest instances first), reads back each unit's stop sweep,
// retires requests that reached their target or sweep budget, and admits new
// ones.  Requests of different sizes and sweep positions therefore share each
// launch.
//
// Exactness: a request whose replicas span several units (e.g. 32 replicas =
// 8 CSR quads) must stop at the first sweep t* at which its best energy over
// ALL replicas reaches the target.  Units run independently inside a chunk,
// each stopping at its own hit, so before such a chunk the request's state is
// copied aside; if some unit hits at t*, the state is restored and all units
// re-run from the chunk start to t* + 1.  Results are therefore identical to
// isg_anneal of the same request, alone.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <climits>
#include <cstdint>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "isg.h"
#include "isg_kernels.h"
#include "isg_runtime.h"

namespace isg {
namespace {

struct Request {
  uint64_t id = 0;
  const isg_problem *p = nullptr;
  int32_t R = 0, S = 0;
  std::vector<double> betas;
  uint64_t seed = 0;
  int64_t target = ISG_NO_TARGET;
  size_t bytes = 0;
};

struct Slot {
  Request rq;
  isg_result *res = nullptr;
  const DeviceProblem *dp = nullptr;
  int32_t t = 0;         // sweeps completed
  int32_t t_end = 0;     // end of the current chunk
  void *snap = nullptr;  // state copy at the chunk start (multi-unit requests with a target)
  size_t state_bytes = 0;
  int32_t stop = -1;
  bool finished = false;
  bool cancelled = false;  // retired by isg_server_cancel, without a result
};

constexpr int kServeThreads = 512;

size_t state_bytes_of(const isg_result *r) {
  // spins, best, e_cur, e_best are the leading, contiguous part of the allocation
  return (size_t)((char *)r->d_hit - (char *)r->base);
}

size_t request_bytes(const isg_problem *p, int32_t R, int32_t S) {
  const bool msc = p->torus || served_graph_msc(p, kServeThreads);
  const size_t units = msc ? (R + 31) / 32 : (R + 3) / 4;
  const size_t lanes = units * (msc ? 32 : 4);
  const size_t levels = p->torus ? 2 : (size_t)p->kmax + 1;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t b = 2 * al(4 * units * p->n) + 2 * al(4 * lanes) + 2 * al(4 * units) + al(4) +
             2 * al((size_t)R * p->n) + al(4 * levels * S);
  if (units > 1) b += 2 * al(4 * units * p->n) + 2 * al(4 * lanes);  // snapshot
  return b;
}

}  // namespace
}  // namespace isg

using namespace isg;

struct isg_server {
  int device = 0;
  size_t budget = 0;
  int32_t max_slots = 0, chunk = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> queue;
  std::deque<std::pair<uint64_t, isg_result *>> done;
  bool stopping = false;
  uint64_t next_id = 1;
  std::thread worker;
  // worker-owned; the graph unit kernels run on side streams, concurrently with
  // the torus unit kernel, joined back into `stream` by events
  cudaStream_t stream = nullptr;
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t ev_in = nullptr, ev_side[2] = {nullptr, nullptr};
  // pass balancing: each unit kind's kernel time in the last pass (timing
  // events) sets its sweeps-per-chunk factor so that all kinds end together
  cudaEvent_t ev_k0[3] = {nullptr, nullptr, nullptr}, ev_k1[3] = {nullptr, nullptr, nullptr};
  bool kind_timed[3] = {false, false, false};
  double kind_scale[3] = {1.0, 1.0, 1.0};
  std::vector<Slot *> active;
  size_t used = 0;
  size_t cap_t = 0, cap_c = 0, cap_g = 0;
  GraphMscItem *d_g = nullptr, *h_g = nullptr;
  int32_t *d_ord_g = nullptr, *h_ord_g = nullptr;
  TorusBatchItem *d_t = nullptr, *h_t = nullptr;
  CsrBatchItem *d_c = nullptr, *h_c = nullptr;
  int32_t *d_ord_t = nullptr, *h_ord_t = nullptr, *d_ord_c = nullptr, *h_ord_c = nullptr;
  // [0] next_t, [1] next_c, [2] count_t, [3] count_c, [4] next_g, [5] count_g
  int32_t *d_ctl = nullptr, *h_ctl = nullptr;
  int32_t *h_status = nullptr;                 // per unit: hit, done
  size_t cap_status = 0;
  isg_status worker_error = ISG_OK;
  // counters (under mu)
  int64_t n_submitted = 0, n_completed = 0, n_passes = 0, n_replays = 0, n_cancelled = 0;
  std::set<uint64_t> live;     // admitted requests not yet handed back
  std::set<uint64_t> cancels;  // of those, the ones to retire at the next chunk boundary
  int32_t n_active = 0, peak_active = 0;
};

namespace isg {
namespace {

cudaError_t grow(isg_server *s, size_t nt, size_t nc, size_t nstatus, size_t ng = 0) {
  cudaError_t err = cudaSuccess;
  if (ng > s->cap_g) {
    const size_t cap = std::max(ng, 2 * s->cap_g);
    cudaFree(s->d_g);
    cudaFreeHost(s->h_g);
    cudaFree(s->d_ord_g);
    cudaFreeHost(s->h_ord_g);
    err = cudaMalloc(&s->d_g, sizeof(GraphMscItem) * cap);
    if (err == cudaSuccess) err = cudaMallocHost(&s->h_g, sizeof(GraphMscItem) * cap);
    if (err == cudaSuccess) err = cudaMalloc(&s->d_ord_g, 4 * cap);
    if (err == cudaSuccess) err = cudaMallocHost(&s->h_ord_g, 4 * cap);
    if (err != cudaSuccess) return err;
    s->cap_g = cap;
  }
  if (nt > s->cap_t) {
    const size_t cap = std::max(nt, 2 * s->cap_t);
    cudaFree(s->d_t);
    cudaFreeHost(s->h_t);
    cudaFree(s->d_ord_t);
    cudaFreeHost(s->h_ord_t);
    err = cudaMalloc(&s->d_t, sizeof(TorusBatchItem) * cap);
    if (err == cudaSuccess) err = cudaMallocHost(&s->h_t, sizeof(TorusBatchItem) * cap);
    if (err == cudaSuccess) err = cudaMalloc(&s->d_ord_t, 4 * cap);
    if (err == cudaSuccess) err = cudaMallocHost(&s->h_ord_t, 4 * cap);
    if (err != cudaSuccess) return err;
    s->cap_t = cap;
  }
  if (nc > s->cap_c) {
    const size_t cap = std::max(nc, 2 * s->cap_c);
    cudaFree(s->d_c);
    cudaFreeHost(s->h_c);
    cudaFree(s->d_ord_c);
    cudaFreeHost(s->h_ord_c);
    err = cudaMalloc(&s->d_c, sizeof(CsrBatchItem) * cap);
    if (err == cudaSuccess) err = cudaMallocHost(&s->h_c, sizeof(CsrBatchItem) * cap);
    if (err == cudaSuccess) err = cudaMalloc(&s->d_ord_c, 4 * cap);
    if (err == cudaSuccess) err = cudaMallocHost(&s->h_ord_c, 4 * cap);
    if (err != cudaSuccess) return err;
    s->cap_c = cap;
  }
  if (nstatus > s->cap_status) {
    const size_t cap = std::max(nstatus, 2 * s->cap_status);
    cudaFreeHost(s->h_status);
    err = cudaMallocHost(&s->h_status, 4 * cap);
    if (err != cudaSuccess) return err;
    s->cap_status = cap;
  }
  return err;
}

// Device memory an admission leaves free for everything else on the device
// (the CUDA context's own needs, other streams' allocations).
constexpr size_t kFreeHeadroom = size_t(256) << 20;

// Admit queued requests while a slot and memory are free (worker thread): the
// request's state must fit the server's budget and the device's free memory
// (queried once per admission round, less the headroom).  With nothing
// resident a request is admitted regardless; if its allocation then fails it
// is handed back with ISG_ENOMEM.
void admit(isg_server *s) {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    free_b = SIZE_MAX;  // unknown: the budget alone decides
  }
  for (;;) {
    Request rq;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      if (s->queue.empty() || (int32_t)s->active.size() >= s->max_slots) return;
      const size_t need = s->queue.front().bytes;
      if (!s->active.empty() &&
          (s->used + need > s->budget || need > free_b || free_b - need < kFreeHeadroom))
        return;
      rq = std::move(s->queue.front());
      s->queue.pop_front();
      s->live.insert(rq.id);  // cancellable from here on
    }
    free_b = rq.bytes < free_b ? free_b - rq.bytes : 0;
    Slot *sl = new Slot();
    sl->rq = std::move(rq);
    const isg_problem *p = sl->rq.p;
    isg_result *r = new isg_result();
    r->device = s->device;
    r->n = p->n;
    r->R = sl->rq.R;
    r->S = sl->rq.S;
    r->has_target = sl->rq.target != ISG_NO_TARGET;
    // graphs with +-1 weights whose units fit the unit kernel's counters run
    // multi-spin coded (one unit per 32 replicas), other graphs as int8 quads
    const bool gm = !p->torus && served_graph_msc(p, kServeThreads);
    r->msc = p->torus || gm;
    r->relabelled = !p->torus;
    r->kernel = p->torus ? ISG_KERNEL_TORUS_MSC : (gm ? ISG_KERNEL_GRAPH_MSC : ISG_KERNEL_CSR);
    r->units = r->msc ? (r->R + 31) / 32 : (r->R + 3) / 4;
    r->lanes = r->msc ? 32 : 4;
    std::vector<int32_t> levels;
    if (p->torus)
      levels = {2, 4};
    else
      for (int32_t k = 0; k <= p->kmax; ++k) levels.push_back(k);
    std::vector<uint32_t> table;
    build_table(sl->rq.betas.data(), sl->rq.S, levels, table);
    r->table_words = table.size();
    isg_status st = problem_device(p, p->torus ? kNeedTorus : kNeedCsr, &sl->dp);
    if (st == ISG_OK) st = result_alloc(r, s->stream);
    cudaError_t err = cudaSuccess;
    if (st == ISG_OK) {
      err = cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming);
      if (err == cudaSuccess)
        err = cudaMemcpyAsync(r->d_table, table.data(), 4 * table.size(), cudaMemcpyHostToDevice,
                              s->stream);
      if (err == cudaSuccess)
        err = cudaMemsetAsync(r->d_hit, 0xFF, 4 * (size_t)r->units, s->stream);
      sl->state_bytes = state_bytes_of(r);
      if (err == cudaSuccess && r->units > 1 && r->has_target)
        err = cudaMallocAsync(&sl->snap, sl->state_bytes, s->stream);
      if (err != cudaSuccess) st = cuda_fail(err, "admitting a request");
    }
    sl->res = r;
    if (st != ISG_OK) {
      // cannot run it: hand back an empty result that reports the failure
      r->synced = true;
      r->sync_status = st;
      if (sl->snap) cudaFreeAsync(sl->snap, s->stream);
      std::lock_guard<std::mutex> lock(s->mu);
      s->live.erase(sl->rq.id);
      if (s->cancels.erase(sl->rq.id)) {  // cancelled while its admission failed
        r->sync_status = ISG_ECANCELLED;
        ++s->n_cancelled;
      }
      s->done.emplace_back(sl->rq.id, r);
      ++s->n_completed;
      s->cv_done.notify_all();
      delete sl;
      continue;
    }
    r->ctas = 0;
    r->cluster = 1;
    r->threads = kServeThreads;
    s->used += sl->rq.bytes;
    s->active.push_back(sl);
    std::lock_guard<std::mutex> lock(s->mu);
    s->n_active = (int32_t)s->active.size();
    s->peak_active = std::max(s->peak_active, s->n_active);
  }
}

void fill_torus_unit(TorusBatchItem &it, const Slot *sl, int32_t word, int32_t t_begin,
                     int32_t t_end) {
  const isg_result *r = sl->res;
  const isg_problem *p = sl->rq.p;
  TorusSolve &s = it.solve;
  s = {};
  s.L = p->L;
  s.W = p->W;
  s.cbits = sl->dp->cbits;
  s.table = r->d_table;
  s.table_ws = 0;
  s.table_ts = 2;
  s.key0 = (uint32_t)(sl->rq.seed & 0xFFFFFFFFu);
  s.key1 = (uint32_t)(sl->rq.seed >> 32);
  s.rk = round_keys(s.key0, s.key1);
  s.words = r->units;
  s.replicas = r->R;
  s.spins = r->d_spins;
  s.best = r->d_best;
  s.e_cur = r->d_e_cur;
  s.e_best = r->d_e_best;
  s.hit = r->d_hit;
  s.done = r->d_done;
  s.has_target = r->has_target;
  s.target = r->has_target ? (int32_t)sl->rq.target : 0;
  it.word = word;
  it.t_begin = t_begin;
  it.t_end = t_end;
  it.resume = t_begin > 0;
  it.stop_from_hits = 0;
  it.out = nullptr;
  it.out_best = nullptr;
  it.stop = nullptr;
}

void fill_csr_unit(CsrBatchItem &it, const Slot *sl, int32_t quad, int32_t t_begin, int32_t t_end) {
  const isg_result *r = sl->res;
  const isg_problem *p = sl->rq.p;
  CsrSolve &s = it.solve;
  s = {};
  s.n = p->n;
  s.n_colours = p->n_colours;
  s.class_start = sl->dp->class_start;
  s.rowptr = sl->dp->rowptr;
  s.col = sl->dp->col;
  s.wt = sl->dp->wt;
  s.orig = sl->dp->orig;
  s.field = sl->dp->field_r;
  s.kmax = p->kmax;
  s.table = r->d_table;
  s.key0 = (uint32_t)(sl->rq.seed & 0xFFFFFFFFu);
  s.key1 = (uint32_t)(sl->rq.seed >> 32);
  s.quads = r->units;
  s.replicas = r->R;
  s.spins = r->d_spins;
  s.best = r->d_best;
  s.e_cur = r->d_e_cur;
  s.e_best = r->d_e_best;
  s.hit = r->d_hit;
  s.done = r->d_done;
  s.has_target = r->has_target;
  s.target = r->has_target ? (int32_t)sl->rq.target : 0;
  s.mode = p->mode;
  it.quad = quad;
  it.t_begin = t_begin;
  it.t_end = t_end;
  it.resume = t_begin > 0;
  it.stop_from_hits = 0;
}

void fill_gm_unit(GraphMscItem &it, const Slot *sl, int32_t word, int32_t t_begin, int32_t t_end) {
  const isg_result *r = sl->res;
  const isg_problem *p = sl->rq.p;
  GraphMscSolve &s = it.solve;
  s = {};
  s.n = p->n;
  s.n_colours = p->n_colours;
  s.class_start = sl->dp->class_start;
  s.rowptr = sl->dp->rowptr;
  s.col = sl->dp->col;
  s.orig = sl->dp->orig;
  s.field = sl->dp->field_r;
  s.table = r->d_table;
  s.kmax1 = p->kmax + 1;
  s.table_ws = 0;
  s.table_ts = s.kmax1;
  s.key0 = (uint32_t)(sl->rq.seed & 0xFFFFFFFFu);
  s.key1 = (uint32_t)(sl->rq.seed >> 32);
  s.rk = round_keys(s.key0, s.key1);
  s.words = r->units;
  s.replicas = r->R;
  s.spins = r->d_spins;
  s.best = r->d_best;
  s.e_cur = r->d_e_cur;
  s.e_best = r->d_e_best;
  s.hit = r->d_hit;
  s.done = r->d_done;
  s.has_target = r->has_target;
  s.target = r->has_target ? (int32_t)sl->rq.target : 0;
  it.word = word;
  it.t_begin = t_begin;
  it.t_end = t_end;
  it.resume = t_begin > 0;
  it.stop_from_hits = 0;
}

// Unit kind of a slot: 0 torus words, 1 graph words, 2 graph quads.
int kind_of(const Slot *sl) { return sl->res->msc ? (sl->res->relabelled ? 1 : 0) : 2; }

// One launch of the unit kernels over the listed slots, sweeps [t, t_end) each;
// with `timed`, each kind's kernel is bracketed by timing events.
cudaError_t run_units(isg_server *s, const std::vector<Slot *> &slots,
                      const std::vector<int32_t> &t_end, bool timed = false) {
  size_t nt = 0, nc = 0, ng = 0;
  for (size_t k = 0; k < slots.size(); ++k) {
    const isg_result *r = slots[k]->res;
    (r->msc ? (r->relabelled ? ng : nt) : nc) += r->units;
  }
  cudaError_t err = grow(s, nt, nc, 0, ng);
  if (err != cudaSuccess) return err;
  size_t it = 0, ic = 0, ig = 0;
  size_t smem_t = 0, smem_c = 0, smem_g = 0;
  std::vector<std::pair<int32_t, int32_t>> ord_t, ord_c, ord_g;  // (size, index)
  for (size_t k = 0; k < slots.size(); ++k) {
    Slot *sl = slots[k];
    const isg_problem *p = sl->rq.p;
    for (int32_t u = 0; u < sl->res->units; ++u) {
      if (sl->res->msc && !sl->res->relabelled) {
        fill_torus_unit(s->h_t[it], sl, u, sl->t, t_end[k]);
        ord_t.emplace_back(p->n, (int32_t)it++);
        smem_t = std::max(smem_t, torus_batch_max_smem(p->L, p->W));
      } else if (sl->res->msc) {
        fill_gm_unit(s->h_g[ig], sl, u, sl->t, t_end[k]);
        ord_g.emplace_back(p->n, (int32_t)ig++);
        smem_g = std::max(smem_g, gm_smem_bytes(p->n, 1, p->n_colours, 0, 0, 0, p->kmax + 1,
                                                !p->field.empty()));
      } else {
        fill_csr_unit(s->h_c[ic], sl, u, sl->t, t_end[k]);
        ord_c.emplace_back(p->n, (int32_t)ic++);
        smem_c = std::max(smem_c, csr_smem_bytes(p->n, 1, 1, p->n_colours, 0, 0, p->mode, p->kmax));
      }
    }
  }
  auto by_size = [](const std::pair<int32_t, int32_t> &a, const std::pair<int32_t, int32_t> &b) {
    return a.first > b.first || (a.first == b.first && a.second < b.second);
  };
  std::sort(ord_t.begin(), ord_t.end(), by_size);
  std::sort(ord_c.begin(), ord_c.end(), by_size);
  std::sort(ord_g.begin(), ord_g.end(), by_size);
  for (size_t k = 0; k < ord_t.size(); ++k) s->h_ord_t[k] = ord_t[k].second;
  for (size_t k = 0; k < ord_c.size(); ++k) s->h_ord_c[k] = ord_c[k].second;
  for (size_t k = 0; k < ord_g.size(); ++k) s->h_ord_g[k] = ord_g[k].second;
  s->h_ctl[0] = 0;
  s->h_ctl[1] = 0;
  s->h_ctl[2] = (int32_t)nt;
  s->h_ctl[3] = (int32_t)nc;
  s->h_ctl[4] = 0;
  s->h_ctl[5] = (int32_t)ng;
  const int threads = kServeThreads;
  if (nt) {
    err = cudaMemcpyAsync(s->d_t, s->h_t, sizeof(TorusBatchItem) * nt, cudaMemcpyHostToDevice,
                          s->stream);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(s->d_ord_t, s->h_ord_t, 4 * nt, cudaMemcpyHostToDevice, s->stream);
  }
  if (err == cudaSuccess && nc) {
    err = cudaMemcpyAsync(s->d_c, s->h_c, sizeof(CsrBatchItem) * nc, cudaMemcpyHostToDevice,
                          s->stream);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(s->d_ord_c, s->h_ord_c, 4 * nc, cudaMemcpyHostToDevice, s->stream);
  }
  if (err == cudaSuccess && ng) {
    err = cudaMemcpyAsync(s->d_g, s->h_g, sizeof(GraphMscItem) * ng, cudaMemcpyHostToDevice,
                          s->stream);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(s->d_ord_g, s->h_ord_g, 4 * ng, cudaMemcpyHostToDevice, s->stream);
  }
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(s->d_ctl, s->h_ctl, 24, cudaMemcpyHostToDevice, s->stream);
  auto ctas_for = [](size_t units, size_t smem) {
    const int per_sm = std::max(1, std::min<int>(4, (int)((228 * 1024) / (smem + 1024))));
    return (int)std::min<size_t>(units, (size_t)sm_count() * per_sm);
  };
  // the three unit kinds run concurrently (each fills the SMs the others leave)
  for (int k = 0; k < 3; ++k) s->kind_timed[k] = false;
  auto mark = [&](int k, bool begin, cudaStream_t st) {
    if (!timed || err != cudaSuccess) return;
    err = cudaEventRecord(begin ? s->ev_k0[k] : s->ev_k1[k], st);
    if (!begin && err == cudaSuccess) s->kind_timed[k] = true;
  };
  if (err == cudaSuccess && (ng || nc)) err = cudaEventRecord(s->ev_in, s->stream);
  if (err == cudaSuccess && ng) {
    err = cudaStreamWaitEvent(s->side[0], s->ev_in, 0);
    mark(1, true, s->side[0]);
    if (err == cudaSuccess)
      err = gm_batch_launch(s->d_g, s->d_ctl + 5, s->d_ord_g, s->d_ctl + 4, ctas_for(ng, smem_g),
                            threads, smem_g, s->side[0]);
    mark(1, false, s->side[0]);
    if (err == cudaSuccess) err = cudaEventRecord(s->ev_side[0], s->side[0]);
  }
  if (err == cudaSuccess && nc) {
    err = cudaStreamWaitEvent(s->side[1], s->ev_in, 0);
    mark(2, true, s->side[1]);
    if (err == cudaSuccess)
      err = csr_batch_launch(s->d_c, s->d_ctl + 3, s->d_ord_c, s->d_ctl + 1, ctas_for(nc, smem_c),
                             threads, smem_c, s->side[1]);
    mark(2, false, s->side[1]);
    if (err == cudaSuccess) err = cudaEventRecord(s->ev_side[1], s->side[1]);
  }
  if (err == cudaSuccess && nt) {
    mark(0, true, s->stream);
    err = torus_batch_launch(s->d_t, s->d_ctl + 2, s->d_ord_t, s->d_ctl + 0, ctas_for(nt, smem_t),
                             threads, smem_t, s->stream);
    mark(0, false, s->stream);
  }
  if (err == cudaSuccess && ng) err = cudaStreamWaitEvent(s->stream, s->ev_side[0], 0);
  if (err == cudaSuccess && nc) err = cudaStreamWaitEvent(s->stream, s->ev_side[1], 0);
  for (Slot *sl : slots) sl->res->sweep_launches += 1;
  return err;
}

// After a timed pass: scale each kind's chunk so that its kernel would have
// taken as long as the slowest kind's (bounded steps, bounded factors).
void balance_kinds(isg_server *s) {
  float ms[3] = {0.f, 0.f, 0.f}, mx = 0.f;
  int n = 0;
  for (int k = 0; k < 3; ++k) {
    if (!s->kind_timed[k]) continue;
    if (cudaEventElapsedTime(&ms[k], s->ev_k0[k], s->ev_k1[k]) != cudaSuccess || ms[k] <= 0.f) {
      s->kind_timed[k] = false;
      continue;
    }
    mx = std::max(mx, ms[k]);
    ++n;
  }
  if (n < 2) return;
  for (int k = 0; k < 3; ++k) {
    if (!s->kind_timed[k]) continue;
    const double f = std::min(4.0, std::max(0.5, (double)mx / ms[k]));
    s->kind_scale[k] = std::min(64.0, std::max(1.0 / 16, s->kind_scale[k] * f));
  }
}

cudaError_t finish_slot(isg_server *s, Slot *sl) {
  isg_result *r = sl->res;
  cudaError_t err = cudaSuccess;
  int32_t *stop_host = &sl->stop;
  err = cudaMemcpyAsync(r->d_stop, stop_host, 4, cudaMemcpyHostToDevice, s->stream);
  if (err == cudaSuccess) {
    if (r->msc && !r->relabelled) {
      err = unpack_msc(r->d_spins, r->n, r->R, r->d_out, s->stream);
      if (err == cudaSuccess) err = unpack_msc(r->d_best, r->n, r->R, r->d_out_best, s->stream);
    } else if (r->msc) {
      err = unpack_msc_relabel(r->d_spins, r->n, r->R, sl->dp->orig, r->d_out, s->stream);
      if (err == cudaSuccess)
        err = unpack_msc_relabel(r->d_best, r->n, r->R, sl->dp->orig, r->d_out_best, s->stream);
    } else {
      err = unpack_quads(r->d_spins, r->n, r->R, sl->dp->orig, r->d_out, s->stream);
      if (err == cudaSuccess)
        err = unpack_quads(r->d_best, r->n, r->R, sl->dp->orig, r->d_out_best, s->stream);
    }
  }
  r->launches = r->sweep_launches + 2;
  if (err == cudaSuccess) err = cudaEventRecord(r->done, s->stream);
  return err;
}

void worker_main(isg_server *s) {
  cudaSetDevice(s->device);
  for (;;) {
    admit(s);
    {
      std::unique_lock<std::mutex> lock(s->mu);
      if (s->stopping) break;
      if (s->active.empty()) {
        s->cv_work.wait_for(lock, std::chrono::milliseconds(20));
        continue;
      }
    }
    // one chunk for every active request
    std::vector<int32_t> t_end(s->active.size());
    cudaError_t err = cudaSuccess;
    size_t nstatus = 0;
    for (size_t k = 0; k < s->active.size(); ++k) {
      Slot *sl = s->active[k];
      // sweeps_per_chunk is the count for a 10,000-spin instance, scaled by
      // the inverse square root of the instance size (a larger instance does
      // more work per pass, so its time-to-target does not grow in proportion
      // to its size) and by the unit kind's balance factor
      const int64_t sweeps = std::max<int64_t>(
          1, (int64_t)((double)s->chunk * std::sqrt(10000.0 / sl->rq.p->n) *
                       s->kind_scale[kind_of(sl)]));
      t_end[k] = (int32_t)std::min<int64_t>(sl->t + sweeps, sl->rq.S);
      sl->t_end = t_end[k];
      nstatus += 2 * (size_t)sl->res->units;
      if (sl->snap && err == cudaSuccess)
        err = cudaMemcpyAsync(sl->snap, sl->res->base, sl->state_bytes, cudaMemcpyDeviceToDevice,
                              s->stream);
    }
    if (err == cudaSuccess) err = grow(s, 0, 0, nstatus);
    if (err == cudaSuccess) err = run_units(s, s->active, t_end, true);
    {
      std::lock_guard<std::mutex> lock(s->mu);
      ++s->n_passes;
    }
    size_t off = 0;
    for (Slot *sl : s->active) {
      const int32_t u = sl->res->units;
      if (err == cudaSuccess)
        err = cudaMemcpyAsync(s->h_status + off, sl->res->d_hit, 4 * (size_t)u,
                              cudaMemcpyDeviceToHost, s->stream);
      if (err == cudaSuccess)
        err = cudaMemcpyAsync(s->h_status + off + u, sl->res->d_done, 4 * (size_t)u,
                              cudaMemcpyDeviceToHost, s->stream);
      off += 2 * (size_t)u;
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(s->stream);
    if (err == cudaSuccess) balance_kinds(s);
    if (err != cudaSuccess) {
      s->worker_error = cuda_fail(err, "server chunk");
      std::lock_guard<std::mutex> lock(s->mu);
      s->stopping = true;
      s->cv_done.notify_all();
      break;
    }
    // decide per request; collect the multi-unit requests that must re-run to t*
    std::vector<Slot *> redo;
    std::vector<int32_t> redo_end;
    {
      // Decided under the lock: a cancel that arrives before this block applies
      // in this chunk; one that arrives after it finds a request finished here
      // no longer live (EINVAL, normal result) and one still running queued for
      // the next chunk.
      std::lock_guard<std::mutex> lock(s->mu);
      off = 0;
      for (Slot *sl : s->active) {
        const int32_t u = sl->res->units;
        int32_t tstar = INT_MAX;
        for (int32_t q = 0; q < u; ++q)
          if (s->h_status[off + q] >= 0) tstar = std::min(tstar, s->h_status[off + q]);
        off += 2 * (size_t)u;
        if (s->cancels.erase(sl->rq.id)) {
          sl->cancelled = true;
          sl->finished = true;
        } else if (sl->res->has_target && tstar != INT_MAX) {
          sl->stop = tstar;
          sl->finished = true;
          if (u > 1) {
            redo.push_back(sl);
            redo_end.push_back(tstar + 1);
          }
        } else if (sl->t_end >= sl->rq.S) {
          sl->stop = -1;
          sl->finished = true;
        } else {
          sl->t = sl->t_end;
        }
        if (sl->finished) s->live.erase(sl->rq.id);
      }
    }
    if (!redo.empty()) {
      for (Slot *sl : redo) {
        if (err == cudaSuccess)
          err = cudaMemcpyAsync(sl->res->base, sl->snap, sl->state_bytes, cudaMemcpyDeviceToDevice,
                                s->stream);
        if (err == cudaSuccess)
          err = cudaMemsetAsync(sl->res->d_hit, 0xFF, 4 * (size_t)sl->res->units, s->stream);
      }
      if (err == cudaSuccess) err = run_units(s, redo, redo_end);
      std::lock_guard<std::mutex> lock(s->mu);
      ++s->n_replays;
    }
    std::vector<Slot *> keep;
    std::vector<Slot *> fin;
    for (Slot *sl : s->active) (sl->finished ? fin : keep).push_back(sl);
    for (Slot *sl : fin)
      if (err == cudaSuccess && !sl->cancelled) err = finish_slot(s, sl);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s->stream);
    if (err != cudaSuccess) {
      s->worker_error = cuda_fail(err, "server retire");
      std::lock_guard<std::mutex> lock(s->mu);
      s->stopping = true;
      s->cv_done.notify_all();
      break;
    }
    for (Slot *sl : fin) {
      if (sl->snap) cudaFreeAsync(sl->snap, s->stream);
      s->used -= sl->rq.bytes;
      if (sl->cancelled) {
        // handed back without state: its reads return ISG_ECANCELLED
        cudaFreeAsync(sl->res->base, s->stream);
        sl->res->base = nullptr;
        sl->res->synced = true;
        sl->res->sync_status = ISG_ECANCELLED;
      }
      sl->res->stream = nullptr;  // later frees go to the legacy stream
      std::lock_guard<std::mutex> lock(s->mu);
      s->done.emplace_back(sl->rq.id, sl->res);
      ++s->n_completed;
      if (sl->cancelled) ++s->n_cancelled;
      delete sl;
    }
    s->active.swap(keep);
    {
      std::lock_guard<std::mutex> lock(s->mu);
      s->n_active = (int32_t)s->active.size();
    }
    if (!fin.empty()) s->cv_done.notify_all();
  }
}

}  // namespace
}  // namespace isg

extern "C" {

isg_status isg_server_create(size_t device_mem_budget, int32_t max_slots, int32_t sweeps_per_chunk,
                             isg_server **out) {
  if (!out) return fail(ISG_EINVAL, "out must not be NULL");
  *out = nullptr;
  if (max_slots < 1) return fail(ISG_EINVAL, "max_slots must be >= 1");
  if (sweeps_per_chunk < 1) return fail(ISG_EINVAL, "sweeps_per_chunk must be >= 1");
  if (device_mem_budget == 0) return fail(ISG_EINVAL, "device_mem_budget must be > 0");
  isg_server *s = new isg_server();
  s->budget = device_mem_budget;
  s->max_slots = max_slots;
  s->chunk = sweeps_per_chunk;
  cudaError_t err = cudaGetDevice(&s->device);
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  for (int i = 0; i < 2 && err == cudaSuccess; ++i) {
    err = cudaStreamCreateWithFlags(&s->side[i], cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&s->ev_side[i], cudaEventDisableTiming);
  }
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming);
  for (int k = 0; k < 3 && err == cudaSuccess; ++k) {
    err = cudaEventCreate(&s->ev_k0[k]);
    if (err == cudaSuccess) err = cudaEventCreate(&s->ev_k1[k]);
  }
  if (err == cudaSuccess) err = cudaMalloc(&s->d_ctl, 64);
  if (err == cudaSuccess) err = cudaMallocHost(&s->h_ctl, 64);
  if (err != cudaSuccess) {
    if (s->stream) cudaStreamDestroy(s->stream);
    for (int i = 0; i < 2; ++i) {
      if (s->side[i]) cudaStreamDestroy(s->side[i]);
      if (s->ev_side[i]) cudaEventDestroy(s->ev_side[i]);
    }
    if (s->ev_in) cudaEventDestroy(s->ev_in);
    for (int k = 0; k < 3; ++k) {
      if (s->ev_k0[k]) cudaEventDestroy(s->ev_k0[k]);
      if (s->ev_k1[k]) cudaEventDestroy(s->ev_k1[k]);
    }
    cudaFree(s->d_ctl);
    cudaFreeHost(s->h_ctl);
    delete s;
    return cuda_fail(err, "creating the server");
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return ISG_OK;
}

isg_status isg_server_submit(isg_server *s, const isg_problem *p, int32_t replicas,
                             const double *betas, int32_t sweeps, uint64_t seed,
                             int64_t target_energy, uint64_t *request_id) {
  if (!s || !p || !request_id) return fail(ISG_EINVAL, "arguments must not be NULL");
  if (replicas < 1) return fail(ISG_EINVAL, "replicas must be >= 1");
  if (sweeps < 1) return fail(ISG_EINVAL, "sweeps must be >= 1");
  isg_status st = check_betas(betas, sweeps);
  if (st != ISG_OK) return st;
  if (target_energy != ISG_NO_TARGET && (target_energy < INT32_MIN || target_energy > INT32_MAX))
    return fail(ISG_EINVAL, "target energy outside the int32 range");
  if (p->torus ? (p->n / 2 + 255) / 256 > 127
                : csr_smem_bytes(p->n, 1, 1, p->n_colours, 0, 0, p->mode, p->kmax) > 227 * 1024)
    return fail(ISG_EINVAL, "instance too large for the served kernels");
  if (p->torus && torus_batch_max_smem(p->L, p->W) > 227 * 1024)
    return fail(ISG_EINVAL, "torus too large for the served kernels");
  Request rq;
  rq.p = p;
  rq.R = replicas;
  rq.S = sweeps;
  rq.betas.assign(betas, betas + sweeps);
  rq.seed = seed;
  rq.target = target_energy;
  rq.bytes = request_bytes(p, replicas, sweeps);
  if (rq.bytes > s->budget)
    return fail(ISG_EBUSY, "request needs %zu bytes, more than the server budget", rq.bytes);
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->stopping) return fail(ISG_ECANCELLED, "server is shutting down");
  rq.id = s->next_id++;
  *request_id = rq.id;
  ++s->n_submitted;
  s->queue.push_back(std::move(rq));
  s->cv_work.notify_one();
  return ISG_OK;
}

isg_status isg_server_poll(isg_server *s, uint64_t *request_id, isg_result **out, double timeout_s) {
  if (!s || !request_id || !out) return fail(ISG_EINVAL, "arguments must not be NULL");
  std::unique_lock<std::mutex> lock(s->mu);
  const auto deadline =
      std::chrono::steady_clock::now() +
      std::chrono::microseconds((int64_t)(std::max(0.0, timeout_s) * 1e6));
  while (s->done.empty()) {
    if (s->stopping && s->worker_error != ISG_OK)
      return fail(s->worker_error, "server stopped after an error");
    if (s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && s->done.empty())
      return fail(ISG_ETIMEOUT, "no finished request within %g s", timeout_s);
  }
  *request_id = s->done.front().first;
  *out = s->done.front().second;
  s->done.pop_front();
  return ISG_OK;
}

isg_status isg_server_get_stats(isg_server *s, isg_server_stats *out) {
  if (!s || !out) return fail(ISG_EINVAL, "arguments must not be NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  out->submitted = s->n_submitted;
  out->completed = s->n_completed;
  out->queued = (int32_t)s->queue.size();
  out->active = s->n_active;
  out->peak_active = s->peak_active;
  out->passes = s->n_passes;
  out->replays = s->n_replays;
  out->cancelled = s->n_cancelled;
  return ISG_OK;
}

isg_status isg_server_cancel(isg_server *s, uint64_t request_id) {
  if (!s) return fail(ISG_EINVAL, "server must not be NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    if (it->id != request_id) continue;
    // not admitted yet: handed back at once, with no device state
    isg_result *r = new isg_result();
    r->device = s->device;
    r->n = it->p->n;
    r->R = it->R;
    r->S = it->S;
    r->synced = true;
    r->sync_status = ISG_ECANCELLED;
    s->queue.erase(it);
    s->done.emplace_back(request_id, r);
    ++s->n_completed;
    ++s->n_cancelled;
    s->cv_done.notify_all();
    return ISG_OK;
  }
  if (!s->live.count(request_id))
    return fail(ISG_EINVAL, "request %llu is not queued or running (unknown or finished)",
                (unsigned long long)request_id);
  s->cancels.insert(request_id);
  return ISG_OK;
}

isg_status isg_server_destroy(isg_server *s) {
  if (!s) return fail(ISG_EINVAL, "server must not be NULL");
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stopping = true;
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  for (Slot *sl : s->active) {
    if (sl->snap) cudaFreeAsync(sl->snap, s->stream);
    sl->res->stream = s->stream;
    result_free(sl->res);
    delete sl;
  }
  for (auto &d : s->done) {
    d.second->stream = nullptr;
    result_free(d.second);
  }
  cudaStreamSynchronize(s->stream);
  cudaFree(s->d_t);
  cudaFreeHost(s->h_t);
  cudaFree(s->d_c);
  cudaFreeHost(s->h_c);
  cudaFree(s->d_ord_t);
  cudaFreeHost(s->h_ord_t);
  cudaFree(s->d_ord_c);
  cudaFreeHost(s->h_ord_c);
  cudaFree(s->d_g);
  cudaFreeHost(s->h_g);
  cudaFree(s->d_ord_g);
  cudaFreeHost(s->h_ord_g);
  cudaFree(s->d_ctl);
  cudaFreeHost(s->h_ctl);
  cudaFreeHost(s->h_status);
  for (int i = 0; i < 2; ++i) {
    cudaStreamDestroy(s->side[i]);
    cudaEventDestroy(s->ev_side[i]);
  }
  cudaEventDestroy(s->ev_in);
  for (int k = 0; k < 3; ++k) {
    cudaEventDestroy(s->ev_k0[k]);
    cudaEventDestroy(s->ev_k1[k]);
  }
  cudaStreamDestroy(s->stream);
  cudaSetDevice(prev);
  const isg_status st = s->worker_error;
  delete s;
  return st == ISG_OK ? ISG_OK : st;
}

}  // extern "C"
