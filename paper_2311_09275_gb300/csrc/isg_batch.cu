// isg_batch.cu -- many instances in one persistent launch (isg_anneal_batch).
//
// Every instance is cut into work units that one CTA solves from start to
// finish with no cross-CTA synchronisation: the replica words of a torus (32
// replicas each), the replica words of a +-1 graph the multi-spin unit kernel
// takes, and the replica quads (4 each) of any other graph.  The three kinds
// have one persistent kernel each; CTAs take units from a device work counter
// in longest-first order, which keeps the tail short when sizes are uneven,
// and the three kernels run concurrently on forked streams.  An instance with
// a target and several units runs a second pass (the rule of a single solve):
// its units stop at their own hits in the first, and all of them rerun from
// the start to the earliest hit + 1 in the second.  The sequence (counter
// resets, first pass, second pass if any, one batched unpack) is captured
// once into a CUDA graph and launched on the caller's stream.  Each
// instance's result is bit-identical to isg_anneal of it alone: the random
// numbers depend only on (seed, replica, sweep, site), never on which CTA ran
// a unit or when.
//
// Launch shape: threads per CTA and CTAs per SM of the unit kernels, from
// isg_autotune_batch's measurement for the batch's size histogram when there
// is one, else 256 threads and as many CTAs per SM as shared memory allows.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <vector>

#include "isg.h"
#include "isg_kernels.h"
#include "isg_runtime.h"

namespace isg {
namespace {

struct BatchBlock {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr, side[2] = {nullptr, nullptr};
  cudaEvent_t fork[2] = {nullptr, nullptr}, join[4] = {nullptr, nullptr, nullptr, nullptr};
  void *mem = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

void free_block(BatchBlock *b) {
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  if (b->mem) cudaFreeAsync(b->mem, b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaEvent_t e : b->fork)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : b->side)
    if (s) cudaStreamDestroy(s);
  if (b->capture) cudaStreamDestroy(b->capture);
  cudaSetDevice(prev);
  delete b;
}

constexpr int kTorusKind = 0, kGraphWordKind = 1, kQuadKind = 2;

// Unit kind of an instance under `threads` threads per CTA.
int kind_of(const isg_problem *p, int threads) {
  if (p->torus) return kTorusKind;
  return served_graph_msc(p, threads) ? kGraphWordKind : kQuadKind;
}

// Shared memory one unit of the instance needs.
size_t unit_smem(const isg_problem *p, int kind) {
  if (kind == kTorusKind) return torus_batch_max_smem(p->L, p->W);
  if (kind == kGraphWordKind)
    return gm_smem_bytes(p->n, 1, p->n_colours, 0, 0, 0, p->kmax + 1, !p->field.empty());
  return csr_smem_bytes(p->n, 1, 1, p->n_colours, 0, 0, p->mode, p->kmax);
}

// Measured launch shapes: (device, replicas, kinds present, per-kind count of
// instances by size class 2^k vertices) -> (threads, CTAs per SM).
std::mutex g_batch_mu;
std::map<std::vector<int64_t>, std::array<int, 2>> g_batch_shapes;

std::vector<int64_t> batch_key(const isg_problem *const *probs, int32_t count, int32_t R) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<int64_t> key = {dev, R};
  std::array<std::array<int64_t, 32>, 2> hist = {};
  for (int32_t k = 0; k < count; ++k) {
    const isg_problem *p = probs[k];
    int b = 0;
    while ((int64_t(1) << (b + 1)) <= p->n && b < 31) ++b;
    ++hist[p->torus ? 0 : 1][b];
  }
  for (const auto &h : hist) key.insert(key.end(), h.begin(), h.end());
  return key;
}

// The batch with an explicit launch shape (threads per CTA; CTAs per SM,
// 0 = as many as shared memory allows, at most 4).
isg_status batch_impl(const isg_problem *const *probs, int32_t count, int32_t R,
                      const double *betas, int32_t S, const uint64_t *seeds,
                      const int64_t *targets, cudaStream_t stream, isg_result **outs,
                      int threads, int per_sm_req) {
  // validation
  std::vector<int> kind(count);
  size_t smem[3] = {0, 0, 0};
  int64_t max_nr = 0;
  for (int32_t k = 0; k < count; ++k) {
    const isg_problem *p = probs[k];
    if (!p) return fail(ISG_EINVAL, "batch entry %d is NULL", k);
    const int64_t t = targets ? targets[k] : ISG_NO_TARGET;
    if (t != ISG_NO_TARGET && (t < INT32_MIN || t > INT32_MAX))
      return fail(ISG_EINVAL, "target of entry %d outside the int32 range", k);
    kind[k] = kind_of(p, threads);
    // bit-sliced counters of 10 planes hold 4 x sites-per-thread-per-sweep
    if (kind[k] == kTorusKind && (p->n / 2 + threads - 1) / threads > 127)
      return fail(ISG_EINVAL, "batch entry %d (%d sites) is too large for the batched kernel", k,
                  p->n);
    const size_t b = unit_smem(p, kind[k]);
    if (b > 227 * 1024)
      return fail(ISG_EINVAL, "batch entry %d (n = %d) needs more shared memory than a CTA has",
                  k, p->n);
    smem[kind[k]] = std::max(smem[kind[k]], b);
    max_nr = std::max<int64_t>(max_nr, (int64_t)p->n * R);
  }
  for (int32_t k = 0; k < count; ++k) outs[k] = nullptr;

  // thresholds: one table per distinct level set (tori: energy changes 4 and
  // 8; graphs: half energy changes 0..kmax)
  std::map<int32_t, size_t> table_at;  // kmax (-1: tori) -> word offset
  std::vector<uint32_t> tables;
  for (int32_t k = 0; k < count; ++k) {
    const int32_t key = probs[k]->torus ? -1 : probs[k]->kmax;
    if (table_at.count(key)) continue;
    std::vector<int32_t> levels;
    if (key < 0)
      levels = {2, 4};
    else
      for (int32_t q = 0; q <= key; ++q) levels.push_back(q);
    std::vector<uint32_t> t;
    build_table(betas, S, levels, t);
    table_at[key] = tables.size();
    tables.insert(tables.end(), t.begin(), t.end());
  }

  // results and work units
  BatchBlock *blk = new BatchBlock();
  cudaGetDevice(&blk->device);
  blk->stream = stream;
  std::vector<isg_result *> res(count, nullptr);
  std::vector<const DeviceProblem *> dps(count, nullptr);
  isg_status st = ISG_OK;
  auto cleanup = [&](isg_status s) {
    for (auto *r : res)
      if (r) result_free(r);
    free_block(blk);
    return s;
  };
  size_t n_items[3] = {0, 0, 0}, n_items2[3] = {0, 0, 0};
  for (int32_t k = 0; k < count && st == ISG_OK; ++k) {
    const isg_problem *p = probs[k];
    st = problem_device(p, p->torus ? kNeedTorus : kNeedCsr, &dps[k]);
    if (st != ISG_OK) break;
    isg_result *r = new isg_result();
    res[k] = r;
    r->device = blk->device;
    r->stream = stream;
    r->n = p->n;
    r->R = R;
    r->S = S;
    r->msc = kind[k] != kQuadKind;
    r->relabelled = !p->torus;
    r->kernel = kind[k] == kTorusKind ? ISG_KERNEL_TORUS_MSC
                                      : (kind[k] == kGraphWordKind ? ISG_KERNEL_GRAPH_MSC
                                                                   : ISG_KERNEL_CSR);
    r->units = r->msc ? (R + 31) / 32 : (R + 3) / 4;
    r->lanes = r->msc ? 32 : 4;
    r->table_words = 0;
    const int64_t t = targets ? targets[k] : ISG_NO_TARGET;
    r->has_target = t != ISG_NO_TARGET;
    st = result_alloc(r, stream);
    if (st != ISG_OK) break;
    // no unit has reached a target yet
    if (cudaMemsetAsync(r->d_hit, 0xFF, 4 * (size_t)r->units, stream) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming) != cudaSuccess) {
      st = fail(ISG_ECUDA, "preparing the batch's results failed");
      break;
    }
    n_items[kind[k]] += r->units;
    if (r->has_target && r->units > 1) n_items2[kind[k]] += r->units;
  }
  if (st != ISG_OK) return cleanup(st);

  // device memory of the batch: items and orders of both passes, counters,
  // tables, unpack descriptors
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t item_size[3] = {sizeof(TorusBatchItem), sizeof(GraphMscItem),
                               sizeof(CsrBatchItem)};
  size_t o_items[2][3], o_order[2][3], total = 0;
  for (int pass = 0; pass < 2; ++pass)
    for (int q = 0; q < 3; ++q) {
      const size_t n = pass ? n_items2[q] : n_items[q];
      o_items[pass][q] = total;
      total += al(item_size[q] * n);
      o_order[pass][q] = total;
      total += al(4 * n);
    }
  const size_t o_ctl = total;  // [pass][kind]: next counter, unit count
  total += al(4 * 12);
  const size_t o_table = total;
  total += al(4 * tables.size());
  const size_t o_desc = total;
  total += al(sizeof(BatchOutDesc) * count);
  cudaError_t err = cudaMallocAsync(&blk->mem, total, stream);
  if (err != cudaSuccess) {
    blk->mem = nullptr;
    return cleanup(fail(ISG_ENOMEM, "device allocation for the batch failed: %s",
                        cudaGetErrorString(err)));
  }
  char *base = (char *)blk->mem;
  std::vector<TorusBatchItem> it_t[2];
  std::vector<GraphMscItem> it_g[2];
  std::vector<CsrBatchItem> it_c[2];
  std::vector<std::pair<int32_t, int32_t>> ord[2][3];  // (n, item index)
  std::vector<BatchOutDesc> descs(count);
  const uint32_t *d_tables = (const uint32_t *)(base + o_table);
  for (int32_t k = 0; k < count; ++k) {
    const isg_problem *p = probs[k];
    const DeviceProblem *dp = dps[k];
    isg_result *r = res[k];
    const uint32_t *table = d_tables + table_at[p->torus ? -1 : p->kmax];
    const uint32_t key0 = (uint32_t)(seeds[k] & 0xFFFFFFFFu), key1 = (uint32_t)(seeds[k] >> 32);
    const int32_t target = r->has_target ? (int32_t)targets[k] : 0;
    const bool second = r->has_target && r->units > 1;
    for (int pass = 0; pass < (second ? 2 : 1); ++pass) {
      const bool tgt = r->has_target && pass == 0;
      for (int32_t u = 0; u < r->units; ++u) {
        if (kind[k] == kTorusKind) {
          TorusBatchItem it = {};
          TorusSolve &s = it.solve;
          s.L = p->L;
          s.W = p->W;
          s.cbits = dp->cbits;
          s.table = table;
          s.table_ws = 0;
          s.table_ts = 2;
          s.key0 = key0;
          s.key1 = key1;
          s.rk = round_keys(key0, key1);
          s.words = r->units;
          s.replicas = R;
          s.spins = r->d_spins;
          s.best = r->d_best;
          s.e_cur = r->d_e_cur;
          s.e_best = r->d_e_best;
          s.hit = r->d_hit;
          s.done = r->d_done;
          s.has_target = tgt;
          s.target = target;
          it.word = u;
          it.t_end = S;
          it.stop_from_hits = pass;
          ord[pass][kTorusKind].emplace_back(p->n, (int32_t)it_t[pass].size());
          it_t[pass].push_back(it);
        } else if (kind[k] == kGraphWordKind) {
          GraphMscItem it = {};
          GraphMscSolve &s = it.solve;
          s.n = p->n;
          s.n_colours = p->n_colours;
          s.class_start = dp->class_start;
          s.rowptr = dp->rowptr;
          s.col = dp->col;
          s.orig = dp->orig;
          s.field = dp->field_r;
          s.table = table;
          s.kmax1 = p->kmax + 1;
          s.table_ws = 0;
          s.table_ts = s.kmax1;
          s.key0 = key0;
          s.key1 = key1;
          s.rk = round_keys(key0, key1);
          s.words = r->units;
          s.replicas = R;
          s.spins = r->d_spins;
          s.best = r->d_best;
          s.e_cur = r->d_e_cur;
          s.e_best = r->d_e_best;
          s.hit = r->d_hit;
          s.done = r->d_done;
          s.has_target = tgt;
          s.target = target;
          it.word = u;
          it.t_end = S;
          it.stop_from_hits = pass;
          ord[pass][kGraphWordKind].emplace_back(p->n, (int32_t)it_g[pass].size());
          it_g[pass].push_back(it);
        } else {
          CsrBatchItem it = {};
          CsrSolve &s = it.solve;
          s.n = p->n;
          s.n_colours = p->n_colours;
          s.class_start = dp->class_start;
          s.rowptr = dp->rowptr;
          s.col = dp->col;
          s.wt = dp->wt;
          s.orig = dp->orig;
          s.field = dp->field_r;
          s.kmax = p->kmax;
          s.table = table;
          s.key0 = key0;
          s.key1 = key1;
          s.quads = r->units;
          s.replicas = R;
          s.spins = r->d_spins;
          s.best = r->d_best;
          s.e_cur = r->d_e_cur;
          s.e_best = r->d_e_best;
          s.hit = r->d_hit;
          s.done = r->d_done;
          s.has_target = tgt;
          s.target = target;
          s.mode = p->mode;
          it.quad = u;
          it.t_end = S;
          it.stop_from_hits = pass;
          ord[pass][kQuadKind].emplace_back(p->n, (int32_t)it_c[pass].size());
          it_c[pass].push_back(it);
        }
      }
    }
    BatchOutDesc &d = descs[k];
    d.spins = r->d_spins;
    d.best = r->d_best;
    d.orig = p->torus ? nullptr : dp->orig;
    d.hit = r->d_hit;
    d.n = p->n;
    d.R = R;
    d.lanes = r->lanes;
    d.units = r->units;
    d.has_target = r->has_target;
    d.out = r->d_out;
    d.out_best = r->d_out_best;
    d.stop = r->d_stop;
  }

  // uploads: items, longest-first orders, counters, tables, descriptors
  int32_t ctl[12] = {};
  const void *host_items[2][3] = {{it_t[0].data(), it_g[0].data(), it_c[0].data()},
                                  {it_t[1].data(), it_g[1].data(), it_c[1].data()}};
  std::vector<int32_t> orders[2][3];
  for (int pass = 0; pass < 2 && err == cudaSuccess; ++pass)
    for (int q = 0; q < 3 && err == cudaSuccess; ++q) {
      auto &o = ord[pass][q];
      std::stable_sort(o.begin(), o.end(), [](const std::pair<int32_t, int32_t> &a,
                                              const std::pair<int32_t, int32_t> &b) {
        return a.first > b.first;
      });
      const size_t n = o.size();
      ctl[pass * 6 + q * 2 + 1] = (int32_t)n;
      if (n == 0) continue;
      std::vector<int32_t> &order = orders[pass][q];
      order.resize(n);
      for (size_t i = 0; i < n; ++i) order[i] = o[i].second;
      err = cudaMemcpyAsync(base + o_items[pass][q], host_items[pass][q], item_size[q] * n,
                            cudaMemcpyHostToDevice, stream);
      if (err == cudaSuccess)
        err = cudaMemcpyAsync(base + o_order[pass][q], order.data(), 4 * n,
                              cudaMemcpyHostToDevice, stream);
    }
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(base + o_ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(base + o_table, tables.data(), 4 * tables.size(),
                          cudaMemcpyHostToDevice, stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(base + o_desc, descs.data(), sizeof(BatchOutDesc) * count,
                          cudaMemcpyHostToDevice, stream);
  // the host arrays go out of scope
  if (err == cudaSuccess) err = cudaStreamSynchronize(stream);

  // capture: counter resets, both passes (kinds on forked streams), unpack
  auto ctas_for = [&](size_t units, size_t bytes) {
    const int fit = std::max(1, std::min<int>(4, (int)((228 * 1024) / (bytes + 1024))));
    const int per_sm = per_sm_req > 0 ? std::min(per_sm_req, fit) : fit;
    return (int32_t)std::min<size_t>(units, (size_t)sm_count() * per_sm);
  };
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&blk->capture, cudaStreamNonBlocking);
  for (int i = 0; i < 2 && err == cudaSuccess; ++i) {
    err = cudaStreamCreateWithFlags(&blk->side[i], cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&blk->fork[i], cudaEventDisableTiming);
  }
  for (int i = 0; i < 4 && err == cudaSuccess; ++i)
    err = cudaEventCreateWithFlags(&blk->join[i], cudaEventDisableTiming);
  int32_t ctas_used[3] = {0, 0, 0};
  if (err == cudaSuccess)
    err = cudaStreamBeginCapture(blk->capture, cudaStreamCaptureModeThreadLocal);
  if (err == cudaSuccess) {
    cudaError_t e = cudaSuccess;
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
      const size_t *ni = pass ? n_items2 : n_items;
      if (ni[0] + ni[1] + ni[2] == 0) continue;
      int32_t *d_ctl = (int32_t *)(base + o_ctl) + pass * 6;
      // zero the three next counters of this pass (the unit counts stay)
      for (int q = 0; q < 3 && e == cudaSuccess; ++q)
        e = cudaMemsetAsync(d_ctl + 2 * q, 0, 4, blk->capture);
      if (e == cudaSuccess) e = cudaEventRecord(blk->fork[pass], blk->capture);
      for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        e = cudaStreamWaitEvent(blk->side[i], blk->fork[pass], 0);
      if (e == cudaSuccess && ni[kTorusKind]) {
        const int32_t c = ctas_for(ni[kTorusKind], smem[kTorusKind]);
        ctas_used[kTorusKind] = std::max(ctas_used[kTorusKind], c);
        e = torus_batch_launch((const TorusBatchItem *)(base + o_items[pass][kTorusKind]),
                               d_ctl + 1, (const int32_t *)(base + o_order[pass][kTorusKind]),
                               d_ctl, c, threads, smem[kTorusKind], blk->capture);
      }
      if (e == cudaSuccess && ni[kGraphWordKind]) {
        const int32_t c = ctas_for(ni[kGraphWordKind], smem[kGraphWordKind]);
        ctas_used[kGraphWordKind] = std::max(ctas_used[kGraphWordKind], c);
        e = gm_batch_launch((const GraphMscItem *)(base + o_items[pass][kGraphWordKind]),
                            d_ctl + 3, (const int32_t *)(base + o_order[pass][kGraphWordKind]),
                            d_ctl + 2, c, threads, smem[kGraphWordKind], blk->side[0]);
      }
      if (e == cudaSuccess && ni[kQuadKind]) {
        const int32_t c = ctas_for(ni[kQuadKind], smem[kQuadKind]);
        ctas_used[kQuadKind] = std::max(ctas_used[kQuadKind], c);
        e = csr_batch_launch((const CsrBatchItem *)(base + o_items[pass][kQuadKind]), d_ctl + 5,
                             (const int32_t *)(base + o_order[pass][kQuadKind]), d_ctl + 4, c,
                             threads, smem[kQuadKind], blk->side[1]);
      }
      for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaEventRecord(blk->join[2 * pass + i], blk->side[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(blk->capture, blk->join[2 * pass + i], 0);
      }
    }
    if (e == cudaSuccess)
      e = batch_unpack((const BatchOutDesc *)(base + o_desc), count, max_nr, blk->capture);
    err = cudaStreamEndCapture(blk->capture, &blk->graph);
    if (err == cudaSuccess) err = e;
  }
  if (err == cudaSuccess) err = cudaGraphInstantiate(&blk->exec, blk->graph, 0);
  if (err != cudaSuccess) {
    cudaStreamSynchronize(stream);
    return cleanup(cuda_fail(err, "capturing the batch"));
  }
  std::shared_ptr<void> shared(blk, [](void *b) { free_block((BatchBlock *)b); });
  isg_result *r0 = res[0];
  r0->timed = true;
  err = cudaEventCreate(&r0->t0);
  if (err == cudaSuccess) err = cudaEventCreate(&r0->t1);
  if (err == cudaSuccess) err = cudaEventRecord(r0->t0, stream);
  if (err == cudaSuccess) err = cudaGraphLaunch(blk->exec, stream);
  if (err == cudaSuccess) err = cudaEventRecord(r0->t1, stream);
  const int kinds_used = (n_items[0] > 0) + (n_items[1] > 0) + (n_items[2] > 0);
  const int passes = (n_items2[0] + n_items2[1] + n_items2[2]) > 0 ? 2 : 1;
  for (int32_t k = 0; k < count && err == cudaSuccess; ++k) {
    res[k]->shared = shared;
    res[k]->launches = k == 0 ? kinds_used * passes + 1 : 0;
    res[k]->sweep_launches = k == 0 ? kinds_used * passes : 0;
    res[k]->ctas = ctas_used[kind[k]];
    res[k]->cluster = 1;
    res[k]->threads = threads;
    err = cudaEventRecord(res[k]->done, stream);
  }
  if (err != cudaSuccess) {
    cudaStreamSynchronize(stream);
    for (auto *r : res) result_free(r);
    return cuda_fail(err, "launching the batch");
  }
  for (int32_t k = 0; k < count; ++k) outs[k] = res[k];
  return ISG_OK;
}

isg_status batch_check(const isg_problem *const *probs, int32_t count, int32_t replicas,
                       const double *betas, int32_t sweeps, const uint64_t *seeds, void *outs) {
  if (!probs || !seeds || !outs) return fail(ISG_EINVAL, "probs, seeds and outs must not be NULL");
  if (count < 1 || count > 65535) return fail(ISG_EINVAL, "count must be in [1, 65535]");
  if (replicas < 1) return fail(ISG_EINVAL, "replicas must be >= 1");
  if (sweeps < 1) return fail(ISG_EINVAL, "sweeps must be >= 1");
  return check_betas(betas, sweeps);
}

}  // namespace
}  // namespace isg

using namespace isg;

extern "C" isg_status isg_anneal_batch(const isg_problem *const *probs, int32_t count,
                                       int32_t replicas, const double *betas, int32_t sweeps,
                                       const uint64_t *seeds, const int64_t *targets,
                                       void *cuda_stream, isg_result **outs) {
  isg_status st = batch_check(probs, count, replicas, betas, sweeps, seeds, outs);
  if (st != ISG_OK) return st;
  int threads = 256, per_sm = 0;
  {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    auto it = g_batch_shapes.find(batch_key(probs, count, replicas));
    if (it != g_batch_shapes.end()) {
      threads = it->second[0];
      per_sm = it->second[1];
    }
  }
  return batch_impl(probs, count, replicas, betas, sweeps, seeds, targets,
                    (cudaStream_t)cuda_stream, outs, threads, per_sm);
}

extern "C" isg_status isg_autotune_batch(const isg_problem *const *probs, int32_t count,
                                         int32_t replicas, const double *betas, int32_t sweeps,
                                         int32_t probe_sweeps, void *cuda_stream,
                                         int32_t *threads, int32_t *ctas_per_sm) {
  std::vector<uint64_t> seeds(std::max(count, 1), 1u);
  std::vector<isg_result *> outs(std::max(count, 1), nullptr);
  isg_status st = batch_check(probs, count, replicas, betas, sweeps, seeds.data(), outs.data());
  if (st != ISG_OK) return st;
  if (probe_sweeps < 1) return fail(ISG_EINVAL, "probe_sweeps must be >= 1");
  // the probe's schedule: sweeps sampled evenly from the whole schedule
  std::vector<double> probe(probe_sweeps);
  for (int32_t k = 0; k < probe_sweeps; ++k)
    probe[k] = betas[(int64_t)k * sweeps / probe_sweeps];
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  float best_ms = 1e30f;
  int best_t = 0, best_p = 0;
  for (int t : {128, 192, 256, 384, 512}) {
    for (int p = 1; p <= 4; ++p) {
      float ms = 0.f;
      bool ok = true;
      for (int rep = 0; rep < 2 && ok; ++rep) {  // the first run warms up
        st = batch_impl(probs, count, replicas, probe.data(), probe_sweeps, seeds.data(),
                        nullptr, stream, outs.data(), t, p);
        if (st == ISG_EINVAL) {
          ok = false;  // a shape this batch cannot take
          break;
        }
        if (st != ISG_OK) return st;
        isg_stats s0;
        const cudaError_t err = cudaStreamSynchronize(stream);
        isg_result_stats(outs[0], &s0);
        ms = s0.sweep_kernel_ms;
        for (int32_t k = 0; k < count; ++k) isg_result_destroy(outs[k]);
        if (err != cudaSuccess) return cuda_fail(err, "autotuning the batch");
      }
      if (ok && ms > 0.f && ms < best_ms) {
        best_ms = ms;
        best_t = t;
        best_p = p;
      }
    }
  }
  if (best_t == 0) return fail(ISG_EINVAL, "no launch shape fits this batch");
  {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    g_batch_shapes[batch_key(probs, count, replicas)] = {best_t, best_p};
  }
  if (threads) *threads = best_t;
  if (ctas_per_sm) *ctas_per_sm = best_p;
  return ISG_OK;
}
