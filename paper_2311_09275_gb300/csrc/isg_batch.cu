// isg_batch.cu -- many tori in one persistent kernel (isg_anneal_batch).
//
// Each instance is one replica word (R <= 32) solved by one CTA from start to
// finish, so no cross-CTA synchronisation is needed.  CTAs take instances from
// a device work counter in longest-first order (largest L*W first), which
// keeps the tail short when sizes are uneven.  The launch sequence (sweep
// kernel + batched unpack) is captured once into a CUDA graph and launched on
// the caller's stream.  Each instance's result is bit-identical to a single
// isg_anneal of it: the random numbers depend only on (seed, replica, sweep,
// site), never on which CTA ran the instance or when.
#include <algorithm>
#include <memory>
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
  cudaStream_t capture = nullptr;
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
  if (b->capture) cudaStreamDestroy(b->capture);
  cudaSetDevice(prev);
  delete b;
}

}  // namespace
}  // namespace isg

using namespace isg;

extern "C" isg_status isg_anneal_batch(const isg_problem *const *probs, int32_t count,
                                       int32_t replicas, const double *betas, int32_t sweeps,
                                       const uint64_t *seeds, const int64_t *targets,
                                       void *cuda_stream, isg_result **outs) {
  if (!probs || !seeds || !outs) return fail(ISG_EINVAL, "probs, seeds and outs must not be NULL");
  if (count < 1 || count > 65535) return fail(ISG_EINVAL, "count must be in [1, 65535]");
  if (replicas < 1 || replicas > 32)
    return fail(ISG_EINVAL, "batched solves carry one replica word: replicas in [1, 32]");
  if (sweeps < 1) return fail(ISG_EINVAL, "sweeps must be >= 1");
  isg_status st = check_betas(betas, sweeps);
  if (st != ISG_OK) return st;
  const int threads = 256;
  size_t smem = 0;
  int max_n = 0;
  for (int32_t k = 0; k < count; ++k) {
    const isg_problem *p = probs[k];
    if (!p || !p->torus) return fail(ISG_EINVAL, "batch entry %d is not a torus instance", k);
    const int64_t t = targets ? targets[k] : ISG_NO_TARGET;
    if (t != ISG_NO_TARGET && (t < INT32_MIN || t > INT32_MAX))
      return fail(ISG_EINVAL, "target of entry %d outside the int32 range", k);
    // bit-sliced counters of 10 planes hold 4 * sites-per-thread-per-sweep
    if ((p->n / 2 + threads - 1) / threads > 127)
      return fail(ISG_EINVAL, "batch entry %d (%d sites) is too large for the batched kernel", k,
                  p->n);
    smem = std::max(smem, torus_batch_max_smem(p->L, p->W));
    max_n = std::max(max_n, p->n);
  }
  if (smem > 227 * 1024) return fail(ISG_EINVAL, "a batch entry needs too much shared memory");
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  for (int32_t k = 0; k < count; ++k) outs[k] = nullptr;

  std::vector<uint32_t> table;
  build_table(betas, sweeps, {2, 4}, table);

  BatchBlock *blk = new BatchBlock();
  cudaGetDevice(&blk->device);
  blk->stream = stream;
  const size_t o_items = 0;
  const size_t o_order = (sizeof(TorusBatchItem) * count + 255) & ~size_t(255);
  const size_t o_next = o_order + ((4 * (size_t)count + 255) & ~size_t(255));
  const size_t o_count = o_next + 256;
  const size_t o_table = o_count + 256;
  const size_t total = o_table + 4 * table.size();
  cudaError_t err = cudaMallocAsync(&blk->mem, total, stream);
  if (err != cudaSuccess) {
    delete blk;
    return fail(ISG_ENOMEM, "device allocation for the batch failed: %s", cudaGetErrorString(err));
  }
  std::shared_ptr<void> shared(blk, [](void *b) { free_block((BatchBlock *)b); });
  char *base = (char *)blk->mem;
  TorusBatchItem *d_items = (TorusBatchItem *)(base + o_items);
  int32_t *d_order = (int32_t *)(base + o_order);
  int32_t *d_next = (int32_t *)(base + o_next);
  int32_t *d_count = (int32_t *)(base + o_count);
  uint32_t *d_table = (uint32_t *)(base + o_table);

  std::vector<TorusBatchItem> items(count);
  std::vector<isg_result *> res(count, nullptr);
  auto cleanup = [&](isg_status s) {
    for (auto *r : res)
      if (r) result_free(r);
    return s;
  };
  for (int32_t k = 0; k < count && st == ISG_OK; ++k) {
    const isg_problem *p = probs[k];
    const DeviceProblem *dp = nullptr;
    st = problem_device(p, kNeedTorus, &dp);
    if (st != ISG_OK) break;
    isg_result *r = new isg_result();
    res[k] = r;
    r->device = blk->device;
    r->stream = stream;
    r->n = p->n;
    r->R = replicas;
    r->S = sweeps;
    r->kernel = ISG_KERNEL_TORUS_MSC;
    r->msc = true;
    r->units = 1;
    r->lanes = 32;
    r->table_words = 0;
    r->shared = shared;
    const int64_t t = targets ? targets[k] : ISG_NO_TARGET;
    r->has_target = t != ISG_NO_TARGET;
    st = result_alloc(r, stream);
    if (st != ISG_OK) break;
    if (cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming) != cudaSuccess) {
      st = fail(ISG_ECUDA, "event creation failed");
      break;
    }
    TorusSolve &s = items[k].solve;
    s.L = p->L;
    s.W = p->W;
    s.cbits = dp->cbits;
    s.table = d_table;
    s.table_ws = 0;
    s.table_ts = 2;
    s.key0 = (uint32_t)(seeds[k] & 0xFFFFFFFFu);
    s.key1 = (uint32_t)(seeds[k] >> 32);
    s.rk = round_keys(s.key0, s.key1);
    s.words = 1;
    s.replicas = replicas;
    s.spins = r->d_spins;
    s.best = r->d_best;
    s.e_cur = r->d_e_cur;
    s.e_best = r->d_e_best;
    s.hit = r->d_hit;
    s.done = r->d_done;
    s.has_target = r->has_target;
    s.target = r->has_target ? (int32_t)t : 0;
    items[k].word = 0;
    items[k].t_begin = 0;
    items[k].t_end = sweeps;
    items[k].resume = 0;
    items[k].out = r->d_out;
    items[k].out_best = r->d_out_best;
    items[k].stop = r->d_stop;
  }
  if (st != ISG_OK) return cleanup(st);

  std::vector<int32_t> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return probs[a]->n > probs[b]->n; });

  err = cudaMemcpyAsync(d_items, items.data(), sizeof(TorusBatchItem) * count,
                        cudaMemcpyHostToDevice, stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(d_order, order.data(), 4 * (size_t)count, cudaMemcpyHostToDevice, stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(d_table, table.data(), 4 * table.size(), cudaMemcpyHostToDevice, stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(d_count, &count, 4, cudaMemcpyHostToDevice, stream);

  // persistent CTAs: as many as fit per SM by shared memory (at most 4)
  const int per_sm = std::max(1, std::min<int>(4, (int)((228 * 1024) / (smem + 1024))));
  const int ctas = std::min(count, sm_count() * per_sm);
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&blk->capture, cudaStreamNonBlocking);
  if (err == cudaSuccess) err = cudaStreamBeginCapture(blk->capture, cudaStreamCaptureModeThreadLocal);
  if (err == cudaSuccess) {
    cudaError_t e0 = cudaMemsetAsync(d_next, 0, 4, blk->capture);
    cudaError_t e1 = e0 != cudaSuccess ? e0
                                       : torus_batch_launch(d_items, d_count, d_order, d_next, ctas,
                                                            threads, smem, blk->capture);
    cudaError_t e2 = batch_finish(d_items, count, max_n, replicas, blk->capture);
    err = cudaStreamEndCapture(blk->capture, &blk->graph);
    if (err == cudaSuccess) err = e1 != cudaSuccess ? e1 : e2;
  }
  if (err == cudaSuccess) err = cudaGraphInstantiate(&blk->exec, blk->graph, 0);
  isg_result *r0 = res[0];
  if (err == cudaSuccess) {
    r0->timed = true;
    err = cudaEventCreate(&r0->t0);
    if (err == cudaSuccess) err = cudaEventCreate(&r0->t1);
    if (err == cudaSuccess) err = cudaEventRecord(r0->t0, stream);
  }
  if (err == cudaSuccess) err = cudaGraphLaunch(blk->exec, stream);
  if (err == cudaSuccess) err = cudaEventRecord(r0->t1, stream);
  for (int32_t k = 0; k < count && err == cudaSuccess; ++k) {
    res[k]->launches = k == 0 ? 2 : 0;
    res[k]->sweep_launches = k == 0 ? 1 : 0;
    res[k]->ctas = ctas;
    res[k]->cluster = 1;
    res[k]->threads = threads;
    err = cudaEventRecord(res[k]->done, stream);
  }
  if (err != cudaSuccess) {
    cudaStreamSynchronize(stream);
    return cleanup(cuda_fail(err, "launching the batch"));
  }
  for (int32_t k = 0; k < count; ++k) outs[k] = res[k];
  return ISG_OK;
}
