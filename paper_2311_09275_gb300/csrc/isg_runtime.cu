// isg_runtime.cu -- host runtime behind the C ABI of include/isg.h: instance
// building and validation, colouring and colour-major relabelling,
// acceptance tables, device residency, launch orchestration, results.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <array>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <set>
#include <string>
#include <vector>

#include "isg.h"
#include "isg_kernels.h"
#include "isg_runtime.h"

namespace isg {

thread_local std::string g_last_error;

isg_status fail(isg_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

isg_status cuda_fail(cudaError_t err, const char *what) {
  return fail(ISG_ECUDA, "%s: %s", what, cudaGetErrorString(err));
}

#define ISG_CUDA(call)                                   \
  do {                                                   \
    cudaError_t err_ = (call);                           \
    if (err_ != cudaSuccess) return cuda_fail(err_, #call); \
  } while (0)

// ------------------------------------------------------------------ problems

namespace {

isg_status colour_and_relabel(isg_problem *p);

isg_status finish_problem(isg_problem *p) {
  // kmax and total weight
  p->kmax = 0;
  int64_t wsum = 0, wabs = 0;
  for (int32_t i = 0; i < p->n; ++i) {
    int64_t a = p->field.empty() ? 0 : std::llabs((long long)p->field[i]);
    wabs += a;
    for (int64_t q = p->rowptr[i]; q < p->rowptr[i + 1]; ++q) {
      a += std::llabs((long long)p->wt[q]);
      if (p->col[q] > i) {
        wsum += p->wt[q];
        wabs += std::llabs((long long)p->wt[q]);
      }
    }
    p->kmax = std::max<int64_t>(p->kmax, a);
  }
  if (wabs >= (int64_t(1) << 30))
    return fail(ISG_EINVAL, "sum of |w| + |h| = %lld is >= 2^30 (int32 energies)",
                (long long)wabs);
  p->total_weight = wsum;
  p->m = p->rowptr[p->n] / 2;
  return colour_and_relabel(p);
}

// Greedy colouring by ascending id: colour[v] is the smallest c >= 0 that no
// neighbour u < v has.
void colour_greedy(isg_problem *p) {
  std::vector<int32_t> used(p->n + 1, -1);
  p->n_colours = 1;
  for (int32_t v = 0; v < p->n; ++v) {
    for (int64_t q = p->rowptr[v]; q < p->rowptr[v + 1]; ++q)
      if (p->col[q] < v) used[p->colour[p->col[q]]] = v;
    int32_t c = 0;
    while (used[c] == v) ++c;
    p->colour[v] = c;
    p->n_colours = std::max(p->n_colours, c + 1);
  }
}

// Smallest-last colouring (Matula and Beck 1983): repeatedly remove a vertex
// of smallest remaining degree, the smallest id among ties (vertices still
// present are kept in ordered buckets by remaining degree); colour in the
// reverse removal order with the smallest colour no coloured neighbour has;
// number the classes by their smallest vertex.
void colour_smallest_last(isg_problem *p) {
  const int32_t n = p->n;
  std::vector<int32_t> deg(n), order;
  order.reserve(n);
  int32_t dtop = 0;
  for (int32_t v = 0; v < n; ++v) {
    deg[v] = (int32_t)(p->rowptr[v + 1] - p->rowptr[v]);
    dtop = std::max(dtop, deg[v]);
  }
  std::vector<std::set<int32_t>> bucket(dtop + 1);
  for (int32_t v = 0; v < n; ++v) bucket[deg[v]].insert(v);
  std::vector<char> removed(n, 0);
  int32_t dmin = 0;
  for (int32_t step = 0; step < n; ++step) {
    while (bucket[dmin].empty()) ++dmin;
    const int32_t v = *bucket[dmin].begin();
    bucket[dmin].erase(bucket[dmin].begin());
    removed[v] = 1;
    order.push_back(v);
    for (int64_t q = p->rowptr[v]; q < p->rowptr[v + 1]; ++q) {
      const int32_t u = p->col[q];
      if (removed[u]) continue;
      bucket[deg[u]].erase(u);
      bucket[--deg[u]].insert(u);
      dmin = std::min(dmin, deg[u]);
    }
  }
  std::vector<int32_t> used(n + 1, -1);
  std::fill(p->colour.begin(), p->colour.end(), -1);
  p->n_colours = 1;
  for (int32_t step = n - 1; step >= 0; --step) {
    const int32_t v = order[step];
    for (int64_t q = p->rowptr[v]; q < p->rowptr[v + 1]; ++q)
      if (p->colour[p->col[q]] >= 0) used[p->colour[p->col[q]]] = v;
    int32_t c = 0;
    while (used[c] == v) ++c;
    p->colour[v] = c;
    p->n_colours = std::max(p->n_colours, c + 1);
  }
  std::vector<int32_t> rename(p->n_colours, -1);
  int32_t next = 0;
  for (int32_t v = 0; v < n; ++v)
    if (rename[p->colour[v]] < 0) rename[p->colour[v]] = next++;
  for (int32_t v = 0; v < n; ++v) p->colour[v] = rename[p->colour[v]];
}

// Colour classes (the problem's colouring method) and everything derived from
// them: the colour-major relabelling, relabelled CSR and fields, kernel modes.
isg_status colour_and_relabel(isg_problem *p) {
  p->colour.assign(p->n, 0);
  if (p->torus) {
    for (int32_t i = 0; i < p->n; ++i) p->colour[i] = ((i / p->W) + (i % p->W)) & 1;
    p->n_colours = 2;
  } else if (p->colouring == ISG_COLOURING_SMALLEST_LAST) {
    colour_smallest_last(p);
  } else {
    colour_greedy(p);
  }
  // colour-major relabelling: order[new] = original id
  p->class_start.assign(p->n_colours + 1, 0);
  for (int32_t i = 0; i < p->n; ++i) p->class_start[p->colour[i] + 1]++;
  for (int32_t c = 0; c < p->n_colours; ++c) p->class_start[c + 1] += p->class_start[c];
  p->order.assign(p->n, 0);
  std::vector<int32_t> fill(p->class_start.begin(), p->class_start.end() - 1);
  for (int32_t i = 0; i < p->n; ++i) p->order[fill[p->colour[i]]++] = i;
  if (!p->torus) {
    // Inside a class the update order is free.  Vertices are taken in groups
    // of 32 of similar degree (one warp's worth: uniform neighbour-loop trip
    // counts), and the groups in bit-reversed order, so that every contiguous
    // slice of a class (one CTA's share) holds a like mix of degrees.
    std::vector<int32_t> cls, grp;
    for (int32_t c = 0; c < p->n_colours; ++c) {
      const int32_t a = p->class_start[c], b = p->class_start[c + 1];
      cls.assign(p->order.begin() + a, p->order.begin() + b);
      std::stable_sort(cls.begin(), cls.end(), [p](int32_t x, int32_t y) {
        return p->rowptr[x + 1] - p->rowptr[x] > p->rowptr[y + 1] - p->rowptr[y];
      });
      const int32_t G = (b - a + 31) / 32;
      int bits = 0;
      while ((1 << bits) < G) ++bits;
      auto rev = [bits](int32_t g) {
        int32_t r = 0;
        for (int k = 0; k < bits; ++k) r |= ((g >> k) & 1) << (bits - 1 - k);
        return r;
      };
      grp.resize(G);
      for (int32_t g = 0; g < G; ++g) grp[g] = g;
      std::sort(grp.begin(), grp.end(), [&rev](int32_t x, int32_t y) { return rev(x) < rev(y); });
      int32_t o = a;
      for (int32_t g : grp)
        for (int32_t j = 32 * g; j < std::min(32 * g + 32, b - a); ++j) p->order[o++] = cls[j];
    }
  }
  std::vector<int32_t> inv(p->n);
  for (int32_t v = 0; v < p->n; ++v) inv[p->order[v]] = v;
  p->field_r.clear();
  if (!p->field.empty()) {
    p->field_r.resize(p->n);
    for (int32_t v = 0; v < p->n; ++v) p->field_r[v] = p->field[p->order[v]];
  }
  p->rowptr_r.assign(p->n + 1, 0);
  p->col_r.resize(p->rowptr[p->n]);
  p->wt_r.resize(p->rowptr[p->n]);
  for (int32_t v = 0; v < p->n; ++v) {
    const int32_t i = p->order[v];
    p->rowptr_r[v + 1] = p->rowptr_r[v] + (int32_t)(p->rowptr[i + 1] - p->rowptr[i]);
    int32_t o = p->rowptr_r[v];
    for (int64_t q = p->rowptr[i]; q < p->rowptr[i + 1]; ++q, ++o) {
      p->col_r[o] = inv[p->col[q]];
      p->wt_r[o] = p->wt[q];
    }
  }
  // field mode of the colour-class kernel: all weights +1, all +-1 (the sign
  // rides in bit 31 of the relabelled neighbour id), or general; the packed
  // per-lane counts of the first two need degrees <= 255
  bool all_pos = true, all_unit = true;
  int64_t max_deg = 0;
  for (int32_t v = 0; v < p->n; ++v) max_deg = std::max<int64_t>(max_deg, p->rowptr[v + 1] - p->rowptr[v]);
  for (int32_t w : p->wt) {
    all_pos &= (w == 1);
    all_unit &= (w == 1 || w == -1);
  }
  // instances with local fields take the general path (the field enters the
  // per-lane sums, which the packed counts of modes 0 and 1 do not carry)
  p->mode = (max_deg > 255 || !p->field.empty()) ? 2 : (all_pos ? 0 : (all_unit ? 1 : 2));
  p->dmax = (int32_t)max_deg;
  p->unit_pos = all_pos;
  if (p->mode == 1)
    for (size_t o = 0; o < p->col_r.size(); ++o)
      if (p->wt_r[o] < 0) p->col_r[o] = (int32_t)((uint32_t)p->col_r[o] | 0x80000000u);
  return ISG_OK;
}

// Symmetric CSR from an edge list with validation (range, loops, duplicates).
isg_status csr_from_edges(isg_problem *p, int32_t n, int64_t m, const int32_t *u, const int32_t *v,
                          const int32_t *w) {
  if (n < 1) return fail(ISG_EINVAL, "n must be >= 1 (got %d)", n);
  if (m < 0) return fail(ISG_EINVAL, "m must be >= 0");
  if (2 * m >= (int64_t(1) << 31)) return fail(ISG_EINVAL, "too many edges (2m >= 2^31)");
  if (m > 0 && (!u || !v || !w)) return fail(ISG_EINVAL, "edge arrays must not be NULL");
  p->n = n;
  p->rowptr.assign(n + 1, 0);
  for (int64_t e = 0; e < m; ++e) {
    if (u[e] < 0 || u[e] >= n || v[e] < 0 || v[e] >= n)
      return fail(ISG_EINVAL, "edge %lld has an endpoint outside [0, %d)", (long long)e, n);
    if (u[e] == v[e]) return fail(ISG_EINVAL, "edge %lld is a self-loop", (long long)e);
    p->rowptr[u[e] + 1]++;
    p->rowptr[v[e] + 1]++;
  }
  for (int32_t i = 0; i < n; ++i) p->rowptr[i + 1] += p->rowptr[i];
  p->col.resize(2 * m);
  p->wt.resize(2 * m);
  std::vector<int64_t> fill(p->rowptr.begin(), p->rowptr.end() - 1);
  for (int64_t e = 0; e < m; ++e) {
    p->col[fill[u[e]]] = v[e];
    p->wt[fill[u[e]]++] = w[e];
    p->col[fill[v[e]]] = u[e];
    p->wt[fill[v[e]]++] = w[e];
  }
  std::vector<std::pair<int32_t, int32_t>> row;
  for (int32_t i = 0; i < n; ++i) {
    row.clear();
    for (int64_t q = p->rowptr[i]; q < p->rowptr[i + 1]; ++q) row.emplace_back(p->col[q], p->wt[q]);
    std::sort(row.begin(), row.end());
    for (size_t k = 0; k < row.size(); ++k) {
      if (k > 0 && row[k].first == row[k - 1].first)
        return fail(ISG_EINVAL, "vertices %d and %d are joined by more than one edge", i,
                    row[k].first);
      p->col[p->rowptr[i] + k] = row[k].first;
      p->wt[p->rowptr[i] + k] = row[k].second;
    }
  }
  return ISG_OK;
}

void free_device(isg_problem *p) {
  for (auto &d : p->dev) {
    if (d.device < 0) continue;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(d.device);
    cudaFree(d.cbits);
    cudaFree(d.class_start);
    cudaFree(d.rowptr);
    cudaFree(d.col);
    cudaFree(d.wt);
    cudaFree(d.orig);
    cudaFree(d.rowptr_o);
    cudaFree(d.col_o);
    cudaFree(d.wt_o);
    cudaFree(d.field_r);
    cudaFree(d.field_o);
    cudaFree(d.gloff);
    cudaSetDevice(prev);
  }
  p->dev.clear();
}

template <typename T>
cudaError_t upload(T **dst, const T *src, size_t count) {
  const size_t bytes = sizeof(T) * std::max<size_t>(count, 1);
  cudaError_t err = cudaMalloc((void **)dst, bytes);
  if (err != cudaSuccess) return err;
  if (count == 0) return cudaMemset(*dst, 0, bytes);
  return cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice);
}

}  // namespace

// Device-resident copy of an instance on the current device: each group of
// arrays is uploaded once, on the first call that needs it.
isg_status problem_device(const isg_problem *cp, unsigned need, const DeviceProblem **out,
                          size_t *uploaded) {
  isg_problem *p = const_cast<isg_problem *>(cp);
  int device = 0;
  ISG_CUDA(cudaGetDevice(&device));
  std::lock_guard<std::mutex> lock(p->mu);
  DeviceProblem *d = nullptr;
  for (auto &x : p->dev)
    if (x.device == device) d = &x;
  if (!d) {
    if (p->dev.size() >= 64) return fail(ISG_EINVAL, "instance used on too many devices");
    p->dev.emplace_back();
    d = &p->dev.back();
    d->device = device;
  }
  if (!p->torus) need &= ~unsigned(kNeedTorus);
  cudaError_t err = cudaSuccess;
  size_t bytes = 0;
  if ((need & kNeedTorus) && !(d->have & kNeedTorus)) {
    std::vector<uint8_t> cb(p->n);
    for (int32_t i = 0; i < p->n; ++i)
      cb[i] = (uint8_t)((p->jr[i] < 0 ? 1 : 0) | (p->jd[i] < 0 ? 2 : 0));
    err = upload(&d->cbits, cb.data(), cb.size());
    bytes += cb.size();
    if (err == cudaSuccess) d->have |= kNeedTorus;
  }
  if (err == cudaSuccess && (need & kNeedCsr) && !(d->have & kNeedCsr)) {
    err = upload(&d->class_start, p->class_start.data(), p->class_start.size());
    if (err == cudaSuccess) err = upload(&d->rowptr, p->rowptr_r.data(), p->rowptr_r.size());
    if (err == cudaSuccess) err = upload(&d->col, p->col_r.data(), p->col_r.size());
    if (err == cudaSuccess) err = upload(&d->wt, p->wt_r.data(), p->wt_r.size());
    if (err == cudaSuccess) err = upload(&d->orig, p->order.data(), p->order.size());
    if (err == cudaSuccess && !p->field_r.empty())
      err = upload(&d->field_r, p->field_r.data(), p->field_r.size());
    // the staged graph kernel's precomputed masks: one word per threshold level
    std::vector<int32_t> gloff(p->n + 1, 0);
    int64_t gl = 0;
    for (int32_t v = 0; v < p->n; ++v) {
      gloff[v] = (int32_t)std::min<int64_t>(gl, INT32_MAX);
      const int64_t h = p->field_r.empty() ? 0 : std::abs((int64_t)p->field_r[v]);
      gl += (p->rowptr_r[v + 1] - p->rowptr_r[v] + h + 1) / 2;
    }
    gloff[p->n] = (int32_t)std::min<int64_t>(gl, INT32_MAX);
    d->gl = gl;
    if (err == cudaSuccess) err = upload(&d->gloff, gloff.data(), gloff.size());
    bytes += 4 * (p->class_start.size() + p->rowptr_r.size() + p->col_r.size() +
                  p->wt_r.size() + p->order.size() + p->field_r.size() + gloff.size());
    if (err == cudaSuccess) d->have |= kNeedCsr;
  }
  if (err == cudaSuccess && (need & kNeedEnergy) && !(d->have & kNeedEnergy)) {
    err = upload(&d->rowptr_o, p->rowptr.data(), p->rowptr.size());
    if (err == cudaSuccess) err = upload(&d->col_o, p->col.data(), p->col.size());
    if (err == cudaSuccess) err = upload(&d->wt_o, p->wt.data(), p->wt.size());
    if (err == cudaSuccess && !p->field.empty())
      err = upload(&d->field_o, p->field.data(), p->field.size());
    bytes += 8 * p->rowptr.size() + 4 * (p->col.size() + p->wt.size() + p->field.size());
    if (err == cudaSuccess) d->have |= kNeedEnergy;
  }
  d->bytes_uploaded += bytes;
  if (uploaded) *uploaded = bytes;
  if (err != cudaSuccess) return cuda_fail(err, "uploading the instance");
  *out = d;
  return ISG_OK;
}

// ------------------------------------------------------------------ tables

// T[t][k] = min(floor(2^32 exp(-beta_t * 2k)), 2^32 - 1) for the levels used.
void build_table(const double *betas, int32_t sweeps, const std::vector<int32_t> &levels,
                 std::vector<uint32_t> &out) {
  out.resize((size_t)sweeps * levels.size());
  for (int32_t t = 0; t < sweeps; ++t)
    for (size_t j = 0; j < levels.size(); ++j) {
      const double x = std::floor(std::ldexp(std::exp(-betas[t] * (double)(2 * levels[j])), 32));
      out[(size_t)t * levels.size() + j] = x >= 4294967295.0 ? 4294967295u : (uint32_t)x;
    }
}

isg_status check_betas(const double *betas, int32_t sweeps) {
  if (!betas) return fail(ISG_EINVAL, "betas must not be NULL");
  for (int32_t t = 0; t < sweeps; ++t)
    if (!std::isfinite(betas[t]) || betas[t] < 0)
      return fail(ISG_EINVAL, "beta[%d] = %g is not finite and >= 0", t, betas[t]);
  return ISG_OK;
}

// ------------------------------------------------------------------ results

// Allocations of solve state still to fail (isg_debug_fail_allocations).
std::atomic<int32_t> g_fail_allocations{0};

isg_status result_alloc(isg_result *r, cudaStream_t stream) {
  int32_t pending = g_fail_allocations.load();
  while (pending > 0 && !g_fail_allocations.compare_exchange_weak(pending, pending - 1)) {
  }
  if (pending > 0) {
    r->base = nullptr;
    return fail(ISG_ENOMEM, "device allocation failed (injected by isg_debug_fail_allocations)");
  }
  const size_t n = (size_t)r->n, R = (size_t)r->R, units = (size_t)r->units;
  const size_t lanes = units * r->lanes;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += al(bytes);
    return o;
  };
  const size_t o_spins = take(sizeof(uint32_t) * units * n);
  const size_t o_best = take(sizeof(uint32_t) * units * n);
  const size_t o_ecur = take(sizeof(int32_t) * lanes);
  const size_t o_ebest = take(sizeof(int32_t) * lanes);
  const size_t o_hit = take(sizeof(int32_t) * units);
  const size_t o_done = take(sizeof(int32_t) * units);
  const size_t o_stop = take(sizeof(int32_t));
  const size_t o_out = take(R * n);
  const size_t o_outb = take(R * n);
  const size_t o_table = take(sizeof(uint32_t) * r->table_words);
  r->bytes = off;
  cudaError_t err = cudaMallocAsync(&r->base, off, stream);
  if (err != cudaSuccess) {
    r->base = nullptr;
    return fail(ISG_ENOMEM, "device allocation of %zu bytes failed: %s", off,
                cudaGetErrorString(err));
  }
  char *b = (char *)r->base;
  r->d_spins = (uint32_t *)(b + o_spins);
  r->d_best = (uint32_t *)(b + o_best);
  r->d_e_cur = (int32_t *)(b + o_ecur);
  r->d_e_best = (int32_t *)(b + o_ebest);
  r->d_hit = (int32_t *)(b + o_hit);
  r->d_done = (int32_t *)(b + o_done);
  r->d_stop = (int32_t *)(b + o_stop);
  r->d_out = (int8_t *)(b + o_out);
  r->d_out_best = (int8_t *)(b + o_outb);
  r->d_table = (uint32_t *)(b + o_table);
  return ISG_OK;
}

isg_status result_sync(const isg_result *cr) {
  isg_result *r = const_cast<isg_result *>(cr);
  std::lock_guard<std::mutex> lock(r->mu);
  if (r->synced) return r->sync_status;
  r->synced = true;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(r->device);
  cudaError_t err = cudaEventSynchronize(r->done);
  const size_t lanes = (size_t)r->units * r->lanes;
  r->h_e_cur.resize(lanes);
  r->h_e_best.resize(lanes);
  r->h_done.resize(r->units);
  int32_t stop = -1;
  if (err == cudaSuccess)
    err = cudaMemcpy(r->h_e_cur.data(), r->d_e_cur, 4 * lanes, cudaMemcpyDeviceToHost);
  if (err == cudaSuccess)
    err = cudaMemcpy(r->h_e_best.data(), r->d_e_best, 4 * lanes, cudaMemcpyDeviceToHost);
  if (err == cudaSuccess)
    err = cudaMemcpy(r->h_done.data(), r->d_done, 4 * (size_t)r->units, cudaMemcpyDeviceToHost);
  if (err == cudaSuccess) err = cudaMemcpy(&stop, r->d_stop, 4, cudaMemcpyDeviceToHost);
  if (err == cudaSuccess && r->timed) err = cudaEventElapsedTime(&r->kernel_ms, r->t0, r->t1);
  cudaSetDevice(prev);
  if (err != cudaSuccess) {
    r->sync_status = cuda_fail(err, "waiting for the solve");
    return r->sync_status;
  }
  r->hit_sweep = r->has_target ? stop : -1;
  r->sweeps_done = 0;
  for (int32_t u = 0; u < r->units; ++u) {
    if (r->h_done[u] < 0) {
      // the graph kernel's wait for a class from its cluster peers gave up
      r->sync_status = fail(ISG_ECUDA, "replica word %d: a wait for its cluster peers timed out",
                            u);
      return r->sync_status;
    }
    r->sweeps_done = std::max(r->sweeps_done, r->h_done[u]);
  }
  r->sync_status = ISG_OK;
  return ISG_OK;
}

void result_free(isg_result *r) {
  if (!r) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(r->device);
  if (r->done) cudaEventSynchronize(r->done);
  if (r->base) cudaFreeAsync(r->base, r->stream);
  if (r->d_table_ext) cudaFreeAsync(r->d_table_ext, r->stream);
  if (r->pt_mem) cudaFreeAsync(r->pt_mem, r->stream);
  if (r->pt_exec) cudaGraphExecDestroy(r->pt_exec);
  if (r->pt_graph) cudaGraphDestroy(r->pt_graph);
  if (r->pt_capture) cudaStreamDestroy(r->pt_capture);
  if (r->pm_sweeps) cudaStreamDestroy(r->pm_sweeps);
  if (r->pm_masks) cudaStreamDestroy(r->pm_masks);
  for (cudaEvent_t e : r->pm_ev)
    if (e) cudaEventDestroy(e);
  if (r->done) cudaEventDestroy(r->done);
  if (r->t0) cudaEventDestroy(r->t0);
  if (r->t1) cudaEventDestroy(r->t1);
  cudaSetDevice(prev);
  delete r;
}

// ------------------------------------------------------------------ launch shapes

int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1)
      v = 152;
    cached = v;
  }
  return cached;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Torus kernel shape without measurements: the smallest power-of-two cluster
// that puts at least ~0.8 x SMs CTAs on the device (bands of >= 2 rows), then
// enough threads for ~3 sites per thread per colour phase (a multiple of 64:
// 80 x 100 in clusters of 4 gets 384, the measured best).
void torus_shape(int L, int W, int words, int &cluster, int &threads) {
  const int sms = sm_count();
  if (cluster <= 0) {
    cluster = 1;
    while (cluster < 8 && words * cluster < (sms * 4) / 5 && L / (cluster * 2) >= 2) cluster *= 2;
  }
  if (threads <= 0) {
    const int nr = (L + cluster - 1) / cluster;
    const int per_phase = nr * (W / 2);
    threads = std::min(512, std::max(64, round_up((per_phase + 2) / 3, 64)));
  }
}

void csr_shape(int quads, int max_class, int &cluster, int &threads) {
  const int sms = sm_count();
  if (cluster <= 0) {
    cluster = 1;
    while (cluster < 8 && quads * cluster < (sms * 4) / 5) cluster *= 2;
  }
  if (threads <= 0) {
    const int per_phase = (max_class + cluster - 1) / cluster;
    threads = std::min(512, std::max(64, round_up((per_phase + 2) / 3, 32)));
  }
}

namespace {

// Measured choices: (device, torus?, L or n, W or nnz, replicas)
//   -> (kernel, cluster, threads, quads/CTA)
std::mutex g_shape_mu;
std::map<std::array<int64_t, 6>, std::array<int, 4>> g_shapes;  // tuned shapes by shape_key

std::array<int64_t, 6> shape_key(const isg_problem *p, int replicas) {
  int dev = 0;
  cudaGetDevice(&dev);
  return {dev, p->torus ? 1 : 0, p->torus ? p->L : p->n, p->torus ? p->W : p->rowptr[p->n],
          replicas, p->colouring};
}

bool shape_lookup(const isg_problem *p, int replicas, int &kernel, int &cluster, int &threads,
                  int &qpc) {
  std::lock_guard<std::mutex> lock(g_shape_mu);
  auto it = g_shapes.find(shape_key(p, replicas));
  if (it == g_shapes.end()) return false;
  kernel = it->second[0];
  cluster = it->second[1];
  threads = it->second[2];
  qpc = it->second[3];
  return true;
}

// Owned-slice sizes of the colour-class kernel under a cluster split: the
// largest number of vertices and of adjacency entries any rank owns.
void csr_own_sizes(const isg_problem *p, int K, int &own_n, int &own_nnz) {
  own_n = own_nnz = 0;
  for (int k = 0; k < K; ++k) {
    int64_t nv = 0, ne = 0;
    for (int32_t c = 0; c < p->n_colours; ++c) {
      const int64_t a = p->class_start[c], len = p->class_start[c + 1] - a;
      const int64_t lo = a + len * k / K, hi = a + len * (k + 1) / K;
      nv += hi - lo;
      ne += p->rowptr_r[hi] - p->rowptr_r[lo];
    }
    own_n = std::max<int>(own_n, (int)nv);
    own_nnz = std::max<int>(own_nnz, (int)ne);
  }
}

// Mask table of the staged graph kernel: the largest sum over any rank's owned
// vertices of their threshold levels (d + |h| + 1) / 2 (one mask word each).
int gm_own_levels(const isg_problem *p, int K) {
  int own_lv = 0;
  for (int k = 0; k < K; ++k) {
    int64_t lv = 0;
    for (int32_t c = 0; c < p->n_colours; ++c) {
      const int64_t a = p->class_start[c], len = p->class_start[c + 1] - a;
      const int64_t lo = a + len * k / K, hi = a + len * (k + 1) / K;
      for (int64_t v = lo; v < hi; ++v) {
        const int64_t h = p->field_r.empty() ? 0 : std::abs((int64_t)p->field_r[v]);
        lv += (p->rowptr_r[v + 1] - p->rowptr_r[v] + h + 1) / 2;
      }
    }
    own_lv = std::max<int>(own_lv, (int)lv);
  }
  return own_lv;
}

// Shared memory of the colour-class kernel; staged = adjacency in shared memory.
size_t csr_bytes(const isg_problem *p, int qpc, int K, bool staged) {
  int own_n = 0, own_nnz = 0;
  if (staged) csr_own_sizes(p, K, own_n, own_nnz);
  return csr_smem_bytes(p->n, qpc, K, p->n_colours, own_n, own_nnz, p->mode, p->kmax);
}

int max_class_size(const isg_problem *p) {
  int m = 0;
  for (int32_t c = 0; c < p->n_colours; ++c)
    m = std::max(m, p->class_start[c + 1] - p->class_start[c]);
  return m;
}

// The multi-spin graph kernel needs +-1 weights (all +1 with local fields,
// which it counts as |h| extra bonds) and degree + |h| <= 63 (= kmax).
bool graph_msc_ok(const isg_problem *p) {
  return p->kmax <= 63 && (p->field.empty() ? p->mode <= 1 : p->unit_pos);
}

// Shared memory of the graph kernel; staged = adjacency in shared memory.
size_t gm_bytes(const isg_problem *p, int K, bool staged) {
  int own_n = 0, own_nnz = 0, own_lv = 0;
  if (staged) {
    csr_own_sizes(p, K, own_n, own_nnz);
    own_lv = gm_own_levels(p, K);
  }
  return gm_smem_bytes(p->n, K, p->n_colours, own_n, own_nnz, own_lv, p->kmax + 1,
                       !p->field.empty());
}

// Energy-counter planes of the graph kernel: a thread's accepted degree sum
// per sweep is at most (its vertices per sweep) x (max degree + |h|).
int gm_planes_for(const isg_problem *p, int K, int threads) {
  int own_n = 0, own_nnz = 0;
  csr_own_sizes(p, K, own_n, own_nnz);
  const int64_t per_thread = (own_n + threads - 1) / threads + p->n_colours;
  const int64_t cnt = per_thread * std::max(1, p->kmax);
  return cnt >= (1 << 30) ? -1 : gm_planes((int32_t)cnt);
}

void gm_shape(const isg_problem *p, int words, int &cluster, int &threads) {
  const int sms = sm_count();
  if (cluster <= 0) {
    cluster = 1;
    while (cluster < 16 && words * cluster * 2 <= sms && max_class_size(p) / (cluster * 2) >= 64)
      cluster *= 2;
  }
  if (threads <= 0) threads = 256;
}

TorusSolve make_torus_solve(const isg_problem *p, const DeviceProblem *dp, const isg_result *r,
                            uint64_t seed, bool has_target, int64_t target) {
  TorusSolve s = {};
  s.L = p->L;
  s.W = p->W;
  s.cbits = dp->cbits;
  s.table = r->d_table;
  s.table_ws = 0;
  s.table_ts = 2;
  s.key0 = (uint32_t)(seed & 0xFFFFFFFFu);
  s.key1 = (uint32_t)(seed >> 32);
  s.rk = round_keys(s.key0, s.key1);
  s.words = r->units;
  s.replicas = r->R;
  s.rng_word0 = r->first_replica / 32;
  s.spins = r->d_spins;
  s.best = r->d_best;
  s.e_cur = r->d_e_cur;
  s.e_best = r->d_e_best;
  s.hit = r->d_hit;
  s.done = r->d_done;
  s.has_target = has_target;
  s.target = has_target ? (int32_t)target : 0;
  return s;
}

CsrSolve make_csr_solve(const isg_problem *p, const DeviceProblem *dp, const isg_result *r,
                        uint64_t seed, bool has_target, int64_t target) {
  CsrSolve s = {};
  s.n = p->n;
  s.n_colours = p->n_colours;
  s.class_start = dp->class_start;
  s.rowptr = dp->rowptr;
  s.col = dp->col;
  s.wt = dp->wt;
  s.orig = dp->orig;
  s.field = dp->field_r;
  s.kmax = p->kmax;
  s.table = r->d_table;
  s.key0 = (uint32_t)(seed & 0xFFFFFFFFu);
  s.key1 = (uint32_t)(seed >> 32);
  s.quads = r->units;
  s.replicas = r->R;
  s.rng_quad0 = r->first_replica / 4;
  s.spins = r->d_spins;
  s.best = r->d_best;
  s.e_cur = r->d_e_cur;
  s.e_best = r->d_e_best;
  s.hit = r->d_hit;
  s.done = r->d_done;
  s.has_target = has_target;
  s.target = has_target ? (int32_t)target : 0;
  s.mode = p->mode;
  return s;
}

GraphMscSolve make_gm_solve(const isg_problem *p, const DeviceProblem *dp, const isg_result *r,
                            uint64_t seed, bool has_target, int64_t target) {
  GraphMscSolve s = {};
  s.n = p->n;
  s.n_colours = p->n_colours;
  s.class_start = dp->class_start;
  s.rowptr = dp->rowptr;
  s.col = dp->col;
  s.orig = dp->orig;
  s.field = dp->field_r;
  s.table = r->d_table;
  s.kmax1 = p->kmax + 1;
  s.table_ws = 0;
  s.table_ts = s.kmax1;
  s.key0 = (uint32_t)(seed & 0xFFFFFFFFu);
  s.key1 = (uint32_t)(seed >> 32);
  s.rk = round_keys(s.key0, s.key1);
  s.words = r->units;
  s.replicas = r->R;
  s.rng_word0 = r->first_replica / 32;
  s.spins = r->d_spins;
  s.best = r->d_best;
  s.e_cur = r->d_e_cur;
  s.e_best = r->d_e_best;
  s.hit = r->d_hit;
  s.done = r->d_done;
  s.has_target = has_target;
  s.target = has_target ? (int32_t)target : 0;
  return s;
}

// Device memory for the tables of precomputed graph masks: at most this for
// the two chunks' tables, and chunks chosen automatically hold one table of
// at most kMaskChunkBytes (that stays in L2 while it is read: measured
// faster than larger chunks).
constexpr int64_t kMaskTableBytes = int64_t(1) << 30;
constexpr int64_t kMaskChunkBytes = int64_t(96) << 20;
// Torus: one chunk's table of precomputed masks chosen automatically (80x100
// at 1,024 replicas: 32 sweeps of 2 MB, chunks of 160 sweeps; measured best
// among 120-320).
constexpr int64_t kTorusChunkBytes = int64_t(64) << 20;

// The result's two streams for precomputed masks (sweep kernel at the
// greatest priority, mask kernel at the least) and their events, created on
// first use and kept until the result is freed.
cudaError_t premask_streams(isg_result *r) {
  if (r->pm_sweeps) return cudaSuccess;
  int least = 0, greatest = 0;
  cudaError_t err = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  if (err == cudaSuccess)
    err = cudaStreamCreateWithPriority(&r->pm_sweeps, cudaStreamNonBlocking, greatest);
  if (err == cudaSuccess)
    err = cudaStreamCreateWithPriority(&r->pm_masks, cudaStreamNonBlocking, least);
  for (int i = 0; i < 6 && err == cudaSuccess; ++i)
    err = cudaEventCreateWithFlags(&r->pm_ev[i], cudaEventDisableTiming);
  return err;
}

// Sweeps [t_start, S) of a staged graph solve without a target, with the
// acceptance masks precomputed: chunk k's masks are built by gm_mask_launch
// on a low-priority stream into one of two tables (the table of chunk k - 2
// once its sweeps are done), and the sweep kernel runs chunk k on a
// high-priority stream once they are ready.  The sweep kernel leaves SMs idle
// (one cluster per GPC), which the mask kernel fills; the priorities let the
// sweep kernel's clusters start first when both wait.  Only stream order and
// events connect the two kernels.  cudaErrorMemoryAllocation: the table does
// not fit (nothing was enqueued).
cudaError_t launch_premasked(const isg_problem *p, const DeviceProblem *dp, isg_result *r,
                             uint64_t seed, int cluster, int threads, int own_n, int own_nnz,
                             int own_lv, int planes, int C, int S, int t_start,
                             cudaStream_t stream, int &launches) {
  const size_t chunk_bytes = (size_t)C * (size_t)dp->gl * (size_t)r->units * 4;
  void *buf = nullptr;
  cudaError_t err = cudaMallocAsync(&buf, 2 * chunk_bytes, stream);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return cudaErrorMemoryAllocation;
  }
  err = premask_streams(r);
  cudaStream_t hs = r->pm_sweeps, ms = r->pm_masks;
  cudaEvent_t *ev = r->pm_ev;  // start, end, masks ready (2), sweeps done (2)
  if (err == cudaSuccess) err = cudaEventRecord(ev[0], stream);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(hs, ev[0], 0);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(ms, ev[0], 0);
  const GraphMscSolve s = make_gm_solve(p, dp, r, seed, false, 0);
  int k = 0;
  for (int a = t_start; a < S && err == cudaSuccess; a += C, ++k) {
    const int b = std::min(S, a + C);
    uint32_t *tab = (uint32_t *)((char *)buf + (size_t)(k & 1) * chunk_bytes);
    if (k >= 2) err = cudaStreamWaitEvent(ms, ev[4 + (k & 1)], 0);
    if (err == cudaSuccess) err = gm_mask_launch(s, dp->gloff, dp->gl, a, b - a, tab, ms);
    if (err == cudaSuccess) err = cudaEventRecord(ev[2 + (k & 1)], ms);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(hs, ev[2 + (k & 1)], 0);
    if (err == cudaSuccess) {
      GraphMscLaunch l = {};
      l.t_begin = a;
      l.t_end = b;
      l.resume = a > 0;
      l.cluster = cluster;
      l.threads = threads;
      l.own_n = own_n;
      l.own_nnz = own_nnz;
      l.own_lv = own_lv;
      l.planes = planes;
      l.gmask = tab;
      l.gloff = dp->gloff;
      l.gmask_gl = dp->gl;
      l.gmask_t0 = a;
      err = gm_launch(s, l, hs);
    }
    if (err == cudaSuccess) err = cudaEventRecord(ev[4 + (k & 1)], hs);
    launches += 2;
  }
  r->mask_chunks = k;
  if (err == cudaSuccess) err = cudaEventRecord(ev[1], hs);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(stream, ev[1], 0);
  if (err != cudaSuccess) {
    // nothing may still use the table when it is freed
    if (hs) cudaStreamSynchronize(hs);
    if (ms) cudaStreamSynchronize(ms);
    cudaStreamSynchronize(stream);
  }
  cudaFreeAsync(buf, stream);
  return err;
}

// Sweeps [t_start, S) of a torus solve without a target in the software-
// pipelined build, in chunks of C sweeps, with the masks of the first
// ceil(len / E) sweeps of every chunk after the first precomputed: the sweep
// kernel's clusters leave SMs idle, and torus_mask_launch fills them, on a
// low-priority stream, with the masks of chunk j + 1 while the sweep kernel
// runs chunk j on a high-priority stream.  Chunk j >= 1 reads table j mod 2,
// whose masks wait for the sweeps of chunk j - 2.  Stream order and events
// only.  cudaErrorMemoryAllocation: the tables do not fit (nothing enqueued).
cudaError_t launch_torus_premasked(const isg_problem *p, const DeviceProblem *dp, isg_result *r,
                                   uint64_t seed, int cluster, int threads, int E, int C, int S,
                                   int t_start, cudaStream_t stream, int &launches) {
  const size_t per_sweep = (size_t)2 * (size_t)p->n * (size_t)r->units * 4;
  const size_t chunk_bytes = (size_t)((C + E - 1) / E) * per_sweep;
  void *buf = nullptr;
  cudaError_t err = cudaMallocAsync(&buf, 2 * chunk_bytes, stream);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return cudaErrorMemoryAllocation;
  }
  err = premask_streams(r);
  cudaStream_t hs = r->pm_sweeps, ms = r->pm_masks;
  cudaEvent_t *ev = r->pm_ev;  // start, end, masks ready (2), sweeps done (2)
  if (err == cudaSuccess) err = cudaEventRecord(ev[0], stream);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(hs, ev[0], 0);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(ms, ev[0], 0);
  const TorusSolve s = make_torus_solve(p, dp, r, seed, false, 0);
  const int chunks = (S - t_start + C - 1) / C;
  auto table = [&](int j) { return (uint32_t *)((char *)buf + (size_t)(j & 1) * chunk_bytes); };
  for (int j = 0; j < chunks && err == cudaSuccess; ++j) {
    const int a = t_start + j * C, b = std::min(S, a + C);
    if (j + 1 < chunks) {
      // the next chunk's masks, beside this chunk's sweeps
      const int a1 = b, b1 = std::min(S, a1 + C);
      if (j + 1 >= 3) err = cudaStreamWaitEvent(ms, ev[4 + ((j + 1) & 1)], 0);
      if (err == cudaSuccess)
        err = torus_mask_launch(s, a1, (b1 - a1 + E - 1) / E, table(j + 1), ms);
      if (err == cudaSuccess) err = cudaEventRecord(ev[2 + ((j + 1) & 1)], ms);
      ++launches;
    }
    if (err == cudaSuccess && j >= 1) err = cudaStreamWaitEvent(hs, ev[2 + (j & 1)], 0);
    if (err == cudaSuccess) {
      TorusLaunch l = {};
      l.t_begin = a;
      l.t_end = b;
      l.resume = a > 0;
      l.cluster = cluster;
      l.threads = threads;
      l.pre_tab = j >= 1 ? table(j) : nullptr;
      l.pre_count = j >= 1 ? (b - a + E - 1) / E : 0;
      err = torus_launch(s, l, hs);
    }
    if (err == cudaSuccess) err = cudaEventRecord(ev[4 + (j & 1)], hs);
    ++launches;
  }
  r->mask_chunks = chunks - 1;
  if (err == cudaSuccess) err = cudaEventRecord(ev[1], hs);
  if (err == cudaSuccess) err = cudaStreamWaitEvent(stream, ev[1], 0);
  if (err != cudaSuccess) {
    if (hs) cudaStreamSynchronize(hs);
    if (ms) cudaStreamSynchronize(ms);
    cudaStreamSynchronize(stream);
  }
  cudaFreeAsync(buf, stream);
  return err;
}

// Enqueue the sweeps [0, S) of a prepared result under the given shape:
// one persistent launch, or one launch per sweep (plain); with a target and
// several independently scheduled units, a second pass replays every unit to
// the earliest unit's stop sweep.  Colour-class launches stage the owned
// adjacency in shared memory whenever it fits.
cudaError_t launch_sweeps(const isg_problem *p, const DeviceProblem *dp, isg_result *r,
                          uint64_t seed, bool has_target, int64_t target, bool plain, int cluster,
                          int threads, int qpc, int S, cudaStream_t stream, int &launches,
                          int t_start = 0) {
  cudaError_t err = cudaSuccess;
  const bool gm = r->msc && r->relabelled;
  int own_n = 0, own_nnz = 0, own_lv = 0, planes = 0;
  if (!r->msc && csr_bytes(p, qpc, cluster, true) <= 227 * 1024)
    csr_own_sizes(p, cluster, own_n, own_nnz);
  if (gm) {
    if (gm_bytes(p, cluster, true) <= 227 * 1024) {
      csr_own_sizes(p, cluster, own_n, own_nnz);
      own_lv = gm_own_levels(p, cluster);
    }
    planes = gm_planes_for(p, cluster, threads);
    if (planes < 0) return cudaErrorInvalidConfiguration;
  }
  r->staged = own_n > 0;
  r->mask_chunks = 0;
  if (gm && own_n > 0 && !has_target && !plain && r->mask_chunk >= 0 && dp->gl > 0 &&
      S > t_start) {
    // precomputed masks, in chunks whose two tables fit kMaskTableBytes
    // (chosen here: a table of at most kMaskChunkBytes and at least 64 sweeps)
    const int64_t per_sweep = dp->gl * (int64_t)r->units * 4;
    const int64_t left = S - t_start;
    const int64_t C = r->mask_chunk > 0 ? std::min<int64_t>(r->mask_chunk, left)
                                        : std::min<int64_t>(left, kMaskChunkBytes / per_sweep);
    if (C >= 1 && 2 * C * per_sweep <= kMaskTableBytes && (r->mask_chunk > 0 || C >= 64)) {
      err = launch_premasked(p, dp, r, seed, cluster, threads, own_n, own_nnz, own_lv, planes,
                             (int)C, S, t_start, stream, launches);
      if (err != cudaErrorMemoryAllocation) return err;
      err = cudaSuccess;  // no room for the table: the sweep kernel builds the masks
    }
  }
  if (r->msc && !gm && !has_target && !plain && r->mask_chunk >= 0 && S > t_start &&
      torus_pipelined(p->L, p->W, cluster, threads)) {
    // masks of one sweep in E precomputed on the SMs the clusters leave idle:
    // E from the busy and idle SM counts (a sweep with its masks read costs
    // about 0.3 of one that draws them, and the mask kernel draws about 1.3
    // times as fast per SM as the sweep kernel consumes)
    const int busy = r->units * cluster, idle = sm_count() - busy;
    if (idle > 0) {
      const int E = std::max(1, (int)std::lround(1.0 + 0.75 * busy / idle));
      const int64_t per_sweep = (int64_t)2 * p->n * r->units * 4;
      const int64_t left = S - t_start;
      // chosen here: a table of at most kTorusChunkBytes, and at least four chunks
      int64_t C = r->mask_chunk > 0 ? (int64_t)r->mask_chunk
                                    : std::min<int64_t>(std::max<int64_t>(1, kTorusChunkBytes /
                                                                                 per_sweep) * E,
                                                        (left + 3) / 4);
      C = std::max<int64_t>(C, 2);
      if (C < left && 2 * ((C + E - 1) / E) * per_sweep <= kMaskTableBytes) {
        err = launch_torus_premasked(p, dp, r, seed, cluster, threads, E, (int)C, S, t_start,
                                     stream, launches);
        if (err != cudaErrorMemoryAllocation) return err;
        err = cudaSuccess;  // no room for the tables: the sweep kernel draws every mask
      }
    }
  }
  const int passes = (has_target && r->units > 1) ? 2 : 1;
  for (int pass = 0; pass < passes && err == cudaSuccess; ++pass) {
    const int first = plain ? t_start : -1;
    for (int t = first; t < (plain ? S : 0) && err == cudaSuccess; ++t) {
      const int t0 = plain ? t : t_start, t1 = plain ? t + 1 : S;
      if (gm) {
        GraphMscSolve s = make_gm_solve(p, dp, r, seed, has_target && pass == 0, target);
        GraphMscLaunch l = {};
        l.t_begin = t0;
        l.t_end = t1;
        l.resume = t0 > 0;
        l.stop_from_hits = pass == 1;
        l.cluster = cluster;
        l.threads = threads;
        l.own_n = own_n;
        l.own_nnz = own_nnz;
        l.own_lv = own_lv;
        l.planes = planes;
        err = gm_launch(s, l, stream);
      } else if (r->msc) {
        TorusSolve s = make_torus_solve(p, dp, r, seed, has_target && pass == 0, target);
        TorusLaunch l = {};
        l.t_begin = t0;
        l.t_end = t1;
        l.resume = t0 > 0;
        l.stop_from_hits = pass == 1;
        l.cluster = cluster;
        l.threads = threads;
        err = torus_launch(s, l, stream);
      } else {
        CsrSolve s = make_csr_solve(p, dp, r, seed, has_target && pass == 0, target);
        CsrLaunch l = {};
        l.t_begin = t0;
        l.t_end = t1;
        l.resume = t0 > 0;
        l.stop_from_hits = pass == 1;
        l.cluster = cluster;
        l.threads = threads;
        l.quads_per_cta = qpc;
        l.own_n = own_n;
        l.own_nnz = own_nnz;
        err = csr_launch(s, l, stream);
      }
      ++launches;
      if (!plain) break;
    }
  }
  return err;
}

// Final and best states into int8 [R][n] in the caller's vertex order.
cudaError_t unpack_result(const isg_problem *p, const DeviceProblem *dp, const isg_result *r,
                          cudaStream_t stream) {
  cudaError_t err;
  if (r->msc && !r->relabelled) {
    err = unpack_msc(r->d_spins, p->n, r->R, r->d_out, stream);
    if (err == cudaSuccess) err = unpack_msc(r->d_best, p->n, r->R, r->d_out_best, stream);
  } else if (r->msc) {
    err = unpack_msc_relabel(r->d_spins, p->n, r->R, dp->orig, r->d_out, stream);
    if (err == cudaSuccess)
      err = unpack_msc_relabel(r->d_best, p->n, r->R, dp->orig, r->d_out_best, stream);
  } else {
    err = unpack_quads(r->d_spins, p->n, r->R, dp->orig, r->d_out, stream);
    if (err == cudaSuccess)
      err = unpack_quads(r->d_best, p->n, r->R, dp->orig, r->d_out_best, stream);
  }
  return err;
}

isg_result *new_result(const isg_problem *p, int32_t R, int32_t S, bool msc, bool has_target,
                       cudaStream_t stream) {
  isg_result *r = new isg_result();
  cudaGetDevice(&r->device);
  r->stream = stream;
  r->n = p->n;
  r->R = R;
  r->S = S;
  r->has_target = has_target;
  r->msc = msc;
  r->units = msc ? (R + 31) / 32 : (R + 3) / 4;
  r->lanes = msc ? 32 : 4;
  return r;
}

// Threshold levels (half energy changes k) a kernel reads: the torus kernel
// only k = 2 and 4, the graph kernels every k = 0..kmax.
void table_levels(const isg_problem *p, bool torus_words, std::vector<int32_t> &levels) {
  levels.clear();
  if (torus_words) {
    levels = {2, 4};
  } else {
    for (int32_t k = 0; k <= p->kmax; ++k) levels.push_back(k);
  }
}

}  // namespace

// The persistent graph-unit kernel runs a whole replica word in one CTA: it
// needs an instance without fields that the multi-spin graph kernel takes
// (field instances are served as int8 quads, as AUTO runs them), and counts
// that fit its fixed counter planes.
bool served_graph_msc(const isg_problem *p, int threads) {
  if (!graph_msc_ok(p) || !p->field.empty()) return false;
  const int64_t per_thread = (p->n + threads - 1) / threads + p->n_colours;
  return per_thread * std::max(1, p->kmax) < (int64_t(1) << kGraphMscBatchPlanes);
}

// ------------------------------------------------------------------ anneal

// Solve state of a checkpoint: int8 [R][n] final and best spins (+1/-1, the
// caller's vertex order) after the first t_done sweeps of the schedule.
struct ResumeState {
  const int8_t *spins = nullptr, *best = nullptr;
  int32_t t_done = 0;
};

// Pack a checkpoint into the result's device layout (the inverse of the
// unpack kernels: 32-lane words or int8 quads, relabelled vertex order for the
// colour-class kernels; padding lanes hold +1), with the energies of both
// states and t_done as every unit's sweeps done.
isg_status upload_resume(const isg_problem *p, isg_result *r, const ResumeState &rs,
                         cudaStream_t stream) {
  const size_t n = (size_t)p->n, R = (size_t)r->R, units = (size_t)r->units;
  const size_t lanes = units * r->lanes;
  for (const int8_t *a : {rs.spins, rs.best})
    for (size_t x = 0; x < R * n; ++x)
      if (a[x] != 1 && a[x] != -1) return fail(ISG_EINVAL, "spin %zu is not +1 or -1", x);
  std::vector<int64_t> e64(R);
  std::vector<int32_t> e_cur(lanes, 0), e_best(lanes, 0), done(units, rs.t_done);
  isg_status st = isg_energy(p, rs.spins, (int32_t)R, e64.data());
  if (st != ISG_OK) return st;
  for (size_t q = 0; q < R; ++q) e_cur[q] = (int32_t)e64[q];
  st = isg_energy(p, rs.best, (int32_t)R, e64.data());
  if (st != ISG_OK) return st;
  for (size_t q = 0; q < R; ++q) e_best[q] = (int32_t)e64[q];
  auto pack = [&](const int8_t *a, std::vector<uint32_t> &w) {
    w.assign(units * n, r->msc ? 0xFFFFFFFFu : 0x01010101u);
    for (size_t q = 0; q < R; ++q)
      for (size_t v = 0; v < n; ++v) {
        const size_t i = r->relabelled ? (size_t)p->order[v] : v;
        uint32_t &x = w[(q / r->lanes) * n + v];
        if (r->msc) {
          const uint32_t bit = 1u << (q & 31);
          x = a[q * n + i] > 0 ? (x | bit) : (x & ~bit);
        } else {
          const int sh = 8 * (int)(q & 3);
          x = (x & ~(0xFFu << sh)) | ((uint32_t)(uint8_t)a[q * n + i] << sh);
        }
      }
  };
  std::vector<uint32_t> ws, wb;
  pack(rs.spins, ws);
  pack(rs.best, wb);
  cudaError_t err = cudaMemcpyAsync(r->d_spins, ws.data(), 4 * ws.size(), cudaMemcpyHostToDevice,
                                    stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(r->d_best, wb.data(), 4 * wb.size(), cudaMemcpyHostToDevice, stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(r->d_e_cur, e_cur.data(), 4 * lanes, cudaMemcpyHostToDevice, stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(r->d_e_best, e_best.data(), 4 * lanes, cudaMemcpyHostToDevice, stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(r->d_done, done.data(), 4 * units, cudaMemcpyHostToDevice, stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(stream);  // the host vectors go away
  if (err != cudaSuccess) return cuda_fail(err, "uploading the checkpoint");
  r->h2d_bytes += 4 * (int64_t)(ws.size() + wb.size() + 2 * lanes + units);
  return ISG_OK;
}

isg_status anneal_impl(const isg_problem *p, int32_t R, const double *betas, int32_t S,
                       uint64_t seed, int64_t target, const isg_options *opts, cudaStream_t stream,
                       isg_result **out, const ResumeState *rs = nullptr) {
  if (!p || !out) return fail(ISG_EINVAL, "problem and out must not be NULL");
  if (R < 1) return fail(ISG_EINVAL, "replicas must be >= 1 (got %d)", R);
  if (S < 1) return fail(ISG_EINVAL, "sweeps must be >= 1 (got %d)", S);
  isg_status st = check_betas(betas, S);
  if (st != ISG_OK) return st;
  if (rs && (!rs->spins || !rs->best))
    return fail(ISG_EINVAL, "checkpoint spins must not be NULL");
  if (rs && (rs->t_done < 1 || rs->t_done > S))
    return fail(ISG_EINVAL, "sweeps_done must be in [1, sweeps] (got %d)", rs->t_done);
  isg_options o = {};
  if (opts) o = *opts;
  int kernel = o.kernel;
  // AUTO with no explicit shape: the autotuner's measured choice if there is one
  int t_kernel = 0, t_cluster = 0, t_threads = 0, t_qpc = 0;
  const bool tuned = kernel == ISG_KERNEL_AUTO && o.cluster_ctas == 0 && o.threads == 0 &&
                     o.quads_per_cta == 0 &&
                     shape_lookup(p, R, t_kernel, t_cluster, t_threads, t_qpc);
  if (tuned) kernel = t_kernel;
  if (kernel == ISG_KERNEL_AUTO)
    // the multi-spin graph kernel also takes unit-weight instances with fields
    // (measured faster than the int8 kernel on them since its staged build
    // keeps the threshold masks of the next sweep in shared memory)
    kernel = p->torus ? ISG_KERNEL_TORUS_MSC
                      : (graph_msc_ok(p) ? ISG_KERNEL_GRAPH_MSC : ISG_KERNEL_CSR);
  if (kernel < ISG_KERNEL_AUTO || kernel > ISG_KERNEL_GRAPH_MSC)
    return fail(ISG_EINVAL, "unknown kernel %d", kernel);
  if (kernel == ISG_KERNEL_TORUS_MSC && !p->torus)
    return fail(ISG_EINVAL, "the multi-spin-coded torus kernel needs a torus instance");
  if (kernel == ISG_KERNEL_GRAPH_MSC && !graph_msc_ok(p))
    return fail(ISG_EINVAL,
                "the multi-spin-coded graph kernel needs weights +-1 (all +1 with local fields) "
                "and degree + |h| <= 63");
  const bool plain = kernel == ISG_KERNEL_PLAIN;
  const bool gm = kernel == ISG_KERNEL_GRAPH_MSC;
  const bool tmsc = p->torus && (kernel == ISG_KERNEL_TORUS_MSC || plain);
  const bool msc = tmsc || gm;  // 32-lane replica words
  if (o.cluster_ctas < 0 || o.cluster_ctas > 16)
    return fail(ISG_EINVAL, "cluster_ctas must be in [0, 16]");
  // the torus kernel has a 64-register build for CTAs of up to 1,024 threads
  const int max_threads = tmsc ? 1024 : 512;
  if (o.threads != 0 && (o.threads < 32 || o.threads > max_threads || o.threads % 32))
    return fail(ISG_EINVAL, "threads must be a multiple of 32 in [32, %d]", max_threads);
  const bool has_target = target != ISG_NO_TARGET;
  if (has_target && (target < INT32_MIN || target > INT32_MAX))
    return fail(ISG_EINVAL, "target energy outside the int32 range");

  // launch shape: explicit, else measured (isg_autotune), else the default rule
  if (o.quads_per_cta < 0 || o.quads_per_cta > 2)
    return fail(ISG_EINVAL, "quads_per_cta must be 0, 1 or 2");
  if (o.mask_chunk < -1) return fail(ISG_EINVAL, "mask_chunk must be -1, 0 or positive");
  if (o.first_replica < 0 || o.first_replica % 32 != 0 ||
      (int64_t)o.first_replica + R > INT32_MAX)
    return fail(ISG_EINVAL, "first_replica must be a multiple of 32 in [0, 2^31 - 1 - replicas]");
  const int units = msc ? (R + 31) / 32 : (R + 3) / 4;
  int cluster = plain ? 1 : o.cluster_ctas, threads = o.threads, qpc = o.quads_per_cta;
  if (tuned) {
    cluster = t_cluster;
    threads = t_threads;
    qpc = t_qpc;
  }
  if (qpc <= 0 || plain) qpc = 1;
  if (tmsc) {
    torus_shape(p->L, p->W, units, cluster, threads);
    if (cluster > p->L) cluster = p->L;
    if (torus_smem_bytes(p->L, p->W, cluster) > 227 * 1024)
      return fail(ISG_EINVAL, "torus %dx%d needs more shared memory than a CTA has", p->L, p->W);
  } else if (gm) {
    gm_shape(p, units, cluster, threads);
    if (gm_bytes(p, cluster, false) > 227 * 1024)
      return fail(ISG_EINVAL, "instance with n = %d needs more shared memory than a CTA has",
                  p->n);
    if (gm_planes_for(p, cluster, threads) < 0)
      return fail(ISG_EINVAL, "too many vertices per thread for the graph kernel's counters");
  } else {
    csr_shape((units + qpc - 1) / qpc, max_class_size(p), cluster, threads);
    if (csr_bytes(p, qpc, cluster, false) > 227 * 1024)
      return fail(ISG_EINVAL, "instance with n = %d needs more shared memory than a CTA has",
                  p->n);
  }

  const DeviceProblem *dp = nullptr;
  size_t uploaded = 0;
  st = problem_device(p, tmsc ? kNeedTorus : kNeedCsr, &dp, &uploaded);
  if (st != ISG_OK) return st;

  isg_result *r = new_result(p, R, S, msc, has_target, stream);
  r->first_replica = o.first_replica;
  r->mask_chunk = o.mask_chunk;
  r->h2d_bytes = (int64_t)uploaded;
  r->relabelled = !tmsc;
  r->kernel = kernel;
  std::vector<int32_t> levels;
  table_levels(p, tmsc, levels);
  std::vector<uint32_t> table;
  build_table(betas, S, levels, table);
  r->table_words = table.size();
  r->h2d_bytes += 4 * (int64_t)table.size();

  st = result_alloc(r, stream);
  if (st != ISG_OK) {
    delete r;
    return st;
  }
  cudaError_t err = cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming);
  if (err == cudaSuccess && o.time_kernels) {
    r->timed = true;
    err = cudaEventCreate(&r->t0);
    if (err == cudaSuccess) err = cudaEventCreate(&r->t1);
  }
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(r->d_table, table.data(), 4 * table.size(), cudaMemcpyHostToDevice,
                          stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(r->d_hit, 0xFF, 4 * (size_t)r->units, stream);
  if (err != cudaSuccess) {
    result_free(r);
    return cuda_fail(err, "preparing the solve");
  }
  if (rs) {
    st = upload_resume(p, r, *rs, stream);
    if (st != ISG_OK) {
      result_free(r);
      return st;
    }
  }
  r->ctas = (msc ? r->units : (r->units + qpc - 1) / qpc) * cluster;
  r->cluster = cluster;
  r->threads = threads;

  int launches = 0;
  if (r->timed) err = cudaEventRecord(r->t0, stream);
  if (err == cudaSuccess)
    err = launch_sweeps(p, dp, r, seed, has_target, target, plain, cluster, threads, qpc, S, stream,
                        launches, rs ? rs->t_done : 0);
  const int sweep_launches = launches;
  if (r->timed && err == cudaSuccess) err = cudaEventRecord(r->t1, stream);
  if (err == cudaSuccess) {
    err = reduce_hits(r->d_hit, r->units, r->d_stop, stream);
    ++launches;
  }
  if (err == cudaSuccess) {
    err = unpack_result(p, dp, r, stream);
    launches += 2;
  }
  if (err == cudaSuccess) err = cudaEventRecord(r->done, stream);
  if (err != cudaSuccess) {
    cudaStreamSynchronize(stream);
    result_free(r);
    return cuda_fail(err, "launching the sweeps");
  }
  r->launches = launches;
  r->sweep_launches = sweep_launches;
  if (!has_target) {
    r->prob = p;
    r->seed = seed;
    r->betas.assign(betas, betas + S);
    r->plain = plain;
    r->qpc = qpc;
  }
  *out = r;
  return ISG_OK;
}

// Continue a solve for more sweeps: sweeps S .. S + extra - 1 of one longer
// schedule, started from the state the solve ended with.  The threshold table
// is rebuilt for the whole schedule (the kernels index it by sweep), and the
// kernels resume from the device state as between the launches of a plain
// solve, so the result equals one solve of the concatenated schedule.
isg_status continue_impl(const isg_problem *p, isg_result *r, const double *betas,
                         int32_t extra, cudaStream_t stream) {
  if (!p || !r) return fail(ISG_EINVAL, "problem and result must not be NULL");
  if (r->prob != p)
    return fail(ISG_EINVAL, "the result is not an isg_anneal solve of this problem without a "
                            "target energy");
  if (extra < 1) return fail(ISG_EINVAL, "sweeps must be >= 1 (got %d)", extra);
  isg_status st = check_betas(betas, extra);
  if (st != ISG_OK) return st;
  if ((int64_t)r->S + extra > INT32_MAX) return fail(ISG_EINVAL, "schedule longer than 2^31 - 1");
  st = result_sync(r);  // the earlier sweeps have finished
  if (st != ISG_OK) return st;
  const bool tmsc = r->msc && !r->relabelled;
  const DeviceProblem *dp = nullptr;
  size_t uploaded = 0;
  st = problem_device(p, tmsc ? kNeedTorus : kNeedCsr, &dp, &uploaded);
  if (st != ISG_OK) return st;
  std::vector<double> all(r->betas);
  all.insert(all.end(), betas, betas + extra);
  std::vector<int32_t> levels;
  table_levels(p, tmsc, levels);
  std::vector<uint32_t> table;
  build_table(all.data(), (int32_t)all.size(), levels, table);
  uint32_t *d_table = nullptr;
  cudaError_t err = cudaMallocAsync(&d_table, 4 * table.size(), stream);
  if (err != cudaSuccess)
    return fail(ISG_ENOMEM, "device allocation of %zu bytes failed: %s", 4 * table.size(),
                cudaGetErrorString(err));
  err = cudaMemcpyAsync(d_table, table.data(), 4 * table.size(), cudaMemcpyHostToDevice, stream);
  if (err != cudaSuccess) {
    cudaFreeAsync(d_table, stream);
    return cuda_fail(err, "uploading the threshold table");
  }
  if (r->d_table_ext) cudaFreeAsync(r->d_table_ext, stream);
  r->d_table_ext = d_table;
  r->d_table = d_table;
  r->table_words = table.size();
  r->h2d_bytes += (int64_t)uploaded + 4 * (int64_t)table.size();
  const int32_t s_old = r->S;
  r->S = (int32_t)all.size();
  r->betas.swap(all);
  r->stream = stream;
  int launches = 0;
  if (r->timed) err = cudaEventRecord(r->t0, stream);
  if (err == cudaSuccess)
    err = launch_sweeps(p, dp, r, r->seed, false, 0, r->plain, r->cluster, r->threads, r->qpc,
                        r->S, stream, launches, s_old);
  const int sweep_launches = launches;
  if (r->timed && err == cudaSuccess) err = cudaEventRecord(r->t1, stream);
  if (err == cudaSuccess) {
    err = unpack_result(p, dp, r, stream);
    launches += 2;
  }
  if (err == cudaSuccess) err = cudaEventRecord(r->done, stream);
  {
    std::lock_guard<std::mutex> lock(r->mu);
    r->synced = false;
  }
  if (err != cudaSuccess) {
    cudaStreamSynchronize(stream);
    r->prob = nullptr;  // the state is no longer a valid solve
    return cuda_fail(err, "launching the continued sweeps");
  }
  r->launches += launches;
  r->sweep_launches += sweep_launches;
  return ISG_OK;
}

// ------------------------------------------------------------------ tempering

// Parallel tempering on a torus: word k = temperature slot k (32 chains), one
// torus-kernel launch of `per_round` sweeps per round at each word's own beta,
// then the exchange kernel over the pairs of the round's parity.
isg_status tempering_impl(const isg_problem *p, int32_t K, const double *betas, int32_t rounds,
                          int32_t per_round, int32_t icm_slots, uint64_t seed,
                          const isg_options *opts, cudaStream_t stream, isg_result **out) {
  if (!out) return fail(ISG_EINVAL, "out must not be NULL");
  *out = nullptr;
  if (!p) return fail(ISG_EINVAL, "problem must not be NULL");
  // tori run on the multi-spin torus kernel, +-1 graphs (all +1 with local
  // fields) of degree + |h| <= 63 on the multi-spin graph kernel, other graphs
  // (general integer weights, fields on other weights) on the int8 kernel
  const bool gm = !p->torus && graph_msc_ok(p);
  const bool quad = !p->torus && !gm;
  if (K < 1 || K > 4096) return fail(ISG_EINVAL, "temperatures must be in [1, 4096]");
  if (rounds < 1 || per_round < 1 || (int64_t)rounds * per_round > INT32_MAX)
    return fail(ISG_EINVAL, "rounds and sweeps_per_round must be >= 1 (product < 2^31)");
  isg_status st = check_betas(betas, K);
  if (st != ISG_OK) return st;
  if (icm_slots < 0 || icm_slots > K) return fail(ISG_EINVAL, "icm_slots must be in [0, K]");
  if (icm_slots > 0 && !gm && 8 * (size_t)p->n > 227 * 1024 - 4096)
    return fail(ISG_EINVAL, "cluster moves on a torus need 8 bytes of shared memory per site "
                            "(n <= 28544)");
  if (icm_slots > 0 && quad)
    return fail(ISG_EINVAL, "cluster moves need a torus or a graph the multi-spin kernel takes "
                            "(weights +-1, all +1 with local fields, degree + |h| <= 63)");
  if (icm_slots > 0 && gm && pt_cluster_graph_smem(p->n) > 227 * 1024 - 4096)
    return fail(ISG_EINVAL, "cluster moves on a graph need 12 bytes of shared memory per vertex "
                            "(n <= 19029)");
  isg_options o = {};
  if (opts) o = *opts;
  const int mkernel =
      quad ? ISG_KERNEL_CSR : (gm ? ISG_KERNEL_GRAPH_MSC : ISG_KERNEL_TORUS_MSC);
  if (o.kernel != ISG_KERNEL_AUTO && o.kernel != mkernel)
    return fail(ISG_EINVAL, "parallel tempering of this instance uses kernel %d", mkernel);
  if (o.quads_per_cta < 0 || o.quads_per_cta > 2)
    return fail(ISG_EINVAL, "quads_per_cta must be 0, 1 or 2");
  if (o.cluster_ctas < 0 || o.cluster_ctas > 16)
    return fail(ISG_EINVAL, "cluster_ctas must be in [0, 16]");
  if (o.threads != 0 && (o.threads < 32 || o.threads > 1024 || o.threads % 32))
    return fail(ISG_EINVAL, "threads must be a multiple of 32 in [32, 1024]");
  const int32_t R = 32 * K, S = rounds * per_round;
  int cluster = o.cluster_ctas, threads = o.threads;
  int t_kernel = 0, t_cluster = 0, t_threads = 0, t_qpc = 0;
  if (cluster == 0 && threads == 0 && shape_lookup(p, R, t_kernel, t_cluster, t_threads, t_qpc) &&
      t_kernel == mkernel) {
    cluster = t_cluster;
    threads = t_threads;
  }
  int own_n = 0, own_nnz = 0, own_lv = 0, planes = 0;
  // int8 kernel: 8 quads per slot; a CTA's 1 or 2 quads lie in one slot
  const int qpc = quad ? (o.quads_per_cta > 0 ? o.quads_per_cta : 1) : 1;
  if (quad) {
    csr_shape((8 * K + qpc - 1) / qpc, max_class_size(p), cluster, threads);
    if (csr_bytes(p, qpc, cluster, false) > 227 * 1024)
      return fail(ISG_EINVAL, "instance with n = %d needs more shared memory than a CTA has",
                  p->n);
    if (csr_bytes(p, qpc, cluster, true) <= 227 * 1024) csr_own_sizes(p, cluster, own_n, own_nnz);
  } else if (!gm) {
    torus_shape(p->L, p->W, K, cluster, threads);
    if (cluster > p->L) cluster = p->L;
    if (torus_smem_bytes(p->L, p->W, cluster) > 227 * 1024)
      return fail(ISG_EINVAL, "torus %dx%d needs more shared memory than a CTA has", p->L, p->W);
  } else {
    gm_shape(p, K, cluster, threads);
    if (gm_bytes(p, cluster, false) > 227 * 1024)
      return fail(ISG_EINVAL, "instance with n = %d needs more shared memory than a CTA has",
                  p->n);
    planes = gm_planes_for(p, cluster, threads);
    if (planes < 0)
      return fail(ISG_EINVAL, "too many vertices per thread for the graph kernel's counters");
    if (gm_bytes(p, cluster, true) <= 227 * 1024) {
      csr_own_sizes(p, cluster, own_n, own_nnz);
      own_lv = gm_own_levels(p, cluster);
    }
  }

  const DeviceProblem *dp = nullptr;
  size_t uploaded = 0;
  st = problem_device(p, p->torus ? kNeedTorus : kNeedCsr, &dp, &uploaded);
  if (st != ISG_OK) return st;
  isg_result *r = new_result(p, R, S, !quad, false, stream);
  r->h2d_bytes = (int64_t)uploaded;
  r->relabelled = !p->torus;
  r->kernel = mkernel;
  // [K][levels]: slot k's thresholds (torus: energy changes 4 and 8; graphs:
  // every half energy change k = 0..kmax)
  std::vector<int32_t> levels;
  table_levels(p, p->torus, levels);
  std::vector<uint32_t> table;
  build_table(betas, K, levels, table);
  r->table_words = table.size();

  // exchange thresholds: pair k, |E_k - E_{k+1}| = d in the direction that
  // makes a = (beta_k - beta_{k+1}) (E_k - E_{k+1}) negative; the table ends
  // where every pair's threshold has reached 0 (|E| <= sum |w|)
  const int32_t pairs = K - 1;
  // |E_k - E_{k+1}| <= 2 (sum |w| + sum |h|)
  int64_t abs_sum = 0;
  if (p->torus) {
    abs_sum = 2 * (int64_t)p->n;
  } else {
    for (const int32_t w : p->wt) abs_sum += w < 0 ? -(int64_t)w : w;
    abs_sum /= 2;  // each edge is in the CSR twice
    for (const int32_t h : p->field) abs_sum += h < 0 ? -(int64_t)h : h;
  }
  const int64_t dmax = 2 * abs_sum;
  std::vector<int8_t> sgn(std::max(pairs, 1), 0);
  int64_t xlen = 1;
  for (int32_t k = 0; k < pairs; ++k) {
    const double db = betas[k] - betas[k + 1];
    sgn[k] = db > 0 ? 1 : (db < 0 ? -1 : 0);
    for (int64_t d = xlen; d <= dmax && sgn[k] != 0; ++d) {
      const double a = db * (double)(-(int64_t)sgn[k] * d);
      if (std::floor(std::ldexp(std::exp(a), 32)) < 1.0) break;
      xlen = d + 1;
    }
  }
  std::vector<uint32_t> xtable((size_t)std::max(pairs, 1) * xlen, 0u);
  for (int32_t k = 0; k < pairs; ++k)
    for (int64_t d = 0; d < xlen && sgn[k] != 0; ++d) {
      const double a = (betas[k] - betas[k + 1]) * (double)(-(int64_t)sgn[k] * d);
      const double x = std::floor(std::ldexp(std::exp(a), 32));
      xtable[(size_t)k * xlen + d] = x >= 4294967295.0 ? 4294967295u : (uint32_t)x;
    }
  r->h2d_bytes += 4 * (int64_t)(table.size() + xtable.size()) + (int64_t)sgn.size();

  st = result_alloc(r, stream);
  if (st != ISG_OK) {
    delete r;
    return st;
  }
  const size_t o_acc = 0, o_flip = 8 * (size_t)std::max(pairs, 1);
  const size_t o_x = o_flip + 8 * (size_t)K;
  const size_t o_sgn = o_x + 4 * xtable.size();
  cudaError_t err = cudaMallocAsync(&r->pt_mem, o_sgn + sgn.size(), stream);
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming);
  if (err == cudaSuccess && o.time_kernels) {
    r->timed = true;
    err = cudaEventCreate(&r->t0);
    if (err == cudaSuccess) err = cudaEventCreate(&r->t1);
  }
  char *pm = (char *)r->pt_mem;
  r->d_accepted = (unsigned long long *)(pm + o_acc);
  r->d_flipped = (unsigned long long *)(pm + o_flip);
  r->pt_pairs = pairs;
  r->pt_slots = K;
  r->pt_attempted.assign(std::max(pairs, 0), 0);
  for (int32_t q = 0; q < rounds; ++q)
    for (int32_t k = q % 2; k + 1 < K; k += 2) r->pt_attempted[k] += 32;
  if (err == cudaSuccess) err = cudaMemsetAsync(pm + o_acc, 0, o_x, stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(pm + o_x, xtable.data(), 4 * xtable.size(), cudaMemcpyHostToDevice,
                          stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(pm + o_sgn, sgn.data(), sgn.size(), cudaMemcpyHostToDevice, stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(r->d_table, table.data(), 4 * table.size(), cudaMemcpyHostToDevice,
                          stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(r->d_hit, 0xFF, 4 * (size_t)r->units, stream);
  if (err != cudaSuccess) {
    cudaStreamSynchronize(stream);
    result_free(r);
    return cuda_fail(err, "preparing parallel tempering");
  }
  r->ctas = (quad ? (8 * K + qpc - 1) / qpc : K) * cluster;
  r->cluster = cluster;
  r->threads = threads;
  r->staged = own_n > 0;

  // one row of thresholds per word, the same every sweep
  TorusSolve s = {};
  GraphMscSolve gs = {};
  CsrSolve qs = {};
  if (quad) {
    qs = make_csr_solve(p, dp, r, seed, false, 0);
    qs.slot_quads = 8;
  } else if (!gm) {
    s = make_torus_solve(p, dp, r, seed, false, 0);
    s.table_ws = 2;
    s.table_ts = 0;
  } else {
    gs = make_gm_solve(p, dp, r, seed, false, 0);
    gs.table_ws = gs.kmax1;
    gs.table_ts = 0;
  }
  const uint32_t key0 = (uint32_t)(seed & 0xFFFFFFFFu), key1 = (uint32_t)(seed >> 32);
  int launches = 0;
  // the rounds are captured once on a private stream and launched as one CUDA
  // graph on the caller's stream (a few microseconds per round instead of a
  // host launch sequence)
  auto enqueue_rounds = [&](cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    for (int32_t q = 0; q < rounds && e == cudaSuccess; ++q) {
      if (quad) {
        CsrLaunch l = {};
        l.t_begin = q * per_round;
        l.t_end = (q + 1) * per_round;
        l.resume = q > 0;
        l.cluster = cluster;
        l.threads = threads;
        l.quads_per_cta = qpc;
        l.own_n = own_n;
        l.own_nnz = own_nnz;
        e = csr_launch(qs, l, st);
      } else if (!gm) {
        TorusLaunch l = {};
        l.t_begin = q * per_round;
        l.t_end = (q + 1) * per_round;
        l.resume = q > 0;
        l.cluster = cluster;
        l.threads = threads;
        e = torus_launch(s, l, st);
      } else {
        GraphMscLaunch l = {};
        l.t_begin = q * per_round;
        l.t_end = (q + 1) * per_round;
        l.resume = q > 0;
        l.cluster = cluster;
        l.threads = threads;
        l.own_n = own_n;
        l.own_nnz = own_nnz;
        l.own_lv = own_lv;
        l.planes = planes;
        e = gm_launch(gs, l, st);
      }
      if (e == cudaSuccess && icm_slots > 0)
        e = gm ? pt_cluster_graph(r->d_spins, r->d_e_cur, p->n, dp->rowptr, dp->col, dp->orig,
                                  dp->field_r, p->kmax, K - icm_slots, icm_slots, q, key0, key1,
                                  r->d_flipped, st)
               : pt_cluster(r->d_spins, r->d_e_cur, dp->cbits, p->L, p->W, K - icm_slots,
                            icm_slots, q, key0, key1, r->d_flipped, st);
      if (e == cudaSuccess)
        e = (quad ? pt_exchange_quads : pt_exchange)(
            r->d_spins, r->d_e_cur, p->n, K, q % 2, q, key0, key1, (const int8_t *)(pm + o_sgn),
            (const uint32_t *)(pm + o_x), (int32_t)xlen, r->d_accepted, st);
    }
    return e;
  };
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&r->pt_capture, cudaStreamNonBlocking);
  if (err == cudaSuccess)
    err = cudaStreamBeginCapture(r->pt_capture, cudaStreamCaptureModeThreadLocal);
  if (err == cudaSuccess) {
    const cudaError_t e1 = enqueue_rounds(r->pt_capture);
    err = cudaStreamEndCapture(r->pt_capture, &r->pt_graph);
    if (err == cudaSuccess) err = e1;
  }
  if (err == cudaSuccess) err = cudaGraphInstantiate(&r->pt_exec, r->pt_graph, 0);
  if (r->timed && err == cudaSuccess) err = cudaEventRecord(r->t0, stream);
  if (err == cudaSuccess) err = cudaGraphLaunch(r->pt_exec, stream);
  launches += rounds * (icm_slots > 0 ? 3 : 2);
  const int sweep_launches = rounds;
  if (r->timed && err == cudaSuccess) err = cudaEventRecord(r->t1, stream);
  if (err == cudaSuccess) err = reduce_hits(r->d_hit, r->units, r->d_stop, stream);
  if (err == cudaSuccess)
    err = quad ? unpack_quads(r->d_spins, p->n, R, dp->orig, r->d_out, stream)
               : gm ? unpack_msc_relabel(r->d_spins, p->n, R, dp->orig, r->d_out, stream)
                    : unpack_msc(r->d_spins, p->n, R, r->d_out, stream);
  if (err == cudaSuccess)
    err = quad ? unpack_quads(r->d_best, p->n, R, dp->orig, r->d_out_best, stream)
               : gm ? unpack_msc_relabel(r->d_best, p->n, R, dp->orig, r->d_out_best, stream)
                    : unpack_msc(r->d_best, p->n, R, r->d_out_best, stream);
  launches += 3;
  if (err == cudaSuccess) err = cudaEventRecord(r->done, stream);
  if (err != cudaSuccess) {
    cudaStreamSynchronize(stream);
    result_free(r);
    return cuda_fail(err, "launching parallel tempering");
  }
  r->launches = launches;
  r->sweep_launches = sweep_launches;
  *out = r;
  return ISG_OK;
}

// ------------------------------------------------------------------ autotune

isg_status autotune_impl(const isg_problem *p, int32_t R, int32_t probe, cudaStream_t stream,
                         isg_options *best) {
  if (!p) return fail(ISG_EINVAL, "problem must not be NULL");
  if (R < 1 || probe < 1) return fail(ISG_EINVAL, "replicas and probe_sweeps must be >= 1");
  // candidate kernel families: the torus kernel for tori; for +-1 graphs both
  // the multi-spin graph kernel and the int8 colour-class kernel
  std::vector<int> kernels;
  if (p->torus)
    kernels = {ISG_KERNEL_TORUS_MSC};
  else if (graph_msc_ok(p))
    kernels = {ISG_KERNEL_GRAPH_MSC, ISG_KERNEL_CSR};
  else
    kernels = {ISG_KERNEL_CSR};
  float best_ms = 1e30f;
  int best_kernel = 0, best_cluster = 0, best_threads = 0, best_qpc = 1;
  for (const int kernel : kernels) {
  const bool msc = kernel == ISG_KERNEL_TORUS_MSC;  // torus words
  const bool gm = kernel == ISG_KERNEL_GRAPH_MSC;   // graph words
  const DeviceProblem *dp = nullptr;
  isg_status st = problem_device(p, msc ? kNeedTorus : kNeedCsr, &dp);
  if (st != ISG_OK) return st;
  // scratch solve at a mid-schedule temperature (both torus thresholds non-zero)
  isg_result *r = new_result(p, R, probe, msc || gm, false, stream);
  r->relabelled = !msc;
  std::vector<int32_t> levels;
  table_levels(p, msc, levels);
  std::vector<double> betas(probe, 1.0);
  std::vector<uint32_t> table;
  build_table(betas.data(), probe, levels, table);
  r->table_words = table.size();
  // tori: shapes are ranked with every mask drawn, since a probe's few sweeps
  // would make the torus chunks too short to compare (the chosen shape then
  // precomputes in solves where that pays); graphs: with the masks chosen as
  // in a solve (a probe of 64 or more sweeps makes one chunk of precomputed
  // masks, whose build and data-flow synchronisation favour other shapes)
  r->mask_chunk = p->torus ? -1 : 0;
  st = result_alloc(r, stream);
  if (st != ISG_OK) {
    delete r;
    return st;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(r->d_table, table.data(), 4 * table.size(), cudaMemcpyHostToDevice,
                          stream);
  const int units = r->units;
  const int max_class = msc ? 0 : max_class_size(p);
  std::vector<int> thread_opts = {128, 192, 256, 384, 512};
  if (msc) thread_opts.insert(thread_opts.end(), {640, 768, 1024});
  for (int qpc = 1; qpc <= (msc || gm ? 1 : 2) && err == cudaSuccess; ++qpc)
  for (int cluster = 1; cluster <= 16 && err == cudaSuccess; ++cluster) {
    if (msc && (cluster > p->L || torus_smem_bytes(p->L, p->W, cluster) > 227 * 1024)) continue;
    if (gm && gm_bytes(p, cluster, false) > 227 * 1024) continue;
    if (!msc && !gm && csr_bytes(p, qpc, cluster, false) > 227 * 1024) continue;
    const int groups = msc || gm ? units : (units + qpc - 1) / qpc;
    if (cluster > 1 && groups * cluster > 4 * sm_count()) continue;
    for (int threads : thread_opts) {
      if (msc) {
        if (torus_sites_per_thread(p->L, p->W, cluster, threads) * 4 >= 1024) continue;
        if (torus_max_active_clusters(p->L, p->W, units, cluster, threads) < 1) continue;
      } else if (threads > round_up((max_class + cluster - 1) / cluster, 32) + 32) {
        continue;
      } else if (gm && gm_planes_for(p, cluster, threads) < 0) {
        continue;
      }
      int launches = 0;
      // untimed warm launch, then one timed launch of the probe
      cudaError_t e = launch_sweeps(p, dp, r, 1, false, 0, false, cluster, threads, qpc, probe,
                                    stream, launches);
      if (e == cudaSuccess) e = cudaEventRecord(e0, stream);
      if (e == cudaSuccess)
        e = launch_sweeps(p, dp, r, 1, false, 0, false, cluster, threads, qpc, probe, stream,
                          launches);
      if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
      if (e != cudaSuccess) {
        // a shape the device cannot launch: skip it (launch errors are not sticky)
        cudaGetLastError();
        if (cudaStreamSynchronize(stream) != cudaSuccess) {
          err = e;
          break;
        }
        continue;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best_kernel = kernel;
        best_cluster = cluster;
        best_threads = threads;
        best_qpc = qpc;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(stream);
  cudaFreeAsync(r->base, stream);
  r->base = nullptr;
  delete r;
  if (err != cudaSuccess) return cuda_fail(err, "autotuning");
  }  // kernel families
  if (best_cluster == 0) return fail(ISG_EINVAL, "no launch shape fits this instance");
  {
    std::lock_guard<std::mutex> lock(g_shape_mu);
    g_shapes[shape_key(p, R)] = {best_kernel, best_cluster, best_threads, best_qpc};
  }
  if (best) {
    best->kernel = best_kernel;
    best->cluster_ctas = best_cluster;
    best->threads = best_threads;
    best->time_kernels = 0;
    best->quads_per_cta = best_kernel == ISG_KERNEL_CSR ? best_qpc : 0;
  }
  return ISG_OK;
}

}  // namespace isg

// ====================================================================== C ABI

using namespace isg;

extern "C" {

const char *isg_last_error(void) { return g_last_error.c_str(); }

const char *isg_version(void) { return "isg 0.1 (sm_103a)"; }

isg_status isg_acceptance_table(const double *betas, int32_t sweeps, int32_t kmax,
                                uint32_t *out) {
  if (!betas || !out) return fail(ISG_EINVAL, "betas and out must not be NULL");
  if (sweeps < 1) return fail(ISG_EINVAL, "sweeps must be >= 1 (got %d)", sweeps);
  if (kmax < 0) return fail(ISG_EINVAL, "kmax must be >= 0 (got %d)", kmax);
  const isg_status st = check_betas(betas, sweeps);
  if (st != ISG_OK) return st;
  std::vector<int32_t> levels(kmax + 1);
  std::iota(levels.begin(), levels.end(), 0);
  std::vector<uint32_t> table;
  build_table(betas, sweeps, levels, table);
  std::copy(table.begin(), table.end(), out);
  return ISG_OK;
}

isg_status isg_problem_create_edges(int32_t n, int64_t m, const int32_t *u, const int32_t *v,
                                    const int32_t *w, isg_problem **out) {
  if (!out) return fail(ISG_EINVAL, "out must not be NULL");
  *out = nullptr;
  isg_problem *p = new isg_problem();
  isg_status st = csr_from_edges(p, n, m, u, v, w);
  if (st == ISG_OK) st = finish_problem(p);
  if (st != ISG_OK) {
    delete p;
    return st;
  }
  *out = p;
  return ISG_OK;
}

isg_status isg_problem_create_fields(int32_t n, int64_t m, const int32_t *u, const int32_t *v,
                                    const int32_t *w, const int32_t *h, isg_problem **out) {
  if (!out) return fail(ISG_EINVAL, "out must not be NULL");
  *out = nullptr;
  isg_problem *p = new isg_problem();
  isg_status st = csr_from_edges(p, n, m, u, v, w);
  if (st == ISG_OK && h) p->field.assign(h, h + n);
  if (st == ISG_OK) st = finish_problem(p);
  if (st != ISG_OK) {
    delete p;
    return st;
  }
  *out = p;
  return ISG_OK;
}

isg_status isg_problem_create_csr(int32_t n, const int64_t *rowptr, const int32_t *col,
                                  const int32_t *w, isg_problem **out) {
  if (!out) return fail(ISG_EINVAL, "out must not be NULL");
  *out = nullptr;
  if (n < 1) return fail(ISG_EINVAL, "n must be >= 1 (got %d)", n);
  if (!rowptr) return fail(ISG_EINVAL, "rowptr must not be NULL");
  if (rowptr[0] != 0) return fail(ISG_EINVAL, "rowptr[0] must be 0");
  for (int32_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return fail(ISG_EINVAL, "rowptr must be non-decreasing");
  const int64_t nnz = rowptr[n];
  if (nnz % 2) return fail(ISG_EINVAL, "a symmetric CSR has an even number of entries");
  if (nnz > 0 && (!col || !w)) return fail(ISG_EINVAL, "col and w must not be NULL");
  // collect (i < j) entries, checking that each has its mirror with the same weight
  std::vector<int32_t> eu, ev, ew;
  for (int32_t i = 0; i < n; ++i)
    for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
      const int32_t j = col[q];
      if (j < 0 || j >= n) return fail(ISG_EINVAL, "column %d outside [0, %d)", j, n);
      if (j == i) return fail(ISG_EINVAL, "vertex %d has a self-loop", i);
      bool mirrored = false;
      for (int64_t z = rowptr[j]; z < rowptr[j + 1]; ++z)
        if (col[z] == i && w[z] == w[q]) mirrored = true;
      if (!mirrored)
        return fail(ISG_EINVAL, "entry (%d, %d) has no mirror (%d, %d) of equal weight", i, j, j,
                    i);
      if (i < j) {
        eu.push_back(i);
        ev.push_back(j);
        ew.push_back(w[q]);
      }
    }
  if ((int64_t)eu.size() * 2 != nnz) return fail(ISG_EINVAL, "CSR entries are not symmetric");
  return isg_problem_create_edges(n, (int64_t)eu.size(), eu.data(), ev.data(), ew.data(), out);
}

isg_status isg_problem_create_torus(int32_t L, int32_t W, const int8_t *j_right,
                                    const int8_t *j_down, isg_problem **out) {
  if (!out) return fail(ISG_EINVAL, "out must not be NULL");
  *out = nullptr;
  if (L < 4 || W < 4 || (L & 1) || (W & 1))
    return fail(ISG_EINVAL, "torus sides must be even and >= 4 (got %d x %d)", L, W);
  if ((int64_t)L * W >= (int64_t(1) << 28)) return fail(ISG_EINVAL, "torus too large");
  if (!j_right || !j_down) return fail(ISG_EINVAL, "coupling arrays must not be NULL");
  const int32_t n = L * W;
  for (int32_t i = 0; i < n; ++i)
    if ((j_right[i] != 1 && j_right[i] != -1) || (j_down[i] != 1 && j_down[i] != -1))
      return fail(ISG_EINVAL, "torus coupling at site %d is not +1 or -1", i);
  std::vector<int32_t> u(2 * (size_t)n), v(2 * (size_t)n), w(2 * (size_t)n);
  for (int32_t r = 0; r < L; ++r)
    for (int32_t c = 0; c < W; ++c) {
      const int32_t i = r * W + c;
      u[2 * i] = i;
      v[2 * i] = r * W + (c + 1) % W;
      w[2 * i] = j_right[i];
      u[2 * i + 1] = i;
      v[2 * i + 1] = ((r + 1) % L) * W + c;
      w[2 * i + 1] = j_down[i];
    }
  isg_problem *p = new isg_problem();
  p->torus = true;
  p->L = L;
  p->W = W;
  p->jr.assign(j_right, j_right + n);
  p->jd.assign(j_down, j_down + n);
  isg_status st = csr_from_edges(p, n, 2 * (int64_t)n, u.data(), v.data(), w.data());
  if (st == ISG_OK) st = finish_problem(p);
  if (st != ISG_OK) {
    delete p;
    return st;
  }
  *out = p;
  return ISG_OK;
}

isg_status isg_problem_info(const isg_problem *p, int32_t *n, int64_t *m, int64_t *total_weight,
                            int32_t *n_colors, int32_t *colors) {
  if (!p) return fail(ISG_EINVAL, "problem must not be NULL");
  if (n) *n = p->n;
  if (m) *m = p->m;
  if (total_weight) *total_weight = p->total_weight;
  if (n_colors) *n_colors = p->n_colours;
  if (colors) std::copy(p->colour.begin(), p->colour.end(), colors);
  return ISG_OK;
}

isg_status isg_problem_set_colouring(isg_problem *p, int32_t method) {
  if (!p) return fail(ISG_EINVAL, "problem must not be NULL");
  if (method != ISG_COLOURING_GREEDY && method != ISG_COLOURING_SMALLEST_LAST)
    return fail(ISG_EINVAL, "unknown colouring %d", method);
  if (p->torus) return fail(ISG_EINVAL, "a torus keeps its (r + c) mod 2 checkerboard");
  std::lock_guard<std::mutex> lock(p->mu);
  if (!p->dev.empty())
    return fail(ISG_EBUSY, "the instance already has device state: set the colouring before "
                           "its first solve");
  p->colouring = method;
  return colour_and_relabel(p);
}

void isg_problem_destroy(isg_problem *p) {
  if (!p) return;
  free_device(p);
  delete p;
}

isg_status isg_anneal(const isg_problem *p, int32_t replicas, const double *betas, int32_t sweeps,
                      uint64_t seed, int64_t target_energy, void *cuda_stream, isg_result **out) {
  return anneal_impl(p, replicas, betas, sweeps, seed, target_energy, nullptr,
                     (cudaStream_t)cuda_stream, out);
}

isg_status isg_autotune(const isg_problem *p, int32_t replicas, int32_t probe_sweeps,
                        void *cuda_stream, isg_options *best) {
  return autotune_impl(p, replicas, probe_sweeps, (cudaStream_t)cuda_stream, best);
}

isg_status isg_anneal_ex(const isg_problem *p, int32_t replicas, const double *betas,
                         int32_t sweeps, uint64_t seed, int64_t target_energy,
                         const isg_options *opts, void *cuda_stream, isg_result **out) {
  return anneal_impl(p, replicas, betas, sweeps, seed, target_energy, opts,
                     (cudaStream_t)cuda_stream, out);
}

isg_status isg_anneal_resume(const isg_problem *p, int32_t replicas, const double *betas,
                             int32_t sweeps, uint64_t seed, int32_t sweeps_done,
                             const int8_t *spins, const int8_t *best_spins,
                             const isg_options *opts, void *cuda_stream, isg_result **out) {
  ResumeState rs;
  rs.spins = spins;
  rs.best = best_spins;
  rs.t_done = sweeps_done;
  return anneal_impl(p, replicas, betas, sweeps, seed, ISG_NO_TARGET, opts,
                     (cudaStream_t)cuda_stream, out, &rs);
}

isg_status isg_debug_fail_allocations(int32_t count) {
  if (count < 0) return fail(ISG_EINVAL, "count must be >= 0 (got %d)", count);
  isg::g_fail_allocations.store(count);
  return ISG_OK;
}

isg_status isg_anneal_continue(const isg_problem *p, isg_result *result, const double *betas,
                               int32_t sweeps, void *cuda_stream) {
  return continue_impl(p, result, betas, sweeps, (cudaStream_t)cuda_stream);
}

isg_status isg_energy(const isg_problem *p, const int8_t *spins, int32_t replicas,
                      int64_t *energies) {
  if (!p || !spins || !energies) return fail(ISG_EINVAL, "arguments must not be NULL");
  if (replicas < 1 || replicas > 65535) return fail(ISG_EINVAL, "replicas must be in [1, 65535]");
  const DeviceProblem *dp = nullptr;
  isg_status st = problem_device(p, kNeedEnergy, &dp);
  if (st != ISG_OK) return st;
  const int blocks = std::max(1, std::min(64, (p->n + 255) / 256));
  const size_t sbytes = (size_t)replicas * p->n;
  void *mem = nullptr;
  cudaStream_t stream = 0;
  const size_t need = ((sbytes + 255) & ~size_t(255)) + 8 * (size_t)replicas * blocks +
                      8 * (size_t)replicas;
  ISG_CUDA(cudaMallocAsync(&mem, need, stream));
  int8_t *d_s = (int8_t *)mem;
  int64_t *d_scratch = (int64_t *)((char *)mem + ((sbytes + 255) & ~size_t(255)));
  int64_t *d_e = d_scratch + (size_t)replicas * blocks;
  cudaError_t err = cudaMemcpyAsync(d_s, spins, sbytes, cudaMemcpyHostToDevice, stream);
  if (err == cudaSuccess)
    err = energy_csr(dp->rowptr_o, dp->col_o, dp->wt_o, p->n, d_s, replicas, d_scratch, blocks,
                     d_e, stream, dp->field_o);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(energies, d_e, 8 * (size_t)replicas, cudaMemcpyDeviceToHost, stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(stream);
  cudaFreeAsync(mem, stream);
  if (err != cudaSuccess) return cuda_fail(err, "isg_energy");
  return ISG_OK;
}

isg_status isg_result_final(const isg_result *r, int8_t *spins, int32_t *energies,
                            int32_t *sweeps_done) {
  if (!r) return fail(ISG_EINVAL, "result must not be NULL");
  isg_status st = result_sync(r);
  if (st != ISG_OK) return st;
  if (spins) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(r->device);
    cudaError_t err = cudaMemcpy(spins, r->d_out, (size_t)r->R * r->n, cudaMemcpyDeviceToHost);
    cudaSetDevice(prev);
    if (err != cudaSuccess) return cuda_fail(err, "reading final spins");
  }
  if (energies)
    for (int32_t k = 0; k < r->R; ++k) energies[k] = r->h_e_cur[k];
  if (sweeps_done) *sweeps_done = r->sweeps_done;
  return ISG_OK;
}

isg_status isg_best(const isg_result *r, int32_t *best_energy, int32_t *best_replica,
                    int8_t *best_spins, int32_t *per_replica_best, int32_t *hit_sweep) {
  if (!r) return fail(ISG_EINVAL, "result must not be NULL");
  isg_status st = result_sync(r);
  if (st != ISG_OK) return st;
  int32_t be = INT32_MAX, br = 0;
  for (int32_t k = 0; k < r->R; ++k)
    if (r->h_e_best[k] < be) {
      be = r->h_e_best[k];
      br = k;
    }
  if (best_energy) *best_energy = be;
  if (best_replica) *best_replica = br;
  if (per_replica_best)
    for (int32_t k = 0; k < r->R; ++k) per_replica_best[k] = r->h_e_best[k];
  if (hit_sweep) *hit_sweep = r->hit_sweep;
  if (best_spins) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(r->device);
    cudaError_t err = cudaMemcpy(best_spins, r->d_out_best + (size_t)br * r->n, (size_t)r->n,
                                 cudaMemcpyDeviceToHost);
    cudaSetDevice(prev);
    if (err != cudaSuccess) return cuda_fail(err, "reading best spins");
  }
  return ISG_OK;
}

isg_status isg_result_shape(const isg_result *r, int32_t *n, int32_t *replicas, int32_t *sweeps) {
  if (!r) return fail(ISG_EINVAL, "result must not be NULL");
  if (n) *n = r->n;
  if (replicas) *replicas = r->R;
  if (sweeps) *sweeps = r->S;
  return ISG_OK;
}

isg_status isg_result_best_all(const isg_result *r, int8_t *best_spins) {
  if (!r || !best_spins) return fail(ISG_EINVAL, "arguments must not be NULL");
  isg_status st = result_sync(r);
  if (st != ISG_OK) return st;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(r->device);
  cudaError_t err =
      cudaMemcpy(best_spins, r->d_out_best, (size_t)r->R * r->n, cudaMemcpyDeviceToHost);
  cudaSetDevice(prev);
  if (err != cudaSuccess) return cuda_fail(err, "reading best spins");
  return ISG_OK;
}

isg_status isg_parallel_tempering(const isg_problem *p, int32_t temperatures,
                                  const double *betas, int32_t rounds, int32_t sweeps_per_round,
                                  int32_t icm_slots, uint64_t seed, const isg_options *opts,
                                  void *cuda_stream, isg_result **out) {
  return tempering_impl(p, temperatures, betas, rounds, sweeps_per_round, icm_slots, seed, opts,
                        (cudaStream_t)cuda_stream, out);
}

isg_status isg_result_cluster_flips(const isg_result *r, int64_t *flipped, int32_t temperatures) {
  if (!r || !flipped) return fail(ISG_EINVAL, "arguments must not be NULL");
  if (temperatures != r->pt_slots || temperatures < 1)
    return fail(ISG_EINVAL, "the result has %d temperature slots", r->pt_slots);
  isg_status st = result_sync(r);
  if (st != ISG_OK) return st;
  std::vector<unsigned long long> f(temperatures);
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(r->device);
  cudaError_t err = cudaMemcpy(f.data(), r->d_flipped, 8 * (size_t)temperatures,
                               cudaMemcpyDeviceToHost);
  cudaSetDevice(prev);
  if (err != cudaSuccess) return cuda_fail(err, "reading cluster-move sizes");
  for (int32_t k = 0; k < temperatures; ++k) flipped[k] = (int64_t)f[k];
  return ISG_OK;
}

isg_status isg_result_exchanges(const isg_result *r, int64_t *accepted, int64_t *attempted,
                                int32_t pairs) {
  if (!r) return fail(ISG_EINVAL, "result must not be NULL");
  if (pairs != r->pt_pairs || (pairs > 0 && (!accepted || !attempted)))
    return fail(ISG_EINVAL, "the result has %d exchange pairs", r->pt_pairs);
  isg_status st = result_sync(r);
  if (st != ISG_OK) return st;
  if (pairs <= 0) return ISG_OK;
  std::vector<unsigned long long> acc(pairs);
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(r->device);
  cudaError_t err = cudaMemcpy(acc.data(), r->d_accepted, 8 * (size_t)pairs,
                               cudaMemcpyDeviceToHost);
  cudaSetDevice(prev);
  if (err != cudaSuccess) return cuda_fail(err, "reading exchange counts");
  for (int32_t k = 0; k < pairs; ++k) {
    accepted[k] = (int64_t)acc[k];
    attempted[k] = r->pt_attempted[k];
  }
  return ISG_OK;
}

isg_status isg_result_stats(const isg_result *r, isg_stats *stats) {
  if (!r || !stats) return fail(ISG_EINVAL, "arguments must not be NULL");
  isg_status st = result_sync(r);
  if (st != ISG_OK) return st;
  stats->sweep_kernel_ms = r->timed ? r->kernel_ms : -1.0f;
  stats->launches = r->launches;
  stats->sweep_launches = r->sweep_launches;
  stats->kernel = r->kernel;
  stats->ctas = r->ctas;
  stats->cluster_ctas = r->cluster;
  stats->threads = r->threads;
  stats->h2d_bytes = r->h2d_bytes;
  stats->staged = r->staged;
  stats->first_replica = r->first_replica;
  stats->mask_chunks = r->mask_chunks;
  return ISG_OK;
}

void isg_result_destroy(isg_result *r) { result_free(r); }

}  // extern "C"
