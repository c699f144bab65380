// csr_msc.cu -- host entry points of the multi-spin-coded colour-class sweep
// (kernels in csr_msc.cuh): shared-memory sizes, counter planes, launches
// without local fields, the persistent unit kernel, and the kernel that
// precomputes acceptance masks for the staged sweep kernel.
#include "csr_msc.cuh"

namespace isg {
namespace {

// Persistent unit kernel: each CTA takes whole replica words of any instance
// without fields from the queue (K = 1, adjacency not staged).
__global__ void __launch_bounds__(512) gm_batch_kernel(const GraphMscItem *items,
                                                       const int32_t *count_dev,
                                                       const int32_t *order, int32_t *next) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int item;
  const int count = *count_dev;
  const GraphMscLaunch none = {};
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(next, 1);
    __syncthreads();
    const int it = item;
    __syncthreads();
    if (it >= count) break;
    const GraphMscItem u = items[order[it]];
    int t_end = u.t_end;
    if (u.stop_from_hits) {
      // the solve's stop sweep from the first pass (uniform across the CTA)
      int m = INT_MAX;
      for (int w = 0; w < u.solve.words; ++w)
        if (u.solve.hit[w] >= 0 && u.solve.hit[w] < m) m = u.solve.hit[w];
      if (m == INT_MAX) continue;  // no unit reached the target: the first pass stands
      if (m + 1 < t_end) t_end = m + 1;
    }
    gm_word<kGraphMscBatchPlanes, false, false, false>(u.solve, none, u.word, 0, 1, u.t_begin,
                                                       t_end, u.resume, smem);
    __syncthreads();
  }
}

// Acceptance masks of sweeps [t0, t0 + nt) for every replica word and vertex,
// for the staged graph kernel to read instead of drawing them: one CTA per
// (sweep, word), masks of vertex v (relabelled) at out[(sweep - t0, word)
// table of gl words][gloff[v] + level], one word per threshold level
// (d + |h| + 1) / 2, as the sweep kernel builds them itself.
__global__ void __launch_bounds__(256) gm_mask_kernel(GraphMscSolve s, const int32_t *gloff,
                                                      int64_t gl, int32_t t0, uint32_t *out) {
  const int w = (int)(blockIdx.x % (unsigned)s.words);
  const int tt = (int)(blockIdx.x / (unsigned)s.words);
  const int t = t0 + tt;
  const uint32_t uword = (uint32_t)(w + s.rng_word0);
  BlockPrefix bp[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) bp[q] = block_prefix(8u * uword + (uint32_t)q, (uint32_t)t, s.rk);
  const uint32_t *row = s.table + (size_t)w * s.table_ws + (size_t)t * s.table_ts;
  uint32_t *o = out + ((int64_t)tt * s.words + w) * gl;
  for (int v = threadIdx.x; v < s.n; v += blockDim.x) {
    int d = s.rowptr[v + 1] - s.rowptr[v];
    if (s.field) d += abs(s.field[v]);
    const int levels = (d + 1) / 2;
    if (levels == 0) continue;
    uint4 u[8];
    vertex_uniforms((uint32_t)s.orig[v], bp, s.rk, u);
    const uint32_t umin = uniform_min(u);
    uint32_t *ov = o + gloff[v];
    for (int lv = 0; lv < levels; ++lv) {
      const uint32_t T = __ldg(row + d - 2 * lv);
      ov[lv] = T > umin ? uniforms_below(u, T) : 0u;
    }
  }
}

}  // namespace

size_t gm_smem_bytes(int32_t n, int32_t cluster, int32_t n_colours, int32_t own_n,
                     int32_t own_nnz, int32_t own_lv, int32_t kmax1, bool fields) {
  return gm_layout(n, cluster, n_colours, own_n, own_nnz, own_lv, kmax1, fields).total;
}

int gm_planes(int32_t max_count) {
  for (int np : {6, 8, 10, 12, 14})
    if (max_count < (1 << np)) return np;
  return -1;
}

cudaError_t gm_launch(const GraphMscSolve &s, const GraphMscLaunch &l, cudaStream_t stream) {
  return s.field ? gm_launch_fields(s, l, stream) : gm_launch_impl<false>(s, l, stream);
}

cudaError_t gm_mask_launch(const GraphMscSolve &s, const int32_t *gloff_dev, int64_t gl, int32_t t0,
                           int32_t nt, uint32_t *out_dev, cudaStream_t stream) {
  const int64_t grid = (int64_t)nt * s.words;
  if (nt < 1 || grid > INT32_MAX) return cudaErrorInvalidValue;
  gm_mask_kernel<<<(unsigned)grid, 256, 0, stream>>>(s, gloff_dev, gl, t0, out_dev);
  return cudaGetLastError();
}

cudaError_t gm_batch_launch(const GraphMscItem *items_dev, const int32_t *count_dev,
                            const int32_t *order_dev, int32_t *next_dev, int32_t ctas,
                            int32_t threads, size_t smem, cudaStream_t stream) {
  cudaError_t err = cudaFuncSetAttribute(gm_batch_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  gm_batch_kernel<<<ctas, threads, smem, stream>>>(items_dev, count_dev, order_dev, next_dev);
  return cudaGetLastError();
}

}  // namespace isg
