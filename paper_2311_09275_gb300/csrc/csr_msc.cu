// csr_msc.cu -- host entry points of the multi-spin-coded colour-class sweep
// (kernels in csr_msc.cuh): shared-memory sizes, counter planes, launches
// without local fields, and the persistent unit kernel.
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
