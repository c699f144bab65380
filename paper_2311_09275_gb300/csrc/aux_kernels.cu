// aux_kernels.cu -- result unpacking and full-energy evaluation.
#include <climits>

#include "isg_device.cuh"
#include "isg_kernels.h"

namespace isg {
namespace {

// out[r][i] = bit (r mod 32) of words[r / 32][i] ? +1 : -1; one thread per
// (replica, site), consecutive threads along i (coalesced int8 stores).
__global__ void unpack_msc_kernel(const uint32_t *__restrict__ words, int n, int R,
                                  int8_t *__restrict__ out) {
  const int64_t total = (int64_t)n * R;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(x / n);
    const int i = (int)(x - (int64_t)r * n);
    const uint32_t w = words[(size_t)(r >> 5) * n + i];
    out[x] = ((w >> (r & 31)) & 1u) ? 1 : -1;
  }
}

// out[r][orig[v]] = bit (r mod 32) of words[r / 32][v] ? +1 : -1.
__global__ void unpack_msc_relabel_kernel(const uint32_t *__restrict__ words, int n, int R,
                                          const int32_t *__restrict__ orig,
                                          int8_t *__restrict__ out) {
  const int64_t total = (int64_t)n * R;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(x / n);
    const int v = (int)(x - (int64_t)r * n);
    const uint32_t w = words[(size_t)(r >> 5) * n + v];
    out[(size_t)r * n + orig[v]] = ((w >> (r & 31)) & 1u) ? 1 : -1;
  }
}

// out[r][orig[v]] = byte (r mod 4) of quads[r / 4][v] (int8 +1/-1).
__global__ void unpack_quads_kernel(const uint32_t *__restrict__ quads, int n, int R,
                                    const int32_t *__restrict__ orig, int8_t *__restrict__ out) {
  const int64_t total = (int64_t)n * R;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(x / n);
    const int v = (int)(x - (int64_t)r * n);
    const uint32_t w = quads[(size_t)(r >> 2) * n + v];
    out[(size_t)r * n + orig[v]] = (int8_t)(uint8_t)(w >> (8 * (r & 3)));
  }
}

// scratch[r * blocks + b] = sum over vertices i of block b's range of
// sum_{j > i} w_ij s_i s_j for replica r (edges counted once, at the lower end).
__global__ void energy_partial_kernel(const int64_t *__restrict__ rowptr,
                                      const int32_t *__restrict__ col,
                                      const int32_t *__restrict__ wt,
                                      const int32_t *__restrict__ field, int n,
                                      const int8_t *__restrict__ spins, int64_t *scratch) {
  const int r = blockIdx.y;
  const int8_t *s = spins + (size_t)r * n;
  int64_t acc = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int32_t si = s[i];
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const int j = col[p];
      if (j > i) acc += (int64_t)wt[p] * si * s[j];
    }
    if (field) acc += (int64_t)field[i] * si;
  }
  __shared__ int64_t red[32];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, off);
  if (lane_id() == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    int64_t v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, off);
    if (threadIdx.x == 0) scratch[(size_t)r * gridDim.x + blockIdx.x] = v;
  }
}

__global__ void energy_finish_kernel(const int64_t *scratch, int blocks, int R, int64_t *out) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    int64_t e = 0;
    for (int b = 0; b < blocks; ++b) e += scratch[(size_t)r * blocks + b];
    out[r] = e;
  }
}

__global__ void reduce_hits_kernel(const int32_t *hit, int count, int32_t *out) {
  int m = INT_MAX;
  for (int q = threadIdx.x; q < count; q += blockDim.x)
    if (hit[q] >= 0 && hit[q] < m) m = hit[q];
  m = __reduce_min_sync(0xFFFFFFFFu, m);
  __shared__ int red[32];
  if (lane_id() == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    int v = INT_MAX;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = red[w] < v ? red[w] : v;
    *out = (v == INT_MAX) ? -1 : v;
  }
}

// Row blockIdx.y of the grid unpacks solve blockIdx.y: out[r][orig[v]] from
// state unit r / lanes at vertex v (bit r mod 32 of a word, byte r mod 4 of a
// quad); the first block also reduces the units' hit sweeps to the stop.
__global__ void batch_unpack_kernel(const BatchOutDesc *__restrict__ descs) {
  const BatchOutDesc d = descs[blockIdx.y];
  const int n = d.n;
  const int64_t total = (int64_t)n * d.R;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(x / n);
    const int v = (int)(x - (int64_t)r * n);
    const size_t at = (size_t)r * n + (d.orig ? d.orig[v] : v);
    const size_t src = (size_t)(r / d.lanes) * n + v;
    if (d.lanes == 32) {
      d.out[at] = ((d.spins[src] >> (r & 31)) & 1u) ? 1 : -1;
      d.out_best[at] = ((d.best[src] >> (r & 31)) & 1u) ? 1 : -1;
    } else {
      d.out[at] = (int8_t)(uint8_t)(d.spins[src] >> (8 * (r & 3)));
      d.out_best[at] = (int8_t)(uint8_t)(d.best[src] >> (8 * (r & 3)));
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int m = INT_MAX;
    for (int u = 0; d.has_target && u < d.units; ++u)
      if (d.hit[u] >= 0 && d.hit[u] < m) m = d.hit[u];
    *d.stop = m == INT_MAX ? -1 : m;
  }
}

int grid_for(int64_t total, int threads) {
  int64_t g = (total + threads - 1) / threads;
  if (g > 152 * 16) g = 152 * 16;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

cudaError_t unpack_msc(const uint32_t *words, int32_t n, int32_t R, int8_t *out,
                       cudaStream_t stream) {
  unpack_msc_kernel<<<grid_for((int64_t)n * R, 256), 256, 0, stream>>>(words, n, R, out);
  return cudaGetLastError();
}

cudaError_t unpack_msc_relabel(const uint32_t *words, int32_t n, int32_t R, const int32_t *orig,
                               int8_t *out, cudaStream_t stream) {
  unpack_msc_relabel_kernel<<<grid_for((int64_t)n * R, 256), 256, 0, stream>>>(words, n, R, orig,
                                                                               out);
  return cudaGetLastError();
}

cudaError_t unpack_quads(const uint32_t *quads, int32_t n, int32_t R, const int32_t *orig,
                         int8_t *out, cudaStream_t stream) {
  unpack_quads_kernel<<<grid_for((int64_t)n * R, 256), 256, 0, stream>>>(quads, n, R, orig, out);
  return cudaGetLastError();
}

cudaError_t energy_csr(const int64_t *rowptr, const int32_t *col, const int32_t *wt, int32_t n,
                       const int8_t *spins, int32_t R, int64_t *scratch, int32_t blocks,
                       int64_t *energies, cudaStream_t stream, const int32_t *field) {
  energy_partial_kernel<<<dim3(blocks, R), 256, 0, stream>>>(rowptr, col, wt, field, n, spins,
                                                               scratch);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  energy_finish_kernel<<<(R + 255) / 256, 256, 0, stream>>>(scratch, blocks, R, energies);
  return cudaGetLastError();
}

cudaError_t batch_unpack(const BatchOutDesc *descs_dev, int32_t count, int64_t max_nr,
                         cudaStream_t stream) {
  int64_t gx = (max_nr + 255) / 256;
  if (gx > 64) gx = 64;
  if (gx < 1) gx = 1;
  batch_unpack_kernel<<<dim3((unsigned)gx, (unsigned)count), 256, 0, stream>>>(descs_dev);
  return cudaGetLastError();
}

cudaError_t reduce_hits(const int32_t *hit, int32_t count, int32_t *out, cudaStream_t stream) {
  reduce_hits_kernel<<<1, 256, 0, stream>>>(hit, count, out);
  return cudaGetLastError();
}

}  // namespace isg
