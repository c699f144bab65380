// pipe_peaks.cu -- throughput of the two integer instructions the sweep kernels
// are made of, measured on the device at hand: the three-input logic op
// (lop3: Philox's XORs, the spin logic, the threshold masks) and the widening
// 32x32->64 multiply by a constant (mul.wide.u32: Philox's products).  These
// rates are the denominators of the sweep kernels' roofline.
//
// Each thread runs eight independent chains; every step's eight results
// depend only on the previous step, so the pipes, not latencies, set the rate
// once each SM holds enough warps.  A second pair of kernels runs the sweeps'
// own Philox code alone, an upper bound on any sweep's rate.
#include <cuda_runtime.h>

#include <cstdint>

#include "isg.h"
#include "isg_device.cuh"
#include "isg_runtime.h"

namespace isg {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;  // steps per loop iteration

__device__ __forceinline__ uint32_t lop3_xor(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// The Philox product: full 64-bit product of a word and a constant, with no
// addend (a 64-bit addend costs extra instructions on both pipes).
__device__ __forceinline__ uint64_t mul_wide_c(uint32_t a, uint32_t b) {
  uint64_t d;
  asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(d) : "r"(a), "r"(b));
  return d;
}

__global__ void __launch_bounds__(256) lop3_rate_kernel(uint32_t *sink, int iters, uint32_t seed) {
  uint32_t x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = seed * (threadIdx.x + 1u) + 0x9E3779B9u * k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      uint32_t y[kChains];
#pragma unroll
      for (int k = 0; k < kChains; ++k)
        y[k] = lop3_xor(x[k], x[(k + 1) % kChains], x[(k + 3) % kChains]);
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = y[k];
    }
  }
  uint32_t acc = 0u;
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc ^= x[k];
  if (acc == seed) sink[blockIdx.x] = acc;  // keeps the chains live
}

// Each step is one Philox half-round: the widening product of the chain word
// and a constant, then the XOR of its two halves with a key word (lop3, on the
// other pipe, at half the multiply's issue cost), exactly the sweeps' form.
__global__ void __launch_bounds__(256) mad_rate_kernel(uint32_t *sink, int iters, uint32_t seed) {
  uint32_t x[kChains];
  const uint32_t mul = 0xD2511F53u ^ (seed & 2u);
  const uint32_t key = 0x9E3779B9u * seed;
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (seed + threadIdx.x) * 0x85EBCA6Bu + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) {
        const uint64_t p = mul_wide_c(x[k], mul);
        x[k] = lop3_xor((uint32_t)(p >> 32), (uint32_t)p, key);
      }
    }
  }
  uint32_t acc = 0u;
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc ^= x[k];
  if (acc == seed) sink[blockIdx.x] = acc;
}

// The sweep's random numbers alone: per site the round-1/2 prefix and eight
// factored Philox4x32-10 blocks (32 uniforms), folded so none is dropped.
// With kMasks, the uniforms are also turned into the sweep's two threshold
// masks.  Their rates bound a sweep from above: every attempt needs one
// uniform.
template <bool kMasks>
__global__ void __launch_bounds__(512) philox_rate_kernel(RoundKeys rk, int sites, uint32_t T4,
                                                          uint32_t T8, uint32_t *sink) {
  BlockPrefix bp[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) bp[q] = block_prefix(24u + q, 7u, rk);
  uint32_t acc = 0u;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < sites; i += gridDim.x * blockDim.x) {
    const SitePrefix sp = site_prefix((uint32_t)i, rk);
    uint32_t a4[2] = {0u, 0u}, a8[2] = {0u, 0u};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint4 u = philox10_factored(sp, bp[q], rk);
      if (kMasks) {
        uint32_t &x4 = a4[q & 1], &x8 = a8[q & 1];
        if (u.x < T4) x4 |= 1u << (4 * q);
        if (u.y < T4) x4 |= 2u << (4 * q);
        if (u.z < T4) x4 |= 4u << (4 * q);
        if (u.w < T4) x4 |= 8u << (4 * q);
        if (u.x < T8) x8 |= 1u << (4 * q);
        if (u.y < T8) x8 |= 2u << (4 * q);
        if (u.z < T8) x8 |= 4u << (4 * q);
        if (u.w < T8) x8 |= 8u << (4 * q);
      } else {
        acc ^= u.x ^ u.y ^ u.z ^ u.w;
      }
    }
    acc ^= (a4[0] | a4[1]) ^ (a8[0] | a8[1]);
  }
  if (acc == 0x12345678u) sink[blockIdx.x] = acc;
}

template <typename Launch>
cudaError_t best_ms_of(Launch launch, cudaStream_t stream, float &best_ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  best_ms = 1e30f;
  for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {  // the first run warms up
    err = cudaEventRecord(e0, stream);
    if (err == cudaSuccess) err = launch();
    if (err == cudaSuccess) err = cudaEventRecord(e1, stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && rep > 0 && ms < best_ms) best_ms = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return err;
}

}  // namespace
}  // namespace isg

using namespace isg;

extern "C" isg_status isg_philox_rates(void *cuda_stream, double *uniforms_per_s,
                                       double *masked_per_s) {
  if (!uniforms_per_s || !masked_per_s) return fail(ISG_EINVAL, "outputs must not be NULL");
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  const int blocks = sm_count() * 2, threads = 512, sites = sm_count() * 512 * 64;
  uint32_t *sink = nullptr;
  cudaError_t err = cudaMallocAsync(&sink, 4 * (size_t)blocks, stream);
  const RoundKeys rk = round_keys(1u, 0u);
  float ms0 = 0.f, ms1 = 0.f;
  if (err == cudaSuccess)
    err = best_ms_of([&] {
      philox_rate_kernel<false><<<blocks, threads, 0, stream>>>(rk, sites, 0x40000000u,
                                                                 0x10000000u, sink);
      return cudaGetLastError();
    }, stream, ms0);
  if (err == cudaSuccess)
    err = best_ms_of([&] {
      philox_rate_kernel<true><<<blocks, threads, 0, stream>>>(rk, sites, 0x40000000u,
                                                                0x10000000u, sink);
      return cudaGetLastError();
    }, stream, ms1);
  if (sink) cudaFreeAsync(sink, stream);
  if (err != cudaSuccess) return cuda_fail(err, "measuring the Philox rates");
  *uniforms_per_s = 32.0 * sites / (ms0 * 1e-3);
  *masked_per_s = 32.0 * sites / (ms1 * 1e-3);
  return ISG_OK;
}

extern "C" isg_status isg_integer_peaks(void *cuda_stream, double *lop3_per_s,
                                        double *mul_wide_per_s) {
  if (!lop3_per_s || !mul_wide_per_s) return fail(ISG_EINVAL, "outputs must not be NULL");
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  const int blocks = sm_count() * 8, threads = 256, iters = 2048;
  const double per_launch = (double)blocks * threads * iters * kUnroll * kChains;
  uint32_t *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaMallocAsync(&sink, 4 * (size_t)blocks, stream);
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  double rate[2] = {0.0, 0.0};
  for (int which = 0; which < 2 && err == cudaSuccess; ++which) {
    float best_ms = 1e30f;
    for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {  // first run warms up
      err = cudaEventRecord(e0, stream);
      if (err == cudaSuccess) {
        if (which == 0)
          lop3_rate_kernel<<<blocks, threads, 0, stream>>>(sink, iters, 12345u);
        else
          mad_rate_kernel<<<blocks, threads, 0, stream>>>(sink, iters, 12345u);
        err = cudaGetLastError();
      }
      if (err == cudaSuccess) err = cudaEventRecord(e1, stream);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      if (err == cudaSuccess && rep > 0 && ms < best_ms) best_ms = ms;
    }
    if (err == cudaSuccess) rate[which] = per_launch / (best_ms * 1e-3);
  }
  if (sink) cudaFreeAsync(sink, stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_fail(err, "measuring integer pipe rates");
  *lop3_per_s = rate[0];
  *mul_wide_per_s = rate[1];
  return ISG_OK;
}
