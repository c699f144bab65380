// isg_noalloc.cu -- isg_energy_noalloc: energies of device-resident spin
// configurations without any device-memory allocation.
//
// Some callers cannot allocate device memory at the moment they need this
// check: a process whose device memory is entirely reserved up front by
// another allocator (a framework's caching pool or a fixed serving budget),
// so that any further cudaMalloc fails or fragments it, and latency-critical
// loops that must not enter the driver's allocator and its locks.  For them
// this entry point takes only caller-owned buffers and keeps its per-block
// partial sums in a statically sized array that is part of the library image.
#include <cstdint>
#include <mutex>

#include "isg.h"
#include "isg_kernels.h"
#include "isg_runtime.h"

namespace isg {
namespace {

// Per-block partial energies: blocks x replicas int64 values.  Every device
// that loads the library holds this array until the process exits.
constexpr int kNoallocBlocks = 32;
constexpr int kNoallocMaxReplicas = 2048;
constexpr size_t kNoallocSlots = (size_t)kNoallocBlocks * kNoallocMaxReplicas;  // 512 KiB
static __device__ __align__(256) int64_t g_energy_scratch[kNoallocSlots];

// Device address of the array, looked up once per device (host code may not
// use the array's name as a device address).
std::mutex g_scratch_mu;
int64_t *g_scratch_ptr[64] = {};

isg_status scratch_address(int device, int64_t **out) {
  if (device < 0 || device >= 64) return fail(ISG_EINVAL, "device index %d out of range", device);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[device]) {
    void *ptr = nullptr;
    const cudaError_t err = cudaGetSymbolAddress(&ptr, g_energy_scratch);
    if (err != cudaSuccess) return cuda_fail(err, "looking up the static scratch array");
    g_scratch_ptr[device] = (int64_t *)ptr;
  }
  *out = g_scratch_ptr[device];
  return ISG_OK;
}

}  // namespace
}  // namespace isg

extern "C" isg_status isg_energy_noalloc(int32_t n, const int64_t *rowptr_dev,
                                         const int32_t *col_dev, const int32_t *w_dev,
                                         const int8_t *spins_dev, int32_t replicas,
                                         int64_t *energies_dev, void *cuda_stream) {
  using namespace isg;
  if (n < 1) return fail(ISG_EINVAL, "n must be >= 1 (got %d)", n);
  if (!rowptr_dev || !col_dev || !w_dev || !spins_dev || !energies_dev)
    return fail(ISG_EINVAL, "device pointers must not be NULL");
  if (replicas < 1 || replicas > kNoallocMaxReplicas)
    return fail(ISG_EINVAL,
                "isg_energy_noalloc handles 1..%d replicas per call (got %d): its scratch is a "
                "fixed %zu-byte array",
                kNoallocMaxReplicas, replicas, sizeof(int64_t) * kNoallocSlots);
  int device = 0;
  cudaError_t err = cudaGetDevice(&device);
  if (err != cudaSuccess) return cuda_fail(err, "cudaGetDevice");
  int64_t *scratch = nullptr;
  isg_status st = scratch_address(device, &scratch);
  if (st != ISG_OK) return st;
  const int blocks = (n + 255) / 256 < kNoallocBlocks ? (n + 255) / 256 : kNoallocBlocks;
  // each block writes its own slot before the finishing pass reads it, so the
  // previous call's contents never leak into this one
  err = energy_csr(rowptr_dev, col_dev, w_dev, n, spins_dev, replicas, scratch, blocks,
                   energies_dev, (cudaStream_t)cuda_stream);
  if (err != cudaSuccess) return cuda_fail(err, "isg_energy_noalloc");
  return ISG_OK;
}
