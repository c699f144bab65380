// tempering.cu -- the exchange step of parallel tempering on multi-spin-coded
// state: replica word k holds 32 chains at temperature slot k, so exchanging
// the configurations of chain c between slots k and k+1 moves bit c of every
// site word between the two words (a masked swap), and swaps the chains'
// energies.
#include "isg_device.cuh"
#include "isg_kernels.h"

namespace isg {
namespace {

constexpr uint32_t kTagExchange = 2u;

// One CTA per slot pair (k, k+1), k = parity + 2 * blockIdx.x.
__global__ void __launch_bounds__(256) pt_exchange_kernel(
    uint32_t *spins, int32_t *e_cur, int n, int K, int parity, int round, PhiloxKey key,
    const int8_t *sgn, const uint32_t *xtable, int xlen, unsigned long long *accepted) {
  const int k = parity + 2 * (int)blockIdx.x;
  if (k + 1 >= K) return;
  __shared__ uint32_t s_mask;
  if (threadIdx.x < 32) {
    const int c = (int)threadIdx.x;
    const int32_t ek = e_cur[32 * k + c], ek1 = e_cur[32 * (k + 1) + c];
    const int64_t de = (int64_t)ek - ek1;
    // a = (beta_k - beta_{k+1}) (E_k - E_{k+1}) >= 0: always exchanged
    bool swap = sgn[k] == 0 || de == 0 || (sgn[k] > 0) == (de > 0);
    if (!swap) {
      const int64_t d = de < 0 ? -de : de;
      const uint32_t thr = d < xlen ? xtable[(size_t)k * xlen + d] : 0u;
      const uint4 u = philox10(make_uint4((uint32_t)k, (uint32_t)round, (uint32_t)c >> 2,
                                          kTagExchange), key);
      const uint32_t uc = (c & 3) == 0 ? u.x : (c & 3) == 1 ? u.y : (c & 3) == 2 ? u.z : u.w;
      swap = uc < thr;
    }
    const uint32_t mask = __ballot_sync(0xFFFFFFFFu, swap);
    if (swap) {
      e_cur[32 * k + c] = ek1;
      e_cur[32 * (k + 1) + c] = ek;
    }
    if (c == 0) {
      s_mask = mask;
      if (mask) atomicAdd(&accepted[k], (unsigned long long)__popc(mask));
    }
  }
  __syncthreads();
  const uint32_t mask = s_mask;
  if (mask == 0u) return;
  uint32_t *a = spins + (size_t)k * n;
  uint32_t *b = spins + (size_t)(k + 1) * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const uint32_t x = a[i], y = b[i];
    const uint32_t t = (x ^ y) & mask;
    a[i] = x ^ t;
    b[i] = y ^ t;
  }
}

}  // namespace

cudaError_t pt_exchange(uint32_t *spins, int32_t *e_cur, int32_t n, int32_t K, int32_t parity,
                        int32_t round, uint32_t key0, uint32_t key1, const int8_t *sgn,
                        const uint32_t *xtable, int32_t xlen, unsigned long long *accepted,
                        cudaStream_t stream) {
  const int pairs = (K - parity) / 2;  // pairs (k, k+1) with k = parity, parity + 2, ...
  if (pairs <= 0) return cudaSuccess;
  pt_exchange_kernel<<<pairs, 256, 0, stream>>>(spins, e_cur, n, K, parity, round,
                                                 PhiloxKey{key0, key1}, sgn, xtable, xlen,
                                                 accepted);
  return cudaGetLastError();
}

}  // namespace isg
