// isg_device.cuh -- device building blocks shared by the annealing kernels:
// the counter-based random numbers, bit-matrix column counts for multi-spin
// coding, and thread-block-cluster helpers.
#pragma once

#include <cooperative_groups.h>
#include <cstdint>

#include "isg_kernels.h"

namespace isg {

namespace cg = cooperative_groups;

// Counter tags of the two random streams (the fourth counter word).
constexpr uint32_t kTagSweep = 0u;
constexpr uint32_t kTagInit = 1u;

// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11).  Each round
// multiplies counter words 0 and 2 by two fixed odd constants (full 64-bit
// products), and mixes the high halves with the other two words and the
// round key; the key advances by two Weyl increments between rounds.  The
// key is the same for every thread of a solve, so the ten round keys are
// uniform values the compiler keeps out of the per-thread work.
struct PhiloxKey {
  uint32_t k0, k1;
};

// Full 64-bit product of two 32-bit words, written as one widening multiply
// (measured faster than separate high- and low-half multiplies).
__device__ __forceinline__ void mul_wide(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo) {
  const uint64_t p = (uint64_t)a * b;
  hi = (uint32_t)(p >> 32);
  lo = (uint32_t)p;
}

__device__ __forceinline__ uint4 philox10(uint4 c, PhiloxKey key) {
  constexpr uint32_t kMulA = 0xD2511F53u;
  constexpr uint32_t kMulB = 0xCD9E8D57u;
  constexpr uint32_t kWeylA = 0x9E3779B9u;
  constexpr uint32_t kWeylB = 0xBB67AE85u;
  uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    uint32_t hiA, loA, hiB, loB;
    mul_wide(kMulA, c.x, hiA, loA);
    mul_wide(kMulB, c.z, hiB, loB);
    c = make_uint4(hiB ^ c.y ^ k0, loB, hiA ^ c.w ^ k1, loA);
    k0 += kWeylA;
    k1 += kWeylB;
  }
  return c;
}

// ---------------------------------------------------------------------------
// Sweep uniforms with rounds 1-2 factored.  For the counter (i, t, b, 0) of
// site i, sweep t and replica block b, round 1 multiplies counter word 0 (=i)
// and word 2 (=b); round 2 multiplies round 1's words 0 and 2.  Round 1's
// word 0 and 1 depend only on (b, t) and its words 2 and 3 only on i, so:
//   after round 2:  ( hi(B*Y2) ^ A_b,  lo(B*Y2),  P_b ^ Y3,  C_b )
// with, per site,  Y2 = hi(A*i) ^ k1[0],  Y3 = lo(A*i),
// and, per (b, t), X0 = hi(B*b) ^ t ^ k0[0],  A_b = lo(B*b) ^ k0[1],
//                  P_b = hi(A*X0) ^ k1[1],   C_b = lo(A*X0),
// where A, B are the two round multipliers.  Rounds 3..10 then run in full.
// The result equals philox10((i, t, b, 0), key) exactly.
constexpr uint32_t kPhiloxMulA = 0xD2511F53u;
constexpr uint32_t kPhiloxMulB = 0xCD9E8D57u;

struct BlockPrefix {
  uint32_t a, p, c;  // A_b, P_b, C_b of the factorisation above
};

__device__ __forceinline__ BlockPrefix block_prefix(uint32_t b, uint32_t t, const RoundKeys &k) {
  uint32_t hb, lb, hx, lx;
  mul_wide(kPhiloxMulB, b, hb, lb);
  const uint32_t x0 = hb ^ t ^ k.k0[0];
  mul_wide(kPhiloxMulA, x0, hx, lx);
  BlockPrefix r;
  r.a = lb ^ k.k0[1];
  r.p = hx ^ k.k1[1];
  r.c = lx;
  return r;
}

struct SitePrefix {
  uint32_t hb, lb, y3;  // hi(B*Y2), lo(B*Y2), Y3
};

__device__ __forceinline__ SitePrefix site_prefix(uint32_t i, const RoundKeys &k) {
  uint32_t hi;
  SitePrefix r;
  mul_wide(kPhiloxMulA, i, hi, r.y3);
  const uint32_t y2 = hi ^ k.k1[0];
  mul_wide(kPhiloxMulB, y2, r.hb, r.lb);
  return r;
}

// Philox4x32-10 of counter (i, t, b, 0) from its two prefixes.
__device__ __forceinline__ uint4 philox10_factored(const SitePrefix &sp, const BlockPrefix &bp,
                                                   const RoundKeys &k) {
  uint4 c = make_uint4(sp.hb ^ bp.a, sp.lb, bp.p ^ sp.y3, bp.c);
#pragma unroll
  for (int round = 2; round < 10; ++round) {
    uint32_t hiA, loA, hiB, loB;
    mul_wide(kPhiloxMulA, c.x, hiA, loA);
    mul_wide(kPhiloxMulB, c.z, hiB, loB);
    c = make_uint4(hiB ^ c.y ^ k.k0[round], loB, hiA ^ c.w ^ k.k1[round], loA);
  }
  return c;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// 32x32 bit-matrix transpose across a warp: lane t enters with row t and
// leaves with column t (bit j of the result = bit t of lane j's input).
// Recursive swap of off-diagonal blocks, 16 -> 8 -> 4 -> 2 -> 1.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (int j = 16; j >= 1; j >>= 1) {
    const uint32_t m = (j == 16) ? 0x0000FFFFu
                     : (j == 8)  ? 0x00FF00FFu
                     : (j == 4)  ? 0x0F0F0F0Fu
                     : (j == 2)  ? 0x33333333u
                                 : 0x55555555u;
    const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, j);
    x = (lane & j) ? ((x & ~m) | ((y >> j) & m)) : ((x & m) | ((y << j) & ~m));
  }
  return x;
}

// Bit-sliced per-lane counter: plane k holds bit k of 32 independent counts
// (one per bit position = one per replica of a multi-spin word).
template <int NP>
struct SlicedCounter {
  uint32_t p[NP];

  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int k = 0; k < NP; ++k) p[k] = 0u;
  }

  // Adds the 3-bit per-lane value (x2 x1 x0).
  __device__ __forceinline__ void add3(uint32_t x0, uint32_t x1, uint32_t x2) {
    uint32_t c = p[0] & x0;
    p[0] ^= x0;
    uint32_t t = p[1] ^ x1;
    uint32_t c2 = (p[1] & x1) | (t & c);
    p[1] = t ^ c;
    c = c2;
    t = p[2] ^ x2;
    c2 = (p[2] & x2) | (t & c);
    p[2] = t ^ c;
    c = c2;
#pragma unroll
    for (int k = 3; k < NP; ++k) {
      const uint32_t cc = p[k] & c;
      p[k] ^= c;
      c = cc;
    }
  }

  // Adds the 2-bit per-lane value (x1 x0).
  __device__ __forceinline__ void add2(uint32_t x0, uint32_t x1) { add3(x0, x1, 0u); }

  // Adds 2^b to the lanes set in x (a carry enters at plane b).
  __device__ __forceinline__ void add_at(int b, uint32_t x) {
    uint32_t c = x;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      if (k >= b) {
        const uint32_t cc = p[k] & c;
        p[k] ^= c;
        c = cc;
      }
    }
  }

  // Adds the per-lane value whose bit-slices are a[0..NA-1].
  template <int NA>
  __device__ __forceinline__ void add_sliced(const uint32_t (&a)[NA]) {
    uint32_t c = 0u;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const uint32_t ak = k < NA ? a[k] : 0u;
      const uint32_t s = p[k] ^ ak ^ c;
      c = (p[k] & ak) | (c & (p[k] ^ ak));
      p[k] = s;
    }
  }

  // Sum over the warp's 32 threads of the count of bit position `lane`
  // (returned in that lane).  Must be called by all 32 lanes.
  __device__ __forceinline__ int32_t warp_lane_total() const {
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < NP; ++k) s += __popc(warp_transpose32(p[k])) << k;
    return s;
  }
};

// Cluster barrier with release/acquire ordering of shared-memory traffic
// (including distributed shared memory) between the CTAs of the cluster.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t cluster_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;\n" : "=r"(r));
  return r;
}

// Address of the same shared-memory object in CTA `rank` of the cluster.
template <typename T>
__device__ __forceinline__ T *peer_smem(T *local, uint32_t rank) {
  return cg::this_cluster().map_shared_rank(local, rank);
}

// Store v at shared-memory address a (a CTA-local shared address) of CTA
// `rank` of the cluster, through the 32-bit cluster window.
__device__ __forceinline__ void st_cluster_u32(uint32_t a, uint32_t rank, uint32_t v) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("st.shared::cluster.u32 [%0], %1;\n" ::"r"(ra), "r"(v));
}

}  // namespace isg
