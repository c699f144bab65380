// torus_msc.cu -- checkerboard Metropolis sweeps on L x W +-1 tori with
// multi-spin coding: 32 replicas per uint32 word, one bit per replica.
//
// Per site and replica word the kernel forms the four "unsatisfied bond"
// words (bond (i,j) is unsatisfied when w_ij s_i s_j = +1), counts them
// bit-sliced (U = 0..4 per replica), and flips replicas with U >= 2 (energy
// change d = 8 - 4U <= 0) outright and those with U = 1 (d = 4) or U = 0
// (d = 8) when their Philox uniform is below the sweep's threshold.
//
// Layout: a cluster of K CTAs owns one replica word of one instance; CTA k
// holds a band of rows plus one halo row above and below in shared memory.
// Sites of one colour never neighbour each other, so a colour phase needs no
// intra-phase synchronisation; updated band-edge rows are written straight
// into the neighbouring CTA's halo (distributed shared memory), and one
// cluster barrier separates the phases.  Per-replica energy changes are
// accumulated in bit-sliced counters and reduced once per sweep.  The
// acceptance masks of a thread's first site of the next phase depend only on
// its uniforms and the sweep's thresholds: they are built between the
// thread's arrival at the phase barrier and the wait for it.
#include <climits>
#include <type_traits>

#include "isg_device.cuh"
#include "isg_kernels.h"

namespace isg {
namespace {

struct Band {
  int r0, nr;
};

__host__ __device__ __forceinline__ Band band_of(int L, int K, int k) {
  const int r0 = (int)((int64_t)k * L / K);
  const int r1 = (int)((int64_t)(k + 1) * L / K);
  return {r0, r1 - r0};
}

__host__ __device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Per-lane energy sums of the cluster: three rotating accumulators of 32
// lanes in every CTA.
constexpr int kAccWords = 3 * 32;

struct SmemLayout {
  size_t spin, best, cb, part, bars, total;
};

__host__ __device__ __forceinline__ SmemLayout layout_of(int nr, int W, int K) {
  SmemLayout m;
  m.spin = 0;
  m.best = m.spin + sizeof(uint32_t) * (size_t)(nr + 2) * W;
  m.cb = m.best + sizeof(uint32_t) * (size_t)nr * W;
  m.part = align16(m.cb + (size_t)(nr + 2) * W);
  m.bars = align16(m.part + sizeof(int32_t) * kAccWords);  // two mbarriers, an error flag
  m.total = align16(m.bars + 32);
  return m;
}

__device__ __forceinline__ uint32_t sign_mask(uint32_t bit) { return 0u - (bit & 1u); }

// Initial spins of sites i for the 32 replicas of `word`: bit l = top bit of
// word (l mod 4) of Philox(i, 0, 8*word + l/4, init tag).
__device__ __forceinline__ uint32_t initial_word(uint32_t i, uint32_t word, PhiloxKey key) {
  uint32_t s = 0u;
#pragma unroll
  for (uint32_t q = 0; q < 8; ++q) {
    const uint4 u = philox10(make_uint4(i, 0u, 8u * word + q, kTagInit), key);
    s |= ((u.x >> 31) << (4 * q)) | ((u.y >> 31) << (4 * q + 1)) | ((u.z >> 31) << (4 * q + 2)) |
         ((u.w >> 31) << (4 * q + 3));
  }
  return s;
}

__device__ __forceinline__ void sync_group(int K) {
  if (K == 1)
    __syncthreads();
  else
    cluster_barrier();
}

// The two halves of the group barrier: work between them overlaps the wait
// for the other CTAs (a CTA-wide barrier when the group is one CTA).
__device__ __forceinline__ void group_arrive(int K) {
  if (K > 1) asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void group_wait(int K) {
  if (K > 1)
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
  else
    __syncthreads();
}

// Data flow between the CTAs of a word (pipelined build): halo cells are
// sent with st.async and the energy sums with red.async, both completing on
// the receiver's mbarrier, so a CTA starts its next phase once its own
// threads and the expected bytes have arrived.  Addresses here are 32-bit
// shared::cluster addresses (mapa of a CTA-local one).
__device__ __forceinline__ uint32_t map_rank(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ __forceinline__ void st_async_cl(uint32_t a, uint32_t v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.u32 [%0], %1, [%2];\n" ::"r"(
                   a),
               "r"(v), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void red_async_add_cl(uint32_t a, int32_t v, uint32_t bar) {
  asm volatile(
      "red.async.relaxed.cluster.shared::cluster.mbarrier::complete_tx::bytes.add.s32 [%0], %1, "
      "[%2];\n" ::"r"(a),
      "r"(v), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint32_t bar, bool expect, uint32_t bytes) {
  if (expect)
    asm volatile(
        "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 st, [%0], "
        "%1;\n}\n" ::"r"(bar),
        "r"(bytes)
        : "memory");
  else
    asm volatile(
        "{\n .reg .b64 st;\n mbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n}\n" ::"r"(
            bar)
        : "memory");
}

__device__ __forceinline__ bool bar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], "
      "%2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// try_wait attempts before a wait counts as failed (far beyond any phase)
constexpr uint32_t kTorusWaitLimit = 1u << 22;

// Atomic add of v at shared-memory address a (a CTA-local shared address) of
// CTA `rank` of the cluster, through the 32-bit cluster window.
__device__ __forceinline__ void red_cluster_add(uint32_t a, uint32_t rank, int32_t v) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("red.shared::cluster.add.s32 [%0], %1;\n" ::"r"(ra), "r"(v) : "memory");
}

// Sum over the whole cluster of the bit-sliced counters, per lane (= per
// replica of the word): every warp adds its lane totals into accumulator m of
// every CTA of the cluster (atomic adds, local or remote), one group barrier,
// then every warp reads the 32 sums; no CTA-wide barrier or serial section is
// needed.  The three accumulators rotate (m = 0, 1, 2, 0, ...): once read, a
// call clears the one the next call adds into, last read two calls before, a
// group barrier lying between any two calls.  `during` runs between the
// arrival at the barrier and the wait for it.
template <int NP, typename During>
__device__ __forceinline__ int32_t cluster_lane_sum(const SlicedCounter<NP> &cnt, int32_t *acc,
                                                    int &m, int K, During during) {
  const int lane = (int)lane_id();
  int32_t *cur = acc + 32 * m;
  const int32_t tot = cnt.warp_lane_total();
  if (K == 1) {
    atomicAdd(cur + lane, tot);
  } else {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(cur + lane);
    for (int q = 0; q < K; ++q) red_cluster_add(a, (uint32_t)q, tot);
  }
  group_arrive(K);
  during();
  group_wait(K);
  const int32_t sum = cur[lane];
  m = m == 2 ? 0 : m + 1;
  if (threadIdx.x < 32) acc[32 * m + lane] = 0;
  return sum;
}

// Acceptance masks of one site-word: lanes whose uniform is below T4 (r4) and
// below T8 (r8, only with kTwoThresholds).  The 32 uniforms are 8 Philox
// blocks of 4 sharing the site's round-1/2 prefix; the masks are built by
// compare + predicated OR into two partial accumulators (measured faster than
// packing 4-bit nibbles, and than moving the compares onto the multiply-add
// pipe).  They do not depend on the spins.
template <bool kTwoThresholds>
__device__ __forceinline__ void site_masks(uint32_t site, const BlockPrefix (&bp)[8],
                                           const RoundKeys &rk, uint32_t T4, uint32_t T8,
                                           uint32_t &r4, uint32_t &r8) {
  const SitePrefix sp = site_prefix(site, rk);
  uint32_t a4[2] = {0u, 0u}, a8[2] = {0u, 0u};
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const uint4 u = philox10_factored(sp, bp[q], rk);
    uint32_t &x4 = a4[q & 1], &x8 = a8[q & 1];
    if (u.x < T4) x4 |= 1u << (4 * q);
    if (u.y < T4) x4 |= 2u << (4 * q);
    if (u.z < T4) x4 |= 4u << (4 * q);
    if (u.w < T4) x4 |= 8u << (4 * q);
    if (kTwoThresholds) {
      if (u.x < T8) x8 |= 1u << (4 * q);
      if (u.y < T8) x8 |= 2u << (4 * q);
      if (u.z < T8) x8 |= 4u << (4 * q);
      if (u.w < T8) x8 |= 8u << (4 * q);
    }
  }
  r4 = a4[0] | a4[1];
  r8 = a8[0] | a8[1];
}

// Masks of this thread's first site of colour c in the band (the phase's
// first loop iteration), drawn ahead of the phase; false if it has none.
__device__ __forceinline__ bool first_site_masks(int W, int r0, int nr, int c,
                                                 const BlockPrefix (&bp)[8], const RoundKeys &rk,
                                                 uint32_t T4, uint32_t T8, uint32_t &r4,
                                                 uint32_t &r8) {
  const int half = W >> 1;
  const int lr = 1 + (int)threadIdx.x / half;
  if (lr > nr) return false;
  const int j = (int)threadIdx.x - (lr - 1) * half;
  const int gr = r0 + lr - 1;
  const uint32_t site = (uint32_t)(gr * W + 2 * j + ((c + gr) & 1));
  if (T8 != 0u)
    site_masks<true>(site, bp, rk, T4, T8, r4, r8);
  else
    site_masks<false>(site, bp, rk, T4, T8, r4, r8);
  return true;
}

// One colour phase of one replica word: this thread's sites of colour c in
// the CTA's band; the first one's masks come in (pre4, pre8) when `ready`.
// Replicas in `imp` improved their best energy at the end of the previous
// sweep; their best state is taken here, site by site, from the spins as they
// stand before this phase updates them (unchanged since that sweep's end).
template <int NP, bool kTwoThresholds>
__device__ __forceinline__ void sweep_phase(uint32_t *spin, uint32_t *best, const uint8_t *cb,
                                            uint32_t *up_peer, uint32_t *down_peer, int W, int r0,
                                            int nr, int c, const BlockPrefix (&bp)[8],
                                            const RoundKeys &rk, uint32_t T4, uint32_t T8,
                                            uint32_t imp, SlicedCounter<NP> &cnt, uint32_t pre4,
                                            uint32_t pre8, bool ready) {
  const int half = W >> 1;
  const int step_rows = blockDim.x / half;
  const int step_cols = blockDim.x - step_rows * half;
  int lr = 1 + (int)threadIdx.x / half;
  int j = (int)threadIdx.x - (lr - 1) * half;
  while (lr <= nr) {
    const int gr = r0 + lr - 1;
    const int col = 2 * j + ((c + gr) & 1);
    const int x = lr * W + col;
    const int xl = (col == 0) ? x + W - 1 : x - 1;
    const int xr = (col == W - 1) ? x - W + 1 : x + 1;
    const uint32_t s0 = spin[x];
    if (imp != 0u) {
      uint32_t &bx = best[x - W];
      bx = (bx & ~imp) | (s0 & imp);
    }
    const uint32_t cbx = cb[x];
    const uint32_t a = ~(s0 ^ spin[xr] ^ sign_mask(cbx));
    const uint32_t b = ~(s0 ^ spin[xl] ^ sign_mask(cb[xl]));
    const uint32_t cu = ~(s0 ^ spin[x - W] ^ sign_mask(cb[x - W] >> 1));
    const uint32_t d = ~(s0 ^ spin[x + W] ^ sign_mask(cbx >> 1));
    // U = a + b + cu + d bit-sliced as (u2 u1 u0)
    const uint32_t s1 = a ^ b, c1 = a & b, s2 = cu ^ d, c2 = cu & d;
    const uint32_t u0 = s1 ^ s2;
    const uint32_t u1 = (c1 ^ c2) | (s1 & s2);
    const uint32_t u2 = c1 & c2;
    const uint32_t eq0 = ~(u0 | u1 | u2);
    const uint32_t eq1 = u0 & ~u1;
    const uint32_t ge2 = u1 | u2;
    uint32_t r4 = pre4, r8 = pre8;
    if (!ready) site_masks<kTwoThresholds>((uint32_t)(gr * W + col), bp, rk, T4, T8, r4, r8);
    ready = false;
    const uint32_t acc = ge2 | (eq1 & r4) | (eq0 & r8);
    const uint32_t sn = s0 ^ acc;
    spin[x] = sn;
    if (lr == 1) up_peer[col] = sn;
    if (lr == nr) down_peer[col] = sn;
    // v = accepted ? 4 - U : 2  (the energy change is 4 (v - 2))
    cnt.add3(acc & u0, (acc & (u0 ^ u1)) | ~acc, acc & eq0);
    j += step_cols;
    lr += step_rows;
    if (j >= half) {
      j -= half;
      ++lr;
    }
  }
}

// Software-pipelined colour phase (a thread with at most kPipeSites sites per
// phase): at each of its positions the thread updates its site of colour c
// with the masks drawn earlier (mc4, mc8) and draws the masks of the other
// colour's site at the same position for the next phase (into mo4, mo8, with
// that phase's block prefixes bp and thresholds To4, To8): the random numbers
// do not depend on the spins, so the independent Philox work of one site and
// the dependent spin logic of another share one straight-line loop body that
// the compiler interleaves.  Both masks are always built (a threshold of 0
// gives an empty mask).
constexpr int kPipeSites = 3;

// LOAD: the other colour's masks are read from a precomputed table (q4, q8:
// that sweep's two mask planes of this word, indexed by site) instead of
// drawn; they are first used in the next phase, which hides the load.
// The band's boundary rows go to the neighbours' halo rows with st.async
// (up_halo, down_halo: their halo rows' cluster addresses; up_bar, down_bar:
// their mbarriers of this phase).
template <int NP, bool LOAD>
__device__ __forceinline__ void pipe_phase(uint32_t *spin, uint32_t *best, const uint8_t *cb,
                                           uint32_t up_halo, uint32_t down_halo, uint32_t up_bar,
                                           uint32_t down_bar, int W, int r0,
                                           int nr, int c, const BlockPrefix (&bp)[8],
                                           const RoundKeys &rk, uint32_t To4, uint32_t To8,
                                           uint32_t imp, SlicedCounter<NP> &cnt,
                                           const uint32_t (&mc4)[kPipeSites],
                                           const uint32_t (&mc8)[kPipeSites],
                                           uint32_t (&mo4)[kPipeSites],
                                           uint32_t (&mo8)[kPipeSites], const uint32_t *q4,
                                           const uint32_t *q8) {
  const int half = W >> 1;
  const int step_rows = blockDim.x / half;
  const int step_cols = blockDim.x - step_rows * half;
  int lr = 1 + (int)threadIdx.x / half;
  int j = (int)threadIdx.x - (lr - 1) * half;
#pragma unroll
  for (int i = 0; i < kPipeSites; ++i) {
    if (lr <= nr) {
      const int gr = r0 + lr - 1;
      const int par = (c + gr) & 1;
      const int col = 2 * j + par;
      // the other colour's site at this position, for the next phase
      const uint32_t osite = (uint32_t)(gr * W + 2 * j + (par ^ 1));
      if (LOAD) {
        mo4[i] = __ldg(q4 + osite);
        mo8[i] = __ldg(q8 + osite);
      } else {
        site_masks<true>(osite, bp, rk, To4, To8, mo4[i], mo8[i]);
      }
      const int x = lr * W + col;
      const int xl = (col == 0) ? x + W - 1 : x - 1;
      const int xr = (col == W - 1) ? x - W + 1 : x + 1;
      const uint32_t s0 = spin[x];
      if (imp != 0u) {
        uint32_t &bx = best[x - W];
        bx = (bx & ~imp) | (s0 & imp);
      }
      const uint32_t cbx = cb[x];
      const uint32_t a = ~(s0 ^ spin[xr] ^ sign_mask(cbx));
      const uint32_t b = ~(s0 ^ spin[xl] ^ sign_mask(cb[xl]));
      const uint32_t cu = ~(s0 ^ spin[x - W] ^ sign_mask(cb[x - W] >> 1));
      const uint32_t d = ~(s0 ^ spin[x + W] ^ sign_mask(cbx >> 1));
      const uint32_t s1 = a ^ b, c1 = a & b, s2 = cu ^ d, c2 = cu & d;
      const uint32_t u0 = s1 ^ s2;
      const uint32_t u1 = (c1 ^ c2) | (s1 & s2);
      const uint32_t u2 = c1 & c2;
      const uint32_t eq0 = ~(u0 | u1 | u2);
      const uint32_t eq1 = u0 & ~u1;
      const uint32_t ge2 = u1 | u2;
      const uint32_t acc = ge2 | (eq1 & mc4[i]) | (eq0 & mc8[i]);
      const uint32_t sn = s0 ^ acc;
      spin[x] = sn;
      if (lr == 1) st_async_cl(up_halo + 4u * (uint32_t)col, sn, up_bar);
      if (lr == nr) st_async_cl(down_halo + 4u * (uint32_t)col, sn, down_bar);
      cnt.add3(acc & u0, (acc & (u0 ^ u1)) | ~acc, acc & eq0);
    }
    j += step_cols;
    lr += step_rows;
    if (j >= half) {
      j -= half;
      ++lr;
    }
  }
}

// The masks of this thread's sites of colour c (the pipeline's first phase),
// drawn, or with LOAD read from a precomputed table as in pipe_phase.
template <bool LOAD>
__device__ __forceinline__ void pipe_prologue(int W, int r0, int nr, int c,
                                              const BlockPrefix (&bp)[8], const RoundKeys &rk,
                                              uint32_t T4, uint32_t T8,
                                              uint32_t (&m4)[kPipeSites],
                                              uint32_t (&m8)[kPipeSites], const uint32_t *q4,
                                              const uint32_t *q8) {
  const int half = W >> 1;
  const int step_rows = blockDim.x / half;
  const int step_cols = blockDim.x - step_rows * half;
  int lr = 1 + (int)threadIdx.x / half;
  int j = (int)threadIdx.x - (lr - 1) * half;
#pragma unroll
  for (int i = 0; i < kPipeSites; ++i) {
    m4[i] = m8[i] = 0u;
    if (lr <= nr) {
      const int gr = r0 + lr - 1;
      const uint32_t site = (uint32_t)(gr * W + 2 * j + ((c + gr) & 1));
      if (LOAD) {
        m4[i] = __ldg(q4 + site);
        m8[i] = __ldg(q8 + site);
      } else {
        site_masks<true>(site, bp, rk, T4, T8, m4[i], m8[i]);
      }
    }
    j += step_cols;
    lr += step_rows;
    if (j >= half) {
      j -= half;
      ++lr;
    }
  }
}

// kPrefetch: draw the first site's masks of each phase during the barrier
// before it (off in the 64-register build, where the extra live state spills).
// kPipe: the software-pipelined phases (every thread has at most kPipeSites
// sites per phase).
// PRE (pipelined build only): the masks of the sweeps [t_begin, t_begin +
// pre_count), precomputed by torus_mask_kernel, are read from pre_tab
// [t - t_begin][word][2 planes][L*W] instead of drawn.
template <int NP, bool kPrefetch, bool kPipe = false, bool PRE = false>
__device__ void torus_word(const TorusSolve &s, int word, int k, int K, int t_begin, int t_end,
                           int resume, uint8_t *smem, const uint32_t *pre_tab = nullptr,
                           int pre_count = 0) {
  const int L = s.L, W = s.W, n = L * W;
  const Band band = band_of(L, K, k);
  const int r0 = band.r0, nr = band.nr;
  // every CTA of the cluster uses the layout of the tallest band, so that a
  // shared-memory offset means the same array in every peer
  const SmemLayout lay = layout_of((L + K - 1) / K, W, K);
  uint32_t *spin = reinterpret_cast<uint32_t *>(smem + lay.spin);
  uint32_t *best = reinterpret_cast<uint32_t *>(smem + lay.best);  // band rows only
  uint8_t *cb = smem + lay.cb;
  int32_t *acc = reinterpret_cast<int32_t *>(smem + lay.part);  // energy accumulators
  int acc_m = 0;                                                   // the next one to add into
  const PhiloxKey key{s.key0, s.key1};
  const uint32_t uword = (uint32_t)(word + s.rng_word0);  // Philox counters only
  const int rem = s.replicas - 32 * word;
  const uint32_t valid = rem >= 32 ? 0xFFFFFFFFu : ((1u << rem) - 1u);
  uint32_t *gspin = s.spins + (size_t)word * n;
  uint32_t *gbest = s.best + (size_t)word * n;
  const int lane = (int)lane_id();

  if (resume && s.has_target && s.hit[word] >= 0) return;  // this solve already stopped
  if (resume && t_begin >= t_end) return;                   // nothing left to run
  if (!resume && s.has_target && k == 0 && threadIdx.x == 0) s.hit[word] = -1;

  // band rows and halos: global row r0 - 1 + lr for lr = 0..nr+1
  for (int x = threadIdx.x; x < (nr + 2) * W; x += blockDim.x) {
    const int lr = x / W;
    const int c = x - lr * W;
    int gr = r0 - 1 + lr;
    gr = gr < 0 ? gr + L : (gr >= L ? gr - L : gr);
    const int i = gr * W + c;
    cb[x] = s.cbits[i];
    const uint32_t v = resume ? gspin[i] : initial_word((uint32_t)i, uword, key);
    spin[x] = v;
    if (lr >= 1 && lr <= nr) best[x - W] = resume ? gbest[i] : v;
  }
  for (int x = threadIdx.x; x < kAccWords; x += blockDim.x) acc[x] = 0;
  // pipelined build: this CTA's mbarriers (alternating phases) and error flag
  const uint32_t bar_l = (uint32_t)__cvta_generic_to_shared(smem + lay.bars);
  int *dferr = reinterpret_cast<int *>(smem + lay.bars + 16);
  if (kPipe && threadIdx.x == 0) {
    bar_init(bar_l, blockDim.x);
    bar_init(bar_l + 8, blockDim.x);
    *dferr = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // peers write into this CTA's halo rows (and accumulators) only after every
  // CTA has loaded (and cleared) them
  sync_group(K);

  // per-lane (replica) energies, kept identically by every warp
  int32_t e = 0, e_best = 0;
  SlicedCounter<NP> cnt;
  if (!resume) {
    // E = sum over bonds of (+1 unsatisfied, -1 satisfied) = 2 U_tot - 2n
    cnt.clear();
    for (int idx = threadIdx.x; idx < nr * W; idx += blockDim.x) {
      const int x = W + idx;
      const int c = idx % W;
      const uint32_t s0 = spin[x];
      const uint32_t cbx = cb[x];
      const uint32_t a = ~(s0 ^ spin[c == W - 1 ? x - W + 1 : x + 1] ^ sign_mask(cbx));
      const uint32_t d = ~(s0 ^ spin[x + W] ^ sign_mask(cbx >> 1));
      cnt.add2(a ^ d, a & d);
    }
    e = 2 * cluster_lane_sum<NP>(cnt, acc, acc_m, K, [] {}) - 2 * n;
    e_best = e;
  } else {
    e = s.e_cur[word * 32 + lane];
    e_best = s.e_best[word * 32 + lane];
  }

  const int kup = (k + K - 1) % K, kdown = (k + 1) % K;
  uint32_t *up_peer = (K == 1 ? spin : peer_smem(spin, (uint32_t)kup)) +
                      (size_t)(band_of(L, K, kup).nr + 1) * W;
  uint32_t *down_peer = (K == 1 ? spin : peer_smem(spin, (uint32_t)kdown));

  int t = t_begin;
  int hit = -1;
  uint32_t imp = 0u;  // replicas whose best state is the state at the start of sweep t
  // thresholds of the next sweep are loaded one sweep ahead
  const uint32_t *trow = s.table + (size_t)word * s.table_ws;
  uint32_t T4n = 0u, T8n = 0u;
  if (t < t_end) T4n = trow[(size_t)t * s.table_ts], T8n = trow[(size_t)t * s.table_ts + 1];
  // the (block, sweep) part of Philox rounds 1-2, uniform across the CTA
  BlockPrefix bp[8];
  auto sweep_prefix = [&](int tt) {
#pragma unroll
    for (int q = 0; q < 8; ++q) bp[q] = block_prefix(8u * uword + (uint32_t)q, (uint32_t)tt, s.rk);
  };
  if (kPipe) {
    // masks of colour 0 (m0) and colour 1 (m1) of this thread's sites, each
    // drawn during the phase before the one that uses them
    uint32_t m04[kPipeSites], m08[kPipeSites], m14[kPipeSites], m18[kPipeSites];
    // PRE: sweeps [t_begin, t_pre) read their masks from the table
    const int t_pre = (PRE && pre_tab != nullptr) ? min(t_end, t_begin + pre_count) : t_begin;
    auto planes = [&](int tt) {
      return pre_tab + ((int64_t)(tt - t_begin) * s.words + word) * 2 * n;
    };
    if (t < t_end) {
      sweep_prefix(t);
      if (PRE && t < t_pre)
        pipe_prologue<true>(W, r0, nr, 0, bp, s.rk, T4n, T8n, m04, m08, planes(t), planes(t) + n);
      else
        pipe_prologue<false>(W, r0, nr, 0, bp, s.rk, T4n, T8n, m04, m08, nullptr, nullptr);
    }
    bool stop = false;
    // Phases ordered by data flow: a CTA sends its boundary rows' new cells to
    // the neighbours' halos (st.async) and, at a sweep's end, its warps' energy
    // sums to every CTA's accumulator (red.async), all completing on the
    // receiver's mbarrier; it waits on its own for its threads and the bytes
    // expected: one colour's cells of its two halo rows (W words), plus the
    // peers' sums at a sweep's end.  A neighbour completes a phase only after
    // every boundary cell it reads from this CTA has been updated, and so after
    // this CTA's reads of the halo next to it: no write can overtake a read,
    // and no CTA runs more than one phase ahead (two mbarriers).  A wait that
    // gives up sets the error flag (done = -1 for the host); later waits are
    // skipped, and one cluster barrier ends the kernel.
    const uint32_t up_halo = map_rank(
        (uint32_t)__cvta_generic_to_shared(spin + (size_t)(band_of(L, K, kup).nr + 1) * W),
        (uint32_t)kup);
    const uint32_t down_halo = map_rank((uint32_t)__cvta_generic_to_shared(spin), (uint32_t)kdown);
    const uint32_t up_bar0 = map_rank(bar_l, (uint32_t)kup);
    const uint32_t down_bar0 = map_rank(bar_l, (uint32_t)kdown);
    const uint32_t energy_bytes = 4u * 32u * (blockDim.x / 32u) * (uint32_t)(K - 1);
    int gph = 0;       // phases so far: mbarrier gph & 1
    uint32_t par = 0;  // each mbarrier's current phase parity
    auto df_wait = [&]() {
      const int i = gph & 1;
      uint32_t tries = 0;
      while (!bar_try_wait(bar_l + 8u * (uint32_t)i, (par >> i) & 1u)) {
        if (*(volatile int *)dferr) break;
        if (++tries >= kTorusWaitLimit) {
          atomicExch(dferr, 1);
          break;
        }
      }
      par ^= 1u << i;
      ++gph;
    };
    // one sweep; LOAD0: the masks phase 0 prepares (colour 1 of sweep t) come
    // from the table, LOAD1: those phase 1 prepares (colour 0 of sweep t + 1)
    auto sweep = [&](auto load0, auto load1) {
      constexpr bool LOAD0 = decltype(load0)::value, LOAD1 = decltype(load1)::value;
      const uint32_t T4 = T4n, T8 = T8n;
      const bool more = t + 1 < t_end;
      if (more) {
        T4n = trow[(size_t)(t + 1) * s.table_ts];
        T8n = trow[(size_t)(t + 1) * s.table_ts + 1];
      }
      cnt.clear();
      // colour 0 of sweep t; prepares colour 1 of sweep t
      uint32_t pb = 8u * (uint32_t)(gph & 1);
      pipe_phase<NP, LOAD0>(spin, best, cb, up_halo, down_halo, up_bar0 + pb, down_bar0 + pb, W,
                            r0, nr, 0, bp, s.rk, T4, T8, imp, cnt, m04, m08, m14, m18,
                            LOAD0 ? planes(t) : nullptr, LOAD0 ? planes(t) + n : nullptr);
      bar_arrive(bar_l + pb, threadIdx.x == 0, 4u * (uint32_t)W);
      if (more) sweep_prefix(t + 1);
      df_wait();
      // colour 1 of sweep t; prepares colour 0 of sweep t + 1 (unused after the last)
      pb = 8u * (uint32_t)(gph & 1);
      pipe_phase<NP, LOAD1>(spin, best, cb, up_halo, down_halo, up_bar0 + pb, down_bar0 + pb, W,
                            r0, nr, 1, bp, s.rk, T4n, T8n, imp, cnt, m14, m18, m04, m08,
                            LOAD1 ? planes(t + 1) : nullptr, LOAD1 ? planes(t + 1) + n : nullptr);
      // the sweep's energy change: every warp's lane sums into every CTA's
      // accumulator acc_m (three rotate: the one the next sweep adds into is
      // cleared once this one is read)
      {
        int32_t *cur = acc + 32 * acc_m;
        const int32_t tot = cnt.warp_lane_total();
        const uint32_t a = (uint32_t)__cvta_generic_to_shared(cur + lane);
        for (int q = 0; q < K; ++q)
          if (q != k)
            red_async_add_cl(map_rank(a, (uint32_t)q), tot, map_rank(bar_l + pb, (uint32_t)q));
        atomicAdd(cur + lane, tot);
        bar_arrive(bar_l + pb, threadIdx.x == 0, 4u * (uint32_t)W + energy_bytes);
        df_wait();
        const int32_t sum = cur[lane];
        acc_m = acc_m == 2 ? 0 : acc_m + 1;
        if (threadIdx.x < 32) acc[32 * acc_m + lane] = 0;
        e += 4 * (sum - 2 * n);
      }
      const bool better = e < e_best;
      if (better) e_best = e;
      imp = __ballot_sync(0xFFFFFFFFu, better) & valid;
      if (s.has_target) {
        const int32_t mn =
            __reduce_min_sync(0xFFFFFFFFu, ((valid >> lane) & 1u) ? e_best : INT_MAX);
        if (mn <= s.target) {
          hit = t;
          stop = true;
        }
      }
    };
    if (PRE) {
      // masks read for both phases, then the sweep whose successor draws them
      for (; !stop && t + 1 < t_pre; ++t) sweep(std::true_type{}, std::true_type{});
      if (!stop && t < t_pre) {
        sweep(std::true_type{}, std::false_type{});
        ++t;
      }
    }
    for (; !stop && t < t_end; ++t) sweep(std::false_type{}, std::false_type{});
  }
  // masks of this thread's first site of the next phase, drawn while the
  // group barrier before that phase completes (they do not depend on spins)
  uint32_t pre4 = 0u, pre8 = 0u;
  bool ready = false;
  if (!kPipe && kPrefetch && t < t_end) {
    sweep_prefix(t);
    ready = first_site_masks(W, r0, nr, 0, bp, s.rk, T4n, T8n, pre4, pre8);
  }
  for (; !kPipe && t < t_end; ++t) {
    const uint32_t T4 = T4n, T8 = T8n;
    const bool more = t + 1 < t_end;
    if (more) {
      T4n = trow[(size_t)(t + 1) * s.table_ts];
      T8n = trow[(size_t)(t + 1) * s.table_ts + 1];
    }
    if (!kPrefetch) sweep_prefix(t);
    cnt.clear();
    for (int c = 0; c < 2; ++c) {
      if (T8 != 0u)
        sweep_phase<NP, true>(spin, best, cb, up_peer, down_peer, W, r0, nr, c, bp, s.rk, T4, T8,
                              imp, cnt, pre4, pre8, ready);
      else
        sweep_phase<NP, false>(spin, best, cb, up_peer, down_peer, W, r0, nr, c, bp, s.rk, T4, T8,
                               imp, cnt, pre4, pre8, ready);
      if (c == 0) {
        group_arrive(K);
        if (kPrefetch) ready = first_site_masks(W, r0, nr, 1, bp, s.rk, T4, T8, pre4, pre8);
        group_wait(K);
      }
    }
    ready = false;
    e += 4 * (cluster_lane_sum<NP>(cnt, acc, acc_m, K, [&] {
                if (kPrefetch && more) {
                  sweep_prefix(t + 1);
                  ready = first_site_masks(W, r0, nr, 0, bp, s.rk, T4n, T8n, pre4, pre8);
                }
              }) -
              2 * n);
    const bool better = e < e_best;
    if (better) e_best = e;
    imp = __ballot_sync(0xFFFFFFFFu, better) & valid;
    if (s.has_target) {
      const int32_t mn =
          __reduce_min_sync(0xFFFFFFFFu, ((valid >> lane) & 1u) ? e_best : INT_MAX);
      if (mn <= s.target) {
        hit = t;
        ++t;
        break;
      }
    }
  }

  // every phase update of the cluster precedes the last group barrier
  for (int idx = threadIdx.x; idx < nr * W; idx += blockDim.x) {
    const uint32_t v = spin[W + idx];
    gspin[r0 * W + idx] = v;
    gbest[r0 * W + idx] = (best[idx] & ~imp) | (v & imp);
  }
  if (k == 0) {
    if (threadIdx.x < 32) {
      s.e_cur[word * 32 + lane] = e;
      s.e_best[word * 32 + lane] = e_best;
    }
    if (threadIdx.x == 0) {
      if (s.has_target && hit >= 0) s.hit[word] = hit;
      s.done[word] = t;
    }
  }
  if (kPipe) {
    cluster_barrier();  // no CTA leaves while another may still send to it
    if (threadIdx.x == 0 && *(volatile int *)dferr) atomicMin(&s.done[word], -1);
  }
}

// MAXT = 1024 caps registers at 64 per thread so that 1,024 threads fit one SM;
// MAXT = 384 (CTAs of at most 384 threads, six counter planes: the 80 x 100
// workload's shape) lets the compiler keep more of the eight Philox blocks in
// flight (144 registers against 116 in the 512-thread build: +1.2 %)
template <int NP, int MAXT, bool PIPE = false, bool PRE = false>
__global__ void __launch_bounds__(MAXT, 1) torus_kernel(TorusSolve s, TorusLaunch l) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int K = l.cluster;
  const int k = (int)(blockIdx.x % K);
  const int word = (int)(blockIdx.x / K);
  int t_end = l.t_end;
  if (l.stop_from_hits) {
    int m = INT_MAX;
    for (int w = 0; w < s.words; ++w)
      if (s.hit[w] >= 0 && s.hit[w] < m) m = s.hit[w];
    if (m != INT_MAX && m + 1 < t_end) t_end = m + 1;
  }
  torus_word<NP, (MAXT <= 512), PIPE, PRE>(s, word, k, K, l.t_begin, t_end, l.resume, smem,
                                           l.pre_tab, l.pre_count);
}

// One CTA per unit with a CTA-wide barrier (nothing to overlap): no mask
// prefetch, so that the kernel stays at 64 registers and two CTAs per SM.
template <int NP>
__global__ void __launch_bounds__(512, 2) torus_batch_kernel(const TorusBatchItem *items,
                                                          const int32_t *count_dev,
                                                          const int32_t *order, int32_t *next) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int item;
  const int count = *count_dev;
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(next, 1);
    __syncthreads();
    const int it = item;
    __syncthreads();
    if (it >= count) break;
    const TorusBatchItem u = items[order[it]];
    int t_end = u.t_end;
    if (u.stop_from_hits) {
      // the solve's stop sweep from the first pass (uniform across the CTA)
      int m = INT_MAX;
      for (int w = 0; w < u.solve.words; ++w)
        if (u.solve.hit[w] >= 0 && u.solve.hit[w] < m) m = u.solve.hit[w];
      if (m == INT_MAX) continue;  // no unit reached the target: the first pass stands
      if (m + 1 < t_end) t_end = m + 1;
    }
    torus_word<NP, false>(u.solve, u.word, 0, 1, u.t_begin, t_end, u.resume, smem);
    __syncthreads();
  }
}

// Acceptance masks of the sweeps a, a + 1, ... for every word and site of a
// torus solve, for the pipelined sweep kernel to read instead of drawing
// them: one CTA per (sweep, word); site i's masks at out[(t - a, word)]
// [plane][i], plane 0 against the threshold of an energy change of 4, plane 1
// of 8, as site_masks builds them.
__global__ void __launch_bounds__(256) torus_mask_kernel(TorusSolve s, int32_t a, uint32_t *out) {
  const int w = (int)(blockIdx.x % (unsigned)s.words);
  const int p = (int)(blockIdx.x / (unsigned)s.words);
  const int t = a + p;
  const int n = s.L * s.W;
  const uint32_t uword = (uint32_t)(w + s.rng_word0);
  BlockPrefix bp[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) bp[q] = block_prefix(8u * uword + (uint32_t)q, (uint32_t)t, s.rk);
  const uint32_t *row = s.table + (size_t)w * s.table_ws + (size_t)t * s.table_ts;
  const uint32_t T4 = row[0], T8 = row[1];
  uint32_t *o = out + ((int64_t)p * s.words + w) * 2 * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    uint32_t r4, r8;
    site_masks<true>((uint32_t)i, bp, s.rk, T4, T8, r4, r8);
    o[i] = r4;
    o[n + i] = r8;
  }
}

int np_for(int sites_per_thread_sweep, int sites_per_thread_band, int threads) {
  const int need = 4 * sites_per_thread_sweep > 2 * sites_per_thread_band
                       ? 4 * sites_per_thread_sweep
                       : 2 * sites_per_thread_band;
  if (need < (1 << 5) && threads <= 384) return 5;  // (five planes: the 384-thread build only)
  if (need < (1 << 6)) return 6;
  if (need < (1 << 8)) return 8;
  if (need < (1 << 10)) return 10;
  return -1;
}

template <typename Kern>
cudaError_t prepare_clustered(Kern kernel, size_t smem, int cluster) {
  cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err == cudaSuccess && cluster > 8)
    err = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return err;
}

template <typename Kern>
int max_active_clusters(Kern kernel, int grid, int threads, size_t smem, int cluster) {
  if (prepare_clustered(kernel, smem, cluster) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename Kern>
cudaError_t launch_clustered(Kern kernel, int grid, int threads, size_t smem, int cluster,
                             cudaStream_t stream, const TorusSolve &s, const TorusLaunch &l) {
  cudaError_t err = prepare_clustered(kernel, smem, cluster);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, s, l);
}

}  // namespace

size_t torus_smem_bytes(int32_t L, int32_t W, int32_t cluster) {
  int nr_max = 0;
  for (int k = 0; k < cluster; ++k) {
    const int nr = band_of(L, cluster, k).nr;
    if (nr > nr_max) nr_max = nr;
  }
  return layout_of(nr_max, W, cluster).total;
}

int32_t torus_sites_per_thread(int32_t L, int32_t W, int32_t cluster, int32_t threads) {
  const int nr = (L + cluster - 1) / cluster;
  const int per_phase = (nr * (W / 2) + threads - 1) / threads;
  return 2 * per_phase;
}

int torus_max_active_clusters(int32_t L, int32_t W, int32_t words, int32_t cluster,
                              int32_t threads) {
  const size_t smem = torus_smem_bytes(L, W, cluster);
  const int nr = (L + cluster - 1) / cluster;
  const int np = np_for(torus_sites_per_thread(L, W, cluster, threads),
                        (nr * W + threads - 1) / threads, threads);
  const int grid = words * cluster;
  const bool wide = threads > 512;
  switch (np) {
    case 5:
      return max_active_clusters(torus_kernel<5, 384>, grid, threads, smem, cluster);
    case 6:
      if (threads <= 384)
        return max_active_clusters(torus_kernel<6, 384>, grid, threads, smem, cluster);
      return wide ? max_active_clusters(torus_kernel<6, 1024>, grid, threads, smem, cluster)
                  : max_active_clusters(torus_kernel<6, 512>, grid, threads, smem, cluster);
    case 8:
      return wide ? max_active_clusters(torus_kernel<8, 1024>, grid, threads, smem, cluster)
                  : max_active_clusters(torus_kernel<8, 512>, grid, threads, smem, cluster);
    case 10:
      return wide ? max_active_clusters(torus_kernel<10, 1024>, grid, threads, smem, cluster)
                  : max_active_clusters(torus_kernel<10, 512>, grid, threads, smem, cluster);
    default: return 0;
  }
}

bool torus_pipelined(int32_t L, int32_t W, int32_t cluster, int32_t threads) {
  const int nr = (L + cluster - 1) / cluster;
  const int spt = torus_sites_per_thread(L, W, cluster, threads);
  const int np = np_for(spt, (nr * W + threads - 1) / threads, threads);
  return threads <= 384 && spt / 2 <= kPipeSites && (np == 5 || np == 6);
}

cudaError_t torus_mask_launch(const TorusSolve &s, int32_t a, int32_t count, uint32_t *out_dev,
                              cudaStream_t stream) {
  const int64_t grid = (int64_t)count * s.words;
  if (count < 1 || grid > INT32_MAX) return cudaErrorInvalidValue;
  torus_mask_kernel<<<(unsigned)grid, 256, 0, stream>>>(s, a, out_dev);
  return cudaGetLastError();
}

cudaError_t torus_launch(const TorusSolve &s, const TorusLaunch &l, cudaStream_t stream) {
  const int K = l.cluster;
  const size_t smem = torus_smem_bytes(s.L, s.W, K);
  const int nr = (s.L + K - 1) / K;
  const int spt = torus_sites_per_thread(s.L, s.W, K, l.threads);
  const int band_spt = (nr * s.W + l.threads - 1) / l.threads;
  const int np = np_for(spt, band_spt, l.threads);
  const int grid = s.words * K;
  if (l.threads > 1024) return cudaErrorInvalidValue;
  const bool wide = l.threads > 512;
  // software-pipelined phases when every thread has at most kPipeSites sites per phase
  const bool pipe = l.threads <= 384 && spt / 2 <= kPipeSites;
  const bool pre = pipe && l.pre_tab != nullptr && l.pre_count > 0;
  switch (np) {
    case 5:
      if (pre)
        return launch_clustered(torus_kernel<5, 384, true, true>, grid, l.threads, smem, K,
                                stream, s, l);
      return pipe ? launch_clustered(torus_kernel<5, 384, true>, grid, l.threads, smem, K,
                                     stream, s, l)
                  : launch_clustered(torus_kernel<5, 384>, grid, l.threads, smem, K, stream, s, l);
    case 6:
      if (l.threads <= 384 && pre)
        return launch_clustered(torus_kernel<6, 384, true, true>, grid, l.threads, smem, K,
                                stream, s, l);
      if (l.threads <= 384 && pipe)
        return launch_clustered(torus_kernel<6, 384, true>, grid, l.threads, smem, K, stream, s,
                                l);
      if (l.threads <= 384)
        return launch_clustered(torus_kernel<6, 384>, grid, l.threads, smem, K, stream, s, l);
      return wide ? launch_clustered(torus_kernel<6, 1024>, grid, l.threads, smem, K, stream, s, l)
                  : launch_clustered(torus_kernel<6, 512>, grid, l.threads, smem, K, stream, s, l);
    case 8:
      return wide ? launch_clustered(torus_kernel<8, 1024>, grid, l.threads, smem, K, stream, s, l)
                  : launch_clustered(torus_kernel<8, 512>, grid, l.threads, smem, K, stream, s, l);
    case 10:
      return wide
                 ? launch_clustered(torus_kernel<10, 1024>, grid, l.threads, smem, K, stream, s, l)
                 : launch_clustered(torus_kernel<10, 512>, grid, l.threads, smem, K, stream, s, l);
    default: return cudaErrorInvalidValue;
  }
}

size_t torus_batch_max_smem(int32_t L, int32_t W) { return layout_of(L, W, 1).total; }

cudaError_t torus_batch_launch(const TorusBatchItem *items_dev, const int32_t *count_dev,
                               const int32_t *order_dev, int32_t *next_dev, int32_t ctas,
                               int32_t threads, size_t smem, cudaStream_t stream) {
  // ten counter planes hold 4 x sites-per-thread-per-sweep for every torus the
  // batched forms accept (at most 127 sites per thread and colour phase)
  cudaError_t err = cudaFuncSetAttribute(torus_batch_kernel<10>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  torus_batch_kernel<10><<<ctas, threads, smem, stream>>>(items_dev, count_dev, order_dev,
                                                           next_dev);
  return cudaGetLastError();
}

}  // namespace isg
