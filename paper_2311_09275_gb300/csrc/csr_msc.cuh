// csr_msc.cuh -- colour-class Metropolis sweeps on +-1-weighted sparse graphs
// with multi-spin coding: 32 replicas per uint32 word, one bit per replica.
//
// Per vertex v of degree d and replica word, the kernel forms one
// "unsatisfied bond" word per neighbour (bond (v,j) is unsatisfied when
// w_vj s_v s_j = +1), counts them bit-sliced (U = 0..d per replica), and
// flips a replica when its half energy change k = d - 2U is <= 0, or when its
// Philox uniform is below the sweep's threshold for k.  The uphill replicas
// of a vertex sit at a few levels U = 0..(d-1)/2; each occupied level costs
// one threshold mask over the 32 uniforms.
//
// Layout: a cluster of K CTAs owns one replica word; every CTA keeps the
// whole word in shared memory, updates 1/K of each colour class (contiguous
// after the colour-major relabel) and writes each new word into all K copies
// through distributed shared memory; one cluster barrier separates classes.
// A CTA stages the adjacency of the slices it owns in shared memory when it
// fits, and then keeps their best state there too.  Per-replica energy
// changes are accumulated in bit-sliced counters (sum over accepted flips of
// d, and of U: the change is 2 (d - 2U)) and reduced once per sweep.  The
// uniforms do not depend on the spins: a thread draws those of its first
// vertex of the next class between its arrival at the class barrier and the
// wait for it, so that the Philox work overlaps the barrier.
//
// Local fields (instances whose weights are all +1): the term h s of vertex
// v counts as |h| extra bonds to a fixed +1 spin with coupling sign(h), so d
// becomes d + |h| and U gains |h| in the replicas where h s = +|h|; the
// kernel is otherwise unchanged (build FIELD).
#pragma once

#include <climits>

#include "isg_device.cuh"
#include "isg_kernels.h"

namespace isg {
namespace {

constexpr int kPlanesU = 6;  // per-lane bond counts up to 63 (degree <= 63)

__host__ __device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

struct GmSmem {
  size_t spin, lrow, lorig, lcol, lbest, lfield, lmoff, lmask, ocls, trow, part, lane_acc, bars,
      total;
};

// own_n, own_nnz, own_lv: the largest owned vertex, adjacency and threshold-
// level count of any rank (0: adjacency not staged, and no mask table).
__host__ __device__ __forceinline__ GmSmem gm_layout(int n, int K, int n_colours, int own_n,
                                                     int own_nnz, int own_lv, int kmax1,
                                                     bool fields) {
  GmSmem m;
  m.spin = 0;
  m.lrow = align16(sizeof(uint32_t) * (size_t)n);
  m.lorig = align16(m.lrow + (own_n ? sizeof(int32_t) * ((size_t)own_n + 1) : 0));
  m.lcol = align16(m.lorig + sizeof(int32_t) * (size_t)own_n);
  m.lbest = align16(m.lcol + sizeof(int32_t) * (size_t)own_nnz);
  m.lfield = align16(m.lbest + sizeof(uint32_t) * (size_t)own_n);
  m.lmoff = align16(m.lfield + (fields ? sizeof(int32_t) * (size_t)own_n : 0));
  m.lmask = align16(m.lmoff + (own_n ? sizeof(int32_t) * ((size_t)own_n + 1) : 0));
  m.ocls = align16(m.lmask + 2 * sizeof(uint32_t) * (size_t)own_lv);
  // class slice table: slice bounds, first slot, mask work of each class's window,
  // and the bytes the peers send in each class
  m.trow = align16(m.ocls + sizeof(int32_t) * (5 * (size_t)n_colours + 1));
  m.part = align16(m.trow + 2 * sizeof(uint32_t) * (size_t)kmax1);
  m.lane_acc = m.part + 2 * sizeof(int32_t) * 32 * (size_t)K;
  m.bars = align16(m.lane_acc + sizeof(int32_t) * 32);  // two mbarriers and an error flag
  m.total = align16(m.bars + 32);
  return m;
}

__device__ __forceinline__ void sync_group(int K) {
  if (K == 1)
    __syncthreads();
  else
    cluster_barrier();
}

__device__ __forceinline__ void own_range(int a, int b, int k, int K, int &lo, int &hi) {
  const int len = b - a;
  lo = a + (int)((int64_t)len * k / K);
  hi = a + (int)((int64_t)len * (k + 1) / K);
}

// Per-lane int32 contributions summed over the CTA and published to every CTA
// of the cluster as part[k][lane]; ends with the group barrier.
__device__ __forceinline__ void publish_lanes(int32_t v, int32_t *lane_acc, int32_t *part, int k,
                                              int K) {
  atomicAdd(&lane_acc[lane_id()], v);
  __syncthreads();
  if (threadIdx.x < 32) {
    const int32_t x = lane_acc[threadIdx.x];
    lane_acc[threadIdx.x] = 0;
    if (K == 1) {
      part[threadIdx.x] = x;
    } else {
      for (int r = 0; r < K; ++r) peer_smem(part, (uint32_t)r)[k * 32 + threadIdx.x] = x;
    }
  }
  sync_group(K);
}

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

// Lanes whose bit-sliced count equals v.
__device__ __forceinline__ uint32_t count_equals(const uint32_t (&u)[kPlanesU], int v) {
  uint32_t eq = 0xFFFFFFFFu;
#pragma unroll
  for (int p = 0; p < kPlanesU; ++p) eq &= ((v >> p) & 1) ? u[p] : ~u[p];
  return eq;
}

struct GmAdj {
  const int32_t *row, *col, *orig;
};

// The 32 uniforms of one vertex word in one sweep: Philox4x32-10 blocks
// 8 word + q (q = 0..7) of the vertex's original id, from the sweep's block
// prefixes.
__device__ __forceinline__ void vertex_uniforms(uint32_t orig, const BlockPrefix (&bp)[8],
                                                const RoundKeys &rk, uint4 (&uu)[8]) {
  const SitePrefix sp = site_prefix(orig, rk);
#pragma unroll
  for (int q = 0; q < 8; ++q) uu[q] = philox10_factored(sp, bp[q], rk);
}

// Smallest of a vertex's 32 uniforms.  A level whose threshold does not
// exceed it accepts none of its replicas, so its 32 compares can be skipped
// without changing the result (late in an annealing schedule, when the
// thresholds are small, this is the usual case).
__device__ __forceinline__ uint32_t uniform_min(const uint4 (&uu)[8]) {
  uint32_t m[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) m[q] = min(min(uu[q].x, uu[q].y), min(uu[q].z, uu[q].w));
  return min(min(min(m[0], m[1]), min(m[2], m[3])), min(min(m[4], m[5]), min(m[6], m[7])));
}

// Lanes whose uniform is below T.
__device__ __forceinline__ uint32_t uniforms_below(const uint4 (&uu)[8], uint32_t T) {
  uint32_t m0 = 0u, m1 = 0u;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    uint32_t &m = (q & 1) ? m1 : m0;
    if (uu[q].x < T) m |= 1u << (4 * q);
    if (uu[q].y < T) m |= 2u << (4 * q);
    if (uu[q].z < T) m |= 4u << (4 * q);
    if (uu[q].w < T) m |= 8u << (4 * q);
  }
  return m0 | m1;
}

// Lanes where the field term h s of a vertex with word s0 is +|h| (bit 1 =
// spin +1), counted as unsatisfied extra bonds.
__device__ __forceinline__ uint32_t field_unsat(uint32_t s0, int32_t hv) {
  return hv > 0 ? s0 : ~s0;
}

// 4-byte asynchronous copy from global to shared memory (both 4-byte
// aligned), completed by cp_async_wait_all in the issuing thread.
__device__ __forceinline__ void cp_async4(uint32_t *dst_smem, const uint32_t *src_gmem) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src_gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Cluster data flow between the CTAs that share a word: a CTA sends each new
// word to its peers with st.async, which completes on the receiver's
// mbarrier, so a receiver knows that a class is complete in its copy once the
// expected bytes have arrived and its own threads have arrived.
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n}\n" ::"r"(
          bar)
      : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 st, [%0], "
      "%1;\n}\n" ::"r"(bar),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], "
      "%2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// v into CTA `rank`'s copy of the shared word at local address a, completing
// 4 bytes on that CTA's mbarrier at local address bar.
__device__ __forceinline__ void st_async_u32(uint32_t a, uint32_t rank, uint32_t v,
                                             uint32_t bar) {
  uint32_t ra, rb;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(rb) : "r"(bar), "r"(rank));
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.u32 [%0], %1, [%2];\n" ::"r"(
                   ra),
               "r"(v), "r"(rb)
               : "memory");
}

// try_wait attempts before a wait counts as failed (far beyond any phase)
constexpr uint32_t kDataflowWaitLimit = 1u << 22;

// Acceptance sources of update_vertex.
enum GmAccept { kAcceptPre = 0, kAcceptLazy = 1, kAcceptMasks = 2 };

// One vertex of one replica word (adjacency entries [p0, p1); and, FIELD, its
// local field hv).  Its acceptance masks come from its 32 uniforms, pre
// (kAcceptPre: drawn by the caller) or filled by draw(uu) only when some
// replica is uphill (kAcceptLazy), or are read per level from mk (kAcceptMasks:
// mk[lv] = lanes whose uniform is below the threshold of k = d - 2 lv, built
// ahead of the phase).  Returns the new word; accumulates the accepted flips'
// d and U into the energy counters.
template <int NP, bool FIELD, int ACCEPT, typename Draw>
__device__ __forceinline__ uint32_t update_vertex(const uint32_t *spin, int v, int p0, int p1,
                                                  const GmAdj &a, const uint32_t *row,
                                                  const uint4 (&pre)[8], Draw draw,
                                                  const uint32_t *mk, int32_t hv,
                                                  SlicedCounter<NP> &cd, SlicedCounter<NP> &cu) {
  const uint32_t s0 = spin[v];
  int d = p1 - p0;
  uint32_t u[kPlanesU];
#pragma unroll
  for (int p = 0; p < kPlanesU; ++p) u[p] = 0u;
  for (int p = p0; p < p1; ++p) {
    const int e = a.col[p];
    const uint32_t neg = (uint32_t)(e >> 31);            // all ones for weight -1
    uint32_t c = ~(s0 ^ spin[e & 0x7FFFFFFF] ^ neg);     // unsatisfied bond
#pragma unroll
    for (int q = 0; q < kPlanesU; ++q) {
      const uint32_t cc = u[q] & c;
      u[q] ^= c;
      c = cc;
    }
  }
  if (FIELD && hv != 0) {
    // |h| extra bonds, unsatisfied in the lanes of field_unsat
    const uint32_t f = field_unsat(s0, hv);
    const int ha = hv > 0 ? hv : -hv;
#pragma unroll
    for (int b = 0; b < kPlanesU; ++b) {
      if ((ha >> b) & 1) {
        uint32_t c = f;
#pragma unroll
        for (int q = b; q < kPlanesU; ++q) {
          const uint32_t cc = u[q] & c;
          u[q] ^= c;
          c = cc;
        }
      }
    }
    d += ha;
  }
  // uphill lanes: U <= (d - 1) / 2, i.e. k = d - 2U > 0; those at level U
  // flip when their uniform is below the threshold of k = d - 2U
  const int levels = (d + 1) / 2;
  uint32_t acc;
  if (ACCEPT == kAcceptMasks) {
    uint32_t up = 0u, yes = 0u;
    for (int lv = 0; lv < levels; ++lv) {
      const uint32_t eq = count_equals(u, lv);
      up |= eq;
      yes |= eq & mk[lv];
    }
    acc = ~up | yes;
  } else if (ACCEPT == kAcceptLazy) {
    uint32_t up = 0u;
    for (int lv = 0; lv < levels; ++lv) up |= count_equals(u, lv);
    acc = ~up;
    if (up != 0u) {
      uint4 uu[8];
      draw(uu);
      const uint32_t umin = uniform_min(uu);
      for (int lv = 0; lv < levels; ++lv) {
        const uint32_t T = row[d - 2 * lv];
        if (T <= umin) continue;
        const uint32_t eq = count_equals(u, lv);
        if (eq != 0u) acc |= eq & uniforms_below(uu, T);
      }
    }
  } else {
    // the uphill lanes are rejected unless their level's threshold admits them
    uint32_t up = 0u, yes = 0u;
    const uint32_t umin = uniform_min(pre);
    for (int lv = 0; lv < levels; ++lv) {
      const uint32_t eq = count_equals(u, lv);
      up |= eq;
      const uint32_t T = row[d - 2 * lv];
      if (eq != 0u && T > umin) yes |= eq & uniforms_below(pre, T);
    }
    acc = ~up | yes;
  }
  // energy change of the accepted lanes: 2 (d - 2U); d <= 63 (6 bits)
  uint32_t da[kPlanesU];
#pragma unroll
  for (int b = 0; b < kPlanesU; ++b) da[b] = ((d >> b) & 1) ? acc : 0u;
  cd.add_sliced(da);
  uint32_t ua[kPlanesU];
#pragma unroll
  for (int p = 0; p < kPlanesU; ++p) ua[p] = u[p] & acc;
  cu.add_sliced(ua);
  return s0 ^ acc;
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


// STAGED (adjacency of the owned slices in shared memory): the acceptance
// masks of every owned vertex for sweep t + 1 are built during sweep t, an
// even share in each class's barrier window, into a table of two sweeps; the
// update then reads masks instead of drawing uniforms.  PRE (staged, masks
// precomputed in device memory by gm_mask_kernel, at L.gmask): each thread
// instead copies a few of the next sweep's mask words into the table
// asynchronously, awaited before the sweep's last barrier.  Otherwise, PREFETCH: draw the next
// phase's first uniforms during the group barrier (off in the unit kernel,
// whose CTA-wide barrier leaves nothing to overlap).
template <int NP, bool STAGED, bool FIELD, bool PREFETCH = true, bool PRE = false>
__device__ void gm_word(const GraphMscSolve &s, const GraphMscLaunch &L, int word, int k, int K,
                        int t_begin, int t_end, int resume, uint8_t *smem) {
  constexpr bool PF = PREFETCH && !STAGED;
  constexpr bool MG = STAGED && PRE;
  const int n = s.n;
  const int nc = s.n_colours;
  const int B = (int)blockDim.x;
  const GmSmem lay = gm_layout(n, K, nc, STAGED ? L.own_n : 0, STAGED ? L.own_nnz : 0,
                               STAGED ? L.own_lv : 0, s.kmax1, FIELD);
  const bool has_field = FIELD && s.field != nullptr;
  uint32_t *spin = reinterpret_cast<uint32_t *>(smem + lay.spin);
  // per class: this rank's slice [clo, chi) and the slot of its first vertex
  // (the vertex itself when the adjacency is not staged)
  int32_t *clo = reinterpret_cast<int32_t *>(smem + lay.ocls);
  int32_t *chi = clo + nc;
  int32_t *cob = chi + nc;
  int32_t *qlo = cob + nc;  // staged: mask work [qlo[c], qlo[c + 1]) in class c's window
  int32_t *expb = qlo + nc + 1;  // bytes the peers send into this copy in class c
  // clusters: this CTA's two mbarriers (alternating class phases) and error flag
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + lay.bars);
  int *dferr = reinterpret_cast<int *>(smem + lay.bars + 16);
  const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(bars);
  uint32_t *trow = reinterpret_cast<uint32_t *>(smem + lay.trow);
  int32_t *part = reinterpret_cast<int32_t *>(smem + lay.part);
  int32_t *lane_acc = reinterpret_cast<int32_t *>(smem + lay.lane_acc);
  const uint32_t *wtab = s.table + (size_t)word * s.table_ws;  // this word's threshold rows
  const PhiloxKey key{s.key0, s.key1};
  const uint32_t uword = (uint32_t)(word + s.rng_word0);  // Philox counters only
  const int rem = s.replicas - 32 * word;
  const uint32_t valid = rem >= 32 ? 0xFFFFFFFFu : ((1u << rem) - 1u);
  uint32_t *gspin = s.spins + (size_t)word * n;
  uint32_t *gbest = s.best + (size_t)word * n;
  const int lane = (int)lane_id();

  if (resume && s.has_target && s.hit[word] >= 0) return;
  if (resume && t_begin >= t_end) return;
  if (!resume && s.has_target && k == 0 && threadIdx.x == 0) s.hit[word] = -1;

  for (int v = threadIdx.x; v < n; v += blockDim.x)
    spin[v] = resume ? gspin[v] : initial_word((uint32_t)s.orig[v], uword, key);

  if (threadIdx.x == 0) {
    int ov = 0;
    for (int c = 0; c < nc; ++c) {
      int lo, hi;
      own_range(s.class_start[c], s.class_start[c + 1], k, K, lo, hi);
      clo[c] = lo;
      chi[c] = hi;
      cob[c] = STAGED ? ov : lo;
      ov += hi - lo;
      expb[c] = 4 * ((s.class_start[c + 1] - s.class_start[c]) - (hi - lo));
    }
    if (MG && K > 1) {
      mbar_init(bar0, (uint32_t)B);
      mbar_init(bar0 + 8, (uint32_t)B);
      *dferr = 0;
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (STAGED) {
      // the owned slots' mask work, an even share per class window (measured
      // faster than shares weighted by the threads idle in the window's
      // classes: those put two items in a row on some threads)
      for (int c = 0; c < nc; ++c) qlo[c] = (int)((int64_t)ov * c / nc);
      qlo[nc] = ov;
      // a thread builds its share of the last window after arriving at the
      // sweep's last barrier, so the next barrier it reaches lies after the
      // next sweep's first class: that window takes no slot of the first class
      if (nc > 1) qlo[nc - 1] = max(qlo[nc - 1], chi[0] - clo[0]);
    }
  }
  __syncthreads();
  GmAdj adj;
  // staged: best state (and fields) of the owned vertices by slot (else in
  // global memory)
  uint32_t *lbest = reinterpret_cast<uint32_t *>(smem + lay.lbest);
  int32_t *lfield = reinterpret_cast<int32_t *>(smem + lay.lfield);
  // staged: each owned slot's first entry in the mask table (two sweeps of
  // L.own_lv words), one per threshold level (d + |h| + 1) / 2
  int32_t *lmoff = reinterpret_cast<int32_t *>(smem + lay.lmoff);
  uint32_t *lmask = reinterpret_cast<uint32_t *>(smem + lay.lmask);
  if (STAGED) {
    int32_t *lrow = reinterpret_cast<int32_t *>(smem + lay.lrow);
    int32_t *lorig = reinterpret_cast<int32_t *>(smem + lay.lorig);
    int32_t *lcol = reinterpret_cast<int32_t *>(smem + lay.lcol);
    int ebase = 0;
    for (int c = 0; c < nc; ++c) {
      const int lo = clo[c], hi = chi[c], ob = cob[c];
      const int e0 = s.rowptr[lo], e1 = s.rowptr[hi];
      for (int i = threadIdx.x; i <= hi - lo; i += blockDim.x) {
        lrow[ob + i] = s.rowptr[lo + i] - e0 + ebase;
        if (i < hi - lo) {
          const int v = lo + i;
          lorig[ob + i] = s.orig[v];
          if (resume) lbest[ob + i] = gbest[v];
          if (FIELD) lfield[ob + i] = has_field ? s.field[v] : 0;
        }
      }
      for (int p = threadIdx.x; p < e1 - e0; p += blockDim.x) lcol[ebase + p] = s.col[e0 + p];
      ebase += e1 - e0;
    }
    adj = {lrow, lcol, lorig};
    __syncthreads();
    if (threadIdx.x < 32) {
      // exclusive prefix of the slots' level counts: a contiguous chunk per lane
      const int cnt = qlo[nc];
      const int chunk = (cnt + 31) / 32;
      const int a0 = min(lane * chunk, cnt), a1 = min(a0 + chunk, cnt);
      auto levels_of = [&](int i) {
        int d = lrow[i + 1] - lrow[i];
        if (FIELD) d += abs(lfield[i]);
        return (d + 1) / 2;
      };
      int sum = 0;
      for (int i = a0; i < a1; ++i) sum += levels_of(i);
      int incl = sum;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off) incl += y;
      }
      int run = incl - sum;
      for (int i = a0; i < a1; ++i) {
        lmoff[i] = run;
        run += levels_of(i);
      }
      if (lane == 31) lmoff[cnt] = incl;
    }
  } else {
    adj = {s.rowptr, s.col, s.orig};
  }
  if (threadIdx.x < 32) lane_acc[threadIdx.x] = 0;
  // threshold rows: two buffers, the next sweep's row prefetched a sweep ahead
  // (staged: the masks are built a sweep ahead, and the rows two sweeps ahead)
  for (int tt = t_begin; tt < min(t_end, t_begin + (STAGED ? 2 : 1)); ++tt)
    for (int x = threadIdx.x; x < s.kmax1; x += blockDim.x)
      trow[(tt & 1) * s.kmax1 + x] = wtab[(size_t)tt * s.table_ts + x];
  // peers write into this CTA's copy of the word only after every CTA has loaded it
  sync_group(K);

  int32_t e = 0, e_best = 0;  // per lane = replica bit, kept identically by every warp
  if (!resume) {
    // E = sum over bonds of (+1 unsatisfied, -1 satisfied), each bond once
    SlicedCounter<NP> cu;
    cu.clear();
    int32_t bonds = 0;
    for (int c = 0; c < nc; ++c) {
      const int lo = clo[c], hi = chi[c];
      for (int v = lo + threadIdx.x; v < hi; v += blockDim.x) {
        const uint32_t s0 = spin[v];
        for (int p = s.rowptr[v]; p < s.rowptr[v + 1]; ++p) {
          const int ee = s.col[p];
          const int j = ee & 0x7FFFFFFF;
          if (j <= v) continue;
          cu.add_at(0, ~(s0 ^ spin[j] ^ (uint32_t)(ee >> 31)));
          ++bonds;
        }
        if (has_field) {
          // h s = +|h| or -|h|: |h| bonds, unsatisfied in the lanes of field_unsat
          const int32_t hv = s.field[v];
          const int ha = hv > 0 ? hv : -hv;
          const uint32_t f = field_unsat(s0, hv);
#pragma unroll
          for (int b = 0; b < kPlanesU; ++b)
            if ((ha >> b) & 1) cu.add_at(b, f);
          bonds += ha;
        }
        if (STAGED) lbest[cob[c] + (v - lo)] = s0;
        else gbest[v] = s0;
      }
    }
    const int32_t tot = 2 * cu.warp_lane_total() - __reduce_add_sync(0xFFFFFFFFu, bonds);
    publish_lanes(tot, lane_acc, part, k, K);
    for (int r = 0; r < K; ++r) e += part[r * 32 + lane];
    e_best = e;
  } else {
    e = s.e_cur[word * 32 + lane];
    e_best = s.e_best[word * 32 + lane];
  }

  // Random numbers do not depend on the spins: the uniforms of a thread's
  // first vertex of the next class (or of the next sweep's first class) are
  // drawn between the arrival at the group barrier and the wait for it.
  BlockPrefix bp[8];
  uint4 uu[8];
  bool ready = false;  // uu holds the uniforms of this thread's next vertex
  auto sweep_prefix = [&](int tt) {
#pragma unroll
    for (int q = 0; q < 8; ++q) bp[q] = block_prefix(8u * uword + (uint32_t)q, (uint32_t)tt, s.rk);
  };
  auto draw_first = [&](int c) {
    if (!PF) return;
    ready = clo[c] + (int)threadIdx.x < chi[c];
    if (ready) vertex_uniforms((uint32_t)adj.orig[cob[c] + threadIdx.x], bp, s.rk, uu);
  };
  if (PF && t_begin < t_end) {
    sweep_prefix(t_begin);
    draw_first(0);
  }
  // staged: the masks of slot j for sweep tt (block prefixes bp of sweep tt,
  // thresholds mrow), and the share of them built in class c's window
  auto masks_of = [&](int j, const uint32_t *mrow, uint32_t *mout) {
    int d = adj.row[j + 1] - adj.row[j];
    if (FIELD) d += abs(lfield[j]);
    const int levels = (d + 1) / 2;
    if (levels == 0) return;
    uint4 w[8];
    vertex_uniforms((uint32_t)adj.orig[j], bp, s.rk, w);
    const uint32_t umin = uniform_min(w);
    uint32_t *o = mout + lmoff[j];
    for (int lv = 0; lv < levels; ++lv) {
      const uint32_t T = mrow[d - 2 * lv];
      o[lv] = T > umin ? uniforms_below(w, T) : 0u;
    }
  };
  auto mask_window = [&](int c, int tt) {
    // items go to threads in descending order: first those idle in this
    // class and the next, last those with a vertex in both
    const uint32_t *mrow = trow + (tt & 1) * s.kmax1;
    uint32_t *mout = lmask + (size_t)(tt & 1) * L.own_lv;
    for (int j = qlo[c] + B - 1 - (int)threadIdx.x; j < qlo[c + 1]; j += B) masks_of(j, mrow, mout);
  };
  // precomputed masks: word q of the owned table (class-major over the owned
  // slices, like the slots) sits at src(q) in a sweep's table of all vertices
  const int own_words = STAGED ? lmoff[qlo[nc]] : 0;
  auto src_of = [&](int q) {
    int c = 0;
    while (c + 1 < nc && q >= lmoff[cob[c + 1]]) ++c;
    return L.gloff[clo[c]] + (q - lmoff[cob[c]]);
  };
  auto gmask_of = [&](int tt) {
    return L.gmask + ((int64_t)(tt - L.gmask_t0) * s.words + word) * L.gmask_gl;
  };
  if (STAGED && t_begin < t_end) {
    uint32_t *m0 = lmask + (size_t)(t_begin & 1) * L.own_lv;
    if (MG) {
      const uint32_t *g = gmask_of(t_begin);
      for (int q = threadIdx.x; q < own_words; q += B) m0[q] = g[src_of(q)];
    } else {
      sweep_prefix(t_begin);
      for (int j = threadIdx.x; j < qlo[nc]; j += B) masks_of(j, trow + (t_begin & 1) * s.kmax1, m0);
    }
    __syncthreads();
  }

  int t = t_begin;
  int hit = -1;
  uint32_t imp = 0u;  // replicas whose best state is the state at the start of sweep t
  const int x0 = (int)threadIdx.x, x1 = (int)(threadIdx.x + blockDim.x);
  // clusters with precomputed masks: class phases ordered by data flow
  // (st.async into the peers' copies, completing on their mbarriers) instead
  // of cluster barriers (measured faster there; with the masks built in the
  // kernel, whose window work runs while other warps wait, it was not).  A peer
  // starts class c + 1 only once this CTA's whole class c has arrived, which
  // this CTA sends only after all its reads of class c, so no peer runs more
  // than one phase ahead and two alternating mbarriers suffice.  A wait that
  // gives up sets the error flag (read by the host as done = -1); later waits
  // are skipped, so the kernel still ends.
  const bool DF = MG && K > 1;
  int gph = 0;       // class phases so far: mbarrier gph & 1
  uint32_t par = 0;  // each mbarrier's current phase parity
  auto df_arrive = [&](int bytes) {
    const uint32_t bar = bar0 + 8u * (uint32_t)(gph & 1);
    if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, (uint32_t)bytes);
    else mbar_arrive(bar);
  };
  auto df_wait = [&]() {
    const int i = gph & 1;
    const uint32_t bar = bar0 + 8u * (uint32_t)i;
    uint32_t tries = 0;
    while (!mbar_try_wait(bar, (par >> i) & 1u)) {
      if (*(volatile int *)dferr) break;
      if (++tries >= kDataflowWaitLimit) {
        atomicExch(dferr, 1);
        break;
      }
    }
    par ^= 1u << i;
    ++gph;
  };
  for (; t < t_end; ++t) {
    const uint32_t *row = trow + (t & 1) * s.kmax1;
    const bool more = t + 1 < t_end;
    // thresholds of sweep t + 1 (staged: t + 2) into registers now, into the
    // free row buffer at the end of the sweep (kmax1 <= 64 <= 2 x threads)
    constexpr int ahead = STAGED ? 2 : 1;
    const bool more_a = t + ahead < t_end;
    const uint32_t *gnext = wtab + (size_t)(t + ahead) * s.table_ts;
    const uint32_t p0 = (more_a && x0 < s.kmax1) ? gnext[x0] : 0u;
    const uint32_t p1 = (more_a && x1 < s.kmax1) ? gnext[x1] : 0u;
    if (!PREFETCH && !STAGED) sweep_prefix(t);
    if (STAGED && more && !MG) sweep_prefix(t + 1);  // for the masks of sweep t + 1
    if (MG && more) {
      // precomputed masks of sweep t + 1: asynchronous copies into the table
      // buffer this sweep does not read, awaited before the sweep's last barrier
      const uint32_t *g = gmask_of(t + 1);
      uint32_t *mn = lmask + (size_t)((t + 1) & 1) * L.own_lv;
      for (int q = threadIdx.x; q < own_words; q += B) cp_async4(mn + q, g + src_of(q));
    }
    const uint32_t *mcur = lmask + (size_t)(t & 1) * (STAGED ? L.own_lv : 0);
    SlicedCounter<NP> cd, cu;
    cd.clear();
    cu.clear();
    for (int c = 0; c < nc; ++c) {
      const int lo = clo[c], hi = chi[c], ob = cob[c];
      // adjacency in global memory: the next vertex's row bounds and id are
      // loaded one iteration ahead, off the current vertex's dependent chain
      int n0 = 0, n1 = 0, norig = 0;
      if (!STAGED && lo + (int)threadIdx.x < hi) {
        const int vn = lo + (int)threadIdx.x;
        n0 = adj.row[vn];
        n1 = adj.row[vn + 1];
        norig = adj.orig[vn];
      }
      for (int v = lo + threadIdx.x; v < hi; v += blockDim.x) {
        const int i = ob + (v - lo);
        int p0, p1, og;
        if (STAGED) {
          p0 = adj.row[i];
          p1 = adj.row[i + 1];
          og = 0;  // the masks are already built
        } else {
          p0 = n0;
          p1 = n1;
          og = norig;
          const int vn = v + (int)blockDim.x;
          if (vn < hi) {
            n0 = adj.row[vn];
            n1 = adj.row[vn + 1];
            norig = adj.orig[vn];
          }
        }
        // improved replicas take their best state from v as it stood at the
        // end of the previous sweep (v has not been updated since)
        if (imp != 0u) {
          if (STAGED) lbest[i] = (lbest[i] & ~imp) | (spin[v] & imp);
          else gbest[v] = (gbest[v] & ~imp) | (spin[v] & imp);
        }
        const int32_t hv = !has_field ? 0 : (STAGED ? lfield[i] : __ldg(&s.field[v]));
        auto draw = [&](uint4 (&out)[8]) { vertex_uniforms((uint32_t)og, bp, s.rk, out); };
        if (PF && !ready) vertex_uniforms((uint32_t)og, bp, s.rk, uu);
        ready = false;
        constexpr int accept = STAGED ? kAcceptMasks : (PF ? kAcceptPre : kAcceptLazy);
        const uint32_t sn = update_vertex<NP, FIELD, accept>(
            spin, v, p0, p1, adj, row, uu, draw, STAGED ? mcur + lmoff[i] : nullptr, hv, cd, cu);
        if (K == 1) {
          spin[v] = sn;
        } else if (DF) {
          spin[v] = sn;
          const uint32_t a = (uint32_t)__cvta_generic_to_shared(spin + v);
          const uint32_t bar = bar0 + 8u * (uint32_t)(gph & 1);
          for (int r = 0; r < K; ++r)
            if (r != k) st_async_u32(a, (uint32_t)r, sn, bar);
        } else {
          const uint32_t a = (uint32_t)__cvta_generic_to_shared(spin + v);
          for (int r = 0; r < K; ++r) st_cluster_u32(a, (uint32_t)r, sn);
        }
      }
      if (c + 1 < nc) {
        if (DF) df_arrive(expb[c]);
        else group_arrive(K);
        draw_first(c + 1);
        if (STAGED && more && !MG) mask_window(c, t + 1);
        if (DF) df_wait();
        else group_wait(K);
      }
    }
    if (more_a) {
      uint32_t *nrow = trow + ((t + ahead) & 1) * s.kmax1;
      if (x0 < s.kmax1) nrow[x0] = p0;
      if (x1 < s.kmax1) nrow[x1] = p1;
    }
    if (MG && more) cp_async_wait_all();
    // per-lane energy change, summed over the CTA and published to every CTA
    int32_t *pbuf = part + ((t + 1) & 1) * 32 * K;
    atomicAdd(&lane_acc[lane], 2 * (cd.warp_lane_total() - 2 * cu.warp_lane_total()));
    __syncthreads();
    if (threadIdx.x < 32) {
      const int32_t x = lane_acc[threadIdx.x];
      lane_acc[threadIdx.x] = 0;
      if (K == 1) {
        pbuf[threadIdx.x] = x;
      } else if (!DF) {
        for (int r = 0; r < K; ++r) peer_smem(pbuf, (uint32_t)r)[k * 32 + threadIdx.x] = x;
      } else {
        pbuf[k * 32 + threadIdx.x] = x;
        const uint32_t a = (uint32_t)__cvta_generic_to_shared(pbuf + k * 32 + threadIdx.x);
        const uint32_t bar = bar0 + 8u * (uint32_t)(gph & 1);
        for (int r = 0; r < K; ++r)
          if (r != k) st_async_u32(a, (uint32_t)r, x, bar);
      }
    }
    // the last class and the peers' partial sums complete the sweep's last phase
    if (DF) df_arrive(expb[nc - 1] + 4 * 32 * (K - 1));
    else group_arrive(K);
    if (PF && more) {
      sweep_prefix(t + 1);
      draw_first(0);
    }
    if (STAGED && more && !MG) mask_window(nc - 1, t + 1);
    if (DF) df_wait();
    else group_wait(K);
    if (STAGED && nc == 1 && !MG) __syncthreads();  // one class: its masks were built just now
    int32_t dsum = 0;
    for (int r = 0; r < K; ++r) dsum += pbuf[r * 32 + lane];
    e += dsum;
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

  // every update of the cluster precedes the last group barrier (with data
  // flow: one cluster barrier, after which no CTA sends to another)
  if (DF) cluster_barrier();
  for (int c = 0; c < nc; ++c) {
    const int lo = clo[c], hi = chi[c];
    for (int v = lo + threadIdx.x; v < hi; v += blockDim.x) {
      const uint32_t x = spin[v];
      gspin[v] = x;
      if (STAGED) gbest[v] = (lbest[cob[c] + (v - lo)] & ~imp) | (x & imp);
      else if (imp != 0u) gbest[v] = (gbest[v] & ~imp) | (x & imp);
    }
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
  if (DF) {
    cluster_barrier();  // after rank 0's done store
    if (threadIdx.x == 0 && *(volatile int *)dferr) atomicMin(&s.done[word], -1);
  }
}

template <int NP, bool STAGED, bool FIELD, bool PRE = false>
__global__ void __launch_bounds__(512) gm_kernel(GraphMscSolve s, GraphMscLaunch l) {
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
  gm_word<NP, STAGED, FIELD, true, PRE>(s, l, word, k, K, l.t_begin, t_end, l.resume, smem);
}

template <typename Kern>
cudaError_t launch_gm(Kern kernel, int grid, const GraphMscSolve &s, const GraphMscLaunch &l,
                      size_t smem, cudaStream_t stream) {
  cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err == cudaSuccess && l.cluster > 8)
    err = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(l.threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = l.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, s, l);
}

// Launch of the sweep kernel for the solve's shape; FIELD selects the build
// that adds local fields.
template <bool FIELD>
cudaError_t gm_launch_impl(const GraphMscSolve &s, const GraphMscLaunch &l, cudaStream_t stream) {
  const bool staged = l.own_n > 0;
  const size_t smem = gm_layout(s.n, l.cluster, s.n_colours, staged ? l.own_n : 0,
                                staged ? l.own_nnz : 0, staged ? l.own_lv : 0, s.kmax1, FIELD)
                          .total;
  const int grid = s.words * l.cluster;
  const bool pre = staged && l.gmask != nullptr;
  switch (l.planes * 4 + (staged ? 1 : 0) + (pre ? 2 : 0)) {
#define ISG_GM_CASE(NPV)                                                                     \
  case NPV * 4 + 3:                                                                          \
    return launch_gm(gm_kernel<NPV, true, FIELD, true>, grid, s, l, smem, stream);           \
  case NPV * 4 + 1:                                                                          \
    return launch_gm(gm_kernel<NPV, true, FIELD>, grid, s, l, smem, stream);                 \
  case NPV * 4:                                                                              \
    return launch_gm(gm_kernel<NPV, false, FIELD>, grid, s, l, smem, stream);
    ISG_GM_CASE(6) ISG_GM_CASE(8) ISG_GM_CASE(10) ISG_GM_CASE(12) ISG_GM_CASE(14)
#undef ISG_GM_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// The local-field builds (compiled in their own translation unit).
cudaError_t gm_launch_fields(const GraphMscSolve &s, const GraphMscLaunch &l,
                             cudaStream_t stream);

}  // namespace isg
