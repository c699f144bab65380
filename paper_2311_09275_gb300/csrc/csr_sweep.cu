// csr_sweep.cu -- colour-class Metropolis sweeps on arbitrary sparse graphs.
//
// Vertices are relabelled colour-major, so a colour class is a contiguous id
// range and no two vertices of a class are adjacent: a class is updated in
// parallel with no intra-class ordering.  Spins are int8 (+1/-1) packed four
// replicas per uint32 ("quad"); one Philox block yields the four replicas'
// uniforms of one vertex.
//
// Layout: a cluster of K CTAs owns Q replica quads of one instance.  Every
// CTA keeps a full copy of those quads' spins in shared memory, updates 1/K
// of each colour class and writes each new word to all K copies (distributed
// shared memory); one cluster barrier separates the classes.  The slice of
// each class a CTA owns is a contiguous id range, so its adjacency is a
// contiguous slice of the CSR: when it fits, the CTA stages those slices
// (row offsets, neighbour ids, weights, original ids) in shared memory once,
// and every neighbour gather of the sweep loop is a shared-memory load.  A
// thread draws the Philox blocks (and reads the field) of its first vertex of
// the next class between its arrival at the class barrier and the wait for it.
//
// Local fields: for graphs whose weights are all +1, or all +1/-1, the four
// lanes' counts of -1 neighbours are summed in one 32-bit add per neighbour
// (one byte per lane, degree <= 255); general integer weights sum per lane.
#include <climits>

#include "isg_device.cuh"
#include "isg_kernels.h"

namespace isg {
namespace {

__host__ __device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

struct CsrSmem {
  size_t spin, lrow, lorig, lcol, lwt, ocls, trow, part, lane_acc, total;
};

// own_n / own_nnz: the largest owned vertex / adjacency count of any rank
// (0 = not staged); trow_n: threshold entries cached per sweep (0 = none).
__host__ __device__ __forceinline__ CsrSmem csr_layout(int n, int Q, int K, int n_colours,
                                                       int own_n, int own_nnz, bool weights,
                                                       int trow_n) {
  CsrSmem m;
  m.spin = 0;
  m.lrow = align16(sizeof(uint32_t) * (size_t)n * Q);
  m.lorig = align16(m.lrow + (own_n ? sizeof(int32_t) * ((size_t)own_n + 1) : 0));
  m.lcol = align16(m.lorig + sizeof(int32_t) * (size_t)own_n);
  m.lwt = align16(m.lcol + sizeof(int32_t) * (size_t)own_nnz);
  m.ocls = align16(m.lwt + (weights ? sizeof(int32_t) * (size_t)own_nnz : 0));
  m.trow = align16(m.ocls + sizeof(int32_t) * 3 * (size_t)n_colours);  // class slice table
  m.part = align16(m.trow + 2 * sizeof(uint32_t) * (size_t)trow_n);
  m.lane_acc = m.part + 2 * sizeof(int32_t) * 4 * (size_t)Q * K;
  m.total = align16(m.lane_acc + sizeof(int32_t) * 4 * (size_t)Q);
  return m;
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

// Spin (+1/-1) of lane l of a packed word: byte l, sign-extended.
__device__ __forceinline__ int32_t lane8(uint32_t w, int l) {
  return ((int32_t)(w << (24 - 8 * l))) >> 24;
}

// Own slice of the id range [a, b) for rank k of K.
__device__ __forceinline__ void own_range(int a, int b, int k, int K, int &lo, int &hi) {
  const int len = b - a;
  lo = a + (int)((int64_t)len * k / K);
  hi = a + (int)((int64_t)len * (k + 1) / K);
}

// Per-lane int32 values summed over the CTA, published to every CTA of the
// cluster as part[k][slot]; ends with the group barrier, `during` running
// between the arrival and the wait.
template <int Q, typename During>
__device__ __forceinline__ void publish(const int32_t (&vals)[Q][4], int32_t *lane_acc,
                                        int32_t *part, int k, int K, During during) {
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int32_t s = __reduce_add_sync(0xFFFFFFFFu, vals[q][l]);
      if (lane_id() == 0 && s != 0) atomicAdd(&lane_acc[q * 4 + l], s);
    }
  __syncthreads();
  if (threadIdx.x < 4 * Q) {
    const int32_t v = lane_acc[threadIdx.x];
    lane_acc[threadIdx.x] = 0;
    if (K == 1) {
      part[threadIdx.x] = v;
    } else {
      for (int r = 0; r < K; ++r) peer_smem(part, (uint32_t)r)[k * 4 * Q + threadIdx.x] = v;
    }
  }
  group_arrive(K);
  during();
  group_wait(K);
}

// Best-state blend of vertex v for the improved lanes (byte masks bm[q]); kept
// out of line so that the rarely taken blend costs the sweep loop no registers.
template <int Q>
__device__ __noinline__ void blend_best(uint32_t *best, const uint32_t *spin, int n, int v,
                                        int quad0, const uint32_t (&bm)[Q]) {
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    if (bm[q] == 0u) continue;
    uint32_t &gb = best[(size_t)(quad0 + q) * n + v];
    gb = (gb & ~bm[q]) | (spin[q * n + v] & bm[q]);
  }
}

// Sources of one vertex's adjacency: staged in shared memory or global.
struct Adj {
  const int32_t *row;   // row offsets (local when staged)
  const int32_t *col;   // neighbours (relabelled ids; bit 31 = negative weight in mode 1)
  const int32_t *wt;    // weights (mode 2)
  const int32_t *orig;  // original ids
};

// Half energy changes kk[l] = -s_l h_l of the Q quads of vertex v (row slot
// i), where h_l = hv + sum_j w_vj s_j (hv: the vertex's local field, or 0).
template <int Q, int MODE>
__device__ __forceinline__ void fields(const uint32_t *spin, int n, int v, int p0, int p1,
                                       const Adj &a, int32_t hv, int32_t (&kk)[Q][4]) {
  if (MODE == 2) {
    int32_t h[Q][4];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int l = 0; l < 4; ++l) h[q][l] = hv;
    for (int p = p0; p < p1; ++p) {
      const int j = a.col[p];
      const int32_t wv = a.wt[p];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const uint32_t su = spin[q * n + j];
#pragma unroll
        for (int l = 0; l < 4; ++l) h[q][l] += wv * lane8(su, l);
      }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const uint32_t sv = spin[q * n + v];
#pragma unroll
      for (int l = 0; l < 4; ++l) kk[q][l] = -lane8(sv, l) * h[q][l];
    }
  } else {
    // count, per lane, the -1 spins among positive (and negative) neighbours
    uint32_t cpos[Q], cneg[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) cpos[q] = cneg[q] = 0u;
    int dneg = 0;
    for (int p = p0; p < p1; ++p) {
      const int e = a.col[p];
      const int j = e & 0x7FFFFFFF;
      const uint32_t neg = MODE == 1 ? (uint32_t)(e >> 31) : 0u;  // all ones if w = -1
      if (MODE == 1) dneg -= (int)neg;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const uint32_t minus = (spin[q * n + j] >> 1) & 0x01010101u;  // 1 per lane with s = -1
        if (MODE == 1) {
          cneg[q] += minus & neg;
          cpos[q] += minus & ~neg;
        } else {
          cpos[q] += minus;
        }
      }
    }
    const int dpos = (p1 - p0) - dneg;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const uint32_t sv = spin[q * n + v];
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        // h = hv + (dpos - 2 * minus_pos) - (dneg - 2 * minus_neg)
        int32_t h = hv + dpos - 2 * (int32_t)((cpos[q] >> (8 * l)) & 0xFFu);
        if (MODE == 1) h -= dneg - 2 * (int32_t)((cneg[q] >> (8 * l)) & 0xFFu);
        const int32_t m = -(int32_t)((sv >> (8 * l + 1)) & 1u);  // -1 if s_l = -1
        kk[q][l] = ((-h) ^ m) - m;                               // -s_l h
      }
    }
  }
}

template <int Q, int MODE, bool STAGED>
__device__ void csr_solve(const CsrSolve &s, const CsrLaunch &L, int quad0, int k, int K,
                          int t_begin, int t_end, int resume, uint8_t *smem) {
  const int n = s.n;
  const int trow_n = (s.kmax + 1 <= kCsrTableCache) ? s.kmax + 1 : 0;
  const CsrSmem lay = csr_layout(n, Q, K, s.n_colours, STAGED ? L.own_n : 0,
                                 STAGED ? L.own_nnz : 0, MODE == 2, trow_n);
  uint32_t *spin = reinterpret_cast<uint32_t *>(smem + lay.spin);  // [Q][n]
  int32_t *part = reinterpret_cast<int32_t *>(smem + lay.part);
  int32_t *lane_acc = reinterpret_cast<int32_t *>(smem + lay.lane_acc);
  uint32_t *trow = reinterpret_cast<uint32_t *>(smem + lay.trow);
  // per class: this rank's slice [clo, chi) and the row slot of its first
  // vertex (the vertex itself when the adjacency is not staged)
  const int nc = s.n_colours;
  int32_t *clo = reinterpret_cast<int32_t *>(smem + lay.ocls);
  int32_t *chi = clo + nc;
  int32_t *cob = chi + nc;
  const PhiloxKey key{s.key0, s.key1};
  const int lane = (int)lane_id();

  if (resume && s.has_target && s.hit[quad0] >= 0) return;
  if (resume && t_begin >= t_end) return;

  // spins of the Q quads, relabelled order
  for (int x = threadIdx.x; x < n * Q; x += blockDim.x) {
    const int q = x / n;
    const int v = x - q * n;
    const int gq = quad0 + q;
    uint32_t w;
    if (gq >= s.quads) {
      w = 0x01010101u;
    } else if (resume) {
      w = s.spins[(size_t)gq * n + v];
    } else {
      const uint4 u = philox10(make_uint4((uint32_t)s.orig[v], 0u, (uint32_t)(gq + s.rng_quad0), kTagInit), key);
      w = ((u.x >> 31) ? 0x01u : 0xFFu) | (((u.y >> 31) ? 0x01u : 0xFFu) << 8) |
          (((u.z >> 31) ? 0x01u : 0xFFu) << 16) | (((u.w >> 31) ? 0x01u : 0xFFu) << 24);
    }
    spin[x] = w;
  }

  if (threadIdx.x == 0) {
    int ov = 0;
    for (int c = 0; c < nc; ++c) {
      int lo, hi;
      own_range(s.class_start[c], s.class_start[c + 1], k, K, lo, hi);
      clo[c] = lo;
      chi[c] = hi;
      cob[c] = STAGED ? ov : lo;
      ov += hi - lo;
    }
  }
  __syncthreads();
  // adjacency of the owned slices: staged copy (local row ids) or global
  Adj adj;
  if (STAGED) {
    int32_t *lrow = reinterpret_cast<int32_t *>(smem + lay.lrow);
    int32_t *lorig = reinterpret_cast<int32_t *>(smem + lay.lorig);
    int32_t *lcol = reinterpret_cast<int32_t *>(smem + lay.lcol);
    int32_t *lwt = reinterpret_cast<int32_t *>(smem + lay.lwt);
    int ebase = 0;
    for (int c = 0; c < nc; ++c) {
      const int lo = clo[c], hi = chi[c], ob = cob[c];
      const int e0 = s.rowptr[lo], e1 = s.rowptr[hi];
      for (int i = threadIdx.x; i <= hi - lo; i += blockDim.x) {
        lrow[ob + i] = s.rowptr[lo + i] - e0 + ebase;
        if (i < hi - lo) lorig[ob + i] = s.orig[lo + i];
      }
      for (int p = threadIdx.x; p < e1 - e0; p += blockDim.x) {
        lcol[ebase + p] = s.col[e0 + p];
        if (MODE == 2) lwt[ebase + p] = s.wt[e0 + p];
      }
      ebase += e1 - e0;
    }
    adj = {lrow, lcol, lwt, lorig};
  } else {
    adj = {s.rowptr, s.col, s.wt, s.orig};
  }
  if (threadIdx.x < 4 * Q) lane_acc[threadIdx.x] = 0;
  const int kmax1 = s.kmax + 1;
  // threshold rows: one schedule (row t for sweep t), or in parallel tempering
  // one row per temperature slot of slot_quads quads (the same every sweep)
  const uint32_t *wtab =
      s.slot_quads ? s.table + (size_t)(quad0 / s.slot_quads) * kmax1 : s.table;
  const size_t tstride = s.slot_quads ? 0 : (size_t)kmax1;
  // cached threshold rows: two buffers, the next sweep's row loaded a sweep ahead
  if (trow_n && t_begin < t_end)
    for (int i = threadIdx.x; i < trow_n; i += blockDim.x)
      trow[(t_begin & 1) * trow_n + i] = wtab[(size_t)t_begin * tstride + i];
  // peers write into this CTA's copy of the quads only after every CTA has loaded it
  sync_group(K);

  // bookkeeping lanes: lane = q * 4 + l, kept identically by every warp
  int32_t e = 0, e_best = 0;
  const int my_q = lane >> 2;
  const int my_r = 4 * (quad0 + my_q) + (lane & 3);
  const bool valid = (lane < 4 * Q) && (quad0 + my_q < s.quads) && (my_r < s.replicas);

  if (!resume) {
    // E = sum over edges once (at the lower relabelled end), general per-lane sums
    int32_t vals[Q][4];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int l = 0; l < 4; ++l) vals[q][l] = 0;
    for (int c = 0; c < s.n_colours; ++c) {
      int lo, hi;
      own_range(s.class_start[c], s.class_start[c + 1], k, K, lo, hi);
      for (int v = lo + threadIdx.x; v < hi; v += blockDim.x) {
        const int p0 = s.rowptr[v], p1 = s.rowptr[v + 1];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const uint32_t sv = spin[q * n + v];
          for (int p = p0; p < p1; ++p) {
            const int u = s.col[p] & 0x7FFFFFFF;
            if (u <= v) continue;
            const int32_t wv = s.wt[p];
            const uint32_t su = spin[q * n + u];
#pragma unroll
            for (int l = 0; l < 4; ++l) vals[q][l] += wv * lane8(sv, l) * lane8(su, l);
          }
          if (MODE == 2 && s.field) {
            const int32_t hv = s.field[v];
#pragma unroll
            for (int l = 0; l < 4; ++l) vals[q][l] += hv * lane8(sv, l);
          }
          if (quad0 + q < s.quads) s.best[(size_t)(quad0 + q) * n + v] = sv;
        }
      }
    }
    publish<Q>(vals, lane_acc, part, k, K, [] {});  // publication 0 uses buffer 0
    int32_t tot = 0;
    if (lane < 4 * Q)
      for (int r = 0; r < K; ++r) tot += part[r * 4 * Q + lane];
    e = tot;
    e_best = e;
  } else if (valid) {
    e = s.e_cur[my_r];
    e_best = s.e_best[my_r];
  }

  // Random numbers and fields do not depend on the spins: those of a thread's
  // first vertex of the next class (or of the next sweep's first class) are
  // drawn between the arrival at the group barrier and the wait for it.
  uint4 pu[Q];
  int32_t phv = 0;
  bool ready = false;  // pu, phv hold this thread's next vertex's uniforms and field
  auto draw_first = [&](int c, int tt) {
    const int v = clo[c] + (int)threadIdx.x;
    ready = v < chi[c];
    if (ready) {
      const uint32_t ov = (uint32_t)adj.orig[cob[c] + threadIdx.x];
#pragma unroll
      for (int q = 0; q < Q; ++q)
        pu[q] = philox10(
            make_uint4(ov, (uint32_t)tt, (uint32_t)(quad0 + q + s.rng_quad0), kTagSweep), key);
      if (MODE == 2 && s.field) phv = __ldg(&s.field[v]);
    }
  };
  if (t_begin < t_end) draw_first(0, t_begin);

  int t = t_begin;
  int hit = -1;
  uint32_t imp = 0u;  // lanes whose best state is the state at the start of sweep t
  constexpr int kPre = 2;  // entries per thread prefetched in registers (the rest: at the end)
  for (; t < t_end; ++t) {
    const uint32_t *row = wtab + (size_t)t * tstride;
    const bool more = t + 1 < t_end;
    uint32_t pre[kPre];
    if (trow_n) {
      row = trow + (t & 1) * trow_n;
#pragma unroll
      for (int j = 0; j < kPre; ++j) {
        const int x = (int)threadIdx.x + j * (int)blockDim.x;
        pre[j] = (more && x < trow_n) ? wtab[(size_t)(t + 1) * tstride + x] : 0u;
      }
    }
    // byte masks of the improved lanes of each quad
    uint32_t bm[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const uint32_t m4 = (imp >> (4 * q)) & 0xFu;
      bm[q] = ((m4 & 1u) ? 0xFFu : 0u) | ((m4 & 2u) ? 0xFF00u : 0u) |
              ((m4 & 4u) ? 0xFF0000u : 0u) | ((m4 & 8u) ? 0xFF000000u : 0u);
    }
    int32_t de[Q][4];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int l = 0; l < 4; ++l) de[q][l] = 0;
    for (int c = 0; c < nc; ++c) {
      const int lo = clo[c], hi = chi[c], ob = cob[c];  // ob: row slot of vertex lo
      for (int v = lo + threadIdx.x; v < hi; v += blockDim.x) {
        const int i = ob + (v - lo);
        const int p0 = adj.row[i], p1 = adj.row[i + 1];
        const uint32_t ov = (uint32_t)adj.orig[i];
        if (imp != 0u) {
          // improved lanes take their best state from v as it stood at the end
          // of the previous sweep (v has not been updated since)
          blend_best<Q>(s.best, spin, n, v, quad0, bm);
        }
        int32_t kk[Q][4];
        // local fields ride only with general weights (field instances run in mode 2)
        fields<Q, MODE>(spin, n, v, p0, p1, adj,
                        (MODE == 2 && s.field) ? (ready ? phv : __ldg(&s.field[v])) : 0, kk);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          // lanes with kk > 0 are uphill; the rest are always taken
          uint32_t up = 0u;
#pragma unroll
          for (int l = 0; l < 4; ++l) up |= (kk[q][l] > 0 ? 1u : 0u) << l;
          uint32_t acc = ~up & 0xFu;
          if (up != 0u) {
            const uint4 u =
                ready ? pu[q]
                      : philox10(make_uint4(ov, (uint32_t)t,
                                            (uint32_t)(quad0 + q + s.rng_quad0), kTagSweep),
                                 key);
            if ((up & 1u) && u.x < row[kk[q][0]]) acc |= 1u;
            if ((up & 2u) && u.y < row[kk[q][1]]) acc |= 2u;
            if ((up & 4u) && u.z < row[kk[q][2]]) acc |= 4u;
            if ((up & 8u) && u.w < row[kk[q][3]]) acc |= 8u;
          }
          uint32_t flip = 0u;
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            if ((acc >> l) & 1u) {
              flip |= 0xFEu << (8 * l);
              de[q][l] += 2 * kk[q][l];
            }
          }
          if (flip) {
            const uint32_t sn = spin[q * n + v] ^ flip;
            if (K == 1) {
              spin[q * n + v] = sn;
            } else {
              for (int r = 0; r < K; ++r) peer_smem(spin, (uint32_t)r)[q * n + v] = sn;
            }
          }
        }
        ready = false;
      }
      if (c + 1 < nc) {
        group_arrive(K);
        draw_first(c + 1, t);
        group_wait(K);
      }
    }
    if (trow_n && more) {
      // the other buffer's last reads were in the previous sweep
      uint32_t *nrow = trow + ((t + 1) & 1) * trow_n;
#pragma unroll
      for (int j = 0; j < kPre; ++j) {
        const int x = (int)threadIdx.x + j * (int)blockDim.x;
        if (x < trow_n) nrow[x] = pre[j];
      }
      for (int x = (int)threadIdx.x + kPre * (int)blockDim.x; x < trow_n; x += blockDim.x)
        nrow[x] = wtab[(size_t)(t + 1) * tstride + x];
    }
    // sweep t is publication t + 1 (the initial energy is publication 0)
    int32_t *pbuf = part + ((t + 1) & 1) * 4 * Q * K;
    publish<Q>(de, lane_acc, pbuf, k, K, [&] {
      if (more) draw_first(0, t + 1);
    });
    int32_t tot = 0;
    if (lane < 4 * Q)
      for (int r = 0; r < K; ++r) tot += pbuf[r * 4 * Q + lane];
    e += tot;
    const bool better = valid && e < e_best;
    if (better) e_best = e;
    imp = __ballot_sync(0xFFFFFFFFu, better);
    if (s.has_target) {
      const int32_t mn = __reduce_min_sync(0xFFFFFFFFu, valid ? e_best : INT_MAX);
      if (mn <= s.target) {
        hit = t;
        ++t;
        break;
      }
    }
  }

  // every update of the cluster precedes the last group barrier
  if (imp != 0u) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const uint32_t m4 = (imp >> (4 * q)) & 0xFu;
      if (m4 == 0u) continue;
      const uint32_t bmq = ((m4 & 1u) ? 0xFFu : 0u) | ((m4 & 2u) ? 0xFF00u : 0u) |
                           ((m4 & 4u) ? 0xFF0000u : 0u) | ((m4 & 8u) ? 0xFF000000u : 0u);
      uint32_t *gb = s.best + (size_t)(quad0 + q) * n;
      for (int c = 0; c < s.n_colours; ++c) {
        int lo, hi;
        own_range(s.class_start[c], s.class_start[c + 1], k, K, lo, hi);
        for (int v = lo + threadIdx.x; v < hi; v += blockDim.x)
          gb[v] = (gb[v] & ~bmq) | (spin[q * n + v] & bmq);
      }
    }
  }

  // write back own vertices (every CTA holds all; each writes its slice)
  for (int c = 0; c < s.n_colours; ++c) {
    int lo, hi;
    own_range(s.class_start[c], s.class_start[c + 1], k, K, lo, hi);
    for (int q = 0; q < Q; ++q) {
      if (quad0 + q >= s.quads) continue;
      for (int v = lo + threadIdx.x; v < hi; v += blockDim.x)
        s.spins[(size_t)(quad0 + q) * n + v] = spin[q * n + v];
    }
  }
  if (k == 0) {
    if (threadIdx.x < 32 && valid) {
      s.e_cur[my_r] = e;
      s.e_best[my_r] = e_best;
    }
    if (threadIdx.x == 0) {
      for (int q = 0; q < Q; ++q) {
        if (quad0 + q >= s.quads) continue;
        if (s.has_target && hit >= 0) s.hit[quad0 + q] = hit;
        s.done[quad0 + q] = t;
      }
    }
  }
}

// Single-quad packed-count builds are held to 64 registers (two CTAs per SM),
// which the general-weights build cannot reach without spilling.
template <int Q, int MODE, bool STAGED>
__global__ void __launch_bounds__(512, (Q == 1 && MODE != 2) ? 2 : 1)
    csr_kernel(CsrSolve s, CsrLaunch l) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int K = l.cluster;
  const int k = (int)(blockIdx.x % K);
  const int quad0 = (int)(blockIdx.x / K) * Q;
  int t_end = l.t_end;
  if (l.stop_from_hits) {
    int m = INT_MAX;
    for (int q = 0; q < s.quads; ++q)
      if (s.hit[q] >= 0 && s.hit[q] < m) m = s.hit[q];
    if (m != INT_MAX && m + 1 < t_end) t_end = m + 1;
  }
  csr_solve<Q, MODE, STAGED>(s, l, quad0, k, K, l.t_begin, t_end, l.resume, smem);
}

template <typename Kern>
cudaError_t launch_csr(Kern kernel, int grid, const CsrSolve &s, const CsrLaunch &l, size_t smem,
                       cudaStream_t stream) {
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

// Two CTAs per SM (64 registers): the units are independent CTAs.
__global__ void __launch_bounds__(512, 2) csr_batch_kernel(const CsrBatchItem *items,
                                                           const int32_t *count_dev,
                                                           const int32_t *order, int32_t *next) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int item;
  const int count = *count_dev;
  const CsrLaunch none = {};
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(next, 1);
    __syncthreads();
    const int it = item;
    __syncthreads();
    if (it >= count) break;
    const CsrBatchItem u = items[order[it]];
    int t_end = u.t_end;
    if (u.stop_from_hits) {
      // the solve's stop sweep from the first pass (uniform across the CTA)
      int m = INT_MAX;
      for (int q = 0; q < u.solve.quads; ++q)
        if (u.solve.hit[q] >= 0 && u.solve.hit[q] < m) m = u.solve.hit[q];
      if (m == INT_MAX) continue;  // no unit reached the target: the first pass stands
      if (m + 1 < t_end) t_end = m + 1;
    }
    // field mode is per instance: dispatch (uniform across the CTA)
    if (u.solve.mode == 0)
      csr_solve<1, 0, false>(u.solve, none, u.quad, 0, 1, u.t_begin, t_end, u.resume, smem);
    else if (u.solve.mode == 1)
      csr_solve<1, 1, false>(u.solve, none, u.quad, 0, 1, u.t_begin, t_end, u.resume, smem);
    else
      csr_solve<1, 2, false>(u.solve, none, u.quad, 0, 1, u.t_begin, t_end, u.resume, smem);
    __syncthreads();
  }
}

}  // namespace

size_t csr_smem_bytes(int32_t n, int32_t quads_per_cta, int32_t cluster, int32_t n_colours,
                      int32_t own_n, int32_t own_nnz, int32_t mode, int32_t kmax) {
  const int trow_n = (kmax + 1 <= kCsrTableCache) ? kmax + 1 : 0;
  return csr_layout(n, quads_per_cta, cluster, n_colours, own_n, own_nnz, mode == 2, trow_n)
      .total;
}

cudaError_t csr_launch(const CsrSolve &s, const CsrLaunch &l, cudaStream_t stream) {
  const int Q = l.quads_per_cta;
  const bool staged = l.own_n > 0;
  const size_t smem = csr_smem_bytes(s.n, Q, l.cluster, s.n_colours, staged ? l.own_n : 0,
                                     staged ? l.own_nnz : 0, s.mode, s.kmax);
  const int groups = (s.quads + Q - 1) / Q;
  const int grid = groups * l.cluster;
#define ISG_CSR_CASE(QV, MV, SV)                                                    \
  if (Q == QV && s.mode == MV && staged == SV)                                      \
    return launch_csr(csr_kernel<QV, MV, SV>, grid, s, l, smem, stream);
  ISG_CSR_CASE(1, 0, true) ISG_CSR_CASE(1, 1, true) ISG_CSR_CASE(1, 2, true)
  ISG_CSR_CASE(1, 0, false) ISG_CSR_CASE(1, 1, false) ISG_CSR_CASE(1, 2, false)
  ISG_CSR_CASE(2, 0, true) ISG_CSR_CASE(2, 1, true) ISG_CSR_CASE(2, 2, true)
  ISG_CSR_CASE(2, 0, false) ISG_CSR_CASE(2, 1, false) ISG_CSR_CASE(2, 2, false)
#undef ISG_CSR_CASE
  return cudaErrorInvalidValue;
}

cudaError_t csr_batch_launch(const CsrBatchItem *items_dev, const int32_t *count_dev,
                             const int32_t *order_dev, int32_t *next_dev, int32_t ctas,
                             int32_t threads, size_t smem, cudaStream_t stream) {
  cudaError_t err = cudaFuncSetAttribute(csr_batch_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  csr_batch_kernel<<<ctas, threads, smem, stream>>>(items_dev, count_dev, order_dev, next_dev);
  return cudaGetLastError();
}

}  // namespace isg
