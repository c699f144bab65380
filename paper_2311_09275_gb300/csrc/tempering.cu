// tempering.cu -- the exchange step and the Houdayer cluster moves of
// parallel tempering on multi-spin-coded state: replica word k holds 32 chains
// at temperature slot k, so exchanging the configurations of chain c between
// slots k and k+1 moves bit c of every site word between the two words (a
// masked swap) and swaps the chains' energies; a cluster move flips, in both
// chains of a pair within one word, the connected component of a drawn site
// among the sites where they differ (on a torus by ring scans, on a graph by
// passes over its adjacency).
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

// The same exchange on int8 quad state (4 chains per uint32, one byte each):
// slot k holds quads 8k .. 8k+7, chain c in byte c mod 4 of quad 8k + c / 4.
__global__ void __launch_bounds__(256) pt_exchange_quads_kernel(
    uint32_t *quads, int32_t *e_cur, int n, int K, int parity, int round, PhiloxKey key,
    const int8_t *sgn, const uint32_t *xtable, int xlen, unsigned long long *accepted) {
  const int k = parity + 2 * (int)blockIdx.x;
  if (k + 1 >= K) return;
  __shared__ uint32_t s_mask;
  if (threadIdx.x < 32) {
    const int c = (int)threadIdx.x;
    const int32_t ek = e_cur[32 * k + c], ek1 = e_cur[32 * (k + 1) + c];
    const int64_t de = (int64_t)ek - ek1;
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
  for (int x = threadIdx.x; x < 8 * n; x += blockDim.x) {
    const int j = x / n, v = x - j * n;  // quad j of the slot, vertex v
    const uint32_t m4 = (mask >> (4 * j)) & 0xFu;
    if (m4 == 0u) continue;
    const uint32_t bm = ((m4 & 1u) ? 0xFFu : 0u) | ((m4 & 2u) ? 0xFF00u : 0u) |
                        ((m4 & 4u) ? 0xFF0000u : 0u) | ((m4 & 8u) ? 0xFF000000u : 0u);
    uint32_t *a = quads + (size_t)(8 * k + j) * n + v;
    uint32_t *b = quads + (size_t)(8 * (k + 1) + j) * n + v;
    const uint32_t t = (*a ^ *b) & bm;
    *a ^= t;
    *b ^= t;
  }
}

// One warp spreads cluster bits along a ring of `len` sites (base + x*stride,
// x = 0..len-1, closed by a wrap edge) through runs of differing sites, in
// both directions.  Each lane owns a segment; a segment maps an incoming
// carry k to G | (P & k) (G: its carry out from k = 0, P: AND of its D), and
// these maps compose associatively, so a warp scan of them gives every lane
// its incoming carry; the wrap carry is the whole ring's G (the least fixed
// point of k = G | (P & k)).  A site at ring position x that gains a bit
// marks ring x of the other orientation in `mark` (one bit per ring).  Bits
// are only ever set (atomically: rings crossing this one may grow at the same
// time; a bit they set after this ring read the site is marked for the next
// pass by them).  Returns whether a bit was set.
__device__ bool ring_spread(uint32_t *C, const uint32_t *D, int base, int len, int stride,
                            uint32_t *mark) {
  const int lane = (int)(threadIdx.x & 31u);
  const int seg = (len + 31) / 32;
  const int x0 = min(len, lane * seg), x1 = min(len, x0 + seg);
  bool changed = false;
  for (int dir = 0; dir < 2; ++dir) {
    uint32_t g = 0u, pm = 0xFFFFFFFFu;
    for (int x = x0; x < x1; ++x) {
      const int i = base + (dir == 0 ? x : len - 1 - x) * stride;
      const uint32_t d = D[i];
      g = C[i] | (d & g);
      pm &= d;
    }
    // inclusive scan of (g, pm) in lane order: later (g, pm) after earlier (g', pm')
    uint32_t G = g, Pm = pm;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t Ge = __shfl_up_sync(0xFFFFFFFFu, G, o);
      const uint32_t Pe = __shfl_up_sync(0xFFFFFFFFu, Pm, o);
      if (lane >= o) {
        G = G | (Pm & Ge);
        Pm = Pm & Pe;
      }
    }
    const uint32_t g_all = __shfl_sync(0xFFFFFFFFu, G, 31);
    uint32_t ge = __shfl_up_sync(0xFFFFFFFFu, G, 1), pe = __shfl_up_sync(0xFFFFFFFFu, Pm, 1);
    if (lane == 0) {
      ge = 0u;
      pe = 0xFFFFFFFFu;
    }
    uint32_t carry = ge | (pe & g_all);
    // marks gathered per mark word along the segment, one atomic per word
    int mw = -1;
    uint32_t mm = 0u;
    for (int x = x0; x < x1; ++x) {
      const int pos = dir == 0 ? x : len - 1 - x;
      const int i = base + pos * stride;
      const uint32_t cur = C[i];
      const uint32_t v = cur | (D[i] & carry);
      if (v != cur) {
        atomicOr(&C[i], v);  // rings of both orientations grow at once
        changed = true;
        if ((pos >> 5) != mw) {
          if (mm) atomicOr(&mark[mw], mm);
          mw = pos >> 5;
          mm = 0u;
        }
        mm |= 1u << (pos & 31);
      }
      carry = v;
    }
    if (mm) atomicOr(&mark[mw], mm);
    __syncwarp();
  }
  return changed;
}

// ring_spread for rings of up to 32 x SEG sites with each lane's segment held
// in registers across both directions (one shared-memory read per site); the
// backward direction scans the lanes in descending order.  Same result as
// ring_spread.
template <int SEG>
__device__ bool ring_spread_reg(uint32_t *C, const uint32_t *D, int base, int len, int stride,
                                uint32_t *mark) {
  const int lane = (int)(threadIdx.x & 31u);
  const int seg = (len + 31) / 32;
  const int x0 = min(len, lane * seg), cnt = min(len, x0 + seg) - x0;
  uint32_t d[SEG], c[SEG], c_in[SEG];
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    const int i = base + (x0 + j) * stride;
    d[j] = j < cnt ? D[i] : 0u;
    c[j] = j < cnt ? C[i] : 0u;
    c_in[j] = c[j];
  }
  // forward: increasing positions, lanes in ascending order
  {
    uint32_t g = 0u, pm = 0xFFFFFFFFu;
#pragma unroll
    for (int j = 0; j < SEG; ++j)
      if (j < cnt) {
        g = c[j] | (d[j] & g);
        pm &= d[j];
      }
    uint32_t G = g, Pm = pm;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t Ge = __shfl_up_sync(0xFFFFFFFFu, G, o);
      const uint32_t Pe = __shfl_up_sync(0xFFFFFFFFu, Pm, o);
      if (lane >= o) {
        G = G | (Pm & Ge);
        Pm = Pm & Pe;
      }
    }
    const uint32_t g_all = __shfl_sync(0xFFFFFFFFu, G, 31);
    uint32_t ge = __shfl_up_sync(0xFFFFFFFFu, G, 1), pe = __shfl_up_sync(0xFFFFFFFFu, Pm, 1);
    if (lane == 0) {
      ge = 0u;
      pe = 0xFFFFFFFFu;
    }
    uint32_t carry = ge | (pe & g_all);
#pragma unroll
    for (int j = 0; j < SEG; ++j)
      if (j < cnt) {
        c[j] |= d[j] & carry;
        carry = c[j];
      }
  }
  // backward: decreasing positions, lanes in descending order
  {
    uint32_t g = 0u, pm = 0xFFFFFFFFu;
#pragma unroll
    for (int j = SEG - 1; j >= 0; --j)
      if (j < cnt) {
        g = c[j] | (d[j] & g);
        pm &= d[j];
      }
    uint32_t G = g, Pm = pm;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t Ge = __shfl_down_sync(0xFFFFFFFFu, G, o);
      const uint32_t Pe = __shfl_down_sync(0xFFFFFFFFu, Pm, o);
      if (lane + o < 32) {
        G = G | (Pm & Ge);
        Pm = Pm & Pe;
      }
    }
    const uint32_t g_all = __shfl_sync(0xFFFFFFFFu, G, 0);
    uint32_t ge = __shfl_down_sync(0xFFFFFFFFu, G, 1), pe = __shfl_down_sync(0xFFFFFFFFu, Pm, 1);
    if (lane == 31) {
      ge = 0u;
      pe = 0xFFFFFFFFu;
    }
    uint32_t carry = ge | (pe & g_all);
#pragma unroll
    for (int j = SEG - 1; j >= 0; --j)
      if (j < cnt) {
        c[j] |= d[j] & carry;
        carry = c[j];
      }
  }
  // write back the sites that gained bits, marking their crossing rings
  bool changed = false;
  int mw = -1;
  uint32_t mm = 0u;
#pragma unroll
  for (int j = 0; j < SEG; ++j)
    if (j < cnt && c[j] != c_in[j]) {
      const int pos = x0 + j;
      atomicOr(&C[base + pos * stride], c[j]);
      changed = true;
      if ((pos >> 5) != mw) {
        if (mm) atomicOr(&mark[mw], mm);
        mw = pos >> 5;
        mm = 0u;
      }
      mm |= 1u << (pos & 31);
    }
  if (mm) atomicOr(&mark[mw], mm);
  __syncwarp();
  return changed;
}

// Ring update dispatched on the ring length.
__device__ __forceinline__ bool ring_update(uint32_t *C, const uint32_t *D, int base, int len,
                                            int stride, uint32_t *mark) {
  if (len <= 128) return ring_spread_reg<4>(C, D, base, len, stride, mark);
  if (len <= 256) return ring_spread_reg<8>(C, D, base, len, stride, mark);
  return ring_spread(C, D, base, len, stride, mark);
}

// Houdayer cluster moves on one slot word per CTA (slots k0 + blockIdx.x):
// chains 2m and 2m+1 (lanes) form pair m.  D[i] holds, at bit 2m, whether
// the pair differs at site i; C[i] grows, at the same bits, the connected
// component of the drawn differing site among differing sites.  Both chains
// then flip C, and the word's 32 energies are recomputed.
template <int NP>
__global__ void __launch_bounds__(1024) pt_cluster_kernel(uint32_t *spins, int32_t *e_cur,
                                                          const uint8_t *cbits, int L, int W,
                                                          int k0, int round, PhiloxKey key,
                                                          unsigned long long *flipped) {
  extern __shared__ __align__(16) uint32_t sm[];
  const int n = L * W;
  const int k = k0 + (int)blockIdx.x;
  uint32_t *D = sm, *C = sm + n;
  // rings (rows, columns) holding sites that gained a bit since the ring was
  // last spread: only those can spread further
  const int rwords = (L + 31) / 32, cwords = (W + 31) / 32;
  uint32_t *rdirty = sm + 2 * n, *cdirty = rdirty + rwords;  // two buffers each: this pass, next
  uint32_t *rdirty1 = cdirty + cwords, *cdirty1 = rdirty1 + rwords;
  __shared__ int32_t wsum[32][16];
  __shared__ int64_t pick[16];
  __shared__ int changed;
  uint32_t *word = spins + (size_t)k * n;
  const int nt = (int)blockDim.x, tid = (int)threadIdx.x;
  const int chunk = (n + nt - 1) / nt;
  const int i0 = min(n, tid * chunk), i1 = min(n, i0 + chunk);
  for (int w = (int)threadIdx.x; w < 2 * (rwords + cwords); w += (int)blockDim.x) rdirty[w] = 0u;
  // 1. differing sites per pair, and this thread's count of them per pair
  int32_t cnt[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) cnt[m] = 0;
  for (int i = i0; i < i1; ++i) {
    const uint32_t w = word[i];
    const uint32_t d = (w ^ (w >> 1)) & 0x55555555u;
    D[i] = d;
    C[i] = 0u;
#pragma unroll
    for (int m = 0; m < 16; ++m) cnt[m] += (d >> (2 * m)) & 1u;
  }
  // 2. exclusive prefix of the counts over threads (warp scan, then warp totals)
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  int32_t pre[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    int32_t x = cnt[m];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    pre[m] = x - cnt[m];
    if (lane == 31) wsum[warp][m] = x;
  }
  __syncthreads();
  if (tid < 16) {
    int64_t tot = 0;
    for (int w = 0; w < nw; ++w) {
      const int32_t v = wsum[w][tid];
      wsum[w][tid] = (int32_t)tot;  // exclusive offset of warp w
      tot += v;
    }
    // 3. the drawn site of pair m: the (u mod D)-th differing site
    if (tot > 0) {
      const uint4 u = philox10(make_uint4((uint32_t)k, (uint32_t)round, (uint32_t)tid, 3u), key);
      pick[tid] = (int64_t)((uint64_t)u.x % (uint64_t)tot);
    } else {
      pick[tid] = -1;
    }
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int64_t p = pick[m];
    const int64_t lo = (int64_t)wsum[warp][m] + pre[m];
    if (p >= lo && p < lo + cnt[m]) {
      int64_t seen = lo;
      for (int i = i0; i < i1; ++i)
        if ((D[i] >> (2 * m)) & 1u) {
          if (seen == p) {
            C[i] |= 1u << (2 * m);
            atomicOr(&rdirty[(i / W) >> 5], 1u << ((i / W) & 31));
            atomicOr(&cdirty[(i % W) >> 5], 1u << ((i % W) & 31));
            break;
          }
          ++seen;
        }
    }
  }
  __syncthreads();
  // 4. grow the clusters to their components (bits only ever get set, so any
  //    order of updates reaches the same fixed point).  A pass spreads, one
  //    warp per ring, the bits along whole runs of differing sites of every
  //    row and column marked since it was last spread, rows and columns at
  //    once; sites that gain bits mark the crossing rings for the next pass.
  //    The number of passes follows the number of turns of the clusters'
  //    paths, not their length; growth ends when a pass sets no bit.
  for (int pass = 0;; ++pass) {
    uint32_t *rcur = (pass & 1) ? rdirty1 : rdirty, *ccur = (pass & 1) ? cdirty1 : cdirty;
    uint32_t *rnxt = (pass & 1) ? rdirty : rdirty1, *cnxt = (pass & 1) ? cdirty : cdirty1;
    if (tid == 0) changed = 0;
    __syncthreads();
    bool any = false;
    for (int g = warp; g < L + W; g += nw) {
      if (g < L) {
        if ((rcur[g >> 5] >> (g & 31)) & 1u) any |= ring_update(C, D, g * W, W, 1, cnxt);
      } else {
        const int c = g - L;
        if ((ccur[c >> 5] >> (c & 31)) & 1u) any |= ring_update(C, D, c, L, W, rnxt);
      }
    }
    if (any) changed = 1;
    __syncthreads();
    for (int w = tid; w < rwords + cwords; w += nt) rcur[w] = 0u;  // rcur, ccur: adjacent
    const bool more = changed != 0;
    // every thread has read `changed` and cleared this pass's marks before the
    // next pass marks them again
    __syncthreads();
    if (!more) break;
  }
  // 5. flip the clusters in both chains; recount the word's unsatisfied bonds
  SlicedCounter<NP> cntu;
  cntu.clear();
  unsigned long long flips = 0;
  for (int i = i0; i < i1; ++i) {
    const uint32_t cl = C[i];
    flips += __popc(cl);
    if (cl) word[i] ^= cl | (cl << 1);
  }
  __syncthreads();  // global writes of this CTA visible to its own threads
  for (int i = i0; i < i1; ++i) {
    const int r = i / W, c = i - r * W;
    const int ir = r * W + (c == W - 1 ? 0 : c + 1), id = (r == L - 1 ? 0 : r + 1) * W + c;
    const uint32_t s0 = word[i];
    const uint32_t cb = cbits[i];
    const uint32_t a = ~(s0 ^ word[ir] ^ (0u - (cb & 1u)));
    const uint32_t d = ~(s0 ^ word[id] ^ (0u - ((cb >> 1) & 1u)));
    cntu.add2(a ^ d, a & d);
  }
  const int32_t tot = cntu.warp_lane_total();
  __shared__ int32_t lane_tot[32];
  if (tid < 32) lane_tot[tid] = 0;
  __syncthreads();
  atomicAdd(&lane_tot[lane], tot);
  for (int o = 16; o > 0; o >>= 1) flips += __shfl_down_sync(0xFFFFFFFFu, flips, o);
  if (lane == 0 && flips) atomicAdd(&flipped[k], flips);
  __syncthreads();
  if (tid < 32) e_cur[32 * k + tid] = 2 * lane_tot[tid] - 2 * n;  // E = 2 U - 2n (torus)
}

// Houdayer cluster moves on graph slot words (the multi-spin graph layout:
// vertices relabelled colour-major; col holds relabelled neighbours with bit 31
// set for weight -1; orig maps a relabelled vertex to the caller's id), one
// CTA per slot k0 + blockIdx.x.  As on the torus: D[v] has, at bit 2m, whether
// pair m differs at v; the drawn site is the (u mod D)-th differing vertex in
// the caller's vertex order; C[v] grows the connected component of the drawn
// vertex among differing vertices, by passes over the vertices that can still
// gain a bit, each taking the bits of its neighbours (in place, so a pass may
// carry a bit over several edges; bits only get set, so the fixed point is the
// component whatever the order); both chains flip C and the word's 32
// energies are recounted over the edges (and the local fields, weights +1).
template <int NP>
__global__ void __launch_bounds__(1024) pt_cluster_graph_kernel(
    uint32_t *spins, int32_t *e_cur, int n, const int32_t *rowptr, const int32_t *col,
    const int32_t *orig, const int32_t *field, int k0, int round, PhiloxKey key,
    unsigned long long *flipped) {
  extern __shared__ __align__(16) uint32_t sm[];
  const int k = k0 + (int)blockIdx.x;
  uint32_t *D = sm, *C = sm + n;
  int32_t *inv = reinterpret_cast<int32_t *>(sm + 2 * n);  // caller's id -> relabelled
  __shared__ int32_t wsum[32][16];
  __shared__ int64_t pick[16];
  __shared__ int changed;
  uint32_t *word = spins + (size_t)k * n;
  const int nt = (int)blockDim.x, tid = (int)threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int v = tid; v < n; v += nt) {
    const uint32_t w = word[v];
    D[v] = (w ^ (w >> 1)) & 0x55555555u;
    C[v] = 0u;
    inv[orig[v]] = v;
  }
  __syncthreads();
  // 1. differing vertices per pair, counted over this thread's chunk of the
  //    caller's ids
  const int chunk = (n + nt - 1) / nt;
  const int i0 = min(n, tid * chunk), i1 = min(n, i0 + chunk);
  int32_t cnt[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) cnt[m] = 0;
  for (int i = i0; i < i1; ++i) {
    const uint32_t d = D[inv[i]];
#pragma unroll
    for (int m = 0; m < 16; ++m) cnt[m] += (d >> (2 * m)) & 1u;
  }
  // 2. exclusive prefix of the counts over threads (warp scan, then warp totals)
  int32_t pre[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    int32_t x = cnt[m];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    pre[m] = x - cnt[m];
    if (lane == 31) wsum[warp][m] = x;
  }
  __syncthreads();
  if (tid < 16) {
    int64_t tot = 0;
    for (int w = 0; w < nw; ++w) {
      const int32_t v = wsum[w][tid];
      wsum[w][tid] = (int32_t)tot;  // exclusive offset of warp w
      tot += v;
    }
    // 3. the drawn vertex of pair m: the (u mod D)-th differing one
    if (tot > 0) {
      const uint4 u = philox10(make_uint4((uint32_t)k, (uint32_t)round, (uint32_t)tid, 3u), key);
      pick[tid] = (int64_t)((uint64_t)u.x % (uint64_t)tot);
    } else {
      pick[tid] = -1;
    }
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int64_t p = pick[m];
    const int64_t lo = (int64_t)wsum[warp][m] + pre[m];
    if (p >= lo && p < lo + cnt[m]) {
      int64_t seen = lo;
      for (int i = i0; i < i1; ++i) {
        const int v = inv[i];
        if ((D[v] >> (2 * m)) & 1u) {
          if (seen == p) {
            atomicOr(&C[v], 1u << (2 * m));
            break;
          }
          ++seen;
        }
      }
    }
  }
  __syncthreads();
  // 4. grow the clusters: a differing vertex takes the bits of its neighbours
  for (;;) {
    if (tid == 0) changed = 0;
    __syncthreads();
    bool any = false;
    for (int v = tid; v < n; v += nt) {
      const uint32_t want = D[v] & ~C[v];
      if (want == 0u) continue;
      uint32_t nb = 0u;
      for (int q = rowptr[v]; q < rowptr[v + 1]; ++q) nb |= C[col[q] & 0x7FFFFFFF];
      const uint32_t add = want & nb;
      if (add) {
        atomicOr(&C[v], add);
        any = true;
      }
    }
    if (any) changed = 1;
    __syncthreads();
    const bool more = changed != 0;
    __syncthreads();  // every thread has read `changed` before the next pass clears it
    if (!more) break;
  }
  // 5. flip the clusters in both chains; recount the word's unsatisfied bonds
  unsigned long long flips = 0;
  for (int v = tid; v < n; v += nt) {
    const uint32_t cl = C[v];
    flips += __popc(cl);
    if (cl) word[v] ^= cl | (cl << 1);
  }
  __syncthreads();  // global writes of this CTA visible to its own threads
  SlicedCounter<NP> cntu;
  cntu.clear();
  int32_t bonds = 0;
  for (int v = tid; v < n; v += nt) {
    const uint32_t s0 = word[v];
    for (int q = rowptr[v]; q < rowptr[v + 1]; ++q) {
      const int e = col[q];
      const int j = e & 0x7FFFFFFF;
      if (j <= v) continue;  // each edge once
      cntu.add_at(0, ~(s0 ^ word[j] ^ (uint32_t)(e >> 31)));
      ++bonds;
    }
    if (field) {
      // h s = +|h| or -|h|: |h| bonds, unsatisfied where h s = +|h|
      const int32_t hv = field[v];
      const int32_t ha = hv > 0 ? hv : -hv;
      const uint32_t f = hv > 0 ? s0 : ~s0;
#pragma unroll
      for (int b = 0; b < 6; ++b)
        if ((ha >> b) & 1) cntu.add_at(b, f);
      bonds += ha;
    }
  }
  const int32_t tot = cntu.warp_lane_total();
  const int32_t wb = __reduce_add_sync(0xFFFFFFFFu, bonds);
  __shared__ int32_t lane_tot[32];
  __shared__ int32_t bond_tot;
  if (tid < 32) lane_tot[tid] = 0;
  if (tid == 0) bond_tot = 0;
  __syncthreads();
  atomicAdd(&lane_tot[lane], tot);
  if (lane == 0) atomicAdd(&bond_tot, wb);
  for (int o = 16; o > 0; o >>= 1) flips += __shfl_down_sync(0xFFFFFFFFu, flips, o);
  if (lane == 0 && flips) atomicAdd(&flipped[k], flips);
  __syncthreads();
  if (tid < 32) e_cur[32 * k + tid] = 2 * lane_tot[tid] - bond_tot;  // E = 2 U - bonds
}

}  // namespace

size_t pt_cluster_graph_smem(int32_t n) { return 12 * (size_t)n; }

cudaError_t pt_cluster_graph(uint32_t *spins, int32_t *e_cur, int32_t n, const int32_t *rowptr,
                             const int32_t *col, const int32_t *orig, const int32_t *field,
                             int32_t kmax, int32_t k0, int32_t slots, int32_t round,
                             uint32_t key0, uint32_t key1, unsigned long long *flipped,
                             cudaStream_t stream) {
  if (slots <= 0) return cudaSuccess;
  const int threads = 1024;
  const size_t smem = pt_cluster_graph_smem(n);
  // a thread's unsatisfied-bond count: (vertices per thread) x (degree + |h|) <= kmax each
  const int64_t per_thread = (int64_t)((n + threads - 1) / threads) * (kmax > 0 ? kmax : 1);
  cudaError_t err;
  if (per_thread < (1 << 10)) {
    err = cudaFuncSetAttribute(pt_cluster_graph_kernel<10>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err == cudaSuccess)
      pt_cluster_graph_kernel<10><<<slots, threads, smem, stream>>>(
          spins, e_cur, n, rowptr, col, orig, field, k0, round, PhiloxKey{key0, key1}, flipped);
  } else if (per_thread < (1 << 14)) {
    err = cudaFuncSetAttribute(pt_cluster_graph_kernel<14>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err == cudaSuccess)
      pt_cluster_graph_kernel<14><<<slots, threads, smem, stream>>>(
          spins, e_cur, n, rowptr, col, orig, field, k0, round, PhiloxKey{key0, key1}, flipped);
  } else {
    return cudaErrorInvalidValue;
  }
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

cudaError_t pt_cluster(uint32_t *spins, int32_t *e_cur, const uint8_t *cbits, int32_t L,
                       int32_t W, int32_t k0, int32_t slots, int32_t round, uint32_t key0,
                       uint32_t key1, unsigned long long *flipped, cudaStream_t stream) {
  if (slots <= 0) return cudaSuccess;
  const int threads = 1024;
  const size_t smem = 8 * (size_t)L * W + 8 * (size_t)((L + 31) / 32 + (W + 31) / 32);
  const int per_thread = (L * W + threads - 1) / threads;  // sites per thread, 2 bonds each
  cudaError_t err;
  if (2 * per_thread < (1 << 6)) {
    err = cudaFuncSetAttribute(pt_cluster_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (err == cudaSuccess)
      pt_cluster_kernel<6><<<slots, threads, smem, stream>>>(spins, e_cur, cbits, L, W, k0, round,
                                                             PhiloxKey{key0, key1}, flipped);
  } else {
    err = cudaFuncSetAttribute(pt_cluster_kernel<10>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (err == cudaSuccess)
      pt_cluster_kernel<10><<<slots, threads, smem, stream>>>(spins, e_cur, cbits, L, W, k0,
                                                              round, PhiloxKey{key0, key1},
                                                              flipped);
  }
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

cudaError_t pt_exchange_quads(uint32_t *quads, int32_t *e_cur, int32_t n, int32_t K,
                              int32_t parity, int32_t round, uint32_t key0, uint32_t key1,
                              const int8_t *sgn, const uint32_t *xtable, int32_t xlen,
                              unsigned long long *accepted, cudaStream_t stream) {
  const int pairs = (K - parity) / 2;
  if (pairs <= 0) return cudaSuccess;
  pt_exchange_quads_kernel<<<pairs, 256, 0, stream>>>(quads, e_cur, n, K, parity, round,
                                                       PhiloxKey{key0, key1}, sgn, xtable, xlen,
                                                       accepted);
  return cudaGetLastError();
}

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
