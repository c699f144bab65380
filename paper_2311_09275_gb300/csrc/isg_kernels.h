// isg_kernels.h -- interface between the host runtime (isg_runtime.cu) and
// the annealing kernels (torus_msc.cu, csr_sweep.cu, aux_kernels.cu).
// Plain structs of device pointers and sizes; no host-side logic here.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace isg {

// The ten Philox4x32-10 round keys of a seed: the key words advanced by the
// two Weyl increments before every round after the first.
struct RoundKeys {
  uint32_t k0[10], k1[10];
};

__host__ __device__ inline RoundKeys round_keys(uint32_t key0, uint32_t key1) {
  RoundKeys r;
  for (int i = 0; i < 10; ++i) {
    r.k0[i] = key0 + (uint32_t)i * 0x9E3779B9u;
    r.k1[i] = key1 + (uint32_t)i * 0xBB67AE85u;
  }
  return r;
}

// ---------------------------------------------------------------- torus, multi-spin coded
// One replica word = 32 replicas packed bitwise (bit l of a word is replica
// 32*word + l; bit 1 means spin +1).  State arrays are [word][L*W].
struct TorusSolve {
  int32_t L, W;
  const uint8_t *cbits;      // [L*W] bit0: j_right == -1, bit1: j_down == -1
  const uint32_t *table;     // thresholds for energy changes 4 and 8 of word w, sweep t at
                             // table[w * table_ws + t * table_ts + {0, 1}]
  int32_t table_ws, table_ts;  // annealing: 0, 2 (one schedule); tempering: 2, 0 (one beta per word)
  uint32_t key0, key1;       // Philox key (seed)
  RoundKeys rk;              // round_keys(key0, key1)
  int32_t words;             // replica words of this solve
  int32_t replicas;          // R (lanes >= R of the last word are padding)
  int32_t rng_word0;         // global replica word of word 0 (its Philox counters)
  uint32_t *spins;           // [words][L*W] state in/out
  uint32_t *best;            // [words][L*W]
  int32_t *e_cur;            // [words*32]
  int32_t *e_best;           // [words*32]
  int32_t *hit;              // [words] first sweep whose end met the target, else -1
  int32_t *done;             // [words] sweeps completed
  int32_t has_target;
  int32_t target;
};

struct TorusLaunch {
  int32_t t_begin, t_end;    // sweeps run by this launch
  int32_t resume;            // 0: start from the initial (Philox) state
  int32_t stop_from_hits;    // 1: end at min over words of hit[] + 1 (second pass)
  int32_t cluster;           // CTAs per replica word (band split of the rows)
  int32_t threads;
  // software-pipelined build only: the acceptance masks of the sweeps
  // [t_begin, t_begin + pre_count), precomputed by torus_mask_launch, at
  // pre_tab[t - t_begin][word][2][L*W] (nullptr: all drawn)
  const uint32_t *pre_tab;
  int32_t pre_count;
};

// Dynamic shared memory one CTA needs for a torus solve split over `cluster` CTAs.
size_t torus_smem_bytes(int32_t L, int32_t W, int32_t cluster);
// Whether torus_launch runs the software-pipelined build for this shape (the
// one that reads TorusLaunch::pre_tab; the others draw every mask).
bool torus_pipelined(int32_t L, int32_t W, int32_t cluster, int32_t threads);
// Masks of the sweeps [a, a + count) of every word of the solve into out_dev
// ([count][words][2][L*W] uint32, the layout TorusLaunch::pre_tab reads).
cudaError_t torus_mask_launch(const TorusSolve &s, int32_t a, int32_t count, uint32_t *out_dev,
                              cudaStream_t stream);
// Largest number of sites a thread updates per sweep under this launch shape.
int32_t torus_sites_per_thread(int32_t L, int32_t W, int32_t cluster, int32_t threads);
cudaError_t torus_launch(const TorusSolve &s, const TorusLaunch &l, cudaStream_t stream);
// Clusters of this shape the device can hold at once (0: the shape cannot launch).
int torus_max_active_clusters(int32_t L, int32_t W, int32_t words, int32_t cluster,
                              int32_t threads);

// Work units of the persistent kernels: one replica word of one torus, run by
// one CTA over sweeps [t_begin, t_end).  Used by the batched and served forms.
struct TorusBatchItem {
  TorusSolve solve;
  int32_t word;
  int32_t t_begin, t_end;
  int32_t resume;
  int32_t stop_from_hits;    // second pass of a multi-unit solve with a target: run from the
                             // start to (min over the solve's units of hit) + 1, nothing if
                             // no unit reached the target
  int8_t *out;               // (unused by the kernels)
  int8_t *out_best;
  int32_t *stop;
};
// count_dev: number of units; order_dev: unit indices, longest first;
// next_dev: zeroed work counter.
cudaError_t torus_batch_launch(const TorusBatchItem *items_dev, const int32_t *count_dev,
                               const int32_t *order_dev, int32_t *next_dev, int32_t ctas,
                               int32_t threads, size_t smem, cudaStream_t stream);
size_t torus_batch_max_smem(int32_t L, int32_t W);

// ---------------------------------------------------------------- CSR colour classes
// Vertices relabelled colour-major (class 0 first, ascending original id in a
// class).  Spins are int8 packed four replicas per uint32 ("quad"), state
// arrays [quad][n] in relabelled order.
struct CsrSolve {
  int32_t n;
  int32_t n_colours;
  const int32_t *class_start;  // [n_colours + 1] (relabelled ids)
  const int32_t *rowptr;       // [n + 1]
  const int32_t *col;          // [nnz] relabelled neighbour ids
  const int32_t *wt;           // [nnz]
  const int32_t *orig;         // [n] original id of each relabelled vertex
  const int32_t *field;        // [n] local fields h (relabelled order), or nullptr
  int32_t kmax;                // max_i (sum_j |w_ij| + |h_i|)
  const uint32_t *table;       // [sweeps][kmax + 1]; with slot_quads: [slots][kmax + 1]
  int32_t slot_quads;          // 0: annealing (row t for sweep t); > 0: parallel tempering,
                               // quad q at slot q / slot_quads, row slot every sweep
  uint32_t key0, key1;
  int32_t quads;               // ceil(R / 4)
  int32_t replicas;
  int32_t rng_quad0;           // global replica quad of quad 0 (its Philox counters)
  uint32_t *spins;             // [quads][n]
  uint32_t *best;              // [quads][n]
  int32_t *e_cur;              // [quads*4]
  int32_t *e_best;             // [quads*4]
  int32_t *hit;                // [quads]
  int32_t *done;               // [quads]
  int32_t has_target;
  int32_t target;
  int32_t mode;                // weights: 0 all +1, 1 all +-1 (col bit 31 = -1), 2 general
};

struct CsrLaunch {
  int32_t t_begin, t_end;
  int32_t resume;
  int32_t stop_from_hits;
  int32_t cluster;             // CTAs sharing one quad (each holds a full copy)
  int32_t threads;
  int32_t quads_per_cta;       // replica quads one CTA carries (1 or 2)
  int32_t own_n, own_nnz;      // largest owned slice of any rank; 0 = adjacency not staged
};

// Threshold entries cached in shared memory per sweep (larger tables are read
// from global memory).
constexpr int kCsrTableCache = 256;

size_t csr_smem_bytes(int32_t n, int32_t quads_per_cta, int32_t cluster, int32_t n_colours,
                      int32_t own_n, int32_t own_nnz, int32_t mode, int32_t kmax);
cudaError_t csr_launch(const CsrSolve &s, const CsrLaunch &l, cudaStream_t stream);

// Work unit: one replica quad of one instance, one CTA, sweeps [t_begin, t_end).
struct CsrBatchItem {
  CsrSolve solve;
  int32_t quad;
  int32_t t_begin, t_end;
  int32_t resume;
  int32_t stop_from_hits;      // as TorusBatchItem::stop_from_hits
};
cudaError_t csr_batch_launch(const CsrBatchItem *items_dev, const int32_t *count_dev,
                             const int32_t *order_dev, int32_t *next_dev, int32_t ctas,
                             int32_t threads, size_t smem, cudaStream_t stream);

// ---------------------------------------------------------------- graphs, multi-spin coded
// +-1-weighted graphs (all weights +1 when there are local fields) with
// degree + |h| <= 63: replica words like the torus kernel, vertices
// relabelled colour-major like the colour-class kernel.  State arrays are
// [word][n] in relabelled order.
struct GraphMscSolve {
  int32_t n;
  int32_t n_colours;
  const int32_t *class_start;  // [n_colours + 1]
  const int32_t *rowptr;       // [n + 1]
  const int32_t *col;          // relabelled neighbour ids, bit 31 set for weight -1
  const int32_t *orig;         // [n]
  const int32_t *field;        // [n] local fields h (relabelled order), or nullptr
  const uint32_t *table;       // thresholds by half energy change k of word w, sweep t at
                               // table[w * table_ws + t * table_ts + k]
  int32_t table_ws, table_ts;  // annealing: 0, kmax1; tempering: kmax1, 0
  int32_t kmax1;               // kmax + 1 (<= 64)
  uint32_t key0, key1;
  RoundKeys rk;
  int32_t words;
  int32_t replicas;
  int32_t rng_word0;           // global replica word of word 0 (its Philox counters)
  uint32_t *spins;             // [words][n]
  uint32_t *best;              // [words][n]
  int32_t *e_cur;              // [words*32]
  int32_t *e_best;             // [words*32]
  int32_t *hit;                // [words]
  int32_t *done;               // [words]
  int32_t has_target;
  int32_t target;
};

struct GraphMscLaunch {
  int32_t t_begin, t_end;
  int32_t resume;
  int32_t stop_from_hits;
  int32_t cluster;             // CTAs sharing one word (each holds a full copy)
  int32_t threads;
  int32_t own_n, own_nnz;      // largest owned slice of any rank; 0 = adjacency not staged
  int32_t own_lv;              // staged: largest owned sum of threshold levels (d + |h| + 1) / 2
  int32_t planes;              // bit planes of the energy counters (6..14)
  // staged: acceptance masks of sweeps [gmask_t0, t_end) precomputed by
  // gm_mask_launch ([sweep - gmask_t0][word][gmask_gl] words, vertex v's at
  // gloff[v]), or nullptr to build them in the kernel
  const uint32_t *gmask;
  const int32_t *gloff;        // [n + 1] prefix of the levels in relabelled order
  int64_t gmask_gl;            // gloff[n]
  int32_t gmask_t0;
};

// Bit planes of the persistent unit kernel's energy counters: a unit's
// (vertices per thread per sweep) x (max degree) must stay below 2^12.
constexpr int kGraphMscBatchPlanes = 12;

struct GraphMscItem {
  GraphMscSolve solve;
  int32_t word;
  int32_t t_begin, t_end;
  int32_t resume;
  int32_t stop_from_hits;      // as TorusBatchItem::stop_from_hits
};

// fields: the instance has local fields (staged slices then hold them too);
// own_lv sizes the staged kernel's mask table (0 when not staged).
size_t gm_smem_bytes(int32_t n, int32_t cluster, int32_t n_colours, int32_t own_n,
                     int32_t own_nnz, int32_t own_lv, int32_t kmax1, bool fields);
// Smallest supported plane count holding counts up to max_count (-1: none).
int gm_planes(int32_t max_count);
cudaError_t gm_launch(const GraphMscSolve &s, const GraphMscLaunch &l, cudaStream_t stream);
// Acceptance masks of sweeps [t0, t0 + nt) of every word of the solve into
// out_dev ([nt][words][gl] uint32, the layout GraphMscLaunch::gmask reads).
cudaError_t gm_mask_launch(const GraphMscSolve &s, const int32_t *gloff_dev, int64_t gl, int32_t t0,
                           int32_t nt, uint32_t *out_dev, cudaStream_t stream);
cudaError_t gm_batch_launch(const GraphMscItem *items_dev, const int32_t *count_dev,
                            const int32_t *order_dev, int32_t *next_dev, int32_t ctas,
                            int32_t threads, size_t smem, cudaStream_t stream);

// ---------------------------------------------------------------- auxiliary kernels
// Unpack words [words][n] in relabelled order into int8 [R][n] caller order.
cudaError_t unpack_msc_relabel(const uint32_t *words, int32_t n, int32_t R, const int32_t *orig,
                               int8_t *out, cudaStream_t stream);
// Unpack multi-spin words [words][n] into int8 [R][n] (+1/-1).
cudaError_t unpack_msc(const uint32_t *words, int32_t n, int32_t R, int8_t *out,
                       cudaStream_t stream);
// Unpack quads [quads][n] (relabelled order) into int8 [R][n] original order.
cudaError_t unpack_quads(const uint32_t *quads, int32_t n, int32_t R, const int32_t *orig,
                         int8_t *out, cudaStream_t stream);
// Energies of R configurations spins[R][n] (int8) over a CSR (original ids):
// per-block partial sums in scratch[R * blocks], then one sum per replica.
// Parallel tempering: exchange configurations between replica words k and
// k+1 (k = parity, parity + 2, ...; k + 1 < K), lane by lane, after round
// `round`.  sgn[k] = sign of beta_k - beta_{k+1}; xtable[k][d] = threshold of
// an exchange whose energy difference |E_k - E_{k+1}| = d < xlen raises the
// exponent's magnitude (0 beyond xlen); accepted[k] counts exchanges.
cudaError_t pt_exchange(uint32_t *spins, int32_t *e_cur, int32_t n, int32_t K, int32_t parity,
                        int32_t round, uint32_t key0, uint32_t key1, const int8_t *sgn,
                        const uint32_t *xtable, int32_t xlen, unsigned long long *accepted,
                        cudaStream_t stream);

// Parallel tempering: one Houdayer cluster move per chain pair (lanes 2m,
// 2m+1) on slot words k0 .. k0+slots-1 of an L x W torus state; flipped[k]
// gains the cluster sizes.  Needs 8 L W bytes of shared memory per CTA.
// Parallel tempering on int8 quad state (slot k = quads 8k .. 8k+7, chain c in
// byte c mod 4 of quad 8k + c / 4): the exchange step of pt_exchange.
cudaError_t pt_exchange_quads(uint32_t *quads, int32_t *e_cur, int32_t n, int32_t K,
                              int32_t parity, int32_t round, uint32_t key0, uint32_t key1,
                              const int8_t *sgn, const uint32_t *xtable, int32_t xlen,
                              unsigned long long *accepted, cudaStream_t stream);

// Parallel tempering on a graph (multi-spin graph layout): one Houdayer move per
// chain pair on slot words k0 .. k0+slots-1; needs pt_cluster_graph_smem(n)
// bytes of shared memory per CTA (kmax: the instance's max degree + |h|).
size_t pt_cluster_graph_smem(int32_t n);
cudaError_t pt_cluster_graph(uint32_t *spins, int32_t *e_cur, int32_t n, const int32_t *rowptr,
                             const int32_t *col, const int32_t *orig, const int32_t *field,
                             int32_t kmax, int32_t k0, int32_t slots, int32_t round,
                             uint32_t key0, uint32_t key1, unsigned long long *flipped,
                             cudaStream_t stream);
cudaError_t pt_cluster(uint32_t *spins, int32_t *e_cur, const uint8_t *cbits, int32_t L,
                       int32_t W, int32_t k0, int32_t slots, int32_t round, uint32_t key0,
                       uint32_t key1, unsigned long long *flipped, cudaStream_t stream);

cudaError_t energy_csr(const int64_t *rowptr, const int32_t *col, const int32_t *wt, int32_t n,
                       const int8_t *spins, int32_t R, int64_t *scratch, int32_t blocks,
                       int64_t *energies, cudaStream_t stream,
                       const int32_t *field = nullptr);
// One solve of a batch for the unpack: its state [units][n] (words of 32
// lanes or quads of 4), relabelled graphs' original ids (nullptr for a
// torus), per-unit hit sweeps, and where its int8 [R][n] states and stop go.
struct BatchOutDesc {
  const uint32_t *spins, *best;
  const int32_t *orig;
  const int32_t *hit;
  int32_t n, R, lanes, units, has_target;
  int8_t *out, *out_best;
  int32_t *stop;               // min over units of hit (-1: none or no target)
};
// Unpack every solve of a batch (one launch): final and best states into
// int8 [R][n] in the caller's vertex order, and the stop sweep.
cudaError_t batch_unpack(const BatchOutDesc *descs_dev, int32_t count, int64_t max_nr,
                         cudaStream_t stream);
// Reduce per-word / per-quad hit sweeps to the solve's stop sweep.
cudaError_t reduce_hits(const int32_t *hit, int32_t count, int32_t *out, cudaStream_t stream);

}  // namespace isg
