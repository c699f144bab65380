/*
 * isg_oracle.h -- plain, slow CPU oracle for the replica-parallel Metropolis
 * annealing sweep over sparse Ising / MaxCut instances.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load or call this code.  The product (the
 * CUDA library and its Python binding) never does, and shares no code with it.
 *
 * Problem (paper Sec. I and Sec. II.A): binary spins s_i in {-1,+1}, pairwise
 * integer couplings w_ij on a sparse graph; MaxCut value
 * cut(s) = sum_{(i,j)} w_ij (1 - s_i s_j) / 2.  The oracle minimises
 * E(s) = sum_{(i,j)} w_ij s_i s_j, so cut = (W_tot - E) / 2.  Optional integer
 * local fields h_i (the sparse QUBO and independent-set forms of Sec. I and
 * Sec. II.C, which lack spin-reversal symmetry) add sum_i h_i s_i to E; every
 * `field` argument below may be NULL for none.
 *
 * Method: the paper's own heuristic ("Cosm", Sec. III.A) is undisclosed; it is
 * iterative and counts its work in sweeps.  The computation reproduced here is
 * single-spin-flip Metropolis simulated annealing in colour-class order, the
 * sweep that heuristics of this class spend their time in.
 */
#ifndef ISG_ORACLE_H
#define ISG_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11).  out = Philox(ctr, key). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Symmetric CSR of an undirected edge list; neighbours sorted ascending.
 * rowptr has n+1 entries, col/wt have 2m.  Returns 0, or -1 on a bad edge
 * (out of range or self-loop) or a duplicate pair. */
int orc_build_csr(int32_t n, int64_t m, const int32_t *u, const int32_t *v, const int32_t *w,
                  int64_t *rowptr, int32_t *col, int32_t *wt);

/* Edge list of an L x W torus: vertex i = r*W + c; for each i (ascending) the
 * edge to (r, c+1 mod W) with weight j_right[i], then the edge to
 * (r+1 mod L, c) with weight j_down[i].  u, v, w have 2*L*W entries. */
void orc_torus_edges(int32_t L, int32_t W, const int8_t *j_right, const int8_t *j_down,
                     int32_t *u, int32_t *v, int32_t *w);

/* Greedy colouring by ascending vertex id: colour[v] is the smallest c >= 0
 * not used by a neighbour u < v.  Returns the number of colours. */
int32_t orc_greedy_colouring(int32_t n, const int64_t *rowptr, const int32_t *col, int32_t *colour);

/* Smallest-last colouring (Matula and Beck, J. ACM 30(3), 1983), the colour
 * classes of the sweep on graphs: repeatedly remove, from the graph that is
 * left, a vertex of smallest remaining degree (the smallest id among ties);
 * colour the vertices in the reverse of that removal order, each with the
 * smallest c >= 0 that no already coloured neighbour has; then number the
 * classes in increasing order of their smallest vertex.  At most degeneracy + 1
 * colours.  Returns the number of colours. */
int32_t orc_smallest_last_colouring(int32_t n, const int64_t *rowptr, const int32_t *col,
                                    int32_t *colour);

/* Acceptance thresholds: table[t*(kmax+1) + k] = min(floor(2^32 exp(-beta_t * 2k)), 2^32-1)
 * for k = 0..kmax (energy increase d = 2k), in FP64. */
void orc_accept_table(int32_t sweeps, const double *betas, int32_t kmax, uint32_t *table);

/* E(s) = sum over edges w_ij s_i s_j + sum_i h_i s_i for one configuration
 * s[0..n-1] (+/-1). */
int64_t orc_energy(int32_t n, const int64_t *rowptr, const int32_t *col, const int32_t *wt,
                   const int32_t *field, const int8_t *s);

/* Metropolis annealing, one independent chain per listed replica.
 *
 * Inputs: CSR (rowptr, col, wt), fields (or NULL; the local field of vertex i
 * is h_i + sum_j w_ij s_j), colour[n] (classes 0..n_colours-1), the
 * replica indices to run (rep_ids[0..n_rep-1], each < 2^31), sweeps S,
 * betas[S], seed, optional target (has_target != 0), shuffle_seed (0 = sites
 * of a class in ascending id; otherwise a seeded shuffle of each class, which
 * must not change any result), check_energy (recompute E after every sweep
 * and fail on a mismatch with the tracked value), nthreads.
 *
 * Outputs per listed replica k (row-major [n_rep][n] spins in vertex order):
 * s_final, e_final, s_best, e_best; plus hit_sweep (first sweep t at whose end
 * min_k e_best <= target, else -1) and sweeps_done.  With a target every
 * replica of the solve must be listed.  Returns 0, -1 on bad arguments, -2 on
 * an energy-tracking mismatch. */
int orc_anneal(int32_t n, const int64_t *rowptr, const int32_t *col, const int32_t *wt,
               const int32_t *field, const int32_t *colour, int32_t n_colours,
               int32_t n_rep, const int32_t *rep_ids, int32_t sweeps, const double *betas,
               uint64_t seed, int has_target, int64_t target, uint64_t shuffle_seed,
               int check_energy, int nthreads,
               int8_t *s_final, int32_t *e_final, int8_t *s_best, int32_t *e_best,
               int32_t *hit_sweep, int32_t *sweeps_done);

/* Parallel tempering over K temperature slots x 32 independent chains
 * (replica r = 32 k + c at betas[k]): `rounds` rounds of `per_round` sweeps
 * each, every round followed by configuration exchanges between slot pairs
 * (k, k+1), k = round mod 2, accepted with probability
 * min(1, exp((beta_k - beta_{k+1}) (E_k - E_{k+1}))) by the exchange uniform
 * (tag 2, counter (k, round, c / 4, 2), word c mod 4) against
 * floor(2^32 exp(.)).  Outputs per replica ([32K][n] spins): s_final, e_final,
 * s_best, e_best (best states stay with the slot, checked at sweep ends);
 * accepted[k] / attempted[k] exchange counts of pair (k, k+1), k < K-1.
 * With icm_slots > 0, every round's sweeps are followed (before the
 * exchanges) by one Houdayer cluster move per chain pair (2m, 2m+1), m < 16,
 * on each of the last icm_slots slots: a site where the two differ is drawn
 * (the (u mod D)-th in vertex order, u word 0 of Philox(seed, (k, round, m,
 * 3)), D the number of such sites), its connected component among the
 * differing sites is flipped in both chains, and their energies are
 * recomputed; flipped[k] sums the cluster sizes of slot k.
 * Returns 0, or -1 on bad arguments. */
int orc_parallel_tempering(int32_t n, const int64_t *rowptr, const int32_t *col, const int32_t *wt,
                           const int32_t *field, const int32_t *colour, int32_t n_colours,
                           int32_t K, const double *betas, int32_t rounds, int32_t per_round,
                           int32_t icm_slots, uint64_t seed, int nthreads, int8_t *s_final,
                           int32_t *e_final, int8_t *s_best, int32_t *e_best, int64_t *accepted,
                           int64_t *attempted, int64_t *flipped);

/* Initial spins of the listed replicas (the state before sweep 0). */
void orc_initial_spins(int32_t n, int32_t n_rep, const int32_t *rep_ids, uint64_t seed, int8_t *s);

/* Exhaustive enumeration over all 2^n states (n <= 30) in Gray-code order.
 * Returns the minimum energy; writes one minimising state to argmin (if not
 * NULL) and, if hist is not NULL, the number of states with energy
 * E = e_lo + k into hist[k] for k = 0..(e_hi - e_lo) where
 * e_lo = -(sum|w| + sum|h|), e_hi = -e_lo. */
int64_t orc_enumerate(int32_t n, const int64_t *rowptr, const int32_t *col, const int32_t *wt,
                      const int32_t *field, int8_t *argmin, uint64_t *hist);

#ifdef __cplusplus
}
#endif
#endif
