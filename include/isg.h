/*
 * isg.h -- C ABI of libisg: replica-parallel Metropolis annealing of sparse
 * Ising / MaxCut instances on one NVIDIA GB300 (sm_103a).
 *
 * Problem (paper Sec. I, Sec. II.A and Table I): n binary spins s_i in {-1,+1}
 * with integer pairwise couplings w_ij on a sparse graph -- a toroidal square
 * grid with +-1 couplings (the 2D Edwards-Anderson spin glass form of the Gset
 * torus instances) or an arbitrary sparse graph (e.g. unweighted MaxCut on a
 * random graph, like G70).  The library minimises
 *
 *     E(s) = sum_{edges (i,j)} w_ij s_i s_j ,
 *
 * so the MaxCut value of Sec. II.A is cut(s) = (W_tot - E(s)) / 2 with
 * W_tot = sum w_ij (returned by isg_problem_info).
 *
 * Method.  The paper's heuristic is iterative, counts its work in sweeps and
 * withholds its details (Sec. III.A).  The library runs the computation such
 * heuristics spend their time in: simulated annealing by single-spin-flip
 * Metropolis sweeps over R independent replicas.  Sweep t (0-based) visits
 * the colour classes in ascending order (torus: colour (r + c) mod 2; graphs:
 * greedy colouring by ascending vertex id, or the smallest-last colouring
 * selected by isg_problem_set_colouring) and, for every vertex i of the
 * class and every replica, computes h_i = sum_j w_ij s_j and the energy change
 * d = -2 s_i h_i of flipping s_i; the flip is taken when d <= 0, or when
 * u < floor(2^32 exp(-beta_t d)) for the replica's 32-bit uniform u.  The
 * uniform of replica r at vertex i in sweep t is word (r mod 4) of
 * Philox4x32-10(key = (seed mod 2^32, seed >> 32), counter = (i, t, r / 4, 0))
 * (Salmon et al., SC'11); initial spins are s_i = +1 iff the top bit of word
 * (r mod 4) of Philox4x32-10(key, (i, 0, r / 4, 1)) is set.  i is the vertex
 * id as given by the caller.  Energies are tracked incrementally; each
 * replica's best state is checked at the end of every sweep (strictly lower
 * energy replaces it; the initial state is the first candidate).
 * Results are a pure function of (instance, replicas, betas, seed): they do
 * not depend on the kernel chosen, its blocking, the batch a solve is in, or
 * whether the schedule ran in one call or was continued or restarted from a
 * checkpoint (isg_anneal_continue, isg_anneal_resume).
 *
 * Conventions.
 *  - All input arrays are caller-owned HOST memory and are copied; the caller
 *    may free them when the call returns.  Handles are library-owned and are
 *    released with the matching *_destroy call.
 *  - Spins cross the boundary as int8 +1/-1, row-major [replica][vertex] in
 *    the caller's vertex order.
 *  - Every call returns a status and never aborts the process; on failure the
 *    calling thread's message is available from isg_last_error().
 *  - Device work runs on the current CUDA device at the time of the call, on
 *    the given stream (NULL = the legacy default stream).  Calls that return
 *    results to the host synchronise with that work.
 */
#ifndef ISG_H
#define ISG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ISG_OK = 0,
    ISG_EINVAL = 1,      /* invalid argument or instance */
    ISG_ENOMEM = 2,      /* host or device allocation failed */
    ISG_ECUDA = 3,       /* a CUDA call failed (no device, launch error, ...) */
    ISG_ETIMEOUT = 4,    /* nothing ready within the requested time */
    ISG_EBUSY = 5,       /* resource limit reached (server slots, memory budget) */
    ISG_ECANCELLED = 6   /* the request was cancelled or the server stopped */
} isg_status;

typedef struct isg_problem isg_problem;
typedef struct isg_result isg_result;
typedef struct isg_server isg_server;

/* Sentinel for "no target energy". */
#define ISG_NO_TARGET INT64_MIN

/* ---------------------------------------------------------------- problems */

/* Instance from an undirected edge list (paper Sec. II.A: weighted MaxCut /
 * Ising form).  n >= 1 vertices; m >= 0 edges (u[e], v[e]) with weight w[e].
 * EINVAL: an endpoint outside [0, n), a self-loop, a repeated pair, or
 * sum |w| >= 2^30 (energies are exact int32).  Zero weights are allowed. */
isg_status isg_problem_create_edges(int32_t n, int64_t m, const int32_t *u, const int32_t *v,
                                    const int32_t *w, isg_problem **out);

/* The same with integer local fields h[n] (NULL = none): the energy becomes
 * E(s) = sum_(i,j) w_ij s_i s_j + sum_i h_i s_i, the form of sparse QUBO and of
 * independent-set problems (Sec. I; Sec. II.C notes they lack spin-reversal
 * symmetry).  A flip of i changes E by -2 s_i (h_i + sum_j w_ij s_j).  Such
 * instances run on the int8 colour-class kernel (ISG_KERNEL_CSR, PLAIN, and
 * AUTO's choice) and, when every weight is +1 and deg_i + |h_i| <= 63 for all
 * i, also on the multi-spin graph kernel (ISG_KERNEL_GRAPH_MSC, which counts
 * h_i s_i as |h_i| extra bonds; parallel tempering uses it); the torus kernel
 * rejects them.  total_weight of
 * isg_problem_info stays sum w, so the MaxCut identity cut = (W - E) / 2 does
 * not apply.  EINVAL as isg_problem_create_edges, with sum |w| + sum |h| >= 2^30
 * in place of the weight bound.  h is copied. */
isg_status isg_problem_create_fields(int32_t n, int64_t m, const int32_t *u, const int32_t *v,
                                     const int32_t *w, const int32_t *h, isg_problem **out);

/* Instance from a symmetric CSR: rowptr[n+1] (rowptr[0] = 0), col/w of
 * rowptr[n] entries; entry (i, j, w) must have its mirror (j, i, w).
 * Same validity rules as isg_problem_create_edges. */
isg_status isg_problem_create_csr(int32_t n, const int64_t *rowptr, const int32_t *col,
                                  const int32_t *w, isg_problem **out);

/* L x W toroidal square grid (paper Sec. II.A, Table I: 2n edges, degree 4).
 * Vertex i = r*W + c; j_right[i] couples i to (r, c+1 mod W) and j_down[i]
 * couples i to (r+1 mod L, c); each coupling is +1 or -1.  L and W must be
 * even (two-colour checkerboard) and >= 4 (no doubled edges). */
isg_status isg_problem_create_torus(int32_t L, int32_t W, const int8_t *j_right,
                                    const int8_t *j_down, isg_problem **out);

/* Sizes of an instance.  Any output pointer may be NULL.  n_colors is the
 * number of colour classes; colors[n] receives each vertex's class. */
isg_status isg_problem_info(const isg_problem *p, int32_t *n, int64_t *m, int64_t *total_weight,
                            int32_t *n_colors, int32_t *colors);

/* Colourings of a graph's sweep classes.  GREEDY (the default): for v = 0..n-1,
 * colour[v] = the smallest c >= 0 that no neighbour u < v has.  SMALLEST_LAST
 * (Matula and Beck, J. ACM 30(3), 1983): repeatedly remove a vertex of
 * smallest remaining degree (the smallest id among ties), colour the vertices
 * in the reverse of that removal order, each with the smallest c >= 0 that no
 * already coloured neighbour has, and number the classes in increasing order
 * of their smallest vertex; at most degeneracy + 1 classes (sparse random
 * graphs: 3 where greedy gives 5), and every class is one cluster-wide phase
 * per sweep.  Both are valid Metropolis sweep orders; they give different
 * (equally valid) chains. */
typedef enum {
    ISG_COLOURING_GREEDY = 0,
    ISG_COLOURING_SMALLEST_LAST = 1
} isg_colouring;

/* Re-colours a graph instance with `method` (an isg_colouring).  Call it before
 * the instance's first solve or submission: EBUSY once the instance holds
 * device state.  EINVAL: NULL, an unknown method, or a torus (tori keep their
 * (r + c) mod 2 checkerboard). */
isg_status isg_problem_set_colouring(isg_problem *p, int32_t method);

void isg_problem_destroy(isg_problem *p);

/* ---------------------------------------------------------------- annealing */

/* Kernel families.  AUTO picks the multi-spin-coded torus kernel for tori,
 * the multi-spin-coded graph kernel for graphs whose weights are all +1 or -1
 * (all +1 when there are local fields) and whose degree + |h| is <= 63, and
 * the int8 CSR colour-class kernel otherwise;
 * PLAIN runs one kernel launch per sweep (state kept in device memory between
 * launches), the one-instance-per-launch baseline of the batched form. */
typedef enum {
    ISG_KERNEL_AUTO = 0,
    ISG_KERNEL_TORUS_MSC = 1,
    ISG_KERNEL_CSR = 2,
    ISG_KERNEL_PLAIN = 3,
    ISG_KERNEL_GRAPH_MSC = 4
} isg_kernel;

typedef struct {
    int32_t kernel;        /* isg_kernel */
    int32_t cluster_ctas;  /* CTAs that share one replica block (1..16); 0 = tuned/default */
    int32_t threads;       /* threads per CTA (multiple of 32, <= 512; <= 1024 for the
                              torus kernel); 0 = tuned/default */
    int32_t time_kernels;  /* nonzero: time the sweep launches with CUDA events */
    int32_t quads_per_cta; /* colour-class kernel: replica quads per CTA (1, 2); 0 = tuned/default */
    int32_t first_replica; /* global index of this call's replica 0, a multiple of 32 (0 = the
                              usual): local replica j draws the random numbers of replica
                              first_replica + j, so calls at first_replica 0, R, 2R, ... on
                              any devices together equal one solve of all their replicas
                              (a replica-sharded solve; a target applies to this call's
                              replicas only).  Results stay indexed 0..R-1 locally. */
    int32_t mask_chunk;    /* multi-spin graph kernel with its adjacency in shared memory
                              (isg_stats.staged), solves without a target: the acceptance
                              masks (32 uniforms against each threshold level of a vertex)
                              are built either inside the sweep kernel (-1) or for chunks
                              of up to mask_chunk sweeps (> 0) by a second kernel, on
                              device memory and the SMs the sweep kernel leaves idle, on a
                              low-priority stream one chunk ahead of the sweep kernel,
                              when the tables of two chunks fit 1 GiB of device memory
                              (else inside the kernel).  The results are the same.
                              0 = automatic: precomputed in chunks of at most 96 MiB of
                              masks (a chunk table that stays in L2), when such a chunk
                              holds at least 64 sweeps.  EINVAL below -1. */
} isg_options;

/* Anneal R = replicas independent chains for S = sweeps sweeps at inverse
 * temperatures betas[S] (finite, >= 0) with the given seed.  With
 * target_energy != ISG_NO_TARGET the solve stops at the end of the first sweep
 * t* at which the lowest best energy over all replicas is <= target_energy;
 * the reported state is the state after sweep t*.  The work is enqueued on
 * cuda_stream; *out receives a result handle (library-owned).
 * EINVAL: R < 1, S < 1, a beta that is negative or not finite, an instance too
 * large for the chosen kernel; ECUDA: no device or a launch failed. */
isg_status isg_anneal(const isg_problem *p, int32_t replicas, const double *betas, int32_t sweeps,
                      uint64_t seed, int64_t target_energy, void *cuda_stream, isg_result **out);

/* Launch-shape autotuner.  Times the sweep kernel of this instance and
 * replica count under every admissible shape (CTAs per replica block, threads
 * per CTA) for probe_sweeps sweeps on the current device, writes the fastest
 * into *best (may be NULL) and remembers it, so that later solves of the same
 * (instance shape, replicas) with cluster_ctas = threads = 0 use it.  Results
 * never depend on the shape.  Synchronises the stream.  probe_sweeps >= 1. */
isg_status isg_autotune(const isg_problem *p, int32_t replicas, int32_t probe_sweeps,
                        void *cuda_stream, isg_options *best);

/* isg_anneal with explicit kernel options (opts may be NULL = defaults). */
isg_status isg_anneal_ex(const isg_problem *p, int32_t replicas, const double *betas,
                         int32_t sweeps, uint64_t seed, int64_t target_energy,
                         const isg_options *opts, void *cuda_stream, isg_result **out);

/* Resume a finished solve (checkpoint/resume in one process): run `sweeps`
 * more sweeps at betas[0..sweeps-1] from the state the solve ended with, as
 * sweeps S .. S + sweeps - 1 of one schedule (S = the sweeps run so far).  The
 * random numbers are keyed by sweep index, so the result then equals, bit for
 * bit, isg_anneal of the concatenated schedule with the same seed: final and
 * best states, energies and sweeps done.  Same kernel and launch shape as the
 * solve.  result must come from isg_anneal / isg_anneal_ex on problem p
 * without a target energy (p still alive); it can be continued again.
 * Enqueued on cuda_stream after the earlier sweeps have finished (this call
 * waits for them).  EINVAL for NULL, another problem, a result with a target
 * or of the batched, served or tempering forms, sweeps < 1 or a bad beta. */
isg_status isg_anneal_continue(const isg_problem *p, isg_result *result, const double *betas,
                               int32_t sweeps, void *cuda_stream);

/* Restart a solve from a checkpoint (across processes): the states a solve of
 * the same problem, replicas, seed and schedule held after sweeps_done sweeps,
 * as read with isg_result_final (spins) and isg_result_best_all (best_spins):
 * int8 [replicas][n], +1/-1, the caller's vertex order, caller-owned host
 * memory.  Runs sweeps sweeps_done .. sweeps - 1 of betas[0..sweeps-1] and
 * returns a result equal, bit for bit, to isg_anneal of the whole schedule
 * (energies are recomputed from the states; the solve's kernel and shape
 * follow opts as in isg_anneal_ex, and may differ from the first run's).  No
 * target energy.  EINVAL for NULL, 1 > sweeps_done or sweeps_done > sweeps, a
 * spin that is not +1/-1, and what isg_anneal_ex rejects. */
isg_status isg_anneal_resume(const isg_problem *p, int32_t replicas, const double *betas,
                             int32_t sweeps, uint64_t seed, int32_t sweeps_done,
                             const int8_t *spins, const int8_t *best_spins,
                             const isg_options *opts, void *cuda_stream, isg_result **out);

/* Anneal count instances (tori and graphs, uneven sizes, any mix) in one
 * launch sequence captured in a CUDA graph.  Every instance is cut into work
 * units that one CTA runs from start to finish: torus replica words (32
 * replicas), replica words of +-1 graphs without fields, and replica quads (4)
 * of other graphs; each unit kind has one persistent kernel whose CTAs take
 * units longest-first, and the kinds run concurrently.  All instances share
 * replicas, betas and sweeps; seeds[k] and targets[k] (targets may be NULL =
 * none) are per instance.  An instance with a target and several units
 * follows the stop rule of isg_anneal (its units rerun from the start to the
 * earliest unit's hit + 1 in a second pass).  outs[count] receive one result
 * handle each; every result equals isg_anneal of that instance alone, bit for
 * bit.  The launch shape (threads per CTA, CTAs per SM) is the one
 * isg_autotune_batch measured for this batch's replicas and size histogram,
 * else 256 threads and as many CTAs per SM as shared memory allows.  The
 * call enqueues its uploads and the graph on cuda_stream and waits for the
 * uploads.  EINVAL: NULL arguments, count outside [1, 65535], replicas or
 * sweeps < 1, a bad beta, a target outside int32, or an instance too large for
 * one CTA's shared memory. */
isg_status isg_anneal_batch(const isg_problem *const *probs, int32_t count, int32_t replicas,
                            const double *betas, int32_t sweeps, const uint64_t *seeds,
                            const int64_t *targets, void *cuda_stream, isg_result **outs);

/* Launch-shape autotuner of the batched form: runs the batch for probe_sweeps
 * sweeps, their inverse temperatures sampled evenly from betas[0..sweeps),
 * under every threads per CTA in {128, 192, 256, 384, 512} and CTAs per SM in
 * 1..4 that fits, and remembers the fastest for batches of the same replicas
 * and size histogram (instances per size class 2^k vertices, tori and graphs
 * apart) on this device; isg_anneal_batch then uses it.  Results never depend
 * on the shape.  threads and ctas_per_sm (either may be NULL) receive the
 * choice.  Synchronises the stream.  EINVAL as isg_anneal_batch, or
 * probe_sweeps < 1. */
isg_status isg_autotune_batch(const isg_problem *const *probs, int32_t count, int32_t replicas,
                              const double *betas, int32_t sweeps, int32_t probe_sweeps,
                              void *cuda_stream, int32_t *threads, int32_t *ctas_per_sm);

/* Parallel tempering (Sec. II.C: replicas at different temperatures that
 * exchange configurations) on any instance: a torus on the multi-spin torus
 * kernel; a graph with weights +-1 (all +1 with local fields) and
 * degree + |h| <= 63 on the multi-spin graph kernel; any other graph (general
 * integer weights, fields with other weights) on the int8 colour-class kernel
 * (slot k = quads 8k .. 8k+7).  Vertex order inside the state is the
 * library's; results come back in the caller's vertex order as everywhere
 * else.  temperatures = K slots with
 * inverse temperatures betas[K] (finite, >= 0, any order), 32 independent
 * chains per slot: R = 32 K replicas, replica r = 32 k + c is chain c at slot
 * k.  Each of `rounds` rounds runs sweeps_per_round sweeps of every replica at
 * its slot's beta (sweep t = round * sweeps_per_round + j draws the annealing
 * uniforms of replica r), then exchanges the configurations (and energies) of
 * chain c between slots k and k+1, for k = round mod 2, 2 + round mod 2, ...,
 * with probability min(1, exp((beta_k - beta_{k+1}) (E_k - E_{k+1}))): always
 * when the exponent is >= 0, else when the uniform word (c mod 4) of
 * Philox(seed, (k, round, c / 4, 2)) is below floor(2^32 exp(exponent)), FP64
 * on the host.  Best states and energies stay with the slot (checked at sweep
 * ends).  No target.  With icm_slots > 0, each round's sweeps are followed,
 * before the exchanges, by a Houdayer cluster move (Sec. II.C's replica
 * cluster moves) in each chain pair (2m, 2m+1) of the last icm_slots slots:
 * the sites where the pair differs span a subgraph; the (u mod D)-th of them
 * in vertex order (D their number, u = word 0 of Philox(seed, (k, round, m,
 * 3))) seeds the cluster, its connected component among the differing sites,
 * which both chains flip (exchanging their spins there, so E_a + E_b is
 * unchanged); the chains' energies are then recomputed.  On a graph the
 * subgraph's edges are the instance's edges and the vertex order is the
 * caller's.  The result is read
 * like isg_anneal's (R = 32 K, S = rounds * sweeps_per_round); exchange counts
 * by isg_result_exchanges, cluster sizes by isg_result_cluster_flips.  opts
 * may be NULL (kernel AUTO or the instance's kernel; cluster, threads and
 * quads_per_cta as isg_anneal).  EINVAL: K outside [1, 4096], rounds or
 * sweeps_per_round < 1, a bad beta, icm_slots outside [0, K], icm_slots > 0
 * on an instance of the int8 kernel, on a torus with n > 28,544 or on a graph
 * with n > 19,029 (the sites' difference and cluster bits in shared memory). */
isg_status isg_parallel_tempering(const isg_problem *p, int32_t temperatures,
                                  const double *betas, int32_t rounds, int32_t sweeps_per_round,
                                  int32_t icm_slots, uint64_t seed, const isg_options *opts,
                                  void *cuda_stream, isg_result **out);

/* Sizes of the cluster moves of a parallel-tempering result: flipped[k] =
 * sites flipped per chain of a pair, summed over pairs and rounds, for each of
 * the `temperatures` slots.  EINVAL for another slot count.  Waits. */
isg_status isg_result_cluster_flips(const isg_result *r, int64_t *flipped, int32_t temperatures);

/* Exchange counts of a parallel-tempering result: accepted[k] and attempted[k]
 * for slot pairs (k, k+1), k < pairs = K - 1 (EINVAL for another pairs value,
 * and for results of other calls unless pairs = 0).  Waits for the solve. */
isg_status isg_result_exchanges(const isg_result *r, int64_t *accepted, int64_t *attempted,
                                int32_t pairs);

/* Energies E(s) of R host configurations spins[R][n] (+-1) into energies[R],
 * computed on the device (a check of the tracked energies); local fields
 * included. */
isg_status isg_energy(const isg_problem *p, const int8_t *spins, int32_t replicas,
                      int64_t *energies);

/* isg_energy for callers that cannot allocate device memory when they call it
 * (a process whose device memory is fully reserved by another allocator, or a
 * latency-critical loop that must stay out of the driver's allocator).  No
 * counterpart in the paper: this is a library convenience.
 * All arguments are DEVICE pointers owned by the caller: a symmetric CSR in
 * the caller's vertex ids (rowptr_dev[n+1] int64, col_dev/w_dev[rowptr[n]];
 * couplings only: local fields are not part of this energy),
 * spins_dev[replicas][n] int8 +-1, and energies_dev[replicas] int64 (output).
 * The work is enqueued on cuda_stream (NULL = legacy default stream) and
 * nothing is allocated or freed: per-block partial sums live in a fixed
 * 512 KiB array inside the library that every device loading the library
 * keeps until the process exits.  replicas must be in [1, 2048] (EINVAL
 * otherwise).  The first call on a device looks up that array's device
 * address and keeps it for the life of the process (it assumes the device's
 * primary context is not reset meanwhile); make that first call before any
 * stream capture.  All calls share the array, so
 * calls whose work overlaps on the GPU (different streams, no ordering) race
 * and give wrong energies; calls ordered on one stream are fine. */
isg_status isg_energy_noalloc(int32_t n, const int64_t *rowptr_dev, const int32_t *col_dev,
                              const int32_t *w_dev, const int8_t *spins_dev, int32_t replicas,
                              int64_t *energies_dev, void *cuda_stream);

/* Final state: spins[R][n] (may be NULL), energies[R] (may be NULL) and the
 * number of sweeps run.  Waits for the solve to finish. */
isg_status isg_result_final(const isg_result *r, int8_t *spins, int32_t *energies,
                            int32_t *sweeps_done);

/* Best state: the lowest best energy over replicas and its replica (ties go
 * to the lowest replica index), that replica's best spins[n] (may be NULL),
 * every replica's best energy per_replica_best[R] (may be NULL) and the first
 * sweep at which the target was reached (-1 if none or no target). */
isg_status isg_best(const isg_result *r, int32_t *best_energy, int32_t *best_replica,
                    int8_t *best_spins, int32_t *per_replica_best, int32_t *hit_sweep);

/* Sizes of a result: vertices n, replicas R and the sweep budget S.  Does not
 * wait for the solve.  Any output pointer may be NULL. */
isg_status isg_result_shape(const isg_result *r, int32_t *n, int32_t *replicas, int32_t *sweeps);

/* All replicas' best states best_spins[R][n]. */
isg_status isg_result_best_all(const isg_result *r, int8_t *best_spins);

typedef struct {
    float sweep_kernel_ms;   /* CUDA-event time of the sweep launches (time_kernels), else -1 */
    int32_t launches;        /* kernel launches this solve made (all kernels of the library) */
    int32_t sweep_launches;  /* launches of the sweep kernel */
    int32_t kernel;          /* isg_kernel actually used */
    int32_t ctas;            /* CTAs of the sweep kernel */
    int32_t cluster_ctas;    /* CTAs per cluster */
    int32_t threads;         /* threads per CTA */
    int64_t h2d_bytes;       /* host-to-device bytes the solve copied: its threshold table
                                and the instance arrays uploaded for it (0 if resident) */
    int32_t staged;          /* colour-class kernels: 1 if each CTA holds the adjacency of the
                                vertices it updates in shared memory (the multi-spin graph
                                kernel then also keeps its vertices' acceptance masks for the
                                next sweep there), else 0 */
    int32_t first_replica;   /* isg_options.first_replica of the solve (0 for other forms) */
    int32_t mask_chunks;     /* chunks of precomputed acceptance masks (isg_options.mask_chunk);
                                0: built inside the sweep kernel */
} isg_stats;

isg_status isg_result_stats(const isg_result *r, isg_stats *stats);

void isg_result_destroy(isg_result *r);

/* ---------------------------------------------------------------- serving */

/* A continuous-batching annealing server on the current device.  Requests
 * are admitted while a slot is free and their device state fits both in
 * device_mem_budget bytes and in the device's free memory at admission
 * (cudaMemGetInfo, less 256 MiB left for others; with nothing resident a
 * request is admitted regardless, and comes back with a result whose reads
 * return ISG_ENOMEM if its allocation fails).  Admitted requests run together
 * in chunks of one persistent kernel launch; each runs until its target or
 * its sweep budget.
 * A chunk advances every request by sweeps_per_chunk x sqrt(10,000 / n)
 * sweeps (n its spin count; at least 1), times a per-unit-kind factor (torus
 * words, graph words, graph quads) that the server adapts after every chunk
 * so that the kinds' kernels, which run concurrently, take equal time: a
 * larger instance does more work per chunk than a smaller one, but not in
 * proportion to its size.
 * A request's result equals isg_anneal of the same arguments, bit for bit.
 * max_slots >= 1, sweeps_per_chunk >= 1. */
isg_status isg_server_create(size_t device_mem_budget, int32_t max_slots,
                             int32_t sweeps_per_chunk, isg_server **out);

/* Queue a request (the problem handle must outlive the request).  Returns at
 * once with its id.  EINVAL on bad arguments; ECANCELLED after shutdown. */
isg_status isg_server_submit(isg_server *s, const isg_problem *p, int32_t replicas,
                             const double *betas, int32_t sweeps, uint64_t seed,
                             int64_t target_energy, uint64_t *request_id);

/* Wait up to timeout_s seconds for any finished request; on success returns
 * its id and a result handle (owned by the caller).  ETIMEOUT if none. */
isg_status isg_server_poll(isg_server *s, uint64_t *request_id, isg_result **out,
                           double timeout_s);

/* Cancel a queued or running request.  A queued one is handed back at once, a
 * running one at the end of the chunk in progress (its state is dropped); in
 * both cases isg_server_poll returns it with a result whose reads return
 * ISG_ECANCELLED: a cancel that returns ISG_OK always takes effect, even when
 * the request would have reached its target or budget in that chunk.  EINVAL
 * for NULL or an id that is neither queued nor running (unknown, or already
 * decided finished at a chunk end: its result is then the normal one). */
isg_status isg_server_cancel(isg_server *s, uint64_t request_id);

/* Stop the server; unfinished requests are dropped.  */
isg_status isg_server_destroy(isg_server *s);

typedef struct {
    int64_t submitted;    /* requests accepted by isg_server_submit */
    int64_t completed;    /* requests handed to isg_server_poll's queue */
    int32_t queued;       /* waiting for a slot or memory now */
    int32_t active;       /* resident now */
    int32_t peak_active;  /* most requests resident at once so far */
    int64_t passes;       /* chunk passes run (one launch of the unit kernels each) */
    int64_t replays;      /* passes re-run to a multi-unit request's stop sweep */
    int64_t cancelled;    /* requests handed back by isg_server_cancel */
} isg_server_stats;

/* Host-side fault injection for tests: the next `count` allocations of solve
 * state (isg_anneal and its variants, served admissions) fail as if the
 * device were out of memory, without any device work: the solve returns
 * ISG_ENOMEM, and a served request is handed back with a result whose reads
 * return ISG_ENOMEM while the server carries on.  count = 0 clears it.  Process
 * wide.  EINVAL for count < 0. */
isg_status isg_debug_fail_allocations(int32_t count);

/* Counters of the server (a consistent snapshot).  EINVAL for NULL. */
isg_status isg_server_get_stats(isg_server *s, isg_server_stats *out);

/* ---------------------------------------------------------------- misc */

/* The acceptance thresholds the kernels use, computed on the host exactly as
 * the solve paths compute them: out[t * (kmax + 1) + k] =
 * min(floor(2^32 exp(-betas[t] * 2k)), 2^32 - 1) for sweeps t < sweeps and
 * half energy changes k = 0..kmax (an uphill flip of energy change d = 2k is
 * taken when its uniform u < out[t][k]).  FP64 with the C library's exp.
 * out is caller-owned host memory of sweeps * (kmax + 1) words.  EINVAL for
 * NULL pointers, sweeps < 1, kmax < 0 or a beta that is not finite and >= 0.
 * No device work. */
isg_status isg_acceptance_table(const double *betas, int32_t sweeps, int32_t kmax,
                                uint32_t *out);

/* Measured throughput of the two integer instructions the sweep kernels are
 * built from, on the current device: three-input logic ops (lop3) and
 * widening 32x32->64 multiplies by a constant (mul.wide.u32, the Philox
 * product; each followed by one lop3, which runs on the other pipe), in
 * thread-instructions per second over the whole device.  The paper has no
 * counterpart: these are the denominators of the sweep kernels' roofline.
 * Runs two short kernels (about 10 ms each) on cuda_stream (NULL = legacy
 * default stream) and synchronises with them; allocates 4 bytes per CTA,
 * stream-ordered.  EINVAL for NULL outputs, ECUDA if a launch fails. */
isg_status isg_integer_peaks(void *cuda_stream, double *lop3_per_s, double *mul_wide_per_s);

/* Measured rates, on the current device, of the sweep kernels' random numbers
 * alone: uniforms per second of the factored Philox4x32-10 stream the sweeps
 * draw (per site: the round-1/2 prefix and 8 blocks = 32 uniforms), without
 * (uniforms_per_s) and with (masked_per_s) the two threshold masks the torus
 * sweep builds from them.  Every attempt needs one uniform, so these bound a
 * sweep's attempts/s from above.  No counterpart in the paper: a roofline aid.
 * Runs two short kernels on cuda_stream and synchronises.  EINVAL for NULL. */
isg_status isg_philox_rates(void *cuda_stream, double *uniforms_per_s, double *masked_per_s);

/* Message of the last failed call on this thread ("" if none). */
const char *isg_last_error(void);

/* Library version string. */
const char *isg_version(void);

#ifdef __cplusplus
}
#endif
#endif
