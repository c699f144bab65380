/*
 * isg_oracle.c -- plain, slow, obviously correct CPU oracle (C99 + pthreads).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load or call this file's library.  It
 * shares no code with the CUDA path: its own Philox, its own acceptance table,
 * its own colouring, its own energy and its own sweep loop.
 *
 * Every function follows a stated definition; none is blocked, fused or
 * reordered beyond what that definition allows.  See isg_oracle.h for the
 * argument conventions.
 */
#include "isg_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 3.3 and Table 2).  One round maps
 * (c0,c1,c2,c3) with key (k0,k1) to
 *   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0));
 * the key is bumped by the Weyl constants before every round after the first. */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout of the method's random numbers.  Replica r at vertex i in
 * sweep t draws word (r mod 4) of Philox(key = seed, ctr = (i, t, r/4, tag)),
 * with tag 0 for the Metropolis uniforms and tag 1 (t = 0) for the initial
 * spins.  i is the vertex id of the instance as given. */
#define ORC_TAG_SWEEP 0u
#define ORC_TAG_INIT 1u
#define ORC_TAG_EXCHANGE 2u
#define ORC_TAG_CLUSTER 3u

static uint32_t orc_draw(uint64_t seed, uint32_t i, uint32_t t, uint32_t r, uint32_t tag) {
    uint32_t ctr[4] = {i, t, r >> 2, tag};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[r & 3u];
}

void orc_initial_spins(int32_t n, int32_t n_rep, const int32_t *rep_ids, uint64_t seed, int8_t *s) {
    for (int32_t k = 0; k < n_rep; ++k)
        for (int32_t i = 0; i < n; ++i)
            s[(int64_t)k * n + i] =
                (orc_draw(seed, (uint32_t)i, 0u, (uint32_t)rep_ids[k], ORC_TAG_INIT) >> 31) ? 1 : -1;
}

/* ------------------------------------------------------------------------ */
/* Instance forms. */

static int orc_cmp_pair(const void *a, const void *b) {
    const int64_t *x = (const int64_t *)a, *y = (const int64_t *)b;
    return (x[0] > y[0]) - (x[0] < y[0]);
}

int orc_build_csr(int32_t n, int64_t m, const int32_t *u, const int32_t *v, const int32_t *w,
                  int64_t *rowptr, int32_t *col, int32_t *wt) {
    if (n < 1 || m < 0) return -1;
    for (int64_t e = 0; e < m; ++e)
        if (u[e] < 0 || u[e] >= n || v[e] < 0 || v[e] >= n || u[e] == v[e]) return -1;
    memset(rowptr, 0, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t e = 0; e < m; ++e) {
        rowptr[u[e] + 1]++;
        rowptr[v[e] + 1]++;
    }
    for (int32_t i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int32_t i = 0; i < n; ++i) fill[i] = rowptr[i];
    for (int64_t e = 0; e < m; ++e) {
        col[fill[u[e]]] = v[e]; wt[fill[u[e]]++] = w[e];
        col[fill[v[e]]] = u[e]; wt[fill[v[e]]++] = w[e];
    }
    free(fill);
    /* sort each row by neighbour id (pairs of (col, wt)) and reject duplicates */
    int status = 0;
    for (int32_t i = 0; i < n && status == 0; ++i) {
        int64_t a = rowptr[i], b = rowptr[i + 1];
        int64_t len = b - a;
        if (len < 2) continue;
        int64_t *pairs = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)len);
        for (int64_t p = 0; p < len; ++p) {
            pairs[2 * p] = col[a + p];
            pairs[2 * p + 1] = wt[a + p];
        }
        qsort(pairs, (size_t)len, 2 * sizeof(int64_t), orc_cmp_pair);
        for (int64_t p = 0; p < len; ++p) {
            col[a + p] = (int32_t)pairs[2 * p];
            wt[a + p] = (int32_t)pairs[2 * p + 1];
            if (p > 0 && col[a + p] == col[a + p - 1]) status = -1;
        }
        free(pairs);
    }
    return status;
}

void orc_torus_edges(int32_t L, int32_t W, const int8_t *j_right, const int8_t *j_down,
                     int32_t *u, int32_t *v, int32_t *w) {
    for (int32_t r = 0; r < L; ++r)
        for (int32_t c = 0; c < W; ++c) {
            int32_t i = r * W + c;
            u[2 * i] = i;
            v[2 * i] = r * W + (c + 1) % W;
            w[2 * i] = j_right[i];
            u[2 * i + 1] = i;
            v[2 * i + 1] = ((r + 1) % L) * W + c;
            w[2 * i + 1] = j_down[i];
        }
}

int32_t orc_greedy_colouring(int32_t n, const int64_t *rowptr, const int32_t *col, int32_t *colour) {
    /* used[c] == v+1 marks colour c as taken by a lower neighbour of v */
    int32_t *used = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t n_colours = 0;
    for (int32_t v = 0; v < n; ++v) {
        for (int64_t p = rowptr[v]; p < rowptr[v + 1]; ++p) {
            int32_t u = col[p];
            if (u < v) used[colour[u]] = v + 1;
        }
        int32_t c = 0;
        while (used[c] == v + 1) ++c;
        colour[v] = c;
        if (c + 1 > n_colours) n_colours = c + 1;
    }
    free(used);
    return n_colours;
}

int32_t orc_smallest_last_colouring(int32_t n, const int64_t *rowptr, const int32_t *col,
                                    int32_t *colour) {
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    uint8_t *removed = (uint8_t *)calloc((size_t)n + 1, 1);
    int32_t *used = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    for (int32_t v = 0; v < n; ++v) deg[v] = rowptr[v + 1] - rowptr[v];
    /* removal order: each step scans every vertex still present for the
     * smallest remaining degree (first, i.e. smallest, id among ties) */
    for (int32_t step = 0; step < n; ++step) {
        int32_t best = -1;
        for (int32_t v = 0; v < n; ++v)
            if (!removed[v] && (best < 0 || deg[v] < deg[best])) best = v;
        removed[best] = 1;
        order[step] = best;
        for (int64_t p = rowptr[best]; p < rowptr[best + 1]; ++p)
            if (!removed[col[p]]) --deg[col[p]];
    }
    /* colour in reverse removal order: smallest colour no coloured neighbour has */
    for (int32_t v = 0; v < n; ++v) colour[v] = -1;
    for (int32_t c = 0; c <= n; ++c) used[c] = -1;
    int32_t n_colours = 0;
    for (int32_t step = n - 1; step >= 0; --step) {
        const int32_t v = order[step];
        for (int64_t p = rowptr[v]; p < rowptr[v + 1]; ++p)
            if (colour[col[p]] >= 0) used[colour[col[p]]] = v;
        int32_t c = 0;
        while (used[c] == v) ++c;
        colour[v] = c;
        if (c + 1 > n_colours) n_colours = c + 1;
    }
    /* number the classes by their smallest vertex */
    int32_t *rename = used;
    for (int32_t c = 0; c < n_colours; ++c) rename[c] = -1;
    int32_t next = 0;
    for (int32_t v = 0; v < n; ++v)
        if (rename[colour[v]] < 0) rename[colour[v]] = next++;
    for (int32_t v = 0; v < n; ++v) colour[v] = rename[colour[v]];
    free(deg);
    free(order);
    free(removed);
    free(used);
    return n_colours;
}

/* ------------------------------------------------------------------------ */
/* Acceptance table: a move that raises the energy by d > 0 is accepted with
 * probability exp(-beta_t d); the threshold on a 32-bit uniform u is
 * floor(2^32 exp(-beta_t d)), capped at 2^32 - 1, computed in FP64. */
void orc_accept_table(int32_t sweeps, const double *betas, int32_t kmax, uint32_t *table) {
    for (int32_t t = 0; t < sweeps; ++t)
        for (int32_t k = 0; k <= kmax; ++k) {
            double p = exp(-betas[t] * (double)(2 * k));
            double x = floor(ldexp(p, 32));
            table[(int64_t)t * (kmax + 1) + k] = (x >= 4294967295.0) ? 4294967295u : (uint32_t)x;
        }
}

int64_t orc_energy(int32_t n, const int64_t *rowptr, const int32_t *col, const int32_t *wt,
                   const int32_t *field, const int8_t *s) {
    int64_t e = 0;
    for (int32_t i = 0; i < n; ++i) {
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (col[p] > i) e += (int64_t)wt[p] * s[i] * s[col[p]];
        if (field) e += (int64_t)field[i] * s[i];
    }
    return e;
}

/* ------------------------------------------------------------------------ */
/* Annealing. */

typedef struct {
    int32_t n;
    const int64_t *rowptr;
    const int32_t *col;
    const int32_t *wt;
    const int32_t *field;       /* local fields h_i, or NULL */
    const int32_t *order;       /* vertices grouped by colour class */
    const int64_t *class_start; /* n_colours + 1 entries */
    int32_t n_colours;
    const uint32_t *table;
    int32_t kmax;
    uint64_t seed;
    const double *betas;
    int check_energy;
    int has_target;
    int64_t target;
    int32_t run_sweeps;         /* sweeps to run in this pass */
    const int32_t *rep_ids;
    int32_t k_begin, k_end;     /* listed replicas handled by this worker */
    int8_t *s_final;
    int32_t *e_final;
    int8_t *s_best;
    int32_t *e_best;
    int32_t *hit;               /* per listed replica: first sweep with e_best <= target */
    int status;
} orc_job;

static void orc_run_replica(orc_job *J, int32_t k) {
    const int32_t n = J->n;
    const uint32_t r = (uint32_t)J->rep_ids[k];
    int8_t *s = J->s_final + (int64_t)k * n;
    int8_t *best = J->s_best + (int64_t)k * n;
    for (int32_t i = 0; i < n; ++i)
        s[i] = (orc_draw(J->seed, (uint32_t)i, 0u, r, ORC_TAG_INIT) >> 31) ? 1 : -1;
    int64_t e = orc_energy(n, J->rowptr, J->col, J->wt, J->field, s);
    int64_t e_best = e;
    memcpy(best, s, (size_t)n);
    J->hit[k] = -1;
    for (int32_t t = 0; t < J->run_sweeps; ++t) {
        const uint32_t *row = J->table + (int64_t)t * (J->kmax + 1);
        for (int32_t c = 0; c < J->n_colours; ++c) {
            for (int64_t q = J->class_start[c]; q < J->class_start[c + 1]; ++q) {
                int32_t i = J->order[q];
                int64_t h = J->field ? J->field[i] : 0;
                for (int64_t p = J->rowptr[i]; p < J->rowptr[i + 1]; ++p)
                    h += (int64_t)J->wt[p] * s[J->col[p]];
                int64_t kk = -(int64_t)s[i] * h; /* energy change of the flip is 2*kk */
                int accept;
                if (kk <= 0)
                    accept = 1;
                else
                    accept = orc_draw(J->seed, (uint32_t)i, (uint32_t)t, r, ORC_TAG_SWEEP) < row[kk];
                if (accept) {
                    s[i] = (int8_t)(-s[i]);
                    e += 2 * kk;
                }
            }
        }
        if (J->check_energy && orc_energy(n, J->rowptr, J->col, J->wt, J->field, s) != e) {
            J->status = -2;
            return;
        }
        if (e < e_best) {
            e_best = e;
            memcpy(best, s, (size_t)n);
        }
        if (J->has_target && e_best <= J->target) {
            J->hit[k] = t;
            break;
        }
    }
    J->e_final[k] = (int32_t)e;
    J->e_best[k] = (int32_t)e_best;
}

static void *orc_worker(void *arg) {
    orc_job *J = (orc_job *)arg;
    for (int32_t k = J->k_begin; k < J->k_end && J->status == 0; ++k) orc_run_replica(J, k);
    return NULL;
}

static uint64_t orc_splitmix(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int orc_run_pass(orc_job *proto, int32_t n_rep, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n_rep) nthreads = n_rep;
    orc_job *jobs = (orc_job *)malloc(sizeof(orc_job) * (size_t)nthreads);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int w = 0; w < nthreads; ++w) {
        jobs[w] = *proto;
        jobs[w].k_begin = (int32_t)((int64_t)n_rep * w / nthreads);
        jobs[w].k_end = (int32_t)((int64_t)n_rep * (w + 1) / nthreads);
        jobs[w].status = 0;
    }
    for (int w = 1; w < nthreads; ++w) pthread_create(&th[w], NULL, orc_worker, &jobs[w]);
    orc_worker(&jobs[0]);
    for (int w = 1; w < nthreads; ++w) pthread_join(th[w], NULL);
    int status = 0;
    for (int w = 0; w < nthreads; ++w)
        if (jobs[w].status != 0) status = jobs[w].status;
    free(jobs);
    free(th);
    return status;
}

int orc_anneal(int32_t n, const int64_t *rowptr, const int32_t *col, const int32_t *wt,
               const int32_t *field, const int32_t *colour, int32_t n_colours,
               int32_t n_rep, const int32_t *rep_ids, int32_t sweeps, const double *betas,
               uint64_t seed, int has_target, int64_t target, uint64_t shuffle_seed,
               int check_energy, int nthreads,
               int8_t *s_final, int32_t *e_final, int8_t *s_best, int32_t *e_best,
               int32_t *hit_sweep, int32_t *sweeps_done) {
    if (n < 1 || n_rep < 1 || sweeps < 1 || n_colours < 1) return -1;
    for (int32_t i = 0; i < n; ++i)
        if (colour[i] < 0 || colour[i] >= n_colours) return -1;
    /* kmax = max_i (sum_j |w_ij| + |h_i|) bounds the energy change of any
     * single flip by 2*kmax */
    int64_t kmax = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t a = field ? llabs((long long)field[i]) : 0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) a += llabs((long long)wt[p]);
        if (a > kmax) kmax = a;
    }
    uint32_t *table = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)sweeps * (size_t)(kmax + 1));
    orc_accept_table(sweeps, betas, (int32_t)kmax, table);

    /* colour classes in ascending order, vertices of a class by ascending id */
    int64_t *class_start = (int64_t *)calloc((size_t)n_colours + 1, sizeof(int64_t));
    for (int32_t i = 0; i < n; ++i) class_start[colour[i] + 1]++;
    for (int32_t c = 0; c < n_colours; ++c) class_start[c + 1] += class_start[c];
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_colours);
    for (int32_t c = 0; c < n_colours; ++c) fill[c] = class_start[c];
    for (int32_t i = 0; i < n; ++i) order[fill[colour[i]]++] = i;
    free(fill);
    if (shuffle_seed != 0) {
        uint64_t st = shuffle_seed;
        for (int32_t c = 0; c < n_colours; ++c) {
            int64_t a = class_start[c], len = class_start[c + 1] - a;
            for (int64_t q = len - 1; q > 0; --q) {
                int64_t j = (int64_t)(orc_splitmix(&st) % (uint64_t)(q + 1));
                int32_t tmp = order[a + q];
                order[a + q] = order[a + j];
                order[a + j] = tmp;
            }
        }
    }

    int32_t *hit = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_rep);
    orc_job job;
    memset(&job, 0, sizeof(job));
    job.n = n; job.rowptr = rowptr; job.col = col; job.wt = wt; job.field = field;
    job.order = order; job.class_start = class_start; job.n_colours = n_colours;
    job.table = table; job.kmax = (int32_t)kmax; job.seed = seed; job.betas = betas;
    job.check_energy = check_energy; job.has_target = has_target; job.target = target;
    job.run_sweeps = sweeps; job.rep_ids = rep_ids;
    job.s_final = s_final; job.e_final = e_final; job.s_best = s_best; job.e_best = e_best;
    job.hit = hit;

    /* Pass 1: every replica runs until its own best reaches the target (or all
     * sweeps).  The solve's stopping sweep is the earliest of those. */
    int status = orc_run_pass(&job, n_rep, nthreads);
    int32_t t_stop = -1;
    if (status == 0 && has_target)
        for (int32_t k = 0; k < n_rep; ++k)
            if (hit[k] >= 0 && (t_stop < 0 || hit[k] < t_stop)) t_stop = hit[k];
    if (status == 0 && t_stop >= 0) {
        /* Pass 2: replay every replica to the end of the stopping sweep. */
        job.has_target = 0;
        job.run_sweeps = t_stop + 1;
        status = orc_run_pass(&job, n_rep, nthreads);
    }
    *hit_sweep = t_stop;
    *sweeps_done = (t_stop >= 0) ? t_stop + 1 : sweeps;

    free(hit);
    free(order);
    free(class_start);
    free(table);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Parallel tempering (Sec. II.C: replicas at different temperatures that
 * exchange configurations across temperatures).  32 independent ladders
 * ("chains" c = 0..31); replica r = 32 k + c sits at temperature slot k with
 * inverse temperature betas[k].  Round q: every replica runs `per_round`
 * sweeps (global sweep index t = q * per_round + j, the annealing sweep at
 * beta_k); then, for every slot pair (k, k+1) with k = q mod 2, k+1 < K, and
 * every chain, the two configurations (and their energies) are exchanged
 * with probability min(1, exp(a)), a = (beta_k - beta_{k+1}) (E_k - E_{k+1}):
 * always when a >= 0, else when the exchange uniform u < floor(2^32 exp(a)),
 * u = word (c mod 4) of Philox(seed, (k, q, c / 4, 2)).  Best states stay
 * with the slot and are checked at sweep ends. */

typedef struct {
    int32_t n, K, rounds, per_round, n_colours;
    const int64_t *rowptr;
    const int32_t *col, *wt, *field, *order;
    const int64_t *class_start;
    const double *betas;
    const uint32_t *table; /* [K][kmax + 1]: slot k's Metropolis thresholds */
    int32_t kmax;
    uint64_t seed;
    int32_t c_begin, c_end;
    int8_t *s_final, *s_best;
    int32_t *e_final, *e_best;
    int64_t *accepted, *attempted; /* [32][K - 1] per chain, summed by the caller */
    int32_t icm_slots;             /* Houdayer moves on slots k >= K - icm_slots */
    int64_t *flipped;              /* [K] sites flipped by cluster moves (per chain pair) */
} orc_pt_job;

/* Houdayer cluster move on chains a and b of one slot (Sec. II.C's replica
 * cluster moves): the sites where the two configurations differ span a
 * subgraph; one of them is drawn (the (u mod D)-th differing site in vertex
 * order, D their number, u word 0 of Philox(seed, (k, q, m, 3)) for pair m),
 * its connected component in that subgraph is the cluster, and both chains
 * flip it - i.e. they exchange their spins on the cluster, which leaves
 * E_a + E_b unchanged.  Returns the cluster size (0 when a = b). */
static int64_t orc_houdayer(const orc_pt_job *J, int8_t *sa, int8_t *sb, uint32_t k, uint32_t q,
                            uint32_t m, int32_t *stack, uint8_t *in) {
    const int32_t n = J->n;
    int64_t D = 0;
    for (int32_t i = 0; i < n; ++i) D += sa[i] != sb[i];
    if (D == 0) return 0;
    uint32_t ctr[4] = {k, q, m, ORC_TAG_CLUSTER};
    uint32_t key[2] = {(uint32_t)(J->seed & 0xFFFFFFFFu), (uint32_t)(J->seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    int64_t pick = (int64_t)(out[0] % (uint64_t)D), seen = 0;
    int32_t root = -1;
    for (int32_t i = 0; i < n && root < 0; ++i)
        if (sa[i] != sb[i] && seen++ == pick) root = i;
    memset(in, 0, (size_t)n);
    int64_t top = 0, size = 0;
    stack[top++] = root;
    in[root] = 1;
    while (top > 0) {
        const int32_t i = stack[--top];
        ++size;
        for (int64_t p = J->rowptr[i]; p < J->rowptr[i + 1]; ++p) {
            const int32_t j = J->col[p];
            if (!in[j] && sa[j] != sb[j]) {
                in[j] = 1;
                stack[top++] = j;
            }
        }
    }
    for (int32_t i = 0; i < n; ++i)
        if (in[i]) {
            sa[i] = (int8_t)(-sa[i]);
            sb[i] = (int8_t)(-sb[i]);
        }
    return size;
}

/* The chains of one pair (c = 2m, 2m + 1) run together: cluster moves couple
 * them; chains of different pairs never interact. */
static void orc_pt_pair(orc_pt_job *J, int32_t m) {
    const int32_t n = J->n, K = J->K;
    int64_t *e = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)K);   /* [2][K] */
    int64_t *eb = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)K);
    int8_t *tmp = (int8_t *)malloc((size_t)n);
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    uint8_t *in = (uint8_t *)malloc((size_t)n);
    for (int32_t h = 0; h < 2; ++h)
        for (int32_t k = 0; k < K; ++k) {
            const uint32_t r = (uint32_t)(32 * k + 2 * m + h);
            int8_t *s = J->s_final + (int64_t)r * n;
            for (int32_t i = 0; i < n; ++i)
                s[i] = (orc_draw(J->seed, (uint32_t)i, 0u, r, ORC_TAG_INIT) >> 31) ? 1 : -1;
            e[h * K + k] = orc_energy(n, J->rowptr, J->col, J->wt, J->field, s);
            eb[h * K + k] = e[h * K + k];
            memcpy(J->s_best + (int64_t)r * n, s, (size_t)n);
        }
    for (int32_t q = 0; q < J->rounds; ++q) {
        /* sweeps of every replica at its slot's beta */
        for (int32_t h = 0; h < 2; ++h)
            for (int32_t k = 0; k < K; ++k) {
                const uint32_t r = (uint32_t)(32 * k + 2 * m + h);
                int8_t *s = J->s_final + (int64_t)r * n;
                const uint32_t *row = J->table + (int64_t)k * (J->kmax + 1);
                for (int32_t j = 0; j < J->per_round; ++j) {
                    const uint32_t t = (uint32_t)(q * J->per_round + j);
                    for (int32_t cc = 0; cc < J->n_colours; ++cc)
                        for (int64_t z = J->class_start[cc]; z < J->class_start[cc + 1]; ++z) {
                            const int32_t i = J->order[z];
                            int64_t hf = J->field ? J->field[i] : 0;
                            for (int64_t p = J->rowptr[i]; p < J->rowptr[i + 1]; ++p)
                                hf += (int64_t)J->wt[p] * s[J->col[p]];
                            const int64_t kk = -(int64_t)s[i] * hf;
                            if (kk <= 0 ||
                                orc_draw(J->seed, (uint32_t)i, t, r, ORC_TAG_SWEEP) < row[kk]) {
                                s[i] = (int8_t)(-s[i]);
                                e[h * K + k] += 2 * kk;
                            }
                        }
                    if (e[h * K + k] < eb[h * K + k]) {
                        eb[h * K + k] = e[h * K + k];
                        memcpy(J->s_best + (int64_t)r * n, s, (size_t)n);
                    }
                }
            }
        /* Houdayer cluster moves between the pair's two chains on the last
         * icm_slots slots */
        for (int32_t k = K - J->icm_slots; k < K; ++k) {
            if (k < 0) continue;
            int8_t *sa = J->s_final + (int64_t)(32 * k + 2 * m) * n;
            int8_t *sb = J->s_final + (int64_t)(32 * k + 2 * m + 1) * n;
            const int64_t size = orc_houdayer(J, sa, sb, (uint32_t)k, (uint32_t)q, (uint32_t)m,
                                              stack, in);
            if (size > 0) {
                e[k] = orc_energy(n, J->rowptr, J->col, J->wt, J->field, sa);
                e[K + k] = orc_energy(n, J->rowptr, J->col, J->wt, J->field, sb);
                J->flipped[(int64_t)m * K + k] += size;
            }
        }
        /* exchanges between neighbouring slots, chain by chain */
        for (int32_t h = 0; h < 2; ++h) {
            const int32_t c = 2 * m + h;
            int64_t *ec = e + h * K;
            for (int32_t k = q % 2; k + 1 < K; k += 2) {
                const double a = (J->betas[k] - J->betas[k + 1]) * (double)(ec[k] - ec[k + 1]);
                int swap = a >= 0.0;
                if (!swap) {
                    const double x = floor(ldexp(exp(a), 32));
                    const uint32_t thr = x >= 4294967295.0 ? 4294967295u : (uint32_t)x;
                    swap = orc_draw(J->seed, (uint32_t)k, (uint32_t)q, (uint32_t)c,
                                    ORC_TAG_EXCHANGE) < thr;
                }
                J->attempted[(int64_t)c * (K - 1) + k]++;
                if (swap) {
                    J->accepted[(int64_t)c * (K - 1) + k]++;
                    int8_t *a_s = J->s_final + (int64_t)(32 * k + c) * n;
                    int8_t *b_s = J->s_final + (int64_t)(32 * (k + 1) + c) * n;
                    memcpy(tmp, a_s, (size_t)n);
                    memcpy(a_s, b_s, (size_t)n);
                    memcpy(b_s, tmp, (size_t)n);
                    const int64_t te = ec[k];
                    ec[k] = ec[k + 1];
                    ec[k + 1] = te;
                }
            }
        }
    }
    for (int32_t h = 0; h < 2; ++h)
        for (int32_t k = 0; k < K; ++k) {
            J->e_final[32 * k + 2 * m + h] = (int32_t)e[h * K + k];
            J->e_best[32 * k + 2 * m + h] = (int32_t)eb[h * K + k];
        }
    free(e);
    free(eb);
    free(tmp);
    free(stack);
    free(in);
}

static void *orc_pt_worker(void *arg) {
    orc_pt_job *J = (orc_pt_job *)arg;
    for (int32_t m = J->c_begin; m < J->c_end; ++m) orc_pt_pair(J, m);
    return NULL;
}

int orc_parallel_tempering(int32_t n, const int64_t *rowptr, const int32_t *col, const int32_t *wt,
                           const int32_t *field, const int32_t *colour, int32_t n_colours,
                           int32_t K, const double *betas, int32_t rounds, int32_t per_round,
                           int32_t icm_slots, uint64_t seed, int nthreads, int8_t *s_final,
                           int32_t *e_final, int8_t *s_best, int32_t *e_best, int64_t *accepted,
                           int64_t *attempted, int64_t *flipped) {
    if (n < 1 || K < 1 || rounds < 1 || per_round < 1 || n_colours < 1) return -1;
    if (icm_slots < 0 || icm_slots > K) return -1;
    for (int32_t i = 0; i < n; ++i)
        if (colour[i] < 0 || colour[i] >= n_colours) return -1;
    int64_t kmax = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t a = field ? llabs((long long)field[i]) : 0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) a += llabs((long long)wt[p]);
        if (a > kmax) kmax = a;
    }
    uint32_t *table = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)K * (size_t)(kmax + 1));
    orc_accept_table(K, betas, (int32_t)kmax, table);
    int64_t *class_start = (int64_t *)calloc((size_t)n_colours + 1, sizeof(int64_t));
    for (int32_t i = 0; i < n; ++i) class_start[colour[i] + 1]++;
    for (int32_t c = 0; c < n_colours; ++c) class_start[c + 1] += class_start[c];
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_colours);
    for (int32_t c = 0; c < n_colours; ++c) fill[c] = class_start[c];
    for (int32_t i = 0; i < n; ++i) order[fill[colour[i]]++] = i;
    free(fill);
    const int32_t pairs = K > 1 ? K - 1 : 1;
    int64_t *acc = (int64_t *)calloc((size_t)32 * pairs, sizeof(int64_t));
    int64_t *att = (int64_t *)calloc((size_t)32 * pairs, sizeof(int64_t));
    int64_t *flp = (int64_t *)calloc((size_t)16 * K, sizeof(int64_t));

    if (nthreads < 1) nthreads = 1;
    if (nthreads > 16) nthreads = 16;
    orc_pt_job *jobs = (orc_pt_job *)malloc(sizeof(orc_pt_job) * (size_t)nthreads);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int w = 0; w < nthreads; ++w) {
        orc_pt_job *J = &jobs[w];
        memset(J, 0, sizeof(*J));
        J->n = n; J->K = K; J->rounds = rounds; J->per_round = per_round;
        J->n_colours = n_colours; J->rowptr = rowptr; J->col = col; J->wt = wt;
        J->field = field; J->order = order; J->class_start = class_start; J->betas = betas;
        J->table = table; J->kmax = (int32_t)kmax; J->seed = seed;
        J->c_begin = 16 * w / nthreads; J->c_end = 16 * (w + 1) / nthreads;  /* chain pairs */
        J->s_final = s_final; J->s_best = s_best; J->e_final = e_final; J->e_best = e_best;
        J->accepted = acc; J->attempted = att; J->icm_slots = icm_slots; J->flipped = flp;
    }
    for (int w = 1; w < nthreads; ++w) pthread_create(&th[w], NULL, orc_pt_worker, &jobs[w]);
    orc_pt_worker(&jobs[0]);
    for (int w = 1; w < nthreads; ++w) pthread_join(th[w], NULL);
    for (int32_t k = 0; k + 1 < K; ++k) {
        accepted[k] = 0;
        attempted[k] = 0;
        for (int32_t c = 0; c < 32; ++c) {
            accepted[k] += acc[(int64_t)c * (K - 1) + k];
            attempted[k] += att[(int64_t)c * (K - 1) + k];
        }
    }
    for (int32_t k = 0; k < K; ++k) {
        flipped[k] = 0;
        for (int32_t m = 0; m < 16; ++m) flipped[k] += flp[(int64_t)m * K + k];
    }
    free(flp);
    free(jobs);
    free(th);
    free(acc);
    free(att);
    free(order);
    free(class_start);
    free(table);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exhaustive enumeration in Gray-code order: state g differs from g-1 in the
 * spin of index ctz(g), so each step costs one local-field evaluation. */
int64_t orc_enumerate(int32_t n, const int64_t *rowptr, const int32_t *col, const int32_t *wt,
                      const int32_t *field, int8_t *argmin, uint64_t *hist) {
    int8_t *s = (int8_t *)malloc((size_t)n);
    int64_t wabs = 0;
    for (int32_t i = 0; i < n; ++i) {
        s[i] = -1;
        if (field) wabs += llabs((long long)field[i]);
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (col[p] > i) wabs += llabs((long long)wt[p]);
    }
    int64_t e = orc_energy(n, rowptr, col, wt, field, s);
    int64_t e_min = e;
    uint64_t g_min = 0;
    if (hist) hist[e + wabs]++;
    uint64_t count = (uint64_t)1 << n;
    for (uint64_t g = 1; g < count; ++g) {
        int32_t j = __builtin_ctzll(g);
        int64_t h = field ? field[j] : 0;
        for (int64_t p = rowptr[j]; p < rowptr[j + 1]; ++p) h += (int64_t)wt[p] * s[col[p]];
        e += -2 * (int64_t)s[j] * h;
        s[j] = (int8_t)(-s[j]);
        if (hist) hist[e + wabs]++;
        if (e < e_min) {
            e_min = e;
            g_min = g;
        }
    }
    if (argmin) {
        uint64_t gray = g_min ^ (g_min >> 1); /* bit i set <=> spin i flipped from -1 */
        for (int32_t i = 0; i < n; ++i) argmin[i] = ((gray >> i) & 1u) ? 1 : -1;
    }
    free(s);
    return e_min;
}
