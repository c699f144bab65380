// isg_runtime.h -- host-side objects behind the opaque handles of isg.h.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "isg.h"

namespace isg {

// What a caller needs resident: the torus coupling bits (multi-spin kernel),
// the relabelled CSR (colour-class kernel), or the original-id CSR (energies).
enum DeviceNeed : unsigned { kNeedTorus = 1u, kNeedCsr = 2u, kNeedEnergy = 4u };

// Instance arrays resident on one device (each group uploaded on first need).
struct DeviceProblem {
  int device = -1;
  unsigned have = 0;               // DeviceNeed bits already uploaded
  size_t bytes_uploaded = 0;
  uint8_t *cbits = nullptr;        // torus only: bit0 j_right == -1, bit1 j_down == -1
  int32_t *class_start = nullptr;  // colour-major relabelled CSR
  int32_t *rowptr = nullptr;
  int32_t *col = nullptr;
  int32_t *wt = nullptr;
  int32_t *field_r = nullptr;      // local fields, relabelled order (nullptr: none)
  int32_t *gloff = nullptr;        // [n + 1] prefix of the threshold levels (d + |h| + 1) / 2
  int64_t gl = 0;                  // gloff[n]: mask words of one replica word and sweep
  int32_t *orig = nullptr;         // relabelled -> original id
  int64_t *rowptr_o = nullptr;     // CSR in original ids (energy checks)
  int32_t *col_o = nullptr;
  int32_t *wt_o = nullptr;
  int32_t *field_o = nullptr;      // local fields, original order (nullptr: none)
};

}  // namespace isg

struct isg_problem {
  bool torus = false;
  int32_t n = 0, L = 0, W = 0;
  int64_t m = 0, total_weight = 0;
  int32_t kmax = 0;                        // max_i (sum_j |w_ij| + |h_i|)
  int32_t mode = 2;                        // weights: 0 all +1, 1 all +-1, 2 general (CsrSolve)
  int32_t dmax = 0;                        // largest degree
  bool unit_pos = false;                   // every weight is +1
  std::vector<int8_t> jr, jd;              // torus couplings
  std::vector<int64_t> rowptr;             // CSR, original ids, rows sorted
  std::vector<int32_t> col, wt;
  std::vector<int32_t> field;              // local fields h (empty: none)
  int32_t colouring = 0;                   // isg_colouring of a graph's classes
  std::vector<int32_t> colour;
  int32_t n_colours = 0;
  std::vector<int32_t> order;              // relabelled -> original
  std::vector<int32_t> class_start;
  std::vector<int32_t> rowptr_r, col_r, wt_r;  // relabelled CSR
  std::vector<int32_t> field_r;            // relabelled fields (empty: none)
  std::mutex mu;
  std::deque<isg::DeviceProblem> dev;      // one per device; element addresses stay valid
};

struct isg_result {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr, t0 = nullptr, t1 = nullptr;
  bool timed = false;
  int32_t n = 0, R = 0, S = 0;
  int32_t first_replica = 0;               // global index of replica 0 (Philox counters)
  bool has_target = false;
  int32_t kernel = 0;
  bool msc = false;                        // 32-lane replica words (torus or graph kernel)
  bool relabelled = false;                 // state in colour-major vertex order
  int32_t units = 0, lanes = 0;            // replica words (32 lanes) or quads (4 lanes)
  size_t table_words = 0;
  void *base = nullptr;                    // one device allocation holding everything
  size_t bytes = 0;
  std::shared_ptr<void> shared;            // device memory shared with other results (batches)
  uint32_t *d_spins = nullptr, *d_best = nullptr, *d_table = nullptr;
  int32_t *d_e_cur = nullptr, *d_e_best = nullptr, *d_hit = nullptr, *d_done = nullptr,
          *d_stop = nullptr;
  int8_t *d_out = nullptr, *d_out_best = nullptr;  // [R][n] +-1, original vertex order
  int32_t launches = 0, sweep_launches = 0, ctas = 0, cluster = 0, threads = 0;
  int64_t h2d_bytes = 0;                   // table + instance arrays uploaded for this solve
  int32_t staged = 0;                      // colour-class launches hold their adjacency in smem
  // parallel tempering: exchange tables and counters (one allocation), pairs K - 1
  void *pt_mem = nullptr;
  unsigned long long *d_accepted = nullptr;
  unsigned long long *d_flipped = nullptr;  // [K] cluster-move sizes per slot
  int32_t pt_pairs = 0, pt_slots = 0;
  cudaGraph_t pt_graph = nullptr;          // the rounds, captured once and launched as a graph
  cudaGraphExec_t pt_exec = nullptr;
  cudaStream_t pt_capture = nullptr;
  std::vector<int64_t> pt_attempted;
  // filled on first synchronisation
  std::mutex mu;
  bool synced = false;
  isg_status sync_status = ISG_OK;
  std::vector<int32_t> h_e_cur, h_e_best, h_done;
  int32_t hit_sweep = -1, sweeps_done = 0;
  float kernel_ms = -1.0f;
  // a single isg_anneal solve without a target, kept for isg_anneal_continue:
  // its instance, seed, schedule so far and launch shape (prob is null otherwise)
  const isg_problem *prob = nullptr;
  uint64_t seed = 0;
  std::vector<double> betas;
  bool plain = false;
  int32_t qpc = 1;
  int32_t mask_chunk = 0;                  // isg_options.mask_chunk of the solve
  int32_t mask_chunks = 0;                 // chunks of precomputed masks launched
  // precomputed graph masks: the sweep kernel's high-priority stream, the mask
  // kernel's low-priority stream, and their events (created on first use)
  cudaStream_t pm_sweeps = nullptr, pm_masks = nullptr;
  cudaEvent_t pm_ev[6] = {};
  uint32_t *d_table_ext = nullptr;         // threshold table of a continued schedule
};

namespace isg {

isg_status fail(isg_status st, const char *fmt, ...);
isg_status cuda_fail(cudaError_t err, const char *what);
isg_status problem_device(const isg_problem *p, unsigned need, const DeviceProblem **out,
                          size_t *uploaded = nullptr);
isg_status check_betas(const double *betas, int32_t sweeps);
void build_table(const double *betas, int32_t sweeps, const std::vector<int32_t> &levels,
                 std::vector<uint32_t> &out);
isg_status result_alloc(isg_result *r, cudaStream_t stream);
isg_status result_sync(const isg_result *r);
void result_free(isg_result *r);
int sm_count();
void torus_shape(int L, int W, int words, int &cluster, int &threads);
bool served_graph_msc(const isg_problem *p, int threads);

}  // namespace isg
