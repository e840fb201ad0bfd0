// Host-side handle of the C-ABI layer, shared by the step driver
// (bd_capi.cu) and the differentiated rollout driver (rollout.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "bd_internal.h"

struct RepHost {
  bd_params p;
  double L = 0, wall_lo = 0, wall_hi = 0;
  bool periodic = false;       // periodic box (no ghost points, torus triangulation)
  int n = 0;                   // disks
  int ext_base = 0;            // first index in the concatenated external arrays
  int slot_begin = 0, slot_end = 0;
  int ghost_base = 0, ng = 0;  // ghost vertex ids ghost_base .. ghost_base + ng - 1
  int tri_base = 0, nt = 0;
  int iblock_base = 0, n_iblocks = 0;
  int tile_begin = 0, tile_end = 0;
};

struct BdRollout;   // recorded rollout and adjoint buffers (rollout.cu)

struct bd_handle {
  cudaStream_t stream = nullptr;
  BdDev d;
  BdConst c;
  std::vector<RepHost> reps;
  std::vector<BdRep> h_rep;
  int n = 0, np = 0, np_i = 0, nt = 0, ng = 0;
  std::vector<int> ext_of_int;    // internal slot -> concatenated external index (-1 = empty)
  std::vector<int> int_of_ext;    // concatenated external index -> internal slot
  std::vector<double> host_pos;   // (np + ng) * 2 mirror used for uploads
  int dt_grid = 0, dt_block = 0;
  int vc_grid = 0, vc_block = 0;   // Verlet-list overlap correction launch
  int64_t step = 0;
  double2 *d_fsum = nullptr;
  BdCtl *h_ctl = nullptr;          // pinned
  std::vector<void *> dev_allocs;
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;   // pairs (start, end) per timed launch
  double force_ms = 0.0;
  int64_t force_launches = 0;
  int64_t last_launches = 0;
  int tune_tiles = 0;              // j tiles per work item chosen for the sweep
  int fpart_slots = 0;             // partial-force slots allocated
  std::vector<int> fpart_cap;      // per replica: chunks that fit
  BdRollout *ro = nullptr;         // differentiated rollout state (lazily created)
  // one step as a CUDA graph, replayed by bd_step (captured on a private
  // stream; valid while the kernel-argument tables equal the captured ones)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t step_graph = nullptr;
  cudaEvent_t graph_ev[2] = {nullptr, nullptr};   // force timing inside the graph
  BdDev graph_d;
  BdConst graph_c;
  bool graph_timed = false;
  bool graph_off = false;          // capture failed or disabled (BD_NO_GRAPH)
  int graph_launches = 0;          // kernels in one replay
  // Sec. 4.3 halving of rejected moves: depth limit and the step-start state
  int max_halvings = 0;
  double2 *hs_pos = nullptr;
  float4 *hs_work = nullptr;
  float *hs_theta = nullptr;
  int4 *hs_tv = nullptr, *hs_tn = nullptr;
  int *hs_vt = nullptr;
  bd_step_stats last_stats = {};   // counters of the last bd_step / bd_batch_step / bd_set_state
  int shard_rank = 0, shard_world = 1;   // force sharding (bd_set_force_shard)
  double stage_ns[5] = {0, 0, 0, 0, 0};   // triangulation-kernel stage times since the last reset
  int64_t stage_cnt[5] = {0, 0, 0, 0, 0};
};

namespace bdcapi {
// the user's n_species x n_species table (row-major; one species: alpha[0])
// into the replica's BD_MAX_SPECIES-wide FP64 and FP32 tables
void rep_set_alpha(BdRep &B, const double *alpha, int n_species);
int cuda_fail(cudaError_t e);
int read_ctl(bd_handle *h);                // copy the control block to h_ctl (synchronises)
cudaError_t reset_stats(bd_handle *h);     // zero the per-call statistics
int finish_status(bd_handle *h, int status);
void rollout_release(bd_handle *h);        // free the rollout buffers
void add_stage_times(bd_handle *h);        // accumulate the stage times of the last read_ctl
void fill_stats(bd_handle *h, int status, int64_t halvings);   // h->last_stats from h_ctl
}  // namespace bdcapi

// adjoint kernels (adjoint.cu)
cudaError_t bd_adj_rp_em(const BdDev &d, const BdConst &c, long long step, int k_local, cudaStream_t s);
cudaError_t bd_adj_rp_pass(const BdDev &d, const BdConst &c, int pass, int pb, int pe, cudaStream_t s);
cudaError_t bd_adj_vjp_pass(const BdDev &d, const BdConst &c, int pass, int pb, int pe, const double2 *z,
                            double2 *lam, double2 *mud, cudaStream_t s);
int bd_adj_force_chunks(const BdConst &c, int *jchunk);
cudaError_t bd_adj_vjp_em(const BdDev &d, const BdConst &c, int k_local, const double2 *x, const float *th,
                          double2 *lam, double2 *jpart, double *gpart, double *grad, cudaStream_t s);
cudaError_t bd_adj_msd(const BdDev &d, const BdConst &c, const double2 *x0, double *acc, double target,
                       double dscale, double2 *lam, double *loss, cudaStream_t s);
// pair-distance histogram of the disk slots' positions x (n disks) into h[32]
// (hpart: np x 32 doubles of scratch); with h0 also w = dL/dh, the loss
// sum_b (h_b - h0_b)^2 (loss may be NULL) and, with lam, dscale dL/dx
cudaError_t bd_adj_hist(const BdDev &d, const BdConst &c, int n, const double2 *x, double *hpart, double *h,
                        const double *h0, double *w, double *loss, double2 *lam, double dscale, cudaStream_t s);
