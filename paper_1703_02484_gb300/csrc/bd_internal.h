// Internal layout shared by the C-ABI layer and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bd.h"

// tile sizes of the all-pairs sweep (Sec. 4.1 tiling of Nyland et al.)
#define BD_TJ 256            // j-tile: disks staged per shared-memory stage
#define BD_FT 128            // threads per force block
#define BD_IPT 4             // i disks per thread
#define BD_IB (BD_FT * BD_IPT)  // i disks per force block
// symmetric sweep: blocks of BD_SB consecutive slots (two j tiles); species
// segments are padded to whole blocks so a block holds one species
#define BD_SB 512

// species per system (the long-range table is stored BD_MAX_SPECIES wide)
#define BD_MAX_SPECIES 4

// Verlet list capacity per disk (hard disks of radius a have at most ~40
// neighbours within 5.6a even at close packing)
#define BD_VL_MAX 64

// threads (and i disks) per block of the all-pairs force adjoint
#define BD_ADJ_T 128

// a check pass's verdict bits for the triangle it visits (held in registers)
#define BD_TRI_INVERTED 1
#define BD_TRI_DIRTY 2
// tv[t].w bits 24-31: the low byte of the generation of the check pass that
// must test the triangle's edges (set by flips and by flip candidates left
// unresolved; a stale byte that happens to match only adds tests)
#define BD_TRI_STAMP_SHIFT 24
// periodic box: corner k of a triangle sits at pos[v_k] + L (sx_k, sy_k);
// each component is a 2-bit two's-complement field of tv[t].w (0, 1 = +1,
// 3 = -1): sx_k at bit 8 + 4k, sy_k at bit 10 + 4k.  Zero for walls.
#define BD_TRI_SHIFT_BITS 0xFFF00

// device control block of the triangulation kernel
struct BdCtl {
  unsigned int bar_count;
  int status;
  unsigned int exit_count;         // blocks that have left the triangulation kernel
  unsigned int pad0[29];
  unsigned int bar_gen;            // on a 128-byte line of its own: the blocks waiting at a
  unsigned int pad1[31];           // barrier poll it, and only it
  unsigned long long epoch;        // flip-round counter, grows across launches
  int cnt[4][8];                   // per-phase counters, rotated every barrier
  // statistics accumulated over a bd_step call
  long long st_corr_iters;
  long long st_overlap_pairs;
  long long st_flip_rounds;
  long long st_flips;
  long long st_repair_flips;
  long long st_inverted;
  long long st_steps;
  int st_max_corr_iters;
  int st_rejected;
  unsigned long long st_max_overlap_bits;   // double bits of the deepest overlap (monotone for >= 0)
  int st_fail_phase;               // 1 reversal, 2 repair stuck, 3 repair rounds, 4 Lawson rounds, 5 overlap passes
  int vl_need;                     // Verlet rebuild requested for this step
  long long st_verlet_rebuilds;
  long long st_substeps;           // pieces of halved steps that completed
  long long st_tri_visits;         // triangles examined by the check passes
  long long st_exact;              // orientation, in-circle and reversal tests that the FP32
                                   // filters left undecided (decided by the exact grid path)
  long long st_barriers;           // grid barriers passed by the triangulation kernel
  int st_fail_item;                // an offending triangle (repair) or edge corner (reversal)
  int st_fail_count;               // inverted triangles / reversed edges at the failure
  int n_set_moved;                 // disks that bd_set_state moved (its repair runs only if any)
  // wall time of the triangulation kernel's stages as its lead thread sees
  // them (each stage's work plus its closing grid barrier): P check/mark/scan,
  // R inversion repair, F Lawson flips, A apply corrections
  unsigned long long st_stage_ns[5];   // [4]: check passes that visit a list
  long long st_stage_cnt[5];
  // rollout log cursors (not reset per call)
  int log_npass;                   // committed correction passes
  int log_npairs;                  // logged pairs
  int log_overflow;
  int log_step;                    // rollout step being recorded (-1 = none)
  long long step_dev;              // index of the next step (advanced by the triangulation kernel)
  int n_wrapped;                   // periodic box: disks that re-entered in the last move (consumed
                                   // by the triangulation kernel's shift pass; not a statistic)
  int act_n[3];                    // lengths of the rotating triangle lists (zeroed at kernel exit)
  int cl_n[3];                     // lengths of the candidate lists (zeroed at kernel exit)
  unsigned act_gen;                // next list generation (grows across launches)
  // set by the host (bd_set_wait_limit), kept across calls: the time limit of a
  // grid barrier wait (0 = BD_BARRIER_TIMEOUT_NS) and, for tests of the
  // timeout path, the generation of the barrier (1 = the first of a launch) that
  // waits for one block more than the launch has (0 = none)
  unsigned bar_hold;
  unsigned bar_pad;
  unsigned long long bar_limit_ns;
};

// counter slots within BdCtl::cnt[phase % 4]
enum { C_INV = 0, C_REJECT = 1, C_FLIPS = 2, C_OVERLAP = 3, C_CAND = 4, C_LOSE = 5, C_OVADJ = 6 };

// Per-replica parameters (a handle advances R >= 1 independent systems; a
// single system is R = 1).  Device-resident table read by the kernels.
struct BdRep {
  double L, wall_lo, wall_hi;
  // periodic box (Sec. 2.1): the side is a multiple of the position grid and
  // exactly representable in FP32 (Lf), LQ = L / q
  int periodic;
  float Lf, hLf, invLf;
  long long LQ;
  double dt, amp, amp_r, v0;
  double eps, kappa, r_cut, skin, rl2, cell_size;
  double alpha_d[BD_MAX_SPECIES * BD_MAX_SPECIES];   // A[s_i][s_j] at [BD_MAX_SPECIES s_i + s_j]
  float alpha[BD_MAX_SPECIES * BD_MAX_SPECIES];
  unsigned long long seed;
  unsigned int replica;
  int law;
  int ncell, cell_base;          // short range: cells per side, first cell
  int nchunk;                    // long range: j chunks (partial-force slots)
  int slot_begin, slot_end;      // internal disk slots of this replica
  int n;                         // disks
};

struct BdDev {
  // disks (internal order, np slots), then the ghost points of every replica
  double2 *pos, *prev, *pos0;
  float4 *work;            // (x_hi, y_hi, x_lo, y_lo) FP32 pair of each coordinate
  float *theta, *theta0;
  uint8_t *species;        // 255 = empty slot
  int *ext_id;             // index within its replica (-1 = empty slot): the Philox counter
  int *rep_of;             // replica of each slot (-1 = empty slot)
  int *ext_glob;           // each slot's index in the caller's order over all replicas (-1 = empty)
  double2 *xfer_xy;        // [n] state transfers in the caller's order: positions,
  float *xfer_th;          //   directions,
  uint8_t *xfer_sp;        //   species
  uint8_t *moved;
  float2 *dmove;           // position less prev, FP32 (disks with the moved flag; the reversal filter)
  long long *rep_stats;    // [R][3] per-replica counters of a bd_batch_step call: correction passes that
                           // moved the replica, Lawson flips, inverted triangles
  unsigned long long *rep_mark;   // [R] the last correction pass counted for each replica (a stamp
                                  // unique to the pass: never repeats within a handle's life)
  uint8_t *wrap;           // periodic box: re-entries of the last move (bits 0-1 x, 2-3 y; 1 = -L, 3 = +L)
  double2 *disp;
  // polydisperse disks (null when every disk has radius a): per slot its
  // radius and its wall bounds (lo, hi) on the position grid
  double *rad;
  float2 *radf;            // the radius as an FP32 (hi, lo) pair (the short-range law's length scale)
  double2 *wall;
  const BdRep *rep;        // [R]
  // triangulation (corner table), all replicas
  int4 *tv, *tn;
  // undo journal of a triangulation launch: jmark[t] = the launch's stamp
  // (odd, so a cleared 0 matches no launch) once triangle t is journaled,
  // (jtv[t], jtn[t]) its corners and neighbours before the launch changed it
  int4 *jtv, *jtn;
  unsigned *jmark;
  // 2 x nt flip claims: the round of epoch e claims in half e % 2 (so a round
  // can claim for the next while its own claims are read)
  unsigned long long *claim;
  int *vt;                 // per vertex: one corner holding it (kept by the flips)
  // tinv = 1 while a triangle is inverted (set by a check pass, cleared by
  // the triangle's flip); clist = 3 x nt: the triangles that registered a flip
  // candidate for the round of epoch e sit in list e % 3 (BdCtl::cl_n)
  uint8_t *tinv;
  int *clist;
  unsigned *clmark;        // per triangle: the epoch of the candidate list it last joined
  int *act;                // 3 x nt: rotating lists of the triangles a check pass visits
  unsigned *act_mark;      // 3 x nt: generation at which a triangle joined each list
  // force sweep
  int *iperm;              // spatial order of i per block (np_i slots, -1 = none)
  float2 *iorigin;         // per i-block origin (integers)
  uint8_t *tile_species;   // species of each j tile
  int4 *items;             // work items (i block, first tile, end tile, partial slot)
  double2 *fpart;          // [max_nchunk][np] partial forces
  // symmetric sweep (each unordered pair once, both disks updated)
  int4 *sitems;            // (block, first tile, end tile, first j-partial tile)
  int2 *sblock;            // per block: (replica, species)
  float2 *sorigin;         // per block: integer origin for re-centring
  float2 *ipart;           // [item][BD_SB] i-side partial forces
  float2 *jpart;           // [j-partial tile][BD_TJ] j-side partial forces
  int *red_iptr, *red_iidx;  // per block: the items whose i side it is
  int *red_jptr, *red_jidx;  // per tile: the j-partial tiles that hold it
  // short range: Verlet lists (column-major ELL) and the cell grids
  int *vl_idx, *vl_cnt;
  double2 *vl_ref;
  int *cell_count, *cell_start, *cell_cursor, *cell_idx, *cell_of, *scan_sums;
  uint8_t *vc_hit;         // Verlet-list overlap correction: the disk overlapped in the last pass
  // rollout log for the adjoint (null when not recording)
  uint8_t *log_refl;       // [step][np] wall-reflection flags of the Euler-Maruyama move
  uint8_t *log_pflags;     // [pass][np] bit 16: capped; bits 1,2,4,8: reflections of the pass
  int2 *log_pairs;         // overlapping pairs of every committed correction pass
  int *log_pass_begin;     // [pass + 1] first pair of each pass
  int *log_step_pass;      // [step + 1] first pass of each step
  BdCtl *ctl;
};

struct BdConst {
  int n, np, np_i, nt, ntiles, n_iblocks;
  int R;                   // replicas
  int n_items;             // force work items (long range)
  int max_nchunk;          // partial-force slots
  int ncell_total;         // short range: cells of all replicas
  int any_long, any_short;
  int any_periodic;        // some replica has a periodic box
  int precision, n_species;
  double a, sigma;
  double q, inv_q;
  int qshift;              // q = 2^-qshift
  // Algorithm 2's displacement sums over the triangulation edges are added as
  // fixed-point integers (order-independent, so every run sums to the same
  // bits): a value v is held as rint(v * disp_scale), disp_scale = 2^(qshift + F)
  double disp_scale, disp_unscale;
  // force sharding (bd_set_force_shard): the symmetric sweep runs work items
  // [sitem0, sitem0 + n_sitems) of the plan
  int sitem0;
  unsigned long long sig2q_hi, sig2q_lo;  // ceil((sigma/q)^2 (1 + 1e-9)) as 128-bit
  int max_corr_iters, max_flip_rounds;
  int force_variant;       // 0: scalar FP32 sweep, 1: packed f32x2 sweep, 2, 3: symmetric packed sweeps
  int n_sitems;            // symmetric sweep work items
  int overlap_verlet;      // 1: Algorithm 2 over the Verlet lists, no triangulation kept
  int tri_lists;           // check passes after the first of a move: 0 lists when a full pass
                           // is throughput-bound (many triangles per thread), 1 always lists,
                           // 2 always full (environment variable BD_TRI_LISTS at init)
  int tri_fuse;            // 1: a Lawson round tests the outer edges of its flips and keeps the
                           // overlap sums (no check pass between rounds); 0: a check pass after
                           // every round (environment variable BD_TRI_FUSE at init)
  double vl_reach2;        // squared displacement since the list build below which the lists
                           // still hold every pair closer than sigma
  int log_pairs_cap, log_pass_cap;   // rollout log capacities
};

// launchers (kernels_*.cu)
cudaError_t bd_launch_force_long(const BdDev &d, const BdConst &c, cudaStream_t s);
cudaError_t bd_launch_force_long_variant(const BdDev &d, const BdConst &c, int variant, cudaStream_t s);
// node: piece of the step in the heap numbering of halved steps (1 = the whole step)
cudaError_t bd_launch_integrate(const BdDev &d, const BdConst &c, int64_t step, int log_step,
                                cudaStream_t s, int node = 1);
// mode 0: a whole time step; 1: repair after new positions (no correction);
// 2: a piece of a halved step (as 0, but the step counter does not advance)
cudaError_t bd_launch_dt(const BdDev &d, const BdConst &c, int mode, cudaStream_t s, int grid, int block,
                         int log_step = -1);
int bd_dt_grid(int *grid, int *block);
int bd_dt_grid_for(int work_items, int *grid, int *block);
int bd_force_blocks_per_sm(int variant);
cudaError_t bd_launch_work_copy(const BdDev &d, const BdConst &c, cudaStream_t s);
// caller-order positions (and directions) in xfer_* -> checked, grid-rounded slots; a
// disk outside the box sets status BD_ERR_INIT_OVERLAP and nothing is stored
cudaError_t bd_launch_state_in(const BdDev &d, const BdConst &c, int with_theta, cudaStream_t s);
// slots -> caller-order positions, directions and species in xfer_*
cudaError_t bd_launch_state_out(const BdDev &d, const BdConst &c, cudaStream_t s);
// periodic box, after new positions were set (pos0 = old): the re-entry of
// each disk (wrap bytes, n_wrapped) for the triangulation's corner shifts
cudaError_t bd_launch_periodic_wraps(const BdDev &d, const BdConst &c, cudaStream_t s);
cudaError_t bd_launch_force_short(const BdDev &d, const BdConst &c, cudaStream_t s);
int bd_short_launches();
cudaError_t bd_launch_force_sum(const BdDev &d, const BdConst &c, double2 *out, cudaStream_t s);
cudaError_t bd_launch_force_sym(const BdDev &d, const BdConst &c, int variant, cudaStream_t s);
// advance = 0: a piece of a halved step (the step counter does not advance);
// advance = -1: positions set from outside, a pair closer than sigma rejects them
// (BD_ERR_INIT_OVERLAP, restored from pos0) and nothing is corrected
cudaError_t bd_launch_overlap_verlet(const BdDev &d, const BdConst &c, cudaStream_t s, int grid, int block,
                                     int advance = 1);
// a halved step completed: advance the device step counter and the step count
cudaError_t bd_launch_advance_step(const BdDev &d, cudaStream_t s);
// after a timed-out grid barrier: undo the step (or the new positions of
// bd_set_state) from the step-start copies and the undo journal, as their own
// failure path does, and clear the flip claims and list marks the abandoned
// launch may have left
cudaError_t bd_launch_restore_step(const BdDev &d, const BdConst &c, cudaStream_t s);
int bd_vcorr_grid_for(int work_items, int *grid, int *block);
int bd_force_launches(int variant);   // kernel launches of one long-range force evaluation
int bd_force_sym_blocks_per_sm(int variant, int periodic);   // resident blocks of the symmetric sweep
// Philox words and clamped normals (FP32 and FP64 forms) for n counters (uint4 each)
cudaError_t bd_launch_noise_sample(unsigned long long seed, unsigned replica, int n, const void *ctr, void *words,
                                   float *z32, double *z64, cudaStream_t s);
