/*
 * bd.h -- C ABI of the GB300 Brownian hard-disk time stepper.
 *
 * The library advances N hard disks of radius a (diameter sigma = 2a) in a
 * square box [0, L]^2 with reflecting walls or periodic boundaries (Sec. 2.1,
 * bd_params.boundary), following the per-step method
 * of Carter, Hitschfeld, Navarro & Soto, "GPU parallel simulation algorithm
 * of Brownian particles with excluded volume using Delaunay triangulations"
 * (arXiv:1703.02484), Algorithm 1 (Sec. 4.1): forces, Euler-Maruyama update
 * with noise, inverted-triangle check and repair (Sec. 4.3), Delaunay edge
 * flips, and overlap correction over the triangulation edges (Algorithm 2,
 * Sec. 4.4).  Every per-step stage runs in CUDA kernels on one GPU; the only
 * host-side geometry is the initial Delaunay triangulation built once in
 * bd_init, as in the paper (Sec. 4.1).
 *
 * Conventions
 *  - Every int-returning call returns BD_OK (0) or a negative BD_ERR_* code;
 *    bd_strerror() names it.
 *  - Host arrays passed in are copied; the caller keeps ownership.  Output
 *    arrays are caller-allocated host memory of the documented size.
 *  - Device memory is owned by the handle and released by bd_free.
 *  - All work is queued on the CUDA stream given to bd_init (NULL = the
 *    legacy default stream); each call returns after its work has finished.
 *  - After any error other than BD_ERR_ARG / BD_ERR_NOMEM at init the handle
 *    stays usable and holds the last good state (the state before the
 *    rejected step).
 *  - Handles are independent; one handle must not be used from two host
 *    threads at once.
 *  - Coordinates are stored on a dyadic grid (a multiple of 2^-s with
 *    2^-s about 1e-12 L): positions passed in are rounded to it.
 */
#ifndef BD_H
#define BD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  BD_OK = 0,
  BD_ERR_ARG = -1,                 /* invalid argument or parameter */
  BD_ERR_CUDA = -2,                /* a CUDA runtime call failed */
  BD_ERR_INIT_OVERLAP = -3,        /* initial disks overlap or leave the box */
  BD_ERR_STEP_REJECTED = -4,       /* Sec. 4.3: a pair passed through each other,
                                      or an inverted triangle could not be repaired;
                                      the step was undone */
  BD_ERR_OVERLAP_NOT_CONVERGED = -5, /* Algorithm 2 hit max_corr_iters; step undone */
  BD_ERR_FLIP_NOT_CONVERGED = -6,  /* edge flips hit max_flip_rounds; step undone */
  BD_ERR_DEVICE_TIMEOUT = -7,      /* a bounded device-side wait gave up */
  BD_ERR_NOMEM = -8,               /* device or host allocation failed */
  BD_ERR_TRIANGULATION = -9,       /* the initial triangulation could not be built */
  BD_ERR_UNSUPPORTED = -10         /* parameter combination not implemented */
};

enum { BD_LAW_NONE = 0, BD_LAW_LONG = 1, BD_LAW_SHORT = 2 };

/* Simulation parameters.  Sec. 4.2 keeps N, D, dt and sigma in constant
 * memory; the pair-force charges are those of Sec. 2.2. */
typedef struct bd_params {
  int32_t n;             /* number of disks, >= 1 */
  int32_t n_species;     /* 1 to 4 */
  double a;              /* disk radius (> 0); sigma = 2a */
  double box_L;          /* box side; <= 0 => sqrt(n pi a^2 / area_fraction) (Sec. 6) */
  double area_fraction;  /* used only when box_L <= 0 */
  int32_t law;           /* BD_LAW_NONE, BD_LAW_LONG (Sec. 2.2, f = r/r^3, all pairs),
                            BD_LAW_SHORT (WCA core + Yukawa tail, cut at r_cut, Verlet lists) */
  int32_t precision;     /* 0: forces and increments in FP32; 1: in FP64 */
  double alpha[16];      /* long range: the n_species x n_species table A, row-major
                            (A[s_i][s_j] at alpha[s_i * n_species + s_j]; one species: alpha[0]),
                            coefficient of the force ON species s_i FROM species s_j,
                            F_i = sum_j A (r_i - r_j)/|r_ij|^3 (= mu_i alpha_j of Sec. 2.2, which
                            allows any number of species); A > 0 repels */
  double eps, kappa;     /* short range: energy scale and Yukawa inverse length */
  double r_cut, skin;    /* short range: cut-off radius and Verlet skin */
  double D;              /* translational diffusion coefficient */
  double Dr;             /* rotational diffusion coefficient (Sec. 7) */
  double v0;             /* self-propulsion speed (Sec. 7) */
  double dt;             /* time step */
  uint64_t seed;         /* Philox key */
  int32_t replica;       /* xored into the upper key word (independent streams) */
  int32_t max_corr_iters;  /* cap on Algorithm 2 passes per step (default 1000) */
  int32_t max_flip_rounds; /* cap on flip rounds per triangulation update (default 4096) */
  int32_t literal_noise;   /* 1: noise amplitude sqrt(D dt) as printed in Eq. (integration);
                              0 (default): sqrt(2 D dt) per component */
  int64_t step0;         /* index of the first step (Philox counter), for resumed runs */
  int32_t overlap_mode;  /* which pairs Algorithm 2 tests (Sec. 4.4):
                            BD_OVERLAP_DELAUNAY (default): the edges of the Delaunay
                              triangulation maintained every step (Sec. 4.1, 4.3);
                            BD_OVERLAP_VERLET: the Verlet lists of the short-range force
                              (the paper's short-range path, Sec. 5 and Fig. "overlaps"):
                              no triangulation is kept; short-range law only */
  int32_t max_dt_halvings; /* Sec. 4.3: a move rejected because a pair passed through each
                              other (or an inverted triangle could not be repaired, or a disk
                              outran its Verlet list) is "repeated with a lower dt".  0
                              (default): the step is rejected.  H in 1..20: the rejected move
                              is replaced by two moves of half its length, each with forces at
                              its own start and fresh noise (Philox counter word 3 =
                              256 * piece, pieces numbered as a binary heap from the whole
                              step, piece 1, whose noise is unchanged); a rejected half is
                              halved again, down to dt / 2^H.  Single-system handles only
                              (bd_batch_init returns BD_ERR_UNSUPPORTED for H > 0); recorded
                              rollouts (bd_rollout) do not halve. */
  int32_t boundary;        /* BD_BOUNDARY_WALLS (default): reflecting walls, centres in
                              [a, L - a], the triangulation closed by fixed ghost points;
                              BD_BOUNDARY_PERIODIC: the paper's periodic box (Sec. 2.1):
                              centres in [0, L), pair vectors take their minimum image, a disk
                              leaving one side re-enters at the other, and the triangulation
                              is the Delaunay triangulation of the flat torus (Sec. 4.1), kept
                              without ghost points (2n triangles, corners carry image shifts,
                              bd_get_tri_shifts).  L is rounded to the nearest FP32 value.
                              Periodic handles need n >= 16 and L >= 8 sigma; the all-pairs
                              sweeps use their minimum-image forms there; recorded rollouts
                              (bd_rollout) are walls-only. */
  int32_t placement;       /* start positions when bd_init gets xy == NULL:
                              BD_PLACE_RSA (default): random sequential addition of centres in
                              [a, L - a]^2, pairwise at least sigma apart;
                              BD_PLACE_LATTICE: the paper's start (Sec. 4.1): a triangular
                              lattice over [a, L - a]^2 with N* >= n sites (the widest spacing
                              s >= sigma that gives enough), n of them chosen by reservoir
                              sampling, each moved by a uniform offset within (s - sigma)/2
                              (mirrored when it would leave the box) so the set is in general
                              position and no two centres come closer than sigma.  Both draw from Philox streams
                              of `seed` (bd_place_disks gives the same positions). */
} bd_params;

enum { BD_OVERLAP_DELAUNAY = 0, BD_OVERLAP_VERLET = 1 };
enum { BD_BOUNDARY_WALLS = 0, BD_BOUNDARY_PERIODIC = 1 };
enum { BD_PLACE_RSA = 0, BD_PLACE_LATTICE = 1 };

/* Counters of one bd_step call (the paper's per-step metrics, Sec. 6). */
typedef struct bd_step_stats {
  int64_t steps_done;       /* steps completed by this call */
  int64_t corr_iters;       /* Algorithm 2 passes that moved disks, summed over steps */
  int64_t overlap_pairs;    /* overlapping triangulation edges found, summed */
  int64_t flip_rounds;      /* edge-flip rounds that flipped at least one edge */
  int64_t flips;            /* Delaunay (Lawson) flips */
  int64_t repair_flips;     /* inverted-triangle repair flips (Sec. 4.3) */
  int64_t inverted;         /* inverted triangles detected */
  int32_t max_corr_iters;   /* largest number of passes in one step */
  int32_t rejected;         /* 1 if the call stopped at a rejected step */
  int32_t verlet_rebuilds;  /* short range: neighbour-list rebuilds */
  int32_t fail_phase;       /* why a step was undone: 0 none, 1 a pair passed through each other
                               (Sec. 4.3), 2 an inverted triangle had no repair flip, 3 repair
                               rounds exhausted, 4 flip rounds exhausted, 5 correction passes
                               exhausted, 6 a disk outran its Verlet list, 7 positions set by
                               bd_set_state overlap */
  double max_overlap;       /* deepest overlap sigma - r seen */
  int32_t fail_item;        /* internal id of an offending triangle or edge (diagnostic) */
  int32_t fail_count;       /* inverted triangles or reversed edges at the failure */
  int64_t barriers;         /* grid-wide barriers of the device-side loops (all steps) */
  int64_t substeps;         /* moves shorter than dt that completed (max_dt_halvings > 0) */
  int64_t halvings;         /* rejected moves that were replaced by their two halves */
  int64_t tri_visits;       /* triangles examined by the check passes (a pass after the
                               first of a move visits only the triangles near moved
                               disks, flips and overlaps) */
  int64_t exact_tests;      /* orientation, in-circle and pair-reversal tests among disks
                               that the FP32 filters left undecided and the exact
                               integer path decided (near-degenerate inputs: nearly
                               collinear or cocircular points, nearly perpendicular
                               moves); tests with a ghost point are always exact and
                               are not counted */
} bd_step_stats;

typedef struct bd_handle bd_handle;

/* Fill *p with defaults: n=0, one species, a=1, FP32, no forces, D=1, dt=1e-4,
 * max_corr_iters=1000, max_flip_rounds=4096.  Returns BD_OK or BD_ERR_ARG
 * (p == NULL). */
int bd_default_params(bd_params *p);

/* Algorithm 1 lines 1-2 (Sec. 4.1): take the starting positions and build
 * the Delaunay triangulation once on the host, then move everything to the
 * device.
 *   p        parameters (copied).
 *   xy       2n doubles (x0, y0, x1, y1, ...), centres in [a, L-a]^2, no two
 *            closer than 2a; NULL => seeded random sequential addition.
 *   species  n bytes in {0, .., n_species-1}; NULL => all 0.
 *   theta    n floats (self-propulsion directions); NULL => all 0.
 *   stream   cudaStream_t to queue work on; NULL = legacy default stream.
 *   out      receives the handle.
 * Errors: BD_ERR_ARG (bad parameter), BD_ERR_INIT_OVERLAP (overlap or centre
 * outside [a, L-a]), BD_ERR_TRIANGULATION, BD_ERR_NOMEM, BD_ERR_CUDA. */
int bd_init(const bd_params *p, const double *xy, const uint8_t *species, const float *theta,
            void *stream, bd_handle **out);

/* Algorithm 1 lines 3-8: advance nsteps time steps.  Each step is one replay
 * of a CUDA graph holding its launch sequence (captured on first use and
 * again whenever the handle's kernel tables change; the environment variable
 * BD_NO_GRAPH, or a failed capture, selects plain launches instead).  Each step computes the
 * forces (Sec. 2.2), applies Eq. (integration) with truncated Philox noise
 * (Sec. 2.4) and self-propulsion (Sec. 7), reflects at the walls, checks
 * r0.r1 < 0 on every triangulation edge and repairs inverted triangles
 * (Sec. 4.3), restores the Delaunay property by edge flips, and iterates
 * Algorithm 2 (Sec. 4.4) until no triangulation edge is shorter than sigma,
 * re-checking and flipping after every correction pass.  With
 * bd_params.max_dt_halvings > 0 a rejected step is redone as halves (plain
 * launches, one synchronisation per piece) before the call gives up on it.
 *   stats  optional (NULL allowed): counters of this call.
 * Returns BD_OK, or BD_ERR_STEP_REJECTED / BD_ERR_OVERLAP_NOT_CONVERGED /
 * BD_ERR_FLIP_NOT_CONVERGED (the failing step is undone and the call stops;
 * stats->steps_done says how many steps completed), BD_ERR_DEVICE_TIMEOUT,
 * BD_ERR_CUDA, BD_ERR_ARG (nsteps < 0). */
int bd_step(bd_handle *h, int32_t nsteps, bd_step_stats *stats);

/* The counters of the last bd_step, bd_batch_step (the whole batch's) or
 * bd_set_state call on h, in the form bd_step fills: for bd_set_state they
 * describe the repair of the carried-over triangulation (inverted triangles
 * found and repair flips, Sec. 4.3; Lawson flips; filter fall-throughs), with
 * steps_done 0.  Errors: BD_ERR_ARG (NULL argument). */
int bd_last_stats(bd_handle *h, bd_step_stats *stats);

/* The time step's noise for given Philox counters, computed on the device by
 * the same code the step uses (Sec. 2.4; Philox4x32-10 as the stream
 * generator): key (seed mod 2^32, (seed >> 32) xor replica); counter i is
 * counters[4i .. 4i+3] (the step uses (disk, step mod 2^32, step >> 32, tag)).
 *   words      4n words out (NULL to skip): the Philox block of each counter.
 *   normals32  3n floats out (NULL to skip): (xi_x, xi_y, n_theta), each
 *              Box-Muller normal truncated to [-3, 3], as the FP32 step forms them.
 *   normals64  3n doubles out (NULL to skip): the same as the FP64 step forms them.
 * Host arrays; device scratch is allocated and freed inside; synchronous on
 * the legacy default stream.  Errors: BD_ERR_ARG, BD_ERR_NOMEM, BD_ERR_CUDA. */
int bd_noise_sample(uint64_t seed, int32_t replica, int32_t n, const uint32_t *counters, uint32_t *words,
                    float *normals32, double *normals64);

/* Change the caps on the device-side loops of later steps (bd_params
 * max_corr_iters: Algorithm 2 passes per step, Sec. 4.4; max_flip_rounds:
 * inversion-repair and Lawson flip rounds per triangulation update, Sec. 4.3).
 * A step that reaches a cap is undone and bd_step returns
 * BD_ERR_OVERLAP_NOT_CONVERGED or BD_ERR_FLIP_NOT_CONVERGED (repair rounds:
 * BD_ERR_STEP_REJECTED).  Errors: BD_ERR_ARG (a cap below 1). */
int bd_set_loop_caps(bd_handle *h, int32_t max_corr_iters, int32_t max_flip_rounds);

/* Time limit of the device-side waits of h's persistent kernels (the grid
 * barriers of the triangulation kernel and of the Verlet-list correction):
 * a barrier that waits longer sets BD_ERR_DEVICE_TIMEOUT, every block leaves
 * its kernel, and the call that launched it undoes the step (or the new
 * positions of bd_set_state) from its step-start copies and returns
 * BD_ERR_DEVICE_TIMEOUT, the handle usable.  Default 2 s.
 *   seconds       1e-3 .. 60.
 *   hold_barrier  0 for normal use.  k > 0 makes the k-th grid barrier of every
 *                 later launch of those kernels wait for one block more than
 *                 the launch has, so that it runs out: a way to test the
 *                 timeout path that faults nothing (each block gives up after
 *                 `seconds`).  Set it back to 0 to step normally.
 * Errors: BD_ERR_ARG, BD_ERR_CUDA. */
int bd_set_wait_limit(bd_handle *h, double seconds, int32_t hold_barrier);

/* ---- Force sharding over several GPUs (no counterpart in the paper) ----
 * Of one step only the all-pairs force sum divides cleanly among processes:
 * the triangulation stages need every position.  A sharded system runs on
 * every rank in full, each rank computing its share of the symmetric
 * sweep's work items (split by pair count) and all ranks adding their
 * partial forces with one all-reduce per step; every rank then advances the
 * same state with the same forces (the correction's sums are
 * order-independent), so the ranks stay identical.  Per step:
 *   bd_step_begin(h, F)            this rank's partial forces into F,
 *   all-reduce (sum) of F over the ranks (e.g. NCCL, by the caller),
 *   bd_step_end(h, F, stats)       the move and the correction with F.
 *
 * bd_set_force_shard: make h rank `rank` of `world` (world = 1: the whole
 * sweep).  Single-system handles with the long-range law in FP32, without
 * step halving (BD_ERR_UNSUPPORTED otherwise); a one-sided sweep is replaced
 * by the symmetric one.  While world > 1 bd_step returns BD_ERR_UNSUPPORTED
 * and bd_compute_forces returns this rank's partial force.
 * bd_force_slots: the length of F in double2 entries (the handle's internal
 * disk slots, padding included; the layout is the library's).
 * bd_step_begin: F is a DEVICE pointer to 2 * slots doubles, caller-owned;
 *   returns when F holds the partial forces.
 * bd_step_end: F as summed over the ranks (DEVICE, 2 * slots doubles); one
 *   time step as bd_step takes it, with these forces.  Returns as bd_step.
 * Errors: BD_ERR_ARG, BD_ERR_UNSUPPORTED, BD_ERR_CUDA and bd_step's. */
int bd_set_force_shard(bd_handle *h, int32_t rank, int32_t world);
int bd_force_slots(bd_handle *h, int32_t *slots);
int bd_step_begin(bd_handle *h, double *forces);
int bd_step_end(bd_handle *h, const double *forces, bd_step_stats *stats);

/* bd_init for polydisperse disks (Sec. 2.3: the method extends directly to
 * disks whose radii do not differ too much).  Disk i has radius radii[i] in
 * (0, p->a] (p->a is the largest radius; it lays out the ghost points and
 * sizes the cell grids).  A pair overlaps when closer than a_i + a_j; each disk
 * of an overlapping pair moves a_i + a_j - r (Eq. (overlaps)); a disk's summed
 * correction is truncated at half its own radius (Sec. 4.4); centres stay in
 * [a_i, L - a_i] with walls; the short-range law's length scale is a_i + a_j;
 * the long-range law does not involve radii.
 * With BD_OVERLAP_DELAUNAY the radii must satisfy max <= sqrt(2) min: then the
 * overlapping pair with the smallest centre distance is a Delaunay edge (a
 * disk inside its diametral disk would make a closer overlapping pair), so
 * the loop over Delaunay edges still proves that no pair overlaps; wider
 * ratios need BD_OVERLAP_VERLET (short-range law), which tests every listed
 * pair.  Single-system handles; bd_rollout returns BD_ERR_UNSUPPORTED.
 *   xy      required (2n doubles), radii required (n doubles, caller order);
 *           the other arguments as bd_init.
 * Errors: as bd_init; BD_ERR_ARG (a radius outside (0, a], NULL xy or radii),
 * BD_ERR_UNSUPPORTED (radius ratio above sqrt(2) with the Delaunay overlap
 * correction), BD_ERR_INIT_OVERLAP (a pair closer than a_i + a_j, or a centre
 * outside [a_i, L - a_i]). */
int bd_init_radii(const bd_params *p, const double *xy, const uint8_t *species, const float *theta,
                  const double *radii, void *stream, bd_handle **out);

/* Batched replicas (no counterpart in the paper; it serves ensembles of
 * independent systems).  R systems of possibly different N, box, law and
 * parameters advance together: every kernel launch of a step works on all of
 * them (the all-pairs sweep over a work list of (replica, i block, j chunk)
 * items whose chunk size and kernel variant an autotuner picks at init by
 * timing), so a step costs one launch sequence however many replicas there
 * are.  All replicas must share the disk radius a, precision and loop caps.
 *   R        number of replicas (>= 1).
 *   p        R parameter sets; replica r draws its noise from key (p[r].seed,
 *            p[r].replica), so a replica evolves exactly as bd_init would
 *            advance it alone.
 *   xy, species, theta   concatenated per-replica arrays in replica order
 *            (2*sum n, sum n, sum n) or NULL (each replica: RSA from its seed,
 *            species 0, theta 0).
 * bd_step, bd_get_state, bd_set_state and bd_compute_forces then act on the
 * concatenation (external index = replica offset + index within replica);
 * bd_get_replica returns one replica in its own ids.
 * Errors: as bd_init. */
int bd_batch_init(int32_t R, const bd_params *p, const double *xy, const uint8_t *species,
                  const float *theta, void *stream, bd_handle **out);

/* bd_step on a batched handle with per-replica counters (every replica
 * advances the same steps in the same launches).  per_replica (R entries, or
 * NULL) receives, for replica r: corr_iters (Algorithm 2 passes that moved a
 * disk of r), flips (Lawson flips in r's triangulation) and inverted (its
 * inverted triangles detected); the other fields are the batch's (steps done,
 * overlap pairs, flip rounds, repair flips, rejection).  Returns as bd_step. */
int bd_batch_step(bd_handle *h, int32_t nsteps, bd_step_stats *per_replica);

/* One replica of a handle in its own numbering: xy (2n), theta (n), tri
 * (3*n_tri; disks 0..n-1, then its ghost points in bd_ghost_points order),
 * its disk count n and box side L.  Any output may be NULL.
 * Errors: BD_ERR_ARG (bad r), BD_ERR_CUDA. */
int bd_get_replica(bd_handle *h, int32_t r, double *xy, float *theta, int32_t *tri, int32_t *n_tri,
                   int32_t *n, double *L);

/* The all-pairs sweep's tuning: j tiles (256 disks each) per work item, the
 * kernel variant (0 scalar FP32 one-sided, 1 packed f32x2 one-sided, 2 and 3
 * symmetric packed f32x2 -- each unordered pair once -- with 4 warps x 4 or
 * 2 warps x 8 disks per lane) and the number of work items.  Periodic boxes
 * take the minimum-image forms of variants 0, 2 and 3 (1 falls back to 0).
 * bd_init picks the FP32 variant and chunk size by timing the candidates on
 * the device; the environment variables BD_FORCE_VARIANT (0-3) and
 * BD_FORCE_TILES fix them (BD_NCHUNK = k: a single system's one-sided
 * sweeps split each row of tiles into k chunks).  BD_TRI_LISTS selects the
 * triangulation's check passes: 0 (default) the triangles of a list once a
 * full pass has more than four triangles per thread, 1 always lists, 2
 * always full passes. */
int bd_get_tuning(bd_handle *h, int32_t *tiles_per_item, int32_t *variant, int32_t *n_items);

/* Copy the current state to host memory ("Ensure P updated to current
 * time", Algorithm 1).  Any pointer may be NULL to skip that output.  With
 * BD_OVERLAP_VERLET no triangulation is kept: *n_tri is 0 and tri untouched.
 *   xy       2n doubles, external disk order.
 *   theta    n floats.   species  n bytes.
 *   tri      3*n_tri ints: the current Delaunay triangulation of the disks
 *            plus the ghost points of bd_ghost_points (ids n, n+1, ...),
 *            counter-clockwise; the buffer must hold 3*(2(n+G)-6) ints where
 *            G is the ghost count (bd_ghost_points).  Periodic box: the
 *            triangulation of the torus, 2n triangles of disk ids, whose
 *            corner shifts bd_get_tri_shifts gives.
 *   n_tri    receives the number of triangles, 2(n+G)-6 (periodic: 2n).
 *   step     receives the index of the next step.
 * Positions, directions and species are permuted to external order on the
 * device and copied straight into the caller's arrays (one copy each; page-
 * locked arrays make it a direct transfer).  The call returns when the
 * copies are complete.
 * Errors: BD_ERR_ARG (h == NULL), BD_ERR_CUDA. */
int bd_get_state(bd_handle *h, double *xy, float *theta, uint8_t *species, int32_t *tri,
                 int32_t *n_tri, int64_t *step);

/* Replace positions (and, if theta != NULL, directions) with host values in
 * external order, e.g. to resume from a checkpoint.  The triangulation is
 * carried over and repaired on the device (inverted-triangle repair and edge
 * flips, Sec. 4.3), so moves should be small compared with the disk spacing.
 * No two disks may be closer than sigma: the device scans the repaired
 * Delaunay triangulation's edges, which hold the closest pair (Verlet-list
 * handles scan their neighbour lists, rebuilt first when a disk moved more
 * than skin/2 from where they were built).  The arrays are copied to the device as they
 * are (page-locked arrays make it a direct transfer); the range checks (finite;
 * with walls a centre in [a, L-a] up to 1e-9 L), the rounding to the position
 * grid and the permutation to the internal order run there.  Only disks
 * whose grid position changed count as moved: the repair re-tests their
 * triangles, and a state set back unchanged needs no repair.  The call
 * returns when the new state is in place and checked.
 * Errors: BD_ERR_ARG, BD_ERR_INIT_OVERLAP (a centre outside the box, or a
 * pair closer than sigma; state unchanged), BD_ERR_STEP_REJECTED (repair
 * failed; state unchanged), BD_ERR_CUDA. */
int bd_set_state(bd_handle *h, const double *xy, const float *theta);

/* The pair force of Sec. 2.2 (or the short-range law) at the current
 * positions, as the step computes it, summed to FP64: F receives 2n doubles
 * in external order.  Errors: BD_ERR_ARG, BD_ERR_CUDA. */
int bd_compute_forces(bd_handle *h, double *F);

/* Short-range law only: the Verlet lists as last built (Sec. 2.1): disks
 * within r_cut + skin of each disk at the last rebuild, decided in FP64 as
 * (x_i - x_j)^2 + (y_i - y_j)^2 < (r_cut + skin)^2.  counts receives n ints;
 * idx receives, for disk i, its first min(counts[i], max_per) neighbours in
 * ascending external index at idx[i*max_per ...].  Lists are built on the
 * first force evaluation (bd_compute_forces or the first step).
 * Errors: BD_ERR_ARG, BD_ERR_UNSUPPORTED (long-range handle), BD_ERR_CUDA. */
int bd_get_neighbors(bd_handle *h, int32_t max_per, int32_t *counts, int32_t *idx);

/* Periodic box: the image shifts of the triangle corners returned by
 * bd_get_state (or bd_get_replica for replica r; r < 0 = the whole handle).
 * shifts receives 6 bytes per triangle, (sx, sy) for corners 0, 1, 2: corner
 * k of triangle t lies at xy[tri[3t + k]] + L (sx, sy), each in {-1, 0, 1},
 * and corner 0 at shift (0, 0).  With walls every shift is 0.
 * Errors: BD_ERR_ARG, BD_ERR_CUDA. */
int bd_get_tri_shifts(bd_handle *h, int32_t r, int8_t *shifts);

/* Position-grid step q (coordinates are multiples of q) and box side L. */
int bd_get_geometry(bd_handle *h, double *q, double *L);

/* Enable (1) or disable (0) CUDA-event timing of the force kernel launches
 * made by bd_step, and read the accumulated figures: total milliseconds and
 * number of timed launches since the last reset (reset = 1 clears them). */
int bd_force_timing(bd_handle *h, int enable, int reset, double *total_ms, int64_t *launches);

/* Number of kernel launches queued by the last bd_step call. */
int64_t bd_last_launch_count(bd_handle *h);

/* Time spent in the stages of the triangulation kernel by bd_step and
 * bd_rollout since the last reset, as the paper splits a step's time into
 * its stages (Sec. 6): ms[0] the validity check / Lawson marks / overlap scan
 * passes (Sec. 4.3-4.4), ms[1] inversion repair (Sec. 4.3), ms[2] Lawson flip
 * rounds, ms[3] applying the capped corrections (Algorithm 2), ms[4] the part
 * of ms[0] spent in check passes that visit only a list of triangles; each
 * stage's work plus its closing grid barrier, measured on the device clock.
 * phases[k] counts the stage's passes.  ms and phases hold 5 entries; either
 * may be NULL; reset = 1 clears the totals after reading.  The force and
 * integration kernels are separate launches (bd_force_timing covers the
 * force). */
int bd_stage_times(bd_handle *h, int reset, double *ms, int64_t *phases);

/* Start positions as bd_init draws them when it gets xy == NULL (Sec. 4.1
 * placement, bd_params.placement): n centres in [a, L - a]^2, pairwise at
 * least 2a apart, from the Philox streams of seed.  Host only (no GPU).
 *   xy  receives 2n doubles.  With the lattice every site is jittered (an
 *   offset that would leave the box is mirrored), so the start is in general
 *   position.  Errors: BD_ERR_ARG (n < 1, L <= 2a, a <= 0, unknown
 *   placement, or no placement found: the area fraction is too high for the
 *   lattice -- its spacing must exceed 2a by at least 2e-6 a so that the
 *   sites can be jittered -- or random addition jammed). */
int bd_place_disks(int32_t n, double L, double a, int32_t placement, uint64_t seed, double *xy);

/* Host only: the fixed ghost points that close the triangulation of a box of
 * side L for disks of radius a.  The paper's periodic box needs none; with
 * walls they replace the torus and keep the triangles at the walls well
 * shaped.  With C = ceil(L), W = S = ceil(2a) and
 * off(k, s) = ((7919k + 104729s) mod 257)/1024, in this order:
 *   four far corners (-F,-F), (G,-F), (G,G), (-F,G), F = C + 3W, G = 2C + 3W;
 *   bottom row  (x, y) = (-W + kS + off(k,0), -W - off(k,4)),
 *   top row     (-W + kS + off(k,1), C + W + off(k,5)), while -W + kS <= C + W;
 *   left column (-W - off(k,6), -W + S/2 + kS + off(k,2)),
 *   right column (C + W + off(k,7), -W + S/2 + kS + off(k,3)), while the
 *   un-offset y < C + W.
 *   xy     NULL to query the count, else 2*(*count) doubles to fill.
 *   count  in: capacity (points) when xy != NULL; out: number of points.
 * Errors: BD_ERR_ARG. */
int bd_ghost_points(double L, double a, double *xy, int32_t *count);

/* Host only (no GPU needed): the Delaunay triangulation bd_init builds
 * (Sec. 4.1), for n centres in a box of side L (disk radius a) plus the
 * ghost points of bd_ghost_points (ids n, n+1, ...).
 *   xy         2n doubles; centres inside (0, L)^2, no duplicates.
 *   xy_grid    optional 2n doubles: the centres rounded to the position grid
 *              (the coordinates the triangulation is exact for).
 *   tri        3*(2(n+G)-6) ints, counter-clockwise triangles.
 *   n_tri      receives 2(n+G)-6.
 * Errors: BD_ERR_ARG, BD_ERR_TRIANGULATION (duplicate point). */
int bd_triangulate(int32_t n, const double *xy, double L, double a, double *xy_grid, int32_t *tri,
                   int32_t *n_tri);

/* Host only (no GPU needed): the Delaunay triangulation of the flat torus
 * (periodic box, Sec. 2.1 and 4.1) that bd_init builds for
 * boundary = BD_BOUNDARY_PERIODIC, for n >= 3 centres in a box of side L
 * (rounded to FP32 as bd_params.box_L is).
 *   xy         2n doubles, any real coordinates (taken modulo L).
 *   xy_grid    optional 2n doubles: the centres brought into [0, L) on the
 *              position grid (the coordinates the triangulation is exact for).
 *   tri        3*(2n) ints, counter-clockwise triangles of disk ids.
 *   shifts     6*(2n) bytes: (sx, sy) of each corner, corner k of triangle t
 *              at xy_grid[tri[3t + k]] + L (sx, sy); corner 0 at (0, 0).
 *   n_tri      receives 2n.
 * Errors: BD_ERR_ARG, BD_ERR_TRIANGULATION (duplicate point, or a point set
 * whose torus triangulation is not a simplicial complex, e.g. too few points). */
int bd_triangulate_periodic(int32_t n, const double *xy, double L, double *xy_grid, int32_t *tri,
                            int8_t *shifts, int32_t *n_tri);

/* All-pairs long-range force for callers that cannot allocate device memory
 * (no counterpart in the paper; it exists for users whose device memory is
 * owned and budgeted by a host framework's allocator, whose loops cannot
 * afford the device synchronisation of cudaMalloc/cudaFree, or whose device
 * footprint must be fixed when the library is loaded).
 *   n        number of disks, 1 <= n <= 65536 (larger n returns BD_ERR_ARG).
 *   xy       DEVICE pointer, 2n doubles (x0, y0, x1, y1, ...), caller-owned,
 *            16-byte aligned (read as pairs).
 *   species  DEVICE pointer, n bytes, 0 or non-zero (= species 1).
 *   alpha    HOST pointer, 4 doubles A[s_i][s_j] as in bd_params.alpha.
 *   F        DEVICE pointer, 2n doubles, 16-byte aligned: receives
 *            F_i = sum_j A (r_i - r_j)/|r_ij|^3.
 *   stream   cudaStream_t to queue on (NULL = legacy default stream); the call
 *            returns once the work is queued.
 * Allocates nothing: its scratch (about 9 MB) is a static device array that
 * every GPU loading the library holds until exit.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) with the device
 * current; make that first call before any stream capture.  Every call shares
 * the array: calls whose work overlaps on the GPU race and must be serialised.
 * Errors: BD_ERR_ARG (n out of range, NULL pointer, xy or F not 16-byte
 * aligned), BD_ERR_CUDA. */
int bd_forces_noalloc(int32_t n, const double *xy, const uint8_t *species, const double alpha[4],
                      double *F, void *stream);

/* ---- Differentiated rollout (no counterpart in the paper) ----
 * Gradients of a loss of a whole rollout with respect to the pair-force table
 * A (bd_params.alpha, Sec. 2.2) and the self-propulsion speed v0 (Sec. 7), by
 * a hand-written reverse-mode adjoint.  The differentiated map is the time
 * step with its random and discrete choices frozen as the recorded run made
 * them: the Philox noise, the wall reflections of every move, and for every
 * correction pass (Algorithm 2) its overlapping pairs and which disks had
 * their displacement capped at sigma/4.  Rounding to the position grid is
 * taken as the identity.  Long-range law, walls, one or two species and
 * single-system handles only.
 * Pair terms of the adjoint are computed in FP32, every sum in FP64. */

enum { BD_LOSS_MSD = 0, BD_LOSS_HIST = 1 };

/* Replace the force table (alpha: 4 doubles, the table of one or two species
 * as bd_params.alpha, NULL = keep) and the self-propulsion speed (v0; NaN =
 * keep) of every replica.  Discards a recorded rollout.  Errors: BD_ERR_ARG
 * (non-finite alpha), BD_ERR_UNSUPPORTED (alpha given and a replica has more
 * than two species), BD_ERR_CUDA. */
int bd_set_force_params(bd_handle *h, const double *alpha, double v0);

/* Set the index of the next step (the Philox counter of its noise). */
int bd_set_step(bd_handle *h, int64_t step);

/* Advance nsteps steps exactly as bd_step does, recording the frozen choices
 * and a checkpoint (positions, directions) every ckpt_every steps, then form
 * the loss at the final positions x_T against the positions x_0 at the call:
 *   BD_LOSS_MSD:  L = sum over species s of (MSD_s - target)^2,
 *                 MSD_s = mean over disks of species s of |x_T - x_0|^2.
 *   BD_LOSS_HIST: L = sum over bins b of (h_b(x_T) - h_b(x_0))^2, the
 *                 pair-distance histogram of x_T against that of the start:
 *                 h_b(x) = (1/n) sum over pairs i < j of
 *                 exp(-(r_ij - c_b)^2 / (2 s^2)), 32 bins of width a/4 over
 *                 [2a, 10a] (c_b = 2a + (b + 1/2) a/4), s = a/4; pairs
 *                 farther than 12.5a (weight < 1e-24) are skipped; target is
 *                 not used.  Sums in FP64, in a fixed order.
 *   loss   receives L (may be NULL).   stats  as bd_step (may be NULL).
 * Device memory: nsteps*N bytes of reflection flags, N bytes per correction
 * pass, 8 bytes per overlapping pair, 20*N bytes per checkpoint.
 * On a step failure the handle holds the state before the failed step, as
 * bd_step leaves it, and no rollout is recorded.
 * Errors: BD_ERR_ARG (nsteps < 1, ckpt_every < 1), BD_ERR_UNSUPPORTED
 * (short-range law, batched handle, unknown loss_kind), the bd_step errors,
 * BD_ERR_NOMEM, BD_ERR_CUDA. */
int bd_rollout(bd_handle *h, int32_t nsteps, int32_t ckpt_every, int32_t loss_kind, double target,
               double *loss, bd_step_stats *stats);

/* Reverse pass of the last recorded rollout: grad receives 5 doubles,
 * dL/dA00, dL/dA01, dL/dA10, dL/dA11, dL/dv0 (one species: dL/dalpha[0] in
 * slot 0 and zeros in 1..3).  Segments are replayed from their checkpoints;
 * the handle's state is not changed.  May be called more than once.
 * Errors: BD_ERR_ARG (no recorded rollout), BD_ERR_NOMEM, BD_ERR_CUDA. */
int bd_rollout_vjp(bd_handle *h, double *grad);

/* The loss of the recorded rollout replayed with frozen choices from its
 * start with another force table / speed (alpha NULL or v0 NaN = as
 * recorded): the function bd_rollout_vjp differentiates, for finite
 * differences.  The handle's state and recorded rollout are not changed.
 * Errors: BD_ERR_ARG (no recorded rollout), BD_ERR_CUDA. */
int bd_rollout_replay(bd_handle *h, const double *alpha, double v0, double *loss);

/* Positions of the recorded rollout in external order (2n doubles): which = 0
 * the start x_0, which = 1 where the last replay stopped: x_T after
 * bd_rollout_replay (the reverse pass of bd_rollout_vjp ends its replays at
 * the end of the first checkpoint segment).  Errors: BD_ERR_ARG. */
int bd_rollout_positions(bd_handle *h, int32_t which, double *xy);

/* Size of the recorded log: correction passes and overlapping pairs. */
int bd_rollout_log_size(bd_handle *h, int32_t *n_pass, int32_t *n_pairs);

/* sizeof(bd_params) and sizeof(bd_step_stats) as this library was built,
 * for bindings that lay the structures out themselves.  Either pointer may be
 * NULL.  Always BD_OK. */
int bd_struct_sizes(int32_t *params_bytes, int32_t *stats_bytes);

/* Release the handle and its device memory (NULL is ignored). */
void bd_free(bd_handle *h);

/* Static description of a status code. */
const char *bd_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* BD_H */
