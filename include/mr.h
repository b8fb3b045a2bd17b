/*
 * mr.h — C ABI of the GB300 block-based multiresolution solver.
 *
 * The library advances  d_t phi = N(phi)  on a graded quad/octree of blocks
 * (Sroka et al., arXiv:1902.00088).  One call of mr_step() is the paper's time
 * step (Sec. 2.1): refine every block by one level (safety zone), synchronise
 * ghost nodes and evolve with classic RK4 (Sec. 3, Sec. 4), then coarsen blocks
 * whose wavelet details fall below eps (Sec. 2.3).  Everything runs in CUDA
 * kernels on one GPU; the library owns all device memory.
 *
 * Conventions for every entry point
 *   - Return value: MR_OK (0) or an mr_status error code; entry points never
 *     abort.  mr_last_error() gives a static description of the last failure.
 *   - A context lives on one CUDA device (the one current at mr_create) and
 *     enqueues its work on the stream given in mr_params (NULL = legacy default
 *     stream).  Calls return after enqueueing, except where noted
 *     ("synchronises"): those wait for the stream and report device-side
 *     errors (capacity exhausted, broken invariants, non-finite values).
 *   - Host pointers are owned by the caller and only read/written during the
 *     call.  Block lists are exported in canonical order: by tree, then by the
 *     Hilbert index (Skilling 2004) of the block's lower-corner cell on the
 *     tree's finest lattice (the paper orders blocks on a space-filling curve,
 *     Sec. 2.5).
 *   - Field layout of one block: [var][z][y][x] over the Bs^d interior nodes
 *     (block nodes 0..Bs-1 per axis, Sec. 2.2); node (i,j,k) of a block at
 *     level l with block coordinates (cx,cy,cz) sits at
 *     x0 + ((cx*(Bs-1)+i), (cy*(Bs-1)+j), (cz*(Bs-1)+k)) * dx_l,
 *     dx_l = L / (2^l (Bs-1)).
 */
#ifndef MR_H
#define MR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mr_status;
#define MR_OK 0
#define MR_EINVAL 1     /* bad argument or parameter combination */
#define MR_ENOMEM 2     /* device or host allocation failed */
#define MR_ECAPACITY 3  /* block pool or free-slot stack exhausted */
#define MR_ECUDA 4      /* a CUDA runtime call failed */
#define MR_ETIMEOUT 5   /* a bounded device wait gave up */
#define MR_ENAN 6       /* a non-finite value was found in a block norm */
#define MR_EINTERNAL 7  /* a device-side invariant check failed (e.g. non-graded tree) */

/* Arithmetic of the stored fields (Sec. 3 uses FP64 throughout). */
#define MR_PREC_FP64 0       /* y_n, RK accumulator, stage fields and stencils in FP64 */
#define MR_PREC_FP32 1       /* everything FP32 (details optionally FP64) */
#define MR_PREC_FP32_ACC64 2 /* stage fields and stencils FP32; y_n and RK accumulator FP64 */

/* Right-hand sides N(phi) (one kind per context). */
#define MR_RHS_ADV 0    /* -u . grad phi, constant u = rhs[0..2] (Sec. 3 advection equation) */
#define MR_RHS_SWIRL 1  /* -u . grad phi, u of Sec. 3 Eq. (1), t_a = rhs[0]; 2D only */
#define MR_RHS_NS 2     /* compressible Navier-Stokes (Sec. 4) in flux form on q = (rho, rho u,
                           rho v, E); rhs = {gamma, mu, Pr, r_th}; 2D, nvar 4.  r_th > 0: the
                           shock-capturing filter (mr_filter) runs after the RK step of every
                           mr_step and graph step */
#define MR_RHS_NS_SKEW 3  /* the same equations in the skew-symmetric form Sec. 4 uses (Reiss &
                           Sesterhenn 2014) on the square-root variables q = (sqrt(rho),
                           sqrt(rho) u, sqrt(rho) v, p); rhs as for MR_RHS_NS */

/* Initial conditions (evaluated on the device from per-lattice factor tables). */
#define MR_IC_GAUSS 0   /* prod_a exp(-d_a^2/(2 sigma^2)), nearest periodic image:
                           ic = {cx, cy, cz, sigma} (Sec. 3 uses beta = 2 sigma^2) */
#define MR_IC_MIXING 1  /* temporal mixing layer: ic = {delta, U0, Mach, gamma, amp,
                           a_1..a_8, phi_1..phi_8}; rho = 1 */
#define MR_IC_NONE 2    /* no analytic field; blocks come from mr_set_blocks */
#define MR_IC_SHEAR_LAYER 3  /* double shear layer of Sec. 4: layers at x = xc -+ hw, profile
                           s(x) = (tanh((x - xc + hw)/lw) - tanh((x - xc - hw)/lw)) / 2,
                           rho = rho0 + (rho1 - rho0) s, v = v0 + (v1 - v0) s,
                           u = amp sin(2 pi (y - yc)), p = p0;
                           ic = {rho1, rho0, v1, v0, lw, p0, amp, hw, xc, yc}; NS kinds only,
                           stored in the kind's variables (gamma = rhs[0]) */

/* mr_adapt modes (Sec. 2.1 / 2.3). */
#define MR_ADAPT_REFINE_ALL 0      /* every block below Jmax gains one level */
#define MR_ADAPT_REFINE_FLAGGED 1  /* refinement indicators (status +1, Sec. 2.3) from the caller's
                                      mask (mr_set_refine_mask), closed under gradedness (Sec. 2.2:
                                      a leaf one level coarser than a refined block is refined too,
                                      until nothing changes), then refined */
#define MR_ADAPT_COARSEN 2         /* detail thresholding + completeness/gradedness, merge */
#define MR_ADAPT_FLAGS_ONLY 3      /* details and flags of the current grid, no merge (inspection) */
#define MR_ADAPT_PROPOSE 4         /* learned proposal only (needs MR_REFINE_LEARNED): flags = +1
                                      where the network or the exact fallback asks for refinement,
                                      before the gradedness closure; no refinement (inspection and
                                      replay; read with mr_get_flags) */
#define MR_ADAPT_REFINE_STEP 5     /* the refinement mr_step performs: refine all, or (learned mode)
                                      proposal + fallback + gradedness closure + refinement */

typedef struct {
  int32_t dim;          /* 2 or 3 */
  int32_t Bs;           /* block points per direction: 17 or 33 (odd, Sec. 2.2) */
  int32_t ng;           /* ghost layer width: 4 */
  int32_t nvar;         /* variables per node: 1 (advection) or 4 (NS) */
  int32_t precision;    /* MR_PREC_* */
  int32_t detail_fp64;  /* 1: threshold decisions in FP64 (FP32 fields: certified FP32
                           evaluation, FP64 where needed); 0: FP32 details, also for the
                           FP64 state of MR_PREC_FP32_ACC64; MR_PREC_FP64 always FP64 */
  int32_t rhs_kind;     /* MR_RHS_* */
  int32_t ntrees;       /* independent trees advanced together (>= 1) */
  int64_t capacity;     /* pool slots over all trees; a refine-all needs
                           (1 + 2^d) x active blocks transiently */
  int32_t max_rounds;   /* coarsening rounds per adapt; 0 = until stable (<= Jmax - Jmin) */
  int32_t norm_kind;    /* 0: details unnormalised; 1: divided per variable by max |q_v| */
  double L;             /* edge of the periodic domain */
  void* stream;         /* cudaStream_t, NULL = legacy default stream */
} mr_params;

typedef struct {
  int32_t Jmin, Jmax;   /* level range, 1 <= Jmin <= Jmax; level l has 2^l blocks per direction */
  double eps;           /* detail threshold (Sec. 2.3, strict <) */
  double x0[3];         /* domain origin */
  int32_t ic_kind;      /* MR_IC_* */
  double ic[32];        /* IC parameters, see MR_IC_* */
  double rhs[8];        /* RHS parameters, see MR_RHS_* */
} mr_tree_desc;

typedef struct {
  int32_t level;
  int32_t tree;
  uint64_t treecode;     /* Sec. 2.2: one base-2^d digit per level, digit = bx + 2by + 4bz */
  int32_t coords[3];     /* block coordinates at its level */
  int32_t pad;
  uint64_t hilbert_key;  /* Hilbert index of the lower-corner cell at Jmax resolution */
} mr_block_info;

typedef struct mr_ctx_s* mr_ctx;

/* Creates a context with ntrees trees described by trees[0..ntrees-1] and
 * allocates the block pool (capacity slots).  Trees start empty: call
 * mr_init_tree or mr_set_blocks.  Errors: MR_EINVAL (unsupported dim/Bs/ng/
 * nvar/precision/rhs combination, Jmin < 1, Jmax > 10 (2D) / 7 (3D)),
 * MR_ENOMEM, MR_ECUDA.  *out is NULL on failure. */
mr_status mr_create(const mr_params* p, const mr_tree_desc* trees, mr_ctx* out);
void mr_destroy(mr_ctx ctx);
const char* mr_last_error(mr_ctx ctx);

/* Builds the initial grid of every tree (synchronises): uniform at Jmin with the
 * analytic field, then Jmax-Jmin times refine all + analytic field + coarsen
 * until stable.  (The paper does not describe its initialisation.) */
mr_status mr_init_tree(mr_ctx ctx);

/* Sets the RHS parameters of one tree (tree >= 0) or all trees (tree = -1);
 * rhs_params has 8 doubles, meaning per MR_RHS_*.  The kind must equal
 * mr_params.rhs_kind. */
mr_status mr_set_rhs(mr_ctx ctx, int32_t rhs_kind, int32_t tree, const double* rhs_params);

/* Ghost-node synchronisation of the current field (Sec. 2.2, 2.5): same-level
 * copy, fine-to-coarse injection, coarse-to-fine 4th-order interpolating-
 * wavelet prediction; block-edge (conditional) nodes shared with a finer block
 * take the finer value.  The overwritten edge nodes are stored; ghost layers
 * are written to the tile buffer read by mr_get_tiles. */
mr_status mr_sync_ghosts(mr_ctx ctx);

/* One classic RK4 step over all blocks without adaptation (ghosts synchronised
 * before each stage).  t, dt: host arrays of ntrees doubles (time and step of
 * each tree). */
mr_status mr_rk_step(mr_ctx ctx, const double* t, const double* dt);

/* Grid adaptation, mode MR_ADAPT_*.  COARSEN runs rounds of sync + details +
 * flags + merge until no family merges (or max_rounds) and synchronises. */
mr_status mr_adapt(mr_ctx ctx, int32_t mode);

/* One full multiresolution step (Sec. 2.1): refine all, RK4, the shock filter
 * (Navier-Stokes trees with r_th > 0, Sec. 4), coarsen.
 * Synchronises once per coarsening round when max_rounds = 0. */
mr_status mr_step(mr_ctx ctx, const double* t, const double* dt);

/* Shock-capturing filter of Bogey, de Cacqueray & Bailly (2009), which Sec. 4
 * applies after every time step with threshold r_th = rhs[3], on every
 * Navier-Stokes tree with r_th > 0 (others are unchanged).  On the synchronised
 * field, per direction a and node n: dilatation th (2nd-order central
 * differences of u and v), Dth_n = (-th_{n+1} + 2 th_n - th_{n-1}) / 4,
 * M_n = ((Dth_n - Dth_{n+1})^2 + (Dth_n - Dth_{n-1})^2) / 2,
 * r_n = M_n dx^2 / c_n^2 + 1e-16 (c^2 = gamma p / rho),
 * s_n = max(0, 1 - r_th / r_n); every stored variable q becomes
 * q_n - sum_a (s_{n+1/2} F_{n+1/2} - s_{n-1/2} F_{n-1/2}) with
 * F_{n+1/2} = -(q_{n+1} - q_n) / 4 and s_{n+1/2} = (s_n + s_{n+1}) / 2, both
 * directions from the unfiltered field.  MR_EINVAL unless rhs_kind is
 * MR_RHS_NS or MR_RHS_NS_SKEW.  Asynchronous (errors at the next synchronising
 * call). */
mr_status mr_filter(mr_ctx ctx);

/* Number of blocks of a tree (tree = -1: all trees).  Synchronises. */
mr_status mr_num_blocks(mr_ctx ctx, int32_t tree, int64_t* n);

/* Copies the blocks of tree (or all, tree = -1) in canonical order to host
 * buffers of room cap: info (nullable) and fields (nullable, n x nvar x Bs^d
 * doubles, converted from the stored precision).  *n = number of blocks;
 * MR_EINVAL if cap < *n.  Synchronises. */
mr_status mr_get_blocks(mr_ctx ctx, int32_t tree, int64_t cap, int64_t* n,
                        mr_block_info* info, double* fields);

/* Synchronised tiles (n x nvar x (Bs+2ng)^d doubles, ghosts included) of the
 * current field, canonical order.  Runs a ghost synchronisation first.  Synchronises. */
mr_status mr_get_tiles(mr_ctx ctx, int32_t tree, int64_t cap, int64_t* n, double* tiles);

/* Neighbour table (Sec. 2.2: 16 relations in 2D, 74 in 3D): nbr[b*R + r] is the
 * canonical index (within the exported list of the same tree) of relation r of
 * block b, or -1; dl the level difference (neighbour - block).  Relation order:
 * faces, edges, corners (by number of nonzero direction components); directions
 * with x varying fastest; a non-corner direction has one entry for a same-level
 * or coarser neighbour then one per finer block touching the face/edge (x fastest
 * over the free axes); a corner has one entry at any level.  Synchronises. */
mr_status mr_get_neighbors(mr_ctx ctx, int32_t tree, int64_t cap, int32_t* nbr, int8_t* dl);
int32_t mr_num_relations(int32_t dim);

/* Refinement status and largest normalised detail of each block after the last
 * details evaluation (mr_adapt COARSEN or mr_step): flag -2 = merged or can be
 * coarsened, -1 unused, 0 keep, +1 refine.  With FP32 fields and FP64 details
 * (detail_fp64, per-variable normalisation off) the detail is evaluated in
 * FP32 and re-evaluated in FP64 only for blocks whose FP32 value lies within
 * its rounding bound of eps: the flags are those of the FP64 evaluation, and
 * max_detail is the FP64 value for those blocks, the FP32 one (within
 * 32 * 2^-24 * max|field| of it) for the others.  Synchronises. */
mr_status mr_get_flags(mr_ctx ctx, int32_t tree, int64_t cap, int8_t* flags, double* max_detail);

/* Replaces all trees by the given blocks (restart/replay).  n blocks with
 * levels, trees (nullable = all tree 0), coords (n x 3) and fields (nullable =
 * zero; n x nvar x Bs^d doubles), any order.  The grid must be a complete,
 * graded partition of each tree's domain (checked: MR_EINTERNAL).  Synchronises. */
mr_status mr_set_blocks(mr_ctx ctx, int64_t n, const int32_t* level, const int32_t* tree,
                        const int32_t* coords, const double* fields);

/* Per-block refinement mask for MR_ADAPT_REFINE_FLAGGED, canonical order over
 * all trees (n = total block count): +1 refine, 0 keep.  Blocks at Jmax are
 * never refined; the gradedness closure may add blocks. */
mr_status mr_set_refine_mask(mr_ctx ctx, int64_t n, const int8_t* mask);

/* Error of tree against the analytic IC advected by constant u over time t (for
 * the swirl pass t = 0 at t = t_a): out = {L2 abs, L2 of exact, Linf abs, Linf of
 * exact}, unique nodes (each block's last node per axis dropped), weights dx^d.
 * Synchronises. */
mr_status mr_error(mr_ctx ctx, int32_t tree, double t, double* out);

/* Same result as mr_error (up to the rounding of the exact field's exp, which
 * is evaluated on the device here, and the order of the atomic sums) without
 * allocating device memory, for callers that cannot call cudaMalloc/cudaFree:
 * processes whose device memory is fully held by another allocator, or code
 * that must avoid the device synchronisation of cudaFree.  No counterpart in
 * the paper.  Its scratch (three factor tables and four accumulators) lives in
 * one file-scope device array of 3 * 16384 + 4 doubles that every GPU loading
 * the library keeps until exit; (Bs-1) * 2^Jmax of the tree must be <= 16384,
 * else MR_EINVAL.  The call makes the context's device current for its
 * duration (the caller's current device is restored); its first call on a
 * device looks up the array's address there (cudaGetSymbolAddress, once per
 * device even with concurrent host threads): make it before any stream
 * capture.  All calls on a device share the array; the accumulators are cleared
 * at the start of each call, and calls that overlap on the GPU race on it.
 * Synchronises. */
mr_status mr_error_noalloc(mr_ctx ctx, int32_t tree, double t, double* out);

/* Kernel launches enqueued by this process so far (for throughput claims),
 * including the coarsening rounds that graph-captured steps of ctx ran on the
 * device (read from the device: synchronises once graph steps were run). */
int64_t mr_launch_count(mr_ctx ctx);

/* Phase timers and work counters (tracing).  Phases: 0 refine (with the
 * proposal), 1 RK4 stages, 2 details of a coarsening round, 3 flags, merge and
 * list rebuild, 4 synchronisation/export, 5 shock filter (with its copy back
 * into the state).  ms[p] is device time between CUDA
 * events recorded on the context's stream around the phase (only while timing
 * is enabled); stage_blocks counts the blocks processed by all RK stage
 * launches, stage_launches those launches; det_blocks the blocks whose details
 * were evaluated (blocks whose neighbourhood did not change since the previous
 * round reuse theirs), det_launches the host-driven coarsening rounds. */
typedef struct {
  double ms[6];
  int64_t phase_calls[6];
  int64_t stage_launches;
  int64_t stage_blocks;
  int64_t steps;
  int64_t det_launches;
  int64_t det_blocks;
} mr_stats;
mr_status mr_enable_timing(mr_ctx ctx, int32_t on);

/* Graph-captured stepping (batched serving).  The time and step of every tree
 * live on the device (mr_set_time); mr_step_graph enqueues nsteps full steps
 * (refine all, RK4, coarsening rounds, time advance) as replays of one CUDA
 * graph captured at the first call, with no host synchronisation: every launch
 * loops over device-side block counts, and the coarsening rounds (max_rounds, or
 * Jmax - Jmin) become empty once a round merged nothing.  The swirl time factor
 * is evaluated with the device cos in this mode.  Errors are reported by the next
 * synchronising call.  The graph is captured on a private stream and replayed on
 * the context's stream.  In MR_REFINE_LEARNED mode the captured step runs the
 * proposal (features, network, fallback, gradedness closure) and the miss check on
 * the device; mr_set_refine_mode, mr_proposal_set with a new tau and
 * mr_proposal_train make the next call capture the step again.  While training
 * samples are being collected (mr_proposal_collect) this call fails with
 * MR_EINVAL: collection runs in mr_step. */
mr_status mr_set_time(mr_ctx ctx, const double* t, const double* dt);  /* ntrees each; synchronises */
mr_status mr_get_time(mr_ctx ctx, double* t);                          /* synchronises */
mr_status mr_step_graph(mr_ctx ctx, int64_t nsteps);
/* Form of the captured step: 1 = coarsening rounds in a conditional while-node
 * (rounds run only while a family merged), 0 = a fixed number of rounds that
 * become empty once nothing merges (used where conditional nodes are not
 * available), -1 = no graph captured yet. */
int32_t mr_graph_mode(mr_ctx ctx);
/* Launch overlap (off by default): the kernels of a step are launched with
 * programmatic dependent launch, so that each one is scheduled while the
 * previous one finishes; every kernel first waits for its predecessor's
 * completion and memory, so results are identical with the overlap on or off.
 * In captured steps it changed the step time by less than the run-to-run
 * spread (the kernels' own latency dominates, not the launch gaps).
 * Where a graph with such launches cannot be captured or instantiated the
 * context turns the overlap off and captures plain launches.  Setting it drops
 * the captured step.  mr_get_launch_overlap returns 1 / 0 (-1: no context). */
mr_status mr_set_launch_overlap(mr_ctx ctx, int32_t on);
int32_t mr_get_launch_overlap(mr_ctx ctx);
/* Blocks of the adapted grid at the start of every graph step since the last
 * reset (up to 65536 entries); *n = entries recorded.  Synchronises. */
mr_status mr_get_step_history(mr_ctx ctx, int64_t cap, int32_t* out, int64_t* n, int32_t reset);
/* Times graph steps with 1, 2, 3, 4, 6, 8 and occupancy-limited CTAs per SM for
 * the block kernels and, in 2D, both forms of the RK stage (one CTA per block,
 * one warp per block; the second for 17^2 advection blocks only), and for the
 * warp form on FP32 fields 2, 4 or 8 blocks per CTA with the state and
 * accumulator rows staged by bulk copies or loaded (steps steps each; the
 * solution advances during tuning) and keeps the fastest; *best = CTAs per SM
 * (0 = occupancy) + 100 x form + 1000 x blocks per CTA + 10000 x staging.
 * Without tuning the 2D stage on 17^2 blocks uses one warp per block once the
 * grid holds at least 8 blocks per SM, 4 blocks per CTA, rows staged.
 * Synchronises. */
mr_status mr_autotune(mr_ctx ctx, int32_t steps, int32_t* best);
/* Fixes the launch configuration instead of the autotuner: ctas_per_sm
 * persistent CTAs per SM for the block kernels (0 = as many as occupancy
 * allows, at most 32) and the form of the 2D stage and details kernels on 17^2
 * advection blocks (stage_form 1 = one warp per block, 0 = one CTA per block,
 * -1 = by block count: warps once the grid holds 8 blocks per SM).  Results do
 * not depend on either choice.  MR_EINVAL for values out of range or the warp
 * form where it does not exist.  Drops the captured step. */
mr_status mr_set_tuning(mr_ctx ctx, int32_t ctas_per_sm, int32_t stage_form);
/* Warp-per-block form of the 2D stage on FP32 fields: blocks_per_cta (2, 4 or
 * 8 warps per CTA, one block each) and staging (1: the state and accumulator
 * rows of a block are copied to shared memory by the bulk-copy engine while
 * its ghost layer is gathered; 0: loaded by the threads).  Results do not
 * depend on either.  MR_EINVAL for other values.  Drops the captured step. */
mr_status mr_set_warp_form(mr_ctx ctx, int32_t blocks_per_cta, int32_t staging);
/* Synchronises; accumulates pending timers into *out. */
mr_status mr_get_stats(mr_ctx ctx, mr_stats* out);
mr_status mr_reset_stats(mr_ctx ctx);

/* ------------------------------------------------------------------------
 * Learned refinement proposal (2D).  Refine-all (Sec. 2.1 step 1) refines every
 * block for safety; most of that refinement is removed again by the coarsening
 * of the same step.  A small per-block CNN (three 3x3 convolutions with 16
 * channels, the last two with stride 2, ReLU, global max pool, linear, sigmoid;
 * 4961 parameters, FP32 master weights, BF16-rounded weights with FP32
 * accumulation at inference) reads the synchronised tile of a block (channel 0:
 * variable 0 minus its centre value over its largest deviation; channel 1:
 * log10(1e-3 + |d|/(s_v eps)) of the block's details) and predicts p = P(the
 * refinement is kept).  In mode 1 a block below Jmax is refined when p >= tau
 * OR its own largest detail is >= eps (exact fallback); the +1 flags are then
 * closed under gradedness.  After the step a block left unrefined whose details
 * are >= eps counts as a miss (the miss check). */
#define MR_REFINE_ALL 0
#define MR_REFINE_LEARNED 1
mr_status mr_set_refine_mode(mr_ctx ctx, int32_t mode);  /* MR_EINVAL without a network */

/* Training data: while on, every mr_step records (features, label) of each
 * block before the refinement; label 1 iff the refinement was needed: after the
 * step the block's region is subdivided (the refinement was kept), or the block
 * is a leaf again with details >= eps (the miss check's event); 0 otherwise; no
 * label for blocks at Jmax or with own details >= eps (the fallback refines
 * those anyway).
 * capacity: samples to reserve (device memory: capacity x 2 x (Bs+8)^2 floats). */
mr_status mr_proposal_collect(mr_ctx ctx, int32_t on, int64_t capacity);
mr_status mr_proposal_dataset(mr_ctx ctx, int64_t* n_labelled, int64_t* n_positive);

/* Trains on the collected samples with the library's forward/backward kernels
 * and Adam (lr, betas 0.9/0.999): weighted binary cross entropy (positives
 * weighted w_pos; w_pos <= 0 weights them by n_negative / n_positive),
 * mini-batches of `batch` in a fixed interleaved order.  init (nullable, 4961
 * floats): starting parameters (else continue from the current ones).  A
 * `holdout` fraction of each class (every k-th sample) is not trained on; tau
 * is the largest threshold with recall >= `recall` on the held-out positives
 * (with the BF16 inference weights).  Synchronises. */
mr_status mr_proposal_train(mr_ctx ctx, const float* init, int32_t epochs, int32_t batch, float lr,
                            float w_pos, float recall, float holdout, float* tau, float* loss);
mr_status mr_proposal_set(mr_ctx ctx, const float* params /* nullable */, float tau);
mr_status mr_proposal_get(mr_ctx ctx, float* params, float* tau);
/* Counters since the last reset: {blocks below Jmax considered, refined by the
 * network, refined by the fallback only, misses, added by the gradedness closure}. */
mr_status mr_proposal_stats(mr_ctx ctx, int64_t* out5, int32_t reset);
/* Forward and backward of the network on host inputs x (n x 2 x (Bs+8)^2),
 * labels y (n): probabilities, gradient of the mean weighted BCE (4961 floats)
 * and the loss.  Synchronises. */
mr_status mr_cnn_eval(mr_ctx ctx, const float* params, const float* x, const float* y, int64_t n,
                      float w_pos, float* prob, float* grad, float* loss);

#ifdef __cplusplus
}
#endif
#endif /* MR_H */
