// Internal definitions shared by the host API (mr_api.cu) and the kernels
// (mr_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mr.h"

namespace mr {

constexpr int kMaxTrees = 128;
constexpr int kMaxLevel = 11;  // 2D Jmax <= 10, 3D Jmax <= 7 (dense per-level tables)
constexpr int kG = 4;          // ghost layer width

// Device error codes (bit flags OR-ed into Counters::err).
constexpr int kErrCapacity = 1;
constexpr int kErrGraded = 2;    // ring cell without a leaf at l-1..l+1, stencil outside ring
constexpr int kErrNaN = 4;
constexpr int kErrLayout = 8;    // set_blocks: overlap / gap / unsorted input
constexpr int kErrTimeout = 16;

// Entries (int4) of a block's class-box owner table: 7^d class boxes of the
// ring around the block, then one entry of flags.
constexpr int reg_entries(int d) { return (d == 3 ? 343 : 49) + 1; }

// Navier-Stokes right-hand sides (flux form or skew-symmetric form, Sec. 4).
__host__ __device__ constexpr bool is_ns(int kind) { return kind == MR_RHS_NS || kind == MR_RHS_NS_SKEW; }

// Per-tree constants (device copy).
struct TreeDev {
  int32_t Jmin, Jmax;
  double eps;
  float epsf[2];                    // eps rounded down and up to FP32 (certified FP32 decisions)
  int64_t N;                        // finest-lattice intervals per axis: (Bs-1) << Jmax
  int64_t tab_off[kMaxLevel + 1];   // offset of level l's dense slot table
  int64_t lat_off;                  // offset of this tree's lattice tables (N entries each)
  int64_t cell_off;                 // offset of this tree's finest-cell array (2^(d Jmax))
  double cD[kMaxLevel + 1];         // 1 / (12 dx_l)
  float cDf[kMaxLevel + 1];         // cD rounded to FP32 (once, on creation)
  double dx[kMaxLevel + 1];         // dx_l = L / (2^l (Bs-1))
  double rhs[8];
  float rhsf[8];                    // rhs rounded to FP32
  double nsd[4];                    // Navier-Stokes: gamma - 1, mu, kappa = mu gamma / ((gamma - 1) Pr), gamma
  float nsf[4];                     // the same rounded to FP32
  double rth;                       // shock-filter threshold r_th (rhs[3]); <= 0: no filter
  float rthf;                       // r_th rounded to FP32
  float fh2[kMaxLevel + 1];         // FP32 roundings of 1 / (2 dx_l) and dx_l^2 (filter sensor)
  float fdx2[kMaxLevel + 1];
  double x0[3];
  int32_t ic_kind;
  double ic_e0, ic_amp;             // mixing layer: p0/(gamma-1) and perturbation amplitude
  double ic_sl[5];                  // double shear layer: rho1, rho0, v1, v0, p0
};

// Device counters (one instance per context).
struct Counters {
  int32_t n_act;    // active blocks (all trees)
  int32_t n_free;   // free-slot stack height
  int32_t n_new;    // size of the list being built
  int32_t n_alloc;  // slots requested by a refine
  int32_t merged;   // families merged in the last coarsening round
  int32_t err;      // kErr* bits
  int32_t n_round;  // blocks a coarsening round works on (0 once no family merged)
  int32_t done;     // a coarsening round merged nothing: later rounds of the step skip
  unsigned long long stage_blocks;  // blocks processed by RK stage launches
  int32_t hist_n;   // entries written to the step history
  int32_t rounds;   // coarsening rounds run in the current graph step
  int32_t round_id;     // coarsening rounds so far (monotonic); merged mothers are stamped with it
  int32_t first_round;  // the current round is the first of an adapt: every block is evaluated
  unsigned long long det_blocks;  // blocks whose details a coarsening round evaluated
  int32_t topo;       // tree generation: changes with every refinement, merge or import
  int32_t plan_topo;  // generation the stage plans were built for (-1: none)
  unsigned long long graph_rounds;  // coarsening-round bodies run by graph while nodes
  unsigned int ctas_done;  // CTAs of the running commit kernel that finished (last one resets)
};
constexpr int kMaxVar = 4;  // variables per node (advection 1, Navier-Stokes 4; checked at creation)
constexpr int kMaxHist = 1 << 16;  // step history: blocks of the adapted grid before each step

// Device-resident time of every tree (graph-captured steps advance it on the
// device): t, dt, and the RK stage coefficients of the current step.
struct TreeTime {
  double t, dt;
  double ca[4], cy[4], ct[4];
  float caf[4], cyf[4], ctf[4];  // the same rounded to FP32
};

// Lattice tables: per tree, kNumLat tables of N doubles, indexed by the node
// index U in [0, N) on the finest lattice of the tree.
enum LatTable {
  kLatGx = 0, kLatGy, kLatGz,   // Gaussian factors (IC)
  kLatSwA, kLatSwB,             // swirl factors sin^2(pi x), sin(2 pi x)
  kLatNsU, kLatNsE, kLatNsS,    // mixing layer: u(y), exp(-(y/delta)^2), sum_k a_k sin(2 pi k x + phi_k)
  kLatSlS, kLatSlU,             // double shear layer: layer profile s(x), u(y) = amp sin(2 pi (y - yc))
  kNumLat
};

// Per-stage RK4 scalars of every tree, passed by value to the stage kernel.
struct StageArgs {
  double ca[kMaxTrees];   // accumulator coefficient: dt/6, dt/3, dt/3, dt/6
  double cy[kMaxTrees];   // next-stage coefficient: dt/2, dt/2, dt, (unused)
  double ct[kMaxTrees];   // swirl time factor cos(pi t_s / t_a)
  float caf[kMaxTrees], cyf[kMaxTrees], ctf[kMaxTrees];  // the same rounded to FP32
  int32_t copy_state;     // Navier-Stokes stage 3: also store the new state in the stage
                          // type into Yb (the shock filter's source)
};

// Everything a kernel needs to know about the pool and the tree tables.
struct PoolView {
  int dim, Bs, nvar, rhs_kind, norm_kind, prec, ntrees;
  int64_t vs;              // per-variable stride of a block in the pool (elements)
  int64_t cap;             // slots
  const TreeDev* trees;
  int8_t* lvl;             // per slot, -1 unused
  int16_t* tree;
  int32_t* crd;            // per slot x3
  uint64_t* hkey;
  int8_t* f1;              // per slot, first flag pass
  int8_t* flag;            // per slot
  double* md;              // per slot x nvar, max |detail|
  double* mdet;            // per slot
  double* bmax;            // per slot x nvar, max |q_v| of the synchronised interior
  int32_t* act;            // current active list (positions -> slot)
  int32_t* act_next;
  int32_t* freelist;
  int32_t* tab;            // dense per-tree per-level leaf tables (-1 = no leaf)
  const double* lat;       // lattice tables
  const float* latf;       // the same rounded to FP32 (FP32 stage velocities)
  double* svar;            // per tree x nvar threshold scale
  int32_t* cells;          // finest-cell marks (set_blocks validation / ranking)
  int32_t* emit;           // scan input  [cap] x2 (int2)
  int32_t* eoff;           // scan output [cap] x2 (int2)
  int32_t* partial;        // scan partials
  int32_t* pos_of_slot;
  int32_t* stamp;          // per slot: round_id of the round that created the block (merges)
  int32_t* plan;           // per active position: stage plan (slot, level/tree, coords, neighbours)
  int4* regs;              // per active position: class-box owners of a block whose neighbourhood is
                           // not uniform (RingD::NREG entries + flags), built with the stage plan
  Counters* cnt;
  const TreeTime* tt;      // stage coefficients from device memory (graph mode), or null
};

// ---------------------------------------------------------------- launchers --
// Fields are passed as void* and interpreted by prec: y and acc hold the state
// type (double for FP64 / FP32_ACC64, float for FP32), Ya/Yb the stage type
// (double for FP64, float otherwise).  Yn (Navier-Stokes with FP32 stages and
// an FP64 state only, else null): y_n rounded to the stage type, written by the
// first RK stage and read by the next two instead of the FP64 state.
struct Fields {
  void* y;
  void* acc;
  void* Ya;
  void* Yb;
  void* Yn;
};

// Control of the coarsening rounds, folded into the kernel that ends a round:
// it prepares the next round (blocks to evaluate, round id, threshold scales
// reset to svar_v) and, in a captured step (has_h), sets the conditional of
// the while node that repeats the rounds (continue while a family merged and
// fewer than max_rounds ran).
struct RoundCtl {
  double svar_v;
  cudaGraphConditionalHandle h;
  int has_h;
  int max_rounds;
};

struct LaunchCfg {
  int num_sms;
  int grid_mult;  // persistent CTAs per SM for the stage kernel (0 = occupancy)
  int stage_form;  // 2D stage: 0 one CTA per block, 1 one warp per block, -1 by block count
  int n_hint;      // block count last read by the host (chooses the form when -1)
  int pdl;         // step kernels use programmatic dependent launch (launch_k)
  int warp_blocks; // 2D warp-per-block stage on FP32 fields: blocks (warps) per CTA, 2, 4 or 8
  int staging;     // ... and whether its state/accumulator rows are staged by bulk copies (1) or loaded (0)
};

#ifdef __CUDACC__
// First statement of every kernel of the library: wait until the kernels this
// launch depends on have completed and their writes are visible (a no-op for a
// launch without programmatic dependency), then let the next kernel of the
// stream be scheduled, so that its launch overlaps this kernel's execution.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
#endif

// Kernel launch; with pdl the launch may begin before the previous kernel of
// the stream has finished (the kernel waits for it in pdl_enter).  Errors are
// reported through cudaGetLastError like those of a <<< >>> launch.
template <typename... KArgs, typename... Args>
inline void launch_k(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, args...);
}

// Per-dimension launchers (explicitly instantiated in mr_k2*.cu / mr_k3*.cu).
template <int D> void launch_plan(const PoolView& pv, const LaunchCfg& lc, cudaStream_t st);
template <int D> void launch_stage(const PoolView& pv, const Fields& f, int stage,
                                   const StageArgs& sa, const LaunchCfg& lc, cudaStream_t st);
template <int D> void launch_refine(const PoolView& pv, const Fields& f, int mode,
                                    const int8_t* mask, const LaunchCfg& lc, cudaStream_t st);
template <int D> void launch_ic(const PoolView& pv, const Fields& f, const LaunchCfg& lc,
                                cudaStream_t st);
template <int D> void launch_rounds_begin(const PoolView& pv, const LaunchCfg& lc, cudaStream_t st);
template <int D> void launch_coarsen_round(const PoolView& pv, const Fields& f, bool fp64,
                                           bool merge, const RoundCtl& rc, const LaunchCfg& lc, cudaStream_t st);
template <int D> void launch_round_details(const PoolView& pv, const Fields& f, bool fp64,
                                           const LaunchCfg& lc, cudaStream_t st);
template <int D> void launch_round_merge(const PoolView& pv, const Fields& f, bool merge, const RoundCtl& rc,
                                         const LaunchCfg& lc, cudaStream_t st);
template <int D> void launch_sync(const PoolView& pv, const Fields& f, double* tiles,
                                  const LaunchCfg& lc, cudaStream_t st);
template <int D> void launch_neighbors(const PoolView& pv, const int4* rel, int R, int32_t* nbr,
                                       int8_t* dl, const LaunchCfg& lc, cudaStream_t st);
template <int D> void launch_export(const PoolView& pv, const Fields& f, mr_block_info* info,
                                    double* fields, int8_t* flags, double* mdet,
                                    const LaunchCfg& lc, cudaStream_t st);
template <int D> void launch_set_blocks(const PoolView& pv, const Fields& f, int phase, int64_t n,
                                        const int32_t* lvl, const int32_t* tree,
                                        const int32_t* crd, const double* fields, int64_t ncells,
                                        int ntrees, int64_t ntab, const LaunchCfg& lc,
                                        cudaStream_t st);
template <int D> void launch_error(const PoolView& pv, const Fields& f, int tree, const double* ex,
                                   double* out4, const LaunchCfg& lc, cudaStream_t st);
// Navier-Stokes of Sec. 4 (mr_ns.cu): RK stage in the skew-symmetric form
// (2D, B = 17 or 33), and the shock-capturing filter of the state, in place,
// from the copy of the state in the stage type in Yb (written by the last RK
// stage with StageArgs::copy_state, or first by the filter itself with copy);
// it needs the stage plan of the current grid.
template <int B> void launch_stage_nss(const PoolView& pv, const Fields& f, int stage,
                                       const StageArgs& sa, const LaunchCfg& lc, cudaStream_t st);
void launch_filter(const PoolView& pv, const Fields& f, bool copy, const LaunchCfg& lc, cudaStream_t st);

// Exclusive scan of n int2 pairs (emit -> eoff); totals written to tot[0..1].
// n_dev: device count (nullable), else n_host.
// `partial` needs 2 * ceil(n_max / kScanChunk) + 2 ints.
constexpr int kScanChunk = 2048;
void launch_scan2(const int32_t* in, int32_t* out, int32_t* partial, const int32_t* n_dev,
                  int64_t n_host, int32_t* tot, cudaStream_t st, int64_t n_expect = -1, bool pdl = false);
void count_launch(int n = 1);
int64_t kernel_launches();

}  // namespace mr
