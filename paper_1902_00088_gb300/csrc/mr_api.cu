// Host side of the C ABI declared in include/mr.h: parameter validation,
// device memory, per-tree constants and the order of kernel launches that
// makes up a multiresolution step (Sec. 2.1 of Sroka et al., arXiv:1902.00088).
//
// Host code never computes field values.  It only prepares constants once per
// context or per call: per-level coefficients 1/(12 dx), RK4 stage weights
// dt/6, dt/3, dt/2, the swirl time factor cos(pi t_s / t_a), and per-lattice
// tables of 1D transcendental factors (Gaussian, sin^2, tanh profiles) that the
// device kernels multiply together.  Evaluating those factors with the host's
// IEEE libm keeps the GPU fields bit-identical to an FP64 CPU evaluation of the
// same formulas.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "mr_cnn.h"
#include "mr_internal.h"

using namespace mr;

struct mr_ctx_s {
  mr_params p;
  std::vector<mr_tree_desc> td;
  std::vector<TreeDev> tdev;
  int dev = 0;
  cudaStream_t st = nullptr;
  LaunchCfg lc{};
  int64_t S = 0, vs = 0, ntab = 0, ncells = 0, nlat = 0, nscan = 0;
  size_t ts = 8, ty = 8;  // bytes of state / stage types
  // device memory
  void* y = nullptr; void* acc = nullptr; void* Ya = nullptr; void* Yb = nullptr; void* Yn = nullptr;
  int8_t *lvl = nullptr, *f1 = nullptr, *flag = nullptr, *mask = nullptr;
  int16_t* tree = nullptr;
  int32_t* stamp = nullptr;
  int32_t* plan = nullptr;  // S x 32: stage plans of the active blocks
  int4* regs = nullptr;     // S x (NREG + 1): class-box owner tables built with the plans
  int32_t *crd = nullptr, *act = nullptr, *act_next = nullptr, *freelist = nullptr, *tab = nullptr,
          *cells = nullptr, *emit = nullptr, *eoff = nullptr, *partial = nullptr, *pos = nullptr;
  uint64_t* hkey = nullptr;
  double *md = nullptr, *mdet = nullptr, *bmax = nullptr, *lat = nullptr, *svar = nullptr;
  float* latf = nullptr;
  Counters* cnt = nullptr;
  TreeDev* trees = nullptr;
  int4* rel = nullptr;
  int nrel = 0;
  std::vector<void*> owned;
  std::string err;
  bool has_blocks = false;
  // tracing
  bool timing = false;
  struct Pending { int phase; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  mr_stats stats{};
  int64_t stage_launches = 0;
  // graph-captured steps
  TreeTime* ttime = nullptr;
  int32_t* hist = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t body_stream = nullptr;
  bool graph_while = true;  // coarsening rounds as a conditional while-node (else fixed rounds)
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_kernels = 0;  // kernel nodes of the captured step
  int64_t graph_body = 0;     // of which in the while-node body (run once per coarsening round)
  int64_t graph_steps = 0;    // captured steps launched
  bool capturing = false;
  // learned refinement proposal
  int refine_mode = 0;  // 0 refine all (Sec. 2.1), 1 learned proposal + fallback + closure
  float* cnn_w = nullptr; float* cnn_m = nullptr; float* cnn_v = nullptr; float* cnn_g = nullptr;
  __nv_bfloat16* cnn_wb = nullptr;
  float cnn_tau = 0.5f;
  int cnn_t = 0;
  bool cnn_ready = false;
  float *feat = nullptr, *prob = nullptr, *mpre = nullptr;
  int64_t feat_cap = 0;
  int8_t* skip = nullptr;
  int32_t *skip_key = nullptr, *pcounts = nullptr, *changed = nullptr;
  int32_t* gcounts = nullptr;  // proposal counters of graph replays (5, folded into prop_stats)
  int64_t prop_stats[5] = {0, 0, 0, 0, 0};
  bool collect = false;
  float *ds_feat = nullptr, *ds_label = nullptr, *ds_mpre = nullptr;
  int32_t* ds_key = nullptr;
  int64_t ds_cap = 0, ds_n = 0;
};

namespace mr {
__global__ void k_step_begin(Counters* c, int32_t* hist);
__global__ void k_time_coef(TreeTime* tt, const TreeDev* trees, int ntrees, int swirl);
__global__ void k_time_advance(TreeTime* tt, int ntrees);
}

namespace {

mr_status fail(mr_ctx c, mr_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, MR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

// Device buffer owned by one host call, released on every return path
// (stream-ordered when allocated on a stream).
template <typename T>
struct TmpBuf {
  T* p = nullptr;
  cudaStream_t st = nullptr;
  bool async = false;
  TmpBuf() = default;
  TmpBuf(const TmpBuf&) = delete;
  TmpBuf& operator=(const TmpBuf&) = delete;
  ~TmpBuf() {
    if (!p) return;
    if (async) cudaFreeAsync(p, st);
    else cudaFree(p);
  }
  cudaError_t alloc(size_t bytes) { return cudaMalloc((void**)&p, bytes); }
  T* release() {  // hands the buffer to the caller
    T* q = p;
    p = nullptr;
    return q;
  }
  cudaError_t alloc_on(size_t bytes, cudaStream_t s) {
    async = true;
    st = s;
    return cudaMallocAsync((void**)&p, bytes, s);
  }
};

template <typename T>
cudaError_t dalloc(mr_ctx c, T** p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, n ? n * sizeof(T) : 16);
  if (e == cudaSuccess) {
    c->owned.push_back(q);
    *p = (T*)q;
  }
  return e;
}

PoolView view(mr_ctx c) {
  PoolView v{};
  v.dim = c->p.dim; v.Bs = c->p.Bs; v.nvar = c->p.nvar; v.rhs_kind = c->p.rhs_kind;
  v.norm_kind = c->p.norm_kind; v.prec = c->p.precision; v.ntrees = c->p.ntrees;
  v.vs = c->vs; v.cap = c->S; v.trees = c->trees;
  v.lvl = c->lvl; v.tree = c->tree; v.crd = c->crd; v.hkey = c->hkey; v.f1 = c->f1;
  v.flag = c->flag; v.md = c->md; v.mdet = c->mdet; v.bmax = c->bmax; v.act = c->act;
  v.act_next = c->act_next; v.freelist = c->freelist; v.tab = c->tab; v.lat = c->lat; v.latf = c->latf;
  v.svar = c->svar; v.cells = c->cells; v.emit = c->emit; v.eoff = c->eoff;
  v.partial = c->partial; v.pos_of_slot = c->pos; v.cnt = c->cnt; v.stamp = c->stamp;
  v.plan = c->plan;
  v.regs = c->regs;
  return v;
}
Fields fields(mr_ctx c) { return Fields{c->y, c->acc, c->Ya, c->Yb, c->Yn}; }


// RHS-derived per-tree constants (creation and mr_set_rhs).
void rhs_consts(int kind, const double* rhs, TreeDev& td) {
  for (int a = 0; a < 8; ++a) td.rhs[a] = rhs[a];
  for (int a = 0; a < 8; ++a) td.rhsf[a] = (float)rhs[a];
  const double gam = rhs[0], mud = rhs[1], Pr = rhs[2];
  td.nsd[0] = gam - 1.0;
  td.nsd[1] = mud;
  td.nsd[2] = Pr != 0.0 && gam != 1.0 ? mud * gam / ((gam - 1.0) * Pr) : 0.0;
  td.nsd[3] = gam;
  for (int a = 0; a < 4; ++a) td.nsf[a] = (float)td.nsd[a];
  td.rth = is_ns(kind) ? rhs[3] : 0.0;
  td.rthf = (float)td.rth;
}

// 1D factor tables of one tree on its finest lattice (node index U in [0, N)).
void lattice_tables(const mr_params& p, const mr_tree_desc& t, int64_t N, double* out) {
  const double h = p.L / (double)N;
  for (int64_t U = 0; U < N; ++U) {
    double x[3];
    for (int a = 0; a < 3; ++a) x[a] = t.x0[a] + (double)U * h;
    if (t.ic_kind == MR_IC_GAUSS) {
      const double s = t.ic[3];
      for (int a = 0; a < 3; ++a) {
        double dd = (x[a] - 0.0) - t.ic[a];
        while (dd >= 0.5 * p.L) dd -= p.L;
        while (dd < -0.5 * p.L) dd += p.L;
        out[(kLatGx + a) * N + U] = std::exp(-(dd * dd) / (2.0 * s * s));
      }
    }
    if (p.rhs_kind == MR_RHS_SWIRL) {
      const double sv = std::sin(M_PI * x[0]);
      out[kLatSwA * N + U] = sv * sv;
      out[kLatSwB * N + U] = std::sin(2.0 * M_PI * x[0]);
    }
    if (t.ic_kind == MR_IC_SHEAR_LAYER) {
      const double lw = t.ic[4], amp = t.ic[6], hw = t.ic[7], xc = t.ic[8], yc = t.ic[9];
      out[kLatSlS * N + U] = 0.5 * (std::tanh((x[0] - (xc - hw)) / lw) - std::tanh((x[0] - (xc + hw)) / lw));
      out[kLatSlU * N + U] = amp * std::sin(2.0 * M_PI * (x[1] - yc));
    }
    if (t.ic_kind == MR_IC_MIXING) {
      const double delta = t.ic[0], U0 = t.ic[1];
      const double yy = x[1];
      out[kLatNsU * N + U] = U0 * ((std::tanh(2.0 * yy / delta) - std::tanh(2.0 * (yy - 0.5) / delta)) -
                                   std::tanh(2.0 * (yy + 0.5) / delta));
      out[kLatNsE * N + U] = std::exp(-(yy / delta) * (yy / delta));
      double s = 0.0;
      for (int k = 0; k < 8; ++k)
        s += t.ic[5 + k] * std::sin(2.0 * M_PI * (double)(k + 1) * x[0] + t.ic[13 + k]);
      out[kLatNsS * N + U] = s;
    }
  }
}

// Relation list of Sec. 2.2 in the order documented in mr.h.
std::vector<int4> relation_list(int dim) {
  std::vector<int4> r;
  for (int nnz = 1; nnz <= dim; ++nnz)
    for (int sz = (dim == 3 ? -1 : 0); sz <= (dim == 3 ? 1 : 0); ++sz)
      for (int sy = -1; sy <= 1; ++sy)
        for (int sx = -1; sx <= 1; ++sx) {
          if ((sx != 0) + (sy != 0) + (sz != 0) != nnz) continue;
          r.push_back(make_int4(sx, sy, sz, -1));
          if (nnz < dim)
            for (int sub = 0; sub < (1 << (dim - nnz)); ++sub) r.push_back(make_int4(sx, sy, sz, sub));
        }
  return r;
}

mr_status check_device(mr_ctx ctx) {
  CK(cudaStreamSynchronize(ctx->st));
  CK(cudaGetLastError());
  Counters h;
  CK(cudaMemcpy(&h, ctx->cnt, sizeof(h), cudaMemcpyDeviceToHost));
  if (h.err) {
    const int e = h.err;
    cudaMemsetAsync(&ctx->cnt->err, 0, sizeof(int32_t), ctx->st);
    cudaStreamSynchronize(ctx->st);
    if (e & kErrCapacity) return fail(ctx, MR_ECAPACITY, "block pool exhausted (raise capacity)");
    if (e & kErrNaN) return fail(ctx, MR_ENAN, "non-finite value in a block norm");
    if (e & kErrTimeout) return fail(ctx, MR_ETIMEOUT, "device wait timed out");
    if (e & kErrLayout) return fail(ctx, MR_EINTERNAL, "blocks are not a complete, non-overlapping partition");
    return fail(ctx, MR_EINTERNAL, "tree is not graded (level jump > 1 between touching blocks)");
  }
  return MR_OK;
}

Counters read_counters(mr_ctx ctx) {
  Counters h{};
  cudaStreamSynchronize(ctx->st);
  cudaMemcpy(&h, ctx->cnt, sizeof(h), cudaMemcpyDeviceToHost);
  ctx->lc.n_hint = h.n_act;
  return h;
}

template <typename F2, typename F3>
void by_dim(mr_ctx c, F2 f2, F3 f3) {
  if (c->p.dim == 2) f2(); else f3();
}

// Records CUDA events around a phase on the context's stream when timing is on.
struct PhaseTimer {
  mr_ctx c;
  int phase;
  cudaEvent_t a = nullptr, b = nullptr;
  PhaseTimer(mr_ctx c_, int ph) : c(c_), phase(ph) {
    c->stats.phase_calls[ph] += 1;
    if (!c->timing || c->capturing) return;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, c->st);
  }
  ~PhaseTimer() {
    if (!c->timing || c->capturing) return;
    cudaEventRecord(b, c->st);
    c->pending.push_back({phase, a, b});
  }
};

void flush_timers(mr_ctx c) {
  for (auto& p : c->pending) {
    float ms = 0.f;
    cudaEventSynchronize(p.b);
    cudaEventElapsedTime(&ms, p.a, p.b);
    c->stats.ms[p.phase] += ms;
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  c->pending.clear();
}

void do_refine(mr_ctx c, int mode) {
  PhaseTimer tm(c, 0);
  PoolView pv = view(c);
  by_dim(c, [&] { launch_refine<2>(pv, fields(c), mode, c->mask, c->lc, c->st); },
         [&] { launch_refine<3>(pv, fields(c), mode, c->mask, c->lc, c->st); });
}
void do_ic(mr_ctx c) {
  PoolView pv = view(c);
  by_dim(c, [&] { launch_ic<2>(pv, fields(c), c->lc, c->st); },
         [&] { launch_ic<3>(pv, fields(c), c->lc, c->st); });
}
int max_rounds_of(mr_ctx ctx);

// Round control of host-driven rounds (no conditional node).
RoundCtl round_ctl(mr_ctx c, cudaGraphConditionalHandle h = 0, bool has_h = false) {
  RoundCtl rc{};
  rc.svar_v = c->p.norm_kind == 1 ? 0.0 : 1.0;
  rc.h = h;
  rc.has_h = has_h ? 1 : 0;
  rc.max_rounds = max_rounds_of(c);
  return rc;
}

// State of the first coarsening round (later rounds are prepared by the
// kernel that ends the previous one).
void rounds_begin(mr_ctx c, cudaStream_t st) {
  PoolView pv = view(c);
  by_dim(c, [&] { launch_rounds_begin<2>(pv, c->lc, st); }, [&] { launch_rounds_begin<3>(pv, c->lc, st); });
}

void do_round(mr_ctx c, bool merge) {
  PoolView pv = view(c);
  const bool fp64 = c->p.detail_fp64 != 0;
  const RoundCtl rc = round_ctl(c);
  c->stats.det_launches += 1;
  {
    PhaseTimer tm(c, 2);
    by_dim(c, [&] { launch_round_details<2>(pv, fields(c), fp64, c->lc, c->st); },
           [&] { launch_round_details<3>(pv, fields(c), fp64, c->lc, c->st); });
  }
  PhaseTimer tm(c, 3);
  by_dim(c, [&] { launch_round_merge<2>(pv, fields(c), merge, rc, c->lc, c->st); },
         [&] { launch_round_merge<3>(pv, fields(c), merge, rc, c->lc, c->st); });
}

int max_rounds_of(mr_ctx ctx) {
  int jspan = 0;
  for (auto& t : ctx->td) jspan = std::max(jspan, t.Jmax - t.Jmin);
  const int r = ctx->p.max_rounds > 0 ? ctx->p.max_rounds : jspan;
  return r < 1 ? 1 : r;
}

mr_status coarsen_until_stable(mr_ctx ctx) {
  const int rounds = max_rounds_of(ctx);
  launch_k(ctx->lc.pdl, k_step_begin, 1, 1, 0, ctx->st, ctx->cnt, nullptr);
  count_launch();
  rounds_begin(ctx, ctx->st);
  for (int r = 0; r < rounds; ++r) {
    do_round(ctx, true);
    mr_status s = check_device(ctx);
    if (s) return s;
    if (read_counters(ctx).merged == 0) break;
  }
  return MR_OK;
}


// ------------------------------------------------ learned proposal (host) ---
int64_t feat_len(mr_ctx c) {
  const int64_t T = cnn_tile(c->p.Bs);
  return 2 * T * T;
}

mr_status ensure_cnn(mr_ctx ctx) {
  if (ctx->cnn_w) return MR_OK;
  if (ctx->p.dim != 2) return fail(ctx, MR_EINVAL, "the learned proposal is 2D");
  // each buffer joins the context's owned list as it is allocated (a failed
  // call leaks nothing); cnn_w, which marks the set complete, is assigned last
  float* w = nullptr;
  CK(dalloc(ctx, &ctx->cnn_m, kCnnParams));
  CK(dalloc(ctx, &ctx->cnn_v, kCnnParams));
  CK(dalloc(ctx, &ctx->cnn_g, kCnnParams));
  CK(dalloc(ctx, &ctx->cnn_wb, kCnnParams));
  CK(dalloc(ctx, &ctx->skip, ctx->S));
  CK(dalloc(ctx, &ctx->skip_key, ctx->S));
  CK(dalloc(ctx, &ctx->pcounts, 4));
  CK(dalloc(ctx, &ctx->gcounts, 5));
  CK(dalloc(ctx, &w, kCnnParams));
  CK(cudaMemset(ctx->gcounts, 0, 5 * 4));
  CK(cudaMemset(w, 0, kCnnParams * 4));
  CK(cudaMemset(ctx->cnn_m, 0, kCnnParams * 4));
  CK(cudaMemset(ctx->cnn_v, 0, kCnnParams * 4));
  CK(cudaMemset(ctx->cnn_g, 0, kCnnParams * 4));
  CK(cudaMemset(ctx->skip, 0, ctx->S));
  ctx->cnn_w = w;
  return MR_OK;
}

// per-step feature buffer for n blocks (grows; freed with the context)
mr_status ensure_feat(mr_ctx ctx, int64_t n) {
  if (n <= ctx->feat_cap) return MR_OK;
  const int64_t cap = std::max<int64_t>(n, ctx->feat_cap * 2);
  CK(cudaStreamSynchronize(ctx->st));
  if (ctx->feat) { cudaFree(ctx->feat); cudaFree(ctx->prob); cudaFree(ctx->mpre); }
  ctx->feat = nullptr;
  ctx->prob = nullptr;
  ctx->mpre = nullptr;
  ctx->feat_cap = 0;
  CK(cudaMalloc(&ctx->feat, cap * feat_len(ctx) * 4));
  CK(cudaMalloc(&ctx->prob, cap * 4));
  CK(cudaMalloc(&ctx->mpre, cap * 4));
  ctx->feat_cap = cap;
  return MR_OK;
}

// Gradedness closure of the +1 flags (passes until one changes nothing; the
// closure is monotone, so at most one pass per level plus one).
mr_status close_flags(mr_ctx ctx, int8_t* skip, int* added) {
  PoolView pv = view(ctx);
  int jspan = 0;
  for (auto& t : ctx->td) jspan = std::max(jspan, t.Jmax - t.Jmin);
  *added = 0;
  for (int it = 0; it <= jspan + 1; ++it) {
    CK(cudaMemsetAsync(ctx->changed, 0, 4, ctx->st));
    launch_close(pv, skip, ctx->changed, ctx->st);
    int ch = 0;
    CK(cudaMemcpyAsync(&ch, ctx->changed, 4, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    *added += ch;
    if (ch == 0) break;
  }
  return MR_OK;
}

// The learned proposal without refinement: flags = +1 where the network or the
// exact fallback asks for refinement (before the gradedness closure).
mr_status propose_only(mr_ctx ctx) {
  if (ctx->refine_mode != 1 || !ctx->cnn_ready)
    return fail(ctx, MR_EINVAL, "the proposal needs a trained network (mr_set_refine_mode learned)");
  const Counters h = read_counters(ctx);
  mr_status s = ensure_feat(ctx, h.n_act);
  if (s) return s;
  PoolView pv = view(ctx);
  launch_features(pv, ctx->y, ctx->feat, ctx->mpre, 0, ctx->lc.num_sms, ctx->st);
  launch_infer(pv, ctx->p.Bs, ctx->feat, ctx->cnn_wb, ctx->prob, -1, ctx->lc.num_sms, ctx->st);
  CK(cudaMemsetAsync(ctx->pcounts, 0, 16, ctx->st));
  launch_propose(pv, ctx->prob, ctx->mpre, ctx->cnn_tau, ctx->skip, ctx->pcounts, ctx->st);
  return MR_OK;
}

// Refinement by the caller's indicators (mr_set_refine_mask), closed under
// gradedness, then refined.
mr_status refine_flagged(mr_ctx ctx) {
  PoolView pv = view(ctx);
  launch_mask_flags(pv, ctx->mask, ctx->st);
  int added = 0;
  mr_status s = close_flags(ctx, nullptr, &added);
  if (s) return s;
  do_refine(ctx, 2);
  return MR_OK;
}

// Refinement of a step: refine all, or the learned proposal (network or
// fallback), closed under gradedness, with the unrefined blocks remembered for
// the miss check.  Also records training samples when collecting.
mr_status refine_for_step(mr_ctx ctx, int64_t* collected) {
  *collected = 0;
  if (ctx->refine_mode == 0 && !ctx->collect) {
    do_refine(ctx, MR_ADAPT_REFINE_ALL);
    return MR_OK;
  }
  const Counters h = read_counters(ctx);
  const int64_t n = h.n_act;
  PoolView pv = view(ctx);
  float* fbuf = nullptr;
  if (ctx->collect && ctx->ds_n + n <= ctx->ds_cap) {
    fbuf = ctx->ds_feat + ctx->ds_n * feat_len(ctx);
    launch_sample_keys(pv, ctx->ds_key, ctx->ds_n, ctx->st);
    *collected = n;
  }
  mr_status s = ensure_feat(ctx, n);
  if (s) return s;
  launch_features(pv, ctx->y, fbuf ? fbuf : ctx->feat, ctx->mpre, 0, ctx->lc.num_sms, ctx->st);
  if (fbuf) CK(cudaMemcpyAsync(ctx->ds_mpre + ctx->ds_n, ctx->mpre, n * 4, cudaMemcpyDeviceToDevice, ctx->st));
  if (ctx->refine_mode == 0) {
    do_refine(ctx, MR_ADAPT_REFINE_ALL);
    return MR_OK;
  }
  launch_infer(pv, ctx->p.Bs, fbuf ? fbuf : ctx->feat, ctx->cnn_wb, ctx->prob, -1, ctx->lc.num_sms, ctx->st);
  CK(cudaMemsetAsync(ctx->pcounts, 0, 16, ctx->st));
  launch_propose(pv, ctx->prob, ctx->mpre, ctx->cnn_tau, ctx->skip, ctx->pcounts, ctx->st);
  int added = 0;
  s = close_flags(ctx, ctx->skip, &added);
  if (s) return s;
  launch_skip_key(pv, ctx->skip, ctx->skip_key, ctx->st);
  int32_t cnt[4];
  CK(cudaMemcpyAsync(cnt, ctx->pcounts, 16, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (int k = 0; k < 3; ++k) ctx->prop_stats[k] += cnt[k];
  ctx->prop_stats[4] += added;
  do_refine(ctx, 2);
  return MR_OK;
}

mr_status after_step(mr_ctx ctx, int64_t collected) {
  PoolView pv = view(ctx);
  if (collected > 0) {
    launch_label(pv, ctx->ds_key + 4 * ctx->ds_n, ctx->ds_mpre + ctx->ds_n, collected,
                 ctx->ds_label + ctx->ds_n, ctx->st);
    ctx->ds_n += collected;
  }
  if (ctx->refine_mode == 1) {
    CK(cudaMemsetAsync(ctx->pcounts, 0, 16, ctx->st));
    launch_miss_check(pv, ctx->skip, ctx->skip_key, ctx->pcounts, ctx->st);
    int32_t cnt[4];
    CK(cudaMemcpyAsync(cnt, ctx->pcounts, 16, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    ctx->prop_stats[3] += cnt[3];
  }
  return MR_OK;
}

// The shock filter of Sec. 4 runs after the RK step when a Navier-Stokes tree
// has r_th > 0 (needs the stage plan of the current grid).
bool filter_on(mr_ctx ctx) {
  if (!is_ns(ctx->p.rhs_kind)) return false;
  for (auto& t : ctx->tdev)
    if (t.rth > 0.0) return true;
  return false;
}
void do_filter(mr_ctx ctx, cudaStream_t st, bool copy) {
  launch_filter(view(ctx), fields(ctx), copy, ctx->lc, st);
}

mr_status rk_step(mr_ctx ctx, const double* t, const double* dt) {
  PoolView pv = view(ctx);
  const Fields f = fields(ctx);
  by_dim(ctx, [&] { launch_plan<2>(pv, ctx->lc, ctx->st); }, [&] { launch_plan<3>(pv, ctx->lc, ctx->st); });
  PhaseTimer tm(ctx, 1);  // the four stage launches
  ctx->stats.stage_launches += 4;
  const bool filt = filter_on(ctx);
  for (int s = 0; s < 4; ++s) {
    StageArgs sa;
    std::memset(&sa, 0, sizeof(sa));
    sa.copy_state = filt ? 1 : 0;
    for (int k = 0; k < ctx->p.ntrees; ++k) {
      const double h = dt[k];
      const double ca[4] = {h / 6.0, h / 3.0, h / 3.0, h / 6.0};
      const double cy[4] = {h / 2.0, h / 2.0, h, 0.0};
      const double tsv[4] = {t[k], t[k] + 0.5 * h, t[k] + 0.5 * h, t[k] + h};
      sa.ca[k] = ca[s];
      sa.cy[k] = cy[s];
      sa.ct[k] = ctx->p.rhs_kind == MR_RHS_SWIRL ? std::cos(M_PI * tsv[s] / ctx->td[k].rhs[0]) : 0.0;
      sa.caf[k] = (float)sa.ca[k];
      sa.cyf[k] = (float)sa.cy[k];
      sa.ctf[k] = (float)sa.ct[k];
    }
    by_dim(ctx, [&] { launch_stage<2>(pv, f, s, sa, ctx->lc, ctx->st); },
           [&] { launch_stage<3>(pv, f, s, sa, ctx->lc, ctx->st); });
  }
  CK(cudaGetLastError());
  return MR_OK;
}

mr_status set_blocks_dev(mr_ctx ctx, int64_t n, const int32_t* lvl, const int32_t* tree,
                         const int32_t* crd, const double* fld) {
  // Host arrays -> device staging, then the device builds the pool.
  TmpBuf<int32_t> dl, dt, dc;
  TmpBuf<double> df;
  const int nv = ctx->p.nvar;
  int64_t ni = 1;
  for (int a = 0; a < ctx->p.dim; ++a) ni *= ctx->p.Bs;
  CK(dl.alloc_on(std::max<int64_t>(n, 1) * 4, ctx->st));
  CK(dc.alloc_on(std::max<int64_t>(n, 1) * 12, ctx->st));
  if (tree) CK(dt.alloc_on(std::max<int64_t>(n, 1) * 4, ctx->st));
  if (fld) CK(df.alloc_on(std::max<int64_t>(n, 1) * nv * ni * 8, ctx->st));
  CK(cudaMemcpyAsync(dl.p, lvl, n * 4, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(dc.p, crd, n * 12, cudaMemcpyHostToDevice, ctx->st));
  if (tree) CK(cudaMemcpyAsync(dt.p, tree, n * 4, cudaMemcpyHostToDevice, ctx->st));
  if (fld) CK(cudaMemcpyAsync(df.p, fld, n * nv * ni * 8, cudaMemcpyHostToDevice, ctx->st));
  PoolView pv = view(ctx);
  auto phase = [&](int ph) {
    by_dim(ctx,
           [&] { launch_set_blocks<2>(pv, fields(ctx), ph, n, dl.p, dt.p, dc.p, df.p, ctx->ncells, ctx->p.ntrees, ctx->ntab, ctx->lc, ctx->st); },
           [&] { launch_set_blocks<3>(pv, fields(ctx), ph, n, dl.p, dt.p, dc.p, df.p, ctx->ncells, ctx->p.ntrees, ctx->ntab, ctx->lc, ctx->st); });
  };
  phase(1);
  mr_status s0 = check_device(ctx);
  if (s0 == MR_OK) {
    phase(2);
    s0 = check_device(ctx);
  }
  if (s0 != MR_OK) phase(0);  // rejected input: leave an empty, consistent pool
  if (s0 != MR_OK) {
    std::string msg = ctx->err;
    check_device(ctx);
    ctx->err = msg;
    ctx->has_blocks = false;
    return s0;
  }
  mr_status s = check_device(ctx);
  ctx->has_blocks = s == MR_OK;
  return s;
}

int64_t range_of_tree(mr_ctx ctx, int32_t tree, int64_t* first) {
  // blocks are ordered by tree: find [first, first + count) from exported info
  Counters h = read_counters(ctx);
  *first = 0;
  if (tree < 0) return h.n_act;
  std::vector<int16_t> tr(h.n_act);
  std::vector<int32_t> act(h.n_act);
  cudaMemcpy(act.data(), ctx->act, h.n_act * 4, cudaMemcpyDeviceToHost);
  std::vector<int16_t> all(ctx->S);
  cudaMemcpy(all.data(), ctx->tree, ctx->S * 2, cudaMemcpyDeviceToHost);
  int64_t f = -1, n = 0;
  for (int64_t p = 0; p < h.n_act; ++p)
    if (all[act[p]] == tree) {
      if (f < 0) f = p;
      ++n;
    }
  *first = f < 0 ? 0 : f;
  return n;
}

}  // namespace

extern "C" {

const char* mr_last_error(mr_ctx ctx) { return ctx ? ctx->err.c_str() : "null context"; }
int32_t mr_num_relations(int32_t dim) { return dim == 2 ? 16 : (dim == 3 ? 74 : 0); }
int64_t mr_launch_count(mr_ctx ctx) {
  // the host counts one while-node body per graph step; the device counts the
  // bodies that ran
  if (!ctx || ctx->graph_body == 0 || ctx->graph_steps == 0) return kernel_launches();
  const Counters h = read_counters(ctx);
  return kernel_launches() + ((int64_t)h.graph_rounds - ctx->graph_steps) * ctx->graph_body;
}

mr_status mr_create(const mr_params* p, const mr_tree_desc* trees, mr_ctx* out) {
  if (!out) return MR_EINVAL;
  *out = nullptr;
  if (!p || !trees) return MR_EINVAL;
  mr_ctx ctx = new mr_ctx_s();
  ctx->p = *p;
  const mr_params& P = ctx->p;
  auto bad = [&](const char* m) { mr_status s = fail(ctx, MR_EINVAL, m); delete ctx; return s; };
  if (P.dim != 2 && P.dim != 3) return bad("dim must be 2 or 3");
  if (!(P.Bs == 17 || (P.Bs == 33 && P.dim == 2))) return bad("Bs must be 17 (2D/3D) or 33 (2D)");
  if (P.ng != kG) return bad("ng must be 4");
  if (P.ntrees < 1 || P.ntrees > kMaxTrees) return bad("ntrees out of range");
  if (P.precision < 0 || P.precision > 2) return bad("unknown precision");
  if (P.rhs_kind == MR_RHS_SWIRL && P.dim != 2) return bad("swirl is 2D");
  const bool ns = is_ns(P.rhs_kind);
  if (ns && (P.dim != 2 || P.nvar != 4)) return bad("Navier-Stokes is 2D with nvar 4");
  if (P.rhs_kind != MR_RHS_ADV && P.rhs_kind != MR_RHS_SWIRL && !ns) return bad("unknown rhs_kind");
  if (!ns && P.nvar != 1) return bad("advection has nvar 1");
  if (P.capacity < 1 || P.capacity > (1LL << 30)) return bad("capacity out of range");
  if (!(P.L > 0)) return bad("L must be positive");
  const int maxJ = P.dim == 2 ? 10 : 7;
  for (int k = 0; k < P.ntrees; ++k) {
    const mr_tree_desc& t = trees[k];
    if (t.Jmin < 1 || t.Jmax < t.Jmin || t.Jmax > maxJ) return bad("need 1 <= Jmin <= Jmax <= 10 (2D) / 7 (3D)");
    if (t.ic_kind < 0 || t.ic_kind > 3) return bad("unknown ic_kind");
    if (t.ic_kind == MR_IC_GAUSS && !(t.ic[3] > 0)) return bad("Gaussian sigma must be positive");
    if (P.rhs_kind == MR_RHS_SWIRL && !(t.rhs[0] > 0)) return bad("swirl period must be positive");
    if (ns && !(t.rhs[0] > 1.0 && t.rhs[1] >= 0.0 && t.rhs[2] > 0.0))
      return bad("Navier-Stokes needs gamma > 1, mu >= 0, Pr > 0");
    if (ns && t.ic_kind == MR_IC_GAUSS) return bad("Navier-Stokes needs a flow IC or set_blocks");
    if (!ns && (t.ic_kind == MR_IC_MIXING || t.ic_kind == MR_IC_SHEAR_LAYER)) return bad("flow ICs need a Navier-Stokes RHS");
    if (t.ic_kind == MR_IC_MIXING && P.rhs_kind != MR_RHS_NS) return bad("the mixing-layer IC is in flux-form variables");
    if (t.ic_kind == MR_IC_SHEAR_LAYER && !(t.ic[0] > 0 && t.ic[1] > 0 && t.ic[4] > 0 && t.ic[5] > 0))
      return bad("shear layer needs rho1, rho0, lw, p0 > 0");
    ctx->td.push_back(t);
  }
  mr_status st = MR_OK;
  {
    cudaGetDevice(&ctx->dev);
    ctx->st = (cudaStream_t)P.stream;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, ctx->dev) != cudaSuccess) {
      st = fail(ctx, MR_ECUDA, "no CUDA device");
      delete ctx;
      return st;
    }
    ctx->lc.num_sms = prop.multiProcessorCount;
    ctx->lc.grid_mult = 0;
    ctx->lc.stage_form = -1;
    ctx->lc.warp_blocks = 4;
    ctx->lc.staging = 1;
    ctx->lc.pdl = 0;
    ctx->lc.n_hint = 0;
  }
  const int d = P.dim, B = P.Bs, nv = P.nvar;
  int64_t ni = 1;
  for (int a = 0; a < d; ++a) ni *= B;
  ctx->vs = (ni + 3) & ~3LL;
  ctx->S = P.capacity;
  ctx->ts = P.precision == MR_PREC_FP32 ? 4 : 8;
  ctx->ty = P.precision == MR_PREC_FP64 ? 8 : 4;
  // per-tree constants
  int64_t tab = 0, cells = 0, lat = 0;
  for (int k = 0; k < P.ntrees; ++k) {
    const mr_tree_desc& t = ctx->td[k];
    TreeDev td{};
    td.Jmin = t.Jmin; td.Jmax = t.Jmax; td.eps = t.eps;
    {
      const float f = (float)t.eps;
      td.epsf[0] = (double)f > t.eps ? std::nextafter(f, -INFINITY) : f;
      td.epsf[1] = (double)f < t.eps ? std::nextafter(f, INFINITY) : f;
    }
    td.N = (int64_t)(B - 1) << t.Jmax;
    for (int l = 0; l <= kMaxLevel; ++l) {
      td.tab_off[l] = tab;
      if (l <= t.Jmax) tab += (int64_t)1 << (d * l);
      const double dx = P.L / (double)((int64_t)(B - 1) << l);
      td.dx[l] = dx;
      td.cD[l] = 1.0 / (12.0 * dx);
      td.cDf[l] = (float)td.cD[l];
      td.fh2[l] = (float)(0.5 / dx);
      td.fdx2[l] = (float)(dx * dx);
    }
    td.lat_off = lat;
    lat += (int64_t)kNumLat * td.N;
    td.cell_off = cells;
    cells += (int64_t)1 << (d * t.Jmax);
    rhs_consts(P.rhs_kind, t.rhs, td);
    for (int a = 0; a < 3; ++a) td.x0[a] = t.x0[a];
    td.ic_kind = t.ic_kind;
    if (t.ic_kind == MR_IC_MIXING) {
      const double U0 = t.ic[1], Ma = t.ic[2], gam = t.ic[3];
      const double c0 = U0 / Ma;
      const double p0 = c0 * c0 / gam;
      td.ic_e0 = p0 / (gam - 1.0);
      td.ic_amp = t.ic[4];
    }
    if (t.ic_kind == MR_IC_SHEAR_LAYER) {
      td.ic_sl[0] = t.ic[0]; td.ic_sl[1] = t.ic[1]; td.ic_sl[2] = t.ic[2]; td.ic_sl[3] = t.ic[3];
      td.ic_sl[4] = t.ic[5];
    }
    ctx->tdev.push_back(td);
  }
  ctx->ntab = tab;
  ctx->ncells = cells;
  ctx->nlat = lat;
  ctx->nscan = std::max<int64_t>(ctx->S, cells);
  auto alloc_all = [&]() -> cudaError_t {
    cudaError_t e = cudaSuccess;
    const int64_t S = ctx->S;
    if ((e = dalloc(ctx, (char**)&ctx->y, S * nv * ctx->vs * ctx->ts))) return e;
    if ((e = dalloc(ctx, (char**)&ctx->acc, S * nv * ctx->vs * ctx->ts))) return e;
    if ((e = dalloc(ctx, (char**)&ctx->Ya, S * nv * ctx->vs * ctx->ty))) return e;
    if ((e = dalloc(ctx, (char**)&ctx->Yb, S * nv * ctx->vs * ctx->ty))) return e;
    if (P.precision == MR_PREC_FP32_ACC64 && is_ns(P.rhs_kind))
      if ((e = dalloc(ctx, (char**)&ctx->Yn, S * nv * ctx->vs * ctx->ty))) return e;
    if ((e = dalloc(ctx, &ctx->lvl, S))) return e;
    if ((e = dalloc(ctx, &ctx->f1, S))) return e;
    if ((e = dalloc(ctx, &ctx->flag, S))) return e;
    if ((e = dalloc(ctx, &ctx->mask, S))) return e;
    if ((e = dalloc(ctx, &ctx->changed, 1))) return e;
    if ((e = dalloc(ctx, &ctx->tree, S))) return e;
    if ((e = dalloc(ctx, &ctx->crd, 3 * S))) return e;
    if ((e = dalloc(ctx, &ctx->hkey, S))) return e;
    if ((e = dalloc(ctx, &ctx->md, S * nv))) return e;
    if ((e = dalloc(ctx, &ctx->bmax, S * nv))) return e;
    if ((e = dalloc(ctx, &ctx->mdet, S))) return e;
    if ((e = dalloc(ctx, &ctx->act, S))) return e;
    if ((e = dalloc(ctx, &ctx->act_next, S))) return e;
    if ((e = dalloc(ctx, &ctx->freelist, S))) return e;
    if ((e = dalloc(ctx, &ctx->pos, S))) return e;
    if ((e = dalloc(ctx, &ctx->stamp, S))) return e;
    if ((e = cudaMemset(ctx->stamp, 0, S * 4))) return e;
    if ((e = dalloc(ctx, &ctx->plan, S * 32))) return e;
    if ((e = dalloc(ctx, &ctx->regs, S * reg_entries(d)))) return e;
    if ((e = dalloc(ctx, &ctx->tab, ctx->ntab))) return e;
    if ((e = dalloc(ctx, &ctx->cells, 2 * ctx->ncells))) return e;
    if ((e = dalloc(ctx, &ctx->emit, 2 * ctx->nscan))) return e;
    if ((e = dalloc(ctx, &ctx->eoff, 2 * ctx->nscan))) return e;
    if ((e = dalloc(ctx, &ctx->partial, 2 * (ctx->nscan / kScanChunk + 2)))) return e;
    if ((e = dalloc(ctx, &ctx->lat, ctx->nlat))) return e;
    if ((e = dalloc(ctx, &ctx->latf, ctx->nlat))) return e;
    if ((e = dalloc(ctx, &ctx->svar, (int64_t)P.ntrees * nv))) return e;
    if ((e = dalloc(ctx, &ctx->cnt, 1))) return e;
    if ((e = dalloc(ctx, &ctx->trees, P.ntrees))) return e;
    if ((e = dalloc(ctx, &ctx->ttime, P.ntrees))) return e;
    if ((e = dalloc(ctx, &ctx->hist, kMaxHist))) return e;
    if ((e = cudaMemset(ctx->ttime, 0, P.ntrees * sizeof(TreeTime)))) return e;
    std::vector<int4> rel = relation_list(d);
    ctx->nrel = (int)rel.size();
    if ((e = dalloc(ctx, &ctx->rel, rel.size()))) return e;
    if ((e = cudaMemcpy(ctx->rel, rel.data(), rel.size() * sizeof(int4), cudaMemcpyHostToDevice))) return e;
    if ((e = cudaMemcpy(ctx->trees, ctx->tdev.data(), P.ntrees * sizeof(TreeDev), cudaMemcpyHostToDevice))) return e;
    std::vector<double> hl(ctx->nlat, 0.0);
    for (int k = 0; k < P.ntrees; ++k)
      lattice_tables(P, ctx->td[k], ctx->tdev[k].N, hl.data() + ctx->tdev[k].lat_off);
    if ((e = cudaMemcpy(ctx->lat, hl.data(), ctx->nlat * 8, cudaMemcpyHostToDevice))) return e;
    std::vector<float> hf(hl.begin(), hl.end());
    if ((e = cudaMemcpy(ctx->latf, hf.data(), ctx->nlat * 4, cudaMemcpyHostToDevice))) return e;
    if ((e = cudaMemset(ctx->cnt, 0, sizeof(Counters)))) return e;
    const int32_t no_plan = -1;
    if ((e = cudaMemcpy(&ctx->cnt->plan_topo, &no_plan, 4, cudaMemcpyHostToDevice))) return e;
    if ((e = cudaMemset(ctx->mask, 0, S))) return e;
    if ((e = cudaMemset(ctx->lvl, 0xff, S))) return e;
    if ((e = cudaMemset(ctx->tab, 0xff, ctx->ntab * 4))) return e;
    return cudaDeviceSynchronize();
  };
  cudaError_t e = alloc_all();
  if (e != cudaSuccess) {
    st = fail(ctx, e == cudaErrorMemoryAllocation ? MR_ENOMEM : MR_ECUDA, cudaGetErrorString(e));
    cudaGetLastError();
    mr_destroy(ctx);
    return st;
  }
  *out = ctx;
  return MR_OK;
}

void mr_destroy(mr_ctx ctx) {
  if (!ctx) return;
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  else cudaDeviceSynchronize();
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->body_stream) cudaStreamDestroy(ctx->body_stream);
  if (ctx->feat) { cudaFree(ctx->feat); cudaFree(ctx->prob); cudaFree(ctx->mpre); }
  if (ctx->ds_feat) { cudaFree(ctx->ds_feat); cudaFree(ctx->ds_label); cudaFree(ctx->ds_mpre); cudaFree(ctx->ds_key); }
  for (void* q : ctx->owned) cudaFree(q);
  delete ctx;
}

mr_status mr_set_blocks(mr_ctx ctx, int64_t n, const int32_t* level, const int32_t* tree,
                        const int32_t* coords, const double* flds) {
  if (!ctx) return MR_EINVAL;
  if (n < 1 || n > ctx->S || !level || !coords) return fail(ctx, MR_EINVAL, "bad block list");
  return set_blocks_dev(ctx, n, level, tree, coords, flds);
}

mr_status mr_init_tree(mr_ctx ctx) {
  if (!ctx) return MR_EINVAL;
  // uniform grid at Jmin of every tree
  std::vector<int32_t> lv, tr, cr;
  for (int k = 0; k < ctx->p.ntrees; ++k) {
    const int J = ctx->td[k].Jmin;
    const int64_t n = (int64_t)1 << J;
    for (int64_t z = 0; z < (ctx->p.dim == 3 ? n : 1); ++z)
      for (int64_t yy = 0; yy < n; ++yy)
        for (int64_t x = 0; x < n; ++x) {
          lv.push_back(J); tr.push_back(k);
          cr.push_back((int32_t)x); cr.push_back((int32_t)yy); cr.push_back((int32_t)z);
        }
  }
  if ((int64_t)lv.size() > ctx->S) return fail(ctx, MR_ECAPACITY, "capacity below the Jmin grid");
  mr_status s = set_blocks_dev(ctx, (int64_t)lv.size(), lv.data(), tr.data(), cr.data(), nullptr);
  if (s) return s;
  do_ic(ctx);
  int jspan = 0;
  for (auto& t : ctx->td) jspan = std::max(jspan, t.Jmax - t.Jmin);
  for (int it = 0; it < jspan; ++it) {
    do_refine(ctx, MR_ADAPT_REFINE_ALL);
    if ((s = check_device(ctx))) return s;
    do_ic(ctx);
    if ((s = coarsen_until_stable(ctx))) return s;
  }
  return check_device(ctx);
}

namespace {
void drop_graph(mr_ctx ctx);
}

mr_status mr_set_rhs(mr_ctx ctx, int32_t rhs_kind, int32_t tree, const double* rp) {
  if (!ctx || !rp) return MR_EINVAL;
  if (rhs_kind != ctx->p.rhs_kind) return fail(ctx, MR_EINVAL, "rhs kind differs from the context's");
  if (tree < -1 || tree >= ctx->p.ntrees) return fail(ctx, MR_EINVAL, "tree out of range");
  if (is_ns(rhs_kind) && !(rp[0] > 1.0 && rp[1] >= 0.0 && rp[2] > 0.0))
    return fail(ctx, MR_EINVAL, "Navier-Stokes needs gamma > 1, mu >= 0, Pr > 0");
  const bool filtered = filter_on(ctx);
  for (int k = 0; k < ctx->p.ntrees; ++k) {
    if (tree >= 0 && k != tree) continue;
    for (int a = 0; a < 8; ++a) ctx->td[k].rhs[a] = rp[a];
    rhs_consts(rhs_kind, rp, ctx->tdev[k]);
  }
  if (filter_on(ctx) != filtered) drop_graph(ctx);  // a captured step has the filter launch or not
  cudaError_t e = cudaMemcpyAsync(ctx->trees, ctx->tdev.data(), ctx->p.ntrees * sizeof(TreeDev),
                                  cudaMemcpyHostToDevice, ctx->st);
  if (e != cudaSuccess) return fail(ctx, MR_ECUDA, cudaGetErrorString(e));
  if (ctx->p.rhs_kind == MR_RHS_SWIRL) {
    // lattice tables do not depend on the swirl period; nothing else to rebuild
  }
  return cudaStreamSynchronize(ctx->st) == cudaSuccess ? MR_OK : fail(ctx, MR_ECUDA, "sync");
}

mr_status mr_sync_ghosts(mr_ctx ctx) {
  if (!ctx) return MR_EINVAL;
  PoolView pv = view(ctx);
  by_dim(ctx, [&] { launch_sync<2>(pv, fields(ctx), nullptr, ctx->lc, ctx->st); },
         [&] { launch_sync<3>(pv, fields(ctx), nullptr, ctx->lc, ctx->st); });
  return cudaGetLastError() == cudaSuccess ? MR_OK : fail(ctx, MR_ECUDA, "launch");
}

mr_status mr_rk_step(mr_ctx ctx, const double* t, const double* dt) {
  if (!ctx || !t || !dt) return MR_EINVAL;
  return rk_step(ctx, t, dt);
}

mr_status mr_adapt(mr_ctx ctx, int32_t mode) {
  if (!ctx) return MR_EINVAL;
  if (mode == MR_ADAPT_REFINE_ALL) {
    do_refine(ctx, mode);
    return check_device(ctx);
  }
  if (mode == MR_ADAPT_REFINE_FLAGGED) {
    mr_status s = refine_flagged(ctx);
    return s ? s : check_device(ctx);
  }
  if (mode == MR_ADAPT_PROPOSE) {
    mr_status s = propose_only(ctx);
    return s ? s : check_device(ctx);
  }
  if (mode == MR_ADAPT_REFINE_STEP) {
    if (ctx->collect) return fail(ctx, MR_EINVAL, "MR_ADAPT_REFINE_STEP while collecting samples");
    int64_t collected = 0;
    mr_status s = refine_for_step(ctx, &collected);
    return s ? s : check_device(ctx);
  }
  if (mode == MR_ADAPT_COARSEN) return coarsen_until_stable(ctx);
  if (mode == 3) {  // details and flags only (no merge), for inspection
    launch_k(ctx->lc.pdl, k_step_begin, 1, 1, 0, ctx->st, ctx->cnt, nullptr);
    rounds_begin(ctx, ctx->st);
    do_round(ctx, false);
    return check_device(ctx);
  }
  return fail(ctx, MR_EINVAL, "unknown adapt mode");
}

mr_status mr_step(mr_ctx ctx, const double* t, const double* dt) {
  if (!ctx || !t || !dt) return MR_EINVAL;
  ctx->stats.steps += 1;
  int64_t collected = 0;
  mr_status s = refine_for_step(ctx, &collected);
  if (s) return s;
  s = rk_step(ctx, t, dt);
  if (s) return s;
  if (filter_on(ctx)) {
    PhaseTimer tm(ctx, 5);
    do_filter(ctx, ctx->st, false);  // the last RK stage left the state's copy
  }
  s = coarsen_until_stable(ctx);
  if (s) return s;
  return after_step(ctx, collected);
}

mr_status mr_filter(mr_ctx ctx) {
  if (!ctx) return MR_EINVAL;
  if (!is_ns(ctx->p.rhs_kind)) return fail(ctx, MR_EINVAL, "the shock filter needs a Navier-Stokes RHS");
  PoolView pv = view(ctx);
  launch_plan<2>(pv, ctx->lc, ctx->st);
  do_filter(ctx, ctx->st, true);
  CK(cudaGetLastError());
  return MR_OK;
}

mr_status mr_num_blocks(mr_ctx ctx, int32_t tree, int64_t* n) {
  if (!ctx || !n) return MR_EINVAL;
  mr_status s = check_device(ctx);
  if (s) return s;
  int64_t first = 0;
  *n = range_of_tree(ctx, tree, &first);
  return MR_OK;
}

mr_status mr_get_blocks(mr_ctx ctx, int32_t tree, int64_t cap, int64_t* n, mr_block_info* info,
                        double* flds) {
  if (!ctx || !n) return MR_EINVAL;
  mr_status s = check_device(ctx);
  if (s) return s;
  int64_t first = 0;
  const int64_t cnt = range_of_tree(ctx, tree, &first);
  *n = cnt;
  if (cap < cnt) return fail(ctx, MR_EINVAL, "output buffer too small");
  const Counters h = read_counters(ctx);
  int64_t ni = 1;
  for (int a = 0; a < ctx->p.dim; ++a) ni *= ctx->p.Bs;
  const int64_t per = ctx->p.nvar * ni;
  // stream-ordered staging (no device-wide synchronisation of cudaMalloc /
  // cudaFree); one synchronisation after the copies to the host
  TmpBuf<mr_block_info> dinfo;
  TmpBuf<double> dfld;
  CK(dinfo.alloc_on(std::max<int64_t>(h.n_act, 1) * sizeof(mr_block_info), ctx->st));
  if (flds) CK(dfld.alloc_on(std::max<int64_t>(h.n_act, 1) * per * 8, ctx->st));
  PoolView pv = view(ctx);
  by_dim(ctx, [&] { launch_export<2>(pv, fields(ctx), dinfo.p, dfld.p, nullptr, nullptr, ctx->lc, ctx->st); },
         [&] { launch_export<3>(pv, fields(ctx), dinfo.p, dfld.p, nullptr, nullptr, ctx->lc, ctx->st); });
  if (info) CK(cudaMemcpyAsync(info, dinfo.p + first, cnt * sizeof(mr_block_info), cudaMemcpyDeviceToHost, ctx->st));
  if (flds) CK(cudaMemcpyAsync(flds, dfld.p + first * per, cnt * per * 8, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  CK(cudaGetLastError());
  return MR_OK;
}

mr_status mr_get_tiles(mr_ctx ctx, int32_t tree, int64_t cap, int64_t* n, double* tiles) {
  if (!ctx || !n || !tiles) return MR_EINVAL;
  mr_status s = check_device(ctx);
  if (s) return s;
  int64_t first = 0;
  const int64_t cnt = range_of_tree(ctx, tree, &first);
  *n = cnt;
  if (cap < cnt) return fail(ctx, MR_EINVAL, "output buffer too small");
  const Counters h = read_counters(ctx);
  int64_t tile = 1;
  for (int a = 0; a < ctx->p.dim; ++a) tile *= ctx->p.Bs + 2 * ctx->p.ng;
  const int64_t per = ctx->p.nvar * tile;
  TmpBuf<double> dt;
  CK(dt.alloc(std::max<int64_t>(h.n_act, 1) * per * 8));
  PoolView pv = view(ctx);
  by_dim(ctx, [&] { launch_sync<2>(pv, fields(ctx), dt.p, ctx->lc, ctx->st); },
         [&] { launch_sync<3>(pv, fields(ctx), dt.p, ctx->lc, ctx->st); });
  s = check_device(ctx);
  if (!s) CK(cudaMemcpy(tiles, dt.p + first * per, cnt * per * 8, cudaMemcpyDeviceToHost));
  return s;
}

mr_status mr_get_neighbors(mr_ctx ctx, int32_t tree, int64_t cap, int32_t* nbr, int8_t* dl) {
  if (!ctx || !nbr || !dl) return MR_EINVAL;
  mr_status s = check_device(ctx);
  if (s) return s;
  int64_t first = 0;
  const int64_t cnt = range_of_tree(ctx, tree, &first);
  if (cap < cnt) return fail(ctx, MR_EINVAL, "output buffer too small");
  const Counters h = read_counters(ctx);
  const int R = ctx->nrel;
  TmpBuf<int32_t> dn;
  TmpBuf<int8_t> dd;
  CK(dn.alloc(std::max<int64_t>(h.n_act, 1) * R * 4));
  CK(dd.alloc(std::max<int64_t>(h.n_act, 1) * R));
  // position of every slot in the list
  std::vector<int32_t> act(h.n_act), pos(ctx->S, -1);
  CK(cudaMemcpy(act.data(), ctx->act, h.n_act * 4, cudaMemcpyDeviceToHost));
  for (int64_t p = 0; p < h.n_act; ++p) pos[act[p]] = (int32_t)(p - first);
  CK(cudaMemcpy(ctx->pos, pos.data(), ctx->S * 4, cudaMemcpyHostToDevice));
  PoolView pv = view(ctx);
  by_dim(ctx, [&] { launch_neighbors<2>(pv, ctx->rel, R, dn.p, dd.p, ctx->lc, ctx->st); },
         [&] { launch_neighbors<3>(pv, ctx->rel, R, dn.p, dd.p, ctx->lc, ctx->st); });
  CK(cudaStreamSynchronize(ctx->st));
  CK(cudaMemcpy(nbr, dn.p + first * R, cnt * R * 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(dl, dd.p + first * R, cnt * R, cudaMemcpyDeviceToHost));
  return MR_OK;
}

mr_status mr_get_flags(mr_ctx ctx, int32_t tree, int64_t cap, int8_t* flg, double* mdet) {
  if (!ctx) return MR_EINVAL;
  mr_status s = check_device(ctx);
  if (s) return s;
  int64_t first = 0;
  const int64_t cnt = range_of_tree(ctx, tree, &first);
  if (cap < cnt) return fail(ctx, MR_EINVAL, "output buffer too small");
  const Counters h = read_counters(ctx);
  TmpBuf<int8_t> df;
  TmpBuf<double> dm;
  CK(df.alloc(std::max<int64_t>(h.n_act, 1)));
  CK(dm.alloc(std::max<int64_t>(h.n_act, 1) * 8));
  PoolView pv = view(ctx);
  by_dim(ctx, [&] { launch_export<2>(pv, fields(ctx), nullptr, nullptr, df.p, dm.p, ctx->lc, ctx->st); },
         [&] { launch_export<3>(pv, fields(ctx), nullptr, nullptr, df.p, dm.p, ctx->lc, ctx->st); });
  CK(cudaStreamSynchronize(ctx->st));
  if (flg) CK(cudaMemcpy(flg, df.p + first, cnt, cudaMemcpyDeviceToHost));
  if (mdet) CK(cudaMemcpy(mdet, dm.p + first, cnt * 8, cudaMemcpyDeviceToHost));
  return MR_OK;
}

mr_status mr_set_refine_mask(mr_ctx ctx, int64_t n, const int8_t* mask) {
  if (!ctx || !mask) return MR_EINVAL;
  const Counters h = read_counters(ctx);
  if (n != h.n_act) return fail(ctx, MR_EINVAL, "mask length differs from the block count");
  CK(cudaMemcpyAsync(ctx->mask, mask, n, cudaMemcpyHostToDevice, ctx->st));
  return check_device(ctx);
}

mr_status mr_error(mr_ctx ctx, int32_t tree, double t, double* out) {
  if (!ctx || !out || tree < 0 || tree >= ctx->p.ntrees) return MR_EINVAL;
  const mr_tree_desc& td = ctx->td[tree];
  if (td.ic_kind != MR_IC_GAUSS) return fail(ctx, MR_EINVAL, "error needs the Gaussian IC");
  const int64_t N = ctx->tdev[tree].N;
  const double h = ctx->p.L / (double)N;
  std::vector<double> ex(3 * N, 1.0);
  for (int a = 0; a < ctx->p.dim; ++a) {
    const double shift = ctx->p.rhs_kind == MR_RHS_ADV ? td.rhs[a] * t : 0.0;
    for (int64_t U = 0; U < N; ++U) {
      const double x = td.x0[a] + (double)U * h;
      double dd = (x - shift) - td.ic[a];
      while (dd >= 0.5 * ctx->p.L) dd -= ctx->p.L;
      while (dd < -0.5 * ctx->p.L) dd += ctx->p.L;
      const double s = td.ic[3];
      ex[a * N + U] = std::exp(-(dd * dd) / (2.0 * s * s));
    }
  }
  TmpBuf<double> dex, dout;
  CK(dex.alloc(3 * N * 8));
  CK(dout.alloc(4 * 8));
  CK(cudaMemcpy(dex.p, ex.data(), 3 * N * 8, cudaMemcpyHostToDevice));
  CK(cudaMemset(dout.p, 0, 32));
  PoolView pv = view(ctx);
  by_dim(ctx, [&] { launch_error<2>(pv, fields(ctx), tree, dex.p, dout.p, ctx->lc, ctx->st); },
         [&] { launch_error<3>(pv, fields(ctx), tree, dex.p, dout.p, ctx->lc, ctx->st); });
  CK(cudaStreamSynchronize(ctx->st));
  double o[4];
  CK(cudaMemcpy(o, dout.p, 32, cudaMemcpyDeviceToHost));
  out[0] = std::sqrt(o[0]); out[1] = std::sqrt(o[1]); out[2] = o[2]; out[3] = o[3];
  return MR_OK;
}

mr_status mr_set_time(mr_ctx ctx, const double* t, const double* dt) {
  if (!ctx || !t || !dt) return MR_EINVAL;
  std::vector<TreeTime> h(ctx->p.ntrees);
  for (int k = 0; k < ctx->p.ntrees; ++k) {
    h[k] = TreeTime{};
    h[k].t = t[k];
    h[k].dt = dt[k];
  }
  CK(cudaStreamSynchronize(ctx->st));
  CK(cudaMemcpy(ctx->ttime, h.data(), h.size() * sizeof(TreeTime), cudaMemcpyHostToDevice));
  return MR_OK;
}

mr_status mr_get_time(mr_ctx ctx, double* t) {
  if (!ctx || !t) return MR_EINVAL;
  std::vector<TreeTime> h(ctx->p.ntrees);
  CK(cudaStreamSynchronize(ctx->st));
  CK(cudaMemcpy(h.data(), ctx->ttime, h.size() * sizeof(TreeTime), cudaMemcpyDeviceToHost));
  for (int k = 0; k < ctx->p.ntrees; ++k) t[k] = h[k].t;
  return MR_OK;
}

namespace {
// One step with no host synchronisation, for capture: time coefficients from
// the device, refine all, four stages, a fixed number of coarsening rounds that
// become empty once a round merged nothing, time advance.
void enqueue_graph_prologue(mr_ctx ctx, cudaStream_t st) {
  PoolView pv = view(ctx);
  pv.tt = ctx->ttime;
  const Fields f = fields(ctx);
  const int nt = ctx->p.ntrees;
  launch_k(ctx->lc.pdl, k_step_begin, 1, 1, 0, st, ctx->cnt, ctx->hist);
  launch_k(ctx->lc.pdl, k_time_coef, (nt + 127) / 128, 128, 0, st, ctx->ttime, ctx->trees, nt, ctx->p.rhs_kind == MR_RHS_SWIRL);
  count_launch(2);
  int mode = MR_ADAPT_REFINE_ALL;
  if (ctx->refine_mode == 1) {
    // learned proposal with the exact fallback, closed under gradedness: the
    // closure is monotone, so a fixed number of passes (one more than the
    // level span) reaches its fixpoint and later passes change nothing
    launch_features(pv, ctx->y, ctx->feat, ctx->mpre, 0, ctx->lc.num_sms, st);
    launch_infer(pv, ctx->p.Bs, ctx->feat, ctx->cnn_wb, ctx->prob, -1, ctx->lc.num_sms, st);
    launch_propose(pv, ctx->prob, ctx->mpre, ctx->cnn_tau, ctx->skip, ctx->gcounts, st);
    int jspan = 0;
    for (auto& t : ctx->td) jspan = std::max(jspan, t.Jmax - t.Jmin);
    for (int it = 0; it <= jspan; ++it) launch_close(pv, ctx->skip, ctx->gcounts + 4, st);
    launch_skip_key(pv, ctx->skip, ctx->skip_key, st);
    mode = 2;
  }
  by_dim(ctx, [&] { launch_refine<2>(pv, f, mode, ctx->mask, ctx->lc, st); },
         [&] { launch_refine<3>(pv, f, mode, ctx->mask, ctx->lc, st); });
  by_dim(ctx, [&] { launch_plan<2>(pv, ctx->lc, st); }, [&] { launch_plan<3>(pv, ctx->lc, st); });
  StageArgs sa;
  std::memset(&sa, 0, sizeof(sa));
  sa.copy_state = filter_on(ctx) ? 1 : 0;
  for (int s = 0; s < 4; ++s)
    by_dim(ctx, [&] { launch_stage<2>(pv, f, s, sa, ctx->lc, st); },
           [&] { launch_stage<3>(pv, f, s, sa, ctx->lc, st); });
  if (filter_on(ctx)) launch_filter(pv, f, false, ctx->lc, st);
}

void enqueue_round(mr_ctx ctx, cudaStream_t st, const RoundCtl& rc) {
  PoolView pv = view(ctx);
  pv.tt = ctx->ttime;
  const Fields f = fields(ctx);
  const bool fp64 = ctx->p.detail_fp64 != 0;
  by_dim(ctx, [&] { launch_coarsen_round<2>(pv, f, fp64, true, rc, ctx->lc, st); },
         [&] { launch_coarsen_round<3>(pv, f, fp64, true, rc, ctx->lc, st); });
}

void enqueue_epilogue(mr_ctx ctx, cudaStream_t st) {
  const int nt = ctx->p.ntrees;
  if (ctx->refine_mode == 1) {
    PoolView pv = view(ctx);
    launch_miss_check(pv, ctx->skip, ctx->skip_key, ctx->gcounts, st);
  }
  k_time_advance<<<(nt + 127) / 128, 128, 0, st>>>(ctx->ttime, nt);
  count_launch();
}

// One step with no host synchronisation, for capture: time coefficients from
// the device, refine all, four stages, coarsening rounds, time advance.  The
// rounds are a conditional while-node (a round runs again only after a round
// that merged a family, at most max_rounds times); without conditional nodes
// they are a fixed number of rounds that become empty once one merged nothing.
cudaError_t capture_step(mr_ctx ctx, cudaGraph_t* out, bool use_while) {
  cudaStream_t cs = ctx->cap_stream;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  enqueue_graph_prologue(ctx, cs);
  rounds_begin(ctx, cs);
  if (use_while) {
    cudaStreamCaptureStatus status;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t nd = 0;
    cudaGraphConditionalHandle h = 0;
    cudaGraphNode_t cn = nullptr;
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)] = {};
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
    e = cudaStreamGetCaptureInfo(cs, &status, nullptr, &g, &deps, &edata, &nd);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      e = cudaGraphAddNode(&cn, g, deps, edata, nd, &cp);
    }
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &cn, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(ctx->body_stream, cp.conditional.phGraph_out[0], nullptr,
                                                            nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const int64_t b0 = kernel_launches();
      // the round's last kernel sets the condition of the next iteration
      enqueue_round(ctx, ctx->body_stream, round_ctl(ctx, h, true));
      ctx->graph_body = kernel_launches() - b0;
      cudaGraph_t body = nullptr;
      e = cudaStreamEndCapture(ctx->body_stream, &body);
    }
    if (e != cudaSuccess) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(cs, &junk);
      if (junk) cudaGraphDestroy(junk);
      cudaGetLastError();
      return e;
    }
  } else {
    for (int r = 0; r < max_rounds_of(ctx); ++r) enqueue_round(ctx, cs, round_ctl(ctx));
  }
  enqueue_epilogue(ctx, cs);
  return cudaStreamEndCapture(cs, out);
}

// The captured step bakes in the refinement mode and the threshold tau; a
// change of either captures the step again at the next replay.
void drop_graph(mr_ctx ctx) {
  if (ctx->gexec) {
    cudaStreamSynchronize(ctx->st);
    cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
  }
}

mr_status build_graph(mr_ctx ctx) {
  drop_graph(ctx);
  read_counters(ctx);  // block count for the choice of the stage form
  if (ctx->collect) return fail(ctx, MR_EINVAL, "training samples are collected by host-driven steps (mr_step)");
  if (ctx->refine_mode == 1) {
    mr_status s = ensure_feat(ctx, ctx->S);
    if (s) return s;
  }
  if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  if (!ctx->body_stream) CK(cudaStreamCreateWithFlags(&ctx->body_stream, cudaStreamNonBlocking));
  CK(cudaStreamSynchronize(ctx->st));
  cudaGraph_t g = nullptr;
  ctx->capturing = true;
  const int64_t k0 = kernel_launches();
  cudaError_t e = capture_step(ctx, &g, ctx->graph_while);
  if (e != cudaSuccess && ctx->lc.pdl) {  // programmatic edges not capturable: plain launches
    cudaGetLastError();
    ctx->lc.pdl = 0;
    count_launch((int)-(kernel_launches() - k0));
    ctx->graph_body = 0;
    e = capture_step(ctx, &g, ctx->graph_while);
  }
  if (e != cudaSuccess && ctx->graph_while) {  // no conditional nodes: fixed rounds
    cudaGetLastError();
    ctx->graph_while = false;
    count_launch((int)-(kernel_launches() - k0));
    ctx->graph_body = 0;
    e = capture_step(ctx, &g, false);
  }
  // kernel nodes per replay (a while-body counts once; replays add them)
  ctx->graph_kernels = kernel_launches() - k0;
  count_launch((int)-ctx->graph_kernels);
  ctx->capturing = false;
  if (e != cudaSuccess) return fail(ctx, MR_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&ctx->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess && ctx->lc.pdl) {  // capture again with plain launches
    cudaGetLastError();
    ctx->gexec = nullptr;
    ctx->lc.pdl = 0;
    return build_graph(ctx);
  }
  if (e != cudaSuccess) return fail(ctx, MR_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return MR_OK;
}
}  // namespace

mr_status mr_step_graph(mr_ctx ctx, int64_t nsteps) {
  if (!ctx || nsteps < 0) return MR_EINVAL;
  if (!ctx->gexec) {
    mr_status s = build_graph(ctx);
    if (s) return s;
  }
  for (int64_t i = 0; i < nsteps; ++i) CK(cudaGraphLaunch(ctx->gexec, ctx->st));
  count_launch((int)(ctx->graph_kernels * nsteps));
  if (ctx->graph_while) ctx->graph_steps += nsteps;
  ctx->stats.steps += nsteps;
  ctx->stats.stage_launches += 4 * nsteps;
  return MR_OK;
}

mr_status mr_set_launch_overlap(mr_ctx ctx, int32_t on) {
  if (!ctx) return MR_EINVAL;
  drop_graph(ctx);
  ctx->lc.pdl = on ? 1 : 0;
  return MR_OK;
}

int32_t mr_get_launch_overlap(mr_ctx ctx) { return ctx ? ctx->lc.pdl : -1; }

int32_t mr_graph_mode(mr_ctx ctx) {
  if (!ctx || !ctx->gexec) return -1;
  return ctx->graph_while ? 1 : 0;
}

mr_status mr_get_step_history(mr_ctx ctx, int64_t cap, int32_t* out, int64_t* n, int32_t reset) {
  if (!ctx || !n) return MR_EINVAL;
  mr_status s = check_device(ctx);
  if (s) return s;
  const Counters h = read_counters(ctx);
  *n = h.hist_n;
  if (out && cap > 0) CK(cudaMemcpy(out, ctx->hist, std::min<int64_t>(cap, h.hist_n) * 4, cudaMemcpyDeviceToHost));
  if (reset) {
    int32_t z = 0;
    CK(cudaMemcpy(&ctx->cnt->hist_n, &z, 4, cudaMemcpyHostToDevice));
  }
  return MR_OK;
}

mr_status mr_autotune(mr_ctx ctx, int32_t steps, int32_t* best_out) {
  if (!ctx || steps < 1) return MR_EINVAL;
  // candidates: CTAs per SM x form of the 2D stage (one CTA per block, one warp
  // per block); for the warp form on FP32 fields also blocks per CTA and the
  // staging of the rows (bulk copies or loads)
  struct Cand { int mult, form, wb, stg; };
  std::vector<Cand> cands;
  const int mults[] = {1, 2, 3, 4, 6, 8, 0};
  for (int m : mults) cands.push_back({m, 0, 4, 1});
  const bool warp_ok = ctx->p.dim == 2 && ctx->p.Bs == 17 && !is_ns(ctx->p.rhs_kind);
  if (warp_ok) {
    for (int m : mults) cands.push_back({m, 1, 4, 1});
    if (ctx->p.precision == MR_PREC_FP32) {
      for (int wb : {2, 8})
        for (int stg : {0, 1}) cands.push_back({0, 1, wb, stg});
      cands.push_back({0, 1, 4, 0});
    }
  }
  float best = 1e30f;
  Cand bc = cands[0];
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  for (const Cand& c : cands) {
    ctx->lc.grid_mult = c.mult;
    ctx->lc.stage_form = c.form;
    ctx->lc.warp_blocks = c.wb;
    ctx->lc.staging = c.stg;
    mr_status s = build_graph(ctx);
    if (s) return s;
    CK(cudaGraphLaunch(ctx->gexec, ctx->st));  // warm
    CK(cudaEventRecord(a, ctx->st));
    for (int i = 0; i < steps; ++i) CK(cudaGraphLaunch(ctx->gexec, ctx->st));
    count_launch((int)(ctx->graph_kernels * (steps + 1)));
    if (ctx->graph_while) ctx->graph_steps += steps + 1;
    CK(cudaEventRecord(b, ctx->st));
    CK(cudaEventSynchronize(b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, a, b));
    ctx->stats.steps += steps + 1;
    if (ms < best) { best = ms; bc = c; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  ctx->lc.grid_mult = bc.mult;
  ctx->lc.stage_form = bc.form;
  ctx->lc.warp_blocks = bc.wb;
  ctx->lc.staging = bc.stg;
  mr_status s = build_graph(ctx);
  if (s) return s;
  if (best_out) *best_out = bc.mult + 100 * bc.form + 1000 * bc.wb + 10000 * bc.stg;
  return check_device(ctx);
}


mr_status mr_set_warp_form(mr_ctx ctx, int32_t blocks_per_cta, int32_t staging) {
  if (!ctx || (blocks_per_cta != 2 && blocks_per_cta != 4 && blocks_per_cta != 8) || (staging != 0 && staging != 1))
    return MR_EINVAL;
  if (ctx->lc.warp_blocks != blocks_per_cta || ctx->lc.staging != staging) drop_graph(ctx);
  ctx->lc.warp_blocks = blocks_per_cta;
  ctx->lc.staging = staging;
  return MR_OK;
}

mr_status mr_set_tuning(mr_ctx ctx, int32_t ctas_per_sm, int32_t stage_form) {
  if (!ctx || ctas_per_sm < 0 || ctas_per_sm > 32 || stage_form < -1 || stage_form > 1) return MR_EINVAL;
  if (stage_form == 1 && (ctx->p.dim != 2 || ctx->p.Bs != 17 || is_ns(ctx->p.rhs_kind)))
    return fail(ctx, MR_EINVAL, "the warp-per-block form is for 2D advection on 17^2 blocks");
  if (ctx->lc.grid_mult != ctas_per_sm || ctx->lc.stage_form != stage_form) drop_graph(ctx);
  ctx->lc.grid_mult = ctas_per_sm;
  ctx->lc.stage_form = stage_form;
  return MR_OK;
}

mr_status mr_set_refine_mode(mr_ctx ctx, int32_t mode) {
  if (!ctx || (mode != 0 && mode != 1)) return MR_EINVAL;
  if (mode == 1) {
    mr_status s = ensure_cnn(ctx);
    if (s) return s;
    if (!ctx->cnn_ready) return fail(ctx, MR_EINVAL, "no trained or loaded proposal network");
  }
  if (mode != ctx->refine_mode) drop_graph(ctx);
  ctx->refine_mode = mode;
  return MR_OK;
}

mr_status mr_proposal_collect(mr_ctx ctx, int32_t on, int64_t capacity) {
  if (!ctx) return MR_EINVAL;
  mr_status s = ensure_cnn(ctx);
  if (s) return s;
  if (on && capacity > ctx->ds_cap) {
    CK(cudaStreamSynchronize(ctx->st));
    TmpBuf<float> f, l, mp;
    TmpBuf<int32_t> k;
    CK(f.alloc(capacity * feat_len(ctx) * 4));
    CK(l.alloc(capacity * 4));
    CK(mp.alloc(capacity * 4));
    CK(k.alloc(capacity * 16));
    if (ctx->ds_n > 0) {
      CK(cudaMemcpy(f.p, ctx->ds_feat, ctx->ds_n * feat_len(ctx) * 4, cudaMemcpyDeviceToDevice));
      CK(cudaMemcpy(l.p, ctx->ds_label, ctx->ds_n * 4, cudaMemcpyDeviceToDevice));
      CK(cudaMemcpy(mp.p, ctx->ds_mpre, ctx->ds_n * 4, cudaMemcpyDeviceToDevice));
      CK(cudaMemcpy(k.p, ctx->ds_key, ctx->ds_n * 16, cudaMemcpyDeviceToDevice));
    }
    if (ctx->ds_feat) { cudaFree(ctx->ds_feat); cudaFree(ctx->ds_label); cudaFree(ctx->ds_mpre); cudaFree(ctx->ds_key); }
    ctx->ds_feat = f.release(); ctx->ds_label = l.release(); ctx->ds_mpre = mp.release(); ctx->ds_key = k.release();
    ctx->ds_cap = capacity;
  }
  ctx->collect = on != 0;
  return MR_OK;
}

mr_status mr_proposal_dataset(mr_ctx ctx, int64_t* n, int64_t* npos) {
  if (!ctx || !n) return MR_EINVAL;
  CK(cudaStreamSynchronize(ctx->st));
  std::vector<float> l(ctx->ds_n);
  if (ctx->ds_n) CK(cudaMemcpy(l.data(), ctx->ds_label, ctx->ds_n * 4, cudaMemcpyDeviceToHost));
  int64_t nv = 0, np = 0;
  for (float v : l) { if (v >= 0.f) ++nv; if (v > 0.5f) ++np; }
  *n = nv;
  if (npos) *npos = np;
  return MR_OK;
}

mr_status mr_proposal_set(mr_ctx ctx, const float* params, float tau) {
  if (!ctx) return MR_EINVAL;
  mr_status s = ensure_cnn(ctx);
  if (s) return s;
  if (params) {
    CK(cudaMemcpy(ctx->cnn_w, params, kCnnParams * 4, cudaMemcpyHostToDevice));
    launch_to_bf16(ctx->cnn_w, ctx->cnn_wb, ctx->st);
    CK(cudaStreamSynchronize(ctx->st));
    ctx->cnn_ready = true;
  }
  if (tau != ctx->cnn_tau) drop_graph(ctx);
  ctx->cnn_tau = tau;
  return MR_OK;
}

mr_status mr_proposal_get(mr_ctx ctx, float* params, float* tau) {
  if (!ctx || !ctx->cnn_w) return MR_EINVAL;
  CK(cudaStreamSynchronize(ctx->st));
  if (params) CK(cudaMemcpy(params, ctx->cnn_w, kCnnParams * 4, cudaMemcpyDeviceToHost));
  if (tau) *tau = ctx->cnn_tau;
  return MR_OK;
}

mr_status mr_proposal_train(mr_ctx ctx, const float* init, int32_t epochs, int32_t batch, float lr,
                            float w_pos, float recall, float holdout, float* tau_out, float* loss_out) {
  if (!ctx || epochs < 0 || batch < 1 || !(recall > 0.f && recall <= 1.f) || !(holdout >= 0.f && holdout < 1.f))
    return MR_EINVAL;
  mr_status s = ensure_cnn(ctx);
  if (s) return s;
  CK(cudaStreamSynchronize(ctx->st));
  // labelled samples (blocks below Jmax), in collection order; the last
  // `holdout` fraction chooses the threshold
  std::vector<float> lab(ctx->ds_n);
  if (ctx->ds_n) CK(cudaMemcpy(lab.data(), ctx->ds_label, ctx->ds_n * 4, cudaMemcpyDeviceToHost));
  // stratified split: every k-th positive and every k-th negative is held out
  std::vector<int32_t> train_ids, hold_ids;
  int64_t npos = 0, nneg = 0;
  const int64_t every = holdout > 0.f ? std::max<int64_t>(2, (int64_t)std::llround(1.0 / holdout)) : 0;
  for (int64_t i = 0; i < ctx->ds_n; ++i) {
    if (lab[i] < 0.f) continue;
    const bool pos = lab[i] > 0.5f;
    const int64_t r = pos ? npos++ : nneg++;
    if (every && r % every == every - 1) hold_ids.push_back((int32_t)i);
    else train_ids.push_back((int32_t)i);
  }
  if (npos == 0 || nneg == 0) return fail(ctx, MR_EINVAL, "need labelled samples of both classes");
  if (!(w_pos > 0.f)) w_pos = (float)nneg / (float)npos;  // balance the classes
  std::vector<int32_t> valid(train_ids);
  valid.insert(valid.end(), hold_ids.begin(), hold_ids.end());
  const int64_t nv = (int64_t)valid.size();
  const int64_t nho = (int64_t)hold_ids.size();
  const int64_t ntr = nv - nho;
  if (ntr < 1) return fail(ctx, MR_EINVAL, "no labelled samples collected");
  // training order: a fixed interleave of the training samples (stride coprime
  // with their count), so batches mix steps without a random draw
  std::vector<int32_t> order(ntr);
  int64_t stride = 7919;
  while (std::gcd(stride, ntr) != 1) ++stride;
  for (int64_t i = 0; i < ntr; ++i) order[i] = valid[(i * stride) % ntr];
  TmpBuf<int32_t> didx;
  TmpBuf<float> dloss, dprob;
  CK(didx.alloc(std::max<int64_t>(nv, 1) * 4));
  CK(dloss.alloc(4));
  CK(dprob.alloc(std::max<int64_t>(nv, 1) * 4));
  CK(cudaMemcpy(didx.p, order.data(), ntr * 4, cudaMemcpyHostToDevice));
  if (nho > 0) CK(cudaMemcpy(didx.p + ntr, valid.data() + ntr, nho * 4, cudaMemcpyHostToDevice));
  if (init) {
    CK(cudaMemcpy(ctx->cnn_w, init, kCnnParams * 4, cudaMemcpyHostToDevice));
    CK(cudaMemset(ctx->cnn_m, 0, kCnnParams * 4));
    CK(cudaMemset(ctx->cnn_v, 0, kCnnParams * 4));
    ctx->cnn_t = 0;
  }
  CK(cudaMemset(ctx->cnn_g, 0, kCnnParams * 4));
  float last = 0.f;
  for (int e = 0; e < epochs; ++e) {
    CK(cudaMemsetAsync(dloss.p, 0, 4, ctx->st));
    for (int64_t s0 = 0; s0 < ntr; s0 += batch) {
      const int nb = (int)std::min<int64_t>(batch, ntr - s0);
      launch_train(ctx->p.Bs, ctx->ds_feat, ctx->ds_label, didx.p, s0, nb, ctx->cnn_w, w_pos, ctx->cnn_g,
                   dloss.p, nullptr, ctx->lc.num_sms, ctx->st);
      launch_adam(ctx->cnn_w, ctx->cnn_m, ctx->cnn_v, ctx->cnn_g, lr, ++ctx->cnn_t, ctx->cnn_wb, ctx->st);
    }
    CK(cudaMemcpyAsync(&last, dloss.p, 4, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  }
  launch_to_bf16(ctx->cnn_w, ctx->cnn_wb, ctx->st);
  // threshold: largest tau keeping recall >= target on the held-out samples
  // (all samples when there is no hold-out), with the BF16 inference weights
  const int64_t ne = nho > 0 ? nho : ntr;
  const int32_t* eidx = nho > 0 ? didx.p + ntr : didx.p;
  TmpBuf<float> gfeat;
  CK(gfeat.alloc(ne * feat_len(ctx) * 4));
  std::vector<int32_t> hidx(ne);
  CK(cudaMemcpy(hidx.data(), eidx, ne * 4, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < ne; ++i)
    CK(cudaMemcpyAsync(gfeat.p + i * feat_len(ctx), ctx->ds_feat + (int64_t)hidx[i] * feat_len(ctx),
                       feat_len(ctx) * 4, cudaMemcpyDeviceToDevice, ctx->st));
  PoolView pv = view(ctx);
  launch_infer(pv, ctx->p.Bs, gfeat.p, ctx->cnn_wb, dprob.p, ne, ctx->lc.num_sms, ctx->st);
  std::vector<float> pr(ne);
  CK(cudaMemcpyAsync(pr.data(), dprob.p, ne * 4, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  std::vector<float> ppos;
  for (int64_t i = 0; i < ne; ++i)
    if (lab[hidx[i]] > 0.5f) ppos.push_back(std::isfinite(pr[i]) ? pr[i] : 0.f);
  float tau = 0.5f;
  if (!ppos.empty()) {
    std::sort(ppos.begin(), ppos.end());
    const int64_t miss = (int64_t)std::floor((1.0 - recall) * (double)ppos.size());
    tau = std::nextafter(ppos[miss], 0.f);
  }
  drop_graph(ctx);
  ctx->cnn_tau = tau;
  ctx->cnn_ready = true;
  if (tau_out) *tau_out = tau;
  if (loss_out) *loss_out = last;
  return MR_OK;
}

mr_status mr_proposal_stats(mr_ctx ctx, int64_t* out, int32_t reset) {
  if (!ctx || !out) return MR_EINVAL;
  if (ctx->gcounts) {  // fold in the counters of graph replays
    int32_t g[5];
    CK(cudaStreamSynchronize(ctx->st));
    CK(cudaMemcpy(g, ctx->gcounts, sizeof(g), cudaMemcpyDeviceToHost));
    CK(cudaMemset(ctx->gcounts, 0, sizeof(g)));
    for (int k = 0; k < 5; ++k) ctx->prop_stats[k] += g[k];
  }
  for (int k = 0; k < 5; ++k) out[k] = ctx->prop_stats[k];
  if (reset) for (int k = 0; k < 5; ++k) ctx->prop_stats[k] = 0;
  return MR_OK;
}

mr_status mr_cnn_eval(mr_ctx ctx, const float* params, const float* x, const float* y, int64_t n,
                      float w_pos, float* prob, float* grad, float* loss) {
  if (!ctx || !params || !x || !y || n < 1) return MR_EINVAL;
  mr_status s = ensure_cnn(ctx);
  if (s) return s;
  const int64_t fl = feat_len(ctx);
  TmpBuf<float> dx, dy, dw, dg, dl, dp;
  CK(dx.alloc(n * fl * 4));
  CK(dy.alloc(n * 4));
  CK(dw.alloc(kCnnParams * 4));
  CK(dg.alloc(kCnnParams * 4));
  CK(dl.alloc(4));
  CK(dp.alloc(n * 4));
  CK(cudaMemcpy(dx.p, x, n * fl * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dy.p, y, n * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dw.p, params, kCnnParams * 4, cudaMemcpyHostToDevice));
  CK(cudaMemset(dg.p, 0, kCnnParams * 4));
  CK(cudaMemset(dl.p, 0, 4));
  launch_train(ctx->p.Bs, dx.p, dy.p, nullptr, 0, (int)n, dw.p, w_pos, dg.p, dl.p, dp.p, ctx->lc.num_sms, ctx->st);
  CK(cudaStreamSynchronize(ctx->st));
  if (prob) CK(cudaMemcpy(prob, dp.p, n * 4, cudaMemcpyDeviceToHost));
  if (grad) CK(cudaMemcpy(grad, dg.p, kCnnParams * 4, cudaMemcpyDeviceToHost));
  if (loss) CK(cudaMemcpy(loss, dl.p, 4, cudaMemcpyDeviceToHost));
  return MR_OK;
}

mr_status mr_enable_timing(mr_ctx ctx, int32_t on) {
  if (!ctx) return MR_EINVAL;
  ctx->timing = on != 0;
  return MR_OK;
}

mr_status mr_get_stats(mr_ctx ctx, mr_stats* out) {
  if (!ctx || !out) return MR_EINVAL;
  mr_status s = check_device(ctx);
  if (s) return s;
  flush_timers(ctx);
  Counters h = read_counters(ctx);
  ctx->stats.stage_blocks = (int64_t)h.stage_blocks;
  ctx->stats.det_blocks = (int64_t)h.det_blocks;
  *out = ctx->stats;
  return MR_OK;
}

mr_status mr_reset_stats(mr_ctx ctx) {
  if (!ctx) return MR_EINVAL;
  cudaStreamSynchronize(ctx->st);
  flush_timers(ctx);
  ctx->stats = mr_stats{};
  unsigned long long z = 0;
  cudaMemcpy(&ctx->cnt->stage_blocks, &z, sizeof(z), cudaMemcpyHostToDevice);
  cudaMemcpy(&ctx->cnt->det_blocks, &z, sizeof(z), cudaMemcpyHostToDevice);
  return MR_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------
// Error norms without device allocation (mr_error_noalloc).
//
// mr_error above allocates its scratch (the exact-field factor tables and the
// four accumulators) with cudaMalloc on every call.  Some callers cannot do
// that: processes whose device memory is fully reserved by another allocator
// (a framework's caching allocator that owns the pool), or callers that must
// not pay the device-wide synchronisation that cudaFree implies.  This variant
// keeps its scratch in one file-scope device array instead.
//
// Scratch: 3 factor tables of N = (Bs - 1) 2^Jmax doubles (one per axis) plus
// 4 accumulators, N <= kNoAllocMaxN.  Every GPU that loads the library holds
// the array (3 * 16384 + 4 doubles = 393,248 bytes) until the process exits.
// All calls on a device share it and it keeps the last call's contents: the
// accumulators are cleared at the start of each call, and calls whose work
// overlaps on the GPU (different streams or threads without ordering) race on
// it.
constexpr int64_t kNoAllocMaxN = 16384;
static __device__ __align__(256) double g_noalloc_scratch[3 * kNoAllocMaxN + 4];

namespace {

constexpr int kMaxDevices = 64;
std::once_flag g_noalloc_once[kMaxDevices];
double* g_noalloc_ptr[kMaxDevices] = {nullptr};
cudaError_t g_noalloc_err[kMaxDevices] = {cudaSuccess};

// Device address of the scratch array on device `dev`, which must be the
// current device.  In host code the array's name is only a stand-in, so the
// address is looked up once per device (std::call_once: concurrent first calls
// from several host threads look it up once) and cached.
cudaError_t noalloc_scratch(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::call_once(g_noalloc_once[dev], [dev] {
    void* p = nullptr;
    g_noalloc_err[dev] = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (g_noalloc_err[dev] == cudaSuccess) g_noalloc_ptr[dev] = (double*)p;
  });
  if (g_noalloc_err[dev] != cudaSuccess) return g_noalloc_err[dev];
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

// Makes the context's device current for the lifetime of the guard and
// restores the caller's device afterwards.
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
    else if (err == cudaSuccess) prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Factor tables of the exact field (Gaussian advected by constant u over t):
// ex[a][U] = exp(-d^2 / (2 sigma^2)), d the nearest periodic image of
// x0_a + U h - u_a t - c_a; axes beyond the dimension hold 1.
__global__ void k_noalloc_tables(double* ex, int64_t N, int dim, double L, double x00, double x01,
                                 double x02, double s0, double s1, double s2, double c0, double c1,
                                 double c2, double sigma) {
  pdl_enter();
  const double x0[3] = {x00, x01, x02}, sh[3] = {s0, s1, s2}, c[3] = {c0, c1, c2};
  const double h = L / (double)N;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < 3 * N;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(q / N);
    const int64_t U = q % N;
    if (a >= dim) { ex[q] = 1.0; continue; }
    const double x = x0[a] + (double)U * h;
    double dd = (x - sh[a]) - c[a];
    while (dd >= 0.5 * L) dd -= L;
    while (dd < -0.5 * L) dd += L;
    ex[q] = exp(-(dd * dd) / (2.0 * sigma * sigma));
  }
}

}  // namespace

extern "C" mr_status mr_error_noalloc(mr_ctx ctx, int32_t tree, double t, double* out) {
  if (!ctx || !out || tree < 0 || tree >= ctx->p.ntrees) return MR_EINVAL;
  const mr_tree_desc& td = ctx->td[tree];
  if (td.ic_kind != MR_IC_GAUSS) return fail(ctx, MR_EINVAL, "error needs the Gaussian IC");
  const int64_t N = ctx->tdev[tree].N;
  if (N > kNoAllocMaxN)
    return fail(ctx, MR_EINVAL, "mr_error_noalloc: (Bs-1)*2^Jmax = " + std::to_string(N) +
                                    " exceeds its scratch limit of " + std::to_string(kNoAllocMaxN));
  // the scratch array of the context's device (not of whatever device the
  // caller has current)
  DeviceGuard guard(ctx->dev);
  CK(guard.err);
  double* scratch = nullptr;
  CK(noalloc_scratch(ctx->dev, &scratch));
  double* ex = scratch;
  double* acc = scratch + 3 * kNoAllocMaxN;
  double sh[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < ctx->p.dim; ++a) sh[a] = ctx->p.rhs_kind == MR_RHS_ADV ? td.rhs[a] * t : 0.0;
  CK(cudaMemsetAsync(acc, 0, 4 * sizeof(double), ctx->st));
  k_noalloc_tables<<<ctx->lc.num_sms * 2, 256, 0, ctx->st>>>(ex, N, ctx->p.dim, ctx->p.L, td.x0[0], td.x0[1],
                                                            td.x0[2], sh[0], sh[1], sh[2], td.ic[0], td.ic[1],
                                                            td.ic[2], td.ic[3]);
  CK(cudaGetLastError());
  count_launch();
  PoolView pv = view(ctx);
  by_dim(ctx, [&] { launch_error<2>(pv, fields(ctx), tree, ex, acc, ctx->lc, ctx->st); },
         [&] { launch_error<3>(pv, fields(ctx), tree, ex, acc, ctx->lc, ctx->st); });
  double o[4];
  CK(cudaMemcpyAsync(o, acc, sizeof(o), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  out[0] = std::sqrt(o[0]); out[1] = std::sqrt(o[1]); out[2] = o[2]; out[3] = o[3];
  return MR_OK;
}
