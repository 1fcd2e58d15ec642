// C ABI of the non-Hermitian FEAST hot path: context, contour integration,
// Rayleigh-Ritz and the outer loop of Fig. alg:three.  Host code here only
// sizes, sequences and checks device work; every numerical step runs in the
// kernels of band.cu, spmm.cu, dense.cu and rr.cu.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "feast_nh.h"
#include "kernels.h"
#include "rr.cuh"

static std::atomic<uint64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// CUDA-event pairs around launches of one kernel, harvested at sync points.
// Workspace comes from one stream-ordered memory pool per device, owned by
// the library, whose release threshold keeps freed memory reserved: a
// destroyed context's workspace serves the next context without cudaMalloc /
// cudaFree of gigabytes (the caching idea of PyTorch's allocator).
// feast_nh_release_memory() hands the reserved memory back to the driver.
// Without a pool (creation refused), plain cudaMalloc / cudaFree.
namespace pool {
constexpr int kMaxDev = 64;
std::mutex mu;
cudaMemPool_t p[kMaxDev] = {};
bool tried[kMaxDev] = {};

cudaMemPool_t get() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!tried[dev]) {
    tried[dev] = true;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&p[dev], &props) == cudaSuccess) {
      uint64_t keep = ~0ull;
      cudaMemPoolSetAttribute(p[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      cudaGetLastError();
      p[dev] = nullptr;
    }
  }
  return p[dev];
}

// bytes on stream s from the pool (in stream order) or from cudaMalloc
cudaError_t alloc(void **ptr, size_t bytes, cudaStream_t s, bool *pooled) {
  cudaMemPool_t mp = get();
  *pooled = mp != nullptr;
  return mp ? cudaMallocFromPoolAsync(ptr, bytes, mp, s) : cudaMalloc(ptr, bytes);
}
void release(void *ptr, bool pooled, cudaStream_t s) {
  if (pooled)
    cudaFreeAsync(ptr, s);
  else
    cudaFree(ptr);
}
}  // namespace pool

struct EvPool {
  static constexpr int kCap = 96;
  cudaEvent_t a[kCap] = {}, b[kCap] = {};
  int used = 0, made = 0;
  double ms = 0;
  int launches = 0;
};

struct feast_nh_ctx {
  int n = 0, m0 = 0, ne = 0;
  cudaStream_t s = nullptr;
  feast_nh_opts o{};
  feast_nh_contour con{};
  double alpha = 1.0;
  std::vector<cxd> hz, hw;
  cxd *dz = nullptr, *dw = nullptr, *dzc = nullptr, *dwc = nullptr;
  CsrView A{}, AH{}, B{}, BH{};
  bool hasB = false;
  std::vector<void *> allocs;
  std::vector<bool> pooled;  // allocs[i] came from the library's pool
  int kl = -1, ku = -1;     // band of (z B - A)
  int klp = 0, kup = 0;     // stored band widths (kl rounded up to even, kl+ku+1 even)
  void *bandT = nullptr;    // FP32: transposed factors for the conjugate-transpose solves
  void *kwork = nullptr;    // BiCGStab workspace
  std::vector<unsigned char> tma;  // tensor maps of band and bandT (empty: no TMA path)
  int nf = 0;              // shifted matrices factorised (ne, or ne/2 with conjugate node pairs)
  std::vector<int> fmap;   // node -> factor slot | conjugate << 16
  cxd *dzf = nullptr;      // shifts of the factorised matrices
  bool factored = false;
  void *band = nullptr;
  void *ysc = nullptr;
  void *dinv = nullptr;
  cxd *Yw = nullptr, *Yhw = nullptr, *Qw = nullptr, *Qhw = nullptr, *Uw = nullptr, *Uhw = nullptr, *T1 = nullptr,
      *T2 = nullptr, *BYw = nullptr, *BhYw = nullptr;
  cxd *Xn = nullptr, *Xhn = nullptr;
  void *Rn = nullptr, *Rhn = nullptr;
  double *part = nullptr;
  double *bynorm2 = nullptr;
  int *d_done = nullptr, *d_err = nullptr, *d_ext = nullptr;
  int *d_fxy = nullptr;  // column exponent fields of the tensor-core projections
  double *d_maxrel = nullptr;
  cxd *BQ = nullptr, *gam = nullptr, *V = nullptr, *Vinv = nullptr, *S = nullptr, *Sh = nullptr, *AU = nullptr,
      *BU = nullptr, *BUinv = nullptr, *Mred = nullptr, *lam = nullptr, *lamc = nullptr, *W = nullptr,
      *Winv = nullptr, *Wh = nullptr, *swork = nullptr, *gpart = nullptr, *rho = nullptr, *prev_rho = nullptr;
  int *prev_inside = nullptr, *ord = nullptr;
  double *colp = nullptr, *cn = nullptr, *res = nullptr;
  int gchunks = 1;
  int gmax = 1216;
  RRStatus *d_st = nullptr, *h_st = nullptr;
  double *h_small = nullptr;
  int have_prev = 0;
  double *pn = nullptr, *pmax = nullptr;
  int *pidx = nullptr;
  cxd *pval = nullptr, *pdot = nullptr, *sx = nullptr, *sxh = nullptr;
  std::string err;
  cudaEvent_t ev[6] = {};
  double t_factor = 0, inner_res = 0;
  int inner_steps = 0;
  bool krylov_ok = true;
  double last_inner_tol = 0;  // tolerance the last filter's inner solves aimed at
  int n_inner_fail = 0;       // filters of the current solve that missed it
  double *d_piv = nullptr;    // pivot statistics of the banded factors (2 doubles)
  double piv_min = 0, piv_max = 0;
  unsigned inject_bits = 0;   // host-requested device error bits (testing aid)
  bool rr_only = false;       // Rayleigh-Ritz workspace only (one problem of a batch)
  int max_nnz[2] = {0, 0};    // longest row of A and of A^H
  void *fgwork = nullptr;     // FGMRES workspace
  cxf *dfg = nullptr;         // FGMRES correction (node-major, complex float)
  cxd *adiag = nullptr, *bdiag = nullptr;  // diagonals of A and B (Jacobi)
  feast_nh_net *net = nullptr;              // learned preconditioner (not owned)
  int net_N = 0, net_nfeat = 0;
  float net_kappa = 1.f;
  float *net_feat = nullptr, *net_scratch = nullptr;
  int krylov_its = 0;         // FGMRES iterations in the current call
  std::string fg_err;
  bool own_stream = false;
  EvPool ev_solve, ev_resid;
};

namespace {

struct Fail {
  feast_nh_status st;
};

#define CKC(...)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (__VA_ARGS__);                                                        \
    if (e_ != cudaSuccess) {                                                               \
      ctx->err = std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_);                \
      throw Fail{e_ == cudaErrorMemoryAllocation ? FEAST_NH_ENOMEM : FEAST_NH_ECUDA};      \
    }                                                                                      \
  } while (0)

#define REQ(cond, msg)                   \
  do {                                   \
    if (!(cond)) {                       \
      ctx->err = msg;                    \
      throw Fail{FEAST_NH_EINVAL};       \
    }                                    \
  } while (0)

template <typename P>
P *dalloc(feast_nh_ctx *ctx, size_t bytes) {
  void *p = nullptr;
  if (bytes == 0) bytes = 16;
  bool pooled = false;
  CKC(pool::alloc(&p, bytes, ctx->s, &pooled));
  ctx->allocs.push_back(p);
  ctx->pooled.push_back(pooled);
  return reinterpret_cast<P *>(p);
}

void check_launch(feast_nh_ctx *ctx, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
    throw Fail{FEAST_NH_ECUDA};
  }
}

void compute_nodes(const feast_nh_contour &c, std::vector<cxd> &z, std::vector<cxd> &w) {
  z.resize(c.ne);
  w.resize(c.ne);
  if (c.kind == 2) {
    for (int j = 0; j < c.ne; ++j) {
      z[j] = mk(c.z[2 * j], c.z[2 * j + 1]);
      w[j] = mk(c.w[2 * j], c.w[2 * j + 1]);
    }
    return;
  }
  for (int j = 0; j < c.ne; ++j) trapezoid_node(c.kind, c.c_re, c.c_im, c.r, c.ratio, c.angle, c.ne, j, z[j], w[j]);
}

CsrView make_view(const feast_nh_csr &M) {
  CsrView v;
  v.n = M.n;
  v.nnz = M.nnz;
  v.rowptr = M.rowptr;
  v.colind = M.colind;
  v.val = reinterpret_cast<const double *>(M.val);
  v.cplx = M.dtype == FEAST_NH_C64;
  v.conj_vals = 0;
  return v;
}

CsrView transpose_view(feast_nh_ctx *ctx, const CsrView &M) {
  CsrView t = M;
  int32_t *rp = dalloc<int32_t>(ctx, (size_t)(M.n + 1) * sizeof(int32_t));
  int32_t *ci = dalloc<int32_t>(ctx, (size_t)M.nnz * sizeof(int32_t));
  double *va = dalloc<double>(ctx, (size_t)M.nnz * (M.cplx ? 2 : 1) * sizeof(double));
  int32_t *work = dalloc<int32_t>(ctx, (size_t)M.n * sizeof(int32_t));
  CKC(csr_transpose(M, rp, ci, va, work, ctx->s));
  t.rowptr = rp;
  t.colind = ci;
  t.val = va;
  t.conj_vals = M.cplx ? 1 : 0;
  return t;
}

// Event pair around the next launch (only with opts.timing and a free slot).
int ev_begin(feast_nh_ctx *ctx, EvPool &p) {
  if (!ctx->o.timing || p.used >= EvPool::kCap) return -1;
  const int k = p.used++;
  if (k >= p.made) {
    CKC(cudaEventCreate(&p.a[k]));
    CKC(cudaEventCreate(&p.b[k]));
    p.made = k + 1;
  }
  CKC(cudaEventRecord(p.a[k], ctx->s));
  return k;
}
void ev_end(feast_nh_ctx *ctx, EvPool &p, int k) {
  if (k >= 0) CKC(cudaEventRecord(p.b[k], ctx->s));
}
// After a stream synchronisation: add up the recorded intervals.
void ev_harvest(EvPool &p) {
  for (int k = 0; k < p.used; ++k) {
    float t = 0;
    if (cudaEventElapsedTime(&t, p.a[k], p.b[k]) == cudaSuccess) {
      p.ms += t;
      p.launches += 1;
    }
  }
  p.used = 0;
}

const void *tma_ptr(const feast_nh_ctx *ctx) { return ctx->tma.empty() ? nullptr : ctx->tma.data(); }

bool cs_mode(const feast_nh_ctx *ctx) { return ctx->o.problem == FEAST_NH_PROBLEM_COMPLEX_SYMMETRIC; }
bool fp32(const feast_nh_ctx *ctx) { return ctx->o.precision == FEAST_NH_PREC_FP32_IR; }
bool krylov(const feast_nh_ctx *ctx) { return ctx->o.inner_kind == FEAST_NH_INNER_BICGSTAB; }
bool fgmres(const feast_nh_ctx *ctx) { return ctx->o.inner_kind == FEAST_NH_INNER_FGMRES; }
bool banded(const feast_nh_ctx *ctx) { return ctx->o.inner_kind == FEAST_NH_INNER_BANDED; }

// FGMRES operator and right preconditioner of one side (0: eq. qr, 1: eq. ql)
struct FgSide {
  feast_nh_ctx *ctx;
  int side, m;
};
void fg_apply(void *p, const cxf *x, cxf *y, cudaStream_t s) {
  const FgSide *f = static_cast<const FgSide *>(p);
  feast_nh_ctx *ctx = f->ctx;
  if (f->side == 0)
    launch_multishift_spmm_f32(ctx->A, ctx->hasB ? &ctx->B : nullptr, ctx->ne, ctx->dz, 0, x, y, f->m, 0,
                               ctx->max_nnz[0], s);
  else
    launch_multishift_spmm_f32(ctx->AH, ctx->hasB ? &ctx->BH : nullptr, ctx->ne, ctx->dz, 1, x, y, f->m, 0,
                               ctx->max_nnz[1], s);
}
void fg_precond(void *p, const cxf *v, cxf *z, cudaStream_t s) {
  const FgSide *f = static_cast<const FgSide *>(p);
  feast_nh_ctx *ctx = f->ctx;
  const size_t count = (size_t)ctx->ne * ctx->n * f->m;
  if (ctx->o.precond == FEAST_NH_PRECOND_JACOBI) {
    launch_fg_jacobi(v, ctx->dz, f->side, ctx->adiag, ctx->hasB ? ctx->bdiag : nullptr, z, ctx->ne, ctx->n, f->m, s);
  } else if (ctx->o.precond == FEAST_NH_PRECOND_LEARNED && ctx->net) {
    const size_t S = (size_t)ctx->ne * f->m;
    const size_t np = net_precondition_scratch_floats(ctx->n, ctx->ne, f->m) - S;
    if (net_precondition(ctx->net, v, z, ctx->ne, ctx->n, f->m, ctx->dz, f->side, ctx->net_kappa, ctx->net_feat,
                         ctx->net_nfeat, ctx->net_scratch, ctx->net_scratch + np, s) != 0)
      ctx->fg_err = "the learned preconditioner failed";
  } else {
    cudaMemcpyAsync(z, v, count * sizeof(cxf), cudaMemcpyDeviceToDevice, s);
  }
}

void factorize(feast_nh_ctx *ctx) {
  if (!banded(ctx)) {
    ctx->factored = true;
    ctx->t_factor = 0;
    return;
  }
  const CsrView *Bp = ctx->hasB ? &ctx->B : nullptr;
  CKC(cudaEventRecord(ctx->ev[4], ctx->s));
  CKC(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->s));
  if (fp32(ctx)) {
    launch_band_build<float>(ctx->A, Bp, ctx->klp, ctx->kup, ctx->nf, ctx->dzf, (cxf *)ctx->band, ctx->s);
    CKC(band_factor<float>(ctx->n, ctx->klp, ctx->kup, ctx->nf, (cxf *)ctx->band, ctx->d_err, ctx->s));
    launch_band_diag_inv<float>(ctx->n, ctx->klp, ctx->kup, ctx->nf, (const cxf *)ctx->band, (cxf *)ctx->dinv, ctx->s);
    if (!ctx->tma.empty())
      launch_band_transpose(ctx->n, ctx->klp, ctx->kup, ctx->nf, (const cxf *)ctx->band, (cxf *)ctx->bandT, ctx->s);
  } else {
    launch_band_build<double>(ctx->A, Bp, ctx->klp, ctx->kup, ctx->nf, ctx->dzf, (cxd *)ctx->band, ctx->s);
    CKC(band_factor<double>(ctx->n, ctx->klp, ctx->kup, ctx->nf, (cxd *)ctx->band, ctx->d_err, ctx->s));
  }
  CKC(cudaEventRecord(ctx->ev[5], ctx->s));
  if (fp32(ctx))
    launch_band_pivot_stats<float>(ctx->n, ctx->klp, ctx->kup, ctx->nf, (const cxf *)ctx->band, ctx->d_piv, ctx->s);
  else
    launch_band_pivot_stats<double>(ctx->n, ctx->klp, ctx->kup, ctx->nf, (const cxd *)ctx->band, ctx->d_piv, ctx->s);
  int herr = 0;
  double piv[2] = {0, 0};
  CKC(cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
  CKC(cudaMemcpyAsync(piv, ctx->d_piv, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  CKC(cudaStreamSynchronize(ctx->s));
  ctx->piv_min = piv[0];
  ctx->piv_max = piv[1];
  float ms = 0;
  cudaEventElapsedTime(&ms, ctx->ev[4], ctx->ev[5]);
  ctx->t_factor = ms;
  if (herr & DEVERR_ZERO_PIVOT) {
    ctx->err = "zero pivot in the banded factorisation of (z_j B - A): a node lies on an eigenvalue";
    throw Fail{FEAST_NH_ESINGULAR};
  }
  ctx->factored = true;
}

// Step 1 of Fig. alg:three on n x m blocks.  inner_tol: refinement target
// (negative: opts.inner_tol).
void do_filter(feast_nh_ctx *ctx, const cxd *Y, const cxd *Yh, cxd *Q, cxd *Qh, int m, double inner_tol = -1.0,
               bool first_pass = false) {
  if (inner_tol < 0) inner_tol = ctx->o.inner_tol;
  if (!ctx->factored) factorize(ctx);
  const bool cs = cs_mode(ctx);
  const int n = ctx->n, ne = ctx->ne;
  const CsrView *Bp = ctx->hasB ? &ctx->B : nullptr;
  const CsrView *BHp = ctx->hasB ? &ctx->BH : nullptr;
  const cxd *BY = Y, *BhYh = cs ? nullptr : Yh;
  if (ctx->hasB) {
    launch_spmm(ctx->B, nullptr, nullptr, Y, ctx->BYw, m, nullptr, nullptr, ctx->s);
    BY = ctx->BYw;
    if (!cs) {
      launch_spmm(ctx->BH, nullptr, nullptr, Yh, ctx->BhYw, m, nullptr, nullptr, ctx->s);
      BhYh = ctx->BhYw;
    }
  }
  const size_t xns = (size_t)n * m;
  if (krylov(ctx)) {
    // batched BiCGStab on every (node, column) system, then Q = sum_j w_j X_j
    double rel_r = 0, rel_l = 0;
    int kb = ev_begin(ctx, ctx->ev_solve);
    const int it_r = krylov_bicgstab(ctx->A, Bp, ne, ctx->dz, ctx->dw, BY, m, ctx->m0, inner_tol, ctx->o.inner_max,
                                     ctx->kwork, ctx->Xn, &rel_r, ctx->s);
    ev_end(ctx, ctx->ev_solve, kb);
    launch_multishift_residual<double>(ctx->A, Bp, ne, ctx->dz, ctx->dw, ctx->Xn, BY, nullptr, Q, nullptr, m, nullptr,
                                       ctx->s);
    int it_l = 0;
    if (!cs) {
      kb = ev_begin(ctx, ctx->ev_solve);
      it_l = krylov_bicgstab(ctx->AH, BHp, ne, ctx->dzc, ctx->dwc, BhYh, m, ctx->m0, inner_tol, ctx->o.inner_max,
                             ctx->kwork, ctx->Xhn, &rel_l, ctx->s);
      ev_end(ctx, ctx->ev_solve, kb);
      launch_multishift_residual<double>(ctx->AH, BHp, ne, ctx->dzc, ctx->dwc, ctx->Xhn, BhYh, nullptr, Qh, nullptr, m,
                                         nullptr, ctx->s);
    }
    ctx->inner_steps = it_r > it_l ? it_r : it_l;
    ctx->inner_res = rel_r > rel_l ? rel_r : rel_l;
    ctx->krylov_ok = !(ctx->inner_res > inner_tol);
  } else if (fgmres(ctx)) {
    // FP32 FGMRES (right preconditioner opts.precond) inside FP64 iterative
    // refinement: each step asks FGMRES for a relative reduction of
    // max(1e-5, the step's target); the FP64 residual decides convergence
    const double tfg = std::fmax(1e-5, inner_tol);
    const int restart = ctx->o.krylov_restart;
    auto fg = [&](int side, const cxf *b, cxd *X, int mode) {
      FgSide fs{ctx, side, m};
      FgmresOp op{&fs, fg_apply, fg_precond};
      double rel = 0;
      const int k = ev_begin(ctx, ctx->ev_solve);
      ctx->krylov_its += fgmres_solve(op, b, ctx->dfg, n, m, ne, ctx->m0, restart, ctx->o.krylov_max, tfg,
                                      ctx->fgwork, &rel, ctx->s);
      ev_end(ctx, ctx->ev_solve, k);
      if (!ctx->fg_err.empty()) {
        ctx->err = ctx->fg_err;
        ctx->fg_err.clear();
        throw Fail{FEAST_NH_EINVAL};
      }
      launch_cxf_accumulate(X, ctx->dfg, (size_t)ne * n * m, mode, ctx->s);
    };
    CKC(cudaMemsetAsync(ctx->d_done, 0, sizeof(int), ctx->s));
    launch_broadcast_cxf(BY, (cxf *)ctx->Rn, (size_t)n * m, ne, ctx->s);
    fg(0, (const cxf *)ctx->Rn, ctx->Xn, 0);
    if (!cs) {
      launch_broadcast_cxf(BhYh, (cxf *)ctx->Rhn, (size_t)n * m, ne, ctx->s);
      fg(1, (const cxf *)ctx->Rhn, ctx->Xhn, 0);
    }
    int g = launch_colnorm2(BY, m, m, n, ctx->colp, ctx->s);
    launch_reduce_parts(ctx->colp, g, m, ctx->bynorm2, ctx->s);
    if (!cs) {
      g = launch_colnorm2(BhYh, m, m, n, ctx->colp, ctx->s);
      launch_reduce_parts(ctx->colp, g, m, ctx->bynorm2 + m, ctx->s);
    }
    const int steps = ctx->o.inner_max < 1 ? 1 : ctx->o.inner_max;
    for (int it = 0; it < steps; ++it) {
      int kr = ev_begin(ctx, ctx->ev_resid);
      const int gm = launch_multishift_residual<float>(ctx->A, Bp, ne, ctx->dz, ctx->dw, ctx->Xn, BY, (cxf *)ctx->Rn,
                                                       nullptr, ctx->part, m, nullptr, ctx->s);
      ev_end(ctx, ctx->ev_resid, kr);
      if (!cs) {
        kr = ev_begin(ctx, ctx->ev_resid);
        launch_multishift_residual<float>(ctx->AH, BHp, ne, ctx->dzc, ctx->dwc, ctx->Xhn, BhYh, (cxf *)ctx->Rhn,
                                          nullptr, ctx->part + (size_t)gm * ne * m, m, nullptr, ctx->s);
        ev_end(ctx, ctx->ev_resid, kr);
      }
      launch_residual_check(ctx->part, gm, ne, m, ctx->bynorm2, cs ? 1 : 2, inner_tol, ctx->d_maxrel, ctx->d_done,
                            ctx->s);
      CKC(cudaMemcpyAsync(ctx->h_small + 2, ctx->d_done, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
      CKC(cudaStreamSynchronize(ctx->s));
      int done = 0;
      std::memcpy(&done, ctx->h_small + 2, sizeof(int));
      ctx->inner_steps = it + 1;
      if (done) break;
      if (it + 1 < steps) {
        fg(0, (const cxf *)ctx->Rn, ctx->Xn, 1);
        if (!cs) fg(1, (const cxf *)ctx->Rhn, ctx->Xhn, 1);
      }
    }
    launch_node_sum(ne, ctx->dw, ctx->Xn, xns, n, m, Q, ctx->s);
    if (!cs) launch_node_sum(ne, ctx->dwc, ctx->Xhn, xns, n, m, Qh, ctx->s);
  } else {
    // banded direct solves with iterative refinement: FP32 factors (chosen
    // form) or FP64 factors (plain form; the unpivoted factors of a general
    // pencil can lose accuracy, which the refinement restores or reports)
    const bool f32 = fp32(ctx);
    CKC(cudaMemsetAsync(ctx->d_done, 0, sizeof(int), ctx->s));
    auto solve = [&](const void *rR, const void *rL, size_t rns, int mode) {
      const int k = ev_begin(ctx, ctx->ev_solve);
      if (f32)
        CKC(band_solve_sides<float, float>(n, ctx->klp, ctx->kup, ne, ctx->fmap.data(), (const cxf *)ctx->band,
                                           (const cxf *)ctx->dinv, (const cxf *)rR, (const cxf *)rL, rns, m,
                                           ctx->Xn, cs ? nullptr : ctx->Xhn, xns, mode, (cxf *)ctx->ysc, nullptr,
                                           ctx->s, tma_ptr(ctx), ctx->d_err));
      else
        CKC(band_solve_sides<double, double>(n, ctx->klp, ctx->kup, ne, ctx->fmap.data(), (const cxd *)ctx->band,
                                             nullptr, (const cxd *)rR, (const cxd *)rL, rns, m, ctx->Xn,
                                             cs ? nullptr : ctx->Xhn, xns, mode, (cxd *)ctx->ysc, nullptr, ctx->s));
      ev_end(ctx, ctx->ev_solve, k);
    };
    if (f32) {
      // the first solve takes the right-hand sides in single precision (the
      // factors' precision; the refinement restores the rest): they are
      // staged in the first n x m entries of the residual buffers, which the
      // first residual overwrites
      launch_to_cxf(BY, (cxf *)ctx->Rn, (size_t)n * m, ctx->s);
      if (!cs) launch_to_cxf(BhYh, (cxf *)ctx->Rhn, (size_t)n * m, ctx->s);
      solve(ctx->Rn, cs ? nullptr : ctx->Rhn, 0, 0);
    } else {
      solve(BY, cs ? nullptr : BhYh, 0, 0);
    }
    int g = launch_colnorm2(BY, m, m, n, ctx->colp, ctx->s);
    launch_reduce_parts(ctx->colp, g, m, ctx->bynorm2, ctx->s);
    if (!cs) {
      g = launch_colnorm2(BhYh, m, m, n, ctx->colp, ctx->s);
      launch_reduce_parts(ctx->colp, g, m, ctx->bynorm2 + m, ctx->s);
    }
    // The loose first pass of a solve (inner tolerance >= 1e-2, FP32 factors)
    // keeps its single solve unchecked: it only supplies the start subspace of
    // the second iteration, whose refinement verifies the factors; its largest
    // residual is recorded as NaN ("not measured")
    const bool unchecked = first_pass && f32;
    const int steps = unchecked ? 0 : (ctx->o.inner_max < 1 ? 1 : ctx->o.inner_max);
    if (unchecked) {
      CKC(cudaMemsetAsync(ctx->d_maxrel, 0xFF, sizeof(double), ctx->s));
      ctx->inner_steps = 1;
    }
    for (int it = 0; it < steps; ++it) {
      // residuals only: the node sum Q is formed once, from the final X
      int kr = ev_begin(ctx, ctx->ev_resid);
      const int gm = f32 ? launch_multishift_residual<float>(ctx->A, Bp, ne, ctx->dz, ctx->dw, ctx->Xn, BY,
                                                             (cxf *)ctx->Rn, nullptr, ctx->part, m, nullptr, ctx->s)
                         : launch_multishift_residual<double>(ctx->A, Bp, ne, ctx->dz, ctx->dw, ctx->Xn, BY,
                                                              (cxd *)ctx->Rn, nullptr, ctx->part, m, nullptr, ctx->s);
      ev_end(ctx, ctx->ev_resid, kr);
      if (!cs) {
        kr = ev_begin(ctx, ctx->ev_resid);
        double *pl = ctx->part + (size_t)gm * ne * m;
        if (f32)
          launch_multishift_residual<float>(ctx->AH, BHp, ne, ctx->dzc, ctx->dwc, ctx->Xhn, BhYh, (cxf *)ctx->Rhn,
                                            nullptr, pl, m, nullptr, ctx->s);
        else
          launch_multishift_residual<double>(ctx->AH, BHp, ne, ctx->dzc, ctx->dwc, ctx->Xhn, BhYh, (cxd *)ctx->Rhn,
                                             nullptr, pl, m, nullptr, ctx->s);
        ev_end(ctx, ctx->ev_resid, kr);
      }
      launch_residual_check(ctx->part, gm, ne, m, ctx->bynorm2, cs ? 1 : 2, inner_tol, ctx->d_maxrel, ctx->d_done,
                            ctx->s);
      // one 4-byte read per refinement step decides whether to go on
      CKC(cudaMemcpyAsync(ctx->h_small + 2, ctx->d_done, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
      CKC(cudaStreamSynchronize(ctx->s));
      int done = 0;
      std::memcpy(&done, ctx->h_small + 2, sizeof(int));
      ctx->inner_steps = it + 1;
      if (done) break;
      if (it + 1 < steps) solve(ctx->Rn, cs ? nullptr : ctx->Rhn, xns, 1);
    }
    launch_node_sum(ne, ctx->dw, ctx->Xn, xns, n, m, Q, ctx->s);
    if (!cs) launch_node_sum(ne, ctx->dwc, ctx->Xhn, xns, n, m, Qh, ctx->s);
  }
  if (cs) launch_copy_conj(Q, Qh, (size_t)n * m, ctx->s);
  ctx->last_inner_tol = inner_tol;
  if (ctx->inject_bits) {
    launch_or_bits(ctx->d_err, (int)ctx->inject_bits, ctx->s);
    ctx->inject_bits = 0;
  }
  check_launch(ctx, "contour integration");
}

// Status of the device error word (host copy), FEAST_NH_OK if clear.
feast_nh_status status_from_err(feast_nh_ctx *ctx, int herr) {
  if (herr & DEVERR_TIMEOUT) {
    ctx->err = "a bounded wait for a tile load in the triangular solves gave up";
    return FEAST_NH_ETIMEOUT;
  }
  if (herr & DEVERR_ZERO_PIVOT) {
    ctx->err = "zero pivot in the banded factorisation of (z_j B - A): a node lies on an eigenvalue";
    return FEAST_NH_ESINGULAR;
  }
  if (herr & DEVERR_QR_NOCONV) {
    ctx->err = "small dense eigenproblem (B_Q or reduced): QR iteration did not converge";
    return FEAST_NH_ECUDA;
  }
  return FEAST_NH_OK;
}

// Whether the last filter's shifted solves stopped above their tolerance
// (largest relative residual in h_small[0] after read_status / read_inner).
bool inner_missed(const feast_nh_ctx *ctx) {
  if (krylov(ctx)) return !ctx->krylov_ok;
  const double r = ctx->h_small[0];
  if (std::isnan(r)) return false;  // the unchecked first pass
  return !(r <= ctx->last_inner_tol);
}

// Step 5.d: the converged pairs first, normalised (||x|| = 1, largest entry
// real > 0, x^^H B x = 1), from the Ritz blocks Y, Yh (n x mt, ld mt).
void finalize_output(feast_nh_ctx *ctx, const cxd *Y, const cxd *Yh, int mt, int mout, cxd *X, cxd *Xh, int ldo,
                     double *lambda, double *res) {
  cudaStream_t s = ctx->s;
  const int n = ctx->n;
  const cxd *BYf = Y;
  if (ctx->hasB) {
    launch_spmm(ctx->B, nullptr, nullptr, Y, ctx->T1, mt, nullptr, nullptr, s);
    BYf = ctx->T1;
  }
  const int gp = launch_colstats(Y, Yh, BYf, mt, n, ctx->pn, ctx->pmax, ctx->pidx, ctx->pval, ctx->pdot, s);
  launch_finalize(mt, gp, ctx->pn, ctx->pmax, ctx->pidx, ctx->pval, ctx->pdot, ctx->sx, ctx->sxh, Y, Yh, n,
                  ctx->ord, mout, X, Xh, ldo, ctx->lam, ctx->res, lambda, res, s);
  check_launch(ctx, "output");
}

RRParams rr_params(const feast_nh_ctx *ctx) {
  RRParams p{};
  p.kind = ctx->con.kind;
  p.ne = ctx->ne;
  p.c_re = ctx->con.c_re;
  p.c_im = ctx->con.c_im;
  p.r = ctx->con.r;
  p.ratio = ctx->con.ratio;
  p.angle = ctx->con.angle;
  p.alpha = ctx->alpha;
  p.eps = ctx->o.eps;
  for (int j = 0; j < ctx->ne && j < kMaxNe; ++j) p.cz[j] = ctx->hz[j];
  return p;
}

void read_status(feast_nh_ctx *ctx) {
  CKC(cudaMemcpyAsync(ctx->h_st, ctx->d_st, sizeof(RRStatus), cudaMemcpyDeviceToHost, ctx->s));
  CKC(cudaMemcpyAsync(ctx->h_small, ctx->d_maxrel, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  CKC(cudaMemcpyAsync(ctx->h_small + 1, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
  CKC(cudaStreamSynchronize(ctx->s));
  ev_harvest(ctx->ev_solve);
  ev_harvest(ctx->ev_resid);
}

// G = X^H Y (mx x my) and Z = X S over the n rows, on the tensor cores in
// exact digit products (FP64-accurate) or in FP64 on the CUDA cores, as
// opts.projection says.
static void proj_gram(feast_nh_ctx *ctx, const cxd *X, int ldx, int mx, const cxd *Y, int ldy, int my, cxd *G) {
  if (ctx->o.projection == FEAST_NH_PROJ_TENSOR)
    gram_tc(X, ldx, mx, Y, ldy, my, ctx->n, G, reinterpret_cast<long long *>(ctx->gpart),
            gram_tc_chunks(ctx->n, mx, my), ctx->d_fxy, ctx->d_err, ctx->s);
  else
    gram(X, ldx, mx, Y, ldy, my, ctx->n, G, ctx->gpart, ctx->gchunks, ctx->s);
}
static void proj_block(feast_nh_ctx *ctx, const cxd *X, int ldx, int mx, const cxd *S, int lds, int mz, cxd *Z,
                       int ldz) {
  if (ctx->o.projection == FEAST_NH_PROJ_TENSOR)
    block_tc(X, ldx, mx, S, lds, mz, ctx->n, Z, ldz, ctx->d_err, ctx->s);
  else
    block_times_small(X, ldx, mx, S, lds, mz, ctx->n, Z, ldz, ctx->s);
}

// Steps 2-5 of Fig. alg:three.  Returns the new subspace size.
int do_rr(feast_nh_ctx *ctx, const cxd *Q, const cxd *Qh, int m, cxd *Y, cxd *Yh) {
  const int n = ctx->n;
  const bool cs = cs_mode(ctx);
  cudaStream_t s = ctx->s;
  const CsrView *Bp = ctx->hasB ? &ctx->B : nullptr;
  const CsrView *BHp = ctx->hasB ? &ctx->BH : nullptr;
  // 2.a  B_Q = Q^^H B Q
  const cxd *BQq = Q;
  if (ctx->hasB) {
    launch_spmm(ctx->B, nullptr, nullptr, Q, ctx->T1, m, nullptr, nullptr, s);
    BQq = ctx->T1;
  }
  proj_gram(ctx, Qh, m, m, BQq, m, m, ctx->BQ);
  // 3.a  B_Q = V Gamma V^^H ; 2.b spurious ; 3.b-3.c resize and sort
  small_eig(ctx->BQ, m, ctx->gam, ctx->V, ctx->swork, ctx->d_err, s);
  if (!cs) small_inv(ctx->V, m, ctx->Vinv, ctx->swork, ctx->d_err, s);
  launch_gamma_prep(m, ctx->BQ, ctx->gam, ctx->V, ctx->Vinv, ctx->prev_rho, ctx->prev_inside, ctx->have_prev,
                    ctx->o.mu, ctx->o.eta, cs ? 1 : 0, ctx->S, ctx->Sh, ctx->ord, ctx->d_st, s);
  check_launch(ctx, "B_Q eigendecomposition");
  read_status(ctx);
  const int mt = ctx->h_st->m_tilde;
  if (mt < 1) {
    ctx->err = "B_Q is zero: the filtered subspace vanished";
    throw Fail{FEAST_NH_ESINGULAR};
  }
  // 3.d  U = Q V Gamma^{-1/2}, Uh = Qh Vh Gamma^{-H/2}        (eq. uu)
  proj_block(ctx, Q, m, m, ctx->S, m, mt, ctx->Uw, mt);
  proj_block(ctx, Qh, m, m, ctx->Sh, m, mt, ctx->Uhw, mt);
  // 4.a  A_U = Uh^H A U, B_U = Uh^H B U
  launch_spmm(ctx->A, nullptr, nullptr, ctx->Uw, ctx->T1, mt, nullptr, nullptr, s);
  proj_gram(ctx, ctx->Uhw, mt, mt, ctx->T1, mt, mt, ctx->AU);
  const cxd *BUu = ctx->Uw;
  if (ctx->hasB) {
    launch_spmm(ctx->B, nullptr, nullptr, ctx->Uw, ctx->T2, mt, nullptr, nullptr, s);
    BUu = ctx->T2;
  }
  proj_gram(ctx, ctx->Uhw, mt, mt, BUu, mt, mt, ctx->BU);
  // 4.b  A_U W = B_U W Lambda via eig(B_U^{-1} A_U); Wh^H = W^{-1} B_U^{-1}
  small_inv(ctx->BU, mt, ctx->BUinv, ctx->swork, ctx->d_err, s);
  small_mm(ctx->BUinv, 0, ctx->AU, 0, ctx->Mred, mt, mt, mt, s);
  small_eig(ctx->Mred, mt, ctx->lam, ctx->W, ctx->swork, ctx->d_err, s);
  if (cs) {
    launch_cs_wnorm(mt, ctx->BU, ctx->W, ctx->Wh, s);
  } else {
    small_inv(ctx->W, mt, ctx->Winv, ctx->swork, ctx->d_err, s);
    small_mm(ctx->BUinv, 1, ctx->Winv, 1, ctx->Wh, mt, mt, mt, s);
  }
  // 4.c  rho_a(lambda)
  launch_rho(mt, ctx->ne, ctx->dz, ctx->dw, ctx->lam, ctx->rho, s);
  // 4.d  Y = U W, Yh = Uh Wh; column scale ||y_i|| = 1
  proj_block(ctx, ctx->Uw, mt, mt, ctx->W, mt, mt, Y, mt);
  proj_block(ctx, ctx->Uhw, mt, mt, ctx->Wh, mt, mt, Yh, mt);
  if (!cs) {
    int g = launch_colnorm2(Y, mt, mt, n, ctx->colp, s);
    launch_reduce_parts(ctx->colp, g, mt, ctx->cn, s);
    launch_scale_pairs(Y, Yh, ctx->cn, mt, n, s);
  }
  // 5.b  residuals of eq. (res), both sides
  launch_copy_conj(ctx->lam, ctx->lamc, mt, s);
  const int np = mt;
  int g1 = launch_spmm(ctx->A, Bp, ctx->lam, Y, ctx->T1, mt, ctx->colp, ctx->colp + (size_t)ctx->gmax * kMaxM0, s);
  launch_reduce_parts(ctx->colp, g1, np, ctx->cn, s);
  launch_reduce_parts(ctx->colp + (size_t)ctx->gmax * kMaxM0, g1, np, ctx->cn + kMaxM0, s);
  int g2 = launch_spmm(ctx->AH, BHp, ctx->lamc, Yh, ctx->T2, mt, ctx->colp, ctx->colp + (size_t)ctx->gmax * kMaxM0, s);
  launch_reduce_parts(ctx->colp, g2, np, ctx->cn + 2 * kMaxM0, s);
  launch_reduce_parts(ctx->colp + (size_t)ctx->gmax * kMaxM0, g2, np, ctx->cn + 3 * kMaxM0, s);
  // 5.a, 5.c  inside count, spurious-corrected count, convergence, ordering
  launch_converge(rr_params(ctx), mt, ctx->lam, ctx->rho, ctx->cn, ctx->res, ctx->ord, ctx->prev_rho,
                  ctx->prev_inside, ctx->d_st, s);
  check_launch(ctx, "Rayleigh-Ritz");
  ctx->have_prev = 1;
  return mt;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void feast_nh_default_opts(feast_nh_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->eps = 1e-10;
  o->eta = 1e-16;
  o->mu = 0.1;
  o->inner_tol = 1e-10;
  o->max_iter = 100;
  o->inner_max = 12;
  o->inner_kind = FEAST_NH_INNER_BANDED;
  o->precision = FEAST_NH_PREC_FP64;
  o->problem = FEAST_NH_PROBLEM_GENERAL;
  o->krylov_max = 1000;
  o->krylov_restart = 30;
  o->precond = FEAST_NH_PRECOND_JACOBI;
  o->projection = FEAST_NH_PROJ_TENSOR;
}

const char *feast_nh_strerror(feast_nh_status s) {
  switch (s) {
    case FEAST_NH_OK: return "success";
    case FEAST_NH_EINVAL: return "invalid argument";
    case FEAST_NH_ENOMEM: return "device allocation failed";
    case FEAST_NH_ECUDA: return "CUDA error";
    case FEAST_NH_ENOCONV: return "outer iteration cap reached before convergence";
    case FEAST_NH_EINNER: return "inner solve did not reach its tolerance";
    case FEAST_NH_ESINGULAR: return "singular shifted matrix or vanished subspace";
    case FEAST_NH_ETIMEOUT: return "bounded device wait gave up";
  }
  return "unknown status";
}

const char *feast_nh_last_error(const feast_nh_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

feast_nh_status feast_nh_nodes(const feast_nh_contour *c, double *z, double *w) {
  if (!c || !z || !w || c->ne < 1 || c->ne > kMaxNe || (c->kind == 2 && (!c->z || !c->w)) || c->kind < 0 ||
      c->kind > 2)
    return FEAST_NH_EINVAL;
  std::vector<cxd> hz, hw;
  compute_nodes(*c, hz, hw);
  for (int j = 0; j < c->ne; ++j) {
    z[2 * j] = hz[j].re;
    z[2 * j + 1] = hz[j].im;
    w[2 * j] = hw[j].re;
    w[2 * j + 1] = hw[j].im;
  }
  return FEAST_NH_OK;
}

feast_nh_status feast_nh_release_memory(void) {
  std::lock_guard<std::mutex> lk(pool::mu);
  for (int d = 0; d < pool::kMaxDev; ++d)
    if (pool::p[d] && cudaMemPoolTrimTo(pool::p[d], 0) != cudaSuccess) return FEAST_NH_ECUDA;
  return FEAST_NH_OK;
}

void feast_nh_destroy(feast_nh_ctx *ctx) {
  if (!ctx) return;
  if (ctx->s) cudaStreamSynchronize(ctx->s);
  for (size_t i = 0; i < ctx->allocs.size(); ++i) pool::release(ctx->allocs[i], ctx->pooled[i], ctx->s);
  if (ctx->s) cudaStreamSynchronize(ctx->s);
  if (ctx->h_st) cudaFreeHost(ctx->h_st);
  if (ctx->h_small) cudaFreeHost(ctx->h_small);
  for (auto &e : ctx->ev)
    if (e) cudaEventDestroy(e);
  for (EvPool *p : {&ctx->ev_solve, &ctx->ev_resid})
    for (int k = 0; k < p->made; ++k) {
      cudaEventDestroy(p->a[k]);
      cudaEventDestroy(p->b[k]);
    }
  if (ctx->own_stream && ctx->s) cudaStreamDestroy(ctx->s);
  delete ctx;
}

}  // extern "C"

namespace {

// Context set-up shared by feast_nh_init and the problems of a batch
// (rr_only: no inner-solver workspace; the batch solves the shifted systems).
// Throws Fail.
void init_ctx(feast_nh_ctx *ctx, const feast_nh_csr *A, const feast_nh_csr *B, const feast_nh_contour *contour,
              int32_t m0, const feast_nh_opts *opts, void *stream, bool rr_only) {
  {
    REQ(A && A->rowptr && A->colind && A->val && A->n > 0 && A->nnz > 0, "A must be a non-empty device CSR");
    REQ(A->dtype == FEAST_NH_R64 || A->dtype == FEAST_NH_C64, "A.dtype must be R64 or C64");
    REQ(!B || (B->rowptr && B->colind && B->val && B->n == A->n && B->nnz > 0), "B must match A's order");
    REQ(!B || B->dtype == FEAST_NH_R64 || B->dtype == FEAST_NH_C64, "B.dtype must be R64 or C64");
    REQ(contour && contour->ne >= 1 && contour->ne <= kMaxNe, "contour.ne must be in [1, 64]");
    REQ(contour->kind >= 0 && contour->kind <= 2, "contour.kind must be 0, 1 or 2");
    REQ(contour->kind == 2 || contour->r > 0, "contour radius must be positive");
    REQ(contour->kind != 1 || contour->ratio > 0, "ellipse ratio must be positive");
    REQ(contour->kind != 2 || (contour->z && contour->w), "custom contour needs z and w");
    REQ(m0 >= 1 && m0 <= kMaxM0 && m0 <= A->n, "m0 must be in [1, min(128, n)]");
    if (opts) ctx->o = *opts; else feast_nh_default_opts(&ctx->o);
    REQ(ctx->o.inner_kind == FEAST_NH_INNER_BANDED || ctx->o.inner_kind == FEAST_NH_INNER_BICGSTAB ||
            ctx->o.inner_kind == FEAST_NH_INNER_FGMRES,
        "inner_kind must be BANDED, BICGSTAB or FGMRES");
    REQ(ctx->o.inner_kind != FEAST_NH_INNER_FGMRES || ctx->o.precision == FEAST_NH_PREC_FP32_IR,
        "the FGMRES inner solver runs FP32 sweeps inside FP64 refinement (precision FP32_IR)");
    REQ(ctx->o.inner_kind != FEAST_NH_INNER_FGMRES ||
            (ctx->o.krylov_restart >= 1 && ctx->o.krylov_restart <= 64 && ctx->o.krylov_max >= 1),
        "FGMRES needs 1 <= krylov_restart <= 64 and krylov_max >= 1");
    REQ(ctx->o.precond >= FEAST_NH_PRECOND_NONE && ctx->o.precond <= FEAST_NH_PRECOND_LEARNED, "bad precond");
    REQ(ctx->o.inner_kind != FEAST_NH_INNER_BICGSTAB || ctx->o.precision == FEAST_NH_PREC_FP64,
        "the BiCGStab inner solver runs in FP64");
    REQ(ctx->o.inner_max >= 1, "inner_max must be >= 1");
    REQ(ctx->o.projection == FEAST_NH_PROJ_FP64 || ctx->o.projection == FEAST_NH_PROJ_TENSOR, "bad projection");
    REQ(ctx->o.precision == FEAST_NH_PREC_FP64 || ctx->o.precision == FEAST_NH_PREC_FP32_IR, "bad precision");
    REQ(ctx->o.problem == FEAST_NH_PROBLEM_GENERAL || ctx->o.problem == FEAST_NH_PROBLEM_COMPLEX_SYMMETRIC,
        "bad problem kind");
    REQ(ctx->o.max_iter >= 1 && ctx->o.eps > 0 && ctx->o.eta >= 0 && ctx->o.mu > 0, "bad tolerances");
    REQ((size_t)contour->ne * m0 <= 2048, "ne * m0 must not exceed 2048");
    ctx->s = reinterpret_cast<cudaStream_t>(stream);
    ctx->rr_only = rr_only;
    ctx->n = A->n;
    ctx->m0 = m0;
    ctx->ne = contour->ne;
    ctx->con = *contour;
    ctx->con.z = ctx->con.w = nullptr;
    compute_nodes(*contour, ctx->hz, ctx->hw);
    if (contour->kind == 2) {
      double cr = 0, ci = 0, rr = 0;
      for (auto &z : ctx->hz) { cr += z.re / ctx->ne; ci += z.im / ctx->ne; }
      for (auto &z : ctx->hz) rr = std::fmax(rr, std::hypot(z.re - cr, z.im - ci));
      ctx->alpha = std::hypot(cr, ci) + rr;
    } else {
      const double ratio = contour->kind == 1 ? contour->ratio : 1.0;
      ctx->alpha = std::hypot(contour->c_re, contour->c_im) + contour->r * std::fmax(1.0, ratio);
    }
    const int n = ctx->n, ne = ctx->ne;
    for (auto &e : ctx->ev) CKC(cudaEventCreate(&e));
    std::vector<cxd> zc(ne), wc(ne);
    for (int j = 0; j < ne; ++j) {
      zc[j] = conj(ctx->hz[j]);
      wc[j] = conj(ctx->hw[j]);
    }
    ctx->dz = dalloc<cxd>(ctx, ne * sizeof(cxd));
    ctx->dw = dalloc<cxd>(ctx, ne * sizeof(cxd));
    ctx->dzc = dalloc<cxd>(ctx, ne * sizeof(cxd));
    ctx->dwc = dalloc<cxd>(ctx, ne * sizeof(cxd));
    CKC(cudaMemcpyAsync(ctx->dz, ctx->hz.data(), ne * sizeof(cxd), cudaMemcpyHostToDevice, ctx->s));
    CKC(cudaMemcpyAsync(ctx->dw, ctx->hw.data(), ne * sizeof(cxd), cudaMemcpyHostToDevice, ctx->s));
    CKC(cudaMemcpyAsync(ctx->dzc, zc.data(), ne * sizeof(cxd), cudaMemcpyHostToDevice, ctx->s));
    CKC(cudaMemcpyAsync(ctx->dwc, wc.data(), ne * sizeof(cxd), cudaMemcpyHostToDevice, ctx->s));
    ctx->A = make_view(*A);
    if (B) {
      ctx->hasB = true;
      ctx->B = make_view(*B);
    }
    // band of (z B - A); also validates the CSR arrays (row pointers within
    // [0, nnz] and non-decreasing, column indices in [0, n)) before any
    // kernel scatters through them
    ctx->d_ext = dalloc<int>(ctx, 4 * sizeof(int));
    launch_band_extent(ctx->A, ctx->hasB ? &ctx->B : nullptr, ctx->d_ext, ctx->s);
    int ext[3] = {0, 0, 0};
    CKC(cudaMemcpyAsync(ext, ctx->d_ext, 3 * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    CKC(cudaStreamSynchronize(ctx->s));
    REQ(ext[2] == 0, "malformed CSR: a row pointer or a column index of A or B is out of range");
    ctx->AH = transpose_view(ctx, ctx->A);
    if (B) ctx->BH = transpose_view(ctx, ctx->B);
    {
      int *d_mx = dalloc<int>(ctx, 2 * sizeof(int));
      CKC(cudaMemsetAsync(d_mx, 0, 2 * sizeof(int), ctx->s));
      launch_max_row_nnz(ctx->A, d_mx, ctx->s);
      launch_max_row_nnz(ctx->AH, d_mx + 1, ctx->s);
      CKC(cudaMemcpyAsync(ctx->max_nnz, d_mx, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
      CKC(cudaStreamSynchronize(ctx->s));
    }
    ctx->kl = ext[0];
    ctx->ku = ext[1];
    // stored band: kl rounded up to even and kl+ku+1 even, so that band rows and
    // the TMA box origins are 16-byte aligned (extra diagonals hold zeros)
    ctx->klp = ctx->kl + (ctx->kl & 1);
    ctx->kup = ctx->ku + ((ctx->klp + ctx->ku + 1) & 1);
    // Real pencil and a node set closed under conjugation (Sec. 2.4, Table
    // tab:solve): (conj(z) B - A) = conj(z B - A), so only one matrix of each
    // conjugate pair is factorised and the other uses the conjugated factors.
    {
      const bool real_pencil = !ctx->A.cplx && (!ctx->hasB || !ctx->B.cplx);
      ctx->fmap.assign(ne, -1);
      std::vector<cxd> zf;
      for (int j = 0; j < ne; ++j) {
        if (ctx->fmap[j] >= 0) continue;
        int partner = -1;
        if (real_pencil) {
          const double tol = 1e-13 * (1.0 + std::hypot(ctx->hz[j].re, ctx->hz[j].im));
          for (int k = 0; k < ne; ++k)
            if (k != j && ctx->fmap[k] < 0 &&
                std::hypot(ctx->hz[k].re - ctx->hz[j].re, ctx->hz[k].im + ctx->hz[j].im) <= tol) {
              partner = k;
              break;
            }
        }
        const int slot = (int)zf.size();
        const int rep = (partner >= 0 && ctx->hz[j].im < 0) ? partner : j;
        zf.push_back(ctx->hz[rep]);
        ctx->fmap[rep] = slot;
        if (partner >= 0) ctx->fmap[rep == j ? partner : j] = slot | (1 << 16);
      }
      ctx->nf = (int)zf.size();
      ctx->dzf = dalloc<cxd>(ctx, ctx->nf * sizeof(cxd));
      CKC(cudaMemcpyAsync(ctx->dzf, zf.data(), ctx->nf * sizeof(cxd), cudaMemcpyHostToDevice, ctx->s));
    }
    const bool f32 = fp32(ctx);
    const bool fits = rr_only || !banded(ctx) || (f32 ? (band_fits<float>(ctx->klp, ctx->kup) &&
                             (band_tma_fits(ctx->klp, ctx->kup) || band_solve_fits<float>(ctx->klp, ctx->kup)))
                          : (band_fits<double>(ctx->klp, ctx->kup) && band_solve_fits<double>(ctx->klp, ctx->kup)));
    if (!fits) {
      char msg[160];
      std::snprintf(msg, sizeof msg, "band (kl=%d, ku=%d) too wide for the banded inner solver", ctx->kl, ctx->ku);
      REQ(false, msg);
    }
    const size_t es = f32 ? sizeof(cxf) : sizeof(cxd);
    const bool inner = !rr_only;
    const size_t band_elems = (!banded(ctx) || !inner) ? 0 : (size_t)ctx->nf * n * (ctx->klp + ctx->kup + 1);
    ctx->band = dalloc<void>(ctx, band_elems * es);
    if (krylov(ctx) && inner) ctx->kwork = dalloc<void>(ctx, krylov_work_bytes(n, m0, ne));
    if (inner && f32 && banded(ctx) && band_tma_fits(ctx->klp, ctx->kup)) {
      ctx->bandT = dalloc<void>(ctx, band_elems * es);
      ctx->tma.assign(band_tma_bytes(), 0);
      if (!band_tma_make(ctx->tma.data(), n, ctx->klp, ctx->kup, ctx->nf, (const cxf *)ctx->band,
                         (const cxf *)ctx->bandT))
        ctx->tma.clear();
    }
    const size_t yse = (!banded(ctx) || !inner) ? 0
                       : f32   ? band_solve_scratch_elems<float>(n, m0, ne)
                               : band_solve_scratch_elems<double>(n, m0, ne);
    ctx->ysc = dalloc<void>(ctx, yse * es);
    if (inner && f32 && banded(ctx)) ctx->dinv = dalloc<void>(ctx, band_diag_inv_elems(n, ctx->nf) * sizeof(cxf));
    if (inner && fgmres(ctx)) {
      ctx->fgwork = dalloc<void>(ctx, fgmres_work_bytes(n, m0, ne, ctx->o.krylov_restart));
      ctx->dfg = dalloc<cxf>(ctx, (size_t)ne * n * m0 * sizeof(cxf));
      ctx->adiag = dalloc<cxd>(ctx, (size_t)n * sizeof(cxd));
      launch_csr_diag(ctx->A, ctx->adiag, ctx->s);
      if (B) {
        ctx->bdiag = dalloc<cxd>(ctx, (size_t)n * sizeof(cxd));
        launch_csr_diag(ctx->B, ctx->bdiag, ctx->s);
      }
      ctx->net_feat = dalloc<float>(ctx, 32 * sizeof(float));
      ctx->net_scratch = dalloc<float>(ctx, net_precondition_scratch_floats(n, ne, m0) * sizeof(float));
    }
    const size_t blk = (size_t)n * m0 * sizeof(cxd);
    if (inner) {
      ctx->Yw = dalloc<cxd>(ctx, blk);
      ctx->Yhw = dalloc<cxd>(ctx, blk);
      ctx->Qw = dalloc<cxd>(ctx, blk);
      ctx->Qhw = dalloc<cxd>(ctx, blk);
    }
    ctx->Uw = dalloc<cxd>(ctx, blk);
    ctx->Uhw = dalloc<cxd>(ctx, blk);
    ctx->T1 = dalloc<cxd>(ctx, blk);
    ctx->T2 = dalloc<cxd>(ctx, blk);
    if (ctx->hasB) {
      ctx->BYw = dalloc<cxd>(ctx, blk);
      ctx->BhYw = dalloc<cxd>(ctx, blk);
    }
    if (inner) {
      ctx->Xn = dalloc<cxd>(ctx, blk * ne);
      ctx->Xhn = dalloc<cxd>(ctx, blk * ne);
    }
    if (inner && !krylov(ctx)) {
      // refinement residuals in the factors' precision
      ctx->Rn = dalloc<void>(ctx, (size_t)n * m0 * ne * es);
      ctx->Rhn = dalloc<void>(ctx, (size_t)n * m0 * ne * es);
    }
    ctx->gmax = spmm_max_grid();
    ctx->part = dalloc<double>(ctx, inner ? (size_t)2 * ctx->gmax * 2048 * sizeof(double) : 16);
    ctx->bynorm2 = dalloc<double>(ctx, 2 * kMaxM0 * sizeof(double));
    ctx->d_done = dalloc<int>(ctx, sizeof(int));
    ctx->d_err = dalloc<int>(ctx, sizeof(int));
    ctx->d_maxrel = dalloc<double>(ctx, sizeof(double));
    ctx->d_piv = dalloc<double>(ctx, 2 * sizeof(double));
    CKC(cudaMemsetAsync(ctx->d_maxrel, 0, sizeof(double), ctx->s));
    const size_t sm = (size_t)kMaxM0 * kMaxM0 * sizeof(cxd);
    ctx->BQ = dalloc<cxd>(ctx, sm);
    ctx->V = dalloc<cxd>(ctx, sm);
    ctx->Vinv = dalloc<cxd>(ctx, sm);
    ctx->S = dalloc<cxd>(ctx, sm);
    ctx->Sh = dalloc<cxd>(ctx, sm);
    ctx->AU = dalloc<cxd>(ctx, sm);
    ctx->BU = dalloc<cxd>(ctx, sm);
    ctx->BUinv = dalloc<cxd>(ctx, sm);
    ctx->Mred = dalloc<cxd>(ctx, sm);
    ctx->W = dalloc<cxd>(ctx, sm);
    ctx->Winv = dalloc<cxd>(ctx, sm);
    ctx->Wh = dalloc<cxd>(ctx, sm);
    ctx->swork = dalloc<cxd>(ctx, 3 * sm);
    ctx->gchunks = gram_chunks(n);
    ctx->gpart = dalloc<cxd>(ctx, std::max((size_t)ctx->gchunks * sm, gram_tc_part_max(n)));
    ctx->d_fxy = dalloc<int>(ctx, 2 * kMaxM0 * sizeof(int));
    ctx->gam = dalloc<cxd>(ctx, kMaxM0 * sizeof(cxd));
    ctx->lam = dalloc<cxd>(ctx, kMaxM0 * sizeof(cxd));
    ctx->lamc = dalloc<cxd>(ctx, kMaxM0 * sizeof(cxd));
    ctx->rho = dalloc<cxd>(ctx, kMaxM0 * sizeof(cxd));
    ctx->prev_rho = dalloc<cxd>(ctx, kMaxM0 * sizeof(cxd));
    ctx->prev_inside = dalloc<int>(ctx, kMaxM0 * sizeof(int));
    ctx->ord = dalloc<int>(ctx, kMaxM0 * sizeof(int));
    ctx->colp = dalloc<double>(ctx, (size_t)2 * ctx->gmax * kMaxM0 * sizeof(double));
    ctx->cn = dalloc<double>(ctx, 4 * kMaxM0 * sizeof(double));
    ctx->res = dalloc<double>(ctx, kMaxM0 * sizeof(double));
    ctx->d_st = dalloc<RRStatus>(ctx, sizeof(RRStatus));
    ctx->pn = dalloc<double>(ctx, (size_t)304 * kMaxM0 * sizeof(double));
    ctx->pmax = dalloc<double>(ctx, (size_t)304 * kMaxM0 * sizeof(double));
    ctx->pidx = dalloc<int>(ctx, (size_t)304 * kMaxM0 * sizeof(int));
    ctx->pval = dalloc<cxd>(ctx, (size_t)304 * kMaxM0 * sizeof(cxd));
    ctx->pdot = dalloc<cxd>(ctx, (size_t)304 * kMaxM0 * sizeof(cxd));
    ctx->sx = dalloc<cxd>(ctx, kMaxM0 * sizeof(cxd));
    ctx->sxh = dalloc<cxd>(ctx, kMaxM0 * sizeof(cxd));
    CKC(cudaMemsetAsync(ctx->d_st, 0, sizeof(RRStatus), ctx->s));
    CKC(cudaMallocHost((void **)&ctx->h_st, sizeof(RRStatus)));
    CKC(cudaMallocHost((void **)&ctx->h_small, 4 * sizeof(double)));
    CKC(cudaStreamSynchronize(ctx->s));
    check_launch(ctx, "init");
  }
}

}  // namespace

extern "C" {

feast_nh_status feast_nh_init(feast_nh_ctx **out, const feast_nh_csr *A, const feast_nh_csr *B,
                              const feast_nh_contour *contour, int32_t m0, const feast_nh_opts *opts,
                              void *stream) {
  if (!out) return FEAST_NH_EINVAL;
  *out = nullptr;
  feast_nh_ctx *ctx = new feast_nh_ctx();
  try {
    init_ctx(ctx, A, B, contour, m0, opts, stream, false);
  } catch (const Fail &f) {
    feast_nh_destroy(ctx);
    return f.st;
  }
  *out = ctx;
  return FEAST_NH_OK;
}

feast_nh_status feast_nh_filter(feast_nh_ctx *ctx, const void *Y, const void *Yh, void *Q, void *Qh, int32_t m) {
  if (!ctx) return FEAST_NH_EINVAL;
  try {
    REQ(Y && Q && Qh && m >= 1 && m <= ctx->m0, "filter: bad block pointers or m");
    REQ(cs_mode(ctx) || Yh, "filter: Yh is required unless the problem is complex symmetric");
    CKC(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->s));
    ctx->krylov_its = 0;
    do_filter(ctx, (const cxd *)Y, (const cxd *)Yh, (cxd *)Q, (cxd *)Qh, m);
    // the filter's status: device error word and the largest relative
    // residual of the shifted solves (one small read)
    CKC(cudaMemcpyAsync(ctx->h_small, ctx->d_maxrel, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    CKC(cudaMemcpyAsync(ctx->h_small + 1, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    CKC(cudaStreamSynchronize(ctx->s));
    int herr = 0;
    std::memcpy(&herr, ctx->h_small + 1, sizeof(int));
    const feast_nh_status es = status_from_err(ctx, herr);
    if (es != FEAST_NH_OK) return es;
    if (!krylov(ctx)) ctx->inner_res = ctx->h_small[0];
    if (inner_missed(ctx)) {
      char msg[200];
      if (krylov(ctx))
        std::snprintf(msg, sizeof msg, "BiCGStab stopped at inner_max iterations above inner_tol (largest relative "
                                       "residual %.3g; outputs hold the last iterate)", ctx->inner_res);
      else
        std::snprintf(msg, sizeof msg, "the refined shifted solves stopped at inner_max steps above inner_tol "
                                       "(largest relative residual %.3g; outputs hold the last iterate)",
                      ctx->inner_res);
      ctx->err = msg;
      return FEAST_NH_EINNER;
    }
  } catch (const Fail &f) {
    return f.st;
  }
  return FEAST_NH_OK;
}

feast_nh_status feast_nh_rr(feast_nh_ctx *ctx, const void *Q, const void *Qh, int32_t m, double *lambda, void *Y,
                            void *Yh, int32_t *m_new, feast_nh_info *info) {
  if (!ctx) return FEAST_NH_EINVAL;
  try {
    REQ(Q && Qh && lambda && Y && Yh && m_new && m >= 1 && m <= ctx->m0, "rr: bad arguments");
    CKC(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->s));
    const int mt = do_rr(ctx, (const cxd *)Q, (const cxd *)Qh, m, (cxd *)Y, (cxd *)Yh);
    CKC(cudaMemcpyAsync(lambda, ctx->lam, (size_t)mt * sizeof(cxd), cudaMemcpyDeviceToDevice, ctx->s));
    read_status(ctx);
    *m_new = mt;
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->m_tilde = mt;
      info->m_r = ctx->h_st->m_r;
      info->m_s = ctx->h_st->m_s;
      info->m = ctx->h_st->m;
      info->converged = ctx->h_st->conv;
      info->max_res = ctx->h_st->max_res;
      info->kl = ctx->kl;
      info->ku = ctx->ku;
      info->n_factorizations = banded(ctx) ? ctx->nf : 0;
      info->pivot_min = ctx->piv_min;
      info->pivot_max = ctx->piv_max;
    }
    int herr = 0;
    std::memcpy(&herr, ctx->h_small + 1, sizeof(int));
    const feast_nh_status es = status_from_err(ctx, herr);
    if (es != FEAST_NH_OK) return es;
  } catch (const Fail &f) {
    return f.st;
  }
  return FEAST_NH_OK;
}

feast_nh_status feast_nh_solve(feast_nh_ctx *ctx, const void *Y0, const void *Yh0, double *lambda, void *X,
                               void *Xh, double *res, int32_t *m_found, feast_nh_info *info) {
  if (!ctx) return FEAST_NH_EINVAL;
  feast_nh_status ret = FEAST_NH_OK;
  try {
    const bool cs = cs_mode(ctx);
    REQ(Y0 && (cs || Yh0) && lambda && X && Xh && m_found, "solve: bad arguments");
    const int n = ctx->n, m0 = ctx->m0;
    cudaStream_t s = ctx->s;
    CKC(cudaEventRecord(ctx->ev[0], s));
    CKC(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s));
    ctx->factored = false;  // each solve factorises afresh and keeps the factors for its iterations
    ctx->have_prev = 0;
    ctx->n_inner_fail = 0;
    ctx->krylov_its = 0;
    ev_harvest(ctx->ev_solve);
    ev_harvest(ctx->ev_resid);
    ctx->ev_solve.ms = ctx->ev_resid.ms = 0;
    ctx->ev_solve.launches = ctx->ev_resid.launches = 0;
    CKC(cudaMemcpyAsync(ctx->Yw, Y0, (size_t)n * m0 * sizeof(cxd), cudaMemcpyDeviceToDevice, s));
    if (cs)
      launch_copy_conj(ctx->Yw, ctx->Yhw, (size_t)n * m0, s);
    else
      CKC(cudaMemcpyAsync(ctx->Yhw, Yh0, (size_t)n * m0 * sizeof(cxd), cudaMemcpyDeviceToDevice, s));
    int m = m0, it = 0, mt = m0;
    double t_filter = 0, t_rr = 0;
    bool conv = false;
    for (it = 1; it <= ctx->o.max_iter; ++it) {
      if (!ctx->factored) factorize(ctx);
      CKC(cudaEventRecord(ctx->ev[1], s));
      // The first iteration only supplies the start subspace of the second,
      // whose filter damps its errors by the convergence rate: its shifted
      // systems need only the accuracy of the single-precision factors (one
      // unchecked FP32 solve; with FP64 factors a relative residual of 1e-2
      // stops the refinement), later iterations are refined to
      // opts.inner_tol and verify the factors.
      const double tol_it = it == 1 ? std::fmax(ctx->o.inner_tol, 1e-2) : ctx->o.inner_tol;
      do_filter(ctx, ctx->Yw, ctx->Yhw, ctx->Qw, ctx->Qhw, m, tol_it, it == 1);
      CKC(cudaEventRecord(ctx->ev[2], s));
      mt = do_rr(ctx, ctx->Qw, ctx->Qhw, m, ctx->Yw, ctx->Yhw);
      CKC(cudaEventRecord(ctx->ev[3], s));
      read_status(ctx);
      // Sec. 2.7 compares the next B_Q with these Ritz values; Ritz values
      // from a filter that was not solved to inner_tol (the 1e-2 first pass,
      // unless the banded FP64 factors met inner_tol anyway) are no reference
      if (!(tol_it <= ctx->o.inner_tol || (banded(ctx) && ctx->h_small[0] <= ctx->o.inner_tol))) ctx->have_prev = 0;
      float a = 0, b = 0;
      cudaEventElapsedTime(&a, ctx->ev[1], ctx->ev[2]);
      cudaEventElapsedTime(&b, ctx->ev[2], ctx->ev[3]);
      t_filter += a;
      t_rr += b;
      int herr = 0;
      std::memcpy(&herr, ctx->h_small + 1, sizeof(int));
      const feast_nh_status es = status_from_err(ctx, herr);
      if (es != FEAST_NH_OK) throw Fail{es};
      if (!krylov(ctx)) ctx->inner_res = ctx->h_small[0];
      if (inner_missed(ctx)) ++ctx->n_inner_fail;
      conv = ctx->h_st->conv != 0;
      if (conv) break;
      m = mt;
    }
    if (it > ctx->o.max_iter) it = ctx->o.max_iter;
    const int mout = ctx->h_st->m;
    finalize_output(ctx, ctx->Yw, ctx->Yhw, mt, mout, (cxd *)X, (cxd *)Xh, m0, lambda, res);
    CKC(cudaEventRecord(ctx->ev[3], s));
    CKC(cudaStreamSynchronize(s));
    float tot = 0;
    cudaEventElapsedTime(&tot, ctx->ev[0], ctx->ev[3]);
    *m_found = mout;
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->iterations = it;
      info->m_tilde = mt;
      info->m_r = ctx->h_st->m_r;
      info->m_s = ctx->h_st->m_s;
      info->m = mout;
      info->converged = conv;
      info->kl = ctx->kl;
      info->ku = ctx->ku;
      info->max_res = ctx->h_st->max_res;
      info->inner_res = ctx->inner_res;
      info->inner_steps = ctx->inner_steps;
      info->t_factor_ms = ctx->t_factor;
      info->t_filter_ms = t_filter;
      info->t_rr_ms = t_rr;
      info->t_total_ms = tot;
      info->t_solve_kernel_ms = ctx->ev_solve.ms;
      info->t_resid_kernel_ms = ctx->ev_resid.ms;
      info->n_solve_launches = ctx->ev_solve.launches;
      info->n_resid_launches = ctx->ev_resid.launches;
      info->n_factorizations = banded(ctx) ? ctx->nf : 0;
      info->inner_fail = ctx->n_inner_fail;
      info->pivot_min = ctx->piv_min;
      info->pivot_max = ctx->piv_max;
      info->krylov_iterations = ctx->krylov_its;
    }
    if (!conv) {
      if (ctx->n_inner_fail > 0) {
        char msg[200];
        std::snprintf(msg, sizeof msg,
                      "no convergence within max_iter outer iterations; the shifted solves of %d filter(s) stopped "
                      "above their tolerance (largest relative residual %.3g)",
                      ctx->n_inner_fail, ctx->inner_res);
        ctx->err = msg;
        ret = FEAST_NH_EINNER;
      } else {
        ctx->err = "no convergence within max_iter outer iterations";
        ret = FEAST_NH_ENOCONV;
      }
    }
  } catch (const Fail &f) {
    return f.st;
  }
  return ret;
}

uint64_t feast_nh_kernel_launches(void) { return g_launches.load(); }

feast_nh_status feast_nh_multishift_spmm(feast_nh_ctx *ctx, const void *P, void *V, int32_t m, int32_t side) {
  if (!ctx) return FEAST_NH_EINVAL;
  try {
    REQ(P && V && m >= 1 && m <= ctx->m0 && (side == 0 || side == 1), "multishift_spmm: bad arguments");
    REQ(!ctx->rr_only, "multishift_spmm: context has no operator");
    if (side == 0)
      launch_multishift_spmm_f32(ctx->A, ctx->hasB ? &ctx->B : nullptr, ctx->ne, ctx->dz, 0, (const cxf *)P,
                                 (cxf *)V, m, 0, ctx->max_nnz[0], ctx->s);
    else
      launch_multishift_spmm_f32(ctx->AH, ctx->hasB ? &ctx->BH : nullptr, ctx->ne, ctx->dz, 1, (const cxf *)P,
                                 (cxf *)V, m, 0, ctx->max_nnz[1], ctx->s);
    check_launch(ctx, "multishift_spmm");
  } catch (const Fail &f) {
    return f.st;
  }
  return FEAST_NH_OK;
}

feast_nh_status feast_nh_small_eig(feast_nh_ctx *ctx, const void *M, int32_t m, void *lambda, void *V) {
  if (!ctx) return FEAST_NH_EINVAL;
  try {
    REQ(M && lambda && V && m >= 1 && m <= kMaxM0, "small_eig: bad arguments (1 <= m <= 128)");
    CKC(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->s));
    small_eig((const cxd *)M, m, (cxd *)lambda, (cxd *)V, ctx->swork, ctx->d_err, ctx->s);
    check_launch(ctx, "small_eig");
    CKC(cudaMemcpyAsync(ctx->h_small + 1, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    CKC(cudaStreamSynchronize(ctx->s));
    int herr = 0;
    std::memcpy(&herr, ctx->h_small + 1, sizeof(int));
    const feast_nh_status es = status_from_err(ctx, herr);
    if (es != FEAST_NH_OK) return es;
  } catch (const Fail &f) {
    return f.st;
  }
  return FEAST_NH_OK;
}

feast_nh_status feast_nh_gram(feast_nh_ctx *ctx, const void *X, const void *Y, int32_t mx, int32_t my, void *G,
                              int32_t method) {
  if (!ctx) return FEAST_NH_EINVAL;
  try {
    REQ(X && Y && G && mx >= 1 && mx <= kMaxM0 && my >= 1 && my <= kMaxM0 &&
            (method == FEAST_NH_PROJ_FP64 || method == FEAST_NH_PROJ_TENSOR),
        "gram: bad arguments (1 <= mx, my <= 128, method FP64 or TENSOR)");
    const int keep = ctx->o.projection;
    ctx->o.projection = method;
    CKC(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->s));
    proj_gram(ctx, (const cxd *)X, mx, mx, (const cxd *)Y, my, my, (cxd *)G);
    ctx->o.projection = keep;
    check_launch(ctx, "gram");
    CKC(cudaMemcpyAsync(ctx->h_small + 1, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    CKC(cudaStreamSynchronize(ctx->s));
    int herr = 0;
    std::memcpy(&herr, ctx->h_small + 1, sizeof(int));
    const feast_nh_status es = status_from_err(ctx, herr);
    if (es != FEAST_NH_OK) return es;
  } catch (const Fail &f) {
    return f.st;
  }
  return FEAST_NH_OK;
}

feast_nh_status feast_nh_block_product(feast_nh_ctx *ctx, const void *X, const void *S, int32_t mx, int32_t mz,
                                       void *Z, int32_t method) {
  if (!ctx) return FEAST_NH_EINVAL;
  try {
    REQ(X && S && Z && mx >= 1 && mx <= kMaxM0 && mz >= 1 && mz <= kMaxM0 &&
            (method == FEAST_NH_PROJ_FP64 || method == FEAST_NH_PROJ_TENSOR),
        "block_product: bad arguments (1 <= mx, mz <= 128, method FP64 or TENSOR)");
    const int keep = ctx->o.projection;
    ctx->o.projection = method;
    CKC(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->s));
    proj_block(ctx, (const cxd *)X, mx, mx, (const cxd *)S, mz, mz, (cxd *)Z, mz);
    ctx->o.projection = keep;
    check_launch(ctx, "block_product");
    CKC(cudaMemcpyAsync(ctx->h_small + 1, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    CKC(cudaStreamSynchronize(ctx->s));
    int herr = 0;
    std::memcpy(&herr, ctx->h_small + 1, sizeof(int));
    const feast_nh_status es = status_from_err(ctx, herr);
    if (es != FEAST_NH_OK) return es;
  } catch (const Fail &f) {
    return f.st;
  }
  return FEAST_NH_OK;
}

feast_nh_status feast_nh_set_network(feast_nh_ctx *ctx, feast_nh_net *net, int32_t N, float kappa,
                                     const float *features, int32_t nfeat) {
  if (!ctx) return FEAST_NH_EINVAL;
  try {
    REQ(fgmres(ctx), "set_network: the context's inner solver is not FGMRES");
    REQ(net && N >= 2 && (long long)N * N == ctx->n, "set_network: the operator is not on an N x N grid (n = N^2)");
    REQ(nfeat >= 0 && nfeat <= 28 && (nfeat == 0 || features), "set_network: 0 <= nfeat <= 28");
    ctx->net = net;
    ctx->net_N = N;
    ctx->net_kappa = kappa;
    ctx->net_nfeat = nfeat;
    if (nfeat) CKC(cudaMemcpy(ctx->net_feat, features, nfeat * sizeof(float), cudaMemcpyHostToDevice));
  } catch (const Fail &f) {
    return f.st;
  }
  return FEAST_NH_OK;
}

feast_nh_status feast_nh_learned_pairs(feast_nh_ctx *ctx, const void *R, int32_t m, int32_t N, float kappa,
                                      const float *features, int32_t nfeat, float *Xin, float *T) {
  if (!ctx) return FEAST_NH_EINVAL;
  try {
    REQ(banded(ctx) && !ctx->rr_only, "learned_pairs: needs the banded direct solver (exact solves)");
    REQ(R && Xin && T && m >= 1 && m <= ctx->m0, "learned_pairs: bad arguments");
    REQ(N >= 2 && (long long)N * N == ctx->n, "learned_pairs: the operator is not on an N x N grid");
    REQ(nfeat >= 0 && nfeat <= 28 && (nfeat == 0 || features), "learned_pairs: 0 <= nfeat <= 28");
    CKC(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->s));
    // exact node solutions X_j = (z_j B - A)^{-1} R (both sides are solved;
    // the right side's node blocks are kept), refined to opts.inner_tol
    do_filter(ctx, (const cxd *)R, (const cxd *)R, ctx->T1, ctx->T2, m);
    float *feat = nullptr;
    if (nfeat) {
      feat = reinterpret_cast<float *>(ctx->cn);  // 4 * 128 doubles of room
      CKC(cudaMemcpyAsync(feat, features, nfeat * sizeof(float), cudaMemcpyHostToDevice, ctx->s));
    }
    const int g = launch_colnorm2((const cxd *)R, m, m, ctx->n, ctx->colp, ctx->s);
    launch_reduce_parts(ctx->colp, g, m, ctx->bynorm2, ctx->s);
    launch_learned_pairs((const cxd *)R, ctx->Xn, ctx->ne, ctx->n, m, ctx->dz, kappa, feat, nfeat, ctx->bynorm2, Xin,
                         T, ctx->s);
    check_launch(ctx, "learned_pairs");
    CKC(cudaMemcpyAsync(ctx->h_small, ctx->d_maxrel, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    CKC(cudaStreamSynchronize(ctx->s));
    if (!(ctx->h_small[0] <= ctx->o.inner_tol)) {
      ctx->err = "learned_pairs: the shifted solves stopped above inner_tol";
      return FEAST_NH_EINNER;
    }
  } catch (const Fail &f) {
    return f.st;
  }
  return FEAST_NH_OK;
}

feast_nh_status feast_nh_operator_loss(feast_nh_ctx *ctx, const float *out, const float *T, int32_t m, int32_t N,
                                      int32_t side, float *gout, double *loss) {
  if (!ctx) return FEAST_NH_EINVAL;
  try {
    REQ(out && T && gout && loss && m >= 1 && m <= ctx->m0 && (side == 0 || side == 1), "operator_loss: bad arguments");
    REQ(N >= 2 && (long long)N * N == ctx->n, "operator_loss: the operator is not on an N x N grid");
    double *dl = ctx->d_maxrel;  // one double of device scratch
    CKC(cudaMemsetAsync(dl, 0, sizeof(double), ctx->s));
    const CsrView &M = side == 0 ? ctx->A : ctx->AH;
    const CsrView &MH = side == 0 ? ctx->AH : ctx->A;
    float *ybuf = reinterpret_cast<float *>(ctx->dfg ? (void *)ctx->dfg : (void *)ctx->Xn);
    launch_operator_loss(M, MH, ctx->ne, ctx->n, m, ctx->dz, side, out, T, ybuf, gout, dl, ctx->s);
    check_launch(ctx, "operator_loss");
    CKC(cudaMemcpyAsync(loss, dl, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    CKC(cudaStreamSynchronize(ctx->s));
  } catch (const Fail &f) {
    return f.st;
  }
  return FEAST_NH_OK;
}

feast_nh_status feast_nh_inject_device_error(feast_nh_ctx *ctx, uint32_t bits) {
  if (!ctx) return FEAST_NH_EINVAL;
  ctx->inject_bits |= bits;
  return FEAST_NH_OK;
}

feast_nh_status feast_nh_multishift_residual(feast_nh_ctx *ctx, const void *X, const void *BY, void *R, void *Q,
                                             int32_t m, int32_t r_single) {
  if (!ctx) return FEAST_NH_EINVAL;
  try {
    REQ(X && BY && R && m >= 1 && m <= ctx->m0, "multishift_residual: bad arguments");
    const CsrView *Bp = ctx->hasB ? &ctx->B : nullptr;
    if (r_single)
      launch_multishift_residual<float>(ctx->A, Bp, ctx->ne, ctx->dz, ctx->dw, (const cxd *)X, (const cxd *)BY,
                                        (cxf *)R, (cxd *)Q, nullptr, m, nullptr, ctx->s);
    else
      launch_multishift_residual<double>(ctx->A, Bp, ctx->ne, ctx->dz, ctx->dw, (const cxd *)X, (const cxd *)BY,
                                         (cxd *)R, (cxd *)Q, nullptr, m, nullptr, ctx->s);
    check_launch(ctx, "multishift_residual");
  } catch (const Fail &f) {
    return f.st;
  }
  return FEAST_NH_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Many independent problems (Sec. 4.1: contours are independent): the contour
// integration of every problem runs in one persistent launch (batch.cu); the
// Rayleigh-Ritz step of each problem runs on that problem's own stream, all
// problems concurrently, with the single-problem kernels.
// ---------------------------------------------------------------------------
struct feast_nh_batch {
  int nprob = 0, ne = 0, m0 = 0;
  size_t ntot = 0;
  cudaStream_t s = nullptr;
  feast_nh_opts o{};
  std::vector<feast_nh_ctx *> ctx;
  std::vector<BatchProb> hp;
  std::vector<int> mt, conv, iters, mfound;
  BatchProb *dprob = nullptr;
  BatchTile *dtiles = nullptr;
  int ntiles = 0, tile_rows = 128, threads = 256, grid = 0, max_tiles = 0;
  cxd *Y = nullptr, *Yh = nullptr, *Q = nullptr, *Qh = nullptr, *diag = nullptr, *X = nullptr;
  BatchLaunch L{};
  BatchStats *h_stats = nullptr;
  int *h_err = nullptr;
  std::vector<void *> allocs;
  std::vector<bool> pooled;
  std::string err;
  cudaEvent_t ev[4] = {};
  std::vector<cudaEvent_t> ev_rr;
  double t_autotune = 0;
  int krylov_its = 0, refine_steps = 0, inner_fail = 0;
  double inner_res = 0;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};  // filter launch sequence (first / later tolerance)
  cudaStream_t gs = nullptr;                      // private stream the sequence is captured and replayed on
  cudaEvent_t gev[2] = {nullptr, nullptr};        // ordering with the caller's stream
  bool graph_ok = true;                           // stream capture of the sequence available
  int graph_used = 0;
};

namespace {

#define BCK(...)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (__VA_ARGS__);                                                        \
    if (e_ != cudaSuccess) {                                                               \
      b->err = std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_);                  \
      throw Fail{e_ == cudaErrorMemoryAllocation ? FEAST_NH_ENOMEM : FEAST_NH_ECUDA};      \
    }                                                                                      \
  } while (0)
#define BREQ(cond, msg)                  \
  do {                                   \
    if (!(cond)) {                       \
      b->err = msg;                      \
      throw Fail{FEAST_NH_EINVAL};       \
    }                                    \
  } while (0)

template <typename P>
P *balloc(feast_nh_batch *b, size_t bytes) {
  void *p = nullptr;
  if (bytes == 0) bytes = 16;
  bool pooled = false;
  BCK(pool::alloc(&p, bytes, b->s, &pooled));
  b->allocs.push_back(p);
  b->pooled.push_back(pooled);
  return reinterpret_cast<P *>(p);
}

bool batch_fp32(const feast_nh_batch *b) { return b->o.precision == FEAST_NH_PREC_FP32_IR; }

// Tiles of `rows` consecutive rows of one problem, problems in order.
void batch_tiles(feast_nh_batch *b, int rows) {
  std::vector<BatchTile> t;
  for (int p = 0; p < b->nprob; ++p) {
    b->hp[p].tb = (int)t.size();
    for (int r0 = 0; r0 < b->hp[p].n; r0 += rows) t.push_back(BatchTile{p, r0, std::min(b->hp[p].n, r0 + rows), 0});
    b->hp[p].te = (int)t.size();
  }
  b->ntiles = (int)t.size();
  BREQ(b->ntiles <= b->max_tiles, "batch: tile table overflow");
  // pageable host sources: these copies complete before the call returns
  BCK(cudaMemcpyAsync(b->dtiles, t.data(), t.size() * sizeof(BatchTile), cudaMemcpyHostToDevice, b->s));
  BCK(cudaMemcpyAsync(b->dprob, b->hp.data(), b->hp.size() * sizeof(BatchProb), cudaMemcpyHostToDevice, b->s));
  BCK(cudaStreamSynchronize(b->s));
  b->tile_rows = rows;
}

void batch_upload_probs(feast_nh_batch *b) {
  BCK(cudaMemcpyAsync(b->dprob, b->hp.data(), b->hp.size() * sizeof(BatchProb), cudaMemcpyHostToDevice, b->s));
}

// One launch of the batched contour integration; returns after the launch is
// enqueued.  tol: refinement target of the shifted solves.
void batch_filter_run(feast_nh_batch *b, double tol, int nsteps, int kmax) {
  b->L.ntiles = b->ntiles;
  b->L.tol = tol;
  b->L.nsteps = nsteps;
  b->L.kmax = kmax;
  const cudaError_t e = batch_fp32(b) ? batch_filter_launch<float>(b->L, b->grid, b->threads, b->s)
                                      : batch_filter_launch<double>(b->L, b->grid, b->threads, b->s);
  BCK(e);
}

// The launch sequence of one contour integration (resets of the barrier, the
// counters and the statistics, the cooperative kernel, the read-back of the
// statistics and the error word into pinned host memory) captured once as a
// CUDA graph per tolerance and replayed each outer iteration.  If the stream
// capture is not available the same sequence is launched directly.
void batch_filter_iteration(feast_nh_batch *b, int which, double tol) {
  // the caller's stream may be the legacy default stream, which cannot be
  // captured: the sequence runs on the batch's own stream, ordered by events
  BCK(cudaEventRecord(b->gev[0], b->s));
  BCK(cudaStreamWaitEvent(b->gs, b->gev[0], 0));
  cudaStream_t s = b->gs;
  auto enqueue = [&]() -> cudaError_t {
    b->L.ntiles = b->ntiles;
    b->L.tol = tol;
    b->L.nsteps = b->o.inner_max;
    b->L.kmax = b->o.krylov_max;
    cudaError_t e = batch_fp32(b) ? batch_filter_launch<float>(b->L, b->grid, b->threads, s)
                                  : batch_filter_launch<double>(b->L, b->grid, b->threads, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->h_stats, b->L.stats, sizeof(BatchStats), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_err, b->L.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    return e;
  };
  if (!b->gexec[which] && b->graph_ok) {
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    const cudaError_t e1 = ok ? enqueue() : cudaErrorUnknown;
    const cudaError_t e2 = ok ? cudaStreamEndCapture(s, &g) : cudaErrorUnknown;
    ok = ok && e1 == cudaSuccess && e2 == cudaSuccess && g;
    if (ok && cudaGraphInstantiate(&b->gexec[which], g, 0) != cudaSuccess) {
      b->gexec[which] = nullptr;
      ok = false;
    }
    if (g) cudaGraphDestroy(g);
    if (!ok) {
      b->graph_ok = false;
      cudaGetLastError();  // a refused capture leaves no error behind
    }
  }
  if (b->gexec[which]) {
    BCK(cudaGraphLaunch(b->gexec[which], s));
    note_launch();
    b->graph_used = 1;
  } else {
    BCK(enqueue());
    b->graph_used = 0;
  }
  BCK(cudaEventRecord(b->gev[1], s));
  BCK(cudaStreamWaitEvent(b->s, b->gev[1], 0));
}

// Project autotuner: times the persistent launch (three Krylov iterations of
// one refinement step on a fixed input) for each candidate shape -- threads
// per CTA, CTAs per SM (the cooperative grid), rows per tile -- and keeps
// the fastest.
void batch_autotune(feast_nh_batch *b) {
  int sms = 152, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  launch_fill_pattern(b->Y, b->ntot * b->m0, b->s);
  launch_fill_pattern(b->Yh, b->ntot * b->m0, b->s);
  float best = 1e30f;
  int bt = 256, bg = 0, br = 128;
  const int threads_c[] = {256, 512};
  const int rows_c[] = {64, 256};
  BCK(cudaEventRecord(b->ev[2], b->s));
  for (int th : threads_c) {
    const int occ = batch_fp32(b) ? batch_filter_max_ctas_per_sm<float>(th) : batch_filter_max_ctas_per_sm<double>(th);
    if (occ < 1) continue;
    for (int per_sm = 1; per_sm <= std::min(occ, 2); per_sm *= 2)
      for (int rows : rows_c) {
        batch_tiles(b, rows);
        b->threads = th;
        b->grid = std::min(sms * per_sm, std::max(1, b->ntiles));
        batch_filter_run(b, 0.0, 1, 3);
        BCK(cudaEventRecord(b->ev[0], b->s));
        batch_filter_run(b, 0.0, 1, 3);
        BCK(cudaEventRecord(b->ev[1], b->s));
        BCK(cudaEventSynchronize(b->ev[1]));
        float ms = 0;
        BCK(cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
        if (ms < best) {
          best = ms;
          bt = th;
          bg = b->grid;
          br = rows;
        }
      }
  }
  BCK(cudaEventRecord(b->ev[3], b->s));
  BCK(cudaEventSynchronize(b->ev[3]));
  float tot = 0;
  cudaEventElapsedTime(&tot, b->ev[2], b->ev[3]);
  b->t_autotune = tot;
  BREQ(bg > 0, "no launch shape of the batched solver fits this device");
  b->threads = bt;
  b->grid = bg;
  batch_tiles(b, br);
  int herr = 0;
  BCK(cudaMemcpyAsync(&herr, b->L.err, sizeof(int), cudaMemcpyDeviceToHost, b->s));
  BCK(cudaStreamSynchronize(b->s));
  BREQ(!(herr & DEVERR_TIMEOUT), "a grid barrier of the batched solver gave up while tuning");
}

void batch_destroy_impl(feast_nh_batch *b) {
  if (!b) return;
  if (b->s) cudaStreamSynchronize(b->s);
  for (auto *c : b->ctx) feast_nh_destroy(c);
  for (size_t i = 0; i < b->allocs.size(); ++i) pool::release(b->allocs[i], b->pooled[i], b->s);
  if (b->s) cudaStreamSynchronize(b->s);
  if (b->h_stats) cudaFreeHost(b->h_stats);
  if (b->h_err) cudaFreeHost(b->h_err);
  for (auto &e : b->ev)
    if (e) cudaEventDestroy(e);
  for (auto &e : b->ev_rr)
    if (e) cudaEventDestroy(e);
  for (auto &g : b->gexec)
    if (g) cudaGraphExecDestroy(g);
  for (auto &e : b->gev)
    if (e) cudaEventDestroy(e);
  if (b->gs) {
    cudaStreamSynchronize(b->gs);
    cudaStreamDestroy(b->gs);
  }
  delete b;
}

}  // namespace

extern "C" {

feast_nh_status feast_nh_batch_init(feast_nh_batch **out, int32_t nprob, const feast_nh_csr *A,
                                    const feast_nh_contour *contours, int32_t m0, const feast_nh_opts *opts,
                                    void *stream) {
  if (!out) return FEAST_NH_EINVAL;
  *out = nullptr;
  feast_nh_batch *b = new feast_nh_batch();
  try {
    BREQ(nprob >= 1 && A && contours, "batch: nprob >= 1 problems with matrices and contours");
    BREQ(m0 >= 1 && m0 <= kMaxM0, "batch: m0 must be in [1, 128]");
    if (opts) b->o = *opts; else feast_nh_default_opts(&b->o);
    BREQ(b->o.inner_kind == FEAST_NH_INNER_BICGSTAB, "batch: the inner solver is BiCGStab (inner_kind)");
    BREQ(b->o.problem == FEAST_NH_PROBLEM_GENERAL, "batch: general problems only");
    BREQ(b->o.krylov_max >= 1 && b->o.inner_max >= 1, "batch: krylov_max and inner_max must be >= 1");
    const int ne = contours[0].ne;
    BREQ(ne >= 1 && ne <= kBatchMaxNe, "batch: contour.ne must be in [1, 16]");
    b->nprob = nprob;
    b->ne = ne;
    b->m0 = m0;
    b->s = reinterpret_cast<cudaStream_t>(stream);
    b->hp.assign(nprob, BatchProb{});
    b->mt.assign(nprob, m0);
    b->conv.assign(nprob, 0);
    b->iters.assign(nprob, 0);
    b->mfound.assign(nprob, 0);
    for (auto &e : b->ev) BCK(cudaEventCreateWithFlags(&e, cudaEventDefault));
    for (auto &e : b->gev) BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    BCK(cudaStreamCreateWithFlags(&b->gs, cudaStreamNonBlocking));
    // per-problem contexts (Rayleigh-Ritz workspace, transposed CSR, nodes)
    feast_nh_opts ro = b->o;
    ro.inner_kind = FEAST_NH_INNER_BANDED;
    ro.precision = FEAST_NH_PREC_FP64;
    size_t off = 0;
    for (int p = 0; p < nprob; ++p) {
      BREQ(contours[p].ne == ne, "batch: every contour must have the same ne");
      BREQ(A[p].n >= m0, "batch: every problem needs n >= m0");
      cudaStream_t sp = nullptr;
      BCK(cudaStreamCreateWithFlags(&sp, cudaStreamNonBlocking));
      feast_nh_ctx *c = new feast_nh_ctx();
      c->s = sp;
      c->own_stream = true;
      b->ctx.push_back(c);
      try {
        init_ctx(c, &A[p], nullptr, &contours[p], m0, &ro, sp, true);
      } catch (const Fail &f) {
        b->err = "batch problem " + std::to_string(p) + ": " + c->err;
        throw;
      }
      c->own_stream = true;
      BatchProb &bp = b->hp[p];
      bp.A = c->A;
      bp.AH = c->AH;
      bp.off = off;
      bp.n = A[p].n;
      bp.m = m0;
      bp.active = 1;
      for (int j = 0; j < ne; ++j) {
        bp.z[j] = c->hz[j];
        bp.w[j] = c->hw[j];
      }
      off += (size_t)A[p].n;
      cudaEvent_t e = nullptr;
      BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      b->ev_rr.push_back(e);
    }
    b->ntot = off;
    const size_t blk = b->ntot * m0;         // right-hand-side block elements
    const size_t nblk = blk * ne;            // node-major block elements
    const size_t es = batch_fp32(b) ? sizeof(cxf) : sizeof(cxd);
    b->Y = balloc<cxd>(b, blk * sizeof(cxd));
    b->Yh = balloc<cxd>(b, blk * sizeof(cxd));
    b->Q = balloc<cxd>(b, blk * sizeof(cxd));
    b->Qh = balloc<cxd>(b, blk * sizeof(cxd));
    b->X = balloc<cxd>(b, nblk * sizeof(cxd));
    b->diag = balloc<cxd>(b, b->ntot * sizeof(cxd));
    for (int p = 0; p < nprob; ++p) launch_csr_diag(b->hp[p].A, b->diag + b->hp[p].off, b->s);
    for (int k = 0; k < 9; ++k) b->L.kblk[k] = balloc<void>(b, nblk * es);
    // tiles: room for the smallest tile size the tuner tries
    int maxt = 0;
    for (int p = 0; p < nprob; ++p) maxt += ceil_div(b->hp[p].n, 64);
    b->max_tiles = maxt;
    b->dtiles = balloc<BatchTile>(b, (size_t)maxt * sizeof(BatchTile));
    b->dprob = balloc<BatchProb>(b, (size_t)nprob * sizeof(BatchProb));
    const size_t PS = (size_t)ne * m0;
    b->L.part = balloc<void>(b, (size_t)maxt * 2 * PS * es);
    b->L.partd = balloc<double>(b, (size_t)maxt * PS * sizeof(double));
    b->L.partb = balloc<double>(b, (size_t)maxt * m0 * sizeof(double));
    const size_t S = (size_t)nprob * PS;
    BatchScal &sc = b->L.sc;
    sc.rho = balloc<cxd>(b, S * sizeof(cxd));
    sc.alpha = balloc<cxd>(b, S * sizeof(cxd));
    sc.omega = balloc<cxd>(b, S * sizeof(cxd));
    sc.beta = balloc<cxd>(b, S * sizeof(cxd));
    sc.bn2 = balloc<double>(b, (size_t)nprob * m0 * sizeof(double));
    sc.rel = balloc<double>(b, S * sizeof(double));
    sc.stop2 = balloc<double>(b, S * sizeof(double));
    sc.act = balloc<int>(b, S * sizeof(int));
    sc.act0 = balloc<int>(b, S * sizeof(int));
    b->L.bar = balloc<unsigned>(b, 4 * sizeof(unsigned));
    b->L.ctl = balloc<int>(b, 8 * sizeof(int));
    b->L.stats = balloc<BatchStats>(b, sizeof(BatchStats));
    b->L.err = balloc<int>(b, sizeof(int));
    BCK(cudaMemsetAsync(b->L.err, 0, sizeof(int), b->s));
    BCK(cudaMallocHost((void **)&b->h_stats, sizeof(BatchStats)));
    BCK(cudaMallocHost((void **)&b->h_err, sizeof(int)));
    b->L.nprob = nprob;
    b->L.ne = ne;
    b->L.m0 = m0;
    b->L.side0 = 0;
    b->L.side1 = 1;
    b->L.prob = b->dprob;
    b->L.tiles = b->dtiles;
    b->L.Y = b->Y;
    b->L.Yh = b->Yh;
    b->L.Q = b->Q;
    b->L.Qh = b->Qh;
    b->L.diag = b->diag;
    b->L.X = b->X;
    b->L.tau_min = batch_fp32(b) ? 1e-5 : 0.0;
    // a grid barrier waits at most ~8 s (at 2 GHz) before the launch gives up
    b->L.spin_limit = 16000000000LL;
    batch_upload_probs(b);
    BCK(cudaStreamSynchronize(b->s));
    for (auto *c : b->ctx) BCK(cudaStreamSynchronize(c->s));
    batch_autotune(b);
  } catch (const Fail &f) {
    feast_nh_status st = f.st;
    std::string msg = b->err;
    batch_destroy_impl(b);
    (void)msg;
    return st;
  }
  *out = b;
  return FEAST_NH_OK;
}

void feast_nh_batch_destroy(feast_nh_batch *b) { batch_destroy_impl(b); }

const char *feast_nh_batch_last_error(const feast_nh_batch *b) { return b ? b->err.c_str() : ""; }

feast_nh_status feast_nh_batch_solve(feast_nh_batch *b, const void *Y0, const void *Yh0, double *lambda, void *X,
                                     void *Xh, double *res, int32_t *m_found, int32_t *iterations,
                                     feast_nh_batch_info *info) {
  if (!b) return FEAST_NH_EINVAL;
  feast_nh_status ret = FEAST_NH_OK;
  try {
    BREQ(Y0 && Yh0 && lambda && X && Xh && res && m_found, "batch_solve: bad arguments");
    cudaStream_t s = b->s;
    const int np = b->nprob, m0 = b->m0;
    BCK(cudaEventRecord(b->ev[0], s));
    BCK(cudaMemcpyAsync(b->Y, Y0, b->ntot * m0 * sizeof(cxd), cudaMemcpyDeviceToDevice, s));
    BCK(cudaMemcpyAsync(b->Yh, Yh0, b->ntot * m0 * sizeof(cxd), cudaMemcpyDeviceToDevice, s));
    BCK(cudaMemsetAsync(b->L.err, 0, sizeof(int), s));
    for (int p = 0; p < np; ++p) {
      b->hp[p].m = m0;
      b->hp[p].active = 1;
      b->mt[p] = m0;
      b->conv[p] = 0;
      b->iters[p] = 0;
      b->mfound[p] = 0;
      b->ctx[p]->have_prev = 0;
    }
    b->krylov_its = b->refine_steps = b->inner_fail = 0;
    b->inner_res = 0;
    double t_filter = 0, t_rr = 0;
    int it = 0;
    std::vector<feast_nh_status> pst(np, FEAST_NH_OK);
    for (it = 1; it <= b->o.max_iter; ++it) {
      batch_upload_probs(b);
      BCK(cudaEventRecord(b->ev[1], s));
      // the first outer iteration only supplies the start subspace of the
      // second: its shifted solves stop at a relative residual of 1e-2
      const double tol_it = it == 1 ? std::fmax(b->o.inner_tol, 1e-2) : b->o.inner_tol;
      batch_filter_iteration(b, it == 1 ? 0 : 1, tol_it);
      BCK(cudaEventRecord(b->ev[2], s));
      // Rayleigh-Ritz of every active problem on its own stream, concurrently
      std::vector<std::thread> th;
      for (int p = 0; p < np; ++p) {
        if (!b->hp[p].active) continue;
        th.emplace_back([b, p, &pst, tol_it]() {
          feast_nh_ctx *c = b->ctx[p];
          try {
            if (cudaStreamWaitEvent(c->s, b->ev[2], 0) != cudaSuccess) throw Fail{FEAST_NH_ECUDA};
            const size_t o = b->hp[p].off * b->m0;
            const int mt = do_rr(c, b->Q + o, b->Qh + o, b->hp[p].m, b->Y + o, b->Yh + o);
            read_status(c);
            if (tol_it > b->o.inner_tol) c->have_prev = 0;  // no spurious-test reference (Sec. 2.7)
            b->mt[p] = mt;
            b->conv[p] = c->h_st->conv;
            b->mfound[p] = c->h_st->m;
            if (cudaEventRecord(b->ev_rr[p], c->s) != cudaSuccess) throw Fail{FEAST_NH_ECUDA};
          } catch (const Fail &f) {
            pst[p] = f.st;
          }
        });
      }
      for (auto &t : th) t.join();
      for (int p = 0; p < np; ++p) {
        if (pst[p] != FEAST_NH_OK) {
          b->err = "batch problem " + std::to_string(p) + ": " + b->ctx[p]->err;
          throw Fail{pst[p]};
        }
        if (b->hp[p].active) BCK(cudaStreamWaitEvent(s, b->ev_rr[p], 0));
      }
      BCK(cudaEventRecord(b->ev[3], s));
      BCK(cudaEventSynchronize(b->ev[3]));
      float a = 0, c = 0;
      cudaEventElapsedTime(&a, b->ev[1], b->ev[2]);
      cudaEventElapsedTime(&c, b->ev[2], b->ev[3]);
      t_filter += a;
      t_rr += c;
      if (*b->h_err & DEVERR_TIMEOUT) {
        b->err = "a grid barrier of the batched contour integration gave up";
        throw Fail{FEAST_NH_ETIMEOUT};
      }
      const BatchStats &st = *b->h_stats;
      b->krylov_its += st.krylov_its[0] + st.krylov_its[1];
      b->refine_steps += st.steps[0] + st.steps[1];
      const double mr = std::fmax(__builtin_bit_cast(double, st.maxrel_bits[0]),
                                  __builtin_bit_cast(double, st.maxrel_bits[1]));
      b->inner_res = mr;
      if (st.unconverged[0] + st.unconverged[1] > 0) ++b->inner_fail;
      int nact = 0;
      for (int p = 0; p < np; ++p) {
        if (!b->hp[p].active) continue;
        b->iters[p] = it;
        if (b->conv[p]) {
          b->hp[p].active = 0;
        } else {
          b->hp[p].m = b->mt[p];
          ++nact;
        }
      }
      if (nact == 0) break;
    }
    if (it > b->o.max_iter) it = b->o.max_iter;
    // 5.d per problem: converged pairs first, normalised, into X, Xh (ld m0)
    int nconv = 0;
    double maxres = 0;
    for (int p = 0; p < np; ++p) {
      feast_nh_ctx *c = b->ctx[p];
      const size_t o = b->hp[p].off * m0;
      BCK(cudaStreamWaitEvent(c->s, b->ev[3], 0));
      finalize_output(c, b->Y + o, b->Yh + o, b->mt[p], b->mfound[p], (cxd *)X + o, (cxd *)Xh + o, m0,
                      lambda + (size_t)2 * p * m0, res + (size_t)p * m0);
      BCK(cudaEventRecord(b->ev_rr[p], c->s));
      BCK(cudaStreamWaitEvent(s, b->ev_rr[p], 0));
      m_found[p] = b->mfound[p];
      if (iterations) iterations[p] = b->iters[p];
      nconv += b->conv[p] ? 1 : 0;
      maxres = std::fmax(maxres, c->h_st->max_res);
    }
    BCK(cudaEventRecord(b->ev[3], s));
    BCK(cudaEventSynchronize(b->ev[3]));
    float tot = 0;
    cudaEventElapsedTime(&tot, b->ev[0], b->ev[3]);
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->iterations = it;
      info->converged_problems = nconv;
      info->inner_fail = b->inner_fail;
      info->krylov_iterations = b->krylov_its;
      info->refine_steps = b->refine_steps;
      info->threads = b->threads;
      info->tile_rows = b->tile_rows;
      info->grid = b->grid;
      info->max_res = maxres;
      info->inner_res = b->inner_res;
      info->t_filter_ms = t_filter;
      info->t_rr_ms = t_rr;
      info->t_total_ms = tot;
      info->t_autotune_ms = b->t_autotune;
      info->graph = b->graph_used;
    }
    if (nconv < np) {
      b->err = "some problems did not converge within max_iter outer iterations";
      ret = b->inner_fail ? FEAST_NH_EINNER : FEAST_NH_ENOCONV;
    }
  } catch (const Fail &f) {
    return f.st;
  }
  return ret;
}

}  // extern "C"
