// C ABI of the non-Hermitian FEAST hot path: context, contour integration,
// Rayleigh-Ritz and the outer loop of Fig. alg:three.  Host code here only
// sizes, sequences and checks device work; every numerical step runs in the
// kernels of band.cu, spmm.cu, dense.cu and rr.cu.
#include <atomic>
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
  CKC(cudaMalloc(&p, bytes));
  ctx->allocs.push_back(p);
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

void factorize(feast_nh_ctx *ctx) {
  if (krylov(ctx)) {
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
void do_filter(feast_nh_ctx *ctx, const cxd *Y, const cxd *Yh, cxd *Q, cxd *Qh, int m, double inner_tol = -1.0) {
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
  } else if (!fp32(ctx)) {
    int k = ev_begin(ctx, ctx->ev_solve);
    CKC(band_solve_sides<double, double>(n, ctx->klp, ctx->kup, ne, ctx->fmap.data(), (const cxd *)ctx->band, nullptr,
                                         BY, BhYh, 0, m,
                                         ctx->Xn,
                                         cs ? nullptr : ctx->Xhn, xns, 0, (cxd *)ctx->ysc, nullptr, ctx->s));
    ev_end(ctx, ctx->ev_solve, k);
    // Q = sum_j w_j X_j in the same pass that measures each shifted system's
    // residual, so that an inaccurate direct solve is reported, not hidden
    const int gm = launch_multishift_residual<double>(ctx->A, Bp, ne, ctx->dz, ctx->dw, ctx->Xn, BY, nullptr, Q,
                                                      ctx->part, m, nullptr, ctx->s);
    if (!cs)
      launch_multishift_residual<double>(ctx->AH, BHp, ne, ctx->dzc, ctx->dwc, ctx->Xhn, BhYh, nullptr, Qh,
                                         ctx->part + (size_t)gm * ne * m, m, nullptr, ctx->s);
    int g = launch_colnorm2(BY, m, m, n, ctx->colp, ctx->s);
    launch_reduce_parts(ctx->colp, g, m, ctx->bynorm2, ctx->s);
    if (!cs) {
      g = launch_colnorm2(BhYh, m, m, n, ctx->colp, ctx->s);
      launch_reduce_parts(ctx->colp, g, m, ctx->bynorm2 + m, ctx->s);
    }
    launch_residual_check(ctx->part, gm, ne, m, ctx->bynorm2, cs ? 1 : 2, inner_tol, ctx->d_maxrel, ctx->d_done,
                          ctx->s);
    ctx->inner_steps = 1;
  } else {
    CKC(cudaMemsetAsync(ctx->d_done, 0, sizeof(int), ctx->s));
    // the first solve takes the right-hand sides in single precision (the
    // factors' precision; the refinement restores the rest): they are staged
    // in the first n x m entries of the residual buffers, which the first
    // residual overwrites
    launch_to_cxf(BY, (cxf *)ctx->Rn, (size_t)n * m, ctx->s);
    if (!cs) launch_to_cxf(BhYh, (cxf *)ctx->Rhn, (size_t)n * m, ctx->s);
    int k0 = ev_begin(ctx, ctx->ev_solve);
    CKC(band_solve_sides<float, float>(n, ctx->klp, ctx->kup, ne, ctx->fmap.data(), (const cxf *)ctx->band,
                                       (const cxf *)ctx->dinv, (const cxf *)ctx->Rn,
                                       cs ? nullptr : (const cxf *)ctx->Rhn, 0, m, ctx->Xn, cs ? nullptr : ctx->Xhn,
                                       xns, 0, (cxf *)ctx->ysc, nullptr, ctx->s, tma_ptr(ctx), ctx->d_err));
    ev_end(ctx, ctx->ev_solve, k0);
    int g = launch_colnorm2(BY, m, m, n, ctx->colp, ctx->s);
    launch_reduce_parts(ctx->colp, g, m, ctx->bynorm2, ctx->s);
    if (!cs) {
      g = launch_colnorm2(BhYh, m, m, n, ctx->colp, ctx->s);
      launch_reduce_parts(ctx->colp, g, m, ctx->bynorm2 + m, ctx->s);
    }
    const int steps = ctx->o.inner_max < 1 ? 1 : ctx->o.inner_max;
    for (int it = 0; it < steps; ++it) {
      int kr = ev_begin(ctx, ctx->ev_resid);
      // residuals only: the node sum Q is formed once, from the final X
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
      // one 4-byte read per refinement step decides whether to go on
      CKC(cudaMemcpyAsync(ctx->h_small + 2, ctx->d_done, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
      CKC(cudaStreamSynchronize(ctx->s));
      int done = 0;
      std::memcpy(&done, ctx->h_small + 2, sizeof(int));
      ctx->inner_steps = it + 1;
      if (done) break;
      if (it + 1 < steps) {
        int ks = ev_begin(ctx, ctx->ev_solve);
        CKC(band_solve_sides<float, float>(n, ctx->klp, ctx->kup, ne, ctx->fmap.data(), (const cxf *)ctx->band,
                                           (const cxf *)ctx->dinv, (const cxf *)ctx->Rn,
                                           cs ? nullptr : (const cxf *)ctx->Rhn, xns, m, ctx->Xn,
                                           cs ? nullptr : ctx->Xhn, xns, 1, (cxf *)ctx->ysc, nullptr, ctx->s,
                                           tma_ptr(ctx), ctx->d_err));
        ev_end(ctx, ctx->ev_solve, ks);
      }
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
  return !(r <= ctx->last_inner_tol);
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
  gram(Qh, m, m, BQq, m, m, n, ctx->BQ, ctx->gpart, ctx->gchunks, s);
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
  block_times_small(Q, m, m, ctx->S, m, mt, n, ctx->Uw, mt, s);
  block_times_small(Qh, m, m, ctx->Sh, m, mt, n, ctx->Uhw, mt, s);
  // 4.a  A_U = Uh^H A U, B_U = Uh^H B U
  launch_spmm(ctx->A, nullptr, nullptr, ctx->Uw, ctx->T1, mt, nullptr, nullptr, s);
  gram(ctx->Uhw, mt, mt, ctx->T1, mt, mt, n, ctx->AU, ctx->gpart, ctx->gchunks, s);
  const cxd *BUu = ctx->Uw;
  if (ctx->hasB) {
    launch_spmm(ctx->B, nullptr, nullptr, ctx->Uw, ctx->T2, mt, nullptr, nullptr, s);
    BUu = ctx->T2;
  }
  gram(ctx->Uhw, mt, mt, BUu, mt, mt, n, ctx->BU, ctx->gpart, ctx->gchunks, s);
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
  block_times_small(ctx->Uw, mt, mt, ctx->W, mt, mt, n, Y, mt, s);
  block_times_small(ctx->Uhw, mt, mt, ctx->Wh, mt, mt, n, Yh, mt, s);
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

void feast_nh_destroy(feast_nh_ctx *ctx) {
  if (!ctx) return;
  if (ctx->s) cudaStreamSynchronize(ctx->s);
  for (void *p : ctx->allocs) cudaFree(p);
  if (ctx->h_st) cudaFreeHost(ctx->h_st);
  if (ctx->h_small) cudaFreeHost(ctx->h_small);
  for (auto &e : ctx->ev)
    if (e) cudaEventDestroy(e);
  for (EvPool *p : {&ctx->ev_solve, &ctx->ev_resid})
    for (int k = 0; k < p->made; ++k) {
      cudaEventDestroy(p->a[k]);
      cudaEventDestroy(p->b[k]);
    }
  delete ctx;
}

feast_nh_status feast_nh_init(feast_nh_ctx **out, const feast_nh_csr *A, const feast_nh_csr *B,
                              const feast_nh_contour *contour, int32_t m0, const feast_nh_opts *opts,
                              void *stream) {
  if (!out) return FEAST_NH_EINVAL;
  *out = nullptr;
  feast_nh_ctx *ctx = new feast_nh_ctx();
  try {
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
    REQ(ctx->o.inner_kind == FEAST_NH_INNER_BANDED || ctx->o.inner_kind == FEAST_NH_INNER_BICGSTAB,
        "inner_kind must be BANDED or BICGSTAB");
    REQ(ctx->o.inner_kind != FEAST_NH_INNER_BICGSTAB || ctx->o.precision == FEAST_NH_PREC_FP64,
        "the BiCGStab inner solver runs in FP64");
    REQ(ctx->o.inner_max >= 1, "inner_max must be >= 1");
    REQ(ctx->o.precision == FEAST_NH_PREC_FP64 || ctx->o.precision == FEAST_NH_PREC_FP32_IR, "bad precision");
    REQ(ctx->o.problem == FEAST_NH_PROBLEM_GENERAL || ctx->o.problem == FEAST_NH_PROBLEM_COMPLEX_SYMMETRIC,
        "bad problem kind");
    REQ(ctx->o.max_iter >= 1 && ctx->o.eps > 0 && ctx->o.eta >= 0 && ctx->o.mu > 0, "bad tolerances");
    REQ((size_t)contour->ne * m0 <= 2048, "ne * m0 must not exceed 2048");
    ctx->s = reinterpret_cast<cudaStream_t>(stream);
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
    ctx->AH = transpose_view(ctx, ctx->A);
    if (B) {
      ctx->hasB = true;
      ctx->B = make_view(*B);
      ctx->BH = transpose_view(ctx, ctx->B);
    }
    // band of (z B - A)
    ctx->d_ext = dalloc<int>(ctx, 4 * sizeof(int));
    launch_band_extent(ctx->A, ctx->hasB ? &ctx->B : nullptr, ctx->d_ext, ctx->s);
    int ext[3] = {0, 0, 0};
    CKC(cudaMemcpyAsync(ext, ctx->d_ext, 3 * sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
    CKC(cudaStreamSynchronize(ctx->s));
    REQ(ext[2] == 0, "a column index of A or B is outside [0, n)");
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
    const bool fits = krylov(ctx) || (f32 ? (band_fits<float>(ctx->klp, ctx->kup) &&
                             (band_tma_fits(ctx->klp, ctx->kup) || band_solve_fits<float>(ctx->klp, ctx->kup)))
                          : (band_fits<double>(ctx->klp, ctx->kup) && band_solve_fits<double>(ctx->klp, ctx->kup)));
    if (!fits) {
      char msg[160];
      std::snprintf(msg, sizeof msg, "band (kl=%d, ku=%d) too wide for the banded inner solver", ctx->kl, ctx->ku);
      REQ(false, msg);
    }
    const size_t es = f32 ? sizeof(cxf) : sizeof(cxd);
    const size_t band_elems = krylov(ctx) ? 0 : (size_t)ctx->nf * n * (ctx->klp + ctx->kup + 1);
    ctx->band = dalloc<void>(ctx, band_elems * es);
    if (krylov(ctx)) ctx->kwork = dalloc<void>(ctx, krylov_work_bytes(n, m0, ne));
    if (f32 && !krylov(ctx) && band_tma_fits(ctx->klp, ctx->kup)) {
      ctx->bandT = dalloc<void>(ctx, band_elems * es);
      ctx->tma.assign(band_tma_bytes(), 0);
      if (!band_tma_make(ctx->tma.data(), n, ctx->klp, ctx->kup, ctx->nf, (const cxf *)ctx->band,
                         (const cxf *)ctx->bandT))
        ctx->tma.clear();
    }
    const size_t yse = krylov(ctx) ? 0
                       : f32   ? band_solve_scratch_elems<float>(n, m0, ne)
                               : band_solve_scratch_elems<double>(n, m0, ne);
    ctx->ysc = dalloc<void>(ctx, yse * es);
    if (f32 && !krylov(ctx)) ctx->dinv = dalloc<void>(ctx, band_diag_inv_elems(n, ctx->nf) * sizeof(cxf));
    const size_t blk = (size_t)n * m0 * sizeof(cxd);
    ctx->Yw = dalloc<cxd>(ctx, blk);
    ctx->Yhw = dalloc<cxd>(ctx, blk);
    ctx->Qw = dalloc<cxd>(ctx, blk);
    ctx->Qhw = dalloc<cxd>(ctx, blk);
    ctx->Uw = dalloc<cxd>(ctx, blk);
    ctx->Uhw = dalloc<cxd>(ctx, blk);
    ctx->T1 = dalloc<cxd>(ctx, blk);
    ctx->T2 = dalloc<cxd>(ctx, blk);
    if (ctx->hasB) {
      ctx->BYw = dalloc<cxd>(ctx, blk);
      ctx->BhYw = dalloc<cxd>(ctx, blk);
    }
    ctx->Xn = dalloc<cxd>(ctx, blk * ne);
    ctx->Xhn = dalloc<cxd>(ctx, blk * ne);
    if (f32) {
      ctx->Rn = dalloc<void>(ctx, (size_t)n * m0 * ne * sizeof(cxf));
      ctx->Rhn = dalloc<void>(ctx, (size_t)n * m0 * ne * sizeof(cxf));
    }
    ctx->gmax = spmm_max_grid();
    ctx->part = dalloc<double>(ctx, (size_t)2 * ctx->gmax * 2048 * sizeof(double));
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
    ctx->gpart = dalloc<cxd>(ctx, (size_t)ctx->gchunks * sm);
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
  } catch (const Fail &f) {
    std::string msg = ctx->err;
    feast_nh_destroy(ctx);
    (void)msg;
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
      info->n_factorizations = krylov(ctx) ? 0 : ctx->nf;
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
      // systems need only the accuracy of the single-precision factors (a
      // relative residual of 1e-2 stops the refinement), later iterations
      // are refined to opts.inner_tol.
      const double tol_it = it == 1 ? std::fmax(ctx->o.inner_tol, 1e-2) : ctx->o.inner_tol;
      do_filter(ctx, ctx->Yw, ctx->Yhw, ctx->Qw, ctx->Qhw, m, tol_it);
      CKC(cudaEventRecord(ctx->ev[2], s));
      mt = do_rr(ctx, ctx->Qw, ctx->Qhw, m, ctx->Yw, ctx->Yhw);
      CKC(cudaEventRecord(ctx->ev[3], s));
      read_status(ctx);
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
    // 5.d  converged pairs first, normalised (||x|| = 1, max entry real > 0, x^^H B x = 1)
    const cxd *BYf = ctx->Yw;
    if (ctx->hasB) {
      launch_spmm(ctx->B, nullptr, nullptr, ctx->Yw, ctx->T1, mt, nullptr, nullptr, s);
      BYf = ctx->T1;
    }
    const int gp = launch_colstats(ctx->Yw, ctx->Yhw, BYf, mt, n, ctx->pn, ctx->pmax, ctx->pidx, ctx->pval,
                                   ctx->pdot, s);
    launch_finalize(mt, gp, ctx->pn, ctx->pmax, ctx->pidx, ctx->pval, ctx->pdot, ctx->sx, ctx->sxh, ctx->Yw,
                    ctx->Yhw, n, ctx->ord, mout, (cxd *)X, (cxd *)Xh, m0, ctx->lam, ctx->res, lambda, res, s);
    check_launch(ctx, "output");
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
      info->n_factorizations = krylov(ctx) ? 0 : ctx->nf;
      info->inner_fail = ctx->n_inner_fail;
      info->pivot_min = ctx->piv_min;
      info->pivot_max = ctx->piv_max;
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
