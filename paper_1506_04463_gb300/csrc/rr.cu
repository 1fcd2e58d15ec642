// Control kernels of the Rayleigh-Ritz step and of the convergence test
// (Fig. alg:three steps 2.b, 3.b-3.d, 4.b-4.c, 5).  All run as one CTA on
// the m <= 128 reduced quantities; the n-sized work is in dense.cu / spmm.cu.
#include <float.h>
#include "rr.cuh"

// Steps 2.b and 3.b-3.c: spurious count against the previous Ritz values,
// stable sort of gamma by decreasing modulus, resize (eq. resize) and the
// bi-orthonormalising coefficients of eq. (uu):
//   S  = V[:, ord] Gamma^{-1/2},   Sh = Vh[:, ord] Gamma^{-H/2},  Vh = V^{-H}.
// Complex symmetric: V scaled to v^T v = 1 and Vh = conj(V) (Sec. 2.4).
__global__ void k_gamma_prep(int m, const cxd *BQ, const cxd *gam, const cxd *V, const cxd *Vinv,
                             const cxd *prev_rho, const int *prev_inside, int have_prev, double mu, double eta,
                             int cs, cxd *S, cxd *Sh, int *ord, RRStatus *st) {
  __shared__ int o[kMaxM0];
  __shared__ cxd g[kMaxM0];
  __shared__ cxd tcs[kMaxM0];
  __shared__ int mt_s;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) {
    int ms = 0;
    if (have_prev) {
      for (int i = 0; i < m; ++i) {
        if (!prev_inside[i]) continue;
        const cxd r2 = prev_rho[i] * prev_rho[i];
        const cxd d = BQ[(size_t)i * m + i];
        const double den = cabs(r2);
        const double q = den > 0 ? cabs(r2 - d) / den : INFINITY;
        if (!(q < mu)) ++ms;
      }
    }
    st->m_s = ms;
    for (int i = 0; i < m; ++i) o[i] = i;
    for (int i = 1; i < m; ++i) {  // stable insertion sort, |gamma| descending
      int key = o[i];
      double kv = cabs(gam[key]);
      int j = i - 1;
      while (j >= 0 && cabs(gam[o[j]]) < kv) {
        o[j + 1] = o[j];
        --j;
      }
      o[j + 1] = key;
    }
    const double gmax = cabs(gam[o[0]]);
    int mt = 0;
    while (mt < m && cabs(gam[o[mt]]) >= eta * gmax && gmax > 0) ++mt;
    mt_s = mt;
    st->m_tilde = mt;
  }
  __syncthreads();
  const int mt = mt_s;
  for (int b = tid; b < m; b += nt) {
    ord[b] = o[b];
    const cxd sq = csqrt(gam[o[b]]);
    g[b] = cdiv(mk(1.0, 0.0), sq);
    if (cs) {
      cxd t = mk(0.0, 0.0);
      for (int a = 0; a < m; ++a) cfma(t, V[(size_t)a * m + o[b]], V[(size_t)a * m + o[b]]);
      tcs[b] = csqrt(t);
    }
  }
  __syncthreads();
  for (int e = tid; e < m * m; e += nt) {
    const int a = e / m, b = e - a * m;
    if (b >= mt) {
      S[e] = mk(0.0, 0.0);
      Sh[e] = mk(0.0, 0.0);
      continue;
    }
    const int src = o[b];
    cxd v = V[(size_t)a * m + src];
    if (cs) {
      v = cdiv(v, tcs[b]);
      S[e] = v * g[b];
      Sh[e] = conj(v) * conj(g[b]);
    } else {
      S[e] = v * g[b];
      Sh[e] = conj(Vinv[(size_t)src * m + a]) * conj(g[b]);
    }
  }
}

// Complex symmetric reduced problem: scale W so that w^T B_U w = 1, Wh = conj(W).
__global__ void k_cs_wnorm(int m, const cxd *BU, cxd *W, cxd *Wh) {
  __shared__ cxd t[kMaxM0];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = tid; k < m; k += nt) {
    cxd s = mk(0.0, 0.0);
    for (int a = 0; a < m; ++a) {
      cxd bw = mk(0.0, 0.0);
      for (int b = 0; b < m; ++b) cfma(bw, BU[(size_t)a * m + b], W[(size_t)b * m + k]);
      cfma(s, W[(size_t)a * m + k], bw);
    }
    t[k] = csqrt(s);
  }
  __syncthreads();
  for (int e = tid; e < m * m; e += nt) {
    const int k = e % m;
    cxd v = cdiv(W[e], t[k]);
    W[e] = v;
    Wh[e] = conj(v);
  }
}

// Step 4.c: rho_a(lambda_i) = sum_j w_j / (z_j - lambda_i)   (eq. rational).
__global__ void k_rho(int m, int ne, const cxd *z, const cxd *w, const cxd *lam, cxd *rho) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    cxd s = mk(0.0, 0.0);
    for (int j = 0; j < ne; ++j) s = s + cdiv(w[j], z[j] - lam[i]);
    rho[i] = s;
  }
}

// Y[:, i] /= ||y_i||, Yh[:, i] *= ||y_i|| (column scale of the Ritz vectors).
__global__ void k_scale_pairs(cxd *Y, cxd *Yh, const double *nrm2, int m, size_t count) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % m);
    const double s = sqrt(nrm2[c]);
    if (s > 0) {
      Y[e] = (1.0 / s) * Y[e];
      Yh[e] = s * Yh[e];
    }
  }
}

__device__ __forceinline__ bool inside_contour(cxd l, const RRParams &p) {
  if (!(isfinite(l.re) && isfinite(l.im))) return false;
  if (p.kind == 2) {
    bool in = false;
    for (int k = 0; k < p.ne; ++k) {
      const cxd a = p.cz[k], b = p.cz[(k + 1) % p.ne];
      if ((a.im > l.im) != (b.im > l.im)) {
        double xc = a.re + (l.im - a.im) * (b.re - a.re) / (b.im - a.im);
        if (l.re < xc) in = !in;
      }
    }
    return in;
  }
  const double ca = cos(p.angle), sa = sin(p.angle);
  const double dx = l.re - p.c_re, dy = l.im - p.c_im;
  const double u = ca * dx + sa * dy, v = -sa * dx + ca * dy;
  const double a = p.r, b = p.r * (p.kind == 0 ? 1.0 : p.ratio);
  return (u / a) * (u / a) + (v / b) * (v / b) <= 1.0;
}

// Step 5: inside count m_r, residuals of eq. (res), m = m_r - m_s, converged
// pairs ordered by increasing residual; saves rho and the inside flags for the
// spurious test of the next iteration.
__global__ void k_converge(RRParams p, int mt, const cxd *lam, const cxd *rho, const double *cn, double *res,
                           int *ord, cxd *prev_rho, int *prev_inside, RRStatus *st) {
  __shared__ int ins[kMaxM0];
  __shared__ double rs[kMaxM0];
  const int tid = threadIdx.x;
  for (int i = tid; i < mt; i += blockDim.x) {
    const bool in = inside_contour(lam[i], p);
    ins[i] = in;
    double r = INFINITY;
    if (in) {
      const double r1 = cn[i] / (p.alpha * cn[kMaxM0 + i]);
      const double r2 = cn[2 * kMaxM0 + i] / (p.alpha * cn[3 * kMaxM0 + i]);
      r = fmax(r1, r2);
      if (!(r == r)) r = INFINITY;
    }
    rs[i] = r;
    res[i] = r;
    prev_rho[i] = rho[i];
    prev_inside[i] = in;
  }
  __syncthreads();
  if (tid == 0) {
    int mr = 0;
    for (int i = 0; i < mt; ++i) mr += ins[i];
    int k = 0;
    for (int i = 0; i < mt; ++i)
      if (ins[i]) ord[k++] = i;
    for (int i = 1; i < k; ++i) {  // stable insertion sort by residual
      int key = ord[i];
      int j = i - 1;
      while (j >= 0 && rs[ord[j]] > rs[key]) {
        ord[j + 1] = ord[j];
        --j;
      }
      ord[j + 1] = key;
    }
    for (int i = 0; i < mt; ++i)
      if (!ins[i]) ord[k++] = i;
    const int m = mr - st->m_s;
    double mx = 0.0;
    bool conv = m >= 1;
    for (int i = 0; i < m && i < mr; ++i) {
      mx = fmax(mx, rs[ord[i]]);
      if (!(rs[ord[i]] < p.eps)) conv = false;
    }
    // 5.d: on convergence every inside pair below eps is returned (at least m)
    int mout = m > 0 ? m : 0;
    if (conv) {
      mout = 0;
      while (mout < mr && rs[ord[mout]] < p.eps) ++mout;
    }
    st->m_r = mr;
    st->m = mout;
    st->conv = conv ? 1 : 0;
    st->max_res = m >= 1 ? mx : INFINITY;
  }
}

// Column statistics for the output normalisation: ||y||^2, the entry of
// largest modulus (first index on ties) and y^^H (B y).
__global__ void k_colstats(const cxd *Y, const cxd *Yh, const cxd *BY, int m, int n, int rows_per_cta,
                           double *pn, double *pmax, int *pidx, cxd *pval, cxd *pdot) {
  const int c = threadIdx.x;
  if (c >= m) return;
  const int rbeg = blockIdx.x * rows_per_cta, rend = min(n, rbeg + rows_per_cta);
  double s = 0.0, best = -1.0;
  int bi = 0;
  cxd bv = mk(0.0, 0.0), d = mk(0.0, 0.0);
  for (int i = rbeg; i < rend; ++i) {
    const cxd y = Y[(size_t)i * m + c];
    const double a2 = abs2(y);
    s += a2;
    if (a2 > best) {
      best = a2;
      bi = i;
      bv = y;
    }
    cfma_cj(d, Yh[(size_t)i * m + c], BY[(size_t)i * m + c]);
  }
  const size_t o = (size_t)blockIdx.x * m + c;
  pn[o] = s;
  pmax[o] = best;
  pidx[o] = bi;
  pval[o] = bv;
  pdot[o] = d;
}

__global__ void k_finalize_coeffs(int m, int nparts, const double *pn, const double *pmax, const int *pidx,
                                  const cxd *pval, const cxd *pdot, cxd *sx, cxd *sxh) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m) return;
  double s = 0.0, best = -1.0;
  int bi = 0x7fffffff;
  cxd bv = mk(1.0, 0.0), d = mk(0.0, 0.0);
  for (int p = 0; p < nparts; ++p) {
    const size_t o = (size_t)p * m + c;
    s += pn[o];
    if (pmax[o] > best || (pmax[o] == best && pidx[o] < bi)) {
      best = pmax[o];
      bi = pidx[o];
      bv = pval[o];
    }
    d = d + pdot[o];
  }
  const double nrm = sqrt(s);
  const double av = cabs(bv);
  cxd ph = av > 0 ? mk(bv.re / av, -bv.im / av) : mk(1.0, 0.0);  // conj(phase)
  const cxd scale = (nrm > 0 ? 1.0 / nrm : 1.0) * ph;
  const cxd t = scale * d;  // x^^H B x after scaling x
  sx[c] = scale;
  sxh[c] = cdiv(mk(1.0, 0.0), conj(t));
}

// X[:, k] = sx[src] Y[:, src], Xh[:, k] = sxh[src] Yh[:, src], src = ord[k].
__global__ void k_gather_out(const cxd *Y, const cxd *Yh, int m, int n, const int *ord, int mout, const cxd *sx,
                             const cxd *sxh, cxd *X, cxd *Xh, int ldo) {
  const size_t count = (size_t)n * mout;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / mout;
    const int k = (int)(e - i * mout);
    const int src = ord[k];
    X[i * ldo + k] = sx[src] * Y[i * m + src];
    Xh[i * ldo + k] = sxh[src] * Yh[i * m + src];
  }
}
__global__ void k_gather_small(const cxd *lam, const double *res, const int *ord, int mout, double *lam_out,
                               double *res_out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= mout) return;
  lam_out[2 * k] = lam[ord[k]].re;
  lam_out[2 * k + 1] = lam[ord[k]].im;
  if (res_out) res_out[k] = res[ord[k]];
}

// ---------------------------------------------------------------------------
void launch_gamma_prep(int m, const cxd *BQ, const cxd *gam, const cxd *V, const cxd *Vinv, const cxd *prev_rho,
                       const int *prev_inside, int have_prev, double mu, double eta, int cs, cxd *S, cxd *Sh,
                       int *ord, RRStatus *st, cudaStream_t s) {
  k_gamma_prep<<<1, 256, 0, s>>>(m, BQ, gam, V, Vinv, prev_rho, prev_inside, have_prev, mu, eta, cs, S, Sh, ord,
                                 st);
  note_launch();
}
void launch_cs_wnorm(int m, const cxd *BU, cxd *W, cxd *Wh, cudaStream_t s) {
  k_cs_wnorm<<<1, 128, 0, s>>>(m, BU, W, Wh);
  note_launch();
}
void launch_rho(int m, int ne, const cxd *z, const cxd *w, const cxd *lam, cxd *rho, cudaStream_t s) {
  k_rho<<<1, 128, 0, s>>>(m, ne, z, w, lam, rho);
  note_launch();
}
void launch_scale_pairs(cxd *Y, cxd *Yh, const double *nrm2, int m, int n, cudaStream_t s) {
  size_t count = (size_t)n * m;
  k_scale_pairs<<<grid_for(count), 256, 0, s>>>(Y, Yh, nrm2, m, count);
  note_launch();
}
void launch_converge(const RRParams &p, int mt, const cxd *lam, const cxd *rho, const double *cn, double *res,
                     int *ord, cxd *prev_rho, int *prev_inside, RRStatus *st, cudaStream_t s) {
  k_converge<<<1, 128, 0, s>>>(p, mt, lam, rho, cn, res, ord, prev_rho, prev_inside, st);
  note_launch();
}
int launch_colstats(const cxd *Y, const cxd *Yh, const cxd *BY, int m, int n, double *pn, double *pmax, int *pidx,
                    cxd *pval, cxd *pdot, cudaStream_t s) {
  int g = min(304, ceil_div(n, 64));
  int rpc = ceil_div(n, g);
  g = ceil_div(n, rpc);
  k_colstats<<<g, 128, 0, s>>>(Y, Yh, BY, m, n, rpc, pn, pmax, pidx, pval, pdot);
  note_launch();
  return g;
}
void launch_finalize(int m, int nparts, const double *pn, const double *pmax, const int *pidx, const cxd *pval,
                     const cxd *pdot, cxd *sx, cxd *sxh, const cxd *Y, const cxd *Yh, int n, const int *ord, int mout,
                     cxd *X, cxd *Xh, int ldo, const cxd *lam, const double *res, double *lam_out, double *res_out,
                     cudaStream_t s) {
  k_finalize_coeffs<<<1, 128, 0, s>>>(m, nparts, pn, pmax, pidx, pval, pdot, sx, sxh);
  note_launch();
  size_t count = (size_t)n * mout;
  if (count) {
    k_gather_out<<<grid_for(count), 256, 0, s>>>(Y, Yh, m, n, ord, mout, sx, sxh, X,
                                                                                 Xh, ldo);
    note_launch();
  }
  if (mout) {
    k_gather_small<<<1, 128, 0, s>>>(lam, res, ord, mout, lam_out, res_out);
    note_launch();
  }
}
