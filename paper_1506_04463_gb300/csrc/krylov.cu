// Batched BiCGStab for the shifted systems of the contour integration:
// (z_j B - A) X_j = B Y for every node j and column c at once (eq. qr), and
// the conjugate-transpose systems of eq. (ql) through the transposed CSR with
// conjugated nodes.  Every (node, column) pair is an independent system with
// its own scalars; converged columns are frozen.  The operator is the fused
// multi-shift product of spmm.cu: with no right-hand side it returns
// -(z_j B - A) P_j, so the recurrences below carry that sign.
//
// State blocks (node-major ne x n x m, complex128): X, R, Rh (shadow), P, V, S, T.
#include <vector>

#include "kernels.h"

namespace {
constexpr int kDotThreads = 256;
constexpr int kDotMaxPairs = 8;  // ne*m <= 2048
}  // namespace

// Per-CTA partial column dots of up to three pairs (a_k, b_k):
// part[k][cta][pair] = sum_i conj(a_k[i]) b_k[i] over the CTA's rows.
struct DotArgs {
  const cxd *a[3];
  const cxd *b[3];
  int nd;
};
__global__ void __launch_bounds__(kDotThreads) k_coldots(DotArgs d, int n, int P, int m, size_t xns, int rows_per_cta,
                                                         cxd *part) {
  const int tid = threadIdx.x;
  const int rbeg = blockIdx.x * rows_per_cta, rend = min(n, rbeg + rows_per_cta);
  cxd acc[3][kDotMaxPairs];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int q = 0; q < kDotMaxPairs; ++q) acc[k][q] = mk(0.0, 0.0);
  for (int i = rbeg; i < rend; ++i) {
#pragma unroll
    for (int q = 0; q < kDotMaxPairs; ++q) {
      const int pair = tid + kDotThreads * q;
      if (pair < P) {
        const int j = pair / m, c = pair - j * m;
        const size_t o = (size_t)j * xns + (size_t)i * m + c;
#pragma unroll
        for (int k = 0; k < 3; ++k)
          if (k < d.nd) cfma_cj(acc[k][q], d.a[k][o], d.b[k][o]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (k >= d.nd) break;
#pragma unroll
    for (int q = 0; q < kDotMaxPairs; ++q) {
      const int pair = tid + kDotThreads * q;
      if (pair < P) part[((size_t)k * gridDim.x + blockIdx.x) * P + pair] = acc[k][q];
    }
  }
}

// Sum the partials (fixed order) into out[k][pair].
__global__ void k_dots_reduce(const cxd *part, int nparts, int P, int nd, cxd *out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nd * P) return;
  const int k = e / P, pair = e - k * P;
  cxd s = mk(0.0, 0.0);
  for (int p = 0; p < nparts; ++p) s = s + part[((size_t)k * nparts + p) * P + pair];
  out[e] = s;
}

// Scalar updates.  Notation: the operator output holds V' = -M P, T' = -M S.
struct KScal {
  cxd *rho, *alpha, *omega, *beta;
  double *bn2;     // ||b||^2 per column
  double *relres;  // ||r|| / ||b|| per column
  int *active;     // 1 while the column iterates
};

// after <rh, V'>: alpha = rho / <rh, M p> = -rho / <rh, V'>
__global__ void k_scal_alpha(int P, KScal s, const cxd *d_rhv) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P || !s.active[c]) return;
  const cxd den = -d_rhv[c];
  s.alpha[c] = abs2(den) > 0 ? cdiv(s.rho[c], den) : mk(0.0, 0.0);
  if (!(abs2(den) > 0)) s.active[c] = 0;  // breakdown: keep the current iterate
}
// after <T', S>, <T', T'>: omega = <t, s>/<t, t> = -<T', S>/<T', T'>
__global__ void k_scal_omega(int P, KScal s, const cxd *d_ts, const cxd *d_tt) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P || !s.active[c]) return;
  const double tt = d_tt[c].re;
  s.omega[c] = tt > 0 ? (-1.0 / tt) * d_ts[c] : mk(0.0, 0.0);
}
// after <rh, r>, <r, r>: beta for the next p, convergence test, done flag
__global__ void k_scal_next(int P, KScal s, const cxd *d_rhr, const cxd *d_rr, double tol, int *d_nactive) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < P) {
    const double rel = sqrt(d_rr[c].re / (s.bn2[c] > 0 ? s.bn2[c] : 1.0));
    s.relres[c] = rel;
    if (s.active[c]) {
      if (!(rel > tol) || !(rel == rel)) {
        s.active[c] = 0;
      } else {
        const cxd rho_new = d_rhr[c];
        const cxd om = s.omega[c];
        if (abs2(om) > 0 && abs2(s.rho[c]) > 0)
          s.beta[c] = cdiv(rho_new, s.rho[c]) * cdiv(s.alpha[c], om);
        else
          s.active[c] = 0;
        s.rho[c] = rho_new;
      }
    }
    if (s.active[c]) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0 && cnt) atomicAdd(d_nactive, cnt);
}

// p = r + beta (p + omega V')   (p - omega v with v = -V')
__global__ void k_upd_p(size_t count, int P, int m, size_t xns, KScal s, const cxd *R, const cxd *V, cxd *Pv) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const size_t j = e / xns, rem = e - j * xns;
    const int c = (int)(j * m + rem % m);
    if (!s.active[c]) continue;
    cxd t = Pv[e];
    cfma(t, s.omega[c], V[e]);
    cxd out = R[e];
    cfma(out, s.beta[c], t);
    Pv[e] = out;
  }
}
// s = r - alpha v = r + alpha V'
__global__ void k_upd_s(size_t count, int m, size_t xns, KScal s, const cxd *R, const cxd *V, cxd *S) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const size_t j = e / xns, rem = e - j * xns;
    const int c = (int)(j * m + rem % m);
    if (!s.active[c]) continue;
    cxd out = R[e];
    cfma(out, s.alpha[c], V[e]);
    S[e] = out;
  }
}
// x += alpha p + omega s; r = s - omega t = s + omega T'
__global__ void k_upd_xr(size_t count, int m, size_t xns, KScal s, const cxd *Pv, const cxd *S, const cxd *T, cxd *X,
                         cxd *R) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const size_t j = e / xns, rem = e - j * xns;
    const int c = (int)(j * m + rem % m);
    if (!s.active[c]) continue;
    cxd x = X[e];
    cfma(x, s.alpha[c], Pv[e]);
    cfma(x, s.omega[c], S[e]);
    X[e] = x;
    cxd r = S[e];
    cfma(r, s.omega[c], T[e]);
    R[e] = r;
  }
}
// initial state: X = 0, R = Rh = P = BY (broadcast to every node), V = 0;
// rho = alpha = omega = 1, active = 1
__global__ void k_krylov_init(size_t count, int m, size_t xns, const cxd *BY, cxd *X, cxd *R, cxd *Rh, cxd *Pv,
                              cxd *V) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const size_t rem = e % xns;
    const cxd b = BY[rem];
    X[e] = mk(0.0, 0.0);
    R[e] = b;
    Rh[e] = b;
    Pv[e] = mk(0.0, 0.0);
    V[e] = mk(0.0, 0.0);
  }
}
__global__ void k_scal_rho0(int P, KScal s, const cxd *d_rhr) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < P) s.rho[c] = d_rhr[c];
}
__global__ void k_krylov_scal_init(int P, int m, KScal s, const double *bn2_cols) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P) return;
  s.rho[c] = mk(1.0, 0.0);
  s.alpha[c] = mk(1.0, 0.0);
  s.omega[c] = mk(1.0, 0.0);
  s.beta[c] = mk(0.0, 0.0);
  s.bn2[c] = bn2_cols[c % m];
  s.relres[c] = 1.0;
  s.active[c] = s.bn2[c] > 0;
}

// ----------------------------------------------------------------------------
struct KrylovWork {
  cxd *X, *R, *Rh, *P, *V, *S, *T;
  cxd *part;      // 3 x grid x P partial dots
  cxd *dots;      // 3 x P
  KScal sc;
  int *nactive;   // device counter
  double *colp;   // column-norm partials of BY
};

static int dots_grid(int n) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int g = sms * 4;
  return g > n ? (n < 1 ? 1 : n) : g;
}

static void coldots(const DotArgs &d, int n, int P, int m, size_t xns, cxd *part, cxd *out, cudaStream_t s) {
  const int g0 = dots_grid(n);
  const int rpc = ceil_div(n, g0), g = ceil_div(n, rpc);
  k_coldots<<<g, kDotThreads, 0, s>>>(d, n, P, m, xns, rpc, part);
  note_launch();
  k_dots_reduce<<<ceil_div(d.nd * P, 256), 256, 0, s>>>(part, g, P, d.nd, out);
  note_launch();
}

size_t krylov_work_bytes(int n, int m0, int ne) {
  const size_t blk = (size_t)ne * n * m0 * sizeof(cxd);
  const int P = ne * m0;
  return 7 * blk + (size_t)3 * dots_grid(n) * P * sizeof(cxd) + (size_t)3 * P * sizeof(cxd) +
         (size_t)4 * P * sizeof(cxd) + (size_t)2 * P * sizeof(double) + P * sizeof(int) + 64 +
         (size_t)608 * kMaxM0 * sizeof(double) + kMaxM0 * sizeof(double);
}

// Carve the workspace.  Returns the end pointer.
static unsigned char *krylov_carve(unsigned char *w, int n, int m0, int ne, KrylovWork &k, double **bycol) {
  const size_t blk = (size_t)ne * n * m0;
  const int P = ne * m0;
  auto take = [&](size_t bytes) {
    unsigned char *p = w;
    w += (bytes + 255) & ~(size_t)255;
    return p;
  };
  k.X = (cxd *)take(blk * sizeof(cxd));
  k.R = (cxd *)take(blk * sizeof(cxd));
  k.Rh = (cxd *)take(blk * sizeof(cxd));
  k.P = (cxd *)take(blk * sizeof(cxd));
  k.V = (cxd *)take(blk * sizeof(cxd));
  k.S = (cxd *)take(blk * sizeof(cxd));
  k.T = (cxd *)take(blk * sizeof(cxd));
  k.part = (cxd *)take((size_t)3 * dots_grid(n) * P * sizeof(cxd));
  k.dots = (cxd *)take((size_t)3 * P * sizeof(cxd));
  k.sc.rho = (cxd *)take(P * sizeof(cxd));
  k.sc.alpha = (cxd *)take(P * sizeof(cxd));
  k.sc.omega = (cxd *)take(P * sizeof(cxd));
  k.sc.beta = (cxd *)take(P * sizeof(cxd));
  k.sc.bn2 = (double *)take(P * sizeof(double));
  k.sc.relres = (double *)take(P * sizeof(double));
  k.sc.active = (int *)take(P * sizeof(int));
  k.nactive = (int *)take(64);
  k.colp = (double *)take((size_t)608 * kMaxM0 * sizeof(double));
  *bycol = (double *)take(kMaxM0 * sizeof(double));
  return w;
}

// Solve (z_j B - A) X_j = BY for all nodes (M given as the CSR pair and node
// shifts), X_j in Xout (node-major).  Checks convergence every `check`
// iterations (a 4-byte read).  Returns the iterations done; *maxrel gets the
// largest relative residual.
int krylov_bicgstab(const CsrView &A, const CsrView *B, int ne, const cxd *d_z, const cxd *d_w, const cxd *BY, int m,
                    int m0, double tol, int max_it, void *work, cxd *Xout, double *maxrel, cudaStream_t s) {
  const int n = A.n, P = ne * m;
  const size_t xns = (size_t)n * m;
  const size_t count = (size_t)ne * xns;
  KrylovWork k;
  double *bycol = nullptr;
  krylov_carve(reinterpret_cast<unsigned char *>(work), n, m0, ne, k, &bycol);
  k.X = Xout;  // the solution goes straight to the caller's node blocks
  const unsigned g = grid_for(count);
  // ||BY_c||^2
  {
    const int gc = launch_colnorm2(BY, m, m, n, k.colp, s);
    launch_reduce_parts(k.colp, gc, m, bycol, s);
  }
  k_krylov_init<<<g, 256, 0, s>>>(count, m, xns, BY, k.X, k.R, k.Rh, k.P, k.V);
  note_launch();
  k_krylov_scal_init<<<ceil_div(P, 256), 256, 0, s>>>(P, m, k.sc, bycol);
  note_launch();
  // rho_0 = <rh, r> = <b, b>
  {
    DotArgs d{};
    d.a[0] = k.Rh;
    d.b[0] = k.R;
    d.nd = 1;
    coldots(d, n, P, m, xns, k.part, k.dots, s);
    k_scal_rho0<<<ceil_div(P, 256), 256, 0, s>>>(P, k.sc, k.dots);
    note_launch();
    // first p = r: beta = 0 with p = v = 0
  }
  int it = 0;
  int h_active = P;
  const int check = 8;
  for (it = 0; it < max_it && h_active > 0; ++it) {
    k_upd_p<<<g, 256, 0, s>>>(count, P, m, xns, k.sc, k.R, k.V, k.P);
    note_launch();
    // V' = -(z B - A) P
    launch_multishift_residual<double>(A, B, ne, d_z, d_w, k.P, nullptr, k.V, nullptr, nullptr, m, nullptr, s);
    {
      DotArgs d{};
      d.a[0] = k.Rh;
      d.b[0] = k.V;
      d.nd = 1;
      coldots(d, n, P, m, xns, k.part, k.dots, s);
      k_scal_alpha<<<ceil_div(P, 256), 256, 0, s>>>(P, k.sc, k.dots);
      note_launch();
    }
    k_upd_s<<<g, 256, 0, s>>>(count, m, xns, k.sc, k.R, k.V, k.S);
    note_launch();
    launch_multishift_residual<double>(A, B, ne, d_z, d_w, k.S, nullptr, k.T, nullptr, nullptr, m, nullptr, s);
    {
      DotArgs d{};
      d.a[0] = k.T;
      d.b[0] = k.S;
      d.a[1] = k.T;
      d.b[1] = k.T;
      d.nd = 2;
      coldots(d, n, P, m, xns, k.part, k.dots, s);
      k_scal_omega<<<ceil_div(P, 256), 256, 0, s>>>(P, k.sc, k.dots, k.dots + P);
      note_launch();
    }
    k_upd_xr<<<g, 256, 0, s>>>(count, m, xns, k.sc, k.P, k.S, k.T, k.X, k.R);
    note_launch();
    {
      DotArgs d{};
      d.a[0] = k.Rh;
      d.b[0] = k.R;
      d.a[1] = k.R;
      d.b[1] = k.R;
      d.nd = 2;
      coldots(d, n, P, m, xns, k.part, k.dots, s);
      cudaMemsetAsync(k.nactive, 0, sizeof(int), s);
      k_scal_next<<<ceil_div(P, 256), 256, 0, s>>>(P, k.sc, k.dots, k.dots + P, tol, k.nactive);
      note_launch();
    }
    if ((it + 1) % check == 0 || it + 1 == max_it) {
      cudaMemcpyAsync(&h_active, k.nactive, sizeof(int), cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
    }
  }
  // largest relative residual over the columns
  {
    std::vector<double> rel(P);
    cudaMemcpyAsync(rel.data(), k.sc.relres, P * sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    double mx = 0;
    for (double v : rel) mx = (v > mx || !(v == v)) ? v : mx;
    *maxrel = mx;
  }
  return it;
}
