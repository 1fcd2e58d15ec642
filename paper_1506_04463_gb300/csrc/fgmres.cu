// Batched flexible GMRES (restarted, FGMRES(k)) for the shifted systems of
// the contour integration, (z_j B - A) d_jc = r_jc for every node j and
// column c at once, in complex FP32, with a right preconditioner that may
// change from step to step (the learned network is not a fixed linear map,
// so the flexible form keeps the preconditioned directions Z).
//
// Every (node, column) system has its own Arnoldi basis, Hessenberg matrix
// and Givens rotations; the block kernels below run all systems in one pass:
// node-major blocks ne x n x m (row-major n x m per node, complex float),
// system s = j*m + c.  Orthogonalisation is classical Gram-Schmidt applied
// twice (one pass for the dot products of all previous basis vectors, one
// for the update, repeated).  Scalars and the small least-squares problems
// are FP64.  Converged systems are frozen (their columns are skipped).
#include <vector>

#include "kernels.h"

namespace {
constexpr int kFgMaxK = 64;
constexpr int kFgThreads = 256;
}  // namespace

// partial[chunk][l][s] = sum over the chunk's rows of conj(V_l) * w  (l < nv)
__global__ void __launch_bounds__(kFgThreads) k_fg_dots(const cxf *const *V, int nv, const cxf *w, int ne, int n,
                                                        int m, int rows_per_cta, const int *active, cxd *partial) {
  const int S = ne * m;
  const int r0 = blockIdx.x * rows_per_cta, r1 = min(n, r0 + rows_per_cta);
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    if (!active[s]) continue;
    const int j = s / m, c = s - j * m;
    const size_t base = (size_t)j * n * m + c;
    for (int l = 0; l < nv; ++l) {
      const cxf *Vl = V[l];
      cxf acc = mk(0.f, 0.f);
      for (int i = r0; i < r1; ++i) cfma_cj(acc, Vl[base + (size_t)i * m], w[base + (size_t)i * m]);
      partial[((size_t)blockIdx.x * nv + l) * S + s] = ccast<double>(acc);
    }
  }
}
// out[l][s] = sum_chunks partial (fixed order); also optionally |w|^2 sums
__global__ void k_fg_dots_reduce(const cxd *partial, int nchunks, int nv, int S, cxd *out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nv * S) return;
  cxd acc = mk(0.0, 0.0);
  for (int p = 0; p < nchunks; ++p) acc = acc + partial[(size_t)p * nv * S + e];
  out[e] = acc;
}
// w -= sum_l h[l][s] V_l ; H[s][l][col] += h[l][s] (the Gram-Schmidt coefficients)
__global__ void k_fg_orth_update(const cxf *const *V, int nv, const cxd *h, cxf *w, int ne, int n, int m,
                                 const int *active, cxd *H, int kmax, int col) {
  const int S = ne * m;
  const size_t count = (size_t)ne * n * m;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const size_t j = e / ((size_t)n * m), rem = e - j * n * m;
    const int c = (int)(rem % m);
    const int s = (int)j * m + c;
    if (!active[s]) continue;
    cxf acc = w[e];
    for (int l = 0; l < nv; ++l) cfms(acc, ccast<float>(h[(size_t)l * S + s]), V[l][e]);
    w[e] = acc;
  }
  if (blockIdx.x == 0)
    for (int q = threadIdx.x; q < nv * S; q += blockDim.x) {
      const int l = q / S, s = q - l * S;
      if (active[s]) {
        cxd &hv = H[((size_t)s * (kmax + 1) + l) * kmax + col];
        hv = hv + h[q];
      }
    }
}
// per system: h_{col+1,col} = ||w|| (from the reduced |w|^2), v_{col+1} = w / h;
// Givens rotations on column col, residual estimate, convergence
struct FgScal {
  cxd *H;        // S x (kmax+1) x kmax
  cxd *cs, *sn;  // S x kmax (cs real, stored complex)
  cxd *g;        // S x (kmax+1)
  double *beta;  // |r0| per system
  double *resid; // current residual estimate |g_{col+1}|
  int *active;   // still iterating
  int *nact;     // count of active systems after this step
};
__global__ void k_fg_arnoldi_tail(FgScal sc, const cxd *wn2, int S, int kmax, int col, double tol, cxd *invh) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  invh[s] = mk(0.0, 0.0);
  if (!sc.active[s]) return;
  const double hn = sqrt(fmax(wn2[s].re, 0.0));
  cxd *Hs = sc.H + (size_t)s * (kmax + 1) * kmax;
  Hs[(size_t)(col + 1) * kmax + col] = mk(hn, 0.0);
  invh[s] = hn > 0 ? mk(1.0 / hn, 0.0) : mk(0.0, 0.0);
  // apply the previous rotations to column col
  for (int l = 0; l < col; ++l) {
    const cxd c = sc.cs[(size_t)s * kmax + l], sn = sc.sn[(size_t)s * kmax + l];
    const cxd a = Hs[(size_t)l * kmax + col], b = Hs[(size_t)(l + 1) * kmax + col];
    Hs[(size_t)l * kmax + col] = c * a + sn * b;
    Hs[(size_t)(l + 1) * kmax + col] = c * b - conj(sn) * a;
  }
  // new rotation zeroing H[col+1][col]
  const cxd a = Hs[(size_t)col * kmax + col], b = Hs[(size_t)(col + 1) * kmax + col];
  const double na = cabs(a), nb = cabs(b);
  cxd c, sn;
  if (nb == 0.0) {
    c = mk(1.0, 0.0);
    sn = mk(0.0, 0.0);
  } else if (na == 0.0) {
    c = mk(0.0, 0.0);
    sn = (1.0 / nb) * conj(b);  // rotates (0, b) to (|b|, 0)
  } else {
    const double r = hypot(na, nb);
    c = mk(na / r, 0.0);
    sn = (1.0 / (na * r)) * (a * conj(b));  // (a / |a|) conj(b) / r
  }
  sc.cs[(size_t)s * kmax + col] = c;
  sc.sn[(size_t)s * kmax + col] = sn;
  Hs[(size_t)col * kmax + col] = c * a + sn * b;
  Hs[(size_t)(col + 1) * kmax + col] = mk(0.0, 0.0);
  cxd *gs = sc.g + (size_t)s * (kmax + 1);
  const cxd gc = gs[col];
  gs[col] = c * gc;
  gs[col + 1] = (-1.0) * conj(sn) * gc;
  const double res = cabs(gs[col + 1]);
  sc.resid[s] = res;
  if (!(res > tol * sc.beta[s]) || !(hn > 0) || !(res == res)) sc.active[s] = 0;
  if (sc.active[s]) atomicAdd(sc.nact, 1);
}
// v = w * invh (per system), only systems that got a new column
__global__ void k_fg_scale(const cxf *w, const cxd *invh, cxf *v, int ne, int n, int m) {
  const size_t count = (size_t)ne * n * m;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const size_t j = e / ((size_t)n * m), rem = e - j * n * m;
    const int s = (int)j * m + (int)(rem % m);
    v[e] = ccast<float>(invh[s]) * w[e];
  }
}
// start of a cycle: beta = |r| per system, v0 = r / beta, g = (beta, 0, ...)
__global__ void k_fg_start(FgScal sc, const cxd *rn2, int S, int kmax, double tol_abs_scale, const double *bnorm,
                           double tol, cxd *invh) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const double b = sqrt(fmax(rn2[s].re, 0.0));
  sc.beta[s] = bnorm ? bnorm[s] : b;
  for (int q = 0; q < (kmax + 1) * kmax; ++q) sc.H[(size_t)s * (kmax + 1) * kmax + q] = mk(0.0, 0.0);
  for (int q = 0; q <= kmax; ++q) sc.g[(size_t)s * (kmax + 1) + q] = mk(0.0, 0.0);
  sc.g[(size_t)s * (kmax + 1)] = mk(b, 0.0);
  sc.resid[s] = b;
  const bool go = b > tol * sc.beta[s] && b == b && b > 0;
  sc.active[s] = go ? 1 : 0;
  invh[s] = go ? mk(1.0 / b, 0.0) : mk(0.0, 0.0);
  if (go) atomicAdd(sc.nact, 1);
  (void)tol_abs_scale;
}
// y = H^{-1} g (upper triangular, k columns) per system; y into ycoef[s][l]
__global__ void k_fg_solve_small(FgScal sc, int S, int kmax, int k, const int *used, cxd *ycoef) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int kk = used[s];
  const cxd *Hs = sc.H + (size_t)s * (kmax + 1) * kmax;
  const cxd *gs = sc.g + (size_t)s * (kmax + 1);
  cxd *y = ycoef + (size_t)s * kmax;
  for (int l = 0; l < kmax; ++l) y[l] = mk(0.0, 0.0);
  for (int l = kk - 1; l >= 0; --l) {
    cxd acc = gs[l];
    for (int q = l + 1; q < kk; ++q) cfms(acc, Hs[(size_t)l * kmax + q], y[q]);
    const cxd d = Hs[(size_t)l * kmax + l];
    y[l] = (abs2(d) > 0) ? cdiv(acc, d) : mk(0.0, 0.0);
  }
  (void)k;
}
// d += sum_l y_l Z_l
__global__ void k_fg_update_x(const cxf *const *Z, int k, const cxd *ycoef, int kmax, cxf *d, int ne, int n, int m) {
  const size_t count = (size_t)ne * n * m;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const size_t j = e / ((size_t)n * m), rem = e - j * n * m;
    const int s = (int)j * m + (int)(rem % m);
    cxf acc = d[e];
    for (int l = 0; l < k; ++l) cfma(acc, ccast<float>(ycoef[(size_t)s * kmax + l]), Z[l][e]);
    d[e] = acc;
  }
}
// r = b - op(d): op output o = (zB - A) d, so r = b - o
__global__ void k_fg_sub(const cxf *b, const cxf *o, cxf *r, size_t count) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    r[e] = b[e] - o[e];
}
// Jacobi / identity preconditioner: z = v / (z_j b_ii - a_ii) (diag given) or z = v
__global__ void k_fg_jacobi(const cxf *v, const cxd *zn, int conj_z, const cxd *adiag, const cxd *bdiag, cxf *z,
                            int ne, int n, int m) {
  const size_t count = (size_t)ne * n * m;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const size_t j = e / ((size_t)n * m), rem = e - j * n * m;
    const int i = (int)(rem / m);
    if (!adiag) {
      z[e] = v[e];
      continue;
    }
    cxd zj = zn[j];
    if (conj_z) zj = conj(zj);
    cxd a = adiag[i], bd = bdiag ? bdiag[i] : mk(1.0, 0.0);
    if (conj_z) {
      a = conj(a);
      bd = conj(bd);
    }
    const cxd dd = zj * bd - a;
    z[e] = ccast<float>(cdiv(mk(1.0, 0.0), dd)) * v[e];
  }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
size_t fgmres_work_bytes(int n, int m0, int ne, int kmax) {
  const size_t blk = (size_t)ne * n * m0 * sizeof(cxf);
  const size_t S = (size_t)ne * m0;
  const int chunks = 1216;
  return (2 * (size_t)kmax + 4) * blk + (size_t)chunks * (kmax + 1) * S * sizeof(cxd) +
         S * ((size_t)(kmax + 1) * kmax + 3 * kmax + 2 * (kmax + 1) + 8) * sizeof(cxd) + (64 << 10) +
         2 * (size_t)(2 * kmax + 4) * sizeof(void *);
}

namespace {
struct FgWork {
  std::vector<cxf *> V, Z;
  cxf *w, *o, *r;
  cxd *partial, *dots, *invh, *ycoef;
  FgScal sc;
  int *used;
  const cxf **dV, **dZ;
  int chunks;
};

FgWork fg_carve(void *work, int n, int m0, int ne, int kmax) {
  FgWork f;
  unsigned char *p = reinterpret_cast<unsigned char *>(work);
  auto take = [&](size_t bytes) {
    unsigned char *q = p;
    p += (bytes + 255) & ~(size_t)255;
    return q;
  };
  const size_t blk = (size_t)ne * n * m0 * sizeof(cxf);
  const size_t S = (size_t)ne * m0;
  f.chunks = 1216;
  f.V.resize(kmax + 1);
  f.Z.resize(kmax);
  for (int l = 0; l <= kmax; ++l) f.V[l] = (cxf *)take(blk);
  for (int l = 0; l < kmax; ++l) f.Z[l] = (cxf *)take(blk);
  f.w = (cxf *)take(blk);
  f.o = (cxf *)take(blk);
  f.r = (cxf *)take(blk);
  f.partial = (cxd *)take((size_t)f.chunks * (kmax + 1) * S * sizeof(cxd));
  f.dots = (cxd *)take((kmax + 1) * S * sizeof(cxd));
  f.invh = (cxd *)take(S * sizeof(cxd));
  f.ycoef = (cxd *)take(S * kmax * sizeof(cxd));
  f.sc.H = (cxd *)take(S * (kmax + 1) * kmax * sizeof(cxd));
  f.sc.cs = (cxd *)take(S * kmax * sizeof(cxd));
  f.sc.sn = (cxd *)take(S * kmax * sizeof(cxd));
  f.sc.g = (cxd *)take(S * (kmax + 1) * sizeof(cxd));
  f.sc.beta = (double *)take(S * sizeof(double));
  f.sc.resid = (double *)take(S * sizeof(double));
  f.sc.active = (int *)take(S * sizeof(int));
  f.sc.nact = (int *)take(64);
  f.used = (int *)take(S * sizeof(int));
  f.dV = (const cxf **)take((kmax + 1) * sizeof(void *));
  f.dZ = (const cxf **)take(kmax * sizeof(void *));
  return f;
}

void fg_dots(FgWork &f, int nv, const cxf *w, int ne, int n, int m, cudaStream_t s) {
  const int S = ne * m;
  int chunks = std::min(f.chunks, n);
  const int rpc = ceil_div(n, chunks);
  chunks = ceil_div(n, rpc);
  k_fg_dots<<<chunks, kFgThreads, 0, s>>>(f.dV, nv, w, ne, n, m, rpc, f.sc.active, f.partial);
  note_launch();
  k_fg_dots_reduce<<<ceil_div(nv * S, 256), 256, 0, s>>>(f.partial, chunks, nv, S, f.dots);
  note_launch();
}
}  // namespace

int fgmres_solve(const FgmresOp &op, const cxf *b, cxf *d, int n, int m, int ne, int m0, int kmax, int maxit,
                 double tol, void *work, double *maxrel, cudaStream_t s) {
  if (kmax > kFgMaxK) kmax = kFgMaxK;
  FgWork f = fg_carve(work, n, m0, ne, kmax);
  const int S = ne * m;
  const size_t count = (size_t)ne * n * m;
  const unsigned gb = grid_for(count);
  // device arrays of block pointers
  std::vector<const cxf *> hv(f.V.begin(), f.V.end()), hz(f.Z.begin(), f.Z.end());
  cudaMemcpyAsync(f.dV, hv.data(), hv.size() * sizeof(void *), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(f.dZ, hz.data(), hz.size() * sizeof(void *), cudaMemcpyHostToDevice, s);
  // |b| per system (the convergence reference), via the dot kernel on b, b
  cudaMemsetAsync(d, 0, count * sizeof(cxf), s);
  // all systems active for the norm of b
  std::vector<int> ones(S, 1);
  cudaMemcpyAsync(f.sc.active, ones.data(), S * sizeof(int), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(f.r, b, count * sizeof(cxf), cudaMemcpyDeviceToDevice, s);
  {
    const cxf *vb[1] = {b};
    cudaMemcpyAsync(f.dV, vb, sizeof(void *), cudaMemcpyHostToDevice, s);
    fg_dots(f, 1, b, ne, n, m, s);
  }
  // keep |b|^2 in partial-free storage: beta of the first start is |b|
  cudaMemcpyAsync(f.dV, hv.data(), hv.size() * sizeof(void *), cudaMemcpyHostToDevice, s);
  int its = 0;
  int h_nact = 0;
  bool first = true;
  for (int cycle = 0; its < maxit; ++cycle) {
    // r = b - op(d) (d = 0 on the first cycle: r = b)
    if (!first) {
      op.apply(op.ctx, d, f.o, s);
      k_fg_sub<<<gb, 256, 0, s>>>(b, f.o, f.r, count);
      note_launch();
      cudaMemcpyAsync(f.sc.active, ones.data(), S * sizeof(int), cudaMemcpyHostToDevice, s);
      const cxf *vr[1] = {f.r};
      cudaMemcpyAsync(f.dV, vr, sizeof(void *), cudaMemcpyHostToDevice, s);
      fg_dots(f, 1, f.r, ne, n, m, s);
      cudaMemcpyAsync(f.dV, hv.data(), hv.size() * sizeof(void *), cudaMemcpyHostToDevice, s);
    }
    cudaMemsetAsync(f.sc.nact, 0, sizeof(int), s);
    // beta of the first cycle is |b| itself (kept in sc.beta across cycles)
    k_fg_start<<<ceil_div(S, 128), 128, 0, s>>>(f.sc, f.dots, S, kmax, 0.0, first ? nullptr : f.sc.beta, tol,
                                                f.invh);
    note_launch();
    first = false;
    k_fg_scale<<<gb, 256, 0, s>>>(f.r, f.invh, f.V[0], ne, n, m);
    note_launch();
    cudaMemcpyAsync(&h_nact, f.sc.nact, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (h_nact == 0) break;
    int col = 0;
    for (col = 0; col < kmax && its < maxit; ++col, ++its) {
      op.precond(op.ctx, f.V[col], f.Z[col], s);
      op.apply(op.ctx, f.Z[col], f.w, s);
      for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
        fg_dots(f, col + 1, f.w, ne, n, m, s);
        k_fg_orth_update<<<gb, 256, 0, s>>>(f.dV, col + 1, f.dots, f.w, ne, n, m, f.sc.active, f.sc.H, kmax, col);
        note_launch();
      }
      {
        const cxf *vw[1] = {f.w};
        cudaMemcpyAsync(f.dV + kmax, vw, sizeof(void *), cudaMemcpyHostToDevice, s);
      }
      // |w|^2 through the dot kernel with V_kmax := w
      {
        const cxf **dv = f.dV + kmax;
        const int chunks = ceil_div(n, ceil_div(n, std::min(f.chunks, n)));
        const int rpc = ceil_div(n, chunks);
        k_fg_dots<<<chunks, kFgThreads, 0, s>>>(dv, 1, f.w, ne, n, m, rpc, f.sc.active, f.partial);
        note_launch();
        k_fg_dots_reduce<<<ceil_div(S, 256), 256, 0, s>>>(f.partial, chunks, 1, S, f.dots);
        note_launch();
      }
      cudaMemcpyAsync(f.dV + kmax, &hv[kmax], sizeof(void *), cudaMemcpyHostToDevice, s);
      cudaMemsetAsync(f.sc.nact, 0, sizeof(int), s);
      k_fg_arnoldi_tail<<<ceil_div(S, 128), 128, 0, s>>>(f.sc, f.dots, S, kmax, col, tol, f.invh);
      note_launch();
      k_fg_scale<<<gb, 256, 0, s>>>(f.w, f.invh, f.V[col + 1], ne, n, m);
      note_launch();
      // used columns per system: every system uses col + 1 columns this cycle
      // (frozen systems have zero rows in H and g beyond their last column)
      cudaMemcpyAsync(&h_nact, f.sc.nact, sizeof(int), cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
      if (h_nact == 0) {
        ++col;
        ++its;
        break;
      }
    }
    // d += Z y with y = H^{-1} g over the columns built in this cycle
    std::vector<int> used(S, col);
    cudaMemcpyAsync(f.used, used.data(), S * sizeof(int), cudaMemcpyHostToDevice, s);
    k_fg_solve_small<<<ceil_div(S, 128), 128, 0, s>>>(f.sc, S, kmax, col, f.used, f.ycoef);
    note_launch();
    k_fg_update_x<<<gb, 256, 0, s>>>(f.dZ, col, f.ycoef, kmax, d, ne, n, m);
    note_launch();
    if (h_nact == 0) break;
  }
  // true residual of the result, relative to |b|
  op.apply(op.ctx, d, f.o, s);
  k_fg_sub<<<gb, 256, 0, s>>>(b, f.o, f.r, count);
  note_launch();
  cudaMemcpyAsync(f.sc.active, ones.data(), S * sizeof(int), cudaMemcpyHostToDevice, s);
  {
    const cxf *vr[1] = {f.r};
    cudaMemcpyAsync(f.dV, vr, sizeof(void *), cudaMemcpyHostToDevice, s);
    fg_dots(f, 1, f.r, ne, n, m, s);
  }
  std::vector<cxd> rr(S);
  std::vector<double> bb(S);
  cudaMemcpyAsync(rr.data(), f.dots, S * sizeof(cxd), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(bb.data(), f.sc.beta, S * sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  double mx = 0;
  for (int q = 0; q < S; ++q) {
    const double rel = bb[q] > 0 ? sqrt(fmax(rr[q].re, 0.0)) / bb[q] : 0.0;
    mx = (rel > mx || !(rel == rel)) ? rel : mx;
  }
  *maxrel = mx;
  return its;
}

void launch_fg_jacobi(const cxf *v, const cxd *zn, int conj_z, const cxd *adiag, const cxd *bdiag, cxf *z, int ne,
                      int n, int m, cudaStream_t s) {
  k_fg_jacobi<<<grid_for((size_t)ne * n * m), 256, 0, s>>>(v, zn, conj_z, adiag, bdiag, z, ne, n, m);
  note_launch();
}

// X (complex double) = d (mode 0) or X += d (mode 1), d complex float
__global__ void k_cxf_accumulate(cxd *X, const cxf *d, size_t count, int mode) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const cxd v = ccast<double>(d[e]);
    X[e] = mode ? X[e] + v : v;
  }
}
void launch_cxf_accumulate(cxd *X, const cxf *d, size_t count, int mode, cudaStream_t s) {
  k_cxf_accumulate<<<grid_for(count), 256, 0, s>>>(X, d, count, mode);
  note_launch();
}
// out[j] = (complex float) B Y for every node j (node-major copies of one block)
__global__ void k_broadcast_cxf(const cxd *BY, cxf *out, size_t nm, int ne) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nm * ne; e += (size_t)gridDim.x * blockDim.x)
    out[e] = ccast<float>(BY[e % nm]);
}
void launch_broadcast_cxf(const cxd *BY, cxf *out, size_t nm, int ne, cudaStream_t s) {
  k_broadcast_cxf<<<grid_for(nm * ne), 256, 0, s>>>(BY, out, nm, ne);
  note_launch();
}
