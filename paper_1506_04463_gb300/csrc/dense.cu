// Dense kernels of the Rayleigh-Ritz step (Fig. alg:three steps 2-4):
//  * tall-skinny projections G = X^H Y (B_Q, A_U, B_U) and block updates
//    Z = X S (U = Q V Gamma^{-1/2}, Y = U W), FP64 complex;
//  * single-CTA m x m work (m <= 128): eigendecomposition of a general complex
//    matrix (Householder Hessenberg reduction, single-shift complex QR with
//    Wilkinson shifts, back-substitution for the eigenvectors), Gauss-Jordan
//    inverse, small products.
#include <float.h>
#include "kernels.h"

// ---------------------------------------------------------------------------
// G = X^H Y
// ---------------------------------------------------------------------------
constexpr int kGT = 64;   // output tile
constexpr int kGR = 16;   // rows staged per step

__global__ void __launch_bounds__(256) k_gram_partial(const cxd *__restrict__ X, int ldx, int mx,
                                                      const cxd *__restrict__ Y, int ldy, int my, int n,
                                                      int rows_per_chunk, cxd *__restrict__ partial) {
  __shared__ cxd Xs[kGR][kGT];
  __shared__ cxd Ys[kGR][kGT];
  const int chunk = blockIdx.x;
  const int a0 = blockIdx.y * kGT, b0 = blockIdx.z * kGT;
  const int rbeg = chunk * rows_per_chunk, rend = min(n, rbeg + rows_per_chunk);
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  cxd acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mk(0.0, 0.0);
  for (int r0 = rbeg; r0 < rend; r0 += kGR) {
    for (int idx = tid; idx < kGR * kGT; idx += 256) {
      int rr = idx / kGT, cc = idx - rr * kGT;
      int r = r0 + rr;
      Xs[rr][cc] = (r < rend && a0 + cc < mx) ? X[(size_t)r * ldx + a0 + cc] : mk(0.0, 0.0);
      Ys[rr][cc] = (r < rend && b0 + cc < my) ? Y[(size_t)r * ldy + b0 + cc] : mk(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < kGR; ++rr) {
      cxd xa[4], yb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) xa[i] = Xs[rr][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) yb[j] = Ys[rr][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma_cj(acc[i][j], xa[i], yb[j]);
    }
    __syncthreads();
  }
  cxd *P = partial + (size_t)chunk * mx * my;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int a = a0 + ty + 16 * i;
    if (a >= mx) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int b = b0 + tx + 16 * j;
      if (b < my) P[(size_t)a * my + b] = acc[i][j];
    }
  }
}

__global__ void k_gram_reduce(const cxd *partial, int nchunks, int count, cxd *G) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
    cxd s = mk(0.0, 0.0);
    for (int c = 0; c < nchunks; ++c) s = s + partial[(size_t)c * count + e];
    G[e] = s;
  }
}

int gram_chunks(int n) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int c = 2 * sms;
  int byrows = ceil_div(n, 64);
  return c < byrows ? c : (byrows < 1 ? 1 : byrows);
}

void gram(const cxd *X, int ldx, int mx, const cxd *Y, int ldy, int my, int n, cxd *G, cxd *partial, int nchunks,
          cudaStream_t s) {
  const int rpc = ceil_div(n, nchunks);
  const int nc = ceil_div(n, rpc);
  dim3 grid(nc, ceil_div(mx, kGT), ceil_div(my, kGT));
  k_gram_partial<<<grid, 256, 0, s>>>(X, ldx, mx, Y, ldy, my, n, rpc, partial);
  note_launch();
  k_gram_reduce<<<ceil_div(mx * my, 256), 256, 0, s>>>(partial, nc, mx * my, G);
  note_launch();
}

// ---------------------------------------------------------------------------
// Z = X S  (n x mx times mx x mz)
// ---------------------------------------------------------------------------
constexpr int kBT = 64, kBK = 16;
__global__ void __launch_bounds__(256) k_block_small(const cxd *__restrict__ X, int ldx, int mx,
                                                     const cxd *__restrict__ S, int lds, int mz, int n,
                                                     cxd *__restrict__ Z, int ldz) {
  __shared__ cxd Xs[kBT][kBK + 1];
  __shared__ cxd Ss[kBK][kBT];
  const int r0 = blockIdx.x * kBT, b0 = blockIdx.y * kBT;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  cxd acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mk(0.0, 0.0);
  for (int a0 = 0; a0 < mx; a0 += kBK) {
    for (int idx = tid; idx < kBT * kBK; idx += 256) {
      int rr = idx / kBK, aa = idx - rr * kBK;
      int r = r0 + rr, a = a0 + aa;
      Xs[rr][aa] = (r < n && a < mx) ? X[(size_t)r * ldx + a] : mk(0.0, 0.0);
    }
    for (int idx = tid; idx < kBK * kBT; idx += 256) {
      int aa = idx / kBT, bb = idx - aa * kBT;
      int a = a0 + aa, b = b0 + bb;
      Ss[aa][bb] = (a < mx && b < mz) ? S[(size_t)a * lds + b] : mk(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int aa = 0; aa < kBK; ++aa) {
      cxd xr[4], sb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) xr[i] = Xs[ty + 16 * i][aa];
#pragma unroll
      for (int j = 0; j < 4; ++j) sb[j] = Ss[aa][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], xr[i], sb[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = r0 + ty + 16 * i;
    if (r >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int b = b0 + tx + 16 * j;
      if (b < mz) Z[(size_t)r * ldz + b] = acc[i][j];
    }
  }
}

void block_times_small(const cxd *X, int ldx, int mx, const cxd *S, int lds, int mz, int n, cxd *Z, int ldz,
                       cudaStream_t s) {
  dim3 grid(ceil_div(n, kBT), ceil_div(mz, kBT));
  k_block_small<<<grid, 256, 0, s>>>(X, ldx, mx, S, lds, mz, n, Z, ldz);
  note_launch();
}

// ---------------------------------------------------------------------------
// column 2-norms (partials), conj copy, broadcast
// ---------------------------------------------------------------------------
__global__ void k_colnorm2(const cxd *X, int ld, int m, int n, int rows_per_cta, double *partial) {
  __shared__ double red[256];
  const int tid = threadIdx.x;
  const int lanes = 256 / m;
  const int c = tid % m, lr = tid / m;
  double a = 0.0;
  const int rbeg = blockIdx.x * rows_per_cta, rend = min(n, rbeg + rows_per_cta);
  if (lr < lanes)
    for (int i = rbeg + lr; i < rend; i += lanes) a += abs2(X[(size_t)i * ld + c]);
  red[tid] = a;
  __syncthreads();
  if (tid < m) {
    double s = 0.0;
    for (int l = 0; l < lanes; ++l) s += red[l * m + tid];
    partial[(size_t)blockIdx.x * m + tid] = s;
  }
}
int launch_colnorm2(const cxd *X, int ld, int m, int n, double *partial, cudaStream_t s) {
  int g = min(608, ceil_div(n, 64));
  int rpc = ceil_div(n, g);
  g = ceil_div(n, rpc);
  k_colnorm2<<<g, 256, 0, s>>>(X, ld, m, n, rpc, partial);
  note_launch();
  return g;
}

__global__ void k_copy_conj(const cxd *X, cxd *Y, size_t count) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    Y[e] = conj(X[e]);
}
void launch_copy_conj(const cxd *X, cxd *Y, size_t count, cudaStream_t s) {
  k_copy_conj<<<grid_for(count), 256, 0, s>>>(X, Y, count);
  note_launch();
}
__global__ void k_broadcast(const cxd *X, cxd *Y, size_t count, int copies) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    cxd v = X[e];
    for (int k = 0; k < copies; ++k) Y[(size_t)k * count + e] = v;
  }
}
void launch_broadcast_block(const cxd *X, cxd *Y, size_t count, int copies, cudaStream_t s) {
  k_broadcast<<<grid_for(count), 256, 0, s>>>(X, Y, count, copies);
  note_launch();
}

// ---------------------------------------------------------------------------
// small products C = op(A) op(B): (m x k) (k x n)
// ---------------------------------------------------------------------------
__global__ void k_small_mm(const cxd *A, int opA, const cxd *B, int opB, cxd *C, int m, int k, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * n; e += gridDim.x * blockDim.x) {
    int i = e / n, j = e - i * n;
    cxd s = mk(0.0, 0.0);
    for (int l = 0; l < k; ++l) {
      cxd a = opA ? conj(A[(size_t)l * m + i]) : A[(size_t)i * k + l];
      cxd b = opB ? conj(B[(size_t)j * k + l]) : B[(size_t)l * n + j];
      cfma(s, a, b);
    }
    C[e] = s;
  }
}
void small_mm(const cxd *A, int opA, const cxd *B, int opB, cxd *C, int m, int k, int n, cudaStream_t s) {
  k_small_mm<<<ceil_div(m * n, 128), 128, 0, s>>>(A, opA, B, opB, C, m, k, n);
  note_launch();
}

__device__ __forceinline__ double cabs1(cxd a) { return fabs(a.re) + fabs(a.im); }
// 1 / d for d != 0, scaled by a power of two (exact) so |d|^2 cannot over- or
// underflow; one FP64 division instead of the two of a complex quotient
__device__ __forceinline__ cxd crecip(cxd d) {
  const double sc = fmax(fabs(d.re), fabs(d.im));
  const int e = ilogb(sc);
  const double f = scalbn(1.0, -e);
  const cxd ds = mk(d.re * f, d.im * f);
  const double r = f / abs2(ds);
  return mk(ds.re * r, -ds.im * r);
}

// ---------------------------------------------------------------------------
// Gauss-Jordan inverse with partial pivoting (one CTA)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_small_inv(const cxd *A, int m, cxd *Ainv, cxd *W, int *err) {
  __shared__ cxd f[kMaxM0];
  __shared__ double bv[512];
  __shared__ int bi[512];
  __shared__ int piv_s;
  __shared__ cxd dinv_s;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < m * m; e += nt) {
    W[e] = A[e];
    int i = e / m, j = e - i * m;
    Ainv[e] = mk(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int p = 0; p < m; ++p) {
    double best = -1.0;
    int bidx = p;
    for (int i = p + tid; i < m; i += nt) {
      double v = cabs1(W[(size_t)i * m + p]);  // |re| + |im|, as in LAPACK's pivot search
      if (v > best) { best = v; bidx = i; }
    }
    bv[tid] = best;
    bi[tid] = bidx;
    __syncthreads();
    for (int o = nt / 2; o; o >>= 1) {
      if (tid < o) {
        if (bv[tid + o] > bv[tid] || (bv[tid + o] == bv[tid] && bi[tid + o] < bi[tid])) {
          bv[tid] = bv[tid + o];
          bi[tid] = bi[tid + o];
        }
      }
      __syncthreads();
    }
    if (tid == 0) {
      piv_s = bi[0];
      if (!(bv[0] > 0.0)) atomicOr(err, DEVERR_SINGULAR_SMALL);
    }
    __syncthreads();
    const int pr = piv_s;
    if (pr != p) {
      for (int j = tid; j < m; j += nt) {
        cxd t = W[(size_t)p * m + j];
        W[(size_t)p * m + j] = W[(size_t)pr * m + j];
        W[(size_t)pr * m + j] = t;
        t = Ainv[(size_t)p * m + j];
        Ainv[(size_t)p * m + j] = Ainv[(size_t)pr * m + j];
        Ainv[(size_t)pr * m + j] = t;
      }
    }
    __syncthreads();
    if (tid == 0) {
      const cxd d = W[(size_t)p * m + p];
      dinv_s = (d.re != 0.0 || d.im != 0.0) ? crecip(d) : mk(0.0, 0.0);
    }
    __syncthreads();
    const cxd dinv = dinv_s;
    for (int j = tid; j < m; j += nt) {
      W[(size_t)p * m + j] = W[(size_t)p * m + j] * dinv;
      Ainv[(size_t)p * m + j] = Ainv[(size_t)p * m + j] * dinv;
    }
    for (int i = tid; i < m; i += nt) f[i] = W[(size_t)i * m + p];
    __syncthreads();
    for (int e = tid; e < m * m; e += nt) {
      int i = e / m, j = e - i * m;
      if (i == p) continue;
      cfms(W[e], f[i], W[(size_t)p * m + j]);
      cfms(Ainv[e], f[i], Ainv[(size_t)p * m + j]);
    }
    __syncthreads();
  }
}
void small_inv(const cxd *A, int m, cxd *Ainv, cxd *work, int *d_err, cudaStream_t s) {
  k_small_inv<<<1, 512, 0, s>>>(A, m, Ainv, work, d_err);
  note_launch();
}

// ---------------------------------------------------------------------------
// eigendecomposition of a general complex m x m matrix (one CTA)
// ---------------------------------------------------------------------------


// work layout: H (m*m; used when H does not fit in shared memory), Z (m*m), E (m*m).
// H lives in dynamic shared memory (odd row stride) when it fits.  The QR
// sweeps are explicit single-shift steps: the left rotations are formed and
// applied by four warps, each thread owning one column, with one 128-thread
// barrier per rotation; the right rotations of the whole sweep are then
// applied row by row (rows are independent) to H and to Z.
__device__ __forceinline__ void givens(cxd a, cxd b, double &c, cxd &s) {
  // (c, s) with c real, c^2 + |s|^2 = 1 and [c s; -conj(s) c] [a; b] = [r; 0]:
  // c = |a| / rho, s = a conj(b) / (|a| rho), rho^2 = |a|^2 + |b|^2.  The
  // entries are scaled by a power of two (exact) near 1 / max|.|, and both
  // |a| rho and c come from one reciprocal square root of |a|^2 rho^2.
  {
    // usual magnitudes: |a|^2 |a|^2+|b|^2 far from over- and underflow, no scaling
    const double aa2 = abs2(a), t = aa2 + abs2(b);
    if (aa2 > 1e-140 && t < 1e140) {
      const double r1 = rsqrt(aa2 * t);
      c = aa2 * r1;
      s = r1 * (a * conj(b));
      return;
    }
  }
  const double sc = fmax(fmax(fabs(a.re), fabs(a.im)), fmax(fabs(b.re), fabs(b.im)));
  if (sc == 0.0) {
    c = 1.0;
    s = mk(0.0, 0.0);
    return;
  }
  const double inv = scalbn(1.0, -ilogb(sc));
  const cxd as = inv * a, bs = inv * b;
  const double aa2 = abs2(as), t = aa2 + abs2(bs);
  if (aa2 < 1e-280) {  // |a| negligible (or zero) next to |b|
    const double rr = rsqrt(t), ra = aa2 > 0.0 ? rsqrt(aa2) : 0.0;
    c = aa2 * ra * rr;
    s = aa2 > 0.0 ? (ra * rr) * (as * conj(bs)) : mk(bs.re * rr, -bs.im * rr);
    return;
  }
  const double r1 = rsqrt(aa2 * t);
  c = aa2 * r1;
  s = r1 * (as * conj(bs));
}

__global__ void __launch_bounds__(256, 1) k_small_eig(const cxd *A, int m, cxd *lam, cxd *V, cxd *work, int *err,
                                                   int hsm) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ cxd v[kMaxM0];
  __shared__ double red[256];
  __shared__ cxd gs[kMaxM0];  // rotation sines of the current sweep
  __shared__ double gcs[kMaxM0];
  __shared__ int sh_l, sh_hi, sh_done;
  __shared__ cxd sh_mu;
  __shared__ double dsc[kMaxM0];  // balancing: H = D^{-1} A D, D = diag(dsc)
  __shared__ int hskip_s;         // Householder step: reflector scalars from warp 0
  __shared__ double hsc_s;
  __shared__ cxd hbeta_s;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
  const int ld = hsm ? (m | 1) : m;
  cxd *H = hsm ? reinterpret_cast<cxd *>(dsm) : work;
  cxd *Z = work + (size_t)m * m;
  cxd *E = work + 2 * (size_t)m * m;
  for (int e = tid; e < m * m; e += nt) {
    const int i = e / m, j = e - i * m;
    H[(size_t)i * ld + j] = A[e];
    Z[e] = mk(i == j ? 1.0 : 0.0, 0.0);
  }
  for (int i = tid; i < m; i += nt) dsc[i] = 1.0;
  __syncthreads();
  // ---- balancing (Parlett-Reinsch, powers of two, one warp): for each i
  // scale column i by f and row i by 1/f so that their off-diagonal 1-norms
  // (|re| + |im|) come within a factor 2 of each other, until a whole pass
  // changes nothing.  Exact in floating point; it keeps the entries of a
  // reduced matrix whose rows and columns differ in scale by orders of
  // magnitude comparable, so the local deflation test below is meaningful.
  if (tid < 32) {
    for (int pass = 0; pass < 64; ++pass) {
      bool changed = false;
      for (int i = 0; i < m; ++i) {
        double c = 0.0, r = 0.0;
        for (int j = lane; j < m; j += 32)
          if (j != i) {
            c += cabs1(H[(size_t)j * ld + i]);
            r += cabs1(H[(size_t)i * ld + j]);
          }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          c += __shfl_xor_sync(0xffffffffu, c, o);
          r += __shfl_xor_sync(0xffffffffu, r, o);
        }
        if (c == 0.0 || r == 0.0) continue;
        const double s = c + r;
        double f = 1.0;
        for (int q = 0; q < 64 && c < 0.5 * r; ++q) {
          c *= 2.0;
          r *= 0.5;
          f *= 2.0;
        }
        for (int q = 0; q < 64 && c >= 2.0 * r; ++q) {
          c *= 0.5;
          r *= 2.0;
          f *= 0.5;
        }
        if (c + r >= 0.95 * s) continue;
        changed = true;
        const double fi = 1.0 / f;  // exact: f is a power of two
        for (int j = lane; j < m; j += 32) {
          H[(size_t)j * ld + i] = f * H[(size_t)j * ld + i];
          H[(size_t)i * ld + j] = fi * H[(size_t)i * ld + j];
        }
        if (lane == 0) dsc[i] *= f;
        __syncwarp();
      }
      if (!changed) break;
    }
  }
  __syncthreads();
  // ---- Householder reduction to upper Hessenberg form: H = Z^H A Z ----
  for (int k = 0; k + 2 < m; ++k) {
    const int L = m - k - 1;
    // the reflector's scalars, once, in warp 0 (an FP64 instruction costs the
    // same for one lane as for 32, so redundant copies in every warp are not free)
    if (tid < 32) {
      double nrm2 = 0.0;
      for (int i = lane; i < L; i += 32) nrm2 += abs2(H[(size_t)(k + 1 + i) * ld + k]);
#pragma unroll
      for (int o = 16; o; o >>= 1) nrm2 += __shfl_xor_sync(0xffffffffu, nrm2, o);
      if (lane == 0) {
        int skip = nrm2 == 0.0;
        cxd beta = mk(0.0, 0.0);
        double sc = 0.0;
        if (!skip) {
          const double nrm = sqrt(nrm2);
          const cxd x0 = H[(size_t)(k + 1) * ld + k];
          const double ax0 = cabs(x0);
          const cxd ph = ax0 > 0 ? mk(x0.re / ax0, x0.im / ax0) : mk(1.0, 0.0);
          beta = mk(-ph.re * nrm, -ph.im * nrm);
          // |v|^2 = nrm2 - |x0|^2 + |x0 - beta|^2
          const double vn2 = nrm2 - abs2(x0) + abs2(x0 - beta);
          skip = vn2 == 0.0;
          if (!skip) sc = 2.0 / vn2;
        }
        hskip_s = skip;
        hsc_s = sc;
        hbeta_s = beta;
      }
    }
    for (int i = tid; i < L; i += nt) v[i] = H[(size_t)(k + 1 + i) * ld + k];
    __syncthreads();
    if (hskip_s) continue;
    const cxd beta = hbeta_s;
    const double sc = hsc_s;
    if (tid == 0) v[0] = v[0] - beta;
    __syncthreads();
    // left: H[k+1.., j] -= v (v^H H[k+1.., j]) sc, four threads per column
    for (int base = 0; base < m - k; base += nt >> 2) {  // uniform trip count: all lanes shuffle
      const int jj = base + (tid >> 2), j = k + jj, part = tid & 3;
      const bool act = jj < m - k;
      cxd w = mk(0.0, 0.0);
      if (act)
        for (int i = part; i < L; i += 4) cfma_cj(w, v[i], H[(size_t)(k + 1 + i) * ld + j]);
      w.re += __shfl_xor_sync(0xffffffffu, w.re, 1);
      w.im += __shfl_xor_sync(0xffffffffu, w.im, 1);
      w.re += __shfl_xor_sync(0xffffffffu, w.re, 2);
      w.im += __shfl_xor_sync(0xffffffffu, w.im, 2);
      w = sc * w;
      if (act)
        for (int i = part; i < L; i += 4) cfms(H[(size_t)(k + 1 + i) * ld + j], v[i], w);
    }
    __syncthreads();
    // right: every row of H and of Z, columns k+1..
    for (int r = tid; r < 2 * m; r += nt) {
      cxd *M = r < m ? H + (size_t)r * ld : Z + (size_t)(r - m) * m;
      cxd s = mk(0.0, 0.0);
      for (int i = 0; i < L; ++i) cfma(s, M[k + 1 + i], v[i]);
      s = sc * s;
      for (int i = 0; i < L; ++i) {
        cxd &h = M[k + 1 + i];
        // h -= s * conj(v_i)
        h.re -= s.re * v[i].re + s.im * v[i].im;
        h.im -= s.im * v[i].re - s.re * v[i].im;
      }
    }
    __syncthreads();
    for (int i = 1 + tid; i < L; i += nt) H[(size_t)(k + 1 + i) * ld + k] = mk(0.0, 0.0);
    if (tid == 0) H[(size_t)(k + 1) * ld + k] = beta;
    __syncthreads();
  }
  // ---- shifted QR iteration to upper triangular (Schur) form ----
  // A subdiagonal entry is negligible when it is below eps times its two
  // diagonal neighbours, or, once 20 sweeps have not deflated the current
  // eigenvalue, below m * eps * max|h_ij| (the size of the rounding errors of
  // a sweep): without that fallback a graded matrix whose small eigenvalues
  // sit at the rounding level never deflates.
  {
    double hmax = 0.0;
    for (int e = tid; e < m * m; e += nt) {
      const int i = e / m, j = e - i * m;
      if (j + 1 >= i) hmax = fmax(hmax, cabs1(H[(size_t)i * ld + j]));
    }
    red[tid] = hmax;
    __syncthreads();
    for (int o = nt / 2; o; o >>= 1) {
      if (tid < o) red[tid] = fmax(red[tid], red[tid + o]);
      __syncthreads();
    }
  }
  const double hfloor = (double)m * DBL_EPSILON * red[0];
  __syncthreads();
  if (tid == 0) {
    sh_hi = m - 1;
    sh_done = 0;
  }
  __syncthreads();
  int its = 0, total = 0;
  const int maxtotal = 40 * m;
  while (true) {
    if (tid < 32) {
      // warp 0 runs the deflation test and the shift with the same values in
      // every lane (lane 0 writes the results): the largest l <= hi whose
      // subdiagonal is negligible, 32 candidates per vote, 0 if none
      const int hi = sh_hi;
      int l = 0;
      for (int base = hi; base >= 1; base -= 32) {
        const int lc = base - lane;
        bool neg = false;
        if (lc >= 1) {
          const double s = cabs1(H[(size_t)(lc - 1) * ld + lc - 1]) + cabs1(H[(size_t)lc * ld + lc]);
          const double sub = cabs1(H[(size_t)lc * ld + lc - 1]);
          neg = sub <= DBL_EPSILON * s || (its >= 20 && sub <= hfloor) || sub < 1e-300;
        }
        const unsigned vote = __ballot_sync(0xffffffffu, neg);
        if (vote) {
          l = base - (__ffs(vote) - 1);
          break;
        }
      }
      __syncwarp();
      if (lane == 0) {
        if (l > 0) H[(size_t)l * ld + l - 1] = mk(0.0, 0.0);
        sh_l = l;
      }
      if (l == hi) {
        if (lane == 0) sh_hi = hi - 1;
        its = 0;
      } else {
        ++its;
        ++total;
        const cxd a = H[(size_t)(hi - 1) * ld + hi - 1], b = H[(size_t)(hi - 1) * ld + hi];
        const cxd c = H[(size_t)hi * ld + hi - 1], d = H[(size_t)hi * ld + hi];
        cxd mu;
        if (its % 11 == 10) {
          mu = d + mk(0.75 * cabs1(c), 0.0);
        } else {
          const cxd half = mk(0.5 * (a.re - d.re), 0.5 * (a.im - d.im));
          const cxd disc = csqrt(half * half + b * c);
          const cxd mid = mk(0.5 * (a.re + d.re), 0.5 * (a.im + d.im));
          const cxd m1 = mid + disc, m2 = mid - disc;
          mu = abs2(m1 - d) < abs2(m2 - d) ? m1 : m2;
        }
        if (lane == 0) sh_mu = mu;
        if (total > maxtotal && lane == 0) {
          atomicOr(err, DEVERR_QR_NOCONV);
          sh_done = 1;
        }
      }
      __syncwarp();
      if (lane == 0 && sh_hi < 1) sh_done = 1;
    }
    __syncthreads();
    if (sh_done) break;
    const int l = sh_l, hi = sh_hi;
    if (l >= hi) {
      __syncthreads();
      continue;
    }
    const cxd mu = sh_mu;
    for (int i = l + tid; i <= hi; i += nt) H[(size_t)i * ld + i] = H[(size_t)i * ld + i] - mu;
    __syncthreads();
    // left rotations: warps 0-3, one per SM sub-partition (each sub-partition's
    // FP64 pipe serves one warp at a time), thread 32w + lane owning column
    // j = 4 lane + w; the owner of column k forms rotation k from its own
    // column and publishes it through shared memory, one 128-thread named
    // barrier per rotation
    if (tid < 128) {
      const int j = 4 * lane + (tid >> 5);
      for (int k = l; k < hi; ++k) {
        if (j == k) {
          double c;
          cxd s;
          givens(H[(size_t)k * ld + k], H[(size_t)(k + 1) * ld + k], c, s);
          gcs[k] = c;
          gs[k] = s;
        }
        asm volatile("bar.sync 1, 128;\n" ::: "memory");
        if (j >= k && j < m) {
          const double c = gcs[k];
          const cxd s = gs[k];
          cxd *p1 = H + (size_t)k * ld + j, *p2 = p1 + ld;
          const cxd h1 = *p1, h2 = *p2;
          *p1 = c * h1 + s * h2;
          *p2 = c * h2 - conj(s) * h1;
        }
      }
    }
    __syncthreads();
    // right rotations of the sweep: H rows 0..hi (row r meets rotations
    // k >= r - 2) and all rows of Z, each row carried through k in order
    for (int r = tid; r <= hi + m; r += nt) {
      cxd *M;
      int k0;
      if (r <= hi) {
        M = H + (size_t)r * ld;
        k0 = max(l, r - 2);
      } else {
        M = Z + (size_t)(r - hi - 1) * m;
        k0 = l;
      }
      if (k0 >= hi) continue;
      cxd h1 = M[k0];
      for (int k = k0; k < hi; ++k) {
        const double c = gcs[k];
        const cxd s = gs[k];
        const cxd h2 = M[k + 1];
        M[k] = c * h1 + conj(s) * h2;
        h1 = c * h2 - s * h1;
      }
      M[hi] = h1;
    }
    __syncthreads();
    for (int i = l + tid; i <= hi; i += nt) H[(size_t)i * ld + i] = H[(size_t)i * ld + i] + mu;
    __syncthreads();
  }
  // ---- eigenvectors of the triangular T = H, then V = Z E ----
  double tnorm = 0.0;
  for (int e = tid; e < m * m; e += nt) {
    const int i = e / m, j = e - i * m;
    if (j >= i) tnorm = fmax(tnorm, cabs1(H[(size_t)i * ld + j]));
  }
  red[tid] = tnorm;
  __syncthreads();
  for (int o = nt / 2; o; o >>= 1) {
    if (tid < o) red[tid] = fmax(red[tid], red[tid + o]);
    __syncthreads();
  }
  const double small = fmax(red[0], 1e-300) * DBL_EPSILON;
  __syncthreads();
  for (int k = tid; k < m; k += nt) {
    const cxd tk = H[(size_t)k * ld + k];
    for (int j = k + 1; j < m; ++j) E[(size_t)j * m + k] = mk(0.0, 0.0);
    E[(size_t)k * m + k] = mk(1.0, 0.0);
    for (int j = k - 1; j >= 0; --j) {
      cxd s = mk(0.0, 0.0);
      for (int l2 = j + 1; l2 <= k; ++l2) cfma(s, H[(size_t)j * ld + l2], E[(size_t)l2 * m + k]);
      cxd d = H[(size_t)j * ld + j] - tk;
      if (cabs1(d) < small) d = mk(small, 0.0);
      E[(size_t)j * m + k] = -(s * crecip(d));
    }
    lam[k] = tk;
  }
  __syncthreads();
  for (int e = tid; e < m * m; e += nt) {
    const int i = e / m, k = e - i * m;
    cxd s = mk(0.0, 0.0);
    for (int l2 = 0; l2 <= k; ++l2) cfma(s, Z[(size_t)i * m + l2], E[(size_t)l2 * m + k]);
    V[e] = dsc[i] * s;  // eigenvectors of A = D (eigenvectors of H)
  }
  __syncthreads();
  for (int k = tid; k < m; k += nt) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += abs2(V[(size_t)i * m + k]);
    s = s > 0 ? 1.0 / sqrt(s) : 1.0;
    for (int i = 0; i < m; ++i) V[(size_t)i * m + k] = s * V[(size_t)i * m + k];
  }
}

void small_eig(const cxd *A, int m, cxd *lam, cxd *V, cxd *work, int *d_err, cudaStream_t s) {
  const size_t hbytes = (size_t)m * (m | 1) * sizeof(cxd);
  const int hsm = hbytes <= 200 * 1024;
  if (hsm) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_small_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr = true;
    }
  }
  k_small_eig<<<1, 256, hsm ? hbytes : 0, s>>>(A, m, lam, V, work, d_err, hsm);
  note_launch();
}

// Host-requested device error bits (fault-injection aid): *err |= bits.
__global__ void k_or_bits(int *err, int bits) { atomicOr(err, bits); }
void launch_or_bits(int *d_err, int bits, cudaStream_t s) {
  k_or_bits<<<1, 1, 0, s>>>(d_err, bits);
  note_launch();
}
