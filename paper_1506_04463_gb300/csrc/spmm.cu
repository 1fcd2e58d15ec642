// Sparse products of the contour filter and of the Rayleigh-Ritz step.
//
//  * k_multishift_residual: one pass over A (and B) applies every shift z_j
//    to every column: R_j = B Y - (z_j B - A) X_j, the residual of the shifted
//    systems of eq. (qr) for all quadrature nodes at once, and optionally
//    the filtered block Q = sum_j w_j X_j (eq. qr) in fixed node order.
//  * k_node_sum: Q = sum_j w_j X_j alone, once per filter in the refined form.
//  * k_spmm: Out = M1 X - s_c M2 X with a per-column shift, used for B Q,
//    A U, B U and the eigen-residuals of eq. (res).
//  * csr transpose for the conjugate-transpose products A^H, B^H (eq. ql and
//    the left residual of eq. res).
#include "kernels.h"

template <bool CPLX>
__device__ __forceinline__ void csr_fma(cxd &acc, const CsrView &M, int64_t k, const cxd &x) {
  if (CPLX) {
    cxd v = reinterpret_cast<const cxd *>(M.val)[k];
    if (M.conj_vals) v.im = -v.im;
    cfma(acc, v, x);
  } else {
    const double v = M.val[k];
    acc.re = fma(v, x.re, acc.re);
    acc.im = fma(v, x.im, acc.im);
  }
}

// ---------------------------------------------------------------------------
// multi-shift residual + node accumulation
// ---------------------------------------------------------------------------
constexpr int kMsThreads = 256;
constexpr int kMsMaxPairs = 8;  // ne*m <= 2048

template <typename Tout, bool ACPLX, bool BCPLX>
__global__ void __launch_bounds__(kMsThreads)
    k_multishift_residual(CsrView A, CsrView B, int hasB, int ne, const cxd *__restrict__ z,
                          const cxd *__restrict__ w, const cxd *__restrict__ X, size_t xns,
                          const cxd *__restrict__ BY, cx<Tout> *__restrict__ R, cxd *__restrict__ Q,
                          double *__restrict__ partial, int m, int rows_per_cta, const int *skip) {
  if (skip && *skip) return;
  __shared__ cxd zs[kMaxNe], ws[kMaxNe];
  const int tid = threadIdx.x;
  if (tid < ne) {
    zs[tid] = z[tid];
    ws[tid] = w[tid];
  }
  __syncthreads();
  const int P = ne * m;
  const int n = A.n;
  const int rbeg = blockIdx.x * rows_per_cta;
  const int rend = min(n, rbeg + rows_per_cta);
  double nacc[kMsMaxPairs];
#pragma unroll
  for (int q = 0; q < kMsMaxPairs; ++q) nacc[q] = 0.0;

  for (int i = rbeg; i < rend; ++i) {
    const int64_t ka = A.rowptr[i], kae = A.rowptr[i + 1];
#pragma unroll
    for (int q = 0; q < kMsMaxPairs; ++q) {
      const int pair = tid + kMsThreads * q;
      if (pair < P) {
        const int j = pair / m, c = pair - j * m;
        const cxd *Xj = X + (size_t)j * xns;
        cxd acc = BY ? BY[(size_t)i * m + c] : mk(0.0, 0.0);
        cxd bx;
        if (hasB) {
          bx = mk(0.0, 0.0);
          for (int64_t k = B.rowptr[i]; k < B.rowptr[i + 1]; ++k)
            csr_fma<BCPLX>(bx, B, k, Xj[(size_t)B.colind[k] * m + c]);
        } else {
          bx = Xj[(size_t)i * m + c];
        }
        cfms(acc, zs[j], bx);
        for (int64_t k = ka; k < kae; ++k) csr_fma<ACPLX>(acc, A, k, Xj[(size_t)A.colind[k] * m + c]);
        const cx<Tout> ro = ccast<Tout>(acc);
        if (R) R[(size_t)j * xns + (size_t)i * m + c] = ro;
        // the norm of the stored residual, squared in its own precision
        nacc[q] += (double)(ro.re * ro.re + ro.im * ro.im);
      }
    }
    if (Q) {
      for (int c = tid; c < m; c += kMsThreads) {
        cxd qv = mk(0.0, 0.0);
        for (int j = 0; j < ne; ++j) cfma(qv, ws[j], X[(size_t)j * xns + (size_t)i * m + c]);
        Q[(size_t)i * m + c] = qv;
      }
    }
  }
  if (partial) {
#pragma unroll
    for (int q = 0; q < kMsMaxPairs; ++q) {
      const int pair = tid + kMsThreads * q;
      if (pair < P) partial[(size_t)blockIdx.x * P + pair] = nacc[q];
    }
  }
}

// Q = sum_j w_j X_j (eq. q00 with the nodes' solutions), row-major n x m,
// nodes summed in fixed order
__global__ void k_node_sum(int ne, const cxd *__restrict__ w, const cxd *__restrict__ X, size_t xns, size_t nm,
                           cxd *__restrict__ Q) {
  __shared__ cxd ws[kMaxNe];
  if (threadIdx.x < ne) ws[threadIdx.x] = w[threadIdx.x];
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nm; e += (size_t)gridDim.x * blockDim.x) {
    cxd q = mk(0.0, 0.0);
    for (int j = 0; j < ne; ++j) cfma(q, ws[j], X[(size_t)j * xns + e]);
    Q[e] = q;
  }
}
void launch_node_sum(int ne, const cxd *d_w, const cxd *X, size_t xns, int n, int m, cxd *Q, cudaStream_t s) {
  const size_t nm = (size_t)n * m;
  k_node_sum<<<grid_for(nm), 256, 0, s>>>(ne, d_w, X, xns, nm, Q);
  note_launch();
}
// complex128 -> complex64 copy (single-precision right-hand sides)
__global__ void k_to_cxf(const cxd *__restrict__ X, cxf *__restrict__ Y, size_t count) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    Y[e] = ccast<float>(X[e]);
}
void launch_to_cxf(const cxd *X, cxf *Y, size_t count, cudaStream_t s) {
  k_to_cxf<<<grid_for(count), 256, 0, s>>>(X, Y, count);
  note_launch();
}

int spmm_max_grid() {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * 8;
}

static int ms_grid(int n) {
  int g = spmm_max_grid();
  if (g > n) g = n;
  return g < 1 ? 1 : g;
}

template <typename Tout>
int launch_multishift_residual(const CsrView &A, const CsrView *B, int ne, const cxd *d_z, const cxd *d_w,
                               const cxd *X, const cxd *BY, cx<Tout> *R, cxd *Q, double *partial, int m,
                               const int *d_skip, cudaStream_t s) {
  const int grid = ms_grid(A.n);
  const int rpc = ceil_div(A.n, grid);
  const int g = ceil_div(A.n, rpc);
  const size_t xns = (size_t)A.n * m;
  CsrView Bv = B ? *B : A;
  const bool bc = B ? B->cplx : false;
#define MS_LAUNCH(AC, BC)                                                                                \
  k_multishift_residual<Tout, AC, BC><<<g, kMsThreads, 0, s>>>(A, Bv, B != nullptr, ne, d_z, d_w, X, xns, \
                                                               BY, R, Q, partial, m, rpc, d_skip)
  if (A.cplx) {
    if (bc) MS_LAUNCH(true, true); else MS_LAUNCH(true, false);
  } else {
    if (bc) MS_LAUNCH(false, true); else MS_LAUNCH(false, false);
  }
  note_launch();
#undef MS_LAUNCH
  return g;
}
template int launch_multishift_residual<double>(const CsrView &, const CsrView *, int, const cxd *, const cxd *,
                                                const cxd *, const cxd *, cxd *, cxd *, double *, int, const int *,
                                                cudaStream_t);
template int launch_multishift_residual<float>(const CsrView &, const CsrView *, int, const cxd *, const cxd *,
                                               const cxd *, const cxd *, cxf *, cxd *, double *, int, const int *,
                                               cudaStream_t);

// Relative residual of every (side, node, column): ||R||_2 / ||B Y||_2, summed
// over the per-CTA partials in fixed order; the maximum is folded in with an
// integer atomicMax on the bits of the (non-negative) double, which is
// order-independent.
// Same product with the grid capped at max_grid CTAs, so that the partial
// sums fit a caller-provided buffer of max_grid * ne * m doubles.
template <typename Tout>
int launch_multishift_residual_capped(const CsrView &A, const CsrView *B, int ne, const cxd *d_z, const cxd *d_w,
                                      const cxd *X, const cxd *BY, cx<Tout> *R, cxd *Q, double *partial, int m,
                                      int max_grid, cudaStream_t s) {
  int grid = ms_grid(A.n);
  if (grid > max_grid) grid = max_grid;
  const int rpc = ceil_div(A.n, grid);
  const int g = ceil_div(A.n, rpc);
  const size_t xns = (size_t)A.n * m;
  CsrView Bv = B ? *B : A;
  const bool bc = B ? B->cplx : false;
#define MS_LAUNCH(AC, BC)                                                                                \
  k_multishift_residual<Tout, AC, BC><<<g, kMsThreads, 0, s>>>(A, Bv, B != nullptr, ne, d_z, d_w, X, xns, \
                                                               BY, R, Q, partial, m, rpc, nullptr)
  if (A.cplx) {
    if (bc) MS_LAUNCH(true, true); else MS_LAUNCH(true, false);
  } else {
    if (bc) MS_LAUNCH(false, true); else MS_LAUNCH(false, false);
  }
#undef MS_LAUNCH
  note_launch();
  return g;
}
template int launch_multishift_residual_capped<double>(const CsrView &, const CsrView *, int, const cxd *,
                                                       const cxd *, const cxd *, const cxd *, cxd *, cxd *, double *,
                                                       int, int, cudaStream_t);

__global__ void k_residual_rel(const double *partial, int nparts, int P, int m, const double *bynorm2, int nsides,
                               unsigned long long *maxbits) {
  __shared__ double red[128];
  double mx = 0.0;
  const int sp = blockIdx.x * blockDim.x + threadIdx.x;
  if (sp < nsides * P) {
    const int side = sp / P, pair = sp - side * P;
    const double *pb = partial + (size_t)side * nparts * P;
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += pb[(size_t)p * P + pair];
    const double d = bynorm2[side * m + pair % m];
    const double rel = d > 0 ? sqrt(s / d) : sqrt(s);
    mx = (rel == rel) ? rel : INFINITY;
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(maxbits, (unsigned long long)__double_as_longlong(red[0]));
}
__global__ void k_residual_done(const unsigned long long *maxbits, double tol, double *maxrel, int *done) {
  const double v = __longlong_as_double((long long)*maxbits);
  *maxrel = v;
  *done = v <= tol ? 1 : 0;
}

void launch_residual_check(const double *partial, int nparts, int ne, int m, const double *bynorm2, int nsides,
                           double tol, double *d_maxrel, int *d_done, cudaStream_t s) {
  // d_maxrel doubles as the atomic accumulator (bits of a non-negative double)
  unsigned long long *bits = reinterpret_cast<unsigned long long *>(d_maxrel);
  cudaMemsetAsync(bits, 0, sizeof(unsigned long long), s);
  const int total = nsides * ne * m;
  k_residual_rel<<<ceil_div(total, 128), 128, 0, s>>>(partial, nparts, ne * m, m, bynorm2, nsides, bits);
  note_launch();
  k_residual_done<<<1, 1, 0, s>>>(bits, tol, d_maxrel, d_done);
  note_launch();
}

// ---------------------------------------------------------------------------
// single-shift products with per-column shift and column 1-norms
// ---------------------------------------------------------------------------
template <bool C1, bool C2>
__global__ void __launch_bounds__(256) k_spmm(CsrView M1, CsrView M2, int hasM2, const cxd *__restrict__ shift,
                                              const cxd *__restrict__ X, cxd *__restrict__ Out, int m,
                                              int rows_per_cta, double *p1, double *p2) {
  __shared__ double r1[256], r2[256];
  const int tid = threadIdx.x;
  const int lanes = 256 / m;  // m <= 128 -> lanes >= 2
  const int c = tid % m, lr = tid / m;
  const bool active = lr < lanes;
  const int n = M1.n;
  const int rbeg = blockIdx.x * rows_per_cta, rend = min(n, rbeg + rows_per_cta);
  double a1 = 0.0, a2 = 0.0;
  const cxd sh = (shift && active) ? shift[c] : mk(0.0, 0.0);
  if (active) {
    for (int i = rbeg + lr; i < rend; i += lanes) {
      cxd acc = mk(0.0, 0.0);
      for (int64_t k = M1.rowptr[i]; k < M1.rowptr[i + 1]; ++k)
        csr_fma<C1>(acc, M1, k, X[(size_t)M1.colind[k] * m + c]);
      cxd bx;
      if (hasM2) {
        bx = mk(0.0, 0.0);
        for (int64_t k = M2.rowptr[i]; k < M2.rowptr[i + 1]; ++k)
          csr_fma<C2>(bx, M2, k, X[(size_t)M2.colind[k] * m + c]);
      } else {
        bx = X[(size_t)i * m + c];
      }
      if (shift) cfms(acc, sh, bx);
      Out[(size_t)i * m + c] = acc;
      a1 += cabs(acc);
      a2 += cabs(bx);
    }
  }
  if (!p1) return;
  r1[tid] = a1;
  r2[tid] = a2;
  __syncthreads();
  if (tid < m) {
    double s1 = 0.0, s2 = 0.0;
    for (int l = 0; l < lanes; ++l) {
      s1 += r1[l * m + tid];
      s2 += r2[l * m + tid];
    }
    p1[(size_t)blockIdx.x * m + tid] = s1;
    if (p2) p2[(size_t)blockIdx.x * m + tid] = s2;
  }
}

int launch_spmm(const CsrView &M1, const CsrView *M2, const cxd *shift, const cxd *X, cxd *Out, int m, double *p1,
                double *p2, cudaStream_t s) {
  const int grid = ms_grid(M1.n);
  const int rpc = ceil_div(M1.n, grid);
  const int g = ceil_div(M1.n, rpc);
  CsrView M2v = M2 ? *M2 : M1;
  const bool c2 = M2 ? M2->cplx : false;
#define SP_LAUNCH(A1, A2) k_spmm<A1, A2><<<g, 256, 0, s>>>(M1, M2v, M2 != nullptr, shift, X, Out, m, rpc, p1, p2)
  if (M1.cplx) {
    if (c2) SP_LAUNCH(true, true); else SP_LAUNCH(true, false);
  } else {
    if (c2) SP_LAUNCH(false, true); else SP_LAUNCH(false, false);
  }
  note_launch();
#undef SP_LAUNCH
  return g;
}

__global__ void k_reduce_parts(const double *parts, int nparts, int m, double *out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += parts[(size_t)p * m + c];
    out[c] = s;
  }
}
void launch_reduce_parts(const double *parts, int nparts, int m, double *out, cudaStream_t s) {
  k_reduce_parts<<<ceil_div(m, 256), 256, 0, s>>>(parts, nparts, m, out);
  note_launch();
}

// ---------------------------------------------------------------------------
// deterministic CSR transpose
// ---------------------------------------------------------------------------
__global__ void k_count_cols(CsrView A, int32_t *cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x)
    for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) atomicAdd(&cnt[A.colind[k]], 1);
}
// exclusive scan of cnt[0..n) into out[0..n], single CTA
__global__ void k_scan(const int32_t *cnt, int n, int32_t *out) {
  __shared__ int32_t part[1024];
  const int t = threadIdx.x, nt = blockDim.x;
  const int chunk = ceil_div(n, nt);
  const int b = t * chunk, e = min(n, b + chunk);
  int32_t s = 0;
  for (int i = b; i < e; ++i) s += cnt[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int32_t run = 0;
    for (int i = 0; i < nt; ++i) {
      int32_t v = part[i];
      part[i] = run;
      run += v;
    }
    out[n] = run;
  }
  __syncthreads();
  int32_t run = part[t];
  for (int i = b; i < e; ++i) {
    out[i] = run;
    run += cnt[i];
  }
}
__global__ void k_fill_t(CsrView A, const int32_t *rowptr_t, int32_t *cursor, int32_t *colind_t, double *val_t) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x)
    for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
      int c = A.colind[k];
      int pos = rowptr_t[c] + atomicAdd(&cursor[c], 1);
      colind_t[pos] = i;
      if (A.cplx) {
        val_t[2 * (size_t)pos] = A.val[2 * k];
        val_t[2 * (size_t)pos + 1] = A.val[2 * k + 1];
      } else {
        val_t[pos] = A.val[k];
      }
    }
}
__global__ void k_sort_rows(int n, const int32_t *rowptr, int32_t *colind, double *val, int cplx) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int b = rowptr[r], e = rowptr[r + 1];
    for (int i = b + 1; i < e; ++i) {
      int key = colind[i];
      double v0 = cplx ? val[2 * (size_t)i] : val[i];
      double v1 = cplx ? val[2 * (size_t)i + 1] : 0.0;
      int j = i - 1;
      while (j >= b && colind[j] > key) {
        colind[j + 1] = colind[j];
        if (cplx) {
          val[2 * (size_t)(j + 1)] = val[2 * (size_t)j];
          val[2 * (size_t)(j + 1) + 1] = val[2 * (size_t)j + 1];
        } else {
          val[j + 1] = val[j];
        }
        --j;
      }
      colind[j + 1] = key;
      if (cplx) {
        val[2 * (size_t)(j + 1)] = v0;
        val[2 * (size_t)(j + 1) + 1] = v1;
      } else {
        val[j + 1] = v0;
      }
    }
  }
}

cudaError_t csr_transpose(const CsrView &A, int32_t *rowptr_t, int32_t *colind_t, double *val_t, int32_t *work,
                          cudaStream_t s) {
  const int n = A.n;
  const int grid = min(4096, ceil_div(n, 256));
  cudaMemsetAsync(work, 0, (size_t)n * sizeof(int32_t), s);
  k_count_cols<<<grid, 256, 0, s>>>(A, work);
  note_launch();
  k_scan<<<1, 1024, 0, s>>>(work, n, rowptr_t);
  note_launch();
  cudaMemsetAsync(work, 0, (size_t)n * sizeof(int32_t), s);
  k_fill_t<<<grid, 256, 0, s>>>(A, rowptr_t, work, colind_t, val_t);
  note_launch();
  k_sort_rows<<<grid, 256, 0, s>>>(n, rowptr_t, colind_t, val_t, A.cplx);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP32 multi-shift operator of the Krylov sweeps: V_j = (z_j B - A) P_j for
// every node j and column c in one pass over A and B (left side: the
// conjugate-transpose CSR with conj(z_j)).  P, V: node-major ne blocks of
// n x m complex float, row-major.  One warp per (node, row) task, tasks
// node-major so that the warps in flight sweep neighbouring rows of one node
// (stencil neighbours are read from L2); a lane holds VW consecutive columns
// (VW = 2: one 16-byte load per gathered row), the CSR row is read by all
// lanes at the same address (broadcast).
// ---------------------------------------------------------------------------
template <int VW> struct VecF;
template <> struct VecF<1> { using T = float2; };
template <> struct VecF<2> { using T = float4; };

template <bool CPLX>
__device__ __forceinline__ cxf csr_valf(const CsrView &M, int64_t k) {
  if (CPLX) {
    const cxd v = reinterpret_cast<const cxd *>(M.val)[k];
    return mk((float)v.re, M.conj_vals ? -(float)v.im : (float)v.im);
  }
  return mk((float)M.val[k], 0.f);
}

template <int VW>
__device__ __forceinline__ void vfms(typename VecF<VW>::T &acc, cxf a, const typename VecF<VW>::T &x) {
  // acc -= a * x (VW complex lanes)
  acc.x = fmaf(-a.re, x.x, acc.x);
  acc.x = fmaf(a.im, x.y, acc.x);
  acc.y = fmaf(-a.re, x.y, acc.y);
  acc.y = fmaf(-a.im, x.x, acc.y);
  if constexpr (VW == 2) {
    acc.z = fmaf(-a.re, x.z, acc.z);
    acc.z = fmaf(a.im, x.w, acc.z);
    acc.w = fmaf(-a.re, x.w, acc.w);
    acc.w = fmaf(-a.im, x.z, acc.w);
  }
}
template <int VW>
__device__ __forceinline__ void vfma(typename VecF<VW>::T &acc, cxf a, const typename VecF<VW>::T &x) {
  acc.x = fmaf(a.re, x.x, acc.x);
  acc.x = fmaf(-a.im, x.y, acc.x);
  acc.y = fmaf(a.re, x.y, acc.y);
  acc.y = fmaf(a.im, x.x, acc.y);
  if constexpr (VW == 2) {
    acc.z = fmaf(a.re, x.z, acc.z);
    acc.z = fmaf(-a.im, x.w, acc.z);
    acc.w = fmaf(a.re, x.w, acc.w);
    acc.w = fmaf(a.im, x.z, acc.w);
  }
}

// One warp per row i, all nodes: the row's CSR entries (up to KMAX) are
// loaded once into registers and reused for every node j; the gathers of one
// node (one 16-byte load per lane and entry) are independent, so a lane has
// up to KMAX + 1 loads in flight per node.  Rows longer than KMAX, and a
// non-identity B, take the general loop.
template <bool ACPLX, bool BCPLX, bool HASB, int VW, int KMAX>
__global__ void __launch_bounds__(256) k_multishift_spmm_f32(CsrView A, CsrView B, int ne, const cxd *__restrict__ z,
                                                             int conj_z, const cxf *__restrict__ P,
                                                             cxf *__restrict__ V, int n, int m) {
  using V4 = typename VecF<VW>::T;
  __shared__ cxf zs[kMaxNe];
  if (threadIdx.x < ne) {
    const cxd zz = z[threadIdx.x];
    zs[threadIdx.x] = mk((float)zz.re, conj_z ? -(float)zz.im : (float)zz.im);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)(((long long)gridDim.x * blockDim.x) >> 5);
  const size_t xns = (size_t)n * m;
  for (int i = warp; i < n; i += nwarps) {
    const int64_t ka = A.rowptr[i];
    const int nk = (int)(A.rowptr[i + 1] - ka);
    int col[KMAX];
    cxf av[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      col[k] = k < nk ? A.colind[ka + k] : i;
      av[k] = k < nk ? csr_valf<ACPLX>(A, ka + k) : mk(0.f, 0.f);
    }
    const bool fast = !HASB && nk <= KMAX;
    for (int c = lane * VW; c < m; c += 32 * VW) {
#pragma unroll 2
      for (int j = 0; j < ne; ++j) {
        const cxf *Pj = P + (size_t)j * xns;
        V4 acc;
        acc.x = acc.y = 0.f;
        if constexpr (VW == 2) acc.z = acc.w = 0.f;
        if (fast) {
          V4 xs[KMAX];
#pragma unroll
          for (int k = 0; k < KMAX; ++k) xs[k] = *reinterpret_cast<const V4 *>(Pj + (size_t)col[k] * m + c);
          vfma<VW>(acc, zs[j], *reinterpret_cast<const V4 *>(Pj + (size_t)i * m + c));
#pragma unroll
          for (int k = 0; k < KMAX; ++k) vfms<VW>(acc, av[k], xs[k]);
        } else {
          if (HASB) {
            V4 bx;
            bx.x = bx.y = 0.f;
            if constexpr (VW == 2) bx.z = bx.w = 0.f;
            for (int64_t k = B.rowptr[i]; k < B.rowptr[i + 1]; ++k)
              vfma<VW>(bx, csr_valf<BCPLX>(B, k), *reinterpret_cast<const V4 *>(Pj + (size_t)B.colind[k] * m + c));
            vfma<VW>(acc, zs[j], bx);
          } else {
            vfma<VW>(acc, zs[j], *reinterpret_cast<const V4 *>(Pj + (size_t)i * m + c));
          }
          for (int k = 0; k < nk; ++k)
            vfms<VW>(acc, csr_valf<ACPLX>(A, ka + k), *reinterpret_cast<const V4 *>(Pj + (size_t)A.colind[ka + k] * m + c));
        }
        *reinterpret_cast<V4 *>(V + (size_t)j * xns + (size_t)i * m + c) = acc;
      }
    }
  }
}

// Longest row of a CSR matrix (entries), for the register row length of the
// FP32 operator.
__global__ void k_max_row_nnz(CsrView A, int *out) {
  int mx = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x)
    mx = max(mx, (int)(A.rowptr[i + 1] - A.rowptr[i]));
  for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}
void launch_max_row_nnz(const CsrView &A, int *d_out, cudaStream_t s) {
  k_max_row_nnz<<<min(1024, ceil_div(A.n, 256)), 256, 0, s>>>(A, d_out);
  note_launch();
}

template <int KMAX>
static long long spmm_f32_dispatch(const CsrView &A, const CsrView *B, int ne, const cxd *d_z, int conj_z,
                                   const cxf *P, cxf *V, int m, int grid_per_sm, cudaStream_t s) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  CsrView Bv = B ? *B : A;
  const bool bc = B ? B->cplx : false;
  const bool vec2 = (m % 2) == 0;
  long long g = 0;
#define SPF(AC, BC, HB, VW)                                                                                 \
  do {                                                                                                      \
    auto kern = k_multishift_spmm_f32<AC, BC, HB, VW, KMAX>;                                                \
    int occ = 0;                                                                                            \
    if (grid_per_sm > 0) occ = grid_per_sm;                                                                 \
    else if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0) != cudaSuccess || occ < 1) \
      occ = 1;                                                                                              \
    g = (long long)sms * occ;                                                                               \
    const long long need = (A.n + 7) / 8; /* 8 warps per CTA, one row each */                              \
    if (g > need) g = need;                                                                                 \
    if (g < 1) g = 1;                                                                                       \
    kern<<<(unsigned)g, 256, 0, s>>>(A, Bv, ne, d_z, conj_z, P, V, A.n, m);                                 \
  } while (0)
#define SPF_VW(AC, BC, HB) \
  do {                     \
    if (vec2) SPF(AC, BC, HB, 2); else SPF(AC, BC, HB, 1); \
  } while (0)
  if (!B) {
    if (A.cplx) SPF_VW(true, false, false); else SPF_VW(false, false, false);
  } else if (bc) {
    if (A.cplx) SPF_VW(true, true, true); else SPF_VW(false, true, true);
  } else {
    if (A.cplx) SPF_VW(true, false, true); else SPF_VW(false, false, true);
  }
#undef SPF_VW
#undef SPF
  return g;
}

int launch_multishift_spmm_f32(const CsrView &A, const CsrView *B, int ne, const cxd *d_z, int conj_z, const cxf *P,
                               cxf *V, int m, int grid_per_sm, int max_row_nnz, cudaStream_t s) {
  // register row length: the smallest that holds the longest row (longer
  // rows and a non-identity B take the general loop of the same kernel)
  long long g;
  if (max_row_nnz <= 5) g = spmm_f32_dispatch<5>(A, B, ne, d_z, conj_z, P, V, m, grid_per_sm, s);
  else if (max_row_nnz <= 7) g = spmm_f32_dispatch<7>(A, B, ne, d_z, conj_z, P, V, m, grid_per_sm, s);
  else if (max_row_nnz <= 9) g = spmm_f32_dispatch<9>(A, B, ne, d_z, conj_z, P, V, m, grid_per_sm, s);
  else g = spmm_f32_dispatch<16>(A, B, ne, d_z, conj_z, P, V, m, grid_per_sm, s);
  note_launch();
  return (int)g;
}
