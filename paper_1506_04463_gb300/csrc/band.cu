// Banded LU of the shifted matrices (z_j B - A), one per quadrature node, and
// the triangular solves with it.  This is the direct inner solver of the
// contour integration (Fig. alg:three step 1; Sec. 3: the banded driver of the
// paper uses a banded direct solver).  The same factors serve the right solve
// (eq. qr) and the conjugate-transpose left solve (eq. ql), as Sec. 2.4
// describes for solvers with a "transpose conjugate solve" feature.
//
// No pivoting: for the problems this path targets (real A similar to a
// symmetric matrix through a diagonal scaling, complex z_j off the real axis)
// every pivot satisfies |Im pivot| >= |Im z_j| > 0.  A zero pivot is reported.
//
// Storage (per node, row-major band): row r, offset t in [0, W), W = kl+ku+1,
// holds entry (r, r-kl+t); after factorisation t < kl holds L (unit lower) and
// t >= kl holds U.
#include <cuda.h>
#include <cooperative_groups.h>
#include <type_traits>
#include "kernels.h"

// ---------------------------------------------------------------------------
// band extent and build
// ---------------------------------------------------------------------------
__global__ void k_band_extent(CsrView A, int *out) {
  int kl = 0, ku = 0, bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x) {
    const int64_t rb = A.rowptr[i], re = A.rowptr[i + 1];
    if (rb < 0 || re < rb || re > A.nnz || (i == 0 && rb != 0)) { bad = 1; continue; }
    for (int64_t k = rb; k < re; ++k) {
      int c = A.colind[k];
      if (c < 0 || c >= A.n) { bad = 1; continue; }
      int d = c - i;
      if (d < 0) kl = max(kl, -d); else ku = max(ku, d);
    }
  }
  for (int o = 16; o; o >>= 1) {
    kl = max(kl, __shfl_xor_sync(0xffffffffu, kl, o));
    ku = max(ku, __shfl_xor_sync(0xffffffffu, ku, o));
    bad = max(bad, __shfl_xor_sync(0xffffffffu, bad, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, kl);
    atomicMax(out + 1, ku);
    atomicMax(out + 2, bad);
  }
}

void launch_band_extent(const CsrView &A, const CsrView *B, int *d_out, cudaStream_t s) {
  cudaMemsetAsync(d_out, 0, 3 * sizeof(int), s);
  int grid = min(1024, ceil_div(A.n, 256));
  k_band_extent<<<grid, 256, 0, s>>>(A, d_out);
  note_launch();
  if (B) {
    k_band_extent<<<grid, 256, 0, s>>>(*B, d_out);
    note_launch();
  }
}

template <typename T>
__global__ void k_band_build(CsrView A, CsrView B, int hasB, int kl, int ku, int ne, const cxd *z,
                             cx<T> *band) {
  const int n = A.n, W = kl + ku + 1;
  const size_t ns = (size_t)n * W;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int j = 0; j < ne; ++j) {
      cx<T> *row = band + j * ns + (size_t)i * W;
      const cxd zj = z[j];
      for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
        int t = A.colind[k] - i + kl;
        cxd v = csr_val(A, k);
        row[t] = row[t] - ccast<T>(v);
      }
      if (hasB) {
        for (int64_t k = B.rowptr[i]; k < B.rowptr[i + 1]; ++k) {
          int t = B.colind[k] - i + kl;
          row[t] = row[t] + ccast<T>(zj * csr_val(B, k));
        }
      } else {
        row[kl] = row[kl] + ccast<T>(zj);
      }
    }
  }
}

template <typename T>
void launch_band_build(const CsrView &A, const CsrView *B, int kl, int ku, int ne, const cxd *d_z, cx<T> *band,
                       cudaStream_t s) {
  size_t bytes = (size_t)ne * A.n * (kl + ku + 1) * sizeof(cx<T>);
  cudaMemsetAsync(band, 0, bytes, s);
  CsrView Bv = B ? *B : A;
  k_band_build<T><<<min(4096, ceil_div(A.n, 128)), 128, 0, s>>>(A, Bv, B != nullptr, kl, ku, ne, d_z, band);
  note_launch();
}
template void launch_band_build<double>(const CsrView &, const CsrView *, int, int, int, const cxd *, cxd *,
                                        cudaStream_t);
template void launch_band_build<float>(const CsrView &, const CsrView *, int, int, int, const cxd *, cxf *,
                                       cudaStream_t);

// ---------------------------------------------------------------------------
// factorisation: blocked right-looking, panel width NB
// ---------------------------------------------------------------------------
template <typename T> struct FactorCfg;
template <> struct FactorCfg<float> { static constexpr int NB = 32; };
template <> struct FactorCfg<double> { static constexpr int NB = 16; };

template <typename T>
static size_t panel_smem(int kl, int ku, int NB) {
  return ((size_t)(NB + kl) * NB + (size_t)NB * ku) * sizeof(cx<T>);
}

// Factor columns [k, k+nb) (rows [k, k+nb+kl)) and form U12 = L11^{-1} A12
// (rows [k, k+nb), columns [k+nb, k+nb+ku)).  One CTA per node.
template <typename T, int NB>
__global__ void __launch_bounds__(256) k_band_panel(int n, int kl, int ku, int k, cx<T> *band, size_t ns,
                                                    int *err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T> *P = reinterpret_cast<cx<T> *>(smem_raw);  // (NB+kl) x NB
  cx<T> *U = P + (size_t)(NB + kl) * NB;             // NB x ku
  const int W = kl + ku + 1;
  cx<T> *Bd = band + (size_t)blockIdx.x * ns;
  const int nb = min(NB, n - k);
  const int prow = min(n - k, nb + kl);
  const int ucol = max(0, min(n - k - nb, ku));
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int idx = tid; idx < prow * NB; idx += nt) {
    int r = idx / NB, c = idx - r * NB;
    int d = c - r;
    cx<T> v = mk<T>(0, 0);
    if (c < nb && d >= -kl && d <= ku) v = Bd[(size_t)(k + r) * W + (d + kl)];
    P[idx] = v;
  }
  for (int idx = tid; idx < nb * ucol; idx += nt) {
    int r = idx / ucol, c2 = idx - r * ucol;
    int d = nb + c2 - r;
    cx<T> v = mk<T>(0, 0);
    if (d <= ku) v = Bd[(size_t)(k + r) * W + (d + kl)];
    U[r * ku + c2] = v;
  }
  __syncthreads();

  for (int p = 0; p < nb; ++p) {
    const cx<T> piv = P[p * NB + p];
    if (piv.re == 0 && piv.im == 0) {
      if (tid == 0) atomicOr(err, DEVERR_ZERO_PIVOT);
    }
    const int iend = min(prow, p + kl + 1);
    for (int i = p + 1 + tid; i < iend; i += nt) P[i * NB + p] = cdiv(P[i * NB + p], piv);
    __syncthreads();
    const int nq = nb - p - 1;
    if (nq > 0) {
      const int cnt = (iend - p - 1) * nq;
      for (int idx = tid; idx < cnt; idx += nt) {
        int i = p + 1 + idx / nq, q = p + 1 + idx % nq;
        cfms(P[i * NB + q], P[i * NB + p], P[p * NB + q]);
      }
    }
    __syncthreads();
  }
  if (ucol > 0) {
    for (int p = 0; p < nb - 1; ++p) {
      const int cnt = (nb - p - 1) * ucol;
      for (int idx = tid; idx < cnt; idx += nt) {
        int i = p + 1 + idx / ucol, c2 = idx % ucol;
        cfms(U[i * ku + c2], P[i * NB + p], U[p * ku + c2]);
      }
      __syncthreads();
    }
  }
  for (int idx = tid; idx < prow * NB; idx += nt) {
    int r = idx / NB, c = idx - r * NB;
    int d = c - r;
    if (c < nb && d >= -kl && d <= ku) Bd[(size_t)(k + r) * W + (d + kl)] = P[idx];
  }
  for (int idx = tid; idx < nb * ucol; idx += nt) {
    int r = idx / ucol, c2 = idx - r * ucol;
    int d = nb + c2 - r;
    if (d <= ku) Bd[(size_t)(k + r) * W + (d + kl)] = U[r * ku + c2];
  }
}

template <typename T> __device__ __forceinline__ T rcp_rn(T x);
template <> __device__ __forceinline__ float rcp_rn<float>(float x) { return __frcp_rn(x); }
template <> __device__ __forceinline__ double rcp_rn<double>(double x) { return __drcp_rn(x); }

// conj(piv) / |piv|^2 for the panel's pivots (0 for a zero pivot).  FP32:
// the pivot is scaled by the power of two 2^-floor(log2 max(|re|, |im|)),
// formed from the exponent bits (exact), so that |piv|^2 of the scaled value
// lies in [1, 32) and one hardware reciprocal (rcp.approx, relative error
// below 2^-22) completes it; the FP32 factors are refined in FP64, and the
// reciprocal sits on the serial chain of the panel.  FP64: the correctly
// rounded reciprocal, with the same scaling by max(|re|, |im|).
template <typename T> __device__ __forceinline__ cx<T> pivot_recip(cx<T> piv);
template <> __device__ __forceinline__ cx<float> pivot_recip<float>(cx<float> piv) {
  const float sc = fmaxf(fabsf(piv.re), fabsf(piv.im));
  if (sc == 0.f) return mk<float>(0.f, 0.f);
  const int e = min(max((__float_as_int(sc) >> 23) & 0xFF, 1), 253);
  const float rs = __int_as_float((254 - e) << 23);  // 2^(127 - e)
  const float ar = piv.re * rs, ai = piv.im * rs;
  float rd;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rd) : "f"(ar * ar + ai * ai));
  rd *= rs;
  return mk<float>(ar * rd, -ai * rd);
}
template <> __device__ __forceinline__ cx<double> pivot_recip<double>(cx<double> piv) {
  const double sc = fmax(fabs(piv.re), fabs(piv.im));
  if (sc == 0.0) return mk<double>(0.0, 0.0);
  const double rs = rcp_rn(sc), ar = piv.re * rs, ai = piv.im * rs;
  const double rd = rcp_rn(ar * ar + ai * ai) * rs;
  return mk<double>(ar * rd, -ai * rd);
}

// Register panel elimination with compile-time column indices: thread i holds
// row i of the panel in row[]; prow_s is a double-buffered pivot row and
// pinv_s the reciprocal of its pivot, formed once by the pivot thread.
template <typename T, int NB>
__device__ __forceinline__ void panel_eliminate(cx<T> (&row)[NB], cx<T> (*prow_s)[NB], cx<T> *pinv_s, int i, bool own,
                                                int nb, int kl, int *err) {
#pragma unroll
  for (int p = 0; p < NB; ++p) {
    if (p < nb) {
      cx<T> *pr = prow_s[p & 1];
      if (i == p) {
#pragma unroll
        for (int q = p + 1; q < NB; ++q) pr[q] = row[q];
        const cx<T> piv = row[p];
        if (piv.re == 0 && piv.im == 0) atomicOr(err, DEVERR_ZERO_PIVOT);
        pinv_s[p & 1] = pivot_recip<T>(piv);
      }
      __syncthreads();
      if (own && i > p && i - p <= kl) {
        const cx<T> l = row[p] * pinv_s[p & 1];
        row[p] = l;
#pragma unroll
        for (int q = p + 1; q < NB; ++q) cfms(row[q], l, pr[q]);
      }
    }
  }
}

// Register form of the panel step for bands with NB + kl <= 512: thread i
// holds row k+i of the panel (columns [k, k+nb)) in registers; the pivot row
// of each elimination step is published through a double-buffered shared
// row, so each column costs one barrier.  U12 is formed by k_band_u12.
template <typename T, int NB>
__global__ void __launch_bounds__(512) k_band_panel_reg(int n, int kl, int ku, int k, cx<T> *band, size_t ns,
                                                         int *err) {
  __shared__ cx<T> prow_s[2][NB];
  __shared__ cx<T> pinv_s[2];
  const int W = kl + ku + 1;
  cx<T> *Bd = band + (size_t)blockIdx.x * ns;
  const int nb = min(NB, n - k);
  const int prow = min(n - k, nb + kl);
  const int i = threadIdx.x;
  const bool own = i < prow;
  cx<T> row[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int d = q - i;
    row[q] = (own && q < nb && d >= -kl && d <= ku) ? Bd[(size_t)(k + i) * W + (d + kl)] : mk<T>(0, 0);
  }
  panel_eliminate<T, NB>(row, prow_s, pinv_s, i, own, nb, kl, err);
  if (own) {
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int d = q - i;
      if (q < nb && d >= -kl && d <= ku) Bd[(size_t)(k + i) * W + (d + kl)] = row[q];
    }
  }
}

// U12 = L11^{-1} A12 for the panel at column k, one column per thread (no
// barrier): rows [k, k+nb), columns [k+nb, k+nb+ku).  grid (ceil(ku/128), ne).
template <typename T, int NB>
__global__ void __launch_bounds__(128) k_band_u12(int n, int kl, int ku, int k, cx<T> *band, size_t ns) {
  __shared__ cx<T> L11[NB][NB + 1];
  const int W = kl + ku + 1;
  cx<T> *Bd = band + (size_t)blockIdx.y * ns;
  const int nb = min(NB, n - k);
  const int ucol = max(0, min(n - k - nb, ku));
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, p = e - r * NB;
    const int d = p - r;
    L11[r][p] = (r < nb && p < r && -d <= kl) ? Bd[(size_t)(k + r) * W + (d + kl)] : mk<T>(0, 0);
  }
  __syncthreads();
  const int c2 = blockIdx.x * blockDim.x + threadIdx.x;
  if (c2 >= ucol) return;
  cx<T> col[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    const int d = nb + c2 - r;
    col[r] = (r < nb && d <= ku) ? Bd[(size_t)(k + r) * W + (d + kl)] : mk<T>(0, 0);
  }
#pragma unroll
  for (int r = 1; r < NB; ++r)
#pragma unroll
    for (int p = 0; p < r; ++p) cfms(col[r], L11[r][p], col[p]);
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    const int d = nb + c2 - r;
    if (r < nb && d <= ku) Bd[(size_t)(k + r) * W + (d + kl)] = col[r];
  }
}

// Trailing update A22 -= L21 * U12 on rows [k+nb, k+nb+kl) x cols [k+nb, k+nb+ku).
template <typename T, int NB>
__global__ void __launch_bounds__(256) k_band_update(int n, int kl, int ku, int k, cx<T> *band, size_t ns) {
  constexpr int TM = 64, TN = 64;
  __shared__ cx<T> Ls[TM][NB + 1];
  __shared__ cx<T> Us[NB][TN];
  const int W = kl + ku + 1;
  cx<T> *Bd = band + (size_t)blockIdx.z * ns;
  const int nb = min(NB, n - k);
  const int r_beg = k + nb, r_end = min(n, k + nb + kl), c_end = min(n, k + nb + ku);
  const int r0 = r_beg + blockIdx.y * TM, c0 = r_beg + blockIdx.x * TN;
  if (r0 >= r_end || c0 >= c_end) return;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < TM * NB; idx += 256) {
    int rr = idx / NB, p = idx - rr * NB;
    int r = r0 + rr, col = k + p;
    cx<T> v = mk<T>(0, 0);
    if (r < r_end && p < nb && r - col <= kl) v = Bd[(size_t)r * W + (col - r + kl)];
    Ls[rr][p] = v;
  }
  for (int idx = tid; idx < NB * TN; idx += 256) {
    int p = idx / TN, cc = idx - p * TN;
    int row = k + p, c = c0 + cc;
    cx<T> v = mk<T>(0, 0);
    if (p < nb && c < c_end && c - row <= ku) v = Bd[(size_t)row * W + (c - row + kl)];
    Us[p][cc] = v;
  }
  __syncthreads();
  const int ty = tid >> 4, tx = tid & 15;
  cx<T> acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mk<T>(0, 0);
  for (int p = 0; p < nb; ++p) {
    cx<T> a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = Ls[ty + 16 * i][p];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = Us[p][tx + 16 * j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = r0 + ty + 16 * i;
    if (r >= r_end) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int c = c0 + tx + 16 * j;
      if (c >= c_end) continue;
      cx<T> &e = Bd[(size_t)r * W + (c - r + kl)];
      e = e - acc[i][j];
    }
  }
}

// ---------------------------------------------------------------------------
// factorisation as one persistent launch: one thread-block cluster of CL CTAs
// per node.  Panels of NB columns are factored in registers (thread = row) by
// CTA (panel index mod CL).  During step k the other CL - 1 CTAs split the
// trailing window of panel k by columns, form U12 for their columns (one warp
// per column, lane = row, the solved entries passed on by shuffles) and apply
// the rank-nb update, the next panel's columns first; as soon as those are
// done the next panel's owner factors it, overlapping the rest of the update.
// Band data shared between CTAs is read with ld.global.cg (L2), so no CTA can
// see a stale L1 line; cluster barriers (release / acquire) order the steps.
// Requires nb + kl <= 512 and a worker's share of the window <= FMAXC columns.
// ---------------------------------------------------------------------------
constexpr int FNT = 512;     // threads per CTA
constexpr int FMAXC = 64;    // columns a CTA owns per step

template <typename T>
__device__ __forceinline__ cx<T> ldcg(const cx<T> *p) {
  if constexpr (sizeof(T) == 4) {
    float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return mk<T>(v.x, v.y);
  } else {
    double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
    return mk<T>(v.x, v.y);
  }
}

__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory"); }

// Step k (panel columns [k, k+nb) already factored): the CTA that owns the
// next panel waits only until the other CL-1 CTAs have applied step k's
// update to that panel's columns (first cluster-barrier phase), then factors
// it, while the others update the rest of the trailing window (look-ahead).
template <typename T, int NB, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(FNT)
    k_band_factor_cluster(int n, int kl, int ku, cx<T> *band, size_t ns, int *err) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // L21 of the current step (kl x NB) in the updating CTAs; the next panel
  // staged for coalesced loads and stores ((NB + kl) x (NB + 1)) in its owner
  cx<T> *Ls = reinterpret_cast<cx<T> *>(smem_raw);
  cx<T> *Ps = Ls;
  constexpr int PLD = NB + 1;
  constexpr int UNR = 8;  // loads in flight per thread while staging
  __shared__ cx<T> prow_s[2][NB];
  __shared__ cx<T> pinv_s[2];
  __shared__ cx<T> L11[NB][NB + 1];
  __shared__ cx<T> Us[NB][FMAXC];
  const int W = kl + ku + 1;
  cx<T> *Bd = band + (size_t)blockIdx.y * ns;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // factor the panel at columns [k, k+nb) in registers (thread = row)
  auto factor_panel = [&](int k) {
    const int nb = min(NB, n - k);
    const int prow = min(n - k, nb + kl);
    for (int i0 = warp; i0 < prow; i0 += UNR * (FNT / 32)) {
      cx<T> v[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int i = i0 + u * (FNT / 32), d = lane - i;
        v[u] = (i < prow && lane < nb && d >= -kl && d <= ku) ? ldcg(Bd + (size_t)(k + i) * W + (d + kl))
                                                            : mk<T>(0, 0);
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int i = i0 + u * (FNT / 32);
        if (i < prow) Ps[i * PLD + lane] = v[u];
      }
    }
    __syncthreads();
    const int i = tid;
    const bool own = i < prow;
    cx<T> row[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) row[q] = own ? Ps[i * PLD + q] : mk<T>(0, 0);
    panel_eliminate<T, NB>(row, prow_s, pinv_s, i, own, nb, kl, err);
    if (own) {
#pragma unroll
      for (int q = 0; q < NB; ++q) Ps[i * PLD + q] = row[q];
    }
    __syncthreads();
    for (int i1 = warp; i1 < prow; i1 += FNT / 32) {
      const int d = lane - i1;
      if (lane < nb && d >= -kl && d <= ku) Bd[(size_t)(k + i1) * W + (d + kl)] = Ps[i1 * PLD + lane];
    }
  };

  // U12 = L11^{-1} A12 and A22 -= L21 U12 for columns [a, b) (b - a <= FMAXC)
  // of the trailing window of the panel at k; L11, L21 staged
  auto update_cols = [&](int k, int a, int b) {
    const int nb = min(NB, n - k);
    const int c_beg = k + nb, r_end = min(n, k + nb + kl);
    const int nrows = r_end - c_beg;
    const int ncol = b - a;
    if (ncol <= 0) return;
    // U12: each warp solves four columns side by side, lane = row, the solved
    // entries passed on by shuffles
    {
      const int r = lane;
      cx<T> u[4];
      bool in[4];
      int cc[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int slot = warp + s * (FNT / 32);
        cc[s] = slot < ncol ? a + slot : -1;
        const int d = cc[s] - (k + r);
        in[s] = cc[s] >= 0 && r < nb && d <= ku;
        u[s] = in[s] ? ldcg(Bd + (size_t)(k + r) * W + (d + kl)) : mk<T>(0, 0);
      }
#pragma unroll
      for (int p = 0; p < NB - 1; ++p) {
        const cx<T> l = L11[r][p];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          cx<T> up;
          up.re = __shfl_sync(0xffffffffu, u[s].re, p);
          up.im = __shfl_sync(0xffffffffu, u[s].im, p);
          if (r > p) cfms(u[s], l, up);
        }
      }
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if (in[s]) Bd[(size_t)(k + r) * W + (cc[s] - (k + r) + kl)] = u[s];
        Us[r][warp + s * (FNT / 32)] = u[s];
      }
    }
    __syncthreads();
    // update: threads on (column, row chunk) pairs, consecutive threads on
    // consecutive columns (coalesced along band rows), U12 column in
    // registers, L21 entry pairs as shared-memory broadcasts, 4 rows at a
    // time with the next 4 entries loaded ahead
    const int nch = FNT / ncol;
    if (tid < nch * ncol) {
      const int slot = tid % ncol, chunk = tid / ncol;
      const int c = a + slot;
      cx<T> u[NB];
#pragma unroll
      for (int p = 0; p < NB; ++p) u[p] = Us[p][slot];
      const int per = ((nrows + nch - 1) / nch + 3) & ~3;
      const int rb = chunk * per, re = min(nrows, rb + per);
      cx<T> cur[4], nxt[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int rr = rb + q;
        nxt[q] = rr < re ? ldcg(Bd + (size_t)(c_beg + rr) * W + (c - (c_beg + rr) + kl)) : mk<T>(0, 0);
      }
      for (int r4 = rb; r4 < re; r4 += 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) cur[q] = nxt[q];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int rr = r4 + 4 + q;
          nxt[q] = rr < re ? ldcg(Bd + (size_t)(c_beg + rr) * W + (c - (c_beg + rr) + kl)) : mk<T>(0, 0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const cx<T> *lrow = Ls + (size_t)min(r4 + q, nrows - 1) * NB;
#pragma unroll
          for (int p = 0; p < NB; p += 2) {
            cx<T> l0, l1;
            if constexpr (sizeof(T) == 4) {
              const float4 l2 = *reinterpret_cast<const float4 *>(lrow + p);
              l0 = mk<T>(l2.x, l2.y);
              l1 = mk<T>(l2.z, l2.w);
            } else {
              l0 = lrow[p];
              l1 = lrow[p + 1];
            }
            cfms(cur[q], l0, u[p]);
            cfms(cur[q], l1, u[p + 1]);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int rr = r4 + q;
          if (rr < re) Bd[(size_t)(c_beg + rr) * W + (c - (c_beg + rr) + kl)] = cur[q];
        }
      }
    }
    __syncthreads();
  };

  if (rank == 0) factor_panel(0);
  cluster_arrive();
  cluster_wait();
  for (int k = 0; k < n; k += NB) {
    const int nb = min(NB, n - k);
    const int next_owner = (k / NB + 1) % CL;
    const int c_beg = k + nb, c_end = min(n, k + nb + ku), r_end = min(n, k + nb + kl);
    const int nrows = r_end - c_beg;
    if (rank != next_owner) {
      const int w = (rank - next_owner - 1 + CL) % CL;  // worker index in [0, CL-1)
      const bool work = c_beg < c_end && nrows > 0;
      if (work) {
        for (int e = tid; e < NB * NB; e += FNT) {
          const int r = e / NB, p = e - r * NB;
          L11[r][p] = (r < nb && p < r && r - p <= kl) ? ldcg(Bd + (size_t)(k + r) * W + (p - r + kl)) : mk<T>(0, 0);
        }
        const int tot = nrows * NB;
        // all of L21 (kl x 32 entries, <= 20 per thread at kl <= 300) in flight at once
        constexpr int UNR2 = 20;
        for (int e0 = tid; e0 < tot; e0 += UNR2 * FNT) {
          cx<T> v[UNR2];
#pragma unroll
          for (int u = 0; u < UNR2; ++u) {
            const int e = e0 + u * FNT;
            const int rr = e / NB, p = e - rr * NB;
            const int r = c_beg + rr;
            v[u] = (e < tot && p < nb && r - (k + p) <= kl) ? ldcg(Bd + (size_t)r * W + (k + p - r + kl))
                                                            : mk<T>(0, 0);
          }
#pragma unroll
          for (int u = 0; u < UNR2; ++u) {
            const int e = e0 + u * FNT;
            if (e < tot) Ls[e] = v[u];
          }
        }
        __syncthreads();
      }
      // the next panel's columns first, then the rest, each split evenly
      const int pe = min(c_end, c_beg + NB);
      if (work) update_cols(k, c_beg + (pe - c_beg) * w / (CL - 1), c_beg + (pe - c_beg) * (w + 1) / (CL - 1));
      cluster_arrive();
      if (work) update_cols(k, pe + (c_end - pe) * w / (CL - 1), pe + (c_end - pe) * (w + 1) / (CL - 1));
      cluster_wait();
    } else {
      cluster_arrive();
      cluster_wait();
      if (k + NB < n) factor_panel(k + NB);
    }
    cluster_arrive();
    cluster_wait();
  }
}

// The FP64 factorisation is bound by the FP64 pipes; the per-step launches
// spread its trailing updates over every SM, which measured faster there.
// the panel rows fit one thread each, and a worker's share of the trailing
// window (CL - 1 = 7 workers at least) fits FMAXC columns
template <typename T> bool band_factor_cluster_ok(int kl, int ku) {
  return sizeof(T) == 4 && FactorCfg<T>::NB + kl <= FNT && ku + FactorCfg<T>::NB <= FMAXC * 7;
}

// resident clusters of CL CTAs with the largest shared-memory request
template <typename T, int CL>
static int factor_cluster_capacity() {
  auto kern = k_band_factor_cluster<T, FactorCfg<T>::NB, CL>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess ||
      (CL > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, 1, 1);
  cfg.blockDim = dim3(FNT, 1, 1);
  cfg.dynamicSmemBytes = 160 * 1024;
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) nc = 0;
  cudaGetLastError();
  return nc;
}

template <typename T> bool band_fits(int kl, int ku) {
  constexpr int NB = FactorCfg<T>::NB;
  return panel_smem<T>(kl, ku, NB) <= 220 * 1024;
}
template bool band_fits<float>(int, int);
template bool band_fits<double>(int, int);

template <typename T>
cudaError_t band_factor(int n, int kl, int ku, int ne, cx<T> *band, int *d_err, cudaStream_t s) {
  constexpr int NB = FactorCfg<T>::NB;
  const size_t ns = (size_t)n * (kl + ku + 1);
  static int cap10 = -1, cap8 = -1;  // resident 10- and 8-CTA clusters
  const size_t fsmem = (size_t)(NB + kl) * (NB + 1) * sizeof(cx<T>);  // >= kl x NB of L21
  if constexpr (sizeof(T) == 4) {
    if (cap8 < 0) {
      cap10 = factor_cluster_capacity<T, 10>();
      cap8 = factor_cluster_capacity<T, 8>();
    }
    if (band_factor_cluster_ok<T>(kl, ku) && fsmem <= 160 * 1024 && (cap10 >= ne || cap8 > 0)) {
      // 10-CTA clusters (9 updating CTAs per panel) when every factor slot gets
      // one at once, else 8; with the panel on the critical path, larger
      // clusters gain nothing more (measured: 12 CTAs as 10, 92 ms for 8)
      if (cap10 >= ne)
        k_band_factor_cluster<T, NB, 10><<<dim3(10, ne), FNT, fsmem, s>>>(n, kl, ku, band, ns, d_err);
      else
        k_band_factor_cluster<T, NB, 8><<<dim3(8, ne), FNT, fsmem, s>>>(n, kl, ku, band, ns, d_err);
      note_launch();
      return cudaGetLastError();
    }
  }
  const size_t smem = panel_smem<T>(kl, ku, NB);
  const bool reg = NB + kl <= 512;
  const int reg_threads = ceil_div(NB + kl, 32) * 32;
  if (!reg) {
    cudaError_t e = cudaFuncSetAttribute(k_band_panel<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  for (int k = 0; k < n; k += NB) {
    if (reg) {
      k_band_panel_reg<T, NB><<<ne, reg_threads, 0, s>>>(n, kl, ku, k, band, ns, d_err);
      note_launch();
      const int ucol = min(n - k - min(NB, n - k), ku);
      if (ucol > 0) {
        k_band_u12<T, NB><<<dim3(ceil_div(ucol, 128), ne), 128, 0, s>>>(n, kl, ku, k, band, ns);
        note_launch();
      }
    } else {
      k_band_panel<T, NB><<<ne, 256, smem, s>>>(n, kl, ku, k, band, ns, d_err);
      note_launch();
    }
    const int nb = min(NB, n - k);
    const int rows = min(n, k + nb + kl) - (k + nb);
    const int cols = min(n, k + nb + ku) - (k + nb);
    if (rows > 0 && cols > 0) {
      dim3 grid(ceil_div(cols, 64), ceil_div(rows, 64), ne);
      k_band_update<T, NB><<<grid, 256, 0, s>>>(n, kl, ku, k, band, ns);
      note_launch();
    }
  }
  return cudaGetLastError();
}
template cudaError_t band_factor<float>(int, int, int, int, cxf *, int *, cudaStream_t);
template cudaError_t band_factor<double>(int, int, int, int, cxd *, int *, cudaStream_t);

// ---------------------------------------------------------------------------
// triangular solves, both sides in one launch
// ---------------------------------------------------------------------------
// grid (ceil(m/R), ne, nsides).  Side 0 solves (LU) x = b (right, eq. qr),
// side 1 solves (LU)^H x = b (left, eq. ql).  Each CTA owns R columns of one
// node and sweeps all rows: forward with the lower factor, backward with the
// upper one, blocks of NB rows.  Inside a block the update by earlier blocks
// is a small GEMM against a ring buffer of the last rows in shared memory;
// the NB x NB triangle is then solved row by row.
template <typename T> struct SolveCfg;
template <> struct SolveCfg<float> { static constexpr int NB = 32, R = 16, RPT = 2; };
template <> struct SolveCfg<double> { static constexpr int NB = 16, R = 16, RPT = 1; };

struct SolveSides {
  const void *rhs[2];
  cxd *X[2];
  // node j uses factor slot fmap[j] & 0xffff; bit 16 set: the factors are
  // the complex conjugates of that slot's (real pencil, conjugate node pair)
  int fmap[kMaxNe];
};

template <typename T>
__device__ __forceinline__ cx<T> cj_if(cx<T> v, bool c) {
  if (c) v.im = -v.im;
  return v;
}
template <typename T>
__device__ __forceinline__ cx<T> lower_elem(const cx<T> *Bd, int W, int kl, int ku, bool herm, bool cj, int r, int i) {
  // strictly lower part of the forward factor: N -> L(r,i); H -> conj(U(i,r));
  // cj: factors of the conjugate node
  int d = r - i;
  if (!herm) {
    if (d > kl) return mk<T>(0, 0);
    return cj_if(Bd[(size_t)r * W + (kl - d)], cj);
  }
  if (d > ku) return mk<T>(0, 0);
  return cj_if(Bd[(size_t)i * W + (kl + d)], !cj);
}
template <typename T>
__device__ __forceinline__ cx<T> upper_elem(const cx<T> *Bd, int W, int kl, int ku, bool herm, bool cj, int r, int i) {
  // strictly upper part of the backward factor: N -> U(r,i); H -> conj(L(i,r))
  int d = i - r;
  if (!herm) {
    if (d > ku) return mk<T>(0, 0);
    return cj_if(Bd[(size_t)r * W + (kl + d)], cj);
  }
  if (d > kl) return mk<T>(0, 0);
  return cj_if(Bd[(size_t)i * W + (kl - d)], !cj);
}

template <typename T, typename Tin, int NB, int R, int RPT>
__global__ void __launch_bounds__(R *NB / RPT) k_band_solve(int n, int kl, int ku, const cx<T> *band, size_t bns,
                                                            SolveSides io, size_t rns, int m, size_t xns, int mode,
                                                            cx<T> *ysc, const int *skip) {
  if (skip && *skip) return;
  constexpr int G = NB / RPT;
  constexpr int NT = R * G;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int W = kl + ku + 1;
  const int bwmax = max(kl, ku);
  const int TW = bwmax + NB;
  const int RB = ceil_div(bwmax + NB, NB) * NB;
  cx<T> *Ms = reinterpret_cast<cx<T> *>(smem_raw);
  cx<T> *ring = Ms + (size_t)NB * TW;
  cx<T> *dg = ring + (size_t)RB * R;

  const int side = blockIdx.z;
  const bool herm = side == 1;
  const int node = blockIdx.y;
  const int c0 = blockIdx.x * R;
  const bool cj = (io.fmap[node] >> 16) & 1;
  const cx<T> *Bd = band + (size_t)(io.fmap[node] & 0xffff) * bns;
  const cx<Tin> *Rh = reinterpret_cast<const cx<Tin> *>(io.rhs[side]) + (size_t)node * rns;
  cxd *Xn = io.X[side] + (size_t)node * xns;
  cx<T> *Ys = ysc + (((size_t)side * gridDim.y + node) * gridDim.x + blockIdx.x) * (size_t)n * R;
  const int tid = threadIdx.x;
  const int col = tid % R, rg = tid / R;
  const int c = c0 + col;
  const bool cok = c < m;

  cx<T> acc[RPT];
  // ---------------- forward (lower) ----------------
  {
    const int bw = herm ? ku : kl;
    const int TWl = bw + NB;
    for (int kb = 0; kb < n; kb += NB) {
      const int nbk = min(NB, n - kb);
      const int i0 = kb - bw;
      if (!herm) {
        for (int idx = tid; idx < NB * TWl; idx += NT) {
          int rr = idx / TWl, ii = idx - rr * TWl;
          int r = kb + rr, i = i0 + ii;
          cx<T> v = mk<T>(0, 0);
          if (rr < nbk && i >= 0 && i < r) v = lower_elem(Bd, W, kl, ku, false, cj, r, i);
          Ms[idx] = v;
        }
      } else {
        for (int idx = tid; idx < NB * TWl; idx += NT) {
          int ii = idx / NB, rr = idx - ii * NB;
          int r = kb + rr, i = i0 + ii;
          cx<T> v = mk<T>(0, 0);
          if (rr < nbk && i >= 0 && i < r) v = lower_elem(Bd, W, kl, ku, true, cj, r, i);
          Ms[rr * TWl + ii] = v;
        }
      }
      if (tid < nbk) dg[tid] = herm ? cj_if(Bd[(size_t)(kb + tid) * W + kl], !cj) : mk<T>(1, 0);
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        int r = kb + rg + G * s;
        acc[s] = (r < n && cok) ? ccast<T>(Rh[(size_t)r * m + c]) : mk<T>(0, 0);
      }
      __syncthreads();
      const int istart = max(0, i0);
      int slot = istart % RB;
      for (int i = istart; i < kb; ++i) {
        const cx<T> yv = ring[slot * R + col];
#pragma unroll
        for (int s = 0; s < RPT; ++s) cfms(acc[s], Ms[(rg + G * s) * TWl + (i - i0)], yv);
        if (++slot == RB) slot = 0;
      }
      for (int p = 0; p < nbk; ++p) {
        const int rs = (kb + p) % RB;
#pragma unroll
        for (int s = 0; s < RPT; ++s) {
          if (rg + G * s == p) {
            cx<T> v = herm ? cdiv(acc[s], dg[p]) : acc[s];
            ring[rs * R + col] = v;
            Ys[(size_t)(kb + p) * R + col] = v;
          }
        }
        __syncthreads();
        const cx<T> yv = ring[rs * R + col];
#pragma unroll
        for (int s = 0; s < RPT; ++s) {
          int rr = rg + G * s;
          if (rr > p && rr < nbk) cfms(acc[s], Ms[rr * TWl + (kb + p - i0)], yv);
        }
      }
      __syncthreads();
    }
  }
  // ---------------- backward (upper) ----------------
  {
    const int bw = herm ? kl : ku;
    const int TWu = bw + NB;
    const int nblk = ceil_div(n, NB);
    for (int b = nblk - 1; b >= 0; --b) {
      const int kb = b * NB;
      const int nbk = min(NB, n - kb);
      if (!herm) {
        for (int idx = tid; idx < NB * TWu; idx += NT) {
          int rr = idx / TWu, ii = idx - rr * TWu;
          int r = kb + rr, i = kb + ii;
          cx<T> v = mk<T>(0, 0);
          if (rr < nbk && i > r && i < n) v = upper_elem(Bd, W, kl, ku, false, cj, r, i);
          Ms[idx] = v;
        }
      } else {
        for (int idx = tid; idx < NB * TWu; idx += NT) {
          int ii = idx / NB, rr = idx - ii * NB;
          int r = kb + rr, i = kb + ii;
          cx<T> v = mk<T>(0, 0);
          if (rr < nbk && i > r && i < n) v = upper_elem(Bd, W, kl, ku, true, cj, r, i);
          Ms[rr * TWu + ii] = v;
        }
      }
      if (tid < nbk) dg[tid] = herm ? mk<T>(1, 0) : cj_if(Bd[(size_t)(kb + tid) * W + kl], cj);
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        int r = kb + rg + G * s;
        acc[s] = (r < n) ? Ys[(size_t)r * R + col] : mk<T>(0, 0);
      }
      __syncthreads();
      const int iend = min(n, kb + nbk + bw);
      int slot = (kb + nbk) % RB;
      for (int i = kb + nbk; i < iend; ++i) {
        const cx<T> xv = ring[slot * R + col];
#pragma unroll
        for (int s = 0; s < RPT; ++s) cfms(acc[s], Ms[(rg + G * s) * TWu + (i - kb)], xv);
        if (++slot == RB) slot = 0;
      }
      for (int p = nbk - 1; p >= 0; --p) {
        const int rs = (kb + p) % RB;
#pragma unroll
        for (int s = 0; s < RPT; ++s) {
          if (rg + G * s == p) {
            cx<T> v = herm ? acc[s] : cdiv(acc[s], dg[p]);
            ring[rs * R + col] = v;
            if (cok) {
              cxd *xp = Xn + (size_t)(kb + p) * m + c;
              cxd vd = ccast<double>(v);
              *xp = mode ? (*xp + vd) : vd;
            }
          }
        }
        __syncthreads();
        const cx<T> xv = ring[rs * R + col];
#pragma unroll
        for (int s = 0; s < RPT; ++s) {
          int rr = rg + G * s;
          if (rr < p) cfms(acc[s], Ms[rr * TWu + p], xv);
        }
      }
      __syncthreads();
    }
  }
}

// Inverses of the 16 x 16 diagonal blocks of L (unit lower) and U (upper) of
// every node's factors, so that the triangular solves finish each 16-row
// block with a dense product instead of a sequential substitution.  One warp
// per block: lanes 0..15 form column j of L11^{-1}, lanes 16..31 column j of
// U11^{-1}.  Output per (node, block): [L^{-1} | L^{-T} | U^{-1} | U^{-T}],
// so that every solve reads its inverse with consecutive lanes.
constexpr int DIB = 16;
template <typename T>
__device__ __forceinline__ cx<T> band_ld(const cx<T> *B, size_t o) { return B[o]; }
template <typename T>
__global__ void __launch_bounds__(256) k_band_diag_inv(int n, int kl, int ku, const cx<T> *band, size_t ns,
                                                       cx<T> *dinv) {
  __shared__ cx<T> Lb[8][DIB][DIB + 1];
  __shared__ cx<T> Ub[8][DIB][DIB + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblk = ceil_div(n, DIB);
  const int b = blockIdx.x * 8 + warp;
  const int node = blockIdx.y;
  if (b >= nblk) return;
  const int W = kl + ku + 1;
  const cx<T> *Bd = band + (size_t)node * ns;
  const int kb = b * DIB, nbk = min(DIB, n - kb);
  for (int e = lane; e < DIB * DIB; e += 32) {
    const int r = e / DIB, c = e % DIB;
    cx<T> lv = mk<T>(r == c ? 1 : 0, 0), uv = mk<T>(r == c ? 1 : 0, 0);
    if (r < nbk && c < nbk) {
      const int d = c - r;
      if (d < 0 && -d <= kl) lv = band_ld(Bd, (size_t)(kb + r) * W + (d + kl));
      if (d >= 0 && d <= ku) uv = band_ld(Bd, (size_t)(kb + r) * W + (d + kl));
    }
    Lb[warp][r][c] = lv;
    Ub[warp][r][c] = uv;
  }
  __syncwarp();
  const int j = lane & 15;
  cx<T> x[DIB];
  if (lane < 16) {
#pragma unroll
    for (int i = 0; i < DIB; ++i) {
      cx<T> v = mk<T>(i == j ? 1 : 0, 0);
#pragma unroll
      for (int p = 0; p < i; ++p) cfms(v, Lb[warp][i][p], x[p]);
      x[i] = v;
    }
  } else {
#pragma unroll
    for (int i = DIB - 1; i >= 0; --i) {
      cx<T> v = mk<T>(i == j ? 1 : 0, 0);
#pragma unroll
      for (int p = i + 1; p < DIB; ++p) cfms(v, Ub[warp][i][p], x[p]);
      x[i] = cdiv(v, Ub[warp][i][i]);
    }
  }
  // [L^{-1} | L^{-T} | U^{-1} | U^{-T}], each row-major 16 x 16
  cx<T> *out = dinv + ((size_t)node * nblk + b) * (4 * DIB * DIB) + (lane < 16 ? 0 : 2 * DIB * DIB);
#pragma unroll
  for (int i = 0; i < DIB; ++i) {
    out[i * DIB + j] = x[i];
    out[DIB * DIB + j * DIB + i] = x[i];
  }
}

template <typename T>
void launch_band_diag_inv(int n, int kl, int ku, int ne, const cx<T> *band, cx<T> *dinv, cudaStream_t s) {
  const int nblk = ceil_div(n, DIB);
  k_band_diag_inv<T><<<dim3(ceil_div(nblk, 8), ne), 256, 0, s>>>(n, kl, ku, band, (size_t)n * (kl + ku + 1), dinv);
  note_launch();
}
template void launch_band_diag_inv<float>(int, int, int, int, const cxf *, cxf *, cudaStream_t);
size_t band_diag_inv_elems(int n, int ne) { return (size_t)ne * ceil_div(n, DIB) * 4 * DIB * DIB; }

// Smallest and largest pivot modulus |u_rr| over every factor slot.  The
// factorisation does not pivot, so a pivot that is tiny against the largest
// one flags factors that may be inaccurate; the iterative refinement then
// decides whether the solves still reach their tolerance.  Both values go to
// out[0..1] as bits of non-negative doubles (atomicMin / atomicMax on them is
// order-independent); out[0] must start at +inf bits and out[1] at 0.
template <typename T>
__global__ void k_band_pivot_stats(int n, int kl, int ku, int nslots, const cx<T> *__restrict__ band,
                                   unsigned long long *out) {
  const int W = kl + ku + 1;
  const size_t ns = (size_t)n * W;
  double lo = INFINITY, hi = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * nslots;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t slot = e / n, r = e - slot * n;
    const cx<T> u = band[slot * ns + r * W + kl];
    const double a = hypot((double)u.re, (double)u.im);
    const double av = (a == a) ? a : 0.0;  // NaN pivots count as zero
    lo = fmin(lo, av);
    hi = fmax(hi, av);
  }
  for (int o = 16; o; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(out, (unsigned long long)__double_as_longlong(lo));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(hi));
  }
}
__global__ void k_pivot_stats_init(unsigned long long *out) {
  out[0] = (unsigned long long)__double_as_longlong(INFINITY);
  out[1] = 0ull;
}
template <typename T>
void launch_band_pivot_stats(int n, int kl, int ku, int nslots, const cx<T> *band, double *d_out, cudaStream_t s) {
  unsigned long long *o = reinterpret_cast<unsigned long long *>(d_out);
  k_pivot_stats_init<<<1, 1, 0, s>>>(o);
  note_launch();
  k_band_pivot_stats<T><<<grid_for((size_t)n * nslots), 256, 0, s>>>(n, kl, ku, nslots, band, o);
  note_launch();
}
template void launch_band_pivot_stats<float>(int, int, int, int, const cxf *, double *, cudaStream_t);
template void launch_band_pivot_stats<double>(int, int, int, int, const cxd *, double *, cudaStream_t);

// Transposed copy of the factors for the conjugate-transpose solves: row r of
// Bt holds column r of the factored band (lower width ku, upper width kl), so
// that both sides read their tiles along rows.
__global__ void k_band_transpose(int n, int kl, int ku, int nslots, const cxf *__restrict__ B, cxf *__restrict__ Bt) {
  const int W = kl + ku + 1;
  const size_t per = (size_t)n * W, total = per * nslots;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t slot = e / per, rem = e - slot * per;
    const int r = (int)(rem / W), tp = (int)(rem - (size_t)r * W);
    const int i = r - ku + tp;  // Bt(r, tp) = B entry (i, r)
    cxf v = mk(0.f, 0.f);
    if (i >= 0 && i < n) v = B[slot * per + (size_t)i * W + (kl + ku - tp)];
    Bt[e] = v;
  }
}
void launch_band_transpose(int n, int kl, int ku, int nslots, const cxf *B, cxf *Bt, cudaStream_t s) {
  const size_t total = (size_t)n * (kl + ku + 1) * nslots;
  size_t g = (total + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  k_band_transpose<<<(unsigned)g, 256, 0, s>>>(n, kl, ku, nslots, B, Bt);
  note_launch();
}

// FP32 variant.  The band range of each row block is split across the 8 warps
// of the CTA; each lane keeps a 2 x 4 register tile (rows rl+8q, columns
// cl+4t).  The factor tile of the next block is fetched with cp.async into a
// second shared-memory buffer while the current block computes, so the
// global-memory latency is off the critical path.  Partial sums are reduced
// through shared memory and the NB x NB triangle is solved warp-locally (each
// warp owns 2 of the R = 16 columns, one row per lane; rows are finalised in
// order and broadcast with shuffles).
namespace ks {
constexpr int NB = 16, R = 16, WARPS = 16, NT = 32 * WARPS;
constexpr int RED_LD = R + 1;
constexpr int DLD = NB + 1;  // padded row stride of the diagonal-block inverse tile
__host__ __device__ inline int tw_pad(int bw) { return (bw + NB) | 1; }
__host__ __device__ inline int ring_rows(int bw) { return ceil_div(bw + NB, NB) * NB; }
}  // namespace ks

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Issue the copies of one factor tile (and its diagonal) into shared memory.
// Step s < nblk: forward block s; s >= nblk: backward block 2*nblk-1-s.
// N side:  fwd tile (r, i) = L(r, i), i in [kb-kl, r);   diag 1
//          bwd tile (r, i) = U(r, i), i in (r, r+ku];    diag U(r, r)
// H side:  fwd tile (r, i) = U(i, r)^*, i in [kb-ku, r); diag U(r, r)^*
//          bwd tile (r, i) = L(i, r)^*, i in (r, r+kl];  diag 1
// (conjugation is applied when the tile is read)
template <bool HERM>
__device__ __forceinline__ void ks_fetch(const cxf *Bd, const cxf *Dv, int n, int kl, int ku, int W, int nblk,
                                         int step, cxf *Mb, cxf *db, int TWP) {
  using namespace ks;
  const bool fwd = step < nblk;
  const int b = fwd ? step : 2 * nblk - 1 - step;
  const int kb = b * NB;
  const int nbk = min(NB, n - kb);
  const int bw = fwd ? (HERM ? ku : kl) : (HERM ? kl : ku);
  const int TWl = bw + NB;
  const int ibase = fwd ? kb - bw : kb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!HERM) {
    // warp = tile row, lanes along the row (consecutive band entries)
    for (int rr = warp; rr < NB; rr += NT / 32) {
      const int r = kb + rr;
      cxf *dst = Mb + rr * TWP;
      const cxf *srow = Bd + (size_t)r * W + (kl - r);  // srow[i] = band(r, i)
      for (int ii = lane; ii < TWl; ii += 32) {
        const int i = ibase + ii;
        const bool ok = rr < nbk && (fwd ? (i >= 0 && i < r && r - i <= bw) : (i > r && i < n && i - r <= bw));
        cp_async8(dst + ii, ok ? srow + i : Bd, ok);
      }
    }
  } else {
    // half-warp = tile column (one band row i), lanes along the 16 tile rows
    const int rr = lane & 15;
    const int r = kb + rr;
    for (int ii = 2 * warp + (lane >> 4); ii < TWl; ii += NT / 16) {
      const int i = ibase + ii;
      const bool ok = rr < nbk && (fwd ? (i >= 0 && i < r && r - i <= bw) : (i > r && i < n && i - r <= bw));
      cp_async8(Mb + rr * TWP + ii, ok ? Bd + (size_t)i * W + (r - i + kl) : Bd, ok);
    }
  }
  // inverse of the diagonal block: L11^{-1} for N-forward / H-backward,
  // U11^{-1} for N-backward / H-forward (the H sides use its conjugate transpose)
  {
    const bool useL = fwd != HERM;
    const cxf *src = Dv + (size_t)b * (4 * NB * NB) + (useL ? 0 : 2 * NB * NB);
    for (int e = threadIdx.x; e < NB * NB; e += NT) cp_async8(db + (e / NB) * DLD + e % NB, src + e, true);
  }
  cp_async_commit();
}

template <bool HERM, typename Tin>
__device__ __forceinline__ void ks_body(int n, int kl, int ku, const cxf *Bd, const cxf *Dv, const cx<Tin> *Rh,
                                        cxd *Xn, cxf *Ys, int m, int mode, int c0, bool cj,
                                        unsigned char *smem_raw) {
  // conjugate the factor values read from the tiles: HERM (conjugate-transpose
  // solve) and cj (conjugate node) toggle it
  const float vsg = (HERM != cj) ? -1.f : 1.f;
  using namespace ks;
  const int W = kl + ku + 1;
  const int bwmax = max(kl, ku);
  const int TWP = tw_pad(bwmax);
  const int RB = ring_rows(bwmax);
  cxf *Mbuf = reinterpret_cast<cxf *>(smem_raw);      // 2 x NB x TWP
  cxf *ring = Mbuf + (size_t)2 * NB * TWP;             // RB x R
  cxf *red = ring + (size_t)RB * R;                    // WARPS x NB x RED_LD
  cxf *dbuf = red + (size_t)WARPS * NB * RED_LD;       // 2 x NB x DLD (diagonal-block inverse)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rl = lane >> 2, cl = lane & 3;
  const bool owner = warp < R / 2;  // warps that own two columns each for the in-block solve
  const int tc = 2 * (warp % (R / 2)) + (lane >> 4), tr = lane & 15;
  const int gc = c0 + tc;
  const bool cok = owner && gc < m;
  const int nblk = ceil_div(n, NB);
  const int nsteps = 2 * nblk;
  const unsigned full = 0xffffffffu;

  ks_fetch<HERM>(Bd, Dv, n, kl, ku, W, nblk, 0, Mbuf, dbuf, TWP);
  for (int step = 0; step < nsteps; ++step) {
    const bool fwd = step < nblk;
    const int b = fwd ? step : 2 * nblk - 1 - step;
    const int kb = b * NB;
    const int nbk = min(NB, n - kb);
    const int bw = fwd ? (HERM ? ku : kl) : (HERM ? kl : ku);
    const int ibase = fwd ? kb - bw : kb;
    cxf *Ms = Mbuf + (size_t)(step & 1) * NB * TWP;
    cxf *dg = dbuf + (size_t)(step & 1) * NB * DLD;
    // right-hand side of the row this lane finalises
    cxf acc2 = mk(0.f, 0.f);
    {
      const int r = kb + tr;
      if (r < n && cok) acc2 = fwd ? ccast<float>(Rh[(size_t)r * m + gc]) : Ys[(size_t)r * R + tc];
    }
    cp_async_wait_all();
    __syncthreads();
    if (step + 1 < nsteps)
      ks_fetch<HERM>(Bd, Dv, n, kl, ku, W, nblk, step + 1, Mbuf + (size_t)((step + 1) & 1) * NB * TWP,
                     dbuf + (size_t)((step + 1) & 1) * NB * DLD, TWP);
    // ---- GEMM over the rows already solved, split over warps ----
    int hlo, hhi;
    if (fwd) {
      hlo = max(0, kb - bw);
      hhi = kb;
    } else {
      hlo = kb + nbk;
      hhi = min(n, kb + nbk + bw);
    }
    const int len = max(hhi - hlo, 0);
    const int per = ceil_div(len, WARPS);
    const int wlo = hlo + warp * per, whi = min(hhi, wlo + per);
    cxf acc[2][4];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[q][t] = mk(0.f, 0.f);
    if (wlo < whi) {
      int slot = wlo % RB;
#pragma unroll 4
      for (int i = wlo; i < whi; ++i) {
        cxf mv[2], yv[4];
        const int col = i - ibase;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          mv[q] = Ms[(rl + 8 * q) * TWP + col];
          mv[q].im *= vsg;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) yv[t] = ring[slot * R + cl + 4 * t];
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int t = 0; t < 4; ++t) cfma(acc[q][t], mv[q], yv[t]);
        if (++slot == RB) slot = 0;
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int t = 0; t < 4; ++t) red[(warp * NB + rl + 8 * q) * RED_LD + cl + 4 * t] = acc[q][t];
    __syncthreads();
    if (owner) {
      cxf sum = mk(0.f, 0.f);
#pragma unroll
      for (int w = 0; w < WARPS; ++w) sum = sum + red[(w * NB + tr) * RED_LD + tc];
      acc2 = acc2 - sum;
    }
    // ---- in-block solve: x = D acc with D the inverse of the diagonal block ----
    if (owner) {
      cxf x = mk(0.f, 0.f);
#pragma unroll
      for (int p = 0; p < NB; ++p) {
        cxf a;
        a.re = __shfl_sync(full, acc2.re, (lane & 16) | p);
        a.im = __shfl_sync(full, acc2.im, (lane & 16) | p);
        cxf dv;
        dv = HERM ? dg[p * DLD + tr] : dg[tr * DLD + p];
        dv.im *= vsg;
        cfma(x, dv, a);
      }
      acc2 = x;
    }
    // ---- publish the block's solution ----
    if (owner && tr < nbk) {
      const int r = kb + tr;
      ring[(r % RB) * R + tc] = acc2;
      if (fwd) {
        Ys[(size_t)r * R + tc] = acc2;
      } else if (cok) {
        cxd *xp = Xn + (size_t)r * m + gc;
        const cxd vd = ccast<double>(acc2);
        *xp = mode ? (*xp + vd) : vd;
      }
    }
  }
  cp_async_wait_all();
}

template <typename Tin>
__global__ void __launch_bounds__(ks::NT) k_band_solve_ks(int n, int kl, int ku, const cxf *band, size_t bns,
                                                          const cxf *dinv, SolveSides io, size_t rns, int m,
                                                          size_t xns, int mode, cxf *ysc, const int *skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int side = blockIdx.z;
  const int node = blockIdx.y;
  const int c0 = blockIdx.x * ks::R;
  const int slot = io.fmap[node] & 0xffff;
  const bool cj = (io.fmap[node] >> 16) & 1;
  const cxf *Bd = band + (size_t)slot * bns;
  const cx<Tin> *Rh = reinterpret_cast<const cx<Tin> *>(side ? io.rhs[1] : io.rhs[0]) + (size_t)node * rns;
  cxd *Xn = (side ? io.X[1] : io.X[0]) + (size_t)node * xns;
  cxf *Ys = ysc + (((size_t)side * gridDim.y + node) * gridDim.x + blockIdx.x) * (size_t)n * ks::R;
  const cxf *Dv = dinv + (size_t)slot * ceil_div(n, ks::NB) * (4 * ks::NB * ks::NB);
  if (side)
    ks_body<true, Tin>(n, kl, ku, Bd, Dv, Rh, Xn, Ys, m, mode, c0, cj, smem_raw);
  else
    ks_body<false, Tin>(n, kl, ku, Bd, Dv, Rh, Xn, Ys, m, mode, c0, cj, smem_raw);
}

static size_t solve_smem_ks(int kl, int ku) {
  const int bwmax = kl > ku ? kl : ku;
  return ((size_t)2 * ks::NB * ks::tw_pad(bwmax) + (size_t)ks::ring_rows(bwmax) * ks::R +
          (size_t)ks::WARPS * ks::NB * ks::RED_LD + 2 * ks::NB * ks::DLD) * sizeof(cxf);
}

// ---------------------------------------------------------------------------
// FP32 triangular solves with TMA tile loads.  Same block algorithm as above;
// the factor tile of the next 16-row block (two boxes of BX band entries x 16
// rows, from the row-major band for the right side and from its transpose for
// the conjugate-transpose side) and the inverse of its diagonal block are
// fetched by one thread with cp.async.bulk(.tensor) into the other buffer,
// completing on an mbarrier; every thread waits on it with a bounded spin.
// Row stride BX with BX/2 odd keeps the 8 rows read by a warp on distinct
// shared-memory banks.
// ---------------------------------------------------------------------------
struct SolveTma {
  CUtensorMap tmB, tmBt;  // 3D {W, n, slots} maps of the band and its transpose
  int BX;                 // box width (entries), even, BX/2 odd
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *m, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *m, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tm, int x, int y, int z, uint64_t *m) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(m))
      : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *m) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(m))
               : "memory");
}

namespace kt {
constexpr int NB = 16, R = 16, WARPS = 16, NT = 32 * WARPS, OWNERS = R / 2, LSLD = NB + 1;
// owner warps take DELTA fewer window rows each than the other warps, to make
// room for the block solve they do at the start of every step
constexpr int DELTA = 4;
constexpr long long kSpinLimit = 1ll << 26;
__host__ __device__ inline int ring_rows(int bw) { return ceil_div(bw + NB, NB) * NB; }
__host__ __device__ inline size_t smem_bytes(int BX, int bwmax) {
  return (size_t)(2 * 2 * NB * BX + 4 * 256 + 2 * NB * LSLD + ring_rows(bwmax) * R + 2 * WARPS * 256) *
             sizeof(cxf) +
         2 * sizeof(uint64_t);
}
// conflict-free slot of partial sum (row, col) in a warp's 16 x 16 block, for
// both the 4 x 4 lane grid that writes it and the 16-row column that reads it
// ring rows keep column c at 4 (c & 3) + (c >> 2), so that the four columns
// c, c + 4, c + 8, c + 12 a lane multiplies are one 32-byte run
__host__ __device__ inline int rperm(int c) { return ((c & 3) << 2) | (c >> 2); }
__device__ __forceinline__ int rsw(int row, int col) { return row * 16 + (col ^ (((row & 3) << 2) | (row >> 2))); }
// acc += op(a) b and acc -= op(a) b, op = conj when NEG
template <bool NEG> __device__ __forceinline__ void mac(cxf &acc, cxf a, cxf b) {
  if constexpr (NEG)
    cfma_cj(acc, a, b);
  else
    cfma(acc, a, b);
}
template <bool NEG> __device__ __forceinline__ void msc(cxf &acc, cxf a, cxf b) {
  if constexpr (NEG) {
    acc.re = fmaf(-a.re, b.re, acc.re);
    acc.re = fmaf(-a.im, b.im, acc.re);
    acc.im = fmaf(-a.re, b.im, acc.im);
    acc.im = fmaf(a.im, b.re, acc.im);
  } else {
    cfms(acc, a, b);
  }
}
}  // namespace kt

// One CTA: one (node, side, 16 right-hand-side columns) system, forward then
// backward sweep over 16-row blocks.  Step s solves block s of the sweep:
//   y = rhs_s - P_s - Lsub_s x_{s-1},  x_s = D_s y,
// where P_s is the product of the factor rows of block s with the solution
// rows of its window older than block s-1, Lsub_s the factor entries of block
// s in the columns of block s-1, and D_s the inverse of the diagonal block.
// P_{s+1} and Lsub_{s+1} need nothing from block s, so all 16 warps compute
// them during step s (split over window rows) while the 8 owner warps (one
// thread per entry of the 16 x 16 block) first do the short block solve for
// step s: one barrier per step, and the serial part overlaps the product.
template <bool HERM, bool NEG, typename Tin>
__device__ __forceinline__ void kt_body(int n, int klp, int kup, int BX, const CUtensorMap *tm, const cxf *Dv,
                                        const cx<Tin> *Rh, cxd *Xn, cxf *Ys, int m, int mode, int c0, int slot,
                                        int *err, unsigned char *smem_raw) {
  using namespace kt;
  const int lw = HERM ? kup : klp;  // lower width of the band the tiles come from
  const int uw = HERM ? klp : kup;  // upper width
  const int RB = ring_rows(max(lw, uw));
  const int BOXE = NB * BX;
  cxf *Mbuf = reinterpret_cast<cxf *>(smem_raw);  // 2 stages x 2 boxes x BOXE
  cxf *dbuf = Mbuf + (size_t)4 * BOXE;            // 4 stages x 256, p-major inverse
  cxf *Lsub = dbuf + 4 * 256;                     // 2 x NB x LSLD
  cxf *ring = Lsub + 2 * NB * LSLD;               // RB x R solution rows
  cxf *red = ring + (size_t)RB * R;               // 2 x WARPS x 256 partial sums
  uint64_t *mbar = reinterpret_cast<uint64_t *>(red + (size_t)2 * WARPS * 256);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rl = lane >> 2, cl = lane & 3;
  const bool owner = warp < OWNERS;
  const int tc = 2 * (warp % OWNERS) + (lane >> 4), tr = lane & 15;
  const int gc = c0 + tc;
  const bool cok = owner && gc < m;
  const int nblk = ceil_div(n, NB);
  const int nsteps = 2 * nblk;
  const unsigned full = 0xffffffffu;
  const uint32_t tx_bytes = (uint32_t)(2 * BOXE * sizeof(cxf) + 256 * sizeof(cxf));

  auto issue = [&](int j) {
    const bool f = j < nblk;
    const int b = f ? j : 2 * nblk - 1 - j;
    cxf *dst = Mbuf + (size_t)(j & 1) * 2 * BOXE;
    uint64_t *mb = &mbar[j & 1];
    // TMA box origins must be even (16-byte aligned); the forward tile starts 16
    // entries left of the band so that out-of-band entries come in as zeros
    const int x0 = f ? -NB : (lw & ~1);
    // inverse layouts per block: [L^{-1} | L^{-T} | U^{-1} | U^{-T}]; p-major reads
    const int off = HERM ? (f ? 512 : 0) : (f ? 256 : 768);
    mbar_expect_tx(mb, tx_bytes);
    tma_load_3d(dst, tm, x0, b * NB, slot, mb);
    tma_load_3d(dst + BOXE, tm, x0 + BX, b * NB, slot, mb);
    bulk_load(dbuf + (j & 3) * 256, Dv + (size_t)b * 1024 + off, 256 * sizeof(cxf), mb);
  };
  bool timed_out = false;
  int confirmed = -1;  // tiles [0, confirmed] have landed (as seen by this thread)
  auto spin = [&](int j) -> bool {
    long long spins = 0;
    while (!mbar_try_wait(&mbar[j & 1], (uint32_t)((j >> 1) & 1))) {
      if (++spins > kSpinLimit) return false;
    }
    return true;
  };
  auto wait_tile = [&](int j) {
    if (timed_out) return;
    if (spin(j)) {
      confirmed = j;
    } else {
      timed_out = true;
      atomicOr(err, DEVERR_TIMEOUT);
    }
  };
  int issued = -1;  // thread 0: last tile issued
  // right-hand side of step j for this owner thread (0 outside the system)
  auto load_rhs = [&](int j) -> cxf {
    const bool f = j < nblk;
    const int b = f ? j : 2 * nblk - 1 - j;
    const int r = b * NB + tr;
    if (!(r < n && cok)) return mk(0.f, 0.f);
    return f ? ccast<float>(Rh[(size_t)r * m + gc]) : Ys[(size_t)r * R + tc];
  };
  auto load_xold = [&](int j) -> cxd {
    const int b = 2 * nblk - 1 - j;
    const int r = b * NB + tr;
    if (j < nblk || !mode || !(r < n && cok)) return mk(0.0, 0.0);
    return Xn[(size_t)r * m + gc];
  };
  // Lsub_j and P_j for step j from its tile (stage j & 1)
  auto prepare = [&](int j) {
    const bool f = j < nblk;
    const int b = f ? j : 2 * nblk - 1 - j;
    const int kb = b * NB;
    const cxf *Ms = Mbuf + (size_t)(j & 1) * 2 * BOXE;
    cxf *Ls = Lsub + (j & 1) * NB * LSLD;
    // band offset of (row kb + r, column i) relative to the box origin:
    // forward tt = i - (kb + r) + lw + NB (origin -NB), backward
    // tt = i - (kb + r) + (lw & 1) (origin lw rounded down to even)
    const int tbase = f ? lw + NB - kb : (lw & 1) - kb;
    if (tid >= NT - NB * NB) {  // non-owner warps
      const int r = (tid - (NT - NB * NB)) >> 4, p = tid & 15;
      const int i = f ? kb - NB + p : kb + NB + p;  // columns of the previous block of the sweep
      const int d = i - (kb + r);
      cxf v = mk(0.f, 0.f);
      if (i >= 0 && i < n && (f ? d >= -lw : d <= uw)) {
        const int tt = i + tbase - r;
        v = Ms[r * BX + tt + (tt < BX ? 0 : BOXE - BX)];
      }
      Ls[r * LSLD + p] = v;
    }
    // window rows older than the previous block
    int hlo, hhi;
    if (f) {
      hlo = max(0, kb - lw);
      hhi = max(0, kb - NB);
    } else {
      hlo = kb + 2 * NB;
      hhi = min(n, kb + NB + uw);
    }
    const int len = max(hhi - hlo, 0);
    const int per_o = max(0, ceil_div(len + OWNERS * DELTA, WARPS) - DELTA);
    const int per_n = ceil_div(len - OWNERS * per_o, WARPS - OWNERS);
    const int wlo = owner ? hlo + warp * per_o : hlo + OWNERS * per_o + (warp - OWNERS) * per_n;
    const int whi = min(hhi, wlo + (owner ? per_o : per_n));
    cxf acc[2][4];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[q][t] = mk(0.f, 0.f);
    // Segments of [wlo, whi) on which every row of the tile reads the same box
    // and the ring rows are contiguous: plain pointer walks there; the <= 15
    // columns where rows straddle the two boxes pick the box per entry.
    const int e0 = BX - tbase;  // rows r read box 1 from column e0 + r on
    int a = wlo;
    while (a < whi) {
      const int rs = a % RB;
      int b = min(whi, a + (RB - rs));
      const int mode_ = a < e0 ? 0 : (a < e0 + NB - 1 ? 1 : 2);
      b = min(b, mode_ == 0 ? e0 : (mode_ == 1 ? e0 + NB - 1 : b));
      const cxf *py = ring + (size_t)rs * R + 4 * cl;
      if (mode_ != 1) {
        const int off = mode_ == 0 ? 0 : BOXE - BX;
        const cxf *p0 = Ms + rl * BX + (a + tbase - rl) + off;
        const cxf *p1 = Ms + (rl + 8) * BX + (a + tbase - rl - 8) + off;
        const int cnt = b - a;
#pragma unroll 8
        for (int k = 0; k < cnt; ++k) {
          const cxf mv0 = p0[k], mv1 = p1[k];
          const float4 ya = *reinterpret_cast<const float4 *>(py + k * R);
          const float4 yb = *reinterpret_cast<const float4 *>(py + k * R + 2);
          const cxf yv[4] = {mk(ya.x, ya.y), mk(ya.z, ya.w), mk(yb.x, yb.y), mk(yb.z, yb.w)};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            mac<NEG>(acc[0][t], mv0, yv[t]);
            mac<NEG>(acc[1][t], mv1, yv[t]);
          }
        }
      } else {
        for (int i = a; i < b; ++i) {
          cxf mv[2];
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int tt = i + tbase - (rl + 8 * q);
            mv[q] = Ms[(rl + 8 * q) * BX + tt + (tt < BX ? 0 : BOXE - BX)];
          }
          const float4 ya = *reinterpret_cast<const float4 *>(py + (i - a) * R);
          const float4 yb = *reinterpret_cast<const float4 *>(py + (i - a) * R + 2);
          const cxf yv[4] = {mk(ya.x, ya.y), mk(ya.z, ya.w), mk(yb.x, yb.y), mk(yb.z, yb.w)};
#pragma unroll
          for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int t = 0; t < 4; ++t) mac<NEG>(acc[q][t], mv[q], yv[t]);
        }
      }
      a = b;
    }
    cxf *rw = red + ((size_t)(j & 1) * WARPS + warp) * 256;
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int t = 0; t < 4; ++t) rw[rsw(rl + 8 * q, cl + 4 * t)] = acc[q][t];
  };

  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    issue(0);
    issue(1);
    issued = 1;
  }
  wait_tile(0);
  prepare(0);
  __syncthreads();
  cxf rhs_next = owner ? load_rhs(0) : mk(0.f, 0.f);
  cxd xold_next = mk(0.0, 0.0);
  cxf xprev = mk(0.f, 0.f);
  for (int s = 0; s < nsteps; ++s) {
    if (tid == 0 && s + 2 < nsteps && !timed_out) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      issue(s + 2);
      issued = s + 2;
    }
    if (owner) {
      const bool fwd = s < nblk;
      const int b = fwd ? s : 2 * nblk - 1 - s;
      const int kb = b * NB;
      const int nbk = min(NB, n - kb);
      const cxf rhs = rhs_next;
      const cxd xold = xold_next;
      const cxf *rr = red + (size_t)(s & 1) * WARPS * 256 + rsw(tr, tc);
      cxf psum[4];
#pragma unroll
      for (int w = 0; w < 4; ++w) psum[w] = rr[w * 256];
#pragma unroll
      for (int w = 4; w < WARPS; ++w) psum[w & 3] = psum[w & 3] + rr[w * 256];
      cxf y = rhs - ((psum[0] + psum[1]) + (psum[2] + psum[3]));
      const bool has_last = fwd ? s > 0 : s > nblk;
      if (has_last) {
        const cxf *Ls = Lsub + (s & 1) * NB * LSLD + tr * LSLD;
#pragma unroll
        for (int p = 0; p < NB; ++p) {
          cxf a;
          a.re = __shfl_sync(full, xprev.re, (lane & 16) | p);
          a.im = __shfl_sync(full, xprev.im, (lane & 16) | p);
          msc<NEG>(y, Ls[p], a);
        }
      }
      // in-block solve: x = D y, D the inverse of the diagonal block (p-major)
      const cxf *dg = dbuf + (s & 3) * 256;
      cxf x0 = mk(0.f, 0.f), x1 = mk(0.f, 0.f);
#pragma unroll
      for (int p = 0; p < NB; p += 2) {
        cxf a0, a1;
        a0.re = __shfl_sync(full, y.re, (lane & 16) | p);
        a0.im = __shfl_sync(full, y.im, (lane & 16) | p);
        a1.re = __shfl_sync(full, y.re, (lane & 16) | (p + 1));
        a1.im = __shfl_sync(full, y.im, (lane & 16) | (p + 1));
        mac<NEG>(x0, dg[p * NB + tr], a0);
        mac<NEG>(x1, dg[(p + 1) * NB + tr], a1);
      }
      const cxf x = x0 + x1;
      xprev = x;
      if (tr < nbk) {
        const int r = kb + tr;
        ring[(r % RB) * R + rperm(tc)] = x;
        if (fwd) {
          Ys[(size_t)r * R + tc] = x;
        } else if (cok) {
          const cxd vd = ccast<double>(x);
          Xn[(size_t)r * m + gc] = mode ? (xold + vd) : vd;
        }
      }
      // operands of the next step, after the stores above: the first backward
      // step reads the rows the last forward step has just written
      if (s + 1 < nsteps) {
        rhs_next = load_rhs(s + 1);
        xold_next = load_xold(s + 1);
      }
    }
    if (s + 1 < nsteps) {
      wait_tile(s + 1);
      prepare(s + 1);
    }
    __syncthreads();
  }
  // after a timed-out wait, let the copies still in flight land (bounded)
  // before the CTA's shared memory is released
  if (tid == 0 && timed_out)
    for (int j = confirmed + 1; j <= issued; ++j)
      if (!spin(j)) break;
}

template <typename Tin>
__global__ void __launch_bounds__(kt::NT) k_band_solve_tma(int n, int klp, int kup, const __grid_constant__ SolveTma tma,
                                                           const cxf *dinv, SolveSides io, size_t rns, int m,
                                                           size_t xns, int mode, cxf *ysc, int *err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int side = blockIdx.z;
  const int node = blockIdx.y;
  const int c0 = blockIdx.x * kt::R;
  const int slot = io.fmap[node] & 0xffff;
  const bool cj = (io.fmap[node] >> 16) & 1;
  const cx<Tin> *Rh = reinterpret_cast<const cx<Tin> *>(side ? io.rhs[1] : io.rhs[0]) + (size_t)node * rns;
  cxd *Xn = (side ? io.X[1] : io.X[0]) + (size_t)node * xns;
  cxf *Ys = ysc + (((size_t)side * gridDim.y + node) * gridDim.x + blockIdx.x) * (size_t)n * kt::R;
  const cxf *Dv = dinv + (size_t)slot * ceil_div(n, kt::NB) * 1024;
  // the conjugate-transpose side reads conj(factor) entries; a conjugate node
  // reads conj of its partner's factors; both together cancel
  if (side) {
    if (cj)
      kt_body<true, false, Tin>(n, klp, kup, tma.BX, &tma.tmBt, Dv, Rh, Xn, Ys, m, mode, c0, slot, err, smem_raw);
    else
      kt_body<true, true, Tin>(n, klp, kup, tma.BX, &tma.tmBt, Dv, Rh, Xn, Ys, m, mode, c0, slot, err, smem_raw);
  } else {
    if (cj)
      kt_body<false, true, Tin>(n, klp, kup, tma.BX, &tma.tmB, Dv, Rh, Xn, Ys, m, mode, c0, slot, err, smem_raw);
    else
      kt_body<false, false, Tin>(n, klp, kup, tma.BX, &tma.tmB, Dv, Rh, Xn, Ys, m, mode, c0, slot, err, smem_raw);
  }
}

// Tensor maps of a band array (slots x n x W, 8-byte entries) for TMA loads of
// 16-row boxes; BX as above.  Returns false if the band is too wide.
typedef CUresult (*PFN_encodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static PFN_encodeTiled get_encode() {
  static PFN_encodeTiled fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_encodeTiled>(p);
  }
  return fn;
}
int band_tma_box(int klp, int kup) {
  // two boxes must cover: forward tiles [0, lw + 16), backward tiles up to
  // uw + 16 + (lw & 1), for (lw, uw) = (klp, kup) and (kup, klp)
  const int need = ceil_div(max(max(klp, kup) + 16, max(kup + 17 + (klp & 1), klp + 17 + (kup & 1))), 2);
  int bx = need < 2 ? 2 : need;
  while (bx % 4 != 2) ++bx;  // even, bx/2 odd
  return bx;
}
bool band_tma_fits(int klp, int kup) {
  const int bx = band_tma_box(klp, kup);
  return bx <= 254 && kt::smem_bytes(bx, max(klp, kup)) <= 220 * 1024;
}
bool band_tma_make(void *tma_out, int n, int klp, int kup, int nslots, const cxf *band, const cxf *bandT) {
  SolveTma *t = reinterpret_cast<SolveTma *>(tma_out);
  PFN_encodeTiled enc = get_encode();
  if (!enc || !band_tma_fits(klp, kup) || n < 16 || ((klp + kup + 1) & 1) || (klp & 1)) return false;
  t->BX = band_tma_box(klp, kup);
  const cuuint64_t W = (cuuint64_t)(klp + kup + 1);
  const cuuint64_t dims[3] = {W, (cuuint64_t)n, (cuuint64_t)nslots};
  const cuuint64_t strides[2] = {W * 8, W * 8 * (cuuint64_t)n};
  const cuuint32_t box[3] = {(cuuint32_t)t->BX, 16, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  for (int k = 0; k < 2; ++k) {
    CUresult r = enc(k == 0 ? &t->tmB : &t->tmBt, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                     const_cast<cxf *>(k == 0 ? band : bandT), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
  }
  return true;
}
size_t band_tma_bytes() { return sizeof(SolveTma); }

template <typename T>
static size_t solve_smem(int kl, int ku) {
  constexpr int NB = SolveCfg<T>::NB, R = SolveCfg<T>::R;
  int bwmax = kl > ku ? kl : ku;
  int TW = bwmax + NB;
  int RB = ceil_div(bwmax + NB, NB) * NB;
  return ((size_t)NB * TW + (size_t)RB * R + NB) * sizeof(cx<T>);
}

// rhs/X pointers for the two sides are packed by the caller through the
// globals below (set by band_solve_sides).
template <typename T, typename Tin>
cudaError_t band_solve_sides(int n, int kl, int ku, int ne, const int *fmap, const cx<T> *band, const cx<T> *dinv,
                             const cx<Tin> *rhsR, const cx<Tin> *rhsL, size_t rns, int m, cxd *XR, cxd *XL,
                             size_t xns, int mode, cx<T> *ysc, const int *skip, cudaStream_t s, const void *tma,
                             int *err) {
  SolveSides io;
  io.rhs[0] = rhsR;
  io.rhs[1] = rhsL ? rhsL : rhsR;
  io.X[0] = XR;
  io.X[1] = XL ? XL : XR;
  for (int j = 0; j < kMaxNe; ++j) io.fmap[j] = (fmap && j < ne) ? fmap[j] : j;
  const int nsides = (rhsL && XL) ? 2 : 1;
  const size_t bns = (size_t)n * (kl + ku + 1);
  if constexpr (std::is_same<T, float>::value) {
    if (tma) {
      const SolveTma &tm = *reinterpret_cast<const SolveTma *>(tma);
      const size_t smem = kt::smem_bytes(tm.BX, kl > ku ? kl : ku);
      auto kern = k_band_solve_tma<Tin>;
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      dim3 grid(ceil_div(m, kt::R), ne, nsides);
      kern<<<grid, kt::NT, smem, s>>>(n, kl, ku, tm, dinv, io, rns, m, xns, mode, ysc, err);
      note_launch();
      return cudaGetLastError();
    }
    const size_t smem = solve_smem_ks(kl, ku);
    auto kern = k_band_solve_ks<Tin>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(ceil_div(m, ks::R), ne, nsides);
    kern<<<grid, ks::NT, smem, s>>>(n, kl, ku, band, bns, dinv, io, rns, m, xns, mode, ysc, skip);
    note_launch();
  } else {
    constexpr int NB = SolveCfg<T>::NB, R = SolveCfg<T>::R, RPT = SolveCfg<T>::RPT;
    constexpr int NT = R * NB / RPT;
    const size_t smem = solve_smem<T>(kl, ku);
    auto kern = k_band_solve<T, Tin, NB, R, RPT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(ceil_div(m, R), ne, nsides);
    kern<<<grid, NT, smem, s>>>(n, kl, ku, band, bns, io, rns, m, xns, mode, ysc, skip);
    note_launch();
  }
  return cudaGetLastError();
}
template cudaError_t band_solve_sides<float, float>(int, int, int, int, const int *, const cxf *, const cxf *, const cxf *, const cxf *,
                                                    size_t, int, cxd *, cxd *, size_t, int, cxf *, const int *,
                                                    cudaStream_t, const void *, int *);
template cudaError_t band_solve_sides<float, double>(int, int, int, int, const int *, const cxf *, const cxf *, const cxd *, const cxd *,
                                                     size_t, int, cxd *, cxd *, size_t, int, cxf *, const int *,
                                                     cudaStream_t, const void *, int *);
template cudaError_t band_solve_sides<double, double>(int, int, int, int, const int *, const cxd *, const cxd *, const cxd *, const cxd *,
                                                      size_t, int, cxd *, cxd *, size_t, int, cxd *, const int *,
                                                      cudaStream_t, const void *, int *);

template <typename T> size_t band_solve_scratch_elems(int n, int m, int ne) {
  constexpr int R = SolveCfg<T>::R;
  return (size_t)2 * ne * ceil_div(m, R) * (size_t)n * R;
}
template size_t band_solve_scratch_elems<float>(int, int, int);
template size_t band_solve_scratch_elems<double>(int, int, int);

template <typename T> bool band_solve_fits(int kl, int ku) {
  if (std::is_same<T, float>::value) return solve_smem_ks(kl, ku) <= 220 * 1024;
  return solve_smem<T>(kl, ku) <= 220 * 1024;
}
template bool band_solve_fits<float>(int, int);
template bool band_solve_fits<double>(int, int);
