// Multi-shift residual with per-(node, column) norms that allocates nothing.
//
// Some callers cannot call cudaMalloc: a host application that owns all of
// the device memory through its own pool or memory budget, a latency-bound
// loop where the implicit synchronisation of cudaMalloc/cudaFree is not
// acceptable, or an embedding that must not change its device-memory
// footprint after start-up.  For them this entry point computes, like
// feast_nh_multishift_residual, R_j = B Y - (z_j B - A) X_j and
// Q = sum_j w_j X_j, and in addition ||R_jc||_2 / ||(BY)_c||_2, taking no
// context: its scratch (quadrature nodes, per-CTA partial sums, column norms)
// is the file-scope device array below, which every GPU that loads the
// library holds until the process exits.
#include <cmath>
#include <mutex>

#include "feast_nh.h"
#include "kernels.h"

namespace {

constexpr int kNaMaxGrid = 256;                      // CTAs of the residual kernel
constexpr int kNaMaxPairs = 2048;                    // ne * m
constexpr int kNaColParts = 608;                     // CTAs of the column-norm kernel
// layout (doubles): nodes z, w (2 * 64 complex) | ||BY_c||^2 (128) |
//                   column-norm partials (608 * 128) | residual partials (256 * 2048)
constexpr size_t kNaOffNodes = 0;
constexpr size_t kNaOffBy = kNaOffNodes + 4 * kMaxNe;
constexpr size_t kNaOffCol = kNaOffBy + kMaxM0;
constexpr size_t kNaOffPart = kNaOffCol + (size_t)kNaColParts * kMaxM0;
constexpr size_t kNaDoubles = kNaOffPart + (size_t)kNaMaxGrid * kNaMaxPairs;  // 602,624 doubles, 4.6 MiB

static __device__ __align__(256) double g_noalloc_scratch[kNaDoubles];

std::mutex g_na_mutex;
double *g_na_ptr[64] = {};  // device address of g_noalloc_scratch, per device

// Contour passed to the node kernel by value: the parameters of a circle or
// ellipse, or (kind 2) the caller's nodes and weights themselves (2 KiB at
// most), so that no host buffer has to outlive the call.
struct NaContour {
  int kind, ne;
  double c_re, c_im, r, ratio, angle;
  cxd z[kMaxNe], w[kMaxNe];
};

// zw[0..ne) = nodes, zw[ne..2ne) = weights (trapezoidal rule of Sec. 2.3 for
// kinds 0/1, the caller's values for kind 2).
__global__ void k_na_nodes(NaContour c, cxd *zw) {
  const int j = threadIdx.x;
  if (j >= c.ne) return;
  cxd z, w;
  if (c.kind == 2) {
    z = c.z[j];
    w = c.w[j];
  } else {
    trapezoid_node(c.kind, c.c_re, c.c_im, c.r, c.ratio, c.angle, c.ne, j, z, w);
  }
  zw[j] = z;
  zw[c.ne + j] = w;
}

__global__ void k_na_relres(const double *partial, int nparts, int P, int m, const double *bynorm2, double *relres) {
  const int pair = blockIdx.x * blockDim.x + threadIdx.x;
  if (pair >= P) return;
  double s = 0.0;
  for (int p = 0; p < nparts; ++p) s += partial[(size_t)p * P + pair];
  const double d = bynorm2[pair % m];
  relres[pair] = d > 0 ? sqrt(s / d) : sqrt(s);
}

CsrView na_view(const feast_nh_csr &M) {
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

}  // namespace

extern "C" feast_nh_status feast_nh_multishift_residual_noalloc(const feast_nh_csr *A, const feast_nh_csr *B,
                                                                const feast_nh_contour *contour, const void *X,
                                                                const void *BY, void *R, void *Q, double *relres,
                                                                int32_t m, void *stream) {
  if (!A || !A->rowptr || !A->colind || !A->val || A->n < 1 || A->nnz < 1) return FEAST_NH_EINVAL;
  if (A->dtype != FEAST_NH_R64 && A->dtype != FEAST_NH_C64) return FEAST_NH_EINVAL;
  if (B && (!B->rowptr || !B->colind || !B->val || B->n != A->n || B->nnz < 1 ||
            (B->dtype != FEAST_NH_R64 && B->dtype != FEAST_NH_C64)))
    return FEAST_NH_EINVAL;
  if (!contour || contour->ne < 1 || contour->ne > kMaxNe || contour->kind < 0 || contour->kind > 2 ||
      (contour->kind == 2 && (!contour->z || !contour->w)) || (contour->kind != 2 && !(contour->r > 0)) ||
      (contour->kind == 1 && !(contour->ratio > 0)))
    return FEAST_NH_EINVAL;
  if (!X || !BY || !R || !relres || m < 1 || m > kMaxM0 || contour->ne * m > kNaMaxPairs) return FEAST_NH_EINVAL;
  // an error left pending by the caller's earlier work is not this call's:
  // report it before enqueuing anything, so that later checks see only ours
  if (cudaGetLastError() != cudaSuccess) return FEAST_NH_ECUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FEAST_NH_ECUDA;
  double *base = nullptr;
  {
    // set-up, once per device with that device current: the host-side name
    // of the array is only a stand-in, kernels need its device address
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FEAST_NH_ECUDA;
      g_na_ptr[dev] = static_cast<double *>(p);
    }
    base = g_na_ptr[dev];
  }
  const int ne = contour->ne;
  NaContour nc{};
  nc.kind = contour->kind;
  nc.ne = ne;
  nc.c_re = contour->c_re;
  nc.c_im = contour->c_im;
  nc.r = contour->r;
  nc.ratio = contour->ratio;
  nc.angle = contour->angle;
  if (contour->kind == 2)
    for (int j = 0; j < ne; ++j) {
      nc.z[j] = mk(contour->z[2 * j], contour->z[2 * j + 1]);
      nc.w[j] = mk(contour->w[2 * j], contour->w[2 * j + 1]);
    }
  cxd *dz = reinterpret_cast<cxd *>(base + kNaOffNodes);
  const cxd *dw = dz + ne;
  k_na_nodes<<<1, kMaxNe, 0, s>>>(nc, dz);
  note_launch();
  if (cudaGetLastError() != cudaSuccess) return FEAST_NH_ECUDA;
  const CsrView Av = na_view(*A);
  CsrView Bv;
  if (B) Bv = na_view(*B);
  const int n = A->n;
  // ||(BY)_c||^2: every partial slot used is rewritten by this call
  const int gc = launch_colnorm2((const cxd *)BY, m, m, n, base + kNaOffCol, s);
  launch_reduce_parts(base + kNaOffCol, gc, m, base + kNaOffBy, s);
  if (cudaGetLastError() != cudaSuccess) return FEAST_NH_ECUDA;
  const int gm = launch_multishift_residual_capped<double>(Av, B ? &Bv : nullptr, ne, dz, dw, (const cxd *)X,
                                                           (const cxd *)BY, (cxd *)R, (cxd *)Q, base + kNaOffPart,
                                                           m, kNaMaxGrid, s);
  if (cudaGetLastError() != cudaSuccess) return FEAST_NH_ECUDA;
  const int P = ne * m;
  k_na_relres<<<ceil_div(P, 128), 128, 0, s>>>(base + kNaOffPart, gm, P, m, base + kNaOffBy, relres);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? FEAST_NH_OK : FEAST_NH_ECUDA;
}
