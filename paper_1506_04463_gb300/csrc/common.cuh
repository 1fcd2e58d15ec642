// Shared device/host helpers for the FEAST non-Hermitian CUDA path (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#define HD __host__ __device__ __forceinline__

template <typename T>
struct __align__(2 * sizeof(T)) cx {
  T re, im;
};
using cxd = cx<double>;
using cxf = cx<float>;

template <typename T> HD cx<T> mk(T r, T i) { cx<T> z; z.re = r; z.im = i; return z; }
template <typename T> HD cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T> HD cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T> HD cx<T> operator-(cx<T> a) { return mk(-a.re, -a.im); }
template <typename T> HD cx<T> operator*(cx<T> a, cx<T> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T> HD cx<T> operator*(T s, cx<T> a) { return mk(s * a.re, s * a.im); }
template <typename T> HD cx<T> conj(cx<T> a) { return mk(a.re, -a.im); }
template <typename T> HD T abs2(cx<T> a) { return a.re * a.re + a.im * a.im; }
template <typename T> HD T cabs(cx<T> a) { return hypot(a.re, a.im); }
// acc += a*b
template <typename T> HD void cfma(cx<T> &acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc -= a*b
template <typename T> HD void cfms(cx<T> &acc, cx<T> a, cx<T> b) {
  acc.re = fma(-a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(-a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}
// acc += conj(a)*b
template <typename T> HD void cfma_cj(cx<T> &acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}
template <typename T> HD cx<T> cdiv(cx<T> a, cx<T> b) {
  // Smith's algorithm
  if (fabs(b.re) >= fabs(b.im)) {
    T r = b.im / b.re, d = b.re + r * b.im;
    return mk((a.re + r * a.im) / d, (a.im - r * a.re) / d);
  } else {
    T r = b.re / b.im, d = b.im + r * b.re;
    return mk((a.re * r + a.im) / d, (a.im * r - a.re) / d);
  }
}
template <typename To, typename Ti> HD cx<To> ccast(cx<Ti> a) { return mk((To)a.re, (To)a.im); }

// Principal square root.
HD cxd csqrt(cxd a) {
  double r = hypot(a.re, a.im);
  if (r == 0.0) return mk(0.0, 0.0);
  double t = sqrt(0.5 * (r + fabs(a.re)));
  if (a.re >= 0) return mk(t, a.im / (2 * t));
  return mk(fabs(a.im) / (2 * t), a.im >= 0 ? t : -t);
}

// Trapezoidal rule on a circle (kind 0) or ellipse (kind 1), Sec. 2.1 / 2.3:
// node j (0-based) at t = pi(2j+1)/ne, z = c + e^{i phi}(a cos t + i b sin t),
// b = ratio*a, and weight w = z'(t)/(i ne) = e^{i phi}(b cos t + i a sin t)/ne.
// Shared by the host setup of a context and by the device-side node kernel of
// the allocation-free entry point.
HD void trapezoid_node(int kind, double c_re, double c_im, double a, double ratio, double phi_in, int ne, int j,
                       cx<double> &z, cx<double> &w) {
  const double b = a * (kind == 0 ? 1.0 : ratio);
  const double phi = kind == 0 ? 0.0 : phi_in;
  const double cp = cos(phi), sp = sin(phi);
  const double th = 3.14159265358979323846 * (2.0 * j + 1.0) / ne;
  const double ct = cos(th), st = sin(th);
  const double xr = a * ct, xi = b * st;
  z = mk(c_re + cp * xr - sp * xi, c_im + sp * xr + cp * xi);
  const double wr = b * ct, wi = a * st;
  w = mk((cp * wr - sp * wi) / ne, (sp * wr + cp * wi) / ne);
}

// CSR view of a caller-owned matrix (device pointers).  `cplx` selects
// interleaved complex values; `conj_vals` conjugates them on read (used with
// a transposed CSR to apply A^H).
struct CsrView {
  int n;
  int64_t nnz;
  const int32_t *rowptr;
  const int32_t *colind;
  const double *val;
  int cplx;
  int conj_vals;
};

__device__ __forceinline__ cxd csr_val(const CsrView &M, int64_t k) {
  if (M.cplx) {
    cxd v = reinterpret_cast<const cxd *>(M.val)[k];
    if (M.conj_vals) v.im = -v.im;
    return v;
  }
  return mk(M.val[k], 0.0);
}

// Device error word bits.
enum : int { DEVERR_ZERO_PIVOT = 1, DEVERR_QR_NOCONV = 2, DEVERR_SINGULAR_SMALL = 4, DEVERR_BAD_INDEX = 8,
             DEVERR_TIMEOUT = 16 };

constexpr int kMaxNe = 64;     // quadrature nodes
constexpr int kMaxM0 = 128;    // subspace size

__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Process-wide count of kernels this library launched (feast_nh_kernel_launches).
void note_launch();

// Grid size for a grid-stride loop over `count` elements with 256 threads.
inline unsigned grid_for(size_t count) {
  size_t g = (count + 255) / 256;
  if (g > 4096) g = 4096;
  return (unsigned)(g < 1 ? 1 : g);
}
