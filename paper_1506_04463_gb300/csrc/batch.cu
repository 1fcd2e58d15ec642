// Contour integration for many independent problems in one persistent launch.
//
// Every problem p has its own sparse A_p (B = I), its own contour (nodes
// z_pj, weights w_pj, j < ne) and its own subspace size m_p <= m0.  One
// cooperative kernel solves, for every problem, node and column at once,
//     (z_pj I - A_p) X_pj = Y_p           (eq. qr)   and then
//     (z_pj I - A_p)^H Xh_pj = Yh_p       (eq. ql),
// and forms Q_p = sum_j w_pj X_pj and Qh_p = sum_j conj(w_pj) Xh_pj (fixed
// node order).  The shifted systems are solved by iterative refinement:
// the residual R = Y - (z I - A) X in FP64 arithmetic, a correction D from
// Jacobi-preconditioned BiCGStab in T (float: the single-precision sweeps;
// double: the plain form, one refinement step), X += D.  The Krylov scalars
// of every (problem, node, column) system are its own; converged systems
// are frozen.  All phases of all refinement steps and Krylov iterations run
// inside the one launch, separated by a grid barrier with a bounded wait.
//
// Layout.  Rows of all problems are concatenated; problem p owns rows
// [off_p, off_p + n_p).  A right-hand-side / output block (Y, Q) holds
// problem p's n_p x m_p row-major block at element offset off_p * m0.  A
// node-major block (X and the Krylov blocks) holds problem p's ne blocks of
// n_p x m_p at element offset ne * off_p * m0: entry (j, i, c) at
// ne*off_p*m0 + (j*n_p + i)*m_p + c.  Work is cut into tiles of consecutive
// rows of one problem; each CTA takes tiles grid-stride, each thread takes
// systems (j, c) and walks the tile's rows, so that a warp reads consecutive
// columns of one row (coalesced) and keeps its partial dot products in
// registers; per-tile partials are reduced per system in fixed tile order.
#include "kernels.h"

namespace {

template <typename T>
__device__ __forceinline__ cx<T> crecip(cx<T> a) {
  // 1/a with one scaling to keep |a|^2 in range
  const T s = fmax(fabs(a.re), fabs(a.im));
  if (!(s > 0)) return mk<T>(0, 0);
  const T ar = a.re / s, ai = a.im / s;
  const T d = ar * ar + ai * ai;
  return mk<T>(ar / (d * s), -ai / (d * s));
}

// grid barrier: arrival counter + generation word; bounded wait
__device__ bool grid_bar(unsigned *bar, int *abort_flag, int *err, long long limit) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned *vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (*(volatile int *)abort_flag) { ok = 0; break; }
        if (clock64() - t0 > limit) {
          atomicOr(err, DEVERR_TIMEOUT);
          atomicExch(abort_flag, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*(volatile int *)abort_flag) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

template <typename T> __device__ __forceinline__ cx<T> ldc(const cx<T> *p, size_t e) { return p[e]; }

}  // namespace

template <typename T>
struct BatchKernelArgs {
  int nprob, ne, m0, ntiles, side0, side1;
  const BatchProb *prob;
  const BatchTile *tiles;
  const cxd *Y, *Yh;
  cxd *Q, *Qh;
  const cxd *diag;       // a_ii per concatenated row
  cxd *X;
  cx<T> *r, *rh, *p, *v, *y, *s, *z, *t, *d;
  cx<T> *part;           // ntiles x 2 x PS partial dots
  double *partd;         // ntiles x PS partial |r|^2 (FP64 residual)
  double *partb;         // ntiles x m0 partial |Y_c|^2
  BatchScal sc;
  unsigned *bar;
  int *ctl;              // [0] abort, [1..4] counters
  BatchStats *stats;
  int *err;
  double tol, tau_min;
  int nsteps, kmax;
  long long spin_limit;
};

namespace {

// Reduce the per-tile partials of every system (fixed tile order).
template <typename T, typename F>
__device__ void for_systems(const BatchKernelArgs<T> &a, F f) {
  const int PS = a.ne * a.m0;
  const int total = a.nprob * PS;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < total; s += gridDim.x * blockDim.x) {
    const int p = s / PS, q = s - p * PS;
    const BatchProb &pr = a.prob[p];
    if (!pr.active) continue;
    const int j = q / a.m0, c = q - j * a.m0;
    if (c >= pr.m || j >= a.ne) continue;
    f(s, p, q, j, c, pr);
  }
}

// Loop over the tiles of active problems; body(tile, problem, j, c, sys, base)
// is called once per (tile, system) for the thread's systems.
template <typename T, bool ONLY_ACTIVE, typename F>
__device__ void for_tile_systems(const BatchKernelArgs<T> &a, F f) {
  const int PS = a.ne * a.m0;
  for (int ti = blockIdx.x; ti < a.ntiles; ti += gridDim.x) {
    const BatchTile tl = a.tiles[ti];
    const BatchProb &pr = a.prob[tl.p];
    if (!pr.active) continue;
    const int m = pr.m;
    const int P = a.ne * m;
    for (int q = threadIdx.x; q < P; q += blockDim.x) {
      const int j = q / m, c = q - j * m;
      const int sys = tl.p * PS + j * a.m0 + c;
      if (ONLY_ACTIVE && !a.sc.act[sys]) continue;
      f(ti, tl, pr, j, c, sys);
    }
  }
}

}  // namespace

template <typename T>
__global__ void __launch_bounds__(512) k_batch_filter(BatchKernelArgs<T> a) {
  const int PS = a.ne * a.m0;
  int *abort_flag = a.ctl;
  for (int side = a.side0; side <= a.side1; ++side) {
    const cxd *BYb = side == 0 ? a.Y : a.Yh;
    cxd *Qb = side == 0 ? a.Q : a.Qh;
    int kry_total = 0, steps_done = 0;
    for (int step = 0;; ++step) {
      // ---- R = BY - (z I - A) X in FP64; Krylov start r = rh = R, d = 0 ----
      for_tile_systems<T, false>(a, [&](int ti, const BatchTile &tl, const BatchProb &pr, int j, int c, int sys) {
        const int n = pr.n, m = pr.m;
        const size_t nb = (size_t)a.ne * pr.off * a.m0 + (size_t)j * n * m;
        const cxd zj = side == 0 ? pr.z[j] : conj(pr.z[j]);
        const CsrView &M = side == 0 ? pr.A : pr.AH;
        const cxd *Xb = a.X + nb;
        const cxd *By = BYb + pr.off * a.m0;
        const bool done = step > 0 && !a.sc.act0[sys];
        double acc2 = 0.0, accb = 0.0;
        for (int i = tl.r0; i < tl.r1; ++i) {
          const cxd b = By[(size_t)i * m + c];
          if (step == 0 && j == 0) accb += abs2(b);
          if (done) continue;
          cxd rr = b;
          if (step > 0) {
            cfms(rr, zj, Xb[(size_t)i * m + c]);
            for (int64_t k = M.rowptr[i]; k < M.rowptr[i + 1]; ++k) cfma(rr, csr_val(M, k), Xb[(size_t)M.colind[k] * m + c]);
          } else {
            a.X[nb + (size_t)i * m + c] = mk(0.0, 0.0);
          }
          const cx<T> ro = ccast<T>(rr);
          a.r[nb + (size_t)i * m + c] = ro;
          a.rh[nb + (size_t)i * m + c] = ro;
          a.d[nb + (size_t)i * m + c] = mk<T>(0, 0);
          acc2 += abs2(rr);
        }
        a.partd[(size_t)ti * PS + j * a.m0 + c] = acc2;
        if (step == 0 && j == 0) a.partb[(size_t)ti * a.m0 + c] = accb;
      });
      if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl[1] = 0;
      if (!grid_bar(a.bar, abort_flag, a.err, a.spin_limit)) return;
      // ---- refinement check: relative residual per system ----
      for_systems(a, [&](int s, int p, int q, int j, int c, const BatchProb &pr) {
        if (step == 0) {
          double b = 0.0;
          for (int ti = pr.tb; ti < pr.te; ++ti) b += a.partb[(size_t)ti * a.m0 + c];
          if (j == 0) a.sc.bn2[p * a.m0 + c] = b;
          a.sc.act0[s] = 1;
        }
        if (!a.sc.act0[s]) { a.sc.act[s] = 0; return; }
        double b = 0.0;
        if (step == 0) {
          for (int ti = pr.tb; ti < pr.te; ++ti) b += a.partb[(size_t)ti * a.m0 + c];
        } else {
          b = a.sc.bn2[p * a.m0 + c];
        }
        double r2 = 0.0;
        for (int ti = pr.tb; ti < pr.te; ++ti) r2 += a.partd[(size_t)ti * PS + q];
        const double rel = b > 0 ? sqrt(r2 / b) : sqrt(r2);
        a.sc.rel[s] = rel;
        if (rel <= a.tol || !(rel == rel) || step >= a.nsteps) {
          a.sc.act0[s] = 0;
          a.sc.act[s] = 0;
          return;
        }
        // Krylov start: rho = (rh, r) = |r|^2; tolerance relative to |r0|
        a.sc.rho[s] = mk(r2, 0.0);
        a.sc.alpha[s] = mk(1.0, 0.0);
        a.sc.omega[s] = mk(1.0, 0.0);
        const double want = 0.5 * a.tol * (b > 0 ? sqrt(b) : 1.0);
        const double tau = fmax(a.tau_min, want / sqrt(r2));
        a.sc.stop2[s] = tau * tau * r2;
        a.sc.act[s] = 1;
        atomicAdd(&a.ctl[1], 1);
      });
      if (!grid_bar(a.bar, abort_flag, a.err, a.spin_limit)) return;
      const int nact = *(volatile int *)&a.ctl[1];
      if (nact == 0 || step >= a.nsteps) { steps_done = step; break; }
      // ---- Jacobi-preconditioned BiCGStab on the active systems ----
      int it = 0;
      for (it = 0; it < a.kmax; ++it) {
        // p = r + beta (p - omega v);  y = K^{-1} p
        for_tile_systems<T, true>(a, [&](int ti, const BatchTile &tl, const BatchProb &pr, int j, int c, int sys) {
          const int n = pr.n, m = pr.m;
          const size_t nb = (size_t)a.ne * pr.off * a.m0 + (size_t)j * n * m;
          const cx<T> beta = ccast<T>(a.sc.beta[sys]);
          const cx<T> om = ccast<T>(a.sc.omega[sys]);
          const cxd zj = side == 0 ? pr.z[j] : conj(pr.z[j]);
          for (int i = tl.r0; i < tl.r1; ++i) {
            const size_t e = nb + (size_t)i * m + c;
            cx<T> pv = a.r[e];
            if (it > 0) {
              cx<T> tmp = a.p[e];
              cfms(tmp, om, a.v[e]);
              cfma(pv, beta, tmp);
            }
            a.p[e] = pv;
            const cxd dg = a.diag[pr.off + i];
            const cx<T> kd = ccast<T>(zj - (side == 0 ? dg : conj(dg)));
            a.y[e] = crecip(kd) * pv;
          }
        });
        if (!grid_bar(a.bar, abort_flag, a.err, a.spin_limit)) return;
        // v = (z I - A) y ;  partial (rh, v)
        for_tile_systems<T, true>(a, [&](int ti, const BatchTile &tl, const BatchProb &pr, int j, int c, int sys) {
          const int n = pr.n, m = pr.m;
          const size_t nb = (size_t)a.ne * pr.off * a.m0 + (size_t)j * n * m;
          const cx<T> zj = ccast<T>(side == 0 ? pr.z[j] : conj(pr.z[j]));
          const CsrView &M = side == 0 ? pr.A : pr.AH;
          const cx<T> *yb = a.y + nb;
          cx<T> dot = mk<T>(0, 0);
          for (int i = tl.r0; i < tl.r1; ++i) {
            cx<T> acc = zj * yb[(size_t)i * m + c];
            for (int64_t k = M.rowptr[i]; k < M.rowptr[i + 1]; ++k) {
              const cx<T> av = ccast<T>(csr_val(M, k));
              cfms(acc, av, yb[(size_t)M.colind[k] * m + c]);
            }
            a.v[nb + (size_t)i * m + c] = acc;
            cfma_cj(dot, a.rh[nb + (size_t)i * m + c], acc);
          }
          a.part[((size_t)ti * 2) * PS + j * a.m0 + c] = dot;
        });
        if (!grid_bar(a.bar, abort_flag, a.err, a.spin_limit)) return;
        // alpha = rho / (rh, v)
        for_systems(a, [&](int s, int p, int q, int j, int c, const BatchProb &pr) {
          if (!a.sc.act[s]) return;
          cxd den = mk(0.0, 0.0);
          for (int ti = pr.tb; ti < pr.te; ++ti) den = den + ccast<double>(a.part[((size_t)ti * 2) * PS + q]);
          if (!(abs2(den) > 0) || !(den.re == den.re)) {
            a.sc.act[s] = 0;  // breakdown: keep the current correction
            return;
          }
          a.sc.alpha[s] = cdiv(a.sc.rho[s], den);
        });
        if (!grid_bar(a.bar, abort_flag, a.err, a.spin_limit)) return;
        // s = r - alpha v;  z = K^{-1} s
        for_tile_systems<T, true>(a, [&](int ti, const BatchTile &tl, const BatchProb &pr, int j, int c, int sys) {
          const int n = pr.n, m = pr.m;
          const size_t nb = (size_t)a.ne * pr.off * a.m0 + (size_t)j * n * m;
          const cx<T> al = ccast<T>(a.sc.alpha[sys]);
          const cxd zj = side == 0 ? pr.z[j] : conj(pr.z[j]);
          for (int i = tl.r0; i < tl.r1; ++i) {
            const size_t e = nb + (size_t)i * m + c;
            cx<T> sv = a.r[e];
            cfms(sv, al, a.v[e]);
            a.s[e] = sv;
            const cxd dg = a.diag[pr.off + i];
            const cx<T> kd = ccast<T>(zj - (side == 0 ? dg : conj(dg)));
            a.z[e] = crecip(kd) * sv;
          }
        });
        if (!grid_bar(a.bar, abort_flag, a.err, a.spin_limit)) return;
        // t = (z I - A) z ;  partial (t, s), (t, t)
        for_tile_systems<T, true>(a, [&](int ti, const BatchTile &tl, const BatchProb &pr, int j, int c, int sys) {
          const int n = pr.n, m = pr.m;
          const size_t nb = (size_t)a.ne * pr.off * a.m0 + (size_t)j * n * m;
          const cx<T> zj = ccast<T>(side == 0 ? pr.z[j] : conj(pr.z[j]));
          const CsrView &M = side == 0 ? pr.A : pr.AH;
          const cx<T> *zb = a.z + nb;
          cx<T> ts = mk<T>(0, 0);
          T tt = 0;
          for (int i = tl.r0; i < tl.r1; ++i) {
            cx<T> acc = zj * zb[(size_t)i * m + c];
            for (int64_t k = M.rowptr[i]; k < M.rowptr[i + 1]; ++k) {
              const cx<T> av = ccast<T>(csr_val(M, k));
              cfms(acc, av, zb[(size_t)M.colind[k] * m + c]);
            }
            a.t[nb + (size_t)i * m + c] = acc;
            cfma_cj(ts, acc, a.s[nb + (size_t)i * m + c]);
            tt += abs2(acc);
          }
          a.part[((size_t)ti * 2) * PS + j * a.m0 + c] = ts;
          a.part[((size_t)ti * 2 + 1) * PS + j * a.m0 + c] = mk<T>(tt, 0);
        });
        if (!grid_bar(a.bar, abort_flag, a.err, a.spin_limit)) return;
        // omega = (t, s) / (t, t)
        for_systems(a, [&](int s, int p, int q, int j, int c, const BatchProb &pr) {
          if (!a.sc.act[s]) return;
          cxd ts = mk(0.0, 0.0);
          double tt = 0.0;
          for (int ti = pr.tb; ti < pr.te; ++ti) {
            ts = ts + ccast<double>(a.part[((size_t)ti * 2) * PS + q]);
            tt += (double)a.part[((size_t)ti * 2 + 1) * PS + q].re;
          }
          a.sc.omega[s] = tt > 0 ? (1.0 / tt) * ts : mk(0.0, 0.0);
        });
        if (!grid_bar(a.bar, abort_flag, a.err, a.spin_limit)) return;
        // d += alpha y + omega z ; r = s - omega t ; partial (rh, r), (r, r)
        for_tile_systems<T, true>(a, [&](int ti, const BatchTile &tl, const BatchProb &pr, int j, int c, int sys) {
          const int n = pr.n, m = pr.m;
          const size_t nb = (size_t)a.ne * pr.off * a.m0 + (size_t)j * n * m;
          const cx<T> al = ccast<T>(a.sc.alpha[sys]);
          const cx<T> om = ccast<T>(a.sc.omega[sys]);
          cx<T> hr = mk<T>(0, 0);
          T rr2 = 0;
          for (int i = tl.r0; i < tl.r1; ++i) {
            const size_t e = nb + (size_t)i * m + c;
            cx<T> dv = a.d[e];
            cfma(dv, al, a.y[e]);
            cfma(dv, om, a.z[e]);
            a.d[e] = dv;
            cx<T> rv = a.s[e];
            cfms(rv, om, a.t[e]);
            a.r[e] = rv;
            cfma_cj(hr, a.rh[e], rv);
            rr2 += abs2(rv);
          }
          a.part[((size_t)ti * 2) * PS + j * a.m0 + c] = hr;
          a.part[((size_t)ti * 2 + 1) * PS + j * a.m0 + c] = mk<T>(rr2, 0);
        });
        if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl[2 + (it & 1)] = 0;
        if (!grid_bar(a.bar, abort_flag, a.err, a.spin_limit)) return;
        // beta = (rho'/rho)(alpha/omega); stop on |r|^2 <= stop2 or breakdown
        for_systems(a, [&](int s, int p, int q, int j, int c, const BatchProb &pr) {
          if (!a.sc.act[s]) return;
          cxd hr = mk(0.0, 0.0);
          double rr2 = 0.0;
          for (int ti = pr.tb; ti < pr.te; ++ti) {
            hr = hr + ccast<double>(a.part[((size_t)ti * 2) * PS + q]);
            rr2 += (double)a.part[((size_t)ti * 2 + 1) * PS + q].re;
          }
          const cxd om = a.sc.omega[s];
          if (!(rr2 > a.sc.stop2[s]) || !(rr2 == rr2) || !(abs2(om) > 0) || !(abs2(a.sc.rho[s]) > 0)) {
            a.sc.act[s] = 0;
            return;
          }
          a.sc.beta[s] = cdiv(hr, a.sc.rho[s]) * cdiv(a.sc.alpha[s], om);
          a.sc.rho[s] = hr;
          atomicAdd(&a.ctl[2 + (it & 1)], 1);
        });
        if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl[2 + ((it + 1) & 1)] = 0;
        if (!grid_bar(a.bar, abort_flag, a.err, a.spin_limit)) return;
        if (*(volatile int *)&a.ctl[2 + (it & 1)] == 0) { ++it; break; }
      }
      kry_total += it;
      // ---- X += D for the systems refined in this step ----
      for_tile_systems<T, false>(a, [&](int ti, const BatchTile &tl, const BatchProb &pr, int j, int c, int sys) {
        if (!a.sc.act0[sys]) return;
        const int n = pr.n, m = pr.m;
        const size_t nb = (size_t)a.ne * pr.off * a.m0 + (size_t)j * n * m;
        for (int i = tl.r0; i < tl.r1; ++i) {
          const size_t e = nb + (size_t)i * m + c;
          const cx<T> dv = a.d[e];
          cxd x = a.X[e];
          x.re += (double)dv.re;
          x.im += (double)dv.im;
          a.X[e] = x;
        }
      });
      if (!grid_bar(a.bar, abort_flag, a.err, a.spin_limit)) return;
    }
    // ---- Q = sum_j w_j X_j (left: conj(w_j)), fixed node order; stats ----
    for (int ti = blockIdx.x; ti < a.ntiles; ti += gridDim.x) {
      const BatchTile tl = a.tiles[ti];
      const BatchProb &pr = a.prob[tl.p];
      if (!pr.active) continue;
      const int n = pr.n, m = pr.m;
      const size_t xb = (size_t)a.ne * pr.off * a.m0;
      for (int c = threadIdx.x; c < m; c += blockDim.x)
        for (int i = tl.r0; i < tl.r1; ++i) {
          cxd qv = mk(0.0, 0.0);
          for (int j = 0; j < a.ne; ++j) {
            const cxd wj = side == 0 ? pr.w[j] : conj(pr.w[j]);
            cfma(qv, wj, a.X[xb + ((size_t)j * n + i) * m + c]);
          }
          Qb[pr.off * a.m0 + (size_t)i * m + c] = qv;
        }
    }
    for_systems(a, [&](int s, int p, int q, int j, int c, const BatchProb &pr) {
      const double rel = a.sc.rel[s];
      const double v = (rel == rel) ? rel : INFINITY;
      atomicMax(&a.stats->maxrel_bits[side], (unsigned long long)__double_as_longlong(v));
      if (!(rel <= a.tol)) atomicAdd(&a.stats->unconverged[side], 1);
    });
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.stats->krylov_its[side] = kry_total;
      a.stats->steps[side] = steps_done;
    }
    if (!grid_bar(a.bar, abort_flag, a.err, a.spin_limit)) return;
  }
}

template <typename T>
static BatchKernelArgs<T> make_args(const BatchLaunch &L) {
  BatchKernelArgs<T> a{};
  a.nprob = L.nprob;
  a.ne = L.ne;
  a.m0 = L.m0;
  a.ntiles = L.ntiles;
  a.side0 = L.side0;
  a.side1 = L.side1;
  a.prob = L.prob;
  a.tiles = L.tiles;
  a.Y = L.Y;
  a.Yh = L.Yh;
  a.Q = L.Q;
  a.Qh = L.Qh;
  a.diag = L.diag;
  a.X = L.X;
  cx<T> *const *kb = reinterpret_cast<cx<T> *const *>(L.kblk);
  a.r = kb[0];
  a.rh = kb[1];
  a.p = kb[2];
  a.v = kb[3];
  a.y = kb[4];
  a.s = kb[5];
  a.z = kb[6];
  a.t = kb[7];
  a.d = kb[8];
  a.part = reinterpret_cast<cx<T> *>(L.part);
  a.partd = L.partd;
  a.partb = L.partb;
  a.sc = L.sc;
  a.bar = L.bar;
  a.ctl = L.ctl;
  a.stats = L.stats;
  a.err = L.err;
  a.tol = L.tol;
  a.tau_min = L.tau_min;
  a.nsteps = L.nsteps;
  a.kmax = L.kmax;
  a.spin_limit = L.spin_limit;
  return a;
}

template <typename T>
int batch_filter_max_ctas_per_sm(int threads) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_filter<T>, threads, 0) != cudaSuccess) nb = 0;
  cudaGetLastError();
  return nb;
}
template int batch_filter_max_ctas_per_sm<float>(int);
template int batch_filter_max_ctas_per_sm<double>(int);

template <typename T>
cudaError_t batch_filter_launch(const BatchLaunch &L, int grid, int threads, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(L.bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(L.ctl, 0, 8 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(L.stats, 0, sizeof(BatchStats), s);
  if (e != cudaSuccess) return e;
  BatchKernelArgs<T> a = make_args<T>(L);
  void *params[] = {&a};
  e = cudaLaunchCooperativeKernel((const void *)k_batch_filter<T>, dim3(grid), dim3(threads), params, 0, s);
  note_launch();
  return e;
}
template cudaError_t batch_filter_launch<float>(const BatchLaunch &, int, int, cudaStream_t);
template cudaError_t batch_filter_launch<double>(const BatchLaunch &, int, int, cudaStream_t);

__global__ void k_csr_diag(CsrView A, cxd *diag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x) {
    cxd d = mk(0.0, 0.0);
    for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k)
      if (A.colind[k] == i) d = d + csr_val(A, k);
    diag[i] = d;
  }
}
void launch_csr_diag(const CsrView &A, cxd *diag, cudaStream_t s) {
  k_csr_diag<<<grid_for((size_t)A.n), 256, 0, s>>>(A, diag);
  note_launch();
}
__global__ void k_fill_pattern(cxd *X, size_t count) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    // a fixed integer hash mapped to [-1, 1]
    unsigned long long h = (e + 1) * 0x9E3779B97F4A7C15ull;
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 29;
    X[e] = mk((double)(h & 0xFFFFF) / 524288.0 - 1.0, (double)((h >> 20) & 0xFFFFF) / 524288.0 - 1.0);
  }
}
void launch_fill_pattern(cxd *X, size_t count, cudaStream_t s) {
  k_fill_pattern<<<grid_for(count), 256, 0, s>>>(X, count);
  note_launch();
}
