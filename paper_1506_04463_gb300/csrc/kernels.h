// Internal launchers shared between the translation units of the library.
#pragma once
#include "common.cuh"

// ---------------- band.cu : banded LU of (z_j B - A) -----------------------
// Row-major band storage: node j, row r, offset t in [0, W), W = kl+ku+1,
// holds entry (r, r - kl + t) of the matrix / of its L (t < kl) and U (t >= kl)
// factors.
void launch_band_extent(const CsrView &A, const CsrView *B, int *d_out, cudaStream_t s);
template <typename T>
void launch_band_build(const CsrView &A, const CsrView *B, int kl, int ku, int ne, const cxd *d_z,
                       cx<T> *band, cudaStream_t s);
template <typename T>
cudaError_t band_factor(int n, int kl, int ku, int ne, cx<T> *band, int *d_err, cudaStream_t s);
// Solve with the factors of every node at once, right side (LU) x = b and,
// if rhsL/XL are given, left side (LU)^H x = b in the same launch.  rhs:
// node-major blocks (or one shared block when rns == 0) of n x m with row
// stride m, element type Tin.  X (double complex, node stride xns) gets the
// solution (mode 0) or has it added (mode 1).  Skipped when *skip != 0.
// fmap (host, ne entries, NULL: identity): node j uses factor slot fmap[j] &
// 0xffff, conjugated when bit 16 is set.
// tma (FP32 only, may be NULL): tensor maps from band_tma_make; err: device
// error word (DEVERR_TIMEOUT if a bounded wait gave up).
template <typename T, typename Tin>
cudaError_t band_solve_sides(int n, int kl, int ku, int ne, const int *fmap, const cx<T> *band, const cx<T> *dinv,
                             const cx<Tin> *rhsR, const cx<Tin> *rhsL, size_t rns, int m, cxd *XR, cxd *XL,
                             size_t xns, int mode, cx<T> *ysc, const int *skip, cudaStream_t s,
                             const void *tma = nullptr, int *err = nullptr);
// TMA tile loads for the FP32 solves: tensor maps of the band and of its
// transpose (opaque buffer of band_tma_bytes()); false if not available.
bool band_tma_fits(int klp, int kup);
bool band_tma_make(void *tma_out, int n, int klp, int kup, int nslots, const cxf *band, const cxf *bandT);
size_t band_tma_bytes();
void launch_band_transpose(int n, int kl, int ku, int nslots, const cxf *B, cxf *Bt, cudaStream_t s);
template <typename T> size_t band_solve_scratch_elems(int n, int m, int ne);
// Inverses of the 16 x 16 diagonal blocks of L and U (FP32 solve path).
template <typename T>
void launch_band_diag_inv(int n, int kl, int ku, int ne, const cx<T> *band, cx<T> *dinv, cudaStream_t s);
size_t band_diag_inv_elems(int n, int ne);
// Smallest / largest pivot modulus over all factor slots -> d_out[0], d_out[1].
template <typename T>
void launch_band_pivot_stats(int n, int kl, int ku, int nslots, const cx<T> *band, double *d_out, cudaStream_t s);
template <typename T> bool band_fits(int kl, int ku);
template <typename T> bool band_solve_fits(int kl, int ku);

// ---------------- spmm.cu : sparse products --------------------------------
// Q = sum_j w_j X_j over the node-major blocks X; complex128 -> complex64 copy
void launch_node_sum(int ne, const cxd *d_w, const cxd *X, size_t xns, int n, int m, cxd *Q, cudaStream_t s);
void launch_to_cxf(const cxd *X, cxf *Y, size_t count, cudaStream_t s);
// R_j = BY - (z_j B - A) X_j for all nodes j (node-major X, R), optional
// Q = sum_j w_j X_j, per-CTA partial sums of |R_j,c|^2 into partial
// [gridDim][ne*m].  Returns the grid size used (for the reduction).
template <typename Tout>
int launch_multishift_residual(const CsrView &A, const CsrView *B, int ne, const cxd *d_z, const cxd *d_w,
                               const cxd *X, const cxd *BY, cx<Tout> *R, cxd *Q, double *partial, int m,
                               const int *d_skip, cudaStream_t s);
// As above with at most max_grid CTAs (partial holds max_grid * ne * m doubles).
template <typename Tout>
int launch_multishift_residual_capped(const CsrView &A, const CsrView *B, int ne, const cxd *d_z, const cxd *d_w,
                                      const cxd *X, const cxd *BY, cx<Tout> *R, cxd *Q, double *partial, int m,
                                      int max_grid, cudaStream_t s);
// Reduce the partial sums into relative residuals ||R_jc|| / ||BY_c|| and set
// *d_done = 1 when all are <= tol.  bynorm2[c] = ||BY_c||^2.  nsides blocks of
// partials (each nparts x ne*m) and of bynorm2 (each m) are checked together.
void launch_residual_check(const double *partial, int nparts, int ne, int m, const double *bynorm2, int nsides,
                           double tol, double *d_maxrel, int *d_done, cudaStream_t s);
// FP32 multi-shift operator V_j = (z_j B - A) P_j (conj_z: conj(z_j), for the
// conjugate-transpose CSR pair) over node-major complex-float blocks; returns
// the grid used.  grid_per_sm <= 0: 8 CTAs of 256 threads per SM.
// max_row_nnz: longest row of A (launch_max_row_nnz), selects the register row length.
int launch_multishift_spmm_f32(const CsrView &A, const CsrView *B, int ne, const cxd *d_z, int conj_z, const cxf *P,
                               cxf *V, int m, int grid_per_sm, int max_row_nnz, cudaStream_t s);
void launch_max_row_nnz(const CsrView &A, int *d_out, cudaStream_t s);
// Out = M1 X - shift_c (M2 X)  (M2 == NULL: identity), row-major n x m blocks.
// If p1/p2 != NULL, per-CTA partial column 1-norms of Out and of (M2 X).
int launch_spmm(const CsrView &M1, const CsrView *M2, const cxd *shift, const cxd *X, cxd *Out, int m,
                double *p1, double *p2, cudaStream_t s);
// Largest grid the sparse kernels use (8 CTAs per SM).
int spmm_max_grid();
// Column reductions of partial arrays [nparts][m] -> out[m] (fixed order).
void launch_reduce_parts(const double *parts, int nparts, int m, double *out, cudaStream_t s);
// Transposed CSR (deterministic: entries of each row ordered by column).
cudaError_t csr_transpose(const CsrView &A, int32_t *rowptr_t, int32_t *colind_t, double *val_t,
                          int32_t *work, cudaStream_t s);

// ---------------- krylov.cu : batched BiCGStab ------------------------------
size_t krylov_work_bytes(int n, int m0, int ne);
int krylov_bicgstab(const CsrView &A, const CsrView *B, int ne, const cxd *d_z, const cxd *d_w, const cxd *BY, int m,
                    int m0, double tol, int max_it, void *work, cxd *Xout, double *maxrel, cudaStream_t s);

// ---------------- batch.cu : many problems in one persistent launch --------
constexpr int kBatchMaxNe = 16;
// One problem of a batch (device array).  A and AH: its CSR and conjugate
// transpose with local column indices; rows [off, off + n) of the
// concatenated row space; m columns per node; tiles [tb, te).
struct BatchProb {
  CsrView A, AH;
  size_t off;
  int n, m, active, tb, te, pad;
  cxd z[kBatchMaxNe], w[kBatchMaxNe];
};
struct BatchTile {
  int p, r0, r1, pad;
};
// Per-system state (nprob * ne * m0 entries each).
struct BatchScal {
  cxd *rho, *alpha, *omega, *beta;
  double *bn2;    // ||Y_c||^2 per (problem, column): nprob * m0
  double *rel;    // relative residual of the last refinement check
  double *stop2;  // Krylov stopping threshold on |r|^2
  int *act;       // iterating in the current Krylov solve
  int *act0;      // not yet refined to tolerance
};
struct BatchStats {
  unsigned long long maxrel_bits[2];
  int unconverged[2];
  int krylov_its[2];
  int steps[2];
};
struct BatchLaunch {
  int nprob, ne, m0, ntiles, side0, side1;
  const BatchProb *prob;
  const BatchTile *tiles;
  const cxd *Y, *Yh;
  cxd *Q, *Qh;
  const cxd *diag;
  cxd *X;
  void *kblk[9];   // r, rh, p, v, y, s, z, t, d in the Krylov precision
  void *part;
  double *partd, *partb;
  BatchScal sc;
  unsigned *bar;
  int *ctl;
  BatchStats *stats;
  int *err;
  double tol, tau_min;
  int nsteps, kmax;
  long long spin_limit;
};
// Cooperative launch of the batched contour integration in precision T
// (float: FP32 Krylov sweeps + FP64 refinement; double: plain FP64).
template <typename T>
cudaError_t batch_filter_launch(const BatchLaunch &L, int grid, int threads, cudaStream_t s);
template <typename T> int batch_filter_max_ctas_per_sm(int threads);
// diag[i] = A_ii (sum of the stored diagonal entries of row i).
void launch_csr_diag(const CsrView &A, cxd *diag, cudaStream_t s);
// Deterministic fill of a block with values in [-1, 1] (autotuning input).
void launch_fill_pattern(cxd *X, size_t count, cudaStream_t s);

// ---------------- fgmres.cu : batched flexible GMRES (FP32) -----------------
// The operator (y = (z_j B - A) x for every node, node-major complex-float
// blocks) and the right preconditioner (z ~ (z_j B - A)^{-1} v), supplied by
// the caller.
struct FgmresOp {
  void *ctx;
  void (*apply)(void *ctx, const cxf *x, cxf *y, cudaStream_t s);
  void (*precond)(void *ctx, const cxf *v, cxf *z, cudaStream_t s);
};
size_t fgmres_work_bytes(int n, int m0, int ne, int kmax);
// Solves op(d) = b for every (node, column) system to |b - op d| <= tol |b|
// (or maxit iterations) with restart length kmax; d (node-major, complex
// float) is overwritten.  Returns the iterations done; *maxrel gets the
// largest true relative residual.
int fgmres_solve(const FgmresOp &op, const cxf *b, cxf *d, int n, int m, int ne, int m0, int kmax, int maxit,
                 double tol, void *work, double *maxrel, cudaStream_t s);
void launch_fg_jacobi(const cxf *v, const cxd *zn, int conj_z, const cxd *adiag, const cxd *bdiag, cxf *z, int ne,
                      int n, int m, cudaStream_t s);

void launch_cxf_accumulate(cxd *X, const cxf *d, size_t count, int mode, cudaStream_t s);
void launch_broadcast_cxf(const cxd *BY, cxf *out, size_t nm, int ne, cudaStream_t s);

// ---------------- net.cu : the learned preconditioner's network ----------------
struct feast_nh_net;
// z = network(v) for all ne*m systems of a node-major complex-float block on
// the net's N x N grid (n = N^2); part/rms: scratch of
// net_precondition_scratch_floats floats.
int net_precondition(feast_nh_net *net, const cxf *v, cxf *z, int ne, int n, int m, const cxd *zn, int conj_z,
                     float kappa, const float *feat, int nfeat, float *part, float *rms, cudaStream_t s);
size_t net_precondition_scratch_floats(int n, int ne, int m);
int *net_error_word(feast_nh_net *n);
// Training pairs for the network from node solutions X (node-major) of R.
void launch_learned_pairs(const cxd *R, const cxd *X, int ne, int n, int m, const cxd *z, float kappa,
                          const float *feat, int nfeat, const double *rn2, float *Xin, float *T, cudaStream_t s);
// Operator-norm loss || (z_j I - A)(out - T) ||^2 of network output images and its gradient.
void launch_operator_loss(const CsrView &M, const CsrView &MH, int ne, int n, int m, const cxd *z, int side,
                          const float *out, const float *T, float *ybuf, float *gout, double *loss, cudaStream_t s);

// ---------------- dense.cu : tall-skinny and small dense kernels -----------
// G = X^H Y (mx x my), X: n x mx (ld ldx), Y: n x my (ld ldy); partial buffer
// of size nchunks*mx*my complex.
void gram(const cxd *X, int ldx, int mx, const cxd *Y, int ldy, int my, int n, cxd *G, cxd *partial,
          int nchunks, cudaStream_t s);
int gram_chunks(int n);
// The same products on the tensor cores, FP64-accurate (exact digit products,
// csrc/proj.cu).  FXY: 2 * kMaxM0 ints of scratch; part: at least
// gram_tc_part_bytes(nchunks, mx, my) bytes; err: device error word.
void gram_tc(const cxd *X, int ldx, int mx, const cxd *Y, int ldy, int my, int n, cxd *G, long long *part,
             int nchunks, int *FXY, int *err, cudaStream_t s);
int gram_tc_chunks(int n, int mx, int my);
size_t gram_tc_part_bytes(int nchunks, int mx, int my);
size_t gram_tc_part_max(int n);
void block_tc(const cxd *X, int ldx, int mx, const cxd *S, int lds, int mz, int n, cxd *Z, int ldz, int *err,
              cudaStream_t s);
// Z (n x mz, ld ldz) = X (n x mx, ld ldx) * S (mx x mz, row-major, ld lds)
void block_times_small(const cxd *X, int ldx, int mx, const cxd *S, int lds, int mz, int n, cxd *Z, int ldz,
                       cudaStream_t s);
// Column 2-norms^2 partials of a row-major block.
int launch_colnorm2(const cxd *X, int ld, int m, int n, double *partial, cudaStream_t s);
void launch_copy_conj(const cxd *X, cxd *Y, size_t count, cudaStream_t s);
void launch_broadcast_block(const cxd *X, cxd *Y, size_t count, int copies, cudaStream_t s);

// *d_err |= bits (host-side fault injection through the device error word).
void launch_or_bits(int *d_err, int bits, cudaStream_t s);

// Small single-CTA work on m x m matrices in global memory (row-major).
void small_eig(const cxd *A, int m, cxd *lam, cxd *V, cxd *work, int *d_err, cudaStream_t s);
void small_inv(const cxd *A, int m, cxd *Ainv, cxd *work, int *d_err, cudaStream_t s);
// C = op(A) * op(B), all m x m (or general k), op: 0 none, 1 conj-transpose.
void small_mm(const cxd *A, int opA, const cxd *B, int opB, cxd *C, int m, int k, int n, cudaStream_t s);

