// Launchers of the Rayleigh-Ritz control kernels (rr.cu).
#pragma once
#include "kernels.h"

struct RRStatus {
  int m_tilde, m_r, m_s, m, conv, pad;
  double max_res;
};


// Contour data for the inside test; custom contours carry their nodes.
struct RRParams {
  int kind, ne;
  double c_re, c_im, r, ratio, angle, alpha, eps;
  cxd cz[kMaxNe];
};

void launch_gamma_prep(int m, const cxd *BQ, const cxd *gam, const cxd *V, const cxd *Vinv, const cxd *prev_rho,
                       const int *prev_inside, int have_prev, double mu, double eta, int cs, cxd *S, cxd *Sh,
                       int *ord, RRStatus *st, cudaStream_t s);
void launch_cs_wnorm(int m, const cxd *BU, cxd *W, cxd *Wh, cudaStream_t s);
void launch_rho(int m, int ne, const cxd *z, const cxd *w, const cxd *lam, cxd *rho, cudaStream_t s);
void launch_scale_pairs(cxd *Y, cxd *Yh, const double *nrm2, int m, int n, cudaStream_t s);
void launch_converge(const RRParams &p, int mt, const cxd *lam, const cxd *rho, const double *cn, double *res,
                     int *ord, cxd *prev_rho, int *prev_inside, RRStatus *st, cudaStream_t s);
int launch_colstats(const cxd *Y, const cxd *Yh, const cxd *BY, int m, int n, double *pn, double *pmax, int *pidx,
                    cxd *pval, cxd *pdot, cudaStream_t s);
void launch_finalize(int m, int nparts, const double *pn, const double *pmax, const int *pidx, const cxd *pval,
                     const cxd *pdot, cxd *sx, cxd *sxh, const cxd *Y, const cxd *Yh, int n, const int *ord, int mout,
                     cxd *X, cxd *Xh, int ldo, const cxd *lam, const double *res, double *lam_out, double *res_out,
                     cudaStream_t s);
