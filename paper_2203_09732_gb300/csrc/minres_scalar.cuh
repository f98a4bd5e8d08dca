// Scalar recurrences of the preconditioned MINRES of Algorithm 2 (Appendix A),
// run on one device thread at the end of a reduction, and the solver's vector
// set. Shared by every solver form (minres.cu, minres_sb.cu).
#pragma once
#include "common.cuh"

namespace hs {

// q_k and q_{k-1} alternate between q0 and q1 by the parity of k, and so do
// d_{k-1} and d_{k-2} between d0 and d1 (see minres.cu).
struct MinresVecs {
  void* q0; void* q1; void* d0; void* d1; void* p; void* x;
};

// minres_sb.cu: the superblock form for long chains (pc: 0 identity, 1 Jacobi,
// 2 row norm). *used = false (and HS_OK) where no superblock plan applies;
// otherwise the solve ran and the state is in hd->h_state, x in v.x.
hs_status minres_solve_sb(hs_handle* hd, const void* b, const MinresVecs& v, hs_dtype dt,
                          int pc, double tol, long long kmax, bool* used);

// Scalar part of pass B (Givens rotation of Algorithm 2), on one thread.
__device__ __forceinline__ void givens_update(MinresState& S, double sumsq) {
  const double bn = sumsq >= 0.0 ? sqrt(sumsq) : NAN;        // beta_{k+1}
  const double a = S.alpha, bk = S.beta;
  const double cp = S.c_prev, sp = S.s_prev, dh = S.delta_hat, eps = S.eps;
  const double delta = cp * dh + sp * a;                     // delta_k
  const double gh = -sp * dh + cp * a;                       // hat gamma_k
  const double eps_n = sp * bn;                              // epsilon_{k+1}
  const double dh_n = cp * bn;                               // hat delta_{k+1}
  const double gamma = sqrt(gh * gh + bn * bn);              // gamma_k
  if (!isfinite(bn) || !isfinite(gamma)) {
    S.status = HS_NONFINITE; S.done = 2; S.pending = 0;
    return;
  }
  if (gamma == 0.0) {
    S.status = HS_BREAKDOWN; S.done = 2; S.pending = 0;
    return;
  }
  const double c = gh / gamma, sn = bn / gamma;              // c_k, s_k
  const double tau = c * S.phi;                              // tau_k
  const double phi = -sn * S.phi;                            // phi_k
  S.cq = 1.0 / (bk * gamma);
  S.cd1 = -delta / gamma;
  S.cd2 = -eps / gamma;
  S.tau = tau;
  S.pending = 1;
  S.beta_prev = bk; S.beta = bn;
  S.delta_hat = dh_n; S.eps = eps_n;
  S.c_prev = c; S.s_prev = sn; S.phi = phi;
  S.k = S.k + 1;
  if (fabs(phi) < S.tol_abs || bn == 0.0 || S.k > S.kmax) S.done = 1;
}

__device__ __forceinline__ void init_state(MinresState& S, double sumsq, double zero_m,
                                           double tol, long long kmax, double sigma) {
  const double beta1 = sumsq >= 0.0 ? sqrt(sumsq) : NAN;     // NaN/Inf propagate
  S.beta_prev = 1.0; S.beta = beta1; S.beta1 = beta1; S.alpha = 0.0;
  S.c_prev = 1.0; S.s_prev = 0.0; S.delta_hat = 0.0; S.eps = 0.0; S.phi = beta1;
  S.tol_abs = tol * beta1; S.cq = S.cd1 = S.cd2 = S.tau = 0.0; S.sigma = sigma;
  S.k = 1; S.kmax = kmax; S.pending = 0; S.pad = 0;
  S.status = zero_m > 0 ? HS_BAD_ARG : (isfinite(beta1) ? HS_OK : HS_NONFINITE);
  S.done = (S.status != HS_OK || beta1 == 0.0 || kmax <= 0 || beta1 < S.tol_abs) ? 2 : 0;
}

}  // namespace hs
