// Shift-invert Lanczos (Algorithm 1) as a stepper, so that one driver can run
// a single chain (hs_lanczos_eigs) and another many chains in lockstep with
// their inner solves batched (sweep.cu): lz_start sets v_1; each step solves
// (H - sigma) x = v_k (the caller's solve writes r.x) and lz_step does the
// rest of the step (three-term recurrence, full reorthogonalisation, Ritz
// estimates); lz_finish extracts and certifies the Ritz pairs.
#pragma once
#include <chrono>
#include <vector>

#include "common.cuh"

namespace hs {

struct LzRun {
  hs_handle* hd = nullptr;
  int K = 0, m = 0;
  double tol = 0.0;
  double* V = nullptr;   // m + 1 basis vectors (device, n each)
  double* x = nullptr;   // the solve's output
  double* w = nullptr;
  double* tmp = nullptr;
  std::vector<double> alpha, beta, h, theta, Y;
  double beta_k = 0.0;   // beta_k multiplying v_{k-1}
  int k = 0;             // current step (0-based): the solve's right-hand side is V + k n
  int steps = 0, nconv = 0;
  bool done = false;
  double solve_s = 0.0;
  long long minres_iters = 0;
  int sweeps = 0, unconverged_solves = 0;
  std::chrono::steady_clock::time_point t0;
  const double* rhs() const { return V + (size_t)k * (size_t)hd->n; }
};

// Checks the arguments, allocates the basis on the handle and sets v_1 (from
// v0_dev, or a seeded N(0,1) vector), normalised.
hs_status lz_start(LzRun& r, hs_handle* hd, int K, int m_max, double tol,
                   unsigned long long seed, const double* v0_dev);
// The rest of step k after its solve (status of the solve, its iterations and
// refinement sweeps); sets r.done when the K pairs converged, the space is
// exhausted or m steps were taken.
hs_status lz_step(LzRun& r, hs_status solve_status, long long iters, int sweeps);
// Ritz pairs of the K largest |theta| ordered by |E - sigma| (ties by E),
// certified in FP64: E = <psi|H|psi> and ||H psi - E psi||.
hs_status lz_finish(LzRun& r, double* evals_host, double* evecs_dev, double* resid_host,
                    hs_lanczos_info* info);

}  // namespace hs
