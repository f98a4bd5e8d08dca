// Outer loop: nested shift-invert Lanczos (Algorithm 1) with full
// reorthogonalisation, Ritz extraction and FP64 certification; the
// extremal-eigenvalue Lanczos that sets sigma = (E_min + E_max) / 2
// (Sec. IV A); and the host eigensolver of the tridiagonal T_k.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "lanczos.cuh"

namespace hs {

// Symmetric tridiagonal eigenproblem by the implicit QL algorithm with a
// Wilkinson-type shift (Martin & Wilkinson, "The implicit QL algorithm",
// Numer. Math. 12 (1968); the EISPACK routine imtql2), accumulating the plane
// rotations into Y. d: diagonal (overwritten by eigenvalues), e: off-diagonal.
hs_status tridiag_eig(int k, const double* alpha, const double* beta, double* theta, double* Y) {
  std::vector<double> d(alpha, alpha + k), e(k, 0.0);
  for (int i = 0; i + 1 < k; ++i) e[i] = beta[i];
  std::vector<double> Z;
  if (Y) {
    Z.assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) Z[(size_t)i * k + i] = 1.0;  // column-major
  }
  const double eps = std::numeric_limits<double>::epsilon();
  // an off-diagonal entry is negligible relative to its neighbours on the
  // diagonal, or below eps ||T|| (a perturbation no larger than the backward
  // error of the whole reduction; without it a block of zero eigenvalues that
  // carries rounding-level off-diagonals never splits)
  double anorm = 0.0;
  for (int i = 0; i < k; ++i) anorm = std::max(anorm, std::fabs(d[i]) + std::fabs(e[i]));
  for (int l = 0; l < k; ++l) {
    int iter = 0;
    while (true) {
      int m = l;
      for (; m + 1 < k; ++m) {
        const double scale = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (std::fabs(e[m]) <= eps * scale || std::fabs(e[m]) <= eps * anorm) break;
      }
      if (m == l) break;
      if (++iter > 60) return HS_NOT_CONVERGED;
      // shift from the leading 2x2 of the unreduced block
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
      double s = 1.0, c = 1.0, p = 0.0;
      int i = m - 1;
      bool underflow = false;
      for (; i >= l; --i) {
        const double f = s * e[i];
        const double b = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {  // split: recover and restart this block
          d[i + 1] -= p;
          e[m] = 0.0;
          underflow = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
        if (Y) {
          double* zi = &Z[(size_t)i * k];
          double* zj = &Z[(size_t)(i + 1) * k];
          for (int q = 0; q < k; ++q) {
            const double t = zj[q];
            zj[q] = s * zi[q] + c * t;
            zi[q] = c * zi[q] - s * t;
          }
        }
      }
      if (underflow) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  // sort ascending
  std::vector<int> idx(k);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return d[a] < d[b]; });
  for (int i = 0; i < k; ++i) theta[i] = d[idx[i]];
  if (Y)
    for (int i = 0; i < k; ++i)
      std::memcpy(Y + (size_t)i * k, &Z[(size_t)idx[i] * k], sizeof(double) * k);
  return HS_OK;
}

static hs_status ensure_lz(hs_handle* hd, size_t nvec) {
  if (hd->lz_vectors >= nvec) return HS_OK;
  dev_free(hd, hd->lz);
  hd->lz = nullptr;
  hd->lz_vectors = 0;
  if (dev_alloc(hd, (void**)&hd->lz, nvec * sizeof(double) * (size_t)hd->n) != HS_OK)
    return fail(hd, HS_OOM, "Lanczos basis allocation failed");
  hd->lz_vectors = nvec;
  return HS_OK;
}

}  // namespace hs

using namespace hs;

extern "C" hs_status hs_extremal(hs_handle* hd, int max_steps, double tol, double* emin_out,
                                 double* emax_out, double* mid_out) {
  if (!hd) return HS_BAD_ARG;
  if (max_steps <= 0) max_steps = 600;
  max_steps = (int)std::min<long long>(max_steps, hd->n);
  const long long n = hd->n;
  hs_status st = ensure_lz(hd, 3);
  if (st != HS_OK) return st;
  double* v = hd->lz;
  double* vp = hd->lz + n;
  double* w = hd->lz + 2 * n;
  if ((st = vsplitmix(hd, 0x5EEDULL, v, n)) != HS_OK) return st;
  double nn;
  if ((st = vdot(hd, v, v, n, &nn)) != HS_OK) return st;
  if ((st = vscale_to(hd, 1.0 / std::sqrt(nn), v, v, n)) != HS_OK) return st;
  HS_CUDA_TRY(hd, cudaMemsetAsync(vp, 0, sizeof(double) * n, hd->stream));
  std::vector<double> a, b;  // b[j] couples j and j+1
  double bprev = 0.0, lo_old = NAN, hi_old = NAN, lo = 0, hi = 0;
  for (int j = 0; j < max_steps; ++j) {
    if ((st = launch_matvec(hd, v, w, HS_F64, 0)) != HS_OK) return st;
    if ((st = vaxpby(hd, -bprev, vp, 1.0, w, n)) != HS_OK) return st;
    double al;
    if ((st = vdot(hd, v, w, n, &al)) != HS_OK) return st;
    if ((st = vaxpby(hd, -al, v, 1.0, w, n)) != HS_OK) return st;
    double bb;
    if ((st = vdot(hd, w, w, n, &bb)) != HS_OK) return st;
    const double bn = std::sqrt(bb);
    a.push_back(al);
    const bool last = (j + 1 == max_steps) || bn <= 1e-14 * std::fabs(al);
    if ((j + 1) % 10 == 0 || last) {
      std::vector<double> th(a.size());
      if ((st = tridiag_eig((int)a.size(), a.data(), b.data(), th.data(), nullptr)) != HS_OK)
        return fail(hd, st, "tridiagonal eigensolver did not converge");
      lo = th.front();
      hi = th.back();
      if (std::fabs(lo - lo_old) <= tol * std::max(1.0, std::fabs(lo)) &&
          std::fabs(hi - hi_old) <= tol * std::max(1.0, std::fabs(hi)))
        break;
      lo_old = lo;
      hi_old = hi;
    }
    if (last) break;
    b.push_back(bn);
    // vp <- v, v <- w / bn
    HS_CUDA_TRY(hd, cudaMemcpyAsync(vp, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, hd->stream));
    if ((st = vscale_to(hd, 1.0 / bn, w, v, n)) != HS_OK) return st;
    bprev = bn;
  }
  if (emin_out) *emin_out = lo;
  if (emax_out) *emax_out = hi;
  if (mid_out) *mid_out = 0.5 * (lo + hi);
  return HS_OK;
}

namespace hs {

hs_status lz_start(LzRun& r, hs_handle* hd, int K, int m_max, double tol,
                   unsigned long long seed, const double* v0_dev) {
  r = LzRun();
  r.t0 = std::chrono::steady_clock::now();
  r.hd = hd;
  const long long n = hd->n;
  if (K < 1 || K > n) return fail(hd, HS_BAD_ARG, "hs_lanczos_eigs: bad K or output");
  r.K = K;
  r.tol = tol > 0 ? tol : 1e-10;
  int m = m_max > 0 ? m_max : std::max(130, 3 * K + 30);
  m = (int)std::min<long long>(m, n);
  if (m < K) m = K;
  if (m > 500) return fail(hd, HS_BAD_ARG, "m_max > 500");
  if (K * m > 4096 * 8) return fail(hd, HS_BAD_ARG, "K * m too large");
  r.m = m;
  // basis V (m + 1 vectors), x, w, scratch
  hs_status st = ensure_lz(hd, (size_t)m + 4);
  if (st != HS_OK) return st;
  r.V = hd->lz;
  r.x = hd->lz + (size_t)(m + 1) * n;
  r.w = r.x + n;
  r.tmp = r.w + n;
  r.h.assign(m + 1, 0.0);
  double nn;
  if (v0_dev) HS_CUDA_TRY(hd, cudaMemcpyAsync(r.V, v0_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, hd->stream));
  else if ((st = vsplitmix(hd, seed, r.V, n)) != HS_OK) return st;
  if ((st = vdot(hd, r.V, r.V, n, &nn)) != HS_OK) return st;
  if (!(nn > 0) || !std::isfinite(nn)) return fail(hd, HS_BAD_ARG, "start vector is zero or non-finite");
  return vscale_to(hd, 1.0 / std::sqrt(nn), r.V, r.V, n);
}

hs_status lz_step(LzRun& r, hs_status solve_status, long long iters, int sweeps) {
  hs_handle* hd = r.hd;
  const long long n = hd->n;
  const int k = r.k;
  r.minres_iters += iters;
  r.sweeps += sweeps;
  if (solve_status != HS_OK && solve_status != HS_NOT_CONVERGED) return solve_status;
  // a solve that hit its iteration cap feeds an inexact (H - sigma)^-1 v_k
  // into the recurrence; the final FP64 residuals still certify the pairs,
  // and the count is reported
  if (solve_status == HS_NOT_CONVERGED) ++r.unconverged_solves;
  double* V = r.V;
  double* vk = V + (size_t)k * n;
  double* w = r.w;
  hs_status st;
  // w = x - beta_k v_{k-1}; alpha_k = v_k . w; w -= alpha_k v_k
  HS_CUDA_TRY(hd, cudaMemcpyAsync(w, r.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, hd->stream));
  if (k > 0 && (st = vaxpby(hd, -r.beta_k, V + (size_t)(k - 1) * n, 1.0, w, n)) != HS_OK) return st;
  double al;
  if ((st = vdot(hd, vk, w, n, &al)) != HS_OK) return st;
  if ((st = vaxpby(hd, -al, vk, 1.0, w, n)) != HS_OK) return st;
  // full reorthogonalisation against v_1..v_k, two classical Gram-Schmidt passes
  for (int pass = 0; pass < 2; ++pass) {
    if ((st = vmultidot(hd, V, k + 1, w, n, r.h.data())) != HS_OK) return st;
    if ((st = vmultiaxpy(hd, V, k + 1, r.h.data(), w, n)) != HS_OK) return st;
  }
  double bb;
  if ((st = vdot(hd, w, w, n, &bb)) != HS_OK) return st;
  const double bn = std::sqrt(bb);
  r.alpha.push_back(al);
  r.steps = k + 1;
  // Ritz values of T_k and the residual estimates beta_{k+1} |y_{k,i}|
  const int kk = r.steps;
  if (kk >= r.K) {
    r.theta.assign(kk, 0.0);
    r.Y.assign((size_t)kk * kk, 0.0);
    if ((st = tridiag_eig(kk, r.alpha.data(), r.beta.data(), r.theta.data(), r.Y.data())) != HS_OK)
      return fail(hd, st, "tridiagonal eigensolver did not converge");
    std::vector<int> ord(kk);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(),
                     [&](int a, int b) { return std::fabs(r.theta[a]) > std::fabs(r.theta[b]); });
    r.nconv = 0;
    for (int q = 0; q < r.K; ++q) {
      const int i = ord[q];
      const double est = bn * std::fabs(r.Y[(size_t)i * kk + kk - 1]);
      if (est <= r.tol * std::fabs(r.theta[i])) ++r.nconv;
    }
  }
  if (r.nconv == r.K || bn <= 1e-13 * std::fabs(al) || k + 1 == r.m) {
    r.done = true;
    return HS_OK;
  }
  r.beta.push_back(bn);
  if ((st = vscale_to(hd, 1.0 / bn, w, V + (size_t)(k + 1) * n, n)) != HS_OK) return st;
  r.beta_k = bn;
  r.k = k + 1;
  return HS_OK;
}

hs_status lz_finish(LzRun& r, double* evals_host, double* evecs_dev, double* resid_host,
                    hs_lanczos_info* info) {
  using clk = std::chrono::steady_clock;
  hs_handle* hd = r.hd;
  const long long n = hd->n;
  const int K = r.K;
  hs_status st;
  // Ritz pairs: K largest |theta|, then ordered by |E - sigma| (ties by E)
  const auto tr = clk::now();
  const int kk = r.steps;
  if (kk < K) return fail(hd, HS_NOT_CONVERGED, "Lanczos stopped before K steps");
  std::vector<int> ord(kk);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(),
                   [&](int a, int b) { return std::fabs(r.theta[a]) > std::fabs(r.theta[b]); });
  ord.resize(K);
  std::vector<double> Ew(K);
  for (int q = 0; q < K; ++q) Ew[q] = hd->sigma + 1.0 / r.theta[ord[q]];
  std::vector<int> o2(K);
  std::iota(o2.begin(), o2.end(), 0);
  std::stable_sort(o2.begin(), o2.end(), [&](int a, int b) {
    const double da = std::fabs(Ew[a] - hd->sigma), db = std::fabs(Ew[b] - hd->sigma);
    return da != db ? da < db : Ew[a] < Ew[b];
  });
  std::vector<double> Ysel((size_t)K * kk);
  for (int q = 0; q < K; ++q)
    std::memcpy(&Ysel[(size_t)q * kk], &r.Y[(size_t)ord[o2[q]] * kk], sizeof(double) * kk);
  // psi = V_k Y (into evecs_dev, or one vector at a time into tmp)
  double max_res = 0.0;
  double* w = r.w;
  for (int q = 0; q < K; ++q) {
    double* psi = evecs_dev ? evecs_dev + (size_t)q * n : r.tmp;
    if ((st = vritz(hd, r.V, kk, &Ysel[(size_t)q * kk], 1, psi, n)) != HS_OK) return st;
    double pp, pHp, HH;
    if ((st = launch_matvec(hd, psi, w, HS_F64, 0)) != HS_OK) return st;
    if ((st = vdot(hd, psi, psi, n, &pp)) != HS_OK) return st;
    if ((st = vdot(hd, psi, w, n, &pHp)) != HS_OK) return st;
    const double E = pHp / pp;
    // ||H psi - E psi||^2 for unit psi
    if ((st = vscale_to(hd, 1.0 / std::sqrt(pp), psi, psi, n)) != HS_OK) return st;
    if ((st = vaxpby(hd, -E, psi, 1.0 / std::sqrt(pp), w, n)) != HS_OK) return st;
    if ((st = vdot(hd, w, w, n, &HH)) != HS_OK) return st;
    evals_host[q] = E;
    const double res = std::sqrt(std::max(HH, 0.0));
    if (resid_host) resid_host[q] = res;
    max_res = std::max(max_res, res);
  }
  if (info) {
    info->steps = r.steps;
    info->converged = r.nconv;
    info->minres_iters = r.minres_iters;
    info->sweeps = r.sweeps;
    info->unconverged_solves = r.unconverged_solves;
    info->sigma = hd->sigma;
    info->max_resid = max_res;
    info->seconds_solve = r.solve_s;
    info->seconds_total = std::chrono::duration<double>(clk::now() - r.t0).count();
    info->seconds_ritz = std::chrono::duration<double>(clk::now() - tr).count();
  }
  if (r.nconv < K) {
    hd->err = "Lanczos reached m_max before all wanted pairs converged";
    return HS_NOT_CONVERGED;
  }
  return HS_OK;
}

}  // namespace hs

extern "C" hs_status hs_lanczos_eigs(hs_handle* hd, int K, int m_max, double tol,
                                     unsigned long long seed, const double* v0_dev, int mixed,
                                     hs_precond pc, double minres_tol, double inner_tol,
                                     long long minres_kmax, double* evals_host,
                                     double* evecs_dev, double* resid_host,
                                     hs_lanczos_info* info) {
  using clk = std::chrono::steady_clock;
  if (!hd) return HS_BAD_ARG;
  if (!evals_host) return fail(hd, HS_BAD_ARG, "hs_lanczos_eigs: bad K or output");
  if (!(minres_tol > 0)) minres_tol = 1e-12;
  const long long kcap = minres_kmax > 0 ? minres_kmax : 50 * hd->n;
  if (info) std::memset(info, 0, sizeof(*info));
  LzRun r;
  hs_status st = lz_start(r, hd, K, m_max, tol, seed, v0_dev);
  if (st != HS_OK) return st;
  hs_minres_info mi;
  while (!r.done) {
    const auto ts = clk::now();
    std::memset(&mi, 0, sizeof(mi));
    if (mixed) st = minres_mixed(hd, r.rhs(), r.x, minres_tol, kcap, pc, inner_tol > 0 ? inner_tol : 1e-5, &mi);
    else st = minres_solve64(hd, r.rhs(), r.x, minres_tol, kcap, pc, &mi);
    r.solve_s += std::chrono::duration<double>(clk::now() - ts).count();
    if ((st = lz_step(r, st, mi.iters, mixed ? mi.sweeps : 1)) != HS_OK) {
      if (info) { info->minres_iters = r.minres_iters; info->sweeps = r.sweeps; }
      return st;
    }
  }
  return lz_finish(r, evals_host, evecs_dev, resid_host, info);
}

extern "C" hs_status hs_eigs_host(int L, const double* h_host, double sigma, int K, int m_max,
                                  double tol, unsigned long long seed, int mixed, hs_precond pc,
                                  double minres_tol, double inner_tol, long long minres_kmax,
                                  int sm_budget, double* evals_host, double* evecs_host,
                                  double* resid_host, double* z_host, hs_lanczos_info* info) {
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return HS_CUDA;
  }
  hs_handle* hd = nullptr;
  hs_status st = hs_create(L, h_host, sigma, s, &hd);
  if (st != HS_OK) { cudaStreamDestroy(s); return st; }
  hs_set_sm_budget(hd, sm_budget);
  double* ev = nullptr;
  if (dev_alloc(hd, (void**)&ev, sizeof(double) * (size_t)K * hd->n) != HS_OK) {
    hs_free(hd);
    cudaStreamDestroy(s);
    return HS_OOM;
  }
  st = hs_lanczos_eigs(hd, K, m_max, tol, seed, nullptr, mixed, pc, minres_tol, inner_tol,
                       minres_kmax, evals_host, ev, resid_host, info);
  if ((st == HS_OK || st == HS_NOT_CONVERGED) && z_host) {
    hs_status s2 = hs_twist(hd, ev, K, z_host);
    if (s2 != HS_OK) st = s2;
  }
  if ((st == HS_OK || st == HS_NOT_CONVERGED) && evecs_host) {
    if (cudaMemcpyAsync(evecs_host, ev, sizeof(double) * (size_t)K * hd->n,
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      st = HS_CUDA;
    }
  }
  dev_free(hd, ev);
  hs_free(hd);
  cudaStreamDestroy(s);
  return st;
}
