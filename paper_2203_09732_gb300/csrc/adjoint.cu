// Derivatives of the twist overlap of an eigenpair with respect to the fields:
// the adjoint (reverse-mode) form of first-order perturbation theory.
//
// For a non-degenerate eigenpair (E, psi) of H, psi real and normalised,
// z = <psi|U_twist|psi> = sum_a psi_a^2 u_a (Sec. III) and dH/dh_j = -Sz_j
// (Eq. (1)), so dpsi/dh_j = (H - E)^+ Sz_j psi, the pseudo-inverse acting on
// the complement of psi. With w = psi * u (element-wise, complex):
//   dz/dh_j = 2 w^T (H - E)^+ Sz_j psi = 2 lambda^T (Sz_j psi),
//   lambda = (H - E)^+ P w,  P = I - psi psi^T,
// i.e. one solve per eigenpair (two real ones, for Re w and Im w) gives all L
// derivatives: (H - E) lambda = P w by the preconditioned MINRES of
// Algorithm 2 with the shift E (consistent: P w is orthogonal to the null
// direction psi), then lambda is projected onto the complement of psi. Then
// d|z|^2/dh_j = 2 Re(conj(z) dz/dh_j); and dE/dh_j = -<psi|Sz_j|psi>
// (Hellmann-Feynman) comes from the same per-site sums.
#include <cmath>
#include <cstring>
#include <vector>

#include "rows.cuh"

namespace hs {

namespace {

struct Roots {
  double re[32], im[32];     // u for t mod L = r, global phase included
};

// w = psi * u_alpha (re, im), u from the bin of t = tlow + thigh mod L.
__global__ void __launch_bounds__(HV_THREADS) k_twist_weight(Geo g, const double* __restrict__ psi,
                                                             Roots u, double* __restrict__ wr,
                                                             double* __restrict__ wi) {
  extern __shared__ __align__(16) char smem[];
  const RowSmem<double> s = row_smem_setup<double>(smem, g);
  const uint32_t L = (uint32_t)g.L;
  const int lane = threadIdx.x & 31;
  for_blocks(g, 0.0, [&](const Hdr& h) {
    for (int r = lane; r < h.C; r += 32) {
      const uint32_t i = h.R + r;
      const uint32_t bin = (le_tlow(s.low[h.off + r].packed) + (uint32_t)h.thigh) % L;
      const double c = psi[i];
      wr[i] = c * u.re[bin];
      wi[i] = c * u.im[bin];
    }
  });
}

constexpr int SITES = LMAX + 1;   // L site sums and the total

// Per-CTA partials of sum_a a_a b_a over the rows with site j up (j < L) and
// over all rows (index L): part[cta * SITES + j]. The state of a row is the
// block's high bits (from the unranked first row of the block) and the low
// pattern of the row.
__global__ void __launch_bounds__(HV_THREADS) k_site_sums(Geo g, const uint32_t* __restrict__ binom,
                                                          const double* __restrict__ a,
                                                          const double* __restrict__ b,
                                                          double* __restrict__ part) {
  extern __shared__ __align__(16) char smem[];
  __shared__ double sacc[HV_WARPS][SITES];
  const RowSmem<double> s = row_smem_setup<double>(smem, g);
  const int L = g.L, N = L / 2, k = g.k;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int W = LMAX / 2 + 2;
  double acc[SITES];
#pragma unroll
  for (int j = 0; j < SITES; ++j) acc[j] = 0.0;
  for_blocks(g, 0.0, [&](const Hdr& h) {
    // the block's high bits: unrank its first row
    uint32_t r0 = h.R, s0 = 0;
    int p = L - 1;
    for (int c = N; c >= 1; --c) {
      while (__ldg(binom + p * W + c) > r0) --p;
      s0 |= 1u << p;
      r0 -= __ldg(binom + p * W + c);
      --p;
    }
    const uint32_t hi = s0 >> k << k;
    for (int r = lane; r < h.C; r += 32) {
      const uint32_t i = h.R + r;
      const double v = a[i] * b[i];
      const uint32_t st = hi | le_pat(s.low[h.off + r].packed);
      acc[SITES - 1] += v;
#pragma unroll
      for (int j = 0; j < LMAX; ++j)
        if ((st >> j) & 1u) acc[j] += v;
    }
  });
  // warp sums, then the CTA's sum in a fixed order
#pragma unroll
  for (int j = 0; j < SITES; ++j) {
    double v = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sacc[wid][j] = v;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < SITES; j += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < HV_WARPS; ++w) t += sacc[w][j];
    part[(size_t)blockIdx.x * SITES + j] = t;
  }
}

// out[j] = sum_a a_a b_a s_j(a) with s_j = +-1/2 (j < L), out[L] = sum_a a_a b_a.
hs_status site_sums(hs_handle* hd, const double* a, const double* b, double* out) {
  const size_t sm = row_smem_bytes<double>((int)hd->low.size());
  if (sm > 48 * 1024)
    HS_CUDA_TRY(hd, cudaFuncSetAttribute(k_site_sums, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm));
  const int grid = row_grid(hd);
  k_site_sums<<<grid, HV_THREADS, sm, hd->stream>>>(hd->geo(), hd->d_binom, a, b, hd->d_partial);
  count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  std::vector<double> host((size_t)grid * SITES);
  HS_CUDA_TRY(hd, cudaMemcpyAsync(host.data(), hd->d_partial, host.size() * sizeof(double),
                                  cudaMemcpyDeviceToHost, hd->stream));
  HS_CUDA_TRY(hd, cudaStreamSynchronize(hd->stream));
  double t[SITES] = {0};
  for (int c = 0; c < grid; ++c)
    for (int j = 0; j < SITES; ++j) t[j] += host[(size_t)c * SITES + j];
  const int L = hd->L;
  for (int j = 0; j < L; ++j) out[j] = t[j] - 0.5 * t[SITES - 1];   // up: +1/2, down: -1/2
  out[L] = t[SITES - 1];
  return HS_OK;
}

}  // namespace

hs_status set_sigma_dev(hs_handle* hd, double sigma);   // api.cu

}  // namespace hs

using namespace hs;

extern "C" hs_status hs_twist_grad(hs_handle* hd, const double* psi_dev, const double* evals_host,
                                   int K, double tol, double* z_host, double* dz2_host,
                                   double* dE_host, hs_minres_info* info) {
  if (!hd) return HS_BAD_ARG;
  if (K < 1 || !psi_dev || !evals_host || !dz2_host)
    return fail(hd, HS_BAD_ARG, "hs_twist_grad: bad arguments");
  for (int q = 0; q < K; ++q)
    if (!std::isfinite(evals_host[q])) return fail(hd, HS_BAD_ARG, "hs_twist_grad: bad eigenvalue");
  if (!(tol > 0)) tol = 1e-10;
  const long long n = hd->n;
  const int L = hd->L;
  hs_status st = ensure_reduce(hd);
  if (st != HS_OK) return st;
  // scratch: unit psi, w_re, w_im, lambda (4 vectors)
  double* ws = nullptr;
  if (dev_alloc(hd, (void**)&ws, sizeof(double) * 4 * (size_t)n) != HS_OK)
    return fail(hd, HS_OOM, "hs_twist_grad: allocation failed");
  double* u = ws;
  double* wr = ws + n;
  double* wi = ws + 2 * n;
  double* lam = ws + 3 * n;
  Roots roots;
  const double ph = -M_PI * (L + 1) / 2.0;
  for (int r = 0; r < 32; ++r) {
    const double a = (r < L ? 2.0 * M_PI * r / L : 0.0) + ph;
    roots.re[r] = std::cos(a);
    roots.im[r] = std::sin(a);
  }
  const double sigma0 = hd->sigma;
  const size_t sm = row_smem_bytes<double>((int)hd->low.size());
  if (info) std::memset(info, 0, sizeof(*info));
  for (int q = 0; q < K && st == HS_OK; ++q) {
    const double* psi = psi_dev + (size_t)q * n;
    double nn;
    if ((st = vdot(hd, psi, psi, n, &nn)) != HS_OK) break;
    if (!(nn > 0)) { st = fail(hd, HS_BAD_ARG, "hs_twist_grad: zero vector"); break; }
    if ((st = vscale_to(hd, 1.0 / std::sqrt(nn), psi, u, n)) != HS_OK) break;
    // z and w = psi * u
    double zz[2];
    if ((st = launch_twist(hd, u, 1, zz)) != HS_OK) break;
    if (z_host) { z_host[2 * q] = zz[0]; z_host[2 * q + 1] = zz[1]; }
    if (sm > 48 * 1024 &&
        cudaFuncSetAttribute(k_twist_weight, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
            cudaSuccess) {
      cudaGetLastError();
      st = fail(hd, HS_CUDA, "hs_twist_grad: shared memory");
      break;
    }
    k_twist_weight<<<row_grid(hd), HV_THREADS, sm, hd->stream>>>(hd->geo(), u, roots, wr, wi);
    count_launches(1);
    if (cudaGetLastError() != cudaSuccess) { st = fail(hd, HS_CUDA, "hs_twist_grad: launch"); break; }
    // Hellmann-Feynman: dE/dh_j = -<psi|Sz_j|psi>
    double sums[LMAX + 1];
    if (dE_host) {
      if ((st = site_sums(hd, u, u, sums)) != HS_OK) break;
      for (int j = 0; j < L; ++j) dE_host[(size_t)q * L + j] = -sums[j];
    }
    // lambda = (H - E)^+ P w for the real and imaginary parts; dz_j = 2 sum lambda s_j psi
    double dz[2][LMAX];
    if ((st = set_sigma_dev(hd, evals_host[q])) != HS_OK) break;
    for (int part = 0; part < 2 && st == HS_OK; ++part) {
      double* w = part ? wi : wr;
      double pw;
      if ((st = vdot(hd, u, w, n, &pw)) != HS_OK) break;
      if ((st = vaxpby(hd, -pw, u, 1.0, w, n)) != HS_OK) break;
      hs_minres_info mi{};
      st = minres_solve64(hd, w, lam, tol, 50 * n, HS_PC_ROWNORM, &mi);
      if (info) { info->iters += mi.iters; info->sweeps += 1; info->phi = std::max(info->phi, mi.phi); }
      if (st == HS_NOT_CONVERGED) { hd->err = "hs_twist_grad: adjoint solve reached its cap"; }
      else if (st != HS_OK) break;
      hs_status keep = st;
      double pl;
      if ((st = vdot(hd, u, lam, n, &pl)) != HS_OK) break;
      if ((st = vaxpby(hd, -pl, u, 1.0, lam, n)) != HS_OK) break;
      if ((st = site_sums(hd, lam, u, sums)) != HS_OK) break;
      for (int j = 0; j < L; ++j) dz[part][j] = 2.0 * sums[j];
      if (keep == HS_NOT_CONVERGED) st = keep;
    }
    if (st != HS_OK && st != HS_NOT_CONVERGED) break;
    // d|z|^2/dh_j = 2 Re(conj(z) dz_j)
    for (int j = 0; j < L; ++j)
      dz2_host[(size_t)q * L + j] = 2.0 * (zz[0] * dz[0][j] + zz[1] * dz[1][j]);
    if (st == HS_NOT_CONVERGED) break;
  }
  const hs_status st2 = set_sigma_dev(hd, sigma0);
  dev_free(hd, ws);
  if (info) info->status = st;
  if (st == HS_OK && st2 != HS_OK) st = st2;
  return st;
}
