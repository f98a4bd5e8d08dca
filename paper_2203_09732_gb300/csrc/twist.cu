// Twist overlap z = <psi| U_twist |psi>, U_twist = exp[i 2pi/L sum_j j Sz_j]
// (Sec. III). In the Sz basis U is diagonal with u_alpha = exp(i 2pi/L (t - L(L+1)/4)),
// t = sum of the (1-based) sites that are up, so
//   z = exp(-i pi (L+1)/2) sum_{r=0}^{L-1} W_r exp(i 2pi r / L),
//   W_r = sum_{alpha: t_alpha = r mod L} c_alpha^2   (Appendix B's z = sum c^2 u).
// The kernel accumulates the L bins W_r in FP64; t = tlow(p) + thigh(H).
#include <cmath>

#include "rows.cuh"

namespace hs {

constexpr int TW_WARPS = HV_THREADS / 32;

__global__ void __launch_bounds__(HV_THREADS) k_twist(Geo g, const double* __restrict__ psi,
                                                      double* __restrict__ partial) {
  extern __shared__ __align__(16) char smem[];
  __shared__ double bins[TW_WARPS][32];
  const RowSmem<double> s = row_smem_setup<double>(smem, g);
  for (int i = threadIdx.x; i < TW_WARPS * 32; i += blockDim.x) (&bins[0][0])[i] = 0.0;
  __syncthreads();
  const uint32_t L = (uint32_t)g.L;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for_blocks(g, 0.0, [&](const Hdr& h) {
    for (int r = lane; r < h.C; r += 32) {
      const double c = psi[h.R + r];
      const uint32_t bin = (le_tlow(s.low[h.off + r].packed) + (uint32_t)h.thigh) % L;
      atomicAdd(&bins[wid][bin], c * c);
    }
  });
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = 0.0;
    for (int w = 0; w < TW_WARPS; ++w) v += bins[w][threadIdx.x];
    partial[blockIdx.x * 32 + threadIdx.x] = v;
  }
}

hs_status launch_twist(hs_handle* hd, const double* psi, int K, double* z_host) {
  hs_status st = ensure_reduce(hd);
  if (st != HS_OK) return st;
  const size_t sm = row_smem_bytes<double>((int)hd->low.size());
  if (sm > 48 * 1024)
    HS_CUDA_TRY(hd, cudaFuncSetAttribute(k_twist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm));
  const int grid = row_grid(hd);
  const int L = hd->L;
  for (int q = 0; q < K; ++q) {
    k_twist<<<grid, HV_THREADS, sm, hd->stream>>>(hd->geo(), psi + (long long)q * hd->n,
                                                  hd->d_partial); count_launches(1);
    HS_CUDA_TRY(hd, cudaGetLastError());
    HS_CUDA_TRY(hd, cudaMemcpyAsync(hd->h_pinned, hd->d_partial, sizeof(double) * grid * 32,
                                    cudaMemcpyDeviceToHost, hd->stream));
    HS_CUDA_TRY(hd, cudaStreamSynchronize(hd->stream));
    double W[32] = {0};
    for (int c = 0; c < grid; ++c)
      for (int r = 0; r < 32; ++r) W[r] += hd->h_pinned[c * 32 + r];
    double re = 0, im = 0;
    for (int r = 0; r < L; ++r) {
      const double a = 2.0 * M_PI * r / L;
      re += W[r] * std::cos(a);
      im += W[r] * std::sin(a);
    }
    // global phase exp(-i pi (L+1)/2): L even, so (L+1)/2 is a half-integer
    const double ph = -M_PI * (L + 1) / 2.0;
    const double cr = std::cos(ph), ci = std::sin(ph);
    z_host[2 * q] = re * cr - im * ci;
    z_host[2 * q + 1] = re * ci + im * cr;
  }
  return HS_OK;
}

}  // namespace hs
