// FP64 vector kernels of the outer shift-invert Lanczos loop (Algorithm 1):
// dot products, the two passes of classical Gram-Schmidt against the stored
// basis V_k (h = V^T w, w -= V h), Ritz-vector assembly V_k y_i, the
// SplitMix64 start vector, and the FP64 <-> FP32 conversions of the
// refinement loop.
#include "common.cuh"

namespace hs {

constexpr int VT = 256;
constexpr int MD_COLS = 8;     // columns per multidot pass
constexpr int MD_GRID_MAX = 1024;

static int vgrid(const hs_handle* hd, long long n) {
  long long g = (n + VT - 1) / VT;
  return (int)std::max<long long>(1, std::min<long long>(g, (long long)hd->num_sms * 4));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// part[cta * ldp + col0 + j] = sum over this CTA's rows of V_{col0+j}[i] w[i]
__global__ void __launch_bounds__(VT) k_multidot(const double* __restrict__ V, int ncol, int col0,
                                                 const double* __restrict__ w, long long n,
                                                 double* __restrict__ part, int ldp) {
  __shared__ double sred[VT / 32][MD_COLS];
  double acc[MD_COLS];
#pragma unroll
  for (int j = 0; j < MD_COLS; ++j) acc[j] = 0.0;
  const int nc = min(MD_COLS, ncol - col0);
  for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT) {
    const double wi = w[i];
#pragma unroll
    for (int j = 0; j < MD_COLS; ++j)
      if (j < nc) acc[j] += V[(long long)(col0 + j) * n + i] * wi;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < MD_COLS; ++j) {
    const double v = warp_sum(acc[j]);
    if (lane == 0) sred[wid][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < nc) {
    double t = 0.0;
    for (int q = 0; q < VT / 32; ++q) t += sred[q][threadIdx.x];
    part[(long long)blockIdx.x * ldp + col0 + threadIdx.x] = t;
  }
}

// out[j] = sum_c part[c * ldp + j], fixed order (one warp per column).
__global__ void k_colsum(const double* __restrict__ part, int nparts, int ncol, int ldp,
                         double* __restrict__ out) {
  const int j = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= ncol) return;
  double t = 0.0;
  for (int c = lane; c < nparts; c += 32) t += part[(long long)c * ldp + j];
  t = warp_sum(t);
  if (lane == 0) out[j] = t;
}

// w[i] -= sum_j c[j] V_j[i]
__global__ void __launch_bounds__(VT) k_multiaxpy(const double* __restrict__ V, int ncol,
                                                  const double* __restrict__ c,
                                                  double* __restrict__ w, long long n) {
  extern __shared__ double sc[];
  for (int j = threadIdx.x; j < ncol; j += VT) sc[j] = c[j];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT) {
    double s = 0.0;
    for (int j = 0; j < ncol; ++j) s += sc[j] * V[(long long)j * n + i];
    w[i] -= s;
  }
}

// psi_q[i] = sum_j V_j[i] Y[j + q * ldy], q < K
__global__ void __launch_bounds__(VT) k_ritz(const double* __restrict__ V, int k,
                                             const double* __restrict__ Y, int K,
                                             double* __restrict__ psi, long long n) {
  extern __shared__ double sy[];
  for (int t = threadIdx.x; t < k * K; t += VT) sy[t] = Y[t];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT) {
    for (int q0 = 0; q0 < K; q0 += 8) {
      double acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = 0.0;
      for (int j = 0; j < k; ++j) {
        const double v = V[(long long)j * n + i];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q0 + q < K) acc[q] += v * sy[(q0 + q) * k + j];
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (q0 + q < K) psi[(long long)(q0 + q) * n + i] = acc[q];
    }
  }
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y,
                        long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

__global__ void k_scale_to(double a, const double* __restrict__ x, double* __restrict__ y,
                           long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

// SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator:
// value i = mix(seed + (i + 1) * 0x9E3779B97F4A7C15), mapped to [-1, 1).
__global__ void k_splitmix(unsigned long long seed, double* __restrict__ v, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    v[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  }
}

__global__ void k_f64_to_f32(const double* __restrict__ x, double scale, float* __restrict__ y,
                             long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)(x[i] * scale);
}

__global__ void k_axpy_f32(double a, const float* __restrict__ x, double* __restrict__ y,
                           long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] += a * (double)x[i];
}

// ---------------------------------------------------------------------------
static hs_status ensure_md(hs_handle* hd, int ncol, double** part, double** out) {
  // partial sums live in the reduction scratch: MD_GRID_MAX x (ncol) doubles
  static_assert(MD_GRID_MAX <= RED_MAX_CTAS, "scratch");
  if (ncol > 512) return fail(hd, HS_BAD_ARG, "too many columns for multidot");
  hs_status st = ensure_reduce(hd);
  if (st != HS_OK) return st;
  *part = hd->d_partial + RED_MAX_CTAS * 4;   // after the row-kernel slots
  *out = hd->d_partial;                       // reuse the first slots for the result
  return HS_OK;
}

hs_status vmultidot(hs_handle* hd, const double* V, int k, const double* w, long long n,
                    double* out) {
  double *part, *res;
  hs_status st = ensure_md(hd, k, &part, &res);
  if (st != HS_OK) return st;
  const int grid = std::min(vgrid(hd, n), MD_GRID_MAX);
  for (int c0 = 0; c0 < k; c0 += MD_COLS)
    k_multidot<<<grid, VT, 0, hd->stream>>>(V, k, c0, w, n, part, k); count_launches(1);
  k_colsum<<<(k + 7) / 8, 256, 0, hd->stream>>>(part, grid, k, k, res); count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  HS_CUDA_TRY(hd, cudaMemcpyAsync(hd->h_pinned, res, sizeof(double) * k, cudaMemcpyDeviceToHost,
                                  hd->stream));
  HS_CUDA_TRY(hd, cudaStreamSynchronize(hd->stream));
  for (int j = 0; j < k; ++j) out[j] = hd->h_pinned[j];
  return HS_OK;
}

hs_status vdot(hs_handle* hd, const double* a, const double* b, long long n, double* out) {
  return vmultidot(hd, a, 1, b, n, out);
}

hs_status vmultiaxpy(hs_handle* hd, const double* V, int k, const double* c, double* w,
                     long long n) {
  if (k <= 0) return HS_OK;
  double *part, *res;
  hs_status st = ensure_md(hd, k, &part, &res);
  if (st != HS_OK) return st;
  for (int j = 0; j < k; ++j) hd->h_pinned[j] = c[j];
  HS_CUDA_TRY(hd, cudaMemcpyAsync(res, hd->h_pinned, sizeof(double) * k, cudaMemcpyHostToDevice,
                                  hd->stream));
  k_multiaxpy<<<vgrid(hd, n), VT, sizeof(double) * k, hd->stream>>>(V, k, res, w, n); count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  // the coefficients are read from pinned memory by the copy; keep it alive
  HS_CUDA_TRY(hd, cudaStreamSynchronize(hd->stream));
  return HS_OK;
}

hs_status vritz(hs_handle* hd, const double* V, int k, const double* Y, int K, double* psi,
                long long n) {
  if (k * K > 4096) return fail(hd, HS_BAD_ARG, "Ritz assembly: k * K > 4096");
  double *part, *res;
  hs_status st = ensure_md(hd, 1, &part, &res);
  if (st != HS_OK) return st;
  for (int t = 0; t < k * K; ++t) hd->h_pinned[t] = Y[t];
  HS_CUDA_TRY(hd, cudaMemcpyAsync(part, hd->h_pinned, sizeof(double) * k * K,
                                  cudaMemcpyHostToDevice, hd->stream));
  k_ritz<<<vgrid(hd, n), VT, sizeof(double) * k * K, hd->stream>>>(V, k, part, K, psi, n); count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  HS_CUDA_TRY(hd, cudaStreamSynchronize(hd->stream));
  return HS_OK;
}

hs_status vaxpby(hs_handle* hd, double a, const double* x, double b, double* y, long long n) {
  k_axpby<<<vgrid(hd, n), VT, 0, hd->stream>>>(a, x, b, y, n); count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  return HS_OK;
}

hs_status vscale_to(hs_handle* hd, double a, const double* x, double* y, long long n) {
  k_scale_to<<<vgrid(hd, n), VT, 0, hd->stream>>>(a, x, y, n); count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  return HS_OK;
}

hs_status vsplitmix(hs_handle* hd, unsigned long long seed, double* v, long long n) {
  k_splitmix<<<vgrid(hd, n), VT, 0, hd->stream>>>(seed, v, n); count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  return HS_OK;
}

hs_status vcopy_f64_to_f32(hs_handle* hd, const double* x, double scale, float* y, long long n) {
  k_f64_to_f32<<<vgrid(hd, n), VT, 0, hd->stream>>>(x, scale, y, n); count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  return HS_OK;
}

hs_status vaxpy_f32_to_f64(hs_handle* hd, double a, const float* x, double* y, long long n) {
  k_axpy_f32<<<vgrid(hd, n), VT, 0, hd->stream>>>(a, x, y, n); count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  return HS_OK;
}

}  // namespace hs
