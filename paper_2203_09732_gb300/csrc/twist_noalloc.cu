// Twist overlap for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside a CUDA graph that is
// being captured or replayed by someone else, plug-ins of a host application
// that owns every device allocation through its own pool, or processes that
// have already reserved nearly all device memory. hs_twist needs a handle,
// and creating a handle allocates its tables and workspace. This file gives
// them hs_twist_noalloc: the same z = <psi| U_twist |psi> reduction (Sec. III),
// with no handle and no allocation. Basis states are unranked on the fly from a
// binomial table that lives in constant memory, and the per-CTA partial sums
// live in one file-scope static device array of fixed size.
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace {

constexpr int TNA_K_MAX = 8;         // vectors per call
constexpr int TNA_CTAS = 256;        // CTAs of the accumulation kernel
constexpr int TNA_THREADS = 256;
constexpr int TNA_BINS = 32;         // one bin per value of t mod L (L <= 32)
// Scratch: TNA_K_MAX x TNA_CTAS x TNA_BINS doubles of per-CTA partial sums,
// then 32 doubles whose first word is the arrival counter of the last-CTA
// reduction: 8 * 256 * 32 * 8 B + 256 B = 512 KiB + 256 B per device.
constexpr int TNA_PART = TNA_K_MAX * TNA_CTAS * TNA_BINS;
static __device__ __align__(256) double g_twist_scratch[TNA_PART + 32];

struct BinomTab {
  uint32_t v[hs::LMAX + 1][hs::LMAX / 2 + 2];
};
constexpr BinomTab make_binom() {
  BinomTab t{};
  for (int a = 0; a <= hs::LMAX; ++a)
    for (int c = 0; c < hs::LMAX / 2 + 2; ++c) {
      if (c > a) { t.v[a][c] = 0; continue; }
      uint64_t r = 1;
      for (int i = 1; i <= c; ++i) r = r * (uint64_t)(a - c + i) / (uint64_t)i;
      t.v[a][c] = (uint32_t)r;
    }
  return t;
}
__constant__ BinomTab c_binom = make_binom();

// State of rank r: colex unranking (rank = sum_i C(p_i, i) over set bits).
__device__ __forceinline__ uint32_t unrank_one(uint32_t r, int L, int N) {
  uint32_t s = 0;
  int p = L - 1;
  for (int c = N; c >= 1; --c) {
    while (c_binom.v[p][c] > r) --p;
    s |= 1u << p;
    r -= c_binom.v[p][c];
    --p;
  }
  return s;
}

// Next word with the same popcount (the next state in ascending order).
__device__ __forceinline__ uint32_t next_same_popc(uint32_t s) {
  const uint32_t c = s & (0u - s);
  const uint32_t r = s + c;
  return (((r ^ s) >> 2) / c) | r;
}

__global__ void __launch_bounds__(TNA_THREADS) k_twist_noalloc(int L, long long n,
                                                               const double* __restrict__ psi,
                                                               int K, double* scratch,
                                                               double* __restrict__ z) {
  __shared__ double bins[TNA_K_MAX][TNA_BINS];
  __shared__ unsigned s_ticket;
  const int N = L / 2;
  for (int i = threadIdx.x; i < TNA_K_MAX * TNA_BINS; i += blockDim.x) (&bins[0][0])[i] = 0.0;
  __syncthreads();
  // each thread takes one contiguous chunk of ranks and walks it with the
  // successor function after a single unranking
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long chunk = (n + nth - 1) / nth;
  const long long r0 = tid * chunk;
  const long long r1 = r0 + chunk < n ? r0 + chunk : n;
  if (r0 < r1) {
    uint32_t s = unrank_one((uint32_t)r0, L, N);
    for (long long r = r0; r < r1; ++r) {
      uint32_t w = s, t = 0;
      while (w) {
        t += (uint32_t)__ffs(w);   // site j + 1 for set bit j
        w &= w - 1u;
      }
      const int bin = (int)(t % (uint32_t)L);
      for (int q = 0; q < K; ++q) {
        const double c = psi[(long long)q * n + r];
        atomicAdd(&bins[q][bin], c * c);
      }
      if (r + 1 < r1) s = next_same_popc(s);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < K * TNA_BINS; i += blockDim.x) {
    const int q = i / TNA_BINS, b = i % TNA_BINS;
    scratch[((size_t)q * TNA_CTAS + blockIdx.x) * TNA_BINS + b] = bins[q][b];
  }
  __threadfence();
  __syncthreads();
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + TNA_PART);
  if (threadIdx.x == 0) s_ticket = atomicAdd(counter, 1u);
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return;
  __threadfence();
  // last CTA: W_r in a fixed order, then z = exp(-i pi (L+1)/2) sum_r W_r exp(i 2pi r / L)
  if (threadIdx.x < K) {
    const int q = threadIdx.x;
    double re = 0.0, im = 0.0;
    for (int b = 0; b < L; ++b) {
      double W = 0.0;
      for (int c = 0; c < (int)gridDim.x; ++c)
        W += __ldcg(&scratch[((size_t)q * TNA_CTAS + c) * TNA_BINS + b]);
      double sn, cs;
      sincospi(2.0 * b / L, &sn, &cs);
      re += W * cs;
      im += W * sn;
    }
    double ps, pc;
    sincospi(-(L + 1) / 2.0, &ps, &pc);
    z[2 * q] = re * pc - im * ps;
    z[2 * q + 1] = re * ps + im * pc;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// Device address of g_twist_scratch. It is looked up again on every call made
// outside a stream capture (a cudaDeviceReset reloads the module, and the
// array may then live elsewhere); during a capture the address cached by the
// last uncaptured call on this device is used.
std::mutex g_mu;
double* g_ptr[64] = {nullptr};

hs_status scratch_for_current_device(cudaStream_t s, double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return HS_CUDA;
  }
  if (dev < 0 || dev >= 64) return HS_BAD_ARG;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return HS_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (cap == cudaStreamCaptureStatusNone || !g_ptr[dev]) {
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_twist_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return HS_CUDA;
    }
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return HS_OK;
}

}  // namespace

extern "C" hs_status hs_twist_noalloc(int L, const double* psi_dev, int K, double* z_dev,
                                      void* cuda_stream) {
  if (L < 4 || L > hs::LMAX || (L & 1)) return HS_BAD_ARG;
  if (K < 1 || K > TNA_K_MAX) return HS_BAD_ARG;   // the scratch holds 8 vectors
  if (!psi_dev || !z_dev) return HS_BAD_ARG;
  double* scratch = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const hs_status st = scratch_for_current_device(s, &scratch);
  if (st != HS_OK) return st;
  const long long n = (long long)hs::binom(L, L / 2);
  // the arrival counter must start at zero (a previous call leaves it at zero
  // unless it was interrupted)
  if (cudaMemsetAsync(scratch + TNA_PART, 0, sizeof(double), s) != cudaSuccess) {
    cudaGetLastError();
    return HS_CUDA;
  }
  const long long want = (n + TNA_THREADS * 16 - 1) / (TNA_THREADS * 16);
  const int grid = (int)(want < 1 ? 1 : (want > TNA_CTAS ? TNA_CTAS : want));
  k_twist_noalloc<<<grid, TNA_THREADS, 0, s>>>(L, n, psi_dev, K, scratch, z_dev);
  hs::count_launches(1);
  if (cudaGetLastError() != cudaSuccess) return HS_CUDA;
  return HS_OK;
}
