// Matrix-free H x (Eq. (1)), the basis ranking (Sec. I: Sz = 0 sector in
// ascending integer order), the diagonal / preconditioner export (Sec. II) and
// the FP64 refinement residual r = b - (H - sigma) x.
#include <cstdlib>

#include "rows.cuh"

namespace hs {

// ---------------------------------------------------------------------------
// y = (H - sigma * shifted) x. Warps walk the blocks in rank order.
template <typename T>
__global__ void __launch_bounds__(HV_THREADS) k_matvec(Geo g, const T* __restrict__ x,
                                                       T* __restrict__ y, const double* d_sigma,
                                                       int shifted) {
  extern __shared__ __align__(16) char smem[];
  const RowSmem<T> s = row_smem_setup<T>(smem, g);
  const double sigma = shifted ? *d_sigma : 0.0;
  const int lane = threadIdx.x & 31;
  for_blocks(g, sigma, [&](const Hdr& h) {
    T xi[JMAX], hx[JMAX];
    block_hv<T>(x, s, h, xi, hx);
    T* yb = y + h.R + lane;
#pragma unroll
    for (int j = 0; j < JMAX; ++j)
      if (j < h.J && lane + 32 * j < h.C) __stcs(yb + 32 * j, hx[j]);
  });
}

// ---------------------------------------------------------------------------
// Ranking: colex rank of the popcount-N word s = sum_i C(p_i, i) over its set
// bits p_1 < p_2 < ... (equal to the ascending-integer rank of the sector).
__global__ void k_unrank(const uint32_t* __restrict__ binom, int L, int N, long long first,
                         long long count, unsigned int* __restrict__ out) {
  const int W = LMAX / 2 + 2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
       t += (long long)gridDim.x * blockDim.x) {
    uint32_t r = (uint32_t)(first + t);
    uint32_t s = 0;
    int p = L - 1;
    for (int c = N; c >= 1; --c) {
      while (binom[p * W + c] > r) --p;
      s |= 1u << p;
      r -= binom[p * W + c];
      --p;
    }
    out[t] = s;
  }
}

__global__ void k_rank(const uint32_t* __restrict__ binom, int L, int N,
                       const unsigned int* __restrict__ st, long long count,
                       long long* __restrict__ out) {
  const int W = LMAX / 2 + 2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
       t += (long long)gridDim.x * blockDim.x) {
    uint32_t s = st[t];
    if ((L < 32 && (s >> L) != 0u) || __popc(s) != N) { out[t] = -1; continue; }
    long long r = 0;
    int c = 1;
    while (s) {
      const int p = __ffs(s) - 1;
      r += binom[p * W + c];
      ++c;
      s &= s - 1u;
    }
    out[t] = r;
  }
}

// ---------------------------------------------------------------------------
// diag[i] = a_ii, minv[i] = 1 / M_ii (FP64).
__global__ void __launch_bounds__(HV_THREADS) k_diag(Geo g, double* diag, double* minv, int pc,
                                                     const double* d_sigma) {
  extern __shared__ __align__(16) char smem[];
  const RowSmem<double> s = row_smem_setup<double>(smem, g);
  const double sigma = *d_sigma;
  const int lane = threadIdx.x & 31;
  for_blocks(g, sigma, [&](const Hdr& h) {
    for (int r = lane; r < h.C; r += 32) {
      const LowEntry& e = s.low[h.off + r];
      const uint32_t xc = cut_mask(e.packed, h);
      const double am = diag_d(e, h, xc);
      const uint32_t i = h.R + r;
      if (diag) diag[i] = am + sigma;
      if (minv) {
        const int naf = naf_row(e.packed, h, xc);
        const double m = pc == 0 ? 1.0 : (pc == 1 ? fabs(am) : sqrt(am * am + 0.25 * naf));
        minv[i] = 1.0 / m;
      }
    }
  });
}

// ---------------------------------------------------------------------------
// FP64 residual r = b - (H - sigma) x with per-CTA partial sums
// [sum r^2 / M, sum r^2, sum b^2 / M, sum b^2] (host adds them in order).
// MODE: RES_PRODUCT forms the product here; RES_ZERO: x is zero (the first
// refinement sweep), so r = b and x is not read; RES_GIVEN: rv already holds
// (H - sigma) x (from a faster product kernel) and is overwritten in place.
constexpr int RES_PRODUCT = 0, RES_ZERO = 1, RES_GIVEN = 2;
template <int PC, int MODE>
__global__ void __launch_bounds__(HV_THREADS) k_resid64(Geo g, const double* __restrict__ bv,
                                                        const double* __restrict__ x,
                                                        double* __restrict__ rv,
                                                        const double* d_sigma,
                                                        double* partial) {
  extern __shared__ __align__(16) char smem[];
  const RowSmem<double> s = row_smem_setup<double>(smem, g);
  const double sigma = *d_sigma;
  const int lane = threadIdx.x & 31;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for_blocks(g, sigma, [&](const Hdr& h) {
    double xi[JMAX], hx[JMAX];
    if constexpr (MODE == RES_PRODUCT) {
      block_hv<double>(x, s, h, xi, hx);
    } else {
#pragma unroll
      for (int j = 0; j < JMAX; ++j) hx[j] = 0.0;
    }
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
      const int r = lane + 32 * j;
      if (j < h.J && r < h.C) {
        const LowEntry& e = s.low[h.off + r];
        const uint32_t xc = cut_mask(e.packed, h);
        const double m = precond_t<PC, double>(diag_d(e, h, xc), naf_row(e.packed, h, xc));
        const uint32_t i = h.R + r;
        const double bi_ = bv[i];
        const double ri = bi_ - (MODE == RES_GIVEN ? rv[i] : hx[j]);
        rv[i] = ri;
        acc[0] += ri * ri / m;
        acc[1] += ri * ri;
        acc[2] += bi_ * bi_ / m;
        acc[3] += bi_ * bi_;
      }
    }
  });
  block_sum<4>(acc, s.red);
  if (threadIdx.x == 0)
    for (int j = 0; j < 4; ++j) partial[blockIdx.x * 4 + j] = acc[j];
}

// ---------------------------------------------------------------------------
template <typename T>
static size_t smem_of(const hs_handle* hd) {
  return row_smem_bytes<T>((int)hd->low.size());
}

template <typename K>
static hs_status prep_smem(hs_handle* hd, K kern, size_t bytes) {
  if (bytes > 48 * 1024)
    HS_CUDA_TRY(hd, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes));
  return HS_OK;
}

hs_status launch_matvec(hs_handle* hd, const void* x, void* y, hs_dtype dt, int shifted) {
  {
    // superblock forms from L = 24 on: in FP32 the ten-low-bit form (1.2-1.3x
    // faster than the block form there), in FP64 the four-low-bit form (the
    // FP64 pipe bounds every form; it does the fewest FP64 operations).
    // HS_HV_SB=0 turns them off, =1 uses them wherever a plan was built
    // (L >= 22).
    const char* e = getenv("HS_HV_SB");
    const bool on = e ? e[0] == '1' : hd->L >= 24;
    if (on) {
      bool used = false;
      hs_status st = launch_matvec_sb(hd, x, y, dt, shifted, &used);
      if (st != HS_OK || used) return st;
    }
  }
  const Geo g = hd->geo();
  const int grid = row_grid(hd);
  if (dt == HS_F32) {
    const size_t sm = smem_of<float>(hd);
    if (prep_smem(hd, k_matvec<float>, sm) != HS_OK) return HS_CUDA;
    k_matvec<float><<<grid, HV_THREADS, sm, hd->stream>>>(
        g, static_cast<const float*>(x), static_cast<float*>(y), hd->d_sigma, shifted); count_launches(1);
  } else {
    const size_t sm = smem_of<double>(hd);
    if (prep_smem(hd, k_matvec<double>, sm) != HS_OK) return HS_CUDA;
    k_matvec<double><<<grid, HV_THREADS, sm, hd->stream>>>(
        g, static_cast<const double*>(x), static_cast<double*>(y), hd->d_sigma, shifted); count_launches(1);
  }
  HS_CUDA_TRY(hd, cudaGetLastError());
  return HS_OK;
}

hs_status launch_unrank(hs_handle* hd, long long first, long long count, unsigned int* out) {
  if (count <= 0) return HS_OK;
  const int grid = (int)std::min<long long>((count + 255) / 256, hd->num_sms * 8LL);
  k_unrank<<<grid, 256, 0, hd->stream>>>(hd->d_binom, hd->L, hd->N, first, count, out); count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  return HS_OK;
}

hs_status launch_rank(hs_handle* hd, const unsigned int* st, long long count, long long* out) {
  if (count <= 0) return HS_OK;
  const int grid = (int)std::min<long long>((count + 255) / 256, hd->num_sms * 8LL);
  k_rank<<<grid, 256, 0, hd->stream>>>(hd->d_binom, hd->L, hd->N, st, count, out); count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  return HS_OK;
}

hs_status launch_diag(hs_handle* hd, double* diag, hs_precond pc, double* minv) {
  const size_t sm = smem_of<double>(hd);
  if (prep_smem(hd, k_diag, sm) != HS_OK) return HS_CUDA;
  k_diag<<<row_grid(hd), HV_THREADS, sm, hd->stream>>>(hd->geo(), diag, minv, (int)pc,
                                                       hd->d_sigma); count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  return HS_OK;
}

template <int MODE>
static hs_status resid64_t(hs_handle* hd, const double* b, const double* x, double* r,
                           hs_precond pc, int grid, size_t sm) {
  const Geo g = hd->geo();
  switch (pc) {
    case HS_PC_ID:
      if (prep_smem(hd, k_resid64<0, MODE>, sm) != HS_OK) return HS_CUDA;
      k_resid64<0, MODE><<<grid, HV_THREADS, sm, hd->stream>>>(g, b, x, r, hd->d_sigma, hd->d_partial); count_launches(1);
      break;
    case HS_PC_JACOBI:
      if (prep_smem(hd, k_resid64<1, MODE>, sm) != HS_OK) return HS_CUDA;
      k_resid64<1, MODE><<<grid, HV_THREADS, sm, hd->stream>>>(g, b, x, r, hd->d_sigma, hd->d_partial); count_launches(1);
      break;
    default:
      if (prep_smem(hd, k_resid64<2, MODE>, sm) != HS_OK) return HS_CUDA;
      k_resid64<2, MODE><<<grid, HV_THREADS, sm, hd->stream>>>(g, b, x, r, hd->d_sigma, hd->d_partial); count_launches(1);
      break;
  }
  HS_CUDA_TRY(hd, cudaGetLastError());
  return HS_OK;
}

hs_status resid64(hs_handle* hd, const double* b, const double* x, double* r, hs_precond pc,
                  double sums_out[4], bool x_zero) {
  hs_status st = ensure_reduce(hd);
  if (st != HS_OK) return st;
  const size_t sm = smem_of<double>(hd);
  const int grid = row_grid(hd);
  if (x_zero) {
    st = resid64_t<RES_ZERO>(hd, b, x, r, pc, grid, sm);
  } else {
    // where a superblock FP64 product applies (L >= 24) it is faster than the
    // block form's: form (H - sigma) x in r, then r = b - r with the sums
    const char* e = getenv("HS_HV_SB");
    bool used = false;
    if (e ? e[0] == '1' : hd->L >= 24)
      if ((st = launch_matvec_sb(hd, x, r, HS_F64, 1, &used)) != HS_OK) return st;
    st = used ? resid64_t<RES_GIVEN>(hd, b, x, r, pc, grid, sm)
              : resid64_t<RES_PRODUCT>(hd, b, x, r, pc, grid, sm);
  }
  if (st != HS_OK) return st;
  return sum_partials(hd, grid, 4, sums_out);
}

}  // namespace hs
