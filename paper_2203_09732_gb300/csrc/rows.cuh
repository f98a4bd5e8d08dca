// Device helpers for the row kernels: the warp-per-block iterator, the
// diagonal a_ii of Eq. (1), the diagonal preconditioners of Sec. II and the
// matrix-free rows of (H - sigma) x.
#pragma once
#include "common.cuh"

namespace hs {

// Shared memory of a row kernel: the low-pattern table (copied once per CTA),
// one staging buffer per warp for the block's x segment, reduction scratch.
template <typename T>
__host__ __device__ inline size_t row_smem_bytes(int nlow) {
  return sizeof(LowEntry) * (size_t)nlow + sizeof(T) * 32 * JMAX * HV_WARPS +
         sizeof(double) * 32 * 4;
}

template <typename T>
struct RowSmem {
  const LowEntry* low;
  T* xs;            // this warp's staging buffer (32 * JMAX elements)
  double* red;      // 32 * 4 doubles
};

template <typename T>
__device__ inline RowSmem<T> row_smem_setup(char* base, const Geo& g) {
  RowSmem<T> s;
  LowEntry* low = reinterpret_cast<LowEntry*>(base);
  const uint4* src = reinterpret_cast<const uint4*>(g.low);
  uint4* dst = reinterpret_cast<uint4*>(low);
  for (int i = threadIdx.x; i < g.nlow * 2; i += blockDim.x) dst[i] = __ldg(src + i);
  base += sizeof(LowEntry) * g.nlow;
  s.low = low;
  s.xs = reinterpret_cast<T*>(base) + (threadIdx.x >> 5) * (32 * JMAX);
  base += sizeof(T) * 32 * JMAX * HV_WARPS;
  s.red = reinterpret_cast<double*>(base);
  __syncthreads();
  return s;
}

// Warp-uniform view of one block header (lane l holds word l; fields are
// broadcast by shuffles).
struct Hdr {
  uint32_t word;     // this lane's header word
  uint32_t R, Rwrap;
  int32_t bdelta;
  int w, nh, code, thigh;
  int C, off, J;
  double dhs;        // dhigh - sigma
  float dhs_f;
};

__device__ __forceinline__ uint32_t hdr_word(const Geo& g, int bi) {
  return __ldg(reinterpret_cast<const uint32_t*>(g.blocks + bi) + (threadIdx.x & 31));
}

__device__ __forceinline__ Hdr make_hdr(const Geo& g, uint32_t word, double sigma) {
  Hdr h;
  h.word = word;
  const unsigned full = 0xffffffffu;
  h.R = __shfl_sync(full, word, 0);
  h.Rwrap = __shfl_sync(full, word, 1);
  h.bdelta = (int32_t)__shfl_sync(full, word, 2);
  const uint32_t meta = __shfl_sync(full, word, 3);
  const uint32_t lo = __shfl_sync(full, word, 4);
  const uint32_t hi = __shfl_sync(full, word, 5);
  h.w = meta & 0xFF;
  h.nh = (meta >> 8) & 0xFF;
  h.code = (meta >> 16) & 0xFF;
  h.thigh = meta >> 24;
  h.C = g.cls_C[h.w];
  h.off = g.cls_off[h.w];
  h.J = (h.C + 31) >> 5;
  const double dhigh = __hiloint2double((int)hi, (int)lo);
  h.dhs = dhigh - sigma;
  h.dhs_f = (float)h.dhs;
  return h;
}

__device__ __forceinline__ Hdr load_hdr(const Geo& g, int bi, double sigma) {
  return make_hdr(g, hdr_word(g, bi), sigma);
}

__device__ __forceinline__ int32_t hdr_hd(const Hdr& h, int m) {
  return (int32_t)__shfl_sync(0xffffffffu, h.word, 6 + m);
}

// Walk this warp's blocks in rank order (grid stride), prefetching the next
// header while the current block is processed; f(const Hdr&) per block.
template <class F>
__device__ __forceinline__ void for_blocks(const Geo& g, double sigma, F&& f) {
  const int stride = gridDim.x * HV_WARPS;
  int bi = blockIdx.x * HV_WARPS + (threadIdx.x >> 5);
  if (bi >= g.nblocks) return;
  uint32_t word = hdr_word(g, bi);
  while (true) {
    const int nx = bi + stride;
    const uint32_t next = nx < g.nblocks ? hdr_word(g, nx) : 0u;
    f(make_hdr(g, word, sigma));
    if (nx >= g.nblocks) break;
    bi = nx;
    word = next;
  }
}

// cut-bond flip mask: bit 0 = bond (k-1, k), bit 1 = bond (L-1, 0)
__device__ __forceinline__ uint32_t cut_mask(uint32_t packed, const Hdr& h) {
  return le_code(packed) ^ (uint32_t)h.code;
}

// a_ii - sigma
__device__ __forceinline__ float diag_f(const LowEntry& e, const Hdr& h, uint32_t xc) {
  return e.dlow_f + h.dhs_f + (0.5f - 0.5f * (float)__popc(xc));
}
__device__ __forceinline__ double diag_d(const LowEntry& e, const Hdr& h, uint32_t xc) {
  return e.dlow + h.dhs + (0.5 - 0.5 * (double)__popc(xc));
}
template <typename T>
__device__ __forceinline__ T diag_t(const LowEntry& e, const Hdr& h, uint32_t xc) {
  if constexpr (sizeof(T) == 8) return diag_d(e, h, xc);
  else return diag_f(e, h, xc);
}
// number of antiparallel bonds of the row (sum_k |a_ik|^2 = naf / 4)
__device__ __forceinline__ int naf_row(uint32_t packed, const Hdr& h, uint32_t xc) {
  return le_cnt(packed) + h.nh + __popc(xc);
}

// M_ii for preconditioner PC (0 identity, 1 Jacobi, 2 row norm), Sec. II.
template <int PC, typename T>
__device__ __forceinline__ T precond_t(T am, int naf) {
  if (PC == 0) return T(1);
  if (PC == 1) return am < T(0) ? -am : am;
  if constexpr (sizeof(T) == 8) return sqrt(am * am + 0.25 * (double)naf);
  else return sqrtf(am * am + 0.25f * (float)naf);
}

// Gather load. COH = false: read-only path (the vector is not written while
// the kernel runs). COH = true: L2-coherent load, for persistent kernels that
// read vectors other CTAs rewrite between grid barriers.
template <typename T, bool COH = false>
__device__ __forceinline__ T ldx(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}

// Rows of one block: xi[j] = x[R + r_j], hx[j] = ((H - sigma) x)[R + r_j] for
// r_j = lane + 32 j < C, j < h.J. The self, cut and wrap gathers of all J rows
// are issued first, then the high-interior shifts in groups of HG bonds (HG * J
// independent loads in flight per lane, each a coalesced warp access from a
// warp-uniform base); the low-interior neighbours are read from the block's x
// segment staged in shared memory.
template <typename T, bool COH = false>
__device__ __forceinline__ void block_hv(const T* __restrict__ x, const RowSmem<T>& s,
                                         const Hdr& h, T (&xi)[JMAX], T (&hx)[JMAX]) {
#ifndef HS_HG
  constexpr int HG = 2;
#else
  constexpr int HG = HS_HG;
#endif
  const int lane = threadIdx.x & 31;
  const T* xb = x + h.R;
  T side[JMAX];
#pragma unroll
  for (int j = 0; j < JMAX; ++j) {
    xi[j] = T(0);
    side[j] = T(0);
    hx[j] = T(0);
    const int r = lane + 32 * j;
    if (j < h.J && r < h.C) {
      const LowEntry& e = s.low[h.off + r];
      const uint32_t xc = cut_mask(e.packed, h);
      xi[j] = ldx<T, COH>(xb + r);
      const T c1 = (xc & 1u) ? ldx<T, COH>(xb + h.bdelta + r) : T(0);
      const T c2 = (xc & 2u) ? ldx<T, COH>(x + (h.Rwrap + e.wrap_r)) : T(0);
      side[j] = c1 + c2;
    }
  }
  for (int m0 = 0; m0 < h.nh; m0 += HG) {
    T v[HG][JMAX];
#pragma unroll
    for (int mm = 0; mm < HG; ++mm) {
      const bool on = m0 + mm < h.nh;
      const T* xh = xb + (on ? hdr_hd(h, m0 + mm) : 0) + lane;
#pragma unroll
      for (int j = 0; j < JMAX; ++j)
        v[mm][j] = (on && j < h.J && lane + 32 * j < h.C) ? ldx<T, COH>(xh + 32 * j) : T(0);
    }
#pragma unroll
    for (int mm = 0; mm < HG; ++mm)
#pragma unroll
      for (int j = 0; j < JMAX; ++j) hx[j] += v[mm][j];
  }
#pragma unroll
  for (int j = 0; j < JMAX; ++j)
    if (j < h.J) s.xs[lane + 32 * j] = xi[j];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < JMAX; ++j) {
    const int r = lane + 32 * j;
    if (j < h.J && r < h.C) {
      const LowEntry& e = s.low[h.off + r];
      const uint32_t pk = e.packed;
      const uint32_t xc = cut_mask(pk, h);
      T acc = hx[j] + side[j];
      const int cnt = le_cnt(pk);
      const uint32_t w0 = e.nbw[0], w1 = e.nbw[1], w2 = e.nbw[2];
#pragma unroll
      for (int m = 0; m < NB_MAX; ++m) {
        const uint32_t wd = m < 4 ? w0 : (m < 8 ? w1 : w2);
        if (m < cnt) acc += s.xs[(wd >> (8 * (m & 3))) & 0xFFu];
      }
      hx[j] = diag_t<T>(e, h, xc) * xi[j] + T(0.5) * acc;
    }
  }
  __syncwarp();
}

// Block-wide sum of up to 4 doubles per thread; result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sred) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < NV; ++j) sred[wid * 4 + j] = v[j];
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      v[j] = lane < nw ? sred[lane * 4 + j] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
    }
  }
}

// Last-CTA reduction: every CTA writes its NV partials; the CTA that arrives
// last sums all partials in a fixed order (deterministic) and returns true in
// all of its threads with the totals in tot[] (valid in thread 0).
template <int NV>
__device__ __forceinline__ bool last_cta_sum(double (&v)[NV], double* sred, double* partial,
                                             unsigned int* counter, double (&tot)[NV]) {
  __shared__ unsigned int s_ticket;
  block_sum<NV>(v, sred);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) partial[blockIdx.x * 4 + j] = v[j];
    __threadfence();
    s_ticket = atomicAdd(counter, 1u);
  }
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return false;
  __threadfence();
  double a[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) a[j] = 0.0;
  for (int c = threadIdx.x; c < (int)gridDim.x; c += blockDim.x)
#pragma unroll
    for (int j = 0; j < NV; ++j) a[j] += __ldcg(partial + c * 4 + j);
  block_sum<NV>(a, sred);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) tot[j] = a[j];
    *counter = 0u;
  }
  return true;
}


}  // namespace hs
