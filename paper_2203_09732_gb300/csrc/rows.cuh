// Device helpers for the row kernels: the persistent tile loop, the diagonal
// a_ii of Eq. (1), the diagonal preconditioners of Sec. II and the
// matrix-free row of (H - sigma) x.
#pragma once
#include "common.cuh"

namespace hs {

// Shared-memory image of the tables a row kernel reads.
struct RowSmem {
  LowEntry* low;
  uint16_t* nb;
  double* dlow64;
  BlockInfo* blk;   // TILE_G_MAX entries
  double* red;      // 32 * 4 doubles for block reductions
};

__host__ __device__ inline size_t row_smem_bytes(int nlow, int nnb) {
  size_t b = sizeof(BlockInfo) * TILE_G_MAX;
  b += sizeof(LowEntry) * (size_t)nlow;
  b += sizeof(double) * (size_t)nlow;
  b += sizeof(double) * 32 * 4;
  b += sizeof(uint16_t) * (size_t)nnb;
  return (b + 15) & ~size_t(15);
}

__device__ inline RowSmem row_smem_carve(char* base, const Geo& g) {
  RowSmem s;
  s.blk = reinterpret_cast<BlockInfo*>(base);
  base += sizeof(BlockInfo) * TILE_G_MAX;
  s.low = reinterpret_cast<LowEntry*>(base);
  base += sizeof(LowEntry) * g.nlow;
  s.dlow64 = reinterpret_cast<double*>(base);
  base += sizeof(double) * g.nlow;
  s.red = reinterpret_cast<double*>(base);
  base += sizeof(double) * 32 * 4;
  s.nb = reinterpret_cast<uint16_t*>(base);
  return s;
}

// Copy the low-pattern tables to shared memory (once per CTA).
__device__ inline void row_smem_fill(const RowSmem& s, const Geo& g, bool need64) {
  const uint4* src = reinterpret_cast<const uint4*>(g.low);
  uint4* dst = reinterpret_cast<uint4*>(s.low);
  for (int i = threadIdx.x; i < g.nlow; i += blockDim.x) dst[i] = __ldg(src + i);
  for (int i = threadIdx.x; i < g.nnb; i += blockDim.x) s.nb[i] = __ldg(g.nb + i);
  if (need64)
    for (int i = threadIdx.x; i < g.nlow; i += blockDim.x) s.dlow64[i] = __ldg(g.dlow64 + i);
}

// Load the tile's block headers to shared memory and fold sigma into them.
__device__ inline void tile_load(const RowSmem& s, const Geo& g, const Tile& t, double sigma) {
  constexpr int W = sizeof(BlockInfo) / 4;
  const uint32_t* src = reinterpret_cast<const uint32_t*>(g.blocks + t.b0);
  uint32_t* dst = reinterpret_cast<uint32_t*>(s.blk);
  const int words = W * t.G;
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = __ldg(src + i);
  __syncthreads();
  if (threadIdx.x < t.G) {
    BlockInfo& b = s.blk[threadIdx.x];
    b.dhs = b.dhigh - sigma;
    b.dhs_f = (float)b.dhs;
  }
  __syncthreads();
}

// Run f(block, lowindex, r) over every row of the tile (flattened mapping:
// consecutive threads take consecutive rows of a block, so global accesses of
// a warp are contiguous).
template <class F>
__device__ __forceinline__ void tile_rows(const RowSmem& s, const Geo& g, const Tile& t, F&& f) {
  const int C = g.cls_C[t.w];
  const int off = g.cls_off[t.w];
  const int rows = (int)t.G * C;
  const float invC = 1.0f / (float)C;
  for (int idx = threadIdx.x; idx < rows; idx += blockDim.x) {
    int b = (int)((float)idx * invC);
    int r = idx - b * C;
    if (r < 0) { b -= 1; r += C; } else if (r >= C) { b += 1; r -= C; }
    f(s.blk[b], off + r, r);
  }
}

// Number of antiparallel bonds of the row (for the row-norm preconditioner)
// and the cut-bond flip mask: bit 0 = bond (k-1, k), bit 1 = bond (L-1, 0).
__device__ __forceinline__ uint32_t cut_mask(const LowEntry& e, const BlockInfo& b) {
  return le_code(e.packed) ^ (uint32_t)b.code;
}

// a_ii - sigma (sigma folded into dhs by tile_load).
__device__ __forceinline__ float diag_f(const LowEntry& e, const BlockInfo& b, uint32_t xc) {
  return e.dlow_f + b.dhs_f + (0.5f - 0.5f * (float)__popc(xc));
}
__device__ __forceinline__ double diag_d(double dlow, const BlockInfo& b, uint32_t xc) {
  return dlow + b.dhs + (0.5 - 0.5 * (double)__popc(xc));
}
__device__ __forceinline__ int naf_row(const LowEntry& e, const BlockInfo& b, uint32_t xc) {
  return le_cnt(e.packed) + (int)b.nh + __popc(xc);
}

// M_ii for preconditioner PC (0 identity, 1 Jacobi, 2 row norm).
template <int PC>
__device__ __forceinline__ float precond_f(float am, int naf) {
  if (PC == 0) return 1.0f;
  if (PC == 1) return fabsf(am);
  return sqrtf(am * am + 0.25f * (float)naf);
}
template <int PC>
__device__ __forceinline__ double precond_d(double am, int naf) {
  if (PC == 0) return 1.0;
  if (PC == 1) return fabs(am);
  return sqrt(am * am + 0.25 * (double)naf);
}

template <typename T>
__device__ __forceinline__ T ldx(const T* p) { return __ldg(p); }

// Off-diagonal part of row i of H applied to x: (1/2) sum over antiparallel
// bonds of x[target], and the self element x[i]. All gathers of the row are
// issued before any is consumed (predicated, unrolled) so that a thread keeps
// up to ~20 independent loads in flight.
template <typename T>
__device__ __forceinline__ T offdiag_row(const T* __restrict__ x, const RowSmem& s,
                                         const BlockInfo& b, const LowEntry& e, uint32_t r,
                                         uint32_t xc, T& xi) {
  const uint32_t i = b.R + r;
  const int cnt = le_cnt(e.packed);
  const uint16_t* nbp = s.nb + e.nb_off;
  T lo[NB_MAX];
#pragma unroll
  for (int m = 0; m < NB_MAX; ++m) lo[m] = (m < cnt) ? ldx(x + (b.R + nbp[m])) : T(0);
  const T cw = (xc & 1u) ? ldx(x + (uint32_t)((int32_t)i + b.bdelta)) : T(0);
  const T ww = (xc & 2u) ? ldx(x + (b.Rwrap + e.wrap_r)) : T(0);
  xi = ldx(x + i);
  T acc = cw + ww;
  const int nh = b.nh;
  for (int m0 = 0; m0 < nh; m0 += 8) {
    T hv[8];
#pragma unroll
    for (int m = 0; m < 8; ++m)
      hv[m] = (m0 + m < nh) ? ldx(x + (uint32_t)((int32_t)i + b.hd[m0 + m])) : T(0);
#pragma unroll
    for (int m = 0; m < 8; ++m) acc += hv[m];
  }
#pragma unroll
  for (int m = 0; m < NB_MAX; ++m) acc += lo[m];
  return T(0.5) * acc;
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
