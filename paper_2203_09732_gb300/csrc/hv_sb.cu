// Superblock form of y = (H - sigma) x (Eq. (1)) for long chains: one CTA per
// superblock pair {T, T ^ top}. Phase 1 stages x of the pair into shared
// memory by asynchronous copies while it sums the high-bit and (KS-1, KS)
// flips of every row from global memory (coalesced shifted streams); phase 2
// walks the sub-blocks and reads shared memory only. Layout and bond kinds:
// sb.cuh.
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "sb.cuh"

namespace hs {
namespace sb {

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <typename T>
__host__ __device__ inline size_t smem_bytes(int nlow, int km) {
  return sizeof(Low16) * (size_t)nlow + (sizeof(T) == 8 ? sizeof(double) * (size_t)nlow : 0) +
         2 * sizeof(Sup) + sizeof(T) * (size_t)(tile_elems(km) + (2 << km) * SL);
}

template <typename T, int NT, int MINB, int U>
__global__ void __launch_bounds__(NT, MINB) k_matvec_sb(Geo g, const T* __restrict__ x,
                                                        T* __restrict__ y, const double* d_sigma,
                                                        int shifted) {
  extern __shared__ __align__(16) char smem[];
  const int nlow = 1 << g.k;
  Low16* low = reinterpret_cast<Low16*>(smem);
  char* p = smem + sizeof(Low16) * nlow;
  double* dlw = nullptr;
  if constexpr (sizeof(T) == 8) {
    dlw = reinterpret_cast<double*>(p);
    p += sizeof(double) * nlow;
  }
  Sup* sh = reinterpret_cast<Sup*>(p);
  p += 2 * sizeof(Sup);
  const int nsl = 1 << g.km;          // slots per superblock
  T* tile = reinterpret_cast<T*>(p);  // slots of superblock 0, of superblock 1, zero slot
  T* zslot = tile + 2 * nsl * SL;
  T* G = zslot + SL;                  // phase-1 sums, same slots as the tile
  {
    const uint4* s = reinterpret_cast<const uint4*>(g.low);
    uint4* d = reinterpret_cast<uint4*>(low);
    for (int i = threadIdx.x; i < nlow; i += NT) d[i] = __ldg(s + i);
    if constexpr (sizeof(T) == 8)
      for (int i = threadIdx.x; i < nlow; i += NT) dlw[i] = __ldg(g.dlow + i);
    // the zero slot, and the last element of every slot (never staged: rows <= 251)
    for (int i = threadIdx.x; i < SL; i += NT) zslot[i] = T(0);
    for (int i = threadIdx.x; i < 2 * nsl; i += NT) tile[i * SL + ZSLOT] = T(0);
  }
  const double sigma = shifted ? *d_sigma : 0.0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = NT / 32;
  for (int pi = blockIdx.x; pi < g.npairs; pi += gridDim.x) {
    const int2 pr = g.pairs[pi];
    __syncthreads();  // the previous pair is done with sh, the tile and G
    if (threadIdx.x < 2 * SUP_WORDS) {
      const int s = threadIdx.x / SUP_WORDS, wd = threadIdx.x % SUP_WORDS;
      const int id = s ? pr.y : pr.x;
      reinterpret_cast<uint32_t*>(sh + s)[wd] =
          id >= 0 ? __ldg(reinterpret_cast<const uint32_t*>(g.sup + id) + wd) : 0u;
    }
    __syncthreads();
    // phase 1: stage x into the slots, sum the whole-superblock shifts into G
#pragma unroll 1
    for (int s = 0; s < 2; ++s)
      if (sh[s].C) sb_stage<T>(x + sh[s].R, g, (int)(sh[s].meta & 0xFF), tile + s * nsl * SL, warp, NW, lane);
#pragma unroll 1
    for (int s = 0; s < 2; ++s)
      if (sh[s].C) sb_phase1<T, U>(x + sh[s].R, sh[s], G + s * nsl * SL, threadIdx.x, NT);
    cp_async_wait_all();
    __syncthreads();
    // phase 2: one warp per sub-block, shared memory only
    const int nv0 = sh[0].C ? g.nvalid[sh[0].meta & 0xFF] : 0;
    const int nv1 = sh[1].C ? g.nvalid[sh[1].meta & 0xFF] : 0;
    for (int u = warp; u < nv0 + nv1; u += NW) {
      const int s = u >= nv0 ? 1 : 0;
      const int i = s ? u - nv0 : u;
      const Sup& H = sh[s];
      const uint32_t hm = H.meta;
      const int wq = (int)(hm & 0xFF);
      const int m = __ldg(g.order + (wq << g.km) + i);
      const Sub* B = g.sub + (wq << g.km) + m;
      const uint32_t bm = __ldg(&B->meta);
      const int w = (int)(bm & 0xFF);
      const int nmd = (int)((bm >> 8) & 0xFF);
      Lane<T> c;
      c.low = low + g.cls_off[w];
      if constexpr (sizeof(T) == 8) c.dlow = dlw + g.cls_off[w];
      else c.dlow = nullptr;
      c.tl = tile + (s * nsl + m) * SL;
      c.tg = G + s * nsl * SL + __ldg(&B->lo);
      c.tp = tile + ((1 - s) * nsl + m) * SL;
      c.yg = y + H.R + __ldg(&B->lo);
      c.zoff = (int32_t)(zslot - c.tl);
#pragma unroll
      for (int q = 0; q < MD_MAX; ++q) c.md[q] = q < nmd ? __ldg(&B->md[q]) : c.zoff;
      c.nmid = g.km - 1;
      c.C = g.cls_C[w];
      c.bdelta = __ldg(&B->bdelta);
      c.mbit0 = (bm >> 16) & 1u;
      c.ttop = (hm >> 17) & 1u;
      const uint32_t anti_ks = ((bm >> 17) & 1u) ^ ((hm >> 16) & 1u);
      c.uni = (T)(__ldg(&B->dmid) + H.dT - sigma + (anti_ks ? -0.25 : 0.25));
      sb_lane<T>(c, lane);
    }
  }
}

constexpr int NT_SB = 512;

// Device copy of one plan.
struct DevPlan {
  Geo geo{};
  void* mem = nullptr;  // one allocation holding every table
  int grid = 0;
  size_t smem = 0;
  int ok = 0;
};

template <typename T>
static auto kernel_of() {
  return k_matvec_sb<T, NT_SB, 2, 4>;
}

template <typename T>
static hs_status make_dev(hs_handle* hd, int KS, DevPlan** out) {
  *out = nullptr;
  HostPlan P;
  if (!build_plan(hd->L, hd->h, std::min(hd->k, K_MAX), KS, &P)) return HS_OK;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t s_low = al(P.low.size() * sizeof(Low16)), s_dlow = al(P.dlow.size() * sizeof(double)),
               s_sub = al(P.sub.size() * sizeof(Sub)), s_ord = al(P.order.size() * sizeof(uint16_t)),
               s_sup = al(P.sup.size() * sizeof(Sup)), s_pr = al(P.pairs.size() * sizeof(int2));
  const size_t total = s_low + s_dlow + s_sub + s_ord + s_sup + s_pr;
  std::vector<char> host(total, 0);
  size_t o = 0;
  auto put = [&](const void* src, size_t bytes, size_t slot) {
    std::memcpy(host.data() + o, src, bytes);
    const size_t at = o;
    o += slot;
    return at;
  };
  const size_t o_low = put(P.low.data(), P.low.size() * sizeof(Low16), s_low);
  const size_t o_dlow = put(P.dlow.data(), P.dlow.size() * sizeof(double), s_dlow);
  const size_t o_sub = put(P.sub.data(), P.sub.size() * sizeof(Sub), s_sub);
  const size_t o_ord = put(P.order.data(), P.order.size() * sizeof(uint16_t), s_ord);
  const size_t o_sup = put(P.sup.data(), P.sup.size() * sizeof(Sup), s_sup);
  const size_t o_pr = put(P.pairs.data(), P.pairs.size() * sizeof(int2), s_pr);
  DevPlan* d = new DevPlan();
  if (dev_alloc(hd, &d->mem, total) != HS_OK) {
    delete d;
    return fail(hd, HS_OOM, "superblock table allocation failed");
  }
  // pageable source: the copy is staged before the call returns
  if (cudaMemcpyAsync(d->mem, host.data(), total, cudaMemcpyHostToDevice, hd->stream) != cudaSuccess) {
    cudaGetLastError();
    dev_free(hd, d->mem);
    delete d;
    return fail(hd, HS_CUDA, "superblock table upload failed");
  }
  char* base = static_cast<char*>(d->mem);
  Geo& g = d->geo;
  g.low = reinterpret_cast<const Low16*>(base + o_low);
  g.dlow = reinterpret_cast<const double*>(base + o_dlow);
  g.sub = reinterpret_cast<const Sub*>(base + o_sub);
  g.order = reinterpret_cast<const uint16_t*>(base + o_ord);
  g.sup = reinterpret_cast<const Sup*>(base + o_sup);
  g.pairs = reinterpret_cast<const int2*>(base + o_pr);
  g.npairs = (int)P.pairs.size();
  g.k = P.k;
  g.km = P.km;
  g.KS = P.KS;
  for (int i = 0; i < K_MAX + 2; ++i) {
    g.cls_off[i] = P.cls_off[i];
    g.cls_C[i] = P.cls_C[i];
  }
  for (int i = 0; i <= WQ_MAX; ++i) g.nvalid[i] = P.nvalid[i];
  d->smem = smem_bytes<T>((int)P.low.size(), P.km);
  auto kern = kernel_of<T>();
  int nb = 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d->smem) ==
          cudaSuccess &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NT_SB, d->smem) == cudaSuccess &&
      nb > 0) {
    d->grid = std::min(g.npairs, nb * hd->num_sms);
    d->ok = 1;
  } else {
    cudaGetLastError();  // the tile does not fit: the plan stays unused
  }
  *out = d;
  return HS_OK;
}

}  // namespace sb

// Superblock windows of k + 4 bits (16 slots of 256 rows per superblock: x
// slots and sums of a pair take 65 KB in FP32, two CTAs per SM) and at most
// L - 10 bits, so that a chain has at least 512 superblock pairs to spread
// over the GPU. HS_SB_KS32 and HS_SB_KS64 override the window (tuning).
hs_status sb_setup(hs_handle* hd) {
  int ks32 = std::min(hd->k + 4, hd->L - 10), ks64 = std::min(hd->k + 3, hd->L - 10);
  if (const char* e = getenv("HS_SB_KS32")) ks32 = atoi(e);
  if (const char* e = getenv("HS_SB_KS64")) ks64 = atoi(e);
  sb::DevPlan* d = nullptr;
  hs_status st = sb::make_dev<float>(hd, ks32, &d);
  if (st != HS_OK) return st;
  hd->sb_plan[0] = d;
  st = sb::make_dev<double>(hd, ks64, &d);
  if (st != HS_OK) return st;
  hd->sb_plan[1] = d;
  return HS_OK;
}

void sb_release(hs_handle* hd) {
  for (int i = 0; i < 2; ++i) {
    auto* d = static_cast<sb::DevPlan*>(hd->sb_plan[i]);
    if (d) {
      dev_free(hd, d->mem);
      delete d;
    }
    hd->sb_plan[i] = nullptr;
  }
}

hs_status launch_matvec_sb(hs_handle* hd, const void* x, void* y, hs_dtype dt, int shifted,
                           bool* used) {
  *used = false;
  auto* d = static_cast<sb::DevPlan*>(hd->sb_plan[dt == HS_F32 ? 0 : 1]);
  if (!d || !d->ok) return HS_OK;
  const size_t es = dt == HS_F32 ? sizeof(float) : sizeof(double);
  if (((uintptr_t)x % es) != 0 || ((uintptr_t)y % es) != 0) return HS_OK;
  if (dt == HS_F32) {
    sb::kernel_of<float>()<<<d->grid, sb::NT_SB, d->smem, hd->stream>>>(
        d->geo, static_cast<const float*>(x), static_cast<float*>(y), hd->d_sigma, shifted);
  } else {
    sb::kernel_of<double>()<<<d->grid, sb::NT_SB, d->smem, hd->stream>>>(
        d->geo, static_cast<const double*>(x), static_cast<double*>(y), hd->d_sigma, shifted);
  }
  count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  *used = true;
  return HS_OK;
}

}  // namespace hs
