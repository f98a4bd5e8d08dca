// Superblock form of y = (H - sigma) x (Eq. (1)) for long chains: one CTA per
// superblock pair {T, T ^ top}. Phase 1 stages x of the pair into shared
// memory by asynchronous copies while it sums the high-bit and (KS-1, KS)
// flips of every row from global memory (coalesced shifted streams); phase 2
// walks the sub-blocks and reads shared memory only. Layout and bond kinds:
// sb.cuh; the kernel (shared with MINRES pass A): sb_kern.cuh. This file
// builds the plans and launches the product.
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "sb.cuh"
#include "sb_kern.cuh"

namespace hs {
namespace sb {

constexpr int NT_SB = 512;

template <typename T>
static auto kernel_of() {
  return k_sbhv<T, NT_SB, 2, 4, MODE_HV>;
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
  g.dscale = P.dscale;
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
  const sb::MinresArgs none{};
  if (dt == HS_F32) {
    sb::kernel_of<float>()<<<d->grid, sb::NT_SB, d->smem, hd->stream>>>(
        d->geo, static_cast<const float*>(x), static_cast<float*>(y), hd->d_sigma, shifted, none);
  } else {
    sb::kernel_of<double>()<<<d->grid, sb::NT_SB, d->smem, hd->stream>>>(
        d->geo, static_cast<const double*>(x), static_cast<double*>(y), hd->d_sigma, shifted, none);
  }
  count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  *used = true;
  return HS_OK;
}

}  // namespace hs
