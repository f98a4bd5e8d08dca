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
#include "sb4_kern.cuh"
#include "sb_kern.cuh"

namespace hs {
namespace sb {

constexpr int NT_SB = 512;

// The product kernel for a plan with km mid bits: the mid-bond count as a
// compile-time constant for the windows the library uses (km = 4), else read
// from the plan.
template <typename T>
static auto kernel_of(int km) {
  return km == 4 ? k_sbhv<T, NT_SB, 2, 4, MODE_HV, 3> : k_sbhv<T, NT_SB, 2, 4, MODE_HV, 0>;
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
  auto kern = kernel_of<T>(P.km);
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

namespace sb4 {

constexpr int NT4_F = 512;   // FP32: two CTAs of 512 threads per SM
constexpr int NT4_D = 256;   // FP64: more registers per thread

// The kernel for a plan: the mid loop unrolled for the library's windows
// (10 mid bits in FP32, 9 in FP64), a run-time loop for other windows.
template <typename T, int MODE>
using K4 = void (*)(Geo4, const T*, T*, const double*, int, sb::MinresArgs);
template <typename T, int MODE>
K4<T, MODE> kernel4_for(int km) {
  if constexpr (sizeof(T) == 8) {
    if (km == 9) return k_sb4<double, NT4_D, 2, 4, MODE, 9>;
    return k_sb4<double, NT4_D, 2, 4, MODE, 0>;
  } else {
    if (km == 10) return k_sb4<float, NT4_F, 2, 4, MODE, 10>;
    return k_sb4<float, NT4_F, 2, 4, MODE, 0>;
  }
}

template <typename T>
static hs_status make_dev4(hs_handle* hd, int KS, DevPlan4** out) {
  *out = nullptr;
  HostPlan4 P;
  if (!build_plan4(hd->L, hd->h, KS, &P)) return HS_OK;
  const sb::HostPlan& B = P.base;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  struct Part { const void* src; size_t bytes; size_t at; };
  std::vector<Part> parts = {
      {B.sup.data(), B.sup.size() * sizeof(sb::Sup), 0},
      {B.pairs.data(), B.pairs.size() * sizeof(int2), 0},
      {P.slotmap.data(), P.slotmap.size() * sizeof(uint16_t), 0},
      {P.order.data(), P.order.size() * sizeof(uint16_t), 0},
      {P.lo.data(), P.lo.size() * sizeof(uint16_t), 0},
      {P.dmid_f.data(), P.dmid_f.size() * sizeof(float), 0},
      {P.dmid_d.data(), P.dmid_d.size() * sizeof(double), 0},
      {P.dl_f.data(), P.dl_f.size() * sizeof(float), 0},
      {P.dl_d.data(), P.dl_d.size() * sizeof(double), 0}};
  size_t total = 0;
  for (Part& q : parts) {
    q.at = total;
    total += al(q.bytes);
  }
  std::vector<char> host(total, 0);
  for (const Part& q : parts) std::memcpy(host.data() + q.at, q.src, q.bytes);
  DevPlan4* d = new DevPlan4();
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
  Geo4& g = d->geo;
  g.sup = reinterpret_cast<const sb::Sup*>(base + parts[0].at);
  g.pairs = reinterpret_cast<const int2*>(base + parts[1].at);
  g.slotmap = reinterpret_cast<const uint16_t*>(base + parts[2].at);
  g.order = reinterpret_cast<const uint16_t*>(base + parts[3].at);
  g.lo = reinterpret_cast<const uint16_t*>(base + parts[4].at);
  g.dmid_f = reinterpret_cast<const float*>(base + parts[5].at);
  g.dmid_d = reinterpret_cast<const double*>(base + parts[6].at);
  g.dl_f = reinterpret_cast<const float*>(base + parts[7].at);
  g.dl_d = reinterpret_cast<const double*>(base + parts[8].at);
  g.npairs = (int)B.pairs.size();
  g.km = B.km;
  g.KS = B.KS;
  g.cmax = P.cmax;
  for (int i = 0; i <= WQ_MAX; ++i) {
    g.slot_off[i] = P.slot_off[i];
    g.order_off[i] = P.order_off[i];
    g.nvalid[i] = P.nvalid[i];
  }
  g.dscale = B.dscale;
  d->smem = smem_bytes4<T>(g.km, g.cmax);
  auto kern = kernel4_for<T, sb::MODE_HV>(g.km);
  const int nt = sizeof(T) == 8 ? NT4_D : NT4_F;
  int nb = 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d->smem) ==
          cudaSuccess &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, nt, d->smem) == cudaSuccess &&
      nb > 0) {
    d->grid = std::min(g.npairs, nb * hd->num_sms);
    d->ok = 1;
  } else {
    cudaGetLastError();
  }
  *out = d;
  return HS_OK;
}

}  // namespace sb4

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
  // four-low-bit plans (sb4.cuh): 14-bit windows in FP32, 13 in FP64 (the
  // slots and sums of a pair take about 96 KB either way); HS_SB4_KS32 and
  // HS_SB4_KS64 override them (tests of small chains)
  int k32 = std::min(14, hd->L - 6), k64 = std::min(13, hd->L - 6);
  if (const char* e = getenv("HS_SB4_KS32")) k32 = atoi(e);
  if (const char* e = getenv("HS_SB4_KS64")) k64 = atoi(e);
  sb4::DevPlan4* d4 = nullptr;
  if ((st = sb4::make_dev4<float>(hd, k32, &d4)) != HS_OK) return st;
  hd->sb4_plan[0] = d4;
  if ((st = sb4::make_dev4<double>(hd, k64, &d4)) != HS_OK) return st;
  hd->sb4_plan[1] = d4;
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
    auto* d4 = static_cast<sb4::DevPlan4*>(hd->sb4_plan[i]);
    if (d4) {
      dev_free(hd, d4->mem);
      delete d4;
    }
    hd->sb4_plan[i] = nullptr;
  }
}

}  // namespace hs

// The four-low-bit form is the FP64 default (measured at L = 24..28 it is the
// fastest FP64 product: fewer FP64 additions of zeros than the ten-bit form,
// and no gathers from global memory for most bonds, unlike the block form);
// in FP32 the ten-bit form is faster. HS_SB4=1 / 0 selects it, or not, for
// both precisions (tests compare forms).
bool hs_want_sb4(hs_dtype dt) {
  const char* e = getenv("HS_SB4");
  if (e) return e[0] == '1';
  return dt == HS_F64;
}

namespace hs {

hs_status launch_matvec_sb(hs_handle* hd, const void* x, void* y, hs_dtype dt, int shifted,
                           bool* used) {
  *used = false;
  {
    auto* d4 = static_cast<sb4::DevPlan4*>(hd->sb4_plan[dt == HS_F32 ? 0 : 1]);
    const size_t es = dt == HS_F32 ? sizeof(float) : sizeof(double);
    if (hs_want_sb4(dt) && d4 && d4->ok && ((uintptr_t)x % es) == 0 && ((uintptr_t)y % es) == 0) {
      const sb::MinresArgs none{};
      if (dt == HS_F32)
        sb4::kernel4_for<float, sb::MODE_HV>(d4->geo.km)<<<d4->grid, sb4::NT4_F, d4->smem,
                                                            hd->stream>>>(
            d4->geo, static_cast<const float*>(x), static_cast<float*>(y), hd->d_sigma, shifted,
            none);
      else
        sb4::kernel4_for<double, sb::MODE_HV>(d4->geo.km)<<<d4->grid, sb4::NT4_D, d4->smem,
                                                             hd->stream>>>(
            d4->geo, static_cast<const double*>(x), static_cast<double*>(y), hd->d_sigma, shifted,
            none);
      count_launches(1);
      HS_CUDA_TRY(hd, cudaGetLastError());
      *used = true;
      return HS_OK;
    }
  }
  auto* d = static_cast<sb::DevPlan*>(hd->sb_plan[dt == HS_F32 ? 0 : 1]);
  if (!d || !d->ok) return HS_OK;
  const size_t es = dt == HS_F32 ? sizeof(float) : sizeof(double);
  if (((uintptr_t)x % es) != 0 || ((uintptr_t)y % es) != 0) return HS_OK;
  const sb::MinresArgs none{};
  if (dt == HS_F32) {
    sb::kernel_of<float>(d->geo.km)<<<d->grid, sb::NT_SB, d->smem, hd->stream>>>(
        d->geo, static_cast<const float*>(x), static_cast<float*>(y), hd->d_sigma, shifted, none);
  } else {
    sb::kernel_of<double>(d->geo.km)<<<d->grid, sb::NT_SB, d->smem, hd->stream>>>(
        d->geo, static_cast<const double*>(x), static_cast<double*>(y), hd->d_sigma, shifted, none);
  }
  count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  *used = true;
  return HS_OK;
}

}  // namespace hs
