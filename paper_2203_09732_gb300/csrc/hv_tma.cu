// Matrix-free (H - sigma) x (Eq. (1)) with the gathers staged in shared memory
// by the bulk-copy (TMA) engine, for blocks of C(10, w) <= 252 rows (L >= 22).
//
// Each CTA walks its blocks in rank order through an S-stage pipeline. For a
// block, one producer thread bulk-copies every contiguous x segment the block
// reads: its own rows, the partner block of each antiparallel high-interior
// bond, the partner of the cut bond (k-1, k) and of the wrap bond (L-1, 0).
// The copies run S blocks ahead of the computation; the 256 threads then take
// one row each and read every operand from shared memory. The copy engine
// keeps far more bytes in flight per SM than per-thread gathers can, which is
// what limits the gather form at large L.
//
// Alignment: a bulk copy starts and ends on 16-byte boundaries, so each
// segment is widened to the enclosing 16-byte range (start rounded down, end
// rounded up, never past the last whole 16 bytes of x); the few elements
// beyond that (at most 3 FP32 / 1 FP64, only at the very end of x) are read by
// the producer with ordinary loads. Every wait on a stage barrier is bounded:
// on expiry the CTA records an error and leaves.
#include "rows.cuh"

namespace hs {

constexpr int TMA_THREADS = 256;
constexpr int TMA_SEG_MAX = HD_MAX + 3;   // self + high bonds + cut + wrap

struct TmaDesc {           // per stage, written by the producer
  uint32_t hdr[32];        // the block header (BlockInfo words)
  int32_t seg_off[TMA_SEG_MAX];   // element offset of segment data (incl. slack) in the stage buffer
  uint32_t cut_start;      // first row of the cut partner block
  int32_t nseg;
  int32_t block;           // block index, -1 = none
  int32_t pad;
};

__device__ __forceinline__ uint32_t s_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(s_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          s_addr(dst)),
      "l"(src), "r"(bytes), "r"(s_addr(b))
      : "memory");
}

// Producer: describe block bi in stage s and start its copies (thread 0 only).
template <typename T>
__device__ void tma_issue(const Geo& g, const T* __restrict__ x, int bi, TmaDesc* d, T* buf,
                          uint64_t* bar) {
  if (bi >= g.nblocks) {
    d->block = -1;
    __threadfence_block();
    mbar_arrive_tx(bar, 0);
    return;
  }
  const uint32_t* hsrc = reinterpret_cast<const uint32_t*>(g.blocks + bi);
#pragma unroll
  for (int i = 0; i < 32; ++i) d->hdr[i] = __ldg(hsrc + i);
  const uint32_t R = d->hdr[0], Rwrap = d->hdr[1];
  const int32_t bdelta = (int32_t)d->hdr[2];
  const uint32_t meta = d->hdr[3];
  const int w = meta & 0xFF, nh = (meta >> 8) & 0xFF, code = (meta >> 16) & 0xFF;
  const int k = g.k, C = g.cls_C[w];
  // segments: start row and length
  uint32_t st[TMA_SEG_MAX];
  int ln[TMA_SEG_MAX];
  int ns = 0;
  st[ns] = R; ln[ns++] = C;
  for (int m = 0; m < nh; ++m) { st[ns] = R + (uint32_t)(int32_t)d->hdr[6 + m]; ln[ns++] = C; }
  // cut partner: next block (H bit 0 clear, rows with bit k-1 set exist iff w >= 1)
  // or previous block (H bit 0 set, rows with bit k-1 clear exist iff w < k)
  bool cut = (code & 1) ? (w < k) : (w >= 1);
  uint32_t cs = R;
  int cl = 0;
  if (cut) {
    if (code & 1) { cl = g.cls_C[w + 1]; cs = R - (uint32_t)cl; }
    else { cl = g.cls_C[w - 1]; cs = R + (uint32_t)C; }
  }
  d->cut_start = cs;
  st[ns] = cs; ln[ns++] = cut ? cl : 0;
  // wrap partner: block H ^ top (class w - 1 if the top bit is clear, w + 1 if set)
  const bool ht = (code >> 1) & 1;
  const bool wrap = ht ? (w < k) : (w >= 1);
  st[ns] = Rwrap; ln[ns++] = wrap ? g.cls_C[ht ? w + 1 : w - 1] : 0;
  (void)bdelta;
  d->nseg = ns;
  d->block = bi;
  const uint64_t nbytes = (uint64_t)g.n * sizeof(T);
  const uint64_t whole = nbytes & ~uint64_t(15);   // last whole 16-byte boundary of x
  unsigned total = 0;
  int off = 0;   // in elements, 16-byte aligned
  const char* xb = reinterpret_cast<const char*>(x);
  for (int sg = 0; sg < ns; ++sg) {
    if (ln[sg] == 0) { d->seg_off[sg] = off; continue; }
    const uint64_t a = (uint64_t)st[sg] * sizeof(T);
    const uint64_t e = a + (uint64_t)ln[sg] * sizeof(T);
    const uint64_t lo = a & ~uint64_t(15);
    uint64_t hi = (e + 15) & ~uint64_t(15);
    if (hi > whole) hi = whole;
    const int slack = (int)((a - lo) / sizeof(T));
    d->seg_off[sg] = off + slack;
    if (hi > lo) {
      bulk_g2s(buf + off, xb + lo, (unsigned)(hi - lo), bar);
      total += (unsigned)(hi - lo);
    }
    // elements past the last whole 16 bytes of x (only at the very end)
    for (uint64_t p = (hi > lo ? hi : lo); p < e; p += sizeof(T))
      buf[off + (int)((p - lo) / sizeof(T))] = __ldg(reinterpret_cast<const T*>(xb + p));
    off += (int)((((e - lo) + 15) & ~uint64_t(15)) / sizeof(T));
  }
  __threadfence_block();
  mbar_arrive_tx(bar, total);
}

template <typename T, int S>
__global__ void __launch_bounds__(TMA_THREADS) k_matvec_tma(Geo g, const T* __restrict__ x,
                                                            T* __restrict__ y,
                                                            const double* d_sigma, int shifted,
                                                            int stage_elems, int* err,
                                                            unsigned long long limit) {
  extern __shared__ __align__(128) char smem[];
  __shared__ __align__(8) uint64_t bars[S];
  __shared__ TmaDesc desc[S];
  LowEntry* low = reinterpret_cast<LowEntry*>(smem);
  {
    const uint4* src = reinterpret_cast<const uint4*>(g.low);
    uint4* dst = reinterpret_cast<uint4*>(low);
    for (int i = threadIdx.x; i < g.nlow * 2; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  T* stage0 = reinterpret_cast<T*>(smem + ((sizeof(LowEntry) * g.nlow + 127) & ~size_t(127)));
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const double sigma = shifted ? *d_sigma : 0.0;
  const int G = gridDim.x;
  if (threadIdx.x == 0)
    for (int s = 0; s < S; ++s)
      tma_issue<T>(g, x, blockIdx.x + s * G, &desc[s], stage0 + (size_t)s * stage_elems, &bars[s]);
  const int r = threadIdx.x;
  for (int t = 0;; ++t) {
    const int s = t % S;
    const unsigned parity = (unsigned)((t / S) & 1);
    // bounded wait for the stage's copies
    bool ok = true;
    unsigned long long it = 0;
    while (!mbar_try(&bars[s], parity)) {
      if (++it > limit) { ok = false; break; }
    }
    if (__syncthreads_or(!ok)) {
      // give up: record the error, then wait (bounded) for the copies this CTA
      // still has in flight (stages of blocks t .. t+S-1) before leaving, so
      // that no bulk copy lands in shared memory after the CTA is gone
      if (threadIdx.x == 0) {
        atomicExch(err, 1);
        for (int j = 0; j < S; ++j) {
          const int sj = (t + j) % S;
          const unsigned pj = (unsigned)(((t + j) / S) & 1);
          unsigned long long w2 = 0;
          while (!mbar_try(&bars[sj], pj) && ++w2 <= limit) {
          }
        }
      }
      __syncthreads();
      return;
    }
    const TmaDesc& d = desc[s];
    if (d.block < 0) break;
    const T* buf = stage0 + (size_t)s * stage_elems;
    const uint32_t word = d.hdr[threadIdx.x & 31];
    const Hdr h = make_hdr(g, word, sigma);
    if (r < h.C) {
      const LowEntry& e = low[h.off + r];
      const uint32_t pk = e.packed;
      const uint32_t xc = cut_mask(pk, h);
      const T* self = buf + d.seg_off[0];
      const T xi = self[r];
      T acc = T(0);
      for (int m = 0; m < h.nh; ++m) acc += buf[d.seg_off[1 + m] + r];
      if (xc & 1u)
        acc += buf[d.seg_off[h.nh + 1] + (int)(h.R + (uint32_t)r + (uint32_t)h.bdelta - d.cut_start)];
      if (xc & 2u) acc += buf[d.seg_off[h.nh + 2] + (int)e.wrap_r];
      const int cnt = le_cnt(pk);
      const uint32_t w0 = e.nbw[0], w1 = e.nbw[1], w2 = e.nbw[2];
#pragma unroll
      for (int mm = 0; mm < NB_MAX; ++mm) {
        const uint32_t wd = mm < 4 ? w0 : (mm < 8 ? w1 : w2);
        if (mm < cnt) acc += self[(wd >> (8 * (mm & 3))) & 0xFFu];
      }
      __stcs(y + h.R + r, diag_t<T>(e, h, xc) * xi + T(0.5) * acc);
    }
    __syncthreads();   // stage s fully read before it is refilled
    if (threadIdx.x == 0)
      tma_issue<T>(g, x, blockIdx.x + (t + S) * G, &desc[s], stage0 + (size_t)s * stage_elems,
                   &bars[s]);
  }
  // No copy is in flight here: the stages issued after the last block (all
  // later block indices are past the end too) were armed with zero bytes.
}

// Host side ------------------------------------------------------------------
template <typename T, int S>
static hs_status launch_tma_t(hs_handle* hd, const T* x, T* y, int shifted, bool* used) {
  *used = false;
  const int hb = hd->hb;
  const int segmax = (hb - 1) + 3;
  const int cmax = 252;
  const int stage_elems = segmax * (cmax + 32 / (int)sizeof(T) + 16 / (int)sizeof(T));
  const size_t tab = (sizeof(LowEntry) * hd->low.size() + 127) & ~size_t(127);
  const size_t sm = tab + (size_t)S * stage_elems * sizeof(T);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, hd->device);
  if (sm + sizeof(TmaDesc) * S + 64 > (size_t)optin) return HS_OK;
  auto kern = k_matvec_tma<T, S>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
      cudaSuccess) {
    cudaGetLastError();
    return HS_OK;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TMA_THREADS, sm);
  if (per_sm < 1) return HS_OK;
  const int grid = std::max(1, std::min((int)hd->blocks.size(), per_sm * hd->num_sms));
  hs_status st = ensure_reduce(hd);
  if (st != HS_OK) return st;
  int* err = reinterpret_cast<int*>(hd->d_counter + 12);
  HS_CUDA_TRY(hd, cudaMemsetAsync(err, 0, sizeof(int), hd->stream));
  const unsigned long long limit = 1ull << 20;   // try_wait polls (each may suspend briefly)
  kern<<<grid, TMA_THREADS, sm, hd->stream>>>(hd->geo(), x, y, hd->d_sigma, shifted, stage_elems,
                                              err, limit);
  count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  *used = true;
  return HS_OK;
}

// Returns HS_OK with *used = false when the staged form does not apply.
hs_status launch_matvec_tma(hs_handle* hd, const void* x, void* y, hs_dtype dt, int shifted,
                            bool* used) {
  *used = false;
  if (hd->k != 10) return HS_OK;
  if (dt == HS_F32)
    return launch_tma_t<float, 4>(hd, static_cast<const float*>(x), static_cast<float*>(y),
                                  shifted, used);
  return launch_tma_t<double, 3>(hd, static_cast<const double*>(x), static_cast<double*>(y),
                                 shifted, used);
}

}  // namespace hs
