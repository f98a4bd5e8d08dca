// Two-level ("superblock") form of the matrix-free product (H - sigma) x of
// Eq. (1) for long chains.
//
// A state word s of the Sz = 0 sector is split into three fields:
//   p = low k bits, m = the next km bits ("mid"), T = the top tb = L - KS bits,
//   KS = k + km.
// Because the rank is the ascending-integer (colex) order of the sector, all
// states with the same T form one contiguous rank range (a superblock) of
// C(KS, wq) rows, wq = L/2 - popcount(T); inside it, the states with the same m
// form a contiguous sub-block of C(k, w) rows, w = wq - popcount(m), ordered
// by the colex rank r of p. The L bonds of Eq. (1) fall into six kinds:
//   low interior  (j, j+1), j + 1 < k    : same sub-block, r -> r' (per-pattern table);
//   cut (k-1, k)                         : sub-block m ^ 1, r -> r -+ C(k-1, .);
//   mid interior  (j, j+1), k <= j < KS-1 : sub-block m ^ (3 << (j-k)), same r;
//   wrap (L-1, 0)                        : superblock T ^ top (the "partner"),
//                                          sub-block m, rank of p ^ 1;
//   bond (KS-1, KS)                      : superblock T ^ 1, one contiguous half
//                                          of the superblock shifted as a whole;
//   high interior (j, j+1), j >= KS      : superblock T', the whole superblock
//                                          shifted as a whole.
// A CTA takes the superblock pair {T, T ^ top}. Phase 1 stages x of the pair
// into shared memory with asynchronous copies (one warp per sub-block, a
// contiguous run of rows each) and, over the pair's rows in rank order with
// many loads in flight, sums the last two kinds, which are the same shift for
// whole superblocks, into a second shared buffer G. Phase 2 walks the
// sub-blocks (one warp each, lane l takes rows l + 32 j) and reads shared
// memory only. In shared memory each sub-block of x has a slot of SL = 256
// elements (rows 0..C(k, w)-1 <= 251); the last element of every slot and one
// whole extra slot stay zero, so a row reads a zero instead of branching where
// a bond is parallel or a neighbour-list entry is unused.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

namespace hs {
namespace sb {

constexpr int K_MAX = 10;     // low bits (C(10, 5) = 252 rows fit a slot)
constexpr int KM_MAX = 8;     // mid bits (slot index m << 8 | r fits 16 bits)
constexpr int MD_MAX = KM_MAX - 1;
constexpr int HH_MAX = 16;    // high interior bonds (tb <= 17)
constexpr int JMAX = 8;       // rows per lane of one sub-block (C(k, w) <= 256)
constexpr int WQ_MAX = 24;    // superblock classes wq = 0 .. KS
constexpr int SL = 256;       // slot length (elements)
constexpr int ZSLOT = SL - 1; // always-zero element of every slot

// One entry per low pattern p, index cls_off[w] + colex rank of p; 16 bytes.
struct Low16 {
  float dlow_f;      // Ising terms of the low interior bonds + fields on sites 0..k-1
  uint32_t nb0, nb1; // neighbour ranks 0..7 of the low interior flips, 8 bits each
  uint32_t meta;     // neighbour 8 | wrap_r << 8 | count << 16 | code << 20
};
static_assert(sizeof(Low16) == 16, "Low16 is 16 bytes");
// Unused neighbour entries hold ZSLOT. code: bit 0 = bit k-1 of p, bit 1 =
// bit 0 of p; wrap_r = colex rank of p ^ 1.

// One entry per (superblock class wq, mid pattern m), index wq << km | m; 64 bytes.
struct Sub {
  uint32_t lo;       // first row of sub-block m inside a class-wq superblock
  int32_t bdelta;    // slot-relative offset of the cut-bond (k-1, k) flip
  uint32_t meta;     // w | nmd << 8 | (m & 1) << 16 | mtop bit << 17 | valid << 24
  float dmid_f;      // dmid rounded to FP32 (the FP32 kernels' diagonal)
  double dmid;       // Ising terms of the mid interior bonds + fields on sites k..KS-1
  int32_t md[MD_MAX];  // slot-relative offsets of the antiparallel mid interior flips
  uint32_t pad[3];
};
static_assert(sizeof(Sub) == 64, "Sub is 64 bytes");

// One entry per valid top pattern T, in ascending T; 96 bytes.
struct Sup {
  uint32_t R;        // first row
  uint32_t C;        // rows, C(KS, wq)
  uint32_t meta;     // wq | nh << 8 | (T & 1) << 16 | top bit << 17
  uint32_t ka;       // rows [ka, kb) flip bond (KS-1, KS) ...
  double dT;         // Ising terms of the high interior bonds + fields on sites KS..L-1
  int32_t hd[HH_MAX];  // row offsets of the antiparallel high interior flips
  uint32_t kb;
  int32_t kd;        // ... to row + kd (in superblock T ^ 1)
};
static_assert(sizeof(Sup) == 96, "Sup is 96 bytes");
constexpr int SUP_WORDS = sizeof(Sup) / 4;

// Everything the kernel needs, passed by value.
struct Geo {
  const Low16* low;
  const double* dlow;          // FP64 Ising + field terms of the low table
  const Sub* sub;
  const uint16_t* order;       // per class wq: valid m sorted by decreasing sub-block size
  const Sup* sup;
  const int2* pairs;           // superblock indices {T0, T0 | top}, -1 where absent
  int npairs, k, km, KS;
  int cls_off[K_MAX + 2];
  int cls_C[K_MAX + 2];
  int nvalid[WQ_MAX + 1];      // valid m per class
  double dscale;               // L/4 + sum_j |h_j| / 2: bound of |a_ii|
};

// Host tables of one plan.
struct HostPlan {
  int k = 0, km = 0, KS = 0, tb = 0;
  std::vector<Low16> low;
  std::vector<double> dlow;
  std::vector<Sub> sub;
  std::vector<uint16_t> order;
  std::vector<Sup> sup;
  std::vector<int2> pairs;
  int cls_off[K_MAX + 2] = {0};
  int cls_C[K_MAX + 2] = {0};
  int nvalid[WQ_MAX + 1] = {0};
  double dscale = 0.0;
};

inline uint64_t binom64(int n, int r) {
  if (r < 0 || n < 0 || r > n) return 0;
  uint64_t v = 1;
  for (int i = 1; i <= r; ++i) v = v * (uint64_t)(n - r + i) / (uint64_t)i;
  return v;
}

inline int colex_rank_host(uint32_t p) {
  int r = 0, c = 1;
  while (p) {
    int pos = 0;
    while (!((p >> pos) & 1u)) ++pos;
    r += (int)binom64(pos, c);
    ++c;
    p &= p - 1u;
  }
  return r;
}

inline int popc_host(uint32_t v) {
  int c = 0;
  for (; v; v &= v - 1u) ++c;
  return c;
}

// Build the plan for chain length L with fields h[0..L-1], k low bits and a
// KS-bit window. Returns false (and leaves the plan empty) if the split does
// not apply: needs 2 <= k <= K_MAX, 1 <= KS - k <= km_max, 2 <= L - KS <= HH_MAX + 1.
// The per-sub-block mid offsets (Sub::md, read by the product of this file)
// are filled only for km <= KM_MAX; a larger km_max serves sb4.cuh, which
// finds mid neighbours by bit arithmetic instead.
inline bool build_plan(int L, const double* h, int k, int KS, HostPlan* P, int km_max = KM_MAX) {
  *P = HostPlan{};
  const int N = L / 2, km = KS - k, tb = L - KS;
  if (k < 2 || k > K_MAX || km < 1 || km > km_max || tb < 2 || tb - 1 > HH_MAX || KS > WQ_MAX)
    return false;
  P->k = k;
  P->km = km;
  P->KS = KS;
  P->tb = tb;
  P->dscale = 0.25 * L;
  for (int j = 0; j < L; ++j) P->dscale += 0.5 * (h[j] < 0 ? -h[j] : h[j]);
  // low patterns
  int off = 0;
  for (int w = 0; w <= k; ++w) {
    P->cls_off[w] = off;
    P->cls_C[w] = (int)binom64(k, w);
    off += P->cls_C[w];
  }
  P->low.assign((size_t)1 << k, Low16{});
  P->dlow.assign((size_t)1 << k, 0.0);
  std::vector<int> fill(k + 1, 0);
  for (uint32_t p = 0; p < (1u << k); ++p) {
    const int w = popc_host(p);
    const int li = P->cls_off[w] + fill[w]++;
    Low16 e{};
    double d = 0.0;
    int cnt = 0;
    uint32_t nb[9];
    for (int q = 0; q < 9; ++q) nb[q] = (uint32_t)ZSLOT;
    for (int j = 0; j + 1 < k; ++j) {
      const int a = (p >> j) & 1, b = (p >> (j + 1)) & 1;
      if (a == b) {
        d += 0.25;
      } else {
        d -= 0.25;
        nb[cnt++] = (uint32_t)colex_rank_host(p ^ (3u << j));
      }
    }
    for (int j = 0; j < k; ++j) d -= h[j] * (((p >> j) & 1) ? 0.5 : -0.5);
    e.dlow_f = (float)d;
    e.nb0 = nb[0] | nb[1] << 8 | nb[2] << 16 | nb[3] << 24;
    e.nb1 = nb[4] | nb[5] << 8 | nb[6] << 16 | nb[7] << 24;
    const uint32_t code = ((p >> (k - 1)) & 1u) | ((p & 1u) << 1);
    e.meta = nb[8] | (uint32_t)colex_rank_host(p ^ 1u) << 8 | (uint32_t)cnt << 16 | code << 20;
    P->low[li] = e;
    P->dlow[li] = d;
  }
  // sub-blocks: lo(wq, m) = rows of the valid m' < m
  const int nm = 1 << km;
  const int nwq = KS + 1;
  std::vector<int64_t> lo((size_t)nwq * nm, -1);
  for (int wq = 0; wq < nwq; ++wq) {
    int64_t acc = 0;
    for (int m = 0; m < nm; ++m) {
      const int w = wq - popc_host((uint32_t)m);
      if (w < 0 || w > k) continue;
      lo[(size_t)wq * nm + m] = acc;
      acc += (int64_t)binom64(k, w);
    }
  }
  P->sub.assign((size_t)nwq * nm, Sub{});
  P->order.assign((size_t)nwq * nm, 0);
  const uint32_t mtop = 1u << (km - 1);
  for (int wq = 0; wq < nwq; ++wq) {
    std::vector<int> valid;
    for (int m = 0; m < nm; ++m) {
      Sub b{};
      const int w = wq - popc_host((uint32_t)m);
      if (w < 0 || w > k) {
        P->sub[(size_t)wq * nm + m] = b;
        continue;
      }
      valid.push_back(m);
      b.lo = (uint32_t)lo[(size_t)wq * nm + m];
      double d = 0.0;
      int nmd = 0;
      for (int j = 0; j + 1 < km; ++j) {
        const int a = (m >> j) & 1, c2 = (m >> (j + 1)) & 1;
        if (a == c2) {
          d += 0.25;
        } else {
          d -= 0.25;
          if (km <= KM_MAX) b.md[nmd] = ((m ^ (3 << j)) - m) * SL;
          ++nmd;
        }
      }
      for (int j = 0; j < km; ++j) d -= h[k + j] * (((m >> j) & 1) ? 0.5 : -0.5);
      b.dmid = d;
      b.dmid_f = (float)d;
      // cut (k-1, k): flips bit k-1 of p and bit 0 of m
      if (m & 1) {  // p gains bit k-1: rank + C(k-1, w+1), in sub-block m ^ 1 (class w + 1)
        b.bdelta = (w + 1 <= k) ? -SL + (int32_t)binom64(k - 1, w + 1) : 0;
      } else {      // p loses bit k-1: rank - C(k-1, w), in sub-block m | 1 (class w - 1)
        b.bdelta = (w >= 1) ? SL - (int32_t)binom64(k - 1, w) : 0;
      }
      b.meta = (uint32_t)w | (uint32_t)nmd << 8 | (uint32_t)(m & 1) << 16 |
               (uint32_t)((m & mtop) ? 1 : 0) << 17 | 1u << 24;
      P->sub[(size_t)wq * nm + m] = b;
    }
    std::stable_sort(valid.begin(), valid.end(), [&](int a, int b) {
      return binom64(k, wq - popc_host((uint32_t)a)) > binom64(k, wq - popc_host((uint32_t)b));
    });
    P->nvalid[wq] = (int)valid.size();
    for (size_t i = 0; i < valid.size(); ++i) P->order[(size_t)wq * nm + i] = (uint16_t)valid[i];
  }
  // superblocks in ascending T (= rank order)
  const uint32_t nT = 1u << tb;
  std::vector<int> idx(nT, -1);
  std::vector<uint32_t> RofT(nT, 0);
  uint64_t R = 0;
  for (uint32_t T = 0; T < nT; ++T) {
    const int wq = N - popc_host(T);
    if (wq < 0 || wq > KS) continue;
    idx[T] = (int)P->sup.size();
    RofT[T] = (uint32_t)R;
    Sup s{};
    s.R = (uint32_t)R;
    s.C = (uint32_t)binom64(KS, wq);
    P->sup.push_back(s);
    R += s.C;
  }
  if (R != binom64(L, N)) return *P = HostPlan{}, false;
  for (uint32_t T = 0; T < nT; ++T) {
    if (idx[T] < 0) continue;
    Sup& s = P->sup[(size_t)idx[T]];
    const int wq = N - popc_host(T);
    double d = 0.0;
    int nh = 0;
    for (int t = 0; t + 1 < tb; ++t) {
      const int a = (T >> t) & 1, c2 = (T >> (t + 1)) & 1;
      if (a == c2) {
        d += 0.25;
      } else {
        d -= 0.25;
        const uint32_t T2 = T ^ (3u << t);
        s.hd[nh++] = (int32_t)((int64_t)RofT[T2] - (int64_t)s.R);
      }
    }
    for (int t = 0; t < tb; ++t) d -= h[KS + t] * (((T >> t) & 1) ? 0.5 : -0.5);
    s.dT = d;
    // bond (KS-1, KS) flips bit KS-1 of the window and bit 0 of T. The window
    // patterns with bit KS-1 clear are the first C(KS-1, wq) ranks.
    const uint32_t cl = (uint32_t)binom64(KS - 1, wq);
    if (idx[T ^ 1u] < 0) {
      s.ka = s.kb = 0;
      s.kd = 0;
    } else if (T & 1u) {  // rows with bit KS-1 clear gain it: rank + C(KS-1, wq+1)
      s.ka = 0;
      s.kb = cl;
      s.kd = (int32_t)((int64_t)RofT[T ^ 1u] - (int64_t)s.R + (int64_t)binom64(KS - 1, wq + 1));
    } else {              // rows with bit KS-1 set lose it: rank - C(KS-1, wq)
      s.ka = cl;
      s.kb = s.C;
      s.kd = (int32_t)((int64_t)RofT[T ^ 1u] - (int64_t)s.R - (int64_t)cl);
    }
    s.meta = (uint32_t)wq | (uint32_t)nh << 8 | (T & 1u) << 16 | ((T >> (tb - 1)) & 1u) << 17;
  }
  // pairs {T0, T0 | top}: largest first, then by the popcount of T0 (neighbouring
  // superblocks share it, which keeps their rows close in time), then by T0
  const uint32_t top = 1u << (tb - 1);
  struct Key { uint32_t rows; int pc; uint32_t T0; };
  std::vector<Key> keys;
  for (uint32_t T0 = 0; T0 < top; ++T0) {
    const int a = idx[T0], b = idx[T0 | top];
    if (a < 0 && b < 0) continue;
    const uint32_t rows = (a >= 0 ? P->sup[a].C : 0u) + (b >= 0 ? P->sup[b].C : 0u);
    keys.push_back({rows, popc_host(T0), T0});
  }
  std::sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
    if (a.rows != b.rows) return a.rows > b.rows;
    if (a.pc != b.pc) return a.pc < b.pc;
    return a.T0 < b.T0;
  });
  for (const Key& q : keys) P->pairs.push_back(make_int2(idx[q.T0], idx[q.T0 | top]));
  return true;
}

// Shared-memory layout of one CTA (elements of T): the slots of superblock 0,
// the slots of superblock 1, one zero slot; G (phase-1 sums) mirrors the
// first two.
__host__ __device__ inline int tile_elems(int km) { return (2 << km) * SL + SL; }

// ---------------------------------------------------------------------------
// Device/host helpers, so that the same row code runs in the kernel and in
// host checks.
#ifdef __CUDA_ARCH__
template <typename T> __device__ __forceinline__ T sb_ldg(const T* p) { return __ldg(p); }
template <typename T> __device__ __forceinline__ void sb_st(T* p, T v) { __stcs(p, v); }
template <typename T>
__device__ __forceinline__ void sb_copy(T* dst, const T* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "n"(sizeof(T))
               : "memory");
}
#else
template <typename T> inline T sb_ldg(const T* p) { return *p; }
template <typename T> inline void sb_st(T* p, T v) { *p = v; }
template <typename T> inline void sb_copy(T* dst, const T* src) { *dst = *src; }
#endif

// Stage the x rows of one superblock (xs[0, C), class wq) into its slots:
// warp wp of nw copies the sub-blocks wp, wp + nw, ... of the class's order
// list, each a contiguous run of rows, lane l the rows l + 32 j.
template <typename T>
__host__ __device__ __forceinline__ void sb_stage(const T* xs, const Geo& g, int wq, T* slots,
                                                  int wp, int nw, int lane) {
  const int nv = g.nvalid[wq];
  for (int u = wp; u < nv; u += nw) {
    const int m = sb_ldg(g.order + (wq << g.km) + u);
    const Sub* B = g.sub + (wq << g.km) + m;
    const int C = g.cls_C[sb_ldg(&B->meta) & 0xFF];
    const T* src = xs + sb_ldg(&B->lo);
    T* dst = slots + m * SL;
    for (int r = lane; r < C; r += 32) sb_copy(dst + r, src + r);
  }
}

// Phase 1 for one superblock H (x rows xs[0, C)): G[i] = sum of x over the
// high interior flips and the (KS-1, KS) flip of row i, in rank order. Thread
// t of nt takes rows t, t + nt, ..., U rows at a time, so that U loads per
// bond are in flight.
template <typename T, int U>
__host__ __device__ __forceinline__ void sb_phase1(const T* xs, const Sup& H, T* G, int t, int nt) {
  const int C = (int)H.C;
  const int nh = (int)((H.meta >> 8) & 0xFF);
  for (int i0 = t; i0 < C; i0 += nt * U) {
    T g[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * nt;
      g[u] = (i < C && (uint32_t)i >= H.ka && (uint32_t)i < H.kb) ? sb_ldg(xs + H.kd + i) : T(0);
    }
#pragma unroll 4
    for (int q = 0; q < nh; ++q) {
      const T* b = xs + H.hd[q];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * nt;
        if (i < C) g[u] += sb_ldg(b + i);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (i0 + u * nt < C) G[i0 + u * nt] = g[u];
  }
}

template <typename T>
struct Lane {
  const Low16* low;      // low table, class w slice
  const double* dlow;    // FP64 low terms, class w slice
  const T* tl;           // this sub-block's slot in the staged x
  const T* tg;           // this sub-block's first row in the phase-1 sums
  const T* tp;           // the wrap partner's slot (superblock T ^ top, same m)
  T* yg;                 // y + R + lo
  int32_t md[MD_MAX];    // mid offsets; unused entries point at the zero slot
  int nmid;              // km - 1
  int C;
  int32_t bdelta, zoff;  // cut offset; zero slot - this slot
  uint32_t mbit0, ttop;
  T uni;                 // dmid + dT - sigma +- 1/4 for bond (KS-1, KS)
};

// Byte q & 3 of wd, zero-extended (one byte permute on the device).
__host__ __device__ __forceinline__ uint32_t sb_byte(uint32_t wd, int q) {
#ifdef __CUDA_ARCH__
  return __byte_perm(wd, 0u, 0x4440u | (uint32_t)(q & 3));
#else
  return (wd >> (8 * (q & 3))) & 0xFFu;
#endif
}

// Phase 2: the rows of one sub-block for one lane (r = lane + 32 j); shared
// memory only, then one coalesced store. A lane past the last row repeats row
// C - 1 and does not store. Returns the lane's sum of x_i y_i over its rows
// (alpha_k of Algorithm 2 when x = q_k). NMID > 0: the number of mid bonds
// (km - 1) known at compile time.
template <typename T, int NMID = 0>
__host__ __device__ __forceinline__ T sb_lane(const Lane<T>& c, int lane) {
  const int J = (c.C + 31) >> 5;
  T dot = T(0);
#pragma unroll
  for (int j = 0; j < JMAX; ++j) {
    if (j >= J) break;
    const int r0 = lane + 32 * j;
    const bool valid = r0 < c.C;
    const int r = valid ? r0 : c.C - 1;
    const Low16 e = c.low[r];
    const T xi = c.tl[r];
    T a = c.tg[r];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const uint32_t wd = q < 4 ? e.nb0 : (q < 8 ? e.nb1 : e.meta);
      a += c.tl[sb_byte(wd, q)];
    }
    if constexpr (NMID > 0) {
#pragma unroll
      for (int q = 0; q < NMID; ++q) a += c.tl[r + c.md[q]];
    } else {
#pragma unroll
      for (int q = 0; q < MD_MAX; ++q)
        if (q < c.nmid) a += c.tl[r + c.md[q]];
    }
    const uint32_t code = (e.meta >> 20) & 3u;
    const uint32_t x0 = (code & 1u) ^ c.mbit0;
    const uint32_t x1 = (code >> 1) ^ c.ttop;
    a += c.tl[r + (x0 ? c.bdelta : c.zoff)];
    a += c.tp[x1 ? (int)((e.meta >> 8) & 0xFFu) : ZSLOT];
    T d;
    if constexpr (sizeof(T) == 8)
      d = c.dlow[r] + c.uni + (0.5 - 0.5 * (double)(x0 + x1));
    else
      d = e.dlow_f + c.uni + (0.5f - 0.5f * (float)(x0 + x1));
    const T yv = d * xi + T(0.5) * a;
    if (valid) {
      sb_st(c.yg + r, yv);
      dot += xi * yv;
    }
  }
  return dot;
}

// Per-row quantities of one sub-block without its neighbours (the MINRES
// passes that need the preconditioner M but no product): a_ii - sigma and the
// number of antiparallel bonds naf (sum_{k != i} a_ik^2 = naf / 4), with the
// same terms and the same order of additions as sb_lane's diagonal.
template <typename T>
struct RowCtx {
  const Low16* low;      // low table, class w slice
  const double* dlow;    // FP64 low terms, class w slice
  T uni;                 // dmid + dT - sigma +- 1/4 for bond (KS-1, KS)
  uint32_t mbit0, ttop;
  int nfix;              // antiparallel mid bonds + bond (KS-1, KS) + high bonds
  int C;                 // rows of the sub-block
};

template <typename T>
__host__ __device__ __forceinline__ T sb_diag(const RowCtx<T>& c, int r, int& naf) {
  const Low16 e = c.low[r];
  const uint32_t code = (e.meta >> 20) & 3u;
  const uint32_t x0 = (code & 1u) ^ c.mbit0;
  const uint32_t x1 = (code >> 1) ^ c.ttop;
  naf = (int)((e.meta >> 16) & 0xFu) + c.nfix + (int)(x0 + x1);
  if constexpr (sizeof(T) == 8)
    return c.dlow[r] + c.uni + (0.5 - 0.5 * (double)(x0 + x1));
  else
    return e.dlow_f + c.uni + (0.5f - 0.5f * (float)(x0 + x1));
}

// M_ii of preconditioner PC (0 identity, 1 Jacobi |a_ii - sigma|, 2 row norm
// sqrt((a_ii - sigma)^2 + naf / 4)), Sec. II.
template <int PC, typename T>
__host__ __device__ __forceinline__ T sb_precond(T am, int naf) {
  if (PC == 0) return T(1);
  if (PC == 1) return am < T(0) ? -am : am;
  if constexpr (sizeof(T) == 8) return sqrt(am * am + 0.25 * (double)naf);
  else return sqrtf(am * am + 0.25f * (float)naf);
}

}  // namespace sb
}  // namespace hs
