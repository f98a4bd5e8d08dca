// Superblock product (H - sigma) x of Eq. (1) with four low bits: one lane
// per sub-block.
//
// The split of a state word is that of sb.cuh with k = 4: p = bits 0..3,
// m = the km = KS - 4 mid bits, T = the top L - KS bits. A sub-block (T, m)
// holds the C(4, w) <= 6 rows whose low pattern p has popcount
// w = L/2 - popcount(T) - popcount(m), in ascending p (= colex) order, so one
// lane can own a whole sub-block in registers. In shared memory every
// sub-block of the CTA's superblock pair {T, T ^ top} has a slot of 8
// elements at index m (slot address m * 8, whatever the class), so the
// neighbours of a row are found by bit arithmetic on m (the slot's elements
// 0..3 and 4..7 live in two arrays of 16-byte entries, at the swizzled index
// swz(m), see below):
//   low interior  (j, j+1), j < 3        : same slot, another row (fixed per class);
//   cut (3, 4)                           : slot m ^ 1, row of p ^ 8 (fixed per class);
//   mid interior  (j, j+1), 4 <= j < KS-1 : slot m ^ (3 << (j-4)), same row;
//   wrap (L-1, 0)                        : the partner superblock's slot m,
//                                          row of p ^ 1 (fixed per class);
//   bond (KS-1, KS) and high interior    : whole-superblock shifts in rank order,
//                                          summed by a flat coalesced pass into G.
// The per-class row maps are compile-time constants (class template W), so
// the row pass is vector loads of whole slots, adds and selects; the work list
// of a superblock is sorted by class so that a warp's lanes share the class.
//
// Bank conflicts: a 16-byte load by a warp is served 8 lanes at a time, one
// pass if the 8 entries fall in distinct 16-byte bank groups (index mod 8).
// swz() below is linear over XOR and a bijection, so swz(m ^ c) =
// swz(m) ^ swz(c): if the 8 lanes of a group have distinct swz(m) mod 8, so
// do their neighbours m ^ c for every bond. The host deals each class run of
// the work list so that every aligned group of 8 lanes has distinct
// swz(m) mod 8 where the run allows it, and a lane whose bond is parallel
// reads the zero entry of its own bank group.
#pragma once
#include "sb.cuh"

namespace hs {
namespace sb4 {

constexpr int K = 4;            // low bits
constexpr int SLOT = 8;         // slot length (C(4, w) <= 6 rows)
constexpr int KM_MAX = 10;      // mid bits: 1024 slots per superblock
constexpr int WQ_MAX = sb::WQ_MAX;

// Swizzled slot index: the low three bits of m mixed with bits 2..7 (a
// bijection on [0, 2^km), linear over XOR).
__host__ __device__ constexpr int swz(int m) { return m ^ ((m >> 2) & 7) ^ ((m >> 5) & 7); }
constexpr int ZERO_ENT = 8;        // zero entries after the slots, one per bank group

// Shared-memory slot arrays of a CTA, in 16-byte entries of 4 elements:
// [lo rows of superblock 0 | lo rows of superblock 1 | hi rows of 0 | hi of 1],
// each array 2^km + ZERO_ENT entries (the last ZERO_ENT are zero). Element offset of
// row r of slot m of superblock 0 (superblock 1: + arr_elems(km)).
__host__ __device__ constexpr int arr_elems(int km) { return ((1 << km) + ZERO_ENT) * 4; }
__host__ __device__ constexpr int slot_elem(int km, int m, int r) {
  return (r >= 4 ? 2 * arr_elems(km) : 0) + swz(m) * 4 + (r & 3);
}

// Low patterns of class w in ascending order.
__host__ __device__ constexpr int cls_size(int w) {
  return w == 0 || w == 4 ? 1 : (w == 2 ? 6 : 4);
}
__host__ __device__ constexpr int pat(int w, int r) {
  // w = 0: 0000; w = 1: 0001 0010 0100 1000; w = 2: 0011 0101 0110 1001 1010 1100;
  // w = 3: 0111 1011 1101 1110; w = 4: 1111
  return w == 0 ? 0
       : w == 1 ? (1 << r)
       : w == 2 ? (r == 0 ? 3 : r == 1 ? 5 : r == 2 ? 6 : r == 3 ? 9 : r == 4 ? 10 : 12)
       : w == 3 ? (15 ^ (8 >> r))
       : 15;
}
__host__ __device__ constexpr int popc4(int p) {
  return (p & 1) + ((p >> 1) & 1) + ((p >> 2) & 1) + ((p >> 3) & 1);
}
// rank of pattern p within its class
__host__ __device__ constexpr int rank4(int p) {
  int r = 0;
  for (int q = 0; q < p; ++q)
    if (popc4(q) == popc4(p)) ++r;
  return r;
}

// Device copy of the tables.
struct Geo4 {
  const sb::Sup* sup;          // superblock headers, ascending T
  const int2* pairs;           // {T0, T0 | top} superblock indices, -1 where absent
  const uint16_t* slotmap;     // per class: flat row i -> slot element m * 8 + r
  const uint16_t* order;       // per class: valid m, sorted by class w then m
  const uint16_t* lo;          // [wq][2^km]: first flat row of sub-block m
  const float* dmid_f;         // [2^km] mid Ising + fields (FP32)
  const double* dmid_d;        // [2^km] (FP64)
  const float* dl_f;           // [top][b0 of m][w][8]: low, cut and wrap Ising + low fields
  const double* dl_d;
  int npairs, km, KS, cmax;    // cmax = largest superblock (rows)
  int slot_off[WQ_MAX + 1];    // offset of class wq in slotmap
  int order_off[WQ_MAX + 1];   // offset of class wq in order
  int nvalid[WQ_MAX + 1];      // valid m of class wq
  double dscale;               // L/4 + sum |h_j| / 2
};

// Host tables.
struct HostPlan4 {
  sb::HostPlan base;           // superblocks, pairs, Sub (lo, dmid) with k = 4
  std::vector<uint16_t> slotmap, order, lo;
  std::vector<float> dmid_f, dl_f;
  std::vector<double> dmid_d, dl_d;
  int slot_off[WQ_MAX + 1] = {0};
  int order_off[WQ_MAX + 1] = {0};
  int nvalid[WQ_MAX + 1] = {0};
  int cmax = 0;
};

// Build the plan for chain length L, fields h[0..L-1] and a KS-bit window
// (k = 4 low bits). False where the split does not apply (km = KS - 4 must be
// 1..10, and the top field must have 2..17 bits).
inline bool build_plan4(int L, const double* h, int KS, HostPlan4* P) {
  *P = HostPlan4{};
  const int km = KS - K;
  if (km < 1 || km > KM_MAX) return false;
  if (!sb::build_plan(L, h, K, KS, &P->base, KM_MAX)) return false;
  const sb::HostPlan& B = P->base;
  const int nm = 1 << km, nwq = KS + 1;
  P->lo.assign((size_t)nwq * nm, 0xFFFFu);
  P->dmid_f.assign(nm, 0.f);
  P->dmid_d.assign(nm, 0.0);
  for (int wq = 0; wq < nwq; ++wq) {
    std::vector<int> valid;
    for (int m = 0; m < nm; ++m) {
      const int w = wq - sb::popc_host((uint32_t)m);
      if (w < 0 || w > K) continue;
      valid.push_back(m);
      const sb::Sub& s = B.sub[(size_t)wq * nm + m];
      P->lo[(size_t)wq * nm + m] = (uint16_t)s.lo;
      P->dmid_d[m] = s.dmid;
      P->dmid_f[m] = (float)s.dmid;
    }
    // by class w (descending popcount of m); within a class run, dealt in
    // rounds of 8 with distinct swz(m) mod 8 (the fullest bank groups first),
    // so that the lanes of an aligned group of 8 hit distinct bank groups
    std::vector<uint16_t> dealt;
    for (int pc = km; pc >= 0; --pc) {
      std::vector<std::vector<int>> bk(8);
      int left = 0;
      for (int m : valid)
        if (sb::popc_host((uint32_t)m) == pc) {
          bk[swz(m) & 7].push_back(m);
          ++left;
        }
      std::vector<size_t> at(8, 0);
      while (left) {
        int ord[8] = {0, 1, 2, 3, 4, 5, 6, 7};
        std::stable_sort(ord, ord + 8, [&](int a, int b) {
          return bk[a].size() - at[a] > bk[b].size() - at[b];
        });
        int took = 0;
        for (int q = 0; q < 8 && took < 8; ++q)
          if (at[ord[q]] < bk[ord[q]].size()) {
            dealt.push_back((uint16_t)bk[ord[q]][at[ord[q]]++]);
            ++took;
            --left;
          }
        // fewer than 8 bank groups left: fill the group from the fullest
        while (took < 8 && left) {
          int f = 0;
          for (int q = 1; q < 8; ++q)
            if (bk[q].size() - at[q] > bk[f].size() - at[f]) f = q;
          dealt.push_back((uint16_t)bk[f][at[f]++]);
          ++took;
          --left;
        }
      }
    }
    P->order_off[wq] = (int)P->order.size();
    P->nvalid[wq] = (int)valid.size();
    P->order.insert(P->order.end(), dealt.begin(), dealt.end());
    // flat row -> element offset in the CTA's slot arrays (superblock 0; add
    // one array length for superblock 1), in rank order (ascending m, then r)
    P->slot_off[wq] = (int)P->slotmap.size();
    int rows = 0;
    for (int m = 0; m < nm; ++m) {
      const int w = wq - sb::popc_host((uint32_t)m);
      if (w < 0 || w > K) continue;
      for (int r = 0; r < cls_size(w); ++r) P->slotmap.push_back((uint16_t)slot_elem(km, m, r));
      rows += cls_size(w);
    }
    if (rows != (int)sb::binom64(KS, wq)) return *P = HostPlan4{}, false;
    P->cmax = std::max(P->cmax, rows);
  }
  // diagonal terms of the low field: dlow(p) + cut Ising (bit 3 of p, bit 0 of
  // m) + wrap Ising (bit 0 of p, top bit of T), per (top, b0 of m, w, r)
  P->dl_f.assign(2 * 2 * 5 * SLOT, 0.f);
  P->dl_d.assign(2 * 2 * 5 * SLOT, 0.0);
  for (int top = 0; top < 2; ++top)
    for (int b0 = 0; b0 < 2; ++b0)
      for (int w = 0; w <= K; ++w)
        for (int r = 0; r < cls_size(w); ++r) {
          const int p = pat(w, r);
          const int li = B.cls_off[w] + r;
          double d = B.dlow[li];
          d += (((p >> 3) & 1) == b0) ? 0.25 : -0.25;
          d += ((p & 1) == top) ? 0.25 : -0.25;
          const size_t at = (((size_t)top * 2 + b0) * 5 + w) * SLOT + r;
          P->dl_d[at] = d;
          P->dl_f[at] = (float)d;
        }
  return true;
}

// ---------------------------------------------------------------------------
// Row code shared by the kernel and the host check.
#ifdef __CUDA_ARCH__
#define SB4_HD __device__ __forceinline__
#else
#define SB4_HD inline
#endif

// Load one 16-byte-aligned entry of 4 elements.
template <typename T>
SB4_HD void ld4(const T* p, T* v) {
#ifdef __CUDA_ARCH__
  if constexpr (sizeof(T) == 4) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
#else
  for (int q = 0; q < 4; ++q) v[q] = p[q];
#endif
}

// One sub-block for one lane: the C(4, W) rows of slot m.
struct LaneIn {
  int m;              // mid pattern
  uint32_t b0;        // bit 0 of m
  uint32_t top;       // top bit of this superblock's T
  int km;
};

// y = (H - sigma) x for the rows of one sub-block. xs: this superblock's lo
// array (its hi array follows 2 arr_elems(km) elements later); xp: the
// partner superblock's lo array (nullptr: no partner); g: the flat G sums from
// the sub-block's first row, overwritten with y; dl: the class table for
// (top, b0); u = dmid + dT - sigma + Ising of bond (KS-1, KS). KM: the number
// of mid bits if known at compile time (0: in.km at run time). Returns
// sum_r x_r y_r.
template <typename T, int W, int KM>
SB4_HD T sb4_rows(const LaneIn& in, const T* xs, const T* xp, T* g, const T* dl, T u) {
  constexpr int C = cls_size(W);
  constexpr bool HI = C > 4;                 // rows 4, 5 live in the hi array
  const int km = KM ? KM : in.km;
  const int nsl = 1 << km;
  const int hi = 2 * arr_elems(km);
  const int pm = swz(in.m);
  T x[SLOT], acc[SLOT], src[SLOT];
  ld4(xs + pm * 4, x);
  if (HI) ld4(xs + hi + pm * 4, x + 4);
#pragma unroll
  for (int r = 0; r < SLOT; ++r) acc[r] = T(0);
  // low interior bonds (j, j+1), j = 0, 1, 2: rows of the same slot
#pragma unroll
  for (int r = 0; r < C; ++r) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int p = pat(W, r);
      if (((p >> j) & 1) != ((p >> (j + 1)) & 1)) acc[r] += x[rank4(p ^ (3 << j))];
    }
  }
  // mid interior bonds (j, j+1) of m: slot m ^ (3 << j), same row; a parallel
  // bond reads the zero entry of the bank group the antiparallel one would use
  const int t = in.m ^ (in.m >> 1);
  auto mid = [&](int j, int cj) {
    const int idx = pm ^ cj;
    const int at = ((t >> j) & 1) ? idx : nsl + (idx & 7);
    ld4(xs + at * 4, src);
    if (HI) ld4(xs + hi + at * 4, src + 4);
#pragma unroll
    for (int r = 0; r < C; ++r) acc[r] += src[r];
  };
  if constexpr (KM > 0) {
#pragma unroll
    for (int j = 0; j < KM - 1; ++j) mid(j, swz(3 << j));
  } else {
    for (int j = 0; j < km - 1; ++j) mid(j, swz(3 << j));
  }
  // cut bond (3, 4): slot m ^ 1, row of p ^ 8 (classes W -+ 1)
  {
    constexpr bool CH = (W + 1 <= 4 && cls_size(W + 1) > 4) || (W >= 1 && cls_size(W - 1) > 4);
    const int idx = pm ^ swz(1);
    ld4(xs + idx * 4, src);
    if (CH) ld4(xs + hi + idx * 4, src + 4);
#pragma unroll
    for (int r = 0; r < C; ++r) {
      const int p = pat(W, r);
      const uint32_t b3 = (uint32_t)((p >> 3) & 1);
      const T v = src[rank4(p ^ 8)];
      acc[r] += (b3 != in.b0) ? v : T(0);
    }
  }
  // wrap bond (L-1, 0): the partner superblock's slot m, row of p ^ 1
  if (xp) {
    constexpr bool WH = (W + 1 <= 4 && cls_size(W + 1) > 4) || (W >= 1 && cls_size(W - 1) > 4);
    ld4(xp + pm * 4, src);
    if (WH) ld4(xp + hi + pm * 4, src + 4);
#pragma unroll
    for (int r = 0; r < C; ++r) {
      const int p = pat(W, r);
      const uint32_t b0p = (uint32_t)(p & 1);
      const T v = src[rank4(p ^ 1)];
      acc[r] += (b0p != in.top) ? v : T(0);
    }
  }
  // whole-superblock shifts, then the row (written over its G entry)
  T dot = T(0);
#pragma unroll
  for (int r = 0; r < C; ++r) {
    const T a = acc[r] + g[r];
    const T d = dl[r] + u;
    const T yv = d * x[r] + T(0.5) * a;
    g[r] = yv;
    dot += x[r] * yv;
  }
  return dot;
}

template <typename T, int KM>
SB4_HD T sb4_rows_any(int w, const LaneIn& in, const T* xs, const T* xp, T* g, const T* dl, T u) {
  switch (w) {
    case 0: return sb4_rows<T, 0, KM>(in, xs, xp, g, dl, u);
    case 1: return sb4_rows<T, 1, KM>(in, xs, xp, g, dl, u);
    case 2: return sb4_rows<T, 2, KM>(in, xs, xp, g, dl, u);
    case 3: return sb4_rows<T, 3, KM>(in, xs, xp, g, dl, u);
    default: return sb4_rows<T, 4, KM>(in, xs, xp, g, dl, u);
  }
}

// Flat pass over the rows of one superblock H (x rows xs[0, C)): G[i] = sum of
// x over its high interior flips and its (KS-1, KS) flip; thread t of nt takes
// rows t, t + nt, ..., U at a time so that U loads per bond are in flight (the
// sums of sb::sb_phase1, with the bounds test only in the last round).
template <typename T, int U>
SB4_HD void sb4_phase1(const T* xs, const sb::Sup& H, T* G, int t, int nt) {
  const int C = (int)H.C;
  const int nh = (int)((H.meta >> 8) & 0xFF);
  const int ka = (int)H.ka, kb = (int)H.kb;
  const T* xk = xs + H.kd;
  int i0 = t;
  for (; i0 + (U - 1) * nt < C; i0 += U * nt) {
    T g[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * nt;
      g[u] = (i >= ka && i < kb) ? xk[i] : T(0);
    }
    // four bonds at a time: 4 U independent loads in flight per thread
    int q = 0;
    for (; q + 4 <= nh; q += 4) {
      T v[4][U];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const T* b = xs + H.hd[q + e] + i0;
#pragma unroll
        for (int u = 0; u < U; ++u) v[e][u] = b[u * nt];
      }
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int u = 0; u < U; ++u) g[u] += v[e][u];
    }
    for (; q < nh; ++q) {
      const T* b = xs + H.hd[q] + i0;
#pragma unroll
      for (int u = 0; u < U; ++u) g[u] += b[u * nt];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) G[i0 + u * nt] = g[u];
  }
  for (; i0 < C; i0 += nt) {
    T g = (i0 >= ka && i0 < kb) ? xk[i0] : T(0);
    for (int q = 0; q < nh; ++q) g += xs[H.hd[q] + i0];
    G[i0] = g;
  }
}

#undef SB4_HD

}  // namespace sb4
}  // namespace hs
