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
// neighbours of a row are found by bit arithmetic on m:
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
#pragma once
#include "sb.cuh"

namespace hs {
namespace sb4 {

constexpr int K = 4;            // low bits
constexpr int SLOT = 8;         // slot length (C(4, w) <= 6 rows)
constexpr int KM_MAX = 10;      // mid bits: 1024 slots per superblock
constexpr int WQ_MAX = sb::WQ_MAX;

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
    // by class w (descending popcount of m), then m: a warp's lanes share w
    std::stable_sort(valid.begin(), valid.end(), [](int a, int b) {
      return sb::popc_host((uint32_t)a) > sb::popc_host((uint32_t)b);
    });
    P->order_off[wq] = (int)P->order.size();
    P->nvalid[wq] = (int)valid.size();
    for (int m : valid) P->order.push_back((uint16_t)m);
    // flat row -> slot element, in rank order (ascending m, then r)
    P->slot_off[wq] = (int)P->slotmap.size();
    int rows = 0;
    for (int m = 0; m < nm; ++m) {
      const int w = wq - sb::popc_host((uint32_t)m);
      if (w < 0 || w > K) continue;
      for (int r = 0; r < cls_size(w); ++r) P->slotmap.push_back((uint16_t)(m * SLOT + r));
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

// Copy N (4 or 8) elements of an 8-aligned slot.
template <typename T, int N>
SB4_HD void ld_slot(const T* p, T (&v)[SLOT]) {
#ifdef __CUDA_ARCH__
  if constexpr (sizeof(T) == 4) {
    const float4 a = reinterpret_cast<const float4*>(p)[0];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    if constexpr (N > 4) {
      const float4 b = reinterpret_cast<const float4*>(p)[1];
      v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < N / 2; ++q) {
      const double2 a = reinterpret_cast<const double2*>(p)[q];
      v[2 * q] = a.x; v[2 * q + 1] = a.y;
    }
  }
#else
  for (int q = 0; q < N; ++q) v[q] = p[q];
#endif
}

// One sub-block for one lane: the C(4, W) rows of slot m of superblock s.
struct LaneIn {
  int m;              // mid pattern
  uint32_t b0;        // bit 0 of m
  uint32_t top;       // top bit of this superblock's T
  int km;
  int nmidb;          // km - 1 mid interior bonds
};

// y = (H - sigma) x for the rows of one sub-block. xs: this superblock's
// slots; xp: the partner superblock's slots (nullptr: no partner); g: the
// flat G sums from the sub-block's first row; dl: the class table for
// (top, b0); u = dmid + dT - sigma + Ising of bond (KS-1, KS); y: output from
// the sub-block's first row. Returns sum_r x_r y_r.
template <typename T, int W>
SB4_HD T sb4_rows(const LaneIn& in, const T* xs, const T* xp, const T* g, const T* dl, T u,
                  T* y) {
  constexpr int C = cls_size(W);
  constexpr int NL = C > 4 ? 8 : 4;          // elements loaded per slot
  T x[SLOT], acc[SLOT], src[SLOT];
  ld_slot<T, NL>(xs + in.m * SLOT, x);
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
  // mid interior bonds: slot m ^ (3 << j), same row
  for (int j = 0; j < in.nmidb; ++j) {
    if (((in.m >> j) ^ (in.m >> (j + 1))) & 1) {
      ld_slot<T, NL>(xs + (in.m ^ (3 << j)) * SLOT, src);
#pragma unroll
      for (int r = 0; r < C; ++r) acc[r] += src[r];
    }
  }
  // cut bond (3, 4): slot m ^ 1, row of p ^ 8 (classes W -+ 1)
  {
    constexpr int NC = (W + 1 <= 4 && cls_size(W + 1) > 4) || (W >= 1 && cls_size(W - 1) > 4) ? 8 : 4;
    ld_slot<T, NC>(xs + (in.m ^ 1) * SLOT, src);
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
    constexpr int NW = (W + 1 <= 4 && cls_size(W + 1) > 4) || (W >= 1 && cls_size(W - 1) > 4) ? 8 : 4;
    ld_slot<T, NW>(xp + in.m * SLOT, src);
#pragma unroll
    for (int r = 0; r < C; ++r) {
      const int p = pat(W, r);
      const uint32_t b0p = (uint32_t)(p & 1);
      const T v = src[rank4(p ^ 1)];
      acc[r] += (b0p != in.top) ? v : T(0);
    }
  }
  // whole-superblock shifts, then the row
  T dot = T(0);
#pragma unroll
  for (int r = 0; r < C; ++r) {
    const T a = acc[r] + g[r];
    const T d = dl[r] + u;
    const T yv = d * x[r] + T(0.5) * a;
    y[r] = yv;
    dot += x[r] * yv;
  }
  return dot;
}

template <typename T>
SB4_HD T sb4_rows_any(int w, const LaneIn& in, const T* xs, const T* xp, const T* g, const T* dl,
                      T u, T* y) {
  switch (w) {
    case 0: return sb4_rows<T, 0>(in, xs, xp, g, dl, u, y);
    case 1: return sb4_rows<T, 1>(in, xs, xp, g, dl, u, y);
    case 2: return sb4_rows<T, 2>(in, xs, xp, g, dl, u, y);
    case 3: return sb4_rows<T, 3>(in, xs, xp, g, dl, u, y);
    default: return sb4_rows<T, 4>(in, xs, xp, g, dl, u, y);
  }
}

// Flat pass over the rows of one superblock H (x rows xs[0, C)): G[i] = sum of
// x over its high interior flips and its (KS-1, KS) flip; thread t of nt takes
// rows t, t + nt, ..., U at a time so that U loads per bond are in flight.
// (The same sums as sb::sb_phase1.)
template <typename T, int U>
SB4_HD void sb4_phase1(const T* xs, const sb::Sup& H, T* G, int t, int nt) {
  sb::sb_phase1<T, U>(xs, H, G, t, nt);
}

#undef SB4_HD

}  // namespace sb4
}  // namespace hs
