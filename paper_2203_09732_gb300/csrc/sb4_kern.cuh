// Kernel of the four-low-bit superblock product (sb4.cuh): y = (H - sigma) x
// (Eq. (1)), one CTA per superblock pair, or, in MINRES mode, pass A of
// Algorithm 2 (p = (H - sigma) q_k and alpha_k = q_k . p / beta_k^2 by a
// last-CTA reduction).
//
// Per pair: (1) every thread takes flat rows of the pair, copies x of each row
// asynchronously into its slot entry (a flat-row -> slot table) and sums the
// whole-superblock shifts of the row into G; (2) after the copies land, one
// lane per sub-block computes its rows from shared memory only and writes them
// over their G entries; (3) the pair's rows are stored from G in rank order,
// coalesced.
#pragma once
#include "minres_scalar.cuh"
#include "rows.cuh"
#include "sb4.cuh"
#include "sb_kern.cuh"

namespace hs {
namespace sb4 {

// Shared memory (elements of T unless noted): the four slot arrays
// (4 arr_elems(km)), G [2][cmax], dmid [2^km], dl [2*2*5*8], uT [2][2],
// Sup [2] (bytes).
template <typename T>
__host__ __device__ inline size_t smem_bytes4(int km, int cmax) {
  const size_t nsl = (size_t)1 << km;
  return sizeof(T) * (4 * (size_t)arr_elems(km) + 2 * (size_t)cmax + nsl + 2 * 2 * 5 * SLOT + 4) +
         2 * sizeof(sb::Sup) + 16;
}

template <typename T, int NT, int MINB, int U, int MODE, int KM>
__global__ void __launch_bounds__(NT, MINB) k_sb4(Geo4 g, const T* __restrict__ x,
                                                  T* __restrict__ y, const double* d_sigma,
                                                  int shifted, sb::MinresArgs ma) {
  extern __shared__ __align__(16) char smem[];
  __shared__ double s_red[32 * 4];
  __shared__ double s_sig;
  __shared__ long long s_k;
  __shared__ int s_done;
  if constexpr (MODE == sb::MODE_MINRES) {
    if (threadIdx.x == 0) {
      const MinresState* st = ma.st;
      s_done = st->done; s_k = st->k; s_sig = st->sigma;
    }
    __syncthreads();
    if (s_done != 0) return;   // finished, or only the last d/x update is left (pass B)
    const bool odd = (s_k & 1) != 0;
    x = (const T*)(odd ? ma.v.q1 : ma.v.q0);   // q_k
    y = (T*)ma.v.p;
  } else {
    if (threadIdx.x == 0) s_sig = shifted ? *d_sigma : 0.0;
    __syncthreads();
  }
  const double sigma = s_sig;
  const int km = KM ? KM : g.km;
  const int nsl = 1 << km;
  const int AE = arr_elems(km);
  T* X = reinterpret_cast<T*>(smem);                 // lo 0 | lo 1 | hi 0 | hi 1
  T* G = X + 4 * (size_t)AE;                         // [2][cmax]
  T* dmid = G + 2 * (size_t)g.cmax;                  // [nsl]
  T* dl = dmid + nsl;                                // [2][2][5][SLOT]
  T* uT = dl + 2 * 2 * 5 * SLOT;                     // [2][2]: dT - sigma +- 1/4 (bond (KS-1, KS))
  sb::Sup* sh = reinterpret_cast<sb::Sup*>(uT + 4);
  const int tid = threadIdx.x;
  {
    const T* dm = sizeof(T) == 8 ? (const T*)g.dmid_d : (const T*)g.dmid_f;
    const T* dt = sizeof(T) == 8 ? (const T*)g.dl_d : (const T*)g.dl_f;
    for (int i = tid; i < nsl; i += NT) dmid[i] = __ldg(dm + i);
    for (int i = tid; i < 2 * 2 * 5 * SLOT; i += NT) dl[i] = __ldg(dt + i);
    // the zero entries at the end of each of the four arrays
    for (int i = tid; i < 4 * ZERO_ENT * 4; i += NT)
      X[(i / (ZERO_ENT * 4)) * AE + nsl * 4 + i % (ZERO_ENT * 4)] = T(0);
  }
  T acc = T(0);
  for (int pi = blockIdx.x; pi < g.npairs; pi += gridDim.x) {
    const int2 pr = g.pairs[pi];
    __syncthreads();  // the previous pair is done with sh, X, G and uT
    if (tid < 2 * sb::SUP_WORDS) {
      const int s = tid / sb::SUP_WORDS, wd = tid % sb::SUP_WORDS;
      const int id = s ? pr.y : pr.x;
      reinterpret_cast<uint32_t*>(sh + s)[wd] =
          id >= 0 ? __ldg(reinterpret_cast<const uint32_t*>(g.sup + id) + wd) : 0u;
    }
    __syncthreads();
    if (tid < 4) {
      // the superblock's share of every diagonal: dT - sigma and the Ising
      // term of bond (KS-1, KS), by the top mid bit (tid & 1)
      const int s = tid >> 1;
      const uint32_t tb0 = (sh[s].meta >> 16) & 1u;   // bit 0 of T
      const double ks = ((uint32_t)(tid & 1) == tb0) ? 0.25 : -0.25;
      uT[tid] = (T)(sh[s].dT - sigma + ks);
    }
    // phase 1: copies into the slots (asynchronous) and the whole-superblock sums
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
      if (!sh[s].C) continue;
      const int wq = (int)(sh[s].meta & 0xFF);
      const uint16_t* map = g.slotmap + g.slot_off[wq];
      const T* xs = x + sh[s].R;
      T* Xs = X + (size_t)s * AE;
      // the slot indices of four rows are loaded before their copies are issued
      const int C = (int)sh[s].C;
      int i = tid;
      for (; i + 3 * NT < C; i += 4 * NT) {
        int e[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) e[q] = __ldg(map + i + q * NT);
#pragma unroll
        for (int q = 0; q < 4; ++q) sb::sb_copy(Xs + e[q], xs + i + q * NT);
      }
      for (; i < C; i += NT) sb::sb_copy(Xs + __ldg(map + i), xs + i);
    }
#pragma unroll 1
    for (int s = 0; s < 2; ++s)
      if (sh[s].C) sb4_phase1<T, U>(x + sh[s].R, sh[s], G + (size_t)s * g.cmax, tid, NT);
    sb::cp_async_wait_all();
    __syncthreads();
    // phase 2: one lane per sub-block, shared memory only; y over G
    const int nv0 = sh[0].C ? g.nvalid[sh[0].meta & 0xFF] : 0;
    const int nv1 = sh[1].C ? g.nvalid[sh[1].meta & 0xFF] : 0;
    // the table entries (m, then lo) of a lane's next task are loaded while
    // it computes the current one
    auto task_m = [&](int u) {
      const int s = u >= nv0 ? 1 : 0;
      const int wq = (int)(sh[s].meta & 0xFF);
      return (int)__ldg(g.order + g.order_off[wq] + (s ? u - nv0 : u));
    };
    auto task_lo = [&](int u, int m) {
      const int wq = (int)(sh[u >= nv0 ? 1 : 0].meta & 0xFF);
      return (int)__ldg(g.lo + ((size_t)wq << km) + m);
    };
    int m_next = tid < nv0 + nv1 ? task_m(tid) : 0;
    int lo_next = tid < nv0 + nv1 ? task_lo(tid, m_next) : 0;
    for (int u = tid; u < nv0 + nv1; u += NT) {
      const int s = u >= nv0 ? 1 : 0;
      const sb::Sup& H = sh[s];
      const uint32_t hm = H.meta;
      const int wq = (int)(hm & 0xFF);
      const int m = m_next;
      const int lo = lo_next;
      if (u + NT < nv0 + nv1) {
        m_next = task_m(u + NT);
        lo_next = task_lo(u + NT, m_next);
      }
      const int w = wq - __popc((unsigned)m);
      LaneIn in;
      in.m = m;
      in.b0 = (uint32_t)m & 1u;
      in.top = (hm >> 17) & 1u;
      in.km = km;
      const T uu = dmid[m] + uT[s * 2 + ((m >> (km - 1)) & 1)];
      const T* xp = sh[1 - s].C ? X + (size_t)(1 - s) * AE : nullptr;
      const T* dlw = dl + (((int)in.top * 2 + (int)in.b0) * 5 + w) * SLOT;
      acc += sb4_rows_any<T, KM>(w, in, X + (size_t)s * AE, xp, G + (size_t)s * g.cmax + lo, dlw,
                                 uu);
    }
    __syncthreads();
    // phase 3: the pair's rows in rank order
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
      const T* Gs = G + (size_t)s * g.cmax;
      T* ys = y + sh[s].R;
      for (int i = tid; i < (int)sh[s].C; i += NT) ys[i] = Gs[i];
    }
  }
  if constexpr (MODE == sb::MODE_MINRES) {
    double vv[1] = {(double)acc}, tot[1];
    if (last_cta_sum<1>(vv, s_red, ma.partial, ma.counter, tot) && threadIdx.x == 0) {
      MinresState* st = ma.st;
      const double bk = st->beta;
      st->alpha = tot[0] / (bk * bk);                        // alpha_k = q_k . p_k / beta_k^2
      if (!isfinite(st->alpha)) { st->status = HS_NONFINITE; st->done = 2; st->pending = 0; }
    }
  }
}

// Device copy of one plan.
struct DevPlan4 {
  Geo4 geo{};
  void* mem = nullptr;
  int grid = 0;
  size_t smem = 0;
  int ok = 0;
};

}  // namespace sb4
}  // namespace hs
