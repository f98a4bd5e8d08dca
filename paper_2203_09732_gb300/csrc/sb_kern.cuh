// Kernels of the superblock layout (sb.cuh) for long chains:
//   k_sbhv   : y = (H - sigma) x (Eq. (1)), one CTA per superblock pair; in
//              MINRES mode it is pass A of Algorithm 2: p = (H - sigma) q_k and
//              alpha_k = q_k . p / beta_k^2.
//   k_sbrows : the MINRES passes that need the preconditioner but no product:
//              the initial pass (q_1 = M^-1 b, beta_1) and pass B: the pending
//              d/x update of iteration k - 1 (it needs gamma_{k-1}, known only
//              after the previous pass B) fused with q_{k+1}, beta_{k+1} and the
//              Givens rotation. Pass B reads q_{k-1} once for both.
// The MINRES passes end in a last-CTA reduction that runs the scalar
// recurrences on the device (minres_scalar.cuh), so a whole iteration is two
// launches and no host round trip.
#pragma once
#include "minres_scalar.cuh"
#include "rows.cuh"
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

// Device copy of one plan.
struct DevPlan {
  Geo geo{};
  void* mem = nullptr;  // one allocation holding every table
  int grid = 0;         // grid of the H x kernel on all SMs
  size_t smem = 0;      // dynamic shared memory of the H x kernel
  int ok = 0;
};

// Extras of the MINRES modes: the solver's vectors and device scalars.
struct MinresArgs {
  MinresVecs v;
  MinresState* st;
  double* partial;
  unsigned* counter;
};

constexpr int MODE_HV = 0;       // plain product
constexpr int MODE_MINRES = 1;   // MINRES pass A

template <typename T, int NT, int MINB, int U, int MODE, int NMID = 0>
__global__ void __launch_bounds__(NT, MINB) k_sbhv(Geo g, const T* __restrict__ x,
                                                   T* __restrict__ y, const double* d_sigma,
                                                   int shifted, MinresArgs ma) {
  extern __shared__ __align__(16) char smem[];
  __shared__ double s_red[32 * 4];
  __shared__ double s_c[1];
  __shared__ long long s_k;
  __shared__ int s_done;
  __shared__ float s_dts[2];   // dT - sigma of the pair's superblocks (FP32 kernels)
  double sigma = 0.0;
  if constexpr (MODE == MODE_MINRES) {
    if (threadIdx.x == 0) {
      const MinresState* st = ma.st;
      s_done = st->done; s_k = st->k; s_c[0] = st->sigma;
    }
    __syncthreads();
    if (s_done != 0) return;   // finished, or only the last d/x update is left (pass B)
    sigma = s_c[0];
    const bool odd = (s_k & 1) != 0;
    x = (const T*)(odd ? ma.v.q1 : ma.v.q0);   // q_k
    y = (T*)ma.v.p;
  } else {
    sigma = shifted ? *d_sigma : 0.0;
  }
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
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = NT / 32;
  T acc = T(0);
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
    // the superblocks' share of the diagonal, once per pair: FP32 kernels add
    // it to the sub-blocks' FP32 terms (no FP64 arithmetic per sub-block)
    if constexpr (sizeof(T) == 4)
      if (threadIdx.x < 2) s_dts[threadIdx.x] = (float)(sh[threadIdx.x].dT - sigma);
    // phase 1: stage x into the slots (asynchronous) while the sums of the
    // whole-superblock shifts go into G
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
      if constexpr (sizeof(T) == 4)
        c.uni = __ldg(&B->dmid_f) + s_dts[s] + (anti_ks ? -0.25f : 0.25f);
      else
        c.uni = __ldg(&B->dmid) + H.dT - sigma + (anti_ks ? -0.25 : 0.25);
      acc += sb_lane<T, NMID>(c, lane);
    }
  }
  if constexpr (MODE == MODE_MINRES) {
    double vv[1] = {(double)acc}, tot[1];
    if (last_cta_sum<1>(vv, s_red, ma.partial, ma.counter, tot) && threadIdx.x == 0) {
      MinresState* st = ma.st;
      const double bk = st->beta;
      st->alpha = tot[0] / (bk * bk);                        // alpha_k = q_k . p_k / beta_k^2
      if (!isfinite(st->alpha)) { st->status = HS_NONFINITE; st->done = 2; st->pending = 0; }
    }
  }
}

constexpr int ROWS_INIT = 0;   // q_1 = M^-1 b, beta_1
constexpr int ROWS_B = 1;      // pass B of Algorithm 2

// One warp per sub-block, lane l takes rows l + 32 j; the preconditioner is
// recomputed per row from the tables (nothing of size n is stored for it).
template <typename T, int PC, int MODE, int NT>
__global__ void __launch_bounds__(NT, sizeof(T) == 8 ? 1 : 2) k_sbrows(Geo g, const T* __restrict__ bv, MinresArgs ma,
                                                  double tol, long long kmax,
                                                  const double* d_sigma) {
  extern __shared__ __align__(16) char smem[];
  __shared__ Sup sh[2];
  __shared__ double s_red[32 * 4];
  __shared__ double s_c[8];
  __shared__ long long s_k;
  __shared__ int s_done, s_pending;
  double sigma;
  bool doQ = true, doC = false;
  if constexpr (MODE == ROWS_B) {
    if (threadIdx.x == 0) {
      const MinresState* st = ma.st;
      s_done = st->done; s_pending = st->pending; s_k = st->k;
      const double bk = st->beta;
      s_c[0] = 1.0 / bk; s_c[1] = st->alpha / bk; s_c[2] = bk / st->beta_prev;
      s_c[3] = st->sigma;
      s_c[4] = st->cq; s_c[5] = st->cd1; s_c[6] = st->cd2; s_c[7] = st->tau;
    }
    __syncthreads();
    if (s_done == 2) return;
    doQ = s_done == 0;        // done == 1: only the last d/x update is left
    doC = s_pending != 0;
    sigma = s_c[3];
  } else {
    sigma = *d_sigma;
  }
  const int nlow = 1 << g.k;
  Low16* low = reinterpret_cast<Low16*>(smem);
  double* dlw = reinterpret_cast<double*>(smem + sizeof(Low16) * nlow);
  {
    const uint4* s = reinterpret_cast<const uint4*>(g.low);
    uint4* d = reinterpret_cast<uint4*>(low);
    for (int i = threadIdx.x; i < nlow; i += NT) d[i] = __ldg(s + i);
    if constexpr (sizeof(T) == 8)
      for (int i = threadIdx.x; i < nlow; i += NT) dlw[i] = __ldg(g.dlow + i);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = NT / 32;
  const MinresVecs& v = ma.v;
  const bool odd = MODE == ROWS_B ? (s_k & 1) != 0 : false;
  const T* qc = (const T*)(odd ? v.q1 : v.q0);   // q_k
  T* qn = (T*)(odd ? v.q0 : v.q1);               // q_{k-1} -> q_{k+1}
  const T* pv = (const T*)v.p;
  const T c1 = MODE == ROWS_B ? (T)s_c[0] : T(0);
  const T c2 = MODE == ROWS_B ? (T)s_c[1] : T(0);
  const T c3 = MODE == ROWS_B ? (T)s_c[2] : T(0);
  const T cq = MODE == ROWS_B ? (T)s_c[4] : T(0);
  const T cd1 = MODE == ROWS_B ? (T)s_c[5] : T(0);
  const T cd2 = MODE == ROWS_B ? (T)s_c[6] : T(0);
  const T tau = MODE == ROWS_B ? (T)s_c[7] : T(0);
  const T* dA = (const T*)(odd ? v.d1 : v.d0);   // d_{k-2}
  T* dB = (T*)(odd ? v.d0 : v.d1);               // d_{k-3} -> d_{k-1}
  T* xv = (T*)v.x;
  // rounding bound of a_ii - sigma as assembled from the tables (a few
  // additions of terms up to dscale + |sigma|)
  const T mtiny = (T)(8.0 * (sizeof(T) == 8 ? 2.220446049250313e-16 : 1.1920928955078125e-7) *
                      (g.dscale + fabs(sigma)));
  T acc = T(0), zm = T(0);
  for (int pi = blockIdx.x; pi < g.npairs; pi += gridDim.x) {
    const int2 pr = g.pairs[pi];
    __syncthreads();
    if (threadIdx.x < 2 * SUP_WORDS) {
      const int s = threadIdx.x / SUP_WORDS, wd = threadIdx.x % SUP_WORDS;
      const int id = s ? pr.y : pr.x;
      reinterpret_cast<uint32_t*>(sh + s)[wd] =
          id >= 0 ? __ldg(reinterpret_cast<const uint32_t*>(g.sup + id) + wd) : 0u;
    }
    __syncthreads();
    const int nv0 = sh[0].C ? g.nvalid[sh[0].meta & 0xFF] : 0;
    const int nv1 = sh[1].C ? g.nvalid[sh[1].meta & 0xFF] : 0;
    for (int u = warp; u < nv0 + nv1; u += NW) {
      const int s = u >= nv0 ? 1 : 0;
      const int ii = s ? u - nv0 : u;
      const Sup& H = sh[s];
      const uint32_t hm = H.meta;
      const int wq = (int)(hm & 0xFF);
      const int m = __ldg(g.order + (wq << g.km) + ii);
      const Sub* B = g.sub + (wq << g.km) + m;
      const uint32_t bm = __ldg(&B->meta);
      const int w = (int)(bm & 0xFF);
      RowCtx<T> c;
      c.low = low + g.cls_off[w];
      c.dlow = sizeof(T) == 8 ? dlw + g.cls_off[w] : nullptr;
      c.mbit0 = (bm >> 16) & 1u;
      c.ttop = (hm >> 17) & 1u;
      const uint32_t anti_ks = ((bm >> 17) & 1u) ^ ((hm >> 16) & 1u);
      c.nfix = (int)((bm >> 8) & 0xFF) + (int)anti_ks + (int)((hm >> 8) & 0xFF);
      c.uni = (T)(__ldg(&B->dmid) + H.dT - sigma + (anti_ks ? -0.25 : 0.25));
      c.C = g.cls_C[w];
      const uint32_t base = H.R + __ldg(&B->lo);
      // RB rows per lane at a time: every load of the batch is issued before
      // any arithmetic or store, so that 6 RB loads per lane are in flight
      constexpr int RB = 4;
      for (int r0 = lane; r0 < c.C; r0 += 32 * RB) {
        T va[RB], vb[RB], vc[RB], vd[RB], ve[RB], vf[RB];
#pragma unroll
        for (int j = 0; j < RB; ++j) {
          const int r = r0 + 32 * j;
          const uint32_t i = base + (uint32_t)(r < c.C ? r : 0);
          const bool ok = r < c.C;
          if constexpr (MODE == ROWS_INIT) {
            va[j] = ok ? bv[i] : T(0);
          } else {
            va[j] = ok ? qn[i] : T(0);                                // q_{k-1}
            vb[j] = ok && doC ? dA[i] : T(0);                         // d_{k-2}
            vc[j] = ok && doC ? dB[i] : T(0);                         // d_{k-3}
            vd[j] = ok && doC ? xv[i] : T(0);                         // x
            ve[j] = ok && doQ ? pv[i] : T(0);                         // p
            vf[j] = ok && doQ ? qc[i] : T(0);                         // q_k
          }
        }
#pragma unroll
        for (int j = 0; j < RB; ++j) {
          const int r = r0 + 32 * j;
          if (r >= c.C) continue;
          int naf;
          const T am = sb_diag<T>(c, r, naf);
          const T mm = sb_precond<PC, T>(am, naf);
          const uint32_t i = base + (uint32_t)r;
          if constexpr (MODE == ROWS_INIT) {
            // a Jacobi entry at the rounding level of a_ii - sigma counts as
            // a_ii = sigma (Sec. II assumes a_ii != sigma)
            const bool zero = !(mm > mtiny);
            zm += zero ? T(1) : T(0);
            const T q = zero ? T(0) : va[j] / mm;
            ((T*)v.q1)[i] = q;
            ((T*)v.q0)[i] = T(0);
            ((T*)v.d0)[i] = T(0);
            ((T*)v.d1)[i] = T(0);
            ((T*)v.x)[i] = T(0);
            acc += q * va[j];
          } else {
            if (doC) {
              // d_{k-1} = (q_{k-1} / beta_{k-1} - delta d_{k-2} - eps d_{k-3}) / gamma_{k-1};
              // x_{k-1} = x_{k-2} + tau_{k-1} d_{k-1}
              const T d = cq * va[j] + cd1 * vb[j] + cd2 * vc[j];
              dB[i] = d;
              xv[i] = vd[j] + tau * d;
            }
            if (doQ) {
              // q_{k+1} = M^-1 p / beta_k - (alpha_k / beta_k) q_k - (beta_k / beta_{k-1}) q_{k-1}
              const T q = (ve[j] / mm) * c1 - c2 * vf[j] - c3 * va[j];
              qn[i] = q;
              acc += mm * q * q;                             // beta_{k+1}^2 = q . M q
            }
          }
        }
      }
    }
  }
  double vv[2] = {(double)acc, (double)zm}, tot[2];
  if (last_cta_sum<2>(vv, s_red, ma.partial, ma.counter, tot) && threadIdx.x == 0) {
    if constexpr (MODE == ROWS_INIT) {
      MinresState S;
      init_state(S, tot[0], tot[1], tol, kmax, sigma);
      *ma.st = S;
    } else {
      MinresState S = *ma.st;
      if (doQ) {
        givens_update(S, tot[0]);     // sets the pending update of iteration k
      } else {
        S.pending = 0;                // the last update is applied
        S.done = 2;
      }
      *ma.st = S;
    }
  }
}

template <typename T>
__host__ __device__ inline size_t rows_smem_bytes(int nlow) {
  return sizeof(Low16) * (size_t)nlow + (sizeof(T) == 8 ? sizeof(double) * (size_t)nlow : 0);
}

}  // namespace sb
}  // namespace hs
