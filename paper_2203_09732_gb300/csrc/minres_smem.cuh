// Device pieces of the shared-memory-resident MINRES forms (minres.cu:
// k_minres_smem, two reductions per iteration; minres_pipe.cu: k_minres_smem1,
// one): the bounded grid-barrier words, the per-CTA reduction slots, the rows
// of one block with its own segment in shared memory, CTA-wide sums and the
// scalar recurrences of Algorithm 2 (Appendix A) on one thread.
#pragma once
#include "minres_scalar.cuh"
#include "rows.cuh"

namespace hs {

// M_ii of a row (preconditioner pc) and, in am, a_ii - sigma.
template <typename T, int PC>
__device__ __forceinline__ T row_m(const LowEntry& e, const Hdr& h, T& am) {
  const uint32_t xc = cut_mask(e.packed, h);
  am = diag_t<T>(e, h, xc);
  return precond_t<PC, T>(am, naf_row(e.packed, h, xc));
}

struct GridBar {
  unsigned* count;
  unsigned* gen;
  int* err;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Per-CTA slot of the fused reduction + barrier (two partial sums and the
// generation number that marks them as published).
struct Slot {
  double v0, v1;
  unsigned gen;
  unsigned pad[3];
};

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Rows of one block whose own segment (self and low-interior neighbours) is
// read from shared memory xl; the other gathers come from global xg.
// The rows are lane + 32 (j0 + j), j < JM: the block's 32-row chunks j0 on.
template <typename T, int JM>
__device__ __forceinline__ void block_hv_loc(const T* __restrict__ xg, const T* xl, const T* dg,
                                             const LowEntry* low, const Hdr& h, T (&xi)[JM],
                                             T (&hx)[JM], int j0 = 0) {
  const int lane = threadIdx.x & 31;
  const T* xb = xg + h.R;
  T side[JM];
#pragma unroll
  for (int j = 0; j < JM; ++j) {
    xi[j] = T(0);
    side[j] = T(0);
    hx[j] = T(0);
    const int r = lane + 32 * (j0 + j);
    if (j0 + j < h.J && r < h.C) {
      const LowEntry& e = low[h.off + r];
      const uint32_t xc = cut_mask(e.packed, h);
      xi[j] = xl[r];
      const T c1 = (xc & 1u) ? ldx<T, true>(xb + h.bdelta + r) : T(0);
      const T c2 = (xc & 2u) ? ldx<T, true>(xg + (h.Rwrap + e.wrap_r)) : T(0);
      side[j] = c1 + c2;
    }
  }
  constexpr int HG = 4;
  for (int m0 = 0; m0 < h.nh; m0 += HG) {
    T v[HG][JM];
#pragma unroll
    for (int mm = 0; mm < HG; ++mm) {
      const bool on = m0 + mm < h.nh;
      const T* xh = xb + (on ? hdr_hd(h, m0 + mm) : 0) + lane + 32 * j0;
#pragma unroll
      for (int j = 0; j < JM; ++j)
        v[mm][j] = (on && j0 + j < h.J && lane + 32 * (j0 + j) < h.C) ? ldx<T, true>(xh + 32 * j)
                                                                      : T(0);
    }
    // only the bonds that exist: the count is the same for the whole warp, so
    // this skips FP64 adds of zero (the FP64 pipe bounds this pass)
#pragma unroll
    for (int mm = 0; mm < HG; ++mm)
      if (m0 + mm < h.nh)
#pragma unroll
        for (int j = 0; j < JM; ++j) hx[j] += v[mm][j];
  }
#pragma unroll
  for (int j = 0; j < JM; ++j) {
    const int r = lane + 32 * (j0 + j);
    if (j0 + j < h.J && r < h.C) {
      const LowEntry& e = low[h.off + r];
      const uint32_t pk = e.packed;
      T acc = hx[j] + side[j];
      const int cnt = le_cnt(pk);
      const uint32_t w0 = e.nbw[0], w1 = e.nbw[1], w2 = e.nbw[2];
#pragma unroll
      for (int m = 0; m < NB_MAX; ++m) {
        const uint32_t wd = m < 4 ? w0 : (m < 8 ? w1 : w2);
        if (m < cnt) acc += xl[(wd >> (8 * (m & 3))) & 0xFFu];
      }
      hx[j] = dg[r] * xi[j] + T(0.5) * acc;
    }
  }
}

// CTA-wide sum of two per-thread values; totals land in every lane of warp 0.
// FP32 values are reduced in FP32 within warps (one FP64 add tree of 32 warp
// sums follows); FP64 values go through shared memory so that one warp does the
// FP64 additions (FP64 throughput on this part is a small fraction of FP32).
template <typename T>
__device__ __forceinline__ void cta_sum2(T a, T b, double* stmp, double& o0, double& o1) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) { stmp[2 * wid] = (double)a; stmp[2 * wid + 1] = (double)b; }
    __syncthreads();
    if (wid == 0) {
      o0 = lane < nw ? stmp[2 * lane] : 0.0;
      o1 = lane < nw ? stmp[2 * lane + 1] : 0.0;
    }
  } else {
    stmp[threadIdx.x] = a;
    stmp[blockDim.x + threadIdx.x] = b;
    __syncthreads();
    if (wid == 0) {
      o0 = 0.0;
      o1 = 0.0;
      for (int i = lane; i < (int)blockDim.x; i += 32) {
        o0 += stmp[i];
        o1 += stmp[blockDim.x + i];
      }
    }
  }
  if (wid == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      o0 += __shfl_xor_sync(0xffffffffu, o0, o);
      o1 += __shfl_xor_sync(0xffffffffu, o1, o);
    }
  }
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Slot reduction for grids of at most 256 CTAs, called by warp 0 with the
// CTA's totals in (c0, c1): publish, poll every slot with independent relaxed
// loads, one acquire fence, then a fixed-order sum (identical in every CTA).
__device__ __forceinline__ bool slot_reduce_w0(Slot* slots, int G, int cta, unsigned gen,
                                               double c0, double c1, double (&tot)[2],
                                               unsigned long long limit, int* err) {
  const int lane = threadIdx.x & 31;
  Slot* buf = slots + (size_t)(gen & 1u) * G;
  if (lane == 0) {
    buf[cta].v0 = c0;
    buf[cta].v1 = c1;
    st_release_u32(&buf[cta].gen, gen);   // orders the partials and, after the
  }                                              // CTA barrier, the CTA's vector stores
  int ok = 1;
  unsigned long long it = 0;
  while (true) {
    unsigned gv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int c = lane + 32 * q;
      gv[q] = c < G ? ld_relaxed_u32(&buf[c].gen) : gen;
    }
    bool mine = true;
#pragma unroll
    for (int q = 0; q < 8; ++q) mine = mine && (gv[q] == gen);
    if (__all_sync(0xffffffffu, mine)) break;
    if (++it > limit) { ok = 0; if (lane == 0) atomicExch(err, 1); break; }
    if ((it & 255ull) == 0 && ld_relaxed_i32(err)) { ok = 0; break; }
  }
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  double a0 = 0.0, a1 = 0.0;
  if (ok) {
    double v0[8], v1[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int c = lane + 32 * q;
      v0[q] = c < G ? __ldcg(&buf[c].v0) : 0.0;
      v1[q] = c < G ? __ldcg(&buf[c].v1) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) { a0 += v0[q]; a1 += v1[q]; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    }
  }
  tot[0] = a0;
  tot[1] = a1;
  return __all_sync(0xffffffffu, ok) != 0;
}

template <typename T>
__host__ __device__ inline size_t smr_bytes(int nlow, int hdr_cap, int rows_cap, int nt) {
  size_t b = sizeof(LowEntry) * (size_t)nlow + 128 * (size_t)hdr_cap;
  b = (b + 15) & ~size_t(15);
  b += 9 * sizeof(T) * (size_t)rows_cap;
  b = (b + 15) & ~size_t(15);
  return b + sizeof(double) * (sizeof(T) == 8 ? 2 * (size_t)nt : 64);
}

// Scalar recurrences of Algorithm 2 on one thread, with one reciprocal per
// divisor (FP64 division and square root are slow here): same quantities as
// givens_update.
__device__ __forceinline__ void givens_fast(MinresState& S, double sumsq, double& ib) {
  const double bn = sumsq >= 0.0 ? sqrt(sumsq) : NAN;        // beta_{k+1}
  const double a = S.alpha, bk = S.beta;
  const double cp = S.c_prev, sp = S.s_prev, dh = S.delta_hat, eps = S.eps;
  const double delta = cp * dh + sp * a;                     // delta_k
  const double gh = -sp * dh + cp * a;                       // hat gamma_k
  const double gamma = sqrt(gh * gh + bn * bn);              // gamma_k
  if (!isfinite(bn) || !isfinite(gamma)) {
    S.status = HS_NONFINITE; S.done = 2; S.pending = 0;
    return;
  }
  if (gamma == 0.0) {
    S.status = HS_BREAKDOWN; S.done = 2; S.pending = 0;
    return;
  }
  const double rg = 1.0 / gamma;
  const double c = gh * rg, sn = bn * rg;                    // c_k, s_k
  S.tau = c * S.phi;                                         // tau_k
  S.phi = -sn * S.phi;                                       // phi_k
  S.cq = rg * ib;                                            // 1 / (beta_k gamma_k)
  S.cd1 = -delta * rg;
  S.cd2 = -eps * rg;
  S.pending = 1;
  S.eps = sp * bn;                                           // epsilon_{k+1}
  S.delta_hat = cp * bn;                                     // hat delta_{k+1}
  S.beta_prev = bk; S.beta = bn;
  S.c_prev = c; S.s_prev = sn;
  S.k = S.k + 1;
  ib = bn > 0.0 ? 1.0 / bn : 0.0;
  if (fabs(S.phi) < S.tol_abs || bn == 0.0 || S.k > S.kmax) S.done = 1;
}


// Reduction of NV <= SLOTN_VALS values: slot of one CTA (64 bytes).
constexpr int SLOTN_VALS = 6;
struct SlotN {
  double v[SLOTN_VALS];
  unsigned gen;
  unsigned pad[3];
};

// CTA-wide sums of NV per-thread values into sout[0..NV-1] (shared memory),
// visible to every thread on return. Only the first nact warps hold values.
// FP32 values are summed in FP32 within a warp and in FP64 across warps; FP64
// values are staged in shared memory (stmp: NV * blockDim.x doubles) and
// warp j adds value j, so the FP64 additions spread over NV warps.
template <typename T, int NV>
__device__ __forceinline__ void cta_sumN(const T (&a)[NV], int nact, double* stmp, double* sout) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      T v = a[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && wid < nact) stmp[j * 32 + wid] = (double)v;
    }
    __syncthreads();
    if (wid < NV) {
      double t = lane < nact ? stmp[wid * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) sout[wid] = t;
    }
  } else {
    const int nt = blockDim.x;
    if (wid < nact)
#pragma unroll
      for (int j = 0; j < NV; ++j) stmp[j * nt + threadIdx.x] = a[j];
    __syncthreads();
    if (wid < NV) {
      double t = 0.0;
      for (int i = lane; i < nact * 32; i += 32) t += stmp[wid * nt + i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) sout[wid] = t;
    }
  }
  __syncthreads();
}

// The slot reduction of slot_reduce_w0 for NV values (grids of at most 256
// CTAs), called by warp 0 with the CTA's sums in c (shared memory): publish
// with a release store of the generation, poll every slot with relaxed loads
// (bounded by limit), one acquire fence, then a fixed-order sum so that every
// CTA ends with identical totals in tot (all lanes).
template <int NV>
__device__ __forceinline__ bool slot_reduceN_w0(SlotN* slots, int G, int cta, unsigned gen,
                                                const double* c, double (&tot)[NV],
                                                unsigned long long limit, int* err) {
  const int lane = threadIdx.x & 31;
  SlotN* buf = slots + (size_t)(gen & 1u) * G;
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) buf[cta].v[j] = c[j];
    st_release_u32(&buf[cta].gen, gen);
  }
  int ok = 1;
  unsigned long long it = 0;
  while (true) {
    unsigned gv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int cc = lane + 32 * q;
      gv[q] = cc < G ? ld_relaxed_u32(&buf[cc].gen) : gen;
    }
    bool mine = true;
#pragma unroll
    for (int q = 0; q < 8; ++q) mine = mine && (gv[q] == gen);
    if (__all_sync(0xffffffffu, mine)) break;
    if (++it > limit) { ok = 0; if (lane == 0) atomicExch(err, 1); break; }
    if ((it & 255ull) == 0 && ld_relaxed_i32(err)) { ok = 0; break; }
  }
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  double acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = 0.0;
  if (ok) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int cc = lane + 32 * q;
      if (cc < G)
#pragma unroll
        for (int j = 0; j < NV; ++j) acc[j] += __ldcg(&buf[cc].v[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < NV; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
    tot[j] = acc[j];
  }
  return __all_sync(0xffffffffu, ok) != 0;
}

// One solve of a job queue: the realisation's geometry, right-hand side and
// solution (device, n elements of the solver's type), final state and
// parameters.
struct SmemJob {
  Geo g;
  const void* b;
  void* x;
  MinresState* st;
  double sigma, tol;
  long long kmax;
};

// Static shared memory of the shared-memory kernels (state, job, scalars),
// with a margin, for the fit check against the opt-in limit.
constexpr size_t SMEM_STATIC_BYTES = sizeof(MinresState) + sizeof(SmemJob) + 32 * 8 + 64;

// A job queue of a shared-memory solver launch: groups of S CTAs, each taking
// jobs until the queue is empty (head[0]: next job, atomic; head[1]: number of
// jobs, both set before the launch); jobs == nullptr runs the kernel parameter
// job0 alone, with one group. All jobs of a queue have the same L (one block
// plan, cta_first, for the S CTAs of any group; nlow low-table entries).
// slots: 2 S reduction slots per group; w[0..2]: the group's global vectors
// for the gathers, group g at w[i] + g ws_stride elements. Waits give up after
// limit polls and set *err. A launch serves up to two queues (two chain
// lengths): its first ctas0 CTAs take queue 0, the rest queue 1.
struct SmemQueue {
  const SmemJob* jobs;
  int* head;
  int S;
  int nlow;
  void* slots;
  int* err;
  unsigned long long limit;
  const int* cta_first;
  int rows_cap;
  void* w[3];
  long long ws_stride;
};

// Per-CTA context of a group's solves in the two-reduction shared-memory
// form: its queue, place in the group, reduction slots, global gather
// vectors, shared-memory layout and the shared scalars of the solve.
template <typename T>
struct Grp2 {
  const SmemQueue* q;
  int G, cta, b0, nbk;
  Slot* slots;
  T* qg0;
  T* qg1;
  char* smem;
  size_t off_rows;
  double* stmp;
  unsigned gen;
  MinresState* S;
  const SmemJob* sj;
  double* sbuf;
  double* s_ib;
  double* s_ibp;
  int* s_ok;
};

// Layout (the same for every job of a queue): low table, block headers of
// the CTA, 9 row arrays, reduction scratch.
template <typename T>
__device__ __forceinline__ Grp2<T> grp2_setup(const SmemQueue& q, int lb, char* smem,
                                              MinresState* S, const SmemJob* sj, double* sbuf,
                                              double* s_ib, double* s_ibp, int* s_ok) {
  Grp2<T> c;
  c.q = &q;
  c.G = q.S;
  const int grp = lb / c.G;
  c.cta = lb - grp * c.G;
  c.slots = reinterpret_cast<Slot*>(q.slots) + (size_t)grp * 2 * c.G;
  c.qg0 = reinterpret_cast<T*>(q.w[0]) + (size_t)grp * q.ws_stride;
  c.qg1 = reinterpret_cast<T*>(q.w[1]) + (size_t)grp * q.ws_stride;
  c.b0 = q.cta_first[c.cta];
  c.nbk = q.cta_first[c.cta + 1] - c.b0;
  c.smem = smem;
  size_t off = sizeof(LowEntry) * q.nlow + 128 * (size_t)c.nbk;
  c.off_rows = (off + 15) & ~size_t(15);
  size_t off_tmp = c.off_rows + 9 * sizeof(T) * (size_t)q.rows_cap;
  off_tmp = (off_tmp + 15) & ~size_t(15);
  c.stmp = reinterpret_cast<double*>(smem + off_tmp);
  c.gen = 0;
  c.S = S;
  c.sj = sj;
  c.sbuf = sbuf;
  c.s_ib = s_ib;
  c.s_ibp = s_ibp;
  c.s_ok = s_ok;
  return c;
}

// A group reduction of two values per thread (CTA sums, then the slots);
// totals in every thread; false when the wait gave up.
template <typename T>
__device__ __forceinline__ bool grp_reduce2(Grp2<T>& c, T a, T b, double (&tot)[2]) {
  double c0, c1;
  cta_sum2<T>(a, b, c.stmp, c0, c1);
  ++c.gen;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (wid == 0) {
    double t[2];
    const bool okw = slot_reduce_w0(c.slots, c.G, c.cta, c.gen, c0, c1, t, c.q->limit, c.q->err);
    if (lane == 0) { c.sbuf[0] = t[0]; c.sbuf[1] = t[1]; *c.s_ok = okw; }
  }
  __syncthreads();
  tot[0] = c.sbuf[0];
  tot[1] = c.sbuf[1];
  return *c.s_ok != 0;
}

// One solve of the two-reduction shared-memory form by one CTA of a group:
// the job in *c.sj (geometry, right-hand side, solution, state, parameters).
// The group's CTAs call it together; it ends with x and the final state
// written, and returns false when a wait of the group gave up (HS_TIMEOUT in
// the state).
template <typename T, int PC, int JM, int NT>
__device__ __forceinline__ bool smem_solve2(Grp2<T>& c) {
  MinresState& S = *c.S;
  const SmemJob& sj = *c.sj;
  double& s_ib = *c.s_ib;
  double& s_ibp = *c.s_ibp;
  char* smem = c.smem;
  const int b0 = c.b0, nbk = c.nbk, cta = c.cta, rows_cap = c.q->rows_cap;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* qg0 = c.qg0;
  T* qg1 = c.qg1;
  auto reduce = [&](T a, T b, double (&tot)[2]) -> bool { return grp_reduce2(c, a, b, tot); };
  bool ok = true;
  const Geo& g = sj.g;
  const T* __restrict__ bv = reinterpret_cast<const T*>(sj.b);
  T* xout = reinterpret_cast<T*>(sj.x);
  const double sigma = sj.sigma;
  LowEntry* low = reinterpret_cast<LowEntry*>(smem);
  {
    const uint4* src = reinterpret_cast<const uint4*>(g.low);
    uint4* dst = reinterpret_cast<uint4*>(low);
    for (int i = threadIdx.x; i < g.nlow * 2; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  uint32_t* hdrs = reinterpret_cast<uint32_t*>(smem + sizeof(LowEntry) * c.q->nlow);
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(g.blocks + b0);
    for (int i = threadIdx.x; i < nbk * 32; i += blockDim.x) hdrs[i] = __ldg(src + i);
  }
  T* QL0 = reinterpret_cast<T*>(smem + c.off_rows);
  T* QL1 = QL0 + rows_cap;
  T* P = QL0 + 2 * rows_cap;
  T* D0 = QL0 + 3 * rows_cap;
  T* D1 = QL0 + 4 * rows_cap;
  T* X = QL0 + 5 * rows_cap;
  T* MV = QL0 + 6 * rows_cap;        // M_ii
  T* MI = QL0 + 7 * rows_cap;        // 1 / M_ii
  T* DG = QL0 + 8 * rows_cap;        // a_ii - sigma (rebuilding it costs ~4 FP64 operations a row)
  const uint32_t Rbase = nbk > 0 ? __ldg(&g.blocks[b0].R) : 0u;
  __syncthreads();
  // Work of a pass, f(h, l0, j0, nj): chunks j0 .. j0 + nj - 1 (32 rows each)
  // of one block. Either whole blocks dealt round-robin to the warps, or, in
  // FP64 where that leaves the slowest warp with more chunks, single chunks
  // dealt round-robin in block order (the same choice in every pass of the
  // solve). Measured on 152 SMs (two-reduction form, us per iteration): FP64
  // L = 16 21.8 -> 19.6, L = 20 41.2 -> 38.1; FP32 slower by chunks (L = 20:
  // 19.9 -> 35.5), so FP32 keeps whole blocks.
  constexpr int NW = NT / 32;
  auto block_chunks = [&](int lb) {
    return (g.cls_C[hdrs[lb * 32 + 3] & 0xFFu] + 31) >> 5;   // word 3: w | ...
  };
  bool by_chunk = false;
  if constexpr (sizeof(T) == 8) {
    int tot = 0, worst = 0;
    for (int w = 0; w < NW; ++w) {
      int mine = 0;
      for (int lb = w; lb < nbk; lb += NW) mine += block_chunks(lb);
      worst = max(worst, mine);
      tot += mine;
    }
    by_chunk = (tot + NW - 1) / NW < worst;
  }
  auto each_part = [&](auto&& f) {
    if constexpr (sizeof(T) == 8) {
      if (by_chunk) {
        int t = 0;                               // chunks before block lb
        for (int lb = 0; lb < nbk; ++lb) {
          const int J = block_chunks(lb);
          int jc = (wid - t) % NW;
          if (jc < 0) jc += NW;
          if (jc < J) {
            const Hdr h = make_hdr(g, hdrs[lb * 32 + lane], sigma);
            for (; jc < J; jc += NW) f(h, h.R - Rbase, jc, 1);
          }
          t += J;
        }
        return;
      }
    }
    for (int lb = wid; lb < nbk; lb += NW) {
      const Hdr h = make_hdr(g, hdrs[lb * 32 + lane], sigma);
      f(h, h.R - Rbase, 0, h.J);
    }
  };
  // the rows of a part, one per lane and chunk
  auto each_row = [&](const Hdr& h, int j0, int nj, auto&& g_row) {
    for (int j = j0; j < j0 + nj; ++j) {
      const int r = lane + 32 * j;
      if (r < h.C) g_row(r);
    }
  };
  {
    T acc = T(0), zm = T(0);
    each_part([&](const Hdr& h, uint32_t l0, int j0, int nj) {
      each_row(h, j0, nj, [&](int r) {
        T am;
        const T m = row_m<T, PC>(low[h.off + r], h, am);
        const uint32_t i = h.R + r;
        const uint32_t l = l0 + r;
        const T b = bv[i];
        zm += (m == T(0)) ? T(1) : T(0);
        const T mi = m == T(0) ? T(0) : T(1) / m;
        const T qv = b * mi;
        MV[l] = m; MI[l] = mi; DG[l] = am;
        QL1[l] = qv; qg1[i] = qv;
        QL0[l] = T(0); D0[l] = T(0); D1[l] = T(0); X[l] = T(0);
        acc += qv * b;
      });
    });
    double tot[2];
    ok = reduce(acc, zm, tot);
    if (ok && threadIdx.x == 0) {
      init_state(S, tot[0], tot[1], sj.tol, sj.kmax, sigma);
      s_ib = S.beta > 0.0 ? 1.0 / S.beta : 0.0;
      s_ibp = 1.0;                     // 1 / beta_0
    }
    __syncthreads();
  }
  while (ok && S.done != 2) {
    const long long k = S.k;
    const bool odd = (k & 1) != 0;
    T* QLc = odd ? QL1 : QL0;          // q_k
    T* QLp = odd ? QL0 : QL1;          // q_{k-1} -> q_{k+1}
    const T* qgc = odd ? qg1 : qg0;    // q_k (global, for gathers)
    T* qgn = odd ? qg0 : qg1;          // q_{k+1}
    T* DA = odd ? D1 : D0;             // d_{k-2}
    T* DB = odd ? D0 : D1;             // d_{k-3} -> d_{k-1}
    const bool doC = S.pending != 0, doMV = S.done == 0;
    const T cq = (T)S.cq, cd1 = (T)S.cd1, cd2 = (T)S.cd2, tau = (T)S.tau;
    T acc = T(0);
    each_part([&](const Hdr& h, uint32_t l0, int j0, int nj) {
      if (doC)
        each_row(h, j0, nj, [&](int r) {
          const uint32_t l = l0 + r;
          const T d = cq * QLp[l] + cd1 * DA[l] + cd2 * DB[l];
          DB[l] = d;
          X[l] += tau * d;
        });
      if (doMV) {
        if (sizeof(T) == 8 && by_chunk) {  // one chunk
          T xi[1], hx[1];
          block_hv_loc<T, 1>(qgc, QLc + l0, DG + l0, low, h, xi, hx, j0);
          const int r = lane + 32 * j0;
          if (r < h.C) {
            P[l0 + r] = hx[0];
            acc += xi[0] * hx[0];
          }
        } else {                         // a whole block
          T xi[JM], hx[JM];
          block_hv_loc<T, JM>(qgc, QLc + l0, DG + l0, low, h, xi, hx);
#pragma unroll
          for (int j = 0; j < JM; ++j) {
            const int r = lane + 32 * j;
            if (j < h.J && r < h.C) {
              P[l0 + r] = hx[j];
              acc += xi[j] * hx[j];
            }
          }
        }
      }
    });
    if (!doMV) {
      __syncthreads();
      if (threadIdx.x == 0) { S.pending = 0; S.done = 2; }
      __syncthreads();
      break;
    }
    double tot[2];
    if (!(ok = reduce(acc, T(0), tot))) break;
    if (threadIdx.x == 0) {
      S.pending = 0;
      S.alpha = tot[0] * s_ib * s_ib;                   // q.p / beta_k^2
      if (!isfinite(S.alpha)) { S.status = HS_NONFINITE; S.done = 2; }
    }
    __syncthreads();
    if (S.done == 2) break;
    const T c1 = (T)s_ib, c2 = (T)(S.alpha * s_ib), c3 = (T)(S.beta * s_ibp);
    T acc2 = T(0);
    each_part([&](const Hdr& h, uint32_t l0, int j0, int nj) {
      each_row(h, j0, nj, [&](int r) {
        const uint32_t l = l0 + r;
        const T qv = P[l] * MI[l] * c1 - c2 * QLc[l] - c3 * QLp[l];
        QLp[l] = qv;
        qgn[h.R + r] = qv;
        acc2 += MV[l] * qv * qv;
      });
    });
    if (!(ok = reduce(acc2, T(0), tot))) break;
    if (threadIdx.x == 0) {
      double ib = s_ib;
      givens_fast(S, tot[0], ib);
      s_ibp = s_ib;
      s_ib = ib;
    }
    __syncthreads();
  }
  __syncthreads();
  each_part([&](const Hdr& h, uint32_t l0, int j0, int nj) {
    each_row(h, j0, nj, [&](int r) { xout[h.R + r] = X[l0 + r]; });
  });
  if (cta == 0 && threadIdx.x == 0) {
    if (!ok) { S.status = HS_TIMEOUT; S.done = 2; }
    *sj.st = S;
  }
  return ok;
}

// MinresState.pad of a one-reduction solve that ended because the expansion
// of beta_{k+1}^2 cancelled to rounding level (status HS_BREAKDOWN): the solve
// is to be redone by the two-reduction form.
constexpr int PIPE_EXPANSION = 1;

// Launches of the two-reduction (minres.cu) and one-reduction (minres_pipe.cu)
// kernels (k: low bits of the block layout). Asynchronous on s; HS_CUDA
// without a message when the form does not fit in shared memory or the
// cooperative launch is refused.
// ngroups[i] groups of q[i].S CTAs serve queue i (ngroups[1] = 0: one queue);
// hdr_cap[i]: most blocks per CTA of queue i's plan; smem is sized for the
// larger of the two layouts.
hs_status launch_smem2(hs_dtype dt, int pc, int k, int device, cudaStream_t s,
                       const SmemJob& job0, const SmemQueue (&q)[2], const int (&ngroups)[2],
                       const int (&hdr_cap)[2]);
hs_status launch_smem1(hs_dtype dt, int pc, int k, int device, cudaStream_t s,
                       const SmemJob& job0, const SmemQueue (&q)[2], const int (&ngroups)[2],
                       const int (&hdr_cap)[2], int rperiod);
int pipe_replace_period();

// One solve of the handle in a shared-memory form (minres.cu): one job, one
// group of all the handle's SMs; x in v.x and the state in hd->h_state.
hs_status solve_smem_job(hs_handle* hd, const void* b, const MinresVecs& v, hs_dtype dt, int pc,
                         double tol, long long kmax, bool one);

// Contiguous block ranges per CTA with balanced row counts, cached per grid
// size (minres.cu).
hs_status smr_plan(hs_handle* hd, int G, int** d_first, int* rows_cap, int* hdr_cap);

}  // namespace hs
