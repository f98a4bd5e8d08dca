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
template <typename T, int JM>
__device__ __forceinline__ void block_hv_loc(const T* __restrict__ xg, const T* xl, const T* dg,
                                             const LowEntry* low, const Hdr& h, T (&xi)[JM],
                                             T (&hx)[JM]) {
  const int lane = threadIdx.x & 31;
  const T* xb = xg + h.R;
  T side[JM];
#pragma unroll
  for (int j = 0; j < JM; ++j) {
    xi[j] = T(0);
    side[j] = T(0);
    hx[j] = T(0);
    const int r = lane + 32 * j;
    if (j < h.J && r < h.C) {
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
      const T* xh = xb + (on ? hdr_hd(h, m0 + mm) : 0) + lane;
#pragma unroll
      for (int j = 0; j < JM; ++j)
        v[mm][j] = (on && j < h.J && lane + 32 * j < h.C) ? ldx<T, true>(xh + 32 * j) : T(0);
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
    const int r = lane + 32 * j;
    if (j < h.J && r < h.C) {
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
