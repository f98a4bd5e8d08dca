// Preconditioned MINRES of Algorithm 2 (Appendix A) on (H - sigma) x = b,
// fused with the matrix-free H x, plus the FP64 iterative refinement driver.
//
// Reformulation (same arithmetic in exact arithmetic): the listing keeps both
// z_k and q_k = M^-1 z_k. With M diagonal, z_k = M q_k, so only q is stored:
//   q_{k+1} = M^-1 p_k / beta_k - (alpha_k / beta_k) q_k - (beta_k / beta_{k-1}) q_{k-1}
//   beta_{k+1}^2 = q_{k+1} . z_{k+1} = sum_i M_ii q_{k+1,i}^2.
// One iteration is two passes, each ending in a last-CTA reduction that runs
// the scalar recurrences on the device (no host round trip):
//   pass A_k: [d_{k-1} = (q_{k-1}/beta_{k-1} - delta d_{k-2} - eps d_{k-3}) / gamma;
//              x += tau d_{k-1}]  (the update of iteration k-1, now that
//              gamma_{k-1} is known)  +  p_k = (H - sigma) q_k, alpha_k = q_k.p_k / beta_k^2
//   pass B_k:  q_{k+1} (above), beta_{k+1}; Givens rotation of the listing.
// Vectors: q (2, ping-pong by k parity), d (2), p, x.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "minres_smem.cuh"

namespace hs {

// ---------------------------------------------------------------------------
// Row passes shared by the per-pass kernels and the persistent kernel. Each
// adds this thread's contribution to the pass's reduction into acc.
template <typename T, int PC>
__device__ __forceinline__ void rows_init(const Geo& g, const RowSmem<T>& s, double sigma,
                                          const T* __restrict__ bv, const MinresVecs& v, T& acc,
                                          int& zero_m) {
  T* q0 = (T*)v.q0; T* q1 = (T*)v.q1; T* d0 = (T*)v.d0; T* d1 = (T*)v.d1; T* x = (T*)v.x;
  const int lane = threadIdx.x & 31;
  for_blocks(g, sigma, [&](const Hdr& h) {
    for (int r = lane; r < h.C; r += 32) {
      T am;
      const T m = row_m<T, PC>(s.low[h.off + r], h, am);
      const uint32_t i = h.R + r;
      const T b = bv[i];
      zero_m += (m == T(0));
      const T q = m == T(0) ? T(0) : b / m;
      q1[i] = q; q0[i] = T(0); d0[i] = T(0); d1[i] = T(0); x[i] = T(0);
      acc += q * b;
    }
  });
}

// pass A_k: optional pending d/x update of iteration k-1, then p = (H - sigma) q_k.
template <typename T, bool COH>
__device__ __forceinline__ void rows_A(const Geo& g, const RowSmem<T>& s, double sigma,
                                       const MinresVecs& v, long long k, bool doC, bool doMV,
                                       T cq, T cd1, T cd2, T tau, T& acc) {
  const bool odd = (k & 1) != 0;
  const T* qc = (const T*)(odd ? v.q1 : v.q0);   // q_k
  const T* qp = (const T*)(odd ? v.q0 : v.q1);   // q_{k-1}
  const T* dA = (const T*)(odd ? v.d1 : v.d0);   // d_{k-2}
  T* dB = (T*)(odd ? v.d0 : v.d1);               // d_{k-3} -> d_{k-1}
  T* p = (T*)v.p;
  T* x = (T*)v.x;
  const int lane = threadIdx.x & 31;
  for_blocks(g, sigma, [&](const Hdr& h) {
    if (doC) {
      for (int r = lane; r < h.C; r += 32) {
        const uint32_t i = h.R + r;
        const T d = cq * qp[i] + cd1 * dA[i] + cd2 * dB[i];
        dB[i] = d;
        x[i] += tau * d;
      }
    }
    if (doMV) {
      T xi[JMAX], hx[JMAX];
      block_hv<T, COH>(qc, s, h, xi, hx);
#pragma unroll
      for (int j = 0; j < JMAX; ++j) {
        const int r = lane + 32 * j;
        if (j < h.J && r < h.C) {
          p[h.R + r] = hx[j];
          acc += xi[j] * hx[j];
        }
      }
    }
  });
}

// pass B_k: q_{k+1} = M^-1 p / beta_k - (alpha_k / beta_k) q_k - (beta_k / beta_{k-1}) q_{k-1}
template <typename T, int PC>
__device__ __forceinline__ void rows_B(const Geo& g, const RowSmem<T>& s, double sigma,
                                       const MinresVecs& v, long long k, T c1, T c2, T c3,
                                       T& acc) {
  const bool odd = (k & 1) != 0;
  const T* qc = (const T*)(odd ? v.q1 : v.q0);   // q_k
  T* qn = (T*)(odd ? v.q0 : v.q1);               // q_{k-1} -> q_{k+1}
  const T* p = (const T*)v.p;
  const int lane = threadIdx.x & 31;
  for_blocks(g, sigma, [&](const Hdr& h) {
    for (int r = lane; r < h.C; r += 32) {
      const uint32_t i = h.R + r;
      T m = T(1), am;
      if (PC != 0) m = row_m<T, PC>(s.low[h.off + r], h, am);
      const T q = (p[i] / m) * c1 - c2 * qc[i] - c3 * qn[i];
      qn[i] = q;
      acc += m * q * q;
    }
  });
}

// ---------------------------------------------------------------------------
// Persistent form: one cooperative launch runs the whole solve. Every CTA
// writes its partial sum, meets the others at a bounded grid barrier and then
// adds all partials in the same fixed order, so every CTA holds identical
// scalars without a second barrier.

// Returns false in every thread if the wait hit its limit or another CTA
// reported an error; the caller then leaves the kernel.
__device__ __forceinline__ bool grid_sync(const GridBar& gb, unsigned long long limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g0 = ld_acquire_u32(gb.gen);
    __threadfence();
    const unsigned a = atomicAdd(gb.count, 1u);
    if (a == gridDim.x - 1) {
      atomicExch(gb.count, 0u);
      __threadfence();
      atomicAdd(gb.gen, 1u);
    } else {
      unsigned long long it = 0;
      while (ld_acquire_u32(gb.gen) == g0) {
        if (++it > limit) { atomicExch(gb.err, 1); ok = 0; break; }
        if ((it & 1023ull) == 0 && ld_relaxed_i32(gb.err)) { ok = 0; break; }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Sum the per-CTA partials (NV values, stride 2) in a fixed order; thread 0..31
// of every CTA compute the same totals. Result broadcast through shared memory.
template <int NV>
__device__ __forceinline__ void sum_all(const double* part, double (&tot)[NV], double* sbuf) {
  if (threadIdx.x < 32) {
    double a[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) a[j] = 0.0;
    for (int c = threadIdx.x; c < (int)gridDim.x; c += 32)
#pragma unroll
      for (int j = 0; j < NV; ++j) a[j] += __ldcg(part + 2 * c + j);
#pragma unroll
    for (int j = 0; j < NV; ++j)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a[j] += __shfl_xor_sync(0xffffffffu, a[j], o);
    if (threadIdx.x == 0)
#pragma unroll
      for (int j = 0; j < NV; ++j) sbuf[j] = a[j];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) tot[j] = sbuf[j];
}

template <typename T, int PC>
__global__ void __launch_bounds__(HV_THREADS) k_minres_persist(Geo g, const T* __restrict__ bv,
                                                               MinresVecs v, MinresState* st,
                                                               double tol, long long kmax,
                                                               const double* d_sigma,
                                                               double* part, GridBar gb,
                                                               unsigned long long limit) {
  extern __shared__ __align__(16) char smem[];
  __shared__ MinresState S;
  __shared__ double sbuf[4];
  const RowSmem<T> s = row_smem_setup<T>(smem, g);
  const double sigma = *d_sigma;
  const int G = gridDim.x;
  int red = 0;   // reduction counter -> partial buffer parity
  auto reduce = [&](double v0, double v1, double (&tot)[2]) -> bool {
    double vv[2] = {v0, v1};
    block_sum<2>(vv, s.red);
    double* buf = part + (size_t)(red & 1) * 2 * G;
    if (threadIdx.x == 0) { buf[2 * blockIdx.x] = vv[0]; buf[2 * blockIdx.x + 1] = vv[1]; }
    ++red;
    if (!grid_sync(gb, limit)) return false;
    sum_all<2>(buf, tot, sbuf);
    return true;
  };
  bool ok = true;
  {
    T acc = T(0);
    int zm = 0;
    rows_init<T, PC>(g, s, sigma, bv, v, acc, zm);
    double tot[2];
    ok = reduce((double)acc, (double)zm, tot);
    if (ok && threadIdx.x == 0) init_state(S, tot[0], tot[1], tol, kmax, sigma);
    __syncthreads();
  }
  while (ok && S.done != 2) {
    // pass A
    const bool doC = S.pending != 0, doMV = S.done == 0;
    T acc = T(0);
    rows_A<T, true>(g, s, sigma, v, S.k, doC, doMV, (T)S.cq, (T)S.cd1, (T)S.cd2, (T)S.tau, acc);
    if (!doMV) {                       // the final pending update only
      __syncthreads();
      if (threadIdx.x == 0) { S.pending = 0; S.done = 2; }
      __syncthreads();
      break;
    }
    double tot[2];
    if (!(ok = reduce((double)acc, 0.0, tot))) break;
    if (threadIdx.x == 0) {
      S.pending = 0;
      S.alpha = tot[0] / (S.beta * S.beta);
      if (!isfinite(S.alpha)) { S.status = HS_NONFINITE; S.done = 2; }
    }
    __syncthreads();
    if (S.done == 2) break;
    // pass B
    const double bk = S.beta;
    T acc2 = T(0);
    rows_B<T, PC>(g, s, sigma, v, S.k, (T)(1.0 / bk), (T)(S.alpha / bk), (T)(bk / S.beta_prev),
                  acc2);
    if (!(ok = reduce((double)acc2, 0.0, tot))) break;
    if (threadIdx.x == 0) givens_update(S, tot[0]);
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (!ok) { S.status = HS_TIMEOUT; S.done = 2; }
    *st = S;
  }
}

// ---------------------------------------------------------------------------
// Shared-memory-resident persistent form, for problems whose per-SM share of
// the vectors fits on chip (L <= 20 in FP64, L <= 22 in FP32). One CTA per SM
// owns a contiguous range of blocks; its rows of p, d_{k-1}, d_{k-2}, x and of
// both q iterates stay in shared memory for the whole solve, so the only
// global traffic per iteration is the gather of q_k for the off-diagonal
// terms and the write of q_{k+1}. Same arithmetic, same order as the other
// forms (rows_* above).

template <typename T, int PC, int JM, int NT>
__global__ void __launch_bounds__(NT, 1) k_minres_smem(SmemJob job0, SmemQueue q0, SmemQueue q1,
                                                       int ctas0) {
  extern __shared__ __align__(16) char smem[];
  __shared__ MinresState S;
  __shared__ SmemJob sj;
  __shared__ double sbuf[4];
  __shared__ double s_ib, s_ibp;
  __shared__ int s_ok;
  const bool second = (int)blockIdx.x >= ctas0;
  const SmemQueue& q = second ? q1 : q0;
  Grp2<T> c = grp2_setup<T>(q, (int)blockIdx.x - (second ? ctas0 : 0), smem, &S, &sj, sbuf, &s_ib,
                            &s_ibp, &s_ok);
  for (int njob = 0;; ++njob) {
    // the next job: CTA 0 of the group takes it from the queue and a group
    // reduction hands the index to the other CTAs
    int jid = 0;
    if (q.jobs) {
      double tot[2];
      const T v = (c.cta == 0 && threadIdx.x == 0) ? (T)atomicAdd(q.head, 1) : T(0);
      if (!grp_reduce2(c, v, T(0), tot)) break;
      jid = (int)tot[0];
      if (jid >= __ldcg(q.head + 1)) break;
    } else if (njob > 0) {
      break;
    }
    if (threadIdx.x == 0) sj = q.jobs ? q.jobs[jid] : job0;
    __syncthreads();
    if (!smem_solve2<T, PC, JM, NT>(c)) break;
  }
}

// Per-pass kernels (graph path, used when a cooperative launch is not
// available): the same row passes, with last-CTA reductions.
template <typename T, int PC>
__global__ void __launch_bounds__(HV_THREADS) k_minres_init(Geo g, const T* __restrict__ bv,
                                                            MinresVecs v, MinresState* st,
                                                            double tol, long long kmax,
                                                            double* partial, unsigned* counter,
                                                            const double* d_sigma) {
  extern __shared__ __align__(16) char smem[];
  const RowSmem<T> s = row_smem_setup<T>(smem, g);
  const double sigma = *d_sigma;
  T acc = T(0);
  int zero_m = 0;
  rows_init<T, PC>(g, s, sigma, bv, v, acc, zero_m);
  double vv[2] = {(double)acc, (double)zero_m}, tot[2];
  if (last_cta_sum<2>(vv, s.red, partial, counter, tot) && threadIdx.x == 0) {
    MinresState S;
    init_state(S, tot[0], tot[1], tol, kmax, sigma);
    *st = S;
  }
}

template <typename T, int PC>
__global__ void __launch_bounds__(HV_THREADS) k_minres_A(Geo g, MinresVecs v, MinresState* st,
                                                         double* partial, unsigned* counter) {
  extern __shared__ __align__(16) char smem[];
  __shared__ double s_c[5];
  __shared__ long long s_k;
  __shared__ int s_pending, s_done;
  if (threadIdx.x == 0) {
    s_done = st->done; s_pending = st->pending; s_k = st->k;
    s_c[0] = st->cq; s_c[1] = st->cd1; s_c[2] = st->cd2; s_c[3] = st->tau; s_c[4] = st->sigma;
  }
  __syncthreads();
  if (s_done == 2) return;
  const RowSmem<T> s = row_smem_setup<T>(smem, g);
  T acc = T(0);
  rows_A<T, false>(g, s, s_c[4], v, s_k, s_pending != 0, s_done == 0, (T)s_c[0], (T)s_c[1], (T)s_c[2],
            (T)s_c[3], acc);
  double vv[1] = {(double)acc}, tot[1];
  if (last_cta_sum<1>(vv, s.red, partial, counter, tot) && threadIdx.x == 0) {
    if (s_done == 0) {
      const double bk = st->beta;
      st->alpha = tot[0] / (bk * bk);
      if (!isfinite(st->alpha)) { st->status = HS_NONFINITE; st->done = 2; }
    } else {
      st->done = 2;
    }
    st->pending = 0;
  }
}

template <typename T, int PC>
__global__ void __launch_bounds__(HV_THREADS) k_minres_B(Geo g, MinresVecs v, MinresState* st,
                                                         double* partial, unsigned* counter) {
  extern __shared__ __align__(16) char smem[];
  __shared__ double s_c[4];
  __shared__ long long s_k;
  __shared__ int s_done;
  if (threadIdx.x == 0) {
    s_done = st->done; s_k = st->k;
    const double bk = st->beta;
    s_c[0] = 1.0 / bk; s_c[1] = st->alpha / bk; s_c[2] = bk / st->beta_prev; s_c[3] = st->sigma;
  }
  __syncthreads();
  if (s_done != 0) return;
  const RowSmem<T> s = row_smem_setup<T>(smem, g);
  T acc = T(0);
  rows_B<T, PC>(g, s, s_c[3], v, s_k, (T)s_c[0], (T)s_c[1], (T)s_c[2], acc);
  double vv[1] = {(double)acc}, tot[1];
  if (last_cta_sum<1>(vv, s.red, partial, counter, tot) && threadIdx.x == 0) {
    MinresState S = *st;
    givens_update(S, tot[0]);
    *st = S;
  }
}

// ---------------------------------------------------------------------------
// Host drivers.
template <typename T>
static hs_status ensure_ws(hs_handle* hd, MinresVecs& v) {
  const size_t vec = ((size_t)hd->n * sizeof(T) + 255) & ~size_t(255);
  const size_t need = 6 * vec;
  void** ws = sizeof(T) == 8 ? &hd->ws64 : &hd->ws32;
  size_t* wsb = sizeof(T) == 8 ? &hd->ws64_bytes : &hd->ws32_bytes;
  if (*wsb < need) {
    dev_free(hd, *ws);
    *ws = nullptr; *wsb = 0;
    cudaGraphExec_t* gr = sizeof(T) == 8 ? hd->graph64 : hd->graph32;
    for (int i = 0; i < 3; ++i)
      if (gr[i]) { cudaGraphExecDestroy(gr[i]); gr[i] = nullptr; }
    sb_graphs_release(hd, sizeof(T) == 8 ? 1 : 0);
    if (dev_alloc(hd, ws, need) != HS_OK)
      return fail(hd, HS_OOM, "MINRES workspace allocation failed");
    *wsb = need;
  }
  char* b = (char*)*ws;
  v.q0 = b; v.q1 = b + vec; v.d0 = b + 2 * vec; v.d1 = b + 3 * vec; v.p = b + 4 * vec;
  v.x = b + 5 * vec;
  if (!hd->d_state) {
    hs_status st = dev_alloc(hd, (void**)&hd->d_state, sizeof(MinresState));
    if (st != HS_OK) return st;
    hd->h_state = static_cast<MinresState*>(host_pinned_get(sizeof(MinresState)));
    if (!hd->h_state) return fail(hd, HS_OOM, "pinned host allocation failed");
  }
  return ensure_reduce(hd);
}

template <typename T, int PC>
static void enqueue_iters(hs_handle* hd, const MinresVecs& v, int iters, cudaStream_t s) {
  const Geo g = hd->geo();
  const size_t sm = row_smem_bytes<T>((int)hd->low.size());
  const int grid = row_grid(hd);
  for (int it = 0; it < iters; ++it) {
    k_minres_A<T, PC><<<grid, HV_THREADS, sm, s>>>(g, v, hd->d_state, hd->d_partial,
                                                   hd->d_counter + 1);
    k_minres_B<T, PC><<<grid, HV_THREADS, sm, s>>>(g, v, hd->d_state, hd->d_partial,
                                                   hd->d_counter + 2);
  }
}

template <typename T, int PC>
static hs_status set_attrs(hs_handle* hd) {
  const size_t sm = row_smem_bytes<T>((int)hd->low.size());
  if (sm > 48 * 1024) {
    HS_CUDA_TRY(hd, cudaFuncSetAttribute(k_minres_init<T, PC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    HS_CUDA_TRY(hd, cudaFuncSetAttribute(k_minres_A<T, PC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    HS_CUDA_TRY(hd, cudaFuncSetAttribute(k_minres_B<T, PC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  }
  return HS_OK;
}

// Iterations per captured graph: more for small (latency-bound) problems.
static int chunk_iters(const hs_handle* hd) {
  if (hd->n <= (1LL << 20)) return 64;
  if (hd->n <= (1LL << 24)) return 16;
  return 4;
}

template <typename T, int PC>
static hs_status get_graph(hs_handle* hd, const MinresVecs& v, cudaGraphExec_t& exec) {
  cudaGraphExec_t* gr = sizeof(T) == 8 ? hd->graph64 : hd->graph32;
  const int iters = chunk_iters(hd);
  if (gr[PC]) { exec = gr[PC]; return HS_OK; }
  cudaStream_t cs;
  HS_CUDA_TRY(hd, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    enqueue_iters<T, PC>(hd, v, iters, cs);
    e = cudaStreamEndCapture(cs, &graph);
  }
  if (e == cudaSuccess) {
    e = cudaGraphInstantiate(&gr[PC], graph, 0);
    cudaGraphDestroy(graph);
  }
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return fail(hd, HS_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  exec = gr[PC];
  return HS_OK;
}

// Contiguous block ranges per CTA with balanced row counts (cached per grid).
hs_status smr_plan(hs_handle* hd, int G, int** d_first, int* rows_cap, int* hdr_cap) {
  if (hd->smr_grid == G && hd->d_smr_first) {
    *d_first = hd->d_smr_first; *rows_cap = hd->smr_rows_cap; *hdr_cap = hd->smr_hdr_cap;
    return HS_OK;
  }
  const int nb = (int)hd->blocks.size();
  std::vector<int> first(G + 1, nb);
  const double per = (double)hd->n / G;
  int b = 0;
  for (int c = 0; c < G; ++c) {
    first[c] = b;
    const double end = per * (c + 1);
    while (b < nb && (c == G - 1 || (double)hd->blocks[b].R + hd->cls_C[hd->blocks[b].w] <= end + 0.5 * hd->cls_C[hd->blocks[b].w]))
      ++b;
  }
  first[G] = nb;
  int rc = 0, hc = 0;
  for (int c = 0; c < G; ++c) {
    const int lo = first[c], hi = first[c + 1];
    long long rows = 0;
    for (int i = lo; i < hi; ++i) rows += hd->cls_C[hd->blocks[i].w];
    rc = std::max<int>(rc, (int)rows);
    hc = std::max(hc, hi - lo);
  }
  rc = (rc + 3) & ~3;
  dev_free(hd, hd->d_smr_first);
  hd->d_smr_first = nullptr;
  {
    hs_status st = dev_alloc(hd, (void**)&hd->d_smr_first, sizeof(int) * (G + 1));
    if (st != HS_OK) return st;
  }
  // pageable source: the copy is staged before the call returns
  HS_CUDA_TRY(hd, cudaMemcpyAsync(hd->d_smr_first, first.data(), sizeof(int) * (G + 1),
                                  cudaMemcpyHostToDevice, hd->stream));
  hd->smr_grid = G; hd->smr_rows_cap = rc; hd->smr_hdr_cap = hc;
  *d_first = hd->d_smr_first; *rows_cap = rc; *hdr_cap = hc;
  return HS_OK;
}

// Launch of the two-reduction kernel for one or two queues; HS_CUDA without a
// message when it does not fit in shared memory or the cooperative launch is
// refused.
template <typename T, int PC, int JM, int NT>
static hs_status launch2_t(int device, cudaStream_t s, const SmemJob& job0,
                           const SmemQueue (&q)[2], const int (&ng)[2], const int (&hc)[2]) {
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  size_t sm = smr_bytes<T>(q[0].nlow, hc[0], q[0].rows_cap, NT);
  if (ng[1] > 0) sm = std::max(sm, smr_bytes<T>(q[1].nlow, hc[1], q[1].rows_cap, NT));
  if (sm + SMEM_STATIC_BYTES > (size_t)optin) return HS_CUDA;
  if (cudaFuncSetAttribute(k_minres_smem<T, PC, JM, NT>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) {
    cudaGetLastError();
    return HS_CUDA;
  }
  SmemJob j = job0;
  SmemQueue q0 = q[0], q1 = ng[1] > 0 ? q[1] : q[0];
  int ctas0 = ng[0] * q[0].S;
  void* args[] = {&j, &q0, &q1, &ctas0};
  const int grid = ctas0 + (ng[1] > 0 ? ng[1] * q[1].S : 0);
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_minres_smem<T, PC, JM, NT>,
                                                    dim3(grid), dim3(NT), args, sm, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HS_CUDA;
  }
  count_launches(1);
  return HS_OK;
}

// Blocks of at most 96 rows (k <= 8) take 3 rows per lane and 1024 threads
// (FP32) or 512 (FP64 rows need more than the 64 registers a 1024-thread CTA
// allows); larger blocks 8 rows per lane and 512 threads.
template <typename T, int PC>
static hs_status launch2_pc(int k, int device, cudaStream_t s, const SmemJob& job0,
                            const SmemQueue (&q)[2], const int (&ng)[2], const int (&hc)[2]) {
  if (k <= 8) {
    if constexpr (sizeof(T) == 8) return launch2_t<T, PC, 3, 512>(device, s, job0, q, ng, hc);
    else return launch2_t<T, PC, 3, 1024>(device, s, job0, q, ng, hc);
  }
  return launch2_t<T, PC, JMAX, 512>(device, s, job0, q, ng, hc);
}

hs_status launch_smem2(hs_dtype dt, int pc, int k, int device, cudaStream_t s,
                       const SmemJob& job0, const SmemQueue (&q)[2], const int (&ng)[2],
                       const int (&hc)[2]) {
  if (dt == HS_F64)
    return pc == 0 ? launch2_pc<double, 0>(k, device, s, job0, q, ng, hc)
         : pc == 1 ? launch2_pc<double, 1>(k, device, s, job0, q, ng, hc)
                   : launch2_pc<double, 2>(k, device, s, job0, q, ng, hc);
  return pc == 0 ? launch2_pc<float, 0>(k, device, s, job0, q, ng, hc)
       : pc == 1 ? launch2_pc<float, 1>(k, device, s, job0, q, ng, hc)
                 : launch2_pc<float, 2>(k, device, s, job0, q, ng, hc);
}

// One solve in a shared-memory form (one job, one group of G CTAs): the queue
// of the handle's workspace. one = the one-reduction kernel (minres_pipe.cu).
// HS_CUDA without a message when the form does not apply.
hs_status solve_smem_job(hs_handle* hd, const void* b, const MinresVecs& v, hs_dtype dt, int pc,
                         double tol, long long kmax, bool one) {
  const int bud = hd->sm_budget.load(std::memory_order_relaxed);
  const int G = std::max(1, std::min(hd->num_sms, bud > 0 ? bud : hd->num_sms));
  if (G > 256) return HS_CUDA;
  int* first = nullptr;
  int rows_cap = 0, hdr_cap = 0;
  hs_status st = smr_plan(hd, G, &first, &rows_cap, &hdr_cap);
  if (st != HS_OK) return st;
  HS_CUDA_TRY(hd, cudaMemsetAsync(hd->d_counter + 10, 0, sizeof(unsigned), hd->stream));
  // generation slots start from zero for every solve (a stale generation left
  // by a previous solve must never read as an arrival)
  HS_CUDA_TRY(hd, cudaMemsetAsync(hd->d_partial, 0, 2 * sizeof(SlotN) * G, hd->stream));
  unsigned long long limit = 1ull << 22;
  if (const char* e = getenv("HS_BARRIER_LIMIT")) limit = strtoull(e, nullptr, 10);
  SmemJob job{hd->geo(), b, v.x, hd->d_state, hd->sigma, tol, kmax};
  SmemQueue q{};
  q.jobs = nullptr;
  q.head = nullptr;
  q.S = G;
  q.nlow = (int)hd->low.size();
  q.slots = hd->d_partial;
  q.err = reinterpret_cast<int*>(hd->d_counter + 10);
  q.limit = limit;
  q.cta_first = first;
  q.rows_cap = rows_cap;
  q.w[0] = v.q0; q.w[1] = v.q1; q.w[2] = v.p;
  q.ws_stride = 0;
  const SmemQueue qs[2] = {q, q};
  const int ng[2] = {1, 0}, hc[2] = {hdr_cap, 0};
  st = one ? launch_smem1(dt, pc, hd->k, hd->device, hd->stream, job, qs, ng, hc,
                          pipe_replace_period())
           : launch_smem2(dt, pc, hd->k, hd->device, hd->stream, job, qs, ng, hc);
  if (st != HS_OK) return st;
  HS_CUDA_TRY(hd, cudaMemcpyAsync(hd->h_state, hd->d_state, sizeof(MinresState),
                                  cudaMemcpyDeviceToHost, hd->stream));
  HS_CUDA_TRY(hd, cudaStreamSynchronize(hd->stream));
  const MinresState& S = *hd->h_state;
  if (one && S.status == HS_BREAKDOWN && S.pad == PIPE_EXPANSION) return HS_CUDA;
  return HS_OK;
}

template <typename T, int PC>
static hs_status solve_smem(hs_handle* hd, const T* b, const MinresVecs& v, double tol,
                            long long kmax) {
  return solve_smem_job(hd, b, v, sizeof(T) == 8 ? HS_F64 : HS_F32, PC, tol, kmax, false);
}

template <typename T, int PC>
static int persist_grid(hs_handle* hd, size_t sm) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_minres_persist<T, PC>, HV_THREADS,
                                                    sm) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int bud = hd->sm_budget.load(std::memory_order_relaxed);
  const int sms = bud > 0 ? std::min(bud, hd->num_sms) : hd->num_sms;
  const int cap = std::min(per_sm, 4) * sms;
  return std::min(cap, row_grid(hd));
}

// Persistent solve; returns HS_CUDA (without an error message) when the
// cooperative launch is unavailable so that the caller falls back.
template <typename T, int PC>
static hs_status solve_persist(hs_handle* hd, const T* b, const MinresVecs& v, double tol,
                               long long kmax) {
  const size_t sm = row_smem_bytes<T>((int)hd->low.size());
  if (sm > 48 * 1024 &&
      cudaFuncSetAttribute(k_minres_persist<T, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm) != cudaSuccess) {
    cudaGetLastError();
    return HS_CUDA;
  }
  const int grid = persist_grid<T, PC>(hd, sm);
  if (grid < 1) return HS_CUDA;
  Geo g = hd->geo();
  GridBar gb{hd->d_counter + 8, hd->d_counter + 9, reinterpret_cast<int*>(hd->d_counter + 10)};
  HS_CUDA_TRY(hd, cudaMemsetAsync(hd->d_counter + 8, 0, 3 * sizeof(unsigned), hd->stream));
  double* part = hd->d_partial;                       // 2 x grid x 2 doubles
  const double* ds = hd->d_sigma;
  MinresState* st = hd->d_state;
  // Polls of the barrier word (about a microsecond each) before a wait gives
  // up with HS_TIMEOUT; HS_BARRIER_LIMIT overrides it (tests of the timeout).
  unsigned long long limit = 1ull << 22;
  if (const char* e = getenv("HS_BARRIER_LIMIT")) limit = strtoull(e, nullptr, 10);
  MinresVecs vv = v;
  void* args[] = {&g, (void*)&b, &vv, &st, &tol, &kmax, (void*)&ds, &part, &gb, &limit};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_minres_persist<T, PC>, dim3(grid),
                                              dim3(HV_THREADS), args, sm, hd->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HS_CUDA;
  }
  count_launches(1);
  HS_CUDA_TRY(hd, cudaMemcpyAsync(hd->h_state, hd->d_state, sizeof(MinresState),
                                  cudaMemcpyDeviceToHost, hd->stream));
  HS_CUDA_TRY(hd, cudaStreamSynchronize(hd->stream));
  return HS_OK;
}

template <typename T, int PC>
static hs_status solve_graph(hs_handle* hd, const T* b, const MinresVecs& v, double tol,
                             long long kmax) {
  hs_status st;
  if ((st = set_attrs<T, PC>(hd)) != HS_OK) return st;
  const Geo g = hd->geo();
  const size_t sm = row_smem_bytes<T>((int)hd->low.size());
  const int grid = row_grid(hd);
  k_minres_init<T, PC><<<grid, HV_THREADS, sm, hd->stream>>>(
      g, b, v, hd->d_state, tol, kmax, hd->d_partial, hd->d_counter + 0, hd->d_sigma); count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  cudaGraphExec_t exec;
  if ((st = get_graph<T, PC>(hd, v, exec)) != HS_OK) return st;
  int between = 1;
  while (true) {
    for (int j = 0; j < between; ++j) {
      HS_CUDA_TRY(hd, cudaGraphLaunch(exec, hd->stream));
      count_launches(2ull * chunk_iters(hd));
    }
    HS_CUDA_TRY(hd, cudaMemcpyAsync(hd->h_state, hd->d_state, sizeof(MinresState),
                                    cudaMemcpyDeviceToHost, hd->stream));
    HS_CUDA_TRY(hd, cudaStreamSynchronize(hd->stream));
    const MinresState& S = *hd->h_state;
    if (S.done == 2) break;
    between = S.done == 1 ? 1 : std::min(between * 2, 16);
  }
  return HS_OK;
}

// Solver path: 0 = persistent if possible, 1 = force the graph path.
static int g_force_graph = -1;
static bool force_graph() {
  if (g_force_graph < 0) {
    const char* e = getenv("HS_MINRES_GRAPH");
    g_force_graph = (e && e[0] == '1') ? 1 : 0;
  }
  return g_force_graph == 1;
}

// HS_MINRES_GLOBAL=1 skips the shared-memory-resident form (tests compare forms).
static bool force_global() {
  const char* e = getenv("HS_MINRES_GLOBAL");
  return e && e[0] == '1';
}

// The superblock form (minres_sb.cu) takes the solves the shared-memory form
// cannot hold, from L = 24 on. HS_MINRES_SB=0 turns it off; =1 makes it the
// first choice wherever a superblock plan exists (tests compare forms).
static int sb_choice(const hs_handle* hd) {
  const char* e = getenv("HS_MINRES_SB");
  if (e) return e[0] == '1' ? 2 : 0;
  return hd->L >= 24 ? 1 : 0;
}

// The one-reduction form (minres_pipe.cu) is the first choice for FP64 solves
// with the identity or row-norm preconditioner while a CTA holds at most 1024
// rows: there the second grid reduction of the two-reduction form is a third
// of the iteration (measured at L = 14..18 on 152 SMs: 18.5 -> 14.2, 20.7 ->
// 14.9 and 22.6 -> 18.9 us per iteration, the same iteration counts, true
// residuals within 2x of the tolerance at 1e-12). With more rows per CTA the
// extra FP64 vector work cancels the gain (L = 20 on 152 SMs, L = 16 on 6).
// Not for Jacobi, whose ill-conditioned recurrence lets the carried p drift
// (true residuals 10-100x the tolerance), nor by default for FP32, whose
// drift costs the refinement sweeps more than the faster iterations win.
// HS_MINRES_PIPE=1 makes it the first choice wherever it fits, =0 turns it off.
static bool pipe_choice(const hs_handle* hd, bool f64, int pc) {
  const char* e = getenv("HS_MINRES_PIPE");
  if (e) return e[0] == '1';
  if (!f64 || pc == 1) return false;
  const int bud = hd->sm_budget.load(std::memory_order_relaxed);
  const int G = std::max(1, std::min(hd->num_sms, bud > 0 ? bud : hd->num_sms));
  return hd->n <= 1024LL * G;
}

template <typename T, int PC>
static hs_status try_sb(hs_handle* hd, const T* b, const MinresVecs& v, double tol,
                        long long kmax) {
  bool used = false;
  const hs_status s2 = minres_solve_sb(hd, b, v, sizeof(T) == 8 ? HS_F64 : HS_F32, PC, tol,
                                       kmax, &used);
  return (used || s2 != HS_OK) ? s2 : HS_CUDA;
}

template <typename T, int PC>
static hs_status solve_pc(hs_handle* hd, const T* b, T* x, double tol, long long kmax,
                          hs_minres_info* info) {
  MinresVecs v;
  hs_status st = ensure_ws<T>(hd, v);
  if (st != HS_OK) return st;
  st = HS_CUDA;
  int form = 0;
  const int sbc = sb_choice(hd);
  if (sbc == 2 && (st = try_sb<T, PC>(hd, b, v, tol, kmax)) != HS_CUDA) form = HS_FORM_SUPERBLOCK;
  if (st == HS_CUDA && !force_graph() && !force_global() && pipe_choice(hd, sizeof(T) == 8, PC) &&
      (st = solve_smem_job(hd, b, v, sizeof(T) == 8 ? HS_F64 : HS_F32, PC, tol, kmax, true)) !=
          HS_CUDA)
    form = HS_FORM_SMEM1;
  if (st == HS_CUDA && !force_graph() && !force_global() &&
      (st = solve_smem<T, PC>(hd, b, v, tol, kmax)) != HS_CUDA)
    form = HS_FORM_SMEM;
  if (st == HS_CUDA && !force_graph() && sbc == 1 &&
      (st = try_sb<T, PC>(hd, b, v, tol, kmax)) != HS_CUDA)
    form = HS_FORM_SUPERBLOCK;
  if (st == HS_CUDA && !force_graph() &&
      (st = solve_persist<T, PC>(hd, b, v, tol, kmax)) != HS_CUDA)
    form = HS_FORM_PERSISTENT;
  if (st == HS_CUDA) {
    form = HS_FORM_GRAPH;
    if ((st = solve_graph<T, PC>(hd, b, v, tol, kmax)) != HS_OK) return st;
  }
  if (st != HS_OK) return st;
  const MinresState S = *hd->h_state;
  HS_CUDA_TRY(hd, cudaMemcpyAsync(x, v.x, sizeof(T) * hd->n, cudaMemcpyDeviceToDevice,
                                  hd->stream));
  hs_status out = (hs_status)S.status;
  if (out == HS_OK && S.beta1 > 0 && !(std::fabs(S.phi) < S.tol_abs) && S.beta != 0.0)
    out = HS_NOT_CONVERGED;
  if (info) {
    info->iters += S.k - 1;
    info->phi = S.beta1 > 0 ? std::fabs(S.phi) / S.beta1 : 0.0;
    info->status = out;
    info->form = form;
  }
  if (out != HS_OK && out != HS_NOT_CONVERGED)
    return fail(hd, out, out == HS_BREAKDOWN ? "MINRES breakdown (gamma_k = 0)"
                         : out == HS_BAD_ARG ? "Jacobi preconditioner needs a_ii != sigma"
                         : out == HS_TIMEOUT ? "grid barrier wait exceeded its limit"
                                             : "non-finite value in MINRES");
  if (out == HS_NOT_CONVERGED) hd->err = "MINRES reached kmax before the tolerance";
  return out;
}

template <typename T>
static hs_status solve_any(hs_handle* hd, const T* b, T* x, double tol, long long kmax,
                           hs_precond pc, hs_minres_info* info) {
  switch (pc) {
    case HS_PC_ID: return solve_pc<T, 0>(hd, b, x, tol, kmax, info);
    case HS_PC_JACOBI: return solve_pc<T, 1>(hd, b, x, tol, kmax, info);
    default: return solve_pc<T, 2>(hd, b, x, tol, kmax, info);
  }
}

hs_status minres_solve64(hs_handle* hd, const double* b, double* x, double tol, long long kmax,
                         hs_precond pc, hs_minres_info* info) {
  return solve_any<double>(hd, b, x, tol, kmax, pc, info);
}

hs_status minres_solve32(hs_handle* hd, const float* b, float* x, double tol, long long kmax,
                         hs_precond pc, hs_minres_info* info) {
  return solve_any<float>(hd, b, x, tol, kmax, pc, info);
}

// FP64 iterative refinement around FP32 MINRES:
//   r = b - (H - sigma) x (FP64); stop if ||r||_{M^-1} <= tol ||b||_{M^-1};
//   solve (H - sigma) dx = r / ||r||_2 in FP32 to inner_tol; x += ||r||_2 dx.
hs_status minres_mixed(hs_handle* hd, const double* b, double* x, double tol, long long kmax,
                       hs_precond pc, double inner_tol, hs_minres_info* info) {
  const long long n = hd->n;
  // FP64 residual + FP32 rhs/solution scratch live after the Lanczos-independent
  // FP64 workspace: reuse ws64 slots q0 (residual) and d0/d1 (FP32 pair).
  MinresVecs v64;
  hs_status st = ensure_ws<double>(hd, v64);
  if (st != HS_OK) return st;
  double* r = (double*)v64.q0;
  float* r32 = (float*)v64.d0;           // n floats fit in an n-double slot
  float* dx32 = (float*)v64.d1;
  HS_CUDA_TRY(hd, cudaMemsetAsync(x, 0, sizeof(double) * n, hd->stream));
  double sums[4];
  long long left = kmax;
  double best = INFINITY;
  int stall = 0;
  hs_status out = HS_NOT_CONVERGED;
  int sweeps = 0;
  for (int sweep = 0; sweep < 64; ++sweep) {
    // x = 0 before the first sweep: r = b without a product
    if ((st = resid64(hd, b, x, r, pc, sums, sweep == 0)) != HS_OK) return st;
    const double bM = std::sqrt(sums[2]), rM = std::sqrt(sums[0]);
    const double rel = bM > 0 ? rM / bM : 0.0;
    if (info) {
      info->resid_minv = rel;
      info->resid_2 = sums[3] > 0 ? std::sqrt(sums[1] / sums[3]) : 0.0;
    }
    if (!std::isfinite(rel)) return fail(hd, HS_NONFINITE, "non-finite residual");
    if (rel <= tol || bM == 0.0) { out = HS_OK; break; }
    if (left <= 0) break;
    if (rel < 0.5 * best) { best = rel; stall = 0; }
    else if (++stall >= 3) break;
    if (rel < best) best = rel;
    const double rn = std::sqrt(sums[1]);
    if ((st = vcopy_f64_to_f32(hd, r, 1.0 / rn, r32, n)) != HS_OK) return st;
    // the inner solve need not go below what the outer tolerance asks for
    const double itol = std::max(inner_tol, 0.5 * tol / rel);
    hs_minres_info in{};
    st = minres_solve32(hd, r32, dx32, itol, left, pc, &in);
    if (st != HS_OK && st != HS_NOT_CONVERGED) return st;
    left -= in.iters;
    if (info) { info->iters += in.iters; info->phi = in.phi; info->form = in.form; }
    ++sweeps;
    // minres_solve32 used ws32; the FP32 solution was copied to dx32
    if ((st = vaxpy_f32_to_f64(hd, rn, dx32, x, n)) != HS_OK) return st;
  }
  if (info) { info->sweeps += sweeps; info->status = out; }
  if (out != HS_OK) hd->err = "refinement stopped before the tolerance";
  return out;
}

}  // namespace hs
