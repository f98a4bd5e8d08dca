// Preconditioned MINRES of Algorithm 2 (Appendix A) with one global reduction
// per iteration, shared-memory resident like k_minres_smem (one CTA per SM,
// each CTA's rows of every vector on chip; L <= 20).
//
// Algorithm 2 needs two global sums per iteration: alpha_k = q_k . p_k / beta_k^2
// before q_{k+1} can be formed, and beta_{k+1}^2 = q_{k+1} . M q_{k+1} after it.
// Here both come from one exchange, by two changes that leave the arithmetic
// of exact arithmetic unchanged:
//   * the product is applied to v_k = M^-1 p_k instead of to q_{k+1}, and p is
//     carried by the three-term recurrence of q (H - sigma is linear):
//       q_{k+1} = v_k / beta_k - a q_k - c q_{k-1},
//       p_{k+1} = (H - sigma) v_k / beta_k - a p_k - c p_{k-1},
//     a = alpha_k / beta_k, c = beta_k / beta_{k-1};
//   * beta_{k+1}^2, the M-norm of q_{k+1} as formed above, is expanded in sums
//     that exist before alpha_k is known:
//       beta_{k+1}^2 = S2 / beta_k^2 + a^2 S4 + c^2 S6
//                      - 2 a S1 / beta_k - 2 c S3 / beta_k + 2 a c S5,
//     S1 = q_k.p_k, S2 = p_k.M^-1 p_k, S3 = p_k.q_{k-1}, S4 = q_k.M q_k,
//     S5 = q_k.M q_{k-1}, S6 = q_{k-1}.M q_{k-1} (S4 of the step before). The
//     expansion does not assume M-orthogonality of the computed q.
// One iteration: the scalars of step k (alpha_k, beta_{k+1}, the Givens
// rotation) from the sums on one thread; one pass over the rows: d_k and x_k,
// (H - sigma) v_k (gathering v_k), q_{k+1}, p_{k+1}, v_{k+1} = M^-1 p_{k+1}, the
// five sums of step k+1 and the store of v_{k+1}; then one reduction, which is
// also the barrier that publishes v_{k+1}.
//
// Rounding makes p drift from (H - sigma) q; every R steps p_{k+1} is instead
// formed as the product with q_{k+1} (that step publishes q_{k+1} first: one
// extra barrier). Where the expansion cancels to rounding level (beta_{k+1}^2
// below EXPANSION_FLOOR of its terms) the solve ends with HS_BREAKDOWN and
// pad = PIPE_EXPANSION, and the caller solves again with the two-reduction form.
#include <algorithm>
#include <cstdlib>

#include "minres_smem.cuh"

namespace hs {

namespace {

constexpr int PIPE_NV = 5;           // S1..S5 (S6 is carried)

// Smallest beta_{k+1}^2 / mag (mag: the sum of the expansion's terms in
// magnitude) that the expansion is trusted with: its relative error is about
// u mag / beta_{k+1}^2, at most 1e-8 (FP64) or 6e-5 (FP32) above the floor.
// Below it (in practice: a Krylov space that has run out, as for n <= 8 or a
// right-hand side inside an invariant subspace) the solve is handed back.
template <typename T>
constexpr double EXPANSION_FLOOR = sizeof(T) == 8 ? 1e-8 : 1e-3;

// Shared memory: low table, block headers, 12 row arrays, reduction staging.
template <typename T>
size_t smr1_bytes(int nlow, int hdr_cap, int rows_cap, int nt) {
  size_t b = sizeof(LowEntry) * (size_t)nlow + 128 * (size_t)hdr_cap;
  b = (b + 15) & ~size_t(15);
  b += 12 * sizeof(T) * (size_t)rows_cap;
  b = (b + 15) & ~size_t(15);
  return b + sizeof(double) * PIPE_NV * (sizeof(T) == 8 ? (size_t)nt : 32);
}

template <typename T, int PC, int JM, int NT>
__global__ void __launch_bounds__(NT, 1) k_minres_smem1(SmemJob job0, SmemQueue q0, SmemQueue q1,
                                                        int ctas0, int rperiod) {
  extern __shared__ __align__(16) char smem[];
  __shared__ MinresState S;
  __shared__ SmemJob sj;
  __shared__ double s_sum[PIPE_NV + 1];   // S1..S5 of the current step, S6
  __shared__ double s_cta[PIPE_NV];
  __shared__ double s_c[3];               // 1/beta_k, a, c of the vector update
  __shared__ double s_ib, s_ibp;          // 1/beta_k, 1/beta_{k-1}
  __shared__ int s_ok;
  const bool second = (int)blockIdx.x >= ctas0;
  const SmemQueue& q = second ? q1 : q0;
  const int lb0 = (int)blockIdx.x - (second ? ctas0 : 0);
  const int G = q.S, grp = lb0 / G, cta = lb0 - grp * G;
  SlotN* slots = reinterpret_cast<SlotN*>(q.slots) + (size_t)grp * 2 * G;
  T* vg0 = reinterpret_cast<T*>(q.w[0]) + (size_t)grp * q.ws_stride;
  T* vg1 = reinterpret_cast<T*>(q.w[1]) + (size_t)grp * q.ws_stride;
  T* qg = reinterpret_cast<T*>(q.w[2]) + (size_t)grp * q.ws_stride;
  const int b0 = q.cta_first[cta], nbk = q.cta_first[cta + 1] - b0;
  const int rows_cap = q.rows_cap;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int nact = min(nbk, NT / 32);               // warps that hold rows (set per job below)
  // layout (the same for every job of the launch): low table, block headers,
  // 12 row arrays, reduction staging
  size_t off_rows = sizeof(LowEntry) * q.nlow + 128 * (size_t)nbk;
  off_rows = (off_rows + 15) & ~size_t(15);
  size_t off_tmp = off_rows + 12 * sizeof(T) * (size_t)rows_cap;
  off_tmp = (off_tmp + 15) & ~size_t(15);
  double* stmp = reinterpret_cast<double*>(smem + off_tmp);
  LowEntry* low = reinterpret_cast<LowEntry*>(smem);
  uint32_t* hdrs = reinterpret_cast<uint32_t*>(smem + sizeof(LowEntry) * q.nlow);
  T* Q0 = reinterpret_cast<T*>(smem + off_rows);   // q_j in Q[j & 1]
  T* Q1 = Q0 + rows_cap;
  T* P0 = Q0 + 2 * rows_cap;                  // p_j in P[j & 1]
  T* P1 = Q0 + 3 * rows_cap;
  T* D0 = Q0 + 4 * rows_cap;                  // d_j in D[j & 1]
  T* D1 = Q0 + 5 * rows_cap;
  T* V0 = Q0 + 6 * rows_cap;                  // v_j (own rows) in V[j & 1]
  T* V1 = Q0 + 7 * rows_cap;
  T* X = Q0 + 8 * rows_cap;
  T* MV = Q0 + 9 * rows_cap;                  // M_ii
  T* MI = Q0 + 10 * rows_cap;                 // 1 / M_ii
  T* DG = Q0 + 11 * rows_cap;                 // a_ii - sigma
  unsigned gen = 0;
  auto reduce = [&](const T (&a)[PIPE_NV]) -> bool {
    cta_sumN<T, PIPE_NV>(a, nact, stmp, s_cta);
    ++gen;
    if (wid == 0) {
      double t[PIPE_NV];
      const bool okw = slot_reduceN_w0<PIPE_NV>(slots, G, cta, gen, s_cta, t, q.limit, q.err);
      if (lane == 0) {
#pragma unroll
        for (int j = 0; j < PIPE_NV; ++j) s_sum[j] = t[j];
        s_ok = okw;
      }
    }
    __syncthreads();
    return s_ok != 0;
  };
  // a reduction of one value held by thread 0 (the others contribute 0)
  auto reduce_one = [&](double v) -> bool {
    __syncthreads();
    if (threadIdx.x < PIPE_NV) s_cta[threadIdx.x] = threadIdx.x == 0 ? v : 0.0;
    __syncthreads();
    ++gen;
    if (wid == 0) {
      double t[PIPE_NV];
      const bool okw = slot_reduceN_w0<PIPE_NV>(slots, G, cta, gen, s_cta, t, q.limit, q.err);
      if (lane == 0) {
#pragma unroll
        for (int j = 0; j < PIPE_NV; ++j) s_sum[j] = t[j];
        s_ok = okw;
      }
    }
    __syncthreads();
    return s_ok != 0;
  };
  bool ok = true;
  for (int njob = 0;; ++njob) {
    // the next job: CTA 0 of the group takes it from the queue and a group
    // reduction hands the index to the other CTAs (all warps take part)
    int jid = 0;
    if (q.jobs) {
      if (!(ok = reduce_one(cta == 0 && threadIdx.x == 0 ? (double)atomicAdd(q.head, 1) : 0.0)))
        break;
      jid = (int)s_sum[0];
      if (jid >= __ldcg(q.head + 1)) break;
    } else if (njob > 0) {
      break;
    }
    if (threadIdx.x == 0) sj = q.jobs ? q.jobs[jid] : job0;
    __syncthreads();
    const Geo& g = sj.g;
    const T* __restrict__ bv = reinterpret_cast<const T*>(sj.b);
    T* xout = reinterpret_cast<T*>(sj.x);
    const double sigma = sj.sigma;
    {
      const uint4* src = reinterpret_cast<const uint4*>(g.low);
      uint4* dst = reinterpret_cast<uint4*>(low);
      for (int i = threadIdx.x; i < g.nlow * 2; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(g.blocks + b0);
      for (int i = threadIdx.x; i < nbk * 32; i += blockDim.x) hdrs[i] = __ldg(src + i);
    }
    const uint32_t Rbase = nbk > 0 ? __ldg(&g.blocks[b0].R) : 0u;
    __syncthreads();
    // Work of a pass, f(h, l0, j0, nj): chunks j0 .. j0 + nj - 1 (32 rows
    // each) of one block: whole blocks dealt round-robin to the warps, or, in
    // FP64 where that leaves the slowest warp with more chunks, single chunks
    // dealt round-robin in block order (as in smem_solve2). Each pass reads
    // v_k and writes v_{k+1} in different arrays, so chunks of one block may
    // run on different warps.
    constexpr int NW = NT / 32;
    auto block_chunks = [&](int lb) {
      return (g.cls_C[hdrs[lb * 32 + 3] & 0xFFu] + 31) >> 5;
    };
    bool by_chunk = false;
    nact = min(nbk, NW);
    if constexpr (sizeof(T) == 8) {
      int tot = 0, worst = 0;
      for (int w = 0; w < NW; ++w) {
        int mine = 0;
        for (int lb = w; lb < nbk; lb += NW) mine += block_chunks(lb);
        worst = max(worst, mine);
        tot += mine;
      }
      by_chunk = (tot + NW - 1) / NW < worst;
      if (by_chunk) nact = min(tot, NW);
    }
    auto each_part = [&](auto&& f) {
      if constexpr (sizeof(T) == 8) {
        if (by_chunk) {
          int t = 0;
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
    auto each_row = [&](const Hdr& h, int j0, int nj, auto&& g_row) {
      for (int j = j0; j < j0 + nj; ++j) {
        const int r = lane + 32 * j;
        if (r < h.C) g_row(r);
      }
    };
    // the product of a part's rows, then upd(r, x_r, ((H - sigma) x)_r) per row
    auto part_hv = [&](const T* xgl, const T* xloc, const Hdr& h, uint32_t l0, int j0, int nj,
                       auto&& upd) {
      if (sizeof(T) == 8 && by_chunk) {
        T xi[1], hx[1];
        block_hv_loc<T, 1>(xgl, xloc + l0, DG + l0, low, h, xi, hx, j0);
        const int r = lane + 32 * j0;
        if (r < h.C) upd(r, xi[0], hx[0]);
      } else {
        T xi[JM], hx[JM];
        block_hv_loc<T, JM>(xgl, xloc + l0, DG + l0, low, h, xi, hx);
#pragma unroll
        for (int j = 0; j < JM; ++j) {
          const int r = lane + 32 * j;
          if (j < h.J && r < h.C) upd(r, xi[j], hx[j]);
        }
      }
      (void)nj;
    };
    // q_1 = M^-1 b (x_0 = 0), q_0 = p_0 = 0, d_0 = d_{-1} = 0; q_1 is published
    // for the first product
    {
      T a[PIPE_NV] = {};
      each_part([&](const Hdr& h, uint32_t l0, int j0, int nj) {
        each_row(h, j0, nj, [&](int r) {
          T am;
          const T m = row_m<T, PC>(low[h.off + r], h, am);
          const uint32_t i = h.R + r;
          const uint32_t l = l0 + r;
          const T b = bv[i];
          a[1] += (m == T(0)) ? T(1) : T(0);
          const T mi = m == T(0) ? T(0) : T(1) / m;
          const T q = b * mi;
          MV[l] = m; MI[l] = mi; DG[l] = am;
          Q1[l] = q; qg[i] = q;
          Q0[l] = T(0); P0[l] = T(0); D0[l] = T(0); D1[l] = T(0); X[l] = T(0);
          a[0] += q * b;
        });
      });
      ok = reduce(a);
      if (ok && threadIdx.x == 0) {
        init_state(S, s_sum[0], s_sum[1], sj.tol, sj.kmax, sigma);
        s_ib = S.beta > 0.0 ? 1.0 / S.beta : 0.0;
        s_ibp = 1.0;                             // 1 / beta_0
      }
      __syncthreads();
    }
    // p_1 = (H - sigma) q_1, v_1 and the sums of step 1 (S3 = S5 = S6 = 0)
    if (ok && S.done == 0) {
      T a[PIPE_NV] = {};
      each_part([&](const Hdr& h, uint32_t l0, int j0, int nj) {
        part_hv(qg, Q1, h, l0, j0, nj, [&](int r, T xv, T hv) {
          const uint32_t l = l0 + r;
          const T p = hv;
          const T v = MI[l] * p;
          P1[l] = p; V1[l] = v; vg1[h.R + r] = v;
          a[0] += xv * p;
          a[1] += p * v;
          a[3] += MV[l] * xv * xv;
        });
      });
      ok = reduce(a);
      if (threadIdx.x == 0) s_sum[PIPE_NV] = 0.0;
      __syncthreads();
    }
    while (ok && S.done == 0) {
      // scalars of step k
      if (threadIdx.x == 0) {
        const double bk = S.beta, ib = s_ib;
        const double S1 = s_sum[0], S2 = s_sum[1], S3 = s_sum[2], S4 = s_sum[3], S5 = s_sum[4];
        const double S6 = s_sum[5];
        const double alpha = S1 * ib * ib;                         // alpha_k
        const double a = alpha * ib, c = bk * s_ibp;
        const double b2 = S2 * ib * ib + a * a * S4 + c * c * S6 - 2.0 * a * S1 * ib -
                          2.0 * c * S3 * ib + 2.0 * a * c * S5;   // beta_{k+1}^2
        // the terms' magnitude: b2 carries a rounding error of about
        // u mag, with u the unit roundoff of the vectors
        const double mag = S2 * ib * ib + a * a * S4 + c * c * S6 + fabs(2.0 * a * S1 * ib) +
                           fabs(2.0 * c * S3 * ib) + fabs(2.0 * a * c * S5);
        s_c[0] = ib; s_c[1] = a; s_c[2] = c;
        s_sum[5] = S4;
        S.alpha = alpha;
        if (!isfinite(alpha) || !isfinite(b2)) {
          S.status = HS_NONFINITE; S.done = 2; S.pending = 0;
        } else if (!(b2 > EXPANSION_FLOOR<T> * mag)) {
          S.status = HS_BREAKDOWN; S.pad = PIPE_EXPANSION; S.done = 2; S.pending = 0;
        } else {
          double ibn = ib;
          givens_fast(S, b2, ibn);
          s_ibp = ib;
          s_ib = ibn;
        }
      }
      __syncthreads();
      if (S.done == 2) break;
      const long long kk = S.k - 1;               // the step just rotated
      const bool doMV = S.done == 0;
      const bool repl = doMV && rperiod > 0 && (kk % rperiod) == 0;
      const bool odd = (kk & 1) != 0;
      const T* Qk = odd ? Q1 : Q0;                // q_k
      T* Qm = odd ? Q0 : Q1;                      // q_{k-1} -> q_{k+1}
      const T* Pk = odd ? P1 : P0;                // p_k
      T* Pm = odd ? P0 : P1;                      // p_{k-1} -> p_{k+1}
      const T* Dm = odd ? D0 : D1;                // d_{k-1}
      T* Dk = odd ? D1 : D0;                      // d_{k-2} -> d_k
      const T* vgk = odd ? vg1 : vg0;             // v_k
      T* vgn = odd ? vg0 : vg1;                   // v_{k+1}
      const T* Vk = odd ? V1 : V0;                // v_k (own rows)
      T* Vn = odd ? V0 : V1;                      // v_{k+1}
      const T cq = (T)S.cq, cd1 = (T)S.cd1, cd2 = (T)S.cd2, tau = (T)S.tau;
      const T c1 = (T)s_c[0], c2 = (T)s_c[1], c3 = (T)s_c[2];
      T a[PIPE_NV] = {};
      each_part([&](const Hdr& h, uint32_t l0, int j0, int nj) {
        // d_k = (q_k / beta_k - delta_k d_{k-1} - eps_k d_{k-2}) / gamma_k, x_k
        each_row(h, j0, nj, [&](int r) {
          const uint32_t l = l0 + r;
          const T d = cq * Qk[l] + cd1 * Dm[l] + cd2 * Dk[l];
          Dk[l] = d;
          X[l] += tau * d;
        });
        if (!doMV) return;
        if (repl) {
          each_row(h, j0, nj, [&](int r) {
            const uint32_t l = l0 + r;
            const T q = c1 * Vk[l] - c2 * Qk[l] - c3 * Qm[l];
            Qm[l] = q;
            qg[h.R + r] = q;
          });
          return;
        }
        part_hv(vgk, Vk, h, l0, j0, nj, [&](int r, T xv, T hv) {   // xv = v_k
          const uint32_t l = l0 + r;
          const T qo = Qk[l];
          const T q = c1 * xv - c2 * qo - c3 * Qm[l];
          const T p = c1 * hv - c2 * Pk[l] - c3 * Pm[l];
          const T v = MI[l] * p;
          Qm[l] = q; Pm[l] = p; Vn[l] = v; vgn[h.R + r] = v;
          const T mq = MV[l] * q;
          a[0] += q * p; a[1] += p * v; a[2] += p * qo; a[3] += mq * q; a[4] += mq * qo;
        });
      });
      if (!doMV) {                                // the last d/x update only
        __syncthreads();
        if (threadIdx.x == 0) { S.pending = 0; S.done = 2; }
        __syncthreads();
        break;
      }
      if (repl) {
        // publish q_{k+1}, then p_{k+1} = (H - sigma) q_{k+1}
        if (!(ok = reduce(a))) break;
        each_part([&](const Hdr& h, uint32_t l0, int j0, int nj) {
          part_hv(qg, Qm, h, l0, j0, nj, [&](int r, T xv, T hv) {   // xv = q_{k+1}
            const uint32_t l = l0 + r;
            const T qo = Qk[l];
            const T q = xv;
            const T p = hv;
            const T v = MI[l] * p;
            Pm[l] = p; Vn[l] = v; vgn[h.R + r] = v;
            const T mq = MV[l] * q;
            a[0] += q * p; a[1] += p * v; a[2] += p * qo; a[3] += mq * q; a[4] += mq * qo;
          });
        });
      }
      if (!(ok = reduce(a))) break;
    }
    __syncthreads();
    each_part([&](const Hdr& h, uint32_t l0, int j0, int nj) {
      each_row(h, j0, nj, [&](int r) { xout[h.R + r] = X[l0 + r]; });
    });
    if (cta == 0 && threadIdx.x == 0) {
      if (!ok) { S.status = HS_TIMEOUT; S.done = 2; }
      *sj.st = S;
    }
    if (!ok) break;
  }
}

}  // namespace

// Steps between replacements of p by a product: HS_MINRES_PIPE_R, else 20.
// Measured at L = 14..18 (FP64, tolerance 1e-12, row norm): without
// replacement the true residual ends 5-900x above the tolerance; R = 50 1.0-3.4x,
// R = 20 1.0-1.9x (the two-reduction form 0.9-1.3x), at the same iteration
// counts, wherever the two-reduction form reaches the tolerance; each
// replacement costs one extra barrier.
int pipe_replace_period() {
  if (const char* e = getenv("HS_MINRES_PIPE_R")) return std::max(0, atoi(e));
  return 20;
}

namespace {

// Launch for one or two queues; HS_CUDA without a message when it does not
// fit in shared memory or the cooperative launch is refused.
template <typename T, int PC, int JM, int NT>
hs_status launch1_t(int device, cudaStream_t s, const SmemJob& job0, const SmemQueue (&q)[2],
                    const int (&ng)[2], const int (&hc)[2], int rperiod) {
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  size_t sm = smr1_bytes<T>(q[0].nlow, hc[0], q[0].rows_cap, NT);
  if (ng[1] > 0) sm = std::max(sm, smr1_bytes<T>(q[1].nlow, hc[1], q[1].rows_cap, NT));
  if (sm + SMEM_STATIC_BYTES > (size_t)optin) return HS_CUDA;
  if (cudaFuncSetAttribute(k_minres_smem1<T, PC, JM, NT>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) {
    cudaGetLastError();
    return HS_CUDA;
  }
  SmemJob j = job0;
  SmemQueue q0 = q[0], q1 = ng[1] > 0 ? q[1] : q[0];
  int ctas0 = ng[0] * q[0].S;
  int rp = rperiod;
  void* args[] = {&j, &q0, &q1, &ctas0, &rp};
  const int grid = ctas0 + (ng[1] > 0 ? ng[1] * q[1].S : 0);
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_minres_smem1<T, PC, JM, NT>,
                                                    dim3(grid), dim3(NT), args, sm, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HS_CUDA;
  }
  count_launches(1);
  return HS_OK;
}

// blocks of at most 96 rows (k <= 8, every chain up to L = 20): 3 rows per
// lane; larger blocks 8 rows per lane and 256 threads (a few blocks per CTA
// at most, and no register spills in FP64)
template <typename T, int PC>
hs_status launch1_pc(int k, int device, cudaStream_t s, const SmemJob& job0,
                     const SmemQueue (&q)[2], const int (&ng)[2], const int (&hc)[2],
                     int rperiod) {
  if (k <= 8) return launch1_t<T, PC, 3, 512>(device, s, job0, q, ng, hc, rperiod);
  return launch1_t<T, PC, JMAX, 256>(device, s, job0, q, ng, hc, rperiod);
}

}  // namespace

hs_status launch_smem1(hs_dtype dt, int pc, int k, int device, cudaStream_t s,
                       const SmemJob& job0, const SmemQueue (&q)[2], const int (&ng)[2],
                       const int (&hc)[2], int rperiod) {
  if (dt == HS_F64)
    return pc == 0 ? launch1_pc<double, 0>(k, device, s, job0, q, ng, hc, rperiod)
         : pc == 1 ? launch1_pc<double, 1>(k, device, s, job0, q, ng, hc, rperiod)
                   : launch1_pc<double, 2>(k, device, s, job0, q, ng, hc, rperiod);
  return pc == 0 ? launch1_pc<float, 0>(k, device, s, job0, q, ng, hc, rperiod)
       : pc == 1 ? launch1_pc<float, 1>(k, device, s, job0, q, ng, hc, rperiod)
                 : launch1_pc<float, 2>(k, device, s, job0, q, ng, hc, rperiod);
}

}  // namespace hs
