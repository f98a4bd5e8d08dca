// Batched disorder sweep: many realisations (of up to two chain lengths) in
// one persistent cooperative launch. CTA groups take realisations from one
// queue per chain length and run all of Algorithm 1 on each: every inner
// solve (Algorithm 2, the two-reduction shared-memory form), the three-term
// recurrence, full reorthogonalisation and the convergence test on T_k, with
// group-local reductions; the host sets the start vectors before and extracts
// and certifies the Ritz pairs after. The group size per (L, preconditioner,
// SM count) comes from a short timing run, cached in a JSON file. The twist
// overlaps (Sec. III) of every realisation's pairs give |z|^2 averaged over
// the pairs of each realisation, then its mean and standard deviation over the
// realisations of each length (Sec. IV B-C).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <sys/stat.h>

#include "lanczos.cuh"
#include "minres_smem.cuh"

namespace hs {

namespace {

// A measured schedule: S CTAs per group, the form (one = the one-reduction
// kernel) and the iterations per second of one group.
struct Tune {
  int S = 0;
  int one = 0;
  double rate = 0.0;
};

// The cache: HS_SWEEP_TUNE, else $HOME/.cache/hs_sweep_tune.json; one entry
// per line, {"key": {"S": s, "one": o, "rate": r}, ...}.
std::string tune_path() {
  if (const char* e = getenv("HS_SWEEP_TUNE")) return e;
  const char* home = getenv("HOME");
  return std::string(home ? home : ".") + "/.cache/hs_sweep_tune.json";
}

std::map<std::string, Tune> tune_read() {
  std::map<std::string, Tune> m;
  FILE* f = fopen(tune_path().c_str(), "r");
  if (!f) return m;
  char line[512], key[128];
  while (fgets(line, sizeof line, f)) {
    Tune t;
    if (sscanf(line, " \"%127[^\"]\": {\"S\": %d, \"one\": %d, \"rate\": %lf}", key, &t.S, &t.one,
               &t.rate) == 4 &&
        t.S > 0)
      m[key] = t;
  }
  fclose(f);
  return m;
}

void tune_write(const std::map<std::string, Tune>& m) {
  const std::string p = tune_path();
  const size_t slash = p.find_last_of('/');
  if (slash != std::string::npos) mkdir(p.substr(0, slash).c_str(), 0755);   // may exist
  FILE* f = fopen(p.c_str(), "w");
  if (!f) return;                     // an unwritable cache only costs a re-tune
  fprintf(f, "{\n");
  size_t i = 0;
  for (const auto& kv : m) {
    fprintf(f, "\"%s\": {\"S\": %d, \"one\": %d, \"rate\": %.6g}%s\n", kv.first.c_str(),
            kv.second.S, kv.second.one, kv.second.rate, ++i < m.size() ? "," : "");
  }
  fprintf(f, "}\n");
  fclose(f);
}

// One chain length of the sweep: its realisations, plan and queue.
struct Class {
  int L = 0;
  std::vector<int> idx;              // realisations (input order)
  hs_handle* hd0 = nullptr;          // representative handle: owns the block plan
  Tune tune;
  int tuned = 0;                     // 1 = timed in this call, 0 = from the cache, -1 = forced
  int ngroups = 0;
  int* first = nullptr;
  int rows_cap = 0, hdr_cap = 0;
  int cap = 0;                       // job capacity
  SlotN* slots = nullptr;
  double* ws = nullptr;
  SmemJob* jobs = nullptr;
  MinresState* states = nullptr;
  int* head = nullptr;               // [0] next job, [1] number of jobs
  SmemJob* h_jobs = nullptr;         // pinned mirrors
  MinresState* h_states = nullptr;
  int* h_head = nullptr;
  long long n = 0;
  // block plans by group size, owned here
  struct Plan { int* first = nullptr; int rows_cap = 0, hdr_cap = 0; };
  std::map<int, Plan> plans;
  int S_round = 0;                   // group size of the next launch
};

void free_class(Class& c) {
  for (auto& kv : c.plans) cudaFree(kv.second.first);
  cudaFree(c.slots); cudaFree(c.ws); cudaFree(c.jobs); cudaFree(c.states); cudaFree(c.head);
  cudaFreeHost(c.h_jobs); cudaFreeHost(c.h_states); cudaFreeHost(c.h_head);
  c = Class();
}

hs_status alloc_class(Class& c, int num_sms) {
  c.cap = std::max((int)c.idx.size(), num_sms);
  const size_t nslot = 2 * (size_t)num_sms;
  if (cudaMalloc(&c.slots, nslot * sizeof(SlotN)) != cudaSuccess ||
      cudaMalloc(&c.ws, 3 * (size_t)c.n * num_sms * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c.jobs, c.cap * sizeof(SmemJob)) != cudaSuccess ||
      cudaMalloc(&c.states, c.cap * sizeof(MinresState)) != cudaSuccess ||
      cudaMalloc(&c.head, 2 * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&c.h_jobs, c.cap * sizeof(SmemJob)) != cudaSuccess ||
      cudaMallocHost(&c.h_states, c.cap * sizeof(MinresState)) != cudaSuccess ||
      cudaMallocHost(&c.h_head, 2 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return HS_OOM;
  }
  return HS_OK;
}

// The queue of a class for a launch with S CTAs per group (the plan must be
// the current one of c.hd0).
SmemQueue make_queue(const Class& c, int S, int* err, unsigned long long limit) {
  SmemQueue q{};
  q.jobs = c.jobs;
  q.head = c.head;
  q.S = S;
  q.nlow = (int)c.hd0->low.size();
  q.slots = c.slots;
  q.err = err;
  q.limit = limit;
  q.cta_first = c.first;
  q.rows_cap = c.rows_cap;
  q.w[0] = c.ws;
  q.w[1] = c.ws + c.n;
  q.w[2] = c.ws + 2 * c.n;
  q.ws_stride = 3 * c.n;
  return q;
}

// The class's plan for groups of S CTAs (made once per S, copied out of the
// handle's one-plan cache), made current in c.first / rows_cap / hdr_cap.
hs_status use_plan(Class& c, int S, cudaStream_t s) {
  auto it = c.plans.find(S);
  if (it == c.plans.end()) {
    int* f = nullptr;
    int rc = 0, hc = 0;
    hs_status st = smr_plan(c.hd0, S, &f, &rc, &hc);
    if (st != HS_OK) return st;
    Class::Plan p;
    if (cudaMalloc(&p.first, sizeof(int) * (S + 1)) != cudaSuccess ||
        cudaMemcpyAsync(p.first, f, sizeof(int) * (S + 1), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess) {
      cudaGetLastError();
      cudaFree(p.first);
      return HS_OOM;
    }
    p.rows_cap = rc;
    p.hdr_cap = hc;
    it = c.plans.emplace(S, p).first;
  }
  c.first = it->second.first;
  c.rows_cap = it->second.rows_cap;
  c.hdr_cap = it->second.hdr_cap;
  return HS_OK;
}

SmemJob job_for(hs_handle* hd, const double* b, double* x, MinresState* st, double tol,
                long long kmax) {
  return SmemJob{hd->geo(), b, x, st, hd->sigma, tol, kmax};
}

// Launch of up to two queues (ng[i] groups of S[i] CTAs; ng[1] = 0: one).
hs_status launch_pair(const Class* c0, const Class* c1, int pc, bool one, int k, int device,
                      cudaStream_t s, int* err, unsigned long long limit) {
  const SmemQueue q0 = make_queue(*c0, c0->S_round, err, limit);
  const SmemQueue qs[2] = {q0, c1 ? make_queue(*c1, c1->S_round, err, limit) : q0};
  const int ng[2] = {c0->ngroups, c1 ? c1->ngroups : 0};
  const int hc[2] = {c0->hdr_cap, c1 ? c1->hdr_cap : 0};
  const SmemJob none{};
  return one ? launch_smem1(HS_F64, pc, k, device, s, none, qs, ng, hc, pipe_replace_period())
             : launch_smem2(HS_F64, pc, k, device, s, none, qs, ng, hc);
}

// Iterations per second of one group: one launch of `groups` groups of S CTAs,
// each running `iters` iterations (tolerance 0) of a job on the start vector
// of one of the class's realisations. 0 when the form does not fit.
double time_groups(Class& c, const std::vector<LzRun>& runs, int pc, int S, bool one, int groups,
                   int iters, int device, cudaStream_t s, int* err, hs_status* st) {
  *st = HS_OK;
  if (smr_plan(c.hd0, S, &c.first, &c.rows_cap, &c.hdr_cap) != HS_OK) return 0.0;
  for (int g = 0; g < groups; ++g) {
    const LzRun& r = runs[c.idx[g % c.idx.size()]];
    c.h_jobs[g] = job_for(r.hd, r.rhs(), r.x, c.states + g, 0.0, iters);
  }
  c.h_head[0] = 0;
  c.h_head[1] = groups;
  const int keep_S = c.S_round;
  const int keep_ng = c.ngroups;
  c.S_round = S;
  c.ngroups = groups;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double rate = 0.0;
  if (cudaMemcpyAsync(c.jobs, c.h_jobs, groups * sizeof(SmemJob), cudaMemcpyHostToDevice, s) ==
          cudaSuccess &&
      cudaMemcpyAsync(c.head, c.h_head, 2 * sizeof(int), cudaMemcpyHostToDevice, s) ==
          cudaSuccess &&
      cudaMemsetAsync(c.slots, 0, 2 * (size_t)S * groups * sizeof(SlotN), s) == cudaSuccess &&
      cudaMemsetAsync(err, 0, sizeof(int), s) == cudaSuccess) {
    cudaEventRecord(e0, s);
    const hs_status ls = launch_pair(&c, nullptr, pc, one, c.hd0->k, device, s, err, 1ull << 22);
    cudaEventRecord(e1, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      *st = HS_CUDA;
    } else if (ls == HS_OK) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms > 0) rate = iters / (ms * 1e-3);
    }
  } else {
    cudaGetLastError();
    *st = HS_CUDA;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c.S_round = keep_S;
  c.ngroups = keep_ng;
  return rate;
}

// The best (S, form) of a class on the whole GPU: group sizes from the
// smallest that fits up to four times it, both forms, by throughput
// (groups x iterations per second of a group).
hs_status tune_class(Class& c, const std::vector<LzRun>& runs, int pc, int num_sms, int device,
                     cudaStream_t s, int* err, int only_form) {
  const int iters = 200;
  Tune best;
  double best_tp = 0.0;
  for (int one = 0; one < 2; ++one) {
    if (only_form >= 0 && one != only_form) continue;
    int smin = 0;
    for (int S = 1; S <= num_sms && !smin; ++S) {
      hs_status st;
      const double r = time_groups(c, runs, pc, S, one, 1, 8, device, s, err, &st);
      if (st != HS_OK) return st;
      if (r > 0) smin = S;
    }
    if (!smin) continue;
    std::vector<int> cand = {smin, smin + 1, (3 * smin + 1) / 2, 2 * smin, 3 * smin, 4 * smin};
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    for (int S : cand) {
      if (S > num_sms) break;
      const int groups = num_sms / S;
      hs_status st;
      const double r = time_groups(c, runs, pc, S, one, groups, iters, device, s, err, &st);
      if (st != HS_OK) return st;
      if (r * groups > best_tp) {
        best_tp = r * groups;
        best.S = S;
        best.one = one;
        best.rate = r;
      }
    }
  }
  if (!best.S) return HS_CUDA;
  c.tune = best;
  c.tuned = 1;
  return HS_OK;
}

// ---------------------------------------------------------------------------
// Device-resident form: a group takes a realisation from its queue and runs
// all of Algorithm 1 on it (every inner solve by smem_solve2, the rest of each
// step with group reductions, the convergence test on T_k), then takes the
// next. The host only sets v_1 before and extracts the Ritz pairs after.

constexpr int SWEEP_MMAX = 256;   // Lanczos steps per realisation
constexpr int VRED = SWEEP_MMAX + 8;
// the step's scratch behind the solve's shared memory: CTA partials and
// Gram-Schmidt coefficients (VRED each), the QL arrays (SWEEP_MMAX each)
constexpr size_t SWEEP_SCRATCH = sizeof(double) * (2 * VRED + 3 * SWEEP_MMAX);

// One realisation: its geometry and shift, basis V ((m + 1) n, v_1 set), the
// solve's output x and scratch w (n each), and where its results go.
struct SweepReal {
  Geo g;
  double sigma;
  double* V;
  double* x;
  double* w;
  double* alpha;          // m: alpha_1.. (device)
  double* beta;           // m: beta_2.. (beta[j] couples steps j and j + 1)
  MinresState* st;        // state of the last inner solve
  int* res;               // [0] steps, [1] converged pairs, [2] status, [3] unconverged solves
  long long* iters;       // MINRES iterations of all its solves
};

// The device form's arguments of one queue: its realisations, queue head
// ([0] next, [1] count), K, m, tolerances; per group: 2 S x VRED doubles and
// 2 S generation words for the group's vector reductions.
struct SweepArgs {
  const SweepReal* reals;
  int* head;
  int K, m;
  double tol, minres_tol;
  double* vbuf;
  unsigned* vgen;
};

// Sum over the group of nv <= VRED per-CTA values part[] (shared memory) into
// out[] (shared memory), the same fixed order in every CTA; false when the
// wait gave up.
__device__ __forceinline__ bool grp_reduce_vec(const Grp2<double>& c, double* vbuf, unsigned* vgen,
                                               unsigned& vg, const double* part, int nv,
                                               double* out, int* s_ok) {
  ++vg;
  const unsigned par = vg & 1u;
  double* mine = vbuf + ((size_t)par * c.G + c.cta) * VRED;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) mine[j] = part[j];
  __syncthreads();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) st_release_u32(vgen + (size_t)par * c.G + c.cta, vg);
  if (wid == 0) {
    int ok = 1;
    unsigned long long it = 0;
    while (true) {
      bool all = true;
      for (int cc = lane; cc < c.G; cc += 32) all = all && ld_relaxed_u32(vgen + (size_t)par * c.G + cc) == vg;
      if (__all_sync(0xffffffffu, all)) break;
      if (++it > c.q->limit) { ok = 0; if (lane == 0) atomicExch(c.q->err, 1); break; }
      if ((it & 255ull) == 0 && ld_relaxed_i32(c.q->err)) { ok = 0; break; }
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) *s_ok = ok;
  }
  __syncthreads();
  if (!*s_ok) return false;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) {
    double t = 0.0;
    for (int cc = 0; cc < c.G; ++cc) t += __ldcg(vbuf + ((size_t)par * c.G + cc) * VRED + j);
    out[j] = t;
  }
  __syncthreads();
  return true;
}

// Convergence test of step kk = k + 1 on one thread: eigenvalues theta and the
// last components zl of the eigenvectors of T_kk by the implicit QL of
// tridiag_eig (only the last row of the rotations is kept); the number of the
// K largest |theta| with beta_{k+1} |zl| <= tol |theta|. -1 if QL did not
// converge.
__device__ int ritz_converged(int kk, const double* alpha, const double* beta, double bn, int K,
                              double tol, double* d, double* e, double* zl) {
  for (int i = 0; i < kk; ++i) {
    d[i] = alpha[i];
    e[i] = i + 1 < kk ? beta[i] : 0.0;
    zl[i] = i == kk - 1 ? 1.0 : 0.0;
  }
  const double eps = 2.220446049250313e-16;
  double anorm = 0.0;
  for (int i = 0; i < kk; ++i) anorm = fmax(anorm, fabs(d[i]) + fabs(e[i]));
  for (int l = 0; l < kk; ++l) {
    int iter = 0;
    while (true) {
      int m = l;
      for (; m + 1 < kk; ++m) {
        const double scale = fabs(d[m]) + fabs(d[m + 1]);
        if (fabs(e[m]) <= eps * scale || fabs(e[m]) <= eps * anorm) break;
      }
      if (m == l) break;
      if (++iter > 60) return -1;
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
      double s = 1.0, cc = 1.0, p = 0.0;
      bool underflow = false;
      for (int i = m - 1; i >= l; --i) {
        const double f = s * e[i];
        const double b = cc * e[i];
        r = hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= p;
          e[m] = 0.0;
          underflow = true;
          break;
        }
        s = f / r;
        cc = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * cc * b;
        p = s * r;
        d[i + 1] = g + p;
        g = cc * r - b;
        const double t = zl[i + 1];
        zl[i + 1] = s * zl[i] + cc * t;
        zl[i] = cc * zl[i] - s * t;
      }
      if (underflow) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  // the K largest |theta| (selection; e[] marks the chosen)
  int nconv = 0;
  for (int i = 0; i < kk; ++i) e[i] = 0.0;
  for (int q = 0; q < K && q < kk; ++q) {
    int best = -1;
    for (int i = 0; i < kk; ++i)
      if (e[i] == 0.0 && (best < 0 || fabs(d[i]) > fabs(d[best]))) best = i;
    e[best] = 1.0;
    if (bn * fabs(zl[best]) <= tol * fabs(d[best])) ++nconv;
  }
  return nconv;
}

template <int PC, int JM, int NT>
__global__ void __launch_bounds__(NT, 1) k_sweep(SweepArgs a0, SmemQueue q0, SweepArgs a1,
                                                 SmemQueue q1, int ctas0) {
  extern __shared__ __align__(16) char smem[];
  __shared__ MinresState S;
  __shared__ SmemJob sj;
  __shared__ double sbuf[4];
  __shared__ double s_ib, s_ibp;
  __shared__ int s_ok;
  __shared__ SweepReal sr;
  __shared__ double s_alpha[SWEEP_MMAX], s_beta[SWEEP_MMAX];
  __shared__ double s_part[NT / 32][8];
  __shared__ int s_flag[2];
  const bool second = (int)blockIdx.x >= ctas0;
  const SmemQueue& q = second ? q1 : q0;
  const SweepArgs& A = second ? a1 : a0;
  const int lb = (int)blockIdx.x - (second ? ctas0 : 0);
  Grp2<double> c = grp2_setup<double>(q, lb, smem, &S, &sj, sbuf, &s_ib, &s_ibp, &s_ok);
  const int grp = lb / c.G;
  double* vbuf = A.vbuf + (size_t)grp * 2 * c.G * VRED;
  unsigned* vgen = A.vgen + (size_t)grp * 2 * c.G;
  unsigned vg = 0;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // scratch after the solve's layout (its reduction scratch ends there)
  double* part = c.stmp + 2 * NT;
  double* hcoef = part + VRED;
  double* qd = hcoef + VRED;
  double* qe = qd + SWEEP_MMAX;
  double* qz = qe + SWEEP_MMAX;
  while (true) {
    double tot[2];
    const double v = (c.cta == 0 && threadIdx.x == 0) ? (double)atomicAdd(A.head, 1) : 0.0;
    if (!grp_reduce2(c, v, 0.0, tot)) return;
    const int rid = (int)tot[0];
    if (rid >= __ldcg(A.head + 1)) return;
    if (threadIdx.x == 0) sr = A.reals[rid];
    __syncthreads();
    const long long n = sr.g.n;
    // this CTA's rows
    long long lo = 0, hi = 0;
    if (c.nbk > 0) {
      lo = __ldg(&sr.g.blocks[c.b0].R);
      const BlockInfo* lastb = sr.g.blocks + c.b0 + c.nbk - 1;
      hi = (long long)__ldg(&lastb->R) + sr.g.cls_C[lastb->w];
    }
    int k = 0, unconv = 0, status = HS_OK;
    long long iters = 0;
    double bk = 0.0;
    bool done = false;
    while (!done) {
      const double* vk = sr.V + (size_t)k * n;
      // (H - sigma) x = v_k
      if (threadIdx.x == 0) sj = SmemJob{sr.g, vk, sr.x, sr.st, sr.sigma, A.minres_tol, 50 * n};
      __syncthreads();
      if (!smem_solve2<double, PC, JM, NT>(c)) return;
      const int s_status = S.status;
      if (s_status != HS_OK) { status = s_status; break; }
      iters += S.k - 1;
      if (S.beta1 > 0 && !(fabs(S.phi) < S.tol_abs) && S.beta != 0.0) ++unconv;
      __syncthreads();
      // w = x - beta_k v_{k-1}; alpha_k = v_k . w; w -= alpha_k v_k
      const double* vkm = k > 0 ? sr.V + (size_t)(k - 1) * n : nullptr;
      double pa = 0.0;
      for (long long i = lo + threadIdx.x; i < hi; i += NT) {
        const double wi = sr.x[i] - (k > 0 ? bk * vkm[i] : 0.0);
        sr.w[i] = wi;
        pa += vk[i] * wi;
      }
      if (!grp_reduce2(c, pa, 0.0, tot)) return;
      const double al = tot[0];
      for (long long i = lo + threadIdx.x; i < hi; i += NT) sr.w[i] -= al * vk[i];
      // full reorthogonalisation against v_1..v_k: two classical Gram-Schmidt passes
      for (int pass = 0; pass < 2; ++pass) {
        for (int j0 = 0; j0 <= k; j0 += 8) {
          double acc[8];
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) acc[jj] = 0.0;
          for (long long i = lo + threadIdx.x; i < hi; i += NT) {
            const double wi = sr.w[i];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj)
              if (j0 + jj <= k) acc[jj] += sr.V[(size_t)(j0 + jj) * n + i] * wi;
          }
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            double t = acc[jj];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) s_part[wid][jj] = t;
          }
          __syncthreads();
          if (threadIdx.x < 8 && j0 + (int)threadIdx.x <= k) {
            double t = 0.0;
            for (int w = 0; w < NT / 32; ++w) t += s_part[w][threadIdx.x];
            part[j0 + threadIdx.x] = t;
          }
          __syncthreads();
        }
        if (!grp_reduce_vec(c, vbuf, vgen, vg, part, k + 1, hcoef, &s_ok)) return;
        for (long long i = lo + threadIdx.x; i < hi; i += NT) {
          double wi = sr.w[i];
          for (int j = 0; j <= k; ++j) wi -= hcoef[j] * sr.V[(size_t)j * n + i];
          sr.w[i] = wi;
        }
      }
      double pb = 0.0;
      for (long long i = lo + threadIdx.x; i < hi; i += NT) pb += sr.w[i] * sr.w[i];
      if (!grp_reduce2(c, pb, 0.0, tot)) return;
      const double bn = sqrt(fmax(tot[0], 0.0));
      // the convergence test (every CTA's thread 0 on the same numbers)
      if (threadIdx.x == 0) {
        s_alpha[k] = al;
        const int kk = k + 1;
        int nconv = 0;
        if (kk >= A.K) nconv = ritz_converged(kk, s_alpha, s_beta, bn, A.K, A.tol, qd, qe, qz);
        const bool stop = nconv == A.K || bn <= 1e-13 * fabs(al) || kk == A.m;
        s_flag[0] = stop ? 1 : 0;
        s_flag[1] = nconv;
        if (!stop) s_beta[k] = bn;
      }
      __syncthreads();
      done = s_flag[0] != 0;
      if (!done) {
        double* vn = sr.V + (size_t)(k + 1) * n;
        const double ib = 1.0 / bn;
        for (long long i = lo + threadIdx.x; i < hi; i += NT) vn[i] = sr.w[i] * ib;
        bk = bn;
        ++k;
      }
      __syncthreads();
    }
    if (c.cta == 0 && threadIdx.x == 0) {
      const int steps = status == HS_OK ? k + 1 : k;
      for (int j = 0; j < steps; ++j) sr.alpha[j] = s_alpha[j];
      for (int j = 0; j + 1 < steps; ++j) sr.beta[j] = s_beta[j];
      sr.res[0] = steps;
      sr.res[1] = status == HS_OK ? s_flag[1] : 0;
      sr.res[2] = status;
      sr.res[3] = unconv;
      *sr.iters = iters;
    }
    __syncthreads();
  }
}

// Launch of the device form for one or two queues (two-reduction solves,
// FP64); HS_CUDA when it does not fit or the cooperative launch is refused.
template <int PC, int JM, int NT>
hs_status launch_sweep_t(int device, cudaStream_t s, const SweepArgs (&a)[2],
                         const SmemQueue (&q)[2], const int (&ng)[2], const int (&hc)[2]) {
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, k_sweep<PC, JM, NT>) != cudaSuccess) {
    cudaGetLastError();
    return HS_CUDA;
  }
  size_t sm = smr_bytes<double>(q[0].nlow, hc[0], q[0].rows_cap, NT);
  if (ng[1] > 0) sm = std::max(sm, smr_bytes<double>(q[1].nlow, hc[1], q[1].rows_cap, NT));
  sm += SWEEP_SCRATCH;
  if (sm + fa.sharedSizeBytes > (size_t)optin) return HS_CUDA;
  if (cudaFuncSetAttribute(k_sweep<PC, JM, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm) != cudaSuccess) {
    cudaGetLastError();
    return HS_CUDA;
  }
  SweepArgs a0 = a[0], a1 = ng[1] > 0 ? a[1] : a[0];
  SmemQueue q0 = q[0], q1 = ng[1] > 0 ? q[1] : q[0];
  int ctas0 = ng[0] * q[0].S;
  void* args[] = {&a0, &q0, &a1, &q1, &ctas0};
  const int grid = ctas0 + (ng[1] > 0 ? ng[1] * q[1].S : 0);
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_sweep<PC, JM, NT>, dim3(grid),
                                                    dim3(NT), args, sm, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HS_CUDA;
  }
  count_launches(1);
  return HS_OK;
}

hs_status launch_sweep(int pc, int k, int device, cudaStream_t s, const SweepArgs (&a)[2],
                       const SmemQueue (&q)[2], const int (&ng)[2], const int (&hc)[2]) {
  if (k <= 8)
    return pc == 0 ? launch_sweep_t<0, 3, 512>(device, s, a, q, ng, hc)
         : pc == 1 ? launch_sweep_t<1, 3, 512>(device, s, a, q, ng, hc)
                   : launch_sweep_t<2, 3, 512>(device, s, a, q, ng, hc);
  return pc == 0 ? launch_sweep_t<0, JMAX, 512>(device, s, a, q, ng, hc)
       : pc == 1 ? launch_sweep_t<1, JMAX, 512>(device, s, a, q, ng, hc)
                 : launch_sweep_t<2, JMAX, 512>(device, s, a, q, ng, hc);
}

// Groups per class: as many as fit for one class; for two, the split of the
// SMs that minimises the longer of the two classes' round times, with work
// proportional to realisations x n and speed to groups x the group rate.
void split_groups(Class* cls, int ncls, int num_sms) {
  if (ncls == 1) {
    // fewer realisations than groups: one group each, as large as the SMs
    // allow (unless the size is forced)
    const int nr = (int)cls[0].idx.size();
    if (cls[0].tuned != -1 && (long long)nr * cls[0].tune.S < num_sms)
      cls[0].tune.S = std::min(256, std::max(cls[0].tune.S, num_sms / nr));
    cls[0].ngroups = std::max(1, num_sms / cls[0].tune.S);
    return;
  }
  double best = 1e300;
  int b0 = 1;
  const double w0 = (double)cls[0].idx.size() * cls[0].n, w1 = (double)cls[1].idx.size() * cls[1].n;
  for (int g0 = 1; g0 * cls[0].tune.S + cls[1].tune.S <= num_sms; ++g0) {
    const int g1 = (num_sms - g0 * cls[0].tune.S) / cls[1].tune.S;
    const double t = std::max(w0 / (g0 * cls[0].tune.rate), w1 / (g1 * cls[1].tune.rate));
    if (t < best) { best = t; b0 = g0; }
  }
  cls[0].ngroups = b0;
  cls[1].ngroups = std::max(1, (num_sms - b0 * cls[0].tune.S) / cls[1].tune.S);
}

}  // namespace

}  // namespace hs

using namespace hs;

extern "C" hs_status hs_sweep(int B, const int* L_host, const double* h_host, int K, int m_max,
                              double tol, unsigned long long seed, double minres_tol,
                              hs_precond pc, double* evals_host, double* resid_host,
                              double* z_host, double* zz_host, hs_sweep_info* info) {
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  if (B < 1 || !L_host || !h_host || K < 1 || !evals_host) return HS_BAD_ARG;
  if (pc != HS_PC_ID && pc != HS_PC_JACOBI && pc != HS_PC_ROWNORM) return HS_BAD_ARG;
  if (!(minres_tol > 0)) minres_tol = 1e-12;
  if (!(tol > 0)) tol = 1e-10;
  if (info) std::memset(info, 0, sizeof(*info));
  // chain lengths: at most two values
  Class cls[2];
  int ncls = 0;
  for (int r = 0; r < B; ++r) {
    const int L = L_host[r];
    if (L < 4 || L > LMAX || (L & 1)) return HS_BAD_ARG;
    int c = 0;
    while (c < ncls && cls[c].L != L) ++c;
    if (c == ncls) {
      if (ncls == 2) return HS_BAD_ARG;
      cls[ncls++].L = L;
    }
    cls[c].idx.push_back(r);
  }
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return HS_CUDA;
  }
  std::vector<hs_handle*> hd(B, nullptr);
  std::vector<LzRun> runs(B);
  int* err = nullptr;
  double* evbuf = nullptr;
  // device form: per class its realisations, alpha/beta, results, iterations
  // and the groups' vector-reduction buffers
  struct Dev {
    SweepReal* reals = nullptr;
    double* ab = nullptr;
    int* res = nullptr;
    long long* iters = nullptr;
    double* vbuf = nullptr;
    unsigned* vgen = nullptr;
  } dv[2];
  hs_status st = HS_OK;
  int device = 0, num_sms = 0;
  cudaGetDevice(&device);
  cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device);
  auto cleanup = [&](hs_status out) {
    cudaStreamSynchronize(s);
    for (int c = 0; c < ncls; ++c) {
      free_class(cls[c]);
      cudaFree(dv[c].reals); cudaFree(dv[c].ab); cudaFree(dv[c].res); cudaFree(dv[c].iters);
      cudaFree(dv[c].vbuf); cudaFree(dv[c].vgen);
    }
    cudaFree(err);
    cudaFree(evbuf);
    for (hs_handle* h : hd)
      if (h) hs_free(h);
    cudaStreamDestroy(s);
    cudaGetLastError();
    return out;
  };
  // handles (sigma = midpoint of the spectrum) and start vectors
  {
    size_t off = 0;
    for (int r = 0; r < B; ++r) {
      st = hs_create(L_host[r], h_host + off, NAN, s, &hd[r]);
      off += L_host[r];
      if (st != HS_OK) return cleanup(st);
      if ((st = lz_start(runs[r], hd[r], K, m_max, tol, seed + (unsigned long long)r, nullptr)) !=
          HS_OK)
        return cleanup(st);
      if (runs[r].m > SWEEP_MMAX) return cleanup(fail(hd[r], HS_BAD_ARG, "hs_sweep: m_max > 256"));
    }
  }
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return cleanup(HS_OOM);
  // group size per class: forced (HS_SWEEP_S), cached or timed
  auto tunes = tune_read();
  bool tunes_changed = false;
  for (int c = 0; c < ncls; ++c) {
    Class& C = cls[c];
    C.hd0 = hd[C.idx[0]];
    C.n = C.hd0->n;
    if ((st = alloc_class(C, num_sms)) != HS_OK) return cleanup(st);
    char key[96];
    snprintf(key, sizeof key, "L%d_pc%d_f64_sm%d", C.L, (int)pc, num_sms);
    if (const char* fs = getenv("HS_SWEEP_S")) {
      C.tune.S = std::max(1, std::min(num_sms, atoi(fs)));
      C.tune.rate = 1.0;
      C.tuned = -1;
    } else if (tunes.count(key)) {
      C.tune = tunes[key];
      C.tuned = 0;
    } else {
      if ((st = tune_class(C, runs, pc, num_sms, device, s, err, 0)) != HS_OK) return cleanup(st);
      tunes[key] = C.tune;
      tunes_changed = true;
    }
    C.tune.one = 0;
  }
  if (tunes_changed) tune_write(tunes);
  // one kernel shape per launch: the rows-per-lane template follows k <= 8
  const int k_lo = cls[0].hd0->k;
  for (int c = 1; c < ncls; ++c)
    if ((cls[c].hd0->k <= 8) != (k_lo <= 8)) return cleanup(HS_BAD_ARG);
  // realisation records
  for (int c = 0; c < ncls; ++c) {
    Class& C = cls[c];
    Dev& D = dv[c];
    const int nr = (int)C.idx.size();
    if (cudaMalloc(&D.reals, sizeof(SweepReal) * nr) != cudaSuccess ||
        cudaMalloc(&D.ab, sizeof(double) * 2 * SWEEP_MMAX * nr) != cudaSuccess ||
        cudaMalloc(&D.res, sizeof(int) * 4 * nr) != cudaSuccess ||
        cudaMalloc(&D.iters, sizeof(long long) * nr) != cudaSuccess ||
        cudaMalloc(&D.vbuf, sizeof(double) * 2 * (size_t)num_sms * VRED) != cudaSuccess ||
        cudaMalloc(&D.vgen, sizeof(unsigned) * 2 * (size_t)num_sms) != cudaSuccess) {
      cudaGetLastError();
      return cleanup(HS_OOM);
    }
    std::vector<SweepReal> hr(nr);
    for (int j = 0; j < nr; ++j) {
      const int r = C.idx[j];
      SweepReal& R = hr[j];
      R.g = hd[r]->geo();
      R.sigma = hd[r]->sigma;
      R.V = runs[r].V;
      R.x = runs[r].x;
      R.w = runs[r].w;
      R.alpha = D.ab + (size_t)2 * SWEEP_MMAX * j;
      R.beta = R.alpha + SWEEP_MMAX;
      R.st = C.states + j;
      R.res = D.res + 4 * j;
      R.iters = D.iters + j;
    }
    C.h_head[0] = 0;
    C.h_head[1] = nr;
    if (cudaMemcpyAsync(D.reals, hr.data(), sizeof(SweepReal) * nr, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(C.head, C.h_head, 2 * sizeof(int), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemsetAsync(D.res, 0, sizeof(int) * 4 * nr, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return cleanup(HS_CUDA);
    }
  }
  const double t_setup = std::chrono::duration<double>(clk::now() - t0).count();
  // the launch: groups per class from the split of the SMs; a group size that
  // does not fit the kernel's shared memory grows by one CTA until it fits
  const auto ts = clk::now();
  const unsigned long long limit = 1ull << 22;
  hs_status ls = HS_CUDA;
  for (int attempt = 0; attempt < 64 && ls == HS_CUDA; ++attempt) {
    split_groups(cls, ncls, num_sms);
    int used = 0;
    for (int c = 0; c < ncls; ++c) {
      cls[c].S_round = cls[c].tune.S;
      used += cls[c].ngroups * cls[c].tune.S;
      if ((st = use_plan(cls[c], cls[c].tune.S, s)) != HS_OK) return cleanup(st);
    }
    if (used > num_sms) break;
    SweepArgs a[2];
    SmemQueue q[2];
    int ng[2] = {0, 0}, hc[2] = {0, 0};
    for (int c = 0; c < ncls; ++c) {
      Class& C = cls[c];
      a[c] = SweepArgs{dv[c].reals, C.head, K, runs[C.idx[0]].m, tol, minres_tol, dv[c].vbuf,
                       dv[c].vgen};
      q[c] = make_queue(C, C.tune.S, err, limit);
      ng[c] = C.ngroups;
      hc[c] = C.hdr_cap;
      if (cudaMemsetAsync(C.slots, 0, 2 * (size_t)num_sms * sizeof(SlotN), s) != cudaSuccess ||
          cudaMemsetAsync(dv[c].vgen, 0, sizeof(unsigned) * 2 * (size_t)num_sms, s) !=
              cudaSuccess) {
        cudaGetLastError();
        return cleanup(HS_CUDA);
      }
    }
    if (ncls == 1) { a[1] = a[0]; q[1] = q[0]; }
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) {
      cudaGetLastError();
      return cleanup(HS_CUDA);
    }
    ls = launch_sweep((int)pc, k_lo, device, s, a, q, ng, hc);
    if (ls == HS_CUDA)
      for (int c = 0; c < ncls; ++c) cls[c].tune.S += 1;
  }
  if (ls != HS_OK) return cleanup(fail(hd[0], HS_CUDA, "hs_sweep: no group size fits"));
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(HS_CUDA);
  }
  const double t_solve = std::chrono::duration<double>(clk::now() - ts).count();
  // results into the Lanczos runs; Ritz pairs, twist overlaps, |z|^2
  long long total_iters = 0;
  int max_steps = 0;
  hs_status first_err = HS_OK;
  for (int c = 0; c < ncls; ++c) {
    Class& C = cls[c];
    const int nr = (int)C.idx.size();
    std::vector<double> ab((size_t)2 * SWEEP_MMAX * nr);
    std::vector<int> res(4 * (size_t)nr);
    std::vector<long long> its(nr);
    if (cudaMemcpy(ab.data(), dv[c].ab, sizeof(double) * ab.size(), cudaMemcpyDeviceToHost) !=
            cudaSuccess ||
        cudaMemcpy(res.data(), dv[c].res, sizeof(int) * res.size(), cudaMemcpyDeviceToHost) !=
            cudaSuccess ||
        cudaMemcpy(its.data(), dv[c].iters, sizeof(long long) * nr, cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
      cudaGetLastError();
      return cleanup(HS_CUDA);
    }
    int timeout = 0;
    cudaMemcpy(&timeout, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (timeout) return cleanup(fail(hd[0], HS_TIMEOUT, "hs_sweep: a group's wait gave up"));
    for (int j = 0; j < nr; ++j) {
      LzRun& R = runs[C.idx[j]];
      const int steps = res[4 * j];
      const double* al = &ab[(size_t)2 * SWEEP_MMAX * j];
      R.alpha.assign(al, al + steps);
      R.beta.assign(al + SWEEP_MMAX, al + SWEEP_MMAX + std::max(0, steps - 1));
      R.steps = steps;
      R.k = std::max(0, steps - 1);
      R.nconv = res[4 * j + 1];
      R.unconverged_solves = res[4 * j + 3];
      R.minres_iters = its[j];
      R.done = true;
      total_iters += its[j];
      max_steps = std::max(max_steps, steps);
      if (res[4 * j + 2] != HS_OK && first_err == HS_OK) first_err = (hs_status)res[4 * j + 2];
      if (steps > 0) {
        R.theta.assign(steps, 0.0);
        R.Y.assign((size_t)steps * steps, 0.0);
        if (tridiag_eig(steps, R.alpha.data(), R.beta.data(), R.theta.data(), R.Y.data()) != HS_OK &&
            first_err == HS_OK)
          first_err = HS_NOT_CONVERGED;
      }
    }
  }
  long long nmax = 0;
  for (int r = 0; r < B; ++r) nmax = std::max(nmax, hd[r]->n);
  if (cudaMalloc(&evbuf, sizeof(double) * (size_t)K * nmax) != cudaSuccess) return cleanup(HS_OOM);
  int converged = 0;
  double max_res = 0.0;
  std::vector<double> zz(B, 0.0), zb(2 * (size_t)K);
  for (int r = 0; r < B; ++r) {
    hs_lanczos_info li{};
    const hs_status fs = runs[r].steps >= K
                             ? lz_finish(runs[r], evals_host + (size_t)r * K, evbuf,
                                         resid_host ? resid_host + (size_t)r * K : nullptr, &li)
                             : HS_NOT_CONVERGED;
    if (fs != HS_OK && fs != HS_NOT_CONVERGED) return cleanup(fs);
    if (fs == HS_OK) ++converged;
    if (runs[r].steps < K) continue;
    max_res = std::max(max_res, li.max_resid);
    if ((st = launch_twist(hd[r], evbuf, K, zb.data())) != HS_OK) return cleanup(st);
    double a = 0.0;
    for (int q = 0; q < K; ++q) a += zb[2 * q] * zb[2 * q] + zb[2 * q + 1] * zb[2 * q + 1];
    zz[r] = a / K;
    if (z_host) std::memcpy(z_host + 2 * (size_t)K * r, zb.data(), sizeof(double) * 2 * K);
    if (zz_host) zz_host[r] = zz[r];
  }
  if (info) {
    info->realisations = B;
    info->converged = converged;
    info->max_steps = max_steps;
    info->launches = 1;
    info->minres_iters = total_iters;
    info->nclass = ncls;
    for (int c = 0; c < ncls; ++c) {
      info->L[c] = cls[c].L;
      info->S[c] = cls[c].tune.S;
      info->groups[c] = cls[c].ngroups;
      info->tuned[c] = cls[c].tuned;
      double m = 0.0;
      for (int r : cls[c].idx) m += zz[r];
      m /= cls[c].idx.size();
      double v = 0.0;
      for (int r : cls[c].idx) v += (zz[r] - m) * (zz[r] - m);
      info->zz_mean[c] = m;
      info->zz_std[c] = cls[c].idx.size() > 1 ? std::sqrt(v / (cls[c].idx.size() - 1)) : 0.0;
    }
    info->max_resid = max_res;
    info->seconds_setup = t_setup;
    info->seconds_solve = t_solve;
    info->seconds_total = std::chrono::duration<double>(clk::now() - t0).count();
  }
  if (first_err != HS_OK && first_err != HS_NOT_CONVERGED) return cleanup(first_err);
  return cleanup(converged == B ? HS_OK : HS_NOT_CONVERGED);
}
