// Batched disorder sweep: many realisations (of up to two chain lengths) run
// Algorithm 1 in lockstep rounds; each round's inner solves (Algorithm 2, one
// per realisation still running) go to one persistent cooperative launch whose
// CTA groups take them from per-length job queues (minres.cu,
// minres_pipe.cu), and the round's copies and launch are replayed from a CUDA
// graph. The group size and the form per (L, preconditioner, SM count) come
// from a short timing run, cached in a JSON file. The twist overlaps (Sec. III)
// of every realisation's pairs give |z|^2 averaged over the pairs of each
// realisation, then its mean and standard deviation over the realisations of
// each length (Sec. IV B-C).
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
};

void free_class(Class& c) {
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

SmemJob job_for(hs_handle* hd, const double* b, double* x, MinresState* st, double tol,
                long long kmax) {
  return SmemJob{hd->geo(), b, x, st, hd->sigma, tol, kmax};
}

// Launch of up to two queues (ng[i] groups of S[i] CTAs; ng[1] = 0: one).
hs_status launch_pair(const Class* c0, const Class* c1, int pc, bool one, int k, int device,
                      cudaStream_t s, int* err, unsigned long long limit) {
  const SmemQueue q0 = make_queue(*c0, c0->tune.S, err, limit);
  const SmemQueue qs[2] = {q0, c1 ? make_queue(*c1, c1->tune.S, err, limit) : q0};
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
  const Tune keep = c.tune;
  const int keep_ng = c.ngroups;
  c.tune.S = S;
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
  c.tune = keep;
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

// Groups per class: as many as fit for one class; for two, the split of the
// SMs that minimises the longer of the two classes' round times, with work
// proportional to realisations x n and speed to groups x the group rate.
void split_groups(Class* cls, int ncls, int num_sms) {
  if (ncls == 1) {
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
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  hs_status st = HS_OK;
  int device = 0, num_sms = 0;
  cudaGetDevice(&device);
  cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device);
  auto cleanup = [&](hs_status out) {
    cudaStreamSynchronize(s);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (int c = 0; c < ncls; ++c) free_class(cls[c]);
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
    }
  }
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return cleanup(HS_OOM);
  // schedule per class: forced (HS_SWEEP_S, HS_SWEEP_FORM = 1 or 2), cached or timed
  auto tunes = tune_read();
  bool tunes_changed = false;
  for (int c = 0; c < ncls; ++c) {
    Class& C = cls[c];
    C.hd0 = hd[C.idx[0]];
    C.n = C.hd0->n;
    if ((st = alloc_class(C, num_sms)) != HS_OK) return cleanup(st);
    char key[96];
    snprintf(key, sizeof key, "L%d_pc%d_f64_sm%d", C.L, (int)pc, num_sms);
    const char* fs = getenv("HS_SWEEP_S");
    const char* ff = getenv("HS_SWEEP_FORM");
    const int form = ff ? (ff[0] == '1' ? 1 : 0) : -1;
    if (fs || ff) {
      if (fs) {
        C.tune.S = std::max(1, atoi(fs));
        C.tune.one = form == 1 ? 1 : 0;
        C.tune.rate = 1.0;
      } else if ((st = tune_class(C, runs, pc, num_sms, device, s, err, form)) != HS_OK) {
        return cleanup(st);
      }
      C.tuned = -1;
    } else if (tunes.count(key)) {
      C.tune = tunes[key];
      C.tuned = 0;
    } else {
      if ((st = tune_class(C, runs, pc, num_sms, device, s, err, -1)) != HS_OK) return cleanup(st);
      tunes[key] = C.tune;
      tunes_changed = true;
    }
  }
  if (tunes_changed) tune_write(tunes);
  // the two classes share one launch, so one form: the one-reduction form
  // only where both chose it (a group size chosen for it also fits the
  // two-reduction form, which needs less shared memory, not the reverse)
  const bool one = cls[0].tune.one != 0 && (ncls == 1 || cls[1].tune.one != 0);
  split_groups(cls, ncls, num_sms);
  for (int c = 0; c < ncls; ++c) {
    if ((st = smr_plan(cls[c].hd0, cls[c].tune.S, &cls[c].first, &cls[c].rows_cap,
                       &cls[c].hdr_cap)) != HS_OK)
      return cleanup(st);
  }
  const double t_setup = std::chrono::duration<double>(clk::now() - t0).count();
  // rounds
  const auto ts = clk::now();
  const unsigned long long limit = 1ull << 22;
  // one kernel shape per launch: the rows-per-lane template follows k <= 8
  const int k_lo = cls[0].hd0->k;
  for (int c = 1; c < ncls; ++c)
    if ((cls[c].hd0->k <= 8) != (k_lo <= 8)) return cleanup(HS_BAD_ARG);
  int rounds = 0, launches = 0, use_graph = 0;
  bool graph_tried = false;
  long long total_iters = 0;
  auto enqueue_round = [&]() -> hs_status {
    for (int c = 0; c < ncls; ++c) {
      Class& C = cls[c];
      HS_CUDA_TRY(hd[0], cudaMemcpyAsync(C.jobs, C.h_jobs, C.cap * sizeof(SmemJob),
                                         cudaMemcpyHostToDevice, s));
      HS_CUDA_TRY(hd[0], cudaMemcpyAsync(C.head, C.h_head, 2 * sizeof(int),
                                         cudaMemcpyHostToDevice, s));
      HS_CUDA_TRY(hd[0], cudaMemsetAsync(C.slots, 0, 2 * (size_t)num_sms * sizeof(SlotN), s));
    }
    HS_CUDA_TRY(hd[0], cudaMemsetAsync(err, 0, sizeof(int), s));
    hs_status ls = launch_pair(&cls[0], ncls == 2 ? &cls[1] : nullptr, pc, one, k_lo, device, s,
                               err, limit);
    if (ls != HS_OK) return ls;
    for (int c = 0; c < ncls; ++c)
      HS_CUDA_TRY(hd[0], cudaMemcpyAsync(cls[c].h_states, cls[c].states,
                                         cls[c].cap * sizeof(MinresState),
                                         cudaMemcpyDeviceToHost, s));
    return HS_OK;
  };
  std::vector<int> active;
  while (true) {
    // jobs of the round: one per realisation still running
    int njobs_total = 0;
    for (int c = 0; c < ncls; ++c) {
      Class& C = cls[c];
      int j = 0;
      for (int r : C.idx) {
        if (runs[r].done) continue;
        C.h_jobs[j] = job_for(hd[r], runs[r].rhs(), runs[r].x, C.states + j, minres_tol,
                              50 * hd[r]->n);
        ++j;
      }
      C.h_head[0] = 0;
      C.h_head[1] = j;
      njobs_total += j;
    }
    if (!njobs_total) break;
    // the round's copies and launch, captured once and replayed
    if (!graph_tried) {
      graph_tried = true;
      if (!getenv("HS_SWEEP_NOGRAPH") &&
          cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const hs_status cs = enqueue_round();
        const cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (cs == HS_OK && ce == cudaSuccess && graph &&
            cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
          use_graph = 1;
        } else {
          if (graph) cudaGraphDestroy(graph);
          graph = nullptr;
          exec = nullptr;
        }
        cudaGetLastError();
      }
    }
    if (use_graph) {
      if (cudaGraphLaunch(exec, s) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(HS_CUDA);
      }
      if (rounds > 0) count_launches(1);   // the capture counted the first
    } else if ((st = enqueue_round()) != HS_OK) {
      return cleanup(st);
    }
    ++launches;
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return cleanup(HS_CUDA);
    }
    // one-reduction solves whose expansion cancelled: again, two-reduction form
    if (one) {
      for (int c = 0; c < ncls; ++c) {
        Class& C = cls[c];
        int nre = 0;
        for (int j = 0; j < C.h_head[1]; ++j)
          if (C.h_states[j].status == HS_BREAKDOWN && C.h_states[j].pad == PIPE_EXPANSION)
            C.h_jobs[nre++] = C.h_jobs[j];   // states of the first nre slots are rewritten
        if (!nre) continue;
        std::vector<int> where;
        for (int j = 0; j < C.h_head[1]; ++j)
          if (C.h_states[j].status == HS_BREAKDOWN && C.h_states[j].pad == PIPE_EXPANSION)
            where.push_back(j);
        for (int q = 0; q < nre; ++q) C.h_jobs[q].st = C.states + q;
        int head2[2] = {0, nre};
        memcpy(C.h_head, head2, sizeof head2);
        const int ng_keep = C.ngroups;
        C.ngroups = std::max(1, std::min(ng_keep, nre));
        if (cudaMemcpyAsync(C.jobs, C.h_jobs, nre * sizeof(SmemJob), cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(C.head, C.h_head, 2 * sizeof(int), cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaMemsetAsync(C.slots, 0, 2 * (size_t)num_sms * sizeof(SlotN), s) != cudaSuccess ||
            cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) {
          cudaGetLastError();
          return cleanup(HS_CUDA);
        }
        st = launch_pair(&C, nullptr, pc, false, k_lo, device, s, err, limit);
        C.ngroups = ng_keep;
        if (st != HS_OK) return cleanup(st);
        ++launches;
        std::vector<MinresState> redo(nre);
        if (cudaMemcpyAsync(redo.data(), C.states, nre * sizeof(MinresState),
                            cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
          cudaGetLastError();
          return cleanup(HS_CUDA);
        }
        for (int q = 0; q < nre; ++q) C.h_states[where[q]] = redo[q];
      }
    }
    ++rounds;
    // the rest of each realisation's step
    for (int c = 0; c < ncls; ++c) {
      Class& C = cls[c];
      int j = 0;
      for (int r : C.idx) {
        if (runs[r].done) continue;
        const MinresState& S = C.h_states[j++];
        hs_status out = (hs_status)S.status;
        if (out == HS_OK && S.beta1 > 0 && !(std::fabs(S.phi) < S.tol_abs) && S.beta != 0.0)
          out = HS_NOT_CONVERGED;
        if (out == HS_TIMEOUT) return cleanup(fail(hd[r], HS_TIMEOUT, "sweep: a group's wait gave up"));
        total_iters += std::max(0LL, S.k - 1);
        if ((st = lz_step(runs[r], out, std::max(0LL, S.k - 1), 1)) != HS_OK) return cleanup(st);
      }
    }
  }
  const double t_solve = std::chrono::duration<double>(clk::now() - ts).count();
  // Ritz pairs, twist overlaps, |z|^2 per realisation and per length
  long long nmax = 0;
  for (int r = 0; r < B; ++r) nmax = std::max(nmax, hd[r]->n);
  if (cudaMalloc(&evbuf, sizeof(double) * (size_t)K * nmax) != cudaSuccess) return cleanup(HS_OOM);
  int converged = 0;
  double max_res = 0.0;
  std::vector<double> zz(B, 0.0), zb(2 * (size_t)K);
  for (int r = 0; r < B; ++r) {
    hs_lanczos_info li;
    const hs_status fs = lz_finish(runs[r], evals_host + (size_t)r * K, evbuf,
                                   resid_host ? resid_host + (size_t)r * K : nullptr, &li);
    if (fs != HS_OK && fs != HS_NOT_CONVERGED) return cleanup(fs);
    if (fs == HS_OK) ++converged;
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
    info->rounds = rounds;
    info->launches = launches;
    info->graph = use_graph;
    info->minres_iters = total_iters;
    info->nclass = ncls;
    for (int c = 0; c < ncls; ++c) {
      info->L[c] = cls[c].L;
      info->S[c] = cls[c].tune.S;
      info->groups[c] = cls[c].ngroups;
      info->form[c] = one ? HS_FORM_SMEM1 : HS_FORM_SMEM;
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
  return cleanup(converged == B ? HS_OK : HS_NOT_CONVERGED);
}
