// Handle creation (host construction of the ranking tables), utilities and
// the thin C-ABI entry points of include/hs.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <new>

#include "common.cuh"

#include <atomic>
#include <map>
#include <mutex>

namespace hs {

static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];
static int g_pool_state[64];  // 0 unknown, 1 pool, 2 no pool (plain cudaMalloc)

static cudaMemPool_t pool_for(int dev) {
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (g_pool_state[dev] == 0) {
    g_pool_state[dev] = 2;
    int ok = 0;
    if (cudaDeviceGetAttribute(&ok, cudaDevAttrMemoryPoolsSupported, dev) == cudaSuccess && ok) {
      cudaMemPoolProps props;
      std::memset(&props, 0, sizeof(props));
      props.allocType = cudaMemAllocationTypePinned;
      props.handleTypes = cudaMemHandleTypeNone;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      cudaMemPool_t pool;
      if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
        uint64_t keep = ~0ull;  // keep freed memory in the pool
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = pool;
        g_pool_state[dev] = 1;
      }
    }
    cudaGetLastError();
  }
  return g_pool_state[dev] == 1 ? g_pool[dev] : nullptr;
}

hs_status dev_alloc(hs_handle* hd, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 256;
  cudaMemPool_t pool = pool_for(hd->device);
  const cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, hd->stream)
                             : cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(hd, HS_OOM, "device allocation failed");
  }
  return HS_OK;
}

void dev_free(hs_handle* hd, void* p) {
  if (!p) return;
  if (pool_for(hd->device)) cudaFreeAsync(p, hd->stream);
  else cudaFree(p);
}

static std::mutex g_pin_mu;
static std::multimap<size_t, void*> g_pin_free;

void* host_pinned_get(size_t bytes) {
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    auto it = g_pin_free.find(bytes);
    if (it != g_pin_free.end()) {
      void* q = it->second;
      g_pin_free.erase(it);
      return q;
    }
  }
  void* q = nullptr;
  if (cudaMallocHost(&q, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return q;
}

void host_pinned_put(void* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.emplace(bytes, p);
}

static std::atomic<unsigned long long> g_launches{0};
void count_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

hs_status fail(hs_handle* hd, hs_status st, const std::string& msg) {
  if (hd) hd->err = msg;
  return st;
}

uint32_t binom(int n, int r) {
  if (r < 0 || n < 0 || r > n) return 0;
  uint64_t v = 1;
  for (int i = 1; i <= r; ++i) v = v * (uint64_t)(n - r + i) / (uint64_t)i;
  return (uint32_t)v;
}

int row_grid(const hs_handle* hd) {
  const int need = ((int)hd->blocks.size() + HV_WARPS - 1) / HV_WARPS;
  return std::max(1, std::min(need, hd->grid_hv));
}

hs_status ensure_reduce(hs_handle* hd) {
  if (hd->d_partial) return HS_OK;
  const size_t nd = (size_t)RED_MAX_CTAS * 4 + 1024 * 512 + 8192;
  hs_status st = dev_alloc(hd, (void**)&hd->d_partial, nd * sizeof(double));
  if (st != HS_OK) return st;
  if ((st = dev_alloc(hd, (void**)&hd->d_counter, 16 * sizeof(unsigned int))) != HS_OK) return st;
  HS_CUDA_TRY(hd, cudaMemsetAsync(hd->d_counter, 0, 16 * sizeof(unsigned int), hd->stream));
  hd->h_pinned = static_cast<double*>(host_pinned_get(PINNED_RED_BYTES));
  if (!hd->h_pinned) return fail(hd, HS_OOM, "pinned host allocation failed");
  return HS_OK;
}

hs_status sum_partials(hs_handle* hd, int nparts, int width, double* out) {
  HS_CUDA_TRY(hd, cudaMemcpyAsync(hd->h_pinned, hd->d_partial, sizeof(double) * nparts * 4,
                                  cudaMemcpyDeviceToHost, hd->stream));
  HS_CUDA_TRY(hd, cudaStreamSynchronize(hd->stream));
  for (int j = 0; j < width; ++j) out[j] = 0.0;
  for (int c = 0; c < nparts; ++c)
    for (int j = 0; j < width; ++j) out[j] += hd->h_pinned[c * 4 + j];
  return HS_OK;
}

// colex rank of a k-bit pattern among patterns of the same popcount
static int colex_rank(uint32_t p) {
  int r = 0, c = 1;
  while (p) {
    const int pos = __builtin_ctz(p);
    r += (int)binom(pos, c);
    ++c;
    p &= p - 1u;
  }
  return r;
}

// Build the low-pattern table and the block headers (see common.cuh).
static hs_status build_tables(hs_handle* hd) {
  const int L = hd->L, N = hd->N, k = hd->k, hb = hd->hb;
  if (hb - 1 > HD_MAX) return fail(hd, HS_BAD_ARG, "too many high bits for the block header");
  int off = 0;
  for (int w = 0; w <= k; ++w) {
    hd->cls_off[w] = off;
    hd->cls_C[w] = (int)binom(k, w);
    off += hd->cls_C[w];
  }
  const int nlow = off;  // 2^k
  hd->low.assign(nlow, LowEntry{});
  std::vector<int> fill(k + 1, 0);
  for (uint32_t p = 0; p < (1u << k); ++p) {  // ascending = colex within each class
    const int w = __builtin_popcount(p);
    const int r = fill[w]++;
    const int li = hd->cls_off[w] + r;
    LowEntry e;
    std::memset(&e, 0, sizeof(e));
    double d = 0.0;
    int cnt = 0;
    for (int j = 0; j + 1 < k; ++j) {
      const int a = (p >> j) & 1, b = (p >> (j + 1)) & 1;
      if (a == b) {
        d += 0.25;
      } else {
        d -= 0.25;
        const uint32_t rn = (uint32_t)colex_rank(p ^ (3u << j));
        if (rn > 255u) return fail(hd, HS_BAD_ARG, "neighbour rank does not fit 8 bits");
        e.nbw[cnt >> 2] |= rn << (8 * (cnt & 3));
        ++cnt;
      }
    }
    uint32_t tlow = 0;
    for (int j = 0; j < k; ++j) {
      const int up = (p >> j) & 1;
      d -= hd->h[j] * (up ? 0.5 : -0.5);
      if (up) tlow += (uint32_t)(j + 1);
    }
    const uint32_t code = ((p >> (k - 1)) & 1u) | ((p & 1u) << 1);
    e.packed = p | ((uint32_t)cnt << 16) | (code << 20) | (tlow << 24);
    e.wrap_r = (uint16_t)colex_rank(p ^ 1u);
    e.dlow_f = (float)d;
    e.dlow = d;
    hd->low[li] = e;
  }
  // blocks in ascending H (= rank order)
  const uint32_t nH = 1u << hb;
  std::vector<uint32_t> Rof(nH, 0xFFFFFFFFu);
  hd->blocks.clear();
  hd->blocks.reserve(nH);
  uint64_t R = 0;
  for (uint32_t H = 0; H < nH; ++H) {
    const int w = N - __builtin_popcount(H);
    if (w < 0 || w > k) continue;
    Rof[H] = (uint32_t)R;
    BlockInfo b;
    std::memset(&b, 0, sizeof(b));
    b.R = (uint32_t)R;
    b.w = (uint8_t)w;
    b.code = (uint8_t)((H & 1u) | (((H >> (hb - 1)) & 1u) << 1));
    // cut bond (k-1, k)
    if (H & 1u) b.bdelta = (w < k) ? -(int32_t)binom(k - 1, w) : 0;
    else b.bdelta = (w >= 1) ? (int32_t)binom(k - 1, w - 1) : 0;
    double d = 0.0;
    int nh = 0;
    for (int j = 0; j + 1 < hb; ++j) {
      const int a = (H >> j) & 1, c2 = (H >> (j + 1)) & 1;
      if (a == c2) {
        d += 0.25;
      } else {
        d -= 0.25;
        const int P = k + j;
        const int below = w + __builtin_popcount(H & ((1u << j) - 1u));
        const int32_t dl = (int32_t)binom(P, below);
        b.hd[nh++] = a ? dl : -dl;
      }
    }
    uint32_t th = 0;
    for (int j = 0; j < hb; ++j) {
      const int up = (H >> j) & 1;
      d -= hd->h[k + j] * (up ? 0.5 : -0.5);
      if (up) th += (uint32_t)(k + j + 1);
    }
    b.nh = (uint8_t)nh;
    b.thigh = (uint8_t)(th % (uint32_t)L);
    b.dhigh = d;
    hd->blocks.push_back(b);
    // the wrap partner is filled below; remember H in Rwrap for now
    hd->blocks.back().Rwrap = H;
    R += binom(k, w);
  }
  if ((long long)R != hd->n) return fail(hd, HS_BAD_ARG, "internal: block sizes do not sum to n");
  for (auto& b : hd->blocks) {
    const uint32_t Hw = b.Rwrap ^ (1u << (hb - 1));
    b.Rwrap = Rof[Hw] == 0xFFFFFFFFu ? 0u : Rof[Hw];
  }
  return HS_OK;
}

template <typename T>
static hs_status upload(hs_handle* hd, T** dst, const std::vector<T>& src) {
  const size_t bytes = std::max<size_t>(sizeof(T), src.size() * sizeof(T));
  hs_status st = dev_alloc(hd, (void**)dst, bytes);
  if (st != HS_OK) return st;
  // pageable source: the copy is staged before the call returns
  if (!src.empty())
    HS_CUDA_TRY(hd, cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T),
                                    cudaMemcpyHostToDevice, hd->stream));
  return HS_OK;
}

hs_status set_sigma_dev(hs_handle* hd, double sigma) {
  hd->sigma = sigma;
  HS_CUDA_TRY(hd, cudaMemcpyAsync(hd->d_sigma, &hd->sigma, sizeof(double), cudaMemcpyHostToDevice,
                                  hd->stream));
  HS_CUDA_TRY(hd, cudaStreamSynchronize(hd->stream));
  return HS_OK;
}

}  // namespace hs

hs::Geo hs_handle::geo() const {
  hs::Geo g;
  g.low = d_low;
  g.blocks = d_blocks;
  g.nblocks = (int)blocks.size();
  g.k = k;
  g.L = L;
  g.nlow = (int)low.size();
  for (int i = 0; i < hs::KLO_MAX + 2; ++i) {
    g.cls_off[i] = cls_off[i];
    g.cls_C[i] = cls_C[i] > 0 ? cls_C[i] : 1;
  }
  g.n = (uint32_t)n;
  return g;
}

using namespace hs;

extern "C" {

static const char* kNullHandle = "null handle";

unsigned long long hs_kernel_launches(void) { return g_launches.load(); }

const char* hs_last_error(const hs_handle* hd) { return hd ? hd->err.c_str() : kNullHandle; }

hs_status hs_create(int L, const double* h_host, double sigma, void* cuda_stream,
                    hs_handle** out) {
  if (!out) return HS_BAD_ARG;
  *out = nullptr;
  if (L < 4 || L > LMAX || (L & 1) || !h_host) return HS_BAD_ARG;
  for (int j = 0; j < L; ++j)
    if (!std::isfinite(h_host[j])) return HS_BAD_ARG;
  if (std::isinf(sigma)) return HS_BAD_ARG;
  hs_handle* hd = new (std::nothrow) hs_handle();
  if (!hd) return HS_OOM;
  hd->L = L;
  hd->N = L / 2;
  // low bits: 10 (blocks of up to 252 rows) for large chains, 8 below L = 22
  // so that small chains still have enough blocks to spread over the GPU;
  // HS_KLO overrides it (tuning)
  int kk = L >= 22 ? 10 : 8;
  if (const char* e = getenv("HS_KLO")) kk = atoi(e);
  hd->k = std::max(2, std::min(std::min(KLO_MAX, kk), L - 2));
  hd->hb = L - hd->k;
  hd->n = (long long)binom(L, L / 2);
  for (int j = 0; j < L; ++j) hd->h[j] = h_host[j];
  hd->stream = static_cast<cudaStream_t>(cuda_stream);
  hs_status st = HS_OK;
  auto bail = [&](hs_status s) { hs_free(hd); return s; };
  if (cudaGetDevice(&hd->device) != cudaSuccess) { cudaGetLastError(); return bail(HS_CUDA); }
  if (cudaDeviceGetAttribute(&hd->num_sms, cudaDevAttrMultiProcessorCount, hd->device) !=
      cudaSuccess) {
    cudaGetLastError();
    return bail(HS_CUDA);
  }
  hd->grid_hv = std::min(RED_MAX_CTAS, hd->num_sms * 4);
  if ((st = build_tables(hd)) != HS_OK) return bail(st);
  if ((st = upload(hd, &hd->d_low, hd->low)) != HS_OK) return bail(st);
  if ((st = upload(hd, &hd->d_blocks, hd->blocks)) != HS_OK) return bail(st);
  {
    const int W = LMAX / 2 + 2;
    std::vector<uint32_t> bt((LMAX + 1) * W);
    for (int a = 0; a <= LMAX; ++a)
      for (int c = 0; c < W; ++c) bt[a * W + c] = binom(a, c);
    if ((st = upload(hd, &hd->d_binom, bt)) != HS_OK) return bail(st);
  }
  // superblock plans for long chains; HS_SB_PLANS=1 builds them for any L
  // whose windows apply (tests of the superblock forms on small chains)
  {
    const char* e = getenv("HS_SB_PLANS");
    const bool plans = L >= 22 || (e && e[0] == '1');
    if (plans && (st = sb_setup(hd)) != HS_OK) return bail(st);
  }
  if ((st = dev_alloc(hd, (void**)&hd->d_sigma, sizeof(double))) != HS_OK) return bail(st);
  if ((st = ensure_reduce(hd)) != HS_OK) return bail(st);
  if (std::isnan(sigma)) {
    double emin, emax, mid;
    if ((st = set_sigma_dev(hd, 0.0)) != HS_OK) return bail(st);
    if ((st = hs_extremal(hd, 600, 1e-12, &emin, &emax, &mid)) != HS_OK) return bail(st);
    sigma = mid;
  }
  if ((st = set_sigma_dev(hd, sigma)) != HS_OK) return bail(st);
  *out = hd;
  return HS_OK;
}

void hs_free(hs_handle* hd) {
  if (!hd) return;
  if (hd->stream || true) cudaStreamSynchronize(hd->stream);
  for (int i = 0; i < 3; ++i) {
    if (hd->graph32[i]) cudaGraphExecDestroy(hd->graph32[i]);
    if (hd->graph64[i]) cudaGraphExecDestroy(hd->graph64[i]);
  }
  dev_free(hd, hd->d_low);
  dev_free(hd, hd->d_blocks);
  dev_free(hd, hd->d_binom);
  dev_free(hd, hd->d_sigma);
  dev_free(hd, hd->d_partial);
  dev_free(hd, hd->d_counter);
  dev_free(hd, hd->ws32);
  dev_free(hd, hd->ws64);
  dev_free(hd, hd->d_state);
  dev_free(hd, hd->lz);
  dev_free(hd, hd->d_smr_first);
  sb_graphs_release(hd, 0);
  sb_graphs_release(hd, 1);
  sb_release(hd);
  host_pinned_put(hd->h_pinned, PINNED_RED_BYTES);
  host_pinned_put(hd->h_state, sizeof(MinresState));
  cudaGetLastError();
  delete hd;
}

hs_status hs_set_sm_budget(hs_handle* hd, int nsm) {
  if (!hd) return HS_BAD_ARG;
  if (nsm < 0) return fail(hd, HS_BAD_ARG, "hs_set_sm_budget: negative SM count");
  hd->sm_budget.store(nsm, std::memory_order_relaxed);
  return HS_OK;
}

hs_status hs_dim(const hs_handle* hd, long long* n_out) {
  if (!hd || !n_out) return HS_BAD_ARG;
  *n_out = hd->n;
  return HS_OK;
}

hs_status hs_get_sigma(const hs_handle* hd, double* s) {
  if (!hd || !s) return HS_BAD_ARG;
  *s = hd->sigma;
  return HS_OK;
}

hs_status hs_set_sigma(hs_handle* hd, double sigma) {
  if (!hd) return HS_BAD_ARG;
  if (!std::isfinite(sigma)) return fail(hd, HS_BAD_ARG, "sigma must be finite");
  HS_CUDA_TRY(hd, cudaStreamSynchronize(hd->stream));
  return set_sigma_dev(hd, sigma);
}

hs_status hs_unrank(hs_handle* hd, long long first, long long count, unsigned int* states_dev) {
  if (!hd) return HS_BAD_ARG;
  if (count < 0 || first < 0 || first + count > hd->n || (count > 0 && !states_dev))
    return fail(hd, HS_BAD_ARG, "hs_unrank: range outside [0, n)");
  return launch_unrank(hd, first, count, states_dev);
}

hs_status hs_rank(hs_handle* hd, const unsigned int* states_dev, long long count,
                  long long* ranks_dev) {
  if (!hd) return HS_BAD_ARG;
  if (count < 0 || (count > 0 && (!states_dev || !ranks_dev)))
    return fail(hd, HS_BAD_ARG, "hs_rank: bad arguments");
  return launch_rank(hd, states_dev, count, ranks_dev);
}

hs_status hs_diag(hs_handle* hd, double* diag_dev, hs_precond pc, double* minv_dev) {
  if (!hd) return HS_BAD_ARG;
  if (pc < HS_PC_ID || pc > HS_PC_ROWNORM) return fail(hd, HS_BAD_ARG, "bad preconditioner");
  if (!diag_dev && !minv_dev) return HS_OK;
  return launch_diag(hd, diag_dev, pc, minv_dev);
}

hs_status hs_matvec(hs_handle* hd, const void* x_dev, void* y_dev, hs_dtype dtype, int shifted) {
  if (!hd) return HS_BAD_ARG;
  if (!x_dev || !y_dev || x_dev == y_dev) return fail(hd, HS_BAD_ARG, "hs_matvec: bad pointers");
  if (dtype != HS_F32 && dtype != HS_F64) return fail(hd, HS_BAD_ARG, "hs_matvec: bad dtype");
  const uintptr_t es = dtype == HS_F32 ? sizeof(float) : sizeof(double);
  if ((uintptr_t)x_dev % es || (uintptr_t)y_dev % es)
    return fail(hd, HS_BAD_ARG, "hs_matvec: vectors not aligned to their element size");
  return launch_matvec(hd, x_dev, y_dev, dtype, shifted ? 1 : 0);
}

hs_status hs_minres(hs_handle* hd, const double* b_dev, double* x_dev, double tol, long long kmax,
                    hs_precond pc, int mixed, double inner_tol, hs_minres_info* info) {
  if (!hd) return HS_BAD_ARG;
  if (!b_dev || !x_dev || b_dev == x_dev) return fail(hd, HS_BAD_ARG, "hs_minres: bad pointers");
  if (!(tol >= 0) || pc < HS_PC_ID || pc > HS_PC_ROWNORM)
    return fail(hd, HS_BAD_ARG, "hs_minres: bad tolerance or preconditioner");
  if (kmax <= 0) kmax = 20 * hd->n;
  if (info) std::memset(info, 0, sizeof(*info));
  hs_status st;
  if (!mixed) {
    st = minres_solve64(hd, b_dev, x_dev, tol, kmax, pc, info);
    if (info) {
      info->sweeps = 1;
      double sums[4];
      double* r = nullptr;
      if (dev_alloc(hd, (void**)&r, sizeof(double) * hd->n) == HS_OK) {
        if (resid64(hd, b_dev, x_dev, r, pc, sums) == HS_OK) {
          info->resid_minv = sums[2] > 0 ? std::sqrt(sums[0] / sums[2]) : 0.0;
          info->resid_2 = sums[3] > 0 ? std::sqrt(sums[1] / sums[3]) : 0.0;
        }
        dev_free(hd, r);
      } else {
        hd->err.clear();
      }
    }
    return st;
  }
  const double itol = inner_tol > 0 ? inner_tol : 1e-5;
  return minres_mixed(hd, b_dev, x_dev, tol, kmax, pc, itol, info);
}

hs_status hs_minres_f32(hs_handle* hd, const float* b_dev, float* x_dev, double tol,
                        long long kmax, hs_precond pc, hs_minres_info* info) {
  if (!hd) return HS_BAD_ARG;
  if (!b_dev || !x_dev || (const void*)b_dev == (void*)x_dev)
    return fail(hd, HS_BAD_ARG, "hs_minres_f32: bad pointers");
  if (!(tol >= 0) || pc < HS_PC_ID || pc > HS_PC_ROWNORM)
    return fail(hd, HS_BAD_ARG, "hs_minres_f32: bad tolerance or preconditioner");
  if (kmax <= 0) kmax = 20 * hd->n;
  if (info) std::memset(info, 0, sizeof(*info));
  hs_status st = minres_solve32(hd, b_dev, x_dev, tol, kmax, pc, info);
  if (info) info->sweeps = 1;
  return st;
}

hs_status hs_twist(hs_handle* hd, const double* psi_dev, int K, double* z_host) {
  if (!hd) return HS_BAD_ARG;
  if (K < 0 || (K > 0 && (!psi_dev || !z_host))) return fail(hd, HS_BAD_ARG, "hs_twist: bad arguments");
  return launch_twist(hd, psi_dev, K, z_host);
}

hs_status hs_tridiag_eig(int k, const double* alpha, const double* beta, double* theta, double* Y) {
  if (k < 1 || !alpha || !theta || (k > 1 && !beta)) return HS_BAD_ARG;
  return tridiag_eig(k, alpha, beta, theta, Y);
}

}  // extern "C"
