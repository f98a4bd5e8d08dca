// The paper's other observables of the eigenpairs (Sec. IV B):
//   bipartite entanglement entropy S = -Tr rho_A log rho_A, A = sites 1..L/2;
//   level spacing ratio r_k = min(d_k, d_{k-1}) / max(d_k, d_{k-1}).
//
// Split a state word at bit L/2: s = (s_B << L/2) | s_A (s_A = sites of A).
// In rank order the states with the same s_B form one contiguous run of
// C(L/2, a) rows, a = L/2 - popcount(s_B) up spins in A, ordered by the colex
// rank of s_A. So the coefficient block Psi_a (rows: s_A with a up spins,
// columns: s_B with L/2 - a up spins) has contiguous columns, and rho_A is
// block diagonal with blocks rho_a = Psi_a Psi_a^T. The blocks are formed on
// the device (k_rho: 32 x 32 tiles, the columns streamed through shared
// memory, FP64); their eigenvalues are found on the host (Householder
// reduction to tridiagonal form, then the implicit QL of lanczos.cu), one
// thread per block.
#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "common.cuh"

namespace hs {
namespace {

constexpr int RT = 32;       // tile edge
constexpr int RCH = 16;      // columns per shared-memory chunk

struct RhoTask {
  int cls;                   // a
  int ti, tj;                // tile row, tile column (tj <= ti)
};

// rho_a[i][j] for one 32 x 32 tile: 256 threads, each a 2 x 2 patch.
__global__ void __launch_bounds__(256) k_rho(const double* __restrict__ psi,
                                             const uint32_t* __restrict__ cols,
                                             const int* __restrict__ col_off,
                                             const int* __restrict__ dim,
                                             const long long* __restrict__ out_off,
                                             const RhoTask* __restrict__ tasks, double* rho) {
  __shared__ double sa[RCH][RT + 1], sb[RCH][RT + 1];
  const RhoTask t = tasks[blockIdx.x];
  const int d = dim[t.cls];
  const int c0 = col_off[t.cls], c1 = col_off[t.cls + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int cb = c0; cb < c1; cb += RCH) {
    __syncthreads();
    // stage RCH columns: rows of the tile row and of the tile column
    for (int e = threadIdx.x; e < RCH * RT; e += 256) {
      const int c = e / RT, r = e % RT;
      double va = 0.0, vb = 0.0;
      if (cb + c < c1) {
        const uint32_t base = cols[cb + c];
        const int ra = t.ti * RT + r, rb = t.tj * RT + r;
        if (ra < d) va = psi[base + ra];
        if (rb < d) vb = psi[base + rb];
      }
      sa[c][r] = va;
      sb[c][r] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < RCH; ++c) {
      const double a0 = sa[c][2 * ty], a1 = sa[c][2 * ty + 1];
      const double b0 = sb[c][2 * tx], b1 = sb[c][2 * tx + 1];
      acc[0][0] += a0 * b0;
      acc[0][1] += a0 * b1;
      acc[1][0] += a1 * b0;
      acc[1][1] += a1 * b1;
    }
  }
  double* out = rho + out_off[t.cls];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int r = t.ti * RT + 2 * ty + i, c = t.tj * RT + 2 * tx + j;
      if (r < d && c < d) out[(size_t)r * d + c] = acc[i][j];
    }
}

// Eigenvalues of the symmetric n x n matrix A (row-major, overwritten):
// Householder reflections H_k = I - v v^T / h reduce it to tridiagonal form
// (each applied as the symmetric rank-two update A -= v w^T + w v^T), then the
// implicit QL iteration of tridiag_eig.
hs_status sym_eigvals(int n, double* A, double* w) {
  if (n == 1) {
    w[0] = A[0];
    return HS_OK;
  }
  std::vector<double> d(n), e(n, 0.0), v(n), p(n);
  for (int k = 0; k + 2 < n; ++k) {
    // x = A[k+1.., k]
    double xx = 0.0;
    for (int i = k + 1; i < n; ++i) xx += A[(size_t)i * n + k] * A[(size_t)i * n + k];
    const double xn = std::sqrt(xx);
    const double x0 = A[(size_t)(k + 1) * n + k];
    d[k] = A[(size_t)k * n + k];
    if (xn == 0.0) {
      e[k] = 0.0;
      continue;
    }
    const double alpha = x0 >= 0.0 ? -xn : xn;      // the new subdiagonal entry
    e[k] = alpha;
    // v = x - alpha e_1, h = v^T v / 2
    for (int i = k + 1; i < n; ++i) v[i] = A[(size_t)i * n + k];
    v[k + 1] -= alpha;
    const double h = xx - alpha * x0;               // (v^T v) / 2
    // p = A v / h on the trailing block
    for (int i = k + 1; i < n; ++i) {
      double s = 0.0;
      const double* row = A + (size_t)i * n;
      for (int j = k + 1; j < n; ++j) s += row[j] * v[j];
      p[i] = s / h;
    }
    // w = p - (p^T v / (2 h)) v; A -= v w^T + w v^T
    double pv = 0.0;
    for (int i = k + 1; i < n; ++i) pv += p[i] * v[i];
    const double kk = pv / (2.0 * h);
    for (int i = k + 1; i < n; ++i) p[i] -= kk * v[i];
    for (int i = k + 1; i < n; ++i) {
      double* row = A + (size_t)i * n;
      const double vi = v[i], wi = p[i];
      for (int j = k + 1; j < n; ++j) row[j] -= vi * p[j] + wi * v[j];
    }
  }
  d[n - 2] = A[(size_t)(n - 2) * n + (n - 2)];
  d[n - 1] = A[(size_t)(n - 1) * n + (n - 1)];
  e[n - 2] = A[(size_t)(n - 1) * n + (n - 2)];
  return tridiag_eig(n, d.data(), e.data(), w, nullptr);
}

}  // namespace
}  // namespace hs

using namespace hs;

extern "C" hs_status hs_sym_eigvals(int n, double* a_host, double* w_host) {
  if (n < 1 || !a_host || !w_host) return HS_BAD_ARG;
  return sym_eigvals(n, a_host, w_host);
}

extern "C" hs_status hs_level_ratio(const double* evals_host, int K, double* r_host,
                                    double* mean_out) {
  if (K < 3 || !evals_host) return HS_BAD_ARG;
  std::vector<double> e(evals_host, evals_host + K);
  for (double v : e)
    if (!std::isfinite(v)) return HS_BAD_ARG;
  std::sort(e.begin(), e.end());
  double sum = 0.0;
  for (int k = 1; k + 1 < K; ++k) {
    const double d0 = e[k] - e[k - 1], d1 = e[k + 1] - e[k];
    const double lo = std::min(d0, d1), hi = std::max(d0, d1);
    const double r = hi > 0.0 ? lo / hi : 1.0;       // equal levels: ratio 1 by continuity
    if (r_host) r_host[k - 1] = r;
    sum += r;
  }
  if (mean_out) *mean_out = sum / (K - 2);
  return HS_OK;
}

extern "C" hs_status hs_entanglement(hs_handle* hd, const double* psi_dev, int K,
                                     double* S_host) {
  if (!hd) return HS_BAD_ARG;
  if (K < 1 || !psi_dev || !S_host) return fail(hd, HS_BAD_ARG, "hs_entanglement: bad arguments");
  const int L = hd->L, Lh = L / 2, N = L / 2;
  // columns of each block: the runs of the s_B (ascending) with a = Lh - popcount(s_B)
  std::vector<std::vector<uint32_t>> col(Lh + 1);
  uint64_t R = 0;
  for (uint32_t sB = 0; sB < (1u << (L - Lh)); ++sB) {
    const int a = N - __builtin_popcount(sB);
    if (a < 0 || a > Lh) continue;
    col[a].push_back((uint32_t)R);
    R += binom(Lh, a);
  }
  if ((long long)R != hd->n) return fail(hd, HS_BAD_ARG, "internal: column runs do not sum to n");
  std::vector<uint32_t> cols;
  std::vector<int> col_off(Lh + 2, 0), dim(Lh + 1);
  std::vector<long long> out_off(Lh + 2, 0);
  std::vector<RhoTask> tasks;
  for (int a = 0; a <= Lh; ++a) {
    col_off[a] = (int)cols.size();
    cols.insert(cols.end(), col[a].begin(), col[a].end());
    dim[a] = (int)binom(Lh, a);
    out_off[a + 1] = out_off[a] + (long long)dim[a] * dim[a];
    const int nt = (dim[a] + RT - 1) / RT;
    for (int ti = 0; ti < nt; ++ti)
      for (int tj = 0; tj <= ti; ++tj) tasks.push_back({a, ti, tj});
  }
  col_off[Lh + 1] = (int)cols.size();
  const long long total = out_off[Lh + 1];
  // device tables and the blocks
  auto bytes_al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t bc = bytes_al(cols.size() * 4), bo = bytes_al(col_off.size() * 4),
               bd = bytes_al(dim.size() * 4), bf = bytes_al(out_off.size() * 8),
               bt = bytes_al(tasks.size() * sizeof(RhoTask)), br = (size_t)total * 8;
  char* mem = nullptr;
  if (dev_alloc(hd, (void**)&mem, bc + bo + bd + bf + bt + br) != HS_OK)
    return fail(hd, HS_OOM, "hs_entanglement: allocation failed");
  std::vector<char> host(bc + bo + bd + bf + bt, 0);
  std::copy((char*)cols.data(), (char*)cols.data() + cols.size() * 4, host.data());
  std::copy((char*)col_off.data(), (char*)col_off.data() + col_off.size() * 4, host.data() + bc);
  std::copy((char*)dim.data(), (char*)dim.data() + dim.size() * 4, host.data() + bc + bo);
  std::copy((char*)out_off.data(), (char*)out_off.data() + out_off.size() * 8, host.data() + bc + bo + bd);
  std::copy((char*)tasks.data(), (char*)tasks.data() + tasks.size() * sizeof(RhoTask),
            host.data() + bc + bo + bd + bf);
  hs_status st = HS_OK;
  std::vector<double> rho((size_t)total);
  if (cudaMemcpyAsync(mem, host.data(), host.size(), cudaMemcpyHostToDevice, hd->stream) !=
      cudaSuccess) {
    cudaGetLastError();
    dev_free(hd, mem);
    return fail(hd, HS_CUDA, "hs_entanglement: table upload failed");
  }
  const uint32_t* d_cols = (const uint32_t*)mem;
  const int* d_off = (const int*)(mem + bc);
  const int* d_dim = (const int*)(mem + bc + bo);
  const long long* d_out = (const long long*)(mem + bc + bo + bd);
  const RhoTask* d_tasks = (const RhoTask*)(mem + bc + bo + bd + bf);
  double* d_rho = (double*)(mem + bc + bo + bd + bf + bt);
  for (int q = 0; q < K && st == HS_OK; ++q) {
    k_rho<<<(unsigned)tasks.size(), 256, 0, hd->stream>>>(psi_dev + (size_t)q * hd->n, d_cols, d_off,
                                                          d_dim, d_out, d_tasks, d_rho);
    count_launches(1);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(rho.data(), d_rho, br, cudaMemcpyDeviceToHost, hd->stream) != cudaSuccess ||
        cudaStreamSynchronize(hd->stream) != cudaSuccess) {
      cudaGetLastError();
      st = fail(hd, HS_CUDA, "hs_entanglement: rho blocks failed");
      break;
    }
    // mirror the lower triangle, eigenvalues per block (largest blocks first,
    // one host thread each), S = -sum lambda log lambda with lambda / Tr rho
    std::vector<std::vector<double>> lam(Lh + 1);
    std::vector<int> order(Lh + 1);
    for (int a = 0; a <= Lh; ++a) order[a] = a;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return dim[x] > dim[y]; });
    std::vector<hs_status> bst(Lh + 1, HS_OK);
    const unsigned nthr = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(),
                                                          (unsigned)(Lh + 1)));
    std::vector<std::thread> pool;
    std::atomic<int> next{0};
    for (unsigned t = 0; t < nthr; ++t)
      pool.emplace_back([&]() {
        for (int i = next++; i <= Lh; i = next++) {
          const int a = order[i], d = dim[a];
          double* A = rho.data() + out_off[a];
          for (int r = 0; r < d; ++r)
            for (int c = r + 1; c < d; ++c) A[(size_t)r * d + c] = A[(size_t)c * d + r];
          lam[a].assign(d, 0.0);
          bst[a] = sym_eigvals(d, A, lam[a].data());
        }
      });
    for (auto& th : pool) th.join();
    double tr = 0.0, s = 0.0;
    for (int a = 0; a <= Lh; ++a) {
      if (bst[a] != HS_OK) st = fail(hd, bst[a], "hs_entanglement: eigenvalues did not converge");
      for (double l : lam[a]) tr += l;
    }
    if (st != HS_OK) break;
    if (!(tr > 0.0)) {
      st = fail(hd, HS_BAD_ARG, "hs_entanglement: zero vector");
      break;
    }
    for (int a = 0; a <= Lh; ++a)
      for (double l : lam[a]) {
        const double x = l / tr;
        if (x > 0.0) s -= x * std::log(x);
      }
    S_host[q] = s;
  }
  dev_free(hd, mem);
  return st;
}
