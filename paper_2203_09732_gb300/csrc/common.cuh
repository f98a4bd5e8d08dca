// Internal declarations shared by the translation units of libhs.
//
// Data layout (all device vectors are in rank order, ascending state words):
//   A state word s of the Sz = 0 sector is split into k low bits
//   p = s & (2^k - 1) and hb = L - k high bits H = s >> k. All states with the
//   same H form one contiguous rank range (a "block") of C(k, w) rows,
//   w = L/2 - popcount(H), ordered by the colex rank r of p among k-bit words of
//   popcount w. So rank(s) = R_H + r, and blocks are ordered by H.
//   Bonds of Eq. (1) fall in four kinds:
//     low interior  (j, j+1), j + 1 < k : target stays in the block, r -> r'
//                                         (per-pattern neighbour list);
//     high interior (j, j+1), j >= k    : target = row + delta_H, the same
//                                         delta for every row of the block;
//     cut (k-1, k)                      : target = row + C(k-1, w-1) or
//                                         row - C(k-1, w), per block;
//     wrap (L-1, 0)                     : target = R_{H ^ top} + rank(p ^ 1).
//   One warp processes one block at a time (lane l takes rows l + 32 j); the
//   per-pattern table lives in shared memory, the 128-byte block header is read
//   with one coalesced load and broadcast by shuffles.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/hs.h"

// hv_sb.cu: whether the four-low-bit superblock form (sb4.cuh) serves products
// and MINRES pass A of precision dt where its plan applies
bool hs_want_sb4(hs_dtype dt);

namespace hs {

constexpr int LMAX = 32;
constexpr int KLO_MAX = 10;            // low bits per state (C(10, 5) = 252 rows per block)
constexpr int NB_MAX = KLO_MAX - 1;    // low interior bonds
constexpr int HD_MAX = 26;             // high interior bonds held by a block header
constexpr int HV_THREADS = 256;
constexpr int HV_WARPS = HV_THREADS / 32;
constexpr int JMAX = 8;                // rows per lane per block (C <= 256)
constexpr int RED_MAX_CTAS = 4096;     // partial-sum slots per reduction

// One entry per low pattern p, indexed by off[w] + r (class w, colex rank r); 32 bytes.
struct LowEntry {
  uint32_t packed;   // pat (bits 0..15) | nb_cnt << 16 | code << 20 | tlow << 24
  uint16_t wrap_r;   // colex rank of p ^ 1 in its class
  uint16_t pad;
  float dlow_f;      // dlow rounded to FP32
  uint32_t nbw[3];   // up to 9 neighbour ranks r' (uint8 each, same class)
  double dlow;       // Ising terms of low interior bonds + fields on low sites
};
static_assert(sizeof(LowEntry) == 32, "LowEntry is 32 bytes");
// code = bit (k-1) of p | bit 0 of p << 1; tlow = sum of (j + 1) over set bits j < k.

__host__ __device__ inline uint32_t le_pat(uint32_t pk) { return pk & 0xFFFFu; }
__host__ __device__ inline int le_cnt(uint32_t pk) { return (pk >> 16) & 0xF; }
__host__ __device__ inline uint32_t le_code(uint32_t pk) { return (pk >> 20) & 0x3; }
__host__ __device__ inline uint32_t le_tlow(uint32_t pk) { return pk >> 24; }

// One 128-byte header per valid high pattern H, in rank order (ascending H).
// Word layout (read by lane = word index): 0 R, 1 Rwrap, 2 bdelta,
// 3 w | nh << 8 | code << 16 | thigh << 24, 4-5 dhigh, 6.. hd[].
struct BlockInfo {
  uint32_t R;        // rank of the block's first row
  uint32_t Rwrap;    // first row of block H ^ top (only read when the wrap bond flips)
  int32_t bdelta;    // row offset of the cut-bond (k-1, k) flip
  uint8_t w;         // low popcount
  uint8_t nh;        // antiparallel high interior bonds
  uint8_t code;      // bit 0 of H | top bit of H << 1
  uint8_t thigh;     // sum of (j + 1) over set high bits j >= k, mod L
  double dhigh;      // Ising terms of high interior bonds + fields on high sites
  int32_t hd[HD_MAX];  // row offsets of the antiparallel high interior flips
};
static_assert(sizeof(BlockInfo) == 128, "BlockInfo is 128 bytes");

// Everything a row kernel needs, passed by value.
struct Geo {
  const LowEntry* low;
  const BlockInfo* blocks;
  int nblocks;
  int k, L, nlow;
  int cls_off[KLO_MAX + 2];
  int cls_C[KLO_MAX + 2];
  uint32_t n;
};

// MINRES device state (one per solver instance), all FP64 scalars.
struct MinresState {
  double beta_prev, beta, beta1;     // beta_{k-1}, beta_k, beta_1
  double alpha;                      // alpha_k
  double c_prev, s_prev;             // c_{k-1}, s_{k-1}
  double delta_hat, eps;             // hat delta_k, epsilon_k
  double phi;                        // phi_{k-1} (phi_k after pass B)
  double tol_abs;                    // tol * beta_1
  double cq, cd1, cd2, tau;          // pending d/x update (C step) coefficients
  double sigma;                      // shift used by the solve
  long long k;                       // current iteration index (1-based)
  long long kmax;
  int pending;                       // 1: apply the d/x update in the next pass A
  int done;                          // 0 running, 1 stop after pending update, 2 finished
  int status;                        // hs_status
  int pad;
};

}  // namespace hs

// The opaque handle of the C ABI.
struct hs_handle {
  int L = 0, N = 0, k = 0, hb = 0;
  long long n = 0;
  double h[hs::LMAX] = {0};
  double sigma = 0;
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 0;
  std::string err;

  // host tables
  std::vector<hs::LowEntry> low;
  std::vector<hs::BlockInfo> blocks;
  int cls_off[hs::KLO_MAX + 2] = {0};
  int cls_C[hs::KLO_MAX + 2] = {0};

  // device copies
  hs::LowEntry* d_low = nullptr;
  hs::BlockInfo* d_blocks = nullptr;
  uint32_t* d_binom = nullptr;       // (LMAX + 1) x (LMAX / 2 + 2)
  double* d_sigma = nullptr;         // device copy of sigma
  int grid_hv = 0;                   // grid of the row kernels

  // reductions
  double* d_partial = nullptr;
  unsigned int* d_counter = nullptr;
  double* h_pinned = nullptr;        // pinned host staging (RED_MAX_CTAS * 64 doubles)

  // MINRES workspace (lazily allocated)
  void* ws32 = nullptr;  size_t ws32_bytes = 0;
  void* ws64 = nullptr;  size_t ws64_bytes = 0;
  hs::MinresState* d_state = nullptr;
  hs::MinresState* h_state = nullptr;  // pinned
  cudaGraphExec_t graph32[3] = {nullptr, nullptr, nullptr};
  cudaGraphExec_t graph64[3] = {nullptr, nullptr, nullptr};

  // shared-memory-resident MINRES plan
  // SMs a persistent solve may use (0 = all); read once at the start of each
  // solve, and may be set from another host thread while a solve runs
  std::atomic<int> sm_budget{0};
  int smr_grid = 0, smr_rows_cap = 0, smr_hdr_cap = 0;
  int* d_smr_first = nullptr;

  // superblock H x plans (hv_sb.cu): [0] FP32, [1] FP64; null where not built
  void* sb_plan[2] = {nullptr, nullptr};
  // four-low-bit superblock plans (sb4.cuh): [0] FP32, [1] FP64
  void* sb4_plan[2] = {nullptr, nullptr};
  // superblock MINRES chunk graphs (minres_sb.cu), [precision][preconditioner],
  // with the grids (pass A, pass B) and the workspace they were captured for
  cudaGraphExec_t sbgraph[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  int sbgraph_key[2][3][2] = {};
  void* sbgraph_ws[2] = {nullptr, nullptr};

  // Lanczos workspace
  double* lz = nullptr; size_t lz_vectors = 0;

  hs::Geo geo() const;
};

namespace hs {

// launch accounting -----------------------------------------------------------
void count_launches(unsigned long long k);

// memory (api.cu) --------------------------------------------------------------
// Device buffers come from a library-owned memory pool, stream-ordered on the
// handle's stream (cudaMallocFromPoolAsync / cudaFreeAsync): creating and
// freeing handles never synchronises the device, so solves on other streams
// keep running. The pool keeps freed memory for reuse. Pinned host staging
// blocks come from a process-wide cache and are reused, never released.
hs_status dev_alloc(hs_handle* hd, void** p, size_t bytes);
void dev_free(hs_handle* hd, void* p);
void* host_pinned_get(size_t bytes);
void host_pinned_put(void* p, size_t bytes);
constexpr size_t PINNED_RED_BYTES = (size_t)RED_MAX_CTAS * 64 * sizeof(double);

// error helpers -------------------------------------------------------------
hs_status fail(hs_handle* hd, hs_status st, const std::string& msg);
#define HS_CUDA_TRY(hd, call)                                                   \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess)                                                      \
      return ::hs::fail((hd), HS_CUDA, std::string(#call) + ": " +              \
                                           cudaGetErrorString(e_));             \
  } while (0)

// launchers implemented in hv.cu -------------------------------------------
hs_status launch_matvec(hs_handle* hd, const void* x, void* y, hs_dtype dt, int shifted);
// hv_sb.cu: superblock form for long chains; *used = false if it does not apply
hs_status sb_setup(hs_handle* hd);
void sb_release(hs_handle* hd);
hs_status launch_matvec_sb(hs_handle* hd, const void* x, void* y, hs_dtype dt, int shifted,
                           bool* used);
hs_status launch_unrank(hs_handle* hd, long long first, long long count, unsigned int* out);
hs_status launch_rank(hs_handle* hd, const unsigned int* st, long long count, long long* out);
hs_status launch_diag(hs_handle* hd, double* diag, hs_precond pc, double* minv);
// FP64 r = b - (H - sigma) x; returns sum r^2/M and sum r^2 and the same for b.
// x_zero: x is zero (r = b; x is not read).
hs_status resid64(hs_handle* hd, const double* b, const double* x, double* r, hs_precond pc,
                  double sums_out[4], bool x_zero = false);

// minres_sb.cu: destroy the cached superblock MINRES graphs of precision ti
// (0 FP32, 1 FP64), e.g. before the workspace they point into is freed
void sb_graphs_release(hs_handle* hd, int ti);

// minres.cu -----------------------------------------------------------------
hs_status minres_solve64(hs_handle* hd, const double* b, double* x, double tol, long long kmax,
                         hs_precond pc, hs_minres_info* info);
hs_status minres_solve32(hs_handle* hd, const float* b, float* x, double tol, long long kmax,
                         hs_precond pc, hs_minres_info* info);
hs_status minres_mixed(hs_handle* hd, const double* b, double* x, double tol, long long kmax,
                       hs_precond pc, double inner_tol, hs_minres_info* info);

// vec.cu: FP64 vector kernels (Lanczos) ------------------------------------
hs_status vdot(hs_handle* hd, const double* a, const double* b, long long n, double* out);
hs_status vmultidot(hs_handle* hd, const double* V, int k, const double* w, long long n,
                    double* out);  // out[j] = V_j . w
hs_status vmultiaxpy(hs_handle* hd, const double* V, int k, const double* c, double* w,
                     long long n);  // w -= sum_j c_j V_j
hs_status vaxpby(hs_handle* hd, double a, const double* x, double b, double* y, long long n);
hs_status vscale_to(hs_handle* hd, double a, const double* x, double* y, long long n);
hs_status vsplitmix(hs_handle* hd, unsigned long long seed, double* v, long long n);
hs_status vritz(hs_handle* hd, const double* V, int k, const double* Y, int K, double* psi,
                long long n);  // psi_i = sum_j V_j Y[j + i k]
hs_status vcopy_f64_to_f32(hs_handle* hd, const double* x, double scale, float* y, long long n);
hs_status vaxpy_f32_to_f64(hs_handle* hd, double a, const float* x, double* y, long long n);

// twist.cu ------------------------------------------------------------------
hs_status launch_twist(hs_handle* hd, const double* psi, int K, double* z_host);

// host utilities --------------------------------------------------------------
uint32_t binom(int n, int r);
hs_status ensure_reduce(hs_handle* hd);
hs_status sum_partials(hs_handle* hd, int nparts, int width, double* out);
int row_grid(const hs_handle* hd);
hs_status tridiag_eig(int k, const double* alpha, const double* beta, double* theta, double* Y);

}  // namespace hs
