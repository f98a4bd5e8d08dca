// Internal declarations shared by the translation units of libhs.
//
// Data layout (all device vectors are in rank order, ascending state words):
//   A state word s of the Sz = 0 sector is split into k low bits
//   p = s & (2^k - 1) and hb = L - k high bits H = s >> k. All states with the
//   same H form one contiguous rank range (a "block") of C(k, w) rows,
//   w = L/2 - popcount(H), ordered by the colex rank r of p among k-bit words of
//   popcount w. So rank(s) = R_H + r.
//   Bonds of Eq. (1) fall in four kinds:
//     low interior  (j, j+1), j + 1 < k : target stays in the block, r -> r'
//                                         (per-pattern neighbour list);
//     high interior (j, j+1), j >= k    : target = row + delta_H, the same
//                                         delta for every row of the block;
//     cut (k-1, k)                      : target = row + C(k-1, w-1) or
//                                         row - C(k-1, w), per block;
//     wrap (L-1, 0)                     : target = R_{H ^ top} + rank(p ^ 1).
//   Low tables live in shared memory; per-block data in a tile header.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hs.h"

namespace hs {

constexpr int LMAX = 32;
constexpr int KLO_MAX = 10;            // low bits per state
constexpr int NB_MAX = KLO_MAX - 1;    // low interior bonds
constexpr int HD_MAX = LMAX - 3;       // high interior bonds (hb - 1 <= 29)
constexpr int TILE_G_MAX = 32;         // blocks per tile
constexpr int HV_THREADS = 256;
constexpr int RED_MAX_CTAS = 4096;     // partial-sum slots per reduction

// One entry per low pattern p, indexed by off[w] + r (class w, colex rank r).
struct LowEntry {
  uint32_t packed;   // pat (bits 0..15) | nb_cnt << 16 | code << 20 | tlow << 24
  uint16_t nb_off;   // first neighbour in the nb list
  uint16_t wrap_r;   // colex rank of p ^ 1 in its class
  float dlow_f;      // dlow rounded to FP32
  float pad;
};
// code = bit (k-1) of p | bit 0 of p << 1; tlow = sum of (j + 1) over set bits j < k.

__host__ __device__ inline uint32_t le_pat(uint32_t pk) { return pk & 0xFFFFu; }
__host__ __device__ inline int le_cnt(uint32_t pk) { return (pk >> 16) & 0xF; }
__host__ __device__ inline uint32_t le_code(uint32_t pk) { return (pk >> 20) & 0x3; }
__host__ __device__ inline uint32_t le_tlow(uint32_t pk) { return pk >> 24; }

// One entry per valid high pattern H (160 bytes; copied to shared memory as
// 40 words per tile block).
struct BlockInfo {
  uint32_t R;        // rank of the block's first row
  uint32_t Rwrap;    // first row of block H ^ top (only read when the wrap bond flips)
  int32_t bdelta;    // row offset of the cut-bond (k-1, k) flip
  uint32_t H;
  uint8_t w;         // low popcount
  uint8_t nh;        // antiparallel high interior bonds
  uint8_t code;      // bit 0 of H | top bit of H << 1
  uint8_t thigh;     // sum of (j + 1) over set high bits j >= k, mod L
  float dhs_f;       // shared-memory copy only: (float)(dhigh - sigma)
  double dhigh;      // Ising terms of high interior bonds + fields on high sites
  double dhs;        // shared-memory copy only: dhigh - sigma
  int32_t hd[HD_MAX];  // row offsets of the antiparallel high interior flips
  int32_t pad;
};
static_assert(sizeof(BlockInfo) % 8 == 0, "BlockInfo must be a whole number of words");

struct Tile {
  uint32_t b0;       // first block (index into the class-sorted block array)
  uint16_t G;        // blocks in the tile (all of class w)
  uint16_t w;
};

// Everything a row-loop kernel needs, passed by value.
struct Geo {
  const LowEntry* low;
  const uint16_t* nb;
  const double* dlow64;
  const BlockInfo* blocks;
  const Tile* tiles;
  int ntiles;
  int k, L, nlow, nnb;
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

struct Reduce {                      // last-CTA reduction scratch
  double* partial;                   // RED_MAX_CTAS * 4 doubles
  unsigned int* counter;             // one counter per pass kind
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
  std::vector<double> dlow64;
  std::vector<uint16_t> nb;
  std::vector<hs::BlockInfo> blocks;
  std::vector<hs::Tile> tiles;
  int cls_off[hs::KLO_MAX + 2] = {0};
  int cls_C[hs::KLO_MAX + 2] = {0};

  // device copies
  hs::LowEntry* d_low = nullptr;
  uint16_t* d_nb = nullptr;
  double* d_dlow64 = nullptr;
  hs::BlockInfo* d_blocks = nullptr;
  hs::Tile* d_tiles = nullptr;
  uint32_t* d_binom = nullptr;       // (LMAX + 1) x (LMAX / 2 + 2)
  double* d_sigma = nullptr;         // device copy of sigma
  int grid_hv = 0;                   // persistent grid of the row kernels

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
  int graph_iters = 0;

  // Lanczos workspace
  double* lz = nullptr; size_t lz_vectors = 0;

  hs::Geo geo() const;
};

namespace hs {

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
hs_status launch_unrank(hs_handle* hd, long long first, long long count, unsigned int* out);
hs_status launch_rank(hs_handle* hd, const unsigned int* st, long long count, long long* out);
hs_status launch_diag(hs_handle* hd, double* diag, hs_precond pc, double* minv);
// FP64 r = b - (H - sigma) x; returns sum r^2/M and sum r^2 and the same for b.
hs_status resid64(hs_handle* hd, const double* b, const double* x, double* r, hs_precond pc,
                  double sums_out[4]);

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
