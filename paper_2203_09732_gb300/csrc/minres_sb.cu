// Preconditioned MINRES of Algorithm 2 (Appendix A) for long chains, on the
// superblock layout (sb.cuh). One iteration is two launches:
//   pass A (k_sbhv, MINRES mode): the pending d/x update of iteration k - 1,
//          p = (H - sigma) q_k from a shared-memory tile per superblock pair,
//          alpha_k from a last-CTA reduction;
//   pass B (k_sbrows): q_{k+1} and beta_{k+1} with the preconditioner
//          recomputed per row, then the Givens rotation on the device.
// The scalars never leave the device; chunks of iterations are replayed from
// a captured CUDA graph, and the host reads the state once per replay to see
// whether the solve has finished. Same vectors and arithmetic as minres.cu.
#include <algorithm>
#include <cstdlib>

#include "common.cuh"
#include "minres_scalar.cuh"
#include "sb4_kern.cuh"
#include "sb_kern.cuh"

namespace hs {

namespace {

constexpr int NT_A = 512;   // pass A: as the product kernel
constexpr int NT_R = 512;   // init and pass B
constexpr int SB_CHUNK = 8; // iterations per graph replay

template <typename T>
auto kern_A(int km) {
  return km == 4 ? sb::k_sbhv<T, NT_A, 2, 4, sb::MODE_MINRES, 3>
                 : sb::k_sbhv<T, NT_A, 2, 4, sb::MODE_MINRES, 0>;
}
// pass A on the four-low-bit layout (sb4.cuh), where its plan applies
constexpr int NT_A4F = 512, NT_A4D = 256;
template <typename T>
constexpr int nt_a4() { return sizeof(T) == 8 ? NT_A4D : NT_A4F; }
template <typename T>
using KA4 = void (*)(sb4::Geo4, const T*, T*, const double*, int, sb::MinresArgs);
template <typename T>
KA4<T> kern_A4(int km) {
  if constexpr (sizeof(T) == 8) {
    if (km == 9) return sb4::k_sb4<T, nt_a4<T>(), 2, 4, sb::MODE_MINRES, 9>;
  } else {
    if (km == 10) return sb4::k_sb4<T, nt_a4<T>(), 2, 4, sb::MODE_MINRES, 10>;
  }
  return sb4::k_sb4<T, nt_a4<T>(), 2, 4, sb::MODE_MINRES, 0>;
}


template <typename T, int PC, int MODE>
auto kern_R() { return sb::k_sbrows<T, PC, MODE, NT_R>; }

// Grid of a kernel: resident CTAs per SM times the SMs this handle may use,
// at most one CTA per superblock pair and at most RED_MAX_CTAS partials.
template <typename K>
int grid_of(hs_handle* hd, K kern, int nt, size_t smem, int npairs) {
  int per_sm = 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int bud = hd->sm_budget.load(std::memory_order_relaxed);
  const int sms = bud > 0 ? std::min(bud, hd->num_sms) : hd->num_sms;
  return std::min(std::min(npairs, per_sm * sms), RED_MAX_CTAS);
}

template <typename T, int PC>
hs_status solve_t(hs_handle* hd, const T* b, const MinresVecs& v, double tol, long long kmax,
                  bool* used) {
  *used = false;
  const int ti = sizeof(T) == 8 ? 1 : 0;
  auto* d = static_cast<sb::DevPlan*>(hd->sb_plan[ti]);
  if (!d || !d->ok) return HS_OK;
  const sb::Geo& g = d->geo;
  auto* d4 = static_cast<sb4::DevPlan4*>(hd->sb4_plan[ti]);
  const bool use4 = hs_want_sb4(sizeof(T) == 8 ? HS_F64 : HS_F32) && d4 && d4->ok;
  const size_t smA = use4 ? d4->smem : d->smem;
  const size_t smR = sb::rows_smem_bytes<T>(1 << g.k);
  const int gA = use4 ? grid_of(hd, kern_A4<T>(d4->geo.km), nt_a4<T>(), smA, d4->geo.npairs)
                      : grid_of(hd, kern_A<T>(g.km), NT_A, smA, g.npairs);
  const int gI = grid_of(hd, kern_R<T, PC, sb::ROWS_INIT>(), NT_R, smR, g.npairs);
  const int gB = grid_of(hd, kern_R<T, PC, sb::ROWS_B>(), NT_R, smR, g.npairs);
  if (gA < 1 || gI < 1 || gB < 1) return HS_OK;
  *used = true;
  sb::MinresArgs ma;
  ma.v = v;
  ma.st = hd->d_state;
  ma.partial = hd->d_partial;
  // initial pass: q_1 = M^-1 b, beta_1, state
  ma.counter = hd->d_counter + 0;
  kern_R<T, PC, sb::ROWS_INIT>()<<<gI, NT_R, smR, hd->stream>>>(g, b, ma, tol, kmax, hd->d_sigma);
  count_launches(1);
  HS_CUDA_TRY(hd, cudaGetLastError());
  // the chunk graph, cached per (precision, preconditioner) for these grids
  // and this workspace
  cudaGraphExec_t& exec = hd->sbgraph[ti][PC];
  int* key = hd->sbgraph_key[ti][PC];
  const int keyA = gA | (use4 ? 1 << 30 : 0);
  if (exec && (key[0] != keyA || key[1] != gB || hd->sbgraph_ws[ti] != v.q0)) {
    cudaGraphExecDestroy(exec);
    exec = nullptr;
  }
  if (!exec) {
    cudaStream_t cs;
    HS_CUDA_TRY(hd, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      sb::MinresArgs mA = ma, mB = ma;
      mA.counter = hd->d_counter + 1;
      mB.counter = hd->d_counter + 2;
      for (int it = 0; it < SB_CHUNK; ++it) {
        if (use4)
          kern_A4<T>(d4->geo.km)<<<gA, nt_a4<T>(), smA, cs>>>(d4->geo, nullptr, nullptr,
                                                              hd->d_sigma, 1, mA);
        else
          kern_A<T>(g.km)<<<gA, NT_A, smA, cs>>>(g, nullptr, nullptr, hd->d_sigma, 1, mA);
        kern_R<T, PC, sb::ROWS_B>()<<<gB, NT_R, smR, cs>>>(g, nullptr, mB, 0.0, 0, hd->d_sigma);
      }
      e = cudaStreamEndCapture(cs, &graph);
    }
    if (e == cudaSuccess) {
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      exec = nullptr;
      return fail(hd, HS_CUDA, std::string("superblock MINRES graph: ") + cudaGetErrorString(e));
    }
    key[0] = keyA;
    key[1] = gB;
    hd->sbgraph_ws[ti] = v.q0;
  }
  int between = 1;
  while (true) {
    for (int j = 0; j < between; ++j) {
      HS_CUDA_TRY(hd, cudaGraphLaunch(exec, hd->stream));
      count_launches(2ull * SB_CHUNK);
    }
    HS_CUDA_TRY(hd, cudaMemcpyAsync(hd->h_state, hd->d_state, sizeof(MinresState),
                                    cudaMemcpyDeviceToHost, hd->stream));
    HS_CUDA_TRY(hd, cudaStreamSynchronize(hd->stream));
    const MinresState& S = *hd->h_state;
    if (S.done == 2) break;
    between = S.done == 1 ? 1 : std::min(between * 2, 8);
  }
  return HS_OK;
}

}  // namespace

hs_status minres_solve_sb(hs_handle* hd, const void* b, const MinresVecs& v, hs_dtype dt,
                          int pc, double tol, long long kmax, bool* used) {
  if (dt == HS_F32) {
    const float* bf = static_cast<const float*>(b);
    switch (pc) {
      case 0: return solve_t<float, 0>(hd, bf, v, tol, kmax, used);
      case 1: return solve_t<float, 1>(hd, bf, v, tol, kmax, used);
      default: return solve_t<float, 2>(hd, bf, v, tol, kmax, used);
    }
  }
  const double* bd = static_cast<const double*>(b);
  switch (pc) {
    case 0: return solve_t<double, 0>(hd, bd, v, tol, kmax, used);
    case 1: return solve_t<double, 1>(hd, bd, v, tol, kmax, used);
    default: return solve_t<double, 2>(hd, bd, v, tol, kmax, used);
  }
}

void sb_graphs_release(hs_handle* hd, int ti) {
  for (int pc = 0; pc < 3; ++pc)
    if (hd->sbgraph[ti][pc]) {
      cudaGraphExecDestroy(hd->sbgraph[ti][pc]);
      hd->sbgraph[ti][pc] = nullptr;
    }
  hd->sbgraph_ws[ti] = nullptr;
}

}  // namespace hs
