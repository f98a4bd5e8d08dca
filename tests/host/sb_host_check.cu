// Host check of the superblock H x arithmetic (test infrastructure).
//
// Runs the per-row code of the superblock kernel on the CPU: the same plan
// tables (build_plan), the same staging (sb_stage), sums (sb_phase1) and row
// pass (sb_lane) from sb.cuh, driven in the kernel's order over every pair.
// The staged buffers and the guard regions around x hold NaN, so that a read
// of anything not staged shows up in y. Usage:
//   sb_host_check L k KS sigma shift dir
// reads dir/h.bin (L doubles) and dir/x.bin (n doubles), writes dir/y64.bin
// and dir/y32.bin (n doubles each; the FP32 result widened), and the
// preconditioner entries of the MINRES row passes: dir/mrow.bin (row norm),
// dir/mjac.bin (Jacobi), dir/mrow32.bin (row norm in FP32, widened). shift
// offsets x and y by that many elements from a 16-byte boundary.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_2203_09732_gb300/csrc/sb.cuh"

using namespace hs::sb;

template <typename T>
static void run(const HostPlan& P, const T* x, T* y, double sigma) {
  const int nsl = 1 << P.km;
  std::vector<T> tile(tile_elems(P.km), (T)NAN);
  std::vector<T> G(2 * nsl * SL, (T)NAN);
  T* zslot = tile.data() + 2 * nsl * SL;
  for (int i = 0; i < SL; ++i) zslot[i] = T(0);
  Geo g{};
  g.order = P.order.data();
  g.sub = P.sub.data();
  g.km = P.km;
  for (int i = 0; i < K_MAX + 2; ++i) g.cls_C[i] = P.cls_C[i];
  for (int i = 0; i <= WQ_MAX; ++i) g.nvalid[i] = P.nvalid[i];
  const int NW = 5, NT = 96;  // emulated warps and threads (any counts)
  Sup sh[2];
  for (const int2 pr : P.pairs) {
    sh[0] = pr.x >= 0 ? P.sup[pr.x] : Sup{};
    sh[1] = pr.y >= 0 ? P.sup[pr.y] : Sup{};
    for (int i = 0; i < 2 * nsl * SL; ++i) tile[i] = (i % SL == ZSLOT) ? T(0) : (T)NAN;
    for (T& v : G) v = (T)NAN;
    for (int s = 0; s < 2; ++s) {
      if (!sh[s].C) continue;
      for (int w = 0; w < NW; ++w)
        for (int lane = 0; lane < 32; ++lane)
          sb_stage<T>(x + sh[s].R, g, (int)(sh[s].meta & 0xFF), tile.data() + s * nsl * SL, w, NW,
                      lane);
      for (int t = 0; t < NT; ++t)
        sb_phase1<T, 4>(x + sh[s].R, sh[s], G.data() + s * nsl * SL, t, NT);
    }
    const int nv0 = sh[0].C ? P.nvalid[sh[0].meta & 0xFF] : 0;
    const int nv1 = sh[1].C ? P.nvalid[sh[1].meta & 0xFF] : 0;
    for (int u = 0; u < nv0 + nv1; ++u) {
      const int s = u >= nv0 ? 1 : 0;
      const int i = s ? u - nv0 : u;
      const Sup& H = sh[s];
      const uint32_t hm = H.meta;
      const int wq = (int)(hm & 0xFF);
      const int m = P.order[(wq << P.km) + i];
      const Sub& B = P.sub[(wq << P.km) + m];
      const uint32_t bm = B.meta;
      const int w = (int)(bm & 0xFF);
      const int nmd = (int)((bm >> 8) & 0xFF);
      Lane<T> c;
      c.low = P.low.data() + P.cls_off[w];
      c.dlow = P.dlow.data() + P.cls_off[w];
      c.tl = tile.data() + (s * nsl + m) * SL;
      c.tg = G.data() + s * nsl * SL + B.lo;
      c.tp = tile.data() + ((1 - s) * nsl + m) * SL;
      c.yg = y + H.R + B.lo;
      c.zoff = (int32_t)(zslot - c.tl);
      for (int q = 0; q < MD_MAX; ++q) c.md[q] = q < nmd ? B.md[q] : c.zoff;
      c.nmid = P.km - 1;
      c.C = P.cls_C[w];
      c.bdelta = B.bdelta;
      c.mbit0 = (bm >> 16) & 1u;
      c.ttop = (hm >> 17) & 1u;
      const uint32_t anti_ks = ((bm >> 17) & 1u) ^ ((hm >> 16) & 1u);
      c.uni = (T)(B.dmid + H.dT - sigma + (anti_ks ? -0.25 : 0.25));
      for (int lane = 0; lane < 32; ++lane) sb_lane<T>(c, lane);
    }
  }
}

// The preconditioner entries of the MINRES row passes (k_sbrows): per row,
// a_ii - sigma and the antiparallel-bond count from RowCtx / sb_diag, then
// M_ii from sb_precond, in the kernel's order over pairs and sub-blocks.
template <typename T, int PC>
static void precond_rows(const HostPlan& P, T* out, double sigma) {
  for (const int2 pr : P.pairs) {
    for (int s = 0; s < 2; ++s) {
      const int id = s ? pr.y : pr.x;
      if (id < 0) continue;
      const Sup& H = P.sup[id];
      const uint32_t hm = H.meta;
      const int wq = (int)(hm & 0xFF);
      for (int i = 0; i < P.nvalid[wq]; ++i) {
        const int m = P.order[(wq << P.km) + i];
        const Sub& B = P.sub[(wq << P.km) + m];
        const uint32_t bm = B.meta;
        const int w = (int)(bm & 0xFF);
        RowCtx<T> c;
        c.low = P.low.data() + P.cls_off[w];
        c.dlow = P.dlow.data() + P.cls_off[w];
        c.mbit0 = (bm >> 16) & 1u;
        c.ttop = (hm >> 17) & 1u;
        const uint32_t anti_ks = ((bm >> 17) & 1u) ^ ((hm >> 16) & 1u);
        c.nfix = (int)((bm >> 8) & 0xFF) + (int)anti_ks + (int)((hm >> 8) & 0xFF);
        c.uni = (T)(B.dmid + H.dT - sigma + (anti_ks ? -0.25 : 0.25));
        c.C = P.cls_C[w];
        for (int r = 0; r < c.C; ++r) {
          int naf;
          const T am = sb_diag<T>(c, r, naf);
          out[H.R + B.lo + r] = sb_precond<PC, T>(am, naf);
        }
      }
    }
  }
}

static bool read_all(const char* fn, void* p, size_t bytes) {
  FILE* f = fopen(fn, "rb");
  if (!f) return false;
  const size_t got = fread(p, 1, bytes, f);
  fclose(f);
  return got == bytes;
}

static bool write_all(const char* fn, const void* p, size_t bytes) {
  FILE* f = fopen(fn, "wb");
  if (!f) return false;
  const size_t put = fwrite(p, 1, bytes, f);
  fclose(f);
  return put == bytes;
}

int main(int argc, char** argv) {
  if (argc != 7) {
    fprintf(stderr, "usage: sb_host_check L k KS sigma shift dir\n");
    return 2;
  }
  const int L = atoi(argv[1]), k = atoi(argv[2]), KS = atoi(argv[3]);
  const double sigma = atof(argv[4]);
  const int shift = atoi(argv[5]);
  const char* dir = argv[6];
  char fn[1024];
  std::vector<double> h(L);
  snprintf(fn, sizeof fn, "%s/h.bin", dir);
  if (!read_all(fn, h.data(), sizeof(double) * L)) return 3;
  HostPlan P;
  if (!build_plan(L, h.data(), k, KS, &P)) {
    printf("plan does not apply\n");
    return 4;
  }
  const size_t n = (size_t)binom64(L, L / 2);
  std::vector<double> xs(n);
  snprintf(fn, sizeof fn, "%s/x.bin", dir);
  if (!read_all(fn, xs.data(), sizeof(double) * n)) return 3;
  const size_t guard = 4096;
  std::vector<double> xb(n + 2 * guard + 8, NAN), yb(n + 2 * guard + 8, NAN);
  double* x = xb.data() + guard + shift;
  double* y = yb.data() + guard + shift;
  for (size_t i = 0; i < n; ++i) x[i] = xs[i];
  run<double>(P, x, y, sigma);
  snprintf(fn, sizeof fn, "%s/y64.bin", dir);
  if (!write_all(fn, y, sizeof(double) * n)) return 5;
  std::vector<float> xf(n + 2 * guard + 8, NAN), yf(n + 2 * guard + 8, NAN);
  float* x4 = xf.data() + guard + shift;
  float* y4 = yf.data() + guard + shift;
  for (size_t i = 0; i < n; ++i) x4[i] = (float)xs[i];
  run<float>(P, x4, y4, sigma);
  std::vector<double> y32(n);
  for (size_t i = 0; i < n; ++i) y32[i] = y4[i];
  snprintf(fn, sizeof fn, "%s/y32.bin", dir);
  if (!write_all(fn, y32.data(), sizeof(double) * n)) return 5;
  // preconditioner entries (row norm and Jacobi, FP64 and FP32 widened)
  std::vector<double> mr(n, NAN), mj(n, NAN), m32(n, NAN);
  std::vector<float> mf(n, NAN);
  precond_rows<double, 2>(P, mr.data(), sigma);
  precond_rows<double, 1>(P, mj.data(), sigma);
  precond_rows<float, 2>(P, mf.data(), sigma);
  for (size_t i = 0; i < n; ++i) m32[i] = mf[i];
  snprintf(fn, sizeof fn, "%s/mrow.bin", dir);
  if (!write_all(fn, mr.data(), sizeof(double) * n)) return 5;
  snprintf(fn, sizeof fn, "%s/mjac.bin", dir);
  if (!write_all(fn, mj.data(), sizeof(double) * n)) return 5;
  snprintf(fn, sizeof fn, "%s/mrow32.bin", dir);
  if (!write_all(fn, m32.data(), sizeof(double) * n)) return 5;
  printf("ok n=%zu pairs=%zu\n", n, P.pairs.size());
  return 0;
}
