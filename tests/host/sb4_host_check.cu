// Host check of the four-low-bit superblock product (test infrastructure).
//
// Runs the kernel's own code from sb4.cuh on the CPU: the plan (build_plan4),
// the flat-row -> slot copies, the whole-superblock sums (sb_phase1) and the
// per-lane row code (sb4_rows_any), pair by pair in the kernel's order. Every
// slot element that the copies do not fill, G and the guard regions around x
// hold NaN, so that a read of anything not staged shows up in y; a wrong
// neighbour or diagonal term shows up against the oracle's explicit H. Usage:
//   sb4_host_check L KS sigma dir
// reads dir/h.bin (L doubles) and dir/x.bin (n doubles), writes dir/y64.bin and
// dir/y32.bin (the FP32 result widened).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_2203_09732_gb300/csrc/sb4.cuh"

using namespace hs;
using namespace hs::sb4;

template <typename T>
static void run(const HostPlan4& P, const T* x, T* y, double sigma) {
  const sb::HostPlan& B = P.base;
  const int km = B.km, nsl = 1 << km, AE = arr_elems(km);
  std::vector<T> X(4 * (size_t)AE), G(2 * (size_t)P.cmax);
  const std::vector<T> dl = [&] {
    std::vector<T> v(P.dl_d.size());
    for (size_t i = 0; i < v.size(); ++i) v[i] = sizeof(T) == 8 ? (T)P.dl_d[i] : (T)P.dl_f[i];
    return v;
  }();
  const int NT = 96;  // emulated threads of phase 1 (any count)
  for (const int2 pr : B.pairs) {
    sb::Sup sh[2];
    sh[0] = pr.x >= 0 ? B.sup[pr.x] : sb::Sup{};
    sh[1] = pr.y >= 0 ? B.sup[pr.y] : sb::Sup{};
    for (T& v : X) v = (T)NAN;
    for (int a = 0; a < 4; ++a)
      for (int e = 0; e < ZERO_ENT * 4; ++e) X[(size_t)a * AE + nsl * 4 + e] = T(0);
    for (T& v : G) v = (T)NAN;
    T uT[4];
    for (int t = 0; t < 4; ++t) {
      const int s = t >> 1;
      const uint32_t tb0 = (sh[s].meta >> 16) & 1u;
      uT[t] = (T)(sh[s].dT - sigma + (((uint32_t)(t & 1) == tb0) ? 0.25 : -0.25));
    }
    for (int s = 0; s < 2; ++s) {
      if (!sh[s].C) continue;
      const int wq = (int)(sh[s].meta & 0xFF);
      const uint16_t* map = P.slotmap.data() + P.slot_off[wq];
      for (uint32_t i = 0; i < sh[s].C; ++i) X[(size_t)s * AE + map[i]] = x[sh[s].R + i];
      for (int t = 0; t < NT; ++t)
        sb4_phase1<T, 4>(x + sh[s].R, sh[s], G.data() + (size_t)s * P.cmax, t, NT);
    }
    const int nv0 = sh[0].C ? P.nvalid[sh[0].meta & 0xFF] : 0;
    const int nv1 = sh[1].C ? P.nvalid[sh[1].meta & 0xFF] : 0;
    for (int u = 0; u < nv0 + nv1; ++u) {
      const int s = u >= nv0 ? 1 : 0;
      const int i = s ? u - nv0 : u;
      const sb::Sup& H = sh[s];
      const uint32_t hm = H.meta;
      const int wq = (int)(hm & 0xFF);
      const int m = P.order[P.order_off[wq] + i];
      const int w = wq - sb::popc_host((uint32_t)m);
      const int lo = P.lo[((size_t)wq << km) + m];
      LaneIn in;
      in.m = m;
      in.b0 = (uint32_t)m & 1u;
      in.top = (hm >> 17) & 1u;
      in.km = km;
      const T dm = sizeof(T) == 8 ? (T)P.dmid_d[m] : (T)P.dmid_f[m];
      const T uu = dm + uT[s * 2 + ((m >> (km - 1)) & 1)];
      const T* xp = sh[1 - s].C ? X.data() + (size_t)(1 - s) * AE : nullptr;
      const T* dlw = dl.data() + (((int)in.top * 2 + (int)in.b0) * 5 + w) * SLOT;
      // the run-time mid loop and, for the library's windows, the unrolled one
      T* gs = G.data() + (size_t)s * P.cmax + lo;
      if (km == 10) sb4_rows_any<T, 10>(w, in, X.data() + (size_t)s * AE, xp, gs, dlw, uu);
      else if (km == 9) sb4_rows_any<T, 9>(w, in, X.data() + (size_t)s * AE, xp, gs, dlw, uu);
      else sb4_rows_any<T, 0>(w, in, X.data() + (size_t)s * AE, xp, gs, dlw, uu);
    }
    for (int s = 0; s < 2; ++s)
      for (uint32_t i = 0; i < sh[s].C; ++i) y[sh[s].R + i] = G[(size_t)s * P.cmax + i];
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
  if (argc != 5) {
    fprintf(stderr, "usage: sb4_host_check L KS sigma dir\n");
    return 2;
  }
  const int L = atoi(argv[1]), KS = atoi(argv[2]);
  const double sigma = atof(argv[3]);
  const char* dir = argv[4];
  char fn[1024];
  std::vector<double> h(L);
  snprintf(fn, sizeof fn, "%s/h.bin", dir);
  if (!read_all(fn, h.data(), sizeof(double) * L)) return 3;
  HostPlan4 P;
  if (!build_plan4(L, h.data(), KS, &P)) {
    printf("plan does not apply\n");
    return 4;
  }
  const size_t n = (size_t)sb::binom64(L, L / 2);
  std::vector<double> xs(n);
  snprintf(fn, sizeof fn, "%s/x.bin", dir);
  if (!read_all(fn, xs.data(), sizeof(double) * n)) return 3;
  const size_t guard = 1 << 20;
  std::vector<double> xb(n + 2 * guard, NAN), yb(n + 2 * guard, NAN);
  for (size_t i = 0; i < n; ++i) xb[guard + i] = xs[i];
  run<double>(P, xb.data() + guard, yb.data() + guard, sigma);
  snprintf(fn, sizeof fn, "%s/y64.bin", dir);
  if (!write_all(fn, yb.data() + guard, sizeof(double) * n)) return 5;
  std::vector<float> xf(n + 2 * guard, NAN), yf(n + 2 * guard, NAN);
  for (size_t i = 0; i < n; ++i) xf[guard + i] = (float)xs[i];
  run<float>(P, xf.data() + guard, yf.data() + guard, sigma);
  std::vector<double> y32(n);
  for (size_t i = 0; i < n; ++i) y32[i] = yf[guard + i];
  snprintf(fn, sizeof fn, "%s/y32.bin", dir);
  if (!write_all(fn, y32.data(), sizeof(double) * n)) return 5;
  printf("ok n=%zu pairs=%zu cmax=%d\n", n, P.base.pairs.size(), P.cmax);
  return 0;
}
