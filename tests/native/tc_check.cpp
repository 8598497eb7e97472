// Host check of the tensor-core tangent assembly of the spring kernel (csrc/k_spring.cu):
// the digits of the spring tables in MMA fragment order (host_spring_digits), the balanced
// digits the kernel cuts from a tangent pair (the same single-precision operations, IEEE,
// no contraction), the per-pair sums the MMAs accumulate (computed here exactly, in
// integers), the warps' double-float partial sums and their combination in the kernel's
// order -- against sum_k G_k T_k[ij] in long double.
// Prints: worst error relative to sum_k |G_k T_k[ij]|, largest per-pair sum over 2^24 (the
// bound below which FP32 holds every partial sum exactly), layout mismatches, worst digit
// error of T, worst digit error of G (relative to 2^eG), largest |digit| of G.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "../../paper_2604_02755_gb300/csrc/df64.cuh"

// the CUDA vector type of the library's signature (its mangled name is all that links)
struct uint2 {
  uint32_t x, y;
};

namespace ns {
int host_spring_directions(int S, double *q, double *w);
void host_spring_digits(int S, const double *T, uint2 *frag, int *et);
}  // namespace ns
using namespace ns;

static float bf16_to_float(uint32_t h) {
  const uint32_t b = h << 16;
  float f;
  memcpy(&f, &b, 4);
  return f;
}

static int sym6(int i, int j) {  // packed upper triangle, row by row
  if (i > j) std::swap(i, j);
  return i * 6 - i * (i - 1) / 2 + (j - i);
}

// the kernel's digit pairs (i + j <= 7, level by level) and its warp count
static const int kDig = 7, kMaxL = 7, kWarps = 8;

int main(int argc, char **argv) {
  const int S = argc > 1 ? atoi(argv[1]) : 150;
  const int npts = argc > 2 ? atoi(argv[2]) : 2000;
  std::vector<double> q(6 * S), T(21 * (size_t)S);
  double w = 0;
  if (host_spring_directions(S, q.data(), &w)) return 2;
  for (int k = 0; k < S; ++k)
    for (int i = 0; i < 6; ++i)
      for (int j = i; j < 6; ++j) T[21 * (size_t)k + sym6(i, j)] = w * q[6 * k + i] * q[6 * k + j];
  const int KS = (S + 15) / 16;
  std::vector<uint2> frag((size_t)kDig * KS * 3 * 32);
  int et[21];
  host_spring_digits(S, T.data(), frag.data(), et);
  // decode the fragments back into digits b[j][k][n]; every (k, n) must be written once
  std::vector<int> b((size_t)kDig * 16 * KS * 24, 0), seen((size_t)kDig * 16 * KS * 24, 0);
  long mismatches = 0;
  for (int j = 0; j < kDig; ++j)
    for (int ks = 0; ks < KS; ++ks)
      for (int nt = 0; nt < 3; ++nt)
        for (int lane = 0; lane < 32; ++lane) {
          const uint2 v = frag[(((size_t)j * KS + ks) * 3 + nt) * 32 + lane];
          const int n = 8 * nt + lane / 4, k0 = 16 * ks + 2 * (lane % 4);
          const int ks4[4] = {k0, k0 + 1, k0 + 8, k0 + 9};
          const uint32_t hs[4] = {v.x & 0xFFFF, v.x >> 16, v.y & 0xFFFF, v.y >> 16};
          for (int e = 0; e < 4; ++e) {
            const size_t at = ((size_t)j * 16 * KS + ks4[e]) * 24 + n;
            b[at] = (int)bf16_to_float(hs[e]);
            seen[at]++;
          }
        }
  for (size_t i = 0; i < seen.size(); ++i) mismatches += seen[i] != 1;
  double worst_t = 0.0;  // digits of T against T (relative to 2^eT)
  for (int k = 0; k < 16 * KS; ++k)
    for (int n = 0; n < 24; ++n) {
      long double r = 0.0L;
      for (int j = 0; j < kDig; ++j) r += ldexpl((long double)b[((size_t)j * 16 * KS + k) * 24 + n], -7 * (j + 1));
      const long double ref = (k < S && n < 21) ? ldexpl((long double)T[21 * (size_t)k + n], -et[n]) : 0.0L;
      worst_t = fmax(worst_t, (double)fabsl(r - ref));
      if (!(k < S && n < 21) && r != 0.0L) mismatches++;
    }
  int pi[64], pj[64], np = 0;
  for (int L = 0; L <= kMaxL; ++L)
    for (int i = 0; i <= L; ++i)
      if (i < kDig && L - i < kDig) {
        pi[np] = i;
        pj[np] = L - i;
        ++np;
      }
  // tangents of random points: G in [1e-4, 1] G0, as float pairs
  std::mt19937_64 rng(5);
  std::uniform_real_distribution<double> U(0.0, 1.0);
  double worst = 0.0, cmax = 0.0, worst_g = 0.0;
  int amax = 0;
  for (int p = 0; p < npts; ++p) {
    const double G0 = 1.0e6 * exp(8.0 * U(rng));
    const int eg = ilogb(G0) + 1;
    const float gfix = ldexpf(1.0f, 49 - eg);
    std::vector<int> a((size_t)kDig * S);
    std::vector<long double> G(S);
    for (int k = 0; k < S; ++k) {
      const double g = G0 * exp(-9.2 * U(rng));
      const float gh = (float)g, gl = (float)(g - (double)gh);
      G[k] = (long double)gh + (long double)gl;
      // the kernel's balanced digits (tangent_digits)
      float r = df_mul(gh, gfix);
      const float c = rintf(df_mul(gl, gfix));
      long double rep = 0.0L;
      for (int i = 0; i < kDig; ++i) {
        const float wv = ldexpf(1.0f, -(42 - 7 * i)), W = ldexpf(1.0f, 42 - 7 * i);
        const float v = df_mul(df_add(r, c), wv);
        const float d = df_sub(df_add(v, 12582912.0f), 12582912.0f);
        r = df_fma(-d, W, r);
        const float db = bf16_to_float(df_bits(d) >> 16);
        if (db != d) mismatches++;  // a digit that bf16 does not hold exactly
        a[(size_t)i * S + k] = (int)d;
        amax = std::max(amax, std::abs((int)d));
        rep += ldexpl((long double)d, -7 * (i + 1));
      }
      worst_g = fmax(worst_g, (double)fabsl(rep - ldexpl(G[k], -eg)));
    }
    for (int n = 0; n < 21; ++n) {
      long double ref = 0.0L, mag = 0.0L;
      for (int k = 0; k < S; ++k) {
        ref += G[k] * (long double)T[21 * (size_t)k + n];
        mag += fabsl(G[k] * (long double)T[21 * (size_t)k + n]);
      }
      // warp w: pairs w, w + 8, ...; each pair's exact integer sum scaled by 2^-7(i+j) and
      // added into the warp's pair sum; then the warps' sums in order
      float sh = 0.0f, sl = 0.0f;
      for (int wp = 0; wp < kWarps; ++wp) {
        float vh = 0.0f, vl = 0.0f;
        for (int pr = wp; pr < np; pr += kWarps) {
          long long C = 0;
          for (int k = 0; k < S; ++k)
            C += (long long)a[(size_t)pi[pr] * S + k] * b[((size_t)pj[pr] * 16 * KS + k) * 24 + n];
          cmax = fmax(cmax, fabs((double)C) / 16777216.0);
          float s, e;
          two_sum(vh, df_mul((float)C, ldexpf(1.0f, -7 * (pi[pr] + pj[pr]))), s, e);
          vh = s;
          vl = df_add(vl, e);
        }
        float t, e;
        two_sum(sh, vh, t, e);
        sh = t;
        sl = df_add(sl, df_add(e, vl));
      }
      const long double D = ldexpl((long double)sh + (long double)sl, eg + et[n] - 14);
      if (mag > 0) worst = fmax(worst, (double)(fabsl(D - ref) / mag));
    }
  }
  printf("%.3e %.4f %ld %.3e %.3e %d\n", worst, cmax, mismatches, worst_t, worst_g, amax);
  return 0;
}
