// Host check of the tensor-core tangent assembly of the spring kernel (csrc/k_spring.cu):
// the digits of the spring tables in MMA fragment order (host_spring_digits), the digits
// the kernel cuts from a tangent pair, the level sums the MMAs accumulate (computed here
// exactly, in integers) and the double-float recombination -- against
// sum_k G_k T_k[ij] in long double.  Single-precision operations are IEEE on both sides
// (no contraction); __float2ull_rz / __float2ll_rn are truncation / round-to-nearest.
// Prints: worst error relative to sum_k |G_k T_k[ij]|, largest level sum over 2^23 (the
// exactness bound of the FP32 accumulators), layout mismatches, worst digit error of T.
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
  std::vector<uint2> frag((size_t)8 * KS * 3 * 32);
  int et[21];
  host_spring_digits(S, T.data(), frag.data(), et);
  // decode the fragments back into digits b[j][k][n]; every (k, n) must be written once
  std::vector<int> b((size_t)8 * 16 * KS * 24, 0), seen((size_t)8 * 16 * KS * 24, 0);
  long mismatches = 0;
  for (int j = 0; j < 8; ++j)
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
      for (int j = 0; j < 8; ++j) r += ldexpl((long double)b[((size_t)j * 16 * KS + k) * 24 + n], -6 * (j + 1));
      const long double ref = (k < S && n < 21) ? ldexpl((long double)T[21 * (size_t)k + n], -et[n]) : 0.0L;
      worst_t = fmax(worst_t, (double)fabsl(r - ref));
      if (!(k < S && n < 21) && r != 0.0L) mismatches++;
    }
  // tangents of random points: G in [1e-4, 1] G0, as float pairs
  std::mt19937_64 rng(5);
  std::uniform_real_distribution<double> U(0.0, 1.0);
  double worst = 0.0, cmax = 0.0;
  for (int p = 0; p < npts; ++p) {
    const double G0 = 1.0e6 * exp(8.0 * U(rng));
    const int eg = ilogb(G0) + 1;
    const float gfix = ldexpf(1.0f, 48 - eg);
    std::vector<int> a((size_t)8 * S);
    std::vector<long double> G(S);
    for (int k = 0; k < S; ++k) {
      const double g = G0 * exp(-9.2 * U(rng));
      const float gh = (float)g, gl = (float)(g - (double)gh);
      G[k] = (long double)gh + (long double)gl;
      const float xh = df_mul(gh, gfix), xl = df_mul(gl, gfix);
      long long X = (long long)(unsigned long long)truncf(xh) + (long long)llrintf(xl);
      X = X < 0 ? 0 : (X > 0xFFFFFFFFFFFFll ? 0xFFFFFFFFFFFFll : X);
      for (int i = 0; i < 8; ++i) a[(size_t)i * S + k] = (int)(((unsigned long long)X >> (42 - 6 * i)) & 63u);
    }
    for (int n = 0; n < 21; ++n) {
      long double ref = 0.0L, mag = 0.0L;
      for (int k = 0; k < S; ++k) {
        ref += G[k] * (long double)T[21 * (size_t)k + n];
        mag += fabsl(G[k] * (long double)T[21 * (size_t)k + n]);
      }
      float vh = 0.0f, vl = 0.0f;
      for (int L = 8; L >= 0; --L) {
        long long C = 0;
        for (int i = L < 8 ? 0 : L - 7; i <= L && i < 8; ++i)
          for (int k = 0; k < S; ++k)
            C += (long long)a[(size_t)i * S + k] * b[((size_t)(L - i) * 16 * KS + k) * 24 + n];
        cmax = fmax(cmax, fabs((double)C) / 8388608.0);
        float s, e;
        two_sum((float)C, df_mul(vh, 0.015625f), s, e);
        two_sum(s, df_add(e, df_mul(vl, 0.015625f)), vh, vl);
      }
      const long double D = ldexpl((long double)vh + (long double)vl, eg + et[n] - 12);
      if (mag > 0) worst = fmax(worst, (double)(fabsl(D - ref) / mag));
    }
  }
  printf("%.3e %.4f %ld %.3e\n", worst, cmax, mismatches, worst_t);
  return 0;
}
