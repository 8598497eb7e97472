// Accuracy of the double-float power (paper_2604_02755_gb300/csrc/df64.cuh) run on the
// host with the library's own tables, against long-double powl.  IEEE single-precision
// arithmetic gives the same results on the CPU as on the GPU when multiply-adds are not
// contracted (-ffp-contract=off) and fma is the fused operation.
// Prints: worst relative error of x^beta, worst error weighted as it enters the spring's
// stress and tangent ((1 + beta) alpha w / (1 + (1 + beta) alpha w), alpha = 2^beta), and
// the count of inputs the routine declined.
#include <cmath>
#include <cstdio>
#include <random>

#include "../../paper_2604_02755_gb300/csrc/df64.cuh"

namespace ns {
void host_powf_tables(float *out);
}
using namespace ns;

int main(int argc, char **argv) {
  const double lx0 = argc > 1 ? atof(argv[1]) : -18.4, lx1 = argc > 2 ? atof(argv[2]) : 5.3;
  const int n = argc > 3 ? atoi(argv[3]) : 1000000;
  static float tab[kPowFLen];
  host_powf_tables(tab);
  std::mt19937_64 rng(11);
  std::uniform_real_distribution<double> U(0.0, 1.0);
  double worst = 0.0, worst_w = 0.0;
  int declined = 0;
  for (int it = 0; it < n; ++it) {
    const double lx = lx0 + (lx1 - lx0) * U(rng);
    const long double b = 0.5L + 1.3L * (long double)U(rng);
    const float t = (float)exp(0.5 * lx);  // an FP32 seed
    const double itref = exp(0.5 * lx) * (1.0 + 1e-3 * U(rng));
    const float ih = (float)itref, il = (float)(itref - (double)ih);
    PowBeta B;
    B.bh = (float)b;
    B.bl = (float)(b - (long double)B.bh);
    const long double b0 = roundl(b * 32768.0L) / 32768.0L, b1 = roundl((b - b0) * 2147483648.0L) / 2147483648.0L;
    B.b0 = (float)b0;
    B.b1 = (float)b1;
    B.b2 = (float)(b - b0 - b1);
    float xh, xl, wh, wl;
    two_prod(t, ih, xh, xl);
    xl = df_fma(t, il, xl);
    if (!df64_pow(xh, xl, B, tab, wh, wl)) {
      ++declined;
      continue;
    }
    const long double x = (long double)t * ((long double)ih + (long double)il);
    const long double ref = powl(x, b), got = (long double)wh + (long double)wl;
    const double rel = (double)fabsl(got / ref - 1.0L);
    const long double aw = powl(2.0L, b) * ref;
    const double relw = rel * (double)((1.0L + b) * aw / (1.0L + (1.0L + b) * aw));
    if (rel > worst) worst = rel;
    if (relw > worst_w) worst_w = relw;
  }
  printf("%.6e %.6e %d\n", worst, worst_w, declined);
  return 0;
}
