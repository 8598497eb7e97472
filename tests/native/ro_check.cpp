// One double-float Halley step of the spring law's skeleton root (csrc/df64.cuh,
// df64_ro_halley) from an FP32 Newton seed, run on the host with the library's tables,
// against the root and tangent solved in long double.  Prints the worst relative errors of
// the root and of the tangent, the worst relative step |d|, and the count of declined inputs.
#include <cmath>
#include <cstdio>
#include <random>

#include "../../paper_2604_02755_gb300/csrc/df64.cuh"

namespace ns {
void host_powf_tables(float *out);
}
using namespace ns;

static void split(long double v, float &h, float &l) {
  h = (float)v;
  l = (float)(v - (long double)h);
}

int main(int argc, char **argv) {
  const int n = argc > 1 ? atoi(argv[1]) : 200000;
  const float stop = argc > 2 ? (float)atof(argv[2]) : 1e-3f;  // the seed's stopping step
  static float tab[kPowFLen];
  host_powf_tables(tab);
  std::mt19937_64 rng(5);
  std::uniform_real_distribution<double> U(0.0, 1.0);
  double wt = 0.0, wg = 0.0, wd = 0.0;
  int declined = 0;
  for (int it = 0; it < n; ++it) {
    const long double rho = 1600 + 500 * U(rng), vs = 100 + 600 * U(rng);
    const long double G0 = rho * vs * vs, gref = powl(10.0L, -4.0L + 2.3L * U(rng));
    const long double hmax = 0.05L + 0.25L * U(rng);
    const long double beta = 2 * M_PI * hmax / (2 - M_PI * hmax), alpha = powl(2.0L, beta);
    const long double itref = 1.0L / (G0 * gref);
    const long double ga = gref * powl(10.0L, -8.0L + 10.3L * U(rng));  // gamma / gamma_ref in [1e-8, 200]
    RoPairs P;
    split(1.0L / G0, P.iG0h, P.iG0l);
    split(alpha, P.alh, P.all);
    split(alpha * (1 + beta), P.ab1h, P.ab1l);
    split(G0, P.G0h, P.G0l);
    split(itref, P.itrh, P.itrl);
    P.hab1b = (float)(alpha * (1 + beta) * beta / 2);
    P.c2 = (float)(beta * (beta - 1) / 2);
    P.pb.bh = (float)beta;
    P.pb.bl = (float)(beta - (long double)P.pb.bh);
    const long double b0 = roundl(beta * 32768.0L) / 32768.0L, b1 = roundl((beta - b0) * 2147483648.0L) / 2147483648.0L;
    P.pb.b0 = (float)b0;
    P.pb.b1 = (float)b1;
    P.pb.b2 = (float)(beta - b0 - b1);
    // long-double root of tau/G0 (1 + alpha (tau itref)^beta) = ga
    long double tau = G0 * ga;
    for (int k = 0; k < 200; ++k) {
      const long double w = powl(tau * itref, beta);
      const long double f = tau / G0 * (1 + alpha * w) - ga, fp = (1 + alpha * (1 + beta) * w) / G0;
      const long double nt = tau - f / fp;
      if (fabsl(nt - tau) <= 1e-19L * tau) {
        tau = nt;
        break;
      }
      tau = nt > 0 ? nt : tau / 2;
    }
    const long double Gref = G0 / (1 + alpha * (1 + beta) * powl(tau * itref, beta));
    // FP32 Newton seed, stopped at a relative step like the device's
    const float gaf = (float)ga, G0f = (float)G0, iG0f = (float)(1 / G0), itf = (float)itref, bf = (float)beta,
                af = (float)alpha;
    float t = G0f * gaf;
    for (int k = 0; k < 40; ++k) {
      const float pw = powf(t * itf, bf);
      const float step = (t * iG0f * (1 + af * pw) - gaf) * (G0f / (1 + af * (1 + bf) * pw));
      float tn = t - step;
      if (!(tn > 0)) tn = 0.5f * t;
      const bool conv = fabsf(step) <= stop * t;
      t = tn;
      if (conv) break;
    }
    float gah, gal;
    split(ga, gah, gal);
    float th, tl, d, Gh, Gl;
    if (!df64_ro_halley(t, gah, gal, P, tab, th, tl, d, Gh, Gl)) {
      ++declined;
      continue;
    }
    const double et = (double)fabsl(((long double)th + tl) / tau - 1), eg = (double)fabsl(((long double)Gh + Gl) / Gref - 1);
    if (et > wt) wt = et;
    if (eg > wg) wg = eg;
    if (fabs(d) > wd) wd = fabs(d);
  }
  printf("%.6e %.6e %.6e %d\n", wt, wg, wd, declined);
  return 0;
}
