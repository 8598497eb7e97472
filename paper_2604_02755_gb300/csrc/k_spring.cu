// Multi-spring constitutive update at every integration point (Sec. 2.1, Eq. 2):
// spring strains gamma_k = q_k . eps, modified Ramberg-Osgood skeleton with the
// Masing rule per spring (40-byte state), tangent D = Kb m m^T + w sum_k G_k q_k q_k^T.
#include "kern_common.cuh"

namespace ns {

struct RoPar {
  double G0, tref, alpha, beta;  // tref = G0 * gamma_ref
  double iG0, itref;             // reciprocals
};

// ---------------------------------------------------------------------------------------
// FP64 power x^beta for x > 0 (normal), table-driven after Tang (ACM TOMS 1989, 1990):
//   ln x = e ln2 + ln(1/r_j) + ln(1 + u),  u = m r_j - 1,  |u| <= 2^-8,
//     m in [1,2) the mantissa, j its top 7 bits, r_j ~ 1/(1 + (j + 1/2)/128);
//   exp y = 2^(k/64) exp(f),  k = round(64 y / ln2),  |f| <= ln2/128.
// Tables (built on the host in extended precision): r_j, -ln r_j as hi + lo, 2^(i/64),
// and the split constants ln2 and ln2/64 whose high parts have trailing zero bits so
// that products with small integers are exact.  Relative error ~ ulp(|beta ln x|).
struct PowTab {
  const double *r, *lhi, *llo, *t64;  // [128], [128], [128], [64]
  double ln2hi, ln2lo, l64hi, l64lo;
};

__device__ __forceinline__ double ln_pos(double x, const PowTab &tb) {
  const long long bits = __double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7ff) - 1023;
  const long long mb = (bits & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL;
  const int j = (int)((mb >> 45) & 127);
  const double m = __longlong_as_double(mb);
  const double u = fma(m, __ldg(tb.r + j), -1.0);
  // ln(1+u) = u - u^2/2 + u^3/3 - ... (7 terms; |u| <= 2^-8 leaves < 1e-20)
  double p = fma(u, -1.0 / 7.0, 1.0 / 6.0);
  p = fma(u, p, -1.0 / 5.0);
  p = fma(u, p, 1.0 / 4.0);
  p = fma(u, p, -1.0 / 3.0);
  p = fma(u, p, 0.5);
  const double u2 = u * u;
  const double lnp = fma(-u2, p, u);  // u - u^2 (1/2 - u/3 + ...)
  const double ed = (double)e;
  return fma(ed, tb.ln2hi, __ldg(tb.lhi + j)) + (fma(ed, tb.ln2lo, __ldg(tb.llo + j)) + lnp);
}

__device__ __forceinline__ double exp_tab(double y, const PowTab &tb) {
  if (y < -700.0) return 0.0;
  if (y > 700.0) return __longlong_as_double(0x7FF0000000000000LL);
  const double kd = rint(y * (64.0 / 0.6931471805599453));
  const int k = (int)kd;
  double f = fma(-kd, tb.l64hi, y);
  f = fma(-kd, tb.l64lo, f);
  // exp(f) - 1, degree 6 (|f| <= ln2/128 leaves < 3e-20)
  double q = fma(f, 1.0 / 720.0, 1.0 / 120.0);
  q = fma(f, q, 1.0 / 24.0);
  q = fma(f, q, 1.0 / 6.0);
  q = fma(f, q, 0.5);
  q = fma(f, q, 1.0);
  q *= f;
  const double t = __ldg(tb.t64 + (k & 63));
  const double r = fma(t, q, t);
  const int sh = k >> 6;  // floor(k / 64)
  return r * __longlong_as_double((long long)(sh + 1023) << 52);
}

__device__ __forceinline__ double pow_pos(double x, double beta, const PowTab &tb) {
  return exp_tab(beta * ln_pos(x, tb), tb);
}

// Skeleton strain of a stress g(tau) = (tau/G0)(1 + alpha |tau/tref|^beta) and the root
// tau = F(ga) for ga > 0 (g is odd, increasing, convex for tau > 0; tau <= G0 ga).
//  1. FP32 Newton (from the guess when it lies in (0, G0 ga], else from G0 ga) to ~1e-7.
//  2. FP64 safeguarded Newton from that seed; the power is evaluated once with pow_pos and
//     carried to each new iterate by the series (1 + d)^beta (|d| <= 1e-4: error < 1e-19),
//     re-evaluated whenever an iterate moves further.  Stops when a Newton step is below
//     1e-12 tau (the remaining error then is below rounding).
// *pw returns |F/tref|^beta at the returned root (for the tangent 1/g'(F)).
__device__ double ro_F(double ga, double guess, const RoPar &p, const PowTab &tb, double *pw) {
  if (ga == 0.0) {
    *pw = 0.0;
    return 0.0;
  }
  const double hi = p.G0 * ga;
  const float itrf = (float)p.itref, af = (float)p.alpha, bf = (float)p.beta, gaf = (float)ga,
              iG0f = (float)p.iG0, hif = (float)hi;
  float t = (guess > 0.0 && guess < hi) ? (float)guess : hif;
  if (!(t > 0.0f)) t = hif;
  for (int it = 0; it < 40 && t > 0.0f; ++it) {
    const float pwf = powf(t * itrf, bf);
    const float step = (t * iG0f * (1.0f + af * pwf) - gaf) / ((1.0f + af * (1.0f + bf) * pwf) * iG0f);
    float tn = t - step;
    if (!(tn > 0.0f)) tn = 0.5f * t;
    if (tn > hif) tn = hif;
    const bool conv = fabsf(step) <= 2e-7f * t;
    t = tn;
    if (conv) break;
  }
  double tau = (double)t;
  if (!(tau > 0.0) || !(tau <= hi)) tau = hi;
  const double b = p.beta, c2 = b * (b - 1.0) * 0.5, c3 = c2 * (b - 2.0) * (1.0 / 3.0),
               c4 = c3 * (b - 3.0) * 0.25;
  double w = pow_pos(tau * p.itref, b, tb), tw = tau;
  double itw = (double)(1.0f / (float)tw);
  itw = itw * (2.0 - tw * itw);
  double lo = 0.0, up = hi;
  for (int it = 0; it < 200; ++it) {
    const double gval = tau * p.iG0 * (1.0 + p.alpha * w);
    if (gval == ga) break;
    if (gval > ga)
      up = tau;
    else
      lo = tau;
    const double step = (gval - ga) * p.G0 / (1.0 + p.alpha * (1.0 + b) * w);
    double nt = tau - step;
    const bool newton = nt >= lo && nt <= up;
    if (!newton) nt = 0.5 * (lo + up);
    const double last = nt - tau;
    tau = nt;
    const double d = (tau - tw) * itw;
    if (fabs(d) <= 1e-4)
      w *= fma(d, fma(d, fma(d, fma(d, c4, c3), c2), b), 1.0);  // w now belongs to tau
    else
      w = pow_pos(tau * p.itref, b, tb);
    tw = tau;
    itw = (double)(1.0f / (float)tw);
    itw = itw * (2.0 - tw * itw);
    if (newton && fabs(last) <= 1e-12 * tau) break;
  }
  *pw = w;
  return tau;
}

__device__ __forceinline__ double ro_tangent_from_pw(double pw, const RoPar &p) {
  return p.G0 / (1.0 + p.alpha * (1.0 + p.beta) * pw);
}

__device__ __forceinline__ double signed_F(double x, double guess_abs, const RoPar &p, const PowTab &tb, double *pw) {
  const double f = ro_F(fabs(x), guess_abs, p, tb, pw);
  return x < 0.0 ? -f : f;
}

// One spring (Masing bookkeeping of the documented reading): virgin -> skeleton in the
// direction of motion; reversal stores (gamma_old, tau_old) and follows
// tau = tR + 2 F((gamma - gR)/2); moving outward past gmax returns to the skeleton.
// The previous value on the same curve seeds the root search.  Returns the tangent.
__device__ double spring_update(double g, double dg, const RoPar &p, const PowTab &tb, double &tau, double &gR,
                                double &tR, double &gmax, int &dir, int &mode) {
  double pw;
  if (dg != 0.0) {
    const int sgn = dg > 0.0 ? 1 : -1;
    bool same_curve = true;
    if (dir == 0) {
      dir = sgn;
      mode = 0;
      same_curve = false;
    } else if (sgn != dir) {
      gR = g - dg;
      tR = tau;
      mode = 1;
      dir = sgn;
      same_curve = false;
    }
    if (mode == 0) {
      tau = signed_F(g, same_curve ? fabs(tau) : 0.0, p, tb, &pw);
      if (fabs(g) > gmax) gmax = fabs(g);
    } else {
      const double f = signed_F(0.5 * (g - gR), same_curve ? 0.5 * fabs(tau - tR) : 0.0, p, tb, &pw);
      tau = tR + 2.0 * f;
      if (fabs(g) >= gmax && g * (double)dir > 0.0) {
        mode = 0;
        tau = signed_F(g, fabs(tau), p, tb, &pw);
        gmax = fabs(g);
      }
    }
    return ro_tangent_from_pw(pw, p);
  }
  const double te = (mode == 0) ? tau : 0.5 * (tau - tR);
  pw = (te == 0.0) ? 0.0 : pow_pos(fabs(te) * p.itref, p.beta, tb);
  return ro_tangent_from_pw(pw, p);
}

// Block = a tile of TP consecutive points (TP multiple of 4) with all their S springs.
// Phase 1: each thread updates springs of the tile (coalesced state access), stores
// G_k in shared memory.  Phase 2: D_p[ij] = Kb [i,j < 3] + sum_k G_k T_k[ij].
__global__ void __launch_bounds__(kBlock) k_springs(const double *__restrict__ q, const double *__restrict__ T, int S,
                                                    int TP, const MatConst *__restrict__ mc,
                                                    const int32_t *__restrict__ mat_e, const int32_t *__restrict__ mat_p,
                                                    const double *__restrict__ eps, double *tau_a, double *gR_a,
                                                    double *tR_a, double *gmax_a, int32_t *dir_a, int32_t *mode_a,
                                                    int64_t base, int64_t p0, int64_t p1, double *D, int64_t epad,
                                                    double *dpts, const double *__restrict__ ptab) {
  extern __shared__ double Gs[];
  const PowTab tb{ptab, ptab + 128, ptab + 256, ptab + 384, __ldg(ptab + 448), __ldg(ptab + 449), __ldg(ptab + 450),
                  __ldg(ptab + 451)};
  const int64_t pt = p0 + (int64_t)blockIdx.x * TP;
  const int np = (int)((p1 - pt) < TP ? (p1 - pt) : TP);
  const int nspr = np * S;
  for (int g = threadIdx.x; g < nspr; g += blockDim.x) {
    const int lp = g / S, k = g - lp * S;
    const int64_t p = pt + lp;
    const int mt = mat_p ? mat_p[p] : mat_e[p >> 2];
    const MatConst &m = mc[mt];
    const RoPar rp{m.G0, m.G0 * m.gref, m.alpha_ro, m.beta_ro, 1.0 / m.G0, 1.0 / (m.G0 * m.gref)};
    const double *ep = eps + 12 * p;
    const double *qk = q + 6 * k;
    double gam = 0.0, dgam = 0.0;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const double qc = __ldg(qk + c);
      gam += qc * __ldg(ep + c);
      dgam += qc * __ldg(ep + 6 + c);
    }
    const int64_t si = (p - base) * S + k;
    double tau = tau_a[si], gR = gR_a[si], tR = tR_a[si], gmax = gmax_a[si];
    int dir = dir_a[si], mode = mode_a[si];
    const double G = spring_update(gam, dgam, rp, tb, tau, gR, tR, gmax, dir, mode);
    if (dgam != 0.0) {
      tau_a[si] = tau;
      gR_a[si] = gR;
      tR_a[si] = tR;
      gmax_a[si] = gmax;
      dir_a[si] = dir;
      mode_a[si] = mode;
    }
    Gs[g] = G;
  }
  __syncthreads();
  const int nout = np * 21;
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    const int lp = o % np, ij = o / np;
    const int64_t p = pt + lp;
    const int mt = mat_p ? mat_p[p] : mat_e[p >> 2];
    const bool nn = ij < 3 || ij == 6 || ij == 7 || ij == 11;  // (i,j) both < 3
    double acc = nn ? mc[mt].Kb : 0.0;
    const double *Gp = Gs + lp * S;
    for (int k = 0; k < S; ++k) acc += Gp[k] * __ldg(T + 21 * k + ij);
    if (dpts)
      dpts[21 * p + ij] = acc;
    else
      D[((p & 3) * 21 + ij) * epad + (p >> 2)] = acc;
  }
}

static int tile_points(int S) {
  int te = 4096 / (4 * S);
  int p2 = 1;
  while (p2 * 2 <= te && p2 < 64) p2 *= 2;
  return 4 * p2;
}

cudaError_t launch_springs(const SpringTables &tab, const MatConst *mc, const int32_t *mat_of_elem,
                           const int32_t *mat_of_point, const double *eps, SpringSoA st, int64_t base, int64_t p0,
                           int64_t p1, double *D, int64_t epad, double *dpts, cudaStream_t s) {
  if (p1 <= p0) return cudaSuccess;
  const int TP = tile_points(tab.S);
  const size_t smem = sizeof(double) * TP * tab.S;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_springs, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  const unsigned nb = (unsigned)((p1 - p0 + TP - 1) / TP);
  k_springs<<<nb, kBlock, smem, s>>>(tab.q, tab.T, tab.S, TP, mc, mat_of_elem, mat_of_point, eps, st.tau, st.gR,
                                     st.tR, st.gmax, st.dir, st.mode, base, p0, p1, D, epad, dpts, tab.pow);
  return cudaGetLastError();
}

// Elastic tangent (every spring at G0): D = Kb m m^T + G0 sum_k T_k.
__global__ void k_elastic_D(const double *__restrict__ Tsum, const MatConst *__restrict__ mc,
                            const int32_t *__restrict__ mat, double *D, int64_t epad, int64_t e0, int64_t e1) {
  const int64_t e = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= e1) return;
  const MatConst &m = mc[mat[e]];
  for (int q = 0; q < 4; ++q)
    for (int ij = 0; ij < 21; ++ij) {
      const bool nn = ij < 3 || ij == 6 || ij == 7 || ij == 11;
      D[(q * 21 + ij) * epad + e] = (nn ? m.Kb : 0.0) + m.G0 * Tsum[ij];
    }
}

cudaError_t launch_elastic_D(const SpringTables &tab, const MatConst *mc, const int32_t *mat, double *D, int64_t epad,
                             int64_t e0, int64_t e1, cudaStream_t s) {
  if (e1 <= e0) return cudaSuccess;
  // tab.T holds S rows followed by one extra row with their sum
  k_elastic_D<<<(unsigned)((e1 - e0 + kBlock - 1) / kBlock), kBlock, 0, s>>>(tab.T + 21 * tab.S, mc, mat, D, epad, e0,
                                                                             e1);
  return cudaGetLastError();
}

__global__ void k_D_to_f32(const double *D, float *D32, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    D32[i] = (float)D[i];
}

cudaError_t launch_D_to_f32(const double *D, float *D32, int64_t epad, int64_t, cudaStream_t s) {
  const int64_t n = 84 * epad;
  k_D_to_f32<<<152 * 8, kBlock, 0, s>>>(D, D32, n);
  return cudaGetLastError();
}

}  // namespace ns
