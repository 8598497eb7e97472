// Multi-spring constitutive update at every integration point (Sec. 2.1, Eq. 2):
// spring strains gamma_k = q_k . eps, modified Ramberg-Osgood skeleton with the
// Masing rule per spring (40-byte state), tangent D = Kb m m^T + w sum_k G_k q_k q_k^T.
#include <algorithm>
#include <atomic>

#include "kern_common.cuh"

namespace ns {

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
  // 2^floor(k/64) built in the exponent field; the clamp turns underflow into 0 and
  // keeps overflow finite (neither occurs for the strains of the spring law)
  const int sh = max(-1023, min(1023, k >> 6));
  return r * __longlong_as_double((long long)(sh + 1023) << 52);
}

__device__ __forceinline__ double pow_pos(double x, double beta, const PowTab &tb) {
  return exp_tab(beta * ln_pos(x, tb), tb);
}

// Sign, zero and magnitude tests on the IEEE bit pattern (integer pipes; the FP64 pipe
// is the scarce resource of this kernel).  For non-negative doubles the bit patterns
// order like the values.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool d_is_zero(double x) { return (dbits(x) << 1) == 0; }
__device__ __forceinline__ bool d_sign(double x) { return dbits(x) < 0; }
__device__ __forceinline__ double d_abs(double x) { return __longlong_as_double(dbits(x) & 0x7FFFFFFFFFFFFFFFLL); }
__device__ __forceinline__ double d_copysign(double m, double s) {
  return __longlong_as_double((dbits(m) & 0x7FFFFFFFFFFFFFFFLL) | (dbits(s) & (long long)0x8000000000000000ULL));
}

// FP32 reciprocal refined once in FP64 (relative error ~1e-14).
__device__ __forceinline__ double rcp1(double x) {
  double r = (double)(1.0f / (float)x);
  return r * fma(-x, r, 2.0);
}

// Safeguarded FP64 Newton on g(tau) = ga from tau in (0, hi]: bisection replaces steps that
// leave the bracket; the power is re-evaluated at every iterate.  Used only when the
// fast path below does not certify convergence.
__device__ double ro_F_safe(double ga, double tau, const MatConst &p, const PowTab &tb, double *pw) {
  const double hi = p.G0 * ga;
  double lo = 0.0, up = hi, w = pow_pos(tau * p.itref, p.beta_ro, tb);
  for (int it = 0; it < 200; ++it) {
    const double gval = tau * p.iG0 * (1.0 + p.alpha_ro * w);
    if (gval == ga) break;
    if (gval > ga)
      up = tau;
    else
      lo = tau;
    const double step = (gval - ga) * p.G0 / (1.0 + p.ab1 * w);
    double nt = tau - step;
    const bool newton = nt >= lo && nt <= up;
    if (!newton) nt = 0.5 * (lo + up);
    const double last = nt - tau;
    tau = nt;
    w = pow_pos(tau * p.itref, p.beta_ro, tb);
    if (newton && fabs(last) <= 1e-15 * tau) break;
  }
  *pw = w;
  return tau;
}

// G0 / g'(tau) with g' = 1 + alpha (1 + beta) pw.
__device__ __forceinline__ double ro_tangent_from_pw(double pw, const MatConst &p) {
  return p.G0 * rcp1(fma(p.ab1, pw, 1.0));
}

// A positive FP64 modulus as an unevaluated sum of two floats: the high part is G with its
// low 29 significand bits cleared, built as a float from the bit pattern on the integer
// pipes (G in the normal float range), the low part the rounded rest.
__device__ __forceinline__ float2 split_pair(double G) {
  const long long gb = __double_as_longlong(G);
  const double Ghi = __longlong_as_double(gb & ~0x1FFFFFFFLL);
  const unsigned int fb = (unsigned int)((((gb >> 52) & 0x7FF) - 896) << 23) | (unsigned int)((gb >> 29) & 0x7FFFFF);
  return make_float2(__uint_as_float(fb), (float)(G - Ghi));
}

// Any double as an unevaluated float pair: the high part is v with its low 29 significand
// bits cleared, the low part the rest rounded to a float -- both built on the integer and
// FP32 pipes (GB300 runs FP64 conversions at 1/64 of the FP32 rate): the rest is the low
// 29 significand bits times 2^(e - 52), converted from the integer (round to nearest) and
// scaled by an exact power of two.  Values outside the normal float range (zero included)
// are rounded to one float; for |v| < 2^-74 the rest is formed in FP64.
__device__ __forceinline__ void dsplit(double v, float &h, float &l) {
  const long long b = __double_as_longlong(v);
  const int ed = (int)((b >> 52) & 0x7FF);
  if (ed > 896 && ed < 1151) {
    const unsigned int sg = (unsigned int)((b >> 32) & 0x80000000LL);
    h = __uint_as_float(sg | (unsigned int)((ed - 896) << 23) | (unsigned int)((b >> 29) & 0x7FFFFF));
    if (ed >= 949) {
      const unsigned int m29 = (unsigned int)(b & 0x1FFFFFFFLL);
      const float lo = __uint2float_rn(m29);  // exact below 2^24, else rounded to nearest
      l = m29 ? __uint_as_float(__float_as_uint(lo * __uint_as_float((unsigned int)(ed - 948) << 23)) | sg) : 0.0f;
    } else {
      l = (float)(v - __longlong_as_double(b & ~0x1FFFFFFFLL));
    }
  } else {
    h = (float)v;
    l = 0.0f;
  }
}

// A float as a double, exactly, on the integer pipes (normal floats and zero; subnormal
// floats -- below 1.2e-38, which the spring law's pairs do not hold -- become zero).
__device__ __forceinline__ double f2d(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned int e = (b >> 23) & 0xFF;
  const unsigned long long sg = (unsigned long long)(b & 0x80000000u) << 32;
  const unsigned long long r =
      e ? (sg | ((unsigned long long)(e + 896) << 52) | ((unsigned long long)(b & 0x7FFFFF) << 29)) : sg;
  return __longlong_as_double((long long)r);
}

// The value of a float pair as a double: the two parts converted exactly, one FP64 add.
__device__ __forceinline__ double pair_to_double(float h, float l) { return f2d(h) + f2d(l); }

// A double truncated to a float (a starting guess, not a result): the high part of dsplit.
__device__ __forceinline__ float d2f_guess(double v) {
  const long long b = __double_as_longlong(v);
  const int ed = (int)((b >> 52) & 0x7FF);
  if (ed > 896 && ed < 1151)
    return __uint_as_float((unsigned int)((b >> 32) & 0x80000000LL) | (unsigned int)((ed - 896) << 23) |
                           (unsigned int)((b >> 29) & 0x7FFFFF));
  return (float)v;
}

// -v by its sign bit
__device__ __forceinline__ double d_neg(double v) {
  return __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ULL);
}

// Root tau = F(ga) of the skeleton g(tau) = (tau/G0)(1 + alpha (tau/tref)^beta) = ga >= 0
// (g odd, increasing, convex for tau > 0, tau <= G0 ga) and the tangent G = 1/g'(tau) as a
// float pair; or -- when `solve` is false -- only the tangent at tau = ga (the current
// stress).  The usual path:
//  1. FP32 Newton from the guess if it lies in (0, G0 ga], else from G0 ga, until a step
//     is below 1e-3 of the iterate (Newton's quadratic convergence leaves the new iterate
//     within ~1e-6 of the root, which the cubic step below turns into rounding);
//  2. one Halley step from that FP32 seed in double-float arithmetic on the FP32 pipes
//     (df64_ro_halley: the power, the residual against ga, the step and the tangent at
//     the new root; root to ~2^-47, tangent to ~2^-45).
// When the seed did not converge, the step exceeds 2e-5 of the root, or the power's
// argument is out of its range, the FP64 path takes over: table-driven FP64 power, FP64
// Halley step and, unless that certifies, the safeguarded Newton loop.
__device__ __forceinline__ double ro_solve(bool solve, double ga, double guess, const MatConst &p, const PowTab &tb,
                                           const float *__restrict__ tabf, float2 *Gp) {
  double tau = ga;
  bool seeded = true;
  if (solve) {
    const float gaf = (float)ga, hif = p.G0_f * gaf, gs = (float)guess;
    float t = (gs > 0.0f && gs < hif) ? gs : hif;
    seeded = false;
    for (int it = 0; it < 40 && t > 0.0f; ++it) {
      const float pwf = __powf(t * p.itref_f, p.beta_f);
      const float gp = 1.0f + p.alpha_f * (1.0f + p.beta_f) * pwf;
      const float step = (t * p.iG0_f * (1.0f + p.alpha_f * pwf) - gaf) * __fdividef(p.G0_f, gp);
      float tn = t - step;
      if (!(tn > 0.0f)) tn = 0.5f * t;
      if (tn > hif) tn = hif;
      const bool conv = fabsf(step) <= 1e-3f * t;
      t = tn;
      if (conv) {
        seeded = true;
        break;
      }
    }
    if (seeded && t > 0.0f) {
      const float gal = (float)(ga - (double)gaf);
      float th, tl, d, Gh, Gl;
      if (df64_ro_halley(t, gaf, gal, p.rp, tabf, th, tl, d, Gh, Gl) && fabsf(d) <= 2e-5f) {
        *Gp = make_float2(Gh, Gl);
        return (double)th + (double)tl;
      }
    }
    tau = (t > 0.0f) ? (double)t : p.G0 * ga;  // FP32 underflow: start from the linear bound
  }
  if (d_is_zero(tau)) {  // zero strain (or zero stress): the power vanishes, G = G0
    *Gp = split_pair(p.G0);
    return 0.0;
  }
  double w = pow_pos(tau * p.itref, p.beta_ro, tb);
  if (solve) {
    // Halley: step = h / (1 - h f''/(2 f')) with h = f/f' the Newton step; |h f''/(2 f')|
    // is ~ the seed error (~1e-6), so 1/(1 - c) = 1 + c to far below rounding
    const double it0 = rcp1(tau);
    const double gval = tau * p.iG0 * fma(p.alpha_ro, w, 1.0);
    const double rg = rcp1(fma(p.ab1, w, 1.0));
    const double h = (gval - ga) * p.G0 * rg;
    const double hc = h * p.hab1b * w * it0 * rg;
    const double step = fma(h, hc, h);
    const double d = -step * it0;
    tau -= step;
    w *= fma(d, fma(d, fma(d, p.c3, p.c2), p.beta_ro), 1.0);
    if (!(seeded && fabs(d) <= 2e-5)) {
      const double hi = p.G0 * ga;
      tau = ro_F_safe(ga, (tau > 0.0 && tau <= hi) ? tau : hi, p, tb, &w);
    }
  }
  *Gp = split_pair(ro_tangent_from_pw(w, p));
  return tau;
}

// As ro_solve (solving), for ga = gah + gal > 0 given as a float pair (the usual path
// never forms ga in FP64).
__device__ __forceinline__ double ro_solve_pair(float gah, float gal, float guess, const MatConst &p,
                                                const PowTab &tb, const float *__restrict__ tabf, float2 *Gp,
                                                unsigned &ev) {
  if (!(gah > 0.0f)) {  // zero strain: zero stress, G = G0
    *Gp = split_pair(p.G0);
    return 0.0;
  }
  const float hif = p.G0_f * gah;
  float t = (guess > 0.0f && guess < hif) ? guess : hif;
  bool seeded = false;
  for (int it = 0; it < 40 && t > 0.0f; ++it) {
    const float pwf = __powf(t * p.itref_f, p.beta_f);
    const float gp = 1.0f + p.alpha_f * (1.0f + p.beta_f) * pwf;
    const float step = (t * p.iG0_f * (1.0f + p.alpha_f * pwf) - gah) * __fdividef(p.G0_f, gp);
    float tn = t - step;
    if (!(tn > 0.0f)) tn = 0.5f * t;
    if (tn > hif) tn = hif;
    const bool conv = fabsf(step) <= 1e-3f * t;
    t = tn;
    if (conv) {
      seeded = true;
      break;
    }
  }
  if (seeded && t > 0.0f) {
    float th, tl, d, Gh, Gl;
    if (df64_ro_halley(t, gah, gal, p.rp, tabf, th, tl, d, Gh, Gl) && fabsf(d) <= 2e-5f) {
      *Gp = make_float2(Gh, Gl);
      return pair_to_double(th, tl);
    }
  }
  // the FP64 path from the seed (or from the linear bound)
  ev |= 4u;
  const double ga = (double)gah + (double)gal;
  double tau = (t > 0.0f) ? (double)t : p.G0 * ga;
  double w = pow_pos(tau * p.itref, p.beta_ro, tb);
  const double it0 = rcp1(tau);
  const double gval = tau * p.iG0 * fma(p.alpha_ro, w, 1.0);
  const double rg = rcp1(fma(p.ab1, w, 1.0));
  const double h = (gval - ga) * p.G0 * rg;
  const double hc = h * p.hab1b * w * it0 * rg;
  const double step = fma(h, hc, h);
  const double d = -step * it0;
  tau -= step;
  w *= fma(d, fma(d, fma(d, p.c3, p.c2), p.beta_ro), 1.0);
  if (!(seeded && fabs(d) <= 2e-5)) {
    const double hi = p.G0 * ga;
    tau = ro_F_safe(ga, (tau > 0.0 && tau <= hi) ? tau : hi, p, tb, &w);
  }
  *Gp = split_pair(ro_tangent_from_pw(w, p));
  return tau;
}

// One spring (Masing bookkeeping of the documented reading): virgin -> skeleton in the
// direction of motion; reversal stores (gamma_old, tau_old) and follows
// tau = tR + 2 F((gamma - gR)/2); moving outward with |gamma| >= gmax returns to the
// skeleton tau = F(gamma) (decided before the root solve, so each spring solves once).
// With no increment the state is kept and only the tangent is evaluated.
// Returns the tangent dtau/dgamma at the end state as a float pair.
// The spring strain gamma = gh + gl comes as a normalised float pair (the dot product
// q_k . eps in double-float arithmetic); the stored state stays FP64, and comparisons
// with it are made on pair differences.  Of the increment dgamma only the sign is needed
// unless the spring reverses: dh carries that sign (and is exactly zero for no
// increment); when !dexact the pair dh + dl = q_k . deps is formed at a reversal.
// ev collects what happened: 1 the spring moved, 2 it reversed, 4 its root took the FP64 path.
__device__ __forceinline__ void pair_dot6(const float2 *__restrict__ q, const float2 *e, float &sh, float &sl);
__device__ __forceinline__ float2 spring_update_pair(float gh, float gl, float dh, float dl, bool dexact,
                                                     const float2 *__restrict__ qk, const float2 *de,
                                                     const MatConst &p, const PowTab &tb,
                                                     const float *__restrict__ tabf, double &tau, double &gR,
                                                     double &tR, double &gmax, int &dir, int &mode,
                                                     unsigned &ev) {
  float2 G;
  if (dh == 0.0f) {  // no increment: only the tangent at the current state
    const double x = (mode == 0) ? tau : 0.5 * (tau - tR);
    ro_solve(false, d_abs(x), 0.0, p, tb, tabf, &G);
    return G;
  }
  ev |= 1u;
  const int sgn = dh < 0.0f ? -1 : 1;
  bool same = true;
  if (dir == 0) {
    dir = sgn;
    mode = 0;
    same = false;
  } else if (sgn != dir) {  // reversal: (gamma - dgamma, tau) becomes the branch origin
    if (!dexact) pair_dot6(qk, de, dh, dl);
    float rh, rl;
    pair_add(gh, gl, -dh, -dl, rh, rl);
    gR = pair_to_double(rh, rl);
    tR = tau;
    mode = 1;
    dir = sgn;
    same = false;
    ev |= 2u;
  }
  // |gamma| - gmax as a pair
  const bool gneg = gh < 0.0f;
  const float agh = fabsf(gh), agl = gneg ? -gl : gl;
  float mh, ml, ch, cl;
  dsplit(gmax, mh, ml);
  pair_add(agh, agl, -mh, -ml, ch, cl);
  const bool beyond = ch > 0.0f || (ch == 0.0f && cl >= 0.0f);
  // outward (gamma on the side of dir, nonzero) with |gamma| >= gmax: back on the skeleton
  const bool outward = gh != 0.0f && (gneg == (dir < 0));
  float guess = 0.0f;
  if (mode == 1 && outward && beyond) {
    mode = 0;
    guess = fabsf(d2f_guess(tau));
  } else if (same) {
    guess = (mode == 0) ? fabsf(d2f_guess(tau)) : 0.5f * fabsf(d2f_guess(tau) - d2f_guess(tR));
  }
  float xh = gh, xl = gl;
  if (mode == 1) {  // (gamma - gR) / 2
    float rh, rl;
    dsplit(gR, rh, rl);
    pair_add(gh, gl, -rh, -rl, xh, xl);
    xh *= 0.5f;
    xl *= 0.5f;
  }
  const bool xneg = xh < 0.0f;
  const double f = ro_solve_pair(fabsf(xh), xneg ? -xl : xl, guess, p, tb, tabf, &G, ev);
  const double fs = xneg ? d_neg(f) : f;
  if (mode == 0) {
    tau = fs;
    if (ch > 0.0f || (ch == 0.0f && cl > 0.0f)) gmax = pair_to_double(agh, agl);
  } else {
    tau = fma(2.0, fs, tR);
  }
  return G;
}

// Sign of q_k . e from an FP32 dot of the pairs' high parts.  Its error is below
// 2^-20.9 sum |q_i e_i| (six fused steps, plus the dropped low parts, each under 2^-24 of
// its high part), so beyond 2^-18 of that sum the sign is certain and equals that of the
// pair dot product; a zero sum means every product, hence the dot, is exactly zero.
// Returns false when the sign is not settled (the caller forms the pair dot).
__device__ __forceinline__ bool dot6_sign(const float2 *__restrict__ q, const float2 *e, float &s) {
  float a = 0.0f, b = 0.0f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float qh = __ldg(&q[i].x), eh = e[i].x;
    a = fmaf(qh, eh, a);
    b = fmaf(fabsf(qh), fabsf(eh), b);
  }
  s = a;
  return b == 0.0f || fabsf(a) > 0x1p-18f * b;
}

// gamma = q_k . e for a float-pair direction q (6) and a float-pair strain e (6), as a
// normalised pair: exact products (FMA error terms) and compensated sums.
__device__ __forceinline__ void pair_dot6(const float2 *__restrict__ q, const float2 *e, float &sh, float &sl) {
  float s = 0.0f, c = 0.0f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float2 qi = __ldg(q + i), ei = e[i];
    float p, pe, t, te;
    two_prod(qi.x, ei.x, p, pe);
    pe = df_add(pe, df_fma(qi.x, ei.y, df_mul(qi.y, ei.x)));
    two_sum(s, p, t, te);
    s = t;
    c = df_add(c, df_add(te, pe));
  }
  fast_two_sum(s, c, sh, sl);
}

// ------------------------------------------------------------------ tangent assembly on tensor cores
// D_p[ij] = Kb [i,j < 3] + sum_k G_pk T_k[ij] is a dense (points x S) . (S x 21) product.
// It runs on the tensor cores (warp-level bf16 MMA, FP32 accumulation) with FP64-level
// accuracy by splitting both operands into 6-bit integer digits: G_pk 2^-eG =
// sum_i a_i 2^-6(i+1) (a_i in 0..63, eG per material with 2^eG > G0 >= G),
// T_k[ij] 2^-eT[ij] = sum_j b_j 2^-6(j+1) (|b_j| <= 63, one exponent per column ij).
// Every digit is exact in bf16, every digit product exact in FP32, and the sum over k of
// the products of one level L = i + j (at most 8 pairs x S x 63^2 < 2^23 for S <= 256) is
// an integer that FP32 holds exactly, so the MMA accumulators C_L are exact;
// D = Kb + 2^(eG + eT[ij] - 12) sum_{L <= 8} 2^-6L C_L, the levels combined in
// double-float arithmetic.  The digits beyond the eighth and the levels above 8 leave an
// error below 2^-47 of G0 sum_k |T_k[ij]|.
constexpr int kDigits = 8;
constexpr int kLevels = 9;  // digit-pair levels L = i + j kept: 0 .. 8
constexpr int kTcMaxS = 256;

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

// c += a . b for one 16 x 8 x 16 tile: a row-major bf16 (4 registers), b column-major bf16
// (2 registers), c FP32 (rows lane/4 and lane/4 + 8, columns 2 (lane % 4) + {0, 1})
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// bf16 bits of a small non-negative integer d (< 2^8): 2^23 + d as a float, minus 2^23
__device__ __forceinline__ unsigned short bf16_of_digit(uint32_t d) {
  return (unsigned short)(__float_as_uint(__uint_as_float(0x4B000000u | d) - 8388608.0f) >> 16);
}

// row stride (bf16 elements) of a digit plane: 16 * ks + 8, so that the eight rows one
// ldmatrix reads fall in distinct shared-memory banks
__host__ __device__ inline int tc_stride(int ks) { return 16 * ks + 8; }

// Block = a tile of TP consecutive points (TP multiple of 4) with all their S springs.
// Phase 1: each thread updates springs of the tile (coalesced state access), stores
// G_k in shared memory.  Phase 2: D_p[ij] = Kb [i,j < 3] + sum_k G_k T_k[ij].
// MINB: resident blocks per SM the registers are budgeted for (1: the compiler's choice,
// 80 registers, three blocks; 4: 64 registers with a few bytes spilled, a third more
// warps to hide the root solve's latencies) -- the autotuner picks.
// TC: phase 1 stores the tangents as digit planes and phase 2 assembles D on the tensor
// cores (TP a multiple of 16, S <= 256; tfrag holds the digits of T in MMA fragment order).
template <int MINB, bool TC>
__global__ void __launch_bounds__(kBlock, MINB) k_springs(const float2 *__restrict__ q2, const float2 *__restrict__ T2, int S,
                                                    int TP, const MatConst *__restrict__ mc,
                                                    const int32_t *__restrict__ mat_e, const int32_t *__restrict__ mat_p,
                                                    const double *__restrict__ eps, double *tau_a, double *gR_a,
                                                    double *tR_a, double *gmax_a, int32_t *dir_a, int32_t *mode_a,
                                                    int64_t base, int64_t p0, int64_t p1, double *D, int64_t epad,
                                                    double *dpts, const double *__restrict__ ptab,
                                                    const float *__restrict__ ptabf, const uint2 *__restrict__ tfrag,
                                                    const double *__restrict__ tsc, int eps_pairs,
                                                    unsigned long long *cnt) {
  // shared: [TP][S] tangents as float pairs (or, TC, [8][TP][stride] bf16 digit planes),
  // then [TP][12] strains as pairs
  extern __shared__ float2 Gs[];
  __shared__ unsigned evc[3];  // the block's springs moved, reversed, with an FP64 root
  const int KS = (S + 15) >> 4, KST = tc_stride(KS);
  unsigned short *planes = reinterpret_cast<unsigned short *>(Gs);
  const PowTab tb{ptab, ptab + 128, ptab + 256, ptab + 384, __ldg(ptab + 448), __ldg(ptab + 449), __ldg(ptab + 450),
                  __ldg(ptab + 451)};
  const int64_t pt = p0 + (int64_t)blockIdx.x * TP;
  const int np = (int)((p1 - pt) < TP ? (p1 - pt) : TP);
  const int nspr = np * S;
  if (threadIdx.x < 3) evc[threadIdx.x] = 0u;
  // phase 0: the tile's strains and increments as float pairs (once per point, not per spring)
  float2 *Es = TC ? reinterpret_cast<float2 *>(planes + (size_t)kDigits * TP * KST) : Gs + (size_t)TP * S;
  for (int i = threadIdx.x; i < np * 12; i += blockDim.x) {
    if (eps_pairs) {  // already pairs (the strain kernel's double-float output)
      Es[i] = reinterpret_cast<const float2 *>(eps)[12 * pt + i];
    } else {
      float h, l;
      dsplit(eps[12 * pt + i], h, l);
      Es[i] = make_float2(h, l);
    }
  }
  if (TC) {  // zero digits in the padded springs S .. 16 KS - 1 (every plane, every row)
    const int pad = 16 * KS - S, nz = kDigits * TP * pad;
    for (int i = threadIdx.x; i < nz; i += blockDim.x) {
      const int row = i / pad;
      planes[(size_t)row * KST + S + (i - row * pad)] = 0;
    }
  }
  __syncthreads();
  // spring g = lp * S + k of the tile; (lp, k) advanced by the block stride without a
  // division per spring
  const int dlp = (int)blockDim.x / S, dk = (int)blockDim.x - dlp * S;
  int lp = (int)threadIdx.x / S, k = (int)threadIdx.x - lp * S;
  // springs moved (bits 0-9), reversed (10-19) and with an FP64 root (20-29) by this thread
  // (a thread updates at most ceil(TP S / 256) <= 1,024 springs of its block)
  unsigned evn = 0;
  for (int g = threadIdx.x; g < nspr; g += blockDim.x, lp += dlp, k += dk) {
    if (k >= S) {
      k -= S;
      ++lp;
    }
    const int64_t p = pt + lp;
    const int mt = mat_p ? mat_p[p] : mat_e[p >> 2];
    const MatConst &rp = mc[mt];
    float gh, gl, dh, dl = 0.0f;
    pair_dot6(q2 + 6 * k, Es + 12 * lp, gh, gl);
    const bool sure = dot6_sign(q2 + 6 * k, Es + 12 * lp + 6, dh);
    if (!sure) pair_dot6(q2 + 6 * k, Es + 12 * lp + 6, dh, dl);
    const int64_t si = (p - base) * S + k;
    double tau = tau_a[si], gR = gR_a[si], tR = tR_a[si], gmax = gmax_a[si];
    int dir = dir_a[si], mode = mode_a[si];
    unsigned ev = 0;
    const float2 G = spring_update_pair(gh, gl, dh, dl, !sure, q2 + 6 * k, Es + 12 * lp + 6, rp, tb, ptabf, tau, gR,
                                        tR, gmax, dir, mode, ev);
    evn += (ev & 1u) | ((ev & 2u) << 9) | ((ev & 4u) << 18);
    if (dh != 0.0f) {
      tau_a[si] = tau;
      gR_a[si] = gR;
      tR_a[si] = tR;
      gmax_a[si] = gmax;
      dir_a[si] = dir;
      mode_a[si] = mode;
    }
    if (TC) {
      // G 2^(48 - eG) as a 48-bit integer from the pair, then its eight 6-bit digits
      const float sc = rp.gfix;
      long long X = (long long)__float2ull_rz(G.x * sc) + __float2ll_rn(G.y * sc);
      X = X < 0 ? 0 : (X > 0xFFFFFFFFFFFFll ? 0xFFFFFFFFFFFFll : X);
      const unsigned long long U = (unsigned long long)X;
      unsigned short *dst = planes + (size_t)lp * KST + k;
#pragma unroll
      for (int i = 0; i < kDigits; ++i)
        dst[(size_t)i * TP * KST] = bf16_of_digit((uint32_t)(U >> (42 - 6 * i)) & 63u);
    } else {
      Gs[g] = G;  // the tangent as an unevaluated float pair for the double-float accumulation
    }
  }
  if (cnt) {
    const unsigned n_moved = __reduce_add_sync(0xffffffffu, evn & 1023u);
    const unsigned n_rev = __reduce_add_sync(0xffffffffu, (evn >> 10) & 1023u);
    const unsigned n_fp64 = __reduce_add_sync(0xffffffffu, (evn >> 20) & 1023u);
    if ((threadIdx.x & 31) == 0 && (n_moved | n_rev | n_fp64)) {
      atomicAdd_block(&evc[0], n_moved);
      atomicAdd_block(&evc[1], n_rev);
      atomicAdd_block(&evc[2], n_fp64);
    }
  }
  __syncthreads();
  if (cnt && threadIdx.x < 3 && evc[threadIdx.x])
    atomicAdd(cnt + 3 * (blockIdx.x % kSpringCountSlots) + threadIdx.x, (unsigned long long)evc[threadIdx.x]);
  if (TC) {
    // one warp per (16-point tile, 8-column tile) of D; level by level, deepest first, each
    // level's digit-pair MMAs accumulated in two alternating sets, then folded into
    // v = sum_L 2^-6L C_L by Horner's rule in double-float arithmetic
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntask = (TP >> 4) * 3;
    for (int task = warp; task < ntask; task += kBlock >> 5) {
      const int mt = task / 3, nt = task - mt * 3;
      const uint32_t arow = (uint32_t)__cvta_generic_to_shared(
          planes + (size_t)(mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8) * KST + (lane >> 4) * 8);
      const uint2 *bt = tfrag + (size_t)nt * 32 + lane;
      float vh[4] = {0.0f, 0.0f, 0.0f, 0.0f}, vl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      for (int L = kLevels - 1; L >= 0; --L) {
        float c0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, c1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int i = L < kDigits ? 0 : L - kDigits + 1; i <= L && i < kDigits; ++i) {
          const uint32_t ai = arow + (uint32_t)((size_t)i * TP * KST * 2);
          const uint2 *bj = bt + (size_t)(L - i) * KS * 3 * 32;
          int ks = 0;
          for (; ks + 1 < KS; ks += 2) {
            uint32_t a0[4], a1[4];
            ldsm_x4(a0, ai + (uint32_t)(ks * 32));
            ldsm_x4(a1, ai + (uint32_t)(ks * 32 + 32));
            mma_bf16(c0, a0, __ldg(bj + (size_t)ks * 96));
            mma_bf16(c1, a1, __ldg(bj + (size_t)(ks + 1) * 96));
          }
          if (ks < KS) {
            uint32_t a0[4];
            ldsm_x4(a0, ai + (uint32_t)(ks * 32));
            mma_bf16(c0, a0, __ldg(bj + (size_t)ks * 96));
          }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {  // c0 + c1 is exact (an integer below 2^23)
          float s, e;
          two_sum(c0[r] + c1[r], vh[r] * 0.015625f, s, e);
          two_sum(s, e + vl[r] * 0.015625f, vh[r], vl[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int lp = mt * 16 + (lane >> 2) + (r >> 1) * 8, ij = nt * 8 + 2 * (lane & 3) + (r & 1);
        if (lp < np && ij < 21) {
          const int64_t p = pt + lp;
          const MatConst &m = mc[mat_p ? mat_p[p] : mat_e[p >> 2]];
          const bool nn = ij < 3 || ij == 6 || ij == 7 || ij == 11;  // (i,j) both < 3
          const double val = (nn ? m.Kb : 0.0) + m.dsc * (__ldg(tsc + ij) * ((double)vh[r] + (double)vl[r]));
          if (dpts)
            dpts[21 * (p - p0) + ij] = val;
          else
            D[((p & 3) * 21 + ij) * epad + (p >> 2)] = val;
        }
      }
    }
    return;
  }
  const int nout = np * 21;
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    const int lp = o % np, ij = o / np;
    const int64_t p = pt + lp;
    const int mt = mat_p ? mat_p[p] : mat_e[p >> 2];
    const bool nn = ij < 3 || ij == 6 || ij == 7 || ij == 11;  // (i,j) both < 3
    // sum_k G_k T_k[ij] in double-float arithmetic on the FP32 pipes: exact products
    // (FMA error terms), cross terms, and compensated (two-sum) accumulation -- about
    // 48 significand bits, far below the FP64 rounding of the tangent itself
    const float2 *Gp = Gs + lp * S;
    float sh0 = 0.0f, sl0 = 0.0f, sh1 = 0.0f, sl1 = 0.0f;
    int k = 0;
    for (; k + 1 < S; k += 2) {
      {
        const float2 g2 = Gp[k], t2 = T2[21 * k + ij];
        const float pr = g2.x * t2.x, er = fmaf(g2.x, t2.x, -pr), cr = fmaf(g2.x, t2.y, g2.y * t2.x);
        const float sn = sh0 + pr, bv = sn - sh0;
        sl0 += ((sh0 - (sn - bv)) + (pr - bv)) + (er + cr);
        sh0 = sn;
      }
      {
        const float2 g2 = Gp[k + 1], t2 = T2[21 * (k + 1) + ij];
        const float pr = g2.x * t2.x, er = fmaf(g2.x, t2.x, -pr), cr = fmaf(g2.x, t2.y, g2.y * t2.x);
        const float sn = sh1 + pr, bv = sn - sh1;
        sl1 += ((sh1 - (sn - bv)) + (pr - bv)) + (er + cr);
        sh1 = sn;
      }
    }
    if (k < S) {
      const float2 g2 = Gp[k], t2 = T2[21 * k + ij];
      const float pr = g2.x * t2.x, er = fmaf(g2.x, t2.x, -pr), cr = fmaf(g2.x, t2.y, g2.y * t2.x);
      const float sn = sh0 + pr, bv = sn - sh0;
      sl0 += ((sh0 - (sn - bv)) + (pr - bv)) + (er + cr);
      sh0 = sn;
    }
    const double acc = (nn ? mc[mt].Kb : 0.0) + ((f2d(sh0) + f2d(sh1)) + (f2d(sl0) + f2d(sl1)));
    if (dpts)
      dpts[21 * (p - p0) + ij] = acc;
    else
      D[((p & 3) * 21 + ij) * epad + (p >> 2)] = acc;
  }
}

// Points per block: whole elements (a multiple of 4), about 4096 springs per block by
// default; the G_k of a block's springs and its points' strains sit in shared memory as
// float pairs (8 bytes each, <= 200 KB).
int spring_tile_default(int S) {
  int te = 4096 / (4 * S);
  int p2 = 1;
  while (p2 * 2 <= te && p2 < 64) p2 *= 2;
  return 4 * p2;
}
bool spring_tile_ok(int tp, int S) { return tp >= 4 && tp % 4 == 0 && (size_t)tp * (S + 12) * 8 <= 200 * 1024; }
// shared memory of a launch: float-pair tangents, or the tensor path's digit planes
static size_t spring_smem(int tp, int S, bool tc) {
  const size_t strains = sizeof(float2) * (size_t)tp * 12;
  if (tc) return (size_t)kDigits * tp * tc_stride((S + 15) / 16) * 2 + strains;
  return sizeof(float2) * (size_t)tp * S + strains;
}
static bool spring_tc_ok(const SpringTables &tab, int tp) {
  return tab.tc && tab.tfrag && tab.tsc && tab.S <= kTcMaxS && tp % 16 == 0 && spring_smem(tp, tab.S, true) <= 200 * 1024;
}

cudaError_t launch_springs(const SpringTables &tab, const MatConst *mc, const int32_t *mat_of_elem,
                           const int32_t *mat_of_point, const double *eps, SpringSoA st, int64_t base, int64_t p0,
                           int64_t p1, double *D, int64_t epad, double *dpts, cudaStream_t s, bool eps_pairs) {
  if (p1 <= p0) return cudaSuccess;
  const int TP = spring_tile_ok(tab.tp, tab.S) ? tab.tp : spring_tile_default(tab.S);
  const bool tc = spring_tc_ok(tab, TP);
  const size_t smem = spring_smem(TP, tab.S, tc);
  // the shared-memory opt-in is a per-device attribute, set once per device (any thread)
  static std::atomic<unsigned long long> attr_done{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(attr_done.load() & bit)) {
    cudaFuncSetAttribute(k_springs<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_springs<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_springs<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_springs<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_done.fetch_or(bit);
  }
  const unsigned nb = (unsigned)((p1 - p0 + TP - 1) / TP);
#define NS_SPRINGS(MB, TC)                                                                                         \
  k_springs<MB, TC><<<nb, kBlock, smem, s>>>(tab.q2, tab.T2, tab.S, TP, mc, mat_of_elem, mat_of_point, eps, st.tau, \
                                             st.gR, st.tR, st.gmax, st.dir, st.mode, base, p0, p1, D, epad, dpts,  \
                                             tab.pow, tab.powf, tab.tfrag, tab.tsc, eps_pairs ? 1 : 0, tab.cnt)
  if (tab.minb == 4) {
    if (tc)
      NS_SPRINGS(4, true);
    else
      NS_SPRINGS(4, false);
  } else {
    if (tc)
      NS_SPRINGS(1, true);
    else
      NS_SPRINGS(1, false);
  }
#undef NS_SPRINGS
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

// FP16 copy of the tangent for the inner operator, scaled by 1/G0 of the element's material
// so that the entries (Kb/G0 + 4/3 at most, ~6 for Poisson's ratio 0.4) sit well inside the
// FP16 range; blockIdx.y = pair j of entries (2j, 2j+1).
__global__ void k_D_to_f16(const double *__restrict__ D, const int32_t *__restrict__ mat,
                           const MatConst *__restrict__ mc, __half2 *D16, int64_t epad, int64_t E) {
  const int64_t j = blockIdx.y;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const double s = mc[mat[e]].iG0;
    D16[j * epad + e] = __floats2half2_rn((float)(D[2 * j * epad + e] * s), (float)(D[(2 * j + 1) * epad + e] * s));
  }
}

cudaError_t launch_D_to_f16(const double *D, const int32_t *mat, const MatConst *mc, void *D16, int64_t epad,
                            int64_t E, cudaStream_t s) {
  if (E <= 0) return cudaSuccess;
  const unsigned nx = (unsigned)std::min<int64_t>((E + kBlock - 1) / kBlock, 152 * 2);
  k_D_to_f16<<<dim3(nx, 42), kBlock, 0, s>>>(D, mat, mc, static_cast<__half2 *>(D16), epad, E);
  return cudaGetLastError();
}

}  // namespace ns
