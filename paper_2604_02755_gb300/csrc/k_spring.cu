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
// accuracy by cutting both operands into 7-bit integer digits, exact in bf16:
//   G_pk 2^-eG = sum_i a_i 2^-7(i+1)  (balanced digits: a_0 in 0..128, |a_i| <= 65 after;
//                                       eG per material with 2^eG > G0 >= G),
//   T_k[ij] 2^-eT[ij] = sum_j b_j 2^-7(j+1)  (|b_j| <= 127, one exponent per column ij).
// Every digit product is exact in FP32, and the sum over the springs of one digit pair
// (i, j) is an integer below S 128 127 < 2^22 for S <= 256, so the MMA accumulator C_ij
// holds it exactly.  The pairs with i + j <= 7 (34 of the 49) are kept and combined in
// double-float arithmetic: D = Kb + 2^(eG + eT[ij] - 14) sum_ij 2^-7(i+j) C_ij.  The
// dropped pairs (each term below 5 65 127 2^-70 < 2^-54) and the digits' own truncation
// leave an error near 2^-49 of 2^(eG + eT[ij]) per spring.  All eight warps of the block
// take part (warp w takes the pairs w, w + 8, ...), and the warps' double-float partial
// sums are added in shared memory.  (Dropping the two pairs (1, 6) and (6, 1) as well
// would give each warp four, but their terms reach 2^-50 of the scale and the error of D
// relative to sum_k |G_k T_k| grows fivefold for tangents far below G0.)
constexpr int kDigits = 7;
constexpr int kMaxLevel = 7;  // digit pairs i + j <= 7 kept
constexpr int kTcMaxS = 256;
constexpr int kTcTile = 16;   // points per block on the tensor-core path: one 16-row MMA tile
struct TcPairs {
  unsigned char i[64], j[64];
  int n;
};
constexpr TcPairs make_tc_pairs() {
  TcPairs t{};
  for (int L = 0; L <= kMaxLevel; ++L)
    for (int i = 0; i <= L; ++i)
      if (i < kDigits && L - i < kDigits) {
        t.i[t.n] = (unsigned char)i;
        t.j[t.n] = (unsigned char)(L - i);
        ++t.n;
      }
  return t;
}
constexpr TcPairs kTcPairs = make_tc_pairs();
constexpr int kPairs = kTcPairs.n;
static_assert(kPairs == 34, "digit pairs with i + j <= 7");
__constant__ TcPairs c_tc_pairs = kTcPairs;
// shared bytes of the warps' partial sums: [8 warps][3 column tiles][4 registers][32 lanes] pairs
constexpr size_t kTcRedBytes = (size_t)(kBlock / 32) * 3 * 4 * 32 * sizeof(float2);

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

// The tangent G (a float pair) as seven balanced 7-bit digits of X = G 2^(49 - eG) in bf16:
// X = sum_i a_i 2^(42 - 7i).  Each digit is the rounded quotient of the remainder (the
// high part's remainder plus the rounded low part, for the decision only) by its weight;
// the remainder is updated exactly (a digit times its weight has at most 8 significant
// bits and the new remainder is below half a weight), so the digits represent the high
// part plus the rounded low part to within half a unit of 2^-49 2^eG.  |v| <= 128, so the
// magic-constant rounding (1.5 2^23) is exact, and an integer of at most 8 significant
// bits is its own bf16 (the top half of its float bits).
__device__ __forceinline__ void tangent_digits(float2 G, float gfix, unsigned short *dst, size_t plane) {
  float r = df_mul(G.x, gfix);
  const float c = rintf(df_mul(G.y, gfix));
#pragma unroll
  for (int i = 0; i < kDigits; ++i) {
    const float w = __uint_as_float((uint32_t)(127 - (42 - 7 * i)) << 23);  // 2^-(42 - 7i)
    const float W = __uint_as_float((uint32_t)(127 + (42 - 7 * i)) << 23);  // 2^(42 - 7i)
    const float v = df_mul(df_add(r, c), w);
    const float d = df_sub(df_add(v, 12582912.0f), 12582912.0f);
    r = df_fma(-d, W, r);
    dst[i * plane] = (unsigned short)(__float_as_uint(d) >> 16);
  }
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
// cores (TP = 16, S <= 256; tfrag holds the digits of T in MMA fragment order).
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
    // the state is read and written once per launch: streaming accesses (evict first), so
    // that L1 keeps what every spring of the block reuses (directions, tables, digits of T)
    double tau = __ldcs(tau_a + si), gR = __ldcs(gR_a + si), tR = __ldcs(tR_a + si), gmax = __ldcs(gmax_a + si);
    int dir = __ldcs(dir_a + si), mode = __ldcs(mode_a + si);
    unsigned ev = 0;
    const float2 G = spring_update_pair(gh, gl, dh, dl, !sure, q2 + 6 * k, Es + 12 * lp + 6, rp, tb, ptabf, tau, gR,
                                        tR, gmax, dir, mode, ev);
    evn += (ev & 1u) | ((ev & 2u) << 9) | ((ev & 4u) << 18);
    if (dh != 0.0f) {
      __stcs(tau_a + si, tau);
      __stcs(gR_a + si, gR);
      __stcs(tR_a + si, tR);
      __stcs(gmax_a + si, gmax);
      __stcs(dir_a + si, dir);
      __stcs(mode_a + si, mode);
    }
    if (TC) {
      tangent_digits(G, rp.gfix, planes + (size_t)lp * KST + k, (size_t)TP * KST);
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
    // warp w multiplies the digit pairs w, w + 8, ... for the three 8-column tiles of D
    // (16 x 24 >= 16 x 21): per pair, the MMAs over the spring slices accumulate the exact
    // integer C_ij, which is scaled by 2^-7(i+j) and added into the warp's double-float
    // partial sums
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t arow =
        (uint32_t)__cvta_generic_to_shared(planes + (size_t)((lane & 7) + ((lane >> 3) & 1) * 8) * KST + (lane >> 4) * 8);
    float vh[3][4], vl[3][4];
#pragma unroll
    for (int n = 0; n < 3; ++n)
#pragma unroll
      for (int r = 0; r < 4; ++r) vh[n][r] = vl[n][r] = 0.0f;
    for (int pr = warp; pr < kPairs; pr += kBlock >> 5) {
      const int di = c_tc_pairs.i[pr], dj = c_tc_pairs.j[pr];
      const uint32_t ai = arow + (uint32_t)((size_t)di * TP * KST * 2);
      const uint2 *bj = tfrag + (size_t)dj * KS * 96 + lane;
      float c0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, c1[4] = {0.0f, 0.0f, 0.0f, 0.0f}, c2[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      for (int ks = 0; ks < KS; ++ks) {
        uint32_t a[4];
        ldsm_x4(a, ai + (uint32_t)(ks * 32));
        const uint2 *b = bj + (size_t)ks * 96;
        mma_bf16(c0, a, __ldg(b));
        mma_bf16(c1, a, __ldg(b + 32));
        mma_bf16(c2, a, __ldg(b + 64));
      }
      const float sc = __uint_as_float((uint32_t)(127 - 7 * (di + dj)) << 23);  // 2^-7(i+j), exact scaling
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        float sh, e;
        two_sum(vh[0][r], df_mul(c0[r], sc), sh, e);
        vh[0][r] = sh;
        vl[0][r] = df_add(vl[0][r], e);
        two_sum(vh[1][r], df_mul(c1[r], sc), sh, e);
        vh[1][r] = sh;
        vl[1][r] = df_add(vl[1][r], e);
        two_sum(vh[2][r], df_mul(c2[r], sc), sh, e);
        vh[2][r] = sh;
        vl[2][r] = df_add(vl[2][r], e);
      }
    }
    __syncthreads();  // every warp is done with the digit planes: their space takes the partial sums
    float2 *red = Gs;  // [warp][column tile][register][lane]
#pragma unroll
    for (int n = 0; n < 3; ++n)
#pragma unroll
      for (int r = 0; r < 4; ++r) red[((warp * 3 + n) * 4 + r) * 32 + lane] = make_float2(vh[n][r], vl[n][r]);
    __syncthreads();
    for (int o = threadIdx.x; o < kTcTile * 21; o += blockDim.x) {
      const int lp = o & (kTcTile - 1), ij = o >> 4;
      if (lp >= np) continue;
      // fragment position of (row lp, column ij): rows lane/4 (+8 in registers 2, 3),
      // columns 2 (lane % 4) + register % 2
      const int n = ij >> 3, col = ij & 7;
      const int src = ((lp & 7) << 2) | (col >> 1), r = ((lp >> 3) << 1) | (col & 1);
      float sh = 0.0f, sl = 0.0f;
#pragma unroll
      for (int w = 0; w < (kBlock >> 5); ++w) {
        const float2 v = red[((w * 3 + n) * 4 + r) * 32 + src];
        float t, e;
        two_sum(sh, v.x, t, e);
        sh = t;
        sl = df_add(sl, df_add(e, v.y));
      }
      const int64_t p = pt + lp;
      const MatConst &m = mc[mat_p ? mat_p[p] : mat_e[p >> 2]];
      const bool nn = ij < 3 || ij == 6 || ij == 7 || ij == 11;  // (i,j) both < 3
      const double val = (nn ? m.Kb : 0.0) + m.dsc * (__ldg(tsc + ij) * (f2d(sh) + f2d(sl)));
      if (dpts)
        dpts[21 * (p - p0) + ij] = val;
      else
        D[((p & 3) * 21 + ij) * epad + (p >> 2)] = val;
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
  if (tc) return std::max((size_t)kDigits * tp * tc_stride((S + 15) / 16) * 2, kTcRedBytes) + strains;
  return sizeof(float2) * (size_t)tp * S + strains;
}
static bool spring_tc_ok(const SpringTables &tab, int tp) {
  return tab.tc && tab.tfrag && tab.tsc && tab.S <= kTcMaxS && tp == kTcTile && spring_smem(tp, tab.S, true) <= 200 * 1024;
}

cudaError_t launch_springs(const SpringTables &tab, const MatConst *mc, const int32_t *mat_of_elem,
                           const int32_t *mat_of_point, const double *eps, SpringSoA st, int64_t base, int64_t p0,
                           int64_t p1, double *D, int64_t epad, double *dpts, cudaStream_t s, bool eps_pairs) {
  if (p1 <= p0) return cudaSuccess;
  // the tensor-core assembly works on 16-point tiles; otherwise the tuned or default tile
  const int TP = spring_tc_ok(tab, kTcTile) ? kTcTile : (spring_tile_ok(tab.tp, tab.S) ? tab.tp : spring_tile_default(tab.S));
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
  // shared-memory carveout: what the resident blocks need and no more, so that the rest of
  // the SM's 256 KB stays L1 for the data every block reuses (set when it changes: a
  // per-device attribute of each instantiation).  The resident blocks are counted from the
  // registers and the largest carveout (228 KB) -- not from the occupancy query, which
  // answers for the carveout currently set and would keep a small one small.
  {
    const int inst = (tab.minb == 4 ? 2 : 0) + (tc ? 1 : 0);
    const void *fn = inst == 3 ? (const void *)k_springs<4, true>
                     : inst == 2 ? (const void *)k_springs<4, false>
                     : inst == 1 ? (const void *)k_springs<1, true>
                                 : (const void *)k_springs<1, false>;
    static std::atomic<int> regs_of[64][4];   // zero-initialised: 0 = not queried yet
    static std::atomic<int> last_pct[64][4];  // 0 = not set yet (pct >= 1)
    int regs = regs_of[dev & 63][inst].load();
    if (regs == 0) {
      cudaFuncAttributes fa;
      if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess && fa.numRegs > 0) regs = fa.numRegs;
      regs_of[dev & 63][inst].store(regs);
    }
    if (regs > 0) {
      const int by_regs = 65536 / (((regs + 7) / 8) * 8 * kBlock);
      const int by_smem = (int)((228 * 1024) / (smem + 1024));
      const int bps = std::max(1, std::min(by_regs, by_smem));
      const size_t need = (size_t)bps * (smem + 1024);
      const int pct = (int)std::max<size_t>(1, std::min<size_t>(100, (need * 100 + 228 * 1024 - 1) / (228 * 1024)));
      if (last_pct[dev & 63][inst].exchange(pct) != pct)
        cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    }
    cudaGetLastError();
  }
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

__global__ void k_tune_sample(const float2 *__restrict__ eps, const int32_t *__restrict__ mat_e, int64_t p0,
                              int64_t np, float2 *out, int32_t *mat_out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float2 *e = eps + 12 * (p0 + i);
  float2 *o = out + 12 * i;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    float h, l;
    pair_add(e[c].x, e[c].y, e[6 + c].x, e[6 + c].y, h, l);
    o[c] = make_float2(h, l);
    o[6 + c] = e[6 + c];
  }
  if ((i & 3) == 0) mat_out[i >> 2] = mat_e[(p0 + i) >> 2];
}

cudaError_t launch_tune_sample(const double *eps_pairs, const int32_t *mat_e, int64_t e0, int64_t ne, float2 *eps_out,
                               int32_t *mat_out, int64_t out_elem, cudaStream_t s) {
  const int64_t np = 4 * ne;
  if (np <= 0) return cudaSuccess;
  k_tune_sample<<<(unsigned)((np + kBlock - 1) / kBlock), kBlock, 0, s>>>(
      reinterpret_cast<const float2 *>(eps_pairs), mat_e, 4 * e0, np, eps_out + 12 * 4 * out_elem,
      mat_out + out_elem);
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
