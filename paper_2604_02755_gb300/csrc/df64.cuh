// Power x^beta in double-float arithmetic (pairs of FP32 numbers, ~48 significand bits)
// for the spring law's root solve.  GB300 issues FP32 arithmetic at 64 times its FP64
// rate, so evaluating the power on the FP32 pipes leaves the scarce FP64 pipe to the
// parts of the update that need FP64 state.
//
// Method (table-driven logarithm and exponential after Tang, ACM TOMS 1989/1990, with
// the error-free transformations of Dekker and Knuth for the pairs):
//   x = 2^e m (1 + eps),   m in [1, 2),   j = top 7 bits of m's fraction,
//   A = ln(m (1 + eps)) = -ln r_j + ln(1 + u) + eps - eps^2/2,   u = m r_j - 1 (|u| < 2^-7.9),
//   beta e = nb + phi (nb an integer, 0 <= phi < 1),   y = phi ln2 + beta A   (|y| < 2.5),
//   k = round(64 y / ln2),   f = y - k ln2/64   (|f| <= ln2/128),
//   x^beta = 2^(nb + floor(k/64)) 2^((k mod 64)/64) exp(f).
// Taking the integer part of beta e out before the exponential keeps its argument small,
// so the pair's ~48 bits give a relative error near 2^-47 for any x; ln2/64 is split into
// three floats whose leading two carry few significant bits, so that k times them is
// exact; r_j, -ln r_j and 2^(i/64) are tables built on the host in extended precision.
// The series keep the pair precision only where the terms are large enough to need it.
//
// Written for both the device and the host (the host build must not contract
// multiply-adds: -ffp-contract=off), so that the same arithmetic can be checked on a CPU.
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define NS_HD __host__ __device__ __forceinline__
#else
#define NS_HD inline
#endif

namespace ns {

// floats of the power tables (device array of kPowFLen floats)
//   [0, 128)   r_j                   [128, 256) -ln r_j, high     [256, 384) -ln r_j, low
//   [384, 448) 2^(i/64), high        [448, 512) 2^(i/64), low
//   [512, 520) ln2 as a pair, ln2/64 in three parts (d0 d1 d2, the first two with few
//              significant bits), 64/ln2, 0, 0
constexpr int kPowFLen = 520;

#if defined(__CUDA_ARCH__)
NS_HD float df_add(float a, float b) { return __fadd_rn(a, b); }
NS_HD float df_sub(float a, float b) { return __fsub_rn(a, b); }
NS_HD float df_mul(float a, float b) { return __fmul_rn(a, b); }
NS_HD float df_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
NS_HD uint32_t df_bits(float x) { return __float_as_uint(x); }
NS_HD float df_from_bits(uint32_t b) { return __uint_as_float(b); }
NS_HD float df_rint(float x) { return rintf(x); }
NS_HD float df_rcp(float x) { return __frcp_rn(x); }
#else
NS_HD float df_add(float a, float b) { return a + b; }
NS_HD float df_sub(float a, float b) { return a - b; }
NS_HD float df_mul(float a, float b) { return a * b; }
NS_HD float df_fma(float a, float b, float c) { return fmaf(a, b, c); }
NS_HD uint32_t df_bits(float x) {
  uint32_t b;
  memcpy(&b, &x, 4);
  return b;
}
NS_HD float df_from_bits(uint32_t b) {
  float x;
  memcpy(&x, &b, 4);
  return x;
}
NS_HD float df_rint(float x) { return rintf(x); }
NS_HD float df_rcp(float x) { return 1.0f / x; }
#endif

// a + b = s + e exactly (any order of magnitudes)
NS_HD void two_sum(float a, float b, float &s, float &e) {
  s = df_add(a, b);
  const float bb = df_sub(s, a);
  e = df_add(df_sub(a, df_sub(s, bb)), df_sub(b, bb));
}
// a * b = p + e exactly
NS_HD void two_prod(float a, float b, float &p, float &e) {
  p = df_mul(a, b);
  e = df_fma(a, b, -p);
}

// Exponent beta in the forms the power needs: a pair (bh + bl, ~48 bits) for beta times the
// small log A, and three parts for beta times the binary exponent e, which must stay exact
// to ~2^-56 |e| (an error in beta enters x^beta multiplied by ln x): b0 a multiple of 2^-15,
// b1 a multiple of 2^-31 (both with at most 16 significant bits, so b0 e and b1 e are
// exact for |e| < 256), b2 the float rest.
struct PowBeta {
  float bh, bl, b0, b1, b2;
};

// (xh + xl)^beta for a pair with xh a normal float in [2^-100, 2^100] (else false);
// result (wh, wl).
NS_HD bool df64_pow(float xh, float xl, const PowBeta &B, const float *__restrict__ tab, float &wh, float &wl) {
  const float bh = B.bh, bl = B.bl;
  const uint32_t xb = df_bits(xh);
  const int ef = (int)((xb >> 23) & 0xff);
  if ((xb >> 31) || ef < 27 || ef > 227) return false;  // outside [2^-100, 2^100]: caller falls back
  const float fe = (float)(ef - 127);
  const int j = (int)((xb >> 16) & 127);
  const float m = df_from_bits((xb & 0x007fffffu) | 0x3f800000u);
  const float eps = df_mul(xl, df_rcp(xh));  // |eps| ~ 2^-24; only its leading bits matter
  const float *c = tab + 512;
  // beta e = nb + phi, nb an integer, phi in [0, 1) as a pair: the whole exponent
  // 2^(beta e) is split off, so the argument left for exp stays within |y| < 2.5
  const float s0 = df_mul(B.b0, fe);  // exact, a multiple of b0's last bit
  const float nb = floorf(s0);
  float ph, pl;
  two_sum(df_sub(s0, nb), df_mul(B.b1, fe), ph, pl);  // s0 - nb and b1 e exact
  pl = df_fma(B.b2, fe, pl);
  // u = m r_j - 1 as a pair: the product's rounding error is exact, p - 1 is exact (Sterbenz)
  float p, pe;
  two_prod(m, tab[j], p, pe);
  float u1, u2;
  two_sum(df_sub(p, 1.0f), pe, u1, u2);  // |u2| <= ulp(u1)/2
  // ln(1 + u) = u - u^2/2 + u^3/3 - u^4/4 + u^5/5 - u^6/6 (+ O(2^-55)); u1 u2 ~ 2^-40 kept
  float sq, sqe;
  two_prod(u1, u1, sq, sqe);
  float P = df_fma(u1, -1.0f / 6.0f, 0.2f);
  P = df_fma(u1, P, -0.25f);
  P = df_fma(u1, P, 1.0f / 3.0f);
  P = df_mul(df_mul(df_mul(u1, u1), u1), P);
  float l1h, l1l;
  two_sum(u1, df_mul(-0.5f, sq), l1h, l1l);
  l1l = df_add(l1l, df_add(df_add(u2, df_mul(-u1, u2)), df_add(df_mul(-0.5f, sqe), P)));
  // A = ln m (1 + eps) = -ln r_j + ln(1 + u) + eps - eps^2/2,  |A| < ln2
  float a1, a2;
  two_sum(tab[128 + j], l1h, a1, a2);
  a2 = df_add(df_add(a2, tab[256 + j]), df_add(l1l, df_fma(-0.5f * eps, eps, eps)));
  // y = phi ln2 + beta A
  float q1, q2;
  two_prod(bh, a1, q1, q2);
  q2 = df_add(q2, df_fma(bh, a2, df_mul(bl, a1)));
  float r1, r2;
  two_prod(ph, c[0], r1, r2);
  r2 = df_add(r2, df_fma(ph, c[1], df_mul(pl, c[0])));
  float yh, yl;
  two_sum(r1, q1, yh, yl);
  yl = df_add(yl, df_add(r2, q2));
  // exp(y): k = round(64 y / ln2), f = y - k ln2/64 (the first subtraction is exact)
  const float kf = df_rint(df_mul(yh, c[5]));
  const int k = (int)kf;
  const float fh0 = df_sub(yh, df_mul(kf, c[2]));
  float gh, gl;
  two_sum(fh0, -df_mul(kf, c[3]), gh, gl);
  gl = df_add(gl, df_sub(yl, df_mul(kf, c[4])));
  float g1, g2;
  two_sum(gh, gl, g1, g2);  // |f| <= ln2/128 + tiny
  // exp(f) - 1 = f + f^2/2 + f^3/6 + f^4/24 + f^5/120 (+ O(2^-54))
  float fs, fse;
  two_prod(g1, g1, fs, fse);
  float Q = df_fma(g1, 1.0f / 120.0f, 1.0f / 24.0f);
  Q = df_fma(g1, Q, 1.0f / 6.0f);
  Q = df_mul(df_mul(df_mul(g1, g1), g1), Q);
  float E1, E2;
  two_sum(g1, df_mul(0.5f, fs), E1, E2);
  E2 = df_add(df_add(E2, g2), df_add(df_fma(0.5f, fse, df_mul(g1, g2)), Q));
  // 2^(i/64) (1 + E)
  const int i = k & 63;
  const float Th = tab[384 + i], Tl = tab[448 + i];
  float th, tl;
  two_prod(Th, E1, th, tl);
  float s1, s2;
  two_sum(Th, th, s1, s2);
  s2 = df_add(df_add(s2, Tl), df_add(tl, df_fma(Th, E2, df_mul(Tl, E1))));
  // times 2^(nb + floor(k/64)), a normal float for the accepted range of x
  const int n = (int)nb + (k >> 6);
  if (n < -120 || n > 120) return false;
  const float sc = df_from_bits((uint32_t)(n + 127) << 23);
  wh = df_mul(s1, sc);
  wl = df_mul(s2, sc);
  return true;
}

// ---------------------------------------------------------------------------------------
// Pair arithmetic used by the root step below (results renormalised: |lo| <= ulp(hi)/2).
NS_HD void fast_two_sum(float a, float b, float &s, float &e) {  // |a| >= |b|
  s = df_add(a, b);
  e = df_sub(b, df_sub(s, a));
}
NS_HD void pair_mul(float ah, float al, float bh, float bl, float &ph, float &pl) {
  float p, e;
  two_prod(ah, bh, p, e);
  e = df_add(e, df_fma(ah, bl, df_mul(al, bh)));
  fast_two_sum(p, e, ph, pl);
}
NS_HD void pair_add(float ah, float al, float bh, float bl, float &sh, float &sl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e = df_add(e, df_add(al, bl));
  fast_two_sum(s, e, sh, sl);
}
NS_HD void pair_rcp(float bh, float bl, float &rh, float &rl) {  // 1 / (bh + bl), one Newton step
  const float r0 = df_rcp(bh);
  const float e = df_sub(df_fma(-bh, r0, 1.0f), df_mul(bl, r0));
  fast_two_sum(r0, df_mul(r0, e), rh, rl);
}

// Material constants of the spring law as float pairs (built on the host).
struct RoPairs {
  float iG0h, iG0l;    // 1 / G0
  float alh, all;      // alpha = 2^beta
  float ab1h, ab1l;    // alpha (1 + beta)
  float G0h, G0l;      // G0
  float itrh, itrl;    // 1 / (G0 gamma_ref)
  float hab1b, c2;     // alpha (1 + beta) beta / 2 and beta (beta - 1) / 2 (small corrections)
  PowBeta pb;          // beta
};

// One Halley step of the skeleton equation g(tau) = tau/G0 (1 + alpha (tau itref)^beta)
// = ga > 0 from the FP32 seed t, in pair arithmetic, with the tangent at the new root:
//   w0 = (t itref)^beta,  r = g(t) - ga,  h = r / g'(t) = r G0 / (1 + alpha (1 + beta) w0),
//   step = h (1 + h g''/(2 g')),  tau1 = t - step,  d = -step / t,
//   w1 = w0 (1 + d)^beta ~ w0 (1 + beta d + beta (beta - 1)/2 d^2),
//   G = G0 / (1 + alpha (1 + beta) w1)  (= 1 / g'(tau1), the spring's tangent).
// ga = gah + gal.  Returns false when the power declines its input (the caller falls back
// to FP64).  The residual r is a small difference of two pairs, so tau1 is accurate to
// about 2^-47 tau, and G to about 2^-45.
NS_HD bool df64_ro_halley(float t, float gah, float gal, const RoPairs &P, const float *__restrict__ tab,
                          float &tauh, float &taul, float &d, float &Gh, float &Gl) {
  float xh, xl, wh, wl;
  two_prod(t, P.itrh, xh, xl);
  xl = df_fma(t, P.itrl, xl);
  if (!df64_pow(xh, xl, P.pb, tab, wh, wl)) return false;
  // r = t iG0 (1 + alpha w0) - ga
  float ah, al, th, tl, gh, gl, rh, rl;
  pair_mul(P.alh, P.all, wh, wl, ah, al);
  pair_add(1.0f, 0.0f, ah, al, ah, al);
  two_prod(t, P.iG0h, th, tl);
  tl = df_fma(t, P.iG0l, tl);
  pair_mul(th, tl, ah, al, gh, gl);
  pair_add(gh, gl, -gah, -gal, rh, rl);
  // h = r G0 / (1 + ab1 w0)
  float bh, bl, qh, ql, hh, hl;
  pair_mul(P.ab1h, P.ab1l, wh, wl, bh, bl);
  pair_add(1.0f, 0.0f, bh, bl, bh, bl);
  pair_rcp(bh, bl, qh, ql);
  pair_mul(rh, rl, P.G0h, P.G0l, hh, hl);
  pair_mul(hh, hl, qh, ql, hh, hl);
  // Halley: the correction factor h g''/(2 g') ~ the seed's relative error, needed to ~1e-7
  const float rt = df_rcp(t);
  const float hc = df_mul(df_mul(df_mul(hh, P.hab1b), df_mul(wh, rt)), qh);
  float sh, sl;
  two_sum(hh, df_mul(hh, hc), sh, sl);
  sl = df_add(sl, hl);
  two_sum(t, -sh, tauh, taul);
  taul = df_sub(taul, sl);
  // d = -step / t as a pair (1/t refined once)
  const float et = df_fma(-t, rt, 1.0f);
  float dh, dl;
  two_prod(sh, rt, dh, dl);
  dl = df_add(dl, df_fma(df_mul(sh, rt), et, df_mul(sl, rt)));
  d = -dh;
  // w1 = w0 (1 + beta d + c2 d^2), c3 d^3 < 1e-16 dropped
  float zh, zl, vh, vl;
  pair_mul(P.pb.bh, P.pb.bl, -dh, -dl, zh, zl);
  zl = df_fma(df_mul(P.c2, dh), dh, zl);
  pair_mul(wh, wl, zh, zl, vh, vl);
  pair_add(wh, wl, vh, vl, wh, wl);
  // G = G0 / (1 + ab1 w1)
  pair_mul(P.ab1h, P.ab1l, wh, wl, bh, bl);
  pair_add(1.0f, 0.0f, bh, bl, bh, bl);
  pair_rcp(bh, bl, qh, ql);
  pair_mul(P.G0h, P.G0l, qh, ql, Gh, Gl);
  return true;
}

// ---------------------------------------------------------------------------------------
// A double-float number as an arithmetic type (renormalised after every operation), so
// that templated element kernels written for float and double also run in pair
// arithmetic on the FP32 pipes.  Constants convert exactly enough from double.
struct dd {
  float h, l;
  dd() = default;
  NS_HD dd(float v) : h(v), l(0.0f) {}
  NS_HD dd(int v) : h((float)v), l(0.0f) {}
  NS_HD dd(double v) : h((float)v), l((float)(v - (double)(float)v)) {}
  NS_HD dd(float hi, float lo) : h(hi), l(lo) {}
  NS_HD explicit operator double() const { return (double)h + (double)l; }
};
NS_HD dd operator+(dd a, dd b) {
  dd r;
  pair_add(a.h, a.l, b.h, b.l, r.h, r.l);
  return r;
}
NS_HD dd operator-(dd a) { return dd(-a.h, -a.l); }
NS_HD dd operator-(dd a, dd b) { return a + (-b); }
NS_HD dd operator*(dd a, dd b) {
  dd r;
  pair_mul(a.h, a.l, b.h, b.l, r.h, r.l);
  return r;
}
NS_HD dd &operator+=(dd &a, dd b) { return a = a + b; }
NS_HD dd &operator-=(dd &a, dd b) { return a = a - b; }
NS_HD dd &operator*=(dd &a, dd b) { return a = a * b; }
NS_HD bool operator==(dd a, dd b) { return a.h == b.h && a.l == b.l; }
NS_HD bool operator!=(dd a, dd b) { return !(a == b); }

#if defined(__CUDACC__)
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
#endif

// A double as a pair: on the device the high part is the double with its low 29
// significand bits cleared and the low part the rounded rest, both on the integer and FP32
// pipes (dsplit); zero and values outside the normal float range are rounded to one float.
NS_HD dd dd_from_double(double v) {
#if defined(__CUDA_ARCH__)
  dd r;
  dsplit(v, r.h, r.l);
  return r;
#else
  return dd(v);
#endif
}

}  // namespace ns
