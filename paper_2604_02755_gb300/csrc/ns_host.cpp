// Host-side set-up of the time stepper: multi-spring geometry, material
// constants and greedy element colouring.  Runs once per context.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "ns_internal.h"

namespace ns {

namespace {

void matmul6(const double *A, const double *B, double *C) {
  double T[36];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double s = 0.0;
      for (int k = 0; k < 6; ++k) s += A[i * 6 + k] * B[k * 6 + j];
      T[i * 6 + j] = s;
    }
  memcpy(C, T, sizeof(T));
}

// Inverse square root of a symmetric positive definite 6x6 by the coupled
// Newton-Schulz (Denman-Beavers type) iteration on A/c with c = ||A||_F:
//   Y <- Y (3I - Z Y)/2,  Z <- (3I - Z Y) Z /2,   Y -> (A/c)^(1/2), Z -> (A/c)^(-1/2).
void inv_sqrt6(const double *A, double *out) {
  double c = 0.0;
  for (int i = 0; i < 36; ++i) c += A[i] * A[i];
  c = sqrt(c);
  double Y[36], Z[36], M[36];
  for (int i = 0; i < 36; ++i) {
    Y[i] = A[i] / c;
    Z[i] = (i % 7 == 0) ? 1.0 : 0.0;
  }
  for (int it = 0; it < 200; ++it) {
    matmul6(Z, Y, M);
    double dev = 0.0;
    for (int i = 0; i < 36; ++i) {
      const double id = (i % 7 == 0) ? 1.0 : 0.0;
      dev += (M[i] - id) * (M[i] - id);
      M[i] = 0.5 * (3.0 * id - M[i]);
    }
    matmul6(Y, M, Y);
    matmul6(M, Z, Z);
    if (dev < 1e-30) break;
  }
  const double sc = 1.0 / sqrt(c);
  for (int i = 0; i < 36; ++i) out[i] = Z[i] * sc;
}

}  // namespace

// Spring directions (Sec. 2.1 multi-spring model; geometry per the documented reading):
// plane normal n_k on a hemispherical Fibonacci lattice (z = 1 - (k+1/2)/S, azimuth
// k pi (3 - sqrt5)), slip s_k in the plane at angle 2 pi frac(k sqrt2) from
// t1 = (-sin phi, cos phi, 0) towards t2 = n x t1, shear projection
// p_k = (2 nx sx, 2 ny sy, 2 nz sz, ny sz + nz sy, nx sz + nz sx, nx sy + ny sx);
// q_k = T p_k with T = (2S/5 Ddev)^(1/2) P^(+1/2), P = sum p p^T, so that
// (5/(2S)) sum q q^T = Ddev = diag(2,2,2,1,1,1) - (2/3) m m^T exactly.
int host_spring_directions(int S, double *q, double *w) {
  if (S < 5) return -1;
  std::vector<double> p(6 * (size_t)S);
  double P[36] = {0};
  const double golden = M_PI * (3.0 - sqrt(5.0));
  for (int k = 0; k < S; ++k) {
    const double z = 1.0 - (k + 0.5) / S, r = sqrt(1.0 - z * z), phi = golden * k;
    const double n[3] = {r * cos(phi), r * sin(phi), z};
    const double t1[3] = {-sin(phi), cos(phi), 0.0};
    const double t2[3] = {n[1] * t1[2] - n[2] * t1[1], n[2] * t1[0] - n[0] * t1[2], n[0] * t1[1] - n[1] * t1[0]};
    double f = sqrt(2.0) * k;
    f -= floor(f);
    const double cs = cos(2.0 * M_PI * f), sn = sin(2.0 * M_PI * f);
    double sl[3];
    for (int c = 0; c < 3; ++c) sl[c] = cs * t1[c] + sn * t2[c];
    double *pk = &p[6 * (size_t)k];
    pk[0] = 2.0 * n[0] * sl[0];
    pk[1] = 2.0 * n[1] * sl[1];
    pk[2] = 2.0 * n[2] * sl[2];
    pk[3] = n[1] * sl[2] + n[2] * sl[1];
    pk[4] = n[0] * sl[2] + n[2] * sl[0];
    pk[5] = n[0] * sl[1] + n[1] * sl[0];
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) P[i * 6 + j] += pk[i] * pk[j];
  }
  // P has the volumetric direction m = (1,1,1,0,0,0) as its null vector; adding the
  // projector m m^T / 3 makes it invertible without changing the other eigenpairs.
  double Pm[36], Pih[36];
  for (int i = 0; i < 36; ++i) Pm[i] = P[i] + ((i / 6 < 3 && i % 6 < 3) ? 1.0 / 3.0 : 0.0);
  inv_sqrt6(Pm, Pih);
  for (int i = 0; i < 36; ++i) Pih[i] -= (i / 6 < 3 && i % 6 < 3) ? 1.0 / 3.0 : 0.0;
  // (Ddev)^(1/2) = sqrt2 (I - 11^T/3) on the normal block, I on the shear block
  double Dh[36] = {0};
  const double sc = sqrt(2.0 * S / 5.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Dh[i * 6 + j] = sc * sqrt(2.0) * ((i == j ? 1.0 : 0.0) - 1.0 / 3.0);
  for (int i = 3; i < 6; ++i) Dh[i * 6 + i] = sc;
  double T[36];
  matmul6(Dh, Pih, T);
  for (int k = 0; k < S; ++k)
    for (int i = 0; i < 6; ++i) {
      double s = 0.0;
      for (int j = 0; j < 6; ++j) s += T[i * 6 + j] * p[6 * (size_t)k + j];
      q[6 * (size_t)k + i] = s;
    }
  *w = 5.0 / (2.0 * S);
  return 0;
}

// Greedy first-fit colouring in element order.
int host_colouring(int64_t E, int64_t N, const int32_t *conn, int32_t *colour, int32_t *nc) {
  std::vector<uint64_t> used((size_t)N, 0);
  int32_t ncol = 0;
  for (int64_t e = 0; e < E; ++e) {
    uint64_t taken = 0;
    for (int a = 0; a < 10; ++a) taken |= used[(size_t)conn[e * 10 + a]];
    if (~taken == 0) return -1;
    const int c = __builtin_ctzll(~taken);
    colour[e] = c;
    if (c + 1 > ncol) ncol = c + 1;
    for (int a = 0; a < 10; ++a) used[(size_t)conn[e * 10 + a]] |= (1ull << c);
  }
  *nc = ncol;
  return 0;
}

// Coarse level of the two-level preconditioner: the vertices of the quadratic mesh, numbered
// in ascending node order; every node is interpolated from two coarse nodes (a vertex twice,
// an edge node from its edge's end vertices, smaller index first).  Fails (-1) when a node
// is a vertex of one element and an edge node of another, or an edge node is listed under
// two different edges.
int64_t host_coarse_map(int64_t E, int64_t N, const int32_t *conn, int32_t *cid, int32_t *par) {
  static const int kEdge[6][2] = {{0, 1}, {1, 2}, {0, 2}, {0, 3}, {1, 3}, {2, 3}};
  std::vector<uint8_t> kind((size_t)N, 0);  // 1 vertex, 2 edge node
  for (int64_t e = 0; e < E; ++e)
    for (int a = 0; a < 10; ++a) {
      uint8_t &k = kind[(size_t)conn[e * 10 + a]];
      const uint8_t want = a < 4 ? 1 : 2;
      if (k && k != want) return -1;
      k = want;
    }
  int64_t nc = 0;
  for (int64_t n = 0; n < N; ++n) {
    cid[n] = kind[(size_t)n] == 1 ? (int32_t)(nc++) : -1;
    par[2 * n] = par[2 * n + 1] = cid[n];
  }
  for (int64_t e = 0; e < E; ++e)
    for (int k = 0; k < 6; ++k) {
      const int64_t n = conn[e * 10 + 4 + k];
      const int32_t a = cid[conn[e * 10 + kEdge[k][0]]], b = cid[conn[e * 10 + kEdge[k][1]]];
      const int32_t lo = a < b ? a : b, hi = a < b ? b : a;
      if (par[2 * n] < 0) {
        par[2 * n] = lo;
        par[2 * n + 1] = hi;
      } else if (par[2 * n] != lo || par[2 * n + 1] != hi) {
        return -1;
      }
    }
  return nc;
}

void host_input_velocity(const double *acc, int64_t n, double dt, double *vin) {
  for (int cc = 0; cc < 3; ++cc) vin[cc] = 0.0;
  for (int64_t k = 1; k <= n; ++k)
    for (int cc = 0; cc < 3; ++cc) {
      const double a0 = acc[3 * (k - 1) + cc], a1 = (k < n) ? acc[3 * k + cc] : 0.0;
      vin[3 * k + cc] = vin[3 * (k - 1) + cc] + 0.5 * dt * (a0 + a1);
    }
}

// Derived constants: G0 = rho Vs^2, bulk Kb = rho (Vp^2 - 4/3 Vs^2); RO exponent
// beta = 2 pi h_max / (2 - pi h_max) (loop damping tends to h_max), alpha = 2^beta
// (secant G0/2 at gamma_ref); Rayleigh a = 2 h w1 w2/(w1 + w2), b = 2 h/(w1 + w2).
void host_material_constants(const ns_material &m, double f1, double f2, MatConst *o) {
  o->rho = m.rho;
  o->vs = m.vs;
  o->vp = m.vp;
  o->G0 = m.rho * m.vs * m.vs;
  o->Kb = m.rho * (m.vp * m.vp - 4.0 / 3.0 * m.vs * m.vs);
  o->gref = m.gamma_ref;
  o->beta_ro = 2.0 * M_PI * m.h_max / (2.0 - M_PI * m.h_max);
  o->alpha_ro = exp2(o->beta_ro);
  const double w1 = 2.0 * M_PI * f1, w2 = 2.0 * M_PI * f2;
  o->ray_a = 2.0 * m.rayleigh_h * w1 * w2 / (w1 + w2);
  o->ray_b = 2.0 * m.rayleigh_h / (w1 + w2);
  o->iG0 = 1.0 / o->G0;
  o->itref = 1.0 / (o->G0 * o->gref);
  o->ab1 = o->alpha_ro * (1.0 + o->beta_ro);
  o->ab1b = o->ab1 * o->beta_ro;
  o->c2 = o->beta_ro * (o->beta_ro - 1.0) * 0.5;
  o->c3 = o->c2 * (o->beta_ro - 2.0) / 3.0;
  o->hab1b = 0.5 * o->ab1b;
  o->itref_f = (float)o->itref;
  o->iG0_f = (float)o->iG0;
  o->alpha_f = (float)o->alpha_ro;
  o->beta_f = (float)o->beta_ro;
  o->G0_f = (float)o->G0;
  o->pad_f = 0.0f;
  o->eg = ilogb(o->G0) + 1;  // 2^eg > G0
  o->gfix = ldexpf(1.0f, 49 - o->eg);
  o->dsc = ldexp(1.0, o->eg);
  // float pairs for the double-float root step, from extended-precision values
  auto split = [](long double v, float &h, float &l) {
    h = (float)v;
    l = (float)(v - (long double)h);
  };
  const long double b = (long double)o->beta_ro, G0 = (long double)o->G0;
  const long double al = exp2l(b), itr = 1.0L / (G0 * (long double)o->gref);
  RoPairs &r = o->rp;
  split(1.0L / G0, r.iG0h, r.iG0l);
  split(al, r.alh, r.all);
  split(al * (1.0L + b), r.ab1h, r.ab1l);
  split(G0, r.G0h, r.G0l);
  split(itr, r.itrh, r.itrl);
  r.hab1b = (float)(al * (1.0L + b) * b * 0.5L);
  r.c2 = (float)(b * (b - 1.0L) * 0.5L);
  // beta as a pair, and as b0 (a multiple of 2^-15) + b1 (a multiple of 2^-31) + b2
  split(b, r.pb.bh, r.pb.bl);
  const long double b0 = roundl(b * 32768.0L) / 32768.0L;
  const long double b1 = roundl((b - b0) * 2147483648.0L) / 2147483648.0L;
  r.pb.b0 = (float)b0;
  r.pb.b1 = (float)b1;
  r.pb.b2 = (float)(b - b0 - b1);
}

// Tables of the double-float power (df64.cuh), in extended precision: r_j = 1/(1 + (j +
// 1/2)/128) rounded to float, -ln r_j of that float as a float pair, 2^(i/64) as a pair,
// ln2 as a pair, ln2/64 as d0 (multiple of 2^-18) + d1 (multiple of 2^-30) + d2, 64/ln2.
void host_powf_tables(float *out) {
  const long double LN2 = 0.693147180559945309417232121458176568L;
  for (int j = 0; j < 128; ++j) {
    const float r = (float)(1.0L / (1.0L + ((long double)j + 0.5L) / 128.0L));
    const long double l = -logl((long double)r);
    out[j] = r;
    out[128 + j] = (float)l;
    out[256 + j] = (float)(l - (long double)(float)l);
  }
  for (int i = 0; i < 64; ++i) {
    const long double t = exp2l((long double)i / 64.0L);
    out[384 + i] = (float)t;
    out[448 + i] = (float)(t - (long double)(float)t);
  }
  out[512] = (float)LN2;
  out[513] = (float)(LN2 - (long double)(float)LN2);
  const long double L64 = LN2 / 64.0L;
  const long double d0 = roundl(L64 * 262144.0L) / 262144.0L;
  const long double d1 = roundl((L64 - d0) * 1073741824.0L) / 1073741824.0L;
  out[514] = (float)d0;
  out[515] = (float)d1;
  out[516] = (float)(L64 - d0 - d1);
  out[517] = (float)(64.0L / LN2);
  out[518] = 0.0f;
  out[519] = 0.0f;
}

// Tables of the FP64 power used by the spring law (table-driven logarithm and exponential
// after Tang): r_j = 1/(1 + (j + 1/2)/128) rounded to double, -ln r_j split in two
// doubles, 2^(i/64), and ln2, ln2/64 split so that the high parts have trailing zero bits.
void host_pow_tables(double *out) {
  const long double LN2 = 0.693147180559945309417232121458176568L;
  for (int j = 0; j < 128; ++j) {
    const double r = (double)(1.0L / (1.0L + ((long double)j + 0.5L) / 128.0L));
    const long double l = -logl((long double)r);
    out[j] = r;
    out[128 + j] = (double)l;
    out[256 + j] = (double)(l - (long double)(double)l);
  }
  for (int i = 0; i < 64; ++i) out[384 + i] = (double)exp2l((long double)i / 64.0L);
  auto trunc_bits = [](double x, int drop) {
    uint64_t b;
    memcpy(&b, &x, 8);
    b &= ~((1ull << drop) - 1ull);
    memcpy(&x, &b, 8);
    return x;
  };
  const double l2h = trunc_bits((double)LN2, 11);
  out[448] = l2h;
  out[449] = (double)(LN2 - (long double)l2h);
  const double l64h = trunc_bits((double)(LN2 / 64.0L), 20);
  out[450] = l64h;
  out[451] = (double)(LN2 / 64.0L - (long double)l64h);
}

// Digits of the spring tables for the tensor-core tangent assembly (k_spring.cu).  Column
// ij has its own exponent et[ij] (max_k |T_k[ij]| 2^-et in [1/4, 1/2)); each
// T_k[ij] 2^-et[ij] is rounded to 49 bits and cut into seven 7-bit digits from the top,
// each carrying the sign of T_k[ij], stored as bf16 (exact for |d| <= 127) in the register
// order of the B operand of a 16x8x16 MMA: entry ((j * KS + ks) * 3 + nt) * 32 + lane
// holds digit j of rows k = 16 ks + 2 (lane % 4) + {0, 1} (low half first) and, in .y, of
// the rows 8 further on, column ij = 8 nt + lane / 4; rows k >= S and columns ij >= 21
// are 0.
void host_spring_digits(int S, const double *T, uint2 *frag, int *et) {
  for (int n = 0; n < 21; ++n) {
    double mx = 0.0;
    for (int k = 0; k < S; ++k) mx = fmax(mx, fabs(T[21 * (size_t)k + n]));
    et[n] = (mx > 0.0 ? ilogb(mx) : 0) + 2;
  }
  const int KS = (S + 15) / 16;
  auto digit = [&](int k, int n, int j) -> uint32_t {
    if (k >= S || n >= 21) return 0u;
    const double t = ldexp(T[21 * (size_t)k + n], -et[n]);
    const uint64_t X = (uint64_t)llround(fabs(t) * 0x1p49);
    const int d = (int)((X >> (42 - 7 * j)) & 127u);
    const float f = (float)(t < 0.0 ? -d : d);
    uint32_t bits;
    memcpy(&bits, &f, 4);
    return bits >> 16;
  };
  for (int j = 0; j < 7; ++j)
    for (int ks = 0; ks < KS; ++ks)
      for (int nt = 0; nt < 3; ++nt)
        for (int lane = 0; lane < 32; ++lane) {
          const int n = 8 * nt + (lane >> 2), k0 = 16 * ks + 2 * (lane & 3);
          uint2 v;
          v.x = digit(k0, n, j) | (digit(k0 + 1, n, j) << 16);
          v.y = digit(k0 + 8, n, j) | (digit(k0 + 9, n, j) << 16);
          frag[(((size_t)j * KS + ks) * 3 + nt) * 32 + lane] = v;
        }
}

}  // namespace ns
