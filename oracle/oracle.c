/* Plain FP64 CPU oracle (test infrastructure; see oracle.h).
 *
 * Follows the paper's statement of the problem step by step:
 *   Eq. 1 (Sec. 2.1)  implicit Newmark-beta increment with the lagged tangent,
 *                     and the updates of q, u, v, a listed below it;
 *   Eq. 2             K_e = sum_j w_j B^T D_j B over the integration points;
 *   Sec. 2.1          multi-spring D from 1D springs with a modified
 *                     Ramberg-Osgood skeleton and the Masing rule, 40 B/spring;
 *   Sec. 2.2          3x3 block-Jacobi preconditioned CG;
 *   Sec. 2.3          relative tolerance 1e-8.
 * Element matrices are formed explicitly and applied element by element; no
 * blocking, fusion or reordering.  Where the paper is silent the readings are
 * the documented ones: 4-point degree-2 rule, consistent mass, Rayleigh
 * C = alpha M + beta K^n calibrated at two frequencies, Lysmer dashpots on the
 * bottom and side faces with the outcrop (2E) input on the bottom, the spring
 * geometry and Masing bookkeeping described at or_spring_dirs/or_spring_update.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Built twice from this one source: plain (single thread) and with -fopenmp.  The
 * OpenMP pragmas only split loops whose iterations are independent (element matrices,
 * element contributions, per-node gathers in a fixed order, per-point spring updates,
 * elementwise vector updates); every sum keeps the order of the single-thread build,
 * so both builds give bit-identical results. */
int or_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

static const int EDGE[6][2] = {{0, 1}, {1, 2}, {0, 2}, {0, 3}, {1, 3}, {2, 3}};
static const double DLDXI[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

/* ------------------------------------------------------------------ shape functions */

/* Quadratic tetrahedron shape functions in barycentric coordinates:
 * vertex N_i = L_i (2 L_i - 1), edge N_ab = 4 L_a L_b. */
void or_shape(const double L[4], double N[10]) {
  for (int i = 0; i < 4; ++i) N[i] = L[i] * (2.0 * L[i] - 1.0);
  for (int k = 0; k < 6; ++k) N[4 + k] = 4.0 * L[EDGE[k][0]] * L[EDGE[k][1]];
}

/* Derivatives with respect to the reference coordinates (xi, eta, zeta), where
 * L0 = 1 - xi - eta - zeta, L1 = xi, L2 = eta, L3 = zeta. */
void or_shape_dref(const double L[4], double dN[10][3]) {
  for (int i = 0; i < 4; ++i)
    for (int c = 0; c < 3; ++c) dN[i][c] = (4.0 * L[i] - 1.0) * DLDXI[i][c];
  for (int k = 0; k < 6; ++k) {
    int a = EDGE[k][0], b = EDGE[k][1];
    for (int c = 0; c < 3; ++c) dN[4 + k][c] = 4.0 * (L[a] * DLDXI[b][c] + L[b] * DLDXI[a][c]);
  }
}

/* Isoparametric map: J[r][c] = sum_i X[i][r] dN_i/dxi_c; physical gradients
 * G = J^{-T} dNref.  Returns det J. */
double or_grad(const double X[10][3], const double L[4], double G[10][3]) {
  double dN[10][3], J[3][3] = {{0}};
  or_shape_dref(L, dN);
  for (int i = 0; i < 10; ++i)
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) J[r][c] += X[i][r] * dN[i][c];
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  double Ji[3][3]; /* inverse of J */
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  /* dN/dxi_c = sum_r dN/dx_r J[r][c]  =>  dN/dx_r = sum_c dN/dxi_c Ji[c][r] */
  for (int i = 0; i < 10; ++i)
    for (int r = 0; r < 3; ++r) {
      double s = 0.0;
      for (int c = 0; c < 3; ++c) s += dN[i][c] * Ji[c][r];
      G[i][r] = s;
    }
  return det;
}

/* Strain-displacement matrix (6 x 30), Voigt xx yy zz yz xz xy, engineering shear. */
void or_bmatrix(const double G[10][3], double B[6][30]) {
  memset(B, 0, sizeof(double) * 6 * 30);
  for (int i = 0; i < 10; ++i) {
    const double *d = G[i];
    B[0][3 * i + 0] = d[0];
    B[1][3 * i + 1] = d[1];
    B[2][3 * i + 2] = d[2];
    B[3][3 * i + 1] = d[2];
    B[3][3 * i + 2] = d[1];
    B[4][3 * i + 0] = d[2];
    B[4][3 * i + 2] = d[0];
    B[5][3 * i + 0] = d[1];
    B[5][3 * i + 1] = d[0];
  }
}

/* Four integration points (Eq. 2 reading: Q = 4): barycentric (a,b,b,b) and
 * permutations, a = (5 + 3 sqrt5)/20, b = (5 - sqrt5)/20, each weighted by a
 * quarter of the element volume (degree-2 exact). */
void or_quad_points(double L[4][4], double *wfrac) {
  const double a = (5.0 + 3.0 * sqrt(5.0)) / 20.0, b = (5.0 - sqrt(5.0)) / 20.0;
  for (int q = 0; q < 4; ++q)
    for (int i = 0; i < 4; ++i) L[q][i] = (i == q) ? a : b;
  *wfrac = 0.25;
}

/* Eq. 2: K_e = sum_q w_q B_q^T D_q B_q, w_q = detJ_q / 6 / 4. */
void or_element_stiffness(const double X[10][3], const double D[4][6][6], double K[30][30]) {
  double L[4][4], wf, G[10][3], B[6][30], DB[6][30];
  or_quad_points(L, &wf);
  memset(K, 0, sizeof(double) * 900);
  for (int q = 0; q < 4; ++q) {
    double det = or_grad(X, L[q], G);
    double w = det / 6.0 * wf;
    or_bmatrix(G, B);
    for (int r = 0; r < 6; ++r)
      for (int j = 0; j < 30; ++j) {
        double s = 0.0;
        for (int k = 0; k < 6; ++k) s += D[q][r][k] * B[k][j];
        DB[r][j] = s;
      }
    for (int i = 0; i < 30; ++i)
      for (int j = 0; j < 30; ++j) {
        double s = 0.0;
        for (int r = 0; r < 6; ++r) s += B[r][i] * DB[r][j];
        K[i][j] += w * s;
      }
  }
}

/* 4-point Gauss-Legendre rule on [0,1]. */
static void gl4(double t[4], double w[4]) {
  double x1 = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0)), x2 = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
  double w1 = (18.0 + sqrt(30.0)) / 36.0, w2 = (18.0 - sqrt(30.0)) / 36.0;
  double x[4] = {-x2, -x1, x1, x2}, ww[4] = {w2, w1, w1, w2};
  for (int i = 0; i < 4; ++i) {
    t[i] = 0.5 * (1.0 + x[i]);
    w[i] = 0.5 * ww[i];
  }
}

/* Consistent mass (scalar part), M_ab = rho * integral N_a N_b dV, by the
 * collapsed (Duffy) map xi = u, eta = (1-u) v, zeta = (1-u)(1-v) w with
 * Gauss-Legendre in u, v, w -- exact for the degree-4 integrand. */
void or_element_mass(const double X[10][3], double rho, double M[10][10]) {
  double t[4], w[4], N[10], G[10][3];
  gl4(t, w);
  memset(M, 0, sizeof(double) * 100);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      for (int k = 0; k < 4; ++k) {
        double u = t[i], v = t[j], ww = t[k];
        double xi = u, eta = (1.0 - u) * v, zeta = (1.0 - u) * (1.0 - v) * ww;
        double jac = (1.0 - u) * (1.0 - u) * (1.0 - v);
        double L[4] = {1.0 - xi - eta - zeta, xi, eta, zeta};
        double det = or_grad(X, L, G);
        or_shape(L, N);
        double wt = w[i] * w[j] * w[k] * jac * det * rho;
        for (int a = 0; a < 10; ++a)
          for (int b = 0; b < 10; ++b) M[a][b] += wt * N[a] * N[b];
      }
}

/* Lysmer viscous boundary on a flat six-node face: traction -rho [Vp n n^T +
 * Vs (I - n n^T)] v, giving C_f = integral N_a N_b dA (x) rho [Vs I + (Vp - Vs) n n^T].
 * Face shape functions: vertex l_i (2 l_i - 1), edge 4 l_a l_b on edges (0,1) (1,2) (0,2);
 * integral by the collapsed map s = u, t = (1-u) v with Gauss-Legendre. */
void or_face_dashpot(const double FX[3][3], double rho, double vs, double vp, double C[18][18]) {
  double e1[3], e2[3], nrm[3];
  for (int c = 0; c < 3; ++c) {
    e1[c] = FX[1][c] - FX[0][c];
    e2[c] = FX[2][c] - FX[0][c];
  }
  nrm[0] = e1[1] * e2[2] - e1[2] * e2[1];
  nrm[1] = e1[2] * e2[0] - e1[0] * e2[2];
  nrm[2] = e1[0] * e2[1] - e1[1] * e2[0];
  double len = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
  double area = 0.5 * len;
  for (int c = 0; c < 3; ++c) nrm[c] /= len;
  static const int FE[3][2] = {{0, 1}, {1, 2}, {0, 2}};
  double t[4], w[4], Mf[6][6] = {{0}};
  gl4(t, w);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = t[i], tt = (1.0 - t[i]) * t[j];
      double l[3] = {1.0 - s - tt, s, tt};
      double N[6];
      for (int a = 0; a < 3; ++a) N[a] = l[a] * (2.0 * l[a] - 1.0);
      for (int k = 0; k < 3; ++k) N[3 + k] = 4.0 * l[FE[k][0]] * l[FE[k][1]];
      double wt = w[i] * w[j] * (1.0 - t[i]) * 2.0 * area; /* reference triangle area 1/2 */
      for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) Mf[a][b] += wt * N[a] * N[b];
    }
  double T[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) T[r][c] = rho * ((r == c ? vs : 0.0) + (vp - vs) * nrm[r] * nrm[c]);
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b)
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) C[3 * a + r][3 * b + c] = Mf[a][b] * T[r][c];
}

/* ------------------------------------------------------------------ spring law */

/* Modified Ramberg-Osgood skeleton, written strain-of-stress:
 *   g(tau) = (tau/G0) (1 + alpha |tau / (G0 gamma_ref)|^beta)
 * with alpha = 2^beta (secant modulus G0/2 at gamma_ref) and
 * beta = 2 pi h_max / (2 - pi h_max) (Masing loop damping tends to h_max). */
void or_ro_params(double rho, double vs, double gamma_ref, double h_max, or_ro *p) {
  p->G0 = rho * vs * vs;
  p->gref = gamma_ref;
  p->beta = 2.0 * M_PI * h_max / (2.0 - M_PI * h_max);
  p->alpha = pow(2.0, p->beta);
}

double or_ro_g(double tau, const or_ro *p) {
  double x = fabs(tau) / (p->G0 * p->gref);
  return tau / p->G0 * (1.0 + p->alpha * pow(x, p->beta));
}

double or_ro_dg(double tau, const or_ro *p) {
  double x = fabs(tau) / (p->G0 * p->gref);
  return (1.0 + p->alpha * (1.0 + p->beta) * pow(x, p->beta)) / p->G0;
}

/* Skeleton stress of a strain: root of g(tau) = gamma.  g is odd, increasing
 * and convex for tau > 0, so Newton started at the upper bound G0 |gamma|
 * decreases monotonically to the root. */
double or_ro_F(double gamma, const or_ro *p) {
  if (gamma == 0.0) return 0.0;
  double ga = fabs(gamma);
  double tau = p->G0 * ga;
  for (int it = 0; it < 1000; ++it) {
    double step = (or_ro_g(tau, p) - ga) / or_ro_dg(tau, p);
    tau -= step;
    if (fabs(step) <= 1e-15 * tau) break;
  }
  return gamma > 0.0 ? tau : -tau;
}

/* Tangent dtau/dgamma of the current state: skeleton 1/g'(tau); Masing branch
 * tau = tR + 2 F((gamma - gR)/2) has tangent 1/g'((tau - tR)/2). */
double or_spring_tangent(const or_spring *s, const or_ro *p) {
  if (s->mode == 0) return 1.0 / or_ro_dg(s->tau, p);
  return 1.0 / or_ro_dg(0.5 * (s->tau - s->tR), p);
}

/* One spring, strain moving to g_new by the increment dg (so from g_new - dg).
 *  - dg == 0: state unchanged;
 *  - virgin (dir 0): start on the skeleton in the direction of dg;
 *  - dg against dir: reversal -- remember (g_old, tau_old), follow the branch;
 *  - skeleton: tau = F(g_new), gmax = max(gmax, |g_new|);
 *  - branch: tau = tR + 2 F((g_new - gR)/2); once |g_new| >= gmax while moving
 *    outward, back to the skeleton with tau = F(g_new).
 * Returns the tangent at the end state. */
double or_spring_update(or_spring *s, double g_new, double dg, const or_ro *p) {
  if (dg != 0.0) {
    double g_old = g_new - dg;
    int sgn = dg > 0.0 ? 1 : -1;
    if (s->dir == 0) {
      s->dir = sgn;
      s->mode = 0;
    } else if (sgn != s->dir) {
      s->gR = g_old;
      s->tR = s->tau;
      s->mode = 1;
      s->dir = sgn;
    }
    if (s->mode == 0) {
      s->tau = or_ro_F(g_new, p);
      if (fabs(g_new) > s->gmax) s->gmax = fabs(g_new);
    } else {
      s->tau = s->tR + 2.0 * or_ro_F(0.5 * (g_new - s->gR), p);
      if (fabs(g_new) >= s->gmax && g_new * (double)s->dir > 0.0) {
        s->mode = 0;
        s->tau = or_ro_F(g_new, p);
        s->gmax = fabs(g_new);
      }
    }
  }
  return or_spring_tangent(s, p);
}

/* ------------------------------------------------------------------ multi-spring geometry */

/* Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (n <= 6):
 * A = V diag(lam) V^T. */
static void jacobi_eig(int n, const double *A_in, double *lam, double *V) {
  double A[36];
  memcpy(A, A_in, sizeof(double) * n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += A[i * n + j] * A[i * n + j];
        if (i != j) off += A[i * n + j] * A[i * n + j];
      }
    if (off <= 1e-32 * tot) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (apq == 0.0) continue;
        double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        /* A <- R^T A R with R the rotation in the (p,q) plane */
        for (int k = 0; k < n; ++k) {
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) lam[i] = A[i * n + i];
}

/* Spring directions q_k (Voigt 6-vectors) and weight w (reading of the
 * multi-spring geometry, Sec. 2.1):
 *   plane normal n_k: hemispherical Fibonacci point, z = 1 - (k + 1/2)/S,
 *     azimuth phi = k pi (3 - sqrt 5);
 *   slip s_k = cos psi t1 + sin psi t2, t1 = (-sin phi, cos phi, 0),
 *     t2 = n x t1, psi = 2 pi frac(k sqrt 2);
 *   p_k = shear-strain projection: gamma = 2 n.eps.s = p_k . eps_voigt;
 *   q_k = T p_k with T = c Ddev^(1/2) P^(+1/2), P = sum p p^T, c = sqrt(2S/5),
 *     Ddev = diag(2,2,2,1,1,1) - (2/3) m m^T,  so  w sum_k q_k q_k^T = Ddev
 *     with w = 5/(2S).  P^(+1/2) is taken as (P + m m^T/3)^(-1/2) - m m^T/3.
 * Returns 0, or -1 if S < 5. */
int or_spring_dirs(int S, double *q, double *w) {
  if (S < 5) return -1;
  double *p = (double *)malloc(sizeof(double) * 6 * S);
  double P[36] = {0};
  const double ga = M_PI * (3.0 - sqrt(5.0));
  for (int k = 0; k < S; ++k) {
    double z = 1.0 - (k + 0.5) / S;
    double r = sqrt(1.0 - z * z);
    double phi = k * ga;
    double n[3] = {r * cos(phi), r * sin(phi), z};
    double t1[3] = {-sin(phi), cos(phi), 0.0};
    double t2[3] = {n[1] * t1[2] - n[2] * t1[1], n[2] * t1[0] - n[0] * t1[2], n[0] * t1[1] - n[1] * t1[0]};
    double fr = k * sqrt(2.0);
    fr -= floor(fr);
    double psi = 2.0 * M_PI * fr;
    double s[3];
    for (int c = 0; c < 3; ++c) s[c] = cos(psi) * t1[c] + sin(psi) * t2[c];
    double *pk = p + 6 * k;
    pk[0] = 2.0 * n[0] * s[0];
    pk[1] = 2.0 * n[1] * s[1];
    pk[2] = 2.0 * n[2] * s[2];
    pk[3] = n[1] * s[2] + n[2] * s[1];
    pk[4] = n[0] * s[2] + n[2] * s[0];
    pk[5] = n[0] * s[1] + n[1] * s[0];
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) P[i * 6 + j] += pk[i] * pk[j];
  }
  double Pm[36], Pim[36], lam[6], V[36];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) Pm[i * 6 + j] = P[i * 6 + j] + ((i < 3 && j < 3) ? 1.0 / 3.0 : 0.0);
  jacobi_eig(6, Pm, lam, V);
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double s = 0.0;
      for (int k = 0; k < 6; ++k) s += V[i * 6 + k] / sqrt(lam[k]) * V[j * 6 + k];
      Pim[i * 6 + j] = s - ((i < 3 && j < 3) ? 1.0 / 3.0 : 0.0);
    }
  /* Ddev^(1/2): sqrt2 (I - 11^T/3) on the normal block, identity on the shear block */
  double Dh[36] = {0};
  double c = sqrt(2.0 * S / 5.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Dh[i * 6 + j] = c * sqrt(2.0) * ((i == j ? 1.0 : 0.0) - 1.0 / 3.0);
  for (int i = 3; i < 6; ++i) Dh[i * 6 + i] = c;
  double T[36];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double s = 0.0;
      for (int k = 0; k < 6; ++k) s += Dh[i * 6 + k] * Pim[k * 6 + j];
      T[i * 6 + j] = s;
    }
  for (int k = 0; k < S; ++k)
    for (int i = 0; i < 6; ++i) {
      double s = 0.0;
      for (int j = 0; j < 6; ++j) s += T[i * 6 + j] * p[6 * k + j];
      q[6 * k + i] = s;
    }
  *w = 5.0 / (2.0 * S);
  free(p);
  return 0;
}

/* D = Kb m m^T + w sum_k G_k q_k q_k^T with every G_k = G0 (virgin state). */
void or_elastic_D(int S, const double *q, double w, double Kb, double G0, double D[6][6]) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) D[i][j] = (i < 3 && j < 3) ? Kb : 0.0;
  for (int k = 0; k < S; ++k)
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) D[i][j] += w * G0 * q[6 * k + i] * q[6 * k + j];
}

/* One integration point: spring strains gamma_k = q_k.eps, increments
 * q_k.deps, spring updates, then D = Kb m m^T + w sum_k G_k q_k q_k^T. */
void or_point_update(int S, const double *q, double w, double Kb, const or_ro *p, const double eps[6],
                     const double deps[6], or_spring *sp, double D[6][6]) {
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) D[i][j] = (i < 3 && j < 3) ? Kb : 0.0;
  for (int k = 0; k < S; ++k) {
    double g = 0.0, dg = 0.0;
    for (int i = 0; i < 6; ++i) {
      g += q[6 * k + i] * eps[i];
      dg += q[6 * k + i] * deps[i];
    }
    double G = or_spring_update(&sp[k], g, dg, p);
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) D[i][j] += w * G * q[6 * k + i] * q[6 * k + j];
  }
}

/* ------------------------------------------------------------------ model level */

typedef struct {
  double rho, vs, vp, Kb, ray_a, ray_b;
  or_ro ro;
} matc;

static void material_constants(const or_model *m, matc *mc) {
  double w1 = 2.0 * M_PI * m->f1, w2 = 2.0 * M_PI * m->f2;
  for (int i = 0; i < m->n_mat; ++i) {
    const double *r = m->matprops + 6 * i;
    mc[i].rho = r[0];
    mc[i].vs = r[1];
    mc[i].vp = r[2];
    mc[i].Kb = r[0] * (r[2] * r[2] - 4.0 / 3.0 * r[1] * r[1]);
    /* Rayleigh C = a M + b K with damping ratio h at w1 and w2 */
    mc[i].ray_a = 2.0 * r[5] * w1 * w2 / (w1 + w2);
    mc[i].ray_b = 2.0 * r[5] / (w1 + w2);
    or_ro_params(r[0], r[1], r[3], r[4], &mc[i].ro);
  }
}

int or_state_init(const or_model *m, or_state *s) {
  int S = m->n_springs;
  double *q = (double *)malloc(sizeof(double) * 6 * (S > 5 ? S : 5)), w;
  if (or_spring_dirs(S, q, &w) != 0) {
    free(q);
    return -1;
  }
  matc *mc = (matc *)malloc(sizeof(matc) * m->n_mat);
  material_constants(m, mc);
  size_t nv = (size_t)m->n_nodes * 3;
  memset(s->u, 0, sizeof(double) * nv);
  memset(s->v, 0, sizeof(double) * nv);
  memset(s->a, 0, sizeof(double) * nv);
  memset(s->q, 0, sizeof(double) * nv);
  memset(s->du, 0, sizeof(double) * nv);
  for (int64_t e = 0; e < m->n_elems; ++e) {
    const matc *c = &mc[m->mat[e]];
    for (int qp = 0; qp < 4; ++qp) or_elastic_D(S, q, w, c->Kb, c->ro.G0, (double(*)[6])(s->D + (e * 4 + qp) * 36));
  }
  memset(s->th, 0, sizeof(or_spring) * (size_t)m->n_elems * 4 * S);
  s->step = 0;
  s->iters = 0;
  s->relres = 0.0;
  free(q);
  free(mc);
  return 0;
}

/* Outcrop input velocity at t_n = n dt: trapezoidal integral of the given
 * acceleration from v(0) = 0; samples beyond the record count as zero. */
double or_input_velocity(const or_model *m, int64_t n, int comp) {
  double v = 0.0;
  for (int64_t k = 1; k <= n; ++k) {
    double a0 = (k - 1 < m->n_samples) ? m->acc[(k - 1) * 3 + comp] : 0.0;
    double a1 = (k < m->n_samples) ? m->acc[k * 3 + comp] : 0.0;
    v += 0.5 * m->dt * (a0 + a1);
  }
  return v;
}

void or_strain(const or_model *m, int64_t e, int qp, const double *u, double eps[6]) {
  double L[4][4], wf, G[10][3], B[6][30], ue[30];
  or_quad_points(L, &wf);
  or_grad((const double(*)[3])(m->X + e * 30), L[qp], G);
  or_bmatrix(G, B);
  for (int a = 0; a < 10; ++a)
    for (int c = 0; c < 3; ++c) ue[3 * a + c] = u[(size_t)m->conn[e * 10 + a] * 3 + c];
  for (int r = 0; r < 6; ++r) {
    double s = 0.0;
    for (int j = 0; j < 30; ++j) s += B[r][j] * ue[j];
    eps[r] = s;
  }
}

typedef struct {
  double *K;  /* [E][30][30] stiffness with the current D */
  double *M;  /* [E][10][10] scalar mass */
  double *Cf; /* [F][18][18] dashpots */
  matc *mc;
  /* node -> (element, local node) incidence, elements ascending: entries
   * inc[inc_off[n] .. inc_off[n+1]) hold 10 e + a for conn[e][a] == n */
  int64_t *inc_off, *inc;
} opset;

static void ops_build(const or_model *m, const double *D, opset *o) {
  o->mc = (matc *)malloc(sizeof(matc) * m->n_mat);
  material_constants(m, o->mc);
  o->K = (double *)malloc(sizeof(double) * 900 * (size_t)m->n_elems);
  o->M = (double *)malloc(sizeof(double) * 100 * (size_t)m->n_elems);
  o->Cf = (double *)malloc(sizeof(double) * 324 * (size_t)(m->n_faces > 0 ? m->n_faces : 1));
  o->inc_off = (int64_t *)calloc((size_t)m->n_nodes + 1, sizeof(int64_t));
  o->inc = (int64_t *)malloc(sizeof(int64_t) * 10 * (size_t)(m->n_elems > 0 ? m->n_elems : 1));
  for (int64_t i = 0; i < 10 * m->n_elems; ++i) o->inc_off[m->conn[i] + 1]++;
  for (int64_t n = 0; n < m->n_nodes; ++n) o->inc_off[n + 1] += o->inc_off[n];
  {
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m->n_nodes > 0 ? m->n_nodes : 1));
    memcpy(fill, o->inc_off, sizeof(int64_t) * (size_t)m->n_nodes);
    for (int64_t i = 0; i < 10 * m->n_elems; ++i) o->inc[fill[m->conn[i]]++] = i; /* ascending e */
    free(fill);
  }
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m->n_elems; ++e) {
    const double(*X)[3] = (const double(*)[3])(m->X + e * 30);
    or_element_stiffness(X, (const double(*)[6][6])(D + e * 144), (double(*)[30])(o->K + e * 900));
    or_element_mass(X, o->mc[m->mat[e]].rho, (double(*)[10])(o->M + e * 100));
  }
  for (int64_t f = 0; f < m->n_faces; ++f) {
    const matc *c = &o->mc[m->fmat[f]];
    or_face_dashpot((const double(*)[3])(m->FX + f * 9), c->rho, c->vs, c->vp, (double(*)[18])(o->Cf + f * 324));
  }
}

static void ops_free(opset *o) {
  free(o->K);
  free(o->M);
  free(o->Cf);
  free(o->mc);
  free(o->inc_off);
  free(o->inc);
}

static void face_apply(const or_model *m, const opset *o, int64_t f, double cC, const double *x, const double *xconst,
                       double *y) {
  const int32_t *fn = m->faces + f * 6;
  double xe[18];
  for (int a = 0; a < 6; ++a)
    for (int c = 0; c < 3; ++c) xe[3 * a + c] = xconst ? xconst[c] : x[(size_t)fn[a] * 3 + c];
  const double *C = o->Cf + f * 324;
  for (int i = 0; i < 18; ++i) {
    double s = 0.0;
    for (int j = 0; j < 18; ++j) s += C[i * 18 + j] * xe[j];
    y[(size_t)fn[i / 3] * 3 + i % 3] += cC * s;
  }
}

/* One element-level term y += cM M_e x + cK K_e x; with `rayleigh` set the coefficients
 * are scale * (a, b) of the element's material instead (the Rayleigh part of C^n). */
typedef struct {
  const double *x;
  double cM, cK, scale;
  int rayleigh;
} eterm;

/* y += the terms, element by element in ascending order and term by term within an
 * element -- the additions of a loop over elements applying each term in turn.  The
 * element contributions are formed first (independently per element), then every node
 * adds those of its elements in ascending element order, term by term, so each entry of
 * y receives the same additions in the same order as in that loop. */
static void elems_apply(const or_model *m, const opset *o, int nt, const eterm *t, double *y) {
  const int64_t E = m->n_elems;
  double *Y = (double *)malloc(sizeof(double) * 30 * (size_t)nt * (size_t)(E > 0 ? E : 1));
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < E; ++e) {
    const matc *c = &o->mc[m->mat[e]];
    for (int k = 0; k < nt; ++k) {
      double *ye = Y + ((size_t)e * nt + k) * 30;
      const double cM = t[k].rayleigh ? t[k].scale * c->ray_a : t[k].cM;
      const double cK = t[k].rayleigh ? t[k].scale * c->ray_b : t[k].cK;
      memset(ye, 0, sizeof(double) * 30);
      /* y_e = cK K_e x_e + cM M_e x_e (scalar mass per displacement component) */
      const int32_t *cn = m->conn + e * 10;
      double xe[30];
      for (int a = 0; a < 10; ++a)
        for (int cc = 0; cc < 3; ++cc) xe[3 * a + cc] = t[k].x[(size_t)cn[a] * 3 + cc];
      const double *K = o->K + e * 900, *M = o->M + e * 100;
      for (int i = 0; i < 30; ++i) {
        double s = 0.0;
        for (int j = 0; j < 30; ++j) s += K[i * 30 + j] * xe[j];
        ye[i] = cK * s;
      }
      for (int a = 0; a < 10; ++a)
        for (int cc = 0; cc < 3; ++cc) {
          double s = 0.0;
          for (int b = 0; b < 10; ++b) s += M[a * 10 + b] * xe[3 * b + cc];
          ye[3 * a + cc] += cM * s;
        }
    }
  }
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < m->n_nodes; ++n)
    for (int64_t j = o->inc_off[n]; j < o->inc_off[n + 1]; ++j) {
      const int64_t e = o->inc[j] / 10, a = o->inc[j] % 10;
      for (int k = 0; k < nt; ++k)
        for (int cc = 0; cc < 3; ++cc) y[(size_t)n * 3 + cc] += Y[((size_t)e * nt + k) * 30 + 3 * a + cc];
    }
  free(Y);
}

/* y = A x with A = 4/dt^2 M + 2/dt C^n + K^n (Eq. 1), C^n = a M + b K^n + C_b. */
static void apply_A(const or_model *m, const opset *o, const double *x, double *y) {
  double dt = m->dt;
  memset(y, 0, sizeof(double) * 3 * (size_t)m->n_nodes);
  const eterm t[3] = {{x, 4.0 / (dt * dt), 0.0, 0.0, 0}, /* 4/dt^2 M */
                      {x, 0.0, 0.0, 2.0 / dt, 1},         /* 2/dt (a M + b K) */
                      {x, 0.0, 1.0, 0.0, 0}};             /* K */
  elems_apply(m, o, 3, t, y);
  for (int64_t f = 0; f < m->n_faces; ++f) face_apply(m, o, f, 2.0 / dt, x, NULL, y); /* 2/dt C_b */
}

/* which: 0 K, 1 M, 2 C_b (faces), 3 A, 4 Rayleigh C (a M + b K, no faces) */
int or_operator(const or_model *m, const double *D, int which, const double *x, double *y) {
  opset o;
  ops_build(m, D, &o);
  memset(y, 0, sizeof(double) * 3 * (size_t)m->n_nodes);
  if (which == 3) {
    apply_A(m, &o, x, y);
  } else {
    eterm t = {x, 0.0, 0.0, 0.0, 0};
    if (which == 0) t.cK = 1.0;
    if (which == 1) t.cM = 1.0;
    if (which == 4) {
      t.rayleigh = 1;
      t.scale = 1.0;
    }
    if (which != 2) elems_apply(m, &o, 1, &t, y);
    if (which == 2)
      for (int64_t f = 0; f < m->n_faces; ++f) face_apply(m, &o, f, 1.0, x, NULL, y);
  }
  ops_free(&o);
  return 0;
}

static double dotv(size_t n, const double *a, const double *b) {
  double s = 0.0;
  for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* 3x3 inverse by cofactors; returns 0 on a singular block. */
static int inv3(const double A[3][3], double R[3][3]) {
  double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
               A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  if (det == 0.0) return 0;
  R[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
  R[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
  R[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
  R[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / det;
  R[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
  R[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
  R[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
  R[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
  R[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
  return 1;
}

/* One time step n -> n+1.  Returns 0, -2 if CG did not converge, -3 on a
 * singular preconditioner block, -1 on bad input. */
int or_step(const or_model *m, or_state *s) {
  const int S = m->n_springs;
  const double dt = m->dt;
  const size_t N3 = (size_t)m->n_nodes * 3;
  const int64_t n = s->step + 1; /* this step computes the state at t_n = n dt */
  opset o;
  ops_build(m, s->D, &o); /* K^n from the tangent left by step n-1 (lagged, Alg. 4) */

  double *b = (double *)calloc(N3, sizeof(double));
  double *t1 = (double *)calloc(N3, sizeof(double));
  double *x = (double *)malloc(sizeof(double) * N3);
  double *r = (double *)malloc(sizeof(double) * N3);
  double *z = (double *)malloc(sizeof(double) * N3);
  double *p = (double *)malloc(sizeof(double) * N3);
  double *Ap = (double *)malloc(sizeof(double) * N3);
  double *Jinv = (double *)calloc((size_t)m->n_nodes * 9, sizeof(double));
  int status = 0;

  /* right-hand side of Eq. 1: f^n - q^{n-1} + C^n v^{n-1} + M (a^{n-1} + 4/dt v^{n-1}) */
  for (size_t i = 0; i < N3; ++i) t1[i] = s->a[i] + 4.0 / dt * s->v[i];
  {
    const eterm t[2] = {{s->v, 0.0, 0.0, 1.0, 1}, /* Rayleigh part of C^n v */
                        {t1, 1.0, 0.0, 0.0, 0}};  /* M (a + 4/dt v) */
    elems_apply(m, &o, 2, t, b);
  }
  double vin[3];
  for (int c = 0; c < 3; ++c) vin[c] = or_input_velocity(m, n, c);
  for (int64_t f = 0; f < m->n_faces; ++f) {
    face_apply(m, &o, f, 1.0, s->v, NULL, b); /* boundary part of C^n v */
    if (m->fkind[f] == 0) face_apply(m, &o, f, 1.0, NULL, vin, b); /* f^n = C_b,bottom v_in(t_n) */
  }
  for (size_t i = 0; i < N3; ++i) b[i] -= s->q[i];

  /* 3x3 block-Jacobi preconditioner: diagonal node blocks of A */
  {
    double *Jd = (double *)calloc((size_t)m->n_nodes * 9, sizeof(double));
    /* each node adds its elements' diagonal blocks in ascending element order */
#pragma omp parallel for schedule(static)
    for (int64_t nd = 0; nd < m->n_nodes; ++nd)
      for (int64_t jj = o.inc_off[nd]; jj < o.inc_off[nd + 1]; ++jj) {
        const int64_t e = o.inc[jj] / 10, a = o.inc[jj] % 10;
        const matc *c = &o.mc[m->mat[e]];
        double cM = 4.0 / (dt * dt) + 2.0 / dt * c->ray_a, cK = 1.0 + 2.0 / dt * c->ray_b;
        const double *K = o.K + e * 900, *M = o.M + e * 100;
        double *J = Jd + (size_t)nd * 9;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            J[i * 3 + j] += cK * K[(3 * a + i) * 30 + 3 * a + j] + (i == j ? cM * M[a * 10 + a] : 0.0);
      }
    for (int64_t f = 0; f < m->n_faces; ++f) {
      const double *C = o.Cf + f * 324;
      for (int a = 0; a < 6; ++a) {
        double *J = Jd + (size_t)m->faces[f * 6 + a] * 9;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) J[i * 3 + j] += 2.0 / dt * C[(3 * a + i) * 18 + 3 * a + j];
      }
    }
    for (int64_t i = 0; i < m->n_nodes; ++i)
      if (!inv3((const double(*)[3])(Jd + i * 9), (double(*)[3])(Jinv + i * 9))) status = -3;
    free(Jd);
  }

  /* preconditioned CG on A du = b, stop at ||r|| <= tol ||b|| (recursive residual) */
  int iters = 0;
  double bn = sqrt(dotv(N3, b, b)), rn = 0.0;
  if (status == 0) {
    if (bn == 0.0) {
      memset(x, 0, sizeof(double) * N3);
    } else {
      if (m->x0_prev)
        memcpy(x, s->du, sizeof(double) * N3);
      else
        memset(x, 0, sizeof(double) * N3);
      apply_A(m, &o, x, Ap);
      for (size_t i = 0; i < N3; ++i) r[i] = b[i] - Ap[i];
      rn = sqrt(dotv(N3, r, r));
      if (rn > m->tol * bn) {
        double rz = 0.0;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < m->n_nodes; ++i)
          for (int k = 0; k < 3; ++k) {
            double sum = 0.0;
            for (int j = 0; j < 3; ++j) sum += Jinv[i * 9 + k * 3 + j] * r[i * 3 + j];
            z[i * 3 + k] = sum;
          }
        memcpy(p, z, sizeof(double) * N3);
        rz = dotv(N3, r, z);
        int conv = 0;
        for (int it = 1; it <= m->max_iter; ++it) {
          apply_A(m, &o, p, Ap);
          double alpha = rz / dotv(N3, p, Ap);
#pragma omp parallel for schedule(static)
          for (size_t i = 0; i < N3; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * Ap[i];
          }
          rn = sqrt(dotv(N3, r, r));
          iters = it;
          if (rn <= m->tol * bn) {
            conv = 1;
            break;
          }
#pragma omp parallel for schedule(static)
          for (int64_t i = 0; i < m->n_nodes; ++i)
            for (int k = 0; k < 3; ++k) {
              double sum = 0.0;
              for (int j = 0; j < 3; ++j) sum += Jinv[i * 9 + k * 3 + j] * r[i * 3 + j];
              z[i * 3 + k] = sum;
            }
          double rz_new = dotv(N3, r, z);
          double beta = rz_new / rz;
          rz = rz_new;
#pragma omp parallel for schedule(static)
          for (size_t i = 0; i < N3; ++i) p[i] = z[i] + beta * p[i];
        }
        if (!conv) status = -2;
      }
    }
  }
  s->iters = iters;
  s->relres = bn > 0.0 ? rn / bn : 0.0;

  if (status == 0) {
    /* q^n = q^{n-1} + K^n du; u, v, a updates below Eq. 1 */
    {
      const eterm t = {x, 0.0, 1.0, 0.0, 0};
      elems_apply(m, &o, 1, &t, s->q);
    }
    for (size_t i = 0; i < N3; ++i) {
      double v_old = s->v[i];
      s->u[i] += x[i];
      s->v[i] = -v_old + 2.0 / dt * x[i];
      s->a[i] = -s->a[i] - 4.0 / dt * v_old + 4.0 / (dt * dt) * x[i];
      s->du[i] = x[i];
    }
    /* multi-spring update at every integration point: D^n and theta^n (Eq. 2) */
    double *qd = (double *)malloc(sizeof(double) * 6 * S), w;
    or_spring_dirs(S, qd, &w);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t e = 0; e < m->n_elems; ++e) {
      const matc *c = &o.mc[m->mat[e]];
      for (int qp = 0; qp < 4; ++qp) {
        double eps[6], deps[6];
        or_strain(m, e, qp, s->u, eps);
        or_strain(m, e, qp, x, deps);
        or_point_update(S, qd, w, c->Kb, &c->ro, eps, deps, s->th + ((size_t)e * 4 + qp) * S,
                        (double(*)[6])(s->D + (e * 4 + qp) * 36));
      }
    }
    free(qd);
    s->step = n;
  }
  ops_free(&o);
  free(b);
  free(t1);
  free(x);
  free(r);
  free(z);
  free(p);
  free(Ap);
  free(Jinv);
  return status;
}

/* Greedy first-fit element colouring in element order: each element takes the
 * smallest colour not used by an earlier element sharing a node with it.
 * Returns the number of colours, or -1 if more than 64 would be needed. */
int or_colouring(int64_t n_elems, int64_t n_nodes, const int32_t *conn, int32_t *colour) {
  uint64_t *used = (uint64_t *)calloc((size_t)n_nodes, sizeof(uint64_t));
  int nc = 0;
  for (int64_t e = 0; e < n_elems; ++e) {
    uint64_t taken = 0;
    for (int a = 0; a < 10; ++a) taken |= used[conn[e * 10 + a]];
    int c = 0;
    while (c < 64 && (taken >> c) & 1ull) ++c;
    if (c == 64) {
      free(used);
      return -1;
    }
    colour[e] = c;
    if (c + 1 > nc) nc = c + 1;
    for (int a = 0; a < 10; ++a) used[conn[e * 10 + a]] |= 1ull << c;
  }
  free(used);
  return nc;
}

/* ------------------------------------------------------------------ two-level preconditioner pieces
 * Sec. 2.2 names EBE-IPCG with a multigrid preconditioner after [SC14], whose details
 * are not in the paper.  Reading: the coarse level is the linear (4-node) tetrahedral
 * model on the same elements, reached from the quadratic model by linear interpolation
 * P (a vertex keeps its value, an edge node takes the mean of its edge's end vertices)
 * and its transpose; the coarse operator is the linear-element discretisation of the
 * same equation, which for straight elements equals P^T A P. */

int64_t or_coarse_map(int64_t n_elems, int64_t n_nodes, const int32_t *conn, int32_t *cid, int32_t *par) {
  /* role of each node: 0 unseen, 1 vertex, 2 edge node */
  int8_t *role = (int8_t *)calloc((size_t)(n_nodes > 0 ? n_nodes : 1), 1);
  int64_t status = 0;
  for (int64_t e = 0; e < n_elems && status == 0; ++e)
    for (int a = 0; a < 10; ++a) {
      const int32_t n = conn[e * 10 + a];
      const int8_t r = a < 4 ? 1 : 2;
      if (role[n] != 0 && role[n] != r) status = -1;
      role[n] = r;
    }
  int64_t nc = 0;
  for (int64_t n = 0; n < n_nodes; ++n) {
    cid[n] = role[n] == 1 ? (int32_t)nc++ : -1;
    par[2 * n] = par[2 * n + 1] = cid[n];
  }
  for (int64_t e = 0; e < n_elems && status == 0; ++e)
    for (int k = 0; k < 6; ++k) {
      const int32_t n = conn[e * 10 + 4 + k];
      int32_t c0 = cid[conn[e * 10 + EDGE[k][0]]], c1 = cid[conn[e * 10 + EDGE[k][1]]];
      if (c0 > c1) {
        const int32_t t = c0;
        c0 = c1;
        c1 = t;
      }
      if (par[2 * n] == -1) {
        par[2 * n] = c0;
        par[2 * n + 1] = c1;
      } else if (par[2 * n] != c0 || par[2 * n + 1] != c1) {
        status = -1;
      }
    }
  free(role);
  return status == 0 ? nc : -1;
}

/* grad L1..L3 are the rows of J^{-1}, J = [x1 - x0, x2 - x0, x3 - x0] (columns);
 * grad L0 = -(grad L1 + grad L2 + grad L3); V = det J / 6. */
void or_p1_grads(const double X[4][3], double g[4][3], double *vol) {
  double J[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) J[r][c] = X[c + 1][r] - X[0][r];
  double Ji[3][3];
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) g[k + 1][c] = Ji[k][c];
  for (int c = 0; c < 3; ++c) g[0][c] = -(g[1][c] + g[2][c] + g[3][c]);
  *vol = det / 6.0;
}

/* Coarse element: K1 = V B^T Dbar B (B the 6 x 12 strain matrix of the linear element,
 * Voigt xx yy zz yz xz xy with engineering shear) and M1 = rho V (1 + delta_ab) / 20. */
static void coarse_element(const double X[4][3], const double Dbar[6][6], double rho, double K[12][12],
                           double M[4][4]) {
  double g[4][3], V;
  or_p1_grads(X, g, &V);
  double B[6][12];
  memset(B, 0, sizeof(B));
  for (int a = 0; a < 4; ++a) {
    const double gx = g[a][0], gy = g[a][1], gz = g[a][2];
    B[0][3 * a] = gx;
    B[1][3 * a + 1] = gy;
    B[2][3 * a + 2] = gz;
    B[3][3 * a + 1] = gz;
    B[3][3 * a + 2] = gy;
    B[4][3 * a] = gz;
    B[4][3 * a + 2] = gx;
    B[5][3 * a] = gy;
    B[5][3 * a + 1] = gx;
  }
  for (int i = 0; i < 12; ++i)
    for (int j = 0; j < 12; ++j) {
      double s = 0.0;
      for (int p = 0; p < 6; ++p)
        for (int q = 0; q < 6; ++q) s += B[p][i] * Dbar[p][q] * B[q][j];
      K[i][j] = V * s;
    }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) M[a][b] = rho * V * (a == b ? 2.0 : 1.0) / 20.0;
}

/* Coarse dashpot face: (A (1 + delta_ab) / 12) rho [Vs I + (Vp - Vs) n n^T]. */
static void coarse_face(const double FX[3][3], double rho, double vs, double vp, double C[9][9]) {
  double a[3], b[3], n[3];
  for (int c = 0; c < 3; ++c) {
    a[c] = FX[1][c] - FX[0][c];
    b[c] = FX[2][c] - FX[0][c];
  }
  n[0] = a[1] * b[2] - a[2] * b[1];
  n[1] = a[2] * b[0] - a[0] * b[2];
  n[2] = a[0] * b[1] - a[1] * b[0];
  const double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  const double area = 0.5 * len;
  for (int c = 0; c < 3; ++c) n[c] /= len;
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) {
      const double w = area * (p == q ? 2.0 : 1.0) / 12.0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          C[3 * p + i][3 * q + j] = w * rho * ((i == j ? vs : 0.0) + (vp - vs) * n[i] * n[j]);
    }
}

int or_coarse_operator(const or_model *m, const double *D, int which, int64_t n_coarse, const int32_t *cid,
                       const double *xc, double *yc) {
  if (which < 0 || which > 3) return -1;
  matc *mc = (matc *)malloc(sizeof(matc) * m->n_mat);
  material_constants(m, mc);
  const double dt = m->dt;
  memset(yc, 0, sizeof(double) * 3 * (size_t)n_coarse);
  for (int64_t e = 0; e < m->n_elems; ++e) {
    const matc *c = &mc[m->mat[e]];
    double X[4][3], Dbar[6][6], K[12][12], M[4][4];
    for (int a = 0; a < 4; ++a)
      for (int k = 0; k < 3; ++k) X[a][k] = m->X[e * 30 + 3 * a + k];
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) {
        double s = 0.0;
        for (int q = 0; q < 4; ++q) s += D[((size_t)e * 4 + q) * 36 + 6 * i + j];
        Dbar[i][j] = 0.25 * s;
      }
    coarse_element(X, Dbar, c->rho, K, M);
    double cM = 0.0, cK = 0.0;
    if (which == 0) cK = 1.0;
    if (which == 1) cM = 1.0;
    if (which == 3) {
      cM = 4.0 / (dt * dt) + 2.0 / dt * c->ray_a;
      cK = 1.0 + 2.0 / dt * c->ray_b;
    }
    if (which == 2) continue;
    int32_t cn[4];
    for (int a = 0; a < 4; ++a) cn[a] = cid[m->conn[e * 10 + a]];
    for (int a = 0; a < 4; ++a)
      for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int b = 0; b < 4; ++b)
          for (int j = 0; j < 3; ++j)
            s += (cK * K[3 * a + i][3 * b + j] + (i == j ? cM * M[a][b] : 0.0)) * xc[(size_t)cn[b] * 3 + j];
        yc[(size_t)cn[a] * 3 + i] += s;
      }
  }
  if (which == 2 || which == 3) {
    const double cC = which == 2 ? 1.0 : 2.0 / dt;
    for (int64_t f = 0; f < m->n_faces; ++f) {
      const matc *c = &mc[m->fmat[f]];
      double C[9][9];
      coarse_face((const double(*)[3])(m->FX + f * 9), c->rho, c->vs, c->vp, C);
      int32_t cn[3];
      for (int p = 0; p < 3; ++p) cn[p] = cid[m->faces[f * 6 + p]];
      for (int p = 0; p < 3; ++p)
        for (int i = 0; i < 3; ++i) {
          double s = 0.0;
          for (int q = 0; q < 3; ++q)
            for (int j = 0; j < 3; ++j) s += C[3 * p + i][3 * q + j] * xc[(size_t)cn[q] * 3 + j];
          yc[(size_t)cn[p] * 3 + i] += cC * s;
        }
    }
  }
  free(mc);
  return 0;
}
