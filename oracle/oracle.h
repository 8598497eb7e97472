/* Plain FP64 CPU oracle of one implicit Newmark-beta step of the nonlinear
 * ground-response method (Sec. 2.1, Eqs. 1-2).  TEST INFRASTRUCTURE ONLY:
 * the tests, the smoke check and the benchmark's CPU-baseline leg may call it;
 * the library never does.  It shares no code with the CUDA path.
 *
 * Units: SI.  Vectors are node-major [n][3].  Element node order: vertices
 * 0-3, then edges (0,1) (1,2) (0,2) (0,3) (1,3) (2,3).  Voigt order of strain
 * and stress: xx yy zz yz xz xy, shear strains in engineering form.
 */
#ifndef NS_ORACLE_H
#define NS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Per-spring state, 40 bytes (Sec. 2.1: four doubles and two flags). */
typedef struct {
  double tau;   /* current spring stress */
  double gR;    /* strain at the last reversal */
  double tR;    /* stress at the last reversal */
  double gmax;  /* largest |strain| reached on the skeleton */
  int32_t dir;  /* loading direction: 0 virgin, +1, -1 */
  int32_t mode; /* 0 skeleton, 1 Masing branch */
} or_spring;

typedef struct {
  int64_t n_nodes, n_elems, n_faces;
  const int32_t *conn;    /* [E][10] */
  const double *X;        /* [E][10][3] element node coordinates */
  const int32_t *mat;     /* [E] */
  int32_t n_mat;
  const double *matprops; /* [n_mat][6]: rho, vs, vp, gamma_ref, h_max, rayleigh_h */
  const int32_t *faces;   /* [F][6] */
  const double *FX;       /* [F][3][3] face vertex coordinates */
  const int32_t *fmat;    /* [F] material of the face's element */
  const int32_t *fkind;   /* [F] 0 bottom (input applied), 1 side */
  int32_t n_springs;
  double dt, tol;
  int32_t max_iter;
  double f1, f2;          /* Rayleigh calibration frequencies (Hz) */
  int64_t n_samples;
  const double *acc;      /* [n_samples][3] outcrop acceleration at t = k dt */
  int32_t x0_prev;        /* 1: CG starts from the previous increment, 0: from zero */
} or_model;

typedef struct {
  double *u, *v, *a, *q, *du; /* [N][3] */
  double *D;                  /* [E][4][6][6] tangent at the integration points */
  or_spring *th;              /* [E][4][S] */
  int64_t step;               /* steps taken */
  int32_t iters;              /* CG iterations of the last step */
  double relres;              /* final recursive relative residual of the last step */
} or_state;

/* --- element level ----------------------------------------------------- */
void or_shape(const double L[4], double N[10]);
void or_shape_dref(const double L[4], double dN[10][3]);
double or_grad(const double X[10][3], const double L[4], double G[10][3]);
void or_bmatrix(const double G[10][3], double B[6][30]);
void or_quad_points(double L[4][4], double *wfrac);
void or_element_stiffness(const double X[10][3], const double D[4][6][6], double K[30][30]);
void or_element_mass(const double X[10][3], double rho, double M[10][10]);
void or_face_dashpot(const double FX[3][3], double rho, double vs, double vp, double C[18][18]);

/* --- spring law -------------------------------------------------------- */
typedef struct { double G0, gref, alpha, beta; } or_ro;
void or_ro_params(double rho, double vs, double gamma_ref, double h_max, or_ro *p);
double or_ro_g(double tau, const or_ro *p);
double or_ro_dg(double tau, const or_ro *p);
double or_ro_F(double gamma, const or_ro *p);
double or_spring_update(or_spring *s, double g_new, double dg, const or_ro *p);
double or_spring_tangent(const or_spring *s, const or_ro *p);

/* --- multi-spring point -------------------------------------------------- */
int or_spring_dirs(int S, double *q /*[S][6]*/, double *w);
void or_point_update(int S, const double *q, double w, double Kb, const or_ro *p, const double eps[6],
                     const double deps[6], or_spring *sp, double D[6][6]);
void or_elastic_D(int S, const double *q, double w, double Kb, double G0, double D[6][6]);

/* --- whole model ------------------------------------------------------- */
int or_state_init(const or_model *m, or_state *s);
int or_step(const or_model *m, or_state *s);
int or_operator(const or_model *m, const double *D, int which, const double *x, double *y);
int or_colouring(int64_t n_elems, int64_t n_nodes, const int32_t *conn, int32_t *colour);

/* --- two-level (P2 -> P1) preconditioner pieces (Sec. 2.2, after [SC14]) --------
 * The coarse model is the linear 4-node tetrahedral model on the same elements: its
 * nodes are the vertices of the quadratic mesh.  cid [n_nodes]: coarse index of each
 * vertex node (vertices numbered in ascending fine-node order) or -1 for an edge node;
 * par [n_nodes][2]: the coarse indices that interpolate the node -- (c, c) for a vertex,
 * the two end vertices of its edge (ascending) for an edge node.  Returns the coarse node
 * count, or -1 if a node is both a vertex and an edge node or its edge is inconsistent. */
int64_t or_coarse_map(int64_t n_elems, int64_t n_nodes, const int32_t *conn, int32_t *cid, int32_t *par);
/* Linear-tetrahedron gradients of the barycentric coordinates and volume. */
void or_p1_grads(const double X[4][3], double g[4][3], double *vol);
/* Coarse operator y_c = Op_c x_c on [n_coarse][3] vectors, element by element from the
 * vertex coordinates: which 0 K1 (V B^T Dbar B, Dbar the mean of the element's four
 * point tangents), 1 M1 (rho V (1 + delta_ab) / 20), 2 Cb1 (dashpots, A (1 + delta_ab)/12
 * times rho [Vs I + (Vp - Vs) n n^T]), 3 A1 = (4/dt^2 + 2a/dt) M1 + (1 + 2b/dt) K1 +
 * 2/dt Cb1.  For straight elements this is P^T Op P with P the linear interpolation of
 * the vertices onto the quadratic nodes. */
int or_coarse_operator(const or_model *m, const double *D, int which, int64_t n_coarse, const int32_t *cid,
                       const double *xc, double *yc);
double or_input_velocity(const or_model *m, int64_t n, int comp);
void or_strain(const or_model *m, int64_t e, int qp, const double *u, double eps[6]);

#ifdef __cplusplus
}
#endif
#endif
