// Two-level preconditioner of the flexible CG (Sec. 2.2: EBE-IPCG with a multigrid
// preconditioner after [SC14]).  The coarse level is the linear 4-node tetrahedral model
// on the same elements (the vertices of the quadratic mesh); P interpolates it linearly
// onto the quadratic nodes and P^T restricts.  For straight elements the coarse operator
// below equals P^T A P: stiffness V B^T Dbar B with Dbar the mean of the element's four
// point tangents, consistent mass rho V (1 + delta_ab) / 20, dashpot faces
// A (1 + delta_ab) / 12 rho [Vs I + (Vp - Vs) n n^T].  Everything here is FP32 arithmetic
// with FP64 reductions, like the inner solve it prepares.
#include "kern_common.cuh"

namespace ns {

// sigma = D e for a symmetric 6x6 packed as its upper triangle, row major (sym6)
__device__ __forceinline__ void stress21(const float d[21], const float e[6], float s[6]) {
  s[0] = d[0] * e[0] + d[1] * e[1] + d[2] * e[2] + d[3] * e[3] + d[4] * e[4] + d[5] * e[5];
  s[1] = d[1] * e[0] + d[6] * e[1] + d[7] * e[2] + d[8] * e[3] + d[9] * e[4] + d[10] * e[5];
  s[2] = d[2] * e[0] + d[7] * e[1] + d[11] * e[2] + d[12] * e[3] + d[13] * e[4] + d[14] * e[5];
  s[3] = d[3] * e[0] + d[8] * e[1] + d[12] * e[2] + d[15] * e[3] + d[16] * e[4] + d[17] * e[5];
  s[4] = d[4] * e[0] + d[9] * e[1] + d[13] * e[2] + d[16] * e[3] + d[18] * e[4] + d[19] * e[5];
  s[5] = d[5] * e[0] + d[10] * e[1] + d[14] * e[2] + d[17] * e[3] + d[19] * e[4] + d[20] * e[5];
}

// ------------------------------------------------------------------ per-step set-up

// Dbar[k][e] = (D[k][e] + D[21 + k][e] + D[42 + k][e] + D[63 + k][e]) / 4 in FP32
__global__ void k_mg_dbar(const double *__restrict__ D, float *Dbar, int64_t epad, int64_t E) {
  const int k = blockIdx.y;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const double s = (D[k * epad + e] + D[(21 + k) * epad + e]) + (D[(42 + k) * epad + e] + D[(63 + k) * epad + e]);
    Dbar[k * epad + e] = (float)(0.25 * s);
  }
}

cudaError_t launch_mg_dbar(const double *D, float *Dbar, int64_t epad, int64_t E, cudaStream_t s) {
  if (E <= 0) return cudaSuccess;
  const unsigned nx = (unsigned)std::min<int64_t>((E + kBlock - 1) / kBlock, 152 * 2);
  k_mg_dbar<<<dim3(nx, 21), kBlock, 0, s>>>(D, Dbar, epad, E);
  return cudaGetLastError();
}

// Diagonal 3x3 blocks (packed xx yy zz yz xz xy) of the coarse A: per element vertex a,
// cK V B_a^T Dbar B_a + cM V / 10 I.
template <bool ATOMIC>
__global__ void __launch_bounds__(kBlock)
    k_mg_jacobi(int64_t e0, int64_t e1, const int32_t *__restrict__ ids, const int32_t *__restrict__ conn1,
                const float *__restrict__ geom, const int32_t *__restrict__ mat, const float *__restrict__ Dbar,
                int64_t epad, const OpCoef *__restrict__ op, float *Jd) {
  const int64_t i = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= e1) return;
  const int64_t e = ids ? (int64_t)ids[i] : i;
  const int mt = ldg(mat + e);
  float g[4][3], vol, d[21];
  load_grads(geom, epad, e, g, vol);
#pragma unroll
  for (int k = 0; k < 21; ++k) d[k] = ldg(Dbar + k * epad + e);
  const float cK = (float)op->kK[mt] * vol, cM = (float)op->mK[mt] * vol * 0.1f;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const float gx = g[a][0], gy = g[a][1], gz = g[a][2];
    // columns of B_a as Voigt strains, and Dbar times each
    const float cx[6] = {gx, 0.0f, 0.0f, 0.0f, gz, gy}, cy[6] = {0.0f, gy, 0.0f, gz, 0.0f, gx},
                cz[6] = {0.0f, 0.0f, gz, gy, gx, 0.0f};
    float sx[6], sy[6], sz[6];
    stress21(d, cx, sx);
    stress21(d, cy, sy);
    stress21(d, cz, sz);
    auto dot6 = [](const float *u, const float *v) {
      return u[0] * v[0] + u[1] * v[1] + u[2] * v[2] + u[3] * v[3] + u[4] * v[4] + u[5] * v[5];
    };
    const float blk[6] = {cK * dot6(cx, sx) + cM, cK * dot6(cy, sy) + cM, cK * dot6(cz, sz) + cM,
                          cK * dot6(cy, sz), cK * dot6(cx, sz), cK * dot6(cx, sy)};
    float *J = Jd + 6 * (int64_t)ldg(conn1 + a * epad + e);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      if (ATOMIC)
        atomicAdd(J + k, blk[k]);
      else
        J[k] += blk[k];
    }
  }
}

cudaError_t launch_mg_jacobi(const DevMesh &m, const MgLevel &c, const OpCoef *op, float *Jd, const int32_t *ids,
                             int64_t e0, int64_t e1, bool atomic, cudaStream_t s) {
  if (e1 <= e0) return cudaSuccess;
  const unsigned nb = (unsigned)((e1 - e0 + kBlock - 1) / kBlock);
  if (atomic)
    k_mg_jacobi<true><<<nb, kBlock, 0, s>>>(e0, e1, ids, c.conn1, m.geom32, m.mat, c.Dbar, m.epad, op, Jd);
  else
    k_mg_jacobi<false><<<nb, kBlock, 0, s>>>(e0, e1, ids, c.conn1, m.geom32, m.mat, c.Dbar, m.epad, op, Jd);
  return cudaGetLastError();
}

// Lysmer matrix rho [Vs I + (Vp - Vs) n n^T] of a face, packed xx yy zz yz xz xy
__device__ __forceinline__ void lysmer(const MatConst &p, float nx, float ny, float nz, float L[6]) {
  const float r = (float)p.rho, vs = (float)p.vs, dv = (float)(p.vp - p.vs);
  L[0] = r * (vs + dv * nx * nx);
  L[1] = r * (vs + dv * ny * ny);
  L[2] = r * (vs + dv * nz * nz);
  L[3] = r * dv * ny * nz;
  L[4] = r * dv * nx * nz;
  L[5] = r * dv * nx * ny;
}

template <bool ATOMIC>
__global__ void __launch_bounds__(kBlock)
    k_mg_jacobi_faces(int64_t f0, int64_t f1, const int32_t *__restrict__ ids, const int32_t *__restrict__ cfn,
                      int64_t fpad, const double *__restrict__ fgeom, const int32_t *__restrict__ fmat,
                      const MatConst *__restrict__ mc, float cC, float *Jd) {
  const int64_t i = f0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= f1) return;
  const int64_t f = ids ? (int64_t)ids[i] : i;
  float L[6];
  lysmer(mc[fmat[f]], (float)fgeom[fpad + f], (float)fgeom[2 * fpad + f], (float)fgeom[3 * fpad + f], L);
  const float w = cC * (float)fgeom[f] * (1.0f / 6.0f);
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    float *J = Jd + 6 * (int64_t)cfn[p * fpad + f];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      if (ATOMIC)
        atomicAdd(J + k, w * L[k]);
      else
        J[k] += w * L[k];
    }
  }
}

cudaError_t launch_mg_jacobi_faces(const DevMesh &m, const MgLevel &c, const MatConst *mc, float cC, float *Jd,
                                   const int32_t *ids, int64_t f0, int64_t f1, bool atomic, cudaStream_t s) {
  if (f1 <= f0) return cudaSuccess;
  const unsigned nb = (unsigned)((f1 - f0 + kBlock - 1) / kBlock);
  if (atomic)
    k_mg_jacobi_faces<true><<<nb, kBlock, 0, s>>>(f0, f1, ids, c.cfnode, m.fpad, m.fgeom, m.fmat, mc, cC, Jd);
  else
    k_mg_jacobi_faces<false><<<nb, kBlock, 0, s>>>(f0, f1, ids, c.cfnode, m.fpad, m.fgeom, m.fmat, mc, cC, Jd);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ coarse operator

// y_c += (cK K1 + cM M1) x_c over elements [e0, e1) (or ids[e0, e1)); with DOT the block
// partial of x_e . y_e goes to dot[blockIdx.x].  Vectors are [Nc][4] rows.
template <bool ATOMIC, bool DOT>
__global__ void __launch_bounds__(kBlock)
    k_mg_ebe(int64_t e0, int64_t e1, const int32_t *__restrict__ ids, const int32_t *__restrict__ conn1,
             const float *__restrict__ geom, const int32_t *__restrict__ mat, const float *__restrict__ Dbar,
             int64_t epad, const OpCoef *__restrict__ op, const float *__restrict__ x, float *y, double *dot,
             const int32_t *skip) {
  if (skip && *skip) return;
  const int64_t i = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double mydot = 0.0;
  if (i < e1) {
    const int64_t e = ids ? (int64_t)ids[i] : i;
    int nd[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) nd[a] = ldg(conn1 + a * epad + e);
    const int mt = ldg(mat + e);
    float g[4][3], vol, xa[4][3];
    load_grads(geom, epad, e, g, vol);
#pragma unroll
    for (int a = 0; a < 4; ++a) load_node<4>(x, nd[a], xa[a]);
    float eps[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      eps[0] += g[a][0] * xa[a][0];
      eps[1] += g[a][1] * xa[a][1];
      eps[2] += g[a][2] * xa[a][2];
      eps[3] += g[a][2] * xa[a][1] + g[a][1] * xa[a][2];
      eps[4] += g[a][2] * xa[a][0] + g[a][0] * xa[a][2];
      eps[5] += g[a][1] * xa[a][0] + g[a][0] * xa[a][1];
    }
    float d[21], sig[6];
#pragma unroll
    for (int k = 0; k < 21; ++k) d[k] = ldg(Dbar + k * epad + e);
    stress21(d, eps, sig);
    const float cK = (float)op->kK[mt] * vol, cM = (float)op->mK[mt] * vol * 0.05f;
    float sx[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int r = 0; r < 3; ++r) sx[r] += xa[a][r];
    float ld = 0.0f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      float f[3], ya[3];
      voigt_times(sig, g[a], f);
#pragma unroll
      for (int r = 0; r < 3; ++r) ya[r] = cK * f[r] + cM * (xa[a][r] + sx[r]);
      if (DOT) ld += xa[a][0] * ya[0] + xa[a][1] * ya[1] + xa[a][2] * ya[2];
      add_node<4, ATOMIC>(y, nd[a], ya);
    }
    mydot = (double)ld;
  }
  if (DOT) {
    const double s = block_sum(mydot);
    if (threadIdx.x == 0) dot[blockIdx.x] = s;
  }
}

cudaError_t launch_mg_ebe(const DevMesh &m, const MgLevel &c, const OpCoef *op, const float *x, float *y,
                          const int32_t *ids, int64_t e0, int64_t e1, bool atomic, double *dot, const int32_t *skip,
                          cudaStream_t s) {
  if (e1 <= e0) return cudaSuccess;
  const unsigned nb = (unsigned)((e1 - e0 + kBlock - 1) / kBlock);
#define NS_MG_EBE(A, DT)                                                                                        \
  k_mg_ebe<A, DT><<<nb, kBlock, 0, s>>>(e0, e1, ids, c.conn1, m.geom32, m.mat, c.Dbar, m.epad, op, x, y, dot, \
                                        skip)
  if (atomic) {
    if (dot)
      NS_MG_EBE(true, true);
    else
      NS_MG_EBE(true, false);
  } else {
    if (dot)
      NS_MG_EBE(false, true);
    else
      NS_MG_EBE(false, false);
  }
#undef NS_MG_EBE
  return cudaGetLastError();
}

// y_c += cC C1 x_c over faces, C1 = A (1 + delta_pq) / 12 Lysmer
template <bool ATOMIC, bool DOT>
__global__ void __launch_bounds__(kBlock)
    k_mg_faces(int64_t f0, int64_t f1, const int32_t *__restrict__ ids, const int32_t *__restrict__ cfn, int64_t fpad,
               const double *__restrict__ fgeom, const int32_t *__restrict__ fmat, const MatConst *__restrict__ mc,
               float cC, const float *__restrict__ x, float *y, double *dot, const int32_t *skip) {
  if (skip && *skip) return;
  const int64_t i = f0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double mydot = 0.0;
  if (i < f1) {
    const int64_t f = ids ? (int64_t)ids[i] : i;
    int nd[3];
    float xp[3][3], L[6];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      nd[p] = cfn[p * fpad + f];
      load_node<4>(x, nd[p], xp[p]);
    }
    lysmer(mc[fmat[f]], (float)fgeom[fpad + f], (float)fgeom[2 * fpad + f], (float)fgeom[3 * fpad + f], L);
    const float w = cC * (float)fgeom[f] * (1.0f / 12.0f);
    float ld = 0.0f;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      float v[3], yp[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) v[r] = xp[p][r] + (xp[0][r] + xp[1][r] + xp[2][r]);
      yp[0] = w * (L[0] * v[0] + L[5] * v[1] + L[4] * v[2]);
      yp[1] = w * (L[5] * v[0] + L[1] * v[1] + L[3] * v[2]);
      yp[2] = w * (L[4] * v[0] + L[3] * v[1] + L[2] * v[2]);
      if (DOT) ld += xp[p][0] * yp[0] + xp[p][1] * yp[1] + xp[p][2] * yp[2];
      add_node<4, ATOMIC>(y, nd[p], yp);
    }
    mydot = (double)ld;
  }
  if (DOT) {
    const double s = block_sum(mydot);
    if (threadIdx.x == 0) dot[blockIdx.x] = s;
  }
}

cudaError_t launch_mg_faces(const DevMesh &m, const MgLevel &c, const MatConst *mc, float cC, const float *x, float *y,
                            const int32_t *ids, int64_t f0, int64_t f1, bool atomic, double *dot, const int32_t *skip,
                            cudaStream_t s) {
  if (f1 <= f0) return cudaSuccess;
  const unsigned nb = (unsigned)((f1 - f0 + kBlock - 1) / kBlock);
#define NS_MG_FACES(A, DT)                                                                                          \
  k_mg_faces<A, DT><<<nb, kBlock, 0, s>>>(f0, f1, ids, c.cfnode, m.fpad, m.fgeom, m.fmat, mc, cC, x, y, dot, skip)
  if (atomic) {
    if (dot)
      NS_MG_FACES(true, true);
    else
      NS_MG_FACES(true, false);
  } else {
    if (dot)
      NS_MG_FACES(false, true);
    else
      NS_MG_FACES(false, false);
  }
#undef NS_MG_FACES
  return cudaGetLastError();
}

// ------------------------------------------------------------------ restriction and prolongation

__device__ __forceinline__ float4 sym3_f4(const float *J, const float4 r) {
  return make_float4(J[0] * r.x + J[5] * r.y + J[4] * r.z, J[5] * r.x + J[1] * r.y + J[3] * r.z,
                     J[4] * r.x + J[3] * r.y + J[2] * r.z, 0.0f);
}

// Coarse right-hand side and start of the coarse PCG: r_c = P^T (r / ||r||) gathered per
// coarse node in the listed order (rlist entries n >= 0: the vertex itself, weight 1;
// ~n < 0: an edge node n, weight 1/2), z_c = Jc r_c, p_c = z_c, x_c = 0, Ap_c = 0;
// partials of r_c.r_c (twice: the coarse b.b and r.r) and r_c.z_c.
__global__ void __launch_bounds__(kBlock)
    k_mg_restrict_init(const double *__restrict__ r, const CgScalars *so, const int64_t *__restrict__ rptr,
                       const int32_t *__restrict__ rlist, const float *__restrict__ J, float4 *rc, float4 *zc,
                       float4 *pc, float4 *xc, float4 *Apc, int64_t Nc, double *part) {
  if (so->done) return;
  const double sc = 1.0 / sqrt(so->rr);
  double rr = 0.0, rz = 0.0;
  const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < Nc; v += (int64_t)gridDim.x * blockDim.x) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int64_t j = rptr[v]; j < rptr[v + 1]; ++j) {
      const int32_t t = rlist[j];
      const int64_t n = t >= 0 ? t : ~t;
      const double w = t >= 0 ? 1.0 : 0.5;
      a0 += w * r[3 * n];
      a1 += w * r[3 * n + 1];
      a2 += w * r[3 * n + 2];
    }
    const float4 rv = make_float4((float)(a0 * sc), (float)(a1 * sc), (float)(a2 * sc), 0.0f);
    const float4 zv = sym3_f4(J + 6 * v, rv);
    rc[v] = rv;
    zc[v] = zv;
    pc[v] = zv;
    xc[v] = zero;
    Apc[v] = zero;
    rr += (double)rv.x * rv.x + (double)rv.y * rv.y + (double)rv.z * rv.z;
    rz += (double)rv.x * zv.x + (double)rv.y * zv.y + (double)rv.z * zv.z;
  }
  const double s0 = block_sum(rr), s1 = block_sum(rz);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0;
    part[gridDim.x + blockIdx.x] = s0;
    part[2 * gridDim.x + blockIdx.x] = s1;
  }
}

cudaError_t launch_mg_restrict_init(const double *r, const CgScalars *so, const MgLevel &c, float *rc, float *zc,
                                    float *pc, float *xc, float *Apc, double *part, cudaStream_t s) {
  k_mg_restrict_init<<<vec_blocks(c.Nc), kBlock, 0, s>>>(
      r, so, c.rptr, c.rlist, c.Jinv32, reinterpret_cast<float4 *>(rc), reinterpret_cast<float4 *>(zc),
      reinterpret_cast<float4 *>(pc), reinterpret_cast<float4 *>(xc), reinterpret_cast<float4 *>(Apc), c.Nc, part);
  return cudaGetLastError();
}

// x_in = P x_c (a vertex takes its coarse value, an edge node the mean of its two), Ap_in = 0
__global__ void k_mg_prolong(const float4 *__restrict__ xc, const int2 *__restrict__ par, float4 *xin, float4 *Apin,
                             int64_t N, const CgScalars *so) {
  if (so->done) return;
  const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const int2 p = par[n];
    const float4 a = xc[p.x], b = xc[p.y];
    xin[n] = p.x == p.y ? a : make_float4(0.5f * (a.x + b.x), 0.5f * (a.y + b.y), 0.5f * (a.z + b.z), 0.0f);
    Apin[n] = zero;
  }
}

cudaError_t launch_mg_prolong(const MgLevel &c, const float *xc, float *xin, float *Apin, int64_t N,
                              const CgScalars *so, cudaStream_t s) {
  k_mg_prolong<<<vec_blocks(N), kBlock, 0, s>>>(reinterpret_cast<const float4 *>(xc), c.par,
                                                  reinterpret_cast<float4 *>(xin), reinterpret_cast<float4 *>(Apin), N,
                                                  so);
  return cudaGetLastError();
}

// Start of the fine inner PCG from x_in = P x_c: r_in = r / ||r|| - A x_in, z = J r_in,
// p = z, Ap = 0; partials of b.b (b = r / ||r||), r_in.r_in, r_in.z.
__global__ void __launch_bounds__(kBlock)
    k_mg_fine_init(const double *__restrict__ r, const CgScalars *so, const float *__restrict__ J, float4 *rin,
                   float4 *zin, float4 *pin, float4 *Apin, int64_t N, double *part) {
  if (so->done) return;
  const double sc = 1.0 / sqrt(so->rr);
  double bb = 0.0, rr = 0.0, rz = 0.0;
  const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 ap = Apin[i];
    const float b0 = (float)(r[3 * i] * sc), b1 = (float)(r[3 * i + 1] * sc), b2 = (float)(r[3 * i + 2] * sc);
    const float4 rv = make_float4(b0 - ap.x, b1 - ap.y, b2 - ap.z, 0.0f);
    const float4 zv = sym3_f4(J + 6 * i, rv);
    rin[i] = rv;
    zin[i] = zv;
    pin[i] = zv;
    Apin[i] = zero;
    bb += (double)b0 * b0 + (double)b1 * b1 + (double)b2 * b2;
    rr += (double)rv.x * rv.x + (double)rv.y * rv.y + (double)rv.z * rv.z;
    rz += (double)rv.x * zv.x + (double)rv.y * zv.y + (double)rv.z * zv.z;
  }
  const double s0 = block_sum(bb), s1 = block_sum(rr), s2 = block_sum(rz);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0;
    part[gridDim.x + blockIdx.x] = s1;
    part[2 * gridDim.x + blockIdx.x] = s2;
  }
}

cudaError_t launch_mg_fine_init(const double *r, const CgScalars *so, const float *J, float *rin, float *zin,
                                float *pin, float *Apin, int64_t N, double *part, cudaStream_t s) {
  k_mg_fine_init<<<vec_blocks(N), kBlock, 0, s>>>(r, so, J, reinterpret_cast<float4 *>(rin),
                                                    reinterpret_cast<float4 *>(zin), reinterpret_cast<float4 *>(pin),
                                                    reinterpret_cast<float4 *>(Apin), N, part);
  return cudaGetLastError();
}

}  // namespace ns
