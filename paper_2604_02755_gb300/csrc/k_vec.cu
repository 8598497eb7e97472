// Node-vector kernels: preconditioned CG (Sec. 2.2; 3x3 block Jacobi) with
// warp-shuffle block reductions finished in a fixed order (deterministic),
// the Newmark-beta updates below Eq. 1, surface gathers and conversions.
#include "kern_common.cuh"

namespace ns {

int vec_blocks(int64_t n_nodes) {
  int64_t nb = (n_nodes + kBlock - 1) / kBlock;
  const int64_t cap = 152 * 8;
  if (nb > cap) nb = cap;
  if (nb < 1) nb = 1;
  return (int)nb;
}

// Loop bounds of one block of a node-vector kernel: its member's slice [a0, a1) (w entries
// per node) when the launch is cut by members, else a grid-stride loop over [0, n).
struct VRange {
  int64_t i, end, step;
  int m;
};
__device__ __forceinline__ VRange vrange(const Seg *seg, int64_t n, int w) {
  if (seg) {
    const Seg sg = seg[blockIdx.x];
    return {sg.a0 * w + threadIdx.x, sg.a1 * w, (int64_t)blockDim.x, sg.m};
  }
  return {blockIdx.x * (int64_t)blockDim.x + threadIdx.x, n, (int64_t)gridDim.x * blockDim.x, 0};
}
static int vgrid(int64_t N, const SegList &sg) { return sg.seg ? sg.n : vec_blocks(N); }

// Block sum of the partial slots of value k that belong to member m (all n slots without members).
__device__ double part_sum(const double *__restrict__ part, int n, int k, const PartMap &pm, int m) {
  double acc = 0.0;
  const double *pk = part + (int64_t)k * n;
  if (!pm.off1) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += pk[i];
  } else {
    for (int i = pm.off1[m] + threadIdx.x; i < pm.off1[m + 1]; i += blockDim.x) acc += pk[i];
    if (pm.off2)
      for (int i = pm.base2 + pm.off2[m] + threadIdx.x; i < pm.base2 + pm.off2[m + 1]; i += blockDim.x) acc += pk[i];
  }
  return block_sum(acc);
}

__global__ void k_fill(double *x, double v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

__global__ void k_negate_copy(double *dst, const double *src, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = -src[i];
}

cudaError_t launch_fill(double *x, double v, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_fill<<<vec_blocks(n), kBlock, 0, s>>>(x, v, n);
  return cudaGetLastError();
}

cudaError_t launch_negate_copy(double *dst, const double *src, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_negate_copy<<<vec_blocks(n), kBlock, 0, s>>>(dst, src, n);
  return cudaGetLastError();
}

// packed symmetric 3x3: xx yy zz yz xz xy
__device__ __forceinline__ void sym3_apply(const double *J, const double r[3], double z[3]) {
  z[0] = J[0] * r[0] + J[5] * r[1] + J[4] * r[2];
  z[1] = J[5] * r[0] + J[1] * r[1] + J[3] * r[2];
  z[2] = J[4] * r[0] + J[3] * r[1] + J[2] * r[2];
}

__global__ void k_invert_blocks(const double *Jd, double *Jinv, float *Jinv32, int64_t N, int32_t *bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double *a = Jd + 6 * i;
    const double xx = a[0], yy = a[1], zz = a[2], yz = a[3], xz = a[4], xy = a[5];
    const double c00 = yy * zz - yz * yz, c11 = xx * zz - xz * xz, c22 = xx * yy - xy * xy;
    const double c12 = xy * xz - xx * yz, c02 = xy * yz - yy * xz, c01 = xz * yz - xy * zz;
    const double det = xx * c00 + xy * c01 + xz * c02;
    if (!(det > 0.0)) {
      atomicCAS(bad, 0, (int32_t)(i + 1));
      continue;
    }
    const double inv[6] = {c00 / det, c11 / det, c22 / det, c12 / det, c02 / det, c01 / det};
    for (int k = 0; k < 6; ++k) {
      Jinv[6 * i + k] = inv[k];
      if (Jinv32) Jinv32[6 * i + k] = (float)inv[k];
    }
  }
}

__global__ void k_invert_blocks32(const float *Jd, float *Jinv32, int64_t N, int32_t *bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const float *a = Jd + 6 * i;
    const float xx = a[0], yy = a[1], zz = a[2], yz = a[3], xz = a[4], xy = a[5];
    const float c00 = yy * zz - yz * yz, c11 = xx * zz - xz * xz, c22 = xx * yy - xy * xy;
    const float c12 = xy * xz - xx * yz, c02 = xy * yz - yy * xz, c01 = xz * yz - xy * zz;
    const float det = xx * c00 + xy * c01 + xz * c02;
    if (!(det > 0.0f)) {
      atomicCAS(bad, 0, (int32_t)(i + 1));
      continue;
    }
    const float id = 1.0f / det;
    const float inv[6] = {c00 * id, c11 * id, c22 * id, c12 * id, c02 * id, c01 * id};
    for (int k = 0; k < 6; ++k) Jinv32[6 * i + k] = inv[k];
  }
}

cudaError_t launch_invert_blocks32(const float *Jd, float *Jinv32, int64_t N, int32_t *bad, cudaStream_t s) {
  k_invert_blocks32<<<vec_blocks(N), kBlock, 0, s>>>(Jd, Jinv32, N, bad);
  return cudaGetLastError();
}

cudaError_t launch_invert_blocks(const double *Jd, double *Jinv, float *Jinv32, int64_t N, int32_t *bad,
                                 cudaStream_t s) {
  k_invert_blocks<<<vec_blocks(N), kBlock, 0, s>>>(Jd, Jinv, Jinv32, N, bad);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ CG

__global__ void __launch_bounds__(kBlock) k_cg_init(const double *__restrict__ b, const double *__restrict__ Ap,
                                                    const double *__restrict__ Jinv, double *r, double *z, double *p,
                                                    int64_t N, double *part, const Seg *seg) {
  const VRange R = vrange(seg, N, 1);
  double bb = 0.0, rr = 0.0, rz = 0.0;
  for (int64_t i = R.i; i < R.end; i += R.step) {
    double rv[3], zv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double bv = b[3 * i + c];
      rv[c] = bv - Ap[3 * i + c];
      bb += bv * bv;
      rr += rv[c] * rv[c];
    }
    sym3_apply(Jinv + 6 * i, rv, zv);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      r[3 * i + c] = rv[c];
      z[3 * i + c] = zv[c];
      p[3 * i + c] = zv[c];
      rz += rv[c] * zv[c];
    }
  }
  const double s0 = block_sum(bb), s1 = block_sum(rr), s2 = block_sum(rz);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0;
    part[gridDim.x + blockIdx.x] = s1;
    part[2 * gridDim.x + blockIdx.x] = s2;
  }
}

cudaError_t launch_cg_init(const double *b, const double *Ap, const double *Jinv, double *r, double *z, double *p,
                           int64_t N, double *part, cudaStream_t s, SegList sg) {
  k_cg_init<<<vgrid(N, sg), kBlock, 0, s>>>(b, Ap, Jinv, r, z, p, N, part, sg.seg);
  return cudaGetLastError();
}

// One block per member, of up to 1,024 threads: the partial arrays of the element operators
// hold one slot per block of 256 elements (31,200 for the large model), and the final sum
// is on the critical path of every CG iteration.
constexpr int kFinalBlock = 1024;
__global__ void __launch_bounds__(kFinalBlock) k_cg_final(const double *__restrict__ part, int n, int nvals,
                                                     CgScalars *scs, int mode, double tol, int max_iter, PartMap pm,
                                                     const CgScalars *gate) {
  CgScalars *sc = scs + blockIdx.x;  // one block per member
  if (gate && gate[blockIdx.x].done) {  // (inner INIT) the member's outer solve has converged
    if (threadIdx.x == 0) sc->done = 1;
    return;
  }
  if (mode != NS_FIN_INIT && mode != NS_FIN_FCG_INIT && sc->done) return;
  double v[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < nvals; ++k) v[k] = part_sum(part, n, k, pm, blockIdx.x);
  if (threadIdx.x != 0) return;
  if (mode == NS_FIN_INIT) {
    sc->bb = v[0];
    sc->rr = v[1];
    sc->rr0 = v[1];
    sc->rz = v[2];
    sc->rz_old = v[2];
    sc->iters = 0;
    sc->alpha = 0.0;
    sc->beta = 0.0;
    sc->done = (v[0] == 0.0) ? 2 : (v[1] <= tol * tol * v[0] ? 1 : 0);
  } else if (mode == NS_FIN_PAP) {
    sc->pAp = v[0];
    sc->alpha = sc->rz_old / v[0];
  } else if (mode == NS_FIN_FCG_INIT) {
    sc->bb = v[0];
    sc->rr = v[1];
    sc->rr0 = v[1];
    sc->iters = 0;
    sc->beta = 0.0;
    sc->pAp = 1.0;
    sc->done = (v[0] == 0.0) ? 2 : (v[1] <= tol * tol * v[0] ? 1 : 0);
  } else if (mode == NS_FIN_FCG_BETA) {
    sc->beta = (sc->iters == 0) ? 0.0 : -v[0] / sc->pAp;
  } else if (mode == NS_FIN_FCG_UPDATE) {
    sc->rr = v[0];
    sc->iters += 1;
    if (v[0] <= tol * tol * sc->bb)
      sc->done = 1;
    else if (sc->iters >= max_iter)
      sc->done = 3;
  } else {
    sc->rr = v[0];
    sc->rz = v[1];
    sc->iters += 1;
    if (v[0] <= tol * tol * sc->bb)
      sc->done = 1;
    else if (sc->iters >= max_iter)
      sc->done = 3;
    sc->beta = v[1] / sc->rz_old;
    sc->rz_old = v[1];
  }
}

cudaError_t launch_cg_final(const double *part, int n, int nvals, CgScalars *sc, int mode, double tol, int max_iter,
                            cudaStream_t s, int M, PartMap pm, const CgScalars *gate) {
  // 1,024 threads where the partials are many; a small problem's few partials sum faster
  // in one block of 256 (a shorter block-wide reduction)
  k_cg_final<<<M, n > 8192 ? kFinalBlock : kBlock, 0, s>>>(part, n, nvals, sc, mode, tol, max_iter, pm, gate);
  return cudaGetLastError();
}

// alpha = (p.r) / (p.A p) of the flexible CG, from two partial arrays (one block per member)
__global__ void __launch_bounds__(kBlock) k_fcg_alpha(const double *__restrict__ pr, int npr,
                                                      const double *__restrict__ pap, int npap, CgScalars *scs,
                                                      PartMap pmr, PartMap pma) {
  CgScalars *sc = scs + blockIdx.x;
  if (sc->done) return;
  const double a = part_sum(pr, npr, 0, pmr, blockIdx.x);
  const double b = part_sum(pap, npap, 0, pma, blockIdx.x);
  if (threadIdx.x == 0) {
    sc->pAp = b;
    sc->alpha = a / b;
  }
}

cudaError_t launch_fcg_alpha(const double *pr, int npr, const double *pap, int npap, CgScalars *sc, cudaStream_t s,
                             int M, PartMap pmr, PartMap pma) {
  k_fcg_alpha<<<M, kBlock, 0, s>>>(pr, npr, pap, npap, sc, pmr, pma);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ flexible outer CG (FP64)
// Flexible CG with one-term orthogonalisation (Notay): z_k = B_k(r_k) (inner FP32 solve),
// p_k = z_k - (z_k.A p_{k-1} / p_{k-1}.A p_{k-1}) p_{k-1}, alpha_k = p_k.r_k / p_k.A p_k.

// z = ||r|| * x_in (undo the inner scaling; x_in is [N][4]); partial z . A p_{k-1}
__global__ void __launch_bounds__(kBlock) k_fcg_gamma(const float4 *__restrict__ xin, double *z,
                                                      const double *__restrict__ Ap, int64_t N, double *part,
                                                      const CgScalars *so, const Seg *seg) {
  const VRange R = vrange(seg, N, 1);
  if (so[R.m].done) return;
  const double nr = sqrt(so[R.m].rr);
  double g = 0.0;
  for (int64_t i = R.i; i < R.end; i += R.step) {
    const float4 xv = xin[i];
    const double z0 = (double)xv.x * nr, z1 = (double)xv.y * nr, z2 = (double)xv.z * nr;
    z[3 * i] = z0;
    z[3 * i + 1] = z1;
    z[3 * i + 2] = z2;
    g += z0 * Ap[3 * i] + z1 * Ap[3 * i + 1] + z2 * Ap[3 * i + 2];
  }
  g = block_sum(g);
  if (threadIdx.x == 0) part[blockIdx.x] = g;
}

// p = z + beta p; partial p . r; Ap = 0 (and Kp = 0 when the solve also accumulates K du)
__global__ void __launch_bounds__(kBlock) k_fcg_p(double *p, const double *__restrict__ z,
                                                  const double *__restrict__ r, double *Ap, double *Kp, int64_t n3,
                                                  double *part, const CgScalars *so, const Seg *seg) {
  const VRange R = vrange(seg, n3, 3);
  if (so[R.m].done) return;
  const double beta = so[R.m].beta;
  double a = 0.0;
  for (int64_t i = R.i; i < R.end; i += R.step) {
    const double pi = z[i] + beta * p[i];
    p[i] = pi;
    a += pi * r[i];
    Ap[i] = 0.0;
    if (Kp) Kp[i] = 0.0;
  }
  a = block_sum(a);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}

// x += alpha p; r -= alpha A p; partial r . r.  With q: q += alpha K p, so that q gains
// K x over the solve when x starts from zero (x = sum alpha_k p_k).
__global__ void __launch_bounds__(kBlock) k_fcg_update(double *x, double *r, const double *__restrict__ p,
                                                       const double *__restrict__ Ap, double *q,
                                                       const double *__restrict__ Kp, int64_t n3, double *part,
                                                       const CgScalars *so, const Seg *seg) {
  const VRange R = vrange(seg, n3, 3);
  if (so[R.m].done) return;
  const double alpha = so[R.m].alpha;
  double a = 0.0;
  for (int64_t i = R.i; i < R.end; i += R.step) {
    x[i] += alpha * p[i];
    if (q) q[i] += alpha * Kp[i];
    const double ri = r[i] - alpha * Ap[i];
    r[i] = ri;
    a += ri * ri;
  }
  a = block_sum(a);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}

// r = b - Ap; partials b.b, r.r
__global__ void __launch_bounds__(kBlock) k_fcg_init(const double *__restrict__ b, const double *__restrict__ Ap,
                                                     double *r, int64_t n3, double *part, const Seg *seg) {
  const VRange R = vrange(seg, n3, 3);
  double bb = 0.0, rr = 0.0;
  for (int64_t i = R.i; i < R.end; i += R.step) {
    const double bv = b[i], rv = bv - Ap[i];
    r[i] = rv;
    bb += bv * bv;
    rr += rv * rv;
  }
  const double s0 = block_sum(bb), s1 = block_sum(rr);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0;
    part[gridDim.x + blockIdx.x] = s1;
  }
}

cudaError_t launch_fcg_init(const double *b, const double *Ap, double *r, int64_t N, double *part, cudaStream_t s, SegList sg) {
  k_fcg_init<<<vgrid(N, sg), kBlock, 0, s>>>(b, Ap, r, 3 * N, part, sg.seg);
  return cudaGetLastError();
}
cudaError_t launch_fcg_gamma(const float *xin, double *z, const double *Ap, int64_t N, double *part,
                             const CgScalars *so, cudaStream_t s, SegList sg) {
  k_fcg_gamma<<<vgrid(N, sg), kBlock, 0, s>>>(reinterpret_cast<const float4 *>(xin), z, Ap, N, part, so, sg.seg);
  return cudaGetLastError();
}
cudaError_t launch_fcg_p(double *p, const double *z, const double *r, double *Ap, double *Kp, int64_t N,
                         double *part, const CgScalars *so, cudaStream_t s, SegList sg) {
  k_fcg_p<<<vgrid(N, sg), kBlock, 0, s>>>(p, z, r, Ap, Kp, 3 * N, part, so, sg.seg);
  return cudaGetLastError();
}
cudaError_t launch_fcg_update(double *x, double *r, const double *p, const double *Ap, double *q, const double *Kp,
                              int64_t N, double *part, const CgScalars *so, cudaStream_t s, SegList sg) {
  k_fcg_update<<<vgrid(N, sg), kBlock, 0, s>>>(x, r, p, Ap, q, Kp, 3 * N, part, so, sg.seg);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ inner FP32 PCG (preconditioner)
// Solves A x_in = r / ||r|| approximately in FP32 (FP64 reductions), block-Jacobi
// preconditioned, from x_in = 0.  Skips when the outer CG is done.  Its vectors are
// [N][4] (x y z and a zero pad) so that the operator gathers and scatters one 16-byte
// row per node.

__device__ __forceinline__ float4 sym3_apply_f(const float *J, const float4 r) {
  return make_float4(J[0] * r.x + J[5] * r.y + J[4] * r.z, J[5] * r.x + J[1] * r.y + J[3] * r.z,
                     J[4] * r.x + J[3] * r.y + J[2] * r.z, 0.0f);
}

__global__ void __launch_bounds__(kBlock) k_in_init(const double *__restrict__ r, const CgScalars *so,
                                                    const float *__restrict__ J, float4 *rin, float4 *zin, float4 *pin,
                                                    float4 *xin, float4 *Apin, int64_t N, double *part, const Seg *seg) {
  const VRange R = vrange(seg, N, 1);
  if (so[R.m].done) return;
  const double sc = 1.0 / sqrt(so[R.m].rr);
  float rr = 0.0f, rz = 0.0f;  // per-thread partials (a few dozen terms) in FP32
  const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int64_t i = R.i; i < R.end; i += R.step) {
    const float4 rv = make_float4((float)(r[3 * i] * sc), (float)(r[3 * i + 1] * sc), (float)(r[3 * i + 2] * sc), 0.0f);
    const float4 zv = sym3_apply_f(J + 6 * i, rv);
    rin[i] = rv;
    zin[i] = zv;
    pin[i] = zv;
    xin[i] = zero;
    Apin[i] = zero;
    rr = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, fmaf(rv.z, rv.z, rr)));
    rz = fmaf(rv.x, zv.x, fmaf(rv.y, zv.y, fmaf(rv.z, zv.z, rz)));
  }
  const double s0 = block_sum((double)rr), s1 = block_sum((double)rz);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0;
    part[gridDim.x + blockIdx.x] = s0;
    part[2 * gridDim.x + blockIdx.x] = s1;
  }
}

__global__ void __launch_bounds__(kBlock) k_in_update(float4 *xin, float4 *rin, float4 *zin,
                                                      const float4 *__restrict__ pin, const float4 *__restrict__ Apin,
                                                      const float *__restrict__ J, int64_t N, double *part,
                                                      const CgScalars *si, const CgScalars *so, const Seg *seg) {
  const VRange R = vrange(seg, N, 1);
  if (so[R.m].done || si[R.m].done) return;
  const float alpha = (float)si[R.m].alpha;
  float rr = 0.0f, rz = 0.0f;
  for (int64_t i = R.i; i < R.end; i += R.step) {
    const float4 pv = pin[i], av = Apin[i];
    float4 xv = xin[i], rv = rin[i];
    xv.x = fmaf(alpha, pv.x, xv.x);
    xv.y = fmaf(alpha, pv.y, xv.y);
    xv.z = fmaf(alpha, pv.z, xv.z);
    rv.x = fmaf(-alpha, av.x, rv.x);
    rv.y = fmaf(-alpha, av.y, rv.y);
    rv.z = fmaf(-alpha, av.z, rv.z);
    xin[i] = xv;
    rin[i] = rv;
    const float4 zv = sym3_apply_f(J + 6 * i, rv);
    zin[i] = zv;
    rr = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, fmaf(rv.z, rv.z, rr)));
    rz = fmaf(rv.x, zv.x, fmaf(rv.y, zv.y, fmaf(rv.z, zv.z, rz)));
  }
  const double s0 = block_sum((double)rr), s1 = block_sum((double)rz);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0;
    part[gridDim.x + blockIdx.x] = s1;
  }
}

__global__ void k_in_pupdate(float4 *pin, const float4 *__restrict__ zin, float4 *Apin, int64_t N, const CgScalars *si,
                             const CgScalars *so, const Seg *seg) {
  const VRange R = vrange(seg, N, 1);
  if (so[R.m].done || si[R.m].done) return;
  const float beta = (float)si[R.m].beta;
  const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int64_t i = R.i; i < R.end; i += R.step) {
    const float4 zv = zin[i];
    float4 pv = pin[i];
    pv.x = fmaf(beta, pv.x, zv.x);
    pv.y = fmaf(beta, pv.y, zv.y);
    pv.z = fmaf(beta, pv.z, zv.z);
    pin[i] = pv;
    Apin[i] = zero;
  }
}

static float4 *f4(float *p) { return reinterpret_cast<float4 *>(p); }
static const float4 *f4(const float *p) { return reinterpret_cast<const float4 *>(p); }

cudaError_t launch_in_init(const double *r, const CgScalars *so, const float *J, float *rin, float *zin, float *pin,
                           float *xin, float *Apin, int64_t N, double *part, cudaStream_t s, SegList sg) {
  k_in_init<<<vgrid(N, sg), kBlock, 0, s>>>(r, so, J, f4(rin), f4(zin), f4(pin), f4(xin), f4(Apin), N, part, sg.seg);
  return cudaGetLastError();
}
cudaError_t launch_in_update(float *xin, float *rin, float *zin, const float *pin, const float *Apin, const float *J,
                             int64_t N, double *part, const CgScalars *si, const CgScalars *so, cudaStream_t s, SegList sg) {
  k_in_update<<<vgrid(N, sg), kBlock, 0, s>>>(f4(xin), f4(rin), f4(zin), f4(pin), f4(Apin), J, N, part, si, so, sg.seg);
  return cudaGetLastError();
}
cudaError_t launch_in_pupdate(float *pin, const float *zin, float *Apin, int64_t N, const CgScalars *si,
                              const CgScalars *so, cudaStream_t s, SegList sg) {
  k_in_pupdate<<<vgrid(N, sg), kBlock, 0, s>>>(f4(pin), f4(zin), f4(Apin), N, si, so, sg.seg);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kBlock) k_cg_update(double *x, double *r, double *z, const double *__restrict__ p,
                                                      const double *__restrict__ Ap, const double *__restrict__ Jinv,
                                                      int64_t N, double *part, const CgScalars *sc, const Seg *seg) {
  const VRange R = vrange(seg, N, 1);
  if (sc[R.m].done) return;
  const double alpha = sc[R.m].alpha;
  double rr = 0.0, rz = 0.0;
  for (int64_t i = R.i; i < R.end; i += R.step) {
    double rv[3], zv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x[3 * i + c] += alpha * p[3 * i + c];
      rv[c] = r[3 * i + c] - alpha * Ap[3 * i + c];
      r[3 * i + c] = rv[c];
      rr += rv[c] * rv[c];
    }
    sym3_apply(Jinv + 6 * i, rv, zv);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      z[3 * i + c] = zv[c];
      rz += rv[c] * zv[c];
    }
  }
  const double s0 = block_sum(rr), s1 = block_sum(rz);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0;
    part[gridDim.x + blockIdx.x] = s1;
  }
}

cudaError_t launch_cg_update(double *x, double *r, double *z, const double *p, const double *Ap, const double *Jinv,
                             int64_t N, double *part, const CgScalars *sc, cudaStream_t s, SegList sg) {
  k_cg_update<<<vgrid(N, sg), kBlock, 0, s>>>(x, r, z, p, Ap, Jinv, N, part, sc, sg.seg);
  return cudaGetLastError();
}

__global__ void k_cg_pupdate(double *p, const double *__restrict__ z, double *Ap, int64_t n3, const CgScalars *sc, const Seg *seg) {
  const VRange R = vrange(seg, n3, 3);
  if (sc[R.m].done) return;
  const double beta = sc[R.m].beta;
  for (int64_t i = R.i; i < R.end; i += R.step) {
    p[i] = z[i] + beta * p[i];
    Ap[i] = 0.0;
  }
}

cudaError_t launch_cg_pupdate(double *p, const double *z, double *Ap, int64_t N, const CgScalars *sc, cudaStream_t s, SegList sg) {
  k_cg_pupdate<<<vgrid(N, sg), kBlock, 0, s>>>(p, z, Ap, 3 * N, sc, sg.seg);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Newmark-beta updates (below Eq. 1)

// du holds the increment; u += du; v <- -v + 2/dt du; a <- -a - 4/dt v_old + 4/dt^2 du.
__global__ void k_newmark(double *u, double *v, double *a, const double *__restrict__ du, int64_t n3, double dt) {
  const double c2 = 2.0 / dt, c4 = 4.0 / dt, c44 = 4.0 / (dt * dt);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = du[i], vo = v[i];
    u[i] += d;
    v[i] = -vo + c2 * d;
    a[i] = -a[i] - c4 * vo + c44 * d;
  }
}

cudaError_t launch_newmark(double *u, double *v, double *a, double *, const double *du, int64_t N, double dt,
                           cudaStream_t s) {
  k_newmark<<<vec_blocks(N), kBlock, 0, s>>>(u, v, a, du, 3 * N, dt);
  return cudaGetLastError();
}

__global__ void k_surface_gather(const int32_t *__restrict__ surf, int64_t Ns, const double *__restrict__ u,
                                 const double *__restrict__ v, const double *__restrict__ a, double *ou, double *ov,
                                 double *oa) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * Ns; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / 3, c = i % 3;
    const int64_t n = surf[s];
    ou[i] = u[3 * n + c];
    ov[i] = v[3 * n + c];
    oa[i] = a[3 * n + c];
  }
}

cudaError_t launch_surface_gather(const int32_t *surf, int64_t Ns, const double *u, const double *v, const double *a,
                                  double *ou, double *ov, double *oa, cudaStream_t s) {
  if (Ns <= 0) return cudaSuccess;
  k_surface_gather<<<vec_blocks(Ns), kBlock, 0, s>>>(surf, Ns, u, v, a, ou, ov, oa);
  return cudaGetLastError();
}

__global__ void k_d_to_f32(const double *src, float *dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

cudaError_t launch_d_to_f32(const double *src, float *dst, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_d_to_f32<<<vec_blocks(n), kBlock, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

__global__ void k_dot_partials(const double *x, const double *y, int64_t n, double *part) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += x[i] * y[i];
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

cudaError_t launch_dot_partials(const double *x, const double *y, int64_t n, double *part, cudaStream_t s) {
  k_dot_partials<<<vec_blocks(n), kBlock, 0, s>>>(x, y, n, part);
  return cudaGetLastError();
}

}  // namespace ns
