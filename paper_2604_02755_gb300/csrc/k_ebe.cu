// Element-by-element kernels (Sec. 2.2, Alg. 4: EBE matrix-vector products):
// geometry set-up, the operator y = mM M xm + mK M xk + kK K xk applied on the fly
// (K_e = sum_q w_q B^T D_q B, Eq. 2), Lysmer dashpot faces, block-Jacobi diagonal
// blocks and integration-point strains for the multi-spring update.
#include <atomic>

#include "kern_common.cuh"

namespace ns {

// ------------------------------------------------------------------ geometry

// grad L1..L3 are the rows of J^{-1}, J = [x1-x0, x2-x0, x3-x0] (columns); V = det J / 6.
// bad[0] receives 1 + the index of an element with non-positive volume or a curved edge.
__global__ void k_geometry(int64_t E, int64_t epad, const int32_t *__restrict__ conn, const double *__restrict__ xyz,
                           double *geom, float *geom32, int32_t *bad) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  double x[10][3];
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    int64_t n = conn[i * epad + e];
#pragma unroll
    for (int c = 0; c < 3; ++c) x[i][c] = xyz[n * 3 + c];
  }
  double J[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) J[r][c] = x[c + 1][r] - x[0][r];
  const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  bool ok = det > 0.0;
  // inverse: Jinv[k][c] = cofactor(c,k)/det -> row k of Jinv is grad L_{k+1}
  double inv[3][3];
  inv[0][0] = c00 / det;
  inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  inv[1][0] = c01 / det;
  inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  inv[2][0] = c02 / det;
  inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  // straight edges: edge node at the midpoint of its vertices
  const int ea[6] = {0, 1, 0, 0, 1, 2}, eb[6] = {1, 2, 2, 3, 3, 3};
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double len = 0.0, dev = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double d = x[eb[k]][c] - x[ea[k]][c];
      double m = 0.5 * (x[eb[k]][c] + x[ea[k]][c]) - x[4 + k][c];
      len += d * d;
      dev += m * m;
    }
    if (!(dev <= 1e-18 * len)) ok = false;
  }
  if (!ok) atomicCAS(bad, 0, (int32_t)(e + 1));
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      geom[(3 * k + c) * epad + e] = inv[k][c];
      geom32[(3 * k + c) * epad + e] = (float)inv[k][c];
    }
  geom[9 * epad + e] = det / 6.0;
  geom32[9 * epad + e] = (float)(det / 6.0);
}

__global__ void k_face_geometry(int64_t F, int64_t fpad, const int32_t *__restrict__ fnode,
                                const double *__restrict__ xyz, double *fgeom) {
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= F) return;
  double x[3][3];
  for (int i = 0; i < 3; ++i) {
    int64_t n = fnode[i * fpad + f];
    for (int c = 0; c < 3; ++c) x[i][c] = xyz[n * 3 + c];
  }
  double a[3], b[3];
  for (int c = 0; c < 3; ++c) {
    a[c] = x[1][c] - x[0][c];
    b[c] = x[2][c] - x[0][c];
  }
  double n0 = a[1] * b[2] - a[2] * b[1], n1 = a[2] * b[0] - a[0] * b[2], n2 = a[0] * b[1] - a[1] * b[0];
  double len = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
  fgeom[0 * fpad + f] = 0.5 * len;
  fgeom[1 * fpad + f] = n0 / len;
  fgeom[2 * fpad + f] = n1 / len;
  fgeom[3 * fpad + f] = n2 / len;
}

cudaError_t launch_geometry(const DevMesh &m, const double *xyz, int32_t *bad, cudaStream_t s) {
  if (m.Eb == 0) return cudaSuccess;
  k_geometry<<<(unsigned)((m.Eb + kBlock - 1) / kBlock), kBlock, 0, s>>>(m.Eb, m.epg, m.conn, xyz, m.geom, m.geom32,
                                                                         bad);
  return cudaGetLastError();
}

cudaError_t launch_face_geometry(const DevMesh &m, const double *xyz, cudaStream_t s) {
  if (m.Fb == 0) return cudaSuccess;
  k_face_geometry<<<(unsigned)((m.Fb + kBlock - 1) / kBlock), kBlock, 0, s>>>(m.Fb, m.fpg, m.fnode, xyz, m.fgeom);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ operator

// Entry m of the [84][epad] point-major tangent of element e: FP64 or FP32 as stored, or
// from FP16 pairs [42][epad] (entries 2j and 2j+1 in one 4-byte word).
__device__ __forceinline__ double dload(const double *__restrict__ D, int64_t epad, int64_t e, int m) {
  return __ldg(D + m * epad + e);
}
__device__ __forceinline__ float dload(const float *__restrict__ D, int64_t epad, int64_t e, int m) {
  return ldg(D + m * epad + e);  // no L1 allocation (kern_common.cuh)
}
__device__ __forceinline__ float dload(const __half2 *__restrict__ D, int64_t epad, int64_t e, int m) {
  unsigned u;
  asm("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(u) : "l"(D + (m >> 1) * epad + e));
  __half2 h;
  memcpy(&h, &u, 4);
  return (m & 1) ? __high2float(h) : __low2float(h);
}
__device__ __forceinline__ dd dload(const dd *__restrict__ D, int64_t epad, int64_t e, int m) {
  return ldg(D + m * epad + e);
}

// Stress of integration point Q from its strain: sig = w D_Q eps; dl(m) gives entry m of
// the element's [84] point-major tangent.
template <typename T, int Q, typename DL>
__device__ __forceinline__ void stress_of(const T eps[6], const DL &dl, T w, T sig[6]) {
  T d[21];
#pragma unroll
  for (int k = 0; k < 21; ++k) d[k] = (T)dl(Q * 21 + k);
  sig[0] = w * (d[0] * eps[0] + d[1] * eps[1] + d[2] * eps[2] + d[3] * eps[3] + d[4] * eps[4] + d[5] * eps[5]);
  sig[1] = w * (d[1] * eps[0] + d[6] * eps[1] + d[7] * eps[2] + d[8] * eps[3] + d[9] * eps[4] + d[10] * eps[5]);
  sig[2] = w * (d[2] * eps[0] + d[7] * eps[1] + d[11] * eps[2] + d[12] * eps[3] + d[13] * eps[4] + d[14] * eps[5]);
  sig[3] = w * (d[3] * eps[0] + d[8] * eps[1] + d[12] * eps[2] + d[15] * eps[3] + d[16] * eps[4] + d[17] * eps[5]);
  sig[4] = w * (d[4] * eps[0] + d[9] * eps[1] + d[13] * eps[2] + d[16] * eps[3] + d[18] * eps[4] + d[19] * eps[5]);
  sig[5] = w * (d[5] * eps[0] + d[10] * eps[1] + d[14] * eps[2] + d[17] * eps[3] + d[19] * eps[4] + d[20] * eps[5]);
}

// Stress of integration point Q: sig = w D_Q eps_Q(x).
template <typename T, int Q, typename DL>
__device__ __forceinline__ void point_stress(const T x[10][3], const T P[4][3], const T g[4][3], const DL &dl, T w,
                                             T sig[6]) {
  T H[3][3], eps[6];
  point_grad<T, Q>(x, P, g, H);
  voigt_strain(H, eps);
  stress_of<T, Q>(eps, dl, w, sig);
}

// One element of the operator: y_e = (kK K_e + mK M_e) x_e + mM M_e xm_e scattered into y
// (nodes nd, material mt, barycentric gradients g, volume vol, tangent entries dl(m));
// returns x_e . y_e when DOT.
// OUTK: the stiffness part K_e xk (unscaled) is also scattered into yk.
template <typename T, int VS, bool HAS_XM, bool ATOMIC, bool DOT, typename DL, bool OUTK = false>
__device__ __forceinline__ T ebe_element(const int nd[10], int mt, const T g[4][3], T vol, const DL &dl,
                                         const OpCoef *__restrict__ op, const typename VecOf<T>::type *__restrict__ xm,
                                         const typename VecOf<T>::type *__restrict__ xk, typename VecOf<T>::type *y,
                                         typename VecOf<T>::type *yk = nullptr) {
  const T cK = (T)op->kK[mt], cMk = (T)op->mK[mt];
  const T cMm = HAS_XM ? (T)op->mM[mt] : (T)0;
  T ye[10][3];
#pragma unroll
  for (int a = 0; a < 10; ++a)
#pragma unroll
    for (int r = 0; r < 3; ++r) ye[a][r] = (T)0;
  if (cK != (T)0) {
    T sig[4][6];  // D eps at the four points, the quadrature weight applied in the force sums
    {
      T x[10][3], P[4][3];
#pragma unroll
      for (int a = 0; a < 10; ++a) load_node<VS>(xk, nd[a], x[a]);
      compute_P(x, P);
      point_stress<T, 0>(x, P, g, dl, (T)1, sig[0]);
      point_stress<T, 1>(x, P, g, dl, (T)1, sig[1]);
      point_stress<T, 2>(x, P, g, dl, (T)1, sig[2]);
      point_stress<T, 3>(x, P, g, dl, (T)1, sig[3]);
    }
    const T w = OUTK ? vol * (T)0.25 : cK * vol * (T)0.25;
    points_force<T>(sig, g, w, ye);
    if (OUTK) {  // K_e x to yk, then the coefficient
#pragma unroll
      for (int a = 0; a < 10; ++a) add_node<VS, ATOMIC>(yk, nd[a], ye[a]);
#pragma unroll
      for (int a = 0; a < 10; ++a)
#pragma unroll
        for (int r = 0; r < 3; ++r) ye[a][r] = cK * ye[a][r];
    }
  }
  if (cMk != (T)0 || cMm != (T)0) {
    const T c = vol * (T)(1.0 / 420.0);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      T w[10];
#pragma unroll
      for (int a = 0; a < 10; ++a) {
        w[a] = cMk * vload<T>(xk + VS * (int64_t)nd[a] + r);
        if (HAS_XM) w[a] += cMm * vload<T>(xm + VS * (int64_t)nd[a] + r);
      }
      mass_apply_1(w, c, ye, r);
    }
  }
  T ld = (T)0;
  if (DOT) {
    // element-local x_e . y_e in the operator's precision (block sums in FP64)
#pragma unroll
    for (int a = 0; a < 10; ++a) {
      T xa[3];
      load_node<VS>(xk, nd[a], xa);
#pragma unroll
      for (int r = 0; r < 3; ++r) ld += xa[r] * ye[a][r];
    }
  }
#pragma unroll
  for (int a = 0; a < 10; ++a) add_node<VS, ATOMIC>(y, nd[a], ye[a]);
  return ld;
}

// L2 prefetch of a block's slice of the element rows (cp.async.bulk.prefetch: the TMA
// engine's linear prefetch, fire and forget): thread r < rows fetches one row's slice, so
// the per-thread loads that follow find the tangent, geometry, connectivity and material
// in L2 instead of waiting on DRAM one dependent load at a time.
__device__ __forceinline__ void l2_prefetch(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
template <typename T, typename TD>
__device__ __forceinline__ void prefetch_tile(int64_t eb, int64_t epad, const int32_t *conn, const T *geom,
                                              const int32_t *mat, const TD *D) {
  // rows start at 256-byte boundaries (epad a multiple of 64, eb of kBlock) and the slice
  // ends inside the row (epad - eb >= 64)
  const int64_t n = (epad - eb) < kBlock ? (epad - eb) : kBlock;
  constexpr int DR = std::is_same<TD, __half2>::value ? 42 : 84;
  const int r = threadIdx.x;
  if (r < DR)
    l2_prefetch(D + r * epad + eb, (uint32_t)(n * sizeof(TD)));
  else if (r < DR + 10)
    l2_prefetch(geom + (r - DR) * epad + eb, (uint32_t)(n * sizeof(T)));
  else if (r < DR + 20)
    l2_prefetch(conn + (r - DR - 10) * epad + eb, (uint32_t)(n * 4));
  else if (r == DR + 20)
    l2_prefetch(mat + eb, (uint32_t)(n * 4));
}

// Operator kernel, one thread per element.  Phases keep the register footprint small:
// (1) gather x, stresses at the four points; (2) nodal forces B^T sig; (3) consistent mass
// one displacement component at a time (re-gathered from cache); (4) scatter.
// FP32 variants are held to two resident blocks per SM (128 registers): the gathers and
// the tangent loads of more warps in flight outweigh the few spilled registers.
template <typename T, typename TD, int VS, bool HAS_XM, bool ATOMIC, bool DOT, bool OUTK = false>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 2 : 1)
    k_ebe(int64_t e0, int64_t e1, const int32_t *__restrict__ ids, const int32_t *__restrict__ conn,
          const T *__restrict__ geom, const int32_t *__restrict__ mat, const TD *__restrict__ D, int64_t epad,
          const OpCoef *__restrict__ op, const typename VecOf<T>::type *__restrict__ xm,
          const typename VecOf<T>::type *__restrict__ xk, typename VecOf<T>::type *y, double *dot,
          const int32_t *skip, const Seg *seg, int prefetch, typename VecOf<T>::type *yk, int64_t epg, int64_t Eb,
          int64_t Nb) {
  int64_t i, end;
  if (seg) {  // members: this block's slice of one member's elements, that member's skip flag
    const Seg sg = seg[blockIdx.x];
    i = sg.a0 + threadIdx.x;
    end = sg.a1;
    if (skip) skip += (int64_t)sg.m * kScStride;
  } else {
    i = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    end = e1;
  }
  if (skip && *skip) return;
  if (prefetch && !seg && !ids && e0 == 0) prefetch_tile(blockIdx.x * (int64_t)kBlock, epad, conn, geom, mat, D);
  double mydot = 0.0;
  if (i < end) {
    const int64_t e = ids ? (int64_t)ids[i] : i;
    int64_t eg;
    int32_t noff;
    shared_elem(e, Eb, Nb, eg, noff);
    int nd[10];
#pragma unroll
    for (int a = 0; a < 10; ++a) nd[a] = ldg(conn + a * epg + eg) + noff;
    const int mt = ldg(mat + e);
    T g[4][3], vol;
    load_grads(geom, epg, eg, g, vol);
    const auto dl = [&](int k) { return dload(D, epad, e, k); };
    mydot = (double)ebe_element<T, VS, HAS_XM, ATOMIC, DOT, decltype(dl), OUTK>(nd, mt, g, vol, dl, op, xm, xk, y, yk);
  }
  if (DOT) {
    double s = block_sum(mydot);
    if (threadIdx.x == 0) dot[blockIdx.x] = s;
  }
}

// ------------------------------------------------------------------ staged FP32 operator
// One block = one tile of kTile consecutive elements.  One thread issues bulk copies
// (cp.async.bulk: the TMA engine's linear form) of the tile's slice of every element row
// -- tangent D (84 rows of FP32, or 42 rows of FP16 pairs), FP32 geometry (10 rows),
// connectivity (10 rows), material (1 row) -- into shared memory, all completing on one
// mbarrier; the threads then compute from shared memory.  The whole tile (~107 KB for
// FP32 D) is in flight at once, where the direct kernel keeps only the loads its
// registers can hold.  Rows start at 256-byte boundaries (epad is a multiple of 64 and
// tiles are 1 KB), and a row copy never reaches past epad.
constexpr int kTile = kBlock;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase 0 (~ a second at most); false if it did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar) {
  for (int it = 0; it < (1 << 22); ++it)
    if (mbar_try_wait(bar, 0)) return true;
  return false;
}

template <typename TD>
__host__ __device__ constexpr int staged_d_rows() {
  return std::is_same<TD, float>::value ? 84 : 42;
}
template <typename TD>
__host__ __device__ constexpr size_t staged_smem() {
  return (size_t)(staged_d_rows<TD>() + 21) * kTile * 4 + 16;
}

__device__ __forceinline__ float dload_s(const float *Ds, int t, int m) { return Ds[m * kTile + t]; }
__device__ __forceinline__ float dload_s(const __half2 *Ds, int t, int m) {
  const __half2 h = Ds[(m >> 1) * kTile + t];
  return (m & 1) ? __high2float(h) : __low2float(h);
}

template <typename TD, bool DOT>
__global__ void __launch_bounds__(kTile, 2)
    k_ebe32_staged(int64_t E, int64_t epad, const int32_t *__restrict__ conn, const float *__restrict__ geom,
                   const int32_t *__restrict__ mat, const TD *__restrict__ D, const OpCoef *__restrict__ op,
                   const float *__restrict__ xk, float *y, double *dot, const int32_t *skip, int32_t *err) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int DR = staged_d_rows<TD>();
  TD *Ds = reinterpret_cast<TD *>(smem);                     // [DR][kTile]
  float *Gs = reinterpret_cast<float *>(smem + (size_t)DR * kTile * 4);  // [10][kTile]
  int32_t *Cs = reinterpret_cast<int32_t *>(Gs + 10 * kTile);          // [10][kTile]
  int32_t *Ms = Cs + 10 * kTile;                                       // [kTile]
  uint64_t *bar = reinterpret_cast<uint64_t *>(Ms + kTile);
  if (skip && *skip) return;
  const int t = threadIdx.x;
  const int64_t e0 = (int64_t)blockIdx.x * kTile;
  const int64_t rowlen = (epad - e0) < kTile ? (epad - e0) : kTile;  // a multiple of 64 elements
  const uint32_t rb = (uint32_t)(rowlen * 4);
  if (t == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (t == 0) {
    mbar_expect_tx(bar, rb * (uint32_t)(DR + 21));
    for (int r = 0; r < DR; ++r) bulk_g2s(Ds + r * kTile, D + r * epad + e0, rb, bar);
    for (int r = 0; r < 10; ++r) bulk_g2s(Gs + r * kTile, geom + r * epad + e0, rb, bar);
    for (int r = 0; r < 10; ++r) bulk_g2s(Cs + r * kTile, conn + r * epad + e0, rb, bar);
    bulk_g2s(Ms, mat + e0, rb, bar);
  }
  if (!mbar_wait_bounded(bar)) {
    // the copies did not complete: report, wait (bounded) for them once more, leave
    if (t == 0) atomicExch(err, 1);
    mbar_wait_bounded(bar);
    return;
  }
  double mydot = 0.0;
  const int64_t e = e0 + t;
  if (e < E) {
    int nd[10];
#pragma unroll
    for (int a = 0; a < 10; ++a) nd[a] = Cs[a * kTile + t];
    const int mt = Ms[t];
    float g[4][3], vol;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) g[k + 1][c] = Gs[(3 * k + c) * kTile + t];
#pragma unroll
    for (int c = 0; c < 3; ++c) g[0][c] = -(g[1][c] + g[2][c] + g[3][c]);
    vol = Gs[9 * kTile + t];
    const auto dl = [&](int k) { return dload_s(Ds, t, k); };
    mydot = (double)ebe_element<float, 4, false, true, DOT>(nd, mt, g, vol, dl, op, nullptr, xk, y);
  }
  if (DOT) {
    double s = block_sum(mydot);
    if (t == 0) dot[blockIdx.x] = s;
  }
}

// ------------------------------------------------------------------ per-warp staged FP32 operator
// One thread per element as in k_ebe, but each warp first issues asynchronous copies
// (cp.async, 16 bytes each, no registers held) of its 32 elements' tangent rows into shared
// memory, then loads connectivity and geometry, gathers x and forms the strains at the four
// points while the tangent is in flight, and only then waits for it: the tangent bytes (336
// of the 468 per element) no longer wait in registers, a few loads at a time.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ float dload_w(const float *Ds, int lane, int m) { return Ds[m * 32 + lane]; }
__device__ __forceinline__ float dload_w(const __half2 *Ds, int lane, int m) {
  const __half2 h = Ds[(m >> 1) * 32 + lane];
  return (m & 1) ? __high2float(h) : __low2float(h);
}
template <typename TD>
__host__ __device__ constexpr size_t warp_staged_smem() {
  return (size_t)staged_d_rows<TD>() * 32 * 4 * (kBlock / 32);
}

template <typename TD, bool DOT>
__global__ void __launch_bounds__(kBlock, 2)
    k_ebe32_warp(int64_t E, int64_t epad, const int32_t *__restrict__ conn, const float *__restrict__ geom,
                 const int32_t *__restrict__ mat, const TD *__restrict__ D, const OpCoef *__restrict__ op,
                 const float *__restrict__ xk, float *y, double *dot, const int32_t *skip, const Seg *seg,
                 int64_t epg, int64_t Eb, int64_t Nb) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int DR = staged_d_rows<TD>();
  int64_t a0, end;
  if (seg) {  // members: this block's slice of one member's elements (starting at a multiple of 32)
    const Seg sg = seg[blockIdx.x];
    a0 = sg.a0;
    end = sg.a1;
    if (skip) skip += (int64_t)sg.m * kScStride;
  } else {
    a0 = (int64_t)blockIdx.x * kBlock;
    end = E;
  }
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ew = a0 + warp * 32, e = ew + lane;
  TD *Ds = reinterpret_cast<TD *>(smem) + (size_t)warp * DR * 32;  // [DR][32]: the warp's tangent rows
  // rows start at 128-byte boundaries (epad a multiple of 64, ew of 32) and the warp's 32
  // entries of a row end inside it (ew < end <= E <= epad)
  if (ew < end) {
#pragma unroll 4
    for (int q = lane; q < DR * 8; q += 32) {
      const int r = q >> 3, part = q & 7;
      cp_async16(Ds + r * 32 + part * 4, D + (size_t)r * epad + ew + part * 4);
    }
  }
  cp_async_commit();
  const bool live = e < end;
  int nd[10], mt = 0;
  float g[4][3], vol = 0.0f, eps[4][6];
  if (live) {
    int64_t eg;  // the stored row of the element (members on one mesh share it) and its node shift
    int32_t noff;
    shared_elem(e, Eb, Nb, eg, noff);
#pragma unroll
    for (int a = 0; a < 10; ++a) nd[a] = ldg(conn + a * epg + eg) + noff;
    mt = ldg(mat + e);
    load_grads(geom, epg, eg, g, vol);
    float x[10][3], P[4][3], H[3][3];
#pragma unroll
    for (int a = 0; a < 10; ++a) load_node<4>(xk, nd[a], x[a]);
    compute_P(x, P);
    point_grad<float, 0>(x, P, g, H);
    voigt_strain(H, eps[0]);
    point_grad<float, 1>(x, P, g, H);
    voigt_strain(H, eps[1]);
    point_grad<float, 2>(x, P, g, H);
    voigt_strain(H, eps[2]);
    point_grad<float, 3>(x, P, g, H);
    voigt_strain(H, eps[3]);
  }
  cp_async_wait_all();
  __syncwarp();  // every lane's copies are complete and visible to the warp
  double mydot = 0.0;
  if (live) {
    const float cK = (float)op->kK[mt], cMk = (float)op->mK[mt];
    float ye[10][3], ld = 0.0f;
#pragma unroll
    for (int a = 0; a < 10; ++a)
#pragma unroll
      for (int r = 0; r < 3; ++r) ye[a][r] = 0.0f;
    if (cK != 0.0f) {
      const auto dl = [&](int k) { return dload_w(Ds, lane, k); };
      float sig[4][6];
      stress_of<float, 0>(eps[0], dl, 1.0f, sig[0]);
      stress_of<float, 1>(eps[1], dl, 1.0f, sig[1]);
      stress_of<float, 2>(eps[2], dl, 1.0f, sig[2]);
      stress_of<float, 3>(eps[3], dl, 1.0f, sig[3]);
      const float w = cK * vol * 0.25f;
      if (DOT) {  // x_e . K_e x_e = sum_q w eps_q . D_q eps_q, from what is in registers
        float e = 0.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int c = 0; c < 6; ++c) e += eps[q][c] * sig[q][c];
        ld = w * e;
      }
      points_force<float>(sig, g, w, ye);
    }
    if (cMk != 0.0f) {  // consistent mass: x gathered again (from cache), one vector load per node
      const float c = vol * (1.0f / 420.0f);
      float xs[10][3];
#pragma unroll
      for (int a = 0; a < 10; ++a) load_node<4>(xk, nd[a], xs[a]);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        float w[10], tm[10][3];
#pragma unroll
        for (int a = 0; a < 10; ++a) {
          w[a] = cMk * xs[a][r];
          tm[a][r] = 0.0f;
        }
        mass_apply_1(w, c, tm, r);
#pragma unroll
        for (int a = 0; a < 10; ++a) {
          ye[a][r] += tm[a][r];
          if (DOT) ld += xs[a][r] * tm[a][r];
        }
      }
    }
    mydot = (double)ld;
#pragma unroll
    for (int a = 0; a < 10; ++a) add_node<4, true>(y, nd[a], ye[a]);
  }
  if (DOT) {
    double sum = block_sum(mydot);
    if (threadIdx.x == 0) dot[blockIdx.x] = sum;
  }
}

// ------------------------------------------------------------------ locally gathered FP32 operator
// One block = kBlock consecutive elements.  Phase 1 gathers the block's distinct nodes (its
// node list, usually ~0.3 of its 10 kBlock element-node slots in a structured numbering)
// from x into shared memory with independent loads; phase 2 computes every element from
// shared memory (local 16-bit connectivity) and adds its forces into a shared accumulator
// with shared atomics; phase 3 adds the accumulator to y, one global vector atomic per
// distinct node.  The element arithmetic is ebe_element's (same point stresses, nodal
// forces and consistent mass), so only the order of the FP32 sums differs.
template <bool DOT, typename DL>
__device__ __forceinline__ float ebe_element_local(const int nd[10], int mt, const float g[4][3], float vol,
                                                   const DL &dl, const OpCoef *__restrict__ op, const float4 *xs,
                                                   float *ys) {
  const float cK = (float)op->kK[mt], cMk = (float)op->mK[mt];
  float ye[10][3];
#pragma unroll
  for (int a = 0; a < 10; ++a)
#pragma unroll
    for (int r = 0; r < 3; ++r) ye[a][r] = 0.0f;
  if (cK != 0.0f) {
    float sig[4][6];
    {
      float x[10][3], P[4][3];
#pragma unroll
      for (int a = 0; a < 10; ++a) {
        const float4 q = xs[nd[a]];
        x[a][0] = q.x;
        x[a][1] = q.y;
        x[a][2] = q.z;
      }
      compute_P(x, P);
      point_stress<float, 0>(x, P, g, dl, 1.0f, sig[0]);
      point_stress<float, 1>(x, P, g, dl, 1.0f, sig[1]);
      point_stress<float, 2>(x, P, g, dl, 1.0f, sig[2]);
      point_stress<float, 3>(x, P, g, dl, 1.0f, sig[3]);
    }
    points_force<float>(sig, g, cK * vol * 0.25f, ye);
  }
  if (cMk != 0.0f) {
    const float c = vol * (1.0f / 420.0f);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      float w[10];
#pragma unroll
      for (int a = 0; a < 10; ++a) w[a] = cMk * reinterpret_cast<const float *>(xs + nd[a])[r];
      mass_apply_1(w, c, ye, r);
    }
  }
  float ld = 0.0f;
#pragma unroll
  for (int a = 0; a < 10; ++a) {
    const float4 q = xs[nd[a]];
    if (DOT) ld += q.x * ye[a][0] + q.y * ye[a][1] + q.z * ye[a][2];
#pragma unroll
    for (int r = 0; r < 3; ++r) atomicAdd(ys + 4 * nd[a] + r, ye[a][r]);
  }
  return ld;
}

template <typename TD, bool DOT>
__global__ void __launch_bounds__(kBlock, 2)
    k_ebe32_local(int64_t E, int64_t epad, int64_t epg, const uint16_t *__restrict__ lconn,
                  const int32_t *__restrict__ lnode, const int64_t *__restrict__ loff, const float *__restrict__ geom,
                  const int32_t *__restrict__ mat, const TD *__restrict__ D, const OpCoef *__restrict__ op,
                  const float4 *__restrict__ x, float4 *y, double *dot, const int32_t *skip) {
  extern __shared__ float4 lsm[];
  if (skip && *skip) return;
  const int64_t b = blockIdx.x, u0 = loff[b];
  const int n = (int)(loff[b + 1] - u0);
  float4 *xs = lsm;
  float4 *ys = lsm + n;
  const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    xs[i] = __ldg(x + lnode[u0 + i]);
    ys[i] = zero;
  }
  __syncthreads();
  double mydot = 0.0;
  const int64_t e = b * kBlock + threadIdx.x;
  if (e < E) {
    int nd[10];
#pragma unroll
    for (int a = 0; a < 10; ++a) nd[a] = (int)__ldg(lconn + a * epg + e);
    const int mt = ldg(mat + e);
    float g[4][3], vol;
    load_grads(geom, epg, e, g, vol);
    const auto dl = [&](int k) { return dload(D, epad, e, k); };
    mydot = (double)ebe_element_local<DOT>(nd, mt, g, vol, dl, op, xs, reinterpret_cast<float *>(ys));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(y + lnode[u0 + i], ys[i]);
  if (DOT) {
    const double s = block_sum(mydot);
    if (threadIdx.x == 0) dot[blockIdx.x] = s;
  }
}

template <typename TD>
static cudaError_t local_dispatch(const DevMesh &m, const TD *D, const OpCoef *op, const float *xk, float *y,
                                  double *dot, const int32_t *skip, cudaStream_t s) {
  const size_t smem = (size_t)m.lmax * 2 * sizeof(float4);
  static std::atomic<unsigned long long> done{0};  // per-device shared-memory opt-in
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done.load() & bit)) {
    cudaFuncSetAttribute(k_ebe32_local<TD, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLocalMaxNodes * 32);
    cudaFuncSetAttribute(k_ebe32_local<TD, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLocalMaxNodes * 32);
    done.fetch_or(bit);
  }
  const unsigned nb = (unsigned)((m.E + kBlock - 1) / kBlock);
  const float4 *x4 = reinterpret_cast<const float4 *>(xk);
  float4 *y4 = reinterpret_cast<float4 *>(y);
  if (dot)
    k_ebe32_local<TD, true><<<nb, kBlock, smem, s>>>(m.E, m.epad, m.epg, m.lconn, m.lnode, m.loff, m.geom32, m.mat, D,
                                                    op, x4, y4, dot, skip);
  else
    k_ebe32_local<TD, false><<<nb, kBlock, smem, s>>>(m.E, m.epad, m.epg, m.lconn, m.lnode, m.loff, m.geom32, m.mat,
                                                     D, op, x4, y4, dot, skip);
  return cudaGetLastError();
}

template <typename T, typename TD, int VS, bool HAS_XM>
static cudaError_t ebe_dispatch(const DevMesh &m, const TD *D, const T *geom, const OpCoef *op,
                                const typename VecOf<T>::type *xm, const typename VecOf<T>::type *xk,
                                typename VecOf<T>::type *y, const int32_t *ids, int64_t e0, int64_t e1, bool atomic,
                                double *dot, const int32_t *skip, cudaStream_t s, const SegList &sg,
                                typename VecOf<T>::type *yk = nullptr) {
  if (!sg.seg && e1 <= e0) return cudaSuccess;
  const unsigned nb = sg.seg ? (unsigned)sg.n : (unsigned)((e1 - e0 + kBlock - 1) / kBlock);
  if constexpr (!HAS_XM && VS == 3) {  // the outer CG's applications that also return K x
    if (yk && dot) {
      if (atomic)
        k_ebe<T, TD, VS, HAS_XM, true, true, true><<<nb, kBlock, 0, s>>>(
            e0, e1, ids, m.conn, geom, m.mat, D, m.epad, op, xm, xk, y, dot, skip, sg.seg, m.prefetch, yk, m.epg,
            m.eb_arg(), m.Nb);
      else
        k_ebe<T, TD, VS, HAS_XM, false, true, true><<<nb, kBlock, 0, s>>>(
            e0, e1, ids, m.conn, geom, m.mat, D, m.epad, op, xm, xk, y, dot, skip, sg.seg, m.prefetch, yk, m.epg,
            m.eb_arg(), m.Nb);
      return cudaGetLastError();
    }
  }
#define NS_EBE_LAUNCH(A, DT)                                                                                  \
  k_ebe<T, TD, VS, HAS_XM, A, DT><<<nb, kBlock, 0, s>>>(e0, e1, ids, m.conn, geom, m.mat, D, m.epad, op, xm, xk, y, \
                                                     dot, skip, sg.seg, m.prefetch, nullptr, m.epg, m.eb_arg(), m.Nb)
  if (atomic) {
    if (dot)
      NS_EBE_LAUNCH(true, true);
    else
      NS_EBE_LAUNCH(true, false);
  } else {
    if (dot)
      NS_EBE_LAUNCH(false, true);
    else
      NS_EBE_LAUNCH(false, false);
  }
#undef NS_EBE_LAUNCH
  return cudaGetLastError();
}

cudaError_t launch_ebe64(const DevMesh &m, const double *D, const OpCoef *op, const double *xm, const double *xk,
                         double *y, const int32_t *ids, int64_t e0, int64_t e1, bool atomic, double *dot,
                         const int32_t *skip, cudaStream_t s, SegList sg, const void *D2, double *yk) {
  if (D2 && m.geom2) {  // FP64-accurate operator in double-float arithmetic
    const dd *Dp = static_cast<const dd *>(D2);
    if (xm) return ebe_dispatch<dd, dd, 3, true>(m, Dp, m.geom2, op, xm, xk, y, ids, e0, e1, atomic, dot, skip, s, sg);
    return ebe_dispatch<dd, dd, 3, false>(m, Dp, m.geom2, op, nullptr, xk, y, ids, e0, e1, atomic, dot, skip, s, sg,
                                          yk);
  }
  if (xm)
    return ebe_dispatch<double, double, 3, true>(m, D, m.geom, op, xm, xk, y, ids, e0, e1, atomic, dot, skip, s, sg);
  return ebe_dispatch<double, double, 3, false>(m, D, m.geom, op, nullptr, xk, y, ids, e0, e1, atomic, dot, skip, s,
                                                sg, yk);
}

template <typename TD>
static cudaError_t staged_dispatch(const DevMesh &m, const TD *D, const OpCoef *op, const float *xk, float *y,
                                   double *dot, const int32_t *skip, cudaStream_t s) {
  constexpr size_t smem = staged_smem<TD>();
  // the shared-memory opt-in is a per-device attribute of each instantiation
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done.load() & bit)) {
    cudaFuncSetAttribute(k_ebe32_staged<TD, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_ebe32_staged<TD, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    done.fetch_or(bit);
  }
  const unsigned nb = (unsigned)((m.E + kTile - 1) / kTile);
  if (dot)
    k_ebe32_staged<TD, true><<<nb, kTile, smem, s>>>(m.E, m.epad, m.conn, m.geom32, m.mat, D, op, xk, y, dot, skip,
                                                    m.kerr);
  else
    k_ebe32_staged<TD, false><<<nb, kTile, smem, s>>>(m.E, m.epad, m.conn, m.geom32, m.mat, D, op, xk, y, dot, skip,
                                                     m.kerr);
  return cudaGetLastError();
}

template <typename TD>
static cudaError_t warp_dispatch(const DevMesh &m, const TD *D, const OpCoef *op, const float *xk, float *y,
                                 double *dot, const int32_t *skip, cudaStream_t s, const SegList &sg) {
  constexpr size_t smem = warp_staged_smem<TD>();
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done.load() & bit)) {
    cudaFuncSetAttribute(k_ebe32_warp<TD, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_ebe32_warp<TD, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    done.fetch_or(bit);
  }
  const unsigned nb = sg.seg ? (unsigned)sg.n : (unsigned)((m.E + kBlock - 1) / kBlock);
  if (dot)
    k_ebe32_warp<TD, true><<<nb, kBlock, smem, s>>>(m.E, m.epad, m.conn, m.geom32, m.mat, D, op, xk, y, dot, skip,
                                                   sg.seg, m.epg, m.eb_arg(), m.Nb);
  else
    k_ebe32_warp<TD, false><<<nb, kBlock, smem, s>>>(m.E, m.epad, m.conn, m.geom32, m.mat, D, op, xk, y, dot, skip,
                                                    sg.seg, m.epg, m.eb_arg(), m.Nb);
  return cudaGetLastError();
}

cudaError_t launch_ebe32(const DevMesh &m, const float *D, const OpCoef *op, const float *xk, float *y,
                         const int32_t *ids, int64_t e0, int64_t e1, bool atomic, double *dot, const int32_t *skip,
                         cudaStream_t s, SegList sg, int stage) {
  const bool whole = atomic && !ids && !sg.seg && e0 == 0 && e1 == m.E && m.Msh == 1;
  // the per-warp kernel also takes the members' launch cuts when every cut starts at a
  // multiple of 32 elements (members on one mesh of such a size)
  const bool warp_ok = atomic && !ids && (sg.seg ? m.eseg32 : (e0 == 0 && e1 == m.E));
  if (stage == 1 && whole && m.kerr) return staged_dispatch<float>(m, D, op, xk, y, dot, skip, s);
  if (stage == 2 && warp_ok) return warp_dispatch<float>(m, D, op, xk, y, dot, skip, s, sg);
  if (m.lmax > 0 && atomic && !ids && !sg.seg && e0 == 0 && e1 == m.E && m.Msh == 1)
    return local_dispatch<float>(m, D, op, xk, y, dot, skip, s);
  // inner-solve vectors are [N][4]
  return ebe_dispatch<float, float, 4, false>(m, D, m.geom32, op, nullptr, xk, y, ids, e0, e1, atomic, dot, skip, s,
                                              sg);
}

cudaError_t launch_ebe16(const DevMesh &m, const void *D16, const OpCoef *op, const float *xk, float *y,
                         const int32_t *ids, int64_t e0, int64_t e1, bool atomic, double *dot, const int32_t *skip,
                         cudaStream_t s, SegList sg, int stage) {
  const bool whole = atomic && !ids && !sg.seg && e0 == 0 && e1 == m.E && m.Msh == 1;
  const bool warp_ok = atomic && !ids && (sg.seg ? m.eseg32 : (e0 == 0 && e1 == m.E));
  if (stage == 1 && whole && m.kerr)
    return staged_dispatch<__half2>(m, static_cast<const __half2 *>(D16), op, xk, y, dot, skip, s);
  if (stage == 2 && warp_ok)
    return warp_dispatch<__half2>(m, static_cast<const __half2 *>(D16), op, xk, y, dot, skip, s, sg);
  if (m.lmax > 0 && atomic && !ids && !sg.seg && e0 == 0 && e1 == m.E && m.Msh == 1)
    return local_dispatch<__half2>(m, static_cast<const __half2 *>(D16), op, xk, y, dot, skip, s);
  return ebe_dispatch<float, __half2, 4, false>(m, static_cast<const __half2 *>(D16), m.geom32, op, nullptr, xk, y,
                                                ids, e0, e1, atomic, dot, skip, s, sg);
}

// ------------------------------------------------------------------ dashpot faces

// C_f = (A/180) Mtri (x) rho [Vs I + (Vp - Vs) n n^T]; Mtri*180/A: vertex 6 / -1, vertex vs
// opposite edge -4 (else 0), edge 32 / 16.  Face nodes: v0 v1 v2 e01 e12 e02.
template <typename T, int VS, bool ATOMIC, bool DOT>
__global__ void __launch_bounds__(kBlock) k_faces(int64_t f0, int64_t f1, const int32_t *__restrict__ ids,
                                                  int64_t fpad, const int32_t *__restrict__ fnode,
                                                  const double *__restrict__ fgeom, const int32_t *__restrict__ fmat,
                                                  const int32_t *__restrict__ fkind, const MatConst *__restrict__ mc,
                                                  T cC, const T *__restrict__ x, const double *__restrict__ vin,
                                                  T *y, double *dot, const int32_t *skip, const Seg *seg,
                                                  const int32_t *__restrict__ fmem, int64_t vin_stride, int64_t fpg,
                                                  int64_t Fb, int64_t Nb) {
  int64_t i, end;
  if (seg) {
    const Seg sg = seg[blockIdx.x];
    i = sg.a0 + threadIdx.x;
    end = sg.a1;
    if (skip) skip += (int64_t)sg.m * kScStride;
  } else {
    i = f0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    end = f1;
  }
  if (skip && *skip) return;
  double mydot = 0.0;
  if (i < end) {
    const int64_t f = ids ? (int64_t)ids[i] : i;
    int64_t fg;
    int32_t noff;
    shared_elem(f, Fb, Nb, fg, noff);
    int nd[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) nd[a] = fnode[a * fpg + fg] + noff;
    const T area = (T)fgeom[fg];
    const T n[3] = {(T)fgeom[fpg + fg], (T)fgeom[2 * fpg + fg], (T)fgeom[3 * fpg + fg]};
    const MatConst &mm = mc[fmat[f]];
    const T rvs = (T)(mm.rho * mm.vs), rvd = (T)(mm.rho * (mm.vp - mm.vs));
    const bool inp = vin && fkind[fg] == 0;
    const double *vf = (vin && fmem) ? vin + fmem[f] * vin_stride : vin;  // the face's member's input
    T w[6][3];
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int r = 0; r < 3; ++r) w[a][r] = x[VS * (int64_t)nd[a] + r] + (inp ? (T)vf[r] : (T)0);
    T m[6][3];  // Mtri applied per component
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const T sv = w[0][r] + w[1][r] + w[2][r], se = w[3][r] + w[4][r] + w[5][r];
      m[0][r] = (T)7 * w[0][r] - sv - (T)4 * w[4][r];
      m[1][r] = (T)7 * w[1][r] - sv - (T)4 * w[5][r];
      m[2][r] = (T)7 * w[2][r] - sv - (T)4 * w[3][r];
      m[3][r] = (T)16 * (w[3][r] + se) - (T)4 * w[2][r];
      m[4][r] = (T)16 * (w[4][r] + se) - (T)4 * w[0][r];
      m[5][r] = (T)16 * (w[5][r] + se) - (T)4 * w[1][r];
    }
    const T sc = cC * area * (T)(1.0 / 180.0);
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      const T nm = n[0] * m[a][0] + n[1] * m[a][1] + n[2] * m[a][2];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const T v = sc * (rvs * m[a][r] + rvd * n[r] * nm);
        if (DOT) mydot += (double)x[VS * (int64_t)nd[a] + r] * (double)v;
        T *dst = y + VS * (int64_t)nd[a] + r;
        if (ATOMIC)
          atomic_add(dst, v);
        else
          *dst += v;
      }
    }
  }
  if (DOT) {
    double s = block_sum(mydot);
    if (threadIdx.x == 0) dot[blockIdx.x] = s;
  }
}

template <typename T, int VS>
static cudaError_t faces_dispatch(const DevMesh &m, const MatConst *mc, T cC, const T *x, const double *vin, T *y,
                                  const int32_t *ids, int64_t f0, int64_t f1, bool atomic, double *dot,
                                  const int32_t *skip, cudaStream_t s, const SegList &sg, const int32_t *fmem,
                                  int64_t vin_stride) {
  if (!sg.seg && f1 <= f0) return cudaSuccess;
  if (sg.seg && sg.n == 0) return cudaSuccess;
  const unsigned nb = sg.seg ? (unsigned)sg.n : (unsigned)((f1 - f0 + kBlock - 1) / kBlock);
#define NS_F_LAUNCH(A, DT) \
  k_faces<T, VS, A, DT><<<nb, kBlock, 0, s>>>(f0, f1, ids, m.fpad, m.fnode, m.fgeom, m.fmat, m.fkind, mc, cC, x, vin, y, \
                                              dot, skip, sg.seg, fmem, vin_stride, m.fpg, m.fb_arg(), m.Nb)
  if (atomic) {
    if (dot)
      NS_F_LAUNCH(true, true);
    else
      NS_F_LAUNCH(true, false);
  } else {
    if (dot)
      NS_F_LAUNCH(false, true);
    else
      NS_F_LAUNCH(false, false);
  }
#undef NS_F_LAUNCH
  return cudaGetLastError();
}

cudaError_t launch_faces64(const DevMesh &m, const MatConst *mc, double cC, const double *x, const double *vin,
                           double *y, const int32_t *ids, int64_t f0, int64_t f1, bool atomic, double *dot,
                           const int32_t *skip, cudaStream_t s, SegList sg, const int32_t *fmem, int64_t vin_stride) {
  return faces_dispatch<double, 3>(m, mc, cC, x, vin, y, ids, f0, f1, atomic, dot, skip, s, sg, fmem, vin_stride);
}

cudaError_t launch_faces32(const DevMesh &m, const MatConst *mc, float cC, const float *x, float *y,
                           const int32_t *ids, int64_t f0, int64_t f1, bool atomic, double *dot, const int32_t *skip,
                           cudaStream_t s, SegList sg) {
  return faces_dispatch<float, 4>(m, mc, cC, x, nullptr, y, ids, f0, f1, atomic, dot, skip, s, sg, nullptr, 0);
}

// ------------------------------------------------------------------ block-Jacobi diagonal blocks

// For node i of the element: sum_q w_q B_i^T D_q B_i (3x3) + mass diagonal, packed xx yy zz yz xz xy.
template <typename T, typename TD>
__global__ void __launch_bounds__(kBlock) k_jacobi_elems(int64_t e0, int64_t e1, const int32_t *__restrict__ ids,
                                                         const int32_t *__restrict__ conn,
                                                         const T *__restrict__ geom,
                                                         const int32_t *__restrict__ mat,
                                                         const TD *__restrict__ D, int64_t epad,
                                                         const OpCoef *__restrict__ op, T *Jd, bool atomic,
                                                         int64_t epg, int64_t Eb, int64_t Nb) {
  const int64_t i = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= e1) return;
  const int64_t e = ids ? (int64_t)ids[i] : i;
  int64_t eg;
  int32_t noff;
  shared_elem(e, Eb, Nb, eg, noff);
  const int mt = mat[e];
  const T cK = (T)op->kK[mt], cM = (T)op->mK[mt];
  T g[4][3], vol;
  load_grads(geom, epg, eg, g, vol);
  T acc[10][6];
#pragma unroll
  for (int a = 0; a < 10; ++a)
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[a][k] = (T)0;
  const T w = cK * vol * (T)0.25;
#pragma unroll 1
  for (int q = 0; q < 4; ++q) {
    T d[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) d[k] = w * dload(D, epad, e, q * 21 + k);
#pragma unroll
    for (int a = 0; a < 10; ++a) {
      T gn[3];
      if (a < 4) {
        const T c = (T)4.0 * (a == q ? (T)NS_QA : (T)NS_QB) - (T)1.0;
#pragma unroll
        for (int r = 0; r < 3; ++r) gn[r] = c * g[a][r];
      } else {
        const int pa = (a == 4 || a == 6 || a == 7) ? 0 : (a == 5 || a == 8) ? 1 : 2;
        const int pb = (a == 4) ? 1 : (a == 5 || a == 6) ? 2 : 3;
        const T la = pa == q ? (T)NS_QA : (T)NS_QB, lb = pb == q ? (T)NS_QA : (T)NS_QB;
#pragma unroll
        for (int r = 0; r < 3; ++r) gn[r] = (T)4.0 * (la * g[pb][r] + lb * g[pa][r]);
      }
      // columns of B_i: bx = (g0,0,0,0,g2,g1), by = (0,g1,0,g2,0,g0), bz = (0,0,g2,g1,g0,0)
      T Dbx[6], Dby[6], Dbz[6];
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        Dbx[r] = d[sym6(r, 0)] * gn[0] + d[sym6(r, 4)] * gn[2] + d[sym6(r, 5)] * gn[1];
        Dby[r] = d[sym6(r, 1)] * gn[1] + d[sym6(r, 3)] * gn[2] + d[sym6(r, 5)] * gn[0];
        Dbz[r] = d[sym6(r, 2)] * gn[2] + d[sym6(r, 3)] * gn[1] + d[sym6(r, 4)] * gn[0];
      }
      acc[a][0] += gn[0] * Dbx[0] + gn[2] * Dbx[4] + gn[1] * Dbx[5];  // xx
      acc[a][1] += gn[1] * Dby[1] + gn[2] * Dby[3] + gn[0] * Dby[5];  // yy
      acc[a][2] += gn[2] * Dbz[2] + gn[1] * Dbz[3] + gn[0] * Dbz[4];  // zz
      acc[a][3] += gn[1] * Dbz[1] + gn[2] * Dbz[3] + gn[0] * Dbz[5];  // yz = by . D bz
      acc[a][4] += gn[0] * Dbz[0] + gn[2] * Dbz[4] + gn[1] * Dbz[5];  // xz = bx . D bz
      acc[a][5] += gn[0] * Dby[0] + gn[2] * Dby[4] + gn[1] * Dby[5];  // xy = bx . D by
    }
  }
  const T mv = cM * vol * (T)(6.0 / 420.0), me = cM * vol * (T)(32.0 / 420.0);
#pragma unroll
  for (int a = 0; a < 10; ++a) {
    const T md = a < 4 ? mv : me;
    acc[a][0] += md;
    acc[a][1] += md;
    acc[a][2] += md;
    const int64_t n = conn[a * epg + eg] + noff;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      if (atomic)
        atomic_add(Jd + 6 * n + k, acc[a][k]);
      else
        Jd[6 * n + k] += acc[a][k];
    }
  }
}

template <typename T>
__global__ void k_jacobi_faces(int64_t f0, int64_t f1, const int32_t *__restrict__ ids, int64_t fpad,
                               const int32_t *__restrict__ fnode, const double *__restrict__ fgeom,
                               const int32_t *__restrict__ fmat, const MatConst *__restrict__ mc, double cC,
                               T *Jd, bool atomic, int64_t Fb, int64_t Nb) {
  const int64_t i = f0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= f1) return;
  const int64_t f = ids ? (int64_t)ids[i] : i;
  int64_t fg;
  int32_t noff;
  shared_elem(f, Fb, Nb, fg, noff);
  const double area = fgeom[fg], n[3] = {fgeom[fpad + fg], fgeom[2 * fpad + fg], fgeom[3 * fpad + fg]};
  const MatConst &mm = mc[fmat[f]];
  const double rvs = mm.rho * mm.vs, rvd = mm.rho * (mm.vp - mm.vs);
  const int pr[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
  for (int a = 0; a < 6; ++a) {
    const double md = cC * area / 180.0 * (a < 3 ? 6.0 : 32.0);
    const int64_t nd = fnode[a * fpad + fg] + noff;
    for (int k = 0; k < 6; ++k) {
      const int r = pr[k][0], c = pr[k][1];
      const T v = (T)(md * ((r == c ? rvs : 0.0) + rvd * n[r] * n[c]));
      if (atomic)
        atomic_add(Jd + 6 * nd + k, v);
      else
        Jd[6 * nd + k] += v;
    }
  }
}

cudaError_t launch_jacobi_elems(const DevMesh &m, const double *D, const OpCoef *op, double *Jd, const int32_t *ids,
                                int64_t e0, int64_t e1, bool atomic, cudaStream_t s) {
  if (e1 <= e0) return cudaSuccess;
  k_jacobi_elems<double, double><<<(unsigned)((e1 - e0 + kBlock - 1) / kBlock), kBlock, 0, s>>>(
      e0, e1, ids, m.conn, m.geom, m.mat, D, m.epad, op, Jd, atomic, m.epg, m.eb_arg(), m.Nb);
  return cudaGetLastError();
}

cudaError_t launch_jacobi_elems32(const DevMesh &m, const float *D, const OpCoef *op, float *Jd, const int32_t *ids,
                                  int64_t e0, int64_t e1, bool atomic, cudaStream_t s) {
  if (e1 <= e0) return cudaSuccess;
  k_jacobi_elems<float, float><<<(unsigned)((e1 - e0 + kBlock - 1) / kBlock), kBlock, 0, s>>>(
      e0, e1, ids, m.conn, m.geom32, m.mat, D, m.epad, op, Jd, atomic, m.epg, m.eb_arg(), m.Nb);
  return cudaGetLastError();
}

cudaError_t launch_jacobi_elems16(const DevMesh &m, const void *D16, const OpCoef *op, float *Jd, const int32_t *ids,
                                  int64_t e0, int64_t e1, bool atomic, cudaStream_t s) {
  if (e1 <= e0) return cudaSuccess;
  k_jacobi_elems<float, __half2><<<(unsigned)((e1 - e0 + kBlock - 1) / kBlock), kBlock, 0, s>>>(
      e0, e1, ids, m.conn, m.geom32, m.mat, static_cast<const __half2 *>(D16), m.epad, op, Jd, atomic, m.epg,
      m.eb_arg(), m.Nb);
  return cudaGetLastError();
}

cudaError_t launch_jacobi_faces(const DevMesh &m, const MatConst *mc, double cC, double *Jd, const int32_t *ids,
                                int64_t f0, int64_t f1, bool atomic, cudaStream_t s) {
  if (f1 <= f0) return cudaSuccess;
  k_jacobi_faces<double><<<(unsigned)((f1 - f0 + kBlock - 1) / kBlock), kBlock, 0, s>>>(
      f0, f1, ids, m.fpg, m.fnode, m.fgeom, m.fmat, mc, cC, Jd, atomic, m.fb_arg(), m.Nb);
  return cudaGetLastError();
}

cudaError_t launch_jacobi_faces32(const DevMesh &m, const MatConst *mc, double cC, float *Jd, const int32_t *ids,
                                  int64_t f0, int64_t f1, bool atomic, cudaStream_t s) {
  if (f1 <= f0) return cudaSuccess;
  k_jacobi_faces<float><<<(unsigned)((f1 - f0 + kBlock - 1) / kBlock), kBlock, 0, s>>>(
      f0, f1, ids, m.fpg, m.fnode, m.fgeom, m.fmat, mc, cC, Jd, atomic, m.fb_arg(), m.Nb);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ pair copies for the double-float operator

__global__ void k_to_pairs(const double *__restrict__ src, dd *dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = dd_from_double(src[i]);
}

cudaError_t launch_to_pairs(const double *src, void *dst, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_to_pairs<<<152 * 8, kBlock, 0, s>>>(src, static_cast<dd *>(dst), n);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ strains for the spring update

// Strains for the spring update: eps = B u and deps = B du at the four integration points
// of every element, in double-float arithmetic on the FP32 pipes, stored as the float pairs
// the spring kernel works on (out as float2 [4E][12]: eps then deps per point); one
// thread per element and vector (blockIdx.y: 0 for u, 1 for du).  The nodal values and gradients enter as pairs
// (dd_from_double: two FP64-pipe operations each instead of the FP64 arithmetic).
__global__ void __launch_bounds__(kBlock) k_strain_pairs(int64_t e0, int64_t e1, const int32_t *__restrict__ conn,
                                                         const double *__restrict__ geom, int64_t epg,
                                                         const double *__restrict__ u, const double *__restrict__ du,
                                                         float2 *out, int64_t Eb, int64_t Nb) {
  const int64_t e = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= e1) return;
  int64_t eg;
  int32_t noff;
  shared_elem(e, Eb, Nb, eg, noff);
  const int which = blockIdx.y;
  const double *src = which ? du : u;
  dd g[4][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) g[k + 1][c] = dd_from_double(__ldg(geom + (3 * k + c) * epg + eg));
#pragma unroll
  for (int c = 0; c < 3; ++c) g[0][c] = -(g[1][c] + g[2][c] + g[3][c]);
  dd x[10][3], P[4][3];
#pragma unroll
  for (int a = 0; a < 10; ++a) {
    const int64_t n = ldg(conn + a * epg + eg) + noff;
#pragma unroll
    for (int r = 0; r < 3; ++r) x[a][r] = dd_from_double(__ldg(src + 3 * n + r));
  }
  compute_P(x, P);
  dd H[3][3], eps[6];
  auto put = [&](int q) {  // 16-byte stores: the six pairs start at a 48-byte offset of a 96-byte row
    voigt_strain(H, eps);
    float4 *o = reinterpret_cast<float4 *>(out + (e * 4 + q) * 12 + 6 * which);
#pragma unroll
    for (int k = 0; k < 6; k += 2) o[k / 2] = make_float4(eps[k].h, eps[k].l, eps[k + 1].h, eps[k + 1].l);
  };
  point_grad<dd, 0>(x, P, g, H);
  put(0);
  point_grad<dd, 1>(x, P, g, H);
  put(1);
  point_grad<dd, 2>(x, P, g, H);
  put(2);
  point_grad<dd, 3>(x, P, g, H);
  put(3);
}

cudaError_t launch_strain_pairs(const DevMesh &m, const double *u, const double *du, void *out, int64_t e0, int64_t e1,
                                cudaStream_t s) {
  if (e1 <= e0) return cudaSuccess;
  const dim3 grid((unsigned)((e1 - e0 + kBlock - 1) / kBlock), 2);
  k_strain_pairs<<<grid, kBlock, 0, s>>>(e0, e1, m.conn, m.geom, m.epg, u, du, static_cast<float2 *>(out), m.eb_arg(),
                                         m.Nb);
  return cudaGetLastError();
}

}  // namespace ns
