// Device helpers shared by the library's kernels: quadratic-tetrahedron
// element arithmetic (Sec. 2.1), reductions and atomics.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "ns_internal.h"

namespace ns {

// Barycentric coordinates of the four integration points: (a, b, b, b) and
// permutations, a = (5 + 3 sqrt5)/20, b = (5 - sqrt5)/20 (degree-2 rule).
#define NS_QA 0.58541019662496845446
#define NS_QB 0.13819660112501051518

// local node index of the edge between vertices i and j (order (0,1) (1,2) (0,2) (0,3) (1,3) (2,3))
__host__ __device__ __forceinline__ constexpr int edge_node(int i, int j) {
  return (i < j ? i : j) == 0 ? ((i > j ? i : j) == 1 ? 4 : ((i > j ? i : j) == 2 ? 6 : 7))
                              : ((i < j ? i : j) == 1 ? ((i > j ? i : j) == 2 ? 5 : 8) : 9);
}

// packed index of entry (i, j) of a symmetric 6x6 (upper triangle, row major)
__host__ __device__ __forceinline__ constexpr int sym6(int i, int j) {
  return (i < j ? i : j) * 6 - ((i < j ? i : j) * ((i < j ? i : j) - 1)) / 2 + ((i > j ? i : j) - (i < j ? i : j));
}

// Element rows (connectivity, material, geometry, tangent) are read once per launch: the
// FP32 and integer ones bypass L1 allocation (ld.global.nc.L1::no_allocate) so that L1
// keeps the node gathers, which elements share.
template <typename T>
__device__ __forceinline__ T ldg(const T *p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ float ldg(const float *p) {
  float v;
  asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
template <>
__device__ __forceinline__ int ldg(const int *p) {
  int v;
  asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
// pairs are stored as float2
__device__ __forceinline__ dd ldg(const dd *p) {
  const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
  return dd(v.x, v.y);
}

// Node vectors of an operator in arithmetic type T: T itself, except that the pair type
// works on FP64 vectors (split on load, summed back to FP64 on store).
template <typename T>
struct VecOf {
  using type = T;
};
template <>
struct VecOf<dd> {
  using type = double;
};
template <typename T>
__device__ __forceinline__ T vld(const T *p) {
  return __ldg(p);
}
__device__ __forceinline__ dd vld_dd(const double *p) { return dd_from_double(__ldg(p)); }
template <typename T, typename TV>
__device__ __forceinline__ T vload(const TV *p) {
  if constexpr (std::is_same<T, dd>::value)
    return vld_dd(p);
  else
    return vld(p);
}

__device__ __forceinline__ void atomic_add(double *p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add(float *p, float v) { atomicAdd(p, v); }

// Node vectors are [N][VS]: VS = 3 (packed x y z) or, for the FP32 inner solve, VS = 4
// (x y z and a zero pad, one 16-byte row per node: one vector load per node gather and
// one vector atomic per node scatter).
template <int VS, typename T, typename TV>
__device__ __forceinline__ void load_node(const TV *__restrict__ x, int64_t n, T v[3]) {
  if constexpr (std::is_same<T, dd>::value) {
#pragma unroll
    for (int r = 0; r < 3; ++r) v[r] = vld_dd(x + VS * n + r);
  } else if constexpr (VS == 4 && std::is_same<T, float>::value) {
    const float4 q = __ldg(reinterpret_cast<const float4 *>(x) + n);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
  } else {
#pragma unroll
    for (int r = 0; r < 3; ++r) v[r] = __ldg(x + VS * n + r);
  }
}

template <int VS, bool ATOMIC, typename T, typename TV>
__device__ __forceinline__ void add_node(TV *y, int64_t n, const T v[3]) {
  if constexpr (std::is_same<T, dd>::value) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const double d = (double)v[r];
      if (ATOMIC)
        atomicAdd(y + VS * n + r, d);
      else
        y[VS * n + r] += d;
    }
  } else if constexpr (VS == 4 && std::is_same<T, float>::value) {
    float4 *d = reinterpret_cast<float4 *>(y) + n;
    if (ATOMIC) {
      atomicAdd(d, make_float4(v[0], v[1], v[2], 0.0f));
    } else {
      float4 o = *d;
      o.x += v[0];
      o.y += v[1];
      o.z += v[2];
      *d = o;
    }
  } else {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (ATOMIC)
        atomic_add(y + VS * n + r, v[r]);
      else
        y[VS * n + r] += v[r];
    }
  }
}

// Members that share one mesh are stored member after member: element i of a launch reads
// row i - m Eb of the shared connectivity and geometry, and its nodes are those of the shared
// mesh shifted by m Nb (m = i / Eb, the member).  Eb = 0: no sharing (row i, no shift).
__device__ __forceinline__ void shared_elem(int64_t i, int64_t Eb, int64_t Nb, int64_t &row, int32_t &noff) {
  if (Eb) {
    const int64_t m = i / Eb;
    row = i - m * Eb;
    noff = (int32_t)(m * Nb);
  } else {
    row = i;
    noff = 0;
  }
}

// Barycentric gradients of one element: g[0..3][3], from the stored grad L1..L3.
template <typename T>
__device__ __forceinline__ void load_grads(const T *__restrict__ geom, int64_t epad, int64_t e, T g[4][3], T &vol) {
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) g[k + 1][c] = ldg(geom + (3 * k + c) * epad + e);
#pragma unroll
  for (int c = 0; c < 3; ++c) g[0][c] = -(g[1][c] + g[2][c] + g[3][c]);
  vol = ldg(geom + 9 * epad + e);
}

// Displacement gradient at integration point q: grad u = sum_k G_k (x) grad L_k with
// G_k = P_k + 4(a-b) (q == k ? x_k : x_kq), P_k = (4b-1) x_k + 4b sum_{j != k} x_kj.
template <typename T, int q>
__device__ __forceinline__ void point_grad(const T x[10][3], const T P[4][3], const T g[4][3], T H[3][3]) {
  const T dab = (T)(4.0 * (NS_QA - NS_QB));
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) H[r][c] = (T)0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T Gk[3];
    const int nk = (k == q) ? k : edge_node(k, q);
#pragma unroll
    for (int r = 0; r < 3; ++r) Gk[r] = P[k][r] + dab * x[nk][r];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) H[r][c] += Gk[r] * g[k][c];
  }
}

template <typename T>
__device__ __forceinline__ void compute_P(const T x[10][3], T P[4][3]) {
  const T c1 = (T)(4.0 * NS_QB - 1.0), c2 = (T)(4.0 * NS_QB);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T s[3] = {0, 0, 0};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j != k)
#pragma unroll
        for (int r = 0; r < 3; ++r) s[r] += x[edge_node(k, j)][r];
#pragma unroll
    for (int r = 0; r < 3; ++r) P[k][r] = c1 * x[k][r] + c2 * s[r];
  }
}

template <typename T>
__device__ __forceinline__ void voigt_strain(const T H[3][3], T eps[6]) {
  eps[0] = H[0][0];
  eps[1] = H[1][1];
  eps[2] = H[2][2];
  eps[3] = H[1][2] + H[2][1];
  eps[4] = H[0][2] + H[2][0];
  eps[5] = H[0][1] + H[1][0];
}

// S g for a symmetric stress S in Voigt order (xx, yy, zz, yz, xz, xy)
template <typename T>
__device__ __forceinline__ void voigt_times(const T s[6], const T g[3], T out[3]) {
  out[0] = s[0] * g[0] + s[5] * g[1] + s[4] * g[2];
  out[1] = s[5] * g[0] + s[1] * g[1] + s[3] * g[2];
  out[2] = s[4] * g[0] + s[3] * g[1] + s[2] * g[2];
}

// The nodal forces of the stresses at all four points at once, each with quadrature weight
// w: y_i += w sum_q grad N_i(q) . S_q.  With L_k(q) = a (k = q) or b and
// U_j = 4 w sum_q L_j(q) S_q = 4 w b sum S + 4 w (a - b) S_j, the vertex k gets
// (U_k - w sum S) g_k and the edge node (k, j) gets U_j g_k + U_k g_j -- the same sums as
// point by point, in fewer operations.
template <typename T>
__device__ __forceinline__ void points_force(const T sig[4][6], const T g[4][3], T w, T y[10][3]) {
  const T b4 = (T)(4.0 * NS_QB) * w, d4 = (T)(4.0 * (NS_QA - NS_QB)) * w;
  T sum[6], U[4][6];
#pragma unroll
  for (int c = 0; c < 6; ++c) sum[c] = (sig[0][c] + sig[1][c]) + (sig[2][c] + sig[3][c]);
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int c = 0; c < 6; ++c) U[j][c] = b4 * sum[c] + d4 * sig[j][c];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T V[6], f[3];
#pragma unroll
    for (int c = 0; c < 6; ++c) V[c] = U[k][c] - w * sum[c];
    voigt_times(V, g[k], f);
#pragma unroll
    for (int r = 0; r < 3; ++r) y[k][r] += f[r];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int j = k + 1; j < 4; ++j) {
      T f1[3], f2[3];
      voigt_times(U[j], g[k], f1);
      voigt_times(U[k], g[j], f2);
      const int ne = edge_node(k, j);
#pragma unroll
      for (int r = 0; r < 3; ++r) y[ne][r] += f1[r] + f2[r];
    }
}

// Component r of y += c * 420 * M_ref w, with the exact consistent mass of a straight
// quadratic tetrahedron, M_ref * 420 / V: vertex-vertex 6 (diagonal) / 1; vertex-edge
// -4 (edge touches the vertex) / -6; edge-edge 32 (diagonal) / 16 (sharing a vertex) /
// 8 (opposite).  c carries V / 420 and the coefficient.
template <typename T>
__device__ __forceinline__ void mass_apply_1(const T w[10], T c, T y[10][3], int r) {
  const T sv = w[0] + w[1] + w[2] + w[3];
  const T se = w[4] + w[5] + w[6] + w[7] + w[8] + w[9];
  // vertex i: 5 w_i + sv - 6 se + 2 (sum of the three edges at i)
  const T vb = sv - (T)6 * se;
  y[0][r] += c * ((T)5 * w[0] + vb + (T)2 * (w[4] + w[6] + w[7]));
  y[1][r] += c * ((T)5 * w[1] + vb + (T)2 * (w[4] + w[5] + w[8]));
  y[2][r] += c * ((T)5 * w[2] + vb + (T)2 * (w[5] + w[6] + w[9]));
  y[3][r] += c * ((T)5 * w[3] + vb + (T)2 * (w[7] + w[8] + w[9]));
  // edge (a,b) with opposite edge o: -6 sv + 2 (w_a + w_b) + 16 se + 16 w_e - 8 w_o
  const T eb = (T)16 * se - (T)6 * sv;
  y[4][r] += c * (eb + (T)2 * (w[0] + w[1]) + (T)16 * w[4] - (T)8 * w[9]);
  y[5][r] += c * (eb + (T)2 * (w[1] + w[2]) + (T)16 * w[5] - (T)8 * w[7]);
  y[6][r] += c * (eb + (T)2 * (w[0] + w[2]) + (T)16 * w[6] - (T)8 * w[8]);
  y[7][r] += c * (eb + (T)2 * (w[0] + w[3]) + (T)16 * w[7] - (T)8 * w[5]);
  y[8][r] += c * (eb + (T)2 * (w[1] + w[3]) + (T)16 * w[8] - (T)8 * w[6]);
  y[9][r] += c * (eb + (T)2 * (w[2] + w[3]) + (T)16 * w[9] - (T)8 * w[4]);
}

// Block-wide sum of one double per thread; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

}  // namespace ns
