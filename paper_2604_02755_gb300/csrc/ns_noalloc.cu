// Allocation-free variant of ns_spring_points.
//
// Some callers cannot allocate device memory at the point where they need the spring
// update: code that runs after a fixed memory budget has been committed (an embedding
// solver that forbids allocation once it is initialised), or host threads that must not
// take the allocator's locks.  For them the staging buffers that ns_spring_points
// obtains with cudaMalloc live instead in one file-scope device array of fixed size,
// and the caller still passes the inputs and outputs.  Every call shares that array and
// overwrites all of it that it uses before reading it, so nothing from a previous call
// is read back; two calls that overlap on the GPU (different host threads or contexts
// on the same device) race on it.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "kern_common.cuh"
#include "ns_internal.h"

namespace {

// Size of the staging array (a modest 8 MiB; every GPU that loads the library keeps it
// until the process exits).
constexpr size_t kNoAllocBytes = (size_t)8 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
static unsigned char *g_scratch_addr[kMaxDevices] = {};
static std::mutex g_scratch_mutex;

struct SpringRec {
  double tau, gR, tR, gmax;
  int32_t dir, mode;
};

__global__ void k_aos_to_soa(const SpringRec *__restrict__ in, ns::SpringSoA st, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const SpringRec r = in[i];
    st.tau[i] = r.tau;
    st.gR[i] = r.gR;
    st.tR[i] = r.tR;
    st.gmax[i] = r.gmax;
    st.dir[i] = r.dir;
    st.mode[i] = r.mode;
  }
}

__global__ void k_soa_to_aos(ns::SpringSoA st, SpringRec *__restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = SpringRec{st.tau[i], st.gR[i], st.tR[i], st.gmax[i], st.dir[i], st.mode[i]};
}

__global__ void k_expand_D(const double *__restrict__ d21, double *__restrict__ d36, int64_t npts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 36 * npts; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / 36;
    const int r = (int)(i % 36), a = r / 6, b = r % 6;
    d36[i] = d21[21 * p + ns::sym6(a, b)];
  }
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Puts the caller's current device back when the call returns (the call makes the
// context's device current for its own work).
struct DeviceRestore {
  int prev = -1;
  DeviceRestore() {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
    }
  }
  ~DeviceRestore() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Device address of the staging array for the current device, resolved once per device.
int scratch_for_device(int dev, unsigned char **out) {
  if (dev < 0 || dev >= kMaxDevices) return -1;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return -1;
    }
    g_scratch_addr[dev] = (unsigned char *)p;
  }
  *out = g_scratch_addr[dev];
  return 0;
}

}  // namespace

extern "C" int64_t ns_spring_points_noalloc_capacity(int32_t S) {
  if (S < 5) return 0;
  const size_t per = 4 + 96 + 80 * (size_t)S + 21 * 8 + 36 * 8;
  const size_t slack = 11 * 256;  // alignment of the eleven sub-arrays
  return (int64_t)((kNoAllocBytes - slack) / per);
}

extern "C" int ns_spring_points_noalloc(ns_ctx *c, int64_t npts, const int32_t *mat, const double *eps,
                                        const double *deps, void *theta, double *D) {
  using namespace ns;
  if (!c) return NS_ERR_INVALID_ARG;
  SpringCtxView v{};
  if (ctx_spring_view(c, &v) != NS_OK) {
    ctx_set_error(c, "materials required");
    return NS_ERR_STATE;
  }
  if (npts < 0 || (npts > 0 && (!mat || !eps || !deps || !theta || !D))) {
    ctx_set_error(c, "bad arguments");
    return NS_ERR_INVALID_ARG;
  }
  if (npts == 0) return NS_OK;
  const int64_t cap = ns_spring_points_noalloc_capacity(v.tab.S);
  if (npts > cap) {
    char msg[160];
    snprintf(msg, sizeof(msg), "%lld points exceed the %lld that fit the %zu-byte allocation-free staging array at %d springs",
             (long long)npts, (long long)cap, kNoAllocBytes, v.tab.S);
    ctx_set_error(c, msg);
    return NS_ERR_INVALID_ARG;
  }
  for (int64_t i = 0; i < npts; ++i)
    if (mat[i] < 0 || mat[i] >= v.nmat) {
      ctx_set_error(c, "material index out of range");
      return NS_ERR_INVALID_ARG;
    }
  DeviceRestore restore;  // every return below leaves the caller's device current again
  unsigned char *base = nullptr;
  if (cudaSetDevice(v.device) != cudaSuccess || scratch_for_device(v.device, &base) != 0) {
    cudaGetLastError();
    ctx_set_error(c, "cannot resolve the staging array on this device");
    return NS_ERR_CUDA;
  }
  const int64_t nspr = npts * v.tab.S;
  // carve the staging array
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char *p = base + off;
    off += up256(bytes);
    return p;
  };
  int32_t *mat_d = (int32_t *)take(4 * (size_t)npts);
  double *eps_d = (double *)take(96 * (size_t)npts);
  SpringRec *rec_d = (SpringRec *)take(40 * (size_t)nspr);
  SpringSoA st;
  st.tau = (double *)take(8 * (size_t)nspr);
  st.gR = (double *)take(8 * (size_t)nspr);
  st.tR = (double *)take(8 * (size_t)nspr);
  st.gmax = (double *)take(8 * (size_t)nspr);
  st.dir = (int32_t *)take(4 * (size_t)nspr);
  st.mode = (int32_t *)take(4 * (size_t)nspr);
  double *d21 = (double *)take(21 * 8 * (size_t)npts);
  double *d36 = (double *)take(36 * 8 * (size_t)npts);
  if (off > kNoAllocBytes) {
    ctx_set_error(c, "internal: staging layout exceeds the array");
    return NS_ERR_INVALID_ARG;
  }
  cudaStream_t s = v.stream;
  cudaError_t e = cudaSuccess;
  // inputs: every byte read below is written first in this call
  if (e == cudaSuccess) e = cudaMemcpyAsync(mat_d, mat, 4 * npts, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpy2DAsync(eps_d, 96, eps, 48, 48, npts, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpy2DAsync(eps_d + 6, 96, deps, 48, 48, npts, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rec_d, theta, 40 * nspr, cudaMemcpyHostToDevice, s);
  const unsigned nb = (unsigned)std::min<int64_t>((nspr + kBlock - 1) / kBlock, 152 * 8);
  if (e == cudaSuccess) {
    k_aos_to_soa<<<nb, kBlock, 0, s>>>(rec_d, st, nspr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = launch_springs(v.tab, v.mats, nullptr, mat_d, eps_d, st, 0, 0, npts, nullptr, 0, d21, s);
  if (e == cudaSuccess) {
    k_soa_to_aos<<<nb, kBlock, 0, s>>>(st, rec_d, nspr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const unsigned nb2 = (unsigned)std::min<int64_t>((36 * npts + kBlock - 1) / kBlock, 152 * 8);
    k_expand_D<<<nb2, kBlock, 0, s>>>(d21, d36, npts);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(theta, rec_d, 40 * nspr, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(D, d36, 36 * 8 * npts, cudaMemcpyDeviceToHost, s);
  ctx_count_launches(c, 4);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx_set_error(c, cudaGetErrorString(e));
    return NS_ERR_CUDA;
  }
  return ctx_sync_main(c);
}
