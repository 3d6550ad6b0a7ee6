// Backward (adjoint) of eval_stamp: gradients of s = <gA, A(x, W, L)> + <gb, b(x, W, L)> with
// respect to the node voltages and every device's W and L.
//
// A and b are sums of per-device contributions (Sec. II (ii)), so s is a sum of per-device
// terms and its gradient is a pure gather: pass 1 (one thread per device) reads gA at the
// device's slots and gb at its rows and differentiates its own term with respect to its four
// terminal voltages and W, L; pass 2 (one thread per unknown) sums the terminal gradients of the
// devices attached to that node (the transpose of the stamp scatter). No two threads write the
// same location, so neither colours nor atomics are needed.
//
// The device term needs derivatives of the Jacobian G (second derivatives of the currents).
// They come from running the same hand-derived model (eec_model.cuh) in forward-mode tangent
// arithmetic with six directions (Vd, Vg, Vs, Vb, W, L).
#include <cuda_runtime.h>

#include <map>
#include <mutex>

#include "eec_model.cuh"

namespace eec {

namespace {

// Fixed scratch of eec_eval_stamp_bwd_noalloc: four terminal gradients per device for up to
// EEC_NOALLOC_MAX_DEV devices (16 MiB on every GPU that loads the library). Host code must not
// use this name as an address; noalloc_scratch() resolves the device address.
static __device__ __align__(256) double g_noalloc_gv[4 * (size_t)EEC_NOALLOC_MAX_DEV];

constexpr int kT = 6;

struct T6 {
  double v;
  double d[kT];
  __device__ __forceinline__ T6() : v(0.0) {
#pragma unroll
    for (int i = 0; i < kT; ++i) d[i] = 0.0;
  }
  __device__ __forceinline__ T6(double c) : v(c) {  // NOLINT: constants convert implicitly
#pragma unroll
    for (int i = 0; i < kT; ++i) d[i] = 0.0;
  }
};

__device__ __forceinline__ double sval(const T6& a) { return a.v; }

__device__ __forceinline__ T6 operator+(const T6& a, const T6& b) {
  T6 r; r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < kT; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
__device__ __forceinline__ T6 operator-(const T6& a, const T6& b) {
  T6 r; r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < kT; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
__device__ __forceinline__ T6 operator-(const T6& a) {
  T6 r; r.v = -a.v;
#pragma unroll
  for (int i = 0; i < kT; ++i) r.d[i] = -a.d[i];
  return r;
}
__device__ __forceinline__ T6 operator*(const T6& a, const T6& b) {
  T6 r; r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < kT; ++i) r.d[i] = fma(a.d[i], b.v, a.v * b.d[i]);
  return r;
}
__device__ __forceinline__ T6 operator+(const T6& a, double b) { T6 r = a; r.v += b; return r; }
__device__ __forceinline__ T6 operator+(double a, const T6& b) { T6 r = b; r.v += a; return r; }
__device__ __forceinline__ T6 operator-(const T6& a, double b) { T6 r = a; r.v -= b; return r; }
__device__ __forceinline__ T6 operator-(double a, const T6& b) { return -(b - a); }
__device__ __forceinline__ T6 operator*(const T6& a, double b) {
  T6 r; r.v = a.v * b;
#pragma unroll
  for (int i = 0; i < kT; ++i) r.d[i] = a.d[i] * b;
  return r;
}
__device__ __forceinline__ T6 operator*(double a, const T6& b) { return b * a; }

// d(1/a) = -da / a^2
__device__ __forceinline__ T6 rcp(const T6& a) {
  T6 r; r.v = 1.0 / a.v;
  const double m = -r.v * r.v;
#pragma unroll
  for (int i = 0; i < kT; ++i) r.d[i] = m * a.d[i];
  return r;
}
// d(a^-1/2) = -a^-3/2 da / 2
__device__ __forceinline__ T6 rsqrt_(const T6& a) {
  T6 r; r.v = ::rsqrt(a.v);
  const double m = -0.5 * r.v * r.v * r.v;
#pragma unroll
  for (int i = 0; i < kT; ++i) r.d[i] = m * a.d[i];
  return r;
}
__device__ __forceinline__ T6 exp_(const T6& a) {
  T6 r; r.v = ::exp(a.v);
#pragma unroll
  for (int i = 0; i < kT; ++i) r.d[i] = r.v * a.d[i];
  return r;
}
__device__ __forceinline__ T6 expm1_(const T6& a) {
  T6 r; r.v = ::expm1(a.v);
  const double e = r.v + 1.0;
#pragma unroll
  for (int i = 0; i < kT; ++i) r.d[i] = e * a.d[i];
  return r;
}
__device__ __forceinline__ T6 log1p_(const T6& a) {
  T6 r; r.v = ::log1p(a.v);
  const double m = 1.0 / (1.0 + a.v);
#pragma unroll
  for (int i = 0; i < kT; ++i) r.d[i] = m * a.d[i];
  return r;
}

constexpr int kBwdBlock = 128;

__global__ void __launch_bounds__(kBwdBlock) k_bwd_device(DevTopo T, const double* __restrict__ x,
                                                          const double* __restrict__ gA,
                                                          const double* __restrict__ gb,
                                                          double* __restrict__ gW,
                                                          double* __restrict__ gL) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= T.N) return;
  const long long N = T.N;
  const int4 ti = __ldg(T.tidx + k);
  const int idx[4] = {ti.x, ti.y, ti.z, ti.w};
  double Vv[4];
  T6 V[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    Vv[t] = idx[t] >= 0 ? __ldg(x + idx[t]) : __ldg(T.vfix + ~idx[t]);
    V[t] = T6(Vv[t]);
    V[t].d[t] = 1.0;
  }
  const int meta = __ldg(T.meta + k);
  const CardK& c = T.cards[meta >> 1];
  const double pp = (meta & 1) ? -1.0 : 1.0;
  T6 W(__ldg(T.W + k)), L(__ldg(T.L + k));
  W.d[4] = 1.0;
  L.d[5] = 1.0;
  const PrmS<T6> P = derive_params<T6>(c, W, L);
  EvalOut<T6> o;
  ees_l1<T6, false>(c, pp, P, V, o);
  double ds[kT];
#pragma unroll
  for (int j = 0; j < kT; ++j) ds[j] = 0.0;
  const int term[3] = {0, 2, 3};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int row = idx[term[r]];
    if (row < 0) continue;
    const double wb = __ldg(gb + row);
#pragma unroll
    for (int j = 0; j < kT; ++j) ds[j] -= wb * o.I[term[r]].d[j];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (idx[u] < 0) continue;
      const int s = __ldg(T.slot + (4 * r + u) * N + k);
      const double wa = __ldg(gA + s);
      const double wv = wa + wb * Vv[u];
#pragma unroll
      for (int j = 0; j < kT; ++j) ds[j] = fma(wv, o.G[r][u].d[j], ds[j]);
      ds[u] = fma(wb, o.G[r][u].v, ds[u]);
    }
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) T.gv[t * N + k] = ds[t];
  const int od = __ldg(T.orig + k);
  gW[od] = ds[4];
  gL[od] = ds[5];
}

__global__ void k_bwd_gather(DevTopo T, double* __restrict__ gx) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= T.n) return;
  double s = 0.0;
  const int p1 = __ldg(T.inc_ptr + u + 1);
  for (int p = __ldg(T.inc_ptr + u); p < p1; ++p) s += __ldg(T.gv + __ldg(T.inc_src + p));
  gx[u] = s;
}

// Device address of g_noalloc_gv on the current device, looked up once per device (set-up on the
// first call there) and cached; no allocation.
cudaError_t noalloc_scratch(double** out) {
  static std::mutex mu;
  static std::map<int, double*> cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it == cache.end()) {
    double* ptr = nullptr;
    e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_gv);
    if (e != cudaSuccess) return e;
    it = cache.emplace(dev, ptr).first;
  }
  *out = it->second;
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_bwd_noalloc(const DevTopo& T, const double* x, const double* gA,
                               const double* gb, double* gx, double* gW, double* gL,
                               cudaStream_t s) {
  if (T.N > EEC_NOALLOC_MAX_DEV) return cudaErrorInvalidValue;
  double* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) return e;
  DevTopo Ts = T;
  Ts.gv = scratch;
  if (Ts.N > 0) {
    k_bwd_device<<<(Ts.N + kBwdBlock - 1) / kBwdBlock, kBwdBlock, 0, s>>>(Ts, x, gA, gb, gW, gL);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (Ts.n > 0) k_bwd_gather<<<(Ts.n + 255) / 256, 256, 0, s>>>(Ts, gx);
  return cudaGetLastError();
}

cudaError_t launch_bwd(const DevTopo& T, const double* x, const double* gA, const double* gb,
                       double* gx, double* gW, double* gL, int block, cudaStream_t s) {
  (void)block;
  if (T.N > 0) {
    k_bwd_device<<<(T.N + kBwdBlock - 1) / kBwdBlock, kBwdBlock, 0, s>>>(T, x, gA, gb, gW, gL);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (T.n > 0) k_bwd_gather<<<(T.n + 255) / 256, 256, 0, s>>>(T, gx);
  return cudaGetLastError();
}

}  // namespace eec
