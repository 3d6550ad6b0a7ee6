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
// The device term is s_k = sum_{r,u} c_ru G_ru - sum_r wb_r I_r with c_ru = gA[slot] + wb_r V_u
// over free rows r and free columns u, wb_r = gb[row r]. Its gradient needs second derivatives
// of the currents; they come in three pieces:
//  * channel: I_d = -I_s = p m Ids(vgs, vds, vbs), so its part of s_k is m (g . w) - p m omega Ids
//    with g = dIds/d(vgs, vds, vbs), w the mode-frame weights and omega = wb_d - wb_s. Its
//    gradient needs only the Hessian-vector product H w and the L-derivatives of g and Ids: one
//    forward pass of the hand-derived channel code (eec_model.cuh) in 2-direction tangent
//    arithmetic (direction w in (vgs, vds, vbs), direction L);
//  * junctions: Ij(v), gj(v) and dgj/dv in closed form;
//  * W: the channel current is proportional to W (through U0 Cox W / L only) and the junction
//    currents minus their GMIN part are proportional to W, so d/dW is exact division by W.
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

// Value plus K forward-mode tangents.
template <int K>
struct Tan {
  double v;
  double d[K];
  __device__ __forceinline__ Tan() : v(0.0) {
#pragma unroll
    for (int i = 0; i < K; ++i) d[i] = 0.0;
  }
  __device__ __forceinline__ Tan(double c) : v(c) {  // NOLINT: constants convert implicitly
#pragma unroll
    for (int i = 0; i < K; ++i) d[i] = 0.0;
  }
};

template <int K>
__device__ __forceinline__ double sval(const Tan<K>& a) { return a.v; }

template <int K>
__device__ __forceinline__ Tan<K> operator+(const Tan<K>& a, const Tan<K>& b) {
  Tan<K> r; r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int K>
__device__ __forceinline__ Tan<K> operator-(const Tan<K>& a, const Tan<K>& b) {
  Tan<K> r; r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int K>
__device__ __forceinline__ Tan<K> operator-(const Tan<K>& a) {
  Tan<K> r; r.v = -a.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int K>
__device__ __forceinline__ Tan<K> operator*(const Tan<K>& a, const Tan<K>& b) {
  Tan<K> r; r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = fma(a.d[i], b.v, a.v * b.d[i]);
  return r;
}
template <int K>
__device__ __forceinline__ Tan<K> operator+(const Tan<K>& a, double b) { Tan<K> r = a; r.v += b; return r; }
template <int K>
__device__ __forceinline__ Tan<K> operator+(double a, const Tan<K>& b) { Tan<K> r = b; r.v += a; return r; }
template <int K>
__device__ __forceinline__ Tan<K> operator-(const Tan<K>& a, double b) { Tan<K> r = a; r.v -= b; return r; }
template <int K>
__device__ __forceinline__ Tan<K> operator-(double a, const Tan<K>& b) { return -(b - a); }
template <int K>
__device__ __forceinline__ Tan<K> operator*(const Tan<K>& a, double b) {
  Tan<K> r; r.v = a.v * b;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * b;
  return r;
}
template <int K>
__device__ __forceinline__ Tan<K> operator*(double a, const Tan<K>& b) { return b * a; }

// d(1/a) = -da / a^2
template <int K>
__device__ __forceinline__ Tan<K> rcp(const Tan<K>& a) {
  Tan<K> r; r.v = fm_rcp(a.v);
  const double m = -r.v * r.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = m * a.d[i];
  return r;
}
// d(a^-1/2) = -a^-3/2 da / 2
template <int K>
__device__ __forceinline__ Tan<K> rsqrt_(const Tan<K>& a) {
  Tan<K> r; r.v = fm_rsqrt(a.v);
  const double m = -0.5 * r.v * r.v * r.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = m * a.d[i];
  return r;
}
template <int K>
__device__ __forceinline__ Tan<K> exp_(const Tan<K>& a) {
  Tan<K> r; r.v = fm_exp(a.v);
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = r.v * a.d[i];
  return r;
}
// log(1 + a) for a in [0, 1], given inv_y = 1 / (1 + a)
template <int K>
__device__ __forceinline__ Tan<K> log1p_(const Tan<K>& a, const Tan<K>& inv_y) {
  Tan<K> r; r.v = fm_log1p01(a.v, inv_y.v);
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = inv_y.v * a.d[i];
  return r;
}

using T2 = Tan<2>;

// Junction pieces without the GMIN leak: IjI = Isat (explim(z) - 1), gjI = dIjI/dv, and
// gj2 = d^2 IjI / dv^2 (zero on the linear continuation above z = 40).
__device__ __forceinline__ void junction2(const CardK& c, double Isat, double v, double& IjI,
                                          double& gjI, double& gj2) {
  const double z = v * c.inv_Vt;
  const bool over = z > 40.0;
  const double zc = over ? 40.0 : z;
  const double em1 = fm_expm1(zc);
  const double ez = em1 + 1.0;
  IjI = Isat * (em1 + ez * (over ? z - 40.0 : 0.0));
  gjI = Isat * c.inv_Vt * ez;
  gj2 = over ? 0.0 : gjI * c.inv_Vt;
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
  double V[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) V[t] = idx[t] >= 0 ? __ldg(x + idx[t]) : __ldg(T.vfix + ~idx[t]);
  const int meta = __ldg(T.meta + k);
  const CardK& c = T.cards[meta >> 2];
  // the polarity (p = +1 NMOS, -1 PMOS) and the mode sign m enter as sign-bit flips on the
  // integer pipe, not as multiplications on the FP64 pipe
  const unsigned long long psb = (meta & 1) ? kSignBit : 0ull;
  const bool sbf = (meta >> 1) & 1;   // source and body source-held
  const double W = __ldg(T.W + k), L = __ldg(T.L + k);

  // weights: wb by terminal (rows d, s, b), cw[t][u] = gA[slot] + wb_t V_u over free (t, u)
  const int term[3] = {0, 2, 3};
  double wb[4] = {0.0, 0.0, 0.0, 0.0};
  double cw[4][4];
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int u = 0; u < 4; ++u) cw[t][u] = 0.0;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int t = term[r];
    if (idx[t] < 0) continue;
    wb[t] = __ldg(gb + idx[t]);
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (idx[u] >= 0) cw[t][u] = fma(wb[t], V[u], __ldg(gA + __ldg(T.slot + (4 * r + u) * N + k)));
  }

  // (1) mode frame
  const bool fwd = fm_ge0(flip(V[0] - V[2], psb));
  const int iD = fwd ? 0 : 2, iS = fwd ? 2 : 0;
  const unsigned long long msb = fwd ? 0ull : kSignBit;   // m = +1 forward, -1 reverse
  const double vgs = flip(V[1] - V[iS], psb), vds = flip(V[iD] - V[iS], psb);
  const double vbs = flip(V[3] - V[iS], psb);

  // channel: s_ch = m (g . w) - p m omega Ids with w in mode-frame coordinates
  double wt[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) wt[u] = cw[0][u] - cw[2][u];
  const double omega = wb[0] - wb[2];
  const double w0 = wt[1] - wt[iS], w1 = wt[iD] - wt[iS], w2 = wt[3] - wt[iS];
  // the channel's per-device constants with their L tangents: beta0 ~ W/L, cE ~ L,
  // 1/cE ~ 1/L, lamL ~ 1/L, so d/dL is (+-1/L) times the stored value
  const double* pr = T.prm + k;
  const double iL = fm_rcp(L);
  PrmS<T2> P;
  const double b0 = __ldg(pr + P_BETA0 * N), cE = __ldg(pr + P_CE * N);
  const double icE = __ldg(pr + P_INV_CE * N), lamL = __ldg(pr + P_LAML * N);
  P.beta0 = T2(b0);
  P.beta0.d[1] = -b0 * iL;
  P.cE = T2(cE);
  P.cE.d[1] = cE * iL;
  P.inv_cE = T2(icE);
  P.inv_cE.d[1] = -icE * iL;
  P.lamL = T2(lamL);
  P.lamL.d[1] = -lamL * iL;
  T2 vgs2(vgs), vds2(vds), vbs2(vbs);
  vgs2.d[0] = w0;
  vds2.d[0] = w1;
  vbs2.d[0] = w2;
  // In forward mode a device with source and body held has no free column at s or b: w2 = 0,
  // and the body-effect terms are the constants stored for the forward (no tangent), nor is
  // the vbs chain of the channel needed.
  const bool hoist = sbf && fwd;
  T2 sqs, Vthb, dVth, Ab, dAb;
  if (hoist) {
    const double* q0 = T.bodyk + k;
    sqs = T2(__ldg(q0));
    Vthb = T2(__ldg(q0 + N));
    dVth = T2(__ldg(q0 + 2 * N));
    Ab = T2(__ldg(q0 + 3 * N));
    dAb = T2(__ldg(q0 + 4 * N));
  } else {
    body_terms<T2>(c, vbs2, sqs, Vthb, dVth, Ab, dAb);
  }
  Chan<T2> ch;
  channel<T2>(c, P, vgs2, vds2, Vthb, dVth, Ab, dAb, ch, !hoist);
  const double gm = ch.gm.v, gds = ch.gds.v, gmb = ch.gmb.v, Ids = ch.Ids.v;
  const double pmw = flip(omega, psb ^ msb);       // p m omega
  const double s_ch = flip(gm * w0 + gds * w1 + gmb * w2, msb) - pmw * Ids;
  const double dv0 = flip(ch.gm.d[0], msb) - pmw * gm;    // d s_ch / d vgs (H w is symmetric in w)
  const double dv1 = flip(ch.gds.d[0], msb) - pmw * gds;  // d s_ch / d vds
  const double dv2 = flip(ch.gmb.d[0], msb) - pmw * gmb;  // d s_ch / d vbs
  const double dL =
      flip(ch.gm.d[1] * w0 + ch.gds.d[1] * w1 + ch.gmb.d[1] * w2, msb) - pmw * ch.Ids.d[1];
  double g[4];
  g[1] = flip(dv0, psb);
  g[3] = flip(dv2, psb);
  g[iD] = flip(dv1, psb);
  g[iS] = flip(dv0 + dv1 + dv2, psb ^ kSignBit);

  // junctions (physical d-b and s-b): s_j = kappa gj - rho Ij
  const double Isat = __ldg(pr + P_ISAT * N);
  double IjdI, gjdI, gjd2, IjsI = 0.0, gjsI = 0.0, gjs2 = 0.0;
  const double vbd = flip(V[3] - V[0], psb), vbsj = flip(V[3] - V[2], psb);
  junction2(c, Isat, vbd, IjdI, gjdI, gjd2);
  // with source and body held the source junction carries no weight (rows and columns s, b
  // are not stamped): its terms below are multiplied by zero
  if (!sbf) junction2(c, Isat, vbsj, IjsI, gjsI, gjs2);
  const double gjd = gjdI + c.GMIN, gjs = gjsI + c.GMIN;
  const double kd = cw[0][0] - cw[0][3] - cw[3][0] + cw[3][3];
  const double rd = flip(wb[3] - wb[0], psb);
  const double ddv = flip(kd * gjd2 - rd * gjd, psb);   // p (kd gjd2 - rd gjd)
  g[0] -= ddv;
  g[3] += ddv;
  const double ks = cw[2][2] - cw[2][3] - cw[3][2] + cw[3][3];
  const double rs = flip(wb[3] - wb[2], psb);
  const double dsv = flip(ks * gjs2 - rs * gjs, psb);
  g[2] -= dsv;
  g[3] += dsv;
  // at fixed L the channel terms and the junctions' saturation terms are proportional to W (the
  // GMIN parts, which are not, are left out of the sums above): d s / dW = s / W
  const double dW = (s_ch + kd * gjdI - rd * IjdI + ks * gjsI - rs * IjsI) * fm_rcp(W);

  // direct term d(sum_r wb_r G_ru V_u)/dV_u = sum_r wb_r G_ru
  const double gsum = gm + gds + gmb;
  const double cd[4] = {fwd ? gds : gsum, fwd ? gm : -gm, fwd ? -gsum : -gds, fwd ? gmb : -gmb};
  const double Gd[4] = {cd[0] + gjd, cd[1], cd[2], cd[3] - gjd};
  const double Gs[4] = {-cd[0], -cd[1], gjs - cd[2], -cd[3] - gjs};
  const double Gb[4] = {-gjd, 0.0, -gjs, gjd + gjs};
#pragma unroll
  for (int u = 0; u < 4; ++u) g[u] += wb[0] * Gd[u] + wb[2] * Gs[u] + wb[3] * Gb[u];

#pragma unroll
  for (int t = 0; t < 4; ++t) T.gv[t * N + k] = g[t];
  const int od = __ldg(T.orig + k);
  gW[od] = dW;
  gL[od] = dL;
}

// gx[u] = sum of the terminal gradients at unknown u: one thread per light unknown (summed in
// original-device order), one warp per heavy unknown (lane-strided, fixed butterfly reduction).
constexpr int kGatherBlock = 256;

__global__ void __launch_bounds__(kGatherBlock) k_bwd_gather(DevTopo T, double* __restrict__ gx,
                                                             int nbl) {
  if ((int)blockIdx.x < nbl) {
    const int i = blockIdx.x * kGatherBlock + threadIdx.x;
    if (i >= T.n_inc_light) return;
    const int u = __ldg(T.inc_light + i);
    double s = 0.0;
    const int p1 = __ldg(T.inc_ptr + u + 1);
    for (int p = __ldg(T.inc_ptr + u); p < p1; ++p) s += __ldg(T.gv + __ldg(T.inc_src + p));
    gx[u] = s;
    return;
  }
  const int w = (blockIdx.x - nbl) * (kGatherBlock / 32) + (threadIdx.x >> 5);
  if (w >= T.n_inc_heavy) return;
  const int lane = threadIdx.x & 31;
  const int u = __ldg(T.inc_heavy + w);
  const int p1 = __ldg(T.inc_ptr + u + 1);
  double s = 0.0;
  for (int p = __ldg(T.inc_ptr + u) + lane; p < p1; p += 32) s += __ldg(T.gv + __ldg(T.inc_src + p));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) gx[u] = s;
}

cudaError_t launch_bwd_gather(const DevTopo& T, double* gx, cudaStream_t s) {
  const int nbl = (T.n_inc_light + kGatherBlock - 1) / kGatherBlock;
  const int nbh = (T.n_inc_heavy + kGatherBlock / 32 - 1) / (kGatherBlock / 32);
  if (nbl + nbh == 0) return cudaSuccess;
  k_bwd_gather<<<nbl + nbh, kGatherBlock, 0, s>>>(T, gx, nbl);
  return cudaGetLastError();
}

// Device address of g_noalloc_gv on the current device, looked up once per device and cached; no
// allocation. The lookup loads this file's module on that device (under lazy module loading the
// module, and with it the array, would otherwise appear at the first backward launch).
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

cudaError_t noalloc_setup() {
  double* ptr = nullptr;
  return noalloc_scratch(&ptr);
}

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
  return launch_bwd_gather(Ts, gx, s);
}

cudaError_t launch_bwd(const DevTopo& T, const double* x, const double* gA, const double* gb,
                       double* gx, double* gW, double* gL, int block, cudaStream_t s) {
  (void)block;
  if (T.N > 0) {
    k_bwd_device<<<(T.N + kBwdBlock - 1) / kBwdBlock, kBwdBlock, 0, s>>>(T, x, gA, gb, gW, gL);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_bwd_gather(T, gx, s);
}

}  // namespace eec
