// Evaluate-and-stamp kernels (sm_103a).
//
// Sec. II (i)/(ii): per Newton iteration every device is evaluated at the present bias and its
// contributions are accumulated into A and b. Sec. I / Sec. II: devices of one colour share no
// non-ground node, so their stamps touch disjoint rows and may be plain store-adds; colours run
// one after another. Schedules (Table I analogues):
//   MODE_RMW    one fused evaluate + store-add per device; one launch per colour ("ColorFused")
//               or one persistent launch with a grid barrier between colours ("Color", single
//               parallel region);
//   MODE_ATOMIC uncoloured, FP64 atomicAdd (the lock-based stamping the paper avoids, in its
//               GPU form);
//   MODE_BUFFER evaluate into a per-device buffer ("loadomp"/"Color" buffer), then a stamp of
//               the buffer in colour order;
//   MODE_SORTED evaluate into a contribution buffer laid out by entry (windows of entries sorted
//               by their contribution count), then the per-entry gather of eec_gather.cu
//               (segmented reduction, deterministic, no colours).
// The evaluation is FP64-pipe bound on GB300 (FP64 issues at about 1/64 of the FP32 rate), so
// the kernels aim at a saturated FP64 pipe: one device per thread, few warps per SM suffice;
// parameters are precomputed per device so that no division on W or L is repeated per call.
#include <cuda_runtime.h>

#include <algorithm>

#include "eec_model.cuh"

namespace eec {

namespace {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr unsigned long long kBarrierLimitNs = 1000000000ull;  // 1 s

// Grid-wide barrier for a co-resident (cooperative) grid. bar[0] counts arrivals, bar[1] is the
// generation, bar[2] is this launch's abort word (zeroed with bar[0..1] before every launch).
// Every wait is bounded: after kBarrierLimitNs the waiting block records kStatusTimeout in the
// status word (sticky until the host reads it) and sets the abort word, and every block of the
// grid returns false at its next wait. Waits test only the abort word, so a timeout recorded by
// an earlier launch does not make a later launch give up.
__device__ __forceinline__ bool grid_sync(unsigned* bar, int* status, int absent_block) {
  __shared__ int fail;
  __syncthreads();
  if (absent_block == (int)blockIdx.x) return true;  // test hook: this block never arrives
  if (threadIdx.x == 0) {
    fail = 0;
    const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
    const unsigned gen = ld_acquire_u32(bar + 1);
    __threadfence();
    const unsigned prev = atomicAdd(bar, 1u);
    if (prev == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (ld_acquire_u32(bar + 1) == gen) {
        if (*((volatile unsigned*)(bar + 2))) { fail = 1; break; }
        if (global_ns() - t0 > kBarrierLimitNs) {
          atomicOr(status, kStatusTimeout);
          atomicExch(bar + 2, 1u);
          fail = 1;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return fail == 0;
}

__device__ __forceinline__ PrmS<double> load_prm(const DevTopo& T, int k) {
  const double* p = T.prm;
  const long long N = T.N;
  PrmS<double> P;
  P.beta0 = __ldg(p + P_BETA0 * N + k);
  P.cE = __ldg(p + P_CE * N + k);
  P.inv_cE = __ldg(p + P_INV_CE * N + k);
  P.lamL = __ldg(p + P_LAML * N + k);
  P.Isat = __ldg(p + P_ISAT * N + k);
  P.Coxt = __ldg(p + P_COXT * N + k);
  P.CovS = __ldg(p + P_COVS * N + k);
  P.CovD = __ldg(p + P_COVD * N + k);
  P.IsatVt = __ldg(p + P_ISATVT * N + k);
  P.IsatVtG = __ldg(p + P_ISATVTG * N + k);
  return P;
}

// Device k's terminal unknowns and voltages, its per-device constants and the model at that bias
// (WANT_C: with the charge Jacobian of the transient stamp).
template <bool WANT_Q, bool WANT_C>
__device__ __forceinline__ void eval_model(const DevTopo& T, int k, const double* __restrict__ x,
                                           int idx[4], double V[4], EvalOut<double>& o) {
  const long long N = T.N;
  const int4 ti = __ldg(T.tidx + k);
  idx[0] = ti.x;
  idx[1] = ti.y;
  idx[2] = ti.z;
  idx[3] = ti.w;
#pragma unroll
  for (int t = 0; t < 4; ++t)
    V[t] = idx[t] >= 0 ? __ldg(x + idx[t]) : __ldg(T.vfix + ~idx[t]);
  const int meta = __ldg(T.meta + k);
  const CardK& c = T.cards[meta >> 2];
  const unsigned long long psb = (meta & 1) ? kSignBit : 0ull;
  const bool sbf = (meta >> 1) & 1;
  const PrmS<double> P = load_prm(T, k);
  BodyK bk;
  if (sbf) {
    const double* q0 = T.bodyk + k;
    bk.sqs = __ldg(q0);
    bk.Vthb = __ldg(q0 + N);
    bk.dVth_dvbs = __ldg(q0 + 2 * N);
    bk.Ab = __ldg(q0 + 3 * N);
    bk.dAb_dvbs = __ldg(q0 + 4 * N);
    bk.Ijs = __ldg(q0 + 5 * N);
    bk.gjs = __ldg(q0 + 6 * N);
    bk.Qb = __ldg(q0 + 7 * N);
  }
  ees_l1<double, WANT_Q, WANT_C>(c, psb, P, V, o, sbf, &bk);
}

// Evaluate device at layout position k and stamp (MODE_RMW / MODE_ATOMIC) or buffer it.
template <int MODE, bool WANT_Q>
__device__ __forceinline__ void eval_one(const DevTopo& T, int k, const double* __restrict__ x,
                                         double* A, double* b, double* __restrict__ q,
                                         int dbg) {
  const long long N = T.N;
  int idx[4];
  double V[4];
  EvalOut<double> o;
  eval_model<WANT_Q, false>(T, k, x, idx, V, o);

  // A and b may still be being initialised by the kernel launched just before this one
  // (programmatic dependent launch): wait for it before the first addition
  if (MODE == MODE_RMW || MODE == MODE_ATOMIC) asm volatile("griddepcontrol.wait;" ::: "memory");
  // b row r: -I_r + sum over the free columns u of G[r][u] V_u (held columns are eliminated)
  const int term[3] = {0, 2, 3};
  bool bc_ok = true;
  if (MODE == MODE_SORTED) {
    // the same contributions as MODE_BUFFER, each written to its item in the gather's buffer
    // (gat_pos: the entry's items, in original device order)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (idx[term[r]] < 0) continue;
      double s = -i_entry(o, term[r]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (idx[u] < 0) continue;
        const double g = g_entry(o, r, u);
        s = fma(g, V[u], s);
        T.cbuf[__ldg(T.gat_pos + (4 * r + u) * N + k)] = g;
        if (dbg) bc_ok = bc_ok && isfinite(g);
      }
      T.cbuf[__ldg(T.gat_pos + (kNSlot + r) * N + k)] = s;
      if (dbg) bc_ok = bc_ok && isfinite(s);   // FP64 compares: debug checks only
    }
  } else if (MODE == MODE_BUFFER) {
    // only what a stamp reads is buffered: rows of free terminals, and in them the entries of
    // free columns (the gather and the colour-ordered stamps skip held rows and columns)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if (idx[term[r]] < 0) continue;
      double s = -i_entry(o, term[r]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (idx[u] < 0) continue;
        const double g = g_entry(o, r, u);
        s = fma(g, V[u], s);
        T.buf[(4 * r + u) * N + k] = g;
        if (dbg) bc_ok = bc_ok && isfinite(g);
      }
      T.buf[(kNSlot + r) * N + k] = s;
      if (dbg) bc_ok = bc_ok && isfinite(s);   // FP64 compares: debug checks only
    }
  } else {
    // rows of source-held terminals are not stamped: their entries are not formed
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int row = idx[term[r]];
      if (row < 0) continue;
      double s = -i_entry(o, term[r]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (idx[u] < 0) continue;
        const double g = g_entry(o, r, u);
        s = fma(g, V[u], s);
        const int sl = __ldg(T.slot + (4 * r + u) * N + k);
        if (MODE == MODE_ATOMIC) atomicAdd(A + sl, g);
        else A[sl] += g;
        if (dbg) bc_ok = bc_ok && isfinite(g);
      }
      if (MODE == MODE_ATOMIC) atomicAdd(b + row, s);
      else b[row] += s;
      if (dbg) bc_ok = bc_ok && isfinite(s);   // FP64 compares: debug checks only
    }
  }
  if (WANT_Q) {
    const int od = __ldg(T.orig + k);
#pragma unroll
    for (int t = 0; t < 4; ++t) q[t * N + od] = o.Q[t];
  }
  if (dbg && !bc_ok) atomicOr(T.status, kStatusNumeric);   // a formed entry is not finite
}

// Transient: evaluate with charges and their Jacobian, then stamp all four terminal rows
// (A += G + alpha C, b += -I - ic + (G + alpha C) V) by store-add (one colour) or atomics.
template <int MODE>
__device__ __forceinline__ void eval_one_tran(const DevTopo& T, int k, const double* __restrict__ x,
                                              double* A, double* b, const TranArgs& ta) {
  const long long N = T.N;
  int idx[4];
  double V[4];
  EvalOut<double> o;
  eval_model<true, true>(T, k, x, idx, V, o);
  if (MODE != MODE_BUFFER) asm volatile("griddepcontrol.wait;" ::: "memory");   // see eval_one
  const int od = __ldg(T.orig + k);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const long long at = t * N + od;
    const double ic = ta.alpha * (o.Q[t] - __ldg(ta.qprev + at)) -
                      (ta.iprev ? ta.beta * __ldg(ta.iprev + at) : 0.0);
    ta.q[at] = o.Q[t];
    if (ta.icap) ta.icap[at] = ic;
    const int row = idx[t];
    if (row < 0) continue;
    const int r = t == 0 ? 0 : (t == 2 ? 1 : 2);   // row of G (gate row of G is zero)
    double rhs = -i_entry(o, t) - ic;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (idx[u] < 0) continue;   // entries of held columns are not formed
      const double a = fma(ta.alpha, c_entry(o, t, u), t == 1 ? 0.0 : g_entry(o, r, u));
      if (MODE == MODE_BUFFER) {
        T.buf_tran[(4 * t + u) * N + k] = a;
      } else {
        const int s = t == 1 ? __ldg(T.slot_g + u * N + k) : __ldg(T.slot + (4 * r + u) * N + k);
        if (MODE == MODE_ATOMIC) atomicAdd(A + s, a);
        else A[s] += a;
      }
      rhs = fma(a, V[u], rhs);
    }
    if (MODE == MODE_BUFFER) T.buf_tran[(16 + t) * N + k] = rhs;
    else if (MODE == MODE_ATOMIC) atomicAdd(b + row, rhs);
    else b[row] += rhs;
  }
}

constexpr int kEvalBlock = 128;

template <int MODE>
__global__ void __launch_bounds__(kEvalBlock) k_eval_tran(DevTopo T, int begin, int end,
                                                          const double* __restrict__ x,
                                                          double* A, double* b, TranArgs ta) {
  for (int k = begin + blockIdx.x * blockDim.x + threadIdx.x; k < end;
       k += gridDim.x * blockDim.x)
    eval_one_tran<MODE>(T, k, x, A, b, ta);
}

template <int MODE, bool WANT_Q>
__global__ void __launch_bounds__(kEvalBlock) k_eval(DevTopo T, int begin, int end,
                                                     const double* __restrict__ x, double* A,
                                                     double* b, double* q, int dbg) {
  for (int k = begin + blockIdx.x * blockDim.x + threadIdx.x; k < end;
       k += gridDim.x * blockDim.x)
    eval_one<MODE, WANT_Q>(T, k, x, A, b, q, dbg);
}

// Thread j takes the j-th device of a list of library-order ranges (roff: prefix sums of the
// range lengths). Used where a launch must cover a contiguous span of original device indices,
// which the colour-major layout splits into one range per run of increasing original index.
template <int MODE, bool WANT_Q>
__global__ void __launch_bounds__(kEvalBlock) k_eval_ranges(DevTopo T, const int* __restrict__ rbeg,
                                                            const int* __restrict__ roff, int nr,
                                                            int total, const double* __restrict__ x,
                                                            double* A, double* b, double* q,
                                                            int dbg) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= total) return;
  int lo = 0, hi = nr;  // roff[lo] <= j < roff[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(roff + mid) <= j) lo = mid;
    else hi = mid;
  }
  eval_one<MODE, WANT_Q>(T, __ldg(rbeg + lo) + (j - __ldg(roff + lo)), x, A, b, q, dbg);
}

// One co-resident grid walks the colours; a colour's devices are dealt out in 32-device chunks
// round-robin over the blocks first (chunk i -> block i mod grid, then the next warp of that
// block), so a small colour occupies one warp on each of many SMs instead of whole blocks on a
// few. The FP64 pipe of an SM is narrow; spreading the warps is what shortens a colour. One
// 512-thread block per SM: the same 16 warps per SM as four 128-thread blocks, and a quarter of
// the arrivals at every grid barrier.
constexpr int kPersistBlock = 512;
template <bool WANT_Q>
__global__ void __launch_bounds__(kPersistBlock) k_persistent(DevTopo T, const int* __restrict__ coff,
                                                           int C, const double* __restrict__ x,
                                                           double* A, double* b, double* q,
                                                           int dbg, int absent_block) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  for (int c = 0; c < C; ++c) {
    const int begin = __ldg(coff + c), end = __ldg(coff + c + 1);
    const int nch = (end - begin + 31) >> 5;
    for (int ch = blockIdx.x + gridDim.x * warp; ch < nch; ch += gridDim.x * wpb) {
      const int k = begin + (ch << 5) + lane;
      if (k < end) eval_one<MODE_RMW, WANT_Q>(T, k, x, A, b, q, dbg);
    }
    if (c + 1 < C && !grid_sync(T.bar, T.status, absent_block)) return;
  }
}

__global__ void k_params(DevTopo T, const double* __restrict__ Wo, const double* __restrict__ Lo) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= T.N) return;
  if (Wo) {  // new sizes in original device order
    const int od = T.orig[k];
    T.W[k] = Wo[od];
    T.L[k] = Lo[od];
  }
  const int meta = T.meta[k];
  const CardK& c = T.cards[meta >> 2];
  const PrmS<double> P = derive_params<double>(c, T.W[k], T.L[k]);
  const long long N = T.N;
  if ((meta >> 1) & 1) {  // source and body source-held: hoist the x-independent terms
    const int4 ti = T.tidx[k];
    const unsigned long long psb = (meta & 1) ? kSignBit : 0ull;
    const double vbs = flip(T.vfix[~ti.w] - T.vfix[~ti.z], psb);
    double sqs, Vthb, dVth, Ab, dAb, Ijs, gjs;
    body_terms<double>(c, vbs, sqs, Vthb, dVth, Ab, dAb);
    junction<double>(c, P, vbs, Ijs, gjs);
    double* q0 = T.bodyk + k;
    q0[0] = sqs;
    q0[N] = Vthb;
    q0[2 * N] = dVth;
    q0[3 * N] = Ab;
    q0[4 * N] = dAb;
    q0[5 * N] = Ijs;
    q0[6 * N] = gjs;
    q0[7 * N] = -(P.Coxt * c.K1 * sqs);
  }
  T.prm[P_BETA0 * N + k] = P.beta0;
  T.prm[P_CE * N + k] = P.cE;
  T.prm[P_INV_CE * N + k] = P.inv_cE;
  T.prm[P_LAML * N + k] = P.lamL;
  T.prm[P_ISAT * N + k] = P.Isat;
  T.prm[P_COXT * N + k] = P.Coxt;
  T.prm[P_COVS * N + k] = P.CovS;
  T.prm[P_COVD * N + k] = P.CovD;
  T.prm[P_ISATVT * N + k] = P.IsatVt;
  T.prm[P_ISATVTG * N + k] = P.IsatVtG;
}

// One colour's stamp from the buffer (positions begin..end-1 share no row).
// Add device k's buffered contributions to A and b. Callers stamp one colour at a time, so no
// other thread adds to the same entries meanwhile; the additions are fire-and-forget atomics
// performed in L2 (no load of A into the SM), which give the same sums in the same order as a
// read-modify-write.
__device__ __forceinline__ void stamp_buffered(const DevTopo& T, int k, double* A, double* b) {
  const long long N = T.N;
  const int4 ti = __ldg(T.tidx + k);
  const int rows[3] = {ti.x, ti.z, ti.w};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    if (rows[r] < 0) continue;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int s = __ldg(T.slot + (4 * r + u) * N + k);
      if (s >= 0) atomicAdd(A + s, __ldg(T.buf + (4 * r + u) * N + k));
    }
    atomicAdd(b + rows[r], __ldg(T.buf + (kNSlot + r) * N + k));
  }
}

__global__ void __launch_bounds__(kEvalBlock) k_stamp_buffer(DevTopo T, int begin, int end,
                                                             double* A, double* b) {
  for (int k = begin + blockIdx.x * blockDim.x + threadIdx.x; k < end;
       k += gridDim.x * blockDim.x)
    stamp_buffered(T, k, A, b);
}

// All colours' buffered stamps by one thread-block cluster (kClusterBlocks blocks of
// kClusterThreads threads on as many SMs), colour after colour, with the cluster's hardware
// barrier between colours (release on arrive, acquire on wait; every thread passes it the same
// number of times, so it cannot wait on an absent thread). Between arrive and wait each thread
// loads the read-only data of its first device of the next colour (indices, slots, buffered
// contributions), so that after the barrier only the additions into A and b remain.
constexpr int kClusterBlocks = 8;
constexpr int kClusterThreads = 512;

struct StampPre {
  int rows[3];
  int sl[kNSlot];
  double v[kNContrib];
};

__device__ __forceinline__ void stamp_load(const DevTopo& T, int k, StampPre& p) {
  const long long N = T.N;
  const int4 ti = __ldg(T.tidx + k);
  p.rows[0] = ti.x;
  p.rows[1] = ti.z;
  p.rows[2] = ti.w;
#pragma unroll
  for (int j = 0; j < kNSlot; ++j) p.sl[j] = __ldg(T.slot + j * N + k);
#pragma unroll
  for (int j = 0; j < kNContrib; ++j) p.v[j] = __ldg(T.buf + j * N + k);
}

// The additions are fire-and-forget atomics performed in L2: no load of A on the critical path,
// and the same sum as a read-modify-write (each entry receives one addition per colour, the
// barrier orders the colours, so every entry still adds its contributions in colour order).
__device__ __forceinline__ void stamp_apply(const StampPre& p, double* A, double* b) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    if (p.rows[r] < 0) continue;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int s = p.sl[4 * r + u];
      if (s >= 0) atomicAdd(A + s, p.v[4 * r + u]);
    }
    atomicAdd(b + p.rows[r], p.v[kNSlot + r]);
  }
}

__global__ void __launch_bounds__(kClusterThreads) k_stamp_cluster(DevTopo T,
                                                                  const int* __restrict__ coff,
                                                                  int C, double* A, double* b) {
  const int nthreads = gridDim.x * blockDim.x;   // the grid is one cluster
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  StampPre cur;
  bool have = false;
  if (C > 0) {
    const int k = __ldg(coff) + tid;
    have = k < __ldg(coff + 1);
    if (have) stamp_load(T, k, cur);
  }
  for (int c = 0; c < C; ++c) {
    const int begin = __ldg(coff + c), end = __ldg(coff + c + 1);
    if (have) stamp_apply(cur, A, b);
    for (int k = begin + tid + nthreads; k < end; k += nthreads) {
      StampPre extra;
      stamp_load(T, k, extra);
      stamp_apply(extra, A, b);
    }
    if (c + 1 < C) {
      __syncwarp();   // the .aligned barrier is executed by whole warps
      asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
      const int k = __ldg(coff + c + 1) + tid;
      have = k < __ldg(coff + c + 2);
      if (have) stamp_load(T, k, cur);   // read-only data: safe before the acquire
      __syncwarp();
      asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
  }
}

// The transient buffer, colour after colour, by one cluster as k_stamp_cluster: four rows per
// device (d, g, s, b; the gate row's slots in slot_g), 16 values and 4 right-hand sides.
constexpr int kClusterThreadsTran = 256;

struct StampPreTran {
  int rows[4];
  int sl[16];
  double v[kNContribTran];
};

__device__ __forceinline__ void stamp_load_tran(const DevTopo& T, int k, StampPreTran& p) {
  const long long N = T.N;
  const int4 ti = __ldg(T.tidx + k);
  p.rows[0] = ti.x;
  p.rows[1] = ti.y;
  p.rows[2] = ti.z;
  p.rows[3] = ti.w;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int r = t == 0 ? 0 : (t == 2 ? 1 : 2);
#pragma unroll
    for (int u = 0; u < 4; ++u)
      p.sl[4 * t + u] = t == 1 ? __ldg(T.slot_g + u * N + k) : __ldg(T.slot + (4 * r + u) * N + k);
  }
#pragma unroll
  for (int j = 0; j < kNContribTran; ++j)
    p.v[j] = (p.rows[j < 16 ? j >> 2 : j - 16] >= 0) ? __ldg(T.buf_tran + j * N + k) : 0.0;
}

__device__ __forceinline__ void stamp_apply_tran(const StampPreTran& p, double* A, double* b) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (p.rows[t] < 0) continue;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int s = p.sl[4 * t + u];
      if (s >= 0) atomicAdd(A + s, p.v[4 * t + u]);
    }
    atomicAdd(b + p.rows[t], p.v[16 + t]);
  }
}

__global__ void __launch_bounds__(kClusterThreadsTran) k_stamp_cluster_tran(
    DevTopo T, const int* __restrict__ coff, int C, double* A, double* b) {
  const int nthreads = gridDim.x * blockDim.x;   // the grid is one cluster
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  StampPreTran cur;
  bool have = false;
  if (C > 0) {
    const int k = __ldg(coff) + tid;
    have = k < __ldg(coff + 1);
    if (have) stamp_load_tran(T, k, cur);
  }
  for (int c = 0; c < C; ++c) {
    const int begin = __ldg(coff + c), end = __ldg(coff + c + 1);
    if (have) stamp_apply_tran(cur, A, b);
    for (int k = begin + tid + nthreads; k < end; k += nthreads) {
      StampPreTran extra;
      stamp_load_tran(T, k, extra);
      stamp_apply_tran(extra, A, b);
    }
    if (c + 1 < C) {
      __syncwarp();   // the .aligned barrier is executed by whole warps
      asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
      const int k = __ldg(coff + c + 1) + tid;
      have = k < __ldg(coff + c + 2);
      if (have) stamp_load_tran(T, k, cur);   // read-only data: safe before the acquire
      __syncwarp();
      asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
  }
}

// All colours' buffered stamps in one co-resident launch: the grid adds colour c, passes the
// bounded grid barrier, then adds colour c + 1 — the order of the per-colour launches, without
// a launch (or graph node) per colour. Stamping a colour is a few read-modify-writes per device,
// so a colour costs about one barrier.
constexpr int kStampBlock = 256;
__global__ void __launch_bounds__(kStampBlock) k_stamp_persistent(DevTopo T,
                                                                  const int* __restrict__ coff,
                                                                  int C, double* A, double* b,
                                                                  int absent_block) {
  for (int c = 0; c < C; ++c) {
    const int begin = __ldg(coff + c), end = __ldg(coff + c + 1);
    for (int k = begin + blockIdx.x * blockDim.x + threadIdx.x; k < end;
         k += gridDim.x * blockDim.x)
      stamp_buffered(T, k, A, b);
    if (c + 1 < C && !grid_sync(T.bar, T.status, absent_block)) return;
  }
}

// ---- Pipelined colour schedule -------------------------------------------------------------
// The colour order of Sec. II (devices of one colour stamp lock-free, colours one after another)
// without a barrier between colours: work items of up to kPipeItem devices of one colour, in
// colour order, are taken from a ticket counter. A block evaluates its item's devices into
// registers, then waits until every item of the previous colour has stamped, stamps, and counts
// its item done for its colour. While colour c stamps, later items are already evaluating, so on
// a netlist with few colours the stamps hide under the evaluation; with many small colours the
// chain of per-colour hand-overs (about a microsecond each) sets the time.
// Deadlock freedom: an item only waits for items of lower ticket, and a ticket is only taken by
// a block that is running and finishes its item without waiting for a higher one. Waits are
// bounded (kBarrierLimitNs): a block that gives up records kStatusTimeout and sets the launch's
// abort word, after which every later wait gives up at once (no stamp is applied after an
// abort: A and b are then incomplete and the call reports EEC_ETIMEOUT through eec_status).
// Within a colour no two devices share a row, so every entry receives at most one device's
// additions per colour; the additions are performed in L2 (no load of A into the SM) and each
// entry sums its contributions in colour order, so the result is deterministic and equals the
// per-colour launches' bitwise.
constexpr int kPipeBlock = kPipeItem;

// One work item per block: the block takes the next ticket, evaluates the item's devices,
// waits until every item of the previous colour has stamped, stamps, counts its item done for
// its colour and leaves (the hardware then starts the next block in its place, so a block holds
// no state across items). Work::eval(k) evaluates device k (before any wait); Work::stamp()
// applies its additions (after the previous colour is complete).
template <class Work>
__device__ __forceinline__ void pipe_item(const DevTopo& T, Work& w, int absent_item) {
  __shared__ int4 s_it;
  __shared__ int s_num, s_go;
  unsigned* st = T.pipe;
  if (threadIdx.x == 0) {
    const int it = (int)atomicAdd(st, 1u);
    s_num = it;
    if (it < T.n_pitem) s_it = __ldg(T.pitem + it);
  }
  __syncthreads();
  const int it = s_num;
  if (it < T.n_pitem) {                               // uniform
    const int4 item = s_it;
    const int k = item.x + (int)threadIdx.x;
    const bool valid = k < item.y;
    if (valid) w.eval(k);
    // A and b are initialised by the kernel launched before this one (programmatic dependent
    // launch): wait for it before the first addition
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (threadIdx.x == 0) {
      int go = 1;
      if (item.w > 0) {
        const unsigned* dp = st + kPipeHdr + item.z - 1;
        const unsigned need = (unsigned)item.w;
        if (ld_acquire_u32(dp) < need) {
          const unsigned long long t0 = global_ns();
          while (ld_acquire_u32(dp) < need) {
            if (*((volatile unsigned*)(st + 2))) { go = 0; break; }
            if (global_ns() - t0 > kBarrierLimitNs) {
              atomicOr(T.status, kStatusTimeout);
              atomicExch(st + 2, 1u);
              go = 0;
              break;
            }
          }
        }
      }
      s_go = go;
    }
    __syncthreads();
    if (s_go && valid) w.stamp();
    __syncthreads();                                   // every thread's additions issued
    if (threadIdx.x == 0 && it != absent_item) {
      __threadfence();                                 // ... and performed before the count
      atomicAdd(st + kPipeHdr + item.z, 1u);
    }
  }
  // the last block to leave zeroes the counters for the next launch: every other block has
  // left, and the next launch in the stream starts after this one has completed
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(st + 1, 1u) == gridDim.x - 1) {
      const int nc = T.n_pitem > 0 ? __ldg(&T.pitem[T.n_pitem - 1].z) + 1 : 0;
      for (int j = 0; j < nc; ++j) st[kPipeHdr + j] = 0u;
      st[0] = 0u;
      st[2] = 0u;
      __threadfence();
      st[1] = 0u;
    }
  }
}

// DC work of one device: currents and conductances at x; rows d, s, b stamped. The item's
// contributions and their target slots wait in shared memory (structure of arrays over the
// block's threads), so that no register is held across the wait for the previous colour and the
// kernel keeps the evaluation kernel's occupancy.
constexpr int kPipeDCStage = kNContrib;       // 12 conductances, 3 right-hand sides
template <bool WANT_Q>
struct PipeDC {
  const DevTopo& T;
  const double* __restrict__ x;
  double* A;
  double* b;
  double* __restrict__ q;
  int dbg;
  double* sv;   // [kPipeDCStage][kPipeBlock] shared: values
  int* si;      // [kPipeDCStage][kPipeBlock] shared: A slot of each value, then b rows (-1: none)

  __device__ __forceinline__ void eval(int k) {
    const long long N = T.N;
    const int tid = threadIdx.x;
    int idx[4];
    double V[4];
    EvalOut<double> o;
    eval_model<WANT_Q, false>(T, k, x, idx, V, o);
    const int term[3] = {0, 2, 3};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int row = idx[term[r]];
      si[(kNSlot + r) * kPipeBlock + tid] = row;
      if (row < 0) continue;   // rows of held terminals are not stamped: nothing to form
      double s = -i_entry(o, term[r]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (idx[u] < 0) {
          si[(4 * r + u) * kPipeBlock + tid] = -1;
          continue;
        }
        const double g = g_entry(o, r, u);
        sv[(4 * r + u) * kPipeBlock + tid] = g;
        si[(4 * r + u) * kPipeBlock + tid] = __ldg(T.slot + (4 * r + u) * N + k);
        s = fma(g, V[u], s);
      }
      sv[(kNSlot + r) * kPipeBlock + tid] = s;
    }
    if (WANT_Q) {
      const int od = __ldg(T.orig + k);
#pragma unroll
      for (int t = 0; t < 4; ++t) q[t * N + od] = o.Q[t];
    }
    if (dbg) {   // non-finite values (debug checks only: the tests cost FP64 issue slots)
      bool ok = true;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        if (idx[term[r]] < 0) continue;
        ok = ok && isfinite(sv[(kNSlot + r) * kPipeBlock + tid]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          ok = ok && (idx[u] < 0 || isfinite(sv[(4 * r + u) * kPipeBlock + tid]));
      }
      if (!ok) atomicOr(T.status, kStatusNumeric);
    }
  }

  __device__ __forceinline__ void stamp() {
    const int tid = threadIdx.x;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int row = si[(kNSlot + r) * kPipeBlock + tid];
      if (row < 0) continue;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int sl = si[(4 * r + u) * kPipeBlock + tid];
        if (sl >= 0) atomicAdd(A + sl, sv[(4 * r + u) * kPipeBlock + tid]);
      }
      atomicAdd(b + row, sv[(kNSlot + r) * kPipeBlock + tid]);
    }
  }
};

// Transient work of one device: G + alpha C on all four rows, -I - ic + (G + alpha C) V, staged
// in shared memory as the DC work.
constexpr int kPipeTranStage = kNContribTran;   // 16 values, 4 right-hand sides
struct PipeTran {
  const DevTopo& T;
  const double* __restrict__ x;
  double* A;
  double* b;
  const TranArgs& ta;
  double* sv;   // [kPipeTranStage][kPipeBlock] shared
  int* si;      // [kPipeTranStage][kPipeBlock] shared

  __device__ __forceinline__ void eval(int k) {
    const long long N = T.N;
    const int tid = threadIdx.x;
    int idx[4];
    double V[4];
    EvalOut<double> o;
    eval_model<true, true>(T, k, x, idx, V, o);
    const int od = __ldg(T.orig + k);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const long long at = t * N + od;
      const double ic = ta.alpha * (o.Q[t] - __ldg(ta.qprev + at)) -
                        (ta.iprev ? ta.beta * __ldg(ta.iprev + at) : 0.0);
      ta.q[at] = o.Q[t];
      if (ta.icap) ta.icap[at] = ic;
      si[(16 + t) * kPipeBlock + tid] = idx[t];
      if (idx[t] < 0) continue;   // rows of held terminals are not stamped
      const int r = t == 0 ? 0 : (t == 2 ? 1 : 2);   // row of G (gate row of G is zero)
      double s = -i_entry(o, t) - ic;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (idx[u] < 0) {   // entries of held columns are not formed
          si[(4 * t + u) * kPipeBlock + tid] = -1;
          continue;
        }
        const double v = fma(ta.alpha, c_entry(o, t, u), t == 1 ? 0.0 : g_entry(o, r, u));
        sv[(4 * t + u) * kPipeBlock + tid] = v;
        si[(4 * t + u) * kPipeBlock + tid] =
            t == 1 ? __ldg(T.slot_g + u * N + k) : __ldg(T.slot + (4 * r + u) * N + k);
        s = fma(v, V[u], s);
      }
      sv[(16 + t) * kPipeBlock + tid] = s;
    }
  }

  __device__ __forceinline__ void stamp() {
    const int tid = threadIdx.x;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int row = si[(16 + t) * kPipeBlock + tid];
      if (row < 0) continue;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int sl = si[(4 * t + u) * kPipeBlock + tid];
        if (sl >= 0) atomicAdd(A + sl, sv[(4 * t + u) * kPipeBlock + tid]);
      }
      atomicAdd(b + row, sv[(16 + t) * kPipeBlock + tid]);
    }
  }
};

template <bool WANT_Q>
__global__ void __launch_bounds__(kPipeBlock, 5) k_color_pipe(DevTopo T, const double* __restrict__ x,
                                                             double* A, double* b, double* q,
                                                             int dbg, int absent_item) {
  __shared__ double sv[kPipeDCStage * kPipeBlock];
  __shared__ int si[kPipeDCStage * kPipeBlock];
  PipeDC<WANT_Q> w{T, x, A, b, q, dbg, sv, si};
  pipe_item(T, w, absent_item);
}

__global__ void __launch_bounds__(kPipeBlock, 4) k_color_pipe_tran(DevTopo T,
                                                                  const double* __restrict__ x,
                                                                  double* A, double* b,
                                                                  TranArgs ta) {
  __shared__ double sv[kPipeTranStage * kPipeBlock];
  __shared__ int si[kPipeTranStage * kPipeBlock];
  PipeTran w{T, x, A, b, ta, sv, si};
  pipe_item(T, w, -1);
}

__global__ void k_dfma(double* out, int iters, double a, double c) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, c); x1 = fma(x1, a, c); x2 = fma(x2, a, c); x3 = fma(x3, a, c);
    x4 = fma(x4, a, c); x5 = fma(x5, a, c); x6 = fma(x6, a, c); x7 = fma(x7, a, c);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void k_math_check(int fn, long long n, const double* __restrict__ x, double* ours,
                             double* ref) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  if (fn == 0) {
    ours[i] = fm_exp(v);
    ref[i] = ::exp(v);
  } else if (fn == 1) {
    ours[i] = fm_expm1(v);
    ref[i] = ::expm1(v);
  } else if (fn == 2) {
    ours[i] = fm_log1p01(v, 1.0 / (1.0 + v));
    ref[i] = ::log1p(v);
  } else if (fn == 3) {
    ours[i] = fm_rcp(v);
    ref[i] = 1.0 / v;
  } else {
    ours[i] = fm_rsqrt(v);
    ref[i] = ::rsqrt(v);
  }
}

int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 0x7fffffffLL) g = 0x7fffffffLL;
  return (int)g;
}

}  // namespace

cudaError_t launch_params(const DevTopo& T, cudaStream_t s) {
  if (T.N == 0) return cudaSuccess;
  k_params<<<grid_for(T.N, 256), 256, 0, s>>>(T, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_update_params(const DevTopo& T, const double* W_dev, const double* L_dev,
                                 cudaStream_t s) {
  if (T.N == 0) return cudaSuccess;
  k_params<<<grid_for(T.N, 256), 256, 0, s>>>(T, W_dev, L_dev);
  return cudaGetLastError();
}

// Block size for a launch over n devices: small launches (one colour of a high-conflict circuit)
// use one warp per block so the blocks spread over many SMs; large ones use kEvalBlock.
int eval_block(long long n, int block) {
  if (block > 0) return block;
  return n < 152LL * kEvalBlock ? 32 : kEvalBlock;
}

// Launch with programmatic stream serialisation when pdl: the kernel may begin while the previous
// kernel in the stream runs; it must wait (griddepcontrol.wait) before using that kernel's output.
template <typename... KArgs, typename... Args>
cudaError_t launch_maybe_pdl(void (*kern)(KArgs...), int g, int B, cudaStream_t s, bool pdl,
                             Args... args) {
  if (!pdl) {
    kern<<<g, B, 0, s>>>(args...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(g);
  cfg.blockDim = dim3(B);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

cudaError_t launch_eval(const DevTopo& T, int mode, int begin, int end, const double* x,
                        double* A, double* b, double* q, int block, int dbg, cudaStream_t s,
                        bool pdl) {
  if (end <= begin) return cudaSuccess;
  const int B = eval_block(end - begin, block);
  const int g = grid_for(end - begin, B);
  const bool wq = q != nullptr;
  switch (mode) {
    case MODE_RMW:
      if (wq) k_eval<MODE_RMW, true><<<g, B, 0, s>>>(T, begin, end, x, A, b, q, dbg);
      else k_eval<MODE_RMW, false><<<g, B, 0, s>>>(T, begin, end, x, A, b, q, dbg);
      break;
    case MODE_ATOMIC:
      if (wq) return launch_maybe_pdl(k_eval<MODE_ATOMIC, true>, g, B, s, pdl, T, begin, end, x, A, b, q, dbg);
      return launch_maybe_pdl(k_eval<MODE_ATOMIC, false>, g, B, s, pdl, T, begin, end, x, A, b, q, dbg);
    case MODE_SORTED:
      if (wq) k_eval<MODE_SORTED, true><<<g, B, 0, s>>>(T, begin, end, x, A, b, q, dbg);
      else k_eval<MODE_SORTED, false><<<g, B, 0, s>>>(T, begin, end, x, A, b, q, dbg);
      break;
    default:
      if (wq) k_eval<MODE_BUFFER, true><<<g, B, 0, s>>>(T, begin, end, x, A, b, q, dbg);
      else k_eval<MODE_BUFFER, false><<<g, B, 0, s>>>(T, begin, end, x, A, b, q, dbg);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_eval_ranges(const DevTopo& T, int mode, const int* rbeg, const int* roff,
                               int nr, int total, const double* x, double* A, double* b,
                               double* q, int block, int dbg, cudaStream_t s, bool pdl) {
  if (total <= 0 || nr <= 0) return cudaSuccess;
  const int B = eval_block(total, block);
  const int g = grid_for(total, B);
  const bool wq = q != nullptr;
  if (mode == MODE_ATOMIC) {
    if (wq)
      return launch_maybe_pdl(k_eval_ranges<MODE_ATOMIC, true>, g, B, s, pdl, T, rbeg, roff, nr,
                              total, x, A, b, q, dbg);
    return launch_maybe_pdl(k_eval_ranges<MODE_ATOMIC, false>, g, B, s, pdl, T, rbeg, roff, nr,
                            total, x, A, b, q, dbg);
  } else if (mode == MODE_BUFFER) {
    if (wq) k_eval_ranges<MODE_BUFFER, true><<<g, B, 0, s>>>(T, rbeg, roff, nr, total, x, A, b, q, dbg);
    else k_eval_ranges<MODE_BUFFER, false><<<g, B, 0, s>>>(T, rbeg, roff, nr, total, x, A, b, q, dbg);
  } else if (mode == MODE_SORTED) {
    if (wq) k_eval_ranges<MODE_SORTED, true><<<g, B, 0, s>>>(T, rbeg, roff, nr, total, x, A, b, q, dbg);
    else k_eval_ranges<MODE_SORTED, false><<<g, B, 0, s>>>(T, rbeg, roff, nr, total, x, A, b, q, dbg);
  } else {
    return cudaErrorInvalidValue;   // colour schedules are not order-free
  }
  return cudaGetLastError();
}

cudaError_t launch_eval_tran(const DevTopo& T, int mode, int begin, int end, const double* x,
                             double* A, double* b, const TranArgs& ta, int block, cudaStream_t s) {
  if (end <= begin) return cudaSuccess;
  const int B = eval_block(end - begin, block);
  const int g = grid_for(end - begin, B);
  if (mode == MODE_ATOMIC)
    return launch_maybe_pdl(k_eval_tran<MODE_ATOMIC>, g, B, s, true, T, begin, end, x, A, b, ta);
  else if (mode == MODE_BUFFER) k_eval_tran<MODE_BUFFER><<<g, B, 0, s>>>(T, begin, end, x, A, b, ta);
  else k_eval_tran<MODE_RMW><<<g, B, 0, s>>>(T, begin, end, x, A, b, ta);
  return cudaGetLastError();
}

int persistent_max_blocks_per_sm(int block, bool want_q) {
  (void)block;
  int nb = 0;
  cudaError_t e;
  if (want_q)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persistent<true>, kPersistBlock, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persistent<false>, kPersistBlock, 0);
  return e == cudaSuccess ? nb : 0;
}

cudaError_t launch_persistent(const DevTopo& T, const int* color_off_dev, int n_colors,
                              const double* x, double* A, double* b, double* q, int block,
                              int grid, int dbg, cudaStream_t s, int absent_block) {
  (void)block;
  cudaError_t e = cudaMemsetAsync(T.bar, 0, kBarWords * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  DevTopo Tc = T;
  const int* coff = color_off_dev;
  int C = n_colors;
  const double* xx = x;
  double* AA = A;
  double* bb = b;
  double* qq = q;
  int d = dbg;
  int ab = absent_block;
  void* args[] = {&Tc, &coff, &C, &xx, &AA, &bb, &qq, &d, &ab};
  if (q)
    return cudaLaunchCooperativeKernel((const void*)k_persistent<true>, dim3(grid),
                                       dim3(kPersistBlock), args, 0, s);
  return cudaLaunchCooperativeKernel((const void*)k_persistent<false>, dim3(grid),
                                     dim3(kPersistBlock), args, 0, s);
}

// A <- A_lin, b <- b_lin with the SMs (grid-stride, coalesced): a device-to-device copy on a
// copy engine moves these ~10 MB at about half a TB/s, the SMs at HBM speed.
__global__ void __launch_bounds__(256) k_init_lin(const double* __restrict__ Alin,
                                                  const double* __restrict__ blin, double* A,
                                                  double* b, long long nnz, long long n) {
  // the next kernel (the evaluation) may start now; it waits for this grid before touching A, b
  asm volatile("griddepcontrol.launch_dependents;");
  const long long total = nnz + n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    if (i < nnz) A[i] = __ldg(Alin + i);
    else b[i - nnz] = __ldg(blin + (i - nnz));
  }
}

cudaError_t launch_init_lin(const DevTopo& T, double* A, double* b, cudaStream_t s) {
  const long long total = T.nnz + T.n;
  if (total <= 0) return cudaSuccess;
  long long g = (total + 255) / 256;
  // grid-stride over 4 blocks per SM: enough to stream A_lin and b_lin at full bandwidth, and
  // the evaluation (a programmatic dependent) finds SMs with room for its blocks at once instead
  // of waiting for a full-occupancy copy to drain (1M-FET logic: 0.355 -> 0.350 ms per step)
  if (g > 152LL * 4) g = 152LL * 4;
  k_init_lin<<<(int)g, 256, 0, s>>>(T.Alin, T.blin, A, b, T.nnz, T.n);
  return cudaGetLastError();
}

cudaError_t launch_stamp_cluster(const DevTopo& T, const int* color_off_dev, int n_colors,
                                 double* A, double* b, cudaStream_t s) {
  if (n_colors <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClusterBlocks);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterBlocks;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_stamp_cluster, T, color_off_dev, n_colors, A, b);
}

int stamp_cluster_threads() { return kClusterBlocks * kClusterThreads; }

cudaError_t launch_stamp_cluster_tran(const DevTopo& T, const int* color_off_dev, int n_colors,
                                      double* A, double* b, cudaStream_t s) {
  if (n_colors <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClusterBlocks);
  cfg.blockDim = dim3(kClusterThreadsTran);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterBlocks;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_stamp_cluster_tran, T, color_off_dev, n_colors, A, b);
}

int stamp_persistent_max_blocks_per_sm() {
  int nb = 0;
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stamp_persistent,
                                                                      kStampBlock, 0);
  return e == cudaSuccess ? nb : 0;
}

cudaError_t launch_stamp_persistent(const DevTopo& T, const int* color_off_dev, int n_colors,
                                    double* A, double* b, int grid, cudaStream_t s) {
  if (n_colors <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(T.bar, 0, kBarWords * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  DevTopo Tc = T;
  const int* coff = color_off_dev;
  int C = n_colors;
  double* AA = A;
  double* bb = b;
  int ab = -1;
  void* args[] = {&Tc, &coff, &C, &AA, &bb, &ab};
  return cudaLaunchCooperativeKernel((const void*)k_stamp_persistent, dim3(grid),
                                     dim3(kStampBlock), args, 0, s);
}

cudaError_t launch_stamp_buffer(const DevTopo& T, int begin, int end, double* A, double* b,
                                int block, cudaStream_t s) {
  if (end <= begin) return cudaSuccess;
  const int B = eval_block(end - begin, block);
  k_stamp_buffer<<<grid_for(end - begin, B), B, 0, s>>>(T, begin, end, A, b);
  return cudaGetLastError();
}

int color_pipe_max_blocks_per_sm() {
  int a = 0, b2 = 0, c2 = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_color_pipe<true>, kPipeBlock, 0) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_color_pipe<false>, kPipeBlock, 0) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c2, k_color_pipe_tran, kPipeBlock, 0) !=
          cudaSuccess)
    return 0;
  return std::min(a, std::min(b2, c2));
}

cudaError_t launch_color_pipe(const DevTopo& T, int n_colors_nonempty, const double* x, double* A,
                              double* b, double* q, int grid, int dbg, cudaStream_t s,
                              int absent_item) {
  (void)n_colors_nonempty;
  (void)grid;
  if (T.n_pitem <= 0) return cudaSuccess;
  const int g = T.n_pitem;   // one block per work item (the items are taken by ticket)
  if (q)
    return launch_maybe_pdl(k_color_pipe<true>, g, kPipeBlock, s, true, T, x, A, b, q, dbg,
                            absent_item);
  return launch_maybe_pdl(k_color_pipe<false>, g, kPipeBlock, s, true, T, x, A, b, q, dbg,
                          absent_item);
}

cudaError_t launch_color_pipe_tran(const DevTopo& T, int n_colors_nonempty, const double* x,
                                   double* A, double* b, const TranArgs& ta, int grid,
                                   cudaStream_t s) {
  (void)n_colors_nonempty;
  (void)grid;
  if (T.n_pitem <= 0) return cudaSuccess;
  const int g = T.n_pitem;
  return launch_maybe_pdl(k_color_pipe_tran, g, kPipeBlock, s, true, T, x, A, b, ta);
}

cudaError_t math_check(int fn, long long n, const double* x, double* ours, double* ref,
                       cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_math_check<<<grid_for(n, 256), 256, 0, s>>>(fn, n, x, ours, ref);
  return cudaGetLastError();
}

cudaError_t fp64_peak(int iters, int blocks_per_sm, double* flops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = sms * blocks_per_sm, threads = 256;
  double* out = nullptr;
  e = cudaMalloc(&out, sizeof(double) * blocks * threads);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_dfma<<<blocks, threads>>>(out, iters / 8 + 1, 0.999999, 1e-9);  // warm-up
  cudaEventRecord(e0);
  k_dfma<<<blocks, threads>>>(out, iters, 0.999999, 1e-9);
  cudaEventRecord(e1);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return e;
  *flops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3);
  return cudaGetLastError();
}

}  // namespace eec
