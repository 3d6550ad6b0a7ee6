// The stamp half of the segmented-reduction schedule (EEC_VARIANT_SEGREDUCE): the per-entry
// gather of the contributions that the evaluation (MODE_SORTED) wrote to each entry's items.
//
// Sec. II: stamping accumulates every device's contributions into A and b; the colour order
// makes that lock-free on the CPU. Here the same sums are formed without colours and without
// atomics: each entry of [A ; b] is its linear part plus its own contributions, summed in one
// fixed order, so the result is the same bit for bit on every call.
#include <cuda_runtime.h>

#include "eec_internal.h"

namespace eec {

namespace {

// Segmented reduction: entry e of [A ; b] = its linear part + its contributions, summed in that
// order (deterministic, no colours needed). On this part a warp's FP64 addition occupies the
// SM's FP64 pipe for 16 cycles however many of its lanes are active, and entries average about
// one contribution, so one entry per lane, in entry order, leaves most lanes of every addition
// idle (the longest run of 32 neighbours sets the count). The layout therefore sorts the light
// entries of each window of kGatherWin entries by their count and stores them in groups of 32,
// column-major: one 256-byte load and one addition serve 32 entries of (nearly) equal length.
// One block takes one window: warp wi the groups wi, wi + 8, wi + 16, wi + 24; each thread loads
// the first kGatherAhead items of its four entries before it sums anything (more bytes in flight
// per thread); the sums go through shared memory to one coalesced store of the window's entries.
// 48 registers, 5 blocks per SM (bounded to 40 registers for a sixth block it spills and ran
// slower on the 1M-FET logic: 25.9 against 23.7 us).
// Heavy entries (word and bit line diagonals) take one warp each, in blocks after the windows:
// lane-strided partial sums, then a fixed butterfly reduction.
constexpr int kGatherBlock = 256;
constexpr int kGatherWarps = kGatherBlock / 32;
constexpr int kGatherPerWarp = kGatherGroups / kGatherWarps;   // groups per warp
constexpr int kGatherAhead = 3;   // items loaded before summing (the adds below assume 3)
static_assert(kGatherGroups % kGatherWarps == 0, "whole groups per warp");

__device__ __forceinline__ void put_entry(const DevTopo& T, double* A, double* b, long long e,
                                          double v) {
  if (e < T.nnz) A[e] = v;
  else b[e - T.nnz] = v;
}

// An FP64 addition that the compiler cannot execute speculatively: the adds of a group's rows
// sit behind branches on the (warp-uniform) row count, and a plain addition there is turned into
// an unconditional one plus a select, which would spend FP64-pipe cycles on the padding rows of
// every group (in random logic about 1.7x the useful additions).
__device__ __forceinline__ double add_taken(double a, double x) {
  double r;
  asm volatile("add.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(x));
  return r;
}

__global__ void __launch_bounds__(kGatherBlock) k_gather(DevTopo T, double* A, double* b, int nwin) {
  __shared__ double so[kGatherWin];
  __shared__ unsigned char sf[kGatherWin];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  if ((int)blockIdx.x < nwin) {
    const long long w = blockIdx.x;
    for (int t = threadIdx.x; t < kGatherWin; t += kGatherBlock) sf[t] = 0;
    const int* woff = T.gat_woff + w * (kGatherGroups + 1);
    int o0[kGatherPerWarp], nr[kGatherPerWarp];
    unsigned loc[kGatherPerWarp];
#pragma unroll
    for (int j = 0; j < kGatherPerWarp; ++j) {
      const int g = wi + kGatherWarps * j;
      o0[j] = __ldg(woff + g);
      nr[j] = (__ldg(woff + g + 1) - o0[j]) >> 5;   // the group's rows (0: no entries)
      loc[j] = __ldg(T.gat_loc + w * kGatherWin + 32 * g + lane);
    }
    double v[kGatherPerWarp][kGatherAhead];
#pragma unroll
    for (int j = 0; j < kGatherPerWarp; ++j)
#pragma unroll
      for (int k = 0; k < kGatherAhead; ++k)
        v[j][k] = k < nr[j] ? __ldcs(T.cbuf + o0[j] + 32 * k + lane) : 0.0;
    __syncthreads();   // every flag cleared before any is set
#pragma unroll
    for (int j = 0; j < kGatherPerWarp; ++j) {
      if (nr[j] == 0) continue;
      double sj = v[j][0];
      if (nr[j] > 1) {
        sj = add_taken(sj, v[j][1]);
        if (nr[j] > 2) {
          sj = add_taken(sj, v[j][2]);
          for (int k = kGatherAhead; k < nr[j]; ++k) sj += __ldcs(T.cbuf + o0[j] + 32 * k + lane);
        }
      }
      if (loc[j] != 0xffffu) {   // a lane past the group's entries holds zeros
        so[loc[j]] = sj;
        sf[loc[j]] = 1;
      }
    }
    __syncthreads();
    const long long e0 = w * kGatherWin;
    for (int t = threadIdx.x; t < kGatherWin; t += kGatherBlock)
      if (sf[t]) put_entry(T, A, b, e0 + t, so[t]);   // heavy entries: written by their warp
    return;
  }
  const int h = (blockIdx.x - nwin) * kGatherWarps + wi;
  if (h >= T.n_heavy) return;   // whole warp leaves together
  const int4 hd = __ldg(T.gat_heavy + h);
  double s = 0.0;
  for (int p = hd.y + lane; p < hd.y + hd.z; p += 32) s += __ldcs(T.cbuf + p);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) put_entry(T, A, b, hd.x, s);
}

// Linear parts to the first item of every entry: one thread per slot of a window, then one per
// heavy entry.
__global__ void k_gather_init(DevTopo T) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long slots = (long long)T.n_win * kGatherWin;
  if (t < slots) {
    const unsigned loc = T.gat_loc[t];
    if (loc == 0xffffu) return;
    const long long w = t / kGatherWin;
    const int i = (int)(t % kGatherWin);
    const long long e = w * kGatherWin + loc;
    T.cbuf[T.gat_woff[w * (kGatherGroups + 1) + i / 32] + (i % 32)] =
        e < T.nnz ? T.Alin[e] : T.blin[e - T.nnz];
  } else if (t - slots < T.n_heavy) {
    const int4 hd = T.gat_heavy[t - slots];
    const long long e = hd.x;
    T.cbuf[hd.y] = e < T.nnz ? T.Alin[e] : T.blin[e - T.nnz];
  }
}

}  // namespace

cudaError_t launch_gather(const DevTopo& T, double* A, double* b, cudaStream_t s) {
  const int nbh = (T.n_heavy + kGatherWarps - 1) / kGatherWarps;
  if (T.n_win + nbh == 0) return cudaSuccess;
  k_gather<<<T.n_win + nbh, kGatherBlock, 0, s>>>(T, A, b, T.n_win);
  return cudaGetLastError();
}

cudaError_t launch_gather_init(const DevTopo& T, cudaStream_t s) {
  const long long work = (long long)T.n_win * kGatherWin + T.n_heavy;
  if (work == 0) return cudaSuccess;
  k_gather_init<<<(int)((work + 255) / 256), 256, 0, s>>>(T);
  return cudaGetLastError();
}

}  // namespace eec
