// The stamp half of the segmented-reduction schedule (EEC_VARIANT_SEGREDUCE): the per-entry
// gather of the contributions that the evaluation (MODE_SORTED) wrote in entry order.
//
// Sec. II: stamping accumulates every device's contributions into A and b; the colour order
// makes that lock-free on the CPU. Here the same sums are formed without colours and without
// atomics: each entry of [A ; b] is its linear part plus its own contiguous run of
// contributions, summed in one fixed order, so the result is the same bit for bit on every call.
#include <cuda_runtime.h>

#include "eec_internal.h"

namespace eec {

namespace {

// Segmented reduction: entry e of [A ; b] = linear part + its contributions (deterministic, no
// colours needed). The evaluation has written every entry's contributions contiguously, in
// original-device order, at cbuf[gat_ptr[e] .. gat_ptr[e+1]), so the gather streams cbuf: light
// entries (< kHeavy contributions, nearly all) are summed in order by one thread each, heavy
// entries (diagonals of word and bit lines) are skipped there and take one warp each:
// lane-strided partial sums, then a fixed butterfly reduction. Blocks [0, nbl) cover the
// entries, the rest the heavy ones, in one launch.
// Entries average about one contribution, so the kernel is a chain of two dependent loads per
// entry (run pointer, then the run) plus the linear part and the store; a thread takes
// kGatherPer entries, kGatherBlock apart (each load instruction of a warp stays contiguous), and
// issues all their pointer and linear-part loads, then all their first contributions, before it
// sums anything: more bytes in flight per thread for the same occupancy.
constexpr int kGatherBlock = 256;
constexpr int kGatherPer = 2;     // entries per thread
constexpr int kGatherHead = 2;    // contributions per entry loaded ahead of the sums

__global__ void __launch_bounds__(kGatherBlock) k_gather(DevTopo T, double* A, double* b, int nbl) {
  const long long E = T.nnz + T.n;
  if ((int)blockIdx.x < nbl) {
    const long long e0 = (long long)blockIdx.x * (kGatherBlock * kGatherPer) + threadIdx.x;
    int p0[kGatherPer], cnt[kGatherPer];
    double s[kGatherPer];
#pragma unroll
    for (int j = 0; j < kGatherPer; ++j) {
      const long long e = e0 + (long long)j * kGatherBlock;
      p0[j] = 0;
      cnt[j] = 0;   // past the end: nothing to sum, nothing stored
      s[j] = 0.0;
      if (e < E) {
        p0[j] = __ldg(T.gat_ptr + e);
        cnt[j] = __ldg(T.gat_ptr + e + 1) - p0[j];
        s[j] = e < T.nnz ? __ldg(T.Alin + e) : __ldg(T.blin + (e - T.nnz));
      }
    }
    double v[kGatherPer][kGatherHead];
#pragma unroll
    for (int j = 0; j < kGatherPer; ++j)
#pragma unroll
      for (int t = 0; t < kGatherHead; ++t)
        v[j][t] = (t < cnt[j] && cnt[j] < kHeavy) ? __ldcs(T.cbuf + p0[j] + t) : 0.0;
#pragma unroll
    for (int j = 0; j < kGatherPer; ++j) {
      const long long e = e0 + (long long)j * kGatherBlock;
      if (e >= E || cnt[j] >= kHeavy) continue;   // heavy: a warp of the heavy blocks sums it
      double sj = s[j];
#pragma unroll
      for (int t = 0; t < kGatherHead; ++t)
        if (t < cnt[j]) sj += v[j][t];
      for (int p = p0[j] + kGatherHead; p < p0[j] + cnt[j]; ++p) sj += __ldcs(T.cbuf + p);
      if (e < T.nnz) A[e] = sj;
      else b[e - T.nnz] = sj;
    }
    return;
  }
  const int w = (blockIdx.x - nbl) * (kGatherBlock / 32) + (threadIdx.x >> 5);
  if (w >= T.n_heavy) return;   // whole warp leaves together
  const int lane = threadIdx.x & 31;
  const long long e = __ldg(T.gat_heavy + w);
  const int p0 = __ldg(T.gat_ptr + e), p1 = __ldg(T.gat_ptr + e + 1);
  double s = 0.0;
  for (int p = p0 + lane; p < p1; p += 32) s += __ldcs(T.cbuf + p);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) {
    if (e < T.nnz) A[e] = __ldg(T.Alin + e) + s;
    else b[e - T.nnz] = __ldg(T.blin + (e - T.nnz)) + s;
  }
}

}  // namespace

cudaError_t launch_gather(const DevTopo& T, double* A, double* b, cudaStream_t s) {
  const long long per_block = (long long)kGatherBlock * kGatherPer;
  const int nbl = (int)((T.nnz + T.n + per_block - 1) / per_block);
  const int nbh = (T.n_heavy + kGatherBlock / 32 - 1) / (kGatherBlock / 32);
  if (nbl + nbh == 0) return cudaSuccess;
  k_gather<<<nbl + nbh, kGatherBlock, 0, s>>>(T, A, b, nbl);
  return cudaGetLastError();
}

}  // namespace eec
