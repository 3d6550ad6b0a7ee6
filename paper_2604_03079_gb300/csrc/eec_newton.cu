// Kernels of the DC Newton loop on the GPU (eec_newton_dc): the damped update and the norms
// its convergence test reads. The loop itself (evaluate and stamp, sparse solve, update) is
// driven by the host side of the ABI.
//
// Norms are maxima of non-negative doubles, formed with 64-bit integer atomicMax on the bit
// patterns (for non-negative IEEE doubles the integer order is the numeric order; a NaN has a
// larger pattern than +inf, so it propagates to the maximum and the host sees it).
#include <cuda_runtime.h>

#include "eec_internal.h"

namespace eec {

namespace {

constexpr int kNewtonBlock = 256;

__device__ __forceinline__ void max_abs_into(unsigned long long* slot, double v) {
  // warp maximum first: one atomic per warp
  unsigned long long u = (unsigned long long)__double_as_longlong(fabs(v));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, u, off);
    u = o > u ? o : u;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(slot, u);
}

// stats[0] = max |y - x|
__global__ void __launch_bounds__(kNewtonBlock) k_step_norm(const double* __restrict__ y,
                                                            const double* __restrict__ x, int n,
                                                            unsigned long long* stats) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  max_abs_into(stats, i < n ? y[i] - x[i] : 0.0);
}

// The damped step: per_node = 0, x += s (y - x) with s = min(1, vstep / max|y - x|) (the whole
// step scaled so that no node moves more than vstep); per_node = 1, every node's move clipped to
// [-vstep, vstep] on its own. stats[1] = max |dx|, stats[2] = max |x| after the update.
__global__ void __launch_bounds__(kNewtonBlock) k_damped_update(const double* __restrict__ y,
                                                                double* __restrict__ x, int n,
                                                                double vstep, int per_node,
                                                                unsigned long long* stats) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double m = __longlong_as_double((long long)stats[0]);
  const double s = m > vstep ? vstep / m : 1.0;
  double dx = 0.0, xn = 0.0;
  if (i < n) {
    const double d = y[i] - x[i];
    // comparisons, not fmin/fmax: a NaN step stays NaN and the host sees it
    dx = per_node ? (d > vstep ? vstep : (d < -vstep ? -vstep : d)) : s * d;
    xn = x[i] + dx;
    x[i] = xn;
  }
  max_abs_into(stats + 1, dx);
  max_abs_into(stats + 2, xn);
}

// stats[3] = max |A x - b| (the KCL residual F(x), since A x - b = F(x) for the stamped system)
__global__ void __launch_bounds__(kNewtonBlock) k_residual_norm(const int* __restrict__ rp,
                                                                const int* __restrict__ col,
                                                                const double* __restrict__ A,
                                                                const double* __restrict__ x,
                                                                const double* __restrict__ b,
                                                                int n, unsigned long long* stats) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double r = 0.0;
  if (i < n) {
    r = -b[i];
    for (int p = rp[i]; p < rp[i + 1]; ++p) r = fma(A[p], x[col[p]], r);
  }
  max_abs_into(stats + 3, r);
}

// A[diag[i]] += g for the n node rows: a shunt conductance g from every node to ground (its
// current g v is linear in v, so b is unchanged)
__global__ void __launch_bounds__(kNewtonBlock) k_add_diag(double* __restrict__ A,
                                                           const int* __restrict__ diag, int n,
                                                           double g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A[diag[i]] += g;
}

// One sweep of nonlinear Jacobi relaxation (the relaxation start of eec_newton_dc): every node
// row i moves its own voltage to the zero of its linearised KCL residual with all other
// voltages held, y_i = x_i - F_i(x) / A_ii, the move clipped to [-vmax, vmax]; a row whose
// diagonal is not positive moves nothing. The other rows (rail source currents under modified
// nodal analysis) are copied. Reads x, writes y: every row sees the same iterate, so the sweep
// does not depend on the order of the threads. stats[1] = max |move|; stats[0] += the number of
// rows that moved more than 1 mV (when count is set).
__global__ void __launch_bounds__(kNewtonBlock) k_relax_step(const int* __restrict__ rp,
                                                             const int* __restrict__ col,
                                                             const double* __restrict__ A,
                                                             const double* __restrict__ x,
                                                             const double* __restrict__ b,
                                                             const int* __restrict__ diag,
                                                             int n_node, int n, double vmax,
                                                             double* __restrict__ y,
                                                             unsigned long long* stats,
                                                             int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double dx = 0.0;
  if (i < n) {
    if (i < n_node) {
      double r = -b[i];
      for (int p = rp[i]; p < rp[i + 1]; ++p) r = fma(A[p], x[col[p]], r);
      const double d = A[diag[i]];
      dx = d > 0.0 ? -r / d : 0.0;
      // comparisons, not fmin/fmax: a NaN move stays NaN and the host sees it
      dx = dx > vmax ? vmax : (dx < -vmax ? -vmax : dx);
    }
    y[i] = x[i] + dx;
  }
  max_abs_into(stats + 1, dx);
  if (count) {
    const unsigned moved = __ballot_sync(0xffffffffu, fabs(dx) > 1e-3);
    if ((threadIdx.x & 31) == 0 && moved) atomicAdd(stats, (unsigned long long)__popc(moved));
  }
}

// Rails as MNA unknowns: rail node rail_unk[r] takes its source's voltage, the right-hand side
// of its source equation (row n_node + r).
__global__ void k_rail_fix(double* __restrict__ y, const double* __restrict__ b,
                           const int* __restrict__ rail_unk, int n_node, int n_rail) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_rail) y[rail_unk[r]] = b[n_node + r];
}

int blocks_for(int n) { return n > 0 ? (n + kNewtonBlock - 1) / kNewtonBlock : 1; }

}  // namespace

cudaError_t launch_newton_step(const double* y, double* x, int n, double vstep, int per_node,
                               unsigned long long* stats, cudaStream_t s) {
  k_step_norm<<<blocks_for(n), kNewtonBlock, 0, s>>>(y, x, n, stats);
  k_damped_update<<<blocks_for(n), kNewtonBlock, 0, s>>>(y, x, n, vstep, per_node, stats);
  return cudaGetLastError();
}

cudaError_t launch_residual_norm(const int* rp, const int* col, const double* A, const double* x,
                                 const double* b, int n, unsigned long long* stats,
                                 cudaStream_t s) {
  k_residual_norm<<<blocks_for(n), kNewtonBlock, 0, s>>>(rp, col, A, x, b, n, stats);
  return cudaGetLastError();
}

cudaError_t launch_relax_step(const int* rp, const int* col, const double* A, const double* x,
                              const double* b, const int* diag, int n_node, int n, double vmax,
                              const int* rail_unk, int n_rail, double* y,
                              unsigned long long* stats, int count, cudaStream_t s) {
  k_relax_step<<<blocks_for(n), kNewtonBlock, 0, s>>>(rp, col, A, x, b, diag, n_node, n, vmax, y,
                                                      stats, count);
  if (n_rail > 0) k_rail_fix<<<blocks_for(n_rail), kNewtonBlock, 0, s>>>(y, b, rail_unk, n_node, n_rail);
  return cudaGetLastError();
}

cudaError_t launch_add_diag(double* A, const int* diag, int n, double g, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_add_diag<<<blocks_for(n), kNewtonBlock, 0, s>>>(A, diag, n, g);
  return cudaGetLastError();
}

}  // namespace eec
