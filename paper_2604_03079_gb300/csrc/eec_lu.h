// Sparse LU of eec_newton_dc's solver EEC_SOLVER_LU (eec_lu.cu): the plan, its device view and
// the host and GPU steps. Kept apart from eec_internal.h: the evaluate-and-stamp kernels do not
// depend on it.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

namespace eec {

// Plan of the factorisation P A Q = L U on a fixed pattern (host vectors; see eec_lu.cu).
struct LuPlan {
  int n = 0;
  std::vector<int> prow, pcol;          // row k of P A Q = row prow[k] of A; column j = pcol[j]
  std::vector<int> cptr, crow, cdiag;   // column storage: U part, diagonal, L part
  std::vector<int> a2lu;                // A's CSR entry -> storage position
  std::vector<int> uptr, uk, upos;      // per column j: the k of U(:, j) and U(k, j)'s position
  std::vector<int> mptr, msrc, mdst;    // per (k, j): L(:, k) positions and their targets in j
  std::vector<int> lrptr, lrcol, lrpos; // rows of L (strictly lower): column, position
  std::vector<int> urptr, urcol, urpos; // rows of U (strictly upper): column, position
};
// Device view of a plan plus its value array, a work vector and the flags ([0] first column
// whose pivot fell below tiny x its column's largest L entry, plus 1; [1] a wait timed out;
// [2] first column with a zero or non-finite pivot, plus 1).
struct LuDev {
  int n, nnz_lu, nnz_a;
  const int *cptr, *cdiag, *a2lu, *uptr, *uk, *upos, *mptr, *msrc, *mdst;
  const int *lrptr, *lrcol, *lrpos, *urptr, *urcol, *urpos, *prow, *pcol;
  double* vals;
  double* y;     // [4n] work vector and inverse diagonal (when the factor is not in shared
                 // memory), then the refinement's residual and correction
  int* flag;
  int* gwork;    // [lu_grid_words()] progress words and barrier of the multi-block kernel
  const int* ibase;   // the packed buffer every index array above lives in (16-byte aligned
  long long ilen;     // parts), and its length in ints (a multiple of 4)
};
// Words of LuDev::gwork: a grid barrier and one progress word per warp of the largest grid the
// multi-block kernel launches on this device.
int lu_grid_words();
// Entries the host analysis may create for a pattern of nnz entries in the order's elimination
// graph and in the factor: 32 nnz + 4 Mi (its update list has a budget of its own, in
// eec_lu.cu). Circuit matrices with locality stay far below (the 256 x 256 SRAM: 1.2 nnz);
// randomly wired netlists have no good elimination order and would fill towards a dense factor.
long long lu_entry_budget(long long nnz);
// Host: multiple-minimum-degree column order of the symmetric pattern of A + A^T; false (order left
// empty) when the elimination graph would outgrow lu_entry_budget.
bool lu_min_degree_order(int n, const std::vector<int>& rp, const std::vector<int>& col,
                         std::vector<int>& order);
// Host: block triangular order (strongly connected components of A's directed graph, each
// after the components it reaches; multiple minimum degree inside each); false when a
// component's order outgrows the budget.
bool lu_btf_order(int n, const std::vector<int>& rp, const std::vector<int>& col,
                  std::vector<int>& order);
// Host: longest chains of dependent steps of a plan: refactorisation, forward and backward
// substitution.
void lu_plan_depth(const LuPlan& P, int depth[3]);
// Host: plan of A (CSR) in column order q from one factorisation with threshold partial
// pivoting. Returns 0, EEC_ENUMERIC (a numerically singular column) or EEC_ENOMEM (the factor
// or its update list would outgrow its budget), with err set.
int lu_analyze(int n, const std::vector<int>& rp, const std::vector<int>& col,
               const std::vector<double>& a, const std::vector<int>& q, LuPlan& P,
               std::string& err);
// Host: the GPU's refactorisation and solves, in the same order (a check of the plan).
bool lu_refactor_solve_host(const LuPlan& P, const std::vector<double>& a,
                            const std::vector<double>& b, double tiny, std::vector<double>& x,
                            int* bad_col);
// Refactor A (CSR values, pattern rp/col) on the plan and solve A x = b, with refine one step of
// iterative refinement: in one single-block kernel when the factor fits in shared memory, else in
// one cooperative kernel over every SM (the factor in global memory).
cudaError_t launch_lu_factor_solve(const LuDev& L, const double* A, const int* rp, const int* col,
                                   const double* b, double* x, double tiny, int refine,
                                   cudaStream_t s);

}  // namespace eec
