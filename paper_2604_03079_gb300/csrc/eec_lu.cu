// Sparse LU of the MNA matrix for the GPU Newton loop (eec_newton_dc, solver EEC_SOLVER_LU).
//
// Once the evaluate-and-stamp step is fast the linear solve dominates the Newton iteration
// (Sec. III: matrix solve against device evaluation, Table II); the paper solves with KLU on the
// host. Here the pattern of A never changes between iterations, so the expensive symbolic work is
// done once and only the numbers are recomputed on the GPU every iteration:
//  * host, once per pattern (again only if a pivot degrades): a fill-reducing column order
//    (multiple minimum degree on the symmetric pattern), then one left-looking sparse LU of
//    the first iterate's matrix with threshold partial pivoting (Gilbert-Peierls: the pattern of
//    every column is the set reached in the graph of the L columns before it, so it does not
//    depend on the values). It fixes the row pivot sequence and the structural patterns of L and
//    U, and the plan below;
//  * GPU, every iteration: the numeric refactorisation on that pattern with those pivots, then
//    the two triangular solves, each in one single-block kernel. Columns (rows for the solves)
//    are dealt to the block's 32 warps round robin; a warp waits for the columns its column
//    depends on through a 32-entry progress array in shared memory (column k is final once the
//    warp that owns it has moved past k), so independent columns proceed in parallel and a chain
//    of dependent columns costs one warp step per column. All waits are bounded.
// Storage, column j of the permuted matrix P A Q: its U part (rows k < j, ascending), the
// diagonal, then its L part (rows > j, ascending), in one value array.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <iterator>
#include <set>
#include <string>
#include <vector>

#include "eec_internal.h"
#include "eec_lu.h"

namespace eec {

// ---- host analysis ----------------------------------------------------------------------------

// Minimum-degree order of the symmetric pattern of A + A^T (diagonal ignored), by passes of
// multiple elimination: each pass eliminates, in index order, every node of the current least
// degree that no node eliminated earlier in the pass neighbours, joining each one's remaining
// neighbours into a clique as elimination does. Eliminating one node of least degree at a time
// (ties to the lowest index) would run along a chain of gates node after node, and through a
// batch of circuits circuit after circuit: every column of the order then depends on the one
// before it, and the GPU refactorisation, which deals consecutive columns to different warps,
// becomes one long chain. A pass takes the ends of all chains at once instead (the order's
// consecutive columns are independent) at the same fill. Explicit adjacency; the netlists this
// serves have small degrees away from the rails, which the rule leaves to the end.
long long lu_entry_budget(long long nnz) { return 32 * nnz + (4LL << 20); }

// The update list (one entry per multiply-add of the factorisation) of a pattern of nnz entries
// may hold 128 nnz + 16 Mi entries (the 256 x 256 SRAM: 39 nnz, from the dense block its word
// and bit lines leave at the end of the order), and at most what 32-bit offsets address.
static long long lu_update_budget(long long nnz) {
  return std::min<long long>(128 * nnz + (16LL << 20), 0x7fffffffLL);
}

bool lu_min_degree_order(int n, const std::vector<int>& rp, const std::vector<int>& col,
                         std::vector<int>& order) {
  const long long budget = lu_entry_budget(rp[n]);
  std::vector<std::vector<int>> adj(n);
  for (int i = 0; i < n; ++i)
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const int j = col[e];
      if (j == i) continue;
      adj[i].push_back(j);
      adj[j].push_back(i);
    }
  for (auto& a : adj) {
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
  }
  std::set<std::pair<int, int>> by_deg;   // (degree, node) of the nodes not yet eliminated
  long long total = 0;                      // entries of the elimination graph
  for (int i = 0; i < n; ++i) {
    by_deg.insert({(int)adj[i].size(), i});
    total += (long long)adj[i].size();
  }
  order.clear();
  order.reserve(n);
  std::vector<int> merged, cand;
  std::vector<int> touched(n, 0);   // pass in which a neighbour was eliminated
  int pass = 0;
  while (!by_deg.empty()) {
    const int dmin = by_deg.begin()->first;
    cand.clear();
    for (auto it = by_deg.begin(); it != by_deg.end() && it->first == dmin; ++it)
      cand.push_back(it->second);
    ++pass;
    for (const int v : cand) {
      if (touched[v] == pass) continue;   // its degree changed in this pass
      by_deg.erase({dmin, v});
      order.push_back(v);
      const std::vector<int> nb = std::move(adj[v]);
      adj[v].clear();
      total -= (long long)nb.size();
      for (int a : nb) {
        touched[a] = pass;
        by_deg.erase({(int)adj[a].size(), a});
        total -= (long long)adj[a].size();
        // adj[a] := (adj[a] without v) joined with the other neighbours of v
        merged.clear();
        std::set_union(adj[a].begin(), adj[a].end(), nb.begin(), nb.end(),
                       std::back_inserter(merged));
        merged.erase(std::remove_if(merged.begin(), merged.end(),
                                    [&](int u) { return u == v || u == a; }),
                     merged.end());
        adj[a].swap(merged);
        by_deg.insert({(int)adj[a].size(), a});
        total += (long long)adj[a].size();
      }
      if (total > budget) {   // the fill of this pattern outgrows any useful factor
        order.clear();
        return false;
      }
    }
  }
  return true;
}

// Block triangular order: the strongly connected components of the directed graph of A (an
// edge i -> j for every off-diagonal A(i, j)), each component after every component its edges
// lead to, and each component's columns in the multiple-minimum-degree order of its own
// symmetric pattern. Tarjan's algorithm completes a component only after every component it
// reaches, so its completion order is such an order. With A's diagonal present the permuted
// matrix is block lower triangular: elimination fills only inside the diagonal blocks and the
// rows below them, and a column waits only on columns it reaches. A netlist whose gates are
// wired without loops (a DAG, components of one gate) then factors with almost no fill and a
// chain of dependent columns as long as its logic depth; a minimum-degree order of the
// symmetric pattern ignores the direction and fills. False when a component's minimum-degree
// order outgrows its budget.
bool lu_btf_order(int n, const std::vector<int>& rp, const std::vector<int>& col,
                  std::vector<int>& order) {
  std::vector<int> index(n, -1), low(n, 0), comp(n, -1);
  std::vector<char> on_stack(n, 0);
  std::vector<int> stack, members;          // Tarjan's stack; nodes by component, in order
  std::vector<int> comp_start{0};
  std::vector<std::pair<int, int>> call;    // (node, next edge) of the depth-first search
  int next_index = 0;
  for (int s = 0; s < n; ++s) {
    if (index[s] >= 0) continue;
    index[s] = low[s] = next_index++;
    stack.push_back(s);
    on_stack[s] = 1;
    call.push_back({s, rp[s]});
    while (!call.empty()) {
      const int v = call.back().first;
      const int e = call.back().second;
      if (e < rp[v + 1]) {
        call.back().second = e + 1;
        const int w = col[e];
        if (w == v) continue;
        if (index[w] < 0) {
          index[w] = low[w] = next_index++;
          stack.push_back(w);
          on_stack[w] = 1;
          call.push_back({w, rp[w]});
        } else if (on_stack[w]) {
          low[v] = std::min(low[v], index[w]);
        }
        continue;
      }
      if (low[v] == index[v]) {   // v roots a component: pop it
        const int c = (int)comp_start.size() - 1;
        int w;
        do {
          w = stack.back();
          stack.pop_back();
          on_stack[w] = 0;
          comp[w] = c;
          members.push_back(w);
        } while (w != v);
        comp_start.push_back((int)members.size());
      }
      call.pop_back();
      if (!call.empty()) {
        const int u = call.back().first;
        low[u] = std::min(low[u], low[v]);
      }
    }
  }
  order.clear();
  order.reserve(n);
  std::vector<int> local(n, -1), srp, scol, sub;
  for (size_t c = 0; c + 1 < comp_start.size(); ++c) {
    const int b0 = comp_start[c], b1 = comp_start[c + 1], m = b1 - b0;
    if (m == 1) {
      order.push_back(members[b0]);
      continue;
    }
    std::vector<int> nodes(members.begin() + b0, members.begin() + b1);
    std::sort(nodes.begin(), nodes.end());
    for (int i = 0; i < m; ++i) local[nodes[i]] = i;
    srp.assign(1, 0);
    scol.clear();
    for (int i = 0; i < m; ++i) {
      const int r = nodes[i];
      for (int e = rp[r]; e < rp[r + 1]; ++e)
        if (comp[col[e]] == (int)c) scol.push_back(local[col[e]]);
      srp.push_back((int)scol.size());
    }
    if (!lu_min_degree_order(m, srp, scol, sub)) {
      order.clear();
      return false;
    }
    for (int i : sub) order.push_back(nodes[i]);
  }
  return true;
}

// Longest chains of dependent steps of a plan, which the GPU can take in no fewer steps however
// many warps it has: depth[0] of the refactorisation (column j waits for every column k of
// U(:, j)), depth[1] of the forward substitution (row i waits for the columns of L(i, :)),
// depth[2] of the backward substitution (row i waits for the columns of U(i, :)).
void lu_plan_depth(const LuPlan& P, int depth[3]) {
  const int n = P.n;
  std::vector<int> d(n, 0);
  int best = 0;
  for (int j = 0; j < n; ++j) {
    int m = 0;
    for (int t = P.uptr[j]; t < P.uptr[j + 1]; ++t)
      if (P.uk[t] != j) m = std::max(m, d[P.uk[t]]);
    d[j] = m + 1;
    best = std::max(best, d[j]);
  }
  depth[0] = best;
  best = 0;
  for (int i = 0; i < n; ++i) {
    int m = 0;
    for (int t = P.lrptr[i]; t < P.lrptr[i + 1]; ++t) m = std::max(m, d[P.lrcol[t]]);
    d[i] = m + 1;
    best = std::max(best, d[i]);
  }
  depth[1] = best;
  best = 0;
  for (int i = n - 1; i >= 0; --i) {
    int m = 0;
    for (int t = P.urptr[i]; t < P.urptr[i + 1]; ++t) m = std::max(m, d[P.urcol[t]]);
    d[i] = m + 1;
    best = std::max(best, d[i]);
  }
  depth[2] = best;
}

constexpr double kLuDiagPref = 1e-3;

// Left-looking LU with threshold partial pivoting of B = A(:, q) (A in CSR, symmetric pattern
// not required); plan out. Returns 0, EEC_ENUMERIC for a numerically singular column or
// EEC_ENOMEM when the factor or its update list outgrows lu_entry_budget (err set).
int lu_analyze(int n, const std::vector<int>& rp, const std::vector<int>& col,
               const std::vector<double>& a, const std::vector<int>& q, LuPlan& P,
               std::string& err) {
  const int nnz = rp[n];
  const long long budget = lu_entry_budget(nnz), update_budget = lu_update_budget(nnz);
  long long n_factor = 0;   // entries of L and U so far
  // CSC of A: column c lists (row, CSR position)
  std::vector<int> cp(n + 1, 0), ci(nnz), cpos(nnz);
  for (int e = 0; e < nnz; ++e) cp[col[e] + 1]++;
  for (int c = 0; c < n; ++c) cp[c + 1] += cp[c];
  {
    std::vector<int> fill(cp.begin(), cp.end() - 1);
    for (int i = 0; i < n; ++i)
      for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const int f = fill[col[e]]++;
        ci[f] = i;
        cpos[f] = e;
      }
  }
  // factor: L columns with original row indices (values already divided by the pivot)
  std::vector<std::vector<std::pair<int, double>>> Lc(n);
  std::vector<std::vector<int>> Uk(n);   // U(:, j): pivot steps k < j (pattern only)
  std::vector<int> pinv(n, -1), prow(n, -1);
  std::vector<double> x(n, 0.0);
  std::vector<char> mark(n, 0);
  std::vector<int> pat, topo, stack, head;
  for (int j = 0; j < n; ++j) {
    const int c = q[j];
    // pattern: rows of B(:, j) plus everything reached through the L columns of pivoted rows;
    // topo receives the reached pivot steps in reverse post-order (a valid update order)
    pat.clear();
    topo.clear();
    for (int f = cp[c]; f < cp[c + 1]; ++f) {
      const int i0 = ci[f];
      if (mark[i0]) continue;
      mark[i0] = 1;
      pat.push_back(i0);
      if (pinv[i0] < 0) continue;
      // iterative DFS over pivot steps
      stack.assign(1, pinv[i0]);
      head.assign(1, 0);
      while (!stack.empty()) {
        const int k = stack.back();
        int& h = head.back();
        bool pushed = false;
        while (h < (int)Lc[k].size()) {
          const int i = Lc[k][h++].first;
          if (mark[i]) continue;
          mark[i] = 1;
          pat.push_back(i);
          if (pinv[i] >= 0) {
            stack.push_back(pinv[i]);
            head.push_back(0);
            pushed = true;
            break;
          }
        }
        if (!pushed) {
          topo.push_back(k);
          stack.pop_back();
          head.pop_back();
        }
      }
    }
    for (int f = cp[c]; f < cp[c + 1]; ++f) x[ci[f]] = a[cpos[f]];
    // updates in topological order: reverse of the post-order
    for (int t = (int)topo.size() - 1; t >= 0; --t) {
      const int k = topo[t];
      const double xk = x[prow[k]];
      for (const auto& e : Lc[k]) x[e.first] -= e.second * xk;
    }
    // pivot: the largest unpivoted entry, or the diagonal row c when it is within a factor
    // kLuDiagPref of it (the default threshold of KLU: keeps the diagonal of circuit matrices,
    // whose off-diagonal transconductances would otherwise shift every pivot of a long chain
    // of gates one row down and leave one row to underflow)
    int piv = -1;
    double best = 0.0;
    for (int i : pat)
      if (pinv[i] < 0 && std::fabs(x[i]) > best) {
        best = std::fabs(x[i]);
        piv = i;
      }
    if (piv < 0 || !(best > 0.0) || !std::isfinite(best)) {
      err = "sparse LU: matrix singular at column " + std::to_string(j);
      for (int i : pat) { x[i] = 0.0; mark[i] = 0; }
      return EEC_ENUMERIC;
    }
    if (pinv[c] < 0 && mark[c] && std::fabs(x[c]) >= kLuDiagPref * best) piv = c;
    const double pv = x[piv];
    pinv[piv] = j;
    prow[j] = piv;
    for (int i : pat) {
      if (pinv[i] >= 0 && pinv[i] < j) Uk[j].push_back(pinv[i]);
      else if (i != piv) Lc[j].push_back({i, x[i] / pv});
      x[i] = 0.0;
      mark[i] = 0;
    }
    std::sort(Uk[j].begin(), Uk[j].end());
    n_factor += (long long)Uk[j].size() + 1 + (long long)Lc[j].size();
    if (n_factor > budget) {
      err = "sparse LU: the factor of this pattern would exceed " + std::to_string(budget) +
            " entries (32 per nonzero of A plus 4 Mi): too much fill for a direct solve";
      return EEC_ENOMEM;
    }
  }
  // plan: column storage of P A Q (rows in pivot-step numbering)
  P.n = n;
  P.prow = prow;
  P.pcol = q;
  P.cptr.assign(n + 1, 0);
  for (int j = 0; j < n; ++j) P.cptr[j + 1] = P.cptr[j] + (int)Uk[j].size() + 1 + (int)Lc[j].size();
  const int nlu = P.cptr[n];
  P.crow.assign(nlu, 0);
  P.cdiag.assign(n, 0);
  std::vector<std::vector<int>> Lrows(n);   // L(:, j) rows in pivot-step numbering, ascending
  for (int j = 0; j < n; ++j) {
    int p = P.cptr[j];
    for (int k : Uk[j]) P.crow[p++] = k;
    P.cdiag[j] = p;
    P.crow[p++] = j;
    for (const auto& e : Lc[j]) Lrows[j].push_back(pinv[e.first]);
    std::sort(Lrows[j].begin(), Lrows[j].end());
    for (int r : Lrows[j]) P.crow[p++] = r;
  }
  auto find = [&](int r, int j) -> int {   // position of (r, j) in column j, or -1
    const int* b0 = P.crow.data() + P.cptr[j];
    const int* d = P.crow.data() + P.cdiag[j];
    const int* b1 = P.crow.data() + P.cptr[j + 1];
    if (r < j) {
      const int* f = std::lower_bound(b0, d, r);
      return (f != d && *f == r) ? (int)(f - P.crow.data()) : -1;
    }
    if (r == j) return P.cdiag[j];
    const int* f = std::lower_bound(d + 1, b1, r);
    return (f != b1 && *f == r) ? (int)(f - P.crow.data()) : -1;
  };
  std::vector<int> qinv(n);
  for (int j = 0; j < n; ++j) qinv[q[j]] = j;
  P.a2lu.assign(nnz, -1);
  for (int i = 0; i < n; ++i)
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      P.a2lu[e] = find(pinv[i], qinv[col[e]]);
      if (P.a2lu[e] < 0) {
        err = "sparse LU: an entry of A outside the factor pattern";
        return EEC_ENUMERIC;
      }
    }
  // updates of column j: for every k of U(:, j) (ascending), the entries of L(:, k) go to the
  // rows of column j they hit
  P.uptr.assign(n + 1, 0);
  P.uk.clear();
  P.upos.clear();
  P.mptr.assign(1, 0);
  P.msrc.clear();
  P.mdst.clear();
  for (int j = 0; j < n; ++j) {
    for (int p = P.cptr[j]; p < P.cdiag[j]; ++p) {
      const int k = P.crow[p];
      P.uk.push_back(k);
      P.upos.push_back(p);
      for (int s = P.cdiag[k] + 1; s < P.cptr[k + 1]; ++s) {
        const int d = find(P.crow[s], j);
        if (d < 0) {
          err = "sparse LU: an update outside the factor pattern";
          return EEC_ENUMERIC;
        }
        P.msrc.push_back(s);
        P.mdst.push_back(d);
      }
      if ((long long)P.msrc.size() > update_budget) {
        err = "sparse LU: the update list of this pattern would exceed " +
              std::to_string(update_budget) + " entries: too much fill for a direct solve";
        return EEC_ENOMEM;
      }
      P.mptr.push_back((int)P.msrc.size());
    }
    P.uptr[j + 1] = (int)P.uk.size();
  }
  // rows of L (strictly lower) and of U (strictly upper) for the two substitutions
  std::vector<std::vector<std::pair<int, int>>> lr(n), ur(n);
  for (int j = 0; j < n; ++j)
    for (int p = P.cptr[j]; p < P.cptr[j + 1]; ++p) {
      const int r = P.crow[p];
      if (r > j) lr[r].push_back({j, p});
      else if (r < j) ur[r].push_back({j, p});
    }
  P.lrptr.assign(n + 1, 0);
  P.urptr.assign(n + 1, 0);
  P.lrcol.clear();
  P.lrpos.clear();
  P.urcol.clear();
  P.urpos.clear();
  for (int r = 0; r < n; ++r) {
    for (const auto& e : lr[r]) { P.lrcol.push_back(e.first); P.lrpos.push_back(e.second); }
    for (const auto& e : ur[r]) { P.urcol.push_back(e.first); P.urpos.push_back(e.second); }
    P.lrptr[r + 1] = (int)P.lrcol.size();
    P.urptr[r + 1] = (int)P.urcol.size();
  }
  return 0;
}

// The GPU's refactorisation and substitutions executed on the host in the same order (column by
// column, updates in ascending k, rows in order, the same pivot test): a check of the plan
// without a GPU.
bool lu_refactor_solve_host(const LuPlan& P, const std::vector<double>& a,
                            const std::vector<double>& b, double tiny, std::vector<double>& x,
                            int* bad_col) {
  const int n = P.n;
  std::vector<double> v(P.cptr[n], 0.0), dinv(n);
  for (size_t e = 0; e < P.a2lu.size(); ++e) v[P.a2lu[e]] = a[e];
  for (int j = 0; j < n; ++j) {
    for (int t = P.uptr[j]; t < P.uptr[j + 1]; ++t) {
      const double ukj = v[P.upos[t]];
      for (int m = P.mptr[t]; m < P.mptr[t + 1]; ++m) v[P.mdst[m]] -= v[P.msrc[m]] * ukj;
    }
    dinv[j] = 1.0 / v[P.cdiag[j]];
    for (int p = P.cdiag[j] + 1; p < P.cptr[j + 1]; ++p) v[p] *= dinv[j];
  }
  *bad_col = -1;
  for (int j = 0; j < n && *bad_col < 0; ++j) {
    bool bad = !std::isfinite(dinv[j]) || dinv[j] == 0.0;
    for (int p = P.cdiag[j] + 1; p < P.cptr[j + 1] && !bad; ++p) bad = !(std::fabs(v[p]) < 1.0 / tiny);
    if (bad) *bad_col = j;
  }
  std::vector<double> y(n);
  for (int r = 0; r < n; ++r) {
    double s = 0.0;
    for (int p = P.lrptr[r]; p < P.lrptr[r + 1]; ++p) s += v[P.lrpos[p]] * y[P.lrcol[p]];
    y[r] = b[P.prow[r]] - s;
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = 0.0;
    for (int p = P.urptr[r]; p < P.urptr[r + 1]; ++p) s += v[P.urpos[p]] * y[P.urcol[p]];
    y[r] = (y[r] - s) * dinv[r];
  }
  x.assign(n, 0.0);
  for (int j = 0; j < n; ++j) x[P.pcol[j]] = y[j];
  return *bad_col < 0;
}

// ---- GPU refactorisation and solves -------------------------------------------------------------

namespace {

constexpr int kLuWarps = 32;
constexpr long long kLuSpinLimit = 1LL << 26;   // polls of a progress word before giving up

// Wait until the warp that owns item k (of the round-robin deal) has moved past it. Returns
// false when the bound is reached (recording a timeout in flag[1]) or when another wait has
// already given up: then every later wait returns at once, the block runs to its end with
// meaningless numbers and the host reports the timeout. Control flow stays the same for every
// warp, so no barrier of the block is ever left waiting.
__device__ __forceinline__ bool lu_wait(volatile int* prog, int k, int* flag) {
  long long spins = 0;
  while (prog[k % kLuWarps] <= k) {
    if (*((volatile int*)(flag + 1))) return false;
    if (++spins > kLuSpinLimit) {
      atomicExch(flag + 1, 1);
      return false;
    }
  }
  __threadfence_block();
  return true;
}

// Reciprocal from the FP32 unit's seed and two FP64 corrections (the seed's 2^-23 error cubed:
// far below an ulp): one FP64 dependency chain of three instructions instead of a division.
// FP64 instructions wait about 64 cycles each on this part, and the factorisation and the
// substitutions are chains of dependent steps, so every instruction on a step counts.
__device__ __forceinline__ double lu_rcp(double x) {
  const double y0 = (double)__frcp_rn((float)x);
  const double e = fma(-x, y0, 1.0);
  return fma(y0, fma(e, e, e), y0);
}

// Dot product of the row's entries (positions pos[p0..p1), columns cols[...]) with the vector u,
// each entry's column first waited for. Short rows (the common case in circuit matrices) are
// summed by lane 0 alone, without a shuffle tree of dependent FP64 additions.
__device__ __forceinline__ double lu_row_dot(const int* __restrict__ cols, const int* __restrict__ pos,
                                             int p0, int p1, const double* v, const double* u,
                                             volatile int* prog, int* flag, bool reversed, int n) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  if (p1 - p0 <= 4) {
    if (lane == 0)
      for (int p = p0; p < p1; ++p) {
        const int c = cols[p];
        lu_wait(prog, reversed ? n - 1 - c : c, flag);
        s = fma(v[pos[p]], u[c], s);
      }
    return s;   // meaningful in lane 0
  }
  for (int p = p0 + lane; p < p1; p += 32) {
    const int c = cols[p];
    lu_wait(prog, reversed ? n - 1 - c : c, flag);
    s = fma(v[pos[p]], u[c], s);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

// Forward then backward substitution with the factor in v and the inverse diagonal in dinv
// (y as work): x[pcol] = the solution of P A Q z = P b, i.e. A x = b.
__device__ __forceinline__ void lu_substitute(const LuDev& L, const double* v, const double* dinv,
                                              double* y, volatile int* prog,
                                              const double* b, double* x) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n = L.n;
  // forward (unit lower): y[r] = b[prow[r]] - sum_c L(r, c) y[c], rows in order
  if (lane == 0) prog[w] = w;
  __syncthreads();
  for (int r = w; r < n; r += kLuWarps) {
    const double s = lu_row_dot(L.lrcol, L.lrpos, L.lrptr[r], L.lrptr[r + 1], v,
                                y, prog, L.flag, false, n);
    if (lane == 0) {
      y[r] = b[L.prow[r]] - s;
      __threadfence_block();
      prog[w] = r + kLuWarps;
    }
    __syncwarp();
  }
  __syncthreads();
  // backward: z[r] = (y[r] - sum_c U(r, c) z[c]) / U(r, r), rows from the last (item
  // m = n - 1 - r of the deal), z kept in y's place
  if (lane == 0) prog[w] = w;
  __syncthreads();
  for (int m = w; m < n; m += kLuWarps) {
    const int r = n - 1 - m;
    const double s = lu_row_dot(L.urcol, L.urpos, L.urptr[r], L.urptr[r + 1], v,
                                y, prog, L.flag, true, n);
    if (lane == 0) {
      y[r] = (y[r] - s) * dinv[r];
      __threadfence_block();
      prog[w] = m + kLuWarps;
    }
    __syncwarp();
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) x[L.pcol[r]] = y[r];
}

// Doubles of the shared-memory values region: factor, inverse diagonal, work vector; an even
// count, so that the index arrays after it start on 16 bytes.
__host__ __device__ __forceinline__ long long lu_vals_doubles(const LuDev& L) {
  return ((long long)L.nnz_lu + 2LL * L.n + 1) & ~1LL;
}

// Refactorisation of A on the plan, then x = A^-1 b, in one block; with refine, one step of
// iterative refinement (r = b - A x from A's own CSR values, x += A^-1 r): near an ill-conditioned
// operating point the plain solve leaves Newton short of its residual test. With smem set, the factor's
// values, the inverse diagonal and the work vector live in shared memory (dynamic,
// nnz_lu + 2 n doubles): every access of the column chain is then a shared-memory access
// instead of an L2 round trip. The static pivots are checked after the factorisation, off the
// chain: a pivot below tiny x its column's largest entry leaves an L entry above 1 / tiny.
__global__ void __launch_bounds__(kLuWarps * 32, 1) k_lu_factor_solve(LuDev L, const double* __restrict__ A,
                                                                      const int* __restrict__ rp,
                                                                      const int* __restrict__ col,
                                                                      const double* __restrict__ b,
                                                                      double* x, double tiny,
                                                                      int smem, int refine) {
  extern __shared__ __align__(16) double lu_dyn[];
  __shared__ volatile int prog[kLuWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double* v = smem ? lu_dyn : L.vals;
  double* dinv = smem ? lu_dyn + L.nnz_lu : L.y + L.n;
  double* y = smem ? lu_dyn + L.nnz_lu + L.n : L.y;
  if (smem == 2) {
    // the plan's index arrays too (one packed, 16-byte aligned buffer), after the values: the
    // column chain then reads every index from shared memory instead of L2
    int* sidx = reinterpret_cast<int*>(lu_dyn + lu_vals_doubles(L));
    const int4* src = reinterpret_cast<const int4*>(L.ibase);
    int4* dst = reinterpret_cast<int4*>(sidx);
    for (long long i = threadIdx.x; i < L.ilen / 4; i += blockDim.x) dst[i] = __ldg(src + i);
    L.cptr = sidx + (L.cptr - L.ibase);
    L.cdiag = sidx + (L.cdiag - L.ibase);
    L.a2lu = sidx + (L.a2lu - L.ibase);
    L.uptr = sidx + (L.uptr - L.ibase);
    L.uk = sidx + (L.uk - L.ibase);
    L.upos = sidx + (L.upos - L.ibase);
    L.mptr = sidx + (L.mptr - L.ibase);
    L.msrc = sidx + (L.msrc - L.ibase);
    L.mdst = sidx + (L.mdst - L.ibase);
    L.lrptr = sidx + (L.lrptr - L.ibase);
    L.lrcol = sidx + (L.lrcol - L.ibase);
    L.lrpos = sidx + (L.lrpos - L.ibase);
    L.urptr = sidx + (L.urptr - L.ibase);
    L.urcol = sidx + (L.urcol - L.ibase);
    L.urpos = sidx + (L.urpos - L.ibase);
    L.prow = sidx + (L.prow - L.ibase);
    L.pcol = sidx + (L.pcol - L.ibase);
    __syncthreads();
  }
  if (lane == 0) prog[w] = w;
  for (int p = threadIdx.x; p < L.nnz_lu; p += blockDim.x) v[p] = 0.0;
  __syncthreads();
  for (int e = threadIdx.x; e < L.nnz_a; e += blockDim.x) v[L.a2lu[e]] = __ldg(A + e);
  __syncthreads();
  for (int j = w; j < L.n; j += kLuWarps) {
    const int t1 = L.uptr[j + 1];
    for (int t = L.uptr[j]; t < t1; ++t) {
      const int k = L.uk[t];
      if (lane == 0) lu_wait(prog, k, L.flag);
      __syncwarp();   // orders lane 0's observation before every lane's loads of column k
      const double ukj = v[L.upos[t]];
      const int m1 = L.mptr[t + 1];
      for (int m = L.mptr[t] + lane; m < m1; m += 32)
        v[L.mdst[m]] -= v[L.msrc[m]] * ukj;
      __syncwarp();
    }
    const int pd = L.cdiag[j], p1 = L.cptr[j + 1];
    const double inv = lu_rcp(v[pd]);
    for (int p = pd + 1 + lane; p < p1; p += 32) v[p] *= inv;
    if (lane == 0) dinv[j] = inv;
    __syncwarp();
    __threadfence_block();
    if (lane == 0) prog[w] = j + kLuWarps;
  }
  __syncthreads();
  // pivot check, every column in parallel: |piv| > tiny max|L(:, j) before scaling| holds iff
  // every scaled entry is below 1 / tiny (and the pivot is finite and not zero)
  const double lim = 1.0 / tiny;
  for (int j = threadIdx.x; j < L.n; j += blockDim.x) {
    const double di = dinv[j];
    if (!isfinite(di) || di == 0.0) {
      atomicCAS(L.flag + 2, 0, j + 1);   // zero or non-finite pivot
      continue;
    }
    bool bad = false;
    for (int p = L.cdiag[j] + 1; p < L.cptr[j + 1] && !bad; ++p)
      bad = !(fabs(v[p]) < lim);
    if (bad) atomicCAS(L.flag, 0, j + 1);
  }
  lu_substitute(L, v, dinv, y, prog, b, x);
  if (!refine) return;
  __syncthreads();
  double* r = L.y + 2 * L.n;   // residual, then the correction
  for (int i = threadIdx.x; i < L.n; i += blockDim.x) {
    double s = __ldg(b + i);
    const int e1 = __ldg(rp + i + 1);
    for (int e = __ldg(rp + i); e < e1; ++e) s = fma(-__ldg(A + e), x[__ldg(col + e)], s);
    r[i] = s;
  }
  __syncthreads();
  double* d = r + L.n;
  lu_substitute(L, v, dinv, y, prog, r, d);
  __syncthreads();
  for (int i = threadIdx.x; i < L.n; i += blockDim.x) x[i] += d[i];
}

// ---- the same on every SM: one cooperative kernel ------------------------------------------
//
// When the factor does not fit in one block's shared memory it lives in global memory, and the
// single block's 32 warps spend most of their time waiting for L2 (the 256 x 256 SRAM: 75 ms per
// solve). Here the columns (rows in the substitutions) are dealt round robin to every warp of a
// co-resident grid; a warp publishes its progress in global memory (a fence, then a release
// store), waiters poll it with acquire loads, and grid barriers separate the phases. Values that
// other SMs write (the factor, the inverse diagonal, the work vectors, x) are read and written
// through L2 only (.cg), so no SM reads a stale line from its L1. All waits are bounded as in the
// single-block kernel; after one gives up, every later wait returns at once and the host reports
// the timeout.
constexpr int kLuGridBlock = 256;
constexpr int kLuGridBar = 8;   // gwork[0..1]: barrier count and generation; progress from 8

__device__ __forceinline__ int lu_ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void lu_st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool lu_gwait(const int* prog, int W, int k, int* flag) {
  long long spins = 0;
  while (lu_ld_acquire(prog + (k % W)) <= k) {
    if (*((volatile int*)(flag + 1))) return false;
    if (++spins > kLuSpinLimit) {
      atomicExch(flag + 1, 1);
      return false;
    }
  }
  return true;
}

// Bounded grid barrier (every block of the co-resident grid calls it the same number of times).
__device__ __forceinline__ void lu_grid_sync(int* bar, int* flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const int gen = lu_ld_acquire(bar + 1);
    if (atomicAdd(bar, 1) == (int)gridDim.x - 1) {
      atomicExch(bar, 0);
      __threadfence();
      lu_st_release(bar + 1, gen + 1);
    } else {
      long long spins = 0;
      while (lu_ld_acquire(bar + 1) == gen) {
        if (*((volatile int*)(flag + 1))) break;
        if (++spins > kLuSpinLimit) {
          atomicExch(flag + 1, 1);
          break;
        }
      }
    }
  }
  __syncthreads();
}

// Row-times-vector of the substitutions (as lu_row_dot), all values through L2.
__device__ __forceinline__ double lu_grow_dot(const int* __restrict__ cols, const int* __restrict__ pos,
                                              int p0, int p1, const double* v, const double* u,
                                              const int* prog, int W, int* flag, bool reversed,
                                              int n) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  if (p1 - p0 <= 4) {
    if (lane == 0)
      for (int p = p0; p < p1; ++p) {
        const int c = __ldg(cols + p);
        lu_gwait(prog, W, reversed ? n - 1 - c : c, flag);
        s = fma(__ldcg(v + __ldg(pos + p)), __ldcg(u + c), s);
      }
    return s;   // meaningful in lane 0
  }
  for (int p = p0 + lane; p < p1; p += 32) {
    const int c = __ldg(cols + p);
    lu_gwait(prog, W, reversed ? n - 1 - c : c, flag);
    s = fma(__ldcg(v + __ldg(pos + p)), __ldcg(u + c), s);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

__device__ __forceinline__ void lu_gsubstitute(const LuDev& L, const double* v, const double* dinv,
                                               double* y, int* prog, int* bar, int W, int gw,
                                               const double* b, double* x) {
  const int lane = threadIdx.x & 31;
  const int n = L.n;
  if (lane == 0) lu_st_release(prog + gw, gw);
  lu_grid_sync(bar, L.flag);
  for (int r = gw; r < n; r += W) {
    const double s = lu_grow_dot(L.lrcol, L.lrpos, __ldg(L.lrptr + r), __ldg(L.lrptr + r + 1), v,
                                 y, prog, W, L.flag, false, n);
    if (lane == 0) {
      __stcg(y + r, __ldcg(b + __ldg(L.prow + r)) - s);
      __threadfence();
      lu_st_release(prog + gw, r + W);
    }
    __syncwarp();
  }
  lu_grid_sync(bar, L.flag);
  if (lane == 0) lu_st_release(prog + gw, gw);
  lu_grid_sync(bar, L.flag);
  for (int m = gw; m < n; m += W) {
    const int r = n - 1 - m;
    const double s = lu_grow_dot(L.urcol, L.urpos, __ldg(L.urptr + r), __ldg(L.urptr + r + 1), v,
                                 y, prog, W, L.flag, true, n);
    if (lane == 0) {
      __stcg(y + r, (__ldcg(y + r) - s) * __ldcg(dinv + r));
      __threadfence();
      lu_st_release(prog + gw, m + W);
    }
    __syncwarp();
  }
  lu_grid_sync(bar, L.flag);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    __stcg(x + __ldg(L.pcol + r), __ldcg(y + r));
}

__global__ void __launch_bounds__(kLuGridBlock, 4) k_lu_factor_solve_grid(LuDev L,
                                                                       const double* __restrict__ A,
                                                                       const int* __restrict__ rp,
                                                                       const int* __restrict__ col,
                                                                       const double* __restrict__ b,
                                                                       double* x, double tiny,
                                                                       int refine) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (kLuGridBlock / 32) + (threadIdx.x >> 5);
  const int W = gridDim.x * (kLuGridBlock / 32);
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, GT = gridDim.x * blockDim.x;
  int* bar = L.gwork;
  int* prog = L.gwork + kLuGridBar;
  double* v = L.vals;
  double* y = L.y;
  double* dinv = L.y + L.n;
  if (lane == 0) lu_st_release(prog + gw, gw);
  for (int p = gt; p < L.nnz_lu; p += GT) __stcg(v + p, 0.0);
  lu_grid_sync(bar, L.flag);
  for (int e = gt; e < L.nnz_a; e += GT) __stcg(v + __ldg(L.a2lu + e), __ldg(A + e));
  lu_grid_sync(bar, L.flag);
  for (int j = gw; j < L.n; j += W) {
    const int t1 = __ldg(L.uptr + j + 1);
    for (int t = __ldg(L.uptr + j); t < t1; ++t) {
      const int k = __ldg(L.uk + t);
      if (lane == 0) lu_gwait(prog, W, k, L.flag);
      __syncwarp();   // orders lane 0's observation before every lane's loads of column k
      const double ukj = __ldcg(v + __ldg(L.upos + t));
      const int m1 = __ldg(L.mptr + t + 1);
      for (int m = __ldg(L.mptr + t) + lane; m < m1; m += 32) {
        const int d = __ldg(L.mdst + m);
        __stcg(v + d, fma(-__ldcg(v + __ldg(L.msrc + m)), ukj, __ldcg(v + d)));
      }
      __threadfence_block();
      __syncwarp();
    }
    const int pd = __ldg(L.cdiag + j), p1 = __ldg(L.cptr + j + 1);
    const double inv = lu_rcp(__ldcg(v + pd));
    for (int p = pd + 1 + lane; p < p1; p += 32) __stcg(v + p, __ldcg(v + p) * inv);
    if (lane == 0) __stcg(dinv + j, inv);
    __threadfence();
    __syncwarp();
    if (lane == 0) lu_st_release(prog + gw, j + W);
  }
  lu_grid_sync(bar, L.flag);
  const double lim = 1.0 / tiny;
  for (int j = gt; j < L.n; j += GT) {
    const double di = __ldcg(dinv + j);
    if (!isfinite(di) || di == 0.0) {
      atomicCAS(L.flag + 2, 0, j + 1);
      continue;
    }
    bool bad = false;
    for (int p = __ldg(L.cdiag + j) + 1; p < __ldg(L.cptr + j + 1) && !bad; ++p)
      bad = !(fabs(__ldcg(v + p)) < lim);
    if (bad) atomicCAS(L.flag, 0, j + 1);
  }
  lu_gsubstitute(L, v, dinv, y, prog, bar, W, gw, b, x);
  if (!refine) return;
  lu_grid_sync(bar, L.flag);
  double* r = L.y + 2 * L.n;   // residual, then the correction
  for (int i = gt; i < L.n; i += GT) {
    double s = __ldg(b + i);
    const int e1 = __ldg(rp + i + 1);
    for (int e = __ldg(rp + i); e < e1; ++e) s = fma(-__ldg(A + e), __ldcg(x + __ldg(col + e)), s);
    __stcg(r + i, s);
  }
  lu_grid_sync(bar, L.flag);
  double* d = r + L.n;
  lu_gsubstitute(L, v, dinv, y, prog, bar, W, gw, r, d);
  lu_grid_sync(bar, L.flag);
  for (int i = gt; i < L.n; i += GT) __stcg(x + i, __ldcg(x + i) + __ldcg(d + i));
}

// Blocks of the cooperative grid on the current device (0 if the query fails), cached per device.
int lu_grid_blocks() {
  static int blocks[64] = {};
  int dev = 0, nsm = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 0;
  if (dev < 64 && blocks[dev]) return blocks[dev];
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lu_factor_solve_grid, kLuGridBlock,
                                                    0) != cudaSuccess)
    return 0;
  // 1, 2 and 4 per SM measured within 5 %: the chain of dependent columns sets the time, not
  // the warps
  const int b = nsm * std::min(occ, 2);
  if (dev < 64) blocks[dev] = b;
  return b;
}

}  // namespace

size_t lu_smem_bytes(const LuDev& L) { return sizeof(double) * (size_t)lu_vals_doubles(L); }

cudaError_t launch_lu_factor_solve(const LuDev& L, const double* A, const int* rp, const int* col,
                                   const double* b, double* x, double tiny, int refine,
                                   cudaStream_t s) {
  if (L.n <= 0) return cudaSuccess;
  int dev = 0, max_optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const size_t need = lu_smem_bytes(L);
  const size_t need_idx = need + sizeof(int) * (size_t)L.ilen;
  const size_t fixed = sizeof(int) * kLuWarps;
  const int smem = (L.ibase && need_idx + fixed <= (size_t)max_optin) ? 2
                   : (need + fixed <= (size_t)max_optin ? 1 : 0);
  const size_t dyn = smem == 2 ? need_idx : (smem ? need : 0);
  const int grid = smem ? 0 : lu_grid_blocks();
  if (grid > 0 && L.gwork) {
    // the factor in global memory: the cooperative kernel over every SM (co-resident blocks,
    // or the launch fails), its barrier and progress words cleared first
    const int W = grid * (kLuGridBlock / 32);
    e = cudaMemsetAsync(L.gwork, 0, sizeof(int) * (size_t)(kLuGridBar + W), s);
    if (e != cudaSuccess) return e;
    LuDev Lc = L;
    const double* pA = A;
    const int* prp = rp;
    const int* pcol = col;
    const double* pb = b;
    double* px = x;
    void* args[] = {&Lc, &pA, &prp, &pcol, &pb, &px, &tiny, &refine};
    return cudaLaunchCooperativeKernel((const void*)k_lu_factor_solve_grid, dim3(grid),
                                       dim3(kLuGridBlock), args, 0, s);
  }
  if (smem) {
    e = cudaFuncSetAttribute(k_lu_factor_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dyn);
    if (e != cudaSuccess) return e;
  }
  k_lu_factor_solve<<<1, kLuWarps * 32, dyn, s>>>(L, A, rp, col, b, x, tiny, smem, refine);
  return cudaGetLastError();
}

int lu_grid_words() {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return kLuGridBar + 16 * nsm;   // up to 2 blocks of 8 warps per SM
}

}  // namespace eec
