// Host side of the C ABI declared in include/eec.h: netlist storage, greedy colouring (host),
// MNA pattern and scatter-map construction, device uploads, schedule dispatch, CUDA graphs,
// autotuning and the device status word.
#include <cuda_runtime.h>
// eec_newton_dc uses cuSOLVER's batched sparse QR, which the toolkit marks deprecated in favour
// of cuDSS; cuDSS is not part of the toolkit this library builds against.
#define DISABLE_CUSOLVER_DEPRECATED
#define DISABLE_CUSPARSE_DEPRECATED
#include <cusolverSp.h>
#include <cusparse.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <stdexcept>
#include <string>
#include <vector>

#include "eec_internal.h"
#include "eec_lu.h"

using namespace eec;

struct eec_ctx {
  eec_options opt{};
  std::string err;
  bool has_net = false, has_cards = false, colored = false, built = false;
  bool pattern_ready = false;  // host pattern and layout exist (device upload may be missing)
  // netlist (original device order)
  int n_nodes = 0;
  std::vector<uint8_t> fixed;
  std::vector<double> vfix;
  std::vector<int> rail;       // EEC_RAIL_MNA_BRANCH: held nodes (now free), in node order
  int n_dev = 0;
  std::vector<int> dn;
  std::vector<int8_t> type;
  std::vector<double> W, L;
  std::vector<int> mid;
  std::vector<int> rn;
  std::vector<double> rG;
  std::vector<int> sn;
  std::vector<double> sI;
  double gshunt = 0.0;
  // batch bookkeeping (n_circ == 0: not a batch)
  int n_circ = 0;
  std::vector<int> circ_node_off, circ_dev_off;
  std::vector<int> circ_row_off;
  std::vector<int64_t> circ_nnz_off;
  // cards
  int n_cards = 0;
  std::vector<double> cards;
  std::vector<CardK> cardk;
  // colouring
  std::vector<int> color;
  int C = 0;
  // pattern and layout
  int n = 0;
  long long nnz = 0;
  std::vector<int> unk, row_ptr, col, perm, color_off;
  // device state
  DevTopo d{};
  int* d_coff = nullptr;
  std::vector<void*> dmem;
  int* d_status = nullptr;  // [0] status, [1..kBarWords] grid barrier (see DevTopo::bar)
  bool params_dirty = false;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t auto_exec = nullptr;
  const void* auto_key[4] = {nullptr, nullptr, nullptr, nullptr};
  int auto_variant = -100;
  cudaGraphExec_t user_exec = nullptr;
  int tuned_variant = EEC_VARIANT_SEGREDUCE;
  int tuned_block = 0;         // block size picked by eec_autotune (used when opt.block == 0)
  int auto_block = -1;         // block size baked into the cached graph
  bool auto_ordered = true;    // evaluation launch order baked into the cached graph
  int sms = 0;
  int persist_grid = 0;
  int stamp_grid = 0;          // blocks of the one-launch colour stamp
  int stamp_mode = 0;          // colour-buffered stamp: 0 per-colour launches, 1 grid, 2 cluster
  int pipe_grid = 0;           // blocks of the pipelined colour schedule (resident blocks)
  int pipe_colors = 0;         // non-empty colours (counters of the pipelined schedule)
  long long n_stream = 0;     // items of the segmented reduction's cbuf
  // phase timing and launch counting
  bool prof = false;
  bool graph_all = false;      // eec_batch_capture_graph: every schedule replays a cached graph
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  long long prof_calls = 0;
  long long n_kernels = 0;
  long long auto_kernels = 0;  // kernel nodes of the cached graph
  long long user_kernels = 0;  // kernel nodes of the user graph
  // staging buffers of eec_eval_stamp_host (allocated on its first call)
  double* h_x = nullptr;
  double* h_A = nullptr;
  double* h_b = nullptr;
  double* h_q = nullptr;
  // chunk plan of eec_eval_stamp_host: chunk k = original devices hc_lo[k] .. hc_lo[k+1]-1, as
  // hc_nr[k] library-order ranges at d_hrbeg + hc_rb[k] with prefix sums at d_hroff + hc_ro[k]
  int host_K = 0;  // 0 = no plan yet
  std::vector<int> hc_lo, hc_rb, hc_ro, hc_nr, hc_total;
  int* d_hrbeg = nullptr;
  int* d_hroff = nullptr;
  cudaStream_t side = nullptr;   // charge copies of eec_eval_stamp_host
  cudaStream_t side2 = nullptr;  // second evaluation stream of eec_eval_stamp_host
  // launch order of the order-free evaluations: layout ranges, devices with a free source or
  // body first (eval_nr = 0: plain layout order)
  int eval_nr = 0;
  int* d_erbeg = nullptr;
  int* d_eroff = nullptr;
  bool eval_ordered = true;   // use that order (eec_autotune times both)
  // eec_newton_dc: solver handles and buffers (set up on its first call)
  cusolverSpHandle_t sp = nullptr;
  cusparseMatDescr_t sp_descr = nullptr;
  csrqrInfo_t sp_info = nullptr;
  int* d_rp = nullptr;
  int* d_col = nullptr;
  double* d_y = nullptr;
  double* d_x0 = nullptr;        // starting point, kept for the gshunt-stepping restart
  int* d_diag = nullptr;         // CSR position of the diagonal of every node row
  int* d_rail_unk = nullptr;     // unknown of every rail node (rails as MNA unknowns)
  // eec_transient: A, b and the charges and capacitive currents of two time points
  double* tr_A = nullptr;
  double* tr_b = nullptr;
  double* tr_q = nullptr;
  int newton_info[4] = {0, 0, 0, 0};   // last eec_newton_dc: solves, gshunt stages, sweeps, path
  void* sp_buf = nullptr;
  unsigned long long* d_nstats = nullptr;
  // eec_newton_dc solver 2 (sparse LU): the column order (pattern only), the plan of the last
  // analysis and its device copy (freed and replaced when a pivot degrades)
  std::vector<int> lu_order;
  LuPlan lu;
  LuDev lud{};
  bool lu_ready = false;
  int lu_analyses = 0;
  int* lu_ibuf = nullptr;       // the plan's index arrays, packed (grown, never shrunk)
  size_t lu_icap = 0;
  double* lu_dbuf = nullptr;    // factor values, work vector and inverse diagonal
  size_t lu_dcap = 0;
  int* lu_flag = nullptr;
  int* lu_gwork = nullptr;      // progress words and barrier of the multi-block LU kernel
  std::vector<cudaEvent_t> hev;  // chunk done (K) + side stream done (1) + start of the chunks (1)
};

namespace {

int fail(eec_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

// No C++ exception crosses the C ABI: every entry point runs its body inside a try block and
// reports an exception as an error code (host memory exhausted: EEC_ENOMEM). Called from the
// catch block, so the exception being handled is rethrown here to be told apart.
int abi_exception(eec_ctx* c) noexcept {
  int code = EEC_EINVAL;
  const char* msg = "internal error";
  try {
    throw;
  } catch (const std::bad_alloc&) {
    code = EEC_ENOMEM;
    msg = "out of host memory";
  } catch (const std::length_error&) {
    code = EEC_ENOMEM;
    msg = "a host array would exceed its maximum size";
  } catch (...) {
  }
  if (c) {
    try {
      c->err = msg;
    } catch (...) {
    }
  }
  return code;
}

#define CUDA_TRY(ctx, expr)                                                              \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(ctx, EEC_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));   \
  } while (0)

template <class T>
int dalloc(eec_ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, EEC_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  c->dmem.push_back(*p);
  return EEC_OK;
}

template <class T>
int dupload(eec_ctx* c, T** p, const std::vector<T>& h) {
  int rc = dalloc(c, p, h.size());
  if (rc) return rc;
  if (!h.empty()) CUDA_TRY(c, cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return EEC_OK;
}

void drop_graphs(eec_ctx* c) {
  if (c->auto_exec) cudaGraphExecDestroy(c->auto_exec);
  if (c->user_exec) cudaGraphExecDestroy(c->user_exec);
  c->auto_exec = nullptr;
  c->user_exec = nullptr;
  c->auto_variant = -100;
}

void free_topology(eec_ctx* c) {
  drop_graphs(c);
  c->h_x = c->h_A = c->h_b = c->h_q = nullptr;  // freed with the other device arrays
  c->host_K = 0;
  c->d_hrbeg = c->d_hroff = nullptr;
  c->eval_nr = 0;
  c->d_erbeg = c->d_eroff = nullptr;
  if (!c->dmem.empty() || c->sp_info) cudaDeviceSynchronize();
  if (c->sp_info) cusolverSpDestroyCsrqrInfo(c->sp_info);
  c->sp_info = nullptr;
  c->d_rp = c->d_col = nullptr;
  c->d_y = nullptr;
  c->d_x0 = nullptr;
  c->d_diag = nullptr;
  c->d_rail_unk = nullptr;
  c->tr_A = c->tr_b = c->tr_q = nullptr;   // freed with the other device arrays
  c->sp_buf = nullptr;
  c->d_nstats = nullptr;
  if (c->lu_ibuf) cudaFree(c->lu_ibuf);
  if (c->lu_dbuf) cudaFree(c->lu_dbuf);
  if (c->lu_flag) cudaFree(c->lu_flag);
  if (c->lu_gwork) cudaFree(c->lu_gwork);
  c->lu_gwork = nullptr;
  c->lu_ibuf = nullptr;
  c->lu_dbuf = nullptr;
  c->lu_flag = nullptr;
  c->lu_icap = c->lu_dcap = 0;
  c->lu_order.clear();
  c->lu = LuPlan{};
  c->lud = LuDev{};
  c->lu_ready = false;
  for (void* p : c->dmem) cudaFree(p);
  c->dmem.clear();
  int* st = c->d_status;
  c->d = DevTopo{};
  c->d_coff = nullptr;
  c->d_status = st;
  c->built = false;
}

// Pull sizes changed by eec_update_params back into the host copy before a rebuild.
int sync_params_to_host(eec_ctx* c) {
  if (!c->built || !c->params_dirty) return EEC_OK;
  // eec_update_params may have run on any stream, non-blocking ones included
  CUDA_TRY(c, cudaDeviceSynchronize());
  std::vector<double> Wp(c->n_dev), Lp(c->n_dev);
  CUDA_TRY(c, cudaMemcpy(Wp.data(), c->d.W, sizeof(double) * c->n_dev, cudaMemcpyDeviceToHost));
  CUDA_TRY(c, cudaMemcpy(Lp.data(), c->d.L, sizeof(double) * c->n_dev, cudaMemcpyDeviceToHost));
  for (int k = 0; k < c->n_dev; ++k) {
    c->W[c->perm[k]] = Wp[k];
    c->L[c->perm[k]] = Lp[k];
  }
  c->params_dirty = false;
  return EEC_OK;
}

bool conflict_node(const eec_ctx* c, int node, int term, int rule) {
  if (rule == EEC_CONFLICT_ANY_NONGROUND) return node != 0;
  if (c->fixed[node]) return false;
  if (rule == EEC_CONFLICT_WRITE_ROWS && term == 1) return false;
  return true;
}

// Device -> conflict-node lists and node -> device lists (CSR), duplicates removed per device.
void conflict_incidence(const eec_ctx* c, int rule, std::vector<int>& dev_ptr,
                        std::vector<int>& dev_node, std::vector<int>& node_ptr,
                        std::vector<int>& node_dev) {
  const int N = c->n_dev;
  dev_ptr.assign(N + 1, 0);
  dev_node.clear();
  dev_node.reserve(4 * (size_t)N);
  for (int k = 0; k < N; ++k) {
    int got[4];
    int m = 0;
    for (int t = 0; t < 4; ++t) {
      const int node = c->dn[4 * k + t];
      if (!conflict_node(c, node, t, rule)) continue;
      bool dup = false;
      for (int i = 0; i < m; ++i) dup = dup || got[i] == node;
      if (!dup) got[m++] = node;
    }
    for (int i = 0; i < m; ++i) dev_node.push_back(got[i]);
    dev_ptr[k + 1] = (int)dev_node.size();
  }
  node_ptr.assign(c->n_nodes + 1, 0);
  for (int v : dev_node) node_ptr[v + 1]++;
  for (int i = 0; i < c->n_nodes; ++i) node_ptr[i + 1] += node_ptr[i];
  node_dev.assign(dev_node.size(), 0);
  std::vector<int> fill(node_ptr.begin(), node_ptr.end() - 1);
  for (int k = 0; k < N; ++k)
    for (int p = dev_ptr[k]; p < dev_ptr[k + 1]; ++p) node_dev[fill[dev_node[p]]++] = k;
}

// Greedy colouring in `order`: mark the colours of already-coloured neighbours with the
// visiting device's id, then take the first unmarked colour.
void greedy_host(int N, const std::vector<int>& order, const std::vector<int>& dev_ptr,
                 const std::vector<int>& dev_node, const std::vector<int>& node_ptr,
                 const std::vector<int>& node_dev, std::vector<int>& col, int* n_colors) {
  col.assign(N, -1);
  std::vector<int> mark(64, -1);
  int C = 0;
  for (int i = 0; i < N; ++i) {
    const int v = order[i];
    for (int p = dev_ptr[v]; p < dev_ptr[v + 1]; ++p) {
      const int node = dev_node[p];
      for (int q = node_ptr[node]; q < node_ptr[node + 1]; ++q) {
        const int w = node_dev[q];
        const int cw = col[w];
        if (cw >= 0) {
          if (cw >= (int)mark.size()) mark.resize(2 * cw + 2, -1);
          mark[cw] = v;
        }
      }
    }
    int m = 0;
    while (m < (int)mark.size() && mark[m] == v) ++m;
    col[v] = m;
    C = std::max(C, m + 1);
  }
  *n_colors = C;
}

CardK derive_card(const double* a) {
  const double kB = 1.380649e-23, q = 1.602176634e-19, eps0 = 8.8541878128e-12;
  const double VTH0 = a[0], K1 = a[1], PHI = a[2], NFACT = a[3], U0 = a[4], UA = a[5],
               UB = a[6], VSAT = a[7], TOX = a[8], ETA0 = a[9], DELTA = a[10],
               LAMBDA = a[11], LREF = a[12], JS = a[13], HDIF = a[14], CGSO = a[15],
               CGDO = a[16], XPART = a[17], D1 = a[18], GMIN = a[19], TEMP = a[20];
  CardK k{};
  const double Vt = kB * TEMP / q;
  const double Cox = 3.9 * eps0 / TOX;
  k.VTH0 = VTH0; k.K1 = K1; k.PHI = PHI; k.sqrtPHI = std::sqrt(PHI);
  k.Vt = Vt; k.inv_Vt = 1.0 / Vt; k.twoVt = 2.0 * Vt;
  k.nVt = NFACT * Vt; k.inv_nVt = 1.0 / k.nVt;
  k.UA = UA; k.UB = UB; k.ETA0 = ETA0;
  k.DELTA = DELTA; k.twoDELTA = 2.0 * DELTA; k.fourDELTA = 4.0 * DELTA;
  k.fourD1sq = 4.0 * D1 * D1; k.twoD1sq = 2.0 * D1 * D1;
  k.XPART = XPART; k.GMIN = GMIN;
  k.halfK1 = 0.5 * K1; k.Vthc = VTH0 - K1 * k.sqrtPHI; k.twoUB = 2.0 * UB; k.XPm = XPART - 0.5;
  k.U0Cox = U0 * Cox; k.twoVSAT_U0 = 2.0 * VSAT / U0; k.LAMBDA_LREF = LAMBDA * LREF;
  k.JS_HDIF = JS * HDIF; k.Cox = Cox; k.CGSO = CGSO; k.CGDO = CGDO;
  return k;
}

bool valid_card(const double* a) {
  for (int i = 0; i < EEC_CARD_LEN; ++i)
    if (!std::isfinite(a[i])) return false;
  // TOX, U0, VSAT, NFACT, PHI, TEMP must be positive; the rest non-negative except VTH0/ETA0.
  return a[8] > 0 && a[4] > 0 && a[7] > 0 && a[3] > 0 && a[2] > 0 && a[20] > 0 && a[1] >= 0 &&
         a[10] >= 0 && a[18] >= 0 && a[13] >= 0 && a[14] >= 0;
}

// The segmented reduction's gather plan for entries with gcnt[e] contributions each. Per window
// of kGatherWin entries, the light ones (< kHeavy contributions) are sorted by their count (ties
// in entry order) and dealt to groups of 32, each stored column-major: the gather then adds one
// item of 32 entries per instruction, and each entry's sum keeps the serial order. A group takes
// 32 x (1 + its largest count) items. Heavy entries' runs follow, contiguous. ghead[e] = item of
// entry e's linear part (its contributions follow 32 items apart when light, 1 when heavy);
// gwoff[w (kGatherGroups + 1) + g] = first item of group g of window w, then the window's end;
// gloc[w kGatherWin + slot] = entry - w kGatherWin or 0xffff; gheavy = {entry, first item, items,
// 0}. False when the plan would exceed 2^31 - 1 items.
static_assert(EEC_GATHER_WINDOW == kGatherWin && EEC_GATHER_HEAVY == kHeavy,
              "the gather plan's constants in eec.h");
bool gather_plan(const std::vector<int>& gcnt, std::vector<long long>& ghead,
                 std::vector<int>& gwoff, std::vector<unsigned short>& gloc,
                 std::vector<int4>& gheavy, long long& n_items) {
  const long long E = (long long)gcnt.size();
  const long long n_win = (E + kGatherWin - 1) / kGatherWin;
  ghead.assign(E, 0);
  gwoff.assign((size_t)n_win * (kGatherGroups + 1), 0);
  gloc.assign((size_t)n_win * kGatherWin, 0xffff);
  gheavy.clear();
  long long gitems = 0;
  std::vector<long long> order;
  for (long long w = 0; w < n_win; ++w) {
    const long long e0 = w * kGatherWin, e1 = std::min(E, e0 + kGatherWin);
    order.clear();
    for (long long e = e0; e < e1; ++e)
      if (gcnt[e] < kHeavy) order.push_back(e);
    std::stable_sort(order.begin(), order.end(),
                     [&](long long x, long long y) { return gcnt[x] < gcnt[y]; });
    for (int g = 0; g < kGatherGroups; ++g) {
      gwoff[(size_t)w * (kGatherGroups + 1) + g] = (int)std::min(gitems, 0x7fffffffLL);
      const size_t s0 = (size_t)32 * g, s1 = std::min(order.size(), s0 + 32);
      if (s0 >= s1) continue;
      for (size_t i = s0; i < s1; ++i) {
        ghead[order[i]] = gitems + (long long)(i - s0);
        gloc[(size_t)w * kGatherWin + i] = (unsigned short)(order[i] - e0);
      }
      gitems += 32LL * (1 + gcnt[order[s1 - 1]]);   // the group's rows: its largest run
    }
    gwoff[(size_t)w * (kGatherGroups + 1) + kGatherGroups] = (int)std::min(gitems, 0x7fffffffLL);
  }
  for (long long e = 0; e < E; ++e) {
    if (gcnt[e] < kHeavy) continue;
    ghead[e] = gitems;
    if (gitems + 1 + gcnt[e] <= 0x7fffffffLL)
      gheavy.push_back(make_int4((int)e, (int)gitems, 1 + gcnt[e], 0));
    gitems += 1 + gcnt[e];
  }
  n_items = gitems;
  return gitems <= 0x7fffffffLL;
}

int ensure_buf(eec_ctx* c) {
  if (c->d.buf) return EEC_OK;
  return dalloc(c, &c->d.buf, (size_t)kNContrib * c->n_dev);
}

// The segmented reduction's buffer: every entry's run, its linear part written here once (the
// evaluation overwrites only the contributions).
int ensure_cbuf(eec_ctx* c) {
  if (c->d.cbuf) return EEC_OK;
  int rc = dalloc(c, &c->d.cbuf, std::max<size_t>((size_t)c->n_stream, 1));
  if (rc) return rc;
  CUDA_TRY(c, cudaMemset(c->d.cbuf, 0, std::max<size_t>((size_t)c->n_stream, 1) * sizeof(double)));
  CUDA_TRY(c, launch_gather_init(c->d, 0));
  CUDA_TRY(c, cudaStreamSynchronize(0));
  return EEC_OK;
}

int ensure_gv(eec_ctx* c) {
  if (c->d.gv) return EEC_OK;
  return dalloc(c, &c->d.gv, (size_t)4 * c->n_dev);
}

// Next free profiling event (pool grows on demand, reset by eec_profile_read).
cudaEvent_t prof_event(eec_ctx* c) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_used++];
}

void prof_mark(eec_ctx* c, cudaStream_t s) {
  if (!c->prof) return;
  cudaEvent_t e = prof_event(c);
  if (e) cudaEventRecord(e, s);
}

bool variant_needs_colors(int v) {
  return v == EEC_VARIANT_COLOR_FUSED || v == EEC_VARIANT_PERSISTENT ||
         v == EEC_VARIANT_COLOR_BUFFERED || v == EEC_VARIANT_COLOR_PIPELINED;
}

// Enqueue one evaluate-and-stamp with schedule v on stream s. Returns the number of kernels
// launched in *nk. With profiling on, four events bracket the phases init | evaluate | stamp.
// Every device once, in the cost order of eval_nr (order-free modes only).
cudaError_t launch_eval_all(eec_ctx* c, int mode, const double* x, double* A, double* b,
                            double* q, int blk, int dbg, cudaStream_t s, bool pdl = false) {
  if (c->eval_nr >= 2 && c->eval_ordered)
    return launch_eval_ranges(c->d, mode, c->d_erbeg, c->d_eroff, c->eval_nr, c->n_dev, x, A, b,
                              q, blk, dbg, s, pdl);
  return launch_eval(c->d, mode, 0, c->n_dev, x, A, b, q, blk, dbg, s, pdl);
}

int run_variant(eec_ctx* c, int v, const double* x, double* A, double* b, double* q,
                cudaStream_t s, long long* nk) {
  const DevTopo& T = c->d;
  const int dbg = c->opt.debug_checks ? 1 : 0;
  const int blk = c->opt.block ? c->opt.block : c->tuned_block;
  *nk = 0;
  if (variant_needs_colors(v) && !c->colored)
    return fail(c, EEC_ESTATE, "colour schedules need eec_color before eec_build_scatter");
  auto init_Ab = [&]() -> int {
    CUDA_TRY(c, launch_init_lin(T, A, b, s));
    ++*nk;
    return EEC_OK;
  };
  int rc;
  if (v == EEC_VARIANT_COLOR_BUFFERED && (rc = ensure_buf(c))) return rc;
  if (v == EEC_VARIANT_SEGREDUCE && (rc = ensure_cbuf(c))) return rc;
  prof_mark(c, s);
  switch (v) {
    case EEC_VARIANT_COLOR_FUSED:
      if ((rc = init_Ab())) return rc;
      prof_mark(c, s);
      for (int k = 0; k < c->C; ++k) {
        if (c->color_off[k + 1] <= c->color_off[k]) continue;
        CUDA_TRY(c, launch_eval(T, MODE_RMW, c->color_off[k], c->color_off[k + 1], x, A, b, q,
                                blk, dbg, s));
        ++*nk;
      }
      prof_mark(c, s);
      break;
    case EEC_VARIANT_PERSISTENT:
      if ((rc = init_Ab())) return rc;
      prof_mark(c, s);
      CUDA_TRY(c, launch_persistent(T, c->d_coff, c->C, x, A, b, q, blk, c->persist_grid, dbg, s));
      ++*nk;
      prof_mark(c, s);
      break;
    case EEC_VARIANT_ATOMIC:
      if ((rc = init_Ab())) return rc;
      prof_mark(c, s);
      // overlaps the initialisation unless a profiling event sits between the two launches
      CUDA_TRY(c, launch_eval_all(c, MODE_ATOMIC, x, A, b, q, blk, dbg, s, !c->prof));
      *nk += c->n_dev > 0;
      prof_mark(c, s);
      break;
    case EEC_VARIANT_SEGREDUCE:
      prof_mark(c, s);
      CUDA_TRY(c, launch_eval_all(c, MODE_SORTED, x, A, b, q, blk, dbg, s));
      prof_mark(c, s);
      CUDA_TRY(c, launch_gather(c->d, A, b, s));
      *nk += (c->n_dev > 0) + (c->nnz + c->n > 0);
      break;
    case EEC_VARIANT_COLOR_BUFFERED:
      if ((rc = init_Ab())) return rc;
      prof_mark(c, s);
      CUDA_TRY(c, launch_eval_all(c, MODE_BUFFER, x, A, b, q, blk, dbg, s));
      prof_mark(c, s);
      *nk += c->n_dev > 0;
      // colour order: one launch per colour for a few colours, else one co-resident launch
      // that steps through the colours with a grid barrier
      if (c->stamp_mode == 2) {
        CUDA_TRY(c, launch_stamp_cluster(c->d, c->d_coff, c->C, A, b, s));
        ++*nk;
      } else if (c->stamp_mode == 1) {
        CUDA_TRY(c, launch_stamp_persistent(c->d, c->d_coff, c->C, A, b, c->stamp_grid, s));
        ++*nk;
      } else {
        for (int k = 0; k < c->C; ++k) {
          if (c->color_off[k + 1] <= c->color_off[k]) continue;
          CUDA_TRY(c, launch_stamp_buffer(c->d, c->color_off[k], c->color_off[k + 1], A, b, blk, s));
          ++*nk;
        }
      }
      break;
    case EEC_VARIANT_COLOR_PIPELINED:
      // evaluation and colour-ordered stamping in one launch; it overlaps the initialisation
      // unless a profiling event sits between the two launches (then the phase split is
      // init | evaluate-and-stamp, and the stamp phase is empty)
      if ((rc = init_Ab())) return rc;
      prof_mark(c, s);
      CUDA_TRY(c, launch_color_pipe(T, c->pipe_colors, x, A, b, q, c->pipe_grid, dbg, s));
      *nk += c->d.n_pitem > 0;
      prof_mark(c, s);
      break;
    default:
      return fail(c, EEC_EINVAL, "unknown variant");
  }
  prof_mark(c, s);
  if (c->prof) ++c->prof_calls;
  return EEC_OK;
}

// Chunk plan of eec_eval_stamp_host. The layout is colour-major, then grouped by card and
// polarity, then in original order, so library positions form maximal runs of increasing
// original index; within a run, the devices of an original-index span are contiguous. Chunk k
// is a span of original indices, one range per run. Chunk sizes halve from one chunk to the
// next (weights 2^(K-1-k)): the charges of a chunk (32 B per device at the link's 189 GB/s)
// copy out in less time than the next chunk, half its size, takes to evaluate (about 0.41 ns
// per device), and the last chunk, whose charges go out after the evaluation together with A
// and b, is the smallest. K = opt.host_chunks, or by size: 4 from 2^18 devices, 3 from 2^17,
// 2 from 2^16, else 1; 1 when the runs are too many (> 4096).
int host_plan(eec_ctx* c) {
  if (c->host_K) return EEC_OK;
  const int N = c->n_dev;
  int K = c->opt.host_chunks;
  if (K == 0) K = N >= (1 << 18) ? 4 : N >= (1 << 17) ? 3 : N >= (1 << 16) ? 2 : 1;
  if (K > N) K = N > 0 ? N : 1;
  std::vector<int> run{0};
  for (int p = 1; p < N; ++p)
    if (c->perm[p] < c->perm[p - 1]) run.push_back(p);
  run.push_back(N);
  if (run.size() - 1 > 4096) K = 1;
  c->hc_lo.assign(K + 1, 0);
  c->hc_rb.assign(K, 0);
  c->hc_ro.assign(K, 0);
  c->hc_nr.assign(K, 0);
  c->hc_total.assign(K, 0);
  // boundary k at the fraction (1 - 2^-k) / (1 - 2^-K) of the devices
  for (int k = 0; k < K; ++k)
    c->hc_lo[k] = (int)std::floor((double)N * (1.0 - std::ldexp(1.0, -k)) /
                                  (1.0 - std::ldexp(1.0, -K)));
  c->hc_lo[K] = N;
  std::vector<int> rbeg, roff;
  const int* P = c->perm.data();
  for (int k = 0; k < K; ++k) {
    c->hc_rb[k] = (int)rbeg.size();
    c->hc_ro[k] = (int)roff.size();
    roff.push_back(0);
    int tot = 0;
    for (size_t r = 0; r + 1 < run.size(); ++r) {
      const int p0 = (int)(std::lower_bound(P + run[r], P + run[r + 1], c->hc_lo[k]) - P);
      const int p1 = (int)(std::lower_bound(P + run[r], P + run[r + 1], c->hc_lo[k + 1]) - P);
      if (p1 > p0) {
        rbeg.push_back(p0);
        tot += p1 - p0;
        roff.push_back(tot);
      }
    }
    c->hc_nr[k] = (int)rbeg.size() - c->hc_rb[k];
    c->hc_total[k] = tot;
  }
  if (K > 1) {
    int rc;
    if ((rc = dupload(c, &c->d_hrbeg, rbeg)) || (rc = dupload(c, &c->d_hroff, roff))) return rc;
  }
  c->host_K = K;
  return EEC_OK;
}

int effective_variant(const eec_ctx* c) {
  return c->opt.variant == EEC_VARIANT_AUTO ? c->tuned_variant : c->opt.variant;
}

int capture(eec_ctx* c, int v, const double* x, double* A, double* b, double* q,
            cudaGraphExec_t* out, long long* nk) {
  if (!c->cap_stream)
    CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  // Buffers allocated lazily must exist before capture (no allocation inside a capture).
  if (v == EEC_VARIANT_COLOR_BUFFERED) {
    int rc = ensure_buf(c);
    if (rc) return rc;
  }
  if (v == EEC_VARIANT_SEGREDUCE) {
    int rc = ensure_cbuf(c);
    if (rc) return rc;
  }
  CUDA_TRY(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  const bool prof = c->prof;
  c->prof = false;  // no profiling events inside a graph
  int rc = run_variant(c, v, x, A, b, q, c->cap_stream, nk);
  c->prof = prof;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(c, EEC_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(c, EEC_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
  return EEC_OK;
}

// eval_stamp with schedule v; the per-colour schedules replay a cached CUDA graph unless
// phase timing is on.
// Host-side NVTX range (tracing): marks the enqueue of one library call in profiler timelines.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

int eval_with(eec_ctx* c, int v, const double* x, double* A, double* b, double* q,
              cudaStream_t s) {
  NvtxRange range("eec/eval_stamp");
  if (!c->prof &&
      (c->graph_all || v == EEC_VARIANT_COLOR_FUSED || v == EEC_VARIANT_COLOR_BUFFERED)) {
    const void* key[4] = {x, A, b, q};
    const int blk = c->opt.block ? c->opt.block : c->tuned_block;
    bool hit = c->auto_exec && c->auto_variant == v && c->auto_block == blk &&
               c->auto_ordered == c->eval_ordered;
    for (int i = 0; i < 4 && hit; ++i) hit = key[i] == c->auto_key[i];
    if (!hit) {
      if (c->auto_exec) cudaGraphExecDestroy(c->auto_exec);
      c->auto_exec = nullptr;
      c->auto_variant = -100;
      int rc = capture(c, v, x, A, b, q, &c->auto_exec, &c->auto_kernels);
      if (rc) return rc;
      c->auto_variant = v;
      c->auto_block = blk;
      c->auto_ordered = c->eval_ordered;
      for (int i = 0; i < 4; ++i) c->auto_key[i] = key[i];
    }
    CUDA_TRY(c, cudaGraphLaunch(c->auto_exec, s));
    c->n_kernels += c->auto_kernels;
    return EEC_OK;
  }
  long long nk = 0;
  int rc = run_variant(c, v, x, A, b, q, s, &nk);
  c->n_kernels += nk;
  return rc;
}

int check_pattern(eec_ctx* c) {
  if (!c) return EEC_EINVAL;
  if (!c->pattern_ready) return fail(c, EEC_ESTATE, "call eec_build_scatter first");
  return EEC_OK;
}

int check_built(eec_ctx* c) {
  if (!c) return EEC_EINVAL;
  if (!c->built) return fail(c, EEC_ESTATE, "call eec_build_scatter first");
  return EEC_OK;
}

int store_netlist(eec_ctx* c, int32_t n_nodes, const uint8_t* node_fixed, const double* node_vfix,
                  int32_t n_dev, const int32_t* dev_nodes, const int8_t* dev_type,
                  const double* W, const double* L, const int32_t* model_id, int32_t n_res,
                  const int32_t* res_nodes, const double* res_G, int32_t n_isrc,
                  const int32_t* isrc_nodes, const double* isrc_val, double gshunt) {
  if (n_nodes < 1 || n_dev < 0 || n_res < 0 || n_isrc < 0)
    return fail(c, EEC_EINVAL, "negative size or no ground node");
  if (!node_fixed || !node_vfix || (n_dev && (!dev_nodes || !dev_type || !W || !L || !model_id)) ||
      (n_res && (!res_nodes || !res_G)) || (n_isrc && (!isrc_nodes || !isrc_val)))
    return fail(c, EEC_EINVAL, "NULL array with nonzero size");
  if (!(gshunt >= 0.0) || !std::isfinite(gshunt)) return fail(c, EEC_EINVAL, "gshunt must be >= 0");
  for (long long i = 0; i < 4LL * n_dev; ++i)
    if (dev_nodes[i] < 0 || dev_nodes[i] >= n_nodes) return fail(c, EEC_EINVAL, "device node index out of range");
  for (long long i = 0; i < 2LL * n_res; ++i)
    if (res_nodes[i] < 0 || res_nodes[i] >= n_nodes) return fail(c, EEC_EINVAL, "resistor node index out of range");
  for (long long i = 0; i < 2LL * n_isrc; ++i)
    if (isrc_nodes[i] < 0 || isrc_nodes[i] >= n_nodes) return fail(c, EEC_EINVAL, "source node index out of range");
  for (int k = 0; k < n_dev; ++k) {
    if (dev_type[k] != 1 && dev_type[k] != -1) return fail(c, EEC_EINVAL, "dev_type must be +1 or -1");
    if (!(W[k] > 0) || !(L[k] > 0) || !std::isfinite(W[k]) || !std::isfinite(L[k]))
      return fail(c, EEC_EINVAL, "W and L must be positive and finite");
    if (model_id[k] < 0) return fail(c, EEC_EINVAL, "negative model_id");
  }
  for (int i = 0; i < n_nodes; ++i)
    if (node_fixed[i] && !std::isfinite(node_vfix[i])) return fail(c, EEC_EINVAL, "non-finite fixed voltage");
  free_topology(c);
  c->n_nodes = n_nodes;
  c->fixed.assign(node_fixed, node_fixed + n_nodes);
  for (auto& f : c->fixed) f = f ? 1 : 0;
  c->vfix.assign(node_vfix, node_vfix + n_nodes);
  c->fixed[0] = 1;
  c->vfix[0] = 0.0;
  // modified nodal analysis: a held node becomes an unknown and its source current another one
  c->rail.clear();
  if (c->opt.rail_mode == EEC_RAIL_MNA_BRANCH)
    for (int i = 1; i < n_nodes; ++i)
      if (c->fixed[i]) {
        c->rail.push_back(i);
        c->fixed[i] = 0;
      }
  c->n_dev = n_dev;
  c->dn.assign(dev_nodes, dev_nodes + 4LL * n_dev);
  c->type.assign(dev_type, dev_type + n_dev);
  c->W.assign(W, W + n_dev);
  c->L.assign(L, L + n_dev);
  c->mid.assign(model_id, model_id + n_dev);
  c->rn.assign(res_nodes, res_nodes + 2LL * n_res);
  c->rG.assign(res_G, res_G + n_res);
  c->sn.assign(isrc_nodes, isrc_nodes + 2LL * n_isrc);
  c->sI.assign(isrc_val, isrc_val + n_isrc);
  c->gshunt = gshunt;
  c->has_net = true;
  c->pattern_ready = false;
  c->colored = false;
  c->C = 0;
  c->color.clear();
  c->params_dirty = false;
  c->n_circ = 0;
  return EEC_OK;
}

}  // namespace

extern "C" {

eec_options eec_default_options(void) {
  eec_options o;
  o.variant = EEC_VARIANT_AUTO;
  o.block = 0;
  o.conflict_rule = EEC_CONFLICT_FREE_NODE;
  o.debug_checks = 0;
  o.color_stamp = 0;
  o.host_chunks = 0;
  o.rail_mode = EEC_RAIL_ELIMINATE;
  return o;
}

static int eec_create_body(eec_ctx** out, const eec_options* opt) {
  if (!out) return EEC_EINVAL;
  *out = nullptr;
  eec_ctx* c = new (std::nothrow) eec_ctx;
  if (!c) return EEC_ENOMEM;
  c->opt = opt ? *opt : eec_default_options();
  if (c->opt.variant < EEC_VARIANT_AUTO || c->opt.variant >= EEC_N_VARIANTS ||
      c->opt.conflict_rule < 0 || c->opt.conflict_rule > 2 || c->opt.host_chunks < 0 ||
      c->opt.color_stamp < 0 || c->opt.color_stamp > 3 ||
      c->opt.host_chunks > 64 || c->opt.rail_mode < 0 || c->opt.rail_mode > 1 ||
      !(c->opt.block == 0 || c->opt.block == 8 || c->opt.block == 16 ||
        (c->opt.block % 32 == 0 && c->opt.block <= 128))) {
    delete c;
    return EEC_EINVAL;
  }
  *out = c;  // no CUDA call: host-side steps work without a device
  return EEC_OK;
}
int eec_create(eec_ctx** out, const eec_options* opt) {
  try {
    return eec_create_body(out, opt);
  } catch (...) {
    return abi_exception(nullptr);
  }
}

void eec_destroy(eec_ctx* c) {
  if (!c) return;
  free_topology(c);
  if (c->d_status) cudaFree(c->d_status);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->side2) cudaStreamDestroy(c->side2);
  if (c->sp_descr) cusparseDestroyMatDescr(c->sp_descr);
  if (c->sp) cusolverSpDestroy(c->sp);
  for (cudaEvent_t e : c->hev) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  delete c;
}

const char* eec_last_error(const eec_ctx* c) { return c ? c->err.c_str() : "null context"; }

static int eec_upload_netlist_body(eec_ctx* c, int32_t n_nodes, const uint8_t* node_fixed,
                                   const double* node_vfix, int32_t n_dev, const int32_t* dev_nodes,
                                   const int8_t* dev_type, const double* W, const double* L,
                                   const int32_t* model_id, int32_t n_res, const int32_t* res_nodes,
                                   const double* res_G, int32_t n_isrc, const int32_t* isrc_nodes,
                                   const double* isrc_val, double gshunt) {
  if (!c) return EEC_EINVAL;
  return store_netlist(c, n_nodes, node_fixed, node_vfix, n_dev, dev_nodes, dev_type, W, L,
                       model_id, n_res, res_nodes, res_G, n_isrc, isrc_nodes, isrc_val, gshunt);
}
int eec_upload_netlist(eec_ctx* c, int32_t n_nodes, const uint8_t* node_fixed,
                       const double* node_vfix, int32_t n_dev, const int32_t* dev_nodes,
                       const int8_t* dev_type, const double* W, const double* L,
                       const int32_t* model_id, int32_t n_res, const int32_t* res_nodes,
                       const double* res_G, int32_t n_isrc, const int32_t* isrc_nodes,
                       const double* isrc_val, double gshunt) {
  try {
    return eec_upload_netlist_body(c, n_nodes, node_fixed, node_vfix, n_dev, dev_nodes, dev_type, W,
                                   L, model_id, n_res, res_nodes, res_G, n_isrc, isrc_nodes,
                                   isrc_val, gshunt);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_upload_batch_body(eec_ctx* c, int32_t n_circ, const eec_netlist* nets, double gshunt) {
  if (!c) return EEC_EINVAL;
  if (n_circ < 1 || !nets) return fail(c, EEC_EINVAL, "empty batch");
  if (c->opt.rail_mode != EEC_RAIL_ELIMINATE)
    return fail(c, EEC_EINVAL, "batched uploads take EEC_RAIL_ELIMINATE only");
  long long nodes = 1, devs = 0, res = 0, src = 0;
  for (int k = 0; k < n_circ; ++k) {
    const eec_netlist& m = nets[k];
    if (m.n_nodes < 1 || m.n_dev < 0 || m.n_res < 0 || m.n_isrc < 0)
      return fail(c, EEC_EINVAL, "bad circuit sizes");
    nodes += m.n_nodes - 1;
    devs += m.n_dev;
    res += m.n_res;
    src += m.n_isrc;
  }
  if (nodes > 0x7fffffffLL || devs > 0x7fffffffLL) return fail(c, EEC_EINVAL, "batch too large");
  std::vector<uint8_t> fx(nodes, 0);
  std::vector<double> vf(nodes, 0.0);
  std::vector<int32_t> dnod(4 * devs), rnod(2 * res), snod(2 * src), mids(devs);
  std::vector<int8_t> typ(devs);
  std::vector<double> Wv(devs), Lv(devs), rg(res), sv(src);
  std::vector<int> node_off(n_circ + 1), dev_off(n_circ + 1);
  fx[0] = 1;
  long long nn = 1, nd = 0, nr = 0, ns = 0;
  for (int k = 0; k < n_circ; ++k) {
    const eec_netlist& m = nets[k];
    if (!m.node_fixed || !m.node_vfix || (m.n_dev && (!m.dev_nodes || !m.dev_type || !m.W || !m.L || !m.model_id)) ||
        (m.n_res && (!m.res_nodes || !m.res_G)) || (m.n_isrc && (!m.isrc_nodes || !m.isrc_val)))
      return fail(c, EEC_EINVAL, "NULL array in batch circuit");
    node_off[k] = (int)nn;
    dev_off[k] = (int)nd;
    auto mapn = [&](int v) -> int32_t { return v <= 0 ? 0 : (int32_t)(nn + v - 1); };
    for (int i = 1; i < m.n_nodes; ++i) {
      fx[nn + i - 1] = m.node_fixed[i] ? 1 : 0;
      vf[nn + i - 1] = m.node_vfix[i];
    }
    for (long long i = 0; i < 4LL * m.n_dev; ++i) {
      if (m.dev_nodes[i] < 0 || m.dev_nodes[i] >= m.n_nodes) return fail(c, EEC_EINVAL, "batch device node out of range");
      dnod[4 * nd + i] = mapn(m.dev_nodes[i]);
    }
    for (int i = 0; i < m.n_dev; ++i) {
      typ[nd + i] = m.dev_type[i];
      Wv[nd + i] = m.W[i];
      Lv[nd + i] = m.L[i];
      mids[nd + i] = m.model_id[i];
    }
    for (long long i = 0; i < 2LL * m.n_res; ++i) {
      if (m.res_nodes[i] < 0 || m.res_nodes[i] >= m.n_nodes) return fail(c, EEC_EINVAL, "batch resistor node out of range");
      rnod[2 * nr + i] = mapn(m.res_nodes[i]);
    }
    for (int i = 0; i < m.n_res; ++i) rg[nr + i] = m.res_G[i];
    for (long long i = 0; i < 2LL * m.n_isrc; ++i) {
      if (m.isrc_nodes[i] < 0 || m.isrc_nodes[i] >= m.n_nodes) return fail(c, EEC_EINVAL, "batch source node out of range");
      snod[2 * ns + i] = mapn(m.isrc_nodes[i]);
    }
    for (int i = 0; i < m.n_isrc; ++i) sv[ns + i] = m.isrc_val[i];
    nn += m.n_nodes - 1;
    nd += m.n_dev;
    nr += m.n_res;
    ns += m.n_isrc;
  }
  node_off[n_circ] = (int)nn;
  dev_off[n_circ] = (int)nd;
  int rc = store_netlist(c, (int32_t)nodes, fx.data(), vf.data(), (int32_t)devs, dnod.data(),
                         typ.data(), Wv.data(), Lv.data(), mids.data(), (int32_t)res,
                         rnod.data(), rg.data(), (int32_t)src, snod.data(), sv.data(), gshunt);
  if (rc) return rc;
  c->n_circ = n_circ;
  c->circ_node_off = node_off;
  c->circ_dev_off = dev_off;
  return EEC_OK;
}
int eec_upload_batch(eec_ctx* c, int32_t n_circ, const eec_netlist* nets, double gshunt) {
  try {
    return eec_upload_batch_body(c, n_circ, nets, gshunt);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_set_model_cards_body(eec_ctx* c, int32_t n_cards, const double* cards) {
  if (!c) return EEC_EINVAL;
  if (n_cards < 1 || !cards) return fail(c, EEC_EINVAL, "need at least one card");
  for (int i = 0; i < n_cards; ++i)
    if (!valid_card(cards + (size_t)i * EEC_CARD_LEN)) return fail(c, EEC_EINVAL, "invalid model card " + std::to_string(i));
  c->n_cards = n_cards;
  c->cards.assign(cards, cards + (size_t)n_cards * EEC_CARD_LEN);
  c->cardk.resize(n_cards);
  for (int i = 0; i < n_cards; ++i) c->cardk[i] = derive_card(cards + (size_t)i * EEC_CARD_LEN);
  c->has_cards = true;
  if (c->built) {
    int rc = sync_params_to_host(c);
    if (rc) return rc;
    free_topology(c);
  }
  return EEC_OK;
}
int eec_set_model_cards(eec_ctx* c, int32_t n_cards, const double* cards) {
  try {
    return eec_set_model_cards_body(c, n_cards, cards);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_color_body(eec_ctx* c, const int32_t* order, int32_t algo, int32_t* colors_out,
                          int32_t* n_colors) {
  if (!c) return EEC_EINVAL;
  if (!c->has_net) return fail(c, EEC_ESTATE, "upload a netlist first");
  if (!n_colors) return fail(c, EEC_EINVAL, "n_colors is NULL");
  if (algo < EEC_COLOR_GREEDY_SEQ || algo > EEC_COLOR_JP_RANDOM) return fail(c, EEC_EINVAL, "unknown colouring algorithm");
  const int N = c->n_dev;
  std::vector<int> ord(N);
  if (order) {
    std::vector<char> seen(N, 0);
    for (int i = 0; i < N; ++i) {
      const int v = order[i];
      if (v < 0 || v >= N || seen[v]) return fail(c, EEC_EINVAL, "order is not a permutation");
      seen[v] = 1;
      ord[i] = v;
    }
  } else {
    std::iota(ord.begin(), ord.end(), 0);
  }
  int rc = sync_params_to_host(c);
  if (rc) return rc;
  std::vector<int> dev_ptr, dev_node, node_ptr, node_dev;
  conflict_incidence(c, c->opt.conflict_rule, dev_ptr, dev_node, node_ptr, node_dev);
  std::vector<int> col;
  int C = 0;
  if (algo == EEC_COLOR_GREEDY_SEQ) {
    greedy_host(N, ord, dev_ptr, dev_node, node_ptr, node_dev, col, &C);
  } else {
    std::vector<uint32_t> prio(N);
    if (algo == EEC_COLOR_JP_INDEX) {
      for (int i = 0; i < N; ++i) prio[ord[i]] = (uint32_t)(N - i);
    } else {
      // Hashed priorities (SplitMix64 finaliser of the device index), ties broken by index.
      std::vector<std::pair<uint64_t, int>> h(N);
      for (int v = 0; v < N; ++v) {
        uint64_t z = (uint64_t)v + 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        h[v] = {z ^ (z >> 31), v};
      }
      std::sort(h.begin(), h.end());
      for (int i = 0; i < N; ++i) prio[h[i].second] = (uint32_t)(i + 1);
    }
    std::string err;
    rc = jp_color(N, node_ptr, node_dev, dev_ptr, dev_node, prio, col, &C, err);
    if (rc) return fail(c, rc, err);
  }
  free_topology(c);
  c->pattern_ready = false;
  c->color = col;
  c->C = C;
  c->colored = true;
  if (colors_out) std::copy(col.begin(), col.end(), colors_out);
  *n_colors = C;
  return EEC_OK;
}
int eec_color(eec_ctx* c, const int32_t* order, int32_t algo, int32_t* colors_out,
              int32_t* n_colors) {
  try {
    return eec_color_body(c, order, algo, colors_out, n_colors);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_build_scatter_body(eec_ctx* c, int32_t* n_unknowns, int64_t* nnz_out) {
  if (!c) return EEC_EINVAL;
  if (!c->has_net || !c->has_cards) return fail(c, EEC_ESTATE, "upload a netlist and model cards first");
  for (int k = 0; k < c->n_dev; ++k)
    if (c->mid[k] >= c->n_cards) return fail(c, EEC_EINVAL, "model_id beyond the card table");
  int rc = sync_params_to_host(c);
  if (rc) return rc;
  free_topology(c);
  const int N = c->n_dev;
  // unknowns and the fixed-voltage table
  c->unk.assign(c->n_nodes, -1);
  std::vector<int> fidx(c->n_nodes, -1);
  std::vector<double> vtab;
  int n = 0;
  for (int i = 0; i < c->n_nodes; ++i) {
    if (c->fixed[i]) {
      fidx[i] = (int)vtab.size();
      vtab.push_back(c->vfix[i]);
    } else {
      c->unk[i] = n++;
    }
  }
  const int n_node_unk = n;
  std::vector<int> jr(c->rail.size());   // source-current unknown of each rail
  for (size_t r = 0; r < c->rail.size(); ++r) jr[r] = n++;
  c->n = n;
  // pattern: sorted unique (row, col) keys
  std::vector<uint64_t> keys;
  keys.reserve((size_t)n + 4 * c->rG.size() + 9 * (size_t)N);
  auto key = [](int r, int cc) { return ((uint64_t)(uint32_t)r << 32) | (uint32_t)cc; };
  for (int i = 0; i < n; ++i) keys.push_back(key(i, i));
  for (size_t r = 0; r < c->rG.size(); ++r) {
    const int a = c->unk[c->rn[2 * r]], bb = c->unk[c->rn[2 * r + 1]];
    if (a >= 0 && bb >= 0) { keys.push_back(key(a, bb)); keys.push_back(key(bb, a)); }
  }
  for (int k = 0; k < N; ++k)
    for (int t = 0; t < 4; ++t) {
      const int a = c->unk[c->dn[4 * k + t]];
      if (a < 0) continue;
      for (int u = 0; u < 4; ++u) {
        const int bb = c->unk[c->dn[4 * k + u]];
        if (bb >= 0) keys.push_back(key(a, bb));
      }
    }
  for (size_t r = 0; r < c->rail.size(); ++r) {
    keys.push_back(key(c->unk[c->rail[r]], jr[r]));
    keys.push_back(key(jr[r], c->unk[c->rail[r]]));
  }
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  c->nnz = (long long)keys.size();
  if (c->nnz > 0x7fffffffLL) return fail(c, EEC_EINVAL, "nnz beyond 2^31 is not supported");
  c->row_ptr.assign(n + 1, 0);
  c->col.resize(keys.size());
  for (size_t i = 0; i < keys.size(); ++i) {
    c->row_ptr[(keys[i] >> 32) + 1]++;
    c->col[i] = (int)(keys[i] & 0xffffffffu);
  }
  for (int i = 0; i < n; ++i) c->row_ptr[i + 1] += c->row_ptr[i];
  auto find = [&](int r, int cc) -> int {
    const int* b0 = c->col.data() + c->row_ptr[r];
    const int* b1 = c->col.data() + c->row_ptr[r + 1];
    const int* p = std::lower_bound(b0, b1, cc);
    return (int)(p - c->col.data());
  };
  // layout: colour-major, then card/polarity, then original index
  std::vector<long long> sk(N);
  for (int k = 0; k < N; ++k) {
    const long long colr = c->colored ? c->color[k] : 0;
    const long long sbf = (c->fixed[c->dn[4 * k + 2]] && c->fixed[c->dn[4 * k + 3]]) ? 1 : 0;
    const long long meta = ((long long)c->mid[k] << 2) | (sbf << 1) | (c->type[k] < 0 ? 1 : 0);
    sk[k] = (colr << 32) | meta;
  }
  c->perm.resize(N);
  std::iota(c->perm.begin(), c->perm.end(), 0);
  std::stable_sort(c->perm.begin(), c->perm.end(), [&](int a, int bb) { return sk[a] < sk[bb]; });
  std::vector<int> pos_of(N);
  for (int p = 0; p < N; ++p) pos_of[c->perm[p]] = p;
  const int C = c->colored ? c->C : 1;
  c->color_off.assign(C + 1, 0);
  for (int k = 0; k < N; ++k) c->color_off[(c->colored ? c->color[k] : 0) + 1]++;
  for (int i = 0; i < C; ++i) c->color_off[i + 1] += c->color_off[i];
  // per-position arrays
  std::vector<int4> tidx(N);
  std::vector<int> meta(N), slot((size_t)kNSlot * N, -1), slot_g((size_t)4 * N, -1);
  std::vector<double> Wp(N), Lp(N);
  const int rows_t[3] = {0, 2, 3};
  for (int p = 0; p < N; ++p) {
    const int k = c->perm[p];
    int ti[4];
    for (int t = 0; t < 4; ++t) {
      const int node = c->dn[4 * k + t];
      ti[t] = c->unk[node] >= 0 ? c->unk[node] : ~fidx[node];
    }
    tidx[p] = make_int4(ti[0], ti[1], ti[2], ti[3]);
    const int sbf = (c->fixed[c->dn[4 * k + 2]] && c->fixed[c->dn[4 * k + 3]]) ? 1 : 0;
    meta[p] = (c->mid[k] << 2) | (sbf << 1) | (c->type[k] < 0 ? 1 : 0);
    Wp[p] = c->W[k];
    Lp[p] = c->L[k];
    for (int r = 0; r < 3; ++r) {
      if (ti[rows_t[r]] < 0) continue;
      for (int u = 0; u < 4; ++u)
        if (ti[u] >= 0) slot[(size_t)(4 * r + u) * N + p] = find(ti[rows_t[r]], ti[u]);
    }
    if (ti[1] >= 0)
      for (int u = 0; u < 4; ++u)
        if (ti[u] >= 0) slot_g[(size_t)u * N + p] = find(ti[1], ti[u]);
  }
  // linear part, summed in the natural element order: gshunt, resistors, current sources, then
  // the voltage sources of the rails (modified nodal analysis only)
  std::vector<double> Alin(c->nnz, 0.0), blin(n, 0.0);
  for (int i = 0; i < n_node_unk; ++i) Alin[find(i, i)] += c->gshunt;
  for (size_t r = 0; r < c->rG.size(); ++r) {
    const int ni = c->rn[2 * r], nj = c->rn[2 * r + 1];
    const int a = c->unk[ni], bb = c->unk[nj];
    const double G = c->rG[r];
    if (a >= 0) {
      Alin[find(a, a)] += G;
      if (bb >= 0) Alin[find(a, bb)] -= G;
      else blin[a] += G * c->vfix[nj];
    }
    if (bb >= 0) {
      Alin[find(bb, bb)] += G;
      if (a >= 0) Alin[find(bb, a)] -= G;
      else blin[bb] += G * c->vfix[ni];
    }
  }
  for (size_t s = 0; s < c->sI.size(); ++s) {
    const int a = c->unk[c->sn[2 * s]], bb = c->unk[c->sn[2 * s + 1]];
    if (a >= 0) blin[a] -= c->sI[s];
    if (bb >= 0) blin[bb] += c->sI[s];
  }
  for (size_t r = 0; r < c->rail.size(); ++r) {
    const int a = c->unk[c->rail[r]];
    Alin[find(a, jr[r])] += 1.0;     // KCL at the rail: the source current leaves the node
    Alin[find(jr[r], a)] += 1.0;     // source equation: v_rail = its voltage
    blin[jr[r]] += c->vfix[c->rail[r]];
  }
  // segmented-reduction map: contributions per entry, then the gather plan (gather_plan)
  const long long E = c->nnz + n;
  std::vector<int> gcnt(E, 0);
  for (int k = 0; k < N; ++k) {
    const int p = pos_of[k];
    const int4 t4 = tidx[p];
    const int ti[4] = {t4.x, t4.y, t4.z, t4.w};
    for (int r = 0; r < 3; ++r) {
      const int row = ti[rows_t[r]];
      if (row < 0) continue;
      for (int u = 0; u < 4; ++u) {
        const int s = slot[(size_t)(4 * r + u) * N + p];
        if (s >= 0) gcnt[s]++;
      }
      gcnt[c->nnz + row]++;
    }
  }
  std::vector<long long> ghead;
  std::vector<int> gwoff;
  std::vector<unsigned short> gloc;
  std::vector<int4> gheavy;
  if (!gather_plan(gcnt, ghead, gwoff, gloc, gheavy, c->n_stream))
    return fail(c, EEC_EINVAL, "too many contributions");
  const long long n_win = (long long)gwoff.size() / (kGatherGroups + 1);
  // position in cbuf of every contribution (j, p): the evaluation writes it there
  if ((long long)N * kNContrib > 0x7fffffffLL) return fail(c, EEC_EINVAL, "too many devices");
  std::vector<int> gpos((size_t)kNContrib * N, -1);
  {
    std::vector<long long> fill(E);   // next item of entry e, and the step between its items
    for (long long e = 0; e < E; ++e) fill[e] = ghead[e] + (gcnt[e] < kHeavy ? 32 : 1);
    for (int k = 0; k < N; ++k) {
      const int p = pos_of[k];
      const int4 t4 = tidx[p];
      const int ti[4] = {t4.x, t4.y, t4.z, t4.w};
      for (int r = 0; r < 3; ++r) {
        const int row = ti[rows_t[r]];
        if (row < 0) continue;
        for (int u = 0; u < 4; ++u) {
          const int s = slot[(size_t)(4 * r + u) * N + p];
          if (s >= 0) {
            gpos[(size_t)(4 * r + u) * N + p] = (int)fill[s];
            fill[s] += gcnt[s] < kHeavy ? 32 : 1;
          }
        }
        const long long eb = c->nnz + row;
        gpos[(size_t)(kNSlot + r) * N + p] = (int)fill[eb];
        fill[eb] += gcnt[eb] < kHeavy ? 32 : 1;
      }
    }
  }
  // backward incidence: unknown -> (terminal, position) in original device order
  std::vector<int> iptr(n + 1, 0);
  for (int k = 0; k < N; ++k)
    for (int t = 0; t < 4; ++t) {
      const int a = c->unk[c->dn[4 * k + t]];
      if (a >= 0) iptr[a + 1]++;
    }
  for (int i = 0; i < n; ++i) iptr[i + 1] += iptr[i];
  std::vector<int> isrc(iptr[n]);
  {
    std::vector<int> fill(iptr.begin(), iptr.end() - 1);
    for (int k = 0; k < N; ++k)
      for (int t = 0; t < 4; ++t) {
        const int a = c->unk[c->dn[4 * k + t]];
        if (a >= 0) isrc[fill[a]++] = t * N + pos_of[k];
      }
  }
  std::vector<int> ilight, iheavy;
  for (int u = 0; u < n; ++u) {
    if (iptr[u + 1] - iptr[u] >= kHeavy) iheavy.push_back(u);
    else ilight.push_back(u);
  }
  // batch offsets
  if (c->n_circ > 0) {
    c->circ_row_off.assign(c->n_circ + 1, 0);
    c->circ_nnz_off.assign(c->n_circ + 1, 0);
    int u = 0;
    for (int k = 0; k < c->n_circ; ++k) {
      c->circ_row_off[k] = u;
      for (int i = c->circ_node_off[k]; i < c->circ_node_off[k + 1]; ++i)
        if (c->unk[i] >= 0) ++u;
    }
    c->circ_row_off[c->n_circ] = u;
    for (int k = 0; k <= c->n_circ; ++k) c->circ_nnz_off[k] = c->row_ptr[c->circ_row_off[k]];
  }
  c->pattern_ready = true;
  if (n_unknowns) *n_unknowns = n;
  if (nnz_out) *nnz_out = c->nnz;
  // device part
  if (!c->d_status) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaError_t e = cudaGetLastError();
      return fail(c, EEC_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    CUDA_TRY(c, cudaMalloc(&c->d_status, (1 + kBarWords) * sizeof(int)));
    CUDA_TRY(c, cudaMemset(c->d_status, 0, (1 + kBarWords) * sizeof(int)));
    // the fixed scratch of eec_eval_stamp_bwd_noalloc: resolved here, at set-up, so that its
    // module (and the array) is resident on this device before that entry point's first call
    CUDA_TRY(c, noalloc_setup());
  }
  DevTopo& d = c->d;
  d.N = N;
  d.n = n;
  d.nnz = c->nnz;
  d.n_win = (int)n_win;
  d.n_heavy = (int)gheavy.size();
  d.n_inc_light = (int)ilight.size();
  d.n_inc_heavy = (int)iheavy.size();
  std::vector<int> orig(c->perm.begin(), c->perm.end());
  if ((rc = dupload(c, &d.tidx, tidx)) || (rc = dupload(c, &d.meta, meta)) ||
      (rc = dupload(c, &d.orig, orig)) || (rc = dupload(c, &d.slot, slot)) ||
      (rc = dupload(c, &d.slot_g, slot_g)) ||
      (rc = dupload(c, &d.W, Wp)) || (rc = dupload(c, &d.L, Lp)) ||
      (rc = dalloc(c, &d.prm, (size_t)kNPrm * N)) || (rc = dalloc(c, &d.bodyk, (size_t)kNBody * N)) ||
      (rc = dupload(c, &d.vfix, vtab)) ||
      (rc = dupload(c, &d.cards, c->cardk)) || (rc = dupload(c, &d.Alin, Alin)) ||
      (rc = dupload(c, &d.blin, blin)) || (rc = dupload(c, &d.gat_woff, gwoff)) || (rc = dupload(c, &d.gat_loc, gloc)) ||
      (rc = dupload(c, &d.gat_pos, gpos)) ||
      (rc = dupload(c, &d.gat_heavy, gheavy)) || (rc = dupload(c, &d.inc_ptr, iptr)) ||
      (rc = dupload(c, &d.inc_light, ilight)) || (rc = dupload(c, &d.inc_heavy, iheavy)) ||
      (rc = dupload(c, &d.inc_src, isrc)) || (rc = dupload(c, &c->d_coff, c->color_off))) {
    free_topology(c);
    return rc;
  }
  d.status = c->d_status;
  d.bar = reinterpret_cast<unsigned*>(c->d_status + 1);
  CUDA_TRY(c, launch_params(d, 0));
  CUDA_TRY(c, cudaDeviceSynchronize());
  const int bps = persistent_max_blocks_per_sm(0, false);
  const int bpsq = persistent_max_blocks_per_sm(0, true);
  c->persist_grid = std::max(1, std::min(std::min(bps, bpsq), 1)) * c->sms;   // one block per SM
  // The library streams of eec_eval_stamp_host, created here rather than at its first call:
  // streams are spread over the device's hardware work queues in creation order, and one
  // created after many others (a framework's stream pool) can share the queue of the caller's
  // stream, which serialises the spans that are meant to overlap (measured: 251 -> 283 us)
  if (!c->side) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  if (!c->side2) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking));
  // enough 256-thread blocks for the largest colour, within one co-resident wave (fewer blocks
  // make each barrier cheaper)
  int maxcol = 0;
  for (int k = 0; k < c->C; ++k) maxcol = std::max(maxcol, c->color_off[k + 1] - c->color_off[k]);
  const int sbps = stamp_persistent_max_blocks_per_sm();
  c->stamp_grid = sbps > 0 ? std::max(1, std::min(sbps * c->sms, (maxcol + 255) / 256)) : 0;
  // Colour-buffered stamp: pick the cheapest of per-colour launches (about 4-8 us per colour on
  // GB300), one grid with a grid barrier (3-9 us per colour) and one 8-block cluster with the
  // hardware cluster barrier (1-2 us per colour, plus a round per 4,096 devices of a colour),
  // from the colour sizes; the constants below are conservative for the cluster.
  {
    const double nt = (double)stamp_cluster_threads();
    double t_launch = 0.0, t_grid = 0.0, t_cluster = 0.0;
    for (int k = 0; k < c->C; ++k) {
      const double sz = c->color_off[k + 1] - c->color_off[k];
      t_launch += 8.0;
      t_grid += 7.0 + 2.0 * std::ceil(sz / (256.0 * std::max(1, c->stamp_grid)));
      t_cluster += 0.5 + 2.0 * std::ceil(sz / nt);
    }
    c->stamp_mode = 0;
    double best = t_launch;
    if (c->stamp_grid > 0 && t_grid < best) { best = t_grid; c->stamp_mode = 1; }
    if (t_cluster < best) c->stamp_mode = 2;
    if (c->opt.color_stamp == 1) c->stamp_mode = 0;
    if (c->opt.color_stamp == 2 && c->stamp_grid > 0) c->stamp_mode = 1;
    if (c->opt.color_stamp == 3) c->stamp_mode = 2;
  }
  // Work items of the pipelined colour schedule: the non-empty colours in order, each cut into
  // items of up to kPipeItem positions; every item carries its colour's index among the
  // non-empty colours and the number of items of the colour before it (what it waits for).
  if (c->colored) {
    std::vector<int4> items;
    int j = -1, prev_items = 0, cur_items = 0;
    for (int k = 0; k < c->C; ++k) {
      const int b0 = c->color_off[k], b1 = c->color_off[k + 1];
      if (b1 <= b0) continue;
      if (j >= 0) prev_items = cur_items;
      ++j;
      cur_items = 0;
      for (int p = b0; p < b1; p += kPipeItem) {
        items.push_back(make_int4(p, std::min(p + kPipeItem, b1), j, j > 0 ? prev_items : 0));
        ++cur_items;
      }
    }
    c->pipe_colors = j + 1;
    if ((rc = dupload(c, &d.pitem, items)) ||
        (rc = dalloc(c, &d.pipe, (size_t)kPipeHdr + c->pipe_colors)))
      return rc;
    CUDA_TRY(c, cudaMemset(d.pipe, 0, sizeof(unsigned) * (kPipeHdr + c->pipe_colors)));
    d.n_pitem = (int)items.size();
    c->pipe_grid = std::max(1, color_pipe_max_blocks_per_sm()) * c->sms;
  } else {
    d.n_pitem = 0;
    c->pipe_colors = 0;
  }
  // Launch order of the order-free evaluations: devices with a free source or body (the body
  // effect, the source junction and the vbs chain are evaluated per call) before those with both
  // held, so that the last partial wave of blocks holds the cheaper devices.
  {
    std::vector<int> rb, ro{0};
    for (int want = 0; want < 2; ++want) {
      for (int p = 0; p < N;) {
        const int f = (meta[p] >> 1) & 1;
        int e = p + 1;
        while (e < N && ((meta[e] >> 1) & 1) == f) ++e;
        if (f == want) {
          rb.push_back(p);
          ro.push_back(ro.back() + (e - p));
        }
        p = e;
      }
    }
    c->eval_nr = 0;
    // already in that order when every free-source run precedes every held one
    bool sorted = true;
    for (size_t i = 1; i < rb.size(); ++i) sorted = sorted && rb[i] > rb[i - 1];
    if (rb.size() >= 2 && rb.size() <= 4096 && !sorted) {
      if ((rc = dupload(c, &c->d_erbeg, rb)) || (rc = dupload(c, &c->d_eroff, ro))) return rc;
      c->eval_nr = (int)rb.size();
    }
  }
  c->built = true;
  return EEC_OK;
}
int eec_build_scatter(eec_ctx* c, int32_t* n_unknowns, int64_t* nnz_out) {
  try {
    return eec_build_scatter_body(c, n_unknowns, nnz_out);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_verify_coloring_body(const eec_ctx* cc, int32_t with_gate_rows) {
  eec_ctx* c = const_cast<eec_ctx*>(cc);
  int rc = check_pattern(c);
  if (rc) return rc;
  if (!c->colored) return fail(c, EEC_ESTATE, "not coloured");
  // Within a colour, every written A entry and b row must belong to one device: mark each row
  // with the last (colour, device) that wrote it, visiting the devices colour by colour (the
  // layout order), so that two writers of one row in one colour are visited one after the
  // other. A device writes rows of its free terminals d, s, b (and g when with_gate_rows);
  // every entry it writes lies in one of those rows, so disjoint row sets imply disjoint entry
  // sets.
  std::vector<long long> owner(c->n, -1);
  for (int p = 0; p < c->n_dev; ++p) {
    const int k = c->perm[p];
    const long long tag = (long long)c->color[k] * c->n_dev + k;
    int seen[4];
    int m = 0;
    for (int t = 0; t < 4; ++t) {
      if (t == 1 && !with_gate_rows) continue;
      const int row = c->unk[c->dn[4 * k + t]];
      if (row < 0) continue;
      bool dup = false;
      for (int i = 0; i < m; ++i) dup = dup || seen[i] == row;
      if (dup) continue;
      seen[m++] = row;
      const long long prev = owner[row];
      if (prev >= 0 && prev / c->n_dev == c->color[k])
        return fail(c, EEC_EINVAL, "devices " + std::to_string(prev % c->n_dev) + " and " +
                                       std::to_string(k) + " share colour " +
                                       std::to_string(c->color[k]) + " and write row " +
                                       std::to_string(row));
      owner[row] = tag;
    }
  }
  return EEC_OK;
}
int eec_verify_coloring(const eec_ctx* cc, int32_t with_gate_rows) {
  try {
    return eec_verify_coloring_body(cc, with_gate_rows);
  } catch (...) {
    return abi_exception(const_cast<eec_ctx*>(cc));
  }
}

static int eec_get_pattern_body(const eec_ctx* cc, int32_t* row_ptr, int32_t* col_idx, int32_t* unk_of_node) {
  eec_ctx* c = const_cast<eec_ctx*>(cc);
  int rc = check_pattern(c);
  if (rc) return rc;
  if (row_ptr) std::copy(c->row_ptr.begin(), c->row_ptr.end(), row_ptr);
  if (col_idx) std::copy(c->col.begin(), c->col.end(), col_idx);
  if (unk_of_node) std::copy(c->unk.begin(), c->unk.end(), unk_of_node);
  return EEC_OK;
}
int eec_get_pattern(const eec_ctx* cc, int32_t* row_ptr, int32_t* col_idx, int32_t* unk_of_node) {
  try {
    return eec_get_pattern_body(cc, row_ptr, col_idx, unk_of_node);
  } catch (...) {
    return abi_exception(const_cast<eec_ctx*>(cc));
  }
}

static int eec_get_color_offsets_body(const eec_ctx* cc, int32_t* off) {
  eec_ctx* c = const_cast<eec_ctx*>(cc);
  int rc = check_pattern(c);
  if (rc) return rc;
  if (!c->colored) return fail(c, EEC_ESTATE, "not coloured");
  if (!off) return fail(c, EEC_EINVAL, "off is NULL");
  std::copy(c->color_off.begin(), c->color_off.end(), off);
  return EEC_OK;
}
int eec_get_color_offsets(const eec_ctx* cc, int32_t* off) {
  try {
    return eec_get_color_offsets_body(cc, off);
  } catch (...) {
    return abi_exception(const_cast<eec_ctx*>(cc));
  }
}

static int eec_get_sizes_body(const eec_ctx* cc, int32_t* n_dev, int32_t* n_unknowns, int64_t* nnz,
                              int32_t* n_colors) {
  eec_ctx* c = const_cast<eec_ctx*>(cc);
  int rc = check_pattern(c);
  if (rc) return rc;
  if (n_dev) *n_dev = c->n_dev;
  if (n_unknowns) *n_unknowns = c->n;
  if (nnz) *nnz = c->nnz;
  if (n_colors) *n_colors = c->colored ? c->C : 0;
  return EEC_OK;
}
int eec_get_sizes(const eec_ctx* cc, int32_t* n_dev, int32_t* n_unknowns, int64_t* nnz,
                  int32_t* n_colors) {
  try {
    return eec_get_sizes_body(cc, n_dev, n_unknowns, nnz, n_colors);
  } catch (...) {
    return abi_exception(const_cast<eec_ctx*>(cc));
  }
}

static int eec_get_batch_offsets_body(const eec_ctx* cc, int32_t* row_off, int64_t* nnz_off, int32_t* dev_off) {
  eec_ctx* c = const_cast<eec_ctx*>(cc);
  int rc = check_pattern(c);
  if (rc) return rc;
  if (c->n_circ == 0) return fail(c, EEC_ESTATE, "context was not uploaded as a batch");
  if (row_off) std::copy(c->circ_row_off.begin(), c->circ_row_off.end(), row_off);
  if (nnz_off) std::copy(c->circ_nnz_off.begin(), c->circ_nnz_off.end(), nnz_off);
  if (dev_off) std::copy(c->circ_dev_off.begin(), c->circ_dev_off.end(), dev_off);
  return EEC_OK;
}
int eec_get_batch_offsets(const eec_ctx* cc, int32_t* row_off, int64_t* nnz_off, int32_t* dev_off) {
  try {
    return eec_get_batch_offsets_body(cc, row_off, nnz_off, dev_off);
  } catch (...) {
    return abi_exception(const_cast<eec_ctx*>(cc));
  }
}

static int eec_update_params_body(eec_ctx* c, const double* W_dev, const double* L_dev, void* stream) {
  int rc = check_built(c);
  if (rc) return rc;
  if (!W_dev || !L_dev) return fail(c, EEC_EINVAL, "NULL W or L");
  CUDA_TRY(c, launch_update_params(c->d, W_dev, L_dev, static_cast<cudaStream_t>(stream)));
  c->params_dirty = true;
  return EEC_OK;
}
int eec_update_params(eec_ctx* c, const double* W_dev, const double* L_dev, void* stream) {
  try {
    return eec_update_params_body(c, W_dev, L_dev, stream);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_set_variant_body(eec_ctx* c, int32_t v) {
  if (!c) return EEC_EINVAL;
  if (v < EEC_VARIANT_AUTO || v >= EEC_N_VARIANTS) return fail(c, EEC_EINVAL, "unknown variant");
  c->opt.variant = v;
  return EEC_OK;
}
int eec_set_variant(eec_ctx* c, int32_t v) {
  try {
    return eec_set_variant_body(c, v);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_set_eval_order_body(eec_ctx* c, int32_t cost_order) {
  if (!c) return EEC_EINVAL;
  if (cost_order != 0 && cost_order != 1) return fail(c, EEC_EINVAL, "cost_order must be 0 or 1");
  c->eval_ordered = cost_order == 1;
  return EEC_OK;
}
int eec_set_eval_order(eec_ctx* c, int32_t cost_order) {
  try {
    return eec_set_eval_order_body(c, cost_order);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_get_variant_body(const eec_ctx* c, int32_t* v) {
  if (!c || !v) return EEC_EINVAL;
  *v = effective_variant(c);
  return EEC_OK;
}
int eec_get_variant(const eec_ctx* c, int32_t* v) {
  try {
    return eec_get_variant_body(c, v);
  } catch (...) {
    return abi_exception(const_cast<eec_ctx*>(c));
  }
}

static int eec_eval_stamp_body(eec_ctx* c, const double* x, double* A, double* b, double* q, void* stream) {
  int rc = check_built(c);
  if (rc) return rc;
  if (!x || !A || !b) return fail(c, EEC_EINVAL, "NULL x, A or b");
  return eval_with(c, effective_variant(c), x, A, b, q, static_cast<cudaStream_t>(stream));
}
int eec_eval_stamp(eec_ctx* c, const double* x, double* A, double* b, double* q, void* stream) {
  try {
    return eec_eval_stamp_body(c, x, A, b, q, stream);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_eval_stamp_host_body(eec_ctx* c, const double* x_host, double* A_host, double* b_host,
                                    double* q_host, void* stream) {
  NvtxRange range("eec/eval_stamp_host");
  int rc = check_built(c);
  if (rc) return rc;
  if (!x_host || !A_host || !b_host) return fail(c, EEC_EINVAL, "NULL x, A or b");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!c->h_x) {
    if ((rc = dalloc(c, &c->h_x, c->n)) || (rc = dalloc(c, &c->h_A, c->nnz)) ||
        (rc = dalloc(c, &c->h_b, c->n)))
      return rc;
  }
  if (q_host && !c->h_q && (rc = dalloc(c, &c->h_q, (size_t)4 * c->n_dev))) return rc;
  const int v = effective_variant(c);
  // The charges go out chunk by chunk while later chunks are still evaluated: only the
  // order-free schedules can take a chunk of original device indices in one launch.
  int K = 1;
  if (q_host && !c->prof && (v == EEC_VARIANT_ATOMIC || v == EEC_VARIANT_SEGREDUCE)) {
    if ((rc = host_plan(c))) return rc;
    K = c->host_K;
  }
  CUDA_TRY(c, cudaMemcpyAsync(c->h_x, x_host, sizeof(double) * c->n, cudaMemcpyHostToDevice, s));
  if (K <= 1) {
    if ((rc = eval_with(c, v, c->h_x, c->h_A, c->h_b, q_host ? c->h_q : nullptr, s))) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(A_host, c->h_A, sizeof(double) * c->nnz, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaMemcpyAsync(b_host, c->h_b, sizeof(double) * c->n, cudaMemcpyDeviceToHost, s));
    if (q_host)
      CUDA_TRY(c, cudaMemcpyAsync(q_host, c->h_q, sizeof(double) * 4 * c->n_dev,
                                  cudaMemcpyDeviceToHost, s));
    return EEC_OK;
  }
  if (!c->side) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  if (!c->side2) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking));
  while ((int)c->hev.size() < K + 2) {
    cudaEvent_t e = nullptr;
    CUDA_TRY(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c->hev.push_back(e);
  }
  const int dbg = c->opt.debug_checks ? 1 : 0;
  const int blk = c->opt.block ? c->opt.block : c->tuned_block;
  int mode = MODE_ATOMIC;
  if (v == EEC_VARIANT_ATOMIC) {
    CUDA_TRY(c, launch_init_lin(c->d, c->h_A, c->h_b, s));
    ++c->n_kernels;
  } else {
    if ((rc = ensure_cbuf(c))) return rc;
    mode = MODE_SORTED;
  }
  // Every launch first, then the copies (a copy to pageable memory returns only when done).
  // The chunks alternate between two streams: launched one after the other on one stream, each
  // would end in a partial wave (the last warps' dependent FP64 chain, several microseconds)
  // with the SMs idle; on two streams the next chunk's blocks take the SMs the previous chunk
  // frees. Blocks are dispatched in launch order, so the chunks still finish in order.
  CUDA_TRY(c, cudaEventRecord(c->hev[K + 1], s));
  CUDA_TRY(c, cudaStreamWaitEvent(c->side2, c->hev[K + 1], 0));
  for (int k = 0; k < K; ++k) {
    cudaStream_t sk = (k & 1) ? c->side2 : s;
    CUDA_TRY(c, launch_eval_ranges(c->d, mode, c->d_hrbeg + c->hc_rb[k], c->d_hroff + c->hc_ro[k],
                                   c->hc_nr[k], c->hc_total[k], c->h_x, c->h_A, c->h_b, c->h_q,
                                   blk, dbg, sk));
    c->n_kernels += c->hc_total[k] > 0;
    CUDA_TRY(c, cudaEventRecord(c->hev[k], sk));
  }
  // the stream of the call waits for the chunks of the second stream (the last one suffices)
  const int last_odd = ((K - 1) & 1) ? K - 1 : K - 2;
  if (last_odd >= 1) CUDA_TRY(c, cudaStreamWaitEvent(s, c->hev[last_odd], 0));
  if (mode == MODE_SORTED) {
    CUDA_TRY(c, launch_gather(c->d, c->h_A, c->h_b, s));
    c->n_kernels += (c->nnz + c->n > 0);
  }
  const size_t N = (size_t)c->n_dev;
  for (int k = 0; k < K; ++k) {
    CUDA_TRY(c, cudaStreamWaitEvent(c->side, c->hev[k], 0));
    const size_t lo = (size_t)c->hc_lo[k], cnt = (size_t)(c->hc_lo[k + 1] - c->hc_lo[k]);
    if (!cnt) continue;
    // the chunk's span of each of the four terminal rows, as one strided copy
    CUDA_TRY(c, cudaMemcpy2DAsync(q_host + lo, sizeof(double) * N, c->h_q + lo, sizeof(double) * N,
                                  sizeof(double) * cnt, 4, cudaMemcpyDeviceToHost, c->side));
  }
  CUDA_TRY(c, cudaMemcpyAsync(A_host, c->h_A, sizeof(double) * c->nnz, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(c, cudaMemcpyAsync(b_host, c->h_b, sizeof(double) * c->n, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(c, cudaEventRecord(c->hev[K], c->side));
  CUDA_TRY(c, cudaStreamWaitEvent(s, c->hev[K], 0));
  return EEC_OK;
}
int eec_eval_stamp_host(eec_ctx* c, const double* x_host, double* A_host, double* b_host,
                        double* q_host, void* stream) {
  try {
    return eec_eval_stamp_host_body(c, x_host, A_host, b_host, q_host, stream);
  } catch (...) {
    return abi_exception(c);
  }
}

// Solver state of eec_newton_dc, on its first call: the pattern on the device, the sparse QR's
// analysis (reused by every later factorisation: the pattern never changes) and its workspace.
}  // extern "C" (C++ helpers of eec_newton_dc's solvers)

namespace {

// Arrays every solver of eec_newton_dc uses: the pattern on the device, the solution y, the
// starting point, the diagonal positions and the norms.
int newton_common(eec_ctx* c) {
  if (c->d_rp) return EEC_OK;
  const int n_node = c->n - (int)c->rail.size();
  std::vector<int> diag(n_node);
  for (int i = 0; i < n_node; ++i)
    diag[i] = (int)(std::lower_bound(c->col.begin() + c->row_ptr[i],
                                     c->col.begin() + c->row_ptr[i + 1], i) - c->col.begin());
  std::vector<int> rail_unk(c->rail.size());
  for (size_t r = 0; r < c->rail.size(); ++r) rail_unk[r] = c->unk[c->rail[r]];
  int rc;
  if ((rc = dupload(c, &c->d_rp, c->row_ptr)) || (rc = dupload(c, &c->d_col, c->col)) ||
      (rc = dalloc(c, &c->d_y, c->n)) || (rc = dalloc(c, &c->d_x0, c->n)) ||
      (rc = dupload(c, &c->d_diag, diag)) || (rc = dalloc(c, &c->d_nstats, 4)) ||
      (!rail_unk.empty() && (rc = dupload(c, &c->d_rail_unk, rail_unk))))
    return rc;
  return EEC_OK;
}

// Solver 2: analyse A (device values of the current iterate) on the host -- the column order
// once per pattern, the pivots and the plan from one factorisation -- and upload the plan into
// the context's two LU buffers (one for the index arrays, packed, one for the values; both kept
// and reused by later analyses, grown only when a plan needs more room).
int lu_prepare(eec_ctx* c, const double* A, cudaStream_t s) {
  std::vector<double> a(c->nnz);
  CUDA_TRY(c, cudaMemcpyAsync(a.data(), A, sizeof(double) * c->nnz, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(c, cudaStreamSynchronize(s));
  if (c->lu_order.empty() && !lu_min_degree_order(c->n, c->row_ptr, c->col, c->lu_order))
    return fail(c, EEC_ENOMEM, "sparse LU: the elimination graph of this pattern would exceed " +
                                   std::to_string(lu_entry_budget(c->nnz)) +
                                   " entries: too much fill for a direct solve");
  LuPlan P;
  std::string err;
  int rc = lu_analyze(c->n, c->row_ptr, c->col, a, c->lu_order, P, err);
  if (rc) return fail(c, rc, err);
  const std::vector<int>* parts[] = {&P.cptr, &P.cdiag, &P.a2lu, &P.uptr, &P.uk, &P.upos,
                                     &P.mptr, &P.msrc, &P.mdst, &P.lrptr, &P.lrcol, &P.lrpos,
                                     &P.urptr, &P.urcol, &P.urpos, &P.prow, &P.pcol};
  constexpr int kParts = sizeof(parts) / sizeof(parts[0]);
  std::vector<int> packed;
  size_t off[kParts];
  for (int k = 0; k < kParts; ++k) {
    off[k] = packed.size();
    packed.insert(packed.end(), parts[k]->begin(), parts[k]->end());
    packed.resize((packed.size() + 3) & ~(size_t)3);   // 16-byte aligned starts
  }
  const size_t nd = (size_t)P.cptr[P.n] + 4 * (size_t)P.n;
  c->lu_ready = false;
  if (packed.size() > c->lu_icap) {
    if (c->lu_ibuf) cudaFree(c->lu_ibuf);
    c->lu_ibuf = nullptr;
    c->lu_icap = 0;
    if (cudaMalloc(&c->lu_ibuf, sizeof(int) * (packed.size() + packed.size() / 2)) != cudaSuccess)
      return fail(c, EEC_ENOMEM, "sparse LU: out of memory");
    c->lu_icap = packed.size() + packed.size() / 2;
  }
  if (nd > c->lu_dcap) {
    if (c->lu_dbuf) cudaFree(c->lu_dbuf);
    c->lu_dbuf = nullptr;
    c->lu_dcap = 0;
    if (cudaMalloc(&c->lu_dbuf, sizeof(double) * (nd + nd / 2)) != cudaSuccess)
      return fail(c, EEC_ENOMEM, "sparse LU: out of memory");
    c->lu_dcap = nd + nd / 2;
  }
  if (!c->lu_flag && cudaMalloc(&c->lu_flag, 3 * sizeof(int)) != cudaSuccess)
    return fail(c, EEC_ENOMEM, "sparse LU: out of memory");
  if (!c->lu_gwork) {
    const int words = lu_grid_words();
    if (words > 0 && cudaMalloc(&c->lu_gwork, sizeof(int) * (size_t)words) != cudaSuccess)
      return fail(c, EEC_ENOMEM, "sparse LU: out of memory");
  }
  CUDA_TRY(c, cudaMemcpyAsync(c->lu_ibuf, packed.data(), sizeof(int) * packed.size(),
                              cudaMemcpyHostToDevice, s));
  CUDA_TRY(c, cudaStreamSynchronize(s));   // the host vector dies with this call
  LuDev d{};
  d.n = P.n;
  d.nnz_lu = P.cptr[P.n];
  d.nnz_a = (int)P.a2lu.size();
  const int** dst[] = {&d.cptr, &d.cdiag, &d.a2lu, &d.uptr, &d.uk, &d.upos, &d.mptr, &d.msrc,
                       &d.mdst, &d.lrptr, &d.lrcol, &d.lrpos, &d.urptr, &d.urcol, &d.urpos,
                       &d.prow, &d.pcol};
  for (int k = 0; k < kParts; ++k) *dst[k] = c->lu_ibuf + off[k];
  d.vals = c->lu_dbuf;
  d.y = d.vals + d.nnz_lu;
  d.flag = c->lu_flag;
  d.gwork = c->lu_gwork;
  d.ibase = c->lu_ibuf;
  d.ilen = (long long)packed.size();
  c->lu = std::move(P);
  c->lud = d;
  c->lu_ready = true;
  ++c->lu_analyses;
  return EEC_OK;
}

// Solver 2: factor A on the fixed plan and solve A y = b; analyses again
// (once) when a pivot has fallen below kLuTiny of the largest entry of its column's L part --
// the static pivots no longer make a stable factorisation of this matrix. The unrefined solves
// (Newton steps above 1 mV, where the step is clipped and only its direction counts) accept
// growth up to 1 / kLuTinyFar: a host analysis of a large matrix costs far more than a solve,
// and the bias moves the pivots' sizes on almost every early iteration.
constexpr double kLuTiny = 1e-4;   // a fresh analysis keeps scaled L entries <= 1e3 (kLuDiagPref)
constexpr double kLuTinyFar = 1e-10;
int lu_factor_solve(eec_ctx* c, const double* A, const double* b, double* y, int refine,
                    cudaStream_t s) {
  int rc;
  if (!c->lu_ready && (rc = lu_prepare(c, A, s))) return rc;
  for (int attempt = 0; attempt < 2; ++attempt) {
    CUDA_TRY(c, cudaMemsetAsync(c->lud.flag, 0, 3 * sizeof(int), s));
    CUDA_TRY(c, launch_lu_factor_solve(c->lud, A, c->d_rp, c->d_col, b, y,
                                       refine ? kLuTiny : kLuTinyFar, refine, s));
    c->n_kernels += 1;
    int fl[3] = {0, 0, 0};
    CUDA_TRY(c, cudaMemcpyAsync(fl, c->lud.flag, sizeof fl, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    if (fl[1]) return fail(c, EEC_ETIMEOUT, "sparse LU: a device wait ran past its limit");
    // growth beyond the bound: the pivots of the plan no longer suit this matrix -- analyse it
    // and factor again; growth left after a fresh analysis (rounding of a nearly singular
    // matrix in the GPU's update order) is accepted: the Newton step's own tests judge it
    if ((!fl[0] || attempt == 1) && !fl[2]) return EEC_OK;
    if (attempt == 0 && (rc = lu_prepare(c, A, s))) return rc;
  }
  return fail(c, EEC_ENUMERIC, "sparse LU: a zero or non-finite pivot (singular or non-finite matrix)");
}

}  // namespace

extern "C" {

int newton_setup(eec_ctx* c, const double* A) {
  int rc0 = newton_common(c);
  if (rc0) return rc0;
  if (c->sp_info) return EEC_OK;
  if (!c->sp && cusolverSpCreate(&c->sp) != CUSOLVER_STATUS_SUCCESS)
    return fail(c, EEC_ECUDA, "cusolverSpCreate failed");
  if (!c->sp_descr) {
    if (cusparseCreateMatDescr(&c->sp_descr) != CUSPARSE_STATUS_SUCCESS)
      return fail(c, EEC_ECUDA, "cusparseCreateMatDescr failed");
    cusparseSetMatType(c->sp_descr, CUSPARSE_MATRIX_TYPE_GENERAL);
    cusparseSetMatIndexBase(c->sp_descr, CUSPARSE_INDEX_BASE_ZERO);
  }
  int rc;
  csrqrInfo_t info = nullptr;
  if (cusolverSpCreateCsrqrInfo(&info) != CUSOLVER_STATUS_SUCCESS)
    return fail(c, EEC_ECUDA, "cusolverSpCreateCsrqrInfo failed");
  const int n = c->n, nnz = (int)c->nnz;
  size_t internal = 0, work = 0;
  if (cusolverSpXcsrqrAnalysisBatched(c->sp, n, n, nnz, c->sp_descr, c->d_rp, c->d_col, info) !=
          CUSOLVER_STATUS_SUCCESS ||
      cusolverSpDcsrqrBufferInfoBatched(c->sp, n, n, nnz, c->sp_descr, A, c->d_rp, c->d_col, 1,
                                        info, &internal, &work) != CUSOLVER_STATUS_SUCCESS) {
    cusolverSpDestroyCsrqrInfo(info);
    return fail(c, EEC_ECUDA, "sparse QR analysis failed");
  }
  size_t fb = 0, tb = 0;
  CUDA_TRY(c, cudaMemGetInfo(&fb, &tb));
  if (internal + work > fb / 2) {
    cusolverSpDestroyCsrqrInfo(info);
    return fail(c, EEC_ENOMEM, "sparse QR factor needs " + std::to_string(internal + work) +
                                   " bytes (no fill-reducing order): too large for this netlist");
  }
  char* buf = nullptr;
  if ((rc = dalloc(c, &buf, std::max<size_t>(work, 1)))) {
    cusolverSpDestroyCsrqrInfo(info);
    return rc;
  }
  c->sp_buf = buf;
  c->sp_info = info;
  return EEC_OK;
}

double bits_to_double(unsigned long long u) {
  double d;
  std::memcpy(&d, &u, sizeof d);
  return d;
}

// One damped Newton run from x with g_extra added to the diagonal of every node row after each
// stamp (0: the circuit itself). Returns EEC_OK, EEC_ENOCONV (x holds the last iterate) or an
// error; *iters counts its solves.
static int eec_eval_stamp_tran_body(eec_ctx* c, const double* x, const double* q_prev,
                                    const double* i_prev, double alpha, double beta, double* A,
                                    double* b, double* q, double* icap, void* stream);

// With ta set, every iterate is stamped by the transient companion stamp (eec_eval_stamp_tran)
// instead: one implicit time step's Newton loop.
int newton_run(eec_ctx* c, double* x, double* A, double* b, int max_iter, double vstep,
               int step_rule, int solver, double tol_abs, double tol_rel, double tol_f,
               double g_extra, int* iters, cudaStream_t s, const TranArgs* ta = nullptr) {
  const int v = effective_variant(c), n = c->n, nnz = (int)c->nnz;
  const int n_node = n - (int)c->rail.size();
  int rc;
  unsigned long long hs[4];
  bool small_step = false;
  bool near = false;   // the last step moved no node by more than 1 mV
  *iters = 0;
  for (int it = 0; it <= max_iter; ++it) {
    CUDA_TRY(c, cudaMemsetAsync(c->d_nstats, 0, 4 * sizeof(unsigned long long), s));
    if (ta) {
      if ((rc = eec_eval_stamp_tran_body(c, x, ta->qprev, ta->iprev, ta->alpha, ta->beta, A, b,
                                         ta->q, ta->icap, s)))
        return rc;
    } else if ((rc = eval_with(c, v, x, A, b, nullptr, s))) {
      return rc;
    }
    if (g_extra > 0.0) {
      CUDA_TRY(c, launch_add_diag(A, c->d_diag, n_node, g_extra, s));
      ++c->n_kernels;
    }
    if (small_step) {  // the residual at this iterate decides convergence (A x - b = F(x))
      CUDA_TRY(c, launch_residual_norm(c->d_rp, c->d_col, A, x, b, n, c->d_nstats, s));
      CUDA_TRY(c, cudaMemcpyAsync(hs, c->d_nstats, sizeof hs, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(c, cudaStreamSynchronize(s));
      const double r = bits_to_double(hs[3]);
      if (!std::isfinite(r)) return fail(c, EEC_ENUMERIC, "non-finite KCL residual");
      if (r <= tol_f) return EEC_OK;
    }
    if (it == max_iter) break;
    if (solver == EEC_SOLVER_LU) {
      // refined solves once the steps are small (the converging tail, where the residual test
      // needs the solve's full accuracy); plain ones before
      if ((rc = lu_factor_solve(c, A, b, c->d_y, near ? 1 : 0, s))) return rc;
    } else if (solver == 0) {
      if (cusolverSpDcsrqrsvBatched(c->sp, n, n, nnz, c->sp_descr, A, c->d_rp, c->d_col, b,
                                    c->d_y, 1, c->sp_info, c->sp_buf) != CUSOLVER_STATUS_SUCCESS)
        return fail(c, EEC_ECUDA, "sparse QR solve failed");
    } else {
      int singular = -1;
      if (cusolverSpDcsrlsvqr(c->sp, n, nnz, c->sp_descr, A, c->d_rp, c->d_col, b, 0.0, 2,
                              c->d_y, &singular) != CUSOLVER_STATUS_SUCCESS)
        return fail(c, EEC_ECUDA, "sparse QR solve failed");
      if (singular >= 0)
        return fail(c, EEC_ENUMERIC, "singular matrix (row " + std::to_string(singular) + ")");
    }
    if (solver != EEC_SOLVER_LU) c->n_kernels += 2;
    CUDA_TRY(c, launch_newton_step(c->d_y, x, n, vstep, step_rule, c->d_nstats, s));
    CUDA_TRY(c, cudaMemcpyAsync(hs, c->d_nstats, sizeof hs, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    const double dxm = bits_to_double(hs[1]), xm = bits_to_double(hs[2]);
    if (!std::isfinite(dxm) || !std::isfinite(xm))
      return fail(c, EEC_ENUMERIC, "non-finite Newton step (singular matrix?)");
    small_step = dxm <= tol_abs + tol_rel * xm;
    near = dxm < 1e-3;
    *iters = it + 1;
  }
  return EEC_ENOCONV;
}

// Relaxation start: nonlinear Jacobi sweeps (every node to the zero of its own KCL residual,
// the others held; moves clipped to vmax) from x, in windows of 32 sweeps, until no node moved
// more than tol within a window, or the number of nodes still moving (by more than 1 mV, in a
// window's last sweep) has not fallen over the last four windows, or max_sweeps. A chain of n
// stages settles one stage per sweep (the nodes past the settled front toggle until it reaches
// them, so their count falls by one per sweep), where Newton from the same start needs the
// chain's gain to the n-th power in its linear solve; cross-coupled pairs (latches, memory
// cells) toggle together forever under Jacobi sweeps, which the count detects.
// Returns EEC_OK (settled or not: Newton takes over either way) or an error; *sweeps counts.
int relax_run(eec_ctx* c, double* x, double* A, double* b, double vmax, int max_sweeps, double tol,
              int* sweeps, cudaStream_t s) {
  const int v = effective_variant(c), n = c->n;
  const int n_rail = (int)c->rail.size(), n_node = n - n_rail;
  unsigned long long hs[4];
  std::vector<unsigned long long> moving;   // per window
  int rc;
  *sweeps = 0;
  for (int k = 0; k < max_sweeps; ++k) {
    const bool last = (k & 31) == 31 || k == max_sweeps - 1;
    if ((k & 31) == 0) CUDA_TRY(c, cudaMemsetAsync(c->d_nstats, 0, 4 * sizeof(unsigned long long), s));
    if ((rc = eval_with(c, v, x, A, b, nullptr, s))) return rc;
    CUDA_TRY(c, launch_relax_step(c->d_rp, c->d_col, A, x, b, c->d_diag, n_node, n, vmax,
                                  c->d_rail_unk, n_rail, c->d_y, c->d_nstats, last ? 1 : 0, s));
    c->n_kernels += 1 + (n_rail > 0);
    CUDA_TRY(c, cudaMemcpyAsync(x, c->d_y, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    *sweeps = k + 1;
    if (last) {
      CUDA_TRY(c, cudaMemcpyAsync(hs, c->d_nstats, sizeof hs, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(c, cudaStreamSynchronize(s));
      const double m = bits_to_double(hs[1]);
      if (!std::isfinite(m)) return fail(c, EEC_ENUMERIC, "non-finite relaxation sweep");
      if (m <= tol) return EEC_OK;
      moving.push_back(hs[0]);
      const size_t w = moving.size();
      if (w > 4 && moving[w - 1] >= moving[w - 5]) return EEC_OK;   // no progress: toggling
    }
  }
  return EEC_OK;
}

// Solver state for eec_newton_dc / eec_newton_tran / eec_transient, on their first call.
int newton_begin(eec_ctx* c, double* A, int solver, cudaStream_t s) {
  int rc;
  if (solver == EEC_SOLVER_LU) return newton_common(c);
  if ((rc = newton_setup(c, A))) return rc;
  if (cusolverSpSetStream(c->sp, s) != CUSOLVER_STATUS_SUCCESS)
    return fail(c, EEC_ECUDA, "cusolverSpSetStream failed");
  return EEC_OK;
}

bool newton_args_ok(double* x, double* A, double* b, int32_t max_iter, double vstep,
                    int32_t step_rule, int32_t solver, double tol_abs, double tol_rel,
                    double tol_f) {
  return x && A && b && max_iter >= 1 && vstep > 0.0 && step_rule >= 0 && step_rule <= 1 &&
         solver >= 0 && solver <= EEC_SOLVER_LU && tol_abs >= 0.0 && tol_rel >= 0.0 &&
         tol_f >= 0.0;
}

static int eec_newton_dc_body(eec_ctx* c, double* x, double* A, double* b, int32_t max_iter, double vstep,
                              int32_t step_rule, int32_t solver, double tol_abs, double tol_rel,
                              double tol_f, int32_t* iters_out, void* stream) {
  NvtxRange range("eec/newton_dc");
  int rc = check_built(c);
  if (rc) return rc;
  if (!newton_args_ok(x, A, b, max_iter, vstep, step_rule, solver, tol_abs, tol_rel, tol_f))
    return fail(c, EEC_EINVAL, "bad eec_newton_dc arguments");
  if (c->nnz > 0x7fffffffLL) return fail(c, EEC_EINVAL, "pattern too large for the sparse solver");
  if (iters_out) *iters_out = 0;
  for (int k = 0; k < 4; ++k) c->newton_info[k] = 0;
  if (c->n == 0) return EEC_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((rc = newton_begin(c, A, solver, s))) return rc;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_x0, x, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s));
  int its = 0, total = 0, stages = 0, sweeps = 0, path = 0;
  // gshunt stepping (the oracle's fallback, taken as there both when plain Newton runs out of
  // iterations and when a step fails: a singular matrix or a non-finite step): from x, a shunt
  // of g = 1e-3 S on every node, converge, divide g by 10 and continue from that solution down
  // to the circuit's own gshunt, then solve the circuit itself from there
  auto stepping = [&]() {
    int r = EEC_OK;
    for (double g = 1e-3; r == EEC_OK && g > c->gshunt * 1.0000001; g *= 0.1) {
      r = newton_run(c, x, A, b, max_iter, vstep, step_rule, solver, tol_abs, tol_rel, tol_f,
                     g - c->gshunt, &its, s);
      total += its;
      ++stages;
    }
    if (r == EEC_OK) {
      r = newton_run(c, x, A, b, max_iter, vstep, step_rule, solver, tol_abs, tol_rel, tol_f,
                     0.0, &its, s);
      total += its;
    }
    return r;
  };
  auto failed = [](int r) { return r == EEC_ENOCONV || r == EEC_ENUMERIC; };
  rc = newton_run(c, x, A, b, max_iter, vstep, step_rule, solver, tol_abs, tol_rel, tol_f, 0.0,
                  &its, s);
  total += its;
  if (failed(rc)) {
    path = 1;
    CUDA_TRY(c, cudaMemcpyAsync(x, c->d_x0, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s));
    rc = stepping();
  }
  if (failed(rc)) {
    // relaxation start (beyond the oracle's fallbacks): from the starting point, Jacobi sweeps
    // until the nodes settle, then Newton, then gshunt stepping from the relaxed point. Long
    // chains of gates need it: from a poor start the exact Newton step grows like the stage
    // gain to the power of the chain length and leaves the range of doubles.
    path = 2;
    CUDA_TRY(c, cudaMemcpyAsync(x, c->d_x0, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s));
    const int max_sweeps = (int)std::min<long long>(4LL * c->n + 1024, 1 << 16);
    if ((rc = relax_run(c, x, A, b, 5.0 * vstep, max_sweeps, 1e-6, &sweeps, s))) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_x0, x, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s));
    rc = newton_run(c, x, A, b, max_iter, vstep, step_rule, solver, tol_abs, tol_rel, tol_f, 0.0,
                    &its, s);
    total += its;
    if (failed(rc)) {
      path = 3;
      CUDA_TRY(c, cudaMemcpyAsync(x, c->d_x0, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s));
      rc = stepping();
    }
  }
  c->newton_info[0] = total;
  c->newton_info[1] = stages;
  c->newton_info[2] = sweeps;
  c->newton_info[3] = path;
  if (iters_out) *iters_out = total;
  if (rc == EEC_ENOCONV)
    return fail(c, EEC_ENOCONV, "no convergence within max_iter iterations (gshunt stepping "
                                "and relaxation start included)");
  return rc;
}
int eec_newton_dc(eec_ctx* c, double* x, double* A, double* b, int32_t max_iter, double vstep,
                  int32_t step_rule, int32_t solver, double tol_abs, double tol_rel,
                  double tol_f, int32_t* iters_out, void* stream) {
  try {
    return eec_newton_dc_body(c, x, A, b, max_iter, vstep, step_rule, solver, tol_abs, tol_rel,
                              tol_f, iters_out, stream);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_newton_tran_body(eec_ctx* c, double* x, const double* q_prev,
                                const double* i_prev, double alpha, double beta, double* A,
                                double* b, double* q, double* icap, int32_t max_iter,
                                double vstep, int32_t step_rule, int32_t solver, double tol_abs,
                                double tol_rel, double tol_f, int32_t* iters_out, void* stream) {
  NvtxRange range("eec/newton_tran");
  int rc = check_built(c);
  if (rc) return rc;
  if (!newton_args_ok(x, A, b, max_iter, vstep, step_rule, solver, tol_abs, tol_rel, tol_f) ||
      !q_prev || !q || !std::isfinite(alpha) || !std::isfinite(beta) || alpha < 0.0)
    return fail(c, EEC_EINVAL, "bad eec_newton_tran arguments");
  if (c->nnz > 0x7fffffffLL) return fail(c, EEC_EINVAL, "pattern too large for the sparse solver");
  if (iters_out) *iters_out = 0;
  if (c->n == 0) return EEC_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((rc = newton_begin(c, A, solver, s))) return rc;
  const TranArgs ta{q_prev, i_prev, alpha, beta, q, icap};
  int its = 0;
  rc = newton_run(c, x, A, b, max_iter, vstep, step_rule, solver, tol_abs, tol_rel, tol_f, 0.0,
                  &its, s, &ta);
  if (iters_out) *iters_out = its;
  if (rc == EEC_ENOCONV)
    return fail(c, EEC_ENOCONV, "time step: no convergence within max_iter iterations");
  return rc;
}
int eec_newton_tran(eec_ctx* c, double* x, const double* q_prev, const double* i_prev,
                    double alpha, double beta, double* A, double* b, double* q, double* icap,
                    int32_t max_iter, double vstep, int32_t step_rule, int32_t solver,
                    double tol_abs, double tol_rel, double tol_f, int32_t* iters_out,
                    void* stream) {
  try {
    return eec_newton_tran_body(c, x, q_prev, i_prev, alpha, beta, A, b, q, icap, max_iter, vstep,
                                step_rule, solver, tol_abs, tol_rel, tol_f, iters_out, stream);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_transient_body(eec_ctx* c, double* x, double h, int32_t n_steps, int32_t method,
                              double* traj, int32_t max_iter, double vstep, int32_t step_rule,
                              int32_t solver, double tol_abs, double tol_rel, double tol_f,
                              int32_t* iters_out, void* stream) {
  NvtxRange range("eec/transient");
  int rc = check_built(c);
  if (rc) return rc;
  if (!x || !(h > 0.0) || !std::isfinite(h) || n_steps < 0 || method < 0 || method > 1)
    return fail(c, EEC_EINVAL, "bad eec_transient arguments");
  if (iters_out) *iters_out = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t nq = (size_t)4 * c->n_dev;
  if ((!c->tr_A && (rc = dalloc(c, &c->tr_A, (size_t)c->nnz))) ||
      (!c->tr_b && (rc = dalloc(c, &c->tr_b, (size_t)c->n))) ||
      (!c->tr_q && (rc = dalloc(c, &c->tr_q, 4 * nq))))
    return rc;
  double* qa = c->tr_q;            // charges of the previous time point
  double* qb = c->tr_q + nq;       // charges at the iterate
  double* ia = c->tr_q + 2 * nq;   // capacitive currents of the previous time point
  double* ib = c->tr_q + 3 * nq;
  const double alpha = method == 0 ? 1.0 / h : 2.0 / h;
  const double beta = method == 0 ? 0.0 : 1.0;
  // the charges at t = 0 (the first time point's history: no current through the capacitors)
  CUDA_TRY(c, cudaMemsetAsync(c->tr_q, 0, sizeof(double) * 4 * nq, s));
  if ((rc = eec_eval_stamp_tran_body(c, x, qb, nullptr, 0.0, 0.0, c->tr_A, c->tr_b, qa, nullptr,
                                     s)))
    return rc;
  if (traj) CUDA_TRY(c, cudaMemcpyAsync(traj, x, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, s));
  int total = 0;
  for (int st = 1; st <= n_steps; ++st) {
    int its = 0;
    rc = eec_newton_tran_body(c, x, qa, ia, alpha, beta, c->tr_A, c->tr_b, qb, ib, max_iter, vstep,
                              step_rule, solver, tol_abs, tol_rel, tol_f, &its, stream);
    total += its;
    if (iters_out) *iters_out = total;
    if (rc) {
      if (rc == EEC_ENOCONV)
        return fail(c, EEC_ENOCONV, "time step " + std::to_string(st) +
                                        ": no convergence within max_iter iterations");
      return rc;
    }
    std::swap(qa, qb);
    std::swap(ia, ib);
    if (traj)
      CUDA_TRY(c, cudaMemcpyAsync(traj + (size_t)st * c->n, x, sizeof(double) * c->n,
                                  cudaMemcpyDeviceToDevice, s));
  }
  return EEC_OK;
}
int eec_transient(eec_ctx* c, double* x, double h, int32_t n_steps, int32_t method, double* traj,
                  int32_t max_iter, double vstep, int32_t step_rule, int32_t solver,
                  double tol_abs, double tol_rel, double tol_f, int32_t* iters_out, void* stream) {
  try {
    return eec_transient_body(c, x, h, n_steps, method, traj, max_iter, vstep, step_rule, solver,
                              tol_abs, tol_rel, tol_f, iters_out, stream);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_eval_stamp_tran_body(eec_ctx* c, const double* x, const double* q_prev, const double* i_prev,
                                    double alpha, double beta, double* A, double* b, double* q, double* icap,
                                    void* stream) {
  NvtxRange range("eec/eval_stamp_tran");
  int rc = check_built(c);
  if (rc) return rc;
  if (!x || !q_prev || !A || !b || !q) return fail(c, EEC_EINVAL, "NULL x, q_prev, A, b or q");
  if (!std::isfinite(alpha) || !std::isfinite(beta) || alpha < 0.0)
    return fail(c, EEC_EINVAL, "alpha must be finite and >= 0, beta finite");
  int v = effective_variant(c);
  if (v != EEC_VARIANT_COLOR_FUSED && v != EEC_VARIANT_COLOR_BUFFERED &&
      v != EEC_VARIANT_COLOR_PIPELINED)
    v = EEC_VARIANT_ATOMIC;
  if (v != EEC_VARIANT_ATOMIC && (!c->colored || c->opt.conflict_rule == EEC_CONFLICT_WRITE_ROWS))
    return fail(c, EEC_ESTATE, "transient colour stamping needs a colouring that counts gate rows");
  if (v == EEC_VARIANT_COLOR_BUFFERED && !c->d.buf_tran &&
      (rc = dalloc(c, &c->d.buf_tran, (size_t)kNContribTran * c->n_dev)))
    return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TranArgs ta{q_prev, i_prev, alpha, beta, q, icap};
  const int blk = c->opt.block ? c->opt.block : c->tuned_block;
  CUDA_TRY(c, launch_init_lin(c->d, A, b, s));
  ++c->n_kernels;
  if (v == EEC_VARIANT_ATOMIC) {
    CUDA_TRY(c, launch_eval_tran(c->d, MODE_ATOMIC, 0, c->n_dev, x, A, b, ta, blk, s));
    c->n_kernels += c->n_dev > 0;
  } else if (v == EEC_VARIANT_COLOR_PIPELINED) {
    CUDA_TRY(c, launch_color_pipe_tran(c->d, c->pipe_colors, x, A, b, ta, c->pipe_grid, s));
    c->n_kernels += c->d.n_pitem > 0;
  } else if (v == EEC_VARIANT_COLOR_BUFFERED) {
    // every device into the buffer in one launch, then the colour-ordered stamp by one cluster
    CUDA_TRY(c, launch_eval_tran(c->d, MODE_BUFFER, 0, c->n_dev, x, A, b, ta, blk, s));
    CUDA_TRY(c, launch_stamp_cluster_tran(c->d, c->d_coff, c->C, A, b, s));
    c->n_kernels += 1 + (c->n_dev > 0);
  } else {
    for (int k = 0; k < c->C; ++k) {
      if (c->color_off[k + 1] <= c->color_off[k]) continue;
      CUDA_TRY(c, launch_eval_tran(c->d, MODE_RMW, c->color_off[k], c->color_off[k + 1], x, A, b,
                                   ta, blk, s));
      ++c->n_kernels;
    }
  }
  return EEC_OK;
}
int eec_eval_stamp_tran(eec_ctx* c, const double* x, const double* q_prev, const double* i_prev,
                        double alpha, double beta, double* A, double* b, double* q, double* icap,
                        void* stream) {
  try {
    return eec_eval_stamp_tran_body(c, x, q_prev, i_prev, alpha, beta, A, b, q, icap, stream);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_eval_stamp_bwd_body(eec_ctx* c, const double* x, const double* gA, const double* gb,
                                   double* gx, double* gW, double* gL, void* stream) {
  NvtxRange range("eec/eval_stamp_bwd");
  int rc = check_built(c);
  if (rc) return rc;
  if (!x || !gA || !gb || !gx || !gW || !gL) return fail(c, EEC_EINVAL, "NULL argument");
  if ((rc = ensure_gv(c))) return rc;
  CUDA_TRY(c, launch_bwd(c->d, x, gA, gb, gx, gW, gL, c->opt.block, static_cast<cudaStream_t>(stream)));
  return EEC_OK;
}
int eec_eval_stamp_bwd(eec_ctx* c, const double* x, const double* gA, const double* gb,
                       double* gx, double* gW, double* gL, void* stream) {
  try {
    return eec_eval_stamp_bwd_body(c, x, gA, gb, gx, gW, gL, stream);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_eval_stamp_bwd_noalloc_body(eec_ctx* c, const double* x, const double* gA, const double* gb,
                                           double* gx, double* gW, double* gL, void* stream) {
  int rc = check_built(c);
  if (rc) return rc;
  if (!x || !gA || !gb || !gx || !gW || !gL) return fail(c, EEC_EINVAL, "NULL argument");
  if (c->n_dev > EEC_NOALLOC_MAX_DEV)
    return fail(c, EEC_EINVAL, "eec_eval_stamp_bwd_noalloc: " + std::to_string(c->n_dev) +
                                   " devices exceed the fixed scratch of EEC_NOALLOC_MAX_DEV = " +
                                   std::to_string(EEC_NOALLOC_MAX_DEV) + " devices");
  CUDA_TRY(c, launch_bwd_noalloc(c->d, x, gA, gb, gx, gW, gL, static_cast<cudaStream_t>(stream)));
  return EEC_OK;
}
int eec_eval_stamp_bwd_noalloc(eec_ctx* c, const double* x, const double* gA, const double* gb,
                               double* gx, double* gW, double* gL, void* stream) {
  try {
    return eec_eval_stamp_bwd_noalloc_body(c, x, gA, gb, gx, gW, gL, stream);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_graph_capture_body(eec_ctx* c, const double* x, double* A, double* b, double* q, void* stream) {
  int rc = check_built(c);
  if (rc) return rc;
  if (!x || !A || !b) return fail(c, EEC_EINVAL, "NULL x, A or b");
  if (c->user_exec) cudaGraphExecDestroy(c->user_exec);
  c->user_exec = nullptr;
  // Order the capture after the caller's pending work on `stream` (nothing runs during capture).
  if (stream) CUDA_TRY(c, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  return capture(c, effective_variant(c), x, A, b, q, &c->user_exec, &c->user_kernels);
}
int eec_graph_capture(eec_ctx* c, const double* x, double* A, double* b, double* q, void* stream) {
  try {
    return eec_graph_capture_body(c, x, A, b, q, stream);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_batch_create_body(eec_ctx** out, int32_t n_circ, const eec_netlist* const* nets,
                                 double gshunt, const eec_options* opt) {
  if (!out) return EEC_EINVAL;
  *out = nullptr;
  if (n_circ < 1 || !nets) return EEC_EINVAL;
  std::vector<eec_netlist> flat((size_t)n_circ);
  for (int k = 0; k < n_circ; ++k) {
    if (!nets[k]) return EEC_EINVAL;
    flat[k] = *nets[k];
  }
  eec_ctx* c = nullptr;
  int rc = eec_create(&c, opt);
  if (rc) return rc;
  if ((rc = eec_upload_batch(c, n_circ, flat.data(), gshunt))) {
    eec_destroy(c);
    return rc;
  }
  *out = c;
  return EEC_OK;
}
int eec_batch_create(eec_ctx** out, int32_t n_circ, const eec_netlist* const* nets,
                     double gshunt, const eec_options* opt) {
  try {
    return eec_batch_create_body(out, n_circ, nets, gshunt, opt);
  } catch (...) {
    return abi_exception(nullptr);
  }
}

static int eec_batch_capture_graph_body(eec_ctx* c, void* stream) {
  if (!c) return EEC_EINVAL;
  // no launch of the context may be in flight on the caller's stream while the mode changes
  if (stream) CUDA_TRY(c, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  c->graph_all = true;
  return EEC_OK;
}
int eec_batch_capture_graph(eec_ctx* c, void* stream) {
  try {
    return eec_batch_capture_graph_body(c, stream);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_graph_launch_body(eec_ctx* c, void* stream) {
  int rc = check_built(c);
  if (rc) return rc;
  if (!c->user_exec) return fail(c, EEC_ESTATE, "no graph captured");
  CUDA_TRY(c, cudaGraphLaunch(c->user_exec, static_cast<cudaStream_t>(stream)));
  c->n_kernels += c->user_kernels;
  return EEC_OK;
}
int eec_graph_launch(eec_ctx* c, void* stream) {
  try {
    return eec_graph_launch_body(c, stream);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_profile_enable_body(eec_ctx* c, int32_t enable) {
  if (!c) return EEC_EINVAL;
  if (c->prof && !enable && c->ev_used) cudaDeviceSynchronize();
  c->prof = enable != 0;
  c->ev_used = 0;
  c->prof_calls = 0;
  return EEC_OK;
}
int eec_profile_enable(eec_ctx* c, int32_t enable) {
  try {
    return eec_profile_enable_body(c, enable);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_profile_read_body(eec_ctx* c, double* ms_init, double* ms_eval, double* ms_stamp,
                                 int64_t* n_calls, int64_t* n_kernels) {
  if (!c) return EEC_EINVAL;
  double t[3] = {0.0, 0.0, 0.0};
  if (c->ev_used) {
    CUDA_TRY(c, cudaEventSynchronize(c->ev_pool[c->ev_used - 1]));
    // every call recorded exactly four events: init | evaluate | stamp
    for (size_t i = 0; i + 3 < c->ev_used; i += 4) {
      for (int ph = 0; ph < 3; ++ph) {
        float ms = 0.f;
        CUDA_TRY(c, cudaEventElapsedTime(&ms, c->ev_pool[i + ph], c->ev_pool[i + ph + 1]));
        t[ph] += ms;
      }
    }
  }
  if (ms_init) *ms_init = t[0];
  if (ms_eval) *ms_eval = t[1];
  if (ms_stamp) *ms_stamp = t[2];
  if (n_calls) *n_calls = c->prof_calls;
  if (n_kernels) *n_kernels = c->n_kernels;
  c->ev_used = 0;
  c->prof_calls = 0;
  c->n_kernels = 0;
  return EEC_OK;
}
int eec_profile_read(eec_ctx* c, double* ms_init, double* ms_eval, double* ms_stamp,
                     int64_t* n_calls, int64_t* n_kernels) {
  try {
    return eec_profile_read_body(c, ms_init, ms_eval, ms_stamp, n_calls, n_kernels);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_autotune_body(eec_ctx* c, const double* x, double* A, double* b, double* q, int32_t reps,
                             void* stream, float* ms_out) {
  int rc = check_built(c);
  if (rc) return rc;
  if (!x || !A || !b || reps < 1) return fail(c, EEC_EINVAL, "bad autotune arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  CUDA_TRY(c, cudaEventCreate(&e0));
  CUDA_TRY(c, cudaEventCreate(&e1));
  // Blocks tried when the caller left the choice to the library (opt.block == 0).
  const int cand_auto[4] = {0, 32, 64, 128};
  const int n_cand = c->opt.block ? 1 : 4;
  const int saved_tuned = c->tuned_block;
  float best = 1e30f;
  int best_v = EEC_VARIANT_SEGREDUCE, best_b = 0;
  bool best_o = c->eval_ordered;
  for (int v = 0; v < EEC_N_VARIANTS; ++v) {
    float best_ms_v = -1.0f;
    // the order-free schedules are also timed in both launch orders (cost order, layout order)
    const bool order_free = v == EEC_VARIANT_ATOMIC || v == EEC_VARIANT_SEGREDUCE ||
                            v == EEC_VARIANT_COLOR_BUFFERED;
    const int n_ord = (order_free && c->eval_nr >= 2) ? 2 : 1;
    if (!variant_needs_colors(v) || c->colored) {
      for (int io = 0; io < n_cand * n_ord; ++io) {
        const int ib = io / n_ord;
        c->eval_ordered = n_ord == 2 ? (io % 2 == 0) : true;
        c->tuned_block = c->opt.block ? saved_tuned : cand_auto[ib];
        float ms = -1.0f;
        rc = eval_with(c, v, x, A, b, q, s);
        if (rc == EEC_OK) {
          cudaEventRecord(e0, s);
          for (int r = 0; r < reps && rc == EEC_OK; ++r) rc = eval_with(c, v, x, A, b, q, s);
          cudaEventRecord(e1, s);
          if (cudaEventSynchronize(e1) == cudaSuccess && rc == EEC_OK) {
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= reps;
          }
        }
        if (rc != EEC_OK) {
          c->tuned_block = saved_tuned;
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return rc;
        }
        if (ms >= 0.0f && (best_ms_v < 0.0f || ms < best_ms_v)) best_ms_v = ms;
        if (ms >= 0.0f && ms < best) {
          best = ms;
          best_v = v;
          best_b = c->tuned_block;
          best_o = c->eval_ordered;
        }
      }
    }
    if (ms_out) ms_out[v] = best_ms_v;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->tuned_variant = best_v;
  c->tuned_block = c->opt.block ? saved_tuned : best_b;
  c->eval_ordered = best_o;
  return EEC_OK;
}
int eec_autotune(eec_ctx* c, const double* x, double* A, double* b, double* q, int32_t reps,
                 void* stream, float* ms_out) {
  try {
    return eec_autotune_body(c, x, A, b, q, reps, stream, ms_out);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_get_tuning_body(const eec_ctx* c, int32_t* variant, int32_t* block, int32_t* eval_order) {
  if (!c) return EEC_EINVAL;
  if (variant) *variant = effective_variant(c);
  if (block) *block = c->opt.block ? c->opt.block : c->tuned_block;
  if (eval_order) *eval_order = (c->eval_nr >= 2 && c->eval_ordered) ? 1 : 0;
  return EEC_OK;
}
int eec_get_tuning(const eec_ctx* c, int32_t* variant, int32_t* block, int32_t* eval_order) {
  try {
    return eec_get_tuning_body(c, variant, block, eval_order);
  } catch (...) {
    return abi_exception(const_cast<eec_ctx*>(c));
  }
}

static int eec_status_body(eec_ctx* c, void* stream) {
  if (!c) return EEC_EINVAL;
  if (!c->d_status) return fail(c, EEC_ESTATE, "no device state yet");
  CUDA_TRY(c, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  int st = 0;
  CUDA_TRY(c, cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(c, cudaMemset(c->d_status, 0, sizeof(int)));
  if (st & kStatusTimeout) return fail(c, EEC_ETIMEOUT, "a grid barrier wait ran past its limit");
  if (st & kStatusNumeric) return fail(c, EEC_ENUMERIC, "non-finite value in an evaluated device");
  return EEC_OK;
}
int eec_status(eec_ctx* c, void* stream) {
  try {
    return eec_status_body(c, stream);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_math_check_body(int32_t fn, int64_t n, const double* x, double* ours, double* ref,
                               void* stream) {
  if (fn < 0 || fn > 4 || n < 0 || (n > 0 && (!x || !ours || !ref))) return EEC_EINVAL;
  return math_check(fn, n, x, ours, ref, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? EEC_OK
             : EEC_ECUDA;
}
int eec_math_check(int32_t fn, int64_t n, const double* x, double* ours, double* ref,
                   void* stream) {
  try {
    return eec_math_check_body(fn, n, x, ours, ref, stream);
  } catch (...) {
    return abi_exception(nullptr);
  }
}

static int eec_test_barrier_timeout_body(eec_ctx* c, const double* x, double* A, double* b, void* stream) {
  int rc = check_built(c);
  if (rc) return rc;
  if (!c->colored || c->C < 2) return fail(c, EEC_ESTATE, "needs a coloured context with >= 2 colours");
  if (!x || !A || !b) return fail(c, EEC_EINVAL, "NULL x, A or b");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CUDA_TRY(c, launch_init_lin(c->d, A, b, s));
  if (effective_variant(c) == EEC_VARIANT_COLOR_PIPELINED) {
    if (c->pipe_colors < 2) return fail(c, EEC_ESTATE, "needs >= 2 non-empty colours");
    CUDA_TRY(c, launch_color_pipe(c->d, c->pipe_colors, x, A, b, nullptr, c->pipe_grid, 0, s,
                                  /*absent_item=*/0));
    return EEC_OK;
  }
  CUDA_TRY(c, launch_persistent(c->d, c->d_coff, c->C, x, A, b, nullptr, 0, c->persist_grid, 0, s,
                                /*absent_block=*/0));
  return EEC_OK;
}
int eec_test_barrier_timeout(eec_ctx* c, const double* x, double* A, double* b, void* stream) {
  try {
    return eec_test_barrier_timeout_body(c, x, A, b, stream);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_lu_check_host_ex_body(int32_t n, const int32_t* row_ptr, const int32_t* col,
                                     const double* a, const double* b, int32_t order, double* x,
                                     int32_t* q_out, int64_t* nnz_lu, int32_t* bad_col,
                                     int32_t* depth) {
  if (n < 1 || !row_ptr || !col || !a || !b || !x) return EEC_EINVAL;
  if (order != EEC_LU_ORDER_MMD && order != EEC_LU_ORDER_BTF) return EEC_EINVAL;
  const std::vector<int> rp(row_ptr, row_ptr + n + 1);
  if (rp[0] != 0) return EEC_EINVAL;
  for (int i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) return EEC_EINVAL;
  const std::vector<int> cl(col, col + rp[n]);
  for (int v : cl)
    if (v < 0 || v >= n) return EEC_EINVAL;
  const std::vector<double> av(a, a + rp[n]), bv(b, b + n);
  std::vector<int> q;
  const bool ok = order == EEC_LU_ORDER_BTF ? lu_btf_order(n, rp, cl, q)
                                            : lu_min_degree_order(n, rp, cl, q);
  if (!ok) return EEC_ENOMEM;
  LuPlan P;
  std::string err;
  const int rc = lu_analyze(n, rp, cl, av, q, P, err);
  if (rc) return rc;
  std::vector<double> xv;
  int bad = -1;
  lu_refactor_solve_host(P, av, bv, kLuTiny, xv, &bad);
  std::copy(xv.begin(), xv.end(), x);
  if (q_out) std::copy(q.begin(), q.end(), q_out);
  if (nnz_lu) *nnz_lu = P.cptr[n];
  if (bad_col) *bad_col = bad;
  if (depth) lu_plan_depth(P, depth);
  return EEC_OK;
}
int eec_lu_check_host_ex(int32_t n, const int32_t* row_ptr, const int32_t* col, const double* a,
                         const double* b, int32_t order, double* x, int32_t* q_out,
                         int64_t* nnz_lu, int32_t* bad_col, int32_t* depth) {
  try {
    return eec_lu_check_host_ex_body(n, row_ptr, col, a, b, order, x, q_out, nnz_lu, bad_col,
                                     depth);
  } catch (...) {
    return abi_exception(nullptr);
  }
}
int eec_lu_check_host(int32_t n, const int32_t* row_ptr, const int32_t* col, const double* a,
                      const double* b, double* x, int64_t* nnz_lu, int32_t* bad_col) {
  try {
    return eec_lu_check_host_ex_body(n, row_ptr, col, a, b, EEC_LU_ORDER_MMD, x, nullptr, nnz_lu,
                                     bad_col, nullptr);
  } catch (...) {
    return abi_exception(nullptr);
  }
}

static int eec_gather_plan_host_body(int64_t n_entries, const int32_t* cnt, int64_t* item_of,
                                     int32_t* step_of, int32_t* woff, uint16_t* loc,
                                     int32_t* heavy, int64_t* n_items) {
  if (n_entries < 0 || n_entries > 0x7fffffffLL || (n_entries > 0 && !cnt)) return EEC_EINVAL;
  const std::vector<int> gcnt(cnt, cnt + n_entries);
  for (int v : gcnt)
    if (v < 0) return EEC_EINVAL;
  std::vector<long long> ghead;
  std::vector<int> gwoff;
  std::vector<unsigned short> gloc;
  std::vector<int4> gheavy;
  long long items = 0;
  if (!gather_plan(gcnt, ghead, gwoff, gloc, gheavy, items)) return EEC_EINVAL;
  for (long long e = 0; e < n_entries; ++e) {
    if (item_of) item_of[e] = ghead[e];
    if (step_of) step_of[e] = gcnt[e] < kHeavy ? 32 : 1;
  }
  if (woff) std::copy(gwoff.begin(), gwoff.end(), woff);
  if (loc) std::copy(gloc.begin(), gloc.end(), loc);
  if (heavy)
    for (size_t h = 0; h < gheavy.size(); ++h) {
      heavy[3 * h] = gheavy[h].x;
      heavy[3 * h + 1] = gheavy[h].y;
      heavy[3 * h + 2] = gheavy[h].z;
    }
  if (n_items) *n_items = items;
  return EEC_OK;
}
int eec_gather_plan_host(int64_t n_entries, const int32_t* cnt, int64_t* item_of, int32_t* step_of,
                         int32_t* woff, uint16_t* loc, int32_t* heavy, int64_t* n_items) {
  try {
    return eec_gather_plan_host_body(n_entries, cnt, item_of, step_of, woff, loc, heavy, n_items);
  } catch (...) {
    return abi_exception(nullptr);
  }
}

static int eec_lu_solve_body(eec_ctx* c, const double* A, const double* b, double* x, void* stream) {
  NvtxRange range("eec/lu_solve");
  int rc = check_built(c);
  if (rc) return rc;
  if (!A || !b || !x) return fail(c, EEC_EINVAL, "NULL A, b or x");
  if (c->n == 0) return EEC_OK;
  if ((rc = newton_common(c))) return rc;
  return lu_factor_solve(c, A, b, x, 1, static_cast<cudaStream_t>(stream));
}
int eec_lu_solve(eec_ctx* c, const double* A, const double* b, double* x, void* stream) {
  try {
    return eec_lu_solve_body(c, A, b, x, stream);
  } catch (...) {
    return abi_exception(c);
  }
}

static int eec_lu_stats_body(const eec_ctx* c, int64_t* nnz_lu, int32_t* analyses) {
  if (!c) return EEC_EINVAL;
  if (nnz_lu) *nnz_lu = c->lu_ready ? c->lu.cptr[c->lu.n] : 0;
  if (analyses) *analyses = c->lu_analyses;
  return EEC_OK;
}
int eec_lu_stats(const eec_ctx* c, int64_t* nnz_lu, int32_t* analyses) {
  try {
    return eec_lu_stats_body(c, nnz_lu, analyses);
  } catch (...) {
    return abi_exception(const_cast<eec_ctx*>(c));
  }
}

static int eec_newton_info_body(const eec_ctx* c, int32_t* info) {
  if (!c || !info) return EEC_EINVAL;
  for (int k = 0; k < 4; ++k) info[k] = c->newton_info[k];
  return EEC_OK;
}
int eec_newton_info(const eec_ctx* c, int32_t* info) {
  try {
    return eec_newton_info_body(c, info);
  } catch (...) {
    return abi_exception(const_cast<eec_ctx*>(c));
  }
}

static int eec_fp64_peak_body(int32_t iters, int32_t blocks_per_sm, double* flops) {
  if (iters < 1 || blocks_per_sm < 1 || !flops) return EEC_EINVAL;
  return fp64_peak(iters, blocks_per_sm, flops) == cudaSuccess ? EEC_OK : EEC_ECUDA;
}
int eec_fp64_peak(int32_t iters, int32_t blocks_per_sm, double* flops) {
  try {
    return eec_fp64_peak_body(iters, blocks_per_sm, flops);
  } catch (...) {
    return abi_exception(nullptr);
  }
}

}  // extern "C"
