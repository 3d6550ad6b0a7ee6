// Internal declarations shared by the library's translation units (host and device).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/eec.h"

namespace eec {

// Per-card constants of the EES-L1 level, derived on the host from the EEC_CARD_LEN card.
struct CardK {
  double VTH0, K1, PHI, sqrtPHI;
  double nVt, inv_nVt, Vt, inv_Vt, twoVt;
  double UA, UB, ETA0;
  double DELTA, twoDELTA, fourDELTA;
  double fourD1sq, twoD1sq;
  double XPART, GMIN;
  // constant products: K1/2, VTH0 - K1 sqrt(PHI), 2 UB, XPART - 1/2
  double halfK1, Vthc, twoUB, XPm;
  // factors of the per-device parameters (eval_params)
  double U0Cox, twoVSAT_U0, LAMBDA_LREF, JS_HDIF, Cox, CGSO, CGDO;
};

// x-independent terms of devices whose source and body are source-held: sqs, Vthb, dVth/dvbs,
// Ab, dAb/dvbs, Ijs, gjs, Qb (layout [kNBody][N]).
constexpr int kNBody = 8;

// Per-device derived parameters, stored structure-of-arrays [kNPrm][N] by layout position.
enum Prm : int {
  P_BETA0 = 0, P_CE, P_INV_CE, P_LAML, P_ISAT, P_COXT, P_COVS, P_COVD, P_ISATVT, P_ISATVTG, kNPrm
};

// Contribution slots of one device: rows (d, s, b) x columns (d, g, s, b) -> j = 4 r + u,
// then the three right-hand-side rows j = 12 + r.
constexpr int kNSlot = 12;
constexpr int kNContrib = 15;
// Transient buffer of one device: A values of rows d, g, s, b x columns d, g, s, b at j = 4 t + u,
// then the four right-hand-side rows at j = 16 + t.
constexpr int kNContribTran = 20;

// Device-side topology and parameters, indexed by layout position k (colour-major when coloured).
struct DevTopo {
  int N;            // devices
  int n;            // unknowns
  long long nnz;    // CSR nonzeros
  int4* tidx;       // [N] terminal -> unknown (>= 0) or ~fixed-table index (< 0)
  int* meta;        // [N] (card << 2) | (source and body source-held) << 1 | (type < 0)
  int* orig;        // [N] original device index of each position
  int* slot;        // [kNSlot][N] CSR value index or -1
  int* slot_g;      // [4][N] gate-row slots (transient stamping) or -1
  double* W;        // [N]
  double* L;        // [N]
  double* prm;      // [kNPrm][N]
  double* bodyk;    // [kNBody][N] x-independent body/source-junction terms (flagged devices)
  double* vfix;     // [n_fixed] voltages of source-held nodes
  CardK* cards;     // [n_cards]
  double* Alin;     // [nnz]
  double* blin;     // [n]
  // segmented reduction: the evaluation writes contribution j of the device at position k to
  // cbuf[gat_pos[j * N + k]] (-1: not formed). Entry e (A entries 0..nnz-1, then b rows) is its
  // linear part (written once, when cbuf is allocated), then its contributions in original
  // device order. The entries of window w (kGatherWin consecutive ones) with fewer than kHeavy
  // contributions, sorted by their count (ties in entry order), form groups of 32; group g keeps
  // its items column-major from cbuf[gat_woff[w (kGatherGroups + 1) + g]]: item k of its i-th
  // entry at 32 k + i (item 0 the linear part; zeros past an entry's end). Heavy entries' runs
  // follow, contiguous
  int* gat_woff;           // [n_win (kGatherGroups + 1)] first item of every group, then the end
  unsigned short* gat_loc; // [n_win kGatherWin] slot 32 g + i -> entry - w kGatherWin (0xffff: none)
  int n_win;
  int4* gat_heavy;     // [n_heavy] {entry, first item, items, 0} (one warp each)
  int n_heavy;
  int* gat_pos;        // [kNContrib][N] position of each contribution in cbuf, or -1
  double* cbuf;        // (allocated on first use)
  double* buf;         // [kNContrib][N] (allocated on first use)
  double* buf_tran;    // [kNContribTran][N]: transient values G + alpha C (4 x 4) and 4 rhs
  // backward: unknown u gathers gv[src] over inc_src[inc_ptr[u] .. inc_ptr[u+1])
  int* inc_ptr;     // [n + 1]
  int* inc_src;     // flat index t * N + k into gv
  int* inc_light;   // unknowns with fewer than kHeavy terminals (one thread each)
  int* inc_heavy;   // the others (one warp each)
  int n_inc_light, n_inc_heavy;
  double* gv;       // [4][N] (allocated on first use)
  // pipelined colour schedule: work items of up to kPipeItem devices of one colour, in colour
  // order; item i = {first position, end position, colour j (among the non-empty colours),
  // number of items of colour j - 1 (0 for the first)}
  int4* pitem;      // [n_pitem]
  int n_pitem;
  unsigned* pipe;   // [kPipeHdr + non-empty colours]: ticket, blocks left, abort word, unused,
                    // then per colour the items whose stamps are done (all zero between launches)
  int* status;      // device status word: bit 0 timeout, bit 1 non-finite
  unsigned* bar;    // grid barrier: [0] arrival count, [1] generation, [2] abort word of the
                    // current launch (all kBarWords zeroed before each persistent launch)
};

constexpr int kBarWords = 3;
constexpr int kPipeItem = 128;   // devices per work item of the pipelined colour schedule
constexpr int kPipeHdr = 4;

constexpr int kHeavy = 32;  // contributions from which an entry gets a whole warp in the gather
constexpr int kGatherWin = 1024;  // entries per window of the gather (one block)
constexpr int kGatherGroups = kGatherWin / 32;

constexpr int kStatusTimeout = 1;
constexpr int kStatusNumeric = 2;

// ---- kernels (eec_kernels.cu) ----
// MODE_BUFFER: contributions into buf (layout position-major, read by the colour-ordered stamps);
// MODE_SORTED: contributions into cbuf at gat_pos, each entry's items in device order (read by
// the segmented-reduction gather).
enum StampMode : int { MODE_RMW = 0, MODE_ATOMIC = 1, MODE_BUFFER = 2, MODE_SORTED = 3 };

cudaError_t launch_params(const DevTopo& T, cudaStream_t s);
// W_dev, L_dev in original device order -> per-position W, L and derived parameters.
cudaError_t launch_update_params(const DevTopo& T, const double* W_dev, const double* L_dev,
                                 cudaStream_t s);
// pdl: launch with programmatic stream serialisation (the atomic evaluation may start while the
// linear-part initialisation before it runs; it waits for that kernel before its first addition).
cudaError_t launch_eval(const DevTopo& T, int mode, int begin, int end, const double* x,
                        double* A, double* b, double* q, int block, int dbg, cudaStream_t s,
                        bool pdl = false);
// The devices of a list of library-order ranges: range r starts at position rbeg[r] and holds
// roff[r+1] - roff[r] devices (roff[0] = 0, roff[nr] = total); only for the order-free modes
// MODE_ATOMIC and MODE_BUFFER.
cudaError_t launch_eval_ranges(const DevTopo& T, int mode, const int* rbeg, const int* roff,
                               int nr, int total, const double* x, double* A, double* b,
                               double* q, int block, int dbg, cudaStream_t s, bool pdl = false);
// absent_block >= 0 is a test hook: that block skips every grid barrier, so the other blocks'
// bounded waits expire and the status word records a timeout.
cudaError_t launch_persistent(const DevTopo& T, const int* color_off_dev, int n_colors,
                              const double* x, double* A, double* b, double* q, int block,
                              int grid, int dbg, cudaStream_t s, int absent_block = -1);
int persistent_max_blocks_per_sm(int block, bool want_q);
cudaError_t launch_gather(const DevTopo& T, double* A, double* b, cudaStream_t s);
// writes every entry's linear part to the head of its run in a new cbuf
cudaError_t launch_gather_init(const DevTopo& T, cudaStream_t s);
// A <- A_lin, b <- b_lin (the linear part), one kernel.
cudaError_t launch_init_lin(const DevTopo& T, double* A, double* b, cudaStream_t s);
// Buffered contributions of every colour, in colour order, in one cooperative launch of `grid`
// blocks (co-resident: at most stamp_persistent_max_blocks_per_sm() per SM).
cudaError_t launch_stamp_persistent(const DevTopo& T, const int* color_off_dev, int n_colors,
                                    double* A, double* b, int grid, cudaStream_t s);
int stamp_persistent_max_blocks_per_sm();
// The same by one thread-block cluster with the hardware cluster barrier between colours
// (stamp_cluster_threads() threads in all).
cudaError_t launch_stamp_cluster(const DevTopo& T, const int* color_off_dev, int n_colors,
                                 double* A, double* b, cudaStream_t s);
int stamp_cluster_threads();
// The transient analogue from buf_tran (four rows per device, the gate row's slots in slot_g).
cudaError_t launch_stamp_cluster_tran(const DevTopo& T, const int* color_off_dev, int n_colors,
                                      double* A, double* b, cudaStream_t s);
// DC Newton loop (eec_newton.cu). stats[0] max|y - x|, [1] max|dx|, [2] max|x|, [3] residual, as
// bit patterns of non-negative doubles (zeroed by the caller).
cudaError_t launch_newton_step(const double* y, double* x, int n, double vstep, int per_node,
                               unsigned long long* stats, cudaStream_t s);
cudaError_t launch_residual_norm(const int* rp, const int* col, const double* A, const double* x,
                                 const double* b, int n, unsigned long long* stats,
                                 cudaStream_t s);
// One nonlinear Jacobi sweep from x into y (node rows; rail nodes set to their source voltage
// when rails are MNA unknowns); stats[1] = max |move|, stats[0] += rows moved more than 1 mV
// (when count is set).
cudaError_t launch_relax_step(const int* rp, const int* col, const double* A, const double* x,
                              const double* b, const int* diag, int n_node, int n, double vmax,
                              const int* rail_unk, int n_rail, double* y,
                              unsigned long long* stats, int count, cudaStream_t s);
// A[diag[i]] += g, i < n (the gshunt-stepping homotopy of eec_newton_dc)
cudaError_t launch_add_diag(double* A, const int* diag, int n, double g, cudaStream_t s);
// Transient companion stamp (mode MODE_RMW over one colour range, MODE_ATOMIC over all, or
// MODE_BUFFER over all into buf_tran).
struct TranArgs {
  const double* qprev;  // [4][N_orig] charges of the previous time point
  const double* iprev;  // [4][N_orig] capacitive currents of the previous time point, nullable
  double alpha, beta;   // ic = alpha (q - qprev) - beta iprev
  double* q;            // [4][N_orig] out: charges at x
  double* icap;         // [4][N_orig] out: capacitive currents at x, nullable
};
cudaError_t launch_eval_tran(const DevTopo& T, int mode, int begin, int end, const double* x,
                             double* A, double* b, const TranArgs& ta, int block, cudaStream_t s);
cudaError_t launch_stamp_buffer(const DevTopo& T, int begin, int end, double* A, double* b,
                                int block, cudaStream_t s);
// Pipelined colour schedule: one launch of `grid` blocks (programmatic dependent of the
// initialisation of A and b) that evaluates every device and stamps colour after colour, each
// colour's stamps after every stamp of the colour before it (per-colour completion counters,
// bounded waits). absent_item >= 0 is a test hook: that item never reports its stamps done, so
// the next colour's waits expire and the status word records a timeout.
cudaError_t launch_color_pipe(const DevTopo& T, int n_colors_nonempty, const double* x, double* A,
                              double* b, double* q, int grid, int dbg, cudaStream_t s,
                              int absent_item = -1);
cudaError_t launch_color_pipe_tran(const DevTopo& T, int n_colors_nonempty, const double* x,
                                   double* A, double* b, const TranArgs& ta, int grid,
                                   cudaStream_t s);
int color_pipe_max_blocks_per_sm();
cudaError_t launch_bwd(const DevTopo& T, const double* x, const double* gA, const double* gb,
                       double* gx, double* gW, double* gL, int block, cudaStream_t s);
cudaError_t fp64_peak(int iters, int blocks_per_sm, double* flops);
cudaError_t math_check(int fn, long long n, const double* x, double* ours, double* ref,
                       cudaStream_t s);
// Resolve (once per device) the device address of the fixed scratch array of
// launch_bwd_noalloc on the current device; this loads the module that holds the array.
cudaError_t noalloc_setup();
// Backward with its terminal-gradient scratch in the library's fixed array (no allocation).
cudaError_t launch_bwd_noalloc(const DevTopo& T, const double* x, const double* gA,
                               const double* gb, double* gx, double* gW, double* gL,
                               cudaStream_t s);

// ---- GPU colouring (eec_color.cu) ----
// Jones-Plassmann colouring of the conflict graph given as node -> device incidence (CSR over
// conflict nodes). prio[v] = priority (higher colours first). Returns colours in col (host).
int jp_color(int n_dev, const std::vector<int>& node_ptr, const std::vector<int>& node_dev,
             const std::vector<int>& dev_ptr, const std::vector<int>& dev_node,
             const std::vector<uint32_t>& prio, std::vector<int>& col, int* n_colors,
             std::string& err);

}  // namespace eec
