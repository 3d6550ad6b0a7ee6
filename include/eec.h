/*
 * eec.h — C ABI of the GB300 (sm_103a) MOSFET evaluate-and-stamp library.
 *
 * The library implements the per-Newton-iteration hot path of EEspice (arXiv 2604.03079): every
 * MOSFET instance is evaluated at the present node voltages (terminal currents, charges and
 * linearised conductances: the "compute phase" of Sec. II (i)) and its contributions are
 * accumulated into the shared sparse MNA matrix A and right-hand side b (the "stamp phase" of
 * Sec. II (ii)). Stamping is made lock-free by the paper's conflict graph and greedy colouring
 * (Sec. I, Sec. II): devices that share a non-ground node get different colours, colours run one
 * after another, and the devices of one colour stamp concurrently.
 *
 * Conventions shared by every entry point
 *  - Return value: 0 on success, a negative EEC_E* code on failure. No C++ exception crosses the
 *    ABI: host memory running out inside a call returns EEC_ENOMEM. eec_last_error() returns a
 *    message for the last failure on that context.
 *  - Pointers named *_dev are CUDA device pointers; all others are host pointers. The caller owns
 *    every pointer it passes; the library copies host inputs during the call and keeps no pointer
 *    to them, never frees caller memory, and owns only the device arrays it allocates itself
 *    (released by eec_destroy).
 *  - cuda_stream is a cudaStream_t (NULL = legacy default stream). Calls that take a stream are
 *    asynchronous and stream-ordered unless stated otherwise.
 *  - Unknowns are the free (not source-held) nodes in increasing node order. A is stored in CSR
 *    with sorted column indices; its pattern comes from eec_get_pattern().
 *  - The context is not thread-safe; distinct contexts are independent.
 */
#ifndef EEC_H_
#define EEC_H_

#include <stdint.h>

#if defined(__GNUC__)
#define EEC_API __attribute__((visibility("default")))
#else
#define EEC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define EEC_OK 0
#define EEC_EINVAL (-1)   /* bad argument: size, index, pointer, enum value */
#define EEC_ESTATE (-2)   /* call out of order (e.g. eval before eec_build_scatter) */
#define EEC_ECUDA (-3)    /* a CUDA runtime call failed; message has the CUDA error string */
#define EEC_ETIMEOUT (-4) /* a device-side wait ran past its limit (status word) */
#define EEC_ENUMERIC (-5) /* non-finite value detected by the debug checks (status word) */
#define EEC_ENOCONV (-6)  /* eec_newton_dc: no convergence within max_iter */
#define EEC_ENOMEM (-7)   /* device allocation failed */

/* Evaluation/stamp schedules (Table I analogues). */
#define EEC_VARIANT_AUTO (-1)          /* the autotuner's choice (SEGREDUCE until tuned) */
#define EEC_VARIANT_COLOR_FUSED 0      /* "ColorFused": one fused launch per colour */
#define EEC_VARIANT_PERSISTENT 1       /* one persistent launch, grid barrier between colours */
#define EEC_VARIANT_ATOMIC 2           /* uncoloured, FP64 atomicAdd stamping */
#define EEC_VARIANT_SEGREDUCE 3        /* evaluate to buffer, then per-entry gather (no colours) */
#define EEC_VARIANT_COLOR_BUFFERED 4   /* "Color": evaluate to buffer, then one stamp per colour */
#define EEC_VARIANT_COLOR_PIPELINED 5  /* colour order in one launch: every device evaluated into
                                          registers, each colour stamped once the colour before it
                                          has stamped (per-colour completion counters) */
#define EEC_N_VARIANTS 6

/* Conflict rules for the colouring. */
#define EEC_CONFLICT_FREE_NODE 0   /* share a free node (rails are free only under MNA_BRANCH) [default] */
#define EEC_CONFLICT_ANY_NONGROUND 1 /* share any node but ground (the paper's literal rule) */
#define EEC_CONFLICT_WRITE_ROWS 2  /* share a free node both write as a DC row (d, s or b) */

/* How nodes held by an ideal voltage source (node_fixed) enter the system. */
#define EEC_RAIL_ELIMINATE 0   /* held nodes are not unknowns; their voltages enter through the
                                  device evaluation and b  [default] */
#define EEC_RAIL_MNA_BRANCH 1  /* modified nodal analysis (Sec. I): every non-ground node is an
                                  unknown and every held node adds the current of its source as
                                  an unknown (see eec_build_scatter) */

/* Colouring algorithms. */
#define EEC_COLOR_GREEDY_SEQ 0  /* host greedy in the given order */
#define EEC_COLOR_JP_INDEX 1    /* GPU Jones-Plassmann, priority = position in the order */
#define EEC_COLOR_JP_RANDOM 2   /* GPU Jones-Plassmann, hashed priorities (valid, not greedy) */

/* Model card of the EES-L1 level: EEC_CARD_LEN doubles in this order.
 * VTH0 K1 PHI NFACT U0 UA UB VSAT TOX ETA0 DELTA LAMBDA LREF JS HDIF CGSO CGDO XPART D1 GMIN TEMP */
#define EEC_CARD_LEN 21

typedef struct eec_ctx eec_ctx; /* opaque, library-owned */

typedef struct {
  int32_t variant;       /* EEC_VARIANT_*; default EEC_VARIANT_AUTO */
  int32_t block;         /* threads per block of the evaluate kernels: 0 = library choice (one
                            warp per block for launches under 152 x 128 devices, else 128),
                            or 8, 16, 32, 64, 96, 128 */
  int32_t conflict_rule; /* EEC_CONFLICT_*; default EEC_CONFLICT_FREE_NODE */
  int32_t debug_checks;  /* nonzero: kernels flag non-finite outputs in the status word */
  int32_t color_stamp;   /* stamp of EEC_VARIANT_COLOR_BUFFERED, colour after colour: 0 = chosen
                            from the colour sizes, 1 = one launch per colour, 2 = one co-resident
                            grid with a grid barrier between colours, 3 = one 8-block thread-block
                            cluster with the cluster barrier between colours */
  int32_t host_chunks;   /* eec_eval_stamp_host: chunks whose charges are copied out while later
                            chunks are evaluated, each half the size of the one before; 0 = by
                            size (4 from 2^18 devices, 3 from 2^17, 2 from 2^16, else 1), or
                            1..64 */
  int32_t rail_mode;     /* EEC_RAIL_*; default EEC_RAIL_ELIMINATE. EEC_RAIL_MNA_BRANCH makes the
                            rails shared free nodes, so under EEC_CONFLICT_FREE_NODE all devices on
                            one rail conflict (Table II: 896 colours for the 64-bit adder, one per
                            PMOS). Not available for eec_upload_batch. */
} eec_options;

/* eec_options with every field at its default. */
EEC_API eec_options eec_default_options(void);

/* Create a context. opt may be NULL (defaults). *out receives the handle. */
EEC_API int eec_create(eec_ctx** out, const eec_options* opt);

/* Release the context and every device array it owns. Accepts NULL. Synchronises the device. */
EEC_API void eec_destroy(eec_ctx* ctx);

/* Message for the last failure on ctx ("" if none); valid until the next call on ctx. */
EEC_API const char* eec_last_error(const eec_ctx* ctx);

/*
 * Upload a netlist (Sec. I: the MNA system A x = b of the circuit; Sec. II: FET instances).
 *  n_nodes      nodes 0..n_nodes-1; node 0 is ground.
 *  node_fixed   [n_nodes] 1 = node held by an ideal source at node_vfix[i] volts (ground is
 *               always fixed at 0 V), 0 = free node (an unknown).
 *  dev_nodes    [n_dev*4] terminals d, g, s, b of each MOSFET.
 *  dev_type     [n_dev] +1 NMOS, -1 PMOS.
 *  W, L         [n_dev] channel width and length in metres (> 0).
 *  model_id     [n_dev] row of the card table (eec_set_model_cards).
 *  res_nodes    [n_res*2], res_G [n_res] siemens: linear conductances.
 *  isrc_nodes   [n_isrc*2] (a, b), isrc_val [n_isrc] amperes flowing from a to b through the source.
 *  gshunt       conductance from every free node to ground (keeps gate-only nodes regular).
 * Host arrays, copied. Replaces any previous netlist and resets the colouring and scatter map.
 */
EEC_API int eec_upload_netlist(eec_ctx* ctx, int32_t n_nodes, const uint8_t* node_fixed,
                       const double* node_vfix, int32_t n_dev, const int32_t* dev_nodes,
                       const int8_t* dev_type, const double* W, const double* L,
                       const int32_t* model_id, int32_t n_res, const int32_t* res_nodes,
                       const double* res_G, int32_t n_isrc, const int32_t* isrc_nodes,
                       const double* isrc_val, double gshunt);

/* Model-card table [n_cards*EEC_CARD_LEN] (host, copied). Every model_id must be < n_cards. */
EEC_API int eec_set_model_cards(eec_ctx* ctx, int32_t n_cards, const double* cards);

/*
 * Colour the conflict graph (Sec. I; Sec. II: an edge joins two FETs that share at least one
 * non-ground node; greedy colouring gives each vertex, in visiting order, the smallest colour not
 * used by its already coloured neighbours). The edge rule is opt.conflict_rule.
 *  order       [n_dev] visiting order (a permutation of 0..n_dev-1), NULL = natural order.
 *  algo        EEC_COLOR_*: GREEDY_SEQ (host) and JP_INDEX (GPU) give the same colours for the
 *              same order; JP_RANDOM gives a valid colouring with hashed priorities.
 *  colors_out  [n_dev] host, nullable: colour of each device.
 *  n_colors    host, out: number of colours C.
 * Synchronous. Resets the scatter map.
 */
EEC_API int eec_color(eec_ctx* ctx, const int32_t* order, int32_t algo, int32_t* colors_out,
              int32_t* n_colors);

/*
 * Build the MNA pattern and the per-device scatter map (Sec. II: every device's contributions
 * go to fixed entries of A and b). The pattern holds, over free nodes: the diagonal, resistor
 * pairs, and every (t, u) terminal pair of every device, the gate row included (symmetric).
 * Devices are laid out colour-major on the device (natural order when not coloured).
 * Under EEC_RAIL_MNA_BRANCH the unknowns are the n_nodes - 1 non-ground nodes in node order,
 * then one source current j_r per held node r (node_fixed, ground excepted) in node order;
 * j_r flows from node r through its source to ground. Each adds the entries (r, j_r) = 1 (KCL
 * at r) and (j_r, r) = 1 with b[j_r] = node_vfix[r] (the source equation v_r = node_vfix[r]);
 * the diagonal (j_r, j_r) is in the pattern with value 0, and gshunt goes on node rows only.
 * Out: *n_unknowns, *nnz. Synchronous.
 */
EEC_API int eec_build_scatter(eec_ctx* ctx, int32_t* n_unknowns, int64_t* nnz);

/* Copy the pattern to caller arrays: row_ptr [n+1], col_idx [nnz], unk_of_node [n_nodes]
 * (unknown index of each node, -1 when fixed; under EEC_RAIL_MNA_BRANCH only ground is -1).
 * Any of them may be NULL. */
EEC_API int eec_get_pattern(const eec_ctx* ctx, int32_t* row_ptr, int32_t* col_idx,
                    int32_t* unk_of_node);

/*
 * Host-side race check of the colour schedule (Sec. II: same-colour devices must never stamp
 * the same entry). Verifies that no two devices of one colour write a common row of A or b —
 * rows d, s, b (DC) plus g when with_gate_rows (transient). Returns EEC_EINVAL naming the two
 * devices on a conflict. Needs eec_build_scatter (host part) after eec_color.
 */
EEC_API int eec_verify_coloring(const eec_ctx* ctx, int32_t with_gate_rows);

/* Colour offsets [C+1] (host) of the device layout; colour c holds positions
 * off[c] .. off[c+1]-1. Fails with EEC_ESTATE when not coloured. */
EEC_API int eec_get_color_offsets(const eec_ctx* ctx, int32_t* off);

/*
 * Replace W and L of every device (original device order, length n_dev) without touching the
 * topology; sizing loops call this between evaluations. W_dev, L_dev: device pointers.
 */
EEC_API int eec_update_params(eec_ctx* ctx, const double* W_dev, const double* L_dev, void* cuda_stream);

/* The schedule, block size and evaluation launch order eec_eval_stamp will use (after
 * autotuning, if any). eval_order (nullable): 1 = devices with a free source or body first (a
 * list of layout ranges), 0 = layout order (also when the layout already is in that order). */
EEC_API int eec_get_tuning(const eec_ctx* ctx, int32_t* variant, int32_t* block,
                           int32_t* eval_order);

/* Select the schedule (EEC_VARIANT_*) used by eec_eval_stamp. */
EEC_API int eec_set_variant(eec_ctx* ctx, int32_t variant);

/* Select the evaluation launch order of the order-free schedules (ATOMIC, SEGREDUCE,
 * COLOR_BUFFERED): 1 = devices with a free source or body first (the default), 0 = layout
 * order. eec_autotune sets it to the faster of the two. */
EEC_API int eec_set_eval_order(eec_ctx* ctx, int32_t cost_order);
EEC_API int eec_get_variant(const eec_ctx* ctx, int32_t* variant);

/*
 * One Newton-iteration evaluate-and-stamp (Sec. II (i) compute phase, (ii) stamp phase):
 *   A = A_lin + sum_dev G_dev,   b = b_lin + sum_dev (-I_dev + G_dev V_dev)
 * where I_dev[t] is the current from node t into the device, G_dev[t][u] = dI_t/dV_u over free
 * terminals, A_lin / b_lin hold gshunt, resistors, current sources and source-held nodes.
 *  x_dev        [n] node voltages of the unknowns.
 *  A_values_dev [nnz] out: values of A in the CSR pattern of eec_get_pattern().
 *  b_dev        [n] out.
 *  q_dev        [4*n_dev] out, nullable: terminal charges, terminal-major (q[t*n_dev + k],
 *               t = d, g, s, b), original device order.
 * Asynchronous on cuda_stream. Device errors land in the status word (eec_status).
 */
EEC_API int eec_eval_stamp(eec_ctx* ctx, const double* x_dev, double* A_values_dev, double* b_dev,
                   double* q_dev, void* cuda_stream);

/*
 * eec_eval_stamp with host buffers: x_host [n] in; A_host [nnz], b_host [n], q_host [4*n_dev]
 * (nullable) out, layouts as in eec_eval_stamp. The library copies x into its own device
 * buffer, evaluates and stamps into its own device buffers (allocated on the first call), and
 * copies A, b and q back. Under the order-free schedules (ATOMIC, SEGREDUCE) the devices are
 * evaluated in opt.host_chunks spans of original index (each half the size of the one before),
 * launched alternately on cuda_stream and a library stream so that no launch's tail leaves the
 * SMs idle, and each span's charges are copied on another library stream while the next span is
 * evaluated; the call joins those streams back into cuda_stream. The two library streams are
 * created by eec_build_scatter: CUDA spreads streams over the device's hardware queues in
 * creation order, and library streams created after a large stream pool could share the
 * caller's queue and lose the overlap. Page-locked buffers (cudaHostAlloc / cudaHostRegister) make every copy
 * asynchronous; pageable ones work but the call returns only once their copies are done.
 * Stream-ordered on cuda_stream: the host outputs are valid once the stream has synchronised.
 * Calls on one context share the staging buffers, so calls that overlap on the GPU (unordered
 * streams) race on them.
 */
EEC_API int eec_eval_stamp_host(eec_ctx* ctx, const double* x_host, double* A_host, double* b_host,
                                double* q_host, void* cuda_stream);

/*
 * DC operating point by damped Newton on the GPU (the loop of Sec. II around the compute and
 * stamp phases; the paper solves with KLU on the host). Every iteration: eec_eval_stamp at x
 * (the context's schedule), a sparse direct solve A y = b on the GPU — solver 0: cuSOLVER's
 * batched sparse QR, its pattern analysis done once per context and reused by every iteration,
 * no fill-reducing order; solver 1: cuSOLVER's sparse QR after a symmetric approximate-minimum-
 * degree ordering, analysed on every call; solver EEC_SOLVER_LU (2): the library's sparse LU —
 * on the host, once per context, a multiple-minimum-degree column order and one factorisation of the
 * first iterate's matrix with threshold partial pivoting fix the row pivots and the patterns of
 * L and U; every iteration then refactors the numbers on that pattern and solves on the GPU
 * (one single-block kernel when the factor fits in shared memory, else one cooperative kernel
 * over every SM; with one step of iterative refinement once the steps are below
 * 1 mV), and analyses again on the host if a pivot falls below 1e-4 of the
 * largest entry of its column (1e-10 for the unrefined solves of steps above 1 mV;
 * eec_lu_stats counts the analyses) — then
 * a damped step: step_rule 0 scales the whole step, x += s (y - x) with s = min(1, vstep /
 * max|y - x|); step_rule 1 clips every node's move to [-vstep, vstep] on its own (long chains of
 * gates converge in far fewer iterations).
 * Converged when max|dx| <= tol_abs + tol_rel max|x| and, at the next iterate, the KCL residual
 * max|A x - b| = max|F(x)| <= tol_f amperes. When max_iter solves do not converge, or a solve
 * fails (a singular matrix, a non-finite step), the loop restarts from the starting point with
 * gshunt stepping: a shunt conductance g from every node
 * to ground, g = 1e-3 S, converged, then g / 10 from that solution, down to the netlist's
 * gshunt, then the circuit itself (each stage with max_iter solves). When that fails too, a
 * relaxation start: from the starting point, nonlinear Jacobi sweeps (every node moves to the
 * zero of its own KCL residual with the other voltages held, the move clipped to 5 vstep; up to
 * min(4 n + 1024, 65536) sweeps, until no node moved more than 1 uV in 32 sweeps or the count of
 * nodes moving more than 1 mV stopped falling over 128 sweeps), then Newton
 * from the relaxed point, then gshunt stepping from there. A chain of gates settles one stage
 * per sweep; from a poor start Newton's exact step on a long chain grows like the stage gain to
 * the power of its length and overflows. eec_newton_info reports which path converged.
 *  x_dev       [n] in: starting point (free-node voltages), out: the last iterate.
 *  A_dev, b_dev  [nnz], [n] workspace; out: the stamp at the returned x.
 *  iters_out   (nullable) solves performed, over all stages.
 * Returns EEC_OK, EEC_ENOCONV (a stage ran max_iter solves without meeting both tests: x holds
 * its last iterate), EEC_ENUMERIC (a non-finite step or residual, or a singular matrix),
 * EEC_ETIMEOUT (a bounded wait of the sparse LU's kernels ran out) or EEC_ENOMEM (solver 2: the
 * pattern fills in too much for a direct solve, as randomly wired logic does: its elimination
 * graph or factor would exceed 32 nnz + 4 Mi entries, or its update list 128 nnz + 16 Mi; the
 * 256 x 256 SRAM needs 1.2 nnz and 39 nnz). Solvers 0 and 1 are meant for netlists up to tens of
 * thousands of unknowns (solver 0 checks its factor's size before allocating); solver 2 has
 * solved the 131,840-unknown SRAM. Synchronises cuda_stream once per iteration (and once per
 * 32 relaxation sweeps).
 */
#define EEC_SOLVER_LU 2
EEC_API int eec_newton_dc(eec_ctx* ctx, double* x_dev, double* A_values_dev, double* b_dev,
                          int32_t max_iter, double vstep, int32_t step_rule, int32_t solver,
                          double tol_abs, double tol_rel, double tol_f, int32_t* iters_out,
                          void* cuda_stream);

/*
 * One implicit time step of a transient analysis (NEXT-1 with the GPU Newton loop of
 * eec_newton_dc): damped Newton on the companion system of eec_eval_stamp_tran,
 * F(x) + i_cap(x) = 0 with i_cap = alpha (q(x) - q_prev) - beta i_prev (backward Euler:
 * alpha = 1/h, beta = 0; trapezoidal: alpha = 2/h, beta = 1), from x (normally the previous time
 * point). The solvers, step rules and tests are eec_newton_dc's; no gshunt stepping or
 * relaxation start (a step that does not converge is the caller's cue to shorten h).
 *  x_dev       [n] in: starting point, out: the last iterate (the new time point when EEC_OK).
 *  q_prev_dev  [4 n_dev] charges of the previous time point (original device order).
 *  i_prev_dev  [4 n_dev] (nullable) capacitive currents of the previous time point.
 *  A_dev, b_dev  workspace, out: the companion stamp at the returned x.
 *  q_dev, icap_dev  [4 n_dev] out: charges and (icap nullable) capacitive currents at x: the next
 *              step's q_prev and i_prev.
 * Returns as eec_newton_dc (EEC_ENOCONV: the step ran max_iter solves).
 */
EEC_API int eec_newton_tran(eec_ctx* ctx, double* x_dev, const double* q_prev_dev,
                            const double* i_prev_dev, double alpha, double beta,
                            double* A_values_dev, double* b_dev, double* q_dev, double* icap_dev,
                            int32_t max_iter, double vstep, int32_t step_rule, int32_t solver,
                            double tol_abs, double tol_rel, double tol_f, int32_t* iters_out,
                            void* cuda_stream);

/*
 * A transient analysis of n_steps fixed steps of h seconds from the state x (the sources held at
 * their values, as in the oracle's transient solver): the charges at t = 0, then eec_newton_tran
 * per step with method 0 (backward Euler) or 1 (trapezoidal; the first step's history current
 * is zero). Context-owned device buffers (allocated on the first call) hold A, b and two time
 * points' charges and capacitive currents.
 *  x_dev     [n] in: the state at t = 0, out: the state at t = n_steps h (or at the failed step).
 *  traj_dev  [(n_steps + 1) n] (nullable) out: the state at every time point, row by row.
 *  iters_out (nullable) Newton iterations over all steps.
 * Returns EEC_OK, EEC_EINVAL, EEC_ENOCONV (a step did not converge; the message names it), or
 * eec_newton_dc's other codes. Synchronises cuda_stream once per Newton iteration.
 */
EEC_API int eec_transient(eec_ctx* ctx, double* x_dev, double h, int32_t n_steps, int32_t method,
                          double* traj_dev, int32_t max_iter, double vstep, int32_t step_rule,
                          int32_t solver, double tol_abs, double tol_rel, double tol_f,
                          int32_t* iters_out, void* cuda_stream);

/*
 * The last eec_newton_dc call on this context: info[0] = solves (as iters_out), info[1] = gshunt
 * stepping stages run, info[2] = relaxation sweeps, info[3] = the path that ended the call:
 * 0 plain Newton, 1 gshunt stepping, 2 relaxation start then Newton, 3 relaxation start then
 * gshunt stepping. info [4] host, out.
 */
EEC_API int eec_newton_info(const eec_ctx* ctx, int32_t* info);

/*
 * x = A^-1 b on the context's pattern with the library's sparse LU (the solver EEC_SOLVER_LU of
 * eec_newton_dc): the first call analyses A on the host (column order, row pivots, plan; it
 * synchronises the stream), every call refactors A's numbers and solves with the library's
 * kernel (with one step of iterative refinement), analysing again if a pivot has fallen below 1e-4 of its column's
 * largest L entry.
 *  A_values_dev [nnz], b_dev [n] in (device, unchanged); x_dev [n] out (device).
 * Returns EEC_ENUMERIC for a singular matrix, EEC_ETIMEOUT if a bounded device wait ran out,
 * EEC_ENOMEM when the pattern fills in too much (as for eec_newton_dc's solver 2).
 * Synchronises the stream once per call (the pivot check).
 */
EEC_API int eec_lu_solve(eec_ctx* ctx, const double* A_values_dev, const double* b_dev,
                         double* x_dev, void* cuda_stream);

/*
 * The sparse LU of eec_newton_dc's solver EEC_SOLVER_LU: *nnz_lu = entries of L and U of the
 * current plan (0 before the first solve), *analyses = host analyses so far (1 + the re-analyses
 * after a degraded pivot). Either pointer may be NULL.
 */
EEC_API int eec_lu_stats(const eec_ctx* ctx, int64_t* nnz_lu, int32_t* analyses);

/*
 * Host check of the sparse LU (no GPU; the paper has no counterpart): for an n x n matrix in CSR
 * (row_ptr [n+1], col [nnz], a [nnz], host), the multiple-minimum-degree order, the host factorisation
 * with threshold partial pivoting, then the GPU kernel's refactorisation and triangular solves
 * executed on the host in the GPU's order, for the right-hand side b [n]; x [n] receives the
 * solution of A x = b. *nnz_lu (nullable) = entries of L and U; *bad_col
 * (nullable) = the first column whose refactorised pivot fell below 1e-4 of its column's
 * largest L entry, or -1.
 * Returns EEC_EINVAL for a malformed matrix, EEC_ENUMERIC for a singular one, EEC_ENOMEM when the
 * pattern fills in too much (as for eec_newton_dc's solver 2).
 */
EEC_API int eec_lu_check_host(int32_t n, const int32_t* row_ptr, const int32_t* col, const double* a,
                              const double* b, double* x, int64_t* nnz_lu, int32_t* bad_col);

/*
 * The same host check with a choice of column order, and what the plan implies for the GPU:
 *  order   EEC_LU_ORDER_MMD: the multiple-minimum-degree order of A + A^T that eec_newton_dc's
 *          solver EEC_SOLVER_LU uses (eec_lu_check_host); EEC_LU_ORDER_BTF: block triangular
 *          form, the strongly connected components of A's directed graph (an edge i -> j for
 *          every off-diagonal A(i, j)), each placed after every component its edges reach,
 *          with multiple minimum degree inside each component (with A's diagonal present the
 *          permuted matrix is block lower triangular). Host check only: eec_newton_dc does not
 *          use this order yet.
 *  q_out   [n] (nullable): the column order (the plan eliminates column q_out[k] k-th)
 *  depth   [3] (nullable): the longest chains of dependent steps of the plan, which bound the
 *          GPU's steps however many warps it has: [0] the refactorisation (column j waits for
 *          every column of U(:, j)), [1] the forward substitution (row i waits for the columns
 *          of L(i, :)), [2] the backward substitution (row i waits for those of U(i, :))
 * The other arguments and the errors are those of eec_lu_check_host; EEC_EINVAL for an unknown
 * order.
 */
#define EEC_LU_ORDER_MMD 0
#define EEC_LU_ORDER_BTF 1
EEC_API int eec_lu_check_host_ex(int32_t n, const int32_t* row_ptr, const int32_t* col,
                                 const double* a, const double* b, int32_t order, double* x,
                                 int32_t* q_out, int64_t* nnz_lu, int32_t* bad_col,
                                 int32_t* depth);

/*
 * Host check of the segmented-reduction schedule's gather plan (no GPU; the paper has no
 * counterpart): the layout eec_build_scatter gives the buffer between EEC_VARIANT_SEGREDUCE's
 * evaluation and its per-entry gather, for n_entries A/b entries (A values, then b rows) with
 * cnt[e] >= 0 device contributions each. Entry e occupies 1 + cnt[e] items: its linear part,
 * then its contributions in original device order. Per window of EEC_GATHER_WINDOW entries, the
 * entries with fewer than EEC_GATHER_HEAVY contributions are sorted by their count (ties in entry
 * order) and dealt to groups of 32, each group stored column-major over 32 x (1 + its largest
 * count) items (zeros past an entry's end); the other entries' runs follow all windows,
 * contiguous. Outputs (each nullable, host):
 *  item_of [n_entries]   item of entry e's linear part
 *  step_of [n_entries]   distance between entry e's consecutive items (32 or 1)
 *  woff    [n_win * 33]  n_win = ceil(n_entries / EEC_GATHER_WINDOW): per window the first item
 *                        of each of its 32 groups, then the window's end
 *  loc     [n_win * EEC_GATHER_WINDOW]  per window and slot 32 g + i: entry - w * EEC_GATHER_WINDOW,
 *                        or 0xffff for an empty slot
 *  heavy   [3 * n_heavy] per entry with EEC_GATHER_HEAVY or more contributions, in entry order:
 *                        entry, first item, items
 *  *n_items              the buffer's length in items
 * Returns EEC_EINVAL for a negative count, more than 2^31 - 1 entries, or a plan longer than
 * 2^31 - 1 items.
 */
#define EEC_GATHER_WINDOW 1024
#define EEC_GATHER_HEAVY 32
EEC_API int eec_gather_plan_host(int64_t n_entries, const int32_t* cnt, int64_t* item_of,
                                 int32_t* step_of, int32_t* woff, uint16_t* loc, int32_t* heavy,
                                 int64_t* n_items);

/*
 * Transient companion stamp of one Newton iterate of a time step (the transient loop of Sec. II,
 * Fig. 1, re-forms A x = b at every Newton iteration of every step). The terminal charges q_t
 * are integrated by a one-step rule: the capacitive current into the device is
 *   ic_t = alpha (q_t(x) - q_prev_t) - beta i_prev_t
 * (backward Euler: alpha = 1/h, beta = 0; trapezoidal: alpha = 2/h, beta = 1), and
 *   A = A_lin + sum_dev (G + alpha C),  b = b_lin + sum_dev (-I - ic + (G + alpha C) V)
 * with C_tu = dq_t/dV_u, over all four terminal rows (the gate row now carries current).
 *  q_prev_dev  [4*n_dev] charges at the previous time point (terminal-major, original order),
 *  i_prev_dev  [4*n_dev] capacitive currents there, nullable (zero);
 *  q_dev       [4*n_dev] out: charges at x;  i_dev [4*n_dev] out, nullable: ic at x.
 * Schedule: the per-colour store-add when the variant is EEC_VARIANT_COLOR_FUSED; every device
 * into a buffer, then a colour-ordered stamp by one thread-block cluster, when it is
 * EEC_VARIANT_COLOR_BUFFERED; the pipelined colour order in one launch when it is
 * EEC_VARIANT_COLOR_PIPELINED (the three need a colouring that counts gate rows: not
 * EEC_CONFLICT_WRITE_ROWS); otherwise FP64 atomics.
 */
EEC_API int eec_eval_stamp_tran(eec_ctx* ctx, const double* x_dev, const double* q_prev_dev,
                                const double* i_prev_dev, double alpha, double beta,
                                double* A_values_dev, double* b_dev, double* q_dev, double* i_dev,
                                void* cuda_stream);

/*
 * Gradient of s = sum_e gA[e] A[e] + sum_i gb[i] b[i], with A, b formed at x, with respect to
 * x and to every device's W and L. Read-only gathers (the transpose of the scatter): one pass
 * per device produces terminal and parameter gradients, one pass per unknown gathers them.
 *  gA_dev [nnz], gb_dev [n] in; gx_dev [n], gW_dev [n_dev], gL_dev [n_dev] out (original order).
 */
EEC_API int eec_eval_stamp_bwd(eec_ctx* ctx, const double* x_dev, const double* gA_dev,
                       const double* gb_dev, double* gx_dev, double* gW_dev, double* gL_dev,
                       void* cuda_stream);

/*
 * eec_eval_stamp_bwd_noalloc: the same gradients as eec_eval_stamp_bwd, computed by the same
 * kernels, for callers that cannot allocate device memory. Typical callers: an application whose
 * GPU memory is entirely reserved by its own allocator (a framework's caching pool, a fixed
 * arena), so a cudaMalloc from inside this library would fail or break its accounting; and a
 * latency-critical loop that cannot afford the device-wide synchronisation cudaMalloc and cudaFree
 * can cause. The paper has no counterpart; this is a property of the library interface only.
 *
 * The backward's per-device scratch (four terminal gradients per device, written by the first
 * pass and gathered by the second) lives in one fixed array compiled into the library instead of
 * a buffer allocated on first use. The call makes no cudaMalloc, cudaFree or other allocating
 * call; the caller passes every input and output as in eec_eval_stamp_bwd.
 *  - Limit: the context may hold at most EEC_NOALLOC_MAX_DEV devices (the array is
 *    4 * EEC_NOALLOC_MAX_DEV doubles = 16 MiB); larger contexts are rejected with EEC_EINVAL.
 *  - The array exists on every GPU on which the library's backward module is loaded and stays
 *    allocated until the process exits. eec_build_scatter loads that module on the current
 *    device and looks up the array's device address there (cudaGetSymbolAddress with that device
 *    current), so a context built on a device has the array ready before this entry point's
 *    first call. A first call on a device where no context was built does that set-up itself;
 *    make such a call before any stream capture.
 *  - Every call, from any context, shares the array, and it keeps the last call's contents. Each
 *    call writes every entry it later reads, so nothing needs clearing, but calls whose work
 *    overlaps on the GPU (e.g. on two streams without ordering between them) race on it.
 */
#define EEC_NOALLOC_MAX_DEV 524288
EEC_API int eec_eval_stamp_bwd_noalloc(eec_ctx* ctx, const double* x_dev, const double* gA_dev,
                                       const double* gb_dev, double* gx_dev, double* gW_dev,
                                       double* gL_dev, void* cuda_stream);

/*
 * Capture the current variant's eval_stamp on these buffers into a CUDA graph owned by ctx
 * (replacing any previous one); eec_graph_launch() then replays it on any stream.
 */
EEC_API int eec_graph_capture(eec_ctx* ctx, const double* x_dev, double* A_values_dev, double* b_dev,
                      double* q_dev, void* cuda_stream);
EEC_API int eec_graph_launch(eec_ctx* ctx, void* cuda_stream);

/*
 * Autotuner: time every schedule on these buffers (CUDA events, `reps` calls each after one
 * warm-up), at block sizes 0 (library choice), 32, 64 and 128 unless opt.block fixes it, and
 * for the order-free schedules (ATOMIC, SEGREDUCE, COLOR_BUFFERED) in both evaluation launch
 * orders (devices with a free source or body first, or layout order); select the fastest
 * combination for eec_eval_stamp when the variant is EEC_VARIANT_AUTO (the launch order applies
 * whatever the variant). ms_out [EEC_N_VARIANTS] (nullable) receives each schedule's best mean time
 * per call, negative for a schedule that does not apply (colour schedules without colours).
 * Synchronous.
 */
EEC_API int eec_autotune(eec_ctx* ctx, const double* x_dev, double* A_values_dev, double* b_dev,
                 double* q_dev, int32_t reps, void* cuda_stream, float* ms_out);

/*
 * Synchronise cuda_stream, read and clear the device status word. Returns 0 when no device-side
 * error was recorded, else EEC_ETIMEOUT (a grid barrier gave up waiting) or EEC_ENUMERIC.
 */
EEC_API int eec_status(eec_ctx* ctx, void* cuda_stream);

/*
 * Phase timing, the t_calc / t_stamp split of the paper's Fig. 5. While enabled, every
 * eec_eval_stamp records CUDA events on the caller's stream around its three phases (copy of the
 * linear part into A/b, evaluate — which includes the store-add in the fused schedules — and the
 * separate stamp pass of the buffered schedules) and launches without CUDA graphs.
 * eec_profile_read synchronises the recorded events, returns the accumulated milliseconds per
 * phase over the calls since the last read (any pointer may be NULL) and resets the sums.
 * n_kernels counts the library's kernel launches (graph replays count their kernel nodes) since
 * the last read, whether or not timing is enabled.
 */
EEC_API int eec_profile_enable(eec_ctx* ctx, int32_t enable);
EEC_API int eec_profile_read(eec_ctx* ctx, double* ms_init, double* ms_eval, double* ms_stamp,
                             int64_t* n_calls, int64_t* n_kernels);

/* Sizes of the built context: devices, unknowns, nnz, colours (0 when not coloured). */
EEC_API int eec_get_sizes(const eec_ctx* ctx, int32_t* n_dev, int32_t* n_unknowns, int64_t* nnz,
                  int32_t* n_colors);

/*
 * Batched form: the disjoint union of n_circ netlists as one context whose A is block diagonal
 * (circuit k owns unknowns circ_row_off[k] .. circ_row_off[k+1]-1 and CSR values
 * circ_nnz_off[k] .. circ_nnz_off[k+1]-1). Each circuit is described by the same arrays as
 * eec_upload_netlist, passed as arrays of per-circuit pointers; node 0 of every circuit is the
 * shared ground. Greedy colouring of the union in natural order colours every circuit on its own
 * and merges colour c of all circuits into one phase.
 */
typedef struct {
  int32_t n_nodes;
  const uint8_t* node_fixed;
  const double* node_vfix;
  int32_t n_dev;
  const int32_t* dev_nodes;
  const int8_t* dev_type;
  const double* W;
  const double* L;
  const int32_t* model_id;
  int32_t n_res;
  const int32_t* res_nodes;
  const double* res_G;
  int32_t n_isrc;
  const int32_t* isrc_nodes;
  const double* isrc_val;
} eec_netlist;

EEC_API int eec_upload_batch(eec_ctx* ctx, int32_t n_circ, const eec_netlist* nets, double gshunt);

/* A batched context in one call: eec_create(opt) then eec_upload_batch of the circuits
 * *nets[0] .. *nets[n_circ-1] (an array of pointers; each eec_netlist is copied). On failure
 * *out is NULL and nothing is left allocated. */
EEC_API int eec_batch_create(eec_ctx** out, int32_t n_circ, const eec_netlist* const* nets,
                             double gshunt, const eec_options* opt);

/* From this call on, eec_eval_stamp on ctx replays one CUDA graph of the whole step for every
 * schedule (the colour schedules always do): the graph is captured at the first call with a
 * given x, A, b, q and re-captured when those pointers, the schedule, the block size or the
 * launch order change. The batched pipeline of many small circuits is launch-bound, and a
 * replay issues the step's kernels as one submission. cuda_stream (nullable) is synchronised
 * first, so that no launch of the context is in flight while the mode changes. */
EEC_API int eec_batch_capture_graph(eec_ctx* ctx, void* cuda_stream);

/* After eec_build_scatter on a batch: circ_row_off [n_circ+1], circ_nnz_off [n_circ+1],
 * circ_dev_off [n_circ+1] (first device of each circuit in original order). */
EEC_API int eec_get_batch_offsets(const eec_ctx* ctx, int32_t* circ_row_off, int64_t* circ_nnz_off,
                          int32_t* circ_dev_off);

/*
 * FP64 fused-multiply-add throughput probe: `iters` iterations of 8 independent DFMA chains per
 * thread over a grid of blocks_per_sm * SMs blocks. Writes the measured DFMA rate (FLOP/s,
 * 2 per DFMA) to *flops. Synchronous; used to report the FP64 roofline.
 */
EEC_API int eec_fp64_peak(int32_t iters, int32_t blocks_per_sm, double* flops);

/*
 * Test hook for the failure path of the device-side waits (the paper has no counterpart). When
 * the context's schedule is EEC_VARIANT_COLOR_PIPELINED it launches the pipelined kernel with the
 * first work item never reporting its stamps done, so the next colour's waits run out; otherwise
 * it launches the persistent kernel with one block that never arrives at the grid barriers. The
 * waits give up after their 1 s limit and the status word records EEC_ETIMEOUT (read it with
 * eec_status). Nothing faults or hangs; A and b are left partially stamped. Needs a coloured
 * context with at least two (non-empty) colours.
 */
EEC_API int eec_test_barrier_timeout(eec_ctx* ctx, const double* x_dev, double* A_values_dev,
                                     double* b_dev, void* cuda_stream);

/*
 * Validation hook for the library's own FP64 elementary functions (the table-driven exp, expm1
 * and log1p, and the reciprocal and reciprocal square root, that the model evaluation uses in
 * place of CUDA's). The paper has no counterpart.
 *  fn      0 = exp, 1 = expm1, 2 = log1p (argument in [0, 1], the only range the model uses),
 *          3 = 1/x, 4 = 1/sqrt(x) (normal |x| in [2^-126, 2^128); x > 0 for 4).
 *  x_dev   [n] arguments; ours_dev [n] the library's results; cuda_dev [n] CUDA's exp / expm1 /
 *          log1p / 1.0/x / rsqrt of the same arguments. Asynchronous on cuda_stream.
 */
EEC_API int eec_math_check(int32_t fn, int64_t n, const double* x_dev, double* ours_dev,
                           double* cuda_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* EEC_H_ */
