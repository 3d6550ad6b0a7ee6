/* A plain C99 caller of the whole path on the GPU: device buffers from cudaMalloc, the
 * evaluate-and-stamp of every schedule through include/eec.h, and A, b compared entry by entry
 * with the CPU oracle (linked here through its own C interface; test infrastructure). The
 * netlist is an 8-stage inverter chain with VDD and the input held. Prints "ok" and exits 0 on
 * success; without a GPU it checks the CSR pattern against the oracle's and exits 77. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "eec.h"

/* the oracle's C interface (oracle/oracle.cpp) */
void* ora_create(int32_t n_nodes, const uint8_t* node_fixed, const double* node_vfix,
                 int32_t n_dev, const int32_t* dev_nodes, const int8_t* dev_type, const double* W,
                 const double* L, const int32_t* model_id, int32_t n_res, const int32_t* res_nodes,
                 const double* res_G, int32_t n_isrc, const int32_t* isrc_nodes,
                 const double* isrc_val, double gshunt, int32_t n_cards, const double* cards,
                 int32_t rail_mode);
void ora_destroy(void* h);
int32_t ora_n_unknowns(void* h);
int64_t ora_nnz(void* h);
int ora_pattern(void* h, int32_t* row_ptr, int32_t* col, int32_t* unk_of_node);
int ora_eval_stamp(void* h, const double* x, double* A, double* b, double* q, double* A_scale,
                   double* b_scale);

#define STAGES 8
#define NODES (3 + STAGES)
#define DEVS (2 * STAGES)

static void card(double* c, int nmos) {
  /* VTH0 K1 PHI NFACT U0 UA UB VSAT TOX ETA0 DELTA LAMBDA LREF JS HDIF CGSO CGDO XPART D1 GMIN TEMP */
  const double v[EEC_CARD_LEN] = {0.4, 0.5, 0.8, 1.3, nmos ? 0.04 : 0.012, 1e-9, 1e-19, 1e5,
                                  2e-9, 0.05, 0.01, 0.05, 1e-7, 1e-4, 1e-7, 3e-10, 3e-10,
                                  0.4, 0.01, 1e-12, 300.0};
  memcpy(c, v, sizeof v);
}

#define CUDA_OK(call)                                                   \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) {                                            \
      fprintf(stderr, "%s: %s\n", #call, cudaGetErrorString(e_));       \
      return 10;                                                        \
    }                                                                   \
  } while (0)

int main(void) {
  /* nodes: 0 ground, 1 VDD (held), 2 input (held), 3.. stage outputs */
  uint8_t fixed[NODES] = {0};
  double vfix[NODES] = {0.0};
  int32_t dn[DEVS * 4];
  int8_t type[DEVS];
  double W[DEVS], L[DEVS];
  int32_t mid[DEVS];
  double cards[2 * EEC_CARD_LEN];
  fixed[0] = fixed[1] = fixed[2] = 1;
  vfix[1] = 1.0;
  vfix[2] = 0.35;
  for (int s = 0; s < STAGES; ++s) {
    const int in = s == 0 ? 2 : 2 + s, out = 3 + s;
    const int32_t nm[4] = {out, in, 0, 0}, pm[4] = {out, in, 1, 1};
    memcpy(dn + 8 * s, nm, sizeof nm);
    memcpy(dn + 8 * s + 4, pm, sizeof pm);
    type[2 * s] = 1;
    type[2 * s + 1] = -1;
    W[2 * s] = 1e-6 * (1.0 + 0.1 * s);
    W[2 * s + 1] = 2e-6 * (1.0 + 0.05 * s);
    L[2 * s] = L[2 * s + 1] = 1e-7 * (1.0 + 0.02 * s);
    mid[2 * s] = 0;
    mid[2 * s + 1] = 1;
  }
  card(cards, 1);
  card(cards + EEC_CARD_LEN, 0);

  eec_ctx* ctx = NULL;
  if (eec_create(&ctx, NULL) != EEC_OK) return 2;
  if (eec_upload_netlist(ctx, NODES, fixed, vfix, DEVS, dn, type, W, L, mid, 0, NULL, NULL, 0,
                         NULL, NULL, 1e-12) != EEC_OK ||
      eec_set_model_cards(ctx, 2, cards) != EEC_OK) {
    fprintf(stderr, "setup: %s\n", eec_last_error(ctx));
    return 3;
  }
  int32_t C = 0, n = 0;
  int64_t nnz = 0;
  if (eec_color(ctx, NULL, EEC_COLOR_GREEDY_SEQ, NULL, &C) != EEC_OK) return 4;
  /* without a GPU the host part (pattern) is still built: checked below, then exit 77 */
  const int rc_build = eec_build_scatter(ctx, &n, &nnz);
  if (rc_build != EEC_OK && rc_build != EEC_ECUDA) {
    fprintf(stderr, "scatter: %s\n", eec_last_error(ctx));
    return 4;
  }
  if (rc_build == EEC_ECUDA &&
      eec_get_sizes(ctx, NULL, &n, &nnz, NULL) != EEC_OK) return 4;
  void* o = ora_create(NODES, fixed, vfix, DEVS, dn, type, W, L, mid, 0, NULL, NULL, 0, NULL, NULL,
                       1e-12, 2, cards, 0);
  if (!o || ora_n_unknowns(o) != n || ora_nnz(o) != nnz) return 5;
  int32_t rp[NODES + 1], orp[NODES + 1];
  int32_t* col = malloc(sizeof(int32_t) * (size_t)nnz);
  int32_t* ocol = malloc(sizeof(int32_t) * (size_t)nnz);
  double* x = malloc(sizeof(double) * (size_t)n);
  double* A = malloc(sizeof(double) * (size_t)nnz);
  double* Ao = malloc(sizeof(double) * (size_t)nnz);
  double* As = malloc(sizeof(double) * (size_t)nnz);
  double* b = malloc(sizeof(double) * (size_t)n);
  double* bo = malloc(sizeof(double) * (size_t)n);
  double* bs = malloc(sizeof(double) * (size_t)n);
  if (!col || !ocol || !x || !A || !Ao || !As || !b || !bo || !bs) return 6;
  if (eec_get_pattern(ctx, rp, col, NULL) != EEC_OK || ora_pattern(o, orp, ocol, NULL) != 0) return 7;
  if (memcmp(rp, orp, sizeof(int32_t) * (size_t)(n + 1)) != 0 ||
      memcmp(col, ocol, sizeof(int32_t) * (size_t)nnz) != 0) {
    fprintf(stderr, "pattern differs from the oracle's\n");
    return 8;
  }
  for (int i = 0; i < n; ++i) x[i] = 0.05 + 0.9 * (double)((i * 37) % 17) / 16.0;
  ora_eval_stamp(o, x, Ao, bo, NULL, As, bs);
  if (rc_build == EEC_ECUDA) {
    printf("no GPU: pattern checked\n");
    return 77;
  }

  double *dx = NULL, *dA = NULL, *db = NULL, *dq = NULL;
  CUDA_OK(cudaMalloc((void**)&dx, sizeof(double) * (size_t)n));
  CUDA_OK(cudaMalloc((void**)&dA, sizeof(double) * (size_t)nnz));
  CUDA_OK(cudaMalloc((void**)&db, sizeof(double) * (size_t)n));
  CUDA_OK(cudaMalloc((void**)&dq, sizeof(double) * 4 * DEVS));
  CUDA_OK(cudaMemcpy(dx, x, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice));
  double worst = 0.0;
  for (int v = 0; v < EEC_N_VARIANTS; ++v) {
    if (eec_set_variant(ctx, v) != EEC_OK || eec_eval_stamp(ctx, dx, dA, db, dq, NULL) != EEC_OK ||
        eec_status(ctx, NULL) != EEC_OK) {
      fprintf(stderr, "schedule %d: %s\n", v, eec_last_error(ctx));
      return 9;
    }
    CUDA_OK(cudaMemcpy(A, dA, sizeof(double) * (size_t)nnz, cudaMemcpyDeviceToHost));
    CUDA_OK(cudaMemcpy(b, db, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < nnz; ++k) {
      const double den = fmax(fmax(fabs(Ao[k]), As[k]), 1e-300);
      const double e = fabs(A[k] - Ao[k]) / den;
      if (e > worst) worst = e;
    }
    for (int i = 0; i < n; ++i) {
      const double den = fmax(fmax(fabs(bo[i]), bs[i]), 1e-300);
      const double e = fabs(b[i] - bo[i]) / den;
      if (e > worst) worst = e;
    }
  }
  cudaFree(dx);
  cudaFree(dA);
  cudaFree(db);
  cudaFree(dq);
  ora_destroy(o);
  eec_destroy(ctx);
  free(col);
  free(ocol);
  free(x);
  free(A);
  free(Ao);
  free(As);
  free(b);
  free(bo);
  free(bs);
  if (!(worst <= 1e-12)) {
    fprintf(stderr, "max relative error %g\n", worst);
    return 11;
  }
  printf("ok\n");
  return 0;
}
