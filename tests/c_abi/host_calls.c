/* A plain C99 caller of the library: compiles against include/eec.h alone and links against
 * _libeec.so. Runs the host-side calls (no GPU needed): options, create, upload of a
 * three-stage inverter chain, model cards, greedy colouring, then checks the colour count and
 * the error paths. Prints "ok" and exits 0 on success. */
#include <stdio.h>
#include <string.h>

#include "eec.h"

static double card(double* c, int nmos) {
  /* VTH0 K1 PHI NFACT U0 UA UB VSAT TOX ETA0 DELTA LAMBDA LREF JS HDIF CGSO CGDO XPART D1 GMIN TEMP */
  const double v[EEC_CARD_LEN] = {0.4, 0.5, 0.8, 1.3, nmos ? 0.04 : 0.012, 1e-9, 1e-19, 1e5,
                                  2e-9, 0.05, 0.01, 0.05, 1e-7, 1e-4, 1e-7, 3e-10, 3e-10,
                                  0.4, 0.01, 1e-12, 300.0};
  memcpy(c, v, sizeof v);
  return c[0];
}

int main(void) {
  /* nodes: 0 ground, 1 VDD (held), 2 input (held), 3..5 stage outputs */
  const int32_t n_nodes = 6;
  const uint8_t fixed[6] = {1, 1, 1, 0, 0, 0};
  const double vfix[6] = {0.0, 1.0, 0.5, 0.0, 0.0, 0.0};
  int32_t dn[6 * 4];
  int8_t type[6];
  double W[6], L[6];
  int32_t mid[6];
  for (int s = 0; s < 3; ++s) {
    const int in = s == 0 ? 2 : 2 + s, out = 3 + s;
    const int32_t nm[4] = {out, in, 0, 0}, pm[4] = {out, in, 1, 1};
    memcpy(dn + 8 * s, nm, sizeof nm);
    memcpy(dn + 8 * s + 4, pm, sizeof pm);
    type[2 * s] = 1;
    type[2 * s + 1] = -1;
    W[2 * s] = 1e-6;
    W[2 * s + 1] = 2e-6;
    L[2 * s] = L[2 * s + 1] = 1e-7;
    mid[2 * s] = 0;
    mid[2 * s + 1] = 1;
  }
  double cards[2 * EEC_CARD_LEN];
  card(cards, 1);
  card(cards + EEC_CARD_LEN, 0);

  eec_options opt = eec_default_options();
  if (opt.variant != EEC_VARIANT_AUTO || opt.block != 0 || opt.rail_mode != EEC_RAIL_ELIMINATE) return 1;
  eec_ctx* ctx = NULL;
  if (eec_create(&ctx, &opt) != EEC_OK || !ctx) return 2;
  if (eec_upload_netlist(ctx, n_nodes, fixed, vfix, 6, dn, type, W, L, mid, 0, NULL, NULL, 0,
                         NULL, NULL, 1e-12) != EEC_OK) {
    fprintf(stderr, "upload: %s\n", eec_last_error(ctx));
    return 3;
  }
  if (eec_set_model_cards(ctx, 2, cards) != EEC_OK) return 4;
  int32_t colors[6], C = 0;
  if (eec_color(ctx, NULL, EEC_COLOR_GREEDY_SEQ, colors, &C) != EEC_OK) return 5;
  /* stage s shares its output with stage s + 1's gate: two devices per stage, chains of
     conflicts, so the greedy colouring needs 4 colours (as the 64-stage chain) */
  if (C != 4) {
    fprintf(stderr, "colours: %d\n", (int)C);
    return 6;
  }
  /* error paths: a bad card count and an unknown variant are rejected with a message */
  if (eec_set_model_cards(ctx, 0, cards) != EEC_EINVAL) return 7;
  if (eec_set_variant(ctx, 99) != EEC_EINVAL || strlen(eec_last_error(ctx)) == 0) return 8;
  eec_destroy(ctx);
  eec_destroy(NULL);
  printf("ok\n");
  return 0;
}
