// Serial CPU oracle for the per-Newton-iteration MOSFET evaluation and MNA stamping of EEspice.
//
// TEST INFRASTRUCTURE ONLY. The test-suite, the smoke check and the bench's CPU-baseline leg are
// the only code that may load this library; the product path never does. It shares no code with
// the CUDA library: its model is written once, templated on a scalar, and its Jacobian comes from
// forward-mode dual numbers instead of hand-derived chain rules.
//
// What it computes (paper sections cited by number):
//  * Sec. I / Sec. II (i)-(ii): each Newton-Raphson iteration evaluates every device at the
//    present node voltages ("compute phase") and accumulates its linearised contributions into
//    the MNA matrix A and right-hand side b ("stamp phase"); A x = b is then solved.
//  * Sec. I, Sec. II: the conflict graph (devices are adjacent when they share a node that is not
//    ground) and greedy colouring in a given vertex order (smallest colour unused by already
//    coloured neighbours).
//  * The device model: the paper evaluates BSIM4 v4.82 (Sec. II) but prints no equations; the
//    oracle implements the documented BSIM-style level EES-L1 (mode swap, body effect, softplus
//    effective overdrive, mobility degradation, velocity saturation, smooth Vdseff, channel-length
//    modulation, junction diodes, charge partition). Equations are restated next to the code.
//  * Rails (nodes held by an ideal voltage source) are either eliminated (their voltages enter
//    b) or, in modified nodal analysis (Sec. I builds on MNA), kept as unknowns with one extra
//    unknown per source: its current, with the KCL entry at the rail and the source equation.
//  * The DC Newton loop with a dense LU, the adjoint (transpose) solve and the gradient of a
//    linear functional of (A, b) use no paper equation; they follow textbook definitions.
//  * The same model evaluated on an operation-counting scalar gives the algorithmic work of one
//    device evaluation by operation class (ora_count_ops).
//
// Parity pins (checked by the "not gpu" tests): resistor divider and diode Lambert-W closed forms,
// KCL residual A x - b = F(x), symmetric pattern, model invariants and limits, Jacobian vs central
// differences, brute-force colouring on tiny graphs and hand-derived colour counts; with the rails
// as unknowns, the divider's source current in closed form and source currents equal to minus the
// model's terminal currents.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <utility>
#include <vector>

namespace {

// ---------------------------------------------------------------------------------------------
// Forward-mode dual numbers: value plus N partial derivatives; T may itself be a Dual (nesting
// gives mixed second derivatives).
template <class T, int N>
struct Dual {
  T v;
  T d[N];
  Dual() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = T(0.0); }
  Dual(double c) : v(c) { for (int i = 0; i < N; ++i) d[i] = T(0.0); }  // NOLINT: constants
};

inline double val(double x) { return x; }
template <class T, int N>
double val(const Dual<T, N>& x) { return val(x.v); }

template <class T, int N>
Dual<T, N> operator+(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r; r.v = a.v + b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <class T, int N>
Dual<T, N> operator-(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r; r.v = a.v - b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <class T, int N>
Dual<T, N> operator-(const Dual<T, N>& a) {
  Dual<T, N> r; r.v = -a.v;
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <class T, int N>
Dual<T, N> operator*(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r; r.v = a.v * b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <class T, int N>
Dual<T, N> operator/(const Dual<T, N>& a, const Dual<T, N>& b) {
  Dual<T, N> r; r.v = a.v / b.v;
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
  return r;
}
// Mixed operands with a plain double.
template <class T, int N> Dual<T, N> operator+(const Dual<T, N>& a, double b) { return a + Dual<T, N>(b); }
template <class T, int N> Dual<T, N> operator+(double a, const Dual<T, N>& b) { return Dual<T, N>(a) + b; }
template <class T, int N> Dual<T, N> operator-(const Dual<T, N>& a, double b) { return a - Dual<T, N>(b); }
template <class T, int N> Dual<T, N> operator-(double a, const Dual<T, N>& b) { return Dual<T, N>(a) - b; }
template <class T, int N> Dual<T, N> operator*(const Dual<T, N>& a, double b) { return a * Dual<T, N>(b); }
template <class T, int N> Dual<T, N> operator*(double a, const Dual<T, N>& b) { return Dual<T, N>(a) * b; }
template <class T, int N> Dual<T, N> operator/(const Dual<T, N>& a, double b) { return a / Dual<T, N>(b); }
template <class T, int N> Dual<T, N> operator/(double a, const Dual<T, N>& b) { return Dual<T, N>(a) / b; }

using std::exp;
using std::expm1;
using std::log1p;
using std::sqrt;

template <class T, int N>
Dual<T, N> exp(const Dual<T, N>& a) {
  Dual<T, N> r; r.v = exp(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = r.v * a.d[i];
  return r;
}
template <class T, int N>
Dual<T, N> expm1(const Dual<T, N>& a) {
  Dual<T, N> r; r.v = expm1(a.v);
  T e = exp(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = e * a.d[i];
  return r;
}
template <class T, int N>
Dual<T, N> log1p(const Dual<T, N>& a) {
  Dual<T, N> r; r.v = log1p(a.v);
  T s = 1.0 + a.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / s;
  return r;
}
template <class T, int N>
Dual<T, N> sqrt(const Dual<T, N>& a) {
  Dual<T, N> r; r.v = sqrt(a.v);
  T s = 2.0 * r.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / s;
  return r;
}

// Operation counting: a scalar that counts the floating-point operations of one model
// evaluation (values only, no derivatives) that depend on the terminal voltages. A value derived
// only from the card, W and L is a per-device constant (a GPU computes it once per device or
// card), and operations among constants are not counted.
struct OpCount {
  long long add = 0, mul = 0, div = 0, exp = 0, expm1 = 0, log1p = 0, sqrt = 0;
};
OpCount g_ops;   // one counting evaluation at a time
struct Cnt {
  double v;
  bool dep;      // depends on the terminal voltages
  Cnt() : v(0.0), dep(false) {}
  Cnt(double c) : v(c), dep(false) {}  // NOLINT: constants
  Cnt(double c, bool d) : v(c), dep(d) {}
};
inline double val(const Cnt& x) { return x.v; }
inline Cnt cnt2(double v, const Cnt& a, const Cnt& b, long long* k) {
  if (a.dep || b.dep) ++*k;
  return Cnt(v, a.dep || b.dep);
}
inline Cnt operator+(const Cnt& a, const Cnt& b) { return cnt2(a.v + b.v, a, b, &g_ops.add); }
inline Cnt operator-(const Cnt& a, const Cnt& b) { return cnt2(a.v - b.v, a, b, &g_ops.add); }
inline Cnt operator*(const Cnt& a, const Cnt& b) { return cnt2(a.v * b.v, a, b, &g_ops.mul); }
inline Cnt operator/(const Cnt& a, const Cnt& b) { return cnt2(a.v / b.v, a, b, &g_ops.div); }
inline Cnt operator-(const Cnt& a) { return Cnt(-a.v, a.dep); }   // a sign flip, not counted
inline Cnt operator+(const Cnt& a, double b) { return a + Cnt(b); }
inline Cnt operator+(double a, const Cnt& b) { return Cnt(a) + b; }
inline Cnt operator-(const Cnt& a, double b) { return a - Cnt(b); }
inline Cnt operator-(double a, const Cnt& b) { return Cnt(a) - b; }
inline Cnt operator*(const Cnt& a, double b) { return a * Cnt(b); }
inline Cnt operator*(double a, const Cnt& b) { return Cnt(a) * b; }
inline Cnt operator/(const Cnt& a, double b) { return a / Cnt(b); }
inline Cnt operator/(double a, const Cnt& b) { return Cnt(a) / b; }
inline Cnt cnt1(double v, const Cnt& a, long long* k) {
  if (a.dep) ++*k;
  return Cnt(v, a.dep);
}
inline Cnt exp(const Cnt& a) { return cnt1(std::exp(a.v), a, &g_ops.exp); }
inline Cnt expm1(const Cnt& a) { return cnt1(std::expm1(a.v), a, &g_ops.expm1); }
inline Cnt log1p(const Cnt& a) { return cnt1(std::log1p(a.v), a, &g_ops.log1p); }
inline Cnt sqrt(const Cnt& a) { return cnt1(std::sqrt(a.v), a, &g_ops.sqrt); }

// ---------------------------------------------------------------------------------------------
// EES-L1 model card (field order fixed by the card layout of the interface).
struct Card {
  double VTH0, K1, PHI, NFACT, U0, UA, UB, VSAT, TOX, ETA0, DELTA, LAMBDA, LREF, JS, HDIF, CGSO,
      CGDO, XPART, D1, GMIN, TEMP;
};
constexpr int kCardLen = 21;

Card read_card(const double* c) {
  Card k;
  k.VTH0 = c[0]; k.K1 = c[1]; k.PHI = c[2]; k.NFACT = c[3]; k.U0 = c[4]; k.UA = c[5];
  k.UB = c[6]; k.VSAT = c[7]; k.TOX = c[8]; k.ETA0 = c[9]; k.DELTA = c[10]; k.LAMBDA = c[11];
  k.LREF = c[12]; k.JS = c[13]; k.HDIF = c[14]; k.CGSO = c[15]; k.CGDO = c[16]; k.XPART = c[17];
  k.D1 = c[18]; k.GMIN = c[19]; k.TEMP = c[20];
  return k;
}

// Physical constants (CODATA 2018 exact SI values; vacuum permittivity 2018 recommended value).
constexpr double kBoltzmann = 1.380649e-23;      // J/K
constexpr double kCharge = 1.602176634e-19;      // C
constexpr double kEps0 = 8.8541878128e-12;       // F/m
constexpr double kEpsRelOx = 3.9;                // SiO2

// softplus(z) = max(z, 0) + log(1 + exp(-|z|)), evaluated without overflow.
template <class S>
S softplus(const S& z) {
  if (val(z) >= 0.0) return z + log1p(exp(-z));
  return log1p(exp(z));
}

// expm1 with the exponential continued linearly above z = 40 (junction current limiting):
// z <= 40: exp(z) - 1; z > 40: e^40 (1 + z - 40) - 1.
template <class S>
S explim_m1(const S& z) {
  if (val(z) <= 40.0) return expm1(z);
  return (std::exp(40.0) - 1.0) + std::exp(40.0) * (z - 40.0);
}

// EES-L1 terminal currents I[t] (current flowing from node t into the device, t = d, g, s, b)
// and terminal charges Q[t], for polarity p (+1 NMOS, -1 PMOS) at terminal voltages V[t].
template <class S>
void ees_l1(const Card& c, int p, const S& W, const S& L, const S V[4], S I[4], S Q[4]) {
  const double Vt = kBoltzmann * c.TEMP / kCharge;
  const double Cox = kEpsRelOx * kEps0 / c.TOX;
  const double pp = static_cast<double>(p);

  // (1) Mode: source/drain are swapped when p (Vd - Vs) < 0; a tie keeps the forward mode.
  const S vds0 = pp * (V[0] - V[2]);
  const int mode = (val(vds0) >= 0.0) ? 1 : -1;
  const int iD = (mode > 0) ? 0 : 2;
  const int iS = (mode > 0) ? 2 : 0;
  const S vgs = pp * (V[1] - V[iS]);
  const S vds = pp * (V[iD] - V[iS]);
  const S vbs = pp * (V[3] - V[iS]);

  // (2) Body effect: phis = smooth max(PHI - vbs, 0) with width D1 (written without
  //     cancellation for negative argument), Vth with DIBL.
  const S u = c.PHI - vbs;
  const S R1 = sqrt(u * u + 4.0 * c.D1 * c.D1);
  const S phis = (val(u) >= 0.0) ? 0.5 * (u + R1) : (2.0 * c.D1 * c.D1) / (R1 - u);
  const S sqs = sqrt(phis);
  const S Vth = c.VTH0 + c.K1 * (sqs - std::sqrt(c.PHI)) - c.ETA0 * vds;

  // (3) Effective overdrive, continuous from subthreshold to strong inversion.
  const double nVt = c.NFACT * Vt;
  const S Vgsteff = nVt * softplus((vgs - Vth) / nVt);

  // (4) Bulk-charge factor.
  const S Abulk = 1.0 + c.K1 / (2.0 * sqs);

  // (5) Mobility degradation.
  const S mueff = c.U0 / (1.0 + c.UA * Vgsteff + c.UB * Vgsteff * Vgsteff);

  // (6) Velocity saturation and saturation voltage.
  const S EsatL = 2.0 * c.VSAT * L / mueff;
  const S Vgst2 = Vgsteff + 2.0 * Vt;
  const S Vdsat = EsatL * Vgst2 / (Abulk * EsatL + Vgst2);

  // (7) Smooth min(vds, Vdsat): Vdsat - (t + sqrt(t^2 + 4 DELTA Vdsat))/2, t = Vdsat - vds - DELTA,
  //     written in the algebraically identical cancellation-free form.
  const S t = Vdsat - vds - c.DELTA;
  const S R2 = sqrt(t * t + 4.0 * c.DELTA * Vdsat);
  const S Vdseff = 2.0 * Vdsat * vds / (Vdsat + vds + c.DELTA + R2);

  // (8) Drain current with channel-length modulation.
  const S beta = mueff * Cox * W / L;
  const S F1 = 1.0 - Abulk * Vdseff / (2.0 * Vgst2);
  const S Ids0 = beta * Vgsteff * Vdseff * F1 / (1.0 + Vdseff / EsatL);
  const S Ids = Ids0 * (1.0 + c.LAMBDA * (c.LREF / L) * (vds - Vdseff));

  // (9) Channel current into the physical terminals.
  const S Ichd = pp * static_cast<double>(mode) * Ids;
  const S Ichs = -Ichd;

  // (10) Junction diodes body-drain and body-source, on the physical terminals.
  const S vbd = pp * (V[3] - V[0]);
  const S vbsj = pp * (V[3] - V[2]);
  const S Isat = c.JS * W * c.HDIF;
  const S Ijd = Isat * explim_m1(vbd / Vt) + c.GMIN * vbd;
  const S Ijs = Isat * explim_m1(vbsj / Vt) + c.GMIN * vbsj;

  I[0] = Ichd - pp * Ijd;
  I[1] = S(0.0);
  I[2] = Ichs - pp * Ijs;
  I[3] = pp * (Ijd + Ijs);

  // (11) Charges: depletion, inversion (partitioned to the mode drain by fD, which moves from
  //      1/2 at vds = 0 to XPART in saturation, so the charges are continuous across the
  //      source/drain swap), gate, overlaps.
  const S Coxt = Cox * W * L;
  const S Qb = -(Coxt * c.K1 * sqs);
  const S Qinv = -(Coxt * Vgsteff * F1);
  const S Qg0 = -(Qb + Qinv);
  const S fD = 0.5 - (0.5 - c.XPART) * (Vdseff / Vdsat);
  const S QD = fD * Qinv;
  const S QS = (1.0 - fD) * Qinv;
  const S Qovs = c.CGSO * W * (pp * (V[1] - V[2]));
  const S Qovd = c.CGDO * W * (pp * (V[1] - V[0]));
  const S Qd_int = (mode > 0) ? QD : QS;
  const S Qs_int = (mode > 0) ? QS : QD;
  Q[1] = pp * (Qg0 + Qovs + Qovd);
  Q[0] = pp * (Qd_int - Qovd);
  Q[2] = pp * (Qs_int - Qovs);
  Q[3] = pp * Qb;
}

// ---------------------------------------------------------------------------------------------
// Circuit data and MNA bookkeeping.
struct Circuit {
  int n_nodes = 0;
  std::vector<uint8_t> fixed;
  std::vector<double> vfix;
  // Modified nodal analysis: every held node but ground is an unknown; rail[r] is the r-th held
  // node (in node order) and br[r] the unknown of its source current, which flows from the node
  // through the source to ground.
  std::vector<int> rail, br;
  int n_dev = 0;
  std::vector<int> dn;         // 4 per device: d, g, s, b
  std::vector<int> type;       // +1 / -1
  std::vector<double> W, L;
  std::vector<int> mid;
  std::vector<int> rn;         // 2 per resistor
  std::vector<double> rG;
  std::vector<int> sn;         // 2 per current source
  std::vector<double> sI;
  double gshunt = 0.0;
  std::vector<Card> cards;

  // Unknown numbering: free nodes in increasing node order.
  std::vector<int> unk;        // node -> unknown, -1 when fixed
  int n = 0;
  std::map<std::pair<int, int>, long> where;  // (row, col) -> position in CSR values
  std::vector<int> row_ptr, col;
};

constexpr int kOk = 0;
constexpr int kEinval = -1;
constexpr int kEnoconv = -6;

void build_pattern(Circuit& c) {
  c.unk.assign(c.n_nodes, -1);
  c.n = 0;
  for (int i = 0; i < c.n_nodes; ++i)
    if (!c.fixed[i]) c.unk[i] = c.n++;
  c.br.assign(c.rail.size(), -1);
  for (size_t r = 0; r < c.rail.size(); ++r) c.br[r] = c.n++;
  std::set<std::pair<int, int>> ent;
  for (int i = 0; i < c.n; ++i) ent.insert({i, i});
  for (size_t r = 0; r < c.rail.size(); ++r) {
    ent.insert({c.unk[c.rail[r]], c.br[r]});
    ent.insert({c.br[r], c.unk[c.rail[r]]});
  }
  for (size_t r = 0; r < c.rG.size(); ++r) {
    int a = c.unk[c.rn[2 * r]], b = c.unk[c.rn[2 * r + 1]];
    if (a >= 0 && b >= 0) { ent.insert({a, b}); ent.insert({b, a}); }
  }
  for (int k = 0; k < c.n_dev; ++k)
    for (int t = 0; t < 4; ++t)
      for (int u = 0; u < 4; ++u) {
        int a = c.unk[c.dn[4 * k + t]], b = c.unk[c.dn[4 * k + u]];
        if (a >= 0 && b >= 0) ent.insert({a, b});
      }
  c.row_ptr.assign(c.n + 1, 0);
  c.col.clear();
  c.where.clear();
  long pos = 0;
  for (const auto& e : ent) {
    c.row_ptr[e.first + 1]++;
    c.col.push_back(e.second);
    c.where[e] = pos++;
  }
  for (int i = 0; i < c.n; ++i) c.row_ptr[i + 1] += c.row_ptr[i];
}

double node_voltage(const Circuit& c, const double* x, int node) {
  return c.unk[node] >= 0 ? x[c.unk[node]] : c.vfix[node];
}

// Linear part: gshunt on every free node, resistors, current sources. Adds |term| to the scales.
void stamp_linear(const Circuit& c, double* A, double* b, double* As, double* bs) {
  for (int i = 0; i < c.n_nodes; ++i) {
    int a = c.unk[i];
    if (a < 0) continue;
    long p = c.where.at({a, a});
    A[p] += c.gshunt;
    if (As) As[p] += std::fabs(c.gshunt);
  }
  for (size_t r = 0; r < c.rG.size(); ++r) {
    int ni = c.rn[2 * r], nj = c.rn[2 * r + 1];
    int a = c.unk[ni], bb = c.unk[nj];
    double G = c.rG[r];
    if (a >= 0) {
      long p = c.where.at({a, a});
      A[p] += G; if (As) As[p] += std::fabs(G);
      if (bb >= 0) {
        long q = c.where.at({a, bb});
        A[q] -= G; if (As) As[q] += std::fabs(G);
      } else {
        b[a] += G * c.vfix[nj]; if (bs) bs[a] += std::fabs(G * c.vfix[nj]);
      }
    }
    if (bb >= 0) {
      long p = c.where.at({bb, bb});
      A[p] += G; if (As) As[p] += std::fabs(G);
      if (a >= 0) {
        long q = c.where.at({bb, a});
        A[q] -= G; if (As) As[q] += std::fabs(G);
      } else {
        b[bb] += G * c.vfix[ni]; if (bs) bs[bb] += std::fabs(G * c.vfix[ni]);
      }
    }
  }
  for (size_t s = 0; s < c.sI.size(); ++s) {
    int a = c.unk[c.sn[2 * s]], bb = c.unk[c.sn[2 * s + 1]];
    double I = c.sI[s];
    if (a >= 0) { b[a] -= I; if (bs) bs[a] += std::fabs(I); }
    if (bb >= 0) { b[bb] += I; if (bs) bs[bb] += std::fabs(I); }
  }
  // Voltage source of each rail: its current j joins the KCL sum of the rail node (+j leaves the
  // node), and its own row states v_rail - 0 = vfix.
  for (size_t r = 0; r < c.rail.size(); ++r) {
    const int a = c.unk[c.rail[r]], j = c.br[r];
    long p = c.where.at({a, j}), q = c.where.at({j, a});
    A[p] += 1.0; if (As) As[p] += 1.0;
    A[q] += 1.0; if (As) As[q] += 1.0;
    b[j] += c.vfix[c.rail[r]];
    if (bs) bs[j] += std::fabs(c.vfix[c.rail[r]]);
  }
}

using D4 = Dual<double, 4>;

// Evaluate device k with its Jacobians: I[t], G[t][u] = dI_t/dV_u, Q[t], Cq[t][u] = dQ_t/dV_u.
void device_iv(const Circuit& c, int k, const double Vn[4], double I[4], double G[4][4],
               double Q[4], double Cq[4][4] = nullptr) {
  D4 V[4], Id[4], Qd[4];
  for (int t = 0; t < 4; ++t) { V[t] = D4(Vn[t]); V[t].d[t] = 1.0; }
  ees_l1<D4>(c.cards[c.mid[k]], c.type[k], D4(c.W[k]), D4(c.L[k]), V, Id, Qd);
  for (int t = 0; t < 4; ++t) {
    I[t] = Id[t].v;
    Q[t] = Qd[t].v;
    for (int u = 0; u < 4; ++u) G[t][u] = Id[t].d[u];
    if (Cq)
      for (int u = 0; u < 4; ++u) Cq[t][u] = Qd[t].d[u];
  }
}

// Overlap capacitances of one device (step 11 of the model): the gate-source and gate-drain
// overlap charges CGSO W p (Vg - Vs) and CGDO W p (Vg - Vd) enter q_g with + and q_s, q_d with -,
// so their derivatives are the constants +-CGSO W, +-CGDO W (p^2 = 1), independent of the bias.
void overlap_caps(const Card& cd, double W, double Cov[4][4]) {
  for (int t = 0; t < 4; ++t)
    for (int u = 0; u < 4; ++u) Cov[t][u] = 0.0;
  const double cs = cd.CGSO * W, cdr = cd.CGDO * W;
  Cov[1][1] = cs + cdr;
  Cov[1][2] = -cs;
  Cov[1][0] = -cdr;
  Cov[2][2] = cs;
  Cov[2][1] = -cs;
  Cov[0][0] = cdr;
  Cov[0][1] = -cdr;
}

// Transient companion stamp of one Newton iterate x of a time step (Sec. II, Fig. 1: the
// transient loop re-forms A x = b at every Newton iteration of every time step). The charge of
// terminal t is integrated by a one-step rule: the capacitive current into the device is
// ic_t = alpha (Q_t(x) - qprev_t) - beta iprev_t (backward Euler: alpha = 1/h, beta = 0;
// trapezoidal: alpha = 2/h, beta = 1). Linearising I_t + ic_t at x gives
//   A[t][u] += G_tu + alpha C_tu,  b[t] += -I_t - ic_t + sum_u (G_tu + alpha C_tu) x_u
// over all four terminal rows (the gate row now carries capacitive current).
// Scales (sum of |contribution| per entry, as the DC stamp): a device adds three stamps to A[t][u]
// -- the conductance G_tu, the intrinsic charge capacitance alpha C^int_tu and the overlap
// capacitance alpha C^ov_tu (C = C^int + C^ov) -- each counted by its size; b[t] adds |I_t|,
// the sizes of the terms of ic_t and each stamp's size times |x_u|.
void stamp_tran(const Circuit& c, const double* x, const double* qprev, const double* iprev,
                double alpha, double beta, double* A, double* b, double* q, double* icap,
                double* As, double* bs) {
  const long nnz = static_cast<long>(c.col.size());
  std::fill(A, A + nnz, 0.0);
  std::fill(b, b + c.n, 0.0);
  if (As) std::fill(As, As + nnz, 0.0);
  if (bs) std::fill(bs, bs + c.n, 0.0);
  stamp_linear(c, A, b, As, bs);
  for (int k = 0; k < c.n_dev; ++k) {
    double Vn[4], I[4], G[4][4], Q[4], Cq[4][4], Cov[4][4];
    int u_of[4];
    for (int t = 0; t < 4; ++t) {
      int node = c.dn[4 * k + t];
      u_of[t] = c.unk[node];
      Vn[t] = node_voltage(c, x, node);
    }
    device_iv(c, k, Vn, I, G, Q, Cq);
    overlap_caps(c.cards[c.mid[k]], c.W[k], Cov);
    for (int t = 0; t < 4; ++t) {
      const long at = static_cast<long>(t) * c.n_dev + k;
      const double ic = alpha * (Q[t] - qprev[at]) - (iprev ? beta * iprev[at] : 0.0);
      if (q) q[at] = Q[t];
      if (icap) icap[at] = ic;
      if (u_of[t] < 0) continue;
      double rhs = -I[t] - ic;
      double scale = std::fabs(I[t]) + alpha * (std::fabs(Q[t]) + std::fabs(qprev[at])) +
                     (iprev ? std::fabs(beta * iprev[at]) : 0.0);
      for (int u = 0; u < 4; ++u) {
        if (u_of[u] < 0) continue;
        const double a = G[t][u] + alpha * Cq[t][u];
        long p = c.where.at({u_of[t], u_of[u]});
        A[p] += a;
        const double am = std::fabs(G[t][u]) + alpha * std::fabs(Cq[t][u] - Cov[t][u]) +
                          alpha * std::fabs(Cov[t][u]);
        if (As) As[p] += am;
        rhs += a * Vn[u];
        scale += am * std::fabs(Vn[u]);
      }
      b[u_of[t]] += rhs;
      if (bs) bs[u_of[t]] += scale;
    }
  }
}

// Full stamp in device-index order: A = A_lin + sum_k G_k, b = b_lin + sum_k (-I_k + G_k V_k).
void stamp_all(const Circuit& c, const double* x, double* A, double* b, double* q, double* As,
               double* bs) {
  const long nnz = static_cast<long>(c.col.size());
  std::fill(A, A + nnz, 0.0);
  std::fill(b, b + c.n, 0.0);
  if (As) std::fill(As, As + nnz, 0.0);
  if (bs) std::fill(bs, bs + c.n, 0.0);
  stamp_linear(c, A, b, As, bs);
  for (int k = 0; k < c.n_dev; ++k) {
    double Vn[4], I[4], G[4][4], Q[4];
    int u_of[4];
    for (int t = 0; t < 4; ++t) {
      int node = c.dn[4 * k + t];
      u_of[t] = c.unk[node];
      Vn[t] = node_voltage(c, x, node);
    }
    device_iv(c, k, Vn, I, G, Q);
    if (q)
      for (int t = 0; t < 4; ++t) q[static_cast<long>(t) * c.n_dev + k] = Q[t];
    for (int t = 0; t < 4; ++t) {
      if (u_of[t] < 0) continue;
      double rhs = -I[t];
      double scale = std::fabs(I[t]);
      for (int u = 0; u < 4; ++u) {
        if (u_of[u] < 0) continue;
        long p = c.where.at({u_of[t], u_of[u]});
        A[p] += G[t][u];
        if (As) As[p] += std::fabs(G[t][u]);
        rhs += G[t][u] * Vn[u];
        scale += std::fabs(G[t][u] * Vn[u]);
      }
      b[u_of[t]] += rhs;
      if (bs) bs[u_of[t]] += scale;
    }
  }
}

// KCL residual F(x): net current leaving every free node (no linearisation); on the row of a
// source current, the source equation v_rail - vfix.
void kcl_residual(const Circuit& c, const double* x, double* F) {
  std::fill(F, F + c.n, 0.0);
  for (int i = 0; i < c.n_nodes; ++i)
    if (c.unk[i] >= 0) F[c.unk[i]] += c.gshunt * x[c.unk[i]];
  for (size_t r = 0; r < c.rG.size(); ++r) {
    int ni = c.rn[2 * r], nj = c.rn[2 * r + 1];
    double I = c.rG[r] * (node_voltage(c, x, ni) - node_voltage(c, x, nj));
    if (c.unk[ni] >= 0) F[c.unk[ni]] += I;
    if (c.unk[nj] >= 0) F[c.unk[nj]] -= I;
  }
  for (size_t s = 0; s < c.sI.size(); ++s) {
    int a = c.unk[c.sn[2 * s]], bb = c.unk[c.sn[2 * s + 1]];
    if (a >= 0) F[a] += c.sI[s];
    if (bb >= 0) F[bb] -= c.sI[s];
  }
  for (int k = 0; k < c.n_dev; ++k) {
    double V[4], I[4], Q[4];
    for (int t = 0; t < 4; ++t) V[t] = node_voltage(c, x, c.dn[4 * k + t]);
    ees_l1<double>(c.cards[c.mid[k]], c.type[k], c.W[k], c.L[k], V, I, Q);
    for (int t = 0; t < 4; ++t) {
      int a = c.unk[c.dn[4 * k + t]];
      if (a >= 0) F[a] += I[t];
    }
  }
  for (size_t r = 0; r < c.rail.size(); ++r) {
    const int a = c.unk[c.rail[r]], j = c.br[r];
    F[a] += x[j];
    F[j] = x[a] - c.vfix[c.rail[r]];
  }
}

// Dense LU with partial pivoting; solves M y = r in place (M row-major n x n). Returns false when
// a pivot is exactly zero.
bool dense_solve(std::vector<double>& M, std::vector<double>& r, int n) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = std::fabs(M[static_cast<size_t>(k) * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = std::fabs(M[static_cast<size_t>(i) * n + k]);
      if (v > best) { best = v; piv = i; }
    }
    if (best == 0.0) return false;
    if (piv != k) {
      for (int j = 0; j < n; ++j)
        std::swap(M[static_cast<size_t>(k) * n + j], M[static_cast<size_t>(piv) * n + j]);
      std::swap(r[k], r[piv]);
    }
    const double d = M[static_cast<size_t>(k) * n + k];
    for (int i = k + 1; i < n; ++i) {
      double f = M[static_cast<size_t>(i) * n + k] / d;
      if (f == 0.0) continue;
      M[static_cast<size_t>(i) * n + k] = f;
      for (int j = k + 1; j < n; ++j)
        M[static_cast<size_t>(i) * n + j] -= f * M[static_cast<size_t>(k) * n + j];
      r[i] -= f * r[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = r[i];
    for (int j = i + 1; j < n; ++j) s -= M[static_cast<size_t>(i) * n + j] * r[j];
    r[i] = s / M[static_cast<size_t>(i) * n + i];
  }
  return true;
}

std::vector<double> to_dense(const Circuit& c, const std::vector<double>& A, bool transpose) {
  std::vector<double> M(static_cast<size_t>(c.n) * c.n, 0.0);
  for (int i = 0; i < c.n; ++i)
    for (int p = c.row_ptr[i]; p < c.row_ptr[i + 1]; ++p) {
      int j = c.col[p];
      if (transpose) M[static_cast<size_t>(j) * c.n + i] += A[p];
      else M[static_cast<size_t>(i) * c.n + j] += A[p];
    }
  return M;
}

// Infinity norm; any NaN makes it +inf so that a NaN iterate never passes a convergence test.
double inf_norm(const std::vector<double>& v) {
  double m = 0.0;
  for (double e : v) {
    if (std::isnan(e)) return INFINITY;
    m = std::max(m, std::fabs(e));
  }
  return m;
}

// Damped Newton from x (in/out). Returns iterations used (>0) or -1 when not converged.
int newton(const Circuit& c, std::vector<double>& x, int max_iter, std::vector<double>* hist) {
  const long nnz = static_cast<long>(c.col.size());
  std::vector<double> A(nnz), b(c.n), F(c.n);
  for (int it = 1; it <= max_iter; ++it) {
    if (hist) hist->insert(hist->end(), x.begin(), x.end());
    stamp_all(c, x.data(), A.data(), b.data(), nullptr, nullptr, nullptr);
    std::vector<double> M = to_dense(c, A, false);
    std::vector<double> y = b;
    if (!dense_solve(M, y, c.n)) return -1;
    std::vector<double> dx(c.n);
    for (int i = 0; i < c.n; ++i) dx[i] = y[i] - x[i];
    double m = inf_norm(dx);
    if (m > 0.2) for (double& e : dx) e *= 0.2 / m;
    for (int i = 0; i < c.n; ++i) x[i] += dx[i];
    if (inf_norm(dx) <= 1e-12 + 1e-9 * inf_norm(x)) {
      kcl_residual(c, x.data(), F.data());
      if (inf_norm(F) <= 1e-12) {
        if (hist) hist->insert(hist->end(), x.begin(), x.end());
        return it;
      }
    }
  }
  return -1;
}

}  // namespace

// =============================================================================================
// C interface (ctypes). Every array is a host pointer owned by the caller; sizes as stated.
extern "C" {

void* ora_create(int32_t n_nodes, const uint8_t* node_fixed, const double* node_vfix,
                 int32_t n_dev, const int32_t* dev_nodes, const int8_t* dev_type, const double* W,
                 const double* L, const int32_t* model_id, int32_t n_res, const int32_t* res_nodes,
                 const double* res_G, int32_t n_isrc, const int32_t* isrc_nodes,
                 const double* isrc_val, double gshunt, int32_t n_cards, const double* cards,
                 int32_t rail_mode) {
  if (n_nodes < 1 || n_dev < 0 || n_res < 0 || n_isrc < 0 || n_cards < 1) return nullptr;
  if (rail_mode != 0 && rail_mode != 1) return nullptr;
  Circuit* c = new Circuit;
  c->n_nodes = n_nodes;
  c->fixed.assign(node_fixed, node_fixed + n_nodes);
  c->vfix.assign(node_vfix, node_vfix + n_nodes);
  c->fixed[0] = 1;
  c->vfix[0] = 0.0;
  if (rail_mode == 1)
    for (int i = 1; i < n_nodes; ++i)
      if (c->fixed[i]) { c->rail.push_back(i); c->fixed[i] = 0; }
  c->n_dev = n_dev;
  c->dn.assign(dev_nodes, dev_nodes + 4L * n_dev);
  c->type.assign(dev_type, dev_type + n_dev);
  c->W.assign(W, W + n_dev);
  c->L.assign(L, L + n_dev);
  c->mid.assign(model_id, model_id + n_dev);
  c->rn.assign(res_nodes, res_nodes + 2L * n_res);
  c->rG.assign(res_G, res_G + n_res);
  c->sn.assign(isrc_nodes, isrc_nodes + 2L * n_isrc);
  c->sI.assign(isrc_val, isrc_val + n_isrc);
  c->gshunt = gshunt;
  for (int i = 0; i < n_cards; ++i) c->cards.push_back(read_card(cards + static_cast<long>(i) * kCardLen));
  for (int v : c->dn) if (v < 0 || v >= n_nodes) { delete c; return nullptr; }
  for (int v : c->rn) if (v < 0 || v >= n_nodes) { delete c; return nullptr; }
  for (int v : c->sn) if (v < 0 || v >= n_nodes) { delete c; return nullptr; }
  for (int v : c->mid) if (v < 0 || v >= n_cards) { delete c; return nullptr; }
  for (int v : c->type) if (v != 1 && v != -1) { delete c; return nullptr; }
  build_pattern(*c);
  return c;
}

void ora_destroy(void* h) { delete static_cast<Circuit*>(h); }

int32_t ora_n_unknowns(void* h) { return static_cast<Circuit*>(h)->n; }
int64_t ora_nnz(void* h) { return static_cast<int64_t>(static_cast<Circuit*>(h)->col.size()); }

int ora_pattern(void* h, int32_t* row_ptr, int32_t* col, int32_t* unk_of_node) {
  Circuit& c = *static_cast<Circuit*>(h);
  if (row_ptr) std::copy(c.row_ptr.begin(), c.row_ptr.end(), row_ptr);
  if (col) std::copy(c.col.begin(), c.col.end(), col);
  if (unk_of_node) std::copy(c.unk.begin(), c.unk.end(), unk_of_node);
  return kOk;
}

int ora_set_sizes(void* h, const double* W, const double* L) {
  Circuit& c = *static_cast<Circuit*>(h);
  c.W.assign(W, W + c.n_dev);
  c.L.assign(L, L + c.n_dev);
  return kOk;
}

// A (nnz), b (n); q (4 x n_dev, terminal-major, nullable); A_scale / b_scale (nullable) receive
// the sum of |contribution| per entry, the denominator of the cancellation-aware error metric.
int ora_eval_stamp(void* h, const double* x, double* A, double* b, double* q, double* A_scale,
                   double* b_scale) {
  stamp_all(*static_cast<Circuit*>(h), x, A, b, q, A_scale, b_scale);
  return kOk;
}

int ora_kcl_residual(void* h, const double* x, double* F) {
  kcl_residual(*static_cast<Circuit*>(h), x, F);
  return kOk;
}

// Greedy colouring (Sec. I, Sec. II): visit devices in `order` (NULL = 0..N-1); each takes the
// smallest colour not used by an already coloured neighbour. Devices are neighbours when they
// share a node selected by `rule`: 0 = a free node, 1 = any node other than ground (the paper's
// literal rule, rails included), 2 = a free node that both devices write as a DC row (d, s, b).
int ora_color_greedy(void* h, int32_t rule, const int32_t* order, int32_t* colors,
                     int32_t* n_colors) {
  Circuit& c = *static_cast<Circuit*>(h);
  if (rule < 0 || rule > 2) return kEinval;
  std::vector<std::vector<int>> at(c.n_nodes);
  for (int k = 0; k < c.n_dev; ++k)
    for (int t = 0; t < 4; ++t) {
      int node = c.dn[4 * k + t];
      bool ok = (rule == 1) ? (node != 0) : (c.fixed[node] == 0);
      if (rule == 2 && t == 1) ok = false;
      if (!ok) continue;
      std::vector<int>& v = at[node];
      if (v.empty() || v.back() != k) v.push_back(k);
    }
  std::vector<int> col(c.n_dev, -1);
  std::vector<char> seen_order(c.n_dev, 0);
  int C = 0;
  for (int i = 0; i < c.n_dev; ++i) {
    int v = order ? order[i] : i;
    if (v < 0 || v >= c.n_dev || seen_order[v]) return kEinval;
    seen_order[v] = 1;
    std::set<int> used;
    for (int t = 0; t < 4; ++t) {
      int node = c.dn[4 * v + t];
      if (rule == 2 && t == 1) continue;
      bool ok = (rule == 1) ? (node != 0) : (c.fixed[node] == 0);
      if (!ok) continue;
      for (int w : at[node])
        if (w != v && col[w] >= 0) used.insert(col[w]);
    }
    int m = 0;
    while (used.count(m)) ++m;
    col[v] = m;
    C = std::max(C, m + 1);
  }
  std::copy(col.begin(), col.end(), colors);
  *n_colors = C;
  return kOk;
}

// DC operating point by damped Newton with dense LU (x_io: initial guess in, solution out).
// hist (nullable, (max_iter + 1) x n) receives every iterate x_k at which A, b were formed,
// followed by the converged x. Returns iterations (> 0) or -6 when Newton and the gshunt-stepping
// fallback both fail.
int ora_dc_solve(void* h, double* x_io, int32_t max_iter, double* hist, int32_t* n_hist) {
  Circuit& c = *static_cast<Circuit*>(h);
  std::vector<double> x(x_io, x_io + c.n);
  std::vector<double> hv;
  int it = newton(c, x, max_iter, hist ? &hv : nullptr);
  if (it < 0) {
    const double g0 = c.gshunt;
    x.assign(x_io, x_io + c.n);
    bool ok = true;
    for (double g = 1e-3; ok && g > g0 * 1.0000001; g *= 0.1) {
      c.gshunt = g;
      ok = newton(c, x, max_iter, nullptr) > 0;
    }
    c.gshunt = g0;
    hv.clear();
    it = ok ? newton(c, x, max_iter, hist ? &hv : nullptr) : -1;
    if (it < 0) return kEnoconv;
  }
  std::copy(x.begin(), x.end(), x_io);
  if (hist) {
    long m = std::min<long>(static_cast<long>(hv.size()), static_cast<long>(max_iter + 1) * c.n);
    std::copy(hv.begin(), hv.begin() + m, hist);
    *n_hist = static_cast<int32_t>(m / std::max(c.n, 1));
  }
  return it;
}

// Adjoint solve at x: A(x)^T lambda = e_out (out = unknown index).
int ora_adjoint(void* h, const double* x, int32_t out, double* lambda) {
  Circuit& c = *static_cast<Circuit*>(h);
  if (out < 0 || out >= c.n) return kEinval;
  std::vector<double> A(c.col.size()), b(c.n);
  stamp_all(c, x, A.data(), b.data(), nullptr, nullptr, nullptr);
  std::vector<double> M = to_dense(c, A, true);
  std::vector<double> r(c.n, 0.0);
  r[out] = 1.0;
  if (!dense_solve(M, r, c.n)) return kEinval;
  std::copy(r.begin(), r.end(), lambda);
  return kOk;
}

// Gradient of s = sum_e gA[e] A[e] + sum_i gb[i] b[i] (A, b formed at x) with respect to x,
// W and L, by nested dual numbers: inner level over the four terminal voltages (gives G), outer
// level over (Vd, Vg, Vs, Vb, W, L). Terminal gradients are gathered to unknowns in device order.
int ora_eval_stamp_grad(void* h, const double* x, const double* gA, const double* gb, double* gx,
                        double* gW, double* gL) {
  using D6 = Dual<D4, 6>;
  Circuit& c = *static_cast<Circuit*>(h);
  std::fill(gx, gx + c.n, 0.0);
  for (int k = 0; k < c.n_dev; ++k) {
    D6 V[4], I[4], Q[4];
    int u_of[4];
    double Vn[4];
    for (int t = 0; t < 4; ++t) {
      int node = c.dn[4 * k + t];
      u_of[t] = c.unk[node];
      Vn[t] = node_voltage(c, x, node);
      V[t] = D6(Vn[t]);
      V[t].v.d[t] = 1.0;
      V[t].d[t] = D4(1.0);
    }
    D6 W(c.W[k]), L(c.L[k]);
    W.d[4] = D4(1.0);
    L.d[5] = D4(1.0);
    ees_l1<D6>(c.cards[c.mid[k]], c.type[k], W, L, V, I, Q);
    double ds[6] = {0, 0, 0, 0, 0, 0};
    for (int t = 0; t < 4; ++t) {
      if (u_of[t] < 0) continue;
      const double wb = gb[u_of[t]];
      for (int j = 0; j < 6; ++j) ds[j] += wb * (-I[t].d[j].v);
      for (int u = 0; u < 4; ++u) {
        if (u_of[u] < 0) continue;
        const double wa = gA[c.where.at({u_of[t], u_of[u]})];
        const double Gtu = I[t].v.d[u];
        for (int j = 0; j < 6; ++j) {
          const double dG = I[t].d[j].d[u];
          ds[j] += wa * dG + wb * dG * Vn[u];
        }
        ds[u] += wb * Gtu;
      }
    }
    for (int t = 0; t < 4; ++t)
      if (u_of[t] >= 0) gx[u_of[t]] += ds[t];
    gW[k] = ds[4];
    gL[k] = ds[5];
  }
  return kOk;
}

// One device: I[4], G[16] (row-major dI_t/dV_u), Q[4] for card `card` (kCardLen doubles).
int ora_device_eval(const double* card, int32_t p, double W, double L, const double* V, double* I,
                    double* G, double* Q) {
  if (p != 1 && p != -1) return kEinval;
  Card cd = read_card(card);
  D4 Vd[4], Id[4], Qd[4];
  for (int t = 0; t < 4; ++t) { Vd[t] = D4(V[t]); Vd[t].d[t] = 1.0; }
  ees_l1<D4>(cd, p, D4(W), D4(L), Vd, Id, Qd);
  for (int t = 0; t < 4; ++t) {
    I[t] = Id[t].v;
    if (Q) Q[t] = Qd[t].v;
    if (G) for (int u = 0; u < 4; ++u) G[4 * t + u] = Id[t].d[u];
  }
  return kOk;
}

int32_t ora_card_len(void) { return kCardLen; }

// Algorithmic work of one device evaluation (terminal currents and charges, values only) at V:
// counts[7] = additions/subtractions, multiplications, divisions, exp, expm1, log1p, sqrt of the
// operations that depend on the free terminals (bit t of free_mask: terminal t is on a free
// node; a held terminal's voltage is a constant like the card, W and L).
int ora_count_ops(const double* card, int32_t p, double W, double L, const double* V,
                  int32_t free_mask, int64_t* counts) {
  if (p != 1 && p != -1) return kEinval;
  Card cd = read_card(card);
  Cnt Vc[4], Ic[4], Qc[4];
  for (int t = 0; t < 4; ++t) Vc[t] = Cnt(V[t], ((free_mask >> t) & 1) != 0);
  g_ops = OpCount{};
  ees_l1<Cnt>(cd, p, Cnt(W), Cnt(L), Vc, Ic, Qc);
  const long long k[7] = {g_ops.add, g_ops.mul, g_ops.div, g_ops.exp, g_ops.expm1, g_ops.log1p,
                          g_ops.sqrt};
  for (int i = 0; i < 7; ++i) counts[i] = k[i];
  return kOk;
}

// Transient companion stamp at x (see stamp_tran). qprev, iprev (nullable = zero): [4 x n_dev]
// terminal-major; q_out, i_out (nullable): charges and capacitive currents at x.
int ora_eval_stamp_tran(void* h, const double* x, const double* qprev, const double* iprev,
                        double alpha, double beta, double* A, double* b, double* q_out,
                        double* i_out, double* A_scale, double* b_scale) {
  Circuit& c = *static_cast<Circuit*>(h);
  std::vector<double> zero;
  if (!qprev) {
    zero.assign(4L * c.n_dev, 0.0);
    qprev = zero.data();
  }
  stamp_tran(c, x, qprev, iprev, alpha, beta, A, b, q_out, i_out, A_scale, b_scale);
  return kOk;
}

// Charges and their Jacobian for one device: Q[4], C[16] row-major dQ_t/dV_u.
int ora_device_charge(const double* card, int32_t p, double W, double L, const double* V,
                      double* Q, double* C) {
  if (p != 1 && p != -1) return kEinval;
  Card cd = read_card(card);
  D4 Vd[4], Id[4], Qd[4];
  for (int t = 0; t < 4; ++t) { Vd[t] = D4(V[t]); Vd[t].d[t] = 1.0; }
  ees_l1<D4>(cd, p, D4(W), D4(L), Vd, Id, Qd);
  for (int t = 0; t < 4; ++t) {
    Q[t] = Qd[t].v;
    for (int u = 0; u < 4; ++u) C[4 * t + u] = Qd[t].d[u];
  }
  return kOk;
}

// Transient analysis by a one-step rule (method 0 backward Euler, 1 trapezoidal) with fixed
// step h: from x_io (state at t = 0, charges there, capacitive currents i0 or zero) take n_steps
// steps, each solved by Newton with the companion stamp and every node's update clipped to
// 0.2 V, converged when |dx| <= 1e-12 + 1e-9 |x|. traj [(n_steps + 1) x n]
// receives the states. Returns 0, or -6 when a step's Newton fails.
int ora_tran_solve(void* h, double* x_io, double step, int32_t n_steps, int32_t method,
                   const double* i0, double* traj) {
  Circuit& c = *static_cast<Circuit*>(h);
  if (!(step > 0.0) || n_steps < 0 || method < 0 || method > 1) return kEinval;
  const double alpha = method == 0 ? 1.0 / step : 2.0 / step;
  const double beta = method == 0 ? 0.0 : 1.0;
  const long nq = 4L * c.n_dev;
  const long nnz = static_cast<long>(c.col.size());
  std::vector<double> x(x_io, x_io + c.n), qprev(nq), iprev(nq, 0.0), qn(nq), in(nq);
  std::vector<double> A(nnz), b(c.n), F(c.n);
  if (i0) iprev.assign(i0, i0 + nq);
  stamp_tran(c, x.data(), qprev.data(), nullptr, 0.0, 0.0, A.data(), b.data(), qprev.data(),
             nullptr, nullptr, nullptr);  // charges at t = 0
  std::copy(x.begin(), x.end(), traj);
  for (int s = 1; s <= n_steps; ++s) {
    bool conv = false;
    for (int it = 0; it < 200 && !conv; ++it) {
      stamp_tran(c, x.data(), qprev.data(), iprev.data(), alpha, beta, A.data(), b.data(),
                 qn.data(), in.data(), nullptr, nullptr);
      std::vector<double> M = to_dense(c, A, false);
      std::vector<double> y = b;
      if (!dense_solve(M, y, c.n)) return kEnoconv;
      // per-node step limiting to 0.2 V (uniform scaling can lock into a 2-cycle here)
      std::vector<double> dx(c.n);
      for (int i = 0; i < c.n; ++i) dx[i] = std::max(-0.2, std::min(0.2, y[i] - x[i]));
      for (int i = 0; i < c.n; ++i) x[i] += dx[i];
      conv = inf_norm(dx) <= 1e-12 + 1e-9 * inf_norm(x);
    }
    if (!conv) return kEnoconv;
    stamp_tran(c, x.data(), qprev.data(), iprev.data(), alpha, beta, A.data(), b.data(),
               qn.data(), in.data(), nullptr, nullptr);
    qprev = qn;
    iprev = in;
    std::copy(x.begin(), x.end(), traj + static_cast<long>(s) * c.n);
  }
  std::copy(x.begin(), x.end(), x_io);
  return kOk;
}

}  // extern "C"
