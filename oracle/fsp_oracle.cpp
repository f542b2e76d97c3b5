// fsp_oracle.cpp -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow CPU restatement of the WENO-interpolation-based, upwind-biased,
// free-stream-preserving (WENOIU) schemes of Q. Li and D. Sun, "WENO interpolation-based
// and upwind-biased schemes with free-stream preservation" (arXiv:1810.11103): the
// third- and fifth-order one- and two-midpoint schemes of Section 3 and the seventh-order
// one-midpoint scheme of the Appendix (scheme index 4).
// It is the oracle that the CUDA library is checked against.  Only the test suite,
// the smoke check and the CPU-baseline leg of the benchmark may load it; the product
// path never does.  It shares no code, header or table with the CUDA library.
//
// Everything is written as loops over lines, nodes and interfaces in the order the
// paper states the method: no tiling, fusion or reordering.  Build: g++ -O2
// -ffp-contract=off (no fused multiply-add), so every product is rounded on its own.
//
// The core is templated on the scalar type:
//   double       the oracle proper (FP64)
//   long double  higher precision; shows the free-stream residual is round-off
//   Dual         forward-mode tangent (value + one directional derivative)
//   Counted      counts floating-point operations (+ - * / sqrt, one each)
//   Rev          reverse mode: tapes the operations, then accumulates adjoints backwards
//
// Conventions (identical in meaning, not in code, to the CUDA library):
//   * nodes (i, j), i fastest; unit computational spacing (d xi = d eta = 1);
//   * state Q = (rho, rho u, rho v, E), 4 planes [4][nj][ni];
//   * metrics: 5 planes (xi_x^, xi_y^, eta_x^, eta_y^, J^-1) on a grid extended by
//     G = 4 ghost layers on every side: plane p, node (i, j) at
//     M[p*(nj+8)*(ni+8) + (j+4)*(ni+8) + (i+4)];
//   * boundary faces 0..3 = i-min, i-max, j-min, j-max; codes PERIODIC=0,
//     TRANSMISSIVE=1, DIRICHLET=2, SLIPWALL=3, FARFIELD=4.
//
// Readings of points the paper leaves open are marked "Reading:" where they are used.
// Parity status: every routine is pinned by the tests in tests/test_oracle_*.py
// (Table 3 and Table 4 of the paper, free-stream preservation, closed forms,
// symmetry, conservation, tangent vs finite differences); none is "parity unpinned".

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

namespace orc {

// ----------------------------------------------------------------------------------
// Scalar types
// ----------------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double a) : v(a), d(0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
inline bool operator<=(Dual a, Dual b) { return a.v <= b.v; }
inline bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, s > 0 ? a.d / (2.0 * s) : 0.0);
}
inline Dual fabs(Dual a) { return a.v >= 0 ? a : -a; }
inline double val(Dual a) { return a.v; }

static long long g_flops = 0;
struct Counted {
  double v;
  Counted() : v(0) {}
  Counted(double a) : v(a) {}
};
inline Counted operator+(Counted a, Counted b) { ++g_flops; return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { ++g_flops; return Counted(a.v - b.v); }
inline Counted operator-(Counted a) { return Counted(-a.v); }
inline Counted operator*(Counted a, Counted b) { ++g_flops; return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { ++g_flops; return Counted(a.v / b.v); }
inline Counted& operator+=(Counted& a, Counted b) { a = a + b; return a; }
inline Counted& operator-=(Counted& a, Counted b) { a = a - b; return a; }
inline Counted& operator*=(Counted& a, Counted b) { a = a * b; return a; }
inline bool operator<(Counted a, Counted b) { return a.v < b.v; }
inline bool operator>(Counted a, Counted b) { return a.v > b.v; }
inline bool operator<=(Counted a, Counted b) { return a.v <= b.v; }
inline bool operator>=(Counted a, Counted b) { return a.v >= b.v; }
inline Counted sqrt(Counted a) { ++g_flops; return Counted(std::sqrt(a.v)); }
inline Counted fabs(Counted a) { return Counted(std::fabs(a.v)); }
inline double val(Counted a) { return a.v; }

// Reverse mode (the adjoint, a vector-Jacobian product).  Every operation whose result
// depends on an active value appends one record to a tape: the indices of its at most two
// active operands and the partial derivative of the result with respect to each, taken from
// the values of this evaluation (the branches the evaluation takes are the ones
// differentiated: the mapping branch, the boundary decisions, and a line maximum's lowest
// maximising index).  Walking the tape backwards, each record passes its adjoint to its
// operands, adjoint(operand) += partial * adjoint(result), which gives the transposed
// Jacobian of the whole computation applied to a seed.  Elementary adjoints:
//   c = a + b:  da += dc, db += dc           c = a - b:  da += dc, db -= dc
//   c = a * b:  da += b dc, db += a dc       c = a / b:  da += dc / b, db -= (c / b) dc
//   c = sqrt(a): da += dc / (2 c) (0 at a = 0)           c = |a|: the sign of a, +1 at 0
// Constants (i < 0) record nothing.
struct TapeRec { double pa, pb; int a, b; };
static std::vector<TapeRec> g_tape;
static long long g_rev_extra = 0;   // operations spent on partial derivatives (for the count)
static long long g_rev_edges = 0;   // operations of the reverse sweep (for the count)
struct Rev {
  double v;
  int i;
  Rev() : v(0), i(-1) {}
  Rev(double a) : v(a), i(-1) {}
  Rev(double a, int idx) : v(a), i(idx) {}
};
// `cost`: operations of one operand edge in the reverse sweep (1 for a sum or difference,
// adj += adj_c; 2 for any other operation, a multiply-add).
static inline Rev rev_rec(double v, int a, double pa, int b, double pb, int cost) {
  if (a < 0 && b < 0) return Rev(v);
  g_rev_edges += cost * ((a >= 0) + (b >= 0));
  g_tape.push_back(TapeRec{pa, pb, a, b});
  return Rev(v, (int)(g_tape.size() - 1));
}
static inline Rev rev_leaf(double v) {   // an independent variable: a record with no operands
  g_tape.push_back(TapeRec{0.0, 0.0, -1, -1});
  return Rev(v, (int)(g_tape.size() - 1));
}
inline Rev operator+(Rev a, Rev b) { return rev_rec(a.v + b.v, a.i, 1.0, b.i, 1.0, 1); }
inline Rev operator-(Rev a, Rev b) { return rev_rec(a.v - b.v, a.i, 1.0, b.i, -1.0, 1); }
inline Rev operator-(Rev a) { return rev_rec(-a.v, a.i, -1.0, -1, 0.0, 1); }
inline Rev operator*(Rev a, Rev b) { return rev_rec(a.v * b.v, a.i, b.v, b.i, a.v, 2); }
inline Rev operator/(Rev a, Rev b) {
  const double q = a.v / b.v;
  if (a.i >= 0 || b.i >= 0) g_rev_extra += 1 + (b.i >= 0);   // 1 / b, and q (1 / b) for b
  return rev_rec(q, a.i, 1.0 / b.v, b.i, -q / b.v, 2);
}
inline Rev& operator+=(Rev& a, Rev b) { a = a + b; return a; }
inline Rev& operator-=(Rev& a, Rev b) { a = a - b; return a; }
inline Rev& operator*=(Rev& a, Rev b) { a = a * b; return a; }
inline bool operator<(Rev a, Rev b) { return a.v < b.v; }
inline bool operator>(Rev a, Rev b) { return a.v > b.v; }
inline bool operator<=(Rev a, Rev b) { return a.v <= b.v; }
inline bool operator>=(Rev a, Rev b) { return a.v >= b.v; }
inline Rev sqrt(Rev a) {
  const double s = std::sqrt(a.v);
  if (a.i >= 0) g_rev_extra += 1;                               // 0.5 / s
  return rev_rec(s, a.i, s > 0 ? 0.5 / s : 0.0, -1, 0.0, 2);
}
inline Rev fabs(Rev a) {
  if (a.v < 0) return -a;
  g_rev_edges += a.i >= 0;   // the reverse passes the adjoint through with the sign +1: one operation
  return a;
}
inline double val(Rev a) { return a.v; }

// The reverse sweep: adj[k] holds the adjoint of tape record k on entry (the seeds) and the
// accumulated adjoints on return.
static void rev_sweep(std::vector<double>& adj) {
  for (size_t k = g_tape.size(); k-- > 0;) {
    const double g = adj[k];
    if (g == 0.0) continue;
    const TapeRec& r = g_tape[k];
    if (r.a >= 0) adj[r.a] += r.pa * g;
    if (r.b >= 0) adj[r.b] += r.pb * g;
  }
}

inline double val(double a) { return a; }
inline double val(long double a) { return (double)a; }
using std::sqrt;
using std::fabs;

template <class T> inline T cst(long double c) { return T((double)c); }
template <> inline long double cst<long double>(long double c) { return c; }

// ----------------------------------------------------------------------------------
// Scheme tables (Section 3).  All four variants, with the printed coefficients.
// ----------------------------------------------------------------------------------
enum { S31 = 0, S32 = 1, S51 = 2, S52 = 3, S71 = 4, S74 = 5 };
enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_DIRICHLET = 2, BC_SLIPWALL = 3, BC_FARFIELD = 4,
       BC_LINK = 5 };

// A face joined to a face of another block (multi-block grids).  The blocks partition the
// nodes of one larger structured grid: the ghost at depth k (k = 0 first) beyond face f of
// block B is the node at depth k inward from face `face` of block `nbr`; along the face
// the index runs the same way or `rev`ersed; `off` is added to ghost coordinates.
struct Link { int nbr, face, rev; double off[2]; };

// Index of the node of the neighbour behind face f for a ghost of a block of size ni x nj.
// (gi, gj) is the ghost (outside the range along face f's direction); returns (ni', nj').
static inline void link_map(const Link& L, int f, int ni, int nj, int nni, int nnj, int gi, int gj,
                            int& oi, int& oj) {
  int k, t;
  if (f == 0) { k = -1 - gi; t = gj; }
  else if (f == 1) { k = gi - ni; t = gj; }
  else if (f == 2) { k = -1 - gj; t = gi; }
  else { k = gj - nj; t = gi; }
  const int nt = (L.face < 2) ? nnj : nni;
  if (L.rev) t = nt - 1 - t;
  int depth;
  if (L.face == 0) depth = k;
  else if (L.face == 1) depth = nni - 1 - k;
  else if (L.face == 2) depth = k;
  else depth = nnj - 1 - k;
  if (L.face < 2) { oi = depth; oj = t; } else { oi = t; oj = depth; }
}
static const int G = 4;  // ghost layers of the stored metrics

struct SchemeTab {
  int r;                  // points of each WENO candidate stencil (Table 1)
  long double hmid[2];    // h+ coefficient of f+_{j+1/2+m}, m = 0, -1
  long double hnode[7];   // h+ coefficient of f+_{j+k}, k = -3..3
  long double cnode[4];   // delta^{c,(1)}: a_k multiplying (f_{j+k} - f_{j-k}), k = 1..4
  long double cmid[2];    // delta^{c,(1)}: b_m multiplying (f~_{j+m} - f~_{j-m}), m = 1/2, 3/2
  long double hmidx[2];   // four-midpoint scheme: h+ coefficient of f+_{j+1/2+m}, m = -2, +1
  long double cmid3;      // four-midpoint scheme: b_{5/2}
};

static const SchemeTab TAB[6] = {
  // WENOIU3-1MP: h+ of Eq. (3.4); delta^{c,(1)} of Eq. (3.7).
  {2, {1.0L, 0.0L}, {0.0L, 0.0L, -1.0L / 24, 2.0L / 24, -1.0L / 24, 0.0L, 0.0L},
   {2.0L / 48, -1.0L / 48, 0.0L, 0.0L}, {1.0L, 0.0L}},
  // WENOIU3-2MP: h+ of Eq. (3.8), f_{j+1/2} + (-f_{j-1/2} + 2 f_j - f_{j+1/2})/6;
  // delta^{c,(1)} of Eq. (3.9).
  {2, {1.0L - 1.0L / 6, -1.0L / 6}, {0.0L, 0.0L, 0.0L, 2.0L / 6, 0.0L, 0.0L, 0.0L},
   {2.0L / 12, 0.0L, 0.0L, 0.0L}, {11.0L / 12, -1.0L / 12}},
  // WENOIU5-1MP: h+ of Eq. (3.16); delta^{c,(1)} of Eq. (3.19).
  {3, {1.0L, 0.0L}, {0.0L, 19.0L / 1920, -29.0L / 480, 77.0L / 960, -3.0L / 160, -7.0L / 640, 0.0L},
   {17.0L / 256, -13.0L / 320, 19.0L / 3840, 0.0L}, {1.0L, 0.0L}},
  // WENOIU5-2MP: h+ of Eq. (3.20), f_{j+1/2} + [(-4 f_{j+1} + f_j + f_{j-1}) + (6 f_{j+1/2}
  // - 4 f_{j-1/2})]/30; delta^{c,(1)} of Eq. (3.21).
  {3, {1.0L + 6.0L / 30, -4.0L / 30}, {0.0L, 0.0L, 1.0L / 30, 1.0L / 30, -4.0L / 30, 0.0L, 0.0L},
   {-4.0L / 60, 1.0L / 60, 0.0L, 0.0L}, {19.0L / 15, -1.0L / 15}},
  // WENOIU7-1MP: h+ of the Appendix, scheme (1) with alpha = 1, f_{j+1/2} + (-243 f_{j-3} +
  // 1990 f_{j-2} - 7481 f_{j-1} + 8164 f_j - 341 f_{j+1} - 2378 f_{j+2} + 289 f_{j+3}) / 107520;
  // its eighth-order delta^{c,(1)}: a_1..a_4 = (8841, -6069, 1261, -243/2) / 107520.
  {4, {1.0L, 0.0L},
   {-243.0L / 107520, 1990.0L / 107520, -7481.0L / 107520, 8164.0L / 107520, -341.0L / 107520,
    -2378.0L / 107520, 289.0L / 107520},
   {8841.0L / 107520, -6069.0L / 107520, 1261.0L / 107520, -121.5L / 107520}, {1.0L, 0.0L}},
  // WENOIU7-4MP: h+ of the Appendix, scheme (3), f_{j+1/2} + [(18 f_{j-1} - 66 f_j - 108 f_{j+1})
  // + (-3 f_{j-3/2} - 31 f_{j-1/2} + 179 f_{j+1/2} + 11 f_{j+3/2})] / 420; its delta^{c,(1)}:
  // [3 (f_{j+2} - f_{j-2}) - 32 (f_{j+1} - f_{j-1})] / 140 + [-3 (f~_{j+5/2} - f~_{j-5/2})
  // - 17 (f~_{j+3/2} - f~_{j-3/2}) + 1218 (f~_{j+1/2} - f~_{j-1/2})] / 840.
  {4, {1.0L + 179.0L / 420, -31.0L / 420}, {0.0L, 0.0L, 18.0L / 420, -66.0L / 420, -108.0L / 420, 0.0L, 0.0L},
   {-32.0L / 140, 3.0L / 140, 0.0L, 0.0L}, {1218.0L / 840, -17.0L / 840}, {-3.0L / 420, 11.0L / 420}, -3.0L / 840},
};

// The one-midpoint forms with their free parameter alpha (Eq. 3.5 for WENOIU3-1MP, Eq. 3.17
// for WENOIU5-1MP, the Appendix's scheme (1) for WENOIU7-1MP): h+ = alpha f_{j+1/2} +
// sum_k n_k(alpha) f_{j+k}; alpha = 1 gives the schemes of TAB.  The central operator that the
// metrics need is the central part of the scheme (Eq. 2.7): delta^{c,(1)} = (delta+ + delta-)/2
// with delta+ f_j = h+_{j+1/2} - h+_{j-1/2} and delta- its mirror, which gives
//   b_{1/2} = alpha,  a_d = (n_d - n_{d+1} + n_{1-d} - n_{-d}) / 2  (d = 1..4).
// For alpha = 1 the printed coefficients of TAB are used as they stand.
static SchemeTab scheme_tab(int scheme, long double alpha) {
  if (alpha == 1.0L || scheme < 0 || scheme > 5) return TAB[scheme < 0 || scheme > 5 ? 0 : scheme];
  SchemeTab S = TAB[scheme];
  long double n[7] = {0, 0, 0, 0, 0, 0, 0};   // n[k + 3] = n_k
  const long double a = alpha;
  if (scheme == S31) {          // Eq. (3.5)
    n[2] = a / 8 - 1.0L / 6; n[3] = -3 * a / 4 + 5.0L / 6; n[4] = -3 * a / 8 + 1.0L / 3;
  } else if (scheme == S51) {   // Eq. (3.17)
    n[1] = -3 * a / 128 + 1.0L / 30; n[2] = 5 * a / 32 - 13.0L / 60; n[3] = -45 * a / 64 + 47.0L / 60;
    n[4] = -15 * a / 32 + 9.0L / 20; n[5] = 5 * a / 128 - 1.0L / 20;
  } else if (scheme == S71) {   // Appendix, scheme (1)
    n[0] = 5 * a / 1024 - 1.0L / 140; n[1] = -21 * a / 512 + 5.0L / 84; n[2] = 175 * a / 1024 - 101.0L / 420;
    n[3] = -175 * a / 256 + 319.0L / 420; n[4] = -525 * a / 1024 + 107.0L / 210; n[5] = 35 * a / 512 - 19.0L / 210;
    n[6] = -7 * a / 1024 + 1.0L / 105;
  } else {
    return S;                   // the two-midpoint schemes have no free parameter (checked by the callers)
  }
  auto nk = [&](int k) { return k < -3 || k > 3 ? 0.0L : n[k + 3]; };
  S.hmid[0] = a;
  S.hmid[1] = 0.0L;
  for (int k = 0; k < 7; ++k) S.hnode[k] = n[k];
  for (int d = 1; d <= 4; ++d) S.cnode[d - 1] = (nk(d) - nk(d + 1) + nk(1 - d) - nk(-d)) / 2;
  S.cmid[0] = a;
  S.cmid[1] = 0.0L;
  return S;
}

// ----------------------------------------------------------------------------------
// Run parameters
// ----------------------------------------------------------------------------------
template <class T>
struct Par {
  int scheme = S51;
  int interp = 0;      // midpoint interpolation of nodal metric/coordinate values:
                       // 0 = central Lagrange matched to the order (4 points for the
                       //     third-order schemes, 6 points for the fifth-order ones),
                       // 1 = two-point average.
  int ppm = 1;         // 1: piecewise-polynomial mapping of the weights, Eq. (3.15)/(3.23)
  int linw = 0;        // 1: linear weights omega_k = C_k (no mapping)
  int weights = 0;     // 0: the weights of Eqs. (3.12)-(3.13); 1: WENO-Z weights (Section 7)
  int midsplit = 0;    // splitting of the midpoint flux: 0 Lax-Friedrichs type (Section 2.3),
                       // 1 Steger-Warming, 2 Van Leer (Section 7)
  int bc[4] = {0, 0, 0, 0};
  T gamma = T(1.4), alpha = cst<T>(1.1L), eps = cst<T>(1e-40L);
  long double halpha = 1.0L;   // the free parameter of the one-midpoint forms (3.5), (3.17), Appendix (1)
  SchemeTab tab;               // coefficients of the scheme at halpha
  T bcq[4][4];
  int ni = 0, nj = 0;
};

// ip = {scheme, interp, ppm, linear_weights, bc[4], weights, midsplit}; dp = {gamma, lf_alpha,
// eps, bc_state[4][4], scheme alpha}
template <class T>
static void unpack(const int* ip, const double* dp, int ni, int nj, Par<T>& P) {
  P.scheme = ip[0]; P.interp = ip[1]; P.ppm = ip[2]; P.linw = ip[3];
  for (int f = 0; f < 4; ++f) P.bc[f] = ip[4 + f];
  P.weights = ip[8]; P.midsplit = ip[9];
  P.gamma = T(dp[0]); P.alpha = T(dp[1]); P.eps = T(dp[2]);
  for (int f = 0; f < 4; ++f)
    for (int v = 0; v < 4; ++v) P.bcq[f][v] = T(dp[3 + 4 * f + v]);
  P.halpha = dp[19];
  P.tab = scheme_tab(P.scheme, P.halpha);
  P.ni = ni; P.nj = nj;
}

static inline int floordiv(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

// ----------------------------------------------------------------------------------
// Midpoint interpolation I of nodal values along one grid direction (Section 2.4).
// Reading: the paper asks for a "directionally consistent" linear interpolation and
// names none.  Default: the central Lagrange interpolant whose order matches the
// scheme; option: the two-point average.  phi(k) returns the nodal value at offset k
// from node j; the result approximates the value at j + 1/2.
// ----------------------------------------------------------------------------------
template <class T, class F>
static T interp_mid(int scheme, int interp, F phi) {
  if (interp == 1) return (phi(0) + phi(1)) * cst<T>(0.5L);
  if (scheme == S31 || scheme == S32)   // 4-point Lagrange
    return (cst<T>(-1) * phi(-1) + cst<T>(9) * phi(0) + cst<T>(9) * phi(1) - phi(2)) / cst<T>(16);
  if (scheme == S71 || scheme == S74)   // 8-point Lagrange
    return (cst<T>(-5) * phi(-3) + cst<T>(49) * phi(-2) - cst<T>(245) * phi(-1) + cst<T>(1225) * phi(0)
            + cst<T>(1225) * phi(1) - cst<T>(245) * phi(2) + cst<T>(49) * phi(3) - cst<T>(5) * phi(4))
           / cst<T>(2048);
  // 6-point Lagrange
  return (cst<T>(3) * phi(-2) - cst<T>(25) * phi(-1) + cst<T>(150) * phi(0) + cst<T>(150) * phi(1)
          - cst<T>(25) * phi(2) + cst<T>(3) * phi(3)) / cst<T>(256);
}

// The unit characteristic direction of an interface (Section 3.4): the average of its two
// nodes' direction metrics, normalised.
template <class T>
static void char_dir(T mx0, T my0, T mx1, T my1, T& nx, T& ny) {
  T mbx = cst<T>(0.5L) * (mx0 + mx1);
  T mby = cst<T>(0.5L) * (my0 + my1);
  T mb = sqrt(mbx * mbx + mby * mby);
  nx = mbx / mb;
  ny = mby / mb;
}

// ----------------------------------------------------------------------------------
// Coordinates with ghost nodes.
// Reading (boundaries are not treated in the paper): a periodic direction wraps and
// adds the period vector per wrap; any other direction extends the grid by odd
// reflection about the boundary node, x_{-k} = 2 x_0 - x_k.
// ----------------------------------------------------------------------------------
template <class T>
struct Coords {
  int ni, nj, bc[4];
  T per[2][2];          // per[0] = (dx, dy) added per wrap in i, per[1] likewise in j
  const T* x; const T* y;
  const Link* links = nullptr;       // 4 per block when some face is BC_LINK
  const Coords<T>* blocks = nullptr; // every block of a multi-block grid
  int hops = 0;
  void linked(int f, int i, int j, T& X, T& Y) const {
    const Link& L = links[f];
    const Coords<T>& N = blocks[L.nbr];
    int oi, oj;
    link_map(L, f, ni, nj, N.ni, N.nj, i, j, oi, oj);
    N.at(oi, oj, X, Y);
    X = X + T(L.off[0]); Y = Y + T(L.off[1]);
  }
  void at(int i, int j, T& X, T& Y) const {
    if (j < 0 || j >= nj) {
      if (bc[j < 0 ? 2 : 3] == BC_LINK) { linked(j < 0 ? 2 : 3, i, j, X, Y); return; }
      if (bc[2] == BC_PERIODIC) {
        int q = floordiv(j, nj);
        at(i, j - q * nj, X, Y);
        X = X + T(double(q)) * per[1][0]; Y = Y + T(double(q)) * per[1][1];
        return;
      }
      int jb = (j < 0) ? 0 : nj - 1;
      T X0, Y0, X1, Y1;
      at(i, jb, X0, Y0); at(i, 2 * jb - j, X1, Y1);
      X = cst<T>(2) * X0 - X1; Y = cst<T>(2) * Y0 - Y1;
      return;
    }
    if (i < 0 || i >= ni) {
      if (bc[i < 0 ? 0 : 1] == BC_LINK) { linked(i < 0 ? 0 : 1, i, j, X, Y); return; }
      if (bc[0] == BC_PERIODIC) {
        int q = floordiv(i, ni);
        at(i - q * ni, j, X, Y);
        X = X + T(double(q)) * per[0][0]; Y = Y + T(double(q)) * per[0][1];
        return;
      }
      int ib = (i < 0) ? 0 : ni - 1;
      T X0, Y0, X1, Y1;
      at(ib, j, X0, Y0); at(2 * ib - i, j, X1, Y1);
      X = cst<T>(2) * X0 - X1; Y = cst<T>(2) * Y0 - Y1;
      return;
    }
    X = x[(size_t)j * ni + i]; Y = y[(size_t)j * ni + i];
  }
};

// Central operator delta^{c,(1)} of the scheme (Eq. 2.7 and Eqs. 3.7/3.9/3.19/3.21),
// applied along direction dir at node (i, j) to the coordinate component comp
// (0 = x, 1 = y).  Midpoint values f~ come from the interpolation I above.
template <class T>
static T central_D(const Par<T>& P, const Coords<T>& C, int dir, int comp, int i, int j) {
  const SchemeTab& S = P.tab;
  auto node = [&](int k) {
    T X, Y;
    if (dir == 0) C.at(i + k, j, X, Y); else C.at(i, j + k, X, Y);
    return comp == 0 ? X : Y;
  };
  // midpoint value at node offset k + 1/2
  auto mid = [&](int k) {
    return interp_mid<T>(P.scheme, P.interp, [&](int l) { return node(k + l); });
  };
  T d = T(0);
  for (int k = 1; k <= 4; ++k)
    if (S.cnode[k - 1] != 0.0L) d = d + cst<T>(S.cnode[k - 1]) * (node(k) - node(-k));
  // b_{1/2} (f~_{j+1/2} - f~_{j-1/2}) + b_{3/2} (f~_{j+3/2} - f~_{j-3/2})
  d = d + cst<T>(S.cmid[0]) * (mid(0) - mid(-1));
  if (S.cmid[1] != 0.0L) d = d + cst<T>(S.cmid[1]) * (mid(1) - mid(-2));
  if (S.cmid3 != 0.0L) d = d + cst<T>(S.cmid3) * (mid(2) - mid(-3));
  return d;
}

// Conservative metrics in two dimensions (Eq. 2.3 with z = zeta) and the Jacobian
// (Eq. 2.5, whose 2-D form reduces to x_xi y_eta - x_eta y_xi), on the grid extended by
// G ghost layers.  Every derivative uses the scheme's central operator (Section 2.3).
template <class T>
static void metrics(const Par<T>& P, const Coords<T>& C, T* M) {
  const int ni = P.ni, nj = P.nj, W = ni + 2 * G, H = nj + 2 * G;
  const size_t plane = (size_t)W * H;
  for (int j = -G; j < nj + G; ++j)
    for (int i = -G; i < ni + G; ++i) {
      T x_xi = central_D(P, C, 0, 0, i, j), y_xi = central_D(P, C, 0, 1, i, j);
      T x_eta = central_D(P, C, 1, 0, i, j), y_eta = central_D(P, C, 1, 1, i, j);
      size_t o = (size_t)(j + G) * W + (i + G);
      M[0 * plane + o] = y_eta;        // xi_x^  =  y_eta
      M[1 * plane + o] = -x_eta;       // xi_y^  = -x_eta
      M[2 * plane + o] = -y_xi;        // eta_x^ = -y_xi
      M[3 * plane + o] = x_xi;         // eta_y^ =  x_xi
      M[4 * plane + o] = x_xi * y_eta - x_eta * y_xi;  // J^-1
    }
}

// ----------------------------------------------------------------------------------
// Euler flux, primitives, eigenvectors (Section 2.1, Section 3.4)
// ----------------------------------------------------------------------------------
template <class T>
static T pressure(const T* q, T gamma) {
  T u = q[1] / q[0], v = q[2] / q[0];
  return (gamma - cst<T>(1)) * (q[3] - cst<T>(0.5L) * q[0] * (u * u + v * v));
}

// Metric-weighted flux E^ = mx E + my F (Eq. 2.2, 2-D).
template <class T>
static void flux(const T* q, T mx, T my, T gamma, T* f) {
  T rho = q[0], u = q[1] / rho, v = q[2] / rho;
  T p = (gamma - cst<T>(1)) * (q[3] - cst<T>(0.5L) * rho * (u * u + v * v));
  T U = mx * u + my * v;
  f[0] = rho * U;
  f[1] = rho * u * U + mx * p;
  f[2] = rho * v * U + my * p;
  f[3] = (q[3] + p) * U;
}

// |U^| + c |k^| at a node (the spectral radius inside the MAX of Section 2.3).
template <class T>
static T spectral(const T* q, T mx, T my, T gamma) {
  T rho = q[0], u = q[1] / rho, v = q[2] / rho;
  T p = (gamma - cst<T>(1)) * (q[3] - cst<T>(0.5L) * rho * (u * u + v * v));
  T c = sqrt(gamma * p / rho);
  return fabs(mx * u + my * v) + c * sqrt(mx * mx + my * my);
}

// Splittings of the metric-weighted flux E^ = mx E + my F along k = (mx, my) for the midpoint
// flux f_{j+1/2}; Section 7 names Steger-Warming and Van Leer as alternatives that keep
// free-stream preservation.  sign = +1 gives F+, -1 gives F-; F+ + F- = E^.  With
// n = k/|k|, Un = u.n and the eigenvalues |k| (Un - c, Un, Un + c):
// Steger-Warming: F+- = rho/(2 gamma) [l1+- (1, u - c nx, v - c ny, H - c Un)
//   + 2 (gamma - 1) l2+- (1, u, v, |u|^2/2) + l3+- (1, u + c nx, v + c ny, H + c Un)],
//   l+- = (l +- |l|)/2.
template <class T>
static void split_sw(const T* q, T mx, T my, T gamma, int sign, T* f) {
  T rho = q[0], u = q[1] / rho, v = q[2] / rho;
  T q2 = u * u + v * v;
  T p = (gamma - cst<T>(1)) * (q[3] - cst<T>(0.5L) * rho * q2);
  T c = sqrt(gamma * p / rho);
  T kn = sqrt(mx * mx + my * my), nx = mx / kn, ny = my / kn;
  T Un = u * nx + v * ny, H = (q[3] + p) / rho;
  T l[3] = {kn * (Un - c), kn * Un, kn * (Un + c)};
  for (int i = 0; i < 3; ++i) l[i] = cst<T>(0.5L) * (l[i] + (sign > 0 ? fabs(l[i]) : -fabs(l[i])));
  T a = rho / (cst<T>(2) * gamma), g2 = cst<T>(2) * (gamma - cst<T>(1));
  f[0] = a * (l[0] + g2 * l[1] + l[2]);
  f[1] = a * (l[0] * (u - c * nx) + g2 * l[1] * u + l[2] * (u + c * nx));
  f[2] = a * (l[0] * (v - c * ny) + g2 * l[1] * v + l[2] * (v + c * ny));
  f[3] = a * (l[0] * (H - c * Un) + (gamma - cst<T>(1)) * l[1] * q2 + l[2] * (H + c * Un));
}
// Van Leer, with the normal Mach number M = Un/c: for M >= 1, F+ = E^ and F- = 0 (and the
// reverse for M <= -1); otherwise the mass flux m+- = +- rho c |k| (M +- 1)^2 / 4 and
// F+- = m+- (1, u + nx (-Un +- 2c)/gamma, v + ny (-Un +- 2c)/gamma,
//             ((gamma - 1) Un +- 2c)^2 / (2 (gamma^2 - 1)) + (|u|^2 - Un^2)/2).
template <class T>
static void split_vl(const T* q, T mx, T my, T gamma, int sign, T* f) {
  T rho = q[0], u = q[1] / rho, v = q[2] / rho;
  T q2 = u * u + v * v;
  T p = (gamma - cst<T>(1)) * (q[3] - cst<T>(0.5L) * rho * q2);
  T c = sqrt(gamma * p / rho);
  T kn = sqrt(mx * mx + my * my), nx = mx / kn, ny = my / kn;
  T Un = u * nx + v * ny, M = Un / c;
  if (M >= T(1) || M <= T(-1)) {
    if ((M >= T(1)) == (sign > 0)) {
      flux(q, mx, my, gamma, f);
    } else {
      for (int i = 0; i < 4; ++i) f[i] = T(0);
    }
    return;
  }
  T s = sign > 0 ? T(1) : T(-1);
  T mp = M + s;
  T fm = s * rho * c * kn * mp * mp / cst<T>(4);
  T w = (s * cst<T>(2) * c - Un) / gamma;
  T e = (gamma - cst<T>(1)) * Un + s * cst<T>(2) * c;
  f[0] = fm;
  f[1] = fm * (u + nx * w);
  f[2] = fm * (v + ny * w);
  f[3] = fm * (e * e / (cst<T>(2) * (gamma * gamma - cst<T>(1))) + cst<T>(0.5L) * (q2 - Un * Un));
}

// Left/right eigenvectors of the Jacobian of the flux in direction n (unit vector),
// evaluated at state q (Section 3.4).  Reading: the standard normalisation of the 2-D
// Euler eigenvectors; R columns are the acoustic, entropy, shear and acoustic waves.
template <class T>
static void eigvec(const T* q, T nx, T ny, T gamma, T L[4][4], T R[4][4]) {
  T rho = q[0], u = q[1] / rho, v = q[2] / rho;
  T q2 = u * u + v * v;
  T p = (gamma - cst<T>(1)) * (q[3] - cst<T>(0.5L) * rho * q2);
  T c = sqrt(gamma * p / rho);
  T H = (q[3] + p) / rho;
  T Un = u * nx + v * ny, Ut = v * nx - u * ny;
  T b1 = (gamma - cst<T>(1)) / (c * c), b2 = cst<T>(0.5L) * b1 * q2;
  const T h = cst<T>(0.5L);
  // right eigenvectors as columns
  R[0][0] = T(1);           R[0][1] = T(1);              R[0][2] = T(0);  R[0][3] = T(1);
  R[1][0] = u - c * nx;     R[1][1] = u;                 R[1][2] = -ny;   R[1][3] = u + c * nx;
  R[2][0] = v - c * ny;     R[2][1] = v;                 R[2][2] = nx;    R[2][3] = v + c * ny;
  R[3][0] = H - c * Un;     R[3][1] = h * q2;            R[3][2] = Ut;    R[3][3] = H + c * Un;
  // left eigenvectors as rows
  L[0][0] = h * (b2 + Un / c); L[0][1] = h * (-b1 * u - nx / c); L[0][2] = h * (-b1 * v - ny / c); L[0][3] = h * b1;
  L[1][0] = T(1) - b2;         L[1][1] = b1 * u;                L[1][2] = b1 * v;                L[1][3] = -b1;
  L[2][0] = -Ut;               L[2][1] = -ny;                   L[2][2] = nx;                    L[2][3] = T(0);
  L[3][0] = h * (b2 - Un / c); L[3][1] = h * (-b1 * u + nx / c); L[3][2] = h * (-b1 * v + ny / c); L[3][3] = h * b1;
}

// ----------------------------------------------------------------------------------
// WENO interpolation to the midpoint x_{j+1/2} (Eqs. 3.10-3.13, Table 1), smoothness
// indicators of Eq. (3.22), mapping of Eq. (3.15) (r = 2) or Eq. (3.23) (r = 3).
// u[0..4] = u_{j-2} .. u_{j+2}.
// Reading (Section 5.1): the third-order (r = 2) interpolation takes IS_0 and IS_1 of
// Eq. (3.22), i.e. the three-point stencils {j-2, j-1, j} and {j-1, j, j+1}, instead of
// Eq. (3.14).  The indicators are written in the equivalent sum-of-squares form
// (13/12 (second difference)^2 + 1/4 (first difference)^2), algebraically identical to the
// printed quadratic forms.
// ----------------------------------------------------------------------------------
// With the consecutive differences da = b - a, db = c - b of a three-point stencil
// (a, b, c): second difference a - 2b + c = db - da; the first-difference terms are
// a - 4b + 3c = 3 db - da (IS_0), a - c = -(da + db) (IS_1), 3a - 4b + c = db - 3 da (IS_2).
// Written on differences, every indicator is exactly zero on constant data.
template <class T>
static T is0(T a, T b, T c) {
  T da = b - a, db = c - b;
  T d2 = db - da, d1 = cst<T>(3) * db - da;
  return cst<T>(13.0L / 12) * d2 * d2 + cst<T>(0.25L) * d1 * d1;
}
template <class T>
static T is1(T a, T b, T c) {
  T da = b - a, db = c - b;
  T d2 = db - da, d1 = da + db;
  return cst<T>(13.0L / 12) * d2 * d2 + cst<T>(0.25L) * d1 * d1;
}
template <class T>
static T is2(T a, T b, T c) {
  T da = b - a, db = c - b;
  T d2 = db - da, d1 = db - cst<T>(3) * da;
  return cst<T>(13.0L / 12) * d2 * d2 + cst<T>(0.25L) * d1 * d1;
}

// Smoothness indicators of the r = 4 candidates (WENOIU7).  Reading: the paper gives none
// for r = 4; Eq. (3.22) is the integral over [x_{j-1/2}, x_{j+1/2}] of the squared first and
// second derivatives (times h and h^3) of each candidate's interpolating polynomial, and the
// same definition is applied to the cubics of Table A1 (first to third derivatives, times h,
// h^3, h^5).  Each is the quadratic form d^T A_k d in the differences d_i = u_{o_i} - u_{o_{i-1}}
// of the candidate's four values (stencil j-3+k .. j+k); entries are in units of 1/2880.
static const long double IS4[4][3][3] = {
  {{6649, -16958, 11389}, {-16958, 45076, -31718}, {11389, -31718, 25729}},
  {{3169, -6518, 2989}, {-6518, 17236, -8558}, {2989, -8558, 6649}},
  {{6649, -8558, 2989}, {-8558, 17236, -6518}, {2989, -6518, 3169}},
  {{25729, -31718, 11389}, {-31718, 45076, -16958}, {11389, -16958, 6649}},
};

template <class T>
static T is_r4(int k, const T* v) {
  // the coefficients in the scalar type, converted once (long double is software arithmetic
  // on some hosts)
  static const struct Coef {
    T c[4][3][3];
    Coef() {
      for (int q = 0; q < 4; ++q)
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) c[q][a][b] = cst<T>(IS4[q][a][b] / 2880.0L);
    }
  } A;
  T d[3] = {v[1] - v[0], v[2] - v[1], v[3] - v[2]};
  T s = T(0);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) s = s + A.c[k][a][b] * d[a] * d[b];
  return s;
}

// Piecewise-polynomial mapping g(omega) about C: Eq. (3.15) for order 2, Eq. (3.23) for 3,
// and the fourth-order mapping of the Appendix for r = 4.
template <class T>
static T ppm_map(int order, T w, T C) {
  if (order == 2) {
    if (w <= C) { T s = w / C - cst<T>(1); return C * (cst<T>(1) - s * s); }
    T d = w - C; return C - d * d / (C - cst<T>(1));
  }
  if (order == 4) {
    if (w <= C) { T s = w / C - cst<T>(1); return C * (cst<T>(1) - s * s * s * s); }
    T d = w - C, e = C - cst<T>(1);
    return C - d * d * d * d / (e * e * e);
  }
  if (w <= C) { T s = w / C - cst<T>(1); return C * (cst<T>(1) + s * s * s); }
  T d = w - C, e = C - cst<T>(1);
  return C + d * d * d / (e * e);
}

struct WenoOpt { int ppm, linw, z = 0; };   // z: WENO-Z weights (no mapping)

// WENO interpolation to x_{j+1/2} from u[m + 3] = u_{j+m}, m = -3..3 (Eqs. 3.10-3.13;
// candidates of Table 1, or Table A1 for r = 4).
template <class T>
static T weno_mid(int r, const T* u, const WenoOpt& o, T eps) {
  static const long double b2[2][2] = {{-0.5L, 1.5L}, {0.5L, 0.5L}};
  static const long double c2[2] = {0.25L, 0.75L};
  static const long double b3[3][3] = {{3.0L / 8, -10.0L / 8, 15.0L / 8},
                                       {-1.0L / 8, 6.0L / 8, 3.0L / 8},
                                       {3.0L / 8, 6.0L / 8, -1.0L / 8}};
  static const long double c3[3] = {1.0L / 16, 10.0L / 16, 5.0L / 16};
  static const long double b4[4][4] = {{-5.0L / 16, 21.0L / 16, -35.0L / 16, 35.0L / 16},
                                       {1.0L / 16, -5.0L / 16, 15.0L / 16, 5.0L / 16},
                                       {-1.0L / 16, 9.0L / 16, 9.0L / 16, -1.0L / 16},
                                       {5.0L / 16, 15.0L / 16, -5.0L / 16, 1.0L / 16}};
  static const long double c4[4] = {1.0L / 64, 21.0L / 64, 35.0L / 64, 7.0L / 64};
  const T* uj = u + 3;   // uj[m] = u_{j+m}
  T p[4], IS[4], Ck[4];
  if (r == 4) {
    static const struct Tab4 {
      T b[4][4], c[4];
      Tab4() {
        for (int k = 0; k < 4; ++k) {
          c[k] = cst<T>(c4[k]);
          for (int l = 0; l < 4; ++l) b[k][l] = cst<T>(b4[k][l]);
        }
      }
    } tab4;
    for (int k = 0; k < 4; ++k) {
      // p_k = sum_l b_{k,l} u_{j-r+k+l+1} (Eq. 3.11)
      p[k] = T(0);
      for (int l = 0; l < 4; ++l) p[k] = p[k] + tab4.b[k][l] * uj[k + l - 3];
      Ck[k] = tab4.c[k];
      IS[k] = is_r4(k, uj + k - 3);
    }
  } else if (r == 3) {
    for (int k = 0; k < 3; ++k) {
      p[k] = T(0);
      for (int l = 0; l < 3; ++l) p[k] = p[k] + cst<T>(b3[k][l]) * uj[k + l - 2];
      Ck[k] = cst<T>(c3[k]);
    }
    IS[0] = is0(uj[-2], uj[-1], uj[0]);
    IS[1] = is1(uj[-1], uj[0], uj[1]);
    IS[2] = is2(uj[0], uj[1], uj[2]);
  } else {
    for (int k = 0; k < 2; ++k) {
      p[k] = T(0);
      for (int l = 0; l < 2; ++l) p[k] = p[k] + cst<T>(b2[k][l]) * uj[k + l - 1];
      Ck[k] = cst<T>(c2[k]);
    }
    IS[0] = is0(uj[-2], uj[-1], uj[0]);
    IS[1] = is1(uj[-1], uj[0], uj[1]);
  }
  T w[4];
  if (o.linw) {
    for (int k = 0; k < r; ++k) w[k] = Ck[k];
  } else if (o.z) {
    // WENO-Z weights (Section 7 names them; Borges et al.'s form with the squared ratio):
    // alpha_k = C_k (1 + (tau / (eps + IS_k))^2), omega_k = alpha_k / sum alpha, with the
    // global indicator tau = |IS_0 - IS_{r-1}| (r = 2, 3) or |IS_0 + 3 IS_1 - 3 IS_2 - IS_3|
    // (r = 4).  The mapping is not applied.
    T tau = r == 4 ? fabs(IS[0] + cst<T>(3) * IS[1] - cst<T>(3) * IS[2] - IS[3]) : fabs(IS[0] - IS[r - 1]);
    T a[4], s = T(0);
    for (int k = 0; k < r; ++k) {
      T q = tau / (eps + IS[k]);
      a[k] = Ck[k] * (cst<T>(1) + q * q);
      s = s + a[k];
    }
    for (int k = 0; k < r; ++k) w[k] = a[k] / s;
  } else {
    // alpha_k = C_k / (eps + IS_k)^2, omega_k = alpha_k / sum alpha (Eqs. 3.12-3.13)
    T a[4], s = T(0);
    for (int k = 0; k < r; ++k) { T d = eps + IS[k]; a[k] = Ck[k] / (d * d); s = s + a[k]; }
    for (int k = 0; k < r; ++k) w[k] = a[k] / s;
    if (o.ppm) {
      // map each omega_k with its own C_k, then normalise the mapped values
      T g[4], sg = T(0);
      for (int k = 0; k < r; ++k) { g[k] = ppm_map(r, w[k], Ck[k]); sg = sg + g[k]; }
      for (int k = 0; k < r; ++k) w[k] = g[k] / sg;
    }
  }
  T out = T(0);
  for (int k = 0; k < r; ++k) out = out + w[k] * p[k];   // Eq. (3.10)
  return out;
}

// ----------------------------------------------------------------------------------
// Semi-discrete right-hand side (Sections 2.3, 3, 3.4)
// ----------------------------------------------------------------------------------
template <class T>
struct Field {
  const Par<T>& P;
  const T* M;   // haloed metrics
  const T* Q;   // [4][nj][ni]
  const Link* links = nullptr;        // 4 per block when some face is BC_LINK
  const Field<T>* blocks = nullptr;   // every block of a multi-block grid
  size_t mplane() const { return (size_t)(P.ni + 2 * G) * (P.nj + 2 * G); }
  T met(int p, int i, int j) const {
    return M[p * mplane() + (size_t)(j + G) * (P.ni + 2 * G) + (i + G)];
  }
  T q(int v, int i, int j) const { return Q[(size_t)v * P.ni * P.nj + (size_t)j * P.ni + i]; }

  // State at position s of line L in direction dir, with ghost values by the boundary
  // rule of the face.  Reading (the paper does not treat boundaries): periodic wraps;
  // transmissive copies the boundary node; Dirichlet gives the prescribed state; slip
  // wall mirrors node s about the boundary node and reverses the velocity component
  // along the boundary node's grid-direction normal; far field takes the prescribed
  // state where the prescribed velocity enters through the face, else is transmissive.
  void state(int dir, int L, int s, T* out) const {
    const int n = dir == 0 ? P.ni : P.nj;
    auto rd = [&](int ss, T* o) {
      for (int v = 0; v < 4; ++v) o[v] = dir == 0 ? q(v, ss, L) : q(v, L, ss);
    };
    if (s >= 0 && s < n) { rd(s, out); return; }
    const int face = 2 * dir + (s < 0 ? 0 : 1);
    const int b = s < 0 ? 0 : n - 1;
    switch (P.bc[face]) {
      case BC_PERIODIC: { int ss = s - floordiv(s, n) * n; rd(ss, out); return; }
      case BC_LINK: {   // the neighbour block's node behind the face
        const Link& Lk = links[face];
        const Field<T>& N = blocks[Lk.nbr];
        const int gi = dir == 0 ? s : L, gj = dir == 0 ? L : s;
        int oi, oj;
        link_map(Lk, face, P.ni, P.nj, N.P.ni, N.P.nj, gi, gj, oi, oj);
        for (int v = 0; v < 4; ++v) out[v] = N.q(v, oi, oj);
        return;
      }
      case BC_TRANSMISSIVE: rd(b, out); return;
      case BC_DIRICHLET: for (int v = 0; v < 4; ++v) out[v] = P.bcq[face][v]; return;
      case BC_SLIPWALL: {
        int sm = 2 * b - s;
        rd(sm, out);
        T mx = dir == 0 ? met(0, b, L) : met(2, L, b);
        T my = dir == 0 ? met(1, b, L) : met(3, L, b);
        T mn = sqrt(mx * mx + my * my), nx = mx / mn, ny = my / mn;
        T un = out[1] * nx + out[2] * ny;
        out[1] = out[1] - cst<T>(2) * un * nx;
        out[2] = out[2] - cst<T>(2) * un * ny;
        return;
      }
      case BC_FARFIELD: {
        T mx = dir == 0 ? met(0, b, L) : met(2, L, b);
        T my = dir == 0 ? met(1, b, L) : met(3, L, b);
        T sgn = s < 0 ? T(-1) : T(1);
        T vn = sgn * (P.bcq[face][1] * mx + P.bcq[face][2] * my);   // outward momentum flux
        if (vn < T(0)) { for (int v = 0; v < 4; ++v) out[v] = P.bcq[face][v]; }
        else rd(b, out);
        return;
      }
    }
    rd(b, out);
  }
  void nodemet(int dir, int L, int s, T& mx, T& my) const {
    const int n = dir == 0 ? P.ni : P.nj;
    if (s < -G || s >= n + G) s = s - floordiv(s, n) * n;   // beyond the stored ghosts: periodic
    if (dir == 0) { mx = met(0, s, L); my = met(1, s, L); }
    else { mx = met(2, L, s); my = met(3, L, s); }
  }
};

// A^ of the Lax-Friedrichs-type splitting (Section 2.3): alpha times the maximum of
// |U^| + c |k^| over the interior nodes of the grid line.  Reading: the printed
// MAX(U^ + c|k^|) is taken with |U^| (a wave speed), and the maximum runs over the
// line's interior nodes; ties keep the lowest index (matters only for derivatives).
template <class T>
static T line_lambda(const Field<T>& F, int dir, int L) {
  const int n = dir == 0 ? F.P.ni : F.P.nj;
  T best = T(0);
  for (int s = 0; s < n; ++s) {
    T q[4], mx, my;
    F.state(dir, L, s, q);
    F.nodemet(dir, L, s, mx, my);
    T sp = spectral(q, mx, my, F.P.gamma);
    if (s == 0 || sp > best) best = sp;
  }
  return F.P.alpha * best;
}

// One direction: accumulates (H_{s+1/2} - H_{s-1/2}) into R for every node of every line.
template <class T>
static void sweep(const Field<T>& F, int dir, std::vector<T>& R) {
  const Par<T>& P = F.P;
  const SchemeTab& S = P.tab;
  const int n = dir == 0 ? P.ni : P.nj, nl = dir == 0 ? P.nj : P.ni;
  // nodes s = -OFF .. n+OFF-1 (OFF = 4, or 6 for the four-midpoint scheme) at s + 4 of the
  // arrays below (which start two nodes into their storage); interfaces p + 1/2, p = -nmp ..
  // n-2+nmp, at p + 2 (one interface into the storage)
  const bool four = S.hmidx[0] != 0.0L || S.hmidx[1] != 0.0L;
  const int OFF = four ? 6 : 4;
  const int NB = n + 12, NI = n + 5;
  const WenoOpt wo{P.ppm, P.linw, P.weights};
  std::vector<T> sq(4 * NB), smx(NB), smy(NB), sfp(4 * NB), sfm(4 * NB);
  std::vector<T> sfpm(4 * NI), sfmm(4 * NI), sHh(4 * NI);
  T *q = sq.data() + 8, *mxs = smx.data() + 2, *mys = smy.data() + 2, *fp = sfp.data() + 8, *fm = sfm.data() + 8;
  T *fpm = sfpm.data() + 4, *fmm = sfmm.data() + 4, *Hh = sHh.data() + 4;
  for (int L = 0; L < nl; ++L) {
    const T A = line_lambda(F, dir, L);
    // node states, metrics and split fluxes f+- = (E^ +- A^ Q)/2
    for (int s = -OFF; s < n + OFF; ++s) {
      T qs[4], f[4];
      F.state(dir, L, s, qs);
      F.nodemet(dir, L, s, mxs[s + 4], mys[s + 4]);
      flux(qs, mxs[s + 4], mys[s + 4], P.gamma, f);
      for (int v = 0; v < 4; ++v) {
        q[4 * (s + 4) + v] = qs[v];
        fp[4 * (s + 4) + v] = cst<T>(0.5L) * (f[v] + A * qs[v]);
        fm[4 * (s + 4) + v] = cst<T>(0.5L) * (f[v] - A * qs[v]);
      }
    }
    // interfaces: characteristic WENO interpolation from each side, then split fluxes;
    // h at p + 1/2 (p = -1 .. n-1) uses midpoints p + 1/2 only (one-midpoint schemes) or
    // p - 1/2 .. p + 3/2 (two-midpoint schemes)
    // (the four-midpoint scheme: p - 3/2 .. p + 5/2)
    const int nmp = four ? 3 : S.hmid[1] != 0.0L ? 2 : 1;
    for (int p = -nmp; p <= n - 2 + nmp; ++p) {
      const int c0 = p + 4;                    // node p
      // characteristic direction from the averaged metrics (Section 3.4)
      T nx, ny;
      char_dir<T>(mxs[c0], mys[c0], mxs[c0 + 1], mys[c0 + 1], nx, ny);
      T Qs[2][4];
      for (int side = 0; side < 2; ++side) {
        // side 0 ("+"): eigenvectors at Q_p, stencil p-2..p+2;
        // side 1 ("-"): eigenvectors at Q_{p+1}, mirrored stencil p+3..p-1.
        const int ce = side == 0 ? c0 : c0 + 1;
        T Lm[4][4], Rm[4][4];
        eigvec(&q[4 * ce], nx, ny, P.gamma, Lm, Rm);
        T Wmid[4];
        const int half = S.r == 4 ? 3 : 2;     // stencil j-half .. j+half of the side
        for (int k = 0; k < 4; ++k) {
          T u[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
          for (int m = -half; m <= half; ++m) {
            const int node = side == 0 ? c0 + m : c0 + 1 - m;
            T w = T(0);
            for (int v = 0; v < 4; ++v) w = w + Lm[k][v] * q[4 * node + v];
            u[m + 3] = w;
          }
          Wmid[k] = weno_mid(S.r, u, wo, P.eps);
        }
        for (int v = 0; v < 4; ++v) {
          T acc = T(0);
          for (int k = 0; k < 4; ++k) acc = acc + Rm[v][k] * Wmid[k];
          Qs[side][v] = acc;
        }
      }
      // midpoint metrics by the same interpolation I as the metric evaluation
      T mmx = interp_mid<T>(P.scheme, P.interp, [&](int l) { return mxs[c0 + l]; });
      T mmy = interp_mid<T>(P.scheme, P.interp, [&](int l) { return mys[c0 + l]; });
      T fpl[4], fmi[4];
      if (P.midsplit == 0) {
        // the Lax-Friedrichs-type splitting of the nodes (Section 2.3)
        flux(Qs[0], mmx, mmy, P.gamma, fpl);
        flux(Qs[1], mmx, mmy, P.gamma, fmi);
        for (int v = 0; v < 4; ++v) {
          fpm[4 * (p + 2) + v] = cst<T>(0.5L) * (fpl[v] + A * Qs[0][v]);
          fmm[4 * (p + 2) + v] = cst<T>(0.5L) * (fmi[v] - A * Qs[1][v]);
        }
      } else {
        // Steger-Warming or Van Leer at the midpoint (Section 7)
        if (P.midsplit == 1) { split_sw(Qs[0], mmx, mmy, P.gamma, 1, fpl); split_sw(Qs[1], mmx, mmy, P.gamma, -1, fmi); }
        else { split_vl(Qs[0], mmx, mmy, P.gamma, 1, fpl); split_vl(Qs[1], mmx, mmy, P.gamma, -1, fmi); }
        for (int v = 0; v < 4; ++v) {
          fpm[4 * (p + 2) + v] = fpl[v];
          fmm[4 * (p + 2) + v] = fmi[v];
        }
      }
    }
    // h = h+ + h-; h- mirrors h+ about x_{p+1/2}: f_{p+k} -> f_{p+1-k},
    // f_{p+1/2+m} -> f_{p+1/2-m}
    for (int p = -1; p <= n - 1; ++p) {
      for (int v = 0; v < 4; ++v) {
        T hp = T(0), hm = T(0);
        for (int m = 0; m >= -1; --m) {
          if (S.hmid[-m] == 0.0L) continue;
          hp = hp + cst<T>(S.hmid[-m]) * fpm[4 * (p + m + 2) + v];
          hm = hm + cst<T>(S.hmid[-m]) * fmm[4 * (p - m + 2) + v];
        }
        if (four) {   // f+_{p-3/2}, f+_{p+3/2} and their mirrors f-_{p+5/2}, f-_{p-1/2}
          hp = hp + cst<T>(S.hmidx[0]) * fpm[4 * (p - 2 + 2) + v] + cst<T>(S.hmidx[1]) * fpm[4 * (p + 1 + 2) + v];
          hm = hm + cst<T>(S.hmidx[0]) * fmm[4 * (p + 2 + 2) + v] + cst<T>(S.hmidx[1]) * fmm[4 * (p - 1 + 2) + v];
        }
        for (int k = -3; k <= 3; ++k) {
          if (S.hnode[k + 3] == 0.0L) continue;
          hp = hp + cst<T>(S.hnode[k + 3]) * fp[4 * (p + k + 4) + v];
          hm = hm + cst<T>(S.hnode[k + 3]) * fm[4 * (p + 1 - k + 4) + v];
        }
        Hh[4 * (p + 2) + v] = hp + hm;
      }
    }
    // difference (Eq. 3.2 with unit spacing)
    for (int s = 0; s < n; ++s) {
      const int i = dir == 0 ? s : L, j = dir == 0 ? L : s;
      for (int v = 0; v < 4; ++v) {
        size_t o = (size_t)v * P.ni * P.nj + (size_t)j * P.ni + i;
        R[o] = R[o] + (Hh[4 * (s + 2) + v] - Hh[4 * (s + 1) + v]);
      }
    }
  }
}

// dQ/dt = -(dE^/dxi + dF^/deta) / J^-1 (Eq. 2.2 on a stationary grid).
template <class T>
static void rhs_field(const Field<T>& F, T* dQ) {
  const Par<T>& P = F.P;
  const size_t N = (size_t)P.ni * P.nj;
  std::vector<T> R(4 * N, T(0));
  sweep(F, 0, R);
  sweep(F, 1, R);
  for (int j = 0; j < P.nj; ++j)
    for (int i = 0; i < P.ni; ++i) {
      T Jinv = F.met(4, i, j);
      for (int v = 0; v < 4; ++v) {
        size_t o = (size_t)v * N + (size_t)j * P.ni + i;
        dQ[o] = -R[o] / Jinv;
      }
    }
}

template <class T>
static void rhs(const Par<T>& P, const T* M, const T* Q, T* dQ) {
  Field<T> F{P, M, Q};
  rhs_field(F, dQ);
}

// Third-order TVD Runge-Kutta (Section 6), Shu-Osher form.
template <class T>
static void rk3(const Par<T>& P, const T* M, T* Q, T dt) {
  const size_t N = 4 * (size_t)P.ni * P.nj;
  std::vector<T> R(N), Q1(N), Q2(N);
  rhs(P, M, Q, R.data());
  for (size_t k = 0; k < N; ++k) Q1[k] = Q[k] + dt * R[k];
  rhs(P, M, Q1.data(), R.data());
  for (size_t k = 0; k < N; ++k) Q2[k] = cst<T>(0.75L) * Q[k] + cst<T>(0.25L) * (Q1[k] + dt * R[k]);
  rhs(P, M, Q2.data(), R.data());
  for (size_t k = 0; k < N; ++k)
    Q[k] = cst<T>(1.0L / 3) * Q[k] + cst<T>(2.0L / 3) * (Q2[k] + dt * R[k]);
}

// Reading (the paper uses fixed steps): dt = CFL / max over interior nodes of
// [(|U^_xi| + c |grad xi^|) + (|U^_eta| + c |grad eta^|)] / J^-1.
template <class T>
static T cfl_dt(const Par<T>& P, const T* M, const T* Q, T cfl) {
  Field<T> F{P, M, Q};
  T best = T(0);
  for (int j = 0; j < P.nj; ++j)
    for (int i = 0; i < P.ni; ++i) {
      T q[4];
      for (int v = 0; v < 4; ++v) q[v] = F.q(v, i, j);
      T s = (spectral(q, F.met(0, i, j), F.met(1, i, j), P.gamma) +
             spectral(q, F.met(2, i, j), F.met(3, i, j), P.gamma)) / F.met(4, i, j);
      if (s > best) best = s;
    }
  return cfl / best;
}

// ----------------------------------------------------------------------------------
// Scalar linear advection u_t + u_x = 0 (Section 5.1, Table 3): periodic [-1, 1),
// N nodes, upwind split f+ = u, f- = 0 (reading), classical RK4 with
// dt = 2 / ceil(2 / dx^{5/4}), final time t.
// ----------------------------------------------------------------------------------
static void advect_rhs(int scheme, int N, double dx, const std::vector<double>& u,
                       std::vector<double>& du, int z = 0) {
  const SchemeTab& S = TAB[scheme];
  const WenoOpt wo{1, 0, z};
  auto U = [&](int k) { return u[(size_t)(((k % N) + N) % N)]; };
  std::vector<double> fmid(N), h(N);
  for (int p = 0; p < N; ++p) {              // f+_{p+1/2}
    double st[7];
    for (int m = -3; m <= 3; ++m) st[m + 3] = U(p + m);
    fmid[p] = weno_mid<double>(S.r, st, wo, 1e-40);
  }
  for (int p = 0; p < N; ++p) {              // h_{p+1/2}
    double hp = 0.0;
    for (int m = 0; m >= -1; --m)
      if (S.hmid[-m] != 0.0L) hp += (double)S.hmid[-m] * fmid[(size_t)(((p + m) % N + N) % N)];
    if (S.hmidx[0] != 0.0L) hp += (double)S.hmidx[0] * fmid[(size_t)(((p - 2) % N + N) % N)];
    if (S.hmidx[1] != 0.0L) hp += (double)S.hmidx[1] * fmid[(size_t)(((p + 1) % N + N) % N)];
    for (int k = -3; k <= 3; ++k)
      if (S.hnode[k + 3] != 0.0L) hp += (double)S.hnode[k + 3] * U(p + k);
    h[p] = hp;
  }
  for (int p = 0; p < N; ++p) du[p] = -(h[p] - h[(p + N - 1) % N]) / dx;
}

static void advect1d(int scheme, int N, double tfinal, double* out, double dt_exp = 1.25, int z = 0) {
  const double PI = 3.14159265358979323846;
  const double dx = 2.0 / N;
  auto u0 = [&](double x) { return std::sin(PI * x - std::sin(PI * x) / PI); };
  std::vector<double> u(N), k1(N), k2(N), k3(N), k4(N), tmp(N);
  for (int i = 0; i < N; ++i) u[i] = u0(-1.0 + dx * i);
  const int nsteps = (int)std::ceil(tfinal / std::pow(dx, dt_exp));
  const double dt = tfinal / nsteps;
  for (int st = 0; st < nsteps; ++st) {
    advect_rhs(scheme, N, dx, u, k1, z);
    for (int i = 0; i < N; ++i) tmp[i] = u[i] + 0.5 * dt * k1[i];
    advect_rhs(scheme, N, dx, tmp, k2, z);
    for (int i = 0; i < N; ++i) tmp[i] = u[i] + 0.5 * dt * k2[i];
    advect_rhs(scheme, N, dx, tmp, k3, z);
    for (int i = 0; i < N; ++i) tmp[i] = u[i] + dt * k3[i];
    advect_rhs(scheme, N, dx, tmp, k4, z);
    for (int i = 0; i < N; ++i) u[i] += dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  }
  double s2 = 0.0, smax = 0.0;
  for (int i = 0; i < N; ++i) {
    // exact solution: the initial profile translated by t (period 2)
    double xe = -1.0 + dx * i - tfinal;
    xe = xe - 2.0 * std::floor((xe + 1.0) / 2.0);
    double e = std::fabs(u[i] - u0(xe));
    s2 += e * e; smax = std::max(smax, e);
  }
  out[0] = std::sqrt(s2 / N);   // L2 = root mean square
  out[1] = smax;
  out[2] = (double)nsteps;
}

// ----------------------------------------------------------------------------------
// Exact solution of the 1-D Riemann problem for an ideal gas (used to check Sod):
// pressure in the star region by Newton iteration on the sum of the two wave
// functions (shock: Rankine-Hugoniot, rarefaction: isentropic), then sampling of x/t.
// ----------------------------------------------------------------------------------
static void riemann_exact(double g, const double* WL, const double* WR, double x0, double t,
                          int n, const double* x, double* out) {
  const double rl = WL[0], ul = WL[1], pl = WL[2], rr = WR[0], ur = WR[1], pr = WR[2];
  const double cl = std::sqrt(g * pl / rl), cr = std::sqrt(g * pr / rr);
  auto fk = [&](double p, double rk, double pk, double ck, double& df) {
    if (p > pk) {  // shock
      double A = 2.0 / ((g + 1.0) * rk), B = (g - 1.0) / (g + 1.0) * pk;
      double s = std::sqrt(A / (p + B));
      df = s * (1.0 - 0.5 * (p - pk) / (p + B));
      return (p - pk) * s;
    }
    double e = (g - 1.0) / (2.0 * g);   // rarefaction
    double f = 2.0 * ck / (g - 1.0) * (std::pow(p / pk, e) - 1.0);
    df = 1.0 / (rk * ck) * std::pow(p / pk, -(g + 1.0) / (2.0 * g));
    return f;
  };
  double p = 0.5 * (pl + pr);
  for (int it = 0; it < 100; ++it) {
    double dl, dr;
    double f = fk(p, rl, pl, cl, dl) + fk(p, rr, pr, cr, dr) + (ur - ul);
    double pn = p - f / (dl + dr);
    if (pn < 1e-12) pn = 1e-12;
    if (std::fabs(pn - p) < 1e-15 * (pn + p)) { p = pn; break; }
    p = pn;
  }
  double dl, dr;
  const double fl = fk(p, rl, pl, cl, dl), fr = fk(p, rr, pr, cr, dr);
  const double us = 0.5 * (ul + ur) + 0.5 * (fr - fl);
  for (int k = 0; k < n; ++k) {
    const double S = (x[k] - x0) / t;
    double r, u, pp;
    if (S <= us) {   // left of the contact
      if (p > pl) {
        double SL = ul - cl * std::sqrt((g + 1.0) / (2.0 * g) * p / pl + (g - 1.0) / (2.0 * g));
        if (S <= SL) { r = rl; u = ul; pp = pl; }
        else { r = rl * ((p / pl + (g - 1.0) / (g + 1.0)) / ((g - 1.0) / (g + 1.0) * p / pl + 1.0)); u = us; pp = p; }
      } else {
        double SHL = ul - cl, cs = cl * std::pow(p / pl, (g - 1.0) / (2.0 * g)), STL = us - cs;
        if (S <= SHL) { r = rl; u = ul; pp = pl; }
        else if (S > STL) { r = rl * std::pow(p / pl, 1.0 / g); u = us; pp = p; }
        else {
          u = 2.0 / (g + 1.0) * (cl + (g - 1.0) / 2.0 * ul + S);
          double c = 2.0 / (g + 1.0) * (cl + (g - 1.0) / 2.0 * (ul - S));
          r = rl * std::pow(c / cl, 2.0 / (g - 1.0)); pp = pl * std::pow(c / cl, 2.0 * g / (g - 1.0));
        }
      }
    } else {
      if (p > pr) {
        double SR = ur + cr * std::sqrt((g + 1.0) / (2.0 * g) * p / pr + (g - 1.0) / (2.0 * g));
        if (S >= SR) { r = rr; u = ur; pp = pr; }
        else { r = rr * ((p / pr + (g - 1.0) / (g + 1.0)) / ((g - 1.0) / (g + 1.0) * p / pr + 1.0)); u = us; pp = p; }
      } else {
        double SHR = ur + cr, cs = cr * std::pow(p / pr, (g - 1.0) / (2.0 * g)), STR = us + cs;
        if (S >= SHR) { r = rr; u = ur; pp = pr; }
        else if (S < STR) { r = rr * std::pow(p / pr, 1.0 / g); u = us; pp = p; }
        else {
          u = 2.0 / (g + 1.0) * (-cr + (g - 1.0) / 2.0 * ur + S);
          double c = 2.0 / (g + 1.0) * (cr - (g - 1.0) / 2.0 * (ur - S));
          r = rr * std::pow(c / cr, 2.0 / (g - 1.0)); pp = pr * std::pow(c / cr, 2.0 * g / (g - 1.0));
        }
      }
    }
    out[3 * k + 0] = r; out[3 * k + 1] = u; out[3 * k + 2] = pp;
  }
}

template <class T>
static Coords<T> make_coords(const Par<T>& P, const double* period, const T* x, const T* y) {
  Coords<T> C;
  C.ni = P.ni; C.nj = P.nj;
  for (int f = 0; f < 4; ++f) C.bc[f] = P.bc[f];
  C.per[0][0] = T(period[0]); C.per[0][1] = T(period[1]);
  C.per[1][0] = T(period[2]); C.per[1][1] = T(period[3]);
  C.x = x; C.y = y;
  return C;
}

static int check(const int* ip, int ni, int nj) {
  if (ni < 1 || nj < 1) return 1;
  for (int f = 0; f < 4; ++f)
    if (ip[4 + f] < 0 || ip[4 + f] > BC_FARFIELD) return 5;   // links need the multi-block entry
  if (ip[0] < 0 || ip[0] > 5) return 2;
  // the four-midpoint scheme reaches six nodes beyond a face (its midpoint fluxes from j - 5/2
  // to j + 5/2): periodic directions only, whose ghost metrics wrap
  if (ip[0] == S74 && (ip[4] != BC_PERIODIC || ip[6] != BC_PERIODIC)) return 6;
  if (ip[8] < 0 || ip[8] > 1 || ip[9] < 0 || ip[9] > 2) return 7;
  if ((ip[4] == BC_PERIODIC) != (ip[5] == BC_PERIODIC)) return 3;
  if ((ip[6] == BC_PERIODIC) != (ip[7] == BC_PERIODIC)) return 3;
  if (ip[4] != BC_PERIODIC && ni < 9) return 4;
  if (ip[6] != BC_PERIODIC && nj < 9) return 4;
  return 0;
}

template <class T>
static std::vector<T> conv(const double* a, size_t n) {
  std::vector<T> r(n);
  for (size_t k = 0; k < n; ++k) r[k] = T(a[k]);
  return r;
}

}  // namespace orc

// Free-stream residual computed in the wider type T (metrics and right-hand side both
// in T) for the uniform conservative state q0: returns max |dQ/dt| over all nodes.
namespace orc {
template <class T>
static double fsp_residual(const int* ip, const double* dp, int ni, int nj, const double* period,
                           const double* x, const double* y, const double* q0) {
  Par<T> P; unpack(ip, dp, ni, nj, P);
  const size_t N = (size_t)ni * nj;
  std::vector<T> X = conv<T>(x, N), Y = conv<T>(y, N);
  Coords<T> C = make_coords(P, period, X.data(), Y.data());
  std::vector<T> M((size_t)5 * (ni + 2 * G) * (nj + 2 * G)), Q(4 * N), R(4 * N);
  metrics(P, C, M.data());
  for (int v = 0; v < 4; ++v)
    for (size_t k = 0; k < N; ++k) Q[v * N + k] = T(q0[v]);
  rhs(P, M.data(), Q.data(), R.data());
  double worst = 0.0;
  for (size_t k = 0; k < 4 * N; ++k) worst = std::max(worst, std::fabs(val(R[k])));
  return worst;
}
}  // namespace orc

namespace orc {
// ----------------------------------------------------------------------------------
// Multi-block grids: blocks joined by Link faces (see Link).  Arrays of all blocks are
// concatenated in block order: coordinates ni*nj per block, metrics 5 (ni+8)(nj+8), state
// 4 ni nj.  The line maxima of the splitting are taken per block line.
// ----------------------------------------------------------------------------------
template <class T>
static int mb_setup(const int* ip, const double* dp, int nb, const int* dims, const int* bcs, const int* lk,
                    const double* loff, std::vector<Par<T>>& P, std::vector<Link>& L) {
  if (nb < 1 || ip[0] == S74) return 1;
  P.resize(nb);
  L.resize(4 * (size_t)nb);
  for (int b = 0; b < nb; ++b) {
    unpack(ip, dp, dims[2 * b], dims[2 * b + 1], P[b]);
    for (int f = 0; f < 4; ++f) {
      P[b].bc[f] = bcs[4 * b + f];
      Link& l = L[4 * b + f];
      l.nbr = lk[12 * b + 3 * f]; l.face = lk[12 * b + 3 * f + 1]; l.rev = lk[12 * b + 3 * f + 2];
      l.off[0] = loff ? loff[8 * b + 2 * f] : 0.0; l.off[1] = loff ? loff[8 * b + 2 * f + 1] : 0.0;
      if (P[b].bc[f] == BC_LINK && (l.nbr < 0 || l.nbr >= nb || l.face < 0 || l.face > 3)) return 6;
    }
    if (P[b].ni < 1 || P[b].nj < 1) return 1;
  }
  return 0;
}
}  // namespace orc

using namespace orc;

// the metric entry points: the defaults, then the caller's options (nullable); only the
// scheme's free parameter dp[19] matters for the metrics
static void opts(const double* in, double* dp) {
  for (int k = 3; k < 19; ++k) dp[k] = 0.0;
  dp[19] = 1.0;
  if (in) for (int k = 0; k < 20; ++k) dp[k] = in[k];
}

extern "C" {

// ip = {scheme, interp, ppm, linear_weights, bc[0..3], weights, midsplit}
// dp = {gamma, lf_alpha, eps, bc_state[4][4] (conservative, per face), scheme alpha}
// period = {dx_i, dy_i, dx_j, dy_j}

size_t orc_metrics_len(int ni, int nj) { return (size_t)5 * (ni + 2 * G) * (nj + 2 * G); }

int orc_metrics(const int* ip, const double* dpin, int ni, int nj, const double* period, const double* x,
                const double* y, double* M) {
  if (int e = check(ip, ni, nj)) return e;
  Par<double> P; double dp[20] = {1.4, 1.1, 1e-40}; opts(dpin, dp);
  unpack(ip, dp, ni, nj, P);
  Coords<double> C = make_coords(P, period, x, y);
  metrics(P, C, M);
  return 0;
}

// Tangent of the metrics along (dx, dy).
int orc_metrics_jvp(const int* ip, const double* dpin, int ni, int nj, const double* period, const double* x,
                    const double* y, const double* dx, const double* dy, double* M, double* dM) {
  if (int e = check(ip, ni, nj)) return e;
  Par<Dual> P; double dp[20] = {1.4, 1.1, 1e-40}; opts(dpin, dp);
  unpack(ip, dp, ni, nj, P);
  const size_t N = (size_t)ni * nj;
  std::vector<Dual> X(N), Y(N);
  for (size_t k = 0; k < N; ++k) { X[k] = Dual(x[k], dx[k]); Y[k] = Dual(y[k], dy[k]); }
  Coords<Dual> C = make_coords(P, period, X.data(), Y.data());
  std::vector<Dual> Md(orc_metrics_len(ni, nj));
  metrics(P, C, Md.data());
  for (size_t k = 0; k < Md.size(); ++k) { M[k] = Md[k].v; dM[k] = Md[k].d; }
  return 0;
}

int orc_lambda(const int* ip, const double* dp, int ni, int nj, const double* M, const double* Q,
               double* lam_xi, double* lam_eta) {
  if (int e = check(ip, ni, nj)) return e;
  Par<double> P; unpack(ip, dp, ni, nj, P);
  Field<double> F{P, M, Q};
  for (int j = 0; j < nj; ++j) lam_xi[j] = line_lambda(F, 0, j);
  for (int i = 0; i < ni; ++i) lam_eta[i] = line_lambda(F, 1, i);
  return 0;
}

int orc_rhs(const int* ip, const double* dp, int ni, int nj, const double* M, const double* Q,
            double* dQ) {
  if (int e = check(ip, ni, nj)) return e;
  Par<double> P; unpack(ip, dp, ni, nj, P);
  rhs(P, M, Q, dQ);
  return 0;
}

// Tangent of the right-hand side along (dM, dQ) (either may be null = zero).
int orc_rhs_jvp(const int* ip, const double* dp, int ni, int nj, const double* M, const double* dM,
                const double* Q, const double* dQ, double* R, double* dR) {
  if (int e = check(ip, ni, nj)) return e;
  Par<Dual> P; unpack(ip, dp, ni, nj, P);
  const size_t NM = orc_metrics_len(ni, nj), NQ = 4 * (size_t)ni * nj;
  std::vector<Dual> Md(NM), Qd(NQ), Rd(NQ);
  for (size_t k = 0; k < NM; ++k) Md[k] = Dual(M[k], dM ? dM[k] : 0.0);
  for (size_t k = 0; k < NQ; ++k) Qd[k] = Dual(Q[k], dQ ? dQ[k] : 0.0);
  rhs(P, Md.data(), Qd.data(), Rd.data());
  for (size_t k = 0; k < NQ; ++k) { R[k] = Rd[k].v; dR[k] = Rd[k].d; }
  return 0;
}

int orc_rk3(const int* ip, const double* dp, int ni, int nj, const double* M, double* Q, double dt,
            int nsteps) {
  if (int e = check(ip, ni, nj)) return e;
  Par<double> P; unpack(ip, dp, ni, nj, P);
  for (int s = 0; s < nsteps; ++s) rk3(P, M, Q, dt);
  return 0;
}

// Tangent of nsteps RK3 steps along (dM, dQ); Q and dQ are advanced in place.
int orc_rk3_jvp(const int* ip, const double* dp, int ni, int nj, const double* M, const double* dM,
                double* Q, double* dQ, double dt, int nsteps) {
  if (int e = check(ip, ni, nj)) return e;
  Par<Dual> P; unpack(ip, dp, ni, nj, P);
  const size_t NM = orc_metrics_len(ni, nj), NQ = 4 * (size_t)ni * nj;
  std::vector<Dual> Md(NM), Qd(NQ);
  for (size_t k = 0; k < NM; ++k) Md[k] = Dual(M[k], dM ? dM[k] : 0.0);
  for (size_t k = 0; k < NQ; ++k) Qd[k] = Dual(Q[k], dQ[k]);
  for (int s = 0; s < nsteps; ++s) rk3(P, Md.data(), Qd.data(), Dual(dt));
  for (size_t k = 0; k < NQ; ++k) { Q[k] = Qd[k].v; dQ[k] = Qd[k].d; }
  return 0;
}

double orc_cfl_dt(const int* ip, const double* dp, int ni, int nj, const double* M, const double* Q,
                  double cfl) {
  if (check(ip, ni, nj)) return -1.0;
  Par<double> P; unpack(ip, dp, ni, nj, P);
  return cfl_dt(P, M, Q, cfl);
}

// Floating-point operations of one right-hand side (each + - * / sqrt counts one).
long long orc_count_flops(const int* ip, const double* dp, int ni, int nj, const double* M,
                          const double* Q) {
  if (check(ip, ni, nj)) return -1;
  Par<Counted> P; unpack(ip, dp, ni, nj, P);
  const size_t NM = orc_metrics_len(ni, nj), NQ = 4 * (size_t)ni * nj;
  std::vector<Counted> Mc = conv<Counted>(M, NM), Qc = conv<Counted>(Q, NQ), Rc(NQ);
  g_flops = 0;
  rhs(P, Mc.data(), Qc.data(), Rc.data());
  return g_flops;
}

// Floating-point operations of one interface's characteristic direction (Section 3.4), and of
// one midpoint interpolation I of a nodal quantity (Section 2.4)
// for a scheme and interpolation option: the work per component that a solver storing the
// midpoint metrics once per grid no longer repeats in each right-hand side.
long long orc_count_char_dir() {
  g_flops = 0;
  Counted nx, ny;
  char_dir<Counted>(Counted(1.0), Counted(0.5), Counted(1.25), Counted(0.25), nx, ny);
  return g_flops;
}

long long orc_count_mid_interp(int scheme, int interp) {
  if (scheme < 0 || scheme > 5 || interp < 0 || interp > 1) return -1;
  g_flops = 0;
  const Counted r = interp_mid<Counted>(scheme, interp, [](int l) { return Counted(1.0 + 0.25 * l); });
  (void)r;
  return g_flops;
}

// Floating-point operations by part of one right-hand side:
// out = {line maxima xi, xi sweep without its line maxima, line maxima eta,
//        eta sweep without its line maxima, final division by J^-1}.
int orc_count_flops_parts(const int* ip, const double* dp, int ni, int nj, const double* M,
                          const double* Q, long long* out) {
  if (int e = check(ip, ni, nj)) return e;
  Par<Counted> P; unpack(ip, dp, ni, nj, P);
  const size_t NM = orc_metrics_len(ni, nj), NQ = 4 * (size_t)ni * nj;
  std::vector<Counted> Mc = conv<Counted>(M, NM), Qc = conv<Counted>(Q, NQ), R(NQ, Counted(0.0));
  Field<Counted> F{P, Mc.data(), Qc.data()};
  for (int dir = 0; dir < 2; ++dir) {
    const int nl = dir == 0 ? nj : ni;
    g_flops = 0;
    for (int L = 0; L < nl; ++L) line_lambda(F, dir, L);
    const long long lam = g_flops;
    g_flops = 0;
    sweep(F, dir, R);
    out[2 * dir] = lam;
    out[2 * dir + 1] = g_flops - lam;
  }
  std::vector<Counted> dQ(NQ);
  g_flops = 0;
  rhs(P, Mc.data(), Qc.data(), dQ.data());
  long long total = g_flops;
  out[4] = total - out[0] - out[1] - out[2] - out[3];
  return 0;
}

double orc_fsp_residual(const int* ip, const double* dp, int ni, int nj, const double* period,
                        const double* x, const double* y, const double* q0, int wide) {
  if (check(ip, ni, nj)) return -1.0;
  return wide ? fsp_residual<long double>(ip, dp, ni, nj, period, x, y, q0)
              : fsp_residual<double>(ip, dp, ni, nj, period, x, y, q0);
}

int orc_long_double_digits(void) { return (int)__LDBL_MANT_DIG__; }

double orc_weno(int r, int ppm, int linw, double eps, const double* u7) {
  WenoOpt o{ppm, linw};
  return weno_mid<double>(r, u7, o, eps);
}

double orc_ppm(int order, double w, double C) { return ppm_map<double>(order, w, C); }

void orc_smoothness(const double* u5, double* is3) {
  is3[0] = is0<double>(u5[0], u5[1], u5[2]);
  is3[1] = is1<double>(u5[1], u5[2], u5[3]);
  is3[2] = is2<double>(u5[2], u5[3], u5[4]);
}

void orc_eig(double gamma, const double* q, double nx, double ny, double* L, double* R) {
  double Lm[4][4], Rm[4][4];
  eigvec<double>(q, nx, ny, gamma, Lm, Rm);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) { L[4 * a + b] = Lm[a][b]; R[4 * a + b] = Rm[a][b]; }
}

void orc_scheme_table(int scheme, double alpha,
                      double* out /* r, hmid[2], hnode[7], cnode[4], cmid[2], hmidx[2], cmid3 */) {
  const SchemeTab S = scheme_tab(scheme, alpha);
  out[0] = S.r;
  for (int k = 0; k < 2; ++k) out[1 + k] = (double)S.hmid[k];
  for (int k = 0; k < 7; ++k) out[3 + k] = (double)S.hnode[k];
  for (int k = 0; k < 4; ++k) out[10 + k] = (double)S.cnode[k];
  for (int k = 0; k < 2; ++k) out[14 + k] = (double)S.cmid[k];
  for (int k = 0; k < 2; ++k) out[16 + k] = (double)S.hmidx[k];
  out[18] = (double)S.cmid3;
}

int orc_advect1d(int scheme, int N, double tfinal, double* out) {
  if (scheme < 0 || scheme > 5 || N < 7) return 1;
  advect1d(scheme, N, tfinal, out);
  return 0;
}

// The same with dt = 2 / ceil(2 / dx^dt_exp) (dt_exp = 7/4 keeps the RK4 error below the
// seventh-order spatial error).
int orc_advect1d_dt(int scheme, int N, double tfinal, double dt_exp, double* out) {
  if (scheme < 0 || scheme > 5 || N < 7 || !(dt_exp > 0.0)) return 1;
  advect1d(scheme, N, tfinal, out, dt_exp);
  return 0;
}

// The same with the weight option (weights = 1: WENO-Z).
int orc_advect1d_opts(int scheme, int N, double tfinal, double dt_exp, int weights, double* out) {
  if (scheme < 0 || scheme > 5 || N < 7 || !(dt_exp > 0.0) || weights < 0 || weights > 1) return 1;
  advect1d(scheme, N, tfinal, out, dt_exp, weights);
  return 0;
}

// WENO-Z interpolation to x_{j+1/2} from u7[m + 3] = u_{j+m} (r = 2, 3, 4).
double orc_weno_z(int r, double eps, const double* u7) {
  WenoOpt o{0, 0, 1};
  return weno_mid<double>(r, u7, o, eps);
}

// Midpoint flux splitting mode (1 Steger-Warming, 2 Van Leer) of state q along (mx, my):
// fp = F+, fm = F-, e = E^.
int orc_split_flux(int mode, const double* q, double mx, double my, double gamma, double* fp, double* fm,
                   double* e) {
  if (mode == 1) { split_sw(q, mx, my, gamma, 1, fp); split_sw(q, mx, my, gamma, -1, fm); }
  else if (mode == 2) { split_vl(q, mx, my, gamma, 1, fp); split_vl(q, mx, my, gamma, -1, fm); }
  else return 1;
  flux(q, mx, my, gamma, e);
  return 0;
}

void orc_smoothness4(const double* u7, double* is4) {
  for (int k = 0; k < 4; ++k) is4[k] = is_r4<double>(k, u7 + k);
}

int orc_riemann_exact(double gamma, const double* WL, const double* WR, double x0, double t, int n,
                      const double* x, double* out) {
  riemann_exact(gamma, WL, WR, x0, t, n, x, out);
  return 0;
}


// ---- reverse mode (adjoints) ----
// Each entry point tapes one evaluation with the Rev scalar (every input value a tape
// leaf), seeds the outputs' adjoints and walks the tape backwards.  The outputs are
// accumulated (+=) into the caller's arrays, which the caller zeroes.

// Q_bar += (d dQ/dt / dQ)^T g and M_bar += (d dQ/dt / dM)^T g over the haloed metrics.
int orc_rhs_vjp(const int* ip, const double* dp, int ni, int nj, const double* M, const double* Q,
                const double* g, double* Qbar, double* Mbar) {
  if (int e = check(ip, ni, nj)) return e;
  Par<Rev> P; unpack(ip, dp, ni, nj, P);
  const size_t NM = orc_metrics_len(ni, nj), NQ = 4 * (size_t)ni * nj;
  g_tape.clear();
  std::vector<Rev> Mr(NM), Qr(NQ), Rr(NQ);
  for (size_t k = 0; k < NM; ++k) Mr[k] = rev_leaf(M[k]);
  for (size_t k = 0; k < NQ; ++k) Qr[k] = rev_leaf(Q[k]);
  rhs(P, Mr.data(), Qr.data(), Rr.data());
  std::vector<double> adj(g_tape.size(), 0.0);
  for (size_t k = 0; k < NQ; ++k)
    if (Rr[k].i >= 0) adj[Rr[k].i] += g[k];
  rev_sweep(adj);
  for (size_t k = 0; k < NM; ++k) if (Mbar) Mbar[k] += adj[Mr[k].i];
  for (size_t k = 0; k < NQ; ++k) Qbar[k] += adj[Qr[k].i];
  g_tape.clear();
  g_tape.shrink_to_fit();
  return 0;
}

// Reverse of one RK3 step from Q_n: on entry Qbar = dJ/dQ^{n+1}, on return dJ/dQ^n;
// M_bar (nullable) += the step's metric adjoint.  dt is a constant.
int orc_rk3_vjp(const int* ip, const double* dp, int ni, int nj, const double* M, const double* Qn, double dt,
                double* Qbar, double* Mbar) {
  if (int e = check(ip, ni, nj)) return e;
  Par<Rev> P; unpack(ip, dp, ni, nj, P);
  const size_t NM = orc_metrics_len(ni, nj), NQ = 4 * (size_t)ni * nj;
  g_tape.clear();
  std::vector<Rev> Mr(NM), Q0(NQ), Q(NQ);
  for (size_t k = 0; k < NM; ++k) Mr[k] = rev_leaf(M[k]);
  for (size_t k = 0; k < NQ; ++k) { Q0[k] = rev_leaf(Qn[k]); Q[k] = Q0[k]; }
  rk3(P, Mr.data(), Q.data(), Rev(dt));
  std::vector<double> adj(g_tape.size(), 0.0);
  for (size_t k = 0; k < NQ; ++k)
    if (Q[k].i >= 0) adj[Q[k].i] += Qbar[k];
  rev_sweep(adj);
  for (size_t k = 0; k < NM; ++k) if (Mbar) Mbar[k] += adj[Mr[k].i];
  for (size_t k = 0; k < NQ; ++k) Qbar[k] = adj[Q0[k].i];
  g_tape.clear();
  g_tape.shrink_to_fit();
  return 0;
}

// x_bar += (d M / d x)^T M_bar, y_bar likewise (periodic offsets are constants).
int orc_metrics_vjp(const int* ip, const double* dpin, int ni, int nj, const double* period, const double* x, const double* y,
                    const double* Mbar, double* xbar, double* ybar) {
  if (int e = check(ip, ni, nj)) return e;
  Par<Rev> P; double dp[20] = {1.4, 1.1, 1e-40}; opts(dpin, dp);
  unpack(ip, dp, ni, nj, P);
  const size_t N = (size_t)ni * nj, NM = orc_metrics_len(ni, nj);
  g_tape.clear();
  std::vector<Rev> X(N), Y(N), Mr(NM);
  for (size_t k = 0; k < N; ++k) { X[k] = rev_leaf(x[k]); Y[k] = rev_leaf(y[k]); }
  Coords<Rev> C = make_coords(P, period, X.data(), Y.data());
  metrics(P, C, Mr.data());
  std::vector<double> adj(g_tape.size(), 0.0);
  for (size_t k = 0; k < NM; ++k)
    if (Mr[k].i >= 0) adj[Mr[k].i] += Mbar[k];
  rev_sweep(adj);
  for (size_t k = 0; k < N; ++k) { xbar[k] += adj[X[k].i]; ybar[k] += adj[Y[k].i]; }
  g_tape.clear();
  g_tape.shrink_to_fit();
  return 0;
}

// Operation count of one right-hand-side adjoint, dense in the seed: out = {the forward
// right-hand side (as orc_count_flops), the partial derivatives the forward pass forms for
// its divisions and square roots, the reverse sweep taken densely (whatever the seed: one
// operation per operand edge of a sum or difference, two for any other), tape records}.
int orc_count_vjp_flops(const int* ip, const double* dp, int ni, int nj, const double* M, const double* Q,
                        long long* out) {
  if (int e = check(ip, ni, nj)) return e;
  out[0] = orc_count_flops(ip, dp, ni, nj, M, Q);
  Par<Rev> P; unpack(ip, dp, ni, nj, P);
  const size_t NM = orc_metrics_len(ni, nj), NQ = 4 * (size_t)ni * nj;
  g_tape.clear();
  g_rev_extra = 0;
  g_rev_edges = 0;
  std::vector<Rev> Mr(NM), Qr(NQ), Rr(NQ);
  for (size_t k = 0; k < NM; ++k) Mr[k] = rev_leaf(M[k]);
  for (size_t k = 0; k < NQ; ++k) Qr[k] = rev_leaf(Q[k]);
  rhs(P, Mr.data(), Qr.data(), Rr.data());
  out[1] = g_rev_extra;
  out[2] = g_rev_edges;
  out[3] = (long long)g_tape.size();
  g_tape.clear();
  g_tape.shrink_to_fit();
  return 0;
}

// ---- multi-block entry points ----
// dims: ni, nj per block; bcs: 4 codes per block (BC_LINK = 5 joins a face); lk: per
// block and face (nbr, face, rev); loff: per block and face the ghost coordinate offset
// (nullable); periods: per block the periodic vectors (dx_i, dy_i, dx_j, dy_j).
int orc_mb_metrics(const int* ip, const double* dpin, int nb, const int* dims, const int* bcs, const int* lk,
                   const double* loff, const double* periods, const double* x, const double* y,
                   double* M) {
  std::vector<Par<double>> P;
  std::vector<Link> L;
  double dp[20] = {1.4, 1.1, 1e-40}; opts(dpin, dp);
  if (int e = mb_setup(ip, dp, nb, dims, bcs, lk, loff, P, L)) return e;
  std::vector<Coords<double>> C(nb);
  size_t xo = 0;
  for (int b = 0; b < nb; ++b) {
    C[b] = make_coords(P[b], periods + 4 * b, x + xo, y + xo);
    C[b].links = &L[4 * (size_t)b];
    C[b].blocks = C.data();
    xo += (size_t)P[b].ni * P[b].nj;
  }
  size_t mo = 0;
  for (int b = 0; b < nb; ++b) {
    metrics(P[b], C[b], M + mo);
    mo += orc_metrics_len(P[b].ni, P[b].nj);
  }
  return 0;
}

static void mb_fields(std::vector<Par<double>>& P, std::vector<Link>& L, const double* M, const double* Q,
                      std::vector<Field<double>>& F) {
  const int nb = (int)P.size();
  F.clear();
  F.reserve(nb);
  size_t mo = 0, qo = 0;
  for (int b = 0; b < nb; ++b) {
    F.push_back(Field<double>{P[b], M + mo, Q + qo});
    mo += orc_metrics_len(P[b].ni, P[b].nj);
    qo += 4 * (size_t)P[b].ni * P[b].nj;
  }
  for (int b = 0; b < nb; ++b) { F[b].links = &L[4 * (size_t)b]; F[b].blocks = F.data(); }
}

int orc_mb_rhs(const int* ip, const double* dp, int nb, const int* dims, const int* bcs, const int* lk,
               const double* M, const double* Q, double* dQ) {
  std::vector<Par<double>> P;
  std::vector<Link> L;
  if (int e = mb_setup(ip, dp, nb, dims, bcs, lk, nullptr, P, L)) return e;
  std::vector<Field<double>> F;
  mb_fields(P, L, M, Q, F);
  size_t qo = 0;
  for (int b = 0; b < nb; ++b) {
    rhs_field(F[b], dQ + qo);
    qo += 4 * (size_t)P[b].ni * P[b].nj;
  }
  return 0;
}

// nsteps TVD-RK3 steps of every block in lockstep (all blocks finish a stage before the
// next stage reads their ghosts); Q is updated in place.
int orc_mb_rk3(const int* ip, const double* dp, int nb, const int* dims, const int* bcs, const int* lk,
               const double* M, double* Q, double dt, int nsteps) {
  std::vector<Par<double>> P;
  std::vector<Link> L;
  if (int e = mb_setup(ip, dp, nb, dims, bcs, lk, nullptr, P, L)) return e;
  size_t NQ = 0;
  for (int b = 0; b < nb; ++b) NQ += 4 * (size_t)P[b].ni * P[b].nj;
  std::vector<double> Q1(NQ), Q2(NQ), R(NQ);
  std::vector<Field<double>> F;
  auto all_rhs = [&](const double* Qs) {
    mb_fields(P, L, M, Qs, F);
    size_t qo = 0;
    for (int b = 0; b < nb; ++b) {
      rhs_field(F[b], R.data() + qo);
      qo += 4 * (size_t)P[b].ni * P[b].nj;
    }
  };
  for (int st = 0; st < nsteps; ++st) {
    all_rhs(Q);
    for (size_t k = 0; k < NQ; ++k) Q1[k] = Q[k] + dt * R[k];
    all_rhs(Q1.data());
    for (size_t k = 0; k < NQ; ++k) Q2[k] = 0.75 * Q[k] + 0.25 * (Q1[k] + dt * R[k]);
    all_rhs(Q2.data());
    for (size_t k = 0; k < NQ; ++k) Q[k] = (1.0 / 3) * Q[k] + (2.0 / 3) * (Q2[k] + dt * R[k]);
  }
  return 0;
}
}  // extern "C"

// ==================================================================================
// Three dimensions (Sections 2.1-2.2): Q = (rho, rho u, rho v, rho w, e), the symmetric
// conservative metrics of Eq. (2.4), the Jacobian of Eq. (2.5), and one sweep per grid
// direction xi, eta, zeta, each built exactly like the two-dimensional sweep.
//
// Conventions: nodes (i, j, k), i fastest; state 5 planes [5][nk][nj][ni]; metrics 10
// planes on the grid extended by G = 4 ghost layers on every side: plane 3 d + c holds
// the component c (x, y, z) of the metric of direction d (xi, eta, zeta), i.e. xi_x^,
// xi_y^, xi_z^, eta_x^, ..., zeta_z^, and plane 9 holds J^-1; plane p, node (i, j, k) at
// M[p*P + ((k+4)*(nj+8) + (j+4))*(ni+8) + (i+4)], P = (ni+8)(nj+8)(nk+8).  Faces 0..5 =
// i-min, i-max, j-min, j-max, k-min, k-max; codes PERIODIC = 0, TRANSMISSIVE = 1.
// ==================================================================================
namespace orc {

template <class T>
struct Par3 {
  int scheme = S51, interp = 0, ppm = 1, linw = 0;
  int bc[6] = {0, 0, 0, 0, 0, 0};
  T gamma = T(1.4), alpha = cst<T>(1.1L), eps = cst<T>(1e-40L);
  SchemeTab tab;
  int n[3] = {0, 0, 0};     // ni, nj, nk
  T per[3][3];              // per[a] = (dx, dy, dz) added per wrap in direction a
};

// ip = {scheme, interp, ppm, linear_weights, bc[6]}; dp = {gamma, lf_alpha, eps, period[3][3]}
template <class T>
static void unpack3(const int* ip, const double* dp, int ni, int nj, int nk, Par3<T>& P) {
  P.scheme = ip[0]; P.interp = ip[1]; P.ppm = ip[2]; P.linw = ip[3];
  for (int f = 0; f < 6; ++f) P.bc[f] = ip[4 + f];
  P.gamma = T(dp[0]); P.alpha = T(dp[1]); P.eps = T(dp[2]);
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) P.per[a][c] = T(dp[3 + 3 * a + c]);
  P.tab = TAB[P.scheme];
  P.n[0] = ni; P.n[1] = nj; P.n[2] = nk;
}

// A grid extended by e layers: index of node (i, j, k).
struct Ext3 {
  int e, n[3];
  size_t size() const { return (size_t)(n[0] + 2 * e) * (n[1] + 2 * e) * (n[2] + 2 * e); }
  size_t at(int i, int j, int k) const {
    return ((size_t)(k + e) * (n[1] + 2 * e) + (j + e)) * (n[0] + 2 * e) + (i + e);
  }
};

// Coordinate c of node (i, j, k) of the extended grid.  Reading (as in two dimensions): a
// periodic direction wraps and adds its period vector per wrap; any other direction extends
// the grid by odd reflection about its boundary node, x_{-m} = 2 x_0 - x_m.
template <class T>
static T coord3(const Par3<T>& P, const T* const X[3], int c, int i, int j, int k) {
  int id[3] = {i, j, k};
  for (int a = 0; a < 3; ++a) {
    const int n = P.n[a];
    if (id[a] >= 0 && id[a] < n) continue;
    if (P.bc[2 * a] == BC_PERIODIC) {
      const int q = floordiv(id[a], n);
      id[a] -= q * n;
      return coord3(P, X, c, id[0], id[1], id[2]) + T(double(q)) * P.per[a][c];
    }
    const int b = id[a] < 0 ? 0 : n - 1;
    int m[3] = {id[0], id[1], id[2]};
    m[a] = 2 * b - id[a];
    id[a] = b;
    return cst<T>(2) * coord3(P, X, c, id[0], id[1], id[2]) - coord3(P, X, c, m[0], m[1], m[2]);
  }
  return X[c][((size_t)k * P.n[1] + j) * P.n[0] + i];
}

// The scheme's central operator delta^{c,(1)} (Eq. 2.7, as central_D) of nodal values
// node(m), m = offset along the direction.
template <class T, class F>
static T central1(const Par3<T>& P, F node) {
  const SchemeTab& S = P.tab;
  auto mid = [&](int m) { return interp_mid<T>(P.scheme, P.interp, [&](int l) { return node(m + l); }); };
  T d = T(0);
  for (int m = 1; m <= 4; ++m)
    if (S.cnode[m - 1] != 0.0L) d = d + cst<T>(S.cnode[m - 1]) * (node(m) - node(-m));
  d = d + cst<T>(S.cmid[0]) * (mid(0) - mid(-1));
  if (S.cmid[1] != 0.0L) d = d + cst<T>(S.cmid[1]) * (mid(1) - mid(-2));
  return d;
}

// Metrics (Eq. 2.4) and Jacobian (Eq. 2.5) on the grid extended by G layers.  For direction
// d with the next two directions (a, b) = (d+1, d+2) mod 3, and component c with the next
// two coordinates (p, q) = (c+1, c+2) mod 3:
//   m_{d,c} = 1/2 [ (p_a q)_b - (p_b q)_a + (q_b p)_a - (q_a p)_b ],
// which for d = xi, c = x is Eq. (2.4) as printed; J^-1 = 1/3 sum_{d,c} m_{d,c} (c)_d.  Every
// derivative, inner and outer, is the scheme's central operator (Section 2.3).  Staged as
// coordinates on the grid extended by 12 layers, their derivatives on the grid extended by
// 8, then the metrics.
template <class T>
static void metrics3(const Par3<T>& P, const T* const X[3], T* M) {
  const Ext3 E12{12, {P.n[0], P.n[1], P.n[2]}}, E8{8, {P.n[0], P.n[1], P.n[2]}}, E4{G, {P.n[0], P.n[1], P.n[2]}};
  std::vector<T> C[3], D[3][3];   // C[c]: coordinates; D[a][c]: derivative of c along a
  for (int c = 0; c < 3; ++c) {
    C[c].resize(E12.size());
    for (int k = -12; k < P.n[2] + 12; ++k)
      for (int j = -12; j < P.n[1] + 12; ++j)
        for (int i = -12; i < P.n[0] + 12; ++i) C[c][E12.at(i, j, k)] = coord3(P, X, c, i, j, k);
  }
  auto step = [](int a, int m, int& i, int& j, int& k) { if (a == 0) i += m; else if (a == 1) j += m; else k += m; };
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) {
      D[a][c].resize(E8.size());
      for (int k = -8; k < P.n[2] + 8; ++k)
        for (int j = -8; j < P.n[1] + 8; ++j)
          for (int i = -8; i < P.n[0] + 8; ++i)
            D[a][c][E8.at(i, j, k)] = central1(P, [&](int m) {
              int ii = i, jj = j, kk = k;
              step(a, m, ii, jj, kk);
              return C[c][E12.at(ii, jj, kk)];
            });
    }
  const size_t plane = E4.size();
  for (int k = -G; k < P.n[2] + G; ++k)
    for (int j = -G; j < P.n[1] + G; ++j)
      for (int i = -G; i < P.n[0] + G; ++i) {
        // (f_s g)_t: the derivative along t of the product of the derivative of f along s and g
        auto dprod = [&](int t, int s, int f, int g) {
          return central1(P, [&](int m) {
            int ii = i, jj = j, kk = k;
            step(t, m, ii, jj, kk);
            return D[s][f][E8.at(ii, jj, kk)] * C[g][E12.at(ii, jj, kk)];
          });
        };
        T Jv = T(0);
        for (int d = 0; d < 3; ++d)
          for (int c = 0; c < 3; ++c) {
            const int a = (d + 1) % 3, b = (d + 2) % 3, p = (c + 1) % 3, q = (c + 2) % 3;
            const T m = cst<T>(0.5L) * (dprod(b, a, p, q) - dprod(a, b, p, q) + dprod(a, b, q, p) - dprod(b, a, q, p));
            M[(3 * d + c) * plane + E4.at(i, j, k)] = m;
            Jv = Jv + m * D[d][c][E8.at(i, j, k)];
          }
        M[9 * plane + E4.at(i, j, k)] = Jv / cst<T>(3);
      }
}

// Pressure, metric-weighted flux E^ = m_x E + m_y F + m_z G (Eq. 2.2) and |U^| + c |k^|.
template <class T>
static T pressure3(const T* q, T gamma) {
  T u = q[1] / q[0], v = q[2] / q[0], w = q[3] / q[0];
  return (gamma - cst<T>(1)) * (q[4] - cst<T>(0.5L) * q[0] * (u * u + v * v + w * w));
}
template <class T>
static void flux3(const T* q, const T* m, T gamma, T* f) {
  T rho = q[0], u = q[1] / rho, v = q[2] / rho, w = q[3] / rho;
  T p = (gamma - cst<T>(1)) * (q[4] - cst<T>(0.5L) * rho * (u * u + v * v + w * w));
  T U = m[0] * u + m[1] * v + m[2] * w;
  f[0] = rho * U;
  f[1] = rho * u * U + m[0] * p;
  f[2] = rho * v * U + m[1] * p;
  f[3] = rho * w * U + m[2] * p;
  f[4] = (q[4] + p) * U;
}
template <class T>
static T spectral3(const T* q, const T* m, T gamma) {
  T rho = q[0], u = q[1] / rho, v = q[2] / rho, w = q[3] / rho;
  T p = (gamma - cst<T>(1)) * (q[4] - cst<T>(0.5L) * rho * (u * u + v * v + w * w));
  T c = sqrt(gamma * p / rho);
  return fabs(m[0] * u + m[1] * v + m[2] * w) + c * sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
}

// Left/right eigenvectors of the Jacobian of the flux along the unit direction n at state q
// (Section 3.4 in three dimensions).  Reading: the Un eigenspace takes the entropy wave and two
// shear waves along unit tangents t1, t2: t1 = (a x n)/|a x n| with a the coordinate axis
// least aligned with n (smallest |n_i|, ties to the larger index), t2 = n x t1.  For n in
// the x-y plane this is a = z, t1 = (-ny, nx, 0), t2 = (0, 0, 1): the two-dimensional
// eigenvectors plus a shear wave in w.  R columns: (1, u - c n, H - c Un), (1, u, |u|^2/2),
// (0, t1, u.t1), (0, t2, u.t2), (1, u + c n, H + c Un); L its inverse, with b1 = (gamma - 1)
// / c^2 and b2 = b1 |u|^2 / 2: rows 1/2 (b2 + Un/c, -b1 u - n/c, b1), (1 - b2, b1 u, -b1),
// (-u.t1, t1, 0), (-u.t2, t2, 0), 1/2 (b2 - Un/c, -b1 u + n/c, b1).
template <class T>
static void tangents3(const T* n, T* t1, T* t2) {
  int a = 2;
  for (int i = 1; i >= 0; --i)
    if (fabs(n[i]) < fabs(n[a])) a = i;
  // a x n with a the unit axis
  T x[3];
  if (a == 0) { x[0] = T(0); x[1] = -n[2]; x[2] = n[1]; }
  else if (a == 1) { x[0] = n[2]; x[1] = T(0); x[2] = -n[0]; }
  else { x[0] = -n[1]; x[1] = n[0]; x[2] = T(0); }
  T s = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  for (int i = 0; i < 3; ++i) t1[i] = x[i] / s;
  t2[0] = n[1] * t1[2] - n[2] * t1[1];
  t2[1] = n[2] * t1[0] - n[0] * t1[2];
  t2[2] = n[0] * t1[1] - n[1] * t1[0];
}
template <class T>
static void eigvec3(const T* q, const T* n, T gamma, T L[5][5], T R[5][5]) {
  T rho = q[0], u[3] = {q[1] / rho, q[2] / rho, q[3] / rho};
  T q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  T p = (gamma - cst<T>(1)) * (q[4] - cst<T>(0.5L) * rho * q2);
  T c = sqrt(gamma * p / rho);
  T H = (q[4] + p) / rho;
  T t1[3], t2[3];
  tangents3(n, t1, t2);
  T Un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  T U1 = u[0] * t1[0] + u[1] * t1[1] + u[2] * t1[2];
  T U2 = u[0] * t2[0] + u[1] * t2[1] + u[2] * t2[2];
  T b1 = (gamma - cst<T>(1)) / (c * c), b2 = cst<T>(0.5L) * b1 * q2;
  const T h = cst<T>(0.5L);
  R[0][0] = T(1); R[0][1] = T(1); R[0][2] = T(0); R[0][3] = T(0); R[0][4] = T(1);
  for (int i = 0; i < 3; ++i) {
    R[1 + i][0] = u[i] - c * n[i];
    R[1 + i][1] = u[i];
    R[1 + i][2] = t1[i];
    R[1 + i][3] = t2[i];
    R[1 + i][4] = u[i] + c * n[i];
  }
  R[4][0] = H - c * Un; R[4][1] = h * q2; R[4][2] = U1; R[4][3] = U2; R[4][4] = H + c * Un;
  L[0][0] = h * (b2 + Un / c); L[4][0] = h * (b2 - Un / c);
  L[1][0] = T(1) - b2; L[2][0] = -U1; L[3][0] = -U2;
  for (int i = 0; i < 3; ++i) {
    L[0][1 + i] = h * (-b1 * u[i] - n[i] / c);
    L[1][1 + i] = b1 * u[i];
    L[2][1 + i] = t1[i];
    L[3][1 + i] = t2[i];
    L[4][1 + i] = h * (-b1 * u[i] + n[i] / c);
  }
  L[0][4] = h * b1; L[1][4] = -b1; L[2][4] = T(0); L[3][4] = T(0); L[4][4] = h * b1;
}

}  // namespace orc

namespace orc {

template <class T>
struct Field3 {
  const Par3<T>& P;
  const T* M;   // haloed metrics, 10 planes
  const T* Q;   // [5][nk][nj][ni]
  Ext3 E4() const { return Ext3{G, {P.n[0], P.n[1], P.n[2]}}; }
  T met(int p, int i, int j, int k) const { return M[(size_t)p * E4().size() + E4().at(i, j, k)]; }
  T q(int v, int i, int j, int k) const {
    return Q[(size_t)v * P.n[0] * P.n[1] * P.n[2] + ((size_t)k * P.n[1] + j) * P.n[0] + i];
  }
  // node (i, j, k) of position s on line (l1, l2) of direction d (the other two indices in order)
  void node(int d, int l1, int l2, int s, int& i, int& j, int& k) const {
    if (d == 0) { i = s; j = l1; k = l2; }
    else if (d == 1) { i = l1; j = s; k = l2; }
    else { i = l1; j = l2; k = s; }
  }
  // State at position s with ghosts by the face rule: periodic wraps, transmissive copies the
  // boundary node (the reading of two dimensions).
  void state(int d, int l1, int l2, int s, T* out) const {
    const int n = P.n[d];
    int ss = s;
    if (s < 0 || s >= n) {
      const int face = 2 * d + (s < 0 ? 0 : 1);
      ss = P.bc[face] == BC_PERIODIC ? s - floordiv(s, n) * n : (s < 0 ? 0 : n - 1);
    }
    int i, j, k;
    node(d, l1, l2, ss, i, j, k);
    for (int v = 0; v < 5; ++v) out[v] = q(v, i, j, k);
  }
  void nodemet(int d, int l1, int l2, int s, T* m) const {
    int i, j, k;
    node(d, l1, l2, s, i, j, k);
    for (int c = 0; c < 3; ++c) m[c] = met(3 * d + c, i, j, k);
  }
};

// A^ for line (l1, l2) of direction d: alpha x max over the line's nodes of |U^| + c|k^|.
template <class T>
static T line_lambda3(const Field3<T>& F, int d, int l1, int l2) {
  T best = T(0);
  for (int s = 0; s < F.P.n[d]; ++s) {
    T q[5], m[3];
    F.state(d, l1, l2, s, q);
    F.nodemet(d, l1, l2, s, m);
    T sp = spectral3(q, m, F.P.gamma);
    if (s == 0 || best < sp) best = sp;
  }
  return best * F.P.alpha;
}

// One direction: adds H_{s+1/2} - H_{s-1/2} to R for every node of every line (the
// two-dimensional sweep with five variables and three metric components).
template <class T>
static void sweep3(const Field3<T>& F, int d, std::vector<T>& R) {
  const Par3<T>& P = F.P;
  const SchemeTab& S = P.tab;
  const int n = P.n[d];
  const int n1 = P.n[d == 0 ? 1 : 0], n2 = P.n[d == 2 ? 1 : 2];
  const int NB = n + 8, NI = n + 3;
  const WenoOpt wo{P.ppm, P.linw, 0};
  std::vector<T> q(5 * NB), ms(3 * NB), fp(5 * NB), fm(5 * NB), fpm(5 * NI), fmm(5 * NI), Hh(5 * NI);
  const size_t N = (size_t)P.n[0] * P.n[1] * P.n[2];
  for (int l2 = 0; l2 < n2; ++l2)
    for (int l1 = 0; l1 < n1; ++l1) {
      const T A = line_lambda3(F, d, l1, l2);
      for (int s = -4; s < n + 4; ++s) {
        T qs[5], f[5];
        F.state(d, l1, l2, s, qs);
        F.nodemet(d, l1, l2, s, &ms[3 * (s + 4)]);
        flux3(qs, &ms[3 * (s + 4)], P.gamma, f);
        for (int v = 0; v < 5; ++v) {
          q[5 * (s + 4) + v] = qs[v];
          fp[5 * (s + 4) + v] = cst<T>(0.5L) * (f[v] + A * qs[v]);
          fm[5 * (s + 4) + v] = cst<T>(0.5L) * (f[v] - A * qs[v]);
        }
      }
      const int nmp = S.hmid[1] != 0.0L ? 2 : 1;
      for (int p = -nmp; p <= n - 2 + nmp; ++p) {
        const int c0 = p + 4;
        T mb[3], nn[3], mm[3];
        for (int c = 0; c < 3; ++c) mb[c] = cst<T>(0.5L) * (ms[3 * c0 + c] + ms[3 * (c0 + 1) + c]);
        T mbn = sqrt(mb[0] * mb[0] + mb[1] * mb[1] + mb[2] * mb[2]);
        for (int c = 0; c < 3; ++c) nn[c] = mb[c] / mbn;
        T Qs[2][5];
        for (int side = 0; side < 2; ++side) {
          const int ce = c0 + side;
          T Lm[5][5], Rm[5][5];
          eigvec3(&q[5 * ce], nn, P.gamma, Lm, Rm);
          T Wmid[5];
          const int half = S.r == 4 ? 3 : 2;
          for (int kc = 0; kc < 5; ++kc) {
            T u[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
            for (int m = -half; m <= half; ++m) {
              const int nd = side == 0 ? c0 + m : c0 + 1 - m;
              T w = T(0);
              for (int v = 0; v < 5; ++v) w = w + Lm[kc][v] * q[5 * nd + v];
              u[m + 3] = w;
            }
            Wmid[kc] = weno_mid(S.r, u, wo, P.eps);
          }
          for (int v = 0; v < 5; ++v) {
            T acc = T(0);
            for (int kc = 0; kc < 5; ++kc) acc = acc + Rm[v][kc] * Wmid[kc];
            Qs[side][v] = acc;
          }
        }
        for (int c = 0; c < 3; ++c)
          mm[c] = interp_mid<T>(P.scheme, P.interp, [&](int l) { return ms[3 * (c0 + l) + c]; });
        T fpl[5], fmi[5];
        flux3(Qs[0], mm, P.gamma, fpl);
        flux3(Qs[1], mm, P.gamma, fmi);
        for (int v = 0; v < 5; ++v) {
          fpm[5 * (p + 2) + v] = cst<T>(0.5L) * (fpl[v] + A * Qs[0][v]);
          fmm[5 * (p + 2) + v] = cst<T>(0.5L) * (fmi[v] - A * Qs[1][v]);
        }
      }
      for (int p = -1; p <= n - 1; ++p)
        for (int v = 0; v < 5; ++v) {
          T hp = T(0), hm = T(0);
          for (int m = 0; m >= -1; --m) {
            if (S.hmid[-m] == 0.0L) continue;
            hp = hp + cst<T>(S.hmid[-m]) * fpm[5 * (p + m + 2) + v];
            hm = hm + cst<T>(S.hmid[-m]) * fmm[5 * (p - m + 2) + v];
          }
          for (int k = -3; k <= 3; ++k) {
            if (S.hnode[k + 3] == 0.0L) continue;
            hp = hp + cst<T>(S.hnode[k + 3]) * fp[5 * (p + k + 4) + v];
            hm = hm + cst<T>(S.hnode[k + 3]) * fm[5 * (p + 1 - k + 4) + v];
          }
          Hh[5 * (p + 2) + v] = hp + hm;
        }
      for (int s = 0; s < n; ++s) {
        int i, j, k;
        F.node(d, l1, l2, s, i, j, k);
        for (int v = 0; v < 5; ++v) {
          size_t o = (size_t)v * N + ((size_t)k * P.n[1] + j) * P.n[0] + i;
          R[o] = R[o] + (Hh[5 * (s + 2) + v] - Hh[5 * (s + 1) + v]);
        }
      }
    }
}

// dQ/dt = -(dE^/dxi + dF^/deta + dG^/dzeta) / J^-1 (Eq. 2.2)
template <class T>
static void rhs3(const Par3<T>& P, const T* M, const T* Q, T* dQ) {
  Field3<T> F{P, M, Q};
  const size_t N = (size_t)P.n[0] * P.n[1] * P.n[2];
  std::vector<T> R(5 * N, T(0));
  for (int d = 0; d < 3; ++d) sweep3(F, d, R);
  for (int k = 0; k < P.n[2]; ++k)
    for (int j = 0; j < P.n[1]; ++j)
      for (int i = 0; i < P.n[0]; ++i) {
        T Jinv = F.met(9, i, j, k);
        for (int v = 0; v < 5; ++v) {
          size_t o = (size_t)v * N + ((size_t)k * P.n[1] + j) * P.n[0] + i;
          dQ[o] = -(R[o] / Jinv);
        }
      }
}

template <class T>
static void rk3_3(const Par3<T>& P, const T* M, T* Q, T dt) {
  const size_t N = 5 * (size_t)P.n[0] * P.n[1] * P.n[2];
  std::vector<T> R(N), Q1(N), Q2(N);
  rhs3(P, M, Q, R.data());
  for (size_t k = 0; k < N; ++k) Q1[k] = Q[k] + dt * R[k];
  rhs3(P, M, Q1.data(), R.data());
  for (size_t k = 0; k < N; ++k) Q2[k] = cst<T>(0.25L) * (Q1[k] + dt * R[k]) + cst<T>(0.75L) * Q[k];
  rhs3(P, M, Q2.data(), R.data());
  for (size_t k = 0; k < N; ++k) Q[k] = cst<T>(2.0L / 3) * (Q2[k] + dt * R[k]) + cst<T>(1.0L / 3) * Q[k];
}

static int check3(const int* ip, int ni, int nj, int nk) {
  if (ip[0] < 0 || ip[0] > 4 || ip[1] < 0 || ip[1] > 1) return 1;
  const int n[3] = {ni, nj, nk};
  for (int a = 0; a < 3; ++a) {
    if (ip[4 + 2 * a] < 0 || ip[4 + 2 * a] > 1 || ip[5 + 2 * a] < 0 || ip[5 + 2 * a] > 1) return 2;
    if ((ip[4 + 2 * a] == BC_PERIODIC) != (ip[5 + 2 * a] == BC_PERIODIC)) return 3;
    if (ip[4 + 2 * a] != BC_PERIODIC && n[a] < 13) return 4;   // the reflected ghosts reach 12 nodes in
    if (n[a] < 1) return 4;
  }
  return 0;
}

}  // namespace orc

extern "C" {

// 3-D: ip = {scheme, interp, ppm, linear_weights, bc[6]}; dp = {gamma, lf_alpha, eps,
// period[3][3]}; x, y, z and Q as documented above the three-dimensional section.
size_t orc3_metrics_len(int ni, int nj, int nk) { return (size_t)10 * (ni + 2 * G) * (nj + 2 * G) * (nk + 2 * G); }

int orc3_metrics(const int* ip, const double* dp, int ni, int nj, int nk, const double* x, const double* y,
                 const double* z, double* M) {
  if (int e = check3(ip, ni, nj, nk)) return e;
  Par3<double> P;
  unpack3(ip, dp, ni, nj, nk, P);
  const double* X[3] = {x, y, z};
  metrics3(P, X, M);
  return 0;
}

int orc3_rhs(const int* ip, const double* dp, int ni, int nj, int nk, const double* M, const double* Q, double* dQ) {
  if (int e = check3(ip, ni, nj, nk)) return e;
  Par3<double> P;
  unpack3(ip, dp, ni, nj, nk, P);
  rhs3(P, M, Q, dQ);
  return 0;
}

int orc3_rk3(const int* ip, const double* dp, int ni, int nj, int nk, const double* M, double* Q, double dt,
             int nsteps) {
  if (int e = check3(ip, ni, nj, nk)) return e;
  Par3<double> P;
  unpack3(ip, dp, ni, nj, nk, P);
  for (int s = 0; s < nsteps; ++s) rk3_3(P, M, Q, dt);
  return 0;
}

// line maxima A^ of every line of direction d, lines ordered (l1 fastest, l2)
int orc3_lambda(const int* ip, const double* dp, int ni, int nj, int nk, int d, const double* M, const double* Q,
                double* out) {
  if (int e = check3(ip, ni, nj, nk)) return e;
  Par3<double> P;
  unpack3(ip, dp, ni, nj, nk, P);
  Field3<double> F{P, M, Q};
  const int n1 = P.n[d == 0 ? 1 : 0], n2 = P.n[d == 2 ? 1 : 2];
  for (int l2 = 0; l2 < n2; ++l2)
    for (int l1 = 0; l1 < n1; ++l1) out[(size_t)l2 * n1 + l1] = line_lambda3(F, d, l1, l2);
  return 0;
}

// operation count of one right-hand side (Counted scalar) and of its three sweeps
int orc3_count_flops(const int* ip, const double* dp, int ni, int nj, int nk, const double* M, const double* Q,
                     long long* out) {
  if (int e = check3(ip, ni, nj, nk)) return e;
  Par3<Counted> P;
  unpack3(ip, dp, ni, nj, nk, P);
  const size_t NM = orc3_metrics_len(ni, nj, nk), NQ = 5 * (size_t)ni * nj * nk;
  std::vector<Counted> Mc(M, M + NM), Qc(Q, Q + NQ), R(NQ);
  Field3<Counted> F{P, Mc.data(), Qc.data()};
  g_flops = 0;
  rhs3(P, Mc.data(), Qc.data(), R.data());
  out[0] = g_flops;
  for (int d = 0; d < 3; ++d) {
    std::vector<Counted> Rd(NQ, Counted(0.0));
    g_flops = 0;
    sweep3(F, d, Rd);
    out[1 + d] = g_flops;
  }
  return 0;
}

// the eigenvectors along unit direction n (for the pins)
void orc3_eig(double gamma, const double* q, const double* n, double* L, double* R) {
  double Lm[5][5], Rm[5][5];
  eigvec3(q, n, gamma, Lm, Rm);
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b) { L[5 * a + b] = Lm[a][b]; R[5 * a + b] = Rm[a][b]; }
}

// the metrics in long double (to show the free-stream residual shrinks with the precision):
// residual max |dQ/dt| of the uniform state q0 on the grid, in the given precision
double orc3_fsp_residual(const int* ip, const double* dp, int ni, int nj, int nk, const double* x, const double* y,
                         const double* z, const double* q0, int wide) {
  if (check3(ip, ni, nj, nk)) return -1.0;
  const size_t NN = (size_t)ni * nj * nk;
  auto run = [&](auto zero) -> double {
    using T = decltype(zero);
    Par3<T> P;
    unpack3(ip, dp, ni, nj, nk, P);
    std::vector<T> X[3];
    const double* src[3] = {x, y, z};
    for (int c = 0; c < 3; ++c) { X[c].resize(NN); for (size_t o = 0; o < NN; ++o) X[c][o] = T(src[c][o]); }
    const T* Xp[3] = {X[0].data(), X[1].data(), X[2].data()};
    std::vector<T> M(orc3_metrics_len(ni, nj, nk)), Q(5 * NN), R(5 * NN);
    metrics3(P, Xp, M.data());
    for (int v = 0; v < 5; ++v) for (size_t o = 0; o < NN; ++o) Q[v * NN + o] = T(q0[v]);
    rhs3(P, M.data(), Q.data(), R.data());
    double worst = 0.0;
    for (auto& r : R) worst = std::max(worst, (double)std::fabs((long double)r));
    return worst;
  };
  return wide ? run((long double)0) : run(0.0);
}

}  // extern "C"
