// fsp_device.cuh -- device-side building blocks of the WENOIU right-hand side
// (Li & Sun, arXiv:1810.11103): scheme coefficients, boundary ghosts, Euler flux,
// characteristic projection and the mapped WENO interpolation.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fsp {

constexpr int G = 4;  // ghost layers of the stored metrics

enum { S31 = 0, S32 = 1, S51 = 2, S52 = 3, S71 = 4, S74 = 5 };
enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_DIRICHLET = 2, BC_SLIPWALL = 3, BC_FARFIELD = 4,
       BC_LINK = 5 };

// --------------------------------------------------------------------------------------
// Scheme coefficients (Section 3)
// --------------------------------------------------------------------------------------
// Scheme<S>: r = points per WENO candidate, nmp = midpoints in h+, m0/m1 = h+ coefficients
// of f+_{j+1/2} and f+_{j-1/2}, n(k) = h+ coefficient of f+_{j+k-2} (k = 0..4), hn(k) = h+
// coefficient of f+_{j+k} for any offset k (zero outside the scheme's stencil).
template <int S> struct Scheme;
// WENOIU3-1MP, Eq. (3.4): h+ = f_{j+1/2} + (-f_{j-1} + 2 f_j - f_{j+1}) / 24
template <> struct Scheme<S31> {
  static constexpr int r = 2, nmp = 1;
  static constexpr double m0 = 1.0, m1 = 0.0;
  __host__ __device__ static constexpr double n(int k) {
    return k == 1 || k == 3 ? -1.0 / 24 : k == 2 ? 2.0 / 24 : 0.0;
  }
  __host__ __device__ static constexpr double hn(int k) { return k < -2 || k > 2 ? 0.0 : n(k + 2); }
};
// WENOIU3-2MP, Eq. (3.8): h+ = f_{j+1/2} + (-f_{j-1/2} + 2 f_j - f_{j+1/2}) / 6
template <> struct Scheme<S32> {
  static constexpr int r = 2, nmp = 2;
  static constexpr double m0 = 5.0 / 6, m1 = -1.0 / 6;
  __host__ __device__ static constexpr double n(int k) { return k == 2 ? 2.0 / 6 : 0.0; }
  __host__ __device__ static constexpr double hn(int k) { return k < -2 || k > 2 ? 0.0 : n(k + 2); }
};
// WENOIU5-1MP, Eq. (3.16)
template <> struct Scheme<S51> {
  static constexpr int r = 3, nmp = 1;
  static constexpr double m0 = 1.0, m1 = 0.0;
  __host__ __device__ static constexpr double n(int k) {
    return k == 0 ? 19.0 / 1920 : k == 1 ? -29.0 / 480 : k == 2 ? 77.0 / 960 : k == 3 ? -3.0 / 160 : -7.0 / 640;
  }
  __host__ __device__ static constexpr double hn(int k) { return k < -2 || k > 2 ? 0.0 : n(k + 2); }
};
// WENOIU5-2MP, Eq. (3.20): h+ = f_{j+1/2} + [(-4 f_{j+1} + f_j + f_{j-1}) + (6 f_{j+1/2}
// - 4 f_{j-1/2})] / 30
template <> struct Scheme<S52> {
  static constexpr int r = 3, nmp = 2;
  static constexpr double m0 = 36.0 / 30, m1 = -4.0 / 30;
  __host__ __device__ static constexpr double n(int k) {
    return k == 1 || k == 2 ? 1.0 / 30 : k == 3 ? -4.0 / 30 : 0.0;
  }
  __host__ __device__ static constexpr double hn(int k) { return k < -2 || k > 2 ? 0.0 : n(k + 2); }
};
// WENOIU7-1MP (Appendix, scheme (1) with alpha = 1): h+ = f_{j+1/2} + (-243 f_{j-3} +
// 1990 f_{j-2} - 7481 f_{j-1} + 8164 f_j - 341 f_{j+1} - 2378 f_{j+2} + 289 f_{j+3}) / 107520
template <> struct Scheme<S71> {
  static constexpr int r = 4, nmp = 1;
  static constexpr double m0 = 1.0, m1 = 0.0;
  __host__ __device__ static constexpr double hn(int k) {
    return k == -3 ? -243.0 / 107520 : k == -2 ? 1990.0 / 107520 : k == -1 ? -7481.0 / 107520
         : k == 0 ? 8164.0 / 107520 : k == 1 ? -341.0 / 107520 : k == 2 ? -2378.0 / 107520
         : k == 3 ? 289.0 / 107520 : 0.0;
  }
};

// WENOIU7-4MP (Appendix, scheme (3)): h+ = f_{j+1/2} + [(18 f_{j-1} - 66 f_j - 108 f_{j+1}) +
// (-3 f_{j-3/2} - 31 f_{j-1/2} + 179 f_{j+1/2} + 11 f_{j+3/2})] / 420.  m0, m1 multiply
// f_{j+1/2}, f_{j-1/2}; mA, mB multiply f_{j-3/2}, f_{j+3/2} (nmp = 4: four midpoints).
template <> struct Scheme<S74> {
  static constexpr int r = 4, nmp = 4;
  static constexpr double m0 = 1.0 + 179.0 / 420, m1 = -31.0 / 420, mA = -3.0 / 420, mB = 11.0 / 420;
  __host__ __device__ static constexpr double hn(int k) {
    return k == -1 ? 18.0 / 420 : k == 0 ? -66.0 / 420 : k == 1 ? -108.0 / 420 : 0.0;
  }
};

// The h+ coefficients of a scheme at its free parameter alpha (the one-midpoint forms: Eq. 3.5
// for WENOIU3-1MP, Eq. 3.17 for WENOIU5-1MP, the Appendix's scheme (1) for WENOIU7-1MP; alpha =
// 1 is the printed scheme): m0, m1 multiply f+_{j+1/2}, f+_{j-1/2}; hn[k + 3] multiplies f+_{j+k}.
inline void scheme_coefs(int scheme, double a, double& m0, double& m1, double hn[7]) {
  for (int k = 0; k < 7; ++k) hn[k] = 0.0;
  m1 = 0.0;
  switch (scheme) {
    case S31:
      m0 = a; hn[2] = a / 8 - 1.0 / 6; hn[3] = -3 * a / 4 + 5.0 / 6; hn[4] = -3 * a / 8 + 1.0 / 3;
      if (a == 1.0) for (int k = 0; k < 7; ++k) hn[k] = Scheme<S31>::hn(k - 3);
      break;
    case S32:
      m0 = Scheme<S32>::m0; m1 = Scheme<S32>::m1;
      for (int k = 0; k < 7; ++k) hn[k] = Scheme<S32>::hn(k - 3);
      break;
    case S51:
      m0 = a; hn[1] = -3 * a / 128 + 1.0 / 30; hn[2] = 5 * a / 32 - 13.0 / 60; hn[3] = -45 * a / 64 + 47.0 / 60;
      hn[4] = -15 * a / 32 + 9.0 / 20; hn[5] = 5 * a / 128 - 1.0 / 20;
      if (a == 1.0) for (int k = 0; k < 7; ++k) hn[k] = Scheme<S51>::hn(k - 3);
      break;
    case S52:
      m0 = Scheme<S52>::m0; m1 = Scheme<S52>::m1;
      for (int k = 0; k < 7; ++k) hn[k] = Scheme<S52>::hn(k - 3);
      break;
    case S74:   // no free parameter (its four midpoint coefficients are compile-time constants)
      m0 = Scheme<S74>::m0; m1 = Scheme<S74>::m1;
      for (int k = 0; k < 7; ++k) hn[k] = Scheme<S74>::hn(k - 3);
      break;
    default:
      m0 = a; hn[0] = 5 * a / 1024 - 1.0 / 140; hn[1] = -21 * a / 512 + 5.0 / 84; hn[2] = 175 * a / 1024 - 101.0 / 420;
      hn[3] = -175 * a / 256 + 319.0 / 420; hn[4] = -525 * a / 1024 + 107.0 / 210; hn[5] = 35 * a / 512 - 19.0 / 210;
      hn[6] = -7 * a / 1024 + 1.0 / 105;
      if (a == 1.0) for (int k = 0; k < 7; ++k) hn[k] = Scheme<S71>::hn(k - 3);
      break;
  }
}

// Central operator delta^{c,(1)} of each scheme (Eq. 2.7), used for the metrics:
//   D f_j = sum_k a_k (f_{j+k} - f_{j-k}) + b_{1/2}(f~_{j+1/2} - f~_{j-1/2})
//           + b_{3/2}(f~_{j+3/2} - f~_{j-3/2}),  k = 1..4
struct Central { double a1, a2, a3, b12, b32, a4, b52; };
__host__ __device__ inline Central central_of(int scheme) {
  switch (scheme) {
    case S31: return {2.0 / 48, -1.0 / 48, 0.0, 1.0, 0.0};              // Eq. (3.7)
    case S32: return {2.0 / 12, 0.0, 0.0, 11.0 / 12, -1.0 / 12};        // Eq. (3.9)
    case S51: return {17.0 / 256, -13.0 / 320, 19.0 / 3840, 1.0, 0.0};  // Eq. (3.19)
    case S52: return {-4.0 / 60, 1.0 / 60, 0.0, 19.0 / 15, -1.0 / 15};  // Eq. (3.21)
    case S74:   // the Appendix's operator of WENOIU7-4MP, midpoints to 5/2
      return {-32.0 / 140, 3.0 / 140, 0.0, 1218.0 / 840, -17.0 / 840, 0.0, -3.0 / 840};
    default:  // the Appendix's eighth-order operator of WENOIU7-1MP
      return {8841.0 / 107520, -6069.0 / 107520, 1261.0 / 107520, 1.0, 0.0, -121.5 / 107520};
  }
}
// The same at the free parameter alpha of a one-midpoint scheme: the central part of the
// scheme, (delta+ + delta-)/2 with delta+ f_j = h+_{j+1/2} - h+_{j-1/2}, whose node
// coefficients are a_d = (n_d - n_{d+1} + n_{1-d} - n_{-d}) / 2 and whose midpoint coefficient is
// alpha.  alpha = 1 gives the printed operators above.
inline Central central_of(int scheme, double alpha) {
  if (alpha == 1.0 || scheme == S32 || scheme == S52 || scheme == S74) return central_of(scheme);
  double m0, m1, hn[7];
  scheme_coefs(scheme, alpha, m0, m1, hn);
  auto n = [&](int k) { return k < -3 || k > 3 ? 0.0 : hn[k + 3]; };
  double a[4];
  for (int d = 1; d <= 4; ++d) a[d - 1] = 0.5 * (n(d) - n(d + 1) + n(1 - d) - n(-d));
  return {a[0], a[1], a[2], m0, 0.0, a[3]};
}

// Midpoint value at j+1/2 from nodal values v[k] = f_{j+k-2}, k = 0..5 (f_{j-2}..f_{j+3}).
// interp 1: two-point average; else Lagrange with 4 (third-order schemes) or 6 points.
template <typename T>
__device__ __forceinline__ T mid_interp(int interp, bool sixth, const T* v) {
  if (interp == 1) return T(0.5) * (v[2] + v[3]);
  if (!sixth) return (T(9) * (v[2] + v[3]) - (v[1] + v[4])) * T(1.0 / 16);
  return (T(150) * (v[2] + v[3]) - T(25) * (v[1] + v[4]) + T(3) * (v[0] + v[5])) * T(1.0 / 256);
}

// The same for WENOIU7 from v[k] = f_{j+k-3}, k = 0..7: eight-point Lagrange.
template <typename T>
__device__ __forceinline__ T mid_interp8(int interp, const T* v) {
  if (interp == 1) return T(0.5) * (v[3] + v[4]);
  return (T(1225) * (v[3] + v[4]) - T(245) * (v[2] + v[5]) + T(49) * (v[1] + v[6]) - T(5) * (v[0] + v[7])) *
         T(1.0 / 2048);
}

// --------------------------------------------------------------------------------------
// Kernel parameters (plain data, passed by value)
// --------------------------------------------------------------------------------------
struct Params {
  int ni, nj;
  long long ld;             // row stride of Q-shaped arrays
  int bc[4];
  int interp, ppm, linw;
  int wz, msplit;           // WENO-Z weights; midpoint splitting (0 LF, 1 Steger-Warming, 2 Van Leer)
  double gamma, alpha, eps;
  // halved h+ coefficients (the h combination adds twice the split fluxes): [0] m0/2 of
  // f+_{j+1/2}, [1] m1/2 of f+_{j-1/2}, [5 + k] n_k/2 of f+_{j+k}, k = -3..3; and as float
  double hc[9];
  float hcf[9];
  double bcq[4][4];
  const double* met;        // haloed metrics
  long long mld;            // ni + 2G
  long long mplane;         // (ni + 2G) (nj + 2G)
  // linked faces (multi-block): neighbour block, its face, reversed tangential index,
  // and the neighbour's extents; the neighbour's state comes from a per-block table
  int lnb[4], lface[4], lrev[4], lni[4], lnj[4];
  long long lld[4];
};

// The scheme's coefficients at its free parameter into the kernel parameters.
inline void set_scheme_coefs(Params& P, int scheme, double alpha) {
  double m0, m1, hn[7];
  scheme_coefs(scheme, alpha, m0, m1, hn);
  P.hc[0] = 0.5 * m0;
  P.hc[1] = 0.5 * m1;
  for (int k = 0; k < 7; ++k) P.hc[2 + k] = 0.5 * hn[k];
  for (int i = 0; i < 9; ++i) P.hcf[i] = (float)P.hc[i];
}

// Node of the neighbour behind linked face f for the ghost (gi, gj) of a block of size
// ni x nj: the blocks partition one larger grid, so the ghost at depth k beyond face f is
// the neighbour's node at depth k inward from its face, with the index along the face
// running the same way or reversed.
__host__ __device__ __forceinline__ void link_node(int f, int ni, int nj, int nface, int nrev, int nni,
                                                   int nnj, int gi, int gj, int& oi, int& oj) {
  const int k = f == 0 ? -1 - gi : f == 1 ? gi - ni : f == 2 ? -1 - gj : gj - nj;
  int t = f < 2 ? gj : gi;
  if (nrev) t = (nface < 2 ? nnj : nni) - 1 - t;
  const int d = (nface == 0 || nface == 2) ? k : (nface == 1 ? nni - 1 - k : nnj - 1 - k);
  if (nface < 2) { oi = d; oj = t; } else { oi = t; oj = d; }
}

__device__ __forceinline__ double met_at(const Params& P, int p, int i, int j) {
  return __ldg(P.met + p * P.mplane + (long long)(j + G) * P.mld + (i + G));
}

__device__ __forceinline__ int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// --------------------------------------------------------------------------------------
// Small arithmetic helpers by precision
// --------------------------------------------------------------------------------------
// FP32 uses the hardware's approximate reciprocal and reciprocal square root (PTX
// rcp.approx.ftz / rsqrt.approx.ftz, about 1 ulp) directly: every operand here is a
// positive normal number (densities, sound speeds, metric norms, eps + IS >= 1e-30, sums of
// weights), and a result flushed to zero is the right limit for a vanishing weight.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// FP64 reciprocal: the hardware seed (PTX rcp.approx.ftz.f64) refined once by the
// third-order Householder iteration for f(r) = 1/r - x, r <- r (1 + e + e^2) with
// e = 1 - x r: a seed of relative error d leaves d^3, so one step takes a seed good to 20
// bits past double precision; three fused multiply-adds in all.  It replaces the IEEE
// division on the FP64 pipe for the nonzero normal operands of this code (densities, J^-1,
// sums of weights); the result is within a few ulps of 1/x (fsp_reciprocal_check).
__device__ __forceinline__ double rcp_nr(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}
// FP64 reciprocal square root: the hardware seed (PTX rsqrt.approx.ftz.f64) refined once by
// the third-order step of the binomial series 1/sqrt(x) = y / sqrt(1 - e) = y (1 + e/2 +
// 3 e^2/8 + ...), e = 1 - x y^2: a seed of relative error d leaves about d^3.  Two products
// and three fused multiply-adds, for the positive normal operands of this code (sound speeds
// squared, metric norms); within a few ulps of 1/sqrt(x) (fsp_reciprocal_check).
__device__ __forceinline__ double rsq_nr(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y * y, 1.0);
  return fma(y * e, fma(0.375, e, 0.5), y);
}
__device__ __forceinline__ double rsq(double x) { return rsq_nr(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrt_approx(x); }
// quotient: a times the refined reciprocal in FP64, a times the approximate reciprocal in FP32
__device__ __forceinline__ double quot(double a, double b) { return a * rcp_nr(b); }
__device__ __forceinline__ float quot(float a, float b) { return a * rcp_approx(b); }
// reciprocal: refined in FP64; the approximate reciprocal in FP32
__device__ __forceinline__ double recip(double x) { return rcp_nr(x); }
__device__ __forceinline__ float recip(float x) { return rcp_approx(x); }

// A double rounded to the state type.  from_f64<float> is the hardware conversion (round to
// nearest even).  from_f64_int rounds the same way with integer operations only (zero and
// subnormals to signed zero, overflow to infinity, NaN to a quiet NaN, infinity kept), for the
// mixed path, whose FP64 pipe is its bottleneck.
template <typename T> __device__ __forceinline__ T from_f64(double d);
template <> __device__ __forceinline__ double from_f64<double>(double d) { return d; }
template <> __device__ __forceinline__ float from_f64<float>(double d) { return __double2float_rn(d); }
__device__ __forceinline__ float from_f64_int(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const unsigned ex = (hi >> 20) & 0x7ffu;
  if (ex == 0x7ffu && ((hi & 0xfffffu) | lo)) return __uint_as_float(sign | 0x7fc00000u);   // NaN
  const int e = (int)ex - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);   // top 23 of the 52 mantissa bits
  const unsigned rest = lo & 0x1fffffffu;              // the 29 bits dropped
  m += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
  return __uint_as_float(sign | (((unsigned)e << 23) + m));   // a mantissa carry bumps the exponent
}

// A float widened to double with integer operations only, so that the mixed path queues
// nothing on its bottleneck, the FP64 pipe: a normal float's exponent is rebiased (127 ->
// 1023) and its 23 mantissa bits become the top of the 52 (exact, the hardware's bits);
// infinities and NaN keep their class (NaN its payload's top bits); zero keeps its sign, and
// so do subnormals, which become signed zero (below 1.2e-38, never met as a flux or state
// of this path).  Selects, no branch.
__device__ __forceinline__ double to_f64_int(float x) {
  const unsigned b = __float_as_uint(x), sign = b & 0x80000000u, e = (b >> 23) & 0xffu;
  const unsigned m = (b & 0x7fffffu) >> 3;
  unsigned hi = sign | ((e + 896u) << 20) | m;
  hi = e == 0u ? sign : hi;
  hi = e == 0xffu ? (sign | 0x7ff00000u | m) : hi;
  return __hiloint2double((int)hi, e == 0u ? 0 : (int)(b << 29));
}
// Conversions between the state type and the accumulation type, on the integer pipe where
// they would cost FP64-pipe issue (float <-> double); identity otherwise.
template <typename Acc> __device__ __forceinline__ Acc widen(float x);
template <> __device__ __forceinline__ float widen<float>(float x) { return x; }
template <> __device__ __forceinline__ double widen<double>(float x) { return to_f64_int(x); }
template <typename Acc> __device__ __forceinline__ Acc widen(double x) { return x; }
template <typename Real> __device__ __forceinline__ Real narrow(float x) { return x; }
template <typename Real> __device__ __forceinline__ Real narrow(double x);
template <> __device__ __forceinline__ double narrow<double>(double x) { return x; }
template <> __device__ __forceinline__ float narrow<float>(double x) { return from_f64_int(x); }

// A double rounded to the state type on the integer pipe (identity for double), for kernels
// that convert several metrics per node and leave most issue slots free: there the narrow
// FP64 pipe, which carries the hardware conversion, would be the bound.
template <typename T> __device__ __forceinline__ T from_f64_alu(double d);
template <> __device__ __forceinline__ double from_f64_alu<double>(double d) { return d; }
template <> __device__ __forceinline__ float from_f64_alu<float>(double d) { return from_f64_int(d); }

// x <= 0 from the sign and magnitude bits (integer compare, no floating-point pipe)
__device__ __forceinline__ bool nonpos(double x) { return __double_as_longlong(x) <= 0LL; }
__device__ __forceinline__ bool nonpos(float x) { return __float_as_int(x) <= 0; }

// Ghost state along direction dir for the line `line` (row j for dir 0, column i for
// dir 1) at position g (any integer; interior when 0 <= g < n).
template <typename Real>
__device__ __forceinline__ void load_state(const Params& P, const Real* __restrict__ Q, int dir,
                                           int line, int g, Real q[4],
                                           const Real* const* qtab = nullptr) {
  const int n = dir == 0 ? P.ni : P.nj;
  const long long plane = (long long)P.nj * P.ld;
  auto rd = [&](int gg) {
    const long long o = dir == 0 ? (long long)line * P.ld + gg : (long long)gg * P.ld + line;
#pragma unroll
    for (int v = 0; v < 4; ++v) q[v] = Q[v * plane + o];
  };
  if (g >= 0 && g < n) { rd(g); return; }
  const int face = 2 * dir + (g < 0 ? 0 : 1);
  const int b = g < 0 ? 0 : n - 1;
  const int kind = P.bc[face];
  if (kind == BC_PERIODIC) { rd(pmod(g, n)); return; }
  if (kind == BC_LINK) {
    int oi, oj;
    link_node(face, P.ni, P.nj, P.lface[face], P.lrev[face], P.lni[face], P.lnj[face],
              dir == 0 ? g : line, dir == 0 ? line : g, oi, oj);
    const Real* N = qtab[P.lnb[face]];
    const long long nplane = (long long)P.lnj[face] * P.lld[face], o = (long long)oj * P.lld[face] + oi;
#pragma unroll
    for (int v = 0; v < 4; ++v) q[v] = N[v * nplane + o];
    return;
  }
  if (kind == BC_DIRICHLET) {
#pragma unroll
    for (int v = 0; v < 4; ++v) q[v] = Real(P.bcq[face][v]);
    return;
  }
  const double mx = dir == 0 ? met_at(P, 0, b, line) : met_at(P, 2, line, b);
  const double my = dir == 0 ? met_at(P, 1, b, line) : met_at(P, 3, line, b);
  if (kind == BC_SLIPWALL) {
    rd(2 * b - g);
    const double inv = rsqrt(mx * mx + my * my);
    const Real nx = Real(mx * inv), ny = Real(my * inv);
    const Real un = q[1] * nx + q[2] * ny;
    q[1] = q[1] - Real(2) * un * nx;
    q[2] = q[2] - Real(2) * un * ny;
    return;
  }
  if (kind == BC_FARFIELD) {
    const double vn = (g < 0 ? -1.0 : 1.0) * (P.bcq[face][1] * mx + P.bcq[face][2] * my);
    if (vn < 0.0) {
#pragma unroll
      for (int v = 0; v < 4; ++v) q[v] = Real(P.bcq[face][v]);
      return;
    }
  }
  rd(b);  // transmissive (and far-field outflow)
}

// |U^| + c |k^| (the quantity maximised along a line for A^, Section 2.3)
template <typename Real>
__device__ __forceinline__ Real spectral_radius(const Real q[4], Real mx, Real my, Real gamma) {
  const Real rinv = recip(q[0]);
  const Real u = q[1] * rinv, v = q[2] * rinv;
  const Real p = (gamma - Real(1)) * (q[3] - Real(0.5) * (q[1] * u + q[2] * v));
  // c |k^| = sqrt(gamma p / rho |k^|^2): one square root
  return fabs(mx * u + my * v) + sqrt(gamma * p * rinv * (mx * mx + my * my));
}

// Primitive quantities of a node used by the characteristic projection (Section 3.4).
template <typename Real>
struct Prim {
  Real u, v, c, cinv, H, b1, h2;  // b1 = (gamma-1)/c^2, h2 = |u|^2/2
};

template <typename Real>
__device__ __forceinline__ Prim<Real> prim_of(const Real q[4], Real gamma) {
  Prim<Real> w;
  const Real rinv = recip(q[0]);
  w.u = q[1] * rinv;
  w.v = q[2] * rinv;
  w.h2 = Real(0.5) * (w.u * w.u + w.v * w.v);
  const Real gm1 = gamma - Real(1);
  const Real p = gm1 * (q[3] - q[0] * w.h2);
  const Real c2 = gamma * p * rinv;
  w.cinv = rsq(c2);
  w.c = c2 * w.cinv;
  w.H = (q[3] + p) * rinv;
  w.b1 = gm1 * w.cinv * w.cinv;
  return w;
}

// Per node |U^| + c|k^| of both directions (and the CFL rate) in the state's arithmetic:
// the splitting needs A^ constant along a line, not any particular precision, so the FP32
// paths take their line maxima in float.
template <typename Real>
__device__ __forceinline__ void node_speeds(const Params& P, const Real* __restrict__ Q, int i, int j,
                                            Real& sx, Real& se, Real& rate) {
  const long long plane = (long long)P.nj * P.ld, o = (long long)j * P.ld + i;
  Real q[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) q[v] = Q[v * plane + o];
  const Real g = from_f64<Real>(P.gamma);
  sx = spectral_radius(q, from_f64_alu<Real>(met_at(P, 0, i, j)), from_f64_alu<Real>(met_at(P, 1, i, j)), g);
  se = spectral_radius(q, from_f64_alu<Real>(met_at(P, 2, i, j)), from_f64_alu<Real>(met_at(P, 3, i, j)), g);
  rate = (sx + se) * recip(from_f64_alu<Real>(met_at(P, 4, i, j)));
}

// Steger-Warming (mode 1) and Van Leer (mode 2) splittings of the metric-weighted flux along
// k = (mx, my) for the midpoint flux (an option beyond the paper's, Section 7); returns twice
// F+ (sign > 0) or twice F- (sign < 0), F+ + F- = E^.  With n = k/|k|, Un = u.n:
// Steger-Warming F+- = rho/(2 gamma) [l0+- (1, u - c nx, v - c ny, H - c Un) + 2 (gamma - 1)
// l1+- (1, u, v, |u|^2/2) + l2+- (1, u + c nx, v + c ny, H + c Un)], l = |k| (Un - c, Un, Un + c),
// l+- = (l +- |l|)/2; Van Leer with M = Un/c: F+ = E^, F- = 0 for M >= 1 (the reverse for
// M <= -1), else m+- = +- rho c |k| (M +- 1)^2 / 4 and F+- = m+- (1, u + nx (-Un +- 2c)/gamma,
// v + ny (-Un +- 2c)/gamma, ((gamma - 1) Un +- 2c)^2 / (2 (gamma^2 - 1)) + (|u|^2 - Un^2)/2).
template <typename T>
__device__ __forceinline__ void split_mid2(int mode, int sign, const T q[4], T mx, T my, T gamma, T f[4]) {
  const T rinv = recip(q[0]);
  const T u = q[1] * rinv, v = q[2] * rinv, q2 = u * u + v * v;
  const T p = (gamma - T(1)) * (q[3] - T(0.5) * q[0] * q2);
  const T c = sqrt(gamma * p * rinv);
  const T kn = sqrt(mx * mx + my * my), ki = recip(kn), nx = mx * ki, ny = my * ki;
  const T Un = u * nx + v * ny;
  const T s = sign > 0 ? T(1) : T(-1);
  if (mode == 1) {
    const T H = (q[3] + p) * rinv;
    T l0 = kn * (Un - c), l1 = kn * Un, l2 = kn * (Un + c);
    l0 = T(0.5) * (l0 + s * fabs(l0));
    l1 = T(0.5) * (l1 + s * fabs(l1));
    l2 = T(0.5) * (l2 + s * fabs(l2));
    const T a = q[0] / gamma, g2 = T(2) * (gamma - T(1));
    f[0] = a * (l0 + g2 * l1 + l2);
    f[1] = a * (l0 * (u - c * nx) + g2 * l1 * u + l2 * (u + c * nx));
    f[2] = a * (l0 * (v - c * ny) + g2 * l1 * v + l2 * (v + c * ny));
    f[3] = a * (l0 * (H - c * Un) + (gamma - T(1)) * l1 * q2 + l2 * (H + c * Un));
    return;
  }
  const T M = Un * recip(c);
  if (M >= T(1) || M <= T(-1)) {
    if ((M >= T(1)) == (sign > 0)) {
      const T U = kn * Un;
      f[0] = T(2) * q[0] * U;
      f[1] = T(2) * (q[1] * U + mx * p);
      f[2] = T(2) * (q[2] * U + my * p);
      f[3] = T(2) * (q[3] + p) * U;
    } else {
      f[0] = f[1] = f[2] = f[3] = T(0);
    }
    return;
  }
  const T mp = M + s;
  const T fm = T(0.5) * s * q[0] * c * kn * mp * mp;   // twice the mass flux
  const T w = (s * T(2) * c - Un) / gamma;
  const T e = (gamma - T(1)) * Un + s * T(2) * c;
  f[0] = fm;
  f[1] = fm * (u + nx * w);
  f[2] = fm * (v + ny * w);
  f[3] = fm * (e * e / (T(2) * (gamma * gamma - T(1))) + T(0.5) * (q2 - Un * Un));
}

// --------------------------------------------------------------------------------------
// Characteristic projection (Section 3.4): left eigenvector rows of the flux Jacobian at
// a node along the unit direction (nx, ny); R is applied in factored form in recon().
// --------------------------------------------------------------------------------------
template <typename Real>
struct Eig {
  Real L[4][4];
  Real u, v, c, H, Un, Ut, nx, ny, h2;

  __device__ __forceinline__ void build(const Prim<Real>& w, Real nx_, Real ny_) {
    nx = nx_; ny = ny_;
    u = w.u; v = w.v; c = w.c; H = w.H; h2 = w.h2;
    Un = u * nx + v * ny;
    Ut = v * nx - u * ny;
    const Real b1 = w.b1, b2 = b1 * h2;
    const Real hb1 = Real(0.5) * b1, hb2 = Real(0.5) * b2;
    const Real hc = Real(0.5) * w.cinv;
    const Real hUc = Un * hc, hnxc = nx * hc, hnyc = ny * hc;
    L[0][0] = hb2 + hUc; L[0][1] = -hb1 * u - hnxc; L[0][2] = -hb1 * v - hnyc; L[0][3] = hb1;
    L[1][0] = Real(1) - b2; L[1][1] = b1 * u; L[1][2] = b1 * v; L[1][3] = -b1;
    L[2][0] = -Ut; L[2][1] = -ny; L[2][2] = nx; L[2][3] = Real(0);
    L[3][0] = hb2 - hUc; L[3][1] = -hb1 * u + hnxc; L[3][2] = -hb1 * v + hnyc; L[3][3] = hb1;
  }
  __device__ __forceinline__ Real project(int k, Real d0, Real d1, Real d2, Real d3) const {
    if (k == 2) return L[2][0] * d0 + L[2][1] * d1 + L[2][2] * d2;
    return L[k][0] * d0 + L[k][1] * d1 + L[k][2] * d2 + L[k][3] * d3;
  }
  // dq = R W with R's columns (1, u - c nx, v - c ny, H - c Un), (1, u, v, |u|^2/2),
  // (0, -ny, nx, Ut), (1, u + c nx, v + c ny, H + c Un)
  __device__ __forceinline__ void recon(const Real W[4], Real q[4]) const {
    const Real s = W[0] + W[3], d = W[3] - W[0];
    const Real a = s + W[1];
    q[0] = a;
    q[1] = u * a + c * nx * d - ny * W[2];
    q[2] = v * a + c * ny * d + nx * W[2];
    q[3] = H * s + c * Un * d + h2 * W[1] + Ut * W[2];
  }
};

// --------------------------------------------------------------------------------------
// The same projection and reconstruction for the right-hand-side sweeps, arranged for fewer
// operations.  Node quantities that do not depend on the direction are computed once per
// staged node (NodeChar), for a reconstruction scale S (weno_scale: the interpolated
// characteristic values arrive multiplied by S, which the reconstruction divides out exactly).
// The rows of L satisfy L_0 + L_3 = e_0 - L_1 and L_0 - L_3 = (Un, -nx, -ny, 0) / c, so
//   w_1 = L_1 dq,  w_0, w_3 = (dq_0 - w_1) / 2 +- (Un dq_0 - nx dq_1 - ny dq_2) / (2c),
//   w_2 = -Ut dq_0 - ny dq_1 + nx dq_2
// (the same values as Eig::project up to rounding), and the reconstruction adds R W / S to
// the centre state in one chain of fused multiply-adds.
// --------------------------------------------------------------------------------------
template <typename Real>
struct NodeChar {
  Real u, v, hc, a10;      // u, v, 1/(2c), 1 - b2            (b1 = (gamma-1)/c^2, b2 = b1 |u|^2/2)
  Real b1u, b1v, b1, cs;   // b1 u, b1 v, b1, c/S
  Real us, vs, Hs, h2s;    // u/S, v/S, H/S, |u|^2/(2S)
};

// Node quantities and the pressure of state q (reconstruction scale SC).
template <typename Real, int SC>
__device__ __forceinline__ NodeChar<Real> node_char(const Real q[4], Real gamma, Real& p) {
  NodeChar<Real> w;
  const Real rinv = recip(q[0]);
  const Real u = q[1] * rinv, v = q[2] * rinv;
  const Real h2 = Real(0.5) * (u * u + v * v);
  const Real gm1 = gamma - Real(1);
  p = gm1 * (q[3] - q[0] * h2);
  const Real c2 = gamma * p * rinv;
  const Real cinv = rsq(c2);
  const Real c = c2 * cinv;
  const Real H = (q[3] + p) * rinv;
  const Real b1 = gm1 * cinv * cinv;
  constexpr Real is = Real(1.0 / SC);
  w.u = u; w.v = v; w.hc = Real(0.5) * cinv; w.a10 = fma(-b1, h2, Real(1));
  w.b1u = b1 * u; w.b1v = b1 * v; w.b1 = b1; w.cs = c * is;
  w.us = u * is; w.vs = v * is; w.Hs = H * is; w.h2s = h2 * is;
  return w;
}

// The direction-independent part of the projection of a state difference d at a node:
// A = L_1 d (the entropy row does not depend on the direction) and S = (d_0 - A) / 2.
template <typename Real>
__device__ __forceinline__ void char_common(const NodeChar<Real>& w, const Real d[4], Real& A, Real& S) {
  A = fma(w.a10, d[0], fma(w.b1u, d[1], fma(w.b1v, d[2], -w.b1 * d[3])));
  S = Real(0.5) * (d[0] - A);
}

// The direction-dependent part of one side of an interface: the eigen-system of the centre
// node along the unit direction (nx, ny), and the reconstruction back to the state (scale SC).
template <typename Real, int SC>
struct CharDir {
  Real Ut, Unc, nxc, nyc, nx, ny;
  Real us, vs, Hs, h2s, csnx, csny, csUn, Uts;
  __device__ __forceinline__ void build(const NodeChar<Real>& w, Real nx_, Real ny_) {
    nx = nx_; ny = ny_;
    const Real Un = w.u * nx + w.v * ny;
    Ut = w.v * nx - w.u * ny;
    Unc = Un * w.hc; nxc = nx * w.hc; nyc = ny * w.hc;
    us = w.us; vs = w.vs; Hs = w.Hs; h2s = w.h2s;
    csnx = w.cs * nx; csny = w.cs * ny; csUn = w.cs * Un; Uts = Ut * Real(1.0 / SC);
  }
  // characteristic values (w_0 .. w_3) of the state difference d, from its common part
  __device__ __forceinline__ void project(const Real d[4], Real A, Real S, Real w[4]) const {
    const Real B = fma(Unc, d[0], -fma(nxc, d[1], nyc * d[2]));
    w[0] = S + B;
    w[1] = A;
    w[2] = fma(-Ut, d[0], fma(-ny, d[1], nx * d[2]));
    w[3] = S - B;
  }
  // Q = qc + R W / S, with R's columns (1, u - c nx, v - c ny, H - c Un), (1, u, v, |u|^2/2),
  // (0, -ny, nx, Ut), (1, u + c nx, v + c ny, H + c Un)
  __device__ __forceinline__ void recon(const Real W[4], const Real qc[4], Real Q[4]) const {
    const Real s = W[0] + W[3], dd = W[3] - W[0], a = s + W[1];
    constexpr Real is = Real(1.0 / SC);
    Q[0] = fma(a, is, qc[0]);
    Q[1] = fma(us, a, fma(csnx, dd, fma(-ny * is, W[2], qc[1])));
    Q[2] = fma(vs, a, fma(csny, dd, fma(nx * is, W[2], qc[2])));
    Q[3] = fma(Hs, s, fma(csUn, dd, fma(h2s, W[1], fma(Uts, W[2], qc[3]))));
  }
};

// One side of an interface (both parts together).
template <typename Real, int SC>
struct CharSide {
  NodeChar<Real> w;
  CharDir<Real, SC> dir;
  __device__ __forceinline__ void build(const NodeChar<Real>& w_, Real nx_, Real ny_) {
    w = w_;
    dir.build(w_, nx_, ny_);
  }
  __device__ __forceinline__ void project(Real d0, Real d1, Real d2, Real d3, Real out[4]) const {
    const Real d[4] = {d0, d1, d2, d3};
    Real A, S;
    char_common(w, d, A, S);
    dir.project(d, A, S, out);
  }
  __device__ __forceinline__ void recon(const Real W[4], const Real qc[4], Real Q[4]) const { dir.recon(W, qc, Q); }
};

// --------------------------------------------------------------------------------------
// WENO interpolation to x_{j+1/2} (Eqs. 3.10-3.13, Table 1), indicators of Eq. (3.22) on
// consecutive differences (for r = 2 the three-point IS_0, IS_1 of Section 5.1), mapping
// of Eq. (3.15) (r = 2) or (3.23) (r = 3).  Written on values relative to the stencil
// centre, u[m+2] = w_{j+m} - w_j (u[2] is not read): the candidates' coefficients sum to
// one and the indicators use differences only, so the interpolant of w is w_j plus the
// returned value, and uniform data give exactly 0.
// Weights.  FP64: omega_k = C_k prod_{l!=k} b_l^2 / sum_m C_m prod_{l!=m} b_l^2,
// b = eps + IS (one reciprocal; b >= eps keeps every product in range).  FP32:
// omega_k proportional to C_k (b_min / b_k)^2, whose terms stay in [0, C_k].
// The mapped weights g_k are normalised in the final quotient sum g p / sum g.
// --------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T is_b(T e, T f, T eps) {
  return eps + T(13.0 / 12) * e * e + T(0.25) * f * f;
}

template <typename T, int K>
__device__ __forceinline__ void raw_weights(const T* b, const T* C, T* w) {
  if constexpr (sizeof(T) == 8) {
    T s[K];
#pragma unroll
    for (int k = 0; k < K; ++k) s[k] = b[k] * b[k];
    T t[K];
    if constexpr (K == 4) {
      const T s01 = s[0] * s[1], s23 = s[2] * s[3];
      t[0] = C[0] * (s[1] * s23);
      t[1] = C[1] * (s[0] * s23);
      t[2] = C[2] * (s01 * s[3]);
      t[3] = C[3] * (s01 * s[2]);
    } else if constexpr (K == 3) {
      t[0] = C[0] * (s[1] * s[2]);
      t[1] = C[1] * (s[0] * s[2]);
      t[2] = C[2] * (s[0] * s[1]);
    } else {
      t[0] = C[0] * s[1];
      t[1] = C[1] * s[0];
    }
    T sum = t[0];
#pragma unroll
    for (int k = 1; k < K; ++k) sum += t[k];
    const T inv = recip(sum);
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = t[k] * inv;
  } else {
    T bmin = b[0];
#pragma unroll
    for (int k = 1; k < K; ++k) bmin = fminf(bmin, b[k]);
    T t[K], sum = T(0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const T r = quot(bmin, b[k]);
      t[k] = C[k] * r * r;
      sum += t[k];
    }
    const T inv = quot(T(1), sum);
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] = t[k] * inv;
  }
}

// The unnormalised weight terms t_k and the reciprocal of their sum (omega_k = t_k inv), as
// raw_weights: FP64 t_k = C_k prod_{l!=k} b_l^2; FP32 t_k = C_k (b_min / b_k)^2.
template <typename T, int K>
__device__ __forceinline__ void raw_terms(const T* b, const T* C, T* t, T& inv) {
  if constexpr (sizeof(T) == 8) {
    T s[K];
#pragma unroll
    for (int k = 0; k < K; ++k) s[k] = b[k] * b[k];
    if constexpr (K == 3) {
      t[0] = C[0] * (s[1] * s[2]);
      t[1] = C[1] * (s[0] * s[2]);
      t[2] = C[2] * (s[0] * s[1]);
    } else {
      t[0] = C[0] * s[1];
      t[1] = C[1] * s[0];
    }
  } else {
    T bmin = b[0];
#pragma unroll
    for (int k = 1; k < K; ++k) bmin = fminf(bmin, b[k]);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const T r = quot(bmin, b[k]);
      t[k] = (C[k] * r) * r;
    }
  }
  T sum = t[0];
#pragma unroll
  for (int k = 1; k < K; ++k) sum += t[k];
  inv = recip(sum);
}

// Indicators of the r = 4 candidates (WENOIU7): the quadratic form, in the three consecutive
// differences (d1, d2, d3) of a candidate's values, of the integral over [x_{j-1/2}, x_{j+1/2}]
// of the squared first to third derivatives of its interpolating cubic (times h, h^3, h^5),
// the definition that gives Eq. (3.22) for r = 3.  Rows (a11, a22, a33, 2 a12, 2 a13,
// 2 a23) / 2880 per candidate k = 0..3.
__host__ __device__ constexpr double is4c(int k, int i) {
  constexpr double A[4][6] = {{6649, 45076, 25729, -33916, 22778, -63436},
                              {3169, 17236, 6649, -13036, 5978, -17116},
                              {6649, 17236, 3169, -17116, 5978, -13036},
                              {25729, 45076, 6649, -63436, 22778, -33916}};
  return A[k][i] / 2880.0;
}
template <typename T>
__device__ __forceinline__ T is_b4(int k, T d1, T d2, T d3, T eps) {
  return eps + d1 * (T(is4c(k, 0)) * d1 + T(is4c(k, 3)) * d2 + T(is4c(k, 4)) * d3) +
         d2 * (T(is4c(k, 1)) * d2 + T(is4c(k, 5)) * d3) + T(is4c(k, 2)) * d3 * d3;
}

// The value weno_delta / weno_delta_x2 return is the interpolant times weno_scale<R>():
// the candidates are formed with integer-free coefficients (below), and the caller divides
// by the scale exactly (a power of two) where it adds the reconstruction to the centre state.
template <int R>
__host__ __device__ constexpr int weno_scale() { return R == 2 ? 4 : R == 3 ? 8 : 1; }

// The three-point differences of Eq. (3.22) on values relative to the centre (u_j = 0):
// IS_0 uses e0 = u_{j-2} - 2 u_{j-1} and f0 = u_{j-2} - 4 u_{j-1}; IS_1 uses e1 = u_{j+1} + u_{j-1}
// and f1 = u_{j+1} - u_{j-1}; IS_2 uses e2 = u_{j+2} - 2 u_{j+1} and f2 = u_{j+2} - 4 u_{j+1}
// (each IS = 13/12 e^2 + 1/4 f^2).  The same differences give the candidates of Table 1:
// 8 p_0 = e0 + 2 f0, 8 p_1 = e1 + 2 f1, 8 p_2 = e2 - 2 f2 (r = 3), and 4 p_0 = f1 - e1,
// 4 p_1 = e1 + f1 (r = 2).  The indicators are taken four times over, b = 4 (eps + IS) =
// 4 eps + 13/3 e^2 + f^2: the weights depend on ratios of the b only.
template <typename T>
__device__ __forceinline__ T is_b4x(T e, T f, T eps4) {
  return fma(T(13.0 / 3) * e, e, fma(f, f, eps4));
}

// WENO-Z weights (an option beyond the paper's, Section 7): t_k = C_k (1 + (tau / b_k)^2) with
// the global indicator tau of the b (differences of the b cancel eps), normalised by the
// reciprocal of their sum; result sum t_k P_k inv.  FP64 forms the ratios directly; FP32
// scales them by b_min (s_k = b_min / b_k <= 1) and writes t_k = C_k (beta + (1 - beta) s_k^2),
// beta = b_min^2 / (b_min^2 + tau^2), so that no term overflows.
template <typename T, int K>
__device__ __forceinline__ T weno_z_combine(const T* b, T tau, const T* C, const T* P) {
  T t[K], sum = T(0);
  if constexpr (sizeof(T) == 8) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const T q = quot(tau, b[k]);
      t[k] = C[k] * fma(q, q, T(1));
      sum += t[k];
    }
  } else {
    T bmin = b[0];
#pragma unroll
    for (int k = 1; k < K; ++k) bmin = fminf(bmin, b[k]);
    T beta;
    if (tau <= bmin) { const T x = quot(tau, bmin); beta = recip(fma(x, x, T(1))); }
    else { const T y = quot(bmin, tau), y2 = y * y; beta = quot(y2, y2 + T(1)); }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const T sk = quot(bmin, b[k]);
      t[k] = C[k] * fma(T(1) - beta, sk * sk, beta);
      sum += t[k];
    }
  }
  T num = t[0] * P[0];
#pragma unroll
  for (int k = 1; k < K; ++k) num = fma(t[k], P[k], num);
  return num * recip(sum);
}

template <int R, typename T>
__device__ __forceinline__ T weno_delta(const T* u, T eps, int ppm, int linw, int wz = 0) {
  if constexpr (R == 4) {
    // Table A1 candidates relative to w_j, u[m+3] = w_{j+m} - w_j (u[3] is not read)
    const T p[4] = {T(-5.0 / 16) * u[0] + T(21.0 / 16) * u[1] - T(35.0 / 16) * u[2],
                    T(1.0 / 16) * u[1] - T(5.0 / 16) * u[2] + T(5.0 / 16) * u[4],
                    T(-1.0 / 16) * u[2] + T(9.0 / 16) * u[4] - T(1.0 / 16) * u[5],
                    T(15.0 / 16) * u[4] - T(5.0 / 16) * u[5] + T(1.0 / 16) * u[6]};
    const T C[4] = {T(1.0 / 64), T(21.0 / 64), T(35.0 / 64), T(7.0 / 64)};
    if (linw) return C[0] * p[0] + C[1] * p[1] + C[2] * p[2] + C[3] * p[3];
    const T D[6] = {u[1] - u[0], u[2] - u[1], -u[2], u[4], u[5] - u[4], u[6] - u[5]};
    T b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) b[k] = is_b4(k, D[k], D[k + 1], D[k + 2], eps);
    if (wz) return weno_z_combine<T, 4>(b, fabs(b[0] + T(3) * b[1] - T(3) * b[2] - b[3]), C, p);
    T w[4];
    raw_weights<T, 4>(b, C, w);
    if (ppm) {
      // fourth-order mapping of the Appendix: g = C - (w - C)^4 / C^3 (w <= C),
      // C - (w - C)^4 / (C - 1)^3 (w > C)
      constexpr double c4[4] = {1.0 / 64, 21.0 / 64, 35.0 / 64, 7.0 / 64};
      T num = T(0), den = T(0);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const T q = w[k] - C[k], q2 = q * q;
        const T K = nonpos(q) ? T(1.0 / (c4[k] * c4[k] * c4[k]))
                              : T(1.0 / ((c4[k] - 1.0) * (c4[k] - 1.0) * (c4[k] - 1.0)));
        const T g = C[k] - q2 * q2 * K;
        num += g * p[k];
        den += g;
      }
      return quot(num, den);
    }
    return w[0] * p[0] + w[1] * p[1] + w[2] * p[2] + w[3] * p[3];
  } else if constexpr (R == 3) {
    const T e0 = fma(T(-2), u[1], u[0]), f0 = fma(T(-4), u[1], u[0]);
    const T e1 = u[3] + u[1], f1 = u[3] - u[1];
    const T e2 = fma(T(-2), u[3], u[4]), f2 = fma(T(-4), u[3], u[4]);
    const T P[3] = {fma(T(2), f0, e0), fma(T(2), f1, e1), fma(T(-2), f2, e2)};   // 8 p_k
    const T C[3] = {T(1.0 / 16), T(10.0 / 16), T(5.0 / 16)};
    if (linw) return fma(C[0], P[0], fma(C[1], P[1], C[2] * P[2]));
    const T eps4 = T(4) * eps;
    const T b[3] = {is_b4x(e0, f0, eps4), is_b4x(e1, f1, eps4), is_b4x(e2, f2, eps4)};
    if (wz) return weno_z_combine<T, 3>(b, fabs(b[0] - b[2]), C, P);
    T t[3], inv;
    raw_terms<T, 3>(b, C, t, inv);
    if (ppm) {
      // g = C + (w - C)^3 / C^2 (w <= C), C + (w - C)^3 / (C - 1)^2 (w > C)   [Eq. 3.23]
      const T K0[3] = {T(256.0), T(256.0 / 100), T(256.0 / 25)};          // 1 / C^2
      const T K1[3] = {T(256.0 / 225), T(256.0 / 36), T(256.0 / 121)};   // 1 / (C - 1)^2
      T num = T(0), den = T(0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const T q = fma(t[k], inv, -C[k]);                                  // w_k - C_k
        const T g = fma(q * q * q, nonpos(q) ? K0[k] : K1[k], C[k]);
        num = k == 0 ? g * P[0] : fma(g, P[k], num);
        den = k == 0 ? g : den + g;
      }
      return quot(num, den);
    }
    return (t[0] * P[0] + t[1] * P[1] + t[2] * P[2]) * inv;
  } else {
    const T e0 = fma(T(-2), u[1], u[0]), f0 = fma(T(-4), u[1], u[0]);
    const T e1 = u[3] + u[1], f1 = u[3] - u[1];
    const T P[2] = {f1 - e1, e1 + f1};                                      // 4 p_k
    const T C[2] = {T(0.25), T(0.75)};
    if (linw) return fma(C[0], P[0], C[1] * P[1]);
    const T eps4 = T(4) * eps;
    const T b[2] = {is_b4x(e0, f0, eps4), is_b4x(e1, f1, eps4)};
    if (wz) return weno_z_combine<T, 2>(b, fabs(b[0] - b[1]), C, P);
    T t[2], inv;
    raw_terms<T, 2>(b, C, t, inv);
    if (ppm) {
      // g = C - (w - C)^2 / C (w <= C), C - (w - C)^2 / (C - 1) (w > C)   [Eq. 3.15]
      const T K0[2] = {T(-4.0), T(-4.0 / 3)};        // -1 / C
      const T K1[2] = {T(4.0 / 3), T(4.0)};          // -1 / (C - 1)
      T num = T(0), den = T(0);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const T q = fma(t[k], inv, -C[k]);
        const T g = fma(q * q, nonpos(q) ? K0[k] : K1[k], C[k]);
        num = k == 0 ? g * P[0] : fma(g, P[k], num);
        den = k == 0 ? g : den + g;
      }
      return quot(num, den);
    }
    return (t[0] * P[0] + t[1] * P[1]) * inv;
  }
}

// --------------------------------------------------------------------------------------
// FP32 WENO on two characteristic components at once (Blackwell packed two-lane float
// arithmetic).  The same operations as weno_delta<R, float>, lane by lane: additions,
// multiplications and fused multiply-adds are packed; quotients, minima and the mapping's
// branch are taken per lane.
// --------------------------------------------------------------------------------------
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 quot2(float2 a, float2 b) {
  return mul2(a, make_float2(rcp_approx(b.x), rcp_approx(b.y)));
}
// K q with K = Kn for q <= 0 and Kp for q > 0, without a per-lane select: the smaller factor
// times q plus the difference times min(q, 0) or max(q, 0), so that the exact side is the one
// with the smaller factor and the correction never cancels more than one binary digit.
__device__ __forceinline__ float2 kq2(float Kn, float Kp, float2 q) {
  if (fabsf(Kn) >= fabsf(Kp))
    return fma2(bc2(Kn - Kp), make_float2(fminf(q.x, 0.0f), fminf(q.y, 0.0f)), mul2(bc2(Kp), q));
  return fma2(bc2(Kp - Kn), make_float2(fmaxf(q.x, 0.0f), fmaxf(q.y, 0.0f)), mul2(bc2(Kn), q));
}
__device__ __forceinline__ float2 is_b2(float2 e, float2 f, float2 eps) {
  return fma2(mul2(bc2(13.0f / 12), e), e, fma2(mul2(bc2(0.25f), f), f, eps));
}
// raw weights, ratio form C_k (b_min / b_k)^2 normalised (as raw_weights<float, K>)
template <int K>
__device__ __forceinline__ void raw_weights2(const float2* b, const float* C, float2* w) {
  float2 bmin = b[0];
#pragma unroll
  for (int k = 1; k < K; ++k) bmin = make_float2(fminf(bmin.x, b[k].x), fminf(bmin.y, b[k].y));
  float2 t[K], sum;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float2 r = quot2(bmin, b[k]);
    t[k] = mul2(mul2(bc2(C[k]), r), r);
    sum = k == 0 ? t[0] : add2(sum, t[k]);
  }
  const float2 inv = make_float2(rcp_approx(sum.x), rcp_approx(sum.y));
#pragma unroll
  for (int k = 0; k < K; ++k) w[k] = mul2(t[k], inv);
}

// raw terms of two lanes: t_k = C_k (b_min / b_k)^2 and the reciprocal of their sum
template <int K>
__device__ __forceinline__ void raw_terms2(const float2* b, const float* C, float2* t, float2& inv) {
  float2 bmin = b[0];
#pragma unroll
  for (int k = 1; k < K; ++k) bmin = make_float2(fminf(bmin.x, b[k].x), fminf(bmin.y, b[k].y));
  float2 sum;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float2 r = quot2(bmin, b[k]);
    t[k] = mul2(mul2(bc2(C[k]), r), r);
    sum = k == 0 ? t[0] : add2(sum, t[k]);
  }
  inv = make_float2(rcp_approx(sum.x), rcp_approx(sum.y));
}
__device__ __forceinline__ float2 is_b4x2(float2 e, float2 f, float2 eps4) {
  return fma2(mul2(bc2(13.0f / 3), e), e, fma2(f, f, eps4));
}

// NOSEL: the mapping's factor without per-lane selects (kq2), for r = 2 and 3; it saves issue
// slots in the float passes (FP32 marching xi 0.213 -> 0.210 ms) and costs the mixed eta pass
// registers (0.797 -> 0.822 ms), so the callers take it for the FP32 path only.
template <int R, bool NOSEL = false>
__device__ __forceinline__ float2 weno_delta_x2(const float2* u, float eps_, int ppm, int linw, int wz = 0) {
  const float2 eps = bc2(eps_);
  if constexpr (R == 4) {
    const float2 p[4] = {
        fma2(bc2(-5.0f / 16), u[0], fma2(bc2(21.0f / 16), u[1], mul2(bc2(-35.0f / 16), u[2]))),
        fma2(bc2(1.0f / 16), u[1], fma2(bc2(-5.0f / 16), u[2], mul2(bc2(5.0f / 16), u[4]))),
        fma2(bc2(-1.0f / 16), u[2], fma2(bc2(9.0f / 16), u[4], mul2(bc2(-1.0f / 16), u[5]))),
        fma2(bc2(15.0f / 16), u[4], fma2(bc2(-5.0f / 16), u[5], mul2(bc2(1.0f / 16), u[6])))};
    const float C[4] = {1.0f / 64, 21.0f / 64, 35.0f / 64, 7.0f / 64};
    if (linw)
      return fma2(bc2(C[0]), p[0], fma2(bc2(C[1]), p[1], fma2(bc2(C[2]), p[2], mul2(bc2(C[3]), p[3]))));
    const float2 m1 = bc2(-1.0f);
    const float2 D[6] = {fma2(u[0], m1, u[1]), fma2(u[1], m1, u[2]), mul2(u[2], m1), u[4], fma2(u[4], m1, u[5]),
                         fma2(u[5], m1, u[6])};
    float2 b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 d1 = D[k], d2 = D[k + 1], d3 = D[k + 2];
      const float2 r1 = fma2(bc2((float)is4c(k, 0)), d1, fma2(bc2((float)is4c(k, 3)), d2, mul2(bc2((float)is4c(k, 4)), d3)));
      const float2 r2 = fma2(bc2((float)is4c(k, 1)), d2, mul2(bc2((float)is4c(k, 5)), d3));
      b[k] = fma2(d1, r1, fma2(d2, r2, fma2(mul2(bc2((float)is4c(k, 2)), d3), d3, eps)));
    }
    if (wz) {
      float bx[4], by[4], px[4], py[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) { bx[k] = b[k].x; by[k] = b[k].y; px[k] = p[k].x; py[k] = p[k].y; }
      return make_float2(weno_z_combine<float, 4>(bx, fabsf(bx[0] + 3.f * bx[1] - 3.f * bx[2] - bx[3]), C, px),
                         weno_z_combine<float, 4>(by, fabsf(by[0] + 3.f * by[1] - 3.f * by[2] - by[3]), C, py));
    }
    float2 w[4];
    raw_weights2<4>(b, C, w);
    if (ppm) {
      // g = C - (w - C)^4 / C^3 (w <= C), C - (w - C)^4 / (C - 1)^3 (w > C)
      constexpr float K0[4] = {262144.0f, 262144.0f / 9261, 262144.0f / 42875, 262144.0f / 343};
      constexpr float K1[4] = {-262144.0f / 250047, -262144.0f / 79507, -262144.0f / 24389, -262144.0f / 185193};
      float2 num, den;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 q = add2(w[k], bc2(-C[k]));
        const float2 q2 = mul2(q, q);
        const float2 K = make_float2(nonpos(q.x) ? -K0[k] : -K1[k], nonpos(q.y) ? -K0[k] : -K1[k]);
        const float2 g = fma2(mul2(q2, q2), K, bc2(C[k]));
        num = k == 0 ? mul2(g, p[0]) : fma2(g, p[k], num);
        den = k == 0 ? g : add2(den, g);
      }
      return quot2(num, den);
    }
    return fma2(w[0], p[0], fma2(w[1], p[1], fma2(w[2], p[2], mul2(w[3], p[3]))));
  } else if constexpr (R == 3) {
    // the differences and candidates of weno_delta<3> (8 p_k), lane by lane
    const float2 m1 = bc2(-1.0f), m2 = bc2(-2.0f), m4 = bc2(-4.0f), two = bc2(2.0f);
    const float2 e0 = fma2(m2, u[1], u[0]), f0 = fma2(m4, u[1], u[0]);
    const float2 e1 = add2(u[3], u[1]), f1 = fma2(u[1], m1, u[3]);
    const float2 e2 = fma2(m2, u[3], u[4]), f2 = fma2(m4, u[3], u[4]);
    const float2 P[3] = {fma2(two, f0, e0), fma2(two, f1, e1), fma2(m2, f2, e2)};
    const float C[3] = {1.0f / 16, 10.0f / 16, 5.0f / 16};
    if (linw) return fma2(bc2(C[0]), P[0], fma2(bc2(C[1]), P[1], mul2(bc2(C[2]), P[2])));
    const float2 eps4 = bc2(4.0f * eps_);
    const float2 b[3] = {is_b4x2(e0, f0, eps4), is_b4x2(e1, f1, eps4), is_b4x2(e2, f2, eps4)};
    if (wz) {
      const float bx[3] = {b[0].x, b[1].x, b[2].x}, by[3] = {b[0].y, b[1].y, b[2].y};
      const float px[3] = {P[0].x, P[1].x, P[2].x}, py[3] = {P[0].y, P[1].y, P[2].y};
      return make_float2(weno_z_combine<float, 3>(bx, fabsf(bx[0] - bx[2]), C, px),
                         weno_z_combine<float, 3>(by, fabsf(by[0] - by[2]), C, py));
    }
    float2 t[3], inv;
    raw_terms2<3>(b, C, t, inv);
    if (ppm) {
      // g = C + (w - C)^3 / C^2 (w <= C), C + (w - C)^3 / (C - 1)^2 (w > C)   [Eq. 3.23]
      const float K0[3] = {256.0f, 256.0f / 100, 256.0f / 25}, K1[3] = {256.0f / 225, 256.0f / 36, 256.0f / 121};
      float2 num, den;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float2 q = fma2(t[k], inv, bc2(-C[k]));
        float2 g;
        if constexpr (NOSEL) {
          g = fma2(mul2(q, q), kq2(K0[k], K1[k], q), bc2(C[k]));
        } else {
          const float2 K = make_float2(nonpos(q.x) ? K0[k] : K1[k], nonpos(q.y) ? K0[k] : K1[k]);
          g = fma2(mul2(mul2(q, q), q), K, bc2(C[k]));
        }
        num = k == 0 ? mul2(g, P[0]) : fma2(g, P[k], num);
        den = k == 0 ? g : add2(den, g);
      }
      return quot2(num, den);
    }
    return mul2(fma2(t[0], P[0], fma2(t[1], P[1], mul2(t[2], P[2]))), inv);
  } else {
    const float2 m1 = bc2(-1.0f), m2 = bc2(-2.0f), m4 = bc2(-4.0f);
    const float2 e0 = fma2(m2, u[1], u[0]), f0 = fma2(m4, u[1], u[0]);
    const float2 e1 = add2(u[3], u[1]), f1 = fma2(u[1], m1, u[3]);
    const float2 P[2] = {fma2(e1, m1, f1), add2(e1, f1)};                  // 4 p_k
    const float C[2] = {0.25f, 0.75f};
    if (linw) return fma2(bc2(C[0]), P[0], mul2(bc2(C[1]), P[1]));
    const float2 eps4 = bc2(4.0f * eps_);
    const float2 b[2] = {is_b4x2(e0, f0, eps4), is_b4x2(e1, f1, eps4)};
    if (wz) {
      const float bx[2] = {b[0].x, b[1].x}, by[2] = {b[0].y, b[1].y};
      const float px[2] = {P[0].x, P[1].x}, py[2] = {P[0].y, P[1].y};
      return make_float2(weno_z_combine<float, 2>(bx, fabsf(bx[0] - bx[1]), C, px),
                         weno_z_combine<float, 2>(by, fabsf(by[0] - by[1]), C, py));
    }
    float2 t[2], inv;
    raw_terms2<2>(b, C, t, inv);
    if (ppm) {
      // g = C - (w - C)^2 / C (w <= C), C - (w - C)^2 / (C - 1) (w > C)   [Eq. 3.15]
      const float K0[2] = {-4.0f, -4.0f / 3}, K1[2] = {4.0f / 3, 4.0f};
      float2 num, den;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const float2 q = fma2(t[k], inv, bc2(-C[k]));
        float2 g;
        if constexpr (NOSEL) {
          g = fma2(q, kq2(K0[k], K1[k], q), bc2(C[k]));
        } else {
          const float2 K = make_float2(nonpos(q.x) ? K0[k] : K1[k], nonpos(q.y) ? K0[k] : K1[k]);
          g = fma2(mul2(q, q), K, bc2(C[k]));
        }
        num = k == 0 ? mul2(g, P[0]) : fma2(g, P[k], num);
        den = k == 0 ? g : add2(den, g);
      }
      return quot2(num, den);
    }
    return mul2(fma2(t[0], P[0], mul2(t[1], P[1])), inv);
  }
}

}  // namespace fsp
