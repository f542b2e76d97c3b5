// fsp_device.cuh -- device-side building blocks of the WENOIU right-hand side
// (Li & Sun, arXiv:1810.11103): scheme coefficients, boundary ghosts, Euler flux,
// characteristic projection and the mapped WENO interpolation.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fsp {

constexpr int G = 4;  // ghost layers of the stored metrics

enum { S31 = 0, S32 = 1, S51 = 2, S52 = 3 };
enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_DIRICHLET = 2, BC_SLIPWALL = 3, BC_FARFIELD = 4 };

// --------------------------------------------------------------------------------------
// Scheme coefficients (Section 3)
// --------------------------------------------------------------------------------------
template <int S> struct Scheme;
// WENOIU3-1MP, Eq. (3.4): h+ = f_{j+1/2} + (-f_{j-1} + 2 f_j - f_{j+1}) / 24
template <> struct Scheme<S31> {
  static constexpr int r = 2, nmp = 1;
  static constexpr double m0 = 1.0, m1 = 0.0;
  __host__ __device__ static constexpr double n(int k) {
    return k == 1 || k == 3 ? -1.0 / 24 : k == 2 ? 2.0 / 24 : 0.0;
  }
};
// WENOIU3-2MP, Eq. (3.8): h+ = f_{j+1/2} + (-f_{j-1/2} + 2 f_j - f_{j+1/2}) / 6
template <> struct Scheme<S32> {
  static constexpr int r = 2, nmp = 2;
  static constexpr double m0 = 5.0 / 6, m1 = -1.0 / 6;
  __host__ __device__ static constexpr double n(int k) { return k == 2 ? 2.0 / 6 : 0.0; }
};
// WENOIU5-1MP, Eq. (3.16)
template <> struct Scheme<S51> {
  static constexpr int r = 3, nmp = 1;
  static constexpr double m0 = 1.0, m1 = 0.0;
  __host__ __device__ static constexpr double n(int k) {
    return k == 0 ? 19.0 / 1920 : k == 1 ? -29.0 / 480 : k == 2 ? 77.0 / 960 : k == 3 ? -3.0 / 160 : -7.0 / 640;
  }
};
// WENOIU5-2MP, Eq. (3.20): h+ = f_{j+1/2} + [(-4 f_{j+1} + f_j + f_{j-1}) + (6 f_{j+1/2}
// - 4 f_{j-1/2})] / 30
template <> struct Scheme<S52> {
  static constexpr int r = 3, nmp = 2;
  static constexpr double m0 = 36.0 / 30, m1 = -4.0 / 30;
  __host__ __device__ static constexpr double n(int k) {
    return k == 1 || k == 2 ? 1.0 / 30 : k == 3 ? -4.0 / 30 : 0.0;
  }
};

// n(k): h+ coefficient of f+_{j+k-2}, k = 0..4 (node offsets -2..2).

// Central operator delta^{c,(1)} of each scheme (Eq. 2.7), used for the metrics:
//   D f_j = sum_k a_k (f_{j+k} - f_{j-k}) + b_{1/2}(f~_{j+1/2} - f~_{j-1/2})
//           + b_{3/2}(f~_{j+3/2} - f~_{j-3/2})
struct Central { double a1, a2, a3, b12, b32; };
__host__ __device__ inline Central central_of(int scheme) {
  switch (scheme) {
    case S31: return {2.0 / 48, -1.0 / 48, 0.0, 1.0, 0.0};              // Eq. (3.7)
    case S32: return {2.0 / 12, 0.0, 0.0, 11.0 / 12, -1.0 / 12};        // Eq. (3.9)
    case S51: return {17.0 / 256, -13.0 / 320, 19.0 / 3840, 1.0, 0.0};  // Eq. (3.19)
    default:  return {-4.0 / 60, 1.0 / 60, 0.0, 19.0 / 15, -1.0 / 15};  // Eq. (3.21)
  }
}

// Midpoint value at j+1/2 from nodal values v[k] = f_{j+k-2}, k = 0..5 (f_{j-2}..f_{j+3}).
// interp 1: two-point average; else Lagrange with 4 (third-order schemes) or 6 points.
template <typename T>
__device__ __forceinline__ T mid_interp(int interp, bool sixth, const T* v) {
  if (interp == 1) return T(0.5) * (v[2] + v[3]);
  if (!sixth) return (T(9) * (v[2] + v[3]) - (v[1] + v[4])) * T(1.0 / 16);
  return (T(150) * (v[2] + v[3]) - T(25) * (v[1] + v[4]) + T(3) * (v[0] + v[5])) * T(1.0 / 256);
}

// --------------------------------------------------------------------------------------
// Kernel parameters (plain data, passed by value)
// --------------------------------------------------------------------------------------
struct Params {
  int ni, nj;
  long long ld;             // row stride of Q-shaped arrays
  int bc[4];
  int interp, ppm, linw;
  double gamma, alpha, eps;
  double bcq[4][4];
  const double* met;        // haloed metrics
  long long mld;            // ni + 2G
  long long mplane;         // (ni + 2G) (nj + 2G)
};

__device__ __forceinline__ double met_at(const Params& P, int p, int i, int j) {
  return __ldg(P.met + p * P.mplane + (long long)(j + G) * P.mld + (i + G));
}

__device__ __forceinline__ int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// Ghost state along direction dir for the line `line` (row j for dir 0, column i for
// dir 1) at position g (any integer; interior when 0 <= g < n).
template <typename Real>
__device__ __forceinline__ void load_state(const Params& P, const Real* __restrict__ Q, int dir,
                                           int line, int g, Real q[4]) {
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

// Metric-weighted Euler flux E^ = mx E + my F (Eq. 2.2 in 2-D).
template <typename Real>
__device__ __forceinline__ void euler_flux(const Real q[4], Real mx, Real my, Real gm1, Real f[4]) {
  const Real rinv = Real(1) / q[0];
  const Real u = q[1] * rinv, v = q[2] * rinv;
  const Real p = gm1 * (q[3] - Real(0.5) * (q[1] * u + q[2] * v));
  const Real U = mx * u + my * v;
  f[0] = q[0] * U;
  f[1] = q[1] * U + mx * p;
  f[2] = q[2] * U + my * p;
  f[3] = (q[3] + p) * U;
}

// |U^| + c |k^| (the quantity maximised along a line for A^, Section 2.3)
template <typename Real>
__device__ __forceinline__ Real spectral_radius(const Real q[4], Real mx, Real my, Real gamma) {
  const Real rinv = Real(1) / q[0];
  const Real u = q[1] * rinv, v = q[2] * rinv;
  const Real p = (gamma - Real(1)) * (q[3] - Real(0.5) * (q[1] * u + q[2] * v));
  const Real c = sqrt(gamma * p * rinv);
  return fabs(mx * u + my * v) + c * sqrt(mx * mx + my * my);
}

// --------------------------------------------------------------------------------------
// Characteristic projection (Section 3.4): left eigenvector rows at a state q along the
// unit direction (nx, ny); R is applied in factored form in recon().
// --------------------------------------------------------------------------------------
template <typename Real>
struct Eig {
  Real L[4][4];
  Real u, v, c, H, Un, Ut, nx, ny, h2;  // h2 = |u|^2 / 2

  __device__ __forceinline__ void build(const Real q[4], Real nx_, Real ny_, Real gamma) {
    nx = nx_; ny = ny_;
    const Real rinv = Real(1) / q[0];
    u = q[1] * rinv; v = q[2] * rinv;
    h2 = Real(0.5) * (u * u + v * v);
    const Real gm1 = gamma - Real(1);
    const Real p = gm1 * (q[3] - q[0] * h2);
    const Real c2 = gamma * p * rinv;
    c = sqrt(c2);
    const Real cinv = Real(1) / c;
    H = (q[3] + p) * rinv;
    Un = u * nx + v * ny;
    Ut = v * nx - u * ny;
    const Real b1 = gm1 * cinv * cinv;
    const Real b2 = b1 * h2;
    const Real hb1 = Real(0.5) * b1, hb2 = Real(0.5) * b2;
    const Real hUc = Real(0.5) * Un * cinv, hnxc = Real(0.5) * nx * cinv, hnyc = Real(0.5) * ny * cinv;
    L[0][0] = hb2 + hUc; L[0][1] = -hb1 * u - hnxc; L[0][2] = -hb1 * v - hnyc; L[0][3] = hb1;
    L[1][0] = Real(1) - b2; L[1][1] = b1 * u; L[1][2] = b1 * v; L[1][3] = -b1;
    L[2][0] = -Ut; L[2][1] = -ny; L[2][2] = nx; L[2][3] = Real(0);
    L[3][0] = hb2 - hUc; L[3][1] = -hb1 * u + hnxc; L[3][2] = -hb1 * v + hnyc; L[3][3] = hb1;
  }
  // Q = R W with R's columns (1, u - c nx, v - c ny, H - c Un), (1, u, v, |u|^2/2),
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
// WENO interpolation to x_{j+1/2} (Eqs. 3.10-3.13, Table 1) with the indicators of
// Eq. (3.22) (written on consecutive differences; for r = 2 the three-point IS_0, IS_1 of
// Section 5.1) and the mapping of Eq. (3.15) (r = 2) or (3.23) (r = 3).
// u[0..4] = u_{j-2} .. u_{j+2}.  The weights are formed with one reciprocal:
// omega_k = C_k prod_{l != k} b_l^2 / sum_m C_m prod_{l != m} b_l^2, b = eps + IS;
// the mapped weights g_k are normalised in the final quotient sum g p / sum g.
// --------------------------------------------------------------------------------------
template <int R>
__device__ __forceinline__ double weno_mid(const double* u, double eps, int ppm, int linw) {
  if constexpr (R == 3) {
    const double p0 = 0.375 * u[0] - 1.25 * u[1] + 1.875 * u[2];
    const double p1 = -0.125 * u[1] + 0.75 * u[2] + 0.375 * u[3];
    const double p2 = 0.375 * u[2] + 0.75 * u[3] - 0.125 * u[4];
    constexpr double C0 = 1.0 / 16, C1 = 10.0 / 16, C2 = 5.0 / 16;
    if (linw) return C0 * p0 + C1 * p1 + C2 * p2;
    const double d1 = u[1] - u[0], d2 = u[2] - u[1], d3 = u[3] - u[2], d4 = u[4] - u[3];
    const double e0 = d2 - d1, e1 = d3 - d2, e2 = d4 - d3;
    const double f0 = 3.0 * d2 - d1, f1 = d2 + d3, f2 = d4 - 3.0 * d3;
    const double b0 = eps + (13.0 / 12) * e0 * e0 + 0.25 * f0 * f0;
    const double b1 = eps + (13.0 / 12) * e1 * e1 + 0.25 * f1 * f1;
    const double b2 = eps + (13.0 / 12) * e2 * e2 + 0.25 * f2 * f2;
    const double s0 = b0 * b0, s1 = b1 * b1, s2 = b2 * b2;
    const double t0 = C0 * s1 * s2, t1 = C1 * s0 * s2, t2 = C2 * s0 * s1;
    const double inv = 1.0 / (t0 + t1 + t2);
    double w0 = t0 * inv, w1 = t1 * inv, w2 = t2 * inv;
    if (ppm) {
      // g = C + (w - C)^3 / C^2 (w <= C), C + (w - C)^3 / (C - 1)^2 (w > C)   [Eq. 3.23]
      const double q0 = w0 - C0, q1 = w1 - C1, q2 = w2 - C2;
      const double k0 = q0 <= 0.0 ? 1.0 / (C0 * C0) : 1.0 / ((C0 - 1) * (C0 - 1));
      const double k1 = q1 <= 0.0 ? 1.0 / (C1 * C1) : 1.0 / ((C1 - 1) * (C1 - 1));
      const double k2 = q2 <= 0.0 ? 1.0 / (C2 * C2) : 1.0 / ((C2 - 1) * (C2 - 1));
      w0 = C0 + q0 * q0 * q0 * k0;
      w1 = C1 + q1 * q1 * q1 * k1;
      w2 = C2 + q2 * q2 * q2 * k2;
      return (w0 * p0 + w1 * p1 + w2 * p2) / (w0 + w1 + w2);
    }
    return w0 * p0 + w1 * p1 + w2 * p2;
  } else {
    const double p0 = -0.5 * u[1] + 1.5 * u[2];
    const double p1 = 0.5 * u[2] + 0.5 * u[3];
    constexpr double C0 = 0.25, C1 = 0.75;
    if (linw) return C0 * p0 + C1 * p1;
    const double d1 = u[1] - u[0], d2 = u[2] - u[1], d3 = u[3] - u[2];
    const double e0 = d2 - d1, e1 = d3 - d2;
    const double f0 = 3.0 * d2 - d1, f1 = d2 + d3;
    const double b0 = eps + (13.0 / 12) * e0 * e0 + 0.25 * f0 * f0;
    const double b1 = eps + (13.0 / 12) * e1 * e1 + 0.25 * f1 * f1;
    const double s0 = b0 * b0, s1 = b1 * b1;
    const double t0 = C0 * s1, t1 = C1 * s0;
    const double inv = 1.0 / (t0 + t1);
    double w0 = t0 * inv, w1 = t1 * inv;
    if (ppm) {
      // g = C - (w - C)^2 / C (w <= C), C - (w - C)^2 / (C - 1) (w > C)   [Eq. 3.15]
      const double q0 = w0 - C0, q1 = w1 - C1;
      const double k0 = q0 <= 0.0 ? 1.0 / C0 : 1.0 / (C0 - 1);
      const double k1 = q1 <= 0.0 ? 1.0 / C1 : 1.0 / (C1 - 1);
      w0 = C0 - q0 * q0 * k0;
      w1 = C1 - q1 * q1 * k1;
      return (w0 * p0 + w1 * p1) / (w0 + w1);
    }
    return w0 * p0 + w1 * p1;
  }
}

}  // namespace fsp
