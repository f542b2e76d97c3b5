// adjoint_device.cuh -- reverse-mode (vector-Jacobian) building blocks of the WENOIU
// right-hand side, FP64.  Each routine takes the forward inputs, recomputes what it needs,
// and adds the adjoints of its inputs given the adjoint of its output ("bar" quantities).
#pragma once

#include "fsp_device.cuh"

namespace fsp {

// ---- WENO with a tape: the forward pass keeps what the reverse pass needs -------------
// One component's tape, WT slots in shared memory, slot i at p[i * stride].  r = 2, 3: the
// stencil differences u (4: offsets -2, -1, +1, +2), b = eps + IS_k (3), the raw weights (3),
// 1 / sum of the unnormalised weights, 1 / sum of the mapped weights, the interpolant.
// r = 4: u (6: offsets -3..-1, +1..+3), b (4), the weights (4), 1 / sum of the mapped
// weights, the interpolant.
constexpr int WT = 16;

struct Tape {
  double* p;
  int stride;
  __device__ __forceinline__ double& operator[](int i) const { return p[i * stride]; }
};

// Same arithmetic as weno_delta<R, double>, except that the mapped quotient is formed as
// num * (1/den) so that the reverse pass reuses the reciprocal.
template <int R>
__device__ __forceinline__ double weno_fwd_tape(const double* u, double eps, int ppm, int linw, Tape t) {
  if constexpr (R == 4) {
    // u[m + 3] = w_{j+m} - w_j, m = -3..3 (u[3] is not read): Table A1 candidates, the r = 4
    // indicators, C_k / b_k^2 weights and the fourth-order mapping, as weno_delta<4>
    t[0] = u[0]; t[1] = u[1]; t[2] = u[2]; t[3] = u[4]; t[4] = u[5]; t[5] = u[6];
    const double p[4] = {-5.0 / 16 * u[0] + 21.0 / 16 * u[1] - 35.0 / 16 * u[2],
                         1.0 / 16 * u[1] - 5.0 / 16 * u[2] + 5.0 / 16 * u[4],
                         -1.0 / 16 * u[2] + 9.0 / 16 * u[4] - 1.0 / 16 * u[5],
                         15.0 / 16 * u[4] - 5.0 / 16 * u[5] + 1.0 / 16 * u[6]};
    const double C[4] = {1.0 / 64, 21.0 / 64, 35.0 / 64, 7.0 / 64};
    if (linw) return C[0] * p[0] + C[1] * p[1] + C[2] * p[2] + C[3] * p[3];
    const double D[6] = {u[1] - u[0], u[2] - u[1], -u[2], u[4], u[5] - u[4], u[6] - u[5]};
    double b[4], a[4], sa = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      b[k] = is_b4(k, D[k], D[k + 1], D[k + 2], eps);
      a[k] = C[k] * rcp_nr(b[k] * b[k]);
      sa += a[k];
    }
    const double isa = rcp_nr(sa);
    double w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      w[k] = a[k] * isa;
      t[6 + k] = b[k];
      t[10 + k] = w[k];
    }
    double out;
    if (ppm) {
      double num = 0.0, den = 0.0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double q = w[k] - C[k], q2 = q * q;
        const double K = nonpos(q) ? 1.0 / (C[k] * C[k] * C[k]) : 1.0 / ((C[k] - 1.0) * (C[k] - 1.0) * (C[k] - 1.0));
        const double g = C[k] - q2 * q2 * K;
        num += g * p[k];
        den += g;
      }
      const double rden = rcp_nr(den);
      out = num * rden;
      t[14] = rden;
    } else {
      out = w[0] * p[0] + w[1] * p[1] + w[2] * p[2] + w[3] * p[3];
    }
    t[15] = out;
    return out;
  } else {
  t[0] = u[0]; t[1] = u[1]; t[2] = u[3]; t[3] = u[4];
  if constexpr (R == 3) {
    const double p0 = 0.375 * u[0] - 1.25 * u[1];
    const double p1 = -0.125 * u[1] + 0.375 * u[3];
    const double p2 = 0.75 * u[3] - 0.125 * u[4];
    const double C[3] = {1.0 / 16, 10.0 / 16, 5.0 / 16};
    if (linw) return C[0] * p0 + C[1] * p1 + C[2] * p2;
    const double d1 = u[1] - u[0], d2 = -u[1], d3 = u[3], d4 = u[4] - u[3];
    const double b[3] = {is_b(d2 - d1, 3.0 * d2 - d1, eps), is_b(d3 - d2, d2 + d3, eps),
                         is_b(d4 - d3, d4 - 3.0 * d3, eps)};
    const double s[3] = {b[0] * b[0], b[1] * b[1], b[2] * b[2]};
    const double tt[3] = {C[0] * (s[1] * s[2]), C[1] * (s[0] * s[2]), C[2] * (s[0] * s[1])};
    const double iS = rcp_nr(tt[0] + tt[1] + tt[2]);
    const double w[3] = {tt[0] * iS, tt[1] * iS, tt[2] * iS};
    t[4] = b[0]; t[5] = b[1]; t[6] = b[2]; t[7] = w[0]; t[8] = w[1]; t[9] = w[2]; t[10] = iS;
    const double p[3] = {p0, p1, p2};
    double out;
    if (ppm) {
      const double K0[3] = {256.0, 256.0 / 100, 256.0 / 25}, K1[3] = {256.0 / 225, 256.0 / 36, 256.0 / 121};
      double num = 0.0, den = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double q = w[k] - C[k];
        const double g = C[k] + q * q * q * (nonpos(q) ? K0[k] : K1[k]);
        num += g * p[k];
        den += g;
      }
      const double rden = rcp_nr(den);
      out = num * rden;
      t[11] = rden;
    } else {
      out = w[0] * p0 + w[1] * p1 + w[2] * p2;
    }
    t[12] = out;
    return out;
  } else {
    const double p0 = -0.5 * u[1], p1 = 0.5 * u[3];
    const double C[2] = {0.25, 0.75};
    if (linw) return C[0] * p0 + C[1] * p1;
    const double d1 = u[1] - u[0], d2 = -u[1], d3 = u[3];
    const double b[2] = {is_b(d2 - d1, 3.0 * d2 - d1, eps), is_b(d3 - d2, d2 + d3, eps)};
    const double tt[2] = {C[0] * (b[1] * b[1]), C[1] * (b[0] * b[0])};
    const double iS = rcp_nr(tt[0] + tt[1]);
    const double w[2] = {tt[0] * iS, tt[1] * iS};
    t[4] = b[0]; t[5] = b[1]; t[7] = w[0]; t[8] = w[1]; t[10] = iS;
    const double p[2] = {p0, p1};
    double out;
    if (ppm) {
      const double K0[2] = {4.0, 4.0 / 3}, K1[2] = {-4.0 / 3, -4.0};
      double num = 0.0, den = 0.0;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const double q = w[k] - C[k];
        const double g = C[k] - q * q * (nonpos(q) ? K0[k] : K1[k]);
        num += g * p[k];
        den += g;
      }
      const double rden = rcp_nr(den);
      out = num * rden;
      t[11] = rden;
    } else {
      out = w[0] * p0 + w[1] * p1;
    }
    t[12] = out;
    return out;
  }
  }
}

// Reverse of weno_fwd_tape: adds d(out)/du * obar to ub[0], ub[1], ub[3], ub[4] (r = 2, 3;
// the layout of weno_delta_bwd) or ub[0..6] except ub[3] (r = 4), reading the forward values
// from the tape.
template <int R>
__device__ __forceinline__ void weno_bwd_tape(Tape t, int ppm, int linw, double obar, double* ub) {
  if constexpr (R == 4) {
    const double u[7] = {t[0], t[1], t[2], 0.0, t[3], t[4], t[5]};
    const double C[4] = {1.0 / 64, 21.0 / 64, 35.0 / 64, 7.0 / 64};
    double pb[4], Db[6] = {0, 0, 0, 0, 0, 0};
    if (linw) {
#pragma unroll
      for (int k = 0; k < 4; ++k) pb[k] = obar * C[k];
    } else {
      const double p[4] = {-5.0 / 16 * u[0] + 21.0 / 16 * u[1] - 35.0 / 16 * u[2],
                           1.0 / 16 * u[1] - 5.0 / 16 * u[2] + 5.0 / 16 * u[4],
                           -1.0 / 16 * u[2] + 9.0 / 16 * u[4] - 1.0 / 16 * u[5],
                           15.0 / 16 * u[4] - 5.0 / 16 * u[5] + 1.0 / 16 * u[6]};
      const double b[4] = {t[6], t[7], t[8], t[9]}, w[4] = {t[10], t[11], t[12], t[13]};
      double wb[4];
      if (ppm) {
        const double rden = t[14];
        const double numb = obar * rden, denb = -obar * t[15] * rden;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const double q = w[k] - C[k];
          const double K = nonpos(q) ? 1.0 / (C[k] * C[k] * C[k]) : 1.0 / ((C[k] - 1.0) * (C[k] - 1.0) * (C[k] - 1.0));
          const double g = C[k] - q * q * q * q * K;
          pb[k] = numb * g;
          wb[k] = (numb * p[k] + denb) * (-4.0 * q * q * q * K);   // dg/dw = -4 (w - C)^3 K
        }
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) { wb[k] = obar * p[k]; pb[k] = obar * w[k]; }
      }
      // w_k = a_k / sum a, a_k = C_k b_k^-2: d w_k / d b_j = -2 w_j (delta_kj - w_k) / b_j
      const double dotw = wb[0] * w[0] + wb[1] * w[1] + wb[2] * w[2] + wb[3] * w[3];
      const double D[6] = {u[1] - u[0], u[2] - u[1], -u[2], u[4], u[5] - u[4], u[6] - u[5]};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double bb = -2.0 * w[k] * (wb[k] - dotw) * rcp_nr(b[k]);
        // b_k = eps + c0 d1^2 + c1 d2^2 + c2 d3^2 + c3 d1 d2 + c4 d1 d3 + c5 d2 d3
        const double d1 = D[k], d2 = D[k + 1], d3 = D[k + 2];
        Db[k] += bb * (2.0 * is4c(k, 0) * d1 + is4c(k, 3) * d2 + is4c(k, 4) * d3);
        Db[k + 1] += bb * (is4c(k, 3) * d1 + 2.0 * is4c(k, 1) * d2 + is4c(k, 5) * d3);
        Db[k + 2] += bb * (is4c(k, 4) * d1 + is4c(k, 5) * d2 + 2.0 * is4c(k, 2) * d3);
      }
    }
    // candidates and the consecutive differences D, back to u
    ub[0] += -5.0 / 16 * pb[0] - Db[0];
    ub[1] += 21.0 / 16 * pb[0] + 1.0 / 16 * pb[1] + Db[0] - Db[1];
    ub[2] += -35.0 / 16 * pb[0] - 5.0 / 16 * pb[1] - 1.0 / 16 * pb[2] + Db[1] - Db[2];
    ub[4] += 5.0 / 16 * pb[1] + 9.0 / 16 * pb[2] + 15.0 / 16 * pb[3] + Db[3] - Db[4];
    ub[5] += -1.0 / 16 * pb[2] - 5.0 / 16 * pb[3] + Db[4] - Db[5];
    ub[6] += 1.0 / 16 * pb[3] + Db[5];
    return;
  } else {
  const double u0 = t[0], u1 = t[1], u3 = t[2], u4 = t[3];
  if constexpr (R == 3) {
    const double C[3] = {1.0 / 16, 10.0 / 16, 5.0 / 16};
    double pb[3];
    double eb[3] = {0, 0, 0}, fb[3] = {0, 0, 0};
    if (linw) {
#pragma unroll
      for (int k = 0; k < 3; ++k) pb[k] = obar * C[k];
    } else {
      const double p[3] = {0.375 * u0 - 1.25 * u1, -0.125 * u1 + 0.375 * u3, 0.75 * u3 - 0.125 * u4};
      const double b[3] = {t[4], t[5], t[6]};
      const double w[3] = {t[7], t[8], t[9]};
      const double iS = t[10];
      double wb[3];
      if (ppm) {
        const double K0[3] = {256.0, 256.0 / 100, 256.0 / 25}, K1[3] = {256.0 / 225, 256.0 / 36, 256.0 / 121};
        const double rden = t[11];
        const double numb = obar * rden, denb = -obar * t[12] * rden;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const double q = w[k] - C[k];
          const double K = nonpos(q) ? K0[k] : K1[k];
          const double q2K = q * q * K;
          const double g = C[k] + q2K * q;
          const double gb = numb * p[k] + denb;
          pb[k] = numb * g;
          wb[k] = gb * 3.0 * q2K;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) { wb[k] = obar * p[k]; pb[k] = obar * w[k]; }
      }
      const double dotw = wb[0] * w[0] + wb[1] * w[1] + wb[2] * w[2];
      const double tb[3] = {(wb[0] - dotw) * iS * C[0], (wb[1] - dotw) * iS * C[1], (wb[2] - dotw) * iS * C[2]};
      const double s[3] = {b[0] * b[0], b[1] * b[1], b[2] * b[2]};
      const double sb[3] = {tb[1] * s[2] + tb[2] * s[1], tb[0] * s[2] + tb[2] * s[0], tb[0] * s[1] + tb[1] * s[0]};
      const double d1 = u1 - u0, d2 = -u1, d3 = u3, d4 = u4 - u3;
      const double e[3] = {d2 - d1, d3 - d2, d4 - d3};
      const double f[3] = {3.0 * d2 - d1, d2 + d3, d4 - 3.0 * d3};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double bb = sb[k] * 2.0 * b[k];
        eb[k] = bb * (2.0 * 13.0 / 12) * e[k];
        fb[k] = bb * 0.5 * f[k];
      }
    }
    const double d1b = -eb[0] - fb[0];
    const double d2b = eb[0] + 3.0 * fb[0] - eb[1] + fb[1];
    const double d3b = eb[1] + fb[1] - eb[2] - 3.0 * fb[2];
    const double d4b = eb[2] + fb[2];
    ub[0] += 0.375 * pb[0] - d1b;
    ub[1] += -1.25 * pb[0] - 0.125 * pb[1] + d1b - d2b;
    ub[3] += 0.375 * pb[1] + 0.75 * pb[2] + d3b - d4b;
    ub[4] += -0.125 * pb[2] + d4b;
  } else {
    const double C[2] = {0.25, 0.75};
    double pb[2];
    double eb[2] = {0, 0}, fb[2] = {0, 0};
    if (linw) {
      pb[0] = obar * C[0];
      pb[1] = obar * C[1];
    } else {
      const double p[2] = {-0.5 * u1, 0.5 * u3};
      const double b[2] = {t[4], t[5]};
      const double w[2] = {t[7], t[8]};
      const double iS = t[10];
      double wb[2];
      if (ppm) {
        const double K0[2] = {4.0, 4.0 / 3}, K1[2] = {-4.0 / 3, -4.0};
        const double rden = t[11];
        const double numb = obar * rden, denb = -obar * t[12] * rden;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const double q = w[k] - C[k];
          const double K = nonpos(q) ? K0[k] : K1[k];
          const double g = C[k] - q * q * K;
          const double gb = numb * p[k] + denb;
          pb[k] = numb * g;
          wb[k] = -gb * 2.0 * q * K;
        }
      } else {
        for (int k = 0; k < 2; ++k) { wb[k] = obar * p[k]; pb[k] = obar * w[k]; }
      }
      const double dotw = wb[0] * w[0] + wb[1] * w[1];
      const double sb[2] = {(wb[1] - dotw) * iS * C[1], (wb[0] - dotw) * iS * C[0]};
      const double d1 = u1 - u0, d2 = -u1, d3 = u3;
      const double e[2] = {d2 - d1, d3 - d2};
      const double f[2] = {3.0 * d2 - d1, d2 + d3};
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const double bb = sb[k] * 2.0 * b[k];
        eb[k] = bb * (2.0 * 13.0 / 12) * e[k];
        fb[k] = bb * 0.5 * f[k];
      }
    }
    const double d1b = -eb[0] - fb[0];
    const double d2b = eb[0] + 3.0 * fb[0] - eb[1] + fb[1];
    const double d3b = eb[1] + fb[1];
    ub[0] += -d1b;
    ub[1] += -0.5 * pb[0] + d1b - d2b;
    ub[3] += 0.5 * pb[1] + d3b;
  }
  }
}

// ---- node primitives (prim_of), reverse: adds to qb[] from the primitives' adjoints ----
struct PrimBar { double u, v, c, cinv, H, b1, h2; };

__device__ __forceinline__ void prim_bwd(const double q[4], double gamma, PrimBar pb, double* qb) {
  const double gm1 = gamma - 1.0;
  const double rinv = rcp_nr(q[0]);
  const double u = q[1] * rinv, v = q[2] * rinv;
  const double h2 = 0.5 * (u * u + v * v);
  const double p = gm1 * (q[3] - q[0] * h2);
  const double c2 = gamma * p * rinv;
  const double cinv = rsq(c2);
  // b1 = gm1 cinv^2
  pb.cinv += 2.0 * gm1 * cinv * pb.b1;
  // H = (q3 + p) rinv
  double rb = (q[3] + p) * pb.H;
  double q3b = rinv * pb.H, pbar = rinv * pb.H;
  // c = c2 cinv, cinv = c2^(-1/2)
  double c2b = cinv * pb.c;
  pb.cinv += c2 * pb.c;
  c2b += -0.5 * cinv * cinv * cinv * pb.cinv;
  // c2 = gamma p rinv
  pbar += gamma * rinv * c2b;
  rb += gamma * p * c2b;
  // p = gm1 (q3 - q0 h2)
  q3b += gm1 * pbar;
  double q0b = -gm1 * h2 * pbar;
  pb.h2 += -gm1 * q[0] * pbar;
  // h2 = (u^2 + v^2) / 2
  pb.u += u * pb.h2;
  pb.v += v * pb.h2;
  // u = q1 rinv, v = q2 rinv
  qb[1] += rinv * pb.u;
  qb[2] += rinv * pb.v;
  rb += q[1] * pb.u + q[2] * pb.v;
  q0b += -rinv * rinv * rb;
  qb[0] += q0b;
  qb[3] += q3b;
}

// ---- metric-weighted Euler flux E^(q; mx, my), reverse -------------------------------
__device__ __forceinline__ void flux_bwd(const double q[4], double mx, double my, double gm1, const double* fb,
                                         double* qb, double& mxb, double& myb) {
  const double rinv = rcp_nr(q[0]);
  const double u = q[1] * rinv, v = q[2] * rinv;
  const double p = gm1 * (q[3] - 0.5 * (q[1] * u + q[2] * v));
  const double U = mx * u + my * v;
  // f0 = q0 U, f1 = q1 U + mx p, f2 = q2 U + my p, f3 = (q3 + p) U
  const double Ub = q[0] * fb[0] + q[1] * fb[1] + q[2] * fb[2] + (q[3] + p) * fb[3];
  double q0b = U * fb[0];
  double q1b = U * fb[1], q2b = U * fb[2], q3b = U * fb[3];
  const double pbar = mx * fb[1] + my * fb[2] + U * fb[3];
  mxb += p * fb[1] + u * Ub;
  myb += p * fb[2] + v * Ub;
  double ub = mx * Ub, vb = my * Ub;
  // p = gm1 (q3 - (q1 u + q2 v) / 2)
  q3b += gm1 * pbar;
  q1b += -0.5 * gm1 * u * pbar;
  q2b += -0.5 * gm1 * v * pbar;
  ub += -0.5 * gm1 * q[1] * pbar;
  vb += -0.5 * gm1 * q[2] * pbar;
  // u = q1 rinv, v = q2 rinv, rinv = 1 / q0
  q1b += rinv * ub;
  q2b += rinv * vb;
  const double rb = q[1] * ub + q[2] * vb;
  q0b += -rinv * rinv * rb;
  qb[0] += q0b; qb[1] += q1b; qb[2] += q2b; qb[3] += q3b;
}

// ---- |U^| + c |k^|, reverse (|x| has derivative +1 at 0, as in the oracle) -------------
__device__ __forceinline__ void spectral_bwd(const double q[4], double mx, double my, double gamma, double sb,
                                             double* qb, double& mxb, double& myb) {
  const double rinv = rcp_nr(q[0]);
  const double u = q[1] * rinv, v = q[2] * rinv;
  const double h = 0.5 * (q[1] * u + q[2] * v);
  const double p = (gamma - 1.0) * (q[3] - h);
  const double c = sqrt(gamma * p * rinv);
  const double km = sqrt(mx * mx + my * my);
  const double U = mx * u + my * v;
  const double sg = U >= 0.0 ? 1.0 : -1.0;
  double ub = sg * mx * sb, vb = sg * my * sb;
  mxb += sg * u * sb + c * mx / km * sb;
  myb += sg * v * sb + c * my / km * sb;
  const double cb = km * sb;
  // c = sqrt(gamma p rinv)
  const double c2b = cb * 0.5 / c;
  const double pb = gamma * rinv * c2b;
  double rb = gamma * p * c2b;
  // p = (gamma-1)(q3 - (q1 u + q2 v)/2)
  const double gm1 = gamma - 1.0;
  qb[3] += gm1 * pb;
  double q1b = -0.5 * gm1 * u * pb, q2b = -0.5 * gm1 * v * pb;
  ub += -0.5 * gm1 * q[1] * pb;
  vb += -0.5 * gm1 * q[2] * pb;
  q1b += rinv * ub;
  q2b += rinv * vb;
  rb += q[1] * ub + q[2] * vb;
  qb[0] += -rinv * rinv * rb;
  qb[1] += q1b;
  qb[2] += q2b;
}

// ---- one side of the characteristic WENO interpolation, reverse (taped) ---------------
// Forward: Q^s = Q_c + R W, W_k = WENO(L_k dQ_m) with L, R at the centre's primitives w
// and the unit direction (nx, ny); E, W and the WENO tapes (one per characteristic
// component) come from that forward pass.  Given Qsb (adjoint of Q^s), adds the adjoints
// of the centre state (qcb), of the stencil differences (dqb[a][4], a = offsets -2, -1,
// +1, +2, or -3..-1, +1..+3 for r = 4), of the primitives (pbar) and of the direction (nxb,
// nyb).
template <int R>
__device__ __forceinline__ void side_bwd_tape(const Eig<double>& E, const Prim<double>& w, double nx, double ny,
                                              const double (*dq)[4], const double W[4], int ppm, int linw,
                                              const Tape* tape, const double* Qsb, double* qcb, double (*dqb)[4],
                                              PrimBar& pbar, double& nxb, double& nyb) {
  // Q^s = Q_c + dQ
#pragma unroll
  for (int v = 0; v < 4; ++v) qcb[v] += Qsb[v];
  // recon: s = W0 + W3, d = W3 - W0, a = s + W1; dQ = (a, u a + c nx d - ny W2,
  // v a + c ny d + nx W2, H s + c Un d + h2 W1 + Ut W2)
  const double s = W[0] + W[3], d = W[3] - W[0], a = s + W[1];
  const double b0 = Qsb[0], b1 = Qsb[1], b2 = Qsb[2], b3 = Qsb[3];
  double ab = b0 + E.u * b1 + E.v * b2;
  double ub = a * b1, vb = a * b2;
  double cb = nx * d * b1 + ny * d * b2 + E.Un * d * b3;
  double nxb_ = E.c * d * b1 + W[2] * b2;
  double nyb_ = -W[2] * b1 + E.c * d * b2;
  const double db = E.c * nx * b1 + E.c * ny * b2 + E.c * E.Un * b3;
  double Wb[4];
  Wb[2] = -ny * b1 + nx * b2 + E.Ut * b3;
  double Hb = s * b3;
  double sb = E.H * b3;
  double Unb = E.c * d * b3;
  double h2b = W[1] * b3;
  double Utb = W[2] * b3;
  Wb[1] = ab + E.h2 * b3;
  sb += ab;
  Wb[0] = sb - db;
  Wb[3] = sb + db;
  // through WENO and the projection u_m^k = L_k . dQ_m
  double Lb[4][4] = {};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double ubk[7] = {0, 0, 0, 0, 0, 0, 0};
    weno_bwd_tape<R>(tape[k], ppm, linw, Wb[k], ubk);
    // stencil offset index aa -> position in ubk
    constexpr int NA = R == 4 ? 6 : 4;
    constexpr int m4[6] = {0, 1, 2, 4, 5, 6}, m3[6] = {0, 1, 3, 4, 0, 0};
    const int* mlist = R == 4 ? m4 : m3;
#pragma unroll
    for (int aa = 0; aa < NA; ++aa) {
      if (R == 2 && aa == 3) continue;
      const double g = ubk[mlist[aa]];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        Lb[k][v] += g * dq[aa][v];
        dqb[aa][v] += g * E.L[k][v];
      }
    }
  }
  // L rows from the primitives and the direction (see Eig::build)
  const double hb1 = 0.5 * w.b1, b2v = w.b1 * w.h2, hc = 0.5 * w.cinv;
  const double hb2b = Lb[0][0] + Lb[3][0];
  const double hUcb = Lb[0][0] - Lb[3][0];
  const double hb1b = -E.u * Lb[0][1] - E.v * Lb[0][2] + Lb[0][3] - E.u * Lb[3][1] - E.v * Lb[3][2] + Lb[3][3];
  ub += -hb1 * Lb[0][1] - hb1 * Lb[3][1] + w.b1 * Lb[1][1];
  vb += -hb1 * Lb[0][2] - hb1 * Lb[3][2] + w.b1 * Lb[1][2];
  const double hnxcb = -Lb[0][1] + Lb[3][1], hnycb = -Lb[0][2] + Lb[3][2];
  const double b2b = -Lb[1][0] + 0.5 * hb2b;
  double b1b = E.u * Lb[1][1] + E.v * Lb[1][2] - Lb[1][3] + 0.5 * hb1b;
  Utb += -Lb[2][0];
  nyb_ += -Lb[2][1];
  nxb_ += Lb[2][2];
  Unb += hc * hUcb;
  const double hcb = E.Un * hUcb + nx * hnxcb + ny * hnycb;
  nxb_ += hc * hnxcb;
  nyb_ += hc * hnycb;
  const double cinvb = 0.5 * hcb;
  b1b += w.h2 * b2b;
  h2b += w.b1 * b2b;
  (void)b2v;
  // Un = u nx + v ny, Ut = v nx - u ny
  ub += nx * Unb - ny * Utb;
  vb += ny * Unb + nx * Utb;
  nxb_ += E.u * Unb + E.v * Utb;
  nyb_ += E.v * Unb - E.u * Utb;
  pbar.u += ub; pbar.v += vb; pbar.c += cb; pbar.cinv += cinvb; pbar.H += Hb; pbar.b1 += b1b; pbar.h2 += h2b;
  nxb += nxb_;
  nyb += nyb_;
}

}  // namespace fsp
