// metrics.cu -- conservative grid metrics and Jacobian (Section 2.2, Eqs. 2.3 and 2.5 in
// two dimensions) differenced with each scheme's central operator (Eq. 2.7 and
// Eqs. 3.7/3.9/3.19/3.21), on the node range extended by G ghost layers.
#include "fsp_internal.h"

namespace fsp {

struct CoordParams {
  int ni, nj;
  int per_i, per_j;      // 1 if the direction is periodic
  double pi_x, pi_y;     // period vector per wrap in i
  double pj_x, pj_y;     // period vector per wrap in j
  const double* x;
  const double* y;
};

// Index a along a direction of n nodes -> up to two (index, weight) pairs plus a wrap count.
// Periodic: the wrapped node, and the number of periods crossed.  Otherwise odd
// reflection about the boundary node b: x_a = 2 x_b - x_{2b-a} (needs |a - b| < n).
struct Resolved { int idx[2]; double w[2]; int cnt; int wraps; };

__device__ __forceinline__ Resolved resolve(int a, int n, int periodic) {
  Resolved r;
  r.wraps = 0;
  if (a >= 0 && a < n) { r.idx[0] = a; r.w[0] = 1.0; r.cnt = 1; return r; }
  if (periodic) {
    const int m = pmod(a, n);
    r.wraps = (a - m) / n;
    r.idx[0] = m; r.w[0] = 1.0; r.cnt = 1;
    return r;
  }
  const int b = a < 0 ? 0 : n - 1;
  r.idx[0] = b; r.w[0] = 2.0;
  r.idx[1] = 2 * b - a; r.w[1] = -1.0;
  r.cnt = 2;
  return r;
}

__device__ __forceinline__ void coord(const CoordParams& C, int i, int j, double& X, double& Y) {
  const Resolved ri = resolve(i, C.ni, C.per_i), rj = resolve(j, C.nj, C.per_j);
  X = ri.wraps * C.pi_x + rj.wraps * C.pj_x;
  Y = ri.wraps * C.pi_y + rj.wraps * C.pj_y;
  for (int b = 0; b < rj.cnt; ++b)
    for (int a = 0; a < ri.cnt; ++a) {
      const long long o = (long long)rj.idx[b] * C.ni + ri.idx[a];
      const double w = ri.w[a] * rj.w[b];
      X += w * __ldg(C.x + o);
      Y += w * __ldg(C.y + o);
    }
}

// Central derivative of x and y along one direction from 9 nodal values f[k] = f_{j+k-4};
// pts = points of the midpoint interpolation (4, 6, or 8 for WENOIU7).
__device__ __forceinline__ double central_diff(const Central& c, int interp, int pts, const double* f) {
  double d = c.a1 * (f[5] - f[3]) + c.a2 * (f[6] - f[2]) + c.a3 * (f[7] - f[1]) + c.a4 * (f[8] - f[0]);
  if (pts == 8) {
    // midpoint j + m + 1/2 uses f_{j+m-3} .. f_{j+m+4} = f[m+1 .. m+8]
    return d + c.b12 * (mid_interp8(interp, f + 1) - mid_interp8(interp, f + 0));
  }
  // midpoint j + m + 1/2 uses f_{j+m-2} .. f_{j+m+3} = f[m+2 .. m+7]
  const bool sixth = pts == 6;
  const double mp0 = mid_interp(interp, sixth, f + 2);   // j + 1/2
  const double mm0 = mid_interp(interp, sixth, f + 1);   // j - 1/2
  d += c.b12 * (mp0 - mm0);
  if (c.b32 != 0.0) {
    const double mp1 = mid_interp(interp, sixth, f + 3); // j + 3/2
    const double mm1 = mid_interp(interp, sixth, f + 0); // j - 3/2
    d += c.b32 * (mp1 - mm1);
  }
  return d;
}

// The four-midpoint scheme's operator: node terms to +-2 and midpoint terms to 5/2, with the
// eight-point interpolation, from 13 nodal values f[k] = f_{j+k-6}; midpoint j + m + 1/2 uses
// f_{j+m-3} .. f_{j+m+4} = f[m+3 .. m+10].
__device__ __forceinline__ double central_diff13(const Central& c, int interp, const double* f) {
  double d = c.a1 * (f[7] - f[5]) + c.a2 * (f[8] - f[4]);
  d += c.b12 * (mid_interp8(interp, f + 3) - mid_interp8(interp, f + 2));
  d += c.b32 * (mid_interp8(interp, f + 4) - mid_interp8(interp, f + 1));
  d += c.b52 * (mid_interp8(interp, f + 5) - mid_interp8(interp, f + 0));
  return d;
}

// Points of the midpoint interpolation of a scheme.
inline int interp_points(int scheme) { return scheme == S71 || scheme == S74 ? 8 : scheme >= S51 ? 6 : 4; }

__global__ void metrics_kernel(CoordParams C, Central cen, int interp, int pts, double* __restrict__ M) {
  const int W = C.ni + 2 * G, H = C.nj + 2 * G;
  const long long plane = (long long)W * H;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < plane;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % W) - G, j = (int)(t / W) - G;
    // nodal values at offsets -6..6 (the four-midpoint scheme reaches 6; the others use -4..4)
    double fx[13], fy[13], gx[13], gy[13];
    const bool wide = cen.b52 != 0.0;
#pragma unroll
    for (int k = 0; k < 13; ++k) {
      if (!wide && (k < 2 || k > 10)) { fx[k] = fy[k] = gx[k] = gy[k] = 0.0; continue; }
      coord(C, i + k - 6, j, fx[k], fy[k]);   // along xi
      coord(C, i, j + k - 6, gx[k], gy[k]);   // along eta
    }
    double x_xi, y_xi, x_eta, y_eta;
    if (wide) {
      x_xi = central_diff13(cen, interp, fx);
      y_xi = central_diff13(cen, interp, fy);
      x_eta = central_diff13(cen, interp, gx);
      y_eta = central_diff13(cen, interp, gy);
    } else {
      x_xi = central_diff(cen, interp, pts, fx + 2);
      y_xi = central_diff(cen, interp, pts, fy + 2);
      x_eta = central_diff(cen, interp, pts, gx + 2);
      y_eta = central_diff(cen, interp, pts, gy + 2);
    }
    M[0 * plane + t] = y_eta;
    M[1 * plane + t] = -x_eta;
    M[2 * plane + t] = -y_xi;
    M[3 * plane + t] = x_xi;
    M[4 * plane + t] = x_xi * y_eta - x_eta * y_xi;
  }
}

cudaError_t launch_metrics(const fsp_config& cfg, const fsp_block& blk, const double* x,
                           const double* y, double* M, cudaStream_t st) {
  CoordParams C;
  C.ni = blk.ni; C.nj = blk.nj;
  C.per_i = cfg.bc[0] == BC_PERIODIC; C.per_j = cfg.bc[2] == BC_PERIODIC;
  C.pi_x = blk.period[0][0]; C.pi_y = blk.period[0][1];
  C.pj_x = blk.period[1][0]; C.pj_y = blk.period[1][1];
  C.x = x; C.y = y;
  const long long n = (long long)(blk.ni + 2 * G) * (blk.nj + 2 * G);
  const int threads = 256;
  const long long blocks = (n + threads - 1) / threads;
  const int grid = stride_grid(blocks, 16);
  metrics_kernel<<<grid, threads, 0, st>>>(C, central_of(cfg.scheme, scheme_alpha_of(cfg)), cfg.interp, interp_points(cfg.scheme), M);
  return cudaGetLastError();
}

}  // namespace fsp
