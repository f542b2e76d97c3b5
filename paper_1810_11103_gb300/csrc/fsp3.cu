// fsp3.cu -- the three-dimensional path (Sections 2.1-2.2), FP64: five conserved variables,
// the symmetric conservative metrics of Eq. (2.4) and the Jacobian of Eq. (2.5), and one
// sweep per grid direction with the schemes of Section 3 and the Appendix.
//
// Layout: state [5][nk][nj][ni] (i fastest, no padding); metrics 10 planes on the grid
// extended by G = 4 layers, plane 3 d + c = component c (x, y, z) of the metric of direction
// d (xi, eta, zeta), plane 9 = J^-1.  Faces i-, i+, j-, j+, k-, k+: periodic or transmissive.
//
// Kernels:
//   coord_deriv3_kernel  coordinates and their central derivatives on the grid extended by 8
//   metrics3_kernel      Eq. 2.4 from products of those derivatives and coordinates, Eq. 2.5
//   lambda3_kernel       line maxima of |U^| + c|k^| of the three directions (atomics)
//   sweep3_kernel<S, D>  one direction: staged nodes and split fluxes, then per interface the
//                        characteristic WENO of both sides, midpoint fluxes and h, then the
//                        difference into the accumulator or, for zeta, the epilogue (dQ/dt or
//                        an RK3 stage)
#include <cstring>

#include "fsp_internal.h"

namespace fsp {

struct P3 {
  int n[3];                 // ni, nj, nk
  int bc[6];
  double per[3][3];         // period vector added per wrap in direction a
  int scheme, interp, ppm, linw;
  double gamma, alpha, eps;
  const double* met;        // haloed metrics
  long long me[3];          // extended extents n + 2G
  long long mplane;         // (ni + 2G)(nj + 2G)(nk + 2G)
};

__host__ __device__ __forceinline__ long long node3(const P3& P, int i, int j, int k) {
  return ((long long)k * P.n[1] + j) * P.n[0] + i;
}
__device__ __forceinline__ double met3(const P3& P, int p, int i, int j, int k) {
  return __ldg(P.met + p * P.mplane + ((long long)(k + G) * P.me[1] + (j + G)) * P.me[0] + (i + G));
}

// Index a of a direction of n nodes -> at most two (index, weight) pairs and the wraps: a
// periodic direction wraps (the caller adds the period vector per wrap), any other direction
// reflects oddly about its boundary node b, x_a = 2 x_b - x_{2b-a} (|a - b| < n).
struct Res1 { int idx[2]; double w[2]; int cnt, wraps; };
__device__ __forceinline__ Res1 resolve3(int a, int n, bool periodic) {
  Res1 r;
  r.wraps = 0;
  r.cnt = 1;
  r.w[0] = 1.0;
  if (a >= 0 && a < n) { r.idx[0] = a; return r; }
  if (periodic) {
    const int m = pmod(a, n);
    r.wraps = (a - m) / n;
    r.idx[0] = m;
    return r;
  }
  const int b = a < 0 ? 0 : n - 1;
  r.idx[0] = b; r.w[0] = 2.0;
  r.idx[1] = 2 * b - a; r.w[1] = -1.0;
  r.cnt = 2;
  return r;
}

// Coordinate c of node (i, j, k) of the extended grid.
__device__ double coord3(const P3& P, const double* __restrict__ X, int c, int i, int j, int k) {
  const Res1 ri = resolve3(i, P.n[0], P.bc[0] == FSP_BC_PERIODIC);
  const Res1 rj = resolve3(j, P.n[1], P.bc[2] == FSP_BC_PERIODIC);
  const Res1 rk = resolve3(k, P.n[2], P.bc[4] == FSP_BC_PERIODIC);
  double v = ri.wraps * P.per[0][c] + rj.wraps * P.per[1][c] + rk.wraps * P.per[2][c];
  for (int ck = 0; ck < rk.cnt; ++ck)
    for (int cj = 0; cj < rj.cnt; ++cj)
      for (int ci = 0; ci < ri.cnt; ++ci)
        v += ri.w[ci] * rj.w[cj] * rk.w[ck] * __ldg(X + node3(P, ri.idx[ci], rj.idx[cj], rk.idx[ck]));
  return v;
}

// The scheme's central operator delta^{c,(1)} (Eq. 2.7) of nodal values f[m + 4], m = -4..4,
// with the midpoint values from the interpolation I (pts = 4, 6 or 8 points).
__device__ __forceinline__ double central9(const Central& c, int interp, int pts, const double* f) {
  double d = c.a1 * (f[5] - f[3]) + c.a2 * (f[6] - f[2]) + c.a3 * (f[7] - f[1]) + c.a4 * (f[8] - f[0]);
  if (pts == 8) return d + c.b12 * (mid_interp8(interp, f + 1) - mid_interp8(interp, f + 0));
  const bool sixth = pts == 6;
  d += c.b12 * (mid_interp(interp, sixth, f + 2) - mid_interp(interp, sixth, f + 1));
  if (c.b32 != 0.0) d += c.b32 * (mid_interp(interp, sixth, f + 3) - mid_interp(interp, sixth, f + 0));
  return d;
}

// Extended grid of e layers: index of node (i, j, k).
struct Ext {
  int e, n0, n1, n2;
  __host__ __device__ long long size() const { return (long long)(n0 + 2 * e) * (n1 + 2 * e) * (n2 + 2 * e); }
  __host__ __device__ long long at(int i, int j, int k) const {
    return ((long long)(k + e) * (n1 + 2 * e) + (j + e)) * (n0 + 2 * e) + (i + e);
  }
};

// Stage 1: on the grid extended by 8 layers, the coordinates C[c] (3 planes) and their
// derivatives D[a][c] along each direction a (9 planes, plane 3 + 3 a + c).
__global__ void __launch_bounds__(256) coord_deriv3_kernel(P3 P, const double* __restrict__ x,
                                                           const double* __restrict__ y,
                                                           const double* __restrict__ z, Central cen, int pts,
                                                           double* __restrict__ W) {
  const Ext E{8, P.n[0], P.n[1], P.n[2]};
  const long long N = E.size();
  const double* X[3] = {x, y, z};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
    const int W0 = P.n[0] + 16, W1 = P.n[1] + 16;
    const int i = (int)(t % W0) - 8, j = (int)((t / W0) % W1) - 8, k = (int)(t / ((long long)W0 * W1)) - 8;
    for (int c = 0; c < 3; ++c) {
      W[c * N + t] = coord3(P, X[c], c, i, j, k);
      for (int a = 0; a < 3; ++a) {
        double f[9];
#pragma unroll
        for (int m = -4; m <= 4; ++m)
          f[m + 4] = coord3(P, X[c], c, i + (a == 0 ? m : 0), j + (a == 1 ? m : 0), k + (a == 2 ? m : 0));
        W[(3 + 3 * a + c) * N + t] = central9(cen, P.interp, pts, f);
      }
    }
  }
}

// Stage 2: metrics on the grid extended by G layers.  For direction d with the next two
// directions (a, b) = (d+1, d+2) mod 3, and component c with the next two coordinates
// (p, q) = (c+1, c+2) mod 3: m_{d,c} = 1/2 [(p_a q)_b - (p_b q)_a + (q_b p)_a - (q_a p)_b]
// (Eq. 2.4 for d = xi, c = x); J^-1 = 1/3 sum_{d,c} m_{d,c} (c)_d (Eq. 2.5).
__global__ void __launch_bounds__(256) metrics3_kernel(P3 P, const double* __restrict__ W, Central cen, int pts,
                                                       double* __restrict__ M) {
  const Ext E4{G, P.n[0], P.n[1], P.n[2]}, E8{8, P.n[0], P.n[1], P.n[2]};
  const long long N = E4.size(), N8 = E8.size();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
    const int W0 = P.n[0] + 2 * G, W1 = P.n[1] + 2 * G;
    const int i = (int)(t % W0) - G, j = (int)((t / W0) % W1) - G, k = (int)(t / ((long long)W0 * W1)) - G;
    // (f_s g)_t at node (i, j, k): derivative along t of the product D[s][f] C[g]
    auto dprod = [&](int tt, int s, int f, int g) {
      double v[9];
#pragma unroll
      for (int m = -4; m <= 4; ++m) {
        const long long o = E8.at(i + (tt == 0 ? m : 0), j + (tt == 1 ? m : 0), k + (tt == 2 ? m : 0));
        v[m + 4] = W[(3 + 3 * s + f) * N8 + o] * W[g * N8 + o];
      }
      return central9(cen, P.interp, pts, v);
    };
    const long long o8 = E8.at(i, j, k);
    double Jv = 0.0;
    for (int d = 0; d < 3; ++d)
      for (int c = 0; c < 3; ++c) {
        const int a = (d + 1) % 3, b = (d + 2) % 3, p = (c + 1) % 3, q = (c + 2) % 3;
        const double m = 0.5 * (dprod(b, a, p, q) - dprod(a, b, p, q) + dprod(a, b, q, p) - dprod(b, a, q, p));
        M[(3 * d + c) * N + t] = m;
        Jv += m * W[(3 + 3 * d + c) * N8 + o8];
      }
    M[9 * N + t] = Jv * (1.0 / 3.0);
  }
}

// ---- line maxima -------------------------------------------------------------------------
// lam_xi[k nj + j], lam_eta[k ni + i], lam_zeta[j ni + i]: max over the line of |U^| + c|k^|
// (without alpha), taken with atomic maxima of the bit patterns (non-negative doubles).  A
// CTA is 32 i x 8 j threads, each walking LK3 values of k.
constexpr int LK3 = 8;
__device__ __forceinline__ void amax(double* a, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ double spectral3(const double q[5], double mx, double my, double mz, double gamma) {
  const double ri = rcp_nr(q[0]);
  const double u = q[1] * ri, v = q[2] * ri, w = q[3] * ri;
  const double p = (gamma - 1.0) * (q[4] - 0.5 * (q[1] * u + q[2] * v + q[3] * w));
  const double c = sqrt(gamma * p * ri);
  return fabs(mx * u + my * v + mz * w) + c * sqrt(mx * mx + my * my + mz * mz);
}
__global__ void __launch_bounds__(256) lambda3_kernel(P3 P, const double* __restrict__ Q, double* lx, double* ly,
                                                      double* lz) {
  __shared__ double red[8][33];
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
  const int k0 = blockIdx.z * LK3;
  const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
  const bool on = i < P.n[0] && j < P.n[1];
  double sz = 0.0;
  for (int k = k0; k < min(k0 + LK3, P.n[2]); ++k) {
    double sx = 0.0, sy = 0.0;
    if (on) {
      double q[5];
      const long long o = node3(P, i, j, k);
#pragma unroll
      for (int v = 0; v < 5; ++v) q[v] = Q[v * N + o];
      sx = spectral3(q, met3(P, 0, i, j, k), met3(P, 1, i, j, k), met3(P, 2, i, j, k), P.gamma);
      sy = spectral3(q, met3(P, 3, i, j, k), met3(P, 4, i, j, k), met3(P, 5, i, j, k), P.gamma);
      sz = max(sz, spectral3(q, met3(P, 6, i, j, k), met3(P, 7, i, j, k), met3(P, 8, i, j, k), P.gamma));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sx = max(sx, __shfl_xor_sync(0xffffffffu, sx, off));
    if (threadIdx.x == 0 && j < P.n[1]) amax(lx + (long long)k * P.n[1] + j, sx);
    red[threadIdx.y][threadIdx.x] = sy;
    __syncthreads();
    if (threadIdx.y == 0 && i < P.n[0]) {
      double m = red[0][threadIdx.x];
#pragma unroll
      for (int r = 1; r < 8; ++r) m = max(m, red[r][threadIdx.x]);
      amax(ly + (long long)k * P.n[0] + i, m);
    }
    __syncthreads();
  }
  if (on) amax(lz + (long long)j * P.n[0] + i, sz);
}

// ---- sweeps --------------------------------------------------------------------------------
enum { W3_WRITE = 0, W3_ADD = 1, W3_RHS = 2, W3_STAGE = 3 };

// A tile: NL lines of direction D (consecutive j for xi, consecutive i for eta and zeta) x W
// interface slots, with the lines across the lanes of a warp (a warp takes four interface
// positions of 8 lines, so a ragged last tile leaves whole warps idle rather than lanes);
// T output nodes per line and the nodes base - 4 .. base + T + 3 staged.
template <int S, int D>
struct Tile3 {
  static constexpr int NL = 8;
  static constexpr int W = 32;
  static constexpr int NMP = Scheme<S>::nmp;
  static constexpr int T = W - NMP - 1;
  static constexpr int NP = T + 8;
  static constexpr int NN = NL * NP, NW = NL * W;
  static constexpr int THREADS = 128;
  static constexpr int CTAS = 2;       // per SM: one CTA's barrier phases overlap the other's sweeps (three: no faster)
  // shared memory (doubles): per node the state 5, direction metrics 3, split fluxes 5 + 5 and
  // the characteristic data 9 (Node3); h 5 per interface; the two-midpoint schemes' midpoint
  // fluxes 10 per interface; A^ per line
  static constexpr size_t smem_bytes() {
    return sizeof(double) * ((size_t)27 * NN + 5 * (size_t)NW + (NMP == 2 ? 10 * (size_t)NW : 0) + NL);
  }
};

// The direction-free part of the characteristic system at a node (Section 3.4 in three
// dimensions): velocity, |u|^2/2, sound speed and its reciprocal, enthalpy, and
// b1 = (gamma - 1)/c^2, b2 = b1 |u|^2/2.  Staged once per node; both interfaces that use the
// node as a stencil centre read it.
struct Node3 {
  double ux, uy, uz, h2, c, ci, H, b1, b2;
  static constexpr int COUNT = 9;
  // from the state; p receives the pressure
  __device__ __forceinline__ void build(const double q[5], double gamma, double& p) {
    const double ri = rcp_nr(q[0]);
    ux = q[1] * ri; uy = q[2] * ri; uz = q[3] * ri;
    h2 = 0.5 * (ux * ux + uy * uy + uz * uz);
    p = (gamma - 1.0) * (q[4] - q[0] * h2);
    const double c2 = gamma * p * ri;
    ci = rsq(c2);
    c = c2 * ci;
    H = (q[4] + p) * ri;
    b1 = (gamma - 1.0) * ci * ci;
    b2 = b1 * h2;
  }
  __device__ __forceinline__ void store(double* b, int stride, int o) const {
    b[o] = ux; b[stride + o] = uy; b[2 * stride + o] = uz; b[3 * stride + o] = h2; b[4 * stride + o] = c;
    b[5 * stride + o] = ci; b[6 * stride + o] = H; b[7 * stride + o] = b1; b[8 * stride + o] = b2;
  }
  __device__ __forceinline__ void load(const double* b, int stride, int o) {
    ux = b[o]; uy = b[stride + o]; uz = b[2 * stride + o]; h2 = b[3 * stride + o]; c = b[4 * stride + o];
    ci = b[5 * stride + o]; H = b[6 * stride + o]; b1 = b[7 * stride + o]; b2 = b[8 * stride + o];
  }
};

// The unit direction n of an interface and its tangents: the Un eigenspace takes the entropy
// wave and two shear waves along t1 = (a x n)/|a x n|, a the coordinate axis least aligned
// with n (ties to the later axis), and t2 = n x t1.  Shared by the interface's two sides.
struct Dir3 {
  double nx, ny, nz, t1x, t1y, t1z, t2x, t2y, t2z;
  // from the sum of the two nodes' direction metrics (the average's 1/2 cancels)
  __device__ __forceinline__ void build(const double mb[3]) {
    const double rn = rsq(mb[0] * mb[0] + mb[1] * mb[1] + mb[2] * mb[2]);
    nx = mb[0] * rn; ny = mb[1] * rn; nz = mb[2] * rn;
    double x0, x1, x2;
    const double ax = fabs(nx), ay = fabs(ny), az = fabs(nz);
    if (ax < ay && ax < az) { x0 = 0.0; x1 = -nz; x2 = ny; }
    else if (ay < az) { x0 = nz; x1 = 0.0; x2 = -nx; }
    else { x0 = -ny; x1 = nx; x2 = 0.0; }
    const double s = rsq(x0 * x0 + x1 * x1 + x2 * x2);
    t1x = x0 * s; t1y = x1 * s; t1z = x2 * s;
    t2x = ny * t1z - nz * t1y;
    t2y = nz * t1x - nx * t1z;
    t2z = nx * t1y - ny * t1x;
  }
};

// One side of an interface: the eigen-system of the centre node along the interface's
// direction.  Left eigenvectors (rows 0..4 for u - c, u (entropy), the two shear waves, u + c)
// applied to a state difference dq through its common parts P0 = (b2 dq0 - b1 (u.dq - dq4))/2
// and B = c^-1 (Un dq0 - n.dq)/2: w0 = P0 + B, w4 = P0 - B, w1 = dq0 - 2 P0; right
// eigenvectors summed through s = W0 + W4 and c (W4 - W0).
struct Side3 {
  const Node3& w;
  const Dir3& d;
  double Un, U1, U2;
  __device__ __forceinline__ Side3(const Node3& w_, const Dir3& d_) : w(w_), d(d_) {
    Un = w.ux * d.nx + w.uy * d.ny + w.uz * d.nz;
    U1 = w.ux * d.t1x + w.uy * d.t1y + w.uz * d.t1z;
    U2 = w.ux * d.t2x + w.uy * d.t2y + w.uz * d.t2z;
  }
  __device__ __forceinline__ void project(const double dq[5], double o[5]) const {
    const double bu = w.b1 * (w.ux * dq[1] + w.uy * dq[2] + w.uz * dq[3] - dq[4]);
    const double P0 = 0.5 * (w.b2 * dq[0] - bu);
    const double B = 0.5 * w.ci * (Un * dq[0] - (d.nx * dq[1] + d.ny * dq[2] + d.nz * dq[3]));
    o[0] = P0 + B;
    o[1] = dq[0] - 2.0 * P0;
    o[2] = d.t1x * dq[1] + d.t1y * dq[2] + d.t1z * dq[3] - U1 * dq[0];
    o[3] = d.t2x * dq[1] + d.t2y * dq[2] + d.t2z * dq[3] - U2 * dq[0];
    o[4] = P0 - B;
  }
  // Q = qc + sum_k W_k r_k
  __device__ __forceinline__ void recon(const double W[5], const double qc[5], double Q[5]) const {
    const double s = W[0] + W[4], cd = w.c * (W[4] - W[0]), a = s + W[1];
    Q[0] = qc[0] + a;
    Q[1] = qc[1] + a * w.ux + cd * d.nx + W[2] * d.t1x + W[3] * d.t2x;
    Q[2] = qc[2] + a * w.uy + cd * d.ny + W[2] * d.t1y + W[3] * d.t2y;
    Q[3] = qc[3] + a * w.uz + cd * d.nz + W[2] * d.t1z + W[3] * d.t2z;
    Q[4] = qc[4] + s * w.H + W[1] * w.h2 + cd * Un + W[2] * U1 + W[3] * U2;
  }
};

// metric-weighted flux E^ = m_x E + m_y F + m_z G
__device__ __forceinline__ void flux3(const double q[5], const double m[3], double gamma, double f[5]) {
  const double ri = rcp_nr(q[0]);
  const double u = q[1] * ri, v = q[2] * ri, w = q[3] * ri;
  const double p = (gamma - 1.0) * (q[4] - 0.5 * (q[1] * u + q[2] * v + q[3] * w));
  const double U = m[0] * u + m[1] * v + m[2] * w;
  f[0] = q[0] * U;
  f[1] = q[1] * U + m[0] * p;
  f[2] = q[2] * U + m[1] * p;
  f[3] = q[3] * U + m[2] * p;
  f[4] = (q[4] + p) * U;
}

// node of position g on line l of a tile whose other two indices start at (o1, o2)
template <int D>
__device__ __forceinline__ void tile_node(int g, int l, int o1, int o2, int& i, int& j, int& k) {
  if (D == 0) { i = g; j = o1 + l; k = o2; }
  else if (D == 1) { i = o1 + l; j = g; k = o2; }
  else { i = o1 + l; j = o2; k = g; }
}

template <int S, int D, int MODE>
__global__ void __launch_bounds__(Tile3<S, D>::THREADS, Tile3<S, D>::CTAS)
sweep3_kernel(P3 P, const double* __restrict__ Q, const double* __restrict__ lam, double* acc, double* out,
              const double* Qn, double ca, double cb, double dt) {
  using Sh = Tile3<S, D>;
  using Sc = Scheme<S>;
  constexpr int NL = Sh::NL, T = Sh::T, NN = Sh::NN, NW = Sh::NW, NMP = Sh::NMP;
  constexpr int R = Sc::r, H = R == 4 ? 3 : 2, NA = 2 * H, SC = weno_scale<R>();
  extern __shared__ __align__(16) double sm3[];
  double* sq = sm3;                 // [5][NN]
  double* smt = sq + 5 * NN;        // [3][NN]
  double* sfp = smt + 3 * NN;       // [5][NN]
  double* sfm = sfp + 5 * NN;       // [5][NN]
  double* sc = sfm + 5 * NN;        // [Node3::COUNT][NN]
  double* sH = sc + Node3::COUNT * NN;   // [5][NW]
  double* sF = sH + 5 * NW;         // [10][NW] (two-midpoint schemes)
  double* sA = sF + (NMP == 2 ? 10 * NW : 0);   // [NL]
  const int n = P.n[D];
  const int nlines = D == 0 ? P.n[1] : P.n[0];             // lines per tile row
  const int o1 = blockIdx.y * NL;                          // first line (j for xi, i otherwise)
  const int o2 = blockIdx.z;                               // k for xi and eta, j for zeta
  const int base = blockIdx.x * T;
  const long long N = (long long)P.n[0] * P.n[1] * P.n[2];
  auto SI = [](int l, int s) { return s * NL + l; };
  auto WI = [](int l, int p) { return p * NL + l; };
  auto lam_index = [&](int l) -> long long {
    const int a = o1 + l;
    return D == 0 ? (long long)o2 * P.n[1] + a : D == 1 ? (long long)o2 * P.n[0] + a : (long long)o2 * P.n[0] + a;
  };
  if (threadIdx.x < NL) sA[threadIdx.x] = o1 + (int)threadIdx.x < nlines ? P.alpha * lam[lam_index(threadIdx.x)] : 0.0;
  __syncthreads();
  // ---- nodes: state (ghosts by the face rule), direction metrics, split fluxes, characteristic data
  for (int t = threadIdx.x; t < NN; t += Sh::THREADS) {
    const int l = t % NL, s = t / NL;
    if (o1 + l >= nlines) continue;
    const int g = min(base + s - 4, n + 3);   // ghost metrics are stored; ghost states by the face rule
    int gs = g;
    if (g < 0 || g >= n) {
      const bool per = P.bc[2 * D] == FSP_BC_PERIODIC;
      gs = per ? pmod(g, n) : (g < 0 ? 0 : n - 1);
    }
    int i, j, k;
    tile_node<D>(gs, l, o1, o2, i, j, k);
    double q[5];
    const long long o = node3(P, i, j, k);
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v] = Q[v * N + o];
    tile_node<D>(g, l, o1, o2, i, j, k);
    double m[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) m[c] = met3(P, 3 * D + c, i, j, k);
    // the node's characteristic data, and its metric-weighted flux from the same primitives
    Node3 w;
    double pr;
    w.build(q, P.gamma, pr);
    const double U = m[0] * w.ux + m[1] * w.uy + m[2] * w.uz;
    const double f[5] = {q[0] * U, q[1] * U + m[0] * pr, q[2] * U + m[1] * pr, q[3] * U + m[2] * pr,
                         (q[4] + pr) * U};
    const double A = sA[l];
    const int so = SI(l, s);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      sq[v * NN + so] = q[v];
      sfp[v * NN + so] = 0.5 * fma(A, q[v], f[v]);
      sfm[v * NN + so] = 0.5 * fma(-A, q[v], f[v]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) smt[c * NN + so] = m[c];
    w.store(sc, NN, so);
  }
  __syncthreads();
  // ---- interfaces p + 1/2
  const double eps = P.eps;
  for (int t = threadIdx.x; t < NW; t += Sh::THREADS) {
    const int l = t % NL, pi = t / NL;
    const int p = pi - NMP;
    if (o1 + l >= nlines || base + p > n || (NMP == 1 && p > T - 1)) continue;
    const int c0 = p + 4;
    const double A = sA[l];
    double mb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) mb[c] = smt[c * NN + SI(l, c0)] + smt[c * NN + SI(l, c0 + 1)];
    Dir3 dir;
    dir.build(mb);
    double Qs[2][5];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int ce = SI(l, c0 + side);
      double qc[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) qc[v] = sq[v * NN + ce];
      Node3 w;
      w.load(sc, NN, ce);
      const Side3 E(w, dir);
      // characteristic differences to the centre at the stencil offsets -H..-1, +1..+H (the
      // "-" side reads the mirrored nodes), component k at u[k][a or a + 1]; u[k][H] = 0
      double u[5][NA + 1];
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        const int m = a < H ? a - H : a - H + 1;
        const int ua = a < H ? a : a + 1;
        if (R == 2 && m == 2) {
#pragma unroll
          for (int k = 0; k < 5; ++k) u[k][ua] = 0.0;
          continue;
        }
        const int nd = SI(l, side == 0 ? c0 + m : c0 + 1 - m);
        double dq[5], o[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) dq[v] = sq[v * NN + nd] - qc[v];
        E.project(dq, o);
#pragma unroll
        for (int k = 0; k < 5; ++k) u[k][ua] = o[k];
      }
      double Wk[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        u[k][H] = 0.0;
        Wk[k] = weno_delta<R, double>(u[k], eps, P.ppm, P.linw) * (1.0 / SC);
      }
      E.recon(Wk, qc, Qs[side]);
    }
    // midpoint metrics by the interpolation of the metric evaluation
    double mm[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if constexpr (R == 4) {
        double vv[8];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) vv[kk] = smt[c * NN + SI(l, c0 - 3 + kk)];
        mm[c] = mid_interp8(P.interp, vv);
      } else {
        double vv[6];
#pragma unroll
        for (int kk = 0; kk < 6; ++kk) vv[kk] = smt[c * NN + SI(l, c0 - 2 + kk)];
        mm[c] = mid_interp(P.interp, R == 3, vv);
      }
    }
    double fpl[5], fmi[5];
    flux3(Qs[0], mm, P.gamma, fpl);
    flux3(Qs[1], mm, P.gamma, fmi);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      fpl[v] = 0.5 * fma(A, Qs[0][v], fpl[v]);
      fmi[v] = 0.5 * fma(-A, Qs[1][v], fmi[v]);
    }
    if constexpr (NMP == 1) {
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double h = Sc::m0 * (fpl[v] + fmi[v]);
#pragma unroll
        for (int kk = -3; kk <= 3; ++kk) {
          if (Sc::hn(kk) == 0.0) continue;
          h = fma(Sc::hn(kk), sfp[v * NN + SI(l, c0 + kk)] + sfm[v * NN + SI(l, c0 + 1 - kk)], h);
        }
        sH[v * NW + WI(l, pi)] = h;
      }
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        sF[v * NW + WI(l, pi)] = fpl[v];
        sF[(5 + v) * NW + WI(l, pi)] = fmi[v];
      }
    }
  }
  if constexpr (NMP == 2) {
    __syncthreads();
    // h+ uses f+ at p + 1/2 and p - 1/2; h- uses f- at p + 1/2 and p + 3/2
    for (int t = threadIdx.x; t < NW; t += Sh::THREADS) {
      const int l = t % NL, pi = t / NL;
      const int p = pi - NMP;
      if (o1 + l >= nlines || p < -1 || p > T - 1 || base + p > n - 1) continue;
      const int c0 = p + 4;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double h = Sc::m0 * (sF[v * NW + WI(l, pi)] + sF[(5 + v) * NW + WI(l, pi)]) +
                   Sc::m1 * (sF[v * NW + WI(l, pi - 1)] + sF[(5 + v) * NW + WI(l, pi + 1)]);
#pragma unroll
        for (int kk = -3; kk <= 3; ++kk) {
          if (Sc::hn(kk) == 0.0) continue;
          h = fma(Sc::hn(kk), sfp[v * NN + SI(l, c0 + kk)] + sfm[v * NN + SI(l, c0 + 1 - kk)], h);
        }
        sH[v * NW + WI(l, pi)] = h;
      }
    }
  }
  __syncthreads();
  // ---- outputs: node s, H_{s+1/2} - H_{s-1/2}
  for (int t = threadIdx.x; t < NL * T; t += Sh::THREADS) {
    const int l = t % NL, s = t / NL;
    const int g = base + s;
    if (o1 + l >= nlines || g >= n) continue;
    const int pi = s + NMP;
    int i, j, k;
    tile_node<D>(g, l, o1, o2, i, j, k);
    const long long o = node3(P, i, j, k);
    double Rv[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) Rv[v] = sH[v * NW + WI(l, pi)] - sH[v * NW + WI(l, pi - 1)];
    if constexpr (MODE == W3_WRITE) {
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v * N + o] = Rv[v];
    } else if constexpr (MODE == W3_ADD) {
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v * N + o] += Rv[v];
    } else {
      const double mJ = -rcp_nr(met3(P, 9, i, j, k));
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double d = (acc[v * N + o] + Rv[v]) * mJ;
        if constexpr (MODE == W3_RHS) out[v * N + o] = d;
        else out[v * N + o] = ca * Qn[v * N + o] + cb * (sq[v * NN + SI(l, s + 4)] + dt * d);
      }
    }
  }
}

// ---- host side ------------------------------------------------------------------------------
namespace {

size_t al3(size_t b) { return (b + 255) / 256 * 256; }

bool dptr3(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

fsp_status check3(const fsp_config* c, const fsp3_block* b) {
  if (!c || !b) return FSP_ERR_INVALID_ARG;
  if (c->scheme < 0 || c->scheme > 5 || c->interp < 0 || c->interp > 1 || !(c->gamma > 1.0) || !(c->lf_alpha > 0.0) ||
      !(c->eps > 0.0) || c->precision < FSP_FP64 || c->precision > FSP_FP32_MIXED)
    return FSP_ERR_INVALID_ARG;
  if (fsp_status s = check_options(*c)) return s;
  if (c->precision != FSP_FP64 || !default_options(*c) || c->scheme == S74) return FSP_ERR_UNSUPPORTED;
  for (int a = 0; a < 3; ++a) {
    const int n = a == 0 ? b->ni : a == 1 ? b->nj : b->nk;
    const int f0 = b->bc[2 * a], f1 = b->bc[2 * a + 1];
    if (n < 1 || n > 65535) return FSP_ERR_INVALID_ARG;
    if ((f0 != FSP_BC_PERIODIC && f0 != FSP_BC_TRANSMISSIVE) || (f1 != FSP_BC_PERIODIC && f1 != FSP_BC_TRANSMISSIVE))
      return FSP_ERR_UNSUPPORTED;
    if ((f0 == FSP_BC_PERIODIC) != (f1 == FSP_BC_PERIODIC)) return FSP_ERR_INVALID_ARG;
    // the reflected ghost coordinates reach 12 nodes in
    if (f0 != FSP_BC_PERIODIC && n < 13) return FSP_ERR_INVALID_ARG;
  }
  return FSP_OK;
}

P3 make_p3(const fsp_config& c, const fsp3_block& b, const double* metrics) {
  P3 P;
  P.n[0] = b.ni; P.n[1] = b.nj; P.n[2] = b.nk;
  for (int f = 0; f < 6; ++f) P.bc[f] = b.bc[f];
  for (int a = 0; a < 3; ++a)
    for (int cc = 0; cc < 3; ++cc) P.per[a][cc] = b.period[a][cc];
  P.scheme = c.scheme; P.interp = c.interp; P.ppm = c.ppm; P.linw = c.linear_weights;
  P.gamma = c.gamma; P.alpha = c.lf_alpha; P.eps = c.eps;
  P.met = metrics;
  for (int a = 0; a < 3; ++a) P.me[a] = P.n[a] + 2 * G;
  P.mplane = P.me[0] * P.me[1] * P.me[2];
  return P;
}

long long nodes3(const fsp3_block& b) { return (long long)b.ni * b.nj * b.nk; }
size_t lam_count3(const fsp3_block& b) {
  return (size_t)b.nj * b.nk + (size_t)b.ni * b.nk + (size_t)b.ni * b.nj;
}
// right-hand side scratch: line maxima and the accumulator; RK3 adds two stage states
size_t rhs_scratch3(const fsp3_block& b) { return al3(8 * lam_count3(b)) + al3(8 * 5 * (size_t)nodes3(b)); }
size_t rk3_scratch3(const fsp3_block& b) { return rhs_scratch3(b) + 2 * al3(8 * 5 * (size_t)nodes3(b)); }
size_t metrics_scratch3(const fsp3_block& b) {
  return al3(8 * 12 * (size_t)((long long)(b.ni + 16) * (b.nj + 16) * (b.nk + 16)));
}

int grid_of3(long long n) { return stride_grid((n + 255) / 256, 8); }

template <int S, int D, int MODE>
cudaError_t launch_sweep3(const P3& P, const double* Q, const double* lam, double* acc, double* out, const double* Qn,
                          double ca, double cb, double dt, cudaStream_t st) {
  using Sh = Tile3<S, D>;
  auto kern = sweep3_kernel<S, D, MODE>;
  const size_t smem = Sh::smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int n = P.n[D], nlines = D == 0 ? P.n[1] : P.n[0];
  const int outer = D == 2 ? P.n[1] : P.n[2];
  dim3 grid((n + Sh::T - 1) / Sh::T, (nlines + Sh::NL - 1) / Sh::NL, outer);   // each within 65535 (n <= 65535)
  kern<<<grid, Sh::THREADS, smem, st>>>(P, Q, lam, acc, out, Qn, ca, cb, dt);
  return cudaGetLastError();
}

// the line maxima of Q into lam (zeroed first): xi, eta, zeta arrays back to back
cudaError_t launch_lambda3(const P3& P, const double* Q, double* lam, cudaStream_t st) {
  const size_t nl = (size_t)P.n[1] * P.n[2] + (size_t)P.n[0] * P.n[2] + (size_t)P.n[0] * P.n[1];
  cudaError_t e = cudaMemsetAsync(lam, 0, sizeof(double) * nl, st);
  if (e != cudaSuccess) return e;
  dim3 grid((P.n[0] + 31) / 32, (P.n[1] + 7) / 8, (P.n[2] + LK3 - 1) / LK3);
  double* lx = lam;
  double* ly = lx + (size_t)P.n[1] * P.n[2];
  double* lz = ly + (size_t)P.n[0] * P.n[2];
  lambda3_kernel<<<grid, dim3(32, 8), 0, st>>>(P, Q, lx, ly, lz);
  return cudaGetLastError();
}

// one right-hand side (mode 0: out = dQ/dt; mode 1: out = ca Qn + cb (Q + dt dQ/dt))
template <int S>
cudaError_t rhs3_scheme(const P3& P, const double* Q, double* lam, double* acc, double* out, int mode,
                        const double* Qn, double ca, double cb, double dt, cudaStream_t st) {
  cudaError_t e = launch_lambda3(P, Q, lam, st);
  if (e != cudaSuccess) return e;
  const double* lx = lam;
  const double* ly = lx + (size_t)P.n[1] * P.n[2];
  const double* lz = ly + (size_t)P.n[0] * P.n[2];
  if ((e = launch_sweep3<S, 0, W3_WRITE>(P, Q, lx, acc, nullptr, nullptr, 0, 0, 0, st)) != cudaSuccess) return e;
  if ((e = launch_sweep3<S, 1, W3_ADD>(P, Q, ly, acc, nullptr, nullptr, 0, 0, 0, st)) != cudaSuccess) return e;
  if (mode == 0) return launch_sweep3<S, 2, W3_RHS>(P, Q, lz, acc, out, nullptr, 0, 0, 0, st);
  return launch_sweep3<S, 2, W3_STAGE>(P, Q, lz, acc, out, Qn, ca, cb, dt, st);
}

cudaError_t rhs3_launch(const P3& P, const double* Q, double* lam, double* acc, double* out, int mode,
                        const double* Qn, double ca, double cb, double dt, cudaStream_t st) {
  switch (P.scheme) {
    case S31: return rhs3_scheme<S31>(P, Q, lam, acc, out, mode, Qn, ca, cb, dt, st);
    case S32: return rhs3_scheme<S32>(P, Q, lam, acc, out, mode, Qn, ca, cb, dt, st);
    case S51: return rhs3_scheme<S51>(P, Q, lam, acc, out, mode, Qn, ca, cb, dt, st);
    case S52: return rhs3_scheme<S52>(P, Q, lam, acc, out, mode, Qn, ca, cb, dt, st);
    default:  return rhs3_scheme<S71>(P, Q, lam, acc, out, mode, Qn, ca, cb, dt, st);
  }
}

struct Scratch3 { double *lam, *acc, *q1, *q2; };
Scratch3 carve3(const fsp3_block& b, void* ws) {
  char* p = static_cast<char*>(ws);
  Scratch3 s;
  s.lam = reinterpret_cast<double*>(p);
  p += al3(8 * lam_count3(b));
  s.acc = reinterpret_cast<double*>(p);
  p += al3(8 * 5 * (size_t)nodes3(b));
  s.q1 = reinterpret_cast<double*>(p);
  p += al3(8 * 5 * (size_t)nodes3(b));
  s.q2 = reinterpret_cast<double*>(p);
  return s;
}

fsp_status st3(cudaError_t e) {
  if (e == cudaSuccess) return FSP_OK;
  cudaGetLastError();
  return FSP_ERR_CUDA;
}

}  // namespace

}  // namespace fsp

using namespace fsp;

extern "C" {

long long fsp3_metrics_elems(const fsp3_block* b) {
  if (!b) return 0;
  return 10LL * (b->ni + 2 * G) * (b->nj + 2 * G) * (b->nk + 2 * G);
}

fsp_status fsp3_workspace_size(const fsp_config* cfg, const fsp3_block* blk, size_t* bytes) {
  if (!bytes) return FSP_ERR_INVALID_ARG;
  if (fsp_status s = check3(cfg, blk)) return s;
  const size_t a = rk3_scratch3(*blk), b = metrics_scratch3(*blk);
  *bytes = a > b ? a : b;
  return FSP_OK;
}

fsp_status fsp3_metrics(const fsp_config* cfg, const fsp3_block* blk, const double* x, const double* y, const double* z,
                        double* metrics, void* ws, size_t ws_bytes, void* stream) {
  if (fsp_status s = check3(cfg, blk)) return s;
  if (!dptr3(x) || !dptr3(y) || !dptr3(z) || !dptr3(metrics) || !dptr3(ws) || ws_bytes < metrics_scratch3(*blk))
    return FSP_ERR_INVALID_ARG;
  const P3 P = make_p3(*cfg, *blk, metrics);
  const Central cen = central_of(cfg->scheme);
  const int pts = cfg->scheme == S71 ? 8 : cfg->scheme >= S51 ? 6 : 4;
  cudaStream_t st = (cudaStream_t)stream;
  double* W = static_cast<double*>(ws);
  const long long n8 = (long long)(blk->ni + 16) * (blk->nj + 16) * (blk->nk + 16);
  const long long n4 = (long long)(blk->ni + 2 * G) * (blk->nj + 2 * G) * (blk->nk + 2 * G);
  coord_deriv3_kernel<<<grid_of3(n8), 256, 0, st>>>(P, x, y, z, cen, pts, W);
  if (cudaGetLastError() != cudaSuccess) return FSP_ERR_CUDA;
  metrics3_kernel<<<grid_of3(n4), 256, 0, st>>>(P, W, cen, pts, metrics);
  return st3(cudaGetLastError());
}

fsp_status fsp3_line_lambda(const fsp_config* cfg, const fsp3_block* blk, const double* metrics, const double* Q,
                            double* lam, void* stream) {
  if (fsp_status s = check3(cfg, blk)) return s;
  if (!dptr3(metrics) || !dptr3(Q) || !dptr3(lam)) return FSP_ERR_INVALID_ARG;
  return st3(launch_lambda3(make_p3(*cfg, *blk, metrics), Q, lam, (cudaStream_t)stream));
}

fsp_status fsp3_rhs(const fsp_config* cfg, const fsp3_block* blk, const double* metrics, const double* Q, double* dQdt,
                    void* ws, size_t ws_bytes, void* stream) {
  if (fsp_status s = check3(cfg, blk)) return s;
  if (!dptr3(metrics) || !dptr3(Q) || !dptr3(dQdt) || !dptr3(ws) || ws_bytes < rhs_scratch3(*blk))
    return FSP_ERR_INVALID_ARG;
  const Scratch3 w = carve3(*blk, ws);
  return st3(rhs3_launch(make_p3(*cfg, *blk, metrics), Q, w.lam, w.acc, dQdt, 0, nullptr, 0, 0, 0,
                         (cudaStream_t)stream));
}

fsp_status fsp3_rk3_step(const fsp_config* cfg, const fsp3_block* blk, const double* metrics, double* Q, double dt,
                         void* ws, size_t ws_bytes, void* stream) {
  if (fsp_status s = check3(cfg, blk)) return s;
  if (!dptr3(metrics) || !dptr3(Q) || !dptr3(ws) || ws_bytes < rk3_scratch3(*blk)) return FSP_ERR_INVALID_ARG;
  const Scratch3 w = carve3(*blk, ws);
  const P3 P = make_p3(*cfg, *blk, metrics);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = rhs3_launch(P, Q, w.lam, w.acc, w.q1, 1, Q, 0.0, 1.0, dt, st);
  if (e == cudaSuccess) e = rhs3_launch(P, w.q1, w.lam, w.acc, w.q2, 1, Q, 0.75, 0.25, dt, st);
  if (e == cudaSuccess) e = rhs3_launch(P, w.q2, w.lam, w.acc, Q, 1, Q, 1.0 / 3.0, 2.0 / 3.0, dt, st);
  return st3(e);
}

}  // extern "C"
