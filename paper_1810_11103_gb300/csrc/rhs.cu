// rhs.cu -- the semi-discrete right-hand side of the WENOIU schemes (Li & Sun,
// arXiv:1810.11103, Sections 2.3, 3 and 3.4) on one structured block, plus the per-line
// spectral radius of the splitting, the CFL rate and error norms.
//
// One right-hand side = three launches:
//   lambda_kernel      per-line maxima of |U^| + c|k^| (atomic max on the bit patterns of
//                      non-negative doubles, which order like the values)
//   sweep<DIR = 0>     xi direction: H_{i+1/2} - H_{i-1/2} into a scratch accumulator
//   sweep<DIR = 1>     eta direction, adds the xi part, divides by -J^-1 and writes dQ/dt
//                      or a TVD-RK3 stage
// A sweep CTA owns NL grid lines x T output nodes.  It stages the nodes of the tile plus
// four ghosts per side (state, the direction's metrics, node fluxes E^) in shared memory,
// then gives every thread one interface: the characteristic WENO states from both sides,
// the split midpoint fluxes, and the upwind-biased combination h = h+ + h-.
#include "fsp_internal.h"

namespace fsp {

// ------------------------------------------------------------------------------------
// Per-line spectral radius (Section 2.3) and per-node CFL rate
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  // non-negative doubles (and NaN, which then dominates) order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

template <typename Real>
__global__ void __launch_bounds__(256) lambda_kernel(Params P, const Real* __restrict__ Q,
                                                     double* __restrict__ lam_xi,
                                                     double* __restrict__ lam_eta,
                                                     double* __restrict__ cfl_max) {
  __shared__ double col[8][33];
  __shared__ double cfl_s[8];
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
  const bool in = i < P.ni && j < P.nj;
  double sx = 0.0, se = 0.0, rate = 0.0;
  if (in) {
    const long long plane = (long long)P.nj * P.ld, o = (long long)j * P.ld + i;
    double q[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) q[v] = (double)Q[v * plane + o];
    const double g = P.gamma;
    sx = spectral_radius(q, met_at(P, 0, i, j), met_at(P, 1, i, j), g);
    se = spectral_radius(q, met_at(P, 2, i, j), met_at(P, 3, i, j), g);
    rate = (sx + se) / met_at(P, 4, i, j);
  }
  // row maximum across the warp (one row of 32 nodes)
  double rx = sx, rr = rate;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    rx = fmax(rx, __shfl_xor_sync(0xffffffffu, rx, off));
    rr = fmax(rr, __shfl_xor_sync(0xffffffffu, rr, off));
  }
  if (threadIdx.x == 0 && j < P.nj) atomic_max_pos(lam_xi + j, rx);
  col[threadIdx.y][threadIdx.x] = se;
  if (threadIdx.x == 0) cfl_s[threadIdx.y] = rr;
  __syncthreads();
  if (threadIdx.y == 0 && i < P.ni) {
    double m = col[0][threadIdx.x];
#pragma unroll
    for (int r = 1; r < 8; ++r) m = fmax(m, col[r][threadIdx.x]);
    atomic_max_pos(lam_eta + i, m);
  }
  if (cfl_max && threadIdx.x == 0 && threadIdx.y == 0) {
    double m = cfl_s[0];
#pragma unroll
    for (int r = 1; r < 8; ++r) m = fmax(m, cfl_s[r]);
    atomic_max_pos(cfl_max, m);
  }
}

// ------------------------------------------------------------------------------------
// Directional sweep
// ------------------------------------------------------------------------------------
template <int S, int DIR>
struct TileShape {
  static constexpr int NL = DIR == 0 ? 2 : 8;            // grid lines per CTA
  static constexpr int W = DIR == 0 ? 128 : 32;          // interface slots per line
  static constexpr int NMP = Scheme<S>::nmp;
  static constexpr int T = W - NMP - 1;                  // output nodes per line
  static constexpr int NP = T + 8;                       // staged nodes per line (4 ghosts a side)
  static constexpr int PLO = -NMP;                       // first interface p (of p + 1/2)
  static constexpr int THREADS = 256;
  static constexpr size_t smem_bytes() {
    return sizeof(double) * ((size_t)(4 + 2 + 4) * NL * NP + (size_t)(4 + (NMP == 2 ? 8 : 0)) * NL * W);
  }
};

enum { MODE_ACC = 0, MODE_RHS = 1, MODE_STAGE = 2 };

template <int S, int DIR, int MODE>
__global__ void __launch_bounds__(256) sweep_kernel(Params P, const double* __restrict__ Q,
                                                    const double* __restrict__ lam,
                                                    const double* __restrict__ Racc,
                                                    double* out, const double* Qn,
                                                    double ca, double cb, double dt) {
  using Sh = TileShape<S, DIR>;
  using Sc = Scheme<S>;
  constexpr int NL = Sh::NL, W = Sh::W, T = Sh::T, NP = Sh::NP, PLO = Sh::PLO;
  constexpr int NN = NL * NP, NW = NL * W;
  extern __shared__ double smem[];
  double* sQ = smem;           // [4][NN]
  double* sM = sQ + 4 * NN;    // [2][NN]
  double* sE = sM + 2 * NN;    // [4][NN]
  double* sH = sE + 4 * NN;    // [4][NW]
  double* sF = sH + 4 * NW;    // [8][NW], two-midpoint schemes only

  const int n = DIR == 0 ? P.ni : P.nj;
  const int nlines = DIR == 0 ? P.nj : P.ni;
  const int line0 = blockIdx.y * NL;
  const int base = blockIdx.x * T;
  const double gm1 = P.gamma - 1.0;
  const long long plane = (long long)P.nj * P.ld;

  auto SI = [](int l, int s) { return DIR == 0 ? l * NP + s : s * NL + l; };
  auto WI = [](int l, int p) { return DIR == 0 ? l * W + p : p * NL + l; };

  // ---- nodes: state (ghosts by the boundary rule), the direction's metrics, E^ ----
  for (int k = threadIdx.x; k < NN; k += Sh::THREADS) {
    const int l = DIR == 0 ? k / NP : k % NL;
    const int s = DIR == 0 ? k % NP : k / NL;
    const int line = line0 + l;
    if (line >= nlines) continue;
    const int g = min(base + s - 4, n + 3);  // positions past n+3 are never used
    double q[4];
    load_state(P, Q, DIR, line, g, q);
    double mx, my;
    if (DIR == 0) { mx = met_at(P, 0, g, line); my = met_at(P, 1, g, line); }
    else          { mx = met_at(P, 2, line, g); my = met_at(P, 3, line, g); }
    double e[4];
    euler_flux(q, mx, my, gm1, e);
    const int o = SI(l, s);
#pragma unroll
    for (int v = 0; v < 4; ++v) { sQ[v * NN + o] = q[v]; sE[v * NN + o] = e[v]; }
    sM[o] = mx;
    sM[NN + o] = my;
  }
  __syncthreads();

  // ---- interfaces p + 1/2 ----
  for (int k = threadIdx.x; k < NW; k += Sh::THREADS) {
    const int l = DIR == 0 ? k / W : k % NL;
    const int pi = DIR == 0 ? k % W : k / NL;
    const int line = line0 + l;
    const int p = PLO + pi;
    if (line >= nlines || base + p > n) continue;
    const double A = P.alpha * lam[line];
    const int c0 = p + 4;  // staged position of node p

    // characteristic direction: unit vector of the averaged metrics (Section 3.4)
    const double mbx = 0.5 * (sM[SI(l, c0)] + sM[SI(l, c0 + 1)]);
    const double mby = 0.5 * (sM[NN + SI(l, c0)] + sM[NN + SI(l, c0 + 1)]);
    const double rn = 1.0 / sqrt(mbx * mbx + mby * mby);
    const double nx = mbx * rn, ny = mby * rn;

    double Qs[2][4];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int ce = c0 + side;  // "+" side: eigenvectors at Q_p; "-" side: at Q_{p+1}
      double qc[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) qc[v] = sQ[v * NN + SI(l, ce)];
      Eig<double> E;
      E.build(qc, nx, ny, P.gamma);
      double Wm[4];
#pragma unroll
      for (int kc = 0; kc < 4; ++kc) {
        double u[5];
#pragma unroll
        for (int m = -2; m <= 2; ++m) {
          if (Sc::r == 2 && m == 2) { u[4] = 0.0; continue; }
          const int o = SI(l, side == 0 ? c0 + m : c0 + 1 - m);
          const double q0 = sQ[o], q1 = sQ[NN + o], q2 = sQ[2 * NN + o], q3 = sQ[3 * NN + o];
          u[m + 2] = kc == 2 ? (E.L[2][0] * q0 + E.L[2][1] * q1 + E.L[2][2] * q2)
                             : (E.L[kc][0] * q0 + E.L[kc][1] * q1 + E.L[kc][2] * q2 + E.L[kc][3] * q3);
        }
        Wm[kc] = weno_mid<Sc::r>(u, P.eps, P.ppm, P.linw);
      }
      E.recon(Wm, Qs[side]);
    }

    // midpoint metrics by the same interpolation as the metric evaluation (Section 2.4)
    double vx[6], vy[6];
#pragma unroll
    for (int kk = 0; kk < 6; ++kk) {
      const int o = SI(l, c0 - 2 + kk);
      vx[kk] = sM[o];
      vy[kk] = sM[NN + o];
    }
    const double mmx = mid_interp(P.interp, Sc::r == 3, vx);
    const double mmy = mid_interp(P.interp, Sc::r == 3, vy);
    double fp[4], fm[4];
    euler_flux(Qs[0], mmx, mmy, gm1, fp);
    euler_flux(Qs[1], mmx, mmy, gm1, fm);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      fp[v] = 0.5 * (fp[v] + A * Qs[0][v]);
      fm[v] = 0.5 * (fm[v] - A * Qs[1][v]);
    }
    if constexpr (Sc::nmp == 1) {
      // h = h+ + h-: midpoint terms plus the node terms of f+- = (E^ +- A Q)/2, with h-
      // the mirror of h+ about p + 1/2 (f_{p+k} -> f_{p+1-k})
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double h = Sc::m0 * (fp[v] + fm[v]);
#pragma unroll
        for (int kk = -2; kk <= 2; ++kk) {
          if (Sc::n(kk + 2) == 0.0) continue;
          const int a = SI(l, c0 + kk), b = SI(l, c0 + 1 - kk);
          h += Sc::n(kk + 2) * 0.5 * ((sE[v * NN + a] + sE[v * NN + b]) + A * (sQ[v * NN + a] - sQ[v * NN + b]));
        }
        sH[v * NW + WI(l, pi)] = h;
      }
    } else {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        sF[v * NW + WI(l, pi)] = fp[v];
        sF[(4 + v) * NW + WI(l, pi)] = fm[v];
      }
    }
  }

  if constexpr (Sc::nmp == 2) {
    __syncthreads();
    // h+ uses f+ at p+1/2 and p-1/2; h- uses f- at p+1/2 and p+3/2
    for (int k = threadIdx.x; k < NW; k += Sh::THREADS) {
      const int l = DIR == 0 ? k / W : k % NL;
      const int pi = DIR == 0 ? k % W : k / NL;
      const int line = line0 + l;
      const int p = PLO + pi;
      if (line >= nlines || p < -1 || p > T - 1 || base + p > n - 1) continue;
      const double A = P.alpha * lam[line];
      const int c0 = p + 4;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        double h = Sc::m0 * (sF[v * NW + WI(l, pi)] + sF[(4 + v) * NW + WI(l, pi)]) +
                   Sc::m1 * (sF[v * NW + WI(l, pi - 1)] + sF[(4 + v) * NW + WI(l, pi + 1)]);
#pragma unroll
        for (int kk = -2; kk <= 2; ++kk) {
          if (Sc::n(kk + 2) == 0.0) continue;
          const int a = SI(l, c0 + kk), b = SI(l, c0 + 1 - kk);
          h += Sc::n(kk + 2) * 0.5 * ((sE[v * NN + a] + sE[v * NN + b]) + A * (sQ[v * NN + a] - sQ[v * NN + b]));
        }
        sH[v * NW + WI(l, pi)] = h;
      }
    }
  }
  __syncthreads();

  // ---- nodes: difference of h (Eq. 3.2) and the epilogue ----
  for (int k = threadIdx.x; k < NL * T; k += Sh::THREADS) {
    const int l = DIR == 0 ? k / T : k % NL;
    const int s = DIR == 0 ? k % T : k / NL;
    const int line = line0 + l;
    const int g = base + s;
    if (line >= nlines || g >= n) continue;
    const int pi = s - PLO;  // interface s + 1/2
    const int i = DIR == 0 ? g : line, j = DIR == 0 ? line : g;
    const long long o = (long long)j * P.ld + i;
    double R[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) R[v] = sH[v * NW + WI(l, pi)] - sH[v * NW + WI(l, pi - 1)];
    if constexpr (MODE == MODE_ACC) {
#pragma unroll
      for (int v = 0; v < 4; ++v) out[v * plane + o] = R[v];
    } else {
      const double Jinv = met_at(P, 4, i, j);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const double d = -(Racc[v * plane + o] + R[v]) / Jinv;
        if constexpr (MODE == MODE_RHS) {
          out[v * plane + o] = d;
        } else {
          const double qs = sQ[v * NN + SI(l, s + 4)];
          out[v * plane + o] = ca * Qn[v * plane + o] + cb * (qs + dt * d);
        }
      }
    }
  }
}

template <int S, int DIR, int MODE>
static cudaError_t launch_sweep(const Params& P, const double* Q, const double* lam, const double* Racc,
                                double* out, const double* Qn, double ca, double cb, double dt,
                                cudaStream_t st) {
  using Sh = TileShape<S, DIR>;
  const int n = DIR == 0 ? P.ni : P.nj, nlines = DIR == 0 ? P.nj : P.ni;
  dim3 grid((n + Sh::T - 1) / Sh::T, (nlines + Sh::NL - 1) / Sh::NL);
  const size_t smem = Sh::smem_bytes();
  auto kern = sweep_kernel<S, DIR, MODE>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, Sh::THREADS, smem, st>>>(P, Q, lam, Racc, out, Qn, ca, cb, dt);
  return cudaGetLastError();
}

template <int S>
static cudaError_t rhs_scheme(const Params& P, const double* Q, const double* lam_xi,
                              const double* lam_eta, double* Racc, double* out, int mode,
                              const double* Qn, double ca, double cb, double dt, cudaStream_t st) {
  cudaError_t e = launch_sweep<S, 0, MODE_ACC>(P, Q, lam_xi, nullptr, Racc, nullptr, 0, 0, 0, st);
  if (e != cudaSuccess) return e;
  if (mode == 0) return launch_sweep<S, 1, MODE_RHS>(P, Q, lam_eta, Racc, out, nullptr, 0, 0, 0, st);
  return launch_sweep<S, 1, MODE_STAGE>(P, Q, lam_eta, Racc, out, Qn, ca, cb, dt, st);
}

cudaError_t launch_rhs(int scheme, int precision, const Params& P, const void* Q,
                       const double* lam_xi, const double* lam_eta, void* Racc, void* out, int mode,
                       const void* Qn, double ca, double cb, double dt, cudaStream_t st) {
  if (precision != FSP_FP64) return cudaErrorNotSupported;
  auto q = static_cast<const double*>(Q);
  auto r = static_cast<double*>(Racc);
  auto o = static_cast<double*>(out);
  auto qn = static_cast<const double*>(Qn);
  switch (scheme) {
    case S31: return rhs_scheme<S31>(P, q, lam_xi, lam_eta, r, o, mode, qn, ca, cb, dt, st);
    case S32: return rhs_scheme<S32>(P, q, lam_xi, lam_eta, r, o, mode, qn, ca, cb, dt, st);
    case S51: return rhs_scheme<S51>(P, q, lam_xi, lam_eta, r, o, mode, qn, ca, cb, dt, st);
    default:  return rhs_scheme<S52>(P, q, lam_xi, lam_eta, r, o, mode, qn, ca, cb, dt, st);
  }
}

template <int S>
static cudaError_t flux_difference_scheme(const Params& P, const double* Q, const double* lam, int dir,
                                          int mode, const double* acc, double* out, cudaStream_t st) {
  if (dir == 0)
    return mode == 0 ? launch_sweep<S, 0, MODE_ACC>(P, Q, lam, nullptr, out, nullptr, 0, 0, 0, st)
                     : launch_sweep<S, 0, MODE_RHS>(P, Q, lam, acc, out, nullptr, 0, 0, 0, st);
  return mode == 0 ? launch_sweep<S, 1, MODE_ACC>(P, Q, lam, nullptr, out, nullptr, 0, 0, 0, st)
                   : launch_sweep<S, 1, MODE_RHS>(P, Q, lam, acc, out, nullptr, 0, 0, 0, st);
}

cudaError_t launch_flux_difference(int scheme, int precision, const Params& P, const void* Q,
                                   const double* lam, int dir, int mode, const void* acc, void* out,
                                   cudaStream_t st) {
  if (precision != FSP_FP64) return cudaErrorNotSupported;
  auto q = static_cast<const double*>(Q);
  auto a = static_cast<const double*>(acc);
  auto o = static_cast<double*>(out);
  switch (scheme) {
    case S31: return flux_difference_scheme<S31>(P, q, lam, dir, mode, a, o, st);
    case S32: return flux_difference_scheme<S32>(P, q, lam, dir, mode, a, o, st);
    case S51: return flux_difference_scheme<S51>(P, q, lam, dir, mode, a, o, st);
    default:  return flux_difference_scheme<S52>(P, q, lam, dir, mode, a, o, st);
  }
}

cudaError_t launch_lambda(const Params& P, int precision, const void* Q, double* lam_xi,
                          double* lam_eta, double* cfl_max, cudaStream_t st) {
  dim3 block(32, 8), grid((P.ni + 31) / 32, (P.nj + 7) / 8);
  if (precision == FSP_FP64)
    lambda_kernel<double><<<grid, block, 0, st>>>(P, static_cast<const double*>(Q), lam_xi, lam_eta, cfl_max);
  else
    lambda_kernel<float><<<grid, block, 0, st>>>(P, static_cast<const float*>(Q), lam_xi, lam_eta, cfl_max);
  return cudaGetLastError();
}

__global__ void cfl_finish_kernel(const double* cfl_max, double cfl, double* dt_out) {
  *dt_out = cfl / *cfl_max;
}

cudaError_t launch_cfl_finish(const double* cfl_max, double cfl, double* dt_out, cudaStream_t st) {
  cfl_finish_kernel<<<1, 1, 0, st>>>(cfl_max, cfl, dt_out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Norms: per variable, root mean square and maximum of |A - B| over the interior nodes.
// acc[0..3] sums of squares, acc[4..7] maxima (bit-pattern atomic max of |e|).
// ------------------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(256) norms_kernel(int ni, int nj, long long ld, const Real* A,
                                                    const Real* B, double* acc) {
  __shared__ double red[2][8];
  const long long plane = (long long)nj * ld, N = (long long)ni * nj;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int v = 0; v < 4; ++v) {
    double s2 = 0.0, mx = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N;
         t += (long long)gridDim.x * blockDim.x) {
      const long long o = v * plane + (t / ni) * ld + (t % ni);
      double e = (double)A[o] - (B ? (double)B[o] : 0.0);
      s2 += e * e;
      mx = fmax(mx, fabs(e));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      s2 += __shfl_xor_sync(0xffffffffu, s2, off);
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    }
    if (lane == 0) { red[0][warp] = s2; red[1][warp] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < 8; ++w) { a += red[0][w]; b = fmax(b, red[1][w]); }
      atomicAdd(acc + v, a);
      atomic_max_pos(acc + 4 + v, b);
    }
    __syncthreads();
  }
}

// In place: acc = (sums[4], maxima[4]) -> out = (rms_0, max_0, rms_1, max_1, ...).
__global__ void norms_finish_kernel(double* acc, double n) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = acc[k];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    acc[2 * v] = sqrt(a[v] / n);
    acc[2 * v + 1] = a[4 + v];
  }
}

cudaError_t launch_norms(const fsp_block& blk, int precision, const void* A, const void* B,
                         double* out, cudaStream_t st) {
  // out doubles as the accumulator space, then is rewritten in place by one thread
  cudaError_t e = cudaMemsetAsync(out, 0, 8 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  const long long N = (long long)blk.ni * blk.nj;
  const long long want = (N + 255) / 256;
  const int grid = (int)(want < 152 * 4 ? want : 152 * 4);
  if (precision == FSP_FP64)
    norms_kernel<double><<<grid, 256, 0, st>>>(blk.ni, blk.nj, blk.ld, static_cast<const double*>(A),
                                               static_cast<const double*>(B), out);
  else
    norms_kernel<float><<<grid, 256, 0, st>>>(blk.ni, blk.nj, blk.ld, static_cast<const float*>(A),
                                              static_cast<const float*>(B), out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  norms_finish_kernel<<<1, 1, 0, st>>>(out, (double)N);
  return cudaGetLastError();
}

}  // namespace fsp
