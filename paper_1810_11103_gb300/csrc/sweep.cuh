// sweep.cuh -- one direction of the WENOIU right-hand side (Li & Sun, arXiv:1810.11103,
// Sections 2.3, 3 and 3.4) as a tiled CUDA kernel, templated on the arithmetic:
//   Real  state, primitives, characteristic projection and WENO interpolation
//   Acc   metric products, fluxes, the h combination and the difference
// (double/double for FP64, float/float for FP32, float/double for FP32 with FP64 fluxes).
//
// A CTA owns NL grid lines x T output nodes of one direction.  Phase 1 stages every node of
// the tile plus four ghosts a side in shared memory: the state (ghosts by the boundary
// rule), the direction's metrics, the node split fluxes f+- = (E^ +- A^ Q)/2 and the
// primitives the characteristic projection needs.  Phase 2 gives each thread one interface p + 1/2: the eigenvectors at
// Q_p and Q_{p+1} along the averaged metric direction, WENO interpolation of the
// characteristic differences from both sides, the states Q+- at the midpoint, and the split
// midpoint fluxes with the interpolated midpoint metrics.  The h = h+ + h- combination and
// the difference H_{s+1/2} - H_{s-1/2} follow from shared memory; the epilogue writes the
// difference, dQ/dt, or a TVD-RK3 stage.
#pragma once

#include <type_traits>

#include "fsp_device.cuh"

namespace fsp {

enum { MODE_ACC = 0, MODE_RHS = 1, MODE_STAGE = 2 };

// Tile shapes: 256 threads, NL grid lines x W interface slots per CTA.  Variant 0 is the
// default; fsp_batch_tune may pick another per direction for a batch.
//   xi:  (NL, W) = (2, 128), (1, 256), (4, 64)
//   eta: (NL, W) = (8, 32),  (4, 64),  (16, 16)
constexpr int NVARIANT = 3;
constexpr int shape_nl(int dir, int v) {
  return dir == 0 ? (v == 1 ? 1 : v == 2 ? 4 : 2) : (v == 1 ? 4 : v == 2 ? 16 : 8);
}

template <int S, int DIR, typename Real, typename Acc, int V = 0>
struct TileShape {
  static constexpr int NL = shape_nl(DIR, V);       // grid lines per CTA
  static constexpr int W = 256 / NL;                 // interface slots per line
  static constexpr int NMP = Scheme<S>::nmp;
  static constexpr int T = W - NMP - 1;              // output nodes per line
  static constexpr int NP = T + 8;                   // staged nodes per line
  static constexpr int PLO = -NMP;                   // first interface p (of p + 1/2)
  static constexpr int THREADS = 256;
  static constexpr int NN = NL * NP, NW = NL * W;
  static constexpr bool SPLIT_MET = !std::is_same<Real, Acc>::value;
  static constexpr int NO = NL * T;                  // output nodes
  static constexpr size_t base_bytes() {
    return sizeof(Real) * ((size_t)(4 + 7) * NN + (SPLIT_MET ? 2 * NN : 0)) +
           sizeof(Acc) * ((size_t)(8 + 2) * NN + (size_t)4 * NW + (NMP == 2 ? (size_t)8 * NW : 0) + NL);
  }
  // epilogue operands prefetched per output node: the other direction's difference (modes
  // 1, 2), Q^n (mode 2), J^-1 (modes 1, 2); 16-byte aligned after the base regions
  static constexpr size_t ep_off() { return (base_bytes() + 15) / 16 * 16; }
  static constexpr size_t smem_bytes(int mode) {
    return mode == 0 ? base_bytes()
                     : ep_off() + (size_t)NO * (8 + 4 * sizeof(Acc) + (mode == 2 ? 4 * sizeof(Real) : 0));
  }
};

// Host view of the tile shape: output nodes per line T and lines per CTA NL.
inline void tile_dims(int scheme, int dir, int& T, int& NL, int variant = 0) {
  const int nmp = (scheme == S32 || scheme == S52) ? 2 : 1;
  NL = shape_nl(dir, variant);
  T = 256 / NL - nmp - 1;
}

// Asynchronous global-to-shared copies (cp.async, 4 or 8 bytes) of the epilogue operands.
template <int B>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sa), "l"(gmem), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// One tile (bx along the lines, by across them) of one block.  qtab: every block's state
// for linked faces (null for a lone block).
template <int S, int DIR, int MODE, typename Real, typename Acc, int V = 0>
__device__ __forceinline__ void sweep_tile(const Params& P, const Real* __restrict__ Q,
                                           const Real* const* qtab, const double* __restrict__ lam,
                                           const Acc* __restrict__ Dacc, Acc* __restrict__ Dout,
                                           Real* qout, const Real* Qn, double ca, double cb, double dt,
                                           int bx, int by) {
  using Sh = TileShape<S, DIR, Real, Acc, V>;
  using Sc = Scheme<S>;
  constexpr int NL = Sh::NL, W = Sh::W, T = Sh::T, NP = Sh::NP, PLO = Sh::PLO;
  constexpr int NN = Sh::NN, NW = Sh::NW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Acc* sFp = reinterpret_cast<Acc*>(smem_raw);           // [4][NN] node f+ = (E^ + A^ Q)/2
  Acc* sFm = sFp + 4 * NN;                               // [4][NN] node f- = (E^ - A^ Q)/2
  Acc* sMa = sFm + 4 * NN;                               // [2][NN] metrics (flux arithmetic)
  Acc* sH = sMa + 2 * NN;                                // [4][NW] h at interfaces
  Acc* sF = sH + 4 * NW;                                 // [8][NW] f+-_mid (two midpoints)
  Real* sQ = reinterpret_cast<Real*>(sF + (Sh::NMP == 2 ? 8 * NW : 0) + NL);  // [4][NN] (after A^)
  Real* sP = sQ + 4 * NN;                                // [7][NN] primitives
  Real* sMr = Sh::SPLIT_MET ? sP + 7 * NN : nullptr;     // [2][NN] metrics in Real
  Acc* sA = reinterpret_cast<Acc*>(smem_raw) + 10 * NN + 4 * NW + (Sh::NMP == 2 ? 8 * NW : 0);  // [NL] A^

  const int n = DIR == 0 ? P.ni : P.nj;
  const int nlines = DIR == 0 ? P.nj : P.ni;
  const int line0 = by * NL;
  const int base = bx * T;
  const Real gamma = Real(P.gamma);
  const Real eps = sizeof(Real) == 8 ? from_f64<Real>(P.eps) : from_f64<Real>(P.eps < 1e-30 ? 1e-30 : P.eps);
  const long long plane = (long long)P.nj * P.ld;

  auto SI = [](int l, int s) { return DIR == 0 ? l * NP + s : s * NL + l; };
  auto WI = [](int l, int p) { return DIR == 0 ? l * W + p : p * NL + l; };
  auto metR = [&](int c, int o) -> Real {
    if constexpr (Sh::SPLIT_MET) return sMr[c * NN + o];
    else return sMa[c * NN + o];
  };

  // A^ = alpha x line maximum, once per line (Section 2.3)
  if (threadIdx.x < NL) {
    const int line = line0 + threadIdx.x;
    sA[threadIdx.x] = line < nlines ? Acc(P.alpha * lam[line]) : Acc(0);
  }
  __syncthreads();
  // prefetch of the epilogue's global operands, issued now and consumed in the last phase
  // by the same thread (the node mapping of that phase)
  double* sJ = reinterpret_cast<double*>(smem_raw + Sh::ep_off());
  Acc* sDa = reinterpret_cast<Acc*>(sJ + Sh::NO);
  Real* sQn = reinterpret_cast<Real*>(sDa + 4 * Sh::NO);
  if constexpr (MODE != MODE_ACC) {
    for (int k = threadIdx.x; k < Sh::NO; k += Sh::THREADS) {
      const int l = DIR == 0 ? k / T : k % NL;
      const int s = DIR == 0 ? k % T : k / NL;
      const int line = line0 + l;
      const int g = base + s;
      if (line >= nlines || g >= n) continue;
      const int i = DIR == 0 ? g : line, j = DIR == 0 ? line : g;
      const long long o = (long long)j * P.ld + i;
      cp_async<8>(sJ + k, P.met + 4 * P.mplane + (long long)(j + G) * P.mld + (i + G));
#pragma unroll
      for (int v = 0; v < 4; ++v) cp_async<sizeof(Acc)>(sDa + v * Sh::NO + k, Dacc + v * plane + o);
      if constexpr (MODE == MODE_STAGE) {
#pragma unroll
        for (int v = 0; v < 4; ++v) cp_async<sizeof(Real)>(sQn + v * Sh::NO + k, Qn + v * plane + o);
      }
    }
    cp_async_commit();
  }
  // ---- phase 1: nodes ----
  for (int k = threadIdx.x; k < NN; k += Sh::THREADS) {
    const int l = DIR == 0 ? k / NP : k % NL;
    const int s = DIR == 0 ? k % NP : k / NL;
    const int line = line0 + l;
    if (line >= nlines) continue;
    const int g = min(base + s - 4, n + 3);  // positions past n+3 are never used
    Real q[4];
    load_state(P, Q, DIR, line, g, q, qtab);
    double mx, my;
    if (DIR == 0) { mx = met_at(P, 0, g, line); my = met_at(P, 1, g, line); }
    else          { mx = met_at(P, 2, line, g); my = met_at(P, 3, line, g); }
    const Prim<Real> w = prim_of(q, gamma);
    // E^ = mx E + my F with the metric products in Acc
    const Real p = (gamma - Real(1)) * (q[3] - q[0] * w.h2);
    const Acc amx = from_f64<Acc>(mx), amy = from_f64<Acc>(my);
    const Acc U = amx * Acc(w.u) + amy * Acc(w.v);
    const int o = SI(l, s);
    // f+- = (E^ +- A^ Q)/2, the node terms of the split
    const Acc hA = Acc(0.5) * sA[l];
    const Acc E[4] = {Acc(q[0]) * U, Acc(q[1]) * U + amx * Acc(p), Acc(q[2]) * U + amy * Acc(p), Acc(q[3] + p) * U};
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const Acc e = Acc(0.5) * E[v], aq = hA * Acc(q[v]);
      sFp[v * NN + o] = e + aq;
      sFm[v * NN + o] = e - aq;
    }
    sMa[o] = amx;
    sMa[NN + o] = amy;
    if constexpr (Sh::SPLIT_MET) { sMr[o] = from_f64<Real>(mx); sMr[NN + o] = from_f64<Real>(my); }
#pragma unroll
    for (int v = 0; v < 4; ++v) sQ[v * NN + o] = q[v];
    sP[0 * NN + o] = w.u; sP[1 * NN + o] = w.v; sP[2 * NN + o] = w.c; sP[3 * NN + o] = w.cinv;
    sP[4 * NN + o] = w.H; sP[5 * NN + o] = w.b1; sP[6 * NN + o] = w.h2;
  }
  __syncthreads();

  // ---- phase 2: interfaces p + 1/2 ----
  for (int k = threadIdx.x; k < NW; k += Sh::THREADS) {
    const int l = DIR == 0 ? k / W : k % NL;
    const int pi = DIR == 0 ? k % W : k / NL;
    const int line = line0 + l;
    const int p = PLO + pi;
    if (line >= nlines || base + p > n) continue;
    const Acc A = sA[l];
    const int c0 = p + 4;  // staged position of node p
    const int o0 = SI(l, c0), o1 = SI(l, c0 + 1);

    // characteristic direction: unit vector of the averaged metrics (Section 3.4)
    const Real mbx = Real(0.5) * (metR(0, o0) + metR(0, o1));
    const Real mby = Real(0.5) * (metR(1, o0) + metR(1, o1));
    const Real rn = rsq(mbx * mbx + mby * mby);
    const Real nx = mbx * rn, ny = mby * rn;

    Real Qs[2][4];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      // "+" side: eigenvectors at Q_p, stencil p-2..p+2; "-" side: at Q_{p+1}, mirrored
      const int oc = side == 0 ? o0 : o1;
      Prim<Real> w;
      w.u = sP[0 * NN + oc]; w.v = sP[1 * NN + oc]; w.c = sP[2 * NN + oc]; w.cinv = sP[3 * NN + oc];
      w.H = sP[4 * NN + oc]; w.b1 = sP[5 * NN + oc]; w.h2 = sP[6 * NN + oc];
      Eig<Real> E;
      E.build(w, nx, ny);
      const Real qc0 = sQ[oc], qc1 = sQ[NN + oc], qc2 = sQ[2 * NN + oc], qc3 = sQ[3 * NN + oc];
      // state differences to the centre at the stencil offsets -2, -1, +1, +2
      Real dq[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int m = a < 2 ? a - 2 : a - 1;
        if (Sc::r == 2 && m == 2) { dq[a][0] = dq[a][1] = dq[a][2] = dq[a][3] = Real(0); continue; }
        const int o = SI(l, side == 0 ? c0 + m : c0 + 1 - m);
        dq[a][0] = sQ[o] - qc0;
        dq[a][1] = sQ[NN + o] - qc1;
        dq[a][2] = sQ[2 * NN + o] - qc2;
        dq[a][3] = sQ[3 * NN + o] - qc3;
      }
      Real Wm[4];
      if constexpr (std::is_same<Real, float>::value) {
        // components (0, 1) and (2, 3) in the two lanes of packed float arithmetic
#pragma unroll
        for (int kp = 0; kp < 2; ++kp) {
          float2 u[5];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            if (Sc::r == 2 && a == 3) { u[4] = make_float2(0.f, 0.f); continue; }
            u[a < 2 ? a : a + 1] = make_float2(E.project(2 * kp, dq[a][0], dq[a][1], dq[a][2], dq[a][3]),
                                               E.project(2 * kp + 1, dq[a][0], dq[a][1], dq[a][2], dq[a][3]));
          }
          u[2] = make_float2(0.f, 0.f);
          const float2 W2 = weno_delta_x2<Sc::r>(u, eps, P.ppm, P.linw);
          Wm[2 * kp] = W2.x;
          Wm[2 * kp + 1] = W2.y;
        }
      } else {
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
          Real u[5];
          u[0] = E.project(kc, dq[0][0], dq[0][1], dq[0][2], dq[0][3]);
          u[1] = E.project(kc, dq[1][0], dq[1][1], dq[1][2], dq[1][3]);
          u[2] = Real(0);
          u[3] = E.project(kc, dq[2][0], dq[2][1], dq[2][2], dq[2][3]);
          u[4] = Sc::r == 3 ? E.project(kc, dq[3][0], dq[3][1], dq[3][2], dq[3][3]) : Real(0);
          Wm[kc] = weno_delta<Sc::r, Real>(u, eps, P.ppm, P.linw);
        }
      }
      Real dQm[4];
      E.recon(Wm, dQm);
      Qs[side][0] = qc0 + dQm[0];
      Qs[side][1] = qc1 + dQm[1];
      Qs[side][2] = qc2 + dQm[2];
      Qs[side][3] = qc3 + dQm[3];
    }

    // midpoint metrics by the same interpolation as the metric evaluation (Section 2.4)
    Acc vx[6], vy[6];
#pragma unroll
    for (int kk = 0; kk < 6; ++kk) {
      const int o = SI(l, c0 - 2 + kk);
      vx[kk] = sMa[o];
      vy[kk] = sMa[NN + o];
    }
    const Acc mmx = mid_interp(P.interp, Sc::r == 3, vx);
    const Acc mmy = mid_interp(P.interp, Sc::r == 3, vy);
    // split midpoint fluxes f+ = (E^(Q+) + A^ Q+)/2, f- = (E^(Q-) - A^ Q-)/2
    Acc fs[2][4];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const Real* q = Qs[side];
      const Real rinv = recip(q[0]);
      const Real u = q[1] * rinv, v = q[2] * rinv;
      const Real pr = (gamma - Real(1)) * (q[3] - Real(0.5) * (q[1] * u + q[2] * v));
      const Acc U = mmx * Acc(u) + mmy * Acc(v);
      const Acc sg = side == 0 ? A : -A;
      fs[side][0] = Acc(0.5) * (Acc(q[0]) * U + sg * Acc(q[0]));
      fs[side][1] = Acc(0.5) * (Acc(q[1]) * U + mmx * Acc(pr) + sg * Acc(q[1]));
      fs[side][2] = Acc(0.5) * (Acc(q[2]) * U + mmy * Acc(pr) + sg * Acc(q[2]));
      fs[side][3] = Acc(0.5) * (Acc(q[3] + pr) * U + sg * Acc(q[3]));
    }
    if constexpr (Sc::nmp == 1) {
      // h = h+ + h-: the midpoint terms plus the node terms n_k (f+_{p+k} + f-_{p+1-k}),
      // h- the mirror of h+ about p + 1/2
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        Acc h = Acc(Sc::m0) * (fs[0][v] + fs[1][v]);
#pragma unroll
        for (int kk = -2; kk <= 2; ++kk) {
          if (Sc::n(kk + 2) == 0.0) continue;
          const int a = SI(l, c0 + kk), b = SI(l, c0 + 1 - kk);
          h += Acc(Sc::n(kk + 2)) * (sFp[v * NN + a] + sFm[v * NN + b]);
        }
        sH[v * NW + WI(l, pi)] = h;
      }
    } else {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        sF[v * NW + WI(l, pi)] = fs[0][v];
        sF[(4 + v) * NW + WI(l, pi)] = fs[1][v];
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
      const int c0 = p + 4;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        Acc h = Acc(Sc::m0) * (sF[v * NW + WI(l, pi)] + sF[(4 + v) * NW + WI(l, pi)]) +
                Acc(Sc::m1) * (sF[v * NW + WI(l, pi - 1)] + sF[(4 + v) * NW + WI(l, pi + 1)]);
#pragma unroll
        for (int kk = -2; kk <= 2; ++kk) {
          if (Sc::n(kk + 2) == 0.0) continue;
          const int a = SI(l, c0 + kk), b = SI(l, c0 + 1 - kk);
          h += Acc(Sc::n(kk + 2)) * (sFp[v * NN + a] + sFm[v * NN + b]);
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
    Acc R[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) R[v] = sH[v * NW + WI(l, pi)] - sH[v * NW + WI(l, pi - 1)];
    if constexpr (MODE == MODE_ACC) {
#pragma unroll
      for (int v = 0; v < 4; ++v) Dout[v * plane + o] = R[v];
    } else {
      cp_async_wait_all();
      const Acc mJ = -recip(from_f64<Acc>(sJ[k]));
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const Acc d = (sDa[v * Sh::NO + k] + R[v]) * mJ;
        if constexpr (MODE == MODE_RHS) {
          qout[v * plane + o] = Real(d);
        } else {
          const Acc qs = Acc(sQ[v * NN + SI(l, s + 4)]);
          qout[v * plane + o] = Real(Acc(ca) * Acc(sQn[v * Sh::NO + k]) + Acc(cb) * (qs + Acc(dt) * d));
        }
      }
    }
  }
}

template <int S, int DIR, int MODE, typename Real, typename Acc>
__global__ void __launch_bounds__(256, sizeof(Real) == 8 ? 2 : 4)
sweep_kernel(Params P, const Real* __restrict__ Q, const double* __restrict__ lam,
             const Acc* __restrict__ Dacc, Acc* __restrict__ Dout, Real* qout, const Real* Qn,
             double ca, double cb, double dt) {
  sweep_tile<S, DIR, MODE, Real, Acc>(P, Q, nullptr, lam, Dacc, Dout, qout, Qn, ca, cb, dt, blockIdx.x,
                                      blockIdx.y);
}

// ---- many blocks in one launch: CTA b takes tile tiles[b] of block tiles[b].block ----
struct TileRef { int block, bx, by; };

template <typename Real, typename Acc>
struct BatchPass {                 // device arrays indexed by block
  const Params* params;
  const TileRef* tiles;
  const Real* const* q;            // state read by this pass (and by neighbours' ghosts)
  const double* const* lam;        // line maxima of the pass's direction
  const Acc* const* dacc;          // other direction's difference (modes 1, 2)
  Acc* const* dout;                // this direction's difference (mode 0)
  Real* const* qout;               // dQ/dt or the stage state (modes 1, 2)
  const Real* const* qn;           // Q^n of the RK step (mode 2)
};

template <int S, int DIR, int MODE, typename Real, typename Acc, int V>
__global__ void __launch_bounds__(256, sizeof(Real) == 8 ? 2 : 4)
sweep_batch_kernel(BatchPass<Real, Acc> B, double ca, double cb, double dt) {
  __shared__ Params sp;
  const TileRef t = B.tiles[blockIdx.x];
  if (threadIdx.x == 0) sp = B.params[t.block];
  __syncthreads();
  const int b = t.block;
  sweep_tile<S, DIR, MODE, Real, Acc, V>(sp, B.q[b], B.q, B.lam[b], MODE == MODE_ACC ? nullptr : B.dacc[b],
                                      MODE == MODE_ACC ? B.dout[b] : nullptr,
                                      MODE == MODE_ACC ? nullptr : B.qout[b],
                                      MODE == MODE_STAGE ? B.qn[b] : nullptr, ca, cb, dt, t.bx, t.by);
}

// Untyped pass tables (device arrays of per-block pointers) and their typed view.
struct PassTables {
  const void* params;
  const void* tiles;
  void* const* q;
  void* const* lam;
  void* const* dacc;
  void* const* dout;
  void* const* qout;
  void* const* qn;
};

template <typename Real, typename Acc>
BatchPass<Real, Acc> typed_pass(const PassTables& t) {
  BatchPass<Real, Acc> B;
  B.params = static_cast<const Params*>(t.params);
  B.tiles = static_cast<const TileRef*>(t.tiles);
  B.q = reinterpret_cast<const Real* const*>(t.q);
  B.lam = reinterpret_cast<const double* const*>(t.lam);
  B.dacc = reinterpret_cast<const Acc* const*>(t.dacc);
  B.dout = reinterpret_cast<Acc* const*>(t.dout);
  B.qout = reinterpret_cast<Real* const*>(t.qout);
  B.qn = reinterpret_cast<const Real* const*>(t.qn);
  return B;
}

template <int S, int DIR, int MODE, typename Real, typename Acc, int V>
cudaError_t launch_sweep_batch_v(const BatchPass<Real, Acc>& B, int ntiles, double ca, double cb, double dt,
                                 cudaStream_t st) {
  using Sh = TileShape<S, DIR, Real, Acc, V>;
  auto kern = sweep_batch_kernel<S, DIR, MODE, Real, Acc, V>;
  const size_t smem = Sh::smem_bytes(MODE);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (ntiles > 0) kern<<<ntiles, Sh::THREADS, smem, st>>>(B, ca, cb, dt);
  return cudaGetLastError();
}

template <int S, int DIR, int MODE, typename Real, typename Acc>
cudaError_t launch_sweep_batch(const BatchPass<Real, Acc>& B, int ntiles, int v, double ca, double cb, double dt,
                               cudaStream_t st) {
  switch (v) {
    case 1: return launch_sweep_batch_v<S, DIR, MODE, Real, Acc, 1>(B, ntiles, ca, cb, dt, st);
    case 2: return launch_sweep_batch_v<S, DIR, MODE, Real, Acc, 2>(B, ntiles, ca, cb, dt, st);
    default: return launch_sweep_batch_v<S, DIR, MODE, Real, Acc, 0>(B, ntiles, ca, cb, dt, st);
  }
}

template <int S, int DIR, int MODE, typename Real, typename Acc>
cudaError_t launch_sweep(const Params& P, const Real* Q, const double* lam, const Acc* Dacc, Acc* Dout,
                         Real* qout, const Real* Qn, double ca, double cb, double dt, cudaStream_t st) {
  using Sh = TileShape<S, DIR, Real, Acc>;
  const int n = DIR == 0 ? P.ni : P.nj, nlines = DIR == 0 ? P.nj : P.ni;
  dim3 grid((n + Sh::T - 1) / Sh::T, (nlines + Sh::NL - 1) / Sh::NL);
  const size_t smem = Sh::smem_bytes(MODE);
  auto kern = sweep_kernel<S, DIR, MODE, Real, Acc>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, Sh::THREADS, smem, st>>>(P, Q, lam, Dacc, Dout, qout, Qn, ca, cb, dt);
  return cudaGetLastError();
}

// Both directions for one scheme: xi into the accumulator, eta with the epilogue
// (mode 0: dQ/dt, mode 1: RK stage).
template <int S, typename Real, typename Acc>
cudaError_t rhs_passes(const Params& P, const Real* Q, const double* lam_xi, const double* lam_eta,
                       Acc* Racc, Real* out, int mode, const Real* Qn, double ca, double cb, double dt,
                       cudaStream_t st) {
  cudaError_t e = launch_sweep<S, 0, MODE_ACC, Real, Acc>(P, Q, lam_xi, nullptr, Racc, nullptr, nullptr,
                                                          0, 0, 0, st);
  if (e != cudaSuccess) return e;
  if (mode == 0)
    return launch_sweep<S, 1, MODE_RHS, Real, Acc>(P, Q, lam_eta, Racc, nullptr, out, nullptr, 0, 0, 0, st);
  return launch_sweep<S, 1, MODE_STAGE, Real, Acc>(P, Q, lam_eta, Racc, nullptr, out, Qn, ca, cb, dt, st);
}

// One direction through the public per-direction entry (mode 0: difference into D (Acc);
// mode 1: dQ/dt = -(acc + difference) / J^-1 into the state type).
template <int S, typename Real, typename Acc>
cudaError_t flux_difference_passes(const Params& P, const Real* Q, const double* lam, int dir, int mode,
                                   const Acc* acc, void* out, cudaStream_t st) {
  if (dir == 0)
    return mode == 0
               ? launch_sweep<S, 0, MODE_ACC, Real, Acc>(P, Q, lam, nullptr, static_cast<Acc*>(out), nullptr,
                                                         nullptr, 0, 0, 0, st)
               : launch_sweep<S, 0, MODE_RHS, Real, Acc>(P, Q, lam, acc, nullptr, static_cast<Real*>(out),
                                                         nullptr, 0, 0, 0, st);
  return mode == 0
             ? launch_sweep<S, 1, MODE_ACC, Real, Acc>(P, Q, lam, nullptr, static_cast<Acc*>(out), nullptr,
                                                       nullptr, 0, 0, 0, st)
             : launch_sweep<S, 1, MODE_RHS, Real, Acc>(P, Q, lam, acc, nullptr, static_cast<Real*>(out),
                                                       nullptr, 0, 0, 0, st);
}

// Both directions of every block for one scheme (mode 0: dQ/dt, mode 1: RK stage), xi tiles
// of shape variant vx, eta tiles of variant ve.
template <int S, typename Real, typename Acc>
cudaError_t batch_scheme(int mode, const PassTables& xi, int ntx, int vx, const PassTables& eta, int nte, int ve,
                         double ca, double cb, double dt, cudaStream_t st) {
  const BatchPass<Real, Acc> X = typed_pass<Real, Acc>(xi), E = typed_pass<Real, Acc>(eta);
  cudaError_t e = launch_sweep_batch<S, 0, MODE_ACC, Real, Acc>(X, ntx, vx, 0, 0, 0, st);
  if (e != cudaSuccess) return e;
  if (mode == 0) return launch_sweep_batch<S, 1, MODE_RHS, Real, Acc>(E, nte, ve, 0, 0, 0, st);
  return launch_sweep_batch<S, 1, MODE_STAGE, Real, Acc>(E, nte, ve, ca, cb, dt, st);
}

template <typename Real, typename Acc>
cudaError_t batch_dispatch(int scheme, int mode, const PassTables& xi, int ntx, int vx, const PassTables& eta,
                           int nte, int ve, double ca, double cb, double dt, cudaStream_t st) {
  switch (scheme) {
    case S31: return batch_scheme<S31, Real, Acc>(mode, xi, ntx, vx, eta, nte, ve, ca, cb, dt, st);
    case S32: return batch_scheme<S32, Real, Acc>(mode, xi, ntx, vx, eta, nte, ve, ca, cb, dt, st);
    case S51: return batch_scheme<S51, Real, Acc>(mode, xi, ntx, vx, eta, nte, ve, ca, cb, dt, st);
    default:  return batch_scheme<S52, Real, Acc>(mode, xi, ntx, vx, eta, nte, ve, ca, cb, dt, st);
  }
}

// One direction of every block into dout (mode 0 tiles of variant v), with the current line
// maxima.
template <typename Real, typename Acc>
cudaError_t batch_one_direction(int scheme, int dir, const PassTables& t, int ntiles, int v, cudaStream_t st) {
  const BatchPass<Real, Acc> B = typed_pass<Real, Acc>(t);
  switch (scheme * 2 + dir) {
    case 0: return launch_sweep_batch<S31, 0, MODE_ACC, Real, Acc>(B, ntiles, v, 0, 0, 0, st);
    case 1: return launch_sweep_batch<S31, 1, MODE_ACC, Real, Acc>(B, ntiles, v, 0, 0, 0, st);
    case 2: return launch_sweep_batch<S32, 0, MODE_ACC, Real, Acc>(B, ntiles, v, 0, 0, 0, st);
    case 3: return launch_sweep_batch<S32, 1, MODE_ACC, Real, Acc>(B, ntiles, v, 0, 0, 0, st);
    case 4: return launch_sweep_batch<S51, 0, MODE_ACC, Real, Acc>(B, ntiles, v, 0, 0, 0, st);
    case 5: return launch_sweep_batch<S51, 1, MODE_ACC, Real, Acc>(B, ntiles, v, 0, 0, 0, st);
    case 6: return launch_sweep_batch<S52, 0, MODE_ACC, Real, Acc>(B, ntiles, v, 0, 0, 0, st);
    default: return launch_sweep_batch<S52, 1, MODE_ACC, Real, Acc>(B, ntiles, v, 0, 0, 0, st);
  }
}
// Batch passes (shape variants vx, ve for the xi and eta tiles): FP64 in batch_fp64.cu;
// FP32 and mixed in batch_fp32.cu and batch_mixed.cu.
cudaError_t batch_fp64(int scheme, int mode, const PassTables& xi, int ntx, int vx, const PassTables& eta, int nte,
                       int ve, double ca, double cb, double dt, cudaStream_t st);
cudaError_t batch_direction_fp64(int scheme, int dir, const PassTables& t, int ntiles, int v, cudaStream_t st);
cudaError_t batch_fp32(int scheme, bool mixed, int mode, const PassTables& xi, int ntx, int vx,
                       const PassTables& eta, int nte, int ve, double ca, double cb, double dt, cudaStream_t st);
cudaError_t batch_direction_fp32(int scheme, bool mixed, int dir, const PassTables& t, int ntiles, int v,
                                 cudaStream_t st);
cudaError_t batch_mixed(int scheme, int mode, const PassTables& xi, int ntx, int vx, const PassTables& eta,
                        int nte, int ve, double ca, double cb, double dt, cudaStream_t st);
cudaError_t batch_direction_mixed(int scheme, int dir, const PassTables& t, int ntiles, int v, cudaStream_t st);

// Precision instantiations: each lives in its own translation unit.
cudaError_t rhs_fp64(int scheme, const Params& P, const void* Q, const double* lx, const double* le,
                     void* Racc, void* out, int mode, const void* Qn, double ca, double cb, double dt,
                     cudaStream_t st);
cudaError_t rhs_fp32(int scheme, bool mixed, const Params& P, const void* Q, const double* lx,
                     const double* le, void* Racc, void* out, int mode, const void* Qn, double ca,
                     double cb, double dt, cudaStream_t st);
cudaError_t flux_difference_fp64(int scheme, const Params& P, const void* Q, const double* lam, int dir,
                                 int mode, const void* acc, void* out, cudaStream_t st);
cudaError_t flux_difference_fp32(int scheme, bool mixed, const Params& P, const void* Q, const double* lam,
                                 int dir, int mode, const void* acc, void* out, cudaStream_t st);

}  // namespace fsp
