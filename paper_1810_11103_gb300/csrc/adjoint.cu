// adjoint.cu -- the discrete adjoint (vector-Jacobian products) of the WENOIU right-hand
// side, of one TVD-RK3 step and of the metrics, FP64.
//
// Given gbar = dJ/d(dQ/dt), fsp_rhs_vjp adds dJ/dQ and dJ/dM:
//   1. the forward right-hand side (its line maxima and dQ/dt are needed);
//   2. dQ/dt = -(R_xi + R_eta) / J^-1  ->  Rbar = -gbar / J^-1, and the J^-1 term of Mbar;
//   3. per direction, vjp_sweep: each CTA stages the tile as the forward sweep does, then every
//      interface it owns recomputes its forward quantities in registers and runs them in
//      reverse (split midpoint fluxes, the two characteristic WENO interpolations down to the
//      stencil states, the primitives and the averaged direction), the node fluxes and the
//      linear h combination; contributions collect in shared memory and are added to global
//      memory, ghost contributions mapped back through the boundary rule;
//   4. the line maxima of the splitting: the subgradient of max picks the lowest index that
//      attains it (as the oracle's tangent does).
#include <climits>
#include <cstring>

#include "adjoint_device.cuh"
#include "fsp_internal.h"
#include "sweep.cuh"

namespace fsp {

// Ghost adjoint at position g of a line -> the interior it came from (boundary rules).
__device__ __forceinline__ void scatter_ghost(const Params& P, const double* __restrict__ Q, int dir, int line, int g,
                                              const double* qb, double* Qbar, double* Mbar) {
  const int n = dir == 0 ? P.ni : P.nj;
  const long long plane = (long long)P.nj * P.ld;
  auto add = [&](int gg, const double* v4) {
    const long long o = dir == 0 ? (long long)line * P.ld + gg : (long long)gg * P.ld + line;
#pragma unroll
    for (int v = 0; v < 4; ++v)
      if (v4[v] != 0.0) atomicAdd(Qbar + v * plane + o, v4[v]);
  };
  if (g >= 0 && g < n) { add(g, qb); return; }
  const int face = 2 * dir + (g < 0 ? 0 : 1);
  const int b = g < 0 ? 0 : n - 1;
  const int kind = P.bc[face];
  if (kind == BC_PERIODIC) { add(pmod(g, n), qb); return; }
  if (kind == BC_DIRICHLET) return;
  const double mx = dir == 0 ? met_at(P, 0, b, line) : met_at(P, 2, line, b);
  const double my = dir == 0 ? met_at(P, 1, b, line) : met_at(P, 3, line, b);
  if (kind == BC_SLIPWALL) {
    // ghost = Q(2b - g) with the momentum reflected about the unit normal n = m / |m|:
    // q' = q - 2 (q.n) n  ->  qbar = qbar' - 2 (qbar'.n) n, nbar = -2 [(qbar'.n) q + (q.n) qbar']
    const int sm = 2 * b - g;
    const long long o = dir == 0 ? (long long)line * P.ld + sm : (long long)sm * P.ld + line;
    const double q1 = Q[1 * plane + o], q2 = Q[2 * plane + o];
    const double inv = rsqrt(mx * mx + my * my);
    const double nx = mx * inv, ny = my * inv;
    const double pn = qb[1] * nx + qb[2] * ny, qn = q1 * nx + q2 * ny;
    const double r[4] = {qb[0], qb[1] - 2.0 * pn * nx, qb[2] - 2.0 * pn * ny, qb[3]};
    add(sm, r);
    const double nxb = -2.0 * (pn * q1 + qn * qb[1]), nyb = -2.0 * (pn * q2 + qn * qb[2]);
    const double dn = nx * nxb + ny * nyb;
    const double mxb = inv * (nxb - nx * dn), myb = inv * (nyb - ny * dn);
    const long long mo = dir == 0 ? (long long)(line + G) * P.mld + (b + G) : (long long)(b + G) * P.mld + (line + G);
    atomicAdd(Mbar + (2 * dir) * P.mplane + mo, mxb);
    atomicAdd(Mbar + (2 * dir + 1) * P.mplane + mo, myb);
    return;
  }
  if (kind == BC_FARFIELD) {
    const double vn = (g < 0 ? -1.0 : 1.0) * (P.bcq[face][1] * mx + P.bcq[face][2] * my);
    if (vn < 0.0) return;   // inflow: the prescribed state
  }
  add(b, qb);               // transmissive (and far-field outflow)
}

// Tile of the adjoint sweeps: the forward tiles' interface rows (xi 128 interfaces per line,
// eta 32) on half as many lines, for 128-thread CTAs with one interface per thread.  Two
// CTAs fit an SM (about 95 KB of shared memory and 31 K registers each), so the staging,
// node-flux and scatter phases of one overlap the FP64 interface work of the other.
template <int S, int DIR>
struct VjpTile {
  using Base = TileShape<S, DIR, double, double>;
  static constexpr int NL = Base::NL / 2;
  static constexpr int W = Base::W, T = Base::T, NP = Base::NP;
  static constexpr int THREADS = NL * W;
  static constexpr int NN = NL * NP;
  static constexpr size_t smem_bytes() { return sizeof(double) * (27 * (size_t)NN + NL + 4 * (size_t)WT * THREADS); }
};

template <int S, int DIR>
__global__ void __launch_bounds__(VjpTile<S, DIR>::THREADS, 2)
vjp_sweep_kernel(Params P, const double* __restrict__ Q, const double* __restrict__ lam,
                 const double* __restrict__ gbar, double* Qbar, double* Mbar, double* Abar) {
  using Sh = VjpTile<S, DIR>;
  using Sc = Scheme<S>;
  constexpr int NL = Sh::NL, W = Sh::W, T = Sh::T, NP = Sh::NP, NN = Sh::NN;
  constexpr int NMP = Sc::nmp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sQ = reinterpret_cast<double*>(smem_raw);  // [4][NN] state
  double* sM = sQ + 4 * NN;                          // [2][NN] direction metrics
  double* sP = sM + 2 * NN;                          // [7][NN] primitives
  double* sR = sP + 7 * NN;                          // [4][NN] Rbar
  double* sQb = sR + 4 * NN;                         // [4][NN] state adjoint
  double* sMb = sQb + 4 * NN;                        // [2][NN] metric adjoint
  double* sEb = sMb + 2 * NN;                        // [4][NN] node-flux adjoint
  double* sAb = sEb + 4 * NN;                        // [NL] A^ adjoint
  double* sTape = sAb + NL;                          // [4][WT][THREADS] WENO tapes
  Tape tape[4];
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) tape[kc] = Tape{sTape + kc * WT * Sh::THREADS + threadIdx.x, Sh::THREADS};

  const int n = DIR == 0 ? P.ni : P.nj;
  const int nlines = DIR == 0 ? P.nj : P.ni;
  const int line0 = blockIdx.y * NL;
  const int base = blockIdx.x * T;
  const double gamma = P.gamma, gm1 = gamma - 1.0, eps = P.eps;
  const long long plane = (long long)P.nj * P.ld;
  auto SI = [](int l, int s) { return DIR == 0 ? l * NP + s : s * NL + l; };

  if (threadIdx.x < NL) sAb[threadIdx.x] = 0.0;
  for (int k = threadIdx.x; k < NN; k += Sh::THREADS) {
    const int l = DIR == 0 ? k / NP : k % NL;
    const int s = DIR == 0 ? k % NP : k / NL;
    const int line = line0 + l;
    const int o = SI(l, s);
#pragma unroll
    for (int v = 0; v < 4; ++v) { sQb[v * NN + o] = 0.0; sEb[v * NN + o] = 0.0; sR[v * NN + o] = 0.0; }
    sMb[o] = 0.0;
    sMb[NN + o] = 0.0;
    if (line >= nlines) continue;
    const int graw = base + s - 4;
    const int g = min(graw, n + 3);
    double q[4];
    load_state(P, Q, DIR, line, g, q);
    const double mx = DIR == 0 ? met_at(P, 0, g, line) : met_at(P, 2, line, g);
    const double my = DIR == 0 ? met_at(P, 1, g, line) : met_at(P, 3, line, g);
    const Prim<double> w = prim_of(q, gamma);
#pragma unroll
    for (int v = 0; v < 4; ++v) sQ[v * NN + o] = q[v];
    sM[o] = mx;
    sM[NN + o] = my;
    sP[0 * NN + o] = w.u; sP[1 * NN + o] = w.v; sP[2 * NN + o] = w.c; sP[3 * NN + o] = w.cinv;
    sP[4 * NN + o] = w.H; sP[5 * NN + o] = w.b1; sP[6 * NN + o] = w.h2;
    if (graw >= 0 && graw < n) {
      const int i = DIR == 0 ? graw : line, j = DIR == 0 ? line : graw;
      const long long go = (long long)j * P.ld + i;
      const double mJ = -rcp_nr(met_at(P, 4, i, j));
#pragma unroll
      for (int v = 0; v < 4; ++v) sR[v * NN + o] = gbar[v * plane + go] * mJ;
    }
  }
  __syncthreads();

  // interfaces owned by this tile: interface p of the line goes to tile min(max(p,0),n-1)/T
  const int lo = blockIdx.x == 0 ? -NMP : base;
  const int hi = base + T >= n ? n - 2 + NMP : base + T - 1;
  for (int k = threadIdx.x; k < NL * W; k += Sh::THREADS) {
    const int l = DIR == 0 ? k / W : k % NL;
    const int pi = DIR == 0 ? k % W : k / NL;
    const int line = line0 + l;
    const int p = lo + pi;
    if (line >= nlines || p > hi) continue;
    const double A = P.alpha * lam[line];
    const int c0 = p - base + 4;  // staged position of node p
    auto Hb = [&](int c, int v) { return sR[v * NN + SI(l, c)] - sR[v * NN + SI(l, c + 1)]; };
    double fbp[4], fbm[4], Hp[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      Hp[v] = Hb(c0, v);
      fbp[v] = Sc::m0 * Hp[v] + (NMP == 2 ? Sc::m1 * Hb(c0 + 1, v) : 0.0);
      fbm[v] = Sc::m0 * Hp[v] + (NMP == 2 ? Sc::m1 * Hb(c0 - 1, v) : 0.0);
    }
    double Ab = 0.0;
    // node terms of h: n_k (E^ +- A Q)/2 at nodes p+k and p+1-k
#pragma unroll
    for (int kk = -3; kk <= 3; ++kk) {
      if (Sc::hn(kk) == 0.0) continue;
      const double cn = 0.5 * Sc::hn(kk);
      const int a = SI(l, c0 + kk), b = SI(l, c0 + 1 - kk);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const double h = cn * Hp[v];
        atomicAdd(sEb + v * NN + a, h);
        atomicAdd(sEb + v * NN + b, h);
        atomicAdd(sQb + v * NN + a, A * h);
        atomicAdd(sQb + v * NN + b, -A * h);
        Ab += h * (sQ[v * NN + a] - sQ[v * NN + b]);
      }
    }
    // midpoint metrics mm = sum_k c_k m(c0 - 2 + k) and the interface direction
    const int o0 = SI(l, c0), o1 = SI(l, c0 + 1);
    const double mbx = 0.5 * (sM[o0] + sM[o1]), mby = 0.5 * (sM[NN + o0] + sM[NN + o1]);
    const double rn = rsq(mbx * mbx + mby * mby);
    const double nx = mbx * rn, ny = mby * rn;
    // midpoint interpolation over nodes p-2..p+3, or p-3..p+4 for r = 4
    constexpr int NI = Sc::r == 4 ? 8 : 6, IOFF = Sc::r == 4 ? 3 : 2;
    double vx[NI], vy[NI];
#pragma unroll
    for (int kk = 0; kk < NI; ++kk) {
      const int o = SI(l, c0 - IOFF + kk);
      vx[kk] = sM[o];
      vy[kk] = sM[NN + o];
    }
    double mmx, mmy;
    if constexpr (Sc::r == 4) {
      mmx = mid_interp8(P.interp, vx);
      mmy = mid_interp8(P.interp, vy);
    } else {
      mmx = mid_interp(P.interp, Sc::r == 3, vx);
      mmy = mid_interp(P.interp, Sc::r == 3, vy);
    }
    double mmxb = 0.0, mmyb = 0.0, nxb = 0.0, nyb = 0.0;
    // each side: forward once (WENO internals to the tape), then its reverse
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
      const int oc = side == 0 ? o0 : o1;
      Prim<double> w;
      w.u = sP[0 * NN + oc]; w.v = sP[1 * NN + oc]; w.c = sP[2 * NN + oc]; w.cinv = sP[3 * NN + oc];
      w.H = sP[4 * NN + oc]; w.b1 = sP[5 * NN + oc]; w.h2 = sP[6 * NN + oc];
      const double qc[4] = {sQ[oc], sQ[NN + oc], sQ[2 * NN + oc], sQ[3 * NN + oc]};
      // stencil offsets -H..-1, +1..+H (H = 2, or 3 for r = 4); the "-" side mirrored
      constexpr int H = Sc::r == 4 ? 3 : 2, NA = 2 * H;
      double dq[NA][4];
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        const int m = a < H ? a - H : a - H + 1;
        if (Sc::r == 2 && m == 2) { dq[a][0] = dq[a][1] = dq[a][2] = dq[a][3] = 0.0; continue; }
        const int o = SI(l, side == 0 ? c0 + m : c0 + 1 - m);
#pragma unroll
        for (int v = 0; v < 4; ++v) dq[a][v] = sQ[v * NN + o] - qc[v];
      }
      Eig<double> E;
      E.build(w, nx, ny);
      double Wm[4], dQm[4], Qs[4];
#pragma unroll
      for (int kc = 0; kc < 4; ++kc) {
        double u[2 * H + 1];
#pragma unroll
        for (int a = 0; a < NA; ++a)
          u[a < H ? a : a + 1] = (Sc::r == 2 && a == 3) ? 0.0 : E.project(kc, dq[a][0], dq[a][1], dq[a][2], dq[a][3]);
        u[H] = 0.0;
        Wm[kc] = weno_fwd_tape<Sc::r>(u, eps, P.ppm, P.linw, tape[kc]);
      }
      E.recon(Wm, dQm);
#pragma unroll
      for (int v = 0; v < 4; ++v) Qs[v] = qc[v] + dQm[v];
      // split midpoint flux f = (E^(Qs; mm) + sg A Qs) / 2, reverse
      const double sg = side == 0 ? 1.0 : -1.0;
      const double* fb = side == 0 ? fbp : fbm;
      double eb[4], Qsb[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        eb[v] = 0.5 * fb[v];
        Qsb[v] = 0.5 * sg * A * fb[v];
        Ab += 0.5 * sg * fb[v] * Qs[v];
      }
      flux_bwd(Qs, mmx, mmy, gm1, eb, Qsb, mmxb, mmyb);
      // the characteristic interpolation, reverse
      double qcb[4] = {0, 0, 0, 0}, dqb[NA][4] = {};
      PrimBar pb{0, 0, 0, 0, 0, 0, 0};
      side_bwd_tape<Sc::r>(E, w, nx, ny, dq, Wm, P.ppm, P.linw, tape, Qsb, qcb, dqb, pb, nxb, nyb);
      prim_bwd(qc, gamma, pb, qcb);
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        const int m = a < H ? a - H : a - H + 1;
        if (Sc::r == 2 && m == 2) continue;
        const int o = SI(l, side == 0 ? c0 + m : c0 + 1 - m);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          atomicAdd(sQb + v * NN + o, dqb[a][v]);
          qcb[v] -= dqb[a][v];
        }
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) atomicAdd(sQb + v * NN + oc, qcb[v]);
    }
    // midpoint metrics, reverse
    {
      double cw[NI];
#pragma unroll
      for (int kk = 0; kk < NI; ++kk) cw[kk] = 0.0;
      if (P.interp == 1) { cw[IOFF] = cw[IOFF + 1] = 0.5; }
      else if (Sc::r == 4) {
        cw[0] = cw[7] = -5.0 / 2048; cw[1] = cw[6] = 49.0 / 2048; cw[2] = cw[5] = -245.0 / 2048;
        cw[3] = cw[4] = 1225.0 / 2048;
      }
      else if (Sc::r == 3) { cw[0] = cw[5] = 3.0 / 256; cw[1] = cw[4] = -25.0 / 256; cw[2] = cw[3] = 150.0 / 256; }
      else { cw[1] = cw[4] = -1.0 / 16; cw[2] = cw[3] = 9.0 / 16; }
#pragma unroll
      for (int kk = 0; kk < NI; ++kk) {
        if (cw[kk] == 0.0) continue;
        const int o = SI(l, c0 - IOFF + kk);
        atomicAdd(sMb + o, cw[kk] * mmxb);
        atomicAdd(sMb + NN + o, cw[kk] * mmyb);
      }
    }
    // direction n = mb / |mb|, mb = (m(p) + m(p+1)) / 2
    const double dn = nx * nxb + ny * nyb;
    const double mbxb = rn * (nxb - nx * dn), mbyb = rn * (nyb - ny * dn);
    atomicAdd(sMb + o0, 0.5 * mbxb);
    atomicAdd(sMb + o1, 0.5 * mbxb);
    atomicAdd(sMb + NN + o0, 0.5 * mbyb);
    atomicAdd(sMb + NN + o1, 0.5 * mbyb);
    atomicAdd(sAb + l, Ab);
  }
  __syncthreads();

  // node fluxes E^(Q; m), reverse
  for (int k = threadIdx.x; k < NN; k += Sh::THREADS) {
    const int l = DIR == 0 ? k / NP : k % NL;
    const int s = DIR == 0 ? k % NP : k / NL;
    if (line0 + l >= nlines) continue;
    const int o = SI(l, s);
    double eb[4] = {sEb[o], sEb[NN + o], sEb[2 * NN + o], sEb[3 * NN + o]};
    if (eb[0] == 0.0 && eb[1] == 0.0 && eb[2] == 0.0 && eb[3] == 0.0) continue;
    const double q[4] = {sQ[o], sQ[NN + o], sQ[2 * NN + o], sQ[3 * NN + o]};
    double qb[4] = {0, 0, 0, 0}, mxb = 0.0, myb = 0.0;
    flux_bwd(q, sM[o], sM[NN + o], gm1, eb, qb, mxb, myb);
#pragma unroll
    for (int v = 0; v < 4; ++v) sQb[v * NN + o] += qb[v];
    sMb[o] += mxb;
    sMb[NN + o] += myb;
  }
  __syncthreads();

  // scatter the tile's adjoints to global memory
  for (int k = threadIdx.x; k < NN; k += Sh::THREADS) {
    const int l = DIR == 0 ? k / NP : k % NL;
    const int s = DIR == 0 ? k % NP : k / NL;
    const int line = line0 + l;
    const int g = base + s - 4;
    if (line >= nlines || g > n + 3) continue;
    const int o = SI(l, s);
    const double qb[4] = {sQb[o], sQb[NN + o], sQb[2 * NN + o], sQb[3 * NN + o]};
    if (qb[0] != 0.0 || qb[1] != 0.0 || qb[2] != 0.0 || qb[3] != 0.0)
      scatter_ghost(P, Q, DIR, line, g, qb, Qbar, Mbar);
    const long long mo = DIR == 0 ? (long long)(line + G) * P.mld + (g + G) : (long long)(g + G) * P.mld + (line + G);
    if (sMb[o] != 0.0) atomicAdd(Mbar + (2 * DIR) * P.mplane + mo, sMb[o]);
    if (sMb[NN + o] != 0.0) atomicAdd(Mbar + (2 * DIR + 1) * P.mplane + mo, sMb[NN + o]);
  }
  if (threadIdx.x < NL && line0 + (int)threadIdx.x < nlines)
    atomicAdd(Abar + line0 + threadIdx.x, sAb[threadIdx.x]);
}

// J^-1 term: dQ/dt = -R / J^-1  ->  Mbar_J += sum_v gbar_v R_v / J^-2 = -sum_v gbar_v dQdt_v / J^-1
__global__ void jac_bwd_kernel(Params P, const double* __restrict__ gbar, const double* __restrict__ dqdt,
                               double* Mbar) {
  const long long N = (long long)P.ni * P.nj, plane = (long long)P.nj * P.ld;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % P.ni), j = (int)(t / P.ni);
    const long long o = (long long)j * P.ld + i;
    double s = 0.0;
#pragma unroll
    for (int v = 0; v < 4; ++v) s += gbar[v * plane + o] * dqdt[v * plane + o];
    Mbar[4 * P.mplane + (long long)(j + G) * P.mld + (i + G)] += -s / met_at(P, 4, i, j);
  }
}

// Line maxima: the lowest index attaining each maximum (recomputed with the forward's code).
__global__ void argmax_kernel(Params P, const double* __restrict__ Q, const double* __restrict__ lam_xi,
                              const double* __restrict__ lam_eta, int* arg_xi, int* arg_eta) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
  if (i >= P.ni || j >= P.nj) return;
  double sx, se, rate;
  node_speeds(P, Q, i, j, sx, se, rate);
  if (sx == lam_xi[j]) atomicMin(arg_xi + j, i);
  if (se == lam_eta[i]) atomicMin(arg_eta + i, j);
}

// Line maxima, reverse: A^ = alpha max_s sp(Q_s, m_s)  ->  the argmax node gets alpha Abar.
__global__ void lambda_bwd_kernel(Params P, const double* __restrict__ Q, const double* __restrict__ Abar,
                                  const int* __restrict__ arg_xi, const int* __restrict__ arg_eta, double* Qbar,
                                  double* Mbar) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P.ni + P.nj) return;
  const int dir = t < P.nj ? 0 : 1;
  const int line = dir == 0 ? t : t - P.nj;
  const int s = dir == 0 ? arg_xi[line] : arg_eta[line];
  const double ab = P.alpha * Abar[t];
  if (ab == 0.0 || s == INT_MAX) return;
  const int i = dir == 0 ? s : line, j = dir == 0 ? line : s;
  const long long plane = (long long)P.nj * P.ld, o = (long long)j * P.ld + i;
  double q[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) q[v] = Q[v * plane + o];
  double qb[4] = {0, 0, 0, 0}, mxb = 0.0, myb = 0.0;
  spectral_bwd(q, met_at(P, 2 * dir, i, j), met_at(P, 2 * dir + 1, i, j), P.gamma, ab, qb, mxb, myb);
#pragma unroll
  for (int v = 0; v < 4; ++v) atomicAdd(Qbar + v * plane + o, qb[v]);
  const long long mo = (long long)(j + G) * P.mld + (i + G);
  atomicAdd(Mbar + (2 * dir) * P.mplane + mo, mxb);
  atomicAdd(Mbar + (2 * dir + 1) * P.mplane + mo, myb);
}

// out = a x + b y (state-shaped, ld layout; y nullable)
__global__ void axpby_kernel(long long n, double a, const double* x, double b, const double* y, double* out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = a * x[t] + (y ? b * y[t] : 0.0);
}

template <int S, int DIR>
static cudaError_t launch_vjp_sweep(const Params& P, const double* Q, const double* lam, const double* gbar,
                                    double* Qbar, double* Mbar, double* Abar, cudaStream_t st) {
  using Sh = VjpTile<S, DIR>;
  const int n = DIR == 0 ? P.ni : P.nj, nlines = DIR == 0 ? P.nj : P.ni;
  dim3 grid((n + Sh::T - 1) / Sh::T, (nlines + Sh::NL - 1) / Sh::NL);
  const size_t smem = Sh::smem_bytes();
  auto kern = vjp_sweep_kernel<S, DIR>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, Sh::THREADS, smem, st>>>(P, Q, lam, gbar, Qbar, Mbar, Abar);
  return cudaGetLastError();
}

template <int S>
static cudaError_t vjp_scheme(const Params& P, const double* Q, const double* lx, const double* le,
                              const double* gbar, double* Qbar, double* Mbar, double* Abar, cudaStream_t st) {
  cudaError_t e = launch_vjp_sweep<S, 0>(P, Q, lx, gbar, Qbar, Mbar, Abar, st);
  if (e != cudaSuccess) return e;
  return launch_vjp_sweep<S, 1>(P, Q, le, gbar, Qbar, Mbar, Abar + P.nj, st);
}

// the transposed central operator: D phi_j = sum_k w[k+4] phi_{j+k}, k = -4..4
static void central_weights(int scheme, int interp, double alpha, double w[9]) {
  const Central c = central_of(scheme, alpha);
  double cl[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // I(m) = sum_l cl[l+3] phi_{m+l}, l = -3..4
  if (interp == 1) { cl[3] = cl[4] = 0.5; }
  else if (scheme == S71) {
    cl[0] = cl[7] = -5.0 / 2048; cl[1] = cl[6] = 49.0 / 2048; cl[2] = cl[5] = -245.0 / 2048;
    cl[3] = cl[4] = 1225.0 / 2048;
  }
  else if (scheme >= S51) { cl[1] = cl[6] = 3.0 / 256; cl[2] = cl[5] = -25.0 / 256; cl[3] = cl[4] = 150.0 / 256; }
  else { cl[2] = cl[5] = -1.0 / 16; cl[3] = cl[4] = 9.0 / 16; }
  auto C = [&](int l) { return (l >= -3 && l <= 4) ? cl[l + 3] : 0.0; };
  const double a[5] = {0.0, c.a1, c.a2, c.a3, c.a4};
  for (int k = -4; k <= 4; ++k) {
    double v = 0.0;
    if (k > 0) v += a[k];
    if (k < 0) v -= a[-k];
    v += c.b12 * (C(k) - C(k + 1)) + c.b32 * (C(k - 1) - C(k + 2));
    w[k + 4] = v;
  }
}

struct VjpCoord {
  int ni, nj, per_i, per_j;
  double pix, piy, pjx, pjy;   // period vectors per wrap in i and in j
};
struct W9 { double w[9]; };

// index a along a direction of n nodes -> up to two (index, weight) pairs and the wraps
__device__ __forceinline__ int resolve1(int a, int n, int per, int* idx, double* ww, int& cnt) {
  cnt = 1;
  if (a >= 0 && a < n) { idx[0] = a; ww[0] = 1.0; return 0; }
  if (per) { const int m = pmod(a, n); idx[0] = m; ww[0] = 1.0; return (a - m) / n; }
  const int b = a < 0 ? 0 : n - 1;
  idx[0] = b; ww[0] = 2.0; idx[1] = 2 * b - a; ww[1] = -1.0; cnt = 2;
  return 0;
}

// coordinate of node (i, j) of the extended grid (ghost rule as in metrics.cu)
__device__ __forceinline__ void coord_val(const VjpCoord& C, const double* x, const double* y, int i, int j,
                                          double& X, double& Y) {
  int ii[2], jj[2], ci, cj;
  double wi[2], wj[2];
  const int qi = resolve1(i, C.ni, C.per_i, ii, wi, ci), qj = resolve1(j, C.nj, C.per_j, jj, wj, cj);
  X = qi * C.pix + qj * C.pjx;
  Y = qi * C.piy + qj * C.pjy;
  for (int b = 0; b < cj; ++b)
    for (int a = 0; a < ci; ++a) {
      const long long o = (long long)jj[b] * C.ni + ii[a];
      X += wi[a] * wj[b] * x[o];
      Y += wi[a] * wj[b] * y[o];
    }
}

// adds f * (vx, vy) to the adjoints of the coordinates that node (i, j) is made of (the
// period offsets are constants and carry no adjoint)
__device__ __forceinline__ void coord_scatter(const VjpCoord& C, int i, int j, double f, double vx, double vy,
                                              double* xb, double* yb) {
  int ii[2], jj[2], ci, cj;
  double wi[2], wj[2];
  resolve1(i, C.ni, C.per_i, ii, wi, ci);
  resolve1(j, C.nj, C.per_j, jj, wj, cj);
  for (int b = 0; b < cj; ++b)
    for (int a = 0; a < ci; ++a) {
      const long long o = (long long)jj[b] * C.ni + ii[a];
      const double g = f * wi[a] * wj[b];
      if (vx != 0.0) atomicAdd(xb + o, g * vx);
      if (vy != 0.0) atomicAdd(yb + o, g * vy);
    }
}

// Metrics reverse.  Every derivative is D phi_j = sum_k w_k phi_{j+k} (the scheme's central
// operator with the midpoint interpolation folded in); xi_x^ = y_eta, xi_y^ = -x_eta,
// eta_x^ = -y_xi, eta_y^ = x_xi, J^-1 = x_xi y_eta - x_eta y_xi.
__global__ void metrics_vjp_kernel(VjpCoord C, const double* __restrict__ x, const double* __restrict__ y,
                                   const double* __restrict__ Mbar, W9 wts, double* xb, double* yb) {
  const int W = C.ni + 2 * G, H = C.nj + 2 * G;
  const long long plane = (long long)W * H;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < plane;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % W) - G, j = (int)(t / W) - G;
    const double M0 = Mbar[t], M1 = Mbar[plane + t], M2 = Mbar[2 * plane + t], M3 = Mbar[3 * plane + t],
                 M4 = Mbar[4 * plane + t];
    if (M0 == 0.0 && M1 == 0.0 && M2 == 0.0 && M3 == 0.0 && M4 == 0.0) continue;
    double xxi = 0.0, yxi = 0.0, xeta = 0.0, yeta = 0.0;
    if (M4 != 0.0) {
      for (int k = -4; k <= 4; ++k) {
        const double wk = wts.w[k + 4];
        if (wk == 0.0) continue;
        double X, Y;
        coord_val(C, x, y, i + k, j, X, Y);
        xxi += wk * X;
        yxi += wk * Y;
        coord_val(C, x, y, i, j + k, X, Y);
        xeta += wk * X;
        yeta += wk * Y;
      }
    }
    const double xxib = M3 + M4 * yeta, yetab = M0 + M4 * xxi;
    const double xetab = -M1 - M4 * yxi, yxib = -M2 - M4 * xeta;
    for (int k = -4; k <= 4; ++k) {
      const double wk = wts.w[k + 4];
      if (wk == 0.0) continue;
      coord_scatter(C, i + k, j, wk, xxib, yxib, xb, yb);
      coord_scatter(C, i, j + k, wk, xetab, yetab, xb, yb);
    }
  }
}

}  // namespace fsp

using namespace fsp;

namespace {

bool dptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t al(size_t b) { return (b + 255) / 256 * 256; }

// Adjoint workspace, after the forward part of fsp_workspace_size: dQ/dt, a metric-sized
// scratch, line-maxima adjoints and argmax indices, and four state buffers for the RK3 step.
// One recorded RK3 step: the stage states Q^n, Q^(1), Q^(2), their right-hand sides and
// their line maxima (xi lines then eta lines).
struct StepTape { size_t q[3], r[3], lam[3], total; };

StepTape step_tape(const fsp_block& b) {
  StepTape T;
  const size_t state = al(4 * (size_t)b.nj * b.ld * sizeof(double));
  const size_t lam = al(((size_t)b.ni + b.nj) * sizeof(double));
  size_t o = 0;
  for (int k = 0; k < 3; ++k) { T.q[k] = o; o += state; }
  for (int k = 0; k < 3; ++k) { T.r[k] = o; o += state; }
  for (int k = 0; k < 3; ++k) { T.lam[k] = o; o += lam; }
  T.total = o;
  return T;
}

// Adjoint workspace: the forward workspace, then dQ/dt, a metric adjoint for callers
// passing none, line-maximum adjoints and argmax indices, two state temporaries and one
// step tape (fsp_rk3_step_vjp records into it).
struct VjpWs { size_t fwd, dqdt, mbar, abar, arg, t3, gq, tape, total; };

VjpWs vjp_ws(const fsp_config& c, const fsp_block& b, size_t fwd_bytes) {
  VjpWs L;
  const size_t state = al(4 * (size_t)b.nj * b.ld * sizeof(double));
  const size_t met = al(5 * (size_t)(b.ni + 2 * G) * (b.nj + 2 * G) * sizeof(double));
  L.fwd = 0;
  L.dqdt = al(fwd_bytes);
  L.mbar = L.dqdt + state;
  L.abar = L.mbar + met;
  L.arg = L.abar + al(((size_t)b.ni + b.nj) * sizeof(double));
  L.t3 = L.arg + al(((size_t)b.ni + b.nj) * sizeof(int));
  L.gq = L.t3 + state;
  L.tape = L.gq + state;
  L.total = L.tape + step_tape(b).total;
  (void)c;
  return L;
}

bool adjoint_options(const fsp_config& c) {
  return c.scheme != S74 && c.weights == 0 && c.mid_split == 0 && scheme_alpha_of(c) == 1.0;
}

Params params_of(const fsp_config& c, const fsp_block& b, const double* metrics) {
  return make_params(c, b, metrics);
}

#define TRY(expr) \
  do { if ((expr) != cudaSuccess) return FSP_ERR_CUDA; } while (0)

}  // namespace

extern "C" fsp_status fsp_vjp_workspace_size(const fsp_config* cfg, const fsp_block* blk, size_t* bytes) {
  size_t fwd = 0;
  if (fsp_status s = fsp_workspace_size(cfg, blk, &fwd)) return s;
  if (cfg->precision != FSP_FP64 || !adjoint_options(*cfg)) return FSP_ERR_UNSUPPORTED;
  if (!bytes) return FSP_ERR_INVALID_ARG;
  *bytes = vjp_ws(*cfg, *blk, fwd).total;
  return FSP_OK;
}

// The reverse of one right-hand side at Q whose output R = dQ/dt and line maxima lam are
// given: gbar -> Qbar (+=), Mbar (+=).  Uses the abar and arg parts of the workspace.
static fsp_status vjp_core(const fsp_config& c, const fsp_block& b, const double* metrics, const double* Q,
                           const double* R, const double* lam, const double* gbar, double* Qbar, double* Mbar,
                           char* ws, const VjpWs& L, cudaStream_t st) {
  double* abar = reinterpret_cast<double*>(ws + L.abar);
  int* arg = reinterpret_cast<int*>(ws + L.arg);
  const Params P = params_of(c, b, metrics);
  TRY(cudaMemsetAsync(abar, 0, sizeof(double) * (b.ni + b.nj), st));
  TRY(cudaMemsetAsync(arg, 0x7f, sizeof(int) * (b.ni + b.nj), st));
  const long long N = (long long)b.ni * b.nj;
  const int g1 = stride_grid((N + 255) / 256, 8);
  jac_bwd_kernel<<<g1, 256, 0, st>>>(P, gbar, R, Mbar);
  TRY(cudaGetLastError());
  cudaError_t e;
  switch (c.scheme) {
    case S31: e = vjp_scheme<S31>(P, Q, lam, lam + b.nj, gbar, Qbar, Mbar, abar, st); break;
    case S32: e = vjp_scheme<S32>(P, Q, lam, lam + b.nj, gbar, Qbar, Mbar, abar, st); break;
    case S51: e = vjp_scheme<S51>(P, Q, lam, lam + b.nj, gbar, Qbar, Mbar, abar, st); break;
    case S52: e = vjp_scheme<S52>(P, Q, lam, lam + b.nj, gbar, Qbar, Mbar, abar, st); break;
    default:  e = vjp_scheme<S71>(P, Q, lam, lam + b.nj, gbar, Qbar, Mbar, abar, st); break;
  }
  TRY(e);
  dim3 blk(32, 8), grd((b.ni + 31) / 32, (b.nj + 7) / 8);
  argmax_kernel<<<grd, blk, 0, st>>>(P, Q, lam, lam + b.nj, arg, arg + b.nj);
  TRY(cudaGetLastError());
  // arg_xi is at arg[0..nj), arg_eta at arg[nj..); lambda_bwd reads them by line
  lambda_bwd_kernel<<<(b.ni + b.nj + 255) / 256, 256, 0, st>>>(P, Q, abar, arg, arg + b.nj, Qbar, Mbar);
  TRY(cudaGetLastError());
  return FSP_OK;
}

// gbar -> Qbar (+=), Mbar (+=): the forward right-hand side (for R and the line maxima,
// left at the start of the forward workspace), then the core
static fsp_status rhs_vjp_impl(const fsp_config& c, const fsp_block& b, const double* metrics, const double* Q,
                               const double* gbar, double* Qbar, double* Mbar, char* ws, size_t fwd_bytes,
                               cudaStream_t st) {
  const VjpWs L = vjp_ws(c, b, fwd_bytes);
  double* dqdt = reinterpret_cast<double*>(ws + L.dqdt);
  if (fsp_status s = fsp_rhs(&c, &b, metrics, Q, dqdt, ws, fwd_bytes, st)) return s;
  return vjp_core(c, b, metrics, Q, dqdt, reinterpret_cast<const double*>(ws), gbar, Qbar, Mbar, ws, L, st);
}

static int grid_of(long long n) { return stride_grid((n + 255) / 256, 8); }

// The stages of one TVD-RK3 step from the tape's Q^n (already in place), each right-hand
// side and its line maxima kept in the tape; Q^{n+1} written to qout when it is not null.
static fsp_status record_stages(const fsp_config& c, const fsp_block& b, const double* metrics, char* tape,
                                double dt, double* qout, char* ws, size_t fwd_bytes, cudaStream_t st) {
  const StepTape T = step_tape(b);
  const long long n = 4 * (long long)b.nj * b.ld;
  const size_t lam_bytes = sizeof(double) * ((size_t)b.ni + b.nj);
  auto Qk = [&](int k) { return reinterpret_cast<double*>(tape + T.q[k]); };
  auto Rk = [&](int k) { return reinterpret_cast<double*>(tape + T.r[k]); };
  for (int k = 0; k < 3; ++k) {
    if (fsp_status s = fsp_rhs(&c, &b, metrics, Qk(k), Rk(k), ws, fwd_bytes, st)) return s;
    TRY(cudaMemcpyAsync(tape + T.lam[k], ws, lam_bytes, cudaMemcpyDeviceToDevice, st));
    if (k == 0) {
      axpby_kernel<<<grid_of(n), 256, 0, st>>>(n, 1.0, Qk(0), dt, Rk(0), Qk(1));           // Q1 = Qn + dt R0
    } else if (k == 1) {
      axpby_kernel<<<grid_of(n), 256, 0, st>>>(n, 1.0, Qk(1), dt, Rk(1), Qk(2));           // Q1 + dt R1
      axpby_kernel<<<grid_of(n), 256, 0, st>>>(n, 0.75, Qk(0), 0.25, Qk(2), Qk(2));        // Q2
    } else if (qout) {
      axpby_kernel<<<grid_of(n), 256, 0, st>>>(n, 1.0, Qk(2), dt, Rk(2), qout);            // Q2 + dt R2
      axpby_kernel<<<grid_of(n), 256, 0, st>>>(n, 1.0 / 3.0, Qk(0), 2.0 / 3.0, qout, qout);  // Q^{n+1}
    }
    TRY(cudaGetLastError());
  }
  return FSP_OK;
}

// The reverse of a recorded step: a (in: dJ/dQ^{n+1}, out: dJ/dQ^n), Mbar +=.
static fsp_status reverse_stages(const fsp_config& c, const fsp_block& b, const double* metrics,
                                 const char* tape, double dt, double* a, double* Mbar, char* ws, const VjpWs& L,
                                 cudaStream_t st) {
  const StepTape T = step_tape(b);
  const long long n = 4 * (long long)b.nj * b.ld;
  const int grid = grid_of(n);
  auto Qk = [&](int k) { return reinterpret_cast<const double*>(tape + T.q[k]); };
  auto Rk = [&](int k) { return reinterpret_cast<const double*>(tape + T.r[k]); };
  auto Lk = [&](int k) { return reinterpret_cast<const double*>(tape + T.lam[k]); };
  double* t3 = reinterpret_cast<double*>(ws + L.t3);
  double* gq = reinterpret_cast<double*>(ws + L.gq);
  // Q^{n+1} = 1/3 Qn + 2/3 (Q2 + dt R(Q2)): Q2bar = 2/3 a + R_Q2^T (2/3 dt a); a -> 1/3 a
  axpby_kernel<<<grid, 256, 0, st>>>(n, 2.0 / 3.0 * dt, a, 0.0, nullptr, gq);
  axpby_kernel<<<grid, 256, 0, st>>>(n, 2.0 / 3.0, a, 0.0, nullptr, t3);
  if (fsp_status s = vjp_core(c, b, metrics, Qk(2), Rk(2), Lk(2), gq, t3, Mbar, ws, L, st)) return s;
  axpby_kernel<<<grid, 256, 0, st>>>(n, 1.0 / 3.0, a, 0.0, nullptr, a);
  // Q2 = 3/4 Qn + 1/4 (Q1 + dt R(Q1)): a += 3/4 Q2bar; Q1bar = 1/4 Q2bar + R_Q1^T (dt/4 Q2bar)
  axpby_kernel<<<grid, 256, 0, st>>>(n, 0.75, t3, 1.0, a, a);
  axpby_kernel<<<grid, 256, 0, st>>>(n, 0.25 * dt, t3, 0.0, nullptr, gq);
  axpby_kernel<<<grid, 256, 0, st>>>(n, 0.25, t3, 0.0, nullptr, t3);
  if (fsp_status s = vjp_core(c, b, metrics, Qk(1), Rk(1), Lk(1), gq, t3, Mbar, ws, L, st)) return s;
  // Q1 = Qn + dt R(Qn): a += Q1bar + R_Qn^T (dt Q1bar)
  axpby_kernel<<<grid, 256, 0, st>>>(n, 1.0, t3, 1.0, a, a);
  axpby_kernel<<<grid, 256, 0, st>>>(n, dt, t3, 0.0, nullptr, gq);
  if (fsp_status s = vjp_core(c, b, metrics, Qk(0), Rk(0), Lk(0), gq, a, Mbar, ws, L, st)) return s;
  TRY(cudaGetLastError());
  return FSP_OK;
}

// The adjoint covers the FP64 third- and fifth-order schemes (not WENOIU7-1MP) with the
// paper's weights, midpoint splitting and printed schemes (the ppm, linear-weight and
// interpolation options included).
static fsp_status check_vjp(const fsp_config* cfg, const fsp_block* blk, size_t* fwd) {
  if (fsp_status s = fsp_workspace_size(cfg, blk, fwd)) return s;
  if (cfg->precision != FSP_FP64 || !adjoint_options(*cfg)) return FSP_ERR_UNSUPPORTED;
  return FSP_OK;
}

extern "C" {

fsp_status fsp_rhs_vjp(const fsp_config* cfg, const fsp_block* blk, const double* metrics, const void* Q,
                       const void* dQdt_bar, void* Q_bar, double* metrics_bar, void* ws, size_t ws_bytes,
                       void* stream) {
  size_t fwd = 0;
  if (fsp_status s = check_vjp(cfg, blk, &fwd)) return s;
  if (!dptr(metrics) || !dptr(Q) || !dptr(dQdt_bar) || !dptr(Q_bar) || !dptr(ws) || (metrics_bar && !dptr(metrics_bar)))
    return FSP_ERR_INVALID_ARG;
  const VjpWs L = vjp_ws(*cfg, *blk, fwd);
  if (ws_bytes < L.total || reinterpret_cast<uintptr_t>(ws) % 256) return FSP_ERR_INVALID_ARG;
  char* w = static_cast<char*>(ws);
  cudaStream_t st = (cudaStream_t)stream;
  double* Mb = metrics_bar;
  if (!Mb) {
    Mb = reinterpret_cast<double*>(w + L.mbar);
    TRY(cudaMemsetAsync(Mb, 0, fsp_metrics_elems(blk) * sizeof(double), st));
  }
  return rhs_vjp_impl(*cfg, *blk, metrics, static_cast<const double*>(Q), static_cast<const double*>(dQdt_bar),
                      static_cast<double*>(Q_bar), Mb, w, fwd, st);
}

fsp_status fsp_rk3_step_vjp(const fsp_config* cfg, const fsp_block* blk, const double* metrics, const void* Q_n,
                            double dt, void* Q_bar, double* metrics_bar, void* ws, size_t ws_bytes, void* stream) {
  size_t fwd = 0;
  if (fsp_status s = check_vjp(cfg, blk, &fwd)) return s;
  if (!dptr(metrics) || !dptr(Q_n) || !dptr(Q_bar) || !dptr(ws) || (metrics_bar && !dptr(metrics_bar)))
    return FSP_ERR_INVALID_ARG;
  const VjpWs L = vjp_ws(*cfg, *blk, fwd);
  if (ws_bytes < L.total || reinterpret_cast<uintptr_t>(ws) % 256) return FSP_ERR_INVALID_ARG;
  char* w = static_cast<char*>(ws);
  cudaStream_t st = (cudaStream_t)stream;
  double* Mb = metrics_bar;
  if (!Mb) {
    Mb = reinterpret_cast<double*>(w + L.mbar);
    TRY(cudaMemsetAsync(Mb, 0, fsp_metrics_elems(blk) * sizeof(double), st));
  }
  char* tape = w + L.tape;
  TRY(cudaMemcpyAsync(tape + step_tape(*blk).q[0], Q_n, 4 * (size_t)blk->nj * blk->ld * sizeof(double),
                      cudaMemcpyDeviceToDevice, st));
  if (fsp_status s = record_stages(*cfg, *blk, metrics, tape, dt, nullptr, w, fwd, st)) return s;
  return reverse_stages(*cfg, *blk, metrics, tape, dt, static_cast<double*>(Q_bar), Mb, w, L, st);
}

fsp_status fsp_rk3_tape_size(const fsp_config* cfg, const fsp_block* blk, size_t* bytes) {
  size_t fwd = 0;
  if (fsp_status s = check_vjp(cfg, blk, &fwd)) return s;
  if (!bytes) return FSP_ERR_INVALID_ARG;
  *bytes = step_tape(*blk).total;
  return FSP_OK;
}

fsp_status fsp_rk3_step_record(const fsp_config* cfg, const fsp_block* blk, const double* metrics, void* Q,
                               double dt, void* tape, size_t tape_bytes, void* ws, size_t ws_bytes, void* stream) {
  size_t fwd = 0;
  if (fsp_status s = check_vjp(cfg, blk, &fwd)) return s;
  if (!dptr(metrics) || !dptr(Q) || !dptr(tape) || !dptr(ws)) return FSP_ERR_INVALID_ARG;
  if (tape_bytes < step_tape(*blk).total || reinterpret_cast<uintptr_t>(tape) % 256) return FSP_ERR_INVALID_ARG;
  if (ws_bytes < fwd || reinterpret_cast<uintptr_t>(ws) % 256) return FSP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  char* t = static_cast<char*>(tape);
  TRY(cudaMemcpyAsync(t + step_tape(*blk).q[0], Q, 4 * (size_t)blk->nj * blk->ld * sizeof(double),
                      cudaMemcpyDeviceToDevice, st));
  return record_stages(*cfg, *blk, metrics, t, dt, static_cast<double*>(Q), static_cast<char*>(ws), fwd, st);
}

fsp_status fsp_rk3_step_vjp_tape(const fsp_config* cfg, const fsp_block* blk, const double* metrics,
                                 const void* tape, size_t tape_bytes, double dt, void* Q_bar, double* metrics_bar,
                                 void* ws, size_t ws_bytes, void* stream) {
  size_t fwd = 0;
  if (fsp_status s = check_vjp(cfg, blk, &fwd)) return s;
  if (!dptr(metrics) || !dptr(tape) || !dptr(Q_bar) || !dptr(ws) || (metrics_bar && !dptr(metrics_bar)))
    return FSP_ERR_INVALID_ARG;
  if (tape_bytes < step_tape(*blk).total || reinterpret_cast<uintptr_t>(tape) % 256) return FSP_ERR_INVALID_ARG;
  const VjpWs L = vjp_ws(*cfg, *blk, fwd);
  if (ws_bytes < L.total || reinterpret_cast<uintptr_t>(ws) % 256) return FSP_ERR_INVALID_ARG;
  char* w = static_cast<char*>(ws);
  cudaStream_t st = (cudaStream_t)stream;
  double* Mb = metrics_bar;
  if (!Mb) {
    Mb = reinterpret_cast<double*>(w + L.mbar);
    TRY(cudaMemsetAsync(Mb, 0, fsp_metrics_elems(blk) * sizeof(double), st));
  }
  return reverse_stages(*cfg, *blk, metrics, static_cast<const char*>(tape), dt, static_cast<double*>(Q_bar), Mb,
                        w, L, st);
}

fsp_status fsp_metrics_vjp(const fsp_config* cfg, const fsp_block* blk, const double* x, const double* y,
                           const double* metrics_bar, double* x_bar, double* y_bar, void* stream) {
  size_t fwd = 0;
  if (fsp_status s = fsp_workspace_size(cfg, blk, &fwd)) return s;
  if (cfg->scheme == S74) return FSP_ERR_UNSUPPORTED;   // its operator reaches 6 nodes (the weights hold 4)
  if (!dptr(x) || !dptr(y) || !dptr(metrics_bar) || !dptr(x_bar) || !dptr(y_bar)) return FSP_ERR_INVALID_ARG;
  W9 w;
  central_weights(cfg->scheme, cfg->interp, scheme_alpha_of(*cfg), w.w);
  VjpCoord C{blk->ni, blk->nj, cfg->bc[0] == FSP_BC_PERIODIC, cfg->bc[2] == FSP_BC_PERIODIC,
             blk->period[0][0], blk->period[0][1], blk->period[1][0], blk->period[1][1]};
  const long long n = (long long)(blk->ni + 2 * G) * (blk->nj + 2 * G);
  const int grid = stride_grid((n + 255) / 256, 8);
  metrics_vjp_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(C, x, y, metrics_bar, w, x_bar, y_bar);
  return cudaGetLastError() == cudaSuccess ? FSP_OK : FSP_ERR_CUDA;
}

}  // extern "C"
