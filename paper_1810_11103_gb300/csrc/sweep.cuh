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

// MODE_STAGE_L: the RK stage of the marching eta pass that also takes the next stage's line
// maxima (Section 2.3's A^ of both directions) from the states it writes.
enum { MODE_ACC = 0, MODE_RHS = 1, MODE_STAGE = 2, MODE_STAGE_L = 3 };

// Tile shapes: 256 threads, NL grid lines x W interface slots per CTA.  Variant 0 is the
// default; fsp_batch_tune may pick another per direction for a batch.
//   xi:  (NL, W) = (2, 128), (1, 256), (4, 64); variant 3: marching warps (below)
//   eta: (NL, W) = (8, 32),  (4, 64),  (16, 16); variant 3: marching CTAs (below)
constexpr int NVARIANT = 4;                         // variants of each pass
constexpr int MARCH = 3;                            // the marching variant (xi and eta)
constexpr int nvariant(int) { return NVARIANT; }
constexpr int shape_nl(int dir, int v) {
  return dir == 0 ? (v == 1 ? 1 : v == 2 ? 4 : 2) : (v == 1 ? 4 : v == 2 ? 16 : 8);
}

// Shared-memory vectors of 16 bytes.  A 4-value quantity of node o is one float4 (FP32) or
// two double2 held in two arrays of n entries (FP64), so a warp reading consecutive nodes
// issues conflict-free 128-bit loads.
template <typename T>
__device__ __forceinline__ void st4(T* b, int n, int o, T a0, T a1, T a2, T a3) {
  if constexpr (sizeof(T) == 4) {
    reinterpret_cast<float4*>(b)[o] = make_float4(a0, a1, a2, a3);
  } else {
    reinterpret_cast<double2*>(b)[o] = make_double2(a0, a1);
    reinterpret_cast<double2*>(b + 2 * n)[o] = make_double2(a2, a3);
  }
}
template <typename T>
__device__ __forceinline__ void ld4(const T* b, int n, int o, T v[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 t = reinterpret_cast<const float4*>(b)[o];
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
    const double2 s = reinterpret_cast<const double2*>(b)[o], t = reinterpret_cast<const double2*>(b + 2 * n)[o];
    v[0] = s.x; v[1] = s.y; v[2] = t.x; v[3] = t.y;
  }
}
template <typename T>
__device__ __forceinline__ void st2(T* b, int o, T a0, T a1) {
  if constexpr (sizeof(T) == 4) reinterpret_cast<float2*>(b)[o] = make_float2(a0, a1);
  else reinterpret_cast<double2*>(b)[o] = make_double2(a0, a1);
}
template <typename T>
__device__ __forceinline__ void ld2(const T* b, int o, T& x, T& y) {
  if constexpr (sizeof(T) == 4) { const float2 t = reinterpret_cast<const float2*>(b)[o]; x = t.x; y = t.y; }
  else { const double2 t = reinterpret_cast<const double2*>(b)[o]; x = t.x; y = t.y; }
}

// Staged node data of n nodes (tile positions or ring slots), 16-byte vectors:
//   fp, fm  twice the split node fluxes, 2 f+- = E^ +- A^ Q (Acc, 4 values; the 1/2 is taken
//           in h_combine); in mixed precision fp holds the metric-weighted flux E^ and there
//           is no fm
//   ma      direction metrics in Acc (2 values)
//   q       state (Real, 4 values)
//   p0..p2  the node's characteristic data (NodeChar: 12 values)
//   mr      direction metrics rounded to Real (only when Real differs from Acc)
template <typename Real, typename Acc>
struct Staged {
  static constexpr bool SPLIT = !std::is_same<Real, Acc>::value;
  Acc *fp, *fm, *ma;
  Real *q, *p0, *p1, *p2, *mr;
  int n;
  // arrays of padded length (a multiple of 4 nodes keeps every array 16-byte aligned)
  static constexpr int padded(int nn) { return (nn + 3) / 4 * 4; }
  static constexpr size_t bytes(int nn) {
    return sizeof(Acc) * (size_t)padded(nn) * (SPLIT ? 6 : 10) +
           sizeof(Real) * (size_t)padded(nn) * (16 + (SPLIT ? 2 : 0));
  }
  __device__ __forceinline__ void carve(unsigned char* base, int nn0) {
    const int nn = padded(nn0);
    n = nn;
    fp = reinterpret_cast<Acc*>(base);
    fm = SPLIT ? nullptr : fp + 4 * nn;
    ma = fp + (SPLIT ? 4 : 8) * nn;
    q = reinterpret_cast<Real*>(ma + 2 * nn);
    p0 = q + 4 * nn;
    p1 = p0 + 4 * nn;
    p2 = p1 + 4 * nn;
    mr = SPLIT ? p2 + 4 * nn : nullptr;
  }
  __device__ __forceinline__ void store(int o, const Real qq[4], const NodeChar<Real>& w, Acc amx, Acc amy,
                                        const Acc f[4], const Acc g[4], double mx, double my) const {
    st4(fp, n, o, f[0], f[1], f[2], f[3]);
    if constexpr (!SPLIT) st4(fm, n, o, g[0], g[1], g[2], g[3]);
    st2(ma, o, amx, amy);
    if constexpr (SPLIT) st2(mr, o, from_f64_int(mx), from_f64_int(my));
    st4(q, n, o, qq[0], qq[1], qq[2], qq[3]);
    st4(p0, n, o, w.u, w.v, w.hc, w.a10);
    st4(p1, n, o, w.b1u, w.b1v, w.b1, w.cs);
    st4(p2, n, o, w.us, w.vs, w.Hs, w.h2s);
  }
  __device__ __forceinline__ void met_real(int o, Real& x, Real& y) const {
    if constexpr (SPLIT) ld2(mr, o, x, y);
    else ld2(ma, o, x, y);
  }
  __device__ __forceinline__ void chr(int o, NodeChar<Real>& w) const {
    Real a[4], b[4], c[4];
    ld4(p0, n, o, a);
    ld4(p1, n, o, b);
    ld4(p2, n, o, c);
    w.u = a[0]; w.v = a[1]; w.hc = a[2]; w.a10 = a[3];
    w.b1u = b[0]; w.b1v = b[1]; w.b1 = b[2]; w.cs = b[3];
    w.us = c[0]; w.vs = c[1]; w.Hs = c[2]; w.h2s = c[3];
  }
};

// What the h combination needs from one interface (midpoint p + 1/2).  Same precision: f[0],
// f[1] = twice the split midpoint fluxes, 2 f+, 2 f- (the 1/2 is taken in h_combine).  Mixed: f[s] = E^(Q_s) = mm_x E(Q_s) + mm_y F(Q_s)
// (double products of float Cartesian fluxes) and q[s] = Q_s, s = +, -; for one-midpoint
// schemes only their combinations are kept: f[0] = (E^(Q+) + E^(Q-))/2, q[0] = Q+ - Q-.
template <typename Real, typename Acc>
struct Mid {
  Acc f[2][4];
  Real q[2][4];
};

// Midpoint records of two-midpoint schemes in shared memory: per interface and side the 4
// Acc values of Mid::f and, in mixed precision, the 4 Real values of Mid::q; nw interfaces.
template <typename Real, typename Acc>
struct MidStore {
  Acc* f;      // [2 sides][4][nw] (16-byte vectors)
  Real* q;     // [2 sides][4][nw] (mixed precision only)
  int nw;
  static constexpr size_t bytes(int nw) {
    return (sizeof(Acc) + (Staged<Real, Acc>::SPLIT ? sizeof(Real) : 0)) * 8 * (size_t)nw;
  }
  __device__ __forceinline__ void carve(unsigned char* base, int n) {
    nw = n;
    f = reinterpret_cast<Acc*>(base);
    q = Staged<Real, Acc>::SPLIT ? reinterpret_cast<Real*>(f + 8 * n) : nullptr;
  }
  __device__ __forceinline__ void put(int o, const Mid<Real, Acc>& m) const {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      st4(f + 4 * nw * s, nw, o, m.f[s][0], m.f[s][1], m.f[s][2], m.f[s][3]);
      if constexpr (Staged<Real, Acc>::SPLIT) st4(q + 4 * nw * s, nw, o, m.q[s][0], m.q[s][1], m.q[s][2], m.q[s][3]);
    }
  }
  // side s of interface o into m (the other side is left alone)
  __device__ __forceinline__ void get(int o, int s, Mid<Real, Acc>& m) const {
    ld4(f + 4 * nw * s, nw, o, m.f[s]);
    if constexpr (Staged<Real, Acc>::SPLIT) ld4(q + 4 * nw * s, nw, o, m.q[s]);
  }
};

template <int S, int DIR, typename Real, typename Acc, int V = 0>
struct TileShape {
  static constexpr int NL = shape_nl(DIR, V);       // grid lines per CTA
  static constexpr int W = 256 / NL;                 // interface slots per line
  static constexpr int NMP = Scheme<S>::nmp;
  // the four-midpoint scheme: h at p + 1/2 takes the midpoints p - 3/2 .. p + 5/2, whose
  // stencils reach six nodes beyond the outputs; the others reach four
  static constexpr bool FOUR = NMP == 4;
  static constexpr int OFF = FOUR ? 6 : 4;           // staged ghost nodes on each side
  static constexpr int T = FOUR ? W - 5 : W - NMP - 1;   // output nodes per line
  static constexpr int NP = T + 2 * OFF;             // staged nodes per line
  static constexpr int PLO = FOUR ? -3 : -NMP;       // first interface p (of p + 1/2)
  static constexpr int THREADS = 256;
  static constexpr int NN = NL * NP, NW = NL * W;
  static constexpr int NO = NL * T;                  // output nodes
  // shared memory: staged nodes, then h (4 Acc per interface), the two-midpoint fluxes
  // f+- (8 Acc per interface, two-midpoint schemes), A^ per line
  static constexpr size_t o_h() { return Staged<Real, Acc>::bytes(NN); }
  static constexpr size_t o_f() { return o_h() + sizeof(Acc) * 4 * (size_t)NW; }
  static constexpr size_t o_a() { return o_f() + (NMP >= 2 ? MidStore<Real, Acc>::bytes(NW) : 0); }
  static constexpr size_t base_bytes() { return (o_a() + sizeof(Acc) * NL + 15) / 16 * 16; }
  // epilogue operands prefetched per output node: the other direction's difference (modes
  // 1, 2), Q^n (mode 2), J^-1 (modes 1, 2); 16-byte aligned after the base regions
  static constexpr size_t ep_off() { return base_bytes(); }
  static constexpr size_t smem_bytes(int mode) {
    return mode == 0 ? base_bytes()
                     : ep_off() + (size_t)NO * (8 + 4 * sizeof(Acc) + (mode == 2 ? 4 * sizeof(Real) : 0));
  }
};

// Marching xi pass: each warp owns one grid row segment of at most MARCH_SEG nodes and
// walks along it 32 nodes at a time; four warps (four rows of one block) per CTA.  The
// marching passes (xi and eta) are compiled for the default options only (ppm = 1,
// linear_weights = 0, interp = 0); a batch with other options runs the tile variants.
constexpr int MARCH_WARPS = 4;
constexpr int MARCH_SEG = 512;
constexpr int RING = 64;                             // node ring slots per warp
__host__ __device__ constexpr int march_seg_len(int n) {
  const int nseg = (n + MARCH_SEG - 1) / MARCH_SEG;
  const int per = (n + nseg - 1) / nseg;
  return (per + 31) / 32 * 32;
}
// Whether the marching xi pass evaluates the interface sides per centre node (centre_sides,
// which shares each node's stencil differences between its two sides) or per interface
// (interface_mid, both sides of one interface in one lane).  Same results either way.  The
// FP64 pass is bound by its FP64 instructions, which the centre layout cuts (9.12 against
// 9.48 ms on the 64-block cylinder); the float passes are bound by issue at 80-102 registers,
// where the centre layout's extra live state costs more than it saves (FP32 0.212 against
// 0.207 ms).
template <typename Real>
constexpr bool march_centres() { return sizeof(Real) == 8; }

template <int S, typename Real, typename Acc>
struct MarchShape {
  static constexpr int NMP = Scheme<S>::nmp;
  // per warp: the node ring, h per ring slot (4 Acc), f+- at the midpoints (two-midpoint
  // schemes, 8 Acc per slot), Q+ of the interface to the right of each centre node (4 Real
  // per slot), and the raw node prefetch (state, two metrics) of 32 lanes
  static constexpr size_t o_h() { return Staged<Real, Acc>::bytes(RING); }
  static constexpr size_t o_f() { return o_h() + sizeof(Acc) * 4 * RING; }
  static constexpr size_t o_qp() { return o_f() + (NMP == 2 ? MidStore<Real, Acc>::bytes(RING) : 0); }
  static constexpr size_t o_raw() { return o_qp() + (march_centres<Real>() ? sizeof(Real) * 4 * RING : 0); }
  static constexpr size_t warp_bytes() { return o_raw() + 32 * (4 * sizeof(Real) + 16); }
  static constexpr size_t smem_bytes() { return MARCH_WARPS * warp_bytes(); }
};

constexpr int EW = 8;                               // warps (rows per step) of a marching eta CTA
// Whether the marching eta pass evaluates the interface sides per centre node (centre_sides,
// as the FP64 xi pass does): FP64 one-midpoint schemes, whose pass is bound by its FP64
// instructions.  A step then takes the centres r - 1 + w and the interfaces one row behind
// them, so a segment of whole steps ends one output earlier (126 rows in sixteen steps).
__host__ __device__ constexpr bool march_eta_centres(bool fp64, int nmp) { return fp64 && nmp == 1; }
// Steps per segment: sixteen (FP64), 32 (float paths).  Each CTA stages its segment's first
// rows and waits for its first cp.async round trip before the steps overlap them, a cost that
// longer segments spread over more rows; on the 64-block cylinder the eta pass took FP64
// 8.05 -> 7.95 ms (8 -> 16 steps) and FP32 0.250 -> 0.229 -> 0.226 ms (8 -> 16 -> 32 steps).
__host__ __device__ constexpr int march_eta_steps(bool fp64) { return fp64 ? 16 : 32; }
__host__ __device__ constexpr int march_eta_seg(bool fp64, int nmp) {
  return march_eta_steps(fp64) * EW - (2 * nmp - 1) - (march_eta_centres(fp64, nmp) ? 1 : 0);
}

// Host view of the tile shape: output nodes per line T and lines per CTA NL (for the
// marching variant: rows per CTA, and the longest segment a warp walks).
inline void tile_dims(int scheme, int dir, int& T, int& NL, int variant = 0, bool fp64 = false) {
  const int nmp = (scheme == S32 || scheme == S52) ? 2 : 1;
  if (dir == 0 && variant == MARCH) { NL = MARCH_WARPS; T = MARCH_SEG; return; }
  if (dir == 1 && variant == MARCH) { NL = 32; T = march_eta_seg(fp64, nmp); return; }
  NL = shape_nl(dir, variant);
  T = scheme == S74 ? 256 / NL - 5 : 256 / NL - nmp - 1;
}

// Asynchronous global-to-shared copies (cp.async, 4 or 8 bytes).
template <int B>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sa), "l"(gmem), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// --------------------------------------------------------------------------------------
// Per-node and per-interface arithmetic, shared by the tile and the marching kernels (the
// same operations in the same order, so every layout gives the same results)
// Grid-static data of one interface that a batch stores once per step (FP64 and mixed passes):
// the midpoint metrics (mid) and, for FP64, the unit characteristic direction (dir).
struct IfacePre {
  bool mid = false, dir = false;
  double mx = 0.0, my = 0.0, nx = 0.0, ny = 0.0;
};

// --------------------------------------------------------------------------------------
// A node (Section 2.3).  Same precision throughout (Real = Acc): primitives of the projection
// and the split fluxes f+- = (E^ +- A^ Q)/2, E^ = mx E + my F, stored in fp and fm.  Mixed
// precision (float state, double Acc): only the metric-weighted flux E^ = mx E + my F, with the
// Cartesian fluxes E, F in float and the two metric products in double, stored in fp; the
// dissipative part A^ Q of the split is taken at the interfaces from the staged state.
// The split fluxes from the node's characteristic data w and pressure p, already formed.
template <typename Real, typename Acc>
__device__ __forceinline__ void node_split_from(const Real q[4], const NodeChar<Real>& w, Real p, double mx,
                                                double my, Acc hA, Acc& amx, Acc& amy, Acc fp[4], Acc fm[4]);

template <int SC, typename Real, typename Acc>
__device__ __forceinline__ void node_split(const Real q[4], double mx, double my, Real gamma, Acc hA,
                                           NodeChar<Real>& w, Acc& amx, Acc& amy, Acc fp[4], Acc fm[4]) {
  Real p;
  w = node_char<Real, SC>(q, gamma, p);
  node_split_from<Real, Acc>(q, w, p, mx, my, hA, amx, amy, fp, fm);
}

// The characteristic data of an FP64 node as the xi pass stores it for the eta pass of the same
// right-hand side (NC_COUNT planes: the twelve NodeChar values, then the pressure).
constexpr int NC_COUNT = 13;
__device__ __forceinline__ void nc_put(double* b, long long plane, long long o, const NodeChar<double>& w, double p) {
  const double v[NC_COUNT] = {w.u, w.v, w.hc, w.a10, w.b1u, w.b1v, w.b1, w.cs, w.us, w.vs, w.Hs, w.h2s, p};
#pragma unroll
  for (int k = 0; k < NC_COUNT; ++k) b[k * plane + o] = v[k];
}
__device__ __forceinline__ void nc_get(const double* b, long long stride, NodeChar<double>& w, double& p) {
  w.u = b[0]; w.v = b[stride]; w.hc = b[2 * stride]; w.a10 = b[3 * stride];
  w.b1u = b[4 * stride]; w.b1v = b[5 * stride]; w.b1 = b[6 * stride]; w.cs = b[7 * stride];
  w.us = b[8 * stride]; w.vs = b[9 * stride]; w.Hs = b[10 * stride]; w.h2s = b[11 * stride];
  p = b[12 * stride];
}

template <typename Real, typename Acc>
__device__ __forceinline__ void node_split_from(const Real q[4], const NodeChar<Real>& w, Real p, double mx,
                                                double my, Acc hA, Acc& amx, Acc& amy, Acc fp[4], Acc fm[4]) {
  amx = from_f64<Acc>(mx);
  amy = from_f64<Acc>(my);
  if constexpr (Staged<Real, Acc>::SPLIT) {
    const Real ex[4] = {q[1], q[1] * w.u + p, q[2] * w.u, (q[3] + p) * w.u};
    const Real ey[4] = {q[2], q[1] * w.v, q[2] * w.v + p, (q[3] + p) * w.v};
#pragma unroll
    for (int v = 0; v < 4; ++v) fp[v] = amx * widen<Acc>(ex[v]) + amy * widen<Acc>(ey[v]);
  } else {
    // twice the split fluxes, E^ +- A^ Q (the 1/2 is taken in h_combine)
    const Acc U = amx * Acc(w.u) + amy * Acc(w.v);
    const Acc E[4] = {Acc(q[0]) * U, Acc(q[1]) * U + amx * Acc(p), Acc(q[2]) * U + amy * Acc(p),
                      Acc(q[3] + p) * U};
    const Acc A = hA + hA;
    if constexpr (std::is_same<Acc, float>::value) {
#pragma unroll
      for (int v = 0; v < 4; v += 2) {
        const float2 e = make_float2(E[v], E[v + 1]), qq = make_float2(q[v], q[v + 1]);
        const float2 a = fma2(bc2(A), qq, e), b = fma2(bc2(-A), qq, e);
        fp[v] = a.x; fp[v + 1] = a.y;
        fm[v] = b.x; fm[v + 1] = b.y;
      }
    } else {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        fp[v] = fma(A, Acc(q[v]), E[v]);
        fm[v] = fma(-A, Acc(q[v]), E[v]);
      }
    }
  }
}

// The midpoint part of interface p + 1/2 from its two reconstructed states Qs[0] = Q+ and
// Qs[1] = Q-: the midpoint metrics interpolated as in the metric evaluation (Section 2.4) and
// the midpoint fluxes (Section 2.3); at(m) gives the staged index of node p + m.
// msplit (same precision only): 1 Steger-Warming, 2 Van Leer splitting of the midpoint flux
// (an option beyond the paper's, Section 7) instead of the Lax-Friedrichs type.
// pr.mid: the midpoint metrics were interpolated once per step by the batch (FP64 and mixed
// passes, IfacePre); otherwise they are interpolated here from the staged nodes.
template <int S, typename Real, typename Acc, typename At>
__device__ __forceinline__ void mid_fluxes(const Staged<Real, Acc>& st, const At& at, const Real Qs[2][4], Real gamma,
                                           int interp, Acc A, Mid<Real, Acc>& mo, int msplit = 0,
                                           const IfacePre& pr = IfacePre{}) {
  using Sc = Scheme<S>;
  Acc mmx, mmy;
  if (pr.mid) {
    mmx = Acc(pr.mx);
    mmy = Acc(pr.my);
  } else if constexpr (Sc::r == 4) {
    Acc vx[8], vy[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) ld2(st.ma, at(kk - 3), vx[kk], vy[kk]);
    mmx = mid_interp8(interp, vx);
    mmy = mid_interp8(interp, vy);
  } else {
    Acc vx[6], vy[6];
#pragma unroll
    for (int kk = 0; kk < 6; ++kk) ld2(st.ma, at(kk - 2), vx[kk], vy[kk]);
    mmx = mid_interp(interp, Sc::r == 3, vx);
    mmy = mid_interp(interp, Sc::r == 3, vy);
  }
  if constexpr (Staged<Real, Acc>::SPLIT) {
    // Cartesian fluxes of Q+ and Q- in float
    Real ex[2][4], ey[2][4];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const Real* q = Qs[side];
      const Real rinv = recip(q[0]);
      const Real u = q[1] * rinv, v = q[2] * rinv;
      const Real pr = (gamma - Real(1)) * (q[3] - Real(0.5) * (q[1] * u + q[2] * v));
      ex[side][0] = q[1]; ex[side][1] = q[1] * u + pr; ex[side][2] = q[2] * u; ex[side][3] = (q[3] + pr) * u;
      ey[side][0] = q[2]; ey[side][1] = q[1] * v; ey[side][2] = q[2] * v + pr; ey[side][3] = (q[3] + pr) * v;
    }
    if constexpr (Sc::nmp == 1) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        mo.f[0][v] = mmx * widen<Acc>(Real(0.5) * (ex[0][v] + ex[1][v])) +
                     mmy * widen<Acc>(Real(0.5) * (ey[0][v] + ey[1][v]));
        mo.q[0][v] = Qs[0][v] - Qs[1][v];
      }
    } else {
#pragma unroll
      for (int side = 0; side < 2; ++side)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          mo.f[side][v] = mmx * widen<Acc>(ex[side][v]) + mmy * widen<Acc>(ey[side][v]);
          mo.q[side][v] = Qs[side][v];
        }
    }
  } else {
    if (msplit) {
      split_mid2<Real>(msplit, 1, Qs[0], mmx, mmy, gamma, mo.f[0]);
      split_mid2<Real>(msplit, -1, Qs[1], mmx, mmy, gamma, mo.f[1]);
      return;
    }
    // twice the split midpoint fluxes: E^(Q+) + A^ Q+ and E^(Q-) - A^ Q-, with
    // E^ = (rho U, rho u U + mx p, rho v U + my p, (E + p) U)
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const Real* q = Qs[side];
      const Real rinv = recip(q[0]);
      const Real u = q[1] * rinv, v = q[2] * rinv;
      const Real pr = (gamma - Real(1)) * (q[3] - Real(0.5) * (q[1] * u + q[2] * v));
      const Acc U = mmx * Acc(u) + mmy * Acc(v);
      const Acc Us = side == 0 ? U + A : U - A;
      mo.f[side][0] = Acc(q[0]) * Us;
      mo.f[side][1] = fma(Acc(q[1]), Us, mmx * Acc(pr));
      mo.f[side][2] = fma(Acc(q[2]), Us, mmy * Acc(pr));
      mo.f[side][3] = fma(Acc(q[3]), Us, Acc(pr) * U);
    }
  }
}

// The WENO interpolation of one side's four characteristic components from their
// differences wd[a][k] at the stencil offsets -H..-1, +1..+H (the result scaled by
// weno_scale<R>); FP32 runs components (0, 1) and (2, 3) in the two lanes of packed float
// arithmetic.
template <int R, typename Real, bool NOSEL = false>
__device__ __forceinline__ void side_weno(const Real (*wd)[4], Real eps, int ppm, int linw, Real Wm[4], int wz = 0) {
  constexpr int H = R == 4 ? 3 : 2, NA = 2 * H;
  if constexpr (std::is_same<Real, float>::value) {
#pragma unroll
    for (int kp = 0; kp < 2; ++kp) {
      float2 u[NA + 1];
#pragma unroll
      for (int a = 0; a < NA; ++a) u[a < H ? a : a + 1] = make_float2(wd[a][2 * kp], wd[a][2 * kp + 1]);
      u[H] = make_float2(0.f, 0.f);
      const float2 W2 = weno_delta_x2<R, NOSEL>(u, eps, ppm, linw, wz);
      Wm[2 * kp] = W2.x;
      Wm[2 * kp + 1] = W2.y;
    }
  } else {
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      Real u[NA + 1];
#pragma unroll
      for (int a = 0; a < NA; ++a) u[a < H ? a : a + 1] = wd[a][kc];
      u[H] = Real(0);
      Wm[kc] = weno_delta<R, Real>(u, eps, ppm, linw, wz);
    }
  }
}

// Unit characteristic direction of interface p + 1/2 from the staged metrics of nodes p and
// p + 1 (the average's factor 1/2 cancels in the normalisation).
template <typename Real, typename Acc>
__device__ __forceinline__ void char_direction(const Staged<Real, Acc>& st, int o0, int o1, Real& nx, Real& ny) {
  Real m0x, m0y, m1x, m1y;
  st.met_real(o0, m0x, m0y);
  st.met_real(o1, m1x, m1y);
  const Real mbx = m0x + m1x, mby = m0y + m1y;
  const Real rn = rsq(mbx * mbx + mby * mby);
  nx = mbx * rn;
  ny = mby * rn;
}

// The two interface sides centred at node c (at(m) = the staged index of node c + m): the
// "+" side of interface c + 1/2 (eigenvectors of Q_c along n+ = n_{c+1/2}, stencil c-H..c+H)
// and the "-" side of interface c - 1/2 (eigenvectors of Q_c along n- = n_{c-1/2}, the
// mirrored stencil).  Both read the same state differences, whose direction-free projection
// part is taken once; each side's arithmetic is that of interface_mid, so the results agree
// bit for bit.  Qp = Q+_{c+1/2}, Qm = Q-_{c-1/2}.
template <int S, typename Real, typename Acc, typename At>
__device__ __forceinline__ void centre_sides(const Staged<Real, Acc>& st, const At& at, Real npx, Real npy,
                                             Real nmx, Real nmy, Real eps, Real Qp[4], Real Qm[4]) {
  using Sc = Scheme<S>;
  constexpr int SC = weno_scale<Sc::r>();
  constexpr int H = Sc::r == 4 ? 3 : 2, NA = 2 * H;
  const int oc = at(0);
  NodeChar<Real> w;
  st.chr(oc, w);
  Real qc[4];
  ld4(st.q, st.n, oc, qc);
  CharDir<Real, SC> Ep, Em;
  Ep.build(w, npx, npy);
  Em.build(w, nmx, nmy);
  // neighbour k = -H..-1, 1..H at index a (k = a - H, or a - H + 1): difference and common part
  Real d[NA][4], cA[NA], cS[NA];
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    const int k = a < H ? a - H : a - H + 1;
    Real t[4];
    ld4(st.q, st.n, at(k), t);
    if constexpr (std::is_same<Real, float>::value) {
#pragma unroll
      for (int v = 0; v < 4; v += 2) {
        const float2 dd = fma2(make_float2(qc[v], qc[v + 1]), bc2(-1.0f), make_float2(t[v], t[v + 1]));
        d[a][v] = dd.x;
        d[a][v + 1] = dd.y;
      }
    } else {
#pragma unroll
      for (int v = 0; v < 4; ++v) d[a][v] = t[v] - qc[v];
    }
    char_common(w, d[a], cA[a], cS[a]);
  }
  // "+" side: offset m reads neighbour m; "-" side: offset m reads neighbour -m (index NA-1-a)
  Real wp[NA][4], wm[NA][4];
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    const int m = a < H ? a - H : a - H + 1;
    if (Sc::r == 2 && m == 2) {
#pragma unroll
      for (int v = 0; v < 4; ++v) wp[a][v] = wm[a][v] = Real(0);
      continue;
    }
    Ep.project(d[a], cA[a], cS[a], wp[a]);
    Em.project(d[NA - 1 - a], cA[NA - 1 - a], cS[NA - 1 - a], wm[a]);
  }
  Real Wp[4], Wm[4];
  side_weno<Sc::r, Real>(wp, eps, 1, 0, Wp);
  side_weno<Sc::r, Real>(wm, eps, 1, 0, Wm);
  Ep.recon(Wp, qc, Qp);
  Em.recon(Wm, qc, Qm);
}

// The interface p + 1/2 between staged nodes at(0) (node p) and at(1) (node p + 1); at(m)
// gives the staged index of node p + m, m = -2..3.  Characteristic direction from the
// averaged metrics (Section 3.4), eigenvectors at Q_p ("+" side, stencil p-2..p+2) and at
// Q_{p+1} ("-" side, the mirror), WENO interpolation of the characteristic differences, the
// states Q+- at the midpoint, and the midpoint fluxes with the midpoint metrics interpolated
// as in the metric evaluation (Section 2.4).
// DEF: the configuration options take their defaults as compile-time constants (mapped
// nonlinear weights, order-matched midpoint interpolation), so the marching kernels carry no
// branches on them; the tile kernels read them at run time.
template <int S, typename Real, typename Acc, bool DEF = false, typename At>
__device__ __forceinline__ void interface_mid(const Staged<Real, Acc>& st, const At& at, Real gamma, Real eps,
                                              int ppm_, int linw_, int interp_, Acc A, Mid<Real, Acc>& mo,
                                              int wz_ = 0, int msplit_ = 0, const IfacePre& pr = IfacePre{}) {
  using Sc = Scheme<S>;
  constexpr int SC = weno_scale<Sc::r>();
  const int ppm = DEF ? 1 : ppm_, linw = DEF ? 0 : linw_, interp = DEF ? 0 : interp_;
  const int wz = DEF ? 0 : wz_, msplit = DEF ? 0 : msplit_;
  const int o0 = at(0), o1 = at(1);
  Real nx, ny;
  if constexpr (std::is_same<Real, double>::value) {
    if (pr.dir) { nx = pr.nx; ny = pr.ny; }
    else char_direction(st, o0, o1, nx, ny);
  } else {
    char_direction(st, o0, o1, nx, ny);
  }

  Real Qs[2][4];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int oc = side == 0 ? o0 : o1;
    NodeChar<Real> w;
    st.chr(oc, w);
    CharSide<Real, SC> E;
    E.build(w, nx, ny);
    Real qc[4];
    ld4(st.q, st.n, oc, qc);
    // characteristic differences to the centre at the stencil offsets -H..-1, +1..+H (H = 2,
    // or 3 for r = 4); the "-" side reads the mirrored nodes
    constexpr int H = Sc::r == 4 ? 3 : 2, NA = 2 * H;
    Real wd[NA][4];
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      const int m = a < H ? a - H : a - H + 1;
      if (Sc::r == 2 && m == 2) { wd[a][0] = wd[a][1] = wd[a][2] = wd[a][3] = Real(0); continue; }
      Real t[4];
      ld4(st.q, st.n, at(side == 0 ? m : 1 - m), t);
      E.project(t[0] - qc[0], t[1] - qc[1], t[2] - qc[2], t[3] - qc[3], wd[a]);
    }
    Real Wm[4];
    side_weno<Sc::r, Real, std::is_same<Acc, float>::value>(wd, eps, ppm, linw, Wm, wz);
    E.recon(Wm, qc, Qs[side]);
  }

  mid_fluxes<S, Real, Acc>(st, at, Qs, gamma, interp, A, mo, msplit, pr);
}

// h+ coefficient n_k of the node flux f+_{p+k} (0 outside the scheme's stencil)
template <int S>
__host__ __device__ constexpr double hnode(int k) { return Scheme<S>::hn(k); }

// The halved h+ coefficients of the h combination: the printed scheme's as compile-time
// constants (RT false: the marching kernels), or those at the free parameter of the
// one-midpoint forms from the kernel parameters (RT true: the tile kernels).  The stencil's
// support is the same for every alpha, so which terms exist stays a compile-time fact.
template <int S, bool RT>
struct HalfCoef {
  const Params& P;
  __device__ __forceinline__ double m0() const { return RT ? P.hc[0] : 0.5 * Scheme<S>::m0; }
  __device__ __forceinline__ double m1() const { return RT ? P.hc[1] : 0.5 * Scheme<S>::m1; }
  __device__ __forceinline__ double n(int k) const { return RT ? P.hc[5 + k] : 0.5 * Scheme<S>::hn(k); }
  __device__ __forceinline__ float m0f() const { return RT ? P.hcf[0] : float(0.5 * Scheme<S>::m0); }
  __device__ __forceinline__ float m1f() const { return RT ? P.hcf[1] : float(0.5 * Scheme<S>::m1); }
  __device__ __forceinline__ float nf(int k) const { return RT ? P.hcf[5 + k] : float(0.5 * Scheme<S>::hn(k)); }
};

// h = h+ + h- at p + 1/2 (Eqs. 3.4, 3.8, 3.16, 3.20; h- the mirror of h+), the midpoint
// terms m0 (f+_{p+1/2} + f-_{p+1/2}) + m1 (f+_{p-1/2} + f-_{p+3/2}) plus the node terms
// n_k (f+_{p+k} + f-_{p+1-k}), from the staged and midpoint values of 2 f+- (coefficients
// halved).  `c` is the interface p + 1/2; for two-midpoint schemes
// `lo` holds the plus side at p - 1/2 and `hi` the minus side at p + 3/2.
// Mixed precision: with f+- = (E^ +- A^ Q)/2 the terms regroup into a central part in the
// metric-weighted fluxes, (1/2) sum_d (n_{-d} + n_{1+d}) (E^_{p-d} + E^_{p+1+d}) plus the
// midpoint means, taken in double, and a dissipative part in the states,
// (A^/2) [sum_d (n_{-d} - n_{1+d}) (Q_{p-d} - Q_{p+1+d}) + m0 (Q+ - Q-) + m1 (Q+_{p-1/2} -
// Q-_{p+3/2})], taken in float.  In a uniform flow every state difference is exactly zero,
// so the free-stream residual is that of the double part.
template <int S, typename Real, typename Acc, bool RT = false, typename At>
__device__ __forceinline__ void h_combine(const Staged<Real, Acc>& st, const At& at, Acc A,
                                          const Mid<Real, Acc>& c, const Mid<Real, Acc>& lo,
                                          const Mid<Real, Acc>& hi, Acc h[4], const Params& P) {
  using Sc = Scheme<S>;
  const HalfCoef<S, RT> K{P};
  if constexpr (Staged<Real, Acc>::SPLIT) {
    Acc he[4];
    Real hq[4];
    const double m0 = 2.0 * K.m0(), m1 = 2.0 * K.m1();
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      if constexpr (Sc::nmp == 1) {
        he[v] = Acc(m0) * c.f[0][v];
        hq[v] = Real(m0) * c.q[0][v];
      } else {
        he[v] = Acc(K.m0()) * (c.f[0][v] + c.f[1][v]) + Acc(K.m1()) * (lo.f[0][v] + hi.f[1][v]);
        hq[v] = Real(m0) * (c.q[0][v] - c.q[1][v]) + Real(m1) * (lo.q[0][v] - hi.q[1][v]);
      }
    }
#pragma unroll
    for (int d = 0; d <= 3; ++d) {
      // which terms exist is the printed scheme's (the same support at every alpha)
      if (0.5 * (hnode<S>(-d) + hnode<S>(1 + d)) == 0.0 && hnode<S>(-d) - hnode<S>(1 + d) == 0.0) continue;
      const double ce = K.n(-d) + K.n(1 + d), cq = 2.0 * (K.n(-d) - K.n(1 + d));
      Acc a[4], b[4];
      Real qa[4], qb[4];
      ld4(st.fp, st.n, at(-d), a);
      ld4(st.fp, st.n, at(1 + d), b);
      ld4(st.q, st.n, at(-d), qa);
      ld4(st.q, st.n, at(1 + d), qb);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        if (RT || ce != 0.0) he[v] += Acc(ce) * (a[v] + b[v]);
        if (RT || cq != 0.0) hq[v] += Real(cq) * (qa[v] - qb[v]);
      }
    }
    const Real hA = Real(0.5) * from_f64_int(A);
#pragma unroll
    for (int v = 0; v < 4; ++v) h[v] = he[v] + widen<Acc>(hA * hq[v]);
  } else if constexpr (std::is_same<Acc, float>::value) {
    // the same in the two lanes of packed float arithmetic, components (0, 1) and (2, 3)
#pragma unroll
    for (int v = 0; v < 4; v += 2) {
      const float2 c0 = make_float2(c.f[0][v], c.f[0][v + 1]), c1 = make_float2(c.f[1][v], c.f[1][v + 1]);
      float2 hh = mul2(bc2(K.m0f()), add2(c0, c1));
      if constexpr (Sc::nmp == 2) {
        const float2 l0 = make_float2(lo.f[0][v], lo.f[0][v + 1]), h1 = make_float2(hi.f[1][v], hi.f[1][v + 1]);
        hh = fma2(bc2(K.m1f()), add2(l0, h1), hh);
      }
      h[v] = hh.x;
      h[v + 1] = hh.y;
    }
#pragma unroll
    for (int kk = -3; kk <= 3; ++kk) {
      if (Sc::hn(kk) == 0.0) continue;
      Acc a[4], b[4];
      ld4(st.fp, st.n, at(kk), a);
      ld4(st.fm, st.n, at(1 - kk), b);
#pragma unroll
      for (int v = 0; v < 4; v += 2) {
        const float2 hh = fma2(bc2(K.nf(kk)),
                               add2(make_float2(a[v], a[v + 1]), make_float2(b[v], b[v + 1])),
                               make_float2(h[v], h[v + 1]));
        h[v] = hh.x;
        h[v + 1] = hh.y;
      }
    }
  } else {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      if constexpr (Sc::nmp == 1) h[v] = Acc(K.m0()) * (c.f[0][v] + c.f[1][v]);
      else h[v] = Acc(K.m0()) * (c.f[0][v] + c.f[1][v]) + Acc(K.m1()) * (lo.f[0][v] + hi.f[1][v]);
    }
#pragma unroll
    for (int kk = -3; kk <= 3; ++kk) {
      if (Sc::hn(kk) == 0.0) continue;
      Acc a[4], b[4];
      ld4(st.fp, st.n, at(kk), a);
      ld4(st.fm, st.n, at(1 - kk), b);
#pragma unroll
      for (int v = 0; v < 4; ++v) h[v] += Acc(K.n(kk)) * (a[v] + b[v]);
    }
  }
}


// h at p + 1/2 for the four-midpoint scheme (same precision only): h+ = m0 f+_{p+1/2} +
// m1 f+_{p-1/2} + mA f+_{p-3/2} + mB f+_{p+3/2} + sum_k n_k f+_{p+k} and h- its mirror about
// p + 1/2 (f-_{p+1/2}, f-_{p+3/2}, f-_{p+5/2}, f-_{p-1/2}; f-_{p+1-k}), from the records of
// the interfaces p - 2 .. p + 2 (mids[m + 2] = interface p + m) and the staged 2 f+- (halved
// coefficients).
template <int S, typename Real, typename Acc, typename At>
__device__ __forceinline__ void h_combine4(const Staged<Real, Acc>& st, const At& at, const Mid<Real, Acc>* mids,
                                           Acc h[4]) {
  static_assert(!Staged<Real, Acc>::SPLIT, "the four-midpoint scheme is built for one precision");
  using Sc = Scheme<S>;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    h[v] = Acc(0.5 * Sc::m0) * (mids[2].f[0][v] + mids[2].f[1][v]) +
           Acc(0.5 * Sc::m1) * (mids[1].f[0][v] + mids[3].f[1][v]) +
           Acc(0.5 * Sc::mA) * (mids[0].f[0][v] + mids[4].f[1][v]) +
           Acc(0.5 * Sc::mB) * (mids[3].f[0][v] + mids[1].f[1][v]);
  }
#pragma unroll
  for (int kk = -3; kk <= 3; ++kk) {
    if (Sc::hn(kk) == 0.0) continue;
    Acc a[4], b[4];
    ld4(st.fp, st.n, at(kk), a);
    ld4(st.fm, st.n, at(1 - kk), b);
#pragma unroll
    for (int v = 0; v < 4; ++v) h[v] += Acc(0.5 * Sc::hn(kk)) * (a[v] + b[v]);
  }
}

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
  constexpr int NL = Sh::NL, W = Sh::W, T = Sh::T, NP = Sh::NP, PLO = Sh::PLO, OFF = Sh::OFF;
  constexpr int NN = Sh::NN, NW = Sh::NW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Staged<Real, Acc> st;
  st.carve(smem_raw, NN);
  Acc* sH = reinterpret_cast<Acc*>(smem_raw + Sh::o_h());   // h at interfaces (4 values)
  MidStore<Real, Acc> sF;                                   // midpoint records (two-midpoint)
  sF.carve(smem_raw + Sh::o_f(), NW);
  Acc* sA = reinterpret_cast<Acc*>(smem_raw + Sh::o_a());   // A^ per line

  const int n = DIR == 0 ? P.ni : P.nj;
  const int nlines = DIR == 0 ? P.nj : P.ni;
  const int line0 = by * NL;
  const int base = bx * T;
  const Real gamma = Real(P.gamma);
  const Real eps = sizeof(Real) == 8 ? from_f64<Real>(P.eps) : from_f64<Real>(P.eps < 1e-30 ? 1e-30 : P.eps);
  const long long plane = (long long)P.nj * P.ld;

  auto SI = [](int l, int s) { return DIR == 0 ? l * NP + s : s * NL + l; };
  auto WI = [](int l, int p) { return DIR == 0 ? l * W + p : p * NL + l; };

  // A^ = alpha x line maximum, once per line (Section 2.3)
  if (threadIdx.x < NL) {
    const int line = line0 + threadIdx.x;
    sA[threadIdx.x] = line < nlines ? Acc(P.alpha * lam[line]) : Acc(0);
  }
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
  // ---- phase 1: nodes.  FP64: one node per thread and round.  Otherwise the global loads of
  // both rounds are issued before any arithmetic, so the second (partial) round does not wait
  // for a second memory latency.
  if constexpr (sizeof(Real) == 8) {
    __syncthreads();  // A^ in shared memory
    for (int k = threadIdx.x; k < NN; k += Sh::THREADS) {
      const int l = DIR == 0 ? k / NP : k % NL;
      const int s = DIR == 0 ? k % NP : k / NL;
      const int line = line0 + l;
      if (line >= nlines) continue;
      const int g = min(base + s - OFF, n + OFF - 1);
      // beyond the stored ghost metrics (the four-midpoint scheme, periodic only): wrap
      const int gm = (Sh::FOUR && (g < -G || g >= n + G)) ? pmod(g, n) : g;
      Real q[4];
      load_state(P, Q, DIR, line, g, q, qtab);
      double mx, my;
      if (DIR == 0) { mx = met_at(P, 0, gm, line); my = met_at(P, 1, gm, line); }
      else          { mx = met_at(P, 2, line, gm); my = met_at(P, 3, line, gm); }
      NodeChar<Real> w;
      Acc amx, amy, fp[4], fm[4];
      node_split<weno_scale<Sc::r>(), Real, Acc>(q, mx, my, gamma, Acc(0.5) * sA[l], w, amx, amy, fp, fm);
      st.store(SI(l, s), q, w, amx, amy, fp, fm, mx, my);
    }
  } else {
  constexpr int NR = (NN + Sh::THREADS - 1) / Sh::THREADS;
  Real qv[NR][4];
  double mxv[NR], myv[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int k = threadIdx.x + r * Sh::THREADS;
    const int l = DIR == 0 ? k / NP : k % NL;
    const int s = DIR == 0 ? k % NP : k / NL;
    const int line = line0 + l;
    if (k >= NN || line >= nlines) continue;
    const int g = min(base + s - OFF, n + OFF - 1);  // positions past n+OFF-1 are never used
    const int gm = (Sh::FOUR && (g < -G || g >= n + G)) ? pmod(g, n) : g;
    load_state(P, Q, DIR, line, g, qv[r], qtab);
    if (DIR == 0) { mxv[r] = met_at(P, 0, gm, line); myv[r] = met_at(P, 1, gm, line); }
    else          { mxv[r] = met_at(P, 2, line, gm); myv[r] = met_at(P, 3, line, gm); }
  }
  __syncthreads();  // A^ in shared memory
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int k = threadIdx.x + r * Sh::THREADS;
    const int l = DIR == 0 ? k / NP : k % NL;
    const int s = DIR == 0 ? k % NP : k / NL;
    const int line = line0 + l;
    if (k >= NN || line >= nlines) continue;
    NodeChar<Real> w;
    Acc amx, amy, fp[4], fm[4];
    node_split<weno_scale<Sc::r>(), Real, Acc>(qv[r], mxv[r], myv[r], gamma, Acc(0.5) * sA[l], w, amx, amy, fp, fm);
    st.store(SI(l, s), qv[r], w, amx, amy, fp, fm, mxv[r], myv[r]);
  }
  }
  __syncthreads();

  // ---- phase 2: interfaces p + 1/2 ----
  for (int k = threadIdx.x; k < NW; k += Sh::THREADS) {
    const int l = DIR == 0 ? k / W : k % NL;
    const int pi = DIR == 0 ? k % W : k / NL;
    const int line = line0 + l;
    const int p = PLO + pi;
    // one-midpoint schemes use interfaces -1 .. T-1 (the last slot is spare); the
    // four-midpoint scheme's h at n - 1/2 reads the interface n + 3/2
    if (line >= nlines || base + p > n + (Sh::FOUR ? 1 : 0) || (Sc::nmp == 1 && p > T - 1)) continue;
    const int c0 = p + OFF;  // staged position of node p
    auto at = [&](int m) { return SI(l, c0 + m); };
    Mid<Real, Acc> mo;
    interface_mid<S, Real, Acc>(st, at, gamma, eps, P.ppm, P.linw, P.interp, sA[l], mo, P.wz, P.msplit);
    if constexpr (Sc::nmp == 1) {
      Acc h[4];
      h_combine<S, Real, Acc, true>(st, at, sA[l], mo, mo, mo, h, P);
      st4(sH, NW, WI(l, pi), h[0], h[1], h[2], h[3]);
    } else {
      sF.put(WI(l, pi), mo);
    }
  }

  if constexpr (Sc::nmp >= 2) {
    __syncthreads();
    // h+ uses f+ at p+1/2 and p-1/2; h- uses f- at p+1/2 and p+3/2 (four midpoints: also
    // f+ at p-3/2, p+3/2 and f- at p+5/2, p-1/2)
    for (int k = threadIdx.x; k < NW; k += Sh::THREADS) {
      const int l = DIR == 0 ? k / W : k % NL;
      const int pi = DIR == 0 ? k % W : k / NL;
      const int line = line0 + l;
      const int p = PLO + pi;
      if (line >= nlines || p < -1 || p > T - 1 || base + p > n - 1) continue;
      const int c0 = p + OFF;
      auto at = [&](int m) { return SI(l, c0 + m); };
      Acc h[4];
      if constexpr (Sh::FOUR) {
        Mid<Real, Acc> mids[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
          sF.get(WI(l, pi - 2 + m), 0, mids[m]);
          sF.get(WI(l, pi - 2 + m), 1, mids[m]);
        }
        h_combine4<S, Real, Acc>(st, at, mids, h);
      } else {
        Mid<Real, Acc> c, lo, hi;
        sF.get(WI(l, pi), 0, c);
        sF.get(WI(l, pi), 1, c);
        sF.get(WI(l, pi - 1), 0, lo);
        sF.get(WI(l, pi + 1), 1, hi);
        h_combine<S, Real, Acc, true>(st, at, sA[l], c, lo, hi, h, P);
      }
      st4(sH, NW, WI(l, pi), h[0], h[1], h[2], h[3]);
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
    Acc hp[4], hm[4], R[4];
    ld4(sH, NW, WI(l, pi), hp);
    ld4(sH, NW, WI(l, pi - 1), hm);
#pragma unroll
    for (int v = 0; v < 4; ++v) R[v] = hp[v] - hm[v];
    if constexpr (MODE == MODE_ACC) {
#pragma unroll
      for (int v = 0; v < 4; ++v) Dout[v * plane + o] = R[v];
    } else {
      cp_async_wait_all();
      Real qs[4];
      if constexpr (MODE == MODE_STAGE) ld4(st.q, st.n, SI(l, s + OFF), qs);
      const Acc mJ = -recip(from_f64<Acc>(sJ[k]));
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const Acc d = (sDa[v * Sh::NO + k] + R[v]) * mJ;
        if constexpr (MODE == MODE_RHS) {
          qout[v * plane + o] = narrow<Real>(d);
        } else {
          qout[v * plane + o] =
              narrow<Real>(Acc(ca) * widen<Acc>(sQn[v * Sh::NO + k]) + Acc(cb) * (widen<Acc>(qs[v]) + Acc(dt) * d));
        }
      }
    }
  }
}

// --------------------------------------------------------------------------------------
// Marching xi pass.  A warp walks one row segment [s0, s1) of a block 32 nodes at a time.
// Every step t (lane L):
//   nodes       m = s0 + K + 32 t + L  into ring slot m mod 64 (state and metrics staged by
//               cp.async during the previous step when the node is interior)
//   centres     c = s0 - NMP + 32 t + L: the "+" side of interface c + 1/2 and the "-" side of
//               interface c - 1/2, which share the node's stencil differences (centre_sides);
//               Q+ goes to the ring, Q- stays in the lane
//   interfaces  q = c - 1: Q+ from the centre q (lane L - 1, or lane 31 a step earlier) and
//               this lane's Q-; midpoint fluxes (and for one-midpoint schemes h)
//   h           (two-midpoint schemes) at q - 1, from the midpoint ring
//   outputs     node s = the interface just completed, H_s - H_{s-1} from the h ring
// with K = 3 (one midpoint) or 2 (two midpoints), so that every stencil node of a step's
// centres and interfaces is in the ring; a start-up pass stages the nodes s0 - NMP - H ..
// s0 + K - 1 (H = 2, or 3 for WENOIU7).  The ring holds the at most 40 nodes a step reads;
// the warp synchronises between the phases only.
// --------------------------------------------------------------------------------------
template <int S, int MODE, typename Real, typename Acc>
__device__ __forceinline__ void march_row(const Params& P, const Real* __restrict__ Q, const Real* const* qtab,
                                          double lamv, const Acc* __restrict__ Dacc, Acc* __restrict__ Dout,
                                          Real* qout, const Real* Qn, double ca, double cb, double dt, int row,
                                          int s0, int s1, unsigned char* wsm, const double* __restrict__ mid = nullptr,
                                          double* __restrict__ ncout = nullptr) {
  using Ms = MarchShape<S, Real, Acc>;
  constexpr int NMP = Scheme<S>::nmp;
  constexpr int K = NMP == 1 ? 3 : 2;
  constexpr int H = Scheme<S>::r == 4 ? 3 : 2;     // stencil half-width of the interpolation
  constexpr bool CENTRE = march_centres<Real>();
  const int L = threadIdx.x & 31;
  Staged<Real, Acc> st;
  st.carve(wsm, RING);
  Acc* rH = reinterpret_cast<Acc*>(wsm + Ms::o_h());
  MidStore<Real, Acc> rF;
  rF.carve(wsm + Ms::o_f(), RING);
  Real* rQp = reinterpret_cast<Real*>(wsm + Ms::o_qp());              // Q+ per centre slot
  Real* rawq = reinterpret_cast<Real*>(wsm + Ms::o_raw());           // [4][32]
  double* rawm = reinterpret_cast<double*>(rawq + 4 * 32);           // [2][32]
  const int n = P.ni;
  const Real gamma = Real(P.gamma);
  const Real eps = sizeof(Real) == 8 ? from_f64<Real>(P.eps) : from_f64<Real>(P.eps < 1e-30 ? 1e-30 : P.eps);
  const long long plane = (long long)P.nj * P.ld;
  const Acc A = Acc(P.alpha * lamv);
  const Acc hA = Acc(0.5) * A;
  const Real* Qrow = Q + (long long)row * P.ld;
  const double* M0 = P.met + (long long)(row + G) * P.mld + G;   // xi_x^ of node (i, row) at M0[i]
  const double* M1 = M0 + P.mplane;                                // xi_y^
  // the row's interfaces q = -2 .. ni as the batch stored them once per step (double
  // accumulation only): planes midpoint xi_x^, xi_y^, then (FP64) the unit direction
  const bool pre = std::is_same<Acc, double>::value && mid != nullptr;
  const bool pdir = std::is_same<Real, double>::value && pre;
  const double* MXr = pre ? mid + (long long)row * (n + 3) + 2 : nullptr;
  const long long mstr = (long long)P.nj * (n + 3);

  // the node stage of one position: interior nodes from the cp.async staging (if staged),
  // else through the boundary rule; positions past n + 3 are never read
  auto stage_node = [&](int m, bool staged) {
    if (m > s1 + 3 || m > n + 3) return;
    Real q[4];
    double mx, my;
    if (staged) {
#pragma unroll
      for (int v = 0; v < 4; ++v) q[v] = rawq[v * 32 + L];
      mx = rawm[L];
      my = rawm[32 + L];
    } else {
      load_state(P, Q, 0, row, m, q, qtab);
      mx = met_at(P, 0, m, row);
      my = met_at(P, 1, m, row);
    }
    Acc amx, amy, fp[4], fm[4];
    Real pr;
    const NodeChar<Real> w = node_char<Real, weno_scale<Scheme<S>::r>()>(q, gamma, pr);
    node_split_from<Real, Acc>(q, w, pr, mx, my, hA, amx, amy, fp, fm);
    st.store(m & (RING - 1), q, w, amx, amy, fp, fm, mx, my);
    // FP64: the row's own nodes' characteristic data for the eta pass of this right-hand side
    if constexpr (std::is_same<Real, double>::value && MODE == MODE_ACC && NMP == 1)
      if (ncout && m >= s0 && m < s1) nc_put(ncout, plane, (long long)row * P.ld + m, w, pr);
  };
  // cp.async of node m's state and metrics into this lane's staging slot (interior only)
  auto prefetch = [&](int m) -> bool {
    if (m < 0 || m >= n || m > s1 + 3) return false;
#pragma unroll
    for (int v = 0; v < 4; ++v) cp_async<sizeof(Real)>(rawq + v * 32 + L, Qrow + v * plane + m);
    cp_async<8>(rawm + L, M0 + m);
    cp_async<8>(rawm + 32 + L, M1 + m);
    return true;
  };

  // start-up: the nodes s0 - NMP - H .. s0 + K - 1, and the first step's nodes in flight
  if (L < K + NMP + H) stage_node(s0 - NMP - H + L, false);
  bool staged = prefetch(s0 + K + L);
  cp_async_commit();
  const int steps = (s1 - s0 + 2 * NMP + 31) / 32;   // until the interface s1 + NMP - 2
  for (int t = 0; t < steps; ++t) {
    const int m = s0 + K + 32 * t + L;
    cp_async_wait_all();
    stage_node(m, staged);
    __syncwarp();
    staged = prefetch(m + 32);       // the next step's node, in flight during this step
    cp_async_commit();
    // centres s0 - NMP .. s1 + NMP - 1
    const int c = s0 - NMP + 32 * t + L;
    Real Qm[4];
    if constexpr (CENTRE) {
      if (c <= s1 + NMP - 1) {
        auto at = [&](int mm) { return (c + mm) & (RING - 1); };
        Real npx, npy, nmx, nmy;
        if (pdir) {
          npx = Real(MXr[c + 2 * mstr]);
          npy = Real(MXr[c + 3 * mstr]);
          nmx = Real(MXr[c - 1 + 2 * mstr]);
          nmy = Real(MXr[c - 1 + 3 * mstr]);
        } else {
          char_direction(st, at(0), at(1), npx, npy);
          char_direction(st, at(-1), at(0), nmx, nmy);
        }
        Real Qp[4];
        centre_sides<S, Real, Acc>(st, at, npx, npy, nmx, nmy, eps, Qp, Qm);
        st4(rQp, RING, c & (RING - 1), Qp[0], Qp[1], Qp[2], Qp[3]);
      }
      __syncwarp();
    }
    // interfaces s0 - NMP .. s1 + NMP - 2
    const int q = c - 1;
    if (q >= s0 - NMP && q <= s1 + NMP - 2) {
      auto at = [&](int mm) { return (q + mm) & (RING - 1); };
      IfacePre pr;
      if (pre) {
        pr.mid = true;
        pr.mx = MXr[q];
        pr.my = MXr[q + mstr];
      }
      Mid<Real, Acc> mo;
      if constexpr (CENTRE) {
        Real Qs[2][4];
        ld4(rQp, RING, q & (RING - 1), Qs[0]);
#pragma unroll
        for (int v = 0; v < 4; ++v) Qs[1][v] = Qm[v];
        mid_fluxes<S, Real, Acc>(st, at, Qs, gamma, 0, A, mo, 0, pr);
      } else {
        if (pdir) {
          pr.dir = true;
          pr.nx = MXr[q + 2 * mstr];
          pr.ny = MXr[q + 3 * mstr];
        }
        interface_mid<S, Real, Acc, true>(st, at, gamma, eps, P.ppm, P.linw, P.interp, A, mo, 0, 0, pr);
      }
      if constexpr (NMP == 1) {
        Acc h[4];
        h_combine<S, Real, Acc>(st, at, A, mo, mo, mo, h, P);
        st4(rH, RING, q & (RING - 1), h[0], h[1], h[2], h[3]);
      } else {
        rF.put(q & (RING - 1), mo);
      }
    }
    __syncwarp();
    int s = q;
    if constexpr (NMP == 2) {
      // h at p = q - 1 from the midpoint fluxes at p - 1/2, p + 1/2, p + 3/2
      const int p = q - 1;
      if (p >= s0 - 1 && p <= s1 - 1) {
        auto at = [&](int mm) { return (p + mm) & (RING - 1); };
        Mid<Real, Acc> cm, lo, hi;
        rF.get(p & (RING - 1), 0, cm);
        rF.get(p & (RING - 1), 1, cm);
        rF.get((p - 1) & (RING - 1), 0, lo);
        rF.get((p + 1) & (RING - 1), 1, hi);
        Acc h[4];
        h_combine<S, Real, Acc>(st, at, A, cm, lo, hi, h, P);
        st4(rH, RING, p & (RING - 1), h[0], h[1], h[2], h[3]);
      }
      __syncwarp();
      s = p;
    }
    // outputs: node s, H_{s+1/2} - H_{s-1/2}
    if (s >= s0 && s < s1) {
      Acc hp[4], hm[4], R[4];
      ld4(rH, RING, s & (RING - 1), hp);
      ld4(rH, RING, (s - 1) & (RING - 1), hm);
#pragma unroll
      for (int v = 0; v < 4; ++v) R[v] = hp[v] - hm[v];
      const long long o = (long long)row * P.ld + s;
      if constexpr (MODE == MODE_ACC) {
#pragma unroll
        for (int v = 0; v < 4; ++v) Dout[v * plane + o] = R[v];
      } else {
        const Acc mJ = -recip(from_f64<Acc>(__ldg(P.met + 4 * P.mplane + (long long)(row + G) * P.mld + s + G)));
        Real qs[4];
        if constexpr (MODE == MODE_STAGE) ld4(st.q, st.n, s & (RING - 1), qs);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const Acc d = (Dacc[v * plane + o] + R[v]) * mJ;
          if constexpr (MODE == MODE_RHS) {
            qout[v * plane + o] = narrow<Real>(d);
          } else {
            qout[v * plane + o] =
                narrow<Real>(Acc(ca) * widen<Acc>(Qn[v * plane + o]) + Acc(cb) * (widen<Acc>(qs[v]) + Acc(dt) * d));
          }
        }
      }
    }
    __syncwarp();   // the next step overwrites ring slots read above
  }
  cp_async_wait_all();
}

// --------------------------------------------------------------------------------------
// Marching eta pass.  A CTA of EW warps owns 32 adjacent columns (one per lane) and a row
// segment [s0, s1) of one block; it walks the segment EW rows per step, warp w taking row
// r + w of the step starting at row r.  Per step (1MP / 2MP):
//   nodes       m = r + K + w (K = 2, 3 for WENOIU7) into the ring (row slot m mod ERING),
//               state, metrics and the
//               epilogue operands of the next step staged by cp.async during this step
//   centres     (FP64 1MP) c = r - 1 + w: both interface sides centred at node c
//               (centre_sides), Q+ of c + 1/2 into a ring, Q- of c - 1/2 kept by the thread
//   interfaces  q = r - NMP + w (FP64 1MP: q = c - 1, Q+ from the warp below): midpoint
//               fluxes, h (1MP) or the midpoint record (2MP)
//   h           (2MP) at q - 1 from the records of q - 2 .. q
//   outputs     node s = the interface just completed
// with a block barrier after each phase that hands data to other warps.  The ring holds the
// at most 15 rows a step reads or stages; the start-up stages the rows below r + K.
// --------------------------------------------------------------------------------------
constexpr int ERING = 16;                           // row slots of its ring
constexpr int MARCH_ETA = 3;                        // the marching eta variant
template <int S, typename Real, typename Acc>
struct MarchEtaShape {
  static constexpr int NMP = Scheme<S>::nmp;
  static constexpr int NS = ERING * 32;             // ring entries (row slot x lane)
  static constexpr int NT = EW * 32;                // threads
  static constexpr bool CENTRE = march_eta_centres(sizeof(Real) == 8, NMP);
  static constexpr int SEG = march_eta_seg(sizeof(Real) == 8, NMP);
  static constexpr size_t o_h() { return Staged<Real, Acc>::bytes(NS); }
  static constexpr size_t o_f() { return o_h() + sizeof(Acc) * 4 * NS; }
  // Q+ of the interface above each centre node (4 Real per ring slot)
  static constexpr size_t o_qp() { return o_f() + (NMP == 2 ? MidStore<Real, Acc>::bytes(NS) : 0); }
  static constexpr size_t o_raw() { return o_qp() + (CENTRE ? sizeof(Real) * 4 * NS : 0); }
  // per thread: next node's state and two metrics; then two buffers (steps t even and odd)
  // of the epilogue operands: J^-1, the xi metrics (MODE_STAGE_L), the other direction's
  // difference, Q^n (stage modes)
  // FP64 one-midpoint schemes: the next node's stored characteristic data (NC_COUNT doubles per
  // thread); the two-midpoint schemes' midpoint records leave no room for it
  static constexpr bool NC = sizeof(Real) == 8 && NMP == 1;
  static constexpr size_t o_nc() { return o_raw() + (size_t)NT * (4 * sizeof(Real) + 16); }
  static constexpr size_t o_ep() { return o_nc() + (NC ? (size_t)NT * NC_COUNT * 8 : 0); }
  static constexpr size_t ep_bytes(int mode) {
    return mode == 0 ? 0
                     : (size_t)NT * (8 + (mode == 3 ? 16 : 0) + 4 * sizeof(Acc) + (mode >= 2 ? 4 * sizeof(Real) : 0));
  }
  static constexpr size_t smem_bytes(int mode) { return o_ep() + 2 * ep_bytes(mode); }
};

template <int S, int MODE, typename Real, typename Acc>
__device__ __forceinline__ void march_col(const Params& P, const Real* __restrict__ Q, const Real* const* qtab,
                                          const double* __restrict__ lam, const Acc* __restrict__ Dacc,
                                          Acc* __restrict__ Dout, Real* qout, const Real* Qn, double ca, double cb,
                                          double dt, int c0, int s0, int s1, unsigned char* sm,
                                          double* lxo = nullptr, double* leo = nullptr,
                                          const double* __restrict__ mid = nullptr,
                                          const double* __restrict__ ncin = nullptr) {
  using Ms = MarchEtaShape<S, Real, Acc>;
  constexpr bool STAGE = MODE >= MODE_STAGE, LAM = MODE == MODE_STAGE_L;
  constexpr int NMP = Scheme<S>::nmp;
  constexpr int H = Scheme<S>::r == 4 ? 3 : 2;     // stencil half-width of the interpolation
  constexpr int K = H == 3 ? 3 : 2;                 // rows staged ahead of the step's first row
  const int L = threadIdx.x & 31, w = threadIdx.x >> 5, tid = threadIdx.x;
  const int col = c0 + L;
  const bool on = col < P.ni;
  Staged<Real, Acc> st;
  st.carve(sm, Ms::NS);
  Acc* rH = reinterpret_cast<Acc*>(sm + Ms::o_h());
  MidStore<Real, Acc> rF;
  rF.carve(sm + Ms::o_f(), Ms::NS);
  Real* rawq = reinterpret_cast<Real*>(sm + Ms::o_raw());              // [4][NT]
  double* rawm = reinterpret_cast<double*>(rawq + 4 * Ms::NT);         // [2][NT]
  double* rawc = reinterpret_cast<double*>(sm + Ms::o_nc());            // [NC_COUNT][NT] (FP64)
  Real* rQp = reinterpret_cast<Real*>(sm + Ms::o_qp());                 // Q+ per centre slot
  constexpr bool CENTRE = Ms::CENTRE;
  const bool usenc = Ms::NC && ncin != nullptr;
  // epilogue buffer k: J^-1 [NT], xi metrics [2][NT] (MODE_STAGE_L), difference [4][NT], Q^n [4][NT]
  auto eJ = [&](int k) { return reinterpret_cast<double*>(sm + Ms::o_ep() + k * Ms::ep_bytes(MODE)); };
  auto eX = [&](int k) { return eJ(k) + Ms::NT; };
  auto eD = [&](int k) { return reinterpret_cast<Acc*>(eJ(k) + (LAM ? 3 : 1) * Ms::NT); };
  auto eQ = [&](int k) { return reinterpret_cast<Real*>(eD(k) + 4 * Ms::NT); };
  const int n = P.nj;
  const Real gamma = Real(P.gamma);
  const Real eps = sizeof(Real) == 8 ? from_f64<Real>(P.eps) : from_f64<Real>(P.eps < 1e-30 ? 1e-30 : P.eps);
  const long long plane = (long long)P.nj * P.ld;
  const Acc A = on ? Acc(P.alpha * lam[col]) : Acc(0);
  const Acc hA = Acc(0.5) * A;
  auto slot = [&](int row) { return (row & (ERING - 1)) * 32 + L; };
  // the column's interfaces q = -2 .. nj as the batch stored them once per step (double
  // accumulation only): planes midpoint eta_x^, eta_y^, then (FP64) the unit direction
  const bool pre = std::is_same<Acc, double>::value && mid != nullptr;
  const bool pdir = std::is_same<Real, double>::value && pre;
  const long long mstr = (long long)(P.nj + 3) * P.ni;

  auto stage_node = [&](int m, bool staged) {
    if (!on || m > s1 + 3 || m > n + 3) return;
    Real q[4];
    double mx, my;
    if (staged) {
#pragma unroll
      for (int v = 0; v < 4; ++v) q[v] = rawq[v * Ms::NT + tid];
      mx = rawm[tid];
      my = rawm[Ms::NT + tid];
    } else {
      load_state(P, Q, 1, col, m, q, qtab);
      mx = met_at(P, 2, col, m);
      my = met_at(P, 3, col, m);
    }
    NodeChar<Real> pw;
    Acc amx, amy, fp[4], fm[4];
    if constexpr (std::is_same<Real, double>::value) {
      if (staged && usenc) {
        // the xi pass of this right-hand side formed them from the same state
        double pr;
        nc_get(rawc + tid, Ms::NT, pw, pr);
        node_split_from<Real, Acc>(q, pw, pr, mx, my, hA, amx, amy, fp, fm);
      } else {
        node_split<weno_scale<Scheme<S>::r>(), Real, Acc>(q, mx, my, gamma, hA, pw, amx, amy, fp, fm);
      }
    } else {
      node_split<weno_scale<Scheme<S>::r>(), Real, Acc>(q, mx, my, gamma, hA, pw, amx, amy, fp, fm);
    }
    st.store(slot(m), q, pw, amx, amy, fp, fm, mx, my);
  };
  // cp.async of node (col, m) into this thread's staging slot (interior rows only), and of the
  // epilogue operands of output node (col, s) into epilogue buffer k (every slot is private
  // to its thread)
  auto prefetch = [&](int m, int s, int k) -> bool {
    bool ok = false;
    if (on && m >= 0 && m < n && m <= s1 + 3) {
      const long long o = (long long)m * P.ld + col;
#pragma unroll
      for (int v = 0; v < 4; ++v) cp_async<sizeof(Real)>(rawq + v * Ms::NT + tid, Q + v * plane + o);
      const double* mp = P.met + (long long)(m + G) * P.mld + (col + G);
      cp_async<8>(rawm + tid, mp + 2 * P.mplane);
      cp_async<8>(rawm + Ms::NT + tid, mp + 3 * P.mplane);
      if (usenc) {
#pragma unroll
        for (int k = 0; k < NC_COUNT; ++k) cp_async<8>(rawc + k * Ms::NT + tid, ncin + k * plane + o);
      }
      ok = true;
    }
    if constexpr (MODE != MODE_ACC) {
      if (on && s >= s0 && s < s1) {
        const long long o = (long long)s * P.ld + col;
        const double* ms = P.met + (long long)(s + G) * P.mld + (col + G);
        cp_async<8>(eJ(k) + tid, ms + 4 * P.mplane);
        if constexpr (LAM) {
          cp_async<8>(eX(k) + tid, ms);
          cp_async<8>(eX(k) + Ms::NT + tid, ms + P.mplane);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) cp_async<sizeof(Acc)>(eD(k) + v * Ms::NT + tid, Dacc + v * plane + o);
        if constexpr (STAGE) {
#pragma unroll
          for (int v = 0; v < 4; ++v) cp_async<sizeof(Real)>(eQ(k) + v * Ms::NT + tid, Qn + v * plane + o);
        }
      }
    }
    return ok;
  };
  Real colmax = Real(0);                                   // MODE_STAGE_L: this thread's eta maximum
  const int lag = CENTRE ? 2 : NMP == 1 ? 1 : 3;          // output s = r - lag + w
  // start-up: rows s0 - 2 - NMP .. s0 + K - 1
  if (w < K + NMP + H) stage_node(s0 - NMP - H + w, false);
  bool staged = prefetch(s0 + K + w, s0 - lag + w, 0);
  cp_async_commit();
  const int steps = (s1 - s0 + 2 * NMP - 1 + (CENTRE ? 1 : 0) + EW - 1) / EW;
  for (int t = 0; t < steps; ++t) {
    const int r = s0 + EW * t;
    const int m = r + K + w;
    cp_async_wait_all();
    stage_node(m, staged);
    // this step's output node; its epilogue operands stay in buffer t & 1 until the output
    // phase, while the next step's arrive in the other buffer
    const int s = r - lag + w;
    staged = prefetch(m + EW, s + EW, (t + 1) & 1);
    cp_async_commit();
    __syncthreads();
    // centre layout: centre c = r - 1 + w takes the "+" side of interface c + 1/2 (to the Q+
    // ring, read by the warp above or by warp 0 a step later) and the "-" side of c - 1/2
    Real Qm[4];
    if constexpr (CENTRE) {
      const int c = r - 1 + w;
      if (on && c <= s1) {
        auto at = [&](int mm) { return slot(c + mm); };
        Real npx, npy, nmx, nmy;
        if (pdir) {
          const long long mo_ = (long long)(c + 2) * P.ni + col;   // interface c; c - 1 one row below
          npx = mid[mo_ + 2 * mstr];
          npy = mid[mo_ + 3 * mstr];
          nmx = mid[mo_ - P.ni + 2 * mstr];
          nmy = mid[mo_ - P.ni + 3 * mstr];
        } else {
          char_direction(st, at(0), at(1), npx, npy);
          char_direction(st, at(-1), at(0), nmx, nmy);
        }
        Real Qp[4];
        centre_sides<S, Real, Acc>(st, at, npx, npy, nmx, nmy, eps, Qp, Qm);
        st4(rQp, Ms::NS, slot(c), Qp[0], Qp[1], Qp[2], Qp[3]);
      }
      __syncthreads();
    }
    const int q = r - NMP - (CENTRE ? 1 : 0) + w;
    Real qs[4] = {Real(0), Real(0), Real(0), Real(0)};
    if (on && q >= s0 - NMP && q <= s1 + NMP - 2) {
      auto at = [&](int mm) { return slot(q + mm); };
      IfacePre pr;
      if (pre) {
        const long long mo_ = (long long)(q + 2) * P.ni + col;
        pr.mid = true;
        pr.mx = mid[mo_];
        pr.my = mid[mo_ + mstr];
        if (pdir && !CENTRE) {
          pr.dir = true;
          pr.nx = mid[mo_ + 2 * mstr];
          pr.ny = mid[mo_ + 3 * mstr];
        }
      }
      Mid<Real, Acc> mo;
      if constexpr (CENTRE) {
        // Q+ from centre q, Q- from this thread's centre q + 1
        Real Qs[2][4];
        ld4(rQp, Ms::NS, slot(q), Qs[0]);
#pragma unroll
        for (int v = 0; v < 4; ++v) Qs[1][v] = Qm[v];
        mid_fluxes<S, Real, Acc>(st, at, Qs, gamma, 0, A, mo, 0, pr);
      } else {
        interface_mid<S, Real, Acc, true>(st, at, gamma, eps, P.ppm, P.linw, P.interp, A, mo, 0, 0, pr);
      }
      if constexpr (NMP == 1) {
        Acc h[4];
        h_combine<S, Real, Acc>(st, at, A, mo, mo, mo, h, P);
        st4(rH, Ms::NS, slot(q), h[0], h[1], h[2], h[3]);
      } else {
        rF.put(slot(q), mo);
      }
    }
    if constexpr (NMP == 2) {
      __syncthreads();
      const int p = q - 1;
      if (on && p >= s0 - 1 && p <= s1 - 1) {
        auto at = [&](int mm) { return slot(p + mm); };
        Mid<Real, Acc> c, lo, hi;
        rF.get(slot(p), 0, c);
        rF.get(slot(p), 1, c);
        rF.get(slot(p - 1), 0, lo);
        rF.get(slot(p + 1), 1, hi);
        Acc h[4];
        h_combine<S, Real, Acc>(st, at, A, c, lo, hi, h, P);
        st4(rH, Ms::NS, slot(p), h[0], h[1], h[2], h[3]);
      }
    }
    // node s's staged state (and eta metrics) before the barrier: after it, warps that run
    // ahead restage the ring
    Real emx = Real(0), emy = Real(0);
    if constexpr (STAGE) {
      if (on && s >= s0 && s < s1) {
        ld4(st.q, st.n, slot(s), qs);
        if constexpr (LAM) st.met_real(slot(s), emx, emy);
      }
    }
    __syncthreads();
    // outputs: node s, H_{s+1/2} - H_{s-1/2}
    Real sx = Real(0);
    if (on && s >= s0 && s < s1) {
      Acc hp[4], hm[4], R[4];
      ld4(rH, Ms::NS, slot(s), hp);
      ld4(rH, Ms::NS, slot(s - 1), hm);
#pragma unroll
      for (int v = 0; v < 4; ++v) R[v] = hp[v] - hm[v];
      const long long o = (long long)s * P.ld + col;
      if constexpr (MODE == MODE_ACC) {
#pragma unroll
        for (int v = 0; v < 4; ++v) Dout[v * plane + o] = R[v];
      } else {
        const int k = t & 1;
        const Acc mJ = -recip(from_f64<Acc>(eJ(k)[tid]));
        Real qo[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const Acc d = (eD(k)[v * Ms::NT + tid] + R[v]) * mJ;
          if constexpr (MODE == MODE_RHS) {
            qo[v] = narrow<Real>(d);
          } else {
            qo[v] = narrow<Real>(Acc(ca) * widen<Acc>(eQ(k)[v * Ms::NT + tid]) +
                                 Acc(cb) * (widen<Acc>(qs[v]) + Acc(dt) * d));
          }
          qout[v * plane + o] = qo[v];
        }
        if constexpr (LAM) {
          // |U^| + c|k^| of the written state, as the line-maxima kernel takes it
          sx = spectral_radius(qo, from_f64_alu<Real>(eX(k)[tid]), from_f64_alu<Real>(eX(k)[Ms::NT + tid]), gamma);
          colmax = max(colmax, spectral_radius(qo, emx, emy, gamma));
        }
      }
    }
    if constexpr (LAM) {
      // row s's maximum over this CTA's 32 columns (the step is uniform over the warp)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) sx = max(sx, __shfl_xor_sync(0xffffffffu, sx, off));
      if (L == 0 && s >= s0 && s < s1)
        atomicMax(reinterpret_cast<unsigned long long*>(lxo + s), (unsigned long long)__double_as_longlong((double)sx));
    }
  }
  cp_async_wait_all();
  if constexpr (LAM) {
    // each column's maximum over the CTA's segment (the staging area is free now)
    __syncthreads();
    rawq[tid] = colmax;
    __syncthreads();
    if (w == 0 && on) {
      Real mc = rawq[L];
#pragma unroll
      for (int k = 1; k < EW; ++k) mc = max(mc, rawq[k * 32 + L]);
      atomicMax(reinterpret_cast<unsigned long long*>(leo + col), (unsigned long long)__double_as_longlong((double)mc));
    }
  }
}

// Resident CTAs per SM the kernels are compiled for (register budget): FP64 2, FP32 4, mixed 3
// for the 256-thread tiles; FP64 3, FP32 and mixed 5 for the 128-thread marching xi CTAs (102
// registers for the float passes: five FP32 CTAs measured 3 % faster than six at 80).
template <typename Real, typename Acc>
constexpr int tile_ctas() { return sizeof(Real) == 8 ? 2 : std::is_same<Real, Acc>::value ? 4 : 3; }
template <typename Real, typename Acc>
constexpr int march_ctas() { return sizeof(Real) == 8 ? 3 : 5; }

template <int S, int DIR, int MODE, typename Real, typename Acc>
__global__ void __launch_bounds__(256, tile_ctas<Real, Acc>())
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
  double* const* lxo;              // line maxima of the written state, xi and eta (MODE_STAGE_L)
  double* const* leo;
  const double* const* mid;        // midpoint metrics of the pass's direction (or null)
  const double* const* nc;         // FP64 node characteristic data: written by xi, read by eta (or null)
};

template <int S, int DIR, int MODE, typename Real, typename Acc, int V>
__global__ void __launch_bounds__(256, tile_ctas<Real, Acc>())
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

// Marching xi pass of many blocks: CTA b takes rows 4 by .. 4 by + 3 (one per warp) of
// block tiles[b].block, segment tiles[b].bx of each row.
template <int S, int MODE, typename Real, typename Acc>
__global__ void __launch_bounds__(32 * MARCH_WARPS, march_ctas<Real, Acc>())
march_batch_kernel(BatchPass<Real, Acc> B, double ca, double cb, double dt) {
  using Ms = MarchShape<S, Real, Acc>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Params sp;
  const TileRef t = B.tiles[blockIdx.x];
  if (threadIdx.x == 0) sp = B.params[t.block];
  __syncthreads();
  const int b = t.block;
  const int warp = threadIdx.x >> 5;
  const int row = t.by * MARCH_WARPS + warp;
  if (row >= sp.nj) return;   // whole warps only; no block-wide barrier follows
  const int seg = march_seg_len(sp.ni);
  const int s0 = t.bx * seg, s1 = min(sp.ni, s0 + seg);
  if (s0 >= s1) return;
  march_row<S, MODE, Real, Acc>(sp, B.q[b], B.q, B.lam[b][row], MODE == MODE_ACC ? nullptr : B.dacc[b],
                                MODE == MODE_ACC ? B.dout[b] : nullptr, MODE == MODE_ACC ? nullptr : B.qout[b],
                                MODE == MODE_STAGE ? B.qn[b] : nullptr, ca, cb, dt, row, s0, s1,
                                smem_raw + warp * Ms::warp_bytes(), B.mid ? B.mid[b] : nullptr,
                                B.nc ? const_cast<double*>(B.nc[b]) : nullptr);
}

// Marching eta pass of many blocks: CTA b takes the 32 columns from 32 by of block
// tiles[b].block, row segment bx (bx along the lines, by across them, as for the tiles).
// Register budget: two 256-thread CTAs per SM for the float paths (128 registers measured
// faster than three CTAs at 80), one for FP64.
template <typename Real, typename Acc>
constexpr int march_eta_ctas() { return sizeof(Real) == 8 ? 1 : 2; }

template <int S, int MODE, typename Real, typename Acc>
__global__ void __launch_bounds__(32 * EW, march_eta_ctas<Real, Acc>())
march_eta_batch_kernel(BatchPass<Real, Acc> B, double ca, double cb, double dt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Params sp;
  const TileRef t = B.tiles[blockIdx.x];
  if (threadIdx.x == 0) sp = B.params[t.block];
  __syncthreads();
  const int b = t.block;
  const int seg = MarchEtaShape<S, Real, Acc>::SEG;
  const int s0 = t.bx * seg, s1 = min(sp.nj, s0 + seg);
  march_col<S, MODE, Real, Acc>(sp, B.q[b], B.q, B.lam[b], MODE == MODE_ACC ? nullptr : B.dacc[b],
                                MODE == MODE_ACC ? B.dout[b] : nullptr, MODE == MODE_ACC ? nullptr : B.qout[b],
                                MODE >= MODE_STAGE ? B.qn[b] : nullptr, ca, cb, dt, t.by * 32, s0, s1, smem_raw,
                                MODE == MODE_STAGE_L ? B.lxo[b] : nullptr, MODE == MODE_STAGE_L ? B.leo[b] : nullptr,
                                B.mid ? B.mid[b] : nullptr, B.nc ? B.nc[b] : nullptr);
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
  void* const* lxo;     // MODE_STAGE_L only
  void* const* leo;
  void* const* mid;     // per block: midpoint metrics of this direction, or null (marching passes)
  void* const* nc;      // per block: FP64 node characteristic data (xi writes, eta reads), or null
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
  B.lxo = reinterpret_cast<double* const*>(t.lxo);
  B.leo = reinterpret_cast<double* const*>(t.leo);
  B.mid = reinterpret_cast<const double* const*>(t.mid);
  B.nc = reinterpret_cast<const double* const*>(t.nc);
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

template <int S, int MODE, typename Real, typename Acc>
cudaError_t launch_march_batch(const BatchPass<Real, Acc>& B, int ntiles, double ca, double cb, double dt,
                               cudaStream_t st) {
  auto kern = march_batch_kernel<S, MODE, Real, Acc>;
  const size_t smem = MarchShape<S, Real, Acc>::smem_bytes();
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (ntiles > 0) kern<<<ntiles, 32 * MARCH_WARPS, smem, st>>>(B, ca, cb, dt);
  return cudaGetLastError();
}

template <int S, int MODE, typename Real, typename Acc>
cudaError_t launch_march_eta_batch(const BatchPass<Real, Acc>& B, int ntiles, double ca, double cb, double dt,
                                   cudaStream_t st) {
  auto kern = march_eta_batch_kernel<S, MODE, Real, Acc>;
  const size_t smem = MarchEtaShape<S, Real, Acc>::smem_bytes(MODE);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (ntiles > 0) kern<<<ntiles, 32 * EW, smem, st>>>(B, ca, cb, dt);
  return cudaGetLastError();
}

template <int S, int DIR, int MODE, typename Real, typename Acc>
cudaError_t launch_sweep_batch(const BatchPass<Real, Acc>& B, int ntiles, int v, double ca, double cb, double dt,
                               cudaStream_t st) {
  if constexpr (MODE == MODE_STAGE_L) {
    // the line maxima are taken by the marching eta pass only
    if (DIR == 1 && v == MARCH) return launch_march_eta_batch<S, MODE, Real, Acc>(B, ntiles, ca, cb, dt, st);
    return cudaErrorNotSupported;
  }
  if (v == MARCH) {
    if constexpr (DIR == 0) return launch_march_batch<S, MODE, Real, Acc>(B, ntiles, ca, cb, dt, st);
    else return launch_march_eta_batch<S, MODE, Real, Acc>(B, ntiles, ca, cb, dt, st);
  }
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

// Both directions of every block for one scheme, xi tiles of shape variant vx, eta tiles of
// variant ve.  Mode 0: dQ/dt; 1: RK stage; 2: RK stage that also takes the next stage's line
// maxima (marching eta only).
template <int S, typename Real, typename Acc>
cudaError_t batch_scheme(int mode, const PassTables& xi, int ntx, int vx, const PassTables& eta, int nte, int ve,
                         double ca, double cb, double dt, cudaStream_t st) {
  const BatchPass<Real, Acc> X = typed_pass<Real, Acc>(xi), E = typed_pass<Real, Acc>(eta);
  cudaError_t e = launch_sweep_batch<S, 0, MODE_ACC, Real, Acc>(X, ntx, vx, 0, 0, 0, st);
  if (e != cudaSuccess) return e;
  if (mode == 0) return launch_sweep_batch<S, 1, MODE_RHS, Real, Acc>(E, nte, ve, 0, 0, 0, st);
  if (mode == 2) {
    if constexpr (std::is_same<Real, Acc>::value)
      return launch_sweep_batch<S, 1, MODE_STAGE_L, Real, Acc>(E, nte, ve, ca, cb, dt, st);
    return cudaErrorNotSupported;   // not built for mixed precision
  }
  return launch_sweep_batch<S, 1, MODE_STAGE, Real, Acc>(E, nte, ve, ca, cb, dt, st);
}

template <typename Real, typename Acc>
cudaError_t batch_dispatch(int scheme, int mode, const PassTables& xi, int ntx, int vx, const PassTables& eta,
                           int nte, int ve, double ca, double cb, double dt, cudaStream_t st) {
  switch (scheme) {
    case S31: return batch_scheme<S31, Real, Acc>(mode, xi, ntx, vx, eta, nte, ve, ca, cb, dt, st);
    case S32: return batch_scheme<S32, Real, Acc>(mode, xi, ntx, vx, eta, nte, ve, ca, cb, dt, st);
    case S51: return batch_scheme<S51, Real, Acc>(mode, xi, ntx, vx, eta, nte, ve, ca, cb, dt, st);
    case S52: return batch_scheme<S52, Real, Acc>(mode, xi, ntx, vx, eta, nte, ve, ca, cb, dt, st);
    default:  return batch_scheme<S71, Real, Acc>(mode, xi, ntx, vx, eta, nte, ve, ca, cb, dt, st);
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
    case 7: return launch_sweep_batch<S52, 1, MODE_ACC, Real, Acc>(B, ntiles, v, 0, 0, 0, st);
    case 8: return launch_sweep_batch<S71, 0, MODE_ACC, Real, Acc>(B, ntiles, v, 0, 0, 0, st);
    default: return launch_sweep_batch<S71, 1, MODE_ACC, Real, Acc>(B, ntiles, v, 0, 0, 0, st);
  }
}
// Batch passes (shape variants vx, ve for the xi and eta tiles; mode as for batch_scheme):
// FP64 in batch_fp64.cu; FP32 and mixed in batch_fp32.cu and batch_mixed.cu.
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
