// batch.cu -- many structured blocks joined by linked faces, advanced together.
//
// A multi-block grid (the paper's motivating case, Section 1) is a set of blocks whose
// faces are either physical boundaries or links to a face of another block.  The blocks
// partition the nodes of one larger grid: the ghosts behind a linked face are the
// neighbour's own nodes, read directly from the neighbour's state by the tile loaders, so
// the halo exchange is fused into the sweeps and needs no copies and no waits (each launch
// boundary orders the RK stages).  Each pass is one launch over a tile table that spans
// every block; the hardware CTA scheduler hands tiles to SMs as slots free up, which
// balances the uneven blocks.  The whole RK3 step can be captured once as a CUDA graph.
// Line maxima of the splitting are taken per block line.
#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fsp_internal.h"
#include "sweep.cuh"

namespace fsp {

// ---- metrics with linked faces -------------------------------------------------------
struct CoordBlock {
  int ni, nj, bc[4], lnb[4], lface[4], lrev[4];
  double loff[4][2];
  double per[2][2];
  const double* x;
  const double* y;
};

// Coordinates of node (i, j) of block b, any (i, j) within eight layers of the block:
// ghost indices are resolved face by face (j first, then i) through links (the
// neighbour's node plus the link's offset), periodic wraps (plus the period vector) or
// odd reflection about the boundary node (a weighted pair of nodes).
__device__ void coord_mb(const CoordBlock* __restrict__ B, int b, int i, int j, double& X, double& Y) {
  struct Item { double w; int b, i, j; };
  Item st[16];
  int n = 1;
  st[0] = {1.0, b, i, j};
  X = 0.0;
  Y = 0.0;
  for (int guard = 0; n > 0 && guard < 64; ++guard) {
    const Item it = st[--n];
    const CoordBlock& C = B[it.b];
    const bool jout = it.j < 0 || it.j >= C.nj, iout = it.i < 0 || it.i >= C.ni;
    if (!jout && !iout) {
      const long long o = (long long)it.j * C.ni + it.i;
      X += it.w * __ldg(C.x + o);
      Y += it.w * __ldg(C.y + o);
      continue;
    }
    if (n > 13) break;  // cannot happen for blocks of at least 9 nodes; keeps the stack in bounds
    const int dirj = jout ? 1 : 0;
    const int f = jout ? (it.j < 0 ? 2 : 3) : (it.i < 0 ? 0 : 1);
    const int kind = C.bc[f];
    if (kind == BC_LINK) {
      int oi, oj;
      const CoordBlock& N = B[C.lnb[f]];
      link_node(f, C.ni, C.nj, C.lface[f], C.lrev[f], N.ni, N.nj, it.i, it.j, oi, oj);
      X += it.w * C.loff[f][0];
      Y += it.w * C.loff[f][1];
      st[n++] = {it.w, C.lnb[f], oi, oj};
    } else if (kind == BC_PERIODIC) {
      const int len = dirj ? C.nj : C.ni, a = dirj ? it.j : it.i;
      const int m = pmod(a, len), q = (a - m) / len;
      X += it.w * q * C.per[dirj][0];
      Y += it.w * q * C.per[dirj][1];
      st[n++] = dirj ? Item{it.w, it.b, it.i, m} : Item{it.w, it.b, m, it.j};
    } else {
      const int len = dirj ? C.nj : C.ni, a = dirj ? it.j : it.i;
      const int bd = a < 0 ? 0 : len - 1;
      st[n++] = dirj ? Item{2.0 * it.w, it.b, it.i, bd} : Item{2.0 * it.w, it.b, bd, it.j};
      st[n++] = dirj ? Item{-it.w, it.b, it.i, 2 * bd - a} : Item{-it.w, it.b, 2 * bd - a, it.j};
    }
  }
}

// f[k] = f_{j+k-4}; pts = points of the midpoint interpolation (4, 6, or 8 for WENOIU7)
__device__ __forceinline__ double central_diff9(const Central& c, int interp, int pts, const double* f) {
  double d = c.a1 * (f[5] - f[3]) + c.a2 * (f[6] - f[2]) + c.a3 * (f[7] - f[1]) + c.a4 * (f[8] - f[0]);
  if (pts == 8) return d + c.b12 * (mid_interp8(interp, f + 1) - mid_interp8(interp, f + 0));
  const bool sixth = pts == 6;
  d += c.b12 * (mid_interp(interp, sixth, f + 2) - mid_interp(interp, sixth, f + 1));
  if (c.b32 != 0.0) d += c.b32 * (mid_interp(interp, sixth, f + 3) - mid_interp(interp, sixth, f + 0));
  return d;
}

__global__ void metrics_mb_kernel(const CoordBlock* __restrict__ B, int b, Central cen, int interp, int pts,
                                  double* __restrict__ M) {
  const int ni = B[b].ni, nj = B[b].nj;
  const int W = ni + 2 * G, H = nj + 2 * G;
  const long long plane = (long long)W * H;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < plane;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % W) - G, j = (int)(t / W) - G;
    double fx[9], fy[9], gx[9], gy[9];
    for (int k = 0; k < 9; ++k) {
      coord_mb(B, b, i + k - 4, j, fx[k], fy[k]);
      coord_mb(B, b, i, j + k - 4, gx[k], gy[k]);
    }
    const double x_xi = central_diff9(cen, interp, pts, fx), y_xi = central_diff9(cen, interp, pts, fy);
    const double x_eta = central_diff9(cen, interp, pts, gx), y_eta = central_diff9(cen, interp, pts, gy);
    M[0 * plane + t] = y_eta;
    M[1 * plane + t] = -x_eta;
    M[2 * plane + t] = -y_xi;
    M[3 * plane + t] = x_xi;
    M[4 * plane + t] = x_xi * y_eta - x_eta * y_xi;
  }
}

// ---- line maxima of every block in one launch ------------------------------------------
// Rows per thread of the line maxima: four in float (the kernel waits on memory, and four
// independent rows keep more loads in flight), one in double (bound by the FP64 pipe's
// square roots, where more resident warps hide their latency better).
template <typename Real>
constexpr int lam_rows() { return sizeof(Real) == 4 ? 4 : 1; }

template <typename Real>
__global__ void __launch_bounds__(256) lambda_batch_kernel(const Params* __restrict__ Ps,
                                                           const TileRef* __restrict__ tiles,
                                                           const Real* const* q, double* const* lamx,
                                                           double* const* lame) {
  // maxima in the state's arithmetic, one conversion per line at the atomic; a tile is 32
  // columns by 8 x lam_rows() rows, thread (x, y) taking rows y, y + 8, ...
  constexpr int NR = lam_rows<Real>();
  __shared__ Real col[8][33];
  const TileRef t = tiles[blockIdx.x];
  const Params& P = Ps[t.block];
  const Real* Q = q[t.block];
  const int ni = P.ni, nj = P.nj;
  const int i = t.bx * 32 + threadIdx.x;
  const long long plane = (long long)nj * P.ld;
  const Real g = from_f64<Real>(P.gamma);
  Real qq[NR][4];
  double m[NR][4];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int j = t.by * 8 * NR + threadIdx.y + 8 * r;
    if (i >= ni || j >= nj) continue;
    const long long o = (long long)j * P.ld + i;
#pragma unroll
    for (int v = 0; v < 4; ++v) qq[r][v] = Q[v * plane + o];
#pragma unroll
    for (int c = 0; c < 4; ++c) m[r][c] = met_at(P, c, i, j);
  }
  Real se = Real(0);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int j = t.by * 8 * NR + threadIdx.y + 8 * r;
    Real sx = Real(0);
    if (i < ni && j < nj) {
      // |U^| + c|k^| in the state's arithmetic (the splitting only needs A^ constant per line)
      sx = spectral_radius(qq[r], from_f64_alu<Real>(m[r][0]), from_f64_alu<Real>(m[r][1]), g);
      se = max(se, spectral_radius(qq[r], from_f64_alu<Real>(m[r][2]), from_f64_alu<Real>(m[r][3]), g));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sx = max(sx, __shfl_xor_sync(0xffffffffu, sx, off));
    if (threadIdx.x == 0 && j < nj)
      atomicMax(reinterpret_cast<unsigned long long*>(lamx[t.block] + j),
                (unsigned long long)__double_as_longlong((double)sx));
  }
  col[threadIdx.y][threadIdx.x] = se;
  __syncthreads();
  if (threadIdx.y == 0 && i < ni) {
    Real mx = col[0][threadIdx.x];
#pragma unroll
    for (int r = 1; r < 8; ++r) mx = max(mx, col[r][threadIdx.x]);
    atomicMax(reinterpret_cast<unsigned long long*>(lame[t.block] + i),
              (unsigned long long)__double_as_longlong((double)mx));
  }
}

// Grid-static data of every interface of every block (FP64 and mixed batches), for the
// marching passes: the interpolation I of the metric evaluation (Section 2.4) of the two
// direction metrics at the midpoint, and the unit characteristic direction of Section 3.4
// (the summed metrics of the interface's two nodes, normalised).  xi interfaces q + 1/2 of
// each row at [c][row][q + 2] of [4][nj][ni + 3], eta interfaces of each column at
// [c][q + 2][col] of [4][nj + 3][ni], c = midpoint x, y, direction x, y; q = -2 .. n for the
// direction (the centre-node layout reads both neighbours of every centre) and wherever the
// interpolation's stencil lies within the stored ghost layers for the midpoint.  The same
// stored metrics and the same functions as the passes would apply to their staged nodes.
// Grid (gx, blocks): the CTAs of row y stride over block y's interfaces.
template <int R, bool DIR>
__global__ void __launch_bounds__(256) mid_batch_kernel(const Params* __restrict__ Ps, double* const* mxt,
                                                        double* const* met) {
  const Params& P = Ps[blockIdx.y];
  double* MX = mxt[blockIdx.y];
  double* ME = met[blockIdx.y];
  const int ni = P.ni, nj = P.nj;
  const long long sx = (long long)nj * (ni + 3), se = (long long)(nj + 3) * ni;
  constexpr int NP = R == 4 ? 8 : 6, OFF = R == 4 ? 3 : 2;
  auto interp = [&](const double* v) {
    if constexpr (R == 4) return mid_interp8(P.interp, v);
    else return mid_interp(P.interp, R == 3, v);
  };
  // store interface q (-2 .. len) of a line whose metric components c = 0, 1 at node k are m(c, k)
  auto line = [&](double* out, long long stride, int q, int len, auto m) {
    if (q - OFF >= -G && q - OFF + NP - 1 <= len + G - 1) {
      double vx[NP], vy[NP];
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        vx[k] = m(0, q - OFF + k);
        vy[k] = m(1, q - OFF + k);
      }
      out[0] = interp(vx);
      out[stride] = interp(vy);
    }
    if constexpr (DIR) {
      // nodes q and q + 1 lie within the ghost layers for q = -2 .. len
      const double mbx = m(0, q) + m(0, q + 1), mby = m(1, q) + m(1, q + 1);
      const double rn = rsq(mbx * mbx + mby * mby);
      out[2 * stride] = mbx * rn;
      out[3 * stride] = mby * rn;
    }
  };
  // xi: CTA x takes rows x, x + gx, ..., its threads the interfaces of a row; eta: CTA x takes
  // the interface rows q + 2 = x, x + gx, ..., its threads the columns
  for (int row = blockIdx.x; row < nj; row += gridDim.x)
    for (int q = (int)threadIdx.x - 2; q <= ni; q += 256)
      line(MX + (long long)row * (ni + 3) + q + 2, sx, q, ni, [&](int c, int k) { return met_at(P, c, k, row); });
  for (int r = blockIdx.x; r < nj + 3; r += gridDim.x)
    for (int col = threadIdx.x; col < ni; col += 256)
      line(ME + (long long)r * ni + col, se, r - 2, nj, [&](int c, int k) { return met_at(P, 2 + c, col, k); });
}

}  // namespace fsp

using namespace fsp;

// ---- the handle ----------------------------------------------------------------------
struct fsp_batch {
  fsp_config cfg;
  int nb = 0;
  int device = 0;
  std::vector<fsp_block> blk;
  std::vector<int> bc;               // 4 per block
  std::vector<fsp_link> links;       // 4 per block
  std::vector<Params> params;        // host copy
  std::vector<CoordBlock> coords;    // host copy
  std::vector<TileRef> tx, te, tl;   // xi, eta and line-maxima tiles
  int vx = 0, ve = 0;                // tile shape variants of the xi and eta passes
  size_t tx_cap = 0, te_cap = 0;     // device table capacity (the largest variant)
  // device memory (one allocation)
  char* dmem = nullptr;
  Params* d_params = nullptr;
  CoordBlock* d_coords = nullptr;
  TileRef *d_tx = nullptr, *d_te = nullptr, *d_tl = nullptr;
  double* d_lam = nullptr;            // line maxima, two buffers (A, then B) of lam_count each
  size_t lam_count = 0;
  std::vector<size_t> lam_off, acc_off, st_off;
  char* d_acc = nullptr;             // xi differences, one per block
  double* d_mid = nullptr;           // midpoint metrics per block (FP64 and mixed; see mid_batch_kernel)
  std::vector<size_t> mid_off;       // in doubles
  double* d_nc = nullptr;            // FP64 node characteristic data per block ([NC_COUNT][nj][ld])
  std::vector<size_t> nc_off;        // in doubles
  char* d_q1 = nullptr;              // RK stage states
  char* d_q2 = nullptr;
  void** d_tab = nullptr;            // pointer tables, nb entries each (see Tab)
  bool bound = false;
  std::vector<double*> M;
  std::vector<char*> Q;              // bound states (device)
  cudaGraphExec_t gexec = nullptr;
  double gdt = 0.0;
};

namespace {

// pointer tables inside d_tab
enum Tab { T_Q0 = 0, T_Q1, T_Q2, T_ACC, T_LX, T_LE, T_LX2, T_LE2, T_OUT, T_MX, T_ME, T_NC, T_COUNT };

size_t al(size_t b) { return (b + 255) / 256 * 256; }

bool dev_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t state_size(int prec) { return prec == FSP_FP64 ? 8 : 4; }
size_t acc_elem(int prec) { return prec == FSP_FP32 ? 4 : 8; }

fsp_status check_batch(const fsp_config* c, int nb, const fsp_block* blk, const int* bc, const fsp_link* lk) {
  if (!c || nb < 1 || !blk || !bc || !lk) return FSP_ERR_INVALID_ARG;
  if (c->scheme < 0 || c->scheme > 5 || c->precision < FSP_FP64 || c->precision > FSP_FP32_MIXED ||
      c->interp < 0 || c->interp > 1 || !(c->gamma > 1.0) || !(c->lf_alpha > 0.0) || !(c->eps > 0.0))
    return FSP_ERR_INVALID_ARG;
  if (fsp_status s = check_options(*c)) return s;
  if (c->scheme == S74) return FSP_ERR_UNSUPPORTED;   // six ghost layers: linked faces provide four
  for (int b = 0; b < nb; ++b) {
    const fsp_block& B = blk[b];
    if (B.ni < 1 || B.nj < 1 || B.ld < B.ni || B.ni > 8 * 65535 || B.nj > 2 * 65535) return FSP_ERR_INVALID_ARG;
    for (int f = 0; f < 4; ++f) {
      const int k = bc[4 * b + f];
      if (k < FSP_BC_PERIODIC || k > FSP_BC_LINK) return FSP_ERR_INVALID_ARG;
      const int along = f < 2 ? B.ni : B.nj, across = f < 2 ? B.nj : B.ni;
      if (k == FSP_BC_LINK) {
        const fsp_link& L = lk[4 * b + f];
        if (L.nbr < 0 || L.nbr >= nb || L.face < 0 || L.face > 3) return FSP_ERR_INVALID_ARG;
        const fsp_block& N = blk[L.nbr];
        // the faces must match node for node, and the neighbour must hold 4 ghost layers
        if ((L.face < 2 ? N.nj : N.ni) != across) return FSP_ERR_INVALID_ARG;
        if ((L.face < 2 ? N.ni : N.nj) < 4) return FSP_ERR_INVALID_ARG;
      } else if (k != FSP_BC_PERIODIC && along < 9) {
        return FSP_ERR_INVALID_ARG;
      }
    }
    if ((bc[4 * b] == FSP_BC_PERIODIC) != (bc[4 * b + 1] == FSP_BC_PERIODIC)) return FSP_ERR_INVALID_ARG;
    if ((bc[4 * b + 2] == FSP_BC_PERIODIC) != (bc[4 * b + 3] == FSP_BC_PERIODIC)) return FSP_ERR_INVALID_ARG;
  }
  return FSP_OK;
}

template <typename T>
T* carve(char*& cur, size_t count) {
  T* p = reinterpret_cast<T*>(cur);
  cur += al(count * sizeof(T));
  return p;
}

// The tiles of one direction in shape variant v, longest first.  CTAs start in table order,
// so with blocks of different sizes the short tiles fill the last wave instead of a few long
// ones running on an otherwise idle GPU (a marching xi CTA walks whole rows, 64 to 512 nodes
// on the cylinder).  The order does not change any result.
void tiles_for(const fsp_batch* h, int dir, int v, std::vector<TileRef>& out) {
  int T0, NL0;
  const bool fp64 = h->cfg.precision == FSP_FP64;
  tile_dims(h->cfg.scheme, dir, T0, NL0, v, fp64);
  std::vector<std::pair<long long, TileRef>> w;
  for (int b = 0; b < h->nb; ++b) {
    const fsp_block& B = h->blk[b];
    const int n = dir == 0 ? B.ni : B.nj, nl = dir == 0 ? B.nj : B.ni;
    int T = T0, NL = NL0;
    if (dir == 0 && v == MARCH) T = march_seg_len(n);   // rows split into equal segments
    if (dir == 1 && v == MARCH) {
      const int nmp = (h->cfg.scheme == S32 || h->cfg.scheme == S52) ? 2 : 1;
      T = march_eta_seg(fp64, nmp);
      NL = 32;
    }
    for (int by = 0; by < (nl + NL - 1) / NL; ++by)
      for (int bx = 0; bx < (n + T - 1) / T; ++bx) {
        // work: outputs along the line plus the stencil halo, times the lines
        const long long len = std::min(T, n - bx * T) + 8, lines = std::min(NL, nl - by * NL);
        w.push_back({len * lines, TileRef{b, bx, by}});
      }
  }
  std::stable_sort(w.begin(), w.end(), [](const std::pair<long long, TileRef>& a,
                                          const std::pair<long long, TileRef>& c) { return a.first > c.first; });
  out.clear();
  out.reserve(w.size());
  for (const auto& e : w) out.push_back(e.second);
}

// Switch one direction to shape variant v: the host and device tile tables (the device is
// synchronised first, since queued launches may read the table) and any captured graph.
// The marching passes are compiled for the default options only (sweep.cuh, default_options).
fsp_status set_tiles(fsp_batch* h, int dir, int v) {
  if (v < 0 || v >= nvariant(dir)) return FSP_ERR_INVALID_ARG;
  if (v == MARCH && !default_options(h->cfg)) return FSP_ERR_UNSUPPORTED;
  std::vector<TileRef>& t = dir == 0 ? h->tx : h->te;
  tiles_for(h, dir, v, t);
  if (cudaDeviceSynchronize() != cudaSuccess) return FSP_ERR_CUDA;
  if (cudaMemcpy(dir == 0 ? h->d_tx : h->d_te, t.data(), sizeof(TileRef) * t.size(), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return FSP_ERR_CUDA;
  (dir == 0 ? h->vx : h->ve) = v;
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
  return FSP_OK;
}

}  // namespace

extern "C" {

fsp_status fsp_batch_create(const fsp_config* cfg, int nblocks, const fsp_block* blocks, const int* bc,
                            const fsp_link* links, fsp_batch** out) {
  if (!out) return FSP_ERR_INVALID_ARG;
  *out = nullptr;
  if (fsp_status s = check_batch(cfg, nblocks, blocks, bc, links)) return s;
  fsp_batch* h = new (std::nothrow) fsp_batch();
  if (!h) return FSP_ERR_NOMEM;
  h->cfg = *cfg;
  h->nb = nblocks;
  if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return FSP_ERR_CUDA; }
  h->blk.assign(blocks, blocks + nblocks);
  h->bc.assign(bc, bc + 4 * nblocks);
  h->links.assign(links, links + 4 * nblocks);
  // host descriptors
  h->params.resize(nblocks);
  h->coords.resize(nblocks);
  size_t lam = 0, acc = 0, st = 0, mid = 0, nc = 0;
  for (int b = 0; b < nblocks; ++b) {
    const fsp_block& B = blocks[b];
    Params& P = h->params[b];
    std::memset(&P, 0, sizeof(P));
    P.ni = B.ni; P.nj = B.nj; P.ld = B.ld;
    P.interp = cfg->interp; P.ppm = cfg->ppm; P.linw = cfg->linear_weights;
    P.wz = cfg->weights; P.msplit = cfg->mid_split;
    P.gamma = cfg->gamma; P.alpha = cfg->lf_alpha; P.eps = cfg->eps;
    set_scheme_coefs(P, cfg->scheme, scheme_alpha_of(*cfg));
    for (int f = 0; f < 4; ++f) {
      P.bc[f] = bc[4 * b + f];
      for (int v = 0; v < 4; ++v) P.bcq[f][v] = cfg->bc_state[f][v];
      const fsp_link& L = links[4 * b + f];
      if (P.bc[f] == FSP_BC_LINK) {
        const fsp_block& N = blocks[L.nbr];
        P.lnb[f] = L.nbr; P.lface[f] = L.face; P.lrev[f] = L.reversed ? 1 : 0;
        P.lni[f] = N.ni; P.lnj[f] = N.nj; P.lld[f] = N.ld;
      }
    }
    P.mld = (long long)B.ni + 2 * G;
    P.mplane = P.mld * ((long long)B.nj + 2 * G);
    CoordBlock& C = h->coords[b];
    std::memset(&C, 0, sizeof(C));
    C.ni = B.ni; C.nj = B.nj;
    for (int f = 0; f < 4; ++f) {
      C.bc[f] = P.bc[f]; C.lnb[f] = P.lnb[f]; C.lface[f] = P.lface[f]; C.lrev[f] = P.lrev[f];
      C.loff[f][0] = links[4 * b + f].offset[0]; C.loff[f][1] = links[4 * b + f].offset[1];
    }
    for (int a = 0; a < 2; ++a)
      for (int k = 0; k < 2; ++k) C.per[a][k] = B.period[a][k];
    h->lam_off.push_back(lam);
    lam += (size_t)B.ni + B.nj;
    h->acc_off.push_back(acc);
    acc += al(4 * (size_t)B.nj * B.ld * acc_elem(cfg->precision));
    h->st_off.push_back(st);
    st += al(4 * (size_t)B.nj * B.ld * state_size(cfg->precision));
    // stored interface data (double accumulation only): xi [4][nj][ni + 3], eta [4][nj + 3][ni]
    h->mid_off.push_back(mid);
    if (cfg->precision != FSP_FP32) mid += al(8 * 4 * ((size_t)B.nj * (B.ni + 3) + (size_t)(B.nj + 3) * B.ni)) / 8;
    h->nc_off.push_back(nc);
    if (cfg->precision == FSP_FP64 && cfg->scheme != S32 && cfg->scheme != S52)
      nc += al(8 * (size_t)NC_COUNT * B.nj * B.ld) / 8;
    const int lr = 8 * (cfg->precision == FSP_FP64 ? lam_rows<double>() : lam_rows<float>());
    for (int by = 0; by < (B.nj + lr - 1) / lr; ++by)
      for (int bx = 0; bx < (B.ni + 31) / 32; ++bx) h->tl.push_back({b, bx, by});
  }
  h->lam_count = lam;
  for (int v = 0; v < NVARIANT; ++v) {
    std::vector<TileRef> t;
    tiles_for(h, 0, v, t);
    h->tx_cap = std::max(h->tx_cap, t.size());
    tiles_for(h, 1, v, t);
    h->te_cap = std::max(h->te_cap, t.size());
  }
  tiles_for(h, 0, 0, h->tx);
  tiles_for(h, 1, 0, h->te);
  const size_t bytes = al(sizeof(Params) * nblocks) + al(sizeof(CoordBlock) * nblocks) +
                       al(sizeof(TileRef) * h->tx_cap) + al(sizeof(TileRef) * h->te_cap) +
                       al(sizeof(TileRef) * h->tl.size()) + al(sizeof(double) * 2 * lam) + acc + 2 * st +
                       al(sizeof(void*) * T_COUNT * nblocks) + sizeof(double) * (mid + nc);
  if (cudaMalloc(&h->dmem, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return FSP_ERR_NOMEM;
  }
  char* cur = h->dmem;
  h->d_params = carve<Params>(cur, nblocks);
  h->d_coords = carve<CoordBlock>(cur, nblocks);
  h->d_tx = carve<TileRef>(cur, h->tx_cap);
  h->d_te = carve<TileRef>(cur, h->te_cap);
  h->d_tl = carve<TileRef>(cur, h->tl.size());
  h->d_lam = carve<double>(cur, 2 * lam);
  h->d_acc = cur; cur += acc;
  h->d_q1 = cur; cur += st;
  h->d_q2 = cur; cur += st;
  h->d_tab = reinterpret_cast<void**>(cur);
  cur += al(sizeof(void*) * T_COUNT * nblocks);
  h->d_mid = mid ? reinterpret_cast<double*>(cur) : nullptr;
  h->d_nc = nc ? reinterpret_cast<double*>(cur) + mid : nullptr;
  bool ok = cudaMemcpy(h->d_params, h->params.data(), sizeof(Params) * nblocks, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(h->d_tx, h->tx.data(), sizeof(TileRef) * h->tx.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(h->d_te, h->te.data(), sizeof(TileRef) * h->te.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(h->d_tl, h->tl.data(), sizeof(TileRef) * h->tl.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) { fsp_batch_destroy(h); return FSP_ERR_CUDA; }
  *out = h;
  return FSP_OK;
}

fsp_status fsp_batch_bind(fsp_batch* h, const double* const* x, const double* const* y, double* const* metrics,
                          void* const* Q) {
  if (!h || !x || !y || !metrics || !Q) return FSP_ERR_INVALID_ARG;
  for (int b = 0; b < h->nb; ++b)
    if (!dev_ptr(x[b]) || !dev_ptr(y[b]) || !dev_ptr(metrics[b]) || !dev_ptr(Q[b])) return FSP_ERR_INVALID_ARG;
  const int nb = h->nb;
  std::vector<void*> tab((size_t)T_COUNT * nb, nullptr);
  h->M.assign(metrics, metrics + nb);
  h->Q.resize(nb);
  for (int b = 0; b < nb; ++b) h->Q[b] = (char*)Q[b];
  for (int b = 0; b < nb; ++b) {
    h->params[b].met = metrics[b];
    h->coords[b].x = x[b];
    h->coords[b].y = y[b];
    tab[T_Q0 * nb + b] = Q[b];
    tab[T_Q1 * nb + b] = h->d_q1 + h->st_off[b];
    tab[T_Q2 * nb + b] = h->d_q2 + h->st_off[b];
    tab[T_ACC * nb + b] = h->d_acc + h->acc_off[b];
    tab[T_LX * nb + b] = h->d_lam + h->lam_off[b];
    tab[T_LE * nb + b] = h->d_lam + h->lam_off[b] + h->blk[b].nj;
    tab[T_LX2 * nb + b] = h->d_lam + h->lam_count + h->lam_off[b];
    tab[T_LE2 * nb + b] = h->d_lam + h->lam_count + h->lam_off[b] + h->blk[b].nj;
    if (h->d_mid) {
      const fsp_block& B = h->blk[b];
      tab[T_MX * nb + b] = h->d_mid + h->mid_off[b];
      tab[T_ME * nb + b] = h->d_mid + h->mid_off[b] + 4 * (size_t)B.nj * (B.ni + 3);
    }
    if (h->d_nc) tab[T_NC * nb + b] = h->d_nc + h->nc_off[b];
  }
  if (cudaMemcpy(h->d_params, h->params.data(), sizeof(Params) * nb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->d_coords, h->coords.data(), sizeof(CoordBlock) * nb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->d_tab, tab.data(), sizeof(void*) * tab.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return FSP_ERR_CUDA;
  h->bound = true;
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
  return FSP_OK;
}

fsp_status fsp_batch_metrics(fsp_batch* h, void* stream) {
  if (!h || !h->bound) return FSP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const Central cen = central_of(h->cfg.scheme, scheme_alpha_of(h->cfg));
  for (int b = 0; b < h->nb; ++b) {
    const long long n = (long long)(h->blk[b].ni + 2 * G) * (h->blk[b].nj + 2 * G);
    const long long want = (n + 255) / 256;
    metrics_mb_kernel<<<stride_grid(want, 8), 256, 0, st>>>(
        h->d_coords, b, cen, h->cfg.interp, h->cfg.scheme == S71 ? 8 : h->cfg.scheme >= S51 ? 6 : 4, h->M[b]);
    if (cudaGetLastError() != cudaSuccess) return FSP_ERR_CUDA;
  }
  return FSP_OK;
}

}  // extern "C"

namespace {

// The midpoint metrics of every block from the bound metrics (FP64 and mixed batches; a
// no-op for FP32, whose passes interpolate in float): launched before each right-hand side,
// RK3 step and tuning run, so metrics written between calls are always taken up.
fsp_status batch_mids(fsp_batch* h, cudaStream_t st) {
  if (!h->d_mid) return FSP_OK;
  const int nb = h->nb, sc = h->cfg.scheme;
  void** T = h->d_tab;
  const dim3 grid(64, nb);
  auto mx = reinterpret_cast<double* const*>(T + T_MX * nb);
  auto me = reinterpret_cast<double* const*>(T + T_ME * nb);
  // the direction is read by the FP64 passes only (the mixed passes take it in float)
  const bool dir = h->cfg.precision == FSP_FP64;
  if (sc == S71) {
    if (dir) mid_batch_kernel<4, true><<<grid, 256, 0, st>>>(h->d_params, mx, me);
    else mid_batch_kernel<4, false><<<grid, 256, 0, st>>>(h->d_params, mx, me);
  } else if (sc == S51 || sc == S52) {
    if (dir) mid_batch_kernel<3, true><<<grid, 256, 0, st>>>(h->d_params, mx, me);
    else mid_batch_kernel<3, false><<<grid, 256, 0, st>>>(h->d_params, mx, me);
  } else {
    if (dir) mid_batch_kernel<2, true><<<grid, 256, 0, st>>>(h->d_params, mx, me);
    else mid_batch_kernel<2, false><<<grid, 256, 0, st>>>(h->d_params, mx, me);
  }
  return cudaGetLastError() == cudaSuccess ? FSP_OK : FSP_ERR_CUDA;
}

// one right-hand side of every block; input table `in`, output table `out`; mode 0:
// dQ/dt, mode 1: RK stage out = ca Q0 + cb (in + dt dQ/dt)
fsp_status batch_lambda(fsp_batch* h, int in, cudaStream_t st) {
  const int nb = h->nb;
  void** T = h->d_tab;
  if (cudaMemsetAsync(h->d_lam, 0, sizeof(double) * h->lam_count, st) != cudaSuccess) return FSP_ERR_CUDA;
  dim3 blk(32, 8);
  if (h->cfg.precision == FSP_FP64)
    lambda_batch_kernel<double><<<(unsigned)h->tl.size(), blk, 0, st>>>(
        h->d_params, h->d_tl, reinterpret_cast<const double* const*>(T + in * nb),
        reinterpret_cast<double* const*>(T + T_LX * nb), reinterpret_cast<double* const*>(T + T_LE * nb));
  else
    lambda_batch_kernel<float><<<(unsigned)h->tl.size(), blk, 0, st>>>(
        h->d_params, h->d_tl, reinterpret_cast<const float* const*>(T + in * nb),
        reinterpret_cast<double* const*>(T + T_LX * nb), reinterpret_cast<double* const*>(T + T_LE * nb));
  return cudaGetLastError() == cudaSuccess ? FSP_OK : FSP_ERR_CUDA;
}

// Line maxima of a stage: LAM_KERNEL takes them from the input state into buffer A;
// LAM_A / LAM_B find them already in that buffer, written by the previous stage's marching
// eta pass.  lam_out (mode 1 only): the buffer (0 A, 1 B) that this stage's marching eta pass
// fills with the maxima of the state it writes, or -1.
enum { LAM_KERNEL = 0, LAM_A = 1, LAM_B = 2 };

fsp_status batch_stage(fsp_batch* h, int in, int out, int mode, double ca, double cb, double dt, cudaStream_t st,
                       int lam_in = LAM_KERNEL, int lam_out = -1) {
  const int nb = h->nb;
  void** T = h->d_tab;
  if (lam_in == LAM_KERNEL)
    if (fsp_status s = batch_lambda(h, in, st)) return s;
  if (lam_out >= 0 &&
      cudaMemsetAsync(h->d_lam + lam_out * h->lam_count, 0, sizeof(double) * h->lam_count, st) != cudaSuccess)
    return FSP_ERR_CUDA;
  const int lx = lam_in == LAM_B ? T_LX2 : T_LX, le = lam_in == LAM_B ? T_LE2 : T_LE;
  PassTables xi{h->d_params, h->d_tx, T + in * nb, T + lx * nb, nullptr, T + T_ACC * nb, nullptr, nullptr};
  PassTables eta{h->d_params, h->d_te, T + in * nb, T + le * nb, T + T_ACC * nb, nullptr, T + out * nb,
                 T + T_Q0 * nb};
  if (h->d_mid) {
    xi.mid = T + T_MX * nb;
    eta.mid = T + T_ME * nb;
  }
  // FP64 with both passes marching: the xi pass leaves each node's characteristic data for
  // the eta pass of the same right-hand side
  // the one-midpoint schemes only: the two-midpoint eta pass has no shared memory left for it
  const bool one_mid = h->cfg.scheme != S32 && h->cfg.scheme != S52;
  if (h->d_nc && one_mid && h->vx == MARCH && h->ve == MARCH) xi.nc = eta.nc = T + T_NC * nb;
  if (lam_out >= 0) {
    eta.lxo = T + (lam_out ? T_LX2 : T_LX) * nb;
    eta.leo = T + (lam_out ? T_LE2 : T_LE) * nb;
    mode = 2;
  }
  const int ntx = (int)h->tx.size(), nte = (int)h->te.size();
  cudaError_t e = h->cfg.precision == FSP_FP64
                      ? batch_fp64(h->cfg.scheme, mode, xi, ntx, h->vx, eta, nte, h->ve, ca, cb, dt, st)
                      : batch_fp32(h->cfg.scheme, h->cfg.precision == FSP_FP32_MIXED, mode, xi, ntx, h->vx, eta,
                                   nte, h->ve, ca, cb, dt, st);
  return e == cudaSuccess ? FSP_OK : FSP_ERR_CUDA;
}

// One TVD-RK3 step.  The first stage's line maxima come from the line-maxima kernel (the
// caller may have written Q between steps); with the marching eta pass, stages 1 and 2 take
// the maxima of the states they write (Q1 into B, Q2 into A) for the stage after.  Not in
// mixed precision, whose eta CTAs would no longer fit two to an SM with the extra operands.
fsp_status batch_rk3(fsp_batch* h, double dt, cudaStream_t st) {
  const bool fuse = h->ve == MARCH && h->cfg.precision != FSP_FP32_MIXED;
  if (fsp_status s = batch_mids(h, st)) return s;
  if (fsp_status s = batch_stage(h, T_Q0, T_Q1, 1, 0.0, 1.0, dt, st, LAM_KERNEL, fuse ? 1 : -1)) return s;
  if (fsp_status s = batch_stage(h, T_Q1, T_Q2, 1, 0.75, 0.25, dt, st, fuse ? LAM_B : LAM_KERNEL, fuse ? 0 : -1))
    return s;
  return batch_stage(h, T_Q2, T_Q0, 1, 1.0 / 3.0, 2.0 / 3.0, dt, st, fuse ? LAM_A : LAM_KERNEL);
}

}  // namespace

extern "C" {

fsp_status fsp_batch_rhs(fsp_batch* h, void* const* dQdt, void* stream) {
  if (!h || !h->bound || !dQdt) return FSP_ERR_INVALID_ARG;
  for (int b = 0; b < h->nb; ++b)
    if (!dev_ptr(dQdt[b])) return FSP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // the output table is copied from pageable memory: the call returns once it is staged
  if (cudaMemcpyAsync(h->d_tab + T_OUT * h->nb, dQdt, sizeof(void*) * h->nb, cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return FSP_ERR_CUDA;
  if (fsp_status s = batch_mids(h, st)) return s;
  return batch_stage(h, T_Q0, T_OUT, 0, 0.0, 0.0, 0.0, st);
}

fsp_status fsp_batch_flux_difference(fsp_batch* h, int dir, void* const* D, void* stream) {
  if (!h || !h->bound || !D || (dir != 0 && dir != 1)) return FSP_ERR_INVALID_ARG;
  for (int b = 0; b < h->nb; ++b)
    if (!dev_ptr(D[b])) return FSP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = h->nb;
  void** T = h->d_tab;
  if (cudaMemcpyAsync(T + T_OUT * nb, D, sizeof(void*) * nb, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return FSP_ERR_CUDA;
  const PassTables t{h->d_params, dir == 0 ? h->d_tx : h->d_te, T + T_Q0 * nb, T + (dir == 0 ? T_LX : T_LE) * nb,
                     nullptr, T + T_OUT * nb, nullptr, nullptr, nullptr, nullptr,
                     h->d_mid ? T + (dir == 0 ? T_MX : T_ME) * nb : nullptr};
  const int nt = (int)(dir == 0 ? h->tx.size() : h->te.size());
  const int v = dir == 0 ? h->vx : h->ve;
  cudaError_t e = h->cfg.precision == FSP_FP64
                      ? batch_direction_fp64(h->cfg.scheme, dir, t, nt, v, st)
                      : batch_direction_fp32(h->cfg.scheme, h->cfg.precision == FSP_FP32_MIXED, dir, t, nt, v, st);
  return e == cudaSuccess ? FSP_OK : FSP_ERR_CUDA;
}

fsp_status fsp_batch_rk3_step(fsp_batch* h, double dt, void* stream) {
  if (!h || !h->bound) return FSP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (h->gexec && dt == h->gdt) return cudaGraphLaunch(h->gexec, st) == cudaSuccess ? FSP_OK : FSP_ERR_CUDA;
  return batch_rk3(h, dt, st);
}

fsp_status fsp_batch_rk3_step_host(fsp_batch* h, const void* const* q_in, void* const* q_out, double dt,
                                   void* stream) {
  if (!h || !h->bound || !q_in || !q_out) return FSP_ERR_INVALID_ARG;
  const int nb = h->nb;
  for (int b = 0; b < nb; ++b) {
    if (!q_in[b] || !q_out[b]) return FSP_ERR_INVALID_ARG;
    cudaPointerAttributes a;
    for (const void* p : {q_in[b], (const void*)q_out[b]}) {
      if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return FSP_ERR_INVALID_ARG; }
      if (a.type == cudaMemoryTypeDevice) return FSP_ERR_INVALID_ARG;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t es = state_size(h->cfg.precision);
  // Runs of blocks whose states sit the same distance apart on the device and in both host
  // arrays, less than 512 bytes beyond each block's end, move as one copy (padding included).
  auto copy_runs = [&](bool in) -> bool {
    for (int b = 0; b < nb;) {
      const char* hs = in ? (const char*)q_in[b] : (const char*)q_out[b];
      size_t len = 4 * (size_t)h->blk[b].nj * h->blk[b].ld * es;
      int e = b + 1;
      for (; e < nb; ++e) {
        const ptrdiff_t gd = h->Q[e] - h->Q[e - 1];
        const ptrdiff_t gi = (const char*)q_in[e] - (const char*)q_in[e - 1];
        const ptrdiff_t go = (const char*)q_out[e] - (const char*)q_out[e - 1];
        const size_t prev = 4 * (size_t)h->blk[e - 1].nj * h->blk[e - 1].ld * es;
        if (gd != gi || gd != go || gd < (ptrdiff_t)prev || gd >= (ptrdiff_t)(prev + 512)) break;
        len = (size_t)(h->Q[e] - h->Q[b]) + 4 * (size_t)h->blk[e].nj * h->blk[e].ld * es;
      }
      const cudaError_t r = in ? cudaMemcpyAsync(h->Q[b], hs, len, cudaMemcpyHostToDevice, st)
                               : cudaMemcpyAsync((char*)q_out[b], h->Q[b], len, cudaMemcpyDeviceToHost, st);
      if (r != cudaSuccess) return false;
      b = e;
    }
    return true;
  };
  if (!copy_runs(true)) return FSP_ERR_CUDA;
  if (fsp_status s = fsp_batch_rk3_step(h, dt, stream)) return s;
  return copy_runs(false) ? FSP_OK : FSP_ERR_CUDA;
}

fsp_status fsp_batch_capture_graph(fsp_batch* h, double dt, void* stream) {
  if (!h || !h->bound) return FSP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
  // one eager step on the caller's stream: kernel attributes are set and modules loaded
  // outside the capture
  if (fsp_status s = batch_rk3(h, dt, st)) return s;
  // record on a private stream (the legacy default stream cannot be captured); nothing
  // runs during the recording, and the graph is later launched on the caller's stream
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return FSP_ERR_CUDA;
  cudaGraph_t g = nullptr;
  fsp_status s = FSP_ERR_CUDA;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    s = batch_rk3(h, dt, cs);
    if (cudaStreamEndCapture(cs, &g) != cudaSuccess) s = FSP_ERR_CUDA;
  }
  cudaStreamDestroy(cs);
  if (s == FSP_OK && g && cudaGraphInstantiate(&h->gexec, g, 0) == cudaSuccess) {
    h->gdt = dt;
  } else {
    h->gexec = nullptr;
    if (s == FSP_OK) s = FSP_ERR_CUDA;
  }
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  return s;
}

}  // extern "C"

namespace {

// Median duration (ms) of one direction's pass over every block (difference mode, into
// the xi accumulators, which the next right-hand side overwrites) in the current variant.
fsp_status time_direction(fsp_batch* h, int dir, cudaStream_t st, float* ms) {
  const int nb = h->nb;
  void** T = h->d_tab;
  const PassTables t{h->d_params, dir == 0 ? h->d_tx : h->d_te, T + T_Q0 * nb, T + (dir == 0 ? T_LX : T_LE) * nb,
                     nullptr, T + T_ACC * nb, nullptr, nullptr, nullptr, nullptr,
                     h->d_mid ? T + (dir == 0 ? T_MX : T_ME) * nb : nullptr};
  const int nt = (int)(dir == 0 ? h->tx.size() : h->te.size());
  const int v = dir == 0 ? h->vx : h->ve;
  auto run = [&]() {
    return h->cfg.precision == FSP_FP64
               ? batch_direction_fp64(h->cfg.scheme, dir, t, nt, v, st)
               : batch_direction_fp32(h->cfg.scheme, h->cfg.precision == FSP_FP32_MIXED, dir, t, nt, v, st);
  };
  constexpr int WARM = 2, REPS = 5;
  cudaEvent_t ev[REPS + 1];
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return FSP_ERR_CUDA;
  bool ok = true;
  for (int k = 0; k < WARM; ++k) ok = ok && run() == cudaSuccess;
  ok = ok && cudaEventRecord(ev[0], st) == cudaSuccess;
  for (int k = 0; k < REPS; ++k) ok = ok && run() == cudaSuccess && cudaEventRecord(ev[k + 1], st) == cudaSuccess;
  ok = ok && cudaEventSynchronize(ev[REPS]) == cudaSuccess;
  std::vector<float> d(REPS);
  for (int k = 0; ok && k < REPS; ++k) ok = cudaEventElapsedTime(&d[k], ev[k], ev[k + 1]) == cudaSuccess;
  for (auto& e : ev) cudaEventDestroy(e);
  if (!ok) return FSP_ERR_CUDA;
  std::sort(d.begin(), d.end());
  *ms = d[REPS / 2];
  return FSP_OK;
}

// The table key: device, scheme and arithmetic options, and the block sizes (FNV-1a hash).
std::string tune_key(const fsp_batch* h) {
  cudaDeviceProp p;
  std::string name = "gpu";
  int sms = 0;
  if (cudaGetDeviceProperties(&p, h->device) == cudaSuccess) { name = p.name; sms = p.multiProcessorCount; }
  for (char& c : name)
    if (c == ' ' || c == '\t') c = '_';
  unsigned long long x = 1469598103934665603ULL;
  auto mix = [&](long long v) {
    for (int k = 0; k < 8; ++k) { x ^= (unsigned long long)((v >> (8 * k)) & 0xff); x *= 1099511628211ULL; }
  };
  for (const fsp_block& B : h->blk) { mix(B.ni); mix(B.nj); }
  char buf[320];
  std::snprintf(buf, sizeof buf, "%s|sm%d|scheme%d|prec%d|interp%d|ppm%d|linw%d|nb%d|%016llx", name.c_str(), sms,
                h->cfg.scheme, h->cfg.precision, h->cfg.interp, h->cfg.ppm, h->cfg.linear_weights, h->nb, x);
  std::string key = buf;
  if (h->cfg.weights || h->cfg.mid_split || scheme_alpha_of(h->cfg) != 1.0) {
    // the options beyond the paper's schemes (keys of the printed schemes stay as they were)
    std::snprintf(buf, sizeof buf, "|wz%d|split%d|alpha%.17g", h->cfg.weights, h->cfg.mid_split,
                  scheme_alpha_of(h->cfg));
    key += buf;
  }
  return key;
}

bool table_lookup(const char* path, const std::string& key, int* vx, int* ve) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == '#') continue;
    char k[512];
    int a, b;
    if (std::sscanf(line, "%511s %d %d", k, &a, &b) == 3 && key == k && a >= 0 && a < nvariant(0) && b >= 0 &&
        b < nvariant(1)) {
      *vx = a;
      *ve = b;
      found = true;  // the last entry for a key wins
    }
  }
  std::fclose(f);
  return found;
}

}  // namespace

extern "C" {

fsp_status fsp_batch_tune(fsp_batch* h, const char* table_path, void* stream) {
  if (!h || !h->bound) return FSP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const std::string key = tune_key(h);
  int best[2] = {-1, -1};
  if (table_path && table_lookup(table_path, key, &best[0], &best[1])) {
    if (fsp_status s = set_tiles(h, 0, best[0])) return s;
    return set_tiles(h, 1, best[1]);
  }
  if (fsp_status s = batch_lambda(h, T_Q0, st)) return s;
  if (fsp_status s = batch_mids(h, st)) return s;
  float best_ms[2] = {0, 0};
  for (int dir = 0; dir < 2; ++dir) {
    for (int v = 0; v < nvariant(dir); ++v) {
      if (v == MARCH && !default_options(h->cfg)) continue;
      if (fsp_status s = set_tiles(h, dir, v)) return s;
      float ms = 0;
      if (fsp_status s = time_direction(h, dir, st, &ms)) return s;
      if (best[dir] < 0 || ms < best_ms[dir]) { best[dir] = v; best_ms[dir] = ms; }
    }
    if (fsp_status s = set_tiles(h, dir, best[dir])) return s;
  }
  if (table_path) {
    FILE* f = std::fopen(table_path, "a");
    if (!f) return FSP_ERR_INVALID_ARG;
    std::fprintf(f, "%s %d %d %.4f %.4f\n", key.c_str(), best[0], best[1], best_ms[0], best_ms[1]);
    std::fclose(f);
  }
  return FSP_OK;
}

fsp_status fsp_batch_set_tile_shape(fsp_batch* h, int dir, int variant) {
  if (!h || (dir != 0 && dir != 1)) return FSP_ERR_INVALID_ARG;
  return set_tiles(h, dir, variant);
}

fsp_status fsp_batch_tile_shape(const fsp_batch* h, int dir, int* variant, int* lines, int* outputs) {
  if (!h || (dir != 0 && dir != 1)) return FSP_ERR_INVALID_ARG;
  const int v = dir == 0 ? h->vx : h->ve;
  int T, NL;
  tile_dims(h->cfg.scheme, dir, T, NL, v, h->cfg.precision == FSP_FP64);
  if (variant) *variant = v;
  if (lines) *lines = NL;
  if (outputs) *outputs = T;
  return FSP_OK;
}

fsp_status fsp_batch_destroy(fsp_batch* h) {
  if (!h) return FSP_OK;
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->dmem) cudaFree(h->dmem);
  delete h;
  return FSP_OK;
}

}  // extern "C"
