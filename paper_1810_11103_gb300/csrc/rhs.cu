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
// The sweep kernel itself is in sweep.cuh.
#include "fsp_internal.h"
#include "sweep.cuh"

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
  // maxima in the state's arithmetic (non-negative values order the same in float and
  // double); one conversion per line at the atomic
  __shared__ Real col[8][33];
  __shared__ Real cfl_s[8];
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
  Real sx = Real(0), se = Real(0), rate = Real(0);
  if (i < P.ni && j < P.nj) node_speeds(P, Q, i, j, sx, se, rate);
  // row maximum across the warp (one row of 32 nodes)
  Real rx = sx, rr = rate;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    rx = max(rx, __shfl_xor_sync(0xffffffffu, rx, off));
    rr = max(rr, __shfl_xor_sync(0xffffffffu, rr, off));
  }
  if (threadIdx.x == 0 && j < P.nj) atomic_max_pos(lam_xi + j, (double)rx);
  col[threadIdx.y][threadIdx.x] = se;
  if (threadIdx.x == 0) cfl_s[threadIdx.y] = rr;
  __syncthreads();
  if (threadIdx.y == 0 && i < P.ni) {
    Real m = col[0][threadIdx.x];
#pragma unroll
    for (int r = 1; r < 8; ++r) m = max(m, col[r][threadIdx.x]);
    atomic_max_pos(lam_eta + i, (double)m);
  }
  if (cfl_max && threadIdx.x == 0 && threadIdx.y == 0) {
    Real m = cfl_s[0];
#pragma unroll
    for (int r = 1; r < 8; ++r) m = max(m, cfl_s[r]);
    atomic_max_pos(cfl_max, (double)m);
  }
}

// ------------------------------------------------------------------------------------
// Directional sweeps (sweep.cuh): FP64 instantiations here, FP32 in rhs_fp32.cu
// ------------------------------------------------------------------------------------
cudaError_t rhs_fp64(int scheme, const Params& P, const void* Q, const double* lx, const double* le,
                     void* Racc, void* out, int mode, const void* Qn, double ca, double cb, double dt,
                     cudaStream_t st) {
  auto q = static_cast<const double*>(Q);
  auto r = static_cast<double*>(Racc);
  auto o = static_cast<double*>(out);
  auto qn = static_cast<const double*>(Qn);
  switch (scheme) {
    case S31: return rhs_passes<S31, double, double>(P, q, lx, le, r, o, mode, qn, ca, cb, dt, st);
    case S32: return rhs_passes<S32, double, double>(P, q, lx, le, r, o, mode, qn, ca, cb, dt, st);
    case S51: return rhs_passes<S51, double, double>(P, q, lx, le, r, o, mode, qn, ca, cb, dt, st);
    case S52: return rhs_passes<S52, double, double>(P, q, lx, le, r, o, mode, qn, ca, cb, dt, st);
    case S74: return rhs_passes<S74, double, double>(P, q, lx, le, r, o, mode, qn, ca, cb, dt, st);
    default:  return rhs_passes<S71, double, double>(P, q, lx, le, r, o, mode, qn, ca, cb, dt, st);
  }
}

cudaError_t flux_difference_fp64(int scheme, const Params& P, const void* Q, const double* lam, int dir,
                                 int mode, const void* acc, void* out, cudaStream_t st) {
  auto q = static_cast<const double*>(Q);
  auto a = static_cast<const double*>(acc);
  switch (scheme) {
    case S31: return flux_difference_passes<S31, double, double>(P, q, lam, dir, mode, a, out, st);
    case S32: return flux_difference_passes<S32, double, double>(P, q, lam, dir, mode, a, out, st);
    case S51: return flux_difference_passes<S51, double, double>(P, q, lam, dir, mode, a, out, st);
    case S52: return flux_difference_passes<S52, double, double>(P, q, lam, dir, mode, a, out, st);
    case S74: return flux_difference_passes<S74, double, double>(P, q, lam, dir, mode, a, out, st);
    default:  return flux_difference_passes<S71, double, double>(P, q, lam, dir, mode, a, out, st);
  }
}

cudaError_t launch_rhs(int scheme, int precision, const Params& P, const void* Q,
                       const double* lam_xi, const double* lam_eta, void* Racc, void* out, int mode,
                       const void* Qn, double ca, double cb, double dt, cudaStream_t st) {
  if (precision == FSP_FP64) return rhs_fp64(scheme, P, Q, lam_xi, lam_eta, Racc, out, mode, Qn, ca, cb, dt, st);
  return rhs_fp32(scheme, precision == FSP_FP32_MIXED, P, Q, lam_xi, lam_eta, Racc, out, mode, Qn, ca, cb,
                  dt, st);
}

cudaError_t launch_flux_difference(int scheme, int precision, const Params& P, const void* Q,
                                   const double* lam, int dir, int mode, const void* acc, void* out,
                                   cudaStream_t st) {
  if (precision == FSP_FP64) return flux_difference_fp64(scheme, P, Q, lam, dir, mode, acc, out, st);
  return flux_difference_fp32(scheme, precision == FSP_FP32_MIXED, P, Q, lam, dir, mode, acc, out, st);
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

// State health: the smallest linear index j ni + i of a node whose state is not finite or not
// physical (rho <= 0 or p <= 0), by an atomic minimum over the unsigned index (all-ones, which
// reads -1 as a signed integer, when every node is valid).
template <typename Real>
__global__ void __launch_bounds__(256) check_state_kernel(int ni, int nj, long long ld, double gm1,
                                                          const Real* __restrict__ Q,
                                                          unsigned long long* __restrict__ first) {
  const long long N = (long long)ni * nj, plane = (long long)nj * ld;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
    const long long o = (t / ni) * ld + t % ni;
    const double r = Q[o], mu = Q[plane + o], mv = Q[2 * plane + o], e = Q[3 * plane + o];
    const double p = gm1 * (e - 0.5 * (mu * mu + mv * mv) / r);
    const bool ok = isfinite(r) && isfinite(mu) && isfinite(mv) && isfinite(e) && r > 0.0 && p > 0.0;
    if (!ok) atomicMin(first, (unsigned long long)t);
  }
}

cudaError_t launch_check_state(const fsp_block& blk, int precision, double gamma, const void* Q, long long* first,
                               cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(first, 0xff, sizeof(long long), st);
  if (e != cudaSuccess) return e;
  const long long N = (long long)blk.ni * blk.nj;
  const long long want = (N + 255) / 256;
  const int grid = stride_grid(want, 4);
  auto f = reinterpret_cast<unsigned long long*>(first);
  if (precision == FSP_FP64)
    check_state_kernel<double><<<grid, 256, 0, st>>>(blk.ni, blk.nj, blk.ld, gamma - 1.0, static_cast<const double*>(Q), f);
  else
    check_state_kernel<float><<<grid, 256, 0, st>>>(blk.ni, blk.nj, blk.ld, gamma - 1.0, static_cast<const float*>(Q), f);
  return cudaGetLastError();
}

cudaError_t launch_norms(const fsp_block& blk, int precision, const void* A, const void* B,
                         double* out, cudaStream_t st) {
  // out doubles as the accumulator space, then is rewritten in place by one thread
  cudaError_t e = cudaMemsetAsync(out, 0, 8 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  const long long N = (long long)blk.ni * blk.nj;
  const long long want = (N + 255) / 256;
  const int grid = stride_grid(want, 4);
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
