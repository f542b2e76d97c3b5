// fsp_internal.h -- declarations shared by the translation units of libfsp.
#pragma once

#include <cuda_runtime.h>

#include "../../include/fsp.h"
#include "fsp_device.cuh"

namespace fsp {

// The scheme's free parameter (0 in the configuration means the printed scheme, 1).
double scheme_alpha_of(const fsp_config& c);
// Whether every option beyond the paper's schemes is at its default (the marching kernels
// and the adjoint take only these).
bool default_options(const fsp_config& c);
// FSP_ERR_INVALID_ARG for an option out of range, FSP_ERR_UNSUPPORTED for a combination without
// kernels (the midpoint splittings in mixed precision).
fsp_status check_options(const fsp_config& c);

// Grid size of a grid-stride launch: the blocks the work needs, at most per_sm resident
// blocks on each multiprocessor of the current device (its count read once per device).
int stride_grid(long long blocks, int per_sm);

// Kernel parameters of one block from the public configuration (host side).
Params make_params(const fsp_config& cfg, const fsp_block& blk, const double* metrics);

// Status of a right-hand-side launch sequence: a scheme/precision pair without kernels
// (cudaErrorNotSupported) is FSP_ERR_UNSUPPORTED, any other failure FSP_ERR_CUDA.
fsp_status rhs_status(cudaError_t e);

// Launchers (enqueue only; return the launch status).
cudaError_t launch_metrics(const fsp_config& cfg, const fsp_block& blk, const double* x,
                           const double* y, double* M, cudaStream_t st);

// Per-line spectral maxima (without the factor alpha) into lam_xi[nj], lam_eta[ni];
// cfl_max (nullable) receives the largest per-node CFL rate.  Buffers must be zeroed.
cudaError_t launch_lambda(const Params& P, int precision, const void* Q, double* lam_xi,
                          double* lam_eta, double* cfl_max, cudaStream_t st);

// One right-hand-side evaluation in two passes.  mode 0: out = dQ/dt.  mode 1: RK stage
// out = ca * Qn + cb * (Q + dt * dQ/dt).  Racc: 4 * nj * ld scratch of the state type.
cudaError_t launch_rhs(int scheme, int precision, const Params& P, const void* Q,
                       const double* lam_xi, const double* lam_eta, void* Racc, void* out,
                       int mode, const void* Qn, double ca, double cb, double dt, cudaStream_t st);

// One direction only: mode 0 writes the difference to out; mode 1 writes
// -(acc + difference) / J^-1.
cudaError_t launch_flux_difference(int scheme, int precision, const Params& P, const void* Q,
                                   const double* lam, int dir, int mode, const void* acc, void* out,
                                   cudaStream_t st);

cudaError_t launch_cfl_finish(const double* cfl_max, double cfl, double* dt_out, cudaStream_t st);

cudaError_t launch_check_state(const fsp_block& blk, int precision, double gamma, const void* Q, long long* first,
                               cudaStream_t st);
cudaError_t launch_norms(const fsp_block& blk, int precision, const void* A, const void* B,
                         double* out, cudaStream_t st);

cudaError_t launch_fma_peak(int precision, int blocks, int iters, void* sink, cudaStream_t st);
cudaError_t launch_round_to_float(const double* in, float* oi, float* oh, long long n, cudaStream_t st);
cudaError_t launch_widen_to_double(const float* in, double* oi, double* oh, long long n, cudaStream_t st);
cudaError_t launch_reciprocal_check(const double* in, double* out, long long n, cudaStream_t st);

}  // namespace fsp
