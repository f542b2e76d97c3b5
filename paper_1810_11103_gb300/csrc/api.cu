// api.cu -- the C ABI of libfsp (include/fsp.h): argument checks on the host, workspace
// layout, and the launch sequences of each entry point.
#include <atomic>
#include <cstring>

#include "fsp_internal.h"

using namespace fsp;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

size_t elem_size(int prec) { return prec == FSP_FP64 ? sizeof(double) : sizeof(float); }
// element size of the xi accumulator: the flux arithmetic's type
size_t acc_size(int prec) { return prec == FSP_FP32 ? sizeof(float) : sizeof(double); }

// Workspace: [lam_xi nj | lam_eta ni | cfl 1] doubles, then the xi accumulator and two
// RK stage buffers, each 4 * nj * ld elements of the state type.
struct WsLayout {
  size_t lam, racc, q1, q2, total;
};

WsLayout ws_layout(const fsp_config& c, const fsp_block& b) {
  WsLayout L;
  const size_t state = 4 * (size_t)b.nj * (size_t)b.ld * elem_size(c.precision);
  const size_t acc = 4 * (size_t)b.nj * (size_t)b.ld * acc_size(c.precision);
  L.lam = 0;
  L.racc = align_up(((size_t)b.ni + b.nj + 1) * sizeof(double));
  L.q1 = L.racc + align_up(acc);
  L.q2 = L.q1 + align_up(state);
  L.total = L.q2 + align_up(state);
  return L;
}

bool device_pointer(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

fsp_status check_cfg(const fsp_config* c, const fsp_block* b) {
  if (!c || !b) return FSP_ERR_INVALID_ARG;
  if (c->scheme < 0 || c->scheme > 5) return FSP_ERR_INVALID_ARG;
  if (c->precision < FSP_FP64 || c->precision > FSP_FP32_MIXED) return FSP_ERR_INVALID_ARG;
  if (c->interp < 0 || c->interp > 1) return FSP_ERR_INVALID_ARG;
  for (int f = 0; f < 4; ++f)
    if (c->bc[f] < FSP_BC_PERIODIC || c->bc[f] > FSP_BC_FARFIELD) return FSP_ERR_INVALID_ARG;
  if ((c->bc[0] == FSP_BC_PERIODIC) != (c->bc[1] == FSP_BC_PERIODIC)) return FSP_ERR_INVALID_ARG;
  if ((c->bc[2] == FSP_BC_PERIODIC) != (c->bc[3] == FSP_BC_PERIODIC)) return FSP_ERR_INVALID_ARG;
  if (!(c->gamma > 1.0) || !(c->lf_alpha > 0.0) || !(c->eps > 0.0)) return FSP_ERR_INVALID_ARG;
  if (fsp_status s = check_options(*c)) return s;
  // the four-midpoint scheme reaches six nodes beyond a face: periodic blocks only, and one
  // precision (its h is not regrouped for the mixed path)
  if (c->scheme == S74 && (c->bc[0] != FSP_BC_PERIODIC || c->bc[2] != FSP_BC_PERIODIC)) return FSP_ERR_UNSUPPORTED;
  if (c->scheme == S74 && c->precision == FSP_FP32_MIXED) return FSP_ERR_UNSUPPORTED;
  if (b->ni < 1 || b->nj < 1 || b->ld < b->ni) return FSP_ERR_INVALID_ARG;
  if (c->bc[0] != FSP_BC_PERIODIC && b->ni < 9) return FSP_ERR_INVALID_ARG;
  if (c->bc[2] != FSP_BC_PERIODIC && b->nj < 9) return FSP_ERR_INVALID_ARG;
  // index arithmetic inside the kernels is 32-bit per direction, 64-bit per plane; the
  // sweep grids put lines on gridDim.y (2 rows or 8 columns per CTA, at most 65535 CTAs)
  if (b->ni > 8 * 65535 || b->nj > 2 * 65535) return FSP_ERR_INVALID_ARG;
  return FSP_OK;
}

fsp_status cuda_status(cudaError_t e) { return e == cudaSuccess ? FSP_OK : FSP_ERR_CUDA; }

#define FSP_TRY(expr)                                  \
  do {                                                 \
    cudaError_t e_ = (expr);                           \
    if (e_ != cudaSuccess) return FSP_ERR_CUDA;        \
  } while (0)

}  // namespace

namespace fsp {

Params make_params(const fsp_config& c, const fsp_block& b, const double* metrics) {
  Params P;
  std::memset(&P, 0, sizeof(P));
  P.ni = b.ni; P.nj = b.nj; P.ld = b.ld;
  for (int f = 0; f < 4; ++f) P.bc[f] = c.bc[f];
  P.interp = c.interp; P.ppm = c.ppm; P.linw = c.linear_weights;
  P.wz = c.weights; P.msplit = c.mid_split;
  P.gamma = c.gamma; P.alpha = c.lf_alpha; P.eps = c.eps;
  set_scheme_coefs(P, c.scheme, scheme_alpha_of(c));
  for (int f = 0; f < 4; ++f)
    for (int v = 0; v < 4; ++v) P.bcq[f][v] = c.bc_state[f][v];
  P.met = metrics;
  P.mld = (long long)b.ni + 2 * G;
  P.mplane = P.mld * ((long long)b.nj + 2 * G);
  return P;
}

double scheme_alpha_of(const fsp_config& c) { return c.scheme_alpha == 0.0 ? 1.0 : c.scheme_alpha; }

bool default_options(const fsp_config& c) {
  return c.ppm == 1 && c.linear_weights == 0 && c.interp == 0 && c.weights == 0 && c.mid_split == 0 &&
         scheme_alpha_of(c) == 1.0;
}

fsp_status check_options(const fsp_config& c) {
  if (c.weights < 0 || c.weights > 1 || c.mid_split < 0 || c.mid_split > 2) return FSP_ERR_INVALID_ARG;
  const double a = scheme_alpha_of(c);
  if (!(a > 0.0) || !(a < 1e6)) return FSP_ERR_INVALID_ARG;
  if (a != 1.0 && (c.scheme == S32 || c.scheme == S52 || c.scheme == S74)) return FSP_ERR_INVALID_ARG;   // no free parameter
  if (c.mid_split != 0 && c.precision == FSP_FP32_MIXED) return FSP_ERR_UNSUPPORTED;
  return FSP_OK;
}

int stride_grid(long long blocks, int per_sm) {
  static std::atomic<int> sms[64];   // multiprocessors per device ordinal, 0 until read
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) n = sms[dev].load(std::memory_order_relaxed);
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 1;
    } else if (dev >= 0 && dev < 64) {
      sms[dev].store(n, std::memory_order_relaxed);
    }
  }
  const long long cap = (long long)n * per_sm;
  return (int)(blocks < 1 ? 1 : blocks < cap ? blocks : cap);
}

fsp_status rhs_status(cudaError_t e) {
  if (e == cudaErrorNotSupported) return FSP_ERR_UNSUPPORTED;
  return e == cudaSuccess ? FSP_OK : FSP_ERR_CUDA;
}

}  // namespace fsp

extern "C" {

const char* fsp_status_string(fsp_status s) {
  switch (s) {
    case FSP_OK: return "ok";
    case FSP_ERR_INVALID_ARG: return "invalid argument";
    case FSP_ERR_UNSUPPORTED: return "unsupported configuration";
    case FSP_ERR_CUDA: return "CUDA error";
    case FSP_ERR_NONFINITE: return "non-finite value";
    case FSP_ERR_TIMEOUT: return "device wait timed out";
    case FSP_ERR_NOMEM: return "out of memory";
  }
  return "unknown status";
}

size_t fsp_metrics_elems(const fsp_block* blk) {
  if (!blk || blk->ni < 1 || blk->nj < 1) return 0;
  return 5 * (size_t)(blk->ni + 2 * G) * (size_t)(blk->nj + 2 * G);
}

fsp_status fsp_workspace_size(const fsp_config* cfg, const fsp_block* blk, size_t* bytes) {
  if (fsp_status s = check_cfg(cfg, blk)) return s;
  if (!bytes) return FSP_ERR_INVALID_ARG;
  *bytes = ws_layout(*cfg, *blk).total;
  return FSP_OK;
}

fsp_status fsp_metrics(const fsp_config* cfg, const fsp_block* blk, const double* x,
                       const double* y, double* metrics, void* stream) {
  if (fsp_status s = check_cfg(cfg, blk)) return s;
  if (!device_pointer(x) || !device_pointer(y) || !device_pointer(metrics)) return FSP_ERR_INVALID_ARG;
  return cuda_status(launch_metrics(*cfg, *blk, x, y, metrics, (cudaStream_t)stream));
}

fsp_status fsp_line_lambda(const fsp_config* cfg, const fsp_block* blk, const double* metrics,
                           const void* Q, double* lam_xi, double* lam_eta, void* stream) {
  if (fsp_status s = check_cfg(cfg, blk)) return s;
  if (!device_pointer(metrics) || !device_pointer(Q) || !device_pointer(lam_xi) ||
      !device_pointer(lam_eta))
    return FSP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  FSP_TRY(cudaMemsetAsync(lam_xi, 0, sizeof(double) * blk->nj, st));
  FSP_TRY(cudaMemsetAsync(lam_eta, 0, sizeof(double) * blk->ni, st));
  const Params P = make_params(*cfg, *blk, metrics);
  return cuda_status(launch_lambda(P, cfg->precision, Q, lam_xi, lam_eta, nullptr, st));
}

static fsp_status check_ws(const fsp_config* cfg, const fsp_block* blk, void* ws, size_t ws_bytes) {
  if (!device_pointer(ws)) return FSP_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return FSP_ERR_INVALID_ARG;
  if (ws_bytes < ws_layout(*cfg, *blk).total) return FSP_ERR_INVALID_ARG;
  return FSP_OK;
}

// lambda pass + two sweeps; `mode` and the stage coefficients as in launch_rhs
static fsp_status rhs_eval(const fsp_config& c, const fsp_block& b, const double* metrics,
                           const void* Q, void* out, int mode, const void* Qn, double ca, double cb,
                           double dt, char* ws, cudaStream_t st) {
  const WsLayout L = ws_layout(c, b);
  double* lam = reinterpret_cast<double*>(ws + L.lam);
  const Params P = make_params(c, b, metrics);
  FSP_TRY(cudaMemsetAsync(lam, 0, sizeof(double) * (b.ni + b.nj), st));
  FSP_TRY(launch_lambda(P, c.precision, Q, lam, lam + b.nj, nullptr, st));
  return rhs_status(launch_rhs(c.scheme, c.precision, P, Q, lam, lam + b.nj, ws + L.racc, out, mode, Qn,
                               ca, cb, dt, st));
}

fsp_status fsp_rhs(const fsp_config* cfg, const fsp_block* blk, const double* metrics,
                   const void* Q, void* dQdt, void* ws, size_t ws_bytes, void* stream) {
  if (fsp_status s = check_cfg(cfg, blk)) return s;
  if (!device_pointer(metrics) || !device_pointer(Q) || !device_pointer(dQdt) || Q == dQdt)
    return FSP_ERR_INVALID_ARG;
  if (fsp_status s = check_ws(cfg, blk, ws, ws_bytes)) return s;
  return rhs_eval(*cfg, *blk, metrics, Q, dQdt, 0, nullptr, 0.0, 0.0, 0.0, static_cast<char*>(ws),
                  (cudaStream_t)stream);
}

fsp_status fsp_flux_difference(const fsp_config* cfg, const fsp_block* blk, const double* metrics,
                               const void* Q, const double* lam, int dir, int mode, const void* acc,
                               void* D, void* stream) {
  if (fsp_status s = check_cfg(cfg, blk)) return s;
  if ((dir != 0 && dir != 1) || (mode != 0 && mode != 1)) return FSP_ERR_INVALID_ARG;
  if (!device_pointer(metrics) || !device_pointer(Q) || !device_pointer(lam) || !device_pointer(D) ||
      D == Q || (mode == 1 && (!device_pointer(acc) || acc == D)))
    return FSP_ERR_INVALID_ARG;
  const Params P = make_params(*cfg, *blk, metrics);
  cudaError_t e = launch_flux_difference(cfg->scheme, cfg->precision, P, Q, lam, dir, mode, acc, D,
                                         (cudaStream_t)stream);
  if (e == cudaErrorNotSupported) return FSP_ERR_UNSUPPORTED;
  return cuda_status(e);
}

fsp_status fsp_rk3_step(const fsp_config* cfg, const fsp_block* blk, const double* metrics,
                        void* Q, double dt, void* ws, size_t ws_bytes, void* stream) {
  if (fsp_status s = check_cfg(cfg, blk)) return s;
  if (!device_pointer(metrics) || !device_pointer(Q)) return FSP_ERR_INVALID_ARG;
  if (fsp_status s = check_ws(cfg, blk, ws, ws_bytes)) return s;
  const WsLayout L = ws_layout(*cfg, *blk);
  char* w = static_cast<char*>(ws);
  void* Q1 = w + L.q1;
  void* Q2 = w + L.q2;
  cudaStream_t st = (cudaStream_t)stream;
  // Q1 = Q + dt R(Q); Q2 = 3/4 Q + 1/4 (Q1 + dt R(Q1)); Q = 1/3 Q + 2/3 (Q2 + dt R(Q2))
  if (fsp_status s = rhs_eval(*cfg, *blk, metrics, Q, Q1, 1, Q, 0.0, 1.0, dt, w, st)) return s;
  if (fsp_status s = rhs_eval(*cfg, *blk, metrics, Q1, Q2, 1, Q, 0.75, 0.25, dt, w, st)) return s;
  return rhs_eval(*cfg, *blk, metrics, Q2, Q, 1, Q, 1.0 / 3.0, 2.0 / 3.0, dt, w, st);
}

fsp_status fsp_cfl_dt(const fsp_config* cfg, const fsp_block* blk, const double* metrics,
                      const void* Q, double cfl, double* dt_out, void* ws, size_t ws_bytes,
                      void* stream) {
  if (fsp_status s = check_cfg(cfg, blk)) return s;
  if (!device_pointer(metrics) || !device_pointer(Q) || !device_pointer(dt_out) || !(cfl > 0.0))
    return FSP_ERR_INVALID_ARG;
  if (fsp_status s = check_ws(cfg, blk, ws, ws_bytes)) return s;
  const WsLayout L = ws_layout(*cfg, *blk);
  double* lam = reinterpret_cast<double*>(static_cast<char*>(ws) + L.lam);
  cudaStream_t st = (cudaStream_t)stream;
  FSP_TRY(cudaMemsetAsync(lam, 0, sizeof(double) * (blk->ni + blk->nj + 1), st));
  const Params P = make_params(*cfg, *blk, metrics);
  FSP_TRY(launch_lambda(P, cfg->precision, Q, lam, lam + blk->nj, lam + blk->nj + blk->ni, st));
  return cuda_status(launch_cfl_finish(lam + blk->nj + blk->ni, cfl, dt_out, st));
}

fsp_status fsp_norms(const fsp_block* blk, int precision, const void* A, const void* B,
                     double* out, void* stream) {
  if (!blk || blk->ni < 1 || blk->nj < 1 || blk->ld < blk->ni) return FSP_ERR_INVALID_ARG;
  if (precision < FSP_FP64 || precision > FSP_FP32_MIXED) return FSP_ERR_INVALID_ARG;
  if (!device_pointer(A) || !device_pointer(out) || (B && !device_pointer(B))) return FSP_ERR_INVALID_ARG;
  return cuda_status(launch_norms(*blk, precision, A, B, out, (cudaStream_t)stream));
}

fsp_status fsp_check_state(const fsp_config* cfg, const fsp_block* blk, const void* Q, long long* first_bad,
                           void* stream) {
  if (fsp_status s = check_cfg(cfg, blk)) return s;
  if (!device_pointer(Q) || !device_pointer(first_bad)) return FSP_ERR_INVALID_ARG;
  return cuda_status(launch_check_state(*blk, cfg->precision, cfg->gamma, Q, first_bad, (cudaStream_t)stream));
}

fsp_status fsp_fma_peak(int precision, int blocks, int iters, void* sink, void* stream) {
  if ((precision != FSP_FP64 && precision != FSP_FP32) || blocks < 1 || iters < 1)
    return FSP_ERR_INVALID_ARG;
  if (!device_pointer(sink)) return FSP_ERR_INVALID_ARG;
  return cuda_status(launch_fma_peak(precision, blocks, iters, sink, (cudaStream_t)stream));
}

fsp_status fsp_round_to_float(const double* in, float* out_int, float* out_hw, long long n, void* stream) {
  if (n < 0) return FSP_ERR_INVALID_ARG;
  if (n == 0) return FSP_OK;
  if (!device_pointer(in) || !device_pointer(out_int) || !device_pointer(out_hw)) return FSP_ERR_INVALID_ARG;
  return cuda_status(launch_round_to_float(in, out_int, out_hw, n, (cudaStream_t)stream));
}

fsp_status fsp_reciprocal_check(const double* in, double* out, long long n, void* stream) {
  if (n < 0) return FSP_ERR_INVALID_ARG;
  if (n == 0) return FSP_OK;
  if (!device_pointer(in) || !device_pointer(out)) return FSP_ERR_INVALID_ARG;
  return cuda_status(launch_reciprocal_check(in, out, n, (cudaStream_t)stream));
}

fsp_status fsp_widen_to_double(const float* in, double* out_int, double* out_hw, long long n, void* stream) {
  if (n < 0) return FSP_ERR_INVALID_ARG;
  if (n == 0) return FSP_OK;
  if (!device_pointer(in) || !device_pointer(out_int) || !device_pointer(out_hw)) return FSP_ERR_INVALID_ARG;
  return cuda_status(launch_widen_to_double(in, out_int, out_hw, n, (cudaStream_t)stream));
}

}  // extern "C"
