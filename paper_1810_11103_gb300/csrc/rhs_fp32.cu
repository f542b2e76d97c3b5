// rhs_fp32.cu -- FP32 instantiations of the directional sweeps (sweep.cuh): the plain
// FP32 path (everything in float, metrics rounded to float on load) and the mixed path
// (state, projection and WENO in float; metric products, fluxes, h and the difference in
// double, so the free-stream residual stays at FP64 round-off).
#include "fsp_internal.h"
#include "sweep.cuh"

namespace fsp {

template <typename Acc>
static cudaError_t rhs_f32(int scheme, const Params& P, const void* Q, const double* lx, const double* le,
                           void* Racc, void* out, int mode, const void* Qn, double ca, double cb, double dt,
                           cudaStream_t st) {
  auto q = static_cast<const float*>(Q);
  auto r = static_cast<Acc*>(Racc);
  auto o = static_cast<float*>(out);
  auto qn = static_cast<const float*>(Qn);
  switch (scheme) {
    case S31: return rhs_passes<S31, float, Acc>(P, q, lx, le, r, o, mode, qn, ca, cb, dt, st);
    case S32: return rhs_passes<S32, float, Acc>(P, q, lx, le, r, o, mode, qn, ca, cb, dt, st);
    case S51: return rhs_passes<S51, float, Acc>(P, q, lx, le, r, o, mode, qn, ca, cb, dt, st);
    case S52: return rhs_passes<S52, float, Acc>(P, q, lx, le, r, o, mode, qn, ca, cb, dt, st);
    case S74:   // one precision only (the mixed regrouping of h is not built for four midpoints)
      if constexpr (std::is_same<Acc, float>::value)
        return rhs_passes<S74, float, Acc>(P, q, lx, le, r, o, mode, qn, ca, cb, dt, st);
      return cudaErrorNotSupported;
    default:  return rhs_passes<S71, float, Acc>(P, q, lx, le, r, o, mode, qn, ca, cb, dt, st);
  }
}

cudaError_t rhs_fp32(int scheme, bool mixed, const Params& P, const void* Q, const double* lx,
                     const double* le, void* Racc, void* out, int mode, const void* Qn, double ca,
                     double cb, double dt, cudaStream_t st) {
  return mixed ? rhs_f32<double>(scheme, P, Q, lx, le, Racc, out, mode, Qn, ca, cb, dt, st)
               : rhs_f32<float>(scheme, P, Q, lx, le, Racc, out, mode, Qn, ca, cb, dt, st);
}

template <typename Acc>
static cudaError_t fd_f32(int scheme, const Params& P, const void* Q, const double* lam, int dir, int mode,
                          const void* acc, void* out, cudaStream_t st) {
  auto q = static_cast<const float*>(Q);
  auto a = static_cast<const Acc*>(acc);
  switch (scheme) {
    case S31: return flux_difference_passes<S31, float, Acc>(P, q, lam, dir, mode, a, out, st);
    case S32: return flux_difference_passes<S32, float, Acc>(P, q, lam, dir, mode, a, out, st);
    case S51: return flux_difference_passes<S51, float, Acc>(P, q, lam, dir, mode, a, out, st);
    case S52: return flux_difference_passes<S52, float, Acc>(P, q, lam, dir, mode, a, out, st);
    case S74:
      if constexpr (std::is_same<Acc, float>::value)
        return flux_difference_passes<S74, float, Acc>(P, q, lam, dir, mode, a, out, st);
      return cudaErrorNotSupported;
    default:  return flux_difference_passes<S71, float, Acc>(P, q, lam, dir, mode, a, out, st);
  }
}

cudaError_t flux_difference_fp32(int scheme, bool mixed, const Params& P, const void* Q, const double* lam,
                                 int dir, int mode, const void* acc, void* out, cudaStream_t st) {
  return mixed ? fd_f32<double>(scheme, P, Q, lam, dir, mode, acc, out, st)
               : fd_f32<float>(scheme, P, Q, lam, dir, mode, acc, out, st);
}

}  // namespace fsp
