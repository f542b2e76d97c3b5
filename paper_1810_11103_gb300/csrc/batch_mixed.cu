// batch_mixed.cu -- mixed FP32/FP64 instantiations of the batched sweeps (sweep.cuh: state,
// projection and WENO in float; metric products, fluxes, h and the difference in double) in
// every tile shape variant.
#include "fsp_internal.h"
#include "sweep.cuh"

namespace fsp {

cudaError_t batch_mixed(int scheme, int mode, const PassTables& xi, int ntx, int vx, const PassTables& eta,
                        int nte, int ve, double ca, double cb, double dt, cudaStream_t st) {
  return batch_dispatch<float, double>(scheme, mode, xi, ntx, vx, eta, nte, ve, ca, cb, dt, st);
}

cudaError_t batch_direction_mixed(int scheme, int dir, const PassTables& t, int ntiles, int v, cudaStream_t st) {
  return batch_one_direction<float, double>(scheme, dir, t, ntiles, v, st);
}

}  // namespace fsp
