// batch_fp32.cu -- FP32 instantiations of the batched sweeps (sweep.cuh) in every tile
// shape variant; the mixed FP32/FP64 ones are in batch_mixed.cu.
#include "fsp_internal.h"
#include "sweep.cuh"

namespace fsp {

cudaError_t batch_fp32(int scheme, bool mixed, int mode, const PassTables& xi, int ntx, int vx,
                       const PassTables& eta, int nte, int ve, double ca, double cb, double dt, cudaStream_t st) {
  if (mixed) return batch_mixed(scheme, mode, xi, ntx, vx, eta, nte, ve, ca, cb, dt, st);
  return batch_dispatch<float, float>(scheme, mode, xi, ntx, vx, eta, nte, ve, ca, cb, dt, st);
}

cudaError_t batch_direction_fp32(int scheme, bool mixed, int dir, const PassTables& t, int ntiles, int v,
                                 cudaStream_t st) {
  if (mixed) return batch_direction_mixed(scheme, dir, t, ntiles, v, st);
  return batch_one_direction<float, float>(scheme, dir, t, ntiles, v, st);
}

}  // namespace fsp
