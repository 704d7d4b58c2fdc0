// Internal interface of the learned pressure stage (unet.cu) for the solver.
#pragma once

#include "../../include/rsv_unet.h"
#include "common.cuh"

namespace rsv {

// corr = s * U(rp / s, standardised lnk) on the network's grid, launched on st (no synchronisation);
// every kernel skips when *gate != 0 (gate may be null).
rsv_status unet_apply_device(rsv_unet *u, cudaStream_t st, const double *rp, const double *lnk, double *corr,
                             const int *gate);
void unet_dims(const rsv_unet *u, int *nx, int *ny, int *nz);
// The network's device error word (synchronises st); 0 when no bounded wait ran out.
int unet_error(rsv_unet *u, cudaStream_t st);

}  // namespace rsv
