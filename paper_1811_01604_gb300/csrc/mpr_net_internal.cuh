// mpr_net_internal.cuh -- what the context code needs from the warm-start network.
#pragma once

#include <cuda_runtime.h>

#include "../../include/mpr.h"
#include "../../include/mpr_net.h"
#include "mpr_internal.cuh"

// Runs the network on B grids of one shape Hin x Win (z, mask: the first grid, grids
// contiguous; zmin, zmax: B host doubles; d_ents: their B consecutive device entries) and
// writes the gap sites of each grid's lattice in lat0 and, if not null, lat1.
mpr_status mprnet_warmstart(mpr_net* net, const float* z, const uint8_t* mask, int B, int Hin, int Win,
                            const double* zmin, const double* zmax, const mpr::EntryDesc* d_ents, float2* lat0,
                            float2* lat1, cudaStream_t st);
const char* mprnet_error(const mpr_net* net);
