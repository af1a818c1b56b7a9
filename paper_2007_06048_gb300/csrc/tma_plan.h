// Tile plan and tensor maps of the TMA step kernel (mmod_step_tma.cu).
#pragma once
#include <cuda.h>

#include "mmod.h"

namespace mmod {

struct TmaPlan {
    int tiles_x = 0, tiles_y = 0;   // x-y tiles covering the plane
    int zchunks = 0;                // z-ranges per tile column
    int zlen = 0;                   // planes per z-range (last one may be shorter)
    int grid = 0;                   // CTAs launched
    int smem = 0;                   // dynamic shared memory per CTA, bytes
    bool rotate = false;            // z queue rotated by unrolling (true) or shifted
};

// Chooses the decomposition for this grid and encodes the tensor maps of both
// wavefield buffers and of the coefficient volume.  Returns false when the
// TMA kernel cannot serve the grid (the caller then uses the plain kernel).
bool make_tma_plan(const mmod_config &cfg, int nxp, float *const u[2], const float *c,
                   CUtensorMap cur_map[2], CUtensorMap prev_map[2], CUtensorMap *c_map, TmaPlan *plan);

}  // namespace mmod
