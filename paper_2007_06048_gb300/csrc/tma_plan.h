// Launch plans of the TMA step kernel (mmod_step_tma.cu).
#pragma once
#include <cuda.h>

#include "mmod.h"

namespace mmod {

constexpr int kMaxTmaVariants = 12;
// Variant used unless a handle selects another: the fastest measured on the
// 240^3 workload (64x16 tile, 2x2 points per thread, z unroll 4).
constexpr int kTmaDefaultVariant = 2;
// The variant whose step kernels can also write g^n = L u^n + s^n (StepArgs::gout).
constexpr int kTmaGVariant = 2;

struct TmaPlan {
    int variant = 0;                // index into the compiled variants
    int tiles_x = 0, tiles_y = 0;   // x-y tiles covering the plane
    int zchunks = 0;                // z-ranges per tile column
    int zlen = 0;                   // planes per z-range (last one may be shorter)
    int grid = 0;                   // CTAs launched
    int block = 0;                  // threads per CTA
    int smem = 0;                   // dynamic shared memory per CTA, bytes
    int occupancy = 0;              // resident CTAs per SM
    int slots = 0;                  // resident CTAs on the device (SMs x occupancy)
    int claim = 0;                  // > 0: work-claiming launch with units of this many planes
};

struct Geom;
// Units and grid of a work-claiming launch of plan (false: the plan's variant
// has no work-claiming form or claim is off).
bool claim_geom(const TmaPlan &plan, int nz, Geom *g, int *units, int *grid);

int tma_variant_count();
const char *tma_variant_name(int v);

// Encodes the tensor maps of both wavefield buffers and of the coefficient
// volume and fills one plan per compiled variant.  Returns false when the TMA
// kernel cannot serve the grid (the caller then uses the plain kernel).
// Tensor maps of one padded volume buffer as the kernel's u^n (halo box) and
// u^{n-1} (tile box) operand.
bool encode_maps(const mmod_config &cfg, int nxp, const float *buf, CUtensorMap *cur, CUtensorMap *prev);

bool make_tma_plan(const mmod_config &cfg, int nxp, float *const u[2], const float *c, CUtensorMap cur_map[2],
                   CUtensorMap prev_map[2], CUtensorMap *c_map, TmaPlan plans[]);

}  // namespace mmod
