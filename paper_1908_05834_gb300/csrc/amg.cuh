// Declarations of the aggregation multigrid preconditioner (amg.cu).
#pragma once

#include "internal.cuh"

namespace bchar {

bool amg_build(bchar_mesh_t m, Amg &amg);
void amg_apply(bchar_mesh_t m, Amg &amg, const double *res, double *z, const CgState *st, bool fp32);
void amg_release(Amg &amg);
void amg_smooth_once(bchar_mesh_t m, Amg &amg);

}  // namespace bchar
