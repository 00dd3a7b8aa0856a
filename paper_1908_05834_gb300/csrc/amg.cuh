// Declarations of the aggregation multigrid preconditioner (amg.cu).
#pragma once

#include "internal.cuh"

namespace bchar {

bool amg_build(bchar_mesh_t m, Amg &amg);
void amg_apply(bchar_mesh_t m, Amg &amg, const double *res, double *z, const CgState *st);
void amg_release(Amg &amg);

}  // namespace bchar
