// Declarations of the aggregation multigrid preconditioner (amg.cu).
#pragma once

#include "internal.cuh"

namespace bchar {

// Builds the hierarchy for the current matrix (the minimisation's weights
// change by orders of magnitude between iterations, so it is built anew each time).
bool amg_build(bchar_mesh_t m, Amg &amg);
// z = M^-1 res (one V-cycle).  With b_ready the caller has already written
// the sign-flipped res into the finest level's right-hand side.  With rp, pa,
// pb the last kernel also writes per-block partial sums of z.res into pa and
// of z.rp into pb (kRedBlocks blocks).
void amg_apply(bchar_mesh_t m, Amg &amg, const double *res, double *z, const CgState *st, bool b_ready = false,
               const double *rp = nullptr, double *pa = nullptr, double *pb = nullptr);
// The finest level's right-hand side.
double *amg_finest_rhs(Amg &amg);
void amg_release(Amg &amg);
void amg_smooth_once(bchar_mesh_t m, Amg &amg);

}  // namespace bchar
