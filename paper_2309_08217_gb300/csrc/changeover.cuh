// changeover.cuh -- the pair radius and the changeover weight of the
// close-encounter levels (Sect. 1), shared by the Bulirsch-Stoer level
// (encounter.cu) and the intermediate levels (levels.cu).
#pragma once

#include "internal.cuh"

namespace genga {
namespace {

// Pair radius r_crit,ij from the a_i, r_crit,i of the step's first kick (the
// kick's rule: Eq. 1 radii or n1 mutual Hill radii).
__device__ __forceinline__ double pair_rcrit(int mode, double n1, double Mstar, double mi, double mj, double ai,
                                             double aj, double rci, double rcj) {
    return (mode == GENGA_RCRIT_EQ1) ? fmax(rci, rcj) : n1 * cbrt((mi + mj) / (3.0 * Mstar)) * 0.5 * (ai + aj);
}

// 1 - K(y) from y = q / (0.9 r_crit) - 1/9, with K the kick's changeover
// weight: 1 for y <= 0, 0 for y >= 1.
__device__ __forceinline__ double keep_weight(double y, int form) {
    if (y <= 0.0) return 1.0;
    if (y >= 1.0) return 0.0;
    if (form == GENGA_K_CHAMBERS) {
        const double y2 = y * y;
        return 1.0 - y2 * rcp_fp64(fma(2.0 * y, y - 1.0, 1.0));  // y^2 / (2y^2 - 2y + 1)
    }
    return 1.0 - y * y * y * (10.0 + y * (6.0 * y - 15.0));
}

}  // namespace
}  // namespace genga
