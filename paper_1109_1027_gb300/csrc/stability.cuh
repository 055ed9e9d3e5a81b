// stability.cuh -- the time-step bound of Eq. (kdfull) from the reduced
// extremes of L_i = (h^2/a)(s|Psi_i|^2 - V_i) and of the boundary term |B_b|
// (Table t:bc2), for host code (nlse_invariants, nlse_invariants_noalloc)
// and for the device-side entry check of nlse_run alike.
#pragma once

#include <cmath>

namespace nlse {

// Extreme entries of the sets G of the Table of Sec. 3.3 (t:sumresults), in
// units of 1/12: {64, -4} in 1D, {128, -8} in 2D, {192, -12} in 3D.  |L - g|
// is convex in L, so the maximum over G and over all points is reached at an
// extreme of G and an extreme of L.
__host__ __device__ inline void g_extremes(int dim, double* gmin, double* gmax) {
    *gmin = -4.0 * dim / 12.0;
    *gmax = 64.0 * dim / 12.0;
}

// dt_max = sqrt(8) h^2 / (a max{ |B|_inf, max_{i, g} |L_i - g| }) (Eq. kdfull)
// from lmin = min_i L_i, lmax = max_i L_i and bmax = max_b |B_b|.
__host__ __device__ inline double dt_bound(int dim, double h, double a, double lmin, double lmax, double bmax) {
    double gmin, gmax;
    g_extremes(dim, &gmin, &gmax);
    double worst = fmax(fabs(lmax - gmin), fabs(lmin - gmax));
    worst = fmax(worst, fmax(fabs(lmin - gmin), fabs(lmax - gmax)));
    worst = fmax(worst, bmax);
    return sqrt(8.0) * h * h / (a * worst);
}

}  // namespace nlse
