// Finite-difference stencil weights and the kernel f, shared by the plan set-up
// and the Bloch k-point path.
#pragma once

#include <cmath>

#include "../../include/kronx.h"

namespace kx {

// Centred weight w_p (unit spacing) of the order-2m second-derivative stencil:
// w_0 = -2 sum_{q=1}^m 1/q^2,  w_p = 2 (-1)^{p+1} (m!)^2 / (p^2 (m-p)! (m+p)!).
// The ratio (m!)^2 / ((m-p)!(m+p)!) is formed as a product to stay exact-ish.
__host__ __device__ inline double fd_weight(int m, int p) {
    if (p == 0) {
        double s = 0.0;
        for (int q = 1; q <= m; ++q) s += 1.0 / ((double)q * q);
        return -2.0 * s;
    }
    double r = 1.0;  // prod_{q=1}^{p} (m - p + q) / (m + q) = m! m! / ((m-p)! (m+p)!)
    for (int q = 1; q <= p; ++q) r *= (double)(m - p + q) / (double)(m + q);
    double sgn = (p % 2 == 1) ? 1.0 : -1.0;
    return 2.0 * sgn * r / ((double)p * p);
}

// f at an eigenvalue lam <= 0 of L (Sec. 3): 4 pi / mu unscreened, and the
// erfc-screened (4 pi / mu)(1 - exp(-mu / (4 w^2))) with f(0) = pi / w^2, mu = -lam.
__host__ __device__ inline double kernel_f_value(int kind, double omega, double lam) {
    double mu = -lam;
    if (kind == KX_UNSCREENED) return 4.0 * M_PI / mu;
    double a = 4.0 * omega * omega;
    return (mu == 0.0) ? M_PI / (omega * omega) : -4.0 * M_PI * expm1(-mu / a) / mu;
}

}  // namespace kx
