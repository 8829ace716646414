// FP64 lattice equilibrium, shared by the initialisation and the training-data
// kernels.
#pragma once

#include "lbm_lattice.cuh"
#include "lbm_step.cuh"

namespace lbmk {

// f0 - w in FP64 from Eq. (discrete_equilibrium) (D3Q27) or the second-order
// Hermite form (D3Q19)
template <int Q>
__device__ __forceinline__ void equilibrium_g(double rho, double ux, double uy, double uz, double (&geq)[Q])
{
    const double a1 = 1.0 / kTheta, a2 = (1.0 - kTheta) / (2.0 * kTheta * kTheta), a0 = -kTheta / (2.0 * kTheta * kTheta);
    static_for<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
        constexpr double w = weight_of(Q, i);
        if constexpr (Q == 27) {
            const double px = cx == 0 ? 1.0 + a0 * ux * ux : 1.0 + cx * a1 * ux + a2 * ux * ux;
            const double py = cy == 0 ? 1.0 + a0 * uy * uy : 1.0 + cy * a1 * uy + a2 * uy * uy;
            const double pz = cz == 0 ? 1.0 + a0 * uz * uz : 1.0 + cz * a1 * uz + a2 * uz * uz;
            geq[i] = w * (rho * px * py * pz - 1.0);
        } else {
            const double cu = cx * ux + cy * uy + cz * uz;
            const double usq = ux * ux + uy * uy + uz * uz;
            geq[i] = w * ((rho - 1.0) + rho * (a1 * cu + 0.5 * a1 * a1 * cu * cu - 0.5 * a1 * usq));
        }
    });
}

}  // namespace lbmk
