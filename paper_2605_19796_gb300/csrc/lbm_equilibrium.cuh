// Lattice equilibrium (FP64, and FP32 for 32- and 16-bit storage), shared by
// the initialisation and the training-data kernels.
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

// f0 - w in FP32 for 32- and 16-bit storage, in the form the step kernels
// use: g = w (rho (P - 1) + drho), with P - 1 = e_x + Y + e_x Y, Y = e_y + e_z +
// e_y e_z built from the small per-axis terms e_a (D3Q27), or the Hermite terms
// (D3Q19), so that no O(1) quantity is rounded in FP32.
template <int Q>
__device__ __forceinline__ void equilibrium_g32(float drho, float ux, float uy, float uz, float (&geq)[Q])
{
    constexpr float a1 = (float)(1.0 / kTheta), a2 = (float)((1.0 - kTheta) / (2.0 * kTheta * kTheta)),
                    a0 = (float)(-kTheta / (2.0 * kTheta * kTheta));
    const float rho = 1.0f + drho;
    const float ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const float ex[3] = {-a1 * ux + a2 * ux2, a0 * ux2, a1 * ux + a2 * ux2};
    const float ey[3] = {-a1 * uy + a2 * uy2, a0 * uy2, a1 * uy + a2 * uy2};
    const float ez[3] = {-a1 * uz + a2 * uz2, a0 * uz2, a1 * uz + a2 * uz2};
    static_for<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
        constexpr float w = (float)weight_of(Q, i);
        if constexpr (Q == 27) {
            const float Y = ey[cy + 1] + ez[cz + 1] + ey[cy + 1] * ez[cz + 1];
            geq[i] = w * (rho * (ex[cx + 1] + Y + ex[cx + 1] * Y) + drho);
        } else {
            const float cu = cx * ux + cy * uy + cz * uz;
            const float usq = ux2 + uy2 + uz2;
            geq[i] = w * (drho + rho * (a1 * cu + 0.5f * a1 * a1 * cu * cu - 0.5f * a1 * usq));
        }
    });
}

}  // namespace lbmk
