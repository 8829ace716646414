// Device-side lattice description for the CUDA path (D3Q19 / D3Q27).
//
// Velocities follow the canonical order published in include/lbm.h:
// D3Q27 index i = 9*(cz+1) + 3*(cy+1) + (cx+1); D3Q19 drops the eight corners.
// Weights: D3Q27 is the Cartesian product of the D1Q3 rule with weights 2/3
// (rest) and 1/6 (moving), App. F "Velocity space discretization" and
// Eq. (discrete_equilibrium); D3Q19 uses the textbook weights 1/3, 1/18, 1/36.
// Everything is constexpr so that fully unrolled population loops fold the
// velocity components (0, +-1) and weights into the arithmetic.
#pragma once

namespace lbmk {

constexpr double kTheta = 1.0 / 3.0;  // theta_R = c_l^2, App. F

__host__ __device__ constexpr int d27_index(int q, int i)
{
    // position of population i of lattice q in the D3Q27 enumeration
    if (q == 27) return i;
    int n = 0;
    for (int j = 0; j < 27; ++j) {
        const int cx = j % 3 - 1, cy = (j / 3) % 3 - 1, cz = j / 9 - 1;
        const int s = (cx != 0) + (cy != 0) + (cz != 0);
        if (s == 3) continue;
        if (n == i) return j;
        ++n;
    }
    return -1;
}

__host__ __device__ constexpr int cx_of(int q, int i) { return d27_index(q, i) % 3 - 1; }
__host__ __device__ constexpr int cy_of(int q, int i) { return (d27_index(q, i) / 3) % 3 - 1; }
__host__ __device__ constexpr int cz_of(int q, int i) { return d27_index(q, i) / 9 - 1; }

__host__ __device__ constexpr int opp_of(int q, int i)
{
    for (int j = 0; j < q; ++j)
        if (cx_of(q, j) == -cx_of(q, i) && cy_of(q, j) == -cy_of(q, i) && cz_of(q, j) == -cz_of(q, i)) return j;
    return -1;
}

__host__ __device__ constexpr double w1d(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }

__host__ __device__ constexpr double weight_of(int q, int i)
{
    const int cx = cx_of(q, i), cy = cy_of(q, i), cz = cz_of(q, i);
    if (q == 27) return w1d(cx) * w1d(cy) * w1d(cz);
    const int s = cx * cx + cy * cy + cz * cz;
    return s == 0 ? 1.0 / 3.0 : (s == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

}  // namespace lbmk
