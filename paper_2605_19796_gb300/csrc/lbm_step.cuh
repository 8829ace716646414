// Fused stream-and-collide step of the kinetic-closure LES solver (sm_103a).
//
// One launch advances every cell of every box by one time step:
//   pull streaming (Eq. streaming, periodic or halfway bounce-back in y)
//   -> rho, u from the streamed populations (App. F.1 step 1)
//   -> equilibrium (Eq. discrete_equilibrium; D3Q19: second-order Hermite)
//   -> strain rate from the neighbours' velocities (Eqs. fd, strain_rate_discrete,
//      one-sided Eqs. fd_boundary_lower/upper at walls)
//   -> closure carrier and SGS trace (KC-MP App. F.3, KC-RB App. F.2)
//   -> clipped turbulent rate (Eq. omega_sgs_operational)
//   -> two-rate relaxation (Eq. kcmp_operational_collision / kcrb_operational_collision)
//   -> store of the post-collision populations.
//
// Data layout: structure of arrays [box][q][z][y][x], x fastest.  Ping-pong
// buffers: the kernel reads buffer A and writes buffer B.
//
// Parallel decomposition: a CTA owns a 32 x TY column of cells and marches it
// through a chunk of z-planes.  The strain rate needs the velocity of the
// x, y and z neighbours at the SAME (post-streaming) time level, so the CTA
// keeps a ring of four velocity planes in shared memory covering its tile plus
// a one-cell (two-cell along a wall axis) halo.  At plane k it pulls plane k+1
// (its own cells and the halo cells), publishes their velocities to the ring,
// synchronises once, and collides plane k with the populations pulled in the
// previous iteration (held in registers).  Four ring slots make a single
// barrier per plane sufficient.
//
// Arithmetic runs on the weight-shifted populations g_i = f_i - w_i, which
// keeps the moment sums free of the O(1) cancellation (sum w_i = 1,
// sum w_i c_i c_i = theta I are exact); the relaxation is affine so the shift
// cancels in every difference.  FP16/BF16 storage holds g_i directly.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <utility>

#include "lbm_internal.h"
#include "lbm_lattice.cuh"
#include "lbm_mlp_infer.cuh"

namespace lbmk {

// ---------------------------------------------------------------- utilities

template <typename F, int... Is>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Is...>)
{
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f)
{
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

template <typename S>
struct StoreTraits;
template <>
struct StoreTraits<double> {
    using R = double;
    static constexpr bool shifted = false;
};
template <>
struct StoreTraits<float> {
    using R = float;
    static constexpr bool shifted = false;
};
template <>
struct StoreTraits<__half> {
    using R = float;
    static constexpr bool shifted = true;
};
template <>
struct StoreTraits<__nv_bfloat16> {
    using R = float;
    static constexpr bool shifted = true;
};

// returns g = f - w
template <typename S, typename R>
__device__ __forceinline__ R load_g(const S* p, R w);
template <>
__device__ __forceinline__ double load_g<double, double>(const double* p, double w)
{
    return __ldg(p) - w;
}
template <>
__device__ __forceinline__ float load_g<float, float>(const float* p, float w)
{
    return __ldg(p) - w;
}
template <>
__device__ __forceinline__ float load_g<__half, float>(const __half* p, float)
{
    return __half2float(__ldg(p));
}
template <>
__device__ __forceinline__ float load_g<__nv_bfloat16, float>(const __nv_bfloat16* p, float)
{
    return __bfloat162float(__ldg(p));
}

template <typename S, typename R>
__device__ __forceinline__ void store_g(S* p, R g, R w);
template <>
__device__ __forceinline__ void store_g<double, double>(double* p, double g, double w)
{
    *p = g + w;
}
template <>
__device__ __forceinline__ void store_g<float, float>(float* p, float g, float w)
{
    *p = g + w;
}
template <>
__device__ __forceinline__ void store_g<__half, float>(__half* p, float g, float)
{
    *p = __float2half_rn(g);
}
template <>
__device__ __forceinline__ void store_g<__nv_bfloat16, float>(__nv_bfloat16* p, float g, float)
{
    *p = __float2bfloat16_rn(g);
}

__device__ __forceinline__ int wrapi(int a, int n)
{
    a %= n;
    return a < 0 ? a + n : a;
}

// A column of cells (fixed x, y) that the CTA pulls plane after plane.
// xs: x-1, x, x+1 (periodic); yr: row offsets of y-1, y, y+1, or -1 where the
// row lies beyond a wall.
struct Col {
    int xs[3];
    int yr[3];
    bool valid;
};

template <int BC>
__device__ __forceinline__ Col make_col(int gx, int gy, int nx, int ny)
{
    Col c;
    gx = wrapi(gx, nx);
    c.xs[0] = gx == 0 ? nx - 1 : gx - 1;
    c.xs[1] = gx;
    c.xs[2] = gx == nx - 1 ? 0 : gx + 1;
    if (BC == BC_WALLS_Y) {
        c.valid = gy >= 0 && gy < ny;
        const int y = c.valid ? gy : 0;
        c.yr[0] = y > 0 ? (y - 1) * nx : -1;
        c.yr[1] = y * nx;
        c.yr[2] = y < ny - 1 ? (y + 1) * nx : -1;
    } else {
        c.valid = true;
        const int y = wrapi(gy, ny);
        c.yr[0] = (y == 0 ? ny - 1 : y - 1) * nx;
        c.yr[1] = y * nx;
        c.yr[2] = (y == ny - 1 ? 0 : y + 1) * nx;
    }
    return c;
}

// Pull the Q streamed populations of cell (col, plane zr[1]) as g = f - w:
// g_i(x) = g_post_i(x - c_i); beyond a y wall, halfway bounce-back
// g_i(x) = g_post_opp(i)(x).  Cell offsets are 32-bit (a box holds fewer
// than 2^31 cells); the population offset i*ps is 64-bit.
template <int Q, typename S, typename R, int BC>
__device__ __forceinline__ void pull(const S* __restrict__ fin, long long ps, const Col& col, const int (&zr)[3],
                                     R (&g)[Q])
{
    static_for<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
        constexpr int io = opp_of(Q, i);
        const R w = (R)weight_of(Q, i);
        if (BC == BC_WALLS_Y && cy != 0) {
            const int row = col.yr[1 - cy];
            const S* src = row >= 0 ? fin + (long long)i * ps + (zr[1 - cz] + row + col.xs[1 - cx])
                                    : fin + (long long)io * ps + (zr[1] + col.yr[1] + col.xs[1]);
            g[i] = load_g<S, R>(src, w);
        } else {
            g[i] = load_g<S, R>(fin + (long long)i * ps + (zr[1 - cz] + col.yr[1 - cy] + col.xs[1 - cx]), w);
        }
    });
}

// drho = sum g (rho = 1 + drho), j = sum g c (sum w c = 0), u = (j + F/2)/rho.
// drho is returned unrounded: the equilibrium uses it directly so that
// sum_i g_eq,i = drho holds to rounding of small quantities (no O(1) term).
// D3Q27 sums over the x-triples: populations i = 3t, 3t+1, 3t+2 share
// (c_y, c_z) with t = 3(c_z + 1) + (c_y + 1) and have c_x = -1, 0, +1;
// s_t = their sum, dx_t = g(+1) - g(-1).
template <typename R>
__device__ __forceinline__ void triples27(const R (&g)[27], R (&s)[9], R (&dx)[9])
{
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        s[t] = (g[3 * t] + g[3 * t + 1]) + g[3 * t + 2];
        dx[t] = g[3 * t + 2] - g[3 * t];
    }
}

template <int Q, typename R>
__device__ __forceinline__ void moments(const R (&g)[Q], R& drho, R& ux, R& uy, R& uz, R Fx, R Fy, R Fz)
{
    R d = 0, jx = 0, jy = 0, jz = 0;
    if constexpr (Q == 27) {
        R s[9], dx[9];
        triples27<R>(g, s, dx);
        const R sym = (s[0] + s[3]) + s[6], sy0 = (s[1] + s[4]) + s[7], syp = (s[2] + s[5]) + s[8];
        const R szm = (s[0] + s[1]) + s[2], szp = (s[6] + s[7]) + s[8];
        d = (sym + sy0) + syp;
        jy = syp - sym;
        jz = szp - szm;
        jx = (((dx[0] + dx[1]) + (dx[2] + dx[3])) + ((dx[4] + dx[5]) + (dx[6] + dx[7]))) + dx[8];
    } else {
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
            d += g[i];
            if (cx == 1) jx += g[i];
            if (cx == -1) jx -= g[i];
            if (cy == 1) jy += g[i];
            if (cy == -1) jy -= g[i];
            if (cz == 1) jz += g[i];
            if (cz == -1) jz -= g[i];
        });
    }
    drho = d;
    const R inv = R(1) / (R(1) + d);
    ux = (jx + R(0.5) * Fx) * inv;
    uy = (jy + R(0.5) * Fy) * inv;
    uz = (jz + R(0.5) * Fz) * inv;
}

// Eq. (omega_sgs_operational): k = |tr m_sgs|/(2 rho_0), rho_0 = 1;
// omega_s = (nu_t/theta + 1/2)^-1 if nu_t = C_nu Delta sqrt(k) > nu, else omega.
template <typename R>
__device__ __forceinline__ R omega_sgs(R tr, R nu, R omega, R cnud)
{
    const R nut = cnud * sqrt(R(0.5) * fabs(tr));
    return nut > nu ? R(1) / (nut * R(1.0 / kTheta) + R(0.5)) : omega;
}

// KC-RR (App. F.4): the 17 high-order D3Q27 Hermite modes of B_high as
// directional degrees (d_x, d_y, d_z), and the recursive-regularised reference
// coefficients of Eq. (kcrr_rr) seeded by a_rr_ab = m_CE_ab:
//   a_rr(a1..ak) = u_ak a_rr(a1..a(k-1)) + sum_{i<k} (prod_{j<k, j != i} u_aj) a_rr(ai ak)
// (isothermal equilibrium coefficients a0(a1..am) = rho u_a1..u_am, divided by
// rho), evaluated over the prefixes of the mode's axis list in ascending order.
__host__ __device__ constexpr int rr_deg(int m, int a)
{
    constexpr int t[17][3] = {{2, 1, 0}, {2, 0, 1}, {0, 2, 1}, {1, 2, 0}, {1, 0, 2}, {0, 1, 2}, {1, 1, 1}, {2, 2, 0}, {2, 0, 2},
                              {0, 2, 2}, {2, 1, 1}, {1, 2, 1}, {1, 1, 2}, {2, 2, 1}, {2, 1, 2}, {1, 2, 2}, {2, 2, 2}};
    return t[m][a];
}
__host__ __device__ constexpr int rr_n(int m) { return rr_deg(m, 0) + rr_deg(m, 1) + rr_deg(m, 2); }
__host__ __device__ constexpr int rr_axis(int m, int k)  // k-th axis of mode m in ascending order
{
    return k < rr_deg(m, 0) ? 0 : (k < rr_deg(m, 0) + rr_deg(m, 1) ? 1 : 2);
}

template <typename R, int M>
__device__ __forceinline__ R rr_coef(const R (&u)[3], const R (&A)[3][3])
{
    constexpr int n = rr_n(M);
    R a = A[rr_axis(M, 0)][rr_axis(M, 1)];
#pragma unroll
    for (int k = 2; k < n; ++k) {
        const int ak = rr_axis(M, k);
        R nxt = u[ak] * a;
#pragma unroll
        for (int i = 0; i < k; ++i) {
            R prod = R(1);
#pragma unroll
            for (int j = 0; j < k; ++j)
                if (j != i) prod *= u[rr_axis(M, j)];
            nxt += prod * A[rr_axis(M, i)][ak];
        }
        a = nxt;
    }
    return a;
}

// One axis of the separable D3Q27 Hermite transform, in place on the 9 lines
// of stride ST (1: x, 3: y, 9: z) of a [z][y][x] block of 27 values.
// Forward: (v(-1), v(0), v(+1)) -> (sum v, sum v c, sum v (c^2 - theta)).
// Inverse: raw coefficients (K0, K1, K2) -> sum_d K_d N_d H_d(c) at c = -1, 0, +1
// with H = (1, c, c^2 - theta) and N = (1, 1/theta, 1/(2 theta^2)) = (1, 3, 9/2),
// i.e. K0 - 3/2 K2 at c = 0 and K0 + 3 K2 -+ 3 K1 at c = -+1.
template <typename R, int ST, bool INV>
__device__ __forceinline__ void herm_axis(R (&v)[27])
{
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        const int o = ST == 1 ? 3 * l : (ST == 3 ? 9 * (l / 3) + l % 3 : l);
        R& a = v[o];
        R& b = v[o + ST];
        R& c = v[o + 2 * ST];
        if constexpr (!INV) {
            const R p = a + c;
            const R s0 = p + b;
            const R s1 = c - a;
            c = p - R(kTheta) * s0;
            a = s0;
            b = s1;
        } else {
            const R t = a - R(1.5) * c;
            const R p = t + R(4.5) * c;
            const R k1 = R(3) * b;
            a = p - k1;
            c = p + k1;
            b = t;
        }
    }
}

// KC-RR collision of one D3Q27 cell on shifted populations (in place), in
// Hermite moment space.  D3Q27 is the tensor product of three 3-point lattices
// and its 27 Hermite polynomials are products of per-axis factors (1, c,
// c^2 - theta), so the projection onto all 27 modes and the reconstruction
// f = w sum_d K_d N_d H_d are three 1D passes each.  The product equilibrium
// has the coefficients E_d = rho ux^dx uy^dy uz^dz, so f_neq's coefficients
// are M_d - E_d (the shifted populations g = f - w have f's coefficients
// except d = 0, since sum_i w_i H_d = 0 for d != 0).  Relaxation as App. F.4:
// second order (1 - omega) m_CE + (1 - omega_s)(m_neq - m_CE), the 17
// high-order modes (1 - omega) a_rr + (1 - omega_s)(a_neq - a_rr), orders 0
// and 1 kept (rho - 1, rho u).
template <typename R>
__device__ __forceinline__ void collide_kcrr(R (&g)[27], R drho, R ux, R uy, R uz, R Sxx, R Syy, R Szz, R Sxy, R Sxz,
                                             R Syz, R omega, R tau_hat, R nu, R cnud)
{
    constexpr int Q = 27;
    const R rho = R(1) + drho;
    herm_axis<R, 1, false>(g);
    herm_axis<R, 3, false>(g);
    herm_axis<R, 9, false>(g);  // g[9 dz + 3 dy + dx] = M_d
    const R rx[3] = {rho, rho * ux, rho * (ux * ux)};
    const R py[3] = {R(1), uy, uy * uy};
    const R pz[3] = {R(1), uz, uz * uz};
    R E[27];
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const R yz = dy == 0 ? pz[dz] : (dz == 0 ? py[dy] : py[dy] * pz[dz]);
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) E[9 * dz + 3 * dy + dx] = (dy == 0 && dz == 0) ? rx[dx] : rx[dx] * yz;
        }
    // second order: m_neq, m_CE = -2 rho theta tau_hat S, rate from tr(m_neq - m_CE)
    constexpr int i2[3][3] = {{2, 4, 10}, {4, 6, 12}, {10, 12, 18}};
    const R Sm[3][3] = {{Sxx, Sxy, Sxz}, {Sxy, Syy, Syz}, {Sxz, Syz, Szz}};
    const R rt = R(-2) * rho * R(kTheta) * tau_hat;
    R A[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) A[a][b] = rt * Sm[a][b];
    R tr = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) tr += (g[i2[a][a]] - E[i2[a][a]]) - A[a][a];
    const R omega_s = omega_sgs(tr, nu, omega, cnud);
    const R om1 = R(1) - omega, os1 = R(1) - omega_s;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a; b < 3; ++b) {
            const int d = i2[a][b];
            g[d] = E[d] + om1 * A[a][b] + os1 * ((g[d] - E[d]) - A[a][b]);
        }
    // high order: recursive-regularised reference from m_CE, two-rate relaxation
    const R uu[3] = {ux, uy, uz};
    static_for<17>([&](auto MI) {
        constexpr int m = decltype(MI)::value;
        constexpr int d = 9 * rr_deg(m, 2) + 3 * rr_deg(m, 1) + rr_deg(m, 0);
        const R ar = rr_coef<R, m>(uu, A);
        g[d] = E[d] + om1 * ar + os1 * ((g[d] - E[d]) - ar);
    });
    g[0] = drho;
    g[1] = E[1];
    g[3] = E[3];
    g[9] = E[9];
    herm_axis<R, 9, true>(g);
    herm_axis<R, 3, true>(g);
    herm_axis<R, 1, true>(g);
    static_for<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        g[i] *= R(weight_of(Q, i));
    });
}

// One-cell collision on shifted populations g (in place -> g_post).
//
// Every closure is evaluated in the common form
//     g_post_i = a g_i + w_i (b (P_i - 1) + c0 + D H_i)
// where f0_i - w_i = w_i (rho (P_i - 1) + drho) is the shifted equilibrium and
// H_i = sum_ab c_ia c_ib M_ab - t is a quadratic form in c_i:
//   BGK:   a = 1 - omega,   b = omega rho,   c0 = omega drho,   D = 0
//   KC-MP: a = 1 - omega,   b, c0 as BGK,    D = (omega - omega_s)/(2 theta^2),
//          M = m_sgs, t = theta tr m_sgs          (f_sgs = w H / (2 theta^2))
//   KC-RB: a = 1 - omega_s, b = omega_s rho, c0 = omega_s drho,
//          D = (omega_s - omega)(-rho tau_hat/theta), M = S,
//          t = theta tr S (Hermite) or 0 (raw)    (f1 = w (-rho tau_hat/theta) H)
// which is f - omega (f - f0 - f_sgs) - omega_s f_sgs (KC-MP, App. F.3) and
// f - omega f1 - omega_s (f - f0 - f1) (KC-RB, App. F.2) rearranged.  For D3Q27
// P - 1 = e_x + Y + e_x Y, Y = e_y + e_z + e_y e_z (the product equilibrium in
// its small per-axis terms, so FP32 rounds without bias); Y and the parts of H
// depend only on (c_y, c_z) and are formed once per pair.
// Second moments Pi'_ab = sum_i g_i c_ia c_ib = Pi_ab - theta delta_ab of the
// shifted populations (xx yy zz xy xz yz); drho = sum g.
template <int Q, typename R>
__device__ __forceinline__ void second_moments(const R (&g)[Q], R drho, R (&P)[6])
{
    R pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
    if constexpr (Q == 27) {
        // from the x-triple sums (triples27): c_x^2 = 1 except the middle
        // member, c_x c_y and c_x c_z from dx, c_y c_z from s
        R s[9], dx[9];
        triples27<R>(g, s, dx);
        const R g0 = (((g[1] + g[4]) + (g[7] + g[10])) + ((g[13] + g[16]) + (g[19] + g[22]))) + g[25];
        pxx = drho - g0;
        pyy = ((s[0] + s[3]) + s[6]) + ((s[2] + s[5]) + s[8]);
        pzz = ((s[0] + s[1]) + s[2]) + ((s[6] + s[7]) + s[8]);
        pxy = ((dx[2] + dx[5]) + dx[8]) - ((dx[0] + dx[3]) + dx[6]);
        pxz = ((dx[6] + dx[7]) + dx[8]) - ((dx[0] + dx[1]) + dx[2]);
        pyz = (s[0] + s[8]) - (s[2] + s[6]);
    } else {
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
            if (cx != 0) pxx += g[i];
            if (cy != 0) pyy += g[i];
            if (cz != 0) pzz += g[i];
            if (cx * cy == 1) pxy += g[i];
            if (cx * cy == -1) pxy -= g[i];
            if (cx * cz == 1) pxz += g[i];
            if (cx * cz == -1) pxz -= g[i];
            if (cy * cz == 1) pyz += g[i];
            if (cy * cz == -1) pyz -= g[i];
        });
    }
    P[0] = pxx;
    P[1] = pyy;
    P[2] = pzz;
    P[3] = pxy;
    P[4] = pxz;
    P[5] = pyz;
}

// Relaxation coefficients of the common collision form (see collide below).
template <typename R>
struct Coef {
    R ca, cb, c0, D, t, Mxx, Myy, Mzz, Mxy, Mxz, Myz;
};

// The per-cell part of the collision: closure carrier, SGS trace, rate (Eq.
// omega_sgs_operational) and the coefficients; P holds the second moments
// (unused for BGK and the learned closure, which takes msgs_in).
template <int Q, typename R, int CL>
__device__ __forceinline__ Coef<R> collide_coef(const R (&P)[6], R drho, R ux, R uy, R uz, R Sxx, R Syy, R Szz,
                                                R Sxy, R Sxz, R Syz, R omega, R tau_hat, R nu, R cnud,
                                                const R* msgs_in = nullptr)
{
    constexpr R th = R(kTheta);
    const R rho = R(1) + drho;
    Coef<R> k;
    k.Mxx = k.Myy = k.Mzz = k.Mxy = k.Mxz = k.Myz = k.t = R(0);
    k.ca = R(1) - omega;
    k.cb = omega * rho;
    k.c0 = omega * drho;
    k.D = R(0);
    if constexpr (CL == CL_LEARNED) {
        // learned closure: the network's m_sgs replaces m_neq - m_CE; the rate and
        // the relaxation are KC-MP's (App. F.3 with the learned SGS moment)
        k.Mxx = msgs_in[0];
        k.Myy = msgs_in[1];
        k.Mzz = msgs_in[2];
        k.Mxy = msgs_in[3];
        k.Mxz = msgs_in[4];
        k.Myz = msgs_in[5];
        const R tr = k.Mxx + k.Myy + k.Mzz;
        const R omega_s = omega_sgs(tr, nu, omega, cnud);
        k.t = th * tr;
        k.D = (omega - omega_s) * R(1.0 / (2.0 * kTheta * kTheta));
    } else if constexpr (CL == CL_KCMP) {
        // m_neq = Pi - rho(uu + theta I) = Pi' - rho uu - theta drho I   (App. F.3)
        // m_CE = -2 rho theta tau_hat S;  m_sgs = m_neq - m_CE
        const R rt = R(-2) * rho * th * tau_hat;
        k.Mxx = P[0] - rho * (ux * ux) - th * drho - rt * Sxx;
        k.Myy = P[1] - rho * (uy * uy) - th * drho - rt * Syy;
        k.Mzz = P[2] - rho * (uz * uz) - th * drho - rt * Szz;
        k.Mxy = P[3] - rho * ux * uy - rt * Sxy;
        k.Mxz = P[4] - rho * ux * uz - rt * Sxz;
        k.Myz = P[5] - rho * uy * uz - rt * Syz;
        const R tr = k.Mxx + k.Myy + k.Mzz;
        const R omega_s = omega_sgs(tr, nu, omega, cnud);
        k.t = th * tr;
        k.D = (omega - omega_s) * R(1.0 / (2.0 * kTheta * kTheta));
    } else if constexpr (CL == CL_KCRB_H || CL == CL_KCRB_RAW) {
        // KC-RB, Hermite or raw first-order reconstruction (App. F.2)
        constexpr bool herm = (CL == CL_KCRB_H);
        const R usq = ux * ux + uy * uy + uz * uz;
        const R trS = Sxx + Syy + Szz;
        // sum_i f1_i |c_i|^2 = -2 rho tau_hat theta trS (Hermite), -5 rho tau_hat theta trS (raw)
        const R trf1 = R(herm ? -2 : -5) * rho * tau_hat * th * trS;
        // tr m_sgs = sum (f - f0 - f1)|c|^2 = tr Pi' - rho |u|^2 - 3 theta drho - tr f1
        const R tr = (P[0] + P[1] + P[2]) - rho * usq - R(3) * th * drho - trf1;
        const R omega_s = omega_sgs(tr, nu, omega, cnud);
        k.Mxx = Sxx;
        k.Myy = Syy;
        k.Mzz = Szz;
        k.Mxy = Sxy;
        k.Mxz = Sxz;
        k.Myz = Syz;
        k.t = herm ? th * trS : R(0);
        k.ca = R(1) - omega_s;
        k.cb = omega_s * rho;
        k.c0 = omega_s * drho;
        k.D = (omega_s - omega) * (-rho * tau_hat * R(1.0 / kTheta));
    }
    return k;
}

// The per-population part of the collision for the populations [LO, HI) of
// one cell (g holds them at 0 .. HI-LO-1), plus the Guo source with a force.
template <int Q, typename R, int CL, bool FORCE, int LO, int HI, int N>
__device__ __forceinline__ void relax(R (&g)[N], const Coef<R>& k, R ux, R uy, R uz, R omega, R Fx, R Fy, R Fz)
{
    static_assert(N >= HI - LO, "populations array too short");
    constexpr R a1 = R(1.0 / kTheta);                                // c u / theta
    constexpr R a2 = R((1.0 - kTheta) / (2.0 * kTheta * kTheta));    // (1 - theta) u^2 / (2 theta^2)
    constexpr R a0 = R(-kTheta / (2.0 * kTheta * kTheta));           // -theta u^2 / (2 theta^2)
    const R ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const R usq = ux2 + uy2 + uz2;
    const R ca = k.ca, cb = k.cb, c0 = k.c0, D = k.D, t = k.t;
    const R Mxx = k.Mxx, Myy = k.Myy, Mzz = k.Mzz, Mxy = k.Mxy, Mxz = k.Mxz, Myz = k.Myz;
    if constexpr (Q == 27) {
        // per-axis equilibrium terms e(c) and the (c_y, c_z) parts
        const R ex[3] = {-a1 * ux + a2 * ux2, a0 * ux2, a1 * ux + a2 * ux2};
        const R ey[3] = {-a1 * uy + a2 * uy2, a0 * uy2, a1 * uy + a2 * uy2};
        const R ez[3] = {-a1 * uz + a2 * uz2, a0 * uz2, a1 * uz + a2 * uz2};
        static_for<HI - LO>([&](auto I) {
            constexpr int i = LO + decltype(I)::value;
            constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
            constexpr R w = R(weight_of(Q, i));
            const R Y = ey[cy + 1] + ez[cz + 1] + ey[cy + 1] * ez[cz + 1];
            const R pm1 = ex[cx + 1] + Y + ex[cx + 1] * Y;
            R K = cb * pm1 + c0;
            if constexpr (CL != CL_BGK) {
                R h = -t;
                if (cy != 0) h += Myy;
                if (cz != 0) h += Mzz;
                if (cy * cz != 0) h += R(2 * cy * cz) * Myz;
                if (cx != 0) h += Mxx + R(2 * cx) * (R(cy) * Mxy + R(cz) * Mxz);
                K += D * h;
            }
            g[i - LO] = ca * g[i - LO] + w * K;
        });
    } else {
        static_for<HI - LO>([&](auto I) {
            constexpr int i = LO + decltype(I)::value;
            constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
            constexpr R w = R(weight_of(Q, i));
            const R cu = R(cx) * ux + R(cy) * uy + R(cz) * uz;
            // D3Q19 second-order Hermite equilibrium: P - 1 = c.u/theta + (c.u)^2/(2 theta^2) - u^2/(2 theta)
            const R pm1 = a1 * cu + R(0.5) * a1 * a1 * cu * cu - R(0.5) * a1 * usq;
            R K = cb * pm1 + c0;
            if constexpr (CL != CL_BGK) {
                R h = -t;
                if (cx != 0) h += Mxx;
                if (cy != 0) h += Myy;
                if (cz != 0) h += Mzz;
                if (cx * cy != 0) h += R(2 * cx * cy) * Mxy;
                if (cx * cz != 0) h += R(2 * cx * cz) * Mxz;
                if (cy * cz != 0) h += R(2 * cy * cz) * Myz;
                K += D * h;
            }
            g[i - LO] = ca * g[i - LO] + w * K;
        });
    }
    if constexpr (FORCE) {
        // Guo source (1 - omega/2) w [(c - u)/theta + (c.u) c/theta^2] . F
        const R pref = R(1) - R(0.5) * omega;
        const R uF = ux * Fx + uy * Fy + uz * Fz;
        static_for<HI - LO>([&](auto I) {
            constexpr int i = LO + decltype(I)::value;
            constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
            constexpr R w = R(weight_of(Q, i));
            const R cF = R(cx) * Fx + R(cy) * Fy + R(cz) * Fz;
            const R cu = R(cx) * ux + R(cy) * uy + R(cz) * uz;
            g[i - LO] += pref * w * ((cF - uF) * a1 + cu * cF * (a1 * a1));
        });
    }
}

// One-cell collision on shifted populations g (in place -> g_post).
//
// Every closure is evaluated in the common form
//     g_post_i = a g_i + w_i (b (P_i - 1) + c0 + D H_i)
// where f0_i - w_i = w_i (rho (P_i - 1) + drho) is the shifted equilibrium and
// H_i = sum_ab c_ia c_ib M_ab - t is a quadratic form in c_i:
//   BGK:   a = 1 - omega,   b = omega rho,   c0 = omega drho,   D = 0
//   KC-MP: a = 1 - omega,   b, c0 as BGK,    D = (omega - omega_s)/(2 theta^2),
//          M = m_sgs, t = theta tr m_sgs          (f_sgs = w H / (2 theta^2))
//   KC-RB: a = 1 - omega_s, b = omega_s rho, c0 = omega_s drho,
//          D = (omega_s - omega)(-rho tau_hat/theta), M = S,
//          t = theta tr S (Hermite) or 0 (raw)    (f1 = w (-rho tau_hat/theta) H)
// which is f - omega (f - f0 - f_sgs) - omega_s f_sgs (KC-MP, App. F.3) and
// f - omega f1 - omega_s (f - f0 - f1) (KC-RB, App. F.2) rearranged.  For D3Q27
// P - 1 = e_x + Y + e_x Y, Y = e_y + e_z + e_y e_z (the product equilibrium in
// its small per-axis terms, so FP32 rounds without bias); Y and the parts of H
// depend only on (c_y, c_z) and are formed once per pair.
template <int Q, typename R, int CL, bool FORCE>
__device__ __forceinline__ void collide(R (&g)[Q], R drho, R ux, R uy, R uz, R Sxx, R Syy, R Szz, R Sxy, R Sxz,
                                        R Syz, R omega, R tau_hat, R nu, R cnud, R Fx, R Fy, R Fz,
                                        const R* msgs_in = nullptr)
{
    if constexpr (CL == CL_KCRR) {
        static_assert(Q == 27, "KC-RR is defined on D3Q27 only");
        static_assert(!FORCE, "KC-RR is built for periodic boxes");
        collide_kcrr<R>(g, drho, ux, uy, uz, Sxx, Syy, Szz, Sxy, Sxz, Syz, omega, tau_hat, nu, cnud);
    } else {
        R P[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
        if constexpr (CL != CL_BGK && CL != CL_LEARNED) second_moments<Q, R>(g, drho, P);
        const Coef<R> k = collide_coef<Q, R, CL>(P, drho, ux, uy, uz, Sxx, Syy, Szz, Sxy, Sxz, Syz, omega, tau_hat,
                                                 nu, cnud, msgs_in);
        relax<Q, R, CL, FORCE, 0, Q>(g, k, ux, uy, uz, omega, Fx, Fy, Fz);
    }
}

// ------------------------------------------------------------------ kernel

// Shared-memory footprint of one CTA: the velocity ring (4 planes x 3
// components x ring cells) and a two-slot stash of the own column's streamed
// populations (the next plane is parked there while the current one collides,
// so only one plane of populations is ever live in registers).
template <int Q, typename R, int BC, int TY>
struct StepShape {
    static constexpr int TX = 32;
    static constexpr int HY = (BC == BC_WALLS_Y) ? 2 : 1;  // ring halo rows (two for one-sided wall stencils)
    static constexpr int RX = TX + 2;
    static constexpr int RY = TY + 2 * HY;
    static constexpr int RN = RX * RY;
    static constexpr int NT = TX * TY;
    static constexpr int NB = RN - NT;  // halo cells of the ring plane
    static constexpr size_t base_bytes = sizeof(R) * (size_t)(4 * 3 * RN + 2 * Q * NT);
    static constexpr size_t smem_bytes = base_bytes;
};

// learned closure: network block and per-warp exchange after the ring and stash
template <int Q, typename R, int BC, int TY, int CL>
constexpr size_t step_smem_bytes()
{
    return StepShape<Q, R, BC, TY>::base_bytes +
           (CL == CL_LEARNED ? (size_t)(MlpLayout::BYTES + TY * MlpLayout::XCH_BYTES) : 0);
}

// network inputs of one cell (the learned closure's 10 inputs: (m_neq - m_CE)/rho,
// invariants of m_CE/rho, tau_hat), standardised, into the warp's exchange row;
// network forward for the warp; the cell's m_sgs back (times rho)
// The populations are read from the shared-memory stash (stride NT) rather
// than kept in registers, so that only the network's fragments are live while
// it runs; the caller reloads them for the collision.
// The ten inputs of one cell, standardised and packed as BF16 pairs (pairs 5-7
// zero); st: the cell's streamed populations in a stash of stride NT, as
// g = f - w, or (RAW) as f itself.
template <int Q, typename R, int NT, bool RAW = false>
__device__ __forceinline__ void learned_inputs(const R* st, R drho, R ux, R uy, R uz, R Sxx, R Syy, R Szz, R Sxy,
                                               R Sxz, R Syz, R tau_hat, const float* xmu, const float* xis,
                                               uint32_t (&xin)[8])
{
    constexpr R th = R(kTheta);
    const R rho = R(1) + drho, irho = R(1) / rho;
    R pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
    static_for<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
        if constexpr (cx != 0 || cy != 0 || cz != 0) {
            const R gi = RAW ? st[i * NT] - (R)weight_of(Q, i) : st[i * NT];
            if (cx != 0) pxx += gi;
            if (cy != 0) pyy += gi;
            if (cz != 0) pzz += gi;
            if (cx * cy == 1) pxy += gi;
            if (cx * cy == -1) pxy -= gi;
            if (cx * cz == 1) pxz += gi;
            if (cx * cz == -1) pxz -= gi;
            if (cy * cz == 1) pyz += gi;
            if (cy * cz == -1) pyz -= gi;
        }
    });
    const R k = R(-2) * th * tau_hat;  // m_CE / rho = k S
    const R a00 = k * Sxx, a11 = k * Syy, a22 = k * Szz, a01 = k * Sxy, a02 = k * Sxz, a12 = k * Syz;
    // inputs 0-5: the KC-MP carrier (m_neq - m_CE)/rho, m_neq = Pi' - rho u u - theta drho I
    R x[10];
    x[0] = (pxx - rho * ux * ux - th * drho) * irho - a00;
    x[1] = (pyy - rho * uy * uy - th * drho) * irho - a11;
    x[2] = (pzz - rho * uz * uz - th * drho) * irho - a22;
    x[3] = (pxy - rho * ux * uy) * irho - a01;
    x[4] = (pxz - rho * ux * uz) * irho - a02;
    x[5] = (pyz - rho * uy * uz) * irho - a12;
    const R tr = a00 + a11 + a22;
    const R tr2 = a00 * a00 + a11 * a11 + a22 * a22 + R(2) * (a01 * a01 + a02 * a02 + a12 * a12);
    x[6] = tr;
    x[7] = R(0.5) * (tr * tr - tr2);
    x[8] = a00 * (a11 * a22 - a12 * a12) - a01 * (a01 * a22 - a12 * a02) + a02 * (a01 * a12 - a11 * a02);
    x[9] = tau_hat;
#pragma unroll
    for (int q = 0; q < 5; ++q)
        xin[q] = pack_bf16(((float)x[2 * q] - xmu[2 * q]) * xis[2 * q], ((float)x[2 * q + 1] - xmu[2 * q + 1]) * xis[2 * q + 1]);
#pragma unroll
    for (int q = 5; q < 8; ++q) xin[q] = 0u;
}

template <int Q, typename R, int NT, bool DUAL = false>
__device__ __forceinline__ void learned_msgs(const R* st, R drho, R ux, R uy, R uz, R Sxx, R Syy, R Szz, R Sxy,
                                             R Sxz, R Syz, R tau_hat, const unsigned char* sm_mlp, unsigned char* xch,
                                             int lane, R (&msgs)[6])
{
    using L = MlpLayout;
    const R rho = R(1) + drho;
    uint32_t xin[8];
    learned_inputs<Q, R, NT>(st, drho, ux, uy, uz, Sxx, Syy, Szz, Sxy, Sxz, Syz, tau_hat,
                             reinterpret_cast<const float*>(sm_mlp + L::XMU),
                             reinterpret_cast<const float*>(sm_mlp + L::XIS), xin);
    __nv_bfloat16* X = reinterpret_cast<__nv_bfloat16*>(xch);
    float* Y = reinterpret_cast<float*>(xch);  // overlays the inputs
    uint32_t* Xrow = reinterpret_cast<uint32_t*>(X + lane * L::XLD);
#pragma unroll
    for (int q = 0; q < 8; ++q) Xrow[q] = xin[q];
    __syncwarp();
    // DUAL: both 16-cell halves of the warp together (where the kernel has
    // the registers for it)
    if constexpr (DUAL)
        mlp_warp_forward_dual(sm_mlp, X, Y, lane);
    else
        mlp_warp_forward(sm_mlp, X, Y, lane);
    __syncwarp();
    const float* ymu = reinterpret_cast<const float*>(sm_mlp + L::YMU);
    const float* ysd = reinterpret_cast<const float*>(sm_mlp + L::YSD);
#pragma unroll
    for (int q = 0; q < 6; ++q) msgs[q] = rho * (R)(Y[lane * 8 + q] * ysd[q] + ymu[q]);
    __syncwarp();
}

template <int Q, typename S, int CL, int BC, int TY>
__global__ void __launch_bounds__(32 * TY, (sizeof(typename StoreTraits<S>::R) == 8 || TY >= 16) ? 1 : 2)
    step_kernel(const StepArgs a)
{
    using R = typename StoreTraits<S>::R;
    using Sh = StepShape<Q, R, BC, TY>;
    constexpr int TX = Sh::TX, HY = Sh::HY, RX = Sh::RX, RN = Sh::RN, NT = Sh::NT, NB = Sh::NB;
    static_assert(NB <= NT, "every halo cell of the ring needs a thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* ring = reinterpret_cast<R*>(smem_raw);  // [4][3][RN]
    R* stash = ring + 4 * 3 * RN;              // [2][Q][NT]
    unsigned char* sm_mlp = smem_raw + Sh::base_bytes;                      // learned closure only
    unsigned char* sm_xch = sm_mlp + MlpLayout::BYTES + threadIdx.y * MlpLayout::XCH_BYTES;
    if constexpr (CL == CL_LEARNED) {
        const uint4* src = static_cast<const uint4*>(a.mlp);
        uint4* dst = reinterpret_cast<uint4*>(sm_mlp);
        for (int k = threadIdx.y * 32 + threadIdx.x; k < MlpLayout::BYTES / 16; k += 32 * TY) dst[k] = src[k];
    }

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int tiles_x = (nx + TX - 1) / TX;
    const int x0 = (int)(blockIdx.x % tiles_x) * TX;
    const int y0 = (int)(blockIdx.x / tiles_x) * TY;
    const int z0 = (int)blockIdx.y * a.zchunk;
    if (z0 >= nz) return;  // uniform over the CTA
    const int z1 = min(nz, z0 + a.zchunk);
    const int box = blockIdx.z;
    const long long ps = a.popstride;
    const int plane = (int)a.plane;
    const S* __restrict__ fin = static_cast<const S*>(a.fin) + (long long)box * a.boxstride;
    S* __restrict__ fout = static_cast<S*>(a.fout) + (long long)box * a.boxstride;

    const double nu_d = a.box_nu[box];
    const R nu = (R)nu_d;
    const R tau_hat = (R)(nu_d / kTheta + 0.5);
    const R omega = (R)(1.0 / (nu_d / kTheta + 0.5));
    const R cnud = (R)a.cnu_delta;
    constexpr bool FORCE = (BC == BC_WALLS_Y);
    const R Fx = FORCE ? (R)a.force[0] : R(0), Fy = FORCE ? (R)a.force[1] : R(0), Fz = FORCE ? (R)a.force[2] : R(0);

    // own column; lanes beyond nx wrap (periodic x) and are not stored
    const int gx = x0 + tx, gy = y0 + ty;
    const bool own_store = gx < nx && gy < ny;
    const Col own = make_col<BC>(gx, gy, nx, ny);
    const int own_r = (ty + HY) * RX + (tx + 1);

    // halo column of this thread (ring cells outside the 32 x TY interior)
    Col hal = own;
    int hal_r = -1;
    if (tid < NB) {
        // the rows y0 - 1 and y0 + TY, then the two columns (every tile reads
        // them), then, with walls, the outer rows y0 - 2 and y0 + TY + 1
        int lx, ly;
        int b = tid;
        if (b < RX) {
            lx = b - 1;
            ly = -1;
        } else if ((b -= RX) < RX) {
            lx = b - 1;
            ly = TY;
        } else if ((b -= RX) < 2 * TY) {
            lx = (b < TY) ? -1 : TX;
            ly = b % TY;
        } else {
            b -= 2 * TY;
            lx = b % RX - 1;
            ly = (b < RX) ? -2 : TY + 1;
        }
        hal = make_col<BC>(x0 + lx, y0 + ly, nx, ny);
        hal_r = (ly + HY) * RX + (lx + 1);
        // The outer rows feed only the one-sided wall stencils (Eqs. fd_boundary):
        // the wall row y = 0 is a tile's first row and reads rows 1, 2 inside it;
        // the wall row y = ny - 1 reads ly = -2 only when it is the tile's first
        // row (y0 = ny - 1).  Otherwise they are not pulled (their ring entries
        // are never read).
        if (BC == BC_WALLS_Y && (ly == -2 || ly == TY + 1) && !(ly == -2 && y0 == ny - 1)) hal.valid = false;
        // the corners are never read either (the stencils are +-1 in x or in y)
        if ((lx == -1 || lx == TX) && (ly < 0 || ly >= TY)) hal.valid = false;
    }

    auto zrows = [&](int z, int (&zr)[3]) {
        const int zc = z < 0 ? z + nz : (z >= nz ? z - nz : z);  // z in [-1, nz]
        zr[0] = (zc == 0 ? nz - 1 : zc - 1) * plane;
        zr[1] = zc * plane;
        zr[2] = (zc == nz - 1 ? 0 : zc + 1) * plane;
    };
    auto rslot = [&](int z) { return (z - z0 + 1) & 3; };
    auto ringp = [&](int s, int c) { return ring + (s * 3 + c) * RN; };
    auto put_u = [&](int z, int r, R vx, R vy, R vz) {
        const int s = rslot(z);
        ringp(s, 0)[r] = vx;
        ringp(s, 1)[r] = vy;
        ringp(s, 2)[r] = vz;
    };

    // velocity of the halo column at plane z into the ring
    auto halo_plane = [&](int z) {
        if (tid < NB) {
            R vx = 0, vy = 0, vz = 0;
            if (hal.valid) {
                int zr[3];
                zrows(z, zr);
                R gh[Q];
                pull<Q, S, R, BC>(fin, ps, hal, zr, gh);
                R dh;
                moments<Q, R>(gh, dh, vx, vy, vz, Fx, Fy, Fz);
            }
            put_u(z, hal_r, vx, vy, vz);
        }
    };
    // own column at plane z: velocity into the ring; populations into the
    // stash slot (z & 1) when `keep`
    auto own_plane = [&](int z, bool keep, R& r, R& vx, R& vy, R& vz) {
        r = 0;
        vx = vy = vz = 0;
        if (own.valid) {
            int zr[3];
            zrows(z, zr);
            R t[Q];
            pull<Q, S, R, BC>(fin, ps, own, zr, t);
            moments<Q, R>(t, r, vx, vy, vz, Fx, Fy, Fz);
            if (keep) {
                R* st = stash + (z & 1) * Q * NT + tid;
#pragma unroll
                for (int i = 0; i < Q; ++i) st[i * NT] = t[i];
            }
        }
        put_u(z, own_r, vx, vy, vz);
    };

    R drho, ux, uy, uz;  // moments of the own cell at plane z
    {
        R r0, v0x, v0y, v0z;
        own_plane(z0 - 1, false, r0, v0x, v0y, v0z);
        halo_plane(z0 - 1);
        halo_plane(z0);
        own_plane(z0, true, drho, ux, uy, uz);
    }
    __syncthreads();

    for (int z = z0; z < z1; ++z) {
        // ---- plane z+1: halo and own column velocities into the ring
        R rn, vnx, vny, vnz;
        halo_plane(z + 1);
        own_plane(z + 1, z + 1 < z1, rn, vnx, vny, vnz);
        __syncthreads();

        // ---- plane z: strain from the ring, closure, relaxation, store
        if (own.valid) {
            // a non-finite component makes the sum non-finite (the moments are O(1))
            if (own_store && !isfinite(drho + ux + uy + uz)) atomicOr(a.flag, 1u);
            const int sm = rslot(z - 1), s0 = rslot(z), sp = rslot(z + 1);
            R du[3][3];  // du[a][b] = d_a u_b
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const R* r0 = ringp(s0, b);
                du[0][b] = R(0.5) * (r0[own_r + 1] - r0[own_r - 1]);
                du[2][b] = R(0.5) * (ringp(sp, b)[own_r] - ringp(sm, b)[own_r]);
                if (BC == BC_WALLS_Y && gy == 0)
                    du[1][b] = R(0.5) * (R(-3) * r0[own_r] + R(4) * r0[own_r + RX] - r0[own_r + 2 * RX]);
                else if (BC == BC_WALLS_Y && gy == ny - 1)
                    du[1][b] = R(0.5) * (R(3) * r0[own_r] - R(4) * r0[own_r - RX] + r0[own_r - 2 * RX]);
                else
                    du[1][b] = R(0.5) * (r0[own_r + RX] - r0[own_r - RX]);
            }
            const R Sxx = du[0][0], Syy = du[1][1], Szz = du[2][2];
            const R Sxy = R(0.5) * (du[0][1] + du[1][0]);
            const R Sxz = R(0.5) * (du[0][2] + du[2][0]);
            const R Syz = R(0.5) * (du[1][2] + du[2][1]);
            R g[Q];
            const R* st = stash + (z & 1) * Q * NT + tid;
            if constexpr (CL == CL_LEARNED) {
                R msgs[6];
                learned_msgs<Q, R, NT, (NT <= 128)>(st, drho, ux, uy, uz, Sxx, Syy, Szz, Sxy, Sxz, Syz, tau_hat, sm_mlp, sm_xch,
                                       tx, msgs);
#pragma unroll
                for (int i = 0; i < Q; ++i) g[i] = st[i * NT];
                collide<Q, R, CL, FORCE>(g, drho, ux, uy, uz, Sxx, Syy, Szz, Sxy, Sxz, Syz, omega, tau_hat, nu, cnud,
                                         Fx, Fy, Fz, msgs);
            } else {
#pragma unroll
                for (int i = 0; i < Q; ++i) g[i] = st[i * NT];
                collide<Q, R, CL, FORCE>(g, drho, ux, uy, uz, Sxx, Syy, Szz, Sxy, Sxz, Syz, omega, tau_hat, nu, cnud,
                                         Fx, Fy, Fz);
            }
            if (own_store) {
                S* dst = fout + (z * plane + own.yr[1] + own.xs[1]);
                static_for<Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    store_g<S, R>(dst + (long long)i * ps, g[i], (R)weight_of(Q, i));
                });
            }
        }
        drho = rn;
        ux = vnx;
        uy = vny;
        uz = vnz;
    }
}

template <int Q, typename S, int CL, int BC, int TY>
cudaError_t prepare_step_t()
{
    return cudaFuncSetAttribute(step_kernel<Q, S, CL, BC, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)step_smem_bytes<Q, typename StoreTraits<S>::R, BC, TY, CL>());
}

template <int Q, typename S, int CL, int BC, int TY>
cudaError_t launch_step_t(const StepArgs& a, int nbatch, cudaStream_t s)
{
    using Sh = StepShape<Q, typename StoreTraits<S>::R, BC, TY>;
    static bool attr_set = false;  // per instantiation; prepare_step_t sets it ahead of stream capture
    if (!attr_set) {
        cudaError_t e = prepare_step_t<Q, S, CL, BC, TY>();
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int tiles = ((a.nx + Sh::TX - 1) / Sh::TX) * ((a.ny + TY - 1) / TY);
    const int chunks = (a.nz + a.zchunk - 1) / a.zchunk;
    dim3 grid(tiles, chunks, nbatch), block(Sh::TX, TY);
    if (CL == CL_LEARNED && !a.mlp) return cudaErrorInvalidValue;
    step_kernel<Q, S, CL, BC, TY><<<grid, block, step_smem_bytes<Q, typename StoreTraits<S>::R, BC, TY, CL>(), s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbmk
