// Fused step kernel on packed FP32 pairs: two cells per thread (sm_100+).
//
// Same update as step_kernel (lbm_step.cuh) for 32-bit arithmetic (FP32, FP16
// and BF16 storage).  A CTA owns a 64 x TY tile of cells; lane l of warp w owns
// the cells (x0 + l, y0 + w) and (x0 + 32 + l, y0 + w).  Every per-cell quantity
// is a pair (cell A, cell B) held in a float2, and the arithmetic runs on the
// paired FP32 instructions (FADD2 / FMUL2 / FFMA2, one issue slot for two
// operations, each rounded exactly as its scalar counterpart): the moment sums,
// the strain, the closure and the relaxation of two cells cost the issue slots
// of one.  The two cells share their y and z address arithmetic.  The halo
// cells of the velocity ring are paired the same way.
//
// Synchronisation as in step_kernel_sb (lbm_step_split.cuh): the halo and own
// loads of a plane are issued together, and each plane's velocities are
// published with an mbarrier arrival and awaited only before the strain that
// reads them, with a five-plane velocity ring.  The population stash holds the
// pairs of the two cells ([2][Q][32*TY] float2).
#pragma once

#include "lbm_mbarrier.cuh"
#include "lbm_step.cuh"

namespace lbmk {

// ------------------------------------------------------------------ float pairs

struct F2 {
    float2 v;
};

__device__ __forceinline__ F2 bc2(float a) { return F2{make_float2(a, a)}; }
__device__ __forceinline__ F2 mk2(float a, float b) { return F2{make_float2(a, b)}; }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator-(F2 a, F2 b)
{
    F2 r;
    asm("{\n .reg .b64 pa, pb, pd;\n mov.b64 pa, {%2, %3};\n mov.b64 pb, {%4, %5};\n sub.rn.f32x2 pd, pa, pb;\n"
        " mov.b64 {%0, %1}, pd;\n}\n"
        : "=f"(r.v.x), "=f"(r.v.y)
        : "f"(a.v.x), "f"(a.v.y), "f"(b.v.x), "f"(b.v.y));
    return r;
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return F2{__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2& operator-=(F2& a, F2 b) { return a = a - b; }
__device__ __forceinline__ bool finite2(F2 a) { return isfinite(a.v.x) && isfinite(a.v.y); }

// ------------------------------------------------------------------ columns

// Two columns in the same row: x offsets of cell A (xa) and cell B (xb), one y.
struct Col2 {
    int xa[3], xb[3];
    int yr[3];
    bool valid;
};

template <int BC>
__device__ __forceinline__ Col2 make_col2(int gxa, int gxb, int gy, int nx, int ny)
{
    const Col ca = make_col<BC>(gxa, gy, nx, ny), cb = make_col<BC>(gxb, gy, nx, ny);
    Col2 c;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        c.xa[k] = ca.xs[k];
        c.xb[k] = cb.xs[k];
        c.yr[k] = ca.yr[k];
    }
    c.valid = ca.valid;
    return c;
}

// pull of the two cells of a row pair (the scalar pull, Eq. streaming, per cell)
template <int Q, typename S, int BC>
__device__ __forceinline__ void pull2(const S* __restrict__ fin, long long ps, const Col2& col, const int (&zr)[3],
                                      F2 (&g)[Q])
{
    static_for<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
        constexpr int io = opp_of(Q, i);
        const float w = (float)weight_of(Q, i);
        if (BC == BC_WALLS_Y && cy != 0) {
            const int row = col.yr[1 - cy];
            if (row >= 0) {
                const S* src = fin + (long long)i * ps + (zr[1 - cz] + row);
                g[i] = mk2(load_g<S, float>(src + col.xa[1 - cx], w), load_g<S, float>(src + col.xb[1 - cx], w));
            } else {
                const S* src = fin + (long long)io * ps + (zr[1] + col.yr[1]);
                g[i] = mk2(load_g<S, float>(src + col.xa[1], w), load_g<S, float>(src + col.xb[1], w));
            }
        } else {
            const S* src = fin + (long long)i * ps + (zr[1 - cz] + col.yr[1 - cy]);
            g[i] = mk2(load_g<S, float>(src + col.xa[1 - cx], w), load_g<S, float>(src + col.xb[1 - cx], w));
        }
    });
}

// pull of two unrelated cells (halo pairs); an invalid cell (beyond a wall) reads 0
template <int Q, typename S, int BC>
__device__ __forceinline__ void pull_any2(const S* __restrict__ fin, long long ps, const Col& ca, const Col& cb,
                                          bool va, bool vb, const int (&zr)[3], F2 (&g)[Q])
{
    float ga[Q], gb[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) ga[i] = gb[i] = 0.f;
    if (va) pull<Q, S, float, BC>(fin, ps, ca, zr, ga);
    if (vb) pull<Q, S, float, BC>(fin, ps, cb, zr, gb);
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = mk2(ga[i], gb[i]);
}

// drho = sum g, u = (sum g c + F/2) / (1 + drho), per cell (the scalar moments)
template <int Q>
__device__ __forceinline__ void moments2(const F2 (&g)[Q], F2& drho, F2& ux, F2& uy, F2& uz, float Fx, float Fy,
                                         float Fz)
{
    F2 d = bc2(0.f), jx = bc2(0.f), jy = bc2(0.f), jz = bc2(0.f);
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
    drho = d;
    const F2 inv = mk2(1.f / (1.f + d.v.x), 1.f / (1.f + d.v.y));
    ux = (jx + bc2(0.5f * Fx)) * inv;
    uy = (jy + bc2(0.5f * Fy)) * inv;
    uz = (jz + bc2(0.5f * Fz)) * inv;
}

__device__ __forceinline__ F2 omega_sgs2(F2 tr, float nu, float omega, float cnud)
{
    return mk2(omega_sgs<float>(tr.v.x, nu, omega, cnud), omega_sgs<float>(tr.v.y, nu, omega, cnud));
}

// collision of two cells: the common form g <- a g + w (b (P - 1) + c0 + D H(c))
// of collide() (lbm_step.cuh) with BGK, KC-MP and KC-RB carriers, on pairs
template <int Q, int CL, bool FORCE>
__device__ __forceinline__ void collide2(F2 (&g)[Q], F2 drho, F2 ux, F2 uy, F2 uz, F2 Sxx, F2 Syy, F2 Szz, F2 Sxy,
                                         F2 Sxz, F2 Syz, float omega, float tau_hat, float nu, float cnud, float Fx,
                                         float Fy, float Fz)
{
    static_assert(CL == CL_BGK || CL == CL_KCMP || CL == CL_KCRB_H || CL == CL_KCRB_RAW, "closure not paired");
    constexpr float th = (float)kTheta;
    constexpr float a1 = (float)(1.0 / kTheta);
    constexpr float a2 = (float)((1.0 - kTheta) / (2.0 * kTheta * kTheta));
    constexpr float a0 = (float)(-kTheta / (2.0 * kTheta * kTheta));
    const F2 rho = bc2(1.f) + drho;
    const F2 ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;

    F2 Mxx = bc2(0.f), Myy = Mxx, Mzz = Mxx, Mxy = Mxx, Mxz = Mxx, Myz = Mxx, t = Mxx;
    F2 ca = bc2(1.f - omega), cb = bc2(omega) * rho, c0 = bc2(omega) * drho, D = bc2(0.f);
    if constexpr (CL != CL_BGK) {
        F2 pxx = bc2(0.f), pyy = pxx, pzz = pxx, pxy = pxx, pxz = pxx, pyz = pxx;
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
        if constexpr (CL == CL_KCMP) {
            // m_sgs = Pi' - rho u u - theta drho I + 2 rho theta tau_hat S   (App. F.3)
            const F2 nrho = bc2(0.f) - rho;
            const F2 rt = bc2(2.f * th * tau_hat) * rho;
            const F2 tdr = bc2(th) * drho;
            Mxx = fma2(rt, Sxx, fma2(nrho, ux2, pxx) - tdr);
            Myy = fma2(rt, Syy, fma2(nrho, uy2, pyy) - tdr);
            Mzz = fma2(rt, Szz, fma2(nrho, uz2, pzz) - tdr);
            Mxy = fma2(rt, Sxy, fma2(nrho, ux * uy, pxy));
            Mxz = fma2(rt, Sxz, fma2(nrho, ux * uz, pxz));
            Myz = fma2(rt, Syz, fma2(nrho, uy * uz, pyz));
            const F2 tr = Mxx + Myy + Mzz;
            const F2 omega_s = omega_sgs2(tr, nu, omega, cnud);
            t = bc2(th) * tr;
            D = (bc2(omega) - omega_s) * bc2((float)(1.0 / (2.0 * kTheta * kTheta)));
        } else {  // KC-RB (App. F.2), Hermite or raw first-order reconstruction
            constexpr bool herm = (CL == CL_KCRB_H);
            const F2 trS = Sxx + Syy + Szz;
            const F2 usq = ux2 + uy2 + uz2;
            const F2 trf1 = bc2((herm ? -2.f : -5.f) * tau_hat * th) * rho * trS;
            const F2 tr = (((pxx + pyy) + pzz) - rho * usq) - bc2(3.f * th) * drho - trf1;
            const F2 omega_s = omega_sgs2(tr, nu, omega, cnud);
            Mxx = Sxx;
            Myy = Syy;
            Mzz = Szz;
            Mxy = Sxy;
            Mxz = Sxz;
            Myz = Syz;
            t = herm ? bc2(th) * trS : bc2(0.f);
            ca = bc2(1.f) - omega_s;
            cb = omega_s * rho;
            c0 = omega_s * drho;
            D = (omega_s - bc2(omega)) * (bc2(-tau_hat * a1) * rho);
        }
    }

    if constexpr (Q == 27) {
        const F2 A1 = bc2(a1), A2 = bc2(a2), A0 = bc2(a0);
        const F2 ex[3] = {fma2(A2, ux2, bc2(-a1) * ux), A0 * ux2, fma2(A2, ux2, A1 * ux)};
        const F2 ey[3] = {fma2(A2, uy2, bc2(-a1) * uy), A0 * uy2, fma2(A2, uy2, A1 * uy)};
        const F2 ez[3] = {fma2(A2, uz2, bc2(-a1) * uz), A0 * uz2, fma2(A2, uz2, A1 * uz)};
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
            constexpr float w = (float)weight_of(Q, i);
            const F2 Y = fma2(ey[cy + 1], ez[cz + 1], ey[cy + 1] + ez[cz + 1]);
            const F2 pm1 = fma2(ex[cx + 1], Y, ex[cx + 1] + Y);
            F2 K = fma2(cb, pm1, c0);
            if constexpr (CL != CL_BGK) {
                F2 h = bc2(0.f) - t;
                if (cy != 0) h += Myy;
                if (cz != 0) h += Mzz;
                if (cy * cz == 1) h = fma2(bc2(2.f), Myz, h);
                if (cy * cz == -1) h = fma2(bc2(-2.f), Myz, h);
                if (cx != 0) {
                    F2 e = bc2(0.f);
                    if (cy == 1) e = Mxy;
                    if (cy == -1) e = bc2(0.f) - Mxy;
                    if (cz == 1) e = (cy != 0) ? e + Mxz : Mxz;
                    if (cz == -1) e = (cy != 0) ? e - Mxz : bc2(0.f) - Mxz;
                    h += (cy != 0 || cz != 0) ? fma2(bc2(2.f * cx), e, Mxx) : Mxx;
                }
                K = fma2(D, h, K);
            }
            g[i] = fma2(ca, g[i], bc2(w) * K);
        });
    } else {
        const F2 A1 = bc2(a1), half = bc2(0.5f);
        const F2 usq = ux2 + uy2 + uz2;
        const F2 base = bc2(-0.5f * a1) * usq;
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
            constexpr float w = (float)weight_of(Q, i);
            F2 cu = bc2(0.f);
            if (cx == 1) cu = ux;
            if (cx == -1) cu = bc2(0.f) - ux;
            if (cy == 1) cu = (cx != 0) ? cu + uy : uy;
            if (cy == -1) cu = (cx != 0) ? cu - uy : bc2(0.f) - uy;
            if (cz == 1) cu = (cx != 0 || cy != 0) ? cu + uz : uz;
            if (cz == -1) cu = (cx != 0 || cy != 0) ? cu - uz : bc2(0.f) - uz;
            // D3Q19 second-order Hermite equilibrium: P - 1 = c.u/theta + (c.u)^2/(2 theta^2) - u^2/(2 theta)
            const F2 acu = A1 * cu;
            const F2 pm1 = (cx == 0 && cy == 0 && cz == 0) ? base : fma2(half * acu, acu, acu + base);
            F2 K = fma2(cb, pm1, c0);
            if constexpr (CL != CL_BGK) {
                F2 h = bc2(0.f) - t;
                if (cx != 0) h += Mxx;
                if (cy != 0) h += Myy;
                if (cz != 0) h += Mzz;
                if (cx * cy != 0) h = fma2(bc2(2.f * cx * cy), Mxy, h);
                if (cx * cz != 0) h = fma2(bc2(2.f * cx * cz), Mxz, h);
                if (cy * cz != 0) h = fma2(bc2(2.f * cy * cz), Myz, h);
                K = fma2(D, h, K);
            }
            g[i] = fma2(ca, g[i], bc2(w) * K);
        });
    }
    if constexpr (FORCE) {
        // Guo source (1 - omega/2) w [(c - u)/theta + (c.u) c/theta^2] . F
        const float pref = 1.f - 0.5f * omega;
        const F2 uF = fma2(ux, bc2(Fx), fma2(uy, bc2(Fy), uz * bc2(Fz)));
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
            constexpr float w = (float)weight_of(Q, i);
            const float cF = (float)cx * Fx + (float)cy * Fy + (float)cz * Fz;
            const F2 cu = fma2(bc2((float)cx), ux, fma2(bc2((float)cy), uy, bc2((float)cz) * uz));
            const F2 term = fma2(cu * bc2(cF), bc2(a1 * a1), (bc2(cF) - uF) * bc2(a1));
            g[i] = fma2(bc2(pref * w), term, g[i]);
        });
    }
}

// ------------------------------------------------------------------ kernel

template <int Q, int BC, int TY>
struct PairShape {
    static constexpr int TX = 64;  // cells per tile row (two per lane)
    static constexpr int HY = (BC == BC_WALLS_Y) ? 2 : 1;
    static constexpr int RX = TX + 2;
    static constexpr int RY = TY + 2 * HY;
    static constexpr int RN = RX * RY;
    static constexpr int NT = 32 * TY;  // threads
    static constexpr int NB = RN - TX * TY;  // halo cells of the ring plane
    static constexpr int NBP = (NB + 1) / 2;  // halo threads (two halo cells each)
    static constexpr size_t ring_off = 16;
    static constexpr size_t stash_off = ring_off + sizeof(float) * (size_t)(5 * 3 * RN);
    static constexpr size_t bytes = stash_off + sizeof(float2) * (size_t)(2 * Q * NT);
};

template <int Q, int BC, int TY>
__device__ __forceinline__ void ring_cell(int b, int& lx, int& ly)
{
    using P = PairShape<Q, BC, TY>;
    if (b < P::HY * P::RX) {
        lx = b % P::RX - 1;
        ly = b / P::RX - P::HY;
    } else if ((b -= P::HY * P::RX) < P::HY * P::RX) {
        lx = b % P::RX - 1;
        ly = TY + b / P::RX;
    } else {
        b -= P::HY * P::RX;
        lx = (b < TY) ? -1 : P::TX;
        ly = b % TY;
    }
}

template <int Q, typename S, int CL, int BC, int TY>
__global__ void __launch_bounds__(32 * TY, TY >= 8 ? 1 : 2) step_kernel_x2(const StepArgs a)
{
    using P = PairShape<Q, BC, TY>;
    constexpr int TX = P::TX, HY = P::HY, RX = P::RX, RN = P::RN, NT = P::NT, NB = P::NB, NBP = P::NBP;
    static_assert(NBP <= NT, "every halo pair needs a thread");
    extern __shared__ __align__(16) unsigned char smem_x2[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_x2);
    float* ring = reinterpret_cast<float*>(smem_x2 + P::ring_off);    // [5][3][RN]
    F2* stash = reinterpret_cast<F2*>(smem_x2 + P::stash_off);        // [2][Q][NT]

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
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
    const float nu = (float)nu_d;
    const float tau_hat = (float)(nu_d / kTheta + 0.5);
    const float omega = (float)(1.0 / (nu_d / kTheta + 0.5));
    const float cnud = (float)a.cnu_delta;
    constexpr bool FORCE = (BC == BC_WALLS_Y);
    const float Fx = FORCE ? (float)a.force[0] : 0.f, Fy = FORCE ? (float)a.force[1] : 0.f,
                Fz = FORCE ? (float)a.force[2] : 0.f;

    // own cells: A = (x0 + tx, y0 + ty), B = (x0 + 32 + tx, y0 + ty)
    const int gxa = x0 + tx, gxb = x0 + 32 + tx, gy = y0 + ty;
    const bool store_a = gxa < nx && gy < ny, store_b = gxb < nx && gy < ny;
    const Col2 own = make_col2<BC>(gxa, gxb, gy, nx, ny);
    const int own_ra = (ty + HY) * RX + (tx + 1), own_rb = own_ra + 32;

    // halo pair of this thread: ring cells tid and tid + NBP (the second may not exist)
    Col h1 = make_col<BC>(gxa, gy, nx, ny), h2 = h1;
    int h1_r = -1, h2_r = -1;
    bool h1_ok = false, h2_ok = false;
    if (tid < NBP) {
        int lx, ly;
        ring_cell<Q, BC, TY>(tid, lx, ly);
        h1 = make_col<BC>(x0 + lx, y0 + ly, nx, ny);
        h1_r = (ly + HY) * RX + (lx + 1);
        h1_ok = h1.valid;
        if (tid + NBP < NB) {
            ring_cell<Q, BC, TY>(tid + NBP, lx, ly);
            h2 = make_col<BC>(x0 + lx, y0 + ly, nx, ny);
            h2_r = (ly + HY) * RX + (lx + 1);
            h2_ok = h2.valid;
        }
    }

    if (tid == 0) {
        mbar_init(&mbar[0], NT);
        mbar_init(&mbar[1], NT);
    }
    __syncthreads();

    auto zrows = [&](int z, int (&zr)[3]) {
        const int zc = wrapi(z, nz);
        zr[0] = (zc == 0 ? nz - 1 : zc - 1) * plane;
        zr[1] = zc * plane;
        zr[2] = (zc == nz - 1 ? 0 : zc + 1) * plane;
    };
    auto rslot = [&](int z) { return (z - z0 + 1) % 5; };
    auto ringp = [&](int s, int c) { return ring + (s * 3 + c) * RN; };
    auto put_u = [&](int z, int r, float vx, float vy, float vz) {
        const int s = rslot(z);
        ringp(s, 0)[r] = vx;
        ringp(s, 1)[r] = vy;
        ringp(s, 2)[r] = vz;
    };
    auto load_plane = [&](int z, bool keep, bool halo, F2& r, F2& vx, F2& vy, F2& vz) {
        int zr[3];
        zrows(z, zr);
        const bool do_h = halo && tid < NBP;
        F2 t[Q], gh[Q];
        if (own.valid) pull2<Q, S, BC>(fin, ps, own, zr, t);
        if (do_h) pull_any2<Q, S, BC>(fin, ps, h1, h2, h1_ok, h2_ok, zr, gh);
        r = vx = vy = vz = bc2(0.f);
        if (own.valid) {
            moments2<Q>(t, r, vx, vy, vz, Fx, Fy, Fz);
            if (keep) {
                F2* st = stash + (z & 1) * Q * NT + tid;
#pragma unroll
                for (int i = 0; i < Q; ++i) st[i * NT] = t[i];
            }
        }
        put_u(z, own_ra, vx.v.x, vy.v.x, vz.v.x);
        put_u(z, own_rb, vx.v.y, vy.v.y, vz.v.y);
        if (do_h) {
            F2 dh, hx, hy, hz;
            moments2<Q>(gh, dh, hx, hy, hz, Fx, Fy, Fz);
            put_u(z, h1_r, h1_ok ? hx.v.x : 0.f, h1_ok ? hy.v.x : 0.f, h1_ok ? hz.v.x : 0.f);
            if (h2_r >= 0) put_u(z, h2_r, h2_ok ? hx.v.y : 0.f, h2_ok ? hy.v.y : 0.f, h2_ok ? hz.v.y : 0.f);
        }
    };
    auto arrive = [&](int p) { mbar_arrive(&mbar[(p - z0) & 1]); };
    auto wait = [&](int p) { return mbar_wait_bounded(&mbar[(p - z0) & 1], (unsigned)((p - z0) >> 1) & 1u); };

    F2 drho, ux, uy, uz;  // moments of the own cells at plane z
    {
        F2 r0, v0x, v0y, v0z;
        load_plane(z0 - 1, false, false, r0, v0x, v0y, v0z);
        load_plane(z0, true, true, drho, ux, uy, uz);
        arrive(z0);
    }

    for (int z = z0; z < z1; ++z) {
        F2 rn, vnx, vny, vnz;
        load_plane(z + 1, z + 1 < z1, z + 1 < z1, rn, vnx, vny, vnz);
        arrive(z + 1);
        if (!wait(z)) {
            atomicOr(a.flag, kFlagTimeout);
            return;
        }
        if (own.valid) {
            if ((store_a || store_b) && !(finite2(drho) && finite2(ux) && finite2(uy) && finite2(uz)))
                atomicOr(a.flag, kFlagNonfinite);
            const int sm = rslot(z - 1), s0 = rslot(z), sp = rslot(z + 1);
            F2 du[3][3];  // du[a][b] = d_a u_b, cells A and B
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const float* r0 = ringp(s0, b);
                const float* rp = ringp(sp, b);
                const float* rm = ringp(sm, b);
                du[0][b] = bc2(0.5f) * (mk2(r0[own_ra + 1], r0[own_rb + 1]) - mk2(r0[own_ra - 1], r0[own_rb - 1]));
                du[2][b] = bc2(0.5f) * (mk2(rp[own_ra], rp[own_rb]) - mk2(rm[own_ra], rm[own_rb]));
                if (BC == BC_WALLS_Y && gy == 0)
                    du[1][b] = bc2(0.5f) * (fma2(bc2(-3.f), mk2(r0[own_ra], r0[own_rb]),
                                                 bc2(4.f) * mk2(r0[own_ra + RX], r0[own_rb + RX])) -
                                            mk2(r0[own_ra + 2 * RX], r0[own_rb + 2 * RX]));
                else if (BC == BC_WALLS_Y && gy == ny - 1)
                    du[1][b] = bc2(0.5f) * (fma2(bc2(3.f), mk2(r0[own_ra], r0[own_rb]),
                                                 bc2(-4.f) * mk2(r0[own_ra - RX], r0[own_rb - RX])) +
                                            mk2(r0[own_ra - 2 * RX], r0[own_rb - 2 * RX]));
                else
                    du[1][b] = bc2(0.5f) * (mk2(r0[own_ra + RX], r0[own_rb + RX]) - mk2(r0[own_ra - RX], r0[own_rb - RX]));
            }
            const F2 Sxx = du[0][0], Syy = du[1][1], Szz = du[2][2];
            const F2 Sxy = bc2(0.5f) * (du[0][1] + du[1][0]);
            const F2 Sxz = bc2(0.5f) * (du[0][2] + du[2][0]);
            const F2 Syz = bc2(0.5f) * (du[1][2] + du[2][1]);
            F2 g[Q];
            const F2* st = stash + (z & 1) * Q * NT + tid;
#pragma unroll
            for (int i = 0; i < Q; ++i) g[i] = st[i * NT];
            collide2<Q, CL, FORCE>(g, drho, ux, uy, uz, Sxx, Syy, Szz, Sxy, Sxz, Syz, omega, tau_hat, nu, cnud, Fx,
                                   Fy, Fz);
            const int row = z * plane + own.yr[1];
            if (store_a) {
                S* dst = fout + (row + own.xa[1]);
                static_for<Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    store_g<S, float>(dst + (long long)i * ps, g[i].v.x, (float)weight_of(Q, i));
                });
            }
            if (store_b) {
                S* dst = fout + (row + own.xb[1]);
                static_for<Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    store_g<S, float>(dst + (long long)i * ps, g[i].v.y, (float)weight_of(Q, i));
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
cudaError_t prepare_x2_t()
{
    return cudaFuncSetAttribute(step_kernel_x2<Q, S, CL, BC, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)PairShape<Q, BC, TY>::bytes);
}

template <int Q, typename S, int CL, int BC, int TY>
cudaError_t launch_x2_t(const StepArgs& a, int nbatch, cudaStream_t s)
{
    using P = PairShape<Q, BC, TY>;
    static bool attr_set = false;  // per instantiation; prepare_x2_t sets it ahead of stream capture
    if (!attr_set) {
        cudaError_t e = prepare_x2_t<Q, S, CL, BC, TY>();
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int tiles = ((a.nx + P::TX - 1) / P::TX) * ((a.ny + TY - 1) / TY);
    const int chunks = (a.nz + a.zchunk - 1) / a.zchunk;
    dim3 grid(tiles, chunks, nbatch), block(32, TY);
    step_kernel_x2<Q, S, CL, BC, TY><<<grid, block, P::bytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbmk
