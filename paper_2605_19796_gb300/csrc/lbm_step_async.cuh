// Fused step kernel, asynchronous-copy pipeline (sm_103a), for FP32 storage
// and periodic boxes.
//
// Same update and same CTA decomposition as step_kernel (lbm_step.cuh): a CTA
// owns a 32 x TY column of cells and marches it through a chunk of z-planes,
// with the neighbour velocities of the finite-difference strain held in a
// shared-memory ring.  The difference is how the streamed (pulled)
// populations reach the SM: every thread issues 4-byte cp.async copies of its
// own cell's Q pulled values (and, for the first NB threads, of one halo
// cell's) straight into shared memory, two planes ahead of the plane being
// collided.  No registers hold prefetched data and the loads of plane z+2
// overlap the moments of plane z+1 and the collision of plane z.
//
// Shared memory per CTA: three own-population slots [3][Q][32*TY], two halo
// slots [2][Q][NB] and a three-plane velocity ring [3][3][34*(TY+2)], all
// 32-bit words.  For D3Q27 and TY = 8 that is 113 KB, two CTAs per SM.
//
// Per plane z (two barriers):
//   wait for plane z+1's copies; barrier
//   issue the copies of plane z+2 (into the slots of planes z-1 / z, consumed)
//   moments of plane z+1 (own cell and halo cells) -> ring
//   barrier
//   strain of plane z from the ring, collision, store
#pragma once

#include "lbm_step.cuh"

namespace lbmk {

__device__ __forceinline__ void cp_async4(uint32_t smem_addr, const void* gptr)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr), "l"(gptr) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int Q, int TY>
struct AsyncShape {
    static constexpr int TX = 32;
    static constexpr int RX = TX + 2;
    static constexpr int RY = TY + 2;
    static constexpr int RN = RX * RY;
    static constexpr int NT = TX * TY;
    static constexpr int NB = RN - NT;
    static constexpr int OWN_WORDS = 3 * Q * NT;
    static constexpr int HALO_WORDS = 2 * Q * NB;
    static constexpr int RING_WORDS = 3 * 3 * RN;
    static constexpr size_t smem_bytes = 4 * (size_t)(OWN_WORDS + HALO_WORDS + RING_WORDS);
};

template <int Q, int CL, int TY>
__global__ void __launch_bounds__(32 * TY, TY <= 4 ? 3 : (TY == 8 ? 2 : 1)) step_kernel_async(const StepArgs a)
{
    using R = float;
    using Sh = AsyncShape<Q, TY>;
    constexpr int TX = Sh::TX, RX = Sh::RX, RN = Sh::RN, NT = Sh::NT, NB = Sh::NB;
    static_assert(NB <= NT, "every halo cell of the ring needs a thread");
    extern __shared__ __align__(16) unsigned char smem_async[];
    float* own_buf = reinterpret_cast<float*>(smem_async);  // [3][Q][NT]
    float* halo_buf = own_buf + Sh::OWN_WORDS;              // [2][Q][NB]
    float* ring = halo_buf + Sh::HALO_WORDS;                // [3][3][RN]
    const uint32_t own_s = (uint32_t)__cvta_generic_to_shared(own_buf);
    const uint32_t halo_s = (uint32_t)__cvta_generic_to_shared(halo_buf);

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
    const float* __restrict__ fin = static_cast<const float*>(a.fin) + (long long)box * a.boxstride;
    float* __restrict__ fout = static_cast<float*>(a.fout) + (long long)box * a.boxstride;

    const double nu_d = a.box_nu[box];
    const R nu = (R)nu_d;
    const R tau_hat = (R)(nu_d / kTheta + 0.5);
    const R omega = (R)(1.0 / (nu_d / kTheta + 0.5));
    const R cnud = (R)a.cnu_delta;

    const int gx = x0 + tx, gy = y0 + ty;
    const bool own_store = gx < nx && gy < ny;
    const Col own = make_col<BC_PERIODIC>(gx, gy, nx, ny);
    const int own_r = (ty + 1) * RX + (tx + 1);

    Col hal = own;
    int hal_r = 0;
    if (tid < NB) {
        int lx, ly;
        int b = tid;
        if (b < RX) {
            lx = b - 1;
            ly = -1;
        } else if ((b -= RX) < RX) {
            lx = b - 1;
            ly = TY;
        } else {
            b -= RX;
            lx = (b < TY) ? -1 : TX;
            ly = b % TY;
        }
        hal = make_col<BC_PERIODIC>(x0 + lx, y0 + ly, nx, ny);
        hal_r = (ly + 1) * RX + (lx + 1);
    }

    auto oslot = [&](int p) { return (p - z0 + 1) % 3; };
    auto hslot = [&](int p) { return (p - z0 + 1) & 1; };
    auto rslot = [&](int p) { return (p - z0 + 1) % 3; };

    // cp.async of the pulled populations of plane p: own column and halo column
    auto issue = [&](int p) {
        const int zc = wrapi(p, nz);
        int zr[3];
        zr[0] = (zc == 0 ? nz - 1 : zc - 1) * plane;
        zr[1] = zc * plane;
        zr[2] = (zc == nz - 1 ? 0 : zc + 1) * plane;
        const uint32_t od = own_s + 4u * (uint32_t)(oslot(p) * Q * NT + tid);
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
            cp_async4(od + 4u * (uint32_t)(i * NT), fin + (long long)i * ps + (zr[1 - cz] + own.yr[1 - cy] + own.xs[1 - cx]));
        });
        if (tid < NB) {
            const uint32_t hd = halo_s + 4u * (uint32_t)(hslot(p) * Q * NB + tid);
            static_for<Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
                cp_async4(hd + 4u * (uint32_t)(i * NB),
                          fin + (long long)i * ps + (zr[1 - cz] + hal.yr[1 - cy] + hal.xs[1 - cx]));
            });
        }
        cp_async_commit();
    };

    // moments of shifted populations read from shared memory (stride between populations)
    auto smem_moments = [&](const float* src, int stride, R& d, R& vx, R& vy, R& vz) {
        R g[Q];
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            g[i] = src[i * stride] - R(weight_of(Q, i));
        });
        moments<Q, R>(g, d, vx, vy, vz, R(0), R(0), R(0));
    };
    auto put_u = [&](int p, int r, R vx, R vy, R vz) {
        float* rg = ring + rslot(p) * 3 * RN;
        rg[r] = vx;
        rg[RN + r] = vy;
        rg[2 * RN + r] = vz;
    };
    // moments of plane p: own cell (returned) and halo cell, velocities into the ring
    auto plane_moments = [&](int p, R& d, R& vx, R& vy, R& vz) {
        smem_moments(own_buf + oslot(p) * Q * NT + tid, NT, d, vx, vy, vz);
        put_u(p, own_r, vx, vy, vz);
        if (tid < NB) {
            R dh, hx, hy, hz;
            smem_moments(halo_buf + hslot(p) * Q * NB + tid, NB, dh, hx, hy, hz);
            put_u(p, hal_r, hx, hy, hz);
        }
    };

    R drho, ux, uy, uz;
    issue(z0 - 1);
    issue(z0);
    cp_async_wait<1>();
    __syncthreads();
    {
        R d0, v0x, v0y, v0z;
        plane_moments(z0 - 1, d0, v0x, v0y, v0z);
    }
    cp_async_wait<0>();
    __syncthreads();
    if (z0 + 1 <= z1) issue(z0 + 1);
    plane_moments(z0, drho, ux, uy, uz);

    for (int z = z0; z < z1; ++z) {
        cp_async_wait<0>();
        __syncthreads();  // plane z+1 landed; slots of planes z-1 (own) and z (halo) are free
        if (z + 2 <= z1) issue(z + 2);
        R dn, vnx, vny, vnz;
        plane_moments(z + 1, dn, vnx, vny, vnz);
        __syncthreads();  // ring of plane z+1 complete

        if (own_store && !(isfinite(drho) && isfinite(ux) && isfinite(uy) && isfinite(uz))) atomicOr(a.flag, 1u);
        const float* rm = ring + rslot(z - 1) * 3 * RN;
        const float* r0 = ring + rslot(z) * 3 * RN;
        const float* rp = ring + rslot(z + 1) * 3 * RN;
        R du[3][3];  // du[a][b] = d_a u_b
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            du[0][b] = R(0.5) * (r0[b * RN + own_r + 1] - r0[b * RN + own_r - 1]);
            du[1][b] = R(0.5) * (r0[b * RN + own_r + RX] - r0[b * RN + own_r - RX]);
            du[2][b] = R(0.5) * (rp[b * RN + own_r] - rm[b * RN + own_r]);
        }
        const R Sxx = du[0][0], Syy = du[1][1], Szz = du[2][2];
        const R Sxy = R(0.5) * (du[0][1] + du[1][0]);
        const R Sxz = R(0.5) * (du[0][2] + du[2][0]);
        const R Syz = R(0.5) * (du[1][2] + du[2][1]);
        R g[Q];
        const float* st = own_buf + oslot(z) * Q * NT + tid;
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            g[i] = st[i * NT] - R(weight_of(Q, i));
        });
        collide<Q, R, CL, false>(g, drho, ux, uy, uz, Sxx, Syy, Szz, Sxy, Sxz, Syz, omega, tau_hat, nu, cnud, R(0),
                                 R(0), R(0));
        if (own_store) {
            float* dst = fout + (z * plane + own.yr[1] + own.xs[1]);
            static_for<Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                dst[(long long)i * ps] = g[i] + R(weight_of(Q, i));
            });
        }
        drho = dn;
        ux = vnx;
        uy = vny;
        uz = vnz;
    }
}

template <int Q, int CL, int TY>
cudaError_t prepare_async_t()
{
    using Sh = AsyncShape<Q, TY>;
    return cudaFuncSetAttribute(step_kernel_async<Q, CL, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Sh::smem_bytes);
}

template <int Q, int CL, int TY>
cudaError_t launch_step_async_t(const StepArgs& a, int nbatch, cudaStream_t s)
{
    using Sh = AsyncShape<Q, TY>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = prepare_async_t<Q, CL, TY>();
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int tiles = ((a.nx + Sh::TX - 1) / Sh::TX) * ((a.ny + TY - 1) / TY);
    const int chunks = (a.nz + a.zchunk - 1) / a.zchunk;
    dim3 grid(tiles, chunks, nbatch), block(Sh::TX, TY);
    step_kernel_async<Q, CL, TY><<<grid, block, Sh::smem_bytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbmk
