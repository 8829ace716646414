// Fused step kernel, register-prefetch pipeline (sm_103a).
//
// Same update, CTA decomposition, velocity ring and population stash as
// step_kernel (lbm_step.cuh); only the schedule of the global loads differs.
// In step_kernel every thread pulls plane k+1 and uses the loaded values at
// once, so each plane's load latency is exposed and the warps of a CTA reach
// the per-plane barrier in lock step.  Here the own-cell pull runs two planes
// ahead: at plane k a thread issues the Q loads of plane k+2 into registers,
// then computes the halo velocities of plane k+1 and collides plane k, and
// only then consumes the loads (moments of plane k+2 into the ring, the
// populations into the stash).  The loads are in flight during the collision.
//
// Ring slots (four, single barrier per plane): at plane k the CTA reads the
// velocities of planes k-1, k, k+1 and writes plane k+2 (own cells) and plane
// k+1 (halo cells, positions the plane-k reads do not touch); k+2 and k-2
// share a slot, and plane k-2 was last read before the previous barrier.
// Stash slots (two, thread-private): plane k+2 overwrites plane k after the
// collision of plane k has read it.
#pragma once

#include "lbm_step.cuh"

namespace lbmk {

template <int Q, typename S, int CL, int BC, int TY>
__global__ void __launch_bounds__(32 * TY, (sizeof(typename StoreTraits<S>::R) == 8 || TY >= 16) ? 1 : 2)
    step_kernel_pf(const StepArgs a)
{
    using R = typename StoreTraits<S>::R;
    using Sh = StepShape<Q, R, BC, TY>;
    constexpr int TX = Sh::TX, HY = Sh::HY, RX = Sh::RX, RN = Sh::RN, NT = Sh::NT, NB = Sh::NB;
    static_assert(NB <= NT, "every halo cell of the ring needs a thread");
    static_assert(CL != CL_LEARNED, "the learned closure runs in step_kernel");
    extern __shared__ __align__(16) unsigned char smem_pf[];
    R* ring = reinterpret_cast<R*>(smem_pf);  // [4][3][RN]
    R* stash = ring + 4 * 3 * RN;             // [2][Q][NT]

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

    const int gx = x0 + tx, gy = y0 + ty;
    const bool own_store = gx < nx && gy < ny;
    const Col own = make_col<BC>(gx, gy, nx, ny);
    const int own_r = (ty + HY) * RX + (tx + 1);

    Col hal = own;
    int hal_r = -1;
    if (tid < NB) {
        int lx, ly;
        int b = tid;
        if (b < HY * RX) {
            lx = b % RX - 1;
            ly = b / RX - HY;
        } else if ((b -= HY * RX) < HY * RX) {
            lx = b % RX - 1;
            ly = TY + b / RX;
        } else {
            b -= HY * RX;
            lx = (b < TY) ? -1 : TX;
            ly = b % TY;
        }
        hal = make_col<BC>(x0 + lx, y0 + ly, nx, ny);
        hal_r = (ly + HY) * RX + (lx + 1);
    }

    auto zrows = [&](int z, int (&zr)[3]) {
        const int zc = wrapi(z, nz);
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
    auto stash_put = [&](int z, const R (&t)[Q]) {
        R* st = stash + (z & 1) * Q * NT + tid;
#pragma unroll
        for (int i = 0; i < Q; ++i) st[i * NT] = t[i];
    };

    // ---- prologue: planes z0-1 (velocity), z0 and z0+1 (velocity, stash), halo of z0
    R drho = 0, ux = 0, uy = 0, uz = 0;  // moments of the own cell at plane z
    R dn = 0, vnx = 0, vny = 0, vnz = 0; // ... at plane z+1
    {
        int zr[3];
        R t[Q];
        R r0 = 0, v0x = 0, v0y = 0, v0z = 0;
        if (own.valid) {
            zrows(z0 - 1, zr);
            pull<Q, S, R, BC>(fin, ps, own, zr, t);
            moments<Q, R>(t, r0, v0x, v0y, v0z, Fx, Fy, Fz);
        }
        put_u(z0 - 1, own_r, v0x, v0y, v0z);
        if (tid < NB) {
            R vx = 0, vy = 0, vz = 0;
            if (hal.valid) {
                zrows(z0, zr);
                R gh[Q];
                pull<Q, S, R, BC>(fin, ps, hal, zr, gh);
                R dh;
                moments<Q, R>(gh, dh, vx, vy, vz, Fx, Fy, Fz);
            }
            put_u(z0, hal_r, vx, vy, vz);
        }
        if (own.valid) {
            zrows(z0, zr);
            pull<Q, S, R, BC>(fin, ps, own, zr, t);
            moments<Q, R>(t, drho, ux, uy, uz, Fx, Fy, Fz);
            stash_put(z0, t);
        }
        put_u(z0, own_r, ux, uy, uz);
        if (own.valid) {
            zrows(z0 + 1, zr);
            pull<Q, S, R, BC>(fin, ps, own, zr, t);
            moments<Q, R>(t, dn, vnx, vny, vnz, Fx, Fy, Fz);
            if (z0 + 1 < z1) stash_put(z0 + 1, t);
        }
        put_u(z0 + 1, own_r, vnx, vny, vnz);
    }
    __syncthreads();

    for (int z = z0; z < z1; ++z) {
        // ---- issue: halo pull of plane z+1, own pull of plane z+2 (consumed after the collision)
        const bool do_halo = tid < NB && z + 1 < z1;
        const bool do_pf = own.valid && z + 2 <= z1;
        R gh[Q];
        if (do_halo && hal.valid) {
            int zr[3];
            zrows(z + 1, zr);
            pull<Q, S, R, BC>(fin, ps, hal, zr, gh);
        }
        R pf[Q];
        if (do_pf) {
            int zr[3];
            zrows(z + 2, zr);
            pull<Q, S, R, BC>(fin, ps, own, zr, pf);
        }
        // ---- halo velocities of plane z+1
        if (do_halo) {
            R vx = 0, vy = 0, vz = 0;
            if (hal.valid) {
                R dh;
                moments<Q, R>(gh, dh, vx, vy, vz, Fx, Fy, Fz);
            }
            put_u(z + 1, hal_r, vx, vy, vz);
        }

        // ---- plane z: strain from the ring, closure, relaxation, store
        if (own.valid) {
            if (own_store && !(isfinite(drho) && isfinite(ux) && isfinite(uy) && isfinite(uz))) atomicOr(a.flag, 1u);
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
#pragma unroll
            for (int i = 0; i < Q; ++i) g[i] = st[i * NT];
            collide<Q, R, CL, FORCE>(g, drho, ux, uy, uz, Sxx, Syy, Szz, Sxy, Sxz, Syz, omega, tau_hat, nu, cnud, Fx,
                                     Fy, Fz);
            if (own_store) {
                S* dst = fout + (z * plane + own.yr[1] + own.xs[1]);
                static_for<Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    store_g<S, R>(dst + (long long)i * ps, g[i], (R)weight_of(Q, i));
                });
            }
        }

        // ---- consume the prefetch: velocity of plane z+2, populations into the freed stash slot
        R d2 = 0, w2x = 0, w2y = 0, w2z = 0;
        if (do_pf) {
            moments<Q, R>(pf, d2, w2x, w2y, w2z, Fx, Fy, Fz);
            if (z + 2 < z1) stash_put(z + 2, pf);
        }
        if (z + 2 <= z1) put_u(z + 2, own_r, w2x, w2y, w2z);
        __syncthreads();
        drho = dn;
        ux = vnx;
        uy = vny;
        uz = vnz;
        dn = d2;
        vnx = w2x;
        vny = w2y;
        vnz = w2z;
    }
}

template <int Q, typename S, int CL, int BC, int TY>
cudaError_t prepare_pf_t()
{
    return cudaFuncSetAttribute(step_kernel_pf<Q, S, CL, BC, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)StepShape<Q, typename StoreTraits<S>::R, BC, TY>::base_bytes);
}

template <int Q, typename S, int CL, int BC, int TY>
cudaError_t launch_pf_t(const StepArgs& a, int nbatch, cudaStream_t s)
{
    using Sh = StepShape<Q, typename StoreTraits<S>::R, BC, TY>;
    static bool attr_set = false;  // per instantiation; prepare_pf_t sets it ahead of stream capture
    if (!attr_set) {
        cudaError_t e = prepare_pf_t<Q, S, CL, BC, TY>();
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int tiles = ((a.nx + Sh::TX - 1) / Sh::TX) * ((a.ny + TY - 1) / TY);
    const int chunks = (a.nz + a.zchunk - 1) / a.zchunk;
    dim3 grid(tiles, chunks, nbatch), block(Sh::TX, TY);
    step_kernel_pf<Q, S, CL, BC, TY><<<grid, block, Sh::base_bytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbmk
