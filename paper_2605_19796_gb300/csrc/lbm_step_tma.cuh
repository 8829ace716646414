// Fused step kernel with TMA-staged populations (sm_103a), FP32 storage,
// periodic boxes whose nx is a multiple of 32 and ny a multiple of TY.
//
// Same update and CTA decomposition as step_kernel (lbm_step.cuh): a CTA owns
// a 32 x TY column of cells and marches it through a chunk of z-planes, the
// strain's neighbour velocities coming from a shared-memory ring.  The pull
// is done by the Tensor Memory Accelerator: for plane p and population i one
// cp.async.bulk.tensor copies the box
//     x in [x0 - 4, x0 + 36)   (40 floats, 16-byte aligned start)
//     y in [y0 - 1 - c_iy, y0 + TY + 1 - c_iy)
//     z  = p - c_iz (periodic), population i of this box
// into a shared-memory stage, so that the streamed population i of ring cell
// (lx, ly) (lx in [-1, 32], ly in [-1, TY]) is stage[i][ly + 1][lx + 4 - c_ix]:
// the pull becomes an index shift and the halo costs no extra instructions.
// Coordinates that fall outside the box are filled with zeros by the TMA unit;
// CTAs on a periodic edge overwrite the entries they need with plain loads of
// the wrapped cells ("patch") before use.
//
// Pipeline: NS >= 3 stages, each completed by an mbarrier (expect_tx bytes); plane
// p lives in stage (p - z0 + 1) mod NS.  Per plane z:
//   wait for plane z+1 (bounded poll; a timeout sets LBM_ERR_TIMEOUT's flag bit
//   and the CTA drains its copies and leaves), patch edges, moments of plane
//   z+1 -> velocity ring, barrier, issue the copies of plane z+NS-1 into the
//   stage of plane z-1 (free since the barrier), collide plane z from its stage.
#pragma once

#include <cuda.h>

#include "lbm_mbarrier.cuh"
#include "lbm_step.cuh"

namespace lbmk {

__device__ __forceinline__ void tma_load_4d(void* smem_dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            uint64_t* bar)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(d),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(b)
        : "memory");
}

template <int Q, int TY, int NS>
struct TmaShape {
    static constexpr int TX = 32;
    static constexpr int BW = 40;               // box width (floats)
    static constexpr int BH = TY + 2;           // box height (rows)
    static constexpr int BOX = BW * BH;         // floats per population box
    static constexpr int BOXP = (BOX + 31) / 32 * 32;  // padded to 128 bytes
    static constexpr int STAGE = Q * BOXP;      // floats per stage
    static constexpr int RX = TX + 2;
    static constexpr int RN = RX * (TY + 2);
    static constexpr int NT = TX * TY;
    static constexpr int NB = RN - NT;
    static constexpr size_t smem_bytes = 4 * (size_t)(NS * STAGE + 4 * 3 * RN) + 8 * NS + 16 + 128;
};

template <int Q, int CL, int TY, int NS>
__global__ void __launch_bounds__(32 * TY, 1)
    step_kernel_tma(const __grid_constant__ CUtensorMap tmap, const StepArgs a)
{
    using R = float;
    using Sh = TmaShape<Q, TY, NS>;
    constexpr int TX = Sh::TX, BW = Sh::BW, BH = Sh::BH, BOXP = Sh::BOXP, STAGE = Sh::STAGE;
    constexpr int RX = Sh::RX, RN = Sh::RN, NT = Sh::NT, NB = Sh::NB;
    static_assert(NB <= NT, "every halo cell of the ring needs a thread");
    static_assert(NS >= 3, "plane z+1 must be in flight before plane z+NS-1 is issued");
    extern __shared__ __align__(128) unsigned char smem_tma[];
    // 128-byte aligned stages first, then the ring and the barriers
    float* stages = reinterpret_cast<float*>(((uintptr_t)smem_tma + 127) & ~(uintptr_t)127);
    float* ring = stages + NS * STAGE;                                   // [4][3][RN]
    uint64_t* mbar = reinterpret_cast<uint64_t*>(ring + 4 * 3 * RN);     // [NS]

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int tiles_x = nx / TX;
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
    const bool edge_x = (x0 == 0) || (x0 + TX == nx);
    const bool edge_y = (y0 == 0) || (y0 + TY == ny);

    const double nu_d = a.box_nu[box];
    const R nu = (R)nu_d;
    const R tau_hat = (R)(nu_d / kTheta + 0.5);
    const R omega = (R)(1.0 / (nu_d / kTheta + 0.5));
    const R cnud = (R)a.cnu_delta;

    const int own_r = (ty + 1) * RX + (tx + 1);
    const int own_b = (ty + 1) * BW + (tx + 4);  // stage index of own cell for c_x = 0
    int hal_r = 0, hal_b = 0;
    if (tid < NB) {
        int lx, ly, b = tid;
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
        hal_r = (ly + 1) * RX + (lx + 1);
        hal_b = (ly + 1) * BW + (lx + 4);
    }

    auto sidx = [&](int p) { return (p - z0 + 1) % NS; };
    auto sparity = [&](int p) { return (unsigned)(((p - z0 + 1) / NS) & 1); };
    auto rslot = [&](int p) { return (p - z0 + 1) & 3; };

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&mbar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();

    // thread 0: the Q box copies of plane p into its stage
    auto issue = [&](int p) {
        const int s = sidx(p);
        float* st = stages + s * STAGE;
        mbar_expect_tx(&mbar[s], (unsigned)(Q * Sh::BOX * 4));
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cy = cy_of(Q, i), cz = cz_of(Q, i);
            tma_load_4d(st + i * BOXP, &tmap, x0 - 4, y0 - 1 - cy, wrapi(p - cz, nz), box * Q + i, &mbar[s]);
        });
    };

    // replace the zero-filled out-of-range entries of plane p's boxes by the
    // periodic images (edge CTAs only; uniform per CTA)
    auto patch = [&](int p) {
        float* st = stages + sidx(p) * STAGE;
        if (edge_x) {
            // columns 2, 3 (x0 = 0) and 36, 37 (x0 + 32 = nx): 4 per row over all rows
            for (int k = tid; k < Q * BH * 4; k += NT) {
                const int i = k / (BH * 4), rem = k % (BH * 4), r = rem / 4, cc = rem % 4;
                const int c = cc < 2 ? 2 + cc : 34 + cc;
                const int xs = x0 - 4 + c;
                if (xs >= 0 && xs < nx) continue;
                const int cyi = cy_of(Q, i), czi = cz_of(Q, i);
                const int ys = wrapi(y0 - 1 - cyi + r, ny), zs = wrapi(p - czi, nz);
                st[i * BOXP + r * BW + c] = __ldg(fin + (long long)i * ps + ((long long)zs * plane + ys * nx + wrapi(xs, nx)));
            }
        }
        if (edge_y) {
            // rows whose y lies outside [0, ny): columns 2..37
            for (int k = tid; k < Q * BH * 36; k += NT) {
                const int i = k / (BH * 36), rem = k % (BH * 36), r = rem / 36, c = 2 + rem % 36;
                const int cyi = cy_of(Q, i);
                const int ysr = y0 - 1 - cyi + r;
                if (ysr >= 0 && ysr < ny) continue;
                const int czi = cz_of(Q, i);
                const int ys = wrapi(ysr, ny), zs = wrapi(p - czi, nz), xs = wrapi(x0 - 4 + c, nx);
                st[i * BOXP + r * BW + c] = __ldg(fin + (long long)i * ps + ((long long)zs * plane + ys * nx + xs));
            }
        }
    };

    auto put_u = [&](int p, int r, R vx, R vy, R vz) {
        float* rg = ring + rslot(p) * 3 * RN;
        rg[r] = vx;
        rg[RN + r] = vy;
        rg[2 * RN + r] = vz;
    };
    // moments of plane p from its stage: own cell (returned) and halo cell -> ring
    auto plane_moments = [&](int p, R& d, R& vx, R& vy, R& vz) {
        const float* st = stages + sidx(p) * STAGE;
        R g[Q];
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            g[i] = st[i * BOXP + own_b - cx_of(Q, i)] - R(weight_of(Q, i));
        });
        moments<Q, R>(g, d, vx, vy, vz, R(0), R(0), R(0));
        put_u(p, own_r, vx, vy, vz);
        if (tid < NB) {
            R gh[Q];
            static_for<Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                gh[i] = st[i * BOXP + hal_b - cx_of(Q, i)] - R(weight_of(Q, i));
            });
            R dh, hx, hy, hz;
            moments<Q, R>(gh, dh, hx, hy, hz, R(0), R(0), R(0));
            put_u(p, hal_r, hx, hy, hz);
        }
    };

    // bounded wait for plane p (all threads poll); returns false on a timeout
    // after draining this CTA's copies in flight
    auto wait_plane = [&](int p, int last_issued) -> bool {
        bool ok = mbar_wait_bounded(&mbar[sidx(p)], sparity(p));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(a.flag, kFlagTimeout);
                for (int q = p; q <= last_issued; ++q) mbar_wait_bounded(&mbar[sidx(q)], sparity(q));
            }
            __syncthreads();
            return false;
        }
        if (edge_x || edge_y) {
            patch(p);
            __syncthreads();
        }
        return true;
    };

    int last = z0 - 1;  // highest plane whose copies are issued
    if (tid == 0)
        for (int p = z0 - 1; p <= min(z1, z0 + NS - 2); ++p) issue(p);
    last = min(z1, z0 + NS - 2);

    R drho, ux, uy, uz;
    if (!wait_plane(z0 - 1, last)) return;
    {
        R d0, v0x, v0y, v0z;
        plane_moments(z0 - 1, d0, v0x, v0y, v0z);
    }
    if (!wait_plane(z0, last)) return;
    plane_moments(z0, drho, ux, uy, uz);

    for (int z = z0; z < z1; ++z) {
        if (!wait_plane(z + 1, last)) return;
        R dn, vnx, vny, vnz;
        plane_moments(z + 1, dn, vnx, vny, vnz);
        __syncthreads();  // ring of plane z+1 complete; every read of plane z-1's stage is done
        const int nxt = z + NS - 1;
        if (nxt <= z1) {
            if (tid == 0) issue(nxt);
            last = nxt;
        }

        if (!(isfinite(drho) && isfinite(ux) && isfinite(uy) && isfinite(uz))) atomicOr(a.flag, kFlagNonfinite);
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
        const float* st = stages + sidx(z) * STAGE;
        R g[Q];
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            g[i] = st[i * BOXP + own_b - cx_of(Q, i)] - R(weight_of(Q, i));
        });
        collide<Q, R, CL, false>(g, drho, ux, uy, uz, Sxx, Syy, Szz, Sxy, Sxz, Syz, omega, tau_hat, nu, cnud, R(0),
                                 R(0), R(0));
        float* dst = fout + ((long long)z * plane + (y0 + ty) * nx + (x0 + tx));
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            dst[(long long)i * ps] = g[i] + R(weight_of(Q, i));
        });
        drho = dn;
        ux = vnx;
        uy = vny;
        uz = vnz;
    }
}

template <int Q, int CL, int TY, int NS>
cudaError_t prepare_tma_t()
{
    using Sh = TmaShape<Q, TY, NS>;
    return cudaFuncSetAttribute(step_kernel_tma<Q, CL, TY, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Sh::smem_bytes);
}

template <int Q, int CL, int TY, int NS>
cudaError_t launch_step_tma_t(const StepArgs& a, int nbatch, cudaStream_t s)
{
    using Sh = TmaShape<Q, TY, NS>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = prepare_tma_t<Q, CL, TY, NS>();
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int tiles = (a.nx / Sh::TX) * (a.ny / TY);
    const int chunks = (a.nz + a.zchunk - 1) / a.zchunk;
    dim3 grid(tiles, chunks, nbatch), block(Sh::TX, TY);
    if (!a.tmap_in) return cudaErrorInvalidValue;
    step_kernel_tma<Q, CL, TY, NS><<<grid, block, Sh::smem_bytes, s>>>(*static_cast<const CUtensorMap*>(a.tmap_in), a);
    return cudaGetLastError();
}

}  // namespace lbmk
