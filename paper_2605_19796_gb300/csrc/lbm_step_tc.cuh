// Fused step of the learned closure with its network on the tcgen05 tensor
// cores (variant 15), periodic boxes, 32 x 4 tiles (sm_103a).
//
// The update is step_kernel's for the learned closure (pull streaming, Eq.
// streaming; moments, App. F.1 step 1; equilibrium, Eq. discrete_equilibrium;
// strain, Eqs. fd and strain_rate_discrete; m_sgs from the network; rate, Eq.
// omega_sgs_operational; KC-MP's two-rate relaxation, App. F.3; store).  The
// mapping onto the GPU differs:
//
//  * The CTA's 128 cells (one per thread, 32 x 4) are the 128 rows of every
//    layer's GEMM (lbm_mlp_tc.cuh): one thread issues a layer's MMAs, all wait
//    on an mbarrier for their completion and then run the epilogue of their
//    own row.
//  * The plane's pulls and moments come first (register pull, as step_kernel),
//    then the network and the collision; the three CTAs per SM (165 registers,
//    59 KB of shared memory, 128 TMEM columns each) overlap one another's
//    pulls and MMA round trips.  Spreading the pulls of the plane after next
//    over the MMA latencies (a third stash slot, the own pulls by cp.async or
//    in registers) was measured slower (7.4 against 9.3 GLUPS at 256^3): the
//    larger shared-memory footprint cut the L1 share that the neighbours'
//    pulls hit.
#pragma once

#include "lbm_mlp_tc.cuh"
#include "lbm_step.cuh"

namespace lbmk {

template <int Q>
struct TcShape {
    static constexpr int TX = 32, TY = 4, NT = 128, HY = 1;
    static constexpr int RX = TX + 2, RY = TY + 2, RN = RX * RY, NB = RN - NT;
    static constexpr size_t ring_bytes = sizeof(float) * 4 * 3 * RN;
    static constexpr size_t stash_bytes = sizeof(float) * 2 * Q * NT;
    static constexpr size_t mlp_off = (ring_bytes + stash_bytes + 127) / 128 * 128;
    static constexpr size_t smem_bytes = mlp_off + MlpTcLayout::BYTES;
    static_assert(smem_bytes <= 74 * 1024, "three CTAs per SM");
};

template <int Q, typename S>
__global__ void __launch_bounds__(128, 3) step_kernel_tc(const StepArgs a)
{
    using R = float;
    static_assert(sizeof(typename StoreTraits<S>::R) == 4, "FP32 arithmetic");
    using Sh = TcShape<Q>;
    constexpr int TX = Sh::TX, RX = Sh::RX, RN = Sh::RN, NT = Sh::NT, NB = Sh::NB, HY = Sh::HY;
    extern __shared__ __align__(16) unsigned char smem_tc[];
    R* ring = reinterpret_cast<R*>(smem_tc);     // [4][3][RN]
    R* stash = ring + 4 * 3 * RN;                // [2][Q][NT]
    unsigned char* sm = smem_tc + Sh::mlp_off;  // network (MlpTcLayout)

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    mlp_tc_repack(static_cast<const unsigned char*>(a.mlp), sm, tid, NT);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int tiles_x = (nx + TX - 1) / TX;
    const int x0 = (int)(blockIdx.x % tiles_x) * TX;
    const int y0 = (int)(blockIdx.x / tiles_x) * 4;
    const int z0 = (int)blockIdx.y * a.zchunk;
    if (z0 >= nz) return;  // uniform over the CTA, before any allocation
    const int z1 = min(nz, z0 + a.zchunk);
    const int box = blockIdx.z;
    const long long ps = a.popstride;
    const int plane = (int)a.plane;
    const S* __restrict__ fin = static_cast<const S*>(a.fin) + (long long)box * a.boxstride;
    S* __restrict__ fout = static_cast<S*>(a.fout) + (long long)box * a.boxstride;

    // TMEM (warp 0 allocates 128 columns), the MMA mbarrier, the re-laid
    // weights made visible to the tensor cores
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + MlpTcLayout::TMEM_SLOT);
    if (ty == 0) {
        tm_alloc(slot, MlpTcLayout::TM_COLS);
        tm_relinquish();
    }
    if (tid == 0) {
        mbar_init(reinterpret_cast<uint64_t*>(sm + MlpTcLayout::MBAR), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    fence_proxy_async_smem();
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tm_base = *slot;
    const uint32_t tm_row = tm_base + ((uint32_t)(32 * ty) << 16);
    unsigned phase = 0;
    bool ok = true;

    const double nu_d = a.box_nu[box];
    const R nu = (R)nu_d;
    const R tau_hat = (R)(nu_d / kTheta + 0.5);
    const R omega = (R)(1.0 / (nu_d / kTheta + 0.5));
    const R cnud = (R)a.cnu_delta;

    // own column (lanes beyond nx and rows beyond ny wrap; they compute but do not store)
    const int gx = x0 + tx, gy = y0 + ty;
    const bool own_store = gx < nx && gy < ny;
    const Col own = make_col<BC_PERIODIC>(gx, gy, nx, ny);
    const int own_r = (ty + HY) * RX + (tx + 1);
    // halo column: rows y0 - 1 and y0 + 4, then the columns x0 - 1 and x0 + 32
    // (the corners are never read)
    Col hal = own;
    int hal_r = -1;
    if (tid < NB) {
        int lx, ly, b = tid;
        if (b < RX) {
            lx = b - 1;
            ly = -1;
        } else if ((b -= RX) < RX) {
            lx = b - 1;
            ly = 4;
        } else {
            b -= RX;
            lx = (b < 4) ? -1 : TX;
            ly = b % 4;
        }
        hal = make_col<BC_PERIODIC>(x0 + lx, y0 + ly, nx, ny);
        hal_r = (ly + HY) * RX + (lx + 1);
        if ((lx == -1 || lx == TX) && (ly < 0 || ly >= 4)) hal.valid = false;
    }

    auto zrows = [&](int z, int (&zr)[3]) {
        const int zc = z < 0 ? z + nz : (z >= nz ? z - nz : z);  // z in [-1, nz]
        zr[0] = (zc == 0 ? nz - 1 : zc - 1) * plane;
        zr[1] = zc * plane;
        zr[2] = (zc == nz - 1 ? 0 : zc + 1) * plane;
    };
    auto rslot = [&](int z) { return (z - z0 + 1) & 3; };  // z >= z0 - 1
    auto ringp = [&](int s, int c) { return ring + (s * 3 + c) * RN; };
    auto put_u = [&](int z, int r, R vx, R vy, R vz) {
        const int s = rslot(z);
        ringp(s, 0)[r] = vx;
        ringp(s, 1)[r] = vy;
        ringp(s, 2)[r] = vz;
    };
    auto halo_plane = [&](int z) {
        if (tid < NB) {
            R vx = 0, vy = 0, vz = 0;
            if (hal.valid) {
                int zr[3];
                zrows(z, zr);
                R gh[Q];
                pull<Q, S, R, BC_PERIODIC>(fin, ps, hal, zr, gh);
                R dh;
                moments<Q, R>(gh, dh, vx, vy, vz, R(0), R(0), R(0));
            }
            put_u(z, hal_r, vx, vy, vz);
        }
    };
    // own cell at plane z: velocity into the ring; with `keep` the populations
    // into the stash slot (z & 1)
    auto own_plane = [&](int z, bool keep, R& r, R& vx, R& vy, R& vz) {
        int zr[3];
        zrows(z, zr);
        R t[Q];
        pull<Q, S, R, BC_PERIODIC>(fin, ps, own, zr, t);
        moments<Q, R>(t, r, vx, vy, vz, R(0), R(0), R(0));
        if (keep) {
            R* st = stash + (z & 1) * Q * NT + tid;
#pragma unroll
            for (int i = 0; i < Q; ++i) st[i * NT] = t[i];
        }
        put_u(z, own_r, vx, vy, vz);
    };

    R d0, u0x, u0y, u0z;  // moments of the own cell at plane z
    {
        R r, vx, vy, vz;
        own_plane(z0 - 1, false, r, vx, vy, vz);
        halo_plane(z0 - 1);
        halo_plane(z0);
        own_plane(z0, true, d0, u0x, u0y, u0z);
    }
    __syncthreads();

    using T = MlpTcLayout;
    for (int z = z0; z < z1; ++z) {
        // ---- plane z+1: halo and own velocities into the ring
        R d1, u1x, u1y, u1z;
        halo_plane(z + 1);
        own_plane(z + 1, z + 1 < z1, d1, u1x, u1y, u1z);
        __syncthreads();

        // ---- plane z: strain, network inputs; every thread takes part in the
        // CTA-wide network
        if (own_store && !isfinite(d0 + u0x + u0y + u0z)) atomicOr(a.flag, kFlagNonfinite);
        const R* st = stash + (z & 1) * Q * NT + tid;
        R Sxx, Syy, Szz, Sxy, Sxz, Syz;
        uint32_t xin[8];
        {
            const int sm_ = rslot(z - 1), s0 = rslot(z), sp = rslot(z + 1);
            R du[3][3];
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const R* r0 = ringp(s0, b);
                du[0][b] = R(0.5) * (r0[own_r + 1] - r0[own_r - 1]);
                du[1][b] = R(0.5) * (r0[own_r + RX] - r0[own_r - RX]);
                du[2][b] = R(0.5) * (ringp(sp, b)[own_r] - ringp(sm_, b)[own_r]);
            }
            Sxx = du[0][0];
            Syy = du[1][1];
            Szz = du[2][2];
            Sxy = R(0.5) * (du[0][1] + du[1][0]);
            Sxz = R(0.5) * (du[0][2] + du[2][0]);
            Syz = R(0.5) * (du[1][2] + du[2][1]);
            learned_inputs<Q, R, NT>(st, d0, u0x, u0y, u0z, Sxx, Syy, Szz, Sxy, Sxz, Syz, tau_hat,
                                     reinterpret_cast<const float*>(sm + T::XMU),
                                     reinterpret_cast<const float*>(sm + T::XIS), xin);
        }
        float y[6];
        ok = mlp_cta_forward_tc(sm, tm_base, tm_row, xin, y, phase, tid, ok);
        if (!__syncthreads_and(ok)) break;  // CTA-uniform
        // ---- plane z: collision with the network's m_sgs, store
        {
            const float* ymu = reinterpret_cast<const float*>(sm + T::YMU);
            const float* ysd = reinterpret_cast<const float*>(sm + T::YSD);
            const R rho = R(1) + d0;
            R msgs[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) msgs[q] = rho * (R)(y[q] * ysd[q] + ymu[q]);
            R g[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) g[i] = st[i * NT];
            collide<Q, R, CL_LEARNED, false>(g, d0, u0x, u0y, u0z, Sxx, Syy, Szz, Sxy, Sxz, Syz, omega, tau_hat, nu,
                                             cnud, R(0), R(0), R(0), msgs);
            if (own_store) {
                S* dst = fout + (z * plane + own.yr[1] + own.xs[1]);
                static_for<Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    store_g<S, R>(dst + (long long)i * ps, g[i], (R)weight_of(Q, i));
                });
            }
        }
        d0 = d1;
        u0x = u1x;
        u0y = u1y;
        u0z = u1z;
    }
    if (!ok && tid == 0) atomicOr(a.flag, kFlagTimeout);
    // every TMEM access of the CTA has completed before warp 0 frees the columns
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (ty == 0) tm_dealloc(tm_base, MlpTcLayout::TM_COLS);
}

template <int Q, typename S>
cudaError_t prepare_tc_t()
{
    return cudaFuncSetAttribute(step_kernel_tc<Q, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TcShape<Q>::smem_bytes);
}

template <int Q, typename S>
cudaError_t launch_tc_t(const StepArgs& a, int nbatch, cudaStream_t s)
{
    static bool attr_set = false;  // per instantiation; prepare_tc_t sets it ahead of stream capture
    if (!attr_set) {
        cudaError_t e = prepare_tc_t<Q, S>();
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (!a.mlp) return cudaErrorInvalidValue;
    const int tiles = ((a.nx + 31) / 32) * ((a.ny + 3) / 4);
    const int chunks = (a.nz + a.zchunk - 1) / a.zchunk;
    dim3 grid(tiles, chunks, nbatch), block(32, 4);
    step_kernel_tc<Q, S><<<grid, block, TcShape<Q>::smem_bytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbmk
