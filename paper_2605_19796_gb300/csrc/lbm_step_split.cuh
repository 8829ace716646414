// Fused step kernel with a split arrive/wait barrier (sm_103a).
//
// Same update, CTA decomposition and population stash as step_kernel
// (lbm_step.cuh).  Two scheduling changes:
//
//  * The threads that own a halo column issue the pulls of their halo cell and
//    of their own cell together, so a plane costs them one load latency, not two.
//  * The per-plane __syncthreads is split.  After publishing the velocities of
//    plane k+1 to the ring a thread ARRIVES on an mbarrier and goes on; it WAITS
//    (for the phase of plane k, completed one iteration earlier by the
//    slowest thread) only right before it reads the neighbour velocities of
//    plane k.  Warps with no halo work therefore run up to a plane ahead
//    instead of idling at a barrier while the halo warps finish.
//
// Ring slots: warps may drift by one plane, so the ring holds five planes.  At
// plane k a thread reads planes k-1, k, k+1 and writes plane k+1 (before its
// arrival); the fastest thread may already write plane k+2 while the slowest
// still reads k-1..k+1, and it cannot write plane k+3 (into the slot of plane
// k-2) before the slowest has arrived for plane k+1, which it does after its
// last read of plane k-2.  (The asynchronous-halo schedule below moves the
// arrival after the reads and needs four planes.)
// (Keeping the z-neighbours in registers instead would allow four slots but
// pushes the register count past the two-CTA budget; eight slots, for a mask
// instead of a modulo, cost more L1 than they save.)
// Plane p arrives on mbarrier (p - z0) & 1, phase ((p - z0) >> 1) & 1; a thread
// arrives for plane p only after it waited for plane p-2 on the same mbarrier,
// so an arrival never lands in an older phase.  Waits are bounded: on timeout
// the step's status flag gets the timeout bit and the thread returns.
#pragma once

#include "lbm_mbarrier.cuh"
#include "lbm_step.cuh"

namespace lbmk {

// c_y, c_z of a population index known only at run time (prefetch loop)
template <int Q>
__device__ __forceinline__ int d27_of_rt(int i)
{
    if constexpr (Q == 27) {
        return i;
    } else {
        int r = 0;
        static_for<Q>([&](auto I) {
            if (i == decltype(I)::value) r = d27_index(Q, decltype(I)::value);
        });
        return r;
    }
}

// Asynchronous 4- or 8-byte global -> shared copy (cp.async, through L1), its
// group commit, and the wait for all of the thread's committed groups (or all
// but the newest).  A copy lands only in the issuing thread's own stash column
// and only that thread reads it after its wait, so no barrier is involved.
template <int N>
__device__ __forceinline__ void cp_async_ca(uint32_t dst, const void* src)
{
    static_assert(N == 4 || N == 8, "cp.async.ca copies 4, 8 or 16 bytes");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(dst), "l"(src), "n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory"); }

// The Q source addresses of pull() (same periodic wrap and halfway bounce-back),
// copied raw (f, not f - w) into the stash column at dst, stride `stride` bytes.
template <int Q, typename S, int BC>
__device__ __forceinline__ void pull_async(const S* __restrict__ fin, long long ps, const Col& col, const int (&zr)[3],
                                           uint32_t dst, uint32_t stride)
{
    static_for<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
        constexpr int io = opp_of(Q, i);
        const S* src;
        if (BC == BC_WALLS_Y && cy != 0) {
            const int row = col.yr[1 - cy];
            src = row >= 0 ? fin + (long long)i * ps + (zr[1 - cz] + row + col.xs[1 - cx])
                           : fin + (long long)io * ps + (zr[1] + col.yr[1] + col.xs[1]);
        } else {
            src = fin + (long long)i * ps + (zr[1 - cz] + col.yr[1 - cy] + col.xs[1 - cx]);
        }
        cp_async_ca<sizeof(S)>(dst + (uint32_t)i * stride, src);
    });
}

// AH (asynchronous halo, with AS): a one-plane halo slot [Q][NB] after the
// stash and four ring planes (the arrival moves after the strain reads,
// below), taken only where two CTAs per SM still fit the 164 KB shared-memory
// carveout (1 KB reserved per CTA), so that L1 keeps about 92 KB; FP64 runs
// one CTA per SM and always fits.  Without AH the ring holds five planes.
template <int Q, typename R, int BC, int TY, bool AS = false>
struct SplitShape {
    using Sh = StepShape<Q, R, BC, TY>;
    static constexpr size_t ring_off = 16;  // two mbarriers
    static constexpr size_t with_halo = ring_off + sizeof(R) * (size_t)(4 * 3 * Sh::RN + 2 * Q * Sh::NT + Q * Sh::NB);
    static constexpr bool AH = AS && (sizeof(R) == 8 || with_halo + 1024 <= 164 * 1024 / 2);
    static constexpr int NSLOT = AH ? 4 : 5;
    static constexpr size_t stash_off = ring_off + sizeof(R) * (size_t)(NSLOT * 3 * Sh::RN);
    static constexpr size_t hstash_off = stash_off + sizeof(R) * (size_t)(2 * Q * Sh::NT);
    static constexpr size_t bytes = hstash_off + (AH ? sizeof(R) * (size_t)(Q * Sh::NB) : 0);
};

// dynamic shared memory of one CTA; the learned closure adds the packed network
// block and the per-warp input/output exchange after the split-barrier layout
template <int Q, typename R, int BC, int TY, bool AS, int CL>
constexpr size_t sb_smem_bytes()
{
    return SplitShape<Q, R, BC, TY, AS>::bytes +
           (CL == CL_LEARNED ? (size_t)(MlpLayout::BYTES + TY * MlpLayout::XCH_BYTES) : 0);
}

// L2PF: at plane k the CTA prefetches into L2 the source rows its pull of
// plane k+2 will read (one 128-byte line per population and row: the tile's
// x-range, for the tile rows and the two halo rows), so that the loads of that
// plane's load phase meet L2 rather than DRAM; no registers or shared memory
// hold the prefetched data and HBM traffic is unchanged.
// AS: the pulls go to shared memory by cp.async, raw, one plane ahead, and no
// registers hold them in flight.  The own column's copies of plane k+2 are
// issued into the stash slot that plane k's populations leave as soon as the
// collision has read them; with AH (see SplitShape) the halo cell's copies of
// plane k+2 go to a one-plane halo slot right after the moments of plane k+1
// have been taken from it (without AH the halo cells pull through registers).
// The copies are waited for at the top of iteration k+1, so their latency runs
// under plane k's collision and stores.  The moments of a plane and the
// collision read the stash and subtract w.  With AH the ring holds four planes:
// a thread arrives for plane k+1 only after its strain reads of plane k's
// stencil (planes k-1..k+1), so the fastest thread, which writes plane p after
// passing the barrier of plane p-2, overwrites the slot of plane p-4 only once
// every thread has read it for the last time (its strain of iteration p-3).
// 32- and 64-bit storage only (the stash holds the stored values as they are).
template <int Q, typename S, int CL, int BC, int TY, bool L2PF = false, bool AS = false>
__global__ void __launch_bounds__(32 * TY, (sizeof(typename StoreTraits<S>::R) == 8 || TY >= 16) ? 1 : 2)
    step_kernel_sb(const StepArgs a)
{
    using R = typename StoreTraits<S>::R;
    using Sh = StepShape<Q, R, BC, TY>;
    using Sp = SplitShape<Q, R, BC, TY, AS>;
    constexpr int TX = Sh::TX, HY = Sh::HY, RX = Sh::RX, RN = Sh::RN, NT = Sh::NT, NB = Sh::NB;
    static_assert(NB <= NT, "every halo cell of the ring needs a thread");
    static_assert(CL != CL_LEARNED || (!AS && sizeof(R) == 4), "the learned closure reads g = f - w from the stash");
    static_assert(Sp::bytes % 16 == 0, "the network block is copied in 16-byte words");
    static_assert(!AS || sizeof(S) == sizeof(R), "the asynchronous stash holds stored values as they are");
    static_assert(!(AS && L2PF), "one load schedule at a time");
    extern __shared__ __align__(16) unsigned char smem_sb[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_sb);
    R* ring = reinterpret_cast<R*>(smem_sb + Sp::ring_off);     // [NSLOT][3][RN]
    R* stash = reinterpret_cast<R*>(smem_sb + Sp::stash_off);   // [2][Q][NT]
    R* hstash = reinterpret_cast<R*>(smem_sb + Sp::hstash_off); // [Q][NB], AS only
    unsigned char* sm_mlp = smem_sb + Sp::bytes;                 // learned closure only
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

    const int gx = x0 + tx, gy = y0 + ty;
    const bool own_store = gx < nx && gy < ny;
    const Col own = make_col<BC>(gx, gy, nx, ny);
    const int own_r = (ty + HY) * RX + (tx + 1);

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

    if (tid == 0) {
        mbar_init(&mbar[0], NT);
        mbar_init(&mbar[1], NT);
    }
    __syncthreads();

    auto zrows = [&](int z, int (&zr)[3]) {
        const int zc = z < 0 ? z + nz : (z >= nz ? z - nz : z);  // z in [-1, nz]
        zr[0] = (zc == 0 ? nz - 1 : zc - 1) * plane;
        zr[1] = zc * plane;
        zr[2] = (zc == nz - 1 ? 0 : zc + 1) * plane;
    };
    auto rslot = [&](int z) { return (int)((unsigned)(z - z0 + 1) % (unsigned)Sp::NSLOT); };
    auto ringp = [&](int s, int c) { return ring + (s * 3 + c) * RN; };
    auto put_u = [&](int z, int r, R vx, R vy, R vz) {
        const int s = rslot(z);
        ringp(s, 0)[r] = vx;
        ringp(s, 1)[r] = vy;
        ringp(s, 2)[r] = vz;
    };
    // stash slot of plane z for the own column (elements of R, stride NT)
    auto stash_col = [&](int z) { return stash + (z & 1) * Q * NT + tid; };
    // populations g = f - w from an asynchronous stash column (stride NS)
    auto stash_g = [&](const R* st, int ns, R (&g)[Q]) {
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            g[i] = st[i * ns] - (R)weight_of(Q, i);
        });
    };
    auto issue_async = [&](int z) {  // own column, plane z -> its stash slot
        if constexpr (AS) {
            int zr[3];
            zrows(z, zr);
            pull_async<Q, S, BC>(fin, ps, own, zr, (uint32_t)__cvta_generic_to_shared(stash_col(z)),
                                 (uint32_t)(NT * sizeof(R)));
        }
    };
    constexpr bool AH = Sp::AH;
    auto issue_halo_async = [&](int z) {  // halo cell (tid < NB), plane z -> the halo slot
        if constexpr (AH) {
            if (tid < NB && hal.valid) {
                int zr[3];
                zrows(z, zr);
                pull_async<Q, S, BC>(fin, ps, hal, zr, (uint32_t)__cvta_generic_to_shared(hstash + tid),
                                     (uint32_t)(NB * sizeof(R)));
            }
        }
    };

    // pull of plane z: own cell (velocity to the ring; populations to the stash
    // when `keep`) and, with `halo`, the thread's halo cell, loads issued together;
    // with AS and `staged`, both are already in the stash and the halo slot, and
    // the halo cell's pull of the next collided plane is issued once the slot
    // has been read
    auto load_plane = [&](int z, bool keep, bool halo, bool staged, R& r, R& vx, R& vy, R& vz) {
        int zr[3];
        zrows(z, zr);
        const bool do_h = halo && tid < NB;
        R t[Q], gh[Q];
        if (own.valid && !(AS && staged)) pull<Q, S, R, BC>(fin, ps, own, zr, t);
        if (do_h && hal.valid && !(AH && staged)) pull<Q, S, R, BC>(fin, ps, hal, zr, gh);
        r = 0;
        vx = vy = vz = 0;
        if (own.valid) {
            if (AS && staged) stash_g(stash_col(z), NT, t);
            moments<Q, R>(t, r, vx, vy, vz, Fx, Fy, Fz);
            if (!(AS && staged) && keep) {
                R* st = stash + (z & 1) * Q * NT + tid;
#pragma unroll
                for (int i = 0; i < Q; ++i) st[i * NT] = t[i];
            }
        }
        put_u(z, own_r, vx, vy, vz);
        if (do_h) {
            R hx = 0, hy = 0, hz = 0;
            if (hal.valid) {
                if (AH && staged) stash_g(hstash + tid, NB, gh);
                R dh;
                moments<Q, R>(gh, dh, hx, hy, hz, Fx, Fy, Fz);
            }
            put_u(z, hal_r, hx, hy, hz);
            if (AH && staged && z + 1 < z1) issue_halo_async(z + 1);  // the halo slot is free again
        }
    };
    auto arrive = [&](int p) { mbar_arrive(&mbar[(p - z0) & 1]); };
    auto wait = [&](int p) { return mbar_wait_bounded(&mbar[(p - z0) & 1], (unsigned)((p - z0) >> 1) & 1u); };

    R drho, ux, uy, uz;  // moments of the own cell at plane z
    {
        if constexpr (AS) {
            if (own.valid) issue_async(z0);
            issue_halo_async(z0);
            cp_async_commit();
            if (own.valid) issue_async(z0 + 1);  // z0 + 1 <= z1
            cp_async_commit();
        }
        R r0, v0x, v0y, v0z;
        load_plane(z0 - 1, false, false, false, r0, v0x, v0y, v0z);  // z-derivative at z0 only: own column
        if constexpr (AS) cp_async_wait<1>();  // plane z0 (own and, with AH, halo) landed
        load_plane(z0, true, true, true, drho, ux, uy, uz);  // with AH: issues the halo pull of z0 + 1
        if constexpr (AH) cp_async_commit();
        arrive(z0);
    }

    // prefetch items of a plane: (population, row) pairs, rows y0-1-c_y .. y0+TY-c_y
    constexpr int kPfRows = TY + 2;
    auto prefetch_plane = [&](int p) {
        int zr[3];
        zrows(p, zr);
        for (int k = tid; k < Q * kPfRows; k += NT) {
            const int i = k / kPfRows, r = k - i * kPfRows;
            const int d = d27_of_rt<Q>(i);
            const int cy = (d / 3) % 3 - 1, cz = d / 9 - 1;
            int y = y0 - 1 - cy + r;
            if (BC == BC_WALLS_Y) {
                if (y < 0 || y >= ny) continue;
            } else {
                y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
            }
            const S* line = fin + (long long)i * ps + (zr[1 - cz] + y * nx + x0);
            asm volatile("prefetch.global.L2 [%0];" ::"l"(line));
        }
    };

    for (int z = z0; z < z1; ++z) {
        if constexpr (L2PF) {
            if (z + 2 <= z1) prefetch_plane(z + 2);
        }
        // ---- plane z+1: own (and, while it will be collided, halo) velocities into the ring
        R rn, vnx, vny, vnz;
        if constexpr (AS) cp_async_wait<0>();  // plane z+1 (issued one iteration ago) landed
        load_plane(z + 1, z + 1 < z1, z + 1 < z1, true, rn, vnx, vny, vnz);
        if (!AH && z + 1 < z1) arrive(z + 1);

        // ---- plane z: wait until every thread has published it, then strain, closure, relaxation
        if (!wait(z)) {
            atomicOr(a.flag, kFlagTimeout);
            if constexpr (AH) {  // the halo copies of plane z+2 may be in flight: let them land first
                cp_async_commit();
                cp_async_wait<0>();
            }
            return;
        }
        R du[3][3] = {};  // du[a][b] = d_a u_b
        if (own.valid) {
            // a non-finite component makes the sum non-finite (the moments are O(1))
            if (own_store && !isfinite(drho + ux + uy + uz)) atomicOr(a.flag, 1u);
            const int sm = rslot(z - 1), s0 = rslot(z), sp = rslot(z + 1);
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
        }
        // with AH the arrival for plane z+1 also says "done reading planes z-1..z+1"
        if (AH && z + 1 < z1) arrive(z + 1);
        if (own.valid) {
            const R Sxx = du[0][0], Syy = du[1][1], Szz = du[2][2];
            const R Sxy = R(0.5) * (du[0][1] + du[1][0]);
            const R Sxz = R(0.5) * (du[0][2] + du[2][0]);
            const R Syz = R(0.5) * (du[1][2] + du[2][1]);
            R g[Q];
            if constexpr (AS) {
                stash_g(stash_col(z), NT, g);
                if (z + 2 <= z1) issue_async(z + 2);  // into the slot just read
            } else {
                const R* st = stash_col(z);
#pragma unroll
                for (int i = 0; i < Q; ++i) g[i] = st[i * NT];
            }
            if constexpr (CL == CL_LEARNED) {
                // every lane of the warp takes part (periodic columns are always valid)
                R msgs[6];
                learned_msgs<Q, R, NT>(stash_col(z), drho, ux, uy, uz, Sxx, Syy, Szz, Sxy, Sxz, Syz, tau_hat, sm_mlp,
                                       sm_xch, tx, msgs);
                collide<Q, R, CL, FORCE>(g, drho, ux, uy, uz, Sxx, Syy, Szz, Sxy, Sxz, Syz, omega, tau_hat, nu, cnud,
                                         Fx, Fy, Fz, msgs);
            } else {
                collide<Q, R, CL, FORCE>(g, drho, ux, uy, uz, Sxx, Syy, Szz, Sxy, Sxz, Syz, omega, tau_hat, nu, cnud,
                                         Fx, Fy, Fz);
            }
            if (own_store) {
                const int cell = z * plane + own.yr[1] + own.xs[1];
                static_for<Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    store_g<S, R>(fout + ((long long)i * ps + cell), g[i], (R)weight_of(Q, i));
                });
            }
        }
        if constexpr (AS) cp_async_commit();
        drho = rn;
        ux = vnx;
        uy = vny;
        uz = vnz;
    }
}

template <int Q, typename S, int CL, int BC, int TY, bool L2PF = false, bool AS = false>
cudaError_t prepare_sb_t()
{
    return cudaFuncSetAttribute(step_kernel_sb<Q, S, CL, BC, TY, L2PF, AS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sb_smem_bytes<Q, typename StoreTraits<S>::R, BC, TY, AS, CL>());
}

template <int Q, typename S, int CL, int BC, int TY, bool L2PF = false, bool AS = false>
cudaError_t launch_sb_t(const StepArgs& a, int nbatch, cudaStream_t s)
{
    using Sh = StepShape<Q, typename StoreTraits<S>::R, BC, TY>;
    if (CL == CL_LEARNED && !a.mlp) return cudaErrorInvalidValue;
    static bool attr_set = false;  // per instantiation; prepare_sb_t sets it ahead of stream capture
    if (!attr_set) {
        cudaError_t e = prepare_sb_t<Q, S, CL, BC, TY, L2PF, AS>();
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int tiles = ((a.nx + Sh::TX - 1) / Sh::TX) * ((a.ny + TY - 1) / TY);
    const int chunks = (a.nz + a.zchunk - 1) / a.zchunk;
    dim3 grid(tiles, chunks, nbatch), block(Sh::TX, TY);
    step_kernel_sb<Q, S, CL, BC, TY, L2PF, AS>
        <<<grid, block, sb_smem_bytes<Q, typename StoreTraits<S>::R, BC, TY, AS, CL>(), s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbmk
