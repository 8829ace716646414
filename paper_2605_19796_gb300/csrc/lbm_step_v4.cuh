// Fused step kernel with four cells per thread, vector access and a tensor-memory
// stash (sm_103a).
//
// Same update as step_kernel (lbm_step.cuh): pull streaming (Eq. streaming),
// moments (App. F.1 step 1), equilibrium (Eq. discrete_equilibrium), strain
// (Eqs. fd, strain_rate_discrete), closure, rate (Eq. omega_sgs_operational)
// and two-rate relaxation (App. F.2, F.3; KC-RR, App. F.4), store.  D3Q27 and
// D3Q19, periodic boxes and channels with walls in y, nx a multiple of 8.  The
// mapping onto the GPU differs:
//
//  * Each thread owns four consecutive x-cells of one row.  The source row of a
//    population is read with ONE aligned vector load per thread (16 bytes for
//    FP32 storage, 8 for FP16/BF16): for c_x = 0 the four values are the four
//    cells' populations; for c_x = +1 / -1 they are shifted by one cell, and the
//    value that crosses into the neighbouring thread's cells comes from that
//    lane by a warp shuffle (at the ends of a tile row, from one scalar load of
//    the edge lane).  Post-collision values leave as vector stores of the same
//    width.  Address arithmetic, loop control and synchronisation are shared by
//    four cells.
//  * A CTA of 8 warps covers a TX x TY tile (128 x 8: one row per warp, or
//    64 x 16: two rows per warp) and marches a chunk of z-planes; one CTA per SM.
//  * The streamed populations of a plane wait between their pull (which yields
//    the velocity the neighbours' strain needs) and their collision one plane
//    later in tensor memory (TMEM): two slots of 27 x 4 FP32 values per
//    thread, column 4 i + c of a slot holding population i of cell c.  A CTA
//    allocates all 512 columns; the two warps that share a lane quarter take
//    256 each.  The stash thus needs neither shared memory nor registers, and a
//    1024-cell tile (whose halo costs a quarter or less of its own pulls) fits
//    on one SM.
//  * Velocities go through a ring of planes in shared memory: the own cells'
//    and the halo cells' (rows y0 - 1 and y0 + TY, columns x0 - 1 and x0 + TX,
//    one cell per thread from the staged values).  With three slots the
//    z-neighbours of the own cells stay in registers; a thread that writes
//    plane p has passed the barrier of plane p-1 (every thread has published
//    it, after its strain reads of plane p-2), so nobody reads the slot of
//    plane p-3 any more.  With four (v4_ring4: the TMA-staged KC kernels) the
//    strain of plane z reads the slots of planes z - 1, z and z + 1 (the
//    z-neighbours only at the thread's own cells, which it wrote itself),
//    every thread has done its strain reads of plane p-3 when plane p is
//    written, and the 36 registers no longer carried from plane to plane let
//    the periodic box's collision load its TMEM populations one triple ahead,
//    and the walls' TMA kernel run without spills.  Measured (512^3 FP32,
//    GLUPS): KC-MP 26.55 against 26.4, KC-RB raw 27.3 against 26.8; BGK (29.3
//    against 29.7) and the cp.async-staged kernels (FP32 24.0 against 24.6,
//    FP16 28.5 against 29.4, the 64^3 ensemble 21.7 against 22.6) keep three.
//  * The collision relaxes the four cells together, one (c_y, c_z) population
//    triple at a time, in the common form g' = a g + w (b (P - 1) + c0 + D H)
//    of collide() with P - 1 = e_x (1 + Y) + Y, Y = e_y + e_z + e_y e_z, and
//    the quadratic form H split into its (c_y, c_z) part and the c_x terms, so
//    that each population's four results form one vector store.  For FP32
//    storage the "+ w" of the stored f = g' + w comes last, after g' is
//    rounded on its own small scale, so that the mass does not drift.  D3Q19
//    takes its Hermite equilibrium along a triple (V4Cell), and KC-RR collides
//    one cell at a time from the TMEM stash (its Hermite-space collision needs
//    a cell's 27 populations together) before the same vector stores.
#pragma once

#include <cuda.h>

#include <type_traits>

#include "lbm_mbarrier.cuh"
#include "lbm_step.cuh"
#include "lbm_step_split.cuh"
#include "lbm_tmem.cuh"

namespace lbmk {

// ------------------------------------------------------- vector global access

// four consecutive stored values as FP32 (16-bit storage: the stored g = f - w)
__device__ __forceinline__ float4 v4_load(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 v4_load(const __half* p)
{
    const uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&r.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&r.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 v4_load(const __nv_bfloat16* p)
{
    const uint2 r = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float v1_load(const float* p) { return __ldg(p); }
__device__ __forceinline__ float v1_load(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float v1_load(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }

__device__ __forceinline__ void v4_store(float* p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void v4_store(__half* p, float a, float b, float c, float d)
{
    const __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(c, d);
    *reinterpret_cast<uint2*>(p) = make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
}
__device__ __forceinline__ void v4_store(__nv_bfloat16* p, float a, float b, float c, float d)
{
    const __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
    *reinterpret_cast<uint2*>(p) = make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
}

// ------------------------------------------------------------------ shape

// LPR lanes per tile row: 32 (tiles 128 x 8, one row per warp) or 16 (tiles
// 64 x 16, two rows per warp); 8 warps, one CTA per SM.
// TMAS: the interior of the staged rows (x0 .. x0 + TX - 1) is copied by the
// Tensor Memory Accelerator, one cp.async.bulk.tensor per population and plane
// into [27][RY][TX], and only the x-edge chunks (x0 - 4 .. x0 - 1 and x0 + TX ..
// x0 + TX + 3 of every staged row) by cp.async, into [27][RY][8].
// WALLS: a buffer [2][9][TX] for the bounce-back values of the wall rows (the
// cells' own opposite populations, copied with the plane's staging: by
// cp.async, or with TMAS one row box per population and wall by the TMA).
// four ring slots (the z-neighbours read from the ring; in the periodic box
// also the TMEM loads one triple ahead): the TMA-staged kernels with the KC
// closures
__host__ __device__ constexpr bool v4_ring4(bool tmas, int cl, int bc)
{
    return tmas && cl != CL_BGK && cl != CL_LEARNED;
}

template <int LPR, typename S, bool LEARNED = false, bool TMAS = false, bool WALLS = false, bool RZ4 = false>
struct V4Shape {
    static constexpr int NT = 256;
    static constexpr int RPW = 32 / LPR;  // tile rows per warp
    static constexpr int TX = 4 * LPR;
    static constexpr int TY = 8 * RPW;
    static constexpr int RY = TY + 2;      // ring and staged rows: y0 - 1 .. y0 + TY
    static constexpr int RP = TX + 8;      // ring and staging pitch: x0 - 4 .. x0 + TX + 3, own cells at 4 .. TX + 3
    static constexpr int NSLOT = RZ4 ? 4 : 3;
    static_assert(!RZ4 || !LEARNED, "four ring slots: analytic closures");
    static constexpr int NB = 2 * TX + 2 * TY;     // halo cells of a ring plane (no corners)
    static constexpr int NCH = TX / 4;             // 4-cell chunks of a row
    // staged chunks beyond the own ones: halo rows and x-edge chunks (TMAS: the x-edge chunks)
    static constexpr int NPOS = TMAS ? 2 * RY : 2 * NCH + 2 * RY;
    static constexpr size_t ring_off = 32;         // three mbarriers, the TMEM base address
    static constexpr size_t ring_bytes = sizeof(float) * (size_t)NSLOT * 3 * RY * RP;
    static constexpr size_t stg_off = (ring_off + ring_bytes + 127) / 128 * 128;  // TMA destinations: 128-byte aligned
    static constexpr size_t stg_int_bytes = sizeof(S) * (size_t)27 * RY * TX;     // TMAS: [27][RY][TX]
    static constexpr size_t stg_bytes = TMAS ? stg_int_bytes + sizeof(S) * (size_t)27 * RY * 8
                                             : sizeof(S) * (size_t)27 * RY * RP;  // [27][RY][RP], storage format
    static constexpr unsigned tma_bytes = (unsigned)stg_int_bytes;                // bytes the TMA copies per plane
    static_assert(!TMAS || (RY * TX * sizeof(S)) % 128 == 0, "each population's TMA box 128-byte aligned");
    static_assert(!(TMAS && LEARNED), "TMA staging is built for the analytic closures");
    static_assert(!TMAS || (NPOS <= 40 && 40 + 8 * 26 < NT), "TMA issuing threads apart from the x-edge threads");
    static constexpr size_t bb_off = (stg_off + stg_bytes + 127) / 128 * 128;  // TMAS: TMA destinations
    static constexpr size_t bb_bytes = WALLS ? sizeof(S) * (size_t)2 * 9 * TX : 0;
    // learned closure: the packed network and one 32-row exchange per warp
    static constexpr size_t mlp_off = bb_off + bb_bytes;
    static constexpr size_t mlp_bytes = LEARNED ? (size_t)MlpLayout::BYTES + 8 * (size_t)MlpLayout::XCH_BYTES : 0;
    static constexpr size_t used = mlp_off + mlp_bytes;
    // at least 116 KB, so that two CTAs never share an SM (each allocates all
    // 512 TMEM columns; a second one would wait for the first to finish)
    static constexpr size_t smem_bytes = used > 116 * 1024 ? used : 116 * 1024;
    static_assert(smem_bytes <= 227 * 1024, "shared memory of one CTA");
};

// D3Q19 in the four-cell kernel: a population keeps its D3Q27 position
// j = 9 (c_z + 1) + 3 (c_y + 1) + (c_x + 1) for its staged rows, its TMEM
// columns and its triple p = j / 3 along x; D3Q19 has no corners (all three
// components nonzero), so its four triples with c_y c_z != 0 hold the c_x = 0
// population only.  v4_has: position j is a population of lattice Q;
// v4_pop: its index in lattice Q (the population arrays' order).
__host__ __device__ constexpr bool v4_has(int Q, int j)
{
    return Q == 27 || j % 3 == 1 || (j / 3) % 3 == 1 || j / 9 == 1;
}
constexpr unsigned kV4Corners = 0x5140145u;  // bits j of the eight corners: 0, 2, 6, 8, 18, 20, 24, 26
__host__ __device__ constexpr int v4_pop(int Q, int j)
{
    int below = 0;  // corners before position j
    for (int k = 0; k < j; ++k) below += (kV4Corners >> k) & 1u;
    return Q == 27 ? j : j - below;
}
// the same at run time (a thread's population)
__device__ __forceinline__ int v4_pop_rt(int Q, int j) { return Q == 27 ? j : j - __popc(kV4Corners & ((1u << j) - 1u)); }

// relaxation constants of one cell (collide_coef in the per-triple form).
// D3Q27: the product equilibrium's per-axis terms ex, ey, ez.  D3Q19 (second
// order Hermite equilibrium, P - 1 = c.u/theta + (c.u)^2/(2 theta^2) -
// u^2/(2 theta)): qx, qy, qz = u/theta, qq = qx^2/2 and hu = -u^2/(2 theta), so
// that along a triple with B = c_y qy + c_z qz, P - 1 = Y + c_x qx (1 + B) +
// c_x^2 qq with Y = B + B^2/2 + hu.
struct V4Cell {
    float ca, cb, ex[3], ey[3], ez[3], C[5], Dxx, Dxy2, Dxz2;
    float qx, qy, qz, qq, hu;
};

// index of the (c_y, c_z) part of H: (0,0), (+-1,0), (0,+-1), c_y c_z = 1, c_y c_z = -1
__host__ __device__ constexpr int v4_pat(int cy, int cz)
{
    return (cy == 0 && cz == 0) ? 0 : (cz == 0 ? 1 : (cy == 0 ? 2 : (cy * cz == 1 ? 3 : 4)));
}

// asynchronous 16-byte global -> shared copy (L2 only)
__device__ __forceinline__ void cp_async_cg16(uint32_t dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
// one arrival on the mbarrier once all of the thread's earlier cp.async copies have landed
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(a) : "memory");
}
// four consecutive stored values (one 16- or 8-byte chunk)
template <typename S>
__device__ __forceinline__ void cp_async_chunk(uint32_t dst, const S* src)
{
    if constexpr (sizeof(S) == 4)
        cp_async_cg16(dst, src);
    else
        cp_async_ca<8>(dst, src);
}
__device__ __forceinline__ float v4_cvt(float v) { return v; }
__device__ __forceinline__ float v4_cvt(__half v) { return __half2float(v); }
__device__ __forceinline__ float v4_cvt(__nv_bfloat16 v) { return __bfloat162float(v); }
// four staged values as FP32
__device__ __forceinline__ float4 v4_lds(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 v4_lds(const __half* p)
{
    const uint2 r = *reinterpret_cast<const uint2*>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&r.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&r.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 v4_lds(const __nv_bfloat16* p)
{
    const uint2 r = *reinterpret_cast<const uint2*>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

// Learned closure, one cell per lane: the ten network inputs ((m_neq - m_CE)/rho
// from the second moments Pi' = sum g c c of the streamed populations, the
// invariants of m_CE/rho = -2 theta tau_hat S, tau_hat), standardised, into
// the lane's row of the warp's exchange; the BF16 tensor-core forward of the
// warp's 32 rows, one 16-row tile after the other (both at once, as the
// register-pull kernel does, spills here); the cell's m_sgs = rho (y sd +
// mean) back.  The same inputs and network as the register-pull kernel's
// learned_msgs; here the second moments come from the pull's triple sums
// instead of the stash.
__device__ __forceinline__ void v4_learned_msgs(const float (&P)[6], float drho, float ux, float uy, float uz,
                                                float Sxx, float Syy, float Szz, float Sxy, float Sxz, float Syz,
                                                float tau_hat, const unsigned char* sm_mlp, unsigned char* xch,
                                                int lane, float (&msgs)[6])
{
    using L = MlpLayout;
    constexpr float th = (float)kTheta;
    const float rho = 1.f + drho, irho = 1.f / rho;
    const float k = -2.f * th * tau_hat;  // m_CE / rho = k S
    const float a00 = k * Sxx, a11 = k * Syy, a22 = k * Szz, a01 = k * Sxy, a02 = k * Sxz, a12 = k * Syz;
    float x[10];
    x[0] = (P[0] - rho * ux * ux - th * drho) * irho - a00;
    x[1] = (P[1] - rho * uy * uy - th * drho) * irho - a11;
    x[2] = (P[2] - rho * uz * uz - th * drho) * irho - a22;
    x[3] = (P[3] - rho * ux * uy) * irho - a01;
    x[4] = (P[4] - rho * ux * uz) * irho - a02;
    x[5] = (P[5] - rho * uy * uz) * irho - a12;
    const float tr = a00 + a11 + a22;
    const float tr2 = a00 * a00 + a11 * a11 + a22 * a22 + 2.f * (a01 * a01 + a02 * a02 + a12 * a12);
    x[6] = tr;
    x[7] = 0.5f * (tr * tr - tr2);
    x[8] = a00 * (a11 * a22 - a12 * a12) - a01 * (a01 * a22 - a12 * a02) + a02 * (a01 * a12 - a11 * a02);
    x[9] = tau_hat;
    const float* xmu = reinterpret_cast<const float*>(sm_mlp + L::XMU);
    const float* xis = reinterpret_cast<const float*>(sm_mlp + L::XIS);
    __nv_bfloat16* X = reinterpret_cast<__nv_bfloat16*>(xch);
    float* Y = reinterpret_cast<float*>(xch);  // overlays the inputs
    uint32_t* Xrow = reinterpret_cast<uint32_t*>(X + lane * L::XLD);
#pragma unroll
    for (int q = 0; q < 5; ++q)
        Xrow[q] = pack_bf16((x[2 * q] - xmu[2 * q]) * xis[2 * q], (x[2 * q + 1] - xmu[2 * q + 1]) * xis[2 * q + 1]);
#pragma unroll
    for (int q = 5; q < 8; ++q) Xrow[q] = 0u;
    __syncwarp();
    mlp_warp_forward(sm_mlp, X, Y, lane);
    __syncwarp();
    const float* ymu = reinterpret_cast<const float*>(sm_mlp + L::YMU);
    const float* ysd = reinterpret_cast<const float*>(sm_mlp + L::YSD);
#pragma unroll
    for (int q = 0; q < 6; ++q) msgs[q] = rho * (Y[lane * 8 + q] * ysd[q] + ymu[q]);
    __syncwarp();  // every lane has read its outputs before the exchange is reused
}

// Load schedule.  The pulls of a plane are staged in shared memory: for each
// population i the rows y0 - 1 - c_y .. y0 + TY - c_y (the own rows' and the
// y-halo rows' sources) over x0 - 4 .. x0 + TX + 3, as 16-byte (FP32) or
// 8-byte (16-bit) chunks copied by cp.async: each thread copies its own four
// cells' chunk of every population, and NPOS threads one more chunk each (the
// y-halo rows and the x-edge chunks of every row).  The x-halo cells and the
// values that cross a tile edge are read from those edge chunks, so no load
// touches a single scattered value.  A staging mbarrier, on which every
// thread arrives by cp.async.mbarrier.arrive once its copies have landed,
// makes the plane visible to all threads; the ring mbarrier of the plane,
// waited for right after the thread's own arrival, tells that every thread has
// read the staging area, after which the copies of the plane after next are
// issued.  They land while the current plane collides.  Plane p arrives on ring
// mbarrier (p - z0) & 1 (parity ((p - z0) >> 1) & 1) and fills the staging
// area for the (p - z0)-th time (staging mbarrier parity (p - z0) & 1).
// one TMA copy of a box of a 4D tensor map into shared memory, completing on
// the mbarrier (transaction bytes)
__device__ __forceinline__ void v4_tma_load(void* smem_dst, const CUtensorMap* map, int x, int y, int z, int w,
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

// BC = BC_WALLS_Y: halfway bounce-back walls at y = 0 and y = ny - 1 with a body
// force (the channel).  The staged rows stay those of the periodic box; a wall
// row replaces the pulls that cross its wall by the cell's own post-collision
// opposite population (staged with the plane), takes the one-sided
// difference of Eqs. (fd_boundary_lower/upper) across y, the velocity shifted
// by F/2 and Guo's source.  Rows beyond a wall are computed from the periodic
// image and neither stored nor read.  The top wall row must not be the first
// row of its tile ((ny - 1) % TY != 0), so that both rows below it are in the
// ring.
template <int Q, typename S, int CL, int LPR, bool TMAS = false, int BC = BC_PERIODIC>
__global__ void __launch_bounds__(256, 1)
    step_kernel_v4(const StepArgs a, const __grid_constant__ CUtensorMap map_rows, const __grid_constant__ CUtensorMap map_row1,
                   const __grid_constant__ CUtensorMap map_rm1, const __grid_constant__ CUtensorMap map_rm2)
{
    static_assert(Q == 27 || Q == 19, "the four-cell kernel is built for D3Q27 and D3Q19 (population triples along x)");
    static_assert(Q == 27 || CL != CL_LEARNED, "the learned closure's four-cell kernel is D3Q27");
    static_assert(!std::is_same<S, double>::value, "FP32 arithmetic");
    static_assert(CL == CL_BGK || CL == CL_KCMP || CL == CL_KCRB_H || CL == CL_KCRB_RAW || CL == CL_KCRR ||
                      CL == CL_LEARNED,
                  "closure");
    static_assert(CL != CL_KCRR || (Q == 27 && BC == BC_PERIODIC), "KC-RR: D3Q27, periodic boxes");
    constexpr bool LEARNED = CL == CL_LEARNED;
    constexpr bool WALLS = BC == BC_WALLS_Y;
    static_assert(!(WALLS && LEARNED), "the learned closure runs on periodic boxes");
    using Sh = V4Shape<LPR, S, LEARNED, TMAS, WALLS, v4_ring4(TMAS, CL, BC)>;
    constexpr int TX = Sh::TX, TY = Sh::TY, RY = Sh::RY, RP = Sh::RP, NB = Sh::NB, NT = Sh::NT, NCH = Sh::NCH;
    constexpr int NHK = (NB + NT - 1) / NT;  // halo cells per thread (at most)
    constexpr bool SHIFTED = StoreTraits<S>::shifted;
    constexpr unsigned FULL = 0xffffffffu;
    constexpr bool RZ = Sh::NSLOT == 4;  // the own cells' z-neighbours read from the ring

    extern __shared__ __align__(16) unsigned char smem_v4[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_v4);  // [0], [1]: ring planes, [2]: staging
    uint32_t* tm_base_sm = reinterpret_cast<uint32_t*>(smem_v4 + 24);
    float* ring = reinterpret_cast<float*>(smem_v4 + Sh::ring_off);  // [NSLOT][3][RY][RP]
    S* stg = reinterpret_cast<S*>(smem_v4 + Sh::stg_off);            // [27][RY][RP] (TMAS: [27][RY][TX])
    S* stge = stg + 27 * RY * TX;                                     // TMAS: x-edge chunks [27][RY][8]
    S* bbs = reinterpret_cast<S*>(smem_v4 + Sh::bb_off);              // WALLS: [2][9][TX] bounce-back values
    unsigned char* sm_mlp = smem_v4 + Sh::mlp_off;                   // learned closure only
    unsigned char* sm_xch = sm_mlp + MlpLayout::BYTES + (threadIdx.x >> 5) * MlpLayout::XCH_BYTES;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int tiles_x = (nx + TX - 1) / TX;
    const int x0 = (int)(blockIdx.x % tiles_x) * TX;
    const int y0 = (int)(blockIdx.x / tiles_x) * TY;
    const int z0 = (int)blockIdx.y * a.zchunk;
    if (z0 >= nz) return;  // uniform over the CTA, before any allocation
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
    // Guo's source (walls): (1 - omega/2)/theta and (1 - omega/2)/theta^2
    const float gp1 = (1.f - 0.5f * omega) * (float)(1.0 / kTheta), gp2 = gp1 * (float)(1.0 / kTheta);

    // own cells: row ty of the tile (staged row ty + 1), x = xa .. xa + 3
    // (wrapped into the box for lanes beyond nx, which compute but do not store)
    const int lx = lane % LPR;
    const int ty = warp * Sh::RPW + lane / LPR;
    const int gy = y0 + ty, xa = x0 + 4 * lx;
    const bool own_store = gy < ny && xa < nx;
    const int gyw = gy % ny, xaw = xa % nx;
    const int yr_own[3] = {(gyw == 0 ? ny - 1 : gyw - 1) * nx, gyw * nx, (gyw == ny - 1 ? 0 : gyw + 1) * nx};
    const int xl = (x0 + nx - 1) % nx;  // left neighbour of the row's first cell (own pulls of the first plane)
    const int xr = (x0 + TX) % nx;      // right neighbour of the row's last cell
    const int ry_own = ty + 1, rx_own = 4 + 4 * lx;
    // walls: this thread's row at a wall, and the body force
    const bool wall_lo = WALLS && gy == 0, wall_hi = WALLS && gy == ny - 1;
    const float Fx = WALLS ? (float)a.force[0] : 0.f, Fy = WALLS ? (float)a.force[1] : 0.f,
                Fz = WALLS ? (float)a.force[2] : 0.f;

    // the extra staged chunk of this thread (tid < NPOS): staged row, column, global x, source rows
    int pos_r = -1, pos_col = 0, pos_x = 0, yr_pos[3] = {0, 0, 0};
    if (tid < Sh::NPOS) {
        const int p = TMAS ? tid + 2 * NCH : tid;  // TMAS: x-edge chunks only
        if (p < 2 * NCH) {  // y-halo rows
            const int c = p % NCH;
            pos_r = p < NCH ? 0 : RY - 1;
            pos_col = 4 + 4 * c;
            pos_x = (x0 + 4 * c) % nx;
        } else {  // x-edge chunks of every staged row
            const int q = p - 2 * NCH;
            const bool left = q < RY;
            pos_r = left ? q : q - RY;
            pos_col = left ? 0 : TX + 4;
            pos_x = left ? (x0 + nx - 4) % nx : (x0 + TX) % nx;
        }
        const int yy = y0 - 1 + pos_r;
#pragma unroll
        for (int k = 0; k < 3; ++k) yr_pos[k] = wrapi(yy - 1 + k, ny) * nx;
    }
    // halo cells of this thread: h = tid + k NT < NB; y-halo rows first, then
    // the x-halo columns; staged row and x relative to x0
    int hal_rr[NHK], hal_xr[NHK];
#pragma unroll
    for (int k = 0; k < NHK; ++k) {
        const int h = tid + k * NT;
        hal_rr[k] = -1;
        hal_xr[k] = 0;
        if (h < NB) {
            if (h < 2 * TX) {
                hal_rr[k] = h < TX ? 0 : RY - 1;
                hal_xr[k] = h % TX;
            } else {
                const int j = h - 2 * TX;
                hal_rr[k] = j % TY + 1;
                hal_xr[k] = j < TY ? -1 : TX;
            }
        }
    }

    if constexpr (LEARNED) {  // the packed network, visible after the barrier below
        const uint4* src = static_cast<const uint4*>(a.mlp);
        uint4* dst = reinterpret_cast<uint4*>(sm_mlp);
        for (int k = tid; k < MlpLayout::BYTES / 16; k += NT) dst[k] = src[k];
    }
    // TMEM: warp 0 allocates the 512 columns; the two warps of a lane quarter
    // take 256 each; slot s of a thread starts at column 128 s of its share
    if (warp == 0) {
        tm_alloc(tm_base_sm, 512u);
        tm_relinquish();
    }
    if (tid == 0) {
        mbar_init(&mbar[0], NT);
        mbar_init(&mbar[1], NT);
        mbar_init(&mbar[2], NT);
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t tm_all = *tm_base_sm;
    const uint32_t tm_me = tm_all + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * 256);
    auto tslot = [&](int z) { return tm_me + (uint32_t)((z & 1) * 128); };

    auto zrows = [&](int z, int (&zr)[3]) {
        const int zc = z < 0 ? z + nz : (z >= nz ? z - nz : z);  // z in [-1, nz]
        zr[0] = (zc == 0 ? nz - 1 : zc - 1) * plane;
        zr[1] = zc * plane;
        zr[2] = (zc == nz - 1 ? 0 : zc + 1) * plane;
    };
    auto rslot = [&](int z) { return (int)((unsigned)(z - z0 + 1) % (unsigned)Sh::NSLOT); };
    auto ringp = [&](int s, int c) { return ring + (s * 3 + c) * (RY * RP); };
    // staged value of population i, staged row r, column col (x0 - 4 + col)
    auto stg_at = [&](int i, int r, int col) {
        if constexpr (TMAS) {
            if (col < 4) return stge + (i * RY + r) * 8 + col;
            if (col >= TX + 4) return stge + (i * RY + r) * 8 + (col - TX);
            return stg + (i * RY + r) * TX + (col - 4);
        } else {
            return stg + (i * RY + r) * RP + col;
        }
    };

    // cp.async of plane z's pulls into the staging area, then the thread's
    // arrival on the staging mbarrier (completed by the copies)
    auto issue = [&](int z) {
        int zr[3];
        zrows(z, zr);
        if constexpr (TMAS) {
            if (pos_r >= 0) {  // x-edge chunks by cp.async
                static_for<27>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    constexpr int cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
                    if constexpr (v4_has(Q, i)) {
                        const S* base = fin + (long long)v4_pop(Q, i) * ps + zr[1 - cz];
                        cp_async_chunk<S>((uint32_t)__cvta_generic_to_shared(stg_at(i, pos_r, pos_col)),
                                          base + yr_pos[1 - cy] + pos_x);
                    }
                });
                cp_async_commit();
                cp_async_arrive(&mbar[2]);
            } else if (tid >= 40 && (tid - 40) % 8 == 0 && v4_has(Q, (tid - 40) / 8)) {
                // the interior by the TMA: position (tid - 40) / 8, one issuing thread per
                // population, spread over the warps
                const int i = (tid - 40) / 8;
                const int cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
                const int zc = z < 0 ? z + nz : (z >= nz ? z - nz : z);
                const int zsrc = cz == 0 ? zc : (cz == 1 ? (zc == 0 ? nz - 1 : zc - 1) : (zc == nz - 1 ? 0 : zc + 1));
                const int ys = y0 - 1 - cy, w = box * Q + v4_pop_rt(Q, i);
                S* dst = stg + i * RY * TX;
                // walls: issuers 0..8 also copy the bounce-back row qb = i of the lower
                // and the upper wall when the tile holds it (population 26 - j of the
                // wall row at plane z, j the pull that crosses the wall)
                const int jlo = 9 * (i / 3) + 6 + i % 3, jhi = 9 * (i / 3) + i % 3;  // the crossing pulls (i < 9)
                const bool bb_lo = WALLS && i < 9 && y0 == 0 && v4_has(Q, jlo);
                const bool bb_hi = WALLS && i < 9 && y0 <= ny - 1 && ny - 1 < y0 + TY && v4_has(Q, jhi);
                mbar_expect_tx(&mbar[2], Sh::tma_bytes / 27u + (unsigned)((bb_lo + bb_hi) * TX * (int)sizeof(S)));
                const int klo = -ys, khi = ys + RY - ny;  // rows wrapped from the top / to the bottom
                if (ys >= 0 && khi <= 0) {
                    v4_tma_load(dst, &map_rows, x0, ys, zsrc, w, &mbar[2]);
                } else if (klo >= 1 && klo <= 2 && RY - klo <= ny) {
                    // rows ys .. -1 are rows ny + ys .. ny - 1, one at a time; the rest one box
                    for (int r = 0; r < klo; ++r) v4_tma_load(dst + r * TX, &map_row1, x0, ny + ys + r, zsrc, w, &mbar[2]);
                    v4_tma_load(dst + klo * TX, klo == 1 ? &map_rm1 : &map_rm2, x0, 0, zsrc, w, &mbar[2]);
                } else if (ys >= 0 && khi <= 2) {
                    // one box of rows ys .. ny - 1, then rows ny .. are rows 0 .., one at a time
                    v4_tma_load(dst, khi == 1 ? &map_rm1 : &map_rm2, x0, ys, zsrc, w, &mbar[2]);
                    for (int r = RY - khi; r < RY; ++r)
                        v4_tma_load(dst + r * TX, &map_row1, x0, ys + r - ny, zsrc, w, &mbar[2]);
                } else {  // short boxes and ragged last tiles: one row at a time
#pragma unroll 1
                    for (int r = 0; r < RY; ++r)
                        v4_tma_load(dst + r * TX, &map_row1, x0, wrapi(ys + r, ny), zsrc, w, &mbar[2]);
                }
                if constexpr (WALLS) {  // qb = i = 3 (c_z + 1) + (c_x + 1) of the crossing pull
                    if (bb_lo)  // pulls with c_y = +1 cross the lower wall
                        v4_tma_load(bbs + i * TX, &map_row1, x0, 0, zc, box * Q + v4_pop_rt(Q, 26 - jlo), &mbar[2]);
                    if (bb_hi)  // pulls with c_y = -1 cross the upper wall
                        v4_tma_load(bbs + (9 + i) * TX, &map_row1, x0, ny - 1, zc, box * Q + v4_pop_rt(Q, 26 - jhi),
                                    &mbar[2]);
                }
            } else {
                mbar_arrive(&mbar[2]);
            }
            return;
        }
        static_for<27>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
            if constexpr (v4_has(Q, i)) {
                const S* base = fin + (long long)v4_pop(Q, i) * ps + zr[1 - cz];
                cp_async_chunk<S>((uint32_t)__cvta_generic_to_shared(stg_at(i, ry_own, rx_own)),
                                  base + yr_own[1 - cy] + xaw);
                if (pos_r >= 0)
                    cp_async_chunk<S>((uint32_t)__cvta_generic_to_shared(stg_at(i, pos_r, pos_col)),
                                      base + yr_pos[1 - cy] + pos_x);
                // a wall row's bounce-back values: the opposite population (position
                // 26 - i) of its own cells (plane z) for the pulls i that cross the wall,
                // slot 0 lower wall, 1 upper
                if constexpr (WALLS && cy != 0) {
                    if (cy == 1 ? wall_lo : wall_hi) {
                        constexpr int qb = 3 * (cz + 1) + (i % 3);
                        cp_async_chunk<S>(
                            (uint32_t)__cvta_generic_to_shared(bbs + ((cy == 1 ? 0 : 9) + qb) * TX + 4 * lx),
                            fin + (long long)v4_pop(Q, 26 - i) * ps + zr[1] + yr_own[1] + xaw);
                    }
                }
            }
        });
        cp_async_commit();
        cp_async_arrive(&mbar[2]);
    };
    auto staged_wait = [&](int z) { return mbar_wait_bounded(&mbar[2], (unsigned)(z - z0) & 1u); };

    // The own four cells at plane z: moments (drho = sum g, u, and with FULL
    // the second moments Pi' = sum g c c) and, with FULL, the streamed
    // populations g = f - w into the TMEM slot of plane z.  STAGED: from the
    // staging area, else loaded from global memory (first plane of a chunk).
    auto pull_own = [&](auto full_tag, auto staged_tag, int z, float (&dr)[4], float (&u)[3][4], float (&P)[6][4]) {
        constexpr bool FULL = decltype(full_tag)::value;
        constexpr bool STAGED = decltype(staged_tag)::value;
        int zr[3];
        zrows(z, zr);
        float d[4], jx[4], jy[4], jz[4], g0[4], pyy[4], pzz[4], pxy[4], pxz[4], pyz[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) d[c] = jx[c] = jy[c] = jz[c] = g0[c] = pyy[c] = pzz[c] = pxy[c] = pxz[c] = pyz[c] = 0.f;
        const uint32_t ts = tslot(z);
        static_for<9>([&](auto PI) {
            constexpr int p = decltype(PI)::value;
            constexpr int cy = p % 3 - 1, cz = p / 3 - 1;
            const int roff = zr[1 - cz] + yr_own[1 - cy];
            constexpr bool TRIPLE = v4_has(Q, 3 * p);  // D3Q19: c_y c_z != 0 holds c_x = 0 only
            float g[3][4];
            static_for<3>([&](auto CI) {
                constexpr int k = decltype(CI)::value;
                constexpr int cx = k - 1, i = 3 * p + k;
                if constexpr (!v4_has(Q, i)) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) g[k][c] = 0.f;
                    return;
                }
                const S* src = fin + (long long)v4_pop(Q, i) * ps + roff;
                float4 v;
                if constexpr (STAGED)
                    v = v4_lds(stg_at(i, ry_own, rx_own));
                else
                    v = v4_load(src + xaw);
                if constexpr (cx == 1) {  // cell x pulls x - 1
                    float e = __shfl_up_sync(FULL, v.w, 1, LPR);
                    if (lx == 0) e = STAGED ? v4_cvt(*stg_at(i, ry_own, 3)) : v1_load(src + xl);
                    g[k][0] = e;
                    g[k][1] = v.x;
                    g[k][2] = v.y;
                    g[k][3] = v.z;
                } else if constexpr (cx == -1) {  // cell x pulls x + 1
                    float e = __shfl_down_sync(FULL, v.x, 1, LPR);
                    if (lx == LPR - 1) e = STAGED ? v4_cvt(*stg_at(i, ry_own, TX + 4)) : v1_load(src + xr);
                    g[k][0] = v.y;
                    g[k][1] = v.z;
                    g[k][2] = v.w;
                    g[k][3] = e;
                } else {
                    g[k][0] = v.x;
                    g[k][1] = v.y;
                    g[k][2] = v.z;
                    g[k][3] = v.w;
                }
                if constexpr (!SHIFTED) {
                    constexpr float w = (float)weight_of(Q, v4_pop(Q, i));
#pragma unroll
                    for (int c = 0; c < 4; ++c) g[k][c] -= w;
                }
                if constexpr (WALLS && cy != 0) {
                    // halfway bounce-back: a pull across the wall takes the cell's own
                    // post-collision opposite population (same plane); from the staged
                    // copy, read by every thread and selected, so that no branch splits
                    // the triple's loads
                    const bool wl = cy == 1 ? wall_lo : wall_hi;
                    constexpr float w = SHIFTED ? 0.f : (float)weight_of(Q, v4_pop(Q, i));
                    if constexpr (STAGED) {
                        constexpr int qb = 3 * (cz + 1) + (i % 3);
                        const float4 b = v4_lds(bbs + ((cy == 1 ? 0 : 9) + qb) * TX + 4 * lx);
                        g[k][0] = wl ? b.x - w : g[k][0];
                        g[k][1] = wl ? b.y - w : g[k][1];
                        g[k][2] = wl ? b.z - w : g[k][2];
                        g[k][3] = wl ? b.w - w : g[k][3];
                    } else if (wl) {
                        const float4 b = v4_load(fin + (long long)v4_pop(Q, 26 - i) * ps + zr[1] + yr_own[1] + xaw);
                        g[k][0] = b.x - w;
                        g[k][1] = b.y - w;
                        g[k][2] = b.z - w;
                        g[k][3] = b.w - w;
                    }
                }
            });
            if constexpr (FULL) tm_st12(ts + 12u * p, g);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float s = TRIPLE ? (g[0][c] + g[1][c]) + g[2][c] : g[1][c];
                const float dx = TRIPLE ? g[2][c] - g[0][c] : 0.f;
                d[c] += s;
                if constexpr (TRIPLE) jx[c] += dx;
                if constexpr (cy == 1) jy[c] += s;
                if constexpr (cy == -1) jy[c] -= s;
                if constexpr (cz == 1) jz[c] += s;
                if constexpr (cz == -1) jz[c] -= s;
                if constexpr (FULL) {
                    g0[c] += g[1][c];
                    if constexpr (cy != 0) pyy[c] += s;
                    if constexpr (cz != 0) pzz[c] += s;
                    if constexpr (TRIPLE && cy == 1) pxy[c] += dx;
                    if constexpr (TRIPLE && cy == -1) pxy[c] -= dx;
                    if constexpr (TRIPLE && cz == 1) pxz[c] += dx;
                    if constexpr (TRIPLE && cz == -1) pxz[c] -= dx;
                    if constexpr (cy * cz == 1) pyz[c] += s;
                    if constexpr (cy * cz == -1) pyz[c] -= s;
                }
            }
        });
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            dr[c] = d[c];
            const float inv = 1.f / (1.f + d[c]);
            if constexpr (WALLS) {  // u = (sum g c + F/2) / rho
                u[0][c] = (jx[c] + 0.5f * Fx) * inv;
                u[1][c] = (jy[c] + 0.5f * Fy) * inv;
                u[2][c] = (jz[c] + 0.5f * Fz) * inv;
            } else {
                u[0][c] = jx[c] * inv;
                u[1][c] = jy[c] * inv;
                u[2][c] = jz[c] * inv;
            }
            if constexpr (FULL) {
                P[0][c] = d[c] - g0[c];
                P[1][c] = pyy[c];
                P[2][c] = pzz[c];
                P[3][c] = pxy[c];
                P[4][c] = pxz[c];
                P[5][c] = pyz[c];
            }
        }
    };
    auto put_own = [&](int z, const float (&u)[3][4]) {
        const int s = rslot(z);
#pragma unroll
        for (int b = 0; b < 3; ++b)
            *reinterpret_cast<float4*>(ringp(s, b) + ry_own * RP + rx_own) = make_float4(u[b][0], u[b][1], u[b][2], u[b][3]);
    };
    // halo cells at plane z, from the staging area: velocity into the ring
    auto halo_plane = [&](int z) {
        const int s = rslot(z);
#pragma unroll
        for (int k = 0; k < NHK; ++k) {
            if (hal_rr[k] >= 0) {
                const int r = hal_rr[k], xr4 = 4 + hal_xr[k];
                const int yh = y0 - 1 + r;  // the halo cell's row
                const bool hlo = WALLS && yh == 0, hhi = WALLS && yh == ny - 1;
                float gh[Q];
                static_for<27>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    constexpr int cx = i % 3 - 1;
                    if constexpr (v4_has(Q, i)) {
                        constexpr int iq = v4_pop(Q, i);
                        const float v = v4_cvt(*stg_at(i, r, xr4 - cx));
                        gh[iq] = SHIFTED ? v : v - (float)weight_of(Q, iq);
                    }
                });
                if constexpr (WALLS) {
                    if (hlo || hhi) {  // bounce-back at a wall row (x-halo cells)
                        int zr[3];
                        zrows(z, zr);
                        const S* cellp = fin + zr[1] + yh * nx + (x0 + hal_xr[k] + nx) % nx;
                        static_for<27>([&](auto I) {
                            constexpr int i = decltype(I)::value;
                            constexpr int cy = (i / 3) % 3 - 1;
                            if constexpr (cy != 0 && v4_has(Q, i)) {
                                if (cy == 1 ? hlo : hhi) {
                                    constexpr int iq = v4_pop(Q, i);
                                    const float v = v1_load(cellp + (long long)v4_pop(Q, 26 - i) * ps);
                                    gh[iq] = SHIFTED ? v : v - (float)weight_of(Q, iq);
                                }
                            }
                        });
                    }
                }
                float dh, vx, vy, vz;
                moments<Q, float>(gh, dh, vx, vy, vz, Fx, Fy, Fz);
                const int pos = r * RP + xr4;
                ringp(s, 0)[pos] = vx;
                ringp(s, 1)[pos] = vy;
                ringp(s, 2)[pos] = vz;
            }
        }
    };
    auto arrive = [&](int p) { mbar_arrive(&mbar[(p - z0) & 1]); };
    auto wait = [&](int p) { return mbar_wait_bounded(&mbar[(p - z0) & 1], (unsigned)((p - z0) >> 1) & 1u); };

    bool ok = true;
    float um[3][4], dr0[4], u0[3][4], P0[6][4];  // own: u at z - 1; drho, u, Pi' at z
    {
        issue(z0);
        float dd[4], PP[6][4];  // the first plane's z-neighbour, loaded while plane z0 is staged
        pull_own(std::false_type{}, std::false_type{}, z0 - 1, dd, um, PP);
        if constexpr (RZ) put_own(z0 - 1, um);
        ok = __all_sync(FULL, staged_wait(z0));
        if (ok) {
            pull_own(std::true_type{}, std::true_type{}, z0, dr0, u0, P0);
            put_own(z0, u0);
            halo_plane(z0);
            tm_wait_st();
            arrive(z0);
            ok = __all_sync(FULL, wait(z0));  // every thread has read the staging area
            if (ok) issue(z0 + 1);            // z0 + 1 <= z1
        }
    }

    for (int z = z0; z < z1 && ok; ++z) {
        // ---- plane z+1: staged pulls (populations to TMEM while it will be
        // collided), velocities to the ring; then the copies of plane z+2
        float dr1[4], u1[3][4], P1[6][4];
        if (!__all_sync(FULL, staged_wait(z + 1))) {  // warp-uniform: the TMEM accesses stay converged
            ok = false;
            break;
        }
        if (z + 1 < z1) {
            pull_own(std::true_type{}, std::true_type{}, z + 1, dr1, u1, P1);
            put_own(z + 1, u1);
            halo_plane(z + 1);
            tm_wait_st();
            arrive(z + 1);
            // every thread has published plane z+1 (so also plane z) and read the staging area
            if (!__all_sync(FULL, wait(z + 1))) {
                ok = false;
                break;
            }
            if (z + 2 <= z1) issue(z + 2);
        } else {
            pull_own(std::false_type{}, std::true_type{}, z + 1, dr1, u1, P1);  // z-neighbour of the chunk's last plane
            if constexpr (RZ) put_own(z + 1, u1);
        }

        // ---- plane z: neighbours' velocities, strain, closure, relaxation, store
        // du[a][b][c] = d_a u_b of cell c
        float S6[6][4];
        float uo[3][4];  // the own cells' u at z
        {
            float du[3][3][4];
            const int s0 = rslot(z);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const float* r = ringp(s0, b) + ry_own * RP + rx_own;
                if constexpr (RZ) {
                    const float4 c4 = *reinterpret_cast<const float4*>(r);
                    uo[b][0] = c4.x;
                    uo[b][1] = c4.y;
                    uo[b][2] = c4.z;
                    uo[b][3] = c4.w;
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) uo[b][c] = u0[b][c];
                }
                const float ul = r[-1], ur = r[4];
                const float4 yn = *reinterpret_cast<const float4*>(r - RP);
                const float4 yp = *reinterpret_cast<const float4*>(r + RP);
                du[0][b][0] = 0.5f * (uo[b][1] - ul);
                du[0][b][1] = 0.5f * (uo[b][2] - uo[b][0]);
                du[0][b][2] = 0.5f * (uo[b][3] - uo[b][1]);
                du[0][b][3] = 0.5f * (ur - uo[b][2]);
                if (WALLS && wall_lo) {  // one-sided at the lower wall, Eq. (fd_boundary_lower)
                    const float4 y2 = *reinterpret_cast<const float4*>(r + 2 * RP);
                    du[1][b][0] = 0.5f * (-3.f * uo[b][0] + 4.f * yp.x - y2.x);
                    du[1][b][1] = 0.5f * (-3.f * uo[b][1] + 4.f * yp.y - y2.y);
                    du[1][b][2] = 0.5f * (-3.f * uo[b][2] + 4.f * yp.z - y2.z);
                    du[1][b][3] = 0.5f * (-3.f * uo[b][3] + 4.f * yp.w - y2.w);
                } else if (WALLS && wall_hi) {  // one-sided at the upper wall, Eq. (fd_boundary_upper)
                    const float4 y2 = *reinterpret_cast<const float4*>(r - 2 * RP);
                    du[1][b][0] = 0.5f * (3.f * uo[b][0] - 4.f * yn.x + y2.x);
                    du[1][b][1] = 0.5f * (3.f * uo[b][1] - 4.f * yn.y + y2.y);
                    du[1][b][2] = 0.5f * (3.f * uo[b][2] - 4.f * yn.z + y2.z);
                    du[1][b][3] = 0.5f * (3.f * uo[b][3] - 4.f * yn.w + y2.w);
                } else {
                    du[1][b][0] = 0.5f * (yp.x - yn.x);
                    du[1][b][1] = 0.5f * (yp.y - yn.y);
                    du[1][b][2] = 0.5f * (yp.z - yn.z);
                    du[1][b][3] = 0.5f * (yp.w - yn.w);
                }
                if constexpr (RZ) {
                    const float4 zp = *reinterpret_cast<const float4*>(ringp(rslot(z + 1), b) + ry_own * RP + rx_own);
                    const float4 zm = *reinterpret_cast<const float4*>(ringp(rslot(z - 1), b) + ry_own * RP + rx_own);
                    du[2][b][0] = 0.5f * (zp.x - zm.x);
                    du[2][b][1] = 0.5f * (zp.y - zm.y);
                    du[2][b][2] = 0.5f * (zp.z - zm.z);
                    du[2][b][3] = 0.5f * (zp.w - zm.w);
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) du[2][b][c] = 0.5f * (u1[b][c] - um[b][c]);
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                S6[0][c] = du[0][0][c];
                S6[1][c] = du[1][1][c];
                S6[2][c] = du[2][2][c];
                S6[3][c] = 0.5f * (du[0][1][c] + du[1][0][c]);
                S6[4][c] = 0.5f * (du[0][2][c] + du[2][0][c]);
                S6[5][c] = 0.5f * (du[1][2][c] + du[2][1][c]);
            }
        }
        // learned closure: the network's m_sgs of the four cells, one cell slot
        // of every lane per warp-wide forward (32 rows)
        float msg[4][6];
        if constexpr (LEARNED) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float P6[6] = {P0[0][c], P0[1][c], P0[2][c], P0[3][c], P0[4][c], P0[5][c]};
                v4_learned_msgs(P6, dr0[c], uo[0][c], uo[1][c], uo[2][c], S6[0][c], S6[1][c], S6[2][c], S6[3][c],
                                S6[4][c], S6[5][c], tau_hat, sm_mlp, sm_xch, lane, msg[c]);
            }
        }
        if constexpr (CL == CL_KCRR) {
            // KC-RR (App. F.4): its Hermite-space collision needs all 27 populations
            // of a cell at once, so the cells go one at a time: the cell's 27 TMEM
            // columns (12 p + 4 k + c) into registers, collide_kcrr, the results
            // back into the same columns; then every population's four results
            // leave as one vector store, as in the other closures' relaxation
            const uint32_t ts = tslot(z);
            const int cell = z * plane + gyw * nx + xaw;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (own_store && !isfinite(dr0[c] + uo[0][c] + uo[1][c] + uo[2][c])) atomicOr(a.flag, kFlagNonfinite);
                uint32_t r[27];
#pragma unroll
                for (int i = 0; i < 27; ++i) tm_ld1_issue(ts + (uint32_t)(12 * (i / 3) + 4 * (i % 3) + c), r[i]);
                tm_ld_wait9(r);
                tm_ld_wait9(r + 9);
                tm_ld_wait9(r + 18);
                float g[27];
#pragma unroll
                for (int i = 0; i < 27; ++i) g[i] = __uint_as_float(r[i]);
                collide_kcrr<float>(g, dr0[c], uo[0][c], uo[1][c], uo[2][c], S6[0][c], S6[1][c], S6[2][c], S6[3][c],
                                    S6[4][c], S6[5][c], omega, tau_hat, nu, cnud);
#pragma unroll
                for (int i = 0; i < 27; ++i)
                    tm_st1(ts + (uint32_t)(12 * (i / 3) + 4 * (i % 3) + c), __float_as_uint(g[i]));
            }
            tm_wait_st();
            static_for<9>([&](auto PI) {
                constexpr int p = decltype(PI)::value;
                float gp[3][4];
                tm_ld12(ts + 12u * p, gp);
                static_for<3>([&](auto CI) {
                    constexpr int k = decltype(CI)::value, i = 3 * p + k;
                    constexpr float w = (float)weight_of(Q, i);
                    float o[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) o[c] = SHIFTED ? gp[k][c] : gp[k][c] + w;
                    if (own_store) v4_store(fout + ((long long)i * ps + cell), o[0], o[1], o[2], o[3]);
                });
            });
        } else {
            // per-cell relaxation constants
            V4Cell K[4];
            {
                constexpr float a1 = (float)(1.0 / kTheta);
                constexpr float a2 = (float)((1.0 - kTheta) / (2.0 * kTheta * kTheta));
                constexpr float a0 = (float)(-kTheta / (2.0 * kTheta * kTheta));
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (own_store && !isfinite(dr0[c] + uo[0][c] + uo[1][c] + uo[2][c])) atomicOr(a.flag, kFlagNonfinite);
                    const float P6[6] = {P0[0][c], P0[1][c], P0[2][c], P0[3][c], P0[4][c], P0[5][c]};
                    const Coef<float> k = collide_coef<Q, float, CL>(P6, dr0[c], uo[0][c], uo[1][c], uo[2][c], S6[0][c],
                                                                     S6[1][c], S6[2][c], S6[3][c], S6[4][c], S6[5][c],
                                                                     omega, tau_hat, nu, cnud, LEARNED ? msg[c] : nullptr);
                    const float ux = uo[0][c], uy = uo[1][c], uz = uo[2][c];
                    const float ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
                    if constexpr (Q == 27) {
                        K[c].ex[0] = -a1 * ux + a2 * ux2;
                        K[c].ex[1] = a0 * ux2;
                        K[c].ex[2] = a1 * ux + a2 * ux2;
                        K[c].ey[0] = -a1 * uy + a2 * uy2;
                        K[c].ey[1] = a0 * uy2;
                        K[c].ey[2] = a1 * uy + a2 * uy2;
                        K[c].ez[0] = -a1 * uz + a2 * uz2;
                        K[c].ez[1] = a0 * uz2;
                        K[c].ez[2] = a1 * uz + a2 * uz2;
                    } else {
                        K[c].qx = a1 * ux;
                        K[c].qy = a1 * uy;
                        K[c].qz = a1 * uz;
                        K[c].qq = 0.5f * K[c].qx * K[c].qx;
                        K[c].hu = -0.5f * a1 * ((ux2 + uy2) + uz2);
                    }
                    K[c].ca = k.ca;
                    K[c].cb = k.cb;
                    const float c0 = k.c0;
                    if constexpr (CL == CL_BGK) {
#pragma unroll
                        for (int q = 0; q < 5; ++q) K[c].C[q] = c0;
                        K[c].Dxx = K[c].Dxy2 = K[c].Dxz2 = 0.f;
                    } else {
                        const float h0 = -k.t, h1 = k.Myy - k.t, h2 = k.Mzz - k.t, hyz = (k.Myy + k.Mzz) - k.t;
                        K[c].C[0] = c0 + k.D * h0;
                        K[c].C[1] = c0 + k.D * h1;
                        K[c].C[2] = c0 + k.D * h2;
                        K[c].C[3] = c0 + k.D * (hyz + 2.f * k.Myz);
                        K[c].C[4] = c0 + k.D * (hyz - 2.f * k.Myz);
                        K[c].Dxx = k.D * k.Mxx;
                        K[c].Dxy2 = 2.f * k.D * k.Mxy;
                        K[c].Dxz2 = 2.f * k.D * k.Mxz;
                    }
                    if constexpr (WALLS) {
                        // Guo's source over w, P1 (c.F - u.F) + P2 (c.u)(c.F) with P1 = (1 - omega/2)/theta
                        // and P2 = P1/theta: its parts quadratic in c and the constant join the
                        // per-cell quadratic form (the (c_y, c_z) patterns, c_x^2, c_x c_y, c_x c_z),
                        // its part linear in c, uniform over the box, the per-triple constants below
                        const float yF = gp2 * uy * Fy, zF = gp2 * uz * Fz, yzF = gp2 * (uy * Fz + uz * Fy);
                        const float cF = -gp1 * (ux * Fx + uy * Fy + uz * Fz);
                        K[c].C[0] += cF;
                        K[c].C[1] += cF + yF;
                        K[c].C[2] += cF + zF;
                        K[c].C[3] += cF + (yF + zF) + yzF;
                        K[c].C[4] += cF + (yF + zF) - yzF;
                        K[c].Dxx += gp2 * ux * Fx;
                        K[c].Dxy2 += gp2 * (ux * Fy + uy * Fx);
                        K[c].Dxz2 += gp2 * (ux * Fz + uz * Fx);
                    }
                }
            }
            // relaxation, one population triple of the four cells at a time
            {
                const uint32_t ts = tslot(z);
                const int cell = z * plane + gyw * nx + xaw;
                // the triples' populations come from TMEM one triple ahead (PF): the load
                // of triple p + 1 is issued once triple p's has completed (tcgen05.wait::ld
                // waits for all of the thread's loads), and lands while triple p is
                // relaxed and stored and triple p + 1's constants are formed.  Kernels
                // that carry the z-neighbours in registers have no registers for the
                // second triple: they issue each triple's load before forming its
                // constants.
                constexpr bool PF = RZ && !WALLS;
                uint32_t gr[2][12];
                if constexpr (PF) tm_ld12_issue(ts, gr[0]);
                static_for<9>([&](auto PI) {
                    constexpr int p = decltype(PI)::value;
                    constexpr int cy = p % 3 - 1, cz = p / 3 - 1, pat = v4_pat(cy, cz);
                    constexpr int sl = PF ? (p & 1) : 0;
                    if constexpr (!PF) tm_ld12_issue(ts + 12u * p, gr[0]);
                    float Y[4], B[4], Cm[4], Cp[4], Cz[4], YQ[4];
                    // walls: Guo's source part linear in c, P1 (c_y F_y + c_z F_z) on the
                    // triple and P1 F_x c_x
                    float BFg = 0.f;
                    if constexpr (WALLS && cy != 0) BFg += (float)cy * (gp1 * Fy);
                    if constexpr (WALLS && cz != 0) BFg += (float)cz * (gp1 * Fz);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        if constexpr (Q == 27) {  // P - 1 = e_x (1 + Y) + Y along the triple
                            const float ey = K[c].ey[cy + 1], ez = K[c].ez[cz + 1];
                            Y[c] = fmaf(ey, ez, ey + ez);
                            B[c] = 1.f + Y[c];
                        } else {  // D3Q19: P - 1 = Y + c_x qx (1 + Bq) + c_x^2 qq, B = qx (1 + Bq)
                            float Bq = 0.f;
                            if constexpr (cy != 0) Bq = (float)cy * K[c].qy;
                            if constexpr (cz != 0) Bq = fmaf((float)cz, K[c].qz, Bq);
                            Y[c] = fmaf(0.5f * Bq, Bq, Bq + K[c].hu);
                            B[c] = fmaf(K[c].qx, Bq, K[c].qx);
                            YQ[c] = Y[c] + K[c].qq;
                        }
                        Cz[c] = (WALLS && (cy != 0 || cz != 0)) ? K[c].C[pat] + BFg : K[c].C[pat];
                        if constexpr (CL != CL_BGK || WALLS) {
                            float X = WALLS ? gp1 * Fx : 0.f;
                            if constexpr (cy != 0) X += (float)cy * K[c].Dxy2;
                            if constexpr (cz != 0) X += (float)cz * K[c].Dxz2;
                            const float CpD = Cz[c] + K[c].Dxx;
                            Cp[c] = CpD + X;
                            Cm[c] = CpD - X;
                        } else {
                            Cp[c] = Cm[c] = K[c].C[pat];
                        }
                    }
                    tm_ld12_wait(gr[sl]);
                    float g[3][4];
#pragma unroll
                    for (int q = 0; q < 12; ++q) g[q / 4][q % 4] = __uint_as_float(gr[sl][q]);
                    if constexpr (PF && p < 8) tm_ld12_issue(ts + 12u * (p + 1), gr[(p + 1) & 1]);
                    static_for<3>([&](auto CI) {
                        constexpr int k = decltype(CI)::value;
                        constexpr int cx = k - 1, i = 3 * p + k;
                        if constexpr (!v4_has(Q, i)) return;
                        constexpr float w = (float)weight_of(Q, v4_pop(Q, i));
                        float o[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float pm1 = Q == 27 ? fmaf(K[c].ex[k], B[c], Y[c])
                                                      : (cx == 0 ? Y[c] : (cx == 1 ? YQ[c] + B[c] : YQ[c] - B[c]));
                            const float Cc = cx == 0 ? Cz[c] : (cx == 1 ? Cp[c] : Cm[c]);
                            const float Kv = fmaf(K[c].cb, pm1, Cc);
                            // g' = a g + w K rounded on the scale of g, then (FP32 storage)
                            // f = g' + w in one rounding on the scale of w, as in the
                            // one-cell kernels: w (1 + K) rounded first and a g added after
                            // it rounds twice on the scale of w and drifted the mass
                            const float gq = fmaf(K[c].ca, g[k][c], w * Kv);
                            o[c] = SHIFTED ? gq : gq + w;
                        }
                        if (own_store) v4_store(fout + ((long long)v4_pop(Q, i) * ps + cell), o[0], o[1], o[2], o[3]);
                    });
                });
            }
        }  // analytic closures other than KC-RR
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            dr0[c] = dr1[c];
            if constexpr (!RZ) {
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    um[b][c] = u0[b][c];
                    u0[b][c] = u1[b][c];
                }
            }
#pragma unroll
            for (int q = 0; q < 6; ++q) P0[q][c] = P1[q][c];
        }
    }
    if (!ok) {
        atomicOr(a.flag, kFlagTimeout);
        cp_async_wait<0>();  // the thread's copies in flight land before the CTA leaves
    }
    // every TMEM access of the CTA has completed before warp 0 frees the columns
    tm_wait_st();
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (warp == 0) tm_dealloc(tm_all, 512u);
}

// nx a multiple of 8 (aligned vector rows for 32- and 16-bit storage)
inline bool v4_shape_ok(int nx) { return nx % 8 == 0; }


template <int Q, typename S, int CL, int LPR, int BC = BC_PERIODIC>
cudaError_t prepare_v4_t()
{
    cudaError_t e = cudaFuncSetAttribute(step_kernel_v4<Q, S, CL, LPR, false, BC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)V4Shape<LPR, S, CL == CL_LEARNED, false, BC == BC_WALLS_Y>::smem_bytes);
    if constexpr (CL != CL_LEARNED) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(step_kernel_v4<Q, S, CL, LPR, true, BC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)V4Shape<LPR, S, false, true, BC == BC_WALLS_Y, v4_ring4(true, CL, BC)>::smem_bytes);
    }
    return e;
}

// tma: stage the rows' interior by TMA (variant 16; needs the tensor maps and
// every tile full in x, since the TMA fills outside the box with zeros where
// the cp.async path wraps)
template <int Q, typename S, int CL, int LPR, int BC = BC_PERIODIC>
cudaError_t launch_v4_t(const StepArgs& a, int nbatch, cudaStream_t s, bool tma)
{
    using Sh = V4Shape<LPR, S, CL == CL_LEARNED, false, BC == BC_WALLS_Y>;
    if (!v4_shape_ok(a.nx)) return cudaErrorInvalidValue;
    if (CL == CL_LEARNED && !a.mlp) return cudaErrorInvalidValue;
    if (BC == BC_WALLS_Y && (a.ny < 3 || (a.ny - 1) % Sh::TY == 0)) return cudaErrorInvalidValue;
    static bool attr_set = false;  // per instantiation; prepare_v4_t sets it ahead of stream capture
    if (!attr_set) {
        cudaError_t e = prepare_v4_t<Q, S, CL, LPR, BC>();
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int tiles = ((a.nx + Sh::TX - 1) / Sh::TX) * ((a.ny + Sh::TY - 1) / Sh::TY);
    const int chunks = (a.nz + a.zchunk - 1) / a.zchunk;
    dim3 grid(tiles, chunks, nbatch), block(Sh::NT);
    if (tma) {
        if constexpr (CL != CL_LEARNED) {
            if (!a.tmap_rows || !a.tmap_row1 || !a.tmap_rm1 || !a.tmap_rm2 || a.nx % Sh::TX != 0)
                return cudaErrorInvalidValue;
            step_kernel_v4<Q, S, CL, LPR, true, BC>
                <<<grid, block, V4Shape<LPR, S, false, true, BC == BC_WALLS_Y, v4_ring4(true, CL, BC)>::smem_bytes, s>>>(
                a, *static_cast<const CUtensorMap*>(a.tmap_rows), *static_cast<const CUtensorMap*>(a.tmap_row1),
                *static_cast<const CUtensorMap*>(a.tmap_rm1), *static_cast<const CUtensorMap*>(a.tmap_rm2));
            return cudaGetLastError();
        }
        return cudaErrorNotSupported;
    }
    CUtensorMap none{};
    step_kernel_v4<Q, S, CL, LPR, false, BC><<<grid, block, Sh::smem_bytes, s>>>(a, none, none, none, none);
    return cudaGetLastError();
}

}  // namespace lbmk
