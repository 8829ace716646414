// Allocation-free FP64 diagnostics (lbm_diagnostics_noalloc in include/lbm.h).
//
// Some callers cannot call cudaMalloc: a process whose device memory is all
// owned by another allocator (a framework's caching allocator that hands out
// every byte), code that must not trigger the implicit device synchronisation
// cudaMalloc/cudaFree can cause, or a control loop with a fixed memory budget.
// For them this file provides a variant of the diagnostics reduction that
// allocates nothing: its only scratch is a file-scope device array of
// kNaMaxPlanes * 8 partial sums (one row of eight per z-plane) plus a ticket
// word, about 256 KB that every GPU which loads the library holds until the
// process exits.  Instead of a velocity field in scratch memory it recomputes
// the neighbour velocities of the vorticity stencil from the populations.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/lbm.h"
#include "lbm_internal.h"
#include "lbm_step.cuh"

namespace lbmk {
namespace {

constexpr int kNaMaxPlanes = 4096;  // largest nz the scratch holds
constexpr int kNaVals = 8;
constexpr int kNaBlock = 256;
constexpr int kNaMaxDevices = 64;

// [kNaMaxPlanes][8] per-plane partial sums, then one slot whose first word is
// the ticket counter of the single-pass reduction.  Shared by every call on a
// device; partial rows are overwritten by each call, the ticket is cleared
// before each launch.
static __device__ __align__(256) double g_noalloc_scratch[kNaMaxPlanes * kNaVals + 2];

template <typename S>
__device__ __forceinline__ double na_to_f(S v, double w);
template <>
__device__ __forceinline__ double na_to_f<double>(double v, double)
{
    return v;
}
template <>
__device__ __forceinline__ double na_to_f<float>(float v, double)
{
    return (double)v;
}
template <>
__device__ __forceinline__ double na_to_f<__half>(__half v, double w)
{
    return w + (double)__half2float(v);
}
template <>
__device__ __forceinline__ double na_to_f<__nv_bfloat16>(__nv_bfloat16 v, double w)
{
    return w + (double)__bfloat162float(v);
}

struct NaGeom {
    int nx, ny, nz;
    int bc[3];
    double F[3];
    long long ps;
};

// rho and velocity of the stored (post-collision) populations at one cell:
// rho = sum f, u = (sum f c - F/2)/rho (same convention as lbm_moments)
template <int Q, typename S>
__device__ void na_cell(const S* f, const NaGeom& g, int x, int y, int z, double& rho, double (&u)[3])
{
    const long long c = ((long long)z * g.ny + y) * g.nx + x;
    double d = 0, jx = 0, jy = 0, jz = 0;
    static_for<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
        constexpr double w = weight_of(Q, i);
        const double gi = na_to_f<S>(f[i * g.ps + c], w) - w;
        d += gi;
        jx += cx * gi;
        jy += cy * gi;
        jz += cz * gi;
    });
    rho = 1.0 + d;
    u[0] = (jx - 0.5 * g.F[0]) / rho;
    u[1] = (jy - 0.5 * g.F[1]) / rho;
    u[2] = (jz - 0.5 * g.F[2]) / rho;
}

// d u_b / d axis for the two components b != axis: sixth-order centred
// stencil (3/4, -3/20, 1/60) on periodic axes, second-order central or
// one-sided on bounce-back axes
template <int Q, typename S>
__device__ void na_deriv(const S* f, const NaGeom& g, int axis, int x, int y, int z, double (&du)[3])
{
    const int n = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
    const int p = axis == 0 ? x : (axis == 1 ? y : z);
    auto vel = [&](int k, double (&v)[3]) {
        int xx = x, yy = y, zz = z;
        if (axis == 0) xx = k;
        if (axis == 1) yy = k;
        if (axis == 2) zz = k;
        double r;
        na_cell<Q, S>(f, g, xx, yy, zz, r, v);
    };
    double a[3], b[3];
    du[0] = du[1] = du[2] = 0.0;
    if (g.bc[axis] == LBM_PERIODIC) {
        const double cst[3] = {0.75, -0.15, 1.0 / 60.0};
        for (int k = 1; k <= 3; ++k) {
            vel(wrapi(p + k, n), a);
            vel(wrapi(p - k, n), b);
            for (int c = 0; c < 3; ++c) du[c] += cst[k - 1] * (a[c] - b[c]);
        }
        return;
    }
    double m[3];
    if (p > 0 && p < n - 1) {
        vel(p + 1, a);
        vel(p - 1, b);
        for (int c = 0; c < 3; ++c) du[c] = 0.5 * (a[c] - b[c]);
    } else if (p == 0) {
        vel(0, m);
        vel(1, a);
        vel(2, b);
        for (int c = 0; c < 3; ++c) du[c] = 0.5 * (-3.0 * m[c] + 4.0 * a[c] - b[c]);
    } else {
        vel(n - 1, m);
        vel(n - 2, a);
        vel(n - 3, b);
        for (int c = 0; c < 3; ++c) du[c] = 0.5 * (3.0 * m[c] - 4.0 * a[c] + b[c]);
    }
}

// One block per z-plane: per-plane partial sums into the scratch rows, then the
// last block to finish (ticket) adds the rows in plane order into out.
template <int Q, typename S>
__global__ void __launch_bounds__(kNaBlock) na_diag_kernel(const S* f, NaGeom g, double* scratch, double* out)
{
    const int z = blockIdx.x;
    const long long plane = (long long)g.nx * g.ny;
    double acc[kNaVals] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long c = threadIdx.x; c < plane; c += blockDim.x) {
        const int x = (int)(c % g.nx), y = (int)(c / g.nx);
        double r, u[3];
        na_cell<Q, S>(f, g, x, y, z, r, u);
        if (!(isfinite(r) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]))) {
            acc[6] += 1.0;
            continue;
        }
        acc[0] += r;
        acc[1] += r * u[0];
        acc[2] += r * u[1];
        acc[3] += r * u[2];
        const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        acc[4] += 0.5 * r * usq;
        double dx[3], dy[3], dz[3];
        na_deriv<Q, S>(f, g, 0, x, y, z, dx);
        na_deriv<Q, S>(f, g, 1, x, y, z, dy);
        na_deriv<Q, S>(f, g, 2, x, y, z, dz);
        const double wx = dy[2] - dz[1], wy = dz[0] - dx[2], wz = dx[1] - dy[0];
        acc[5] += 0.5 * (wx * wx + wy * wy + wz * wz);
        acc[7] = fmax(acc[7], sqrt(usq));
    }
    __shared__ double red[kNaVals][kNaBlock];
    for (int k = 0; k < kNaVals; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = kNaBlock / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < kNaVals; ++k)
                red[k][threadIdx.x] = (k == 7) ? fmax(red[k][threadIdx.x], red[k][threadIdx.x + s])
                                               : red[k][threadIdx.x] + red[k][threadIdx.x + s];
        __syncthreads();
    }
    __shared__ bool last;
    if (threadIdx.x == 0) {
        for (int k = 0; k < kNaVals; ++k) scratch[z * kNaVals + k] = red[k][0];
        __threadfence();
        unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + kNaMaxPlanes * kNaVals);
        last = atomicAdd(ticket, 1u) == (unsigned int)(g.nz - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double tot[kNaVals] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int p = 0; p < g.nz; ++p)
            for (int k = 0; k < kNaVals; ++k) {
                const double v = __ldcg(scratch + p * kNaVals + k);
                tot[k] = (k == 7) ? fmax(tot[k], v) : tot[k] + v;
            }
        const double N = (double)g.nx * g.ny * g.nz;
        out[0] = tot[0];
        out[1] = tot[1];
        out[2] = tot[2];
        out[3] = tot[3];
        out[4] = tot[4] / N;
        out[5] = tot[5] / N;
        out[6] = tot[6];
        out[7] = tot[7];
    }
}

std::mutex g_na_mu;
void* g_na_ptr[kNaMaxDevices] = {};

// Device address of the scratch array on the current device.  The array's
// host-side name is not a device address, so it is looked up with
// cudaGetSymbolAddress: on every call made outside stream capture (cheap, and
// a device reset that reloaded the module cannot leave a stale address
// behind), and from the per-device cache during capture (the address a call
// outside capture stored there).
cudaError_t na_scratch(cudaStream_t s, double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = p;
    } else if (!g_na_ptr[dev]) {
        return cudaErrorStreamCaptureUnsupported;  // first call on this device during a capture
    }
    *out = static_cast<double*>(g_na_ptr[dev]);
    return cudaSuccess;
}

}  // namespace
}  // namespace lbmk

extern "C" int lbm_diagnostics_noalloc(const void* f_dev, int lattice, int storage, int nx, int ny, int nz,
                                       const int* bc, const double* force, double* out_dev, void* stream)
{
    using namespace lbmk;
    if (!f_dev || !out_dev) return set_last_error(LBM_ERR_ARG, "f_dev and out_dev must be device pointers");
    if (lattice != LBM_D3Q19 && lattice != LBM_D3Q27) return set_last_error(LBM_ERR_ARG, "lattice must be 19 or 27");
    if (nx < 1 || ny < 1 || nz < 1) return set_last_error(LBM_ERR_ARG, "sizes must be >= 1");
    if (nz > kNaMaxPlanes)
        return set_last_error(LBM_ERR_ARG, "lbm_diagnostics_noalloc: nz exceeds 4096, the number of z-planes its "
                                           "static scratch holds");
    if ((long long)nx * ny * nz >= (1LL << 31) - 1) return set_last_error(LBM_ERR_ARG, "a box must hold fewer than 2^31 cells");
    NaGeom g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.ps = (long long)nx * ny * nz;
    for (int a = 0; a < 3; ++a) {
        g.bc[a] = bc ? bc[a] : LBM_PERIODIC;
        g.F[a] = force ? force[a] : 0.0;
        if (g.bc[a] != LBM_PERIODIC && g.bc[a] != LBM_BOUNCEBACK) return set_last_error(LBM_ERR_ARG, "unknown bc");
        const int n = a == 0 ? nx : (a == 1 ? ny : nz);
        if (g.bc[a] == LBM_BOUNCEBACK && n < 3) return set_last_error(LBM_ERR_ARG, "a bounce-back axis needs >= 3 cells");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* scratch = nullptr;
    cudaError_t e = na_scratch(s, &scratch);
    if (e != cudaSuccess)
        return set_last_error(LBM_ERR_CUDA, (std::string("scratch address lookup failed: ") + cudaGetErrorString(e)).c_str());
    e = cudaMemsetAsync(scratch + kNaMaxPlanes * kNaVals, 0, sizeof(double), s);  // ticket
    if (e != cudaSuccess)
        return set_last_error(LBM_ERR_CUDA, (std::string("clearing the ticket failed: ") + cudaGetErrorString(e)).c_str());
    auto launch = [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        if (lattice == 27)
            na_diag_kernel<27, S><<<nz, kNaBlock, 0, s>>>(static_cast<const S*>(f_dev), g, scratch, out_dev);
        else
            na_diag_kernel<19, S><<<nz, kNaBlock, 0, s>>>(static_cast<const S*>(f_dev), g, scratch, out_dev);
        return cudaGetLastError();
    };
    switch (storage) {
    case LBM_FP64: e = launch((double*)nullptr); break;
    case LBM_FP32: e = launch((float*)nullptr); break;
    case LBM_FP16_SHIFTED: e = launch((__half*)nullptr); break;
    case LBM_BF16_SHIFTED: e = launch((__nv_bfloat16*)nullptr); break;
    default: return set_last_error(LBM_ERR_ARG, "unknown storage");
    }
    if (e != cudaSuccess)
        return set_last_error(LBM_ERR_CUDA, (std::string("diagnostics launch failed: ") + cudaGetErrorString(e)).c_str());
    return LBM_OK;
}
