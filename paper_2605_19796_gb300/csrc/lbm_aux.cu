// Auxiliary kernels of liblbm: equilibrium initialisation, moments, storage
// conversions and the FP64 diagnostics reduction.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_internal.h"
#include "lbm_lattice.cuh"
#include "lbm_step.cuh"
#include "lbm_equilibrium.cuh"
#include "lbm_mbarrier.cuh"

namespace lbmk {

namespace {

// storage value <-> FP64 population f (un-shifted)
template <typename S>
__device__ __forceinline__ double to_f(S v, double w);
template <>
__device__ __forceinline__ double to_f<double>(double v, double)
{
    return v;
}
template <>
__device__ __forceinline__ double to_f<float>(float v, double)
{
    return (double)v;
}
template <>
__device__ __forceinline__ double to_f<__half>(__half v, double w)
{
    return w + (double)__half2float(v);
}
template <>
__device__ __forceinline__ double to_f<__nv_bfloat16>(__nv_bfloat16 v, double w)
{
    return w + (double)__bfloat162float(v);
}

template <typename S>
__device__ __forceinline__ S from_f(double f, double w);
template <>
__device__ __forceinline__ double from_f<double>(double f, double)
{
    return f;
}
template <>
__device__ __forceinline__ float from_f<float>(double f, double)
{
    return (float)f;
}
template <>
__device__ __forceinline__ __half from_f<__half>(double f, double w)
{
    return __float2half_rn((float)(f - w));
}
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(double f, double w)
{
    return __float2bfloat16_rn((float)(f - w));
}

// Cells t0 .. t0 + count - 1 of the nbatch x ncell cells; rho [count] and
// u [3][ustride] hold the range's fields (the whole arrays, t0 = 0, or a
// staged chunk), FP64 or FP32 (T).
template <int Q, typename S, typename T>
__global__ void init_kernel(S* f, const T* rho, const T* u, long long ncell, long long ps, long long bs,
                            long long t0, long long count, long long ustride)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count; t += (long long)gridDim.x * blockDim.x) {
        const long long T = t0 + t;
        const long long box = T / ncell, c = T - box * ncell;
        const double r = rho ? (double)rho[t] : 1.0;
        S* fb = f + box * bs + c;
        if constexpr (sizeof(S) == 8) {
            double geq[Q];
            equilibrium_g<Q>(r, (double)u[t], (double)u[ustride + t], (double)u[2 * ustride + t], geq);
            static_for<Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr double w = weight_of(Q, i);
                fb[i * ps] = from_f<S>(w + geq[i], w);
            });
        } else {
            // FP32 arithmetic for FP32 and 16-bit storage (FP64 arithmetic is
            // slow on this GPU and the stored values carry FP32 precision at
            // most); FP32 f is stored as g + w, as the step kernels store it
            float geq[Q];
            equilibrium_g32<Q>((float)(r - 1.0), (float)u[t], (float)u[ustride + t], (float)u[2 * ustride + t], geq);
            static_for<Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                store_g<S, float>(fb + i * ps, geq[i], (float)weight_of(Q, i));
            });
        }
    }
}

// rho = sum f, u = (sum f c - F/2)/rho: the post-collision array carries the
// momentum of time n plus the full force impulse, so the half-force shift is
// subtracted to report the time-n velocity of Guo forcing.
// sum of the FP32-rounded weights (the shift of FP32 arithmetic on stored f)
template <int Q>
__host__ __device__ constexpr double weight_sum_f32()
{
    double s = 0.0;
    for (int i = 0; i < Q; ++i) s += (double)(float)weight_of(Q, i);
    return s;
}

// F32: FP32 arithmetic for 32- and 16-bit storage (the readback path); the
// diagnostics keep FP64 sums.  O: FP64 or FP32 output fields.
template <int Q, typename S, bool F32, typename O>
__global__ void moments_kernel(const S* f, O* rho, O* u, long long ncell, long long ps, long long bs,
                               double Fx, double Fy, double Fz, long long t0, long long count, long long ustride)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count; t += (long long)gridDim.x * blockDim.x) {
        const long long T = t0 + t;
        const long long box = T / ncell, c = T - box * ncell;
        const S* fb = f + box * bs + c;
        if constexpr (F32 && sizeof(S) != 8) {
            // g = f - w(FP32) is exact in FP32 (Sterbenz) or the stored 16-bit
            // value; the x-triple sums of the step kernels; rho = sum f in FP64
            // as sum g + sum w(FP32) for FP32 storage (1 + sum g for the
            // weight-shifted 16-bit storage)
            float g[Q];
            static_for<Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                g[i] = load_g<S, float>(fb + i * ps, (float)weight_of(Q, i));
            });
            float d32, vx, vy, vz;
            moments<Q, float>(g, d32, vx, vy, vz, (float)-Fx, (float)-Fy, (float)-Fz);
            if (rho) rho[t] = (O)((sizeof(S) == 4 ? weight_sum_f32<Q>() : 1.0) + (double)d32);
            if (u) {
                u[t] = (O)vx;
                u[ustride + t] = (O)vy;
                u[2 * ustride + t] = (O)vz;
            }
            continue;
        }
        double d = 0, jx = 0, jy = 0, jz = 0;
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
            constexpr double w = weight_of(Q, i);
            const double g = to_f<S>(fb[i * ps], w) - w;
            d += g;
            jx += cx * g;
            jy += cy * g;
            jz += cz * g;
        });
        const double r = 1.0 + d;
        if (rho) rho[t] = (O)r;
        if (u) {
            u[t] = (O)((jx - 0.5 * Fx) / r);
            u[ustride + t] = (O)((jy - 0.5 * Fy) / r);
            u[2 * ustride + t] = (O)((jz - 0.5 * Fz) / r);
        }
    }
}

template <int Q, typename S>
__global__ void to_f64_kernel(const S* f, double* out, long long ncell, int nbatch, long long ps, long long bs)
{
    const long long total = ncell * nbatch;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const long long box = t / ncell, c = t - box * ncell;
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const long long k = box * bs + i * ps + c;
            out[k] = to_f<S>(f[k], weight_of(Q, i));
        });
    }
}

template <int Q, typename S>
__global__ void from_f64_kernel(S* f, const double* in, long long ncell, int nbatch, long long ps, long long bs)
{
    const long long total = ncell * nbatch;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const long long box = t / ncell, c = t - box * ncell;
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const long long k = box * bs + i * ps + c;
            f[k] = from_f<S>(in[k], weight_of(Q, i));
        });
    }
}

template <int Q, typename S>
__global__ void probe_kernel(const S* f, const int* xyz, int ncells, int nx, int ny, int nz, long long ps, double* out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncells) return;
    const int x = wrapi(xyz[3 * t], nx), y = wrapi(xyz[3 * t + 1], ny), z = wrapi(xyz[3 * t + 2], nz);
    const long long c = ((long long)z * ny + y) * nx + x;
    static_for<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        out[(long long)t * Q + i] = to_f<S>(f[i * ps + c], weight_of(Q, i));
    });
}

int grid_for(long long n, int block)
{
    long long g = (n + block - 1) / block;
    if (g > 152LL * 32) g = 152LL * 32;
    if (g < 1) g = 1;
    return (int)g;
}

template <typename F>
cudaError_t dispatch_storage(int storage, F&& f)
{
    switch (storage) {
    case ST_F64: return f((double*)nullptr);
    case ST_F32: return f((float*)nullptr);
    case ST_F16S: return f((__half*)nullptr);
    case ST_BF16S: return f((__nv_bfloat16*)nullptr);
    default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ diagnostics

constexpr int kDiagBlock = 256;
constexpr int kDiagVals = 8;

__device__ __forceinline__ double u_at(const double* u, long long N, int comp, int x, int y, int z, int nx, int ny)
{
    return u[comp * N + ((long long)z * ny + y) * nx + x];
}

// d u_comp / d axis at (x,y,z): sixth-order centred on periodic axes
// (coefficients 3/4, -3/20, 1/60), second-order central / one-sided on wall axes
__device__ double deriv(const double* u, long long N, int comp, int axis, int x, int y, int z, int nx, int ny, int nz,
                        const int* bcs)
{
    const int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
    const int p = axis == 0 ? x : (axis == 1 ? y : z);
    auto at = [&](int k) {
        int xx = x, yy = y, zz = z;
        if (axis == 0) xx = k;
        if (axis == 1) yy = k;
        if (axis == 2) zz = k;
        return u_at(u, N, comp, xx, yy, zz, nx, ny);
    };
    if (bcs[axis] == 0) {
        const double c1 = 0.75, c2 = -0.15, c3 = 1.0 / 60.0;
        return c1 * (at(wrapi(p + 1, n)) - at(wrapi(p - 1, n))) + c2 * (at(wrapi(p + 2, n)) - at(wrapi(p - 2, n))) +
               c3 * (at(wrapi(p + 3, n)) - at(wrapi(p - 3, n)));
    }
    if (p > 0 && p < n - 1) return 0.5 * (at(p + 1) - at(p - 1));
    if (p == 0) return 0.5 * (-3.0 * at(0) + 4.0 * at(1) - at(2));
    return 0.5 * (3.0 * at(n - 1) - 4.0 * at(n - 2) + at(n - 3));
}

struct DiagBC {
    int b[3];
};

__global__ void __launch_bounds__(kDiagBlock) diag_kernel(const double* rho, const double* u, int nx, int ny, int nz,
                                                          DiagBC bc, double* partials)
{
    const long long N = (long long)nx * ny * nz;
    double acc[kDiagVals] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx);
        const int y = (int)((c / nx) % ny);
        const int z = (int)(c / ((long long)nx * ny));
        const double r = rho[c], ux = u[c], uy = u[N + c], uz = u[2 * N + c];
        const bool fin = isfinite(r) && isfinite(ux) && isfinite(uy) && isfinite(uz);
        if (!fin) {
            acc[6] += 1.0;
            continue;
        }
        acc[0] += r;
        acc[1] += r * ux;
        acc[2] += r * uy;
        acc[3] += r * uz;
        const double usq = ux * ux + uy * uy + uz * uz;
        acc[4] += 0.5 * r * usq;
        const double wx = deriv(u, N, 2, 1, x, y, z, nx, ny, nz, bc.b) - deriv(u, N, 1, 2, x, y, z, nx, ny, nz, bc.b);
        const double wy = deriv(u, N, 0, 2, x, y, z, nx, ny, nz, bc.b) - deriv(u, N, 2, 0, x, y, z, nx, ny, nz, bc.b);
        const double wz = deriv(u, N, 1, 0, x, y, z, nx, ny, nz, bc.b) - deriv(u, N, 0, 1, x, y, z, nx, ny, nz, bc.b);
        acc[5] += 0.5 * (wx * wx + wy * wy + wz * wz);
        acc[7] = fmax(acc[7], sqrt(usq));
    }
    __shared__ double red[kDiagVals][kDiagBlock];
#pragma unroll
    for (int k = 0; k < kDiagVals; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = kDiagBlock / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
#pragma unroll
            for (int k = 0; k < kDiagVals; ++k) {
                if (k == 7)
                    red[k][threadIdx.x] = fmax(red[k][threadIdx.x], red[k][threadIdx.x + s]);
                else
                    red[k][threadIdx.x] += red[k][threadIdx.x + s];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < kDiagVals) partials[blockIdx.x * kDiagVals + threadIdx.x] = red[threadIdx.x][0];
}

// single-block, fixed-order (deterministic) sum of the per-block partials
__global__ void diag_final_kernel(const double* partials, int nblocks, long long N, double* out)
{
    __shared__ double red[kDiagVals][kDiagBlock];
    double acc[kDiagVals] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < kDiagVals; ++k) {
            const double v = partials[b * kDiagVals + k];
            acc[k] = (k == 7) ? fmax(acc[k], v) : acc[k] + v;
        }
    }
#pragma unroll
    for (int k = 0; k < kDiagVals; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = kDiagBlock / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
#pragma unroll
            for (int k = 0; k < kDiagVals; ++k)
                red[k][threadIdx.x] = (k == 7) ? fmax(red[k][threadIdx.x], red[k][threadIdx.x + s])
                                               : red[k][threadIdx.x] + red[k][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = red[0][0];
        out[1] = red[1][0];
        out[2] = red[2][0];
        out[3] = red[3][0];
        out[4] = red[4][0] / (double)N;
        out[5] = red[5][0] / (double)N;
        out[6] = red[6][0];
        out[7] = red[7][0];
    }
}

// ------------------------------------------------------------ dissipation
//
// Dissipation rates of the state the next step collides (a reading: the
// paper reports E_k and enstrophy, Sec. 7.1, and is silent on the
// dissipation): the stored populations pull-streamed (Eq. streaming;
// halfway bounce-back across y walls), then at every node rho, u (App. F.1
// step 1, with the half-force shift), the strain of Eqs. (fd),
// (fd_boundary_lower/upper), (strain_rate_discrete), the closure's clipped
// rate omega_s (Eq. omega_sgs_operational) and nu_eff = theta (1/omega_s -
// 1/2); the reductions are <2 rho nu_eff S:S> and <2 rho nu S:S> in FP64.

// drho = sum g, u, and sum g |c|^2 (g = f - w: the sums stay small, so the
// trace of m_neq below is free of O(1) cancellation) of the streamed state
template <int Q, typename S>
__global__ void pull_moments_kernel(const S* f, int nx, int ny, int nz, int walls, double Fx, double Fy, double Fz,
                                    double* drho, double* u, double* s2)
{
    const long long N = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
        double d = 0, jx = 0, jy = 0, jz = 0, e2 = 0;
        static_for<Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i), io = opp_of(Q, i);
            constexpr double w = weight_of(Q, i);
            const int sy = y - cy;
            long long src;
            if (walls && (sy < 0 || sy >= ny))
                src = (long long)io * N + c;  // halfway bounce-back
            else
                src = (long long)i * N + ((long long)wrapi(z - cz, nz) * ny + wrapi(sy, ny)) * nx + wrapi(x - cx, nx);
            const double g = to_f<S>(f[src], w) - w;
            d += g;
            jx += cx * g;
            jy += cy * g;
            jz += cz * g;
            e2 += (cx * cx + cy * cy + cz * cz) * g;
        });
        const double r = 1.0 + d;
        drho[c] = d;
        u[c] = (jx + 0.5 * Fx) / r;
        u[N + c] = (jy + 0.5 * Fy) / r;
        u[2 * N + c] = (jz + 0.5 * Fz) / r;
        s2[c] = e2;
    }
}

constexpr int kDissBlock = 256;

__global__ void __launch_bounds__(kDissBlock) dissip_kernel(const double* drho, const double* u, const double* s2,
                                                            int nx, int ny, int nz, int walls, int closure, double nu,
                                                            double cnud, double* partials)
{
    const long long N = (long long)nx * ny * nz;
    constexpr double th = kTheta;
    const double tau_hat = nu / th + 0.5, omega = 1.0 / tau_hat;
    double ee = 0.0, em = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
        auto U = [&](int b, int xx, int yy, int zz) { return u[b * N + ((long long)zz * ny + yy) * nx + xx]; };
        double du[3][3];  // du[a][b] = d_a u_b
        for (int b = 0; b < 3; ++b) {
            du[0][b] = (U(b, wrapi(x + 1, nx), y, z) - U(b, wrapi(x - 1, nx), y, z)) / 2.0;
            du[2][b] = (U(b, x, y, wrapi(z + 1, nz)) - U(b, x, y, wrapi(z - 1, nz))) / 2.0;
            if (walls && y == 0)
                du[1][b] = (-3.0 * U(b, x, 0, z) + 4.0 * U(b, x, 1, z) - U(b, x, 2, z)) / 2.0;
            else if (walls && y == ny - 1)
                du[1][b] = (3.0 * U(b, x, ny - 1, z) - 4.0 * U(b, x, ny - 2, z) + U(b, x, ny - 3, z)) / 2.0;
            else
                du[1][b] = (U(b, x, wrapi(y + 1, ny), z) - U(b, x, wrapi(y - 1, ny), z)) / 2.0;
        }
        double S[3][3], ss = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                S[a][b] = 0.5 * (du[b][a] + du[a][b]);
                ss += S[a][b] * S[a][b];
            }
        const double r = 1.0 + drho[c];
        const double ux = u[c], uy = u[N + c], uz = u[2 * N + c];
        double omega_s = omega;
        if (closure == CL_LEARNED) {
            omega_s = nan("");
        } else if (closure != CL_BGK) {
            // tr m_neq = sum f |c|^2 - rho (|u|^2 + 3 theta) = sum g |c|^2 - rho |u|^2 - 3 theta drho
            const double trneq = s2[c] - r * (ux * ux + uy * uy + uz * uz) - 3.0 * th * drho[c];
            const double trS = S[0][0] + S[1][1] + S[2][2];
            // KC-MP, KC-RR: tr (m_neq - m_CE), m_CE = -2 rho theta tau_hat S; KC-RB:
            // tr (f - f0 - f1) |c|^2 with sum f1 |c|^2 = -2 (Hermite) or -5 (raw) rho tau_hat theta tr S
            const double tr = trneq + (closure == CL_KCRB_RAW ? 5.0 : 2.0) * r * th * tau_hat * trS;
            const double nut = cnud * sqrt(fabs(tr) / 2.0);
            if (nut > nu) omega_s = 1.0 / (nut / th + 0.5);
        }
        const double nu_eff = th * (1.0 / omega_s - 0.5);
        ee += 2.0 * r * nu_eff * ss;
        em += 2.0 * r * nu * ss;
    }
    __shared__ double red[2][kDissBlock];
    red[0][threadIdx.x] = ee;
    red[1][threadIdx.x] = em;
    __syncthreads();
    for (int s = kDissBlock / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x < 2) partials[blockIdx.x * 2 + threadIdx.x] = red[threadIdx.x][0];
}

// single-block, fixed-order sum of the partials; out[0], out[1] = the averages
__global__ void dissip_final_kernel(const double* partials, int nblocks, long long N, double* out)
{
    __shared__ double red[2][kDissBlock];
    double a0 = 0.0, a1 = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        a0 += partials[b * 2];
        a1 += partials[b * 2 + 1];
    }
    red[0][threadIdx.x] = a0;
    red[1][threadIdx.x] = a1;
    __syncthreads();
    for (int s = kDissBlock / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = red[0][0] / (double)N;
        out[1] = red[1][0] / (double)N;
    }
}

int diag_blocks(long long ncell)
{
    long long b = (ncell + kDiagBlock - 1) / kDiagBlock;
    if (b > 152LL * 8) b = 152LL * 8;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

template <typename T>
cudaError_t init_equilibrium_t(int q, int storage, void* f, const T* rho, const T* u, long long ncell, int nbatch,
                               long long ps, long long bs, cudaStream_t s, long long t0, long long count,
                               long long ustride)
{
    if (count < 0) count = ncell * nbatch;
    if (ustride < 0) ustride = count;
    const int g = grid_for(count, 256);
    return dispatch_storage(storage, [&](auto tag) -> cudaError_t {
        using S = std::remove_pointer_t<decltype(tag)>;
        if (q == 27)
            init_kernel<27, S, T><<<g, 256, 0, s>>>((S*)f, rho, u, ncell, ps, bs, t0, count, ustride);
        else
            init_kernel<19, S, T><<<g, 256, 0, s>>>((S*)f, rho, u, ncell, ps, bs, t0, count, ustride);
        return cudaGetLastError();
    });
}

cudaError_t launch_init_equilibrium(int q, int storage, void* f, const double* rho, const double* u, long long ncell,
                                    int nbatch, long long ps, long long bs, cudaStream_t s, long long t0,
                                    long long count, long long ustride)
{
    return init_equilibrium_t<double>(q, storage, f, rho, u, ncell, nbatch, ps, bs, s, t0, count, ustride);
}

cudaError_t launch_init_equilibrium(int q, int storage, void* f, const float* rho, const float* u, long long ncell,
                                    int nbatch, long long ps, long long bs, cudaStream_t s, long long t0,
                                    long long count, long long ustride)
{
    return init_equilibrium_t<float>(q, storage, f, rho, u, ncell, nbatch, ps, bs, s, t0, count, ustride);
}

// Self-test of the bounded-wait error path: one thread waits on an mbarrier
// phase that nothing completes; the bounded wait gives up after `polls` polls
// and records the timeout bit in the status flag, as a step kernel would.
__global__ void wait_selftest_kernel(unsigned int* flag, long long polls)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        if (!mbar_wait_polls(&bar, 0u, polls)) atomicOr(flag, kFlagTimeout);
    }
}

cudaError_t launch_wait_selftest(unsigned int* flag, long long polls, cudaStream_t s)
{
    wait_selftest_kernel<<<1, 32, 0, s>>>(flag, polls);
    return cudaGetLastError();
}

template <typename O>
cudaError_t moments_t(int q, int storage, const void* f, O* rho, O* u, long long ncell, int nbatch, long long ps,
                      long long bs, const double* force, cudaStream_t s, bool fp32, long long t0, long long count,
                      long long ustride)
{
    if (count < 0) count = ncell * nbatch;
    if (ustride < 0) ustride = count;
    const int g = grid_for(count, 256);
    return dispatch_storage(storage, [&](auto tag) -> cudaError_t {
        using S = std::remove_pointer_t<decltype(tag)>;
        const double F0 = force[0], F1 = force[1], F2 = force[2];
        if (q == 27) {
            if (fp32)
                moments_kernel<27, S, true, O><<<g, 256, 0, s>>>((const S*)f, rho, u, ncell, ps, bs, F0, F1, F2, t0, count, ustride);
            else
                moments_kernel<27, S, false, O><<<g, 256, 0, s>>>((const S*)f, rho, u, ncell, ps, bs, F0, F1, F2, t0, count, ustride);
        } else {
            if (fp32)
                moments_kernel<19, S, true, O><<<g, 256, 0, s>>>((const S*)f, rho, u, ncell, ps, bs, F0, F1, F2, t0, count, ustride);
            else
                moments_kernel<19, S, false, O><<<g, 256, 0, s>>>((const S*)f, rho, u, ncell, ps, bs, F0, F1, F2, t0, count, ustride);
        }
        return cudaGetLastError();
    });
}

cudaError_t launch_moments(int q, int storage, const void* f, double* rho, double* u, long long ncell, int nbatch,
                           long long ps, long long bs, const double* force, cudaStream_t s, bool fp32, long long t0,
                           long long count, long long ustride)
{
    return moments_t<double>(q, storage, f, rho, u, ncell, nbatch, ps, bs, force, s, fp32, t0, count, ustride);
}

cudaError_t launch_moments(int q, int storage, const void* f, float* rho, float* u, long long ncell, int nbatch,
                           long long ps, long long bs, const double* force, cudaStream_t s, long long t0,
                           long long count, long long ustride)
{
    return moments_t<float>(q, storage, f, rho, u, ncell, nbatch, ps, bs, force, s, true, t0, count, ustride);
}

cudaError_t launch_to_f64(int q, int storage, const void* f, double* out, long long ncell, int nbatch, long long ps,
                          long long bs, cudaStream_t s)
{
    const int g = grid_for(ncell * nbatch, 256);
    return dispatch_storage(storage, [&](auto tag) -> cudaError_t {
        using S = std::remove_pointer_t<decltype(tag)>;
        if (q == 27)
            to_f64_kernel<27, S><<<g, 256, 0, s>>>((const S*)f, out, ncell, nbatch, ps, bs);
        else
            to_f64_kernel<19, S><<<g, 256, 0, s>>>((const S*)f, out, ncell, nbatch, ps, bs);
        return cudaGetLastError();
    });
}

cudaError_t launch_from_f64(int q, int storage, void* f, const double* in, long long ncell, int nbatch, long long ps,
                            long long bs, cudaStream_t s)
{
    const int g = grid_for(ncell * nbatch, 256);
    return dispatch_storage(storage, [&](auto tag) -> cudaError_t {
        using S = std::remove_pointer_t<decltype(tag)>;
        if (q == 27)
            from_f64_kernel<27, S><<<g, 256, 0, s>>>((S*)f, in, ncell, nbatch, ps, bs);
        else
            from_f64_kernel<19, S><<<g, 256, 0, s>>>((S*)f, in, ncell, nbatch, ps, bs);
        return cudaGetLastError();
    });
}

cudaError_t launch_probe(int q, int storage, const void* f, const int* xyz, int ncells, int nx, int ny, int nz,
                         long long ps, double* out, cudaStream_t s)
{
    const int g = (ncells + 127) / 128;
    return dispatch_storage(storage, [&](auto tag) -> cudaError_t {
        using S = std::remove_pointer_t<decltype(tag)>;
        if (q == 27)
            probe_kernel<27, S><<<g, 128, 0, s>>>((const S*)f, xyz, ncells, nx, ny, nz, ps, out);
        else
            probe_kernel<19, S><<<g, 128, 0, s>>>((const S*)f, xyz, ncells, nx, ny, nz, ps, out);
        return cudaGetLastError();
    });
}

long long diag_partials_len(long long ncell) { return (long long)diag_blocks(ncell) * kDiagVals; }

cudaError_t launch_diagnostics(const double* rho, const double* u, int nx, int ny, int nz, const int* bc,
                               double* partials, double* out_dev, cudaStream_t s)
{
    const long long N = (long long)nx * ny * nz;
    const int nb = diag_blocks(N);
    DiagBC b;
    for (int k = 0; k < 3; ++k) b.b[k] = bc[k];
    diag_kernel<<<nb, kDiagBlock, 0, s>>>(rho, u, nx, ny, nz, b, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final_kernel<<<1, kDiagBlock, 0, s>>>(partials, nb, N, out_dev);
    return cudaGetLastError();
}

cudaError_t launch_dissipation(int q, int storage, const void* f, int nx, int ny, int nz, int walls, const double* force,
                               int closure, double nu, double cnud, double* drho, double* u, double* s2,
                               double* partials, double* out_dev, cudaStream_t s)
{
    const long long N = (long long)nx * ny * nz;
    const int g = grid_for(N, 256);
    cudaError_t e = dispatch_storage(storage, [&](auto tag) -> cudaError_t {
        using S = std::remove_pointer_t<decltype(tag)>;
        if (q == 27)
            pull_moments_kernel<27, S><<<g, 256, 0, s>>>((const S*)f, nx, ny, nz, walls, force[0], force[1], force[2],
                                                         drho, u, s2);
        else
            pull_moments_kernel<19, S><<<g, 256, 0, s>>>((const S*)f, nx, ny, nz, walls, force[0], force[1], force[2],
                                                         drho, u, s2);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    const int nb = diag_blocks(N);
    dissip_kernel<<<nb, kDissBlock, 0, s>>>(drho, u, s2, nx, ny, nz, walls, closure, nu, cnud, partials);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dissip_final_kernel<<<1, kDissBlock, 0, s>>>(partials, nb, N, out_dev);
    return cudaGetLastError();
}

}  // namespace lbmk
