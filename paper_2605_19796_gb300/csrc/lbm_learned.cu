// Learned closure: training data (box filter, exact SGS stress, KC-MP-derived
// inputs) and the multilayer perceptron's forward, backward and AdamW kernels.
//
// Network (per cell): x (10) -> standardise -> 3 x [64, SiLU] -> 6 outputs,
// the standardised m_sgs / rho.  Parameters are one flat FP32 vector in the
// order W1 b1 W2 b2 W3 b3 W4 b4 (W row-major [out][in]); the standardisation
// statistics are kept apart (mean and std of the 10 inputs and 6 outputs).
#include <cuda_runtime.h>

#include <string>

#include "../../include/lbm.h"
#include "lbm_internal.h"
#include "lbm_step.cuh"
#include "lbm_equilibrium.cuh"
#include "lbm_mlp_infer.cuh"

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

namespace lbmk {
namespace {

constexpr int kIn = 10, kH = 64, kOut = 6;
__host__ __device__ constexpr int layer_in(int l) { return l == 0 ? kIn : kH; }
__host__ __device__ constexpr int layer_out(int l) { return l == 3 ? kOut : kH; }

__host__ __device__ constexpr int w_off(int l)
{
    int o = 0;
    for (int k = 0; k < l; ++k) o += layer_in(k) * layer_out(k) + layer_out(k);
    return o;
}
__host__ __device__ constexpr int b_off(int l) { return w_off(l) + layer_in(l) * layer_out(l); }
constexpr int kNParam = w_off(4);
static_assert(kNParam == 9414, "10-64-64-64-6 network");

__device__ __forceinline__ float silu(float a) { return a / (1.0f + __expf(-a)); }
__device__ __forceinline__ float silu_grad(float a)
{
    const float s = 1.0f / (1.0f + __expf(-a));
    return s * (1.0f + a * (1.0f - s));
}

// ---------------------------------------------------------------- box filter

// One thread per coarse cell: filtered populations (average of F^3 fine
// cells) and the exact SGS stress of Eq. (m_sgs_2),
// m_sgs = bar(rho u u) - bar(rho u) bar(rho u) / rho_bar.
template <int Q, typename S>
__global__ void filter_kernel(const S* f, int nx, int ny, int nz, int F, double neq_scale, int pull, float* fc,
                              float* msgs)
{
    const int ncx = nx / F, ncy = ny / F, ncz = nz / F;
    const long long Nc = (long long)ncx * ncy * ncz, N = (long long)nx * ny * nz;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= Nc) return;
    const int cx = (int)(t % ncx), cy = (int)((t / ncx) % ncy), cz = (int)(t / ((long long)ncx * ncy));
    double acc[Q], accn[Q];  // filtered populations and filtered f - f0(rho, u) of the fine cells
    for (int i = 0; i < Q; ++i) acc[i] = accn[i] = 0.0;
    const bool rescale = neq_scale != 1.0;
    double r = 0, m[3] = {0, 0, 0}, uu[6] = {0, 0, 0, 0, 0, 0};
    for (int dz = 0; dz < F; ++dz)
        for (int dy = 0; dy < F; ++dy)
            for (int dx = 0; dx < F; ++dx) {
                const int X = cx * F + dx, Y = cy * F + dy, Z = cz * F + dz;
                // population i of this fine cell, or with `pull` its streamed value
                // f_i(x - c_i) (periodic), the pre-collision state of the next step
                auto src = [&](int i, int ex, int ey, int ez) -> long long {
                    if (!pull) return ((long long)Z * ny + Y) * nx + X;
                    const int xs = (X - ex + nx) % nx, ys = (Y - ey + ny) % ny, zs = (Z - ez + nz) % nz;
                    return ((long long)zs * ny + ys) * nx + xs;
                };
                double fv[Q];
                double rr = 0, jx = 0, jy = 0, jz = 0;
                static_for<Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    constexpr double w = weight_of(Q, i);
                    const long long c = src(i, cx_of(Q, i), cy_of(Q, i), cz_of(Q, i));
                    double fi;
                    if constexpr (StoreTraits<S>::shifted)
                        fi = w + (double)load_g<S, float>(f + i * N + c, 0.0f);
                    else
                        fi = (double)f[i * N + c];
                    fv[i] = fi;
                    acc[i] += fi;
                    rr += fi;
                    jx += cx_of(Q, i) * fi;
                    jy += cy_of(Q, i) * fi;
                    jz += cz_of(Q, i) * fi;
                });
                const double ux = jx / rr, uy = jy / rr, uz = jz / rr;
                if (rescale) {
                    double geq[Q];
                    equilibrium_g<Q>(rr, ux, uy, uz, geq);
                    static_for<Q>([&](auto I) {
                        constexpr int i = decltype(I)::value;
                        accn[i] += fv[i] - weight_of(Q, i) - geq[i];
                    });
                }
                r += rr;
                m[0] += jx;
                m[1] += jy;
                m[2] += jz;
                uu[0] += rr * ux * ux;
                uu[1] += rr * uy * uy;
                uu[2] += rr * uz * uz;
                uu[3] += rr * ux * uy;
                uu[4] += rr * ux * uz;
                uu[5] += rr * uy * uz;
            }
    const double inv = 1.0 / ((double)F * F * F);
    for (int i = 0; i < Q; ++i) fc[i * Nc + t] = (float)((acc[i] + (neq_scale - 1.0) * accn[i]) * inv);
    r *= inv;
    for (int k = 0; k < 3; ++k) m[k] *= inv;
    const int A[6] = {0, 1, 2, 0, 0, 1}, B[6] = {0, 1, 2, 1, 2, 2};
    for (int k = 0; k < 6; ++k) msgs[k * Nc + t] = (float)(uu[k] * inv - m[A[k]] * m[B[k]] / r);
}

// ---------------------------------------------------------------- features

template <int Q>
__device__ void cell_moments(const float* f, long long N, long long c, float& rho, float (&u)[3])
{
    double d = 0, jx = 0, jy = 0, jz = 0;
    static_for<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const double g = (double)f[i * N + c] - weight_of(Q, i);
        d += g;
        jx += cx_of(Q, i) * g;
        jy += cy_of(Q, i) * g;
        jz += cz_of(Q, i) * g;
    });
    rho = (float)(1.0 + d);
    u[0] = (float)(jx / (1.0 + d));
    u[1] = (float)(jy / (1.0 + d));
    u[2] = (float)(jz / (1.0 + d));
}

// inputs x [N][10] (and targets t [N][6] when msgs is given) of every cell of
// a population array f (FP32, unshifted, periodic box)
template <int Q>
__global__ void features_kernel(const float* f, int nx, int ny, int nz, float tau_hat, const float* msgs, float* x,
                                float* tgt, float* kcmp)
{
    const long long N = (long long)nx * ny * nz;
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int ix = (int)(c % nx), iy = (int)((c / nx) % ny), iz = (int)(c / ((long long)nx * ny));
    float rho, u[3];
    cell_moments<Q>(f, N, c, rho, u);
    // m_neq = sum (f - f0) c c = Pi - rho (u u + theta I), Pi from the populations
    double P[6] = {0, 0, 0, 0, 0, 0};
    static_for<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int cx = cx_of(Q, i), cy = cy_of(Q, i), cz = cz_of(Q, i);
        const double fi = (double)f[i * N + c];
        P[0] += cx * cx * fi;
        P[1] += cy * cy * fi;
        P[2] += cz * cz * fi;
        P[3] += cx * cy * fi;
        P[4] += cx * cz * fi;
        P[5] += cy * cz * fi;
    });
    const int A[6] = {0, 1, 2, 0, 0, 1}, B[6] = {0, 1, 2, 1, 2, 2};
    float* xr = x + c * 10;
    double mneq[6];  // m_neq / rho
    for (int k = 0; k < 6; ++k)
        mneq[k] = (P[k] - rho * ((double)u[A[k]] * u[B[k]] + (A[k] == B[k] ? kTheta : 0.0))) / rho;
    // S from the central differences of the neighbours' velocities, Eq. (fd)
    float du[3][3];
    const int xp = ix == nx - 1 ? 0 : ix + 1, xm = ix == 0 ? nx - 1 : ix - 1;
    const int yp = iy == ny - 1 ? 0 : iy + 1, ym = iy == 0 ? ny - 1 : iy - 1;
    const int zp = iz == nz - 1 ? 0 : iz + 1, zm = iz == 0 ? nz - 1 : iz - 1;
    const long long nb[3][2] = {{((long long)iz * ny + iy) * nx + xp, ((long long)iz * ny + iy) * nx + xm},
                                {((long long)iz * ny + yp) * nx + ix, ((long long)iz * ny + ym) * nx + ix},
                                {((long long)zp * ny + iy) * nx + ix, ((long long)zm * ny + iy) * nx + ix}};
    for (int a = 0; a < 3; ++a) {
        float rp, up[3], rm, um[3];
        cell_moments<Q>(f, N, nb[a][0], rp, up);
        cell_moments<Q>(f, N, nb[a][1], rm, um);
        for (int b = 0; b < 3; ++b) du[a][b] = 0.5f * (up[b] - um[b]);
    }
    double Am[3][3];  // m_CE / rho = -2 theta tau_hat S
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Am[a][b] = -2.0 * kTheta * tau_hat * 0.5 * ((double)du[a][b] + du[b][a]);
    const double tr = Am[0][0] + Am[1][1] + Am[2][2];
    double tr2 = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) tr2 += Am[a][b] * Am[b][a];
    const double det = Am[0][0] * (Am[1][1] * Am[2][2] - Am[1][2] * Am[2][1]) -
                       Am[0][1] * (Am[1][0] * Am[2][2] - Am[1][2] * Am[2][0]) +
                       Am[0][2] * (Am[1][0] * Am[2][1] - Am[1][1] * Am[2][0]);
    // inputs 0-5: the KC-MP carrier (m_neq - m_CE)/rho (App. F.3), which is also
    // the analytic KC-MP estimate of m_sgs / rho
    for (int k = 0; k < 6; ++k) xr[k] = (float)(mneq[k] - Am[A[k]][B[k]]);
    xr[6] = (float)tr;
    xr[7] = (float)(0.5 * (tr * tr - tr2));
    xr[8] = (float)det;
    xr[9] = tau_hat;
    if (kcmp)
        for (int k = 0; k < 6; ++k) kcmp[c * 6 + k] = xr[k];
    if (msgs && tgt)
        for (int k = 0; k < 6; ++k) tgt[c * 6 + k] = msgs[k * N + c] / rho;
}

// strain rate S (xx yy zz xy xz yz) of every cell of a periodic FP32 population
// array by the central differences of the neighbours' velocities, Eq. (fd),
// as the features kernel forms it
template <int Q>
__global__ void strain_kernel(const float* f, int nx, int ny, int nz, float* s_out)
{
    const long long N = (long long)nx * ny * nz;
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int ix = (int)(c % nx), iy = (int)((c / nx) % ny), iz = (int)(c / ((long long)nx * ny));
    const int xp = ix == nx - 1 ? 0 : ix + 1, xm = ix == 0 ? nx - 1 : ix - 1;
    const int yp = iy == ny - 1 ? 0 : iy + 1, ym = iy == 0 ? ny - 1 : iy - 1;
    const int zp = iz == nz - 1 ? 0 : iz + 1, zm = iz == 0 ? nz - 1 : iz - 1;
    const long long nb[3][2] = {{((long long)iz * ny + iy) * nx + xp, ((long long)iz * ny + iy) * nx + xm},
                                {((long long)iz * ny + yp) * nx + ix, ((long long)iz * ny + ym) * nx + ix},
                                {((long long)zp * ny + iy) * nx + ix, ((long long)zm * ny + iy) * nx + ix}};
    float du[3][3];
    for (int a = 0; a < 3; ++a) {
        float rp, up[3], rm, um[3];
        cell_moments<Q>(f, N, nb[a][0], rp, up);
        cell_moments<Q>(f, N, nb[a][1], rm, um);
        for (int b = 0; b < 3; ++b) du[a][b] = 0.5f * (up[b] - um[b]);
    }
    float* o = s_out + c * 6;
    o[0] = du[0][0];
    o[1] = du[1][1];
    o[2] = du[2][2];
    o[3] = 0.5f * (du[0][1] + du[1][0]);
    o[4] = 0.5f * (du[0][2] + du[2][0]);
    o[5] = 0.5f * (du[1][2] + du[2][1]);
}

// ---------------------------------------------------------------- MLP

// forward of one layer for a batch: A = X W^T + b, H = silu(A) (or H = A for the last layer)
__global__ void mlp_fwd_kernel(const float* __restrict__ X, int n, int in, int out, const float* __restrict__ W,
                               const float* __restrict__ b, float* __restrict__ A, float* __restrict__ H, int act)
{
    __shared__ float Ws[kH * kH + kH];
    for (int k = threadIdx.x; k < out * in; k += blockDim.x) Ws[k] = W[k];
    for (int k = threadIdx.x; k < out; k += blockDim.x) Ws[out * in + k] = b[k];
    __syncthreads();
    const long long total = (long long)n * out;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / out;
        const int o = (int)(t % out);
        float s = Ws[out * in + o];
        const float* xr = X + r * in;
        const float* wr = Ws + o * in;
        for (int k = 0; k < in; ++k) s += xr[k] * wr[k];
        A[t] = s;
        H[t] = act ? silu(s) : s;
    }
}

// loss L = mean (Y - T)^2 over n x 6 values: dY = 2 (Y - T)/(6 n); per-block partial sums of (Y - T)^2
__global__ void mlp_loss_kernel(const float* Y, const float* T, int n, float* dY, double* partial)
{
    __shared__ double red[256];
    double s = 0;
    const long long total = (long long)n * kOut;
    const float scale = 2.0f / (float)total;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const float d = Y[t] - T[t];
        dY[t] = scale * d;
        s += (double)d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// dX = (dA W) * silu'(Aprev): backward through layer l's weights and the previous activation
__global__ void mlp_bwd_data_kernel(const float* __restrict__ dA, int n, int in, int out, const float* __restrict__ W,
                                    const float* __restrict__ Aprev, float* __restrict__ dX)
{
    __shared__ float Ws[kH * kH];
    for (int k = threadIdx.x; k < out * in; k += blockDim.x) Ws[k] = W[k];
    __syncthreads();
    const long long total = (long long)n * in;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / in;
        const int j = (int)(t % in);
        float s = 0;
        const float* dr = dA + r * out;
        for (int o = 0; o < out; ++o) s += dr[o] * Ws[o * in + j];
        dX[t] = s * silu_grad(Aprev[t]);
    }
}

// per-block partial weight gradients: dW[o][k] = sum_r dA[r][o] X[r][k], db[o] = sum_r dA[r][o]
constexpr int kWRows = 256;  // batch rows per block
__global__ void mlp_bwd_weight_kernel(const float* __restrict__ dA, const float* __restrict__ X, int n, int in, int out,
                                      float* __restrict__ partial)
{
    const int r0 = blockIdx.x * kWRows;
    const int r1 = min(n, r0 + kWRows);
    const int np = out * in + out;
    float* p = partial + (long long)blockIdx.x * np;
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
        float s = 0;
        if (e < out * in) {
            const int o = e / in, k = e % in;
            for (int r = r0; r < r1; ++r) s += dA[(long long)r * out + o] * X[(long long)r * in + k];
        } else {
            const int o = e - out * in;
            for (int r = r0; r < r1; ++r) s += dA[(long long)r * out + o];
        }
        p[e] = s;
    }
}
// fixed-order sum of the block partials into the layer's slice of the gradient vector
__global__ void mlp_reduce_kernel(const float* partial, int nblocks, int np, float* grad)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= np) return;
    float s = 0;
    for (int b = 0; b < nblocks; ++b) s += partial[(long long)b * np + e];
    grad[e] = s;
}

// AdamW (decoupled weight decay on the weight matrices only)
__global__ void adamw_kernel(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                             float eps, float wd, float bc1, float bc2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    bool is_w = false;
    for (int l = 0; l < 4; ++l)
        if (k >= w_off(l) && k < b_off(l)) is_w = true;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.0f - b1) * gk;
    const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    float pk = p[k];
    if (is_w && wd != 0.0f) pk -= lr * wd * pk;
    p[k] = pk - lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
}

// tensor-core forward of raw inputs (standardised with the packed statistics):
// each warp evaluates 32 rows with the same device code as the fused step kernel
__global__ void __launch_bounds__(256) mlp_tc_kernel(const uint4* packed, const float* x, int n, float* y)
{
    using L = MlpLayout;
    extern __shared__ __align__(16) unsigned char sm_tc[];
    uint4* dst = reinterpret_cast<uint4*>(sm_tc);
    for (int k = threadIdx.x; k < L::BYTES / 16; k += blockDim.x) dst[k] = packed[k];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* xch = sm_tc + L::BYTES + warp * L::XCH_BYTES;
    const float* xmu = reinterpret_cast<const float*>(sm_tc + L::XMU);
    const float* xis = reinterpret_cast<const float*>(sm_tc + L::XIS);
    const float* ymu = reinterpret_cast<const float*>(sm_tc + L::YMU);
    const float* ysd = reinterpret_cast<const float*>(sm_tc + L::YSD);
    const long long row = ((long long)blockIdx.x * 8 + warp) * 32 + lane;
    const bool ok = row < n;
    uint32_t* Xrow = reinterpret_cast<uint32_t*>(reinterpret_cast<__nv_bfloat16*>(xch) + lane * L::XLD);
    for (int q = 0; q < 5; ++q) {
        const float a = ok ? (x[row * 10 + 2 * q] - xmu[2 * q]) * xis[2 * q] : 0.f;
        const float b = ok ? (x[row * 10 + 2 * q + 1] - xmu[2 * q + 1]) * xis[2 * q + 1] : 0.f;
        Xrow[q] = pack_bf16(a, b);
    }
    for (int q = 5; q < 8; ++q) Xrow[q] = 0u;
    __syncwarp();
    float* Y = reinterpret_cast<float*>(xch);  // overlays the inputs
    mlp_warp_forward(sm_tc, reinterpret_cast<const __nv_bfloat16*>(xch), Y, lane);
    __syncwarp();
    if (ok)
        for (int q = 0; q < 6; ++q) y[row * 6 + q] = Y[lane * 8 + q] * ysd[q] + ymu[q];
}

int grid_n(long long n, int block, int cap = 152 * 16)
{
    long long g = (n + block - 1) / block;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

size_t mlp_packed_bytes() { return MlpLayout::BYTES; }

void mlp_pack(const float* params, const float* stats, unsigned char* out)
{
    using L = MlpLayout;
    std::memset(out, 0, L::BYTES);
    // hidden layers (l < 3) times 1/2: the inference evaluates SiLU(a) as
    // h + h tanh(h) on h = a/2 straight from the accumulator (a power of two,
    // so the scaled BF16 weight is the scaled rounded weight)
    auto putw = [&](int off, int ld, int l) {
        __nv_bfloat16* W = reinterpret_cast<__nv_bfloat16*>(out + off);
        const float* src = params + w_off(l);
        const float sc = l < 3 ? 0.5f : 1.0f;
        for (int o = 0; o < layer_out(l); ++o)
            for (int k = 0; k < layer_in(l); ++k)
                W[o * ld + k] = __float2bfloat16_rn(sc * src[o * layer_in(l) + k]);
    };
    auto putb = [&](int off, int l) {
        float* B = reinterpret_cast<float*>(out + off);
        const float sc = l < 3 ? 0.5f : 1.0f;
        for (int o = 0; o < layer_out(l); ++o) B[o] = sc * params[b_off(l) + o];
    };
    putw(L::W1, L::LD1, 0);
    putw(L::W2, L::LD, 1);
    putw(L::W3, L::LD, 2);
    putw(L::W4, L::LD, 3);
    putb(L::B1, 0);
    putb(L::B2, 1);
    putb(L::B3, 2);
    putb(L::B4, 3);
    float* xmu = reinterpret_cast<float*>(out + L::XMU);
    float* xis = reinterpret_cast<float*>(out + L::XIS);
    float* ymu = reinterpret_cast<float*>(out + L::YMU);
    float* ysd = reinterpret_cast<float*>(out + L::YSD);
    for (int k = 0; k < kIn; ++k) {
        xmu[k] = stats[k];
        xis[k] = 1.0f / stats[kIn + k];
    }
    for (int k = 0; k < kOut; ++k) {
        ymu[k] = stats[2 * kIn + k];
        ysd[k] = stats[2 * kIn + kOut + k];
    }
}

}  // namespace lbmk

using namespace lbmk;

extern "C" {

int lbm_mlp_param_count(void) { return kNParam; }

long long lbm_mlp_packed_bytes(void) { return (long long)MlpLayout::BYTES; }

int lbm_mlp_pack(const float* params, const float* stats, void* out_host)
{
    if (!params || !stats || !out_host) return set_last_error(LBM_ERR_ARG, "lbm_mlp_pack: NULL argument");
    mlp_pack(params, stats, static_cast<unsigned char*>(out_host));
    return LBM_OK;
}

int lbm_read_learned_closure(const char* path, float* params, int nparam, float* stats, int nstats)
{
    if (!path || !params || !stats) return set_last_error(LBM_ERR_ARG, "lbm_read_learned_closure: NULL argument");
    if (nparam != kNParam || nstats != 32)
        return set_last_error(LBM_ERR_ARG, "lbm_read_learned_closure: buffers must hold 9414 parameters and 32 statistics");
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return set_last_error(LBM_ERR_ARG, "lbm_read_learned_closure: cannot open the file");
    char magic[8];
    int32_t counts[2];
    int rc = LBM_OK;
    const char* why = nullptr;
    if (std::fread(magic, 1, 8, fp) != 8 || std::memcmp(magic, "LBMMLP01", 8) != 0) {
        why = "not a network file (magic LBMMLP01 expected)";
    } else if (std::fread(counts, sizeof(int32_t), 2, fp) != 2 || counts[0] != kNParam || counts[1] != 32) {
        why = "parameter or statistics count differs from this network (9414, 32)";
    } else if (std::fread(params, sizeof(float), (size_t)kNParam, fp) != (size_t)kNParam ||
               std::fread(stats, sizeof(float), 32, fp) != 32) {
        why = "file ends early";
    } else {
        unsigned char extra;
        if (std::fread(&extra, 1, 1, fp) != 0) why = "trailing bytes after the statistics";
    }
    std::fclose(fp);
    if (why) rc = set_last_error(LBM_ERR_ARG, (std::string("lbm_read_learned_closure: ") + why).c_str());
    return rc;
}

int lbm_set_learned_closure_file(lbm_handle* h, const char* path)
{
    if (!h || !path) return set_last_error(LBM_ERR_ARG, "lbm_set_learned_closure_file: NULL argument");
    std::vector<float> params(kNParam), stats(32);
    if (int rc = lbm_read_learned_closure(path, params.data(), kNParam, stats.data(), 32)) return rc;
    return lbm_set_learned_closure(h, params.data(), stats.data());
}

int lbm_mlp_forward_tc(const void* packed_dev, const float* x_dev, int n, float* y_dev, void* stream)
{
    if (!packed_dev || !x_dev || !y_dev || n < 1) return set_last_error(LBM_ERR_ARG, "lbm_mlp_forward_tc: bad arguments");
    const int smem = MlpLayout::BYTES + 8 * MlpLayout::XCH_BYTES;
    cudaError_t e = cudaFuncSetAttribute(mlp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) {
        const int blocks = (int)(((long long)n + 255) / 256);
        mlp_tc_kernel<<<blocks, 256, smem, static_cast<cudaStream_t>(stream)>>>(static_cast<const uint4*>(packed_dev),
                                                                               x_dev, n, y_dev);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? LBM_OK : set_last_error(LBM_ERR_CUDA, cudaGetErrorString(e));
}

long long lbm_mlp_workspace_floats(int n)
{
    // activations A, H of the four layers (64 wide, the last 6), dY, dX x2, weight partials, loss partials
    const long long blocks = (n + kWRows - 1) / kWRows;
    return (long long)n * (2 * 3 * kH + 2 * kOut) + (long long)n * kOut + 2LL * n * kH + blocks * (kH * kH + kH) +
           2 * 2048;
}

int lbm_mlp_forward(const float* params, const float* xs, int n, float* ys, float* ws, void* stream)
{
    if (!params || !xs || !ys || !ws || n < 1) return set_last_error(LBM_ERR_ARG, "lbm_mlp_forward: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* A = ws;
    float* H = ws + (long long)n * kH;
    const float* X = xs;
    for (int l = 0; l < 4; ++l) {
        const int in = layer_in(l), out = layer_out(l);
        float* Al = A;
        float* Hl = (l == 3) ? ys : H + (long long)(l & 1) * n * kH;
        mlp_fwd_kernel<<<grid_n((long long)n * out, 256), 256, 0, s>>>(X, n, in, out, params + w_off(l),
                                                                      params + b_off(l), Al, Hl, l < 3);
        X = Hl;
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : set_last_error(LBM_ERR_CUDA, cudaGetErrorString(e));
}

int lbm_mlp_grad(const float* params, const float* xs, const float* ts, int n, float* grad, float* ws, double* loss_out,
                 void* stream)
{
    if (!params || !xs || !ts || !grad || !ws || n < 1) return set_last_error(LBM_ERR_ARG, "lbm_mlp_grad: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // workspace layout
    float* A[4];
    float* H[4];
    float* p = ws;
    for (int l = 0; l < 4; ++l) {
        const int out = layer_out(l);
        A[l] = p;
        p += (long long)n * out;
        H[l] = p;
        p += (long long)n * out;
    }
    float* dY = p;
    p += (long long)n * kOut;
    float* dX[2] = {p, p + (long long)n * kH};
    p += 2LL * n * kH;
    const int wblocks = (n + kWRows - 1) / kWRows;
    float* partial = p;
    p += (long long)wblocks * (kH * kH + kH);
    p += ((uintptr_t)p & 7) ? 1 : 0;                // 8-byte alignment of the loss partials
    double* lpart = reinterpret_cast<double*>(p);   // up to 1024 doubles (the workspace's last 2048 floats)
    const float* X = xs;
    for (int l = 0; l < 4; ++l) {
        const int in = layer_in(l), out = layer_out(l);
        mlp_fwd_kernel<<<grid_n((long long)n * out, 256), 256, 0, s>>>(X, n, in, out, params + w_off(l),
                                                                      params + b_off(l), A[l], H[l], l < 3);
        X = H[l];
    }
    const int lb = grid_n((long long)n * kOut, 256, 1024);
    mlp_loss_kernel<<<lb, 256, 0, s>>>(H[3], ts, n, dY, lpart);
    const float* dcur = dY;
    for (int l = 3; l >= 0; --l) {
        const int in = layer_in(l), out = layer_out(l);
        const float* Xl = l == 0 ? xs : H[l - 1];
        mlp_bwd_weight_kernel<<<wblocks, 256, 0, s>>>(dcur, Xl, n, in, out, partial);
        const int np = out * in + out;
        mlp_reduce_kernel<<<(np + 255) / 256, 256, 0, s>>>(partial, wblocks, np, grad + w_off(l));
        if (l > 0) {
            float* dn = dX[l & 1];
            mlp_bwd_data_kernel<<<grid_n((long long)n * in, 256), 256, 0, s>>>(dcur, n, in, out, params + w_off(l),
                                                                              A[l - 1], dn);
            dcur = dn;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_last_error(LBM_ERR_CUDA, cudaGetErrorString(e));
    if (loss_out) {
        double hp[1024];
        e = cudaMemcpyAsync(hp, lpart, sizeof(double) * lb, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return set_last_error(LBM_ERR_CUDA, cudaGetErrorString(e));
        double tot = 0;
        for (int b = 0; b < lb; ++b) tot += hp[b];
        *loss_out = tot / ((double)n * kOut);
    }
    return LBM_OK;
}

int lbm_mlp_adamw(float* params, const float* grad, float* m, float* v, int step, float lr, float beta1, float beta2,
                  float eps, float wd, void* stream)
{
    if (!params || !grad || !m || !v || step < 1) return set_last_error(LBM_ERR_ARG, "lbm_mlp_adamw: bad arguments");
    const float bc1 = 1.0f - powf(beta1, (float)step), bc2 = 1.0f - powf(beta2, (float)step);
    adamw_kernel<<<(kNParam + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, grad, m, v, kNParam, lr,
                                                                                        beta1, beta2, eps, wd, bc1, bc2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : set_last_error(LBM_ERR_CUDA, cudaGetErrorString(e));
}

int lbm_box_filter(const void* f_dev, int lattice, int storage, int nx, int ny, int nz, int factor, double neq_scale,
                   int pull, float* fc_dev, float* msgs_dev, void* stream)
{
    if (!(neq_scale > 0.0)) return set_last_error(LBM_ERR_ARG, "lbm_box_filter: neq_scale must be > 0");
    if (!f_dev || !fc_dev || !msgs_dev || factor < 1 || nx % factor || ny % factor || nz % factor)
        return set_last_error(LBM_ERR_ARG, "lbm_box_filter: sizes must be multiples of the factor");
    if (lattice != 19 && lattice != 27) return set_last_error(LBM_ERR_ARG, "lattice must be 19 or 27");
    const long long Nc = (long long)(nx / factor) * (ny / factor) * (nz / factor);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int g = (int)((Nc + 127) / 128);
    auto go = [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        if (lattice == 27)
            filter_kernel<27, S><<<g, 128, 0, s>>>(static_cast<const S*>(f_dev), nx, ny, nz, factor, neq_scale, pull,
                                                   fc_dev, msgs_dev);
        else
            filter_kernel<19, S><<<g, 128, 0, s>>>(static_cast<const S*>(f_dev), nx, ny, nz, factor, neq_scale, pull,
                                                   fc_dev, msgs_dev);
    };
    switch (storage) {
    case LBM_FP64: go((double*)nullptr); break;
    case LBM_FP32: go((float*)nullptr); break;
    case LBM_FP16_SHIFTED: go((__half*)nullptr); break;
    case LBM_BF16_SHIFTED: go((__nv_bfloat16*)nullptr); break;
    default: return set_last_error(LBM_ERR_ARG, "unknown storage");
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : set_last_error(LBM_ERR_CUDA, cudaGetErrorString(e));
}

int lbm_closure_features(const float* f_dev, int lattice, int nx, int ny, int nz, double nu, const float* msgs_dev,
                         float* x_dev, float* t_dev, float* kcmp_dev, void* stream)
{
    if (!f_dev || !x_dev || nx < 1 || ny < 1 || nz < 1 || !(nu > 0))
        return set_last_error(LBM_ERR_ARG, "lbm_closure_features: bad arguments");
    const long long N = (long long)nx * ny * nz;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float tau_hat = (float)(nu / kTheta + 0.5);
    const int g = (int)((N + 127) / 128);
    if (lattice == 27)
        features_kernel<27><<<g, 128, 0, s>>>(f_dev, nx, ny, nz, tau_hat, msgs_dev, x_dev, t_dev, kcmp_dev);
    else if (lattice == 19)
        features_kernel<19><<<g, 128, 0, s>>>(f_dev, nx, ny, nz, tau_hat, msgs_dev, x_dev, t_dev, kcmp_dev);
    else
        return set_last_error(LBM_ERR_ARG, "lattice must be 19 or 27");
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : set_last_error(LBM_ERR_CUDA, cudaGetErrorString(e));
}

int lbm_closure_strain(const float* f_dev, int lattice, int nx, int ny, int nz, float* s_dev, void* stream)
{
    if (!f_dev || !s_dev || nx < 1 || ny < 1 || nz < 1)
        return set_last_error(LBM_ERR_ARG, "lbm_closure_strain: bad arguments");
    const long long N = (long long)nx * ny * nz;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int g = (int)((N + 127) / 128);
    if (lattice == 27)
        strain_kernel<27><<<g, 128, 0, s>>>(f_dev, nx, ny, nz, s_dev);
    else if (lattice == 19)
        strain_kernel<19><<<g, 128, 0, s>>>(f_dev, nx, ny, nz, s_dev);
    else
        return set_last_error(LBM_ERR_ARG, "lattice must be 19 or 27");
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : set_last_error(LBM_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"
