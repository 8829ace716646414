// C ABI of liblbm (declared in include/lbm.h): handle lifetime, device
// buffers, launches of the fused step kernel and of the auxiliary kernels.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace lbmk;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t storage_bytes(int storage)
{
    switch (storage) {
    case LBM_FP64: return 8;
    case LBM_FP32: return 4;
    case LBM_FP16_SHIFTED:
    case LBM_BF16_SHIFTED: return 2;
    }
    return 0;
}

}  // namespace

int lbmk::set_last_error(int code, const char* msg) { return fail(code, msg ? msg : ""); }

// a captured run of n steps starting from buffer `parity`
struct GraphEntry {
    int n = 0;
    int parity = 0;
    cudaGraphExec_t exec = nullptr;
};

struct lbm_handle {
    lbm_config cfg;
    std::vector<double> nu;
    int q = 0;
    size_t elem = 0;
    long long ncell = 0;     // cells per box
    long long popstride = 0;
    long long boxstride = 0;
    size_t buf_bytes = 0;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    double* d_nu = nullptr;
    unsigned int* d_flag = nullptr;
    double* d_rho = nullptr;  // diagnostics scratch (lazy): rho [N], u [3][N] of one box
    double* d_u = nullptr;
    double* d_partials = nullptr;
    double* d_diag = nullptr;  // LBM_DIAG_VALUES doubles
    double* d_s2 = nullptr;    // dissipation scratch: sum g |c|^2 of the streamed state [N]
    cudaStream_t stream = nullptr;
    int tile_y = 8;
    int variant = VAR_REGISTER;
    int zchunk = 16;
    int bc_kind = BC_PERIODIC;
    int64_t steps = 0;
    int64_t launches = 0;
    std::vector<GraphEntry> graphs;  // most recent last
    cudaStream_t cap_stream = nullptr;
    void* d_mlp = nullptr;           // packed network parameters (learned closure)
    bool mlp_set = false;
    // host-pointer field transfers (lazy): two staging slots of stage_cells
    // cells, each rho [stage_cells] then u [3][stage_cells], a copy stream and,
    // per slot, "filled" and "drained" events
    double* stage = nullptr;
    long long stage_cells = 0;
    cudaStream_t xstream = nullptr;
    cudaEvent_t ev_filled[2] = {nullptr, nullptr};
    cudaEvent_t ev_drained[2] = {nullptr, nullptr};
    // four-cell kernel's TMA staging: tensor maps of f[0], f[1] (boxes of the
    // tile's RY staged rows, of one row, of RY - 1 and of RY - 2 rows), encoded
    // for v4map_tile (0 = none)
    CUtensorMap v4map[2][4];
    int v4map_tile = 0;
};

namespace {

int check_handle(const lbm_handle* h)
{
    if (!h) return fail(LBM_ERR_ARG, "null handle");
    return LBM_OK;
}

// default z-chunk: enough CTAs to fill the GPU several times over while
// keeping the march long enough that the two extra halo planes per chunk stay cheap
int default_zchunk(int nx, int ny, int nz, int nbatch, int tile_y)
{
    const long long tiles = (long long)((nx + 31) / 32) * ((ny + tile_y - 1) / tile_y) * nbatch;
    const long long target = 152LL * 2 * 8;  // ~8 waves of two CTAs per SM
    long long chunks = (target + tiles - 1) / tiles;
    long long zc = (nz + chunks - 1) / chunks;
    if (zc < 4) zc = 4;
    if (zc > 64) zc = 64;
    if (zc > nz) zc = nz;
    return (int)zc;
}

// four-cell kernel (one 256-thread CTA per SM, tiles 128 x 8 or 64 x 16): 40
// planes (512^3 KC-MP: 40 planes 24.5 GLUPS, 48: 24.5, 32: 24.2, 27: 24.0,
// 64: 24.2), fewer where the box would not give two CTAs per SM
int default_zchunk_vec4(int nx, int ny, int nz, int nbatch, int tile_y)
{
    const int tx = tile_y == 16 ? 64 : 128;
    const long long tiles = (long long)((nx + tx - 1) / tx) * ((ny + tile_y - 1) / tile_y) * nbatch;
    // boxes at most 64 deep (ensembles of small boxes) take 16-plane chunks
    // where that still gives two CTAs per SM (64 x 64^3 boxes, 64 x 16 tiles:
    // 22.55 GLUPS, against 21.43 / 20.93 / 20.97 on chunks of 64 / 32 / 22 planes)
    if (nz <= 64 && nz >= 16 && tiles * ((nz + 15) / 16) >= 2LL * 152) return 16;
    const long long want = (2LL * 152 + tiles - 1) / tiles;  // chunks per tile column for two CTAs per SM
    long long zc = (nz + want - 1) / want;
    // at most 36 planes (512^3 KC-MP with TMA staging, 128 x 8 tiles: 36 planes
    // 27.7 GLUPS, 45: 27.7, 38: 27.6, 40: 27.4, 34: 27.4, 32: 27.3; 256^3: 36
    // planes 27.7, 40: 25.9, 30: 25.7, 28: 26.8, 32: 24.3 - the CTAs of the last
    // wave decide, the short last chunk of a 36-plane split filling it)
    if (zc > 36) zc = 36;
    if (zc < 4) zc = 4;
    if (zc > nz) zc = nz;
    return (int)zc;
}

constexpr int kMaxGraphSteps = 4096;
constexpr size_t kMaxGraphs = 4;

void clear_graphs(lbm_handle* h)
{
    for (auto& g : h->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
}

StepArgs step_args(const lbm_handle* h)
{
    StepArgs a;
    a.nx = h->cfg.nx;
    a.ny = h->cfg.ny;
    a.nz = h->cfg.nz;
    a.zchunk = h->zchunk;
    a.plane = (long long)h->cfg.nx * h->cfg.ny;
    a.popstride = h->popstride;
    a.boxstride = h->boxstride;
    a.box_nu = h->d_nu;
    a.cnu_delta = h->cfg.c_nu * h->cfg.delta;
    for (int k = 0; k < 3; ++k) a.force[k] = h->cfg.force[k];
    a.flag = h->d_flag;
    a.fin = nullptr;
    a.fout = nullptr;
    a.mlp = h->d_mlp;
    a.tmap_rows = nullptr;
    a.tmap_row1 = nullptr;
    a.tmap_rm1 = nullptr;
    a.tmap_rm2 = nullptr;
    return a;
}

// Variant 16 stages the interior of its rows by TMA: (re)encodes the tensor
// maps of both buffers for the handle's tile shape (a failed encoding makes
// its launches fail with cudaErrorInvalidValue).
void ensure_v4_maps(lbm_handle* h)
{
    const int ty = h->tile_y, tx = ty == 16 ? 64 : 128;
    const bool want = h->variant == VAR_VEC4_TMA && h->cfg.nx % tx == 0;
    if (!want || h->v4map_tile == ty) return;
    h->v4map_tile = 0;
    const int rows[4] = {ty + 2, 1, ty + 1, ty};
    for (int b = 0; b < 2; ++b) {
        for (int m = 0; m < 4; ++m) {
            if (encode_v4_map(&h->v4map[b][m], h->f[b], h->cfg.storage, h->cfg.nx, h->cfg.ny, h->cfg.nz, h->q,
                              h->cfg.nbatch, tx, rows[m]) != cudaSuccess) {
                cudaGetLastError();
                return;
            }
        }
    }
    h->v4map_tile = ty;
}

// n step launches starting from buffer `cur`, alternating the ping-pong buffers
cudaError_t enqueue_steps(const lbm_handle* h, int n, int cur, cudaStream_t s)
{
    StepArgs a = step_args(h);
    const bool maps = h->variant == VAR_VEC4_TMA && h->v4map_tile == h->tile_y;
    for (int k = 0; k < n; ++k) {
        a.fin = h->f[cur];
        a.fout = h->f[cur ^ 1];
        a.tmap_rows = maps ? &h->v4map[cur][0] : nullptr;
        a.tmap_row1 = maps ? &h->v4map[cur][1] : nullptr;
        a.tmap_rm1 = maps ? &h->v4map[cur][2] : nullptr;
        a.tmap_rm2 = maps ? &h->v4map[cur][3] : nullptr;
        cudaError_t e = launch_step(h->q, h->cfg.storage, h->cfg.closure, h->bc_kind, h->tile_y, h->variant, a,
                                    h->cfg.nbatch, s);
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    return cudaSuccess;
}

// the executable graph of n steps from the current buffer, captured on first use
cudaError_t step_graph(lbm_handle* h, int n, cudaGraphExec_t* out)
{
    for (size_t k = 0; k < h->graphs.size(); ++k)
        if (h->graphs[k].n == n && h->graphs[k].parity == h->cur) {
            GraphEntry g = h->graphs[k];
            h->graphs.erase(h->graphs.begin() + k);
            h->graphs.push_back(g);
            *out = g.exec;
            return cudaSuccess;
        }
    cudaError_t e = cudaSuccess;
    if (!h->cap_stream) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = prepare_step(h->q, h->cfg.storage, h->cfg.closure, h->bc_kind, h->tile_y, h->variant);
    if (e != cudaSuccess) return e;
    ensure_v4_maps(h);
    e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t el = enqueue_steps(h, n, h->cur, h->cap_stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->cap_stream, &graph);
    if (el != cudaSuccess) e = el;
    GraphEntry g;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    g.n = n;
    g.parity = h->cur;
    if (h->graphs.size() >= kMaxGraphs) {
        cudaGraphExecDestroy(h->graphs.front().exec);
        h->graphs.erase(h->graphs.begin());
    }
    h->graphs.push_back(g);
    *out = g.exec;
    return cudaSuccess;
}

void free_all(lbm_handle* h)
{
    clear_graphs(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (int k = 0; k < 2; ++k)
        if (h->f[k]) cudaFree(h->f[k]);
    if (h->d_nu) cudaFree(h->d_nu);
    if (h->d_flag) cudaFree(h->d_flag);
    if (h->d_rho) cudaFree(h->d_rho);
    if (h->d_u) cudaFree(h->d_u);
    if (h->d_partials) cudaFree(h->d_partials);
    if (h->d_diag) cudaFree(h->d_diag);
    if (h->d_s2) cudaFree(h->d_s2);
    if (h->d_mlp) cudaFree(h->d_mlp);
    if (h->xstream) cudaStreamSynchronize(h->xstream);
    if (h->stage) cudaFree(h->stage);
    for (int k = 0; k < 2; ++k) {
        if (h->ev_filled[k]) cudaEventDestroy(h->ev_filled[k]);
        if (h->ev_drained[k]) cudaEventDestroy(h->ev_drained[k]);
    }
    if (h->xstream) cudaStreamDestroy(h->xstream);
}

int read_flag(lbm_handle* h)
{
    unsigned int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, h->d_flag, sizeof(flag), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reading the status flag");
    if (flag) {
        cudaMemsetAsync(h->d_flag, 0, sizeof(unsigned int), h->stream);
        cudaStreamSynchronize(h->stream);
        if (flag & 2u) return fail(LBM_ERR_TIMEOUT, "a bounded device-side wait of a step kernel gave up");
        return fail(LBM_ERR_NONFINITE, "a non-finite density or velocity was produced by a step");
    }
    return LBM_OK;
}

int ensure_diag_scratch(lbm_handle* h)
{
    if (h->d_rho) return LBM_OK;
    const long long N = h->ncell;
    cudaError_t e = cudaMalloc(&h->d_rho, sizeof(double) * N);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_u, sizeof(double) * 3 * N);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_partials, sizeof(double) * diag_partials_len(N));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_diag, sizeof(double) * LBM_DIAG_VALUES);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_s2, sizeof(double) * N);
    if (e != cudaSuccess) {
        cudaFree(h->d_rho);
        cudaFree(h->d_u);
        cudaFree(h->d_partials);
        cudaFree(h->d_diag);
        cudaFree(h->d_s2);
        h->d_rho = h->d_u = h->d_partials = h->d_diag = h->d_s2 = nullptr;
        cudaGetLastError();
        return fail(LBM_ERR_OOM, "diagnostics scratch allocation failed");
    }
    return LBM_OK;
}

// Cells per staging slot of the host-pointer transfers: 2^21 (64 MB of FP64
// rho and u per slot), so that a chunk's copy (about 0.3 ms) dwarfs its
// kernel launch and the two slots bound the extra device memory at 128 MB.
constexpr long long kStageCells = 1LL << 21;

int ensure_stage(lbm_handle* h)
{
    if (h->stage) return LBM_OK;
    const long long n = h->ncell * h->cfg.nbatch;
    const long long c = n < kStageCells ? n : kStageCells;
    cudaError_t e = cudaMalloc(&h->stage, sizeof(double) * 4 * 2 * (size_t)c);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->xstream, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&h->ev_filled[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_drained[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (h->stage) cudaFree(h->stage);
        h->stage = nullptr;
        for (int k = 0; k < 2; ++k) {
            if (h->ev_filled[k]) cudaEventDestroy(h->ev_filled[k]);
            if (h->ev_drained[k]) cudaEventDestroy(h->ev_drained[k]);
            h->ev_filled[k] = h->ev_drained[k] = nullptr;
        }
        if (h->xstream) cudaStreamDestroy(h->xstream);
        h->xstream = nullptr;
        return fail(LBM_ERR_OOM, "staging ring allocation failed");
    }
    h->stage_cells = c;
    return LBM_OK;
}

struct FileHeader {
    char magic[8];
    int32_t abi, lattice, nx, ny, nz, nbatch, storage, closure;
    int64_t steps;
    uint64_t payload_bytes;
};

// Host-pointer initialisation: the fields go through the two staging slots in
// chunks of stage_cells cells; the copy of chunk k+1 (copy stream) runs while
// the init kernel of chunk k (solver stream) reads the other slot.  T: FP64 or
// FP32 host fields (a slot holds 4 stage_cells doubles, so either fits).
template <typename T>
int init_from_host(lbm_handle* h, const T* rho, const T* u)
{
    if (int rc = check_handle(h)) return rc;
    if (!u) return fail(LBM_ERR_ARG, "u is NULL");
    if (int rc = ensure_stage(h)) return rc;
    const long long n = h->ncell * h->cfg.nbatch, C = h->stage_cells;
    cudaError_t e = cudaSuccess;
    int k = 0;
    for (long long t0 = 0; t0 < n && e == cudaSuccess; t0 += C, ++k) {
        const long long m = n - t0 < C ? n - t0 : C;
        const int sl = k & 1;
        T* srho = reinterpret_cast<T*>(h->stage + (size_t)sl * 4 * C);
        T* su = srho + C;
        e = cudaStreamWaitEvent(h->xstream, h->ev_drained[sl], 0);  // chunk k-2's kernel has read the slot
        if (e == cudaSuccess && rho)
            e = cudaMemcpyAsync(srho, rho + t0, sizeof(T) * m, cudaMemcpyHostToDevice, h->xstream);
        for (int c = 0; c < 3 && e == cudaSuccess; ++c)
            e = cudaMemcpyAsync(su + c * C, u + c * n + t0, sizeof(T) * m, cudaMemcpyHostToDevice, h->xstream);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_filled[sl], h->xstream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_filled[sl], 0);
        if (e == cudaSuccess)
            e = launch_init_equilibrium(h->q, h->cfg.storage, h->f[h->cur], rho ? srho : nullptr, su, h->ncell,
                                        h->cfg.nbatch, h->popstride, h->boxstride, h->stream, t0, m, C);
        if (e == cudaSuccess) {
            h->launches++;
            e = cudaEventRecord(h->ev_drained[sl], h->stream);
        }
    }
    cudaError_t e2 = cudaStreamSynchronize(h->xstream);
    cudaError_t e3 = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3;
    if (e != cudaSuccess) return cuda_fail(e, "lbm_init_velocity");
    h->steps = 0;
    return LBM_OK;
}

// Host-pointer readback: chunk k's moments kernel (solver stream) fills one
// staging slot while the copy stream drains chunk k-1's slot to the host.
// T: FP64 or FP32 host fields.
template <typename T>
int moments_to_host(lbm_handle* h, T* rho, T* u)
{
    if (int rc = check_handle(h)) return rc;
    if (int rc = ensure_stage(h)) return rc;
    const long long n = h->ncell * h->cfg.nbatch, C = h->stage_cells;
    cudaError_t e = cudaSuccess;
    int k = 0;
    for (long long t0 = 0; t0 < n && e == cudaSuccess && (rho || u); t0 += C, ++k) {
        const long long m = n - t0 < C ? n - t0 : C;
        const int sl = k & 1;
        T* srho = reinterpret_cast<T*>(h->stage + (size_t)sl * 4 * C);
        T* su = srho + C;
        e = cudaStreamWaitEvent(h->stream, h->ev_drained[sl], 0);  // chunk k-2's copy has left the slot
        if (e == cudaSuccess) {
            T* dr = rho ? srho : nullptr;
            T* du = u ? su : nullptr;
            if constexpr (sizeof(T) == 8)
                e = launch_moments(h->q, h->cfg.storage, h->f[h->cur], dr, du, h->ncell, h->cfg.nbatch, h->popstride,
                                   h->boxstride, h->cfg.force, h->stream, true, t0, m, C);
            else
                e = launch_moments(h->q, h->cfg.storage, h->f[h->cur], dr, du, h->ncell, h->cfg.nbatch, h->popstride,
                                   h->boxstride, h->cfg.force, h->stream, t0, m, C);
        }
        if (e == cudaSuccess) {
            h->launches++;
            e = cudaEventRecord(h->ev_filled[sl], h->stream);
        }
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->xstream, h->ev_filled[sl], 0);
        if (e == cudaSuccess && rho)
            e = cudaMemcpyAsync(rho + t0, srho, sizeof(T) * m, cudaMemcpyDeviceToHost, h->xstream);
        for (int c = 0; c < 3 && e == cudaSuccess && u; ++c)
            e = cudaMemcpyAsync(u + c * n + t0, su + c * C, sizeof(T) * m, cudaMemcpyDeviceToHost, h->xstream);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_drained[sl], h->xstream);
    }
    cudaError_t e2 = cudaStreamSynchronize(h->xstream);
    cudaError_t e3 = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3;
    if (e != cudaSuccess) return cuda_fail(e, "copying the fields back");
    return read_flag(h);
}

}  // namespace

extern "C" {

void lbm_config_default(lbm_config* cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->lattice = LBM_D3Q27;
    cfg->nx = cfg->ny = cfg->nz = 32;
    cfg->nbatch = 1;
    cfg->closure = LBM_KCMP;
    cfg->c_nu = 0.035;
    cfg->delta = 1.0;
    cfg->storage = LBM_FP32;
}

int lbm_abi_version(void) { return LBM_ABI_VERSION; }

const char* lbm_last_error(void) { return g_err.c_str(); }

int lbm_create(const lbm_config* cfg, lbm_handle** out)
{
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(LBM_ERR_ARG, "cfg is NULL");
    if (cfg->lattice != LBM_D3Q19 && cfg->lattice != LBM_D3Q27) return fail(LBM_ERR_ARG, "lattice must be 19 or 27");
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1 || cfg->nbatch < 1) return fail(LBM_ERR_ARG, "sizes must be >= 1");
    const long long N = (long long)cfg->nx * cfg->ny * cfg->nz;
    if (N >= (1LL << 31) - 1) return fail(LBM_ERR_ARG, "a box must hold fewer than 2^31 cells");
    if (cfg->nbatch > 65535) return fail(LBM_ERR_ARG, "nbatch must be <= 65535");
    if (!cfg->nu) return fail(LBM_ERR_ARG, "nu is NULL");
    for (int b = 0; b < cfg->nbatch; ++b)
        if (!(cfg->nu[b] > 0.0) || !std::isfinite(cfg->nu[b])) return fail(LBM_ERR_ARG, "nu must be finite and > 0");
    if (cfg->closure < LBM_BGK || cfg->closure > LBM_LEARNED) return fail(LBM_ERR_ARG, "unknown closure");
    if (cfg->closure == LBM_KCRR && cfg->lattice != LBM_D3Q27)
        return fail(LBM_ERR_UNSUPPORTED, "KC-RR is defined on D3Q27 only");
    if (!(cfg->c_nu >= 0.0) || !(cfg->delta > 0.0)) return fail(LBM_ERR_ARG, "c_nu must be >= 0 and delta > 0");
    const size_t elem = storage_bytes(cfg->storage);
    if (!elem) return fail(LBM_ERR_ARG, "unknown storage");
    if (cfg->bc[0] != LBM_PERIODIC || cfg->bc[2] != LBM_PERIODIC || (cfg->bc[1] != LBM_PERIODIC && cfg->bc[1] != LBM_BOUNCEBACK))
        return fail(LBM_ERR_UNSUPPORTED, "bounce-back walls are supported on the y axis only");
    const int bc_kind = cfg->bc[1] == LBM_BOUNCEBACK ? BC_WALLS_Y : BC_PERIODIC;
    if (bc_kind == BC_WALLS_Y && cfg->ny < 3) return fail(LBM_ERR_ARG, "a bounce-back axis needs >= 3 cells");
    const bool has_force = cfg->force[0] != 0.0 || cfg->force[1] != 0.0 || cfg->force[2] != 0.0;
    if (has_force && bc_kind != BC_WALLS_Y)
        return fail(LBM_ERR_UNSUPPORTED, "a body force is supported with bounce-back walls (channel) only");
    // the learned closure runs 4-row tiles by default: at 128 threads per CTA
    // its register-pull kernel keeps both halves' network fragments in ~250
    // registers without spilling (8-row tiles cap them at 128 and spill); the
    // rest 8-row tiles
    int tile_y = cfg->tile_y ? cfg->tile_y : (cfg->closure == LBM_LEARNED ? 4 : 8);
    if (cfg->variant != VAR_DEFAULT && cfg->variant != VAR_REGISTER && cfg->variant != VAR_SPLIT &&
        cfg->variant != VAR_SPLIT_PF && cfg->variant != VAR_ASYNC && cfg->variant != VAR_VEC4 &&
        cfg->variant != VAR_TCNET && cfg->variant != VAR_VEC4_TMA)
        return fail(LBM_ERR_ARG, "unknown kernel variant");
    int variant = cfg->variant;
    // measured defaults (512^3 and ensemble timings): periodic D3Q27 with 32- or
    // 16-bit storage and BGK, KC-MP or KC-RB takes the four-cell kernel (tiles
    // 128 x 8, or 64 x 16 for boxes at most 64 wide), for FP32 storage with the
    // rows' interior staged by TMA (16; 512^3 KC-MP 26.6 GLUPS against 24.5 with
    // cp.async, 14) where every tile is full in x and at least eight tile rows
    // span y (the tiles whose staged rows wrap are copied row by row: 64^3
    // ensemble 20.2 against 22.5), else by cp.async (14); otherwise, for FP32
    // storage, KC-RR, D3Q19 and the walls with KC-MP take the split-barrier
    // pull with asynchronous copies (13); periodic D3Q27 otherwise (FP64) takes
    // the split-barrier pull (8); the learned closure on periodic boxes the
    // register pull with the network on the tcgen05 tensor cores (15, 4-row
    // tiles: 9.02 GLUPS at 256^3, against 8.44 for the register pull with
    // mma.sync fragments and 8.32 for the four-cell kernel); the rest the
    // register pull (1).
    // lbm_autotune may pick another launch for a given box
    bool short_chunks = false, vec4_chunks = false;
    if (variant == VAR_DEFAULT) {
        const bool carrier = cfg->closure == LBM_KCMP || cfg->closure == LBM_KCRB_HERMITE ||
                             cfg->closure == LBM_KCRB_RAW || cfg->closure == LBM_KCRR;
        const bool split_built = carrier || cfg->closure == LBM_BGK;
        // 128 x 8 tiles, or 64 x 16 for boxes at most 64 wide and for the channel
        // (512 x 256 x 256 KC-MP: 20.3 GLUPS against 19.9 on 128 x 8 tiles)
        const int v4_ty0 = cfg->tile_y ? cfg->tile_y : ((cfg->nx > 64 && bc_kind == BC_PERIODIC) ? 8 : 16);
        // the channel: FP32, BGK or KC-MP, the top wall row not the first row of a tile
        const bool v4_walls = bc_kind == BC_WALLS_Y && cfg->storage == LBM_FP32 &&
                              (cfg->closure == LBM_KCMP || cfg->closure == LBM_BGK) && (cfg->ny - 1) % v4_ty0 != 0;
        // D3Q27 and D3Q19
        const bool v4_lattice = cfg->lattice == LBM_D3Q27 || cfg->lattice == LBM_D3Q19;
        const bool v4_first = v4_lattice && (bc_kind == BC_PERIODIC || v4_walls) &&
                              cfg->storage != LBM_FP64 && cfg->closure != LBM_LEARNED &&
                              vec4_shape_ok(cfg->nx) && (cfg->tile_y == 0 || cfg->tile_y == 8 || cfg->tile_y == 16);
        const bool pf_first = cfg->lattice == LBM_D3Q27 && bc_kind == BC_PERIODIC && cfg->storage == LBM_FP32 &&
                              (cfg->closure == LBM_KCMP || cfg->closure == LBM_KCRB_HERMITE ||
                               cfg->closure == LBM_KCRB_RAW);
        const int v4_ty = v4_ty0;
        // TMA staging (16) where every tile is full in x, and full in y or the
        // ragged tiles (whose staged rows are copied row by row) are few:
        // periodic boxes (64 x 64^3 ensemble on 64 x 16 tiles: 25.0 GLUPS
        // against 22.5 with cp.async staging), and the channel with KC-MP (512 x
        // 256 x 256 on 64 x 16 tiles: 23.0 against 21.5)
        const bool tma_first = cfg->storage == LBM_FP32 &&
                               (bc_kind == BC_PERIODIC || (v4_walls && cfg->closure == LBM_KCMP)) &&
                               vec4_tma_shape_ok(cfg->nx, v4_ty) && (cfg->ny % v4_ty == 0 || cfg->ny >= 8 * v4_ty);
        if (v4_first && tma_first && step_supported(cfg->lattice, cfg->storage, cfg->closure, bc_kind, v4_ty, VAR_VEC4_TMA)) {
            variant = VAR_VEC4_TMA;
            tile_y = v4_ty;
            vec4_chunks = true;
        } else if (v4_first && cfg->closure != LBM_KCRR &&  // KC-RR on cp.async staging: 19.3 GLUPS, 13: 20.2
                   step_supported(cfg->lattice, cfg->storage, cfg->closure, bc_kind, v4_ty, VAR_VEC4)) {
            variant = VAR_VEC4;
            tile_y = v4_ty;
            vec4_chunks = true;
        } else if (cfg->closure == LBM_LEARNED &&
                   step_supported(cfg->lattice, cfg->storage, cfg->closure, bc_kind, tile_y, VAR_TCNET)) {
            variant = VAR_TCNET;
        } else if (pf_first && step_supported(cfg->lattice, cfg->storage, cfg->closure, bc_kind, tile_y, VAR_SPLIT_PF)) {
            variant = VAR_SPLIT_PF;
            short_chunks = true;
        } else if (carrier && cfg->storage == LBM_FP32 &&
                   step_supported(cfg->lattice, cfg->storage, cfg->closure, bc_kind, tile_y, VAR_ASYNC)) {
            variant = VAR_ASYNC;
        } else if (cfg->lattice == LBM_D3Q27 && split_built && bc_kind == BC_PERIODIC &&
                   step_supported(cfg->lattice, cfg->storage, cfg->closure, bc_kind, tile_y, VAR_SPLIT)) {
            variant = VAR_SPLIT;
        } else {
            variant = VAR_REGISTER;
        }
    } else if (variant == VAR_VEC4 || variant == VAR_VEC4_TMA) {
        vec4_chunks = true;
    }
    if ((variant == VAR_VEC4 || variant == VAR_VEC4_TMA) && !vec4_shape_ok(cfg->nx))
        return fail(LBM_ERR_UNSUPPORTED, "the four-cell variant needs nx % 8 == 0");
    if (variant == VAR_VEC4_TMA && !vec4_tma_shape_ok(cfg->nx, tile_y))
        return fail(LBM_ERR_UNSUPPORTED, "the TMA-staged four-cell variant needs nx % 128 == 0 (64 for tile_y 16)");
    if ((variant == VAR_VEC4 || variant == VAR_VEC4_TMA) && bc_kind == BC_WALLS_Y && (cfg->ny - 1) % tile_y == 0)
        return fail(LBM_ERR_UNSUPPORTED, "the four-cell variants with walls need (ny - 1) % tile_y != 0");
    if (!step_supported(cfg->lattice, cfg->storage, cfg->closure, bc_kind, tile_y, variant))
        return fail(LBM_ERR_UNSUPPORTED, "this lattice/storage/closure/boundary/tile/variant combination is not built");
    if (cfg->zchunk < 0) return fail(LBM_ERR_ARG, "zchunk must be >= 0");

    lbm_handle* h = new (std::nothrow) lbm_handle();
    if (!h) return fail(LBM_ERR_OOM, "host allocation failed");
    h->cfg = *cfg;
    h->nu.assign(cfg->nu, cfg->nu + cfg->nbatch);
    h->cfg.nu = nullptr;
    h->q = cfg->lattice;
    h->elem = elem;
    h->ncell = N;
    h->popstride = N;
    h->boxstride = (long long)h->q * N;
    h->buf_bytes = elem * (size_t)h->boxstride * (size_t)cfg->nbatch;
    h->stream = (cudaStream_t)cfg->cuda_stream;
    h->tile_y = tile_y;
    h->variant = variant;
    h->zchunk = cfg->zchunk ? cfg->zchunk : default_zchunk(cfg->nx, cfg->ny, cfg->nz, cfg->nbatch, tile_y);
    if (!cfg->zchunk && short_chunks && h->zchunk > 16) h->zchunk = 16;
    if (!cfg->zchunk && vec4_chunks) h->zchunk = default_zchunk_vec4(cfg->nx, cfg->ny, cfg->nz, cfg->nbatch, tile_y);
    // the channel with cp.async staging prefers shorter chunks (512 x 256 x 256
    // KC-MP on 64 x 16 tiles: 24 planes 20.7 GLUPS, 40: 20.3, 64: 19.2); with TMA
    // staging it takes the general rule (36 planes 24.3, 32: 24.1, 27: 23.9, 24:
    // 23.4, 43: 22.4)
    if (!cfg->zchunk && vec4_chunks && bc_kind == BC_WALLS_Y && variant == VAR_VEC4 && h->zchunk > 24) h->zchunk = 24;
    // the learned closure's network-heavy CTAs balance better over about twice
    // as many, half as long chunks (256^3, register pull on 4-row tiles: 26
    // planes 8.43 GLUPS, 52 planes 8.28, 16 planes 8.18)
    if (!cfg->zchunk && cfg->closure == LBM_LEARNED && !vec4_chunks && variant != VAR_TCNET) {
        int zc = (h->zchunk + 1) / 2;
        if (zc < 4) zc = 4;
        if (zc < h->zchunk) h->zchunk = zc;
    }
    h->bc_kind = bc_kind;

    cudaError_t e = cudaMalloc(&h->f[0], h->buf_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&h->f[1], h->buf_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_nu, sizeof(double) * cfg->nbatch);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_flag, sizeof(unsigned int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_all(h);
        delete h;
        return fail(e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,
                    std::string("device allocation failed: ") + cudaGetErrorString(e));
    }
    e = prepare_step(h->q, cfg->storage, cfg->closure, bc_kind, tile_y, variant);
    if (e == cudaSuccess) ensure_v4_maps(h);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_nu, h->nu.data(), sizeof(double) * cfg->nbatch, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_flag, 0, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->f[0], 0, h->buf_bytes, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        free_all(h);
        delete h;
        return cuda_fail(e, "lbm_create");
    }
    *out = h;
    return LBM_OK;
}

void lbm_destroy(lbm_handle* h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

int lbm_init_velocity_device(lbm_handle* h, const double* rho_dev, const double* u_dev)
{
    if (int rc = check_handle(h)) return rc;
    if (!u_dev) return fail(LBM_ERR_ARG, "u is NULL");
    cudaError_t e = launch_init_equilibrium(h->q, h->cfg.storage, h->f[h->cur], rho_dev, u_dev, h->ncell,
                                            h->cfg.nbatch, h->popstride, h->boxstride, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "init kernel");
    h->launches++;
    h->steps = 0;
    return LBM_OK;
}

int lbm_init_velocity(lbm_handle* h, const double* rho, const double* u)
{
    return init_from_host(h, rho, u);
}

int lbm_init_velocity_f32(lbm_handle* h, const float* rho, const float* u)
{
    return init_from_host(h, rho, u);
}

int lbm_set_learned_closure(lbm_handle* h, const float* params, const float* stats)
{
    if (int rc = check_handle(h)) return rc;
    if (h->cfg.closure != LBM_LEARNED) return fail(LBM_ERR_ARG, "the handle's closure is not LBM_LEARNED");
    if (!params || !stats) return fail(LBM_ERR_ARG, "params and stats must be given");
    for (int k = 0; k < 10; ++k)
        if (!(stats[10 + k] > 0.0f)) return fail(LBM_ERR_ARG, "input standard deviations must be > 0");
    std::vector<unsigned char> packed(mlp_packed_bytes());
    mlp_pack(params, stats, packed.data());
    cudaError_t e = cudaSuccess;
    if (!h->d_mlp) e = cudaMalloc(&h->d_mlp, packed.size());
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_mlp, packed.data(), packed.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_set_learned_closure");
    h->mlp_set = true;
    clear_graphs(h);
    return LBM_OK;
}

int lbm_step(lbm_handle* h, int nsteps)
{
    if (int rc = check_handle(h)) return rc;
    if (nsteps < 0) return fail(LBM_ERR_ARG, "nsteps must be >= 0");
    if (h->cfg.closure == LBM_LEARNED && !h->mlp_set)
        return fail(LBM_ERR_ARG, "set the network with lbm_set_learned_closure before stepping");
    int left = nsteps;
    // runs of >= 2 steps replay one captured CUDA graph (one graph launch per call)
    while (!h->cfg.disable_graphs && left >= 2) {
        const int n = left > kMaxGraphSteps ? kMaxGraphSteps : left;
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = step_graph(h, n, &exec);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "step graph");
        h->cur ^= (n & 1);
        h->steps += n;
        h->launches += n;
        left -= n;
    }
    if (left > 0) {
        ensure_v4_maps(h);
        cudaError_t e = enqueue_steps(h, left, h->cur, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
        h->cur ^= (left & 1);
        h->steps += left;
        h->launches += left;
    }
    return LBM_OK;
}

int lbm_autotune(lbm_handle* h, int trials)
{
    if (int rc = check_handle(h)) return rc;
    if (trials < 1) trials = 3;
    static const int kVariants[] = {VAR_REGISTER, VAR_SPLIT, VAR_SPLIT_PF, VAR_ASYNC, VAR_VEC4, VAR_TCNET, VAR_VEC4_TMA};
    static const int kTiles[] = {4, 8, 16};
    static const int kChunks[] = {8, 16, 32, 64, 128};
    const int v0 = h->variant, t0 = h->tile_y, z0 = h->zchunk;
    float best = 1e30f;
    int bv = v0, bt = t0, bz = z0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int v : kVariants)
        for (int ty : kTiles) {
            if (e != cudaSuccess) break;
            if (!step_supported(h->q, h->cfg.storage, h->cfg.closure, h->bc_kind, ty, v)) continue;
            if ((v == VAR_VEC4 || v == VAR_VEC4_TMA) && !vec4_shape_ok(h->cfg.nx)) continue;
            if (v == VAR_VEC4_TMA && !vec4_tma_shape_ok(h->cfg.nx, ty)) continue;
            if ((v == VAR_VEC4 || v == VAR_VEC4_TMA) && h->bc_kind == BC_WALLS_Y && (h->cfg.ny - 1) % ty == 0) continue;
            e = prepare_step(h->q, h->cfg.storage, h->cfg.closure, h->bc_kind, ty, v);
            for (int zc : kChunks) {
                if (e != cudaSuccess) break;
                if (zc > h->cfg.nz && zc != kChunks[0]) continue;
                h->variant = v;
                h->tile_y = ty;
                h->zchunk = zc < h->cfg.nz ? zc : h->cfg.nz;
                ensure_v4_maps(h);
                // state-preserving timing: every launch reads the current buffer and
                // writes the other one, so the state the caller sees is unchanged
                e = enqueue_steps(h, 1, h->cur, h->stream);
                float t = 1e30f;
                for (int k = 0; k < trials && e == cudaSuccess; ++k) {
                    e = cudaEventRecord(e0, h->stream);
                    if (e == cudaSuccess) e = enqueue_steps(h, 1, h->cur, h->stream);
                    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    float ms = 0;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                    if (e == cudaSuccess && ms < t) t = ms;
                }
                h->launches += trials + 1;
                if (e == cudaSuccess && t < best) {
                    best = t;
                    bv = v;
                    bt = ty;
                    bz = h->zchunk;
                }
            }
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    h->variant = bv;
    h->tile_y = bt;
    h->zchunk = bz;
    ensure_v4_maps(h);
    clear_graphs(h);
    if (e != cudaSuccess) {
        h->variant = v0;
        h->tile_y = t0;
        h->zchunk = z0;
        return cuda_fail(e, "lbm_autotune");
    }
    return LBM_OK;
}

int lbm_launch_config(const lbm_handle* h, int* variant, int* tile_y, int* zchunk)
{
    if (int rc = check_handle(h)) return rc;
    if (variant) *variant = h->variant;
    if (tile_y) *tile_y = h->tile_y;
    if (zchunk) *zchunk = h->zchunk;
    return LBM_OK;
}

int lbm_host_alloc(size_t bytes, void** out_host)
{
    if (!out_host || bytes == 0) return fail(LBM_ERR_ARG, "lbm_host_alloc: NULL output or zero size");
    *out_host = nullptr;
    cudaError_t e = cudaHostAlloc(out_host, bytes, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out_host = nullptr;
        return fail(LBM_ERR_OOM, "page-locked host allocation failed");
    }
    return LBM_OK;
}

int lbm_host_free(void* host)
{
    if (!host) return LBM_OK;
    cudaError_t e = cudaFreeHost(host);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_host_free");
    return LBM_OK;
}

int lbm_moments_device(lbm_handle* h, double* rho_dev, double* u_dev)
{
    if (int rc = check_handle(h)) return rc;
    cudaError_t e = launch_moments(h->q, h->cfg.storage, h->f[h->cur], rho_dev, u_dev, h->ncell, h->cfg.nbatch,
                                   h->popstride, h->boxstride, h->cfg.force, h->stream, true);
    if (e != cudaSuccess) return cuda_fail(e, "moments kernel");
    h->launches++;
    return LBM_OK;
}

int lbm_moments(lbm_handle* h, double* rho, double* u)
{
    return moments_to_host(h, rho, u);
}

int lbm_moments_f32(lbm_handle* h, float* rho, float* u)
{
    return moments_to_host(h, rho, u);
}

int lbm_wait_selftest(lbm_handle* h, int polls)
{
    if (int rc = check_handle(h)) return rc;
    if (polls < 1) return fail(LBM_ERR_ARG, "polls must be >= 1");
    cudaError_t e = launch_wait_selftest(static_cast<unsigned int*>(h->d_flag), polls, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_wait_selftest");
    ++h->launches;
    return read_flag(h);
}

int lbm_diagnostics(lbm_handle* h, int box, double out[LBM_DIAG_VALUES])
{
    if (int rc = check_handle(h)) return rc;
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    if (box < 0 || box >= h->cfg.nbatch) return fail(LBM_ERR_ARG, "box out of range");
    if (int rc = ensure_diag_scratch(h)) return rc;
    const char* fb = static_cast<const char*>(h->f[h->cur]) + (size_t)box * h->boxstride * h->elem;
    cudaError_t e = launch_moments(h->q, h->cfg.storage, fb, h->d_rho, h->d_u, h->ncell, 1, h->popstride,
                                   h->boxstride, h->cfg.force, h->stream);
    if (e == cudaSuccess)
        e = launch_diagnostics(h->d_rho, h->d_u, h->cfg.nx, h->cfg.ny, h->cfg.nz, h->cfg.bc, h->d_partials, h->d_diag,
                               h->stream);
    // the dissipation rates of the next pre-collision state (the moments
    // scratch is reused: the kernels above have read it by then)
    if (e == cudaSuccess)
        e = launch_dissipation(h->q, h->cfg.storage, fb, h->cfg.nx, h->cfg.ny, h->cfg.nz, h->bc_kind == BC_WALLS_Y,
                               h->cfg.force, h->cfg.closure, h->nu[box], h->cfg.c_nu * h->cfg.delta, h->d_rho, h->d_u,
                               h->d_s2, h->d_partials, h->d_diag + 8, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, h->d_diag, sizeof(double) * LBM_DIAG_VALUES, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "diagnostics");
    h->launches += 6;
    int rc = read_flag(h);
    if (rc == LBM_OK && out[6] > 0) rc = fail(LBM_ERR_NONFINITE, "non-finite cells in the diagnosed box");
    return rc;
}

int lbm_get_populations(lbm_handle* h, double* f)
{
    if (int rc = check_handle(h)) return rc;
    if (!f) return fail(LBM_ERR_ARG, "f is NULL");
    const size_t n = (size_t)h->boxstride * h->cfg.nbatch;
    double* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(double) * n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ERR_OOM, "staging allocation failed");
    }
    e = launch_to_f64(h->q, h->cfg.storage, h->f[h->cur], d, h->ncell, h->cfg.nbatch, h->popstride, h->boxstride,
                      h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaStreamSynchronize(h->stream);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_get_populations");
    h->launches++;
    return LBM_OK;
}

int lbm_set_populations(lbm_handle* h, const double* f)
{
    if (int rc = check_handle(h)) return rc;
    if (!f) return fail(LBM_ERR_ARG, "f is NULL");
    const size_t n = (size_t)h->boxstride * h->cfg.nbatch;
    double* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(double) * n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ERR_OOM, "staging allocation failed");
    }
    e = cudaMemcpyAsync(d, f, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = launch_from_f64(h->q, h->cfg.storage, h->f[h->cur], d, h->ncell, h->cfg.nbatch, h->popstride, h->boxstride,
                            h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaStreamSynchronize(h->stream);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_set_populations");
    h->launches++;
    h->steps = 0;
    return LBM_OK;
}

int lbm_probe(lbm_handle* h, int box, const int* xyz, int ncells, double* out)
{
    if (int rc = check_handle(h)) return rc;
    if (box < 0 || box >= h->cfg.nbatch) return fail(LBM_ERR_ARG, "box out of range");
    if (ncells < 0 || (ncells > 0 && (!xyz || !out))) return fail(LBM_ERR_ARG, "bad probe arguments");
    if (ncells == 0) return LBM_OK;
    int* d_xyz = nullptr;
    double* d_out = nullptr;
    cudaError_t e = cudaMalloc(&d_xyz, sizeof(int) * 3 * ncells);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(double) * h->q * ncells);
    if (e != cudaSuccess) {
        cudaFree(d_xyz);
        cudaGetLastError();
        return fail(LBM_ERR_OOM, "probe staging allocation failed");
    }
    const char* fb = static_cast<const char*>(h->f[h->cur]) + (size_t)box * h->boxstride * h->elem;
    e = cudaMemcpyAsync(d_xyz, xyz, sizeof(int) * 3 * ncells, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = launch_probe(h->q, h->cfg.storage, fb, d_xyz, ncells, h->cfg.nx, h->cfg.ny, h->cfg.nz, h->popstride, d_out,
                         h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, sizeof(double) * h->q * ncells, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaStreamSynchronize(h->stream);
    cudaFree(d_xyz);
    cudaFree(d_out);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_probe");
    h->launches++;
    return LBM_OK;
}

int lbm_population_buffer(lbm_handle* h, const void** ptr, int* elem_bytes)
{
    if (int rc = check_handle(h)) return rc;
    if (ptr) *ptr = h->f[h->cur];
    if (elem_bytes) *elem_bytes = (int)h->elem;
    return LBM_OK;
}

int lbm_synchronize(lbm_handle* h)
{
    if (int rc = check_handle(h)) return rc;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_synchronize");
    return read_flag(h);
}

int lbm_save(lbm_handle* h, const char* path)
{
    if (int rc = check_handle(h)) return rc;
    if (!path) return fail(LBM_ERR_ARG, "path is NULL");
    std::vector<char> buf(h->buf_bytes);
    cudaError_t e = cudaMemcpyAsync(buf.data(), h->f[h->cur], h->buf_bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_save");
    FileHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, "LBMKC01", 8);
    hd.abi = LBM_ABI_VERSION;
    hd.lattice = h->cfg.lattice;
    hd.nx = h->cfg.nx;
    hd.ny = h->cfg.ny;
    hd.nz = h->cfg.nz;
    hd.nbatch = h->cfg.nbatch;
    hd.storage = h->cfg.storage;
    hd.closure = h->cfg.closure;
    hd.steps = h->steps;
    hd.payload_bytes = h->buf_bytes;
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(LBM_ERR_IO, std::string("cannot open ") + path);
    bool ok = std::fwrite(&hd, sizeof(hd), 1, fp) == 1 && std::fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? LBM_OK : fail(LBM_ERR_IO, std::string("write failed: ") + path);
}

int lbm_load(lbm_handle* h, const char* path)
{
    if (int rc = check_handle(h)) return rc;
    if (!path) return fail(LBM_ERR_ARG, "path is NULL");
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(LBM_ERR_IO, std::string("cannot open ") + path);
    FileHeader hd;
    bool ok = std::fread(&hd, sizeof(hd), 1, fp) == 1;
    ok = ok && std::memcmp(hd.magic, "LBMKC01", 8) == 0 && hd.lattice == h->cfg.lattice && hd.nx == h->cfg.nx &&
         hd.ny == h->cfg.ny && hd.nz == h->cfg.nz && hd.nbatch == h->cfg.nbatch && hd.storage == h->cfg.storage &&
         hd.payload_bytes == h->buf_bytes;
    std::vector<char> buf;
    if (ok) {
        buf.resize(h->buf_bytes);
        ok = std::fread(buf.data(), 1, buf.size(), fp) == buf.size();
    }
    std::fclose(fp);
    if (!ok) return fail(LBM_ERR_IO, std::string("file does not match this solver: ") + path);
    cudaError_t e = cudaMemcpyAsync(h->f[h->cur], buf.data(), h->buf_bytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_load");
    h->steps = hd.steps;
    return LBM_OK;
}

int64_t lbm_step_count(const lbm_handle* h) { return h ? h->steps : -1; }

int64_t lbm_kernel_launches(const lbm_handle* h) { return h ? h->launches : -1; }

}  // extern "C"
