// Internal declarations shared by the CUDA translation units of liblbm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmk {

// Records `msg` as the calling thread's lbm_last_error() and returns `code`.
int set_last_error(int code, const char* msg);

enum Closure { CL_BGK = 0, CL_KCMP = 1, CL_KCRB_H = 2, CL_KCRB_RAW = 3, CL_KCRR = 4, CL_LEARNED = 5 };
enum Storage { ST_F64 = 0, ST_F32 = 1, ST_F16S = 2, ST_BF16S = 3 };
enum Boundary { BC_PERIODIC = 0, BC_WALLS_Y = 1 };

// Arguments of one fused step launch (all boxes of the ensemble).
struct StepArgs {
    const void* fin;        // post-collision populations of the previous step
    void* fout;             // post-collision populations of this step
    int nx, ny, nz;
    int zchunk;             // z-planes marched by one CTA
    long long plane;        // nx*ny
    long long popstride;    // nx*ny*nz elements between populations
    long long boxstride;    // q*popstride elements between boxes
    const double* box_nu;   // [nbatch] kinematic viscosity
    double cnu_delta;       // C_nu * Delta
    double force[3];        // body force density (channel); zero otherwise
    unsigned int* flag;     // bit 0: non-finite density/velocity seen, bit 1: a bounded wait timed out
    const void* mlp;        // packed network parameters (learned closure only), MlpLayout::BYTES
    // four-cell kernel with TMA staging: host addresses of the CUtensorMaps of
    // fin (box TX x staged rows RY, TX x 1, TX x (RY - 1) and TX x (RY - 2): the
    // last three for tiles whose staged rows wrap around y), or null
    const void* tmap_rows;
    const void* tmap_row1;
    const void* tmap_rm1;
    const void* tmap_rm2;
};

// tensor map of a population buffer for the four-cell kernel's TMA staging
// (4D: x, y, z, population of box; box box_x x box_rows x 1 x 1)
cudaError_t encode_v4_map(void* map_out /*CUtensorMap*/, const void* buf, int storage, int nx, int ny, int nz, int q,
                          int nbatch, int box_x, int box_rows);

// host: packs 9414 FP32 parameters and 32 standardisation values into the
// shared-memory layout of the fused inference (MlpLayout::BYTES bytes)
size_t mlp_packed_bytes();
void mlp_pack(const float* params, const float* stats, unsigned char* out);

// one-CTA kernel whose bounded mbarrier wait runs out (the timeout error path)
cudaError_t launch_wait_selftest(unsigned int* flag, long long polls, cudaStream_t s);

// Step-kernel variants: register pull (lbm_step.cuh), split arrive/wait
// barrier (lbm_step_split.cuh).  Values 2-7, 9, 10 and 11 belonged to measured
// alternatives that were retired (4: TMA-staged pipeline, 9: two cells per
// thread on packed FP32 pairs; both slower than variants 8, 12, 13 and 14 in
// every case measured); they are refused.
// Variant 14: four cells per thread with vector access and a tensor-memory
// stash (lbm_step_v4.cuh), periodic D3Q27, 32- and 16-bit storage, nx % 8 == 0.
enum Variant {
    VAR_DEFAULT = 0,
    VAR_REGISTER = 1,
    VAR_SPLIT = 8,
    VAR_SPLIT_PF = 12,
    VAR_ASYNC = 13,
    VAR_VEC4 = 14,
    VAR_TCNET = 15,
    VAR_VEC4_TMA = 16
};

// variant 14: box shapes it is built for (nx a multiple of 8)
bool vec4_shape_ok(int nx);
// variant 16: every tile full in x (the TMA does not wrap around the box)
bool vec4_tma_shape_ok(int nx, int tile_y);


// Host-side launchers (lbm_step_*.cu).  Return cudaSuccess or the launch error.
// tile_y selects the CTA tile height (instantiated values: 4, 8, 16).
cudaError_t launch_step(int q, int storage, int closure, int bc, int tile_y, int variant, const StepArgs& a,
                        int nbatch, cudaStream_t s);
// pure host check (no CUDA call): is the combination instantiated?
bool step_supported(int q, int storage, int closure, int bc, int tile_y, int variant);
// sets the kernel's shared-memory attribute (call outside stream capture)
cudaError_t prepare_step(int q, int storage, int closure, int bc, int tile_y, int variant);

// Auxiliary kernels (lbm_aux.cu).
// Cells t0 .. t0 + count - 1 (count < 0: all nbatch x ncell cells) with the
// fields in rho [count], u [3][ustride] (ustride < 0: count)
cudaError_t launch_init_equilibrium(int q, int storage, void* f, const double* rho, const double* u, long long ncell,
                                    int nbatch, long long popstride, long long boxstride, cudaStream_t s,
                                    long long t0 = 0, long long count = -1, long long ustride = -1);
// the same from FP32 fields
cudaError_t launch_init_equilibrium(int q, int storage, void* f, const float* rho, const float* u, long long ncell,
                                    int nbatch, long long popstride, long long boxstride, cudaStream_t s,
                                    long long t0 = 0, long long count = -1, long long ustride = -1);
// fp32: FP32 sums for 32- and 16-bit storage (readback); false: FP64 sums (diagnostics)
cudaError_t launch_moments(int q, int storage, const void* f, double* rho, double* u, long long ncell, int nbatch,
                           long long popstride, long long boxstride, const double* force, cudaStream_t s,
                           bool fp32 = false, long long t0 = 0, long long count = -1, long long ustride = -1);
// FP32 output fields (FP32 sums for 32- and 16-bit storage, FP64 sums for FP64 storage)
cudaError_t launch_moments(int q, int storage, const void* f, float* rho, float* u, long long ncell, int nbatch,
                           long long popstride, long long boxstride, const double* force, cudaStream_t s,
                           long long t0, long long count, long long ustride);
cudaError_t launch_to_f64(int q, int storage, const void* f, double* out, long long ncell, int nbatch,
                          long long popstride, long long boxstride, cudaStream_t s);
cudaError_t launch_from_f64(int q, int storage, void* f, const double* in, long long ncell, int nbatch,
                            long long popstride, long long boxstride, cudaStream_t s);
cudaError_t launch_probe(int q, int storage, const void* f, const int* xyz, int ncells, int nx, int ny, int nz,
                         long long ps, double* out, cudaStream_t s);
// Diagnostics of one box: u must hold that box's FP64 velocity [3][N] and rho
// its density; writes 8 doubles to out_dev (see lbm_diagnostics).
// partials: scratch of diag_partials_len(ncell) doubles.
long long diag_partials_len(long long ncell);
cudaError_t launch_diagnostics(const double* rho, const double* u, int nx, int ny, int nz, const int* bc,
                               double* partials, double* out_dev, cudaStream_t s);
// Dissipation rates of one box's next pre-collision state (f: that box's
// populations; walls: bounce-back in y): out_dev[0] = <2 rho nu_eff S:S>,
// out_dev[1] = <2 rho nu S:S> (NaN for nu_eff of the learned closure).
// drho [N], u [3][N], s2 [N] and partials (diag_partials_len) are scratch.
cudaError_t launch_dissipation(int q, int storage, const void* f, int nx, int ny, int nz, int walls, const double* force,
                               int closure, double nu, double cnud, double* drho, double* u, double* s2,
                               double* partials, double* out_dev, cudaStream_t s);

}  // namespace lbmk
