/*
 * lbm.h - C ABI of the GB300 (sm_103a) kinetic-closure LES lattice-Boltzmann
 * library (liblbm.so).
 *
 * The library advances a three-dimensional lattice-Boltzmann large-eddy
 * simulation whose collision carries the collision-side subgrid closure of
 * Marson & Malaspinas, "Kinetic closure of turbulence: collision-side modeling
 * beyond the filtered Boltzmann equation" (arXiv 2605.19796):
 *
 *   f_post_i = f_i - omega_hat (f_i - f0_i - f_sgs_i) - omega_sgs f_sgs_i      (App. F.1, Eq. operational_two_rate_update)
 *   f_i(x + c_i, t + 1) = f_post_i(x, t)                                     (Eq. streaming)
 *
 * with the shifted rates omega_hat = (nu/theta + 1/2)^-1 and
 * omega_sgs = min(omega_hat, (C_nu Delta sqrt(k_sgs)/theta + 1/2)^-1),
 * k_sgs = |tr m_sgs| / 2 (Eq. omega_sgs_operational), and the SGS carrier f_sgs
 * of the selected closure (KC-MP, App. F.3; KC-RB, App. F.2; KC-RR, App. F.4).
 * Each time step is ONE fused CUDA kernel: pull streaming, moments,
 * equilibrium (Eq. discrete_equilibrium), finite-difference strain
 * (Eqs. fd, strain_rate_discrete, fd_boundary_lower/upper), closure, rate and
 * relaxation, and the store.
 *
 * Conventions
 *  - Lattice units (dx = dt = 1, theta = 1/3).
 *  - Canonical population order: D3Q27 index i = 9*(cz+1) + 3*(cy+1) + (cx+1)
 *    for c in {-1,0,1}^3; D3Q19 is the same enumeration without the eight
 *    corners (|c|^2 = 3).
 *  - Fields are x-fastest: rho[box][z][y][x], u[3][box][z][y][x] (the velocity
 *    component is the slowest index), populations [box][q][z][y][x].
 *  - The state held by a handle is the post-collision population array; after
 *    n steps its moments are the fields at time n.
 *  - All entry points return 0 on success or a negative LBM_ERR_* code; the
 *    message of the last failure on the calling thread is lbm_last_error().
 *  - Host arrays are owned by the caller and only accessed during the call.
 *    Device memory allocated by lbm_create is owned by the handle and freed by
 *    lbm_destroy.
 *  - Work is enqueued on the handle's CUDA stream (cfg.cuda_stream, NULL = the
 *    legacy default stream).  lbm_step returns after enqueueing; calls that
 *    return data to host memory synchronise the stream.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ABI_VERSION 2

/* error codes */
#define LBM_OK 0
#define LBM_ERR_ARG (-1)         /* invalid argument or configuration          */
#define LBM_ERR_OOM (-2)         /* device or host allocation failed           */
#define LBM_ERR_CUDA (-3)        /* a CUDA runtime call failed                 */
#define LBM_ERR_NONFINITE (-4)   /* a NaN/Inf density or velocity was detected */
#define LBM_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up         */
#define LBM_ERR_UNSUPPORTED (-6) /* combination not supported (e.g. KC-RR on D3Q19) */
#define LBM_ERR_IO (-7)          /* file I/O failed or the file does not match  */

/* lattice (App. F "Velocity space discretization"; D3Q19 as an extension) */
#define LBM_D3Q19 19
#define LBM_D3Q27 27

/* collision closure (Sec. 6 and App. F) */
#define LBM_BGK 0          /* resolved BGK: omega_sgs = omega_hat (Sec. 5.1 resolved-BGK limit) */
#define LBM_KCMP 1         /* moment-projected closure, App. F.3 (default, C_nu = 0.035)    */
#define LBM_KCRB_HERMITE 2 /* residual-based closure, Hermite f1, Eq. kcrb_operational_fone  */
#define LBM_KCRB_RAW 3     /* residual-based closure, raw c c : S f1, Eq. kcrb_operational_raw_fone */
#define LBM_KCRR 4         /* recursive kinetic closure, App. F.4 (D3Q27 only)               */
#define LBM_LEARNED 5      /* KC-MP with m_sgs predicted by a network (lbm_set_learned_closure);
                              FP32 arithmetic, periodic boxes                                  */

/* population storage */
#define LBM_FP64 0          /* double storage, double arithmetic (parity mode)               */
#define LBM_FP32 1          /* float storage, float arithmetic                               */
#define LBM_FP16_SHIFTED 2  /* half storage of f_i - w_i, float arithmetic                   */
#define LBM_BF16_SHIFTED 3  /* bfloat16 storage of f_i - w_i, float arithmetic               */

/* boundary condition per axis (both faces) */
#define LBM_PERIODIC 0
#define LBM_BOUNCEBACK 1 /* halfway bounce-back walls; supported on the y axis only */

typedef struct lbm_handle lbm_handle;

typedef struct {
    int lattice;        /* LBM_D3Q19 or LBM_D3Q27                                   */
    int nx, ny, nz;     /* cells per box, each >= 1 (>= 3 along a bounce-back axis)  */
    int nbatch;         /* number of independent boxes (ensemble), >= 1             */
    const double* nu;   /* host array [nbatch]: kinematic viscosity per box, > 0;
                           tau_hat = nu/theta + 1/2 (Eq. omega_t_discrete)          */
    int closure;        /* LBM_BGK .. LBM_KCRR                                      */
    double c_nu;        /* C_nu of Eq. nu_t_sharp_closure (paper: 0.035 KC-MP,
                           0.02 KC-RB and KC-RR)                                    */
    double delta;       /* filter width Delta in lattice units (paper: 1)            */
    int storage;        /* LBM_FP64 .. LBM_BF16_SHIFTED                              */
    int bc[3];          /* per axis x, y, z: LBM_PERIODIC or LBM_BOUNCEBACK          */
    double force[3];    /* uniform body force density (Guo forcing); zero for none   */
    void* cuda_stream;  /* cudaStream_t to enqueue on; NULL = legacy default stream  */
    int tile_y;         /* tuning: rows per CTA tile (0 = library default: 4 for the
                           learned closure, else 8)                                  */
    int zchunk;         /* tuning: z-planes per CTA march (0 = library default)      */
    int variant;        /* tuning: step-kernel variant, 0 = library default
                           (periodic D3Q27 and D3Q19 with FP32/FP16/BF16
                           storage and BGK, KC-MP or KC-RB,
                           nx % 8 == 0: 14, tiles 128 x 8, or 64 x 16 for
                           nx <= 64, and for FP32 storage 16 where nx is a
                           multiple of the tile width and ny a multiple of
                           the tile height or >= 8 tile heights (also for
                           D3Q27 KC-RR); the FP32
                           channel (D3Q27, D3Q19) with BGK or KC-MP, nx % 8
                           == 0 and (ny - 1) % 16 != 0: 14 on 64 x 16 tiles,
                           with KC-MP 16 under the same conditions as the
                           periodic box; else, for
                           FP32 storage, 12 on z-chunks of at most 16 planes
                           for periodic D3Q27 with KC-MP or KC-RB, 13 for
                           KC-RR and walls; else 8 for periodic D3Q27 except
                           the learned closure; the learned closure on
                           periodic boxes with 32- or 16-bit storage: 15;
                           else 1),
                           1 = register pull (every lattice, storage, closure
                           and boundary), 8 = register pull with a split
                           arrive/wait barrier (BGK, KC-MP, KC-RB, KC-RR), 12
                           = 8 with the source rows of the plane after next
                           prefetched into L2, 13 = 8 with the own cell's
                           pulls copied to shared memory by cp.async one
                           plane ahead (FP32 and FP64 storage), 14 = four
                           cells per thread with 128-bit (FP32) / 64-bit
                           (16-bit) vector loads and stores, the pulls staged
                           in shared memory by cp.async one plane ahead and
                           the populations parked in tensor memory until
                           their collision (periodic D3Q27 and D3Q19,
                           FP32/FP16/BF16 storage, BGK/KC-MP/KC-RB, and
                           KC-RR on D3Q27, nx % 8 == 0; and the FP32
                           channel of either lattice, walls in y with a
                           force, BGK/KC-MP,
                           (ny - 1) % tile_y != 0; tile_y 8:
                           128 x 8 tiles, 16: 64 x 16 tiles; the learned
                           closure: 64 x 16 tiles, and 128 x 8 for 16-bit
                           storage; LBM_ERR_UNSUPPORTED otherwise), 15 = the
                           learned closure's register pull on 32 x 4 tiles
                           with the network on the tcgen05 tensor cores (one
                           128-row BF16 GEMM per layer and CTA, accumulators
                           in tensor memory; periodic, 32- and 16-bit
                           storage), 16 = 14 with the interior of the
                           staged rows copied by the Tensor Memory
                           Accelerator (one cp.async.bulk.tensor per
                           population and plane; BGK/KC-MP/KC-RB/KC-RR, nx a
                           multiple of 128, or 64 for tile_y 16;
                           LBM_ERR_UNSUPPORTED otherwise); other values,
                           among them the retired 2-7, 9, 10 and 11:
                           LBM_ERR_ARG */
    int disable_graphs; /* nonzero: lbm_step launches kernels one by one instead of
                           replaying a captured CUDA graph                        */
} lbm_config;

/* Fills cfg with defaults: D3Q27, 32^3, one box, KC-MP, C_nu 0.035, Delta 1,
 * FP32 storage, periodic, no force.  cfg->nu must still be set. */
void lbm_config_default(lbm_config* cfg);

/* Creates a solver for the LES of App. F.1: the lattice (App. F, velocity
 * space discretization), the per-box relaxation time tau_hat = nu/theta + 1/2
 * (Eq. omega_t_discrete), the closure and its C_nu and Delta (Eq.
 * nu_t_sharp_closure; KC-MP App. F.3, KC-RB App. F.2, KC-RR App. F.4), the
 * storage format, the boundaries and the body force are fixed here; the
 * state starts at rest (rho = 1, u = 0).
 * cfg: host, read during the call only (cfg->nu is copied).  Allocates two
 * population buffers (ping-pong) of nbatch*q*nx*ny*nz elements each plus small
 * control buffers on the current CUDA device; the handle owns them.
 * Returns LBM_OK; LBM_ERR_ARG for a malformed configuration (bad sizes,
 * lattice, closure, storage, nu <= 0, C_nu < 0, Delta <= 0, a retired or
 * unknown variant, a box of 2^31 cells or more),
 * LBM_ERR_UNSUPPORTED for a combination that is not built (KC-RR on D3Q19,
 * walls on x or z, a force without walls, a variant not built for the box),
 * LBM_ERR_OOM, LBM_ERR_CUDA.  On failure *out is NULL and nothing is
 * leaked. */
int lbm_create(const lbm_config* cfg, lbm_handle** out);

/* Frees everything the handle owns; NULL is ignored. */
void lbm_destroy(lbm_handle* h);

/* Sets every population to the equilibrium f0(rho, u) (Eq. discrete_equilibrium).
 * rho: host [nbatch*nz*ny*nx] or NULL for rho = 1; u: host [3][nbatch*nz*ny*nx].
 * The equilibrium is evaluated in FP64 for FP64 storage and in FP32 (on its
 * small per-axis terms) for FP32 and 16-bit storage.
 * Synchronises the stream before returning. */
int lbm_init_velocity(lbm_handle* h, const double* rho, const double* u);

/* As lbm_init_velocity from FP32 host fields (same layouts): half the bytes
 * over the host link.  For FP32 and 16-bit storage, whose equilibrium is
 * evaluated in FP32 anyway, the result is the same as from the FP64 fields
 * rounded to FP32; FP64 storage evaluates it in FP64 from the FP32 values.
 * Synchronises the stream before returning. */
int lbm_init_velocity_f32(lbm_handle* h, const float* rho, const float* u);

/* As lbm_init_velocity with device pointers (FP64, same layouts); enqueue only. */
int lbm_init_velocity_device(lbm_handle* h, const double* rho_dev, const double* u_dev);

/* Advances every box by nsteps time steps of App. F.1 (one fused kernel
 * launch per step).  Each step pull-streams the stored post-collision
 * populations (Eq. streaming; halfway bounce-back on wall axes), takes the
 * moments (step 1, with the half-force shift when a force is set), the
 * equilibrium (step 2, Eq. discrete_equilibrium), the finite-difference
 * strain (step 3, Eqs. fd, strain_rate_discrete, fd_boundary_lower/upper),
 * the closure's SGS carrier and trace (step 4), the clipped rate (step 5, Eq.
 * omega_sgs_operational) and the two-rate relaxation (step 6, Eq.
 * operational_two_rate_update, with Guo's source when a force is set), and
 * stores the new post-collision populations into the other buffer (step 7).
 * A call with nsteps >= 2 captures its nsteps launches once into a CUDA graph
 * (cached per step count and buffer parity, up to 4 graphs per handle) and
 * replays it as one graph launch (unless cfg.disable_graphs).  Enqueue only;
 * errors detected on the device (non-finite fields, a bounded wait that gave
 * up) are reported by the next lbm_moments / lbm_diagnostics /
 * lbm_synchronize.  Returns LBM_OK; LBM_ERR_ARG for nsteps < 0 or a NULL
 * handle, LBM_ERR_ARG for the learned closure without a network installed,
 * LBM_ERR_CUDA when a launch fails.  nsteps = 0 does nothing. */
int lbm_step(lbm_handle* h, int nsteps);

/* Times the built step-kernel variants, tile heights and z-chunks on the
 * handle's current state (each candidate `trials` times, best kept) and keeps
 * the fastest for later lbm_step calls.  The state is unchanged: every timed
 * launch reads the current buffer and writes the other one.  Synchronises. */
int lbm_autotune(lbm_handle* h, int trials);

/* Self-test of the error path of the kernels' bounded device-side waits:
 * launches on the handle's stream one CTA that waits on an mbarrier phase
 * nothing completes; its wait gives up after `polls` polls and sets the
 * timeout bit of the handle's status flag, which this call reads back, so the
 * expected result is LBM_ERR_TIMEOUT with the handle still usable (the
 * populations are untouched).  polls < 1: LBM_ERR_ARG. */
int lbm_wait_selftest(lbm_handle* h, int polls);

/* The launch configuration in use: kernel variant, tile height, z-chunk. */
int lbm_launch_config(const lbm_handle* h, int* variant, int* tile_y, int* zchunk);

/* Density and velocity of the current state (App. F.1 step 1, with the
 * half-force shift when a body force is set) into host arrays rho
 * [nbatch*N] and u [3][nbatch*N] (either may be NULL).  Sums in FP64 for FP64
 * storage, in FP32 for FP32 and 16-bit storage (rho assembled in FP64 from
 * the FP32 sum of f - w and the weights; errors of order 1e-7 relative, the
 * precision the stored values carry; lbm_diagnostics always sums in FP64).
 * Synchronises. */
int lbm_moments(lbm_handle* h, double* rho, double* u);

/* As lbm_moments into FP32 host arrays (same layouts): half the bytes over
 * the host link.  For FP32 and 16-bit storage these are the FP32 sums of
 * lbm_moments rounded to FP32 (rho from its FP64 assembly); FP64 storage sums
 * in FP64 and rounds.  Synchronises. */
int lbm_moments_f32(lbm_handle* h, float* rho, float* u);

/* As lbm_moments into device FP64 arrays; enqueue only. */
int lbm_moments_device(lbm_handle* h, double* rho_dev, double* u_dev);

/* Page-locked host memory for the host-pointer transfers (lbm_init_velocity,
 * lbm_moments, lbm_get/set_populations); the paper has no counterpart.  The
 * buffers come from the CUDA runtime's own page-locked allocator, which moves
 * the fields at the host link's full rate; memory locked after allocation by
 * other means was measured slower and with a wide spread on GB300.  *out_host
 * receives the buffer (bytes > 0; LBM_ERR_ARG otherwise, LBM_ERR_OOM if the
 * allocation fails); the caller owns it and releases it with lbm_host_free
 * (NULL is ignored). */
int lbm_host_alloc(size_t bytes, void** out_host);
int lbm_host_free(void* host);

/* FP64 global diagnostics of box `box`, LBM_DIAG_VALUES doubles:
 *  of the stored state (Sec. 7.1, Eq. tgv_energy_enstrophy):
 *   out[0] mass sum, out[1..3] momentum sums, out[4] E_k = <rho|u|^2/2>,
 *   out[5] enstrophy <|curl u|^2/2> with the sixth-order centred curl
 *   (second-order stencils along bounce-back axes), out[6] number of
 *   non-finite cells, out[7] max |u|;
 *  of the state the next step collides (the stored populations pull-streamed,
 *  rho and u of App. F.1 step 1, the strain of Eqs. fd, fd_boundary_lower/upper
 *  and strain_rate_discrete; a reading, the paper being silent on the
 *  dissipation):
 *   out[8] <2 rho nu_eff S:S>, nu_eff = theta (1/omega_s - 1/2) with the
 *   closure's clipped rate omega_s (Eq. omega_sgs_operational; nu for BGK;
 *   NaN for the learned closure), out[9] <2 rho nu S:S>.
 * Averages are arithmetic over the nodes.  Allocates its scratch (about 48
 * bytes per cell) on first use.  Synchronises; returns LBM_ERR_NONFINITE if
 * out[6] > 0.  (ABI version 1 had out[8], without the dissipation.) */
#define LBM_DIAG_VALUES 10
int lbm_diagnostics(lbm_handle* h, int box, double out[LBM_DIAG_VALUES]);

/* Copies the populations, converted to FP64 (shifted storage un-shifted), to
 * host [nbatch][q][nz][ny][nx].  Synchronises. */
int lbm_get_populations(lbm_handle* h, double* f);

/* Sets the populations from host FP64 [nbatch][q][nz][ny][nx].  Synchronises. */
int lbm_set_populations(lbm_handle* h, const double* f);

/* Gathers the populations (FP64, un-shifted) of ncells cells of box `box`:
 * xyz is host int [ncells][3] (x, y, z, each wrapped periodically into the
 * box), out is host double [ncells][q] in canonical order.  Synchronises.
 * Lets callers check sampled cells of lattices too large to copy back. */
int lbm_probe(lbm_handle* h, int box, const int* xyz, int ncells, double* out);

/* Device address and element size (bytes) of the current population buffer
 * (read-only view, valid until the next lbm_step). */
int lbm_population_buffer(lbm_handle* h, const void** ptr, int* elem_bytes);

/* Waits for the handle's stream; returns LBM_ERR_NONFINITE if a step saw a
 * non-finite density or velocity since the last check (the flag is cleared). */
int lbm_synchronize(lbm_handle* h);

/* Writes / reads the state (header + raw populations in storage format).
 * lbm_load requires a file written for the same lattice, sizes, nbatch and
 * storage (LBM_ERR_IO otherwise).  Both synchronise. */
int lbm_save(lbm_handle* h, const char* path);
int lbm_load(lbm_handle* h, const char* path);

/* Steps taken since creation (or since the state in the last lbm_load). */
int64_t lbm_step_count(const lbm_handle* h);

/* Allocation-free variant of the diagnostics reduction (the paper has no
 * counterpart; it is a service for callers that cannot allocate device memory:
 * a process whose device memory is all owned by another allocator, code that
 * must not trigger the implicit device synchronisation of cudaMalloc/cudaFree,
 * or a loop with a fixed memory budget).  Computes the first eight values of
 * lbm_diagnostics (those of the stored state, not the dissipation rates) for
 * ONE box whose populations the caller passes:
 *   f_dev    device pointer to the box's populations in storage format,
 *            [q][nz][ny][nx]: lbm_population_buffer plus the box offset, box b
 *            starting b*q*nx*ny*nz elements (of elem_bytes each) further;
 *   lattice, storage, nx, ny, nz: as in lbm_config (nz <= 4096);
 *   bc       host int[3] (NULL = periodic), force host double[3] (NULL = none);
 *   out_dev  device pointer to 8 doubles, written by the kernel;
 *   stream   cudaStream_t (NULL = legacy default stream).
 * Enqueue only, no synchronisation, no cudaMalloc/cudaFree or other allocating
 * call.  Its scratch is a static device array of 4096 x 8 FP64 partial sums
 * plus a counter (about 256 KB) that every GPU loading the library holds until
 * the process exits; nz > 4096 is rejected with LBM_ERR_ARG.  A call made outside
 * stream capture looks up the array's device address (cudaGetSymbolAddress) on
 * the current device and keeps it; a call during a capture uses the address the
 * last such call kept, so make the first call on each device before any stream
 * capture on it (otherwise LBM_ERR_CUDA).  All calls share
 * the array: calls whose kernels overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller.  Returns LBM_OK,
 * LBM_ERR_ARG or LBM_ERR_CUDA. */
int lbm_diagnostics_noalloc(const void* f_dev, int lattice, int storage, int nx, int ny, int nz, const int* bc,
                            const double* force, double* out_dev, void* stream);

/* ---- Learned closure (training side) ----------------------------------
 * The learned closure replaces KC-MP's m_sgs = m_neq - m_CE (App. F.3) by a
 * network evaluated per cell: 10 inputs (the KC-MP carrier (m_neq - m_CE)/rho:
 * xx yy zz xy xz yz; the trace, second invariant and determinant of m_CE/rho;
 * tau_hat), standardised,
 * three hidden layers of 64 SiLU units, 6 outputs (standardised m_sgs/rho).
 * Parameters: one FP32 vector of lbm_mlp_param_count() values in the order
 * W1 b1 W2 b2 W3 b3 W4 b4 (W row-major [out][in]).  Training data come from
 * fine runs box-filtered to the coarse grid, with the exact SGS stress of
 * Eq. (m_sgs_2) as target.  All pointers below are device pointers; calls
 * are enqueued on `stream` (NULL = legacy default stream). */

/* Number of network parameters (9414). */
int lbm_mlp_param_count(void);

/* Installs the network of a handle created with closure LBM_LEARNED:
 * params (host, lbm_mlp_param_count() FP32 values) and stats (host, 32 FP32
 * values: mean[10] and std[10] of the inputs, mean[6] and std[6] of the
 * outputs).  The step kernel evaluates the network with BF16 weights and
 * activations on the tensor cores (FP32 accumulation) and uses
 * m_sgs = rho (y std + mean) in KC-MP's rate and relaxation (App. F.3).
 * Synchronises. */
int lbm_set_learned_closure(lbm_handle* h, const float* params, const float* stats);

/* The network as a file (the paper has no format for it; this library's):
 * the 8 bytes "LBMMLP01", two little-endian int32 counts (9414 parameters,
 * 32 statistics), then the parameters and the statistics as little-endian
 * FP32 in the orders of lbm_set_learned_closure; nothing after them.
 * lbm_read_learned_closure reads such a file into caller-owned host buffers
 * (nparam and nstats give their lengths and must be 9414 and 32); it touches
 * no device.  A missing file, a wrong magic or count, a short file or
 * trailing bytes: LBM_ERR_ARG (buffers then unspecified).
 * lbm_set_learned_closure_file reads the file and installs the network as
 * lbm_set_learned_closure does.  Synchronises. */
int lbm_read_learned_closure(const char* path, float* params, int nparam, float* stats, int nstats);
int lbm_set_learned_closure_file(lbm_handle* h, const char* path);

/* Bytes of the packed network block the fused inference reads (BF16 weights,
 * FP32 biases and statistics), and the packing itself into host memory. */
long long lbm_mlp_packed_bytes(void);
int lbm_mlp_pack(const float* params, const float* stats, void* out_host);

/* Tensor-core forward with the fused step kernel's code path: raw inputs
 * x [n][10] (device), packed block (device) -> m_sgs/rho estimates y [n][6]
 * (device), BF16 operands and FP32 accumulation. */
int lbm_mlp_forward_tc(const void* packed_dev, const float* x_dev, int n, float* y_dev, void* stream);

/* Floats of device workspace lbm_mlp_forward / lbm_mlp_grad need for a batch of n. */
long long lbm_mlp_workspace_floats(int n);

/* ys [n][6] = network(xs [n][10]) for standardised inputs and outputs. */
int lbm_mlp_forward(const float* params, const float* xs, int n, float* ys, float* workspace, void* stream);

/* Gradient of L = mean over the batch and the 6 outputs of (net(xs) - ts)^2
 * with respect to every parameter into grad [param_count]; the loss (FP64) is
 * written to *loss_out (host) when not NULL, which synchronises the stream. */
int lbm_mlp_grad(const float* params, const float* xs, const float* ts, int n, float* grad, float* workspace,
                 double* loss_out, void* stream);

/* One AdamW step (bias-corrected moments m, v; decoupled weight decay on the
 * weight matrices only); step is 1-based. */
int lbm_mlp_adamw(float* params, const float* grad, float* m, float* v, int step, float lr, float beta1, float beta2,
                  float eps, float weight_decay, void* stream);

/* Box filter of one box's populations (storage format, [q][nz][ny][nx]) by
 * `factor` in every direction: filtered FP32 populations fc [q][nz/F][ny/F][nx/F]
 * and the exact SGS stress msgs [6][...] = bar(rho u u) - bar(rho u) bar(rho u)/rho_bar
 * (Eq. m_sgs_2; components xx yy zz xy xz yz).  Sizes must be multiples of factor.
 * neq_scale r: fc = bar(f) + (r - 1) bar(f - f0(rho, u)), f0 the fine cells' own
 * equilibria; r = 1 is the plain filter, r = F tau_hat_c / tau_hat_f gives the
 * coarse lattice's non-equilibrium part under acoustic scaling (the filtered
 * fine one is F tau_hat_c / tau_hat_f times too small), while the SGS part
 * bar(f0) - f0(rho_bar, u_bar) is kept.  r <= 0: LBM_ERR_ARG.
 * pull != 0: filter the streamed populations f_i(x - c_i) (periodic box, Eq.
 * streaming), i.e. the pre-collision state of the next step, which is the
 * state a step kernel computes its closure inputs from; pull = 0: the stored
 * post-collision populations. */
int lbm_box_filter(const void* f_dev, int lattice, int storage, int nx, int ny, int nz, int factor, double neq_scale,
                   int pull, float* fc_dev, float* msgs_dev, void* stream);

/* Network inputs x [N][10] of every cell of an FP32 population array
 * (periodic box, kinematic viscosity nu of that lattice); when msgs is given,
 * the targets t [N][6] = msgs / rho; when kcmp is given, the analytic KC-MP
 * estimate (m_neq - m_CE) / rho [N][6] (App. F.3, equal to inputs 0-5) for
 * comparison. */
int lbm_closure_features(const float* f_dev, int lattice, int nx, int ny, int nz, double nu, const float* msgs_dev,
                         float* x_dev, float* t_dev, float* kcmp_dev, void* stream);

/* Strain rate S of every cell of an FP32 population array (periodic box; the
 * velocity of App. F.1 step 1, the central differences of Eq. fd and
 * Eq. strain_rate_discrete, as lbm_closure_features forms m_CE from them)
 * into s [N][6] (xx yy zz xy xz yz).  Used to build training targets from
 * the SGS energy transfer -m_sgs : S of the filtered field.  Enqueue only;
 * LBM_ERR_ARG for bad arguments. */
int lbm_closure_strain(const float* f_dev, int lattice, int nx, int ny, int nz, float* s_dev, void* stream);

/* Number of CUDA kernels this handle has launched since creation. */
int64_t lbm_kernel_launches(const lbm_handle* h);

/* Message of the last failure on the calling thread ("" if none). */
const char* lbm_last_error(void);

/* LBM_ABI_VERSION of the loaded library. */
int lbm_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
