// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <string>

#include "../../include/amoebapol.h"

#define AP_WARP 32
#define AP_BLOCK_ATOMS 32          // atoms per block (one warp lane each), paper Sec. 2.3: B_size = 32

// physical constants (readings: the paper gives none)
#define AP_COULOMB 332.063713       // kcal A / (mol e^2)
#define AP_DEBYE 4.80321            // Debye per e*A
#define AP_SQRT_PI 1.7724538509055159
#define AP_SHORT_RANGE 4.0          // A, radius of the learned guess's neighbourhood feature

// 32-byte aligned 4-vector of doubles (the CUDA 13 double4 is deprecated)
struct __align__(32) dvec4 { double x, y, z, w; };

template <class T> struct V4;
template <> struct V4<float> { typedef float4 type; };
template <> struct V4<double> { typedef dvec4 type; };

template <class T> struct FftTypes;
template <> struct FftTypes<float> { typedef cufftComplex cplx; };
template <> struct FftTypes<double> { typedef cufftDoubleComplex cplx; };

// device-side solver state (one per context)
struct PcgState {
    double rz;         // r . z of the current iterate
    double pq;         // accumulator: p . A p
    double rz_new;     // accumulator: r . z after the update
    double zz;         // accumulator: |alpha r|^2 after the update
    double gamma;      // step length of the current iteration
    double beta;       // conjugation coefficient for the next direction
    double eps;        // convergence measure (Debye)
    double eps0;       // measure for the initial guess
    double tol;        // threshold (Debye)
    int iter;          // iterations done
    int max_iter;
    int done;          // 1 when converged or out of iterations
    int status;        // AP_OK / AP_NOT_CONVERGED
    unsigned int blocks_done;   // last-block-done counter of the q = A p kernel
    unsigned int blocks_done2;  // last-block-done counter of the update kernel
    int nonfinite;     // set when a reduction produced NaN/Inf
    int guard;         // iterations started by the graph loop (hard bound on the WHILE node)
};

// 64-bit fixed point (two's complement in unsigned long long so that atomicAdd applies):
// fields, forces and torque terms with 34 fractional bits, the energy with 30 (paper Sec. 2.4)
#define AP_FX_BITS 34
#define AP_FX_EBITS 30
__host__ __device__ __forceinline__ long long ap_to_fx(double v) { return llrint(v * 17179869184.0); }   // 2^34
__device__ __forceinline__ long long ap_to_fx(float v) { return llrintf(v * 17179869184.0f); }
__host__ __device__ __forceinline__ double ap_from_fx(long long a) { return (double)a * (1.0 / 17179869184.0); }
// value k of an accumulator array that holds FP64 numbers or (fixed != 0) fixed-point integers
__device__ __forceinline__ double acc_value(const double *acc, size_t k, int fixed) {
    return fixed ? ap_from_fx(reinterpret_cast<const long long *>(acc)[k]) : acc[k];
}

struct ap_ctx {
    ap_params prm;
    int prec = AP_MIXED;      // arithmetic: AP_MIXED (FP32 pairs/PME) or AP_FP64
    int fixed = 0;            // 1: 64-bit fixed-point accumulation (AP_FIXED)
    int n = 0, n_pad = 0, n_blocks = 0;
    cudaStream_t s0 = nullptr;          // caller's stream
    cudaStream_t s1 = nullptr;          // internal stream (reciprocal branch)
    cudaStream_t s2 = nullptr, s3 = nullptr;   // capture of the solve loop's body (main, reciprocal)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::string err;
    int sm_count = 0;

    // neighbour blocks
    int *perm = nullptr;      // [n_pad] slot -> atom (-1 for padding)
    int *iperm = nullptr;     // [n] atom -> slot
    float4 *bcenter = nullptr;   // [n_blocks] block centre (x,y,z) at the last build
    int2 *tiles = nullptr;       // [cap_tiles] block pairs (I <= J), sorted by I then J
    float4 *tshift = nullptr;    // [cap_tiles] origin of block J relative to block I's, periodic image
                                 // included (c_J - c_I + L k), as hi + lo float pairs with tshift_lo
    float4 *tshift_lo = nullptr; // [cap_tiles]
    int *tile_excl = nullptr;    // [cap_tiles] exclusion-mask slot or -1
    unsigned *excl_mask = nullptr;  // [cap_excl][32]
    int n_tiles = 0, cap_tiles = 0, n_excl_tiles = 0, cap_excl = 0;
    int *tile_off = nullptr;     // [n_blocks+1] first tile of each block
    int minimg = 1;              // per-pair minimum image (small boxes) vs per-tile shifts
    // per-configuration filtered chunks (capacity cap_chunks = cap_tiles chunks of 32)
    int *chunk_j = nullptr;      // [cap][32] j slot or -1
    void *chunk_pos = nullptr;   // T4 [cap][32] j position (image next to block I) and Thole factor
    int *chunk_src = nullptr;    // [cap][32] exclusion source (slot << 5 | j-lane) or -1
    unsigned *chunk_mask = nullptr;  // [cap][32] exclusion bits (i-lane word, bit = chunk position)
    int *chunk_flag = nullptr;   // [cap] 1 if the chunk holds excluded pairs
    int *nchunk = nullptr;       // [n_blocks]
    int2 *work = nullptr;        // [n_blocks + cap] (I, chunk) items, chunk -1 = diagonal block
    int *work_off = nullptr;     // [n_blocks + 1] first item of each block
    int *n_work = nullptr;       // device: [0] work items, [1] in-range pairs of the configuration
    int *item_start = nullptr;   // [work + 1] exclusive prefix of the items' weights (pairs + staging cost)
    int *scan_tmp = nullptr;     // chunk sums of that prefix
    unsigned *pmask = nullptr;   // [work][32] in-range pair bits per item (i-lane word, bit = j-lane)
    unsigned *pmask_t = nullptr; // [work][32] the transpose (j-lane word, bit = i-lane)
    unsigned *smask = nullptr;   // [work][32] pairs closer than AP_SHORT_RANGE (learned-guess feature)
    unsigned *smask_t = nullptr; // its transpose
    unsigned *pstart = nullptr;  // [work][32] each lane's start in the item's pair sides (side_start)
    unsigned *sstart = nullptr;  // the same for the short-range sides
    double *e1s = nullptr;       // [3][n_pad] short-range first-order induced field (feature)
    int cap_chunks = 0;
    int lists_valid = 0;
    // scratch for the build
    int *cell_count = nullptr; int cap_cells = 0;
    int *tmp_int = nullptr; int cap_tmp = 0;
    int *excl_off = nullptr, *excl_atoms = nullptr; int cap_excl_atoms = 0;   // copy of the CSR

    // configuration (sorted slots; element type T = float or double). Positions are stored
    // relative to the origin of the slot's block (its centre at the list build, bcenter):
    // small numbers, so FP32 keeps ~1e-6 A at any box size; pair kernels see differences
    // only, and the chunk positions are formed relative to block I's origin in FP64.
    void *posq = nullptr;     // T4: x, y, z (relative to the block origin), q
    int4 *stb = nullptr;      // [n_pad] smooth-PME stencil origin floor(K x / L) mod K per dimension
    void *stw = nullptr;      // T4 [n_pad] its fractional part K x / L - floor(K x / L), from FP64
    void *dipd = nullptr;     // T4: dx, dy, dz, alpha^-1/2 (Thole)
    void *quad0 = nullptr;    // T4: Qxx, Qxy, Qxz, Qyy
    void *quad1 = nullptr;    // T4: Qyz, Qzz, alpha, 0
    double *alpha = nullptr;  // [n_pad]
    double *E = nullptr;      // [3][n_pad] permanent field (SoA)
    double *acc = nullptr;    // [3][n_pad] real-space accumulator
    void *rec = nullptr;      // T [3][n_pad] reciprocal field from the gather
    double *rot = nullptr;    // [n_pad][9] frame matrices (columns x,y,z)
    double *mpl = nullptr;    // [n_pad][10] local multipoles (sorted), for torques
    int *frame_s = nullptr;   // [n_pad][3] frames in slot indices (type, z-slot, x-slot)
    double *fvec = nullptr;   // [n_pad][6] minimum-image vectors to the z- and x-atoms
    int config_valid = 0;

    // PCG
    double *mu = nullptr, *r = nullptr, *qv = nullptr;   // [3][n_pad]
    double *dg = nullptr;     // [n_pad] diagonal of A: 1/alpha - self coefficient (0 for padding)
    // mixed and fixed-point modes: the PCG vectors in FP32, one float4 (x, y, z, unused) per slot
    float4 *mu_f = nullptr, *r_f = nullptr, *q_f = nullptr;   // [n_pad] each
    float2 *dga_f = nullptr;  // [n_pad] (1/alpha - self coefficient, alpha), 0 for padding
    int *hist_count = nullptr;   // device: steps held by a batch step's trajectory history
    void *p = nullptr;        // T4 [n_pad] search direction
    PcgState *st = nullptr;   // device
    double *red_part = nullptr;   // [3 * ceil(n_pad/256)] per-block partial sums of the PCG dots
    PcgState *st_host = nullptr;  // pinned mirror

    // PME
    int K[3] = {0, 0, 0};
    size_t ngrid = 0, ncgrid = 0;
    void *grid = nullptr;     // T [Kz][Ky][Kx]
    void *cgrid = nullptr;    // complex [Kz][Ky][Kx/2+1]
    void *green = nullptr;    // T [Kz][Ky][Kx/2+1]  B(m) C(m)
    void *grid2 = nullptr;    // second real grid (potential of the permanent multipoles, kept for forces)
    long long *grid_fx = nullptr;   // AP_FIXED: the spread's fixed-point grid (kept cleared)
    cufftHandle plan_r2c = 0, plan_c2r = 0;

    // forces
    double *frc = nullptr;    // [3][n_pad] force accumulator (sorted)
    double *gdip = nullptr;   // [3][n_pad] dU/d(global dipole)
    double *gquad = nullptr;  // [6][n_pad] dU/d(global quadrupole)
    double *red = nullptr;    // small reduction scratch
    double *mu_s = nullptr;   // [3][n_pad] dipoles given to the force call (sorted)
    double *gbuf = nullptr;   // [30][n_pad] PME potential derivatives for the forces
    void *cgrid_v = nullptr;  // complex [Kz][Ky][Kx/2+1]: transform of the permanent potential (virial)
    double *vir_active = nullptr;   // virial accumulator of the force call in progress (or NULL)
    float *mlp_feat = nullptr;   // [n_pad][16] learned-guess features (slot order)
    float *mlp_y = nullptr;      // [n_pad][3] network outputs (slot order)

    // launch shapes chosen by ap_autotune (0 = default)
    int tune_mv_per_sm = 0;   // matvec CTAs per SM (0: as many as fit, the resident grid)
    int tune_pme_threads = 128;
    // Jacobi/DIIS solver (allocated by its first call)
    void *diis_st = nullptr;         // device state: window matrix, coefficients, convergence
    void *diis_st_host = nullptr;    // pinned mirror
    double *diis_y = nullptr;        // [depth][3][n_pad] ring of Jacobi updates y_k
    double *diis_e = nullptr;        // [depth][3][n_pad] ring of their errors e_k
    double *diis_part = nullptr;     // [AP_DIIS_MAX_DEPTH][blocks] partial dots
    int diis_cap = 0;                // window length the rings hold
    int last_solver = 0;             // the last solve: 0 PCG, 1 Jacobi/DIIS, 2 the two-set PCG
    void *dp = nullptr;              // buffers of the two-dipole-set path (allocated on first use)
    cudaGraphExec_t diis_exec = nullptr;
    // graph of the solve loop
    cudaGraphExec_t solve_exec = nullptr;
    int graph_ok = 0;         // 1 when the conditional-while graph is usable
    int graph_tried = 0;
};

// arguments of the real-space kernels that iterate the filtered work items
struct WorkArgs {
    const int2 *work;
    const int *n_work;
    const int *chunk_j;
    const void *chunk_pos;
    const unsigned *chunk_mask;
    const int *chunk_flag;
    const int *tile_excl;      // for the diagonal block's own mask
    const int *tile_off;
    const unsigned *excl_mask;
    const unsigned *pmask;
    const unsigned *pmask_t;
    const unsigned *smask;
    const unsigned *smask_t;
    const unsigned *pstart;    // per (item, lane): packed start of the lane's share of the sides
    const unsigned *sstart;
    const int *item_start;     // exclusive prefix of the item weights; [n_work] = total
};

inline WorkArgs work_args(const ap_ctx *ctx) {
    WorkArgs w;
    w.work = ctx->work;
    w.n_work = ctx->n_work;
    w.chunk_j = ctx->chunk_j;
    w.chunk_pos = ctx->chunk_pos;
    w.chunk_mask = ctx->chunk_mask;
    w.chunk_flag = ctx->chunk_flag;
    w.tile_excl = ctx->tile_excl;
    w.tile_off = ctx->tile_off;
    w.excl_mask = ctx->excl_mask;
    w.pmask = ctx->pmask;
    w.pmask_t = ctx->pmask_t;
    w.smask = ctx->smask;
    w.smask_t = ctx->smask_t;
    w.pstart = ctx->pstart;
    w.sstart = ctx->sstart;
    w.item_start = ctx->item_start;
    return w;
}

// error helpers -------------------------------------------------------------------------
int ap_fail(ap_ctx *c, int code, const std::string &msg);
#define AP_CUDA(call)                                                                    \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return ap_fail(ctx, AP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
#define AP_CUFFT(call)                                                                   \
    do {                                                                                 \
        cufftResult r_ = (call);                                                         \
        if (r_ != CUFFT_SUCCESS)                                                         \
            return ap_fail(ctx, AP_ERR_CUDA, std::string(#call) + ": cufft error " + std::to_string((int)r_)); \
    } while (0)

// launch helpers --------------------------------------------------------------------------
static inline int ap_grid_for(long n, int threads) { return (int)((n + threads - 1) / threads); }

// entry points implemented in the translation units ------------------------------------
int nb_build(ap_ctx *ctx, const double *d_xyz, const int *d_off, const int *d_atoms, int n_excl);
int cfg_load(ap_ctx *ctx, const double *d_xyz, const double *d_mpole, const int *d_frame,
             const double *d_alpha);
int filter_launch(ap_ctx *ctx, cudaStream_t s);
int filter_alloc(ap_ctx *ctx);
int real_field_launch(ap_ctx *ctx, cudaStream_t s);
int real_matvec_launch(ap_ctx *ctx, const void *p, cudaStream_t s);
int real_matvec_resident_per_sm(ap_ctx *ctx);
int short_matvec_launch(ap_ctx *ctx, const void *p, double *out, cudaStream_t s);
int real_forces_launch(ap_ctx *ctx, cudaStream_t s);
int pme_init(ap_ctx *ctx);
int pme_multipole_field(ap_ctx *ctx, cudaStream_t s);              // permanent: grid2 keeps phi_M
// T_rec p -> rec; grid_cleared: the caller has zeroed the context's grid (no clearing here)
int pme_dipole_field(ap_ctx *ctx, const void *p, cudaStream_t s, bool grid_cleared = false);
int dipole_operator_into(ap_ctx *ctx, cudaStream_t main, cudaStream_t aux);   // T p, both branches
// a set of PME work grids and cuFFT plans (the context owns one; others allow concurrent passes)
struct PmeBufs {
    void *grid = nullptr, *cgrid = nullptr;
    long long *grid_fx = nullptr;
    cufftHandle r2c = 0, c2r = 0;
};
int pme_bufs_create(ap_ctx *ctx, PmeBufs *b);
void pme_bufs_destroy(PmeBufs *b);
// T_rec p -> rec_out, on the given grids (NULL: the context's own)
int pme_dipole_field_into(ap_ctx *ctx, const void *p, void *rec_out, const PmeBufs *bufs, cudaStream_t s);
int real_matvec2_launch(ap_ctx *ctx, const void *p0, const void *p1, double *acc0, double *acc1,
                        cudaStream_t s);   // T_real on two dipole sets
int field_finish(ap_ctx *ctx, double *d_field_out);
int pcg_solve(ap_ctx *ctx, const double *d_guess, double tol, int max_iter, double *d_mu,
              ap_solve_info *info);
// energy, forces and (d_virial non-NULL) the virial [9] at caller-order dipoles d_mu
int forces_run(ap_ctx *ctx, const double *d_mu, double *d_energy, double *d_forces, double *d_virial);
// the same with extra terms before the frame chain rule; vir: a virial accumulator (virial_acc) or NULL
int forces_run_ex(ap_ctx *ctx, const double *d_mu, double *d_energy, double *d_forces,
                  int (*extra)(ap_ctx *, cudaStream_t), double *vir);
// forces of -(f/2) mu.T mu alone (mz: zeroed multipoles); vir as above
int mutual_forces_run(ap_ctx *ctx, const double *d_mu, void *const *mz, double *gd, double *gq,
                      double *d_forces, double *vir);
double *virial_acc(ap_ctx *ctx, int which);   // nine device slots: 0 a force call, 1 the mutual pass
int virial_out(ap_ctx *ctx, const double *a, const double *b, double *d_virial);   // a - b -> FP64 [9]
// smooth-PME potential derivatives for the forces; with vir non-NULL also the structure-factor
// share of the virial (permanent-induced and induced-induced, or induced-induced alone for _mu)
int pme_forces_derivs(ap_ctx *ctx, const void *mu4, double *gbuf, cudaStream_t s, double *vir);
int pme_forces_derivs_mu(ap_ctx *ctx, const void *mu4, double *gbuf, cudaStream_t s, double *vir);
int diis_solve(ap_ctx *ctx, const double *d_guess, double tol, int max_iter, int depth, double *d_mu,
               ap_solve_info *info);
void diis_release(ap_ctx *ctx);
int diis_info(ap_ctx *ctx, ap_solve_info *info);   // state of the last DIIS solve; synchronizes
int dp_set_pairs(ap_ctx *ctx, int n_pairs, const int *d_pairs, const double *d_scales);
int dp_fields(ap_ctx *ctx, double *d_field_d, double *d_field_p);
int dp_solve(ap_ctx *ctx, const double *gd, const double *gp, double tol, int max_iter, double *d_mu_d,
             double *d_mu_p, ap_solve_info *info);
int dp_forces(ap_ctx *ctx, const double *d_mu_d, const double *d_mu_p, double *d_energy, double *d_forces,
              double *d_virial);
int dp_info(ap_ctx *ctx, ap_solve_info *info);
int dp_matvec2_launch(ap_ctx *ctx, cudaStream_t s, int clear);
void dp_release(ap_ctx *ctx);
void dp_forget_graph(ap_ctx *ctx);   // drop the captured two-set solve loop (launch shapes changed)
