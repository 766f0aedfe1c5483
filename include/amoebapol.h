/*
 * amoebapol.h - C ABI of the GB300 (sm_103a) AMOEBA induced-dipole solver.
 *
 * The library computes the hot path of a polarizable MD step (paper Sec. 1.2-2.3):
 * the permanent multipole field that forms the right-hand side, the induced dipoles
 * by diagonally preconditioned conjugate gradient on the Thole-damped, Ewald-screened
 * dipole operator (real space over 32-atom blocks + smooth PME), and the polarization
 * energy and forces.
 *
 * Conventions for every call:
 *   - Pointers named d_* are device memory owned by the caller (e.g. the data of a
 *     PyTorch CUDA tensor), contiguous, row-major, in the caller's atom order. The
 *     library never frees them and keeps no pointer to them after the call returns.
 *   - Pointers named h_* are host memory owned by the caller.
 *   - Units: Angstrom, elementary charge, kcal/mol; dipoles in e*A; field in e/A^2;
 *     convergence tolerances in Debye (1 e*A = 4.80321 D).
 *   - Work is enqueued on the stream given to ap_create; a call returns once its work
 *     is enqueued unless it is documented to synchronize.
 *   - Return value: AP_OK (0), a negative AP_ERR_* code, or a positive warning.
 *     No C++ exception crosses the ABI. ap_last_error() describes the last failure.
 *   - A context is used by one host thread at a time.
 *   - Calls operate on "the current configuration": the positions and multipoles most
 *     recently passed to permanent_field(), with the block lists of the last
 *     build_neighbour_blocks().
 */
#ifndef AMOEBAPOL_H
#define AMOEBAPOL_H

#ifdef __cplusplus
extern "C" {
#endif

#define AP_OK               0
#define AP_NOT_CONVERGED    1   /* warning: max_iter reached, output holds the last iterate */
#define AP_ERR_ARG         -1   /* null pointer, bad size, box smaller than 2*(cutoff+buffer) ... */
#define AP_ERR_CUDA        -2   /* a CUDA / cuFFT call failed (message in ap_last_error) */
/* -3 is unused: every internal list grows to fit (build_neighbour_blocks reallocates) */
#define AP_ERR_NONFINITE   -4   /* NaN or Inf found in an input or a reduction */
#define AP_ERR_TIMEOUT     -5   /* a bounded device wait expired */
#define AP_ERR_STATE       -6   /* calls made out of order (e.g. solve before field) */

#define AP_MIXED  0   /* FP32 pair/PME arithmetic, FP64 accumulation and PCG reductions */
#define AP_FP64   1   /* FP64 everywhere (reference-grade, slow on GB300) */
#define AP_FIXED  2   /* FP32 pair/PME arithmetic as AP_MIXED, but fields, forces, torque terms and
                         the PME grid are accumulated in 64-bit fixed point (34 fractional bits;
                         the energy 30), as the paper's fixed-point mode (Sec. 2.4): integer sums
                         do not depend on the order of the additions, so every output is bitwise
                         reproducible from run to run and for any launch shape. Magnitudes must
                         stay below 2^29 in the units of the output (kcal/mol/A, e/A^2). */

#define AP_FRAME_NONE      0   /* multipoles given in the global frame */
#define AP_FRAME_Z_THEN_X  1   /* z toward the z-atom, x from the x-atom orthogonalised */
#define AP_FRAME_BISECTOR  2   /* z along the bisector of the bonds to the z- and x-atoms */

typedef struct ap_ctx ap_ctx;

typedef struct {
    int    n_atoms;       /* atoms in the system (> 0), fixed for the context */
    double box[3];        /* orthorhombic edge lengths, A; each >= 2*(cutoff+buffer) */
    double cutoff;        /* real-space cutoff r_c, A (paper Sec. 3: 7 A) */
    double buffer;        /* neighbour-list buffer, A (lists valid while no atom moved > buffer/2) */
    double ewald_beta;    /* Ewald splitting parameter beta, 1/A */
    int    grid[3];       /* PME grid K_x, K_y, K_z (even, >= 2*pme_order) */
    int    pme_order;     /* B-spline order; must be 5 (the paper's default, Sec. 1.2.2) */
    double thole_a;       /* Thole damping parameter a (AMOEBA: 0.39) */
    int    precision;     /* AP_MIXED, AP_FP64 or AP_FIXED */
} ap_params;

typedef struct {
    int    iterations;    /* PCG iterations performed (matrix-vector products after the initial residual),
                             or DIIS updates taken */
    int    status;        /* AP_OK, AP_NOT_CONVERGED, or AP_ERR_NONFINITE when a reduction of the
                             solve produced NaN or Inf (the solve then stops) */
    double eps_debye;     /* final RMS of alpha_i r_i in Debye (the convergence measure) */
    double eps_initial;   /* the same measure for the initial guess */
} ap_solve_info;

/* Create a context: validates the parameters, allocates device workspace, creates the
 * FFT plans and a second internal stream. `stream` is a cudaStream_t (NULL = legacy
 * default stream). Synchronizes. On failure *out is NULL and the code is returned. */
int ap_create(ap_ctx** out, const ap_params* params, void* stream);

/* Free everything the context owns. Synchronizes its streams first. NULL is a no-op. */
void ap_destroy(ap_ctx* ctx);

/* Message for the last failure on this context (or of the last ap_create when ctx is
 * NULL). The string is owned by the library and valid until the next call. */
const char* ap_last_error(const ap_ctx* ctx);

/* a1 - Neighbour blocks (paper Sec. 2.3: cells with at most 32 atoms, 32-atom groups
 * following the cell numbering, adjacency of groups within cutoff+buffer, and the
 * bonded-pair scaling handled per group pair, Sec. 1.2.1).
 *   d_xyz          [n][3] double, positions (any periodic image).
 *   d_excl_offsets [n+1] int, CSR offsets of the pairs whose permanent->induced scale
 *                  is 0 (1-2 / 1-3 / intramolecular); may list each pair in both rows.
 *   d_excl_atoms   [d_excl_offsets[n]] int, partner atoms.
 *   n_excl_entries the value d_excl_offsets[n] (a host copy, for sizing).
 * Sorts atoms spatially into 32-atom blocks, builds the list of interacting block
 * pairs and their 32x32-bit exclusion masks. Grows internal lists as needed
 * (allocates), synchronizes. Must precede permanent_field(); call again when any atom
 * has moved more than buffer/2 since the last build. */
int build_neighbour_blocks(ap_ctx* ctx, const double* d_xyz, const int* d_excl_offsets,
                           const int* d_excl_atoms, int n_excl_entries);

/* a2+a3 - Permanent field E_i at every atom (right-hand side of A mu = E):
 * Ewald real space over the blocks with Thole damping (scale 0 for excluded pairs),
 * smooth-PME reciprocal space (paper Sec. 1.2.2: spread, FFT, convolution, inverse
 * FFT, gather) and the self term 4 beta^3/(3 sqrt(pi)) d_i.
 *   d_xyz    [n][3] double positions; sets the current configuration.
 *   d_mpole  [n][10] double local-frame multipoles: q, dx, dy, dz,
 *            Qxx, Qxy, Qxz, Qyy, Qyz, Qzz (traceless; potential q/R + d.R/R^3 + R.Q.R/R^5).
 *   d_frame  [n][3] int: AP_FRAME_* type, z-atom, x-atom (-1 when unused).
 *   d_alpha  [n] double polarizabilities, A^3 (> 0).
 *   d_field  [n][3] double output, or NULL to keep the field only inside the context.
 * The context keeps the field for induced_dipoles_pcg() and polarization_energy_forces(). */
int permanent_field(ap_ctx* ctx, const double* d_xyz, const double* d_mpole,
                    const int* d_frame, const double* d_alpha, double* d_field);

/* a4+a5+a6+a7 - Induced dipoles: solve (alpha^-1 - T) mu = E by conjugate gradient with
 * the diagonal preconditioner diag(alpha) (paper Sec. 1.3 and Sec. 3). Every iteration
 * applies T = T_real (blocked pair kernel) + T_rec (smooth PME) + self; the convergence
 * test eps = 4.80321 sqrt(sum |alpha_i r_i|^2 / n) <= tol_debye runs on the device.
 *   d_guess   [n][3] double initial dipoles, or NULL for mu0 = alpha E.
 *   tol_debye convergence threshold, Debye (> 0).
 *   max_iter  iteration limit (>= 1).
 *   d_mu      [n][3] double output dipoles, e*A.
 *   h_info    optional host struct filled with the iteration count and residuals;
 *             when non-NULL the call synchronizes.
 * Returns AP_NOT_CONVERGED (> 0) when max_iter was reached (d_mu holds the last iterate;
 * reported only when h_info is non-NULL).
 * The iteration loop runs as one CUDA graph with a conditional WHILE node (captured on the
 * first call); with the environment variable AP_SOLVE_GRAPH=0 the same kernels are launched
 * one by one with a host-side status read per iteration instead (for profilers that cannot
 * attribute kernels inside conditional graphs). The same holds for induced_dipoles_diis and
 * induced_dipoles_pcg_dp. */
int induced_dipoles_pcg(ap_ctx* ctx, const double* d_guess, double tol_debye, int max_iter,
                        double* d_mu, ap_solve_info* h_info);

/* Longest DIIS window induced_dipoles_diis accepts. */
#define AP_DIIS_MAX_DEPTH 8

/* f3 - Jacobi iteration with DIIS extrapolation, an alternative solver of the same system
 * A mu = E (Sec. 1.3; A = alpha^-1 - T as for the PCG). Step k forms the Jacobi update
 * y_k = alpha (E + T x_k) and its error e_k = y_k - x_k = alpha r_k, stops when
 * eps = 4.80321 sqrt(sum |e_k|^2 / n) <= tol_debye (the PCG's measure) and returns x_k;
 * otherwise x_{k+1} = sum_i c_i y_i over the last `depth` steps, c minimising
 * |sum_i c_i e_i| subject to sum_i c_i = 1 (Pulay's DIIS). Where the window's bordered
 * system is singular the oldest entries are dropped until it is not (one entry: a plain
 * Jacobi step). depth = 1 is plain Jacobi iteration.
 *   d_guess   [n][3] double initial dipoles, or NULL for x_0 = alpha E.
 *   tol_debye convergence threshold, Debye (> 0).
 *   max_iter  limit on the extrapolated updates (>= 1); at most max_iter + 1 applications of T.
 *   depth     DIIS window, 1 .. AP_DIIS_MAX_DEPTH.
 *   d_mu      [n][3] double output dipoles, e*A.
 *   h_info    optional host struct (iterations = updates taken); when non-NULL the call
 *             synchronizes.
 * The first call allocates 2 * depth vectors of 3 * n doubles (kept by the context and grown
 * when a later call asks for a longer window); the call cannot be captured into a graph.
 * Returns AP_NOT_CONVERGED (> 0) when max_iter was reached (reported only with h_info). */
int induced_dipoles_diis(ap_ctx* ctx, const double* d_guess, double tol_debye, int max_iter,
                         int depth, double* d_mu, ap_solve_info* h_info);

/* f1 - AMOEBA's two induced-dipole sets. The polarization interactions carry three scale
 * factors (Sec. 2.3): one for the direct field that induces the d dipoles, one for the field
 * that induces the p dipoles, and one (1 here) for the mutual field. The d and p fields are
 *   E_d = E_c + sum_listed sigma_d F,  E_p = E_c + sum_listed sigma_p F,
 * where E_c is permanent_field()'s field with every excluded pair left out of real space
 * and F is a listed pair's Thole-damped Coulomb field (radial functions lambda_{2n+1} U_n);
 * mu_d = A^-1 E_d, mu_p = A^-1 E_p, and E_pol = -(f/2) sum_i mu_d,i . E_p,i.
 *
 * set_scaled_pairs: the listed pairs and their scales, kept by the context (copied).
 *   d_pairs   [n_pairs][2] int atom indices (caller order), i != j, each pair once.
 *   d_scales  [n_pairs][2] double (sigma_d, sigma_p).
 *   Every listed pair must also be in the exclusion lists given to build_neighbour_blocks
 *   (so that E_c leaves it out); listed pairs farther apart than the cutoff contribute
 *   nothing, as every pair beyond it. Synchronizes; AP_ERR_ARG for an index out of range,
 *   i == j or a non-finite scale. The first call allocates the two-set buffers (about
 *   70 doubles per atom, and a second PME grid pair with its own cuFFT plans). */
int set_scaled_pairs(ap_ctx* ctx, int n_pairs, const int* d_pairs, const double* d_scales);

/* f1 - E_d and E_p of a configuration: runs permanent_field() (E_c, kept for the forces),
 * then the listed-pair terms. d_field_d, d_field_p: [n][3] double outputs, or NULL. */
int permanent_field_dp(ap_ctx* ctx, const double* d_xyz, const double* d_mpole, const int* d_frame,
                       const double* d_alpha, double* d_field_d, double* d_field_p);

/* f1 - Both dipole sets by two diagonal-preconditioned CG recurrences in lockstep: every
 * iteration applies T to both search directions (the pair tensor of every pair evaluated
 * once for both) and the loop stops when the larger of the two convergence measures
 * (4.80321 sqrt(sum |alpha_i r_i|^2 / n), Debye) is <= tol_debye. Guesses: [n][3] double
 * or NULL (alpha E_d, alpha E_p). Outputs d_mu_d, d_mu_p [n][3] double. h_info as for
 * induced_dipoles_pcg (eps fields hold the larger measure); not capturable into a graph. */
int induced_dipoles_pcg_dp(ap_ctx* ctx, const double* d_guess_d, const double* d_guess_p, double tol_debye,
                           int max_iter, double* d_mu_d, double* d_mu_p, ap_solve_info* h_info);

/* f1 - E_pol = -(f/2) sum mu_d . E_p and F = -dE_pol/dx for converged mu_d, mu_p:
 * -(f/2) [mu_p . dE_d + mu_d . dE_p + mu_p . dT mu_d], with the frame (torque) terms.
 *   d_energy [1] double, kcal/mol; d_forces [n][3] double, kcal/mol/A (overwritten).
 *   d_virial [9] double output (row-major V_ab = dE_pol/de_ab, as polarization_energy_forces),
 *            or NULL to skip it. */
int polarization_energy_forces_dp(ap_ctx* ctx, const double* d_mu_d, const double* d_mu_p,
                                  double* d_energy, double* d_forces, double* d_virial);

/* a9 - Polarization energy, forces and virial at fixed dipoles (variational; the paper's
 * real-space loop updates energy, forces and virial together, Sec. 1.2.1, and accumulates them
 * in double precision, Sec. 2.2):
 * E_pol = -(f/2) sum_i mu_i . E_i with f = 332.063713, and F = -dE_pol/dx including the
 * reciprocal-space terms and the forces on frame atoms from multipole rotation.
 *   d_mu      [n][3] double induced dipoles (e.g. from induced_dipoles_pcg).
 *   d_energy  [1] double output, kcal/mol.
 *   d_forces  [n][3] double output, kcal/mol/A (overwritten).
 *   d_virial  [9] double output or NULL: V_ab = dE_pol/de_ab (row-major, kcal/mol), the
 *             derivative under the homogeneous deformation x -> (I + e) x of positions and box
 *             with the local-frame multipoles carried by their frames; at converged dipoles it
 *             equals the derivative at fixed mu. The pressure tensor's polarization share is
 *             -V / volume. Pairs, frame vectors and the reciprocal sum (volume and |m| of the
 *             Ewald kernel, potential derivatives times multipoles) are summed in FP64 (fixed
 *             point in AP_FIXED, reproducible).
 * Uses the configuration and field of the last permanent_field() call. */
int polarization_energy_forces(ap_ctx* ctx, const double* d_mu, double* d_energy,
                               double* d_forces, double* d_virial);

/* a5+a6 alone, for tests and diagnostics: d_out = T v = (T_real + T_rec + self) v for the
 * current configuration; d_v and d_out are [n][3] double in caller order. */
int dipole_field_matvec(ap_ctx* ctx, const double* d_v, double* d_out);

/* Diagnostics for benchmarks: number of 32-atom blocks, interacting block pairs
 * (tiles) and block pairs carrying exclusion masks of the current lists. */
int ap_list_stats(const ap_ctx* ctx, int* h_blocks, int* h_tiles, int* h_excl_tiles);

/* The stream the context enqueues on (cudaStream_t). */
void* ap_stream(const ap_ctx* ctx);

/* Iterations and residuals of the most recent induced_dipoles_pcg(),
 * induced_dipoles_diis() or induced_dipoles_pcg_dp() on this context, including solves
 * launched inside a batch graph. Synchronizes the context's stream. Returns
 * AP_ERR_NONFINITE (h_info still filled, status AP_ERR_NONFINITE) when a reduction of that
 * solve produced NaN or Inf, e.g. from a non-finite input, and AP_OK otherwise. */
int ap_solve_info_last(ap_ctx* ctx, ap_solve_info* h_info);

/* Benchmark support: launch one kernel of the path `reps` times on the context's stream
 * on the current configuration (inputs as left by the last calls), timing each launch
 * with CUDA events, and return the mean duration in ms. The composite ids (9-11: several
 * kernels, library transforms, two streams) are captured once into a CUDA graph and each
 * graph launch is timed, as they run inside the solve. Overwrites scratch buffers only
 * (the stored field, dipoles and lists are untouched). Synchronizes. */
#define AP_KERNEL_REAL_MATVEC       0   /* a5: real-space dipole-field pair kernel */
#define AP_KERNEL_REAL_FIELD        1   /* a2: real-space permanent-field pair kernel */
#define AP_KERNEL_SPREAD_DIPOLES    2   /* a6: B-spline spread of dipoles onto the grid */
#define AP_KERNEL_CONVOLVE          3   /* a3/a6: k-space product with B(m)C(m) */
#define AP_KERNEL_GATHER_FIELD      4   /* a3/a6: B-spline gather of the field */
#define AP_KERNEL_SPREAD_MULTIPOLES 5   /* a3: spread of the permanent multipoles */
#define AP_KERNEL_PAIR_FORCES       6   /* a9: real-space polarization forces and torque sources,
                                           at the dipoles of the last energy/force call */
#define AP_KERNEL_PCG_VECTORS       7   /* a7: one iteration's vector kernels (direction, q = A p
                                           with p.q, update with r.z and |z|^2); advances the last
                                           solve's state, so solve again before using its result */
#define AP_KERNEL_REAL_MATVEC2      8   /* f1: the two-set real-space product on the last two-set
                                          search directions (needs set_scaled_pairs) */
#define AP_KERNEL_FFT_ROUNDTRIP     9   /* a3/a6: the grid's forward transform (cuFFT R2C), the
                                           k-space product and the inverse transform (C2R) */
#define AP_KERNEL_PME_DIPOLES      10   /* a6: the whole reciprocal branch of one operator
                                           application (grid clear, spread, transforms, gather) */
#define AP_KERNEL_DIPOLE_OPERATOR  11   /* a5 + a6: one application of T as inside the PCG solve,
                                           real space on the context's stream and the reciprocal
                                           branch on its second stream, joined */
int ap_time_kernel(ap_ctx* ctx, int which, int reps, double* h_ms);

/* f3 - A minimal rigid-water integrator, for real trajectories of the path (an MD step is one
 * call of an integrator that moves positions and velocities under the forces, paper Sec. 1.1;
 * velocity Verlet is the paper's default, Sec. 2.5-2.6; its benchmarks step at 2 fs,
 * Sec. 2.7). Velocity Verlet in the kick-drift-kick form for rigid three-site molecules: the
 * distances atom0-atom1, atom0-atom2 and atom1-atom2 of every molecule are held by SHAKE after
 * the drift and by RATTLE on the velocities after the second kick (sweeps until the relative
 * violation is below 1e-12, at most 1000). Units: A, fs, amu, kcal/mol/A. One thread per
 * molecule, FP64, async on `stream`; every atom must belong to one molecule.
 *   d_mol      [n_mol][3] int atom indices of each molecule (water: O, H, H).
 *   h_lengths  [3] host doubles: the three constrained distances (water: O-H, O-H, H-H).
 *   d_mass     [n] double masses, amu.
 *   d_forces   [n][3] double total forces at the current positions, kcal/mol/A.
 *   d_status   device int or NULL: bit 0 set if SHAKE, bit 1 if RATTLE did not converge for a
 *              molecule (the caller clears it).
 * ap_md_kick_drift: v += dt/2 F/m, x += dt v, SHAKE, and v = the constrained displacement / dt.
 * ap_md_kick: v += dt/2 F/m with the forces at the new positions, RATTLE, then v *= lambda
 * (> 0: 1 keeps the energy; a Berendsen thermostat, paper Sec. 2.6, passes
 * sqrt(1 + dt/tau (T0/T - 1))); d_kinetic (device double or NULL) receives the kinetic energy
 * after the scale, kcal/mol. Errors through ap_last_error(NULL). */
int ap_md_kick_drift(int n_mol, const int *d_mol, const double *h_lengths, const double *d_mass, double dt_fs,
                     const double *d_forces, double *d_xyz, double *d_vel, int *d_status, void *stream);
int ap_md_kick(int n_mol, const int *d_mol, const double *h_lengths, const double *d_mass, double dt_fs,
               const double *d_forces, const double *d_xyz, double *d_vel, double lambda, double *d_kinetic,
               int *d_status, void *stream);

/* f3 - The van der Waals term of the minimal trajectories: Lennard-Jones between atoms i and j,
 * V = 4 eps_ij [(s_ij/r)^12 - (s_ij/r)^6] with eps_ij = sqrt(eps_i eps_j), s_ij = (s_i + s_j)/2,
 * force-shifted at the context's real-space cutoff rc (V(r) - V(rc) + (r - rc) F(rc), so energy
 * and force vanish there), over every non-excluded pair of the current configuration (the one
 * of the last permanent_field()). The polarization energy alone is attractive; this supplies
 * the repulsion that keeps a liquid from collapsing.
 *   d_lj      [n][2] double (eps kcal/mol, sigma A) in caller order; eps = 0 leaves an atom out.
 *   d_energy  [1] double output, kcal/mol (overwritten).
 *   d_forces  [n][3] double, caller order: the Lennard-Jones forces are ADDED to it. */
int ap_lj_forces(ap_ctx *ctx, const double *d_lj, double *d_energy, double *d_forces);

/* Diagnostics: the FP32 fused multiply-add rate of the current device, measured. The pair
 * kernels (a2, a5, a9) are bound by plain FP32 ALU work, not by a contraction, so their
 * roofline denominator is this rate, SMs x FP32 lanes x 2 flops x clock. A kernel with 8
 * independent FMA chains per thread runs on a grid of (resident CTAs per SM) x (the SM count
 * queried from the device); the best of `reps` launches timed with CUDA events gives
 * *h_tflops (TFLOP/s, FMA = 2 flops) and *h_sm_count the SM count. Allocates 4 bytes and a
 * stream of its own; synchronizes. Errors through ap_last_error(NULL). */
int ap_fp32_peak(int reps, double *h_tflops, int *h_sm_count);

/* Diagnostics: erfc as the FP32 pair kernels evaluate it (the rational approximation of
 * Abramowitz & Stegun 7.1.26 times e^{-x^2} from the kernels' fast exponential) in d_approx,
 * and CUDA's erfcf in d_lib, for the n arguments d_x (x >= 0; device arrays of floats). Async
 * on `stream`; AP_ERR_ARG for a null pointer or n < 1. */
int ap_eval_erfc(const float *d_x, int n, float *d_approx, float *d_lib, void *stream);

/* Batched replicas: many independent systems of uneven size advanced by one CUDA-graph
 * launch (the paper runs independent trajectories as separate jobs; here they share the
 * GPU). Each replica is an ordinary context created with its own non-default stream and
 * with lists already built; ap_batch_capture() records one step of every replica
 * (permanent_field, optional ap_learned_guess, induced_dipoles_pcg, optional
 * polarization_energy_forces) as parallel branches of a single graph. The graph reads and
 * writes the device buffers named in `steps` at capture time: refill their contents
 * (e.g. new positions) and call ap_batch_launch() once per step. Lists are rebuilt
 * outside the graph (build_neighbour_blocks synchronizes); recapture after a rebuild.
 * Per-replica iteration counts: ap_solve_info_last() on each context. */
typedef struct ap_batch ap_batch;
typedef struct {
    const double* d_xyz;         /* [n][3] positions buffer of the replica */
    const double* d_mpole;       /* [n][10] local multipoles */
    const int*    d_frame;       /* [n][3] frames */
    const double* d_alpha;       /* [n] polarizabilities */
    const void*   d_mlp_packed;  /* packed network for the learned guess, or NULL for alpha E */
    double*       d_mu0;         /* [n][3] scratch for the learned guess (NULL if plain) */
    double        tol_debye;
    int           max_iter;
    double*       d_mu;          /* [n][3] output dipoles */
    double*       d_energy;      /* [1] output energy, or NULL to skip energy and forces */
    double*       d_forces;      /* [n][3] output forces, or NULL */
    double*       d_hist;        /* [5][n][3] scratch for the trajectory guess, or NULL: with the
                                    learned guess, each launch starts from the learned guess plus
                                    the linear extrapolation of its error over the two previous
                                    launches (ap_extrapolate_guess with base = learned guess;
                                    the learned guess alone until two launches exist). Holds the
                                    last two dipoles, the last two learned guesses and the guess;
                                    ap_batch_capture() starts a new trajectory. */
    double*       d_hist_lsq;    /* 7 * n * 3 + AP_ADAPTIVE_SCRATCH doubles, zeroed, or NULL: with
                                    the learned guess, each launch starts from the learned guess
                                    plus the adaptive extrapolation of its error over the three
                                    previous launches (ap_adaptive_guess with base = learned
                                    guess; the learned guess alone at the first launch, its
                                    previous error held at the second and third). Holds the last
                                    three dipoles, the last three learned guesses, the guess and
                                    the reduction scratch; takes precedence over d_hist. */
    double*       d_virial;      /* [9] output virial (as polarization_energy_forces), or NULL */
} ap_batch_step;
int ap_batch_create(ap_batch** out, ap_ctx* const* ctxs, int n_ctx);
int ap_batch_capture(ap_batch* b, const ap_batch_step* steps);
int ap_batch_launch(ap_batch* b, void* stream);
void ap_batch_destroy(ap_batch* b);

/* Launch-shape autotuner: times whole PCG solves (four iterations from alpha E, each one
 * graph launch, so the real-space matvec runs concurrently with the PME branch as in any
 * solve) for every combination of the matvec's CTAs per SM (as many as fit, 11, 10, 9, 8,
 * 6 and 3) and the PME spread/gather block size (64, 128 and 256 threads) on the current
 * configuration, and keeps the fastest for this context. Overwrites the state of the last
 * solve (ap_solve_info_last). h_choice[2] (optional) receives the matvec CTAs per SM (0 =
 * as many as fit) and the thread count. Synchronizes. */
int ap_autotune(ap_ctx* ctx, int reps, int* h_choice);

/* a8 - Learned initial guess. The paper has no learned component; any PCG start is
 * valid (the solve converges to the same tolerance), so a better start only saves
 * iterations. A per-atom perceptron 16 -> 128 -> 128 -> 3 (ReLU) maps rotation-invariant
 * features to a correction of the direct-field guess:
 *   mu0_i = alpha_i E_i + 0.02 R_i y_i,   R_i the atom's local frame (identity for
 *   global-frame atoms). Features (16, FP32), with fields divided by 0.05 e/A^2: the
 *   permanent field E_i in the atom's frame (3); the short-range first-order induced
 *   field E1_i = sum_{j: r_ij < 4 A} T_ij (alpha_j E_j) (real-space dipole kernel) in
 *   the same frame (3); E at the z-atom and at the x-atom in i's frame (3 + 3); |E_i|;
 *   |E1_i|; alpha_i; frame kind (0 global, 0.5 Z-then-X, 1 bisector).
 * Master parameters are FP32, ap_mlp_param_count() floats in the order W1 [16][128],
 * b1 [128], W2 [128][128], b2 [128], W3 [128][3], b3 [3] (W[in][out]). The kernels use a
 * packed copy (BF16 weights in tensor-core operand layout, FP32 biases) of
 * ap_mlp_packed_bytes() bytes. Inference and training run on the tcgen05 tensor cores
 * (BF16 operands, FP32 accumulation in tensor memory). */
int ap_mlp_param_count(void);
int ap_mlp_packed_bytes(void);
/* Pack d_params (FP32 master) into d_packed (device, ap_mlp_packed_bytes()). Async. */
int ap_mlp_pack(const float* d_params, void* d_packed, void* stream);
/* y = MLP(feat) for n rows: d_feat [n][16] FP32, d_y [n][3] FP32 (device). Async. */
int ap_mlp_forward(const void* d_packed, const float* d_feat, int n, float* d_y, void* stream);
/* Gradient of L = (1/2n) sum_i |y_i - t_i|^2 over n rows (d_feat [n][16], d_target [n][3])
 * at the parameters held in d_packed, ADDED to d_grad (FP32, ap_mlp_param_count(), master
 * order); the loss is added to *d_loss (double). Forward and backward GEMMs on the tensor
 * cores. Async. */
int ap_mlp_gradient(const void* d_packed, const float* d_feat, const float* d_target, int n,
                    float* d_grad, double* d_loss, void* stream);
/* One Adam step (Kingma & Ba 2015; beta 0.9 / 0.999, eps 1e-8, bias-corrected with `step`
 * >= 1): gradient of the batch at d_packed (which must hold d_params packed), update of
 * d_params with moments d_m, d_v, then d_grad cleared and d_packed re-packed.
 * d_grad must be zero on entry; *d_loss receives the batch loss added. Async. */
int ap_mlp_train_step(float* d_params, float* d_grad, float* d_m, float* d_v, int step, float lr,
                      const float* d_feat, const float* d_target, int n, double* d_loss,
                      void* d_packed, void* stream);
/* AP_OK, or AP_ERR_TIMEOUT once if a bounded tensor-core wait of an earlier MLP kernel
 * gave up (then its outputs are invalid). Synchronizes the device. */
int ap_mlp_status(void);
/* Features of the current configuration (caller order) into d_feat [n][16]; with d_mu
 * [n][3] given, also training targets d_target [n][3] = R^T (mu - alpha E) / 0.02. */
int ap_mlp_features(ap_ctx* ctx, const double* d_mu, float* d_feat, float* d_target);
/* mu0 [n][3] (double, caller order) = the learned guess for the current configuration,
 * to pass as d_guess to induced_dipoles_pcg(). */
int ap_learned_guess(ap_ctx* ctx, const void* d_packed, double* d_mu0);

/* a4 - The direct-field guess mu0 = alpha_i E_i of the current configuration, in caller order
 * (the start induced_dipoles_pcg takes for a NULL guess), as a base for the trajectory guesses
 * below: with it, ap_extrapolate_guess gives the classical zero-order hold of its error,
 * alpha E(t) + (mu - alpha E)(t-1). d_mu0 [n][3] double, device. Async. */
int ap_direct_guess(ap_ctx* ctx, double* d_mu0);

/* Initial guess from the two previous steps of a trajectory (the paper has no predictor;
 * this is the classical extrapolation, optionally on top of a per-step base guess):
 *   d_out = d_base + 2 (d_mu1 - d_base1) - (d_mu2 - d_base2)
 * with d_mu1, d_mu2 the converged dipoles of steps t-1 and t-2 and d_base, d_base1, d_base2
 * the base guesses of steps t, t-1, t-2 (e.g. ap_learned_guess() outputs). Any base pointer
 * may be NULL for zero, so (NULL, mu1, NULL, mu2, NULL) gives 2 mu(t-1) - mu(t-2). All
 * arrays [n][3] double, device, one common atom order; d_out may alias d_base. n >= 1.
 * Async on `stream` (cudaStream_t, NULL = legacy default stream); AP_ERR_ARG for a NULL
 * d_mu1, d_mu2 or d_out or n < 1, AP_ERR_CUDA if the launch fails. */
int ap_extrapolate_guess(int n, const double* d_base, const double* d_mu1, const double* d_base1,
                         const double* d_mu2, const double* d_base2, double* d_out, void* stream);

/* Adaptive trajectory guess: a least-squares predictor on the error of a per-step base
 * guess over the three previous steps (the paper has none):
 *   e_k = d_mu_k - d_base_k, k = 1, 2, 3 (1 = the previous step; NULL bases are zero),
 *   c = (e1 - e2).(e2 - e3) / |e2 - e3|^2 clamped to [0, 1] (0 when e2 = e3),
 *   d_out = d_base + e1 + c (e1 - e2).
 * c is the coefficient that best predicted the previous step's change of e from the change
 * before it: about 0 (hold the last error) for uncorrelated, random-walk motion, about 1
 * (linear extrapolation) for steady motion. All arrays [n][3] double, caller order, device
 * memory; c is computed and used on the device (no synchronization, deterministic).
 *   d_scratch  device memory of AP_ADAPTIVE_SCRATCH doubles, zeroed before its first use;
 *              the call leaves it ready for the next (scratch[0] holds the last c). */
#define AP_ADAPTIVE_SCRATCH 520
int ap_adaptive_guess(int n, const double* d_base, const double* d_mu1, const double* d_base1,
                      const double* d_mu2, const double* d_base2, const double* d_mu3,
                      const double* d_base3, double* d_out, double* d_scratch, void* stream);

/* Polarization energy without allocation - the paper has no counterpart; it is a
 * convenience for callers that cannot allocate device memory: code whose device memory
 * all belongs to another framework's pool, loops that forbid allocation after set-up,
 * and callers that hold no ap_ctx (creating one allocates the whole workspace).
 * Computes E_pol = -(f/2) sum_i mu_i . E_i, f = 332.063713, the energy that
 * polarization_energy_forces() returns for the same dipoles and field.
 *   d_mu, d_field  [n][3] double device arrays (any common atom order).
 *   n              1 <= n <= 16,777,216 (larger n returns AP_ERR_ARG, nothing launched).
 *   d_energy       [1] double device output, kcal/mol.
 *   stream         cudaStream_t to enqueue on (NULL = legacy default stream).
 * Allocates nothing and calls no allocating routine: its scratch is a 32 KB array of
 * block partial sums that every GPU loading the library holds until the process exits.
 * The first call on each device looks up that array's device address (with the
 * device current); make that first call before any stream capture. The address is kept
 * for the rest of the process: after cudaDeviceReset() on a device the array is reloaded
 * elsewhere, so do not call this entry point on that device again. All calls share
 * the array and it keeps the last call's partials, so calls whose kernels overlap on the
 * GPU (e.g. on two streams at once) race and must be serialised by the caller.
 * Errors are described by ap_last_error(NULL). Returns once the work is enqueued. */
int polarization_energy_noalloc(const double* d_mu, const double* d_field, int n,
                                double* d_energy, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* AMOEBAPOL_H */
