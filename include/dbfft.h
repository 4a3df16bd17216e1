/*
 * dbfft.h -- C ABI of the GB300 DBFFT library.
 *
 * DBFFT (Lucarini & Segurado, "DBFFT: A displacement based FFT approach for
 * non-linear homogenization of the mechanical behavior", arXiv 1905.12725)
 * solves the periodic cell problem of a voxel microstructure with the Fourier
 * coefficients of the displacement fluctuation as the unknown. Each linear
 * system is solved matrix-free by a preconditioned conjugate gradient; one
 * operator application is
 *     Fourier gradient -> inverse 3-D FFT -> per-voxel tangent contraction
 *     -> forward 3-D FFT -> Fourier divergence
 * (Sec. 2.2 Eq. lineqf for small strain, Sec. 2.4 Eq. nonlineqf for finite
 * strain) and the preconditioner is one 3x3 block per frequency (Sec. 2.5,
 * Eqs. pred2-pred3).
 *
 * Conventions used by every entry point
 * -------------------------------------
 * Grid: n[0] x n[1] x n[2] voxels, each a power of two in [8, 256] or an
 *   odd length in [9, 245] whose prime factors are 3, 5 and 7; voxel
 *   (i1, i2, i3) is stored at i3 + n3 * (i2 + n2 * i1) (i3 contiguous).
 * Fourier fields ("half spectrum"): layout [B][3][n1][n2][n3/2 + 1],
 *   interleaved complex (re, im), complex128 (FP64) or complex64 (FP32),
 *   forward transform unnormalised with kernel e^{-i xi.x}. Frequency k_i is
 *   stored in FFT order; xi_i = 2 pi k_i / L_i and the Nyquist index of an
 *   even axis carries xi_i = 0 (the paper treats odd grids only, Sec. 2.1;
 *   this is the even-grid reading). The null set Z = {xi = 0} (8 modes on an
 *   all-even grid) carries no unknown: inputs there are ignored and outputs
 *   are zero.
 * Operator: the library applies the Hermitian positive definite form
 *   K = B^H C B with B(u, e) = F^-1(s.u) + E e, which is -1/N times the
 *   paper's d:F(C:F^-1(s.u)). Its solution is the paper's.
 * Macro unknowns (stress and mixed control, Sec. 2.3 and Sec. 2.4 "Stress
 *   and mixed control"): arrays [B][9]. Small strain stores the coefficients
 *   on the orthonormal Mandel basis (order 11, 22, 33, 23, 13, 12) in entries
 *   0..5; finite strain stores F components at index 3i + j. Only the
 *   stress-controlled components are unknowns; the others are ignored on
 *   input and zero on output.
 * Inner product: Re sum over the full spectrum of conj(a) b (the half
 *   spectrum weighted 1 on the k3 = 0 and k3 = n3/2 planes, 2 elsewhere) plus
 *   the dot product of the macro unknowns.
 * Ownership: every pointer passed in is borrowed for the duration of the
 *   call. The context copies the material and load data at creation. Device
 *   pointers must be on the context's device and must be 16-byte aligned.
 * Errors: every entry point returns a dbfft_status; nothing is thrown across
 *   the ABI. On failure dbfft_last_error(ctx) describes the cause. CUDA
 *   errors are reported as DBFFT_E_CUDA and leave the context unusable.
 * Streams: all device work of a context runs on the stream given at
 *   creation; calls return after that work is complete unless stated.
 */
#ifndef DBFFT_H
#define DBFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DBFFT_OK = 0,
    DBFFT_E_ARG = 1,              /* invalid argument or inconsistent sizes           */
    DBFFT_E_UNSUPPORTED_GRID = 2, /* grid size outside the compiled set               */
    DBFFT_E_NOMEM = 3,            /* device allocation failed                         */
    DBFFT_E_CUDA = 4,             /* a CUDA call failed                               */
    DBFFT_E_NOT_CONVERGED = 5,    /* iteration cap hit; results and report written    */
    DBFFT_E_NONFINITE = 6,        /* NaN/Inf met in a residual or a material table    */
    DBFFT_E_TIMEOUT = 7,          /* a bounded device wait gave up                    */
    DBFFT_E_MATERIAL = 8,         /* a local constitutive update failed               */
    DBFFT_E_STATE = 9             /* call not valid in the context's current state    */
} dbfft_status;

enum { DBFFT_SMALL = 0, DBFFT_FINITE = 1 };       /* kinematics (Sec. 2.2 / Sec. 2.4) */
enum { DBFFT_FP64 = 0, DBFFT_MIXED = 1 };        /* precision of the solve           */
enum {                                           /* constitutive model of a phase    */
    DBFFT_ISO_ELASTIC = 0,     /* linear isotropic elasticity (E, nu), small strain     */
    DBFFT_NEO_HOOKE = 1,       /* compressible Neo-Hookean (mu, lambda), finite strain  */
    DBFFT_CP_FCC_POWERLAW = 2, /* small-strain FCC crystal plasticity, power-law flow   */
    DBFFT_SVK = 3,             /* St. Venant-Kirchhoff (mu, lambda), finite strain: the
                                  porous hyperelastic example of Sec. 3; needs mu > 0 and
                                  3 lambda + 2 mu > 0                                   */
    DBFFT_CP_FCC_FINITE = 4    /* FCC crystal plasticity at finite strain, F = Fe Fp
                                  (Sec. 2.4 with the flow rule of Sec. 3): the second
                                  Piola-Kirchhoff stress of the intermediate
                                  configuration is the small-strain model's stress at
                                  the trial Green strain, Fp is advanced by the slip
                                  rates; same phase fields as DBFFT_CP_FCC_POWERLAW,
                                  FINITE kinematics required                         */
};

/* Problem size and solver settings. */
typedef struct {
    int n[3];          /* voxels per axis: powers of two in [8, 256], or odd lengths
                          9 .. 245 whose prime factors are 3, 5, 7 (the paper's odd
                          grids, Sec. 2.1; with nonlinear phases an odd n3 is one
                          of 9, 15, 21, 27, 45, 63, 81; dbfft_adjoint and
                          dbfft_displacement need an even n3)                       */
    double L[3];       /* box edge lengths; 0 means 1                                    */
    int batch;         /* B: right-hand sides solved together (>= 1)                     */
    int n_materials;   /* Bm: distinct material maps; B % Bm == 0; solve b uses map
                          b / (B / Bm), so B / Bm right-hand sides share one map          */
    int kinematics;    /* DBFFT_SMALL or DBFFT_FINITE                                    */
    int precision;     /* DBFFT_FP64: everything FP64. DBFFT_MIXED: FFTs, contraction
                          and inner CG in FP32; residual, update and stresses in FP64     */
    double tol;        /* linear problems: stop at ||b - K x|| <= tol ||b|| (FP64 residual) */
    int max_iter;      /* cap on inner CG iterations per inner solve                     */
    double newton_tol; /* nonlinear: equilibrium residual ||div P||_L2 / ||<P>||         */
    double load_tol;   /* nonlinear: loading residual ||<P>_IJ - Pbar_IJ|| / ||<P>||     */
    double eta_inner;  /* inner CG relative tolerance (refinement and Newton forcing)    */
    int max_newton;    /* cap on Newton (or refinement) steps per increment              */
} dbfft_grid;

/* One phase. Only the fields of its model are read. */
typedef struct {
    int model;                /* DBFFT_ISO_ELASTIC, DBFFT_NEO_HOOKE, DBFFT_CP_FCC_POWERLAW,
                                 DBFFT_SVK, DBFFT_CP_FCC_FINITE                            */
    double E, nu;             /* ISO_ELASTIC                                               */
    double mu, lambda;        /* NEO_HOOKE and SVK: Lame constants                         */
    double C11, C12, C44;     /* CP: cubic stiffness in the crystal frame                  */
    double gdot0, m, tau_c;   /* CP: gdot = gdot0 |tau/tau_c|^(1/m) sign(tau)              */
    double quat[4];           /* CP: unit quaternion (w, x, y, z), crystal -> sample       */
} dbfft_phase;

/* Microstructure. The maps are copied at creation; the caller keeps ownership. */
typedef struct {
    const uint16_t* phase_id; /* [n_materials][n1][n2][n3] phase index per voxel          */
    const double* E_scale;    /* optional [n_materials][n1][n2][n3]: factor on the
                                 stiffness of ISO_ELASTIC voxels (NULL means 1)            */
    int n_phases;
    const dbfft_phase* phases;/* [n_phases] host array; one context uses one model kind    */
    int device_arrays;        /* 0: phase_id and E_scale are host memory; 1: device memory
                                 of the context's GPU (copied device to device on the
                                 context's stream; ids and scales are checked there)       */
} dbfft_materials;

/* Macroscopic load program (Sec. 2.3, Sec. 2.4). */
typedef struct {
    unsigned stress_mask;  /* bit 3i+j set: component ij of the macro stress (sigma or P)
                              is prescribed; otherwise the macro strain (or F) is.
                              Must be symmetric for DBFFT_SMALL.                            */
    const double* target;  /* host [B][9] (row-major 3x3): end-of-ramp value of the
                              prescribed strain / F on strain-controlled components and of
                              the stress on stress-controlled ones                          */
    int n_increments;      /* increment k (0-based) applies the fraction (k+1)/n of the
                              ramp from 0 (small strain) or I (finite strain)               */
    double total_time;     /* rate-dependent models: time step = total_time / n_increments */
} dbfft_load;

/* Optional device allocator (e.g. a framework's caching allocator). */
typedef struct {
    void* (*alloc)(size_t bytes, void* user);
    void (*free)(void* ptr, void* user);
    void* user;
} dbfft_allocator;

/* Per-call report. */
typedef struct {
    int newton_iters;      /* Newton steps (nonlinear) or FP64 refinement steps (linear)  */
    int outer_iters;       /* FP64 residual evaluations                                   */
    long long cg_iters;    /* inner CG iterations summed over the batch                   */
    int cg_iters_max;      /* max over the batch of inner CG iterations                   */
    double eps_eq;         /* max over the batch of ||div sigma||_L2 / ||<sigma>||       */
    double load_res;       /* max over the batch of the loading residual                  */
    double true_rel_res;   /* linear: max over the batch of ||b - K x|| / ||b|| in FP64   */
    double wall_ms;        /* wall time of the call                                       */
} dbfft_report;

typedef struct dbfft_ctx dbfft_ctx;

/* Flags of dbfft_apply. */
enum {
    DBFFT_APPLY_FP32 = 1,     /* fields are complex64 / float, operator in FP32 (else FP64) */
    DBFFT_APPLY_PRECOND = 2,  /* out = M u, the preconditioner of Sec. 2.5 (else K u)      */
    DBFFT_APPLY_RESIDUAL = 4  /* out = b - K u for increment 0 (FP64 only): the residual of
                                 Eq. lineqf / Sec. 2.3 with the macro load                  */
};

/*
 * Create a context: copies the materials and the load, allocates device
 * memory (through *alloc when given, else cudaMalloc) and prepares twiddle
 * tables. stream is a cudaStream_t (NULL: the legacy default stream).
 * Grid limits: see dbfft_grid.n. All phases must use one model kind, and
 * the kind must match the kinematics (ISO_ELASTIC and CP with SMALL,
 * NEO_HOOKE and SVK with FINITE). Errors: E_ARG, E_UNSUPPORTED_GRID, E_NOMEM,
 * E_NONFINITE (a non-finite material parameter), E_CUDA.
 */
dbfft_status dbfft_create(const dbfft_grid* grid, const dbfft_materials* mat,
                          const dbfft_load* load, const dbfft_allocator* alloc,
                          void* stream, dbfft_ctx** out);

/*
 * Apply the DBFFT operator K (Sec. 2.2 Eq. lineqf in SPD form; with macro
 * unknowns the system of Sec. 2.3), its preconditioner M (Sec. 2.5) or the
 * residual b - K u, to a batch of device vectors, with the tangent the
 * context holds now (the stiffness for linear phases; the tangent of the
 * last constitutive update otherwise). u_hat / out: device, layout above;
 * e_in / e_out: device [B][9] macro parts, or NULL when no component is
 * stress-controlled. out may not alias u_hat.
 */
dbfft_status dbfft_apply(dbfft_ctx* ctx, int flags, const void* u_hat, const void* e_in,
                         void* out, void* e_out);

/*
 * Solve load increment inc (0 <= inc < n_increments; increments must be
 * called in order for path-dependent models). Linear phases: PCG (FP64) or
 * FP32 PCG inside FP64 iterative refinement (MIXED) to grid.tol. Nonlinear:
 * Newton (Sec. 2.4, Eq. lineariz) with inner PCG to eta_inner, stopped by
 * newton_tol and load_tol; the preconditioner uses the mean tangent at the
 * first iterate of the increment. rep may be NULL. Returns E_NOT_CONVERGED
 * when a cap is hit (the state and report are still written).
 * From the second inner solve of a context on, an inner PCG runs as one
 * CUDA graph launch (a WHILE node around one iteration); with the
 * environment variable DBFFT_CUDA_GRAPHS=0 at dbfft_create it runs launch
 * by launch instead (same kernels and results; for kernel profilers).
 */
dbfft_status dbfft_solve_increment(dbfft_ctx* ctx, int inc, dbfft_report* rep);

/* Homogenized stress <sigma> (small) or <P> (finite) of the current state,
 * computed in FP64: host out[B][9], row-major 3x3. */
dbfft_status dbfft_homogenized_stress(dbfft_ctx* ctx, double* out);

/*
 * Effective stiffness of linear elastic microstructures: the six unit Mandel
 * macro strains solved as right-hand sides of one batched solve. Requires
 * DBFFT_SMALL, ISO_ELASTIC phases, no stress-controlled components and
 * B == 6 * n_materials. host out[n_materials][6][6], Mandel basis,
 * out[g][i][j] = sigma_i for unit strain j. Overwrites the current solution.
 */
dbfft_status dbfft_homogenized_tangent(dbfft_ctx* ctx, double* out, dbfft_report* rep);

/*
 * Sensitivity of J_b = sum_ij dJ_dsigma[b][ij] <sigma>_ij to the per-voxel
 * Young's modulus E(x) of ISO_ELASTIC phases under full strain control
 * (C(x) = E(x) C1(nu(x))). Solves the forward problem of increment 0 (or
 * reuses it: when the last call that changed the state was a converged
 * dbfft_solve_increment(ctx, 0) or dbfft_adjoint, no forward solve runs and
 * the report counts the adjoint solve alone), then the adjoint problem with
 * the same self-adjoint operator (Sec. 2.2: the system is Hermitian) and
 * assembles
 *   dJ/dE(x) = (1/N) (g + B lam)(x) : C1(x) : eps(x),  g = sym(dJ_dsigma),
 * where lam solves K lam = -B^H C g. dJ_dsigma: host [B][9];
 * dJ_dE: device [B][n1][n2][n3] double. Not available with stress control.
 */
dbfft_status dbfft_adjoint(dbfft_ctx* ctx, const double* dJ_dsigma, double* dJ_dE,
                           dbfft_report* rep);

/*
 * Sensitivity of J_g = sum_IJ G[g][I][J] C_g,IJ, C_g the 6x6 Mandel effective
 * stiffness of material map g (dbfft_homogenized_tangent, Sec. 2.2: the six
 * unit Mandel strains), to the per-voxel Young's modulus E(x) of
 * ISO_ELASTIC phases (C(x) = E(x) C1(nu(x))). C_IJ = (1/N) sum_x
 * eps^I : C : eps^J with eps^I the strain field of unit strain I, and the
 * system is self-adjoint (Sec. 2.2), so the adjoint fields are the forward
 * ones and no further solve is needed:
 *   dJ/dE(x) = (1/N) sum_IJ G_IJ eps^I(x) : C1(x) : eps^J(x).
 * Runs the six unit-strain solves unless the last call that changed the state
 * was a converged dbfft_homogenized_tangent (or this function), then
 * assembles in FP64. Requirements as dbfft_homogenized_tangent, even n3.
 * G: host [n_materials][6][6]; dJ_dE: device [n_materials][n1][n2][n3]
 * double; C_eff: host [n_materials][6][6] or NULL (the stiffness used).
 * Errors: E_ARG, E_STATE, E_UNSUPPORTED_GRID, and those of the solve.
 */
dbfft_status dbfft_tangent_sensitivity(dbfft_ctx* ctx, const double* G, double* dJ_dE, double* C_eff,
                                       dbfft_report* rep);

/*
 * Checkpoints of the crystal-plasticity increments (DBFFT_CP_FCC_POWERLAW):
 * with enable = 1, set before the first increment, every converged increment
 * keeps its stress field (device, B * V * 6 doubles per increment, allocated
 * at the first increment for all n_increments) as the record that
 * dbfft_cp_adjoint sweeps back over. Errors: E_STATE (another model, or
 * increments already solved).
 */
dbfft_status dbfft_set_checkpointing(dbfft_ctx* ctx, int enable);

/*
 * Adjoint of the path-dependent crystal-plasticity increments (Sec. 2.4,
 * Eq. lineariz: each increment is a converged Newton solve with the
 * self-adjoint tangent operator of Sec. 2.2; R14 flow rule). J_b =
 * sum_ij dJ_dsigma[b][ij] <sigma>_ij after the current (last solved)
 * increment; s(x) a factor on the elastic stiffness of voxel x. Returns
 * dJ/ds(x) at s = 1 (the derivative with respect to the logarithm of each
 * voxel's stiffness) in dJ_ds: device [B][n1][n2][n3] double. The reverse
 * sweep runs one FP64 PCG solve per increment, to grid.tol, with the
 * tangent rebuilt from each increment's checkpoint; the state adjoint
 * carries dJ / d(plastic strain) from one increment to the one before.
 * Needs dbfft_set_checkpointing(ctx, 1) before increment 0, the FP64
 * precision and an even n3. The forward state is restored afterwards.
 * Errors: E_ARG, E_STATE, E_UNSUPPORTED_GRID, E_MATERIAL (a checkpoint whose
 * tangent is not positive definite), E_NOT_CONVERGED.
 */
dbfft_status dbfft_cp_adjoint(dbfft_ctx* ctx, const double* dJ_dsigma, double* dJ_ds, dbfft_report* rep);

/* Copy the current FP64 solution: u_hat device complex128 [B][3][n1][n2][n3/2+1]
 * (may be NULL), e host [B][9] (may be NULL). */
dbfft_status dbfft_get_solution(dbfft_ctx* ctx, void* u_hat, double* e);

/*
 * Total displacement of the current solution at the voxel centres
 * (Sec. 2.2, Eqs. disp_decomp and decomp_displ; Sec. 2.4): u(x) = Hbar x +
 * u~(x), u~ the inverse DFT of the unknown u-hat (the periodic fluctuation,
 * zero mean), Hbar the whole macro strain (DBFFT_SMALL) or Fbar - I
 * (DBFFT_FINITE), including the solved stress-controlled components.
 * Voxel (i1, i2, i3) sits at x_a = (i_a + 1/2) L_a / n_a. out: device double
 * [B][3][n1][n2][n3], written in full; the transforms run in FP64 on the
 * context's stream. Errors: E_ARG (null pointer), E_CUDA.
 */
dbfft_status dbfft_displacement(dbfft_ctx* ctx, double* out);

/*
 * Compatibility residual of the current solution (Sec. 3, Eq. chedckcomp and
 * its finite-strain form): small strain |curl (curl eps)^T| / ||<eps>||,
 * finite strain |curl F| / ||<F> - I||, with |.| the root mean square over the
 * cell (Parseval on the half spectrum; the paper takes the maximum over the
 * voxels) and ||.|| the Frobenius norm. Zero up to round-off, since the
 * fluctuation is a gradient by construction. out: host double [B]. Errors:
 * E_ARG, E_STATE (no solution yet), E_CUDA.
 */
dbfft_status dbfft_compatibility(dbfft_ctx* ctx, double* out);

/* One row of the per-pass profile. */
typedef struct {
    char name[40];       /* pass and precision, e.g. "axis3_apply_f32"                  */
    long long launches;  /* launches recorded                                           */
    double ms;           /* summed device time between CUDA events around each launch    */
    double bytes;        /* summed algorithmic DRAM bytes (reads + writes the pass needs) */
} dbfft_profile_entry;

/*
 * Profiling of the context's own kernels (no counterpart in the paper; a
 * measurement aid). dbfft_profile(ctx, 1) clears the table and brackets every
 * later launch on the context's stream with CUDA events; dbfft_profile(ctx, 0)
 * stops. dbfft_profile_read fills up to max_entries rows and returns the
 * number of rows. dbfft_launch_count returns the number of kernels the
 * context has launched since creation.
 */
dbfft_status dbfft_profile(dbfft_ctx* ctx, int enable);
int dbfft_profile_read(dbfft_ctx* ctx, dbfft_profile_entry* out, int max_entries);
long long dbfft_launch_count(const dbfft_ctx* ctx);

/*
 * Operator application that allocates nothing (no counterpart in the paper;
 * this is a deployment aid). Some callers cannot let a library call
 * cudaMalloc: a host application whose device memory is owned by a caching
 * pool (a deep-learning framework that has reserved most of the GPU, where
 * an extra driver allocation can fail or fragment the pool), or a caller
 * that must not pay the latency and implicit device synchronisation of an
 * allocation on its critical path (e.g. a solver calling the operator many
 * times inside its own iteration). This entry point needs no context: it
 * computes out = K u_hat exactly as dbfft_apply does for FP64, small strain,
 * linear isotropic phases and full strain control (no macro unknowns), and
 * keeps its work buffer, its frequency / twiddle tables and a copy of the
 * Lame constants in static device arrays inside the library.
 *
 * n[3]: grid, powers of two in [8, 256]; L[3]: box lengths (NULL: all 1);
 * batch: right-hand sides, each with its own material map;
 * phase_id: device uint16 [batch][n1][n2][n3], every id < n_phases;
 * n_phases: entries of lam and mu, in [1, 65536]; lam, mu: device double
 * [n_phases] Lame constants indexed by phase_id; u_hat, out: device
 * complex128 [batch][3][n1][n2][n3/2+1] (out may not alias u_hat); stream: a
 * cudaStream_t (NULL: legacy default stream).
 *
 * The call is host-synchronous: it returns after the work is done, because
 * it reports the check of the phase ids. An id at or beyond n_phases is
 * never used to index the caller's lam / mu (the copies cover every uint16
 * value); the call then returns DBFFT_E_ARG and out is unspecified. The
 * frequency and twiddle tables are uploaded only when n or L differs from
 * the previous call on the device.
 *
 * Limit: the static work buffer holds 16 MiB, i.e.
 * batch * 6 * n1 * n2 * (n3/2 + 1) * 16 bytes <= 16 MiB (one 64^3 field, or
 * seven 32^3 fields) and batch <= 1024; larger requests return DBFFT_E_ARG
 * and touch no device memory.
 * The buffer is shared by every call in the process and keeps the last
 * call's contents; nothing in it needs to start at zero (each call
 * overwrites what it reads, and clears the phase-check flag itself). Calls
 * that overlap on the GPU (from several streams or threads at once) race on
 * it and must be serialised by the caller. The first call on a device looks
 * up the device addresses of the static arrays; every GPU on which the
 * library's device code is loaded holds the 16 MiB (plus 1 MiB of tables)
 * until the process exits.
 * Errors: E_ARG, E_UNSUPPORTED_GRID, E_CUDA; the message of the calling
 * thread's last failure is dbfft_last_error(NULL).
 */
dbfft_status dbfft_apply_iso_noalloc(const int n[3], const double L[3], int batch, const uint16_t* phase_id,
                                     int n_phases, const double* lam, const double* mu, const void* u_hat,
                                     void* out, void* stream);

/*
 * Autotuner (no counterpart in the paper; launch-shape selection for the
 * GPU). Times candidate launch shapes of the inner solve's passes on the
 * context's own buffers -- the radix and the grid lines per CTA of pass 3,
 * and the columns per CTA of the strided transforms -- and keeps the fastest
 * for later calls. cache_path (may be NULL): a text file of earlier results,
 * one line per GPU / grid / batch / precision / model; a matching line is
 * used without timing, a new result is appended. Results are unchanged by
 * tuning up to floating-point reassociation inside pass 3's block sums.
 * dbfft_tuning returns a short text of the choice (valid until the next call).
 */
dbfft_status dbfft_autotune(dbfft_ctx* ctx, const char* cache_path);
const char* dbfft_tuning(const dbfft_ctx* ctx);

/*
 * Set the launch shape of pass 3 for the operator applications of one inner
 * precision by hand (no counterpart in the paper), in place of the
 * autotuner's choice. fp64: 0 for the FP32 applications, 1 for FP64.
 * pipelined: 0 = one CTA per group of grid lines, loads staged by cp.async;
 * 1 = persistent CTAs looping over tiles of `lines` grid lines with two
 * shared-memory stages filled and drained by bulk copies; 2 = the same with
 * one stage (half the shared memory per CTA); 3 = the line-bulk pass of the
 * FP32 applications on lines of n3 = 64, 128 or 256 values (linear isotropic,
 * small-strain crystal-plasticity and Neo-Hookean models): one tile of
 * `lines` grid lines per CTA moved by bulk copies, each line transformed in
 * place by two register stages (radix: the most threads per CTA, e.g. 192;
 * 0 or 384 for up to 384; -1 for warp lines: every warp takes its own lines
 * of a 16-line tile through all phases; -2 the same with tiles of 8 lines
 * (n3 = 256) or 4 lines (n3 = 64, 128), two lines per warp). radix: 8 or 16 (FP32), 4
 * (FP64), or 32 with the plain kernel when n3 <= 256 (FP32) / 64 (FP64):
 * one thread per grid line, or 32 values of a line per thread beyond
 * (FP32) / 4 (FP64); lines: grid lines per CTA (per tile when pipelined;
 * then even and dividing n1 * n2). Returns DBFFT_E_ARG for a shape that does
 * not exist or does not fit in shared memory; the results of the operator do
 * not depend on the shape beyond floating-point reassociation.
 */
dbfft_status dbfft_set_pass3_shape(dbfft_ctx* ctx, int fp64, int pipelined, int radix, int lines);

/* Right-hand sides per CTA of the line-bulk pass 3 (pipelined = 3 above; an
 * execution choice, no counterpart in the paper). rhs: 0 for the context's
 * default group (the largest divisor of the right-hand sides per material map,
 * at most 8, that the plain pass fits in 256 threads), else 1 to 8 dividing the
 * right-hand sides per material map: fewer per CTA give more, smaller CTAs.
 * dbfft_autotune sets it with the line-bulk shape. Returns DBFFT_E_ARG for a
 * value that does not divide, or (when the line-bulk pass is in use) a tile
 * that no longer fits in shared memory; results do not depend on it beyond
 * floating-point reassociation of the curvature sums.
 */
dbfft_status dbfft_set_pass3_rhs_group(dbfft_ctx* ctx, int rhs);

/*
 * Refresh policy of the preconditioner's reference stiffness for the
 * nonlinear models (Sec. 2.5 takes the volume average of the tangent; the
 * paper computes it at the start of each increment, and its hyperelastic
 * example keeps the initial tangent). DBFFT_PRECOND_PER_INCREMENT (default):
 * the mean tangent at the first Newton iterate of each increment.
 * DBFFT_PRECOND_INITIAL: the mean initial stiffness (K(I) for NEO_HOOKE and
 * SVK, the elastic stiffness for CP), never refreshed.
 * DBFFT_PRECOND_PER_NEWTON: the mean tangent at every Newton iterate. The
 * converged solution does not depend on the policy; the number of CG
 * iterations does. Takes effect at the next dbfft_solve_increment.
 * Errors: E_ARG (unknown policy).
 */
enum { DBFFT_PRECOND_PER_INCREMENT = 0, DBFFT_PRECOND_INITIAL = 1, DBFFT_PRECOND_PER_NEWTON = 2 };
dbfft_status dbfft_set_precond_refresh(dbfft_ctx* ctx, int policy);

/*
 * FP64 fused multiply-add rate of the current device in TFLOP/s (no
 * counterpart in the paper; a measurement aid for the FP64 roofline of the
 * residual chain): eight independent FMA chains per thread, eight 256-thread
 * CTAs per SM, best of four timed launches on `stream`. Allocates a small
 * output buffer with cudaMallocAsync. Errors: E_ARG, E_NOMEM, E_CUDA.
 */
dbfft_status dbfft_fp64_fma_rate(double* tflops, void* stream);

/*
 * L2 copy bandwidth of the current device in GB/s (no counterpart in the
 * paper; a measurement aid for workloads whose fields stay in L2 between
 * passes, such as 64^3 x 6 right-hand sides): 16 MB copied to 16 MB, 32 times
 * over by eight 256-thread CTAs per SM, read and write bytes counted, best of
 * four timed launches on `stream`. Allocates the 32 MB with cudaMallocAsync.
 * Errors: E_ARG, E_NOMEM, E_CUDA.
 */
dbfft_status dbfft_l2_copy_rate(double* gbs, void* stream);

/* Device bytes held by the context. */
size_t dbfft_device_bytes(const dbfft_ctx* ctx);

/* Release the context and its device memory (NULL is a no-op). */
void dbfft_destroy(dbfft_ctx* ctx);

/* Message of the last error of ctx ("" if none); valid until the next call.
 * ctx = NULL: the calling thread's last failure of a context-free call
 * (dbfft_apply_iso_noalloc), "" if none. */
const char* dbfft_last_error(const dbfft_ctx* ctx);

/* Name of a status code. */
const char* dbfft_status_string(dbfft_status s);

#ifdef __cplusplus
}
#endif
#endif /* DBFFT_H */
