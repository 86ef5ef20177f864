/*
 * eelsdda.h -- C ABI of the GB300 (sm_103a) discrete-dipole solver for
 * electron energy-loss (EELS) and cathodoluminescence (CL) probabilities of a
 * particle in an arbitrary, possibly absorbing or Cherenkov, host medium
 * (Kichigin & Yurkin, arXiv:2208.01348).
 *
 * Problem statement followed (Sec. 2 of the paper):
 *   - particle: cubic lattice of nx*ny*nz cells of edge d, each empty or filled
 *     with one of n_mat materials (permittivity eps_p per loss energy);
 *   - host: relative permittivity eps_h with Im eps_h >= 0 (Sec. 2.1);
 *   - electron: kinetic energy (keV) along +z through (x0, y0), z0 = 0 (Sec. 2.2,
 *     Sec. S5);
 *   - per loss energy hbar*omega and beam: the dipole system
 *       alpha~_i^-1 p~_i - sum_{j!=i} G~(r_i - r_j) p~_j = E_inc(r_i)
 *     (point-dipole discretisation of Eq. 8, Green's tensor Eq. 5 with the
 *     complex host wavenumber k = m_h omega / c, Clausius-Mossotti
 *     polarizability with radiative reaction, incident field Eq. 25), then
 *       P_EELS (Eq. 32, 37), P_ext (Eq. 17, 48), P_abs (Eq. 18) and
 *       P_CL (Eq. 42; far field integrated over the sphere), all in eV^-1.
 *
 * Geometry: lattice centred at the origin; cell (ix,iy,iz) has centre
 * ((ix+1/2) - nx/2) d, ((iy+1/2) - ny/2) d, ((iz+1/2) - nz/2) d.  The
 * occupancy array is uint8 [nz][ny][nx] (x fastest): 0 empty, k>0 material k.
 * Dipoles are numbered in that x-fastest order of the occupied cells.
 *
 * Units at the boundary: nm, eV, keV; dipole moments p in SI (C m s, the
 * frequency-domain moment p = 4 pi eps0 eps_h p~).
 *
 * Ownership: the caller owns every buffer passed in.  Host inputs are copied
 * before the call returns; outputs are written only on success (or with
 * EELS_E_NOT_CONVERGED, see below).  A context owns all device memory it
 * allocates and frees it in eels_destroy.  Device-pointer entry points
 * (suffix _dev) read and write caller device memory on the given stream and
 * return once the work is enqueued (the caller synchronises), unless their
 * comment says otherwise.
 *
 * Errors: every int-returning call returns 0 on success or a negative
 * EELS_E_* code; eels_last_error(ctx) describes the last failure of that
 * context (thread-compatible: one thread per context at a time).
 */
#ifndef EELSDDA_H
#define EELSDDA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    EELS_OK = 0,
    EELS_E_INVALID_ARG = -1,   /* bad sizes, d <= 0, Im eps_h < 0 (active host, excluded in Sec. 2.1) */
    EELS_E_BEAM_INSIDE = -2,   /* trajectory crosses an occupied cell: sources and particle overlap (Sec. 2.1) */
    EELS_E_THRESHOLD = -3,     /* |1 - beta_h^2| < 1e-12: gamma_h of Eq. 24 is singular */
    EELS_E_NOT_CONVERGED = -4, /* outputs written; stats flag the unconverged points */
    EELS_E_OOM = -5,           /* device allocation failed */
    EELS_E_CUDA = -6,          /* CUDA runtime error */
    EELS_E_TIMEOUT = -7,       /* a bounded device-side wait expired */
    EELS_E_NO_GRID = -8,       /* eels_set_grid not called */
    EELS_E_UNSUPPORTED = -9    /* e.g. padded FFT length outside the supported range */
};

enum { EELS_FP64 = 0, EELS_MIXED = 1 };          /* precision of the Krylov iterations */
/* Krylov solver: EELS_QMR2 = QMR from coupled two-term recurrences (the variant
 * the paper found fastest, Sec. S5; the default), EELS_QMR = QMR from the
 * three-term Lanczos recurrence (both for complex-symmetric matrices),
 * EELS_BICGSTAB = BiCGStab with the conjugated inner product. */
enum { EELS_QMR = 0, EELS_BICGSTAB = 1, EELS_QMR2 = 2 };
/* Interaction term and polarizability (the options the paper recommends,
 * Sec. S5, "-int igt_so" and "-pol igt_so"; it gives no formulas, this
 * library's reading):
 *   EELS_INT_POINT  the Green's tensor (Eq. 5) between cell centres;
 *   EELS_INT_IGT_SO the Green's tensor averaged over the source cell, with
 *                   exp(ik|R - s|) expanded around the cell centre to second
 *                   order in k and the geometric cell integrals exact, for
 *                   lattice offsets of max-norm <= 3 (the point tensor beyond);
 *   EELS_POL_CM     Clausius-Mossotti with radiative reaction,
 *                   1/alpha = 1/alpha_CM - (2/3) i k^3;
 *   EELS_POL_IGT_SO also the k^2 term of the cell's own field:
 *                   1/alpha = 1/alpha_CM - (2/3)(c1 k^2 d^2 + i k^3 d^3)/d^3,
 *                   c1 = 3 ln(2 + sqrt 3) - pi/2. */
enum { EELS_INT_POINT = 0, EELS_INT_IGT_SO = 1 };
enum { EELS_POL_CM = 0, EELS_POL_IGT_SO = 1 };

typedef struct { double re, im; } eels_c128;

typedef struct eels_ctx eels_ctx;

typedef struct {
    int nx, ny, nz;          /* lattice extents (cells) */
    double d_nm;             /* cell edge (dipole spacing) */
    const uint8_t* occ;      /* host, [nz][ny][nx], 0 = empty, k = material k (1-based) */
    double origin_nm[3];     /* position of the lattice centre in the frame in which the beams
                                (x0, y0) and the phase reference point z0 = 0 of Eq. 25 are given;
                                0, 0, 0 = the lattice centred on the origin.  Moving the lattice
                                by origin_nm is the same problem as moving every trajectory by
                                -origin_nm (the probabilities change only through the beams'
                                positions relative to the particle; p by the phase of the new
                                reference point).  Must be finite (EELS_E_INVALID_ARG) */
} eels_grid;

typedef struct { double x0_nm, y0_nm; } eels_beam;   /* electron along +z, z0 = 0 */

typedef struct {
    double ekin_keV;         /* electron kinetic energy */
    int precision;           /* EELS_FP64: FP64 Krylov; EELS_MIXED: FP32 Krylov + FP64 refinement */
    int solver;              /* EELS_QMR2, EELS_QMR or EELS_BICGSTAB */
    double eps_it;           /* target relative residual ||b - A x|| / ||b|| (FP64) of the Jacobi-scaled system */
    double eps_inner;        /* EELS_MIXED: relative residual target of each FP32 inner solve */
    int max_iter;            /* Krylov iterations per inner solve (and in total for EELS_FP64) */
    int n_dir;               /* far-field directions: 0 = no CL, else 10*4^L+2 (icosphere level L; 2562 = L4) */
    int max_batch;           /* (energy, beam) systems solved together; 0 = choose from free memory */
    int inner_max_iter;      /* EELS_MIXED: FP32 iterations per inner solve before the FP64 residual is
                                recomputed and the inner solve restarts (0 = max_iter) */
    double beam_dir[3];      /* direction of the electron (any non-zero length; default 0, 0, 1).  A
                                beam (x0, y0) is the trajectory through x0 e1 + y0 e2 along n, where
                                (e1, e2, n) is the lattice frame turned by the smallest rotation that
                                takes z to n (a half turn about x for n = -z); the phase of Eq. 25 is
                                referred to that point.  The paper's electron moves along z (Sec. 2.2;
                                the direction option of its solver, Sec. S5) */
    int interaction;         /* EELS_INT_POINT (default) or EELS_INT_IGT_SO */
    int polarizability;      /* EELS_POL_CM (default) or EELS_POL_IGT_SO */
    int device_loop;         /* 0 (default): the host launches the captured iterations in bursts of
                                1 to 8 graph replays and reads the number of active systems between
                                bursts; 1: each inner solve is one graph launch whose WHILE node
                                repeats the captured iterations until no system is active or the
                                iteration budget is spent (no host wait inside a solve; profilers
                                that cannot see into conditional graphs then see none of its kernels).
                                Results are bit-identical either way */
} eels_opts;

typedef struct {
    int iters;               /* Krylov iterations (all inner solves) */
    int refinements;         /* FP64 residual evaluations */
    double residual;         /* final FP64 relative residual of the Jacobi-scaled system */
    int converged;           /* 1 if residual <= eps_it */
} eels_point_stats;

/* Fill opts with defaults: 100 keV, EELS_MIXED, EELS_QMR2, eps_it 1e-8,
 * eps_inner 1e-5, max_iter 20000, n_dir 2562, max_batch 0, inner_max_iter 2000,
 * beam along +z, EELS_INT_POINT, EELS_POL_CM
 * (FP32 Lanczos recurrences lose biorthogonality on hard systems; restarting
 * every 2000 iterations from the FP64 residual keeps the iteration count
 * near that of the FP64 solve; 2000 was the fastest of 1000-4000 on the
 * 128^3-FFT Cherenkov sphere and the rod map). */
void eels_default_opts(eels_opts* opts);

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (may be NULL: the context creates its own non-blocking stream). */
int eels_create(eels_ctx** out, int device, void* cuda_stream);

/* Free every device allocation of the context (NULL allowed). */
void eels_destroy(eels_ctx* ctx);

/* Text of the context's last error ("" if none).  Valid until the next call. */
const char* eels_last_error(const eels_ctx* ctx);

/* Set the particle lattice (copies occ and origin_nm).  Returns
 * EELS_E_INVALID_ARG for non-positive extents or d, a non-finite origin, or
 * an empty lattice; EELS_E_UNSUPPORTED if a padded FFT length (smallest even
 * 7-smooth >= 2n-1 per axis) exceeds 256 (more than 128 cells along an axis).
 * Tuning choices of a lattice shape timed before on this context are
 * restored (eels_tile_widths). */
int eels_set_grid(eels_ctx* ctx, const eels_grid* grid);

/* Number of occupied cells of the current grid (dipoles N). */
int eels_num_dipoles(const eels_ctx* ctx);

/* Padded FFT extents chosen for the current grid. */
int eels_padded_dims(const eels_ctx* ctx, int* mx, int* my, int* mz);

/* Tile widths (z-adjacent lines per block, 8, 16 or 32) of the FFT x pass
 * in FP32 and FP64 that the library picked for the current grid by timing
 * each width on the first eels_solve of a lattice shape (no counterpart in
 * the paper: a tuning step of this implementation).  0 until that solve has
 * run (a size heuristic is used meanwhile).  The choices of every timed
 * shape (lattice and padded dims, contiguous columns, number of materials)
 * are kept by the context: eels_set_grid of a shape timed before restores
 * them instead of timing again. */
int eels_tile_widths(const eels_ctx* ctx, int* xw32, int* xw64);

/* Choices the library timed for the register x pass of the current grid
 * (FFT x lengths 64 and 128, FP32) on the first eels_solve of its shape
 * (no counterpart in the paper: a tuning step of this
 * implementation): *mode 1 = U lines loaded and stored by the threads,
 * 2 = moved by tensor copies (TMA) through shared memory; *spb = beams of
 * one energy one block takes (its staged D-hat serves all of them).  0 and
 * 0 until that solve has run, or when the grid does not use that pass. */
int eels_tuned_xpass(const eels_ctx* ctx, int* mode, int* spb);

/* Every candidate the library timed for the register x pass of the current
 * grid shape (see eels_tuned_xpass): *n receives their number, and the first
 * min(cap, *n) go to mode[i], spb[i] and ms[i] (milliseconds of three
 * launches on the batch of the first solve).  *n = 0 before that solve or when
 * the grid does not use that pass.  Host arrays of cap entries (cap = 0 only
 * counts).  EELS_E_INVALID_ARG for a NULL n or arrays, EELS_E_NO_GRID without
 * a grid. */
int eels_xpass_timings(const eels_ctx* ctx, int cap, int* n, int* mode, int* spb, float* ms);

/*
 * Solve every (energy, beam) point and reduce the losses.  Host buffers.
 *   energy_eV [n_energy]; eps_p [n_energy][n_mat] (relative permittivity of
 *   material k at energy e); eps_h [n_energy]; beams [n_beam].
 * Outputs ([n_energy][n_beam], eV^-1; any may be NULL except p_eels):
 *   p_eels (Eq. 37), p_cl (Eq. 42, requires opts->n_dir > 0), p_ext (Eq. 48),
 *   p_abs (Eq. 18); p_out [n_energy][n_beam][N][3] SI dipoles; stats per point.
 * Returns EELS_E_NOT_CONVERGED (outputs written) if some point missed eps_it.
 */
int eels_solve(eels_ctx* ctx, const eels_opts* opts, int n_energy, const double* energy_eV,
               int n_mat, const eels_c128* eps_p, const eels_c128* eps_h,
               int n_beam, const eels_beam* beams,
               double* p_eels, double* p_cl, double* p_ext, double* p_abs,
               eels_c128* p_out, eels_point_stats* stats);

/*
 * eels_solve with every array argument in DEVICE memory of the context's
 * device (the problem statement of Sec. 2, as for eels_solve): energy_eV
 * [n_energy] double, eps_p [n_energy][n_mat] and eps_h [n_energy]
 * eels_c128, beams [n_beam] eels_beam; outputs p_eels (required), p_cl,
 * p_ext, p_abs [n_energy][n_beam] double, p_out [n_energy][n_beam][N][3]
 * eels_c128, stats [n_energy][n_beam] eels_point_stats (any output but p_eels
 * may be NULL).  opts is a host struct.  The inputs are read, and the
 * outputs written, in the order of cuda_stream (a cudaStream_t; NULL = the
 * legacy default stream, e.g. torch.cuda.current_stream()); the solve itself
 * runs on the context's stream.  The call returns once the outputs are in
 * place (it synchronises cuda_stream).  The caller's current device must be
 * the context's.  Results are bit-identical to eels_solve on the same inputs.
 * Errors as eels_solve, plus EELS_E_INVALID_ARG for a host or foreign-device
 * pointer (checked with cudaPointerGetAttributes before any work).
 */
int eels_solve_dev(eels_ctx* ctx, const eels_opts* opts, int n_energy, const double* energy_eV,
                   int n_mat, const eels_c128* eps_p, const eels_c128* eps_h,
                   int n_beam, const eels_beam* beams,
                   double* p_eels, double* p_cl, double* p_ext, double* p_abs,
                   eels_c128* p_out, eels_point_stats* stats, void* cuda_stream);

/*
 * Asynchronous form of eels_solve.  The inputs are copied before return; the
 * solve runs on a host thread of the library, on the context's stream.  The
 * outputs are written into the caller's buffers (same meaning and layout as
 * eels_solve) while the job runs: they must stay allocated, and neither they
 * nor the context may be used, until eels_job_wait returns.  Returns
 * EELS_E_INVALID_ARG for missing arguments; every other error of the solve is
 * returned by eels_job_wait.
 */
typedef struct eels_job eels_job;
int eels_solve_async(eels_ctx* ctx, const eels_opts* opts, int n_energy, const double* energy_eV,
                     int n_mat, const eels_c128* eps_p, const eels_c128* eps_h,
                     int n_beam, const eels_beam* beams,
                     double* p_eels, double* p_cl, double* p_ext, double* p_abs,
                     eels_c128* p_out, eels_point_stats* stats, eels_job** job);
/* *done = 1 once the job has finished (non-blocking). */
int eels_job_poll(eels_job* job, int* done);
/* Block until the job finishes, free it, and return the eels_solve code. */
int eels_job_wait(eels_job* job);

/* Device-memory footprint (bytes) eels_solve would allocate for a batch of
 * n_systems (energy, beam) systems of this grid under these options. */
int eels_query_footprint(const eels_grid* grid, const eels_opts* opts, int n_systems, size_t* bytes);

/* ------------------------------------------------------------------------
 * Step-level entry points (parity of individual hot-path steps).
 * ---------------------------------------------------------------------- */

/* K0(z), K1(z) for complex z (|arg z| < pi), FP64, on the device: z, k0, k1
 * are DEVICE arrays of n eels_c128 (interleaved re, im).  Enqueued on
 * cuda_stream (NULL = legacy default stream).  Eq. 25 needs them in the
 * fourth quadrant (Sec. 2.2); accuracy ~1e-15 relative there. */
int eels_bessel_k01_dev(const eels_c128* z, eels_c128* k0, eels_c128* k1, int n, void* cuda_stream);

/* Incident field E_inc (Eq. 25) and auxiliary field E_a (Eq. 34) at the
 * dipoles of the current grid, host outputs [N][3] in V s / m (either may be
 * NULL).  eps_h relative permittivity; beam at (x0, y0). */
int eels_incident_field(eels_ctx* ctx, double ekin_keV, double energy_eV, eels_c128 eps_h,
                        eels_beam beam, eels_c128* e_inc, eels_c128* e_aux);

/* eels_incident_field for an electron along beam_dir (see eels_opts.beam_dir;
 * NULL means +z): Eq. 25 and Eq. 34 written in the electron's frame. */
int eels_incident_field_dir(eels_ctx* ctx, double ekin_keV, double energy_eV, eels_c128 eps_h,
                            eels_beam beam, const double* beam_dir, eels_c128* e_inc, eels_c128* e_aux);

/* y = A x for the dipole matrix of the current grid, A = diag(alpha~^-1) - G~
 * in SI (m^-3), x and y host [n_vec][N][3].  precision selects the FP64 or the
 * FP32 FFT path (the same kernels eels_solve uses).  eps_p [n_mat]. */
int eels_apply_matrix(eels_ctx* ctx, int precision, double energy_eV, int n_mat, const eels_c128* eps_p,
                      eels_c128 eps_h, int n_vec, const eels_c128* x, eels_c128* y);

/* Interaction term and polarizability used by eels_apply_matrix and
 * eels_prepare_operator of this context (eels_solve takes them from its
 * eels_opts); default EELS_INT_POINT, EELS_POL_CM.  EELS_E_INVALID_ARG for
 * unknown values. */
int eels_set_interaction(eels_ctx* ctx, int interaction, int polarizability);

/* Prepare the Jacobi-scaled operator A' = I - a^1/2 G~' a^1/2 (lattice
 * units: lengths in d, a = alpha~/d^3) for one system per entry, so that
 * eels_matvec_dev can apply it.  Builds D-hat (FFT of the Green's tensor,
 * Eq. 5, on the padded lattice) in FP64 and FP32; consecutive entries with
 * identical energy and permittivities (the beams of one energy) share one
 * D-hat, which the FFT x pass then reads once for up to 16 of them.  Host
 * inputs as in eels_solve (eps_p [n_energy][n_mat]). */
int eels_prepare_operator(eels_ctx* ctx, int n_energy, const double* energy_eV, int n_mat, const eels_c128* eps_p,
                          const eels_c128* eps_h);

/* y = A' x for n_sys prepared systems (n_sys <= n_energy of the last
 * eels_prepare_operator).  x, y: DEVICE arrays [n_sys][3][N] (component-major
 * per system; dipoles in the library's internal order: the occupied cells
 * sorted by ix, then iy, then iz, iz fastest) of complex64 (precision EELS_MIXED) or complex128
 * (EELS_FP64); x and y must not overlap.  Enqueued on cuda_stream (NULL =
 * legacy default stream); the context's FFT scratch is used, so calls on one
 * context must not overlap in time.  The caller's current device must be the
 * context's (EELS_E_INVALID_ARG otherwise).  This is the FFT matrix-vector
 * product every Krylov iteration applies. */
int eels_matvec_dev(eels_ctx* ctx, int precision, const void* x, void* y, int n_sys, void* cuda_stream);

/* One Krylov solve A' x = b on the operator prepared by
 * eels_prepare_operator (the Jacobi-scaled form of the dipole system of
 * Eq. 8, solved in the paper's code by QMR or BiCGStab, Sec. S5), for n_sys
 * systems (n_sys <= n_energy of the last eels_prepare_operator):
 *   b, x: DEVICE arrays [n_sys][3][N] (component-major per system, dipoles in
 *   the internal order of eels_matvec_dev) of complex64
 *   (precision EELS_MIXED: FP32 vectors and matvecs, FP64 scalars) or
 *   complex128 (EELS_FP64); b and x must not overlap.
 *   solver: EELS_QMR2, EELS_QMR or EELS_BICGSTAB; x starts from 0 and the
 *   solve stops when the (quasi-)residual norm is <= eps ||b|| or after
 *   max_iter iterations.
 *   status, iters: optional HOST arrays [n_sys]: 1 converged, 2 iteration
 *   limit, 3 breakdown (the Lanczos process of QMR fails when v^T v vanishes,
 *   e.g. at a right-hand side with b^T b ~ 0: x is then left at 0), and the
 *   iterations run.
 * b is read after the work already queued on cuda_stream; x is complete in
 * the order of cuda_stream when the call returns (the iterations run on the
 * context's stream, with host reads of the convergence counter between
 * bursts of graph replays).  The caller's current device must be the
 * context's.  Uses the context's Krylov buffers: calls on one context must
 * not overlap in time. */
int eels_krylov_solve_dev(eels_ctx* ctx, int precision, int solver, const void* b, void* x, int n_sys,
                          double eps, int max_iter, int* status, int* iters, void* cuda_stream);

/* Kernels launched by this library in this process so far (graph replays
 * count their kernel nodes). */
long long eels_kernel_launches(void);

/* ------------------------------------------------------------------------
 * The same matrix-vector product for callers that cannot allocate device
 * memory.  The paper has no counterpart; this is a library-integration
 * entry point.  Callers that cannot let a library allocate at the time of
 * the call include real-time or latency-critical loops that must not meet
 * the allocator's implicit synchronisation, and hosts (plugins inside a
 * larger application, frameworks with their own caching pool) that own all
 * device memory and forbid foreign allocations.  eels_matvec_dev_noalloc applies the operator prepared by
 * eels_prepare_operator with the same kernels as eels_matvec_dev, but takes
 * its FFT scratch from one fixed array compiled into the library
 * (EELS_NOALLOC_SCRATCH_BYTES = 64 MiB of device memory, held by every GPU
 * that loads the library until the process exits) and calls no allocator.
 *
 *  - Arguments as for eels_matvec_dev (the current device must be the
 *    context's).  The scratch needed is
 *    n_sys * 3 * My * Nx * Mz * (8 or 16 bytes); larger requests return
 *    EELS_E_UNSUPPORTED ("pass fewer systems per call") before any launch.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, with the context's device made current for the
 *    lookup); make that first call before any stream capture.
 *  - Every call on a device shares the one array and leaves its contents
 *    behind; nothing in it has to start at zero (each call writes every
 *    scratch element it reads first).  Calls that overlap on the GPU (two
 *    streams, two threads, two contexts) race on the array: serialise them. */
#define EELS_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
int eels_matvec_dev_noalloc(eels_ctx* ctx, int precision, const void* x, void* y, int n_sys, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Serving loop.  Requests (one eels_solve each: a lattice, options and its
 * (energy, beam) points) are queued in arrival order; a free worker takes the
 * first waiting request whose device-memory footprint fits the unreserved
 * budget.  Each worker owns a stream and a context, so admitted requests run
 * concurrently on the device.  A request's results do not depend on which
 * other requests run beside it.  The paper runs one independent solver
 * process per parameter set (Sec. 3.1, Sec. S5); this replaces those runs.
 * ---------------------------------------------------------------------- */
typedef struct eels_server eels_server;

enum { EELS_JOB_QUEUED = 0, EELS_JOB_RUNNING = 1, EELS_JOB_DONE = 2, EELS_JOB_FAILED = 3 };
enum { EELS_SERVER_DRYRUN = 1 };   /* workers hold the slot without GPU work (scheduler tests) */

typedef struct {
    int device;
    size_t hbm_budget;       /* bytes admitted requests may reserve (0 = 80% of free memory) */
    int max_concurrent;      /* worker threads / streams, >= 1 */
    int flags;               /* EELS_SERVER_DRYRUN or 0 */
} eels_server_opts;

typedef struct {
    int state;               /* EELS_JOB_* */
    int code;                /* eels_solve return code once finished */
    double t_submit, t_start, t_end;   /* seconds since the server was created */
    size_t footprint;        /* bytes reserved while running */
    int n_points;
} eels_job_info;

int eels_server_create(eels_server** out, const eels_server_opts* opts);

/* Queue a request (all inputs are copied; same meaning as eels_solve).  The
 * request is batched so that its footprint fits hbm_budget / max_concurrent;
 * EELS_E_OOM if even one system exceeds hbm_budget. */
int eels_server_submit(eels_server* s, const eels_grid* grid, const eels_opts* opts, int n_energy,
                       const double* energy_eV, int n_mat, const eels_c128* eps_p, const eels_c128* eps_h,
                       int n_beam, const eels_beam* beams, long long* job_id);

/* Non-blocking status of a request. */
int eels_server_poll(eels_server* s, long long job_id, eels_job_info* info);

/* Block until the request finishes; copy its outputs ([n_energy][n_beam],
 * any may be NULL) and return its eels_solve code. */
int eels_server_wait(eels_server* s, long long job_id, double* p_eels, double* p_cl, double* p_ext, double* p_abs,
                     eels_point_stats* stats, eels_job_info* info);

/* Most requests ever running at once, requests finished, bytes reserved now. */
int eels_server_stats(eels_server* s, int* running_max, int* completed, size_t* in_use);

/* Finish running requests, drop queued ones, join the workers. */
void eels_server_destroy(eels_server* s);

/* Particle-related total light-emission probability P_CL^tot (Eq. 41, in
 * its second form C_enh - C_ext + C_sca): out[i] = p_eels[i] - p_ext[i] +
 * p_cl[i] for i < n, eV^-1, host arrays (out may alias an input).  It is
 * meaningful in a non-absorbing host (Sec. 2.6) and equals p_cl below the
 * Cherenkov threshold.  EELS_E_INVALID_ARG for n < 0 or NULL arrays. */
int eels_cl_total(int n, const double* p_eels, const double* p_ext, const double* p_cl, double* out);

/* Loss of the electron to the host alone (no particle) per unit path
 * length, as a probability density in eV^-1 m^-1: Eq. 29 (Frank-Tamm) with
 * the (2/pi)/(hbar^2 w) of Eq. 37; it does not depend on the loss energy for
 * a host with constant eps_h, and is 0 at and below the Cherenkov threshold
 * (Eq. 28).  eps_h must be real and positive (W0 diverges in an absorbing
 * host, Sec. 2.5): EELS_E_INVALID_ARG otherwise. */
int eels_frank_tamm(double ekin_keV, eels_c128 eps_h, double* dp_dz);

/* A vacuum problem equivalent to a particle in a real host (Sec. 2.7).
 * Eq. 43-44 scale every refractive index by 1/eta and every length by 1/xi;
 * with eta = m_h = sqrt(eps_h) the host becomes vacuum.  Rules (flags):
 *   EELS_SCALE_ENERGY  Eq. 45: xi = 1 -- same lattice and beams, loss
 *                      energy m_h * energy_eV, same probabilities;
 *   EELS_SCALE_LENGTH  Eq. 46: xi = 1/m_h -- lattice spacing and beam
 *                      offsets times m_h, same loss energy, probabilities
 *                      of the vacuum problem divided by m_h;
 *   | EELS_SCALE_ULTRAREL  Eq. S16, only above the Cherenkov threshold
 *                      (beta_h > 1), approximate (quasi-static field,
 *                      Eq. S15): the vacuum problem runs at v = c and its
 *                      probabilities are further divided by beta_h^2.
 * Outputs (host struct): ekin_keV, the vacuum kinetic energy with speed m_h v
 * (Eq. 47), or +inf for v = c (a vacuum solve then takes a kinetic energy
 * large enough that w b / (gamma v) is negligible); energy_eV, the loss
 * energy of the vacuum problem; length_scale, the factor on d_nm and beam
 * offsets; eps_p_scale = 1/eps_h, the factor on every particle permittivity
 * taken at the ORIGINAL loss energy; p_scale, with P_host = p_scale *
 * P_vacuum for P_EELS, P_CL, P_ext and P_abs.  eps_h is real (eta must be,
 * Eq. 43).  EELS_E_INVALID_ARG for eps_h <= 0, ekin_keV <= 0, energy_eV <= 0,
 * unknown flags, or a rule on the wrong side of the threshold (the exact
 * rules need beta_h < 1, Eq. S16 beta_h > 1). */
enum { EELS_SCALE_ENERGY = 0, EELS_SCALE_LENGTH = 1, EELS_SCALE_ULTRAREL = 2 };
typedef struct {
    double ekin_keV, energy_eV, length_scale, eps_p_scale, p_scale;
} eels_vacuum_map;
int eels_vacuum_equivalent(int rule, double ekin_keV, double eps_h, double energy_eV, eels_vacuum_map* out);

/* Extrapolation of one result to zero dipole size (Sec. 3.2): values[i]
 * computed with dipole size d[i] (n >= 3 points, any length unit, d > 0)
 * are fitted with a0 + a1 d + a2 d^2 by least squares with weights d^-6
 * (errors taken to grow as d^3).  *value0 = a0; *ci95 = twice the standard
 * error of a0 (residual-scaled covariance; 0 when n == 3), the nominal 95 %
 * interval.  Host arrays.  EELS_E_INVALID_ARG for n < 3, d <= 0 or a
 * singular fit. */
int eels_extrapolate(int n, const double* d, const double* values, double* value0, double* ci95);

/* The far-field direction grid the CL reduction uses (icosphere with
 * n_dir = 10*4^L+2 vertices): dirs [n_dir][3] unit vectors, weights
 * [n_dir] (sum 4 pi).  Host outputs. */
int eels_directions(int n_dir, double* dirs, double* weights);

#ifdef __cplusplus
}
#endif

#endif /* EELSDDA_H */
