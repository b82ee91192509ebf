/* recon.h: C ABI of the GB300 (sm_103a) iterative Fourier-space reconstruction library.
 *
 * The method is that of Burden, Percival & Howlett, "Reconstruction in Fourier space" (2015):
 * tracers are binned on a mesh, the overdensity is smoothed (Sec. 3), and the redshift-space
 * displacement equation (Eq. Nusser)
 *
 *     div Psi + beta div((Psi . r) r) = -delta / b,          beta = f / b,
 *
 * is solved for a radial line of sight by the fixed-point FFT iteration of Sec. 5.1
 * (Eq. iterative): S_n = delta/b + beta div((Psi_n . r) r), Psi_n+1 = Z[S_n], Z[s](k) = i k s / k^2
 * (Eq. Zeldovich).  Galaxies and randoms are then moved back along Psi (Sec. 1; Eq. Lagrange).
 *
 * Conventions shared by every entry point
 *   - Mesh: cubic, N = nmesh[0] = nmesh[1] = nmesh[2] in {32, 48, 64, 96, 128, 256, 384, 512, 1024};
 *     box side L = box[0] = box[1] = box[2] (Mpc/h); nodes at x_i = i L / N; periodic indexing.
 *   - Real fields are float32 [ix][iy][iz] (iz fastest), N^3 values.
 *   - Complex fields on the r2c half grid are float32 pairs [kx][ky][kz], kz = 0..N/2 (N/2+1
 *     values, kz fastest), forward transform e^{-ik.x} unnormalised.
 *   - Positions are (n, 3) row-major (x, y, z per particle), float64 or float32, in [0, L) up to
 *     periodic wrap: a position outside [0, L) stands for its image in [0, L) (the mesh wraps it,
 *     and a galaxy's radial line of sight runs from the observer to that image).  The grid
 *     coordinate x N / L is one float64 product; the cell fraction is then kept in fixed point
 *     (21 bits on the brick-sorted paths, 32 bits on the direct ones, rounded down).  Weights are
 *     float32 or NULL (unit weights).
 *   - Every call is ordered on the CUDA stream given to recon_create.  Calls that return values to
 *     the host (recon_iterate, recon_get_scalars) synchronise that stream.
 *   - Ownership: the handle owns its device fields (inside the caller's workspace when one is
 *     given).  Input pointers are borrowed for the duration of the call.  Output buffers are the
 *     caller's.  A host pointer must be ordinary or pinned host memory; a device pointer must be
 *     memory of the device that was current at recon_create.
 *   - Errors: every entry point returns a recon_status; no exception crosses the ABI.  After
 *     RECON_ERR_CUDA, recon_last_error gives the CUDA message.  A handle whose call failed with
 *     RECON_ERR_CUDA should be destroyed.
 */
#ifndef RECON_GB300_H
#define RECON_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum recon_status {
  RECON_OK = 0,
  RECON_ERR_INVALID_ARG = 1,   /* a null pointer, a size out of range, an unsupported mesh      */
  RECON_ERR_OOM = 2,           /* device allocation failed or the workspace is too small        */
  RECON_ERR_CUDA = 3,          /* a CUDA runtime error; see recon_last_error                    */
  RECON_ERR_NOT_CONVERGED = 4, /* max_iter reached before tol; all outputs are still valid      */
  RECON_ERR_NONFINITE = 5,     /* a NaN or Inf appeared in the convergence norms                */
  RECON_ERR_STATE = 6,         /* calls out of order (create -> deposit -> smooth -> iterate)   */
  RECON_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up                            */
  RECON_ERR_UNSUPPORTED = 8    /* a valid request this build does not implement                 */
} recon_status;

enum { RECON_LOS_RADIAL = 0, RECON_LOS_FIXED = 1 };
enum { RECON_MEAN_RANDOMS = 0, RECON_MEAN_UNIFORM = 1 };
enum { RECON_F64 = 0, RECON_F32 = 1 };

/* Starting estimates of the iteration (Sec. 5.2).  The estimate is
 * Psi_0 = Z[delta/b] - c (Z[delta/b] . r) r with
 *   PLAIN   c = 0                  (Psi_red,FFT: no RSD correction)
 *   APPROX1 c = beta / (1 + beta)  (Eq. approx1, irrotational approximation)
 *   FFTA    c = 3 beta / (7+3 beta)(Eq. approx2, the "RSD-corrected" first estimate)
 * (the paper writes f where this library uses beta = f / b). */
enum { RECON_START_PLAIN = 0, RECON_START_APPROX1 = 1, RECON_START_FFTA = 2 };

/* The coefficient c of a start (above) for beta = f / b, as recon_iterate uses it; host only.
 * INVALID_ARG for an unknown start, a non-finite or negative beta, or a null c. */
recon_status recon_start_coefficient(int start, double beta, double* c);

/* Fields recon_get_field can export. */
enum {
  RECON_FIELD_RHO_G = 0,     /* CIC density of galaxies (real), valid between deposit and smooth */
  RECON_FIELD_RHO_R = 1,     /* CIC density of randoms (real), same validity                     */
  RECON_FIELD_DELTA = 2,     /* smoothed, masked (optionally lognormal) overdensity (real)       */
  RECON_FIELD_DELTA_K = 3,   /* its forward transform on the half grid, valid after iterate      */
  RECON_FIELD_PSI = 4        /* the final displacement, 3 real fields [comp][ix][iy][iz]         */
};

typedef struct recon_params {
  int nmesh[3];            /* N per axis; must be equal                                        */
  double box[3];           /* L per axis (Mpc/h); must be equal; box origin at 0               */
  double b;                /* linear galaxy bias (Sec. 3.2: b = 1.87 for the CMASS mocks)      */
  double f;                /* growth rate; the solve uses beta = f/b, the galaxy shift uses f   */
  double smooth_R;         /* Gaussian smoothing length R (Mpc/h), S(k) = exp(-k^2 R^2 / 2)    */
  int los_mode;            /* RECON_LOS_RADIAL (observer position) or RECON_LOS_FIXED          */
  double observer[3];      /* radial: observer position (Mpc/h); fixed: LOS direction vector   */
  int periodic;            /* 1: shifted positions wrap modulo L; 0: survey (no wrap)          */
  double mask_frac;        /* survey mask: keep nodes whose smoothed random density exceeds
                              mask_frac x sum w_r / (number of nodes that received random
                              mass in the deposit), i.e. of the survey's mean density (0.01)   */
  int lognormal;           /* 1: delta -> ln(max(1+delta, 1e-6)) - <ln(...)> (Eq. logdelta)    */
  int mean_density_mode;   /* RECON_MEAN_RANDOMS (delta from randoms) or RECON_MEAN_UNIFORM    */
} recon_params;

typedef struct recon_catalog {
  const void* pos;         /* (n, 3) positions, dtype below                                    */
  const float* w;          /* (n) weights or NULL for unit weights                              */
  int64_t n;               /* number of particles, 0 allowed                                    */
  int dtype;               /* RECON_F64 or RECON_F32 (positions)                                */
  int on_device;           /* 1: pos and w are device pointers; 0: host pointers (page-locked
                              host memory is read by the direct deposit kernel in place, other
                              host memory goes through the handle's staging buffer in chunks;
                              a call given host memory returns once it has been read)           */
} recon_catalog;

typedef struct recon_handle recon_handle;

/* Bytes of device workspace recon_create needs for these parameters (fields, reductions, host
 * staging).  Fails with INVALID_ARG for an unsupported mesh. */
recon_status recon_workspace_bytes(const recon_params* p, size_t* bytes);

/* Create a reconstruction context on the current device.
 *   stream     cudaStream_t to order all work on (NULL = legacy default stream)
 *   workspace  device memory of at least recon_workspace_bytes bytes, 256-byte aligned, owned by
 *              the caller and kept alive until recon_destroy; NULL makes the handle allocate it
 *              itself with cudaMalloc (and free it in recon_destroy).  A workspace that is not
 *              256-byte aligned gives INVALID_ARG, one smaller than recon_workspace_bytes OOM. */
recon_status recon_create(const recon_params* p, void* stream, void* workspace,
                          size_t workspace_bytes, recon_handle** out);

/* Replace the parameters of a handle by p (same mesh side N; box, b, f, R, observer, LOS, mask and
 * density options may all change), keeping its buffers.  Resets the call sequence (deposit next).
 * INVALID_ARG if p is invalid or its mesh differs. */
recon_status recon_reconfigure(recon_handle* h, const recon_params* p);

/* CIC mass assignment of galaxies and randoms (Sec. 3: binning; CIC instead of NGP) and the
 * weight sums sum w_g, sum w_r (float64) that give alpha = sum w_g / sum w_r.
 * ran may be NULL (or n = 0) only with RECON_MEAN_UNIFORM. */
recon_status recon_deposit(recon_handle* h, const recon_catalog* gal, const recon_catalog* ran);

/* Gaussian smoothing of both densities (Sec. 3.1, 3.2: smoothed before delta is formed),
 * delta = rho_g,s / (alpha rho_r,s) - 1 inside the binary survey mask and 0 outside (Sec. 3.2), or
 * rho_g,s / rho_bar - 1 in RECON_MEAN_UNIFORM mode, then the optional lognormal transform
 * (Sec. 6, Eq. logdelta). */
recon_status recon_smooth(recon_handle* h);

/* The iteration of Sec. 5.1 from the chosen start.  Runs until rel < tol after at least two
 * updates, or max_iter updates, where rel = |Psi_n+1 - Psi_n| / |Psi_n+1| (L2 over all nodes and
 * components, from the Parseval sum of the sources; the first entry is measured against the
 * uncorrected estimate Z[delta/b]).  On return *n_iter is the number of updates and *rel_change
 * the last rel.  Returns NOT_CONVERGED when max_iter was reached with rel >= tol and tol > 0.
 * By default the loop runs on the device as one CUDA graph (RECON_OPT_GRAPH) and the call blocks
 * once, at the end; max_iter <= 1024 in that mode (larger values use the host-driven loop).  The
 * handle keeps the instantiated graph and relaunches it on the next call with the same start, tol,
 * max_iter, options and parameters (recon_reconfigure or a changed value rebuilds it). */
recon_status recon_iterate(recon_handle* h, int start, double tol, int max_iter, int* n_iter,
                           double* rel_change);

/* Network inputs for the learned start (no counterpart in the paper), after recon_smooth.
 * feat (device, M^3 x 5 float32, channels-last, M = N >> level, level 0..2) holds per coarse node
 * the means over its 2^level-node block of (delta, r_x, r_y, r_z, u_s), u_s = (1 - c)(Psi_s . r)
 * the radial displacement of the analytic start `start` (RECON_START_*; Psi_s = Z[delta/b],
 * c as in recon_iterate).  Computes delta(k), S_-1 and u_s on the mesh and keeps them for
 * recon_iterate_from at the same level.  Consumes the real delta copy (RECON_FIELD_DELTA is no
 * longer available).  UNSUPPORTED if N is not a multiple of 2^level. */
recon_status recon_start_features(recon_handle* h, int start, int level, float* feat);

/* The iteration of recon_iterate started from a supplied radial displacement (the learned warm
 * start feeds the network's output here), same stopping rule, outputs and trace:
 *   level 0: u0 (device, N^3 float32 [ix][iy][iz]) is the displacement on the mesh: P_0 = u0 r;
 *            u0 = the converged Psi . r reproduces the fixed point.
 *   level 1, 2: u0 (device, M^3, M = N >> level) is a prediction of the block means of the
 *            converged Psi . r; P_0 = (u_s + U[u0 - mean(u_s)]) r, where u_s and its block means
 *            come from the last recon_start_features at this level (STATE otherwise) and U is
 *            periodic trilinear interpolation with the coarse node J at mesh index
 *            (J + 1/2) 2^level - 1/2.  u0 = the features' u_s channel gives exactly the analytic
 *            start.  Consumes that preparation.
 * u0 is borrowed for the call. */
recon_status recon_iterate_from(recon_handle* h, const float* u0, int level, double tol, int max_iter, int* n_iter,
                                double* rel_change);

/* Block means (level 0..2, as in recon_start_features) of the radial displacement Psi . r of the
 * final Psi (device, M^3 float32), after an iterate: the training target of the learned start. */
recon_status recon_get_radial(recon_handle* h, int level, float* u);

/* The rel values of the last recon_iterate: up to cap entries into rel (host), count into *n. */
recon_status recon_get_trace(recon_handle* h, double* rel, int cap, int* n);

/* Reconstruction shift (Sec. 1; Eq. Lagrange x = q + Psi reversed): Psi is CIC-interpolated to each
 * particle; galaxies move by -[Psi + f (Psi . r) r] with r from the particle position (its image in
 * [0, L), see the conventions above), randoms by -Psi.  shift_out: (n, 3) float32, required.
 * pos_out: (n, 3) float64 shifted positions (wrapped modulo L when periodic) or NULL.  Both are host
 * or device memory as out_on_device says; particle order is the catalogue's. */
recon_status recon_shift(recon_handle* h, const recon_catalog* cat, int is_galaxy,
                         float* shift_out, double* pos_out, int out_on_device);

/* Copy the final displacement, 3 N^3 float32 [comp][ix][iy][iz], to out (host or device). */
recon_status recon_get_psi(recon_handle* h, float* out, int out_on_device);

/* Copy an internal field (RECON_FIELD_*) to out: N^3 float32 for real fields, N*N*(N/2+1) float32
 * pairs for RECON_FIELD_DELTA_K, 3 N^3 float32 for RECON_FIELD_PSI. */
recon_status recon_get_field(recon_handle* h, int which, float* out, int out_on_device);

/* Scalars of the last calls, float64, into out[8]: sum w_g, sum w_r, alpha, mask threshold,
 * lognormal constant C, number of masked-in nodes, last |dPsi|^2, last |Psi|^2. */
recon_status recon_get_scalars(recon_handle* h, double out[8]);

/* Forward 3-D r2c transform of a real N^3 float32 field (device pointer) into the half grid
 * (device pointer), with the library's own FFT passes; uses the handle's field buffers, so it
 * invalidates the reconstruction state. */
recon_status recon_fft_r2c(recon_handle* h, const float* in_real, float* out_half);

/* Unnormalised inverse c2r transform: half grid (device) -> N^3 real (device), equal to N^3 times
 * the inverse DFT. Invalidates the reconstruction state like recon_fft_r2c. */
recon_status recon_fft_c2r(recon_handle* h, const float* in_half, float* out_real);

/* ---- The finite-difference method of Sec. 2.1 (the paper's comparison method) ----------------
 * Solves Eq. mainpot in configuration space after recon_smooth: A phi = delta / b with A the
 * 7-point Laplacian plus beta times the line-of-sight stencil of Sec. 2.1 (sets A, B and C; beta =
 * f / b; a fixed line of sight takes the second differences only), phi = 0 outside the box, then
 * Psi = -grad phi by central differences.  The linear system is solved with BiCGStab (float32
 * vectors, float64 inner products), right-preconditioned by the exact inverse of the periodic
 * 7-point Laplacian (the library's FFT passes on the handle's first field), until the recursive
 * residual falls below tol x |b|.  psi_out: device (3, N^3) float32.  *n_iter: iterations;
 * *rel_resid: the true residual |A phi - b| / |b| at the end (with phi stored in float32 it
 * bottoms out near 1e-5 for fields smooth over a few cells: rounding at the grid scale times the
 * Laplacian's 12 / g^2).  Allocates its 9 Krylov vectors
 * (9 N^3 float32) with cudaMalloc for the call.  The smoothed delta stays valid, so recon_iterate
 * may follow.  NOT_CONVERGED when max_iter is reached; STATE before recon_smooth. */
recon_status recon_fd_solve(recon_handle* h, double tol, int max_iter, int* n_iter, double* rel_resid,
                            float* psi_out);

/* ---- The paper's front end (Sec. 3.2): FKP weights from the radial number density ------------
 * Mean number density nbar (host, nbins float64) of the catalogue cat (device memory) in nbins
 * equal shells of comoving distance [rmin, rmax) about the handle's observer: counts / (sky_area
 * (r_hi^3 - r_lo^3) / 3), sky_area the survey's solid angle in steradians (the n(z) of the paper in
 * distance).  Distances in float64.  Synchronises the handle's stream. */
recon_status recon_radial_nbar(recon_handle* h, const recon_catalog* cat, int nbins, double rmin, double rmax,
                               double sky_area, double* nbar);

/* FKP weights w = 1 / (1 + nbar(r) P0) (Sec. 3.2; the paper takes P0 = 20000 (Mpc/h)^3) for every
 * particle of cat (device), nbar (host, nbins) of the shell holding its distance, 0 outside
 * [rmin, rmax); w_out: device (n) float32, usable as the catalogue's weights in recon_deposit. */
recon_status recon_fkp_weights(recon_handle* h, const recon_catalog* cat, int nbins, double rmin, double rmax,
                               const double* nbar, double P0, float* w_out);

/* ---- Diagnostics of the paper (computed on the GPU) -------------------------------------------
 * Statistics of a ratio, as in Tables 1-3: out[0] mean and out[1] standard deviation (population)
 * of the ratios inside [lo, hi] (the paper cuts ratios above 3 or below -1: lo = -1, hi = 3; a zero
 * denominator is always cut), out[2] the fraction of points cut, out[3] the number kept.  Sums in
 * float64; each ratio is formed in float64 from float32 inputs.  Synchronise the handle's stream. */

/* Eq. ratio (Sec. 4.3, 5.2): (Psi_num . r) / (Psi_den . r) at every particle of cat (device memory),
 * both displacement fields (device, 3 N^3 float32 [comp][ix][iy][iz], e.g. from recon_get_psi)
 * CIC-interpolated to the particle and projected on the particle's line of sight (radial from the
 * handle's observer, or its fixed direction).  With Psi_num the displacement of the real-space
 * tracers and Psi_den an iterate, this is the paper's convergence statistic. */
recon_status recon_radial_ratio(recon_handle* h, const float* psi_num, const float* psi_den, const recon_catalog* cat,
                                double lo, double hi, double out[4]);

/* The same statistics of num[i] / den[i] over n device float32 values (e.g. the Helmholtz
 * components below, node by node). */
recon_status recon_ratio_stats(recon_handle* h, const float* num, const float* den, int64_t n, double lo, double hi,
                               double out[4]);

/* Sec. 4.1 (Eq. Helmholtz, Eq. irrotational, Eq. solenoidal): the plane-parallel split of
 * (Psi . x) x, Psi_x = psi_x (device, N^3 float32), into grad A (Fourier components
 * (k_j k_x / k^2) Psi_x(k), derivative wavenumbers zero at the Nyquist index) and curl B =
 * (Psi_x) x - grad A; grad_a and curl_b are device (3, N^3) float32 outputs.  Uses the handle's
 * FFT passes and fields, so it invalidates the reconstruction state like recon_fft_r2c. */
recon_status recon_helmholtz_x(recon_handle* h, const float* psi_x, float* grad_a, float* curl_b);

/* Kernel kinds counted and (optionally) timed by the handle. */
enum {
  RECON_K_DEPOSIT = 0,   /* CIC deposit from brick-sorted particles      */
  RECON_K_ZFWD = 1,      /* Z pass, r2c (densities, FFT export)          */
  RECON_K_ZINV = 2,      /* Z pass, c2r of the smoothed densities        */
  RECON_K_ZDELTA = 3,    /* Z pass: z smoothing, delta, r2c              */
  RECON_K_ZPROJ = 4,     /* Z pass: c2r, radial projection, r2c          */
  RECON_K_ZFINAL = 5,    /* Z pass: c2r of the final Psi                 */
  RECON_K_LINE_FWD = 6,      /* plain x-line FFT pass, forward               */
  RECON_K_LINE_INV = 7,      /* plain x-line FFT pass, inverse               */
  RECON_K_CONV = 8,      /* x / y Gaussian smoothing convolutions        */
  RECON_K_KDELTA = 9,    /* y-line pass: delta(k), S_-1 and Z[delta/b]   */
  RECON_K_KITER = 10,    /* y-line pass: source update, norms and Z[S]   */
  RECON_K_SHIFT = 11,    /* sorted CIC interpolation and shift           */
  RECON_K_OTHER = 12,    /* reductions, FFT export passes                */
  RECON_K_SORT = 13,     /* particle pack + brick counting sort          */
  RECON_K_COUNT = 14
};

/* Enable (1) or disable (0) CUDA-event timing of every kernel launch on the handle's stream.
 * Launch counts are always kept. */
recon_status recon_set_timing(recon_handle* h, int enable);

/* Launch count, summed algorithmic bytes (the bytes each launch must read and write at least:
 * its input and output fields and particle arrays) and, if timing was enabled, summed device
 * milliseconds of one kernel kind since the last recon_reset_timing.  Synchronises the stream
 * when timing is on.  Any output pointer may be NULL. */
recon_status recon_get_timing(recon_handle* h, int kind, double* total_ms, int64_t* launches,
                              double* alg_bytes);

/* Zero the launch counts and timings. */
recon_status recon_reset_timing(recon_handle* h);

/* CIC deposit for callers that cannot allocate device memory.  (The paper has no counterpart: it
 * is a service entry point of this library.)  Some callers may not allocate: plugins whose host
 * application owns every device buffer through its own pool, and real-time pipelines that must
 * not enter an allocator (or its synchronisation) once they run.  This call allocates nothing
 * and uses no handle: the caller passes every input and output, and the only scratch (per-block
 * partial sums of the weights) is a fixed 32 KB array inside the library's device image, kept by
 * every device that loads the library until the process exits.
 *   pos     device (n, 3) positions, dtype RECON_F64 or RECON_F32, in [0, box) up to periodic wrap
 *   w       device (n) float32 weights or NULL (unit weights)
 *   n       0 .. 67,108,864 particles per call (the scratch bound); larger n -> INVALID_ARG
 *   nmesh   mesh side, 2 .. 2048; box > 0 is the side length
 *   rho     device nmesh^3 float32, overwritten with the CIC density (zeroed first)
 *   sum_w   device float64, overwritten with the sum of the weights
 *   stream  cudaStream_t the work is ordered on
 * The first call on each device looks up the scratch array's device address (once, with that
 * device current) and keeps it for the process; make that first call before any stream capture
 * begins.  After cudaDeviceReset the kept address is stale: do not call this entry point on a
 * device that was reset since its first call.  Every call shares the
 * one scratch array, which keeps the last call's partial sums: calls that overlap on the GPU (on
 * different streams, or from several host threads without ordering) race on it and must be
 * serialised by the caller.  Errors: INVALID_ARG for bad arguments or too many particles, CUDA
 * for a runtime error. */
recon_status recon_cic_deposit_noalloc(const void* pos, int dtype, const float* w, int64_t n, int nmesh,
                                       double box, float* rho, double* sum_w, void* stream);

/* Handle options (recon_set_option). */
enum {
  RECON_OPT_DEPOSIT_PATH = 0,   /* RECON_PATH_DIRECT (default) or RECON_PATH_SORTED               */
  RECON_OPT_SHIFT_PATH = 1,     /* RECON_PATH_SORTED (default) or RECON_PATH_DIRECT               */
  RECON_OPT_GRAPH = 2,          /* 1 (default): recon_iterate runs the whole loop as one CUDA graph
                                   with a conditional WHILE node and a device-side convergence
                                   test; 0: the host reads the norms after every update.  Kernel
                                   timing (recon_set_timing) always uses the host-driven loop.   */
  RECON_OPT_LINE_TILE = 3,      /* FFT tile of the x-line passes: 0 (default) 16 adjacent columns
                                   (128-byte rows) per tile, 1: 8 columns                         */
  RECON_OPT_REUSE_SORT = 5,     /* 0 (default); 1: a recon_shift of the catalogue last given to
                                   recon_deposit (same pointer, n, dtype and memory kind, no
                                   pos_out) reuses the brick order the sorted deposit made of it
                                   (RECON_PATH_SORTED deposit, n <= 2^25) instead of reading and
                                   sorting the positions again; the caller guarantees they did not
                                   change in between.  While that order is held, shifts of other
                                   catalogues take the direct path.                              */
  RECON_OPT_KSPACE_GENERIC = 4, /* 0 (default): for N = 512 the source update and the projection
                                   pass run in kernels that keep the first and last FFT stages
                                   (and the c2r/r2c pairing) in registers; 1: the generic staged
                                   kernels (same butterflies)                                     */
  RECON_OPT_KITER_TMA = 8,      /* N = 512 register-fused path: 0 (default) one CTA per tile loading its
                                   inputs itself; 1 persistent CTAs whose inputs (A, P_y, delta(k), S)
                                   are streamed into shared memory by the tensor memory accelerator,
                                   the next tile while the current one is transformed.  Same
                                   arithmetic per element (Psi bitwise equal); the norm sums are
                                   accumulated per thread over several tiles, so the trace differs in
                                   float32 rounding.  Slower on GB300 (1.42 against 1.03 ms per
                                   launch), kept as an option.                                    */
  RECON_OPT_ASSIGN = 7,         /* mass assignment of recon_deposit: 0 (default) cloud-in-cell, 1 the
                                   paper's nearest grid point (Sec. 3: node floor(x N / L + 1/2)),
                                   always on the direct (unsorted) deposit kernel.  The shift still
                                   interpolates Psi with CIC.                                     */
  RECON_OPT_FFT_RADIX = 9,      /* radix order of every FFT plan of the handle's mesh: 0 (default)
                                   largest radix first; 1 smallest first, for N = 256 (4 8 8, its
                                   z half-length plan 4 4 8) and N = 384 (6 8 8; 3 8 8), other
                                   meshes UNSUPPORTED.  Same transforms up to float32 rounding;
                                   the batch autotuner times both.                               */
  RECON_OPT_PLANE_BATCH = 6     /* register-fused path (N = 512): 0 (off) or 16, 32, 64 y-planes per
                                   batch; each update then runs its inverse x, projection and forward
                                   x passes batch by batch, so a batch's fields stay in the L2 between
                                   the three passes (same arithmetic, fewer HBM round trips).  A
                                   multiple of the x-line tile width (16, or 8 with RECON_OPT_LINE_TILE) */
};
/* Particle paths: DIRECT handles each particle independently (8 global atomics per deposited
 * particle; 24 scattered reads per interpolated one); SORTED packs the particles, counting-sorts
 * them by 8^3-cell brick and works brick by brick in shared memory (deposit: one global atomic per
 * touched node of the brick; shift: Psi staged once per brick).  Both give the same results up to
 * float32 summation order. */
enum { RECON_PATH_DIRECT = 0, RECON_PATH_SORTED = 1 };

/* Set a handle option (values 0 or 1, RECON_OPT_PLANE_BATCH 0/16/32/64); INVALID_ARG for an unknown
 * option or value; UNSUPPORTED for RECON_OPT_FFT_RADIX 1 on a mesh with one radix order; CUDA if
 * rebuilding the stage tables for another radix order fails. */
recon_status recon_set_option(recon_handle* h, int option, int value);

/* One reconstruction of a batch (recon_batch_run). */
typedef struct recon_batch_item {
  recon_params params;     /* any supported mesh; items are grouped by mesh side               */
  recon_catalog gal;       /* galaxies, as for recon_deposit                                     */
  recon_catalog ran;       /* randoms (ignored with RECON_MEAN_UNIFORM)                          */
  int start;               /* RECON_START_*                                                      */
  double tol;              /* as for recon_iterate                                               */
  int max_iter;            /* 1 .. 1024                                                          */
  float* shift_gal;        /* (n_gal, 3) galaxy shifts, or NULL for none                         */
  float* shift_ran;        /* (n_ran, 3) random shifts, or NULL for none                         */
  int out_on_device;       /* shift buffers are device (1) or host (0) memory                    */
  int n_iter;              /* out: updates done                                                  */
  double rel;              /* out: last |dPsi|/|Psi|                                             */
  int status;              /* out: recon_status of this item (OK or NOT_CONVERGED on success)    */
  float ms;                /* out: device milliseconds from the start to the end of this item's
                              work (in the one-graph mode, between two device timer stamps; work
                              of another size class may overlap it)                              */
} recon_batch_item;

/* Reconstruct many mocks of uneven mesh and catalogue sizes (deposit -> smooth -> iterate ->
 * shift each; a batched form of the method with no counterpart in the paper).  Items are grouped by
 * mesh side; each size class uses one handle (allocated with cudaMalloc, freed before returning).
 * When every catalogue and shift buffer is device memory, each item is one CUDA graph (deposit,
 * smoothing, start, the iteration as a conditional WHILE node with the device-side stopping test,
 * shifts), and the graphs are launched on `stream` back to back, smallest mesh first: the host
 * builds each item's graph while the device runs the items before it, and waits once, at the end.
 * Otherwise the items run one after another through the handle API.  flags is a bitwise OR of
 * RECON_BATCH_*.  With RECON_BATCH_TUNE, a size class not seen before in this process is first
 * tuned on its first item, before the batch runs and outside every item's time: the deposit path,
 * the x-line FFT tile width, at N = 512 the k-space kernel family (register-fused or generic), at
 * N = 256 and 384 the FFT radix order, and the shift path; the fastest are kept for the process
 * (recon_batch_plan).  With RECON_BATCH_ONE_GRAPH the whole batch is one CUDA graph, built before
 * it is launched, with one chain of items per size class and the chains side by side (one item
 * per class in flight).  Other bits: INVALID_ARG.  Returns the first error of any item (per-item
 * statuses in items[i].status), else OK. */
enum { RECON_BATCH_TUNE = 1, RECON_BATCH_ONE_GRAPH = 2 };
recon_status recon_batch_run(recon_batch_item* items, int n_items, void* stream, int flags);

/* The schedule the batch autotuner chose for mesh side nmesh (STATE if none yet): the values of
 * RECON_OPT_LINE_TILE, RECON_OPT_DEPOSIT_PATH, RECON_OPT_SHIFT_PATH and RECON_OPT_FFT_RADIX it
 * runs the class with; any output pointer may be NULL. */
recon_status recon_batch_plan(int nmesh, int* line_tile, int* deposit_path, int* shift_path, int* fft_radix);

/* ---- Learned warm start: a small 3-D U-Net (no counterpart in the paper) ----------------------
 * The network maps, per node of a periodic mesh, 5 input channels — smoothed overdensity delta,
 * the three components of the line of sight r, and the radial displacement u_0 = Psi_0 . r of the
 * Eq. approx2 start — to the radial displacement u = Psi . r of the converged solution of Eq. Nusser
 * (its head adds its output to u_0).  Three levels of widths c1, 2 c1, 4 c1 with two 3x3x3
 * convolutions + ReLU each, 2x2x2 average pooling, nearest-neighbour upsampling, skip
 * concatenation, periodic padding.  Tensors are float32 channels-last on the device:
 * x[(ix n + iy) n + iz][c].  Parameters are one float32 array, layer by layer (enc1a, enc1b, enc2a,
 * enc2b, bota, botb, dec2a, dec2b, dec1a, dec1b, head), each as weights w[tap][cin][cout]
 * (tap = (dx+1) 9 + (dy+1) 3 + (dz+1); the head has one tap) then biases b[cout]. */
typedef struct recon_unet recon_unet;

/* Number of float32 parameters for width c1 (8 or 16). */
recon_status recon_unet_param_count(int c1, size_t* count);
/* Network with float32 master weights and AdamW state; activations stored as bfloat16
 * (bf16_storage = 1) or float32; all sums in float32.  Allocates its own device memory. */
recon_status recon_unet_create(int c1, int bf16_storage, void* stream, recon_unet** out);
recon_status recon_unet_set_params(recon_unet* u, const float* host, size_t count);
recon_status recon_unet_get_params(recon_unet* u, float* host, size_t count);
/* Gradients of the last recon_unet_backward, same layout as the parameters (host copy). */
recon_status recon_unet_get_grads(recon_unet* u, float* host, size_t count);
/* y (device, n^3 float32) = network(x) for x (device, n^3 x 5); n a multiple of 8.  With bfloat16
 * storage, the convolutions of every level whose side is 64 or a multiple of 128 run on the tensor
 * cores (tcgen05.mma, float32 accumulation in tensor memory); the others on the CUDA cores.  Both
 * round every stored activation to bfloat16 at the same points, so they differ only in the order
 * of the float32 sums.  Returns ERR_CUDA if a tensor-core wait timed out. */
recon_status recon_unet_forward(recon_unet* u, const float* x, int n, float* y);
/* Forward, mean squared error against target (device, n^3) and all parameter gradients; *loss
 * (host) receives the loss when not NULL. */
recon_status recon_unet_backward(recon_unet* u, const float* x, const float* target, int n, double* loss);
/* One AdamW step (beta 0.9 / 0.999, decoupled weight decay wd on the weights, not the biases). */
recon_status recon_unet_adamw(recon_unet* u, float lr, float wd);
/* Options: RECON_UNET_OPT_TENSOR_CORES (1 default, 0 = every convolution on the CUDA cores). */
enum { RECON_UNET_OPT_TENSOR_CORES = 0 };
recon_status recon_unet_set_option(recon_unet* u, int option, int value);
/* Output of convolution layer `layer` (0..9, in the parameter order) from the last forward, as
 * float32 on the host (count = side^3 x cout of that layer's level).  STATE if that activation was
 * not stored (the last layer when its 1x1 head was fused into it). */
recon_status recon_unet_get_layer(recon_unet* u, int layer, float* host, size_t count);
/* Number of kernels the tensor-core forward path of recon_unet_forward has launched so far. */
recon_status recon_unet_launch_count(recon_unet* u, long long* count);
recon_status recon_unet_destroy(recon_unet* u);
const char* recon_unet_last_error(recon_unet* u);

/* Release the handle and, if it allocated them, its device buffers. NULL is accepted. */
recon_status recon_destroy(recon_handle* h);

/* Static description of a status code. */
const char* recon_status_str(recon_status s);

/* Last CUDA error text recorded on the handle (empty string if none). */
const char* recon_last_error(recon_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* RECON_GB300_H */
