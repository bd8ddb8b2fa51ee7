/*
 * fdfd.h -- C-ABI of the GB300 (sm_103a) two-level Schwarz neural-operator
 * FGMRES solver for the 2D frequency-domain Maxwell (Ez) FDFD operator of
 * arXiv 2509.03622 ("Accurate and scalable deep Maxwell solvers using
 * multilevel iterative methods").
 *
 * Problem statement (Eq. 1 with the UPML of Methods, Eq. 3-6):
 *     lap E + k0^2 eps E = j w mu0 J   (time dependence e^{+j w t}),
 * on an nx x ny grid of square cells dx, stretched-coordinate PML of npml
 * cells per side (m = 3, R = e^-30 by default), E = 0 outside the grid.
 * The library solves the dx^2-scaled system  A~ E = b~ = dx^2 j w mu0 J.
 *
 * Conventions for every entry point:
 *   - grid arrays are row-major [ny][nx] (x fastest); complex values are
 *     interleaved (re, im) float32 pairs (fdfd_c64);
 *   - "device pointer" = memory the calling process allocated on the
 *     handle's GPU (e.g. a torch tensor's data_ptr); the caller owns it and
 *     keeps it alive until the call returns (all calls below synchronise
 *     the handle's stream before returning unless stated otherwise);
 *   - the library owns the handle and all its workspace, allocated in
 *     fdfd_create / schwarz_setup and freed in fdfd_destroy; no solve
 *     allocates device memory;
 *   - return value 0 = FDFD_OK; > 0 = soft outcome with valid stats;
 *     < 0 = hard error (nothing written to the outputs is meaningful).
 *     No C++ exception crosses this boundary.
 *   - windows: the grid is tiled by 64 x 64 cores; window w (row-major over
 *     cores, nwx = nx/64 per row) is the 80 x 80 block around core w (8 cells
 *     of overlap per side), shifted inward at the grid edge.  nx and ny must
 *     be multiples of 64 and at least 128.
 */
#ifndef FDFD_H
#define FDFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define FDFD_OK             0
#define FDFD_NOT_CONVERGED  1   /* max_iters reached; stats valid            */
#define FDFD_STAGNATED      2   /* 3 restart cycles in a row lowered the true
                                   residual by less than 1%; stats valid      */
#define FDFD_EINVAL        -1   /* bad argument (checked on the host)        */
#define FDFD_ECUDA         -2   /* a CUDA call failed                        */
#define FDFD_ENUMERIC      -3   /* NaN / Inf met in the iteration            */
#define FDFD_ETIMEOUT      -4   /* a bounded device wait ran out; the handle's
                                   neural operator then skips its work in
                                   every later call (recreate the handle)    */
#define FDFD_ENOSETUP      -5   /* schwarz_setup required first              */
#define FDFD_ENOMEM        -6   /* workspace allocation failed               */

/* ---- preconditioners ------------------------------------------------- */
#define FDFD_PRECOND_NONE     0
#define FDFD_PRECOND_JACOBI   1  /* z = D^-1 v, D = diag(A~)                  */
#define FDFD_PRECOND_SCHWARZ  2  /* one two-level Schwarz sweep (Algorithm 3)
                                    with neural local solves (Fig. 2)        */

#define FDFD_PREC_BF16 0
#define FDFD_PREC_FP8  1

typedef struct fdfd_ctx* fdfd_handle;
typedef struct { float re, im; } fdfd_c64;

/* Problem description (Eq. 1; UPML of Methods). */
typedef struct {
  int    nx, ny;        /* grid cells, multiples of 64, >= 128            */
  double dx;            /* cell size in metres                             */
  double wavelength;    /* vacuum wavelength in metres                     */
  int    npml[4];       /* PML cells on the x-, x+, y-, y+ sides           */
  double pml_m;         /* grading exponent m (3 in the paper)             */
  double pml_lnR;       /* ln of the ideal reflectivity (-30)              */
  const float* eps;     /* device ptr [ny][nx] relative permittivity; the
                           library copies it                               */
  void*  stream;        /* cudaStream_t used for all work (NULL = legacy)  */
  int    max_restart;   /* longest FGMRES restart the handle allocates its
                           Krylov space for (V: max_restart + 1 vectors, Z:
                           max_restart): 0 = 32, else 1..64              */
} fdfd_desc;

/* Two-level Schwarz set-up (Sec. 2.2, Methods, Algorithm 3 set-up). */
typedef struct {
  int k_coarse;          /* coarse basis vectors per window; 0 = one-level */
  int precision;         /* FDFD_PREC_BF16: BF16 activations and weights,
                            FP32 accumulation.  FDFD_PREC_FP8: the
                            activation entering each Fourier block and the
                            projection is stored as E4M3 with power-of-two
                            per-channel scales (calibrated at set-up on a
                            seeded random residual and seeded random Robin
                            data, 4x headroom below the E4M3 maximum,
                            saturating), converted to BF16 in
                            shared memory for the tensor cores, the scales
                            folded into the weights that read it; halves
                            the activation traffic (precision pattern).    */
  const float* weights;  /* HOST ptr to the FNO weight blob, float32, in the
                            order: lift_w[32][15], lift_b[32], then per block
                            b = 0..3: R_re[32][32][32][16], R_im[...],
                            W[32][32], bias[32]; then p1_w[128][32], p1_b[128],
                            p2_w[2][128], p2_b[2].  R is indexed
                            [out][in][ky][kx] with ky rows 0..15 = modes
                            0..15 and rows 16..31 = modes -16..-1.          */
  size_t n_weights;      /* number of floats in the blob (4,203,522 for the
                            plain network; see r_rank and modulation)      */
  int inner_iters;       /* local solver of each window (Algorithm 3's
                            M.solve): 0 = one neural-operator application
                            with the residual and Robin data as inputs;
                            m in 1..16 = m steps of NN-preconditioned FGMRES
                            (Algorithm 1) on the window's Robin problem     */
  double ritz_tol;       /* Rayleigh-Ritz truncation of the coarse space
                            (Algorithm 3 set-up, eta, u = eig(H); Sec. 2.2):
                            0 = keep the k orthonormalised trials (span
                            unchanged by the eig step); > 0 = per window,
                            the eigenpairs of H = Q^H Y, Y the Robin data
                            each basis field hands to the neighbours (read
                            on their sides facing the window), and only the
                            Ritz vectors with |eta| >= ritz_tol kept; the
                            basis fields are combined, not solved again.
                            Needs k_coarse <= 64.                           */
  int r_rank;            /* modified FNO (Sec. 2.1): 0 = each block's R is
                            stored in full; r in 1..512 = the blob gives R
                            as rank-r factors theta [32][32][r] and V
                            [r][32][16] (re then im of each, in place of
                            R_re, R_im), R = sum_r theta V, expanded at
                            set-up                                          */
  int modulation;        /* modified FNO (Sec. 2.1, Fig. 2): 1 = the blob
                            ends with the modulation path, conv_w
                            [16][5][3][3] (inputs (k0 dx)^2 eps, Re/Im 1/s_x,
                            Re/Im 1/s_y), conv_b [16], fc_w [2048][144],
                            fc_b [2048]; the real modulation m [4][32][16] of
                            each window (3x3 stride-2 valid convolution,
                            leaky-ReLU, 13x13 average pooling, fully
                            connected) is computed at set-up and block b
                            uses R (1 + m[b]).  Neither option combines
                            with FDFD_PREC_FP8 (FDFD_EINVAL).               */
} schwarz_desc;

typedef struct {
  int    restart;        /* FGMRES restart length, 1..fdfd_desc.max_restart */
  int    max_iters;      /* total inner iterations                        */
  double tol;            /* true relative residual ||b~ - A~ E||/||b~||   */
  int    precond;        /* FDFD_PRECOND_*                                 */
  int    use_x0;         /* 1: start from the contents of E               */
  int    use_graphs;     /* 1: replay each Arnoldi step (preconditioner,
                            matvec, orthogonalisation) as a CUDA graph,
                            captured once per handle, restart length,
                            preconditioner and direction; results are
                            identical to eager launches.  Ignored while
                            live profiling is on (fdfd_profile_start). */
} fdfd_solve_opts;

typedef struct {
  int    iters;          /* inner (Arnoldi) iterations done               */
  int    restarts;       /* cycles completed                              */
  int    status;         /* same as the return value                      */
  double relres_true;    /* FP64 ||b~ - A~ E|| / ||b~|| of the result      */
  double relres_est;     /* last least-squares estimate                   */
  double t_solve_ms;     /* device time of the solve (CUDA events)        */
} fdfd_solve_stats;

typedef struct {
  int n_win, nwx, nwy;   /* windows and their layout                      */
  int k_coarse;          /* 0 if no coarse space set up                   */
  int n_coarse;          /* n_win * k_coarse                               */
  size_t workspace_bytes;/* device memory held by the handle              */
  int graphs_cached;     /* Arnoldi-step graph sets currently captured     */
  int graphs_ok;         /* 0 once a capture failed (eager launches only)  */
  int tuned_dfty_split;  /* autotuned at set-up: DFT-y GEMM variant, 0 =
                            operand tiles by TMA, 1 or 2 = gather with that
                            K split; the environment variable
                            FDFD_DFTY_VARIANT=0|1|2 fixes it instead      */
  int n_coarse_kept;     /* coarse unknowns kept (trials not dropped as
                            dependent, Ritz vectors above ritz_tol)        */
} fdfd_info;

/* ---- handle life cycle ----------------------------------------------- */

/* Create a solver for the problem of Eq. 1 described by *desc: computes the
 * UPML stretching (Methods, Eq. 6) and the 5-point coefficients, copies eps,
 * allocates the Krylov workspace for restarts up to desc.max_restart.  FDFD_EINVAL for bad
 * sizes (nx, ny not multiples of 64 or < 128, npml < 0 or >= n/2, dx or
 * wavelength <= 0).  *out is NULL on error. */
int  fdfd_create(const fdfd_desc* desc, fdfd_handle* out);

/* Replace the permittivity map (device ptr [ny][nx], copied).  Invalidates
 * any coarse space (schwarz_setup must be called again). */
int  fdfd_set_eps(fdfd_handle h, const float* eps_dev);

/* Set up the neural local solver and, if k_coarse > 0, the coarse space of
 * Algorithm 3: pseudo-plane-wave Robin trials, Gram-Schmidt (FP64), the
 * homogeneous neural solves, their traces on the neighbours (B Q), the
 * Galerkin coarse matrix G = Q^H (BQ - Q) (FP64 blocks; the reading of
 * Eq. 7-8 as the Rayleigh-Ritz projection of the interface operator), and
 * its factorisation by block elimination over the window rows (each row's
 * Schur complement inverted in FP32 by LU with partial pivoting; storage
 * (ny/64) (nx/64 k)^2 complex64).  Weights are copied.  FDFD_ENUMERIC if a
 * Schur complement is singular, FDFD_ENOMEM if the factors do not fit. */
int  schwarz_setup(fdfd_handle h, const schwarz_desc* sd);

void fdfd_destroy(fdfd_handle h);
const char* fdfd_status_string(int code);
int  fdfd_get_info(fdfd_handle h, fdfd_info* info);

/* ---- the solve (Algorithm 1 with restarts; Sec. 2.2) ------------------ */

/* Solve A~ E = dx^2 j w mu0 J with flexible GMRES(restart).  J_dev: device
 * [ny][nx] current density (A/m^2); E_dev: device [ny][nx] output (and
 * initial guess if use_x0).  Vectors are complex64; dots, norms and the
 * Hessenberg least squares are FP64; the solution is accumulated in FP64
 * and every restart recomputes the true residual in FP64 (iterative
 * refinement).  Returns FDFD_OK when relres_true <= tol. */
int  fdfd_solve(fdfd_handle h, const fdfd_c64* J_dev, fdfd_c64* E_dev,
                const fdfd_solve_opts* opts, fdfd_solve_stats* stats);

/* As fdfd_solve with HOST buffers: J_host and E_host are host memory; the
 * host<->device copies are part of the call. */
int  fdfd_solve_host(fdfd_handle h, const fdfd_c64* J_host, fdfd_c64* E_host,
                     const fdfd_solve_opts* opts, fdfd_solve_stats* stats);

/* ---- batching pattern (several problems in lock step; Fig. 1a) -------- */
typedef struct fdfd_batch_ctx* fdfd_batch;

/* Group n handles (any grid sizes, wavelengths, permittivities; all on the
 * same stream) for lock-step solves.  max_windows caps the windows of one
 * neural-operator pass (0 = min(total windows, 8192)); the batch allocates
 * that workspace here (about 0.9 MB per window).  The handles must outlive
 * the batch.  FDFD_EINVAL if streams differ. */
int  fdfd_batch_create(fdfd_handle* hs, int n, int max_windows, fdfd_batch* out);

/* FGMRES solves of all problems of the batch in lock step: J_dev[p], E_dev[p]
 * are device pointers of problem p (host arrays of n pointers); stats[p]
 * receives each problem's statistics (t_solve_ms is the batch's time).  With
 * FDFD_PRECOND_SCHWARZ every Arnoldi step applies the neural local solves of
 * all windows of all active problems whose local solver is one network
 * application (inner_iters = 0) as one batch (one launch per operator stage
 * per chunk), using hs[0]'s weights (those handles must have been set up
 * with the same blob); a problem set up with inner_iters > 0 applies its
 * own preconditioner (its windows' NN-FGMRES) in the same lock-step
 * iteration.  Coarse corrections are applied per problem.  Returns the most
 * severe status over the problems. */
int  fdfd_solve_batched(fdfd_batch b, const fdfd_c64* const* J_dev, fdfd_c64* const* E_dev,
                        const fdfd_solve_opts* opts, fdfd_solve_stats* stats);
void fdfd_batch_destroy(fdfd_batch b);

/* Adjoint solve A~^T lam = g (Sec. 2.2, adjoint variable method): g_dev is
 * the device [ny][nx] right-hand side taken as is (no source scaling), the
 * same preconditioners applied to the transposed operator. */
int  fdfd_solve_adjoint(fdfd_handle h, const fdfd_c64* g_dev, fdfd_c64* lam_dev,
                        const fdfd_solve_opts* opts, fdfd_solve_stats* stats);

/* dF/deps = -2 Re( lam * (k0 dx)^2 * E ) per cell (adjoint variable method,
 * with A~ lam-adjoint  A~^T lam = dF/dE).  grad_dev: device float [ny][nx];
 * accumulate = 1 adds to its contents (sum over wavelengths). */
int  fdfd_grad_eps(fdfd_handle h, const fdfd_c64* E_dev, const fdfd_c64* lam_dev,
                   float* grad_dev, int accumulate);

/* ---- live profiling (CUDA events on the handle's stream) -------------- */
#define FDFD_PROF_NCLASS 18
/* kernel classes: 0 stencil A~x (incl. the fused Jacobi form), 1 CGS dots,
 * 2 CGS update + Givens, 3 FP64 residual, 4 solution update / misc vector,
 * 5 neural-operator pack (restriction + inputs), 6 traces, 7 coarse solve
 * and correction, 8 lift GEMM, 9 DFT-x GEMM, 10 DFT-y GEMM, 11 spectral
 * mix GEMM, 12 inverse DFT-y GEMM, 13 fused inverse DFT-x + mixer +
 * activation (+ the next block's DFT-x), 14 projection + prolongation,
 * 15 local Robin operator and Krylov update of the inner NN-FGMRES,
 * 16 FP64 right-hand-side norm (residual of x = 0), 17 unused. */
typedef struct {
  double ms[FDFD_PROF_NCLASS];        /* summed device time per class      */
  long long launches[FDFD_PROF_NCLASS];/* kernel launches per class        */
  long long total_launches;            /* all kernels the handle launched   */
} fdfd_profile;

/* Start recording: from now on every kernel class launched by this handle
 * is bracketed by CUDA events (pool of 16384 pairs; later launches are
 * counted but not timed).  Returns FDFD_EINVAL if already recording. */
int  fdfd_profile_start(fdfd_handle h);
/* Stop, synchronise and report the per-class times and launch counts. */
int  fdfd_profile_stop(fdfd_handle h, fdfd_profile* out);

/* ---- single steps of the hot path (device pointers; parity tests) ---- */

/* y = A~ x (transpose = 0) or y = A~^T x (transpose = 1), complex64; the
 * 5-point stencil of Eq. 1 with UPML (one step of the solve). */
int  fdfd_apply_A(fdfd_handle h, const fdfd_c64* x, fdfd_c64* y, int transpose);

/* z = M(v): one two-level Schwarz sweep from a zero guess -- restriction,
 * neural local solves, restricted prolongation, trace mismatch, coarse
 * solve and correction (Algorithm 3; Sec. 2.2).  Requires schwarz_setup. */
int  fdfd_precond_apply(fdfd_handle h, const fdfd_c64* v, fdfd_c64* z);

/* Algorithm 3 as a solver: the stationary (two-level) Schwarz iteration for
 * A~ u = b (b the right-hand side of the dx^2-scaled system of Eq. 1, device
 * complex64 [ny][nx]; u device complex64 [ny][nx], output only).  Each
 * iteration solves every window's local Robin problem with the restricted
 * source and the current Robin data g (the neural operator, or k inner
 * NN-FGMRES steps when schwarz_setup asked for them), assembles u by
 * restricted prolongation, takes the traces of u (Eq. 2), with a coarse space
 * corrects u for the mismatch between those traces and g (Eq. 8) and takes
 * them again, and blends g = momentum g + (1 - momentum) traces.  It stops
 * after max_iters iterations or once the FP64 relative residual
 * ||b - A~ u|| / ||b|| is <= tol.  g starts at zero, so the first iterate is
 * fdfd_precond_apply(b).  Writes the iterations done and the last relative
 * residual (may be NULL).  FDFD_EINVAL for max_iters < 1, tol < 0 or momentum
 * outside [0, 1); FDFD_ENOSETUP without schwarz_setup; FDFD_ENUMERIC if the
 * residual is not finite (u then holds the last iterate); FDFD_ETIMEOUT as
 * for the solve.  Uses the handle's Krylov workspace; synchronous. */
int  fdfd_schwarz_stationary(fdfd_handle h, const fdfd_c64* b_dev, fdfd_c64* u_dev, int max_iters,
                             double tol, double momentum, int* iters, double* relres);

/* Batched neural local solves (Fig. 2) on n windows: r_win [n][80][80]
 * window residuals, g_win [n][4][80] Robin data (sides x-, x+, y-, y+;
 * Eq. 2), win_id [n] (device int) the window whose eps / PML the solve
 * uses; writes e_win [n][80][80].  Requires schwarz_setup. */
int  fdfd_nno_solve(fdfd_handle h, const fdfd_c64* r_win, const fdfd_c64* g_win,
                    const int* win_id, int n, fdfd_c64* e_win);

/* fdfd_nno_solve for callers that cannot allocate device memory (the paper
 * has no counterpart: this is an interface convenience).  Such callers are,
 * for example, code that must stay within a device-memory budget that its
 * own pool allocator hands out (a cudaMalloc would take memory promised to
 * others), or a latency-bound loop that cannot pay for the device-wide
 * synchronisation an allocation or free may cause.  Same arguments and
 * results as fdfd_nno_solve (the same kernels, bit for bit), but the neural
 * operator's intermediates live in one fixed device array inside the
 * library (about 3.5 MB, held by every GPU that loads the library until the
 * process exits) instead of the handle's workspace, and the call allocates
 * nothing.
 *   - n must be <= 4 windows; larger n returns FDFD_EINVAL (with a message on
 *     stderr) and does nothing.
 *   - The first call on a device (and the first after that device's context
 *     was replaced, e.g. by cudaDeviceReset) looks the array's device address
 *     up; later calls reuse it.
 *   - All calls share the one array, which keeps the last call's contents:
 *     calls that overlap on the GPU (from several streams, threads or
 *     handles) race and corrupt each other's results.  Serialise them.
 *   - Requires schwarz_setup on h (FDFD_ENOSETUP otherwise).  Returns
 *     FDFD_ETIMEOUT without launching anything once a neural pass of h has
 *     given up on a bounded wait (as fdfd_nno_solve does).
 *   - Synchronous: it reads the kernels' error flag back and waits for the
 *     handle's stream. */
int  fdfd_nno_solve_noalloc(fdfd_handle h, const fdfd_c64* r_win, const fdfd_c64* g_win,
                            const int* win_id, int n, fdfd_c64* e_win);

/* Local Robin operator (Eq. 1 restricted to a window, Eq. 2 on its interface
 * sides with zero Robin data, zero ghosts on grid-edge sides): y = A_w x for
 * n windows; x, y device [n][80][80], win_id device int [n].  Does not need
 * schwarz_setup. */
int  fdfd_local_apply(fdfd_handle h, const fdfd_c64* x_win, fdfd_c64* y_win, const int* win_id, int n);

/* Robin traces g = u_o - u_b + j (k0 dx) sqrt(eps_b) u_b (Eq. 2, dx-scaled)
 * of a global field on every window's interface sides: g [n_win][4][80],
 * zero on grid-edge sides. */
int  fdfd_trace_extract(fdfd_handle h, const fdfd_c64* u, fdfd_c64* g);

/* Copy the coarse set-up out for inspection (host pointers, may be NULL):
 * Q [n_win][k][4][80] complex128 (interleaved doubles) orthonormalised trials
 * (rotated by the kept Ritz vectors after a Ritz step); the Galerkin blocks
 * G [n_win][9][k][k] complex128, G[i][j][p][q] = sum over window i's slots of
 * conj(Q_i[p]) times the mismatch that basis vector q of window
 * J = i + (j % 3 - 1, j / 3 - 1) leaves there (its field's traces minus, for
 * J = i, its own data), zero where J lies outside the grid; a dropped unknown
 * (zero trial vector) has a unit diagonal. */
int  fdfd_coarse_export(fdfd_handle h, double* Q_host, double* G_host);

/* The coarse solve alone (reading of Eq. 7 with the Rayleigh-Ritz step of
 * Algorithm 3): for a boundary mismatch e_bc (device [n_win][4][80]
 * complex64) returns z (device [n_win][k] complex64) with
 * G z = -Q^H e_bc, by the block elimination over window rows that the
 * preconditioner uses (FP32).  Synchronous.  FDFD_ENOSETUP without a coarse
 * space. */
int  fdfd_coarse_solve(fdfd_handle h, const fdfd_c64* ebc_dev, fdfd_c64* z_dev);

/* Rayleigh-Ritz data of the coarse set-up (schwarz_desc.ritz_tol > 0), host
 * pointers, each may be NULL: eta_host [n_win][k] Ritz values and H_host
 * [n_win][k][k] row-major Ritz matrices H[p][q] = (q_p, y_q), complex128
 * (interleaved doubles); the values per window in the order the eigen
 * solver returns them.  FDFD_ENOSETUP without a Ritz step. */
int  fdfd_coarse_ritz(fdfd_handle h, double* eta_host, double* H_host);

/* ---- inverse design (Sec. 2.2: density-based optimisation with filtering,
 * projection and Adam, gradients from fdfd_solve_adjoint + fdfd_grad_eps) -- */

/* Design rectangle and its parameterisation: rho in [0, 1] on h x w cells at
 * (x0, y0) of the grid; rho_f = cone filter of rho (weights max(0, R - |d|)
 * over the offsets inside the rectangle, each output divided by its own
 * weight sum); eps = eps_lo + P(rho_f) (eps_hi - eps_lo) with
 * P(x) = (tanh(beta eta) + tanh(beta (x - eta))) /
 *        (tanh(beta eta) + tanh(beta (1 - eta))). */
typedef struct {
  int   x0, y0, w, h;    /* rectangle in cells, inside the grid            */
  float radius;          /* filter radius in cells, 0 < radius <= 16       */
  float beta, eta;       /* projection sharpness (> 0), threshold (0, 1)   */
  float eps_lo, eps_hi;  /* permittivity at rho = 0 and rho = 1            */
} fdfd_design;

/* Adam (Kingma and Ba) with bias correction, as an ascent. */
typedef struct {
  float lr, beta1, beta2, eps;  /* step, moment decays in [0, 1), eps > 0   */
} fdfd_adam;

/* rho [h][w] -> rho_f [h][w] (kept for fdfd_design_grad) and the design
 * rectangle of eps [ny][nx] (the rest of eps untouched); device float32
 * pointers; h supplies the grid and the stream.  Synchronous; FDFD_EINVAL
 * for a rectangle outside the grid or parameters out of range. */
int  fdfd_design_eps(fdfd_handle h, const fdfd_design* d, const float* rho, float* rho_f, float* eps);

/* Chain rule from dF/deps (g_eps [ny][nx], e.g. from fdfd_grad_eps, summed
 * over wavelengths) to dF/drho: g_rho = W^T (P'(rho_f) (eps_hi - eps_lo)
 * g_eps) on the rectangle; work [h][w] is scratch.  Device float32. */
int  fdfd_design_grad(fdfd_handle h, const fdfd_design* d, const float* rho_f, const float* g_eps, float* work,
                      float* g_rho);

/* One Adam ascent step (t = 1, 2, ... counts the steps) on theta [n] with the
 * gradient g [n] times g_scale (e.g. 1 / F at the start, so that the
 * gradient is well above eps), moments m, v [n] (zero before the first
 * step); theta is clipped to [0, 1].  Device float32; synchronous. */
int  fdfd_adam_step(fdfd_handle h, const fdfd_adam* a, int t, float g_scale, float* theta, const float* g,
                    float* m, float* v, int n);

/* ---- figure of merit: port mode overlaps (Sec. 2.2, the inverse design's
 * objective and the source of its adjoint solve) ---------------------------
 * The overlap of a field with a port profile m on the vertical line
 * x = port_x is c = dx sum_{i < nm} conj(m_i) E[y0 + i][port_x]; it is linear
 * in E with dc/dE = conj(m_i) dx on the line.  Gradients of a real loss L
 * follow the conjugate-Wirtinger convention G_z = 2 dL/d conj(z) (what
 * PyTorch's autograd passes; for L = |c|^2, G_c = 2 c). */

/* c_dev [2] (device doubles, re / im, overwritten) = the overlap, summed in
 * FP64.  E [ny][nx] and mode [nm] device complex64.  Asynchronous on
 * `stream` (a cudaStream_t; NULL = the legacy default stream).  FDFD_EINVAL
 * unless nx, ny, nm >= 1, 0 <= port_x < nx, y0 >= 0, y0 + nm <= ny and
 * dx > 0. */
int  fdfd_mode_overlap(const fdfd_c64* E, int nx, int ny, const fdfd_c64* mode, int nm, int port_x, int y0,
                       double dx, double* c_dev, void* stream);

/* The overlap's chain rule: with G_c = gc_re + j gc_im (host values),
 * G_E = G_c conj(dc/dE) = G_c m_i dx on the port line.  grad_E [ny][nx]
 * (device complex64) is overwritten with it, zero elsewhere (accumulate = 0),
 * or has it added (accumulate = 1).  Asynchronous on `stream`; arguments as
 * fdfd_mode_overlap. */
int  fdfd_mode_overlap_grad(int nx, int ny, const fdfd_c64* mode, int nm, int port_x, int y0, double dx,
                            double gc_re, double gc_im, fdfd_c64* grad_E, int accumulate, void* stream);

/* Right-hand side of the adjoint system A~^T lam = dL/dE (Sec. 2.2, adjoint
 * variable method) from a field gradient G_E = 2 dL/d conj(E) of a real
 * loss: g = dL/dE = conj(G_E) / 2, over the handle's grid ([ny][nx] device
 * complex64; g may alias grad_E).  On the handle's stream. */
int  fdfd_adjoint_rhs(fdfd_handle h, const fdfd_c64* grad_E, fdfd_c64* g);

/* Diagnostic: one tile GEMM on the tcgen05 path used by the neural operator
 * (no counterpart in the paper; validates the tensor-core operand encoding).
 * C[M][N] (float32, device) = A . B^T with A bf16 [M][K] (a_mn_major = 0)
 * or [K][M] (a_mn_major = 1), B bf16 [N][K]; M a multiple of 8; (N, K) one
 * of (32,80) (64,160) (64,64) (160,64) (32,16) (128,32).  Synchronous;
 * FDFD_ETIMEOUT if the tensor-core completion wait ran out. */
int  fdfd_selftest_gemm(const void* A, const void* B, float* C, int M, int N, int K, int a_mn_major);

/* Diagnostic of failure detection (no counterpart in the paper): one kernel
 * waits, with the same bound as every pipeline wait (2^22 polls or about one
 * second of device time), on a barrier nothing arrives on.  Returns
 * FDFD_ETIMEOUT when the wait gave up as it must (the expected result; the
 * CUDA context stays usable), FDFD_OK if it completed, FDFD_ECUDA on a CUDA
 * error.  Synchronous on the legacy stream. */
int  fdfd_selftest_wait(void);

/* Failure injection from the host (no counterpart in the paper): mark the
 * handle's neural operator as failed, exactly as a bounded device wait that
 * ran out does.  Every later neural pass of the handle then skips its work
 * and fdfd_solve with FDFD_PRECOND_SCHWARZ returns FDFD_ETIMEOUT at its next
 * restart.  FDFD_ENOSETUP before schwarz_setup. */
int  fdfd_nno_mark_failed(fdfd_handle h);

#ifdef __cplusplus
}
#endif
#endif /* FDFD_H */
