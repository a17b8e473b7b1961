/*
 * lbm.h -- C ABI of the GB300 Shan-Chen droplet/bubble library (liblbm.so).
 *
 * Method: "A Mesoscale Perspective on the Tolman Length" (arXiv:2105.08772).
 *   Sec. II   D3Q19 BGK + Guo-forcing lattice Boltzmann step with the
 *             Shan-Chen pseudopotential force, Eqs. (3)-(8), and the lattice
 *             pressure tensor, Eq. (9).
 *   Sec. III  generalised surface tension sigma[R], Eqs. (21)-(22), surface of
 *             tension R_s, Laplace law Eq. (12), Tolman expansion Eq. (2).
 *   Sec. IV   droplet/bubble set-up (Eq. (23)), P_in/P_out sampling, centre-of-
 *             mass acceptance, the two convergence criteria, equimolar radius.
 *
 * Conventions shared by every entry point
 *   - Device memory: the caller allocates and owns all device memory (the
 *     "workspace") and the CUDA stream; the library only borrows them and
 *     never calls cudaMalloc/cudaFree.  Size the workspace with
 *     lbm_workspace_bytes / lbm_batch_workspace_bytes; it must be 256-byte
 *     aligned and stay valid until the context is destroyed.
 *   - Streams: every device operation is enqueued on the context's stream
 *     (a cudaStream_t passed as void*; NULL = legacy default stream).  Calls
 *     documented "async" return before the GPU work finishes; calls that
 *     return host data synchronise that stream first.
 *   - Host buffers: plain C arrays owned by the caller; the library never
 *     keeps a pointer to them after the call returns.
 *   - Errors: every call returns an lbm_status and never aborts, traps or
 *     exits.  On failure lbm_last_error(ctx) holds a one-line message.  A CUDA
 *     error is reported as LBM_ECUDA.  Arguments are checked before any work is
 *     enqueued (LBM_EINVAL).
 *   - Field layout: a scalar field of a box (nx, ny, nz) is a contiguous
 *     double array indexed (z*ny + y)*nx + x.  Populations are 19 such planes,
 *     population i at offset i*nx*ny*nz, in this velocity order:
 *        0:( 0, 0, 0)
 *        1:(+1, 0, 0)  2:(-1, 0, 0)  3:( 0,+1, 0)  4:( 0,-1, 0)
 *        5:( 0, 0,+1)  6:( 0, 0,-1)
 *        7:(+1,+1, 0)  8:(-1,-1, 0)  9:(+1,-1, 0) 10:(-1,+1, 0)
 *       11:(+1, 0,+1) 12:(-1, 0,-1) 13:(+1, 0,-1) 14:(-1, 0,+1)
 *       15:( 0,+1,+1) 16:( 0,-1,-1) 17:( 0,+1,-1) 18:( 0,-1,+1)
 *     The box is periodic in all three axes.
 *   - The centre node is c = (nx/2, ny/2, nz/2) (integer division), the
 *     "farthest corner" is ((c_a + n_a/2) mod n_a) per axis (for odd sizes
 *     this is (n-1, n-1, n-1), the node Sec. IV names).
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,      /* bad argument (sizes, tau <= 1/2, G >= G_c, null pointer, ...) */
    LBM_ENOMEM = 2,      /* the caller's workspace is too small */
    LBM_ECUDA = 3,       /* a CUDA runtime call failed */
    LBM_ENUMERIC = 4,    /* NaN/Inf or a non-positive density found in the field */
    LBM_ENOTCONV = 5,    /* max_steps reached before either convergence test passed */
    LBM_ENOMIN = 6,      /* result status: sigma[R] has no minimum (C / Delta P <= 0) */
    LBM_ECOLLAPSE = 7,   /* result status: |n_in - n_out| below 1e-2 of the initial contrast */
    LBM_EOFFCENTER = 8,  /* result status: a centre-of-mass coordinate is > 1e-3 off centre */
    LBM_ETIMEOUT = 9     /* a bounded device-side wait ran out (status bit 4) */
} lbm_status;

/* psi(n) kinds (Sec. II below Eq. (8); Sec. IV names the first two). */
typedef enum {
    LBM_PSI_EXP_INV = 0,        /* psi = exp(-1/n)                                   */
    LBM_PSI_ONE_MINUS_EXP = 1,  /* psi = 1 - exp(-n)                                 */
    LBM_PSI_CS = 2              /* psi = sqrt(2 (p_CS(n) - n c_s^2) / (G c_s^2)),
                                   Carnahan-Starling p_CS with a, b, Rgas, T below    */
} lbm_psi_kind;

typedef struct {
    int kind;                   /* lbm_psi_kind */
    double a, b, Rgas, T;       /* Carnahan-Starling constants; ignored unless kind == LBM_PSI_CS */
} lbm_eos;

/* Isotropic forcing stencils for Eq. (8): E4 is the paper's 18-vector
 * D3Q19 stencil with W(1) = 1/6, W(2) = 1/12; E6 (32 vectors, shells
 * |xi|^2 = 1..4) and E8 (92 vectors, shells 1,2,3,4,5,6,8) are the
 * higher-order isotropic stencils the paper cites for the force. */
typedef enum { LBM_E4 = 4, LBM_E6 = 6, LBM_E8 = 8 } lbm_stencil;

/* Population storage.  F64: plain doubles, FP64 arithmetic.  F32_SHIFTED:
 * f_i - w_i n0 stored as float, FP32 collision.  F16_SHIFTED: (f_i - w_i n0)
 * times a per-lattice power of two stored as IEEE half, FP32 collision.  All
 * observables and reductions are FP64 in every mode. */
typedef enum { LBM_F64 = 0, LBM_F32_SHIFTED = 1, LBM_F16_SHIFTED = 2 } lbm_prec;

typedef struct { int nx, ny, nz; } lbm_box;

/* Observables of one lattice (Sec. III, Sec. IV).  status_bits: bit 0 no
 * minimum of sigma[R], bit 1 collapsed, bit 2 off-centre, bit 3 non-finite
 * field, bit 4 a step kernel's bounded wait for its copies ran out since the
 * last initialisation (the field is then invalid; lbm_run_to_convergence
 * returns LBM_ETIMEOUT).  criterion: 0 none, 1 the Delta P test fired, 2 the
 * delta-u test. */
typedef struct {
    double n_in, n_out;         /* density at the centre node and the farthest corner       */
    double P_in, P_out, dP;     /* P^xx of Eq. (9) at those nodes; dP = P_in - P_out         */
    double mass;                /* M = sum_x n                                              */
    double com[3];              /* centre of mass of n - n_out (minimum image about c)       */
    double R_e;                 /* equimolar radius (Sec. IV, last paragraph)                 */
    double C, D;                /* int r^2 (P_out - P_T) dr and int r (P_out - P_T) dr        */
    double R_s;                 /* surface of tension (6 C / dP)^(1/3); NaN if no minimum      */
    double sigma_s;             /* sigma[R_s] = dP R_s / 2 (Eq. (12))                         */
    double max_u;               /* max_x |u_eq|                                               */
    double du;                  /* delta u since the previous observation (Sec. IV)           */
    double dP_rel_change;       /* |dP - dP_prev| / |dP_prev| since the previous observation  */
    long long steps;            /* time steps taken since the last initialisation             */
    unsigned status_bits;
    int criterion;
} lbm_obs;

/* ---------------------------------------------------------------- set-up */

/* Bytes of device workspace one lattice needs (two population buffers of
 * 19 planes, a velocity snapshot for delta u, reduction scratch).  Returns 0
 * for invalid arguments. */
size_t lbm_workspace_bytes(lbm_box box, int stencil, int prec);

/* Create a context for one periodic lattice (Sec. II).  tau: BGK relaxation
 * time of Eq. (4), > 1/2.  G: coupling of Eq. (8); for the two closed-form psi
 * kinds it must be below the critical coupling (-e^2 for exp(-1/n), -4 for
 * 1 - exp(-n); Sec. II below Eq. (10), Sec. IV), else LBM_EINVAL.  Box sides
 * must be >= 3 (E4) or >= 5 (E6/E8) and the box below 2^31 nodes (node offsets
 * within a population plane are 32-bit).  dev_workspace: caller-owned device
 * memory of at least lbm_workspace_bytes bytes, else LBM_ENOMEM.
 * cuda_stream: cudaStream_t used for all work.  *out receives a host-side
 * context (free it with lbm_destroy).  The field is uninitialised until one of
 * the lbm_init_* / lbm_set_populations calls. */
lbm_status lbm_create(lbm_box box, double tau, double G, lbm_eos eos, int stencil, int prec,
                      void* dev_workspace, size_t bytes, void* cuda_stream, lbm_ctx** out);

void lbm_destroy(lbm_ctx* ctx);

/* Initialise a droplet (rho_in > rho_out) or bubble (rho_in < rho_out), Sec. IV
 * Eq. (23): n(r) = (rho_in + rho_out)/2 - (rho_in - rho_out)/2 tanh((r - R)/width),
 * r the minimum-image distance to center[3] = (x, y, z) (host array of 3), fluid at
 * rest: f_i = f_i^eq(n, u = 0) (Eq. (6)).  width = 1 is the paper's profile.
 * For shifted storage the shift n0 is the mean density of a sharp sphere of
 * radius R.  Resets the step counter and the convergence history.  Async. */
lbm_status lbm_init_drop(lbm_ctx* ctx, const double center[3], double R,
                         double rho_in, double rho_out, double width);

/* Initialise from a host density field (nx*ny*nz doubles, layout above), fluid at
 * rest.  The field is copied to the device inside the call (the host buffer may be
 * reused on return).  For shifted storage the shift n0 is the field's mean.
 * LBM_EINVAL (nothing enqueued) for a null buffer or a density that is not
 * positive and finite. */
lbm_status lbm_init_rho(lbm_ctx* ctx, const double* host_rho);

/* Set / get the pre-collision populations f_i(x, t) of Eq. (3) from / to a host
 * buffer of 19*nx*ny*nz doubles (layout above).  set resets the step counter; for
 * shifted storage the shift n0 is the field's mean density; it takes any finite
 * values (LBM_EINVAL for a null buffer or a non-finite value), and a field the
 * step cannot carry (a non-positive or overflowing density) is reported as
 * LBM_ENUMERIC by the next convergence check.  get synchronises. */
lbm_status lbm_set_populations(lbm_ctx* ctx, const double* host_f);
lbm_status lbm_get_populations(lbm_ctx* ctx, double* host_f);

/* ---------------------------------------------------------------- time stepping */

/* Advance n >= 0 time steps of Eq. (3) (collision Eqs. (4)-(8), then streaming).
 * Async on the context stream; repeated calls replay a captured CUDA graph. */
lbm_status lbm_step(lbm_ctx* ctx, long long n);

/* Sec. IV convergence loop: every check_every steps (the paper uses 2^11) compare
 * Delta P and the velocity field with the previous check; stop when
 * |dP(t) - dP(t - check)| / |dP(t - check)| < tol_dP_rel (paper 1e-5) or
 * delta u < tol_du (paper 1e-12), or after max_steps (LBM_ENOTCONV).  A droplet
 * or bubble found collapsed (status bit 1) at two checks in a row ends the loop
 * with LBM_ECOLLAPSE (it cannot come back).  Writes the steps taken and the
 * criterion that fired (0/1/2) when the pointers are non-null.  Synchronises once
 * per check. */
lbm_status lbm_run_to_convergence(lbm_ctx* ctx, long long max_steps, long long check_every,
                                  double tol_dP_rel, double tol_du,
                                  long long* steps_done, int* criterion);

/* ---------------------------------------------------------------- observables */

/* Measure all observables of the current field (FP64 reductions on the device)
 * and copy them to *out.  du and dP_rel_change compare with the previous call
 * (or the previous convergence check); the first call after an init reports 0
 * and NaN.  Synchronises.  Returns LBM_OK even when status_bits are set; the
 * result statuses are in out->status_bits. */
lbm_status lbm_observables(lbm_ctx* ctx, lbm_obs* out);

/* Density n(c + r e_x) and tangential pressure P_T(r) = P^yy(c + r e_x) of
 * Eq. (9) along the +x half axis, r = 0..nx/2 (Sec. III below Eq. (22)).  len
 * must be nx/2 + 1.  Valid after lbm_observables.  Synchronises. */
lbm_status lbm_rho_profile(lbm_ctx* ctx, double* host_out, long long len);
lbm_status lbm_pt_profile(lbm_ctx* ctx, double* host_out, long long len);

/* Normal pressure P_N(r) = P^xx(c + r e_x) of Eq. (9) on the same half axis (used by
 * the flat interface's sigma_0, Eq. (25)).  len = nx/2 + 1.  Synchronises. */
lbm_status lbm_pn_profile(lbm_ctx* ctx, double* host_out, long long len);

/* Generalised surface tension sigma[R] (Eq. (21)) and its notional derivative
 * [dsigma/dR] (Eq. (22)) at m host radii R[k] > 0, from the last lbm_observables:
 * sigma = dP R/3 + C/R^2 and dsigma = dP/3 - 2C/R^3 + 2D/R^2 (the step P_J
 * integrated exactly, P_T by the trapezoid rule on the nodes).  Host arrays. */
lbm_status lbm_sigma_of_R(lbm_ctx* ctx, const double* R, double* sigma, double* dsigma,
                          long long m);

/* Copy the density field n(x) (nx*ny*nz doubles) / the Guo velocity u_eq of
 * Eq. (7) (3 planes of nx*ny*nz doubles: x, y, z components) to the host.
 * Synchronises. */
lbm_status lbm_copy_rho(lbm_ctx* ctx, double* host_out);
lbm_status lbm_copy_velocity(lbm_ctx* ctx, double* host_out);

/* Checkpoint: raw populations + step counter + shift/scale, to / from a file.  A
 * load requires the same box, precision and stencil.  Synchronises. */
lbm_status lbm_save(lbm_ctx* ctx, const char* path);
lbm_status lbm_load(lbm_ctx* ctx, const char* path);

/* Choose the step kernel's configuration for this context by timing every
 * compiled candidate for reps (rounded up to even) steps on the current field.
 * The field advances by those steps (the step counter counts them).  Optional;
 * lbm_create starts from a size-based default.  Synchronises.  *choice (may be
 * null) receives the chosen code (see lbm_set_tile). */
lbm_status lbm_autotune(lbm_ctx* ctx, int reps, long long* choice);

/* Select the step kernel's configuration by the code lbm_autotune reports:
 * kind * 10^8 + bx * 10^6 + by * 10^4 + (kind ? z chunk * 10 + prefetch depth : z chunk),
 * kind 0 the register-load kernel, 1 the cp.async-pipelined kernel, 4 the
 * pipelined kernel with 16-byte row chunks, 5 the unit-tau moment kernel (for
 * tau != 1 the same code runs kind 4), 6 the unit-tau moment kernel fed by element
 * copies (any nx; two CTAs per SM; for tau != 1 the same code runs kind 1), 7 the
 * unit-tau kernel staged by TMA tensor-tile copies (F32, E4, tau = 1, 32 x 8
 * tiles, nx % 4 == 0, nx >= 64, ny % 8 == 0, ny >= 16, nz >= 3; opt-in).  Kinds
 * 1, 4, 6 and 7: F32/F64 storage only, z chunk 0 = chosen by the launcher; 4
 * and 5 need nx % 4 == 0 and nx >= bx + 8; 6 is compiled
 * for 32 x 8 tiles with E4 (depth 1, and depth 2 in F32) and 32 x 4 with E6/E8
 * (depth 1).  Kind 5 also takes F16 storage (E4, 32 x 8 tiles, tau = 1,
 * nx % 8 == 0, nx >= 48).  The default (lbm_create) is kind 5 where it applies,
 * else kind 6, else kind 1 (kind 5 or 0 for F16).  A code that is not compiled
 * for this context's precision, stencil and box gives LBM_EINVAL.  lbm_get_tile
 * returns the current code.  In F32/F64 storage results do not depend on the
 * choice: all kinds do the same arithmetic per node and give bitwise-equal
 * fields.  In F16 storage kinds 5 and 0 sum in different orders, which FP16
 * rounding of the stored populations makes visible (same bound to the FP64
 * result). */
lbm_status lbm_set_tile(lbm_ctx* ctx, long long code);
lbm_status lbm_get_tile(const lbm_ctx* ctx, long long* code);

/* The code (as for lbm_set_tile) of the step kernel configuration that
 * lbm_create starts from for these arguments, without a context or a device:
 * host only, so it also answers on machines without a GPU.  LBM_EINVAL for a
 * null code, an invalid stencil or precision, a box that lbm_create rejects, or
 * tau <= 1/2. */
lbm_status lbm_default_tile(lbm_box box, int stencil, int prec, double tau, long long* code);

/* Shift n0 and storage scale of the populations (F32/F16 modes; 0 and 1 for F64). */
lbm_status lbm_storage_params(const lbm_ctx* ctx, double* n0, double* scale);

const char* lbm_strerror(lbm_status s);
const char* lbm_last_error(const lbm_ctx* ctx);

/* ---------------------------------------------------------------- flat interface */

/* Flat-interface coexistence (Sec. IV, flat-interface paragraph): a strip of gas of
 * width Lx/2 in liquid (Eq. (24), densities rho_g0 / rho_l0; both 0 = start from
 * lbm_coexistence_estimate) on a periodic
 * Lx x m x m box (m = 3 for E4, 5 for E6/E8; a field uniform in y and z is the
 * paper's 2-D strip reduced exactly), run until delta u < tol_du (checked every
 * 2^11 steps) or max_steps.  Returns the bulk densities n_g (strip centre) and n_l
 * (far edge), and sigma_0 = int_{Lx/2}^{Lx} (P_N - P_T) dx (Eq. (25), P from
 * Eq. (9), trapezoid on the nodes).  The workspace (caller-owned device memory)
 * holds lbm_flat_workspace_bytes bytes.  Synchronises; LBM_ENOTCONV still fills
 * the outputs. */
size_t lbm_flat_workspace_bytes(int Lx, int stencil, int prec);

/* Continuum estimate of the flat-interface coexistence (host only, no device
 * work): with P_N constant through a flat interface, the continuum limit of the
 * lattice pressure tensor (Eq. (9)) gives P(n_g) = P(n_l) = p_0 for the bulk
 * pressure of Eq. (10) and int_{n_g}^{n_l} (p_0 - P(n)) psi'(n)/psi(n) dn = 0.
 * Solved by bisection on n_g between the spinodals with Gauss-Legendre
 * quadrature in log n.  The lattice values (lbm_flat_interface) differ from it by
 * the higher-order terms of Eq. (9), ~1e-3 relative.  LBM_EINVAL when P(n) has
 * no van der Waals loop (G at or above G_c) or when the condition has no root
 * (its gas density reaches 0: psi = 1 - exp(-n) below G ~ -6.35).  p0 may be null. */
lbm_status lbm_coexistence_estimate(lbm_eos eos, double G, double* n_g, double* n_l, double* p0);
lbm_status lbm_flat_interface(double tau, double G, lbm_eos eos, int stencil, int prec, int Lx,
                              double rho_l0, double rho_g0, long long max_steps, double tol_du,
                              void* dev_workspace, size_t bytes, void* cuda_stream, double* n_g,
                              double* n_l, double* sigma0, long long* steps);

/* ---------------------------------------------------------------- groups of lattices */

/* Step several existing lattices together: one launch of the step kernel per time
 * step covers all of them (the batch kernel over a table of the contexts), so
 * small lattices fill the GPU as one larger one does.  The paper has no
 * counterpart; its runs are independent lattices, which is what makes this
 * possible.  All contexts need the same stencil and F64 or F32 storage; each
 * keeps its own box, tau, G and psi and evolves bitwise as under lbm_step.
 * lbm_group_workspace_bytes: device bytes for the table of n contexts;
 * lbm_group_create: caller-owned workspace (256-byte aligned), the stream all
 * group work is enqueued on (order it with the contexts' streams; using the same
 * stream does), the contexts stay owned by the caller and must outlive the group.
 * lbm_group_step: advance every lattice n >= 0 steps (async; CUDA graphs of 128
 * steps); afterwards lbm_observables etc. work per context as usual. */
typedef struct lbm_group lbm_group;
size_t lbm_group_workspace_bytes(int n);
lbm_status lbm_group_create(lbm_ctx* const* ctxs, int n, void* dev_workspace, size_t bytes,
                            void* cuda_stream, lbm_group** out);
lbm_status lbm_group_step(lbm_group* g, long long n);
const char* lbm_group_last_error(const lbm_group* g);
void lbm_group_destroy(lbm_group* g);

/* ---------------------------------------------------------------- Tolman fit */

/* Least-squares fit of Eq. (2) / Eq. (12): sigma_s = sigma0 (1 - 2 delta x + c x^2)
 * with x = 1/R_s, negative for bubbles (Sec. IV: bubbles have negative curvature).
 * Host arrays of m entries; entries with non-finite R_s or sigma_s are skipped.
 * quadratic = 0 fits the line (c = 0).  Host-only; needs >= 2 (3) usable points. */
lbm_status lbm_tolman_fit(const double* R_s, const double* sigma_s, const int* is_bubble,
                          long long m, int quadratic, double* sigma0, double* delta, double* c);

/* ---------------------------------------------------------------- batches of lattices */

/* The sweep of Sec. IV (droplets and bubbles of many radii, at several couplings)
 * as one job: independent lattices of uneven boxes advance together, one launch of
 * the step kernel per time step for all of them (captured in a CUDA graph of
 * check_every launches), each until one of the two convergence tests of Sec. IV
 * holds.  Every lattice of a batch has the batch's stencil and storage, and its
 * own box, tau, G, psi and storage shift / scale.  F16_SHIFTED batches take E4
 * and runs with tau = 1, nx % 8 == 0 and nx >= 48 (the FP16 moment kernel):
 * lbm_batch_enqueue returns LBM_EINVAL for other runs.
 *
 * lbm_batch_workspace_bytes: device bytes for `slots` resident lattices whose
 * boxes fit max_box (0 for invalid arguments).  lbm_batch_create: the caller's
 * workspace (256-byte aligned) and stream, as for lbm_create.  lbm_batch_enqueue:
 * queue one run (arguments of lbm_create / lbm_init_drop; box <= max_box), *id
 * receives its index.  lbm_batch_run: run the queue to the end -- a slot takes the
 * next run when its lattice finishes (converged, max_steps reached, or a non-finite
 * field); check_every is rounded up to even; *lattice_updates (may be null)
 * receives the lattice updates done.  Synchronises once per check.
 * A lattice whose droplet or bubble has collapsed (status bit 1) at two checks in
 * a row is finished early with LBM_ECOLLAPSE: it can no longer give a point.
 * lbm_batch_result: the observables of a finished run (criterion filled in) and
 * its outcome: LBM_OK (converged), LBM_ENOTCONV, LBM_ECOLLAPSE, LBM_ENUMERIC,
 * LBM_ETIMEOUT, or the error that stopped its set-up. */
typedef struct lbm_batch lbm_batch;
size_t lbm_batch_workspace_bytes(int slots, lbm_box max_box, int stencil, int prec);
lbm_status lbm_batch_create(int slots, lbm_box max_box, int stencil, int prec, void* dev_workspace,
                            size_t bytes, void* cuda_stream, lbm_batch** out);
lbm_status lbm_batch_enqueue(lbm_batch* b, lbm_box box, double tau, double G, lbm_eos eos,
                             const double center[3], double R, double rho_in, double rho_out,
                             double width, int* id);
lbm_status lbm_batch_run(lbm_batch* b, long long max_steps, long long check_every, double tol_dP_rel,
                         double tol_du, long long* lattice_updates);
lbm_status lbm_batch_result(const lbm_batch* b, int id, lbm_obs* out);
/* Batch autotuner: fills the slots from the queue, times `reps` (>= 2, rounded up
 * to even) launches of the batch step for every candidate -- kernel mode (the
 * row-chunk moment kernel, the element-copy moment kernel, the pipelined kernel,
 * where the queue allows each; F16: the moment kernel only), z chunk (8, 16, 32
 * planes) and slot count (all
 * slots, or half of them when at least four lattices are resident) -- and keeps
 * the one with the most lattice updates per second for lbm_batch_run.  The
 * measured lattices are then started again from their initial drops (runs beyond
 * the chosen slot count go back to the queue), so results do not depend on the
 * tuning.  *choice (may be null) = mode * 10^6 + z chunk * 10^3 + slots (mode:
 * 1 pipelined, 2 row-chunk moment, 3 element-copy moment; 0 mixed tau).
 * Synchronises.  Errors: LBM_EINVAL for a null batch or an empty queue,
 * LBM_ECUDA. */
lbm_status lbm_batch_autotune(lbm_batch* b, int reps, long long* choice);
const char* lbm_batch_last_error(const lbm_batch* b);
void lbm_batch_destroy(lbm_batch* b);

/* ---------------------------------------------------------------- z-slab decomposition */

/* One lattice split along z over `world` slabs (one process and GPU each), for
 * boxes larger than one GPU holds.  The update of Eq. (3) is local (Sec. II,
 * below Eq. (3)): the new populations of a node depend on the stored
 * populations within R + 1 planes, R the force stencil's radius (1 for E4, 2 for
 * E6 / E8).  Each slab is its own context of nx x ny x (owned + 2(R + 1)) nodes:
 * local planes 0..R are the ghost planes below the owned ones, then the owned
 * planes, then R + 1 ghost planes above.  It is stepped as a periodic lattice
 * (lbm_step); the wrap-around then reaches only ghost planes, whose results are
 * discarded, so the owned planes evolve exactly as in the whole lattice.  After
 * every step the ghost planes' needed populations are copied from the
 * neighbouring slabs (slab r - 1 below, r + 1 above, periodic in r).
 *
 * lbm_slab_partition: contiguous, balanced slabs of nz planes; z_begin (host
 * array of world + 1 ints) receives slab r's first global plane in z_begin[r]
 * and nz in z_begin[world].  LBM_EINVAL for a null pointer, nz or world < 1, or
 * a slab thinner than R + 1 planes (its ghost planes would reach past its
 * neighbours). */
lbm_status lbm_slab_partition(int nz, int world, int stencil, int* z_begin);

/* The populations (bit i = population i, order above) that ghost plane k
 * (1..R + 1, counted outward from the owned planes) on side -1 (below) or +1
 * (above) must hold before a step: those with c_z pointing into the slab for
 * k <= R + 1, c_z = 0 for k <= R, c_z pointing away for k <= R - 1 -- 19 R
 * population planes per side, against 19 (R + 1) for whole ghost planes.
 * LBM_EINVAL for a null mask, an unknown stencil, side not +-1 or k out of range. */
lbm_status lbm_slab_halo_mask(int stencil, int side, int k, unsigned* mask);

/* lbm_set_populations with the storage shift and scale given instead of derived
 * from the field, so that every slab of one lattice stores alike (take them
 * from lbm_storage_params of a context holding the whole field, or agree on
 * them across processes).  n0 is ignored for FP64 storage; scale must be 1 for
 * FP64 / FP32 and a power of two for FP16.  LBM_EINVAL otherwise, or as
 * lbm_set_populations. */
lbm_status lbm_set_populations_storage(lbm_ctx* ctx, const double* host_f, double n0, double scale);

/* Device address and size in bytes of population i's plane z of the current
 * state (stored type: 8, 4 or 2 bytes per node; FP32 / FP16 hold
 * (f_i - w_i n0) * scale).  The address is valid until the next step, which
 * swaps the state buffers.  For exchanges between processes (e.g.
 * torch.distributed send / recv of these planes).  LBM_EINVAL for null pointers
 * or an index out of range. */
lbm_status lbm_state_plane(const lbm_ctx* ctx, int i, int z, void** dev_ptr, size_t* bytes);

/* Copy the populations in mask (bit i = population i) of plane src_z of src's
 * current state into plane dst_z of dst's current state (slabs in one process,
 * on the same or peer devices).  Enqueued on dst's stream after the work already
 * queued on src's stream; the caller keeps src from stepping twice more before
 * the copy has run (one stream for all slabs does).  Both contexts must have
 * the same nx, ny, storage precision and storage parameters (LBM_EINVAL
 * otherwise, or for a plane out of range or mask bits above 18). */
lbm_status lbm_halo_copy(lbm_ctx* dst, int dst_z, const lbm_ctx* src, int src_z, unsigned mask);

/* ---------------------------------------------------------------- no-allocation variant */

/* Mass and centre of mass of a density field, for callers that cannot allocate
 * device memory.  The paper has no counterpart to this entry point: it is the
 * mass / centre-of-mass part of lbm_observables, offered for code that holds a
 * density field in its own device buffer but may not call cudaMalloc (or ask a
 * library to) -- e.g. code running inside another framework's memory pool, or
 * at a point of a pipeline where new allocations are not allowed.
 *
 * dev_rho: device array of nx*ny*nz doubles (layout above), read only.
 * n_ref: the outer density (e.g. lbm_obs.n_out); the centre of mass is that of
 * n - n_ref with minimum-image displacements about the centre node, as in
 * lbm_obs.com.  dev_out: device array of 4 doubles, written with
 * {sum_x n, com_x, com_y, com_z}.  Async on cuda_stream.  When
 * sum_x (n - n_ref) is exactly 0 (a field uniform at n_ref, say) there is no
 * centre of mass and com_x, com_y, com_z are NaN; the mass is still written.
 *
 * No device memory is allocated: per-block partial sums go to a fixed scratch
 * array inside the library (160 KiB per device, held until the process exits).
 * Limit: nx*ny*nz <= 33554432 nodes (4096 partial sums of 8192 nodes); larger
 * fields, sides < 1 or null pointers (checked in that order) return LBM_EINVAL
 * with a message in lbm_last_error(NULL).  The first call on a device looks up the scratch's
 * device address with that device current; make that first call before any
 * stream capture.  The address is cached per device index for the life of the
 * process: after a cudaDeviceReset (or anything else that destroys and
 * re-creates the device's primary context) the cached address is stale, so do
 * not call this entry point on a device that was reset after its first call.
 * Every call shares the one scratch array, which keeps the
 * last call's partial sums (each call writes every record it reads, so nothing
 * needs clearing); calls that overlap on the GPU -- on two streams, say --
 * race on it and must be serialised by the caller. */
lbm_status lbm_density_moments_noalloc(const double* dev_rho, int nx, int ny, int nz, double n_ref,
                                       double* dev_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
