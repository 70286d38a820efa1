/*
 * tflbm: GB300 (sm_103a) library for the thin-film D2Q9 lattice Boltzmann
 * method of Zitz, Scagliarini, Maddu, Darhuber and Harting, "A lattice
 * Boltzmann method for thin liquid film hydrodynamics", arXiv:1810.07642.
 *
 * Plain C ABI: plain pointers and sizes, no C++ or PyTorch types.
 *
 * Method (Section II of the paper).  The film height h(x, y, t) is the zeroth
 * moment of nine populations f_l on a periodic square lattice (Eq. speeds,
 * weights w_l).  One time step is
 *   h = sum_l f_l,  h u = sum_l c_l f_l                        (moments)
 *   p = -gamma (lap h + pi_sign * kappa(x) f(h))               (Eqs. pfilm, disjoiningP)
 *   F = -h grad p - nu alpha_delta(h) u + h (gx_body, gy_body) (Eqs. force, forcefric, alphafric)
 *   f*_l = (1 - omega) f_l + omega f_eq_l(h, u) + 3 w_l c_l . F (Eq. LBE)
 *   f_l(x + c_l, t + 1) = f*_l(x, t)                           (streaming)
 * with lap and grad the isotropic stencils of Eqs. (n_laplace) and
 * (derivative), nu = (tau - 1/2)/3, omega = 1/tau and
 * kappa = (1 - cos theta)(n - 1)(m - 1)/((n - m) h_*).
 * Readings of garbled or silent points:
 *   - equilibria (Eq. equilibria) with the printed c_s^2 read as e^2 = 1 (the
 *     printed form breaks the paper's own momentum constraint);
 *   - the printed w_l inside the Laplacian sums is dropped;
 *   - pi_sign = +1 (default) is the physical p = -gamma(lap h + Pi); -1 is the
 *     printed p = -gamma(lap h - Pi), whose precursor film is unstable;
 *   - F is tangential gravity on the liquid column, F = h g_par;
 *   - initial populations are f_l = f_eq_l(h0, u = 0).
 *
 * Conventions for every entry point:
 *   - Fields are contiguous row-major [ny][nx], x fastest; population arrays
 *     are [9][ny][nx] in the order of Eq. (speeds):
 *     (0,0) (1,0) (1,1) (0,1) (-1,1) (-1,0) (-1,-1) (0,-1) (1,-1).
 *   - "device" pointers are CUDA device (or managed) memory on the handle's
 *     device.  The element type of h0, theta, and of every field output is
 *     the compute type: double for TF_LBM_F64, float for the others.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All calls
 *     are asynchronous on it except tf_lbm_mass and tf_lbm_check, which
 *     synchronise it to return a host value.
 *   - Return value: TF_LBM_OK (0) or a negative TF_LBM_ERR_* code; nothing is
 *     thrown across the ABI.  tf_lbm_last_error gives a message.
 *   - The library owns the population buffers and the kappa field; the
 *     caller owns every pointer it passes in.
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef TFLBM_H
#define TFLBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* storage / compute type of the populations */
enum {
    TF_LBM_F32 = 0,  /* FP32 storage and arithmetic                          */
    TF_LBM_F64 = 1,  /* FP64 storage and arithmetic                          */
    TF_LBM_F16 = 2,  /* moving populations in FP16, rest population and all
                        arithmetic in FP32 (see below)                       */
    TF_LBM_BF16 = 3  /* as TF_LBM_F16 with BF16 moving populations           */
};
/* 16-bit storage (TF_LBM_F16, TF_LBM_BF16).  The rest population carries
 * almost all of h; it is kept in FP32 as f_0 - href (href = smallest h0).  The
 * eight moving populations are kept as deviations from the rest equilibrium
 * at href, f_l - f_eq_l(href, 0), in FP16 scaled by 2^10 or in BF16.  Every
 * value is decoded to FP32 before use, and the 16-bit rounding of each
 * collision is folded exactly into the FP32 rest population, so the total
 * volume changes only by FP32 roundings of f_0 - href.  Bytes per lattice
 * update: 2 x (4 + 8 x 2) = 40 (+4 with a theta field), against 72 (+4) in
 * FP32. */

/* return codes */
enum {
    TF_LBM_OK = 0,
    TF_LBM_ERR_ARG = -1,         /* invalid argument (message says which)  */
    TF_LBM_ERR_CUDA = -2,        /* a CUDA runtime call failed              */
    TF_LBM_ERR_NOMEM = -3,       /* device allocation failed                */
    TF_LBM_ERR_NONFINITE = -4,   /* reserved: state check found bad values  */
    TF_LBM_ERR_UNSUPPORTED = -5  /* option not built into this library      */
};

/* bits of the status word returned by tf_lbm_check */
enum {
    TF_LBM_STATUS_NONFINITE = 1,  /* some population or h is NaN or inf */
    TF_LBM_STATUS_NONPOSITIVE = 2, /* some h <= 0 (Pi and alpha singular) */
    TF_LBM_STATUS_TIMEOUT = 4,     /* a step kernel gave up waiting for its
                                      own bulk copies (results invalid)    */
    TF_LBM_STATUS_BOUNDS = 8       /* bounds-checked debug build only
                                      (compiled with TFLBM_CHECK_BOUNDS): a
                                      step kernel computed an index outside
                                      its buffer; the access was redirected
                                      to element 0 (results invalid)       */
};

/* Physical and numerical parameters (lattice units, dx = dt = 1). */
typedef struct tf_lbm_params {
    int32_t nx, ny;       /* periodic lattice size, each >= 1                   */
    int32_t dtype;        /* TF_LBM_F32, TF_LBM_F64, TF_LBM_F16 or TF_LBM_BF16   */
    int32_t n_exp, m_exp; /* exponents of Eq. (disjoiningP), n != m, >= 1     */
    int32_t pi_sign;      /* +1 physical (default) or -1 printed sign of Pi     */
    int32_t forcing;      /* 0: Eq. (LBE) as printed (default): u = j/h, source
                             3 w_l c_l.F.  1: second-order forcing (labelled
                             alternative, not the printed equation): u =
                             (j + F/2)/h with the friction taken at that
                             velocity, u (h + nu alpha/2) = j + F'/2, and the
                             source (1 - omega/2) w_l [3 (c_l - u) +
                             9 (c_l.u) c_l].F.  It reproduces the growth
                             rates and critical wavenumbers of Sec. III A
                             (Eq. RTgrowth); forward steps only (the adjoint
                             entry points reject it)                          */
    double tau;           /* relaxation time, > 1/2; omega = 1/tau             */
    double gamma;         /* surface tension                                    */
    double g;             /* gravity in the equilibria (g < 0: hanging film)    */
    double delta;         /* slip length of Eq. (alphafric), >= 0               */
    double hstar;         /* precursor thickness h_* > 0                        */
    double gx_body;       /* tangential body acceleration: F = h (gx, gy)       */
    double gy_body;
    double theta_uniform; /* contact angle in radians when no theta field      */
} tf_lbm_params;

typedef struct tf_lbm_handle tf_lbm_handle;

/* Kernel launch shape of the fused step (for autotuning).
 *   block_x: CTA width in lattice columns (64, 128 or 256);
 *   rows:    lattice rows marched by one CTA (>= 1): the ny rows are cut
 *            into ceil(ny / rows) near-equal bands.  The shape chosen by
 *            tf_lbm_init (and bands-exact candidates of tf_lbm_tune) instead
 *            uses the number of bands that fills the GPU's resident CTA
 *            slots once, so its bands need not all have `rows` rows; rows
 *            then reports the tallest band, and passing it back to
 *            tf_lbm_set_launch gives ceil(ny / rows) bands;
 *   graph_chunk: steps per captured CUDA graph in tf_lbm_step (0 = none,
 *            otherwise an even number >= 2);
 *   pipeline: 3 = every thread owns two adjacent columns, loads aligned
 *            pairs one (FP32) or two (16-bit) rows ahead, takes the values
 *            that cross a pair boundary from the neighbouring lane and
 *            computes both nodes with paired FP32 instructions (nx even, not
 *            TF_LBM_F64; default at tau = 1 when nx is even, block_x 64 for
 *            TF_LBM_F16 and TF_LBM_BF16, 128 for TF_LBM_F32); 1 = every
 *            thread loads its own column into registers, one row ahead
 *            (default otherwise); 2 = every
 *            thread copies its own populations into shared memory by
 *            asynchronous copies, two rows ahead (TF_LBM_F32 and TF_LBM_F64
 *            only); 0 = row segments streamed into shared memory by bulk
 *            copies four rows ahead (needs nx a multiple of 8, >= 16).
 * Results do not depend on rows or graph_chunk; the pipelines agree to
 * rounding. */
typedef struct tf_lbm_launch {
    int32_t block_x;
    int32_t rows;
    int32_t graph_chunk;
    int32_t pipeline;
} tf_lbm_launch;

/* Create a simulation and set f_l(x, 0) = f_eq_l(h0(x), u = 0).
 *   out:    receives the new handle (NULL on failure).
 *   params: copied; validated (ARG error on nx, ny < 1, tau <= 1/2,
 *           hstar <= 0, n == m, n or m < 1, delta < 0, |pi_sign| != 1,
 *           unknown dtype).
 *   h0:     device [ny][nx] initial film height (not retained).
 *   theta:  device [ny][nx] contact angle theta(x) in radians, or NULL for
 *           params->theta_uniform everywhere.  kappa(x) is computed once,
 *           in double precision, and kept by the library.
 * Uses the current CUDA device; allocates about 2 * 9 * ny * nx elements.
 * Cite: Section II, Eqs. (LBE), (equilibria), (disjoiningP). */
int tf_lbm_init(tf_lbm_handle** out, const tf_lbm_params* params,
                const void* h0, const void* theta, void* stream);

/* Advance the state by nsteps >= 0 time steps of Eq. (LBE) (one fused kernel
 * launch per step, optionally replayed from a captured CUDA graph). */
int tf_lbm_step(tf_lbm_handle* H, int64_t nsteps, void* stream);

/* Write the moments of the current post-streaming populations:
 * h = sum_l f_l and u = sum_l c_l f_l / h (Section II).  Each of h, ux, uy
 * is a device [ny][nx] buffer or NULL to skip it. */
int tf_lbm_moments(tf_lbm_handle* H, void* h, void* ux, void* uy, void* stream);

/* Write the film pressure p (Eq. pfilm) and the total force (Eq. force) of the
 * current state.  Each pointer is a device [ny][nx] buffer or NULL. */
int tf_lbm_pressure_force(tf_lbm_handle* H, void* p, void* fx, void* fy, void* stream);

/* Total liquid volume sum_x h(x) of the current state, accumulated in double
 * precision with compensated summation.  Synchronises `stream`.  The paper
 * states the method conserves mass (Section III B). */
int tf_lbm_mass(tf_lbm_handle* H, double* mass_host, void* stream);

/* Scan the current state: *status_host = OR of TF_LBM_STATUS_* bits (0 when
 * every population and h is finite and every h > 0 and no step kernel timed
 * out).  Synchronises `stream`. */
int tf_lbm_check(tf_lbm_handle* H, int32_t* status_host, void* stream);

/* Copy the post-streaming populations f_l(x, t) out to / in from a device
 * [9][ny][nx] buffer of DOUBLES, whatever the handle's dtype (checkpoint /
 * resume).  For TF_LBM_F32 the export is exact and importing an exported
 * state reproduces the stored values bit for bit; other imported values are
 * rounded to float. */
int tf_lbm_get_state(tf_lbm_handle* H, void* f, void* stream);
int tf_lbm_set_state(tf_lbm_handle* H, const void* f, void* stream);

/* Number of time steps taken since init (set_state does not reset it). */
int64_t tf_lbm_time(const tf_lbm_handle* H);

/* Read or change the launch shape (see tf_lbm_launch). */
int tf_lbm_get_launch(const tf_lbm_handle* H, tf_lbm_launch* out);
int tf_lbm_set_launch(tf_lbm_handle* H, const tf_lbm_launch* in);

/* How long the bulk-copy step kernel (pipeline 0) waits for one of its
 * own row copies before giving up: `polls` tests of the copy's completion
 * barrier (polls < 0 restores the default, 2^22; polls == 0 gives up at
 * once).  A kernel that gives up sets TF_LBM_STATUS_TIMEOUT (tf_lbm_check),
 * stops issuing copies, waits (with the default bound) for the copies it has
 * already issued and returns; the populations of that step are invalid.
 * This exists to exercise that path without a fault: no paper counterpart.
 * Later steps of the same handle keep TF_LBM_STATUS_TIMEOUT set. */
int tf_lbm_set_wait_limit(tf_lbm_handle* H, int32_t polls);

/* ---------------------------------------------------------------- adjoint
 * Reverse-mode derivative of the step (not in the paper; the method's own
 * equations differentiated exactly, Eqs. LBE, equilibria, force, pfilm,
 * disjoiningP, forcefric, alphafric, derivative, n_laplace).  All arrays are
 * device memory of the handle's compute type (double for TF_LBM_F64, float
 * otherwise); population arrays are post-streaming, [9][ny][nx].  With
 * 16-bit storage the derivative is the FP32 scheme's, evaluated on the
 * stored trajectory. */

/* a_t = dL/df(t) from a_next = dL/df(t+1) for one step taken from the
 * post-streaming state f_t; adds dL/dkappa of the step to grad_kappa
 * ([ny][nx], accumulated).  a_t must not alias a_next.  Uses 10 fields of
 * handle-owned scratch (allocated on first use). */
int tf_lbm_adjoint_step(tf_lbm_handle* H, const void* f_t, const void* a_next, void* a_t,
                        void* grad_kappa, void* stream);

/* Gradient tape over nsteps steps with checkpoint-recompute: a copy of the
 * state every `every` steps (<= 0: ceil(sqrt(nsteps))).  h0 and theta
 * (device [ny][nx], theta NULL = params->theta_uniform) must be the ones the
 * handle was created from; they are copied. */
typedef struct tf_lbm_tape tf_lbm_tape;
int tf_lbm_tape_create(tf_lbm_handle* H, const void* h0, const void* theta, int64_t nsteps,
                       int32_t every, tf_lbm_tape** out);
/* Advance the handle by nsteps, storing the checkpoints. */
int tf_lbm_tape_forward(tf_lbm_tape* tape, void* stream);
/* Given grad_h = dL/dh at the final time ([ny][nx]), write dL/dtheta and
 * dL/dh0 (each [ny][nx], or NULL to skip).  Recomputes each segment from its
 * checkpoint; the handle ends at the final state again. */
int tf_lbm_tape_backward(tf_lbm_tape* tape, const void* grad_h, void* grad_theta, void* grad_h0,
                         void* stream);
void tf_lbm_tape_destroy(tf_lbm_tape* tape);

/* ---------------------------------------------------------- autotuning
 * Time candidate launch shapes of the fused step on the handle's own state
 * and keep the fastest.  Each candidate runs 2 untimed and `trial_steps`
 * timed steps (rounded up to even; <= 0 means 16), timed with CUDA events on
 * `stream`.  Candidates: block_x in {64, 128, 256}, every pipeline that
 * applies, and band counts of one, two and three waves of resident CTAs
 * (both balanced bands filling the waves exactly and their rounded-up band
 * heights) and band heights of 2 to 256 rows.  The state is copied aside first (one population
 * buffer of device memory, freed before return) and put back after, so f
 * and tf_lbm_time are as before the call.  The graph chunk is kept.
 * Synchronises `stream`.  best (host, may be NULL) receives the shape now in
 * use. */
int tf_lbm_tune(tf_lbm_handle* H, int32_t trial_steps, tf_lbm_launch* best, void* stream);

/* -------------------------------------------------------- diagnostics
 * Film diagnostics of the current state, computed on the device (Section
 * III): the drop's contact radius from its wetted area and its apex height
 * (Sec. III B: r = sqrt(A / pi), R = (r^2 + h_d^2) / (2 h_d), theta =
 * arcsin(r / R)), its position on the periodic lattice from circular first
 * moments, its sliding velocity U from the momentum over the wetted nodes
 * (Sec. III C: Ca = nu U / gamma with rho = 1), and the amplitude of one
 * Fourier mode of h (Sec. III A: a single-mode amplitude is
 * 2 |mode_cos + i mode_sin| / (nx ny)).  The wetted nodes are those with
 * h > h_wet.  h and j are the moments of the post-streaming populations
 * (Section II); every sum is taken in double precision with compensated
 * summation. */
typedef struct tf_lbm_diag {
    double mass;      /* sum of h over the lattice                          */
    double wet_mass;  /* sum of h over the wetted nodes                     */
    double wet_jx;    /* sum of j_x = sum_l c_lx f_l over the wetted nodes  */
    double wet_jy;    /* sum of j_y over the wetted nodes                   */
    double wet_area;  /* number of wetted nodes                             */
    double h_max;     /* largest h                                          */
    double wet_cos_x; /* sum over wetted nodes of h cos(2 pi x / nx)        */
    double wet_sin_x; /* ... h sin(2 pi x / nx)                             */
    double wet_cos_y; /* ... h cos(2 pi y / ny)                             */
    double wet_sin_y; /* ... h sin(2 pi y / ny)                             */
    double mode_cos;  /* sum over the lattice of h cos(2 pi (mx x / nx + my y / ny)) */
    double mode_sin;  /* ... h sin(...)                                     */
} tf_lbm_diag;
/* out: device pointer to one tf_lbm_diag (twelve doubles), written
 * asynchronously on `stream` (no host synchronisation).  (mode_x, mode_y)
 * are the integer wave numbers (mx, my) of the Fourier sums.  Uses a small
 * handle-owned scratch allocated on first use.  ARG error on a NULL or host
 * `out` or a NaN h_wet. */
int tf_lbm_diagnostics(tf_lbm_handle* H, double h_wet, int32_t mode_x, int32_t mode_y, void* out,
                       void* stream);

/* Term balance of the paper's appendix: the L2 norms (Eq. magnitude,
 * ||phi||_2 = (sum_x phi^2 / (nx ny))^(1/2)) of the x-components of the
 * film-pressure term -h d_x p, the friction term -nu alpha(h) u_x (Eqs.
 * forcefric, alphafric) and the longitudinal dissipation
 * nu lap(h u_x) + 2 nu d_x(div(h u)), the derivatives taken with the
 * stencils of Eqs. (derivative) and (n_laplace).  out: device pointer to
 * three doubles in that order, written asynchronously.  Uses 5 fields of
 * handle-owned scratch (allocated on first use). */
int tf_lbm_term_norms(tf_lbm_handle* H, void* out, void* stream);

/* --------------------------------------------------------------- batches
 * Many independent simulations of uneven sizes (a parameter sweep) advanced
 * together: each step is ONE launch over a table of work items, (domain,
 * column strip, row band), and tf_lbm_batch_step replays CUDA graphs of
 * graph_chunk such launches.  The batch borrows the handles: they stay
 * owned by the caller, must outlive the batch and must all have the same
 * dtype; the per-handle calls (moments, mass, check, diagnostics, state
 * import and export) work between batch steps, as does tf_lbm_step on a
 * single handle.  Handles with a theta field and handles without one may be
 * mixed (the batch then keeps a filled kappa field for the uniform ones).
 * When some handles have tau == 1 and others not, all take the general-tau
 * kernel, so those with tau == 1 match their single-handle results to
 * rounding rather than bit for bit. */
typedef struct tf_lbm_batch tf_lbm_batch;

/* Launch shape of a batch.
 *   block_x, rows: as in tf_lbm_launch, common to all domains (a domain of
 *            ny rows is cut into ceil(ny / rows) near-equal bands);
 *   graph_chunk: steps per captured CUDA graph (0 or even, <= 4096);
 *   queue:   0 = one CTA per work item; 1 = a persistent grid of one wave of
 *            resident CTAs, each taking items from an atomic counter until
 *            none are left;
 *   pipeline: 1 = one column per thread; 3 = two columns per thread, as in
 *            tf_lbm_launch (every domain's nx even, not TF_LBM_F64).  The
 *            default is 3 where it applies and every tau is 1 (as for a
 *            single handle), else 1.  Both run the node arithmetic of the
 *            single-handle kernel of the same pipeline. */
typedef struct tf_lbm_batch_launch {
    int32_t block_x;
    int32_t rows;
    int32_t graph_chunk;
    int32_t queue;
    int32_t pipeline;
} tf_lbm_batch_launch;

/* Create a batch of `count` >= 1 handles (host array, copied).  ARG error
 * on NULL handles, a repeated handle or mixed dtypes. */
int tf_lbm_batch_create(tf_lbm_batch** out, tf_lbm_handle* const* handles, int32_t count, void* stream);
/* Advance every handle of the batch by nsteps >= 0. */
int tf_lbm_batch_step(tf_lbm_batch* B, int64_t nsteps, void* stream);
/* Read or change the launch shape.  set_launch rewrites the work-item
 * table in place, so it first waits for all work on the device
 * (cudaDeviceSynchronize); ARG error on an invalid shape. */
int tf_lbm_batch_get_launch(const tf_lbm_batch* B, tf_lbm_batch_launch* out);
int tf_lbm_batch_set_launch(tf_lbm_batch* B, const tf_lbm_batch_launch* in);
/* As tf_lbm_tune, over block_x, rows, queue and the pipelines that apply,
 * for the whole batch (every handle's state copied aside and put back). */
int tf_lbm_batch_tune(tf_lbm_batch* B, int32_t trial_steps, tf_lbm_batch_launch* best, void* stream);
/* tf_lbm_diagnostics of every handle in two launches: out is a device array
 * of `count` tf_lbm_diag, in the order of the handles. */
int tf_lbm_batch_diagnostics(tf_lbm_batch* B, double h_wet, int32_t mode_x, int32_t mode_y, void* out,
                             void* stream);
/* Number of work items of one batched step (= CTAs without the queue). */
int32_t tf_lbm_batch_items(const tf_lbm_batch* B);
/* Waits for the batch's device work and frees what it owns (not the
 * handles).  NULL ok. */
void tf_lbm_batch_destroy(tf_lbm_batch* B);
/* Message of the last failed call on B (B != NULL), or of the last failed
 * tf_lbm_batch_create on this thread (B == NULL, same as
 * tf_lbm_last_error(NULL)). */
const char* tf_lbm_batch_last_error(const tf_lbm_batch* B);

/* Largest n accepted by tf_lbm_sum_noalloc: 4096 blocks of 16384 elements. */
#define TF_LBM_NOALLOC_MAX_ELEMS 67108864LL

/* Compensated (Neumaier) double-precision sum of x[0 .. n) written to *out,
 * with no memory allocation of any kind.  The paper has no counterpart: this
 * serves callers that cannot allocate device memory, e.g. code inside a host
 * application that owns the device memory budget through its own pool, or
 * loops that cannot afford cudaMalloc's possible device-wide synchronisation.
 * Summing the state exported by tf_lbm_get_state gives the total volume that
 * tf_lbm_mass reports, without a handle-side allocation.
 *   x:   device (or managed) array of n doubles on the current device; may
 *        be NULL when n == 0.
 *   n:   0 <= n <= TF_LBM_NOALLOC_MAX_ELEMS, else TF_LBM_ERR_ARG.
 *   out: device (or managed) double on the current device; written
 *        asynchronously on `stream`.
 * Host pointers and device memory of another GPU are TF_LBM_ERR_ARG.
 * Block partial sums go to a fixed 64 KB file-scope device array that every
 * GPU loading the library keeps until exit.  Its device address is looked up
 * on the first call made on each device, so make that first call before any
 * stream capture.  Calls share the array: calls whose kernels overlap on the
 * GPU (unordered streams) race and give wrong sums.  Errors are described by
 * tf_lbm_last_error(NULL). */
int tf_lbm_sum_noalloc(const double* x, int64_t n, double* out, void* stream);

/* Release everything the handle owns (waits for its device work). NULL ok. */
void tf_lbm_destroy(tf_lbm_handle* H);

/* Message of the last failed call on H (or of the last failed tf_lbm_init
 * on this host thread when H is NULL); "" if none.  Valid until the next
 * call on H. */
const char* tf_lbm_last_error(const tf_lbm_handle* H);

/* Library version, major * 10000 + minor * 100 + patch.  0.2.0 added the
 * pipeline field to tf_lbm_batch_launch (the struct grew by one int32). */
int32_t tf_lbm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TFLBM_H */
