/*
 * dg.h -- C ABI of libdg, a GB300 (sm_103a) implementation of the right-hand
 * side and time step of the modal Discontinuous Galerkin method for 3D
 * isothermal Euler on a periodic Cartesian mesh, driven by Ornstein-Uhlenbeck
 * forcing (Cernetic, Springel, Guillet & Pakmor 2024).
 *
 * ------------------------------------------------------------------------
 * Data layout (all device buffers are owned by the caller, e.g. torch
 * tensors; the library never allocates or frees device memory):
 *   N cells per axis, unit box, h = 1/N; cell c = (iz*N + iy)*N + ix.
 *   degree k in {1,2,3}; b = (k+1)(k+2)(k+3)/6 modes; n = k+1 Gauss points
 *   per axis.  Basis phi_{ijl}(xi) = Pn_i(xi_x) Pn_j(xi_y) Pn_l(xi_z),
 *   Pn_m = sqrt(2m+1) P_m, i+j+l <= k, ordered by total degree, then i
 *   descending, then j descending (mode 0 is the cell mean).
 *   state   u[c][4][b]      var = rho, m_x, m_y, m_z   ("state layout")
 *   vhat    [c][3][b]       projected velocity (Sec. 3.2)
 *   ahat    [c][3][b]       projected driving acceleration (Sec. 4.2)
 *   Element type: double for DG_PREC_F64, float for DG_PREC_F32 / DG_PREC_X3.
 *
 * Conventions:
 *   - every function returns DG_OK (0) or a DG_E* code; nothing throws and
 *     nothing exits; the text of the last error is dg_last_error(ctx).
 *   - kernels run on the caller's stream (dg_opts.stream, a cudaStream_t);
 *     calls that return host values synchronise that stream.
 *   - a context is not thread-safe: one host thread per context.
 * ------------------------------------------------------------------------
 */
#ifndef DG_H
#define DG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define DG_OK 0
#define DG_EINVAL 1        /* bad argument (null pointer, size, mode)           */
#define DG_ECUDA 2         /* a CUDA runtime call failed                         */
#define DG_ENOMEM 3        /* caller's scratch buffer too small                  */
#define DG_EPOSITIVITY 4   /* positivity retries exhausted (state left at u^n)  */
#define DG_ENONFINITE 5    /* a NaN/Inf coefficient was produced                 */
#define DG_ESTATE 6        /* called before dg_set_state                         */

/* ---- precision modes ----------------------------------------------------- */
#define DG_PREC_F64 0      /* everything in FP64 (parity mode)                   */
#define DG_PREC_F32 1      /* FP32 state and arithmetic; FP64 global sums        */
#define DG_PREC_X3 2       /* FP32 state; basis<->quadrature transforms on the
                              tensor cores as split-BF16 x3 products with FP32
                              accumulation; FP64 global sums                      */

/* ---- artificial viscosity modes ------------------------------------------ */
#define DG_AV_OFF 0
#define DG_AV_VNR 1        /* von Neumann-Richtmyer viscous pressure (Sec. 3.1)  */
#define DG_AV_LEARNED 2    /* per-cell coefficient predicted by the MLP           */

/* ---- face flux (Sec. 2: approximate Riemann solver on cell faces) --------- */
#define DG_RIEMANN_RUSANOV 0  /* local Lax-Friedrichs: F* = {F} - max(|v_n|+cs) [U]/2 */
#define DG_RIEMANN_HLL 1      /* HLL with the Davis speed bounds
                                 S_L = min(v_n^L, v_n^R) - cs, S_R = max(v_n^L, v_n^R) + cs */
#define DG_RIEMANN_HLLC 2     /* HLLC (Toro) for p = cs^2 rho, the paper's face solver:
                                 HLL mass and normal momentum; the tangential momenta
                                 cross with the side of the contact wave S_M = m*_n/rho* */

/* status bits reported by dg_step / dg_diagnostics */
#define DG_ST_LIMITED 1u   /* positivity rescaling happened in some cell         */
#define DG_ST_FAIL 2u      /* a cell mean reached the density floor              */
#define DG_ST_NONFINITE 4u /* a NaN/Inf was produced                              */
#define DG_ST_TIMEOUT 8u   /* a tensor-core completion wait gave up (the launch
                              stopped early; reported as DG_ECUDA)              */
#define DG_ST_REPEATED 16u /* positivity by repetition: a step was computed
                              again with troubled cells flattened               */

/* positivity treatment of dg_step (Sec. 3.1, last paragraph) */
#define DG_POS_SCALE 0     /* rescale the high-order weights of every stage
                              output below the floor (default)                  */
#define DG_POS_REPEAT 1    /* also repeat the step from a modified u^n: see
                              dg_step                                           */

typedef struct {
    int32_t n[3];          /* cells per axis; the library requires n[0]=n[1]=n[2],
                              at most 1024 (cell indices fit in 32 bits)         */
    double L[3];           /* box size; the library requires L = 1              */
} dg_mesh;

/* Viscous pressure Pi = alpha rho (h/p)^2 |div v|^2 + beta rho cs (h/p) |div v|
 * for div v < 0, capped at Pi_max = rho (h/p)^2 |div v| / (2 dt)  (Sec. 3.1,
 * p = k+1).  rho_floor is the positivity floor (Sec. 3.1, Sec. 5 uses 1e-3).
 * nu_gate (>= 0): in DG_AV_LEARNED mode a cell whose predicted coefficient
 * nu/(cs h/p) is below nu_gate gets nu = 0, i.e. no viscous pressure at any of
 * its points (the sensor's "no shock here" decision); 0 disables the gate.
 * A tile of 16 consecutive cells whose coefficients are all zero skips the
 * gradient evaluation and div v at its points (the result is the same as
 * with the work done: Pi = 0 there); dg_prof counts those tiles.
 * diffusion (>= 0): eps of div(eps grad u).  The interface gradient is the
 * normal derivative at the face of the polynomial recovered over the face's
 * two cells (degree 2K+1 in the normal direction from the K+1 normal
 * coefficients of each cell, per tangential mode): the paper's "virtual cell"
 * over both neighbours.  The time step is also limited by
 * dt <= cfl (h/(k+1))^2 / (2 eps). */
typedef struct {
    int32_t mode;          /* DG_AV_OFF, DG_AV_VNR, DG_AV_LEARNED                 */
    double alpha;          /* default 2.0                                          */
    double beta;           /* default 0.2                                          */
    double rho_floor;      /* default 1e-3                                         */
    double nu_gate;        /* default 0 (no gating)                                */
    double diffusion;      /* eps of an added div(eps grad u) on all four variables
                              (Sec. 2, diffusion across cell boundaries); 0: off   */
    int32_t fused_infer;   /* DG_AV_LEARNED steps: 1 = the last stage's kernel
                              evaluates the next step's coefficient; 0 (default) =
                              a separate inference launch per step.  Same values. */
} dg_nu_params;

typedef struct {
    int32_t precision;     /* DG_PREC_*                                           */
    int32_t rk_stages;     /* 2 (SSP-RK2) or 3 (SSP-RK3), Sec. 7; in FP32 and x3
                              the third RK3 stage uses b = float(2/3), a = 1 - b,
                              whose sum is exactly one (no steady scaling of the
                              state by the rounded fractions)                    */
    double cfl;            /* dt = cfl h / ((k+1) max sum_d(|v_d| + cs))           */
    void* stream;          /* cudaStream_t; must not be NULL                       */
    void* u[3];            /* three state registers, each N^3*4*b elements; the
                              current state rotates among them (dg_get_state
                              returns it; u[0] receives dg_set_state)            */
    void* vhat;            /* dg_vhat_bytes() bytes, 256-byte aligned: two
                              projected-velocity buffers of N^3*3*b elements (a
                              stage reads one while its epilogue writes the next
                              stage's into the other); the second starts at the
                              first multiple of 256 bytes past the first          */
    void* ahat;            /* N^3*3*b elements                                     */
    void* scratch;         /* >= dg_scratch_bytes(), 256-byte aligned              */
    size_t scratch_bytes;
    int32_t riemann;       /* DG_RIEMANN_*; 0 (Rusanov) when zero-initialised     */
    int32_t x3_backend;    /* DG_PREC_X3 at order 3 without diffusion: 0 (default)
                              = 5th-generation tensor-core kernels (tcgen05 with
                              TMEM accumulators: volume and face kernels per
                              stage, the projection kernel after the last stage
                              and, in driven steps, after every stage; the volume
                              term through a caller-scratch buffer; fused_infer
                              evaluates the sensor in that last projection);
                              1 = the single fused stage kernel on warp-level
                              mma.sync.  Other precisions, orders and the
                              diffusion operator use the fused kernel either way */
    int32_t positivity;    /* DG_POS_*; DG_POS_SCALE when zero-initialised        */
} dg_opts;

/* Driving (Sec. 4.2, eq. ornstein_uhlenbeck_process_time_evolution).  Modes:
 * integer k with kmin2 <= |k|^2 <= kmax2, one of each +-k pair.  Correlation
 * time tc = L/(2 cs mach) (eq. eddy_turnover_time), update interval
 * tc/100, rms acceleration sigma = 2 mach^2 cs^2 / L split evenly over the
 * modes and the solenoidal/compressive parts with weight zeta.  The OU
 * variables are drawn from SplitMix64(seed) + Box-Muller on the host.
 * t_off > 0 switches the driving off once t > t_off. */
typedef struct {
    int32_t on;
    int32_t kmin2, kmax2;
    double zeta;
    double mach;
    uint64_t seed;
    double t_off;
} dg_forcing;

typedef struct {
    double mass, mom[3], ekin, mach, mach_rho, rho_min, rho_max;
    double av_frac;        /* volume fraction with Pi > 0.01 cs^2 rho              */
    double inj_power;      /* int m.(a_h - abar) dV                                */
    double max_speed;      /* max sum_d(|v_d| + cs) over volume points             */
    double av_work;        /* int Pi div v dV                                      */
    uint32_t status;       /* sticky DG_ST_* bits since the last dg_set_state       */
    double t;              /* simulation time                                      */
    int64_t steps;         /* steps taken                                          */
} dg_diag;

/* checkpoint metadata: everything besides the coefficients that a resumed
 * run needs to continue bit-identically */
typedef struct {
    double t;
    int64_t steps;
    double dt_last;
    int32_t forcing_on;
    int32_t forcing_dirty;
    double t_next;
    uint64_t rng;
    int32_t have_spare;
    double spare;
    int32_t nmodes;
    double x[512][3][2];   /* OU variables                                        */
} dg_meta;

typedef struct dg_ctx dg_ctx;

/* Bytes of device scratch a context with these parameters needs.  DG_EINVAL
 * for a mesh dg_init rejects (not n x n x n, or n outside 1..1024) or an
 * order outside 1..3; no device is touched. */
int dg_scratch_bytes(const dg_mesh* mesh, int order, const dg_nu_params* nu, size_t* bytes);
/* Bytes of the projected-velocity buffer dg_opts.vhat must provide (same
 * mesh and order checks; precision 0..2). */
int dg_vhat_bytes(const dg_mesh* mesh, int order, int precision, size_t* bytes);

/* Create a context.  Builds the basis/quadrature tables (Sec. 2.1-2.2),
 * records the caller's buffers and stream.  No kernel runs before
 * dg_set_state.  On error *ctx is NULL. */
int dg_init(dg_ctx** ctx, const dg_mesh* mesh, int order, double cs, const dg_nu_params* nu,
            const dg_opts* opts);
void dg_free(dg_ctx* ctx);
const char* dg_last_error(const dg_ctx* ctx);

/* Copy a state (state layout, element type of the precision mode) into the
 * context; src on the host (pinned or pageable) or on the device. */
int dg_set_state(dg_ctx* ctx, const void* src, int src_on_host);
int dg_get_state(dg_ctx* ctx, void* dst, int dst_on_host);

/* Single evaluation of the semi-discrete right-hand side (Sec. 2.2, eq.
 * weight_evolution):
 *   dw_l/dt = 1/(4h) [ sum_q w_q sum_d dphi_l/dxi_d F_d(U_q)
 *                      - sum_faces sum_s w_s phi_l(xi_s) F*.n ]
 *             + (1/8) sum_q w_q phi_l rho_q (a_h(xi_q) - abar)  (momentum)
 * with the viscous pressure at volume points only (Sec. 3.1), face states
 * from rho and the projected velocity (Sec. 3.2), Rusanov fluxes, and
 * dt_for_pimax fixing Pi_max (<= 0: no cap).  u_in and dudt are device
 * buffers in state layout; ahat (device, [c][3][b]) may be NULL (no forcing).
 * vhat of the context is overwritten. */
int dg_rhs(dg_ctx* ctx, const void* u_in, const void* ahat, void* dudt, double dt_for_pimax);

/* Projection of the primitive velocity onto the basis (Sec. 3.2, eq.
 * weights_equation) by (k+1)^3-point Gauss quadrature: u_in -> vhat_out. */
int dg_project_velocity(dg_ctx* ctx, const void* u_in, void* vhat_out);

/* Advance nsteps SSP-RK steps (Sec. 7).  Per step: driving update when due,
 * dt from the CFL condition on u^n, S stages of (projection, RHS, stage
 * combine, positivity rescaling).  A step in which a cell mean reaches the
 * floor is redone from u^n with dt/2, at most 3 times; then DG_EPOSITIVITY
 * with the state left at u^n.  Synchronises the stream once per step.
 * fixed_dt > 0 replaces the CFL dt (used to replay a recorded sequence).
 *
 * DG_POS_REPEAT (Sec. 3.1, last paragraph, read as the troubled-cell
 * procedure the paper gives for its finite-volume scheme): a cell is troubled
 * when a stage output has negative rho at one of its volume or face Gauss
 * points (before the rescaling), or a volume point with sum_d(|v_d| + cs)
 * above 1.5 times the bound S that set dt (the stage breaks its step's Courant
 * condition; this test is an addition to the paper's text).  The modes l > 0
 * of every troubled cell of u^n that is not flat are multiplied by 1/2 (the
 * first two times in the step) or 0 (the third) and the step is computed
 * again from the modified u^n, with dt from its own S; a flat cell with
 * negative density, or a cell mean at the floor, halves dt for the following
 * attempts.  An attempt whose only troubled cells are flat ones marked for
 * their speed stands (with the rescaled stage outputs).
 * At most 32 attempts and 6 halvings, then DG_EPOSITIVITY with the state left
 * at u^n with its troubled cells flattened.  One more stream synchronisation
 * per repeated attempt; DG_ST_REPEATED reports that a step was repeated. */
int dg_step(dg_ctx* ctx, int nsteps, double fixed_dt, double* t_out, double* dt_last);

/* Configure the driving (Sec. 4.2, eq. ornstein_uhlenbeck_process_time_evolution
 * and the eddy turnover time t_c = L/(2 cs M)): an OU process of the integer
 * modes kmin2 <= |k|^2 <= kmax2 (one of each +-k pair), Helmholtz weight zeta,
 * advanced every t_c/100 at the first step whose time has reached the next
 * update time, switched off after t_off (> 0).  Draws the initial OU state
 * from its stationary law (SplitMix64(seed), Box-Muller) and projects the
 * acceleration onto the basis before the next step.  f->on == 0 switches the
 * driving off (zero acceleration).  DG_EINVAL for mach <= 0, kmin2 < 1,
 * kmax2 < kmin2, kmax2 > 64, zeta outside [0, 1] or more than 512 modes. */
int dg_set_forcing(dg_ctx* ctx, const dg_forcing* f);

/* Use an explicit projected acceleration (device or host, [c][3][b]) and
 * disable the OU schedule. */
int dg_set_forcing_coeffs(dg_ctx* ctx, const void* ahat_src, int src_on_host);

/* Project the acceleration of explicit Fourier modes onto the basis:
 * a(x) = sum_m 2 Re(amp_m exp(2 pi i kvec_m . x)); kvec [nm][3] int32 and
 * amp [nm][3][2] double on the host; result into ctx's ahat. */
int dg_forcing_from_modes(dg_ctx* ctx, int nmodes, const int32_t* kvec, const double* amp);

/* Diagnostics of the current state (Sec. 4.1); FP64 accumulation on the GPU.
 * dt_for_pimax as in dg_rhs.  Synchronises the stream. */
int dg_diagnostics(dg_ctx* ctx, double dt_for_pimax, dg_diag* out);

/* L1 density difference (eq. l1_norm) between two device states, by
 * (k+3)-point Gauss quadrature per axis per cell.  Synchronises. */
int dg_l1_density(dg_ctx* ctx, const void* uA, const void* uB, double* out);

/* ---- learned viscosity sensor (not in the paper: a small network stands in
 * for the shock sensor and is checked against it) -----------------------------
 * Network y = W3 . gelu(W2 gelu(W1 x + b1) + b2) + b3, gelu(z) = z/2 (1 +
 * erf(z/sqrt 2)), 64 hidden units, D = 2b inputs per cell
 *   x = (rho_l / rho_0, |v|hat_l / cs),  |v|hat the Gauss projection of |v|,
 * output y = log(nu / (cs h/p)).  In DG_AV_LEARNED mode the viscous pressure
 * at a volume point is Pi = rho nu |div v| for div v < 0, capped at
 * rho (h/p)^2 |div v| / (2 dt) as in Sec. 3.1; nu is evaluated once per step
 * (BF16 tensor-core inference, FP32 accumulation) and kept for its stages:
 * by a separate inference kernel at the start of the step, or (fused_infer)
 * by the last stage of the previous step, in the same kernel, for the state
 * it writes.  Both give the same values bit for bit; on GB300 the separate
 * launch is the faster of the two.
 * Parameters: FP32 array of dg_av_param_count() floats in the order
 * W1 [64][D] row-major, b1 [64], W2 [64][64], b2 [64], W3 [64], b3. */
typedef struct {
    double lr, beta1, beta2, eps;  /* Adam (Kingma & Ba); 1e-3, 0.9, 0.999, 1e-8 */
    int32_t batch;                 /* <= 4096 */
    int32_t epochs;
} dg_train_opts;

int dg_av_param_count(dg_ctx* ctx, int64_t* n);
/* Set / get the FP32 parameters (host arrays of dg_av_param_count floats);
 * setting them resets the Adam moments. */
int dg_set_av_weights(dg_ctx* ctx, const float* w, size_t n);
int dg_get_av_weights(dg_ctx* ctx, float* w, size_t n);
/* Inputs and plain-sensor targets of every cell of the current state (device
 * buffers x [N^3][2b], y [N^3] FP32): x = (rho_l/rho_0, |v|hat_l/cs) with
 * |v|hat the Gauss projection of |m/rho|; y = log(max(nu_cell, nu_f) /
 * (cs h/p)), nu_cell the Gauss-weighted mean, over the cell's volume points
 * with div v < 0, of the pointwise coefficient Pi/(rho |div v|) of the vNR
 * pressure of Sec. 3.1 (dt_for_pimax fixes the cap), 0 without such points;
 * nu_f = max(beta, 0.05) cs h/p the coefficient of the linear term.  Needs a
 * context created in DG_AV_LEARNED mode (it holds the |v| projection). */
int dg_generate_pairs(dg_ctx* ctx, double dt_for_pimax, float* x, float* y, int64_t cap, int64_t* n_out);
/* Minibatch Adam on the mean squared error of y over (x [n][2b], y [n]),
 * device buffers, batches in the given row order; *loss_out = mean batch
 * loss of the last epoch.  FP32 forward/backward kernels; gradient sums in a
 * fixed order (run to run identical). */
int dg_mlp_train(dg_ctx* ctx, const float* x, const float* y, int64_t n, const dg_train_opts* opts, double* loss_out);
/* Loss and gradient of one batch (n <= 4096) at the current parameters;
 * grad is a device array of dg_av_param_count floats. */
int dg_mlp_grad(dg_ctx* ctx, const float* x, const float* y, int64_t n, float* grad, double* loss);
/* Network output y for explicit inputs (device x [n][2b] -> y [n]), using the
 * BF16 inference kernel of the learned mode. */
int dg_mlp_forward(dg_ctx* ctx, const float* x, int64_t n, float* y);
/* Per-cell coefficient nu of the current state (device float [N^3]),
 * evaluated by the separate inference kernel. */
int dg_av_nu(dg_ctx* ctx, float* nu_out);
/* The coefficient the next dg_step will use for the current state, as the
 * previous learned step left it (device float [N^3]): evaluated by its last
 * stage (fused_infer), else by the inference kernel from the |v| projection
 * that the last stage carried over.
 * DG_ESTATE when none is carried: no successful learned-mode dg_step yet, or
 * a call since then that sets the state, the forcing, the parameters or the
 * network, or runs dg_rhs, dg_diagnostics or the network entry points.
 * Leaves the context unchanged. */
int dg_av_nu_carried(dg_ctx* ctx, float* nu_out);

/* Kernel timing: with profiling on, every launch of the library is bracketed
 * by CUDA events on the context's stream and its duration accumulated per
 * kernel family (read back after the stream is synchronised).  Launch counts
 * are kept whether or not profiling is on. */
typedef struct {
    int64_t launches;      /* kernels launched since the last reset               */
    int64_t n_project, n_rhs, n_force, n_other;
    double ms_project;     /* projection kernel (K_A)                             */
    double ms_rhs;         /* RHS + stage update kernel (K_B)                     */
    double ms_force;       /* forcing projection                                  */
    double ms_other;       /* diagnostics, L1                                     */
    /* volume-term tiles (16 consecutive cells each) the stage kernels ran since
     * the last reset, and those among them that skipped div v and the viscous
     * pressure because every cell's coefficient was zero (DG_AV_LEARNED with
     * nu_gate, or DG_AV_OFF); counted whether or not profiling is on */
    int64_t tiles_volume, tiles_gated;
} dg_prof;
int dg_profile(dg_ctx* ctx, int enable);          /* enable/disable; resets counts */
int dg_profile_read(dg_ctx* ctx, dg_prof* out);   /* synchronises the stream       */

/* Checkpoint metadata (coefficients via dg_get_state / dg_set_state). */
int dg_get_meta(dg_ctx* ctx, dg_meta* out);
int dg_set_meta(dg_ctx* ctx, const dg_meta* in);

/* Right-hand side without any allocation, for callers that cannot allocate
 * device memory: their device memory is all held by their own pool (a
 * framework's caching allocator), or they must not call cudaMalloc/cudaFree
 * after start-up because those calls can synchronise the device and stall
 * every stream.  The paper has no counterpart; this is a service of the
 * library.  Computes the same quantity as dg_rhs (single evaluation of the
 * weak-form right-hand side, same layouts and element types; dudt and u_in
 * are device buffers, ahat a device buffer or NULL) without a context: the
 * caller passes only inputs, outputs and a stream.  The working memory
 * (control block, reduction partials, basis tables, projected velocity)
 * lives in one fixed 64 MiB device array of the library, held by every GPU
 * that loads it until the process exits.  Limit: N^3 * 3 * b * element size
 * plus a 1,180,160-byte head must fit in 64 MiB (N <= 65 at k = 3 in FP32,
 * N <= 51 in FP64); larger meshes return DG_ENOMEM and nothing runs.  Artificial
 * viscosity modes DG_AV_OFF and DG_AV_VNR only, no diffusion operator (nu->diffusion
 * must be 0), Rusanov face fluxes only (it equals dg_rhs of a context created
 * with riemann = DG_RIEMANN_RUSANOV).  Every call looks up the array's device
 * address (cudaGetSymbolAddress, a host-side query); the first call for a
 * given order and precision at that address uploads the tables (again after a
 * device reset): make that first call before any stream capture.  All calls share the array and it keeps the
 * last call's contents; its control block is cleared at every call.  Calls
 * whose GPU work overlaps (other streams, other host threads) race on the
 * array and must be serialised.  Work is enqueued on `stream` (a
 * cudaStream_t); the call does not synchronise.  Errors are also printed to
 * stderr (there is no context to hold them). */
int dg_rhs_noalloc(const dg_mesh* mesh, int order, double cs, const dg_nu_params* nu, int precision,
                   const void* u_in, const void* ahat, void* dudt, double dt_for_pimax, void* stream);

/* ---- turbulence statistics (Sec. 4.1 definitions, Sec. 4.3 measurement) ----
 * Of the current state.  Evaluated in FP64 from the state's coefficients and
 * accumulated in FP64 with atomics: the summation order, and with it the last
 * bits, may vary between calls.  nbins in [1, DG_MAX_BINS].  Each call
 * synchronises the context's stream.  Errors: DG_EINVAL (arguments),
 * DG_ESTATE (no state), DG_ECUDA. */
#define DG_MAX_BINS 2000

/* Volume-weighted PDF of s = log10(rho / rho_mean): hist[i] (host, nbins) is
 * the volume fraction with s in [lo + i ds, lo + (i+1) ds), ds = (hi-lo)/nbins,
 * sampled at the Gauss points of every cell with their weights (the paper bins
 * log density over slices; this uses the whole volume). */
int dg_density_pdf(dg_ctx* ctx, double lo, double hi, int nbins, double* hist);

/* Second-order velocity structure function v(l) = (1/2 <|v(x) - v(x+l)|^2>)^(1/2)
 * (Sec. 4.1) on nbins logarithmic bins between 1/((k+1)N) and 1/2: bin j uses
 * l_j = l_min (l_max/l_min)^((j+1/2)/nbins) and npairs random pairs.  Pair p of
 * bin j takes the SplitMix64 numbers n = (j npairs + p) 5 + r, r = 0..4, of
 * `seed` (n-th output of the generator started at state `seed`, top 53 bits as
 * u in [0,1)): x = (u0, u1, u2), cos(theta) = 2 u3 - 1, phi = 2 pi u4, partner
 * x + l_j (sin theta cos phi, sin theta sin phi, cos theta) wrapped into the box;
 * v = m/rho from the expansions of the cells the points fall in.  l, v: host
 * arrays of nbins. */
int dg_structure_function(dg_ctx* ctx, int nbins, int64_t npairs, uint64_t seed, double* l, double* v);

/* Bytes of the device work buffer dg_power_spectrum needs: the velocity on the
 * Ng = (k+1)N grid (Ng^3 doubles) and its real-to-complex transform
 * (Ng^2 (Ng/2+1) complex doubles). */
int dg_analysis_bytes(const dg_mesh* mesh, int order, size_t* bytes);

/* Velocity power spectrum (Sec. 4.1, Sec. 4.3): v sampled at x_g = (g+1/2)/Ng
 * (k+1 points inside every cell per axis), v_hat = FFT(v)/Ng^3 per component
 * (cuFFT, loaded at run time; its plan holds its own work area), summed over
 * integer wave vectors kappa != 0 in logarithmic shells
 * i = floor(log|kappa| / log(sqrt(3) Ng/2) nbins) (capped at nbins-1).
 * kmean[i] = mean |kappa|, power[i] = sum of |v_hat_x|^2+|v_hat_y|^2+|v_hat_z|^2,
 * count[i] = number of kappa (host arrays of nbins).  E(k) is power / bin
 * width; the powers add up to the variance of the sampled velocity.
 * work: device buffer of dg_analysis_bytes(), 256-byte aligned. */
int dg_power_spectrum(dg_ctx* ctx, void* work, size_t work_bytes, int nbins, double* kmean, double* power,
                      int64_t* count);

/* ---- adiabatic system (Sec. 2.1) -----------------------------------------
 * Five conserved variables per cell, u[cell][var][mode] with var = (rho,
 * m_x, m_y, m_z, e), e the total energy density; ideal-gas equation of state
 * p = (gamma - 1)(e - |m|^2/(2 rho)); flux F_d = (m_d, m v_d + p e_d,
 * (e + p) v_d).  Same mesh, basis, quadrature, SSP-RK schemes and CFL rule
 * as the isothermal context, with the local sound speed c = sqrt(gamma p /
 * rho) in the CFL bound sum_d(|v_d| + c) and in the bulk term of the vNR
 * viscous pressure, which is added to p in the momentum and energy fluxes at
 * the volume points (Sec. 3.1).  Face states: rho from its own expansion, v
 * and p from their Gauss projections (Sec. 3.2); Rusanov flux with lambda =
 * max(|v_n| + c), or HLLC (opts->riemann).  Positivity after every stage:
 * density and pressure at all volume and face points at or above
 * nu->rho_floor (the floor of both); the
 * higher modes of all five variables are scaled by theta_rho theta_p toward
 * the cell mean (theta_p the largest factor keeping p at the floor, from the
 * quadratic in theta); a cell mean at or below the floor fails the step,
 * which is retried with dt/2 up to three times.  FP32 or FP64 (no x3, no
 * learned sensor, no diffusion: DG_EINVAL). */
typedef struct dg_adi_ctx dg_adi_ctx;
typedef struct {
    int32_t precision;     /* DG_PREC_F32 or DG_PREC_F64                          */
    int32_t rk_stages;     /* 2 or 3; stage weights as for dg_opts.rk_stages      */
    double cfl;            /* dt = cfl h / ((k+1) max sum_d(|v_d| + c))           */
    double gamma;          /* adiabatic index, > 1                                */
    void* stream;          /* cudaStream_t; must not be NULL                      */
    void* u[3];            /* three state registers of N^3*5*b elements           */
    void* prim;            /* N^3*4*b elements: projections of v_x, v_y, v_z, p   */
    void* scratch;         /* >= scratch bytes of dg_adi_buffer_bytes, 256-aligned */
    size_t scratch_bytes;
    int32_t riemann;       /* DG_RIEMANN_RUSANOV (0, default) or DG_RIEMANN_HLLC:
                              HLLC of the Euler equations (Davis bounds, contact
                              speed and star states); DG_RIEMANN_HLL: DG_EINVAL */
    int32_t bc[3];         /* per axis DG_BC_*; DG_BC_PERIODIC (0) when
                              zero-initialised                                    */
    double inflow[5];      /* DG_BC_INFLOW: rho, v_x, v_y, v_z, p at the face at
                              coordinate 0 (rho > 0, p > 0)                      */
} dg_adi_opts;

/* Boundaries of the adiabatic system along an axis (its faces at coordinates 0
 * and 1; the paper's Shu-Osher and implosion problems, Sec. 3.1, run between
 * them): the Riemann flux of such a face takes the cell's own trace and a
 * ghost state -- the same trace (outflow, zero gradient), the same trace with
 * the normal velocity negated (reflective wall: no mass or energy crosses), or
 * the prescribed state inflow at the face at 0 with an outflow at 1. */
#define DG_BC_PERIODIC 0
#define DG_BC_OUTFLOW 1
#define DG_BC_REFLECT 2
#define DG_BC_INFLOW 3
/* Sizes in bytes of one state register, the projection buffer and the scratch
 * (null outputs skipped).  DG_EINVAL for a mesh that is not n x n x n with
 * 1 <= n <= 1024, an order outside 1..3 or a precision other than F32/F64. */
int dg_adi_buffer_bytes(const dg_mesh* mesh, int order, int precision, size_t* state_bytes, size_t* prim_bytes,
                        size_t* scratch_bytes);
/* nu: mode DG_AV_OFF or DG_AV_VNR (alpha, beta, rho_floor); the buffers are
 * caller-owned device memory that must outlive the context. */
int dg_adi_init(dg_adi_ctx** ctx, const dg_mesh* mesh, int order, const dg_nu_params* nu, const dg_adi_opts* opts);
void dg_adi_free(dg_adi_ctx* ctx);
const char* dg_adi_last_error(const dg_adi_ctx* ctx);
/* Copy a state [N^3][5][b] in (resets the time) or out; host or device memory. */
int dg_adi_set_state(dg_adi_ctx* ctx, const void* src, int src_on_host);
int dg_adi_get_state(dg_adi_ctx* ctx, void* dst, int to_host);
/* Projections of v and p of a device state into prim_out [N^3][4][b]. */
int dg_adi_project(dg_adi_ctx* ctx, const void* u_in, void* prim_out);
/* Right-hand side du/dt of a device state without the driving (dt_pimax: dt
 * of the viscous-pressure cap, 0 = uncapped); uses the context's projection
 * buffer. */
int dg_adi_rhs(dg_adi_ctx* ctx, const void* u_in, void* dudt, double dt_pimax);
/* nsteps SSP-RK steps (fixed_dt > 0 replaces the CFL dt); *t_out the time
 * since dg_adi_set_state, *dt_last the last step's dt.  Synchronises once per
 * step to read the positivity status; DG_EPOSITIVITY leaves the state at the
 * start of the failed step. */
int dg_adi_step(dg_adi_ctx* ctx, int nsteps, double fixed_dt, double* t_out, double* dt_last);
/* Driving of the adiabatic system (Sec. 4.2), the same OU process and forcing
 * projection as dg_set_forcing with the sound speed cs_ref in its time scale
 * and amplitude; the momentum source rho (a_h - abar) (abar = <rho a_h>/<rho>
 * of each stage's state) and its work m.(a_h - abar) in the energy equation.
 * The injected energy of a step is dt sum_s beta_s W_s with W_s the volume
 * integral of the energy source of stage s and beta_s its weight in u^(n+1)
 * (RK2: 1/2, 1/2; RK3: 1/6, 1/6, 2/3): exactly the change of the total energy. */
int dg_adi_set_forcing(dg_adi_ctx* ctx, const dg_forcing* f, double cs_ref);
/* cs > 0: after every step the uniform temperature p = cs^2 rho is restored (e
 * becomes the projection of rho cs^2/(gamma-1) + |m|^2/(2 rho)); with gamma
 * close to 1 this emulates the isothermal gas and the thermal energy taken out
 * measures the dissipation (Sec. 4.2).  0: off (default).
 * Energy offset: while cs > 0, the fifth variable of every state that
 * dg_adi_set_state, dg_adi_get_state, dg_adi_rhs and dg_adi_project take or give
 * is e - kap rho with kap = cs^2/(gamma - 1) (the energy relative to the
 * isothermal reference), and the pressure projection is that of p - cs^2 rho:
 * near gamma = 1 the reference is 1/(gamma - 1) times the kinetic energy, which
 * single precision would otherwise carry in every coefficient.  The scheme is
 * linear in the state, so this changes the variables, not the discretisation.
 * A state already set is carried to the new offset (e += (kap_old - kap) rho);
 * dg_adi_totals and dg_adi_energy_budget report the energy itself. */
int dg_adi_set_reset(dg_adi_ctx* ctx, double cs);
/* out[0] = injected, out[1] = dissipated energy since dg_adi_set_state. */
int dg_adi_energy_budget(dg_adi_ctx* ctx, double* out);
/* Checkpoint metadata of the adiabatic system: time, steps and the driving's
 * OU state (as dg_meta), and the energy budget of the run (Sec. 4.2).  Resume:
 * dg_adi_set_forcing (same modes) and dg_adi_set_reset as before, then
 * dg_adi_set_state (which zeroes time and budget), then dg_adi_set_meta; the
 * following steps are bit-identical to the uninterrupted run's.  set_meta
 * returns DG_EINVAL when the number of driven modes differs. */
typedef struct {
    dg_meta m;
    double injected;       /* energy injected by the driving since the start     */
    double dissipated;     /* energy taken out by the temperature reset           */
} dg_adi_meta;
int dg_adi_get_meta(dg_adi_ctx* ctx, dg_adi_meta* out);
int dg_adi_set_meta(dg_adi_ctx* ctx, const dg_adi_meta* in);
/* FP64 diagnostics of the current state: out[0..7] = mass, momentum (3),
 * total energy (integrals over the box), kinetic energy (volume quadrature of
 * |m|^2/(2 rho)), minimum density and minimum pressure at the volume points. */
int dg_adi_totals(dg_adi_ctx* ctx, double* out);

#ifdef __cplusplus
}
#endif
#endif
