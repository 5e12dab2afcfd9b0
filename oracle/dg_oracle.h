/*
 * dg_oracle.h -- plain FP64 CPU reference ("oracle") of the modal DG method
 * for 3D isothermal Euler on a periodic Cartesian mesh.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library and its binding) never calls, links or includes anything
 * here, and this file includes nothing from the product.
 *
 * Conventions (shared with the product only by specification, not by code):
 *   - N cells per axis, unit box L = 1, cell size h = 1/N.
 *   - cell index c = (iz*N + iy)*N + ix, cell centre x_c = (i + 1/2) h.
 *   - degree k, b = (k+1)(k+2)(k+3)/6 modes per field, n = k+1 Gauss points
 *     per axis.
 *   - basis phi_{ijl}(xi) = Pn_i(xi_x) Pn_j(xi_y) Pn_l(xi_z), i+j+l <= k,
 *     Pn_m = sqrt(2m+1) P_m (orthonormal: (1/8) int phi_a phi_b = delta_ab).
 *     Mode order: total degree ascending; within a degree i descending, then
 *     j descending.
 *   - state u[c][var][mode], var = (rho, m_x, m_y, m_z).
 *   - forcing / velocity coefficient arrays: [c][3][mode].
 */
#ifndef DG_ORACLE_H
#define DG_ORACLE_H
#include <stdint.h>

typedef struct {
    int32_t N;          /* cells per axis                                   */
    int32_t k;          /* polynomial degree (1..3 used, up to 6 accepted)  */
    double cs;          /* isothermal sound speed                           */
    int32_t av_mode;    /* 0 = no artificial viscosity, 1 = von Neumann-
                           Richtmyer viscous pressure                       */
    double alpha;       /* quadratic vNR coefficient                        */
    double beta;        /* linear (bulk) vNR coefficient                    */
    double rho_floor;   /* positivity floor epsilon                         */
    double cfl;         /* Courant number                                   */
    int32_t rk_stages;  /* 2 (SSP-RK2) or 3 (SSP-RK3)                        */
    int32_t riemann;    /* face flux: 0 Rusanov, 1 HLL, 2 HLLC               */
    double eps_diff;    /* diffusion coefficient of div(eps grad u), 0: off  */
    int32_t pos_mode;   /* positivity: 0 rescale the stage outputs, 1 also
                           repeat the step with troubled cells flattened
                           (orc_step_repeat)                                  */
    int32_t bc[3];      /* adiabatic system, per axis: ORC_BC_*              */
    double inflow[5];   /* ORC_BC_INFLOW: rho, v_x, v_y, v_z, p at the lower
                           face                                              */
} orc_cfg;

/* boundaries of the adiabatic system along an axis (the faces at coordinate 0
 * and 1): periodic; outflow (the ghost state is the cell's own trace);
 * reflective (the same with the normal velocity negated); inflow (the lower
 * face sees the prescribed state cfg->inflow, the upper face is an outflow) */
#define ORC_BC_PERIODIC 0
#define ORC_BC_OUTFLOW 1
#define ORC_BC_REFLECT 2
#define ORC_BC_INFLOW 3

#define ORC_RUSANOV 0
#define ORC_HLL 1
#define ORC_HLLC 2

/* status bits of a stage / step */
#define ORC_LIMITED 1   /* at least one cell was rescaled by the limiter    */
#define ORC_FAIL    2   /* a cell mean fell to or below the floor           */
#define ORC_REPEATED 4  /* the step was repeated with troubled cells
                           flattened (pos_mode 1)                            */

/* positivity by repetition (pos_mode 1): a stage output with negative density
 * at a Gauss point, or whose volume-point wave speed sum_d(|v_d| + cs) exceeds
 * ORC_REPEAT_SPEED times the bound that set dt, troubles its cell; at most
 * ORC_REPEAT_MAX attempts per step and ORC_REPEAT_HALVINGS halvings of dt */
#define ORC_REPEAT_SPEED 1.5
#define ORC_MARK_NEGATIVE 1  /* marks: rho < 0 at a point of a stage output   */
#define ORC_MARK_FAST 2      /* a point faster than the bound                */
#define ORC_REPEAT_MAX 32
#define ORC_REPEAT_HALVINGS 6

/* OU driving state (host side, Sec. 4.2) */
#define ORC_MAX_MODES 512
typedef struct {
    int32_t nmodes;
    int32_t kvec[ORC_MAX_MODES][3];
    double x[ORC_MAX_MODES][3][2];     /* OU variables, real/imag           */
    double zeta, sigma, tc, dt_drive, s, f;
    double t_next, t_off;
    uint64_t rng;                      /* SplitMix64 state                  */
    int32_t have_spare; double spare;  /* Box-Muller second branch          */
    int32_t on;                        /* 0 once switched off at t_off      */
    int32_t dirty;                     /* forcing needs re-projection       */
} orc_ou;

int  orc_nmodes(int k);
void orc_mode_list(int k, int32_t* ijl);
void orc_gauss(int n, double* x, double* w);
double orc_legendre(int m, double x);
double orc_legendre_deriv(int m, double x);

double orc_dt(const orc_cfg* cfg, const double* u);
double orc_recover_dn(int K, const double* cL, const double* cR);
void orc_diffusion_rhs(const orc_cfg* cfg, const double* u, double* dudt);
void orc_project_velocity(const orc_cfg* cfg, const double* u, double* vhat);
void orc_forcing_mean(const orc_cfg* cfg, const double* u, const double* ahat,
                      double abar[3]);
double orc_vnr(const orc_cfg* cfg, double rho, double divv, double dt);
void orc_rusanov(double cs, int d, const double WL[4], const double WR[4],
                 double F[4]);
void orc_hll(double cs, int d, const double WL[4], const double WR[4], double F[4]);
void orc_hllc(double cs, int d, const double WL[4], const double WR[4], double F[4]);
void orc_riemann(int solver, double cs, int d, const double WL[4], const double WR[4],
                 double F[4]);
int orc_rhs(const orc_cfg* cfg, const double* u, const double* ahat,
            double dt_pimax, double* dudt);
int orc_limit(const orc_cfg* cfg, double* u);
double orc_pi_nu(const orc_cfg* cfg, double rho, double divv, double nu, double dt);
int orc_rhs_nu(const orc_cfg* cfg, const double* u, const double* ahat, double dt_pimax, const double* nu_cell,
               double* dudt);
/* adiabatic system: state [c][5][b] (rho, m, e), primitives [c][4][b] (v, p) */
void orc_adi_flux(double gamma, int d, const double U[5], double F[5]);
void orc_adi_rusanov(double gamma, int d, const double WL[5], const double WR[5], double F[5]);
void orc_adi_hllc(double gamma, int d, const double WL[5], const double WR[5], double F[5]);
double orc_adi_vnr(const orc_cfg* cfg, double rho, double c, double divv, double dt);
void orc_adi_project(const orc_cfg* cfg, double gamma, const double* u, double* prim);
int orc_adi_rhs(const orc_cfg* cfg, double gamma, const double* u, double dt_pimax, double* dudt);
double orc_adi_dt(const orc_cfg* cfg, double gamma, const double* u);
int orc_adi_limit(const orc_cfg* cfg, double gamma, double* u);
int orc_adi_step(const orc_cfg* cfg, double gamma, double* u, double dt);
int orc_adi_run(const orc_cfg* cfg, double gamma, double* u, int nsteps, double fixed_dt, double* t,
                double* dt_last);
int orc_adi_rhs_forced(const orc_cfg* cfg, double gamma, const double* u, const double* ahat, double dt_pimax,
                       double* dudt, double* work);
int orc_adi_step_forced(const orc_cfg* cfg, double gamma, double* u, const double* ahat, double dt,
                        double* injected);
double orc_adi_reset(const orc_cfg* cfg, double gamma, double cs, double* u);
int orc_rhs_local(const orc_cfg* cfg, const double* patch, const double* ahat_c, const double abar[3],
                  double dt_pimax, const double* nu, int64_t n, double* out);
void orc_av_features(const orc_cfg* cfg, const double* u, double dt, double* x, double* y);
int orc_step(const orc_cfg* cfg, double* u, const double* ahat, double dt);
int orc_step_flags(const orc_cfg* cfg, double* u, const double* ahat, double dt, double vlim, uint8_t* flag);
double orc_speed_bound(const orc_cfg* cfg, const double* u);
int orc_step_repeat(const orc_cfg* cfg, double* u, const double* ahat, double fixed_dt, double* dt_used,
                    int* attempts, uint8_t* level);

/* turbulence statistics (Sec. 4.1 structure function and power spectrum,
 * Sec. 4.3 density PDF) */
void orc_density_pdf(const orc_cfg* cfg, const double* u, double lo, double hi, int nbins, double* hist);
void orc_structure_function(const orc_cfg* cfg, const double* u, int nbins, int64_t npairs, uint64_t seed,
                            double* l_out, double* v_out);
void orc_sample_velocity(const orc_cfg* cfg, const double* u, double* v_out);
double orc_velocity_at(const orc_cfg* cfg, const double* u, const double x[3], double v[3]);

void orc_ou_init(orc_ou* ou, int kmin2, int kmax2, double zeta, double mach,
                 double cs, double L, uint64_t seed, double t_off);
void orc_ou_advance(orc_ou* ou);
/* driven adiabatic run with the isothermal reset (cs > 0) after every step;
 * accumulates the injected and dissipated energies */
int orc_adi_run_driven(const orc_cfg* cfg, double gamma, double cs, double* u, orc_ou* ou, int use_forcing,
                       double* ahat, int nsteps, double fixed_dt, double* t, double* dt_last, double* injected,
                       double* dissipated);
void orc_ou_amplitudes(const orc_ou* ou, double* ahat_modes /* [nm][3][2] */);
void orc_forcing_project(const orc_cfg* cfg, int nmodes, const int32_t* kvec,
                         const double* amp, double* ahat);
int orc_run(const orc_cfg* cfg, double* u, orc_ou* ou, int use_forcing,
            double* ahat, int nsteps, double* t, double* dt_last);

void orc_diagnostics(const orc_cfg* cfg, const double* u, const double* ahat,
                     double dt, double* out /* ORC_NDIAG */);
#define ORC_NDIAG 13
double orc_l1_density(const orc_cfg* cfg, const double* uA, const double* uB);

uint64_t orc_splitmix64(uint64_t* state);
/* threads of the parallel loops (OpenMP over cells; the interface loop in
 * parity colours): n > 0 sets it; returns the number in use.  Results do not
 * depend on it. */
int orc_set_threads(int n);

#endif
