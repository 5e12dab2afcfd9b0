/*
 * dg_oracle.c -- plain, slow, FP64 CPU reference of the modal Discontinuous
 * Galerkin method of Cernetic, Springel, Guillet & Pakmor (2024), specialised
 * to isothermal Euler (p = cs^2 rho) as used for driven supersonic turbulence.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark.  It shares no code, table or header with
 * the CUDA library and must stay that way.
 *
 * Everything here follows the paper's definitions one step at a time:
 *   - basis expansion and orthonormality ............ Sec. 2.1, eq. (state_vector_expansion)
 *   - weak form / weight evolution ................. Sec. 2.2, eqs. (weakform), (weight_evolution)
 *   - Gauss quadrature with (k+1) points per axis ... Sec. 2.2 and Sec. 7 (v_k, s_k)
 *   - von Neumann-Richtmyer viscous pressure ........ Sec. 3.1 (quadratic + linear term, Pi_max)
 *   - positivity check and rescaling ............... Sec. 3.1, last paragraph before 3.1.1
 *   - step repetition with troubled cells flattened . the same paragraph (orc_step_repeat)
 *   - primitive-variable projection ................ Sec. 3.2, eq. (weights_equation)
 *   - Ornstein-Uhlenbeck driving ................... Sec. 4.2, eqs. (ornstein_uhlenbeck...), (eddy_turnover_time)
 *   - SSP Runge-Kutta stages and dt ~ h/(k+1) ....... Sec. 7
 * Basis values and derivatives are evaluated directly (product of 1D
 * Legendre values) at every point; no sum factorisation, no modal
 * differentiation, no batching.  Readings where the paper is silent are the
 * ones documented with the library (isothermal EOS, Rusanov flux, quotient-rule
 * divergence, CFL formula, OU normalisation, SplitMix64 + Box-Muller).
 */
#include "dg_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* 1D building blocks                                                        */
/* ------------------------------------------------------------------------ */

/* Legendre P_m(x) by Bonnet's recurrence (m+1)P_{m+1} = (2m+1) x P_m - m P_{m-1}. */
double orc_legendre(int m, double x)
{
    if (m == 0) return 1.0;
    double p0 = 1.0, p1 = x;
    for (int j = 1; j < m; ++j) {
        double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

/* P'_m(x) from P'_{j+1} = P'_{j-1} + (2j+1) P_j (valid on the closed interval). */
double orc_legendre_deriv(int m, double x)
{
    if (m == 0) return 0.0;
    if (m == 1) return 1.0;
    double dm1 = 0.0, d0 = 1.0; /* P'_0, P'_1 */
    for (int j = 1; j < m; ++j) {
        double d = dm1 + (2.0 * j + 1.0) * orc_legendre(j, x);
        dm1 = d0;
        d0 = d;
    }
    return d0;
}

/* normalised Legendre sqrt(2m+1) P_m: (1/2) int_{-1}^{1} Pn_a Pn_b = delta_ab */
static double pn(int m, double x) { return sqrt(2.0 * m + 1.0) * orc_legendre(m, x); }
static double dpn(int m, double x) { return sqrt(2.0 * m + 1.0) * orc_legendre_deriv(m, x); }

/* Gauss-Legendre nodes (ascending) and weights: Newton iteration on P_n. */
void orc_gauss(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double dz = orc_legendre(n, z) / orc_legendre_deriv(n, z);
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        double dp = orc_legendre_deriv(n, z);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

int orc_nmodes(int k) { return (k + 1) * (k + 2) * (k + 3) / 6; }

/* complete P_k set: total degree ascending, then i descending, then j descending */
void orc_mode_list(int k, int32_t* ijl)
{
    int c = 0;
    for (int d = 0; d <= k; ++d)
        for (int i = d; i >= 0; --i)
            for (int j = d - i; j >= 0; --j) {
                ijl[3 * c + 0] = i;
                ijl[3 * c + 1] = j;
                ijl[3 * c + 2] = d - i - j;
                ++c;
            }
}

/* ------------------------------------------------------------------------ */
/* per-call tables of basis values at the quadrature points                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int k, b, n, nq, ns;
    int32_t ijl[3 * 84];
    double xg[16], wg[16];
    double* phi;  /* [nq][b]             phi_l(xi_q)                          */
    double* dphi; /* [3][nq][b]          d phi_l / d xi_d at xi_q              */
    double* wq;   /* [nq]                w_a w_b w_c                           */
    double* phif; /* [3][2][ns][b]       phi_l on face (dir d, side 0:-1, 1:+1) */
    double* ws;   /* [ns]                face weights                          */
} tabs;

static double basis(const tabs* T, int l, const double xi[3])
{
    return pn(T->ijl[3 * l], xi[0]) * pn(T->ijl[3 * l + 1], xi[1]) * pn(T->ijl[3 * l + 2], xi[2]);
}

static double basis_grad(const tabs* T, int l, int d, const double xi[3])
{
    double f[3];
    for (int e = 0; e < 3; ++e) f[e] = (e == d) ? dpn(T->ijl[3 * l + e], xi[e]) : pn(T->ijl[3 * l + e], xi[e]);
    return f[0] * f[1] * f[2];
}

/* volume point q = a + n (b + n c) sits at (xg[a], xg[b], xg[c]) */
static void vol_point(const tabs* T, int q, double xi[3])
{
    int n = T->n;
    xi[0] = T->xg[q % n];
    xi[1] = T->xg[(q / n) % n];
    xi[2] = T->xg[q / (n * n)];
}

/* face point s = a + n b on the face normal to d: tangential axes in increasing order */
static void face_point(const tabs* T, int d, int side, int s, double xi[3])
{
    int n = T->n, t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
    xi[d] = side ? 1.0 : -1.0;
    xi[t1] = T->xg[s % n];
    xi[t2] = T->xg[s / n];
}

static void tabs_init(tabs* T, int k, int nquad)
{
    T->k = k;
    T->b = orc_nmodes(k);
    T->n = nquad;
    T->nq = nquad * nquad * nquad;
    T->ns = nquad * nquad;
    orc_mode_list(k, T->ijl);
    orc_gauss(nquad, T->xg, T->wg);
    int b = T->b, nq = T->nq, ns = T->ns;
    T->phi = (double*)malloc(sizeof(double) * nq * b);
    T->dphi = (double*)malloc(sizeof(double) * 3 * nq * b);
    T->wq = (double*)malloc(sizeof(double) * nq);
    T->phif = (double*)malloc(sizeof(double) * 6 * ns * b);
    T->ws = (double*)malloc(sizeof(double) * ns);
    for (int q = 0; q < nq; ++q) {
        double xi[3];
        vol_point(T, q, xi);
        int n = T->n;
        T->wq[q] = T->wg[q % n] * T->wg[(q / n) % n] * T->wg[q / (n * n)];
        for (int l = 0; l < b; ++l) {
            T->phi[q * b + l] = basis(T, l, xi);
            for (int d = 0; d < 3; ++d) T->dphi[(d * nq + q) * b + l] = basis_grad(T, l, d, xi);
        }
    }
    for (int s = 0; s < ns; ++s) T->ws[s] = T->wg[s % T->n] * T->wg[s / T->n];
    for (int d = 0; d < 3; ++d)
        for (int side = 0; side < 2; ++side)
            for (int s = 0; s < ns; ++s) {
                double xi[3];
                face_point(T, d, side, s, xi);
                for (int l = 0; l < b; ++l) T->phif[((d * 2 + side) * ns + s) * b + l] = basis(T, l, xi);
            }
}

static void tabs_free(tabs* T)
{
    free(T->phi);
    free(T->dphi);
    free(T->wq);
    free(T->phif);
    free(T->ws);
}

static double eval(const tabs* T, const double* coef, const double* row)
{
    double s = 0.0;
    for (int l = 0; l < T->b; ++l) s += coef[l] * row[l];
    return s;
}

static int cell_index(int N, int ix, int iy, int iz)
{
    ix = (ix % N + N) % N;
    iy = (iy % N + N) % N;
    iz = (iz % N + N) % N;
    return (iz * N + iy) * N + ix;
}

/* ------------------------------------------------------------------------ */
/* pointwise physics                                                         */
/* ------------------------------------------------------------------------ */

/* von Neumann-Richtmyer viscous pressure (Sec. 3.1): for div v < 0,
 *   Pi = alpha rho (h/p)^2 |div v|^2 + beta rho cs (h/p) |div v|,
 * limited by Pi_max = (1/2) rho (h/p)^2 |div v| / dt with dt fixed at the start
 * of the step; zero for div v >= 0.  p = k+1.  dt <= 0 disables the limit. */
double orc_vnr(const orc_cfg* cfg, double rho, double divv, double dt)
{
    if (cfg->av_mode != 1 || !(divv < 0.0)) return 0.0;
    double hp = (1.0 / cfg->N) / (cfg->k + 1);
    double a = -divv;
    double Pi = cfg->alpha * rho * hp * hp * a * a + cfg->beta * rho * cfg->cs * hp * a;
    if (dt > 0.0) {
        double Pmax = 0.5 * rho * hp * hp * a / dt;
        if (Pi > Pmax) Pi = Pmax;
    }
    return Pi;
}

/* Rusanov (local Lax-Friedrichs) flux along +e_d between a left state and a
 * right state given in primitive form W = (rho, vx, vy, vz):
 *   F* = (F_d(U_L) + F_d(U_R))/2 - lambda (U_R - U_L)/2,
 *   lambda = max(|v_d^L|, |v_d^R|) + cs,
 *   F_d(U) = (rho v_d, rho v_i v_d + cs^2 rho delta_id),  U = (rho, rho v). */
void orc_rusanov(double cs, int d, const double WL[4], const double WR[4], double F[4])
{
    double UL[4], UR[4], FL[4], FR[4];
    UL[0] = WL[0];
    UR[0] = WR[0];
    for (int i = 0; i < 3; ++i) {
        UL[1 + i] = WL[0] * WL[1 + i];
        UR[1 + i] = WR[0] * WR[1 + i];
    }
    FL[0] = UL[1 + d];
    FR[0] = UR[1 + d];
    for (int i = 0; i < 3; ++i) {
        FL[1 + i] = UL[1 + i] * WL[1 + d] + (i == d ? cs * cs * WL[0] : 0.0);
        FR[1 + i] = UR[1 + i] * WR[1 + d] + (i == d ? cs * cs * WR[0] : 0.0);
    }
    double lam = fmax(fabs(WL[1 + d]), fabs(WR[1 + d])) + cs;
    for (int v = 0; v < 4; ++v) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * lam * (UR[v] - UL[v]);
}

/* Conserved state and flux along e_d of a primitive state W = (rho, v). */
static void cons_flux(double cs, int d, const double W[4], double U[4], double F[4])
{
    U[0] = W[0];
    for (int i = 0; i < 3; ++i) U[1 + i] = W[0] * W[1 + i];
    F[0] = U[1 + d];
    for (int i = 0; i < 3; ++i) F[1 + i] = U[1 + i] * W[1 + d] + (i == d ? cs * cs * W[0] : 0.0);
}

/* HLL flux along +e_d (Harten, Lax & van Leer; Toro, Riemann Solvers, ch. 10).
 * The isothermal signal speeds are bounded by the Davis estimates
 *   S_L = min(v_d^L, v_d^R) - cs,   S_R = max(v_d^L, v_d^R) + cs,
 * and the flux is F_L for S_L >= 0, F_R for S_R <= 0, otherwise the flux of
 * the single averaged state between the two waves,
 *   F* = (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L). */
void orc_hll(double cs, int d, const double WL[4], const double WR[4], double F[4])
{
    double UL[4], UR[4], FL[4], FR[4];
    cons_flux(cs, d, WL, UL, FL);
    cons_flux(cs, d, WR, UR, FR);
    const double SL = fmin(WL[1 + d], WR[1 + d]) - cs;
    const double SR = fmax(WL[1 + d], WR[1 + d]) + cs;
    for (int v = 0; v < 4; ++v) {
        if (SL >= 0.0)
            F[v] = FL[v];
        else if (SR <= 0.0)
            F[v] = FR[v];
        else
            F[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) / (SR - SL);
    }
}

/* HLLC flux along +e_d for the isothermal system (Toro's HLLC with p = cs^2 rho,
 * the scheme the paper uses on faces, Sec. 2).  With the HLL speeds S_L, S_R,
 * the star region holds two states separated by the contact wave
 * S_M = m_d* / rho*.  Pressure continuity across the contact makes the density
 * the same on both sides, so rho* and m_d* are the HLL averages
 *   U_hll = (S_R U_R - S_L U_L - (F_R - F_L)) / (S_R - S_L),
 * and each star state carries the tangential velocity of its own side:
 *   U*_K = (rho*, m_d*, rho* v_t^K).
 * The flux is F_L (S_L >= 0), F*_L = F_L + S_L (U*_L - U_L) (S_L < 0 <= S_M),
 * F*_R = F_R + S_R (U*_R - U_R) (S_M < 0 < S_R), F_R (S_R <= 0). */
void orc_hllc(double cs, int d, const double WL[4], const double WR[4], double F[4])
{
    double UL[4], UR[4], FL[4], FR[4];
    cons_flux(cs, d, WL, UL, FL);
    cons_flux(cs, d, WR, UR, FR);
    const double SL = fmin(WL[1 + d], WR[1 + d]) - cs;
    const double SR = fmax(WL[1 + d], WR[1 + d]) + cs;
    if (SL >= 0.0) {
        for (int v = 0; v < 4; ++v) F[v] = FL[v];
        return;
    }
    if (SR <= 0.0) {
        for (int v = 0; v < 4; ++v) F[v] = FR[v];
        return;
    }
    const double rs = (SR * UR[0] - SL * UL[0] - (FR[0] - FL[0])) / (SR - SL);
    const double ms = (SR * UR[1 + d] - SL * UL[1 + d] - (FR[1 + d] - FL[1 + d])) / (SR - SL);
    const double SM = ms / rs;
    const int left = SM >= 0.0;
    const double* W = left ? WL : WR;
    const double* U = left ? UL : UR;
    const double* FK = left ? FL : FR;
    const double SK = left ? SL : SR;
    double Us[4];
    Us[0] = rs;
    for (int i = 0; i < 3; ++i) Us[1 + i] = (i == d) ? ms : rs * W[1 + i];
    for (int v = 0; v < 4; ++v) F[v] = FK[v] + SK * (Us[v] - U[v]);
}

void orc_riemann(int solver, double cs, int d, const double WL[4], const double WR[4], double F[4])
{
    if (solver == ORC_HLL)
        orc_hll(cs, d, WL, WR, F);
    else if (solver == ORC_HLLC)
        orc_hllc(cs, d, WL, WR, F);
    else
        orc_rusanov(cs, d, WL, WR, F);
}

/* ------------------------------------------------------------------------ */
/* CFL time step (Sec. 7: dt proportional to h/(k+1))                        */
/*   dt = cfl h / ((k+1) max_{cells, volume points} sum_d (|v_d| + cs))     */
/* ------------------------------------------------------------------------ */
/* sum_d(|v_d| + cs) at volume point q of cell uc */
static double point_speed(const tabs* T, const orc_cfg* cfg, const double* uc, int q)
{
    const int b = T->b;
    double rho = eval(T, uc, T->phi + q * b), s = 0.0;
    for (int d = 0; d < 3; ++d) s += fabs(eval(T, uc + (1 + d) * b, T->phi + q * b) / rho) + cfg->cs;
    return s;
}

/* S = max over cells and volume points of sum_d(|v_d| + cs) */
double orc_speed_bound(const orc_cfg* cfg, const double* u)
{
    tabs T;
    tabs_init(&T, cfg->k, cfg->k + 1);
    int N = cfg->N, b = T.b, nc = N * N * N;
    double smax = 0.0;
#pragma omp parallel for schedule(static) reduction(max : smax)
    for (int c = 0; c < nc; ++c) {
        const double* uc = u + (size_t)c * 4 * b;
        for (int q = 0; q < T.nq; ++q) {
            double s = point_speed(&T, cfg, uc, q);
            if (s > smax) smax = s;
        }
    }
    tabs_free(&T);
    return smax;
}

double orc_dt(const orc_cfg* cfg, const double* u)
{
    int N = cfg->N;
    double smax = orc_speed_bound(cfg, u);
    double dt = cfg->cfl * (1.0 / N) / ((cfg->k + 1) * smax);
    if (cfg->eps_diff > 0.0) {
        /* explicit diffusion: dt <= cfl (h/(k+1))^2 / (2 eps) */
        const double hp = (1.0 / N) / (cfg->k + 1), dd = cfg->cfl * hp * hp / (2.0 * cfg->eps_diff);
        if (dd < dt) dt = dd;
    }
    return dt;
}

/* ------------------------------------------------------------------------ */
/* primitive projection (Sec. 3.2, eq. weights_equation):                    */
/*   vhat_l = (1/|K|) int_K (m/rho) phi_l dV  by (k+1)^3-point Gauss         */
/* ------------------------------------------------------------------------ */
/* projection of one cell's velocity: vc[i][l] = (1/8) sum_q w_q phi_l(xi_q) m_i/rho */
static void project_cell(const tabs* T, const double* uc, double* vc)
{
    int b = T->b;
    memset(vc, 0, sizeof(double) * 3 * b);
    for (int q = 0; q < T->nq; ++q) {
        const double* ph = T->phi + q * b;
        double rho = eval(T, uc, ph);
        for (int i = 0; i < 3; ++i) {
            double vq = eval(T, uc + (1 + i) * b, ph) / rho;
            for (int l = 0; l < b; ++l) vc[i * b + l] += 0.125 * T->wq[q] * ph[l] * vq;
        }
    }
}

void orc_project_velocity(const orc_cfg* cfg, const double* u, double* vhat)
{
    tabs T;
    tabs_init(&T, cfg->k, cfg->k + 1);
    int N = cfg->N, b = T.b, nc = N * N * N;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nc; ++c) project_cell(&T, u + (size_t)c * 4 * b, vhat + (size_t)c * 3 * b);
    tabs_free(&T);
}

/* mean acceleration abar = <rho a_h> / <rho>, removed so that the forcing adds
 * no net momentum (both averages are volume integrals by quadrature). */
static void forcing_mean_nv(const orc_cfg* cfg, const double* u, int nv, const double* ahat, double abar[3]);

void orc_forcing_mean(const orc_cfg* cfg, const double* u, const double* ahat, double abar[3])
{
    forcing_mean_nv(cfg, u, 4, ahat, abar);
}

/* the same for a state of nv variables per cell (rho first) */
static void forcing_mean_nv(const orc_cfg* cfg, const double* u, int nv, const double* ahat, double abar[3])
{
    tabs T;
    tabs_init(&T, cfg->k, cfg->k + 1);
    int N = cfg->N, b = T.b, nc = N * N * N;
    /* sums over 64 fixed blocks of cells, added in block order: the same
     * result for any number of threads */
    enum { NBLK = 64 };
    double part[NBLK][4];
#pragma omp parallel for schedule(static)
    for (int blk = 0; blk < NBLK; ++blk) {
        double acc[4] = {0, 0, 0, 0};
        for (int c = (int)((long)nc * blk / NBLK); c < (int)((long)nc * (blk + 1) / NBLK); ++c) {
            const double* uc = u + (size_t)c * nv * b;
            const double* ac = ahat + (size_t)c * 3 * b;
            for (int q = 0; q < T.nq; ++q) {
                const double* ph = T.phi + q * b;
                double rho = eval(&T, uc, ph);
                acc[3] += 0.125 * T.wq[q] * rho;
                for (int i = 0; i < 3; ++i) acc[i] += 0.125 * T.wq[q] * rho * eval(&T, ac + i * b, ph);
            }
        }
        for (int i = 0; i < 4; ++i) part[blk][i] = acc[i];
    }
    double num[3] = {0, 0, 0}, den = 0.0;
    for (int blk = 0; blk < NBLK; ++blk) {
        for (int i = 0; i < 3; ++i) num[i] += part[blk][i];
        den += part[blk][3];
    }
    for (int i = 0; i < 3; ++i) abar[i] = num[i] / den;
    tabs_free(&T);
}

/* ------------------------------------------------------------------------ */
/* right-hand side (Sec. 2.2, eq. weight_evolution, |K| = h^3):              */
/*   dw_l/dt = 1/(4h) [ sum_q w_q sum_d dphi_l/dxi_d F_d(U_q)                 */
/*                      - sum_faces sum_s w_s phi_l(xi_s) F*.n_out ]          */
/*             + (1/8) sum_q w_q phi_l rho_q (a_h(xi_q) - abar)   (momentum)  */
/* Volume: conserved values at the internal points, Pi added to the pressure */
/* (Sec. 3.1).  Faces: rho from its own expansion, v from the projected      */
/* velocity, no viscous pressure (Sec. 3.1, 3.2).                            */
/* ------------------------------------------------------------------------ */
static int rhs_impl(const orc_cfg* cfg, const double* u, const double* ahat, double dt_pimax, const double* nu_cell,
                    double* dudt);

int orc_rhs(const orc_cfg* cfg, const double* u, const double* ahat, double dt_pimax, double* dudt)
{
    return rhs_impl(cfg, u, ahat, dt_pimax, NULL, dudt);
}

/* Viscous pressure with a per-cell coefficient nu (av_mode 2, the learned
 * sensor): Pi = rho nu |div v| for div v < 0, with the same cap
 * Pi_max = (1/2) rho (h/p)^2 |div v| / dt as the vNR form (Sec. 3.1). */
double orc_pi_nu(const orc_cfg* cfg, double rho, double divv, double nu, double dt)
{
    if (!(divv < 0.0)) return 0.0;
    double hp = (1.0 / cfg->N) / (cfg->k + 1);
    double Pi = rho * nu * (-divv);
    if (dt > 0.0) {
        double Pmax = 0.5 * rho * hp * hp * (-divv) / dt;
        if (Pi > Pmax) Pi = Pmax;
    }
    return Pi;
}

int orc_rhs_nu(const orc_cfg* cfg, const double* u, const double* ahat, double dt_pimax, const double* nu_cell,
               double* dudt)
{
    return rhs_impl(cfg, u, ahat, dt_pimax, nu_cell, dudt);
}

/* volume integral and forcing source of one cell, added to rc [4][b]; nu < 0:
 * the vNR viscous pressure, else the per-cell coefficient nu */
static void volume_cell(const tabs* Tp, const orc_cfg* cfg, const double* uc, const double* ac, const double abar[3],
                        double nu, double dt_pimax, double* rc)
{
    const tabs T = *Tp;
    int b = T.b, nq = T.nq;
    double h = 1.0 / cfg->N, cs2 = cfg->cs * cfg->cs;
    for (int q = 0; q < nq; ++q) {
        const double* ph = T.phi + q * b;
        double rho = eval(&T, uc, ph), m[3], v[3], drho[3], dmd[3];
        for (int i = 0; i < 3; ++i) {
            m[i] = eval(&T, uc + (1 + i) * b, ph);
            v[i] = m[i] / rho;
        }
        for (int d = 0; d < 3; ++d) {
            const double* dph = T.dphi + ((size_t)d * nq + q) * b;
            drho[d] = (2.0 / h) * eval(&T, uc, dph);
            dmd[d] = (2.0 / h) * eval(&T, uc + (1 + d) * b, dph);
        }
        /* div v = (div m - v . grad rho) / rho */
        double divv = (dmd[0] + dmd[1] + dmd[2] - (v[0] * drho[0] + v[1] * drho[1] + v[2] * drho[2])) / rho;
        double P = cs2 * rho + (nu >= 0.0 ? orc_pi_nu(cfg, rho, divv, nu, dt_pimax) : orc_vnr(cfg, rho, divv, dt_pimax));
        double F[4][3]; /* F[var][d] */
        for (int d = 0; d < 3; ++d) {
            F[0][d] = m[d];
            for (int i = 0; i < 3; ++i) F[1 + i][d] = m[i] * v[d] + (i == d ? P : 0.0);
        }
        for (int l = 0; l < b; ++l) {
            double g[3];
            for (int d = 0; d < 3; ++d) g[d] = T.dphi[((size_t)d * nq + q) * b + l];
            for (int var = 0; var < 4; ++var)
                rc[var * b + l] += T.wq[q] * (g[0] * F[var][0] + g[1] * F[var][1] + g[2] * F[var][2]) / (4.0 * h);
        }
        if (ac) {
            for (int i = 0; i < 3; ++i) {
                double src = rho * (eval(&T, ac + i * b, ph) - abar[i]);
                for (int l = 0; l < b; ++l) rc[(1 + i) * b + l] += 0.125 * T.wq[q] * ph[l] * src;
            }
        }
    }
}

/* numerical flux at face point s of the interface along d between the lower
 * cell L (its xi_d = +1 face) and the upper cell R (its xi_d = -1 face); face
 * states rho from the cells' own expansions, v from their projections */
static void face_flux(const tabs* T, const orc_cfg* cfg, int d, int s, const double* uL, const double* vL,
                      const double* uR, const double* vR, double Fs[4])
{
    int b = T->b, ns = T->ns;
    const double* phL = T->phif + ((size_t)(d * 2 + 1) * ns + s) * b;
    const double* phR = T->phif + ((size_t)(d * 2 + 0) * ns + s) * b;
    double WL[4], WR[4];
    WL[0] = eval(T, uL, phL);
    WR[0] = eval(T, uR, phR);
    for (int i = 0; i < 3; ++i) {
        WL[1 + i] = eval(T, vL + i * b, phL);
        WR[1 + i] = eval(T, vR + i * b, phR);
    }
    orc_riemann(cfg->riemann, cfg->cs, d, WL, WR, Fs);
}

static int rhs_impl(const orc_cfg* cfg, const double* u, const double* ahat, double dt_pimax, const double* nu_cell,
                    double* dudt)
{
    tabs T;
    tabs_init(&T, cfg->k, cfg->k + 1);
    int N = cfg->N, b = T.b, ns = T.ns;
    size_t nc = (size_t)N * N * N;
    double h = 1.0 / N;
    double* vhat = (double*)malloc(sizeof(double) * nc * 3 * b);
    orc_project_velocity(cfg, u, vhat);
    double abar[3] = {0, 0, 0};
    if (ahat) orc_forcing_mean(cfg, u, ahat, abar);
    memset(dudt, 0, sizeof(double) * nc * 4 * b);

    /* volume integral and forcing source, cell by cell */
#pragma omp parallel for schedule(static)
    for (size_t c = 0; c < nc; ++c)
        volume_cell(&T, cfg, u + c * 4 * b, ahat ? ahat + c * 3 * b : NULL, abar, nu_cell ? nu_cell[c] : -1.0,
                    dt_pimax, dudt + c * 4 * b);

    /* surface integral: one pass over interfaces, each flux added to both cells.
     * Per direction d the interfaces are taken in colours by the coordinate i
     * of their lower cell along d (i even, i odd, and for odd N the wrap-around
     * interface i = N - 1 alone), so that no two interfaces of a colour share a
     * cell and the cells of a colour can be updated in parallel; the order of
     * the updates of every cell is the same for any number of threads. */
    for (int d = 0; d < 3; ++d) {
        const double* phL = T.phif + ((size_t)(d * 2 + 1) * ns) * b; /* xi_d = +1 in L */
        const double* phR = T.phif + ((size_t)(d * 2 + 0) * ns) * b; /* xi_d = -1 in R */
        for (int colour = 0; colour < 3; ++colour) {
#pragma omp parallel for schedule(static)
            for (int cL = 0; cL < (int)nc; ++cL) {
                const int ix = cL % N, iy = (cL / N) % N, iz = cL / (N * N);
                const int i = d == 0 ? ix : (d == 1 ? iy : iz);
                const int col = ((N & 1) && i == N - 1) ? 2 : (i & 1);
                if (col != colour) continue;
                int cR = cell_index(N, ix + (d == 0), iy + (d == 1), iz + (d == 2));
                for (int s = 0; s < ns; ++s) {
                    double Fs[4];
                    face_flux(&T, cfg, d, s, u + (size_t)cL * 4 * b, vhat + (size_t)cL * 3 * b,
                              u + (size_t)cR * 4 * b, vhat + (size_t)cR * 3 * b, Fs);
                    for (int var = 0; var < 4; ++var)
                        for (int l = 0; l < b; ++l) {
                            dudt[((size_t)cL * 4 + var) * b + l] -= T.ws[s] * phL[s * b + l] * Fs[var] / (4.0 * h);
                            dudt[((size_t)cR * 4 + var) * b + l] += T.ws[s] * phR[s * b + l] * Fs[var] / (4.0 * h);
                        }
                }
            }
        }
    }
    free(vhat);
    tabs_free(&T);
    orc_diffusion_rhs(cfg, u, dudt); /* + div(eps grad u) when eps > 0 */
    return 0;
}

/* Right-hand side of single cells from their neighbourhoods: the same volume
 * term, face fluxes and lifts as orc_rhs, for cells given with their six face
 * neighbours.  patch [n][7][4][b]: the cell, then its neighbours across the
 * faces -x, +x, -y, +y, -z, +z; ahat_c [n][3][b] or NULL with abar the mean
 * acceleration of the whole field; nu [n] or NULL (vNR).  Without the
 * diffusion operator (it returns -1 when eps_diff > 0). */
int orc_rhs_local(const orc_cfg* cfg, const double* patch, const double* ahat_c, const double abar[3], double dt_pimax,
                  const double* nu, int64_t n, double* out)
{
    if (cfg->eps_diff > 0.0) return -1;
    tabs T;
    tabs_init(&T, cfg->k, cfg->k + 1);
    int b = T.b, ns = T.ns;
    double h = 1.0 / cfg->N;
    double* vh = (double*)malloc(sizeof(double) * 7 * 3 * b);
    const double zero[3] = {0, 0, 0};
    for (int64_t c = 0; c < n; ++c) {
        const double* pc = patch + (size_t)c * 7 * 4 * b;
        double* rc = out + (size_t)c * 4 * b;
        memset(rc, 0, sizeof(double) * 4 * b);
        for (int j = 0; j < 7; ++j) project_cell(&T, pc + j * 4 * b, vh + j * 3 * b);
        volume_cell(&T, cfg, pc, ahat_c ? ahat_c + (size_t)c * 3 * b : NULL, abar ? abar : zero, nu ? nu[c] : -1.0,
                    dt_pimax, rc);
        for (int d = 0; d < 3; ++d) {
            const int jm = 1 + 2 * d, jp = 2 + 2 * d;
            const double* phL = T.phif + ((size_t)(d * 2 + 1) * ns) * b; /* + face of the cell */
            const double* phR = T.phif + ((size_t)(d * 2 + 0) * ns) * b; /* - face of the cell */
            for (int s = 0; s < ns; ++s) {
                double Fp[4], Fm[4];
                face_flux(&T, cfg, d, s, pc, vh, pc + jp * 4 * b, vh + jp * 3 * b, Fp);
                face_flux(&T, cfg, d, s, pc + jm * 4 * b, vh + jm * 3 * b, pc, vh, Fm);
                for (int var = 0; var < 4; ++var)
                    for (int l = 0; l < b; ++l) {
                        rc[var * b + l] -= T.ws[s] * phL[s * b + l] * Fp[var] / (4.0 * h);
                        rc[var * b + l] += T.ws[s] * phR[s * b + l] * Fm[var] / (4.0 * h);
                    }
            }
        }
    }
    free(vh);
    tabs_free(&T);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* positivity (Sec. 3.1): density checked at every volume and face Gauss      */
/* point; if the minimum is below the floor and the mean is above it, all   */
/* higher-order weights of all variables are scaled by                       */
/*   theta = (rho_mean - eps) / (rho_mean - rho_min);                         */
/* a mean at or below the floor is a failure (the step is retried with a     */
/* smaller dt by the time-step loop); with pos_mode 1 only a mean at or      */
/* below zero is.                                                            */
/* ------------------------------------------------------------------------ */
static int limit_impl(const orc_cfg* cfg, double* u, uint8_t* flag)
{
    tabs T;
    tabs_init(&T, cfg->k, cfg->k + 1);
    int N = cfg->N, b = T.b;
    size_t nc = (size_t)N * N * N;
    double eps = cfg->rho_floor;
    int status = 0;
#pragma omp parallel for schedule(static) reduction(| : status)
    for (size_t c = 0; c < nc; ++c) {
        double* uc = u + c * 4 * b;
        double rmin = INFINITY;
        for (int q = 0; q < T.nq; ++q) rmin = fmin(rmin, eval(&T, uc, T.phi + q * b));
        for (int f = 0; f < 6; ++f)
            for (int s = 0; s < T.ns; ++s) rmin = fmin(rmin, eval(&T, uc, T.phif + ((size_t)f * T.ns + s) * b));
        if (flag && rmin < 0.0) flag[c] |= ORC_MARK_NEGATIVE;
        if (rmin < eps) {
            double rbar = uc[0];
            if (rbar > eps) {
                double theta = (rbar - eps) / (rbar - rmin);
                for (int var = 0; var < 4; ++var)
                    for (int l = 1; l < b; ++l) uc[var * b + l] *= theta;
                status |= ORC_LIMITED;
            } else if (cfg->pos_mode != 1 || rbar <= 0.0) {
                /* pos_mode 1: only a mean that is not positive fails; a mean in
                   (0, eps] is left as it is (its negative points mark the cell) */
                status |= ORC_FAIL;
            }
        }
    }
    tabs_free(&T);
    return status;
}

int orc_limit(const orc_cfg* cfg, double* u) { return limit_impl(cfg, u, NULL); }

/* ------------------------------------------------------------------------ */
/* one SSP Runge-Kutta step (Sec. 7) with the limiter after every stage      */
/*   RK2: u1 = un + dt L(un);  un+1 = un/2 + (u1 + dt L(u1))/2               */
/*   RK3: u1 = un + dt L(un);  u2 = 3un/4 + (u1 + dt L(u1))/4;               */
/*        un+1 = un/3 + 2(u2 + dt L(u2))/3                                    */
/* dt also fixes Pi_max for every stage.                                      */
/* ------------------------------------------------------------------------ */
int orc_step(const orc_cfg* cfg, double* u, const double* ahat, double dt)
{
    return orc_step_flags(cfg, u, ahat, dt, 0.0, NULL);
}

/* orc_step; with flag != NULL also marks every cell that a stage troubles:
 * ORC_MARK_NEGATIVE when rho < 0 at one of its volume or face points before the
 * rescaling, ORC_MARK_FAST when after it a volume point has sum_d(|v_d| + cs)
 * > vlim */
int orc_step_flags(const orc_cfg* cfg, double* u, const double* ahat, double dt, double vlim, uint8_t* flag)
{
    int b = orc_nmodes(cfg->k);
    size_t n = (size_t)cfg->N * cfg->N * cfg->N * 4 * b;
    double* un = (double*)malloc(sizeof(double) * n);
    double* us = (double*)malloc(sizeof(double) * n);
    double* L = (double*)malloc(sizeof(double) * n);
    memcpy(un, u, sizeof(double) * n);
    memcpy(us, u, sizeof(double) * n);
    int status = 0;
    static const double a2[2] = {0.0, 0.5}, b2[2] = {1.0, 0.5};
    static const double a3[3] = {0.0, 0.75, 1.0 / 3.0}, b3[3] = {1.0, 0.25, 2.0 / 3.0};
    const double* A = (cfg->rk_stages == 2) ? a2 : a3;
    const double* B = (cfg->rk_stages == 2) ? b2 : b3;
    for (int s = 0; s < cfg->rk_stages; ++s) {
        orc_rhs(cfg, us, ahat, dt, L);
#pragma omp parallel for schedule(static)
        for (size_t i = 0; i < n; ++i) us[i] = A[s] * un[i] + B[s] * (us[i] + dt * L[i]);
        status |= limit_impl(cfg, us, flag);
        if (flag) {
            tabs T;
            tabs_init(&T, cfg->k, cfg->k + 1);
            const int nc = cfg->N * cfg->N * cfg->N;
#pragma omp parallel for schedule(static)
            for (int c = 0; c < nc; ++c)
                for (int q = 0; q < T.nq; ++q)
                    if (point_speed(&T, cfg, us + (size_t)c * 4 * b, q) > vlim) flag[c] |= ORC_MARK_FAST;
            tabs_free(&T);
        }
    }
    memcpy(u, us, sizeof(double) * n);
    free(un);
    free(us);
    free(L);
    return status;
}

/* ------------------------------------------------------------------------ */
/* positivity by repetition of the step (Sec. 3.1, last paragraph, read as   */
/* the troubled-cell procedure the same section gives for the finite-volume */
/* scheme, with "scale all high-order weights" applied to the step's input): */
/*   attempt: S = speed bound of u, dt = cfl h / ((k+1) S) (or fixed_dt)     */
/*   times 2^-h; the step as orc_step_flags with vlim = ORC_REPEAT_SPEED S.   */
/*   Every marked cell of u that is not flat has its higher modes multiplied  */
/*   by 1/2 (its first two times in this step) or 0 (the third); a flat cell */
/*   with negative density, or a cell mean at or below the floor, increments  */
/*   h.  If nothing was scaled and h did not change, the attempt is accepted */
/*   (the stage outputs keep their rescaling, as in orc_step); otherwise the  */
/*   step is attempted again from the modified u.                            */
/* The speed test (a stage output breaking the Courant condition that set    */
/* its dt) is an addition to the paper's text; a flat cell's speed is its    */
/* mean velocity, which the next step's dt takes into account.  Returns the  */
/* status bits (with ORC_REPEATED after more than one attempt), or -1 when   */
/* the attempts or the halvings run out; u then holds u^n with its troubled  */
/* cells flattened.  level [nc] (optional): how often each cell was scaled.   */
/* ------------------------------------------------------------------------ */
int orc_step_repeat(const orc_cfg* cfg, double* u, const double* ahat, double fixed_dt, double* dt_used,
                    int* attempts, uint8_t* level)
{
    const int b = orc_nmodes(cfg->k);
    const size_t nc = (size_t)cfg->N * cfg->N * cfg->N, n = nc * 4 * b;
    double* w = (double*)malloc(sizeof(double) * n);
    uint8_t* flag = (uint8_t*)malloc(nc);
    uint8_t* lev = (uint8_t*)calloc(nc, 1);
    int h = 0, rc = -1;
    for (int att = 0; att < ORC_REPEAT_MAX && h <= ORC_REPEAT_HALVINGS; ++att) {
        const double S = orc_speed_bound(cfg, u);
        const double dt = (fixed_dt > 0.0 ? fixed_dt : orc_dt(cfg, u)) * ldexp(1.0, -h);
        memcpy(w, u, sizeof(double) * n);
        memset(flag, 0, nc);
        const int st = orc_step_flags(cfg, w, ahat, dt, ORC_REPEAT_SPEED * S, flag);
        int flat = 0, scaled = 0;
        for (size_t c = 0; c < nc; ++c) {
            if (!flag[c]) continue;
            double* uc = u + c * 4 * b;
            int nonzero = 0;
            for (int var = 0; var < 4; ++var)
                for (int l = 1; l < b; ++l) nonzero |= uc[var * b + l] != 0.0;
            if (!nonzero) {
                if (flag[c] & ORC_MARK_NEGATIVE) flat = 1;
                continue;
            }
            const double f = lev[c] < 2 ? 0.5 : 0.0;
            for (int var = 0; var < 4; ++var)
                for (int l = 1; l < b; ++l) uc[var * b + l] *= f;
            lev[c] += 1;
            scaled = 1;
        }
        if (!scaled && !flat && !(st & ORC_FAIL)) {
            memcpy(u, w, sizeof(double) * n);
            if (dt_used) *dt_used = dt;
            if (attempts) *attempts = att + 1;
            rc = st | (att > 0 ? ORC_REPEATED : 0);
            break;
        }
        if (flat || (st & ORC_FAIL)) ++h;
    }
    if (level) memcpy(level, lev, nc);
    free(w);
    free(flag);
    free(lev);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Ornstein-Uhlenbeck driving (Sec. 4.2)                                     */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea & Flood 2014), as published. */
uint64_t orc_splitmix64(uint64_t* state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static double uniform53(uint64_t* st) { return (double)(orc_splitmix64(st) >> 11) * (1.0 / 9007199254740992.0); }

/* standard normal by Box-Muller; the cosine branch first, then the sine branch */
static double gauss(orc_ou* ou)
{
    if (ou->have_spare) {
        ou->have_spare = 0;
        return ou->spare;
    }
    double u1 = 1.0 - uniform53(&ou->rng); /* (0, 1] */
    double u2 = uniform53(&ou->rng);
    double r = sqrt(-2.0 * log(u1));
    ou->spare = r * sin(2.0 * ORC_PI * u2);
    ou->have_spare = 1;
    return r * cos(2.0 * ORC_PI * u2);
}

/* Modes: integer k with kmin2 <= |k|^2 <= kmax2, one representative of each
 * +-k pair (first non-zero component positive), lexicographic order.
 * t_c = T = L/(2 cs M) (eq. eddy_turnover_time), update interval t_c/100,
 * f = exp(-dt_drive/t_c).  sigma = 2 M^2 cs^2 / L is the rms acceleration:
 * each real component of x has stationary variance
 * s^2 = sigma^2 / (4 nmodes (2 zeta^2 + (1-zeta)^2)), so that <|a|^2> = sigma^2
 * after the Helmholtz projection with solenoidal weight zeta. */
void orc_ou_init(orc_ou* ou, int kmin2, int kmax2, double zeta, double mach, double cs, double L, uint64_t seed,
                 double t_off)
{
    memset(ou, 0, sizeof(*ou));
    int K = (int)floor(sqrt((double)kmax2) + 1e-9);
    int nm = 0;
    for (int kx = -K; kx <= K; ++kx)
        for (int ky = -K; ky <= K; ++ky)
            for (int kz = -K; kz <= K; ++kz) {
                int r2 = kx * kx + ky * ky + kz * kz;
                if (r2 < kmin2 || r2 > kmax2) continue;
                int first = kx != 0 ? kx : (ky != 0 ? ky : kz);
                if (first <= 0) continue;
                if (nm < ORC_MAX_MODES) {
                    ou->kvec[nm][0] = kx;
                    ou->kvec[nm][1] = ky;
                    ou->kvec[nm][2] = kz;
                }
                ++nm;
            }
    ou->nmodes = nm;
    ou->zeta = zeta;
    ou->tc = L / (2.0 * cs * mach);
    ou->dt_drive = ou->tc / 100.0;
    ou->f = exp(-ou->dt_drive / ou->tc);
    ou->sigma = 2.0 * mach * mach * cs * cs / L;
    ou->s = ou->sigma / sqrt(4.0 * nm * (2.0 * zeta * zeta + (1.0 - zeta) * (1.0 - zeta)));
    ou->rng = seed;
    for (int m = 0; m < nm; ++m)
        for (int i = 0; i < 3; ++i)
            for (int r = 0; r < 2; ++r) ou->x[m][i][r] = ou->s * gauss(ou);
    ou->t_next = ou->dt_drive;
    ou->t_off = t_off;
    ou->on = 1;
    ou->dirty = 1;
}

/* x <- f x + s sqrt(1 - f^2) z  (eq. ornstein_uhlenbeck_process_time_evolution) */
void orc_ou_advance(orc_ou* ou)
{
    double c = ou->s * sqrt(1.0 - ou->f * ou->f);
    for (int m = 0; m < ou->nmodes; ++m)
        for (int i = 0; i < 3; ++i)
            for (int r = 0; r < 2; ++r) ou->x[m][i][r] = ou->f * ou->x[m][i][r] + c * gauss(ou);
}

/* ahat_k = P_zeta(k) x_k,  P_zeta = zeta (I - k k^T/|k|^2) + (1 - zeta) k k^T/|k|^2 */
void orc_ou_amplitudes(const orc_ou* ou, double* amp)
{
    for (int m = 0; m < ou->nmodes; ++m) {
        double kk[3], k2 = 0.0;
        for (int i = 0; i < 3; ++i) {
            kk[i] = ou->kvec[m][i];
            k2 += kk[i] * kk[i];
        }
        for (int r = 0; r < 2; ++r)
            for (int i = 0; i < 3; ++i) {
                double s = 0.0;
                for (int j = 0; j < 3; ++j) {
                    double kkij = kk[i] * kk[j] / k2;
                    double P = ou->zeta * ((i == j ? 1.0 : 0.0) - kkij) + (1.0 - ou->zeta) * kkij;
                    s += P * ou->x[m][j][r];
                }
                amp[(m * 3 + i) * 2 + r] = s;
            }
    }
}

/* a(x) = sum_k 2 Re(ahat_k exp(2 pi i k.x)), projected per cell onto the basis:
 * ahat_l = (1/8) sum_q w_q phi_l(xi_q) a(x_q),  x_q = x_c + (h/2) xi_q. */
void orc_forcing_project(const orc_cfg* cfg, int nmodes, const int32_t* kvec, const double* amp, double* ahat)
{
    tabs T;
    tabs_init(&T, cfg->k, cfg->k + 1);
    int N = cfg->N, b = T.b;
    double h = 1.0 / N;
    for (int iz = 0; iz < N; ++iz)
        for (int iy = 0; iy < N; ++iy)
            for (int ix = 0; ix < N; ++ix) {
                double* ac = ahat + (size_t)cell_index(N, ix, iy, iz) * 3 * b;
                memset(ac, 0, sizeof(double) * 3 * b);
                for (int q = 0; q < T.nq; ++q) {
                    double xi[3];
                    vol_point(&T, q, xi);
                    double x = (ix + 0.5 + 0.5 * xi[0]) * h, y = (iy + 0.5 + 0.5 * xi[1]) * h,
                           z = (iz + 0.5 + 0.5 * xi[2]) * h;
                    double a[3] = {0, 0, 0};
                    for (int m = 0; m < nmodes; ++m) {
                        double th = 2.0 * ORC_PI * (kvec[3 * m] * x + kvec[3 * m + 1] * y + kvec[3 * m + 2] * z);
                        double c = cos(th), s = sin(th);
                        for (int i = 0; i < 3; ++i)
                            a[i] += 2.0 * (amp[(m * 3 + i) * 2] * c - amp[(m * 3 + i) * 2 + 1] * s);
                    }
                    for (int i = 0; i < 3; ++i)
                        for (int l = 0; l < b; ++l) ac[i * b + l] += 0.125 * T.wq[q] * T.phi[q * b + l] * a[i];
                }
            }
    tabs_free(&T);
}

/* ------------------------------------------------------------------------ */
/* time-stepping driver with the driving schedule and the dt retry           */
/* At the start of a step: while t >= t_next advance the OU process and      */
/* t_next += dt_drive; re-project the forcing when it changed.  After t_off  */
/* (if > 0) the forcing is switched off.  A step whose stages report a       */
/* failure is redone from the same state with dt/2, at most 3 times.         */
/* Returns 0, or -1 when the retries are exhausted (state left at u^n).     */
/* pos_mode 1: every step by orc_step_repeat (-1 when it gives up).         */
/* ------------------------------------------------------------------------ */
int orc_run(const orc_cfg* cfg, double* u, orc_ou* ou, int use_forcing, double* ahat, int nsteps, double* t,
            double* dt_last)
{
    int b = orc_nmodes(cfg->k);
    size_t n = (size_t)cfg->N * cfg->N * cfg->N * 4 * b;
    double* bak = (double*)malloc(sizeof(double) * n);
    double* amp = (double*)malloc(sizeof(double) * ORC_MAX_MODES * 6);
    int rc = 0;
    for (int st = 0; st < nsteps; ++st) {
        const double* force = NULL;
        if (use_forcing && ou->on && ou->t_off > 0.0 && *t > ou->t_off) ou->on = 0;
        if (use_forcing && ou->on) {
            while (*t >= ou->t_next) {
                orc_ou_advance(ou);
                ou->t_next += ou->dt_drive;
                ou->dirty = 1;
            }
            if (ou->dirty) {
                orc_ou_amplitudes(ou, amp);
                orc_forcing_project(cfg, ou->nmodes, &ou->kvec[0][0], amp, ahat);
                ou->dirty = 0;
            }
            force = ahat;
        }
        if (cfg->pos_mode == 1) {
            double dtu = 0.0;
            if (orc_step_repeat(cfg, u, force, 0.0, &dtu, NULL, NULL) < 0) {
                rc = -1;
                break;
            }
            *t += dtu;
            if (dt_last) *dt_last = dtu;
            continue;
        }
        double dt = orc_dt(cfg, u);
        int status = ORC_FAIL;
        double dtt = dt;
        memcpy(bak, u, sizeof(double) * n);
        for (int r = 0; r <= 3; ++r) {
            dtt = dt / (double)(1 << r);
            status = orc_step(cfg, u, force, dtt);
            if (!(status & ORC_FAIL)) break;
            memcpy(u, bak, sizeof(double) * n);
        }
        if (status & ORC_FAIL) {
            rc = -1;
            break;
        }
        *t += dtt;
        if (dt_last) *dt_last = dtt;
    }
    free(bak);
    free(amp);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* diagnostics (Sec. 4.1 and the energy bookkeeping of Sec. 4.2)             */
/*  0 mass, 1-3 momentum, 4 kinetic energy, 5 M = <v^2>^(1/2)/cs,            */
/*  6 M_rho = (2 E_kin / M_tot)^(1/2)/cs, 7 min rho, 8 max rho (volume       */
/*  points), 9 volume fraction with Pi > 0.01 cs^2 rho, 10 injected power    */
/*  int m.(a_h - abar) dV, 11 max sum_d(|v_d| + cs), 12 int Pi div v dV.      */
/* ------------------------------------------------------------------------ */
void orc_diagnostics(const orc_cfg* cfg, const double* u, const double* ahat, double dt, double* out)
{
    tabs T;
    tabs_init(&T, cfg->k, cfg->k + 1);
    int N = cfg->N, b = T.b, nq = T.nq;
    size_t nc = (size_t)N * N * N;
    double h = 1.0 / N, V = h * h * h, cs = cfg->cs;
    double abar[3] = {0, 0, 0};
    if (ahat) orc_forcing_mean(cfg, u, ahat, abar);
    for (int i = 0; i < ORC_NDIAG; ++i) out[i] = 0.0;
    out[7] = INFINITY;
    out[8] = -INFINITY;
    for (size_t c = 0; c < nc; ++c) {
        const double* uc = u + c * 4 * b;
        out[0] += uc[0] * V;
        for (int i = 0; i < 3; ++i) out[1 + i] += uc[(1 + i) * b] * V;
        for (int q = 0; q < nq; ++q) {
            const double* ph = T.phi + q * b;
            double wv = 0.125 * T.wq[q] * V;
            double rho = eval(&T, uc, ph), m[3], v2 = 0.0, s = 0.0, drho[3], dmd[3], vd = 0.0, dm = 0.0;
            for (int i = 0; i < 3; ++i) {
                m[i] = eval(&T, uc + (1 + i) * b, ph);
                v2 += (m[i] / rho) * (m[i] / rho);
                s += fabs(m[i] / rho) + cs;
            }
            for (int d = 0; d < 3; ++d) {
                const double* dph = T.dphi + ((size_t)d * nq + q) * b;
                drho[d] = (2.0 / h) * eval(&T, uc, dph);
                dmd[d] = (2.0 / h) * eval(&T, uc + (1 + d) * b, dph);
                vd += (m[d] / rho) * drho[d];
                dm += dmd[d];
            }
            double divv = (dm - vd) / rho;
            double Pi = orc_vnr(cfg, rho, divv, dt);
            out[4] += wv * 0.5 * rho * v2;
            out[5] += wv * v2;
            out[7] = fmin(out[7], rho);
            out[8] = fmax(out[8], rho);
            if (Pi > 0.01 * cs * cs * rho) out[9] += wv;
            if (ahat) {
                const double* ac = ahat + c * 3 * b;
                for (int i = 0; i < 3; ++i) out[10] += wv * m[i] * (eval(&T, ac + i * b, ph) - abar[i]);
            }
            if (s > out[11]) out[11] = s;
            out[12] += wv * Pi * divv;
        }
    }
    double vol = 1.0;
    out[5] = sqrt(out[5] / vol) / cs;
    out[6] = sqrt(2.0 * out[4] / out[0]) / cs;
    out[9] /= vol;
    tabs_free(&T);
}

/* L1 density difference (eq. l1_norm) between two states, by (k+3)-point
 * Gauss quadrature per axis in every cell, divided by the box volume. */
double orc_l1_density(const orc_cfg* cfg, const double* uA, const double* uB)
{
    tabs T;
    tabs_init(&T, cfg->k, cfg->k + 3);
    int N = cfg->N, b = T.b;
    size_t nc = (size_t)N * N * N;
    double h = 1.0 / N, sum = 0.0;
    for (size_t c = 0; c < nc; ++c)
        for (int q = 0; q < T.nq; ++q) {
            double d = eval(&T, uA + c * 4 * b, T.phi + q * b) - eval(&T, uB + c * 4 * b, T.phi + q * b);
            sum += 0.125 * T.wq[q] * fabs(d) * h * h * h;
        }
    tabs_free(&T);
    return sum;
}

/* ------------------------------------------------------------------------ */
/* learned-sensor features and labels (per cell)                             */
/*  x[c][0..b)   = rho_l / rho_0                                              */
/*  x[c][b..2b)  = |v|hat_l / cs, |v|hat the Gauss projection of |m/rho|    */
/*  y[c]         = log(max(nu_cell, nu_f) / (cs h/p)),                       */
/*  nu_cell = Gauss-weighted mean, over the volume points with div v < 0, of */
/*  the pointwise coefficient Pi/(rho |div v|) of the vNR pressure of        */
/*  Sec. 3.1 (cap with dt), the coefficient the learned pressure             */
/*  rho nu |div v| applies at those same points; nu_f = max(beta, 0.05) cs h/p*/
/*  is the coefficient every compressive point receives from the linear term */
/*  (Pi only acts where div v < 0, so cells without compression carry the    */
/*  floor).                                                                   */
/* ------------------------------------------------------------------------ */
void orc_av_features(const orc_cfg* cfg, const double* u, double dt, double* x, double* y)
{
    tabs T;
    tabs_init(&T, cfg->k, cfg->k + 1);
    int N = cfg->N, b = T.b, nq = T.nq;
    size_t nc = (size_t)N * N * N;
    double h = 1.0 / N, hp = h / (cfg->k + 1), ref = cfg->cs * hp;
    for (size_t c = 0; c < nc; ++c) {
        const double* uc = u + c * 4 * b;
        double* xc = x + c * 2 * b;
        for (int l = 0; l < b; ++l) {
            xc[l] = uc[l] / uc[0];
            xc[b + l] = 0.0;
        }
        double nsum = 0.0, wsum = 0.0;
        for (int q = 0; q < nq; ++q) {
            const double* ph = T.phi + q * b;
            double rho = eval(&T, uc, ph), m[3], v[3], drho[3], dmd[3];
            for (int i = 0; i < 3; ++i) {
                m[i] = eval(&T, uc + (1 + i) * b, ph);
                v[i] = m[i] / rho;
            }
            for (int d = 0; d < 3; ++d) {
                const double* dph = T.dphi + ((size_t)d * nq + q) * b;
                drho[d] = (2.0 / h) * eval(&T, uc, dph);
                dmd[d] = (2.0 / h) * eval(&T, uc + (1 + d) * b, dph);
            }
            double divv = (dmd[0] + dmd[1] + dmd[2] - (v[0] * drho[0] + v[1] * drho[1] + v[2] * drho[2])) / rho;
            double speed = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            for (int l = 0; l < b; ++l) xc[b + l] += 0.125 * T.wq[q] * ph[l] * speed / cfg->cs;
            if (divv < 0.0) {
                nsum += T.wq[q] * orc_vnr(cfg, rho, divv, dt) / (rho * (-divv));
                wsum += T.wq[q];
            }
        }
        const double nu = wsum > 0.0 ? nsum / wsum : 0.0;
        const double floor_ = (cfg->beta > 0.05 ? cfg->beta : 0.05) * ref;
        y[c] = log((nu > floor_ ? nu : floor_) / ref);
    }
    tabs_free(&T);
}


/* ------------------------------------------------------------------------ */
/* turbulence statistics                                                     */
/* ------------------------------------------------------------------------ */

/* Volume-weighted PDF of s = log10(rho / rho_mean) (Sec. 4.3 bins the log of
 * the density; here the whole volume, sampled at every cell's Gauss points
 * with their weights, so each sample carries its share of the volume):
 * hist[i] = volume fraction with s in [lo + i ds, lo + (i+1) ds),
 * ds = (hi - lo) / nbins; samples outside [lo, hi) are not counted. */
void orc_density_pdf(const orc_cfg* cfg, const double* u, double lo, double hi, int nbins, double* hist)
{
    tabs T;
    tabs_init(&T, cfg->k, cfg->k + 1);
    const int N = cfg->N, b = T.b;
    const size_t nc = (size_t)N * N * N;
    double mass = 0.0;
    for (size_t c = 0; c < nc; ++c) mass += u[c * 4 * b] / (double)nc;  /* cell means, unit box */
    for (int i = 0; i < nbins; ++i) hist[i] = 0.0;
    const double ds = (hi - lo) / nbins;
    for (size_t c = 0; c < nc; ++c)
        for (int q = 0; q < T.nq; ++q) {
            const double rho = eval(&T, u + c * 4 * b, T.phi + q * b);
            if (!(rho > 0.0)) continue;
            const double sv = log10(rho / mass);
            const int i = (int)floor((sv - lo) / ds);
            if (i >= 0 && i < nbins) hist[i] += T.wq[q] / 8.0 / (double)nc;
        }
    tabs_free(&T);
}

/* velocity v = m / rho at a point x of the periodic unit box, evaluated from
 * the expansions of the cell that contains it; returns rho */
double orc_velocity_at(const orc_cfg* cfg, const double* u, const double x[3], double v[3])
{
    const int N = cfg->N, k = cfg->k, b = orc_nmodes(k);
    int32_t ijl[3 * 84];
    orc_mode_list(k, ijl);
    int ic[3];
    double xi[3];
    for (int d = 0; d < 3; ++d) {
        double y = x[d] - floor(x[d]); /* wrap into [0, 1) */
        double s = y * N;
        int i = (int)floor(s);
        if (i >= N) i = N - 1;
        ic[d] = i;
        xi[d] = 2.0 * (s - i) - 1.0;
    }
    const double* uc = u + (size_t)cell_index(N, ic[0], ic[1], ic[2]) * 4 * b;
    double f[4] = {0.0, 0.0, 0.0, 0.0};
    for (int l = 0; l < b; ++l) {
        const double ph = orc_legendre(ijl[3 * l], xi[0]) * sqrt(2.0 * ijl[3 * l] + 1.0) *
                          orc_legendre(ijl[3 * l + 1], xi[1]) * sqrt(2.0 * ijl[3 * l + 1] + 1.0) *
                          orc_legendre(ijl[3 * l + 2], xi[2]) * sqrt(2.0 * ijl[3 * l + 2] + 1.0);
        for (int var = 0; var < 4; ++var) f[var] += uc[var * b + l] * ph;
    }
    for (int d = 0; d < 3; ++d) v[d] = f[1 + d] / f[0];
    return f[0];
}

/* the n-th number of the SplitMix64 sequence started from seed, as a
 * uniform double in [0, 1) (53 bits) */
static double splitmix_at(uint64_t seed, uint64_t n)
{
    uint64_t st = seed + n * 0x9E3779B97F4A7C15ULL;
    return (double)(orc_splitmix64(&st) >> 11) * (1.0 / 9007199254740992.0);
}

/* Second-order velocity structure function (Sec. 4.1 definition, Sec. 4.3
 * sampling): nbins logarithmic bins between l_min = 1/((k+1) N) and
 * l_max = 1/2; in bin j the separation is the bin's logarithmic centre
 * l_j = l_min (l_max/l_min)^((j + 1/2)/nbins).  Pair p of bin j draws five
 * uniforms u_r = SplitMix64 number n = (j npairs + p) 5 + r of `seed`:
 * x = (u_0, u_1, u_2), cos(theta) = 2 u_3 - 1, phi = 2 pi u_4; the partner
 * is x + l_j (sin theta cos phi, sin theta sin phi, cos theta), wrapped.
 * v_out[j] = (1/2 <|v(x) - v(x + l)|^2>)^(1/2), l_out[j] = l_j. */
void orc_structure_function(const orc_cfg* cfg, const double* u, int nbins, int64_t npairs, uint64_t seed,
                            double* l_out, double* v_out)
{
    const double lmin = 1.0 / ((cfg->k + 1) * (double)cfg->N), lmax = 0.5;
    for (int j = 0; j < nbins; ++j) {
        const double l = lmin * pow(lmax / lmin, (j + 0.5) / nbins);
        double acc = 0.0;
        for (int64_t p = 0; p < npairs; ++p) {
            const uint64_t n0 = ((uint64_t)j * (uint64_t)npairs + (uint64_t)p) * 5u;
            double x[3], y[3], va[3], vb[3];
            for (int d = 0; d < 3; ++d) x[d] = splitmix_at(seed, n0 + d);
            const double ct = 2.0 * splitmix_at(seed, n0 + 3) - 1.0, phi = 2.0 * ORC_PI * splitmix_at(seed, n0 + 4);
            const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
            const double dir[3] = {st * cos(phi), st * sin(phi), ct};
            for (int d = 0; d < 3; ++d) y[d] = x[d] + l * dir[d];
            orc_velocity_at(cfg, u, x, va);
            orc_velocity_at(cfg, u, y, vb);
            for (int d = 0; d < 3; ++d) acc += (va[d] - vb[d]) * (va[d] - vb[d]);
        }
        l_out[j] = l;
        v_out[j] = sqrt(0.5 * acc / (double)npairs);
    }
}

/* Velocity on the regular Fourier grid of Sec. 4.3: N_g = (k+1) N points per
 * axis at x_g = (g + 1/2) / N_g (k+1 points inside every cell, none on a face).
 * v_out[d][gz][gy][gx], d = 0..2. */
void orc_sample_velocity(const orc_cfg* cfg, const double* u, double* v_out)
{
    const int Ng = (cfg->k + 1) * cfg->N;
    const size_t n3 = (size_t)Ng * Ng * Ng;
    for (int gz = 0; gz < Ng; ++gz)
        for (int gy = 0; gy < Ng; ++gy)
            for (int gx = 0; gx < Ng; ++gx) {
                const double x[3] = {(gx + 0.5) / Ng, (gy + 0.5) / Ng, (gz + 0.5) / Ng};
                double v[3];
                orc_velocity_at(cfg, u, x, v);
                const size_t g = ((size_t)gz * Ng + gy) * Ng + gx;
                for (int d = 0; d < 3; ++d) v_out[d * n3 + g] = v[d];
            }
}


/* ------------------------------------------------------------------------ */
/* diffusion operator div(eps grad u) (Sec. 2, diffusion across cell         */
/* boundaries).  The second derivative at an interface comes from a          */
/* "virtual" cell that covers both neighbours: on their union the solution   */
/* is replaced by the one polynomial whose projections onto each cell's      */
/* basis are that cell's coefficients (recovery); its normal derivative at   */
/* the face is the interface gradient.  Weak form on a cell K:               */
/*   (1/|K|) [ -int_K eps grad phi_l . grad u dV                             */
/*             + int_dK eps phi_l (grad u_rec . n) dS ]                      */
/* ------------------------------------------------------------------------ */

/* Gaussian elimination with partial pivoting, A [n][n] row-major, b [n] */
static void solve_dense(int n, double* A, double* b)
{
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * n + c]) > fabs(A[p * n + c])) p = r;
        if (p != c) {
            for (int j = 0; j < n; ++j) {
                double t = A[c * n + j];
                A[c * n + j] = A[p * n + j];
                A[p * n + j] = t;
            }
            double t = b[c];
            b[c] = b[p];
            b[p] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            const double f = A[r * n + c] / A[c * n + c];
            for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int j = r + 1; j < n; ++j) s -= A[r * n + j] * b[j];
        b[r] = s / A[r * n + r];
    }
}

/* 1D recovery across a face.  Coordinate s in half-cell units on the union
 * of the two cells: L = [-2, 0] (s = xi - 1), R = [0, 2] (s = xi + 1).  With
 * the K+1 normalised-Legendre coefficients of each side, find the polynomial
 * r of degree 2K+1 with (1/2) int_{-1}^{1} Pn_a(xi) r(xi -+ 1) dxi = c_a for
 * a = 0..K on both sides; return dr/ds at the face s = 0.  r is expanded in
 * monomials of s and the moments are taken with a 10-point Gauss rule (exact
 * for the degree 3K+1 <= 10 integrands). */
double orc_recover_dn(int K, const double* cL, const double* cR)
{
    const int n = 2 * K + 2;
    double A[64], rhs[8], xg[10], wg[10];
    orc_gauss(10, xg, wg);
    for (int a = 0; a <= K; ++a)
        for (int j = 0; j < n; ++j) {
            double mL = 0.0, mR = 0.0;
            for (int g = 0; g < 10; ++g) {
                const double pa = sqrt(2.0 * a + 1.0) * orc_legendre(a, xg[g]);
                mL += 0.5 * wg[g] * pa * pow(xg[g] - 1.0, j);
                mR += 0.5 * wg[g] * pa * pow(xg[g] + 1.0, j);
            }
            A[a * n + j] = mL;
            A[(K + 1 + a) * n + j] = mR;
        }
    for (int a = 0; a <= K; ++a) {
        rhs[a] = cL[a];
        rhs[K + 1 + a] = cR[a];
    }
    solve_dense(n, A, rhs);
    return rhs[1]; /* d/ds of sum_j r_j s^j at s = 0 */
}

void orc_diffusion_rhs(const orc_cfg* cfg, const double* u, double* dudt)
{
    const double eps = cfg->eps_diff;
    if (!(eps > 0.0)) return;
    tabs T;
    tabs_init(&T, cfg->k, cfg->k + 1);
    const int N = cfg->N, b = T.b, k = cfg->k, nq = T.nq, ns = T.ns;
    const size_t nc = (size_t)N * N * N;
    const double h = 1.0 / N;
    /* the recovered face derivative is linear in the two coefficient columns:
     * its weights, per number of normal modes K+1, from unit columns */
    double wL[4][4], wR[4][4];
    for (int K = 0; K <= k; ++K)
        for (int a = 0; a <= K; ++a) {
            double e[4] = {0, 0, 0, 0}, z[4] = {0, 0, 0, 0};
            e[a] = 1.0;
            wL[K][a] = orc_recover_dn(K, e, z);
            wR[K][a] = orc_recover_dn(K, z, e);
        }
    /* mode index of the degree triple */
    int midx[4][4][4];
    for (int l = 0; l < b; ++l) midx[T.ijl[3 * l]][T.ijl[3 * l + 1]][T.ijl[3 * l + 2]] = l;
    /* volume: -(eps/|K|) int grad phi_l . grad u = -eps (4/h^2) (1/8) sum_q w_q grad_xi phi_l . grad_xi u */
    for (size_t c = 0; c < nc; ++c)
        for (int var = 0; var < 4; ++var) {
            const double* uc = u + (c * 4 + var) * b;
            for (int q = 0; q < nq; ++q) {
                double g[3];
                for (int d = 0; d < 3; ++d) g[d] = eval(&T, uc, T.dphi + ((size_t)d * nq + q) * b);
                for (int l = 0; l < b; ++l) {
                    double s = 0.0;
                    for (int d = 0; d < 3; ++d) s += T.dphi[((size_t)d * nq + q) * b + l] * g[d];
                    dudt[(c * 4 + var) * b + l] -= eps * (4.0 / (h * h)) * 0.125 * T.wq[q] * s;
                }
            }
        }
    /* faces: for each cell's + face along d, L = the cell, R = its neighbour */
    for (int d = 0; d < 3; ++d) {
        const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
        for (int iz = 0; iz < N; ++iz)
            for (int iy = 0; iy < N; ++iy)
                for (int ix = 0; ix < N; ++ix) {
                    const int ic[3] = {ix, iy, iz};
                    int jc[3] = {ix, iy, iz};
                    jc[d] += 1;
                    const size_t cL = (size_t)cell_index(N, ic[0], ic[1], ic[2]);
                    const size_t cR = (size_t)cell_index(N, jc[0], jc[1], jc[2]);
                    for (int var = 0; var < 4; ++var) {
                        const double* uL = u + (cL * 4 + var) * b;
                        const double* uR = u + (cR * 4 + var) * b;
                        /* normal derivative (physical) at the face points */
                        double gs[64];
                        for (int s = 0; s < ns; ++s) gs[s] = 0.0;
                        /* one 1D recovery per tangential degree pair (p1, p2), p1 + p2 <= k */
                        for (int p1 = 0; p1 <= k; ++p1)
                            for (int p2 = 0; p1 + p2 <= k; ++p2) {
                                const int K = k - p1 - p2;
                                double dn = 0.0;
                                for (int a = 0; a <= K; ++a) {
                                    int deg[3];
                                    deg[d] = a;
                                    deg[t1] = p1;
                                    deg[t2] = p2;
                                    const int m = midx[deg[0]][deg[1]][deg[2]];
                                    dn += wL[K][a] * uL[m] + wR[K][a] * uR[m];
                                }
                                dn *= 2.0 / h;
                                for (int s = 0; s < ns; ++s) {
                                    const double x1 = T.xg[s % T.n], x2 = T.xg[s / T.n];
                                    gs[s] += dn * sqrt(2.0 * p1 + 1.0) * orc_legendre(p1, x1) * sqrt(2.0 * p2 + 1.0) *
                                             orc_legendre(p2, x2);
                                }
                            }
                        /* (eps/|K|) int_face phi_l (grad u . n) dS = eps/h^3 (h/2)^2 sum_s w_s phi_l(s) g_s */
                        const double* phL = T.phif + ((size_t)(d * 2 + 1) * ns) * b;
                        const double* phR = T.phif + ((size_t)(d * 2 + 0) * ns) * b;
                        for (int l = 0; l < b; ++l) {
                            double sL = 0.0, sR = 0.0;
                            for (int s = 0; s < ns; ++s) {
                                sL += T.ws[s] * phL[s * b + l] * gs[s];
                                sR += T.ws[s] * phR[s * b + l] * gs[s];
                            }
                            dudt[(cL * 4 + var) * b + l] += eps / (4.0 * h) * sL;
                            dudt[(cR * 4 + var) * b + l] -= eps / (4.0 * h) * sR;
                        }
                    }
                }
    }
    tabs_free(&T);
}

/* ======================================================================== */
/* Adiabatic system (Sec. 2.1: state vector, ideal-gas equation of state,    */
/* flux matrix).  u = (rho, m, e) per cell, [c][5][b]; e is the total energy */
/* density, p = (gamma - 1)(e - |m|^2 / (2 rho)), and the flux along d is    */
/*   F_d = (m_d, m v_d + p e_d, (e + p) v_d).                                */
/* Volume (Sec. 3.1): conserved values at the internal points; the viscous   */
/* pressure Pi is added to p in the momentum and energy fluxes, its bulk     */
/* term with the local sound speed c = sqrt(gamma p / rho).  Faces (Sec.     */
/* 3.2): rho from its own expansion, v and p from their projections onto the */
/* basis; Rusanov flux with lambda = max over both sides of |v_n| + c.       */
/* Positivity (Sec. 3.1): density and pressure at every volume and face      */
/* point; the higher modes of all variables are scaled toward the cell mean. */
/* ======================================================================== */

/* physical flux along d of the conserved state U = (rho, m, e) */
void orc_adi_flux(double gamma, int d, const double U[5], double F[5])
{
    double rho = U[0], v[3] = {U[1] / rho, U[2] / rho, U[3] / rho};
    double p = (gamma - 1.0) * (U[4] - 0.5 * (U[1] * v[0] + U[2] * v[1] + U[3] * v[2]));
    F[0] = U[1 + d];
    for (int i = 0; i < 3; ++i) F[1 + i] = U[1 + i] * v[d] + (i == d ? p : 0.0);
    F[4] = (U[4] + p) * v[d];
}

/* Rusanov flux from primitive face states W = (rho, v_x, v_y, v_z, p) */
void orc_adi_rusanov(double gamma, int d, const double WL[5], const double WR[5], double F[5])
{
    double UL[5], UR[5], FL[5], FR[5];
    const double* W[2] = {WL, WR};
    double* U[2] = {UL, UR};
    for (int s = 0; s < 2; ++s) {
        const double* w = W[s];
        U[s][0] = w[0];
        for (int i = 0; i < 3; ++i) U[s][1 + i] = w[0] * w[1 + i];
        U[s][4] = w[4] / (gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
    }
    orc_adi_flux(gamma, d, UL, FL);
    orc_adi_flux(gamma, d, UR, FR);
    double lL = fabs(WL[1 + d]) + sqrt(gamma * WL[4] / WL[0]);
    double lR = fabs(WR[1 + d]) + sqrt(gamma * WR[4] / WR[0]);
    double lam = lL > lR ? lL : lR;
    for (int v = 0; v < 5; ++v) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * lam * (UR[v] - UL[v]);
}

/* HLLC flux of the Euler equations (the contact wave restored in the HLL
 * two-wave model) from primitive face states W = (rho, v_x, v_y, v_z, p):
 * Davis bounds S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R),
 * contact speed S* = (p_R - p_L + rho_L u_L (S_L - u_L) - rho_R u_R (S_R - u_R))
 *                    / (rho_L (S_L - u_L) - rho_R (S_R - u_R)),
 * star states U*_K = rho_K (S_K - u_K)/(S_K - S*) (1, S* along d, the tangential
 * velocities, E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))),
 * F = F_L, F_L + S_L (U*_L - U_L), F_R + S_R (U*_R - U_R) or F_R by the sign of
 * S_L, S*, S_R (u the normal velocity) */
void orc_adi_hllc(double gamma, int d, const double WL[5], const double WR[5], double F[5])
{
    double U[2][5], Fx[2][5], c[2], un[2];
    const double* W[2] = {WL, WR};
    for (int s = 0; s < 2; ++s) {
        const double* w = W[s];
        U[s][0] = w[0];
        for (int i = 0; i < 3; ++i) U[s][1 + i] = w[0] * w[1 + i];
        U[s][4] = w[4] / (gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
        orc_adi_flux(gamma, d, U[s], Fx[s]);
        c[s] = sqrt(gamma * w[4] / w[0]);
        un[s] = w[1 + d];
    }
    double SL = fmin(un[0] - c[0], un[1] - c[1]), SR = fmax(un[0] + c[0], un[1] + c[1]);
    if (SL >= 0.0) {
        for (int v = 0; v < 5; ++v) F[v] = Fx[0][v];
        return;
    }
    if (SR <= 0.0) {
        for (int v = 0; v < 5; ++v) F[v] = Fx[1][v];
        return;
    }
    double qL = WL[0] * (SL - un[0]), qR = WR[0] * (SR - un[1]);
    double Ss = (WR[4] - WL[4] + un[0] * qL - un[1] * qR) / (qL - qR);
    int s = Ss >= 0.0 ? 0 : 1;
    double SK = s == 0 ? SL : SR, qK = s == 0 ? qL : qR;
    const double* w = W[s];
    double f = qK / (SK - Ss), Us[5];
    Us[0] = f;
    for (int i = 0; i < 3; ++i) Us[1 + i] = f * (i == d ? Ss : w[1 + i]);
    Us[4] = f * (U[s][4] / w[0] + (Ss - un[s]) * (Ss + w[4] / qK));
    for (int v = 0; v < 5; ++v) F[v] = Fx[s][v] + SK * (Us[v] - U[s][v]);
}

/* face flux of the adiabatic system by cfg->riemann: HLLC, else Rusanov */
static void adi_face_flux(int solver, double gamma, int d, const double WL[5], const double WR[5], double F[5])
{
    if (solver == ORC_HLLC)
        orc_adi_hllc(gamma, d, WL, WR, F);
    else
        orc_adi_rusanov(gamma, d, WL, WR, F);
}

/* the boundary faces along d of the last cell cU (its face xi_d = +1, at
 * coordinate 1) and of the first cell cD (its face xi_d = -1, at coordinate 0):
 * ghost states by cfg->bc[d]; each flux goes to its own cell only */
static void adi_boundary_faces(const orc_cfg* cfg, double gamma, const tabs* T, int d, const double* u,
                               const double* prim, int cU, int cD, double h, double* dudt)
{
    const int b = T->b, ns = T->ns, bc = cfg->bc[d];
    for (int upper = 0; upper < 2; ++upper) {
        const int c = upper ? cU : cD;
        const double* ph = T->phif + ((size_t)(d * 2 + upper) * ns) * b;
        for (int s = 0; s < ns; ++s) {
            double W[5], G[5], F[5];
            W[0] = eval(T, u + (size_t)c * 5 * b, ph + s * b);
            for (int i = 0; i < 4; ++i) W[1 + i] = eval(T, prim + ((size_t)c * 4 + i) * b, ph + s * b);
            for (int i = 0; i < 5; ++i) G[i] = W[i];
            if (bc == ORC_BC_REFLECT) G[1 + d] = -W[1 + d];
            if (bc == ORC_BC_INFLOW && !upper)
                for (int i = 0; i < 5; ++i) G[i] = cfg->inflow[i];
            /* along +e_d: the ghost is the upper neighbour of cU, the lower one of cD */
            if (upper)
                adi_face_flux(cfg->riemann, gamma, d, W, G, F);
            else
                adi_face_flux(cfg->riemann, gamma, d, G, W, F);
            const double sgn = upper ? -1.0 : 1.0;
            for (int var = 0; var < 5; ++var)
                for (int l = 0; l < b; ++l)
                    dudt[((size_t)c * 5 + var) * b + l] += sgn * T->ws[s] * ph[s * b + l] * F[var] / (4.0 * h);
        }
    }
}

/* vNR viscous pressure with the local sound speed in the bulk term */
double orc_adi_vnr(const orc_cfg* cfg, double rho, double c, double divv, double dt)
{
    if (cfg->av_mode != 1 || !(divv < 0.0)) return 0.0;
    double hp = (1.0 / cfg->N) / (cfg->k + 1);
    double a = -divv;
    double Pi = cfg->alpha * rho * hp * hp * a * a + cfg->beta * rho * c * hp * a;
    if (dt > 0.0) {
        double Pmax = 0.5 * rho * hp * hp * a / dt;
        if (Pi > Pmax) Pi = Pmax;
    }
    return Pi;
}

static double adi_pressure(double gamma, double rho, const double m[3], double e)
{
    return (gamma - 1.0) * (e - 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / rho);
}

/* projections of v and p of one cell: pc[i][l], i = v_x, v_y, v_z, p */
static void adi_project_cell(const tabs* T, double gamma, const double* uc, double* pc)
{
    int b = T->b;
    memset(pc, 0, sizeof(double) * 4 * b);
    for (int q = 0; q < T->nq; ++q) {
        const double* ph = T->phi + q * b;
        double rho = eval(T, uc, ph), m[3], f[4];
        for (int i = 0; i < 3; ++i) {
            m[i] = eval(T, uc + (1 + i) * b, ph);
            f[i] = m[i] / rho;
        }
        f[3] = adi_pressure(gamma, rho, m, eval(T, uc + 4 * b, ph));
        for (int i = 0; i < 4; ++i)
            for (int l = 0; l < b; ++l) pc[i * b + l] += 0.125 * T->wq[q] * ph[l] * f[i];
    }
}

void orc_adi_project(const orc_cfg* cfg, double gamma, const double* u, double* prim)
{
    tabs T;
    tabs_init(&T, cfg->k, cfg->k + 1);
    int N = cfg->N, b = T.b, nc = N * N * N;
    for (int c = 0; c < nc; ++c) adi_project_cell(&T, gamma, u + (size_t)c * 5 * b, prim + (size_t)c * 4 * b);
    tabs_free(&T);
}

static int adi_rhs_impl(const orc_cfg* cfg, double gamma, const double* u, const double* ahat, double dt_pimax,
                        double* dudt, double* work);

int orc_adi_rhs(const orc_cfg* cfg, double gamma, const double* u, double dt_pimax, double* dudt)
{
    return adi_rhs_impl(cfg, gamma, u, NULL, dt_pimax, dudt, NULL);
}

/* with the driving a_h [c][3][b] (Sec. 4.2): momentum source rho (a_h - abar)
 * and its work m.(a_h - abar) in the energy equation, abar = <rho a_h>/<rho>;
 * *work = the volume integral of the energy source (its cell means times h^3) */
int orc_adi_rhs_forced(const orc_cfg* cfg, double gamma, const double* u, const double* ahat, double dt_pimax,
                       double* dudt, double* work)
{
    return adi_rhs_impl(cfg, gamma, u, ahat, dt_pimax, dudt, work);
}

static int adi_rhs_impl(const orc_cfg* cfg, double gamma, const double* u, const double* ahat, double dt_pimax,
                        double* dudt, double* work)
{
    tabs T;
    tabs_init(&T, cfg->k, cfg->k + 1);
    int N = cfg->N, b = T.b, nq = T.nq, ns = T.ns;
    size_t nc = (size_t)N * N * N;
    double h = 1.0 / N;
    double* prim = (double*)malloc(sizeof(double) * nc * 4 * b);
    orc_adi_project(cfg, gamma, u, prim);
    memset(dudt, 0, sizeof(double) * nc * 5 * b);
    double abar[3] = {0, 0, 0};
    if (ahat) forcing_mean_nv(cfg, u, 5, ahat, abar);

    /* volume integral, cell by cell */
    for (size_t c = 0; c < nc; ++c) {
        const double* uc = u + c * 5 * b;
        double* rc = dudt + c * 5 * b;
        for (int q = 0; q < nq; ++q) {
            const double* ph = T.phi + q * b;
            double rho = eval(&T, uc, ph), m[3], v[3], drho[3], dmd[3];
            for (int i = 0; i < 3; ++i) {
                m[i] = eval(&T, uc + (1 + i) * b, ph);
                v[i] = m[i] / rho;
            }
            double e = eval(&T, uc + 4 * b, ph);
            double p = adi_pressure(gamma, rho, m, e);
            for (int d = 0; d < 3; ++d) {
                const double* dph = T.dphi + ((size_t)d * nq + q) * b;
                drho[d] = (2.0 / h) * eval(&T, uc, dph);
                dmd[d] = (2.0 / h) * eval(&T, uc + (1 + d) * b, dph);
            }
            double divv = (dmd[0] + dmd[1] + dmd[2] - (v[0] * drho[0] + v[1] * drho[1] + v[2] * drho[2])) / rho;
            double c_s = sqrt(gamma * p / rho);
            double P = p + orc_adi_vnr(cfg, rho, c_s, divv, dt_pimax);
            double F[5][3]; /* F[var][d] */
            for (int d = 0; d < 3; ++d) {
                F[0][d] = m[d];
                for (int i = 0; i < 3; ++i) F[1 + i][d] = m[i] * v[d] + (i == d ? P : 0.0);
                F[4][d] = (e + P) * v[d];
            }
            for (int l = 0; l < b; ++l) {
                double g[3];
                for (int d = 0; d < 3; ++d) g[d] = T.dphi[((size_t)d * nq + q) * b + l];
                for (int var = 0; var < 5; ++var)
                    rc[var * b + l] += T.wq[q] * (g[0] * F[var][0] + g[1] * F[var][1] + g[2] * F[var][2]) / (4.0 * h);
            }
            if (ahat) {
                const double* ac = ahat + c * 3 * b;
                double se = 0.0;
                for (int i = 0; i < 3; ++i) {
                    double da = eval(&T, ac + i * b, ph) - abar[i];
                    for (int l = 0; l < b; ++l) rc[(1 + i) * b + l] += 0.125 * T.wq[q] * ph[l] * rho * da;
                    se += m[i] * da;
                }
                for (int l = 0; l < b; ++l) rc[4 * b + l] += 0.125 * T.wq[q] * ph[l] * se;
            }
        }
    }
    if (work) {
        /* the volume term of mode 0 vanishes (grad phi_0 = 0): dudt[c][4][0] is the
         * cell mean of the energy source here, before the surface terms */
        double w = 0.0;
        for (size_t c = 0; c < nc; ++c) w += ahat ? dudt[c * 5 * b + 4 * b] : 0.0;
        *work = w * h * h * h;
    }

    /* surface integral: one pass over interfaces, each flux added to both cells;
     * along an axis with boundaries the interface between the last and the first
     * cell is replaced by the two boundary faces, each with its ghost state */
    for (int iz = 0; iz < N; ++iz)
        for (int iy = 0; iy < N; ++iy)
            for (int ix = 0; ix < N; ++ix) {
                int cL = cell_index(N, ix, iy, iz);
                for (int d = 0; d < 3; ++d) {
                    int cR = cell_index(N, ix + (d == 0), iy + (d == 1), iz + (d == 2));
                    const double* phL = T.phif + ((size_t)(d * 2 + 1) * ns) * b; /* xi_d = +1 in L */
                    const double* phR = T.phif + ((size_t)(d * 2 + 0) * ns) * b; /* xi_d = -1 in R */
                    const int i_d = d == 0 ? ix : (d == 1 ? iy : iz);
                    if (cfg->bc[d] != ORC_BC_PERIODIC && i_d == N - 1) {
                        adi_boundary_faces(cfg, gamma, &T, d, u, prim, cL, cR, h, dudt);
                        continue;
                    }
                    for (int s = 0; s < ns; ++s) {
                        double WL[5], WR[5], Fs[5];
                        WL[0] = eval(&T, u + (size_t)cL * 5 * b, phL + s * b);
                        WR[0] = eval(&T, u + (size_t)cR * 5 * b, phR + s * b);
                        for (int i = 0; i < 4; ++i) {
                            WL[1 + i] = eval(&T, prim + ((size_t)cL * 4 + i) * b, phL + s * b);
                            WR[1 + i] = eval(&T, prim + ((size_t)cR * 4 + i) * b, phR + s * b);
                        }
                        adi_face_flux(cfg->riemann, gamma, d, WL, WR, Fs);
                        for (int var = 0; var < 5; ++var)
                            for (int l = 0; l < b; ++l) {
                                dudt[((size_t)cL * 5 + var) * b + l] -= T.ws[s] * phL[s * b + l] * Fs[var] / (4.0 * h);
                                dudt[((size_t)cR * 5 + var) * b + l] += T.ws[s] * phR[s * b + l] * Fs[var] / (4.0 * h);
                            }
                    }
                }
            }
    free(prim);
    tabs_free(&T);
    return 0;
}

/* dt = cfl h / ((k+1) max over volume points of sum_d (|v_d| + c)) */
double orc_adi_dt(const orc_cfg* cfg, double gamma, const double* u)
{
    tabs T;
    tabs_init(&T, cfg->k, cfg->k + 1);
    int N = cfg->N, b = T.b, nc = N * N * N;
    double smax = 0.0;
    for (int c = 0; c < nc; ++c) {
        const double* uc = u + (size_t)c * 5 * b;
        for (int q = 0; q < T.nq; ++q) {
            const double* ph = T.phi + q * b;
            double rho = eval(&T, uc, ph), m[3];
            for (int i = 0; i < 3; ++i) m[i] = eval(&T, uc + (1 + i) * b, ph);
            double p = adi_pressure(gamma, rho, m, eval(&T, uc + 4 * b, ph));
            double cs = sqrt(gamma * p / rho), s = 0.0;
            for (int d = 0; d < 3; ++d) s += fabs(m[d] / rho) + cs;
            if (s > smax) smax = s;
        }
    }
    tabs_free(&T);
    return cfg->cfl * (1.0 / N) / ((cfg->k + 1) * smax);
}

/* smallest t in [0, 1] with p(ubar + t d) = eps, given p(ubar) > eps and
 * p(ubar + d) < eps: the root of the quadratic rho(t) e(t) - |m(t)|^2/2 -
 * eps rho(t)/(gamma-1) = 0 (positive at t = 0, negative at t = 1) */
static double adi_pressure_root(double gamma, double eps, const double ub[5], const double dv[5])
{
    double g1 = eps / (gamma - 1.0);
    double A = dv[0] * dv[4] - 0.5 * (dv[1] * dv[1] + dv[2] * dv[2] + dv[3] * dv[3]);
    double B = ub[0] * dv[4] + dv[0] * ub[4] - (ub[1] * dv[1] + ub[2] * dv[2] + ub[3] * dv[3]) - g1 * dv[0];
    double C = ub[0] * ub[4] - 0.5 * (ub[1] * ub[1] + ub[2] * ub[2] + ub[3] * ub[3]) - g1 * ub[0];
    double t;
    if (fabs(A) <= 1e-14 * (fabs(B) + fabs(C))) {
        t = -C / B;
    } else {
        double disc = B * B - 4.0 * A * C;
        if (disc < 0.0) disc = 0.0;
        double sq = sqrt(disc);
        double r1 = (-B - sq) / (2.0 * A), r2 = (-B + sq) / (2.0 * A);
        double lo = r1 < r2 ? r1 : r2, hi = r1 < r2 ? r2 : r1;
        t = (lo >= 0.0 && lo <= 1.0) ? lo : hi;
    }
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    return t;
}

/* positivity of density and pressure at every volume and face point (floor
 * eps = rho_floor for both): theta_rho = (rhobar - eps)/(rhobar - rho_min)
 * as in the isothermal system, then on the rho-limited state the largest
 * theta_p in [0, 1] keeping p >= eps at every point; all higher modes of all
 * variables scaled by theta_rho theta_p.  A cell mean with rho or p at or
 * below eps is a failure. */
int orc_adi_limit(const orc_cfg* cfg, double gamma, double* u)
{
    tabs T;
    tabs_init(&T, cfg->k, cfg->k + 1);
    int N = cfg->N, b = T.b, nq = T.nq, npt = T.nq + 6 * T.ns;
    size_t nc = (size_t)N * N * N;
    double eps = cfg->rho_floor;
    int status = 0;
    for (size_t c = 0; c < nc; ++c) {
        double* uc = u + c * 5 * b;
        double ub[5];
        for (int v = 0; v < 5; ++v) ub[v] = uc[v * b];
        double mb[3] = {ub[1], ub[2], ub[3]};
        if (!(ub[0] > eps) || !(adi_pressure(gamma, ub[0], mb, ub[4]) > eps)) {
            status |= ORC_FAIL;
            continue;
        }
        double rmin = INFINITY;
        for (int j = 0; j < npt; ++j) {
            const double* ph = j < nq ? T.phi + j * b : T.phif + (size_t)(j - nq) * b;
            double r = eval(&T, uc, ph);
            if (r < rmin) rmin = r;
        }
        double th_r = rmin < eps ? (ub[0] - eps) / (ub[0] - rmin) : 1.0;
        double th_p = 1.0;
        for (int j = 0; j < npt; ++j) {
            const double* ph = j < nq ? T.phi + j * b : T.phif + (size_t)(j - nq) * b;
            double uq[5], dv[5];
            for (int v = 0; v < 5; ++v) {
                uq[v] = ub[v] + th_r * (eval(&T, uc + v * b, ph) - ub[v]);
                dv[v] = uq[v] - ub[v];
            }
            double mq[3] = {uq[1], uq[2], uq[3]};
            if (adi_pressure(gamma, uq[0], mq, uq[4]) < eps) {
                double t = adi_pressure_root(gamma, eps, ub, dv);
                if (t < th_p) th_p = t;
            }
        }
        double th = th_r * th_p;
        if (th < 1.0) {
            for (int v = 0; v < 5; ++v)
                for (int l = 1; l < b; ++l) uc[v * b + l] *= th;
            status |= ORC_LIMITED;
        }
    }
    tabs_free(&T);
    return status;
}

static int adi_step_impl(const orc_cfg* cfg, double gamma, double* u, const double* ahat, double dt, double* injected);

int orc_adi_step(const orc_cfg* cfg, double gamma, double* u, double dt)
{
    return adi_step_impl(cfg, gamma, u, NULL, dt, NULL);
}

/* one step with the driving; *injected = dt sum_s beta_s W_s, the work of the
 * driving with the weights the SSP-RK scheme gives each stage's right-hand side
 * in u^(n+1) (RK2: 1/2, 1/2; RK3: 1/6, 1/6, 2/3): the change of the total
 * energy over the step */
int orc_adi_step_forced(const orc_cfg* cfg, double gamma, double* u, const double* ahat, double dt, double* injected)
{
    return adi_step_impl(cfg, gamma, u, ahat, dt, injected);
}

static int adi_step_impl(const orc_cfg* cfg, double gamma, double* u, const double* ahat, double dt, double* injected)
{
    int b = orc_nmodes(cfg->k);
    size_t n = (size_t)cfg->N * cfg->N * cfg->N * 5 * b;
    double* un = (double*)malloc(sizeof(double) * n);
    double* us = (double*)malloc(sizeof(double) * n);
    double* L = (double*)malloc(sizeof(double) * n);
    memcpy(un, u, sizeof(double) * n);
    memcpy(us, u, sizeof(double) * n);
    int status = 0;
    static const double a2[2] = {0.0, 0.5}, b2[2] = {1.0, 0.5};
    static const double a3[3] = {0.0, 0.75, 1.0 / 3.0}, b3[3] = {1.0, 0.25, 2.0 / 3.0};
    const double* A = (cfg->rk_stages == 2) ? a2 : a3;
    const double* B = (cfg->rk_stages == 2) ? b2 : b3;
    static const double w2[2] = {0.5, 0.5}, w3[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
    const double* W = (cfg->rk_stages == 2) ? w2 : w3;
    double inj = 0.0;
    for (int s = 0; s < cfg->rk_stages; ++s) {
        double work = 0.0;
        adi_rhs_impl(cfg, gamma, us, ahat, dt, L, &work);
        inj += dt * W[s] * work;
        for (size_t i = 0; i < n; ++i) us[i] = A[s] * un[i] + B[s] * (us[i] + dt * L[i]);
        status |= orc_adi_limit(cfg, gamma, us);
    }
    if (injected) *injected = inj;
    memcpy(u, us, sizeof(double) * n);
    free(un);
    free(us);
    free(L);
    return status;
}

/* nsteps steps with dt from the CFL condition of each step's start (fixed_dt
 * > 0: that dt), halved up to three times when a stage fails */
int orc_adi_run(const orc_cfg* cfg, double gamma, double* u, int nsteps, double fixed_dt, double* t, double* dt_last)
{
    int b = orc_nmodes(cfg->k);
    size_t n = (size_t)cfg->N * cfg->N * cfg->N * 5 * b;
    double* bak = (double*)malloc(sizeof(double) * n);
    int rc = 0;
    for (int st = 0; st < nsteps; ++st) {
        double dt = fixed_dt > 0.0 ? fixed_dt : orc_adi_dt(cfg, gamma, u);
        int status = ORC_FAIL;
        double dtt = dt;
        memcpy(bak, u, sizeof(double) * n);
        for (int r = 0; r <= 3; ++r) {
            dtt = dt / (double)(1 << r);
            status = orc_adi_step(cfg, gamma, u, dtt);
            if (!(status & ORC_FAIL)) break;
            memcpy(u, bak, sizeof(double) * n);
        }
        if (status & ORC_FAIL) {
            rc = -1;
            break;
        }
        *t += dtt;
        if (dt_last) *dt_last = dtt;
    }
    free(bak);
    return rc;
}

/* Uniform temperature restored after a step (Sec. 4.2: the gas is run with an
 * adiabatic index close to 1 and its thermal energy reset): in every cell e
 * becomes the projection of rho cs^2/(gamma-1) + |m|^2/(2 rho), i.e. p = cs^2 rho
 * in the projected sense.  Returns the thermal energy taken out (the volume
 * integral of the old minus the new e): the dissipated energy. */
double orc_adi_reset(const orc_cfg* cfg, double gamma, double cs, double* u)
{
    tabs T;
    tabs_init(&T, cfg->k, cfg->k + 1);
    int N = cfg->N, b = T.b, nc = N * N * N;
    double h = 1.0 / N, diss = 0.0;
    double* en = (double*)malloc(sizeof(double) * b);
    for (int c = 0; c < nc; ++c) {
        double* uc = u + (size_t)c * 5 * b;
        memset(en, 0, sizeof(double) * b);
        for (int q = 0; q < T.nq; ++q) {
            const double* ph = T.phi + q * b;
            double rho = eval(&T, uc, ph), m[3];
            for (int i = 0; i < 3; ++i) m[i] = eval(&T, uc + (1 + i) * b, ph);
            double e = rho * cs * cs / (gamma - 1.0) + 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / rho;
            for (int l = 0; l < b; ++l) en[l] += 0.125 * T.wq[q] * ph[l] * e;
        }
        diss += uc[4 * b] - en[0];
        memcpy(uc + 4 * b, en, sizeof(double) * b);
    }
    free(en);
    tabs_free(&T);
    return diss * h * h * h;
}

/* driven run of the adiabatic system with the isothermal reset (cs > 0) after
 * every step: the driving schedule of orc_run, dt from the CFL condition (or
 * fixed_dt), retries on failure; accumulates the injected and dissipated
 * energies */
int orc_adi_run_driven(const orc_cfg* cfg, double gamma, double cs, double* u, orc_ou* ou, int use_forcing,
                       double* ahat, int nsteps, double fixed_dt, double* t, double* dt_last, double* injected,
                       double* dissipated)
{
    int b = orc_nmodes(cfg->k);
    size_t n = (size_t)cfg->N * cfg->N * cfg->N * 5 * b;
    double* bak = (double*)malloc(sizeof(double) * n);
    double* amp = (double*)malloc(sizeof(double) * ORC_MAX_MODES * 6);
    int rc = 0;
    for (int st = 0; st < nsteps; ++st) {
        const double* force = NULL;
        if (use_forcing && ou->on && ou->t_off > 0.0 && *t > ou->t_off) ou->on = 0;
        if (use_forcing && ou->on) {
            while (*t >= ou->t_next) {
                orc_ou_advance(ou);
                ou->t_next += ou->dt_drive;
                ou->dirty = 1;
            }
            if (ou->dirty) {
                orc_ou_amplitudes(ou, amp);
                orc_forcing_project(cfg, ou->nmodes, &ou->kvec[0][0], amp, ahat);
                ou->dirty = 0;
            }
            force = ahat;
        }
        double dt = fixed_dt > 0.0 ? fixed_dt : orc_adi_dt(cfg, gamma, u);
        int status = ORC_FAIL;
        double dtt = dt, inj = 0.0;
        memcpy(bak, u, sizeof(double) * n);
        for (int r = 0; r <= 3; ++r) {
            dtt = dt / (double)(1 << r);
            status = adi_step_impl(cfg, gamma, u, force, dtt, &inj);
            if (!(status & ORC_FAIL)) break;
            memcpy(u, bak, sizeof(double) * n);
        }
        if (status & ORC_FAIL) {
            rc = -1;
            break;
        }
        *injected += inj;
        if (cs > 0.0) *dissipated += orc_adi_reset(cfg, gamma, cs, u);
        *t += dtt;
        if (dt_last) *dt_last = dtt;
    }
    free(bak);
    free(amp);
    return rc;
}

/* number of threads of the parallel loops (OpenMP; 1 without it) */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
