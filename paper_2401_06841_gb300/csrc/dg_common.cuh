// dg_common.cuh -- compile-time basis description and pointwise physics shared
// by the kernels of libdg (sm_103a).
//
// Basis (Sec. 2.1): phi_{ijl}(xi) = Pn_i(xi_x) Pn_j(xi_y) Pn_l(xi_z),
// Pn_m = sqrt(2m+1) P_m, complete degree-k set, ordered by total degree, then i
// descending, then j descending.  (1/8) int phi_a phi_b = delta_ab.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace dg {

// largest mesh: N^3 cell indices fit in 32 bits
constexpr int kMaxN = 1024;

template <int K>
struct Dims {
    static constexpr int n = K + 1;                          // Gauss points per axis
    static constexpr int b = (K + 1) * (K + 2) * (K + 3) / 6;  // modes per field
    static constexpr int nq = n * n * n;                     // volume points
    static constexpr int ns = n * n;                         // points per face
    static constexpr int nf = 6 * ns;                        // face points per cell
    static constexpr int nl = K + 3;                         // L1-norm points per axis
    static constexpr int nql = nl * nl * nl;
};

template <int K>
struct Modes {
    int i[Dims<K>::b], j[Dims<K>::b], l[Dims<K>::b];
    constexpr Modes() : i{}, j{}, l{}
    {
        int c = 0;
        for (int d = 0; d <= K; ++d)
            for (int a = d; a >= 0; --a)
                for (int e = d - a; e >= 0; --e) {
                    i[c] = a;
                    j[c] = e;
                    l[c] = d - a - e;
                    ++c;
                }
    }
};

constexpr double csqrt(double x)
{
    if (x <= 0.0) return 0.0;
    double r = x > 1.0 ? x : 1.0;
    for (int it = 0; it < 200; ++it) r = 0.5 * (r + x / r);
    return r;
}

// (1/2) int_{-1}^{1} Pn_a(t) Pn_b'(t) dt: Pn_b' = sum_{a<b, a+b odd} sqrt((2a+1)(2b+1)) Pn_a
constexpr double dcoef(int a, int b) { return (a < b && ((a + b) & 1)) ? csqrt((2.0 * a + 1.0) * (2.0 * b + 1.0)) : 0.0; }

// Modal differentiation matrix D_d[m][l] = (1/8) int phi_m dphi_l/dxi_d.  The
// derivative of a degree-k polynomial stays in the span, so
//   d/dxi_d (sum_l c_l phi_l) = sum_m (sum_l D_d[m][l] c_l) phi_m   exactly.
template <int K>
constexpr double Dmat(int d, int m, int l)
{
    constexpr Modes<K> M{};
    int am[3] = {M.i[m], M.j[m], M.l[m]};
    int al[3] = {M.i[l], M.j[l], M.l[l]};
    for (int e = 0; e < 3; ++e)
        if (e != d && am[e] != al[e]) return 0.0;
    return dcoef(am[d], al[d]);
}

template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F&& f)
{
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

// g = scale * D_d c   (gradient coefficients of one field)
template <typename T, int K, int D>
__device__ __forceinline__ void modal_grad(const T* c, T* g, T scale)
{
    constexpr int b = Dims<K>::b;
    static_for<0, b>([&](auto m) {
        T acc = T(0);
        static_for<0, b>([&](auto l) {
            constexpr double v = Dmat<K>(D, decltype(m)::value, decltype(l)::value);
            if constexpr (v != 0.0) acc += T(v) * c[decltype(l)::value];
        });
        g[decltype(m)::value] = acc * scale;
    });
}

// r += scale * D_d^T f   (weak-form volume term from projected flux coefficients)
template <typename T, int K, int D>
__device__ __forceinline__ void modal_grad_T_acc(const T* f, T* r, T scale)
{
    constexpr int b = Dims<K>::b;
    static_for<0, b>([&](auto l) {
        T acc = T(0);
        static_for<0, b>([&](auto m) {
            constexpr double v = Dmat<K>(D, decltype(m)::value, decltype(l)::value);
            if constexpr (v != 0.0) acc += T(v) * f[decltype(m)::value];
        });
        r[decltype(l)::value] += acc * scale;
    });
}

// ---------------------------------------------------------------------------
// control block in the caller's scratch (FP64 global quantities)
// ---------------------------------------------------------------------------
// 1D Gauss rule on [-1, 1] (n = k+1 <= 4 points)
struct Rule1 {
    double x[4], w[4];
};

struct Ctl {
    unsigned int status;     // sticky DG_ST_* bits
    unsigned int cnt_proj;   // last-block counter of the projection kernel
    unsigned int cnt_diag;   // last-block counter of diagnostics / L1
    unsigned int pad0;
    unsigned long long smax; // bits of max sum_d(|v_d|+cs) (positive double)
    double dt;               // dt of the current step (fixes Pi_max), written for the host
    double dt_scale;         // 1, 1/2, 1/4, 1/8 on retries
    double fixed_dt;         // > 0 replaces the CFL dt
    double abar2[2][3];      // <rho a_h>/<rho>, one slot per projected-velocity buffer
    double dt_num;           // cfl h / (k+1)
    double diag[16];         // diagnostics result
    double l1;               // L1 result
    double sn;               // max sum_d(|v_d|+cs) of the state the next step starts from
    double dt_diff;          // explicit diffusion limit cfl (h/(k+1))^2 / (2 eps), 0: none
    unsigned long long tiles_vol, tiles_gated;  // volume-term tiles, and those the learned gate spared div v
};

// kernel flags
enum { F_DT = 1, F_FORCE = 2 };

#define DG_ST_LIMITED_ 1u
#define DG_ST_FAIL_ 2u
#define DG_ST_NONFINITE_ 4u
// positivity by repetition (internal, never reported): a stage marked a
// troubled cell; the flattening found a flat cell with negative density, and
// scaled some cell
#define DG_ST_TROUBLED_ 0x100u
#define DG_ST_FLAT_ 0x200u
#define DG_ST_SCALED_ 0x400u
// per-cell marks: negative density at a Gauss point of a stage output (before
// its rescaling); a volume point of a stage output faster than the bound
#define DG_MARK_NEGATIVE 1u
#define DG_MARK_FAST 2u
// a stage output whose volume-point sum_d(|v_d| + cs) exceeds this factor times
// the bound that set dt troubles its cell
#define DG_REPEAT_SPEED 1.5
#define DG_NDIAG 13

// ---------------------------------------------------------------------------
// pointwise physics
// ---------------------------------------------------------------------------
struct Phys {
    double cs, cs2, h, hp;       // sound speed, cs^2, cell size, h/(k+1)
    double alpha, beta, floor_;  // vNR coefficients, density floor
    int av_mode;                 // 0 off, 1 vNR, 2 learned
    int riemann;                 // face flux: 0 Rusanov, 1 HLL, 2 HLLC
    double nu_gate;              // learned sensor: nu/(cs h/p) below this -> no viscous pressure
    double eps;                  // diffusion coefficient of div(eps grad u), 0: off
    // recovered face derivative d r/ds at the face (s in half cells) from the
    // K+1 normal coefficients of the left and right cell: sum_a recL[K][a] cL_a + recR[K][a] cR_a
    double recL[4][4], recR[4][4];
};

// von Neumann-Richtmyer viscous pressure at a volume point (Sec. 3.1):
// Pi = alpha rho (h/p)^2 D^2 + beta rho cs (h/p) |D| for D = div v < 0,
// limited by rho (h/p)^2 |D| / (2 dt); zero otherwise.  dt <= 0: no limit.
template <typename T>
__device__ __forceinline__ T vnr_pressure(const Phys& P, T rho, T divv, T dt)
{
    if (!(divv < T(0))) return T(0);
    T a = -divv, hp = T(P.hp);
    T Pi = T(P.alpha) * rho * hp * hp * a * a + T(P.beta) * rho * T(P.cs) * hp * a;
    if (dt > T(0)) {
        T Pmax = T(0.5) * rho * hp * hp * a / dt;
        Pi = Pi < Pmax ? Pi : Pmax;
    }
    return Pi;
}

// the same viscous pressure with the coefficients folded once per launch:
//   Pi = rho a (a2 a + b1),  a = -div v > 0,  a2 = alpha (h/p)^2, b1 = beta cs (h/p),
//   Pi <- min(Pi, rho a cap) with cap = (h/p)^2 / (2 dt) (cap < 0: no cap)
template <typename T>
struct AvCoef {
    T a2, b1, cap;
};
template <typename T>
__host__ __device__ inline AvCoef<T> av_coef(const Phys& P, double dt)
{
    AvCoef<T> c;
    c.a2 = T(P.alpha * P.hp * P.hp);
    c.b1 = T(P.beta * P.cs * P.hp);
    c.cap = dt > 0.0 ? T(0.5 * P.hp * P.hp / dt) : T(-1);
    return c;
}
template <typename T>
__device__ __forceinline__ T vnr_pressure(const AvCoef<T>& c, T rho, T divv)
{
    if (!(divv < T(0))) return T(0);
    const T ra = rho * (-divv);
    T Pi = ra * (c.a2 * (-divv) + c.b1);
    if (c.cap >= T(0)) {
        // the cap compares the pressures themselves (rho may be negative at a
        // point of a state the limiter has not seen yet)
        const T Pm = ra * c.cap;
        Pi = Pi < Pm ? Pi : Pm;
    }
    return Pi;
}

// Rusanov flux along +e_d, left/right primitive states (rho, v):
//   F* = (F(U_L) + F(U_R))/2 - lambda (U_R - U_L)/2,
//   lambda = max(|v_d^L|, |v_d^R|) + cs, F(U) = (rho v_d, rho v_i v_d + cs^2 rho delta_id)
template <typename T, int D>
__device__ __forceinline__ void rusanov(T cs, T cs2, const T WL[4], const T WR[4], T F[4])
{
    T UL[4], UR[4];
    UL[0] = WL[0];
    UR[0] = WR[0];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        UL[1 + i] = WL[0] * WL[1 + i];
        UR[1 + i] = WR[0] * WR[1 + i];
    }
    T vl = WL[1 + D], vr = WR[1 + D];
    T lam = fmax(fabs(vl), fabs(vr)) + cs;
    T FL[4], FR[4];
    FL[0] = UL[1 + D];
    FR[0] = UR[1 + D];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        FL[1 + i] = UL[1 + i] * vl + (i == D ? cs2 * WL[0] : T(0));
        FR[1 + i] = UR[1 + i] * vr + (i == D ? cs2 * WR[0] : T(0));
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) F[v] = T(0.5) * (FL[v] + FR[v]) - T(0.5) * lam * (UR[v] - UL[v]);
}

// HLL flux along +e_d with the Davis bounds S_L = min(v_d^L, v_d^R) - cs,
// S_R = max(v_d^L, v_d^R) + cs: the upwind flux when both bounds have one sign,
// else (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L).  With CONTACT
// (HLLC for p = cs^2 rho, the paper's solver) the mass and normal-momentum
// fluxes stay HLL's and the tangential momenta cross the face with the mass
// flux at the tangential velocity of the side the contact wave
// S_M = m_d*/rho* (HLL averages) leaves behind.
template <typename T, int D, bool CONTACT>
__device__ __forceinline__ void hll(T cs, T cs2, const T WL[4], const T WR[4], T F[4])
{
    const T vl = WL[1 + D], vr = WR[1 + D];
    const T SL = fmin(vl, vr) - cs, SR = fmax(vl, vr) + cs;
    T UL[4], UR[4], FL[4], FR[4];
    UL[0] = WL[0];
    UR[0] = WR[0];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        UL[1 + i] = WL[0] * WL[1 + i];
        UR[1 + i] = WR[0] * WR[1 + i];
    }
    FL[0] = UL[1 + D];
    FR[0] = UR[1 + D];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        FL[1 + i] = UL[1 + i] * vl + (i == D ? cs2 * WL[0] : T(0));
        FR[1 + i] = UR[1 + i] * vr + (i == D ? cs2 * WR[0] : T(0));
    }
    if (SL >= T(0)) {
#pragma unroll
        for (int v = 0; v < 4; ++v) F[v] = FL[v];
        return;
    }
    if (SR <= T(0)) {
#pragma unroll
        for (int v = 0; v < 4; ++v) F[v] = FR[v];
        return;
    }
    const T inv = T(1) / (SR - SL);
#pragma unroll
    for (int v = 0; v < 4; ++v) F[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) * inv;
    if constexpr (CONTACT) {
        const T rs = (SR * UR[0] - SL * UL[0] - (FR[0] - FL[0])) * inv;
        const T ms = (SR * UR[1 + D] - SL * UL[1 + D] - (FR[1 + D] - FL[1 + D])) * inv;
        const T* Wup = (ms / rs >= T(0)) ? WL : WR;
#pragma unroll
        for (int t = 0; t < 3; ++t)
            if (t != D) F[1 + t] = F[0] * Wup[1 + t];
    }
}

// the face flux selected by Phys::riemann (uniform over a launch)
template <typename T, int D>
__device__ __forceinline__ void riemann_flux(int solver, T cs, T cs2, const T WL[4], const T WR[4], T F[4])
{
    if (solver == 2)
        hll<T, D, true>(cs, cs2, WL, WR, F);
    else if (solver == 1)
        hll<T, D, false>(cs, cs2, WL, WR, F);
    else
        rusanov<T, D>(cs, cs2, WL, WR, F);
}

// ---------------------------------------------------------------------------
// table layout (element type T) in the caller's scratch, per degree
// ---------------------------------------------------------------------------
template <int K>
struct TabLayout {
    using D = Dims<K>;
    static constexpr int phiT = 0;                              // [b][nq]   phi_l(xi_q)
    static constexpr int wphi = phiT + D::b * D::nq;            // [nq][b]   w_q/8 phi_l(xi_q)
    static constexpr int phifT = wphi + D::nq * D::b;           // [b][nf]   phi_l on face points
    static constexpr int lift = phifT + D::b * D::nf;           // [nf][b]   -sign_f w_s phi_l
    static constexpr int wq = lift + D::nf * D::b;              // [nq]      w_q/8
    static constexpr int phiL = wq + D::nq;                     // [b][nql]  phi_l at L1 points
    static constexpr int wL = phiL + D::b * D::nql;             // [nql]     w/8 at L1 points
    static constexpr int xq = wL + D::nql;                      // [nq][3]   reference coords
    static constexpr int total = xq + 3 * D::nq;
};

}  // namespace dg
