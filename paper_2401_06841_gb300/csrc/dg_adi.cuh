// dg_adi.cuh -- kernels of the adiabatic system (Sec. 2.1): five conserved
// variables u = (rho, m, e) per cell with the ideal-gas equation of state
// p = (gamma - 1)(e - |m|^2 / (2 rho)) and the flux
//   F_d = (m_d, m v_d + p e_d, (e + p) v_d).
// Tile-batched like the isothermal kernels (TC cells per block iteration,
// CUDA-core block products against the same basis tables), FP32 or FP64.
//
// Modes of k_adi:
//   ADI_PROJECT  projections of v and p of u_in (Sec. 3.2) -> pr_out, with the
//                CFL bound max sum_d(|v_d| + c) over the volume points (F_DT)
//   ADI_RHS      right-hand side of u_in -> out
//   ADI_STAGE    right-hand side, SSP-RK stage combine, positivity of density
//                and pressure (Sec. 3.1) -> out = u^(s+1); with F_NEXTPROJ also
//                the projections of u^(s+1) -> pr_out (the next stage's pr_in)
//   ADI_RESET    uniform temperature restored in place (Sec. 4.2): e becomes the
//                projection of rho cs^2/(gamma-1) + |m|^2/(2 rho)
// The right-hand side needs the projections of u_in in pr_in.  With the
// driving (F_FORCE, a_h in ahat) the right-hand side adds rho (a_h - abar) to
// the momentum and its work m.(a_h - abar) to the energy; abar = <rho a_h> /
// <rho> comes from the projections (FP64 sums, deterministic last-block
// reduction into ctl->abar2[abar_out]).  FP64 accumulators in ctl->diag:
// [1] injected energy (stage: beta_s dt times the volume integral of the energy
// source), [2] dissipated energy (reset: the thermal energy taken out).
#pragma once

#include "../../include/dg.h"
#include "dg_launch.cuh"
#include "dg_tile.cuh"

namespace dg {

// gas constants in the element type, each rounded once from its double value on
// the host: near gamma = 1 the difference gamma - 1 formed in single precision
// would carry the rounding of gamma (float(1.0001) - 1 = 1.000166e-4).
// Energy offset: the fifth variable is stored as e_s = e - kap rho (kap = cs^2 /
// (gamma - 1) in reset mode, 0 otherwise), so that the thermal energy of the
// isothermal reference, 1/(gamma - 1) times larger than the kinetic energy, is
// not carried in the state: p = (gamma - 1)(e_s - |m|^2/(2 rho)) + c0 rho with
// c0 = (gamma - 1) kap, the energy flux (e_s + p) v, and the projected pressure
// is the deviation p - c0 rho.  The scheme is linear in the state, so this is
// the same discretisation in other variables.
template <typename T>
struct AdiGas {
    T gamma;   // gamma
    T g1;      // gamma - 1
    T ig1;     // 1 / (gamma - 1)
    T cth;     // reset mode: cs^2 / (gamma - 1), the thermal energy per unit mass
    T kap;     // energy offset per unit mass
    T c0;      // (gamma - 1) kap: the pressure of the offset per unit density
    T cres;    // cth - kap: the thermal energy per unit mass the reset leaves in e_s
    T fill_e;  // e_s of the filler state rho = 1, v = 0, p = 1: (1 - c0)/(gamma - 1)
};

template <typename T>
struct AdiArgs {
    const T* u_in;   // [c][5][b]
    const T* u_n;    // u^n (stage mode)
    T* out;          // dudt or u^(s+1) [c][5][b]
    const T* pr_in;  // [c][4][b] projections of v_x, v_y, v_z, p of u_in
    T* pr_out;       // projection mode output [c][4][b]
    const T* tab;    // TileTab<K, BK_FMA> tables of the element type
    Ctl* ctl;
    long ncell;
    int N;
    Phys ph;         // h, hp, alpha, beta, floor_ (density and pressure floor), av_mode
    double gamma;
    AdiGas<T> gas;   // gamma, gamma - 1, 1/(gamma - 1), cs_reset^2/(gamma - 1) rounded from doubles
    T rk_a, rk_b;
    double dt_pimax; // right-hand-side mode: dt of the viscous-pressure cap
    int flags;       // F_DT (projection mode), F_NEXTPROJ (stage mode), F_FORCE
    const T* ahat;   // [c][3][b] driving (F_FORCE)
    double* partials;  // [grid][16] block partials of the last-block reductions
    int abar_in, abar_out;  // slots of ctl->abar2 read by the right-hand side / written by a projection
    double beta;     // stage mode: weight of this stage's right-hand side in u^(n+1)
    double cs_reset; // reset mode: the isothermal sound speed
    int bc[3];       // boundaries per axis (DG_BC_*)
    double inflow[5];  // DG_BC_INFLOW: rho, v_x, v_y, v_z, p at the face at coordinate 0
};

constexpr int cmax(int a, int b) { return a > b ? a : b; }

// DRIVEN: the right-hand side carries the driving's source rows (4 more
// projected rows per cell); the undriven kernels are compiled without them
template <int K, bool DRIVEN = false>
struct AdiCfg {
    using C = TileCfg<K, BK_FMA>;
    static constexpr int b = C::b, nq = C::nq, ns = C::ns, nf = C::nf, TC = C::TC, NT = C::NT;
    static constexpr int KP = C::KP, NQP = C::NQP, NP = C::NP, B2K = C::B2K, NSP = C::NSP, B2N = C::B2N;
    // evaluated rows per cell: rho, m_x, m_y, m_z, e, grad rho (3), div m; driven: a_h (3)
    static constexpr int FE = DRIVEN ? 12 : 9;
    // m v + P (6), (e + P) v (3); driven: rho (a - abar) (3), m.(a - abar)
    static constexpr int FP = DRIVEN ? 13 : 9;
    static constexpr int LDA = KP, LDV = NQP + 4, LDP = NP, LDC2 = B2K, LDT = NSP + 4, LDL = B2N;
    static constexpr int RE = TC * FE, RP = TC * FP;
    static constexpr int RC = TC * 20;  // face rows ((cell, side, self/neighbour), (rho, v_x, v_y, v_z, p))
    static constexpr int RL = TC * 10;  // flux rows ((cell, side), variable)
    static constexpr int oU = r4(C::tabsz);
    static constexpr int oPr = oU + r4(TC * 5 * b);
    static constexpr int oR = oPr + r4(TC * 4 * b);
    static constexpr int oAh = oR + r4(TC * 5 * b);
    static constexpr int oA = oAh + r4(TC * 3 * b);
    static constexpr int SZA = cmax(RE * LDA, RP * LDP);
    static constexpr int oBig = oA + r4(SZA);
    static constexpr int FA = cmax(RC * LDC2, RL * LDT);
    static constexpr int FB = cmax(RC * LDT, RL * LDL);
    static constexpr int BIG = cmax(cmax(RE * LDV, RP * LDV), FA + FB);
    static constexpr int total = oBig + BIG;
};

// Rusanov flux along Dd from primitive face states W = (rho, v_x, v_y, v_z, p - c0 rho):
// 1/2 (F(U_L) + F(U_R)) - 1/2 lambda (U_R - U_L), lambda = max(|v_n| + c)
template <typename T, int Dd>
__device__ __forceinline__ void adi_rusanov(const AdiGas<T>& G, const T* WL, const T* WR, T* F)
{
    const T g1 = G.g1, gamma = G.gamma;
    T UL[5], UR[5], FL[5], FR[5], ls[2];
    const T* W[2] = {WL, WR};
    T* U[2] = {UL, UR};
    T* Fx[2] = {FL, FR};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const T* w = W[s];
        const T rho = w[0], vn = w[1 + Dd], p = w[4] + G.c0 * rho;  // w[4]: the pressure deviation
        U[s][0] = rho;
        U[s][1] = rho * w[1];
        U[s][2] = rho * w[2];
        U[s][3] = rho * w[3];
        U[s][4] = w[4] / g1 + T(0.5) * rho * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
        Fx[s][0] = U[s][1 + Dd];
        Fx[s][1] = U[s][1] * vn;
        Fx[s][2] = U[s][2] * vn;
        Fx[s][3] = U[s][3] * vn;
        Fx[s][1 + Dd] += p;
        Fx[s][4] = (U[s][4] + p) * vn;
        ls[s] = fabs(vn) + sqrt(gamma * p / rho);
    }
    // the larger of the two (a NaN of the right state propagates, as in the oracle)
    const T lam = ls[0] > ls[1] ? ls[0] : ls[1];
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = T(0.5) * (FL[v] + FR[v]) - T(0.5) * lam * (UR[v] - UL[v]);
}

// HLLC flux along Dd from primitive face states (the contact wave restored in
// the two-wave model): Davis bounds S_L = min(u - c), S_R = max(u + c) over the
// two states, the contact speed S* from the pressures and the mass fluxes
// relative to the bounds, star states U*_K = rho_K (S_K - u_K)/(S_K - S*)
// (1, S* along Dd, the tangential velocities, E_K/rho_K + (S* - u_K)(S* +
// p_K/(rho_K (S_K - u_K)))), and the flux of the region x/t = 0 falls in
template <typename T, int Dd>
__device__ __forceinline__ void adi_hllc(const AdiGas<T>& G, const T* WL, const T* WR, T* F)
{
    const T g1 = G.g1, gamma = G.gamma;
    T U[2][5], Fx[2][5], c[2], un[2], pp[2];
    const T* W[2] = {WL, WR};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const T* w = W[s];
        const T rho = w[0], p = w[4] + G.c0 * rho;  // w[4]: the pressure deviation
        pp[s] = p;
        un[s] = w[1 + Dd];
        U[s][0] = rho;
        U[s][1] = rho * w[1];
        U[s][2] = rho * w[2];
        U[s][3] = rho * w[3];
        U[s][4] = w[4] / g1 + T(0.5) * rho * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
        Fx[s][0] = U[s][1 + Dd];
        Fx[s][1] = U[s][1] * un[s];
        Fx[s][2] = U[s][2] * un[s];
        Fx[s][3] = U[s][3] * un[s];
        Fx[s][1 + Dd] += p;
        Fx[s][4] = (U[s][4] + p) * un[s];
        c[s] = sqrt(gamma * p / rho);
    }
    const T a0 = un[0] - c[0], a1 = un[1] - c[1], b0 = un[0] + c[0], b1 = un[1] + c[1];
    const T SL = a0 < a1 ? a0 : a1, SR = b0 > b1 ? b0 : b1;
    if (SL >= T(0)) {
#pragma unroll
        for (int v = 0; v < 5; ++v) F[v] = Fx[0][v];
        return;
    }
    if (SR <= T(0)) {
#pragma unroll
        for (int v = 0; v < 5; ++v) F[v] = Fx[1][v];
        return;
    }
    const T qL = WL[0] * (SL - un[0]), qR = WR[0] * (SR - un[1]);
    const T Ss = (pp[1] - pp[0] + un[0] * qL - un[1] * qR) / (qL - qR);
    // the side of the contact x/t = 0 lies on (selects keep everything in registers)
    const bool lft = Ss >= T(0);
    const T SK = lft ? SL : SR, qK = lft ? qL : qR, uK = lft ? un[0] : un[1], pK = lft ? pp[0] : pp[1];
    T wK[5], UK[5], FK[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        wK[v] = lft ? WL[v] : WR[v];
        UK[v] = lft ? U[0][v] : U[1][v];
        FK[v] = lft ? Fx[0][v] : Fx[1][v];
    }
    const T f = qK / (SK - Ss);
    T Us[5];
    Us[0] = f;
#pragma unroll
    for (int i = 0; i < 3; ++i) Us[1 + i] = f * (i == Dd ? Ss : wK[1 + i]);
    Us[4] = f * (UK[4] / wK[0] + (Ss - uK) * (Ss + pK / qK));
#pragma unroll
    for (int v = 0; v < 5; ++v) F[v] = FK[v] + SK * (Us[v] - UK[v]);
}

// vNR viscous pressure with the local sound speed c in the bulk term
template <typename T>
__device__ __forceinline__ T adi_vnr(const Phys& P, T rho, T c, T divv, T dt)
{
    if (P.av_mode != 1 || !(divv < T(0))) return T(0);
    const T a = -divv, hp = T(P.hp);
    T Pi = T(P.alpha) * rho * hp * hp * a * a + T(P.beta) * rho * c * hp * a;
    if (dt > T(0)) {
        const T Pm = T(0.5) * rho * hp * hp * a / dt;
        Pi = Pi > Pm ? Pm : Pi;
    }
    return Pi;
}

// smallest t in [0, 1] with p(ub + t d) = eps (p(ub) > eps > p(ub + d)): the
// root of rho p - eps rho = (gamma-1)(rho e_s - |m|^2/2) + c0 rho^2 - eps rho,
// quadratic in t
template <typename T>
__device__ __forceinline__ T adi_pressure_root(const AdiGas<T>& G, T eps, const T* ub, const T* dv)
{
    const T g1 = G.g1, c0 = G.c0;
    const T A = g1 * (dv[0] * dv[4] - T(0.5) * (dv[1] * dv[1] + dv[2] * dv[2] + dv[3] * dv[3])) + c0 * dv[0] * dv[0];
    const T B = g1 * (ub[0] * dv[4] + dv[0] * ub[4] - (ub[1] * dv[1] + ub[2] * dv[2] + ub[3] * dv[3])) +
                T(2) * c0 * ub[0] * dv[0] - eps * dv[0];
    const T C = g1 * (ub[0] * ub[4] - T(0.5) * (ub[1] * ub[1] + ub[2] * ub[2] + ub[3] * ub[3])) + c0 * ub[0] * ub[0] -
                eps * ub[0];
    T t;
    if (fabs(A) <= T(1e-14) * (fabs(B) + fabs(C))) {
        t = -C / B;
    } else {
        T disc = B * B - T(4) * A * C;
        disc = disc < T(0) ? T(0) : disc;
        const T sq = sqrt(disc);
        const T r1 = (-B - sq) / (T(2) * A), r2 = (-B + sq) / (T(2) * A);
        const T lo = r1 < r2 ? r1 : r2, hi = r1 < r2 ? r2 : r1;
        t = (lo >= T(0) && lo <= T(1)) ? lo : hi;
    }
    t = t < T(0) ? T(0) : t;
    return t > T(1) ? T(1) : t;
}

// pressure from the stored variables (e: the offset energy e_s), and its
// deviation p - c0 rho
template <typename T>
__device__ __forceinline__ T adi_pdev(const AdiGas<T>& G, T rho, T mx, T my, T mz, T e)
{
    return G.g1 * (e - T(0.5) * (mx * mx + my * my + mz * mz) / rho);
}
template <typename T>
__device__ __forceinline__ T adi_p(const AdiGas<T>& G, T rho, T mx, T my, T mz, T e)
{
    return adi_pdev<T>(G, rho, mx, my, mz, e) + G.c0 * rho;
}

// copy n elements (a multiple of 4) of a tile from global to shared; elements
// past `valid` get the filler state of a cell (rho = 1, v = 0, p = 1)
template <typename T, int NT, int NV, int B>
__device__ __forceinline__ void adi_load(T* dst, const T* src, int n, int valid, T fill_e)
{
    for (int e = 4 * threadIdx.x; e < n; e += 4 * NT) {
        T v[4];
        ld4_guard<T>(src, e, valid, v);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (e + j >= valid) {
                const int r = (e + j) % (NV * B);
                v[j] = (r == 0) ? T(1) : (NV == 5 && r == 4 * B) ? fill_e : T(0);
            }
        }
        st4<T>(dst + e, v);
    }
}

// projections of v and p of the TC states in sU (Sec. 3.2) -> a.pr_out, and
// with F_DT the CFL bound max sum_d(|v_d| + c) over the volume points of the
// valid cells into smax.  Starts and ends with the block in step.
template <typename T, int K, bool DRIVEN>
__device__ __forceinline__ void adi_project_tile(T* sm, const T* sU, const T* tabs, const AdiArgs<T>& a, long c0,
                                                 int nvalid, T gamma, T& smax, double* sums)
{
    using A = AdiCfg<K, DRIVEN>;
    using C = TileCfg<K, BK_FMA>;
    constexpr int b = A::b, nq = A::nq, TC = A::TC, NT = A::NT, KP = A::KP, NQP = A::NQP, NP = A::NP;
    constexpr int LDA = A::LDA, LDV = A::LDV, LDP = A::LDP;
    const int tid = threadIdx.x;
    T* sA = sm + A::oA;
    T* sP = sA;
    T* sBig = sm + A::oBig;
    // rho, m, e at the volume points
    for (int e = tid; e < TC * 5 * KP; e += NT) {
        const int r = e / KP, l = e % KP;
        sA[r * LDA + l] = l < b ? sU[r * b + l] : T(0);
    }
    __syncthreads();
    mm<T, BK_FMA, TC * 5, NQP, KP, LDA, LDV, NT>(sA, tabs, C::oPhi, sBig);
    __syncthreads();
    constexpr int PER = (TC * NQP + NT - 1) / NT;
    T f[PER][4];
#pragma unroll
    for (int it = 0; it < PER; ++it) {
        const int e = tid + it * NT;
#pragma unroll
        for (int i = 0; i < 4; ++i) f[it][i] = T(0);
        if (e < TC * NQP) {
            const int c = e / NQP, q = e % NQP;
            if (q < nq) {
                const T* v = sBig + (c * 5) * LDV + q;
                const T rho = v[0], ir = rcp<T>(rho);
                const T mx = v[LDV], my = v[2 * LDV], mz = v[3 * LDV];
                f[it][0] = mx * ir;
                f[it][1] = my * ir;
                f[it][2] = mz * ir;
                f[it][3] = adi_pdev<T>(a.gas, rho, mx, my, mz, v[4 * LDV]);  // projected: p - c0 rho
                if ((a.flags & F_DT) && c < nvalid) {
                    const T cs = sqrt(gamma * (f[it][3] + a.gas.c0 * rho) * ir);
                    const T sp = fabs(f[it][0]) + fabs(f[it][1]) + fabs(f[it][2]) + T(3) * cs;
                    smax = sp > smax ? sp : smax;
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < PER; ++it) {
        const int e = tid + it * NT;
        if (e < TC * NQP) {
            const int c = e / NQP, q = e % NQP;
#pragma unroll
            for (int i = 0; i < 4; ++i) sBig[(c * 4 + i) * LDV + q] = f[it][i];
        }
    }
    __syncthreads();
    mm<T, BK_FMA, TC * 4, NP, NQP, LDV, LDP, NT>(sBig, tabs, C::oWPhi, sP);
    __syncthreads();
    for (int e = tid; e < nvalid * 4 * b; e += NT) {
        const int r = e / b, l = e % b;
        a.pr_out[c0 * 4 * b + e] = sP[r * LDP + l];
    }
    // driving: <rho a_h> = sum_l rho_l a_l per cell (orthonormal basis) and <rho>
    if ((a.flags & F_FORCE) && tid < TC * 3) {
        const int c = tid / 3, i = tid % 3;
        if (c < nvalid) {
            const T* ah = sm + A::oAh + (c * 3 + i) * b;
            T s = T(0);
#pragma unroll
            for (int l = 0; l < b; ++l) s += sU[c * 5 * b + l] * ah[l];
            sums[i] += (double)s;
            if (i == 0) sums[3] += (double)sU[c * 5 * b];
        }
    }
    __syncthreads();
}

// sum over the block of one FP64 value per thread, then over the blocks in a
// fixed order (last-block reduction, no waiting): true in the last block, with
// the total in *tot
template <int NT>
__device__ __forceinline__ bool adi_reduce(double* partials, double* s_buf, double* s_tot, unsigned int* counter,
                                           const double* v, int nv)
{
    double mine[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < nv; ++i) {
        s_buf[threadIdx.x] = v[i];
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int j = 0; j < NT; ++j) t += s_buf[j];
            mine[i] = t;
        }
        __syncthreads();
    }
    return last_block_reduce<NT>(partials, mine, nv, counter, s_tot, s_buf);
}

// FP32: two blocks per SM (128 registers); FP64 fits one block in shared memory.
// DRIVEN (right-hand-side modes): the driving's source rows are compiled in
template <typename T, int K, int MODE, bool DRIVEN = false>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_adi(AdiArgs<T> a)
{
    using A = AdiCfg<K, DRIVEN>;
    static_assert(AdiCfg<K, false>::oAh == A::oAh && AdiCfg<K, false>::oA == A::oA, "same leading layout");
    using C = TileCfg<K, BK_FMA>;
    using TT = TileTab<K, BK_FMA>;
    constexpr int b = A::b, nq = A::nq, ns = A::ns, nf = A::nf, TC = A::TC, NT = A::NT;
    constexpr int KP = A::KP, NQP = A::NQP, NP = A::NP, B2K = A::B2K, NSP = A::NSP, B2N = A::B2N;
    constexpr int FE = A::FE, LDA = A::LDA, LDV = A::LDV, LDP = A::LDP, LDC2 = A::LDC2, LDT = A::LDT;
    constexpr int LDL = A::LDL, RE = A::RE, RP = A::RP, RC = A::RC, RL = A::RL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    T* sU = sm + A::oU;
    T* sPr = sm + A::oPr;
    T* sR = sm + A::oR;
    T* sA = sm + A::oA;
    T* sP = sA;
    T* sBig = sm + A::oBig;
    __shared__ unsigned int s_status;
    __shared__ unsigned long long s_smax;
    __shared__ double s_tot[8];
    T* sAh = sm + A::oAh;
    // force: a_h staged and the projections' forcing sums (any mode); the
    // right-hand side's source rows exist only in the DRIVEN kernels
    const bool force = (a.flags & F_FORCE) != 0;
    constexpr bool SRC = DRIVEN && (MODE == ADI_RHS || MODE == ADI_STAGE);
    double sums[4] = {0.0, 0.0, 0.0, 0.0};  // <rho a_h> (3), <rho> of the projected tiles
    double work = 0.0;                      // stage: volume integral of the energy source / h^3
    double diss = 0.0;                      // reset: thermal energy taken out / h^3

    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    for (int e = tid; e < C::tabsz; e += NT) sm[e] = a.tab[e];
    const T* tabs = sm;
    if (tid == 0) {
        s_status = 0u;
        s_smax = 0ull;
    }
    const T gamma = a.gas.gamma, g1 = a.gas.g1, fill_e = a.gas.fill_e;
    const T two_h = T(2.0 / a.ph.h), inv4h = T(0.25 / a.ph.h);
    const T eps = T(a.ph.floor_);
    double dtd = a.dt_pimax;
    if constexpr (MODE == ADI_STAGE) {
        // the step's dt: CFL bound of u^n (projection of stage 1), prescribed dt, retry factor
        const double smax = __longlong_as_double((long long)a.ctl->smax);
        dtd = (a.ctl->fixed_dt > 0.0 ? a.ctl->fixed_dt : a.ctl->dt_num / smax) * a.ctl->dt_scale;
        if (blockIdx.x == 0 && tid == 0) a.ctl->dt = dtd;
    }
    const T dt = T(dtd);
    T ab0 = T(0), ab1 = T(0), ab2 = T(0);
    if (SRC) {
        ab0 = T(a.ctl->abar2[a.abar_in][0]);
        ab1 = T(a.ctl->abar2[a.abar_in][1]);
        ab2 = T(a.ctl->abar2[a.abar_in][2]);
    }
    // sup |phi_m| of the mode m = lane (positivity bound), 0 past the modes
    T my_sup = T(0);
    static_for<0, b>([&](auto m) {
        if (lane == decltype(m)::value) my_sup = T(sup_phi<K>(decltype(m)::value));
    });
    T smax = T(0);
    __syncthreads();

    const long ntile = (a.ncell + TC - 1) / TC;
    for (long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const long c0 = tile * TC;
        const int nvalid = (int)((a.ncell - c0) < TC ? (a.ncell - c0) : TC);
        adi_load<T, NT, 5, b>(sU, a.u_in + c0 * 5 * b, TC * 5 * b, nvalid * 5 * b, fill_e);
        if (force && MODE != ADI_RESET) {
            for (int e = 4 * tid; e < TC * 3 * b; e += 4 * NT) {
                T v[4];
                ld4_guard<T>(a.ahat + c0 * 3 * b, e, nvalid * 3 * b, v);
                st4<T>(sAh + e, v);
            }
        }
        if constexpr (MODE == ADI_PROJECT) {
            __syncthreads();
            adi_project_tile<T, K, DRIVEN>(sm, sU, tabs, a, c0, nvalid, gamma, smax, sums);
        } else if constexpr (MODE == ADI_RESET) {
            __syncthreads();
            // rho, m at the volume points; e = rho cs^2/(gamma-1) + |m|^2/(2 rho) there; projected
            for (int e = tid; e < TC * 4 * KP; e += NT) {
                const int r = e / KP, l = e % KP, c = r / 4, f = r % 4;
                sA[r * LDA + l] = l < b ? sU[(c * 5 + f) * b + l] : T(0);
            }
            __syncthreads();
            mm<T, BK_FMA, TC * 4, NQP, KP, LDA, LDV, NT>(sA, tabs, C::oPhi, sBig);
            __syncthreads();
            const T cres = a.gas.cres;
            constexpr int PER = (TC * NQP + NT - 1) / NT;
            T ev[PER];
#pragma unroll
            for (int it = 0; it < PER; ++it) {
                const int e = tid + it * NT;
                ev[it] = T(0);
                if (e < TC * NQP) {
                    const int c = e / NQP, q = e % NQP;
                    if (q < nq) {
                        const T* v = sBig + (c * 4) * LDV + q;
                        const T rho = v[0], mx = v[LDV], my = v[2 * LDV], mz = v[3 * LDV];
                        ev[it] = rho * cres + T(0.5) * (mx * mx + my * my + mz * mz) / rho;
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int it = 0; it < PER; ++it) {
                const int e = tid + it * NT;
                if (e < TC * NQP) sBig[(e / NQP) * LDV + e % NQP] = ev[it];
            }
            __syncthreads();
            mm<T, BK_FMA, TC, NP, NQP, LDV, LDP, NT>(sBig, tabs, C::oWPhi, sP);
            __syncthreads();
            if (tid < TC && tid < nvalid) diss += (double)sU[(tid * 5 + 4) * b] - (double)sP[tid * LDP];
            for (int e = tid; e < nvalid * b; e += NT) {
                const int c = e / b, l = e % b;
                a.out[(c0 + c) * 5 * b + 4 * b + l] = sP[c * LDP + l];
            }
            __syncthreads();
        } else {
        // ---- right-hand side: stage the projections (and u^n) of the tile ----
        for (int e = 4 * tid; e < TC * 4 * b; e += 4 * NT) {
            T v[4];
            ld4_guard<T>(a.pr_in + c0 * 4 * b, e, nvalid * 4 * b, v);
            st4<T>(sPr + e, v);
        }
        __syncthreads();
        // ---- evaluation coefficients: rho, m, e, grad rho, div m (field-major threads) ----
        for (int e = tid; e < RE; e += NT) {
            const int f = e / TC, c = e % TC;
            const T* u = sU + c * 5 * b;
            T* row = sA + (c * FE + f) * LDA;
            T out[KP];
#pragma unroll
            for (int l = 0; l < KP; ++l) out[l] = T(0);
            if (f < 5) {
#pragma unroll
                for (int l = 0; l < b; ++l) out[l] = u[f * b + l];
            } else if (f == 5) {
                modal_grad<T, K, 0>(u, out, two_h);
            } else if (f == 6) {
                modal_grad<T, K, 1>(u, out, two_h);
            } else if (f == 7) {
                modal_grad<T, K, 2>(u, out, two_h);
            } else if (f == 8) {
                T t2[b];
                modal_grad<T, K, 0>(u + b, out, two_h);
                modal_grad<T, K, 1>(u + 2 * b, t2, two_h);
#pragma unroll
                for (int l = 0; l < b; ++l) out[l] += t2[l];
                modal_grad<T, K, 2>(u + 3 * b, t2, two_h);
#pragma unroll
                for (int l = 0; l < b; ++l) out[l] += t2[l];
            } else if (SRC && f < 12) {
#pragma unroll
                for (int l = 0; l < b; ++l) out[l] = sAh[(c * 3 + f - 9) * b + l];
            }
#pragma unroll
            for (int l = 0; l < KP; l += 4) st4<T>(row + l, out + l);
        }
        __syncthreads();
        mm<T, BK_FMA, RE, NQP, KP, LDA, LDV, NT>(sA, tabs, C::oPhi, sBig);
        __syncthreads();
        // ---- pointwise volume physics (Sec. 3.1: Pi at the internal points) ----
        {
            constexpr int PER = (TC * NQP + NT - 1) / NT;
            constexpr int FP = A::FP;
            T fl[PER][FP];
#pragma unroll
            for (int it = 0; it < PER; ++it) {
                const int e = tid + it * NT;
#pragma unroll
                for (int g = 0; g < FP; ++g) fl[it][g] = T(0);
                if (e < TC * NQP) {
                    const int c = e / NQP, q = e % NQP;
                    if (q < nq) {
                        const T* v = sBig + (c * FE) * LDV + q;
                        const T rho = v[0], ir = rcp<T>(rho);
                        const T mx = v[LDV], my = v[2 * LDV], mz = v[3 * LDV], en = v[4 * LDV];
                        const T vx = mx * ir, vy = my * ir, vz = mz * ir;
                        const T p = g1 * (en - T(0.5) * (mx * vx + my * vy + mz * vz)) + a.gas.c0 * rho;
                        const T divv = (v[8 * LDV] - (vx * v[5 * LDV] + vy * v[6 * LDV] + vz * v[7 * LDV])) * ir;
                        const T cs = sqrt(gamma * p * ir);
                        const T P = p + adi_vnr<T>(a.ph, rho, cs, divv, dt);
                        fl[it][0] = mx * vx + P;
                        fl[it][1] = my * vy + P;
                        fl[it][2] = mz * vz + P;
                        fl[it][3] = mx * vy;
                        fl[it][4] = mx * vz;
                        fl[it][5] = my * vz;
                        fl[it][6] = (en + P) * vx;
                        fl[it][7] = (en + P) * vy;
                        fl[it][8] = (en + P) * vz;
                        if constexpr (SRC) {
                            const T dx = v[9 * LDV] - ab0, dy = v[10 * LDV] - ab1, dz = v[11 * LDV] - ab2;
                            fl[it][9] = rho * dx;
                            fl[it][10] = rho * dy;
                            fl[it][11] = rho * dz;
                            fl[it][12] = mx * dx + my * dy + mz * dz;
                        }
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int it = 0; it < PER; ++it) {
                const int e = tid + it * NT;
                if (e < TC * NQP) {
                    const int c = e / NQP, q = e % NQP;
#pragma unroll
                    for (int g = 0; g < FP; ++g) sBig[(c * FP + g) * LDV + q] = fl[it][g];
                }
            }
        }
        __syncthreads();
        mm<T, BK_FMA, RP, NP, NQP, LDV, LDP, NT>(sBig, tabs, C::oWPhi, sP);
        __syncthreads();
        // ---- volume term in modal space: (2/h) sum_d D_d^T (projected flux along d) ----
        for (int e = tid; e < TC * 5; e += NT) {
            const int v = e / TC, c = e % TC;
            T r[b];
#pragma unroll
            for (int l = 0; l < b; ++l) r[l] = T(0);
            const T* P = sP + c * A::FP * LDP;
            if (v == 0) {
                const T* u = sU + c * 5 * b;
                modal_grad_T_acc<T, K, 0>(u + b, r, two_h);
                modal_grad_T_acc<T, K, 1>(u + 2 * b, r, two_h);
                modal_grad_T_acc<T, K, 2>(u + 3 * b, r, two_h);
            } else if (v < 4) {
                const int i = v - 1;
                const int cx = (i == 0) ? 0 : (i == 1 ? 3 : 4);
                const int cy = (i == 0) ? 3 : (i == 1 ? 1 : 5);
                const int cz = (i == 0) ? 4 : (i == 1 ? 5 : 2);
                modal_grad_T_acc<T, K, 0>(P + cx * LDP, r, two_h);
                modal_grad_T_acc<T, K, 1>(P + cy * LDP, r, two_h);
                modal_grad_T_acc<T, K, 2>(P + cz * LDP, r, two_h);
                if constexpr (SRC) {
#pragma unroll
                    for (int l = 0; l < b; ++l) r[l] += P[(9 + i) * LDP + l];
                }
            } else {
                modal_grad_T_acc<T, K, 0>(P + 6 * LDP, r, two_h);
                modal_grad_T_acc<T, K, 1>(P + 7 * LDP, r, two_h);
                modal_grad_T_acc<T, K, 2>(P + 8 * LDP, r, two_h);
                if constexpr (SRC) {
#pragma unroll
                    for (int l = 0; l < b; ++l) r[l] += P[12 * LDP + l];
                    if (MODE == ADI_STAGE && c < nvalid) work += (double)P[12 * LDP];  // cell mean of the work
                }
            }
#pragma unroll
            for (int l = 0; l < b; ++l) sR[(c * 5 + v) * b + l] = r[l];
        }
        __syncthreads();
        // ---- faces, one direction at a time (Sec. 3.2 face states, Rusanov) ----
        T* sC2 = sBig;
        T* sTr = sBig + A::FA;
        T* sFs = sC2;
        T* sL2 = sTr;
        static_for<0, 3>([&](auto dd) {
            constexpr int Dd = decltype(dd)::value;
            // collapse rows r = ((c*2 + side)*2 + who)*5 + field: field 0 rho (own
            // expansion), 1..4 the projections of v and p; who 1: the neighbour
            for (int r = tid; r < RC; r += NT) {
                const int field = r % 5, who = (r / 5) & 1, side = (r / 10) & 1, c = r / 20;
                T cf[b];
                int fside = side;
                if (who == 0) {
                    const T* src = field == 0 ? sU + c * 5 * b : sPr + (c * 4 + field - 1) * b;
#pragma unroll
                    for (int l = 0; l < b; ++l) cf[l] = src[l];
                } else {
                    fside = 1 - side;
                    const long cc = c0 + c;
                    int xyz[3] = {0, 0, 0};
                    if (cc < a.ncell) cell_xyz(cc, a.N, xyz[0], xyz[1], xyz[2]);
                    const int bcd = a.bc[Dd];
                    if (cc < a.ncell && bcd != DG_BC_PERIODIC && xyz[Dd] == (side ? a.N - 1 : 0)) {
                        // a boundary face: the ghost state is the cell's own trace on it
                        // (outflow; reflective: the normal velocity negated), or the
                        // prescribed inflow state (flat) at the face at coordinate 0
                        fside = side;
                        if (bcd == DG_BC_INFLOW && side == 0) {
                            const double rin = a.inflow[0];
                            const double val = field == 0 ? rin
                                             : field < 4 ? a.inflow[field]
                                                         : a.inflow[4] - (double)a.gas.c0 * rin;
#pragma unroll
                            for (int l = 0; l < b; ++l) cf[l] = l == 0 ? T(val) : T(0);
                        } else {
                            const T* src = field == 0 ? sU + c * 5 * b : sPr + (c * 4 + field - 1) * b;
                            const T sg = (bcd == DG_BC_REFLECT && field == 1 + Dd) ? T(-1) : T(1);
#pragma unroll
                            for (int l = 0; l < b; ++l) cf[l] = sg * src[l];
                        }
                    } else if (cc < a.ncell) {
                        const long nc = neighbour_along<Dd>(cc, xyz[Dd], side, a.N);
                        const T* src = field == 0 ? a.u_in + nc * 5 * b : a.pr_in + (nc * 4 + field - 1) * b;
                        if constexpr (b % 4 == 0) {
#pragma unroll
                            for (int l = 0; l < b; l += 4) ld4<T>(src + l, cf + l);
                        } else {
#pragma unroll
                            for (int l = 0; l < b; ++l) cf[l] = __ldg(src + l);
                        }
                    } else {
                        // past the end: a quiet filler state (rho = 1, v = 0, p = 1: deviation 1 - c0)
#pragma unroll
                        for (int l = 0; l < b; ++l)
                            cf[l] = l != 0 ? T(0) : field == 0 ? T(1) : field == 4 ? T(1) - a.gas.c0 : T(0);
                    }
                }
                T c2[B2K];
                collapse<T, K, Dd, B2K>(cf, fside, c2);
#pragma unroll
                for (int p = 0; p < B2K; p += 4) st4<T>(sC2 + r * LDC2 + p, c2 + p);
            }
            __syncthreads();
            mm<T, BK_FMA, RC, NSP, B2K, LDC2, LDT, NT>(sC2, tabs, C::oPsi, sTr);
            __syncthreads();
            // Rusanov flux at every face point, along +e_d with L the lower cell
            for (int e = tid; e < TC * 2 * NSP; e += NT) {
                const int s = e % NSP, side = (e / NSP) & 1, c = e / (2 * NSP);
                T F[5] = {T(0), T(0), T(0), T(0), T(0)};
                if (s < ns) {
                    const int rs = ((c * 2 + side) * 2 + 0) * 5, rn = ((c * 2 + side) * 2 + 1) * 5;
                    T Ws[5], Wn[5];
#pragma unroll
                    for (int f = 0; f < 5; ++f) {
                        Ws[f] = sTr[(rs + f) * LDT + s];
                        Wn[f] = sTr[(rn + f) * LDT + s];
                    }
                    const T* WLf = side ? Ws : Wn;
                    const T* WRf = side ? Wn : Ws;
                    if (a.ph.riemann == 2)
                        adi_hllc<T, Dd>(a.gas, WLf, WRf, F);
                    else
                        adi_rusanov<T, Dd>(a.gas, WLf, WRf, F);
                }
                // written after every thread has read its traces (the flux rows alias nothing read here)
#pragma unroll
                for (int v = 0; v < 5; ++v) sFs[((c * 2 + side) * 5 + v) * LDT + s] = F[v];
            }
            __syncthreads();
            mm<T, BK_FMA, RL, B2N, NSP, LDT, LDL, NT>(sFs, tabs, C::oPsiL, sL2);
            __syncthreads();
            // + face (side 1): -1/(4h); - face (side 0): +1/(4h)
            for (int e = tid; e < TC * 5; e += NT) {
                const int c = e / 5, v = e % 5;
                T* R = sR + (c * 5 + v) * b;
                T rr[b];
#pragma unroll
                for (int l = 0; l < b; ++l) rr[l] = R[l];
                expand_acc<T, K, Dd>(sL2 + ((c * 2 + 1) * 5 + v) * LDL, 1, -inv4h, rr);
                expand_acc<T, K, Dd>(sL2 + ((c * 2 + 0) * 5 + v) * LDL, 0, inv4h, rr);
#pragma unroll
                for (int l = 0; l < b; ++l) R[l] = rr[l];
            }
            __syncthreads();
        });
        if constexpr (MODE == ADI_RHS) {
            for (int e = tid; e < nvalid * 5 * b; e += NT) a.out[c0 * 5 * b + e] = sR[e];
            __syncthreads();
        } else {
            // ---- SSP-RK stage combine (Sec. 7) ----
            // u^n straight from global memory (read once, coalesced)
            for (int e = tid; e < TC * 5 * b; e += NT) {
                const T un = (a.rk_a != T(0) && e < nvalid * 5 * b) ? a.u_n[c0 * 5 * b + e] : T(0);
                sU[e] = a.rk_a * un + a.rk_b * (sU[e] + dt * sR[e]);
            }
            __syncthreads();
            // ---- positivity of density and pressure (Sec. 3.1), warp per cells ----
            constexpr int NW = NT / 32, CPW = TC / NW, NPT = nq + nf, NPW = (NPT + 31) / 32;
            static_assert(TC % NW == 0, "cells per warp");
            unsigned int st = 0u;
            for (int cl = 0; cl < CPW; ++cl) {
                const int c = wid * CPW + cl;
                T* u = sU + c * 5 * b;
                T ub[5], dl[5];
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    ub[v] = u[v * b];
                    T part = (lane >= 1 && lane < b) ? fabs(u[v * b + (lane < b ? lane : 0)]) * my_sup : T(0);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                    dl[v] = part;
                }
                if (c >= nvalid) continue;  // warp-uniform
                const T pbar = adi_p<T>(a.gas, ub[0], ub[1], ub[2], ub[3], ub[4]);
                if (!(ub[0] > eps) || !(pbar > eps)) {
                    st |= DG_ST_FAIL_;
                    continue;
                }
                // sufficient condition on the box ubar +- delta: no point can be below a floor
                bool ok = ub[0] - dl[0] >= eps;
                if (ok) {
                    // rho p = (gamma-1)(rho e_s - |m|^2/2) + c0 rho^2 >= eps rho on the box
                    const T lr = ub[0] - dl[0], ur = ub[0] + dl[0], le = ub[4] - dl[4];
                    T mm2 = T(0);
#pragma unroll
                    for (int i = 1; i < 4; ++i) {
                        const T mi = fabs(ub[i]) + dl[i];
                        mm2 += mi * mi;
                    }
                    const T re = le >= T(0) ? lr * le : ur * le;
                    ok = g1 * (re - T(0.5) * mm2) + a.gas.c0 * lr * lr - eps * ur > T(0);
                }
                if (ok) continue;
                // exact check at every volume and face point
                const T* phiv = a.tab + TT::phiv;
                const T* phif = a.tab + TT::phif;
                T val[NPW][5];
                T rmin = T(1e30);
#pragma unroll
                for (int j = 0; j < NPW; ++j) {
                    const int pt = lane + 32 * j;
#pragma unroll
                    for (int v = 0; v < 5; ++v) val[j][v] = ub[v];
                    if (pt < NPT) {
#pragma unroll
                        for (int v = 0; v < 5; ++v) {
                            T s = T(0);
                            if (pt < nq) {
#pragma unroll
                                for (int l = 0; l < b; ++l) s += u[v * b + l] * __ldg(phiv + l * nq + pt);
                            } else {
#pragma unroll
                                for (int l = 0; l < b; ++l) s += u[v * b + l] * __ldg(phif + l * nf + (pt - nq));
                            }
                            val[j][v] = s;
                        }
                        rmin = val[j][0] < rmin ? val[j][0] : rmin;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const T other = __shfl_xor_sync(0xffffffffu, rmin, o);
                    rmin = other < rmin ? other : rmin;
                }
                const T th_r = rmin < eps ? (ub[0] - eps) / (ub[0] - rmin) : T(1);
                T th_p = T(1);
#pragma unroll
                for (int j = 0; j < NPW; ++j) {
                    const int pt = lane + 32 * j;
                    if (pt < NPT) {
                        T uq[5], dv[5];
#pragma unroll
                        for (int v = 0; v < 5; ++v) {
                            uq[v] = ub[v] + th_r * (val[j][v] - ub[v]);
                            dv[v] = uq[v] - ub[v];
                        }
                        if (adi_p<T>(a.gas, uq[0], uq[1], uq[2], uq[3], uq[4]) < eps) {
                            const T t = adi_pressure_root<T>(a.gas, eps, ub, dv);
                            th_p = t < th_p ? t : th_p;
                        }
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const T other = __shfl_xor_sync(0xffffffffu, th_p, o);
                    th_p = other < th_p ? other : th_p;
                }
                const T th = th_r * th_p;
                if (th < T(1)) {
                    st |= DG_ST_LIMITED_;
                    for (int e = lane; e < 5 * b; e += 32)
                        if (e % b) u[e] *= th;
                }
                __syncwarp();
            }
            st = __reduce_or_sync(0xffffffffu, st);
            if (lane == 0 && st) atomicOr(&s_status, st);
            __syncthreads();
            for (int e = tid; e < nvalid * 5 * b; e += NT) {
                const T w = sU[e];
                if (!isfinite(w)) atomicOr(&s_status, DG_ST_NONFINITE_);
                a.out[c0 * 5 * b + e] = w;
            }
            __syncthreads();
            // the next stage's projections of v and p, from the new state in shared memory
            if (a.flags & F_NEXTPROJ) adi_project_tile<T, K, DRIVEN>(sm, sU, tabs, a, c0, nvalid, gamma, smax, sums);
        }
        }  // right-hand-side modes
    }
    // ---- block reductions (their buffer is the big region, free after the tile loop) ----
    __syncthreads();
    double* s_buf = reinterpret_cast<double*>(sm + A::oBig);
    static_assert(A::BIG * sizeof(T) >= NT * sizeof(double), "reduction buffer");
    const double h3 = a.ph.h * a.ph.h * a.ph.h;
    if constexpr (MODE == ADI_PROJECT) {
        if (a.flags & F_DT) {
            const double sp = (double)smax;
            atomicMax(&s_smax, (unsigned long long)__double_as_longlong(sp));
            __syncthreads();
            if (tid == 0) atomicMax(&a.ctl->smax, s_smax);
        }
    }
    if constexpr (MODE == ADI_RHS || MODE == ADI_STAGE) {
        if (tid == 0 && s_status) atomicOr(&a.ctl->status, s_status);
    }
    // abar of the projected states: <rho a_h> / <rho>
    if (force && (MODE == ADI_PROJECT || (MODE == ADI_STAGE && (a.flags & F_NEXTPROJ)))) {
        if (adi_reduce<NT>(a.partials, s_buf, s_tot, &a.ctl->cnt_proj, sums, 4) && tid == 0)
            for (int i = 0; i < 3; ++i) a.ctl->abar2[a.abar_out][i] = s_tot[i] / s_tot[3];
    }
    // injected energy of the stage, dissipated energy of the reset (FP64 accumulators)
    if constexpr (MODE == ADI_STAGE) {
        if (SRC && adi_reduce<NT>(a.partials + 8, s_buf, s_tot, &a.ctl->cnt_diag, &work, 1) && tid == 0)
            a.ctl->diag[1] += a.beta * dtd * s_tot[0] * h3;
    }
    if constexpr (MODE == ADI_RESET) {
        if (adi_reduce<NT>(a.partials + 8, s_buf, s_tot, &a.ctl->cnt_diag, &diss, 1) && tid == 0)
            a.ctl->diag[2] += s_tot[0] * h3;
    }
}

// FP64 totals for the diagnostics: per block [mass, m_x, m_y, m_z, energy of
// the stored variable (offset energy e_s), kinetic energy (volume quadrature of
// |m|^2/(2 rho)), min rho, min p at the volume points], summed over blocks on the
// host in block order.  Point values in the state's precision, sums in FP64; c0 =
// (gamma - 1) kap the pressure of the energy offset per unit density.
template <typename T, int K>
__global__ void __launch_bounds__(256) k_adi_totals(const T* __restrict__ u, const T* __restrict__ tab, long ncell,
                                                   double gamma, double c0, double* __restrict__ partials)
{
    using TT = TileTab<K, BK_FMA>;
    constexpr int b = Dims<K>::b, nq = Dims<K>::nq, n = K + 1;
    __shared__ double s_red[256];
    __shared__ double s_w[nq];
    // Gauss weights (per-point volume weights w_q / 8) from the mass identity: the
    // projection weights are the phi_0 = 1 row of the weighted transpose table
    if (threadIdx.x < nq) s_w[threadIdx.x] = (double)tab[TileCfg<K, BK_FMA>::oWPhi + threadIdx.x * TileCfg<K, BK_FMA>::NP];
    __syncthreads();
    (void)n;
    double acc[6] = {0, 0, 0, 0, 0, 0}, rmin = 1e300, pmin = 1e300;
    for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ncell; c += (long)gridDim.x * blockDim.x) {
        const T* uc = u + c * 5 * b;
        for (int v = 0; v < 5; ++v) acc[v] += (double)uc[v * b];  // mode 0: the cell mean
        for (int q = 0; q < nq; ++q) {
            T w[5];
            for (int v = 0; v < 5; ++v) {
                T s = T(0);
                for (int l = 0; l < b; ++l) s += uc[v * b + l] * tab[TT::phiv + l * nq + q];
                w[v] = s;
            }
            const double ke = 0.5 * ((double)w[1] * w[1] + (double)w[2] * w[2] + (double)w[3] * w[3]) / (double)w[0];
            acc[5] += s_w[q] * ke;
            const double p = (gamma - 1.0) * ((double)w[4] - ke) + c0 * (double)w[0];
            rmin = (double)w[0] < rmin ? (double)w[0] : rmin;
            pmin = p < pmin ? p : pmin;
        }
    }
    double vals[8] = {acc[0], acc[1], acc[2], acc[3], acc[4], acc[5], rmin, pmin};
    for (int i = 0; i < 8; ++i) {
        s_red[threadIdx.x] = vals[i];
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = i < 6 ? 0.0 : 1e300;
            for (int j = 0; j < (int)blockDim.x; ++j) t = i < 6 ? t + s_red[j] : (s_red[j] < t ? s_red[j] : t);
            partials[blockIdx.x * 8 + i] = t;
        }
        __syncthreads();
    }
}

}  // namespace dg
