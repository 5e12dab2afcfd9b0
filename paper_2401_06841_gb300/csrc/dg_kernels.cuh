// dg_kernels.cuh -- CUDA-core kernels of libdg (FP64 and FP32), templated on
// the element type T and the degree K.
//
// All kernels walk tiles of TC consecutive cells with a grid sized to the
// resident capacity of the GPU (grid-stride over tiles), stage the tile's
// coefficients in shared memory, and use one thread per (cell, quadrature
// point) for the pointwise work.  Basis tables come from the caller's scratch
// (L1-resident, laid out so that consecutive threads read consecutive words).
//
// Transforms (Sec. 2.2, eq. weight_evolution):
//   evaluation  U(xi_q)  = sum_l c_l phi_l(xi_q)
//   projection  f_l      = sum_q (w_q/8) phi_l(xi_q) f(xi_q)
//   derivatives are taken in modal space (exact for the P_k space):
//     grad coefficients  = (2/h) D_d c,
//     volume term        = (2/h) sum_d D_d^T Fhat_d   with Fhat_d = projection of F_d
#pragma once

#include "dg_common.cuh"

namespace dg {

template <typename T>
struct KArgs {
    const T* u_in;     // u^(s) (state layout)
    const T* u_n;      // u^n for the stage combine
    T* out;            // u^(s+1) (update) or dudt (rhs only)
    T* vhat;           // projected velocity [c][3][b]
    const T* ahat;     // projected acceleration [c][3][b] or nullptr
    const T* tab;      // tables (TabLayout<K>)
    Ctl* ctl;
    double* partials;  // [gridDim][16]
    long ncell;
    int N;
    Phys ph;
    T rk_a, rk_b;      // out = rk_a u_n + rk_b (u_in + dt R)
    double dt_pimax;   // rhs-only mode: dt fixing Pi_max (<= 0: none)
    int flags;         // F_DT | F_FORCE
};

template <int K>
struct Tile {
    static constexpr int TC = (K == 1) ? 32 : (K == 2) ? 8 : 4;  // cells per tile
    static constexpr int NT = TC * Dims<K>::nq;                  // threads per block
};

__device__ __forceinline__ long neighbour(long c, int f, int N)
{
    int ix = (int)(c % N), iy = (int)((c / N) % N), iz = (int)(c / ((long)N * N));
    int d = f >> 1, s = (f & 1) ? 1 : N - 1;
    if (d == 0) ix = (ix + s) % N;
    if (d == 1) iy = (iy + s) % N;
    if (d == 2) iz = (iz + s) % N;
    return ((long)iz * N + iy) * N + ix;
}

// deterministic reduction of per-block partials by the last block to finish
// (counter pattern; no waiting).  Returns true in the last block, with
// s_tot[0..nv) holding the sums over blocks in a fixed order.
template <int NT>
__device__ bool last_block_reduce(double* partials, const double* mine, int nv, unsigned int* counter,
                                  double* s_tot, double* s_buf, unsigned int maxmask = 0u)
{
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        for (int i = 0; i < nv; ++i) partials[(long)blockIdx.x * 16 + i] = mine[i];
        __threadfence();
        unsigned int prev = atomicAdd(counter, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    for (int i = 0; i < nv; ++i) {
        const bool mx = (maxmask >> i) & 1u;
        double acc = mx ? -1e300 : 0.0;
        for (int g = threadIdx.x; g < (int)gridDim.x; g += NT) {
            const double v = __ldcg(partials + (long)g * 16 + i);
            acc = mx ? (v > acc ? v : acc) : acc + v;
        }
        s_buf[threadIdx.x] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = mx ? -1e300 : 0.0;
            for (int j = 0; j < NT; ++j) t = mx ? (s_buf[j] > t ? s_buf[j] : t) : t + s_buf[j];
            s_tot[i] = t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// ---------------------------------------------------------------------------
// K_A: primitive projection (Sec. 3.2, eq. weights_equation), the FP64 sums
// <rho a_h>, <rho> of the momentum-neutral forcing, and at the first stage of
// a step the CFL maximum and dt (Sec. 7: dt ~ h/(k+1)).
// ---------------------------------------------------------------------------
template <typename T, int K>
__global__ void __launch_bounds__(Tile<K>::NT) k_project(KArgs<T> a)
{
    using D = Dims<K>;
    using L = TabLayout<K>;
    constexpr int b = D::b, nq = D::nq, TC = Tile<K>::TC, NT = Tile<K>::NT;
    __shared__ T s_u[TC][4][b];
    __shared__ T s_v[TC][nq][3];
    __shared__ double s_buf[NT];
    __shared__ double s_tot[8];
    __shared__ unsigned long long s_smax;
    const int tid = threadIdx.x;
    const long ntile = (a.ncell + TC - 1) / TC;
    const T* phiT = a.tab + L::phiT;
    const T* wphi = a.tab + L::wphi;
    double sums[4] = {0.0, 0.0, 0.0, 0.0};  // sum rho_l a_il (3), sum rho_0
    if (tid == 0) s_smax = 0ull;
    __syncthreads();
    double smax = 0.0;
    for (long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const long c0 = tile * TC;
        for (int e = tid; e < TC * 4 * b; e += NT) {
            long c = c0 + e / (4 * b);
            (&s_u[0][0][0])[e] = (c < a.ncell) ? a.u_in[c0 * 4 * b + e] : ((e % (4 * b)) == 0 ? T(1) : T(0));
        }
        __syncthreads();
        {
            const int lc = tid / nq, q = tid % nq;
            T r = 0, m0 = 0, m1 = 0, m2 = 0;
#pragma unroll
            for (int l = 0; l < b; ++l) {
                T p = __ldg(phiT + l * nq + q);
                r += s_u[lc][0][l] * p;
                m0 += s_u[lc][1][l] * p;
                m1 += s_u[lc][2][l] * p;
                m2 += s_u[lc][3][l] * p;
            }
            T ir = T(1) / r;
            T v0 = m0 * ir, v1 = m1 * ir, v2 = m2 * ir;
            s_v[lc][q][0] = v0;
            s_v[lc][q][1] = v1;
            s_v[lc][q][2] = v2;
            if ((a.flags & F_DT) && c0 + lc < a.ncell) {
                double s = fabs((double)v0) + fabs((double)v1) + fabs((double)v2) + 3.0 * a.ph.cs;
                smax = s > smax ? s : smax;
            }
        }
        __syncthreads();
        for (int e = tid; e < TC * b; e += NT) {
            const int lc = e / b, l = e % b;
            T v0 = 0, v1 = 0, v2 = 0;
#pragma unroll 8
            for (int q = 0; q < nq; ++q) {
                T w = __ldg(wphi + q * b + l);
                v0 += w * s_v[lc][q][0];
                v1 += w * s_v[lc][q][1];
                v2 += w * s_v[lc][q][2];
            }
            const long c = c0 + lc;
            if (c < a.ncell) {
                a.vhat[c * 3 * b + l] = v0;
                a.vhat[c * 3 * b + b + l] = v1;
                a.vhat[c * 3 * b + 2 * b + l] = v2;
            }
        }
        if ((a.flags & F_FORCE) && tid < TC && c0 + tid < a.ncell) {
            const long c = c0 + tid;
            const T* ac = a.ahat + c * 3 * b;
            for (int i = 0; i < 3; ++i) {
                double s = 0.0;
                for (int l = 0; l < b; ++l) s += (double)s_u[tid][0][l] * (double)ac[i * b + l];
                sums[i] += s;
            }
            sums[3] += (double)s_u[tid][0][0];
        }
        __syncthreads();
    }
    // block reductions: max speed (atomic on the bit pattern; positive doubles
    // order like unsigned integers) and the forcing sums (fixed order)
    if (a.flags & F_DT) {
        atomicMax(&s_smax, (unsigned long long)__double_as_longlong(smax));
        __syncthreads();
        if (tid == 0) atomicMax(&a.ctl->smax, s_smax);
    }
    double mine[4];
    for (int i = 0; i < 4; ++i) {
        s_buf[tid] = sums[i];
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int j = 0; j < NT; ++j) t += s_buf[j];
            mine[i] = t;
        }
        __syncthreads();
    }
    if (last_block_reduce<NT>(a.partials, mine, 4, &a.ctl->cnt_proj, s_tot, s_buf)) {
        if (tid == 0) {
            if (a.flags & F_FORCE) {
                for (int i = 0; i < 3; ++i) a.ctl->abar[i] = s_tot[i] / s_tot[3];
                a.ctl->rho_sum = s_tot[3];
            } else {
                a.ctl->abar[0] = a.ctl->abar[1] = a.ctl->abar[2] = 0.0;
            }
            if (a.flags & F_DT) {
                unsigned long long bits = atomicAdd(&a.ctl->smax, 0ull);
                double sm = __longlong_as_double((long long)bits);
                double dt = a.ctl->fixed_dt > 0.0 ? a.ctl->fixed_dt : a.ctl->dt_num / sm;
                a.ctl->dt = dt * a.ctl->dt_scale;
                a.ctl->smax = 0ull;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// K_B: right-hand side (Sec. 2.2, eq. weight_evolution) with vNR viscous
// pressure at the volume points (Sec. 3.1), projected-velocity face states
// (Sec. 3.2), Rusanov fluxes, forcing source; with UPDATE the SSP-RK stage
// combine (Sec. 7) and the positivity rescaling (Sec. 3.1) are fused in.
// ---------------------------------------------------------------------------
template <typename T, int K>
struct RhsSmem {
    using D = Dims<K>;
    static constexpr int TC = Tile<K>::TC, b = D::b, EC = 12;
    static constexpr int PT = (D::nq * EC > D::nf * 4) ? D::nq * EC : D::nf * 4;
    static constexpr int u = 0;                      // [TC][4][b]
    static constexpr int ec = u + TC * 4 * b;        // [TC][b][EC]
    static constexpr int vh = ec + TC * b * EC;      // [TC][3][b]
    static constexpr int nb = vh + TC * 3 * b;       // [TC][6][4][b]
    static constexpr int pt = nb + TC * 24 * b;      // [TC][PT]
    static constexpr int P = pt + TC * PT;           // [TC][9][b]
    static constexpr int R = P + TC * 9 * b;         // [TC][4][b]
    static constexpr int nw = R + TC * 4 * b;        // [TC][4][b]
    static constexpr int total = nw + TC * 4 * b;
    static constexpr size_t bytes = sizeof(T) * total;
};

template <typename T>
__device__ __forceinline__ void atomic_min_key(void* p, T v);
template <>
__device__ __forceinline__ void atomic_min_key<float>(void* p, float v)
{
    atomicMin((int*)p, float_key(v));
}
template <>
__device__ __forceinline__ void atomic_min_key<double>(void* p, double v)
{
    atomicMin((long long*)p, double_key(v));
}

template <typename T, int K, bool UPDATE>
__global__ void __launch_bounds__(Tile<K>::NT) k_rhs(KArgs<T> a)
{
    using D = Dims<K>;
    using L = TabLayout<K>;
    using S = RhsSmem<T, K>;
    constexpr int b = D::b, nq = D::nq, ns = D::ns, nf = D::nf, TC = Tile<K>::TC, NT = Tile<K>::NT;
    constexpr int EC = S::EC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    T* s_u = sm + S::u;
    T* s_ec = sm + S::ec;
    T* s_vh = sm + S::vh;
    T* s_nb = sm + S::nb;
    T* s_pt = sm + S::pt;
    T* s_P = sm + S::P;
    T* s_R = sm + S::R;
    T* s_nw = sm + S::nw;
    __shared__ int s_minf[TC];
    __shared__ long long s_mind[TC];
    __shared__ unsigned int s_status;

    const int tid = threadIdx.x;
    const long ntile = (a.ncell + TC - 1) / TC;
    const T* phiT = a.tab + L::phiT;
    const T* wphi = a.tab + L::wphi;
    const T* phifT = a.tab + L::phifT;
    const T* lift = a.tab + L::lift;
    const bool force = (a.flags & F_FORCE) != 0;
    const T two_h = T(2.0 / a.ph.h);
    const T inv4h = T(0.25 / a.ph.h);
    const double dtd = UPDATE ? a.ctl->dt : a.dt_pimax;
    const T dt = T(dtd);
    const T abar0 = force ? T(a.ctl->abar[0]) : T(0);
    const T abar1 = force ? T(a.ctl->abar[1]) : T(0);
    const T abar2 = force ? T(a.ctl->abar[2]) : T(0);
    const T cs = T(a.ph.cs), cs2 = T(a.ph.cs2);
    if (tid == 0) s_status = 0u;

    for (long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const long c0 = tile * TC;
        // ---- 1. stage the tile, its forcing and its face neighbours ----
        for (int e = tid; e < TC * 4 * b; e += NT) {
            long c = c0 + e / (4 * b);
            s_u[e] = (c < a.ncell) ? a.u_in[c0 * 4 * b + e] : ((e % (4 * b)) == 0 ? T(1) : T(0));
        }
        for (int e = tid; e < TC * 3 * b; e += NT) {
            const int lc = e / (3 * b), i = (e / b) % 3, l = e % b;
            const long c = c0 + lc;
            s_vh[e] = (c < a.ncell) ? a.vhat[c0 * 3 * b + e] : T(0);
            s_ec[(lc * b + l) * EC + 8 + i] = (force && c < a.ncell) ? a.ahat[c0 * 3 * b + e] : T(0);
        }
        for (int e = tid; e < TC * 24 * b; e += NT) {
            const int lc = e / (24 * b), f = (e / (4 * b)) % 6, v = (e / b) % 4, l = e % b;
            const long c = c0 + lc;
            T val = (v == 0 && l == 0) ? T(1) : T(0);
            if (c < a.ncell) {
                const long nc = neighbour(c, f, a.N);
                val = (v == 0) ? a.u_in[nc * 4 * b + l] : a.vhat[nc * 3 * b + (v - 1) * b + l];
            }
            s_nb[e] = val;
        }
        __syncthreads();
        // ---- 2. modal gradients: rho_x, rho_y, rho_z, div m ----
        for (int e = tid; e < TC * 5; e += NT) {
            const int lc = e / 5, g = e % 5;
            const T* u = s_u + lc * 4 * b;
            T out[b];
            if (g == 0) {
#pragma unroll
                for (int l = 0; l < b; ++l)
                    for (int v = 0; v < 4; ++v) s_ec[(lc * b + l) * EC + v] = u[v * b + l];
                continue;
            }
            if (g == 1) modal_grad<T, K, 0>(u, out, two_h);
            if (g == 2) modal_grad<T, K, 1>(u, out, two_h);
            if (g == 3) modal_grad<T, K, 2>(u, out, two_h);
            if (g == 4) {
                T t[b];
                modal_grad<T, K, 0>(u + b, out, two_h);
                modal_grad<T, K, 1>(u + 2 * b, t, two_h);
#pragma unroll
                for (int l = 0; l < b; ++l) out[l] += t[l];
                modal_grad<T, K, 2>(u + 3 * b, t, two_h);
#pragma unroll
                for (int l = 0; l < b; ++l) out[l] += t[l];
            }
#pragma unroll
            for (int l = 0; l < b; ++l) s_ec[(lc * b + l) * EC + 3 + g] = out[l];
        }
        __syncthreads();
        // ---- 3. pointwise volume physics, one thread per (cell, point) ----
        {
            const int lc = tid / nq, q = tid % nq;
            T f[11];
#pragma unroll
            for (int i = 0; i < 11; ++i) f[i] = T(0);
            const T* ec = s_ec + lc * b * EC;
#pragma unroll
            for (int l = 0; l < b; ++l) {
                const T p = __ldg(phiT + l * nq + q);
#pragma unroll
                for (int i = 0; i < 11; ++i) f[i] += ec[l * EC + i] * p;
            }
            const T rho = f[0], ir = T(1) / rho;
            const T vx = f[1] * ir, vy = f[2] * ir, vz = f[3] * ir;
            // div v = (div m - v . grad rho) / rho   (quotient rule)
            const T divv = (f[7] - (vx * f[4] + vy * f[5] + vz * f[6])) * ir;
            T Pi = T(0);
            if (a.ph.av_mode == 1) Pi = vnr_pressure<T>(a.ph, rho, divv, dt);
            const T P = cs2 * rho + Pi;
            T* o = s_pt + lc * S::PT + q * EC;
            o[0] = f[1] * vx + P;
            o[1] = f[2] * vy + P;
            o[2] = f[3] * vz + P;
            o[3] = f[1] * vy;
            o[4] = f[1] * vz;
            o[5] = f[2] * vz;
            o[6] = rho * (f[8] - abar0);
            o[7] = rho * (f[9] - abar1);
            o[8] = rho * (f[10] - abar2);
        }
        __syncthreads();
        // ---- 4. projection of the 6 flux-tensor components and the forcing ----
        for (int e = tid; e < TC * b * 3; e += NT) {
            const int lc = e / (3 * b), l = (e / 3) % b, g = e % 3;
            const T* pt = s_pt + lc * S::PT + 3 * g;
            T p0 = 0, p1 = 0, p2 = 0;
#pragma unroll 4
            for (int q = 0; q < nq; ++q) {
                const T w = __ldg(wphi + q * b + l);
                p0 += w * pt[q * EC + 0];
                p1 += w * pt[q * EC + 1];
                p2 += w * pt[q * EC + 2];
            }
            T* P = s_P + lc * 9 * b;
            P[(3 * g + 0) * b + l] = p0;
            P[(3 * g + 1) * b + l] = p1;
            P[(3 * g + 2) * b + l] = p2;
        }
        __syncthreads();
        // ---- 5. face traces and Rusanov fluxes (s_pt reused as [TC][nf][4]) ----
        for (int e = tid; e < TC * nf; e += NT) {
            const int lc = e / nf, fs = e % nf, f = fs / ns, s = fs % ns, d = f >> 1;
            const int fo = (f ^ 1) * ns + s;  // same point on the neighbour's opposite face
            const T* u = s_u + lc * 4 * b;
            const T* vh = s_vh + lc * 3 * b;
            const T* nb = s_nb + (lc * 6 + f) * 4 * b;
            T Ws[4] = {0, 0, 0, 0}, Wn[4] = {0, 0, 0, 0};
#pragma unroll
            for (int l = 0; l < b; ++l) {
                const T ps = __ldg(phifT + l * nf + fs), pn = __ldg(phifT + l * nf + fo);
                Ws[0] += u[l] * ps;
                Wn[0] += nb[l] * pn;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    Ws[1 + i] += vh[i * b + l] * ps;
                    Wn[1 + i] += nb[(1 + i) * b + l] * pn;
                }
            }
            T F[4];
            if (f & 1)
                rusanov_dir<T>(d, cs, cs2, Ws, Wn, F);  // + face: this cell is the left state
            else
                rusanov_dir<T>(d, cs, cs2, Wn, Ws, F);  // - face: the neighbour is the left state
            T* o = s_pt + lc * S::PT + fs * 4;
            o[0] = F[0];
            o[1] = F[1];
            o[2] = F[2];
            o[3] = F[3];
        }
        __syncthreads();
        // ---- 6. assemble: volume term in modal space, forcing, surface lift ----
        for (int e = tid; e < TC * 4; e += NT) {
            const int lc = e / 4, v = e % 4;
            T r[b];
#pragma unroll
            for (int l = 0; l < b; ++l) r[l] = T(0);
            const T* P = s_P + lc * 9 * b;
            if (v == 0) {
                const T* u = s_u + lc * 4 * b;
                modal_grad_T_acc<T, K, 0>(u + b, r, two_h);
                modal_grad_T_acc<T, K, 1>(u + 2 * b, r, two_h);
                modal_grad_T_acc<T, K, 2>(u + 3 * b, r, two_h);
            } else {
                const int i = v - 1;
                // F_d(m_i): diagonal i==d -> comp i; off-diagonal pairs (x,y)=3 (x,z)=4 (y,z)=5
                const int cx = (i == 0) ? 0 : (i == 1 ? 3 : 4);
                const int cy = (i == 0) ? 3 : (i == 1 ? 1 : 5);
                const int cz = (i == 0) ? 4 : (i == 1 ? 5 : 2);
                modal_grad_T_acc<T, K, 0>(P + cx * b, r, two_h);
                modal_grad_T_acc<T, K, 1>(P + cy * b, r, two_h);
                modal_grad_T_acc<T, K, 2>(P + cz * b, r, two_h);
#pragma unroll
                for (int l = 0; l < b; ++l) r[l] += P[(6 + i) * b + l];
            }
#pragma unroll
            for (int l = 0; l < b; ++l) s_R[(lc * 4 + v) * b + l] = r[l];
        }
        __syncthreads();
        for (int e = tid; e < TC * b; e += NT) {
            const int lc = e / b, l = e % b;
            const T* F = s_pt + lc * S::PT;
            T r0 = 0, r1 = 0, r2 = 0, r3 = 0;
#pragma unroll 4
            for (int fs = 0; fs < nf; ++fs) {
                const T w = __ldg(lift + fs * b + l);
                r0 += w * F[fs * 4 + 0];
                r1 += w * F[fs * 4 + 1];
                r2 += w * F[fs * 4 + 2];
                r3 += w * F[fs * 4 + 3];
            }
            T* R = s_R + lc * 4 * b;
            R[0 * b + l] += inv4h * r0;
            R[1 * b + l] += inv4h * r1;
            R[2 * b + l] += inv4h * r2;
            R[3 * b + l] += inv4h * r3;
        }
        __syncthreads();
        // ---- 7. epilogue ----
        if constexpr (!UPDATE) {
            for (int e = tid; e < TC * 4 * b; e += NT) {
                const long c = c0 + e / (4 * b);
                if (c < a.ncell) a.out[c0 * 4 * b + e] = s_R[e];
            }
            __syncthreads();
        } else {
            for (int e = tid; e < TC * 4 * b; e += NT) {
                const long c = c0 + e / (4 * b);
                T w = T(0);
                if (c < a.ncell) {
                    // the first stage has rk_a = 0: u^n is not read
                    const T un = (a.rk_a != T(0)) ? a.u_n[c0 * 4 * b + e] : T(0);
                    w = a.rk_a * un + a.rk_b * (s_u[e] + dt * s_R[e]);
                } else {
                    w = ((e % (4 * b)) == 0) ? T(1) : T(0);
                }
                s_nw[e] = w;
            }
            if (tid < TC) {
                s_minf[tid] = 0x7fffffff;
                s_mind[tid] = 0x7fffffffffffffffLL;
            }
            __syncthreads();
            // density at every volume and face Gauss point of the new state
            for (int e = tid; e < TC * (nq + nf); e += NT) {
                const int lc = e / (nq + nf), p = e % (nq + nf);
                const T* r = s_nw + lc * 4 * b;
                T rho = 0;
                if (p < nq) {
#pragma unroll
                    for (int l = 0; l < b; ++l) rho += r[l] * __ldg(phiT + l * nq + p);
                } else {
#pragma unroll
                    for (int l = 0; l < b; ++l) rho += r[l] * __ldg(phifT + l * nf + (p - nq));
                }
                if constexpr (sizeof(T) == 4)
                    atomicMin(&s_minf[lc], float_key((float)rho));
                else
                    atomicMin(&s_mind[lc], double_key((double)rho));
            }
            __syncthreads();
            unsigned int st = 0u;
            for (int e = tid; e < TC * 4 * b; e += NT) {
                const int lc = e / (4 * b), l = e % b;
                const long c = c0 + lc;
                if (c >= a.ncell) continue;
                T rmin;
                if constexpr (sizeof(T) == 4)
                    rmin = (T)key_float(s_minf[lc]);
                else
                    rmin = (T)key_double(s_mind[lc]);
                const T rbar = s_nw[lc * 4 * b];
                const T eps = T(a.ph.floor_);
                T w = s_nw[e];
                if (rmin < eps) {
                    if (rbar > eps) {
                        const T theta = (rbar - eps) / (rbar - rmin);
                        if (l > 0) w *= theta;
                        st |= DG_ST_LIMITED_;
                    } else {
                        st |= DG_ST_FAIL_;
                    }
                }
                if (!isfinite((double)w)) st |= DG_ST_NONFINITE_;
                a.out[c0 * 4 * b + e] = w;
            }
            if (st) atomicOr(&s_status, st);
            __syncthreads();
        }
    }
    if constexpr (UPDATE) {
        __syncthreads();
        if (tid == 0 && s_status) atomicOr(&a.ctl->status, s_status);
    }
}

// ---------------------------------------------------------------------------
// K_force: projection of the driving acceleration of explicit Fourier modes
//   a(x) = sum_m 2 Re(A_m exp(2 pi i k_m . x))   (Sec. 4.2)
//   ahat_l = sum_q (w_q/8) phi_l(xi_q) a(x_q),  x_q = x_c + (h/2) xi_q
// Phases are built per axis from exp(2 pi i x_d) in FP64.
// ---------------------------------------------------------------------------
template <typename T, int K>
__global__ void __launch_bounds__(Tile<K>::NT)
    k_force(const T* tab, int N, long ncell, int nm, const int* kvec, const double* amp, int kmaxc, T* ahat)
{
    using D = Dims<K>;
    using L = TabLayout<K>;
    constexpr int b = D::b, nq = D::nq, TC = Tile<K>::TC, NT = Tile<K>::NT;
    constexpr int KM = 8;  // |k_d| <= 8 supported
    __shared__ T s_a[TC][nq][3];
    __shared__ int s_k[512][3];
    __shared__ T s_amp[512][3][2];
    const int tid = threadIdx.x;
    for (int e = tid; e < nm; e += NT) {
        for (int i = 0; i < 3; ++i) {
            s_k[e][i] = kvec[e * 3 + i];
            s_amp[e][i][0] = T(amp[(e * 3 + i) * 2]);
            s_amp[e][i][1] = T(amp[(e * 3 + i) * 2 + 1]);
        }
    }
    __syncthreads();
    const double h = 1.0 / N;
    const long ntile = (ncell + TC - 1) / TC;
    const T* xq = tab + L::xq;
    const T* wphi = tab + L::wphi;
    for (long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const long c0 = tile * TC;
        {
            const int lc = tid / nq, q = tid % nq;
            const long c = c0 + lc;
            T acc[3] = {0, 0, 0};
            if (c < ncell) {
                const int ix = (int)(c % N), iy = (int)((c / N) % N), iz = (int)(c / ((long)N * N));
                const int ic[3] = {ix, iy, iz};
                T Er[3][2 * KM + 1], Ei[3][2 * KM + 1];
                for (int d = 0; d < 3; ++d) {
                    const double x = (ic[d] + 0.5 + 0.5 * (double)xq[q * 3 + d]) * h;
                    double s1, c1;
                    sincospi(2.0 * x, &s1, &c1);
                    double pr = 1.0, pi = 0.0;
                    Er[d][KM] = T(1);
                    Ei[d][KM] = T(0);
                    for (int m = 1; m <= kmaxc; ++m) {
                        const double nr = pr * c1 - pi * s1, ni = pr * s1 + pi * c1;
                        pr = nr;
                        pi = ni;
                        Er[d][KM + m] = T(pr);
                        Ei[d][KM + m] = T(pi);
                        Er[d][KM - m] = T(pr);
                        Ei[d][KM - m] = T(-pi);
                    }
                }
                for (int m = 0; m < nm; ++m) {
                    const int kx = s_k[m][0] + KM, ky = s_k[m][1] + KM, kz = s_k[m][2] + KM;
                    const T xr = Er[0][kx] * Er[1][ky] - Ei[0][kx] * Ei[1][ky];
                    const T xi = Er[0][kx] * Ei[1][ky] + Ei[0][kx] * Er[1][ky];
                    const T er = xr * Er[2][kz] - xi * Ei[2][kz];
                    const T ei = xr * Ei[2][kz] + xi * Er[2][kz];
#pragma unroll
                    for (int i = 0; i < 3; ++i) acc[i] += T(2) * (s_amp[m][i][0] * er - s_amp[m][i][1] * ei);
                }
            }
            s_a[lc][q][0] = acc[0];
            s_a[lc][q][1] = acc[1];
            s_a[lc][q][2] = acc[2];
        }
        __syncthreads();
        for (int e = tid; e < TC * b; e += NT) {
            const int lc = e / b, l = e % b;
            const long c = c0 + lc;
            T r0 = 0, r1 = 0, r2 = 0;
            for (int q = 0; q < nq; ++q) {
                const T w = __ldg(wphi + q * b + l);
                r0 += w * s_a[lc][q][0];
                r1 += w * s_a[lc][q][1];
                r2 += w * s_a[lc][q][2];
            }
            if (c < ncell) {
                ahat[c * 3 * b + l] = r0;
                ahat[c * 3 * b + b + l] = r1;
                ahat[c * 3 * b + 2 * b + l] = r2;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// K_diag: FP64 diagnostics (Sec. 4.1; injected power and AV work as in the
// energy bookkeeping of Sec. 4.2).  Slots as in dg_diag: 0 mass, 1-3
// momentum, 4 E_kin, 5 <v^2>, 6 (unused here), 7 min rho, 8 max rho, 9 AV
// volume fraction, 10 injected power, 11 max speed, 12 AV work.
// ---------------------------------------------------------------------------
template <typename T, int K>
__global__ void __launch_bounds__(Tile<K>::NT) k_diag(KArgs<T> a)
{
    using D = Dims<K>;
    using L = TabLayout<K>;
    constexpr int b = D::b, nq = D::nq, TC = Tile<K>::TC, NT = Tile<K>::NT, EC = 12;
    __shared__ T s_u[TC][4][b];
    __shared__ T s_ec[TC][b][EC];
    __shared__ double s_buf[NT];
    __shared__ double s_tot[16];
    const int tid = threadIdx.x;
    const long ntile = (a.ncell + TC - 1) / TC;
    const T* phiT = a.tab + L::phiT;
    const T* wq = a.tab + L::wq;
    const bool force = (a.flags & F_FORCE) != 0;
    const double V = a.ph.h * a.ph.h * a.ph.h;
    const T two_h = T(2.0 / a.ph.h);
    const T dt = T(a.dt_pimax);
    double acc[13];
    for (int i = 0; i < 13; ++i) acc[i] = 0.0;
    double mn = 1e300, mx = -1e300, sp = 0.0;
    for (long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const long c0 = tile * TC;
        for (int e = tid; e < TC * 4 * b; e += NT) {
            long c = c0 + e / (4 * b);
            (&s_u[0][0][0])[e] = (c < a.ncell) ? a.u_in[c0 * 4 * b + e] : ((e % (4 * b)) == 0 ? T(1) : T(0));
        }
        for (int e = tid; e < TC * 3 * b; e += NT) {
            const int lc = e / (3 * b), i = (e / b) % 3, l = e % b;
            const long c = c0 + lc;
            s_ec[lc][l][8 + i] = (force && c < a.ncell) ? a.ahat[c0 * 3 * b + e] : T(0);
        }
        __syncthreads();
        for (int e = tid; e < TC * 5; e += NT) {
            const int lc = e / 5, g = e % 5;
            const T* u = &s_u[lc][0][0];
            T out[b];
            if (g == 0) {
                for (int l = 0; l < b; ++l)
                    for (int v = 0; v < 4; ++v) s_ec[lc][l][v] = u[v * b + l];
                continue;
            }
            if (g == 1) modal_grad<T, K, 0>(u, out, two_h);
            if (g == 2) modal_grad<T, K, 1>(u, out, two_h);
            if (g == 3) modal_grad<T, K, 2>(u, out, two_h);
            if (g == 4) {
                T t[b];
                modal_grad<T, K, 0>(u + b, out, two_h);
                modal_grad<T, K, 1>(u + 2 * b, t, two_h);
                for (int l = 0; l < b; ++l) out[l] += t[l];
                modal_grad<T, K, 2>(u + 3 * b, t, two_h);
                for (int l = 0; l < b; ++l) out[l] += t[l];
            }
            for (int l = 0; l < b; ++l) s_ec[lc][l][3 + g] = out[l];
        }
        __syncthreads();
        {
            const int lc = tid / nq, q = tid % nq;
            const long c = c0 + lc;
            if (c < a.ncell) {
                T f[11];
                for (int i = 0; i < 11; ++i) f[i] = T(0);
                for (int l = 0; l < b; ++l) {
                    const T p = __ldg(phiT + l * nq + q);
                    for (int i = 0; i < 11; ++i) f[i] += s_ec[lc][l][i] * p;
                }
                const double w = (double)__ldg(wq + q) * V;
                const double rho = f[0], mxv = f[1], myv = f[2], mzv = f[3];
                const double vx = mxv / rho, vy = myv / rho, vz = mzv / rho;
                const double v2 = vx * vx + vy * vy + vz * vz;
                const double divv = ((double)f[7] - (vx * (double)f[4] + vy * (double)f[5] + vz * (double)f[6])) / rho;
                double Pi = 0.0;
                if (a.ph.av_mode == 1) Pi = (double)vnr_pressure<T>(a.ph, f[0], T(divv), dt);
                acc[4] += w * 0.5 * rho * v2;
                acc[5] += w * v2;
                if (Pi > 0.01 * a.ph.cs2 * rho) acc[9] += w;
                if (force)
                    acc[10] += w * (mxv * ((double)f[8] - a.ctl->abar[0]) + myv * ((double)f[9] - a.ctl->abar[1]) +
                                    mzv * ((double)f[10] - a.ctl->abar[2]));
                acc[12] += w * Pi * divv;
                mn = rho < mn ? rho : mn;
                mx = rho > mx ? rho : mx;
                const double s = fabs(vx) + fabs(vy) + fabs(vz) + 3.0 * a.ph.cs;
                sp = s > sp ? s : sp;
                if (q == 0) {
                    acc[0] += (double)s_u[lc][0][0] * V;
                    acc[1] += (double)s_u[lc][1][0] * V;
                    acc[2] += (double)s_u[lc][2][0] * V;
                    acc[3] += (double)s_u[lc][3][0] * V;
                }
            }
        }
        __syncthreads();
    }
    double mine[16];
    for (int i = 0; i < 13; ++i) {
        double v = acc[i];
        if (i == 7) v = -mn;  // min carried as the max of the negation
        if (i == 8) v = mx;
        if (i == 11) v = sp;
        const bool ismax = (i == 7 || i == 8 || i == 11);
        s_buf[tid] = v;
        __syncthreads();
        if (tid == 0) {
            double t = ismax ? -1e300 : 0.0;
            for (int j = 0; j < NT; ++j) t = ismax ? (s_buf[j] > t ? s_buf[j] : t) : t + s_buf[j];
            mine[i] = t;
        }
        __syncthreads();
    }
    const unsigned int maxmask = (1u << 7) | (1u << 8) | (1u << 11);
    if (last_block_reduce<NT>(a.partials, mine, 13, &a.ctl->cnt_diag, s_tot, s_buf, maxmask)) {
        if (tid == 0) {
            for (int i = 0; i < 13; ++i) a.ctl->diag[i] = s_tot[i];
            a.ctl->diag[7] = -s_tot[7];
        }
    }
}

// ---------------------------------------------------------------------------
// K_l1: (1/V) int |rho_A - rho_B| dV by (k+3)-point Gauss per axis (eq. l1_norm)
// ---------------------------------------------------------------------------
template <typename T, int K>
__global__ void __launch_bounds__(256) k_l1(const T* tab, const T* uA, const T* uB, long ncell, double h,
                                            Ctl* ctl, double* partials)
{
    using D = Dims<K>;
    using L = TabLayout<K>;
    constexpr int b = D::b, nql = D::nql, NT = 256;
    __shared__ double s_buf[NT];
    __shared__ double s_tot[16];
    const T* phiL = tab + L::phiL;
    const T* wL = tab + L::wL;
    const double V = h * h * h;
    double acc = 0.0;
    const long total = ncell * nql;
    for (long e = (long)blockIdx.x * NT + threadIdx.x; e < total; e += (long)gridDim.x * NT) {
        const long c = e / nql;
        const int q = (int)(e % nql);
        double d = 0.0;
        for (int l = 0; l < b; ++l)
            d += ((double)uA[c * 4 * b + l] - (double)uB[c * 4 * b + l]) * (double)__ldg(phiL + l * nql + q);
        acc += (double)__ldg(wL + q) * fabs(d) * V;
    }
    s_buf[threadIdx.x] = acc;
    __syncthreads();
    double mine[1] = {0.0};
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int j = 0; j < NT; ++j) t += s_buf[j];
        mine[0] = t;
    }
    __syncthreads();
    if (last_block_reduce<NT>(partials, mine, 1, &ctl->cnt_diag, s_tot, s_buf)) {
        if (threadIdx.x == 0) ctl->l1 = s_tot[0];
    }
}

}  // namespace dg
