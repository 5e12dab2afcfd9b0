// dg_kernels.cuh -- auxiliary CUDA-core kernels of libdg (FP64 and FP32):
// forcing projection, diagnostics, L1 norm; templated on the element type T
// and the degree K.  The hot-path kernels are in dg_tile.cuh.
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

// coordinates of cell c = (z N + y) N + x; 32-bit arithmetic (N <= kMaxN)
__device__ __forceinline__ void cell_xyz(long c, int N, int& x, int& y, int& z)
{
    const unsigned int u = (unsigned int)c, n = (unsigned int)N, q = u / n;
    x = (int)(u - q * n);
    y = (int)(q % n);
    z = (int)(q / n);
}

// periodic neighbour of cell c across its face along Dd (side 1: +, 0: -),
// given c's coordinate co along Dd
template <int Dd>
__device__ __forceinline__ long neighbour_along(long c, int co, int side, int N)
{
    const long st = Dd == 0 ? 1L : (Dd == 1 ? (long)N : (long)N * N);
    if (side) return co == N - 1 ? c - (long)(N - 1) * st : c + st;
    return co == 0 ? c + (long)(N - 1) * st : c - st;
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
// K_force: projection of the driving acceleration of explicit Fourier modes
//   a(x) = sum_m 2 Re(A_m exp(2 pi i k_m . x))   (Sec. 4.2)
//   ahat_l = sum_q (w_q/8) phi_l(xi_q) a(x_q),  x_q = x_c + (h/2) xi_q
// The tensor Gauss rule, the product basis and the plane waves all factor
// over the axes, so with the 1D factors
//   G[i_c][kap][m] = sum_a (w_a/2) Pn_m(xi_a) exp(2 pi i kap (i_c + 1/2 + xi_a/2) h)
// each mode's projection is G[ix][kx][i_l] G[iy][ky][j_l] G[iz][kz][l_l]:
// the same sum, regrouped.  k_force_axis builds G in FP64 (stored in T);
// k_force forms the products per cell.
// ---------------------------------------------------------------------------
constexpr int kForceKM = 8;  // |k_d| <= 8 supported
constexpr int kForceNK = 2 * kForceKM + 1;

// sqrt(2m+1) P_m(x) by the three-term recurrence
__device__ __forceinline__ double legendre_pn(int m, double x)
{
    double p0 = 1.0, p1 = x;
    if (m == 0) return 1.0;
    for (int j = 2; j <= m; ++j) {
        const double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
    }
    return sqrt(2.0 * m + 1.0) * p1;
}

template <typename T, int K>
__global__ void __launch_bounds__(256) k_force_axis(Rule1 r, int N, int kmaxc, T* G)
{
    constexpr int n = K + 1;
    const int total = N * kForceNK * n;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int m = e % n, kap = (e / n) % kForceNK - kForceKM, ic = e / (n * kForceNK);
        double re = 0.0, im = 0.0;
        if (kap >= -kmaxc && kap <= kmaxc) {
            const double h = 1.0 / N;
            for (int a = 0; a < n; ++a) {
                const double wp = 0.5 * r.w[a] * legendre_pn(m, r.x[a]);
                double sn, cn;
                sincospi(2.0 * kap * ((ic + 0.5 + 0.5 * r.x[a]) * h), &sn, &cn);
                re += wp * cn;
                im += wp * sn;
            }
        }
        G[2 * e] = T(re);
        G[2 * e + 1] = T(im);
    }
}

template <typename T, int K>
__global__ void __launch_bounds__(256) k_force(const T* G, int N, long ncell, int nm, const int* kvec, const double* amp,
                                               T* ahat)
{
    using D = Dims<K>;
    constexpr int b = D::b, n = K + 1;
    constexpr Modes<K> M{};
    __shared__ int s_k[512][3];
    __shared__ T s_amp[512][3][2];
    for (int e = threadIdx.x; e < nm; e += blockDim.x) {
        for (int i = 0; i < 3; ++i) {
            s_k[e][i] = kvec[e * 3 + i] + kForceKM;
            s_amp[e][i][0] = T(2.0 * amp[(e * 3 + i) * 2]);
            s_amp[e][i][1] = T(2.0 * amp[(e * 3 + i) * 2 + 1]);
        }
    }
    __syncthreads();
    const long rowlen = (long)kForceNK * n * 2;  // T words per cell index of G
    for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < ncell; c += (long)gridDim.x * blockDim.x) {
        const int ix = (int)(c % N), iy = (int)((c / N) % N), iz = (int)(c / ((long)N * N));
        const T* gx = G + ix * rowlen;
        const T* gy = G + iy * rowlen;
        const T* gz = G + iz * rowlen;
        T acc[3][b];
#pragma unroll
        for (int v = 0; v < 3; ++v)
#pragma unroll
            for (int l = 0; l < b; ++l) acc[v][l] = T(0);
        for (int m = 0; m < nm; ++m) {
            T x[n][2], y[n][2], z[n][2];
#pragma unroll
            for (int i = 0; i < n; ++i) {
                x[i][0] = __ldg(gx + (s_k[m][0] * n + i) * 2);
                x[i][1] = __ldg(gx + (s_k[m][0] * n + i) * 2 + 1);
                y[i][0] = __ldg(gy + (s_k[m][1] * n + i) * 2);
                y[i][1] = __ldg(gy + (s_k[m][1] * n + i) * 2 + 1);
                z[i][0] = __ldg(gz + (s_k[m][2] * n + i) * 2);
                z[i][1] = __ldg(gz + (s_k[m][2] * n + i) * 2 + 1);
            }
            T A[3][2];
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                A[v][0] = s_amp[m][v][0];
                A[v][1] = s_amp[m][v][1];
            }
            static_for<0, b>([&](auto L) {
                constexpr int l = decltype(L)::value;
                constexpr int i = M.i[l], j = M.j[l], k3 = M.l[l];
                const T pr = x[i][0] * y[j][0] - x[i][1] * y[j][1];
                const T pi = x[i][0] * y[j][1] + x[i][1] * y[j][0];
                const T er = pr * z[k3][0] - pi * z[k3][1];
                const T ei = pr * z[k3][1] + pi * z[k3][0];
#pragma unroll
                for (int v = 0; v < 3; ++v) acc[v][l] += A[v][0] * er - A[v][1] * ei;
            });
        }
        T* out = ahat + c * 3 * b;
#pragma unroll
        for (int v = 0; v < 3; ++v)
#pragma unroll
            for (int l = 0; l < b; ++l) out[v * b + l] = acc[v][l];
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
                    acc[10] += w * (mxv * ((double)f[8] - a.ctl->abar2[0][0]) + myv * ((double)f[9] - a.ctl->abar2[0][1]) +
                                    mzv * ((double)f[10] - a.ctl->abar2[0][2]));
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

// ---------------------------------------------------------------------------
// K_flatten: positivity by repetition (Sec. 3.1, last paragraph): the high-order
// weights of every cell a stage marked are scaled towards the flat expansion
// before the step is computed again (DG_ST_SCALED_); a flat marked cell with
// negative density reports DG_ST_FLAT_ (dt is halved), a flat cell marked for
// its speed alone is left as it is.  One thread per cell; marks are rare.
// ---------------------------------------------------------------------------
template <typename T, int K>
__global__ void __launch_bounds__(256) k_flatten(T* u, unsigned char* trouble, unsigned char* level, long ncell,
                                                 Ctl* ctl)
{
    constexpr int b = Dims<K>::b;
    for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += (long)gridDim.x * blockDim.x) {
        const unsigned char m = trouble[c];
        if (!m) continue;
        trouble[c] = 0;
        T* uc = u + c * 4 * b;
        bool nonzero = false;
        for (int var = 0; var < 4; ++var)
            for (int l = 1; l < b; ++l) nonzero |= uc[var * b + l] != T(0);
        if (!nonzero) {
            if (m & DG_MARK_NEGATIVE) atomicOr(&ctl->status, DG_ST_FLAT_);
            continue;
        }
        const unsigned char lv = level[c];
        const T f = lv < 2 ? T(0.5) : T(0);
        for (int var = 0; var < 4; ++var)
            for (int l = 1; l < b; ++l) uc[var * b + l] *= f;
        level[c] = (unsigned char)(lv + 1);
        atomicOr(&ctl->status, DG_ST_SCALED_);
    }
}

}  // namespace dg
