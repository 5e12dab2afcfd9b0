// dg_tables.cuh -- host construction of the basis tables of the tile kernels,
// shared by the context path (dg_api.cu) and the no-allocation path
// (dg_noalloc.cu): both upload the same bits.  Everything writes into
// caller-provided buffers; nothing here allocates.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/dg.h"
#include "dg_tile.cuh"

namespace dg {
namespace tables {

// Gauss-Legendre rule of n <= 16 points by Golub-Welsch: nodes = eigenvalues of
// the symmetric tridiagonal Jacobi matrix with off-diagonal j/sqrt(4j^2-1)
// (cyclic Jacobi rotations), weights = 2 (first eigenvector entry)^2; the
// rule's symmetry is then enforced exactly.
inline void gauss_rule(int n, long double* x, long double* w)
{
    long double A[16 * 16] = {}, V[16 * 16] = {};
    for (int j = 1; j < n; ++j) {
        long double bj = j / sqrtl(4.0L * j * j - 1.0L);
        A[(j - 1) * n + j] = A[j * n + j - 1] = bj;
    }
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0L;
    for (int sweep = 0; sweep < 100; ++sweep) {
        long double off = 0.0L;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
        if (off < 1e-40L) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                long double apq = A[p * n + q];
                if (fabsl(apq) < 1e-300L) continue;
                long double theta = (A[q * n + q] - A[p * n + p]) / (2.0L * apq);
                long double t = (theta >= 0 ? 1.0L : -1.0L) / (fabsl(theta) + sqrtl(theta * theta + 1.0L));
                long double c = 1.0L / sqrtl(t * t + 1.0L), s = t * c;
                for (int k = 0; k < n; ++k) {  // A <- A J
                    long double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // A <- J^T A
                    long double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {  // V <- V J
                    long double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    int idx[16];
    for (int i = 0; i < n; ++i) idx[i] = i;
    for (int i = 0; i < n; ++i)  // sort ascending
        for (int j = i + 1; j < n; ++j)
            if (A[idx[j] * n + idx[j]] < A[idx[i] * n + idx[i]]) {
                const int tmp = idx[i];
                idx[i] = idx[j];
                idx[j] = tmp;
            }
    for (int i = 0; i < n; ++i) {
        long double xi = A[idx[i] * n + idx[i]];
        x[i] = fabsl(xi) < 1e-30L ? 0.0L : xi;
        w[i] = 2.0L * V[0 * n + idx[i]] * V[0 * n + idx[i]];
    }
    for (int i = 0; i < n / 2; ++i) {  // enforce the exact symmetry of the rule
        long double xs = 0.5L * (x[n - 1 - i] - x[i]), ws = 0.5L * (w[i] + w[n - 1 - i]);
        x[i] = -xs;
        x[n - 1 - i] = xs;
        w[i] = w[n - 1 - i] = ws;
    }
}

// normalised Legendre sqrt(2m+1) P_m(x), three-term recurrence
inline long double pnorm(int m, long double x)
{
    long double p0 = 1.0L, p1 = x;
    if (m == 0) return 1.0L;
    for (int j = 2; j <= m; ++j) {
        long double p2 = ((2.0L * j - 1.0L) * x * p1 - (j - 1.0L) * p0) / j;
        p0 = p1;
        p1 = p2;
    }
    return sqrtl(2.0L * m + 1.0L) * p1;
}

// split of x into bfloat16 hi + lo, each rounded to nearest even
inline uint16_t bf16_rne(float x)
{
    uint32_t u;
    std::memcpy(&u, &x, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return (uint16_t)(u >> 16);
}
inline float bf16_to_float(uint16_t h)
{
    const uint32_t u = (uint32_t)h << 16;
    float x;
    std::memcpy(&x, &u, 4);
    return x;
}

// dense B[K][N] (row-major, zero padded) -> mma.sync m16n8k16 B fragments:
// words [K/16][N/8][lane][hi(k=2t,2t+1) hi(k=2t+8,2t+9) lo(...) lo(...)], n = g
inline void to_fragments(const double* B, int Kd, int Nd, uint32_t* out)
{
    for (int kt = 0; kt < Kd / 16; ++kt)
        for (int nt = 0; nt < Nd / 8; ++nt)
            for (int lane = 0; lane < 32; ++lane) {
                const int g = lane >> 2, t = lane & 3, n = nt * 8 + g;
                uint32_t w[4];
                for (int half = 0; half < 2; ++half) {
                    const int k0 = kt * 16 + 2 * t + 8 * half;
                    uint16_t hi[2], lo[2];
                    for (int j = 0; j < 2; ++j) {
                        const float x = (float)B[(size_t)(k0 + j) * Nd + n];
                        hi[j] = bf16_rne(x);
                        lo[j] = bf16_rne(x - bf16_to_float(hi[j]));
                    }
                    w[half] = (uint32_t)hi[0] | ((uint32_t)hi[1] << 16);
                    w[2 + half] = (uint32_t)lo[0] | ((uint32_t)lo[1] << 16);
                }
                for (int j = 0; j < 4; ++j) out[(((size_t)kt * (Nd / 8) + nt) * 32 + lane) * 4 + j] = w[j];
            }
}

// work buffers of fill_tile_tables: the four dense matrices (zero padded) and the
// table block in doubles
constexpr int kDenseMax = 8192;
constexpr int kTableWordsMax = 16384;
struct Work {
    double dense[4][kDenseMax];  // Phi [KP][NQP], WPhi [NQP][NP], Psi [B2K][NSP], PsiL [NSP][B2N]
    double t[kTableWordsMax];
};

// Tables of the tile kernels (TileTab<K, BK>): the basis at the volume points
// (zero padded), its weighted transpose, the 2D face basis and its weighted
// transpose -- dense for the CUDA-core products, fragment-ordered split-BF16
// for the tensor-core products -- then the dense basis at the volume and face
// points for the exact positivity check.  Written into out as words of the
// element type of prec (FP64, FP32, or FP32 with the BK_X3 fragments); returns
// the bytes written, 0 when out is too small.
template <int K, int BK>
size_t fill_tile_tables(int prec, Work& w, unsigned char* out, size_t cap)
{
    using Cf = TileCfg<K, BK>;
    using TT = TileTab<K, BK>;
    constexpr int b = Cf::b, n = Cf::n, nq = Cf::nq, ns = Cf::ns, nf = Cf::nf;
    constexpr int KP = Cf::KP, NQP = Cf::NQP, NP = Cf::NP, B2 = Cf::B2, B2K = Cf::B2K, NSP = Cf::NSP, B2N = Cf::B2N;
    static_assert(KP * NQP <= kDenseMax && NQP * NP <= kDenseMax && B2K * NSP <= kDenseMax &&
                      NSP * B2N <= kDenseMax && TT::total <= kTableWordsMax,
                  "table work buffers");
    const size_t bytes = (prec == DG_PREC_F64 ? sizeof(double) : sizeof(float)) * (size_t)TT::total;
    if (bytes > cap) return 0;
    constexpr Modes<K> M{};
    constexpr Modes2<K> M2{};
    double* phi_d = w.dense[0];
    double* wphi_d = w.dense[1];
    double* psi_d = w.dense[2];
    double* psil_d = w.dense[3];
    double* t = w.t;
    std::memset(w.dense, 0, sizeof(w.dense));
    std::memset(t, 0, sizeof(double) * TT::total);
    long double xg[16], wg[16];
    gauss_rule(n, xg, wg);
    auto phi = [&](int l, long double a, long double bb, long double c) {
        return pnorm(M.i[l], a) * pnorm(M.j[l], bb) * pnorm(M.l[l], c);
    };
    for (int q = 0; q < nq; ++q) {
        const int ia = q % n, ib = (q / n) % n, ic = q / (n * n);
        const long double wq = wg[ia] * wg[ib] * wg[ic] / 8.0L;
        for (int l = 0; l < b; ++l) {
            const long double p = phi(l, xg[ia], xg[ib], xg[ic]);
            phi_d[(size_t)l * NQP + q] = (double)p;
            wphi_d[(size_t)q * NP + l] = (double)(wq * p);
            t[TT::phiv + l * nq + q] = (double)p;
        }
    }
    for (int s = 0; s < ns; ++s) {
        const int a = s % n, c = s / n;
        const long double ws = wg[a] * wg[c];
        for (int p2 = 0; p2 < B2; ++p2) {
            const long double ps = pnorm(M2.p[p2], xg[a]) * pnorm(M2.q[p2], xg[c]);
            psi_d[(size_t)p2 * NSP + s] = (double)ps;
            psil_d[(size_t)s * B2N + p2] = (double)(ws * ps);
        }
    }
    for (int f = 0; f < 6; ++f) {
        const int d = f >> 1;
        const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
        for (int s = 0; s < ns; ++s) {
            long double xi[3];
            xi[d] = (f & 1) ? 1.0L : -1.0L;
            xi[t1] = xg[s % n];
            xi[t2] = xg[s / n];
            for (int l = 0; l < b; ++l) t[TT::phif + l * nf + f * ns + s] = (double)phi(l, xi[0], xi[1], xi[2]);
        }
    }
    const int sizes[4] = {KP * NQP, NQP * NP, B2K * NSP, NSP * B2N};
    const int offs[4] = {Cf::oPhi, Cf::oWPhi, Cf::oPsi, Cf::oPsiL};
    if (BK == BK_FMA)
        for (int i = 0; i < 4; ++i) std::memcpy(t + offs[i], w.dense[i], sizeof(double) * sizes[i]);
    if (prec == DG_PREC_F64) {
        std::memcpy(out, t, bytes);
        return bytes;
    }
    for (int j = 0; j < TT::total; ++j) {
        const float f = (float)t[j];
        std::memcpy(out + sizeof(float) * j, &f, sizeof(float));
    }
    if (BK == BK_X3) {
        uint32_t frag[kDenseMax];  // one fragment block: K*N words, as many as the dense matrix
        for (int i = 0; i < 4; ++i) {
            const int Kd = i == 0 ? KP : i == 1 ? NQP : i == 2 ? B2K : NSP;
            const int Nd = i == 0 ? NQP : i == 1 ? NP : i == 2 ? NSP : B2N;
            to_fragments(w.dense[i], Kd, Nd, frag);
            std::memcpy(out + sizeof(uint32_t) * offs[i], frag, sizeof(uint32_t) * (size_t)Kd * Nd);
        }
    }
    return bytes;
}

// the same for a run-time degree and precision
inline size_t fill_tile_tables_for(int K, int prec, Work& w, unsigned char* out, size_t cap)
{
    const bool x3 = prec == DG_PREC_X3;
    if (K == 1) return x3 ? fill_tile_tables<1, BK_X3>(prec, w, out, cap) : fill_tile_tables<1, BK_FMA>(prec, w, out, cap);
    if (K == 2) return x3 ? fill_tile_tables<2, BK_X3>(prec, w, out, cap) : fill_tile_tables<2, BK_FMA>(prec, w, out, cap);
    return x3 ? fill_tile_tables<3, BK_X3>(prec, w, out, cap) : fill_tile_tables<3, BK_FMA>(prec, w, out, cap);
}

}  // namespace tables
}  // namespace dg
