// dg_tile.cuh -- tile kernels of libdg: every basis <-> point transform of a
// tile of TC cells is a block-level matrix product staged in shared memory,
// with rows = (cell, field) so that one basis table serves the whole tile.
//
//   evaluation   V[(c,f)][q]  = sum_l A[(c,f)][l] Phi[l][q]          (Sec. 2.1)
//   projection   P[(c,g)][l]  = sum_q F[(c,g)][q] WPhi[q][l]         (Sec. 3.2, eq. weights_equation)
//   face traces  Tr[r][s]     = sum_p C2[r][p] Psi[p][s]             (2D basis on a face)
//   face lift    L2[r][p]     = sum_s Fs[r][s] PsiL[s][p]
// with WPhi = (w_q/8) Phi^T and PsiL = w_s Psi^T.  Derivatives are taken in
// modal space (exact in P_k): grad coefficients (2/h) D_d c and the weak-form
// volume term (2/h) sum_d D_d^T Fhat_d (Sec. 2.2, eq. weight_evolution).
// Traces on a face first collapse the normal direction with the known values
// Pn_m(+-1) = (+-1)^m sqrt(2m+1) and then evaluate a 2D expansion.
//
// The matrix products run on the CUDA cores as register-tiled FMA loops
// (FP64 and FP32 modes).  Shared-memory operands use padded leading
// dimensions (multiples of 4 elements) and 16-byte vector loads.
#pragma once

#include <cuda_bf16.h>

#include "dg_kernels.cuh"
#include "dg_mma.cuh"

namespace dg {

constexpr int r4(int x) { return (x + 3) / 4 * 4; }
constexpr int r8(int x) { return (x + 7) / 8 * 8; }

template <int K>
struct Modes2 {
    static constexpr int B2 = (K + 1) * (K + 2) / 2;
    int p[B2], q[B2];
    constexpr Modes2() : p{}, q{}
    {
        int c = 0;
        for (int d = 0; d <= K; ++d)
            for (int a = d; a >= 0; --a) {
                p[c] = a;
                q[c] = d - a;
                ++c;
            }
    }
};

template <int K>
constexpr int idx2(int p, int q)
{
    constexpr Modes2<K> M{};
    for (int i = 0; i < Modes2<K>::B2; ++i)
        if (M.p[i] == p && M.q[i] == q) return i;
    return -1;
}
// degree along the face normal d, and the 2D mode of the tangential degrees
// (tangential axes in increasing order)
template <int K>
constexpr int normal_deg(int d, int m)
{
    constexpr Modes<K> M{};
    return d == 0 ? M.i[m] : (d == 1 ? M.j[m] : M.l[m]);
}
template <int K>
constexpr int tang_mode(int d, int m)
{
    constexpr Modes<K> M{};
    const int a = (d == 0) ? M.j[m] : M.i[m];
    const int c = (d == 2) ? M.j[m] : M.l[m];
    return idx2<K>(a, c);
}
// sup of |phi_m| over the reference cell
template <int K>
constexpr double sup_phi(int m)
{
    constexpr Modes<K> M{};
    return csqrt((2.0 * M.i[m] + 1.0) * (2.0 * M.j[m] + 1.0) * (2.0 * M.l[m] + 1.0));
}

constexpr int r16(int x) { return (x + 15) / 16 * 16; }

enum { BK_FMA = 0, BK_X3 = 1 };

// BK_FMA: FP32/FP64 register-tiled FMA products; BK_X3: split-BF16 x3 tensor-
// core products (mma.sync m16n8k16, FP32 accumulate) -- K dims padded to 16,
// N dims to 8, row strides chosen for conflict-free fragment loads.
template <int K, int BK = BK_FMA>
struct TileCfg {
    using D = Dims<K>;
    static constexpr bool X = (BK == BK_X3);
    static constexpr int b = D::b, n = D::n, nq = D::nq, ns = D::ns, nf = D::nf;
    static constexpr int TC = (K == 1) ? 32 : 16;  // cells per tile
    static constexpr int NT = 256;                 // threads per block
    // evaluated fields: rho, m, grad rho, div m, a_h (11; the CUDA-core product keeps
    // a twelfth zero row for a 6x8 register tile, the tensor-core product needs 16-row tiles)
    static constexpr int FE = X ? 11 : 12;
    static constexpr int FP = 9;                   // projected components
    static constexpr int B2 = (K + 1) * (K + 2) / 2;
    static constexpr int KP = X ? r16(b) : r4(b);     // evaluation: K (modes)
    static constexpr int NQP = X ? r16(nq) : r8(nq);  // evaluation: N; projection: K (points)
    static constexpr int NP = X ? r8(b) : r4(b);      // projection: N (modes)
    static constexpr int B2K = X ? r16(B2) : r4(B2);  // face trace: K (2D modes)
    static constexpr int NSP = X ? r16(ns) : r4(ns);  // face trace: N; lift: K (face points)
    static constexpr int B2N = X ? r8(B2) : r4(B2);   // lift: N (2D modes)
    static constexpr int PADA = X ? 4 : 0, PADV = 4;
    static constexpr int LDA = KP + PADA;     // evaluation coefficients rows
    static constexpr int LDV = NQP + PADV;    // point values / point fluxes rows
    static constexpr int LDP = NP;            // projections rows
    static constexpr int LDC2 = B2K + PADA;   // collapsed face coefficients rows
    static constexpr int LDT = NSP + PADV;    // face traces / face fluxes rows
    static constexpr int LDL = B2N;           // lifted face fluxes rows
    static constexpr int RE = TC * FE;   // eval rows
    static constexpr int RP = TC * FP;   // projection rows
    static constexpr int RC = TC * 16;   // face rows per direction: cell x side x (self,nbr) x (rho,v)
    static constexpr int RL = TC * 8;    // face flux rows per direction: cell x side x var
    // B operands in shared memory: FMA -> dense T arrays [K][N]; X3 ->
    // fragments, K*N uint32 words [K/16][N/8][32 lanes][hi0 hi1 lo0 lo1]
    static constexpr int szPhi = KP * NQP;
    static constexpr int szWPhi = NQP * NP;
    static constexpr int szPsi = B2K * NSP;
    static constexpr int szPsiL = NSP * B2N;
    // shared-memory layout in elements of T (X3 tables count as 4-byte words
    // inside a float region), every offset a multiple of 4
    static constexpr int oPhi = 0;
    static constexpr int oWPhi = oPhi + szPhi;
    static constexpr int oPsi = oWPhi + szWPhi;
    static constexpr int oPsiL = oPsi + szPsi;
    static constexpr int tabsz = oPsiL + szPsiL;          // table block (global layout)
    static constexpr int smem_tabs = tabsz;               // tables copied to shared memory
    static constexpr int oU = r4(smem_tabs);              // [TC][4][b] state of the tile
    static constexpr int oVH = oU + r4(TC * 4 * b);       // [TC][3][b] own projected velocity
    static constexpr int oR = oVH + r4(TC * 3 * b);       // [TC][4][b] right-hand side
    static constexpr int oUn = oR + r4(TC * 4 * b);       // [TC][4][b] u^n, prefetched (stage mode)
    static constexpr int oAh = oUn + r4(TC * 4 * b);      // [TC][3][b] forcing coefficients of the tile
    // evaluation coefficients [RE][LDA]; the projections [RP][LDP] reuse the
    // region once the evaluation product has consumed the coefficients
    static constexpr int oA = oAh + r4(TC * 3 * b);
    static constexpr int oP = oA;
    static constexpr int SZA = (RE * LDA > RP * LDP) ? RE * LDA : RP * LDP;
    // big region: point values | point fluxes | faces.  Faces: region 1 holds
    // the collapsed coefficients, later the face fluxes; region 2 the traces,
    // later the lifted fluxes (each pair has disjoint lifetimes)
    static constexpr int FA = (RC * LDC2 > RL * LDT) ? RC * LDC2 : RL * LDT;
    static constexpr int FB = (RC * LDT > RL * LDL) ? RC * LDT : RL * LDL;
    static constexpr int BIGV = RE * LDV;
    static constexpr int oBig = oA + SZA;
    static constexpr int BIG = BIGV > FA + FB ? BIGV : FA + FB;
    static constexpr int total = oBig + BIG;
    static constexpr int oC2 = 0, oFs = 0, oTr = FA, oL2 = FA;
};

// tables in the caller's scratch for the tile kernels: the shared-memory
// block (same layout as in shared memory) followed by the dense FP values of
// phi at volume and face points used by the exact positivity check
template <int K, int BK = BK_FMA>
struct TileTab {
    using C = TileCfg<K, BK>;
    static constexpr int tabsz = C::tabsz;
    static constexpr int phiv = r4(tabsz);                        // [b][nq]
    static constexpr int phif = phiv + r4(C::b * C::nq);          // [b][nf]
    static constexpr int total = phif + C::b * C::nf;
};

// --------------------------------------------------------------------------
// vector helpers
// --------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T* o);
template <>
__device__ __forceinline__ void ld4<float>(const float* p, float* o)
{
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
}
template <>
__device__ __forceinline__ void ld4<double>(const double* p, double* o)
{
    const double2 v = *reinterpret_cast<const double2*>(p);
    const double2 w = *reinterpret_cast<const double2*>(p + 2);
    o[0] = v.x;
    o[1] = v.y;
    o[2] = w.x;
    o[3] = w.y;
}
template <typename T>
__device__ __forceinline__ void st4(T* p, const T* o);
template <>
__device__ __forceinline__ void st4<float>(float* p, const float* o)
{
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
}
template <>
__device__ __forceinline__ void st4<double>(double* p, const double* o)
{
    *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(o[2], o[3]);
}

// four elements p[e..e+3] of an array with `valid` readable elements: one
// 16-byte load when the chunk lies inside, element-wise (zero past the end)
// otherwise
template <typename T>
__device__ __forceinline__ void ld4_guard(const T* p, int e, int valid, T* o)
{
    if (e + 3 < valid) {
        ld4<T>(p + e, o);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = (e + j < valid) ? p[e + j] : T(0);
    }
}

// 16-byte asynchronous global -> shared copies (cp.async, cache-global)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// stage `count` elements of a tile into shared memory: 16-byte async copies for
// the chunks that lie inside the `valid` readable elements, plain loads (zero
// past the end) for a straddling chunk.  count and the base pointers are
// multiples of 16 bytes.
template <typename T, int NT>
__device__ __forceinline__ void stage_async(T* dst, const T* src, int count, int valid)
{
    constexpr int V = 16 / sizeof(T);
    for (int e = V * threadIdx.x; e < count; e += V * NT) {
        if (e + V <= valid) {
            cp_async16(dst + e, src + e);
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) dst[e + j] = (e + j < valid) ? src[e + j] : T(0);
        }
    }
}

// as stage_async for a state tile [cells][4][b] (B4 = 4b elements per cell):
// the cells past the end get rho_0 = 1 and zeros elsewhere, so that the
// padded cells stay finite.  Each 16-byte chunk is written by one thread.
template <typename T, int NT, int B4>
__device__ __forceinline__ void stage_async_state(T* dst, const T* src, int count, int valid)
{
    constexpr int V = 16 / sizeof(T);
    for (int e = V * threadIdx.x; e < count; e += V * NT) {
        if (e + V <= valid) {
            cp_async16(dst + e, src + e);
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j)
                dst[e + j] = (e + j < valid) ? src[e + j] : (((e + j) % B4) == 0 ? T(1) : T(0));
        }
    }
}

// reciprocal: in FP32 the hardware approximation (PTX rcp.approx) refined by
// one Newton-Raphson step r <- r + r (1 - x r), within about one ulp of 1/x
template <typename T>
__device__ __forceinline__ T rcp(T x)
{
    if constexpr (sizeof(T) == 4) {
        float r0;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(x));
        const float e = fmaf(-x, r0, 1.0f);
        return fmaf(r0, e, r0);
    } else {
        return T(1) / x;
    }
}

// --------------------------------------------------------------------------
// block GEMM on the CUDA cores: C[M][N] = A[M][K] B[K][N] (row-major, shared)
// thread micro-tile TM x TN with interleaved rows (row = mt + i*M/TM)
// --------------------------------------------------------------------------
constexpr int pick_tn(int N) { return (N % 8 == 0 && N >= 32) ? 8 : 4; }
constexpr int pick_tm(int M, int N, int NT)
{
    const int ncol = N / pick_tn(N);
    for (int tm = 1; tm <= 8; ++tm)
        if (M % tm == 0 && (M / tm) * ncol <= NT) return tm;
    for (int tm = 8; tm >= 1; --tm)
        if (M % tm == 0) return tm;
    return 1;
}

// WL: the product of one warp alone (NT = 32, its own rows), no block-wide split
template <typename T, int M, int N, int KK, int LDA, int LDB, int LDC, int NT, bool WL = false>
__device__ __forceinline__ void gemm_fma(const T* __restrict__ A, const T* __restrict__ B, T* __restrict__ Cm)
{
    constexpr int TN = pick_tn(N), TM = pick_tm(M, N, NT);
    constexpr int MT = M / TM, NCOL = N / TN;
    static_assert(M % TM == 0 && N % TN == 0 && KK % 4 == 0, "gemm shape");
    static_assert(LDA % 4 == 0 && LDB % 4 == 0 && LDC % 4 == 0, "gemm strides");
    for (int t = WL ? (threadIdx.x & 31) : threadIdx.x; t < MT * NCOL; t += NT) {
        const int mt = t / NCOL, nt = t % NCOL;
        T acc[TM][TN];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
#pragma unroll
        for (int k = 0; k < KK; k += 4) {
            T a[TM][4], bb[4][TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) ld4<T>(A + (mt + i * MT) * LDA + k, a[i]);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
#pragma unroll
                for (int j = 0; j < TN; j += 4) ld4<T>(B + (k + kk) * LDB + nt * TN + j, &bb[kk][j]);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[i][j] += a[i][kk] * bb[kk][j];
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; j += 4) st4<T>(Cm + (mt + i * MT) * LDC + nt * TN + j, &acc[i][j]);
    }
}

// --------------------------------------------------------------------------
// block GEMM on the tensor cores, split-BF16 x3 with FP32 accumulation:
//   a = a_hi + a_lo, b = b_hi + b_lo (bf16, round to nearest),
//   a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi   (relative error ~ 2^-16)
// A is FP32 in shared memory, split while forming the fragments; B is stored
// pre-split in fragment order (uint4 per lane and 16x8 tile).
// mma.sync.m16n8k16 fragments (lane = 4 g + t): A regs (g,2t) (g+8,2t)
// (g,2t+8) (g+8,2t+8); B regs (k=2t, n=g) (k=2t+8, n=g); C (g,2t) (g+8,2t).
// --------------------------------------------------------------------------
__device__ __forceinline__ void split_bf16x2(float x0, float x1, uint32_t& hi, uint32_t& lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

template <int M, int N, int KK, int LDA, int LDC, int NT, bool WL = false>
__device__ __forceinline__ void gemm_x3(const float* __restrict__ A, const uint4* __restrict__ Bf,
                                        float* __restrict__ Cm)
{
    constexpr int MT = M / 16, NTL = N / 8, KT = KK / 16, NW = NT / 32;
    static_assert(M % 16 == 0 && N % 8 == 0 && KK % 16 == 0 && LDA % 2 == 0 && LDC % 2 == 0, "x3 shape");
    static_assert(!WL || NT == 32, "a warp-local product runs on one warp");
    const int warp = WL ? 0 : (int)(threadIdx.x >> 5), lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (int mt = warp; mt < MT; mt += NW) {
        float acc[NTL][4];
#pragma unroll
        for (int j = 0; j < NTL; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) {
            const float* ap = A + (mt * 16 + g) * LDA + kt * 16 + 2 * t;
            const float2 x0 = *reinterpret_cast<const float2*>(ap);
            const float2 x1 = *reinterpret_cast<const float2*>(ap + 8 * LDA);
            const float2 x2 = *reinterpret_cast<const float2*>(ap + 8);
            const float2 x3 = *reinterpret_cast<const float2*>(ap + 8 * LDA + 8);
            uint32_t ah[4], al[4];
            split_bf16x2(x0.x, x0.y, ah[0], al[0]);
            split_bf16x2(x1.x, x1.y, ah[1], al[1]);
            split_bf16x2(x2.x, x2.y, ah[2], al[2]);
            split_bf16x2(x3.x, x3.y, ah[3], al[3]);
#pragma unroll
            for (int nt = 0; nt < NTL; ++nt) {
                const uint4 bf = Bf[(kt * NTL + nt) * 32 + lane];
                mma_bf16(acc[nt], al, bf.x, bf.y);
                mma_bf16(acc[nt], ah, bf.z, bf.w);
                mma_bf16(acc[nt], ah, bf.x, bf.y);
            }
        }
#pragma unroll
        for (int nt = 0; nt < NTL; ++nt) {
            *reinterpret_cast<float2*>(Cm + (mt * 16 + g) * LDC + nt * 8 + 2 * t) = make_float2(acc[nt][0], acc[nt][1]);
            *reinterpret_cast<float2*>(Cm + (mt * 16 + g + 8) * LDC + nt * 8 + 2 * t) =
                make_float2(acc[nt][2], acc[nt][3]);
        }
    }
}

// C[M][N] = A[M][KK] B[KK][N] with the backend of the tile configuration;
// B is the table at shared-memory offset OFF
template <typename T, int BK, int M, int N, int KK, int LDA, int LDC, int NT, bool WL = false>
__device__ __forceinline__ void mm(const T* A, const T* tabs, int off, T* Cm)
{
    if constexpr (BK == BK_X3) {
        gemm_x3<M, N, KK, LDA, LDC, NT, WL>(reinterpret_cast<const float*>(A),
                                            reinterpret_cast<const uint4*>(tabs + off), reinterpret_cast<float*>(Cm));
    } else {
        gemm_fma<T, M, N, KK, LDA, N, LDC, NT, WL>(A, tabs + off, Cm);
    }
}

// --------------------------------------------------------------------------
// collapse of a 3D expansion onto the face (d, side): coefficients of the 2D
// expansion in the tangential coordinates
// --------------------------------------------------------------------------
template <typename T, int K, int Dd, int NOUT>
__device__ __forceinline__ void collapse(const T* c, int side, T* c2)
{
    constexpr int b = Dims<K>::b;
#pragma unroll
    for (int p = 0; p < NOUT; ++p) c2[p] = T(0);
    static_for<0, b>([&](auto m) {
        constexpr int nd = normal_deg<K>(Dd, decltype(m)::value);
        constexpr int tm = tang_mode<K>(Dd, decltype(m)::value);
        constexpr double f = csqrt(2.0 * nd + 1.0);
        const T s = (side || !(nd & 1)) ? T(f) : T(-f);
        c2[tm] += s * c[decltype(m)::value];
    });
}

// R[m] += scale * Pn_{normal}(sigma) * L2[tang(m)],  sigma = side ? +1 : -1
template <typename T, int K, int Dd>
__device__ __forceinline__ void expand_acc(const T* L2, int side, T scale, T* R)
{
    constexpr int b = Dims<K>::b;
    static_for<0, b>([&](auto m) {
        constexpr int nd = normal_deg<K>(Dd, decltype(m)::value);
        constexpr int tm = tang_mode<K>(Dd, decltype(m)::value);
        constexpr double f = csqrt(2.0 * nd + 1.0);
        const T s = (side || !(nd & 1)) ? T(f) : T(-f);
        R[decltype(m)::value] += scale * s * L2[tm];
    });
}

// kernel modes: projection only; RHS only; RHS + stage combine (+ the next
// stage's projection with F_NEXTPROJ); the same with the projection of |v|
// for the learned sensor's features (the last stage of a learned-mode step)
// Diffusion across the faces along Dd (div(eps grad u), Sec. 2): the interface
// gradient is the normal derivative of the polynomial recovered over the two
// cells of a face, per tangential mode tau a combination of the two cells'
// normal coefficient columns, g_tau = sum_a recL[K_tau][a] cL + recR[K_tau][a] cR
// (K_tau + 1 normal modes).  Its lift is exact in modal space:
//   + face of the cell: R_m += (2 eps / h^2) Pn_a(+1) g_tau,
//   - face of the cell: R_m -= (2 eps / h^2) Pn_a(-1) g_tau.
template <typename T, int K, int Dd>
__device__ __forceinline__ void diffusion_faces(const Phys& ph, const T* self, const T* minus, const T* plus, T* R)
{
    constexpr int b = Dims<K>::b, B2 = (K + 1) * (K + 2) / 2;
    constexpr Modes<K> M{};
    T gp[B2], gm[B2];
#pragma unroll
    for (int p = 0; p < B2; ++p) gp[p] = gm[p] = T(0);
    static_for<0, b>([&](auto mm) {
        constexpr int m = decltype(mm)::value;
        constexpr int nd = normal_deg<K>(Dd, m), tm = tang_mode<K>(Dd, m);
        constexpr int Kt = K - (M.i[m] + M.j[m] + M.l[m] - nd);
        // + face: left = this cell, right = the + neighbour; - face: left = the - neighbour
        gp[tm] += T(ph.recL[Kt][nd]) * self[m] + T(ph.recR[Kt][nd]) * plus[m];
        gm[tm] += T(ph.recL[Kt][nd]) * minus[m] + T(ph.recR[Kt][nd]) * self[m];
    });
    const T scale = T(2.0 * ph.eps / (ph.h * ph.h));
    static_for<0, b>([&](auto mm) {
        constexpr int m = decltype(mm)::value;
        constexpr int nd = normal_deg<K>(Dd, m), tm = tang_mode<K>(Dd, m);
        constexpr double f = csqrt(2.0 * nd + 1.0);
        constexpr double fm = (nd & 1) ? -f : f;
        R[m] += scale * (T(f) * gp[tm] - T(fm) * gm[tm]);
    });
}

enum { TM_PROJECT = 0, TM_RHS = 1, TM_STAGE = 2, TM_STAGE_VABS = 3 };
enum { F_NEXTPROJ = 4, F_VABS = 8, F_SELFPROJ = 16 };

template <typename T>
struct TArgs {
    const T* u_in;     // u^(s)
    const T* u_n;      // u^n
    T* out;            // u^(s+1) or dudt
    const T* vh_in;    // projected velocity of u_in [c][3][b]
    T* vh_out;         // projected velocity of the output (fused projection / K_A)
    const T* ahat;     // forcing coefficients or nullptr
    const T* tab;      // TileTab tables
    Ctl* ctl;
    double* partials;
    long ncell;
    int N;
    Phys ph;
    T rk_a, rk_b;
    double dt_pimax;
    int flags;         // F_DT | F_FORCE | F_NEXTPROJ | F_VABS
    int abar_in;       // slot of ctl->abar2 read by this stage
    int abar_out;      // slot written by the projection
    const float* nu;   // per-cell viscous coefficient (learned sensor) or nullptr
    T* vabs_out;       // projection of |v| (F_VABS) [c][b] or nullptr
    float* nu_next;    // last stage of a learned step: the coefficient of u^(n+1), or nullptr
    const uint32_t* mlp;  // packed sensor network (MlpPack<2b>) for nu_next
    unsigned char* trouble;  // positivity by repetition: per-cell marks (stage launches), or nullptr
};

// viscous pressure with a per-cell coefficient (learned sensor):
// Pi = rho nu |div v| for div v < 0, capped like the vNR form (Sec. 3.1)
template <typename T>
__device__ __forceinline__ T nu_pressure(const AvCoef<T>& cf, T rho, T divv, T nu)
{
    if (!(divv < T(0))) return T(0);
    const T ra = rho * (-divv);
    T Pi = ra * nu;
    if (cf.cap >= T(0)) {
        const T Pm = ra * cf.cap;
        Pi = Pi < Pm ? Pi : Pm;
    }
    return Pi;
}

// --------------------------------------------------------------------------
// projection of the primitive velocity of the TC states in sU (Sec. 3.2),
// the per-cell forcing sums <rho a_h> = sum_l rho_l a_l and the CFL maximum
// --------------------------------------------------------------------------
// per-cell forcing sums <rho a_h> = sum_l rho_l a_l (orthonormal basis) and <rho>
template <typename T, int K, int BK>
__device__ __forceinline__ void forcing_sums(const T* sm, const T* sU, const TArgs<T>& a, long c0, double* sums)
{
    using C = TileCfg<K, BK>;
    constexpr int b = C::b, TC = C::TC;
    const T* sAh = sm + C::oAh;
    const long nvalid = (a.ncell - c0) < TC ? (a.ncell - c0) : TC;
    if (threadIdx.x < TC * 3) {
        const int c = threadIdx.x / 3, i = threadIdx.x % 3;
        if (c < nvalid) {
            const T* u = sU + c * 4 * b;
            const T* ah = sAh + (c * 3 + i) * b;
            T s = T(0);
#pragma unroll
            for (int l = 0; l < b; ++l) s += u[l] * ah[l];
            sums[i] += (double)s;
            if (i == 0) sums[3] += (double)u[0];
        }
    }
}

template <typename T, int K, int BK, bool VABS = false>
__device__ __forceinline__ void tile_project(T* sm, const T* sU, const T* tabs, const TArgs<T>& a, long c0, bool dt_flag,
                                             T& smax, double* sums, bool with_sums)
{
    constexpr int NPR = VABS ? 4 : 3;  // projected rows per cell: v (and |v|)
    using C = TileCfg<K, BK>;
    constexpr int b = C::b, nq = C::nq, TC = C::TC, NT = C::NT, KP = C::KP, NQP = C::NQP, NP = C::NP;
    constexpr int LDA = C::LDA, LDV = C::LDV, LDP = C::LDP;
    T* sA = sm + C::oA;
    T* sV = sm + C::oBig;
    T* sP = sm + C::oP;
    // rows (cell, field) for rho, m_x, m_y, m_z
    for (int e = threadIdx.x; e < TC * 4 * KP; e += NT) {
        const int r = e / KP, l = e % KP;
        sA[r * LDA + l] = (l < b) ? sU[r * b + l] : T(0);
    }
    __syncthreads();
    mm<T, BK, TC * 4, NQP, KP, LDA, LDV, NT>(sA, tabs, C::oPhi, sV);
    __syncthreads();
    // v = m / rho at the volume points; rows (cell, i) of the projection input
    constexpr int PER = (TC * NQP + NT - 1) / NT;
    T vv[PER][NPR];
#pragma unroll
    for (int it = 0; it < PER; ++it) {
        const int e = threadIdx.x + it * NT;
#pragma unroll
        for (int i = 0; i < NPR; ++i) vv[it][i] = T(0);
        if (e < TC * NQP) {
            const int c = e / NQP, q = e % NQP;
            if (q < nq) {
                const T* v = sV + (c * 4) * LDV + q;
                const T ir = rcp<T>(v[0]);
                vv[it][0] = v[LDV] * ir;
                vv[it][1] = v[2 * LDV] * ir;
                vv[it][2] = v[3 * LDV] * ir;
                if constexpr (VABS)
                    vv[it][NPR - 1] = sqrt(vv[it][0] * vv[it][0] + vv[it][1] * vv[it][1] + vv[it][2] * vv[it][2]);
                if (dt_flag && c0 + c < a.ncell) {
                    const T sp = fabs(vv[it][0]) + fabs(vv[it][1]) + fabs(vv[it][2]);
                    smax = sp > smax ? sp : smax;
                }
                // positivity by repetition: a stage output faster than the
                // Courant condition of its step allows marks its cell
                if (a.trouble && c0 + c < a.ncell &&
                    fabs(vv[it][0]) + fabs(vv[it][1]) + fabs(vv[it][2]) > T(DG_REPEAT_SPEED * a.ctl->sn - 3.0 * a.ph.cs)) {
                    a.trouble[c0 + c] |= DG_MARK_FAST;
                    atomicOr(&a.ctl->status, DG_ST_TROUBLED_);
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < PER; ++it) {
        const int e = threadIdx.x + it * NT;
        if (e < TC * NQP) {
            const int c = e / NQP, q = e % NQP;
            T* f = sV + (c * NPR) * LDV + q;
#pragma unroll
            for (int i = 0; i < NPR; ++i) f[i * LDV] = vv[it][i];
        }
    }
    __syncthreads();
    mm<T, BK, TC * NPR, NP, NQP, LDV, LDP, NT>(sV, tabs, C::oWPhi, sP);
    __syncthreads();
    for (int e = threadIdx.x; e < TC * 3 * b; e += NT) {
        const int r = e / b, l = e % b, c = r / 3, i = r % 3;
        if (c0 + c < a.ncell) a.vh_out[c0 * 3 * b + e] = sP[(c * NPR + i) * LDP + l];
    }
    if constexpr (VABS) {
        if (a.vabs_out) {
            for (int e = threadIdx.x; e < TC * b; e += NT) {
                const int c = e / b, l = e % b;
                if (c0 + c < a.ncell) a.vabs_out[c0 * b + e] = sP[(c * NPR + 3) * LDP + l];
            }
        }
    }
    if (with_sums && (a.flags & F_FORCE)) forcing_sums<T, K, BK>(sm, sU, a, c0, sums);
}

// --------------------------------------------------------------------------
// learned sensor for the next step, evaluated in the last stage after the
// projection of |v| of u^(n+1): features x = (rho_l/rho_0, |v|hat_l/cs) of the
// tile's cells, nu = cs h/p exp(net(x)), 0 below the gate.  The network is the
// one of the separate inference kernel (BF16 inputs, weights and hidden
// activations, FP32 accumulation), spread over the block: warp w computes the
// hidden units 8w..8w+7 of both layers (one n-tile) for all the tile's cells,
// the BF16 activations pass through shared memory, and the first TC/16 warps
// form the outputs.  Products, roundings and accumulation orders are those of
// the separate kernel, so the coefficients agree bit for bit.
// --------------------------------------------------------------------------
// the network of the learned sensor for TC cells, spread over a block of NT =
// 256 threads: feat(c, k) gives input k of cell c (called for c < TC, k < KD);
// sX, sH1, sH2 are shared buffers of TC*KD/2, TC*32 and TC*32 words; writes
// nu_out[c0 + c] for the cells below ncell.  Ends without a trailing barrier.
template <int D, int TC, int NT, typename F>
__device__ __forceinline__ void block_mlp(F&& feat, uint32_t* sX, uint32_t* sH1, uint32_t* sH2, const uint32_t* mlp,
                                          float ref, float gate, long c0, long ncell, float* nu_out)
{
    using PK = MlpPack<D>;
    constexpr int XW = PK::KD / 2, KT1 = PK::KD / 16, MT = TC / 16, HW = MLP_H / 2;
    static_assert(NT / 32 == MLP_H / 8 && TC % 16 == 0, "one warp per 8 hidden units, 16-cell row blocks");
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    for (int e = tid; e < TC * XW; e += NT) {
        const int c = e / XW, k0 = 2 * (e % XW);
        sX[e] = pack_bf16x2(feat(c, k0), feat(c, k0 + 1));
    }
    // the warp's weight fragments and biases, loaded up front (their latency
    // overlaps the feature phase)
    const uint2* B1 = reinterpret_cast<const uint2*>(mlp + PK::w1);
    const uint2* B2 = reinterpret_cast<const uint2*>(mlp + PK::w2);
    const uint2* B3 = reinterpret_cast<const uint2*>(mlp + PK::w3);
    const float* bias = reinterpret_cast<const float*>(mlp + PK::bias);
    uint2 w1f[KT1], w2f[4], w3f[4];
#pragma unroll
    for (int kt = 0; kt < KT1; ++kt) w1f[kt] = __ldg(B1 + (kt * 8 + w) * 32 + lane);
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        w2f[kt] = __ldg(B2 + (kt * 8 + w) * 32 + lane);
        w3f[kt] = __ldg(B3 + kt * 32 + lane);
    }
    const int col = w * 8 + 2 * t;
    const float bs1[2] = {__ldg(bias + col), __ldg(bias + col + 1)};
    const float bs2[2] = {__ldg(bias + MLP_H + col), __ldg(bias + MLP_H + col + 1)};
    const float b3 = __ldg(bias + 2 * MLP_H);
    // A fragment of rows mt*16 + (g, g+8), k-chunk kt, from a [rows][ld] array of BF16 pairs
    auto frag = [&](const uint32_t* src, int ld, int mt, int kt, uint32_t* A) {
        const uint32_t* p = src + (mt * 16 + g) * ld + kt * 8 + t;
        A[0] = p[0];
        A[1] = p[8 * ld];
        A[2] = p[4];
        A[3] = p[8 * ld + 4];
    };
    // bias + GELU of the warp's n-tile, stored as BF16 pairs (rows g, g+8; columns 8w+2t, +1)
    auto act = [&](const float* acc, const float* bs, uint32_t* dst, int mt) {
        dst[(mt * 16 + g) * HW + col / 2] = pack_bf16x2(gelu_infer(acc[0] + bs[0]), gelu_infer(acc[1] + bs[1]));
        dst[(mt * 16 + g + 8) * HW + col / 2] = pack_bf16x2(gelu_infer(acc[2] + bs[0]), gelu_infer(acc[3] + bs[1]));
    };
    __syncthreads();
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < KT1; ++kt) {
            uint32_t A[4];
            frag(sX, XW, mt, kt, A);
            mma_bf16(acc, A, w1f[kt].x, w1f[kt].y);
        }
        act(acc, bs1, sH1, mt);
    }
    __syncthreads();
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            uint32_t A[4];
            frag(sH1, HW, mt, kt, A);
            mma_bf16(acc, A, w2f[kt].x, w2f[kt].y);
        }
        act(acc, bs2, sH2, mt);
    }
    __syncthreads();
    if (w < MT) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            uint32_t A[4];
            frag(sH2, HW, w, kt, A);
            mma_bf16(acc, A, w3f[kt].x, w3f[kt].y);
        }
        if (t == 0) {
            const float y[2] = {acc[0] + b3, acc[2] + b3};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long r = c0 + w * 16 + g + 8 * h;
                if (r < ncell) nu_out[r] = expf(y[h]) < gate ? 0.f : ref * expf(y[h]);
            }
        }
    }
}

// the fused stage kernel's tile: needs the big region free (after the
// projection) and sP holding the projections (rows cell x (v_x, v_y, v_z, |v|))
template <typename T, int K, int BK>
__device__ __forceinline__ void tile_nu(T* sm, const T* sU, const TArgs<T>& a, long c0)
{
    using C = TileCfg<K, BK>;
    constexpr int b = C::b, TC = C::TC, NT = C::NT, LDP = C::LDP, D = 2 * b;
    using PK = MlpPack<D>;
    constexpr int XW = PK::KD / 2, HW = MLP_H / 2;
    static_assert((TC * XW + 2 * TC * HW) * 4 <= C::BIG * (int)sizeof(T), "network buffers in the big region");
    uint32_t* sX = reinterpret_cast<uint32_t*>(sm + C::oBig);  // [TC][XW] BF16 pairs of features
    uint32_t* sH1 = sX + TC * XW;                              // [TC][HW] first hidden layer
    uint32_t* sH2 = sH1 + TC * HW;                             // [TC][HW] second hidden layer
    const T* sP = sm + C::oP;
    const float inv_cs = 1.0f / (float)a.ph.cs;
    auto feat = [&](int c, int k) -> float {
        if (c0 + c >= a.ncell || k >= D) return 0.0f;
        if (k < b) return (float)(sU[c * 4 * b + k] / sU[c * 4 * b]);
        return (float)sP[(c * 4 + 3) * LDP + (k - b)] * inv_cs;
    };
    block_mlp<D, TC, NT>(feat, sX, sH1, sH2, a.mlp, (float)(a.ph.cs * a.ph.hp), (float)a.ph.nu_gate, c0, a.ncell,
                         a.nu_next);
    // the next tile starts with a barrier before it writes the big region
}

// DIFF: the diffusion operator div(eps grad u) is compiled in (a separate
// instantiation, so that the plain scheme carries none of its code)
template <typename T, int K, int MODE, int BK, bool DIFF = false>
__global__ void __launch_bounds__(256) k_tile(TArgs<T> a)
{
    using C = TileCfg<K, BK>;
    using TT = TileTab<K, BK>;
    using Dm = Dims<K>;
    constexpr int b = C::b, nq = C::nq, ns = C::ns, nf = C::nf, TC = C::TC, NT = C::NT;
    constexpr int FE = C::FE, KP = C::KP, NQP = C::NQP, NP = C::NP, B2K = C::B2K, NSP = C::NSP, B2N = C::B2N;
    constexpr int LDA = C::LDA, LDV = C::LDV, LDP = C::LDP, LDC2 = C::LDC2, LDT = C::LDT, LDL = C::LDL;
    constexpr int RE = C::RE, RP = C::RP;
    static_assert(BK == BK_FMA || sizeof(T) == 4, "the tensor-core path is FP32");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    T* sU = sm + C::oU;
    T* sVH = sm + C::oVH;
    T* sR = sm + C::oR;
    T* sA = sm + C::oA;
    T* sP = sm + C::oP;
    T* sBig = sm + C::oBig;
    __shared__ T s_nu[TC];
    __shared__ unsigned int s_status;
    __shared__ double s_tot[8];
    // block reductions after the tile loop use the (then free) big region
    double* s_buf = reinterpret_cast<double*>(sm + C::oBig);
    static_assert(C::BIG * sizeof(T) >= NT * sizeof(double), "reduction buffer");
    __shared__ unsigned long long s_smax;

    const int tid = threadIdx.x;
    // sup |phi_m| of the mode m = lane (positivity bound), 0 past the modes
    T my_sup = T(0);
    static_for<0, b>([&](auto m) {
        if ((int)(tid & 31) == decltype(m)::value) my_sup = T(sup_phi<K>(decltype(m)::value));
    });
    // tables -> shared (once per block)
    for (int e = tid; e < C::smem_tabs; e += NT) sm[e] = a.tab[e];
    const T* tabs = sm;
    T* sUn = sm + C::oUn;
    T* sAh = sm + C::oAh;
    if (tid == 0) {
        s_status = 0u;
        s_smax = 0ull;
    }
    const long ntile = (a.ncell + TC - 1) / TC;
    const bool force = (a.flags & F_FORCE) != 0;
    const T two_h = T(2.0 / a.ph.h);
    const T inv4h = T(0.25 / a.ph.h);
    const T cs = T(a.ph.cs), cs2 = T(a.ph.cs2);
    T smax = T(0);
    double sums[4] = {0.0, 0.0, 0.0, 0.0};
    bool need_div = true;
    uint32_t ntiles = 0, gated = 0;  // volume tiles done, and those without div v
    constexpr bool STAGE = (MODE == TM_STAGE || MODE == TM_STAGE_VABS);
    const bool do_proj = (MODE == TM_PROJECT) || (STAGE && (a.flags & F_NEXTPROJ));
    T dt = T(0), ab0 = T(0), ab1 = T(0), ab2 = T(0);
    AvCoef<T> avc{};
    const T diff_vol = T(-4.0 * a.ph.eps / (a.ph.h * a.ph.h));
    if constexpr (MODE != TM_PROJECT) {
        if constexpr (STAGE) {
            // the step's dt (Sec. 7 CFL condition), fixed for all its stages: from the
            // wave-speed bound of u^n, a prescribed dt, and the retry factor
            const double sn = a.ctl->sn;
            double dtc = a.ctl->dt_num / sn;
            if (a.ctl->dt_diff > 0.0 && a.ctl->dt_diff < dtc) dtc = a.ctl->dt_diff;
            const double dtd = (a.ctl->fixed_dt > 0.0 ? a.ctl->fixed_dt : dtc) * a.ctl->dt_scale;
            dt = T(dtd);
            avc = av_coef<T>(a.ph, dtd);
            if (blockIdx.x == 0 && tid == 0) a.ctl->dt = dtd;
        } else {
            dt = T(a.dt_pimax);
            avc = av_coef<T>(a.ph, a.dt_pimax);
        }
        if (force) {
            ab0 = T(a.ctl->abar2[a.abar_in][0]);
            ab1 = T(a.ctl->abar2[a.abar_in][1]);
            ab2 = T(a.ctl->abar2[a.abar_in][2]);
        }
    }
    // stage mode: the inputs of a tile (u^(s), its projected velocity, a_h, u^n)
    // are fetched asynchronously while the previous tile finishes (its
    // projection for the next stage); u lands in the right-hand-side buffer,
    // free by then, and is moved to the state buffer when the tile starts
    auto issue = [&](long t, T* dU) {
        const long cb = t * TC;
        const int nv = (int)((a.ncell - cb) < TC ? (a.ncell - cb) : TC);
        stage_async_state<T, NT, 4 * b>(dU, a.u_in + cb * 4 * b, TC * 4 * b, nv * 4 * b);
        stage_async<T, NT>(sVH, a.vh_in + cb * 3 * b, TC * 3 * b, nv * 3 * b);
        if (force) stage_async<T, NT>(sAh, a.ahat + cb * 3 * b, TC * 3 * b, nv * 3 * b);
        if (a.rk_a != T(0)) stage_async<T, NT>(sUn, a.u_n + cb * 4 * b, TC * 4 * b, nv * 4 * b);
        cp_async_commit();
    };
    if constexpr (STAGE) {
        if (blockIdx.x < ntile) issue(blockIdx.x, sU);
    }
    __syncthreads();

    for (long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const long c0 = tile * TC;
        const long nvalid = (a.ncell - c0) < TC ? (a.ncell - c0) : TC;
        if constexpr (STAGE) {
            if (tid < TC) s_nu[tid] = (a.ph.av_mode == 2 && tid < nvalid) ? T(a.nu[c0 + tid]) : T(0);
            cp_async_wait_all();
            __syncthreads();
            if (tile != blockIdx.x) {
                // prefetched into the right-hand-side buffer (free at the time):
                // move to the state buffer (fixed buffers keep the addressing static)
                for (int e = 4 * tid; e < TC * 4 * b; e += 4 * NT) {
                    T v[4];
                    ld4<T>(sR + e, v);
                    st4<T>(sU + e, v);
                }
                __syncthreads();
            }
        } else {
            // ---- stage the tile (cells past the end: rho = 1, everything else 0) ----
            for (int e = 4 * tid; e < TC * 4 * b; e += 4 * NT) {
                T v[4];
                ld4_guard<T>(a.u_in + c0 * 4 * b, e, (int)nvalid * 4 * b, v);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if ((e + j) / (4 * b) >= nvalid) v[j] = ((e + j) % (4 * b)) == 0 ? T(1) : T(0);
                st4<T>(sU + e, v);
            }
            if (force) stage_async<T, NT>(sAh, a.ahat + c0 * 3 * b, TC * 3 * b, (int)nvalid * 3 * b);
            cp_async_commit();
            if constexpr (MODE == TM_PROJECT) {
                cp_async_wait_all();
                __syncthreads();
                if (a.flags & F_VABS)
                    tile_project<T, K, BK, true>(sm, sU, tabs, a, c0, (a.flags & F_DT) != 0, smax, sums, true);
                else
                    tile_project<T, K, BK, false>(sm, sU, tabs, a, c0, (a.flags & F_DT) != 0, smax, sums, true);
                __syncthreads();
                continue;
            }
            if (tid < TC) s_nu[tid] = (a.ph.av_mode == 2 && tid < nvalid) ? T(a.nu[c0 + tid]) : T(0);
            for (int e = 4 * tid; e < TC * 3 * b; e += 4 * NT) {
                T v[4];
                ld4_guard<T>(a.vh_in + c0 * 3 * b, e, (int)nvalid * 3 * b, v);
                st4<T>(sVH + e, v);
            }
            cp_async_wait_all();
            __syncthreads();
        }
        if constexpr (MODE != TM_PROJECT) {
            for (int e = tid; e < TC * 3 * b; e += NT) {
                const int c = e / (3 * b), i = (e / b) % 3, l = e % b;
                sA[(c * FE + 8 + i) * LDA + l] = (force && c < nvalid) ? sAh[e] : T(0);
            }
            // the gradient rows and the viscous pressure are needed unless every
            // cell of the tile has a zero coefficient (learned sensor gated off,
            // or no viscosity): a tile-uniform decision (s_nu was written before
            // the last barrier)
            need_div = a.ph.av_mode == 1;
            if (a.ph.av_mode == 2)
                for (int c = 0; c < TC; ++c) need_div |= s_nu[c] != T(0);
            ++ntiles;
            gated += need_div ? 0u : 1u;
            // ---- evaluation coefficients: rho, m, grad rho, div m, (a_h staged above) ----
            // threads run field-major (a warp covers one or two fields, so the
            // per-field branches below do not diverge within it)
            for (int e = tid; e < RE; e += NT) {
                const int f = e / TC, c = e % TC;
                const T* u = sU + c * 4 * b;
                T* row = sA + (c * FE + f) * LDA;
                if (f >= 4 && f < 8 && !need_div) {
#pragma unroll
                    for (int l = 0; l < KP; ++l) row[l] = T(0);
                    continue;
                }
                if (f >= 8 && f < 11) {
#pragma unroll
                    for (int l = b; l < KP; ++l) row[l] = T(0);
                    continue;
                }
                T out[KP];
#pragma unroll
                for (int l = b; l < KP; ++l) out[l] = T(0);
                if (f < 4) {
                    if constexpr (b % 4 == 0) {
#pragma unroll
                        for (int l = 0; l < b; l += 4) ld4<T>(u + f * b + l, out + l);
                    } else {
#pragma unroll
                        for (int l = 0; l < b; ++l) out[l] = u[f * b + l];
                    }
                } else if (f == 4) {
                    modal_grad<T, K, 0>(u, out, two_h);
                } else if (f == 5) {
                    modal_grad<T, K, 1>(u, out, two_h);
                } else if (f == 6) {
                    modal_grad<T, K, 2>(u, out, two_h);
                } else if (f == 7) {
                    T t2[b];
                    modal_grad<T, K, 0>(u + b, out, two_h);
                    modal_grad<T, K, 1>(u + 2 * b, t2, two_h);
#pragma unroll
                    for (int l = 0; l < b; ++l) out[l] += t2[l];
                    modal_grad<T, K, 2>(u + 3 * b, t2, two_h);
#pragma unroll
                    for (int l = 0; l < b; ++l) out[l] += t2[l];
                } else {
#pragma unroll
                    for (int l = 0; l < b; ++l) out[l] = T(0);
                }
                static_assert(KP % 4 == 0 && LDA % 4 == 0, "row vectors");
#pragma unroll
                for (int l = 0; l < KP; l += 4) st4<T>(row + l, out + l);
            }
            __syncthreads();
            // ---- evaluation at the volume points ----
            mm<T, BK, RE, NQP, KP, LDA, LDV, NT>(sA, tabs, C::oPhi, sBig);
            __syncthreads();
            // ---- pointwise volume physics (Sec. 3.1: Pi at internal points only) ----
            constexpr int PER = (TC * NQP + NT - 1) / NT;
            T fl[PER][9];
#pragma unroll
            for (int it = 0; it < PER; ++it) {
                const int e = tid + it * NT;
#pragma unroll
                for (int g = 0; g < 9; ++g) fl[it][g] = T(0);
                if (e < TC * NQP) {
                    const int c = e / NQP, q = e % NQP;
                    if (q < nq) {
                        const T* v = sBig + (c * FE) * LDV + q;
                        const T rho = v[0], ir = rcp<T>(rho);
                        const T mx = v[LDV], my = v[2 * LDV], mz = v[3 * LDV];
                        const T vx = mx * ir, vy = my * ir, vz = mz * ir;
                        T Pi = T(0);
                        if (need_div) {
                            const T divv =
                                (v[7 * LDV] - (vx * v[4 * LDV] + vy * v[5 * LDV] + vz * v[6 * LDV])) * ir;
                            if (a.ph.av_mode == 1)
                                Pi = vnr_pressure<T>(avc, rho, divv);
                            else
                                Pi = nu_pressure<T>(avc, rho, divv, s_nu[c]);
                        }
                        const T P = cs2 * rho + Pi;
                        fl[it][0] = mx * vx + P;
                        fl[it][1] = my * vy + P;
                        fl[it][2] = mz * vz + P;
                        fl[it][3] = mx * vy;
                        fl[it][4] = mx * vz;
                        fl[it][5] = my * vz;
                        fl[it][6] = rho * (v[8 * LDV] - ab0);
                        fl[it][7] = rho * (v[9 * LDV] - ab1);
                        fl[it][8] = rho * (v[10 * LDV] - ab2);
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int it = 0; it < PER; ++it) {
                const int e = tid + it * NT;
                if (e < TC * NQP) {
                    const int c = e / NQP, q = e % NQP;
                    T* f = sBig + (c * 9) * LDV + q;
#pragma unroll
                    for (int g = 0; g < 9; ++g) f[g * LDV] = fl[it][g];
                }
            }
            __syncthreads();
            // ---- projection of the flux tensor and the forcing density ----
            mm<T, BK, RP, NP, NQP, LDV, LDP, NT>(sBig, tabs, C::oWPhi, sP);
            __syncthreads();
            // ---- the face phase is warp-local: warp w owns the cells
            // [w CPW, (w+1) CPW) of the tile, their RCW face rows r = w RCW + rl
            // (rl = lane + 32 j) and their flux rows, so its steps need no
            // block barrier; the neighbour coefficients of the face rows are
            // fetched one face direction ahead, overlapping the previous phase ----
            constexpr int NW = NT / 32, CPW = TC / NW, RCW = CPW * 16, RLW = CPW * 8, NR = RCW / 32;
            static_assert(TC % NW == 0 && RCW % 32 == 0, "face rows per warp");
            static_assert(RLW * LDT <= RCW * LDC2 && RLW * LDL <= RCW * LDT, "warp flux rows fit the row blocks");
            const int wid = tid >> 5, lane = tid & 31;
            T nbr[NR][b];
            // mesh coordinates of the cell of each of the lane's face rows
            int cxyz[NR][3];
#pragma unroll
            for (int j = 0; j < NR; ++j)
                cell_xyz(c0 + ((wid * RCW + lane + 32 * j) >> 4), a.N, cxyz[j][0], cxyz[j][1], cxyz[j][2]);
            auto load_nbr = [&](auto dd) {
                constexpr int Dd = decltype(dd)::value;
#pragma unroll
                for (int j = 0; j < NR; ++j) {
                    const int r = wid * RCW + lane + 32 * j;
                    const int field = r & 3, who = (r >> 2) & 1, side = (r >> 3) & 1, c = r >> 4;
                    const long cc = c0 + c;
                    if (who == 1 && cc < a.ncell) {
                        const long nc = neighbour_along<Dd>(cc, cxyz[j][Dd], side, a.N);
                        const T* src = (field == 0) ? a.u_in + nc * 4 * b : a.vh_in + (nc * 3 + field - 1) * b;
                        if constexpr (b % 4 == 0) {
#pragma unroll
                            for (int l = 0; l < b; l += 4) ld4<T>(src + l, nbr[j] + l);
                        } else {
#pragma unroll
                            for (int l = 0; l < b; ++l) nbr[j][l] = __ldg(src + l);
                        }
                    } else {
#pragma unroll
                        for (int l = 0; l < b; ++l) nbr[j][l] = (field == 0 && l == 0) ? T(1) : T(0);
                    }
                }
            };
            load_nbr(std::integral_constant<int, 0>{});
            // ---- volume term in modal space + forcing source ----
            // (variable-major threads: the v == 0 and v > 0 branches split by warp)
            for (int e = tid; e < TC * 4; e += NT) {
                const int v = e / TC, c = e % TC;
                T r[b];
#pragma unroll
                for (int l = 0; l < b; ++l) r[l] = T(0);
                const T* P = sP + c * 9 * LDP;
                if (v == 0) {
                    const T* u = sU + c * 4 * b;
                    modal_grad_T_acc<T, K, 0>(u + b, r, two_h);
                    modal_grad_T_acc<T, K, 1>(u + 2 * b, r, two_h);
                    modal_grad_T_acc<T, K, 2>(u + 3 * b, r, two_h);
                } else {
                    const int i = v - 1;
                    const int cx = (i == 0) ? 0 : (i == 1 ? 3 : 4);
                    const int cy = (i == 0) ? 3 : (i == 1 ? 1 : 5);
                    const int cz = (i == 0) ? 4 : (i == 1 ? 5 : 2);
                    modal_grad_T_acc<T, K, 0>(P + cx * LDP, r, two_h);
                    modal_grad_T_acc<T, K, 1>(P + cy * LDP, r, two_h);
                    modal_grad_T_acc<T, K, 2>(P + cz * LDP, r, two_h);
                    if constexpr (b % 4 == 0) {
                        T fa[b];
#pragma unroll
                        for (int l = 0; l < b; l += 4) ld4<T>(P + (6 + i) * LDP + l, fa + l);
#pragma unroll
                        for (int l = 0; l < b; ++l) r[l] += fa[l];
                    } else {
#pragma unroll
                        for (int l = 0; l < b; ++l) r[l] += P[(6 + i) * LDP + l];
                    }
                }
                if constexpr (DIFF) {
                    // -(eps/|K|) int grad phi_l . grad u = -eps (4/h^2) sum_d (D_d^T D_d u)_l
                    const T* uv = sU + c * 4 * b + v * b;
                    T t[b];
                    modal_grad<T, K, 0>(uv, t, T(1));
                    modal_grad_T_acc<T, K, 0>(t, r, diff_vol);
                    modal_grad<T, K, 1>(uv, t, T(1));
                    modal_grad_T_acc<T, K, 1>(t, r, diff_vol);
                    modal_grad<T, K, 2>(uv, t, T(1));
                    modal_grad_T_acc<T, K, 2>(t, r, diff_vol);
                }
                if constexpr (b % 4 == 0) {
#pragma unroll
                    for (int l = 0; l < b; l += 4) st4<T>(sR + (c * 4 + v) * b + l, r + l);
                } else {
#pragma unroll
                    for (int l = 0; l < b; ++l) sR[(c * 4 + v) * b + l] = r[l];
                }
            }
            // the face lifts below add to these rows from other threads
            __syncthreads();
            // ---- faces, one direction at a time (Sec. 3.2 face states, Rusanov) ----
            // per warp: collapsed rows and (later) the face fluxes in one block,
            // traces and (later) the lifted fluxes in another
            T* sC2 = sBig + C::oC2 + wid * RCW * LDC2;
            T* sTr = sBig + C::oTr + wid * RCW * LDT;
            T* sFs = sC2;
            T* sL2 = sTr;
            static_for<0, 3>([&](auto dd) {
                constexpr int Dd = decltype(dd)::value;
                // this direction's neighbour rows; start the next direction's loads
                T cur[NR][b];
#pragma unroll
                for (int j = 0; j < NR; ++j)
#pragma unroll
                    for (int l = 0; l < b; ++l) cur[j][l] = nbr[j][l];
                if constexpr (Dd < 2) load_nbr(std::integral_constant<int, Dd + 1>{});
                // collapse rows r = ((c*2 + side)*2 + who)*4 + field (warp-local rl)
#pragma unroll
                for (int j = 0; j < NR; ++j) {
                    const int rl = lane + 32 * j, r = wid * RCW + rl;
                    const int field = r & 3, who = (r >> 2) & 1, side = (r >> 3) & 1, c = r >> 4;
                    T cf[b];
                    int fside = side;
                    if (who == 0) {
                        const T* src = (field == 0) ? sU + c * 4 * b : sVH + (c * 3 + field - 1) * b;
                        if constexpr (b % 4 == 0) {
#pragma unroll
                            for (int l = 0; l < b; l += 4) ld4<T>(src + l, cf + l);
                        } else {
#pragma unroll
                            for (int l = 0; l < b; ++l) cf[l] = src[l];
                        }
                    } else {
                        fside = 1 - side;
#pragma unroll
                        for (int l = 0; l < b; ++l) cf[l] = cur[j][l];
                    }
                    T c2[B2K];
                    collapse<T, K, Dd, B2K>(cf, fside, c2);
                    static_assert(B2K % 4 == 0 && LDC2 % 4 == 0, "row vectors");
#pragma unroll
                    for (int p = 0; p < B2K; p += 4) st4<T>(sC2 + rl * LDC2 + p, c2 + p);
                }
                __syncwarp();
                mm<T, BK, RCW, NSP, B2K, LDC2, LDT, 32, true>(sC2, tabs, C::oPsi, sTr);
                __syncwarp();
                // Riemann flux at every face point; F* along +e_d with L = lower cell
                for (int e = lane; e < CPW * 2 * NSP; e += 32) {
                    const int s = e % NSP, side = (e / NSP) & 1, c = e / (2 * NSP);  // c: the warp's cell
                    T F[4] = {T(0), T(0), T(0), T(0)};
                    if (s < ns) {
                        const int rs = ((c * 2 + side) * 2 + 0) * 4, rn = ((c * 2 + side) * 2 + 1) * 4;
                        T Ws[4], Wn[4];
#pragma unroll
                        for (int f = 0; f < 4; ++f) {
                            Ws[f] = sTr[(rs + f) * LDT + s];
                            Wn[f] = sTr[(rn + f) * LDT + s];
                        }
                        if (side)
                            riemann_flux<T, Dd>(a.ph.riemann, cs, cs2, Ws, Wn, F);
                        else
                            riemann_flux<T, Dd>(a.ph.riemann, cs, cs2, Wn, Ws, F);
                    }
#pragma unroll
                    for (int v = 0; v < 4; ++v) sFs[((c * 2 + side) * 4 + v) * LDT + s] = F[v];
                }
                __syncwarp();
                mm<T, BK, RLW, B2N, NSP, LDT, LDL, 32, true>(sFs, tabs, C::oPsiL, sL2);
                __syncwarp();
                for (int e = lane; e < CPW * 4; e += 32) {
                    const int c = wid * CPW + e / 4, cl = e / 4, v = e % 4;
                    T* R = sR + (c * 4 + v) * b;
                    static_assert(LDL % 4 == 0 && B2N % 4 == 0, "row vectors");
                    T l1[B2N], l0[B2N];
#pragma unroll
                    for (int p = 0; p < B2N; p += 4) {
                        ld4<T>(sL2 + ((cl * 2 + 1) * 4 + v) * LDL + p, l1 + p);
                        ld4<T>(sL2 + ((cl * 2 + 0) * 4 + v) * LDL + p, l0 + p);
                    }
                    // + face (side 1): -1/(4h); - face (side 0): +1/(4h)
                    T rr[b];
                    if constexpr (b % 4 == 0) {
#pragma unroll
                        for (int l = 0; l < b; l += 4) ld4<T>(R + l, rr + l);
                    } else {
#pragma unroll
                        for (int l = 0; l < b; ++l) rr[l] = R[l];
                    }
                    expand_acc<T, K, Dd>(l1, 1, -inv4h, rr);
                    expand_acc<T, K, Dd>(l0, 0, inv4h, rr);
                    if constexpr (DIFF) {
                        if (c0 + c < a.ncell) {
                        // the variable's coefficient rows of both face neighbours
                        T um[b], up[b];
                        int xyz[3];
                        cell_xyz(c0 + c, a.N, xyz[0], xyz[1], xyz[2]);
                        const T* srcm = a.u_in + (neighbour_along<Dd>(c0 + c, xyz[Dd], 0, a.N) * 4 + v) * b;
                        const T* srcp = a.u_in + (neighbour_along<Dd>(c0 + c, xyz[Dd], 1, a.N) * 4 + v) * b;
                        if constexpr (b % 4 == 0) {
#pragma unroll
                            for (int l = 0; l < b; l += 4) {
                                ld4<T>(srcm + l, um + l);
                                ld4<T>(srcp + l, up + l);
                            }
                        } else {
#pragma unroll
                            for (int l = 0; l < b; ++l) {
                                um[l] = __ldg(srcm + l);
                                up[l] = __ldg(srcp + l);
                            }
                        }
                        diffusion_faces<T, K, Dd>(a.ph, sU + c * 4 * b + v * b, um, up, rr);
                        }
                    }
                    if constexpr (b % 4 == 0) {
#pragma unroll
                        for (int l = 0; l < b; l += 4) st4<T>(R + l, rr + l);
                    } else {
#pragma unroll
                        for (int l = 0; l < b; ++l) R[l] = rr[l];
                    }
                }
                // the next direction's collapse rewrites this warp's flux rows
                __syncwarp();
            });
            // ---- epilogue ----
            if constexpr (MODE == TM_RHS) {
                __syncthreads();
                for (int e = tid; e < TC * 4 * b; e += NT) {
                    if (e / (4 * b) < nvalid) a.out[c0 * 4 * b + e] = sR[e];
                }
                __syncthreads();
            } else {
                // SSP-RK stage combine (Sec. 7), new state kept in sU; u^n was prefetched.
                // Warp-local like the face phase: the warp's own cells, whose
                // right-hand-side rows it has just finished (no block barrier)
                const int e0 = wid * CPW * 4 * b;
                for (int el = lane; el < CPW * 4 * b; el += 32) {
                    const int e = e0 + el;
                    T w;
                    if (e / (4 * b) < nvalid) {
                        const T un = (a.rk_a != T(0)) ? sUn[e] : T(0);
                        w = a.rk_a * un + a.rk_b * (sU[e] + dt * sR[e]);
                    } else {
                        w = ((e % (4 * b)) == 0) ? T(1) : T(0);
                    }
                    sU[e] = w;
                }
                __syncwarp();
                // positivity (Sec. 3.1): a cell passes when rho_0 - sum_l |rho_l| sup|phi_l| >= eps;
                // otherwise rho is evaluated at every volume and face Gauss point (lanes
                // over modes for the bound, over points for the check; warp reductions)
                const T eps = T(a.ph.floor_);
                T thr[CPW];  // rescaling factor of the modes l > 0 per cell (1: none)
                unsigned int st = 0u;
#pragma unroll
                for (int cl = 0; cl < CPW; ++cl) {
                    const int c = wid * CPW + cl;
                    const T* r = sU + c * 4 * b;
                    T part = (lane >= 1 && lane < b) ? fabs(r[lane < b ? lane : 0]) * my_sup : T(0);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                    thr[cl] = T(1);
                    if (r[0] - part < eps) {
                        const T* phiv = a.tab + TT::phiv;
                        const T* phif = a.tab + TT::phif;
                        T mn = T(1e30);
                        for (int pt = lane; pt < nq + nf; pt += 32) {
                            T rho = T(0);
                            if (pt < nq) {
#pragma unroll
                                for (int l = 0; l < b; ++l) rho += r[l] * __ldg(phiv + l * nq + pt);
                            } else {
#pragma unroll
                                for (int l = 0; l < b; ++l) rho += r[l] * __ldg(phif + l * nf + (pt - nq));
                            }
                            mn = rho < mn ? rho : mn;
                        }
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            const T other = __shfl_xor_sync(0xffffffffu, mn, o);
                            mn = other < mn ? other : mn;
                        }
                        const T rbar = r[0];
                        if (a.trouble && mn < T(0)) {
                            if (lane == 0 && c0 + c < a.ncell) a.trouble[c0 + c] |= DG_MARK_NEGATIVE;
                            st |= DG_ST_TROUBLED_;
                        }
                        if (mn < eps) {
                            if (rbar > eps) {
                                thr[cl] = (rbar - eps) / (rbar - mn);
                                st |= DG_ST_LIMITED_;
                            } else if (!a.trouble || !(rbar > T(0))) {
                                // positivity by repetition: a mean in (0, eps] stands
                                st |= DG_ST_FAIL_;
                            }
                        }
                    }
                }
                // rescale, store u^(s+1), keep the limited state for the fused projection
                for (int el = lane; el < CPW * 4 * b; el += 32) {
                    const int e = e0 + el, cl = el / (4 * b), l = e % b;
                    T w = sU[e];
                    T th = T(1);
#pragma unroll
                    for (int j = 0; j < CPW; ++j)
                        if (j == cl) th = thr[j];
                    if (l > 0) w *= th;
                    sU[e] = w;
                    if (e / (4 * b) < nvalid) {
                        if (!isfinite(w)) st |= DG_ST_NONFINITE_;
                        a.out[c0 * 4 * b + e] = w;
                    }
                }
                st = __reduce_or_sync(0xffffffffu, st);
                if (lane == 0 && st) atomicOr(&s_status, st);
                if (do_proj && force) {
                    // per-cell forcing sums <rho a_h>, <rho> of the warp's cells (lane = (cell, i))
                    __syncwarp();
                    if (lane < CPW * 3) {
                        const int c = wid * CPW + lane / 3, i = lane % 3;
                        if (c < nvalid) {
                            const T* u = sU + c * 4 * b;
                            const T* ah = sAh + (c * 3 + i) * b;
                            T sacc = T(0);
#pragma unroll
                            for (int l = 0; l < b; ++l) sacc += u[l] * ah[l];
                            sums[i] += (double)sacc;
                            if (i == 0) sums[3] += (double)u[0];
                        }
                    }
                }
                // every warp is done with this tile's staging buffers: fetch the next
                // tile (the next iteration starts with a barrier after the projection)
                __syncthreads();
                if (tile + gridDim.x < ntile) issue(tile + gridDim.x, sR);
                if (do_proj) {
                    tile_project<T, K, BK, MODE == TM_STAGE_VABS>(sm, sU, tabs, a, c0, (a.flags & F_DT) != 0, smax,
                                                                 sums, false);
                    if constexpr (MODE == TM_STAGE_VABS) {
                        if (a.nu_next) tile_nu<T, K, BK>(sm, sU, a, c0);
                    }
                }
            }
        }
    }
    // ---- block-level reductions (their buffer is the big region) ----
    __syncthreads();
    if constexpr (STAGE) {
        if (tid == 0 && s_status) atomicOr(&a.ctl->status, s_status);
    }
    if constexpr (MODE != TM_PROJECT) {
        if (tid == 0 && ntiles > 0) {
            atomicAdd(&a.ctl->tiles_vol, (unsigned long long)ntiles);
            if (gated) atomicAdd(&a.ctl->tiles_gated, (unsigned long long)gated);
        }
    }
    if (do_proj) {
        if (a.flags & F_DT) {
            const double sp = (double)smax + 3.0 * a.ph.cs;
            atomicMax(&s_smax, (unsigned long long)__double_as_longlong(sp));
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
                const int o = a.abar_out;
                if (a.flags & F_FORCE) {
                    for (int i = 0; i < 3; ++i) a.ctl->abar2[o][i] = s_tot[i] / s_tot[3];
                } else {
                    a.ctl->abar2[o][0] = a.ctl->abar2[o][1] = a.ctl->abar2[o][2] = 0.0;
                }
                if (a.flags & F_DT) {
                    // every block of this launch has read ctl->sn before it arrived here
                    const unsigned long long bits = atomicAdd(&a.ctl->smax, 0ull);
                    a.ctl->sn = __longlong_as_double((long long)bits);
                    a.ctl->smax = 0ull;
                }
            }
        }
    }
}

}  // namespace dg
