// dg_tc5_kernels.cuh -- the x3 stage of degree 3 on the 5th-generation tensor
// cores (tcgen05, accumulators in TMEM), as three kernels per SSP-RK stage:
//
//   k5_volume   volume flux integral + driving source (Sec. 2.2, eq.
//               weight_evolution, first and last terms; Sec. 3.1 viscous
//               pressure at the volume points), written to rvol [c][4][b]
//   k5_faces    face states (Sec. 3.2: rho from its own expansion, v from the
//               projected velocity), Riemann fluxes, the surface integral, the
//               sum with rvol, then the SSP-RK combine and the positivity
//               rescaling (Sec. 3.1, Sec. 7) -- or the right-hand side alone
//   k5_project  projection of the primitive velocity (Sec. 3.2, eq.
//               weights_equation) of the new state, its |v| projection, the
//               CFL wave-speed bound and the forcing sums for the next stage
//
// Tiles of 16 consecutive cells.  Every basis <-> point transform is one
// tensor-core product per tile:
//   evaluation  D[(h,q)][(p,f)] = sum_l Phi[q][l] A[(2p+h, f)][l]      M = 128 = 2 x 64 points
//               (two products against the table padded with zero blocks, so
//               rows h = 0 / 1 take the even / odd cells: no dense block-
//               diagonal table is stored)
//   volume      R[(c,v)][l] = sum_{d,q} F_vd(q)/(4h) w_q dphi_l/dxi_d(q)
//                           + sum_q S_v(q) w_q/8 phi_l(q)                M = 64
//   face traces D[(F,s)][(c,fld)] = sum_l phi_l(xi_{F,s}) C[(c,fld)][l]   M = 128 = 6 faces x 16 points
//               (the neighbour across face F: the same table read through a
//               window shifted by one face, lanes of the other faces masked)
//   lift        R[(c,v)][l] += sum_{F,s} (-sigma_F w_s F*_v/(4h)) phi_l(xi_{F,s})
// With point-major accumulators a thread holds all fields of its volume or
// face point: the pointwise physics and the Riemann solver run in registers.
#pragma once

#include "dg_tc5.cuh"
#include "dg_tile.cuh"

namespace dg {

// sizes of the degree-3 tensor-core kernels (bytes unless noted)
struct C5 {
    static constexpr int K = 3, b = 20, n = 4, nq = 64, ns = 16, TC = 16, NT = 256;
    static constexpr int NEV = 96;   // N of the volume evaluation: 8 pairs x 12 rows
    static constexpr int NEP = 32;   // N of the projection's evaluation: 8 pairs x 4 rows
    // tables: Phi [64 q][32 l] K-major blocks (LBO 128, SBO 512), laid out
    // [Z, Phi_hi, Z, Phi_lo, Z]
    static constexpr int PHI_BLK = 4096;
    static constexpr int oPhi = 0, szPhi = 5 * PHI_BLK;
    // G_d [32 l][64 q] = w_q dphi_l/dxi_d(q), K-major (LBO 128, SBO 1024), [d][comp]
    static constexpr int G_BLK = 4096;
    static constexpr int oG = oPhi + szPhi, szG = 6 * G_BLK;
    // face table [160 rows][32 l] K-major (LBO 128, SBO 512), [comp]: 16 slack
    // rows, 96 face points (F, s) = 16 F + s, 32 zero rows, 16 slack rows
    static constexpr int F_ROWS = 160, F_BLK = F_ROWS / 8 * 512;
    static constexpr int oF = oG + szG, szF = 2 * F_BLK;
    static constexpr int oWq = oF + szF;       // [64] float: w_q (product of 1D weights, sum 8)
    static constexpr int oWs = oWq + 256;      // [16] float: w_s (sum 4)
    static constexpr int tab_bytes = oWs + 64;
    // TMEM columns per CTA
    static constexpr int TM_VOL = 128, TM_VOLP = 256, TM_FACE = 256, TM_PROJ = 64;
    // shared memory of the kernels
    struct Vol {  // tables Phi + G + w_q, the tile, the work region
        // the tile (u, a_h) double-buffered: the next tile's copy lands while this one runs
        static constexpr int oPhi = 0, oG = szPhi, oWq = oG + szG, oU = oWq + 256, oAh = oU + 2 * TC * 80 * 4;
        static constexpr int oW = oAh + 2 * TC * 60 * 4;
        static constexpr int EB = 12 * 512;                // evaluation B per (half, comp): 96 rows
        static constexpr int PA = 16 * 1024;               // volume A per comp: 64 rows x 2 slots x 64 q (MN-major)
        static constexpr int work = (4 * EB > 2 * PA) ? 4 * EB : 2 * PA;
        static constexpr int total = oW + work;
        // driven stages that project their input: the second round carries three
        // slots (flux along z, source, projection)
        static constexpr int PA3 = 24 * 1024;
        static constexpr int total3 = oW + ((4 * EB > 2 * PA3) ? 4 * EB : 2 * PA3);
    };
    struct Face {  // face table + w_s, self and neighbour operands (the lift operand reuses them), new state
        static constexpr int oF = 0, oWs = szF, oSelf = oWs + 64, SB = 8 * 512;  // [64 rows][32] per comp
        static constexpr int oNbr = oSelf + 2 * SB;        // [face][comp]
        static constexpr int LA = 12 * 1024;               // lift A per comp: 64 rows x 96 (MN-major)
        static constexpr int oNew = oNbr + 12 * SB;
        static constexpr int oEpi = (oNew + TC * 80 * 4 + 127) / 128 * 128;  // u^(s), u^n, rvol of the tile, fetched
                                                                        // asynchronously (128-byte aligned: TMA)
        static constexpr int total = oEpi + 3 * TC * 80 * 4;
        // the next tile's rows (self and six neighbours: rho 20, v 60 floats per
        // cell) land by asynchronous copies in the self and neighbour operand
        // region once its products are done; entries 84 floats apart (bank spread)
        static constexpr int RAWS = 84;
        static_assert(7 * TC * RAWS * 4 <= 14 * SB, "staging fits the operand region");
        static_assert(oSelf % 16 == 0 && (RAWS * 4) % 16 == 0, "16-byte copies");
    };
    // tiled TMA destinations are 128-byte aligned (the dynamic shared memory starts 1024-aligned)
    static_assert((Vol::oU % 128) == 0 && (Vol::oAh % 128) == 0 && ((TC * 80 * 4) % 128) == 0 &&
                      ((TC * 60 * 4) % 128) == 0 && (Face::oEpi % 128) == 0,
                  "TMA destinations");
    struct Proj {  // Phi + w_q, the tile, evaluation B, projection A
        static constexpr int oPhi = 0, oWq = szPhi, oU = oWq + 256, oAh = oU + 2 * TC * 80 * 4;  // u, a_h: double
        static constexpr int oEB = oAh + 2 * TC * 60 * 4, EB = 4 * 512;
        static constexpr int oPA = oEB + 4 * EB, PA = 8 * 1024;  // 64 rows x 64 q (MN-major)
        static constexpr int total = oPA + 2 * PA;
    };
    static_assert((Proj::oU % 128) == 0 && (Proj::oAh % 128) == 0, "TMA destinations");
};

#define DG_ST_TIMEOUT_ 8u

struct T5Args {
    const float* u_in;   // u^(s): state of the right-hand side / the state to project
    const float* u_n;    // u^n (stage combine)
    float* out;          // u^(s+1) or dudt
    const float* vh_in;  // projected velocity of u_in [c][3][b]
    float* vh_out;       // projection output [c][3][b]
    float* vabs_out;     // projection of |v| [c][b] or nullptr
    const float* ahat;   // forcing [c][3][b] or nullptr
    const float* nu;     // per-cell coefficient (learned sensor) or nullptr
    float* rvol;         // volume term [c][4][b]
    float* vh_self;      // projection of v of u_in [c][3][b] by the volume kernel (stages after the first)
    float* nu_next;      // projection kernel: learned coefficient of u_in [c] (or nullptr)
    const uint32_t* mlp; // packed network of the learned sensor
    int abar_fix;        // face kernel: subtract abar_in's mean acceleration times rho_l from the momentum
                         // right-hand side (the volume kernel's source left it out)
    int tmask;           // tiled TMA descriptors present: 1 u_in, 2 u_n, 4 rvol, 8 ahat
    CUtensorMap tu, tn, tr, ta;  // of u_in, u_n, rvol [c][80] and ahat [c][60]: boxes of 16 cells
    const unsigned char* tab;  // C5 table block
    const float* phiv;   // [b][nq] phi at the volume points (exact positivity check)
    const float* phif;   // [b][nf] phi at the face points
    Ctl* ctl;
    double* partials;
    long ncell;
    int N;
    Phys ph;
    float rk_a, rk_b;
    double dt_pimax;
    int flags;           // F_FORCE, F_DT
    int abar_in, abar_out;
    int stage;           // 1: the step's dt (stage), 0: dt_pimax (right-hand side)
    unsigned char* trouble;  // positivity by repetition: per-cell marks of the stage outputs (or nullptr)
};

namespace k5 {

// copy `bytes` (a multiple of 16) from global to shared
__device__ __forceinline__ void copy16(unsigned char* dst, const unsigned char* src, int bytes)
{
    for (int e = 16 * threadIdx.x; e < bytes; e += 16 * blockDim.x)
        *reinterpret_cast<uint4*>(dst + e) = __ldg(reinterpret_cast<const uint4*>(src + e));
}

// the step's dt (Sec. 7 CFL condition, fixed for all stages) or the given dt
__device__ __forceinline__ double step_dt(const T5Args& a)
{
    if (!a.stage) return a.dt_pimax;
    const double sn = a.ctl->sn;
    double dtc = a.ctl->dt_num / sn;
    if (a.ctl->dt_diff > 0.0 && a.ctl->dt_diff < dtc) dtc = a.ctl->dt_diff;
    return (a.ctl->fixed_dt > 0.0 ? a.ctl->fixed_dt : dtc) * a.ctl->dt_scale;
}

// stage a state tile [16][80] (cells past the end: rho = 1, the rest 0)
__device__ __forceinline__ void load_state(float* s, const float* g, long c0, int nvalid)
{
    for (int e = 4 * threadIdx.x; e < C5::TC * 80; e += 4 * blockDim.x) {
        float4 v;
        if (e / 80 < nvalid)
            v = __ldg(reinterpret_cast<const float4*>(g + c0 * 80 + e));
        else
            v = make_float4((e % 80) == 0 ? 1.f : 0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<float4*>(s + e) = v;
    }
}

// TMA bulk copy of the valid cells of a tile with `per` floats per cell,
// issued by the calling thread on mbarrier `bar` (which must expect the bytes);
// returns the bytes
__device__ __forceinline__ uint32_t bulk_tile(float* s, const float* g, long c0, int nvalid, int per, uint64_t* bar)
{
    const uint32_t bytes = (uint32_t)(nvalid * per * 4);
    tc5::bulk_g2s(s, g + c0 * per, bytes, bar);
    return bytes;
}
// the same for a full tile through a tiled TMA descriptor when there is one
// (the box of 16 cells at row c0), else the 1D bulk copy
__device__ __forceinline__ void tile_copy(float* s, const float* g, const CUtensorMap* map, bool use_map, long c0,
                                          int nvalid, int per, uint64_t* bar)
{
    if (use_map && nvalid == C5::TC)
        tc5::tma_2d(s, map, 0, (int)c0, bar);
    else
        bulk_tile(s, g, c0, nvalid, per, bar);
}
// the filler of the cells past the end (plain stores of all threads)
__device__ __forceinline__ void fill_tail(float* s, int nvalid, int per, float fill0)
{
    for (int e = nvalid * per + threadIdx.x; e < C5::TC * per; e += blockDim.x) s[e] = (e % per) == 0 ? fill0 : 0.f;
}

__device__ __forceinline__ int tile_cells(long ncell, long c0)
{
    return (int)((ncell - c0) < C5::TC ? (ncell - c0) : C5::TC);
}

// one K-major operand row of 20 modes (padded to 32): hi and lo components at
// base and base + cstride; row r of a [rows][32] operand (LBO 128, SBO 512)
__device__ __forceinline__ void put_row(unsigned char* base, int cstride, int r, const float* x20)
{
    float x[32];
#pragma unroll
    for (int l = 0; l < 20; ++l) x[l] = x20[l];
#pragma unroll
    for (int l = 20; l < 32; ++l) x[l] = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint4 hi, lo;
        tc5::split8(x + 8 * j, hi, lo);
        const int o = tc5::koff(r, 8 * j, 128, 512);
        *reinterpret_cast<uint4*>(base + o) = hi;
        *reinterpret_cast<uint4*>(base + cstride + o) = lo;
    }
}

// products of the split: (A component, B component)
__device__ __forceinline__ void prod(int pr, int& ca, int& cb)
{
    ca = (pr == 2) ? 1 : 0;
    cb = (pr == 1) ? 1 : 0;
}

// bounded wait for phase `parity` of an mbarrier, agreed over the block (a
// barrier): false when any thread gave up, which the status records
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, Ctl* ctl, int* s_abort)
{
    const bool ok = tc5::mbar_wait(bar, parity);
    const bool any_failed = __syncthreads_or(!ok) != 0;
    if (any_failed) {
        if (threadIdx.x == 0) {
            atomicOr(&ctl->status, DG_ST_TIMEOUT_);
            *s_abort = 1;
        }
        return false;
    }
    return true;
}

// the same for the block's product barrier, whose phase it advances
__device__ __forceinline__ bool wait_mma(uint64_t* bar, uint32_t& phase, Ctl* ctl, int* s_abort)
{
    const bool ok = tc5::mbar_wait(bar, phase);
    phase ^= 1u;
    const bool any_failed = __syncthreads_or(!ok) != 0;
    if (any_failed) {
        if (threadIdx.x == 0) {
            atomicOr(&ctl->status, DG_ST_TIMEOUT_);
            *s_abort = 1;
        }
        return false;
    }
    tc5::fence_after();
    return true;
}

}  // namespace k5

// --------------------------------------------------------------------------
// volume term + driving source -> rvol
// --------------------------------------------------------------------------
// FORCE: the driving source is added (a_h rows, source slot); GATE: the
// coefficients may vanish on whole tiles (learned sensor, or no viscosity), so
// that div v is evaluated only where a cell of the tile needs it; PROJ: a slot of
// the second round projects v = m/rho of the tile's state onto the basis (Sec.
// 3.2, the primitive projection the face kernel then reads) into an accumulator
// of its own -- the projection launch between stages drops.  Undriven, that slot
// is the source's; driven, a third slot of the round, and the source leaves out
// the mean acceleration (which depends on the whole state): the kernel reduces
// <rho a_h>/<rho> into the abar_out slot and the face kernel subtracts abar rho_l
template <bool FORCE, bool GATE, bool PROJ, bool CHK = false>
__global__ void __launch_bounds__(256, 2) k5_volume(const __grid_constant__ T5Args a)
{
    static_assert(PROJ || !CHK, "the wave-speed marks come with the self-projection");
    constexpr bool P3 = FORCE && PROJ;  // three slots in the second round
    constexpr int TMC = PROJ ? C5::TM_VOLP : C5::TM_VOL;
    using V = C5::Vol;
    constexpr int TC = C5::TC;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(8) uint64_t lbar[2];  // tile copies into buffer 0 / 1
    __shared__ uint32_t tslot;
    __shared__ float s_nu[TC];
    __shared__ int s_abort;
    __shared__ double s_tot[8];
    constexpr int PAX = P3 ? V::PA3 : V::PA;  // bytes per split component of the round operand
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    k5::copy16(sm + V::oPhi, a.tab + C5::oPhi, C5::szPhi + C5::szG);
    if (tid < 64) reinterpret_cast<float*>(sm + V::oWq)[tid] = reinterpret_cast<const float*>(a.tab + C5::oWq)[tid];
    float* const sUb = reinterpret_cast<float*>(sm + V::oU);
    float* const sAhb = reinterpret_cast<float*>(sm + V::oAh);
    const float* sWq = reinterpret_cast<const float*>(sm + V::oWq);
    unsigned char* sW = sm + V::oW;
    if (w == 0) tc5::tmem_alloc(&tslot, TMC);
    if (tid == 0) {
        tc5::mbar_init(&bar, 1);
        tc5::mbar_init(&lbar[0], 1);
        tc5::mbar_init(&lbar[1], 1);
        s_abort = 0;
    }
    tc5::fence_async_smem();
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    const uint32_t tm = tslot;
    uint32_t phase = 0;
    constexpr bool force = FORCE;
    const double dtd = k5::step_dt(a);
    const AvCoef<float> avc = av_coef<float>(a.ph, dtd);
    const float two_h = (float)(2.0 / a.ph.h), i4h = (float)(0.25 / a.ph.h), cs2 = (float)a.ph.cs2;
    // positivity by repetition: the input of a self-projecting stage is the previous
    // stage's output; a point with sum_d |v_d| above this bound marks its cell
    constexpr bool chk = CHK;
    const float vlim = chk ? (float)(DG_REPEAT_SPEED * a.ctl->sn - 3.0 * a.ph.cs) : 0.f;
    float ab[3] = {0.f, 0.f, 0.f};
    if (force && !P3)
        for (int i = 0; i < 3; ++i) ab[i] = (float)a.ctl->abar2[a.abar_in][i];
    double sums[4] = {0.0, 0.0, 0.0, 0.0};  // P3: <rho a_h> (3) and <rho> of the thread's (cell, component)
    // point-major thread: TMEM lane r = 32 (w % 4) + lane = (h, q); pairs p = 4 (w / 4) + 0..3
    const int qw = w & 3, hp = w >> 2, r = 32 * qw + lane, h = r >> 6, q = r & 63;
    const uint32_t tl = tc5::tmem_addr(tm, 32 * qw, 0);
    const long ntile = (a.ncell + TC - 1) / TC;
    // TMA bulk copies of a tile's u (and a_h) into buffer buf, completing on lbar[buf];
    // the cells past the end get the filler from plain stores of all threads
    auto fetch = [&](long t, int buf) {
        const long cb = t * TC;
        const int nv = k5::tile_cells(a.ncell, cb);
        float* su = sUb + buf * TC * 80;
        float* sa = sAhb + buf * TC * 60;
        k5::fill_tail(su, nv, 80, 1.f);
        if (force) k5::fill_tail(sa, nv, 60, 0.f);
        if (tid == 0) {
            tc5::fence_async_smem();
            tc5::mbar_expect_tx(&lbar[buf], (uint32_t)(nv * 80 * 4 + (force ? nv * 60 * 4 : 0)));
            k5::tile_copy(su, a.u_in, &a.tu, a.tmask & 1, cb, nv, 80, &lbar[buf]);
            if (force) k5::tile_copy(sa, a.ahat, &a.ta, a.tmask & 8, cb, nv, 60, &lbar[buf]);
        }
    };
    if (blockIdx.x < ntile) fetch(blockIdx.x, 0);
    int cur = 0;
    uint32_t lph = 0;                                   // bit b: phase of lbar[b]
    uint32_t inflight = blockIdx.x < ntile ? 1u : 0u;   // bit b: copies into buffer b not waited for
    uint32_t ntiles = 0, gated = 0;                     // tiles done, and those without div v
    for (long tile = blockIdx.x; tile < ntile; tile += gridDim.x, cur ^= 1) {
        const long c0 = tile * TC;
        const int nvalid = k5::tile_cells(a.ncell, c0);
        if (tid < TC) s_nu[tid] = (a.ph.av_mode == 2 && tid < nvalid) ? a.nu[c0 + tid] : 0.f;
        if (!k5::wait_bar(&lbar[cur], (lph >> cur) & 1u, a.ctl, &s_abort)) break;
        lph ^= 1u << cur;
        inflight &= ~(1u << cur);
        // the other buffer was consumed by the previous tile: fetch the next one into it
        if (tile + gridDim.x < ntile) {
            fetch(tile + gridDim.x, cur ^ 1);
            inflight |= 1u << (cur ^ 1);
        }
        ++ntiles;
        if (P3 && tid < TC * 3) {
            // per-cell forcing sums <rho a_h> = sum_l rho_l a_l (orthonormal basis) and <rho>
            const int c = tid / 3, i = tid % 3;
            if (c < k5::tile_cells(a.ncell, tile * TC)) {
                const float* u = sUb + cur * TC * 80 + c * 80;
                const float* ah = sAhb + cur * TC * 60 + c * 60 + i * 20;
                float sacc = 0.f;
#pragma unroll
                for (int l = 0; l < 20; ++l) sacc += u[l] * ah[l];
                sums[i] += (double)sacc;
                if (i == 0) sums[3] += (double)u[0];
            }
        }
        const float* sU = sUb + cur * TC * 80;
        const float* sAh = sAhb + cur * TC * 60;
        // the divergence rows and the viscous pressure are needed unless every
        // cell of the tile has a zero coefficient (learned sensor gated off, or
        // no viscosity): a tile-uniform decision
        bool need_div = !GATE;
        if (GATE && a.ph.av_mode == 2)
            for (int c = 0; c < TC; ++c) need_div |= s_nu[c] != 0.f;
        gated += need_div ? 0u : 1u;
        // ---- evaluation operand: three blocks of 32 rows 32 j + 4 p + f' for the
        // pair p = (cells 2p, 2p+1; half h = cell parity): j = 0 rho, m (3);
        // j = 1 D_d rho (3), sum_d D_d m_d (needed for div v only); j = 2 a_h (3),
        // 0 (driven steps only).  Field-major threads f = 4 j + f' ----
        if (tid < TC * 12) {
            const int f = tid >> 4, c = tid & 15, j = f >> 2;
            if (j == 0 || (j == 1 && need_div) || (j == 2 && force)) {
                const float* u = sU + c * 80;
                float x[20];
                if (f < 4) {
#pragma unroll
                    for (int l = 0; l < 20; ++l) x[l] = u[f * 20 + l];
                } else if (f == 4) {
                    modal_grad<float, 3, 0>(u, x, 1.f);
                } else if (f == 5) {
                    modal_grad<float, 3, 1>(u, x, 1.f);
                } else if (f == 6) {
                    modal_grad<float, 3, 2>(u, x, 1.f);
                } else if (f == 7) {
                    float t[20];
                    modal_grad<float, 3, 0>(u + 20, x, 1.f);
                    modal_grad<float, 3, 1>(u + 40, t, 1.f);
#pragma unroll
                    for (int l = 0; l < 20; ++l) x[l] += t[l];
                    modal_grad<float, 3, 2>(u + 60, t, 1.f);
#pragma unroll
                    for (int l = 0; l < 20; ++l) x[l] += t[l];
                } else if (f < 11) {
#pragma unroll
                    for (int l = 0; l < 20; ++l) x[l] = sAh[c * 60 + (f - 8) * 20 + l];
                } else {
#pragma unroll
                    for (int l = 0; l < 20; ++l) x[l] = 0.f;
                }
                k5::put_row(sW + (c & 1) * 2 * V::EB, V::EB, 32 * j + 4 * (c >> 1) + (f & 3), x);
            }
        }
        tc5::fence_async_smem();
        tc5::fence_before();
        __syncthreads();
        if (tid == 0) {
            tc5::fence_after();
            const uint64_t dphi = tc5::sdesc(tc5::saddr(sm + V::oPhi), 128, 512);
            const uint64_t deb = tc5::sdesc(tc5::saddr(sW), 128, 512);
            // blocks j0 .. j0 + nj - 1 into TMEM columns 32 j0 ..
            auto eval = [&](int j0, int nj) {
                const uint32_t ID = tc5::idesc_bf16(128, 32 * nj, 0, 0);
#pragma unroll
                for (int hh = 0; hh < 2; ++hh)
#pragma unroll
                    for (int pr = 0; pr < 3; ++pr) {
                        int ca, cb;
                        k5::prod(pr, ca, cb);
                        const uint32_t ao = (hh == 0 ? 1 + 2 * ca : 2 * ca) * C5::PHI_BLK;
                        const uint32_t bo = (hh * 2 + cb) * V::EB + j0 * 2048;
#pragma unroll
                        for (int ks = 0; ks < 2; ++ks)
                            tc5::mma(tm + 32 * j0, tc5::dadd(dphi, ao + ks * 256), tc5::dadd(deb, bo + ks * 256), ID,
                                     hh + pr + ks > 0);
                    }
            };
            if (need_div) {
                eval(0, force ? 3 : 2);
            } else {
                eval(0, 1);
                if (force) eval(2, 1);
            }
            tc5::commit(&bar);
        }
        __syncwarp();
        if (!k5::wait_mma(&bar, phase, a.ctl, &s_abort)) break;
        // ---- pointwise volume physics (Sec. 3.1: Pi at the volume points) ----
        float st[4][11];  // rho, m (3), v (3), P, source (3) of the thread's 4 (cell, point) items
        const float wq8 = sWq[q] * 0.125f;
        {
            float ev[4][12];
#pragma unroll
            for (int pp = 0; pp < 4; ++pp) {
                const int p = 4 * hp + pp;
                // columns of blocks that were not evaluated are read too (and not used)
                tc5::ld4(tl + 4 * p, ev[pp]);
                tc5::ld4(tl + 32 + 4 * p, ev[pp] + 4);
                tc5::ld4(tl + 64 + 4 * p, ev[pp] + 8);
            }
            tc5::ld_wait();
#pragma unroll
            for (int pp = 0; pp < 4; ++pp) {
                const int c = 2 * (4 * hp + pp) + h;
                const float* v = ev[pp];
                const float rho = v[0], ir = rcp<float>(rho);
                const float vx = v[1] * ir, vy = v[2] * ir, vz = v[3] * ir;
                const float divv = (v[7] * two_h - (vx * v[4] + vy * v[5] + vz * v[6]) * two_h) * ir;
                if (chk && c < nvalid && fabsf(vx) + fabsf(vy) + fabsf(vz) > vlim) {
                    a.trouble[c0 + c] |= DG_MARK_FAST;
                    atomicOr(&a.ctl->status, DG_ST_TROUBLED_);
                }
                float Pi = 0.f;
                if (need_div) {
                    if (a.ph.av_mode == 1)
                        Pi = vnr_pressure<float>(avc, rho, divv);
                    else
                        Pi = nu_pressure<float>(avc, rho, divv, s_nu[c]);
                }
                float* s = st[pp];
                s[0] = rho;
                s[1] = v[1];
                s[2] = v[2];
                s[3] = v[3];
                s[4] = vx;
                s[5] = vy;
                s[6] = vz;
                s[7] = cs2 * rho + Pi;
                s[8] = force ? rho * (v[8] - ab[0]) * wq8 : 0.f;
                s[9] = force ? rho * (v[9] - ab[1]) * wq8 : 0.f;
                s[10] = force ? rho * (v[10] - ab[2]) * wq8 : 0.f;
            }
        }
        tc5::fence_before();
        // ---- volume operand, two slots per round (slot d < 3: flux along d /(4h);
        // slot 3: source w_q/8), rows m = 32 h + 4 p + v, MN-major ----
        // slot kinds: 0 flux along d, 1 source, 2 projection of v, -1 none
        auto kind = [](int d) { return d < 3 ? 0 : d == 3 ? (FORCE ? 1 : (PROJ ? 2 : -1)) : (P3 ? 2 : -1); };
        auto volume_round = [&](auto R_) -> bool {
            constexpr int rnd = decltype(R_)::value;
            constexpr int NSL = (rnd == 1 && P3) ? 3 : 2;
#pragma unroll
            for (int sl = 0; sl < NSL; ++sl) {
                const int d = 2 * rnd + sl, k = 64 * sl + q, kd = kind(d);
                if (kd < 0) break;  // no source without driving
#pragma unroll
                for (int pp = 0; pp < 4; pp += 2) {
                    float x[8];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const float* s = st[pp + e];
                        float* y = x + 4 * e;
                        if (kd == 0) {
                            const float vd = s[4 + d];
                            y[0] = s[1 + d] * i4h;
                            y[1] = (s[1] * vd + (d == 0 ? s[7] : 0.f)) * i4h;
                            y[2] = (s[2] * vd + (d == 1 ? s[7] : 0.f)) * i4h;
                            y[3] = (s[3] * vd + (d == 2 ? s[7] : 0.f)) * i4h;
                        } else if (kd == 2) {
                            // rows i = v_x, v_y, v_z, (none) weighted by w_q/8
                            y[0] = s[4] * wq8;
                            y[1] = s[5] * wq8;
                            y[2] = s[6] * wq8;
                            y[3] = 0.f;
                        } else {
                            y[0] = 0.f;
                            y[1] = s[8];
                            y[2] = s[9];
                            y[3] = s[10];
                        }
                    }
                    uint4 hi, lo;
                    tc5::split8(x, hi, lo);
                    const int p = 4 * hp + pp;
                    const int o = (4 * h + (p >> 1)) * 128 + (k >> 3) * 1024 + (k & 7) * 16;
                    *reinterpret_cast<uint4*>(sW + o) = hi;
                    *reinterpret_cast<uint4*>(sW + PAX + o) = lo;
                }
            }
            tc5::fence_async_smem();
            tc5::fence_before();
            __syncthreads();
            if (tid == 0) {
                tc5::fence_after();
                constexpr uint32_t IDG = tc5::idesc_bf16(64, 32, 1, 0), IDS = tc5::idesc_bf16(64, 32, 1, 1);
                const uint64_t dw = tc5::sdesc(tc5::saddr(sW), 1024, 128);
                const uint64_t dg = tc5::sdesc(tc5::saddr(sm + V::oG), 128, 1024);
                const uint64_t dpm = tc5::sdesc(tc5::saddr(sm + V::oPhi), 512, 128);
#pragma unroll
                for (int sl = 0; sl < NSL; ++sl) {
                    const int d = 2 * rnd + sl, kd = kind(d);
                    if (kd < 0) break;
#pragma unroll
                    for (int pr = 0; pr < 3; ++pr) {
                        int ca, cb;
                        k5::prod(pr, ca, cb);
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint64_t ad = tc5::dadd(dw, ca * PAX + (8 * sl + 2 * ks) * 1024);
                            const bool acc = !(rnd == 0 && sl == 0 && pr == 0 && ks == 0);
                            if (kd == 0)
                                tc5::mma(tm + 96, ad, tc5::dadd(dg, (d * 2 + cb) * C5::G_BLK + ks * 256), IDG, acc);
                            else
                                tc5::mma(kd == 2 ? tm + 128 : tm + 96, ad,
                                         tc5::dadd(dpm, (1 + 2 * cb) * C5::PHI_BLK + ks * 1024), IDS,
                                         kd == 2 ? (pr + ks > 0) : acc);
                        }
                    }
                }
                tc5::commit(&bar);
            }
            __syncwarp();
            return k5::wait_mma(&bar, phase, a.ctl, &s_abort);
        };
        bool ok = volume_round(std::integral_constant<int, 0>{});
        if (ok) ok = volume_round(std::integral_constant<int, 1>{});
        if (!ok) break;
        // ---- rvol: rows m = 16 w + j (j < 16) of the M = 64 accumulator (warps
        // 0-3); the projection of v from its own accumulator (warps 4-7) ----
        if (PROJ && w >= 4) {
            float R[20];
            tc5::ld16(tl + 128, R);
            tc5::ld4(tl + 144, R + 16);
            tc5::ld_wait();
            if (lane < 16) {
                const int m = 16 * (w - 4) + lane, c = 2 * ((m & 31) >> 2) + (m >> 5), i = m & 3;
                if (i < 3 && c < nvalid) {
                    float4* dst = reinterpret_cast<float4*>(a.vh_self + (c0 + c) * 60 + i * 20);
#pragma unroll
                    for (int j = 0; j < 5; ++j) dst[j] = make_float4(R[4 * j], R[4 * j + 1], R[4 * j + 2], R[4 * j + 3]);
                }
            }
        }
        if (w < 4) {
            float R[20];
            tc5::ld16(tl + 96, R);
            tc5::ld4(tl + 112, R + 16);
            tc5::ld_wait();
            if (lane < 16) {
                const int m = 16 * w + lane, c = 2 * ((m & 31) >> 2) + (m >> 5), v = m & 3;
                if (c < nvalid) {
                    float4* dst = reinterpret_cast<float4*>(a.rvol + (c0 + c) * 80 + v * 20);
#pragma unroll
                    for (int j = 0; j < 5; ++j) dst[j] = make_float4(R[4 * j], R[4 * j + 1], R[4 * j + 2], R[4 * j + 3]);
                }
            }
        }
        tc5::fence_before();
        __syncthreads();
        tc5::fence_after();
    }
    // a loop left early: no bulk copy may still write into this block's shared memory
    if (tid == 0)
        for (int bb = 0; bb < 2; ++bb)
            if ((inflight >> bb) & 1u) tc5::mbar_wait(&lbar[bb], (lph >> bb) & 1u);
    if (tid == 0 && ntiles > 0) {
        atomicAdd(&a.ctl->tiles_vol, (unsigned long long)ntiles);
        if (gated) atomicAdd(&a.ctl->tiles_gated, (unsigned long long)gated);
    }
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    if (w == 0) tc5::tmem_dealloc(tm, TMC);
    if constexpr (P3) {
        // mean acceleration <rho a_h>/<rho> of this state into the abar_out slot (the
        // face kernel of the stage subtracts it); the work region is free now
        double* s_buf = reinterpret_cast<double*>(sW);
        double mine[4];
        for (int i = 0; i < 4; ++i) {
            s_buf[tid] = sums[i];
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int j = 0; j < C5::NT; ++j) t += s_buf[j];
                mine[i] = t;
            }
            __syncthreads();
        }
        if (last_block_reduce<C5::NT>(a.partials, mine, 4, &a.ctl->cnt_proj, s_tot, s_buf))
            if (tid == 0)
                for (int i = 0; i < 3; ++i) a.ctl->abar2[a.abar_out][i] = s_tot[i] / s_tot[3];
    }
}

// --------------------------------------------------------------------------
// faces: traces, Riemann fluxes, lift; + rvol; stage combine and positivity
// --------------------------------------------------------------------------
// RS: the face flux (0 Rusanov, 1 HLL, 2 HLLC), one instantiation each
template <int RS>
__global__ void __launch_bounds__(256, 2) k5_faces(const __grid_constant__ T5Args a)
{
    using Fc = C5::Face;
    constexpr int TC = C5::TC, b = C5::b, nq = C5::nq, nf = 96;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(8) uint64_t ebar;  // the epilogue's inputs
    __shared__ int s_nb[7 * C5::TC];
    __shared__ uint32_t tslot;
    __shared__ int s_abort;
    __shared__ unsigned int s_status;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    k5::copy16(sm + Fc::oF, a.tab + C5::oF, C5::szF);
    if (tid < 16) reinterpret_cast<float*>(sm + Fc::oWs)[tid] = reinterpret_cast<const float*>(a.tab + C5::oWs)[tid];
    unsigned char* sSelf = sm + Fc::oSelf;
    unsigned char* sNbr = sm + Fc::oNbr;
    float* sNew = reinterpret_cast<float*>(sm + Fc::oNew);
    float* const sEpi = reinterpret_cast<float*>(sm + Fc::oEpi);  // u^(s) | u^n | rvol
    const float* sWs = reinterpret_cast<const float*>(sm + Fc::oWs);
    if (w == 0) tc5::tmem_alloc(&tslot, C5::TM_FACE);
    if (tid == 0) {
        tc5::mbar_init(&bar, 1);
        tc5::mbar_init(&ebar, 1);
        s_abort = 0;
        s_status = 0u;
    }
    tc5::fence_async_smem();
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    const uint32_t tm = tslot;
    uint32_t phase = 0;
    const double dtd = k5::step_dt(a);
    if (a.stage && blockIdx.x == 0 && tid == 0) a.ctl->dt = dtd;
    const float dt = (float)dtd, i4h = (float)(0.25 / a.ph.h), cs = (float)a.ph.cs, cs2 = (float)a.ph.cs2;
    const float eps = (float)a.ph.floor_;
    float my_sup = 0.f;
    static_for<0, b>([&](auto m) {
        if (lane == decltype(m)::value) my_sup = (float)sup_phi<3>(decltype(m)::value);
    });
    const int qw = w & 3, hw = w >> 2;
    const uint32_t tl = tc5::tmem_addr(tm, 32 * qw, 0);
    const long ntile = (a.ncell + TC - 1) / TC;
    const bool need_un = a.stage && a.rk_a != 0.f;
    float abar_fix[3] = {0.f, 0.f, 0.f};
    if (a.abar_fix)
        for (int i = 0; i < 3; ++i) abar_fix[i] = (float)a.ctl->abar2[a.abar_in][i];
    uint32_t eph = 0;
    bool epi_pending = false;  // the epilogue's copies issued and not waited for
    // neighbour cells of the tile's cells: s_nb[16 fi + c] (fi = 0: the cell, fi = F + 1:
    // across face F), computed for the next tile by warps 4-7 during the epilogue
    auto neighbours = [&](long t, int i) {
        const long cb = t * TC;
        const int fi = i >> 4, c = i & 15;
        const long cc = cb + c;
        long sc = cc < a.ncell ? cc : 0;  // cells past the end: not read
        if (fi > 0 && cc < a.ncell) {
            const int F = fi - 1;
            int xyz[3];
            cell_xyz(cc, a.N, xyz[0], xyz[1], xyz[2]);
            const int d = F >> 1, co = xyz[d];
            const long stp = d == 0 ? 1L : (d == 1 ? (long)a.N : (long)a.N * a.N);
            sc = (F & 1) ? (co == a.N - 1 ? cc - (long)(a.N - 1) * stp : cc + stp)
                         : (co == 0 ? cc + (long)(a.N - 1) * stp : cc - stp);
        }
        s_nb[i] = (int)sc;
    };
    if (blockIdx.x < ntile && tid < 7 * TC) neighbours(blockIdx.x, tid);
    // the K padding (modes 20-31) of the self and neighbour operands is never
    // written by the gathers: zero once (the lift operand that later shares the
    // region leaves finite values there, and the table's padding is zero)
    for (int e = 16 * tid; e < 14 * Fc::SB; e += 16 * C5::NT) *reinterpret_cast<uint4*>(sSelf + e) = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    for (long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const long c0 = tile * TC;
        const int nvalid = k5::tile_cells(a.ncell, c0);
        // the epilogue's inputs (TMA bulk copies) arrive while the faces are computed
        k5::fill_tail(sEpi, nvalid, 80, 1.f);
        if (need_un) k5::fill_tail(sEpi + TC * 80, nvalid, 80, 1.f);
        k5::fill_tail(sEpi + 2 * TC * 80, nvalid, 80, 0.f);
        if (tid == 0) {
            tc5::fence_async_smem();
            tc5::mbar_expect_tx(&ebar, (uint32_t)(nvalid * 80 * 4 * (need_un ? 3 : 2)));
            k5::tile_copy(sEpi, a.u_in, &a.tu, a.tmask & 1, c0, nvalid, 80, &ebar);
            if (need_un) k5::tile_copy(sEpi + TC * 80, a.u_n, &a.tn, a.tmask & 2, c0, nvalid, 80, &ebar);
            k5::tile_copy(sEpi + 2 * TC * 80, a.rvol, &a.tr, a.tmask & 4, c0, nvalid, 80, &ebar);
        }
        epi_pending = true;
        // ---- operands: rows 4 c + fld (rho, v_x, v_y, v_z) of each cell (self) and
        // of its neighbour across each face F.  Coalesced: consecutive threads take
        // consecutive 16-byte chunks of a (cell, face) pair's 20 (rho 5, v 15), all
        // loads in flight before the split ----
        {
            constexpr int NCH = 7 * TC * 20, PER = (NCH + C5::NT - 1) / C5::NT;
            float4 raw[PER];
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int g = tid + i * C5::NT, pi = g / 20, ch = g - 20 * (g / 20), c = pi & 15;
                raw[i] = make_float4(ch == 0 ? 1.f : 0.f, 0.f, 0.f, 0.f);  // past the end: rho = 1, v = 0
                if (g < NCH && c < nvalid) {
                    const long sc = s_nb[pi];
                    const float* src = ch < 5 ? a.u_in + sc * 80 + 4 * ch : a.vh_in + sc * 60 + 4 * (ch - 5);
                    raw[i] = __ldg(reinterpret_cast<const float4*>(src));
                }
            }
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int g = tid + i * C5::NT, pi = g / 20, ch = g - 20 * (g / 20);
                if (g < NCH) {
                    const int fi = pi >> 4, c = pi & 15, fld = ch < 5 ? 0 : 1 + (ch - 5) / 5;
                    const int k = 4 * (ch < 5 ? ch : (ch - 5) % 5);
                    const float x[4] = {raw[i].x, raw[i].y, raw[i].z, raw[i].w};
                    uint2 hi, lo;
                    tc5::split4(x, hi, lo);
                    unsigned char* base = fi == 0 ? sSelf : sNbr + 2 * (fi - 1) * Fc::SB;
                    const int o = tc5::koff(4 * c + fld, k, 128, 512);
                    *reinterpret_cast<uint2*>(base + o) = hi;
                    *reinterpret_cast<uint2*>(base + Fc::SB + o) = lo;
                }
            }
        }
        tc5::fence_async_smem();
        tc5::fence_before();
        __syncthreads();
        if (tid == 0) {
            tc5::fence_after();
            constexpr uint32_t ID = tc5::idesc_bf16(128, 64, 0, 0);
            const uint64_t df = tc5::sdesc(tc5::saddr(sm + Fc::oF), 128, 512);
            const uint64_t ds = tc5::sdesc(tc5::saddr(sSelf), 128, 512);
            const uint64_t dn = tc5::sdesc(tc5::saddr(sNbr), 128, 512);
            // self traces on all six faces (table rows from 16)
#pragma unroll
            for (int pr = 0; pr < 3; ++pr) {
                int ca, cb;
                k5::prod(pr, ca, cb);
#pragma unroll
                for (int ks = 0; ks < 2; ++ks)
                    tc5::mma(tm, tc5::dadd(df, ca * C5::F_BLK + 2 * 512 + ks * 256), tc5::dadd(ds, cb * Fc::SB + ks * 256),
                             ID, pr + ks > 0);
            }
            // neighbour across F: its trace on the opposite face, into the lanes of F
#pragma unroll
            for (int F = 0; F < 6; ++F) {
                const int row0 = (F & 1) ? 0 : 32;  // 16 + 16 (opp(F) - F)
                const uint32_t m0 = F >> 1 == 0 ? ((F & 1) ? 0x0000FFFFu : 0xFFFF0000u) : 0xFFFFFFFFu;
                const uint32_t m1 = F >> 1 == 1 ? ((F & 1) ? 0x0000FFFFu : 0xFFFF0000u) : 0xFFFFFFFFu;
                const uint32_t m2 = F >> 1 == 2 ? ((F & 1) ? 0x0000FFFFu : 0xFFFF0000u) : 0xFFFFFFFFu;
#pragma unroll
                for (int pr = 0; pr < 3; ++pr) {
                    int ca, cb;
                    k5::prod(pr, ca, cb);
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks)
                        tc5::mma_masked(tm + 64, tc5::dadd(df, ca * C5::F_BLK + (row0 / 8) * 512 + ks * 256),
                                        tc5::dadd(dn, (2 * F + cb) * Fc::SB + ks * 256), ID, pr + ks > 0, m0, m1, m2,
                                        0xFFFFFFFFu);
                }
            }
            tc5::commit(&bar);
        }
        __syncwarp();
        if (!k5::wait_mma(&bar, phase, a.ctl, &s_abort)) break;
        // ---- Riemann fluxes at the face points: lane (F, s), F = 2 (w % 4) + lane/16;
        // warps w and w + 4 take cells 0-7 / 8-15.  F* along +e_d, L = lower cell ----
        if (qw < 3) {
            float ws[32], wn[32];
            tc5::ld16(tl + 32 * hw, ws);
            tc5::ld16(tl + 32 * hw + 16, ws + 16);
            tc5::ld16(tl + 64 + 32 * hw, wn);
            tc5::ld16(tl + 64 + 32 * hw + 16, wn + 16);
            tc5::ld_wait();
            const int r = 32 * qw + lane, side = (r >> 4) & 1, s = r & 15;
            const float scale = (side ? -1.f : 1.f) * sWs[s] * i4h;
            float x[32];
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
                const float* S = ws + 4 * cc;
                const float* Nb = wn + 4 * cc;
                float Fl[4];
                const float* L = side ? S : Nb;
                const float* Rr = side ? Nb : S;
                if (qw == 0)
                    riemann_flux<float, 0>(RS, cs, cs2, L, Rr, Fl);
                else if (qw == 1)
                    riemann_flux<float, 1>(RS, cs, cs2, L, Rr, Fl);
                else
                    riemann_flux<float, 2>(RS, cs, cs2, L, Rr, Fl);
#pragma unroll
                for (int v = 0; v < 4; ++v) x[4 * cc + v] = scale * Fl[v];
            }
            tc5::fence_before();
            __syncwarp();
            // lift operand (reuses the neighbour rows): rows m = 4 c + v, K = r, MN-major
#pragma unroll
            for (int cc = 0; cc < 8; cc += 2) {
                uint4 hi, lo;
                tc5::split8(x + 4 * cc, hi, lo);
                const int o = ((8 * hw + cc) >> 1) * 128 + (r >> 3) * 1024 + (r & 7) * 16;
                *reinterpret_cast<uint4*>(sNbr + o) = hi;
                *reinterpret_cast<uint4*>(sNbr + Fc::LA + o) = lo;
            }
        }
        tc5::fence_async_smem();
        tc5::fence_before();
        __syncthreads();
        if (tid == 0) {
            tc5::fence_after();
            constexpr uint32_t ID = tc5::idesc_bf16(64, 32, 1, 1);
            const uint64_t dl = tc5::sdesc(tc5::saddr(sNbr), 1024, 128);
            const uint64_t dfm = tc5::sdesc(tc5::saddr(sm + Fc::oF), 512, 128);
#pragma unroll
            for (int pr = 0; pr < 3; ++pr) {
                int ca, cb;
                k5::prod(pr, ca, cb);
#pragma unroll
                for (int ks = 0; ks < 6; ++ks)
                    tc5::mma(tm + 128, tc5::dadd(dl, ca * Fc::LA + 2 * ks * 1024),
                             tc5::dadd(dfm, cb * C5::F_BLK + 2 * 512 + ks * 1024), ID, pr + ks > 0);
            }
            tc5::commit(&bar);
        }
        __syncwarp();
        if (!k5::wait_mma(&bar, phase, a.ctl, &s_abort)) break;
        if (!k5::wait_bar(&ebar, eph, a.ctl, &s_abort)) break;
        eph ^= 1u;
        epi_pending = false;
        // ---- right-hand side = surface + rvol; stage combine (Sec. 7) ----
        if (w >= 4) {
            if (tid - 128 < 7 * TC && tile + gridDim.x < ntile) neighbours(tile + gridDim.x, tid - 128);
        } else {
            float R[20];
            tc5::ld16(tl + 128, R);
            tc5::ld4(tl + 144, R + 16);
            tc5::ld_wait();
            if (lane < 16) {
                const int m = 16 * w + lane, c = m >> 2, v = m & 3;
                const long e0 = (c0 + c) * 80 + v * 20;
                float* dst = sNew + c * 80 + v * 20;
                if (c < nvalid) {
                    const float4* rv = reinterpret_cast<const float4*>(sEpi + 2 * TC * 80 + c * 80 + v * 20);
#pragma unroll
                    for (int j = 0; j < 5; ++j) {
                        const float4 t = rv[j];
                        R[4 * j] += t.x;
                        R[4 * j + 1] += t.y;
                        R[4 * j + 2] += t.z;
                        R[4 * j + 3] += t.w;
                    }
                    if (a.abar_fix && v > 0) {
                        // the source's mean-acceleration part: -abar_i rho_l (the volume
                        // kernel's quadrature of rho abar against phi_l, orthonormal basis)
                        const float abv = abar_fix[v - 1];
                        const float* rho = sEpi + c * 80;
#pragma unroll
                        for (int l = 0; l < 20; ++l) R[l] -= abv * rho[l];
                    }
                    if (!a.stage) {
                        float4* o4 = reinterpret_cast<float4*>(a.out + e0);
#pragma unroll
                        for (int j = 0; j < 5; ++j) o4[j] = make_float4(R[4 * j], R[4 * j + 1], R[4 * j + 2], R[4 * j + 3]);
                    } else {
                        const float4* us = reinterpret_cast<const float4*>(sEpi + c * 80 + v * 20);
                        const float4* un = reinterpret_cast<const float4*>(sEpi + TC * 80 + c * 80 + v * 20);
#pragma unroll
                        for (int j = 0; j < 5; ++j) {
                            const float4 x = us[j];
                            const float4 y = a.rk_a != 0.f ? un[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                            dst[4 * j] = a.rk_a * y.x + a.rk_b * (x.x + dt * R[4 * j]);
                            dst[4 * j + 1] = a.rk_a * y.y + a.rk_b * (x.y + dt * R[4 * j + 1]);
                            dst[4 * j + 2] = a.rk_a * y.z + a.rk_b * (x.z + dt * R[4 * j + 2]);
                            dst[4 * j + 3] = a.rk_a * y.w + a.rk_b * (x.w + dt * R[4 * j + 3]);
                        }
                    }
                } else {
#pragma unroll
                    for (int l = 0; l < 20; ++l) dst[l] = (v == 0 && l == 0) ? 1.f : 0.f;
                }
            }
        }
        tc5::fence_before();
        __syncthreads();
        if (a.stage) {
            // positivity (Sec. 3.1): warp w takes cells 2w, 2w + 1.  A cell passes when
            // rho_0 - sum_l |rho_l| sup|phi_l| >= eps; otherwise rho is evaluated at every
            // volume and face Gauss point and the modes l > 0 are scaled by theta
            float thr[2];
            unsigned int st = 0u;
#pragma unroll
            for (int cl = 0; cl < 2; ++cl) {
                const float* rr = sNew + (2 * w + cl) * 80;
                float part = (lane >= 1 && lane < b) ? fabsf(rr[lane < b ? lane : 0]) * my_sup : 0.f;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                thr[cl] = 1.f;
                if (rr[0] - part < eps) {
                    float mn = 1e30f;
                    for (int pt = lane; pt < nq + nf; pt += 32) {
                        float rho = 0.f;
                        if (pt < nq) {
#pragma unroll
                            for (int l = 0; l < b; ++l) rho += rr[l] * __ldg(a.phiv + l * nq + pt);
                        } else {
#pragma unroll
                            for (int l = 0; l < b; ++l) rho += rr[l] * __ldg(a.phif + l * nf + (pt - nq));
                        }
                        mn = rho < mn ? rho : mn;
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const float other = __shfl_xor_sync(0xffffffffu, mn, o);
                        mn = other < mn ? other : mn;
                    }
                    const float rbar = rr[0];
                    if (a.trouble && mn < 0.f) {
                        const long cc = c0 + 2 * w + cl;
                        if (lane == 0 && cc < a.ncell) a.trouble[cc] |= DG_MARK_NEGATIVE;
                        st |= DG_ST_TROUBLED_;
                    }
                    if (mn < eps) {
                        if (rbar > eps) {
                            thr[cl] = (rbar - eps) / (rbar - mn);
                            st |= DG_ST_LIMITED_;
                        } else if (!a.trouble || !(rbar > 0.f)) {
                            // positivity by repetition: a mean in (0, eps] stands
                            st |= DG_ST_FAIL_;
                        }
                    }
                }
            }
            for (int el = lane; el < 160; el += 32) {
                const int cl = el / 80, e = 2 * w * 80 + el, l = e % 20;
                float v = sNew[e];
                if (l > 0) v *= (cl ? thr[1] : thr[0]);
                if (e / 80 < nvalid) {
                    if (!isfinite(v)) st |= DG_ST_NONFINITE_;
                    a.out[c0 * 80 + e] = v;
                }
            }
            st = __reduce_or_sync(0xffffffffu, st);
            if (lane == 0 && st) atomicOr(&s_status, st);
        }
        tc5::fence_before();
        __syncthreads();
        tc5::fence_after();
    }
    // a loop left early: no bulk copy may still write into this block's shared memory
    if (tid == 0 && epi_pending) tc5::mbar_wait(&ebar, eph);
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    if (tid == 0 && s_status) atomicOr(&a.ctl->status, s_status);
    if (w == 0) tc5::tmem_dealloc(tm, C5::TM_FACE);
}

// --------------------------------------------------------------------------
// projection of v (and |v|) of a state, CFL bound, forcing sums
// --------------------------------------------------------------------------
template <bool CHK = false>
__global__ void __launch_bounds__(256, 3) k5_project(const __grid_constant__ T5Args a)
{
    using P = C5::Proj;
    constexpr int TC = C5::TC, NT = C5::NT;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(8) uint64_t lbar[2];
    __shared__ uint32_t tslot;
    __shared__ int s_abort;
    __shared__ unsigned long long s_smax;
    __shared__ double s_tot[8];
    __shared__ double s_buf[NT];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    k5::copy16(sm + P::oPhi, a.tab + C5::oPhi, C5::szPhi);
    if (tid < 64) reinterpret_cast<float*>(sm + P::oWq)[tid] = reinterpret_cast<const float*>(a.tab + C5::oWq)[tid];
    float* const sUb = reinterpret_cast<float*>(sm + P::oU);
    float* const sAhb = reinterpret_cast<float*>(sm + P::oAh);
    const float* sWq = reinterpret_cast<const float*>(sm + P::oWq);
    unsigned char* sEB = sm + P::oEB;
    unsigned char* sPA = sm + P::oPA;
    float* const sVa = reinterpret_cast<float*>(sEB);  // |v| rows of the tile (learned sensor), after the products
    if (w == 0) tc5::tmem_alloc(&tslot, C5::TM_PROJ);
    if (tid == 0) {
        tc5::mbar_init(&bar, 1);
        tc5::mbar_init(&lbar[0], 1);
        tc5::mbar_init(&lbar[1], 1);
        s_abort = 0;
        s_smax = 0ull;
    }
    tc5::fence_async_smem();
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    const uint32_t tm = tslot;
    uint32_t phase = 0;
    const bool force = (a.flags & F_FORCE) != 0, dtf = (a.flags & F_DT) != 0;
    const int qw = w & 3, hp = w >> 2, r = 32 * qw + lane, h = r >> 6, q = r & 63;
    const uint32_t tl = tc5::tmem_addr(tm, 32 * qw, 0);
    float smax = 0.f;
    // positivity by repetition (projection of a stage output): read before this
    // launch's last block replaces ctl->sn
    const float vlim = CHK ? (float)(DG_REPEAT_SPEED * a.ctl->sn - 3.0 * a.ph.cs) : 0.f;
    double sums[4] = {0.0, 0.0, 0.0, 0.0};
    const long ntile = (a.ncell + TC - 1) / TC;
    auto fetch = [&](long t, int buf) {
        const long cb = t * TC;
        const int nv = k5::tile_cells(a.ncell, cb);
        float* su = sUb + buf * TC * 80;
        float* sa = sAhb + buf * TC * 60;
        k5::fill_tail(su, nv, 80, 1.f);
        if (force) k5::fill_tail(sa, nv, 60, 0.f);
        if (tid == 0) {
            tc5::fence_async_smem();
            tc5::mbar_expect_tx(&lbar[buf], (uint32_t)(nv * 80 * 4 + (force ? nv * 60 * 4 : 0)));
            k5::tile_copy(su, a.u_in, &a.tu, a.tmask & 1, cb, nv, 80, &lbar[buf]);
            if (force) k5::tile_copy(sa, a.ahat, &a.ta, a.tmask & 8, cb, nv, 60, &lbar[buf]);
        }
    };
    if (blockIdx.x < ntile) fetch(blockIdx.x, 0);
    int cur = 0;
    uint32_t lph = 0;
    uint32_t inflight = blockIdx.x < ntile ? 1u : 0u;
    for (long tile = blockIdx.x; tile < ntile; tile += gridDim.x, cur ^= 1) {
        const long c0 = tile * TC;
        const int nvalid = k5::tile_cells(a.ncell, c0);
        if (!k5::wait_bar(&lbar[cur], (lph >> cur) & 1u, a.ctl, &s_abort)) break;
        lph ^= 1u << cur;
        inflight &= ~(1u << cur);
        if (tile + gridDim.x < ntile) {
            fetch(tile + gridDim.x, cur ^ 1);
            inflight |= 1u << (cur ^ 1);
        }
        const float* sU = sUb + cur * TC * 80;
        const float* sAh = sAhb + cur * TC * 60;
        if (tid < TC * 4) {
            const int f = tid >> 4, c = tid & 15;
            k5::put_row(sEB + (c & 1) * 2 * P::EB, P::EB, 4 * (c >> 1) + f, sU + c * 80 + f * 20);
        }
        tc5::fence_async_smem();
        tc5::fence_before();
        __syncthreads();
        if (tid == 0) {
            tc5::fence_after();
            constexpr uint32_t ID = tc5::idesc_bf16(128, C5::NEP, 0, 0);
            const uint64_t dphi = tc5::sdesc(tc5::saddr(sm + P::oPhi), 128, 512);
            const uint64_t deb = tc5::sdesc(tc5::saddr(sEB), 128, 512);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh)
#pragma unroll
                for (int pr = 0; pr < 3; ++pr) {
                    int ca, cb;
                    k5::prod(pr, ca, cb);
                    const uint32_t ao = (hh == 0 ? 1 + 2 * ca : 2 * ca) * C5::PHI_BLK, bo = (hh * 2 + cb) * P::EB;
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks)
                        tc5::mma(tm, tc5::dadd(dphi, ao + ks * 256), tc5::dadd(deb, bo + ks * 256), ID, hh + pr + ks > 0);
                }
            tc5::commit(&bar);
        }
        __syncwarp();
        if (!k5::wait_mma(&bar, phase, a.ctl, &s_abort)) break;
        // v = m / rho and |v| at the point of the thread's four cells; rows
        // m = 32 h + 4 p + i (i: v_x, v_y, v_z, |v|) weighted by w_q/8
        {
            float ev[4][4];
#pragma unroll
            for (int pp = 0; pp < 4; ++pp) tc5::ld4(tl + 4 * (4 * hp + pp), ev[pp]);
            tc5::ld_wait();
            tc5::fence_before();
            const float wq8 = sWq[q] * 0.125f;
            float x[4][4];
#pragma unroll
            for (int pp = 0; pp < 4; ++pp) {
                const int c = 2 * (4 * hp + pp) + h;
                const float ir = rcp<float>(ev[pp][0]);
                const float vx = ev[pp][1] * ir, vy = ev[pp][2] * ir, vz = ev[pp][3] * ir;
                if (dtf && c < nvalid) {
                    const float sp = fabsf(vx) + fabsf(vy) + fabsf(vz);
                    smax = sp > smax ? sp : smax;
                }
                if (CHK && c < nvalid && fabsf(vx) + fabsf(vy) + fabsf(vz) > vlim) {
                    a.trouble[c0 + c] |= DG_MARK_FAST;
                    atomicOr(&a.ctl->status, DG_ST_TROUBLED_);
                }
                x[pp][0] = vx * wq8;
                x[pp][1] = vy * wq8;
                x[pp][2] = vz * wq8;
                x[pp][3] = sqrtf(vx * vx + vy * vy + vz * vz) * wq8;
            }
#pragma unroll
            for (int pp = 0; pp < 4; pp += 2) {
                uint4 hi, lo;
                tc5::split8(x[pp], hi, lo);
                const int p = 4 * hp + pp;
                const int o = (4 * h + (p >> 1)) * 128 + (q >> 3) * 1024 + (q & 7) * 16;
                *reinterpret_cast<uint4*>(sPA + o) = hi;
                *reinterpret_cast<uint4*>(sPA + P::PA + o) = lo;
            }
        }
        tc5::fence_async_smem();
        tc5::fence_before();
        __syncthreads();
        if (tid == 0) {
            tc5::fence_after();
            constexpr uint32_t ID = tc5::idesc_bf16(64, 32, 1, 1);
            const uint64_t dpa = tc5::sdesc(tc5::saddr(sPA), 1024, 128);
            const uint64_t dpm = tc5::sdesc(tc5::saddr(sm + P::oPhi), 512, 128);
#pragma unroll
            for (int pr = 0; pr < 3; ++pr) {
                int ca, cb;
                k5::prod(pr, ca, cb);
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                    tc5::mma(tm + 32, tc5::dadd(dpa, ca * P::PA + 2 * ks * 1024),
                             tc5::dadd(dpm, (1 + 2 * cb) * C5::PHI_BLK + ks * 1024), ID, pr + ks > 0);
            }
            tc5::commit(&bar);
        }
        __syncwarp();
        if (!k5::wait_mma(&bar, phase, a.ctl, &s_abort)) break;
        if (w < 4) {
            float R[20];
            tc5::ld16(tl + 32, R);
            tc5::ld4(tl + 48, R + 16);
            tc5::ld_wait();
            if (lane < 16) {
                const int m = 16 * w + lane, c = 2 * ((m & 31) >> 2) + (m >> 5), i = m & 3;
                if (c < nvalid) {
                    float* dst = i < 3 ? a.vh_out + (c0 + c) * 60 + i * 20 : (a.vabs_out ? a.vabs_out + (c0 + c) * 20 : nullptr);
                    if (dst) {
                        float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
                        for (int j = 0; j < 5; ++j) d4[j] = make_float4(R[4 * j], R[4 * j + 1], R[4 * j + 2], R[4 * j + 3]);
                    }
                }
                if (a.nu_next && i == 3) {
#pragma unroll
                    for (int l = 0; l < 20; ++l) sVa[c * 20 + l] = R[l];
                }
            }
        }
        if (a.nu_next) {
            // the learned sensor's coefficient of this state (Sec. 7 learned AV), for the
            // next step: features (rho_l/rho_0, |v|hat_l/cs), the network of the
            // inference kernel (same products and roundings); its buffers use the free
            // evaluation region
            __syncthreads();
            using PK = MlpPack<40>;
            uint32_t* sX = reinterpret_cast<uint32_t*>(sEB) + 512;  // after the |v| rows
            uint32_t* sH1 = sX + TC * (PK::KD / 2);
            uint32_t* sH2 = sH1 + TC * (MLP_H / 2);
            const float inv_cs = 1.0f / (float)a.ph.cs;
            auto feat = [&](int c, int k) -> float {
                if (c0 + c >= a.ncell || k >= 40) return 0.0f;
                if (k < 20) return sU[c * 80 + k] / sU[c * 80];
                return sVa[c * 20 + (k - 20)] * inv_cs;
            };
            block_mlp<40, TC, C5::NT>(feat, sX, sH1, sH2, a.mlp, (float)(a.ph.cs * a.ph.hp), (float)a.ph.nu_gate, c0,
                                      a.ncell, a.nu_next);
        }
        // per-cell forcing sums <rho a_h> = sum_l rho_l a_l (orthonormal basis) and <rho>
        if (force && tid < TC * 3) {
            const int c = tid / 3, i = tid % 3;
            if (c < nvalid) {
                const float* u = sU + c * 80;
                const float* ah = sAh + c * 60 + i * 20;
                float s = 0.f;
#pragma unroll
                for (int l = 0; l < 20; ++l) s += u[l] * ah[l];
                sums[i] += (double)s;
                if (i == 0) sums[3] += (double)u[0];
            }
        }
        tc5::fence_before();
        __syncthreads();
        tc5::fence_after();
    }
    if (tid == 0)
        for (int bb = 0; bb < 2; ++bb)
            if ((inflight >> bb) & 1u) tc5::mbar_wait(&lbar[bb], (lph >> bb) & 1u);
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    if (w == 0) tc5::tmem_dealloc(tm, C5::TM_PROJ);
    // ---- block reductions, then the last block of the launch ----
    if (dtf) {
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
            if (force) {
                for (int i = 0; i < 3; ++i) a.ctl->abar2[o][i] = s_tot[i] / s_tot[3];
            } else {
                a.ctl->abar2[o][0] = a.ctl->abar2[o][1] = a.ctl->abar2[o][2] = 0.0;
            }
            if (dtf) {
                const unsigned long long bits = atomicAdd(&a.ctl->smax, 0ull);
                a.ctl->sn = __longlong_as_double((long long)bits);
                a.ctl->smax = 0ull;
            }
        }
    }
}

}  // namespace dg
