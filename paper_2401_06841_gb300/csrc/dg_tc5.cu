// dg_tc5.cu -- host side of the degree-3 x3 tensor-core kernels: the table
// block (basis values at the volume and face Gauss points, weighted basis
// derivatives, quadrature weights) in the operand layouts of the products,
// kernel set-up and launches.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <cstring>

#include "dg_launch.cuh"
#include "dg_tc5_kernels.cuh"

namespace dg {

namespace {

int g_occ_vol[12] = {}, g_occ_face[3] = {0, 0, 0}, g_occ_proj[2] = {0, 0};

// scaled Legendre polynomial Pn_m = sqrt(2m+1) P_m and its derivative, by the
// three-term recurrence and P'_{m+1} = P'_{m-1} + (2m+1) P_m
void legendre(int m, double x, double& p, double& dp)
{
    double P[5] = {1.0, x, 0, 0, 0}, D[5] = {0.0, 1.0, 0, 0, 0};
    for (int j = 1; j < m; ++j) {
        P[j + 1] = ((2.0 * j + 1.0) * x * P[j] - j * P[j - 1]) / (j + 1.0);
        D[j + 1] = D[j - 1] + (2.0 * j + 1.0) * P[j];
    }
    const double s = std::sqrt(2.0 * m + 1.0);
    p = s * P[m];
    dp = s * D[m];
}

uint16_t bf16_rne(float x)
{
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float bf16_to_float(uint16_t h)
{
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// hi and lo BF16 components of value v at byte offset o of two component planes
void put(unsigned char* plane0, unsigned char* plane1, int o, double v)
{
    const float f = (float)v;
    const uint16_t hi = bf16_rne(f);
    const uint16_t lo = bf16_rne(f - bf16_to_float(hi));
    std::memcpy(plane0 + o, &hi, 2);
    std::memcpy(plane1 + o, &lo, 2);
}

}  // namespace

size_t tc5_table_bytes() { return (size_t)C5::tab_bytes; }

// x, w: the 4-point Gauss-Legendre rule on [-1, 1]
int tc5_build_tables(const double* x, const double* w, unsigned char* out, size_t cap)
{
    if (cap < (size_t)C5::tab_bytes) return -1;
    std::memset(out, 0, C5::tab_bytes);
    constexpr int n = C5::n, b = C5::b;
    constexpr Modes<3> M{};
    double P[4][4], dP[4][4];  // [degree][point]
    double Pe[4][2];           // [degree][end: -1, +1]
    for (int m = 0; m <= 3; ++m) {
        for (int a = 0; a < n; ++a) legendre(m, x[a], P[m][a], dP[m][a]);
        double d;
        legendre(m, -1.0, Pe[m][0], d);
        legendre(m, 1.0, Pe[m][1], d);
    }
    float* wq = reinterpret_cast<float*>(out + C5::oWq);
    float* ws = reinterpret_cast<float*>(out + C5::oWs);
    // volume points q = ia + n ib + n^2 ic
    for (int q = 0; q < C5::nq; ++q) {
        const int ia = q % n, ib = (q / n) % n, ic = q / (n * n);
        const double wv = w[ia] * w[ib] * w[ic];
        wq[q] = (float)wv;
        for (int l = 0; l < b; ++l) {
            const int i = M.i[l], j = M.j[l], k = M.l[l];
            const double phi = P[i][ia] * P[j][ib] * P[k][ic];
            // Phi blocks [Z, Phi_hi, Z, Phi_lo, Z]: row q, K = l
            const int o = tc5::koff(q, l, 128, 512);
            put(out + C5::oPhi + 1 * C5::PHI_BLK, out + C5::oPhi + 3 * C5::PHI_BLK, o, phi);
            // G_d: row l, K = q, w_q dphi_l / dxi_d
            const double g[3] = {wv * dP[i][ia] * P[j][ib] * P[k][ic], wv * P[i][ia] * dP[j][ib] * P[k][ic],
                                 wv * P[i][ia] * P[j][ib] * dP[k][ic]};
            const int og = tc5::koff(l, q, 128, 1024);
            for (int d = 0; d < 3; ++d)
                put(out + C5::oG + (2 * d) * C5::G_BLK, out + C5::oG + (2 * d + 1) * C5::G_BLK, og, g[d]);
        }
    }
    // face points (F, s): F = 2 d + side (side 1: xi_d = +1), s = a + n c along the
    // tangential axes t1 < t2; table row 16 + 16 F + s
    for (int F = 0; F < 6; ++F) {
        const int d = F >> 1, side = F & 1, t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
        for (int s = 0; s < C5::ns; ++s) {
            const int ia = s % n, ic = s / n;
            if (F == 0) ws[s] = (float)(w[ia] * w[ic]);
            for (int l = 0; l < b; ++l) {
                const int deg[3] = {M.i[l], M.j[l], M.l[l]};
                double phi = Pe[deg[d]][side];
                phi *= P[deg[t1]][ia] * P[deg[t2]][ic];
                const int o = tc5::koff(16 + 16 * F + s, l, 128, 512);
                put(out + C5::oF, out + C5::oF + C5::F_BLK, o, phi);
            }
        }
    }
    return 0;
}

// blocks of a kernel an SM holds at once, from its registers, shared memory
// and warps, and from the TMEM columns each block allocates for the whole
// launch (the runtime's occupancy query counts one block per SM for kernels
// that allocate tensor memory)
static cudaError_t resident_blocks(const void* fn, int dyn_smem, int tmem_cols, int& out)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_smem))) return e;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared)))
        return e;
    cudaFuncAttributes fa{};
    if ((e = cudaFuncGetAttributes(&fa, fn))) return e;
    int dev = 0, smem_sm = 0, resv = 0, regs_sm = 0, warps_sm = 0;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev))) return e;
    if ((e = cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev))) return e;
    if ((e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev))) return e;
    if ((e = cudaDeviceGetAttribute(&warps_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev))) return e;
    const int regs = (fa.numRegs + 7) & ~7;
    int n = smem_sm / (dyn_smem + (int)fa.sharedSizeBytes + resv);
    n = std::min(n, regs_sm / (regs * C5::NT));
    n = std::min(n, warps_sm / C5::NT);
    n = std::min(n, 512 / tmem_cols);
    out = n < 1 ? 1 : n;
    return cudaSuccess;
}

cudaError_t tc5_setup()
{
    cudaError_t e;
    // [0, 8): gate (1), driving (2), self-projection (4); [8, 12): the self-projecting
    // variants 4-7 with the wave-speed marks of positivity by repetition
    const void* vol[12] = {
        (const void*)k5_volume<false, false, false>,      (const void*)k5_volume<false, true, false>,
        (const void*)k5_volume<true, false, false>,       (const void*)k5_volume<true, true, false>,
        (const void*)k5_volume<false, false, true>,       (const void*)k5_volume<false, true, true>,
        (const void*)k5_volume<true, false, true>,        (const void*)k5_volume<true, true, true>,
        (const void*)k5_volume<false, false, true, true>, (const void*)k5_volume<false, true, true, true>,
        (const void*)k5_volume<true, false, true, true>,  (const void*)k5_volume<true, true, true, true>};
    for (int i = 0; i < 12; ++i) {
        const int v = i < 8 ? i : i - 4;
        if ((e = resident_blocks(vol[i], v < 6 ? C5::Vol::total : C5::Vol::total3, v < 4 ? C5::TM_VOL : C5::TM_VOLP,
                                 g_occ_vol[i])))
            return e;
    }
    if ((e = resident_blocks((const void*)k5_faces<0>, C5::Face::total, C5::TM_FACE, g_occ_face[0]))) return e;
    if ((e = resident_blocks((const void*)k5_faces<1>, C5::Face::total, C5::TM_FACE, g_occ_face[1]))) return e;
    if ((e = resident_blocks((const void*)k5_faces<2>, C5::Face::total, C5::TM_FACE, g_occ_face[2]))) return e;
    if ((e = resident_blocks((const void*)k5_project<false>, C5::Proj::total, C5::TM_PROJ, g_occ_proj[0]))) return e;
    return resident_blocks((const void*)k5_project<true>, C5::Proj::total, C5::TM_PROJ, g_occ_proj[1]);
}

// the driver's tensor-map encoder, found once through the runtime (no link to the
// driver library)
static PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

cudaError_t tc5_make_maps(T5Maps* out, const void* const* bases, const int* per, int n, long ncell)
{
    static_assert(sizeof(CUtensorMap) == sizeof(T5Map::map), "tensor map size");
    out->n = 0;
    if (n > 8 || ncell < C5::TC || ncell > 0x7fffffffL) return cudaErrorInvalidValue;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) return cudaErrorInvalidValue;
    for (int i = 0; i < n; ++i) {
        // rows of `per` floats, boxes of 16 rows: the row pitch and the box's inner
        // extent are multiples of 16 bytes, the base 256-byte aligned by the caller
        if ((reinterpret_cast<uintptr_t>(bases[i]) & 15u) || (per[i] * 4) % 16) return cudaErrorInvalidValue;
        const cuuint64_t dims[2] = {(cuuint64_t)per[i], (cuuint64_t)ncell};
        const cuuint64_t strides[1] = {(cuuint64_t)per[i] * 4};
        const cuuint32_t box[2] = {(cuuint32_t)per[i], (cuuint32_t)C5::TC};
        const cuuint32_t es[2] = {1, 1};
        CUtensorMap* m = reinterpret_cast<CUtensorMap*>(out->m[i].map);
        if (enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(bases[i]), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        out->m[i].base = bases[i];
    }
    out->n = n;
    return cudaSuccess;
}

static const CUtensorMap* find_map(const T5Maps* maps, const void* p)
{
    if (!maps || !p) return nullptr;
    for (int i = 0; i < maps->n; ++i)
        if (maps->m[i].base == p) return reinterpret_cast<const CUtensorMap*>(maps->m[i].map);
    return nullptr;
}

static int grid5(long ntile, int occ, int nsm)
{
    long g = (long)(occ > 0 ? occ : 1) * nsm;
    if (g > ntile) g = ntile;
    if (g > kMaxGrid) g = kMaxGrid;
    return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_tc5(const Launch& L, const T5Launch& t)
{
    if (L.K != 3) return cudaErrorInvalidValue;
    T5Args a{};
    a.u_in = static_cast<const float*>(t.u_in);
    a.u_n = static_cast<const float*>(t.u_n);
    a.out = static_cast<float*>(t.out);
    a.vh_in = static_cast<const float*>(t.vh_in);
    a.vh_out = static_cast<float*>(t.vh_out);
    a.vabs_out = static_cast<float*>(t.vabs_out);
    a.ahat = static_cast<const float*>(t.ahat);
    a.nu = t.nu;
    a.rvol = static_cast<float*>(t.rvol);
    a.tab = static_cast<const unsigned char*>(t.tab5);
    a.phiv = static_cast<const float*>(t.phiv);
    a.phif = static_cast<const float*>(t.phif);
    a.ctl = L.ctl;
    a.partials = L.partials;
    a.ncell = L.ncell;
    a.N = L.N;
    a.ph = L.ph;
    a.rk_a = (float)t.rk_a;
    a.rk_b = (float)t.rk_b;
    a.dt_pimax = t.dt_pimax;
    a.flags = t.flags;
    a.abar_in = t.abar_in;
    a.abar_out = t.abar_out;
    a.nu_next = t.nu_next;
    a.mlp = t.mlp;
    a.trouble = t.trouble;
    // tiled TMA descriptors of the buffers whose whole tiles the kernels stage
    a.tmask = 0;
    if (const CUtensorMap* m = find_map(t.maps, t.u_in)) { a.tu = *m; a.tmask |= 1; }
    if (const CUtensorMap* m = find_map(t.maps, t.u_n)) { a.tn = *m; a.tmask |= 2; }
    if (const CUtensorMap* m = find_map(t.maps, t.rvol)) { a.tr = *m; a.tmask |= 4; }
    if (const CUtensorMap* m = find_map(t.maps, t.ahat)) { a.ta = *m; a.tmask |= 8; }
    if (t.nu_next && (t.kind != T5_PROJECT || !t.mlp)) return cudaErrorInvalidValue;
    if ((t.flags & F_FORCE) && !t.ahat) return cudaErrorInvalidValue;
    const long ntile = (L.ncell + C5::TC - 1) / C5::TC;
    if (t.kind == T5_PROJECT) {
        if (t.trouble)
            k5_project<true><<<grid5(ntile, g_occ_proj[1], L.nsm), C5::NT, C5::Proj::total, L.st>>>(a);
        else
            k5_project<false><<<grid5(ntile, g_occ_proj[0], L.nsm), C5::NT, C5::Proj::total, L.st>>>(a);
        return cudaGetLastError();
    }
    a.stage = (t.kind == T5_STAGE) ? 1 : 0;
    // variants: gating (1); driving (2), the self-projection (4, 6 driven); a driven
    // self-projection also reduces the state's mean acceleration into abar_out,
    // which the face kernel then subtracts (abar_fix, read from abar_in)
    const bool proj = t.vh_self != nullptr, force = (t.flags & F_FORCE) != 0;
    a.vh_self = static_cast<float*>(t.vh_self);
    const int gate = L.ph.av_mode != 1 ? 1 : 0;
    const int vv = proj ? (force ? 6 : 4) + gate : (force ? 2 : 0) + gate;
    const bool marks = proj && t.trouble;  // wave-speed marks of the self-projected stage output
    const int gv = grid5(ntile, g_occ_vol[marks ? vv + 4 : vv], L.nsm);
    const int sv = (proj && force) ? C5::Vol::total3 : C5::Vol::total;
    if (proj && force) a.abar_out = a.abar_in;
    switch (vv) {
    case 0: k5_volume<false, false, false><<<gv, C5::NT, sv, L.st>>>(a); break;
    case 1: k5_volume<false, true, false><<<gv, C5::NT, sv, L.st>>>(a); break;
    case 2: k5_volume<true, false, false><<<gv, C5::NT, sv, L.st>>>(a); break;
    case 3: k5_volume<true, true, false><<<gv, C5::NT, sv, L.st>>>(a); break;
    case 4:
        marks ? k5_volume<false, false, true, true><<<gv, C5::NT, sv, L.st>>>(a)
              : k5_volume<false, false, true><<<gv, C5::NT, sv, L.st>>>(a);
        break;
    case 5:
        marks ? k5_volume<false, true, true, true><<<gv, C5::NT, sv, L.st>>>(a)
              : k5_volume<false, true, true><<<gv, C5::NT, sv, L.st>>>(a);
        break;
    case 6:
        marks ? k5_volume<true, false, true, true><<<gv, C5::NT, sv, L.st>>>(a)
              : k5_volume<true, false, true><<<gv, C5::NT, sv, L.st>>>(a);
        break;
    default:
        marks ? k5_volume<true, true, true, true><<<gv, C5::NT, sv, L.st>>>(a)
              : k5_volume<true, true, true><<<gv, C5::NT, sv, L.st>>>(a);
        break;
    }
    a.abar_fix = (proj && force) ? 1 : 0;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int rs = L.ph.riemann;
    const int gf = grid5(ntile, g_occ_face[rs], L.nsm);
    if (rs == 2)
        k5_faces<2><<<gf, C5::NT, C5::Face::total, L.st>>>(a);
    else if (rs == 1)
        k5_faces<1><<<gf, C5::NT, C5::Face::total, L.st>>>(a);
    else
        k5_faces<0><<<gf, C5::NT, C5::Face::total, L.st>>>(a);
    return cudaGetLastError();
}

}  // namespace dg
