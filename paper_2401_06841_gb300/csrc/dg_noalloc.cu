// dg_noalloc.cu -- dg_rhs_noalloc: the right-hand-side evaluation of dg_rhs for
// callers that cannot allocate device memory.
//
// Who needs it: code whose device memory is all held by its own pool (a
// framework's caching allocator that has reserved the GPU), code that must
// not call cudaMalloc/cudaFree after start-up (cudaMalloc can synchronise the
// device and cudaFree always does, which stalls every stream of a real-time
// or multi-stream pipeline), and code that simply cannot create a context
// object with caller-owned scratch.  Such a caller passes only its input and
// output buffers and a stream.
//
// The working memory this path needs -- the control block, the per-block
// reduction partials, the basis tables and one projected-velocity buffer --
// lives in one file-scope device array of fixed size (kNoAllocBytes, 64 MiB).
// Every GPU that loads the library holds that array until the process exits.
// Nothing here calls cudaMalloc, cudaFree, cudaMallocAsync, a torch allocator,
// or any host allocator: the tables are built in fixed-size static host
// buffers and copied in.
//
// Set-up: every call looks up the device address of the array on the current
// device with cudaGetSymbolAddress -- in host code the array's name is only a
// host-side stand-in, never a device address -- and the first call for a given
// degree and precision at that address builds and uploads the basis tables
// (again after a device reset has moved the array).  Make the first call of
// each degree and precision before any stream capture.
//
// Face flux: Rusanov only (there is no context to carry a choice of solver).
//
// Sharing: all calls on a device use the same array and it keeps the last
// call's contents.  The control block (whose counters and sums must start at
// zero) is cleared on the caller's stream at every call.  Two calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// the array: serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>

#include "../../include/dg.h"
#include "dg_launch.cuh"
#include "dg_tile.cuh"

using namespace dg;

namespace {

constexpr size_t kNoAllocBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

// the working memory of dg_rhs_noalloc on every device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct DevState {
    unsigned char* base = nullptr;  // device address of g_noalloc_scratch at the last call
    int tab_K = 0, tab_prec = -1;   // degree / precision of the uploaded tables
};
DevState g_dev[kMaxDevices];

constexpr size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// fixed layout inside the array: control block, partials, tile tables, vhat
constexpr size_t kOffCtl = 0;
constexpr size_t kOffPartials = a256(sizeof(Ctl));
constexpr size_t kOffTab = kOffPartials + a256(sizeof(double) * 16 * kMaxGrid);
constexpr size_t kTabWords = 16384;  // >= TileTab<K,BK>::total for K <= 3, both backends
constexpr size_t kOffVhat = kOffTab + a256(sizeof(double) * kTabWords);

static_assert(TileTab<3, BK_FMA>::total <= (int)kTabWords && TileTab<3, BK_X3>::total <= (int)kTabWords, "tables");

// ---- basis tables in fixed static host buffers (no host allocation) ----
// Gauss-Legendre by Newton's iteration on the three-term recurrence
void gauss_fixed(int n, long double* x, long double* w)
{
    for (int i = 0; i < n; ++i) {
        long double z = cosl(3.14159265358979323846264338327950288L * (i + 0.75L) / (n + 0.5L)), dp = 0;
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1.0L, p1 = z;
            for (int j = 2; j <= n; ++j) {
                const long double p2 = ((2.0L * j - 1.0L) * z * p1 - (j - 1.0L) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            const long double pn = (n == 0) ? 1.0L : p1, pm = (n == 1) ? 1.0L : p0;
            dp = n * (z * pn - pm) / (z * z - 1.0L);
            const long double dz = pn / dp;
            z -= dz;
            if (fabsl(dz) < 1e-19L) break;
        }
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0L / ((1.0L - z * z) * dp * dp);
    }
}

long double pn_fixed(int m, long double x)
{
    long double p0 = 1.0L, p1 = x;
    if (m == 0) return 1.0L;
    for (int j = 2; j <= m; ++j) {
        const long double p2 = ((2.0L * j - 1.0L) * x * p1 - (j - 1.0L) * p0) / j;
        p0 = p1;
        p1 = p2;
    }
    return sqrtl(2.0L * m + 1.0L) * p1;
}

uint16_t bf16_rne_fixed(float x)
{
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

double g_dense[4][8192];         // Phi, WPhi, Psi, PsiL (dense, zero padded)
double g_tab[kTabWords];         // the table block in doubles
unsigned char g_host[sizeof(double) * kTabWords];  // the table block in the element type

void frag_fixed(const double* B, int Kd, int Nd, uint32_t* out)
{
    for (int kt = 0; kt < Kd / 16; ++kt)
        for (int nt = 0; nt < Nd / 8; ++nt)
            for (int lane = 0; lane < 32; ++lane) {
                const int g = lane >> 2, t = lane & 3, n = nt * 8 + g;
                for (int half = 0; half < 2; ++half) {
                    const int k0 = kt * 16 + 2 * t + 8 * half;
                    uint16_t hi[2], lo[2];
                    for (int j = 0; j < 2; ++j) {
                        const float x = (float)B[(k0 + j) * Nd + n];
                        hi[j] = bf16_rne_fixed(x);
                        uint32_t hb = (uint32_t)hi[j] << 16;
                        float hf;
                        std::memcpy(&hf, &hb, 4);
                        lo[j] = bf16_rne_fixed(x - hf);
                    }
                    const size_t o = (((size_t)kt * (Nd / 8) + nt) * 32 + lane) * 4;
                    out[o + half] = (uint32_t)hi[0] | ((uint32_t)hi[1] << 16);
                    out[o + 2 + half] = (uint32_t)lo[0] | ((uint32_t)lo[1] << 16);
                }
            }
}

template <int K, int BK>
size_t fill_tables(int prec)
{
    using Cf = TileCfg<K, BK>;
    using TT = TileTab<K, BK>;
    constexpr int b = Cf::b, n = Cf::n, nq = Cf::nq, ns = Cf::ns, nf = Cf::nf;
    constexpr int KP = Cf::KP, NQP = Cf::NQP, NP = Cf::NP, B2 = Cf::B2, B2K = Cf::B2K, NSP = Cf::NSP, B2N = Cf::B2N;
    static_assert(KP * NQP <= 8192 && NQP * NP <= 8192 && B2K * NSP <= 8192 && NSP * B2N <= 8192, "dense sizes");
    constexpr Modes<K> M{};
    constexpr Modes2<K> M2{};
    std::memset(g_dense, 0, sizeof(g_dense));
    std::memset(g_tab, 0, sizeof(g_tab));
    long double xg[16], wg[16];
    gauss_fixed(n, xg, wg);
    auto phi = [&](int l, long double a, long double bb, long double c) {
        return pn_fixed(M.i[l], a) * pn_fixed(M.j[l], bb) * pn_fixed(M.l[l], c);
    };
    for (int q = 0; q < nq; ++q) {
        const int ia = q % n, ib = (q / n) % n, ic = q / (n * n);
        const long double wq = wg[ia] * wg[ib] * wg[ic] / 8.0L;
        for (int l = 0; l < b; ++l) {
            const long double p = phi(l, xg[ia], xg[ib], xg[ic]);
            g_dense[0][l * NQP + q] = (double)p;
            g_dense[1][q * NP + l] = (double)(wq * p);
            g_tab[TT::phiv + l * nq + q] = (double)p;
        }
    }
    for (int s = 0; s < ns; ++s) {
        const int a = s % n, c = s / n;
        const long double ws = wg[a] * wg[c];
        for (int p2 = 0; p2 < B2; ++p2) {
            const long double ps = pn_fixed(M2.p[p2], xg[a]) * pn_fixed(M2.q[p2], xg[c]);
            g_dense[2][p2 * NSP + s] = (double)ps;
            g_dense[3][s * B2N + p2] = (double)(ws * ps);
        }
    }
    for (int f = 0; f < 6; ++f) {
        const int d = f >> 1, t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
        for (int s = 0; s < ns; ++s) {
            long double xi[3];
            xi[d] = (f & 1) ? 1.0L : -1.0L;
            xi[t1] = xg[s % n];
            xi[t2] = xg[s / n];
            for (int l = 0; l < b; ++l) g_tab[TT::phif + l * nf + f * ns + s] = (double)phi(l, xi[0], xi[1], xi[2]);
        }
    }
    const int sizes[4] = {KP * NQP, NQP * NP, B2K * NSP, NSP * B2N};
    const int offs[4] = {Cf::oPhi, Cf::oWPhi, Cf::oPsi, Cf::oPsiL};
    if (BK == BK_FMA)
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < sizes[i]; ++j) g_tab[offs[i] + j] = g_dense[i][j];
    if (prec == DG_PREC_F64) {
        std::memcpy(g_host, g_tab, sizeof(double) * TT::total);
        return sizeof(double) * TT::total;
    }
    float* f = reinterpret_cast<float*>(g_host);
    for (int j = 0; j < TT::total; ++j) f[j] = (float)g_tab[j];
    if (BK == BK_X3) {
        uint32_t* w = reinterpret_cast<uint32_t*>(g_host);
        frag_fixed(g_dense[0], KP, NQP, w + Cf::oPhi);
        frag_fixed(g_dense[1], NQP, NP, w + Cf::oWPhi);
        frag_fixed(g_dense[2], B2K, NSP, w + Cf::oPsi);
        frag_fixed(g_dense[3], NSP, B2N, w + Cf::oPsiL);
    }
    return sizeof(float) * TT::total;
}

size_t fill_tables_for(int K, int prec)
{
    const bool x3 = (prec == DG_PREC_X3);
    if (K == 1) return x3 ? fill_tables<1, BK_X3>(prec) : fill_tables<1, BK_FMA>(prec);
    if (K == 2) return x3 ? fill_tables<2, BK_X3>(prec) : fill_tables<2, BK_FMA>(prec);
    return x3 ? fill_tables<3, BK_X3>(prec) : fill_tables<3, BK_FMA>(prec);
}

int report(int code, const char* msg)
{
    fprintf(stderr, "dg_rhs_noalloc: %s\n", msg);
    return code;
}

}  // namespace

extern "C" int dg_rhs_noalloc(const dg_mesh* mesh, int order, double cs, const dg_nu_params* nu, int precision,
                              const void* u_in, const void* ahat, void* dudt, double dt_for_pimax, void* stream)
{
    if (!mesh || !nu || !u_in || !dudt || !stream) return report(DG_EINVAL, "null argument");
    if (order < 1 || order > 3 || precision < 0 || precision > 2) return report(DG_EINVAL, "order or precision");
    if (mesh->n[0] < 1 || mesh->n[0] != mesh->n[1] || mesh->n[0] != mesh->n[2] || mesh->n[0] > kMaxN)
        return report(DG_EINVAL, "mesh");
    for (int d = 0; d < 3; ++d)
        if (mesh->L[d] != 1.0) return report(DG_EINVAL, "box size must be 1");
    if (nu->diffusion != 0.0) return report(DG_EINVAL, "the diffusion operator needs a context (dg_init)");
    if (!(cs > 0.0) || nu->mode < 0 || nu->mode > 1 || !(nu->rho_floor >= 0.0))
        return report(DG_EINVAL, "cs or artificial-viscosity parameters");
    const long N = mesh->n[0];
    const long ncell = N * N * N;
    const size_t b = (size_t)(order + 1) * (order + 2) * (order + 3) / 6;
    const size_t elem = (precision == DG_PREC_F64) ? sizeof(double) : sizeof(float);
    const size_t vh_bytes = (size_t)ncell * 3 * b * elem;
    if (kOffVhat + vh_bytes > kNoAllocBytes) {
        char msg[160];
        snprintf(msg, sizeof(msg), "mesh too large for the fixed working array: needs %zu bytes, limit %zu",
                 (size_t)(kOffVhat + vh_bytes), kNoAllocBytes);
        return report(DG_ENOMEM, msg);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return report(DG_ECUDA, "cudaGetDevice");
    DevState& S = g_dev[dev];
    cudaStream_t st = (cudaStream_t)stream;
    {
        // looked up at every call (a host-side query, no synchronisation): after a
        // device reset the module loads again and the array may sit elsewhere,
        // with no tables in it
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return report(DG_ECUDA, cudaGetErrorString(e));
        if (static_cast<unsigned char*>(p) != S.base) {
            S.base = static_cast<unsigned char*>(p);
            S.tab_K = 0;
            S.tab_prec = -1;
        }
    }
    if (S.tab_K != order || S.tab_prec != precision) {
        const size_t nb = fill_tables_for(order, precision);
        e = cudaMemcpyAsync(S.base + kOffTab, g_host, nb, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = (precision == DG_PREC_F64) ? setup_kernels<double>(order) : setup_kernels<float>(order);
        if (e != cudaSuccess) return report(DG_ECUDA, cudaGetErrorString(e));
        S.tab_K = order;
        S.tab_prec = precision;
    }
    // the control block (last-block counters, forcing sums) starts at zero
    e = cudaMemsetAsync(S.base + kOffCtl, 0, sizeof(Ctl), st);
    if (e != cudaSuccess) return report(DG_ECUDA, cudaGetErrorString(e));
    int nsm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return report(DG_ECUDA, cudaGetErrorString(e));

    Launch L{};
    L.st = st;
    L.K = order;
    L.N = (int)N;
    L.ncell = ncell;
    L.ph.cs = cs;
    L.ph.cs2 = cs * cs;
    L.ph.h = 1.0 / N;
    L.ph.hp = L.ph.h / (order + 1);
    L.ph.alpha = nu->alpha;
    L.ph.beta = nu->beta;
    L.ph.floor_ = nu->rho_floor;
    L.ph.av_mode = nu->mode;
    L.tab = S.base + kOffTab;
    L.ttab = S.base + kOffTab;
    L.ctl = reinterpret_cast<Ctl*>(S.base + kOffCtl);
    L.partials = reinterpret_cast<double*>(S.base + kOffPartials);
    L.nsm = nsm;
    L.bk = (precision == DG_PREC_X3) ? BK_X3 : BK_FMA;
    void* vh = S.base + kOffVhat;

    TileLaunch p{};
    p.mode = TM_PROJECT;
    p.u_in = u_in;
    p.vh_out = vh;
    p.ahat = ahat;
    p.flags = ahat ? F_FORCE : 0;
    p.abar_out = 0;
    TileLaunch r{};
    r.mode = TM_RHS;
    r.u_in = u_in;
    r.out = dudt;
    r.vh_in = vh;
    r.ahat = ahat;
    r.dt_pimax = dt_for_pimax;
    r.flags = ahat ? F_FORCE : 0;
    r.abar_in = 0;
    if (precision == DG_PREC_F64) {
        e = launch_tile<double>(L, p);
        if (e == cudaSuccess) e = launch_tile<double>(L, r);
    } else {
        e = launch_tile<float>(L, p);
        if (e == cudaSuccess) e = launch_tile<float>(L, r);
    }
    if (e != cudaSuccess) return report(DG_ECUDA, cudaGetErrorString(e));
    return DG_OK;
}
