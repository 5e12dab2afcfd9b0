// dg_api.cu -- host side of libdg: the C ABI of include/dg.h, basis and
// quadrature tables, the Ornstein-Uhlenbeck driving process, and the
// orchestration of the kernels on the caller's stream.
//
// The tables are computed here from first principles and share no code with
// any other implementation: Gauss-Legendre nodes and weights come from the
// eigen-decomposition of the Jacobi matrix of the Legendre recurrence
// (Golub & Welsch 1969) by cyclic Jacobi rotations in long double.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/dg.h"

#include <cufft.h>
#include <dlfcn.h>
#include "dg_launch.cuh"
#include "dg_mlp.cuh"
#include "dg_tables.cuh"
#include "dg_tile.cuh"

using namespace dg;

// ---------------------------------------------------------------------------
// basis and quadrature tables
// ---------------------------------------------------------------------------
namespace {

using tables::bf16_rne;
using tables::gauss_rule;
using tables::pnorm;

// Recovery weights of the face gradient: on the union of two cells, s in
// half-cell units (left cell s = xi - 1, right cell s = xi + 1), the polynomial
// r(s) = sum_{j <= 2K+1} d_j P_j(s/2) whose normalised-Legendre moments on each
// cell are that cell's K+1 normal coefficients; dr/ds at s = 0 is linear in
// the 2K+2 coefficients: wL[a] (left), wR[a] (right).
long double leg(int j, long double x)  // P_j(x)
{
    long double p0 = 1.0L, p1 = x;
    if (j == 0) return p0;
    for (int i = 1; i < j; ++i) {
        const long double p2 = ((2.0L * i + 1.0L) * x * p1 - i * p0) / (i + 1.0L);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

void recovery_weights(int K, double* wL, double* wR)
{
    const int n = 2 * K + 2;
    long double xg[12], wg[12];
    gauss_rule(12, xg, wg);
    long double A[8][16] = {};
    for (int a = 0; a <= K; ++a)
        for (int j = 0; j < n; ++j) {
            long double mL = 0.0L, mR = 0.0L;
            for (int g = 0; g < 12; ++g) {
                const long double pa = sqrtl(2.0L * a + 1.0L) * leg(a, xg[g]);
                mL += 0.5L * wg[g] * pa * leg(j, (xg[g] - 1.0L) / 2.0L);
                mR += 0.5L * wg[g] * pa * leg(j, (xg[g] + 1.0L) / 2.0L);
            }
            A[a][j] = mL;
            A[K + 1 + a][j] = mR;
        }
    // inverse by Gauss-Jordan with partial pivoting ([A | I] in 8 x 16)
    for (int i = 0; i < n; ++i) A[i][n + i] = 1.0L;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabsl(A[r][c]) > fabsl(A[p][c])) p = r;
        for (int j = 0; j < 2 * n; ++j) std::swap(A[c][j], A[p][j]);
        const long double inv = 1.0L / A[c][c];
        for (int j = 0; j < 2 * n; ++j) A[c][j] *= inv;
        for (int r = 0; r < n; ++r)
            if (r != c) {
                const long double f = A[r][c];
                for (int j = 0; j < 2 * n; ++j) A[r][j] -= f * A[c][j];
            }
    }
    // dr/ds(0) = sum_j d_j P_j'(0) / 2, P'_{j+1}(0) = P'_{j-1}(0) + (2j+1) P_j(0)
    long double dp[8] = {};
    dp[0] = 0.0L;
    dp[1] = 1.0L;
    for (int j = 1; j + 1 < n; ++j) dp[j + 1] = dp[j - 1] + (2.0L * j + 1.0L) * leg(j, 0.0L);
    for (int a = 0; a < n; ++a) {
        long double w = 0.0L;
        for (int j = 0; j < n; ++j) w += 0.5L * dp[j] * A[j][n + a];
        if (a <= K)
            wL[a] = (double)w;
        else
            wR[a - K - 1] = (double)w;
    }
}

template <int K>
std::vector<double> build_tables()
{
    using Dm = Dims<K>;
    using L = TabLayout<K>;
    constexpr int b = Dm::b, n = Dm::n, nq = Dm::nq, ns = Dm::ns, nf = Dm::nf, nl = Dm::nl, nql = Dm::nql;
    constexpr Modes<K> M{};
    std::vector<double> t(L::total, 0.0);
    long double xg[16], wg[16], xl[16], wl[16];
    gauss_rule(n, xg, wg);
    gauss_rule(nl, xl, wl);
    auto phi = [&](int l, long double a, long double bb, long double c) {
        return pnorm(M.i[l], a) * pnorm(M.j[l], bb) * pnorm(M.l[l], c);
    };
    for (int q = 0; q < nq; ++q) {
        const int ia = q % n, ib = (q / n) % n, ic = q / (n * n);
        const long double wq = wg[ia] * wg[ib] * wg[ic] / 8.0L;
        t[L::wq + q] = (double)wq;
        t[L::xq + 3 * q + 0] = (double)xg[ia];
        t[L::xq + 3 * q + 1] = (double)xg[ib];
        t[L::xq + 3 * q + 2] = (double)xg[ic];
        for (int l = 0; l < b; ++l) {
            const long double p = phi(l, xg[ia], xg[ib], xg[ic]);
            t[L::phiT + l * nq + q] = (double)p;
            t[L::wphi + q * b + l] = (double)(wq * p);
        }
    }
    // face f = 2d + side (side 1: xi_d = +1); point s = a + n*c over the two
    // tangential axes in increasing order
    for (int f = 0; f < 6; ++f) {
        const int d = f >> 1;
        const long double sd = (f & 1) ? 1.0L : -1.0L;
        const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
        for (int s = 0; s < ns; ++s) {
            long double xi[3];
            xi[d] = sd;
            xi[t1] = xg[s % n];
            xi[t2] = xg[s / n];
            const long double ws = wg[s % n] * wg[s / n];
            for (int l = 0; l < b; ++l) {
                const long double p = phi(l, xi[0], xi[1], xi[2]);
                t[L::phifT + l * nf + f * ns + s] = (double)p;
                t[L::lift + (f * ns + s) * b + l] = (double)(-sd * ws * p);
            }
        }
    }
    for (int q = 0; q < nql; ++q) {
        const int ia = q % nl, ib = (q / nl) % nl, ic = q / (nl * nl);
        t[L::wL + q] = (double)(wl[ia] * wl[ib] * wl[ic] / 8.0L);
        for (int l = 0; l < b; ++l) t[L::phiL + l * nql + q] = (double)phi(l, xl[ia], xl[ib], xl[ic]);
    }
    return t;
}

std::vector<double> tables_for(int K)
{
    if (K == 1) return build_tables<1>();
    if (K == 2) return build_tables<2>();
    return build_tables<3>();
}

// tables of the tile kernels in the element type of prec (dg_tables.cuh)
std::vector<char> tile_tables_for(int K, int prec)
{
    std::unique_ptr<tables::Work> w(new tables::Work);
    std::vector<char> out(sizeof(double) * tables::kTableWordsMax);
    const size_t n = tables::fill_tile_tables_for(K, prec, *w, reinterpret_cast<unsigned char*>(out.data()), out.size());
    out.resize(n);
    return out;
}

// Weights (a, b) of an SSP-RK stage out = a u^n + b (u + dt L) as the kernels
// receive them.  In single precision b is rounded to float and a = 1 - b is
// formed exactly, so that a + b = 1 in the kernels' arithmetic: the float
// roundings of 1/3 and 2/3 add up to 1 + 2^-25, and with them every SSP-RK3
// step would scale the state by 1 + 3e-8 on average, a steady drift of mass,
// momentum and energy.  Double precision keeps the rounded fractions (their
// sum is 1 - 2^-54).
static void rk_weights(int rk, int s, bool single, double& a, double& b)
{
    static const double A2[2] = {0.0, 0.5}, B2[2] = {1.0, 0.5};
    static const double A3[3] = {0.0, 0.75, 1.0 / 3.0}, B3[3] = {1.0, 0.25, 2.0 / 3.0};
    a = rk == 2 ? A2[s] : A3[s];
    b = rk == 2 ? B2[s] : B3[s];
    if (single && a != 0.0) {
        b = (double)(float)b;
        a = 1.0 - b;  // exact: b is in [1/4, 1) with a 24-bit significand
    }
}

int ttab_total(int K)
{
    // words of the larger of the two backends' layouts
    auto mx = [](int a, int b) { return a > b ? a : b; };
    if (K == 1) return mx(TileTab<1, BK_FMA>::total, TileTab<1, BK_X3>::total);
    if (K == 2) return mx(TileTab<2, BK_FMA>::total, TileTab<2, BK_X3>::total);
    return mx(TileTab<3, BK_FMA>::total, TileTab<3, BK_X3>::total);
}

int tab_total(int K)
{
    if (K == 1) return TabLayout<1>::total;
    if (K == 2) return TabLayout<2>::total;
    return TabLayout<3>::total;
}

// ---------------------------------------------------------------------------
// Ornstein-Uhlenbeck driving (Sec. 4.2)
// ---------------------------------------------------------------------------
constexpr int kMaxModes = 512;

struct Driver {
    bool on = false, dirty = false;
    int nm = 0, kmaxc = 0;
    int kv[kMaxModes][3];
    double x[kMaxModes][3][2];
    double zeta = 0, tc = 0, dtd = 0, f = 0, s = 0, t_next = 0, t_off = 0;
    uint64_t rng = 0;
    bool have_spare = false;
    double spare = 0;

    // SplitMix64 (Steele, Lea & Flood 2014)
    uint64_t next()
    {
        rng += 0x9E3779B97F4A7C15ULL;
        uint64_t z = rng;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
    double uni() { return (double)(next() >> 11) * 0x1.0p-53; }
    // Box-Muller, cosine branch first, sine branch on the following call
    double normal()
    {
        if (have_spare) {
            have_spare = false;
            return spare;
        }
        const double u1 = 1.0 - uni(), u2 = uni();
        const double r = std::sqrt(-2.0 * std::log(u1));
        const double ang = 2.0 * 3.14159265358979323846 * u2;
        spare = r * std::sin(ang);
        have_spare = true;
        return r * std::cos(ang);
    }
    void init(const dg_forcing& F, double cs)
    {
        const int K = (int)std::floor(std::sqrt((double)F.kmax2) + 1e-9);
        nm = 0;
        kmaxc = 0;
        for (int a = -K; a <= K; ++a)
            for (int b = -K; b <= K; ++b)
                for (int c = -K; c <= K; ++c) {
                    const int r2 = a * a + b * b + c * c;
                    if (r2 < F.kmin2 || r2 > F.kmax2) continue;
                    const int lead = a ? a : (b ? b : c);
                    if (lead <= 0 || nm >= kMaxModes) continue;
                    kv[nm][0] = a;
                    kv[nm][1] = b;
                    kv[nm][2] = c;
                    ++nm;
                }
        kmaxc = K;
        zeta = F.zeta;
        tc = 1.0 / (2.0 * cs * F.mach);   // L = 1
        dtd = tc / 100.0;
        f = std::exp(-dtd / tc);
        const double sigma = 2.0 * F.mach * F.mach * cs * cs;
        s = sigma / std::sqrt(4.0 * nm * (2.0 * zeta * zeta + (1.0 - zeta) * (1.0 - zeta)));
        rng = F.seed;
        have_spare = false;
        for (int m = 0; m < nm; ++m)
            for (int i = 0; i < 3; ++i)
                for (int r = 0; r < 2; ++r) x[m][i][r] = s * normal();
        t_next = dtd;
        t_off = F.t_off;
        on = F.on != 0;
        dirty = true;
    }
    void advance()
    {
        const double c = s * std::sqrt(1.0 - f * f);
        for (int m = 0; m < nm; ++m)
            for (int i = 0; i < 3; ++i)
                for (int r = 0; r < 2; ++r) x[m][i][r] = f * x[m][i][r] + c * normal();
    }
    // amplitudes A_k = P_zeta(k) x_k, P_zeta = zeta (I - kk^T/k^2) + (1-zeta) kk^T/k^2
    void amplitudes(std::vector<double>& amp, std::vector<int>& kvec) const
    {
        amp.assign(nm * 6, 0.0);
        kvec.assign(nm * 3, 0);
        for (int m = 0; m < nm; ++m) {
            double k2 = 0;
            for (int i = 0; i < 3; ++i) {
                kvec[m * 3 + i] = kv[m][i];
                k2 += (double)kv[m][i] * kv[m][i];
            }
            for (int r = 0; r < 2; ++r)
                for (int i = 0; i < 3; ++i) {
                    double acc = 0;
                    for (int j = 0; j < 3; ++j) {
                        const double kk = (double)kv[m][i] * kv[m][j] / k2;
                        acc += (zeta * ((i == j ? 1.0 : 0.0) - kk) + (1.0 - zeta) * kk) * x[m][j][r];
                    }
                    amp[(m * 3 + i) * 2 + r] = acc;
                }
        }
    }
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
// cuFFT, loaded at run time: the power spectrum is its only user, and a
// missing library then fails that call alone
struct CufftApi {
    bool ok = false;
    decltype(&cufftPlan3d) plan3d = nullptr;
    decltype(&cufftExecD2Z) exec_d2z = nullptr;
    decltype(&cufftSetStream) set_stream = nullptr;
    decltype(&cufftDestroy) destroy = nullptr;
};
static const CufftApi& cufft_api()
{
    static const CufftApi api = [] {
        CufftApi a;
        const char* names[] = {"libcufft.so.12", "libcufft.so.11", "libcufft.so"};
        void* h = nullptr;
        for (const char* n : names)
            if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
        if (!h) return a;
        a.plan3d = reinterpret_cast<decltype(a.plan3d)>(dlsym(h, "cufftPlan3d"));
        a.exec_d2z = reinterpret_cast<decltype(a.exec_d2z)>(dlsym(h, "cufftExecD2Z"));
        a.set_stream = reinterpret_cast<decltype(a.set_stream)>(dlsym(h, "cufftSetStream"));
        a.destroy = reinterpret_cast<decltype(a.destroy)>(dlsym(h, "cufftDestroy"));
        a.ok = a.plan3d && a.exec_d2z && a.set_stream && a.destroy;
        return a;
    }();
    return api;
}

struct dg_ctx {
    int N = 0, K = 0, prec = 0, rk = 3, b = 0;
    long ncell = 0;
    double cs = 1, cfl = 0.3, h = 1;
    dg_nu_params nu{};
    cudaStream_t st = nullptr;
    void* reg[3] = {nullptr, nullptr, nullptr};
    int cur = 0;
    int riemann = 0;  // DG_RIEMANN_*
    // projection carried over from the last stage of the previous step:
    // vhat buffer / abar slot pb and ctl->sn already hold the projection,
    // the forcing sums and the wave-speed bound of reg[cur]
    bool carry = false;
    int pb = 0;
    void* vhat = nullptr;
    void* ahat = nullptr;
    char* scratch = nullptr;
    size_t scratch_bytes = 0;
    Ctl* ctl = nullptr;
    double* partials = nullptr;
    void* tab = nullptr;
    void* ttab = nullptr;
    int* d_kvec = nullptr;
    double* d_amp = nullptr;
    void* gtab = nullptr;  // forcing: 1D factors
    double* ana = nullptr; // turbulence statistics accumulators
    cufftHandle fft = 0;   // power-spectrum plan (created on first use)
    int fft_ng = 0;
    Rule1 r1{};            // 1D Gauss rule
    double recL[4][4] = {}, recR[4][4] = {};  // recovery weights of the face gradient
    int nsm = 0;
    bool state_set = false;
    bool forcing_active = false;  // ahat holds a forcing to apply
    Driver drv;
    double t = 0.0, dt_last = 0.0;
    int64_t steps = 0;
    unsigned int status = 0;
    std::string err;
    // learned viscosity sensor
    float* mw = nullptr;       // FP32 master weights
    float* mm = nullptr;       // Adam first moments
    float* mv = nullptr;       // Adam second moments
    float* mg = nullptr;       // gradient
    uint32_t* mpack = nullptr; // packed BF16 inference weights
    double* mloss = nullptr;
    float* mwork = nullptr;
    float* nu_cell = nullptr;  // per-cell coefficient (learned mode)
    float* nu_next = nullptr;  // the next step's coefficient, written by the last stage (learned mode)
    void* vabs = nullptr;      // per-cell |v| projection (learned mode)
    // positivity by repetition (dg_opts.positivity): per-cell marks of an
    // attempt and how often each cell of u^n was scaled in this step
    bool repeat = false;
    unsigned char* trouble = nullptr;
    unsigned char* level = nullptr;
    bool marks_dirty = false;  // marks or levels may be non-zero
    // x3 at order 3: tcgen05 kernels (volume, faces, projection)
    bool tc5 = false;
    void* t5tab = nullptr;
    T5Maps t5maps{};  // tiled TMA descriptors of the state registers, rvol and a_h (tcgen05 kernels)
    void* rvol = nullptr;
    int mlp_D = 0, mlp_P = 0;
    long adam_t = 0;
    bool weights_set = false;
    // profiling: events recorded around launches, resolved in dg_profile_read
    bool prof = false;
    dg_prof counts{};
    struct Pending {
        cudaEvent_t a, b;
        int kind;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    ~dg_ctx()
    {
        for (auto& p : pending) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
        if (fft_ng > 0 && cufft_api().ok) cufft_api().destroy(fft);
    }
};

namespace {

struct ScratchLayout {
    size_t ctl, partials, tab, ttab, kvec, amp, gtab;
    size_t mw, mm, mv, mg, mpack, mloss, mwork;  // learned sensor: weights, Adam moments, grad, packed, loss, work
    size_t nu, nu2, vabs;                        // per-cell coefficients (this and the next step) and |v| projection (learned mode)
    size_t ana;                                  // turbulence statistics: 4 x DG_MAX_BINS doubles + 1
    size_t t5tab, rvol;                          // order 3: tensor-core table block, FP32 volume term [c][4][b]
    size_t trouble, level;                       // positivity by repetition: per-cell marks and levels (bytes)
    size_t total;
};

constexpr int kMlpMaxParams = 64 * 40 + 64 + 64 * 64 + 64 + 64 + 1;
constexpr int kMlpPackWords = 8192;
// positivity by repetition: attempts per step and halvings of dt before DG_EPOSITIVITY
constexpr int kRepeatAttempts = 32;
constexpr int kRepeatHalvings = 6;

ScratchLayout scratch_layout(int K, int N, bool learned = false)
{
    ScratchLayout s{};
    const long ncell = (long)N * N * N;
    size_t off = 0;
    s.ctl = off;
    off = align256(off + sizeof(Ctl));
    s.partials = off;
    off = align256(off + sizeof(double) * 16 * kMaxGrid);
    s.tab = off;
    off = align256(off + sizeof(double) * tab_total(K));
    s.ttab = off;
    off = align256(off + sizeof(double) * ttab_total(K));
    s.kvec = off;
    off = align256(off + sizeof(int) * 3 * kMaxModes);
    s.amp = off;
    off = align256(off + sizeof(double) * 6 * kMaxModes);
    s.gtab = off;
    off = align256(off + sizeof(double) * 2 * (size_t)N * kForceNK * (K + 1));
    s.mw = off;
    off = align256(off + sizeof(float) * kMlpMaxParams);
    s.mm = off;
    off = align256(off + sizeof(float) * kMlpMaxParams);
    s.mv = off;
    off = align256(off + sizeof(float) * kMlpMaxParams);
    s.mg = off;
    off = align256(off + sizeof(float) * kMlpMaxParams);
    s.mpack = off;
    off = align256(off + sizeof(uint32_t) * kMlpPackWords);
    s.mloss = off;
    off = align256(off + sizeof(double) * 16);
    s.mwork = off;
    off = align256(off + sizeof(float) * mlp_work_floats_host());
    s.ana = off;
    off = align256(off + sizeof(double) * (4 * DG_MAX_BINS + 1));
    s.nu = off;
    if (learned) off = align256(off + sizeof(float) * (size_t)ncell);
    s.nu2 = off;
    if (learned) off = align256(off + sizeof(float) * (size_t)ncell);
    s.vabs = off;
    const size_t b = (size_t)(K + 1) * (K + 2) * (K + 3) / 6;
    if (learned) off = align256(off + sizeof(double) * (size_t)ncell * b);
    // order 3: the tables and the volume-term buffer of the tcgen05 x3 kernels
    // (reserved for every precision: the size query does not take one)
    s.t5tab = off;
    if (K == 3) off = align256(off + tc5_table_bytes());
    s.rvol = off;
    if (K == 3) off = align256(off + sizeof(float) * (size_t)ncell * 4 * b);
    s.trouble = off;
    off = align256(off + (size_t)ncell);
    s.level = off;
    off = align256(off + (size_t)ncell);
    s.total = off;
    return s;
}

int fail(dg_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg;
    return code;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(ctx, DG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
    } while (0)

Launch make_launch(const dg_ctx* c)
{
    Launch L{};
    L.st = c->st;
    L.K = c->K;
    L.N = c->N;
    L.ncell = c->ncell;
    L.ph.cs = c->cs;
    L.ph.cs2 = c->cs * c->cs;
    L.ph.h = c->h;
    L.ph.hp = c->h / (c->K + 1);
    L.ph.alpha = c->nu.alpha;
    L.ph.beta = c->nu.beta;
    L.ph.floor_ = c->nu.rho_floor;
    L.ph.av_mode = c->nu.mode;
    L.ph.riemann = c->riemann;
    L.ph.nu_gate = c->nu.nu_gate;
    L.ph.eps = c->nu.diffusion;
    std::memcpy(L.ph.recL, c->recL, sizeof(c->recL));
    std::memcpy(L.ph.recR, c->recR, sizeof(c->recR));
    L.tab = c->tab;
    L.ttab = c->ttab;
    L.ctl = c->ctl;
    L.partials = c->partials;
    L.nsm = c->nsm;
    L.bk = (c->prec == DG_PREC_X3) ? 1 : 0;
    L.r1 = c->r1;
    L.gtab = c->gtab;
    return L;
}

size_t elem(const dg_ctx* c) { return c->prec == DG_PREC_F64 ? sizeof(double) : sizeof(float); }
size_t state_bytes(const dg_ctx* c) { return elem(c) * (size_t)c->ncell * 4 * c->b; }
size_t vec_bytes(const dg_ctx* c) { return elem(c) * (size_t)c->ncell * 3 * c->b; }
// the second projected-velocity buffer starts 256-byte aligned
void* vh_buf(const dg_ctx* c, int i) { return (char*)c->vhat + (size_t)i * align256(vec_bytes(c)); }

enum { KIND_PROJECT = 0, KIND_RHS = 1, KIND_FORCE = 2, KIND_OTHER = 3 };

cudaEvent_t take_event(dg_ctx* c)
{
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// bracket one launch: begin() before, end() after
struct Timed {
    dg_ctx* c;
    int kind;
    cudaEvent_t a = nullptr;
    Timed(dg_ctx* c_, int k) : c(c_), kind(k)
    {
        c->counts.launches += 1;
        if (kind == KIND_PROJECT) c->counts.n_project += 1;
        if (kind == KIND_RHS) c->counts.n_rhs += 1;
        if (kind == KIND_FORCE) c->counts.n_force += 1;
        if (kind == KIND_OTHER) c->counts.n_other += 1;
        if (c->prof) {
            a = take_event(c);
            cudaEventRecord(a, c->st);
        }
    }
    ~Timed()
    {
        if (c->prof && a) {
            cudaEvent_t b = take_event(c);
            cudaEventRecord(b, c->st);
            c->pending.push_back({a, b, kind});
        }
    }
};

// any call other than dg_step may overwrite the projected-velocity buffers,
// the forcing or the state: the next step projects afresh
void drop_carry(dg_ctx* c)
{
    if (c) c->carry = false;
}

// the x3 stage of order 3 on the tcgen05 kernels: a projection launch, or the
// volume + face launches of a right-hand side / stage followed by the
// projection of the stage's output (F_NEXTPROJ)
cudaError_t tile_tc5(dg_ctx* c, const TileLaunch& t)
{
    Launch L = make_launch(c);
    using TT = TileTab<3, BK_X3>;
    T5Launch p{};
    p.tab5 = c->t5tab;
    p.maps = &c->t5maps;
    p.rvol = c->rvol;
    p.phiv = static_cast<const float*>(c->ttab) + TT::phiv;
    p.phif = static_cast<const float*>(c->ttab) + TT::phif;
    p.nu = t.nu;
    p.ahat = t.ahat;
    p.rk_a = t.rk_a;
    p.rk_b = t.rk_b;
    p.dt_pimax = t.dt_pimax;
    p.trouble = t.mode == TM_RHS ? nullptr : t.trouble;
    if (t.mode == TM_PROJECT) {
        Timed tm(c, KIND_PROJECT);
        p.kind = T5_PROJECT;
        p.u_in = t.u_in;
        p.vh_out = t.vh_out;
        p.vabs_out = t.vabs_out;
        p.flags = t.flags;
        p.abar_out = t.abar_out;
        return launch_tc5(L, p);
    }
    {
        Timed tm(c, KIND_RHS);
        p.kind = (t.mode == TM_RHS) ? T5_RHS : T5_STAGE;
        p.u_in = t.u_in;
        p.u_n = t.u_n;
        p.out = t.out;
        p.vh_in = t.vh_in;
        p.vh_self = (t.flags & F_SELFPROJ) ? const_cast<void*>(t.vh_in) : nullptr;
        p.flags = t.flags & F_FORCE;
        p.abar_in = t.abar_in;
        cudaError_t e = launch_tc5(L, p);
        if (e != cudaSuccess) return e;
    }
    if (t.mode != TM_RHS && (t.flags & F_NEXTPROJ)) {
        Timed tm(c, KIND_PROJECT);
        T5Launch q = p;
        q.kind = T5_PROJECT;
        q.u_in = t.out;
        q.vh_out = t.vh_out;
        q.vabs_out = t.vabs_out;
        q.nu_next = t.nu_next;
        q.mlp = t.mlp;
        q.flags = t.flags & (F_FORCE | F_DT);
        q.abar_out = t.abar_out;
        return launch_tc5(L, q);
    }
    return cudaSuccess;
}

cudaError_t tile(dg_ctx* c, const TileLaunch& t)
{
    if (c->tc5) return tile_tc5(c, t);
    Timed tm(c, t.mode == 0 ? KIND_PROJECT : KIND_RHS);
    Launch L = make_launch(c);
    return (c->prec == DG_PREC_F64) ? launch_tile<double>(L, t) : launch_tile<float>(L, t);
}

// projection of u into vhat (+ forcing sums into abar slot, + CFL dt)
cudaError_t project(dg_ctx* c, const void* u, void* vhat, const void* ahat, bool dt_flag, int abar_out)
{
    TileLaunch t{};
    t.mode = 0;
    t.u_in = u;
    t.vh_out = vhat;
    t.ahat = ahat;
    t.flags = (ahat ? F_FORCE : 0) | (dt_flag ? F_DT : 0);
    t.abar_out = abar_out;
    return tile(c, t);
}

// pack FP32 weights into the BF16 fragments of the fused inference kernel
template <int D>
void pack_mlp(const float* w, uint32_t* out)
{
    using PK = MlpPack<D>;
    const MlpLayout L = MlpLayout::make(D);
    auto bf = [](float x) { return (uint32_t)bf16_rne(x); };
    auto frag = [&](auto Bat, int Kd, int Nd, uint32_t* dst) {
        for (int kt = 0; kt < Kd / 16; ++kt)
            for (int nt = 0; nt < Nd / 8; ++nt)
                for (int lane = 0; lane < 32; ++lane) {
                    const int g = lane >> 2, t = lane & 3, n = nt * 8 + g, k0 = kt * 16 + 2 * t;
                    uint32_t* o = dst + (((size_t)kt * (Nd / 8) + nt) * 32 + lane) * 2;
                    o[0] = bf(Bat(k0, n)) | (bf(Bat(k0 + 1, n)) << 16);
                    o[1] = bf(Bat(k0 + 8, n)) | (bf(Bat(k0 + 9, n)) << 16);
                }
    };
    frag([&](int k, int n) { return k < D ? w[L.oW1 + n * D + k] : 0.0f; }, PK::KD, 64, out + PK::w1);
    frag([&](int k, int n) { return w[L.oW2 + n * 64 + k]; }, 64, 64, out + PK::w2);
    frag([&](int k, int n) { return n == 0 ? w[L.oW3 + k] : 0.0f; }, 64, 8, out + PK::w3);
    float* bias = reinterpret_cast<float*>(out + PK::bias);
    for (int j = 0; j < 64; ++j) {
        bias[j] = w[L.ob1 + j];
        bias[64 + j] = w[L.ob2 + j];
    }
    bias[128] = w[L.ob3];
}

int upload_weights(dg_ctx* ctx, const float* w_host)
{
    static_assert(MlpPack<40>::words <= kMlpPackWords, "pack size");
    std::vector<uint32_t> pk(kMlpPackWords, 0u);
    if (ctx->mlp_D == 8) pack_mlp<8>(w_host, pk.data());
    if (ctx->mlp_D == 20) pack_mlp<20>(w_host, pk.data());
    if (ctx->mlp_D == 40) pack_mlp<40>(w_host, pk.data());
    CK(cudaMemcpyAsync(ctx->mw, w_host, sizeof(float) * ctx->mlp_P, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->mpack, pk.data(), sizeof(uint32_t) * kMlpPackWords, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    ctx->weights_set = true;
    return DG_OK;
}

// learned mode: the per-cell coefficient nu = cs h/p exp(net(x)) from u and
// the projection of |v| already in c->vabs
cudaError_t learned_infer(dg_ctx* c, const void* u)
{
    Timed tm(c, KIND_OTHER);
    Launch L = make_launch(c);
    return (c->prec == DG_PREC_F64)
               ? mlp_infer<double>(L, (const double*)u, (const double*)c->vabs, nullptr, c->ncell, c->mpack, c->nu_cell,
                                   nullptr)
               : mlp_infer<float>(L, (const float*)u, (const float*)c->vabs, nullptr, c->ncell, c->mpack, c->nu_cell,
                                  nullptr);
}

// learned mode: projection of |v| of u (v-hat into the scratch slot 1), then the coefficient
cudaError_t learned_nu(dg_ctx* c, const void* u)
{
    TileLaunch t{};
    t.mode = 0;
    t.u_in = u;
    t.vh_out = vh_buf(c, 1);
    t.vabs_out = c->vabs;
    t.flags = F_VABS;
    t.abar_out = 1;
    cudaError_t e = tile(c, t);
    if (e != cudaSuccess) return e;
    return learned_infer(c, u);
}

int upload_forcing(dg_ctx* ctx)
{
    std::vector<double> amp;
    std::vector<int> kv;
    ctx->drv.amplitudes(amp, kv);
    if (ctx->drv.nm == 0) return DG_OK;
    CK(cudaMemcpyAsync(ctx->d_kvec, kv.data(), sizeof(int) * kv.size(), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->d_amp, amp.data(), sizeof(double) * amp.size(), cudaMemcpyHostToDevice, ctx->st));
    Launch L = make_launch(ctx);
    cudaError_t e;
    {
        Timed tm(ctx, KIND_FORCE);
        e = (ctx->prec == DG_PREC_F64)
                ? launch_force<double>(L, ctx->drv.nm, ctx->d_kvec, ctx->d_amp, ctx->drv.kmaxc, (double*)ctx->ahat)
                : launch_force<float>(L, ctx->drv.nm, ctx->d_kvec, ctx->d_amp, ctx->drv.kmaxc, (float*)ctx->ahat);
    }
    CK(e);
    // the host buffers must stay valid until the copies ran
    CK(cudaStreamSynchronize(ctx->st));
    ctx->forcing_active = true;
    return DG_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

// The meshes every entry point accepts: n x n x n cells with 1 <= n <= kMaxN.
static bool cubic_mesh(const dg_mesh* m)
{
    return m->n[0] >= 1 && m->n[0] <= kMaxN && m->n[1] == m->n[0] && m->n[2] == m->n[0];
}

extern "C" {

int dg_scratch_bytes(const dg_mesh* mesh, int order, const dg_nu_params* nu, size_t* bytes)
{
    if (!bytes || !mesh || !nu || order < 1 || order > 3 || !cubic_mesh(mesh)) return DG_EINVAL;
    *bytes = scratch_layout(order, mesh->n[0], nu->mode == DG_AV_LEARNED).total;
    return DG_OK;
}

int dg_vhat_bytes(const dg_mesh* mesh, int order, int precision, size_t* bytes)
{
    if (!mesh || !bytes || order < 1 || order > 3 || precision < 0 || precision > 2 || !cubic_mesh(mesh))
        return DG_EINVAL;
    const size_t n = (size_t)mesh->n[0] * mesh->n[1] * mesh->n[2];
    const size_t b = (size_t)(order + 1) * (order + 2) * (order + 3) / 6;
    const size_t v = n * 3 * b * (precision == DG_PREC_F64 ? sizeof(double) : sizeof(float));
    *bytes = align256(v) + v;
    return DG_OK;
}

int dg_init(dg_ctx** out, const dg_mesh* mesh, int order, double cs, const dg_nu_params* nu, const dg_opts* opts)
{
    if (!out) return DG_EINVAL;
    *out = nullptr;
    if (!mesh || !nu || !opts) return DG_EINVAL;
    if (order < 1 || order > 3) return DG_EINVAL;
    if (!cubic_mesh(mesh)) return DG_EINVAL;
    for (int d = 0; d < 3; ++d)
        if (mesh->L[d] != 1.0) return DG_EINVAL;
    if (!(cs > 0.0)) return DG_EINVAL;
    if (nu->mode < 0 || nu->mode > 2 || !(nu->rho_floor >= 0.0) || !(nu->nu_gate >= 0.0) || !(nu->diffusion >= 0.0) ||
        (nu->fused_infer != 0 && nu->fused_infer != 1))
        return DG_EINVAL;
    if (opts->precision < 0 || opts->precision > 2) return DG_EINVAL;
    if (opts->rk_stages != 2 && opts->rk_stages != 3) return DG_EINVAL;
    if (!(opts->cfl > 0.0)) return DG_EINVAL;
    if (opts->riemann < DG_RIEMANN_RUSANOV || opts->riemann > DG_RIEMANN_HLLC) return DG_EINVAL;
    if (opts->positivity != DG_POS_SCALE && opts->positivity != DG_POS_REPEAT) return DG_EINVAL;
    if (!opts->stream) return DG_EINVAL;
    for (int i = 0; i < 3; ++i)
        if (!opts->u[i]) return DG_EINVAL;
    if (!opts->vhat || !opts->ahat || !opts->scratch) return DG_EINVAL;
    if (((uintptr_t)opts->scratch) & 255u) return DG_EINVAL;
    ScratchLayout sl = scratch_layout(order, mesh->n[0], nu->mode == DG_AV_LEARNED);
    if (opts->scratch_bytes < sl.total) return DG_ENOMEM;

    dg_ctx* ctx = new (std::nothrow) dg_ctx();
    if (!ctx) return DG_ENOMEM;
    ctx->N = mesh->n[0];
    ctx->K = order;
    ctx->b = (order + 1) * (order + 2) * (order + 3) / 6;
    ctx->ncell = (long)ctx->N * ctx->N * ctx->N;
    ctx->h = 1.0 / ctx->N;
    ctx->cs = cs;
    ctx->cfl = opts->cfl;
    ctx->rk = opts->rk_stages;
    ctx->riemann = opts->riemann;
    ctx->prec = opts->precision;
    ctx->nu = *nu;
    ctx->st = (cudaStream_t)opts->stream;
    for (int i = 0; i < 3; ++i) ctx->reg[i] = opts->u[i];
    ctx->vhat = opts->vhat;
    ctx->ahat = opts->ahat;
    ctx->scratch = (char*)opts->scratch;
    ctx->scratch_bytes = opts->scratch_bytes;
    ctx->ctl = (Ctl*)(ctx->scratch + sl.ctl);
    ctx->partials = (double*)(ctx->scratch + sl.partials);
    ctx->tab = ctx->scratch + sl.tab;
    ctx->ttab = ctx->scratch + sl.ttab;
    ctx->d_kvec = (int*)(ctx->scratch + sl.kvec);
    ctx->d_amp = (double*)(ctx->scratch + sl.amp);
    ctx->gtab = ctx->scratch + sl.gtab;
    for (int K = 0; K <= order; ++K) recovery_weights(K, ctx->recL[K], ctx->recR[K]);
    ctx->ana = (double*)(ctx->scratch + sl.ana);
    {
        long double xg[4], wg[4];
        gauss_rule(order + 1, xg, wg);
        for (int a = 0; a <= order; ++a) {
            ctx->r1.x[a] = (double)xg[a];
            ctx->r1.w[a] = (double)wg[a];
        }
    }
    ctx->mw = (float*)(ctx->scratch + sl.mw);
    ctx->mm = (float*)(ctx->scratch + sl.mm);
    ctx->mv = (float*)(ctx->scratch + sl.mv);
    ctx->mg = (float*)(ctx->scratch + sl.mg);
    ctx->mpack = (uint32_t*)(ctx->scratch + sl.mpack);
    ctx->mloss = (double*)(ctx->scratch + sl.mloss);
    ctx->mwork = (float*)(ctx->scratch + sl.mwork);
    ctx->nu_cell = (float*)(ctx->scratch + sl.nu);
    ctx->nu_next = (float*)(ctx->scratch + sl.nu2);
    ctx->vabs = ctx->scratch + sl.vabs;
    ctx->t5tab = ctx->scratch + sl.t5tab;
    ctx->rvol = ctx->scratch + sl.rvol;
    ctx->repeat = opts->positivity == DG_POS_REPEAT;
    ctx->trouble = reinterpret_cast<unsigned char*>(ctx->scratch + sl.trouble);
    ctx->level = reinterpret_cast<unsigned char*>(ctx->scratch + sl.level);
    ctx->marks_dirty = true;
    // order-3 x3 on the tcgen05 kernels (the learned sensor's in-step evaluation,
    // fused_infer, runs in their last projection)
    ctx->tc5 = ctx->prec == DG_PREC_X3 && order == 3 && nu->diffusion == 0.0 && opts->x3_backend == 0;
    ctx->mlp_D = 2 * ctx->b;
    ctx->mlp_P = mlp_params(ctx->mlp_D);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = (ctx->prec == DG_PREC_F64) ? setup_kernels<double>(order) : setup_kernels<float>(order);
    if (e == cudaSuccess && ctx->tc5) e = tc5_setup();
    if (e == cudaSuccess && ctx->tc5) {
        // whole tiles by tiled TMA loads (1D bulk copies where no descriptor could be made)
        const void* bases[5] = {ctx->reg[0], ctx->reg[1], ctx->reg[2], ctx->rvol, ctx->ahat};
        const int per[5] = {80, 80, 80, 80, 60};
        if (tc5_make_maps(&ctx->t5maps, bases, per, 5, ctx->ncell) != cudaSuccess) ctx->t5maps.n = 0;
    }
    if (e != cudaSuccess) {
        fprintf(stderr, "dg_init: %s\n", cudaGetErrorString(e));
        delete ctx;
        return DG_ECUDA;
    }
    // tables in the element type of the precision mode
    std::vector<double> t = tables_for(order);
    std::vector<char> tt = tile_tables_for(order, ctx->prec);
    Ctl c0{};
    c0.dt_scale = 1.0;
    c0.dt_num = ctx->cfl * ctx->h / (order + 1);
    {
        const double hp = ctx->h / (order + 1);
        c0.dt_diff = nu->diffusion > 0.0 ? ctx->cfl * hp * hp / (2.0 * nu->diffusion) : 0.0;
    }
    e = cudaMemcpyAsync(ctx->ctl, &c0, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->st);
    if (e == cudaSuccess) {
        if (ctx->prec == DG_PREC_F64) {
            e = cudaMemcpyAsync(ctx->tab, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice, ctx->st);
        } else {
            std::vector<float> tf(t.begin(), t.end());
            e = cudaMemcpyAsync(ctx->tab, tf.data(), sizeof(float) * tf.size(), cudaMemcpyHostToDevice, ctx->st);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->ttab, tt.data(), tt.size(), cudaMemcpyHostToDevice, ctx->st);
        std::vector<unsigned char> t5;
        if (e == cudaSuccess && ctx->tc5) {
            t5.resize(tc5_table_bytes());
            if (tc5_build_tables(ctx->r1.x, ctx->r1.w, t5.data(), t5.size()) != 0) e = cudaErrorInvalidValue;
            if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->t5tab, t5.data(), t5.size(), cudaMemcpyHostToDevice, ctx->st);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ahat, 0, vec_bytes(ctx), ctx->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    if (e != cudaSuccess) {
        fprintf(stderr, "dg_init: %s\n", cudaGetErrorString(e));
        delete ctx;
        return DG_ECUDA;
    }
    *out = ctx;
    return DG_OK;
}

void dg_free(dg_ctx* ctx) { delete ctx; }

const char* dg_last_error(const dg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int dg_set_state(dg_ctx* ctx, const void* src, int src_on_host)
{
    drop_carry(ctx);
    if (!ctx) return DG_EINVAL;
    if (!src) return fail(ctx, DG_EINVAL, "dg_set_state: null source");
    ctx->cur = 0;
    CK(cudaMemcpyAsync(ctx->reg[0], src, state_bytes(ctx), src_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                       ctx->st));
    unsigned int zero = 0u;
    CK(cudaMemcpyAsync(&ctx->ctl->status, &zero, sizeof(zero), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    ctx->status = 0u;
    ctx->state_set = true;
    return DG_OK;
}

int dg_get_state(dg_ctx* ctx, void* dst, int dst_on_host)
{
    if (!ctx) return DG_EINVAL;
    if (!dst) return fail(ctx, DG_EINVAL, "dg_get_state: null destination");
    if (!ctx->state_set) return fail(ctx, DG_ESTATE, "dg_get_state: no state set");
    CK(cudaMemcpyAsync(dst, ctx->reg[ctx->cur], state_bytes(ctx),
                       dst_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return DG_OK;
}

int dg_project_velocity(dg_ctx* ctx, const void* u_in, void* vhat_out)
{
    drop_carry(ctx);
    if (!ctx) return DG_EINVAL;
    if (!u_in || !vhat_out) return fail(ctx, DG_EINVAL, "dg_project_velocity: null buffer");
    CK(project(ctx, u_in, vhat_out, nullptr, false, 0));
    CK(cudaStreamSynchronize(ctx->st));
    return DG_OK;
}

int dg_rhs(dg_ctx* ctx, const void* u_in, const void* ahat, void* dudt, double dt_for_pimax)
{
    drop_carry(ctx);
    if (!ctx) return DG_EINVAL;
    if (!u_in || !dudt) return fail(ctx, DG_EINVAL, "dg_rhs: null buffer");
    const bool learned = ctx->nu.mode == DG_AV_LEARNED;
    if (learned && !ctx->weights_set) return fail(ctx, DG_ESTATE, "dg_rhs: learned mode needs dg_set_av_weights");
    if (learned) CK(learned_nu(ctx, u_in));
    CK(project(ctx, u_in, vh_buf(ctx, 0), ahat, false, 0));
    TileLaunch t{};
    t.nu = learned ? ctx->nu_cell : nullptr;
    t.mode = 1;
    t.u_in = u_in;
    t.out = dudt;
    t.vh_in = vh_buf(ctx, 0);
    t.ahat = ahat;
    t.dt_pimax = dt_for_pimax;
    t.flags = ahat ? F_FORCE : 0;
    t.abar_in = 0;
    CK(tile(ctx, t));
    unsigned int st = 0u;
    CK(cudaMemcpyAsync(&st, &ctx->ctl->status, sizeof(st), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (st & DG_ST_TIMEOUT) return fail(ctx, DG_ECUDA, "dg_rhs: a tensor-core completion wait timed out");
    return DG_OK;
}

int dg_set_forcing(dg_ctx* ctx, const dg_forcing* f)
{
    drop_carry(ctx);
    if (!ctx) return DG_EINVAL;
    if (!f) return fail(ctx, DG_EINVAL, "dg_set_forcing: null");
    if (f->on && (!(f->mach > 0.0) || f->kmin2 < 1 || f->kmax2 < f->kmin2 || f->kmax2 > 64 || f->zeta < 0.0 ||
                  f->zeta > 1.0))
        return fail(ctx, DG_EINVAL, "dg_set_forcing: bad parameters");
    if (!f->on) {
        ctx->drv.on = false;
        ctx->forcing_active = false;
        CK(cudaMemsetAsync(ctx->ahat, 0, vec_bytes(ctx), ctx->st));
        return DG_OK;
    }
    ctx->drv.init(*f, ctx->cs);
    if (ctx->drv.nm > kMaxModes) return fail(ctx, DG_EINVAL, "dg_set_forcing: too many modes");
    ctx->forcing_active = false;
    return DG_OK;
}

int dg_set_forcing_coeffs(dg_ctx* ctx, const void* src, int src_on_host)
{
    drop_carry(ctx);
    if (!ctx) return DG_EINVAL;
    ctx->drv.on = false;
    if (!src) {
        ctx->forcing_active = false;
        CK(cudaMemsetAsync(ctx->ahat, 0, vec_bytes(ctx), ctx->st));
        return DG_OK;
    }
    CK(cudaMemcpyAsync(ctx->ahat, src, vec_bytes(ctx), src_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                       ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    ctx->forcing_active = true;
    return DG_OK;
}

int dg_forcing_from_modes(dg_ctx* ctx, int nmodes, const int32_t* kvec, const double* amp)
{
    drop_carry(ctx);
    if (!ctx) return DG_EINVAL;
    if (nmodes < 1 || nmodes > kMaxModes || !kvec || !amp) return fail(ctx, DG_EINVAL, "dg_forcing_from_modes: bad args");
    int kmaxc = 0;
    for (int i = 0; i < 3 * nmodes; ++i) kmaxc = std::max(kmaxc, std::abs((int)kvec[i]));
    if (kmaxc > 8) return fail(ctx, DG_EINVAL, "dg_forcing_from_modes: |k_d| > 8");
    CK(cudaMemcpyAsync(ctx->d_kvec, kvec, sizeof(int) * 3 * nmodes, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->d_amp, amp, sizeof(double) * 6 * nmodes, cudaMemcpyHostToDevice, ctx->st));
    Launch L = make_launch(ctx);
    cudaError_t e;
    {
        Timed tm(ctx, KIND_FORCE);
        e = (ctx->prec == DG_PREC_F64)
                ? launch_force<double>(L, nmodes, ctx->d_kvec, ctx->d_amp, kmaxc, (double*)ctx->ahat)
                : launch_force<float>(L, nmodes, ctx->d_kvec, ctx->d_amp, kmaxc, (float*)ctx->ahat);
    }
    CK(e);
    CK(cudaStreamSynchronize(ctx->st));
    ctx->drv.on = false;
    ctx->forcing_active = true;
    return DG_OK;
}

int dg_step(dg_ctx* ctx, int nsteps, double fixed_dt, double* t_out, double* dt_last)
{
    if (!ctx) return DG_EINVAL;
    if (nsteps < 0) return fail(ctx, DG_EINVAL, "dg_step: nsteps < 0");
    if (!ctx->state_set) return fail(ctx, DG_ESTATE, "dg_step: no state set");
    if (ctx->nu.mode == DG_AV_LEARNED && !ctx->weights_set)
        return fail(ctx, DG_ESTATE, "dg_step: learned mode needs dg_set_av_weights");
    for (int st = 0; st < nsteps; ++st) {
        // driving schedule (Sec. 4.2): OU update at the first step with t >= t_next
        if (ctx->drv.on && ctx->drv.t_off > 0.0 && ctx->t > ctx->drv.t_off) {
            ctx->carry = false;
            ctx->drv.on = false;
            ctx->forcing_active = false;
            CK(cudaMemsetAsync(ctx->ahat, 0, vec_bytes(ctx), ctx->st));
        }
        if (ctx->drv.on) {
            while (ctx->t >= ctx->drv.t_next) {
                ctx->drv.advance();
                ctx->drv.t_next += ctx->drv.dtd;
                ctx->drv.dirty = true;
            }
            if (ctx->drv.dirty) {
                ctx->carry = false;  // new a_h: the forcing sums change
                int rc = upload_forcing(ctx);
                if (rc) return rc;
                ctx->drv.dirty = false;
            }
        }
        const bool force = ctx->forcing_active;
        const int A = ctx->cur, B = (ctx->cur + 1) % 3, C = (ctx->cur + 2) % 3;
        // register use: RK3  A->B, (B,A)->C, (C,A)->B ; RK2  A->B, (B,A)->C
        const int in3[3] = {A, B, C}, out3[3] = {B, C, B};
        const int in2[2] = {A, B}, out2[2] = {B, C};
        const int* in = ctx->rk == 2 ? in2 : in3;
        const int* out = ctx->rk == 2 ? out2 : out3;
        bool ok = false;
        double dt = 0.0;
        unsigned int status = 0u;
        const bool learned = ctx->nu.mode == DG_AV_LEARNED;
        const bool fused = learned && ctx->nu.fused_infer;
        const int pb = ctx->pb;
        // positivity by repetition (Sec. 3.1, last paragraph): the stages mark the
        // cells they trouble; the marked cells of u^n (register A) that are not flat
        // are scaled towards their flat expansion and the step is attempted again; a
        // flat cell with negative density, or a failed cell mean, halves dt.
        // Otherwise the rescaled stage outputs stand and a failed mean retries with
        // dt/2, dt/4, dt/8
        const bool repeat = ctx->repeat;
        unsigned char* marks = repeat ? ctx->trouble : nullptr;
        if (repeat && ctx->marks_dirty) {
            CK(cudaMemsetAsync(ctx->trouble, 0, (size_t)ctx->ncell, ctx->st));
            CK(cudaMemsetAsync(ctx->level, 0, (size_t)ctx->ncell, ctx->st));
            ctx->marks_dirty = false;
        }
        const int max_attempts = repeat ? kRepeatAttempts : 4, max_halvings = repeat ? kRepeatHalvings : 3;
        int halvings = 0, attempts = 0;
        for (int retry = 0; retry < max_attempts && halvings <= max_halvings && !ok; ++retry) {
            attempts = retry + 1;
            struct {
                double dt_scale, fixed_dt;
            } hs = {1.0 / (double)(1 << halvings), fixed_dt};
            CK(cudaMemcpyAsync(&ctx->ctl->dt_scale, &hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->st));
            unsigned int zero = 0u;
            CK(cudaMemcpyAsync(&ctx->ctl->status, &zero, sizeof(zero), cudaMemcpyHostToDevice, ctx->st));
            // stage 1 needs the projection of u^n (+ its wave-speed bound): carried
            // over from the last stage of the previous step, else a projection
            // launch; later stages get theirs from the previous stage's epilogue
            // (double-buffered vhat / abar slots, alternating from slot pb)
            const bool use_carry = retry == 0 && ctx->carry;
            ctx->carry = false;
            // learned mode: the coefficient once per step, cached for all stages; the
            // last stage of the previous step evaluated it for u^n (carried), else the
            // |v| projection and the inference run here
            if (learned) {
                if (use_carry && fused)
                    std::swap(ctx->nu_cell, ctx->nu_next);
                else
                    CK(use_carry ? learned_infer(ctx, ctx->reg[A]) : learned_nu(ctx, ctx->reg[A]));
            }
            if (!use_carry) CK(project(ctx, ctx->reg[A], vh_buf(ctx, pb), force ? ctx->ahat : nullptr, true, pb));
            for (int s = 0; s < ctx->rk; ++s) {
                const bool last = s + 1 == ctx->rk;
                TileLaunch t{};
                t.nu = learned ? ctx->nu_cell : nullptr;
                t.mode = (learned && last) ? 3 : 2;
                t.nu_next = (learned && last && fused) ? ctx->nu_next : nullptr;
                t.vabs_out = (learned && last && !fused) ? ctx->vabs : nullptr;
                t.mlp = ctx->mpack;
                t.u_in = ctx->reg[in[s]];
                t.u_n = ctx->reg[A];
                t.out = ctx->reg[out[s]];
                t.vh_in = vh_buf(ctx, (pb + s) & 1);
                t.vh_out = vh_buf(ctx, (pb + s + 1) & 1);
                t.ahat = force ? ctx->ahat : nullptr;
                rk_weights(ctx->rk, s, ctx->prec != DG_PREC_F64, t.rk_a, t.rk_b);
                // every stage projects its output; the last one for the next step,
                // with the CFL bound (and |v| in learned mode).  On the tcgen05 kernels
                // the stages after the first project their own input in the volume
                // kernel instead (driven: with the forcing sums), so only the last
                // stage's output gets a projection launch
                const bool fold = ctx->tc5;
                t.flags = (force ? F_FORCE : 0) | ((fold && !last) ? 0 : F_NEXTPROJ) | (last ? F_DT : 0) |
                          ((fold && s > 0) ? F_SELFPROJ : 0);
                t.abar_in = (pb + s) & 1;
                t.abar_out = (pb + s + 1) & 1;
                t.trouble = marks;
                CK(tile(ctx, t));
            }
            struct {
                unsigned int status;
                double dt;
            } back{};
            CK(cudaMemcpyAsync(&back.status, &ctx->ctl->status, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->st));
            CK(cudaMemcpyAsync(&back.dt, &ctx->ctl->dt, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
            CK(cudaStreamSynchronize(ctx->st));
            status = back.status;
            dt = back.dt;
            ok = !(status & (DG_ST_FAIL | DG_ST_TROUBLED_));
            if (ok) break;
            if (!repeat) {
                ++halvings;
                continue;
            }
            // flatten the marked cells of u^n; a flat one (or a failed mean) halves dt
            ctx->marks_dirty = true;
            CK(cudaMemcpyAsync(&ctx->ctl->status, &zero, sizeof(zero), cudaMemcpyHostToDevice, ctx->st));
            {
                Timed tm(ctx, KIND_OTHER);
                Launch L = make_launch(ctx);
                cudaError_t e = (ctx->prec == DG_PREC_F64)
                                    ? launch_flatten<double>(L, (double*)ctx->reg[A], ctx->trouble, ctx->level)
                                    : launch_flatten<float>(L, (float*)ctx->reg[A], ctx->trouble, ctx->level);
                CK(e);
            }
            unsigned int fst = 0u;
            CK(cudaMemcpyAsync(&fst, &ctx->ctl->status, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->st));
            CK(cudaStreamSynchronize(ctx->st));
            if ((fst & DG_ST_FLAT_) || (status & DG_ST_FAIL)) {
                ++halvings;
            } else if (!(fst & DG_ST_SCALED_)) {
                // only flat cells marked for their speed: the attempt stands
                ok = true;
                break;
            }
        }
        status &= 0xffu;
        if (repeat && attempts > 1) status |= DG_ST_REPEATED;
        if (!ok) {
            ctx->status |= status;
            return fail(ctx, DG_EPOSITIVITY, repeat ? "dg_step: positivity repetitions exhausted"
                                                    : "dg_step: positivity retries exhausted");
        }
        ctx->status |= status;
        ctx->cur = out[ctx->rk - 1];
        ctx->pb = (pb + ctx->rk) & 1;
        ctx->carry = !(status & DG_ST_NONFINITE);
        ctx->t += dt;
        ctx->dt_last = dt;
        ctx->steps += 1;
        if (status & DG_ST_TIMEOUT) return fail(ctx, DG_ECUDA, "dg_step: a tensor-core completion wait timed out");
        if (status & DG_ST_NONFINITE) return fail(ctx, DG_ENONFINITE, "dg_step: non-finite coefficient");
    }
    if (t_out) *t_out = ctx->t;
    if (dt_last) *dt_last = ctx->dt_last;
    return DG_OK;
}

int dg_diagnostics(dg_ctx* ctx, double dt_for_pimax, dg_diag* out)
{
    drop_carry(ctx);
    if (!ctx || !out) return DG_EINVAL;
    if (!ctx->state_set) return fail(ctx, DG_ESTATE, "dg_diagnostics: no state set");
    const void* u = ctx->reg[ctx->cur];
    const bool force = ctx->forcing_active;
    // abar of the current state first (into the control block), then the reductions
    CK(project(ctx, u, vh_buf(ctx, 0), force ? ctx->ahat : nullptr, false, 0));
    Launch L = make_launch(ctx);
    int flags = force ? F_FORCE : 0;
    Timed tm(ctx, KIND_OTHER);
    cudaError_t e = (ctx->prec == DG_PREC_F64)
                        ? launch_diag<double>(L, (const double*)u, (const double*)ctx->ahat, dt_for_pimax, flags)
                        : launch_diag<float>(L, (const float*)u, (const float*)ctx->ahat, dt_for_pimax, flags);
    CK(e);
    double d[16];
    CK(cudaMemcpyAsync(d, ctx->ctl->diag, sizeof(d), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    out->mass = d[0];
    for (int i = 0; i < 3; ++i) out->mom[i] = d[1 + i];
    out->ekin = d[4];
    out->mach = std::sqrt(d[5]) / ctx->cs;
    out->mach_rho = std::sqrt(2.0 * d[4] / d[0]) / ctx->cs;
    out->rho_min = d[7];
    out->rho_max = d[8];
    out->av_frac = d[9];
    out->inj_power = d[10];
    out->max_speed = d[11];
    out->av_work = d[12];
    out->status = ctx->status;
    out->t = ctx->t;
    out->steps = ctx->steps;
    return DG_OK;
}

int dg_l1_density(dg_ctx* ctx, const void* uA, const void* uB, double* out)
{
    if (!ctx || !uA || !uB || !out) return DG_EINVAL;
    Launch L = make_launch(ctx);
    Timed tm(ctx, KIND_OTHER);
    cudaError_t e = (ctx->prec == DG_PREC_F64) ? launch_l1<double>(L, (const double*)uA, (const double*)uB)
                                               : launch_l1<float>(L, (const float*)uA, (const float*)uB);
    CK(e);
    CK(cudaMemcpyAsync(out, &ctx->ctl->l1, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return DG_OK;
}

int dg_set_av_weights(dg_ctx* ctx, const float* w, size_t n)
{
    drop_carry(ctx);
    if (!ctx) return DG_EINVAL;
    if (!w || n != (size_t)ctx->mlp_P) return fail(ctx, DG_EINVAL, "dg_set_av_weights: need dg_av_param_count floats");
    const int rc = upload_weights(ctx, w);
    if (rc) return rc;
    CK(cudaMemsetAsync(ctx->mm, 0, sizeof(float) * ctx->mlp_P, ctx->st));
    CK(cudaMemsetAsync(ctx->mv, 0, sizeof(float) * ctx->mlp_P, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    ctx->adam_t = 0;
    return DG_OK;
}

int dg_get_av_weights(dg_ctx* ctx, float* w, size_t n)
{
    if (!ctx) return DG_EINVAL;
    if (!w || n != (size_t)ctx->mlp_P) return fail(ctx, DG_EINVAL, "dg_get_av_weights: bad size");
    CK(cudaMemcpyAsync(w, ctx->mw, sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return DG_OK;
}

int dg_av_param_count(dg_ctx* ctx, int64_t* n)
{
    if (!ctx || !n) return DG_EINVAL;
    *n = ctx->mlp_P;
    return DG_OK;
}

int dg_mlp_forward(dg_ctx* ctx, const float* x, int64_t n, float* y)
{
    drop_carry(ctx);
    if (!ctx) return DG_EINVAL;
    if (!x || !y || n < 1) return fail(ctx, DG_EINVAL, "dg_mlp_forward: bad arguments");
    if (!ctx->weights_set) return fail(ctx, DG_ESTATE, "dg_mlp_forward: no weights");
    Launch L = make_launch(ctx);
    {
        Timed tm(ctx, KIND_OTHER);
        CK(mlp_infer<float>(L, nullptr, nullptr, x, (long)n, ctx->mpack, nullptr, y));
    }
    CK(cudaStreamSynchronize(ctx->st));
    return DG_OK;
}

int dg_mlp_grad(dg_ctx* ctx, const float* x, const float* y, int64_t n, float* grad, double* loss)
{
    drop_carry(ctx);
    if (!ctx) return DG_EINVAL;
    if (!x || !y || !grad || !loss || n < 1 || n > kMlpBatchMax) return fail(ctx, DG_EINVAL, "dg_mlp_grad: bad arguments");
    if (!ctx->weights_set) return fail(ctx, DG_ESTATE, "dg_mlp_grad: no weights");
    {
        Timed tm(ctx, KIND_OTHER);
        CK(mlp_train_pass(ctx->st, ctx->mlp_D, ctx->mw, x, y, (int)n, ctx->mwork, ctx->mg, ctx->mloss));
    }
    CK(cudaMemcpyAsync(grad, ctx->mg, sizeof(float) * ctx->mlp_P, cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(loss, ctx->mloss, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return DG_OK;
}

int dg_mlp_train(dg_ctx* ctx, const float* x, const float* y, int64_t n, const dg_train_opts* o, double* loss_out)
{
    drop_carry(ctx);
    if (!ctx) return DG_EINVAL;
    if (!x || !y || !o || n < 1 || o->batch < 1 || o->batch > kMlpBatchMax || o->epochs < 1)
        return fail(ctx, DG_EINVAL, "dg_mlp_train: bad arguments");
    if (!ctx->weights_set) return fail(ctx, DG_ESTATE, "dg_mlp_train: initialise the weights first");
    const int D = ctx->mlp_D;
    double last = 0.0;
    std::vector<double> losses;
    for (int ep = 0; ep < o->epochs; ++ep) {
        losses.clear();
        for (int64_t s0 = 0; s0 < n; s0 += o->batch) {
            const int nb = (int)std::min<int64_t>(o->batch, n - s0);
            CK(mlp_train_pass(ctx->st, D, ctx->mw, x + s0 * D, y + s0, nb, ctx->mwork, ctx->mg, ctx->mloss));
            ctx->adam_t += 1;
            const float c1 = (float)(1.0 / (1.0 - std::pow(o->beta1, (double)ctx->adam_t)));
            const float c2 = (float)(1.0 / (1.0 - std::pow(o->beta2, (double)ctx->adam_t)));
            CK(mlp_adam(ctx->st, ctx->mlp_P, ctx->mw, ctx->mg, ctx->mm, ctx->mv, (float)o->lr, (float)o->beta1,
                        (float)o->beta2, (float)o->eps, c1, c2));
            double l = 0.0;
            CK(cudaMemcpyAsync(&l, ctx->mloss, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
            CK(cudaStreamSynchronize(ctx->st));
            losses.push_back(l);
        }
        double sum = 0.0;
        for (double l : losses) sum += l;
        last = sum / losses.size();
    }
    // refresh the packed inference weights from the trained master copy
    std::vector<float> w(ctx->mlp_P);
    CK(cudaMemcpyAsync(w.data(), ctx->mw, sizeof(float) * ctx->mlp_P, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    const int rc = upload_weights(ctx, w.data());
    if (rc) return rc;
    if (loss_out) *loss_out = last;
    return DG_OK;
}

int dg_generate_pairs(dg_ctx* ctx, double dt_for_pimax, float* x, float* y, int64_t cap, int64_t* n_out)
{
    drop_carry(ctx);
    if (!ctx) return DG_EINVAL;
    if (!x || !y || !n_out) return fail(ctx, DG_EINVAL, "dg_generate_pairs: null buffer");
    if (!ctx->state_set) return fail(ctx, DG_ESTATE, "dg_generate_pairs: no state set");
    if (cap < ctx->ncell) return fail(ctx, DG_ENOMEM, "dg_generate_pairs: cap < number of cells");
    if (ctx->nu.mode != DG_AV_LEARNED)
        return fail(ctx, DG_EINVAL, "dg_generate_pairs: needs a context created in DG_AV_LEARNED mode");
    const void* u = ctx->reg[ctx->cur];
    TileLaunch t{};
    t.mode = 0;
    t.u_in = u;
    t.vh_out = vh_buf(ctx, 1);
    t.vabs_out = ctx->vabs;
    t.flags = F_VABS;
    t.abar_out = 1;
    CK(tile(ctx, t));
    Launch L = make_launch(ctx);
    {
        Timed tm(ctx, KIND_OTHER);
        const char* tt = (const char*)ctx->ttab;
        if (ctx->prec == DG_PREC_F64) {
            const double* phiv = (const double*)tt + (ctx->K == 1   ? TileTab<1, BK_FMA>::phiv
                                                      : ctx->K == 2 ? TileTab<2, BK_FMA>::phiv
                                                                    : TileTab<3, BK_FMA>::phiv);
            CK(launch_features<double>(L, (const double*)u, (const double*)ctx->vabs, phiv, dt_for_pimax, x, y));
        } else {
            const bool x3 = ctx->prec == DG_PREC_X3;
            const int off = ctx->K == 1 ? (x3 ? TileTab<1, BK_X3>::phiv : TileTab<1, BK_FMA>::phiv)
                            : ctx->K == 2 ? (x3 ? TileTab<2, BK_X3>::phiv : TileTab<2, BK_FMA>::phiv)
                                          : (x3 ? TileTab<3, BK_X3>::phiv : TileTab<3, BK_FMA>::phiv);
            const float* phiv = (const float*)tt + off;
            CK(launch_features<float>(L, (const float*)u, (const float*)ctx->vabs, phiv, dt_for_pimax, x, y));
        }
    }
    CK(cudaStreamSynchronize(ctx->st));
    *n_out = ctx->ncell;
    return DG_OK;
}

int dg_av_nu_carried(dg_ctx* ctx, float* nu_out)
{
    if (!ctx) return DG_EINVAL;
    if (!nu_out) return fail(ctx, DG_EINVAL, "dg_av_nu_carried: null buffer");
    if (ctx->nu.mode != DG_AV_LEARNED || !ctx->carry)
        return fail(ctx, DG_ESTATE, "dg_av_nu_carried: no coefficient carried from a learned step");
    if (!ctx->nu.fused_infer) CK(learned_infer(ctx, ctx->reg[ctx->cur]));
    const float* src = ctx->nu.fused_infer ? ctx->nu_next : ctx->nu_cell;
    CK(cudaMemcpyAsync(nu_out, src, sizeof(float) * ctx->ncell, cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return DG_OK;
}

int dg_av_nu(dg_ctx* ctx, float* nu_out)
{
    drop_carry(ctx);
    if (!ctx) return DG_EINVAL;
    if (!nu_out) return fail(ctx, DG_EINVAL, "dg_av_nu: null buffer");
    if (ctx->nu.mode != DG_AV_LEARNED || !ctx->weights_set)
        return fail(ctx, DG_ESTATE, "dg_av_nu: needs learned mode with weights");
    if (!ctx->state_set) return fail(ctx, DG_ESTATE, "dg_av_nu: no state set");
    CK(learned_nu(ctx, ctx->reg[ctx->cur]));
    CK(cudaMemcpyAsync(nu_out, ctx->nu_cell, sizeof(float) * ctx->ncell, cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return DG_OK;
}

int dg_profile(dg_ctx* ctx, int enable)
{
    if (!ctx) return DG_EINVAL;
    CK(cudaStreamSynchronize(ctx->st));
    for (auto& p : ctx->pending) {
        ctx->pool.push_back(p.a);
        ctx->pool.push_back(p.b);
    }
    ctx->pending.clear();
    ctx->counts = dg_prof{};
    ctx->prof = enable != 0;
    CK(cudaMemsetAsync(&ctx->ctl->tiles_vol, 0, 2 * sizeof(unsigned long long), ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return DG_OK;
}

int dg_profile_read(dg_ctx* ctx, dg_prof* out)
{
    if (!ctx || !out) return DG_EINVAL;
    CK(cudaStreamSynchronize(ctx->st));
    for (auto& p : ctx->pending) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, p.a, p.b));
        if (p.kind == KIND_PROJECT) ctx->counts.ms_project += ms;
        if (p.kind == KIND_RHS) ctx->counts.ms_rhs += ms;
        if (p.kind == KIND_FORCE) ctx->counts.ms_force += ms;
        if (p.kind == KIND_OTHER) ctx->counts.ms_other += ms;
        ctx->pool.push_back(p.a);
        ctx->pool.push_back(p.b);
    }
    ctx->pending.clear();
    unsigned long long tiles[2] = {0ull, 0ull};
    CK(cudaMemcpy(tiles, &ctx->ctl->tiles_vol, sizeof(tiles), cudaMemcpyDeviceToHost));
    ctx->counts.tiles_volume = (int64_t)tiles[0];
    ctx->counts.tiles_gated = (int64_t)tiles[1];
    *out = ctx->counts;
    return DG_OK;
}

int dg_get_meta(dg_ctx* ctx, dg_meta* m)
{
    if (!ctx || !m) return DG_EINVAL;
    std::memset(m, 0, sizeof(*m));
    m->t = ctx->t;
    m->steps = ctx->steps;
    m->dt_last = ctx->dt_last;
    m->forcing_on = ctx->drv.on ? 1 : 0;
    m->forcing_dirty = ctx->drv.dirty ? 1 : 0;
    m->t_next = ctx->drv.t_next;
    m->rng = ctx->drv.rng;
    m->have_spare = ctx->drv.have_spare ? 1 : 0;
    m->spare = ctx->drv.spare;
    m->nmodes = ctx->drv.nm;
    std::memcpy(m->x, ctx->drv.x, sizeof(double) * 6 * ctx->drv.nm);
    return DG_OK;
}

int dg_set_meta(dg_ctx* ctx, const dg_meta* m)
{
    drop_carry(ctx);
    if (!ctx || !m) return DG_EINVAL;
    if (m->nmodes != ctx->drv.nm) return fail(ctx, DG_EINVAL, "dg_set_meta: call dg_set_forcing with the same modes first");
    ctx->t = m->t;
    ctx->steps = m->steps;
    ctx->dt_last = m->dt_last;
    ctx->drv.on = m->forcing_on != 0;
    ctx->drv.t_next = m->t_next;
    ctx->drv.rng = m->rng;
    ctx->drv.have_spare = m->have_spare != 0;
    ctx->drv.spare = m->spare;
    std::memcpy(ctx->drv.x, m->x, sizeof(double) * 6 * m->nmodes);
    // re-project the current OU amplitudes before the next step
    ctx->drv.dirty = ctx->drv.on;
    if (!ctx->drv.on) ctx->forcing_active = false;
    return DG_OK;
}


// ---------------------------------------------------------------------------
// turbulence statistics
// ---------------------------------------------------------------------------
int dg_density_pdf(dg_ctx* ctx, double lo, double hi, int nbins, double* hist)
{
    if (!ctx) return DG_EINVAL;
    if (!hist || nbins < 1 || nbins > DG_MAX_BINS || !(hi > lo))
        return fail(ctx, DG_EINVAL, "dg_density_pdf: bad bins or null buffer");
    if (!ctx->state_set) return fail(ctx, DG_ESTATE, "dg_density_pdf: no state set");
    double* acc = ctx->ana;
    double* mean = ctx->ana + 4 * DG_MAX_BINS;
    CK(cudaMemsetAsync(ctx->ana, 0, sizeof(double) * (4 * DG_MAX_BINS + 1), ctx->st));
    Launch L = make_launch(ctx);
    {
        Timed tm(ctx, KIND_OTHER);
        const void* u = ctx->reg[ctx->cur];
        CK(ctx->prec == DG_PREC_F64 ? launch_density_pdf<double>(L, (const double*)u, lo, hi, nbins, mean, acc)
                                    : launch_density_pdf<float>(L, (const float*)u, lo, hi, nbins, mean, acc));
    }
    CK(cudaMemcpyAsync(hist, acc, sizeof(double) * nbins, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return DG_OK;
}

int dg_structure_function(dg_ctx* ctx, int nbins, int64_t npairs, uint64_t seed, double* l, double* v)
{
    if (!ctx) return DG_EINVAL;
    if (!l || !v || nbins < 1 || nbins > DG_MAX_BINS || npairs < 1 || npairs > (int64_t(1) << 40) / nbins)
        return fail(ctx, DG_EINVAL, "dg_structure_function: bad bins, pair count or null buffer");
    if (!ctx->state_set) return fail(ctx, DG_ESTATE, "dg_structure_function: no state set");
    double* acc = ctx->ana;
    CK(cudaMemsetAsync(acc, 0, sizeof(double) * nbins, ctx->st));
    Launch L = make_launch(ctx);
    {
        Timed tm(ctx, KIND_OTHER);
        const void* u = ctx->reg[ctx->cur];
        CK(ctx->prec == DG_PREC_F64
               ? launch_structure<double>(L, (const double*)u, nbins, (long)npairs, (unsigned long long)seed, acc)
               : launch_structure<float>(L, (const float*)u, nbins, (long)npairs, (unsigned long long)seed, acc));
    }
    std::vector<double> a(nbins);
    CK(cudaMemcpyAsync(a.data(), acc, sizeof(double) * nbins, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    const double lmin = 1.0 / ((ctx->K + 1) * (double)ctx->N), lmax = 0.5;
    for (int j = 0; j < nbins; ++j) {
        l[j] = lmin * std::pow(lmax / lmin, (j + 0.5) / nbins);
        v[j] = std::sqrt(0.5 * a[j] / (double)npairs);
    }
    return DG_OK;
}

static size_t analysis_bytes(int Ng)
{
    const size_t n3 = (size_t)Ng * Ng * Ng, nc = (size_t)Ng * Ng * (Ng / 2 + 1);
    return align256(sizeof(double) * n3) + 2 * sizeof(double) * nc;
}

int dg_analysis_bytes(const dg_mesh* mesh, int order, size_t* bytes)
{
    if (!mesh || !bytes || order < 1 || order > 3 || mesh->n[0] < 1) return DG_EINVAL;
    *bytes = analysis_bytes((order + 1) * mesh->n[0]);
    return DG_OK;
}

int dg_power_spectrum(dg_ctx* ctx, void* work, size_t work_bytes, int nbins, double* kmean, double* power,
                      int64_t* count)
{
    if (!ctx) return DG_EINVAL;
    if (!kmean || !power || !count || !work || nbins < 1 || nbins > DG_MAX_BINS)
        return fail(ctx, DG_EINVAL, "dg_power_spectrum: bad bins or null buffer");
    if (((uintptr_t)work) & 255u) return fail(ctx, DG_EINVAL, "dg_power_spectrum: work not 256-byte aligned");
    const int Ng = (ctx->K + 1) * ctx->N;
    if (work_bytes < analysis_bytes(Ng)) return fail(ctx, DG_ENOMEM, "dg_power_spectrum: work buffer too small");
    if (!ctx->state_set) return fail(ctx, DG_ESTATE, "dg_power_spectrum: no state set");
    const CufftApi& fft = cufft_api();
    if (!fft.ok) return fail(ctx, DG_ECUDA, "dg_power_spectrum: cuFFT library not found");
    if (ctx->fft_ng != Ng) {
        if (ctx->fft_ng > 0) fft.destroy(ctx->fft);
        ctx->fft_ng = 0;
        if (fft.plan3d(&ctx->fft, Ng, Ng, Ng, CUFFT_D2Z) != CUFFT_SUCCESS)
            return fail(ctx, DG_ECUDA, "dg_power_spectrum: cuFFT plan failed");
        ctx->fft_ng = Ng;
    }
    if (fft.set_stream(ctx->fft, ctx->st) != CUFFT_SUCCESS) return fail(ctx, DG_ECUDA, "dg_power_spectrum: cuFFT stream");
    double* grid = static_cast<double*>(work);
    void* F = static_cast<char*>(work) + align256(sizeof(double) * (size_t)Ng * Ng * Ng);
    double* pw = ctx->ana;
    double* ks = ctx->ana + DG_MAX_BINS;
    unsigned long long* cn = reinterpret_cast<unsigned long long*>(ctx->ana + 2 * DG_MAX_BINS);
    CK(cudaMemsetAsync(ctx->ana, 0, sizeof(double) * 3 * DG_MAX_BINS, ctx->st));
    Launch L = make_launch(ctx);
    const double n3 = (double)Ng * Ng * Ng;
    const void* u = ctx->reg[ctx->cur];
    for (int d = 0; d < 3; ++d) {
        {
            Timed tm(ctx, KIND_OTHER);
            CK(ctx->prec == DG_PREC_F64 ? launch_sample<double>(L, (const double*)u, d, grid)
                                        : launch_sample<float>(L, (const float*)u, d, grid));
        }
        if (fft.exec_d2z(ctx->fft, grid, static_cast<cufftDoubleComplex*>(F)) != CUFFT_SUCCESS)
            return fail(ctx, DG_ECUDA, "dg_power_spectrum: cuFFT execution failed");
        Timed tm(ctx, KIND_OTHER);
        CK(launch_shell(L, F, Ng, nbins, 1.0 / (n3 * n3), d == 0, pw, ks, cn));
    }
    std::vector<double> hp(nbins), hk(nbins);
    std::vector<unsigned long long> hc(nbins);
    CK(cudaMemcpyAsync(hp.data(), pw, sizeof(double) * nbins, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(hk.data(), ks, sizeof(double) * nbins, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaMemcpyAsync(hc.data(), cn, sizeof(unsigned long long) * nbins, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    for (int i = 0; i < nbins; ++i) {
        power[i] = hp[i];
        count[i] = (int64_t)hc[i];
        kmean[i] = hc[i] ? hk[i] / (double)hc[i] : 0.0;
    }
    return DG_OK;
}

}  // extern "C"

// ===========================================================================
// adiabatic system (Sec. 2.1): five conserved variables, ideal-gas equation
// of state; the same basis, tables, quadrature and SSP-RK schemes
// ===========================================================================
struct dg_adi_ctx {
    int N = 0, K = 0, b = 0, prec = DG_PREC_F32, rk = 3, riemann = DG_RIEMANN_RUSANOV;
    long ncell = 0;
    double h = 0.0, gamma = 1.4, cfl = 0.3;
    dg_nu_params nu{};
    cudaStream_t st = nullptr;
    void* reg[3] = {nullptr, nullptr, nullptr};
    int cur = 0;
    void* prim = nullptr;
    void* prim2 = nullptr;  // second projection buffer (scratch)
    void* ahat = nullptr;   // driving a_h [c][3][b] (scratch)
    int* d_kvec = nullptr;
    double* d_amp = nullptr;
    void* gtab = nullptr;
    Rule1 r1{};
    Driver drv;
    bool forcing_active = false;
    double cs_ref = 0.0;    // sound speed the driving is scaled with
    double cs_reset = 0.0;  // > 0: uniform temperature restored after every step
    double kap = 0.0;       // energy offset of the stored state (e_s = e - kap rho): cs_reset^2/(gamma - 1)
    int bc[3] = {DG_BC_PERIODIC, DG_BC_PERIODIC, DG_BC_PERIODIC};  // boundaries per axis
    double inflow[5] = {1.0, 0.0, 0.0, 0.0, 1.0};                   // DG_BC_INFLOW state (rho, v, p)
    double injected = 0.0, dissipated = 0.0;
    char* scratch = nullptr;
    Ctl* ctl = nullptr;
    void* ttab = nullptr;
    double* partials = nullptr;
    int nsm = 1;
    bool state_set = false;
    double t = 0.0, dt_last = 0.0;
    long steps = 0;
    unsigned int status = 0u;
    std::string err;
};

namespace {

int afail(dg_adi_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg;
    return code;
}

#define ACK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return afail(ctx, DG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
    } while (0)

struct AdiScratch {
    size_t ctl, ttab, partials, prim2, ahat, kvec, amp, gtab, total;
};

// control block, tables, reduction partials, the second projection buffer
// (stages alternate between it and the caller's), the driving a_h and the
// forcing projection's mode list, amplitudes and 1D factors
AdiScratch adi_scratch(int K, int N, size_t elem)
{
    const size_t nc = (size_t)N * N * N, b = (size_t)(K + 1) * (K + 2) * (K + 3) / 6;
    AdiScratch s{};
    size_t off = 0;
    s.ctl = off;
    off = align256(off + sizeof(Ctl));
    s.ttab = off;
    off = align256(off + sizeof(double) * ttab_total(K));
    s.partials = off;
    off = align256(off + sizeof(double) * 16 * kMaxGrid);
    s.prim2 = off;
    off = align256(off + nc * 4 * b * elem);
    s.ahat = off;
    off = align256(off + nc * 3 * b * elem);
    s.kvec = off;
    off = align256(off + sizeof(int) * 3 * kMaxModes);
    s.amp = off;
    off = align256(off + sizeof(double) * 6 * kMaxModes);
    s.gtab = off;
    off = align256(off + sizeof(double) * 2 * (size_t)N * kForceNK * (K + 1));
    s.total = off;
    return s;
}

size_t adi_elem(const dg_adi_ctx* c) { return c->prec == DG_PREC_F64 ? sizeof(double) : sizeof(float); }
size_t adi_state_bytes(const dg_adi_ctx* c) { return adi_elem(c) * (size_t)c->ncell * 5 * c->b; }

Launch adi_make_launch(const dg_adi_ctx* c)
{
    Launch L{};
    L.st = c->st;
    L.K = c->K;
    L.N = c->N;
    L.ncell = c->ncell;
    L.ph.h = c->h;
    L.ph.hp = c->h / (c->K + 1);
    L.ph.alpha = c->nu.alpha;
    L.ph.beta = c->nu.beta;
    L.ph.floor_ = c->nu.rho_floor;
    L.ph.av_mode = c->nu.mode;
    L.ph.riemann = c->riemann;
    L.ttab = c->ttab;
    L.ctl = c->ctl;
    L.partials = c->partials;
    L.nsm = c->nsm;
    L.bk = 0;
    L.r1 = c->r1;
    L.gtab = c->gtab;
    return L;
}

cudaError_t adi_go(const dg_adi_ctx* c, const AdiLaunch& t)
{
    const Launch L = adi_make_launch(c);
    AdiLaunch u = t;
    u.kap = c->kap;
    for (int i = 0; i < 3; ++i) u.bc[i] = c->bc[i];
    for (int i = 0; i < 5; ++i) u.inflow[i] = c->inflow[i];
    return c->prec == DG_PREC_F64 ? launch_adi<double>(L, c->gamma, u) : launch_adi<float>(L, c->gamma, u);
}

}  // namespace

extern "C" {

int dg_adi_buffer_bytes(const dg_mesh* mesh, int order, int precision, size_t* state_bytes, size_t* prim_bytes,
                        size_t* scratch_bytes)
{
    if (!mesh || order < 1 || order > 3 || (precision != DG_PREC_F32 && precision != DG_PREC_F64)) return DG_EINVAL;
    if (!cubic_mesh(mesh)) return DG_EINVAL;
    const size_t n = (size_t)mesh->n[0] * mesh->n[1] * mesh->n[2];
    const size_t b = (size_t)(order + 1) * (order + 2) * (order + 3) / 6;
    const size_t el = precision == DG_PREC_F64 ? sizeof(double) : sizeof(float);
    if (state_bytes) *state_bytes = n * 5 * b * el;
    if (prim_bytes) *prim_bytes = n * 4 * b * el;
    if (scratch_bytes) *scratch_bytes = adi_scratch(order, mesh->n[0], el).total;
    return DG_OK;
}

int dg_adi_init(dg_adi_ctx** out, const dg_mesh* mesh, int order, const dg_nu_params* nu, const dg_adi_opts* opts)
{
    if (!out) return DG_EINVAL;
    *out = nullptr;
    if (!mesh || !nu || !opts) return DG_EINVAL;
    if (order < 1 || order > 3) return DG_EINVAL;
    if (!cubic_mesh(mesh)) return DG_EINVAL;
    for (int d = 0; d < 3; ++d)
        if (mesh->L[d] != 1.0) return DG_EINVAL;
    if (nu->mode < 0 || nu->mode > 1 || !(nu->rho_floor >= 0.0) || nu->diffusion != 0.0) return DG_EINVAL;
    if (opts->precision != DG_PREC_F32 && opts->precision != DG_PREC_F64) return DG_EINVAL;
    if (opts->rk_stages != 2 && opts->rk_stages != 3) return DG_EINVAL;
    if (opts->riemann != DG_RIEMANN_RUSANOV && opts->riemann != DG_RIEMANN_HLLC) return DG_EINVAL;
    if (!(opts->cfl > 0.0) || !(opts->gamma > 1.0) || !opts->stream || !opts->prim || !opts->scratch) return DG_EINVAL;
    bool inflow_used = false;
    for (int d = 0; d < 3; ++d) {
        if (opts->bc[d] < DG_BC_PERIODIC || opts->bc[d] > DG_BC_INFLOW) return DG_EINVAL;
        inflow_used |= opts->bc[d] == DG_BC_INFLOW;
    }
    if (inflow_used) {
        for (int i = 0; i < 5; ++i)
            if (!std::isfinite(opts->inflow[i])) return DG_EINVAL;
        if (!(opts->inflow[0] > 0.0) || !(opts->inflow[4] > 0.0)) return DG_EINVAL;
    }
    for (int i = 0; i < 3; ++i)
        if (!opts->u[i]) return DG_EINVAL;
    const AdiScratch sl =
        adi_scratch(order, mesh->n[0], opts->precision == DG_PREC_F64 ? sizeof(double) : sizeof(float));
    if (opts->scratch_bytes < sl.total) return DG_ENOMEM;
    if (((uintptr_t)opts->scratch & 255u) != 0) return DG_EINVAL;
    dg_adi_ctx* ctx = new (std::nothrow) dg_adi_ctx();
    if (!ctx) return DG_ENOMEM;
    ctx->N = mesh->n[0];
    ctx->K = order;
    ctx->b = (order + 1) * (order + 2) * (order + 3) / 6;
    ctx->prec = opts->precision;
    ctx->rk = opts->rk_stages;
    ctx->riemann = opts->riemann;
    for (int d = 0; d < 3; ++d) ctx->bc[d] = opts->bc[d];
    for (int q = 0; q < 5; ++q) ctx->inflow[q] = opts->inflow[q];
    ctx->ncell = (long)ctx->N * ctx->N * ctx->N;
    ctx->h = 1.0 / ctx->N;
    ctx->gamma = opts->gamma;
    ctx->cfl = opts->cfl;
    ctx->nu = *nu;
    ctx->st = static_cast<cudaStream_t>(opts->stream);
    for (int i = 0; i < 3; ++i) ctx->reg[i] = opts->u[i];
    ctx->prim = opts->prim;
    ctx->scratch = static_cast<char*>(opts->scratch);
    ctx->ctl = reinterpret_cast<Ctl*>(ctx->scratch + sl.ctl);
    ctx->ttab = ctx->scratch + sl.ttab;
    ctx->partials = reinterpret_cast<double*>(ctx->scratch + sl.partials);
    ctx->prim2 = ctx->scratch + sl.prim2;
    ctx->ahat = ctx->scratch + sl.ahat;
    ctx->d_kvec = reinterpret_cast<int*>(ctx->scratch + sl.kvec);
    ctx->d_amp = reinterpret_cast<double*>(ctx->scratch + sl.amp);
    ctx->gtab = ctx->scratch + sl.gtab;
    {
        long double xg[4], wg[4];
        gauss_rule(order + 1, xg, wg);
        for (int q = 0; q <= order; ++q) {
            ctx->r1.x[q] = (double)xg[q];
            ctx->r1.w[q] = (double)wg[q];
        }
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, dev);
    const std::vector<char> tt = tile_tables_for(order, ctx->prec);
    Ctl c0{};
    c0.dt_scale = 1.0;
    c0.dt_num = ctx->cfl * ctx->h / (ctx->K + 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->ttab, tt.data(), tt.size(), cudaMemcpyHostToDevice, ctx->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->ctl, &c0, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ctx->ahat, 0, (size_t)ctx->ncell * 3 * ctx->b * adi_elem(ctx), ctx->st);
    if (e == cudaSuccess) e = (ctx->prec == DG_PREC_F64) ? setup_kernels<double>(order) : setup_kernels<float>(order);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    if (e != cudaSuccess) {
        delete ctx;
        return DG_ECUDA;
    }
    *out = ctx;
    return DG_OK;
}

void dg_adi_free(dg_adi_ctx* ctx) { delete ctx; }

const char* dg_adi_last_error(const dg_adi_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int dg_adi_set_state(dg_adi_ctx* ctx, const void* src, int src_on_host)
{
    if (!ctx) return DG_EINVAL;
    if (!src) return afail(ctx, DG_EINVAL, "dg_adi_set_state: null source");
    ctx->cur = 0;
    ACK(cudaMemcpyAsync(ctx->reg[0], src, adi_state_bytes(ctx),
                        src_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, ctx->st));
    ACK(cudaStreamSynchronize(ctx->st));
    ctx->state_set = true;
    ctx->t = 0.0;
    ctx->steps = 0;
    ctx->status = 0u;
    ctx->injected = 0.0;
    ctx->dissipated = 0.0;
    return DG_OK;
}

int dg_adi_get_state(dg_adi_ctx* ctx, void* dst, int to_host)
{
    if (!ctx) return DG_EINVAL;
    if (!dst) return afail(ctx, DG_EINVAL, "dg_adi_get_state: null destination");
    if (!ctx->state_set) return afail(ctx, DG_ESTATE, "dg_adi_get_state: no state set");
    ACK(cudaMemcpyAsync(dst, ctx->reg[ctx->cur], adi_state_bytes(ctx),
                        to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, ctx->st));
    ACK(cudaStreamSynchronize(ctx->st));
    return DG_OK;
}

int dg_adi_project(dg_adi_ctx* ctx, const void* u_in, void* prim_out)
{
    if (!ctx) return DG_EINVAL;
    if (!u_in || !prim_out) return afail(ctx, DG_EINVAL, "dg_adi_project: null buffer");
    AdiLaunch p{};
    p.mode = ADI_PROJECT;
    p.u_in = u_in;
    p.pr_out = prim_out;
    ACK(adi_go(ctx, p));
    ACK(cudaStreamSynchronize(ctx->st));
    return DG_OK;
}

int dg_adi_rhs(dg_adi_ctx* ctx, const void* u_in, void* dudt, double dt_pimax)
{
    if (!ctx) return DG_EINVAL;
    if (!u_in || !dudt) return afail(ctx, DG_EINVAL, "dg_adi_rhs: null buffer");
    if (!(dt_pimax >= 0.0)) return afail(ctx, DG_EINVAL, "dg_adi_rhs: negative dt");
    AdiLaunch p{};
    p.mode = ADI_PROJECT;
    p.u_in = u_in;
    p.pr_out = ctx->prim;
    ACK(adi_go(ctx, p));
    AdiLaunch r{};
    r.mode = ADI_RHS;
    r.u_in = u_in;
    r.out = dudt;
    r.pr_in = ctx->prim;
    r.dt_pimax = dt_pimax;
    ACK(adi_go(ctx, r));
    ACK(cudaStreamSynchronize(ctx->st));
    return DG_OK;
}

int dg_adi_step(dg_adi_ctx* ctx, int nsteps, double fixed_dt, double* t_out, double* dt_last)
{
    if (!ctx) return DG_EINVAL;
    if (nsteps < 0 || !(fixed_dt >= 0.0)) return afail(ctx, DG_EINVAL, "dg_adi_step: bad arguments");
    if (!ctx->state_set) return afail(ctx, DG_ESTATE, "dg_adi_step: no state set");
    static const double W2[2] = {0.5, 0.5}, W3[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
    const double* RW = ctx->rk == 2 ? W2 : W3;
    const size_t ahat_bytes = (size_t)ctx->ncell * 3 * ctx->b * adi_elem(ctx);
    for (int n = 0; n < nsteps; ++n) {
        // driving schedule (Sec. 4.2): OU updates every dt_drive, switched off after t_off
        if (ctx->drv.on && ctx->drv.t_off > 0.0 && ctx->t > ctx->drv.t_off) {
            ctx->drv.on = false;
            ctx->forcing_active = false;
            ACK(cudaMemsetAsync(ctx->ahat, 0, ahat_bytes, ctx->st));
        }
        if (ctx->drv.on) {
            while (ctx->t >= ctx->drv.t_next) {
                ctx->drv.advance();
                ctx->drv.t_next += ctx->drv.dtd;
                ctx->drv.dirty = true;
            }
            if (ctx->drv.dirty) {
                std::vector<double> amp;
                std::vector<int> kv;
                ctx->drv.amplitudes(amp, kv);
                ACK(cudaMemcpyAsync(ctx->d_kvec, kv.data(), sizeof(int) * kv.size(), cudaMemcpyHostToDevice, ctx->st));
                ACK(cudaMemcpyAsync(ctx->d_amp, amp.data(), sizeof(double) * amp.size(), cudaMemcpyHostToDevice,
                                    ctx->st));
                const Launch L = adi_make_launch(ctx);
                ACK(ctx->prec == DG_PREC_F64 ? launch_force<double>(L, ctx->drv.nm, ctx->d_kvec, ctx->d_amp,
                                                                    ctx->drv.kmaxc, (double*)ctx->ahat)
                                             : launch_force<float>(L, ctx->drv.nm, ctx->d_kvec, ctx->d_amp,
                                                                   ctx->drv.kmaxc, (float*)ctx->ahat));
                ACK(cudaStreamSynchronize(ctx->st));  // the host amplitude buffers are reused
                ctx->drv.dirty = false;
                ctx->forcing_active = true;
            }
        }
        const bool force = ctx->forcing_active;
        const int A = ctx->cur, B = (ctx->cur + 1) % 3, C = (ctx->cur + 2) % 3;
        const int in3[3] = {A, B, C}, out3[3] = {B, C, B};
        const int in2[2] = {A, B}, out2[2] = {B, C};
        const int* in = ctx->rk == 2 ? in2 : in3;
        const int* out = ctx->rk == 2 ? out2 : out3;
        bool ok = false;
        unsigned int status = 0u;
        double dt = 0.0, inj = 0.0;
        for (int retry = 0; retry <= 3 && !ok; ++retry) {
            struct {
                double dt_scale, fixed_dt;
            } hs = {1.0 / (double)(1 << retry), fixed_dt};
            ACK(cudaMemcpyAsync(&ctx->ctl->dt_scale, &hs, sizeof(hs), cudaMemcpyHostToDevice, ctx->st));
            ACK(cudaMemsetAsync(&ctx->ctl->status, 0, sizeof(unsigned int), ctx->st));
            ACK(cudaMemsetAsync(&ctx->ctl->smax, 0, sizeof(unsigned long long), ctx->st));
            ACK(cudaMemsetAsync(&ctx->ctl->diag[1], 0, sizeof(double), ctx->st));
            // projections of v and p of u^n (with its CFL bound); every stage but the
            // last projects its output for the next one (alternating buffers)
            void* pr[2] = {ctx->prim, ctx->prim2};
            AdiLaunch p{};
            p.mode = ADI_PROJECT;
            p.u_in = ctx->reg[A];
            p.pr_out = pr[0];
            p.flags = F_DT | (force ? F_FORCE : 0);
            p.ahat = ctx->ahat;
            p.abar_out = 0;
            ACK(adi_go(ctx, p));
            for (int s = 0; s < ctx->rk; ++s) {
                AdiLaunch t{};
                t.mode = ADI_STAGE;
                t.u_in = ctx->reg[in[s]];
                t.u_n = ctx->reg[A];
                t.out = ctx->reg[out[s]];
                t.pr_in = pr[s & 1];
                t.pr_out = pr[(s + 1) & 1];
                t.flags = (s + 1 < ctx->rk ? F_NEXTPROJ : 0) | (force ? F_FORCE : 0);
                t.ahat = ctx->ahat;
                t.abar_in = s & 1;
                t.abar_out = (s + 1) & 1;
                t.beta = RW[s];
                rk_weights(ctx->rk, s, ctx->prec != DG_PREC_F64, t.rk_a, t.rk_b);
                ACK(adi_go(ctx, t));
            }
            struct {
                unsigned int status;
                double dt, inj;
            } back{};
            ACK(cudaMemcpyAsync(&back.status, &ctx->ctl->status, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->st));
            ACK(cudaMemcpyAsync(&back.dt, &ctx->ctl->dt, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
            ACK(cudaMemcpyAsync(&back.inj, &ctx->ctl->diag[1], sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
            ACK(cudaStreamSynchronize(ctx->st));
            status = back.status;
            dt = back.dt;
            inj = back.inj;
            ok = !(status & DG_ST_FAIL);
        }
        ctx->status |= status;
        if (!ok) return afail(ctx, DG_EPOSITIVITY, "dg_adi_step: positivity retries exhausted");
        ctx->cur = out[ctx->rk - 1];
        if (force) ctx->injected += inj;
        if (ctx->cs_reset > 0.0) {
            // uniform temperature restored; the thermal energy taken out is the dissipation
            ACK(cudaMemsetAsync(&ctx->ctl->diag[2], 0, sizeof(double), ctx->st));
            AdiLaunch r{};
            r.mode = ADI_RESET;
            r.u_in = ctx->reg[ctx->cur];
            r.out = ctx->reg[ctx->cur];
            r.cs_reset = ctx->cs_reset;
            ACK(adi_go(ctx, r));
            double d = 0.0;
            ACK(cudaMemcpyAsync(&d, &ctx->ctl->diag[2], sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
            ACK(cudaStreamSynchronize(ctx->st));
            ctx->dissipated += d;
        }
        ctx->t += dt;
        ctx->dt_last = dt;
        ctx->steps += 1;
        if (status & DG_ST_NONFINITE) return afail(ctx, DG_ENONFINITE, "dg_adi_step: non-finite coefficient");
    }
    if (t_out) *t_out = ctx->t;
    if (dt_last) *dt_last = ctx->dt_last;
    return DG_OK;
}

int dg_adi_set_forcing(dg_adi_ctx* ctx, const dg_forcing* f, double cs_ref)
{
    if (!ctx) return DG_EINVAL;
    if (!f) return afail(ctx, DG_EINVAL, "dg_adi_set_forcing: null");
    const size_t ahat_bytes = (size_t)ctx->ncell * 3 * ctx->b * adi_elem(ctx);
    if (!f->on) {
        ctx->drv.on = false;
        ctx->forcing_active = false;
        ACK(cudaMemsetAsync(ctx->ahat, 0, ahat_bytes, ctx->st));
        ACK(cudaStreamSynchronize(ctx->st));
        return DG_OK;
    }
    if (!(cs_ref > 0.0) || !(f->mach > 0.0) || f->kmin2 < 1 || f->kmax2 < f->kmin2 || f->kmax2 > 64 ||
        f->zeta < 0.0 || f->zeta > 1.0)
        return afail(ctx, DG_EINVAL, "dg_adi_set_forcing: bad parameters");
    ctx->drv.init(*f, cs_ref);
    if (ctx->drv.nm > kMaxModes) return afail(ctx, DG_EINVAL, "dg_adi_set_forcing: too many modes");
    ctx->cs_ref = cs_ref;
    ctx->forcing_active = false;
    return DG_OK;
}

int dg_adi_set_reset(dg_adi_ctx* ctx, double cs)
{
    if (!ctx) return DG_EINVAL;
    if (!(cs >= 0.0)) return afail(ctx, DG_EINVAL, "dg_adi_set_reset: negative sound speed");
    ctx->cs_reset = cs;
    // the energy offset of the stored state follows the reset's thermal energy; a
    // state already set is carried over to the new offset
    const double kap = cs > 0.0 ? cs * cs / (ctx->gamma - 1.0) : 0.0;
    if (ctx->state_set && kap != ctx->kap) {
        const Launch L = adi_make_launch(ctx);
        void* u = ctx->reg[ctx->cur];
        ACK(ctx->prec == DG_PREC_F64 ? launch_adi_shift<double>(L, u, ctx->kap - kap)
                                     : launch_adi_shift<float>(L, u, ctx->kap - kap));
        ACK(cudaStreamSynchronize(ctx->st));
    }
    ctx->kap = kap;
    return DG_OK;
}

int dg_adi_energy_budget(dg_adi_ctx* ctx, double* out)
{
    if (!ctx) return DG_EINVAL;
    if (!out) return afail(ctx, DG_EINVAL, "dg_adi_energy_budget: null output");
    out[0] = ctx->injected;
    out[1] = ctx->dissipated;
    return DG_OK;
}

int dg_adi_get_meta(dg_adi_ctx* ctx, dg_adi_meta* m)
{
    if (!ctx || !m) return DG_EINVAL;
    std::memset(m, 0, sizeof(*m));
    m->m.t = ctx->t;
    m->m.steps = ctx->steps;
    m->m.dt_last = ctx->dt_last;
    m->m.forcing_on = ctx->drv.on ? 1 : 0;
    m->m.forcing_dirty = ctx->drv.dirty ? 1 : 0;
    m->m.t_next = ctx->drv.t_next;
    m->m.rng = ctx->drv.rng;
    m->m.have_spare = ctx->drv.have_spare ? 1 : 0;
    m->m.spare = ctx->drv.spare;
    m->m.nmodes = ctx->drv.nm;
    std::memcpy(m->m.x, ctx->drv.x, sizeof(double) * 6 * ctx->drv.nm);
    m->injected = ctx->injected;
    m->dissipated = ctx->dissipated;
    return DG_OK;
}

int dg_adi_set_meta(dg_adi_ctx* ctx, const dg_adi_meta* m)
{
    if (!ctx || !m) return DG_EINVAL;
    if (m->m.nmodes != ctx->drv.nm)
        return afail(ctx, DG_EINVAL, "dg_adi_set_meta: call dg_adi_set_forcing with the same modes first");
    ctx->t = m->m.t;
    ctx->steps = m->m.steps;
    ctx->dt_last = m->m.dt_last;
    ctx->drv.on = m->m.forcing_on != 0;
    ctx->drv.t_next = m->m.t_next;
    ctx->drv.rng = m->m.rng;
    ctx->drv.have_spare = m->m.have_spare != 0;
    ctx->drv.spare = m->m.spare;
    std::memcpy(ctx->drv.x, m->m.x, sizeof(double) * 6 * m->m.nmodes);
    // the forcing is projected again from these OU amplitudes before the next step
    ctx->drv.dirty = ctx->drv.on;
    if (!ctx->drv.on) ctx->forcing_active = false;
    ctx->injected = m->injected;
    ctx->dissipated = m->dissipated;
    return DG_OK;
}

int dg_adi_totals(dg_adi_ctx* ctx, double* out)
{
    if (!ctx) return DG_EINVAL;
    if (!out) return afail(ctx, DG_EINVAL, "dg_adi_totals: null output");
    if (!ctx->state_set) return afail(ctx, DG_ESTATE, "dg_adi_totals: no state set");
    const Launch L = adi_make_launch(ctx);
    int nb = 0;
    const void* u = ctx->reg[ctx->cur];
    ACK(ctx->prec == DG_PREC_F64 ? launch_adi_totals<double>(L, ctx->gamma, ctx->kap, u, ctx->partials, &nb)
                                 : launch_adi_totals<float>(L, ctx->gamma, ctx->kap, u, ctx->partials, &nb));
    std::vector<double> part((size_t)nb * 8);
    ACK(cudaMemcpyAsync(part.data(), ctx->partials, part.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    ACK(cudaStreamSynchronize(ctx->st));
    const double vol = ctx->h * ctx->h * ctx->h;
    double acc[8] = {0, 0, 0, 0, 0, 0, 1e300, 1e300};
    for (int blk = 0; blk < nb; ++blk)
        for (int i = 0; i < 8; ++i) {
            const double v = part[(size_t)blk * 8 + i];
            if (i < 6)
                acc[i] += v;
            else
                acc[i] = v < acc[i] ? v : acc[i];
        }
    // the energy: that of the stored variable plus the offset's kap times the mass
    acc[4] += ctx->kap * acc[0];
    for (int i = 0; i < 6; ++i) out[i] = acc[i] * vol;
    out[6] = acc[6];
    out[7] = acc[7];
    return DG_OK;
}

}  // extern "C"
