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
// or any host allocator: the tables are built by the context path's builder in
// fixed-size static host buffers and copied in.
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
#include "dg_tables.cuh"
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

// ---- basis tables in fixed static host buffers (no host allocation): the
// context path's builder (dg_tables.cuh), so both upload the same bits ----
tables::Work g_work;
unsigned char g_host[sizeof(double) * kTabWords];  // the table block in the element type

size_t fill_tables_for(int K, int prec) { return tables::fill_tile_tables_for(K, prec, g_work, g_host, sizeof(g_host)); }

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
        if (nb == 0) return report(DG_ECUDA, "table block larger than its buffer");
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
