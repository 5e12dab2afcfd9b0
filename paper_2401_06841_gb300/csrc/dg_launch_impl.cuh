// dg_launch_impl.cuh -- launcher bodies, instantiated once per element type by
// dg_f64.cu and dg_f32.cu.
#pragma once

#include "dg_kernels.cuh"
#include "dg_tile.cuh"
#include "dg_launch.cuh"

namespace dg {

template <typename T, int K>
struct Occ {
    static int tile[2][2][4], force, diag;  // [diffusion][back end][mode]
};
template <typename T, int K>
int Occ<T, K>::tile[2][2][4] = {};
template <typename T, int K>
int Occ<T, K>::force = 0;
template <typename T, int K>
int Occ<T, K>::diag = 0;

template <typename T, int K, int MODE, int BK, bool DIFF = false>
static cudaError_t setup_tile()
{
    const size_t sm = sizeof(T) * TileCfg<K, BK>::total;
    cudaError_t e =
        cudaFuncSetAttribute(k_tile<T, K, MODE, BK, DIFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&Occ<T, K>::tile[DIFF][BK][MODE],
                                                         k_tile<T, K, MODE, BK, DIFF>, TileCfg<K, BK>::NT, sm);
}

template <typename T, int K, int BK>
static cudaError_t setup_modes()
{
    cudaError_t e;
    if ((e = setup_tile<T, K, TM_PROJECT, BK>()) != cudaSuccess) return e;
    if ((e = setup_tile<T, K, TM_RHS, BK>()) != cudaSuccess) return e;
    if ((e = setup_tile<T, K, TM_STAGE, BK>()) != cudaSuccess) return e;
    if ((e = setup_tile<T, K, TM_STAGE_VABS, BK>()) != cudaSuccess) return e;
    if ((e = setup_tile<T, K, TM_RHS, BK, true>()) != cudaSuccess) return e;
    if ((e = setup_tile<T, K, TM_STAGE, BK, true>()) != cudaSuccess) return e;
    return setup_tile<T, K, TM_STAGE_VABS, BK, true>();
}

// tile-kernel set-up and launch of one degree; explicitly instantiated per
// translation unit (DG_TILES_*) so that the heaviest degree compiles apart
template <typename T, int K>
cudaError_t setup_tiles()
{
    cudaError_t e;
    if ((e = setup_modes<T, K, BK_FMA>()) != cudaSuccess) return e;
    if constexpr (sizeof(T) == 4) {
        if ((e = setup_modes<T, K, BK_X3>()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T, int K>
static cudaError_t setup_k()
{
    constexpr int NT = Tile<K>::NT;
    cudaError_t e;
    if ((e = setup_tiles<T, K>()) != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&Occ<T, K>::force, k_force<T, K>, 256, 0);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&Occ<T, K>::diag, k_diag<T, K>, NT, 0);
    return e;
}

template <typename T>
cudaError_t setup_kernels(int K)
{
    if (K == 1) return setup_k<T, 1>();
    if (K == 2) return setup_k<T, 2>();
    if (K == 3) return setup_k<T, 3>();
    return cudaErrorInvalidValue;
}

static inline int grid_for(long ntile, int occ, int nsm)
{
    long g = (long)(occ > 0 ? occ : 1) * nsm;
    if (g > ntile) g = ntile;
    if (g > kMaxGrid) g = kMaxGrid;
    if (g < 1) g = 1;
    return (int)g;
}

template <typename T, int K>
static KArgs<T> make_args(const Launch& L)
{
    KArgs<T> a{};
    a.tab = static_cast<const T*>(L.tab);
    a.ctl = L.ctl;
    a.partials = L.partials;
    a.ncell = L.ncell;
    a.N = L.N;
    a.ph = L.ph;
    return a;
}

template <typename T, int K, int BK>
static cudaError_t tile_kb(const Launch& L, const TileLaunch& t)
{
    TArgs<T> a{};
    a.u_in = static_cast<const T*>(t.u_in);
    a.u_n = static_cast<const T*>(t.u_n);
    a.out = static_cast<T*>(t.out);
    a.vh_in = static_cast<const T*>(t.vh_in);
    a.vh_out = static_cast<T*>(t.vh_out);
    a.ahat = static_cast<const T*>(t.ahat);
    a.tab = static_cast<const T*>(L.ttab);
    a.ctl = L.ctl;
    a.partials = L.partials;
    a.ncell = L.ncell;
    a.N = L.N;
    a.ph = L.ph;
    a.rk_a = T(t.rk_a);
    a.rk_b = T(t.rk_b);
    a.dt_pimax = t.dt_pimax;
    a.flags = t.flags;
    a.abar_in = t.abar_in;
    a.abar_out = t.abar_out;
    a.nu = t.nu;
    a.vabs_out = static_cast<T*>(t.vabs_out);
    a.nu_next = t.mode == TM_STAGE_VABS ? t.nu_next : nullptr;
    a.mlp = t.mlp;
    a.trouble = t.mode == TM_PROJECT || t.mode == TM_RHS ? nullptr : t.trouble;
    using Cf = TileCfg<K, BK>;
    const long ntile = (L.ncell + Cf::TC - 1) / Cf::TC;
    const size_t sm = sizeof(T) * Cf::total;
    const bool dif = L.ph.eps > 0.0 && t.mode != TM_PROJECT;
    const int g = grid_for(ntile, Occ<T, K>::tile[dif][BK][t.mode], L.nsm);
    if (t.mode == TM_PROJECT)
        k_tile<T, K, TM_PROJECT, BK><<<g, Cf::NT, sm, L.st>>>(a);
    else if (t.mode == TM_RHS)
        dif ? k_tile<T, K, TM_RHS, BK, true><<<g, Cf::NT, sm, L.st>>>(a)
            : k_tile<T, K, TM_RHS, BK><<<g, Cf::NT, sm, L.st>>>(a);
    else if (t.mode == TM_STAGE)
        dif ? k_tile<T, K, TM_STAGE, BK, true><<<g, Cf::NT, sm, L.st>>>(a)
            : k_tile<T, K, TM_STAGE, BK><<<g, Cf::NT, sm, L.st>>>(a);
    else
        dif ? k_tile<T, K, TM_STAGE_VABS, BK, true><<<g, Cf::NT, sm, L.st>>>(a)
            : k_tile<T, K, TM_STAGE_VABS, BK><<<g, Cf::NT, sm, L.st>>>(a);
    return cudaGetLastError();
}

template <typename T, int K>
cudaError_t tile_k(const Launch& L, const TileLaunch& t)
{
    if constexpr (sizeof(T) == 4) {
        if (L.bk == BK_X3) return tile_kb<T, K, BK_X3>(L, t);
    }
    if (L.bk != BK_FMA) return cudaErrorInvalidValue;
    return tile_kb<T, K, BK_FMA>(L, t);
}

template <typename T, int K>
static cudaError_t force_k(const Launch& L, int nm, const int* kvec, const double* amp, int kmaxc, T* ahat)
{
    if (nm > 512 || kmaxc > kForceKM) return cudaErrorInvalidValue;
    T* G = static_cast<T*>(L.gtab);
    const int ng = L.N * kForceNK * (K + 1);
    k_force_axis<T, K><<<(ng + 255) / 256, 256, 0, L.st>>>(L.r1, L.N, kmaxc, G);
    const long nb = (L.ncell + 255) / 256;
    k_force<T, K><<<grid_for(nb, Occ<T, K>::force, L.nsm), 256, 0, L.st>>>(G, L.N, L.ncell, nm, kvec, amp, ahat);
    return cudaGetLastError();
}

template <typename T, int K>
static cudaError_t diag_k(const Launch& L, const T* u, const T* ahat, double dt_pimax, int flags)
{
    KArgs<T> a = make_args<T, K>(L);
    a.u_in = u;
    a.ahat = ahat;
    a.dt_pimax = dt_pimax;
    a.flags = flags;
    const long ntile = (L.ncell + Tile<K>::TC - 1) / Tile<K>::TC;
    k_diag<T, K><<<grid_for(ntile, Occ<T, K>::diag, L.nsm), Tile<K>::NT, 0, L.st>>>(a);
    return cudaGetLastError();
}

template <typename T, int K>
static cudaError_t l1_k(const Launch& L, const T* uA, const T* uB)
{
    const long total = L.ncell * Dims<K>::nql;
    long g = (total + 255) / 256;
    if (g > 4L * L.nsm) g = 4L * L.nsm;
    if (g > kMaxGrid) g = kMaxGrid;
    k_l1<T, K><<<(int)g, 256, 0, L.st>>>(static_cast<const T*>(L.tab), uA, uB, L.ncell, L.ph.h, L.ctl, L.partials);
    return cudaGetLastError();
}

template <typename T, int K>
static cudaError_t flatten_k(const Launch& L, T* u, unsigned char* trouble, unsigned char* level)
{
    long g = (L.ncell + 255) / 256;
    if (g > 4L * L.nsm) g = 4L * L.nsm;
    if (g < 1) g = 1;
    k_flatten<T, K><<<(int)g, 256, 0, L.st>>>(u, trouble, level, L.ncell, L.ctl);
    return cudaGetLastError();
}

#define DG_DISPATCH(fn, ...)                                   \
    do {                                                       \
        if (L.K == 1) return fn<T, 1>(L, __VA_ARGS__);         \
        if (L.K == 2) return fn<T, 2>(L, __VA_ARGS__);         \
        if (L.K == 3) return fn<T, 3>(L, __VA_ARGS__);         \
        return cudaErrorInvalidValue;                          \
    } while (0)

template <typename T>
cudaError_t launch_tile(const Launch& L, const TileLaunch& t)
{
    DG_DISPATCH(tile_k, t);
}
template <typename T>
cudaError_t launch_force(const Launch& L, int nm, const int* kvec, const double* amp, int kmaxc, T* ahat)
{
    DG_DISPATCH(force_k, nm, kvec, amp, kmaxc, ahat);
}
template <typename T>
cudaError_t launch_diag(const Launch& L, const T* u, const T* ahat, double dt_pimax, int flags)
{
    DG_DISPATCH(diag_k, u, ahat, dt_pimax, flags);
}
template <typename T>
cudaError_t launch_l1(const Launch& L, const T* uA, const T* uB)
{
    DG_DISPATCH(l1_k, uA, uB);
}
template <typename T>
cudaError_t launch_flatten(const Launch& L, T* u, unsigned char* trouble, unsigned char* level)
{
    DG_DISPATCH(flatten_k, u, trouble, level);
}

#define DG_TILES_EXTERN(T, K)                                                   \
    extern template cudaError_t tile_k<T, K>(const Launch&, const TileLaunch&); \
    extern template cudaError_t setup_tiles<T, K>();
#define DG_TILES_INSTANTIATE(T, K)                                       \
    template cudaError_t tile_k<T, K>(const Launch&, const TileLaunch&); \
    template cudaError_t setup_tiles<T, K>();

#define DG_INSTANTIATE(T)                                                                                         \
    template cudaError_t setup_kernels<T>(int);                                                                  \
    template cudaError_t launch_tile<T>(const Launch&, const TileLaunch&);                                       \
    template cudaError_t launch_force<T>(const Launch&, int, const int*, const double*, int, T*);               \
    template cudaError_t launch_diag<T>(const Launch&, const T*, const T*, double, int);                        \
    template cudaError_t launch_l1<T>(const Launch&, const T*, const T*);                                       \
    template cudaError_t launch_flatten<T>(const Launch&, T*, unsigned char*, unsigned char*);

}  // namespace dg
