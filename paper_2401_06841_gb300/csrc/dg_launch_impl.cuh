// dg_launch_impl.cuh -- launcher bodies, instantiated once per element type by
// dg_f64.cu and dg_f32.cu.
#pragma once

#include "dg_kernels.cuh"
#include "dg_launch.cuh"

namespace dg {

template <typename T, int K>
struct Occ {
    static int project, rhs_u, rhs_r, force, diag;
};
template <typename T, int K>
int Occ<T, K>::project = 0;
template <typename T, int K>
int Occ<T, K>::rhs_u = 0;
template <typename T, int K>
int Occ<T, K>::rhs_r = 0;
template <typename T, int K>
int Occ<T, K>::force = 0;
template <typename T, int K>
int Occ<T, K>::diag = 0;

template <typename T, int K>
static cudaError_t setup_k()
{
    using S = RhsSmem<T, K>;
    constexpr int NT = Tile<K>::NT;
    cudaError_t e;
    e = cudaFuncSetAttribute(k_rhs<T, K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_rhs<T, K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&Occ<T, K>::rhs_u, k_rhs<T, K, true>, NT, S::bytes);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&Occ<T, K>::rhs_r, k_rhs<T, K, false>, NT, S::bytes);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&Occ<T, K>::project, k_project<T, K>, NT, 0);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&Occ<T, K>::force, k_force<T, K>, NT, 0);
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

template <typename T, int K>
static cudaError_t project_k(const Launch& L, const T* u, T* vhat, const T* ahat, int flags)
{
    KArgs<T> a = make_args<T, K>(L);
    a.u_in = u;
    a.vhat = vhat;
    a.ahat = ahat;
    a.flags = flags;
    const long ntile = (L.ncell + Tile<K>::TC - 1) / Tile<K>::TC;
    k_project<T, K><<<grid_for(ntile, Occ<T, K>::project, L.nsm), Tile<K>::NT, 0, L.st>>>(a);
    return cudaGetLastError();
}

template <typename T, int K>
static cudaError_t rhs_k(const Launch& L, const T* u_in, const T* u_n, T* out, T* vhat, const T* ahat, T rk_a, T rk_b,
                         bool update, double dt_pimax, int flags)
{
    KArgs<T> a = make_args<T, K>(L);
    a.u_in = u_in;
    a.u_n = u_n;
    a.out = out;
    a.vhat = vhat;
    a.ahat = ahat;
    a.rk_a = rk_a;
    a.rk_b = rk_b;
    a.dt_pimax = dt_pimax;
    a.flags = flags;
    const long ntile = (L.ncell + Tile<K>::TC - 1) / Tile<K>::TC;
    const size_t sm = RhsSmem<T, K>::bytes;
    if (update)
        k_rhs<T, K, true><<<grid_for(ntile, Occ<T, K>::rhs_u, L.nsm), Tile<K>::NT, sm, L.st>>>(a);
    else
        k_rhs<T, K, false><<<grid_for(ntile, Occ<T, K>::rhs_r, L.nsm), Tile<K>::NT, sm, L.st>>>(a);
    return cudaGetLastError();
}

template <typename T, int K>
static cudaError_t force_k(const Launch& L, int nm, const int* kvec, const double* amp, int kmaxc, T* ahat)
{
    const long ntile = (L.ncell + Tile<K>::TC - 1) / Tile<K>::TC;
    k_force<T, K><<<grid_for(ntile, Occ<T, K>::force, L.nsm), Tile<K>::NT, 0, L.st>>>(
        static_cast<const T*>(L.tab), L.N, L.ncell, nm, kvec, amp, kmaxc, ahat);
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

#define DG_DISPATCH(fn, ...)                                   \
    do {                                                       \
        if (L.K == 1) return fn<T, 1>(L, __VA_ARGS__);         \
        if (L.K == 2) return fn<T, 2>(L, __VA_ARGS__);         \
        if (L.K == 3) return fn<T, 3>(L, __VA_ARGS__);         \
        return cudaErrorInvalidValue;                          \
    } while (0)

template <typename T>
cudaError_t launch_project(const Launch& L, const T* u, T* vhat, const T* ahat, int flags)
{
    DG_DISPATCH(project_k, u, vhat, ahat, flags);
}
template <typename T>
cudaError_t launch_rhs(const Launch& L, const T* u_in, const T* u_n, T* out, T* vhat, const T* ahat, T rk_a, T rk_b,
                       bool update, double dt_pimax, int flags)
{
    DG_DISPATCH(rhs_k, u_in, u_n, out, vhat, ahat, rk_a, rk_b, update, dt_pimax, flags);
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

#define DG_INSTANTIATE(T)                                                                                         \
    template cudaError_t setup_kernels<T>(int);                                                                  \
    template cudaError_t launch_project<T>(const Launch&, const T*, T*, const T*, int);                          \
    template cudaError_t launch_rhs<T>(const Launch&, const T*, const T*, T*, T*, const T*, T, T, bool, double,   \
                                       int);                                                                     \
    template cudaError_t launch_force<T>(const Launch&, int, const int*, const double*, int, T*);               \
    template cudaError_t launch_diag<T>(const Launch&, const T*, const T*, double, int);                        \
    template cudaError_t launch_l1<T>(const Launch&, const T*, const T*);

}  // namespace dg
