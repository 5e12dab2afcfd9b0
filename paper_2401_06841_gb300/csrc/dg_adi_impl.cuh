// dg_adi_impl.cuh -- launchers of the adiabatic-system kernels (k = 1..3);
// instantiated per element type in dg_adi_f32.cu and dg_adi_f64.cu.
#pragma once

#include "dg_adi.cuh"
#include "dg_launch.cuh"

namespace dg {

namespace {

template <typename T, int K, int MODE, bool DRIVEN>
int adi_blocks_per_sm()
{
    static int occ = -1;
    if (occ < 0) {
        const int sm = (int)(sizeof(T) * AdiCfg<K, DRIVEN>::total);
        cudaFuncSetAttribute(k_adi<T, K, MODE, DRIVEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_adi<T, K, MODE, DRIVEN>, AdiCfg<K, DRIVEN>::NT, sm) !=
            cudaSuccess)
            o = 1;
        occ = o < 1 ? 1 : o;
    }
    return occ;
}

template <typename T, int K, int MODE, bool DRIVEN = false>
cudaError_t adi_launch(const Launch& L, const AdiArgs<T>& a)
{
    using A = AdiCfg<K, DRIVEN>;
    const long ntile = (L.ncell + A::TC - 1) / A::TC;
    long g = (long)adi_blocks_per_sm<T, K, MODE, DRIVEN>() * L.nsm;
    if (g > ntile) g = ntile;
    if (g < 1) g = 1;
    k_adi<T, K, MODE, DRIVEN><<<(int)g, A::NT, sizeof(T) * A::total, L.st>>>(a);
    return cudaGetLastError();
}

template <typename T, int K>
cudaError_t adi_k(const Launch& L, double gamma, const AdiLaunch& t)
{
    AdiArgs<T> a{};
    a.u_in = static_cast<const T*>(t.u_in);
    a.u_n = static_cast<const T*>(t.u_n);
    a.out = static_cast<T*>(t.out);
    a.pr_in = static_cast<const T*>(t.pr_in);
    a.pr_out = static_cast<T*>(t.pr_out);
    a.tab = static_cast<const T*>(L.ttab);
    a.ctl = L.ctl;
    a.ncell = L.ncell;
    a.N = L.N;
    a.ph = L.ph;
    a.gamma = gamma;
    a.gas.gamma = T(gamma);
    a.gas.g1 = T(gamma - 1.0);
    a.gas.ig1 = T(1.0 / (gamma - 1.0));
    a.gas.cth = T(t.cs_reset * t.cs_reset / (gamma - 1.0));
    a.gas.kap = T(t.kap);
    a.gas.c0 = T((gamma - 1.0) * t.kap);
    a.gas.cres = T(t.cs_reset * t.cs_reset / (gamma - 1.0) - t.kap);
    a.gas.fill_e = T((1.0 - (gamma - 1.0) * t.kap) / (gamma - 1.0));
    a.rk_a = T(t.rk_a);
    a.rk_b = T(t.rk_b);
    a.dt_pimax = t.dt_pimax;
    a.flags = t.flags;
    a.ahat = static_cast<const T*>(t.ahat);
    a.partials = L.partials;
    a.abar_in = t.abar_in;
    a.abar_out = t.abar_out;
    a.beta = t.beta;
    a.cs_reset = t.cs_reset;
    for (int i = 0; i < 3; ++i) a.bc[i] = t.bc[i];
    for (int i = 0; i < 5; ++i) a.inflow[i] = t.inflow[i];
    if ((t.flags & F_FORCE) && !t.ahat) return cudaErrorInvalidValue;
    const bool driven = (t.flags & F_FORCE) != 0;
    if (t.mode == ADI_PROJECT) return adi_launch<T, K, ADI_PROJECT>(L, a);
    if (t.mode == ADI_RESET) return adi_launch<T, K, ADI_RESET>(L, a);
    if (t.mode == ADI_RHS) return driven ? adi_launch<T, K, ADI_RHS, true>(L, a) : adi_launch<T, K, ADI_RHS>(L, a);
    return driven ? adi_launch<T, K, ADI_STAGE, true>(L, a) : adi_launch<T, K, ADI_STAGE>(L, a);
}

template <typename T, int K>
cudaError_t adi_totals_k(const Launch& L, double gamma, double kap, const void* u, double* partials, int* nblocks)
{
    long g = (L.ncell + 255) / 256;
    if (g > 4L * L.nsm) g = 4L * L.nsm;
    if (g > kMaxGrid) g = kMaxGrid;
    if (g < 1) g = 1;
    *nblocks = (int)g;
    k_adi_totals<T, K><<<(int)g, 256, 0, L.st>>>(static_cast<const T*>(u), static_cast<const T*>(L.ttab), L.ncell,
                                                 gamma, (gamma - 1.0) * kap, partials);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_adi(const Launch& L, double gamma, const AdiLaunch& t)
{
    if (L.K == 1) return adi_k<T, 1>(L, gamma, t);
    if (L.K == 2) return adi_k<T, 2>(L, gamma, t);
    return adi_k<T, 3>(L, gamma, t);
}

template <typename T>
cudaError_t launch_adi_totals(const Launch& L, double gamma, double kap, const void* u, double* partials, int* nblocks)
{
    if (L.K == 1) return adi_totals_k<T, 1>(L, gamma, kap, u, partials, nblocks);
    if (L.K == 2) return adi_totals_k<T, 2>(L, gamma, kap, u, partials, nblocks);
    return adi_totals_k<T, 3>(L, gamma, kap, u, partials, nblocks);
}

// e_s += d rho, coefficient by coefficient (a change of the energy offset)
template <typename T>
__global__ void k_adi_shift(T* u, long ncell, int b, T d)
{
    const long n = ncell * b;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const long c = i / b;
        const int l = (int)(i % b);
        u[(c * 5 + 4) * b + l] += d * u[c * 5 * b + l];
    }
}

template <typename T>
cudaError_t launch_adi_shift(const Launch& L, void* u, double d)
{
    const int b = (L.K + 1) * (L.K + 2) * (L.K + 3) / 6;
    long g = (L.ncell * b + 255) / 256;
    if (g > 8L * L.nsm) g = 8L * L.nsm;
    if (g < 1) g = 1;
    k_adi_shift<T><<<(int)g, 256, 0, L.st>>>(static_cast<T*>(u), L.ncell, b, T(d));
    return cudaGetLastError();
}

}  // namespace dg
