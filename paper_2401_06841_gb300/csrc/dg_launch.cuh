// dg_launch.cuh -- internal launch interface between the host API and the
// kernel translation units (one per element type).
#pragma once

#include <cuda_runtime.h>

#include "dg_common.cuh"

namespace dg {

struct Launch {
    cudaStream_t st;
    int K;
    int N;
    long ncell;
    Phys ph;
    const void* tab;     // tables of the element type in use
    Ctl* ctl;
    double* partials;    // [kMaxGrid][16]
    int nsm;             // multiprocessors on the device
};

constexpr int kMaxGrid = 8192;

template <typename T>
cudaError_t setup_kernels(int K);
template <typename T>
cudaError_t launch_project(const Launch& L, const T* u, T* vhat, const T* ahat, int flags);
template <typename T>
cudaError_t launch_rhs(const Launch& L, const T* u_in, const T* u_n, T* out, T* vhat, const T* ahat, T rk_a, T rk_b,
                       bool update, double dt_pimax, int flags);
template <typename T>
cudaError_t launch_force(const Launch& L, int nm, const int* kvec, const double* amp, int kmaxc, T* ahat);
template <typename T>
cudaError_t launch_diag(const Launch& L, const T* u, const T* ahat, double dt_pimax, int flags);
template <typename T>
cudaError_t launch_l1(const Launch& L, const T* uA, const T* uB);

}  // namespace dg
