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
    const void* tab;     // tables of the element type in use (auxiliary kernels)
    const void* ttab;    // tables of the tile kernels
    Ctl* ctl;
    double* partials;    // [kMaxGrid][16]
    int nsm;             // multiprocessors on the device
    int bk;              // 0: CUDA-core products, 1: split-BF16 x3 tensor-core products
};

constexpr int kMaxGrid = 8192;

template <typename T>
cudaError_t setup_kernels(int K);
// tile kernel modes: 0 projection only (velocity projection, forcing sums,
// CFL dt with F_DT), 1 right-hand side only, 2 right-hand side + SSP-RK stage
// (+ the next stage's projection with F_NEXTPROJ)
struct TileLaunch {
    int mode;
    const void* u_in;
    const void* u_n;
    void* out;
    const void* vh_in;
    void* vh_out;
    const void* ahat;
    double rk_a, rk_b;
    double dt_pimax;
    int flags;
    int abar_in, abar_out;
};
template <typename T>
cudaError_t launch_tile(const Launch& L, const TileLaunch& t);
template <typename T>
cudaError_t launch_force(const Launch& L, int nm, const int* kvec, const double* amp, int kmaxc, T* ahat);
template <typename T>
cudaError_t launch_diag(const Launch& L, const T* u, const T* ahat, double dt_pimax, int flags);
template <typename T>
cudaError_t launch_l1(const Launch& L, const T* uA, const T* uB);

}  // namespace dg
