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
    Rule1 r1;            // the 1D Gauss rule
    void* gtab;          // forcing: 1D factors [N][17][k+1][2] of the element type
};

constexpr int kMaxGrid = 8192;

template <typename T>
cudaError_t setup_kernels(int K);
// tile kernel modes: 0 projection only (velocity projection, forcing sums,
// CFL dt with F_DT), 1 right-hand side only, 2 right-hand side + SSP-RK stage
// (+ the next stage's projection with F_NEXTPROJ), 3 as 2 with the projection
// of |v| (vabs_out) for the learned sensor
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
    const float* nu;     // learned sensor: per-cell coefficient
    void* vabs_out;      // learned sensor: projection of |v|
    float* nu_next;      // learned sensor: coefficient of the output, evaluated in the kernel (mode 3)
    const uint32_t* mlp; // learned sensor: packed network for nu_next
    unsigned char* trouble;  // positivity by repetition: per-cell marks of the stage (or nullptr)
};
template <typename T>
cudaError_t launch_tile(const Launch& L, const TileLaunch& t);
template <typename T>
cudaError_t launch_force(const Launch& L, int nm, const int* kvec, const double* amp, int kmaxc, T* ahat);
template <typename T>
cudaError_t launch_diag(const Launch& L, const T* u, const T* ahat, double dt_pimax, int flags);
template <typename T>
cudaError_t launch_l1(const Launch& L, const T* uA, const T* uB);
// positivity by repetition: every marked cell of u [c][4][b] is unmarked and its
// modes l > 0 scaled by 1/2 (level 0, 1) or 0 (level 2), its level incremented;
// a marked cell whose modes l > 0 are all zero sets DG_ST_FLAT_ instead
template <typename T>
cudaError_t launch_flatten(const Launch& L, T* u, unsigned char* trouble, unsigned char* level);

// x3 stage of degree 3 on the tcgen05 tensor cores (dg_tc5.cu): the
// projection kernel, or the volume and face kernels of a right-hand side /
// an SSP-RK stage
enum { T5_PROJECT = 0, T5_RHS = 1, T5_STAGE = 2 };
// tiled TMA descriptors (CUtensorMap, 128 bytes each) of the buffers whose whole
// tiles the tcgen05 kernels stage: a context's state registers, the volume term
// and the driving; a launch finds them by base address
struct T5Map {
    const void* base;
    alignas(64) unsigned char map[128];
};
struct T5Maps {
    int n;
    T5Map m[8];
};
// one map per buffer [ncell][per] FP32 (boxes of 16 cells); DG_EINVAL-like
// cudaErrorInvalidValue when the driver's encoder is missing or refuses
cudaError_t tc5_make_maps(T5Maps* out, const void* const* bases, const int* per, int n, long ncell);

struct T5Launch {
    int kind;
    const void* u_in;
    const void* u_n;
    void* out;
    const void* vh_in;
    void* vh_out;
    void* vabs_out;
    const void* ahat;
    const float* nu;
    void* rvol;          // volume term [c][4][b] FP32 (caller's scratch)
    void* vh_self;       // undriven stages: the volume kernel projects v of u_in here (or nullptr)
    float* nu_next;      // projection: the learned sensor's coefficient of u_in (or nullptr)
    const uint32_t* mlp; // its packed network
    const T5Maps* maps;  // tiled TMA descriptors of the context's buffers (or nullptr)
    unsigned char* trouble;  // positivity by repetition: per-cell marks (or nullptr)
    const void* tab5;    // table block (tc5_build_tables)
    const void* phiv;    // [b][nq] FP32 phi at the volume points
    const void* phif;    // [b][nf] FP32 phi at the face points
    double rk_a, rk_b;
    double dt_pimax;
    int flags;
    int abar_in, abar_out;
};
size_t tc5_table_bytes();
int tc5_build_tables(const double* x, const double* w, unsigned char* out, size_t cap);
cudaError_t tc5_setup();
cudaError_t launch_tc5(const Launch& L, const T5Launch& t);

// adiabatic system (dg_adi.cu): mode 0 projection of v and p (+ CFL bound
// with F_DT, forcing sums with F_FORCE), 1 right-hand side, 2 stage
// (right-hand side, SSP-RK combine, positivity of density and pressure),
// 3 isothermal reset of the thermal energy (in place)
enum { ADI_PROJECT = 0, ADI_RHS = 1, ADI_STAGE = 2, ADI_RESET = 3 };
struct AdiLaunch {
    int mode;
    const void* u_in;
    const void* u_n;
    void* out;
    const void* pr_in;
    void* pr_out;
    double rk_a, rk_b;
    double dt_pimax;
    int flags;
    const void* ahat;       // driving (F_FORCE)
    int abar_in, abar_out;  // ctl->abar2 slots
    double beta;            // stage weight of the injected energy
    double cs_reset;        // reset mode
    double kap;             // energy offset of the stored states: e_s = e - kap rho
    int bc[3];              // boundaries per axis (DG_BC_*)
    double inflow[5];       // DG_BC_INFLOW: rho, v, p at the face at coordinate 0
};
template <typename T>
cudaError_t launch_adi(const Launch& L, double gamma, const AdiLaunch& t);
// per-block FP64 totals [nblocks][8]: mass, momentum (3), energy, kinetic
// energy, min rho and min p at the volume points
template <typename T>
cudaError_t launch_adi_totals(const Launch& L, double gamma, double kap, const void* u, double* partials, int* nblocks);
// e_s += d rho on a state (a change of the energy offset)
template <typename T>
cudaError_t launch_adi_shift(const Launch& L, void* u, double d);

// turbulence statistics (dg_analysis.cu)
template <typename T>
cudaError_t launch_density_pdf(const Launch& L, const T* u, double lo, double hi, int nbins, double* mean,
                               double* hist);
template <typename T>
cudaError_t launch_structure(const Launch& L, const T* u, int nbins, long npairs, unsigned long long seed, double* acc);
template <typename T>
cudaError_t launch_sample(const Launch& L, const T* u, int d, double* out);
cudaError_t launch_shell(const Launch& L, const void* F, int Ng, int nbins, double scale2, int first, double* power,
                         double* ksum, unsigned long long* count);

// learned viscosity sensor
constexpr int kMlpHidden = 64;
constexpr int kMlpBatchMax = 4096;
inline int mlp_params(int D) { return kMlpHidden * D + kMlpHidden + kMlpHidden * kMlpHidden + 2 * kMlpHidden + 1; }
inline size_t mlp_work_floats_host() { return (size_t)6 * kMlpHidden * kMlpBatchMax + kMlpBatchMax; }
cudaError_t mlp_train_pass(cudaStream_t st, int D, const float* W, const float* X, const float* Y, int n, float* work,
                           float* G, double* loss);
cudaError_t mlp_adam(cudaStream_t st, int P, float* W, const float* G, float* m, float* v, float lr, float b1, float b2,
                     float eps, float c1, float c2);
template <typename T>
cudaError_t mlp_infer(const Launch& L, const T* u, const T* vabs, const float* X, long n, const uint32_t* packed,
                      float* nu, float* y);
template <typename T>
cudaError_t launch_features(const Launch& L, const T* u, const T* vabs, const T* phiv, double dt, float* X, float* Y);

}  // namespace dg
