// dg_mlp.cu -- launchers of the learned-sensor kernels (training in FP32,
// fused BF16 inference, features and labels for FP64/FP32 states).
#include "dg_launch.cuh"
#include "dg_launch_impl.cuh"
#include "dg_mlp.cuh"

namespace dg {

template <int D>
static cudaError_t train_pass_d(cudaStream_t st, const float* W, const float* X, const float* Y, int n, float* work,
                                float* G, double* loss)
{
    const MlpLayout L = MlpLayout::make(D);
    const size_t sm = sizeof(float) * L.P;
    const int g = (n + 127) / 128;
    k_mlp_fwd<D><<<g, 128, sm, st>>>(W, X, Y, n, work);
    k_mlp_bwd<D><<<g, 128, sm, st>>>(W, n, work);
    k_mlp_grad<D><<<(L.P + 1 + 255) / 256, 256, 0, st>>>(X, n, work, G, loss);
    return cudaGetLastError();
}

cudaError_t mlp_train_pass(cudaStream_t st, int D, const float* W, const float* X, const float* Y, int n, float* work,
                           float* G, double* loss)
{
    if (n < 1 || n > MLP_BMAX) return cudaErrorInvalidValue;
    if (D == 8) return train_pass_d<8>(st, W, X, Y, n, work, G, loss);
    if (D == 20) return train_pass_d<20>(st, W, X, Y, n, work, G, loss);
    if (D == 40) return train_pass_d<40>(st, W, X, Y, n, work, G, loss);
    return cudaErrorInvalidValue;
}

cudaError_t mlp_adam(cudaStream_t st, int P, float* W, const float* G, float* m, float* v, float lr, float b1, float b2,
                     float eps, float c1, float c2)
{
    k_mlp_adam<<<(P + 255) / 256, 256, 0, st>>>(W, G, m, v, P, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

template <typename T, int K>
static cudaError_t infer_k(const Launch& L, const T* u, const T* vabs, const float* X, long n, const uint32_t* packed,
                           float* nu, float* y)
{
    const float ref = (float)(L.ph.cs * L.ph.hp);
    long g = (n + 127) / 128;
    if (g > 8L * L.nsm) g = 8L * L.nsm;
    if (g < 1) g = 1;
    const float gate = (float)L.ph.nu_gate;
    if (u)
        k_mlp_infer<T, K, true><<<(int)g, 256, 0, L.st>>>(u, vabs, nullptr, n, packed, (float)L.ph.cs, ref, gate, nu,
                                                          y);
    else
        k_mlp_infer<T, K, false><<<(int)g, 256, 0, L.st>>>(nullptr, nullptr, X, n, packed, (float)L.ph.cs, ref, gate,
                                                           nu, y);
    return cudaGetLastError();
}

template <typename T>
cudaError_t mlp_infer(const Launch& L, const T* u, const T* vabs, const float* X, long n, const uint32_t* packed,
                      float* nu, float* y)
{
    DG_DISPATCH(infer_k, u, vabs, X, n, packed, nu, y);
}

template <typename T, int K>
static cudaError_t features_k(const Launch& L, const T* u, const T* vabs, const T* phiv, double dt, float* X, float* Y)
{
    const long ntile = (L.ncell + Tile<K>::TC - 1) / Tile<K>::TC;
    long g = ntile < 4L * L.nsm ? ntile : 4L * L.nsm;
    const T* wq = static_cast<const T*>(L.tab) + TabLayout<K>::wq;
    k_features<T, K><<<(int)g, Tile<K>::NT, 0, L.st>>>(u, vabs, phiv, wq, L.ncell, L.ph, dt, X, Y);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_features(const Launch& L, const T* u, const T* vabs, const T* phiv, double dt, float* X, float* Y)
{
    DG_DISPATCH(features_k, u, vabs, phiv, dt, X, Y);
}

template cudaError_t mlp_infer<float>(const Launch&, const float*, const float*, const float*, long, const uint32_t*,
                                      float*, float*);
template cudaError_t mlp_infer<double>(const Launch&, const double*, const double*, const float*, long,
                                       const uint32_t*, float*, float*);
template cudaError_t launch_features<float>(const Launch&, const float*, const float*, const float*, double, float*,
                                            float*);
template cudaError_t launch_features<double>(const Launch&, const double*, const double*, const double*, double,
                                             float*, float*);

}  // namespace dg
