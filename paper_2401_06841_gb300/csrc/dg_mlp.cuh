// dg_mlp.cuh -- learned viscosity sensor: a per-cell network
//   y = W3 . gelu(W2 gelu(W1 x + b1) + b2) + b3,   gelu(z) = z/2 (1 + erf(z/sqrt 2))
// predicting y = log(nu / (cs h/p)) from x = (rho_l/rho_0, |v|hat_l/cs), the
// normalised modal coefficients of the cell (D = 2b inputs, 64 hidden units).
// Training runs in FP32 on the CUDA cores (forward with stored activations,
// backward, per-parameter gradient sums in a fixed order, Adam); inference is
// one fused kernel with BF16 tensor-core products and FP32 accumulation, the
// accumulator fragments of a layer feeding the next layer's operand fragments
// directly in registers.
//
// Parameter layout (FP32): W1 [64][D], b1 [64], W2 [64][64], b2 [64], W3 [64], b3.
#pragma once

#include <cuda_bf16.h>

#include "dg_tile.cuh"

namespace dg {

constexpr int MLP_BMAX = 4096;  // largest training batch

struct MlpLayout {
    int D, P, oW1, ob1, oW2, ob2, oW3, ob3;
    __host__ __device__ static MlpLayout make(int D)
    {
        MlpLayout L{};
        L.D = D;
        L.oW1 = 0;
        L.ob1 = MLP_H * D;
        L.oW2 = L.ob1 + MLP_H;
        L.ob2 = L.oW2 + MLP_H * MLP_H;
        L.oW3 = L.ob2 + MLP_H;
        L.ob3 = L.oW3 + MLP_H;
        L.P = L.ob3 + 1;
        return L;
    }
};

// training work arrays, each [64][MLP_BMAX] (sample index fastest) plus r [MLP_BMAX]
enum { MW_Z1 = 0, MW_A1 = 1, MW_Z2 = 2, MW_A2 = 3, MW_DZ1 = 4, MW_DZ2 = 5, MW_R = 6 };
constexpr size_t mlp_work_floats() { return (size_t)6 * MLP_H * MLP_BMAX + MLP_BMAX; }

__device__ __forceinline__ float gelu_prime_f(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// forward pass of a batch, one thread per sample; stores z1, a1, z2, a2, r = y^ - y
template <int D>
__global__ void __launch_bounds__(128) k_mlp_fwd(const float* __restrict__ W, const float* __restrict__ X,
                                                 const float* __restrict__ Y, int n, float* __restrict__ work)
{
    const MlpLayout L = MlpLayout::make(D);
    extern __shared__ float sW[];
    for (int e = threadIdx.x; e < L.P; e += blockDim.x) sW[e] = W[e];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x[D];
#pragma unroll
    for (int d = 0; d < D; ++d) x[d] = X[(size_t)i * D + d];
    float a1[MLP_H];
#pragma unroll 4
    for (int j = 0; j < MLP_H; ++j) {
        float z = sW[L.ob1 + j];
#pragma unroll
        for (int d = 0; d < D; ++d) z += sW[L.oW1 + j * D + d] * x[d];
        a1[j] = gelu_f(z);
        work[(size_t)MW_Z1 * MLP_H * MLP_BMAX + (size_t)j * MLP_BMAX + i] = z;
        work[(size_t)MW_A1 * MLP_H * MLP_BMAX + (size_t)j * MLP_BMAX + i] = a1[j];
    }
    float y = sW[L.ob3];
#pragma unroll 4
    for (int j = 0; j < MLP_H; ++j) {
        float z = sW[L.ob2 + j];
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) z += sW[L.oW2 + j * MLP_H + k] * a1[k];
        const float a = gelu_f(z);
        work[(size_t)MW_Z2 * MLP_H * MLP_BMAX + (size_t)j * MLP_BMAX + i] = z;
        work[(size_t)MW_A2 * MLP_H * MLP_BMAX + (size_t)j * MLP_BMAX + i] = a;
        y += sW[L.oW3 + j] * a;
    }
    work[(size_t)6 * MLP_H * MLP_BMAX + i] = y - Y[i];
}

// backward pass, one thread per sample: dz2 = (2 r / n) W3 gelu'(z2),
// dz1 = (W2^T dz2) gelu'(z1)
template <int D>
__global__ void __launch_bounds__(128) k_mlp_bwd(const float* __restrict__ W, int n, float* __restrict__ work)
{
    const MlpLayout L = MlpLayout::make(D);
    extern __shared__ float sW[];
    for (int e = threadIdx.x; e < L.P; e += blockDim.x) sW[e] = W[e];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float d3 = 2.0f * work[(size_t)6 * MLP_H * MLP_BMAX + i] / (float)n;
    float dz2[MLP_H];
#pragma unroll
    for (int j = 0; j < MLP_H; ++j) {
        const float z = work[(size_t)MW_Z2 * MLP_H * MLP_BMAX + (size_t)j * MLP_BMAX + i];
        dz2[j] = d3 * sW[L.oW3 + j] * gelu_prime_f(z);
        work[(size_t)MW_DZ2 * MLP_H * MLP_BMAX + (size_t)j * MLP_BMAX + i] = dz2[j];
    }
#pragma unroll 4
    for (int k = 0; k < MLP_H; ++k) {
        float s = 0.0f;
#pragma unroll
        for (int j = 0; j < MLP_H; ++j) s += sW[L.oW2 + j * MLP_H + k] * dz2[j];
        const float z = work[(size_t)MW_Z1 * MLP_H * MLP_BMAX + (size_t)k * MLP_BMAX + i];
        work[(size_t)MW_DZ1 * MLP_H * MLP_BMAX + (size_t)k * MLP_BMAX + i] = s * gelu_prime_f(z);
    }
}

// gradient of the batch loss, one thread per parameter (fixed summation
// order over the samples, FP64 accumulation); the extra thread P writes the
// mean squared error
template <int D>
__global__ void __launch_bounds__(256) k_mlp_grad(const float* __restrict__ X, int n, const float* __restrict__ work,
                                                  float* __restrict__ G, double* __restrict__ loss)
{
    const MlpLayout L = MlpLayout::make(D);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > L.P) return;
    const float* R = work + (size_t)6 * MLP_H * MLP_BMAX;
    double acc = 0.0;
    if (p == L.P) {
        for (int i = 0; i < n; ++i) acc += (double)R[i] * (double)R[i];
        *loss = acc / n;
        return;
    }
    auto row = [&](int which, int j) { return work + ((size_t)which * MLP_H + j) * MLP_BMAX; };
    if (p < L.ob1) {
        const int j = p / D, d = p % D;
        const float* dz = row(MW_DZ1, j);
        for (int i = 0; i < n; ++i) acc += (double)dz[i] * (double)X[(size_t)i * D + d];
    } else if (p < L.oW2) {
        const float* dz = row(MW_DZ1, p - L.ob1);
        for (int i = 0; i < n; ++i) acc += (double)dz[i];
    } else if (p < L.ob2) {
        const int j = (p - L.oW2) / MLP_H, k = (p - L.oW2) % MLP_H;
        const float* dz = row(MW_DZ2, j);
        const float* a = row(MW_A1, k);
        for (int i = 0; i < n; ++i) acc += (double)dz[i] * (double)a[i];
    } else if (p < L.oW3) {
        const float* dz = row(MW_DZ2, p - L.ob2);
        for (int i = 0; i < n; ++i) acc += (double)dz[i];
    } else if (p < L.ob3) {
        const float* a = row(MW_A2, p - L.oW3);
        for (int i = 0; i < n; ++i) acc += 2.0 * (double)R[i] / n * (double)a[i];
    } else {
        for (int i = 0; i < n; ++i) acc += 2.0 * (double)R[i] / n;
    }
    G[p] = (float)acc;
}

// Adam (Kingma & Ba 2015) with bias corrections c1 = 1/(1-b1^t), c2 = 1/(1-b2^t)
static __global__ void k_mlp_adam(float* __restrict__ W, const float* __restrict__ G, float* __restrict__ m,
                           float* __restrict__ v, int P, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const float g = G[p];
    const float mm = b1 * m[p] + (1.0f - b1) * g;
    const float vv = b2 * v[p] + (1.0f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    W[p] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
}

// ---------------------------------------------------------------------------
// fused inference: one warp per 16 samples, three BF16 mma.sync layers
// packed weights: B1 = W1^T [KD][64], B2 = W2^T [64][64], B3 = W3 as [64][8]
// (column 0), each as fragments [K/16][N/8][32 lanes][2 words], then b1, b2, b3
// ---------------------------------------------------------------------------
// x(r, k): FROMSTATE reads the cell's state (rho_l/rho_0) and |v|hat/cs,
// otherwise an explicit feature matrix X [n][D]
template <typename T, int K, bool FROMSTATE>
__global__ void __launch_bounds__(256) k_mlp_infer(const T* __restrict__ u, const T* __restrict__ vabs,
                                                   const float* __restrict__ X, long n,
                                                   const uint32_t* __restrict__ packed, float cs, float ref,
                                                   float gate, float* __restrict__ nu_out, float* __restrict__ y_out)
{
    constexpr int b = Dims<K>::b, D = 2 * b;
    using PK = MlpPack<D>;
    __shared__ uint32_t sP[PK::words];
    __shared__ float sF[FROMSTATE ? 8 * 16 * D : 1];  // a warp's 16 feature rows (state input)
    for (int e = threadIdx.x; e < PK::words; e += blockDim.x) sP[e] = packed[e];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float inv_cs = 1.0f / cs;
    const long nwarps = (long)gridDim.x * (blockDim.x >> 5);
    for (long base = ((long)blockIdx.x * (blockDim.x >> 5) + warp) * 16; base < n; base += nwarps * 16) {
        float* sf = sF + (FROMSTATE ? warp * 16 * D : 0);
        if constexpr (FROMSTATE) {
            // the 16 rows: lane 2 rl + h loads row rl's rho coefficients (h = 0) or its
            // |v| projection (h = 1), all b loads in flight
            __syncwarp();
            const int rl = lane >> 1, h = lane & 1;
            const long r = base + rl;
            T x[b];
#pragma unroll
            for (int l = 0; l < b; ++l) x[l] = T(0);
            if (r < n) {
                const T* src = h == 0 ? u + r * 4 * b : vabs + r * b;
                if constexpr (sizeof(T) == 4 && b % 4 == 0) {
#pragma unroll
                    for (int l = 0; l < b; l += 4) {
                        const float4 q = __ldg(reinterpret_cast<const float4*>(src + l));
                        x[l] = q.x;
                        x[l + 1] = q.y;
                        x[l + 2] = q.z;
                        x[l + 3] = q.w;
                    }
                } else {
#pragma unroll
                    for (int l = 0; l < b; ++l) x[l] = src[l];
                }
            }
            float* dst = sf + rl * D + h * b;
#pragma unroll
            for (int l = 0; l < b; ++l)
                dst[l] = r >= n ? 0.0f : (h == 0 ? (float)(x[l] / x[0]) : (float)x[l] * inv_cs);
            __syncwarp();
        }
        auto feat = [&](int rl, int k) -> float {
            if constexpr (FROMSTATE) {
                return k < D ? sf[rl * D + k] : 0.0f;
            } else {
                const long r = base + rl;
                if (r >= n || k >= D) return 0.0f;
                return X[r * D + k];
            }
        };
        float y0, y1;
        mlp_infer_warp<D>(feat, sP, y0, y1);
        const long r0 = base + g, r1 = base + g + 8;
        if (t == 0) {
            if (r0 < n) {
                if (nu_out) nu_out[r0] = expf(y0) < gate ? 0.f : ref * expf(y0);
                if (y_out) y_out[r0] = y0;
            }
            if (r1 < n) {
                if (nu_out) nu_out[r1] = expf(y1) < gate ? 0.f : ref * expf(y1);
                if (y_out) y_out[r1] = y1;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// features and labels of the learned sensor for every cell (thread per
// (cell, point)): x = (rho_l/rho_0, |v|hat_l/cs), y = log(max(nu_cell,
// nu_f)/ref), nu_cell = the Gauss-weighted mean of Pi_vNR/(rho |div v|) over
// the compressive points (summed in a fixed order), nu_f = max(beta, 0.05) ref
// the coefficient of the linear term
// ---------------------------------------------------------------------------
template <typename T, int K>
__global__ void __launch_bounds__(Tile<K>::NT) k_features(const T* __restrict__ u, const T* __restrict__ vabs,
                                                          const T* __restrict__ phiv, const T* __restrict__ wq,
                                                          long ncell, Phys ph, double dt, float* __restrict__ X,
                                                          float* __restrict__ Y)
{
    using Dm = Dims<K>;
    constexpr int b = Dm::b, nq = Dm::nq, TC = Tile<K>::TC, NT = Tile<K>::NT, EC = 12;
    __shared__ T s_u[TC][4][b];
    __shared__ T s_ec[TC][b][EC];
    __shared__ T s_phi[b * nq];  // basis at the volume points [b][nq]
    __shared__ T s_nw[TC][nq], s_w[TC][nq];  // w_q nu_q and w_q at compressive points, else 0
    const int tid = threadIdx.x;
    for (int e = tid; e < b * nq; e += NT) s_phi[e] = phiv[e];
    const T two_h = T(2.0 / ph.h);
    const float ref = (float)(ph.cs * ph.hp);
    const long ntile = (ncell + TC - 1) / TC;
    for (long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const long c0 = tile * TC;
        for (int e = tid; e < TC * 4 * b; e += NT) {
            const long c = c0 + e / (4 * b);
            (&s_u[0][0][0])[e] = (c < ncell) ? u[c0 * 4 * b + e] : ((e % (4 * b)) == 0 ? T(1) : T(0));
        }
        __syncthreads();
        for (int e = tid; e < TC * 5; e += NT) {
            const int lc = e / 5, g = e % 5;
            const T* uu = &s_u[lc][0][0];
            T out[b];
            if (g == 0) {
                for (int l = 0; l < b; ++l)
                    for (int v = 0; v < 4; ++v) s_ec[lc][l][v] = uu[v * b + l];
                continue;
            }
            if (g == 1) modal_grad<T, K, 0>(uu, out, two_h);
            if (g == 2) modal_grad<T, K, 1>(uu, out, two_h);
            if (g == 3) modal_grad<T, K, 2>(uu, out, two_h);
            if (g == 4) {
                T t2[b];
                modal_grad<T, K, 0>(uu + b, out, two_h);
                modal_grad<T, K, 1>(uu + 2 * b, t2, two_h);
                for (int l = 0; l < b; ++l) out[l] += t2[l];
                modal_grad<T, K, 2>(uu + 3 * b, t2, two_h);
                for (int l = 0; l < b; ++l) out[l] += t2[l];
            }
            for (int l = 0; l < b; ++l) s_ec[lc][l][3 + g] = out[l];
        }
        __syncthreads();
        static_assert(TC * nq <= NT, "one thread per (cell, point)");
        if (tid < TC * nq) {
            const int lc = tid / nq, q = tid % nq;
            T f[8];
            for (int i = 0; i < 8; ++i) f[i] = T(0);
            for (int l = 0; l < b; ++l) {
                const T p = s_phi[l * nq + q];
                for (int i = 0; i < 8; ++i) f[i] += s_ec[lc][l][i] * p;
            }
            const T rho = f[0], vx = f[1] / rho, vy = f[2] / rho, vz = f[3] / rho;
            const T divv = (f[7] - (vx * f[4] + vy * f[5] + vz * f[6])) / rho;
            T nw = T(0), w = T(0);
            if (divv < T(0)) {
                const T Pi = vnr_pressure<T>(ph, rho, divv, T(dt));
                w = wq[q];
                nw = w * (Pi / (rho * (-divv)));
            }
            s_nw[lc][q] = nw;
            s_w[lc][q] = w;
        }
        __syncthreads();
        for (int e = tid; e < TC * 2 * b; e += NT) {
            const int lc = e / (2 * b), k = e % (2 * b);
            const long c = c0 + lc;
            if (c >= ncell) continue;
            X[c * 2 * b + k] = (k < b) ? (float)(s_u[lc][0][k] / s_u[lc][0][0])
                                       : (float)(vabs[c * b + (k - b)] / T(ph.cs));
        }
        for (int lc = tid; lc < TC; lc += NT) {
            const long c = c0 + lc;
            if (c >= ncell) continue;
            T sn = T(0), sw = T(0);
            for (int q = 0; q < nq; ++q) {
                sn += s_nw[lc][q];
                sw += s_w[lc][q];
            }
            const float nu = sw > T(0) ? (float)(sn / sw) : 0.f;
            const float fl = fmaxf((float)ph.beta, 0.05f) * ref;
            Y[c] = logf(fmaxf(nu, fl) / ref);
        }
        __syncthreads();
    }
}

}  // namespace dg
