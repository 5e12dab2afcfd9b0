// dg_analysis.cu -- turbulence statistics of a state (Sec. 4.1 definitions,
// Sec. 4.3 measurement): the volume-weighted density PDF, the second-order
// velocity structure function, and the velocity sampled on the (k+1)N Fourier
// grid with the shell sums of its power spectrum.  All evaluation in FP64
// from the state's coefficients (FP64 or FP32), accumulation in FP64.
#include "dg_launch.cuh"
#include "dg_launch_impl.cuh"

namespace dg {

// sqrt(2m+1) P_m(x), m = 0..K, by the three-term recurrence
template <int K>
__device__ __forceinline__ void pnorm_all(double x, double* p)
{
    p[0] = 1.0;
    if constexpr (K >= 1) p[1] = x;
#pragma unroll
    for (int m = 2; m <= K; ++m) p[m] = ((2.0 * m - 1.0) * x * p[m - 1] - (m - 1.0) * p[m - 2]) / m;
#pragma unroll
    for (int m = 1; m <= K; ++m) p[m] *= sqrt(2.0 * m + 1.0);
}

// the fields (rho, m_x, m_y, m_z) of one cell at reference point xi
template <typename T, int K>
__device__ __forceinline__ void eval_point(const T* __restrict__ uc, const double xi[3], double f[4])
{
    constexpr int b = Dims<K>::b;
    constexpr Modes<K> M{};
    double px[K + 1], py[K + 1], pz[K + 1];
    pnorm_all<K>(xi[0], px);
    pnorm_all<K>(xi[1], py);
    pnorm_all<K>(xi[2], pz);
    f[0] = f[1] = f[2] = f[3] = 0.0;
    static_for<0, b>([&](auto L) {
        constexpr int l = decltype(L)::value;
        const double ph = px[M.i[l]] * py[M.j[l]] * pz[M.l[l]];
#pragma unroll
        for (int v = 0; v < 4; ++v) f[v] += (double)uc[v * b + l] * ph;
    });
}

// velocity m/rho at a point x of the periodic unit box
template <typename T, int K>
__device__ __forceinline__ void velocity_at(const T* __restrict__ u, int N, const double x[3], double v[3])
{
    int ic[3];
    double xi[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double y = x[d] - floor(x[d]);
        const double s = y * N;
        int i = (int)floor(s);
        if (i >= N) i = N - 1;
        if (i < 0) i = 0;
        ic[d] = i;
        xi[d] = 2.0 * (s - i) - 1.0;
    }
    const long c = ((long)ic[2] * N + ic[1]) * N + ic[0];
    double f[4];
    eval_point<T, K>(u + c * 4 * Dims<K>::b, xi, f);
#pragma unroll
    for (int d = 0; d < 3; ++d) v[d] = f[1 + d] / f[0];
}

// SplitMix64: the n-th output of the sequence started from `seed`, as a
// uniform double in [0, 1) from its top 53 bits
__device__ __forceinline__ double splitmix_u01(unsigned long long seed, unsigned long long n)
{
    unsigned long long z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// mean density (cell means, unit box) -> *mean (accumulated with atomics)
template <typename T, int K>
__global__ void __launch_bounds__(256) k_mean_rho(const T* __restrict__ u, long ncell, double* mean)
{
    constexpr int b = Dims<K>::b;
    __shared__ double s[256];
    double acc = 0.0;
    for (long c = blockIdx.x * 256L + threadIdx.x; c < ncell; c += (long)gridDim.x * 256)
        acc += (double)u[c * 4 * b];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(mean, s[0] / (double)ncell);
}

// volume-weighted histogram of log10(rho / mean) over the Gauss points of
// every cell; each sample carries w_q / 8 / ncell of the volume
template <typename T, int K>
__global__ void __launch_bounds__(256) k_density_pdf(const T* __restrict__ u, long ncell, Rule1 r, const double* mean,
                                                     double lo, double ds, int nbins, double* __restrict__ hist)
{
    constexpr int n = K + 1, nq = n * n * n, b = Dims<K>::b;
    extern __shared__ double s_hist[];
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) s_hist[i] = 0.0;
    __syncthreads();
    const double rm = *mean;
    const long items = ncell * nq;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < items; e += (long)gridDim.x * blockDim.x) {
        const long c = e / nq;
        const int q = (int)(e % nq), a0 = q % n, a1 = (q / n) % n, a2 = q / (n * n);
        const double xi[3] = {r.x[a0], r.x[a1], r.x[a2]};
        double f[4];
        eval_point<T, K>(u + c * 4 * b, xi, f);
        if (!(f[0] > 0.0)) continue;
        const double sv = log10(f[0] / rm);
        const double bin = floor((sv - lo) / ds);
        if (bin >= 0.0 && bin < (double)nbins)
            atomicAdd(&s_hist[(int)bin], r.w[a0] * r.w[a1] * r.w[a2] / 8.0 / (double)ncell);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nbins; i += blockDim.x)
        if (s_hist[i] != 0.0) atomicAdd(&hist[i], s_hist[i]);
}

// structure-function pairs: item = j * npairs + p, five uniforms per item
template <typename T, int K>
__global__ void __launch_bounds__(256) k_structure(const T* __restrict__ u, int N, int nbins, long npairs,
                                                   unsigned long long seed, double lmin, double lmax,
                                                   double* __restrict__ acc)
{
    extern __shared__ double s_acc[];
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) s_acc[i] = 0.0;
    __syncthreads();
    const long items = (long)nbins * npairs;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < items; e += (long)gridDim.x * blockDim.x) {
        const int j = (int)(e / npairs);
        const double l = lmin * pow(lmax / lmin, (j + 0.5) / nbins);
        const unsigned long long n0 = (unsigned long long)e * 5ull;
        double x[3], y[3], va[3], vb[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) x[d] = splitmix_u01(seed, n0 + d);
        const double ct = 2.0 * splitmix_u01(seed, n0 + 3) - 1.0;
        double sp, cp;
        sincospi(2.0 * splitmix_u01(seed, n0 + 4), &sp, &cp);
        const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
        const double dir[3] = {st * cp, st * sp, ct};
#pragma unroll
        for (int d = 0; d < 3; ++d) y[d] = x[d] + l * dir[d];
        velocity_at<T, K>(u, N, x, va);
        velocity_at<T, K>(u, N, y, vb);
        double s = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) s += (va[d] - vb[d]) * (va[d] - vb[d]);
        atomicAdd(&s_acc[j], s);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nbins; i += blockDim.x)
        if (s_acc[i] != 0.0) atomicAdd(&acc[i], s_acc[i]);
}

// velocity component d on the Ng = (K+1) N grid, x_g = (g + 1/2)/Ng:
// out[(gz Ng + gy) Ng + gx]
template <typename T, int K>
__global__ void __launch_bounds__(256) k_sample(const T* __restrict__ u, int N, int d, double* __restrict__ out)
{
    constexpr int p = K + 1, b = Dims<K>::b;
    const int Ng = p * N;
    const long n3 = (long)Ng * Ng * Ng;
    for (long g = blockIdx.x * 256L + threadIdx.x; g < n3; g += (long)gridDim.x * 256) {
        const int gx = (int)(g % Ng), gy = (int)((g / Ng) % Ng), gz = (int)(g / ((long)Ng * Ng));
        const double xi[3] = {(2.0 * (gx % p) + 1.0) / p - 1.0, (2.0 * (gy % p) + 1.0) / p - 1.0,
                              (2.0 * (gz % p) + 1.0) / p - 1.0};
        const long c = ((long)(gz / p) * N + gy / p) * N + gx / p;
        double f[4];
        eval_point<T, K>(u + c * 4 * b, xi, f);
        out[g] = f[1 + d] / f[0];
    }
}

// shell sums of |F|^2 scale^2 over the half spectrum of a real-to-complex
// transform F[gz][gy][kx] (kx = 0..Ng/2); a mode with 0 < kx < Ng/2 stands
// for itself and its conjugate partner.  Bins logarithmic in |kappa|:
// i = floor(log|kappa| / log kmax * nbins), capped at nbins - 1
__global__ void __launch_bounds__(256) k_shell(const double2* __restrict__ F, int Ng, int nbins, double scale2,
                                               int first, double* __restrict__ power, double* __restrict__ ksum,
                                               unsigned long long* __restrict__ count)
{
    extern __shared__ double s_sh[];
    double* s_pow = s_sh;
    double* s_k = s_sh + nbins;
    unsigned long long* s_cnt = reinterpret_cast<unsigned long long*>(s_sh + 2 * nbins);
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
        s_pow[i] = 0.0;
        s_k[i] = 0.0;
        s_cnt[i] = 0ull;
    }
    __syncthreads();
    const int nh = Ng / 2 + 1;
    const long total = (long)Ng * Ng * nh;
    const double lkmax = log(sqrt(3.0) * Ng / 2.0);
    for (long e = blockIdx.x * 256L + threadIdx.x; e < total; e += (long)gridDim.x * 256) {
        const int kx = (int)(e % nh), gy = (int)((e / nh) % Ng), gz = (int)(e / ((long)nh * Ng));
        const int ky = (2 * gy <= Ng) ? gy : gy - Ng, kz = (2 * gz <= Ng) ? gz : gz - Ng;
        const double kk = sqrt((double)kx * kx + (double)ky * ky + (double)kz * kz);
        if (kk == 0.0) continue;
        const double wgt = (kx == 0 || 2 * kx == Ng) ? 1.0 : 2.0;
        int bin = (int)floor(log(kk) / lkmax * nbins);
        if (bin > nbins - 1) bin = nbins - 1;
        if (bin < 0) bin = 0;
        const double2 z = F[e];
        atomicAdd(&s_pow[bin], wgt * (z.x * z.x + z.y * z.y) * scale2);
        if (first) {
            atomicAdd(&s_k[bin], wgt * kk);
            atomicAdd(&s_cnt[bin], (unsigned long long)wgt);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
        if (s_pow[i] != 0.0) atomicAdd(&power[i], s_pow[i]);
        if (first && s_cnt[i]) {
            atomicAdd(&ksum[i], s_k[i]);
            atomicAdd(&count[i], s_cnt[i]);
        }
    }
}

static int grid_of(long items, int nsm)
{
    long g = (items + 255) / 256;
    if (g > 16L * nsm) g = 16L * nsm;
    return g < 1 ? 1 : (int)g;
}

template <typename T, int K>
static cudaError_t pdf_k(const Launch& L, const T* u, double lo, double hi, int nbins, double* mean, double* hist)
{
    k_mean_rho<T, K><<<grid_of(L.ncell, L.nsm), 256, 0, L.st>>>(u, L.ncell, mean);
    const long items = L.ncell * Dims<K>::nq;
    k_density_pdf<T, K><<<grid_of(items, L.nsm), 256, sizeof(double) * nbins, L.st>>>(
        u, L.ncell, L.r1, mean, lo, (hi - lo) / nbins, nbins, hist);
    return cudaGetLastError();
}

template <typename T, int K>
static cudaError_t sfunc_k(const Launch& L, const T* u, int nbins, long npairs, unsigned long long seed, double* acc)
{
    const double lmin = 1.0 / ((K + 1) * (double)L.N), lmax = 0.5;
    k_structure<T, K><<<grid_of((long)nbins * npairs, L.nsm), 256, sizeof(double) * nbins, L.st>>>(
        u, L.N, nbins, npairs, seed, lmin, lmax, acc);
    return cudaGetLastError();
}

template <typename T, int K>
static cudaError_t sample_k(const Launch& L, const T* u, int d, double* out)
{
    const long Ng = (long)(K + 1) * L.N;
    k_sample<T, K><<<grid_of(Ng * Ng * Ng, L.nsm), 256, 0, L.st>>>(u, L.N, d, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_density_pdf(const Launch& L, const T* u, double lo, double hi, int nbins, double* mean,
                               double* hist)
{
    DG_DISPATCH(pdf_k, u, lo, hi, nbins, mean, hist);
}

template <typename T>
cudaError_t launch_structure(const Launch& L, const T* u, int nbins, long npairs, unsigned long long seed, double* acc)
{
    DG_DISPATCH(sfunc_k, u, nbins, npairs, seed, acc);
}

template <typename T>
cudaError_t launch_sample(const Launch& L, const T* u, int d, double* out)
{
    DG_DISPATCH(sample_k, u, d, out);
}

cudaError_t launch_shell(const Launch& L, const void* F, int Ng, int nbins, double scale2, int first, double* power,
                         double* ksum, unsigned long long* count)
{
    const long total = (long)Ng * Ng * (Ng / 2 + 1);
    const size_t sm = (sizeof(double) * 2 + sizeof(unsigned long long)) * nbins;
    k_shell<<<grid_of(total, L.nsm), 256, sm, L.st>>>(static_cast<const double2*>(F), Ng, nbins, scale2, first,
                                                       power, ksum, count);
    return cudaGetLastError();
}

#define DG_ANALYSIS_INSTANTIATE(T)                                                                               \
    template cudaError_t launch_density_pdf<T>(const Launch&, const T*, double, double, int, double*, double*); \
    template cudaError_t launch_structure<T>(const Launch&, const T*, int, long, unsigned long long, double*);   \
    template cudaError_t launch_sample<T>(const Launch&, const T*, int, double*);
DG_ANALYSIS_INSTANTIATE(float)
DG_ANALYSIS_INSTANTIATE(double)

}  // namespace dg
