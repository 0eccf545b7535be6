// mrsim_adc_grouped_noalloc: the grouped with-ADC signal of one window
// (block sums, then every sample from the block sums) for callers that must
// not allocate device memory.  The block sums live in a file-scope static
// device array instead of an allocation; everything else is the caller's.
#include <mutex>

#include "internal.h"

namespace mrsim {
namespace {

constexpr int kMaxGroups = MRSIM_NOALLOC_MAX_GROUPS;
constexpr int kThreads = 256;

// [0, 2 * kMaxGroups): complex block sums (re, im); the next slot holds the
// "group id out of range" flag.  Every GPU that loads the library keeps this
// array (about 1 MiB) until the process exits.
static __device__ __align__(256) double g_na_scratch[2 * kMaxGroups + 32];

__global__ void k_na_clear(double *blk, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        blk[i] = 0.0;
}

// Block sums: blk[g] += Mx + i My over the isochromats of group g.  A warp
// whose lanes share one group adds once; otherwise every lane adds its own.
__global__ void k_na_blocksum(int64_t K, const float *mx, const float *my, const int32_t *gid,
                              int G, double *blk, int *bad) {
    for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x; k0 < K;
         k0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = k0 + threadIdx.x;
        const bool act = k < K;
        int g = act ? gid[k] : -1;
        const bool ok = act && g >= 0 && g < G;
        if (act && !ok) atomicOr(bad, 1);
        float vr = ok ? mx[k] : 0.0f, vi = ok ? my[k] : 0.0f;
        const unsigned full = 0xffffffffu;
        const int g0 = __shfl_sync(full, g, 0);
        if (__all_sync(full, ok && g == g0)) {
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                vr += __shfl_xor_sync(full, vr, d);
                vi += __shfl_xor_sync(full, vi, d);
            }
            if ((threadIdx.x & 31) == 0) {
                atomicAdd(&blk[2 * g0], (double)vr);
                atomicAdd(&blk[2 * g0 + 1], (double)vi);
            }
        } else if (ok) {
            atomicAdd(&blk[2 * g], (double)vr);
            atomicAdd(&blk[2 * g + 1], (double)vi);
        }
    }
}

__device__ __forceinline__ void split(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// One thread per sample: A(t) = sum_g exp(-tau/T2_g) exp(-i 2 pi (pos_g k +
// dB0_g tau)) A_block(g); partial sums of 256 groups in FP32, total in FP64.
__global__ void __launch_bounds__(kThreads) k_na_signal(const double *blk, int G,
                                                        const float *gpos, const float *gdB0,
                                                        const float *gT2, int64_t n_samples,
                                                        const double *tau, const double *kmom,
                                                        double *signal) {
    __shared__ float s_pos[kThreads], s_dB0[kThreads], s_r2[kThreads], s_ar[kThreads],
        s_ai[kThreads];
    const int64_t s = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    const bool act = s < n_samples;
    float t_hi = 0, t_lo = 0, k_hi = 0, k_lo = 0;
    if (act) {
        split(tau[s], t_hi, t_lo);
        split(kmom[s], k_hi, k_lo);
    }
    const float t = t_hi + t_lo;
    double accr = 0.0, acci = 0.0;
    for (int g0 = 0; g0 < G; g0 += kThreads) {
        const int n = min(kThreads, G - g0);
        __syncthreads();
        if (threadIdx.x < n) {
            const int g = g0 + threadIdx.x;
            s_pos[threadIdx.x] = gpos[g];
            s_dB0[threadIdx.x] = gdB0[g];
            const float T2 = gT2[g];
            s_r2[threadIdx.x] = isinf(T2) ? 0.0f : (float)kLog2e / T2;
            s_ar[threadIdx.x] = (float)blk[2 * g];
            s_ai[threadIdx.x] = (float)blk[2 * g + 1];
        }
        __syncthreads();
        float pr = 0.0f, pi = 0.0f;
        if (act) {
            for (int j = 0; j < n; ++j) {
                float c, sn;
                phasor(turns_prod(s_pos[j], k_hi, k_lo) + turns_prod(s_dB0[j], t_hi, t_lo), c, sn);
                const float e = decay(t, s_r2[j]);
                pr += e * (c * s_ar[j] + sn * s_ai[j]);
                pi += e * (c * s_ai[j] - sn * s_ar[j]);
            }
        }
        accr += (double)pr;
        acci += (double)pi;
    }
    if (act) {
        signal[2 * s] = accr;
        signal[2 * s + 1] = acci;
    }
}

// Device address of the static scratch, looked up once per device with that
// device current (host code may not use the symbol itself as an address).
std::mutex g_na_mu;
double *g_na_ptr[256] = {};

int na_scratch(int dev, double **out) {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (dev < 0 || dev >= 256) return MRSIM_EINVAL;
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return MRSIM_ECUDA;
        }
        g_na_ptr[dev] = (double *)p;
    }
    *out = g_na_ptr[dev];
    return MRSIM_OK;
}

}  // namespace
}  // namespace mrsim

extern "C" int mrsim_adc_grouped_noalloc(int64_t K, const float *d_mx, const float *d_my,
                                         const int32_t *d_gid, int32_t n_groups,
                                         const float *d_gpos, const float *d_gdB0,
                                         const float *d_gT2, int64_t n_samples,
                                         const double *d_tau, const double *d_kmom,
                                         double *d_signal, void *stream) {
    using namespace mrsim;
    if (K < 1 || n_samples < 0 || !d_mx || !d_my || !d_gid || !d_gpos || !d_gdB0 || !d_gT2 ||
        (n_samples > 0 && (!d_tau || !d_kmom || !d_signal)))
        return MRSIM_EINVAL;
    if (n_groups < 1 || n_groups > kMaxGroups) return MRSIM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return MRSIM_ECUDA;
    }
    double *blk = nullptr;
    int rc = na_scratch(dev, &blk);
    if (rc) return rc;
    int *bad = reinterpret_cast<int *>(blk + 2 * kMaxGroups);
    cudaStream_t st = (cudaStream_t)stream;
    // the array keeps the previous call's contents: clear the sums and the flag
    k_na_clear<<<(2 * n_groups + kThreads - 1) / kThreads, kThreads, 0, st>>>(blk, 2 * n_groups);
    k_na_clear<<<1, 32, 0, st>>>(blk + 2 * kMaxGroups, 1);
    const int64_t nb = (K + kThreads - 1) / kThreads;
    k_na_blocksum<<<(unsigned)(nb < 4096 ? nb : 4096), kThreads, 0, st>>>(K, d_mx, d_my, d_gid,
                                                                         n_groups, blk, bad);
    if (n_samples > 0)
        k_na_signal<<<(unsigned)((n_samples + kThreads - 1) / kThreads), kThreads, 0, st>>>(
            blk, n_groups, d_gpos, d_gdB0, d_gT2, n_samples, d_tau, d_kmom, d_signal);
    int h_bad = 0;
    cudaError_t e = cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MRSIM_ECUDA;
    }
    return h_bad ? MRSIM_EINVAL : MRSIM_OK;
}
