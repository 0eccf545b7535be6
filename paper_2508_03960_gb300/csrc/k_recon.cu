// Cartesian image reconstruction of simulated k-space (the FFT reconstruction
// of the paper's SE / FSE data, "Simulations #1"; EPI sampled on flat-tops
// only is Cartesian after reversing every other line).  Each acquisition line
// is added into its k-space row and columns, then the centred, normalised
// inverse DFT
//   image[y][x] = 1/(N M) sum K[ky][kx] exp(+i 2 pi ((kx - N/2)(x - N/2) / N
//                                                   + (ky - M/2)(y - M/2) / M))
// is taken as a DFT over the rows and then over the columns, in FP64.  The
// phase index (kx - N/2)(x - N/2) mod N is an exact integer, so every twiddle
// is one sincospi of an exact fraction of a turn.
#include <algorithm>

#include "internal.h"

namespace mrsim {

namespace {

constexpr int kMaxReconN = 2048;
constexpr int kReconThreads = 256;

__global__ void k_recon_scatter(int n_lines, int n_ro, int n_pe, const double *sig,
                                const int32_t *row, const int32_t *col0, const int32_t *dir,
                                double *K) {
    const int64_t n = (int64_t)n_lines * n_ro;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(t / n_ro), i = (int)(t - (int64_t)a * n_ro);
        const int col = (int)((((int64_t)col0[a] + (int64_t)dir[a] * i) % n_ro + n_ro) % n_ro);
        const int64_t o = 2 * ((int64_t)row[a] * n_ro + col);
        atomicAdd(&K[o], sig[2 * t]);
        atomicAdd(&K[o + 1], sig[2 * t + 1]);
    }
}

// out[r][x] = scale * sum_k in[r][k] exp(+i 2 pi (k - L/2)(x - L/2) / L) along
// rows of length L (stride 1) when `rows`, else along columns of length L
// (stride W) for every column x of a W-wide array.  Thread: one output.
__global__ void __launch_bounds__(kReconThreads) k_recon_dft(int L, int W, int n_other, bool rows,
                                                             double scale, const double *in,
                                                             double *out) {
    __shared__ double tw[kMaxReconN][2];
    for (int j = threadIdx.x; j < L; j += blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)j / (double)L, &s, &c);
        tw[j][0] = c;
        tw[j][1] = s;
    }
    __syncthreads();
    // output index along the transformed axis (u) and the other axis (v)
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    if (u >= L || v >= n_other) return;
    const int half = L / 2;
    const int64_t uc = u - half;
    double ar = 0.0, ai = 0.0;
    for (int k = 0; k < L; ++k) {
        const int j = (int)((((int64_t)(k - half) * uc) % L + L) % L);
        const int64_t idx = rows ? (int64_t)v * L + k : (int64_t)k * W + v;
        const double xr = in[2 * idx], xi = in[2 * idx + 1];
        ar += xr * tw[j][0] - xi * tw[j][1];
        ai += xr * tw[j][1] + xi * tw[j][0];
    }
    const int64_t o = rows ? (int64_t)v * L + u : (int64_t)u * W + v;
    out[2 * o] = ar * scale;
    out[2 * o + 1] = ai * scale;
}

}  // namespace

}  // namespace mrsim

using namespace mrsim;

extern "C" int mrsim_recon_cartesian(mrsim_ctx *c, int n_lines, int n_ro, int n_pe,
                                     const double *signal, const int32_t *row,
                                     const int32_t *col0, const int8_t *dir, unsigned flags,
                                     double *image) {
    if (!c) return MRSIM_EINVAL;
    CtxScope scope(c);
    try {
        if (!signal || !row || !col0 || !dir || !image) fail(MRSIM_EINVAL, "NULL argument");
        if (n_lines < 1) fail(MRSIM_EINVAL, "n_lines must be positive");
        if (n_ro < 2 || n_pe < 2 || n_ro % 2 || n_pe % 2 || n_ro > kMaxReconN || n_pe > kMaxReconN)
            fail(MRSIM_EINVAL, "n_ro and n_pe must be even and in [2, 2048]");
        std::vector<int32_t> d32(n_lines);
        for (int a = 0; a < n_lines; ++a) {
            if (row[a] < 0 || row[a] >= n_pe) fail(MRSIM_EINVAL, "row outside [0, n_pe)");
            if (col0[a] < 0 || col0[a] >= n_ro) fail(MRSIM_EINVAL, "col0 outside [0, n_ro)");
            if (dir[a] != 1 && dir[a] != -1) fail(MRSIM_EINVAL, "dir must be +1 or -1");
            d32[a] = dir[a];
        }
        MRSIM_CUDA(cudaSetDevice(c->device));
        const bool dev = (flags & MRSIM_PTR_DEVICE) != 0;
        const int64_t ns = (int64_t)n_lines * n_ro, ng = (int64_t)n_pe * n_ro;
        double *K = (double *)scratch(c, 20, 2 * ng * sizeof(double));
        double *T = (double *)scratch(c, 21, 2 * ng * sizeof(double));
        int32_t *lay = (int32_t *)scratch(c, 19, 3 * (size_t)n_lines * sizeof(int32_t));
        upload(c, lay, row, n_lines * sizeof(int32_t));
        upload(c, lay + n_lines, col0, n_lines * sizeof(int32_t));
        upload(c, lay + 2 * n_lines, d32.data(), n_lines * sizeof(int32_t));
        const double *sig = signal;
        if (!dev) {
            double *hs = (double *)scratch(c, 22, 2 * ns * sizeof(double));
            upload(c, hs, signal, 2 * ns * sizeof(double));
            sig = hs;
        }
        MRSIM_CUDA(cudaMemsetAsync(K, 0, 2 * ng * sizeof(double), c->stream));
        {
            KScope ks(c, "recon_scatter");
            const int blocks = (int)std::max<int64_t>(
                1, std::min<int64_t>((ns + 255) / 256, (int64_t)c->sm_count * 8));
            k_recon_scatter<<<blocks, 256, 0, c->stream>>>(n_lines, n_ro, n_pe, sig, lay,
                                                           lay + n_lines, lay + 2 * n_lines, K);
        }
        double *out = dev ? image : K;
        {
            KScope ks(c, "recon_dft_rows");
            dim3 g((n_ro + kReconThreads - 1) / kReconThreads, n_pe);
            k_recon_dft<<<g, kReconThreads, 0, c->stream>>>(n_ro, n_ro, n_pe, true, 1.0, K, T);
        }
        {
            KScope ks(c, "recon_dft_cols");
            dim3 g((n_pe + kReconThreads - 1) / kReconThreads, n_ro);
            k_recon_dft<<<g, kReconThreads, 0, c->stream>>>(
                n_pe, n_ro, n_ro, false, 1.0 / ((double)n_ro * (double)n_pe), T, out);
        }
        if (!dev)
            MRSIM_CUDA(cudaMemcpyAsync(image, K, 2 * ng * sizeof(double), cudaMemcpyDeviceToHost,
                                       c->stream));
        sync(c);
        c->err.clear();
        return MRSIM_OK;
    } catch (const Error &e) {
        c->err = e.msg;
        return e.code;
    } catch (const std::exception &e) {
        c->err = e.what();
        return MRSIM_EINVAL;
    }
}
