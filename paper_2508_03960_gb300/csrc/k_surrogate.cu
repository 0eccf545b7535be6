// Learned with-RF transitions: a 5 -> 128 -> 128 -> 12 MLP (GELU) per
// slice-selective pulse maps an isochromat group's (z, dB0, b1, T1, T2) to the
// pulse's combined transition [A | b] (Eq. 7).  Everything here is device
// work of the library: training data from the exact FP64 precompute kernel,
// forward / backward / Adam training kernels, inference into the transition
// table, and a validated error grid that sends groups back to exact
// integration where the network's error exceeds the bound.
//
// Precision: the 128 x 128 hidden layer holds 16,384 of the 18,828 weights;
// they are stored in BF16 (FP32 master copies for training).  That layer and,
// in training, every contraction over the samples of a tile (its two backward
// products and the weight gradients of the other layers) run on the tensor
// cores: tcgen05.mma with BF16 operands in shared memory and FP32 accumulators
// in tensor memory.  The layer's input activations enter as an unevaluated sum
// of two BF16 numbers (hi + lo, two MMAs), so they keep ~16 bits.  The 5-wide
// input layer and the 12-wide output layer of each sample are not
// contraction-shaped; they run on FP32 lanes with FP32 weights.
#include <cuda_bf16.h>

#include "internal.h"

namespace mrsim {

namespace {

constexpr int kH = 128;       // hidden width
constexpr int kIn = 5;
constexpr int kOut = 12;

// flat parameter layout (FP32 master, gradients, Adam moments)
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH,
              oW3 = ob2 + kH, ob3 = oW3 + kOut * kH, kNParams = ob3 + kOut;
static_assert(kNParams == 18828, "parameter count");

// GELU a Phi(a), Phi(a) = (1 + erf(a / sqrt 2)) / 2, with erf from the rational
// approximation of Abramowitz & Stegun, Handbook of Mathematical Functions,
// eq. 7.1.26 (Hastings): for z >= 0, erf(z) = 1 - E(z),
// E(z) = (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-z^2), t = 1 / (1 + p z),
// |error| <= 1.5e-7.  Phi(a) = 1 - E / 2 for a >= 0 and E / 2 below.  About a
// third of the instructions of the library erf; the network is trained and
// evaluated with this same function, and tests compare it with an FP64
// network that uses the exact erf.
struct GeluParts {
    float E;  // E(|a| / sqrt 2)
    float g;  // exp(-a^2 / 2)
};
__device__ __forceinline__ GeluParts gelu_parts(float a) {
    const float z = fabsf(a) * 0.70710678118654752f;
    const float t = __fdividef(1.0f, fmaf(0.3275911f, z, 1.0f));
    float q = fmaf(t, 1.061405429f, -1.453152027f);
    q = fmaf(t, q, 1.421413741f);
    q = fmaf(t, q, -0.284496736f);
    q = fmaf(t, q, 0.254829592f);
    const float g = __expf(-z * z);
    return GeluParts{q * t * g, g};
}
__device__ __forceinline__ float gelu_phi(float a, float E) {
    return a >= 0.0f ? fmaf(-0.5f, E, 1.0f) : 0.5f * E;
}
__device__ __forceinline__ float gelu(float a) { return a * gelu_phi(a, gelu_parts(a).E); }
__device__ __forceinline__ float gelu_grad(float a) {  // Phi(a) + a phi(a)
    const GeluParts p = gelu_parts(a);
    return fmaf(a * 0.39894228040143268f, p.g, gelu_phi(a, p.E));
}

// Adam (bias-corrected); zeroes the gradient and refreshes the BF16 copies
__global__ void k_sur_adam(float *P, float *grad, float *m, float *v, int step, float lr,
                           __nv_bfloat16 *W2b, __nv_bfloat16 *W2Tb) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < kNParams; j += gridDim.x * blockDim.x) {
        const float g = grad[j];
        const float mj = b1 * m[j] + (1.0f - b1) * g;
        const float vj = b2 * v[j] + (1.0f - b2) * g * g;
        m[j] = mj;
        v[j] = vj;
        const float p = P[j] - lr * (mj / c1) / (sqrtf(vj / c2) + eps);
        P[j] = p;
        grad[j] = 0.0f;
        if (j >= oW2 && j < ob2) {
            const int o = (j - oW2) / kH, i = (j - oW2) % kH;
            const __nv_bfloat16 pb = __float2bfloat16_rn(p);
            W2b[o * kH + i] = pb;
            W2Tb[i * kH + o] = pb;
        }
    }
}

__global__ void k_sur_bf16_copies(const float *P, __nv_bfloat16 *W2b, __nv_bfloat16 *W2Tb) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < kH * kH; j += gridDim.x * blockDim.x) {
        const int o = j / kH, i = j % kH;
        const __nv_bfloat16 pb = __float2bfloat16_rn(P[oW2 + j]);
        W2b[o * kH + i] = pb;
        W2Tb[i * kH + o] = pb;
    }
}

// ---------------------------------------------------------------- data ----
// splitmix64 (S. Vigna): a counter-based generator, value i of stream seed
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}
__device__ __forceinline__ double u01(uint64_t seed, uint64_t i) {
    return (double)(splitmix64(seed * 0xd1342543de82ef95ull + i) >> 11) * (1.0 / 9007199254740992.0);
}

// Affine maps of the domain: network features (about [-1, 1]) and validation
// cells, fixed per domain so that training, validation and inference agree.
struct FeatCoef {
    float a[5], c[5];         // f = a v + c, v = z, dB0, b1, log T1, log T2
    double lo[5], hi[5];      // the domain (inclusive)
    double cell_scale[4];     // cells per unit of z, dB0, b1 and log T2
};

FeatCoef feat_coef(const SurDomain &d) {
    FeatCoef k;
    for (int i = 0; i < 5; ++i) {
        const bool lg = i >= 3;
        const double lo = lg ? std::log(d.lo[i]) : d.lo[i], hi = lg ? std::log(d.hi[i]) : d.hi[i];
        k.a[i] = (float)(2.0 / (hi - lo));
        k.c[i] = (float)(-1.0 - 2.0 * lo / (hi - lo));
        k.lo[i] = d.lo[i];
        k.hi[i] = d.hi[i];
    }
    const int nb[3] = {kCellsZ, kCellsB0, kCellsB1};
    for (int i = 0; i < 3; ++i) k.cell_scale[i] = nb[i] / (d.hi[i] - d.lo[i]);
    k.cell_scale[3] = kCellsT2 / (std::log(d.hi[4]) - std::log(d.lo[4]));
    return k;
}

// Features of one group/sample.
__device__ __forceinline__ void features(const FeatCoef &k, double z, double dB0, double b1,
                                         double T1, double T2, float *f) {
    f[0] = fmaf(k.a[0], (float)z, k.c[0]);
    f[1] = fmaf(k.a[1], (float)dB0, k.c[1]);
    f[2] = fmaf(k.a[2], (float)b1, k.c[2]);
    f[3] = fmaf(k.a[3], logf((float)T1), k.c[3]);
    f[4] = fmaf(k.a[4], logf((float)T2), k.c[4]);
}

// Draw n samples uniformly in (z, dB0, b1) and log-uniformly in (T1, T2);
// write the precompute parameter block [5][n] (pos, T1, T2, dB0, b1) and the
// network features [n][5].
__global__ void k_sur_sample(SurDomain d, FeatCoef fc, uint64_t seed, int64_t n, double *par,
                             float *X) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double z = d.lo[0] + (d.hi[0] - d.lo[0]) * u01(seed, 5 * k);
        const double dB0 = d.lo[1] + (d.hi[1] - d.lo[1]) * u01(seed, 5 * k + 1);
        const double b1 = d.lo[2] + (d.hi[2] - d.lo[2]) * u01(seed, 5 * k + 2);
        const double T1 = exp(log(d.lo[3]) + (log(d.hi[3]) - log(d.lo[3])) * u01(seed, 5 * k + 3));
        const double T2 = exp(log(d.lo[4]) + (log(d.hi[4]) - log(d.lo[4])) * u01(seed, 5 * k + 4));
        par[k] = z;
        par[n + k] = T1;
        par[2 * n + k] = T2;
        par[3 * n + k] = dB0;
        par[4 * n + k] = b1;
        features(fc, z, dB0, b1, T1, T2, X + 5 * k);
    }
}

// P(phi) multiplies M_xy by exp(-i phi) (free precession, Eq. 4).  Returns
// P(phi) [A P(phi) | b] for a row-major 3x4 affine [A | b].
__device__ __forceinline__ void precess_affine(double (&T)[12], double phi) {
    double s, c;
    sincos(phi, &s, &c);
    for (int r = 0; r < 3; ++r) {  // A <- A P: columns 0, 1 mix
        const double a0 = T[4 * r], a1 = T[4 * r + 1];
        T[4 * r] = c * a0 - s * a1;
        T[4 * r + 1] = s * a0 + c * a1;
    }
    for (int col = 0; col < 4; ++col) {  // P [A | b]: rows 0, 1 mix
        const double r0 = T[col], r1 = T[4 + col];
        T[col] = c * r0 + s * r1;
        T[4 + col] = -s * r0 + c * r1;
    }
}

// half of the precession angle th = 2 pi (gamma_bar z int Gz dt + dB0 T_pulse)
// of an isochromat at (z, dB0) during the pulse.  The half turn count is
// reduced modulo one, so the result is continuous in z and dB0 (reducing th
// first and halving would jump by pi where th wraps).
__device__ __forceinline__ double pulse_half_angle(const SurPulse &p, double z, double dB0) {
    double half_turns = 0.5 * (kGammaBar * z * p.mz + dB0 * p.dur);
    half_turns -= rint(half_turns);
    return kTwoPi * half_turns;
}

// Exact transitions -> network targets: the core C = P(-th/2) [A P(-th/2) | b]
// removes the precession the slice gradient and dB0 impose during the pulse
// (for an isochromat the pulse does not reach, T = P(th) and C = I), which
// leaves a function of z that varies on the scale of the slice profile.
__global__ void k_sur_core(SurPulse pulse, const double *par, int64_t n, const double *T,
                           float *C) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        double t[12];
        for (int e = 0; e < 12; ++e) t[e] = T[k * 12 + e];
        precess_affine(t, -pulse_half_angle(pulse, par[k], par[3 * n + k]));
        for (int e = 0; e < 12; ++e) C[k * 12 + e] = (float)t[e];
    }
}

__device__ __forceinline__ int cell_of(const FeatCoef &k, double z, double dB0, double b1,
                                       double T2) {
    // (the T2 bin from a float logarithm: validation and gate share this function)
    const double v[4] = {z - k.lo[0], dB0 - k.lo[1], b1 - k.lo[2],
                         (double)logf((float)(T2 / k.lo[4]))};
    const int nb[4] = {kCellsZ, kCellsB0, kCellsB1, kCellsT2};
    int c = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        int q = (int)floor(v[a] * k.cell_scale[a]);
        q = q < 0 ? 0 : (q >= nb[a] ? nb[a] - 1 : q);
        c = c * nb[a] + q;
    }
    return c;
}

// validation: largest |error| of any transition entry per (z, dB0, b1, T2) cell
__global__ void k_sur_cell_error(FeatCoef fc, const double *par, int64_t n, const float *Y,
                                 const float *Tgt, unsigned int *cell_err) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        float e = 0.0f;
        for (int r = 0; r < kOut; ++r) e = fmaxf(e, fabsf(Y[k * kOut + r] - Tgt[k * kOut + r]));
        const int c = cell_of(fc, par[k], par[3 * n + k], par[4 * n + k], par[2 * n + k]);
        atomicMax(&cell_err[c], __float_as_uint(e));
    }
}

// largest |entry| difference of the listed groups (non-negative floats order
// like their bit patterns, so an integer max is a float max)
__global__ void k_sur_served_error(const float *out, const double *exact, const int32_t *idx,
                                   const int32_t *cnt, unsigned int *result) {
    const int64_t n = *cnt;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = idx[i];
        float e = 0.0f;
        for (int r = 0; r < kOut; ++r)
            e = fmaxf(e, (float)fabs((double)out[g * kOut + r] - exact[g * kOut + r]));
        atomicMax(result, __float_as_uint(e));
    }
}

// Gate of the groups of one gradient type: a group is served by the network
// when it lies inside the training domain and in a cell whose validated error
// is within the bound (every group when cell_ok is null); otherwise it is
// listed for exact integration.  Both
// lists are appended with one atomic per warp (order within a list is free:
// every group is computed on its own).
__global__ void k_sur_gate(FeatCoef fc, const unsigned char *cell_ok, const double *par,
                           int64_t G, int32_t *srv, int32_t *fb, int32_t *cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t n_up = (G + 31) / 32 * 32;  // whole warps take part in the ballots
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_up;
         g += (int64_t)gridDim.x * blockDim.x) {
        bool served = false;
        const bool live = g < G;
        if (live && !cell_ok) {
            served = true;
        } else if (live) {
            const double z = par[g], T1 = par[G + g], T2 = par[2 * G + g];
            const double dB0 = par[3 * G + g], b1 = par[4 * G + g];
            const bool inside = z >= fc.lo[0] && z <= fc.hi[0] && dB0 >= fc.lo[1] &&
                                dB0 <= fc.hi[1] && b1 >= fc.lo[2] && b1 <= fc.hi[2] &&
                                T1 >= fc.lo[3] && T1 <= fc.hi[3] && T2 >= fc.lo[4] &&
                                T2 <= fc.hi[4];
            served = inside && cell_ok[cell_of(fc, z, dB0, b1, T2)];
        }
        const unsigned ms = __ballot_sync(0xffffffffu, live && served);
        const unsigned mf = __ballot_sync(0xffffffffu, live && !served);
        int bs = 0, bf = 0;
        if (lane == 0) {
            if (ms) bs = atomicAdd(&cnt[1], __popc(ms));
            if (mf) bf = atomicAdd(&cnt[0], __popc(mf));
        }
        bs = __shfl_sync(0xffffffffu, bs, 0);
        bf = __shfl_sync(0xffffffffu, bf, 0);
        const unsigned below = (1u << lane) - 1u;
        if (live && served) srv[bs + __popc(ms & below)] = (int32_t)g;
        if (live && !served) fb[bf + __popc(mf & below)] = (int32_t)g;
    }
}

// ----------------------------------------------------- tensor-core path ----
// Network inference on the 5th-generation tensor cores (tcgen05): a CTA of
// 256 threads takes tiles of 128 served groups.  Thread (w, l) owns row
// r = 32 (w mod 4) + l of the tile (TMEM lane quadrant w mod 4) and half
// h = w / 4 of the hidden units.
//   layer 1 (FP32 lanes): a1 = W1 x + b1, h1 = gelu(a1), written as BF16
//     hi + lo parts into two K-major operand tiles in shared memory
//   layer 2 (tensor cores): one thread issues 16 tcgen05.mma (M = N = 128,
//     K = 16: hi and lo parts of each 16-wide K step) into a 128-column FP32
//     accumulator in tensor memory, then commits them to an mbarrier
//   epilogue (FP32 lanes): tcgen05.ld of the row's 64 accumulator columns,
//     + b2, gelu, the 12 outputs' partial sums; the two halves of a row are
//     added in shared memory and the transition rebuilt from the core.
// Operand tiles use the no-swizzle K-major canonical layout: 8-row x 16-byte
// core matrices, K-adjacent cores 128 bytes apart (LBO), 8-row groups 2048
// bytes apart (SBO); W2 (the B operand, N x K = output x input) is staged once
// per CTA.  Every mbarrier wait is bounded: on expiry the kernel sets an
// error flag, stops issuing, frees its tensor memory and returns.
constexpr int kTcRows = 128;          // groups per tile (MMA M)
constexpr int kTcThreads = 256;
constexpr int kTileBytes = kTcRows * kH * 2;  // one BF16 128 x 128 operand tile
constexpr int kTmemCols = 128;                // FP32 accumulator columns (N)
constexpr uint64_t kWaitNs = 1000000000ull;   // mbarrier wait limit (1 s)

struct TcSmem {
    __align__(16) unsigned char W2[kTileBytes];   // B operand (core-matrix layout)
    __align__(16) unsigned char Ahi[kTileBytes];  // A operand, h1 high parts
    __align__(16) unsigned char Alo[kTileBytes];  // A operand, h1 low parts
    float4 W1b[kH][2];                 // (w0, w1, w2, w3), (w4, b1, 0, 0) per hidden unit
    float b2[kH];
    float4 W3t[kH][3];                 // W3 transposed: 12 outputs per hidden unit
    float b3[kOut];
    float half_turns[kTcRows];
    int grp[kTcRows];
    unsigned long long mbar;
    uint32_t tmem_base;
};

// byte offset of element (row, k) of a 128 x 128 BF16 tile in the layout above
__device__ __forceinline__ uint32_t core_off(int row, int k) {
    return (uint32_t)((((row >> 3) * (kH / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start, LBO and SBO in 16-byte units,
// descriptor version 1 (bit 46), no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major,
// N = 128 (N >> 3 at bit 17), M = 128 (M >> 4 at bit 24)
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) |
                                ((128u >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdescBf16), "r"(accumulate));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// wait for completion of phase `parity` of an mbarrier, at most kWaitNs
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}

// 32 consecutive accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__global__ void __launch_bounds__(kTcThreads, 2)
    k_sur_infer(const float *P, const __nv_bfloat16 *W2b_g, FeatCoef fc, SurPulse pulse,
                const double *par, int64_t G, const int32_t *srv, const int32_t *cnt,
                float *out, int *err, const float *X, int64_t n_x) {
    extern __shared__ __align__(16) unsigned char tc_raw[];
    TcSmem &sm = *reinterpret_cast<TcSmem *>(tc_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = 32 * (warp & 3) + lane, half = warp >> 2;
    // weights: W2 into the B operand layout (row = output o, k = input i)
    for (int j = tid; j < kH * kH / 8; j += kTcThreads) {
        const int o = (j * 8) / kH, i = (j * 8) % kH;
        *reinterpret_cast<int4 *>(sm.W2 + core_off(o, i)) = reinterpret_cast<const int4 *>(W2b_g)[j];
    }
    for (int i = tid; i < kH; i += kTcThreads) {
        const float *w = P + oW1 + i * kIn;
        sm.W1b[i][0] = make_float4(w[0], w[1], w[2], w[3]);
        sm.W1b[i][1] = make_float4(w[4], P[ob1 + i], 0.0f, 0.0f);
        sm.b2[i] = P[ob2 + i];
        sm.W3t[i][0] = make_float4(P[oW3 + 0 * kH + i], P[oW3 + 1 * kH + i], P[oW3 + 2 * kH + i],
                                   P[oW3 + 3 * kH + i]);
        sm.W3t[i][1] = make_float4(P[oW3 + 4 * kH + i], P[oW3 + 5 * kH + i], P[oW3 + 6 * kH + i],
                                   P[oW3 + 7 * kH + i]);
        sm.W3t[i][2] = make_float4(P[oW3 + 8 * kH + i], P[oW3 + 9 * kH + i],
                                   P[oW3 + 10 * kH + i], P[oW3 + 11 * kH + i]);
    }
    if (tid < kOut) sm.b3[tid] = P[ob3 + tid];
    const uint32_t mbar = smem_u32(&sm.mbar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&sm.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = sm.tmem_base;
    const uint32_t a_hi = smem_u32(sm.Ahi), a_lo = smem_u32(sm.Alo), b_w = smem_u32(sm.W2);
    // X != null: rows are the given features, outputs the network's raw ones
    const int64_t n = X ? n_x : *cnt;
    uint32_t phase = 0;
    bool ok = true;
    // the second half's output partial sums share the low-part operand tile,
    // which the MMAs no longer read once their completion is seen
    float(*part)[kOut + 1] = reinterpret_cast<float(*)[kOut + 1]>(sm.Alo);
    for (int64_t tile = blockIdx.x; tile * kTcRows < n && ok; tile += gridDim.x) {
        // the previous tile's partial sums are read before this tile's operands
        // overwrite them
        __syncthreads();
        const int64_t s = tile * kTcRows + row;
        // features of this row's group and layer 1 for this thread's half
        float f[kIn] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        const bool live = s < n;
        if (live && X) {
#pragma unroll
            for (int c = 0; c < kIn; ++c) f[c] = X[s * kIn + c];
            if (half == 0) {
                sm.grp[row] = (int)s;
                sm.half_turns[row] = 0.0f;
            }
        } else if (live) {
            const int64_t g = srv[s];
            const double z = par[g], T1 = par[G + g], T2 = par[2 * G + g];
            const double dB0 = par[3 * G + g], b1 = par[4 * G + g];
            features(fc, z, dB0, b1, T1, T2, f);
            if (half == 0) {
                sm.grp[row] = (int)g;
                const double h = 0.5 * (kGammaBar * z * pulse.mz + dB0 * pulse.dur);
                sm.half_turns[row] = (float)(h - rint(h));
            }
        } else if (half == 0) {
            sm.grp[row] = -1;
        }
#pragma unroll 1
        for (int k8 = half * 8; k8 < half * 8 + 8; ++k8) {  // 8 hidden units per chunk
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float hv[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int i = k8 * 8 + 2 * q + e;
                    const float4 wa = sm.W1b[i][0], wb = sm.W1b[i][1];
                    float a = wb.y;
                    a = fmaf(wa.x, f[0], a);
                    a = fmaf(wa.y, f[1], a);
                    a = fmaf(wa.z, f[2], a);
                    a = fmaf(wa.w, f[3], a);
                    a = fmaf(wb.x, f[4], a);
                    hv[e] = live ? gelu(a) : 0.0f;
                }
                const __nv_bfloat162 hb = __floats2bfloat162_rn(hv[0], hv[1]);
                const __nv_bfloat162 lb =
                    __floats2bfloat162_rn(hv[0] - __low2float(hb), hv[1] - __high2float(hb));
                hi[q] = *reinterpret_cast<const uint32_t *>(&hb);
                lo[q] = *reinterpret_cast<const uint32_t *>(&lb);
            }
            const uint32_t off = core_off(row, k8 * 8);
            *reinterpret_cast<uint4 *>(sm.Ahi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(sm.Alo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        // operands visible to the tensor cores, previous accumulator reads done
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < kH / 16; ++ks) {
                const uint64_t bd = umma_desc(b_w + ks * 256, 128, 2048);
                umma_bf16(tmem, umma_desc(a_hi + ks * 256, 128, 2048), bd, ks > 0 ? 1u : 0u);
                umma_bf16(tmem, umma_desc(a_lo + ks * 256, 128, 2048), bd, 1u);
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    mbar)
                : "memory");
        }
        // every thread waits; the outcome is made the same for the whole CTA
        ok = __syncthreads_and(mbar_wait(mbar, phase)) != 0;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (!ok) {
            if (tid == 0) atomicOr(err, 1);
            // the MMAs may still be in flight: wait once more (bounded)
            // before the tensor memory is freed below
            mbar_wait(mbar, phase ^ 1u);
            break;
        }
        // epilogue: this thread's 64 columns of its row
        float y[kOut];
#pragma unroll
        for (int r = 0; r < kOut; ++r) y[r] = half == 0 ? sm.b3[r] : 0.0f;
#pragma unroll 1
        for (int c32 = 0; c32 < 2; ++c32) {
            const int col0 = half * 64 + c32 * 32;
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)col0, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int o = col0 + j;
                const float h2 = gelu(v[j] + sm.b2[o]);
                const float4 w0 = sm.W3t[o][0], w1 = sm.W3t[o][1], w2 = sm.W3t[o][2];
                y[0] = fmaf(w0.x, h2, y[0]); y[1] = fmaf(w0.y, h2, y[1]);
                y[2] = fmaf(w0.z, h2, y[2]); y[3] = fmaf(w0.w, h2, y[3]);
                y[4] = fmaf(w1.x, h2, y[4]); y[5] = fmaf(w1.y, h2, y[5]);
                y[6] = fmaf(w1.z, h2, y[6]); y[7] = fmaf(w1.w, h2, y[7]);
                y[8] = fmaf(w2.x, h2, y[8]); y[9] = fmaf(w2.y, h2, y[9]);
                y[10] = fmaf(w2.z, h2, y[10]); y[11] = fmaf(w2.w, h2, y[11]);
            }
        }
        if (half == 1) {
#pragma unroll
            for (int r = 0; r < kOut; ++r) part[row][r] = y[r];
        }
        __syncthreads();
        if (half == 0 && sm.grp[row] >= 0) {  // T = P(th/2) [C_A P(th/2) | C_b]
            float T[kOut];
#pragma unroll
            for (int r = 0; r < kOut; ++r) T[r] = y[r] + part[row][r];
            if (X) {  // raw outputs
                float4 *o = reinterpret_cast<float4 *>(out + (int64_t)sm.grp[row] * kOut);
                o[0] = make_float4(T[0], T[1], T[2], T[3]);
                o[1] = make_float4(T[4], T[5], T[6], T[7]);
                o[2] = make_float4(T[8], T[9], T[10], T[11]);
                continue;
            }
            float sn, cs;
            sincospif(2.0f * sm.half_turns[row], &sn, &cs);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const float a0 = T[4 * r], a1 = T[4 * r + 1];
                T[4 * r] = cs * a0 - sn * a1;
                T[4 * r + 1] = sn * a0 + cs * a1;
            }
#pragma unroll
            for (int col = 0; col < 4; ++col) {
                const float r0 = T[col], r1 = T[4 + col];
                T[col] = cs * r0 + sn * r1;
                T[4 + col] = -sn * r0 + cs * r1;
            }
            float4 *o = reinterpret_cast<float4 *>(out + (int64_t)sm.grp[row] * kOut);
            o[0] = make_float4(T[0], T[1], T[2], T[3]);
            o[1] = make_float4(T[4], T[5], T[6], T[7]);
            o[2] = make_float4(T[8], T[9], T[10], T[11]);
        }
    }
    // the accumulator is free once every thread's loads are done
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
}


// ------------------------------------------------------------- training ----
// One CTA per tile of 128 samples (256 threads; a thread holds one sample row
// and half of its 128 columns, as in inference).  The contractions of the
// minibatch step run on the tensor cores, in four groups of tcgen05.mma (BF16
// operands in the same no-swizzle K-major layout, FP32 accumulators in TMEM),
// each committed to the CTA's mbarrier:
//   forward   D1[s][o] = sum_i h1[s][i] W2[o][i]           (h1 as hi + lo)
//   backward  D2[s][i] = sum_o da2[s][o] W2[o][i]          (dh1)
//             D3[o][j] = sum_s da2[s][o] [h1 | 1][s][j]    (dW2; j = 128: db2)
//             D4[o][r] = sum_s h2[s][o] dY[s][r]           (dW3)
//   then      D5[i][c] = sum_s da1[s][i] [x | 1][s][c]     (dW1; c = 5: db1)
// The elementwise work between them (GELU and its derivative, the 12-wide
// output layer, the loss and dY = dL/dy, da2 = (dY W3) gelu'(a2), da1 = dh1
// gelu'(a1)) runs on the FP32 lanes of the row's thread.  The weight gradients
// of the tile leave TMEM once, as FP32 atomics into `grad`.  TMEM columns: D1
// 0-127, D2 128-255, D3 256-399, D4 416-431, D5 448-463 (every 32-column load
// starts at a multiple of 32); 512 are allocated (the shared memory already
// keeps one CTA per SM).
constexpr int kTrCols = 512;
constexpr int kColD2 = 128, kColD3 = 256, kColD4 = 416, kColD5 = 448;
constexpr int kN3 = kH + 16;             // dW2 operand rows: h1^T, the ones row, zero rows
constexpr int kOp16Bytes = 16 * kH * 2;  // a 16-row operand over K = 128

struct TrSmem {
    __align__(16) unsigned char R0[kTileBytes];  // W2 (B, forward) -> h2^T (A, dW3)
    __align__(16) unsigned char R1[kTileBytes];  // W2^T (B, dh1) -> da1^T (A, dW1)
    __align__(16) unsigned char R2[kTileBytes];  // h1 hi (A, forward) -> da2 (A, dh1)
    __align__(16) unsigned char R3[kTileBytes];  // h1 lo (A, forward) -> da2^T (A, dW2)
    __align__(16) unsigned char R4[kN3 * kH * 2];  // [h1^T; 1; 0] (B, dW2)
    __align__(16) unsigned char R5[kOp16Bytes];  // [dY^T; 0] (B, dW3) -> [x^T; 1; 0] (B, dW1)
    float4 W1b[kH][2];                 // (w0, w1, w2, w3), (w4, b1, 0, 0) per hidden unit
    float b2[kH];
    float4 W3t[kH][3];                 // W3 transposed: 12 outputs per hidden unit
    float b3[kOut];
    float X[kTcRows][kIn];
    float Tg[kTcRows][kOut];
    float dY[kTcRows][kOut];
    float part[kTcRows][kOut + 1];     // second half's output partial sums
    float red[kTcThreads / 32];
    unsigned long long mbar;
    uint32_t tmem_base;
};

// instruction descriptor of kind::f16 (D FP32, A and B BF16, K-major, M = 128)
// for N columns
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16_n(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// D (+)= A B over K = 128 (8 MMAs of K = 16) for A and B in the layout of
// core_off, then (if commit) a commit of everything issued to the mbarrier
__device__ __forceinline__ void umma_k128(uint32_t tmem_d, uint32_t a, uint32_t b, uint32_t n) {
#pragma unroll
    for (int ks = 0; ks < kH / 16; ++ks)
        umma_bf16_n(tmem_d, umma_desc(a + ks * 256, 128, 2048), umma_desc(b + ks * 256, 128, 2048),
                    idesc_bf16(n), ks > 0 ? 1u : 0u);
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            mbar)
        : "memory");
}

// operands written by the threads become visible to the tensor cores, and the
// threads' earlier TMEM loads are ordered before the MMAs issued next
__device__ __forceinline__ void to_tensor_cores() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

__device__ __forceinline__ void st_bf16(unsigned char *base, int row, int k, float v) {
    *reinterpret_cast<__nv_bfloat16 *>(base + core_off(row, k)) = __float2bfloat16_rn(v);
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_sur_train(const float *P, const __nv_bfloat16 *W2b_g, const __nv_bfloat16 *W2Tb_g,
                const float *X, const float *Tgt, int64_t n, float inv_n, float *grad,
                double *loss, float *Yout, int *err) {
    extern __shared__ __align__(16) unsigned char tr_raw[];
    TrSmem &sm = *reinterpret_cast<TrSmem *>(tr_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = 32 * (warp & 3) + lane, half = warp >> 2;
    const int64_t s0 = (int64_t)blockIdx.x * kTcRows;
    const int ns = (int)min((int64_t)kTcRows, n - s0);
    const bool live = row < ns;
    // weights: W2 as (N = o, K = i) and W2^T as (N = i, K = o), both K-major
    for (int j = tid; j < kH * kH / 8; j += kTcThreads) {
        const int r = (j * 8) / kH, k = (j * 8) % kH;
        *reinterpret_cast<int4 *>(sm.R0 + core_off(r, k)) = reinterpret_cast<const int4 *>(W2b_g)[j];
        *reinterpret_cast<int4 *>(sm.R1 + core_off(r, k)) =
            reinterpret_cast<const int4 *>(W2Tb_g)[j];
    }
    for (int i = tid; i < kH; i += kTcThreads) {
        const float *w = P + oW1 + i * kIn;
        sm.W1b[i][0] = make_float4(w[0], w[1], w[2], w[3]);
        sm.W1b[i][1] = make_float4(w[4], P[ob1 + i], 0.0f, 0.0f);
        sm.b2[i] = P[ob2 + i];
        sm.W3t[i][0] = make_float4(P[oW3 + 0 * kH + i], P[oW3 + 1 * kH + i], P[oW3 + 2 * kH + i],
                                   P[oW3 + 3 * kH + i]);
        sm.W3t[i][1] = make_float4(P[oW3 + 4 * kH + i], P[oW3 + 5 * kH + i], P[oW3 + 6 * kH + i],
                                   P[oW3 + 7 * kH + i]);
        sm.W3t[i][2] = make_float4(P[oW3 + 8 * kH + i], P[oW3 + 9 * kH + i],
                                   P[oW3 + 10 * kH + i], P[oW3 + 11 * kH + i]);
    }
    if (tid < kOut) sm.b3[tid] = P[ob3 + tid];
    for (int j = tid; j < kTcRows * kIn; j += kTcThreads) {
        const int s = j / kIn;
        sm.X[s][j - s * kIn] = s < ns ? X[s0 * kIn + j] : 0.0f;
    }
    for (int j = tid; j < kTcRows * kOut; j += kTcThreads) {
        const int s = j / kOut;
        sm.Tg[s][j - s * kOut] = s < ns ? Tgt[s0 * kOut + j] : 0.0f;
    }
    // rows 128.. of the dW2 operand: ones over the tile's samples (db2), zeros
    for (int j = tid; j < (kN3 - kH) * kH; j += kTcThreads) {
        const int r = kH + j / kH, s = j % kH;
        st_bf16(sm.R4, r, s, r == kH && s < ns ? 1.0f : 0.0f);
    }
    const uint32_t mbar = smem_u32(&sm.mbar);
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&sm.tmem_base)),
                     "r"(kTrCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    to_tensor_cores();
    const uint32_t tmem = sm.tmem_base;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const uint32_t r0 = smem_u32(sm.R0), r1 = smem_u32(sm.R1), r2 = smem_u32(sm.R2),
                   r3 = smem_u32(sm.R3), r4 = smem_u32(sm.R4), r5 = smem_u32(sm.R5);
    float x[kIn];
#pragma unroll
    for (int c = 0; c < kIn; ++c) x[c] = sm.X[row][c];
    // a1 = W1 x + b1 of hidden unit i
    auto pre1 = [&](int i) {
        const float4 wa = sm.W1b[i][0], wb = sm.W1b[i][1];
        float a = wb.y;
        a = fmaf(wa.x, x[0], a);
        a = fmaf(wa.y, x[1], a);
        a = fmaf(wa.z, x[2], a);
        a = fmaf(wa.w, x[3], a);
        return fmaf(wb.x, x[4], a);
    };
    // ---- layer 1: h1 = gelu(a1) as BF16 hi + lo (forward A) and hi (dW2 B) ----
#pragma unroll 1
    for (int k8 = half * 8; k8 < half * 8 + 8; ++k8) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float hv[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) hv[e] = live ? gelu(pre1(k8 * 8 + 2 * q + e)) : 0.0f;
            const __nv_bfloat162 hb = __floats2bfloat162_rn(hv[0], hv[1]);
            const __nv_bfloat162 lb =
                __floats2bfloat162_rn(hv[0] - __low2float(hb), hv[1] - __high2float(hb));
            hi[q] = *reinterpret_cast<const uint32_t *>(&hb);
            lo[q] = *reinterpret_cast<const uint32_t *>(&lb);
            *reinterpret_cast<__nv_bfloat16 *>(sm.R4 + core_off(k8 * 8 + 2 * q, row)) = hb.x;
            *reinterpret_cast<__nv_bfloat16 *>(sm.R4 + core_off(k8 * 8 + 2 * q + 1, row)) = hb.y;
        }
        const uint32_t off = core_off(row, k8 * 8);
        *reinterpret_cast<uint4 *>(sm.R2 + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4 *>(sm.R3 + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    to_tensor_cores();
    if (tid == 0) {
        umma_k128(tmem, r2, r0, kH);  // h1 hi W2^T
#pragma unroll
        for (int ks = 0; ks < kH / 16; ++ks)  // + h1 lo W2^T
            umma_bf16_n(tmem, umma_desc(r3 + ks * 256, 128, 2048),
                        umma_desc(r0 + ks * 256, 128, 2048), idesc_bf16(kH), 1u);
        umma_commit(mbar);
    }
    uint32_t phase = 0;
    // every thread waits; the outcome is made the same for the whole CTA; on
    // expiry the kernel flags it, waits once more (bounded) for the MMAs in
    // flight, frees its tensor memory and returns
    auto wait_mma = [&]() {
        const bool ok = __syncthreads_and(mbar_wait(mbar, phase)) != 0;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (!ok && tid == 0) atomicOr(err, 1);
        if (!ok) mbar_wait(mbar, phase ^ 1u);
        return ok;
    };
    bool ok = wait_mma();
    if (ok) {
        // ---- output layer, loss and dY = dL/dy ----
        float y[kOut];
#pragma unroll
        for (int r = 0; r < kOut; ++r) y[r] = half == 0 ? sm.b3[r] : 0.0f;
#pragma unroll 1
        for (int c32 = 0; c32 < 2; ++c32) {
            const int col0 = half * 64 + c32 * 32;
            float v[32];
            tmem_ld32(tmem + lane_base + (uint32_t)col0, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int o = col0 + j;
                const float h2 = gelu(v[j] + sm.b2[o]);
                const float4 w0 = sm.W3t[o][0], w1 = sm.W3t[o][1], w2 = sm.W3t[o][2];
                y[0] = fmaf(w0.x, h2, y[0]); y[1] = fmaf(w0.y, h2, y[1]);
                y[2] = fmaf(w0.z, h2, y[2]); y[3] = fmaf(w0.w, h2, y[3]);
                y[4] = fmaf(w1.x, h2, y[4]); y[5] = fmaf(w1.y, h2, y[5]);
                y[6] = fmaf(w1.z, h2, y[6]); y[7] = fmaf(w1.w, h2, y[7]);
                y[8] = fmaf(w2.x, h2, y[8]); y[9] = fmaf(w2.y, h2, y[9]);
                y[10] = fmaf(w2.z, h2, y[10]); y[11] = fmaf(w2.w, h2, y[11]);
            }
        }
        if (half == 1) {
#pragma unroll
            for (int r = 0; r < kOut; ++r) sm.part[row][r] = y[r];
        }
        __syncthreads();
        float lsum = 0.0f;
        if (half == 0) {
#pragma unroll
            for (int r = 0; r < kOut; ++r) {
                float d = 0.0f;
                if (live) {
                    const float yr = y[r] + sm.part[row][r];
                    if (Yout) Yout[(s0 + row) * kOut + r] = yr;
                    const float res = yr - sm.Tg[row][r];
                    lsum = fmaf(res, res, lsum);
                    d = 2.0f * res * inv_n;
                }
                sm.dY[row][r] = d;
                st_bf16(sm.R5, r, row, d);  // dY^T (B of dW3)
            }
#pragma unroll
            for (int r = kOut; r < 16; ++r) st_bf16(sm.R5, r, row, 0.0f);
        }
        // loss and db3 = sum_s dY[s][r]: warp sums, then one atomic per warp
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, d);
        if (lane == 0) sm.red[warp] = lsum;
        if (half == 0) {
#pragma unroll
            for (int r = 0; r < kOut; ++r) {
                float g = sm.dY[row][r];
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) g += __shfl_xor_sync(0xffffffffu, g, d);
                if (lane == 0 && g != 0.0f) atomicAdd(&grad[ob3 + r], g);
            }
        }
        __syncthreads();
        if (tid == 0 && loss) {
            double t = 0.0;
            for (int w = 0; w < kTcThreads / 32; ++w) t += sm.red[w];
            atomicAdd(loss, t);
        }
        // ---- da2 = (dY W3) gelu'(a2): A of dh1, A^T of dW2; h2^T for dW3 ----
#pragma unroll 1
        for (int c32 = 0; c32 < 2; ++c32) {
            const int col0 = half * 64 + c32 * 32;
            float v[32];
            tmem_ld32(tmem + lane_base + (uint32_t)col0, v);
#pragma unroll 1
            for (int j8 = 0; j8 < 32; j8 += 8) {
                uint32_t pk[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float dv[2];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int j = j8 + 2 * q + e, o = col0 + j;
                        const float a2 = v[j] + sm.b2[o];
                        const GeluParts gp = gelu_parts(a2);
                        const float h2 = a2 * gelu_phi(a2, gp.E);
                        const float gd = fmaf(a2 * 0.39894228040143268f, gp.g, gelu_phi(a2, gp.E));
                        const float4 w0 = sm.W3t[o][0], w1 = sm.W3t[o][1], w2 = sm.W3t[o][2];
                        const float *dy = sm.dY[row];
                        float dz = w0.x * dy[0];
                        dz = fmaf(w0.y, dy[1], dz); dz = fmaf(w0.z, dy[2], dz);
                        dz = fmaf(w0.w, dy[3], dz); dz = fmaf(w1.x, dy[4], dz);
                        dz = fmaf(w1.y, dy[5], dz); dz = fmaf(w1.z, dy[6], dz);
                        dz = fmaf(w1.w, dy[7], dz); dz = fmaf(w2.x, dy[8], dz);
                        dz = fmaf(w2.y, dy[9], dz); dz = fmaf(w2.z, dy[10], dz);
                        dz = fmaf(w2.w, dy[11], dz);
                        dv[e] = dz * gd;
                        st_bf16(sm.R3, o, row, dv[e]);             // da2^T (A of dW2)
                        st_bf16(sm.R0, o, row, live ? h2 : 0.0f);  // h2^T (A of dW3)
                    }
                    const __nv_bfloat162 db = __floats2bfloat162_rn(dv[0], dv[1]);
                    pk[q] = *reinterpret_cast<const uint32_t *>(&db);
                }
                *reinterpret_cast<uint4 *>(sm.R2 + core_off(row, col0 + j8)) =
                    make_uint4(pk[0], pk[1], pk[2], pk[3]);  // da2 (A of dh1)
            }
        }
        to_tensor_cores();
        if (tid == 0) {
            umma_k128(tmem + kColD2, r2, r1, kH);   // dh1 = da2 W2
            umma_k128(tmem + kColD3, r3, r4, kN3);  // [dW2 | db2] = da2^T [h1 | 1]
            umma_k128(tmem + kColD4, r0, r5, 16);   // dW3^T = h2^T dY
            umma_commit(mbar);
        }
        ok = wait_mma();
    }
    if (ok) {
        // ---- da1 = dh1 gelu'(a1): A^T of dW1; [x | 1]^T as its B ----
#pragma unroll 1
        for (int c32 = 0; c32 < 2; ++c32) {
            const int col0 = half * 64 + c32 * 32;
            float v[32];
            tmem_ld32(tmem + lane_base + (uint32_t)(kColD2 + col0), v);
#pragma unroll 4
            for (int j = 0; j < 32; ++j) {
                const int i = col0 + j;
                st_bf16(sm.R1, i, row, live ? v[j] * gelu_grad(pre1(i)) : 0.0f);
            }
        }
        if (half == 0) {
#pragma unroll
            for (int c = 0; c < 16; ++c)
                st_bf16(sm.R5, c, row, !live ? 0.0f : c < kIn ? x[c] : c == kIn ? 1.0f : 0.0f);
        }
        to_tensor_cores();
        if (tid == 0) {
            umma_k128(tmem + kColD5, r1, r5, 16);  // [dW1 | db1] = da1^T [x | 1]
            umma_commit(mbar);
        }
        ok = wait_mma();
    }
    if (ok) {
        // ---- the tile's weight gradients, out of TMEM (row = o or i) ----
        const int m = row;
#pragma unroll 1
        for (int c32 = 0; c32 < 2; ++c32) {  // dW2[m][i], this thread's 64 columns
            const int col0 = half * 64 + c32 * 32;
            float v[32];
            tmem_ld32(tmem + lane_base + (uint32_t)(kColD3 + col0), v);
#pragma unroll 4
            for (int j = 0; j < 32; ++j) atomicAdd(&grad[oW2 + m * kH + col0 + j], v[j]);
        }
        float v[32];
        if (half == 0) {
            tmem_ld32(tmem + lane_base + (uint32_t)kColD4, v);  // dW3[r][m], r < 12
#pragma unroll
            for (int r = 0; r < kOut; ++r) atomicAdd(&grad[oW3 + r * kH + m], v[r]);
        } else {
            tmem_ld32(tmem + lane_base + (uint32_t)(kColD3 + kH), v);  // db2[m]
            atomicAdd(&grad[ob2 + m], v[0]);
            tmem_ld32(tmem + lane_base + (uint32_t)kColD5, v);  // dW1[m][c], db1[m]
#pragma unroll
            for (int c = 0; c < kIn; ++c) atomicAdd(&grad[oW1 + m * kIn + c], v[c]);
            atomicAdd(&grad[ob1 + m], v[kIn]);
        }
    }
    // the accumulators are free once every thread's loads are done
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(kTrCols)
                     : "memory");
    }
}

static_assert(sizeof(TrSmem) <= 227 * 1024, "training tile exceeds the per-CTA shared memory");
static_assert(kColD5 + 32 <= kTrCols && kColD3 + kH + 32 <= kTrCols, "TMEM loads stay allocated");


static_assert(2 * (sizeof(TcSmem) + 1024) <= 228 * 1024,
              "two inference CTAs must fit an SM's shared memory");
static_assert(kTcRows * (kOut + 1) * sizeof(float) <= kTileBytes, "partials fit one operand tile");
size_t sur_smem() { return sizeof(TrSmem); }

}  // namespace

void sur_sample(mrsim_ctx *c, const SurDomain &d, uint64_t seed, int64_t n, double *par, float *X) {
    KScope ks(c, "sur_sample");
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->sm_count * 16);
    k_sur_sample<<<std::max(grid, 1), 256, 0, c->stream>>>(d, feat_coef(d), seed, n, par, X);
}

void sur_core(mrsim_ctx *c, const SurPulse &p, const double *par, int64_t n, const double *T,
              float *C) {
    KScope ks(c, "sur_core");
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->sm_count * 16);
    k_sur_core<<<std::max(grid, 1), 256, 0, c->stream>>>(p, par, n, T, C);
}

void sur_bf16_copies(mrsim_ctx *c, const float *P, void *W2b, void *W2Tb) {
    KScope ks(c, "sur_bf16");
    k_sur_bf16_copies<<<64, 256, 0, c->stream>>>(P, (__nv_bfloat16 *)W2b, (__nv_bfloat16 *)W2Tb);
}

void sur_train_step(mrsim_ctx *c, const float *P, const void *W2b, const void *W2Tb,
                    const float *X, const float *T, int64_t n, float *grad, double *loss,
                    float *Yout) {
    static bool attr = false;
    if (!attr) {
        MRSIM_CUDA(cudaFuncSetAttribute(k_sur_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sur_smem()));
        attr = true;
    }
    KScope ks(c, "sur_train");
    const unsigned grid = (unsigned)((n + kTcRows - 1) / kTcRows);
    k_sur_train<<<grid, kTcThreads, sur_smem(), c->stream>>>(
        P, (const __nv_bfloat16 *)W2b, (const __nv_bfloat16 *)W2Tb, X, T, n,
        1.0f / (12.0f * (float)n), grad, loss, Yout, c->dev_err.as<int>() + kErrWordTensor);
}

void sur_tensor_err_reset(mrsim_ctx *c) {
    MRSIM_CUDA(cudaMemsetAsync(c->dev_err.as<int>() + kErrWordTensor, 0, sizeof(int), c->stream));
}

void sur_tensor_err_check(mrsim_ctx *c) {
    int h = 0;
    MRSIM_CUDA(cudaMemcpyAsync(&h, c->dev_err.as<int>() + kErrWordTensor, sizeof(int),
                               cudaMemcpyDeviceToHost, c->stream));
    MRSIM_CUDA(cudaStreamSynchronize(c->stream));
    if (h) fail(MRSIM_ETIMEOUT, "tensor-core training: a bounded mbarrier wait ran out");
}

void sur_adam(mrsim_ctx *c, float *P, float *grad, float *m, float *v, int step, float lr,
              void *W2b, void *W2Tb) {
    KScope ks(c, "sur_adam");
    k_sur_adam<<<(kNParams + 255) / 256, 256, 0, c->stream>>>(
        P, grad, m, v, step, lr, (__nv_bfloat16 *)W2b, (__nv_bfloat16 *)W2Tb);
}

void sur_cell_error(mrsim_ctx *c, const SurDomain &d, const double *par, int64_t n,
                    const float *Y, const float *T, unsigned int *cell_err) {
    KScope ks(c, "sur_cell_error");
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->sm_count * 16);
    k_sur_cell_error<<<std::max(grid, 1), 256, 0, c->stream>>>(feat_coef(d), par, n, Y, T,
                                                                cell_err);
}

namespace {

// launch of the tensor-core inference kernel over up to G rows; X: features
// of n_x rows (raw outputs), else the served groups listed in srv / cnt
void launch_sur_infer(mrsim_ctx *c, const float *P, const void *W2b, const FeatCoef &fc,
                      const SurPulse &pulse, const double *par, int64_t G, const int32_t *srv,
                      const int32_t *cnt, float *out, const float *X, int64_t n_x) {
    static bool attr = false;
    if (!attr) {
        MRSIM_CUDA(cudaFuncSetAttribute(k_sur_infer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sizeof(TcSmem)));
        // the whole unified L1 / shared array as shared memory: two CTAs per SM
        MRSIM_CUDA(cudaFuncSetAttribute(k_sur_infer,
                                        cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared));
        attr = true;
    }
    int *err = c->dev_err.as<int>() + kErrWordTensor;
    MRSIM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), c->stream));
    {
        KScope ks(c, "sur_infer");
        // persistent CTAs over the tiles (the served count is on the device),
        // two per SM: the kernel is built for that (registers and shared
        // memory are asserted above; each CTA holds 128 of the SM's 512 TMEM
        // columns), so one CTA's FP32 layers overlap the other's MMAs
        const int64_t tiles = (G + kTcRows - 1) / kTcRows;
        const unsigned grid =
            (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)c->sm_count * 2));
        k_sur_infer<<<grid, kTcThreads, sizeof(TcSmem), c->stream>>>(
            P, (const __nv_bfloat16 *)W2b, fc, pulse, par, G, srv, cnt, out, err, X, n_x);
    }
    int h = 0;
    MRSIM_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    MRSIM_CUDA(cudaStreamSynchronize(c->stream));
    if (h) fail(MRSIM_ETIMEOUT, "tensor-core inference: a bounded mbarrier wait ran out");
}

}  // namespace

void sur_infer(mrsim_ctx *c, const float *P, const void *W2b, const SurDomain &d,
               const SurPulse &pulse, const unsigned char *cell_ok, const double *par, int64_t G,
               float *out, int32_t *idx, int32_t *cnt) {
    if (G <= 0) return;
    const FeatCoef fc = feat_coef(d);
    int32_t *fb = idx, *srv = idx + G;
    {
        KScope ks(c, "sur_gate");
        const unsigned grid = (unsigned)std::min<int64_t>((G + 255) / 256, (int64_t)c->sm_count * 16);
        k_sur_gate<<<grid, 256, 0, c->stream>>>(fc, cell_ok, par, G, srv, fb, cnt);
    }
    launch_sur_infer(c, P, W2b, fc, pulse, par, G, srv, cnt + 1, out, nullptr, 0);
}

void sur_infer_raw(mrsim_ctx *c, const float *P, const void *W2b, const float *X, int64_t n,
                   float *Y) {
    if (n <= 0) return;
    launch_sur_infer(c, P, W2b, FeatCoef{}, SurPulse{}, nullptr, n, nullptr, nullptr, Y, X, n);
}

void sur_served_error(mrsim_ctx *c, const float *out, const double *exact, const int32_t *idx,
                      const int32_t *cnt, unsigned int *result) {
    KScope ks(c, "sur_served_error");
    k_sur_served_error<<<c->sm_count * 4, 256, 0, c->stream>>>(out, exact, idx, cnt, result);
}

int sur_n_params() { return kNParams; }

}  // namespace mrsim
