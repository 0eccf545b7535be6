// Learned with-RF transitions: a 5 -> 128 -> 128 -> 12 MLP (GELU) per
// slice-selective pulse maps an isochromat group's (z, dB0, b1, T1, T2) to the
// pulse's combined transition [A | b] (Eq. 7).  Everything here is device
// work of the library: training data from the exact FP64 precompute kernel,
// forward / backward / Adam training kernels, inference into the transition
// table, and a validated error grid that sends groups back to exact
// integration where the network's error exceeds the bound.
//
// Precision: the 128 x 128 hidden layer holds 16,384 of the 18,828 weights;
// they are stored in BF16 (FP32 master copies for training) and that layer and
// its two backward products run on the tensor cores (mma.sync m16n8k16, BF16
// inputs, FP32 accumulation).  Its input activations enter as an unevaluated
// sum of two BF16 numbers (hi + lo, two MMAs), so they keep ~16 bits.  The
// 5-wide input layer and the 12-wide output layer are not contraction-shaped;
// they run on FP32 lanes with FP32 weights.
#include <cuda_bf16.h>

#include "internal.h"

namespace mrsim {

namespace {

constexpr int kTS = 64;       // samples per tile
constexpr int kNT = 128;      // threads per tile CTA (4 warps x 16 samples)
constexpr int kH = 128;       // hidden width
constexpr int kIn = 5;
constexpr int kOut = 12;
constexpr int kLdH = kH + 8;  // bf16 row stride of [samples][hidden] tiles
constexpr int kLdT = kTS + 8; // bf16 row stride of [hidden][samples] tiles
constexpr int kLdW = kH + 8;  // bf16 row stride of W2 and W2^T

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

// D += A B for one 16x8x16 tile: A 16x16 row-major, B 16x8 column-major, BF16
// inputs, FP32 accumulators (warp-wide).
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment of rows r0..r0+15, columns k0..k0+15 of a row-major bf16 array
__device__ __forceinline__ void load_a(uint32_t (&a)[4], const __nv_bfloat16 *M, int ld, int r0,
                                       int k0) {
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
    const uint32_t *p0 = reinterpret_cast<const uint32_t *>(M + (r0 + g) * ld + k0 + 2 * t);
    const uint32_t *p1 = reinterpret_cast<const uint32_t *>(M + (r0 + g + 8) * ld + k0 + 2 * t);
    a[0] = p0[0];
    a[1] = p1[0];
    a[2] = p0[4];
    a[3] = p1[4];
}
// B fragment (k0..k0+15) x (n0..n0+7) of a matrix whose column n is stored as
// row n of the bf16 array Mt (so Mt[n][k] = B[k][n])
__device__ __forceinline__ void load_b(uint32_t (&b)[2], const __nv_bfloat16 *Mt, int ld, int n0,
                                       int k0) {
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
    const uint32_t *p = reinterpret_cast<const uint32_t *>(Mt + (n0 + g) * ld + k0 + 2 * t);
    b[0] = p[0];
    b[1] = p[4];
}

struct SurSmem {
    __nv_bfloat16 W2b[kH * kLdW];   // W2[o][i]
    __nv_bfloat16 W2Tb[kH * kLdW];  // W2[o][i] at [i][o]
    __nv_bfloat16 H1b[kTS * kLdH];  // h1[s][i], high part
    union {                          // the forward and backward phases never overlap
        __nv_bfloat16 H1lo[kTS * kLdH];  // h1[s][i] - high part, rounded (forward)
        __nv_bfloat16 dA2b[kTS * kLdH];  // da2[s][o] (backward)
    };
    __nv_bfloat16 H1Tb[kH * kLdT];  // h1[s][i] at [i][s]
    __nv_bfloat16 dA2Tb[kH * kLdT];
    float F[kTS * kH];  // a2, then h2; later da1
    float G[kTS * kH];  // gelu'(a2), then da2
    float W1[kH * kIn], b1[kH], b2[kH], W3[kOut * kH], b3[16];
    float X[kTS * kIn], T[kTS * kOut], dY[kTS * kOut];
    float red[kNT / 32];
};

// weights into shared memory (W2 in BF16; the rest FP32)
__device__ void load_weights(SurSmem &sm, const float *P, const __nv_bfloat16 *W2b_g,
                             const __nv_bfloat16 *W2Tb_g, bool need_T) {
    const int tid = threadIdx.x;
    for (int j = tid; j < kH * kH / 8; j += kNT) {
        const int r = (j * 8) / kH, c = (j * 8) % kH;
        *reinterpret_cast<int4 *>(&sm.W2b[r * kLdW + c]) = reinterpret_cast<const int4 *>(W2b_g)[j];
        if (need_T)
            *reinterpret_cast<int4 *>(&sm.W2Tb[r * kLdW + c]) =
                reinterpret_cast<const int4 *>(W2Tb_g)[j];
    }
    for (int j = tid; j < kH * kIn; j += kNT) sm.W1[j] = P[oW1 + j];
    for (int j = tid; j < kH; j += kNT) {
        sm.b1[j] = P[ob1 + j];
        sm.b2[j] = P[ob2 + j];
    }
    for (int j = tid; j < kOut * kH; j += kNT) sm.W3[j] = P[oW3 + j];
    if (tid < kOut) sm.b3[tid] = P[ob3 + tid];
}

// Forward pass of one tile: h1 (bf16, both layouts), a2 -> F = h2 and
// G = gelu'(a2); outputs y [kTS][12] written to `y` (shared or global).
__device__ void tile_forward(SurSmem &sm, int ns, bool keep_grad) {
    const int tid = threadIdx.x, warp = tid >> 5;
    // layer 1 (FP32): a1 = W1 x + b1, h1 = gelu(a1) rounded to bf16
    for (int j = tid; j < kTS * kH; j += kNT) {
        const int s = j / kH, i = j % kH;
        float a = sm.b1[i];
#pragma unroll
        for (int c = 0; c < kIn; ++c) a = fmaf(sm.W1[i * kIn + c], sm.X[s * kIn + c], a);
        const float h = s < ns ? gelu(a) : 0.0f;
        const __nv_bfloat16 hb = __float2bfloat16_rn(h);
        sm.H1b[s * kLdH + i] = hb;
        sm.H1lo[s * kLdH + i] = __float2bfloat16_rn(h - __bfloat162float(hb));
        sm.H1Tb[i * kLdT + s] = hb;
    }
    __syncthreads();
    // layer 2 on tensor cores: a2[s][o] = sum_i h1[s][i] W2[o][i] + b2[o]
    {
        const int g = (tid & 31) >> 2, t = tid & 3, r0 = warp * 16;
        float acc[16][4];
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const float bl = sm.b2[nt * 8 + 2 * t], bh = sm.b2[nt * 8 + 2 * t + 1];
            acc[nt][0] = bl; acc[nt][1] = bh; acc[nt][2] = bl; acc[nt][3] = bh;
        }
#pragma unroll
        for (int ks = 0; ks < kH / 16; ++ks) {
            uint32_t a[4], al[4];
            load_a(a, sm.H1b, kLdH, r0, ks * 16);
            load_a(al, sm.H1lo, kLdH, r0, ks * 16);
#pragma unroll
            for (int nt = 0; nt < 16; ++nt) {
                uint32_t b[2];
                load_b(b, sm.W2b, kLdW, nt * 8, ks * 16);
                mma16816(acc[nt], a, b);
                mma16816(acc[nt], al, b);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const int c = nt * 8 + 2 * t;
            sm.F[(r0 + g) * kH + c] = acc[nt][0];
            sm.F[(r0 + g) * kH + c + 1] = acc[nt][1];
            sm.F[(r0 + g + 8) * kH + c] = acc[nt][2];
            sm.F[(r0 + g + 8) * kH + c + 1] = acc[nt][3];
        }
    }
    __syncthreads();
    for (int j = tid; j < kTS * kH; j += kNT) {
        const float a = sm.F[j];
        if (keep_grad) sm.G[j] = gelu_grad(a);
        sm.F[j] = gelu(a);
    }
    __syncthreads();
}

// output layer for sample s, output r
__device__ __forceinline__ float out_layer(const SurSmem &sm, int s, int r) {
    float y = sm.b3[r];
    for (int o = 0; o < kH; ++o) y = fmaf(sm.W3[r * kH + o], sm.F[s * kH + o], y);
    return y;
}

__device__ double block_sum(SurSmem &sm, float v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = v;
    __syncthreads();
    double tot = 0;
    for (int w = 0; w < kNT / 32; ++w) tot += sm.red[w];
    __syncthreads();
    return tot;
}

// One training tile: forward, loss, backward; gradients added into `grad`.
// inv_n = 1 / (12 * samples in the whole minibatch).
__global__ void __launch_bounds__(kNT) k_sur_train(const float *P, const __nv_bfloat16 *W2b_g,
                                                   const __nv_bfloat16 *W2Tb_g, const float *X,
                                                   const float *Tgt, int64_t n, float inv_n,
                                                   float *grad, double *loss, float *Yout) {
    extern __shared__ __align__(16) unsigned char raw[];
    SurSmem &sm = *reinterpret_cast<SurSmem *>(raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t s0 = blockIdx.x * (int64_t)kTS;
    const int ns = (int)min((int64_t)kTS, n - s0);
    load_weights(sm, P, W2b_g, W2Tb_g, true);
    for (int j = tid; j < kTS * kIn; j += kNT) sm.X[j] = j < ns * kIn ? X[s0 * kIn + j] : 0.0f;
    for (int j = tid; j < kTS * kOut; j += kNT) sm.T[j] = j < ns * kOut ? Tgt[s0 * kOut + j] : 0.0f;
    __syncthreads();
    tile_forward(sm, ns, true);
    // output layer, residual and dL/dy
    float lsum = 0.0f;
    for (int j = tid; j < kTS * kOut; j += kNT) {
        const int s = j / kOut, r = j % kOut;
        float d = 0.0f;
        if (s < ns) {
            const float y = out_layer(sm, s, r);
            if (Yout) Yout[(s0 + s) * kOut + r] = y;
            const float res = y - sm.T[j];
            lsum += res * res;
            d = 2.0f * res * inv_n;
        }
        sm.dY[j] = d;
    }
    const double ls = block_sum(sm, lsum);
    if (tid == 0 && loss) atomicAdd(loss, ls);
    __syncthreads();
    // dW3[r][o] = sum_s dY[s][r] h2[s][o]; db3[r] = sum_s dY[s][r]
    for (int j = tid; j < kOut * kH; j += kNT) {
        const int r = j / kH, o = j % kH;
        float acc = 0.0f;
        for (int s = 0; s < ns; ++s) acc = fmaf(sm.dY[s * kOut + r], sm.F[s * kH + o], acc);
        atomicAdd(&grad[oW3 + j], acc);
    }
    if (tid < kOut) {
        float acc = 0.0f;
        for (int s = 0; s < ns; ++s) acc += sm.dY[s * kOut + tid];
        atomicAdd(&grad[ob3 + tid], acc);
    }
    // da2[s][o] = (sum_r dY[s][r] W3[r][o]) gelu'(a2[s][o])
    for (int j = tid; j < kTS * kH; j += kNT) {
        const int s = j / kH, o = j % kH;
        float d = 0.0f;
#pragma unroll
        for (int r = 0; r < kOut; ++r) d = fmaf(sm.dY[s * kOut + r], sm.W3[r * kH + o], d);
        d *= sm.G[j];
        sm.G[j] = d;
        const __nv_bfloat16 db = __float2bfloat16_rn(d);
        sm.dA2b[s * kLdH + o] = db;
        sm.dA2Tb[o * kLdT + s] = db;
    }
    __syncthreads();
    if (tid < kH) {
        float acc = 0.0f;
        for (int s = 0; s < ns; ++s) acc += sm.G[s * kH + tid];
        atomicAdd(&grad[ob2 + tid], acc);
    }
    // dh1 = da2 W2 (tensor cores), then da1 = dh1 gelu'(a1) into F
    {
        const int g = (tid & 31) >> 2, t = tid & 3, r0 = warp * 16;
        float acc[16][4];
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < kH / 16; ++ks) {
            uint32_t a[4];
            load_a(a, sm.dA2b, kLdH, r0, ks * 16);
#pragma unroll
            for (int nt = 0; nt < 16; ++nt) {
                uint32_t b[2];
                load_b(b, sm.W2Tb, kLdW, nt * 8, ks * 16);  // B[k=o][n=i] = W2[o][i]
                mma16816(acc[nt], a, b);
            }
        }
        __syncthreads();  // every warp is done reading F (h2) before it becomes da1
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = r0 + g + (q >= 2 ? 8 : 0), i = nt * 8 + 2 * t + (q & 1);
                float a1 = sm.b1[i];
#pragma unroll
                for (int c = 0; c < kIn; ++c) a1 = fmaf(sm.W1[i * kIn + c], sm.X[s * kIn + c], a1);
                sm.F[s * kH + i] = s < ns ? acc[nt][q] * gelu_grad(a1) : 0.0f;
            }
        }
    }
    __syncthreads();
    // dW1[i][c] = sum_s da1[s][i] x[s][c]; db1[i] = sum_s da1[s][i]
    for (int j = tid; j < kH * kIn; j += kNT) {
        const int i = j / kIn, c = j % kIn;
        float acc = 0.0f;
        for (int s = 0; s < ns; ++s) acc = fmaf(sm.F[s * kH + i], sm.X[s * kIn + c], acc);
        atomicAdd(&grad[oW1 + j], acc);
    }
    if (tid < kH) {
        float acc = 0.0f;
        for (int s = 0; s < ns; ++s) acc += sm.F[s * kH + tid];
        atomicAdd(&grad[ob1 + tid], acc);
    }
    // dW2[o][i] = sum_s da2[s][o] h1[s][i] (tensor cores; K = samples)
    {
        const int g = (tid & 31) >> 2, t = tid & 3;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int o0 = warp * 32 + mt * 16;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float acc[8][4];
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
#pragma unroll
                for (int ks = 0; ks < kTS / 16; ++ks) {
                    uint32_t a[4];
                    load_a(a, sm.dA2Tb, kLdT, o0, ks * 16);  // A[m=o][k=s]
#pragma unroll
                    for (int nt = 0; nt < 8; ++nt) {
                        uint32_t b[2];
                        load_b(b, sm.H1Tb, kLdT, (half * 8 + nt) * 8, ks * 16);  // B[k=s][n=i]
                        mma16816(acc[nt], a, b);
                    }
                }
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    const int i = (half * 8 + nt) * 8 + 2 * t;
                    atomicAdd(&grad[oW2 + (o0 + g) * kH + i], acc[nt][0]);
                    atomicAdd(&grad[oW2 + (o0 + g) * kH + i + 1], acc[nt][1]);
                    atomicAdd(&grad[oW2 + (o0 + g + 8) * kH + i], acc[nt][2]);
                    atomicAdd(&grad[oW2 + (o0 + g + 8) * kH + i + 1], acc[nt][3]);
                }
            }
        }
    }
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

static_assert(sizeof(SurSmem) <= 227 * 1024, "tile exceeds the per-CTA shared memory");
static_assert(2 * (sizeof(TcSmem) + 1024) <= 228 * 1024,
              "two inference CTAs must fit an SM's shared memory");
static_assert(kTcRows * (kOut + 1) * sizeof(float) <= kTileBytes, "partials fit one operand tile");
size_t sur_smem() { return sizeof(SurSmem); }

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
    const unsigned grid = (unsigned)((n + kTS - 1) / kTS);
    k_sur_train<<<grid, kNT, sur_smem(), c->stream>>>(
        P, (const __nv_bfloat16 *)W2b, (const __nv_bfloat16 *)W2Tb, X, T, n,
        1.0f / (12.0f * (float)n), grad, loss, Yout);
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
        int occ = 0;
        MRSIM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sur_infer, kTcThreads,
                                                                 sizeof(TcSmem)));
        // persistent CTAs over the tiles (the served count is on the device):
        // every CTA holds 128 of an SM's 512 TMEM columns
        const int64_t tiles = (G + kTcRows - 1) / kTcRows;
        const unsigned grid = (unsigned)std::max<int64_t>(
            1, std::min<int64_t>(tiles, (int64_t)c->sm_count * std::max(std::min(occ, 4), 1)));
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
