// Plain (per-isochromat) kernels: the conventional method the grouped form is
// measured against, and the fallback for subsequences of no known gradient
// type (Sec. 3.1).
//
//  k_plain_rf     Eq. 3 with U = D R (App. A): every isochromat steps through
//                 a with-RF subsequence with M held in registers; the waveform
//                 is staged through shared memory and broadcast to all lanes.
//  k_plain_adc    Eq. 6 per sample: M_xy of every isochromat from a phasor
//                 recurrence inside constant-gradient segments (anchored by an
//                 exactly computed 32-step phasor), summed over the CTA with
//                 warp shuffles and FP64 per-warp accumulators, then one FP64
//                 atomic per (CTA, sample).
//  k_advance      Eqs. 4-5 over the RF-free time between two events.
//  k_plain_rf_affine / k_apply_affine
//                 combined transition per isochromat (Eq. 7) built once per
//                 distinct with-RF content and reused (dynamic caching).
#include "internal.h"

namespace mrsim {

namespace {

constexpr int kThreads = 256;
constexpr int kSegChunk = 128;
constexpr int kAdcBlockSamples = 256;  // samples per CTA row of accumulators
constexpr int kAnchor = 32;            // recurrence steps between exact anchors

template <typename R>
struct Seg;
template <>
struct Seg<float> { using RF = RFSegF; using ADC = ADCSegF; using Adv = AdvF; };
template <>
struct Seg<double> { using RF = RFSegD; using ADC = ADCSegD; using Adv = AdvD; };

template <typename R>
__device__ __forceinline__ R inv_or_zero(float T) {
    return isinf(T) ? (R)0 : (R)1 / (R)T;
}

struct IsoParams {
    float x, y, z, T1, T2, dB0, M0, b1;
};

__device__ __forceinline__ IsoParams load_iso(const PlainState &s, int64_t k) {
    IsoParams p;
    p.x = s.x[k]; p.y = s.y[k]; p.z = s.z[k];
    p.T1 = s.T1[k]; p.T2 = s.T2[k]; p.dB0 = s.dB0[k]; p.M0 = s.M0[k];
    p.b1 = s.b1 ? s.b1[k] : 1.0f;
    return p;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_init_state(PlainState s, const float *M_init) {
    R *Mx = (R *)s.Mx, *My = (R *)s.My, *Mz = (R *)s.Mz;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < s.K;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (M_init) {
            Mx[k] = M_init[k];
            My[k] = M_init[s.K + k];
            Mz[k] = M_init[2 * s.K + k];
        } else {
            Mx[k] = 0;
            My[k] = 0;
            Mz[k] = s.M0[k];
        }
    }
}

template <typename R, int NI>
__global__ void __launch_bounds__(kThreads) k_plain_rf(PlainState s, const typename Seg<R>::RF *segs,
                                                       int n_seg, typename Seg<R>::Adv adv) {
    using RFS = typename Seg<R>::RF;
    __shared__ RFS sseg[kSegChunk];
    R *Mx = (R *)s.Mx, *My = (R *)s.My, *Mz = (R *)s.Mz;
    const int64_t base = blockIdx.x * (int64_t)(kThreads * NI) + threadIdx.x;
    R mx[NI], my[NI], mz[NI], M0[NI], x[NI], y[NI], z[NI], dB0[NI], b1[NI], iT1[NI], iT2[NI];
    R em1[NI], em2[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        int64_t k = base + (int64_t)i * kThreads;
        if (k < s.K) {
            IsoParams p = load_iso(s, k);
            mx[i] = Mx[k]; my[i] = My[k]; mz[i] = Mz[k];
            M0[i] = p.M0; x[i] = p.x; y[i] = p.y; z[i] = p.z; dB0[i] = p.dB0; b1[i] = p.b1;
            iT1[i] = inv_or_zero<R>(p.T1);
            iT2[i] = inv_or_zero<R>(p.T2);
        } else {
            mx[i] = my[i] = mz[i] = M0[i] = x[i] = y[i] = z[i] = dB0[i] = b1[i] = 0;
            iT1[i] = iT2[i] = 0;
        }
        // free precession from the state time to the pulse start (Eqs. 4-5)
        advance<R>(mx[i], my[i], mz[i], M0[i], x[i], y[i], z[i], dB0[i], iT1[i] * (R)kLog2e,
                   iT2[i] * (R)kLog2e, adv);
        em1[i] = em2[i] = 0;
    }
    R dt_prev = (R)-1;
    for (int c0 = 0; c0 < n_seg; c0 += kSegChunk) {
        const int nc = min(kSegChunk, n_seg - c0);
        __syncthreads();
        for (int j = threadIdx.x; j < nc; j += kThreads) sseg[j] = segs[c0 + j];
        __syncthreads();
        for (int j = 0; j < nc; ++j) {
            const RFS g = sseg[j];
            if ((R)g.dt != dt_prev) {
                dt_prev = (R)g.dt;
#pragma unroll
                for (int i = 0; i < NI; ++i) {
                    em1[i] = expm1(-dt_prev * iT1[i]);
                    em2[i] = expm1(-dt_prev * iT2[i]);
                }
            }
            R px[NI], py[NI], pz[NI];
#pragma unroll
            for (int i = 0; i < NI; ++i) {
                px[i] = -b1[i] * (R)g.are;
                py[i] = -b1[i] * (R)g.aim;
                pz[i] = -((R)g.cx * x[i] + (R)g.cy * y[i] + (R)g.cz * z[i] + (R)g.cdw * dB0[i]);
            }
            for (int r = 0; r < (int)g.rep; ++r) {
#pragma unroll
                for (int i = 0; i < NI; ++i)
                    rf_step<R>(mx[i], my[i], mz[i], M0[i], px[i], py[i], pz[i], em1[i], em2[i]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        int64_t k = base + (int64_t)i * kThreads;
        if (k < s.K) {
            Mx[k] = mx[i];
            My[k] = my[i];
            Mz[k] = mz[i];
        }
    }
}

template <typename R>
__device__ __forceinline__ void cmul(R &ar, R &ai, R br, R bi) {
    R r = ar * br - ai * bi;
    R i = ar * bi + ai * br;
    ar = r;
    ai = i;
}

// per-sub-step phasor E2(dt) exp(-i 2 pi (x kx + y ky + z kz + dB0 dt)) and
// its exact B-th power (hi/lo moments scaled by B, a power of two)
__device__ __forceinline__ void seg_phasors(const ADCSegF &g, float x, float y, float z,
                                            float dB0, float rT2, float &z1r, float &z1i,
                                            float &zbr, float &zbi) {
    AdvF a1{g.kx_hi, g.kx_lo, g.ky_hi, g.ky_lo, g.kz_hi, g.kz_lo, g.dt, 0.0f};
    const float B = (float)kAnchor;
    AdvF ab{g.kx_hi * B, g.kx_lo * B, g.ky_hi * B, g.ky_lo * B, g.kz_hi * B, g.kz_lo * B,
            g.dt * B, 0.0f};
    float c, s;
    phasor(adv_turns(a1, x, y, z, dB0), c, s);
    float e = decay(g.dt, rT2);
    z1r = e * c;
    z1i = -e * s;
    phasor(adv_turns(ab, x, y, z, dB0), c, s);
    e = decay(g.dt * B, rT2);
    zbr = e * c;
    zbi = -e * s;
}
__device__ __forceinline__ void seg_phasors(const ADCSegD &g, double x, double y, double z,
                                            double dB0, double rT2, double &z1r, double &z1i,
                                            double &zbr, double &zbi) {
    AdvD a1{g.kx, g.ky, g.kz, g.dt};
    const double B = (double)kAnchor;
    AdvD ab{g.kx * B, g.ky * B, g.kz * B, g.dt * B};
    double c, s;
    phasor(adv_turns(a1, x, y, z, dB0), c, s);
    double e = decay(g.dt, rT2);
    z1r = e * c;
    z1i = -e * s;
    phasor(adv_turns(ab, x, y, z, dB0), c, s);
    e = decay(g.dt * B, rT2);
    zbr = e * c;
    zbi = -e * s;
}

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

template <typename R, int NI>
__global__ void __launch_bounds__(kThreads) k_plain_adc(PlainState s,
                                                        const typename Seg<R>::ADC *segs,
                                                        int n_seg, int64_t n_samples,
                                                        typename Seg<R>::Adv adv,
                                                        double *signal) {
    using ADS = typename Seg<R>::ADC;
    // per-warp sums of each sample: added in R by lane 0 (accw) and folded into
    // FP64 (acc) by the whole warp every kFoldChunks chunks.  A per-sample FP64
    // add by one lane would keep the FP64 pipe, which this GPU has little of,
    // busier than all the FP32 work of the recurrence.
    __shared__ double acc[kThreads / 32][kAdcBlockSamples][2];
    __shared__ R accw[kThreads / 32][sizeof(R) == 4 ? kAdcBlockSamples : 1][2];
    constexpr int kFoldChunks = 8;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t s_lo = (int64_t)blockIdx.y * kAdcBlockSamples;
    const int64_t s_hi = min(s_lo + kAdcBlockSamples, n_samples);
    for (int t = threadIdx.x; t < kAdcBlockSamples; t += kThreads)
        for (int w = 0; w < kThreads / 32; ++w) acc[w][t][0] = acc[w][t][1] = 0.0;
    if constexpr (sizeof(R) == 4)
        for (int t = threadIdx.x; t < kAdcBlockSamples; t += kThreads)
            for (int w = 0; w < kThreads / 32; ++w) accw[w][t][0] = accw[w][t][1] = 0.0f;
    __syncthreads();
    auto fold = [&]() {
        if constexpr (sizeof(R) == 4) {
            __syncwarp();
            for (int t = lane; t < (int)(s_hi - s_lo); t += 32) {
                acc[wid][t][0] += (double)accw[wid][t][0];
                acc[wid][t][1] += (double)accw[wid][t][1];
                accw[wid][t][0] = 0.0f;
                accw[wid][t][1] = 0.0f;
            }
            __syncwarp();
        }
    };
    int since_fold = 0;
    const R *Mx = (const R *)s.Mx, *My = (const R *)s.My;
    const int64_t chunk = (int64_t)kThreads * NI;
    const int64_t n_chunks = (s.K + chunk - 1) / chunk;
    for (int64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        R cr[NI], ci[NI], x[NI], y[NI], z[NI], dB0[NI], rT2[NI];
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            int64_t k = ch * chunk + (int64_t)i * kThreads + threadIdx.x;
            if (k < s.K) {
                x[i] = s.x[k]; y[i] = s.y[k]; z[i] = s.z[k]; dB0[i] = s.dB0[k];
                rT2[i] = inv_or_zero<R>(s.T2[k]) * (R)kLog2e;
                advance_xy<R>(Mx[k], My[k], x[i], y[i], z[i], dB0[i], rT2[i], adv, cr[i], ci[i]);
                // receive coil (Eq. 6): S is constant in time and the sample
                // recurrence below is linear, so weighting the start weights
                // every sample of the window
                if (s.coil_re) cmul(cr[i], ci[i], (R)s.coil_re[k], (R)s.coil_im[k]);
            } else {
                cr[i] = ci[i] = x[i] = y[i] = z[i] = dB0[i] = rT2[i] = 0;
            }
        }
        int64_t smp = 0;
        for (int sg = 0; sg < n_seg && smp < s_hi; ++sg) {
            const ADS g = segs[sg];
            const int64_t rep = (int64_t)g.rep;
            if (smp + rep <= s_lo) {  // whole segment before this CTA's samples: jump
                // exact jump by rep sub-steps: scale the per-step moments by rep
#pragma unroll
                for (int i = 0; i < NI; ++i) {
                    R z1r, z1i, zbr, zbi;
                    seg_phasors(g, x[i], y[i], z[i], dB0[i], rT2[i], z1r, z1i, zbr, zbi);
                    for (int64_t r = 0; r < rep; ++r) cmul(cr[i], ci[i], z1r, z1i);
                }
                smp += rep;
                continue;
            }
            R z1r[NI], z1i[NI], zbr[NI], zbi[NI], ar[NI], ai[NI];
#pragma unroll
            for (int i = 0; i < NI; ++i) {
                seg_phasors(g, x[i], y[i], z[i], dB0[i], rT2[i], z1r[i], z1i[i], zbr[i], zbi[i]);
                ar[i] = cr[i];
                ai[i] = ci[i];
            }
            for (int64_t r0 = 0; r0 < rep; r0 += kAnchor) {
                const int nb = (int)min((int64_t)kAnchor, rep - r0);
#pragma unroll
                for (int i = 0; i < NI; ++i) { cr[i] = ar[i]; ci[i] = ai[i]; }
                for (int q = 0; q < nb; ++q, ++smp) {
                    R vr = 0, vi = 0;
#pragma unroll
                    for (int i = 0; i < NI; ++i) {
                        cmul(cr[i], ci[i], z1r[i], z1i[i]);
                        vr += cr[i];
                        vi += ci[i];
                    }
                    if (smp >= s_lo && smp < s_hi) {
                        vr = warp_sum(vr);
                        vi = warp_sum(vi);
                        if (lane == 0) {
                            if constexpr (sizeof(R) == 4) {
                                accw[wid][smp - s_lo][0] += vr;
                                accw[wid][smp - s_lo][1] += vi;
                            } else {
                                acc[wid][smp - s_lo][0] += (double)vr;
                                acc[wid][smp - s_lo][1] += (double)vi;
                            }
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < NI; ++i) cmul(ar[i], ai[i], zbr[i], zbi[i]);
            }
        }
        if (++since_fold == kFoldChunks) {
            fold();
            since_fold = 0;
        }
    }
    fold();
    __syncthreads();
    for (int t = threadIdx.x; t < (int)(s_hi - s_lo); t += kThreads) {
        double sr = 0, si = 0;
        for (int w = 0; w < kThreads / 32; ++w) {
            sr += acc[w][t][0];
            si += acc[w][t][1];
        }
        sum_add(&signal[2 * (s_lo + t)], sr, s.fx);
        sum_add(&signal[2 * (s_lo + t) + 1], si, s.fx);
    }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_advance(PlainState s, typename Seg<R>::Adv adv) {
    R *Mx = (R *)s.Mx, *My = (R *)s.My, *Mz = (R *)s.Mz;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < s.K;
         k += (int64_t)gridDim.x * blockDim.x) {
        R mx = Mx[k], my = My[k], mz = Mz[k];
        advance<R>(mx, my, mz, (R)s.M0[k], (R)s.x[k], (R)s.y[k], (R)s.z[k], (R)s.dB0[k],
                   inv_or_zero<R>(s.T1[k]) * (R)kLog2e, inv_or_zero<R>(s.T2[k]) * (R)kLog2e, adv);
        Mx[k] = mx;
        My[k] = my;
        Mz[k] = mz;
    }
}

// per-isochromat combined transition (Eq. 7) of one with-RF content, stored
// as 12 planes [row-major 3x4 entry][K]
template <typename R>
__global__ void __launch_bounds__(kThreads) k_plain_rf_affine(PlainState s,
                                                              const typename Seg<R>::RF *segs,
                                                              int n_seg, R *cache) {
    using RFS = typename Seg<R>::RF;
    __shared__ RFS sseg[kSegChunk];
    const int64_t k = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    const bool ok = k < s.K;
    IsoParams p{};
    if (ok) p = load_iso(s, k);
    const R iT1 = ok ? inv_or_zero<R>(p.T1) : (R)0, iT2 = ok ? inv_or_zero<R>(p.T2) : (R)0;
    // columns of [A | b]: unit vectors with M0 = 0, and the zero vector with M0 = 1
    R cx[4] = {1, 0, 0, 0}, cy[4] = {0, 1, 0, 0}, cz[4] = {0, 0, 1, 0};
    R em1 = 0, em2 = 0, dt_prev = (R)-1;
    for (int c0 = 0; c0 < n_seg; c0 += kSegChunk) {
        const int nc = min(kSegChunk, n_seg - c0);
        __syncthreads();
        for (int j = threadIdx.x; j < nc; j += kThreads) sseg[j] = segs[c0 + j];
        __syncthreads();
        for (int j = 0; j < nc; ++j) {
            const RFS g = sseg[j];
            if ((R)g.dt != dt_prev) {
                dt_prev = (R)g.dt;
                em1 = expm1(-dt_prev * iT1);
                em2 = expm1(-dt_prev * iT2);
            }
            const R px = -(R)p.b1 * (R)g.are, py = -(R)p.b1 * (R)g.aim;
            const R pz = -((R)g.cx * (R)p.x + (R)g.cy * (R)p.y + (R)g.cz * (R)p.z +
                           (R)g.cdw * (R)p.dB0);
            for (int r = 0; r < (int)g.rep; ++r) {
#pragma unroll
                for (int col = 0; col < 4; ++col)
                    rf_step<R>(cx[col], cy[col], cz[col], col == 3 ? (R)1 : (R)0, px, py, pz,
                               em1, em2);
            }
        }
    }
    if (ok) {
#pragma unroll
        for (int col = 0; col < 4; ++col) {
            cache[(0 * 4 + col) * s.K + k] = cx[col];
            cache[(1 * 4 + col) * s.K + k] = cy[col];
            cache[(2 * 4 + col) * s.K + k] = cz[col];
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_apply_affine(PlainState s, const R *cache,
                                                           typename Seg<R>::Adv adv) {
    R *Mx = (R *)s.Mx, *My = (R *)s.My, *Mz = (R *)s.Mz;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < s.K;
         k += (int64_t)gridDim.x * blockDim.x) {
        R mx = Mx[k], my = My[k], mz = Mz[k];
        const R M0 = s.M0[k];
        advance<R>(mx, my, mz, M0, (R)s.x[k], (R)s.y[k], (R)s.z[k], (R)s.dB0[k],
                   inv_or_zero<R>(s.T1[k]) * (R)kLog2e, inv_or_zero<R>(s.T2[k]) * (R)kLog2e, adv);
        R T[12];
#pragma unroll
        for (int e = 0; e < 12; ++e) T[e] = cache[e * s.K + k];
        Mx[k] = T[0] * mx + T[1] * my + T[2] * mz + T[3] * M0;
        My[k] = T[4] * mx + T[5] * my + T[6] * mz + T[7] * M0;
        Mz[k] = T[8] * mx + T[9] * my + T[10] * mz + T[11] * M0;
    }
}

template <typename R>
__global__ void k_gather_out(int64_t K, const R *Mx, const R *My, const R *Mz,
                             const int32_t *perm, float *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < K;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = perm ? perm[i] : i;
        out[k] = (float)Mx[i];
        out[K + k] = (float)My[i];
        out[2 * K + k] = (float)Mz[i];
    }
}

int grid_stride_blocks(mrsim_ctx *c, int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)c->sm_count * 16));
}

}  // namespace

template <typename R>
void launch_init_state(mrsim_ctx *c, const PlainState &s, const float *M_init) {
    KScope ks(c, "init_state");
    k_init_state<R><<<grid_stride_blocks(c, s.K), kThreads, 0, c->stream>>>(s, M_init);
}

template <typename R>
void launch_plain_rf(mrsim_ctx *c, const PlainState &s, const void *segs, int n_seg,
                     const void *adv, int ni) {
    using RFS = typename Seg<R>::RF;
    using A = typename Seg<R>::Adv;
    const A a = *(const A *)adv;
    KScope ks(c, sizeof(R) == 4 ? "plain_rf_f32" : "plain_rf_f64");
    if (ni >= 2) {
        unsigned nb = (unsigned)((s.K + kThreads * 2 - 1) / (kThreads * 2));
        k_plain_rf<R, 2><<<nb, kThreads, 0, c->stream>>>(s, (const RFS *)segs, n_seg, a);
    } else {
        unsigned nb = (unsigned)((s.K + kThreads - 1) / kThreads);
        k_plain_rf<R, 1><<<nb, kThreads, 0, c->stream>>>(s, (const RFS *)segs, n_seg, a);
    }
}

template <typename R>
void launch_plain_adc(mrsim_ctx *c, const PlainState &s, const void *segs, int n_seg,
                      int64_t n_samples, const void *adv, double *signal, int ctas_per_sm) {
    using ADS = typename Seg<R>::ADC;
    using A = typename Seg<R>::Adv;
    const A a = *(const A *)adv;
    constexpr int NI = 8;
    const int64_t chunk = (int64_t)kThreads * NI;
    const int64_t n_chunks = (s.K + chunk - 1) / chunk;
    dim3 grid((unsigned)std::max<int64_t>(
                  1, std::min<int64_t>(n_chunks, (int64_t)std::max(1, ctas_per_sm) * c->sm_count)),
              (unsigned)((n_samples + kAdcBlockSamples - 1) / kAdcBlockSamples));
    KScope ks(c, sizeof(R) == 4 ? "plain_adc_f32" : "plain_adc_f64");
    k_plain_adc<R, NI><<<grid, kThreads, 0, c->stream>>>(s, (const ADS *)segs, n_seg, n_samples,
                                                        a, signal);
}

template <typename R>
void launch_advance(mrsim_ctx *c, const PlainState &s, const void *adv) {
    using A = typename Seg<R>::Adv;
    KScope ks(c, "advance");
    k_advance<R><<<grid_stride_blocks(c, s.K), kThreads, 0, c->stream>>>(s, *(const A *)adv);
}

template <typename R>
void launch_plain_rf_affine(mrsim_ctx *c, const PlainState &s, const void *segs, int n_seg,
                            R *cache) {
    using RFS = typename Seg<R>::RF;
    KScope ks(c, "plain_rf_affine");
    unsigned nb = (unsigned)((s.K + kThreads - 1) / kThreads);
    k_plain_rf_affine<R><<<nb, kThreads, 0, c->stream>>>(s, (const RFS *)segs, n_seg, cache);
}

template <typename R>
void launch_apply_affine(mrsim_ctx *c, const PlainState &s, const R *cache, const void *adv) {
    using A = typename Seg<R>::Adv;
    KScope ks(c, "apply_affine");
    k_apply_affine<R><<<grid_stride_blocks(c, s.K), kThreads, 0, c->stream>>>(s, cache,
                                                                             *(const A *)adv);
}

void launch_gather_out(mrsim_ctx *c, int64_t K, const void *Mx, const void *My, const void *Mz,
                       bool fp64, const int32_t *perm, float *out) {
    KScope ks(c, "gather_out");
    if (fp64)
        k_gather_out<double><<<grid_stride_blocks(c, K), kThreads, 0, c->stream>>>(
            K, (const double *)Mx, (const double *)My, (const double *)Mz, perm, out);
    else
        k_gather_out<float><<<grid_stride_blocks(c, K), kThreads, 0, c->stream>>>(
            K, (const float *)Mx, (const float *)My, (const float *)Mz, perm, out);
}

namespace {

constexpr int kBoundBlocks = 256;

// per isochromat (|M0| + |M_init|) max(1, max_j |S_j|) in FP64; each thread
// takes a fixed set of isochromats and each block sums its threads in a
// fixed tree, so the partials do not depend on scheduling
__global__ void __launch_bounds__(kThreads) k_sum_bound(int64_t K, const float *M0,
                                                        const float *M_init, const float *coils,
                                                        int n_coils, double *part) {
    __shared__ double red[kThreads];
    double acc = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x) {
        double m = fabs((double)M0[k]);
        if (M_init) {
            const double a = M_init[k], b = M_init[K + k], c = M_init[2 * K + k];
            m += sqrt(a * a + b * b + c * c);
        }
        double s = 1.0;
        for (int j = 0; j < n_coils; ++j) {
            const double re = coils[2 * K * j + k], im = coils[2 * K * j + K + k];
            s = fmax(s, sqrt(re * re + im * im));
        }
        acc += m * s;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_fixed_to_double(double *buf, int64_t n, double inv) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const long long v = reinterpret_cast<const long long *>(buf)[i];
        buf[i] = (double)v * inv;
    }
}

}  // namespace

double sum_bound(mrsim_ctx *c, const mrsim_phantom_t *ph) {
    if (ph->sum_bound >= 0.0) return ph->sum_bound;
    double *part = (double *)scratch(c, 26, kBoundBlocks * sizeof(double));
    {
        KScope ks(c, "sum_bound");
        k_sum_bound<<<kBoundBlocks, kThreads, 0, c->stream>>>(
            ph->K, ph->M0.as<float>(), ph->has_M_init ? ph->M_init.as<float>() : nullptr,
            ph->n_coils > 0 ? ph->coils.as<float>() : nullptr, ph->n_coils, part);
    }
    double h[kBoundBlocks];
    MRSIM_CUDA(cudaMemcpyAsync(h, part, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    sync(c);
    double b = 0.0;
    for (int i = 0; i < kBoundBlocks; ++i) b += h[i];
    const_cast<mrsim_phantom_t *>(ph)->sum_bound = b;
    return b;
}

void launch_fixed_to_double(mrsim_ctx *c, double *buf, int64_t n, double fx) {
    if (n <= 0) return;
    KScope ks(c, "fixed_to_double");
    k_fixed_to_double<<<grid_stride_blocks(c, n), kThreads, 0, c->stream>>>(buf, n, 1.0 / fx);
}

#define INST(R)                                                                              \
    template void launch_init_state<R>(mrsim_ctx *, const PlainState &, const float *);      \
    template void launch_plain_rf<R>(mrsim_ctx *, const PlainState &, const void *, int,     \
                                     const void *, int);                                     \
    template void launch_plain_adc<R>(mrsim_ctx *, const PlainState &, const void *, int,    \
                                      int64_t, const void *, double *, int);                 \
    template void launch_advance<R>(mrsim_ctx *, const PlainState &, const void *);          \
    template void launch_plain_rf_affine<R>(mrsim_ctx *, const PlainState &, const void *,   \
                                            int, R *);                                       \
    template void launch_apply_affine<R>(mrsim_ctx *, const PlainState &, const R *,         \
                                         const void *);
INST(float)
INST(double)
#undef INST

}  // namespace mrsim
