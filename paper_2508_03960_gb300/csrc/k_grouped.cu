// Grouped-isochromat kernels of the update and with-ADC steps (Sec. 2.3).
//
//  k_fused        the update step of every with-RF subsequence and step 1 of
//                 every with-ADC subsequence (Eq. 9) of a span of the
//                 sequence, with each isochromat's M kept in registers from
//                 the first event to the last.  Between events M is advanced
//                 in closed form (Eqs. 4-5; relaxation subsequences and ADC
//                 windows cost nothing extra because those equations compose).
//                 Isochromats are laid out sorted by their with-ADC group, so
//                 Eq. 9 becomes a segmented warp reduction plus shared-memory
//                 accumulation and one FP64 add per (CTA, group, window).
//  k_event_table  per (event, primary group) advance factor E2 e^{-i phi}, E1.
//  k_group_signal step 2 of the with-ADC method (Eqs. 8, 10): every sample is
//                 the sum over groups of the block sum times the group's
//                 relaxation and phase since the window start.
// The preparation step (Eq. 7) is in k_precompute.cu.
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace mrsim {

namespace {

constexpr int kThreads = 256;

template <typename R>
struct Vec4;
template <>
struct Vec4<float> { using T = float4; };
template <>
struct Vec4<double> { using T = double2; };

template <typename R>
__device__ __forceinline__ void load_row(const R *p, R (&T)[12]) {
    if constexpr (sizeof(R) == 4) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
        float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
        T[0] = a.x; T[1] = a.y; T[2] = a.z; T[3] = a.w;
        T[4] = b.x; T[5] = b.y; T[6] = b.z; T[7] = b.w;
        T[8] = c.x; T[9] = c.y; T[10] = c.z; T[11] = c.w;
    } else {
        const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            double2 v = __ldg(q + i);
            T[2 * i] = v.x;
            T[2 * i + 1] = v.y;
        }
    }
}

// ---- per-(event, primary group) advance factors ----
template <typename R>
struct R4 { R x, y, z, w; };

// P(e, g) = E2 exp(-i 2 pi (pos_g kp_e + pos2_g kp2_e + dB0_g tau_e)),
// E1 = exp(-tau_e / T1_g); pos2 and kp2 belong to the second axis of a
// two-axis primary type (both 0 otherwise).
// The phase is reduced modulo one turn in FP64, the rest is evaluated in R.
template <typename R>
__global__ void k_event_table(const EvAdv *adv, int n_ev, int64_t G, const double *par,
                              R4<R> *out) {
    const int64_t n = (int64_t)n_ev * G;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / G, g = i - e * G;
        const EvAdv ea = adv[e];
        const double pos = par[g], T1 = par[G + g], T2 = par[2 * G + g], dB0 = par[3 * G + g];
        // pos2 (row 5): the second position of a two-axis primary type, else 0
        double ph = pos * ea.kp + par[5 * G + g] * ea.kp2 + dB0 * ea.tau;
        ph -= rint(ph);
        R c, s;
        phasor((R)ph, c, s);
        const R E2 = isinf(T2) ? (R)1 : (R)exp(-ea.tau / T2);
        const R E1 = isinf(T1) ? (R)1 : (R)exp(-ea.tau / T1);
        out[i] = R4<R>{E2 * c, -E2 * s, E1, (R)0};
    }
}

// group-factor tables of many jobs: items of job j are [off[j], off[j+1])
template <typename R>
__global__ void k_event_table_batch(const EvTabJob *jobs, const int64_t *off, int n_jobs,
                                    int64_t total) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_jobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= i) lo = mid; else hi = mid - 1;
        }
        const EvTabJob jb = jobs[lo];
        const int64_t r = i - off[lo];
        const int64_t e = r / jb.G, g = r - e * jb.G;
        const EvAdv ea = jb.adv[e];
        const double pos = jb.par[g], T1 = jb.par[jb.G + g], T2 = jb.par[2 * jb.G + g];
        const double dB0 = jb.par[3 * jb.G + g];
        double ph = pos * ea.kp + jb.par[5 * jb.G + g] * ea.kp2 + dB0 * ea.tau;
        ph -= rint(ph);
        R c, sn;
        phasor((R)ph, c, sn);
        const R E2 = isinf(T2) ? (R)1 : (R)exp(-ea.tau / T2);
        const R E1 = isinf(T1) ? (R)1 : (R)exp(-ea.tau / T1);
        ((R4<R> *)jb.out)[r] = R4<R>{E2 * c, -E2 * sn, E1, (R)0};
    }
}

template <typename R>
__device__ __forceinline__ R4<R> load4(const R4<R> *p) {
    if constexpr (sizeof(R) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        return R4<R>{v.x, v.y, v.z, v.w};
    } else {
        const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
        const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
        return R4<R>{a.x, a.y, b.x, b.y};
    }
}

constexpr int kBatch = 16;            // with-ADC windows per shared-memory flush
constexpr int kAccBytes = 16 * 1024;  // block-sum staging per CTA

// how the fused kernel advances an isochromat between events
enum FusedMode : int {
    FM_FACTOR = 0,  // group-factor table, per-isochromat phasor evaluated
    FM_AXIS = 1,    // group-factor table, per-isochromat phasor from axis tables
    FM_DIRECT = 2,  // every factor from the isochromat's own parameters
    FM_COIL = 4,    // flag: with-ADC terms weighted by a receive-coil sensitivity
};

template <int MASK>
__device__ __forceinline__ float iso_turns_m(const FEvent<float> &ev, float x, float y, float z) {
    float t = 0.0f;
    if constexpr ((MASK & 1) != 0) t += turns_prod(x, ev.k_hi[0], ev.k_lo[0]);
    if constexpr ((MASK & 2) != 0) t += turns_prod(y, ev.k_hi[1], ev.k_lo[1]);
    if constexpr ((MASK & 4) != 0) t += turns_prod(z, ev.k_hi[2], ev.k_lo[2]);
    return t;
}
template <int MASK>
__device__ __forceinline__ double iso_turns_m(const FEvent<double> &ev, double x, double y,
                                              double z) {
    double t = 0.0;
    if constexpr ((MASK & 1) != 0) t += x * ev.k[0];
    if constexpr ((MASK & 2) != 0) t += y * ev.k[1];
    if constexpr ((MASK & 4) != 0) t += z * ev.k[2];
    return t - rint(t);
}

// (cos, sin) of 2 pi sum_{a in MASK} r_a k_a from the event's axis tables:
// entry j of axis a's table holds the phasor of that axis' j-th distinct
// position; the factors of two axes multiply as unit complex numbers.
template <int MASK>
__device__ __forceinline__ void axis_phasor(const FEvent<float> &ev, const float2 *qtab,
                                            const int (&sh)[3], int aidx, float &c, float &s) {
    c = 1.0f;
    s = 0.0f;
    bool first = true;  // resolved at compile time after unrolling
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if ((MASK & (1 << a)) == 0) continue;
        const float2 q = __ldg(qtab + ev.q[a] + ((aidx >> sh[a]) & 0xffff));
        if (first) {
            c = q.x;
            s = q.y;
            first = false;
        } else {
            const float nc = c * q.x - s * q.y;
            s = s * q.x + c * q.y;
            c = nc;
        }
    }
}

// Per-isochromat registers of the fused kernel.  Padding isochromats (past
// K) carry zero magnetization and M0 and valid table rows, so every event
// leaves them at zero and the event loop needs no validity tests.
template <typename R, int NI>
struct Iso {
    R mx[NI], my[NI], mz[NI], M0[NI], x[NI], y[NI], z[NI];
    R dB0[NI], r1[NI], r2[NI];  // direct mode only: dB0, log2(e)/T1, log2(e)/T2
    int pofs[NI];  // primary group (row offset in a group-factor table)
    int tofs[NI];  // 12 * RF group (offset in a combined-transition table)
    int aidx[NI];  // axis mode only: packed axis indices
    R sr[NI], si[NI];  // coil mode only: receive sensitivity S(k, p)
};

// whole advance of one isochromat from the event record (direct mode):
// phase of all three axes and dB0 tau, E2 and E1 from its own T2, T1
__device__ __forceinline__ void direct_factor(const FEvent<float> &ev, float x, float y, float z,
                                              float dB0, float r1, float r2, float &fr, float &fi,
                                              float &E1) {
    const float t = turns_prod(x, ev.k_hi[0], ev.k_lo[0]) + turns_prod(y, ev.k_hi[1], ev.k_lo[1]) +
                    turns_prod(z, ev.k_hi[2], ev.k_lo[2]) + turns_prod(dB0, ev.k_hi[3], ev.k_lo[3]);
    float c, sn;
    phasor(t, c, sn);
    const float tau = ev.k_hi[3] + ev.k_lo[3];
    const float E2 = decay(tau, r2);
    E1 = decay(tau, r1);
    fr = E2 * c;
    fi = -E2 * sn;
}
__device__ __forceinline__ void direct_factor(const FEvent<double> &ev, double x, double y,
                                              double z, double dB0, double r1, double r2,
                                              double &fr, double &fi, double &E1) {
    double t = x * ev.k[0] + y * ev.k[1] + z * ev.k[2] + dB0 * ev.k[3];
    t -= rint(t);
    double c, sn;
    phasor(t, c, sn);
    const double E2 = decay(ev.k[3], r2);
    E1 = decay(ev.k[3], r1);
    fr = E2 * c;
    fi = -E2 * sn;
}

template <typename R, int NI>
__device__ __forceinline__ void ev_advance_direct(Iso<R, NI> &s, const FEvent<R> &ev) {
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        R fr, fi, E1;
        direct_factor(ev, s.x[i], s.y[i], s.z[i], s.dB0[i], s.r1[i], s.r2[i], fr, fi, E1);
        const R nx = fr * s.mx[i] - fi * s.my[i];
        s.my[i] = fr * s.my[i] + fi * s.mx[i];
        s.mx[i] = nx;
        s.mz[i] = s.M0[i] + (s.mz[i] - s.M0[i]) * E1;
    }
}

template <typename R, int NI>
__device__ __forceinline__ void ev_adc_direct(const Iso<R, NI> &s, const FEvent<R> &ev,
                                              R (&vr)[NI], R (&vi)[NI]) {
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        R fr, fi, E1;
        direct_factor(ev, s.x[i], s.y[i], s.z[i], s.dB0[i], s.r1[i], s.r2[i], fr, fi, E1);
        vr[i] = fr * s.mx[i] - fi * s.my[i];
        vi[i] = fr * s.my[i] + fi * s.mx[i];
    }
}

// per-isochromat phasor Q of the axes in MASK (factor-table modes)
template <typename R, int NI, int MASK, int MODE>
__device__ __forceinline__ void iso_q(const Iso<R, NI> &s, int i, const FEvent<R> &ev,
                                      const float2 *qtab, const int (&sh)[3], R &c, R &sn) {
    if constexpr (MODE == FM_AXIS) {
        axis_phasor<MASK>(ev, qtab, sh, s.aidx[i], c, sn);
    } else {
        phasor(iso_turns_m<MASK>(ev, s.x[i], s.y[i], s.z[i]), c, sn);
    }
}

// advance of every isochromat (Eqs. 4-5): M_xy <- P Q M_xy, Mz relaxes with E1.
// A thread's isochromats are consecutive in the layout and mostly share their
// primary group, so the factor row is re-read only where the group changes.
template <typename R, int NI, int MASK, int MODE>
__device__ __forceinline__ void ev_advance(Iso<R, NI> &s, const FEvent<R> &ev, const R4<R> *Pt,
                                           const float2 *qtab, const int (&sh)[3]) {
    const R4<R> *Pe = Pt + ev.prow;
    R4<R> P = load4(Pe + s.pofs[0]);
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        if (i > 0 && s.pofs[i] != s.pofs[i - 1]) P = load4(Pe + s.pofs[i]);
        R fr = P.x, fi = P.y;
        if constexpr (MASK != 0) {
            R c, sn;
            iso_q<R, NI, MASK, MODE>(s, i, ev, qtab, sh, c, sn);
            const R tr = fr * c + fi * sn;  // P * exp(-i psi)
            fi = fi * c - fr * sn;
            fr = tr;
        }
        const R nx = fr * s.mx[i] - fi * s.my[i];
        s.my[i] = fr * s.my[i] + fi * s.mx[i];
        s.mx[i] = nx;
        s.mz[i] = s.M0[i] + (s.mz[i] - s.M0[i]) * P.z;
    }
}

// transverse magnetization of every isochromat times Q (ADC block-sum terms)
template <typename R, int NI, int MASK, int MODE>
__device__ __forceinline__ void ev_adc_terms(const Iso<R, NI> &s, const FEvent<R> &ev,
                                             const float2 *qtab, const int (&sh)[3], R (&vr)[NI],
                                             R (&vi)[NI]) {
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        vr[i] = s.mx[i];
        vi[i] = s.my[i];
        if constexpr (MASK != 0) {
            R c, sn;
            iso_q<R, NI, MASK, MODE>(s, i, ev, qtab, sh, c, sn);
            const R tr = vr[i] * c + vi[i] * sn;
            vi[i] = vi[i] * c - vr[i] * sn;
            vr[i] = tr;
        }
    }
}

constexpr int kEvChunk = 64;  // events staged in shared memory at a time

// Shared memory of one fused CTA (dynamic: larger than the static limit).
template <typename R>
struct FusedSmem {
    __align__(16) unsigned char acc_raw[kAccBytes];  // staged block sums [batch][slot][re, im]
    __align__(16) FEvent<R> sev[kEvChunk];           // staged events
    // per-thread partial sums of warps whose isochromats share one group,
    // [window][thread] (row padded by one entry: conflict-free column reads)
    __align__(16) R tpart[kBatch][kThreads + 1][2];
    R wpart[kBatch][kThreads / 32][2];  // their per-warp sums
    int batch_prow[kBatch], batch_win[kBatch];
    int wslot[kThreads / 32];  // that group's slot, or -1
};

// One chunk of kThreads * NI isochromats (chunk index blk) through all events
// of a span.  All threads of the CTA take part (shared memory, barriers).
template <typename R, int NI, int MODE_FLAGS>
__device__ __forceinline__ void fused_chunk(const FusedArgs<R> &a, int64_t blk,
                                            FusedSmem<R> &sm) {
    constexpr int MODE = MODE_FLAGS & 3;
    constexpr bool COIL = (MODE_FLAGS & FM_COIL) != 0;
    constexpr bool DIRECT = MODE == FM_DIRECT;
    FEvent<R> *sev = sm.sev;
    int *batch_prow = sm.batch_prow, *batch_win = sm.batch_win;
    R *acc = reinterpret_cast<R *>(sm.acc_raw);  // [batch][slot][re, im]
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t chunk = (int64_t)kThreads * NI;
    const int64_t base = blk * chunk;
    const int64_t last = min(base + chunk, a.K) - 1;
    const int32_t *gp = a.gid[a.gtype_p];
    const int32_t *gr = a.gid[a.gtype_r];
    const R4<R> *Pt = reinterpret_cast<const R4<R> *>(a.P_raw);
    const R *Tt = a.T_tab;
    const float2 *qtab = a.qtab;
    const int sh[3] = {a.ax_sh[0], a.ax_sh[1], a.ax_sh[2]};
    double *Ablk = a.Ablk;
    const int32_t g_first = gp[base];
    const int32_t g_last = gp[last];
    const int S = (int)(g_last - g_first + 1);  // primary groups in this chunk
    // windows staged per flush: as many as fit, at most kBatch
    const int B = max(1, min(kBatch, (int)(kAccBytes / (S * 2 * (int)sizeof(R)))));
    const bool stage = S * 2 * (int)sizeof(R) <= kAccBytes;

    // isochromat i of this thread.  With group tables (groups of several
    // isochromats) a thread holds NI consecutive isochromats of the sorted
    // layout (measured faster: the table rows a warp reads are fewer and the
    // warp-level reductions see longer runs).  In direct mode (about one group
    // per isochromat) every isochromat reads its own transition row, and the
    // mapping base + i * kThreads + tid keeps those reads coalesced.
    auto iso_k = [&](int i) -> int64_t {
        return DIRECT ? base + (int64_t)i * kThreads + tid : base + (int64_t)tid * NI + i;
    };
    Iso<R, NI> s;
    int32_t key[NI];  // primary group, or a value sorting last for padding
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        const int64_t k = iso_k(i);
        if (k < a.K) {
            if constexpr (MODE == FM_AXIS) {
                s.aidx[i] = a.aidx[k];
            } else {
                s.x[i] = a.x[k]; s.y[i] = a.y[k]; s.z[i] = a.z[k];
            }
            s.M0[i] = a.M0[k];
            if (a.init_eq) {
                s.mx[i] = 0; s.my[i] = 0; s.mz[i] = s.M0[i];
            } else {
                s.mx[i] = a.Mx[k]; s.my[i] = a.My[k]; s.mz[i] = a.Mz[k];
            }
            key[i] = gp[k];
            s.tofs[i] = 12 * gr[k];
            if constexpr (COIL) {
                s.sr[i] = (R)a.coil_re[k];
                s.si[i] = (R)a.coil_im[k];
            }
            if constexpr (DIRECT) {
                s.dB0[i] = a.dB0[k];
                const float T1 = a.T1[k], T2 = a.T2[k];
                s.r1[i] = isinf(T1) ? (R)0 : (R)kLog2e / (R)T1;
                s.r2[i] = isinf(T2) ? (R)0 : (R)kLog2e / (R)T2;
            }
        } else {
            s.x[i] = s.y[i] = s.z[i] = s.M0[i] = 0;
            s.aidx[i] = 0;
            s.sr[i] = s.si[i] = 0;
            s.mx[i] = s.my[i] = s.mz[i] = 0;
            key[i] = 0x7fffffff;
            s.tofs[i] = 0;
            if constexpr (DIRECT) s.dB0[i] = s.r1[i] = s.r2[i] = 0;
        }
        s.pofs[i] = min(key[i], g_last);
    }
    if (stage)
        for (int t = tid; t < B * S * 2; t += kThreads) acc[t] = 0;
    // a warp whose isochromats all share one primary group stages per-thread
    // partial sums and reduces them at the flush
    const int32_t w0 = __shfl_sync(0xffffffffu, key[0], 0);
    bool uni = true;
#pragma unroll
    for (int i = 0; i < NI; ++i) uni &= (key[i] == w0 || key[i] == 0x7fffffff);
    const bool warp_uni = __all_sync(0xffffffffu, uni) && w0 != 0x7fffffff;
    const int warp = tid >> 5;
    if (lane == 0) sm.wslot[warp] = (warp_uni && stage) ? w0 - g_first : -1;
    // (the flush visits the per-warp partials only if some warp stores them)
    const bool any_uni = __syncthreads_or(warp_uni && stage) != 0;

    int nb = 0;  // windows staged (uniform)
    auto flush = [&]() {
        if (warp_uni && stage) {
            // column sums of this warp's staged partials: lane (h, b) adds
            // the 16 threads of half h for window b, then the halves combine
            __syncwarp();
            const int b = lane & (kBatch - 1), h = lane >> 4;
            R sr = 0, si = 0;
            if (b < nb) {
                const R(*col)[2] = &sm.tpart[b][warp * 32 + h * 16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    sr += col[j][0];
                    si += col[j][1];
                }
            }
            sr += __shfl_xor_sync(0xffffffffu, sr, 16);
            si += __shfl_xor_sync(0xffffffffu, si, 16);
            if (h == 0 && b < nb) {
                sm.wpart[b][warp][0] = sr;
                sm.wpart[b][warp][1] = si;
            }
        }
        __syncthreads();
        for (int t = tid; t < nb * S; t += kThreads) {
            const int b = t / S, slot = t - b * S;
            R sr = acc[2 * t], si = acc[2 * t + 1];
            if (any_uni) {
#pragma unroll
                for (int w = 0; w < kThreads / 32; ++w) {
                    if (sm.wslot[w] == slot) {
                        sr += sm.wpart[b][w][0];
                        si += sm.wpart[b][w][1];
                    }
                }
            }
            if (sr != (R)0 || si != (R)0) {
                R4<R> P{(R)1, (R)0, (R)1, (R)0};
                if constexpr (!DIRECT) P = load4(Pt + batch_prow[b] + g_first + slot);
                const int64_t o = 2 * ((int64_t)batch_win[b] + g_first + slot);
                const double vr = (double)(P.x * sr - P.y * si), vi = (double)(P.x * si + P.y * sr);
                if (slot != 0 && slot != S - 1 && a.fx == 0.0) {
                    // a group strictly inside the chunk has no other contributor
                    *reinterpret_cast<double2 *>(&Ablk[o]) = make_double2(vr, vi);
                } else {
                    // (reproducible sums: the non-uniform warps add theirs
                    // directly, so every slot is added)
                    sum_add(&Ablk[o], vr, a.fx);
                    sum_add(&Ablk[o + 1], vi, a.fx);
                }
            }
            // cleared even when the slot's total is zero: the staged partial
            // of the non-uniform warps can cancel the per-warp sums exactly,
            // and a value left here would be added into a later window
            acc[2 * t] = 0;
            acc[2 * t + 1] = 0;
        }
        __syncthreads();
        nb = 0;
    };

    auto rf_apply = [&](const FEvent<R> &ev, int gtype) {
        const int32_t *g = gtype == a.gtype_r ? nullptr : a.gid[gtype];
        const R *Te = Tt + (int64_t)ev.row * 12;
        R T[12];
        int prev = -1;
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            int off = s.tofs[i];
            if (g) {
                const int64_t k = iso_k(i);
                off = k < a.K ? 12 * g[k] : 0;
            }
            // consecutive isochromats of a thread mostly share their RF group
            if (DIRECT || i == 0 || off != prev) load_row(Te + off, T);
            prev = off;
            const R nx = T[0] * s.mx[i] + T[1] * s.my[i] + T[2] * s.mz[i] + T[3] * s.M0[i];
            const R ny = T[4] * s.mx[i] + T[5] * s.my[i] + T[6] * s.mz[i] + T[7] * s.M0[i];
            const R nz = T[8] * s.mx[i] + T[9] * s.my[i] + T[10] * s.mz[i] + T[11] * s.M0[i];
            s.mx[i] = nx;
            s.my[i] = ny;
            s.mz[i] = nz;
        }
    };

    auto adc_reduce = [&](const FEvent<R> &ev, int gtype, R (&vr)[NI], R (&vi)[NI]) {
        if (gtype == a.gtype_p && stage) {
            R *accb = acc + 2 * nb * S;
            if (warp_uni) {
                R sr = 0, si = 0;
#pragma unroll
                for (int i = 0; i < NI; ++i) { sr += vr[i]; si += vi[i]; }
                sm.tpart[nb][tid][0] = sr;
                sm.tpart[nb][tid][1] = si;
            } else {
                // keys are sorted along the lanes for each i: a segmented
                // inclusive scan leaves each run's sum in the run's last lane
#pragma unroll
                for (int i = 0; i < NI; ++i) {
                    R sr = vr[i], si = vi[i];
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const R orr = __shfl_up_sync(0xffffffffu, sr, d);
                        const R oii = __shfl_up_sync(0xffffffffu, si, d);
                        const int32_t ok2 = __shfl_up_sync(0xffffffffu, key[i], d);
                        if (lane >= d && ok2 == key[i]) { sr += orr; si += oii; }
                    }
                    const int32_t nk = __shfl_down_sync(0xffffffffu, key[i], 1);
                    if ((lane == 31 || nk != key[i]) && key[i] != 0x7fffffff) {
                        if (a.fx > 0.0) {
                            // reproducible sums: the run's term goes to the
                            // block sum as an integer (the shared accumulator's
                            // atomics would depend on the order of the warps)
                            R4<R> P{(R)1, (R)0, (R)1, (R)0};
                            if constexpr (!DIRECT) P = load4(Pt + ev.prow + key[i]);
                            const int64_t o = 2 * ((int64_t)ev.win + key[i]);
                            sum_add(&Ablk[o], (double)(P.x * sr - P.y * si), a.fx);
                            sum_add(&Ablk[o + 1], (double)(P.x * si + P.y * sr), a.fx);
                        } else {
                            atomicAdd(&accb[2 * (key[i] - g_first)], sr);
                            atomicAdd(&accb[2 * (key[i] - g_first) + 1], si);
                        }
                    }
                }
            }
            if (tid == 0) {
                batch_prow[nb] = ev.prow;
                batch_win[nb] = ev.win;
            }
            ++nb;
            if (nb == B) flush();
        } else {
            // a window whose groups are not the layout's: P per isochromat, FP64 atomics
            const int32_t *g = a.gid[gtype];
#pragma unroll
            for (int i = 0; i < NI; ++i) {
                const int64_t k = iso_k(i);
                if (k < a.K) {
                    R4<R> P{(R)1, (R)0, (R)1, (R)0};
                    if constexpr (!DIRECT) P = load4(Pt + ev.prow + s.pofs[i]);
                    const int64_t o = 2 * ((int64_t)ev.win + g[k]);
                    sum_add(&Ablk[o], (double)(P.x * vr[i] - P.y * vi[i]), a.fx);
                    sum_add(&Ablk[o + 1], (double)(P.x * vi[i] + P.y * vr[i]), a.fx);
                }
            }
        }
    };

#define MRSIM_ADV_CASE(M)                                   \
    case M:                                                 \
        ev_advance<R, NI, M, MODE>(s, ev, Pt, qtab, sh);    \
        break;
#define MRSIM_ADC_CASE(M)                                      \
    case M:                                                    \
        ev_adc_terms<R, NI, M, MODE>(s, ev, qtab, sh, vr, vi); \
        break;

    for (int e0 = 0; e0 < a.n_ev; e0 += kEvChunk) {
        const int ne = min(kEvChunk, a.n_ev - e0);
        __syncthreads();
        {
            const int4 *src = reinterpret_cast<const int4 *>(a.ev + e0);
            int4 *dst = reinterpret_cast<int4 *>(sev);
            const int nw = ne * (int)(sizeof(FEvent<R>) / sizeof(int4));
            for (int t = tid; t < nw; t += kThreads) dst[t] = src[t];
        }
        __syncthreads();
        for (int e = 0; e < ne; ++e) {
            const FEvent<R> &ev = sev[e];
            const int op = ev.op;
            const int kind = ev_kind(op), mask = ev_mask(op), gtype = ev_gtype(op);
            if (kind != EV_ADC) {
                if constexpr (DIRECT) {
                    ev_advance_direct<R, NI>(s, ev);
                } else {
                    switch (mask) {
                        MRSIM_ADV_CASE(0) MRSIM_ADV_CASE(1) MRSIM_ADV_CASE(2) MRSIM_ADV_CASE(3)
                        MRSIM_ADV_CASE(4) MRSIM_ADV_CASE(5) MRSIM_ADV_CASE(6) MRSIM_ADV_CASE(7)
                    }
                }
                if (kind == EV_RF) {
                    rf_apply(ev, gtype);
                } else if (a.Mx) {  // EV_END: store the state
#pragma unroll
                    for (int i = 0; i < NI; ++i) {
                        const int64_t k = iso_k(i);
                        if (k < a.K) {
                            a.Mx[k] = s.mx[i];
                            a.My[k] = s.my[i];
                            a.Mz[k] = s.mz[i];
                        }
                    }
                }
            } else {
                R vr[NI], vi[NI];
                if constexpr (DIRECT) {
                    ev_adc_direct<R, NI>(s, ev, vr, vi);
                } else {
                    switch (mask) {
                        MRSIM_ADC_CASE(0) MRSIM_ADC_CASE(1) MRSIM_ADC_CASE(2) MRSIM_ADC_CASE(3)
                        MRSIM_ADC_CASE(4) MRSIM_ADC_CASE(5) MRSIM_ADC_CASE(6) MRSIM_ADC_CASE(7)
                    }
                }
                if constexpr (COIL) {  // Eq. 6 with a receive coil: S(k, p) M_xy
#pragma unroll
                    for (int i = 0; i < NI; ++i) {
                        const R tr = s.sr[i] * vr[i] - s.si[i] * vi[i];
                        vi[i] = s.sr[i] * vi[i] + s.si[i] * vr[i];
                        vr[i] = tr;
                    }
                }
                adc_reduce(ev, gtype, vr, vi);
            }
        }
    }
#undef MRSIM_ADV_CASE
#undef MRSIM_ADC_CASE
    if (nb > 0) flush();
    __syncthreads();
}

// CTAs per SM each instantiation is compiled for: the most that keep it free
// of register spills (the kernel is latency bound, so occupancy pays; the
// shared memory of an FP32 CTA, about 54 KB, lets four share an SM)
template <typename R, int NI, int MODE>
constexpr int fused_min_blocks() {
    constexpr int base = MODE & 3;
    constexpr int b = sizeof(R) == 8 ? 1
                    : base == FM_AXIS ? 4
                    : base == FM_FACTOR ? (NI == 4 ? 3 : 4)
                                        : (NI == 4 ? 2 : NI == 2 ? 3 : 4);
    // the coil's two registers per isochromat do not fit 64 per thread
    return (MODE & FM_COIL) != 0 && b > 3 ? 3 : b;
}

template <typename R, int NI, int MODE>
__global__ void __launch_bounds__(kThreads, (fused_min_blocks<R, NI, MODE>()))
    k_fused(FusedArgs<R> a) {
    extern __shared__ __align__(16) unsigned char fused_smem[];
    fused_chunk<R, NI, MODE>(a, blockIdx.x, *reinterpret_cast<FusedSmem<R> *>(fused_smem));
}

// Persistent form for a batch of jobs: every CTA takes the next (job, chunk)
// work item from a device counter until all chunks of all jobs are done, so
// jobs of very different sizes share the GPU without a tail of idle SMs.
// MODE: the form shared by the launch's jobs (factor tables or direct
// advances, with or without a receive coil).
template <typename R, int NI, int MODE>
__global__ void __launch_bounds__(kThreads, (fused_min_blocks<R, NI, MODE>()))
    k_fused_batch(const FusedArgs<R> *jobs, const int64_t *blk_off, int n_jobs,
                  unsigned long long *counter) {
    extern __shared__ __align__(16) unsigned char fused_smem[];
    FusedSmem<R> &sm = *reinterpret_cast<FusedSmem<R> *>(fused_smem);
    __shared__ FusedArgs<R> ja;
    __shared__ long long item, jblk;
    const int64_t total = blk_off[n_jobs];
    for (;;) {
        if (threadIdx.x == 0) {
            item = (long long)atomicAdd(counter, 1ull);
            if (item < total) {
                int lo = 0, hi = n_jobs - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (blk_off[mid] <= item) lo = mid; else hi = mid - 1;
                }
                ja = jobs[lo];
                jblk = item - blk_off[lo];
            }
        }
        __syncthreads();
        if (item >= total) break;
        fused_chunk<R, NI, MODE>(ja, jblk, sm);
    }
}

template <typename R>
struct GS;
template <>
struct GS<float> { using S = GSampleF; };
template <>
struct GS<double> { using S = GSampleD; };

// phase (turns) of a group at a sample: its positions times the moments on
// its type's axes (pos2: second axis of a two-axis type, else 0) plus dB0 tau
__device__ __forceinline__ float gs_turns(const GSampleF &s, float pos, float pos2, float dB0) {
    return turns_prod(pos, s.k_hi, s.k_lo) + turns_prod(pos2, s.k2_hi, s.k2_lo) +
           turns_prod(dB0, s.tau_hi, s.tau_lo);
}
__device__ __forceinline__ double gs_turns(const GSampleD &s, double pos, double pos2,
                                           double dB0) {
    double v = pos * s.k + pos2 * s.k2 + dB0 * s.tau;
    return v - rint(v);
}
__device__ __forceinline__ float gs_tau(const GSampleF &s) { return s.tau_hi + s.tau_lo; }
__device__ __forceinline__ double gs_tau(const GSampleD &s) { return s.tau; }

constexpr int kGTile = 256;
constexpr int kRun = 8;  // samples per thread on uniform windows

// Uniform window (one ADC segment): a group's term at sample s + j is its term
// at s times z^j, z = E2(dt) exp(-i 2 pi (pos dk + dB0 dt)) (Eqs. 8, 10 with a
// constant gradient).  Thread (run ri, lane gl) takes kRun consecutive samples
// of the block and every LPR-th group of each tile: two phasors and exps per
// (group, run) instead of one per (group, sample).  Partial sums per sample are
// combined over the lanes in FP64 shared memory.
__device__ __forceinline__ void group_signal_runs(const GWin &w, const int4 b, int nsb,
                                                  const GSampleF *smp,
                                                  const GSigTables<float> &tab,
                                                  const double *Ablk, double *signal,
                                                  double fx) {
    __shared__ float s_pos[kGTile], s_dB0[kGTile], s_rT2[kGTile], s_ar[kGTile], s_ai[kGTile];
    __shared__ float s_pos2[kGTile];
    __shared__ double s_red[2][kThreads * kRun];
    const int NR = (nsb + kRun - 1) / kRun;
    int NRp = 1;
    while (NRp < NR) NRp <<= 1;
    const int LPR = kThreads / NRp;
    const int ri = threadIdx.x % NRp, gl = threadIdx.x / NRp;
    const int64_t s0 = (int64_t)b.y + (int64_t)ri * kRun;
    const int len = ri < NR ? min(kRun, (int)((int64_t)b.y + nsb - s0)) : 0;
    GSampleF sm{};
    if (len > 0) sm = smp[s0];
    const float tau0 = sm.tau_hi + sm.tau_lo;
    const float dt = w.dt_hi + w.dt_lo;
    const float *pos = tab.pos[w.gtype], *dB0 = tab.dB0[w.gtype], *rT2 = tab.rT2[w.gtype];
    const float *pos2 = tab.pos2[w.gtype];
    // FP32 partial sums, folded into FP64 every LPR tiles: each partial then
    // covers 256 groups whatever the mapping (an FP64 fold per tile would make
    // the FP64 pipe, a small fraction of the FP32 rate here, the bottleneck)
    double ar_d[kRun], ai_d[kRun];
    float pr[kRun], pi[kRun];
#pragma unroll
    for (int j = 0; j < kRun; ++j) {
        ar_d[j] = ai_d[j] = 0.0;
        pr[j] = pi[j] = 0.0f;
    }
    int tiles = 0;
    for (int g0 = b.z; g0 < b.w; g0 += kGTile) {
        const int n = min(kGTile, b.w - g0);
        __syncthreads();
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            s_pos[t] = pos[g0 + t];
            s_pos2[t] = pos2[g0 + t];
            s_dB0[t] = dB0[g0 + t];
            s_rT2[t] = rT2[g0 + t];
            s_ar[t] = (float)sum_get(&Ablk[2 * (w.ablk + g0 + t)], fx);
            s_ai[t] = (float)sum_get(&Ablk[2 * (w.ablk + g0 + t) + 1], fx);
        }
        __syncthreads();
        if (len > 0) {
            for (int t = gl; t < n; t += LPR) {
                float c, sn, cz, sz;
                phasor(gs_turns(sm, s_pos[t], s_pos2[t], s_dB0[t]), c, sn);
                phasor(turns_prod(s_pos[t], w.dk_hi, w.dk_lo) +
                           turns_prod(s_pos2[t], w.dk2_hi, w.dk2_lo) +
                           turns_prod(s_dB0[t], w.dt_hi, w.dt_lo),
                       cz, sz);
                const float e = decay(tau0, s_rT2[t]), ez = decay(dt, s_rT2[t]);
                // term = E2 exp(-i phi) A with exp(-i phi) = c - i sn
                const float ar = s_ar[t], ai = s_ai[t];
                float ur = e * (c * ar + sn * ai), ui = e * (c * ai - sn * ar);
                const float zr = ez * cz, zi = -ez * sz;
#pragma unroll
                for (int j = 0; j < kRun; ++j) {
                    pr[j] += ur;
                    pi[j] += ui;
                    const float nr = ur * zr - ui * zi;
                    ui = ur * zi + ui * zr;
                    ur = nr;
                }
            }
            if (++tiles == LPR) {
#pragma unroll
                for (int j = 0; j < kRun; ++j) {
                    ar_d[j] += (double)pr[j];
                    ai_d[j] += (double)pi[j];
                    pr[j] = pi[j] = 0.0f;
                }
                tiles = 0;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kRun; ++j) {
        ar_d[j] += (double)pr[j];
        ai_d[j] += (double)pi[j];
    }
    // samples of run ri at [ri * kRun, ...): lane gl's partials
#pragma unroll
    for (int j = 0; j < kRun; ++j) {
        s_red[0][gl * (NRp * kRun) + ri * kRun + j] = ar_d[j];
        s_red[1][gl * (NRp * kRun) + ri * kRun + j] = ai_d[j];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nsb; q += blockDim.x) {
        double sr = 0.0, si = 0.0;
        for (int l = 0; l < LPR; ++l) {
            sr += s_red[0][l * (NRp * kRun) + q];
            si += s_red[1][l * (NRp * kRun) + q];
        }
        sum_add(&signal[2 * ((int64_t)b.y + q)], sr, fx);
        sum_add(&signal[2 * ((int64_t)b.y + q) + 1], si, fx);
    }
    __syncthreads();
}

// block b covers samples [blk.y, blk.y + blockDim) of window blk.x and the
// groups [blk.z, blk.w); partial sums go to the signal with FP64 atomics
template <typename R>
__device__ __forceinline__ void group_signal_block(const GWin *wins, const int4 b,
                                                   const typename GS<R>::S *smp,
                                                   const GSigTables<R> &tab, const double *Ablk,
                                                   double *signal, double fx) {
    __shared__ R s_pos[kGTile], s_dB0[kGTile], s_rT2[kGTile], s_ar[kGTile], s_ai[kGTile];
    __shared__ R s_pos2[kGTile];
    __shared__ double s_red[2][kThreads];
    const GWin w = wins[b.x];
    // samples of this block: [b.y, b.y + nsb).  A window shorter than the
    // block gets several group lanes per sample (lane sl takes groups sl,
    // sl + LPS, ...), combined in shared memory before the FP64 atomics.
    const int nsb = (int)min((long long)kThreads, w.sample0 + w.n_samples - (long long)b.y);
    if constexpr (sizeof(R) == 4) {
        if (w.uniform) {
            group_signal_runs(w, b, nsb, smp, tab, Ablk, signal, fx);
            return;
        }
    }
    int SPB = 32;
    while (SPB < nsb) SPB <<= 1;
    const int LPS = kThreads / SPB;
    const int si = threadIdx.x & (SPB - 1), sl = threadIdx.x / SPB;
    const int64_t s_idx = (int64_t)b.y + si;
    const bool act = si < nsb;
    typename GS<R>::S sm{};
    if (act) sm = smp[s_idx];
    const R tau = act ? (R)gs_tau(sm) : (R)0;
    const R *pos = tab.pos[w.gtype], *dB0 = tab.dB0[w.gtype], *rT2 = tab.rT2[w.gtype];
    const R *pos2 = tab.pos2[w.gtype];
    double accr = 0, acci = 0;
    for (int g0 = b.z; g0 < b.w; g0 += kGTile) {
        const int n = min(kGTile, b.w - g0);
        __syncthreads();
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            s_pos[t] = pos[g0 + t];
            s_pos2[t] = pos2[g0 + t];
            s_dB0[t] = dB0[g0 + t];
            s_rT2[t] = rT2[g0 + t];
            s_ar[t] = (R)sum_get(&Ablk[2 * (w.ablk + g0 + t)], fx);
            s_ai[t] = (R)sum_get(&Ablk[2 * (w.ablk + g0 + t) + 1], fx);
        }
        __syncthreads();
        R pr = 0, pi = 0;
        if (act) {
            for (int t = sl; t < n; t += LPS) {
                R c, s;
                phasor(gs_turns(sm, s_pos[t], s_pos2[t], s_dB0[t]), c, s);
                const R e = decay(tau, s_rT2[t]);
                const R ar = s_ar[t], ai = s_ai[t];
                pr += e * (c * ar + s * ai);
                pi += e * (c * ai - s * ar);
            }
        }
        accr += (double)pr;
        acci += (double)pi;
    }
    if (LPS > 1) {
        s_red[0][threadIdx.x] = accr;
        s_red[1][threadIdx.x] = acci;
        __syncthreads();
        if (sl == 0) {
            for (int l = 1; l < LPS; ++l) {
                accr += s_red[0][l * SPB + si];
                acci += s_red[1][l * SPB + si];
            }
        }
    }
    if (act && sl == 0) {
        sum_add(&signal[2 * s_idx], accr, fx);
        sum_add(&signal[2 * s_idx + 1], acci, fx);
    }
    __syncthreads();
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_group_signal(const GWin *wins, const int4 *blk,
                                                           const typename GS<R>::S *smp,
                                                           GSigTables<R> tab,
                                                           const double *Ablk, double *signal,
                                                           double fx) {
    group_signal_block<R>(wins, blk[blockIdx.x], smp, tab, Ablk, signal, fx);
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_group_signal_batch(const GSigJob<R> *jobs,
                                                                 const int4 *blk,
                                                                 const int *blk_job) {
    const GSigJob<R> &j = jobs[blk_job[blockIdx.x]];
    group_signal_block<R>(j.wins, blk[blockIdx.x], (const typename GS<R>::S *)j.samples, j.tab,
                          j.Ablk, j.signal, j.fx);
}

}  // namespace

template <typename R>
void launch_event_table_batch(mrsim_ctx *c, const EvTabJob *d_jobs, const int64_t *d_off,
                              int n_jobs, int64_t total) {
    if (total <= 0) return;
    KScope ks(c, "event_table_batch");
    const unsigned grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((total + 255) / 256, (int64_t)c->sm_count * 16));
    k_event_table_batch<R><<<grid, 256, 0, c->stream>>>(d_jobs, d_off, n_jobs, total);
}

// The fused kernels take more shared memory than the static limit: every
// instantiation gets the attribute on the context's device (prepare_fused).
template <typename K>
void fused_smem_attr(K kern, size_t bytes) {
    MRSIM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)bytes));
}

template <typename R, int NI, int MODE>
void launch_fused_batch_ni(mrsim_ctx *c, const FusedArgs<R> *d_jobs, const int64_t *d_blk_off,
                           int n_jobs, unsigned long long *d_counter) {
    const size_t smem = sizeof(FusedSmem<R>);
    int per_sm = 1;
    MRSIM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_batch<R, NI, MODE>,
                                                             kThreads, smem));
    k_fused_batch<R, NI, MODE><<<std::max(1, per_sm) * c->sm_count, kThreads, smem, c->stream>>>(
        d_jobs, d_blk_off, n_jobs, d_counter);
}

template <typename R, int MODE>
void launch_fused_batch_m(mrsim_ctx *c, const FusedArgs<R> *d_jobs, const int64_t *d_blk_off,
                          int n_jobs, unsigned long long *d_counter, int ni) {
    if (ni >= 4) launch_fused_batch_ni<R, 4, MODE>(c, d_jobs, d_blk_off, n_jobs, d_counter);
    else if (ni == 2) launch_fused_batch_ni<R, 2, MODE>(c, d_jobs, d_blk_off, n_jobs, d_counter);
    else launch_fused_batch_ni<R, 1, MODE>(c, d_jobs, d_blk_off, n_jobs, d_counter);
}

template <typename R>
void launch_fused_batch(mrsim_ctx *c, const FusedArgs<R> *d_jobs, const int64_t *d_blk_off,
                        int n_jobs, unsigned long long *d_counter, int ni, bool direct,
                        bool coil) {
    KScope ks(c, "fused_batch");
    if (direct && coil)
        launch_fused_batch_m<R, FM_DIRECT | FM_COIL>(c, d_jobs, d_blk_off, n_jobs, d_counter, ni);
    else if (direct)
        launch_fused_batch_m<R, FM_DIRECT>(c, d_jobs, d_blk_off, n_jobs, d_counter, ni);
    else if (coil)
        launch_fused_batch_m<R, FM_FACTOR | FM_COIL>(c, d_jobs, d_blk_off, n_jobs, d_counter, ni);
    else
        launch_fused_batch_m<R, FM_FACTOR>(c, d_jobs, d_blk_off, n_jobs, d_counter, ni);
}

template <typename R>
void launch_group_signal_batch(mrsim_ctx *c, const GSigJob<R> *d_jobs, const int4 *d_blk,
                               const int *d_blk_job, int n_blk) {
    if (n_blk <= 0) return;
    KScope ks(c, "group_signal_batch");
    k_group_signal_batch<R><<<n_blk, kThreads, 0, c->stream>>>(d_jobs, d_blk, d_blk_job);
}

template <typename R, int NI, int MODE>
void launch_fused_ni(mrsim_ctx *c, const FusedArgs<R> &a) {
    const size_t smem = sizeof(FusedSmem<R>);
    const unsigned nb = (unsigned)((a.K + kThreads * NI - 1) / (kThreads * NI));
    k_fused<R, NI, MODE><<<nb, kThreads, smem, c->stream>>>(a);
}

template <typename R, int MODE>
void launch_fused_v(mrsim_ctx *c, const FusedArgs<R> &a, int ni) {
    if (ni >= 4) launch_fused_ni<R, 4, MODE>(c, a);
    else if (ni == 2) launch_fused_ni<R, 2, MODE>(c, a);
    else launch_fused_ni<R, 1, MODE>(c, a);
}

template <typename R, int COIL>
void launch_fused_c(mrsim_ctx *c, const FusedArgs<R> &a, int ni) {
    if (a.direct) {
        launch_fused_v<R, FM_DIRECT | COIL>(c, a, ni);
    } else if constexpr (sizeof(R) == 4) {
        if (a.ax) launch_fused_v<R, FM_AXIS | COIL>(c, a, ni);
        else launch_fused_v<R, FM_FACTOR | COIL>(c, a, ni);
    } else {
        launch_fused_v<R, FM_FACTOR | COIL>(c, a, ni);
    }
}

template <typename R>
void launch_fused(mrsim_ctx *c, const FusedArgs<R> &a, int ni) {
    KScope ks(c, sizeof(R) == 4 ? "fused_grouped_f32" : "fused_grouped_f64");
    if (a.coil_re) launch_fused_c<R, FM_COIL>(c, a, ni);
    else launch_fused_c<R, 0>(c, a, ni);
}

// one thread per (item, entry): exp(-i 2 pi val[j] k) with the phase reduced
// modulo one turn in FP64 and the phasor evaluated in FP64, stored as float
__global__ void k_axis_phase(const AxItem *items, int n_items, int max_n, float2 *out) {
    const int64_t n = (int64_t)n_items * max_n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t it = i / max_n;
        const int j = (int)(i - it * max_n);
        const AxItem a = items[it];
        if (j >= a.n) continue;
        double t = (double)a.val[j] * a.k;
        t -= rint(t);
        double c, s;
        sincospi(2.0 * t, &s, &c);
        out[a.off + j] = make_float2((float)c, (float)s);
    }
}

// shared-memory attribute of every fused kernel on the context's device
// (set before any stream capture, which may not accept attribute changes)
template <typename R, int MODE>
void fused_attr_ni(size_t bytes) {
    fused_smem_attr(k_fused<R, 1, MODE>, bytes);
    fused_smem_attr(k_fused<R, 2, MODE>, bytes);
    fused_smem_attr(k_fused<R, 4, MODE>, bytes);
}

template <int MODE>
void fused_batch_attr(size_t bytes) {
    fused_smem_attr(k_fused_batch<float, 1, MODE>, bytes);
    fused_smem_attr(k_fused_batch<float, 2, MODE>, bytes);
    fused_smem_attr(k_fused_batch<float, 4, MODE>, bytes);
}

void prepare_fused(mrsim_ctx *) {
    const size_t f = sizeof(FusedSmem<float>), d = sizeof(FusedSmem<double>);
    fused_attr_ni<float, FM_FACTOR>(f);
    fused_attr_ni<float, FM_AXIS>(f);
    fused_attr_ni<float, FM_DIRECT>(f);
    fused_attr_ni<float, FM_FACTOR | FM_COIL>(f);
    fused_attr_ni<float, FM_AXIS | FM_COIL>(f);
    fused_attr_ni<float, FM_DIRECT | FM_COIL>(f);
    fused_attr_ni<double, FM_FACTOR>(d);
    fused_attr_ni<double, FM_DIRECT>(d);
    fused_attr_ni<double, FM_FACTOR | FM_COIL>(d);
    fused_attr_ni<double, FM_DIRECT | FM_COIL>(d);
    fused_batch_attr<FM_FACTOR>(f);
    fused_batch_attr<FM_DIRECT>(f);
    fused_batch_attr<FM_FACTOR | FM_COIL>(f);
    fused_batch_attr<FM_DIRECT | FM_COIL>(f);
}

void launch_axis_phase(mrsim_ctx *c, const AxItem *d_items, int n_items, int max_n,
                       float2 *out) {
    if (n_items <= 0 || max_n <= 0) return;
    KScope ks(c, "axis_phase");
    const int64_t n = (int64_t)n_items * max_n;
    const unsigned grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((n + 255) / 256, (int64_t)c->sm_count * 16));
    k_axis_phase<<<grid, 256, 0, c->stream>>>(d_items, n_items, max_n, out);
}

template <typename R>
void launch_event_table(mrsim_ctx *c, const EvAdv *d_adv, int n_ev, int64_t G, const double *par,
                        void *out) {
    if (n_ev <= 0 || G <= 0) return;
    KScope ks(c, sizeof(R) == 4 ? "event_table_f32" : "event_table_f64");
    const int64_t n = (int64_t)n_ev * G;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256,
                                                                          (int64_t)c->sm_count * 16));
    k_event_table<R><<<grid, 256, 0, c->stream>>>(d_adv, n_ev, G, par, (R4<R> *)out);
}

template <typename R>
void launch_group_signal(mrsim_ctx *c, const GWin *d_win, const int4 *d_blk, int n_blk,
                         const void *d_samples, const GSigTables<R> &tab, const double *Ablk,
                         double *signal) {
    if (n_blk <= 0) return;
    KScope ks(c, sizeof(R) == 4 ? "group_signal_f32" : "group_signal_f64");
    k_group_signal<R><<<n_blk, kThreads, 0, c->stream>>>(
        d_win, d_blk, (const typename GS<R>::S *)d_samples, tab, Ablk, signal, c->fx);
}

template void launch_event_table<float>(mrsim_ctx *, const EvAdv *, int, int64_t,
                                        const double *, void *);
template void launch_event_table<double>(mrsim_ctx *, const EvAdv *, int, int64_t,
                                         const double *, void *);
template void launch_fused<float>(mrsim_ctx *, const FusedArgs<float> &, int);
template void launch_event_table_batch<float>(mrsim_ctx *, const EvTabJob *, const int64_t *,
                                              int, int64_t);
template void launch_fused_batch<float>(mrsim_ctx *, const FusedArgs<float> *, const int64_t *,
                                        int, unsigned long long *, int, bool, bool);
template void launch_group_signal_batch<float>(mrsim_ctx *, const GSigJob<float> *,
                                               const int4 *, const int *, int);
template void launch_fused<double>(mrsim_ctx *, const FusedArgs<double> &, int);
template void launch_group_signal<float>(mrsim_ctx *, const GWin *, const int4 *, int,
                                         const void *, const GSigTables<float> &,
                                         const double *, double *);
template void launch_group_signal<double>(mrsim_ctx *, const GWin *, const int4 *, int,
                                          const void *, const GSigTables<double> &,
                                          const double *, double *);

}  // namespace mrsim
