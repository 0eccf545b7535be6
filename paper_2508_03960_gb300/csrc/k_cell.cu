// Cell mode of the fused grouped kernel (FP32; Sec. 2.3 update step and step
// 1 of the with-ADC method, Eq. 9).
//
// The layout sorts isochromats by (with-ADC group, with-RF group).  A cell is
// one run of a single pair: its isochromats share the primary-axis position,
// the secondary-axis position (the with-RF group's axis), T1, T2, dB0 and b1,
// so they differ only in their position on the remaining "free" axis (two
// free axes when the with-RF subsequences carry no one-axis gradient).  Every
// thread holds up to NI isochromats of ONE cell: a cell of n isochromats has
// T = ceil(n / NI) threads, thread j holding isochromats j, j + T, ... (so
// the lanes of a warp read consecutive table entries); missing isochromats
// carry M = M0 = 0 and stay zero.  Every per-group quantity becomes a
// per-thread one:
//
//  RF event:  the closed-form advance from the state time (Eqs. 4-5) factors
//             into the cell's own part Adv (primary and secondary axis phase,
//             dB0 tau, E2, E1) and the free-axis phase Q; the z-rotations Adv
//             and Q commute, so  T Adv Q M = C (Q M)  with one combined affine
//             row C = T Adv per (distinct advance, cell), built by k_cell_rows
//             from the FP32 group-factor and axis-phasor tables the
//             per-isochromat form applies.  Per isochromat: one phasor load
//             (only if the free-axis moment is nonzero) and 12 FMAs.
//  ADC event: the block-sum term of an isochromat is P_g Q_r Q_free M_xy
//             (Eq. 9): the thread sums Q_free M_xy over its isochromats,
//             multiplies once by its cell's secondary-axis phasor Q_r and its
//             group's factor P_g and stages the partial.
//  END event: the advance alone (a combined row with T = I), then the state
//             is stored at the isochromats' layout positions.
//
// M stays in registers from the first event of the span to the last.
#include <algorithm>

#include "internal.h"

namespace mrsim {

namespace {

constexpr int kThreads = 256;
constexpr int kBatch = 16;            // with-ADC windows x coils per shared-memory flush
constexpr int kAccFloats = 2048;      // block-sum staging per CTA (8 KB)
constexpr int kEvChunk = 64;          // events staged in shared memory at a time
constexpr int kPad = 0x7fffffff;      // key of a thread without isochromats

// Shared memory of a CTA for PC receive coils per pass (PC = 0: one coil,
// S = 1): kBatch / max(PC, 1) windows are staged per flush.
template <int PC>
struct CellSmem {
    static constexpr int NC = PC > 0 ? PC : 1;  // coils per pass
    static constexpr int NB = kBatch / NC;      // windows per flush
    __align__(16) float acc[kAccFloats];        // staged block sums [batch][slot][coil][re, im]
    __align__(16) CellEv sev[kEvChunk];         // staged events
    // per-thread partials of warps whose threads share one group,
    // [window][thread][coil, re/im] (row padded: conflict-free column reads)
    __align__(16) float tpart[NB][kThreads + 1][2 * NC];
    float wpart[NB][kThreads / 32][2 * NC];     // their per-warp sums
    int batch_win[NB];
    int wslot[kThreads / 32];                   // that group's slot, or -1
};

// exp(-i 2 pi sum_f r_f k_f) over the free axes from the event's tables
template <int NF>
__device__ __forceinline__ void free_phasor(const float2 *qtab, const int (&qf)[2], int f0,
                                            int f1, float &c, float &s) {
    const float2 q0 = __ldg(qtab + qf[0] + f0);
    c = q0.x;
    s = q0.y;
    if constexpr (NF == 2) {
        const float2 q1 = __ldg(qtab + qf[1] + f1);
        const float nc = __fmaf_rn(c, q1.x, -__fmul_rn(s, q1.y));
        s = __fmaf_rn(s, q1.x, __fmul_rn(c, q1.y));
        c = nc;
    }
}

// RFQ / ADQ / RB: 0 or 1 fixes the phasor flag at compile time, 2 reads it from
// the arguments.  PC: receive coils handled in this pass (0: S = 1).
// OTF: the combined rows are formed by each thread (no row table).
// One CTA's 256 threads of a launch (block blk of the thread list).
template <int NI, int NF, int RFQ, int ADQ, int RB, int PC, bool OTF>
__device__ __forceinline__ void cell_block(const CellArgs &a, int64_t blk, CellSmem<PC> &sm) {
    using Smem = CellSmem<PC>;
    constexpr int NC = Smem::NC, NB = Smem::NB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t t0 = blk * kThreads;
    const int64_t t = t0 + tid;
    const int64_t t_end = min(t0 + kThreads, a.n_thr);  // threads with work in this CTA
    const float2 *qtab = a.qtab;
    const bool rfq = RFQ == 2 ? a.rfq != 0 : RFQ == 1;
    const bool adq = ADQ == 2 ? a.adq != 0 : ADQ == 1;
    const bool rb = RB == 2 ? a.rb != 0 : RB == 1;

    float mx[NI], my[NI], mz[NI], M0[NI];
    float sre[NC][NI], sim[NC][NI];  // receive sensitivities (PC > 0)
    int f0[NI], f1[NI];  // free-axis table indices of each isochromat
    // isochromat i of this thread is layout position start + i * stride
    int key = kPad, cell = 0, start = 0, stride = 0, n = 0, ridx = 0;
    int g_sec = 0, g_none = 0;  // the cell's secondary and no-grads groups (rows per thread)
    if (t < a.n_thr) {
        const int2 d = a.thr[t];
        start = d.x;
        cell = d.y >> 4;
        n = min(d.y & 15, NI);  // descriptors are built for this width
        key = a.cell_gp[cell];
        stride = (a.cell_count[cell] + NI - 1) / NI;
        if constexpr (OTF) {
            if (a.gtype_r >= 0) g_sec = a.cell_gr[cell];
            if (a.gid[G_NONE]) g_none = a.gid[G_NONE][start];
        }
    }
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        int ai = 0;
        if (i < n) {
            const int k = start + i * stride;
            M0[i] = a.M0[k];
            ai = a.aidx[k];
            if (a.init_eq) {
                mx[i] = 0.0f;
                my[i] = 0.0f;
                mz[i] = M0[i];
            } else {
                mx[i] = a.Mx[k];
                my[i] = a.My[k];
                mz[i] = a.Mz[k];
            }
            if constexpr (PC > 0) {
#pragma unroll
                for (int j = 0; j < NC; ++j) {
                    sre[j][i] = a.coil[(2 * j) * a.K + k];
                    sim[j][i] = a.coil[(2 * j + 1) * a.K + k];
                }
            }
        } else {
            M0[i] = mx[i] = my[i] = mz[i] = 0.0f;
            if constexpr (PC > 0) {
#pragma unroll
                for (int j = 0; j < NC; ++j) sre[j][i] = sim[j][i] = 0.0f;
            }
        }
        f0[i] = (ai >> a.f_sh[0]) & 0xffff;
        f1[i] = NF == 2 ? (ai >> a.f_sh[1]) & 0xffff : 0;
        if (i == 0 && (RB != 0 || OTF)) ridx = (ai >> a.r_sh) & 0xffff;
    }
    // primary groups of this CTA: keys rise along the threads and every group
    // between the first and the last one has isochromats here
    const int32_t g_first = a.cell_gp[a.thr[t0].y >> 4];
    const int32_t g_last = a.cell_gp[a.thr[t_end - 1].y >> 4];
    const int S = (int)(g_last - g_first + 1);  // at most kThreads
    const int B = max(1, min(NB, kAccFloats / (2 * NC * S)));
    for (int i = tid; i < B * S * 2 * NC; i += kThreads) sm.acc[i] = 0.0f;
    // a warp whose threads all share one group stages per-thread partials
    const int32_t w0 = __shfl_sync(0xffffffffu, key, 0);
    const bool warp_uni = __all_sync(0xffffffffu, key == w0 || key == kPad) && w0 != kPad;
    if (lane == 0) sm.wslot[warp] = warp_uni ? w0 - g_first : -1;
    const bool any_uni = __syncthreads_or(warp_uni) != 0;
    const float4 *Pt = reinterpret_cast<const float4 *>(a.P_raw);
    const int pkey = key == kPad ? g_first : key;  // group-factor column (padding: any valid)

    int nb = 0;  // windows staged (uniform)
    auto flush = [&]() {
        if (warp_uni) {
            // column sums of this warp's staged partials: lane (h, b) adds
            // 32 / H threads of part h for window b (H = 32 / NB), then the
            // parts combine
            __syncwarp();
            constexpr int H = 32 / NB, J = 32 / H;
            const int b = lane % NB, h = lane / NB;
            float sr[2 * NC];
#pragma unroll
            for (int v = 0; v < 2 * NC; ++v) sr[v] = 0.0f;
            if (b < nb) {
                const float(*col)[2 * NC] = &sm.tpart[b][warp * 32 + h * J];
#pragma unroll
                for (int j = 0; j < J; ++j) {
#pragma unroll
                    for (int v = 0; v < 2 * NC; ++v) sr[v] += col[j][v];
                }
            }
#pragma unroll
            for (int o = 16; o >= NB; o >>= 1) {
#pragma unroll
                for (int v = 0; v < 2 * NC; ++v) sr[v] += __shfl_xor_sync(0xffffffffu, sr[v], o);
            }
            if (h == 0 && b < nb) {
#pragma unroll
                for (int v = 0; v < 2 * NC; ++v) sm.wpart[b][warp][v] = sr[v];
            }
        }
        __syncthreads();
        for (int q = tid; q < nb * S * NC; q += kThreads) {
            const int b = q / (S * NC), r = q - b * S * NC, slot = r / NC, j = r - slot * NC;
            float sr = sm.acc[2 * q], si = sm.acc[2 * q + 1];
            if (any_uni) {
#pragma unroll
                for (int w = 0; w < kThreads / 32; ++w) {
                    if (sm.wslot[w] == slot) {
                        sr += sm.wpart[b][w][2 * j];
                        si += sm.wpart[b][w][2 * j + 1];
                    }
                }
            }
            if (sr != 0.0f || si != 0.0f) {
                const int64_t o =
                    2 * (a.ablk_stride * j + (int64_t)sm.batch_win[b] + g_first + slot);
                if (slot != 0 && slot != S - 1 && a.fx == 0.0) {
                    // a group strictly inside the CTA has no other contributor
                    *reinterpret_cast<double2 *>(&a.Ablk[o]) = make_double2(sr, si);
                } else {
                    // (reproducible sums: the non-uniform warps add theirs
                    // directly, so every slot is added)
                    sum_add(&a.Ablk[o], (double)sr, a.fx);
                    sum_add(&a.Ablk[o + 1], (double)si, a.fx);
                }
            }
            // cleared even when the total is zero: staged partials can cancel
            // exactly, and a value left here would be added to a later window
            sm.acc[2 * q] = 0.0f;
            sm.acc[2 * q + 1] = 0.0f;
        }
        __syncthreads();
        nb = 0;
    };

    auto stage = [&](int win, float (&sr)[NC], float (&si)[NC]) {
        if (warp_uni) {
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                sm.tpart[nb][tid][2 * j] = sr[j];
                sm.tpart[nb][tid][2 * j + 1] = si[j];
            }
        } else {
            // keys rise along the lanes: a segmented inclusive scan leaves each
            // run's sum in the run's last lane
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t ok = __shfl_up_sync(0xffffffffu, key, d);
#pragma unroll
                for (int j = 0; j < NC; ++j) {
                    const float orr = __shfl_up_sync(0xffffffffu, sr[j], d);
                    const float oii = __shfl_up_sync(0xffffffffu, si[j], d);
                    if (lane >= d && ok == key) {
                        sr[j] += orr;
                        si[j] += oii;
                    }
                }
            }
            const int32_t nk = __shfl_down_sync(0xffffffffu, key, 1);
            if ((lane == 31 || nk != key) && key != kPad) {
                if (a.fx > 0.0) {
                    // reproducible sums: the run's total goes to the block sum
                    // as an integer (the shared accumulator's float atomics
                    // would depend on the order of the warps)
#pragma unroll
                    for (int j = 0; j < NC; ++j) {
                        const int64_t o = 2 * (a.ablk_stride * j + (int64_t)win + key);
                        sum_add(&a.Ablk[o], (double)sr[j], a.fx);
                        sum_add(&a.Ablk[o + 1], (double)si[j], a.fx);
                    }
                } else {
                    float *accb = sm.acc + 2 * NC * (nb * S + (key - g_first));
#pragma unroll
                    for (int j = 0; j < NC; ++j) {
                        atomicAdd(accb + 2 * j, sr[j]);
                        atomicAdd(accb + 2 * j + 1, si[j]);
                    }
                }
            }
        }
        if (tid == 0) sm.batch_win[nb] = win;
        ++nb;
        if (nb == B) flush();
    };

    for (int e0 = 0; e0 < a.n_ev; e0 += kEvChunk) {
        const int ne = min(kEvChunk, a.n_ev - e0);
        __syncthreads();
        {
            const int4 *src = reinterpret_cast<const int4 *>(a.ev + e0);
            int4 *dst = reinterpret_cast<int4 *>(sm.sev);
            const int nw = ne * (int)(sizeof(CellEv) / sizeof(int4));
            for (int q = tid; q < nw; q += kThreads) dst[q] = src[q];
        }
        __syncthreads();
#pragma unroll 1
        for (int e = 0; e < ne; ++e) {
            const int4 ev0 = *reinterpret_cast<const int4 *>(&sm.sev[e]);
            const int kind = ev0.x;
            if (kind <= CE_END) {
                // RF: advance and transition, M <- C (Q M); END: the advance
                // alone (C built with T = I), then the state is stored
                float4 r0, r1, r2;
                if constexpr (!OTF) {
                    const float4 *cr =
                        reinterpret_cast<const float4 *>(a.C_tab + ((int64_t)ev0.y + cell) * 12);
                    r0 = __ldg(cr);
                    r1 = __ldg(cr + 1);
                    r2 = __ldg(cr + 2);
                } else {
                    // the row C = T Adv of this cell, as the row table would
                    // hold it: the group factor (E2 e^{-i phi}, E1) of the
                    // cell's primary group, times the secondary-axis phasor,
                    // under the transition of the pulse's group
                    const int4 ev1 = *reinterpret_cast<const int4 *>(&sm.sev[e].qf[0]);
                    const float4 P = __ldg(Pt + sm.sev[e].prow + pkey);
                    float fr = P.x, fi = P.y;
                    if (ev1.z >= 0) {
                        const float2 q = __ldg(qtab + ev1.z + ridx);
                        const float tr = fr * q.x + fi * q.y;  // P exp(-i psi)
                        fi = fi * q.x - fr * q.y;
                        fr = tr;
                    }
                    const float E1 = P.z, u = 1.0f - P.z;
                    if (ev0.z < 0) {
                        r0 = make_float4(fr, -fi, 0.0f, 0.0f);
                        r1 = make_float4(fi, fr, 0.0f, 0.0f);
                        r2 = make_float4(0.0f, 0.0f, E1, u);
                    } else {
                        const int gt =
                            ev0.w == a.gtype_p ? pkey : ev0.w == a.gtype_r ? g_sec : g_none;
                        const float4 *T =
                            reinterpret_cast<const float4 *>(a.T_tab + ((int64_t)ev0.z + gt) * 12);
                        float4 tv[3] = {__ldg(T), __ldg(T + 1), __ldg(T + 2)};
                        float4 rr[3];
#pragma unroll
                        for (int row = 0; row < 3; ++row) {
                            const float4 tt = tv[row];  // A0, A1, A2, b
                            rr[row] = make_float4(tt.x * fr + tt.y * fi, tt.y * fr - tt.x * fi,
                                                  tt.z * E1, fmaf(tt.z, u, tt.w));
                        }
                        r0 = rr[0];
                        r1 = rr[1];
                        r2 = rr[2];
                    }
                }
                int qf[2] = {0, 0};
                if (rfq) {
                    const int4 ev1 = *reinterpret_cast<const int4 *>(&sm.sev[e].qf[0]);
                    qf[0] = ev1.x;
                    qf[1] = ev1.y;
                }
#pragma unroll
                for (int i = 0; i < NI; ++i) {
                    float x = mx[i], y = my[i];
                    if (rfq) {
                        float c, s;
                        free_phasor<NF>(qtab, qf, f0[i], f1[i], c, s);
                        // (c - i s) (x + i y)
                        const float nx = __fmaf_rn(c, x, __fmul_rn(s, y));
                        y = __fmaf_rn(c, y, -__fmul_rn(s, x));
                        x = nx;
                    }
                    const float z = mz[i], m0 = M0[i];
                    mx[i] = __fmaf_rn(r0.w, m0, __fmaf_rn(r0.z, z, __fmaf_rn(r0.y, y, __fmul_rn(r0.x, x))));
                    my[i] = __fmaf_rn(r1.w, m0, __fmaf_rn(r1.z, z, __fmaf_rn(r1.y, y, __fmul_rn(r1.x, x))));
                    mz[i] = __fmaf_rn(r2.w, m0, __fmaf_rn(r2.z, z, __fmaf_rn(r2.y, y, __fmul_rn(r2.x, x))));
                }
                if (kind == CE_END && a.Mx) {
#pragma unroll
                    for (int i = 0; i < NI; ++i) {
                        if (i < n) {
                            const int k = start + i * stride;
                            a.Mx[k] = mx[i];
                            a.My[k] = my[i];
                            a.Mz[k] = mz[i];
                        }
                    }
                }
            } else {
                // with-ADC window: block-sum term P_g Q_r sum_i S_i Q_free M_xy
                // (Eqs. 6, 9); the group factor is issued first, it multiplies
                // the sums
                const float4 P = __ldg(Pt + ev0.y + pkey);
                const int4 ev1 = *reinterpret_cast<const int4 *>(&sm.sev[e].qf[0]);
                float sr[NC], si[NC];
#pragma unroll
                for (int j = 0; j < NC; ++j) sr[j] = si[j] = 0.0f;
                const int qf[2] = {ev1.x, ev1.y};
                // (roundings written out: every 4-wide instantiation, with
                // coils or without, forms the same products and sums, so a unit
                // coil gives the bits of none; reproducible sums and the coil
                // kernels are 4-wide.  The 8-wide form folds the rotation into
                // the sum, two FMAs per component)
#pragma unroll
                for (int i = 0; i < NI; ++i) {
                    float vr = mx[i], vi = my[i];
                    if constexpr (NI == 8 && PC == 0) {
                        if (adq) {
                            float c, s;
                            free_phasor<NF>(qtab, qf, f0[i], f1[i], c, s);
                            sr[0] = fmaf(c, mx[i], fmaf(s, my[i], sr[0]));
                            si[0] = fmaf(c, my[i], fmaf(-s, mx[i], si[0]));
                        } else {
                            sr[0] += vr;
                            si[0] += vi;
                        }
                        continue;
                    }
                    if (adq) {
                        float c, s;
                        free_phasor<NF>(qtab, qf, f0[i], f1[i], c, s);
                        vr = __fmaf_rn(c, mx[i], __fmul_rn(s, my[i]));
                        vi = __fmaf_rn(c, my[i], -__fmul_rn(s, mx[i]));
                    }
                    if constexpr (PC > 0) {
#pragma unroll
                        for (int j = 0; j < NC; ++j) {
                            sr[j] = __fadd_rn(sr[j], __fmaf_rn(sre[j][i], vr,
                                                               -__fmul_rn(sim[j][i], vi)));
                            si[j] = __fadd_rn(si[j], __fmaf_rn(sre[j][i], vi,
                                                               __fmul_rn(sim[j][i], vr)));
                        }
                    } else {
                        sr[0] = __fadd_rn(sr[0], vr);
                        si[0] = __fadd_rn(si[0], vi);
                    }
                }
                // the factor shared by the thread's isochromats: the group's P
                // times the cell's secondary-axis phasor
                float fr = P.x, fi = P.y;
                if (rb) {
                    const float2 q = __ldg(qtab + ev1.z + ridx);
                    const float tr = __fmaf_rn(fr, q.x, __fmul_rn(fi, q.y));  // P exp(-i psi)
                    fi = __fmaf_rn(fi, q.x, -__fmul_rn(fr, q.y));
                    fr = tr;
                }
#pragma unroll
                for (int j = 0; j < NC; ++j) {
                    const float nr = __fmaf_rn(fr, sr[j], -__fmul_rn(fi, si[j]));
                    si[j] = __fmaf_rn(fr, si[j], __fmul_rn(fi, sr[j]));
                    sr[j] = nr;
                }
                if (kind == CE_ADC) {
                    stage(ev0.z, sr, si);
                } else if (n > 0) {
                    // a window of the secondary or no-grads type: its group is
                    // constant in the cell, the thread adds its term directly
                    const int64_t g = a.gid[ev0.w][start];
#pragma unroll
                    for (int j = 0; j < NC; ++j) {
                        const int64_t o = 2 * (a.ablk_stride * j + (int64_t)ev0.z + g);
                        sum_add(&a.Ablk[o], (double)sr[j], a.fx);
                        sum_add(&a.Ablk[o + 1], (double)si[j], a.fx);
                    }
                }
            }
        }
    }
    if (nb > 0) flush();
}

template <int NI, int NF, int RFQ, int ADQ, int RB, int PC, bool OTF>
__global__ void __launch_bounds__(kThreads, (PC >= 2 ? 2 : PC == 1 ? 3 : NI == 4 ? 4 : 2))
    k_fused_cell(CellArgs a) {
    __shared__ CellSmem<PC> sm;
    cell_block<NI, NF, RFQ, ADQ, RB, PC, OTF>(a, blockIdx.x, sm);
}

// Persistent form for a batch of jobs (one coil, phasor flags read at run
// time): every CTA takes the next (job, block) work item from a device counter
// until all blocks of all jobs are done.
template <int NI, int NF, bool OTF>
__global__ void __launch_bounds__(kThreads, (NI == 4 ? 3 : 2))
    k_fused_cell_batch(const CellArgs *jobs, const int64_t *blk_off, int n_jobs,
                       unsigned long long *counter) {
    __shared__ CellSmem<0> sm;
    __shared__ CellArgs ja;
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
        cell_block<NI, NF, 2, 2, 2, 0, OTF>(ja, jblk, sm);
        __syncthreads();  // the item's shared state is free before the next one
    }
}

template <int NI, int NF, bool RFQ, bool ADQ, bool RB>
void launch_cell_v(mrsim_ctx *c, const CellArgs &a) {
    const unsigned nb = (unsigned)((a.n_thr + kThreads - 1) / kThreads);
    k_fused_cell<NI, NF, RFQ, ADQ, RB, 0, false><<<nb, kThreads, 0, c->stream>>>(a);
}
// receive coils: 4 isochromats per thread, phasor flags read at run time
template <int NF, int PC, bool OTF>
void launch_cell_coil(mrsim_ctx *c, const CellArgs &a) {
    const unsigned nb = (unsigned)((a.n_thr + kThreads - 1) / kThreads);
    k_fused_cell<4, NF, 2, 2, 2, PC, OTF><<<nb, kThreads, 0, c->stream>>>(a);
}
// rows formed per thread: phasor flags read at run time
template <int NI, int NF>
void launch_cell_otf(mrsim_ctx *c, const CellArgs &a) {
    const unsigned nb = (unsigned)((a.n_thr + kThreads - 1) / kThreads);
    k_fused_cell<NI, NF, 2, 2, 2, 0, true><<<nb, kThreads, 0, c->stream>>>(a);
}
template <int NI, int NF, bool RFQ, bool ADQ>
void launch_cell_rb(mrsim_ctx *c, const CellArgs &a, bool rb) {
    if (rb) launch_cell_v<NI, NF, RFQ, ADQ, true>(c, a);
    else launch_cell_v<NI, NF, RFQ, ADQ, false>(c, a);
}
template <int NI, int NF>
void launch_cell_q(mrsim_ctx *c, const CellArgs &a, const CellForm &f) {
    if (f.rfq && f.adq) launch_cell_rb<NI, NF, true, true>(c, a, f.rb);
    else if (f.rfq) launch_cell_rb<NI, NF, true, false>(c, a, f.rb);
    else if (f.adq) launch_cell_rb<NI, NF, false, true>(c, a, f.rb);
    else launch_cell_rb<NI, NF, false, false>(c, a, f.rb);
}

// C = T Adv for every (key, cell).  Adv is the advance of Eqs. 4-5 that the
// per-isochromat form applies in FP32 per isochromat, from the same tables:
// the group factor (E2 e^{-i phi_p}, E1) of the cell's primary group at the
// key's first event, times the phasor of the cell's secondary-axis position
// (when that moment is nonzero); T is the cell's combined transition row of
// the key's gradient type (Eq. 7), or the identity for the end of a span.
__global__ void k_cell_rows(const CellKey *keys, int n_keys, int64_t nc, const int32_t *cstart,
                            const int32_t *cgp, const int32_t *cgr, const int32_t *gid_none,
                            int p, int r, const float4 *Pt, const float2 *qtab,
                            const int32_t *aidx, int r_sh, const float *T_tab, float *C) {
    const int64_t n = (int64_t)n_keys * nc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / nc, c = i - j * nc;
        const CellKey k = keys[j];
        const int gp = cgp[c];
        const float4 P = __ldg(Pt + k.prow + gp);
        float fr = P.x, fi = P.y;
        if (k.qr >= 0) {
            const float2 q = __ldg(qtab + k.qr + ((aidx[cstart[c]] >> r_sh) & 0xffff));
            const float tr = fr * q.x + fi * q.y;  // P exp(-i psi)
            fi = fi * q.x - fr * q.y;
            fr = tr;
        }
        // Adv: mx' = fr mx - fi my, my' = fr my + fi mx, mz' = E1 mz + (1 - E1) M0
        const float E1 = P.z, u = 1.0f - P.z;
        float4 *o = reinterpret_cast<float4 *>(C + i * 12);
        if (k.trow < 0) {
            o[0] = make_float4(fr, -fi, 0.0f, 0.0f);
            o[1] = make_float4(fi, fr, 0.0f, 0.0f);
            o[2] = make_float4(0.0f, 0.0f, E1, u);
            continue;
        }
        const int gt = k.gtype == p ? gp : k.gtype == r ? cgr[c] : gid_none[cstart[c]];
        const float4 *T = reinterpret_cast<const float4 *>(T_tab + (k.trow + gt) * 12);
#pragma unroll
        for (int row = 0; row < 3; ++row) {
            const float4 t = __ldg(T + row);  // A0, A1, A2, b
            o[row] = make_float4(t.x * fr + t.y * fi, t.y * fr - t.x * fi, t.z * E1,
                                 fmaf(t.z, u, t.w));
        }
    }
}

}  // namespace

template <bool OTF>
void launch_cell_coils(mrsim_ctx *c, const CellArgs &b, const CellForm &f) {
    if (f.nf == 2) {
        if (f.pc == 4) launch_cell_coil<2, 4, OTF>(c, b);
        else if (f.pc == 2) launch_cell_coil<2, 2, OTF>(c, b);
        else launch_cell_coil<2, 1, OTF>(c, b);
    } else {
        if (f.pc == 4) launch_cell_coil<1, 4, OTF>(c, b);
        else if (f.pc == 2) launch_cell_coil<1, 2, OTF>(c, b);
        else launch_cell_coil<1, 1, OTF>(c, b);
    }
}

void launch_fused_cell(mrsim_ctx *c, const CellArgs &a, const CellForm &f) {
    if (a.n_thr <= 0) return;
    CellArgs b = a;
    b.rfq = f.rfq;
    b.adq = f.adq;
    b.rb = f.rb;
    if (f.pc > 0) {
        KScope ks(c, "fused_cell_coils_f32");
        if (a.otf) launch_cell_coils<true>(c, b, f);
        else launch_cell_coils<false>(c, b, f);
        return;
    }
    KScope ks(c, "fused_cell_f32");
    if (a.otf) {
        if (f.ni == 8) {
            if (f.nf == 2) launch_cell_otf<8, 2>(c, b);
            else launch_cell_otf<8, 1>(c, b);
        } else {
            if (f.nf == 2) launch_cell_otf<4, 2>(c, b);
            else launch_cell_otf<4, 1>(c, b);
        }
        return;
    }
    if (f.ni == 8) {
        if (f.nf == 2) launch_cell_q<8, 2>(c, a, f);
        else launch_cell_q<8, 1>(c, a, f);
    } else {
        if (f.nf == 2) launch_cell_q<4, 2>(c, a, f);
        else launch_cell_q<4, 1>(c, a, f);
    }
}

template <int NI, int NF, bool OTF>
void launch_cell_batch_v(mrsim_ctx *c, const CellArgs *d_jobs, const int64_t *d_blk_off,
                         int n_jobs, unsigned long long *d_counter) {
    int per_sm = 1;
    MRSIM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_fused_cell_batch<NI, NF, OTF>, kThreads, 0));
    k_fused_cell_batch<NI, NF, OTF><<<std::max(1, per_sm) * c->sm_count, kThreads, 0,
                                      c->stream>>>(d_jobs, d_blk_off, n_jobs, d_counter);
}

void launch_fused_cell_batch(mrsim_ctx *c, const CellArgs *d_jobs, const int64_t *d_blk_off,
                             int n_jobs, unsigned long long *d_counter, int ni, int nf,
                             bool otf) {
    KScope ks(c, "fused_cell_batch");
    if (ni == 8) {
        if (nf == 2) otf ? launch_cell_batch_v<8, 2, true>(c, d_jobs, d_blk_off, n_jobs, d_counter)
                         : launch_cell_batch_v<8, 2, false>(c, d_jobs, d_blk_off, n_jobs, d_counter);
        else otf ? launch_cell_batch_v<8, 1, true>(c, d_jobs, d_blk_off, n_jobs, d_counter)
                 : launch_cell_batch_v<8, 1, false>(c, d_jobs, d_blk_off, n_jobs, d_counter);
    } else {
        if (nf == 2) otf ? launch_cell_batch_v<4, 2, true>(c, d_jobs, d_blk_off, n_jobs, d_counter)
                         : launch_cell_batch_v<4, 2, false>(c, d_jobs, d_blk_off, n_jobs, d_counter);
        else otf ? launch_cell_batch_v<4, 1, true>(c, d_jobs, d_blk_off, n_jobs, d_counter)
                 : launch_cell_batch_v<4, 1, false>(c, d_jobs, d_blk_off, n_jobs, d_counter);
    }
}

void launch_cell_rows(mrsim_ctx *c, const CellKey *d_keys, int n_keys, const mrsim_groups *g,
                      const float *T_tab, const void *P_tab, const float2 *qtab, int r_sh,
                      float *C) {
    const int64_t nc = g->n_cells;
    const int64_t n = (int64_t)n_keys * nc;
    if (n <= 0) return;
    const int p = g->primary, r = g->secondary;
    KScope ks(c, "cell_rows");
    const unsigned grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((n + 255) / 256, (int64_t)c->sm_count * 16));
    k_cell_rows<<<grid, 256, 0, c->stream>>>(
        d_keys, n_keys, nc, g->cell_start.as<int32_t>(), g->cell_gp.as<int32_t>(),
        g->cell_gr.as<int32_t>(), g->built[G_NONE] ? g->gid_sorted[G_NONE].as<int32_t>() : nullptr,
        p, r, reinterpret_cast<const float4 *>(P_tab), qtab, g->ax_idx.as<int32_t>(), r_sh, T_tab,
        C);
}

}  // namespace mrsim
