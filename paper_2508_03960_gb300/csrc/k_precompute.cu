// Preparation step of the grouped method (Sec. 2.3): the combined transition
// T_g = U_{N-1} ... U_0 (Eq. 7) of one with-RF content for every group.
//
// Each step's U = I + D (App. A closed forms) is evaluated in the run
// precision as the difference D, so nothing is lost near the identity.  The
// sub-steps of a group are split into contiguous runs; each run is composed
// by one thread and the run products are combined by an ordered tree
// (composition is associative, not commutative):
//   k_precompute        one CTA per group, shared-memory tree (few long tables)
//   k_precompute_lanes  4-32 lanes per group, shuffle tree (many groups)
//   k_precompute_batch  many tables in one launch (batched jobs)
// FP64 tables compose every step in FP64.  FP32 tables compose short blocks
// of steps in FP32 registers (still in difference form) and fold each block
// into the FP64 product.
#include <algorithm>

#include "internal.h"

namespace mrsim {

namespace {

constexpr int kPreThreads = 128;

template <typename R>
struct SegT;
template <>
struct SegT<float> { using RF = RFSegF; };
template <>
struct SegT<double> { using RF = RFSegD; };

__device__ __forceinline__ void compose(double (&C)[12], const double (&B)[12],
                                        const double (&A)[12]) {
    // C = B o A for row-major 3x4 affines (A applied first)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double v = B[4 * r] * A[c] + B[4 * r + 1] * A[4 + c] + B[4 * r + 2] * A[8 + c];
            if (c == 3) v += B[4 * r + 3];
            C[4 * r + c] = v;
        }
    }
}

// T <- (I + E) T + c in FP64, as fused multiply-adds on the difference form
__device__ __forceinline__ void fold_block(double (&T)[12], const float (&E)[9],
                                           const float (&cb)[3]) {
#pragma unroll
    for (int col = 0; col < 4; ++col) {
        const double v0 = T[col], v1 = T[4 + col], v2 = T[8 + col];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const double vr = r == 0 ? v0 : r == 1 ? v1 : v2;
            T[4 * r + col] = fma((double)E[3 * r], v0,
                                 fma((double)E[3 * r + 1], v1, fma((double)E[3 * r + 2], v2, vr)));
        }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) T[4 * r + 3] += (double)cb[r];
}

// Composes sub-steps [s0, s1) of the with-RF span for one group (Eq. 7).
// Each step's U = I + D (App. A closed forms) is evaluated in R precision as
// the difference D.  FP64 tables compose every step in FP64.  FP32 tables
// first compose a few steps in registers in FP32, still in difference form
// (E <- E + D + D E, c <- c + D c + beta), and fold each block into the FP64
// accumulator (a.kb steps per block); because E is small for short blocks its
// FP32 rounding stays at the size of the steps' own FP32 evaluation error.
template <typename R>
__device__ __forceinline__ void compose_run(const PrecompArgs &a, int64_t g, int64_t s0,
                                            int64_t s1, double (&T)[12]) {
    using RFS = typename SegT<R>::RF;
    const RFS *segs = (const RFS *)a.segs;
    const int64_t *seg_off = a.seg_off;
    const double *par = a.par;
    const int64_t G = a.n_groups;
    const int gtype = a.gtype;
#pragma unroll
    for (int e = 0; e < 12; ++e) T[e] = (e % 5 == 0) ? 1.0 : 0.0;
    if (s1 <= s0) return;
    const R pos = (R)par[g], T1 = (R)par[G + g], T2 = (R)par[2 * G + g];
    const R dB0 = (R)par[3 * G + g], b1 = (R)par[4 * G + g];
    // second position of a two-axis type (its rows carry a sixth parameter)
    const int a0 = gtype_axis0(gtype), a1 = gtype_axis1(gtype);
    const R pos2 = a1 >= 0 ? (R)par[5 * G + g] : (R)0;
    const R iT1 = isinf((double)T1) ? (R)0 : (R)1 / T1;
    const R iT2 = isinf((double)T2) ? (R)0 : (R)1 / T2;
    // segment holding step s0 (binary search on the prefix offsets)
    int lo = 0, hi = a.n_seg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (seg_off[mid] <= s0) lo = mid; else hi = mid - 1;
    }
    int j = lo;
    int64_t st = s0;
    R dt_prev = (R)-1, em1 = 0, em2 = 0;
    float E[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, cb[3] = {0, 0, 0};  // open FP32 block
    int nb = 0;
    (void)E; (void)cb; (void)nb;
    while (st < s1) {
        const RFS sg = segs[j];
        const int64_t n_here = min(seg_off[j + 1], s1) - st;
        if ((R)sg.dt != dt_prev) {
            dt_prev = (R)sg.dt;
            em1 = expm1(-dt_prev * iT1);
            em2 = expm1(-dt_prev * iT2);
        }
        const R cax[3] = {(R)sg.cx, (R)sg.cy, (R)sg.cz};
        const R cA = a0 >= 0 ? cax[a0] : (R)0;
        const R cB = a1 >= 0 ? cax[a1] : (R)0;
        const R px = -b1 * (R)sg.are, py = -b1 * (R)sg.aim;
        // the gradient is zero on axes outside the group's type: Bz needs only
        // the group's positions (Sec. 2.4; two positions for a two-axis type)
        const R pz = -(cA * pos + cB * pos2 + (R)sg.cdw * dB0);
        const R th2 = px * px + py * py + pz * pz;
        R s, c2;
        rot_coeffs(th2, s, c2);
        // U - I = r (1 + d_i) + d_i delta_ij with r = R - I = s[phi]x + c2[phi]x^2
        const R r00 = -c2 * (py * py + pz * pz), r11 = -c2 * (px * px + pz * pz);
        const R r22 = -c2 * (px * px + py * py);
        const R r01 = -s * pz + c2 * px * py, r10 = s * pz + c2 * px * py;
        const R r02 = s * py + c2 * px * pz, r20 = -s * py + c2 * px * pz;
        const R r12 = -s * px + c2 * py * pz, r21 = s * px + c2 * py * pz;
        const R f2 = (R)1 + em2, f1 = (R)1 + em1;
        // D = U - I in the run precision (an FP32 table never converts it to
        // FP64: conversions run on the FP64 pipe, a small fraction of the FP32
        // rate on this GPU, and a step's D is formed once per segment)
        const R D[9] = {r00 * f2 + em2, r01 * f2, r02 * f2, r10 * f2, r11 * f2 + em2,
                        r12 * f2, r20 * f1, r21 * f1, r22 * f1 + em1};
        const R bz = -em1;
        if constexpr (sizeof(R) == 8) {
            for (int64_t q = 0; q < n_here; ++q) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const double v0 = T[c], v1 = T[4 + c], v2 = T[8 + c];
                    T[c] = v0 + (D[0] * v0 + D[1] * v1 + D[2] * v2);
                    T[4 + c] = v1 + (D[3] * v0 + D[4] * v1 + D[5] * v2);
                    T[8 + c] = v2 + (D[6] * v0 + D[7] * v1 + D[8] * v2);
                }
                T[11] += bz;
            }
        } else {
            const float(&Df)[9] = D;
            const float bzf = bz;
            for (int64_t q = 0; q < n_here; ++q) {
                float En[9], cn[3];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc)
                        En[3 * r + cc] = fmaf(Df[3 * r], E[cc],
                                              fmaf(Df[3 * r + 1], E[3 + cc],
                                                   fmaf(Df[3 * r + 2], E[6 + cc],
                                                        E[3 * r + cc] + Df[3 * r + cc])));
                    cn[r] = fmaf(Df[3 * r], cb[0], fmaf(Df[3 * r + 1], cb[1],
                                                        fmaf(Df[3 * r + 2], cb[2], cb[r])));
                }
                cn[2] += bzf;
#pragma unroll
                for (int e = 0; e < 9; ++e) E[e] = En[e];
#pragma unroll
                for (int r = 0; r < 3; ++r) cb[r] = cn[r];
                if (++nb == a.kb) {
                    fold_block(T, E, cb);
                    nb = 0;
#pragma unroll
                    for (int e = 0; e < 9; ++e) E[e] = 0.f;
                    cb[0] = cb[1] = cb[2] = 0.f;
                }
            }
        }
        st += n_here;
        ++j;
    }
    if constexpr (sizeof(R) == 4) {
        if (nb) fold_block(T, E, cb);
    }
}

// Combined transition of group g of one table (all threads of the CTA).
template <typename R>
__device__ void precompute_group(const PrecompArgs &a, int64_t g, double (*P)[12]) {
    R *out = (R *)a.out;
    // this thread's contiguous chunk of sub-steps
    double T[12];
    compose_run<R>(a, g, a.n_steps * threadIdx.x / kPreThreads,
                   a.n_steps * (threadIdx.x + 1) / kPreThreads, T);
#pragma unroll
    for (int e = 0; e < 12; ++e) P[threadIdx.x][e] = T[e];
    __syncthreads();
    // ordered tree: P[t] <- P[t + h] o P[t]
    for (int h = 1; h < kPreThreads; h <<= 1) {
        if ((threadIdx.x % (2 * h)) == 0) {
            double A[12], B[12], C[12];
#pragma unroll
            for (int e = 0; e < 12; ++e) {
                A[e] = P[threadIdx.x][e];
                B[e] = P[threadIdx.x + h][e];
            }
            compose(C, B, A);
#pragma unroll
            for (int e = 0; e < 12; ++e) P[threadIdx.x][e] = C[e];
        }
        __syncthreads();
    }
    if (threadIdx.x < 12) out[g * 12 + threadIdx.x] = (R)P[0][threadIdx.x];
    __syncthreads();
}

template <typename R>
__global__ void __launch_bounds__(kPreThreads) k_precompute(PrecompArgs a) {
    __shared__ double P[kPreThreads][12];
    if (a.gidx) {  // only the listed groups
        const int64_t n = *a.gcount;
        for (int64_t b = blockIdx.x; b < n; b += gridDim.x) precompute_group<R>(a, a.gidx[b], P);
    } else {
        for (int64_t g = blockIdx.x; g < a.n_groups; g += gridDim.x) precompute_group<R>(a, g, P);
    }
}

// Combined transitions with L lanes per group (L <= 32, several groups per
// warp): each lane composes a contiguous run of sub-steps in FP64 and the runs
// are combined by an ordered shuffle tree.  For short pulses this keeps the
// tree (which costs about as much FP64 work per level as a run) small.
template <typename R, int L>
__global__ void __launch_bounds__(256) k_precompute_lanes(PrecompArgs a) {
    const int lane = threadIdx.x & (L - 1);
    const int64_t n_items = a.gidx ? (int64_t)*a.gcount : a.n_groups;
    for (int64_t item = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / L;
         item < ((n_items + (256 / L) - 1) / (256 / L)) * (256 / L);
         item += (int64_t)gridDim.x * blockDim.x / L) {
        // every lane of a full warp takes part in the shuffles below
        const bool live = item < n_items;
        const int64_t g = live ? (a.gidx ? (int64_t)a.gidx[item] : item) : 0;
        double T[12];
        compose_run<R>(a, g, live ? a.n_steps * lane / L : 0,
                       live ? a.n_steps * (lane + 1) / L : 0, T);
        // ordered tree over the L lanes: T(lane) <- T(lane + h) o T(lane)
#pragma unroll
        for (int h = 1; h < L; h <<= 1) {
            double B[12];
#pragma unroll
            for (int e = 0; e < 12; ++e) B[e] = __shfl_down_sync(0xffffffffu, T[e], h, L);
            if ((lane % (2 * h)) == 0) {
                double C[12];
                compose(C, B, T);
#pragma unroll
                for (int e = 0; e < 12; ++e) T[e] = C[e];
            }
        }
        if (live && lane == 0) {
            R *out = (R *)a.out + g * 12;
#pragma unroll
            for (int e = 0; e < 12; ++e) out[e] = (R)T[e];
        }
    }
}

// many tables in one launch: block b serves group b - off[t] of table t
template <typename R>
__global__ void __launch_bounds__(kPreThreads) k_precompute_batch(const PrecompArgs *tabs,
                                                                  const int64_t *off, int n_tab,
                                                                  int64_t total) {
    __shared__ double P[kPreThreads][12];
    for (int64_t b = blockIdx.x; b < total; b += gridDim.x) {
        int lo = 0, hi = n_tab - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= b) lo = mid; else hi = mid - 1;
        }
        precompute_group<R>(tabs[lo], b - off[lo], P);
    }
}

}  // namespace

template <typename R>
void launch_precompute(mrsim_ctx *c, const PrecompArgs &a_in) {
    if (a_in.n_groups <= 0) return;
    PrecompArgs a = a_in;
    a.kb = c->tune[MRSIM_TUNE_PRECOMP_STEPS];
    KScope ks(c, sizeof(R) == 4 ? "precompute_f32" : "precompute_f64");
    // lanes per group: the tuned value, or by default the fewest lanes that
    // fill the GPU (every lane ends its run with a partial FP64 fold and every
    // tree level costs about one fold, FP64-pipe work: 27.5M groups of a
    // 200-step pulse take 66 ms with one lane, 90 ms with four); a whole CTA
    // only for few, long tables
    int L = c->tune[MRSIM_TUNE_PRECOMP_LANES];
    if (L == 0) {
        const int64_t fill = (int64_t)c->sm_count * 512;
        L = 1;
        while (L < 32 && a.n_groups * L < fill) L <<= 1;
        if (a.n_groups * 32 < fill && a.n_steps > 64 * 32) L = 128;
    }
    if (L >= 128) {
        const unsigned grid = (unsigned)std::min<int64_t>(a.n_groups, 1 << 20);
        k_precompute<R><<<grid, kPreThreads, 0, c->stream>>>(a);
        return;
    }
    const int64_t threads = a.n_groups * L;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((threads + 255) / 256,
                                                                          (int64_t)c->sm_count * 32));
    switch (L) {
        case 1: k_precompute_lanes<R, 1><<<grid, 256, 0, c->stream>>>(a); break;
        case 2: k_precompute_lanes<R, 2><<<grid, 256, 0, c->stream>>>(a); break;
        case 4: k_precompute_lanes<R, 4><<<grid, 256, 0, c->stream>>>(a); break;
        case 8: k_precompute_lanes<R, 8><<<grid, 256, 0, c->stream>>>(a); break;
        case 16: k_precompute_lanes<R, 16><<<grid, 256, 0, c->stream>>>(a); break;
        default: k_precompute_lanes<R, 32><<<grid, 256, 0, c->stream>>>(a); break;
    }
}

template <typename R>
void launch_precompute_batch(mrsim_ctx *c, const PrecompArgs *d_tabs, const int64_t *d_off,
                             int n_tab, int64_t total) {
    if (total <= 0) return;
    KScope ks(c, "precompute_batch");
    const unsigned grid = (unsigned)std::min<int64_t>(total, 1 << 20);
    k_precompute_batch<R><<<grid, kPreThreads, 0, c->stream>>>(d_tabs, d_off, n_tab, total);
}

template void launch_precompute<float>(mrsim_ctx *, const PrecompArgs &);
template void launch_precompute<double>(mrsim_ctx *, const PrecompArgs &);
template void launch_precompute_batch<float>(mrsim_ctx *, const PrecompArgs *, const int64_t *,
                                             int, int64_t);

}  // namespace mrsim
