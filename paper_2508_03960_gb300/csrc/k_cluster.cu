// Group-reducing preprocessing of a phantom (Sec. 3.3, Fig. 4): a bisecting
// K-means of the isochromats' (T1, T2, dB0), every isochromat then carries its
// cluster's centre values, and M0 is refitted to the T2-weighted images with
// those values.
//
// Features are integers x_i = rint(v_i s_i) (T1 and T2 in 1/64 ms and dB0 in
// 1/64 Hz by default), so every sum is exact: counts, sums and sums of squares
// are 64-bit (squares 128-bit as two words) and do not depend on the order of
// the atomics.  Centres are FP64 means (exact sum / count, one rounding) and
// distances to them are formed with one rounding per operation, so the
// partition does not depend on the launch configuration.
//
// Isochromats with equal features always fall on the same side, so the
// clustering runs over the U distinct keys (features, T1 and T2 bit patterns;
// the latter for the M0 refit), each weighted by its number of isochromats;
// keys are numbered by first occurrence, so "the smallest isochromat index" in
// the tie rules is "the smallest key id".
//
// One split of cluster c (the one with the largest SSE, ties to the smaller
// id; SSEs are compared as exact rationals, 128-bit integers, on the device):
//   a = member farthest from the mean, b = member farthest from a;
//   2-means from centres (a, b): side 1 iff strictly nearer centre 1; centres
//   = side means; until the centres repeat, max_iter passes, or a side would
//   be empty (the previous pass stands).  Side 0 keeps id c, side 1 takes the
//   next id.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace mrsim {

namespace {

constexpr int kClThreads = 256;
constexpr double kMaxFeature = 1048576.0;  // 2^20

// Sums over one side of a split (exact integers).
struct ClStats {
    unsigned long long n;         // sum of weights (isochromats)
    unsigned long long sx[3];     // sum w x_i, two's complement
    unsigned long long sq[3][2];  // sum w x_i^2 as (low, high) words
};

// Device work area of the split in progress.  The split is decided on the
// device: k_cl_choose picks the cluster, k_cl_update advances the 2-means
// passes and decides when they stop, k_cl_commit records the two sides.
struct ClWork {
    double cen[6];                // centres of side 0 and side 1, feature units
    unsigned long long dmax[2];   // farthest-member searches: largest distance
    int32_t umin[2];              // ... and the smallest key id at it
    ClStats st[2];                // sums of the pass in progress
    double kept_cen[6];           // centres of the last pass with both sides filled
    ClStats kept[2];              // ... and its sums
    int32_t cid, nid;             // cluster being split (-1: none left), id of side 1
    int32_t done, have, passes;   // 2-means stopped; a pass was kept; passes run
    int32_t n_cur;                // clusters made so far
};

// Per-thread partial sums (plain data: also held in shared memory).
struct ClAcc {
    unsigned long long n;
    long long sx[3];
    unsigned long long lo[3], hi[3];

    __device__ __forceinline__ void zero() {
        n = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            sx[i] = 0;
            lo[i] = 0;
            hi[i] = 0;
        }
    }

    __device__ __forceinline__ void add(unsigned long long w, int32_t a, int32_t b, int32_t c) {
        const int32_t x[3] = {a, b, c};
        n += w;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            sx[i] += (long long)w * x[i];
            const unsigned long long xx = (unsigned long long)((long long)x[i] * x[i]);
            const unsigned long long pl = w * xx, ph = __umul64hi(w, xx);
            const unsigned long long s = lo[i] + pl;
            hi[i] += ph + (s < pl ? 1ull : 0ull);
            lo[i] = s;
        }
    }
    __device__ __forceinline__ void merge(const ClAcc &o) {
        n += o.n;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            sx[i] += o.sx[i];
            const unsigned long long s = lo[i] + o.lo[i];
            hi[i] += o.hi[i] + (s < o.lo[i] ? 1ull : 0ull);
            lo[i] = s;
        }
    }
    __device__ __forceinline__ void shfl_down(int off) {
        ClAcc o;
        o.n = __shfl_down_sync(0xffffffffu, n, off);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            o.sx[i] = __shfl_down_sync(0xffffffffu, sx[i], off);
            o.lo[i] = __shfl_down_sync(0xffffffffu, lo[i], off);
            o.hi[i] = __shfl_down_sync(0xffffffffu, hi[i], off);
        }
        merge(o);
    }
    __device__ __forceinline__ void flush(ClStats *g) const {
        if (n == 0) return;
        atomicAdd(&g->n, n);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            atomicAdd(&g->sx[i], (unsigned long long)sx[i]);
            const unsigned long long old = atomicAdd(&g->sq[i][0], lo[i]);
            const unsigned long long carry = (old + lo[i] < lo[i]) ? 1ull : 0ull;
            if (hi[i] + carry) atomicAdd(&g->sq[i][1], hi[i] + carry);
        }
    }
};

// ((x0 - m0)^2 + (x1 - m1)^2) + (x2 - m2)^2, one rounding per operation
__device__ __forceinline__ double cl_dist(int32_t a, int32_t b, int32_t c, const double *m) {
    const double d0 = __dsub_rn((double)a, m[0]);
    const double d1 = __dsub_rn((double)b, m[1]);
    const double d2 = __dsub_rn((double)c, m[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
}

__device__ __forceinline__ int cl_side(int32_t a, int32_t b, int32_t c, const double *cen) {
    return cl_dist(a, b, c, cen + 3) < cl_dist(a, b, c, cen) ? 1 : 0;
}

__global__ void k_cl_quant(int64_t K, const float *T1, const float *T2, const float *dB0,
                           double s0, double s1, double s2, int32_t *x, int *err) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x) {
        const float v[3] = {T1[k], T2[k], dB0[k]};
        const double s[3] = {s0, s1, s2};
        bool bad = false;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double q = rint(__dmul_rn((double)v[i], s[i]));
            const bool ok = isfinite(v[i]) && fabs(q) <= kMaxFeature && (i == 2 || q >= 1.0);
            bad |= !ok;
            x[i * K + k] = ok ? (int32_t)q : 0;
        }
        if (bad) atomicOr(err, 1);
    }
}

// rint(v * S) for a float v and an integer scale S < 2^24 in integer
// arithmetic: v = m 2^e with an integer m < 2^24, so v S = (m S) 2^e exactly
// (m S < 2^48; the FP64 product of the other path is exact as well) and
// rint is a right shift rounding half to even.  ok: v finite and the result
// within 2^62 (the caller checks the feature range).
__device__ __forceinline__ long long quant_int(float v, long long S, bool &ok) {
    const uint32_t b = __float_as_uint(v);
    const int ex = (int)((b >> 23) & 0xff);
    ok = ex != 0xff;
    if (!ok) return 0;
    uint64_t m = b & 0x7fffffu;
    int e;
    if (ex == 0) {
        e = -149;  // subnormal: m 2^-149
    } else {
        m |= 0x800000u;
        e = ex - 150;  // m 2^(ex - 127 - 23)
    }
    const uint64_t p = m * (uint64_t)S;
    uint64_t q;
    if (p == 0) {
        q = 0;
    } else if (e >= 0) {
        if (e > 14) {  // beyond 2^62 (p >= 2^0): out of every feature range
            ok = false;
            return 0;
        }
        q = p << e;
    } else if (e <= -64) {
        q = 0;  // below one half
    } else {
        const int k = -e;
        const uint64_t fl = p >> k, rem = p & ((1ull << k) - 1ull), half = 1ull << (k - 1);
        q = fl + ((rem > half || (rem == half && (fl & 1ull))) ? 1ull : 0ull);
    }
    return (b >> 31) ? -(long long)q : (long long)q;
}

__global__ void k_cl_quant_int(int64_t K, const float *T1, const float *T2, const float *dB0,
                               long long s0, long long s1, long long s2, int32_t *x, int *err) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x) {
        const float v[3] = {T1[k], T2[k], dB0[k]};
        const long long s[3] = {s0, s1, s2};
        bool bad = false;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            bool fin;
            const long long q = quant_int(v[i], s[i], fin);
            const bool ok = fin && (q <= (long long)kMaxFeature && q >= -(long long)kMaxFeature) &&
                            (i == 2 || q >= 1);
            bad |= !ok;
            x[i * K + k] = ok ? (int32_t)q : 0;
        }
        if (bad) atomicOr(err, 1);
    }
}

using u128 = unsigned __int128;

// n * SSE of a cluster's exact sums: sum_i (n sum w x_i^2 - (sum w x_i)^2)
__device__ __forceinline__ u128 cl_nsse(const ClStats &s) {
    u128 N = 0;
    for (int i = 0; i < 3; ++i) {
        const u128 sq = ((u128)s.sq[i][1] << 64) | s.sq[i][0];
        const long long x = (long long)s.sx[i];
        const u128 a = x < 0 ? (u128)(-x) : (u128)x;
        N += (u128)s.n * sq - a * a;
    }
    return N;
}

// One cluster of the device table: its exact sums and n * SSE (two words).
struct ClEntry {
    ClStats s;
    unsigned long long N[2];  // low, high
};

// Last-block completion: every block adds one to the counter after its
// results are visible (fence first); the block that brings it to gridDim.x
// finishes the step alone and resets the counter for the next launch.  No
// block waits for another.
__device__ __forceinline__ bool cl_last_block(unsigned int *counter) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int prev = atomicAdd(counter, 1u);
        last = prev == gridDim.x - 1;
        if (last) *counter = 0u;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// the next split, chosen by one block: the cluster with the largest SSE,
// compared as exact rationals N_a / n_a > N_b / n_b, ties to the smaller id
// (clusters of one distinct value have N = 0 and are never split); its mean
// seeds the farthest-member search.  cid = -1 at n_clusters or when nothing
// can be split.
__device__ void cl_choose_block(const ClEntry *tab, int n_clusters, ClWork *w) {
    __shared__ int s_best[kClThreads];
    const int n = w->n_cur;
    const int t = threadIdx.x;
    auto better = [&](int a, int b) {  // a strictly better than b
        if (a < 0) return false;
        if (b < 0) return true;
        const u128 Na = ((u128)tab[a].N[1] << 64) | tab[a].N[0];
        const u128 Nb = ((u128)tab[b].N[1] << 64) | tab[b].N[0];
        const u128 l = Na * (u128)tab[b].s.n, r = Nb * (u128)tab[a].s.n;
        return l > r || (l == r && a < b);
    };
    int best = -1;
    for (int i = t; n < n_clusters && i < n; i += blockDim.x) {
        if (tab[i].N[0] == 0 && tab[i].N[1] == 0) continue;
        if (better(i, best)) best = i;
    }
    s_best[t] = best;
    __syncthreads();
    for (int off = kClThreads / 2; off > 0; off >>= 1) {
        if (t < off && better(s_best[t + off], s_best[t])) s_best[t] = s_best[t + off];
        __syncthreads();
    }
    if (t == 0) {
        best = s_best[0];
        w->cid = best;
        w->nid = n;
        w->done = 0;
        w->have = 0;
        w->passes = 0;
        for (int s = 0; s < 2; ++s) w->st[s] = ClStats{};
        if (best >= 0)
            for (int i = 0; i < 3; ++i) {
                w->cen[i] = (double)(long long)tab[best].s.sx[i] / (double)tab[best].s.n;
                w->cen[3 + i] = 0.0;
            }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kClThreads) k_cl_choose(const ClEntry *tab, int n_clusters,
                                                          ClWork *w) {
    cl_choose_block(tab, n_clusters, w);
}

// the cluster's entry (one thread): exact sums and n * SSE
__device__ __forceinline__ void cl_set_entry(ClEntry &e, const ClStats &s) {
    e.s = s;
    const u128 N = cl_nsse(s);
    e.N[0] = (unsigned long long)N;
    e.N[1] = (unsigned long long)(N >> 64);
}

// One 2-means pass over the keys of the split cluster: sums of each side under
// the centres in w->cen; the last block then advances the passes (an empty side
// ends them, the previous pass standing; otherwise the pass is kept, and they
// end when the side means repeat the centres or after max_iter passes).
// first_entry: the pass that sums cluster 0 (every key) into table entry 0.
__global__ void __launch_bounds__(kClThreads) k_cl_assign(int64_t U, const int32_t *lab,
                                                          const int32_t *tx, const int32_t *wt,
                                                          ClWork *w, int max_iter,
                                                          unsigned int *counter, ClEntry *tab,
                                                          int first_entry) {
    __shared__ double cen[6];
    __shared__ ClAcc part[kClThreads / 32][2];
    const int32_t c = w->cid;
    if (c < 0 || w->done) return;  // nothing left to split, or the passes stopped
    if (threadIdx.x < 6) cen[threadIdx.x] = w->cen[threadIdx.x];
    __syncthreads();
    ClAcc a0, a1;
    a0.zero();
    a1.zero();
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U;
         u += (int64_t)gridDim.x * blockDim.x) {
        if (lab[u] != c) continue;
        const int32_t x0 = tx[u], x1 = tx[U + u], x2 = tx[2 * U + u];
        const unsigned long long wu = (unsigned long long)wt[u];
        if (cl_side(x0, x1, x2, cen))
            a1.add(wu, x0, x1, x2);
        else
            a0.add(wu, x0, x1, x2);
    }
    for (int off = 16; off > 0; off >>= 1) {
        a0.shfl_down(off);
        a1.shfl_down(off);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        part[wid][0] = a0;
        part[wid][1] = a1;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        ClAcc t = part[0][threadIdx.x];
        for (int i = 1; i < kClThreads / 32; ++i) t.merge(part[i][threadIdx.x]);
        t.flush(&w->st[threadIdx.x]);
    }
    if (!cl_last_block(counter) || threadIdx.x != 0) return;
    if (first_entry) {
        cl_set_entry(tab[0], w->st[0]);
        w->n_cur = 1;
        return;
    }
    ++w->passes;
    if (w->st[0].n == 0 || w->st[1].n == 0) {
        w->done = 1;
        return;
    }
    for (int i = 0; i < 6; ++i) w->kept_cen[i] = w->cen[i];
    w->kept[0] = w->st[0];
    w->kept[1] = w->st[1];
    w->have = 1;
    double m[6];
    bool same = true;
    for (int s = 0; s < 2; ++s)
        for (int i = 0; i < 3; ++i) {
            m[3 * s + i] = (double)(long long)w->st[s].sx[i] / (double)w->st[s].n;
            same &= m[3 * s + i] == w->cen[3 * s + i];
        }
    for (int i = 0; i < 6; ++i) w->cen[i] = m[i];
    for (int s = 0; s < 2; ++s) w->st[s] = ClStats{};
    if (same || w->passes >= max_iter) w->done = 1;
}

// exact squared distance of the features of key u to those of key a
__device__ __forceinline__ long long cl_dist_int(const int32_t *tx, int64_t U, int64_t u,
                                                 int32_t a) {
    long long d = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const long long e = (long long)tx[i * U + u] - tx[i * U + a];
        d += e * e;
    }
    return d;
}

// (distance, key) pairs: larger distance first, then the smaller key id
__device__ __forceinline__ bool cl_far_better(unsigned long long d, int32_t u,
                                              unsigned long long bd, int32_t bu) {
    return d > bd || (d == bd && u < bu);
}

// Farthest member of the split cluster (ties to the smallest key id) from
// its mean (stage 0, FP64 distances; distances are >= 0, so their bit
// patterns order like the values) or from the member found before (stage 1,
// exact integer distances).  Per-block results go to far_d / far_u; the last
// block combines them, and after stage 1 seeds the first 2-means pass with
// the two members.
__global__ void __launch_bounds__(kClThreads) k_cl_far(int64_t U, const int32_t *lab,
                                                       const int32_t *tx, ClWork *w, int stage,
                                                       unsigned long long *far_d,
                                                       int32_t *far_u, unsigned int *counter) {
    __shared__ unsigned long long sd[kClThreads];
    __shared__ int32_t su[kClThreads];
    const int32_t c = w->cid;
    if (c < 0) return;
    const int32_t a = stage ? w->umin[0] : 0;
    const double cen[3] = {w->cen[0], w->cen[1], w->cen[2]};
    unsigned long long bd = 0;
    int32_t bu = 0x7fffffff;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U;
         u += (int64_t)gridDim.x * blockDim.x) {
        if (lab[u] != c) continue;
        const unsigned long long d =
            stage ? (unsigned long long)cl_dist_int(tx, U, u, a)
                  : (unsigned long long)__double_as_longlong(
                        cl_dist(tx[u], tx[U + u], tx[2 * U + u], cen));
        if (cl_far_better(d, (int32_t)u, bd, bu)) {
            bd = d;
            bu = (int32_t)u;
        }
    }
    const int t = threadIdx.x;
    sd[t] = bd;
    su[t] = bu;
    __syncthreads();
    for (int off = kClThreads / 2; off > 0; off >>= 1) {
        if (t < off && cl_far_better(sd[t + off], su[t + off], sd[t], su[t])) {
            sd[t] = sd[t + off];
            su[t] = su[t + off];
        }
        __syncthreads();
    }
    if (t == 0) {
        far_d[blockIdx.x] = sd[0];
        far_u[blockIdx.x] = su[0];
    }
    if (!cl_last_block(counter)) return;
    bd = 0;
    bu = 0x7fffffff;
    for (int b = t; b < (int)gridDim.x; b += blockDim.x) {
        const unsigned long long d = far_d[b];
        const int32_t u = far_u[b];
        if (cl_far_better(d, u, bd, bu)) {
            bd = d;
            bu = u;
        }
    }
    sd[t] = bd;
    su[t] = bu;
    __syncthreads();
    for (int off = kClThreads / 2; off > 0; off >>= 1) {
        if (t < off && cl_far_better(sd[t + off], su[t + off], sd[t], su[t])) {
            sd[t] = sd[t + off];
            su[t] = su[t + off];
        }
        __syncthreads();
    }
    if (t == 0) {
        w->umin[stage] = su[0];
        if (stage == 1) {  // centres of the first 2-means pass
            const int32_t m0 = w->umin[0], m1 = su[0];
            for (int i = 0; i < 3; ++i) {
                w->cen[i] = (double)tx[i * U + m0];
                w->cen[3 + i] = (double)tx[i * U + m1];
            }
        }
    }
}

// Members of the split cluster on side 1 under the kept centres move to id
// nid; the last block records both sides in the table and chooses the next
// split.
__global__ void __launch_bounds__(kClThreads) k_cl_label(int64_t U, int32_t *lab,
                                                         const int32_t *tx, ClWork *w,
                                                         ClEntry *tab, int n_clusters,
                                                         unsigned int *counter) {
    __shared__ double cen[6];
    const int32_t c = w->cid, id_new = w->nid;
    if (c < 0 || !w->have) return;
    if (threadIdx.x < 6) cen[threadIdx.x] = w->kept_cen[threadIdx.x];
    __syncthreads();
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U;
         u += (int64_t)gridDim.x * blockDim.x) {
        if (lab[u] != c) continue;
        if (cl_side(tx[u], tx[U + u], tx[2 * U + u], cen)) lab[u] = id_new;
    }
    if (!cl_last_block(counter)) return;
    if (threadIdx.x == 0) {
        cl_set_entry(tab[c], w->kept[0]);
        cl_set_entry(tab[id_new], w->kept[1]);
        w->n_cur = id_new + 1;
    }
    __syncthreads();
    cl_choose_block(tab, n_clusters, w);
}

// M0 refit: M0' = sum_e I_e f_e(c) / sum_e f_e(c)^2 with I_e = M0 f_e(T1, T2)
// and f_e(T1, T2) = (1 - exp(-TR / T1)) exp(-TE_e / T2), i.e. M0' = M0 r with
// r = sum_e f_e(T1, T2) f_e(c) / sum_e f_e(c)^2.  r depends on the exact T1, T2
// and the cluster only, so it is formed once per distinct key (FP64, echoes
// summed in order) and the isochromat pass is a gather.
struct EchoModel {
    int n;
    double tr;
    double te[MRSIM_MAX_ECHOES];
};

__device__ __forceinline__ double t2w(double tr, double te, double T1, double T2) {
    return __dmul_rn(__dsub_rn(1.0, exp(__ddiv_rn(-tr, T1))), exp(__ddiv_rn(-te, T2)));
}

// per cluster: f_e(c) for every echo and sum_e f_e(c)^2
__global__ void k_cl_model(int n, const float *cT1, const float *cT2, EchoModel em, double *fc,
                           double *den) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int e = 0; e < em.n; ++e) {
            const double f = t2w(em.tr, em.te[e], (double)cT1[c], (double)cT2[c]);
            fc[(int64_t)c * MRSIM_MAX_ECHOES + e] = f;
            d = __dadd_rn(d, __dmul_rn(f, f));
        }
        den[c] = d;
    }
}

// per distinct key: the refit factor r (1 where there is no echo or den = 0)
__global__ void k_cl_ratio(int64_t U, const float *tf, const int32_t *lab, const double *fc,
                           const double *den, EchoModel em, double *ratio) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = lab[u];
        const double T1 = (double)tf[u], T2 = (double)tf[U + u], d = em.n ? den[c] : 0.0;
        double r = 1.0;
        if (d > 0.0) {
            double num = 0.0;
            for (int e = 0; e < em.n; ++e)
                num = __dadd_rn(num, __dmul_rn(t2w(em.tr, em.te[e], T1, T2),
                                               fc[(int64_t)c * MRSIM_MAX_ECHOES + e]));
            r = __ddiv_rn(num, d);
        }
        ratio[u] = r;
    }
}

// every isochromat takes its cluster's centre values and M0 r
__global__ void k_cl_apply(int64_t K, const int32_t *uid, const int32_t *lab, const float *cT1,
                           const float *cT2, const float *cdB0, const double *ratio,
                           const float *M0, float *oT1, float *oT2, float *odB0, float *oM0,
                           int32_t *olab) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = uid[k];
        const int32_t c = lab[u];
        olab[k] = c;
        oT1[k] = cT1[c];
        oT2[k] = cT2[c];
        odB0[k] = cdB0[c];
        oM0[k] = (float)__dmul_rn((double)M0[k], ratio[u]);
    }
}

int grid(const mrsim_ctx *c, int64_t n) {
    const int64_t b = (n + kClThreads - 1) / kClThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)c->sm_count * 8));
}

// Host copy of one cluster's exact sums.
struct Cluster {
    uint64_t n = 0;
    int64_t sx[3] = {0, 0, 0};
    u128 sq[3] = {0, 0, 0};
    double mu[3] = {0, 0, 0};  // FP64 mean, feature units
    u128 N = 0;                // n * SSE = sum_i (n sum w x_i^2 - (sum w x_i)^2)

    void set(const ClStats &s) {
        n = s.n;
        N = 0;
        for (int i = 0; i < 3; ++i) {
            sx[i] = (int64_t)s.sx[i];
            sq[i] = ((u128)s.sq[i][1] << 64) | s.sq[i][0];
            mu[i] = n ? (double)sx[i] / (double)n : 0.0;
            const u128 a = (sx[i] < 0) ? (u128)(-sx[i]) : (u128)sx[i];
            N += (u128)n * sq[i] - a * a;
        }
    }
};


}  // namespace

void cluster_phantom(mrsim_ctx *c, const mrsim_phantom_t *ph, int n_clusters,
                     const double scale[3], int max_iter, int n_echo, const double *te, double tr,
                     mrsim_phantom_t *out, DBuf &labels, std::vector<double> &centres) {
    const int64_t K = ph->K;
    if (K > kMaxClusterK) fail(MRSIM_EINVAL, "clustering takes at most 2^28 isochromats");
    // features
    DBuf xq = dalloc(3 * K * sizeof(int32_t));
    int *err = c->dev_err.as<int>();
    MRSIM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), c->stream));
    {
        KScope ks(c, "cluster_quantize");
        // integer scales below 2^24 (the default grid): the same features in
        // integer arithmetic; other scales: FP64 products
        bool int_scale = true;
        for (int i = 0; i < 3; ++i)
            int_scale &= scale[i] >= 1.0 && scale[i] < 16777216.0 && scale[i] == std::floor(scale[i]);
        if (int_scale)
            k_cl_quant_int<<<grid(c, K), kClThreads, 0, c->stream>>>(
                K, ph->T1.as<float>(), ph->T2.as<float>(), ph->dB0.as<float>(),
                (long long)scale[0], (long long)scale[1], (long long)scale[2], xq.as<int32_t>(),
                err);
        else
            k_cl_quant<<<grid(c, K), kClThreads, 0, c->stream>>>(
                K, ph->T1.as<float>(), ph->T2.as<float>(), ph->dB0.as<float>(), scale[0],
                scale[1], scale[2], xq.as<int32_t>(), err);
    }
    int h_err = 0;
    MRSIM_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    sync(c);
    if (h_err)
        fail(MRSIM_EINVAL, "a T1, T2 or dB0 value is not finite, outside +-2^20 clustering "
                           "steps, or (T1, T2) below one step");
    // distinct keys with their weights
    DBuf uid = dalloc(K * sizeof(int32_t));
    DBuf tx, tf, wt;
    const int64_t U = distinct_features(c, K, xq.as<int32_t>(), ph->T1.as<float>(),
                                        ph->T2.as<float>(), uid.as<int32_t>(), tx, tf, wt);
    DBuf lab = dalloc(U * sizeof(int32_t));
    MRSIM_CUDA(cudaMemsetAsync(lab.p, 0, U * sizeof(int32_t), c->stream));
    DBuf work = dalloc(sizeof(ClWork));
    ClWork *w = work.as<ClWork>();
    DBuf table = dalloc((size_t)n_clusters * sizeof(ClEntry));
    ClEntry *tab = table.as<ClEntry>();
    const int32_t *ptx = tx.as<int32_t>(), *pwt = wt.as<int32_t>();
    int32_t *plab = lab.as<int32_t>();
    // passes over the distinct keys: two CTAs per SM (the last-block steps
    // combine one partial per CTA)
    const int gU = (int)std::max<int64_t>(
        1, std::min<int64_t>((U + kClThreads - 1) / kClThreads, (int64_t)c->sm_count * 2));
    DBuf far_d = dalloc(gU * sizeof(unsigned long long)), far_u = dalloc(gU * sizeof(int32_t));
    DBuf counter = dalloc(sizeof(unsigned int));
    MRSIM_CUDA(cudaMemsetAsync(counter.p, 0, sizeof(unsigned int), c->stream));
    unsigned int *cnt = counter.as<unsigned int>();
    // cluster 0 holds every key: one pass with equal centres (every key on
    // side 0, cluster id 0) gives its entry; then the first split is chosen
    {
        ClWork w0{};
        w0.cid = 0;
        upload(c, w, &w0, sizeof(ClWork));
        KScope ks(c, "cluster_assign");
        k_cl_assign<<<gU, kClThreads, 0, c->stream>>>(U, plab, ptx, pwt, w, max_iter, cnt, tab, 1);
        k_cl_choose<<<1, kClThreads, 0, c->stream>>>(tab, n_clusters, w);
    }
    // Splits, decided on the device: the farthest-member searches, 2-means
    // passes queued four at a time (they return at once after the passes
    // stopped), the relabelling, which also records both sides and chooses the
    // next split.  The host reads a few words back once per split.
    constexpr int kPassBatch = 4;
    struct Status { int32_t cid, nid, done, have, passes; } st{};
    for (int split = 1; split < n_clusters; ++split) {
        {
            KScope ks(c, "cluster_farthest");
            k_cl_far<<<gU, kClThreads, 0, c->stream>>>(U, plab, ptx, w, 0,
                                                       far_d.as<unsigned long long>(),
                                                       far_u.as<int32_t>(), cnt);
            k_cl_far<<<gU, kClThreads, 0, c->stream>>>(U, plab, ptx, w, 1,
                                                       far_d.as<unsigned long long>(),
                                                       far_u.as<int32_t>(), cnt);
        }
        for (;;) {
            {
                KScope ks(c, "cluster_assign");
                for (int p = 0; p < kPassBatch; ++p)
                    k_cl_assign<<<gU, kClThreads, 0, c->stream>>>(U, plab, ptx, pwt, w, max_iter,
                                                                  cnt, tab, 0);
            }
            MRSIM_CUDA(cudaMemcpyAsync(&st, &w->cid, sizeof(Status), cudaMemcpyDeviceToHost,
                                       c->stream));
            sync(c);
            if (st.cid < 0 || st.done) break;
        }
        if (st.cid < 0) break;  // every cluster is one distinct value
        if (!st.have) fail(MRSIM_ECUDA, "clustering: the first 2-means pass left a side empty");
        KScope ks(c, "cluster_label");
        k_cl_label<<<gU, kClThreads, 0, c->stream>>>(U, plab, ptx, w, tab, n_clusters, cnt);
    }
    // the clusters' exact sums, back on the host for the centre values
    int32_t n_made = 0;
    MRSIM_CUDA(cudaMemcpyAsync(&n_made, &w->n_cur, sizeof(int32_t), cudaMemcpyDeviceToHost,
                               c->stream));
    sync(c);
    std::vector<ClEntry> hs(std::max(n_made, 1));
    MRSIM_CUDA(cudaMemcpyAsync(hs.data(), tab, n_made * sizeof(ClEntry), cudaMemcpyDeviceToHost,
                               c->stream));
    sync(c);
    std::vector<Cluster> cl(n_made);
    for (int i = 0; i < n_made; ++i) cl[i].set(hs[i].s);
    const int n = (int)cl.size();
    // centre values in phantom units, as stored (float32)
    centres.assign(3 * (size_t)n, 0.0);
    std::vector<float> cf(3 * (size_t)n);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            centres[3 * i + a] = cl[i].mu[a] / scale[a];
            cf[a * n + i] = (float)centres[3 * i + a];
        }
    DBuf dcf = dalloc(cf.size() * sizeof(float));
    upload(c, dcf.p, cf.data(), cf.size() * sizeof(float));
    // the M0 refit factor of every distinct key
    EchoModel em{};
    em.n = n_echo;
    em.tr = tr;
    for (int e = 0; e < n_echo; ++e) em.te[e] = te[e];
    DBuf fc = dalloc((size_t)n * MRSIM_MAX_ECHOES * sizeof(double));
    DBuf den = dalloc((size_t)n * sizeof(double));
    DBuf ratio = dalloc(U * sizeof(double));
    {
        KScope ks(c, "cluster_refit");
        const float *pc = dcf.as<float>();
        k_cl_model<<<(n + kClThreads - 1) / kClThreads, kClThreads, 0, c->stream>>>(
            n, pc, pc + n, em, fc.as<double>(), den.as<double>());
        k_cl_ratio<<<gU, kClThreads, 0, c->stream>>>(U, tf.as<float>(), plab, fc.as<double>(),
                                                     den.as<double>(), em, ratio.as<double>());
    }
    // the new phantom
    auto copy = [&](DBuf &dst, const DBuf &src, size_t bytes) {
        dst = dalloc(bytes);
        MRSIM_CUDA(cudaMemcpyAsync(dst.p, src.p, bytes, cudaMemcpyDeviceToDevice, c->stream));
    };
    const size_t fb = K * sizeof(float);
    out->K = K;
    copy(out->x, ph->x, fb);
    copy(out->y, ph->y, fb);
    copy(out->z, ph->z, fb);
    out->has_b1 = ph->has_b1;
    if (ph->has_b1) copy(out->b1, ph->b1, fb);
    out->has_M_init = ph->has_M_init;
    if (ph->has_M_init) copy(out->M_init, ph->M_init, 3 * fb);
    out->n_coils = ph->n_coils;
    if (ph->n_coils) copy(out->coils, ph->coils, 2 * (size_t)ph->n_coils * fb);
    out->T1 = dalloc(fb);
    out->T2 = dalloc(fb);
    out->dB0 = dalloc(fb);
    out->M0 = dalloc(fb);
    labels = dalloc(K * sizeof(int32_t));
    {
        KScope ks(c, "cluster_apply");
        const float *pc = dcf.as<float>();
        k_cl_apply<<<grid(c, K), kClThreads, 0, c->stream>>>(
            K, uid.as<int32_t>(), plab, pc, pc + n, pc + 2 * n, ratio.as<double>(),
            ph->M0.as<float>(), out->T1.as<float>(), out->T2.as<float>(), out->dB0.as<float>(),
            out->M0.as<float>(), labels.as<int32_t>());
    }
    sync(c);
}

}  // namespace mrsim
