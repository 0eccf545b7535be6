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
#include <queue>
#include <vector>

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

// One node of the split tree: the exact sums of its keys and where its keys
// lie (a contiguous range of one of the two order buffers).
struct ClNode {
    ClStats s;
    int32_t buf, start, count, pad;
};

// One split computed in a round ("slot"): the node, its two children and the
// state of the split's steps.  The host fills the first group of fields; the
// kernels the rest.
struct ClSlot {
    double cen[6];                // centres of side 0 / side 1; cen[0..2] = the mean first
    int32_t node, child0, child1;  // node ids in the tree table
    int32_t buf, start, count;    // the node's keys
    int32_t tile0, n_tiles;       // its tiles in the round's tile list
    double kept_cen[6];           // centres of the last pass with both sides filled
    ClStats st[2];                // sums of the pass in progress
    ClStats kept[2];              // ... and of the kept pass
    int32_t umin[2];              // farthest-member searches: the key found
    int32_t done, have, passes;   // 2-means stopped; a pass was kept; passes run
    unsigned int counter;         // tiles finished in the step in progress
    unsigned int front, back;     // partition: keys placed on side 0 / side 1
};

// Completion per slot: every block adds one to the slot's counter after its
// tile's results are visible (fence first); the block that brings it to
// n_tiles finishes the step for the slot alone and resets the counter.  No
// block waits for another.
__device__ __forceinline__ bool cl_last_tile(ClSlot *w) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int prev = atomicAdd(&w->counter, 1u);
        last = prev == (unsigned int)w->n_tiles - 1u;
        if (last) w->counter = 0u;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// sums written by other blocks' atomics, read from L2
__device__ __forceinline__ ClStats cl_ld_l2(const ClStats *p) {
    ClStats s;
    s.n = __ldcg(&p->n);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        s.sx[i] = __ldcg(&p->sx[i]);
        s.sq[i][0] = __ldcg(&p->sq[i][0]);
        s.sq[i][1] = __ldcg(&p->sq[i][1]);
    }
    return s;
}

// the block's sums of one or two sides, added into dst[0..1] (exact)
__device__ __forceinline__ void cl_block_flush(ClAcc a0, ClAcc a1, ClStats *dst, int sides) {
    __shared__ ClAcc part[kClThreads / 32][2];
    for (int off = 16; off > 0; off >>= 1) {
        a0.shfl_down(off);
        if (sides > 1) a1.shfl_down(off);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        part[wid][0] = a0;
        part[wid][1] = a1;
    }
    __syncthreads();
    if (threadIdx.x < sides) {
        ClAcc t = part[0][threadIdx.x];
        for (int i = 1; i < kClThreads / 32; ++i) t.merge(part[i][threadIdx.x]);
        t.flush(&dst[threadIdx.x]);
    }
}

// Sums of every key: the root node of the tree (its sums zeroed before).
__global__ void __launch_bounds__(kClThreads) k_cl_root(int64_t U, const int32_t *tx,
                                                        const int32_t *wt, int32_t *ord,
                                                        ClNode *root) {
    ClAcc a, none;
    a.zero();
    none.zero();
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U;
         u += (int64_t)gridDim.x * blockDim.x) {
        a.add((unsigned long long)wt[u], tx[u], tx[U + u], tx[2 * U + u]);
        ord[u] = (int32_t)u;
    }
    cl_block_flush(a, none, &root->s, 1);
}

// the tile's keys: [lo, hi) of the slot's range in its order buffer
struct ClTile {
    const int32_t *keys;
    int64_t lo, hi;
};

__device__ __forceinline__ ClTile cl_tile(const ClSlot *w, const int32_t *ord, int64_t U, int t,
                                          int tile_keys) {
    ClTile r;
    r.keys = ord + (int64_t)w->buf * U + w->start;
    r.lo = (int64_t)(t - w->tile0) * tile_keys;
    const int64_t end = r.lo + tile_keys;
    r.hi = end < w->count ? end : (int64_t)w->count;
    return r;
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

// block-wide best (distance, key) pair of the values held by each thread;
// the result in sd[0], su[0]
__device__ __forceinline__ void cl_far_reduce(unsigned long long *sd, int32_t *su,
                                              unsigned long long bd, int32_t bu) {
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
}

// Farthest member of each slot's node (ties to the smallest key id) from the
// node's mean (stage 0, FP64 distances; distances are >= 0, so their bit
// patterns order like the values) or from the member found before (stage 1,
// exact integer distances).  Each tile's best pair goes to far_d / far_u; the
// slot's last tile combines its tiles and, after stage 1, seeds the first
// 2-means pass with the two members.
__global__ void __launch_bounds__(kClThreads) k_cl_far(int64_t U, const int32_t *ord,
                                                       const int32_t *tx, ClSlot *slots,
                                                       const int32_t *tile_slot, int n_tiles,
                                                       int tile_keys, int stage,
                                                       unsigned long long *far_d,
                                                       int32_t *far_u) {
    __shared__ unsigned long long sd[kClThreads];
    __shared__ int32_t su[kClThreads];
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        ClSlot *w = slots + tile_slot[t];
        const ClTile r = cl_tile(w, ord, U, t, tile_keys);
        const int32_t a = stage ? w->umin[0] : 0;
        const double cen[3] = {w->cen[0], w->cen[1], w->cen[2]};
        unsigned long long bd = 0;
        int32_t bu = 0x7fffffff;
        for (int64_t i = r.lo + threadIdx.x; i < r.hi; i += blockDim.x) {
            const int64_t u = r.keys[i];
            const unsigned long long d =
                stage ? (unsigned long long)cl_dist_int(tx, U, u, a)
                      : (unsigned long long)__double_as_longlong(
                            cl_dist(tx[u], tx[U + u], tx[2 * U + u], cen));
            if (cl_far_better(d, (int32_t)u, bd, bu)) {
                bd = d;
                bu = (int32_t)u;
            }
        }
        cl_far_reduce(sd, su, bd, bu);
        if (threadIdx.x == 0) {
            far_d[t] = sd[0];
            far_u[t] = su[0];
        }
        if (cl_last_tile(w)) {
            bd = 0;
            bu = 0x7fffffff;
            for (int j = w->tile0 + threadIdx.x; j < w->tile0 + w->n_tiles; j += blockDim.x) {
                const unsigned long long d = __ldcg(&far_d[j]);
                const int32_t u = __ldcg(&far_u[j]);
                if (cl_far_better(d, u, bd, bu)) {
                    bd = d;
                    bu = u;
                }
            }
            cl_far_reduce(sd, su, bd, bu);
            if (threadIdx.x == 0) {
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
        __syncthreads();
    }
}

// One 2-means pass over the keys of every slot still running: sums of each
// side under the slot's centres; the slot's last tile then advances its passes
// (an empty side ends them, the previous pass standing; otherwise the pass is
// kept, and they end when the side means repeat the centres or after max_iter
// passes).  n_running counts the slots whose passes have not ended.
__global__ void __launch_bounds__(kClThreads) k_cl_pass(int64_t U, const int32_t *ord,
                                                        const int32_t *tx, const int32_t *wt,
                                                        ClSlot *slots, const int32_t *tile_slot,
                                                        int n_tiles, int tile_keys, int max_iter,
                                                        int *n_running) {
    __shared__ double cen[6];
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        ClSlot *w = slots + tile_slot[t];
        if (w->done) continue;  // the same value for every thread of the block
        if (threadIdx.x < 6) cen[threadIdx.x] = w->cen[threadIdx.x];
        __syncthreads();
        const ClTile r = cl_tile(w, ord, U, t, tile_keys);
        ClAcc a0, a1;
        a0.zero();
        a1.zero();
        for (int64_t i = r.lo + threadIdx.x; i < r.hi; i += blockDim.x) {
            const int64_t u = r.keys[i];
            const int32_t x0 = tx[u], x1 = tx[U + u], x2 = tx[2 * U + u];
            const unsigned long long wu = (unsigned long long)wt[u];
            if (cl_side(x0, x1, x2, cen))
                a1.add(wu, x0, x1, x2);
            else
                a0.add(wu, x0, x1, x2);
        }
        cl_block_flush(a0, a1, w->st, 2);
        const bool last = cl_last_tile(w);
        if (last && threadIdx.x == 0) {
            ++w->passes;
            const ClStats st[2] = {cl_ld_l2(&w->st[0]), cl_ld_l2(&w->st[1])};
            bool stop;
            if (st[0].n == 0 || st[1].n == 0) {
                stop = true;
            } else {
                for (int i = 0; i < 6; ++i) w->kept_cen[i] = w->cen[i];
                w->kept[0] = st[0];
                w->kept[1] = st[1];
                w->have = 1;
                double m[6];
                bool same = true;
                for (int s = 0; s < 2; ++s)
                    for (int i = 0; i < 3; ++i) {
                        m[3 * s + i] = (double)(long long)st[s].sx[i] / (double)st[s].n;
                        same &= m[3 * s + i] == w->cen[3 * s + i];
                    }
                for (int i = 0; i < 6; ++i) w->cen[i] = m[i];
                stop = same || w->passes >= max_iter;
            }
            for (int s = 0; s < 2; ++s) w->st[s] = ClStats{};
            if (stop) {
                w->done = 1;
                atomicSub(n_running, 1);
            }
        }
        __syncthreads();
    }
}

// Each slot's keys on side 1 under the kept centres form child 1, the rest
// child 0: the node's range is partitioned into the other order buffer, side 0
// from the front and side 1 from the back (the order inside a range is free:
// ties go by key id and sums are exact).  The slot's last tile records both
// children in the tree table.
__global__ void __launch_bounds__(kClThreads) k_cl_part(int64_t U, int32_t *ord,
                                                        const int32_t *tx, ClSlot *slots,
                                                        const int32_t *tile_slot, int n_tiles,
                                                        int tile_keys, ClNode *nodes, int *err) {
    __shared__ double cen[6];
    const int lane = threadIdx.x & 31;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        ClSlot *w = slots + tile_slot[t];
        if (threadIdx.x < 6) cen[threadIdx.x] = w->kept_cen[threadIdx.x];
        __syncthreads();
        const ClTile r = cl_tile(w, ord, U, t, tile_keys);
        int32_t *dst = ord + (int64_t)(1 - w->buf) * U + w->start;
        const int32_t n = w->count;
        // whole warps take part in the ballots: tiles are whole blocks long
        for (int64_t i = r.lo + threadIdx.x; i < r.lo + tile_keys; i += blockDim.x) {
            const bool live = i < r.hi;
            const int64_t u = live ? r.keys[i] : 0;
            const bool one = live && cl_side(tx[u], tx[U + u], tx[2 * U + u], cen);
            const unsigned m1 = __ballot_sync(0xffffffffu, one);
            const unsigned m0 = __ballot_sync(0xffffffffu, live && !one);
            if (!(m0 | m1)) continue;  // the same for the whole warp
            unsigned b0 = 0, b1 = 0;
            if (lane == 0) {
                if (m0) b0 = atomicAdd(&w->front, (unsigned)__popc(m0));
                if (m1) b1 = atomicAdd(&w->back, (unsigned)__popc(m1));
            }
            b0 = __shfl_sync(0xffffffffu, b0, 0);
            b1 = __shfl_sync(0xffffffffu, b1, 0);
            const unsigned below = (1u << lane) - 1u;
            if (live && !one) dst[b0 + __popc(m0 & below)] = (int32_t)u;
            if (one) dst[n - 1 - (b1 + __popc(m1 & below))] = (int32_t)u;
        }
        if (cl_last_tile(w) && threadIdx.x == 0) {
            const unsigned int front = __ldcg(&w->front), back = __ldcg(&w->back);
            if (!w->have || (int64_t)front + back != n) atomicOr(err, 2);
            const int32_t nf = (int32_t)front;
            ClNode c0, c1;
            c0.s = w->kept[0];
            c0.buf = 1 - w->buf;
            c0.start = w->start;
            c0.count = nf;
            c0.pad = 0;
            c1.s = w->kept[1];
            c1.buf = 1 - w->buf;
            c1.start = w->start + nf;
            c1.count = n - nf;
            c1.pad = 0;
            nodes[w->child0] = c0;
            nodes[w->child1] = c1;
        }
        __syncthreads();
    }
}

// The final clusters: every key of cluster id's node takes label id.  leaf[j]
// = (buf, start, count, id), tiles as in the split kernels (tile0 in leaf_t0).
__global__ void __launch_bounds__(kClThreads) k_cl_leaf_label(int64_t U, const int32_t *ord,
                                                              const int4 *leaf,
                                                              const int32_t *leaf_t0,
                                                              const int32_t *tile_leaf,
                                                              int n_tiles, int tile_keys,
                                                              int32_t *lab) {
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int j = tile_leaf[t];
        const int4 l = leaf[j];
        const int32_t *keys = ord + (int64_t)l.x * U + l.y;
        const int64_t lo = (int64_t)(t - leaf_t0[j]) * tile_keys;
        const int64_t end = lo + tile_keys;
        const int64_t hi = end < l.z ? end : (int64_t)l.z;
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) lab[keys[i]] = l.w;
    }
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


// n * SSE of exact sums, on the host
u128 host_nsse(const ClStats &s) {
    u128 N = 0;
    for (int i = 0; i < 3; ++i) {
        const u128 sq = ((u128)s.sq[i][1] << 64) | s.sq[i][0];
        const int64_t x = (int64_t)s.sx[i];
        const u128 a = x < 0 ? (u128)(-x) : (u128)x;
        N += (u128)s.n * sq - a * a;
    }
    return N;
}

// Host copy of one node of the split tree; c0 / c1 are its children once its
// split is computed (-1 before).
struct TreeNode {
    ClStats s{};
    u128 N = 0;
    int32_t buf = 0, start = 0, count = 0;
    int c0 = -1, c1 = -1;

    void set(const ClNode &e) {
        s = e.s;
        N = host_nsse(s);
        buf = e.buf;
        start = e.start;
        count = e.count;
    }
};

// A leaf in the greedy replay: score N / n, id, tree node.
struct Pick {
    u128 N;
    uint64_t n;
    int id, node;
};

// heap order: b comes out before a when its SSE is larger (exact rationals),
// or equal with the smaller id
struct PickAfter {
    bool operator()(const Pick &a, const Pick &b) const {
        const u128 l = b.N * (u128)a.n, r = a.N * (u128)b.n;
        return l > r || (l == r && b.id < a.id);
    }
};

// The greedy choice replayed on the tree: split the leaf with the largest SSE
// (ties to the smaller id; leaves of one distinct value are never split), side
// 0 keeping the id and side 1 taking the next, until n_clusters.  Returns true
// when every pick had its split computed: leaf_node[id] is then the node of
// every cluster.  Otherwise front lists the picks without a split, in pick
// order (the first is the one the greedy needs next; the later ones are
// counted as splits without their sides and may not be needed).
bool greedy_replay(const std::vector<TreeNode> &tree, int n_clusters,
                   std::vector<int> &leaf_node, std::vector<int> &front) {
    std::priority_queue<Pick, std::vector<Pick>, PickAfter> q;
    auto push = [&](int node, int id) {
        if (tree[node].N != 0) q.push(Pick{tree[node].N, tree[node].s.n, id, node});
    };
    leaf_node.assign(1, 0);
    front.clear();
    push(0, 0);
    bool exact = true;
    for (int n_cur = 1; n_cur < n_clusters && !q.empty(); ++n_cur) {
        const Pick p = q.top();
        q.pop();
        const TreeNode &h = tree[p.node];
        if (h.c0 < 0) {
            front.push_back(p.node);
            exact = false;
            continue;
        }
        if (exact) {
            leaf_node[p.id] = h.c0;
            leaf_node.push_back(h.c1);
        }
        push(h.c0, p.id);
        push(h.c1, n_cur);
    }
    return exact;
}


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
    // ---- the split tree, grown in rounds ----
    // Every split of a cluster depends on its keys alone, not on when it is
    // made, and a split's sides never have a larger SSE than the cluster (the
    // chosen SSEs do not increase).  So the splits the greedy order will make
    // can be computed many at a time: each round, the host replays the greedy
    // choice (largest SSE, ties to the smaller id) on the splits computed so
    // far; the replay's picks that are not computed yet, the first of which
    // the greedy certainly needs, are computed together in one round of
    // kernels over all their keys.  When the replay reaches n_clusters (or
    // runs out of clusters with more than one distinct value) on computed
    // splits alone, it is the sequential result, ids included.
    const int cap = 6 * n_clusters + 8;  // tree nodes (bound below)
    DBuf dnodes = dalloc((size_t)cap * sizeof(ClNode));
    ClNode *pn = dnodes.as<ClNode>();
    DBuf order = dalloc(2 * U * sizeof(int32_t));
    int32_t *pord = order.as<int32_t>();
    const int32_t *ptx = tx.as<int32_t>(), *pwt = wt.as<int32_t>();
    std::vector<TreeNode> tree(1);
    {
        MRSIM_CUDA(cudaMemsetAsync(pn, 0, sizeof(ClNode), c->stream));
        {
            KScope ks(c, "cluster_root");
            k_cl_root<<<grid(c, U), kClThreads, 0, c->stream>>>(U, ptx, pwt, pord, pn);
        }
        ClNode r;
        MRSIM_CUDA(cudaMemcpyAsync(&r, pn, sizeof(ClNode), cudaMemcpyDeviceToHost, c->stream));
        sync(c);
        r.buf = 0;
        r.start = 0;
        r.count = (int32_t)U;
        tree[0].set(r);
        upload(c, pn, &r, sizeof(ClNode));
    }
    // per-round work areas: a slot per split, tiles of at least 256 keys
    const int64_t tile_cap = U / kClThreads + n_clusters + 1;
    DBuf dslots = dalloc((size_t)n_clusters * sizeof(ClSlot));
    DBuf dtiles = dalloc(tile_cap * sizeof(int32_t));
    DBuf far_d = dalloc(tile_cap * sizeof(unsigned long long));
    DBuf far_u = dalloc(tile_cap * sizeof(int32_t));
    DBuf drun = dalloc(sizeof(int));
    ClSlot *psl = dslots.as<ClSlot>();
    int32_t *ptl = dtiles.as<int32_t>();
    int *prun = drun.as<int>();
    std::vector<int> leaf_node, front;
    std::vector<ClSlot> hs;
    std::vector<int32_t> tiles;
    std::vector<ClNode> made;
    constexpr int kPassBatch = 4;
    while (!greedy_replay(tree, n_clusters, leaf_node, front)) {
        // picks after the first only while the table keeps room for the splits
        // the greedy certainly needs (at most n_clusters - 1, two nodes each):
        // the tree never holds more than 4 n + 2 (n - 1) + 1 nodes
        size_t m = 1;
        while (m < front.size() && tree.size() + 2 * (m + 1) <= (size_t)4 * n_clusters) ++m;
        int64_t total = 0;
        for (size_t j = 0; j < m; ++j) total += tree[front[j]].count;
        const int64_t per = (total + 2 * c->sm_count - 1) / (2 * c->sm_count);
        const int tile_keys = (int)std::min<int64_t>(
            16384, std::max<int64_t>(kClThreads, (per + kClThreads - 1) / kClThreads * kClThreads));
        hs.assign(m, ClSlot{});
        tiles.clear();
        for (size_t j = 0; j < m; ++j) {
            TreeNode &h = tree[front[j]];
            ClSlot &s = hs[j];
            for (int i = 0; i < 3; ++i)
                s.cen[i] = (double)(int64_t)h.s.sx[i] / (double)h.s.n;
            s.node = front[j];
            s.child0 = (int32_t)tree.size();
            s.child1 = s.child0 + 1;
            h.c0 = s.child0;
            h.c1 = s.child1;
            tree.emplace_back();
            tree.emplace_back();
            s.buf = h.buf;
            s.start = h.start;
            s.count = h.count;
            s.tile0 = (int32_t)tiles.size();
            s.n_tiles = (int32_t)((h.count + tile_keys - 1) / tile_keys);
            tiles.insert(tiles.end(), s.n_tiles, (int32_t)j);
        }
        const int nt = (int)tiles.size();
        const int g = std::min(nt, c->sm_count * 4);
        const int n_run = (int)m;
        upload(c, psl, hs.data(), m * sizeof(ClSlot));
        upload(c, ptl, tiles.data(), nt * sizeof(int32_t));
        upload(c, prun, &n_run, sizeof(int));
        {
            KScope ks(c, "cluster_farthest");
            for (int stage = 0; stage < 2; ++stage)
                k_cl_far<<<g, kClThreads, 0, c->stream>>>(U, pord, ptx, psl, ptl, nt, tile_keys,
                                                          stage, far_d.as<unsigned long long>(),
                                                          far_u.as<int32_t>());
        }
        for (int batch = 0;; ++batch) {
            if (batch * kPassBatch > max_iter + kPassBatch)
                fail(MRSIM_ECUDA, "clustering: 2-means passes did not stop");
            {
                KScope ks(c, "cluster_pass");
                for (int p = 0; p < kPassBatch; ++p)
                    k_cl_pass<<<g, kClThreads, 0, c->stream>>>(U, pord, ptx, pwt, psl, ptl, nt,
                                                               tile_keys, max_iter, prun);
            }
            int running = 0;
            MRSIM_CUDA(cudaMemcpyAsync(&running, prun, sizeof(int), cudaMemcpyDeviceToHost,
                                       c->stream));
            sync(c);
            if (running == 0) break;
        }
        {
            KScope ks(c, "cluster_partition");
            k_cl_part<<<g, kClThreads, 0, c->stream>>>(U, pord, ptx, psl, ptl, nt, tile_keys, pn,
                                                       err);
        }
        // the children back on the host
        const int first = hs[0].child0;
        made.resize(2 * m);
        MRSIM_CUDA(cudaMemcpyAsync(made.data(), pn + first, 2 * m * sizeof(ClNode),
                                   cudaMemcpyDeviceToHost, c->stream));
        MRSIM_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        sync(c);
        if (h_err) fail(MRSIM_ECUDA, "clustering: a split left a side empty");
        for (size_t j = 0; j < 2 * m; ++j) tree[first + j].set(made[j]);
    }
    const int n_made = (int)leaf_node.size();
    // labels of the distinct keys.  A cluster whose split was computed but not
    // taken may have had its range overwritten by splits below it; the leaves
    // of the computed tree are never overwritten, so every cluster labels the
    // computed leaves under its node.
    DBuf lab = dalloc(U * sizeof(int32_t));
    int32_t *plab = lab.as<int32_t>();
    {
        const int tile_keys = 2048;
        std::vector<int4> leaf;
        std::vector<int32_t> leaf_t0, stack;
        tiles.clear();
        for (int i = 0; i < n_made; ++i) {
            stack.assign(1, leaf_node[i]);
            while (!stack.empty()) {
                const TreeNode &h = tree[stack.back()];
                stack.pop_back();
                if (h.c0 >= 0) {
                    stack.push_back(h.c0);
                    stack.push_back(h.c1);
                    continue;
                }
                leaf_t0.push_back((int32_t)tiles.size());
                tiles.insert(tiles.end(), (h.count + tile_keys - 1) / tile_keys,
                             (int32_t)leaf.size());
                leaf.push_back(make_int4(h.buf, h.start, h.count, i));
            }
        }
        const int n_leaf = (int)leaf.size();
        DBuf dleaf = dalloc(n_leaf * sizeof(int4)), dt0 = dalloc(n_leaf * sizeof(int32_t));
        DBuf dlt = dalloc(tiles.size() * sizeof(int32_t));
        upload(c, dleaf.p, leaf.data(), n_leaf * sizeof(int4));
        upload(c, dt0.p, leaf_t0.data(), n_leaf * sizeof(int32_t));
        upload(c, dlt.p, tiles.data(), tiles.size() * sizeof(int32_t));
        KScope ks(c, "cluster_label");
        const int nt = (int)tiles.size();
        k_cl_leaf_label<<<std::min(nt, c->sm_count * 4), kClThreads, 0, c->stream>>>(
            U, pord, dleaf.as<int4>(), dt0.as<int32_t>(), dlt.as<int32_t>(), nt, tile_keys, plab);
    }
    std::vector<Cluster> cl(n_made);
    for (int i = 0; i < n_made; ++i) cl[i].set(tree[leaf_node[i]].s);
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
        k_cl_ratio<<<grid(c, U), kClThreads, 0, c->stream>>>(U, tf.as<float>(), plab, fc.as<double>(),
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
