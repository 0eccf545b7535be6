// Group builder (Sec. 2.4, Fig. 2): isochromats whose grouping keys are bit
// equal share a group; groups are numbered by first occurrence in isochromat
// index order.  Device hash table keyed by the key words; each slot keeps the
// smallest member index (the representative); representatives are ranked by a
// prefix sum over "is representative" flags, which yields the first-occurrence
// numbering directly.
//
// The same primitive groups (with-ADC gid, with-RF gid) pairs into cells to
// lay the isochromats out sorted by (ADC group, RF group): contiguous runs of
// one ADC group make the block sums of Eq. 9 a segmented reduction, and runs
// of one RF group make the combined-transition lookups warp-uniform.
#include <climits>
#include <algorithm>
#include <cmath>
#include <numeric>

#include "internal.h"

namespace mrsim {

namespace {

constexpr int kErrNaN = 1;
constexpr int kErrTableFull = 2;
constexpr int kErrGrow = 8;  // more distinct keys than the table was sized for

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z ^= z >> 30;
    z *= 0xbf58476d1ce4e5b9ull;
    z ^= z >> 27;
    z *= 0x94d049bb133111ebull;
    z ^= z >> 31;
    return z;
}

// Grouping key of one gradient type: (r_axis, T1, T2, dB0, b1, r_axis2) as
// float32 bit patterns, -0 folded to +0 (Fig. 2; the second position only for
// a two-axis type).  No-grads uses 0 for the position words, one-axis types 0
// for the second; a phantom without b1 uses 1.0f for it.
struct PhantomKey {
    static constexpr int W = 6;
    const float *pos, *T1, *T2, *dB0, *b1, *pos2;
    __device__ __forceinline__ bool words(int64_t k, uint32_t w[W]) const {
        float v[W] = {pos ? pos[k] : 0.0f, T1[k], T2[k], dB0[k], b1 ? b1[k] : 1.0f,
                      pos2 ? pos2[k] : 0.0f};
        bool ok = true;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            ok &= !isnan(v[i]);
            if (v[i] == 0.0f) v[i] = 0.0f;
            w[i] = __float_as_uint(v[i]);
        }
        return ok;
    }
};

// One position axis alone (float32 bit pattern, -0 folded to +0): numbers the
// distinct positions of that axis for the per-axis phasor tables.
struct AxisKey {
    static constexpr int W = 1;
    const float *pos;
    __device__ __forceinline__ bool words(int64_t k, uint32_t w[W]) const {
        float v = pos[k];
        if (v == 0.0f) v = 0.0f;
        w[0] = __float_as_uint(v);
        return !isnan(v);
    }
};

// Clustering key: the three integer features and the float32 bit patterns of
// T1 and T2 (which the M0 refit needs exactly).
struct FeatureKey {
    static constexpr int W = 5;
    const int32_t *x;
    const float *T1, *T2;
    int64_t K;
    __device__ __forceinline__ bool words(int64_t k, uint32_t w[W]) const {
        w[0] = (uint32_t)x[k];
        w[1] = (uint32_t)x[K + k];
        w[2] = (uint32_t)x[2 * K + k];
        w[3] = __float_as_uint(T1[k]);
        w[4] = __float_as_uint(T2[k]);
        return true;
    }
};

// (gid_a, gid_b) pair key for the layout cells.
struct PairKey {
    static constexpr int W = 2;
    const int32_t *a, *b;
    __device__ __forceinline__ bool words(int64_t k, uint32_t w[W]) const {
        w[0] = (uint32_t)a[k];
        w[1] = b ? (uint32_t)b[k] : 0u;
        return true;
    }
};

__device__ __forceinline__ uint64_t key_hash(const uint32_t *w, int n) {
    uint64_t h = 0x9e3779b97f4a7c15ull;
    for (int i = 0; i < n; ++i) h = mix64(h ^ (uint64_t)w[i] ^ ((uint64_t)i << 40));
    return h;
}

// Two-level insert.  A CTA takes a tile of kHashTile consecutive elements,
// numbers the tile's distinct keys in a shared-memory table, probes the global
// table once per distinct key (with the key's smallest index in the tile), and
// hands every element its global slot.  With thousands of groups over millions
// of isochromats a tile holds few distinct keys, so few global probes are made
// and no global slot becomes a hot spot.  Global slot: the owner is any member
// (it only serves key comparisons); minidx ends as the smallest member index.
constexpr int kHashThreads = 256;
constexpr int kHashPer = 4;
constexpr int kHashTile = kHashThreads * kHashPer;
constexpr int kHashLocal = 2 * kHashTile;  // never more than half full

// Global slot of the key of element k (bounded linear probing): claims an
// empty slot (counting the distinct keys; past key_limit the table is
// outgrown and the pass is redone) or finds the slot holding the same key;
// the slot's minimum index then covers k.  0 after an error.
template <class KF>
__device__ int32_t global_probe(const KF &kf, int64_t k, int32_t *owner, int32_t *minidx,
                                uint32_t mask, int key_limit, int *err, int *n_keys) {
    uint32_t w[KF::W];
    kf.words(k, w);
    uint32_t s = (uint32_t)key_hash(w, KF::W) & mask;
    for (uint32_t probes = 0;; ++probes) {
        if (probes > mask) {
            atomicOr(err, kErrTableFull);
            return 0;
        }
        int32_t o = __ldcg(&owner[s]);
        if (o < 0) {
            const int32_t prev = atomicCAS(&owner[s], -1, (int32_t)k);
            if (prev < 0) {
                if (atomicAdd(n_keys, 1) >= key_limit) atomicOr(err, kErrGrow);
                atomicMin(&minidx[s], (int32_t)k);
                return (int32_t)s;
            }
            o = prev;
        }
        uint32_t w2[KF::W];
        kf.words(o, w2);
        bool eq = true;
#pragma unroll
        for (int i = 0; i < KF::W; ++i) eq &= (w2[i] == w[i]);
        if (eq) {
            if ((int32_t)k < __ldcg(&minidx[s])) atomicMin(&minidx[s], (int32_t)k);
            return (int32_t)s;
        }
        s = (s + 1) & mask;
    }
}

template <class KF>
__global__ void __launch_bounds__(kHashThreads)
    k_hash_insert(int64_t K, KF kf, int32_t *owner, int32_t *minidx, int32_t *slot_of,
                  uint32_t mask, int key_limit, int *err, int *n_keys) {
    __shared__ int32_t l_rep[kHashLocal];   // tile index of the entry's first member, -1: free
    __shared__ int32_t l_min[kHashLocal];   // smallest tile index with the entry's key
    __shared__ int32_t l_slot[kHashLocal];  // global slot of the entry's key
    __shared__ int32_t l_used[kHashTile];   // occupied entries
    __shared__ int l_n;
    for (int i = threadIdx.x; i < kHashLocal; i += kHashThreads) {
        l_rep[i] = -1;
        l_min[i] = INT_MAX;
    }
    if (threadIdx.x == 0) l_n = 0;
    __syncthreads();
    for (int64_t base = blockIdx.x * (int64_t)kHashTile; base < K;
         base += (int64_t)gridDim.x * kHashTile) {
        // 1. the tile's distinct keys, numbered in shared memory
        int ent[kHashPer];
#pragma unroll
        for (int r = 0; r < kHashPer; ++r) {
            const int t = r * kHashThreads + threadIdx.x;
            const int64_t k = base + t;
            ent[r] = -1;
            if (k >= K) continue;
            uint32_t w[KF::W];
            if (!kf.words(k, w)) {
                atomicOr(err, kErrNaN);
                continue;
            }
            // local entry: a cheap 32-bit multiplicative fold of the words
            uint32_t hl = 0x9e3779b9u;
#pragma unroll
            for (int i = 0; i < KF::W; ++i) hl = (hl ^ w[i]) * 0x85ebca6bu;
            uint32_t e = (hl ^ (hl >> 15)) & (kHashLocal - 1);
            for (int probes = 0; probes < kHashLocal; ++probes) {
                int32_t rep = *(volatile int32_t *)&l_rep[e];
                if (rep < 0) {
                    rep = atomicCAS(&l_rep[e], -1, t);
                    if (rep < 0) {
                        l_used[atomicAdd(&l_n, 1)] = (int32_t)e;
                        ent[r] = (int)e;
                        break;
                    }
                }
                uint32_t w2[KF::W];
                kf.words(base + rep, w2);
                bool eq = true;
#pragma unroll
                for (int i = 0; i < KF::W; ++i) eq &= (w2[i] == w[i]);
                if (eq) {
                    ent[r] = (int)e;
                    break;
                }
                e = (e + 1) & (kHashLocal - 1);
            }
            if (ent[r] < 0) {  // unreachable: the table has room for every key of a tile
                atomicOr(err, kErrTableFull);
                continue;
            }
            if (t < *(volatile int32_t *)&l_min[ent[r]]) atomicMin(&l_min[ent[r]], t);
        }
        __syncthreads();
        // 2. one global probe per distinct key (bounded linear probing)
        const int nl = l_n;
        for (int u = threadIdx.x; u < nl; u += kHashThreads) {
            const int e = l_used[u];
            int32_t found = 0;
            if (*(volatile int *)err & kErrGrow) {  // the table is outgrown: the pass is redone
                l_slot[e] = found;
                continue;
            }
            found = global_probe(kf, base + l_min[e], owner, minidx, mask, key_limit, err, n_keys);
            l_slot[e] = found;
        }
        __syncthreads();
        // 3. every element's slot; then the used entries are freed
#pragma unroll
        for (int r = 0; r < kHashPer; ++r) {
            const int64_t k = base + r * kHashThreads + threadIdx.x;
            if (k < K) slot_of[k] = ent[r] >= 0 ? l_slot[ent[r]] : 0;
        }
        __syncthreads();
        for (int u = threadIdx.x; u < nl; u += kHashThreads) {
            const int e = l_used[u];
            l_rep[e] = -1;
            l_min[e] = INT_MAX;
        }
        if (threadIdx.x == 0) l_n = 0;
        __syncthreads();
    }
}

// One-word keys (the distinct positions of an axis: hundreds to thousands):
// a CTA keeps a cache key -> global slot in shared memory across all its
// tiles, so after its first tiles a lookup is a shared-memory probe.  Keys new
// to the cache are probed in the global table once per tile, with the tile's
// smallest index of the key (earlier tiles of a CTA hold smaller indices, so a
// key already cached needs no minimum update).  The cache is cleared when more
// than a quarter full at the end of a tile (a tile adds at most kHashTile).
constexpr int kAxisCache = 2048;
constexpr uint32_t kEmptyWord = 0xffffffffu;  // a NaN pattern: never a valid key

template <class KF>
__global__ void __launch_bounds__(kHashThreads)
    k_hash_insert_1w(int64_t K, KF kf, int32_t *owner, int32_t *minidx, int32_t *slot_of,
                     uint32_t mask, int key_limit, int *err, int *n_keys) {
    static_assert(KF::W == 1, "one-word keys");
    static_assert(kAxisCache / 4 + kHashTile <= kAxisCache, "cache room for a tile");
    __shared__ uint32_t c_key[kAxisCache];
    __shared__ int32_t c_slot[kAxisCache];  // global slot; -1 while new in this tile
    __shared__ int32_t c_min[kAxisCache];   // smallest tile index of a key new in this tile
    __shared__ int32_t l_used[kHashTile];   // entries new in this tile
    __shared__ int l_n, c_fill;
    for (int i = threadIdx.x; i < kAxisCache; i += kHashThreads) {
        c_key[i] = kEmptyWord;
        c_slot[i] = -1;
        c_min[i] = INT_MAX;
    }
    if (threadIdx.x == 0) {
        l_n = 0;
        c_fill = 0;
    }
    __syncthreads();
    for (int64_t base = blockIdx.x * (int64_t)kHashTile; base < K;
         base += (int64_t)gridDim.x * kHashTile) {
        int ent[kHashPer];
#pragma unroll
        for (int r = 0; r < kHashPer; ++r) {
            const int t = r * kHashThreads + threadIdx.x;
            const int64_t k = base + t;
            ent[r] = -1;
            if (k >= K) continue;
            uint32_t w[1];
            if (!kf.words(k, w)) {
                atomicOr(err, kErrNaN);
                continue;
            }
            uint32_t e = (w[0] * 0x9e3779b1u) >> 21;  // top 11 bits: [0, kAxisCache)
            for (int probes = 0; probes < kAxisCache; ++probes) {
                uint32_t kk = *(volatile uint32_t *)&c_key[e];
                if (kk == kEmptyWord) {
                    kk = atomicCAS(&c_key[e], kEmptyWord, w[0]);
                    if (kk == kEmptyWord) {
                        l_used[atomicAdd(&l_n, 1)] = (int32_t)e;
                        ent[r] = (int)e;
                        break;
                    }
                }
                if (kk == w[0]) {
                    ent[r] = (int)e;
                    break;
                }
                e = (e + 1) & (kAxisCache - 1);
            }
            if (ent[r] < 0) {  // unreachable: the cache keeps room for a tile
                atomicOr(err, kErrTableFull);
                continue;
            }
            if (*(volatile int32_t *)&c_slot[ent[r]] < 0 && t < *(volatile int32_t *)&c_min[ent[r]])
                atomicMin(&c_min[ent[r]], t);
        }
        __syncthreads();
        const int nl = l_n;
        for (int u = threadIdx.x; u < nl; u += kHashThreads) {
            const int e = l_used[u];
            c_slot[e] = (*(volatile int *)err & kErrGrow)
                            ? 0
                            : global_probe(kf, base + c_min[e], owner, minidx, mask, key_limit,
                                           err, n_keys);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kHashPer; ++r) {
            const int64_t k = base + r * kHashThreads + threadIdx.x;
            if (k < K) slot_of[k] = ent[r] >= 0 ? c_slot[ent[r]] : 0;
        }
        __syncthreads();
        const bool clear = c_fill + nl > kAxisCache / 4;  // uniform: read before the update
        __syncthreads();
        if (clear) {
            for (int i = threadIdx.x; i < kAxisCache; i += kHashThreads) {
                c_key[i] = kEmptyWord;
                c_slot[i] = -1;
                c_min[i] = INT_MAX;
            }
        }
        if (threadIdx.x == 0) {
            c_fill = clear ? 0 : c_fill + nl;
            l_n = 0;
        }
        __syncthreads();
    }
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_rep_flag(int64_t K, const int32_t *slot_of, const int32_t *minidx,
                           int32_t *flag) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x)
        flag[k] = (minidx[slot_of[k]] == (int32_t)k) ? 1 : 0;
}

__global__ void k_assign(int64_t K, const int32_t *slot_of, const int32_t *minidx,
                         const int32_t *rank, int32_t *gid) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x)
        gid[k] = rank[minidx[slot_of[k]]];
}

// ---- exclusive prefix sum of int32 flags (three passes) ----
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t &total) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    int64_t off = 0;
    total = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
        if (w < wid) off += warp_tot[w];
        total += warp_tot[w];
    }
    __syncthreads();
    return off + x - v;
}

__global__ void k_scan_tiles(const int32_t *in, int64_t n, int64_t *tile_sum) {
    int64_t base = blockIdx.x * (int64_t)kScanTile;
    int64_t s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + threadIdx.x * kScanItems + i;
        if (idx < n) s += in[idx];
    }
    int64_t tot;
    block_exclusive_scan(s, tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// exclusive scan of the tile sums in one CTA: thread t sums its contiguous
// chunk, one block scan gives the chunk offsets, and the chunks are written
// back in order
__global__ void k_scan_tile_sums(int64_t *tile_sum, int64_t nt) {
    const int64_t per = (nt + kScanThreads - 1) / kScanThreads;
    const int64_t b = threadIdx.x * per, e = min(nt, b + per);
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += tile_sum[i];
    int64_t tot;
    int64_t ex = block_exclusive_scan(s, tot);
    for (int64_t i = b; i < e; ++i) {
        const int64_t v = tile_sum[i];
        tile_sum[i] = ex;
        ex += v;
    }
}

__global__ void k_scan_apply(const int32_t *in, int64_t n, const int64_t *tile_off,
                             int32_t *out) {
    int64_t base = blockIdx.x * (int64_t)kScanTile;
    int32_t v[kScanItems];
    int64_t s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + threadIdx.x * kScanItems + i;
        v[i] = idx < n ? in[idx] : 0;
        s += v[i];
    }
    int64_t tot;
    int64_t ex = block_exclusive_scan(s, tot) + tile_off[blockIdx.x];
    for (int i = 0; i < kScanItems; ++i) {
        int64_t idx = base + threadIdx.x * kScanItems + i;
        if (idx < n) out[idx] = (int32_t)ex;
        ex += v[i];
    }
}

// per-group parameters from the representatives
__global__ void k_group_table(int64_t K, const int32_t *flag, const int32_t *rank,
                              const float *pos, const float *T1, const float *T2,
                              const float *dB0, const float *b1, const float *pos2,
                              double *o_pos, double *o_T1, double *o_T2, double *o_dB0,
                              double *o_b1, double *o_pos2) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[k]) continue;
        int32_t g = rank[k];
        o_pos[g] = pos ? (double)pos[k] : 0.0;
        o_T1[g] = T1[k];
        o_T2[g] = T2[k];
        o_dB0[g] = dB0[k];
        o_b1[g] = b1 ? (double)b1[k] : 1.0;
        o_pos2[g] = pos2 ? (double)pos2[k] : 0.0;
    }
}

// values of the distinct feature keys from their representatives
__global__ void k_feature_table(int64_t K, const int32_t *flag, const int32_t *rank,
                                const int32_t *x, const float *T1, const float *T2, int32_t *tab,
                                float *tf, int64_t U) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[k]) continue;
        const int32_t u = rank[k];
        tab[u] = x[k];
        tab[U + u] = x[K + k];
        tab[2 * U + u] = x[2 * K + k];
        tf[u] = T1[k];
        tf[U + u] = T2[k];
    }
}

__global__ void k_cell_table(int64_t K, const int32_t *flag, const int32_t *rank,
                             const int32_t *ga, const int32_t *gb, int32_t *oa, int32_t *ob) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[k]) continue;
        int32_t g = rank[k];
        oa[g] = ga[k];
        ob[g] = gb ? gb[k] : 0;
    }
}

// distinct values of one axis from its representatives
__global__ void k_axis_values(int64_t K, const int32_t *flag, const int32_t *rank,
                              const float *pos, float *val) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x)
        if (flag[k]) val[rank[k]] = pos[k] == 0.0f ? 0.0f : pos[k];
}

__global__ void k_pack_axis(int64_t K, const int32_t *lo, const int32_t *hi, int32_t *out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x)
        out[k] = (int32_t)((uint32_t)lo[k] | ((uint32_t)hi[k] << 16));
}

// warp-aggregated atomic add of 1 per element on counter[key]; returns the
// element's slot (old value + rank among same-key lanes)
__device__ __forceinline__ int32_t warp_agg_inc(int32_t *counter, int32_t key, bool active) {
    unsigned am = __ballot_sync(0xffffffffu, active);
    if (!active) return 0;
    unsigned peers = __match_any_sync(am, key);
    int lane = threadIdx.x & 31;
    int leader = __ffs(peers) - 1;
    int32_t base = 0;
    if (lane == leader) base = atomicAdd(&counter[key], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + __popc(peers & ((1u << lane) - 1u));
}

__global__ void k_count(int64_t K, const int32_t *key, int32_t *count) {
    for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x; k0 < K;
         k0 += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = k0 + threadIdx.x;
        bool act = k < K;
        warp_agg_inc(count, act ? key[k] : 0, act);
    }
}

// Dense cells: when (primary groups) x (secondary groups) is small, the cell
// key g_p * G_s + g_s indexes a flag array directly; an exclusive scan of the
// flags numbers the present keys in (g_p, g_s) order, which is the layout's
// cell order, so no hashing or host sort is needed.
__global__ void k_cell_mark(int64_t K, const int32_t *ga, const int32_t *gb, int32_t Gb,
                            int32_t *present) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x)
        present[(int64_t)ga[k] * Gb + (gb ? gb[k] : 0)] = 1;
}

// cell of every isochromat (the rank of its key) and the member count per cell
__global__ void k_cell_assign(int64_t K, const int32_t *ga, const int32_t *gb, int32_t Gb,
                              const int32_t *rank, int32_t *cell, int32_t *count) {
    for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x; k0 < K;
         k0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = k0 + threadIdx.x;
        const bool act = k < K;
        int32_t c = 0;
        if (act) {
            c = rank[(int64_t)ga[k] * Gb + (gb ? gb[k] : 0)];
            cell[k] = c;
        }
        warp_agg_inc(count, c, act);
    }
}

// primary and secondary group of every cell
__global__ void k_cell_keys(int64_t NK, const int32_t *present, const int32_t *rank, int32_t Gb,
                            int32_t *cgp, int32_t *cgr) {
    for (int64_t key = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; key < NK;
         key += (int64_t)gridDim.x * blockDim.x) {
        if (!present[key]) continue;
        const int32_t c = rank[key];
        cgp[c] = (int32_t)(key / Gb);
        cgr[c] = (int32_t)(key % Gb);
    }
}

__global__ void k_scatter(int64_t K, const int32_t *cell, const int32_t *cell_off,
                          int32_t *cursor, int32_t *perm) {
    for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x; k0 < K;
         k0 += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = k0 + threadIdx.x;
        bool act = k < K;
        int32_t c = act ? cell[k] : 0;
        int32_t r = warp_agg_inc(cursor, c, act);
        if (act) perm[cell_off[c] + r] = (int32_t)k;
    }
}

// Thread t of the cell-mode fused kernel: cell c with off[c] <= t < off[c + 1]
// has T = ceil(count / NI) threads; its thread j = t - off[c] takes the cell's
// isochromats j, j + T, j + 2T, ... (at most NI), so the lanes of a warp hold
// consecutive isochromats of the layout at every register index.
__global__ void k_cell_threads(int64_t nc, const int64_t *off, const int32_t *start,
                               const int32_t *count, int NI, int2 *out) {
    const int64_t n = off[nc];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nc - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (off[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const int j = (int)(t - off[lo]);
        const int T = (count[lo] + NI - 1) / NI;
        const int n_iso = (count[lo] - j + T - 1) / T;
        out[t] = make_int2(start[lo] + j, (int)((lo << 4) | n_iso));
    }
}

// Sorts every cell's run of the layout permutation by phantom index (the
// scatter leaves members in atomic order): the layout becomes deterministic,
// and along a cell consecutive positions hold isochromats in phantom order,
// so neighbouring lanes of the fused kernel read neighbouring table entries.
// Runs of at most kWarpSortMax members: one warp each, a bitonic network in
// registers; longer runs: one CTA each, every member placed by the number of
// members below it (they are distinct), counted over the run in shared
// memory.  Runs longer than kSortMax keep the scatter order.
constexpr int kSortMax = 4096;
constexpr int kWarpSortMax = 1024;  // runs up to this length: one warp each

__device__ __forceinline__ int rank_below(const int32_t *v, int n4, int x) {
    const int4 *v4 = reinterpret_cast<const int4 *>(v);
    int r = 0;
    for (int j = 0; j < n4 / 4; ++j) {
        const int4 q = v4[j];
        r += (int)(q.x < x) + (int)(q.y < x) + (int)(q.z < x) + (int)(q.w < x);
    }
    return r;
}

// Bitonic sorting network over 32 J values held by a warp, element i = 32 j +
// lane in v[j]: exchanges at distance d >= 32 stay within a lane, shorter
// ones go through shuffles.  Ascending order.
template <int J>
__device__ __forceinline__ void warp_bitonic(int32_t (&v)[J], int lane) {
    constexpr int kLog = J == 1 ? 5 : J == 2 ? 6 : J == 4 ? 7 : J == 8 ? 8 : J == 16 ? 9 : 10;
    static_assert(J == 1 || J == 2 || J == 4 || J == 8 || J == 16 || J == 32, "J");
#pragma unroll
    for (int lk = 1; lk <= kLog; ++lk) {
        const int k = 1 << lk;
#pragma unroll
        for (int ld = lk - 1; ld >= 0; --ld) {
            const int d = 1 << ld;
            if (d >= 32) {
                const int dj = d >> 5;
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    if ((j & dj) == 0) {
                        const bool up = ((j * 32 + lane) & k) == 0;
                        const int32_t a = v[j], b = v[j | dj];
                        if ((a > b) == up) {
                            v[j] = b;
                            v[j | dj] = a;
                        }
                    }
                }
            } else {
                const bool lower = (lane & d) == 0;
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const int32_t p = __shfl_xor_sync(0xffffffffu, v[j], d);
                    const bool up = ((j * 32 + lane) & k) == 0;
                    v[j] = (lower == up) ? min(v[j], p) : max(v[j], p);
                }
            }
        }
    }
}

// one run of n <= 32 J members, sorted by the warp in registers
template <int J>
__device__ __forceinline__ void warp_sort_run(int32_t *run, int n, int lane) {
    int32_t v[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int i = j * 32 + lane;
        v[j] = i < n ? run[i] : INT_MAX;
    }
    warp_bitonic<J>(v, lane);
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int i = j * 32 + lane;
        if (i < n) run[i] = v[j];
    }
}

__global__ void __launch_bounds__(256) k_sort_cells(const int32_t *cstart, const int32_t *ccount,
                                                    int64_t nc, int32_t *perm) {
    __shared__ __align__(16) int32_t v[kSortMax];  // one longer run
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // runs of at most kWarpSortMax: a warp each, in registers
    for (int64_t c = (int64_t)blockIdx.x * 8 + warp; c < nc; c += (int64_t)gridDim.x * 8) {
        const int n = ccount[c];
        if (n < 2 || n > kWarpSortMax) continue;  // uniform in the warp
        int32_t *run = perm + cstart[c];
        if (n <= 32) warp_sort_run<1>(run, n, lane);
        else if (n <= 64) warp_sort_run<2>(run, n, lane);
        else if (n <= 128) warp_sort_run<4>(run, n, lane);
        else if (n <= 256) warp_sort_run<8>(run, n, lane);
        else if (n <= 512) warp_sort_run<16>(run, n, lane);
        else warp_sort_run<32>(run, n, lane);
    }
    __syncthreads();
    // longer runs: the whole CTA on one run, each member placed by the number
    // of members below it
    for (int64_t c = blockIdx.x; c < nc; c += gridDim.x) {
        const int n = ccount[c];
        if (n <= kWarpSortMax || n > kSortMax) continue;  // uniform in the CTA
        const int n4 = (n + 3) & ~3;
        const int s = cstart[c];
        for (int i = threadIdx.x; i < n4; i += blockDim.x) v[i] = i < n ? perm[s + i] : INT_MAX;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int x = v[i];
            perm[s + rank_below(v, n4, x)] = x;
        }
        __syncthreads();
    }
}

// out[a][i] = in[a][perm[i]] for up to kGatherMax 32-bit arrays in one pass
constexpr int kGatherMax = 24;
struct GatherSet {
    const uint32_t *in[kGatherMax];
    uint32_t *out[kGatherMax];
    int n;
};

// A CTA takes kGatherPer x 256 consecutive layout positions; each thread keeps
// its positions' phantom indices in registers and walks the arrays one at a
// time.  Consecutive phantom indices fall in neighbouring cells of the
// layout, so a sector one load brings into L1 serves the tile's other cells
// before it is evicted, instead of coming from L2 once per member.
constexpr int kGatherPer = 8;
constexpr int kGatherTile = 256 * kGatherPer;

__global__ void __launch_bounds__(256) k_gather_set(int64_t K, const int32_t *perm, GatherSet g) {
    for (int64_t base = blockIdx.x * (int64_t)kGatherTile; base < K;
         base += (int64_t)gridDim.x * kGatherTile) {
        int32_t p[kGatherPer];
#pragma unroll
        for (int r = 0; r < kGatherPer; ++r) {
            const int64_t i = base + r * 256 + threadIdx.x;
            p[r] = i < K ? perm[i] : 0;
        }
        for (int a = 0; a < g.n; ++a) {
            const uint32_t *in = g.in[a];
            uint32_t *out = g.out[a];
            uint32_t v[kGatherPer];  // every load issued before the first store
#pragma unroll
            for (int r = 0; r < kGatherPer; ++r) v[r] = __ldg(in + p[r]);
#pragma unroll
            for (int r = 0; r < kGatherPer; ++r) {
                const int64_t i = base + r * 256 + threadIdx.x;
                if (i < K) out[i] = v[r];
            }
        }
    }
}

template <typename T>
__global__ void k_gather(int64_t K, const int32_t *perm, const T *in, T *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < K;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[perm[i]];
}

int grid_for(mrsim_ctx *c, int64_t n, int threads = 256) {
    int64_t b = (n + threads - 1) / threads;
    int64_t cap = (int64_t)c->sm_count * 16;
    return (int)std::max<int64_t>(1, std::min(b, cap));
}

// Hash-group K elements; writes rank-of-representative gid[K] and returns the
// group count.  flag/rank stay in scratch slots 2/3 for table extraction.  The
// table first gets kHashFirstSlots slots (it then stays in L2 and is cheap to
// clear); if more than half of them fill, the kernel says so and the whole
// pass is redone with room for K distinct keys.  Callers that expect many
// distinct keys (few_keys = false) start with that room.
constexpr uint64_t kHashFirstSlots = 1ull << 21;

template <class KF>
int64_t hash_group(mrsim_ctx *c, int64_t K, const KF &kf, int32_t *gid, int32_t **flag_out,
                   int32_t **rank_out, bool few_keys = true) {
    uint64_t C_full = 1024;
    while (C_full < (uint64_t)(2 * K)) C_full <<= 1;
    if (C_full > (1ull << 31)) fail(MRSIM_EINVAL, "too many isochromats for the group hash table");
    for (uint64_t C = few_keys ? std::min(C_full, kHashFirstSlots) : C_full;; C = C_full) {
        int32_t *owner = (int32_t *)scratch(c, 0, C * sizeof(int32_t));
        int32_t *minidx = (int32_t *)scratch(c, 1, C * sizeof(int32_t));
        int32_t *flag = (int32_t *)scratch(c, 2, K * sizeof(int32_t));
        int32_t *rank = (int32_t *)scratch(c, 3, K * sizeof(int32_t));
        int32_t *slot_of = (int32_t *)scratch(c, 4, K * sizeof(int32_t));
        int64_t nt = (K + kScanTile - 1) / kScanTile;
        int64_t *tsum = (int64_t *)scratch(c, 5, nt * sizeof(int64_t));
        int *err = c->dev_err.as<int>();  // [0] error bits, [1] distinct keys inserted
        MRSIM_CUDA(cudaMemsetAsync(err, 0, 2 * sizeof(int), c->stream));
        MRSIM_CUDA(cudaMemsetAsync(owner, 0xff, C * sizeof(int32_t), c->stream));
        {
            KScope ks(c, "group_fill");
            k_fill_i32<<<grid_for(c, C), 256, 0, c->stream>>>(minidx, C, 0x7fffffff);
        }
        {
            KScope ks(c, "group_hash_insert");
            if constexpr (KF::W == 1)
                k_hash_insert_1w<<<grid_for(c, K, kHashTile), kHashThreads, 0, c->stream>>>(
                    K, kf, owner, minidx, slot_of, (uint32_t)(C - 1), (int)(C / 2), err, err + 1);
            else
                k_hash_insert<<<grid_for(c, K, kHashTile), kHashThreads, 0, c->stream>>>(
                    K, kf, owner, minidx, slot_of, (uint32_t)(C - 1), (int)(C / 2), err, err + 1);
        }
        {
            KScope ks(c, "group_rep_flag");
            k_rep_flag<<<grid_for(c, K), 256, 0, c->stream>>>(K, slot_of, minidx, flag);
        }
        {
            KScope ks(c, "scan_tiles");
            k_scan_tiles<<<(unsigned)nt, kScanThreads, 0, c->stream>>>(flag, K, tsum);
        }
        {
            KScope ks(c, "scan_tile_sums");
            k_scan_tile_sums<<<1, kScanThreads, 0, c->stream>>>(tsum, nt);
        }
        {
            KScope ks(c, "scan_apply");
            k_scan_apply<<<(unsigned)nt, kScanThreads, 0, c->stream>>>(flag, K, tsum, rank);
        }
        {
            KScope ks(c, "group_assign");
            k_assign<<<grid_for(c, K), 256, 0, c->stream>>>(K, slot_of, minidx, rank, gid);
        }
        int h_err = 0;
        int32_t last[2] = {0, 0};
        MRSIM_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        MRSIM_CUDA(cudaMemcpyAsync(&last[0], rank + (K - 1), sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, c->stream));
        MRSIM_CUDA(cudaMemcpyAsync(&last[1], flag + (K - 1), sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, c->stream));
        sync(c);
        if (h_err & kErrNaN) fail(MRSIM_EINVAL, "NaN in a grouping key");
        if ((h_err & kErrGrow) && C < C_full) continue;
        if (h_err & (kErrTableFull | kErrGrow)) fail(MRSIM_ECUDA, "group hash table overflow");
        *flag_out = flag;
        *rank_out = rank;
        return (int64_t)last[0] + last[1];
    }
}

}  // namespace

namespace {

// Group-signal tables of G groups from the FP64 block [pos, T1, T2, dB0, b1,
// pos2]: positions and dB0 as float and double, and log2(e) / T2 (0 for an
// infinite T2), the decay rate in base-2 exponent units.
__global__ void k_group_signal_tables(int64_t G, const double *par, float *pos, float *dB0,
                                      float *rT2, float *pos2, double *pos64, double *dB064,
                                      double *rT264, double *pos264) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x) {
        const double p = par[g], t2 = par[2 * G + g], d = par[3 * G + g], p2 = par[5 * G + g];
        const double r = isinf(t2) ? 0.0 : kLog2e / t2;
        pos[g] = (float)p;
        dB0[g] = (float)d;
        rT2[g] = (float)r;
        pos2[g] = (float)p2;
        pos64[g] = p;
        dB064[g] = d;
        rT264[g] = r;
        pos264[g] = p2;
    }
}

}  // namespace

void build_group_type(mrsim_ctx *c, const mrsim_phantom_t *ph, int gtype, DBuf &gid,
                      int64_t &n_groups, GroupTable &tab) {
    const int64_t K = ph->K;
    const float *axis[3] = {ph->x.as<float>(), ph->y.as<float>(), ph->z.as<float>()};
    const int a0 = gtype_axis0(gtype), a1 = gtype_axis1(gtype);
    const float *pos = a0 >= 0 ? axis[a0] : nullptr;
    const float *pos2 = a1 >= 0 ? axis[a1] : nullptr;
    PhantomKey kf{pos, ph->T1.as<float>(), ph->T2.as<float>(), ph->dB0.as<float>(),
                  ph->has_b1 ? ph->b1.as<float>() : nullptr, pos2};
    gid = dalloc(K * sizeof(int32_t));
    int32_t *flag, *rank;
    n_groups = hash_group(c, K, kf, gid.as<int32_t>(), &flag, &rank);
    const int64_t G = n_groups;
    DBuf t = dalloc(6 * G * sizeof(double));
    double *tp = t.as<double>();
    {
        KScope ks(c, "group_table");
        k_group_table<<<grid_for(c, K), 256, 0, c->stream>>>(
            K, flag, rank, pos, ph->T1.as<float>(), ph->T2.as<float>(), ph->dB0.as<float>(),
            ph->has_b1 ? ph->b1.as<float>() : nullptr, pos2, tp, tp + G, tp + 2 * G, tp + 3 * G,
            tp + 4 * G, tp + 5 * G);
    }
    tab.n = G;
    // device copies used by the precompute and group-signal kernels, formed
    // from the FP64 block on the device
    auto mk = [&](DBuf &d, size_t el) { d = dalloc(std::max<int64_t>(G, 1) * el); };
    mk(tab.d_pos, 4);
    mk(tab.d_dB0, 4);
    mk(tab.d_rT2, 4);
    mk(tab.d_pos2, 4);
    mk(tab.d_pos64, 8);
    mk(tab.d_dB064, 8);
    mk(tab.d_rT264, 8);
    mk(tab.d_pos264, 8);
    {
        KScope ks(c, "group_table");
        k_group_signal_tables<<<grid_for(c, G), 256, 0, c->stream>>>(
            G, tp, tab.d_pos.as<float>(), tab.d_dB0.as<float>(), tab.d_rT2.as<float>(),
            tab.d_pos2.as<float>(), tab.d_pos64.as<double>(), tab.d_dB064.as<double>(),
            tab.d_rT264.as<double>(), tab.d_pos264.as<double>());
    }
    // FP64 parameter block (pos, T1, T2, dB0, b1, pos2) for the precompute kernel
    tab.d_par64 = std::move(t);
}

namespace {

// exclusive prefix sum of n int32 values (three passes) into out
void scan_i32(mrsim_ctx *c, const int32_t *in, int64_t n, int32_t *out) {
    const int64_t nt = (n + kScanTile - 1) / kScanTile;
    int64_t *tsum = (int64_t *)scratch(c, 5, nt * sizeof(int64_t));
    {
        KScope ks(c, "scan_tiles");
        k_scan_tiles<<<(unsigned)nt, kScanThreads, 0, c->stream>>>(in, n, tsum);
    }
    {
        KScope ks(c, "scan_tile_sums");
        k_scan_tile_sums<<<1, kScanThreads, 0, c->stream>>>(tsum, nt);
    }
    {
        KScope ks(c, "scan_apply");
        k_scan_apply<<<(unsigned)nt, kScanThreads, 0, c->stream>>>(in, n, tsum, out);
    }
}

// largest (primary groups) x (secondary groups) laid out through a flag array
constexpr int64_t kDenseCells = 1 << 24;

}  // namespace

void build_layout(mrsim_ctx *c, const mrsim_phantom_t *ph, mrsim_groups *g) {
    const int64_t K = ph->K;
    const int p = g->primary, s = g->secondary;
    const int32_t *ga = g->gid_orig[p].as<int32_t>();
    const int32_t *gb = s >= 0 ? g->gid_orig[s].as<int32_t>() : nullptr;
    const int64_t Ga = g->n_groups[p], Gb = s >= 0 ? g->n_groups[s] : 1;
    DBuf cell = dalloc(K * sizeof(int32_t));  // cell id of every isochromat
    DBuf doff_own;                            // layout offset of every cell id (hashed ids)
    const int32_t *doff = nullptr;
    std::vector<int32_t> s_cnt;  // member counts, cells in layout order
    int64_t nc = 0;
    auto up32 = [&](DBuf &d, const std::vector<int32_t> &v) {
        d = dalloc(std::max<int64_t>(nc, 1) * sizeof(int32_t));
        upload(c, d.p, v.data(), nc * sizeof(int32_t));
    };
    if (Ga * Gb <= kDenseCells) {
        // cell ids are the ranks of the present keys g_p * G_s + g_s: layout order
        const int64_t NK = Ga * Gb;
        DBuf present = dalloc(NK * sizeof(int32_t)), rank = dalloc(NK * sizeof(int32_t));
        MRSIM_CUDA(cudaMemsetAsync(present.p, 0, NK * sizeof(int32_t), c->stream));
        {
            KScope ks(c, "layout_cell_mark");
            k_cell_mark<<<grid_for(c, K), 256, 0, c->stream>>>(K, ga, gb, (int32_t)Gb,
                                                               present.as<int32_t>());
        }
        scan_i32(c, present.as<int32_t>(), NK, rank.as<int32_t>());
        int32_t last[2] = {0, 0};
        MRSIM_CUDA(cudaMemcpyAsync(&last[0], rank.as<int32_t>() + (NK - 1), sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, c->stream));
        MRSIM_CUDA(cudaMemcpyAsync(&last[1], present.as<int32_t>() + (NK - 1), sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, c->stream));
        sync(c);
        nc = (int64_t)last[0] + last[1];
        g->n_cells = nc;
        g->cell_count = dalloc(nc * sizeof(int32_t));
        g->cell_start = dalloc(nc * sizeof(int32_t));
        g->cell_gp = dalloc(nc * sizeof(int32_t));
        g->cell_gr = dalloc(nc * sizeof(int32_t));
        MRSIM_CUDA(cudaMemsetAsync(g->cell_count.p, 0, nc * sizeof(int32_t), c->stream));
        {
            KScope ks(c, "layout_cell_assign");
            k_cell_assign<<<grid_for(c, K), 256, 0, c->stream>>>(
                K, ga, gb, (int32_t)Gb, rank.as<int32_t>(), cell.as<int32_t>(),
                g->cell_count.as<int32_t>());
        }
        {
            KScope ks(c, "layout_cell_table");
            k_cell_keys<<<grid_for(c, NK), 256, 0, c->stream>>>(
                NK, present.as<int32_t>(), rank.as<int32_t>(), (int32_t)Gb,
                g->cell_gp.as<int32_t>(), g->cell_gr.as<int32_t>());
        }
        scan_i32(c, g->cell_count.as<int32_t>(), nc, g->cell_start.as<int32_t>());
        s_cnt.resize(nc);
        MRSIM_CUDA(cudaMemcpyAsync(s_cnt.data(), g->cell_count.p, nc * sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, c->stream));
        sync(c);
        doff = g->cell_start.as<int32_t>();
    } else {
        // hashed cell ids, ordered on the host
        PairKey kf{ga, gb};
        int32_t *flag, *rank;
        nc = hash_group(c, K, kf, cell.as<int32_t>(), &flag, &rank);
        g->n_cells = nc;
        DBuf ca = dalloc(nc * sizeof(int32_t)), cb = dalloc(nc * sizeof(int32_t));
        DBuf cnt = dalloc(nc * sizeof(int32_t));
        {
            KScope ks(c, "layout_cell_table");
            k_cell_table<<<grid_for(c, K), 256, 0, c->stream>>>(K, flag, rank, kf.a, kf.b,
                                                                ca.as<int32_t>(), cb.as<int32_t>());
        }
        MRSIM_CUDA(cudaMemsetAsync(cnt.p, 0, nc * sizeof(int32_t), c->stream));
        {
            KScope ks(c, "layout_count");
            k_count<<<grid_for(c, K), 256, 0, c->stream>>>(K, cell.as<int32_t>(),
                                                           cnt.as<int32_t>());
        }
        std::vector<int32_t> ha(nc), hb(nc), hc(nc);
        MRSIM_CUDA(cudaMemcpyAsync(ha.data(), ca.p, nc * 4, cudaMemcpyDeviceToHost, c->stream));
        MRSIM_CUDA(cudaMemcpyAsync(hb.data(), cb.p, nc * 4, cudaMemcpyDeviceToHost, c->stream));
        MRSIM_CUDA(cudaMemcpyAsync(hc.data(), cnt.p, nc * 4, cudaMemcpyDeviceToHost, c->stream));
        sync(c);
        // cells sorted by (primary gid, secondary gid): both are group ids below
        // known bounds, so two stable counting passes (by the secondary id, then by
        // the primary id) sort in linear time; the pairs are distinct, so the order
        // is the unique sorted one
        std::vector<int32_t> by_b(nc), order(nc);
        {
            std::vector<int32_t> pos(Gb + 1, 0);
            for (int64_t i = 0; i < nc; ++i) ++pos[hb[i] + 1];
            for (int64_t v = 0; v < Gb; ++v) pos[v + 1] += pos[v];
            for (int64_t i = 0; i < nc; ++i) by_b[pos[hb[i]]++] = (int32_t)i;
        }
        {
            std::vector<int32_t> pos(Ga + 1, 0);
            for (int64_t i = 0; i < nc; ++i) ++pos[ha[i] + 1];
            for (int64_t v = 0; v < Ga; ++v) pos[v + 1] += pos[v];
            for (int64_t t = 0; t < nc; ++t) {
                const int32_t i = by_b[t];
                order[pos[ha[i]]++] = i;
            }
        }
        std::vector<int32_t> off(nc);
        int64_t run = 0;
        for (int64_t i = 0; i < nc; ++i) {
            off[order[i]] = (int32_t)run;
            run += hc[order[i]];
        }
        doff_own = dalloc(nc * sizeof(int32_t));
        upload(c, doff_own.p, off.data(), nc * 4);
        doff = doff_own.as<int32_t>();
        // cell tables in layout order, for the cell-mode fused kernel
        std::vector<int32_t> s_start(nc), s_gp(nc), s_gr(nc);
        s_cnt.resize(nc);
        for (int64_t i = 0; i < nc; ++i) {
            const int32_t cc = order[i];
            s_start[i] = off[cc];
            s_cnt[i] = hc[cc];
            s_gp[i] = ha[cc];
            s_gr[i] = hb[cc];
        }
        up32(g->cell_start, s_start);
        up32(g->cell_count, s_cnt);
        up32(g->cell_gp, s_gp);
        up32(g->cell_gr, s_gr);
    }
    build_cell_threads(c, g, s_cnt);
    DBuf cursor = dalloc(nc * sizeof(int32_t));
    MRSIM_CUDA(cudaMemsetAsync(cursor.p, 0, nc * sizeof(int32_t), c->stream));
    g->perm = dalloc(K * sizeof(int32_t));
    {
        KScope ks(c, "layout_scatter");
        k_scatter<<<grid_for(c, K), 256, 0, c->stream>>>(K, cell.as<int32_t>(), doff,
                                                         cursor.as<int32_t>(), g->perm.as<int32_t>());
    }
    {
        KScope ks(c, "layout_sort_cells");
        const unsigned grid = (unsigned)std::max<int64_t>(
            1, std::min<int64_t>(nc, (int64_t)c->sm_count * 16));
        k_sort_cells<<<grid, 256, 0, c->stream>>>(g->cell_start.as<int32_t>(),
                                                  g->cell_count.as<int32_t>(), nc,
                                                  g->perm.as<int32_t>());
    }
    const int32_t *perm = g->perm.as<int32_t>();
    // the per-isochromat arrays in layout order.  Gathered now: M0 and the
    // positions the axis index is built from; the rest (the primary axis
    // position, T1, T2, dB0, b1 and the layout-order group ids, which only the
    // per-isochromat form and the fallbacks read) is allocated now and gathered
    // by the first run that needs it (ensure_layout_arrays)
    GatherSet gs{};
    auto add = [&](DBuf &dst, const void *src) {
        dst = dalloc(K * sizeof(uint32_t));
        gs.in[gs.n] = static_cast<const uint32_t *>(src);
        gs.out[gs.n] = dst.as<uint32_t>();
        ++gs.n;
    };
    const int pa = (g->primary >= G_X && g->primary <= G_Z) ? g->primary - 1 : -1;
    DBuf *pos_dst[3] = {&g->x, &g->y, &g->z};
    const DBuf *pos_src[3] = {&ph->x, &ph->y, &ph->z};
    for (int a = 0; a < 3; ++a)
        if (a != pa) add(*pos_dst[a], pos_src[a]->p);
    add(g->M0, ph->M0.p);
    {
        KScope ks(c, "layout_gather");
        k_gather_set<<<grid_for(c, K, kGatherTile), 256, 0, c->stream>>>(K, perm, gs);
    }
    if (pa >= 0) *pos_dst[pa] = dalloc(K * sizeof(float));
    g->T1 = dalloc(K * sizeof(float));
    g->T2 = dalloc(K * sizeof(float));
    g->dB0 = dalloc(K * sizeof(float));
    g->has_b1 = ph->has_b1;
    if (ph->has_b1) g->b1 = dalloc(K * sizeof(float));
    for (int t = 0; t < kNTypes; ++t)
        if (g->built[t]) g->gid_sorted[t] = dalloc(K * sizeof(int32_t));
    g->rest_pending = true;
    g->has_M_init = ph->has_M_init;
    if (ph->has_M_init) {
        g->M_init = dalloc(3 * K * sizeof(float));
        GatherSet gm{};
        for (int r = 0; r < 3; ++r) {
            gm.in[r] = ph->M_init.as<uint32_t>() + r * K;
            gm.out[r] = g->M_init.as<uint32_t>() + r * K;
        }
        gm.n = 3;
        KScope ks(c, "layout_gather");
        k_gather_set<<<grid_for(c, K, kGatherTile), 256, 0, c->stream>>>(K, perm, gm);
    }
    sync(c);
}

void ensure_layout_arrays(mrsim_ctx *c, const mrsim_groups *cg, const mrsim_phantom_t *ph) {
    if (!cg->rest_pending) return;
    // the arrays were allocated by the group build; only their contents are
    // formed here (the group set is not shared between threads)
    mrsim_groups *g = const_cast<mrsim_groups *>(cg);
    const int64_t K = g->K;
    GatherSet gs{};
    auto add = [&](DBuf &dst, const void *src) {
        gs.in[gs.n] = static_cast<const uint32_t *>(src);
        gs.out[gs.n] = dst.as<uint32_t>();
        ++gs.n;
    };
    const int pa = (g->primary >= G_X && g->primary <= G_Z) ? g->primary - 1 : -1;
    if (pa == 0) add(g->x, ph->x.p);
    if (pa == 1) add(g->y, ph->y.p);
    if (pa == 2) add(g->z, ph->z.p);
    add(g->T1, ph->T1.p);
    add(g->T2, ph->T2.p);
    add(g->dB0, ph->dB0.p);
    if (g->has_b1) add(g->b1, ph->b1.p);
    for (int t = 0; t < kNTypes; ++t)
        if (g->built[t]) add(g->gid_sorted[t], g->gid_orig[t].p);
    static_assert(1 + 4 + kNTypes <= kGatherMax, "gather set too small");
    {
        KScope ks(c, "layout_gather");
        k_gather_set<<<grid_for(c, K, kGatherTile), 256, 0, c->stream>>>(
            K, g->perm.as<int32_t>(), gs);
    }
    MRSIM_CUDA(cudaGetLastError());
    g->rest_pending = false;
}

void build_cell_threads(mrsim_ctx *c, mrsim_groups *g, const std::vector<int32_t> &count) {
    const int64_t nc = (int64_t)count.size();
    g->n_cell_thr[0] = g->n_cell_thr[1] = 0;
    if (nc <= 0 || nc >= (1LL << 27)) return;  // cell index must fit 27 bits
    DBuf d_off = dalloc((nc + 1) * sizeof(int64_t));
    for (int w = 0; w < 2; ++w) {
        const int NI = w == 0 ? 4 : 8;
        std::vector<int64_t> off(nc + 1, 0);
        for (int64_t i = 0; i < nc; ++i) off[i + 1] = off[i] + (count[i] + NI - 1) / NI;
        const int64_t n = off[nc];
        if (n >= (1LL << 31)) return;
        upload(c, d_off.p, off.data(), (nc + 1) * sizeof(int64_t));
        g->cell_thr[w] = dalloc(n * sizeof(int2));
        KScope ks(c, "layout_cell_threads");
        k_cell_threads<<<grid_for(c, n), 256, 0, c->stream>>>(
            nc, d_off.as<int64_t>(), g->cell_start.as<int32_t>(), g->cell_count.as<int32_t>(), NI,
            g->cell_thr[w].as<int2>());
        // the next upload reuses d_off: wait for this expansion first
        sync(c);
        g->n_cell_thr[w] = n;
    }
}

// Distinct positions of the two non-primary axes (layout order) and the
// packed per-isochromat indices into them.  Leaves g->ax_ok false when the
// layout has no primary axis or an axis has too many distinct positions.
void build_axis_index(mrsim_ctx *c, mrsim_groups *g) {
    g->ax_ok = false;
    const int p = g->primary;
    if (p < G_X || p > G_Z) return;
    const int64_t K = g->K;
    const float *pos[3] = {g->x.as<float>(), g->y.as<float>(), g->z.as<float>()};
    int ax[2], n = 0;
    for (int a = 0; a < 3; ++a)
        if (a != p - 1) ax[n++] = a;
    DBuf idx[2];
    for (int i = 0; i < 2; ++i) {
        const int a = ax[i];
        idx[i] = dalloc(K * sizeof(int32_t));
        int32_t *flag, *rank;
        const int64_t nv = hash_group(c, K, AxisKey{pos[a]}, idx[i].as<int32_t>(), &flag, &rank);
        if (nv > kMaxAxisValues) return;
        g->n_ax[a] = nv;
        g->ax_val[a] = dalloc(nv * sizeof(float));
        KScope ks(c, "axis_values");
        k_axis_values<<<grid_for(c, K), 256, 0, c->stream>>>(K, flag, rank, pos[a],
                                                             g->ax_val[a].as<float>());
    }
    g->ax_idx = dalloc(K * sizeof(int32_t));
    {
        KScope ks(c, "axis_pack");
        k_pack_axis<<<grid_for(c, K), 256, 0, c->stream>>>(K, idx[0].as<int32_t>(),
                                                           idx[1].as<int32_t>(),
                                                           g->ax_idx.as<int32_t>());
    }
    sync(c);
    g->ax_ok = true;
}

int64_t distinct_features(mrsim_ctx *c, int64_t K, const int32_t *x, const float *T1,
                          const float *T2, int32_t *id, DBuf &table, DBuf &tf, DBuf &count) {
    int32_t *flag, *rank;
    const int64_t U = hash_group(c, K, FeatureKey{x, T1, T2, K}, id, &flag, &rank, false);
    table = dalloc(3 * U * sizeof(int32_t));
    tf = dalloc(2 * U * sizeof(float));
    count = dalloc(U * sizeof(int32_t));
    MRSIM_CUDA(cudaMemsetAsync(count.p, 0, U * sizeof(int32_t), c->stream));
    {
        KScope ks(c, "feature_table");
        k_feature_table<<<grid_for(c, K), 256, 0, c->stream>>>(
            K, flag, rank, x, T1, T2, table.as<int32_t>(), tf.as<float>(), U);
    }
    {
        KScope ks(c, "feature_count");
        k_count<<<grid_for(c, K), 256, 0, c->stream>>>(K, id, count.as<int32_t>());
    }
    return U;
}

void launch_gather_f32(mrsim_ctx *c, int64_t K, const int32_t *perm, const float *in,
                       float *out) {
    KScope ks(c, "gather");
    k_gather<float><<<grid_for(c, K), 256, 0, c->stream>>>(K, perm, in, out);
}

}  // namespace mrsim
