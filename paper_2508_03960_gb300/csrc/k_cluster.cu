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
// id; SSEs are compared as exact rationals on the host):
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

// Device work area of the split in progress.
struct ClWork {
    double cen[6];                // centres of side 0 and side 1, feature units
    unsigned long long dmax[2];   // farthest-member searches: largest distance
    int32_t umin[2];              // ... and the smallest key id at it
    ClStats st[2];
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

// Sums of each side of the split of cluster c under the centres in w->cen.
__global__ void __launch_bounds__(kClThreads) k_cl_assign(int64_t U, const int32_t *lab, int32_t c,
                                                          const int32_t *tx, const int32_t *wt,
                                                          ClWork *w) {
    __shared__ double cen[6];
    __shared__ ClAcc part[kClThreads / 32][2];
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
}

// Largest distance of a member of cluster c to the centre in w->cen[0..2].
__global__ void k_cl_far_mean(int64_t U, const int32_t *lab, int32_t c, const int32_t *tx,
                              ClWork *w) {
    unsigned long long best = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U;
         u += (int64_t)gridDim.x * blockDim.x) {
        if (lab[u] != c) continue;
        const double d = cl_dist(tx[u], tx[U + u], tx[2 * U + u], w->cen);
        best = max(best, (unsigned long long)__double_as_longlong(d));  // d >= 0
    }
    for (int off = 16; off > 0; off >>= 1)
        best = max(best, __shfl_down_sync(0xffffffffu, best, off));
    if ((threadIdx.x & 31) == 0 && best) atomicMax(&w->dmax[0], best);
}

__global__ void k_cl_pick_mean(int64_t U, const int32_t *lab, int32_t c, const int32_t *tx,
                               ClWork *w) {
    const unsigned long long dm = w->dmax[0];
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U;
         u += (int64_t)gridDim.x * blockDim.x) {
        if (lab[u] != c) continue;
        const double d = cl_dist(tx[u], tx[U + u], tx[2 * U + u], w->cen);
        if ((unsigned long long)__double_as_longlong(d) == dm) atomicMin(&w->umin[0], (int32_t)u);
    }
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

// Largest distance of a member of cluster c to member w->umin[0].
__global__ void k_cl_far_point(int64_t U, const int32_t *lab, int32_t c, const int32_t *tx,
                               ClWork *w) {
    const int32_t a = w->umin[0];
    unsigned long long best = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U;
         u += (int64_t)gridDim.x * blockDim.x) {
        if (lab[u] != c) continue;
        best = max(best, (unsigned long long)cl_dist_int(tx, U, u, a));
    }
    for (int off = 16; off > 0; off >>= 1)
        best = max(best, __shfl_down_sync(0xffffffffu, best, off));
    if ((threadIdx.x & 31) == 0 && best) atomicMax(&w->dmax[1], best);
}

__global__ void k_cl_pick_point(int64_t U, const int32_t *lab, int32_t c, const int32_t *tx,
                                ClWork *w) {
    const int32_t a = w->umin[0];
    const unsigned long long dm = w->dmax[1];
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U;
         u += (int64_t)gridDim.x * blockDim.x) {
        if (lab[u] != c) continue;
        if ((unsigned long long)cl_dist_int(tx, U, u, a) == dm)
            atomicMin(&w->umin[1], (int32_t)u);
    }
}

// centres of the first 2-means pass: the two members found above
__global__ void k_cl_seed(int64_t U, const int32_t *tx, ClWork *w) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int32_t a = w->umin[0], b = w->umin[1];
    for (int i = 0; i < 3; ++i) {
        w->cen[i] = (double)tx[i * U + a];
        w->cen[3 + i] = (double)tx[i * U + b];
    }
}

// members of cluster c on side 1 under w->cen move to cluster id_new
__global__ void k_cl_label(int64_t U, int32_t *lab, int32_t c, int32_t id_new, const int32_t *tx,
                           const ClWork *w) {
    __shared__ double cen[6];
    if (threadIdx.x < 6) cen[threadIdx.x] = w->cen[threadIdx.x];
    __syncthreads();
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < U;
         u += (int64_t)gridDim.x * blockDim.x) {
        if (lab[u] != c) continue;
        if (cl_side(tx[u], tx[U + u], tx[2 * U + u], cen)) lab[u] = id_new;
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

using u128 = unsigned __int128;

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

// SSE_a > SSE_b, i.e. N_a / n_a > N_b / n_b, exactly
bool sse_greater(const Cluster &a, const Cluster &b) { return a.N * b.n > b.N * a.n; }

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
        k_cl_quant<<<grid(c, K), kClThreads, 0, c->stream>>>(
            K, ph->T1.as<float>(), ph->T2.as<float>(), ph->dB0.as<float>(), scale[0], scale[1],
            scale[2], xq.as<int32_t>(), err);
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
    const int32_t *ptx = tx.as<int32_t>(), *pwt = wt.as<int32_t>();
    int32_t *plab = lab.as<int32_t>();
    const int gU = grid(c, U);
    ClStats hs[2];

    // sums of one pass of cluster cl under the device centres
    auto stats_pass = [&](int32_t cl, double *cen_back) {
        MRSIM_CUDA(cudaMemsetAsync(&w->st, 0, sizeof(w->st), c->stream));
        {
            KScope ks(c, "cluster_assign");
            k_cl_assign<<<gU, kClThreads, 0, c->stream>>>(U, plab, cl, ptx, pwt, w);
        }
        MRSIM_CUDA(cudaMemcpyAsync(hs, &w->st, sizeof(hs), cudaMemcpyDeviceToHost, c->stream));
        if (cen_back)
            MRSIM_CUDA(cudaMemcpyAsync(cen_back, &w->cen, 6 * sizeof(double),
                                       cudaMemcpyDeviceToHost, c->stream));
        sync(c);
    };
    auto put_cen = [&](const double *cen) {
        MRSIM_CUDA(cudaMemcpyAsync(&w->cen, cen, 6 * sizeof(double), cudaMemcpyHostToDevice,
                                   c->stream));
    };

    // cluster 0: every key (equal centres put every member on side 0)
    std::vector<Cluster> cl(1);
    {
        const double zero[6] = {0, 0, 0, 0, 0, 0};
        put_cen(zero);
        stats_pass(0, nullptr);
        cl[0].set(hs[0]);
    }
    while ((int)cl.size() < n_clusters) {
        int best = -1;
        for (int i = 0; i < (int)cl.size(); ++i)
            if (cl[i].N > 0 && (best < 0 || sse_greater(cl[i], cl[best]))) best = i;
        if (best < 0) break;  // every cluster is one distinct value
        const int32_t cid = best, nid = (int32_t)cl.size();
        // initial centres: farthest member from the mean, then farthest from it
        const double mu[6] = {cl[best].mu[0], cl[best].mu[1], cl[best].mu[2], 0, 0, 0};
        put_cen(mu);
        MRSIM_CUDA(cudaMemsetAsync(&w->dmax, 0, sizeof(w->dmax), c->stream));
        MRSIM_CUDA(cudaMemsetAsync(&w->umin, 0x7f, sizeof(w->umin), c->stream));
        {
            KScope ks(c, "cluster_farthest");
            k_cl_far_mean<<<gU, kClThreads, 0, c->stream>>>(U, plab, cid, ptx, w);
            k_cl_pick_mean<<<gU, kClThreads, 0, c->stream>>>(U, plab, cid, ptx, w);
            k_cl_far_point<<<gU, kClThreads, 0, c->stream>>>(U, plab, cid, ptx, w);
            k_cl_pick_point<<<gU, kClThreads, 0, c->stream>>>(U, plab, cid, ptx, w);
            k_cl_seed<<<1, 32, 0, c->stream>>>(U, ptx, w);
        }
        double cur[6] = {0, 0, 0, 0, 0, 0};
        double kept_cen[6] = {0, 0, 0, 0, 0, 0};
        ClStats kept[2] = {};
        bool have = false;
        for (int it = 0; it < max_iter; ++it) {
            if (it > 0) put_cen(cur);
            stats_pass(cid, it == 0 ? cur : nullptr);
            if (hs[0].n == 0 || hs[1].n == 0) break;
            std::copy(cur, cur + 6, kept_cen);
            kept[0] = hs[0];
            kept[1] = hs[1];
            have = true;
            double m[6];
            for (int s = 0; s < 2; ++s)
                for (int i = 0; i < 3; ++i)
                    m[3 * s + i] = (double)(int64_t)hs[s].sx[i] / (double)hs[s].n;
            if (std::equal(m, m + 6, cur)) break;
            std::copy(m, m + 6, cur);
        }
        if (!have) fail(MRSIM_ECUDA, "clustering: the first 2-means pass left a side empty");
        put_cen(kept_cen);
        {
            KScope ks(c, "cluster_label");
            k_cl_label<<<gU, kClThreads, 0, c->stream>>>(U, plab, cid, nid, ptx, w);
        }
        cl[best].set(kept[0]);
        cl.emplace_back();
        cl.back().set(kept[1]);
    }
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
