// C ABI of libmrsim (declared in include/mrsim.h) and the host planner that
// turns a classified sequence into kernel launches.
#include <algorithm>
#include <array>
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <functional>
#include <thread>
#include <exception>
#include <map>
#include <new>
#include <unordered_map>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

namespace mrsim {

[[noreturn]] void fail(int code, const std::string &msg) { throw Error{code, msg}; }

void cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        fail(MRSIM_ENOMEM, std::string("out of device memory in ") + what);
    }
    fail(MRSIM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// the context whose entry point is running on this thread (its pool serves
// dalloc); set by the entry points' guard
thread_local mrsim_ctx *tl_ctx = nullptr;

CtxScope::CtxScope(mrsim_ctx *c) : prev(tl_ctx) { tl_ctx = c; }
CtxScope::~CtxScope() { tl_ctx = prev; }

DBuf dalloc(size_t bytes) {
    DBuf d;
    if (bytes == 0) return d;
    const mrsim_ctx *c = tl_ctx;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (c && c->pool && cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;  // unknown: keep out of the stream order
    }
    if (c && c->pool && cs == cudaStreamCaptureStatusNone) {
        const size_t want = (bytes + 255) / 256 * 256;
        cudaError_t e = cudaMallocFromPoolAsync(&d.p, want, c->pool->pool, c->stream);
        if (e != cudaSuccess) {  // hand the pool's idle reserve back, then once more
            cudaGetLastError();
            MRSIM_CUDA(cudaStreamSynchronize(c->stream));
            cudaMemPoolTrimTo(c->pool->pool, 0);
            e = cudaMallocFromPoolAsync(&d.p, want, c->pool->pool, c->stream);
        }
        if (e == cudaSuccess && ((uintptr_t)d.p & 255) == 0) {
            d.bytes = bytes;
            d.pool = c->pool;
            return d;
        }
        cudaGetLastError();
        if (e == cudaSuccess) {  // 256-byte alignment is what the kernels assume
            cudaFreeAsync(d.p, c->stream);
        } else {
            d.p = nullptr;
            fail(MRSIM_ENOMEM, "pool allocation of " + std::to_string(bytes) + " bytes failed");
        }
        d.p = nullptr;
    }
    cudaError_t e = cudaMalloc(&d.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        d.p = nullptr;
        fail(MRSIM_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    d.bytes = bytes;
    return d;
}

void *scratch(mrsim_ctx *c, int slot, size_t bytes) {
    DBuf &b = c->scratch[slot];
    if (b.bytes < bytes) {
        MRSIM_CUDA(cudaStreamSynchronize(c->stream));
        b.reset();
        b = dalloc(std::max<size_t>(bytes, 256));
    }
    return b.p;
}

void upload(mrsim_ctx *c, void *dst, const void *src, size_t bytes) {
    if (bytes == 0) return;
    MRSIM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
}

void sync(mrsim_ctx *c) {
    MRSIM_CUDA(cudaGetLastError());
    MRSIM_CUDA(cudaStreamSynchronize(c->stream));
    prof_flush(c);
}

KScope::KScope(mrsim_ctx *ctx, const char *name) : c(ctx) {
    ++c->launches;
    // a named NVTX range around the launch (profilers can select passes by it)
    nvtxRangePushA(name);
    if (!c->prof_on) return;
    for (size_t i = 0; i < c->prof_names.size(); ++i)
        if (c->prof_names[i] == name) { id = (int)i; break; }
    if (id < 0) {
        id = (int)c->prof_names.size();
        c->prof_names.push_back(name);
        c->prof_count.push_back(0);
        c->prof_ms.push_back(0.0);
    }
    for (cudaEvent_t *e : {&a, &b}) {
        if (!c->ev_pool.empty()) {
            *e = c->ev_pool.back();
            c->ev_pool.pop_back();
        } else if (cudaEventCreate(e) != cudaSuccess) {
            *e = nullptr;
        }
    }
    if (a) cudaEventRecord(a, c->stream);
}

KScope::~KScope() {
    nvtxRangePop();
    if (id < 0 || !a || !b) return;
    cudaEventRecord(b, c->stream);
    c->prof_pending.push_back({id, a, b});
}

void prof_flush(mrsim_ctx *c) {
    for (auto &p : c->prof_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            c->prof_ms[p.id] += ms;
            c->prof_count[p.id] += 1;
        }
        c->ev_pool.push_back(p.a);
        c->ev_pool.push_back(p.b);
    }
    c->prof_pending.clear();
}

namespace {

std::atomic<uint64_t> g_uid{1};

// isochromats per fused-kernel chunk at the context's tuning
inline int64_t kFusedChunk(const mrsim_ctx *c) { return 256LL * c->tune[MRSIM_TUNE_FUSED_NI]; }

inline AdvF make_adv_f(const double mom[3], double tau) {
    auto sp = [](double v, float &hi, float &lo) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    };
    AdvF a;
    sp(kGammaBar * mom[0], a.kx_hi, a.kx_lo);
    sp(kGammaBar * mom[1], a.ky_hi, a.ky_lo);
    sp(kGammaBar * mom[2], a.kz_hi, a.kz_lo);
    sp(tau, a.tau_hi, a.tau_lo);
    return a;
}
inline AdvD make_adv_d(const double mom[3], double tau) {
    return AdvD{kGammaBar * mom[0], kGammaBar * mom[1], kGammaBar * mom[2], tau};
}

template <typename R>
struct AdvOf;
template <>
struct AdvOf<float> {
    using T = AdvF;
    static AdvF make(const double m[3], double t) { return make_adv_f(m, t); }
};
template <>
struct AdvOf<double> {
    using T = AdvD;
    static AdvD make(const double m[3], double t) { return make_adv_d(m, t); }
};

// Bucket key of the with-RF subsequence [b, e): its length and the bit
// patterns of its first, middle and last segments.  It only picks candidate
// contents, which are then compared in full (same_run).
uint64_t run_key(const mrsim_seq *s, int64_t b, int64_t e) {
    uint64_t h = 0x243f6a8885a308d3ull ^ (uint64_t)(e - b);
    auto mix = [&](const void *p, size_t n) {
        uint64_t v = 0;
        std::memcpy(&v, p, n);
        h = (h ^ v) * 0x9e3779b97f4a7c15ull;
        h ^= h >> 29;
    };
    for (int64_t j : {b, b + (e - b) / 2, e - 1}) {
        mix(&s->dt[j], 8);
        mix(&s->rep[j], 4);
        mix(&s->b1re[j], 4);
        mix(&s->b1im[j], 4);
        mix(&s->gx[j], 4);
        mix(&s->gy[j], 4);
        mix(&s->gz[j], 4);
    }
    return h;
}

// bitwise equality of the segments [a, a + n) and [b, b + n)
bool same_run(const mrsim_seq *s, int64_t a, int64_t b, int64_t n) {
    return std::memcmp(&s->dt[a], &s->dt[b], n * sizeof(double)) == 0 &&
           std::memcmp(&s->rep[a], &s->rep[b], n * sizeof(int32_t)) == 0 &&
           std::memcmp(&s->b1re[a], &s->b1re[b], n * sizeof(float)) == 0 &&
           std::memcmp(&s->b1im[a], &s->b1im[b], n * sizeof(float)) == 0 &&
           std::memcmp(&s->gx[a], &s->gx[b], n * sizeof(float)) == 0 &&
           std::memcmp(&s->gy[a], &s->gy[b], n * sizeof(float)) == 0 &&
           std::memcmp(&s->gz[a], &s->gz[b], n * sizeof(float)) == 0;
}

__global__ void k_finite(int64_t n, const float *v, int *err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) atomicOr(err, 1);
}

__device__ __forceinline__ bool finite_f(float v) { return fabsf(v) <= FLT_MAX; }
__device__ __forceinline__ bool finite4(float4 v) {
    return finite_f(v.x) & finite_f(v.y) & finite_f(v.z) & finite_f(v.w);
}
__device__ __forceinline__ bool positive4(float4 v) {
    return (v.x > 0.0f) & (v.y > 0.0f) & (v.z > 0.0f) & (v.w > 0.0f);
}

// Value checks of a phantom (every array 16-byte aligned): non-finite values,
// T1 or T2 not > 0 (NaN fails, +inf passes).  Four isochromats per thread and
// step with 16-byte loads, then the tail; M_init is checked as one flat array.
__global__ void k_validate(int64_t K, const float *x, const float *y, const float *z,
                           const float *T1, const float *T2, const float *dB0, const float *M0,
                           const float *b1, const float *Mi, int *err) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    auto v4 = [](const float *p, int64_t q) { return __ldg(reinterpret_cast<const float4 *>(p) + q); };
    bool ok = true;
    const int64_t K4 = K / 4;
    for (int64_t q = tid; q < K4; q += stride) {
        ok &= finite4(v4(x, q)) & finite4(v4(y, q)) & finite4(v4(z, q)) & finite4(v4(dB0, q)) &
              finite4(v4(M0, q)) & positive4(v4(T1, q)) & positive4(v4(T2, q));
        if (b1) ok &= finite4(v4(b1, q));
    }
    for (int64_t k = 4 * K4 + tid; k < K; k += stride) {
        ok &= finite_f(x[k]) & finite_f(y[k]) & finite_f(z[k]) & finite_f(dB0[k]) &
              finite_f(M0[k]) & (T1[k] > 0.0f) & (T2[k] > 0.0f);
        if (b1) ok &= finite_f(b1[k]);
    }
    if (Mi) {
        const int64_t n = 3 * K, n4 = n / 4;
        for (int64_t q = tid; q < n4; q += stride) ok &= finite4(v4(Mi, q));
        for (int64_t k = 4 * n4 + tid; k < n; k += stride) ok &= finite_f(Mi[k]);
    }
    if (!ok) atomicOr(err, 1);
}

static_assert(G_XY == MRSIM_G_XY && G_XZ == MRSIM_G_XZ && G_YZ == MRSIM_G_YZ,
              "two-axis type numbers");

// Host part of a sequence: subsequence split (Fig. 1), gradient types
// (Sec. 2.4; two_axis: exactly two nonzero axes give G_XY / G_XZ / G_YZ instead
// of G_GENERAL), sample offsets and with-RF content ids.  Needs no device.
// Runs f(0) .. f(n - 1) split over up to `threads` host threads (f must not
// throw); shares whose thread cannot be started run on the calling thread.
template <class F>
void host_parallel(int n, int threads, const F &f) {
    threads = std::max(1, std::min(threads, n));
    auto share = [&](int w) {
        for (int i = (int)((int64_t)n * w / threads); i < (int)((int64_t)n * (w + 1) / threads); ++i)
            f(i);
    };
    std::vector<std::thread> th;
    std::vector<int> inline_share;
    for (int w = 1; w < threads; ++w) {
        try {
            th.emplace_back(share, w);
        } catch (...) {
            inline_share.push_back(w);
        }
    }
    share(0);
    for (int w : inline_share) share(w);
    for (auto &t : th) t.join();
}

// The caller's segment arrays, copied into the sequence.  Long sequences copy
// their eight arrays on eight host threads (one core copies at a fraction of
// the host's memory bandwidth); a thread that cannot be started leaves its
// copy to the calling thread, and a failed copy is rethrown here.
void copy_segments(mrsim_seq *s, int64_t n, const double *dt, const int32_t *rep,
                   const float *b1re, const float *b1im, const float *gx, const float *gy,
                   const float *gz, const uint8_t *adc) {
    s->n_seg = n;
    std::function<void()> jobs[8] = {
        [&] { s->dt.assign(dt, dt + n); },     [&] { s->rep.assign(rep, rep + n); },
        [&] { s->b1re.assign(b1re, b1re + n); }, [&] { s->b1im.assign(b1im, b1im + n); },
        [&] { s->gx.assign(gx, gx + n); },     [&] { s->gy.assign(gy, gy + n); },
        [&] { s->gz.assign(gz, gz + n); },     [&] { s->adc.assign(adc, adc + n); }};
    std::exception_ptr ep[8];
    auto run = [&](int i) {
        try {
            jobs[i]();
        } catch (...) {
            ep[i] = std::current_exception();
        }
    };
    std::vector<std::thread> th;
    bool inline_job[8] = {};
    if (n >= (1 << 16)) {
        th.reserve(7);
        for (int i = 1; i < 8; ++i) {
            try {
                th.emplace_back(run, i);
            } catch (...) {
                inline_job[i] = true;
            }
        }
    } else {
        for (int i = 1; i < 8; ++i) inline_job[i] = true;
    }
    run(0);
    for (int i = 1; i < 8; ++i)
        if (inline_job[i]) run(i);
    for (auto &t : th) t.join();
    for (auto &e : ep)
        if (e) std::rethrow_exception(e);
}

// first index in [j, n) whose class byte differs from v (n if none)
int64_t class_run_end(const uint8_t *cl, int64_t j, int64_t n, uint8_t v) {
    const uint64_t pat = 0x0101010101010101ull * v;
    for (; j + 8 <= n; j += 8) {
        uint64_t w;
        std::memcpy(&w, cl + j, 8);
        if (w != pat) break;
    }
    while (j < n && cl[j] == v) ++j;
    return j;
}

void classify_sequence(mrsim_seq *s, bool two_axis) {
    const int64_t n = s->n_seg;
    // the class of every segment, and whether any segment is invalid or has
    // RF and ADC at once (branch-free passes over one or two arrays each, so
    // that they vectorise)
    auto finite = [](float v) { return std::fabs(v) <= FLT_MAX; };
    const double *dt = s->dt.data();
    const int32_t *rep = s->rep.data();
    const float *bre = s->b1re.data(), *bim = s->b1im.data();
    const float *gx = s->gx.data(), *gy = s->gy.data(), *gz = s->gz.data();
    const uint8_t *adc = s->adc.data();
    std::vector<uint8_t> cl(n);
    int bad = 0;
    for (int64_t j = 0; j < n; ++j) bad |= !(dt[j] > 0.0) | !(dt[j] <= DBL_MAX) | (rep[j] < 1);
    for (int64_t j = 0; j < n; ++j) bad |= !finite(gx[j]) | !finite(gy[j]) | !finite(gz[j]);
    static_assert(SUB_RF == 0 && SUB_ADC == 1 && SUB_RELAX == 2, "class codes");
    for (int64_t j = 0; j < n; ++j) {
        const int rf = (bre[j] != 0.0f) | (bim[j] != 0.0f);
        const int a = adc[j] != 0;
        bad |= !finite(bre[j]) | !finite(bim[j]) | (rf & a);
        cl[j] = (uint8_t)(rf ? SUB_RF : SUB_RELAX - a);
    }
    if (bad) {  // name the first offending segment, invalid before RF with ADC
        for (int64_t j = 0; j < n; ++j) {
            if (!(std::isfinite(s->dt[j]) && s->dt[j] > 0.0) || s->rep[j] < 1 ||
                !std::isfinite(s->b1re[j]) || !std::isfinite(s->b1im[j]) ||
                !std::isfinite(s->gx[j]) || !std::isfinite(s->gy[j]) || !std::isfinite(s->gz[j]))
                fail(MRSIM_EINVAL, "invalid segment " + std::to_string(j));
            if ((s->b1re[j] != 0.0f || s->b1im[j] != 0.0f) && s->adc[j])
                fail(MRSIM_EUNSUPPORTED, "RF and ADC active in segment " + std::to_string(j));
        }
    }
    // split into maximal runs of one class (Fig. 1)
    for (int64_t j = 0; j < n;) {
        Subseq q;
        q.type = cl[j];
        q.seg_begin = j;
        j = class_run_end(cl.data(), j + 1, n, cl[j]);
        q.seg_end = j;
        s->sub.push_back(q);
    }
    // with-RF runs: bucket keys, and (on host threads when there is much to
    // compare) whether each run repeats the first run of its bucket bit for
    // bit, the common case of a sequence repeating a few pulses; the ordered
    // content numbering below then compares only when that fails
    std::vector<int> rf_sub;
    for (size_t i = 0; i < s->sub.size(); ++i)
        if (s->sub[i].type == SUB_RF) rf_sub.push_back((int)i);
    const int n_rf = (int)rf_sub.size();
    std::vector<uint64_t> rf_key(n_rf);
    std::vector<int> rf_cand(n_rf);
    std::vector<uint8_t> rf_same(n_rf, 0);
    {
        std::unordered_map<uint64_t, int> first_of;
        int64_t cmp_segs = 0;
        for (int t = 0; t < n_rf; ++t) {
            const Subseq &q = s->sub[rf_sub[t]];
            rf_key[t] = run_key(s, q.seg_begin, q.seg_end);
            rf_cand[t] = first_of.emplace(rf_key[t], rf_sub[t]).first->second;
            if (rf_cand[t] != rf_sub[t]) cmp_segs += q.seg_end - q.seg_begin;
        }
        auto compare = [&](int t) {
            const Subseq &q = s->sub[rf_sub[t]], &r = s->sub[rf_cand[t]];
            const int64_t len = q.seg_end - q.seg_begin;
            rf_same[t] = rf_cand[t] != rf_sub[t] && r.seg_end - r.seg_begin == len &&
                         same_run(s, r.seg_begin, q.seg_begin, len);
        };
        host_parallel(n_rf, cmp_segs >= (1 << 16) ? 8 : 1, compare);
    }
    int64_t smp = 0;
    std::unordered_map<uint64_t, std::vector<int>> by_hash;
    for (size_t i = 0, t = 0; i < s->sub.size(); ++i) {
        Subseq &q = s->sub[i];
        int first = (int)i;  // the subsequence whose segments this one repeats bit for bit
        if (q.type == SUB_RF) {
            const uint64_t h = rf_key[t];
            const int64_t len = q.seg_end - q.seg_begin;
            int found = rf_same[t] ? s->sub[rf_cand[t]].content : -1;
            ++t;
            if (found < 0) {
                for (int cid : by_hash[h]) {
                    const Subseq &r = s->sub[s->content_first[cid]];
                    if (r.seg_end - r.seg_begin == len &&
                        same_run(s, r.seg_begin, q.seg_begin, len)) {
                        found = cid;
                        break;
                    }
                }
            }
            if (found < 0) {
                found = s->n_content++;
                s->content_first.push_back((int64_t)i);
                s->content_count.push_back(0);
                by_hash[h].push_back(found);
            }
            q.content = found;
            s->content_count[found]++;
            first = (int)s->content_first[found];
        }
        if (first != (int)i) {  // same segments: same type, duration and moments
            const Subseq &r = s->sub[first];
            q.gtype = r.gtype;
            q.dur = r.dur;
            for (int a = 0; a < 3; ++a) q.mom[a] = r.mom[a];
            q.n_samples = r.n_samples;
        } else {
            bool ax = false, ay = false, az = false;
            for (int64_t j = q.seg_begin; j < q.seg_end; ++j) {
                ax |= s->gx[j] != 0.0f;
                ay |= s->gy[j] != 0.0f;
                az |= s->gz[j] != 0.0f;
                const double d = s->dt[j] * s->rep[j];
                q.dur += d;
                q.mom[0] += (double)s->gx[j] * d;
                q.mom[1] += (double)s->gy[j] * d;
                q.mom[2] += (double)s->gz[j] * d;
                if (s->adc[j]) q.n_samples += s->rep[j];
            }
            const int cnt = (int)ax + (int)ay + (int)az;
            q.gtype = cnt == 0   ? G_NONE
                      : cnt == 1 ? (ax ? G_X : ay ? G_Y : G_Z)
                      : cnt == 2 && two_axis ? (!az ? G_XY : !ay ? G_XZ : G_YZ)
                                 : G_GENERAL;
        }
        q.sample0 = smp;
        smp += q.n_samples;
    }
    s->n_samples = smp;
}

void build_sequence(mrsim_ctx *c, mrsim_seq *s) {
    classify_sequence(s, c->tune[MRSIM_TUNE_TWO_AXIS] != 0);
    // device waveforms of every distinct with-RF content
    mrsim_seq *dev = s;
    s->rf_f.resize(s->n_content);
    s->rf_d.resize(s->n_content);
    dev->rf_off.resize(s->n_content);
    s->content_steps.assign(s->n_content, 0);
    for (int cid = 0; cid < s->n_content; ++cid) {
        const Subseq &q = s->sub[s->content_first[cid]];
        const int64_t len = q.seg_end - q.seg_begin;
        std::vector<RFSegF> f(len);
        std::vector<RFSegD> d(len);
        std::vector<int64_t> off(len + 1, 0);
        for (int64_t t = 0; t < len; ++t) {
            const int64_t j = q.seg_begin + t;
            const double dt = s->dt[j];
            d[t] = RFSegD{kGamma * s->b1re[j] * dt, kGamma * s->b1im[j] * dt, kGamma * s->gx[j] * dt,
                          kGamma * s->gy[j] * dt, kGamma * s->gz[j] * dt, kTwoPi * dt, dt,
                          (long long)s->rep[j]};
            f[t] = RFSegF{(float)d[t].are, (float)d[t].aim, (float)d[t].cx, (float)d[t].cy,
                          (float)d[t].cz, (float)d[t].cdw, (float)dt, s->rep[j]};
            off[t + 1] = off[t] + s->rep[j];
        }
        s->content_steps[cid] = off[len];
        s->rf_f[cid] = dalloc(len * sizeof(RFSegF));
        s->rf_d[cid] = dalloc(len * sizeof(RFSegD));
        dev->rf_off[cid] = dalloc((len + 1) * sizeof(int64_t));
        upload(c, s->rf_f[cid].p, f.data(), len * sizeof(RFSegF));
        upload(c, s->rf_d[cid].p, d.data(), len * sizeof(RFSegD));
        upload(c, dev->rf_off[cid].p, off.data(), (len + 1) * sizeof(int64_t));
    }
    // ADC segments and per-sample window-relative (tau, k)
    std::vector<ADCSegF> af;
    std::vector<ADCSegD> ad;
    const int64_t smp = s->n_samples;
    std::vector<GSampleF> gf(std::max<int64_t>(smp, 1));
    std::vector<GSampleD> gd(std::max<int64_t>(smp, 1));
    dev->adc_off.assign(s->sub.size(), -1);
    for (size_t i = 0; i < s->sub.size(); ++i) {
        const Subseq &q = s->sub[i];
        if (q.type != SUB_ADC) continue;
        dev->adc_off[i] = (int64_t)af.size();
        double tau = 0.0, m[3] = {0, 0, 0};
        int64_t si = q.sample0;
        const int ax = gtype_axis0(q.gtype), ax2 = gtype_axis1(q.gtype);
        for (int64_t j = q.seg_begin; j < q.seg_end; ++j) {
            const double dt = s->dt[j];
            const double g[3] = {(double)s->gx[j], (double)s->gy[j], (double)s->gz[j]};
            ADCSegD sd{kGammaBar * g[0] * dt, kGammaBar * g[1] * dt, kGammaBar * g[2] * dt, dt,
                       (long long)s->rep[j]};
            ad.push_back(sd);
            ADCSegF sf;
            auto sp = [](double v, float &hi, float &lo) { hi = (float)v; lo = (float)(v - (double)hi); };
            sp(sd.kx, sf.kx_hi, sf.kx_lo);
            sp(sd.ky, sf.ky_hi, sf.ky_lo);
            sp(sd.kz, sf.kz_hi, sf.kz_lo);
            sf.dt = (float)dt;
            sf.rep = s->rep[j];
            af.push_back(sf);
            if (s->adc[j]) {
                for (int32_t r = 0; r < s->rep[j]; ++r, ++si) {
                    const double ts = tau + (r + 1) * dt;
                    const double ks = ax >= 0 ? kGammaBar * (m[ax] + g[ax] * (r + 1) * dt) : 0.0;
                    const double ks2 =
                        ax2 >= 0 ? kGammaBar * (m[ax2] + g[ax2] * (r + 1) * dt) : 0.0;
                    gd[si] = GSampleD{ts, ks, ks2};
                    GSampleF f;
                    sp(ts, f.tau_hi, f.tau_lo);
                    sp(ks, f.k_hi, f.k_lo);
                    sp(ks2, f.k2_hi, f.k2_lo);
                    gf[si] = f;
                }
            }
            tau += dt * s->rep[j];
            for (int a = 0; a < 3; ++a) m[a] += g[a] * dt * s->rep[j];
        }
    }
    if (!af.empty()) {
        dev->adc_f = dalloc(af.size() * sizeof(ADCSegF));
        dev->adc_d = dalloc(ad.size() * sizeof(ADCSegD));
        upload(c, dev->adc_f.p, af.data(), af.size() * sizeof(ADCSegF));
        upload(c, dev->adc_d.p, ad.data(), ad.size() * sizeof(ADCSegD));
    }
    dev->gs_f = dalloc(gf.size() * sizeof(GSampleF));
    dev->gs_d = dalloc(gd.size() * sizeof(GSampleD));
    upload(c, dev->gs_f.p, gf.data(), gf.size() * sizeof(GSampleF));
    upload(c, dev->gs_d.p, gd.data(), gd.size() * sizeof(GSampleD));
    sync(c);
}

// element stride between the Mx, My and Mz planes of the state buffer: a
// multiple of 64 so that every plane starts 256-byte aligned (vector loads)
inline int64_t plane_stride(int64_t K) { return (K + 63) / 64 * 64; }

PlainState plain_state(const mrsim_phantom_t *ph, void *Mx, void *My, void *Mz) {
    return PlainState{ph->K, ph->x.as<float>(), ph->y.as<float>(), ph->z.as<float>(),
                      ph->T1.as<float>(), ph->T2.as<float>(), ph->dB0.as<float>(),
                      ph->M0.as<float>(), ph->has_b1 ? ph->b1.as<float>() : nullptr, Mx, My, Mz};
}

PlainState sorted_state(const mrsim_groups *g, void *Mx, void *My, void *Mz) {
    return PlainState{g->K, g->x.as<float>(), g->y.as<float>(), g->z.as<float>(),
                      g->T1.as<float>(), g->T2.as<float>(), g->dB0.as<float>(),
                      g->M0.as<float>(), g->has_b1 ? g->b1.as<float>() : nullptr, Mx, My, Mz};
}

// ---------------------------------------------------------------- plain ----
template <typename R>
void run_plain(mrsim_ctx *c, const mrsim_phantom_t *ph, const mrsim_seq *s, bool use_cache,
               double *d_signal, R *M) {
    const int64_t K = ph->K;
    const mrsim_seq &dev = *s;
    const int64_t Kp = plane_stride(K);
    PlainState st = plain_state(ph, M, M + Kp, M + 2 * Kp);
    st.fx = c->fx;
    launch_init_state<R>(c, st, ph->has_M_init ? ph->M_init.as<float>() : nullptr);
    std::vector<DBuf> cache(s->n_content);
    double mom[3] = {0, 0, 0}, tau = 0.0;
    using A = typename AdvOf<R>::T;
    const bool f64 = sizeof(R) == 8;
    for (size_t i = 0; i < s->sub.size(); ++i) {
        const Subseq &q = s->sub[i];
        const A adv = AdvOf<R>::make(mom, tau);
        if (q.type == SUB_RELAX) {
            for (int a = 0; a < 3; ++a) mom[a] += q.mom[a];
            tau += q.dur;
            continue;
        }
        if (q.type == SUB_RF) {
            const int cid = q.content;
            const void *segs = f64 ? s->rf_d[cid].p : s->rf_f[cid].p;
            const int nseg = (int)(q.seg_end - q.seg_begin);
            if (use_cache && s->content_count[cid] > 1) {
                if (!cache[cid].p) {
                    cache[cid] = dalloc(12 * (size_t)K * sizeof(R));
                    launch_plain_rf_affine<R>(c, st, segs, nseg, cache[cid].as<R>());
                }
                launch_apply_affine<R>(c, st, cache[cid].as<R>(), &adv);
            } else {
                launch_plain_rf<R>(c, st, segs, nseg, &adv, c->tune[MRSIM_TUNE_PLAIN_RF_NI]);
            }
            mom[0] = mom[1] = mom[2] = 0.0;
            tau = 0.0;
        } else {
            const void *segs = f64 ? (const void *)(dev.adc_d.as<ADCSegD>() + dev.adc_off[i])
                                   : (const void *)(dev.adc_f.as<ADCSegF>() + dev.adc_off[i]);
            // one launch per receive coil; the state is only read here
            for (int pass = 0; pass < std::max(ph->n_coils, 1); ++pass) {
                if (ph->n_coils > 0) {
                    st.coil_re = ph->coils.as<float>() + 2 * K * pass;
                    st.coil_im = st.coil_re + K;
                }
                launch_plain_adc<R>(c, st, segs, (int)(q.seg_end - q.seg_begin), q.n_samples,
                                    &adv, d_signal + 2 * (s->n_samples * pass + q.sample0),
                                    c->tune[MRSIM_TUNE_ADC_CTAS_PER_SM]);
            }
            for (int a = 0; a < 3; ++a) mom[a] += q.mom[a];
            tau += q.dur;
        }
    }
    const A adv = AdvOf<R>::make(mom, tau);
    launch_advance<R>(c, st, &adv);
    sync(c);
}

// -------------------------------------------------------------- grouped ----
// Host-side plan of one grouped simulation: combined-transition tables, block
// sums of every known with-ADC window, the event list of every span, the
// fallback subsequence after each span and the group-signal blocks.
template <typename R>
struct GPlan {
    int p = 0;          // primary (layout / group-factor) gradient type
    int64_t Gp = 0;     // its group count
    std::vector<std::pair<std::pair<int, int>, int64_t>> tabs;  // ((content, gtype), row)
    int64_t rows = 0;
    std::vector<GWin> wins;
    int64_t ablk_n = 0;
    std::vector<FEvent<R>> ev;
    std::vector<EvAdv> adv;
    struct Span { int64_t b, e; int fallback; };
    std::vector<Span> spans;
    std::vector<int4> blk;  // group-signal blocks (window, first sample, g0, g1)
    bool direct = false;    // factor table too large: advance fully per isochromat
    std::vector<std::array<double, 3>> kd;  // per event: gamma_bar * moment per axis
    bool ax = false;        // per-isochromat phasors from axis tables (FP32 only)
    std::vector<AxItem> ax_items;
    int64_t ax_n = 0;       // table entries of all events
    int ax_max = 0;         // longest table
    // cell form of the fused kernel (FP32): see CellArgs
    bool cell = false;
    bool otf = false;       // cell form with rows formed per thread (no row table)
    int cell_w = 0;         // 0: 4 isochromats per thread, 1: 8
    int free_bits = 0, r_axis = -1;
    CellForm form{};
    std::vector<CellKey> ckeys;  // distinct RF / END advances
    std::vector<CellEv> cev;     // the events in the cell form's record
};

template <typename R>
void plan_grouped(mrsim_ctx *c, const mrsim_seq *s, const mrsim_groups *g, GPlan<R> &P,
                  bool allow_cell = false) {
    // 1) combined transitions for every (content, gradient type) of a known with-RF
    std::map<std::pair<int, int>, int64_t> row_of;
    for (const Subseq &q : s->sub) {
        if (q.type != SUB_RF || q.gtype == G_GENERAL) continue;
        auto key = std::make_pair(q.content, q.gtype);
        if (!row_of.count(key)) {
            row_of[key] = P.rows;
            P.tabs.push_back({key, P.rows});
            P.rows += g->n_groups[q.gtype];
        }
    }
    if (P.rows * 12 > 0x7fffffffLL) fail(MRSIM_EUNSUPPORTED, "combined-transition table too large");
    // 2) block-sum storage per known with-ADC window
    std::vector<int64_t> win_off(s->sub.size(), -1);
    for (size_t i = 0; i < s->sub.size(); ++i) {
        const Subseq &q = s->sub[i];
        if (q.type != SUB_ADC || q.gtype == G_GENERAL || q.n_samples == 0) continue;
        win_off[i] = P.ablk_n;
        GWin w{q.gtype, (int)g->n_groups[q.gtype], P.ablk_n, q.sample0, (int)q.n_samples, 0,
               0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (q.seg_end - q.seg_begin == 1 && s->adc[q.seg_begin]) {
            const int64_t j = q.seg_begin;
            const double dt = s->dt[j];
            const float gs[3] = {s->gx[j], s->gy[j], s->gz[j]};
            const int a0 = gtype_axis0(q.gtype), a1 = gtype_axis1(q.gtype);
            const double dk = a0 >= 0 ? kGammaBar * (double)gs[a0] * dt : 0.0;
            const double dk2 = a1 >= 0 ? kGammaBar * (double)gs[a1] * dt : 0.0;
            w.uniform = 1;
            w.dt_hi = (float)dt;
            w.dt_lo = (float)(dt - (double)w.dt_hi);
            w.dk_hi = (float)dk;
            w.dk_lo = (float)(dk - (double)w.dk_hi);
            w.dk2_hi = (float)dk2;
            w.dk2_lo = (float)(dk2 - (double)w.dk2_hi);
        }
        P.wins.push_back(w);
        P.ablk_n += g->n_groups[q.gtype];
    }
    if (P.ablk_n > 0x7fffffffLL) fail(MRSIM_EUNSUPPORTED, "too many block sums");
    // 3) spans of known-type events; unknown types close the span (plain fallback)
    P.p = g->primary;
    P.Gp = g->n_groups[P.p];
    const int p = P.p;
    int64_t span_begin = 0;
    double mom[3] = {0, 0, 0}, tau = 0.0;
    auto make = [&](int kind, int gtype) {
        FEvent<R> e{};
        const int64_t prow = (int64_t)P.ev.size() * P.Gp;
        if (prow > 0x7fffffffLL) fail(MRSIM_EUNSUPPORTED, "too many events x groups");
        e.prow = (int)prow;
        double k[3];
        for (int a = 0; a < 3; ++a) k[a] = kGammaBar * mom[a];
        int mask = 0;
        const double kt[4] = {k[0], k[1], k[2], tau};
        for (int a = 0; a < 4; ++a) {
            // per-isochromat phase: the axes outside the primary type's
            if (a < 3 && !(gtype_axes(p) & (1 << a)) && k[a] != 0.0) mask |= 1 << a;
            if constexpr (sizeof(R) == 4) {
                e.k_hi[a] = (float)kt[a];
                e.k_lo[a] = (float)(kt[a] - (double)e.k_hi[a]);
            } else {
                e.k[a] = kt[a];
            }
        }
        e.op = ev_op(kind, mask, gtype);
        const int pa0 = gtype_axis0(p), pa1 = gtype_axis1(p);
        P.adv.push_back(EvAdv{pa0 >= 0 ? k[pa0] : 0.0, tau, pa1 >= 0 ? k[pa1] : 0.0});
        P.kd.push_back({k[0], k[1], k[2]});
        return e;
    };
    auto close_span = [&](int fallback) {
        P.ev.push_back(make(EV_END, G_NONE));
        P.spans.push_back({span_begin, (int64_t)P.ev.size(), fallback});
        span_begin = (int64_t)P.ev.size();
        mom[0] = mom[1] = mom[2] = 0.0;
        tau = 0.0;
    };
    for (size_t i = 0; i < s->sub.size(); ++i) {
        const Subseq &q = s->sub[i];
        if (q.type == SUB_RELAX) {
            for (int a = 0; a < 3; ++a) mom[a] += q.mom[a];
            tau += q.dur;
        } else if (q.type == SUB_RF && q.gtype != G_GENERAL) {
            FEvent<R> e = make(EV_RF, q.gtype);
            e.row = (int)row_of.at(std::make_pair(q.content, q.gtype));
            P.ev.push_back(e);
            mom[0] = mom[1] = mom[2] = 0.0;
            tau = 0.0;
        } else if (q.type == SUB_ADC && q.gtype != G_GENERAL) {
            if (q.n_samples > 0) {
                FEvent<R> e = make(EV_ADC, q.gtype);
                e.win = (int)win_off[i];
                P.ev.push_back(e);
            }
            for (int a = 0; a < 3; ++a) mom[a] += q.mom[a];
            tau += q.dur;
        } else {
            close_span((int)i);  // state now at the start of the unclassified subsequence
            if (q.type == SUB_ADC) {
                for (int a = 0; a < 3; ++a) mom[a] += q.mom[a];
                tau += q.dur;
            }
        }
    }
    close_span(-1);
    // the factor table has n_events x G_primary entries: with nearly one group
    // per isochromat it would outgrow the state itself, so advance directly
    P.direct = (int64_t)P.ev.size() * P.Gp > (int64_t)1 << 26 || P.Gp * 4 > g->K;
    if (P.direct)
        for (auto &e : P.ev) e.prow = 0;
    if constexpr (sizeof(R) == 4) {
        // cell form (see CellArgs): every RF type and every with-ADC type must
        // be constant inside a cell (primary, secondary or no-grads)
        // (reproducible sums: 4 per thread, the width of the receive-coil
        // kernels, so that a unit coil gives the same bits as none)
        const int ni = c->fx > 0.0 && c->tune[MRSIM_TUNE_CELL_NI] != 0
                           ? 4 : c->tune[MRSIM_TUNE_CELL_NI];
        P.cell_w = ni == 8 ? 1 : 0;
        const int r = g->secondary;
        P.cell = allow_cell && ni != 0 && !P.direct && g->ax_ok && p >= G_X && p <= G_Z &&
                 g->n_cell_thr[P.cell_w] > 0 && g->n_cell_thr[0] > 0 && g->n_cells > 0;
        P.r_axis = (r >= G_X && r <= G_Z) ? r - 1 : -1;
        P.free_bits = 7 & ~(1 << (p - 1)) & ~(P.r_axis >= 0 ? 1 << P.r_axis : 0);
        const int rbit = P.r_axis >= 0 ? 1 << P.r_axis : 0;
        auto const_in_cell = [&](int gt) {
            return gt == p || gt == r || (gt == G_NONE && g->built[G_NONE]);
        };
        P.form = CellForm{ni, __builtin_popcount(P.free_bits), false, false, false};
        for (size_t i = 0; P.cell && i < P.ev.size(); ++i) {
            const int kind = ev_kind(P.ev[i].op), mask = ev_mask(P.ev[i].op);
            if (kind != EV_END && !const_in_cell(ev_gtype(P.ev[i].op))) P.cell = false;
            if (kind != EV_ADC) P.form.rfq |= (mask & P.free_bits) != 0;
            if (kind == EV_ADC) {
                P.form.adq |= (mask & P.free_bits) != 0;
                P.form.rb |= (mask & rbit) != 0;
            }
        }
        // FP32 factor-table runs take the per-isochromat phasor of every axis in
        // an event's mask from a table over that axis' distinct positions; the
        // cell form applies the same phasors to every event of a kind, so it
        // needs the tables of all free axes (and the secondary axis for with-ADC
        // windows) wherever the form applies them
        auto axis_tables = [&](bool cell) {
            P.ax_items.clear();
            P.ax_n = 0;
            P.ax_max = 0;
            for (size_t i = 0; i < P.ev.size(); ++i) {
                const int kind = ev_kind(P.ev[i].op);
                int need = ev_mask(P.ev[i].op);
                if (cell) {
                    if (kind != EV_ADC && P.form.rfq) need |= P.free_bits;
                    if (kind == EV_ADC && P.form.adq) need |= P.free_bits;
                    if (kind == EV_ADC && P.form.rb) need |= rbit;
                }
                for (int a = 0; a < 3; ++a) {
                    P.ev[i].q[a] = 0;
                    if (!(need & (1 << a))) continue;
                    P.ev[i].q[a] = (int)P.ax_n;
                    P.ax_items.push_back(AxItem{P.kd[i][a], g->ax_val[a].as<float>(),
                                                (int)g->n_ax[a], 0, P.ax_n});
                    P.ax_n += g->n_ax[a];
                    P.ax_max = std::max<int>(P.ax_max, (int)g->n_ax[a]);
                }
            }
            P.ax = P.ax_n <= ((int64_t)1 << 24);
        };
        if (!P.direct && g->ax_ok) {
            axis_tables(P.cell);
            if (P.cell && !P.ax) {
                P.cell = false;
                axis_tables(false);
            }
        }
        if (P.cell) {
            // one key per distinct (transition rows, primary and secondary
            // moments, duration) of an RF or END event: the free-axis moment
            // stays per isochromat.  Moments and durations equal to 1e-12
            // relative share a key: sequences built on an absolute time grid
            // give one repeated interval durations that differ by ~1e-15 s,
            // eight orders of magnitude below what the FP32 factors resolve
            auto near = [](double u, double v) {
                return std::fabs(u - v) <= 1e-12 * std::max(std::fabs(u), std::fabs(v));
            };
            int fa[2] = {-1, -1}, nfa = 0;
            for (int a = 0; a < 3; ++a)
                if (P.free_bits & (1 << a)) fa[nfa++] = a;
            // combined rows: 0 automatic, 1 a table when it fits 1 GiB, 2 per thread
            const int rows_mode = c->tune[MRSIM_TUNE_CELL_ROWS];
            P.otf = rows_mode == 2;
            P.cev.resize(P.ev.size());
            for (size_t i = 0; i < P.ev.size() && P.cell; ++i) {
                const FEvent<R> &e = P.ev[i];
                const int kind = ev_kind(e.op);
                CellEv &ce = P.cev[i];
                ce = CellEv{};
                ce.qf[0] = fa[0] >= 0 ? e.q[fa[0]] : 0;
                ce.qf[1] = fa[1] >= 0 ? e.q[fa[1]] : 0;
                ce.qr = P.r_axis >= 0 ? e.q[P.r_axis] : 0;
                if (kind == EV_ADC) {
                    ce.kind = ev_gtype(e.op) == p ? CE_ADC : CE_ADC_OTHER;
                    ce.row = e.prow;
                    ce.win = e.win;
                    ce.gtype = ev_gtype(e.op);
                    continue;
                }
                // END: the advance alone (identity transition, trow = -1)
                ce.kind = kind == EV_RF ? CE_RF : CE_END;
                CellKey k{};
                k.trow = kind == EV_RF ? e.row : -1;
                k.gtype = kind == EV_RF ? ev_gtype(e.op) : p;
                k.kp = P.kd[i][p - 1];
                k.kr = P.r_axis >= 0 ? P.kd[i][P.r_axis] : 0.0;
                k.tau = P.adv[i].tau;
                k.prow = e.prow;
                k.qr = (P.r_axis >= 0 && (ev_mask(e.op) & rbit)) ? e.q[P.r_axis] : -1;
                // the same key, for the form that builds the row per thread
                ce.win = k.trow;
                ce.gtype = k.gtype;
                ce.qr = k.qr;
                ce.prow = k.prow;
                if (P.otf) continue;
                int id = -1;
                for (size_t j = 0; j < P.ckeys.size() && id < 0; ++j) {
                    const CellKey &o = P.ckeys[j];
                    if (o.trow == k.trow && o.gtype == k.gtype && near(o.kp, k.kp) &&
                        near(o.kr, k.kr) && near(o.tau, k.tau))
                        id = (int)j;
                }
                if (id < 0) {
                    id = (int)P.ckeys.size();
                    P.ckeys.push_back(k);
                    // a row table within 1 GiB (and row indices within int32)
                    // and, unless asked for, within four times the state;
                    // beyond, every thread forms its cell's rows itself
                    const int64_t bytes = (int64_t)P.ckeys.size() * g->n_cells * 48;
                    if (bytes > ((int64_t)1 << 30) ||
                        (rows_mode == 0 && bytes > 4 * 12 * g->K)) {
                        P.otf = true;
                        P.ckeys.clear();
                        for (size_t j = 0; j <= i; ++j)
                            if (P.cev[j].kind <= CE_END) P.cev[j].row = 0;
                        continue;
                    }
                }
                ce.row = (int)((int64_t)id * g->n_cells);
            }
            if (!P.cell) {
                P.cev.clear();
                P.ckeys.clear();
                axis_tables(false);
            }
        }
    }
    // 4) group-signal blocks: 256 samples x a slice of the groups
    if (!P.wins.empty()) {
        int64_t base_blocks = 0, max_g = 1;
        for (const GWin &w : P.wins) {
            base_blocks += (w.n_samples + 255) / 256;
            max_g = std::max<int64_t>(max_g, w.n_groups);
        }
        const int64_t want = 4LL * c->sm_count;
        int64_t split = std::max<int64_t>(1, (want + base_blocks - 1) / base_blocks);
        split = std::min<int64_t>(split, (max_g + 255) / 256);
        for (size_t wi = 0; wi < P.wins.size(); ++wi) {
            const GWin &w = P.wins[wi];
            const int64_t gs =
                std::max<int64_t>(256, ((w.n_groups + split - 1) / split + 255) / 256 * 256);
            for (int64_t s0 = 0; s0 < w.n_samples; s0 += 256)
                for (int64_t g0 = 0; g0 < w.n_groups; g0 += gs)
                    P.blk.push_back(make_int4((int)wi, (int)(w.sample0 + s0), (int)g0,
                                              (int)std::min<int64_t>(w.n_groups, g0 + gs)));
        }
    }
}

template <typename R>
PrecompArgs precomp_args(const mrsim_seq *s, const mrsim_groups *g, int cid, int gt, R *out) {
    const Subseq &q = s->sub[s->content_first[cid]];
    const bool f64 = sizeof(R) == 8;
    return PrecompArgs{f64 ? s->rf_d[cid].p : s->rf_f[cid].p, s->rf_off[cid].as<int64_t>(),
                       (int)(q.seg_end - q.seg_begin), s->content_steps[cid], gt,
                       g->n_groups[gt], g->tab[gt].d_par64.as<double>(), out};
}

template <typename R>
GSigTables<R> sig_tables(const mrsim_groups *g) {
    const bool f64 = sizeof(R) == 8;
    GSigTables<R> tab{};
    for (int t = 0; t < kNTypes; ++t) {
        if (!g->built[t]) continue;
        tab.pos[t] = f64 ? (const R *)g->tab[t].d_pos64.p : (const R *)g->tab[t].d_pos.p;
        tab.dB0[t] = f64 ? (const R *)g->tab[t].d_dB064.p : (const R *)g->tab[t].d_dB0.p;
        tab.rT2[t] = f64 ? (const R *)g->tab[t].d_rT264.p : (const R *)g->tab[t].d_rT2.p;
        tab.pos2[t] = f64 ? (const R *)g->tab[t].d_pos264.p : (const R *)g->tab[t].d_pos2.p;
    }
    return tab;
}

template <typename R>
FusedArgs<R> fused_args(const mrsim_groups *g, int p, R *Mx, R *My, R *Mz, const R *T_tab,
                        const void *P_raw, double *Ablk) {
    FusedArgs<R> fa{};
    fa.K = g->K;
    fa.x = g->x.as<float>(); fa.y = g->y.as<float>(); fa.z = g->z.as<float>();
    fa.T1 = g->T1.as<float>(); fa.T2 = g->T2.as<float>(); fa.dB0 = g->dB0.as<float>();
    fa.M0 = g->M0.as<float>();
    for (int t = 0; t < kNTypes; ++t)
        fa.gid[t] = g->built[t] ? g->gid_sorted[t].as<int32_t>() : nullptr;
    fa.gtype_p = p;
    fa.gtype_r = g->secondary >= 0 ? g->secondary : p;
    fa.Mx = Mx; fa.My = My; fa.Mz = Mz;
    fa.T_tab = T_tab;
    fa.P_raw = P_raw;
    fa.Ablk = Ablk;
    fa.init_eq = g->has_M_init ? 0 : 1;
    return fa;
}

template <typename R>
void run_grouped(mrsim_ctx *c, const mrsim_phantom_t *ph, const mrsim_seq *s,
                 const mrsim_groups *g, double *d_signal, R *M, bool use_sur = false) {
    const int64_t K = ph->K;
    const bool f64 = sizeof(R) == 8;
    using A = typename AdvOf<R>::T;
    GPlan<R> P;
    plan_grouped<R>(c, s, g, P, true);
    // the FP32 cell form alone reads M0 and the axis index of the layout-order
    // arrays; everything else (per-isochromat form, fallbacks, initial
    // states, receive coils, windows and pulses of other group types) needs
    // the rest of them
    bool cell_only = sizeof(R) == 4 && P.cell && !g->has_M_init && ph->n_coils == 0 &&
                     !g->built[G_NONE];
    for (const auto &sp : P.spans) cell_only &= sp.fallback < 0;
    for (const CellEv &e : P.cev) cell_only &= e.kind != CE_ADC_OTHER;
    if (!cell_only) ensure_layout_arrays(c, g, ph);
    R *T_tab = (R *)scratch(c, 6, std::max<int64_t>(P.rows, 1) * 12 * sizeof(R));
    for (auto &t : P.tabs) {
        if constexpr (sizeof(R) == 4) {
            // learned transitions for the slice-selective pulses the network serves
            if (use_sur &&
                sur_table(c, s, g, t.first.first, t.first.second, T_tab + t.second * 12))
                continue;
        }
        launch_precompute<R>(c, precomp_args<R>(s, g, t.first.first, t.first.second,
                                                 T_tab + t.second * 12));
    }
    // block sums of one coil, or of up to four coils per pass in the cell form
    const int coils_per_pass = P.cell && ph->n_coils > 0 ? 4 : 1;
    double *Ablk = (double *)scratch(
        c, 7, std::max<int64_t>(P.ablk_n, 1) * 2 * coils_per_pass * sizeof(double));
    MRSIM_CUDA(cudaMemsetAsync(Ablk, 0, std::max<int64_t>(P.ablk_n, 1) * 2 * sizeof(double),
                               c->stream));
    const int64_t Kp = plane_stride(K);
    PlainState st = sorted_state(g, M, M + Kp, M + 2 * Kp);
    st.fx = c->fx;
    const int n_ev = (int)P.ev.size();
    EvAdv *d_adv = (EvAdv *)scratch(c, 14, n_ev * sizeof(EvAdv));
    void *d_P = scratch(c, 15, (P.direct ? 1 : (size_t)n_ev * std::max<int64_t>(P.Gp, 1)) * 4 *
                                   sizeof(R));
    FEvent<R> *d_ev = (FEvent<R> *)scratch(c, 11, n_ev * sizeof(FEvent<R>));
    upload(c, d_adv, P.adv.data(), n_ev * sizeof(EvAdv));
    upload(c, d_ev, P.ev.data(), n_ev * sizeof(FEvent<R>));
    const int prim = P.p;
    if (!P.direct)
        launch_event_table<R>(c, d_adv, n_ev, P.Gp, g->tab[prim].d_par64.as<double>(), d_P);
    if (g->has_M_init) launch_init_state<R>(c, st, g->M_init.as<float>());
    FusedArgs<R> fa = fused_args<R>(g, P.p, M, M + Kp, M + 2 * Kp, T_tab, d_P, Ablk);
    fa.direct = P.direct ? 1 : 0;
    fa.fx = c->fx;
    if (P.ax) {
        fa.ax = 1;
        fa.aidx = g->ax_idx.as<int32_t>();
        int n = 0;
        for (int a = 0; a < 3; ++a) {
            fa.ax_sh[a] = 0;
            if (a != P.p - 1) fa.ax_sh[a] = 16 * n++;
        }
        if (!P.ax_items.empty()) {
            float2 *qtab = (float2 *)scratch(c, 16, P.ax_n * sizeof(float2));
            AxItem *d_items = (AxItem *)scratch(c, 17, P.ax_items.size() * sizeof(AxItem));
            upload(c, d_items, P.ax_items.data(), P.ax_items.size() * sizeof(AxItem));
            launch_axis_phase(c, d_items, (int)P.ax_items.size(), P.ax_max, qtab);
            fa.qtab = qtab;
        }
    }
    // cell form: combined rows C = T Adv of every distinct RF advance and cell
    CellArgs ca{};
    CellEv *d_cev = nullptr;
    if constexpr (sizeof(R) == 4) {
        if (P.cell) {
            const int nk = P.otf ? 0 : (int)P.ckeys.size();
            float *C_tab = P.otf ? nullptr
                                 : (float *)scratch(c, 23,
                                                    std::max<int64_t>((int64_t)nk * g->n_cells, 1) *
                                                        12 * sizeof(float));
            if (nk > 0) {
                CellKey *d_keys = (CellKey *)scratch(c, 24, nk * sizeof(CellKey));
                upload(c, d_keys, P.ckeys.data(), nk * sizeof(CellKey));
                launch_cell_rows(c, d_keys, nk, g, T_tab, d_P, fa.qtab,
                                 P.r_axis >= 0 ? fa.ax_sh[P.r_axis] : 0, C_tab);
            }
            // per-thread work for the kernel's width: the coil kernels hold
            // 4 isochromats per thread
            const int w = ph->n_coils > 0 ? 0 : P.cell_w;
            ca.n_thr = g->n_cell_thr[w];
            ca.thr = g->cell_thr[w].as<int2>();
            ca.cell_gp = g->cell_gp.as<int32_t>();
            ca.cell_count = g->cell_count.as<int32_t>();
            ca.M0 = fa.M0;
            ca.aidx = fa.aidx;
            ca.Mx = M;
            ca.My = M + Kp;
            ca.Mz = M + 2 * Kp;
            ca.C_tab = C_tab;
            ca.P_raw = d_P;
            ca.Ablk = Ablk;
            ca.fx = c->fx;
            ca.otf = P.otf ? 1 : 0;
            ca.T_tab = T_tab;
            ca.cell_gr = g->cell_gr.as<int32_t>();
            ca.gtype_p = P.p;
            ca.gtype_r = g->secondary;
            ca.qtab = fa.qtab;
            int nf = 0;
            for (int a = 0; a < 3; ++a)
                if (P.free_bits & (1 << a)) ca.f_sh[nf++] = fa.ax_sh[a];
            if (nf < 2) ca.f_sh[1] = 0;
            ca.r_sh = P.r_axis >= 0 ? fa.ax_sh[P.r_axis] : 0;
            for (int t = 0; t < kNTypes; ++t) ca.gid[t] = fa.gid[t];
            d_cev = (CellEv *)scratch(c, 25, P.cev.size() * sizeof(CellEv));
            upload(c, d_cev, P.cev.data(), P.cev.size() * sizeof(CellEv));
        }
    }
    const double z0[3] = {0.0, 0.0, 0.0};
    const A zero = AdvOf<R>::make(z0, 0.0);
    GWin *dw = nullptr;
    int4 *db = nullptr;
    if (!P.blk.empty()) {
        dw = (GWin *)scratch(c, 12, P.wins.size() * sizeof(GWin));
        db = (int4 *)scratch(c, 13, P.blk.size() * sizeof(int4));
        upload(c, dw, P.wins.data(), P.wins.size() * sizeof(GWin));
        upload(c, db, P.blk.data(), P.blk.size() * sizeof(int4));
    }
    // Receive coils (Eq. 6 with P coils, Eq. 9 block sums per (group, coil)):
    // the tables above serve every pass.  The cell form takes up to four coils
    // per pass over the sequence (their state evolution is the same); the
    // per-isochromat form one.
    const int n_coils = ph->n_coils;
    const int64_t ns = s->n_samples;
    const int per_pass = coils_per_pass;
    float *coil_s = n_coils > 0
                        ? (float *)scratch(c, 18, (size_t)2 * per_pass * K * sizeof(float))
                        : nullptr;
    const int64_t ablk_sz = std::max<int64_t>(P.ablk_n, 1) * 2 * per_pass;
    for (int c0 = 0; c0 < std::max(n_coils, 1);) {
        const int rem = n_coils - c0;
        const int pc = n_coils == 0 ? 0 : per_pass == 1 ? 1 : rem >= 4 ? 4 : rem >= 2 ? 2 : 1;
        if (coil_s) {
            // coils c0 .. c0 + pc - 1 in layout order, [coil][re, im][K]
            for (int j = 0; j < pc; ++j) {
                const float *src = ph->coils.as<float>() + 2 * K * (c0 + j);
                launch_gather_f32(c, K, g->perm.as<int32_t>(), src, coil_s + 2 * K * j);
                launch_gather_f32(c, K, g->perm.as<int32_t>(), src + K, coil_s + 2 * K * j + K);
            }
            fa.coil_re = st.coil_re = coil_s;
            fa.coil_im = st.coil_im = coil_s + K;
        }
        if (c0 > 0) {
            MRSIM_CUDA(cudaMemsetAsync(Ablk, 0, ablk_sz * sizeof(double), c->stream));
            if (g->has_M_init) launch_init_state<R>(c, st, g->M_init.as<float>());
        } else if (per_pass > 1) {
            MRSIM_CUDA(cudaMemsetAsync(Ablk, 0, ablk_sz * sizeof(double), c->stream));
        }
        CellForm form = P.form;
        if constexpr (sizeof(R) == 4) {
            form.pc = pc;
            ca.coil = coil_s;
            ca.K = K;
            ca.ablk_stride = std::max<int64_t>(P.ablk_n, 1);
        }
        bool first = true;
        for (const auto &sp : P.spans) {
            fa.ev = d_ev + sp.b;
            fa.n_ev = (int)(sp.e - sp.b);
            fa.init_eq = (first && !g->has_M_init) ? 1 : 0;
            if constexpr (sizeof(R) == 4) {
                if (P.cell) {
                    ca.ev = d_cev + sp.b;
                    ca.n_ev = (int)(sp.e - sp.b);
                    ca.init_eq = fa.init_eq;
                    launch_fused_cell(c, ca, form);
                } else {
                    launch_fused<R>(c, fa, c->tune[MRSIM_TUNE_FUSED_NI]);
                }
            } else {
                launch_fused<R>(c, fa, c->tune[MRSIM_TUNE_FUSED_NI]);
            }
            first = false;
            if (sp.fallback < 0) continue;
            const Subseq &q = s->sub[sp.fallback];
            if (q.type == SUB_RF) {
                launch_plain_rf<R>(c, st, f64 ? s->rf_d[q.content].p : s->rf_f[q.content].p,
                                   (int)(q.seg_end - q.seg_begin), &zero,
                                   c->tune[MRSIM_TUNE_PLAIN_RF_NI]);
            } else {
                const void *segs =
                    f64 ? (const void *)(s->adc_d.as<ADCSegD>() + s->adc_off[sp.fallback])
                        : (const void *)(s->adc_f.as<ADCSegF>() + s->adc_off[sp.fallback]);
                // one launch per coil of this pass (the state is only read)
                for (int j = 0; j < std::max(pc, 1); ++j) {
                    if (coil_s) {
                        st.coil_re = coil_s + 2 * K * j;
                        st.coil_im = st.coil_re + K;
                    }
                    launch_plain_adc<R>(c, st, segs, (int)(q.seg_end - q.seg_begin), q.n_samples,
                                        &zero, d_signal + 2 * (ns * (c0 + j) + q.sample0),
                                        c->tune[MRSIM_TUNE_ADC_CTAS_PER_SM]);
                }
            }
        }
        // every sample from the block sums (Eqs. 8, 10), per coil of the pass
        for (int j = 0; j < std::max(pc, 1); ++j) {
            if (!P.blk.empty())
                launch_group_signal<R>(c, dw, db, (int)P.blk.size(), f64 ? s->gs_d.p : s->gs_f.p,
                                       sig_tables<R>(g), Ablk + 2 * std::max<int64_t>(P.ablk_n, 1) * j,
                                       d_signal + 2 * ns * (c0 + j));
        }
        c0 += std::max(pc, 1);
    }
    sync(c);
}

// --------------------------------------------------------------- batch ----
// All jobs' device work in four launches (batched transition precompute,
// batched group-factor tables, the persistent fused kernel over every job's
// chunks, batched group signal), captured once into a CUDA graph and reused
// while the same jobs are run again.
struct BatchCache {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec = nullptr;
    std::vector<DBuf> bufs;
    std::vector<double *> d_sig;
    std::vector<int64_t> n_samples;
    ~BatchCache() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

std::map<const mrsim_ctx *, std::unique_ptr<BatchCache>> &batch_caches() {
    static std::map<const mrsim_ctx *, std::unique_ptr<BatchCache>> m;
    return m;
}

void run_batch(mrsim_ctx *c, int n, const mrsim_phantom_t *const *ph, const mrsim_seq *const *s,
               const mrsim_groups *const *g, double *const *signals) {
    using R = float;
    // the batched kernels read every layout-order array of a job
    for (int i = 0; i < n; ++i) ensure_layout_arrays(c, g[i], ph[i]);
    std::vector<uint64_t> key;
    for (int i = 0; i < n; ++i) {
        key.push_back(ph[i]->uid);
        key.push_back(ph[i]->coil_uid);
        key.push_back(s[i]->uid);
        key.push_back(g[i]->uid);
    }
    for (int t = 0; t < 8; ++t) key.push_back((uint64_t)c->tune[t]);
    auto &slot = batch_caches()[c];
    if (!slot || slot->key != key) {
        auto bc = std::make_unique<BatchCache>();
        bc->key = key;
        std::vector<GPlan<R>> plans(n);
        // the cell form for jobs without coils whose plan takes it
        for (int i = 0; i < n; ++i) plan_grouped<R>(c, s[i], g[i], plans[i], ph[i]->n_coils == 0);
        // Instances: one per (job, receive coil); the coils of a job share its
        // tables and windows, each has its own block sums, signal and state.
        // An instance keeps its state in device memory when its sequence has
        // subsequences without a type (several fused spans with the
        // per-isochromat fallback between them) or starts from a given state.
        struct Inst { int job, coil; bool state; };
        std::vector<Inst> inst;
        std::vector<int> inst0(n);
        for (int i = 0; i < n; ++i) {
            inst0[i] = (int)inst.size();
            const bool st = plans[i].spans.size() > 1 || g[i]->has_M_init;
            for (int j = 0; j < std::max(ph[i]->n_coils, 1); ++j) inst.push_back(Inst{i, j, st});
        }
        const int ni_ = (int)inst.size();
        // sizes and offsets inside shared device buffers
        int64_t rows = 0, ablk = 0, nev = 0, ptab = 0, nsig = 0, nst = 0, ncoil = 0;
        std::vector<int64_t> o_rows(n), o_ev(n), o_p(n), o_sig(n);
        std::vector<int64_t> o_ablk(ni_), o_st(ni_), o_coil(ni_);
        for (int i = 0; i < n; ++i) {
            o_rows[i] = rows; rows += plans[i].rows;
            o_ev[i] = nev; nev += (int64_t)plans[i].ev.size();
            o_p[i] = ptab;
            if (!plans[i].direct) ptab += (int64_t)plans[i].ev.size() * plans[i].Gp;
            o_sig[i] = nsig; nsig += s[i]->n_samples * std::max(ph[i]->n_coils, 1);
        }
        for (int q = 0; q < ni_; ++q) {
            const int i = inst[q].job;
            o_ablk[q] = ablk; ablk += plans[i].ablk_n;
            o_st[q] = nst;
            if (inst[q].state) nst += 3 * plane_stride(g[i]->K);
            o_coil[q] = ncoil;
            if (ph[i]->n_coils > 0) ncoil += 2 * g[i]->K;
        }
        auto alloc = [&](size_t bytes) {
            bc->bufs.push_back(dalloc(std::max<size_t>(bytes, 256)));
            return bc->bufs.back().p;
        };
        R *T = (R *)alloc(rows * 12 * sizeof(R));
        double *Ab = (double *)alloc(ablk * 2 * sizeof(double));
        FEvent<R> *ev = (FEvent<R> *)alloc(nev * sizeof(FEvent<R>));
        EvAdv *adv = (EvAdv *)alloc(nev * sizeof(EvAdv));
        void *Pt = alloc(ptab * 4 * sizeof(R));
        double *sig = (double *)alloc(std::max<int64_t>(nsig, 1) * 2 * sizeof(double));
        R *Mst = (R *)alloc(nst * sizeof(R));
        float *cmap = (float *)alloc(ncoil * sizeof(float));
        // cell-form jobs: axis phasor tables, combined rows (unless formed per
        // thread), their keys and the event records, each job at its offset
        int64_t nq = 0, ncev = 0, ncrow = 0, nkey = 0;
        std::vector<int64_t> o_q(n), o_cev(n), o_crow(n), o_key(n);
        std::vector<AxItem> items;
        int ax_max = 0;
        for (int i = 0; i < n; ++i) {
            const GPlan<R> &P = plans[i];
            o_q[i] = nq;
            o_cev[i] = ncev;
            o_crow[i] = ncrow;
            o_key[i] = nkey;
            if (!P.cell) continue;
            for (AxItem it : P.ax_items) {
                it.off += nq;
                items.push_back(it);
            }
            ax_max = std::max(ax_max, P.ax_max);
            nq += P.ax_n;
            ncev += (int64_t)P.cev.size();
            if (!P.otf) {
                ncrow += (int64_t)P.ckeys.size() * g[i]->n_cells * 12;
                nkey += (int64_t)P.ckeys.size();
            }
        }
        float2 *qtab = (float2 *)alloc(nq * sizeof(float2));
        CellEv *cev = (CellEv *)alloc(ncev * sizeof(CellEv));
        float *crow = (float *)alloc(ncrow * sizeof(float));
        CellKey *ckey = (CellKey *)alloc(nkey * sizeof(CellKey));
        AxItem *d_items = (AxItem *)alloc(std::max<size_t>(items.size(), 1) * sizeof(AxItem));
        upload(c, d_items, items.data(), items.size() * sizeof(AxItem));
        for (int i = 0; i < n; ++i) {
            const GPlan<R> &P = plans[i];
            if (!P.cell) continue;
            upload(c, cev + o_cev[i], P.cev.data(), P.cev.size() * sizeof(CellEv));
            if (!P.otf)
                upload(c, ckey + o_key[i], P.ckeys.data(), P.ckeys.size() * sizeof(CellKey));
        }
        // bit position of each axis' index in the packed axis index (the
        // primary axis has none)
        auto ax_sh = [&](int i, int (&sh)[3]) {
            int m = 0;
            for (int a = 0; a < 3; ++a) sh[a] = a == plans[i].p - 1 ? 0 : 16 * m++;
        };
        // receive-coil maps in each job's layout order (fixed while the
        // phantom's coils are: the cache key holds their version)
        for (int q = 0; q < ni_; ++q) {
            const int i = inst[q].job, j = inst[q].coil;
            if (ph[i]->n_coils == 0) continue;
            const int64_t K = g[i]->K;
            const float *src = ph[i]->coils.as<float>() + 2 * K * j;
            launch_gather_f32(c, K, g[i]->perm.as<int32_t>(), src, cmap + o_coil[q]);
            launch_gather_f32(c, K, g[i]->perm.as<int32_t>(), src + K, cmap + o_coil[q] + K);
        }
        // descriptors
        std::vector<PrecompArgs> pre;
        std::vector<int64_t> pre_off{0};
        std::vector<EvTabJob> et;
        std::vector<int64_t> et_off{0};
        std::vector<GSigJob<R>> gj;
        std::vector<int4> gblk;
        std::vector<int> gblk_job;
        std::vector<GWin> allwin;
        std::vector<int64_t> win0(n);
        for (int i = 0; i < n; ++i) {
            GPlan<R> &P = plans[i];
            for (auto &t : P.tabs) {
                pre.push_back(precomp_args<R>(s[i], g[i], t.first.first, t.first.second,
                                              T + (o_rows[i] + t.second) * 12));
                pre.back().kb = c->tune[MRSIM_TUNE_PRECOMP_STEPS];
                pre_off.push_back(pre_off.back() + g[i]->n_groups[t.first.second]);
            }
            if (!P.direct) {
                et.push_back(EvTabJob{adv + o_ev[i], P.Gp, g[i]->tab[P.p].d_par64.as<double>(),
                                      (R *)Pt + o_p[i] * 4});
                et_off.push_back(et_off.back() + (int64_t)P.ev.size() * P.Gp);
            }
            win0[i] = (int64_t)allwin.size();
            for (GWin w : P.wins) allwin.push_back(w);
            upload(c, ev + o_ev[i], P.ev.data(), P.ev.size() * sizeof(FEvent<R>));
            upload(c, adv + o_ev[i], P.adv.data(), P.adv.size() * sizeof(EvAdv));
            bc->d_sig.push_back(sig + 2 * o_sig[i]);
            bc->n_samples.push_back(s[i]->n_samples * std::max(ph[i]->n_coils, 1));
        }
        // fused launches: one per (span number, form) over the instances with
        // that span; the per-isochromat fallbacks follow each span number
        size_t n_span = 0;
        for (auto &P : plans) n_span = std::max(n_span, P.spans.size());
        struct Fb { int q, sub; };
        std::vector<std::array<std::vector<FusedArgs<R>>, 4>> fj(n_span);
        std::vector<std::array<std::vector<int64_t>, 4>> fj_off(n_span);
        // cell form: one launch per (span number, free axes, rows per thread)
        std::vector<std::array<std::vector<CellArgs>, 4>> cj(n_span);
        std::vector<std::array<std::vector<int64_t>, 4>> cj_off(n_span);
        int cell_ni = 8;
        std::vector<std::vector<Fb>> fb(n_span);
        auto state = [&](int q, R *&x, R *&y, R *&z) {
            const int64_t Kp = plane_stride(g[inst[q].job]->K);
            x = inst[q].state ? Mst + o_st[q] : nullptr;
            y = x ? x + Kp : nullptr;
            z = x ? x + 2 * Kp : nullptr;
        };
        for (int q = 0; q < ni_; ++q) {
            const int i = inst[q].job;
            GPlan<R> &P = plans[i];
            R *x, *y, *z;
            state(q, x, y, z);
            const int64_t K = g[i]->K;
            const bool coil = ph[i]->n_coils > 0;
            const int form = (P.direct ? 1 : 0) | (coil ? 2 : 0);
            for (size_t k = 0; k < P.spans.size(); ++k) {
                const auto &sp = P.spans[k];
                FusedArgs<R> fa = fused_args<R>(g[i], P.p, x, y, z, T + o_rows[i] * 12,
                                                (R *)Pt + o_p[i] * 4, Ab + 2 * o_ablk[q]);
                fa.ev = ev + o_ev[i] + sp.b;
                fa.n_ev = (int)(sp.e - sp.b);
                fa.init_eq = (k == 0 && !g[i]->has_M_init) ? 1 : 0;
                fa.direct = P.direct ? 1 : 0;
                if (coil) {
                    fa.coil_re = cmap + o_coil[q];
                    fa.coil_im = fa.coil_re + K;
                }
                if (sp.fallback >= 0) fb[k].push_back(Fb{q, sp.fallback});
                if (P.cell) {
                    CellArgs ca{};
                    const int w = P.cell_w;
                    cell_ni = P.form.ni;
                    ca.n_thr = g[i]->n_cell_thr[w];
                    ca.thr = g[i]->cell_thr[w].as<int2>();
                    ca.cell_gp = g[i]->cell_gp.as<int32_t>();
                    ca.cell_count = g[i]->cell_count.as<int32_t>();
                    ca.M0 = fa.M0;
                    ca.aidx = g[i]->ax_idx.as<int32_t>();
                    ca.Mx = x;
                    ca.My = y;
                    ca.Mz = z;
                    ca.init_eq = fa.init_eq;
                    ca.ev = cev + o_cev[i] + sp.b;
                    ca.n_ev = (int)(sp.e - sp.b);
                    ca.C_tab = P.otf ? nullptr : crow + o_crow[i];
                    ca.P_raw = (R *)Pt + o_p[i] * 4;
                    ca.Ablk = Ab + 2 * o_ablk[q];
                    ca.qtab = qtab + o_q[i];
                    int sh[3];
                    ax_sh(i, sh);
                    int nf = 0;
                    for (int a = 0; a < 3; ++a)
                        if (P.free_bits & (1 << a)) ca.f_sh[nf++] = sh[a];
                    if (nf < 2) ca.f_sh[1] = 0;
                    ca.r_sh = P.r_axis >= 0 ? sh[P.r_axis] : 0;
                    for (int t = 0; t < kNTypes; ++t) ca.gid[t] = fa.gid[t];
                    ca.K = K;
                    ca.ablk_stride = std::max<int64_t>(P.ablk_n, 1);
                    ca.rfq = P.form.rfq ? 1 : 0;
                    ca.adq = P.form.adq ? 1 : 0;
                    ca.rb = P.form.rb ? 1 : 0;
                    ca.otf = P.otf ? 1 : 0;
                    ca.T_tab = T + o_rows[i] * 12;
                    ca.cell_gr = g[i]->cell_gr.as<int32_t>();
                    ca.gtype_p = P.p;
                    ca.gtype_r = g[i]->secondary;
                    const int grp = (P.form.nf == 2 ? 1 : 0) | (P.otf ? 2 : 0);
                    auto &co = cj_off[k][grp];
                    if (co.empty()) co.push_back(0);
                    cj[k][grp].push_back(ca);
                    co.push_back(co.back() + (ca.n_thr + 255) / 256);
                    continue;
                }
                auto &off = fj_off[k][form];
                if (off.empty()) off.push_back(0);
                fj[k][form].push_back(fa);
                off.push_back(off.back() + (K + kFusedChunk(c) - 1) / kFusedChunk(c));
            }
            const double *ab = Ab + 2 * o_ablk[q];
            double *sq = sig + 2 * (o_sig[i] + s[i]->n_samples * inst[q].coil);
            gj.push_back(GSigJob<R>{nullptr, s[i]->gs_f.p, sig_tables<R>(g[i]), ab, sq, 0.0});
            gj.back().wins = (const GWin *)(intptr_t)win0[i];  // fixed up after upload
            for (int4 b : P.blk) {
                gblk.push_back(b);
                gblk_job.push_back(q);
            }
        }
        GWin *d_win = (GWin *)alloc(std::max<size_t>(allwin.size(), 1) * sizeof(GWin));
        upload(c, d_win, allwin.data(), allwin.size() * sizeof(GWin));
        for (auto &j : gj) j.wins = d_win + (intptr_t)j.wins;
        auto up = [&](const void *src, size_t bytes) {
            void *d = alloc(bytes);
            upload(c, d, src, bytes);
            return d;
        };
        auto *d_pre = (PrecompArgs *)up(pre.data(), pre.size() * sizeof(PrecompArgs));
        auto *d_pre_off = (int64_t *)up(pre_off.data(), pre_off.size() * sizeof(int64_t));
        auto *d_et = (EvTabJob *)up(et.data(), std::max<size_t>(et.size(), 1) * sizeof(EvTabJob));
        auto *d_et_off = (int64_t *)up(et_off.data(), et_off.size() * sizeof(int64_t));
        struct FL { const FusedArgs<R> *jobs; const int64_t *off; int n, form; };
        std::vector<std::vector<FL>> fl(n_span);
        int n_fl = 0;
        for (size_t k = 0; k < n_span; ++k)
            for (int f = 0; f < 4; ++f) {
                if (fj[k][f].empty()) continue;
                fl[k].push_back(FL{(const FusedArgs<R> *)up(fj[k][f].data(),
                                                            fj[k][f].size() * sizeof(FusedArgs<R>)),
                                   (const int64_t *)up(fj_off[k][f].data(),
                                                       fj_off[k][f].size() * sizeof(int64_t)),
                                   (int)fj[k][f].size(), f});
                ++n_fl;
            }
        struct CL { const CellArgs *jobs; const int64_t *off; int n, nf; bool otf; };
        std::vector<std::vector<CL>> cl(n_span);
        for (size_t k = 0; k < n_span; ++k)
            for (int f = 0; f < 4; ++f) {
                if (cj[k][f].empty()) continue;
                cl[k].push_back(CL{(const CellArgs *)up(cj[k][f].data(),
                                                        cj[k][f].size() * sizeof(CellArgs)),
                                   (const int64_t *)up(cj_off[k][f].data(),
                                                       cj_off[k][f].size() * sizeof(int64_t)),
                                   (int)cj[k][f].size(), (f & 1) ? 2 : 1, (f & 2) != 0});
                ++n_fl;
            }
        auto *d_gj = (GSigJob<R> *)up(gj.data(), gj.size() * sizeof(GSigJob<R>));
        auto *d_gblk = (int4 *)up(gblk.data(), std::max<size_t>(gblk.size(), 1) * sizeof(int4));
        auto *d_gbj = (int *)up(gblk_job.data(), std::max<size_t>(gblk_job.size(), 1) * sizeof(int));
        auto *d_cnt = (unsigned long long *)alloc(std::max(n_fl, 1) * sizeof(unsigned long long));
        sync(c);
        // capture every launch of the batch into one graph
        const bool prof = c->prof_on;
        c->prof_on = false;
        const double z0[3] = {0.0, 0.0, 0.0};
        const typename AdvOf<R>::T zero = AdvOf<R>::make(z0, 0.0);
        cudaGraph_t graph = nullptr;
        MRSIM_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t cap = cudaSuccess;
        try {
            cap = cudaMemsetAsync(Ab, 0, std::max<int64_t>(ablk, 1) * 2 * sizeof(double), c->stream);
            if (cap == cudaSuccess)
                cap = cudaMemsetAsync(sig, 0, std::max<int64_t>(nsig, 1) * 2 * sizeof(double),
                                      c->stream);
            if (cap == cudaSuccess)
                cap = cudaMemsetAsync(d_cnt, 0, std::max(n_fl, 1) * sizeof(*d_cnt), c->stream);
            launch_precompute_batch<R>(c, d_pre, d_pre_off, (int)pre.size(), pre_off.back());
            if (!et.empty())
                launch_event_table_batch<R>(c, d_et, d_et_off, (int)et.size(), et_off.back());
            // cell-form jobs: every job's axis phasors in one launch, then the
            // combined rows of the jobs that read them from a table
            if (!items.empty()) launch_axis_phase(c, d_items, (int)items.size(), ax_max, qtab);
            for (int i = 0; i < n; ++i) {
                const GPlan<R> &P = plans[i];
                if (!P.cell || P.otf || P.ckeys.empty()) continue;
                int sh[3];
                ax_sh(i, sh);
                launch_cell_rows(c, ckey + o_key[i], (int)P.ckeys.size(), g[i], T + o_rows[i] * 12,
                                 (R *)Pt + o_p[i] * 4, qtab + o_q[i],
                                 P.r_axis >= 0 ? sh[P.r_axis] : 0, crow + o_crow[i]);
            }
            for (int q = 0; q < ni_; ++q) {
                const int i = inst[q].job;
                if (!inst[q].state || !g[i]->has_M_init) continue;
                R *x, *y, *z;
                state(q, x, y, z);
                launch_init_state<R>(c, sorted_state(g[i], x, y, z), g[i]->M_init.as<float>());
            }
            int li = 0;
            for (size_t k = 0; k < n_span; ++k) {
                for (const FL &f : fl[k])
                    launch_fused_batch<R>(c, f.jobs, f.off, f.n, d_cnt + li++,
                                          c->tune[MRSIM_TUNE_FUSED_NI], (f.form & 1) != 0,
                                          (f.form & 2) != 0);
                for (const CL &f : cl[k])
                    launch_fused_cell_batch(c, f.jobs, f.off, f.n, d_cnt + li++, cell_ni, f.nf,
                                            f.otf);
                for (const Fb &b : fb[k]) {
                    const int i = inst[b.q].job;
                    const Subseq &qq = s[i]->sub[b.sub];
                    R *x, *y, *z;
                    state(b.q, x, y, z);
                    PlainState st = sorted_state(g[i], x, y, z);
                    if (ph[i]->n_coils > 0) {
                        st.coil_re = cmap + o_coil[b.q];
                        st.coil_im = st.coil_re + g[i]->K;
                    }
                    const int nseg = (int)(qq.seg_end - qq.seg_begin);
                    if (qq.type == SUB_RF) {
                        launch_plain_rf<R>(c, st, s[i]->rf_f[qq.content].p, nseg, &zero,
                                           c->tune[MRSIM_TUNE_PLAIN_RF_NI]);
                    } else {
                        double *out = sig + 2 * (o_sig[i] + s[i]->n_samples * inst[b.q].coil +
                                                 qq.sample0);
                        launch_plain_adc<R>(c, st, s[i]->adc_f.as<ADCSegF>() + s[i]->adc_off[b.sub],
                                            nseg, qq.n_samples, &zero, out,
                                            c->tune[MRSIM_TUNE_ADC_CTAS_PER_SM]);
                    }
                }
            }
            launch_group_signal_batch<R>(c, d_gj, d_gblk, d_gbj, (int)gblk.size());
        } catch (...) {
            cudaStreamEndCapture(c->stream, &graph);
            if (graph) cudaGraphDestroy(graph);
            c->prof_on = prof;
            throw;
        }
        const cudaError_t end = cudaStreamEndCapture(c->stream, &graph);
        c->prof_on = prof;
        MRSIM_CUDA(cap);
        MRSIM_CUDA(end);
        const cudaError_t inst_rc = cudaGraphInstantiate(&bc->exec, graph, 0);
        cudaGraphDestroy(graph);
        MRSIM_CUDA(inst_rc);
        slot = std::move(bc);
    }
    {
        KScope ks(c, "batch_graph");
        MRSIM_CUDA(cudaGraphLaunch(slot->exec, c->stream));
    }
    for (int i = 0; i < n; ++i)
        if (slot->n_samples[i] > 0)
            MRSIM_CUDA(cudaMemcpyAsync(signals[i], slot->d_sig[i],
                                       slot->n_samples[i] * 2 * sizeof(double),
                                       cudaMemcpyDeviceToHost, c->stream));
    sync(c);
}

int set_err(mrsim_ctx *c, int code, const std::string &m) {
    if (c) c->err = m;
    return code;
}

// The value checks of a phantom uploaded with MRSIM_PHANTOM_ASYNC, read at its
// first use (waiting once for the queued checks); a phantom that failed them
// stays unusable.
void phantom_ready(mrsim_ctx *, const mrsim_phantom_t *ph) {
    if (ph->check == 1) {
        // the checks ran on the stream of the context that made the phantom
        int h = 0;
        MRSIM_CUDA(cudaEventSynchronize(ph->checked));
        MRSIM_CUDA(cudaMemcpy(&h, ph->bad.p, sizeof(int), cudaMemcpyDeviceToHost));
        ph->check = h ? 2 : 0;
    }
    if (ph->check == 2)
        fail(MRSIM_EINVAL, "phantom has a non-finite value or T1/T2 <= 0 (checked at first use)");
}

template <class F>
int guard(mrsim_ctx *c, F &&f) {
    CtxScope scope(c);
    try {
        f();
        if (c) c->err.clear();
        return MRSIM_OK;
    } catch (const Error &e) {
        return set_err(c, e.code, e.msg);
    } catch (const std::bad_alloc &) {
        return set_err(c, MRSIM_ENOMEM, "host allocation failed");
    } catch (const std::exception &e) {
        return set_err(c, MRSIM_EINVAL, e.what());
    }
}

// the most frequent gradient type with groups (ties: the smaller number)
int most_frequent(const int cnt[kNTypes]) {
    int best = -1, bc = 0;
    for (int t = 0; t < kNTypes; ++t)
        if (t != G_GENERAL && cnt[t] > bc) { bc = cnt[t]; best = t; }
    return best;
}

}  // namespace
}  // namespace mrsim

using namespace mrsim;

extern "C" {

int mrsim_create(mrsim_ctx **ctx, int device, void *cuda_stream) {
    if (!ctx) return MRSIM_EINVAL;
    *ctx = nullptr;
    mrsim_ctx *c = nullptr;
    try {
        c = new mrsim_ctx();
    } catch (...) {
        return MRSIM_ENOMEM;
    }
    int rc = guard(c, [&] {
        int n = 0;
        MRSIM_CUDA(cudaGetDeviceCount(&n));
        if (device < 0 || device >= n) fail(MRSIM_EINVAL, "no CUDA device " + std::to_string(device));
        c->device = device;
        MRSIM_CUDA(cudaSetDevice(device));
        MRSIM_CUDA(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device));
        if (cuda_stream) {
            c->stream = (cudaStream_t)cuda_stream;
        } else {
            MRSIM_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
            c->own_stream = true;
        }
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        auto pool = std::make_shared<DevPool>();
        MRSIM_CUDA(cudaMemPoolCreate(&pool->pool, &props));
        uint64_t keep = UINT64_MAX;  // keep the reserve between calls
        MRSIM_CUDA(cudaMemPoolSetAttribute(pool->pool, cudaMemPoolAttrReleaseThreshold, &keep));
        pool->stream = c->stream;
        c->pool = std::move(pool);
        c->dev_err = dalloc(64);
        MRSIM_CUDA(cudaMemsetAsync(c->dev_err.p, 0, 64, c->stream));
        prepare_fused(c);
    });
    if (rc) {
        delete c;
        return rc;
    }
    *ctx = c;
    return MRSIM_OK;
}

void mrsim_destroy(mrsim_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    prof_flush(c);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (auto &b : c->scratch) b.reset();
    c->dev_err.reset();
    if (c->pinned) cudaFreeHost(c->pinned);
    batch_caches().erase(c);
    if (c->pool) {  // buffers that outlive the context are freed synchronously
        cudaStreamSynchronize(c->stream);
        c->pool->stream = nullptr;
        cudaMemPoolTrimTo(c->pool->pool, 0);
        c->pool.reset();
    }
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char *mrsim_last_error(const mrsim_ctx *c) { return c ? c->err.c_str() : "no context"; }

int mrsim_phantom(mrsim_ctx *c, int64_t K, const float *x, const float *y, const float *z,
                  const float *T1, const float *T2, const float *dB0, const float *M0,
                  const float *b1, const float *M_init, unsigned flags, mrsim_phantom_t **out) {
    if (!c || !out) return MRSIM_EINVAL;
    *out = nullptr;
    auto p = std::unique_ptr<mrsim_phantom_t>(new (std::nothrow) mrsim_phantom_t());
    if (!p) return set_err(c, MRSIM_ENOMEM, "host allocation failed");
    int rc = guard(c, [&] {
        if (K <= 0 || K > 0x7fffffffLL) fail(MRSIM_EINVAL, "K must be in [1, 2^31 - 1]");
        if (!x || !y || !z || !T1 || !T2 || !dB0 || !M0) fail(MRSIM_EINVAL, "NULL phantom array");
        MRSIM_CUDA(cudaSetDevice(c->device));
        p->ctx = c;
        p->K = K;
        p->uid = g_uid++;
        const cudaMemcpyKind kind = (flags & MRSIM_PTR_DEVICE) ? cudaMemcpyDeviceToDevice
                                                               : cudaMemcpyHostToDevice;
        auto put = [&](DBuf &d, const float *src, int64_t n) {
            d = dalloc(n * sizeof(float));
            MRSIM_CUDA(cudaMemcpyAsync(d.p, src, n * sizeof(float), kind, c->stream));
        };
        put(p->x, x, K); put(p->y, y, K); put(p->z, z, K);
        put(p->T1, T1, K); put(p->T2, T2, K); put(p->dB0, dB0, K); put(p->M0, M0, K);
        if (b1) { put(p->b1, b1, K); p->has_b1 = true; }
        if (M_init) { put(p->M_init, M_init, 3 * K); p->has_M_init = true; }
        const bool async = (flags & MRSIM_PHANTOM_ASYNC) != 0;
        if (async) p->bad = dalloc(sizeof(int));
        int *err = async ? p->bad.as<int>() : c->dev_err.as<int>();
        MRSIM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), c->stream));
        {
            KScope ks(c, "validate_phantom");
            const int blocks = (int)std::min<int64_t>((K + 255) / 256, (int64_t)c->sm_count * 16);
            k_validate<<<blocks, 256, 0, c->stream>>>(
                K, p->x.as<float>(), p->y.as<float>(), p->z.as<float>(), p->T1.as<float>(),
                p->T2.as<float>(), p->dB0.as<float>(), p->M0.as<float>(),
                p->has_b1 ? p->b1.as<float>() : nullptr,
                p->has_M_init ? p->M_init.as<float>() : nullptr, err);
        }
        if (async) {
            MRSIM_CUDA(cudaEventCreateWithFlags(&p->checked, cudaEventDisableTiming));
            MRSIM_CUDA(cudaEventRecord(p->checked, c->stream));
            MRSIM_CUDA(cudaGetLastError());
            p->check = 1;
            return;
        }
        int h = 0;
        MRSIM_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        sync(c);
        if (h) fail(MRSIM_EINVAL, "phantom has a non-finite value or T1/T2 <= 0");
    });
    if (rc == MRSIM_OK) *out = p.release();
    return rc;
}

int mrsim_coils(mrsim_ctx *c, mrsim_phantom_t *ph, int n_coils, const float *sens,
                unsigned flags) {
    if (!c) return MRSIM_EINVAL;
    return guard(c, [&] {
        if (!ph) fail(MRSIM_EINVAL, "NULL phantom");
        phantom_ready(c, ph);
        if (n_coils < 0 || n_coils > MRSIM_MAX_COILS)
            fail(MRSIM_EINVAL, "n_coils must be in [0, " + std::to_string(MRSIM_MAX_COILS) + "]");
        if (n_coils > 0 && !sens) fail(MRSIM_EINVAL, "NULL sensitivities");
        MRSIM_CUDA(cudaSetDevice(c->device));
        if (n_coils == 0) {
            ph->coils.reset();
            ph->n_coils = 0;
            ph->sum_bound = -1.0;
            ph->coil_uid = g_uid++;
            return;
        }
        const int64_t n = 2 * (int64_t)n_coils * ph->K;
        DBuf d = dalloc(n * sizeof(float));
        MRSIM_CUDA(cudaMemcpyAsync(d.p, sens, n * sizeof(float),
                                   (flags & MRSIM_PTR_DEVICE) ? cudaMemcpyDeviceToDevice
                                                              : cudaMemcpyHostToDevice,
                                   c->stream));
        int *err = c->dev_err.as<int>();
        MRSIM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), c->stream));
        {
            KScope ks(c, "validate_coils");
            const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->sm_count * 16);
            k_finite<<<blocks, 256, 0, c->stream>>>(n, d.as<float>(), err);
        }
        int h = 0;
        MRSIM_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        sync(c);
        if (h) fail(MRSIM_EINVAL, "coil sensitivities have a non-finite value");
        ph->coils = std::move(d);
        ph->n_coils = n_coils;
        ph->sum_bound = -1.0;
        ph->coil_uid = g_uid++;
    });
}

int mrsim_phantom_read(mrsim_ctx *c, const mrsim_phantom_t *ph, float *x, float *y, float *z,
                       float *T1, float *T2, float *dB0, float *M0) {
    if (!c) return MRSIM_EINVAL;
    return guard(c, [&] {
        if (!ph) fail(MRSIM_EINVAL, "NULL phantom");
        if (ph->ctx != c) fail(MRSIM_ESTATE, "phantom of another context");
        phantom_ready(c, ph);
        MRSIM_CUDA(cudaSetDevice(c->device));
        const size_t b = ph->K * sizeof(float);
        const std::pair<float *, const DBuf *> f[7] = {{x, &ph->x},   {y, &ph->y},     {z, &ph->z},
                                                       {T1, &ph->T1}, {T2, &ph->T2},   {dB0, &ph->dB0},
                                                       {M0, &ph->M0}};
        for (const auto &e : f)
            if (e.first)
                MRSIM_CUDA(cudaMemcpyAsync(e.first, e.second->p, b, cudaMemcpyDeviceToHost,
                                           c->stream));
        sync(c);
    });
}

int mrsim_cluster(mrsim_ctx *c, const mrsim_phantom_t *ph, int n_clusters, const double *scale,
                  int max_iter, int n_echo, const double *te, double tr, int32_t *labels,
                  double *centres, int *n_out, mrsim_phantom_t **out) {
    if (!c || !out) return MRSIM_EINVAL;
    *out = nullptr;
    if (n_out) *n_out = 0;
    auto p = std::unique_ptr<mrsim_phantom_t>(new (std::nothrow) mrsim_phantom_t());
    if (!p) return set_err(c, MRSIM_ENOMEM, "host allocation failed");
    int n = 0;
    int rc = guard(c, [&] {
        if (!ph) fail(MRSIM_EINVAL, "NULL phantom");
        if (ph->ctx != c) fail(MRSIM_ESTATE, "phantom of another context");
        phantom_ready(c, ph);
        if (n_clusters < 1 || n_clusters > MRSIM_MAX_CLUSTERS)
            fail(MRSIM_EINVAL,
                 "n_clusters must be in [1, " + std::to_string(MRSIM_MAX_CLUSTERS) + "]");
        if (max_iter < 1) fail(MRSIM_EINVAL, "max_iter must be positive");
        const double def[3] = {64000.0, 64000.0, 64.0};
        const double *sc = scale ? scale : def;
        for (int i = 0; i < 3; ++i)
            if (!std::isfinite(sc[i]) || !(sc[i] > 0.0))
                fail(MRSIM_EINVAL, "scale must be finite and positive");
        if (n_echo < 0 || n_echo > MRSIM_MAX_ECHOES)
            fail(MRSIM_EINVAL, "n_echo must be in [0, " + std::to_string(MRSIM_MAX_ECHOES) + "]");
        if (n_echo > 0) {
            if (!te) fail(MRSIM_EINVAL, "NULL echo times");
            for (int e = 0; e < n_echo; ++e)
                if (!std::isfinite(te[e]) || te[e] < 0.0)
                    fail(MRSIM_EINVAL, "echo times must be finite and >= 0");
            if (!std::isfinite(tr) || !(tr > 0.0))
                fail(MRSIM_EINVAL, "repetition time must be finite and positive");
        }
        MRSIM_CUDA(cudaSetDevice(c->device));
        DBuf lab;
        std::vector<double> cen;
        cluster_phantom(c, ph, n_clusters, sc, max_iter, n_echo, te, tr, p.get(), lab, cen);
        n = (int)(cen.size() / 3);
        p->ctx = c;
        p->uid = g_uid++;
        if (labels) {
            MRSIM_CUDA(cudaMemcpyAsync(labels, lab.p, ph->K * sizeof(int32_t),
                                       cudaMemcpyDeviceToHost, c->stream));
            sync(c);
        }
        if (centres) std::copy(cen.begin(), cen.end(), centres);
    });
    if (rc == MRSIM_OK) {
        *out = p.release();
        if (n_out) *n_out = n;
    }
    return rc;
}

int mrsim_sequence(mrsim_ctx *c, int64_t n_seg, const double *dt, const int32_t *rep,
                   const float *b1re, const float *b1im, const float *gx, const float *gy,
                   const float *gz, const uint8_t *adc, mrsim_seq **out) {
    if (!c || !out) return MRSIM_EINVAL;
    *out = nullptr;
    auto s = std::unique_ptr<mrsim_seq>(new (std::nothrow) mrsim_seq());
    if (!s) return set_err(c, MRSIM_ENOMEM, "host allocation failed");
    int rc = guard(c, [&] {
        if (n_seg <= 0) fail(MRSIM_EINVAL, "n_seg must be positive");
        if (!dt || !rep || !b1re || !b1im || !gx || !gy || !gz || !adc)
            fail(MRSIM_EINVAL, "NULL sequence array");
        MRSIM_CUDA(cudaSetDevice(c->device));
        s->ctx = c;
        s->uid = g_uid++;
        copy_segments(s.get(), n_seg, dt, rep, b1re, b1im, gx, gy, gz, adc);
        build_sequence(c, s.get());
    });
    if (rc == MRSIM_OK) *out = s.release();
    return rc;
}

int mrsim_classify(int64_t n_seg, const double *dt, const int32_t *rep, const float *b1re,
                   const float *b1im, const float *gx, const float *gy, const float *gz,
                   const uint8_t *adc, unsigned flags, int64_t cap, int64_t *n_subseq,
                   uint8_t *type, uint8_t *gtype, int64_t *seg_begin, int64_t *seg_end,
                   int64_t *n_samples, int32_t *content_id) {
    if (!n_subseq) return MRSIM_EINVAL;
    *n_subseq = 0;
    if (n_seg <= 0 || !dt || !rep || !b1re || !b1im || !gx || !gy || !gz || !adc ||
        (flags & ~MRSIM_CLASSIFY_TWO_AXIS))
        return MRSIM_EINVAL;
    try {
        mrsim_seq s;
        copy_segments(&s, n_seg, dt, rep, b1re, b1im, gx, gy, gz, adc);
        classify_sequence(&s, (flags & MRSIM_CLASSIFY_TWO_AXIS) != 0);
        const int64_t m = (int64_t)s.sub.size();
        *n_subseq = m;
        if (m > cap) return MRSIM_OK;
        for (int64_t i = 0; i < m; ++i) {
            const Subseq &q = s.sub[i];
            if (type) type[i] = (uint8_t)q.type;
            if (gtype) gtype[i] = (uint8_t)q.gtype;
            if (seg_begin) seg_begin[i] = q.seg_begin;
            if (seg_end) seg_end[i] = q.seg_end;
            if (n_samples) n_samples[i] = q.n_samples;
            if (content_id) content_id[i] = q.content;
        }
        return MRSIM_OK;
    } catch (const Error &e) {
        return e.code;
    } catch (const std::bad_alloc &) {
        return MRSIM_ENOMEM;
    }
}

int mrsim_seq_info(const mrsim_seq *s, int64_t *n_subseq, uint8_t *type, uint8_t *gtype,
                   int64_t *seg_begin, int64_t *seg_end, int64_t *n_samples_total) {
    if (!s) return MRSIM_EINVAL;
    if (n_subseq) *n_subseq = (int64_t)s->sub.size();
    if (n_samples_total) *n_samples_total = s->n_samples;
    for (size_t i = 0; i < s->sub.size(); ++i) {
        if (type) type[i] = (uint8_t)s->sub[i].type;
        if (gtype) gtype[i] = (uint8_t)s->sub[i].gtype;
        if (seg_begin) seg_begin[i] = s->sub[i].seg_begin;
        if (seg_end) seg_end[i] = s->sub[i].seg_end;
    }
    return MRSIM_OK;
}

int mrsim_group(mrsim_ctx *c, const mrsim_phantom_t *ph, const mrsim_seq *s, mrsim_groups **out) {
    if (!c || !out) return MRSIM_EINVAL;
    *out = nullptr;
    auto g = std::unique_ptr<mrsim_groups>(new (std::nothrow) mrsim_groups());
    if (!g) return set_err(c, MRSIM_ENOMEM, "host allocation failed");
    int rc = guard(c, [&] {
        if (!ph || !s) fail(MRSIM_EINVAL, "NULL phantom or sequence");
        phantom_ready(c, ph);
        MRSIM_CUDA(cudaSetDevice(c->device));
        g->ctx = c;
        g->uid = g_uid++;
        g->phantom_uid = ph->uid;
        g->K = ph->K;
        int cnt_rf[kNTypes] = {}, cnt_adc[kNTypes] = {};
        for (const Subseq &q : s->sub) {
            if (q.type == SUB_RF) cnt_rf[q.gtype]++;
            if (q.type == SUB_ADC) cnt_adc[q.gtype]++;
        }
        const int rf_t = most_frequent(cnt_rf), adc_t = most_frequent(cnt_adc);
        g->primary = adc_t >= 0 ? adc_t : (rf_t >= 0 ? rf_t : G_NONE);
        g->secondary = (rf_t >= 0 && rf_t != g->primary) ? rf_t : -1;
        bool need[kNTypes] = {};
        for (int t = 0; t < kNTypes; ++t)
            need[t] = t != G_GENERAL && (cnt_rf[t] > 0 || cnt_adc[t] > 0);
        need[g->primary] = true;
        for (int t = 0; t < kNTypes; ++t) {
            if (!need[t]) continue;
            build_group_type(c, ph, t, g->gid_orig[t], g->n_groups[t], g->tab[t]);
            g->built[t] = true;
        }
        build_layout(c, ph, g.get());
        build_axis_index(c, g.get());
    });
    if (rc == MRSIM_OK) *out = g.release();
    return rc;
}

int mrsim_group_info(const mrsim_groups *g, int gtype, int64_t *n_groups, int32_t *gid) {
    if (!g || gtype < 0 || gtype >= kNTypes || !g->built[gtype]) return MRSIM_EINVAL;
    if (n_groups) *n_groups = g->n_groups[gtype];
    if (gid) {
        if (cudaMemcpyAsync(gid, g->gid_orig[gtype].p, g->K * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, g->ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(g->ctx->stream) != cudaSuccess)
            return MRSIM_ECUDA;
    }
    return MRSIM_OK;
}

int mrsim_run(mrsim_ctx *c, const mrsim_phantom_t *ph, const mrsim_seq *s,
              const mrsim_groups *g, int mode, int precision, double *signal, float *M_final,
              unsigned out_flags) {
    if (!c) return MRSIM_EINVAL;
    return guard(c, [&] {
        if (!ph || !s || !signal) fail(MRSIM_EINVAL, "NULL phantom, sequence or signal");
        phantom_ready(c, ph);
        if (precision != MRSIM_FP32 && precision != MRSIM_FP64) fail(MRSIM_EINVAL, "bad precision");
        if (mode < MRSIM_PLAIN || mode > MRSIM_SURROGATE) fail(MRSIM_EINVAL, "bad mode");
        const bool grouped = mode == MRSIM_GROUPED || mode == MRSIM_SURROGATE;
        if (grouped) {
            if (!g) fail(MRSIM_EINVAL, "grouped mode needs groups");
            if (g->phantom_uid != ph->uid) fail(MRSIM_ESTATE, "groups belong to another phantom");
            for (const Subseq &q : s->sub)
                if ((q.type == SUB_RF || q.type == SUB_ADC) && q.gtype != G_GENERAL &&
                    !g->built[q.gtype])
                    fail(MRSIM_ESTATE, "groups lack a gradient type the sequence uses");
        }
        MRSIM_CUDA(cudaSetDevice(c->device));
        const int64_t K = ph->K, ns = s->n_samples;
        const int64_t nsig = std::max<int64_t>(ns, 1) * std::max(ph->n_coils, 1);  // all coils
        const bool dev_out = (out_flags & MRSIM_OUT_DEVICE) != 0;
        double *d_sig = dev_out ? signal : (double *)scratch(c, 8, nsig * 2 * sizeof(double));
        MRSIM_CUDA(cudaMemsetAsync(d_sig, 0, nsig * 2 * sizeof(double), c->stream));
        // reproducible sums: the signal and block-sum buffers hold integers
        // rint(v fx) during the run, fx = 2^e with 2^56 above any sum's bound
        // (room for 128 times the bound), converted back at the end
        struct FxScope {
            mrsim_ctx *c;
            ~FxScope() { c->fx = 0.0; }
        } fx_scope{c};
        c->fx = 0.0;
        if (c->repro) {
            int ex = 0;
            std::frexp(sum_bound(c, ph) * (1.0 + 1e-9) + 1.0, &ex);
            c->fx = std::ldexp(1.0, 56 - ex);
        }
        const size_t esz = precision == MRSIM_FP64 ? 8 : 4;
        const int64_t Kp = plane_stride(K);
        void *Mst = scratch(c, 9, 3 * Kp * esz);
        if (grouped) {
            if (precision == MRSIM_FP64) {
                if (mode == MRSIM_SURROGATE) fail(MRSIM_EINVAL, "the surrogate runs in FP32");
                run_grouped<double>(c, ph, s, g, d_sig, (double *)Mst);
            } else {
                run_grouped<float>(c, ph, s, g, d_sig, (float *)Mst, mode == MRSIM_SURROGATE);
            }
        } else {
            const bool cache = mode == MRSIM_PLAIN_CACHE;
            if (precision == MRSIM_FP64) run_plain<double>(c, ph, s, cache, d_sig, (double *)Mst);
            else run_plain<float>(c, ph, s, cache, d_sig, (float *)Mst);
        }
        if (M_final) {
            float *d_out = dev_out ? M_final : (float *)scratch(c, 10, 3 * K * sizeof(float));
            launch_gather_out(c, K, Mst, (char *)Mst + Kp * esz, (char *)Mst + 2 * Kp * esz,
                              esz == 8, grouped ? g->perm.as<int32_t>() : nullptr, d_out);
            if (!dev_out)
                MRSIM_CUDA(cudaMemcpyAsync(M_final, d_out, 3 * K * sizeof(float),
                                           cudaMemcpyDeviceToHost, c->stream));
            sync(c);
        }
        if (c->fx > 0.0) launch_fixed_to_double(c, d_sig, nsig * 2, c->fx);
        if (!dev_out && ns > 0)
            MRSIM_CUDA(cudaMemcpyAsync(signal, d_sig, ns * std::max(ph->n_coils, 1) * 2 *
                                                          sizeof(double),
                                       cudaMemcpyDeviceToHost, c->stream));
        sync(c);
    });
}

int mrsim_set_reproducible(mrsim_ctx *c, int on) {
    if (!c) return MRSIM_EINVAL;
    if (on != 0 && on != 1) return set_err(c, MRSIM_EINVAL, "reproducible is 0 or 1");
    c->repro = on;
    return MRSIM_OK;
}

int mrsim_get_reproducible(const mrsim_ctx *c, int *on) {
    if (!c || !on) return MRSIM_EINVAL;
    *on = c->repro;
    return MRSIM_OK;
}

int mrsim_run_batch(mrsim_ctx *c, int n_jobs, const mrsim_phantom_t *const *ph,
                    const mrsim_seq *const *s, const mrsim_groups *const *g,
                    double *const *signals) {
    if (!c) return MRSIM_EINVAL;
    return guard(c, [&] {
        if (n_jobs <= 0 || !ph || !s || !g || !signals) fail(MRSIM_EINVAL, "bad batch arguments");
        for (int i = 0; i < n_jobs; ++i) {
            if (!ph[i] || !s[i] || !g[i] || !signals[i]) fail(MRSIM_EINVAL, "NULL batch entry");
            phantom_ready(c, ph[i]);
            if (g[i]->phantom_uid != ph[i]->uid) fail(MRSIM_ESTATE, "groups of another phantom");
            for (const Subseq &q : s[i]->sub)
                if ((q.type == SUB_RF || q.type == SUB_ADC) && q.gtype != G_GENERAL &&
                    !g[i]->built[q.gtype])
                    fail(MRSIM_ESTATE, "groups lack a gradient type the sequence uses");
        }
        MRSIM_CUDA(cudaSetDevice(c->device));
        run_batch(c, n_jobs, ph, s, g, signals);
    });
}

int mrsim_set_tuning(mrsim_ctx *c, int param, int value) {
    if (!c) return MRSIM_EINVAL;
    static const int allowed[8][8] = {{1, 2, 4, -1, -1, -1, -1, -1},
                                      {1, 2, -1, -1, -1, -1, -1, -1},
                                      {1, 2, 4, 8, -1, -1, -1, -1},
                                      {0, 1, 2, 4, 8, 16, 32, 128},
                                      {1, 2, 4, 8, 16, 32, -1, -1},
                                      {0, 4, 8, -1, -1, -1, -1, -1},
                                      {0, 1, -1, -1, -1, -1, -1, -1},
                                      {0, 1, 2, -1, -1, -1, -1, -1}};
    if (param < 0 || param > 7) return set_err(c, MRSIM_EINVAL, "unknown tuning parameter");
    bool ok = false;
    for (int v : allowed[param]) ok |= v >= 0 && v == value;
    if (!ok) return set_err(c, MRSIM_EINVAL, "value not allowed for this tuning parameter");
    c->tune[param] = value;
    return MRSIM_OK;
}

int mrsim_get_tuning(const mrsim_ctx *c, int param, int *value) {
    if (!c || !value || param < 0 || param > 7) return MRSIM_EINVAL;
    *value = c->tune[param];
    return MRSIM_OK;
}

int mrsim_autotune(mrsim_ctx *c, const mrsim_phantom_t *ph, const mrsim_seq *s,
                   const mrsim_groups *g, int mode, int precision, int reps) {
    if (!c) return MRSIM_EINVAL;
    return guard(c, [&] {
        if (!ph || !s) fail(MRSIM_EINVAL, "NULL phantom or sequence");
        phantom_ready(c, ph);
        if (reps < 1) reps = 1;
        const int64_t ns = std::max<int64_t>(s->n_samples, 1);
        DBuf sig = dalloc(ns * 2 * sizeof(double));
        cudaEvent_t e0, e1;
        MRSIM_CUDA(cudaEventCreate(&e0));
        MRSIM_CUDA(cudaEventCreate(&e1));
        // one parameter at a time, in the order they matter for the mode
        const bool grouped = mode == MRSIM_GROUPED || mode == MRSIM_SURROGATE;
        std::vector<std::pair<int, std::vector<int>>> plan;
        if (grouped && precision == MRSIM_FP32) plan.push_back({MRSIM_TUNE_CELL_NI, {4, 8, 0}});
        if (grouped && precision == MRSIM_FP32) plan.push_back({MRSIM_TUNE_CELL_ROWS, {0, 2}});
        if (grouped) plan.push_back({MRSIM_TUNE_FUSED_NI, {1, 2, 4}});
        if (grouped) plan.push_back({MRSIM_TUNE_PRECOMP_STEPS, {1, 2, 4, 8, 16, 32}});
        if (grouped) plan.push_back({MRSIM_TUNE_PRECOMP_LANES, {0, 1, 2, 4, 8, 16, 32, 128}});
        plan.push_back({MRSIM_TUNE_PLAIN_RF_NI, {1, 2}});
        plan.push_back({MRSIM_TUNE_ADC_CTAS_PER_SM, {1, 2, 4, 8}});
        for (auto &pv : plan) {
            float best = 1e30f;
            int best_v = c->tune[pv.first];
            for (int v : pv.second) {
                c->tune[pv.first] = v;
                // a warm-up run, then the timed repetitions
                int rc = mrsim_run(c, ph, s, g, mode, precision, sig.as<double>(), nullptr,
                                   MRSIM_OUT_DEVICE);
                if (rc) fail(rc, c->err);
                MRSIM_CUDA(cudaEventRecord(e0, c->stream));
                for (int r = 0; r < reps; ++r) {
                    rc = mrsim_run(c, ph, s, g, mode, precision, sig.as<double>(), nullptr,
                                   MRSIM_OUT_DEVICE);
                    if (rc) fail(rc, c->err);
                }
                MRSIM_CUDA(cudaEventRecord(e1, c->stream));
                MRSIM_CUDA(cudaEventSynchronize(e1));
                float ms = 0;
                MRSIM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) { best = ms; best_v = v; }
            }
            c->tune[pv.first] = best_v;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    });
}

int mrsim_profile_enable(mrsim_ctx *c, int on) {
    if (!c) return MRSIM_EINVAL;
    c->prof_on = on != 0;
    return MRSIM_OK;
}

int mrsim_profile_reset(mrsim_ctx *c) {
    if (!c) return MRSIM_EINVAL;
    cudaStreamSynchronize(c->stream);
    prof_flush(c);
    std::fill(c->prof_count.begin(), c->prof_count.end(), 0);
    std::fill(c->prof_ms.begin(), c->prof_ms.end(), 0.0);
    return MRSIM_OK;
}

int mrsim_profile_get(mrsim_ctx *c, int i, char *name, int cap, int64_t *launches, double *ms) {
    if (!c || i < 0 || i >= (int)c->prof_names.size()) return MRSIM_EINVAL;
    if (name && cap > 0) {
        std::snprintf(name, (size_t)cap, "%s", c->prof_names[i].c_str());
    }
    if (launches) *launches = c->prof_count[i];
    if (ms) *ms = c->prof_ms[i];
    return MRSIM_OK;
}

int64_t mrsim_launch_count(const mrsim_ctx *c) { return c ? c->launches : 0; }

void mrsim_free_phantom(mrsim_phantom_t *ph) {
    if (!ph) return;
    if (ph->ctx) cudaSetDevice(ph->ctx->device);
    delete ph;
}

void mrsim_free_seq(mrsim_seq *s) {
    if (!s) return;
    if (s->ctx) cudaSetDevice(s->ctx->device);
    delete s;
}

void mrsim_free_groups(mrsim_groups *g) {
    if (!g) return;
    if (g->ctx) cudaSetDevice(g->ctx->device);
    delete g;
}

}  // extern "C"
