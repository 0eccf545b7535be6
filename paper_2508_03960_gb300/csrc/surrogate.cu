// Host side of the learned with-RF transitions: training loop, validation
// grid, use inside grouped runs, and the C ABI of the surrogate handle.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>

#include "internal.h"

struct mrsim_surrogate {
    mrsim_ctx *ctx = nullptr;
    struct Net {
        // the pulse it was trained on (segments of the with-RF content)
        std::vector<double> dt;
        std::vector<int32_t> rep;
        std::vector<float> b1re, b1im, gx, gy, gz;
        mrsim::DBuf P, W2b, W2Tb, cell_ok;  // FP32 parameters, BF16 W2 copies, u8 cells
        mrsim::SurPulse pulse{};            // precession removed from the targets
        double loss = 0, val_max = 0, cells_ok = 0, val_accept = 0, val_accept_max = 0;
    };
    std::vector<Net> nets;
    mrsim::SurDomain dom{};
    double bound = 1e-3;
};

namespace mrsim {
namespace {

// Glorot-normal initial weights, zero biases (flat layout of the network)
std::vector<float> init_params(uint64_t seed) {
    std::mt19937_64 rng(seed);
    std::vector<float> p(sur_n_params(), 0.0f);
    auto fill = [&](int off, int fan_out, int fan_in) {
        std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / (fan_in + fan_out)));
        for (int i = 0; i < fan_out * fan_in; ++i) p[off + i] = (float)nd(rng);
    };
    fill(0, 128, 5);
    fill(128 * 5 + 128, 128, 128);
    fill(128 * 5 + 128 + 128 * 128 + 128, 12, 128);
    return p;
}

bool same_content(const mrsim_surrogate::Net &n, const mrsim_seq *s, int cid) {
    const Subseq &q = s->sub[s->content_first[cid]];
    const int64_t len = q.seg_end - q.seg_begin;
    if ((int64_t)n.dt.size() != len) return false;
    for (int64_t t = 0; t < len; ++t) {
        const int64_t j = q.seg_begin + t;
        if (n.dt[t] != s->dt[j] || n.rep[t] != s->rep[j] || n.b1re[t] != s->b1re[j] ||
            n.b1im[t] != s->b1im[j] || n.gx[t] != s->gx[j] || n.gy[t] != s->gy[j] ||
            n.gz[t] != s->gz[j])
            return false;
    }
    return true;
}

PrecompArgs exact_args(const mrsim_seq *s, int cid, int64_t G, const double *par, double *out) {
    const Subseq &q = s->sub[s->content_first[cid]];
    return PrecompArgs{s->rf_d[cid].p, s->rf_off[cid].as<int64_t>(), (int)(q.seg_end - q.seg_begin),
                       s->content_steps[cid], G_Z, G, par, out};
}

}  // namespace

bool sur_table(mrsim_ctx *c, const mrsim_seq *s, const mrsim_groups *g, int cid, int gtype,
               float *out) {
    const mrsim_surrogate *S = c->sur;
    if (!S || gtype != G_Z) return false;
    const mrsim_surrogate::Net *net = nullptr;
    for (const auto &n : S->nets)
        if (same_content(n, s, cid)) { net = &n; break; }
    if (!net) return false;
    const int64_t G = g->n_groups[G_Z];
    int32_t *fb = (int32_t *)scratch(c, 4, std::max<int64_t>(2 * G, 1) * sizeof(int32_t));
    int32_t *fb_n = (int32_t *)scratch(c, 3, 64);  // [fallback count, served count]
    MRSIM_CUDA(cudaMemsetAsync(fb_n, 0, 2 * sizeof(int32_t), c->stream));
    const double *par = g->tab[G_Z].d_par64.as<double>();
    sur_infer(c, net->P.as<float>(), net->W2b.p, S->dom, net->pulse,
              net->cell_ok.as<unsigned char>(), par, G, out, fb, fb_n);
    // exact integration (Eq. 7, FP32 steps composed in FP64) of the fallback groups
    const Subseq &q = s->sub[s->content_first[cid]];
    PrecompArgs pa{s->rf_f[cid].p, s->rf_off[cid].as<int64_t>(), (int)(q.seg_end - q.seg_begin),
                   s->content_steps[cid], G_Z, G, par, out};
    pa.gidx = fb;
    pa.gcount = fb_n;
    launch_precompute<float>(c, pa);
    int32_t h = 0;
    MRSIM_CUDA(cudaMemcpyAsync(&h, fb_n, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    MRSIM_CUDA(cudaStreamSynchronize(c->stream));
    c->sur_groups += G - h;
    c->sur_fallback += h;
    return true;
}

}  // namespace mrsim

using namespace mrsim;

namespace {

template <class F>
int sguard(mrsim_ctx *c, F &&f) {
    CtxScope scope(c);
    try {
        f();
        if (c) c->err.clear();
        return MRSIM_OK;
    } catch (const Error &e) {
        if (c) c->err = e.msg;
        return e.code;
    } catch (const std::bad_alloc &) {
        if (c) c->err = "host allocation failed";
        return MRSIM_ENOMEM;
    }
}

}  // namespace

extern "C" {

int mrsim_surrogate_train(mrsim_ctx *c, const mrsim_seq *s, const double *lo, const double *hi,
                          int64_t n_train, int epochs, int batch, double lr, uint64_t seed,
                          double bound, mrsim_surrogate **out) {
    if (!c || !out) return MRSIM_EINVAL;
    *out = nullptr;
    auto S = std::unique_ptr<mrsim_surrogate>(new (std::nothrow) mrsim_surrogate());
    if (!S) return MRSIM_ENOMEM;
    int rc = sguard(c, [&] {
        if (!s || !lo || !hi || n_train < 1024 || epochs < 1 || batch < 64 || !(bound > 0) ||
            !(lr > 0))
            fail(MRSIM_EINVAL, "bad surrogate training arguments");
        for (int a = 0; a < 5; ++a)
            if (!(hi[a] > lo[a]) || !std::isfinite(lo[a]) || !std::isfinite(hi[a]))
                fail(MRSIM_EINVAL, "empty training domain");
        if (!(lo[3] > 0) || !(lo[4] > 0)) fail(MRSIM_EINVAL, "T1 and T2 ranges must be positive");
        MRSIM_CUDA(cudaSetDevice(c->device));
        S->ctx = c;
        S->bound = bound;
        for (int a = 0; a < 5; ++a) { S->dom.lo[a] = lo[a]; S->dom.hi[a] = hi[a]; }
        batch = (batch + 63) / 64 * 64;
        n_train = std::max<int64_t>(batch, n_train / batch * batch);
        const int64_t n_val = std::max<int64_t>(65536, n_train / 4);
        const int NP = sur_n_params();
        // device buffers shared by the networks
        DBuf par = dalloc(5 * std::max(n_train, n_val) * sizeof(double));
        DBuf X = dalloc(5 * std::max(n_train, n_val) * sizeof(float));
        DBuf Td = dalloc(12 * std::max(n_train, n_val) * sizeof(double));
        DBuf T = dalloc(12 * std::max(n_train, n_val) * sizeof(float));
        DBuf Y = dalloc(12 * n_val * sizeof(float));
        DBuf grad = dalloc(NP * sizeof(float)), m = dalloc(NP * sizeof(float)),
             v = dalloc(NP * sizeof(float));
        DBuf loss = dalloc(sizeof(double));
        DBuf cell_err = dalloc(kCells * sizeof(unsigned int));
        for (int cid = 0; cid < s->n_content; ++cid) {
            const Subseq &q = s->sub[s->content_first[cid]];
            if (q.gtype != G_Z) continue;  // slice-selective pulses only
            mrsim_surrogate::Net net;
            for (int64_t j = q.seg_begin; j < q.seg_end; ++j) {
                net.pulse.mz += (double)s->gz[j] * s->dt[j] * s->rep[j];
                net.pulse.dur += s->dt[j] * s->rep[j];
                net.dt.push_back(s->dt[j]); net.rep.push_back(s->rep[j]);
                net.b1re.push_back(s->b1re[j]); net.b1im.push_back(s->b1im[j]);
                net.gx.push_back(s->gx[j]); net.gy.push_back(s->gy[j]); net.gz.push_back(s->gz[j]);
            }
            // training set: exact transitions of random parameter draws
            sur_sample(c, S->dom, seed + 1000ull * cid, n_train, par.as<double>(), X.as<float>());
            launch_precompute<double>(c, exact_args(s, cid, n_train, par.as<double>(), Td.as<double>()));
            sur_core(c, net.pulse, par.as<double>(), n_train, Td.as<double>(), T.as<float>());
            std::vector<float> p0 = init_params(seed + 17 + cid);
            net.P = dalloc(NP * sizeof(float));
            net.W2b = dalloc(128 * 128 * 2);
            net.W2Tb = dalloc(128 * 128 * 2);
            upload(c, net.P.p, p0.data(), NP * sizeof(float));
            MRSIM_CUDA(cudaMemsetAsync(grad.p, 0, NP * sizeof(float), c->stream));
            MRSIM_CUDA(cudaMemsetAsync(m.p, 0, NP * sizeof(float), c->stream));
            MRSIM_CUDA(cudaMemsetAsync(v.p, 0, NP * sizeof(float), c->stream));
            sur_bf16_copies(c, net.P.as<float>(), net.W2b.p, net.W2Tb.p);
            const int64_t steps = n_train / batch;
            const int64_t total = steps * epochs;
            const double lr0 = lr, lr1 = lr * 1e-2;
            int64_t it = 0;
            double last = 0;
            sur_tensor_err_reset(c);
            for (int ep = 0; ep < epochs; ++ep) {
                MRSIM_CUDA(cudaMemsetAsync(loss.p, 0, sizeof(double), c->stream));
                for (int64_t st = 0; st < steps; ++st, ++it) {
                    const double lr = lr1 + 0.5 * (lr0 - lr1) * (1.0 + std::cos(M_PI * it / total));
                    sur_train_step(c, net.P.as<float>(), net.W2b.p, net.W2Tb.p,
                                   X.as<float>() + 5 * st * batch, T.as<float>() + 12 * st * batch,
                                   batch, grad.as<float>(), loss.as<double>(), nullptr);
                    sur_adam(c, net.P.as<float>(), grad.as<float>(), m.as<float>(), v.as<float>(),
                             (int)(it + 1), (float)lr, net.W2b.p, net.W2Tb.p);
                }
                double h = 0;
                MRSIM_CUDA(cudaMemcpyAsync(&h, loss.p, sizeof(double), cudaMemcpyDeviceToHost,
                                           c->stream));
                sync(c);
                sur_tensor_err_check(c);
                last = h / (12.0 * (double)n_train);
            }
            net.loss = last;
            // validation set (new draws): largest error per (z, dB0, b1) cell
            sur_sample(c, S->dom, seed + 1000ull * cid + 500, n_val, par.as<double>(), X.as<float>());
            launch_precompute<double>(c, exact_args(s, cid, n_val, par.as<double>(), Td.as<double>()));
            // validation compares full transitions (the quantity the gate bounds)
            sur_core(c, SurPulse{0.0, 0.0}, par.as<double>(), n_val, Td.as<double>(), T.as<float>());
            DBuf idx = dalloc(2 * n_val * sizeof(int32_t));
            DBuf cnt = dalloc(2 * sizeof(int32_t));
            MRSIM_CUDA(cudaMemsetAsync(cnt.p, 0, 2 * sizeof(int32_t), c->stream));
            sur_infer(c, net.P.as<float>(), net.W2b.p, S->dom, net.pulse, nullptr,
                      par.as<double>(), n_val, Y.as<float>(), idx.as<int32_t>(), cnt.as<int32_t>());
            MRSIM_CUDA(cudaMemsetAsync(cell_err.p, 0, kCells * sizeof(unsigned int), c->stream));
            sur_cell_error(c, S->dom, par.as<double>(), n_val, Y.as<float>(), T.as<float>(),
                           cell_err.as<unsigned int>());
            std::vector<unsigned int> ce(kCells);
            MRSIM_CUDA(cudaMemcpyAsync(ce.data(), cell_err.p, kCells * sizeof(unsigned int),
                                       cudaMemcpyDeviceToHost, c->stream));
            sync(c);
            std::vector<unsigned char> okc(kCells);
            int n_ok = 0;
            double vmax = 0, amax = 0;
            for (int i = 0; i < kCells; ++i) {
                float e;
                std::memcpy(&e, &ce[i], 4);
                vmax = std::max(vmax, (double)e);
                // cells without samples stay exact
                okc[i] = (ce[i] != 0u) && (double)e <= kGateMargin * bound;
                if (okc[i]) { ++n_ok; amax = std::max(amax, (double)e); }
            }
            net.val_max = vmax;
            net.cells_ok = (double)n_ok / kCells;
            net.val_accept = net.cells_ok;  // cells are equal-volume and sampled uniformly
            net.val_accept_max = amax;
            net.cell_ok = dalloc(kCells);
            upload(c, net.cell_ok.p, okc.data(), kCells);
            sync(c);
            S->nets.push_back(std::move(net));
        }
        if (S->nets.empty()) fail(MRSIM_EINVAL, "the sequence has no slice-selective with-RF pulse");
    });
    if (rc == MRSIM_OK) *out = S.release();
    return rc;
}

int mrsim_surrogate_check(mrsim_ctx *c, const mrsim_surrogate *S, const mrsim_seq *s,
                          const mrsim_groups *g, double *max_err, int64_t *n_served) {
    if (!c) return MRSIM_EINVAL;
    return sguard(c, [&] {
        if (!S || !s || !g || !max_err) fail(MRSIM_EINVAL, "NULL argument");
        if (!g->built[G_Z]) fail(MRSIM_ESTATE, "the groups have no Gz-only type");
        MRSIM_CUDA(cudaSetDevice(c->device));
        const int64_t G = g->n_groups[G_Z];
        const double *par = g->tab[G_Z].d_par64.as<double>();
        DBuf out = dalloc(std::max<int64_t>(G, 1) * 12 * sizeof(float));
        DBuf exact = dalloc(std::max<int64_t>(G, 1) * 12 * sizeof(double));
        DBuf idx = dalloc(std::max<int64_t>(2 * G, 1) * sizeof(int32_t));
        DBuf cnt = dalloc(2 * sizeof(int32_t));
        DBuf res = dalloc(sizeof(unsigned int));
        MRSIM_CUDA(cudaMemsetAsync(res.p, 0, sizeof(unsigned int), c->stream));
        int64_t served = 0;
        for (int cid = 0; cid < s->n_content; ++cid) {
            const Subseq &q = s->sub[s->content_first[cid]];
            if (q.type != SUB_RF || q.gtype != G_Z) continue;
            const mrsim_surrogate::Net *net = nullptr;
            for (const auto &n : S->nets)
                if (same_content(n, s, cid)) { net = &n; break; }
            if (!net) continue;
            MRSIM_CUDA(cudaMemsetAsync(cnt.p, 0, 2 * sizeof(int32_t), c->stream));
            sur_infer(c, net->P.as<float>(), net->W2b.p, S->dom, net->pulse,
                      net->cell_ok.as<unsigned char>(), par, G, out.as<float>(),
                      idx.as<int32_t>(), cnt.as<int32_t>());
            // the exact transitions (FP64 steps and composition) of the served groups
            PrecompArgs pa = exact_args(s, cid, G, par, exact.as<double>());
            pa.gidx = idx.as<int32_t>() + G;
            pa.gcount = cnt.as<int32_t>() + 1;
            launch_precompute<double>(c, pa);
            sur_served_error(c, out.as<float>(), exact.as<double>(), idx.as<int32_t>() + G,
                             cnt.as<int32_t>() + 1, res.as<unsigned int>());
            int32_t h[2] = {0, 0};
            MRSIM_CUDA(cudaMemcpyAsync(h, cnt.p, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                       c->stream));
            sync(c);
            served += h[1];
        }
        unsigned int r = 0;
        MRSIM_CUDA(cudaMemcpyAsync(&r, res.p, sizeof(r), cudaMemcpyDeviceToHost, c->stream));
        sync(c);
        float e;
        std::memcpy(&e, &r, sizeof(e));
        *max_err = (double)e;
        if (n_served) *n_served = served;
    });
}

int mrsim_surrogate_stats(const mrsim_surrogate *S, const mrsim_ctx *c, double *out) {
    if (!S || !out) return MRSIM_EINVAL;
    double loss = 0, vmax = 0, ok = 0, acc = 0, amax = 0;
    for (const auto &n : S->nets) {
        loss += n.loss / S->nets.size();
        vmax = std::max(vmax, n.val_max);
        ok += n.cells_ok / S->nets.size();
        acc += n.val_accept / S->nets.size();
        amax = std::max(amax, n.val_accept_max);
    }
    out[0] = (double)S->nets.size();
    out[1] = loss;
    out[2] = vmax;
    out[3] = ok;
    out[4] = acc;
    out[5] = amax;
    out[6] = c ? (double)c->sur_groups : 0.0;
    out[7] = c ? (double)c->sur_fallback : 0.0;
    return MRSIM_OK;
}

int mrsim_surrogate_use(mrsim_ctx *c, const mrsim_surrogate *S) {
    if (!c) return MRSIM_EINVAL;
    c->sur = S;
    c->sur_groups = 0;
    c->sur_fallback = 0;
    return MRSIM_OK;
}

int mrsim_surrogate_eval(mrsim_ctx *c, const float *params, int64_t n, const float *x,
                         const float *t, float *y, float *grad_out, double *loss_out) {
    if (!c) return MRSIM_EINVAL;
    return sguard(c, [&] {
        if (!params || !x || !t || n < 1) fail(MRSIM_EINVAL, "bad arguments");
        MRSIM_CUDA(cudaSetDevice(c->device));
        const int NP = sur_n_params();
        DBuf P = dalloc(NP * 4), W2b = dalloc(128 * 128 * 2), W2Tb = dalloc(128 * 128 * 2);
        DBuf X = dalloc(n * 5 * 4), T = dalloc(n * 12 * 4), Y = dalloc(n * 12 * 4);
        DBuf g = dalloc(NP * 4), L = dalloc(8);
        upload(c, P.p, params, NP * 4);
        upload(c, X.p, x, n * 5 * 4);
        upload(c, T.p, t, n * 12 * 4);
        MRSIM_CUDA(cudaMemsetAsync(g.p, 0, NP * 4, c->stream));
        MRSIM_CUDA(cudaMemsetAsync(L.p, 0, 8, c->stream));
        sur_bf16_copies(c, P.as<float>(), W2b.p, W2Tb.p);
        sur_tensor_err_reset(c);
        sur_train_step(c, P.as<float>(), W2b.p, W2Tb.p, X.as<float>(), T.as<float>(), n,
                       g.as<float>(), L.as<double>(), Y.as<float>());
        sur_tensor_err_check(c);
        if (y) MRSIM_CUDA(cudaMemcpyAsync(y, Y.p, n * 12 * 4, cudaMemcpyDeviceToHost, c->stream));
        if (grad_out)
            MRSIM_CUDA(cudaMemcpyAsync(grad_out, g.p, NP * 4, cudaMemcpyDeviceToHost, c->stream));
        double h = 0;
        MRSIM_CUDA(cudaMemcpyAsync(&h, L.p, 8, cudaMemcpyDeviceToHost, c->stream));
        sync(c);
        if (loss_out) *loss_out = h / (12.0 * (double)n);
    });
}

int mrsim_surrogate_infer(mrsim_ctx *c, const float *params, int64_t n, const float *x,
                          float *y) {
    if (!c) return MRSIM_EINVAL;
    return sguard(c, [&] {
        if (!params || !x || !y || n < 1) fail(MRSIM_EINVAL, "bad arguments");
        MRSIM_CUDA(cudaSetDevice(c->device));
        const int NP = sur_n_params();
        DBuf P = dalloc(NP * 4), W2b = dalloc(128 * 128 * 2), W2Tb = dalloc(128 * 128 * 2);
        DBuf X = dalloc(n * 5 * 4), Y = dalloc(n * 12 * 4);
        upload(c, P.p, params, NP * 4);
        upload(c, X.p, x, n * 5 * 4);
        sur_bf16_copies(c, P.as<float>(), W2b.p, W2Tb.p);
        sur_infer_raw(c, P.as<float>(), W2b.p, X.as<float>(), n, Y.as<float>());
        MRSIM_CUDA(cudaMemcpyAsync(y, Y.p, n * 12 * 4, cudaMemcpyDeviceToHost, c->stream));
        sync(c);
    });
}

void mrsim_free_surrogate(mrsim_surrogate *S) {
    if (!S) return;
    if (S->ctx) {
        cudaSetDevice(S->ctx->device);
        if (S->ctx->sur == S) S->ctx->sur = nullptr;
    }
    delete S;
}

}  // extern "C"
