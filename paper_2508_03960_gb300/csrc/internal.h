// Host-side objects behind the C ABI handles, device buffers and the launch
// scope that counts kernels and (optionally) times them with CUDA events.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/mrsim.h"
#include "common.cuh"

namespace mrsim {

// Stream-ordered device memory pool of one context.  Buffers freed while the
// context lives go back to the pool in stream order (cudaFreeAsync on the
// context's stream) and are reused by later allocations on that stream
// without a device synchronisation; the pool keeps what it has reserved until
// the context is destroyed or an allocation would otherwise fail.  Once the
// context is gone (stream == nullptr), buffers that outlive it are freed with
// the synchronous cudaFree, and the pool itself goes with the last of them.
struct DevPool {
    cudaMemPool_t pool = nullptr;
    cudaStream_t stream = nullptr;
    DevPool() = default;
    DevPool(const DevPool &) = delete;
    DevPool &operator=(const DevPool &) = delete;
    ~DevPool() {
        if (pool) cudaMemPoolDestroy(pool);
    }
};

// Owned device allocation (from the pool of the context that made it, or
// from cudaMalloc where no pool applies).
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
    std::shared_ptr<DevPool> pool;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), bytes(o.bytes), pool(std::move(o.pool)) {
        o.p = nullptr;
        o.bytes = 0;
    }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) {
            reset();
            p = o.p;
            bytes = o.bytes;
            pool = std::move(o.pool);
            o.p = nullptr;
            o.bytes = 0;
        }
        return *this;
    }
    ~DBuf() { reset(); }
    void reset() {
        if (p) {
            if (pool && pool->stream)
                cudaFreeAsync(p, pool->stream);
            else
                cudaFree(p);
        }
        p = nullptr;
        bytes = 0;
        pool.reset();
    }
    template <typename T>
    T *as() const { return static_cast<T *>(p); }
};

// Error carrying a status code and message; thrown inside the library,
// caught at every ABI entry point.
struct Error {
    int code;
    std::string msg;
};

[[noreturn]] void fail(int code, const std::string &msg);
void cuda_check(cudaError_t e, const char *what);
#define MRSIM_CUDA(call) ::mrsim::cuda_check((call), #call)

}  // namespace mrsim

struct mrsim_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // stream-ordered pool of the context's device buffers
    std::shared_ptr<mrsim::DevPool> pool;
    std::string err;
    int64_t launches = 0;
    // profiling
    bool prof_on = false;
    std::vector<std::string> prof_names;
    std::vector<int64_t> prof_count;
    std::vector<double> prof_ms;
    struct Pending { int id; cudaEvent_t a, b; };
    std::vector<Pending> prof_pending;
    std::vector<cudaEvent_t> ev_pool;
    // growable scratch areas reused across calls
    mrsim::DBuf scratch[32];
    // error word written by kernels with bounded waits / bounds checks
    mrsim::DBuf dev_err;
    // pinned host staging for uploads of per-run plans
    void *pinned = nullptr;
    size_t pinned_bytes = 0;
    // active surrogate for MRSIM_SURROGATE runs and the counts of its last use
    const struct mrsim_surrogate *sur = nullptr;
    int64_t sur_groups = 0, sur_fallback = 0;
    // launch parameters chosen by mrsim_autotune (or mrsim_set_tuning)
    int tune[8] = {4, 2, 2, 0, 8, 8, 1, 0};  // indexed by the MRSIM_TUNE_* parameters
    // reproducible sums (mrsim_set_reproducible) and, during a run, the
    // fixed-point scale of the sum buffers (0: FP64 atomics)
    int repro = 0;
    double fx = 0.0;
};

struct mrsim_phantom_t {
    mrsim_ctx *ctx = nullptr;
    int64_t K = 0;
    uint64_t uid = 0;
    mrsim::DBuf x, y, z, T1, T2, dB0, M0, b1, M_init;  // b1 / M_init may be empty
    bool has_b1 = false, has_M_init = false;
    int n_coils = 0;    // receive coils attached by mrsim_coils (0: one coil, S = 1)
    mrsim::DBuf coils;  // float [n_coils][2][K] (re, im planes), phantom order
    double sum_bound = -1.0;  // bound on |any signal or block sum| (< 0: not formed yet)
    uint64_t coil_uid = 0;    // changes whenever mrsim_coils attaches or detaches coils
    // value checks of an upload queued without waiting (MRSIM_PHANTOM_ASYNC):
    // the device flag and whether it is still to be read (1), read and clear
    // (0) or read and set (2)
    mrsim::DBuf bad;
    cudaEvent_t checked = nullptr;  // recorded after the checks
    mutable int check = 0;
    ~mrsim_phantom_t() {
        if (checked) cudaEventDestroy(checked);
    }
};

namespace mrsim {

struct Subseq {
    int type = SUB_RELAX, gtype = G_NONE;
    int64_t seg_begin = 0, seg_end = 0;
    int64_t n_samples = 0, sample0 = 0;
    int content = -1;       // with-RF: content id (bit equality of all segment fields)
    double dur = 0.0;       // seconds
    double mom[3] = {0, 0, 0};  // int G dt over the subsequence (T s / m)
};

struct GroupTable {
    int64_t n = 0;
    DBuf d_par64;                    // [6][n] doubles: pos, T1, T2, dB0, b1, pos2 (pos2: the
                                     // second position of a two-axis type, else 0)
    DBuf d_pos, d_dB0, d_rT2, d_pos2;          // float copies for the group-signal kernel
    DBuf d_pos64, d_dB064, d_rT264, d_pos264;  // double copies for the group-signal kernel
};

}  // namespace mrsim

struct mrsim_seq {
    mrsim_ctx *ctx = nullptr;
    uint64_t uid = 0;
    int64_t n_seg = 0;
    std::vector<double> dt;
    std::vector<int32_t> rep;
    std::vector<float> b1re, b1im, gx, gy, gz;
    std::vector<uint8_t> adc;
    std::vector<mrsim::Subseq> sub;
    int64_t n_samples = 0;
    int n_content = 0;
    std::vector<int64_t> content_first;  // first subsequence of each content
    std::vector<int64_t> content_count;
    std::vector<int64_t> content_steps;  // sub-steps per content
    // device RF waveforms per content and their sub-step offsets [n_seg + 1]
    std::vector<mrsim::DBuf> rf_f, rf_d, rf_off;
    // ADC segments of every window (concatenated) and each subsequence's first one
    mrsim::DBuf adc_f, adc_d;
    std::vector<int64_t> adc_off;
    // per-sample (tau, k) since the start of its window, on the window's axis
    mrsim::DBuf gs_f, gs_d;
};

struct mrsim_groups {
    mrsim_ctx *ctx = nullptr;
    uint64_t uid = 0;
    uint64_t phantom_uid = 0;
    int64_t K = 0;
    // per gradient type (G_GENERAL, number 4, has none)
    bool built[mrsim::kNTypes] = {};
    int64_t n_groups[mrsim::kNTypes] = {};
    mrsim::DBuf gid_orig[mrsim::kNTypes];    // int32 [K], phantom order
    mrsim::DBuf gid_sorted[mrsim::kNTypes];  // int32 [K], layout order
    mrsim::GroupTable tab[mrsim::kNTypes];
    int primary = -1, secondary = -1;  // layout keys (gradient types)
    // the layout-order copies of the primary axis position, T1, T2, dB0, b1 and
    // the group ids are allocated but still to be gathered (ensure_layout_arrays)
    mutable bool rest_pending = false;
    int64_t n_cells = 0;
    // distinct positions of the two axes other than the primary one, numbered
    // by first occurrence in layout order; ax_idx packs both indices per
    // isochromat (lower axis in bits 0-15, higher axis in bits 16-31).
    // ax_ok is false if there is no primary axis or an axis has more than
    // kMaxAxisValues distinct positions.
    bool ax_ok = false;
    int64_t n_ax[3] = {0, 0, 0};
    mrsim::DBuf ax_val[3];  // float [n_ax[a]]
    mrsim::DBuf ax_idx;     // int32 [K], layout order
    // cells: maximal runs of one (primary gid, secondary gid) pair in the
    // layout, in layout order: first isochromat, count and both group ids
    mrsim::DBuf cell_start, cell_count, cell_gp, cell_gr;  // int32 [n_cells]
    // per-thread work of the cell-mode fused kernel for 4 and 8 isochromats
    // per thread: {first layout index, cell << 4 | count}; a cell of n
    // isochromats has ceil(n / NI) threads whose isochromats interleave with
    // stride ceil(n / NI) (a thread never straddles two cells)
    mrsim::DBuf cell_thr[2];
    int64_t n_cell_thr[2] = {0, 0};
    mrsim::DBuf perm;  // int32 [K]: layout position -> phantom index
    mrsim::DBuf x, y, z, T1, T2, dB0, M0, b1, M_init;  // layout order
    bool has_b1 = false, has_M_init = false;
};

namespace mrsim {

// Counts a kernel launch, names it with an NVTX range (host side, around the
// launch) and brackets it with events when profiling is on.
struct KScope {
    mrsim_ctx *c;
    int id = -1;
    cudaEvent_t a = nullptr, b = nullptr;
    KScope(mrsim_ctx *ctx, const char *name);
    ~KScope();
    KScope(const KScope &) = delete;
    KScope &operator=(const KScope &) = delete;
};

// after a synchronize: fold pending event pairs into the per-kernel totals
void prof_flush(mrsim_ctx *c);

// scratch area `slot` of at least `bytes` bytes (grows, contents undefined)
void *scratch(mrsim_ctx *c, int slot, size_t bytes);
// Device allocation from the pool of the context whose entry point runs on
// this thread (CtxScope), else from cudaMalloc.  Throws MRSIM_ENOMEM.
DBuf dalloc(size_t bytes);

// Marks the context whose entry point runs on this thread for the scope's
// lifetime (restores the previous one after).
struct CtxScope {
    mrsim_ctx *prev;
    explicit CtxScope(mrsim_ctx *c);
    ~CtxScope();
    CtxScope(const CtxScope &) = delete;
    CtxScope &operator=(const CtxScope &) = delete;
};
void upload(mrsim_ctx *c, void *dst, const void *src, size_t bytes);
void sync(mrsim_ctx *c);

// word of mrsim_ctx::dev_err set by the tensor-core kernels when a bounded
// mbarrier wait runs out (the other words belong to the group builder)
constexpr int kErrWordTensor = 4;

// ---- learned with-RF transitions (k_surrogate.cu, surrogate.cu) ----
struct SurDomain {
    double lo[5], hi[5];  // z (m), dB0 (Hz), b1, T1 (s), T2 (s)
};
struct SurPulse {
    double mz;   // int Gz dt over the pulse (T s / m)
    double dur;  // pulse duration (s)
};
// validation cells of the gate: z, dB0, b1 uniform, T2 log-uniform over the domain
constexpr int kCellsZ = 64, kCellsB0 = 8, kCellsB1 = 4, kCellsT2 = 4;
constexpr int kCells = kCellsZ * kCellsB0 * kCellsB1 * kCellsT2;
// a cell is served only if its validated largest error is at most this
// fraction of the bound (the validation draws cover a cell only so densely)
constexpr double kGateMargin = 0.5;
void sur_sample(mrsim_ctx *c, const SurDomain &d, uint64_t seed, int64_t n, double *par, float *X);
void sur_core(mrsim_ctx *c, const SurPulse &p, const double *par, int64_t n, const double *T,
              float *C);
void sur_bf16_copies(mrsim_ctx *c, const float *P, void *W2b, void *W2Tb);
void sur_train_step(mrsim_ctx *c, const float *P, const void *W2b, const void *W2Tb,
                    const float *X, const float *T, int64_t n, float *grad, double *loss,
                    float *Yout);
void sur_adam(mrsim_ctx *c, float *P, float *grad, float *m, float *v, int step, float lr,
              void *W2b, void *W2Tb);
// word kErrWordTensor of the context's error area: cleared before training,
// read (synchronising) after it; MRSIM_ETIMEOUT if a bounded wait ran out
void sur_tensor_err_reset(mrsim_ctx *c);
void sur_tensor_err_check(mrsim_ctx *c);
void sur_cell_error(mrsim_ctx *c, const SurDomain &d, const double *par, int64_t n,
                    const float *Y, const float *T, unsigned int *cell_err);
// Gate + network inference for the G groups of one table.  cell_ok == nullptr
// serves every group (validation); otherwise groups outside the domain or in a
// rejected cell go to the fallback list.  idx [2G]: fallback list, then served
// list; cnt [2] (zeroed by the caller): fallback count, served count.
void sur_infer(mrsim_ctx *c, const float *P, const void *W2b, const SurDomain &d,
               const SurPulse &pulse, const unsigned char *cell_ok, const double *par, int64_t G,
               float *out, int32_t *idx, int32_t *cnt);
int sur_n_params();
// the inference kernel on given features X [n][5]: raw outputs Y [n][12]
void sur_infer_raw(mrsim_ctx *c, const float *P, const void *W2b, const float *X, int64_t n,
                   float *Y);
// largest |entry| difference between out (float [G][12]) and exact (double
// [G][12]) over the groups listed in idx[0 .. *cnt); result as float bits
void sur_served_error(mrsim_ctx *c, const float *out, const double *exact, const int32_t *idx,
                      const int32_t *cnt, unsigned int *result);
// run-time use by the grouped planner: fills rows [0, G) of `out` for with-RF
// content `cid` of `s` from the context's active network, then integrates the
// fallback groups exactly; returns false if no network serves this content
bool sur_table(mrsim_ctx *c, const mrsim_seq *s, const mrsim_groups *g, int cid, int gtype,
               float *out);

// ---- group builder (k_group.cu) ----
void build_group_type(mrsim_ctx *c, const mrsim_phantom_t *ph, int gtype, DBuf &gid,
                      int64_t &n_groups, GroupTable &tab);
void build_layout(mrsim_ctx *c, const mrsim_phantom_t *ph, mrsim_groups *g);
// Gathers the layout-order arrays the group build left for later (the
// per-isochromat form, fallbacks, initial states and gid-reading events need
// them); ph is the phantom the groups were built from.  Queued on c's stream.
void ensure_layout_arrays(mrsim_ctx *c, const mrsim_groups *g, const mrsim_phantom_t *ph);
// Distinct keys (x[k], x[K + k], x[2K + k], bits of T1[k], bits of T2[k]) of K
// elements: id[k] in [0, U) numbered by first occurrence, table [3][U] of the
// integer words, tf [2][U] of T1 and T2, count [U] of occurrences.  Returns U.
// Uses scratch slots 0-5.
int64_t distinct_features(mrsim_ctx *c, int64_t K, const int32_t *x, const float *T1,
                          const float *T2, int32_t *id, DBuf &table, DBuf &tf, DBuf &count);
constexpr int64_t kMaxAxisValues = 65535;
// Group-reducing preprocessing (k_cluster.cu): fills `out` (a phantom with the
// cluster centre values and the refitted M0; positions, b1, M_init and coils
// copied), `labels` (device int32 [K]) and `centres` (host [n][3]: T1 s, T2 s,
// dB0 Hz, FP64) for the n <= n_clusters clusters made.  Arguments checked by
// the caller.
constexpr int64_t kMaxClusterK = 1LL << 28;
void cluster_phantom(mrsim_ctx *c, const mrsim_phantom_t *ph, int n_clusters,
                     const double scale[3], int max_iter, int n_echo, const double *te, double tr,
                     mrsim_phantom_t *out, DBuf &labels, std::vector<double> &centres);
void build_axis_index(mrsim_ctx *c, mrsim_groups *g);
// out[i] = in[perm[i]] for i < K (float32)
void launch_gather_f32(mrsim_ctx *c, int64_t K, const int32_t *perm, const float *in, float *out);

// ---- plain path (k_plain.cu) ----
struct PlainState {
    int64_t K;
    const float *x, *y, *z, *T1, *T2, *dB0, *M0, *b1;  // b1 may be null
    void *Mx, *My, *Mz;  // R arrays
    // receive-coil sensitivity (re, im planes, same order as x) for the with-ADC
    // kernels, or null for S = 1
    const float *coil_re = nullptr, *coil_im = nullptr;
    double fx = 0.0;  // fixed-point scale of the signal sums (0: FP64 atomics)
};
template <typename R>
void launch_init_state(mrsim_ctx *c, const PlainState &s, const float *M_init);
template <typename R>
void launch_plain_rf(mrsim_ctx *c, const PlainState &s, const void *segs, int n_seg,
                     const void *adv, int ni);
template <typename R>
void launch_plain_adc(mrsim_ctx *c, const PlainState &s, const void *segs, int n_seg,
                      int64_t n_samples, const void *adv, double *signal, int ctas_per_sm = 2);
// Reproducible sums: a bound on |any signal or block sum| of a run on the
// phantom, sum_k (|M0_k| + |M_init_k|) max(1, max_j |S_jk|) (the magnetisation
// never exceeds |M_init| + |M0| in norm), formed in a fixed order; and the
// in-place conversion of n fixed-point sums (integers i) to i / fx.
double sum_bound(mrsim_ctx *c, const mrsim_phantom_t *ph);
void launch_fixed_to_double(mrsim_ctx *c, double *buf, int64_t n, double fx);
template <typename R>
void launch_advance(mrsim_ctx *c, const PlainState &s, const void *adv);
template <typename R>
void launch_plain_rf_affine(mrsim_ctx *c, const PlainState &s, const void *segs, int n_seg,
                            R *cache);
template <typename R>
void launch_apply_affine(mrsim_ctx *c, const PlainState &s, const R *cache, const void *adv);
void launch_gather_out(mrsim_ctx *c, int64_t K, const void *Mx, const void *My, const void *Mz,
                       bool fp64, const int32_t *perm, float *out);

// ---- grouped path (k_grouped.cu) ----
struct PrecompArgs {
    const void *segs;        // RFSegF / RFSegD of one with-RF content
    const int64_t *seg_off;  // [n_seg + 1] first sub-step of each segment
    int n_seg;
    int64_t n_steps;
    int gtype;
    int64_t n_groups;
    const double *par;       // [5][n_groups]: pos, T1, T2, dB0, b1 (+ pos2 in row 5 for a
                             // two-axis type)
    void *out;               // R [n_groups][12]
    const int32_t *gidx = nullptr;    // optional: only the groups gidx[0 .. *gcount)
    const int32_t *gcount = nullptr;
    int kb = 8;                       // FP32 tables: sub-steps per FP32 register block
};
template <typename R>
void launch_precompute(mrsim_ctx *c, const PrecompArgs &a);

template <typename R>
struct FusedArgs {
    int64_t K;
    const float *x, *y, *z, *T1, *T2, *dB0, *M0;
    const int32_t *gid[kNTypes];  // layout-order gids per gradient type (null if not built)
    int gtype_p, gtype_r;    // ADC-sorted type, preferred RF type (-1: none)
    R *Mx, *My, *Mz;
    int init_eq;
    const FEvent<R> *ev;
    int n_ev;
    const R *T_tab;
    const void *P_raw;       // per-(event, primary group) advance factors, 4 R each
    double *Ablk;            // complex block sums (interleaved re, im)
    int direct;              // 1: no factor table, the whole advance per isochromat
    // axis tables (FP32 factor-table runs): per-isochromat phasors are read
    // from qtab at the event's offsets instead of being evaluated
    int ax;                  // 1: use them
    const int32_t *aidx;     // packed axis indices [K] (layout order)
    const float2 *qtab;      // phasor tables of all events
    int ax_sh[3];            // bit position of each axis' index in aidx
    // receive-coil sensitivity (re, im planes, layout order) or null for S = 1
    const float *coil_re, *coil_im;
    double fx;               // fixed-point scale of the block sums (0: FP64 atomics)
};
// Cell mode of the fused kernel (FP32): every thread holds isochromats of one
// cell, so the positions on the primary axis and (if any) the secondary axis,
// T1, T2, dB0 and b1 are the thread's own; only the phase on the remaining
// ("free") axes differs between its isochromats.  An RF event then applies one
// combined row C = T Adv per cell; a with-ADC event adds Q_free M_xy.  The
// rows are read from a table built per run, or (when cells are too many for
// it) formed by each thread from the transition and group-factor tables.
// Event record of the cell form (32 bytes), decoded on the host.
enum CellEvKind : int { CE_RF = 0, CE_END = 1, CE_ADC = 2, CE_ADC_OTHER = 3 };
struct CellEv {
    int kind;   // CellEvKind (CE_ADC: a window of the primary type)
    int row;    // RF / END: first combined row (key * n_cells), table form;
                // ADC: first group-factor row (event * G_primary)
    int win;    // ADC: offset of the window's block sums (complex entries);
                // RF / END: first transition row of the event's type (-1: END)
    int gtype;  // CE_ADC_OTHER: the window's gradient type; RF: the pulse's type
    int qf[2];  // free-axis phasor table offsets (lower axis first)
    int qr;     // secondary-axis phasor table offset (RF: -1 when the advance
                // has no moment on that axis)
    int prow;   // RF / END: first group-factor row of the event's advance
};
struct CellArgs {
    int64_t n_thr;            // threads that hold isochromats
    const int2 *thr;          // per thread: {first layout index, cell << 4 | count}
    const int32_t *cell_gp;   // primary group of each cell
    const int32_t *cell_count;  // isochromats of each cell (thread stride ceil(count / NI))
    const float *M0;
    const int32_t *aidx;      // packed non-primary axis indices (layout order)
    float *Mx, *My, *Mz;
    int init_eq;
    const CellEv *ev;
    int n_ev;
    const float *C_tab;       // [RF advance keys][cells][12]
    const void *P_raw;        // per-(event, primary group) factors (with-ADC flush)
    double *Ablk;             // complex block sums (interleaved re, im)
    const float2 *qtab;       // per-event axis phasor tables
    int f_sh[2];              // bit position of each free axis' index in aidx
    int r_sh;                 // bit position of the secondary axis' index, or -1
    const int32_t *gid[kNTypes];  // layout-order gids per gradient type (with-ADC
                                  // windows of the secondary or no-grads type)
    // receive coils of this pass (Eq. 6 with P coils): sensitivities S of
    // `n_coil` coils in layout order, [coil][re, im][K]; block sums of coil j
    // at Ablk + 2 * ablk_stride * j.  n_coil = 0: one coil with S = 1.
    const float *coil;
    int64_t K;
    int64_t ablk_stride;
    // phasor flags of the form (kernels compiled for coils read them here)
    int rfq, adq, rb;
    double fx;                // fixed-point scale of the block sums (0: FP64 atomics)
    // rows formed per thread (otf = 1; C_tab unused): the transition table,
    // each cell's secondary group and the layout's primary / secondary types
    int otf;
    const float *T_tab;
    const int32_t *cell_gr;
    int gtype_p, gtype_r;
};
// Which per-isochromat and per-thread phasors a cell-form launch applies
// (fixed for the whole span, so the kernel is specialised on them).
struct CellForm {
    int ni;     // isochromats per thread (4, 8)
    int nf;     // free axes (1, 2)
    bool rfq;   // RF / END events rotate by the free-axis phasor
    bool adq;   // with-ADC events rotate by the free-axis phasor
    bool rb;    // with-ADC events rotate by the secondary-axis phasor
    int pc = 0; // receive coils of this pass (0: none; 1, 2 or 4)
};
// One distinct RF / END advance of a cell run: C rows of every cell for
// transition table rows [trow, trow + G_t) of gradient type gtype (trow < 0:
// no transition, END), after an advance with moments kp (primary axis), kr
// (secondary axis) and duration tau.  prow / qr: the group-factor row and the
// secondary-axis phasor table (-1: kr = 0) of the first event with this key.
struct CellKey {
    int64_t trow;
    int gtype;
    int prow;
    int qr;
    int pad;
    double kp, kr, tau;
};
void launch_fused_cell(mrsim_ctx *c, const CellArgs &a, const CellForm &f);
// Batched cell form: CTAs take (job, block) work items from a device counter;
// every job's CellArgs carries its phasor flags (rfq, adq, rb); one coil.
void launch_fused_cell_batch(mrsim_ctx *c, const CellArgs *d_jobs, const int64_t *d_blk_off,
                             int n_jobs, unsigned long long *d_counter, int ni, int nf, bool otf);
void launch_cell_rows(mrsim_ctx *c, const CellKey *d_keys, int n_keys, const mrsim_groups *g,
                      const float *T_tab, const void *P_tab, const float2 *qtab, int r_sh,
                      float *C);
void build_cell_threads(mrsim_ctx *c, mrsim_groups *g, const std::vector<int32_t> &count);
// one axis table: out[j] = exp(-i 2 pi val[j] k) for j < n (cos, sin)
struct AxItem {
    double k;      // gamma_bar * moment on the axis (cycles/m)
    const float *val;
    int n;
    int pad;
    int64_t off;   // first entry in the table array
};
void launch_axis_phase(mrsim_ctx *c, const AxItem *d_items, int n_items, int max_n,
                       float2 *out);
// shared-memory limits of the fused kernels on the context's device
void prepare_fused(mrsim_ctx *c);
template <typename R>
void launch_fused(mrsim_ctx *c, const FusedArgs<R> &a, int ni);
template <typename R>
void launch_event_table(mrsim_ctx *c, const EvAdv *d_adv, int n_ev, int64_t G, const double *par,
                        void *out);

template <typename R>
struct GSigTables {
    const R *pos[kNTypes], *dB0[kNTypes], *rT2[kNTypes], *pos2[kNTypes];
};
// batched forms (one launch for many jobs)
struct EvTabJob {
    const EvAdv *adv;
    int64_t G;
    const double *par;
    void *out;
};
template <typename R>
struct GSigJob {
    const GWin *wins;
    const void *samples;
    GSigTables<R> tab;
    const double *Ablk;
    double *signal;
    double fx;  // fixed-point scale of the sums (0: FP64 atomics)
};
template <typename R>
void launch_precompute_batch(mrsim_ctx *c, const PrecompArgs *d_tabs, const int64_t *d_off,
                             int n_tab, int64_t total);
template <typename R>
void launch_event_table_batch(mrsim_ctx *c, const EvTabJob *d_jobs, const int64_t *d_off,
                              int n_jobs, int64_t total);
// jobs of one form: factor tables or direct advances (direct), with or
// without a receive-coil sensitivity (coil)
template <typename R>
void launch_fused_batch(mrsim_ctx *c, const FusedArgs<R> *d_jobs, const int64_t *d_blk_off,
                        int n_jobs, unsigned long long *d_counter, int ni, bool direct,
                        bool coil);
template <typename R>
void launch_group_signal_batch(mrsim_ctx *c, const GSigJob<R> *d_jobs, const int4 *d_blk,
                               const int *d_blk_job, int n_blk);

template <typename R>
void launch_group_signal(mrsim_ctx *c, const GWin *d_win, const int4 *d_blk, int n_blk,
                         const void *d_samples, const GSigTables<R> &tab, const double *Ablk,
                         double *signal);

}  // namespace mrsim
