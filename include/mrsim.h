/*
 * mrsim — GB300 (sm_103a) Bloch-equation MR simulator with grouped
 * isochromats.  C ABI.
 *
 * Method: H. Takeshima, "Fast Magnetic Resonance Simulation Using Combined
 * Update with Grouped Isochromats" (arXiv 2508.03960).
 *
 * Problem (Sec. 2.1, Eq. 1): K static isochromats k with position r(k),
 * T1(k), T2(k), off-resonance dB0(k) and equilibrium magnetization M0(k)
 * evolve under a piecewise-constant field B(t) = (b1(k) B1re, b1(k) B1im,
 * G(t).r(k) + dB0(k)/gamma_bar).  The received signal at every ADC sample is
 * A(t) = sum_k (Mx + i My)(k, t)  (Eq. 6, one receive coil, S = 1).
 *
 * Units everywhere: seconds, tesla, T/m, metres, Hz (dB0), dimensionless b1.
 * gamma = 2 pi * 42.577478518e6 rad/s/T.  T1 or T2 = +inf means no
 * relaxation.  Sign conventions: rotation by theta = -gamma |B| dt about
 * B/|B| (Eq. A2) followed by relaxation (Eq. A1); free precession multiplies
 * M_xy by exp(-i gamma int Bz dt) (Eq. 4).
 *
 * Conventions shared by all calls
 *  - Status: every int-returning call returns MRSIM_OK (0) or an MRSIM_E*
 *    code; the message of the last failure is in mrsim_last_error(ctx).
 *  - Ownership: the caller owns every array it passes; the library copies
 *    what it keeps (phantoms go to device memory), so input arrays may be
 *    freed as soon as a call returns.  Handles (mrsim_ctx, mrsim_phantom,
 *    mrsim_seq, mrsim_groups) are owned by the library and released with the
 *    matching mrsim_free_* / mrsim_destroy call.  Output arrays are
 *    caller-allocated.
 *  - Threading: one context per host thread.  All device work of a context
 *    runs on its CUDA stream; every call that produces results is
 *    synchronous at return.
 *  - Pointers: unless a flag says MRSIM_PTR_DEVICE / MRSIM_OUT_DEVICE,
 *    arrays are host memory.
 */
#ifndef MRSIM_H
#define MRSIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MRSIM_OK 0
#define MRSIM_EINVAL 1       /* bad argument: NaN, T <= 0, K <= 0, dt <= 0, repeat < 1, ... */
#define MRSIM_EUNSUPPORTED 2 /* RF and ADC active in the same segment (Sec. 2.1) */
#define MRSIM_ENOMEM 3       /* device or host allocation failed */
#define MRSIM_ECUDA 4        /* a CUDA runtime call or kernel failed */
#define MRSIM_ETIMEOUT 5     /* a bounded wait of a tensor-core kernel ran out (surrogate) */
#define MRSIM_ESTATE 6       /* handles do not belong together (e.g. groups of another phantom) */

/* subsequence types (Fig. 1) */
#define MRSIM_SUB_RF 0
#define MRSIM_SUB_ADC 1
#define MRSIM_SUB_RELAX 2

/* gradient types (Sec. 2.4); MRSIM_G_GENERAL falls back to the conventional method */
#define MRSIM_G_NONE 0
#define MRSIM_G_X 1
#define MRSIM_G_Y 2
#define MRSIM_G_Z 3
#define MRSIM_G_GENERAL 4
/* two-axis types (Gx+Gy, Gx+Gz, Gy+Gz: the paper's open problem, Sec. 5): the
 * isochromats are grouped on both positions, keys (r_a, r_b, T1, T2, dB0[, b1]).
 * Reported by mrsim_classify with MRSIM_CLASSIFY_TWO_AXIS, and by sequences
 * made while MRSIM_TUNE_TWO_AXIS is 1 (the default); otherwise such
 * subsequences are MRSIM_G_GENERAL (simulated per isochromat) */
#define MRSIM_G_XY 5
#define MRSIM_G_XZ 6
#define MRSIM_G_YZ 7

/* run modes */
#define MRSIM_PLAIN 0       /* every isochromat stepped individually (Eq. 3, Eq. 6) */
#define MRSIM_PLAIN_CACHE 1 /* per-isochromat combined transitions reused (Eq. 7, dynamic caching) */
#define MRSIM_GROUPED 2     /* grouped isochromats (Sec. 2.3, Eqs. 8-10) */
#define MRSIM_SURROGATE 3   /* GROUPED with learned with-RF transitions where trained */

/* precision of the per-isochromat arithmetic (FP64 is always used to compose
 * combined transitions and to reduce the signal across isochromats) */
#define MRSIM_FP32 0
#define MRSIM_FP64 1

/* flags */
#define MRSIM_PTR_DEVICE 1u /* mrsim_phantom: input arrays are device pointers */
#define MRSIM_OUT_DEVICE 2u /* mrsim_run: signal and M_final are device pointers */
#define MRSIM_PHANTOM_ASYNC 4u /* mrsim_phantom: return once the copies and checks are queued */

typedef struct mrsim_ctx mrsim_ctx;
typedef struct mrsim_phantom_t mrsim_phantom_t;
typedef struct mrsim_seq mrsim_seq;
typedef struct mrsim_groups mrsim_groups;

/* Create a context on CUDA device `device`.  cuda_stream: a cudaStream_t to
 * run on (not owned), or NULL for a context-owned stream.  The context's
 * device buffers (phantoms, sequences, groups, scratch) come from its own
 * stream-ordered memory pool: memory the library frees is returned in stream
 * order and kept reserved for the context's later calls (freeing never
 * synchronises the device); the reserve is handed back when an allocation
 * would otherwise fail and at mrsim_destroy.
 * Errors: MRSIM_EINVAL (ctx NULL or bad device), MRSIM_ECUDA. */
int mrsim_create(mrsim_ctx **ctx, int device, void *cuda_stream);

/* Release the context, its memory pool's reserve and its stream (if owned).
 * Handles made by the context may still be freed afterwards (synchronously).
 * NULL is a no-op. */
void mrsim_destroy(mrsim_ctx *ctx);

/* Message of the last failure on this context ("" if none).  The string is
 * owned by the context and valid until the next call on it. */
const char *mrsim_last_error(const mrsim_ctx *ctx);

/* Upload a phantom of K isochromats (Sec. 2.1).  Each array has K float32
 * entries: position x, y, z (m), T1_s, T2_s (s, > 0, +inf allowed), dB0_hz,
 * M0.  b1_scale: relative RF amplitude per isochromat, NULL => 1.  M_init:
 * initial magnetization as [3][K] (Mx block, My block, Mz block), NULL =>
 * thermal equilibrium (0, 0, M0).  flags: MRSIM_PTR_DEVICE if the arrays are
 * device pointers on the context's device; MRSIM_PHANTOM_ASYNC to return as
 * soon as the copies and the value checks are queued on the context's stream
 * (host work such as mrsim_sequence then overlaps the transfer): the arrays
 * must then stay valid and unchanged until the context's next call returns,
 * and the value checks are reported by the first call that uses the phantom
 * (MRSIM_EINVAL there, and the phantom stays unusable).  The data are copied.
 * Errors: MRSIM_EINVAL (K <= 0, NULL array, NaN, T <= 0), MRSIM_ENOMEM,
 * MRSIM_ECUDA. */
int mrsim_phantom(mrsim_ctx *ctx, int64_t K, const float *x, const float *y, const float *z,
                  const float *T1_s, const float *T2_s, const float *dB0_hz, const float *M0,
                  const float *b1_scale, const float *M_init, unsigned flags,
                  mrsim_phantom_t **out);

/* Copy a phantom's arrays back to the host (each float32 [K]; a NULL
 * destination is skipped), e.g. the centre values and refitted M0 made by
 * mrsim_cluster.  Errors: MRSIM_EINVAL (NULL ctx or ph), MRSIM_ESTATE
 * (phantom of another context), MRSIM_ECUDA. */
int mrsim_phantom_read(mrsim_ctx *ctx, const mrsim_phantom_t *ph, float *x, float *y, float *z,
                       float *T1_s, float *T2_s, float *dB0_hz, float *M0);

/* Attach the complex receive sensitivities of n_coils coils to a phantom
 * (Eq. 6: A(p, t) = sum_k S(k, p) M_xy(k, t); S constant in time).  sens:
 * float32 [n_coils][2][K]: for coil p, K real parts then K imaginary parts, in
 * the phantom's isochromat order.  n_coils = 0 detaches them (one coil with
 * S = 1, the default).  flags: MRSIM_PTR_DEVICE if sens is a device pointer.
 * The data are copied.  With P >= 1 coils attached, mrsim_run returns one
 * signal per coil (see there); grouped runs make one pass of the fused kernel
 * per coil (Eq. 9 block sums per (group, coil)) after one preparation step.
 * Errors: MRSIM_EINVAL (n_coils outside [0, MRSIM_MAX_COILS], sens NULL with
 * n_coils > 0, non-finite value), MRSIM_ENOMEM, MRSIM_ECUDA. */
#define MRSIM_MAX_COILS 64
int mrsim_coils(mrsim_ctx *ctx, mrsim_phantom_t *ph, int n_coils, const float *sens,
                unsigned flags);

/* Describe a pulse sequence as n_seg run-length segments (Sec. 2.1: B(t) is
 * piecewise constant).  Segment j holds repeat[j] >= 1 sub-steps of dt_s[j]
 * > 0 seconds with constant RF b1_re_T + i b1_im_T (tesla), gradient
 * (gx, gy, gz) (T/m) and adc[j] (1 => one sample at the end of every
 * sub-step).  The call splits the sequence into maximal with-RF (B1 != 0),
 * with-ADC and relaxation subsequences (Fig. 1) and types each by which
 * gradient axes are nonzero anywhere in it (Sec. 2.4; a component is zero
 * when it equals 0.0f).  Host arrays; copied.
 * Errors: MRSIM_EINVAL (n_seg <= 0, dt <= 0, repeat < 1, non-finite value),
 * MRSIM_EUNSUPPORTED (RF and ADC in one segment, "not considered" in
 * Sec. 2.1), MRSIM_ENOMEM. */
int mrsim_sequence(mrsim_ctx *ctx, int64_t n_seg, const double *dt_s, const int32_t *repeat,
                   const float *b1_re_T, const float *b1_im_T, const float *gx_Tpm,
                   const float *gy_Tpm, const float *gz_Tpm, const uint8_t *adc,
                   mrsim_seq **out);

/* The host part of mrsim_sequence on its own, without a context or a device:
 * split the sequence (same arrays and rules as mrsim_sequence) into with-RF /
 * with-ADC / relaxation subsequences (Fig. 1) and type each by its gradient
 * axes (Sec. 2.4; with flags = MRSIM_CLASSIFY_TWO_AXIS a subsequence on exactly
 * two axes is typed MRSIM_G_XY / XZ / YZ instead of MRSIM_G_GENERAL; flags = 0
 * types as mrsim_sequence does).  n_subseq receives the count m; when m <= cap, entry i of
 * each non-NULL output gets subsequence i: type (MRSIM_SUB_*), gtype
 * (MRSIM_G_*), seg_begin / seg_end (segment range), n_samples (ADC samples in
 * it) and content_id (with-RF subsequences: index of its distinct content,
 * numbered by first appearance, two pulses sharing one when every field of
 * every segment is bit-equal; -1 otherwise).  Host arrays.
 * Errors: MRSIM_EINVAL (n_subseq NULL, n_seg <= 0, NULL array, dt <= 0,
 * repeat < 1, non-finite value), MRSIM_EUNSUPPORTED (RF and ADC in one
 * segment), MRSIM_ENOMEM. */
#define MRSIM_CLASSIFY_TWO_AXIS 1u
int mrsim_classify(int64_t n_seg, const double *dt_s, const int32_t *repeat, const float *b1_re_T,
                   const float *b1_im_T, const float *gx_Tpm, const float *gy_Tpm,
                   const float *gz_Tpm, const uint8_t *adc, unsigned flags, int64_t cap,
                   int64_t *n_subseq, uint8_t *type, uint8_t *gtype, int64_t *seg_begin,
                   int64_t *seg_end, int64_t *n_samples, int32_t *content_id);

/* Subsequence table of a sequence.  n_subseq receives the count; each output
 * array (host, n_subseq entries) may be NULL.  type: MRSIM_SUB_*; gtype:
 * MRSIM_G_*; seg_begin/seg_end: half-open segment range; n_samples_total:
 * ADC samples of the whole sequence.  Errors: MRSIM_EINVAL (seq NULL). */
int mrsim_seq_info(const mrsim_seq *seq, int64_t *n_subseq, uint8_t *type, uint8_t *gtype,
                   int64_t *seg_begin, int64_t *seg_end, int64_t *n_samples_total);

/* Build the groups the sequence needs (Sec. 2.4, Fig. 2): for every known
 * gradient type used by a with-RF or with-ADC subsequence, isochromats with
 * bit-equal keys share a group.  Keys: Gx-only (x, T1, T2, dB0[, b1]),
 * Gy-only (y, ...), Gz-only (z, ...), no-grads (T1, T2, dB0[, b1]); -0 and
 * +0 compare equal; b1 joins the key when the phantom has one.  Groups are
 * numbered by first occurrence in isochromat index order.  Also lays the
 * isochromats out in device memory sorted by (with-ADC group, with-RF group).
 * Runs on the device; done once per (phantom, sequence shape).  Layout-order
 * copies that only some run forms read are filled by the first run that
 * needs them, so a group set must not be used by two threads at once.
 * Errors: MRSIM_EINVAL, MRSIM_ENOMEM, MRSIM_ECUDA. */
int mrsim_group(mrsim_ctx *ctx, const mrsim_phantom_t *ph, const mrsim_seq *seq,
                mrsim_groups **out);

/* Group count and (optionally) the group id of every isochromat, in the
 * phantom's original order, for gradient type gtype (MRSIM_G_NONE..Z,
 * MRSIM_G_XY..YZ).  gid: host int32[K] or NULL.  Errors: MRSIM_EINVAL (type
 * not built). */
int mrsim_group_info(const mrsim_groups *groups, int gtype, int64_t *n_groups, int32_t *gid);

/* Simulate the sequence on the phantom and return the received signal.
 * groups: required for MRSIM_GROUPED / MRSIM_SURROGATE (NULL => error),
 * ignored otherwise.  mode: MRSIM_PLAIN, MRSIM_PLAIN_CACHE, MRSIM_GROUPED,
 * MRSIM_SURROGATE.  precision: MRSIM_FP32 or MRSIM_FP64 for the
 * per-isochromat arithmetic.  signal: [P][2 * n_samples_total] doubles,
 * interleaved (re, im), in time order, one block per receive coil (P = the
 * phantom's coil count from mrsim_coils, 1 without coils).  M_final: [3][K] float32 final
 * magnetization in the phantom's order, or NULL.  out_flags:
 * MRSIM_OUT_DEVICE if signal / M_final are device pointers.
 * Errors: MRSIM_EINVAL, MRSIM_ESTATE (groups built for another phantom or
 * without a needed type), MRSIM_ENOMEM, MRSIM_ECUDA, MRSIM_ETIMEOUT
 * (MRSIM_SURROGATE: a bounded wait of the tensor-core inference ran out). */
int mrsim_run(mrsim_ctx *ctx, const mrsim_phantom_t *ph, const mrsim_seq *seq,
              const mrsim_groups *groups, int mode, int precision, double *signal,
              float *M_final, unsigned out_flags);

/* Run n_jobs independent (phantom, sequence) jobs of uneven sizes as one
 * CUDA graph (grouped FP32 steps, FP64 signal sums): every job's transition
 * tables in one launch, its group factors in one, persistent fused kernels
 * that take (job, chunk) work items from a device counter, and every job's
 * group signal in one launch.  Any job mrsim_run takes in MRSIM_GROUPED /
 * FP32 is accepted: subsequences without a type run through the
 * per-isochromat fallback kernels inside the same graph between fused spans;
 * a given M_init, direct advances (about one group per isochromat) and
 * receive coils (one instance of the job per coil) are handled as in
 * mrsim_run.  The graph is kept and relaunched while the same jobs (and
 * coils, and tuning) are run again.  groups[i] must come from
 * mrsim_group(ph[i], seq[i]).  signals[i]: host [P][2 * n_samples_total]
 * doubles as in mrsim_run (P = ph[i]'s coil count, 1 without coils).  Jobs
 * without coils run the cell form of the fused kernel when their plan takes
 * it (MRSIM_TUNE_CELL_NI, MRSIM_TUNE_CELL_ROWS), the others the per-isochromat
 * form (MRSIM_TUNE_FUSED_NI); sums use FP64 atomics whatever
 * mrsim_set_reproducible says.
 * Errors: MRSIM_EINVAL (n_jobs <= 0, NULL arrays or entries), MRSIM_ESTATE
 * (groups of another phantom or without a needed type), MRSIM_ENOMEM,
 * MRSIM_ECUDA. */
int mrsim_run_batch(mrsim_ctx *ctx, int n_jobs, const mrsim_phantom_t *const *ph,
                    const mrsim_seq *const *seq, const mrsim_groups *const *groups,
                    double *const *signals);

/* Group-reducing preprocessing (Sec. 3.3, Fig. 4): cluster the isochromats'
 * (T1, T2, dB0) with a bisecting K-means and return a new phantom in which
 * every isochromat carries its cluster's centre values, so that the groups of
 * Sec. 2.4 number at most n_clusters per position (per no-grads type: at most
 * n_clusters in all).
 *  - Space: integer features x_i = rint(v_i * scale_i) of v = (T1 s, T2 s,
 *    dB0 Hz); scale NULL => {64000, 64000, 64} (1/64 ms and 1/64 Hz steps, one
 *    ms weighing as much as one Hz).  Every |x_i| must be <= 2^20 and x_T1,
 *    x_T2 >= 1 (T1, T2 finite).  Sums over features are exact integers.
 *  - Splits: the cluster with the largest sum of squared distances to its
 *    mean (exact comparison; ties: smaller id) is split by 2-means (Lloyd)
 *    started from the member farthest from its mean and the member farthest
 *    from that one (ties: smallest isochromat index); a member goes to the
 *    new side when strictly nearer its centre; passes repeat until the FP64
 *    centres repeat exactly or max_iter passes (a pass leaving a side empty
 *    is dropped).  The old id keeps one side, the new side gets the next id
 *    (ids 0..n-1 in order of creation).  Stops early, with n < n_clusters,
 *    when every cluster holds one distinct feature value.
 *  - Values: centre_i = (sum x_i / count) / scale_i in FP64 (written to
 *    centres), stored as float32 in the new phantom.
 *  - M0 refit: with n_echo > 0 echo times te_s[e] and repetition time tr_s of
 *    a T2-weighted spin-echo model f_e(T1, T2) = (1 - exp(-tr/T1)) exp(-te_e/T2)
 *    (the paper's T2W scan: TR 4.5 s, TE 20/60/100/140 ms), the new M0 is the
 *    least-squares fit of the modelled images M0 f_e(T1, T2) with the centre
 *    values: M0' = sum_e M0 f_e(T1, T2) f_e(c) / sum_e f_e(c)^2 (FP64); n_echo
 *    = 0 keeps M0.
 * Positions, b1, M_init and receive coils are copied.  labels: host int32 [K]
 * (cluster id per isochromat) or NULL; centres: host double [n_clusters][3]
 * (T1 s, T2 s, dB0 Hz; the first n rows written) or NULL; n_out: n, or NULL.
 * The new phantom is released with mrsim_free_phantom.
 * Errors: MRSIM_EINVAL (NULL ctx/ph/out, n_clusters outside [1,
 * MRSIM_MAX_CLUSTERS], max_iter < 1, scale not finite and > 0, n_echo outside
 * [0, MRSIM_MAX_ECHOES], te not finite >= 0, tr not finite > 0, K > 2^28, a
 * feature out of range), MRSIM_ESTATE (phantom of another context),
 * MRSIM_ENOMEM, MRSIM_ECUDA. */
#define MRSIM_MAX_CLUSTERS 4096
#define MRSIM_MAX_ECHOES 16
int mrsim_cluster(mrsim_ctx *ctx, const mrsim_phantom_t *ph, int n_clusters, const double *scale,
                  int max_iter, int n_echo, const double *te_s, double tr_s, int32_t *labels,
                  double *centres, int *n_out, mrsim_phantom_t **out);

/* Image of one coil's Cartesian k-space signal: the centred, normalised
 * inverse DFT the paper applies to its SE / FSE data ("Simulations #1"; an
 * EPI sampled on gradient flat-tops only is Cartesian after reversing every
 * other line, so it is reconstructed the same way).  signal: [n_lines][2 *
 * n_ro] doubles (re, im), the acquisition lines in ADC-window order, as
 * mrsim_run returns them.  Line a goes to k-space row row[a] (0..n_pe-1,
 * centre n_pe / 2) and its sample i to column (col0[a] + dir[a] * i) mod n_ro
 * (centre n_ro / 2; dir = +1 or -1); samples landing on one point add.  Then
 *   image[y][x] = 1/(n_ro n_pe) sum K[ky][kx] exp(+i 2 pi ((kx - n_ro/2)(x - n_ro/2) / n_ro
 *                                                        + (ky - n_pe/2)(y - n_pe/2) / n_pe))
 * in FP64.  image: [n_pe][2 * n_ro] doubles.  flags: MRSIM_PTR_DEVICE if
 * signal and image are device pointers (row, col0, dir are host arrays).
 * Errors: MRSIM_EINVAL (NULL, n_ro or n_pe odd or outside [2, 2048], a row or
 * col0 out of range, dir not +-1), MRSIM_ENOMEM, MRSIM_ECUDA. */
int mrsim_recon_cartesian(mrsim_ctx *ctx, int n_lines, int n_ro, int n_pe, const double *signal,
                          const int32_t *row, const int32_t *col0, const int8_t *dir,
                          unsigned flags, double *image);

/* ------------------------------------------------------------------------
 * Learned with-RF transitions (MRSIM_SURROGATE mode).
 *
 * A small network (5 -> 128 -> 128 -> 12, GELU, BF16 weights, FP32
 * accumulation; the 128x128 layer on tensor cores) per slice-selective
 * (Gz-only) with-RF pulse maps a group's (z, dB0, b1, T1, T2) to the pulse's
 * combined transition [A | b] (Eq. 7), replacing the per-group preparation
 * step of the grouped method (Sec. 2.3).  It is trained on the device by the
 * library's own forward / backward / Adam kernels on exact transitions of
 * random parameter draws (computed by the FP64 preparation kernel), and
 * validated on new draws: the parameter box is cut into 64 x 8 x 4 x 4 cells
 * in (z, dB0, b1, log T2); a cell is served by the network only if the largest
 * error of any transition entry among its validation samples is at most half
 * of `bound` (the margin stands for parameter values between the validation
 * draws); groups in other cells, or outside the box, fall back to exact
 * integration (per-group fallback above a stated error bound: the learned
 * production pattern; the paper has no learned part). */
typedef struct mrsim_surrogate mrsim_surrogate;

/* Train one network per distinct slice-selective with-RF pulse of `seq`.
 * lo/hi: [5] training box for z (m), dB0 (Hz), b1, T1 (s), T2 (s) (T1, T2
 * drawn log-uniformly, the others uniformly).  n_train draws per pulse,
 * `epochs` passes in minibatches of `batch` (Adam, learning rate `lr`
 * decayed by a cosine to lr/100), `seed` for the counter-based draws, `bound` the per-entry error
 * bound of the fallback gate.  Errors: MRSIM_EINVAL (bad arguments, no
 * slice-selective pulse), MRSIM_ENOMEM, MRSIM_ECUDA, MRSIM_ETIMEOUT (a bounded
 * wait of the tensor-core training or inference kernel ran out). */
int mrsim_surrogate_train(mrsim_ctx *ctx, const mrsim_seq *seq, const double *lo,
                          const double *hi, int64_t n_train, int epochs, int batch, double lr,
                          uint64_t seed, double bound, mrsim_surrogate **out);

/* out[8]: networks, mean final training loss (MSE per entry), largest
 * validation error, fraction of cells served by the network, fraction of
 * validation samples in served cells, largest validation error in served
 * cells, and for the context's runs since mrsim_surrogate_use: groups served
 * by the network, groups integrated exactly.  ctx may be NULL. */
int mrsim_surrogate_stats(const mrsim_surrogate *sur, const mrsim_ctx *ctx, double *out);

/* Check of the gate on a real run: for every slice-selective with-RF pulse of
 * `seq` that `sur` serves, the groups of `groups` the gate serves get the
 * network's transition and, independently, the exact one (FP64 sub-steps and
 * composition, Eq. 7); *max_err is the largest |entry| difference over all of
 * them (0 when none is served), *n_served (may be NULL) the number of served
 * (group, pulse) pairs.  The quantity the gate bounds, measured on the run's
 * own groups instead of validation draws.  Errors: MRSIM_EINVAL (NULL),
 * MRSIM_ESTATE (groups without the Gz-only type), MRSIM_ENOMEM, MRSIM_ECUDA,
 * MRSIM_ETIMEOUT. */
int mrsim_surrogate_check(mrsim_ctx *ctx, const mrsim_surrogate *sur, const mrsim_seq *seq,
                          const mrsim_groups *groups, double *max_err, int64_t *n_served);

/* Make `sur` the network used by this context's MRSIM_SURROGATE runs (NULL:
 * none, every pulse is integrated exactly).  The handle must outlive its use. */
int mrsim_surrogate_use(mrsim_ctx *ctx, const mrsim_surrogate *sur);

/* One forward and backward pass of the network with the given parameters
 * (host float[18828], layout W1[128][5], b1[128], W2[128][128], b2[128],
 * W3[12][128], b3[12]) on n host samples x[n][5] with targets t[n][12]:
 * returns y[n][12], the gradient of the loss sum((y - t)^2) / (12 n) and
 * the loss (any output may be NULL).  The same kernel as training: the
 * tile's contractions on the tensor cores (tcgen05, BF16 operands, FP32
 * accumulation in tensor memory), the rest in FP32.  Errors: MRSIM_EINVAL,
 * MRSIM_ENOMEM, MRSIM_ECUDA, MRSIM_ETIMEOUT (a bounded wait ran out). */
int mrsim_surrogate_eval(mrsim_ctx *ctx, const float *params, int64_t n, const float *x,
                         const float *t, float *y, float *grad, double *loss);

/* The inference kernel of MRSIM_SURROGATE runs (tensor-core 128x128 layer,
 * h1 entering as BF16 hi + lo parts) on n host feature rows x[n][5] with the
 * given parameters (layout as for mrsim_surrogate_eval, W2 rounded to BF16):
 * the network's raw outputs y[n][12], before the precession of the pulse is
 * put back.  Errors: MRSIM_EINVAL, MRSIM_ENOMEM, MRSIM_ECUDA, MRSIM_ETIMEOUT
 * (a bounded wait of the tensor-core kernel ran out). */
int mrsim_surrogate_infer(mrsim_ctx *ctx, const float *params, int64_t n, const float *x,
                          float *y);

void mrsim_free_surrogate(mrsim_surrogate *sur);

/* Launch parameters (one value per context).
 *   MRSIM_TUNE_FUSED_NI        isochromats per thread held in registers by the
 *                              grouped fused kernel: 1, 2 or 4 (default 4)
 *   MRSIM_TUNE_PLAIN_RF_NI     isochromats per thread of the plain with-RF step
 *                              kernel: 1 or 2 (default 2)
 *   MRSIM_TUNE_ADC_CTAS_PER_SM CTAs per SM of the persistent plain with-ADC
 *                              kernel: 1, 2, 4 or 8 (default 2)
 *   MRSIM_TUNE_PRECOMP_LANES   threads composing one group's combined
 *                              transition: 1, 2, 4, 8, 16, 32 (one warp or
 *                              less, shuffle tree) or 128 (a CTA, shared-memory
 *                              tree); 0 (default) takes the fewest lanes that
 *                              fill the GPU, a CTA for few, long tables
 *   MRSIM_TUNE_PRECOMP_STEPS   FP32 runs: sub-steps composed in FP32 registers
 *                              (difference form) before each fold into the
 *                              FP64 combined transition: 1, 2, 4, 8
 *                              (default), 16 or 32 (fewer FP64 folds: the
 *                              fold is FP64-pipe work, a small fraction of
 *                              the FP32 rate on this GPU).  For 200-step sinc pulses the
 *                              composed entries stay within 2e-7 of FP64
 *                              composition at 8 and within 1e-7 at 4 or less
 *                              (an FP32 result is itself rounded to 6e-8);
 *                              at 16 / 32 the signal of a 200-step FSE with
 *                              one group per isochromat moves by 3e-8 / 4e-8
 *                              (rel-L2) from folding every step, and the
 *                              preparation of 6.9M groups takes 31 / 24 ms
 *                              instead of 44 ms at 8;
 *                              FP64 runs compose every sub-step in FP64
 *   MRSIM_TUNE_CELL_NI         FP32 grouped runs: isochromats per thread of the
 *                              cell form of the fused kernel (every thread
 *                              holds isochromats of one (with-ADC group,
 *                              with-RF group) cell and applies one combined
 *                              row per cell to each with-RF subsequence): 4
 *                              or 8 (default); 0 turns the cell form off (the
 *                              per-isochromat form of MRSIM_TUNE_FUSED_NI runs).
 *                              Runs with receive coils, per-isochromat
 *                              advances ("direct" form) or gradient types that
 *                              vary inside a cell use the other form anyway.
 *   MRSIM_TUNE_TWO_AXIS        typing of subsequences whose gradients use exactly
 *                              two axes, for the sequences made by
 *                              mrsim_sequence afterwards: 1 (default) types them
 *                              MRSIM_G_XY / XZ / YZ and groups their isochromats
 *                              on both positions (the extension of the paper's
 *                              Sec. 2.4 keys its Sec. 5 leaves open); 0 types
 *                              them MRSIM_G_GENERAL (per-isochromat fallback).
 *                              Not a launch parameter: mrsim_autotune leaves it.
 *   MRSIM_TUNE_CELL_ROWS       the combined rows C = T Adv of the cell form: 0
 *                              (default) a table per run when it holds at most
 *                              four times the state's bytes (and 1 GiB), else
 *                              formed by each thread from the transition and
 *                              group-factor tables; 1 the table whenever it fits
 *                              1 GiB; 2 always per thread.  Both give the same
 *                              rows up to FP32 rounding order (the per-thread
 *                              form is the same arithmetic as the table builder).
 * mrsim_set_tuning returns MRSIM_EINVAL for another parameter or value. */
#define MRSIM_TUNE_FUSED_NI 0
#define MRSIM_TUNE_PLAIN_RF_NI 1
#define MRSIM_TUNE_ADC_CTAS_PER_SM 2
#define MRSIM_TUNE_PRECOMP_LANES 3
#define MRSIM_TUNE_PRECOMP_STEPS 4
#define MRSIM_TUNE_CELL_NI 5
#define MRSIM_TUNE_TWO_AXIS 6
#define MRSIM_TUNE_CELL_ROWS 7
int mrsim_set_tuning(mrsim_ctx *ctx, int param, int value);
int mrsim_get_tuning(const mrsim_ctx *ctx, int param, int *value);

/* Reproducible sums (not part of the paper's method; an option for users who
 * compare outputs bit for bit).  With on = 1, every later mrsim_run of the
 * context forms the block sums of Eq. 9 and the signal sums of Eqs. 6 / 8 / 10
 * in 64-bit fixed point: each contribution v, which the default path adds with
 * FP64 atomics in an order that varies from run to run, is added as the
 * integer rint(v 2^e), and integer addition does not depend on the order.  e
 * is chosen per phantom from B = sum_k (|M0_k| + |M_init_k|) max(1, max_j
 * |S_jk|), which bounds every sum (the magnetisation's norm never exceeds
 * |M_init| + |M0|): 2^e B < 2^56.  Each contribution is then rounded to 2^-e
 * (about 5e-10 for a 27.5M-isochromat phantom of M0 <= 1; the FP64 path's
 * tolerances hold).  Repeated runs, in FP32 or FP64, give identical signals,
 * and one receive coil with S = 1 gives the signal of no coil (FP32 grouped
 * runs then hold 4 isochromats per thread in the cell form, the receive-coil
 * width, whatever MRSIM_TUNE_CELL_NI says).  mrsim_run_batch and
 * mrsim_adc_grouped_noalloc keep FP64 atomics.  Default 0.
 * Errors: MRSIM_EINVAL (NULL ctx / on, or on not 0 or 1). */
int mrsim_set_reproducible(mrsim_ctx *ctx, int on);
int mrsim_get_reproducible(const mrsim_ctx *ctx, int *on);

/* Autotuner: for the given problem and mode, time every allowed value of each
 * launch parameter the mode uses (one warm-up run plus `reps` timed runs of
 * mrsim_run per value, CUDA events on the context stream, one parameter at a
 * time) and keep the fastest in the context.  Results are identical for
 * every choice up to floating-point summation order.
 * Errors: as mrsim_run. */
int mrsim_autotune(mrsim_ctx *ctx, const mrsim_phantom_t *ph, const mrsim_seq *seq,
                   const mrsim_groups *groups, int mode, int precision, int reps);

/* Per-kernel timing.  With profiling on, every kernel launch of the context
 * is bracketed by CUDA events on the context stream.  mrsim_profile_get
 * returns, for entry i (0-based, in first-launch order), the kernel name
 * (copied into name[cap], NUL-terminated), the number of launches and their
 * summed device time in ms; it returns MRSIM_EINVAL past the last entry.
 * mrsim_profile_reset clears the counters. */
int mrsim_profile_enable(mrsim_ctx *ctx, int on);
int mrsim_profile_reset(mrsim_ctx *ctx);
int mrsim_profile_get(mrsim_ctx *ctx, int i, char *name, int cap, int64_t *launches,
                      double *ms_total);

/* Kernels launched by this context since creation (all modes). */
int64_t mrsim_launch_count(const mrsim_ctx *ctx);

/* ------------------------------------------------------------------------
 * Allocation-free grouped with-ADC signal.  The paper has no counterpart to
 * this call; it exists for host programs that cannot allocate device memory
 * once they are running: programs whose device memory is reserved up front by
 * another allocator (a framework's caching pool or a fixed arena holding
 * nearly all of HBM, where a new cudaMalloc fails or forces the pool to give
 * memory back), and acquisition / reconstruction loops that forbid
 * cudaMalloc / cudaFree after start-up because those calls can block until
 * the device is idle.
 *
 * It computes the signal of one with-ADC window of a known gradient type by
 * the grouped three-step method's first two steps: block sums of the
 * transverse magnetization per group (Eq. 9), then every sample from the
 * block sums (Eqs. 8 and 10).  Its only scratch, the complex block sums, is a
 * static device array of MRSIM_NOALLOC_MAX_GROUPS entries (1 MiB) that every
 * GPU which loads the library keeps until the process exits; nothing is
 * allocated by the call.
 *
 * All pointers are device pointers on the current CUDA device, owned by the
 * caller.  K >= 1 isochromats: d_mx, d_my (float32 [K]) transverse
 * magnetization at the window start; d_gid (int32 [K]) group of each
 * isochromat in [0, n_groups), any order.  Per group (float32 [n_groups]):
 * d_gpos position on the window's gradient axis (m; 0 for a no-grads window),
 * d_gdB0 (Hz), d_gT2 (s, +inf allowed).  Per sample (double [n_samples]):
 * d_tau time since the window start (s), d_kmom gamma_bar times the gradient
 * moment on the window's axis since the window start (cycles/m).  d_signal
 * (double [2 * n_samples], interleaved re, im) is overwritten.  stream: a
 * cudaStream_t, or NULL for the legacy default stream.  Synchronous at
 * return.
 *
 * The first call on a device looks up the device address of the scratch
 * array with that device current and keeps it for the life of the process;
 * make that first call before any stream capture.  The kept address does not
 * survive a reset of the device's primary context (cudaDeviceReset): a
 * program that resets the device must not call this entry point afterwards.
 * Every call shares the array, which keeps the last call's
 * contents (each call clears what it uses first); calls that overlap on the
 * GPU (other streams, other host threads) race on it.
 * Errors: MRSIM_EINVAL (K < 1, n_samples < 0, a NULL pointer, n_groups
 * outside [1, MRSIM_NOALLOC_MAX_GROUPS], or a group id outside [0,
 * n_groups): such isochromats are skipped), MRSIM_ECUDA. */
#define MRSIM_NOALLOC_MAX_GROUPS 65536
int mrsim_adc_grouped_noalloc(int64_t K, const float *d_mx, const float *d_my,
                              const int32_t *d_gid, int32_t n_groups, const float *d_gpos,
                              const float *d_gdB0, const float *d_gT2, int64_t n_samples,
                              const double *d_tau, const double *d_kmom, double *d_signal,
                              void *stream);

void mrsim_free_phantom(mrsim_phantom_t *ph);
void mrsim_free_seq(mrsim_seq *seq);
void mrsim_free_groups(mrsim_groups *groups);

#ifdef __cplusplus
}
#endif

#endif /* MRSIM_H */
