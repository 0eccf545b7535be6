/*
 * FP64 CPU oracle for the grouped-isochromat Bloch simulator.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA library is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the library never does.  It shares
 * no code, header or constant with the CUDA library.
 *
 * What it follows (Takeshima, "Fast Magnetic Resonance Simulation Using
 * Combined Update with Grouped Isochromats"):
 *   - Eq. 1   Bloch equation with relaxation, per isochromat, static r(k).
 *   - Eq. 2-3 piecewise-constant field, step transitions U composed in time
 *             order; U = D R (App. A: rotate by Eq. A2, then relax by Eq. A1).
 *   - Eq. 4-5 closed-form free precession / relaxation when B1 = 0.
 *   - Eq. 6   received signal A(p, t) = sum_k S(k, p) M_xy(k, t) for every
 *             receive coil p (one coil with S = 1 unless sensitivities are
 *             given; S is complex and constant in time).
 *   - Eq. 7   combined transition of a with-RF subsequence (memoised per
 *             isochromat when the same RF content repeats: the "dynamic
 *             caching" of the conventional method, Sec. 2.2).
 *   - Sec. 2.1 / Fig. 1 subsequence split (with-RF / with-ADC / relaxation),
 *             Sec. 2.4 gradient types (Gx-only, Gy-only, Gz-only, no-grads),
 *             Fig. 2 grouping by equal keys; on request also the two-axis
 *             types (Gx+Gy, Gx+Gz, Gy+Gz, grouped on both positions) that
 *             Sec. 5 leaves open.
 *   - Eq. 8-10 grouped with-ADC three-step method and the grouped with-RF
 *             combined transition (Sec. 2.3), used only for the brute-force
 *             "grouped equals ungrouped" check.
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   gamma = 2 pi * 42.577478518e6 rad/s/T; dB0 is given in Hz; segment j's
 *   field holds on [t_j, t_j + dt_j); an ADC sample is taken at the end of
 *   each ADC sub-step; the initial state is (0, 0, M0) unless given; a
 *   gradient component is "zero" when it compares equal to 0.0f; a
 *   subsequence with RF and ADC in one segment is rejected; groups are
 *   numbered by first occurrence in isochromat index order; group keys compare
 *   float32 bit patterns after -0 -> +0, and the RF scale b1 joins every key
 *   when it is supplied.
 *
 * Parity pins: every function here is pinned by a test against mathematics
 * (closed forms, a library DFT, brute force); none is "parity unpinned".
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define OR_PI 3.14159265358979323846
#define OR_GAMMA (2.0 * OR_PI * 42.577478518e6) /* rad s^-1 T^-1 */

enum { OR_OK = 0, OR_EINVAL = -1, OR_EUNSUPPORTED = -2, OR_ENOMEM = -3 };
enum { OR_RF = 0, OR_ADC = 1, OR_RELAX = 2 };
enum { OR_G_NONE = 0, OR_G_X = 1, OR_G_Y = 2, OR_G_Z = 3, OR_G_GENERAL = 4 };
/* two-axis gradient types (the paper's open problem, Sec. 5): a subsequence
 * whose gradients use exactly two axes, grouped on both positions; only made
 * when asked for (two_axis), otherwise such a subsequence is OR_G_GENERAL */
enum { OR_G_XY = 5, OR_G_XZ = 6, OR_G_YZ = 7, OR_N_GTYPES = 8 };

/* position axes (0 = x, 1 = y, 2 = z) of a gradient type; returns their count */
static int type_axes(int g, int ax[2]) {
    switch (g) {
    case OR_G_X: ax[0] = 0; return 1;
    case OR_G_Y: ax[0] = 1; return 1;
    case OR_G_Z: ax[0] = 2; return 1;
    case OR_G_XY: ax[0] = 0; ax[1] = 1; return 2;
    case OR_G_XZ: ax[0] = 0; ax[1] = 2; return 2;
    case OR_G_YZ: ax[0] = 1; ax[1] = 2; return 2;
    default: return 0;
    }
}

typedef struct {
    int64_t n_seg;
    const double *dt;
    const int32_t *rep;
    const float *b1re, *b1im, *gx, *gy, *gz;
    const uint8_t *adc;
} or_seq;

typedef struct {
    int64_t K;
    const float *x, *y, *z, *T1, *T2, *dB0, *M0;
    const float *b1;    /* NULL => 1 */
    const float *Minit; /* [3][K] or NULL => (0, 0, M0) */
    int n_coils;        /* receive coils (>= 1) */
    const float *sens;  /* [n_coils][2][K] (re, im of S(k, p)) or NULL => S = 1 */
} or_phantom;

typedef struct {
    int memo;           /* reuse a with-RF combined transition per isochromat */
    int adc_recurrence; /* FP64 phasor recurrence inside an ADC segment */
    int n_threads;      /* <= 0 => all online CPUs */
} or_opts;

/* ------------------------------------------------------------------------ */
/* Subsequence split and classification (Fig. 1, Sec. 2.1, Sec. 2.4).        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    uint8_t *type, *gtype;
    int64_t *seg_begin, *seg_end, *n_samples;
    int32_t *content_id; /* with-RF: first-occurrence id of its exact content */
    int64_t n_content;
    int64_t *content_count; /* occurrences of each content id */
} or_subseqs;

static int seg_class(const or_seq *s, int64_t j) {
    int rf = (s->b1re[j] != 0.0f) || (s->b1im[j] != 0.0f);
    if (rf && s->adc[j]) return -1;
    return rf ? OR_RF : (s->adc[j] ? OR_ADC : OR_RELAX);
}

static int seg_valid(const or_seq *s, int64_t j) {
    return isfinite(s->dt[j]) && s->dt[j] > 0.0 && s->rep[j] >= 1 &&
           isfinite(s->b1re[j]) && isfinite(s->b1im[j]) && isfinite(s->gx[j]) &&
           isfinite(s->gy[j]) && isfinite(s->gz[j]);
}

static int same_segment(const or_seq *s, int64_t a, int64_t b) {
    return s->dt[a] == s->dt[b] && s->rep[a] == s->rep[b] && s->b1re[a] == s->b1re[b] &&
           s->b1im[a] == s->b1im[b] && s->gx[a] == s->gx[b] && s->gy[a] == s->gy[b] &&
           s->gz[a] == s->gz[b] && s->adc[a] == s->adc[b];
}

static void free_subseqs(or_subseqs *q) {
    free(q->type); free(q->gtype); free(q->seg_begin); free(q->seg_end);
    free(q->n_samples); free(q->content_id); free(q->content_count);
    memset(q, 0, sizeof(*q));
}

static int build_subseqs(const or_seq *s, or_subseqs *q, int two_axis) {
    memset(q, 0, sizeof(*q));
    if (s->n_seg <= 0) return OR_EINVAL;
    int64_t n = 0;
    for (int64_t j = 0; j < s->n_seg; ++j) {
        if (!seg_valid(s, j)) return OR_EINVAL;
        int c = seg_class(s, j);
        if (c < 0) return OR_EUNSUPPORTED;
        if (j == 0 || c != seg_class(s, j - 1)) ++n;
    }
    q->n = n;
    q->type = malloc(n); q->gtype = malloc(n);
    q->seg_begin = malloc(n * sizeof(int64_t)); q->seg_end = malloc(n * sizeof(int64_t));
    q->n_samples = malloc(n * sizeof(int64_t)); q->content_id = malloc(n * sizeof(int32_t));
    if (!q->type || !q->gtype || !q->seg_begin || !q->seg_end || !q->n_samples || !q->content_id) {
        free_subseqs(q);
        return OR_ENOMEM;
    }
    int64_t i = -1;
    for (int64_t j = 0; j < s->n_seg; ++j) {
        int c = seg_class(s, j);
        if (j == 0 || c != seg_class(s, j - 1)) {
            ++i;
            q->type[i] = (uint8_t)c;
            q->seg_begin[i] = j;
        }
        q->seg_end[i] = j + 1;
    }
    for (i = 0; i < n; ++i) {
        int ax = 0, ay = 0, az = 0;
        int64_t ns = 0;
        for (int64_t j = q->seg_begin[i]; j < q->seg_end[i]; ++j) {
            ax |= s->gx[j] != 0.0f;
            ay |= s->gy[j] != 0.0f;
            az |= s->gz[j] != 0.0f;
            if (s->adc[j]) ns += s->rep[j];
        }
        int cnt = ax + ay + az;
        q->gtype[i] = cnt == 0 ? OR_G_NONE
                    : cnt == 1 ? (ax ? OR_G_X : ay ? OR_G_Y : OR_G_Z)
                    : cnt == 2 && two_axis ? (!az ? OR_G_XY : !ay ? OR_G_XZ : OR_G_YZ)
                               : OR_G_GENERAL;
        q->n_samples[i] = ns;
    }
    /* content ids of with-RF subsequences: exact segment-by-segment equality */
    int32_t n_content = 0;
    int64_t *rep_of = malloc(n * sizeof(int64_t));
    if (!rep_of) { free_subseqs(q); return OR_ENOMEM; }
    for (i = 0; i < n; ++i) {
        q->content_id[i] = -1;
        if (q->type[i] != OR_RF) continue;
        int64_t len = q->seg_end[i] - q->seg_begin[i];
        for (int32_t c = 0; c < n_content; ++c) {
            int64_t r = rep_of[c];
            if (q->seg_end[r] - q->seg_begin[r] != len) continue;
            int eq = 1;
            for (int64_t d = 0; d < len && eq; ++d)
                eq = same_segment(s, q->seg_begin[r] + d, q->seg_begin[i] + d);
            if (eq) { q->content_id[i] = c; break; }
        }
        if (q->content_id[i] < 0) {
            rep_of[n_content] = i;
            q->content_id[i] = n_content++;
        }
    }
    free(rep_of);
    q->n_content = n_content;
    q->content_count = calloc(n_content > 0 ? n_content : 1, sizeof(int64_t));
    if (!q->content_count) { free_subseqs(q); return OR_ENOMEM; }
    for (i = 0; i < n; ++i)
        if (q->content_id[i] >= 0) q->content_count[q->content_id[i]]++;
    return OR_OK;
}

int or_classify(const double *dt, const int32_t *rep, const float *b1re, const float *b1im,
                const float *gx, const float *gy, const float *gz, const uint8_t *adc,
                int64_t n_seg, int64_t cap, int64_t *n_sub, uint8_t *type, uint8_t *gtype,
                int64_t *seg_begin, int64_t *seg_end, int64_t *n_samples, int32_t *content_id,
                int two_axis) {
    or_seq s = {n_seg, dt, rep, b1re, b1im, gx, gy, gz, adc};
    or_subseqs q;
    int rc = build_subseqs(&s, &q, two_axis);
    if (rc) return rc;
    *n_sub = q.n;
    if (q.n <= cap) {
        memcpy(type, q.type, q.n);
        memcpy(gtype, q.gtype, q.n);
        memcpy(seg_begin, q.seg_begin, q.n * sizeof(int64_t));
        memcpy(seg_end, q.seg_end, q.n * sizeof(int64_t));
        memcpy(n_samples, q.n_samples, q.n * sizeof(int64_t));
        memcpy(content_id, q.content_id, q.n * sizeof(int32_t));
    }
    free_subseqs(&q);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Grouping (Fig. 2, Sec. 2.4): equal keys -> one group, numbered by first   */
/* occurrence in isochromat index order.                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint32_t k[6];
    int64_t idx;
} or_key;

static int key_cmp(const void *pa, const void *pb) {
    const or_key *a = pa, *b = pb;
    for (int i = 0; i < 6; ++i)
        if (a->k[i] != b->k[i]) return a->k[i] < b->k[i] ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

static int key_bits(float v, uint32_t *out) {
    if (isnan(v)) return OR_EINVAL;
    if (v == 0.0f) v = 0.0f; /* -0 -> +0 */
    memcpy(out, &v, 4);
    return OR_OK;
}

typedef struct {
    int64_t idx, run;
} or_rep;

static int rep_cmp(const void *pa, const void *pb) {
    const or_rep *a = pa, *b = pb;
    return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

/* gtype: OR_G_X / Y / Z use (r_axis, T1, T2, dB0[, b1]); the two-axis types
 * OR_G_XY / XZ / YZ use (r_a, r_b, T1, T2, dB0[, b1]); OR_G_NONE uses
 * (T1, T2, dB0[, b1]).  Writes gid[K], returns the group count. */
int or_group(int64_t K, const float *x, const float *y, const float *z, const float *T1,
             const float *T2, const float *dB0, const float *b1, int gtype, int32_t *gid,
             int64_t *n_groups) {
    if (K <= 0 || gtype < OR_G_NONE || gtype >= OR_N_GTYPES || gtype == OR_G_GENERAL)
        return OR_EINVAL;
    const float *axis[3] = {x, y, z};
    int ax[2];
    const int n_ax = type_axes(gtype, ax);
    const float *pa = n_ax > 0 ? axis[ax[0]] : NULL, *pb = n_ax > 1 ? axis[ax[1]] : NULL;
    or_key *keys = malloc((size_t)K * sizeof(or_key));
    if (!keys) return OR_ENOMEM;
    for (int64_t k = 0; k < K; ++k) {
        int rc = 0;
        rc |= key_bits(pa ? pa[k] : 0.0f, &keys[k].k[0]);
        rc |= key_bits(T1[k], &keys[k].k[1]);
        rc |= key_bits(T2[k], &keys[k].k[2]);
        rc |= key_bits(dB0[k], &keys[k].k[3]);
        rc |= key_bits(b1 ? b1[k] : 1.0f, &keys[k].k[4]);
        rc |= key_bits(pb ? pb[k] : 0.0f, &keys[k].k[5]);
        if (rc) { free(keys); return OR_EINVAL; }
        keys[k].idx = k;
    }
    qsort(keys, (size_t)K, sizeof(or_key), key_cmp);
    /* runs of equal keys; the first element of each run has the smallest index */
    int64_t n_runs = 0;
    int64_t *run_of = malloc((size_t)K * sizeof(int64_t));
    or_rep *reps = malloc((size_t)K * sizeof(or_rep));
    if (!run_of || !reps) { free(keys); free(run_of); free(reps); return OR_ENOMEM; }
    for (int64_t i = 0; i < K; ++i) {
        if (i == 0 || memcmp(keys[i].k, keys[i - 1].k, sizeof(keys[i].k)) != 0) {
            reps[n_runs].idx = keys[i].idx;
            reps[n_runs].run = n_runs;
            ++n_runs;
        }
        run_of[keys[i].idx] = n_runs - 1;
    }
    qsort(reps, (size_t)n_runs, sizeof(or_rep), rep_cmp);
    int64_t *gid_of_run = malloc((size_t)n_runs * sizeof(int64_t));
    if (!gid_of_run) { free(keys); free(run_of); free(reps); return OR_ENOMEM; }
    for (int64_t g = 0; g < n_runs; ++g) gid_of_run[reps[g].run] = g;
    for (int64_t k = 0; k < K; ++k) gid[k] = (int32_t)gid_of_run[run_of[k]];
    *n_groups = n_runs;
    free(keys); free(run_of); free(reps); free(gid_of_run);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Per-isochromat physics.                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    double x, y, z, T1, T2, dB0, M0, b1;
} or_iso;

/* One RF sub-step of length dt: M <- D R M (App. A; Eq. A2 then Eq. A1). */
static void rf_step(double M[3], const or_iso *p, double b1re, double b1im, double gx,
                    double gy, double gz, double dt) {
    double Bx = p->b1 * b1re, By = p->b1 * b1im;
    double Bz = gx * p->x + gy * p->y + gz * p->z + 2.0 * OR_PI * p->dB0 / OR_GAMMA;
    double nB = sqrt(Bx * Bx + By * By + Bz * Bz);
    if (nB > 0.0) {
        double ux = Bx / nB, uy = By / nB, uz = Bz / nB;
        double th = -OR_GAMMA * nB * dt;
        double c = cos(th), s = sin(th), oc = 1.0 - c;
        double R[3][3] = {
            {c + ux * ux * oc, -uz * s + ux * uy * oc, uy * s + ux * uz * oc},
            {uz * s + ux * uy * oc, c + uy * uy * oc, -ux * s + uy * uz * oc},
            {-uy * s + ux * uz * oc, ux * s + uy * uz * oc, c + uz * uz * oc},
        };
        double m0 = M[0], m1 = M[1], m2 = M[2];
        M[0] = R[0][0] * m0 + R[0][1] * m1 + R[0][2] * m2;
        M[1] = R[1][0] * m0 + R[1][1] * m1 + R[1][2] * m2;
        M[2] = R[2][0] * m0 + R[2][1] * m1 + R[2][2] * m2;
    }
    double E2 = exp(-dt / p->T2), E1 = exp(-dt / p->T1);
    M[0] *= E2;
    M[1] *= E2;
    M[2] = E1 * M[2] + (1.0 - E1) * p->M0;
}

/* Same step applied to a 3x4 affine T = [A | b] (the M0 column), i.e.
 * T <- U T with U = D R, so that M(t_N) = A M(t_0) + b M0 (Eq. 7). */
static void rf_step_affine(double T[3][4], const or_iso *p, double b1re, double b1im,
                           double gx, double gy, double gz, double dt) {
    double Bx = p->b1 * b1re, By = p->b1 * b1im;
    double Bz = gx * p->x + gy * p->y + gz * p->z + 2.0 * OR_PI * p->dB0 / OR_GAMMA;
    double nB = sqrt(Bx * Bx + By * By + Bz * Bz);
    double R[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    if (nB > 0.0) {
        double ux = Bx / nB, uy = By / nB, uz = Bz / nB;
        double th = -OR_GAMMA * nB * dt;
        double c = cos(th), s = sin(th), oc = 1.0 - c;
        R[0][0] = c + ux * ux * oc; R[0][1] = -uz * s + ux * uy * oc; R[0][2] = uy * s + ux * uz * oc;
        R[1][0] = uz * s + ux * uy * oc; R[1][1] = c + uy * uy * oc; R[1][2] = -ux * s + uy * uz * oc;
        R[2][0] = -uy * s + ux * uz * oc; R[2][1] = ux * s + uy * uz * oc; R[2][2] = c + uz * uz * oc;
    }
    double E2 = exp(-dt / p->T2), E1 = exp(-dt / p->T1);
    double D[3] = {E2, E2, E1};
    double out[3][4];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 4; ++c)
            out[r][c] = D[r] * (R[r][0] * T[0][c] + R[r][1] * T[1][c] + R[r][2] * T[2][c]);
    out[2][3] += 1.0 - E1;
    memcpy(T, out, sizeof(out));
}

static void affine_apply(double M[3], double T[3][4], double M0) {
    double m0 = M[0], m1 = M[1], m2 = M[2];
    for (int r = 0; r < 3; ++r) M[r] = T[r][0] * m0 + T[r][1] * m1 + T[r][2] * m2 + T[r][3] * M0;
}

/* Eqs. 4-5 over a duration tau with constant gradient g. */
static void free_precess(double M[3], const or_iso *p, double gx, double gy, double gz,
                         double tau) {
    double phi = OR_GAMMA * (gx * p->x + gy * p->y + gz * p->z) * tau + 2.0 * OR_PI * p->dB0 * tau;
    double E2 = exp(-tau / p->T2), E1 = exp(-tau / p->T1);
    double c = cos(phi), s = sin(phi);
    /* M_xy <- M_xy E2 exp(-i phi) */
    double mx = M[0], my = M[1];
    M[0] = E2 * (mx * c + my * s);
    M[1] = E2 * (my * c - mx * s);
    M[2] = p->M0 + (M[2] - p->M0) * E1;
}

static or_iso iso_at(const or_phantom *ph, int64_t k) {
    or_iso p;
    p.x = ph->x[k]; p.y = ph->y[k]; p.z = ph->z[k];
    p.T1 = ph->T1[k]; p.T2 = ph->T2[k]; p.dB0 = ph->dB0[k]; p.M0 = ph->M0[k];
    p.b1 = ph->b1 ? ph->b1[k] : 1.0;
    return p;
}

static void iso_init(const or_phantom *ph, int64_t k, double M[3]) {
    if (ph->Minit) {
        M[0] = ph->Minit[k]; M[1] = ph->Minit[ph->K + k]; M[2] = ph->Minit[2 * ph->K + k];
    } else {
        M[0] = 0.0; M[1] = 0.0; M[2] = ph->M0[k];
    }
}

/* ------------------------------------------------------------------------ */
/* Ungrouped simulation: every isochromat individually.                      */
/* ------------------------------------------------------------------------ */

typedef struct {
    const or_phantom *ph;
    const or_seq *s;
    const or_subseqs *q;
    const or_opts *o;
    int64_t k0, k1, n_samples;
    double *sig;    /* thread-private partial [2 n_samples] */
    double *Mfinal; /* shared [3][K] or NULL */
    int rc;
} or_job;

/* Eq. 6: isochromat k's term of sample smp, weighted by every coil's S(k, p);
 * the signal of coil p occupies [2 n_samples p, 2 n_samples (p + 1)). */
static void add_sample(const or_job *J, int64_t k, int64_t smp, double mx, double my) {
    const or_phantom *ph = J->ph;
    if (!ph->sens) {
        J->sig[2 * smp] += mx;
        J->sig[2 * smp + 1] += my;
        return;
    }
    for (int c = 0; c < ph->n_coils; ++c) {
        const double sr = ph->sens[(2 * (int64_t)c) * ph->K + k];
        const double si = ph->sens[(2 * (int64_t)c + 1) * ph->K + k];
        double *o = J->sig + 2 * J->n_samples * c + 2 * smp;
        o[0] += sr * mx - si * my;
        o[1] += sr * my + si * mx;
    }
}

static void simulate_one(const or_job *J, int64_t k, double (*memo)[3][4], char *have) {
    const or_seq *s = J->s;
    const or_subseqs *q = J->q;
    or_iso p = iso_at(J->ph, k);
    double M[3];
    iso_init(J->ph, k, M);
    if (memo) memset(have, 0, q->n_content);
    int64_t smp = 0;
    for (int64_t i = 0; i < q->n; ++i) {
        if (q->type[i] == OR_RF && memo && q->content_count[q->content_id[i]] > 1) {
            int32_t c = q->content_id[i];
            if (!have[c]) {
                double (*T)[4] = memo[c];
                memset(T, 0, sizeof(double[3][4]));
                T[0][0] = T[1][1] = T[2][2] = 1.0;
                for (int64_t j = q->seg_begin[i]; j < q->seg_end[i]; ++j)
                    for (int32_t r = 0; r < s->rep[j]; ++r)
                        rf_step_affine(T, &p, s->b1re[j], s->b1im[j], s->gx[j], s->gy[j],
                                       s->gz[j], s->dt[j]);
                have[c] = 1;
            }
            affine_apply(M, memo[c], p.M0);
            continue;
        }
        for (int64_t j = q->seg_begin[i]; j < q->seg_end[i]; ++j) {
            double dt = s->dt[j];
            int32_t rep = s->rep[j];
            if (q->type[i] == OR_RF) {
                for (int32_t r = 0; r < rep; ++r)
                    rf_step(M, &p, s->b1re[j], s->b1im[j], s->gx[j], s->gy[j], s->gz[j], dt);
            } else if (q->type[i] == OR_ADC) {
                if (J->o->adc_recurrence) {
                    /* constant field: M_xy(t + dt) = M_xy(t) * E2(dt) exp(-i phi(dt)) */
                    double phi = OR_GAMMA * (s->gx[j] * p.x + s->gy[j] * p.y + s->gz[j] * p.z) * dt +
                                 2.0 * OR_PI * p.dB0 * dt;
                    double E2 = exp(-dt / p.T2);
                    double zr = E2 * cos(phi), zi = -E2 * sin(phi);
                    double mx = M[0], my = M[1];
                    for (int32_t r = 0; r < rep; ++r) {
                        double nx = mx * zr - my * zi, ny = mx * zi + my * zr;
                        mx = nx; my = ny;
                        add_sample(J, k, smp, mx, my);
                        ++smp;
                    }
                    /* M_xy from one closed-form step over the whole segment, Mz likewise */
                    free_precess(M, &p, s->gx[j], s->gy[j], s->gz[j], dt * rep);
                } else {
                    for (int32_t r = 0; r < rep; ++r) {
                        free_precess(M, &p, s->gx[j], s->gy[j], s->gz[j], dt);
                        add_sample(J, k, smp, M[0], M[1]);
                        ++smp;
                    }
                }
            } else {
                free_precess(M, &p, s->gx[j], s->gy[j], s->gz[j], dt * rep);
            }
        }
    }
    if (J->Mfinal) {
        J->Mfinal[k] = M[0];
        J->Mfinal[J->ph->K + k] = M[1];
        J->Mfinal[2 * J->ph->K + k] = M[2];
    }
}

static void *simulate_range(void *arg) {
    or_job *J = arg;
    double (*memo)[3][4] = NULL;
    char *have = NULL;
    if (J->o->memo && J->q->n_content > 0) {
        memo = malloc((size_t)J->q->n_content * sizeof(double[3][4]));
        have = malloc((size_t)J->q->n_content);
        if (!memo || !have) { free(memo); free(have); J->rc = OR_ENOMEM; return NULL; }
    }
    for (int64_t k = J->k0; k < J->k1; ++k) simulate_one(J, k, memo, have);
    free(memo);
    free(have);
    return NULL;
}

static int n_threads_for(const or_opts *o, int64_t K) {
    long n = o->n_threads > 0 ? o->n_threads : sysconf(_SC_NPROCESSORS_ONLN);
    if (n < 1) n = 1;
    if (n > 256) n = 256;
    if (n > K) n = (int)K;
    return (int)n;
}

static int check_phantom(const or_phantom *ph) {
    if (ph->K <= 0) return OR_EINVAL;
    for (int64_t k = 0; k < ph->K; ++k) {
        if (!(ph->T1[k] > 0.0f) || !(ph->T2[k] > 0.0f)) return OR_EINVAL;
        if (!isfinite(ph->x[k]) || !isfinite(ph->y[k]) || !isfinite(ph->z[k]) ||
            !isfinite(ph->dB0[k]) || !isfinite(ph->M0[k]) || (ph->b1 && !isfinite(ph->b1[k])))
            return OR_EINVAL;
    }
    if (ph->n_coils < 1) return OR_EINVAL;
    if (ph->sens)
        for (int64_t i = 0; i < 2 * (int64_t)ph->n_coils * ph->K; ++i)
            if (!isfinite(ph->sens[i])) return OR_EINVAL;
    return OR_OK;
}

/* Ungrouped FP64 simulation.  signal: [n_coils][2 * n_samples] interleaved
 * (re, im); sens: [n_coils][2][K] or NULL (one coil, S = 1; n_coils must then
 * be 1); Mfinal: [3][K] or NULL.  Returns 0 or a negative error code. */
int or_simulate(int64_t K, const float *x, const float *y, const float *z, const float *T1,
                const float *T2, const float *dB0, const float *M0, const float *b1,
                const float *Minit, int64_t n_seg, const double *dt, const int32_t *rep,
                const float *b1re, const float *b1im, const float *gx, const float *gy,
                const float *gz, const uint8_t *adc, int memo, int adc_recurrence,
                int n_threads, int n_coils, const float *sens, double *signal, double *Mfinal) {
    or_phantom ph = {K, x, y, z, T1, T2, dB0, M0, b1, Minit, n_coils, sens};
    if (!sens && n_coils != 1) return OR_EINVAL;
    or_seq s = {n_seg, dt, rep, b1re, b1im, gx, gy, gz, adc};
    or_opts o = {memo, adc_recurrence, n_threads};
    int rc = check_phantom(&ph);
    if (rc) return rc;
    or_subseqs q;
    rc = build_subseqs(&s, &q, 0);
    if (rc) return rc;
    int64_t ns = 0;
    for (int64_t i = 0; i < q.n; ++i) ns += q.n_samples[i];
    int nt = n_threads_for(&o, K);
    or_job *jobs = calloc(nt, sizeof(or_job));
    pthread_t *th = calloc(nt, sizeof(pthread_t));
    const int64_t nsig = 2 * ns * (int64_t)n_coils; /* signal doubles of all coils */
    double *part = calloc((size_t)nt * (size_t)(nsig + 1), sizeof(double));
    if (!jobs || !th || !part) { free(jobs); free(th); free(part); free_subseqs(&q); return OR_ENOMEM; }
    for (int t = 0; t < nt; ++t) {
        jobs[t] = (or_job){&ph, &s, &q, &o, K * t / nt, K * (t + 1) / nt, ns,
                           part + (size_t)t * (size_t)(nsig + 1), Mfinal, 0};
        if (pthread_create(&th[t], NULL, simulate_range, &jobs[t]) != 0) {
            jobs[t].rc = OR_ENOMEM;
            simulate_range(&jobs[t]);
        }
    }
    rc = OR_OK;
    for (int t = 0; t < nt; ++t) {
        pthread_join(th[t], NULL);
        if (jobs[t].rc) rc = jobs[t].rc;
    }
    /* combine per-thread partial signals in thread order (deterministic) */
    for (int64_t i = 0; i < nsig; ++i) {
        double acc = 0.0;
        for (int t = 0; t < nt; ++t) acc += part[(size_t)t * (size_t)(nsig + 1) + i];
        signal[i] = acc;
    }
    free(jobs); free(th); free(part); free_subseqs(&q);
    return rc;
}

/* Combined transition (Eq. 7) of segments [seg_begin, seg_end) for one
 * isochromat with the given parameters, as a row-major 3x4 affine. */
int or_transition(double x, double y, double z, double T1, double T2, double dB0, double b1,
                  const double *dt, const int32_t *rep, const float *b1re, const float *b1im,
                  const float *gx, const float *gy, const float *gz, int64_t seg_begin,
                  int64_t seg_end, double *T_out) {
    or_iso p = {x, y, z, T1, T2, dB0, 0.0, b1};
    double T[3][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}};
    for (int64_t j = seg_begin; j < seg_end; ++j)
        for (int32_t r = 0; r < rep[j]; ++r)
            rf_step_affine(T, &p, b1re[j], b1im[j], gx[j], gy[j], gz[j], dt[j]);
    memcpy(T_out, T, sizeof(T));
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Grouped simulation (Sec. 2.3, Eqs. 8-10), for brute-force equality only.  */
/* Every subsequence is processed for all isochromats before the next one.   */
/* ------------------------------------------------------------------------ */

int or_simulate_grouped(int64_t K, const float *x, const float *y, const float *z,
                        const float *T1, const float *T2, const float *dB0, const float *M0,
                        const float *b1, const float *Minit, int64_t n_seg, const double *dt,
                        const int32_t *rep, const float *b1re, const float *b1im,
                        const float *gx, const float *gy, const float *gz, const uint8_t *adc,
                        int two_axis, double *signal, double *Mfinal) {
    or_phantom ph = {K, x, y, z, T1, T2, dB0, M0, b1, Minit, 1, NULL};
    or_seq s = {n_seg, dt, rep, b1re, b1im, gx, gy, gz, adc};
    int rc = check_phantom(&ph);
    if (rc) return rc;
    or_subseqs q;
    rc = build_subseqs(&s, &q, two_axis);
    if (rc) return rc;
    double *M = malloc((size_t)K * 3 * sizeof(double));
    int32_t *gid[OR_N_GTYPES] = {NULL};
    int64_t ng[OR_N_GTYPES] = {0};
    int64_t *rep_of[OR_N_GTYPES] = {NULL};
    if (!M) { free_subseqs(&q); return OR_ENOMEM; }
    for (int64_t k = 0; k < K; ++k) iso_init(&ph, k, &M[3 * k]);
    /* groups for every known gradient type used by a with-RF / with-ADC subsequence */
    for (int64_t i = 0; i < q.n && rc == OR_OK; ++i) {
        int g = q.gtype[i];
        if (q.type[i] == OR_RELAX || g == OR_G_GENERAL || gid[g]) continue;
        gid[g] = malloc((size_t)K * sizeof(int32_t));
        if (!gid[g]) { rc = OR_ENOMEM; break; }
        rc = or_group(K, x, y, z, T1, T2, dB0, b1, g, gid[g], &ng[g]);
        if (rc) break;
        rep_of[g] = malloc((size_t)ng[g] * sizeof(int64_t));
        if (!rep_of[g]) { rc = OR_ENOMEM; break; }
        for (int64_t k = K - 1; k >= 0; --k) rep_of[g][gid[g][k]] = k; /* first member */
    }
    int64_t smp = 0;
    for (int64_t i = 0; i < q.n && rc == OR_OK; ++i) {
        int g = q.gtype[i];
        int known = g != OR_G_GENERAL;
        if (q.type[i] == OR_RELAX) {
            for (int64_t k = 0; k < K; ++k) {
                or_iso p = iso_at(&ph, k);
                for (int64_t j = q.seg_begin[i]; j < q.seg_end[i]; ++j)
                    free_precess(&M[3 * k], &p, gx[j], gy[j], gz[j], dt[j] * rep[j]);
            }
        } else if (q.type[i] == OR_RF && known) {
            /* preparation step once per group (Sec. 2.3), update step per isochromat */
            double (*T)[3][4] = malloc((size_t)ng[g] * sizeof(double[3][4]));
            if (!T) { rc = OR_ENOMEM; break; }
            for (int64_t G = 0; G < ng[g]; ++G) {
                or_iso p = iso_at(&ph, rep_of[g][G]);
                or_transition(p.x, p.y, p.z, p.T1, p.T2, p.dB0, p.b1, dt, rep, b1re, b1im, gx,
                              gy, gz, q.seg_begin[i], q.seg_end[i], &T[G][0][0]);
            }
            for (int64_t k = 0; k < K; ++k) affine_apply(&M[3 * k], T[gid[g][k]], M0[k]);
            free(T);
        } else if (q.type[i] == OR_RF) {
            for (int64_t k = 0; k < K; ++k) {
                or_iso p = iso_at(&ph, k);
                for (int64_t j = q.seg_begin[i]; j < q.seg_end[i]; ++j)
                    for (int32_t r = 0; r < rep[j]; ++r)
                        rf_step(&M[3 * k], &p, b1re[j], b1im[j], gx[j], gy[j], gz[j], dt[j]);
            }
        } else if (known) {
            /* with-ADC, three steps.  Step 1 (Eq. 9): block sums at t0. */
            double *Ab = calloc((size_t)ng[g] * 2, sizeof(double));
            if (!Ab) { rc = OR_ENOMEM; break; }
            for (int64_t k = 0; k < K; ++k) {
                Ab[2 * gid[g][k]] += M[3 * k];
                Ab[2 * gid[g][k] + 1] += M[3 * k + 1];
            }
            /* Step 2 (Eqs. 8, 10): each sample from the group blocks.  The
             * phase uses the gradient moment of every axis of the type (one
             * axis, or two for the two-axis types). */
            int ax[2];
            const int n_ax = type_axes(g, ax);
            const float *gax[3] = {gx, gy, gz};
            double tau = 0.0, mom[2] = {0.0, 0.0}; /* time and moments since t0 */
            for (int64_t j = q.seg_begin[i]; j < q.seg_end[i]; ++j) {
                double ga[2] = {0.0, 0.0};
                for (int a = 0; a < n_ax; ++a) ga[a] = gax[ax[a]][j];
                for (int32_t r = 0; r < rep[j]; ++r) {
                    double t_s = tau + (r + 1) * dt[j];
                    double m_s[2] = {mom[0] + ga[0] * (r + 1) * dt[j],
                                     mom[1] + ga[1] * (r + 1) * dt[j]};
                    double ar = 0.0, ai = 0.0;
                    for (int64_t G = 0; G < ng[g]; ++G) {
                        or_iso p = iso_at(&ph, rep_of[g][G]);
                        const double pv[3] = {p.x, p.y, p.z};
                        double E2 = exp(-t_s / p.T2);
                        double phi = 2.0 * OR_PI * p.dB0 * t_s;
                        for (int a = 0; a < n_ax; ++a) phi += OR_GAMMA * pv[ax[a]] * m_s[a];
                        double c = cos(phi), sn = sin(phi);
                        double br = Ab[2 * G], bi = Ab[2 * G + 1];
                        ar += E2 * (br * c + bi * sn);
                        ai += E2 * (bi * c - br * sn);
                    }
                    signal[2 * smp] = ar;
                    signal[2 * smp + 1] = ai;
                    ++smp;
                }
                tau += dt[j] * rep[j];
                mom[0] += ga[0] * dt[j] * rep[j];
                mom[1] += ga[1] * dt[j] * rep[j];
            }
            free(Ab);
            /* Step 3 (Eqs. 4-5): every isochromat to the end of the window. */
            for (int64_t k = 0; k < K; ++k) {
                or_iso p = iso_at(&ph, k);
                for (int64_t j = q.seg_begin[i]; j < q.seg_end[i]; ++j)
                    free_precess(&M[3 * k], &p, gx[j], gy[j], gz[j], dt[j] * rep[j]);
            }
        } else {
            /* conventional per-isochromat sampling for an unclassified window */
            int64_t s0 = smp;
            for (int64_t k = 0; k < K; ++k) {
                or_iso p = iso_at(&ph, k);
                smp = s0;
                for (int64_t j = q.seg_begin[i]; j < q.seg_end[i]; ++j)
                    for (int32_t r = 0; r < rep[j]; ++r) {
                        free_precess(&M[3 * k], &p, gx[j], gy[j], gz[j], dt[j]);
                        if (k == 0) signal[2 * smp] = signal[2 * smp + 1] = 0.0;
                        signal[2 * smp] += M[3 * k];
                        signal[2 * smp + 1] += M[3 * k + 1];
                        ++smp;
                    }
            }
        }
    }
    if (rc == OR_OK && Mfinal)
        for (int64_t k = 0; k < K; ++k)
            for (int c = 0; c < 3; ++c) Mfinal[c * K + k] = M[3 * k + c];
    for (int g = 0; g < OR_N_GTYPES; ++g) { free(gid[g]); free(rep_of[g]); }
    free(M);
    free_subseqs(&q);
    return rc;
}
