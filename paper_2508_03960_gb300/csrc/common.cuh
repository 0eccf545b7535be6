// Plain-data records shared by the host planner and the kernels, and the
// per-isochromat math used by every kernel (Eqs. 4-5, Eq. A1-A2).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mrsim {

// 1H gyromagnetic ratio / 2 pi (Hz/T); gamma = 2 pi * kGammaBar rad/s/T.
constexpr double kGammaBar = 42.577478518e6;
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kGamma = kTwoPi * kGammaBar;
constexpr double kLog2e = 1.4426950408889634073599246810019;

enum SubType : int { SUB_RF = 0, SUB_ADC = 1, SUB_RELAX = 2 };
// gradient types (Sec. 2.4); the two-axis types group on both positions
enum GType : int {
    G_NONE = 0, G_X = 1, G_Y = 2, G_Z = 3, G_GENERAL = 4, G_XY = 5, G_XZ = 6, G_YZ = 7
};
constexpr int kNTypes = 8;  // gradient type numbers (G_GENERAL has no groups)
// position axes of a gradient type: a0 (or -1 for no-grads / general) and a1
// (the second axis of a two-axis type, else -1)
__host__ __device__ constexpr int gtype_axis0(int t) {
    return t == G_X ? 0 : t == G_Y ? 1 : t == G_Z ? 2 : t == G_XY ? 0 : t == G_XZ ? 0
         : t == G_YZ ? 1 : -1;
}
__host__ __device__ constexpr int gtype_axis1(int t) {
    return t == G_XY ? 1 : t == G_XZ ? 2 : t == G_YZ ? 2 : -1;
}
// bit mask of the axes of a gradient type
__host__ __device__ constexpr int gtype_axes(int t) {
    return (gtype_axis0(t) >= 0 ? 1 << gtype_axis0(t) : 0) |
           (gtype_axis1(t) >= 0 ? 1 << gtype_axis1(t) : 0);
}
enum EvKind : int { EV_RF = 0, EV_ADC = 1, EV_END = 2 };

// Free-precession parameters of an advance from the state time t_w to a
// later time t (Eqs. 4-5): k = gamma_bar * int_{t_w}^{t} G dt (cycles/m per
// axis) and tau = t - t_w (s).  The FP32 form keeps every double as an
// unevaluated sum hi + lo of two floats so that phases of hundreds of turns
// keep ~1e-7-turn accuracy after reduction modulo one turn.
struct AdvF {
    float kx_hi, kx_lo, ky_hi, ky_lo, kz_hi, kz_lo, tau_hi, tau_lo;
};
struct AdvD {
    double kx, ky, kz, tau;
};

// One RF segment: rotation-vector coefficients per sub-step.
//   phi = -(b1 * are, b1 * aim, cx x + cy y + cz z + cdw dB0)   (radians)
// with are = gamma B1re dt, cx = gamma gx dt (rad/m), cdw = 2 pi dt (rad/Hz).
struct RFSegF {
    float are, aim, cx, cy, cz, cdw, dt;
    int rep;
};
struct RFSegD {
    double are, aim, cx, cy, cz, cdw, dt;
    long long rep;
};

// One ADC segment of a window: per-sub-step moment k = gamma_bar G dt
// (cycles/m, split), the sub-step length and the number of samples.
struct ADCSegF {
    float kx_hi, kx_lo, ky_hi, ky_lo, kz_hi, kz_lo, dt;
    int rep;
};
struct ADCSegD {
    double kx, ky, kz, dt;
    long long rep;
};

// Event of the fused grouped kernel.  Every event first advances M from the
// state time in closed form (Eqs. 4-5).  The advance factors as
//   M_xy <- P(e, g) Q(e, k) M_xy,  Mz <- M0 + (Mz - M0) E1(e, g)
// with the group factor P = E2 exp(-i 2 pi (pos_p k_p + dB0 tau)) and E1 of
// the isochromat's primary (with-ADC) group g, which shares pos_p, dB0, T1
// and T2, taken from a per-(event, group) table, and the per-isochromat
// factor Q = exp(-i 2 pi sum_a r_a k_a) over the other axes whose moment is
// nonzero (bit a of `mask`).  RF: then M <- A M + b M0 with combined
// transition row `row` (+ the isochromat's RF group).  ADC: add Q M_xy into
// the block sum of window `win` (Eq. 9; P is applied once per group).  END:
// store the state.
template <typename R>
struct FEvent;
// 64-byte records (FP32), 48-byte (FP64); op = kind | mask << 2 | gtype << 5
template <>
struct FEvent<float> {
    int op;
    int row;   // RF: first row of the combined-transition table of (content, gtype)
    int prow;  // first row of this event's group-factor table
    int win;   // ADC: offset of this window's block sums (complex entries)
    // gamma_bar * moment per axis (cycles/m) and, in [3], the elapsed time (s),
    // split hi + lo; every axis is filled, `mask` marks the per-isochromat ones
    float k_hi[4], k_lo[4];
    // axis-table runs: first entry of this event's phasor table exp(-i 2 pi v k_a)
    // over the distinct positions v of axis a (only for the axes in `mask`)
    int q[4];
};
template <>
struct FEvent<double> {
    int op, row, prow, win;
    double k[4];  // moments per axis, elapsed time in [3]
};
__host__ __device__ constexpr int ev_op(int kind, int mask, int gtype) {
    return kind | (mask << 2) | (gtype << 5);
}
__host__ __device__ constexpr int ev_kind(int op) { return op & 3; }
__host__ __device__ constexpr int ev_mask(int op) { return (op >> 2) & 7; }
__host__ __device__ constexpr int ev_gtype(int op) { return (op >> 5) & 7; }
// per-event inputs of the group-factor table
struct EvAdv {
    double kp;   // gamma_bar * moment on the primary type's first axis (cycles/m)
    double tau;  // time since the state time (s)
    double kp2;  // ... on its second axis (two-axis primary types; else 0)
};

// A with-ADC window for the grouped signal kernel (Eqs. 8, 10).
struct GWin {
    int gtype;
    int n_groups;
    long long ablk;      // offset of the block sums (complex entries)
    long long sample0;   // first sample (global index)
    int n_samples;
    // 1: the window is one ADC segment (constant gradient, one dwell), so
    // every group's samples form a geometric sequence with step dt (s) and
    // dk = gamma_bar g dt (cycles/m) on the group's axis, as hi + lo floats
    int uniform;
    float dt_hi, dt_lo, dk_hi, dk_lo;
    float dk2_hi, dk2_lo;  // the same on the second axis of a two-axis type
};
// per-sample time and moments since the window start on the group type's
// axes (k2: second axis of a two-axis type, else 0)
struct GSampleF {
    float tau_hi, tau_lo, k_hi, k_lo, k2_hi, k2_lo;
};
struct GSampleD {
    double tau, k, k2;
};

// ------------------------------------------------------------------------
// device helpers
// ------------------------------------------------------------------------
#ifdef __CUDACC__

// Reproducible sums.  With fx > 0 (a power of two) a sum buffer holds 64-bit
// integers and every contribution v is added as rint(v fx): integer addition
// is associative, so the total does not depend on the order in which threads
// add (FP64 atomics make the last bits vary from run to run).  The buffer is
// read back as i / fx.  fx is chosen so that no partial sum can reach 2^62.
__device__ __forceinline__ void sum_add(double *p, double v, double fx) {
    if (fx > 0.0)
        atomicAdd(reinterpret_cast<unsigned long long *>(p),
                  (unsigned long long)__double2ll_rn(v * fx));
    else
        atomicAdd(p, v);
}
__device__ __forceinline__ double sum_get(const double *p, double fx) {
    return fx > 0.0 ? (double)*reinterpret_cast<const long long *>(p) * (1.0 / fx) : *p;
}

// fractional part (turns) of a * (hi + lo), a float32 value times a
// double-length constant: the product a*hi is split exactly with one FMA.
__device__ __forceinline__ float turns_prod(float a, float hi, float lo) {
    float p = a * hi;
    float e = fmaf(a, hi, -p);  // a*hi = p + e exactly
    float r = p - rintf(p);     // exact for |p| < 2^22
    return r + fmaf(a, lo, e);
}

__device__ __forceinline__ float adv_turns(const AdvF &a, float x, float y, float z, float dB0) {
    return turns_prod(x, a.kx_hi, a.kx_lo) + turns_prod(y, a.ky_hi, a.ky_lo) +
           turns_prod(z, a.kz_hi, a.kz_lo) + turns_prod(dB0, a.tau_hi, a.tau_lo);
}
__device__ __forceinline__ double adv_turns(const AdvD &a, double x, double y, double z,
                                            double dB0) {
    double v = x * a.kx + y * a.ky + z * a.kz + dB0 * a.tau;
    return v - rint(v);
}

__device__ __forceinline__ float adv_tau(const AdvF &a) { return a.tau_hi + a.tau_lo; }
__device__ __forceinline__ double adv_tau(const AdvD &a) { return a.tau; }

// exp(-phase) as (cos, sin) of 2 pi * turns
__device__ __forceinline__ void phasor(float turns, float &c, float &s) {
    sincospif(2.0f * turns, &s, &c);
}
__device__ __forceinline__ void phasor(double turns, double &c, double &s) {
    sincospi(2.0 * turns, &s, &c);
}

// exp(-tau / T) with r = log2(e) / T precomputed (r = 0 for T = inf)
__device__ __forceinline__ float decay(float tau, float r) { return exp2f(-tau * r); }
__device__ __forceinline__ double decay(double tau, double r) { return exp2(-tau * r); }

// Free precession and relaxation over an advance (Eqs. 4-5):
//   M_xy <- M_xy exp(-tau/T2) exp(-i 2 pi turns),  Mz <- M0 + (Mz - M0) exp(-tau/T1)
template <typename R, typename A>
__device__ __forceinline__ void advance(R &mx, R &my, R &mz, R M0, R x, R y, R z, R dB0, R rT1,
                                        R rT2, const A &adv) {
    R c, s;
    phasor(adv_turns(adv, x, y, z, dB0), c, s);
    R tau = (R)adv_tau(adv);
    R E2 = decay(tau, rT2), E1 = decay(tau, rT1);
    R nx = E2 * (mx * c + my * s);
    R ny = E2 * (my * c - mx * s);
    mx = nx;
    my = ny;
    mz = M0 + (mz - M0) * E1;
}

// Transverse part only (for ADC block sums).
template <typename R, typename A>
__device__ __forceinline__ void advance_xy(R mx, R my, R x, R y, R z, R dB0, R rT2, const A &adv,
                                           R &ox, R &oy) {
    R c, s;
    phasor(adv_turns(adv, x, y, z, dB0), c, s);
    R E2 = decay((R)adv_tau(adv), rT2);
    ox = E2 * (mx * c + my * s);
    oy = E2 * (my * c - mx * s);
}

// Rotation coefficients for the vector form of Eq. A2:
//   R v = v + s (phi x v) + c2 (phi x (phi x v)),  theta^2 = |phi|^2,
//   s = sin(theta)/theta, c2 = (1 - cos(theta))/theta^2.
// Both are even in theta: for theta^2 <= 1/4 they come from their Maclaurin
// series in theta^2 (truncation < 3e-11 in FP32, < 1e-22 in FP64); above that
// from sin / cos of theta/2.
__device__ __forceinline__ void rot_coeffs(float th2, float &s, float &c2) {
    if (th2 <= 0.25f) {
        s = fmaf(th2, fmaf(th2, fmaf(th2, fmaf(th2, 1.0f / 362880.0f, -1.0f / 5040.0f),
                                     1.0f / 120.0f), -1.0f / 6.0f), 1.0f);
        c2 = fmaf(th2, fmaf(th2, fmaf(th2, fmaf(th2, 1.0f / 3628800.0f, -1.0f / 40320.0f),
                                      1.0f / 720.0f), -1.0f / 24.0f), 0.5f);
    } else {
        float th = sqrtf(th2), sh, ch;
        sincosf(0.5f * th, &sh, &ch);
        s = 2.0f * sh * ch / th;
        c2 = 2.0f * sh * sh / th2;
    }
}
__device__ __forceinline__ void rot_coeffs(double th2, double &s, double &c2) {
    if (th2 <= 0.25) {
        // sum_{n=0}^{8} (-1)^n th2^n / (2n+1)!  and  / (2n+2)!, Horner from n = 8
        s = 1.0 / 355687428096000.0;              //  1/17!
        s = fma(th2, s, -1.0 / 1307674368000.0);  // -1/15!
        s = fma(th2, s, 1.0 / 6227020800.0);      //  1/13!
        s = fma(th2, s, -1.0 / 39916800.0);       // -1/11!
        s = fma(th2, s, 1.0 / 362880.0);          //  1/9!
        s = fma(th2, s, -1.0 / 5040.0);           // -1/7!
        s = fma(th2, s, 1.0 / 120.0);             //  1/5!
        s = fma(th2, s, -1.0 / 6.0);              // -1/3!
        s = fma(th2, s, 1.0);
        c2 = 1.0 / 6402373705728000.0;            //  1/18!
        c2 = fma(th2, c2, -1.0 / 20922789888000.0);  // -1/16!
        c2 = fma(th2, c2, 1.0 / 87178291200.0);      //  1/14!
        c2 = fma(th2, c2, -1.0 / 479001600.0);       // -1/12!
        c2 = fma(th2, c2, 1.0 / 3628800.0);          //  1/10!
        c2 = fma(th2, c2, -1.0 / 40320.0);           // -1/8!
        c2 = fma(th2, c2, 1.0 / 720.0);              //  1/6!
        c2 = fma(th2, c2, -1.0 / 24.0);              // -1/4!
        c2 = fma(th2, c2, 0.5);                      //  1/2!
    } else {
        double th = sqrt(th2), sh, ch;
        sincos(0.5 * th, &sh, &ch);
        s = 2.0 * sh * ch / th;
        c2 = 2.0 * sh * sh / th2;
    }
}

// One RF sub-step on a magnetization vector: M <- D R M (App. A).
// em1 = expm1(-dt/T1), em2 = expm1(-dt/T2) so that relaxation adds small
// increments instead of multiplying by factors close to one.
template <typename R>
__device__ __forceinline__ void rf_step(R &mx, R &my, R &mz, R M0, R px, R py, R pz, R em1,
                                        R em2) {
    R th2 = px * px + py * py + pz * pz;
    R s, c2;
    rot_coeffs(th2, s, c2);
    // q = phi x M ; M += s q + c2 (phi x q)
    R qx = py * mz - pz * my;
    R qy = pz * mx - px * mz;
    R qz = px * my - py * mx;
    R wx = py * qz - pz * qy;
    R wy = pz * qx - px * qz;
    R wz = px * qy - py * qx;
    mx += s * qx + c2 * wx;
    my += s * qy + c2 * wy;
    mz += s * qz + c2 * wz;
    mx += mx * em2;
    my += my * em2;
    mz -= (M0 - mz) * em1;
}

#endif  // __CUDACC__

}  // namespace mrsim
