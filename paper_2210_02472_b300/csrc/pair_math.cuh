// pair_math.cuh -- per-pair arithmetic shared by the pair kernels (one-sided form).
//
// FP64: every operation in FP64; the reciprocal square root is seeded by the FP64
// hardware approximation and refined by the second-order series of (1 - e)^{-1/2},
// y = y0 (1 + e/2 + 3 e^2/8) with e = 1 - r^2 y0^2.
// MIXED: separations from FP32 hi/lo position splits, FP32 arithmetic with the rsqrt
// residual correction folded into the mass-prescaled record constants (2.5 m, -1.5 m).
#pragma once
#include "fsi_internal.cuh"

namespace fsi {

// ---------------------------------------------------------------------------------
// Per-pair arithmetic.
struct MixI {
    float xh, yh, zh, xl, yl, zl;
    float ax, ay, az;
};

template <bool CHK>
__device__ __forceinline__ void mix_acc_pair(const float4 h, const float4 l, const MixI& p,
                                             float eps2f, bool self,
                                             float& fx, float& fy, float& fz) {
    const float dx = (h.x - p.xh) + (l.x - p.xl);
    const float dy = (h.y - p.yh) + (l.y - p.yl);
    const float dz = (h.z - p.zh) + (l.z - p.zl);
    float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2f)));
    if (CHK) r2 = self ? 1.0f : r2;
    const float y = rsqrt_hw(r2);
    const float y2 = y * y;
    const float sres = r2 * y2;                      // 1 - e, e = rsqrt residual
    // m r^-3 = m y^3 (1 - e)^{-3/2} ~ y^3 (2.5 m - 1.5 m (1 - e)); h.w = 2.5 m, l.w = -1.5 m
    float w = (y2 * y) * fmaf(sres, l.w, h.w);
    if (CHK) w = self ? 0.0f : w;                    // excluded pair (self, or masked)
    fx = fmaf(w, dx, fx);
    fy = fmaf(w, dy, fy);
    fz = fmaf(w, dz, fz);
}

template <bool CHK>
__device__ __forceinline__ void mix_grad_pair(const float4 h, const float4 l, const float4 aj,
                                              const MixI& p, float eps2f, bool self,
                                              float& gx, float& gy, float& gz) {
    const float dx = (h.x - p.xh) + (l.x - p.xl);
    const float dy = (h.y - p.yh) + (l.y - p.yl);
    const float dz = (h.z - p.zh) + (l.z - p.zl);
    float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2f)));
    if (CHK) r2 = self ? 1.0f : r2;
    const float y = rsqrt_hw(r2);
    const float y2 = y * y;
    const float sres = r2 * y2;                      // 1 - e
    float w = (y2 * y) * fmaf(sres, l.w, h.w);       // m r^-3
    if (CHK) w = self ? 0.0f : w;                    // excluded pair (self, or masked)
    const float bx = aj.x - p.ax, by = aj.y - p.ay, bz = aj.z - p.az;   // a_ji
    const float dot = fmaf(bx, dx, fmaf(by, dy, bz * dz));
    // -3 m r^-5 = -3 w y^2 (1 + e) = w y^2 (3 (1 - e) - 6)
    const float q = (w * y2) * fmaf(3.0f, sres, -6.0f);
    const float s = q * dot;
    gx = fmaf(w, bx, fmaf(s, dx, gx));
    gy = fmaf(w, by, fmaf(s, dy, gy));
    gz = fmaf(w, bz, fmaf(s, dz, gz));
}

// ---------------------------------------------------------------------------------
// Packed FP32 pairs (add/mul/fma.rn.f32x2, sm_100 and later): two receivers per
// instruction, each half rounding exactly as the scalar form above.
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ void set_half(float2& d, int h, float v) {
    if (h) d.y = v;
    else d.x = v;
}
__device__ __forceinline__ float2 rsqrt2(float2 v) { return make_float2(rsqrt_hw(v.x), rsqrt_hw(v.y)); }

// Float-float accumulation of two sums at once: (hi, lo) += v by the TwoSum of Knuth
// (six FP32 operations, exact error term; s - a formed as fma(a, -1, s), one rounding),
// acc = (hi_0, hi_1, lo_0, lo_1).  Keeps ~48 bits across source tiles without FP64
// instructions (the B300 FP64 unit issues ~1/64 of the FP32 rate).
__device__ __forceinline__ void ff_add2(float4& acc, const float2 v) {
    const float2 m1 = bc2(-1.0f);
    const float2 hi = make_float2(acc.x, acc.y);
    const float2 s = __fadd2_rn(hi, v);
    const float2 bb = __ffma2_rn(hi, m1, s);                  // s - hi
    const float2 e1 = __ffma2_rn(__ffma2_rn(bb, m1, s), m1, hi);   // hi - (s - bb)
    const float2 e2 = __ffma2_rn(bb, m1, v);                  // v - bb
    const float2 lo = __fadd2_rn(make_float2(acc.z, acc.w), __fadd2_rn(e1, e2));
    acc = make_float4(s.x, s.y, lo.x, lo.y);
}

// Scalar float-float accumulation: (hi, lo) += v, TwoSum of Knuth (the exact rounding
// error of hi + v goes into lo).
__device__ __forceinline__ void ff_acc(float& hi, float& lo, float v) {
    const float s = __fadd_rn(hi, v);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
}

// i-side state of a packed pair of particles (low half: particle 2p, high half: 2p+1).
struct X2I {
    float2 nxh, nyh, nzh, nxl, nyl, nzl;   // -xh, -yh, -zh, -xl, -yl, -zl
    float2 nA, nB;                         // -2.5 m_i, +1.5 m_i (near acc j-side weight)
    float2 nm;                             // -m_i
    float2 nax, nay, naz;                  // gradient: -a_i
};

// hi/lo separation of a source from both particles of a pair.
__device__ __forceinline__ void x2_sep_near(const float4 h, const float4 l, const X2I& p,
                                            float2& dx, float2& dy, float2& dz) {
    dx = __fadd2_rn(__fadd2_rn(bc2(h.x), p.nxh), __fadd2_rn(bc2(l.x), p.nxl));
    dy = __fadd2_rn(__fadd2_rn(bc2(h.y), p.nyh), __fadd2_rn(bc2(l.y), p.nyl));
    dz = __fadd2_rn(__fadd2_rn(bc2(h.z), p.nzh), __fadd2_rn(bc2(l.z), p.nzl));
}

// y = r^-1 (hardware), y2 = y^2, sres = r^2 y^2 (= 1 - e), y3 = y^3.
__device__ __forceinline__ void x2_geom(float2 dx, float2 dy, float2 dz, float2 eps2, float2& y2,
                                        float2& sres, float2& y3) {
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, eps2)));
    const float2 y = rsqrt2(r2);
    y2 = __fmul2_rn(y, y);
    sres = __fmul2_rn(r2, y2);
    y3 = __fmul2_rn(y2, y);
}

// One-sided packed terms of source j on both particles of a pair (the pair's particles
// must differ from j): acceleration f += m_j r^-3 d and gradient g += m_j T(d)(a_j - a_i),
// operation for operation mix_acc_pair / mix_grad_pair.
__device__ __forceinline__ void x2_acc_one(const float4 h, const float4 l, const X2I& p, float2 eps2,
                                           float2 (&f)[3]) {
    float2 dx, dy, dz, y2, sres, y3;
    x2_sep_near(h, l, p, dx, dy, dz);
    x2_geom(dx, dy, dz, eps2, y2, sres, y3);
    const float2 w = __fmul2_rn(y3, __ffma2_rn(sres, bc2(l.w), bc2(h.w)));    // m_j r^-3
    f[0] = __ffma2_rn(w, dx, f[0]);
    f[1] = __ffma2_rn(w, dy, f[1]);
    f[2] = __ffma2_rn(w, dz, f[2]);
}

__device__ __forceinline__ void x2_grad_one(const float4 h, const float4 l, const float4 aj, const X2I& p,
                                            float2 eps2, float2 (&g)[3]) {
    float2 dx, dy, dz, y2, sres, y3;
    x2_sep_near(h, l, p, dx, dy, dz);
    x2_geom(dx, dy, dz, eps2, y2, sres, y3);
    const float2 w = __fmul2_rn(y3, __ffma2_rn(sres, bc2(l.w), bc2(h.w)));    // m_j r^-3
    const float2 bx = __fadd2_rn(bc2(aj.x), p.nax), by = __fadd2_rn(bc2(aj.y), p.nay),
                 bz = __fadd2_rn(bc2(aj.z), p.naz);
    const float2 dot = __ffma2_rn(bx, dx, __ffma2_rn(by, dy, __fmul2_rn(bz, dz)));
    const float2 q = __fmul2_rn(__fmul2_rn(w, y2), __ffma2_rn(bc2(3.0f), sres, bc2(-6.0f)));
    const float2 s = __fmul2_rn(q, dot);
    g[0] = __ffma2_rn(w, bx, __ffma2_rn(s, dx, g[0]));
    g[1] = __ffma2_rn(w, by, __ffma2_rn(s, dy, g[1]));
    g[2] = __ffma2_rn(w, bz, __ffma2_rn(s, dz, g[2]));
}

// The same with a source that may be one of the pair's particles (self_lo / self_hi): as
// in the checked scalar forms, r^2 is replaced by 1 and the weight by 0 for that half.
__device__ __forceinline__ void x2_geom_chk(float2 dx, float2 dy, float2 dz, float2 eps2, bool self_lo,
                                            bool self_hi, float2& y2, float2& sres, float2& y3) {
    float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, eps2)));
    r2.x = self_lo ? 1.0f : r2.x;
    r2.y = self_hi ? 1.0f : r2.y;
    const float2 y = rsqrt2(r2);
    y2 = __fmul2_rn(y, y);
    sres = __fmul2_rn(r2, y2);
    y3 = __fmul2_rn(y2, y);
}

__device__ __forceinline__ void x2_acc_one_chk(const float4 h, const float4 l, const X2I& p, float2 eps2,
                                               bool self_lo, bool self_hi, float2 (&f)[3]) {
    float2 dx, dy, dz, y2, sres, y3;
    x2_sep_near(h, l, p, dx, dy, dz);
    x2_geom_chk(dx, dy, dz, eps2, self_lo, self_hi, y2, sres, y3);
    float2 w = __fmul2_rn(y3, __ffma2_rn(sres, bc2(l.w), bc2(h.w)));          // m_j r^-3
    w.x = self_lo ? 0.0f : w.x;
    w.y = self_hi ? 0.0f : w.y;
    f[0] = __ffma2_rn(w, dx, f[0]);
    f[1] = __ffma2_rn(w, dy, f[1]);
    f[2] = __ffma2_rn(w, dz, f[2]);
}

__device__ __forceinline__ void x2_grad_one_chk(const float4 h, const float4 l, const float4 aj, const X2I& p,
                                                float2 eps2, bool self_lo, bool self_hi, float2 (&g)[3]) {
    float2 dx, dy, dz, y2, sres, y3;
    x2_sep_near(h, l, p, dx, dy, dz);
    x2_geom_chk(dx, dy, dz, eps2, self_lo, self_hi, y2, sres, y3);
    float2 w = __fmul2_rn(y3, __ffma2_rn(sres, bc2(l.w), bc2(h.w)));          // m_j r^-3
    w.x = self_lo ? 0.0f : w.x;
    w.y = self_hi ? 0.0f : w.y;
    const float2 bx = __fadd2_rn(bc2(aj.x), p.nax), by = __fadd2_rn(bc2(aj.y), p.nay),
                 bz = __fadd2_rn(bc2(aj.z), p.naz);
    const float2 dot = __ffma2_rn(bx, dx, __ffma2_rn(by, dy, __fmul2_rn(bz, dz)));
    const float2 q = __fmul2_rn(__fmul2_rn(w, y2), __ffma2_rn(bc2(3.0f), sres, bc2(-6.0f)));
    const float2 s = __fmul2_rn(q, dot);
    g[0] = __ffma2_rn(w, bx, __ffma2_rn(s, dx, g[0]));
    g[1] = __ffma2_rn(w, by, __ffma2_rn(s, dy, g[1]));
    g[2] = __ffma2_rn(w, bz, __ffma2_rn(s, dz, g[2]));
}

// FP64 reciprocal square root: the hardware FP64 approximation (no conversion to and from
// FP32 on the FP64 pipe, and the whole FP64 exponent range) refined by the second-order
// step of (1 - e)^{-1/2} above.
__device__ __forceinline__ double rsqrt_f64(double r2) {
    double y0;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(r2));
    const double t = r2 * y0;
    const double e = fma(-t, y0, 1.0);
    const double p = fma(0.375, e, 0.5);
    return fma(y0 * e, p, y0);
}

struct F64I {
    double x, y, z;
    double ax, ay, az;
};

template <bool CHK>
__device__ __forceinline__ void f64_acc_pair(const D4 j, const F64I& p, double eps2,
                                             bool self, double& fx, double& fy, double& fz) {
    const double dx = j.x - p.x, dy = j.y - p.y, dz = j.z - p.z;
    double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
    if (CHK) r2 = self ? 1.0 : r2;
    const double y = rsqrt_f64(r2);
    const double y2 = y * y;
    double w = j.w * (y2 * y);
    if (CHK) w = self ? 0.0 : w;                     // excluded pair (self, or masked)
    fx = fma(w, dx, fx);
    fy = fma(w, dy, fy);
    fz = fma(w, dz, fz);
}

template <bool CHK>
__device__ __forceinline__ void f64_grad_pair(const D4 j, const D4 aj, const F64I& p,
                                              double eps2, bool self,
                                              double& gx, double& gy, double& gz) {
    const double dx = j.x - p.x, dy = j.y - p.y, dz = j.z - p.z;
    double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
    if (CHK) r2 = self ? 1.0 : r2;
    const double y = rsqrt_f64(r2);
    const double y2 = y * y;
    double w = j.w * (y2 * y);
    if (CHK) w = self ? 0.0 : w;                     // excluded pair (self, or masked)
    const double bx = aj.x - p.ax, by = aj.y - p.ay, bz = aj.z - p.az;
    const double dot = fma(bx, dx, fma(by, dy, bz * dz));
    const double s = (w * y2) * (-3.0 * dot);
    gx = fma(w, bx, fma(s, dx, gx));
    gy = fma(w, by, fma(s, dy, gy));
    gz = fma(w, bz, fma(s, dz, gz));
}

}  // namespace fsi

namespace fsi {

// ---------------------------------------------------------------------------------
// Time-step pair update (Sect. 3.4), division-free: the free-fall minimum of
// r^3 / (m_i + m_j) is tracked as the minimum of r^6 / (m_i + m_j)^2 and the fly-by
// minimum of r / |v_ij| as that of r^2 / |v_ij|^2, each as a (numerator, denominator)
// pair compared by cross-multiplication; a_i and the jerk j_i use the softened kernel.
template <class T>
struct StepAcc {
    T ffn, ffd, fbn, fbd;
    T ax, ay, az, jx, jy, jz;
    __device__ __forceinline__ void init() {
        ffn = fbn = (T)INFINITY;
        ffd = fbd = (T)1;
        ax = ay = az = jx = jy = jz = (T)0;
    }
};

// d = r_j - r_i, u = v_j - v_i, ms = m_i + m_j, y = 1/sqrt(|d|^2 + eps2) (refined).
template <class T>
__device__ __forceinline__ void step_pair(StepAcc<T>& s, T dx, T dy, T dz, T du, T dv, T dw,
                                          T d2, T mj, T ms, T y) {
    const T num = d2 * d2 * d2, den = ms * ms;
    if (num * s.ffd < s.ffn * den) { s.ffn = num; s.ffd = den; }
    const T u2 = du * du + dv * dv + dw * dw;
    if (u2 > (T)0 && d2 * s.fbd < s.fbn * u2) { s.fbn = d2; s.fbd = u2; }
    const T y2 = y * y;
    const T w = mj * (y2 * y);
    const T rv = dx * du + dy * dv + dz * dw;
    const T c3 = (T)(-3) * rv * y2;
    s.ax += w * dx; s.ay += w * dy; s.az += w * dz;
    s.jx += w * (c3 * dx + du);
    s.jy += w * (c3 * dy + dv);
    s.jz += w * (c3 * dz + dw);
}

template <class T>
__device__ __forceinline__ double step_finish(const StepAcc<T>& s, double eta_ff, double eta_fb,
                                              double eta_jerk) {
    double e = INFINITY;
    if (isfinite((double)s.ffn)) e = eta_ff * sqrt(sqrt((double)s.ffn / (double)s.ffd));
    if (isfinite((double)s.fbn)) e = fmin(e, eta_fb * sqrt((double)s.fbn / (double)s.fbd));
    const double jn = sqrt((double)s.jx * s.jx + (double)s.jy * s.jy + (double)s.jz * s.jz);
    if (jn > 0.0)
        e = fmin(e, eta_jerk * sqrt((double)s.ax * s.ax + (double)s.ay * s.ay + (double)s.az * s.az) / jn);
    return e;
}

__device__ __forceinline__ float rsqrt_f32_refined(float r2) {
    const float y = rsqrt_hw(r2);
    return y * fmaf(-0.5f * r2, y * y, 1.5f);
}

}  // namespace fsi

namespace fsi {

// ---------------------------------------------------------------------------------
// PN1.0 pair acceleration (two-body 1PN EIH, harmonic coordinates), body i due to j:
//   n = (x_i - x_j)/r,
//   a = m_j/(c^2 r^2) { n [ -v_i^2 - 2 v_j^2 + 4 v_i.v_j + 1.5 (n.v_j)^2 + 5 m_i/r + 4 m_j/r ]
//                      + (v_i - v_j) [ 4 n.v_i - 3 n.v_j ] }
__device__ __forceinline__ void pn_pair(double xi, double yi, double zi, double vxi, double vyi,
                                        double vzi, double mi, double xj, double yj, double zj,
                                        double vxj, double vyj, double vzj, double mj, double ic2,
                                        double& ax, double& ay, double& az, int* err) {
    const double rx = xi - xj, ry = yi - yj, rz = zi - zj;
    const double r2 = rx * rx + ry * ry + rz * rz;
    if (r2 == 0.0) { set_error(err, FSI_ERR_COINCIDENT); return; }
    const double ir = 1.0 / sqrt(r2);
    const double nx = rx * ir, ny = ry * ir, nz = rz * ir;
    const double vi2 = vxi * vxi + vyi * vyi + vzi * vzi;
    const double vj2 = vxj * vxj + vyj * vyj + vzj * vzj;
    const double vivj = vxi * vxj + vyi * vyj + vzi * vzj;
    const double nvi = nx * vxi + ny * vyi + nz * vzi;
    const double nvj = nx * vxj + ny * vyj + nz * vzj;
    const double cn = -vi2 - 2.0 * vj2 + 4.0 * vivj + 1.5 * nvj * nvj + (5.0 * mi + 4.0 * mj) * ir;
    const double cv = 4.0 * nvi - 3.0 * nvj;
    const double pre = mj * ic2 * ir * ir;
    ax += pre * (cn * nx + cv * (vxi - vxj));
    ay += pre * (cn * ny + cv * (vyi - vyj));
    az += pre * (cn * nz + cv * (vzi - vzj));
}

}  // namespace fsi
