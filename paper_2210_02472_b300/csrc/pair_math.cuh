// pair_math.cuh -- per-pair arithmetic shared by the pair kernels (one-sided form).
//
// FP64: every operation in FP64; the reciprocal square root is seeded by the FP32
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

__device__ __forceinline__ double rsqrt_f64(double r2) {
    const double y0 = (double)rsqrt_hw(__double2float_rn(r2));
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
    if (r2 == 0.0) { set_error(err, FSI_ERR_NONFINITE); return; }
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
