// vjp_kernels.cu -- adjoint (vector-Jacobian product) pair kernels, FP64.
//
// For a receiver k and source j != k of one set (d = r_j - r_k, s^2 = |d|^2 + eps2):
//   T(d)    = I / s^3 - 3 d d^T / s^5                      (Jacobian of d / s^3)
//   Q(d, b) = -3/s^5 (b d^T + d b^T + (d.b) I) + 15 (d.b) d d^T / s^7   (d(T(d) b)/dd)
// VJP of the acceleration a_k = sum_j m_j d / s^3 (Sect. 2.1, Eq. new-newton-acc) with
// cotangent u:
//   xbar_k = sum_j T(d) (m_k u_j - m_j u_k),     mbar_k = - sum_j (u_j . d) / s^3
// VJP of the gradient sum G_k = sum_j m_j T(d) (a_j - a_k) (Eq. new-grad-acc) through its
// explicit dependence on r and m (accelerations held fixed), cotangent w:
//   xbar_k = sum_j Q(d, a_j - a_k) (m_k w_j - m_j w_k),
//   mbar_k = - sum_j w_j . T(d) (a_j - a_k)
// (the dependence of G on a has the same pair form as the acceleration's xbar).
//
// The kernels are FP64-pipe bound on B300.  A CTA of 128 receivers loops over a slice of
// the sources (blockIdx.y), staged through shared memory; the slice sums are added to the
// outputs with red.global.add (scaled by sx for xbar and sm for mbar).
#include <algorithm>

#include "fsi_internal.cuh"

namespace fsi {

constexpr int kVjpThreads = 128;
constexpr int kVjpTile = 128;

__device__ __forceinline__ double vjp_rsqrt(double r2) {
    double y0;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(r2));
    const double t = r2 * y0;
    const double e = fma(-t, y0, 1.0);
    return fma(y0 * e, fma(0.375, e, 0.5), y0);
}

__device__ __forceinline__ void red_add_f64(double* p, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" :: "l"(p), "d"(v) : "memory");
}

// kind 0: acceleration VJP (vec = u); kind 1: gradient VJP (vec = w, acc = a).
template <int KIND>
__global__ void __launch_bounds__(kVjpThreads) vjp_pair_kernel(
    int n, const D4* __restrict__ rec, const D4* __restrict__ vec, const D4* __restrict__ acc,
    double eps2, int j_per_slice, double sx, double sm, double* __restrict__ xbar,
    double* __restrict__ mbar, int* err) {
    __shared__ D4 sr[kVjpTile], sv[kVjpTile], sa[KIND == 1 ? kVjpTile : 1];
    const int k = blockIdx.x * kVjpThreads + threadIdx.x;
    const int kk = min(k, n - 1);
    const D4 rk = rec[kk];
    const D4 vk = vec[kk];
    D4 ak = make_d4(0, 0, 0, 0);
    if (KIND == 1) ak = acc[kk];
    const int js = blockIdx.y * j_per_slice;
    const int je = min(n, js + j_per_slice);
    double gx = 0, gy = 0, gz = 0, gm = 0;
    bool bad = false;
    for (int j0 = js; j0 < je; j0 += kVjpTile) {
        __syncthreads();
        const int cnt = min(kVjpTile, je - j0);
        if (threadIdx.x < cnt) {
            sr[threadIdx.x] = rec[j0 + threadIdx.x];
            sv[threadIdx.x] = vec[j0 + threadIdx.x];
            if (KIND == 1) sa[threadIdx.x] = acc[j0 + threadIdx.x];
        }
        __syncthreads();
        for (int t = 0; t < cnt; ++t) {
            if (j0 + t == kk) continue;
            const D4 rj = sr[t], vj = sv[t];
            const double dx = rj.x - rk.x, dy = rj.y - rk.y, dz = rj.z - rk.z;
            const double s2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
            if (s2 == 0.0) { bad = true; continue; }
            const double y = vjp_rsqrt(s2);
            const double y2 = y * y;
            const double y3 = y2 * y;
            const double y5 = y3 * y2;
            // c = m_k v_j - m_j v_k
            const double cx = fma(rk.w, vj.x, -rj.w * vk.x);
            const double cy = fma(rk.w, vj.y, -rj.w * vk.y);
            const double cz = fma(rk.w, vj.z, -rj.w * vk.z);
            const double dc = fma(dx, cx, fma(dy, cy, dz * cz));
            if (KIND == 0) {
                const double t3 = -3.0 * y5 * dc;
                gx += fma(y3, cx, t3 * dx);
                gy += fma(y3, cy, t3 * dy);
                gz += fma(y3, cz, t3 * dz);
                gm -= fma(vj.x, dx, fma(vj.y, dy, vj.z * dz)) * y3;
            } else {
                const D4 aj = sa[t];
                const double bx = aj.x - ak.x, by = aj.y - ak.y, bz = aj.z - ak.z;
                const double db = fma(dx, bx, fma(dy, by, dz * bz));
                const double bc = fma(bx, cx, fma(by, cy, bz * cz));
                const double A = -3.0 * y5;
                const double B = 15.0 * (y5 * y2) * db * dc;
                gx += fma(A, fma(bx, dc, fma(dx, bc, db * cx)), B * dx);
                gy += fma(A, fma(by, dc, fma(dy, bc, db * cy)), B * dy);
                gz += fma(A, fma(bz, dc, fma(dz, bc, db * cz)), B * dz);
                // -w_j . T(d) b
                const double wb = fma(vj.x, bx, fma(vj.y, by, vj.z * bz));
                const double wd = fma(vj.x, dx, fma(vj.y, dy, vj.z * dz));
                gm -= fma(y3, wb, A * db * wd);
            }
        }
    }
    if (k >= n) return;
    if (bad) set_error(err, FSI_ERR_NONFINITE);
    if (xbar) {
        red_add_f64(xbar + k, sx * gx);
        red_add_f64(xbar + (size_t)n + k, sx * gy);
        red_add_f64(xbar + 2 * (size_t)n + k, sx * gz);
    }
    if (mbar) red_add_f64(mbar + k, sm * gm);
}

cudaError_t launch_vjp_pair(int kind, int n, const void* rec, const void* vec, const void* acc,
                            double eps2, double sx, double sm, double* xbar, double* mbar,
                            int* err, int sm_count, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int bx = (n + kVjpThreads - 1) / kVjpThreads;
    // enough CTAs for ~4 per SM, each slice at least 4 tiles
    int slices = (4 * sm_count + bx - 1) / bx;
    slices = std::max(1, std::min(slices, (n + 4 * kVjpTile - 1) / (4 * kVjpTile)));
    int jps = (n + slices - 1) / slices;
    jps = (jps + kVjpTile - 1) / kVjpTile * kVjpTile;
    slices = (n + jps - 1) / jps;
    dim3 grid(bx, slices);
    const D4* r = reinterpret_cast<const D4*>(rec);
    const D4* v = reinterpret_cast<const D4*>(vec);
    const D4* a = reinterpret_cast<const D4*>(acc);
    if (kind == 0) { vjp_pair_kernel<0><<<grid, kVjpThreads, 0, s>>>(n, r, v, a, eps2, jps, sx, sm, xbar, mbar, err); note_launch(); }
    else { vjp_pair_kernel<1><<<grid, kVjpThreads, 0, s>>>(n, r, v, a, eps2, jps, sx, sm, xbar, mbar, err); note_launch(); }
    return cudaGetLastError();
}

// out = a + c * b over 3 x n entries (a == nullptr: out = c * b)
__global__ void lincomb3_kernel(int n3, const double* __restrict__ a, const double* __restrict__ b,
                                double c, double* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n3) out[k] = a ? fma(c, b[k], a[k]) : c * b[k];
}

cudaError_t launch_lincomb3(int n, const double* a, const double* b, double c, double* out,
                            cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int n3 = 3 * n;
    { lincomb3_kernel<<<(n3 + 255) / 256, 256, 0, s>>>(n3, a, b, c, out); note_launch(); }
    return cudaGetLastError();
}

// gm[idx[k]] += src[k]
__global__ void scatter_add1_kernel(int n, const double* __restrict__ src, const int* __restrict__ idx,
                                    double* __restrict__ dst) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = idx ? idx[k] : k;
    dst[i] += src[k];
}

cudaError_t launch_scatter_add1(int n, const double* src, const int* idx, double* dst,
                                cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    { scatter_add1_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, src, idx, dst); note_launch(); }
    return cudaGetLastError();
}

}  // namespace fsi
