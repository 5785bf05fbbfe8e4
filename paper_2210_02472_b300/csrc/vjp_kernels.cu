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

// ---------------------------------------------------------------------------------
// Symmetric form: every unordered pair once.  T(d) and Q(d, b) are even in d and b, and
// c = m_k v_j - m_j v_k changes sign when k and j swap, so the xbar terms of the pair on
// j are those on k with the opposite sign; the mbar terms on j take v_k (and a_k - a_j)
// in place of v_j (a_j - a_k).  Work items (blockIdx.x = b * (1 + nchunk) + c): block b of
// 128 receivers (one per thread) against c = 0: its own tile, one-sided (self pair
// skipped), or c >= 1: chunk c - 1 of the tiles above it, both sides.  The source side
// runs a ring in each warp: at step t lane l pairs its receiver with source (l + t) mod 32
// of a 32-source sub-tile and then hands the source-side sums to lane l - 1, so after 32
// steps lane l holds the warp's total for source l; warps add their totals with red.add.
template <int KIND>
__device__ __forceinline__ void vjp_sym_pair(const D4 rk, const D4 vk, const D4 ak, const D4 rj,
                                             const D4 vj, const D4 aj, double eps2, double (&g)[4],
                                             double (&h)[4], bool& bad) {
    const double dx = rj.x - rk.x, dy = rj.y - rk.y, dz = rj.z - rk.z;
    double s2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
    bad |= s2 == 0.0;
    s2 = s2 == 0.0 ? 1.0 : s2;
    const double y = vjp_rsqrt(s2);
    const double y2 = y * y;
    const double y3 = y2 * y;
    const double y5 = y3 * y2;
    const double cx = fma(rk.w, vj.x, -rj.w * vk.x);
    const double cy = fma(rk.w, vj.y, -rj.w * vk.y);
    const double cz = fma(rk.w, vj.z, -rj.w * vk.z);
    const double dc = fma(dx, cx, fma(dy, cy, dz * cz));
    double tx, ty, tz;
    if (KIND == 0) {
        const double t3 = -3.0 * y5 * dc;
        tx = fma(y3, cx, t3 * dx);
        ty = fma(y3, cy, t3 * dy);
        tz = fma(y3, cz, t3 * dz);
        g[3] -= fma(vj.x, dx, fma(vj.y, dy, vj.z * dz)) * y3;
        h[3] += fma(vk.x, dx, fma(vk.y, dy, vk.z * dz)) * y3;
    } else {
        const double bx = aj.x - ak.x, by = aj.y - ak.y, bz = aj.z - ak.z;
        const double db = fma(dx, bx, fma(dy, by, dz * bz));
        const double bc = fma(bx, cx, fma(by, cy, bz * cz));
        const double A = -3.0 * y5;
        const double B = 15.0 * (y5 * y2) * db * dc;
        tx = fma(A, fma(bx, dc, fma(dx, bc, db * cx)), B * dx);
        ty = fma(A, fma(by, dc, fma(dy, bc, db * cy)), B * dy);
        tz = fma(A, fma(bz, dc, fma(dz, bc, db * cz)), B * dz);
        const double Adb = A * db;
        g[3] -= fma(y3, fma(vj.x, bx, fma(vj.y, by, vj.z * bz)), Adb * fma(vj.x, dx, fma(vj.y, dy, vj.z * dz)));
        h[3] += fma(y3, fma(vk.x, bx, fma(vk.y, by, vk.z * bz)), Adb * fma(vk.x, dx, fma(vk.y, dy, vk.z * dz)));
    }
    g[0] += tx; g[1] += ty; g[2] += tz;
    h[0] -= tx; h[1] -= ty; h[2] -= tz;
}

template <int KIND>
__global__ void __launch_bounds__(kVjpThreads) vjp_sym_kernel(
    int n, const D4* __restrict__ rec, const D4* __restrict__ vec, const D4* __restrict__ acc,
    double eps2, int chunk, int nchunk, double sx, double sm, double* __restrict__ xbar,
    double* __restrict__ mbar, int* err) {
    __shared__ D4 sr[kVjpTile], sv[kVjpTile], sa[KIND == 1 ? kVjpTile : 1];
    const int b = blockIdx.x / (1 + nchunk);
    const int c = blockIdx.x % (1 + nchunk);
    const int ntj = (n + kVjpTile - 1) / kVjpTile;
    const bool diag = (c == 0);
    int t0, t1;
    if (diag) { t0 = b; t1 = min(b + 1, ntj); }
    else { t0 = b + 1 + (c - 1) * chunk; t1 = min(t0 + chunk, ntj); }
    if (t0 >= t1) return;                       // uniform: before any barrier
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = b * kVjpThreads + threadIdx.x;
    const bool kvalid = k < n;
    const int kk = min(k, n - 1);
    const D4 rk = rec[kk];
    D4 vk = vec[kk];
    D4 ak = make_d4(0, 0, 0, 0);
    if (KIND == 1) ak = acc[kk];
    double g[4] = {0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    if (!kvalid) vk = make_d4(0, 0, 0, 0);      // (symmetric items only have full blocks)
    for (int t = t0; t < t1; ++t) {
        const int j0 = t * kVjpTile;
        const int cnt = min(kVjpTile, n - j0);
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            sr[threadIdx.x] = rec[j0 + threadIdx.x];
            sv[threadIdx.x] = vec[j0 + threadIdx.x];
            if (KIND == 1) sa[threadIdx.x] = acc[j0 + threadIdx.x];
        }
        __syncthreads();
        if (diag) {
            double hdummy[4];
            for (int q = 0; q < cnt; ++q) {
                if (j0 + q == kk) continue;
                hdummy[0] = hdummy[1] = hdummy[2] = hdummy[3] = 0.0;
                vjp_sym_pair<KIND>(rk, vk, ak, sr[q], sv[q], KIND == 1 ? sa[q] : ak, eps2, g, hdummy, bad);
            }
        } else {
            // full 32-source sub-tiles of this tile, every warp over every sub-tile
            for (int sub = 0; sub * 32 < cnt; ++sub) {
                const int base = sub * 32;
                const bool sfull = base + 32 <= cnt;
                double h[4] = {0.0, 0.0, 0.0, 0.0};
                for (int st = 0; st < 32; ++st) {
                    const int q = base + ((lane + st) & 31);
                    if (sfull || q < cnt)
                        vjp_sym_pair<KIND>(rk, vk, ak, sr[q], sv[q], KIND == 1 ? sa[q] : ak, eps2, g, h, bad);
#pragma unroll
                    for (int e = 0; e < 4; ++e) h[e] = __shfl_sync(0xffffffffu, h[e], (lane + 1) & 31);
                }
                // lane l now holds the warp's totals for source base + l
                if (base + lane < cnt) {
                    const int j = j0 + base + lane;
                    if (xbar) {
                        red_add_f64(xbar + j, sx * h[0]);
                        red_add_f64(xbar + (size_t)n + j, sx * h[1]);
                        red_add_f64(xbar + 2 * (size_t)n + j, sx * h[2]);
                    }
                    if (mbar) red_add_f64(mbar + j, sm * h[3]);
                }
            }
        }
    }
    (void)warp;
    if (!kvalid) return;
    if (bad) set_error(err, FSI_ERR_NONFINITE);
    if (xbar) {
        red_add_f64(xbar + k, sx * g[0]);
        red_add_f64(xbar + (size_t)n + k, sx * g[1]);
        red_add_f64(xbar + 2 * (size_t)n + k, sx * g[2]);
    }
    if (mbar) red_add_f64(mbar + k, sm * g[3]);
}

constexpr int kVjpSymMin = 2048;    // sets below this many particles take the one-sided form

cudaError_t launch_vjp_pair(int kind, int n, const void* rec, const void* vec, const void* acc,
                            double eps2, double sx, double sm, double* xbar, double* mbar,
                            int* err, int sm_count, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (n >= kVjpSymMin) {
        const long long nb = (n + kVjpThreads - 1) / kVjpThreads;
        // about 8 items per resident CTA (~4 per SM), at most 32 tiles each
        const long long visits = nb * nb / 2 + 1;
        const int chunk = (int)std::max(1LL, std::min(32LL, visits / (32LL * sm_count)));
        const int nchunk = (int)((nb - 1 + chunk - 1) / chunk);
        const long long grid = nb * (1 + nchunk);
        if (grid > 2147483647LL) return cudaErrorInvalidValue;
        const D4* r = reinterpret_cast<const D4*>(rec);
        const D4* v = reinterpret_cast<const D4*>(vec);
        const D4* a = reinterpret_cast<const D4*>(acc);
        if (kind == 0) { vjp_sym_kernel<0><<<(unsigned)grid, kVjpThreads, 0, s>>>(n, r, v, a, eps2, chunk, nchunk, sx, sm, xbar, mbar, err); note_launch(); }
        else { vjp_sym_kernel<1><<<(unsigned)grid, kVjpThreads, 0, s>>>(n, r, v, a, eps2, chunk, nchunk, sx, sm, xbar, mbar, err); note_launch(); }
        return cudaGetLastError();
    }
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
