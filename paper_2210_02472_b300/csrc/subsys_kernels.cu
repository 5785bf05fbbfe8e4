// subsys_kernels.cu -- FSI with binary subsystems (Sect. 2.3, Algorithm 1), kernel side.
//
// The splitting H = T' + U' + sum_s H_S^s keeps the FSI cycle but (i) every acceleration
// and gradient sum ignores the pairs inside one subsystem, (ii) the drifts move only the
// single particles and (iii) each subsystem is advanced by its own Hamiltonian H_S for
// eps/2 twice per cycle.  The subsystems handled here are isolated bound binaries, whose
// H_S flow is the exact two-body motion.
//
// The masked pair passes reuse the id-checked loop of the one-sided pair kernel: every
// particle of the set gets a key -- its global id if single, N + s for both members of
// binary s -- and a source whose key equals the receiver's contributes nothing (the
// receiver itself and its partner).
#include "fsi_internal.cuh"

namespace fsi {

namespace {
constexpr int kSubB = 256;
inline int sub_blocks(long long n) { return (int)((n + kSubB - 1) / kSubB); }
}  // namespace

// where[global id] = position in the set; key[k] = global id (single by default).
__global__ void sub_where_kernel(int n, const int* __restrict__ idx, int* __restrict__ where,
                                 int* __restrict__ key) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int g = idx ? idx[k] : k;
    where[g] = k;
    key[k] = g;
}

// Binary s = (pairs[2s], pairs[2s+1]), global ids: both must be distinct members of the
// set and in no other binary; their keys become N + s and their set positions go to
// ppos[2s], ppos[2s+1].  A violation latches FSI_ERR_ARG.
__global__ void sub_pair_keys_kernel(int n_pairs, const int* __restrict__ pairs, int N,
                                     const int* __restrict__ where, int* __restrict__ key,
                                     int* __restrict__ ppos, int* err) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pairs) return;
    const int g0 = pairs[2 * s], g1 = pairs[2 * s + 1];
    int k0 = -1, k1 = -1;
    if (g0 >= 0 && g0 < N && g1 >= 0 && g1 < N && g0 != g1) {
        k0 = where[g0];
        k1 = where[g1];
    }
    bool ok = k0 >= 0 && k1 >= 0;
    if (ok) ok = atomicCAS(key + k0, g0, N + s) == g0;
    if (ok) ok = atomicCAS(key + k1, g1, N + s) == g1;
    if (!ok) set_error(err, FSI_ERR_ARG);
    ppos[2 * s] = ok ? k0 : -1;
    ppos[2 * s + 1] = ok ? k1 : -1;
}

// Exact two-body motion of binary s over time t (compact 3 x n arrays, FP64).  The relative
// orbit advances by the eccentric-anomaly change x that solves Kepler's equation in
// difference form,  n t = x - C sin x + S (1 - cos x),  C = e cos E0 = 1 - r0/a,
// S = e sin E0 = (r0 . v0) / (mu a)^{1/2}  (Newton steps kept inside the bracket
// [n t - 2e, n t + 2e] by bisection); positions and velocities follow from Lagrange's
// f and g.  An unbound pair latches FSI_ERR_UNSUPPORTED and is left unchanged.
__global__ void kepler_pairs_kernel(int n_pairs, const int* __restrict__ ppos, int n,
                                    double* __restrict__ x, double* __restrict__ v,
                                    const double* __restrict__ m, double t, int* err) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pairs) return;
    const int i = ppos[2 * s], j = ppos[2 * s + 1];
    if (i < 0 || j < 0) return;
    const double mi = m[i], mj = m[j], mu = mi + mj;
    double R[3], V[3], r0[3], u0[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const size_t oi = (size_t)q * n + i, oj = (size_t)q * n + j;
        R[q] = (mi * x[oi] + mj * x[oj]) / mu;
        V[q] = (mi * v[oi] + mj * v[oj]) / mu;
        r0[q] = x[oj] - x[oi];
        u0[q] = v[oj] - v[oi];
    }
    const double r0n = sqrt(r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]);
    const double u2 = u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2];
    const double ru = r0[0] * u0[0] + r0[1] * u0[1] + r0[2] * u0[2];
    const double ia = 2.0 / r0n - u2 / mu;            // 1 / semi-major axis
    if (!(ia > 0.0)) { set_error(err, FSI_ERR_UNSUPPORTED); return; }
    const double a = 1.0 / ia;
    const double sq = sqrt(mu * a);
    const double nm = sq * ia * ia;                   // mean motion (mu / a^3)^{1/2}
    const double C = 1.0 - r0n * ia, S = ru / sq;
    const double e = sqrt(C * C + S * S);
    const double M = nm * t;
    double lo = M - 2.0 * e - 1e-300, hi = M + 2.0 * e + 1e-300;
    double xe = M;
    for (int it = 0; it < 100; ++it) {
        double sx, cx;
        sincos(xe, &sx, &cx);
        const double F = xe - C * sx + S * (1.0 - cx) - M;
        if (F > 0.0) hi = fmin(hi, xe);
        else lo = fmax(lo, xe);
        double xn = xe - F / (1.0 - C * cx + S * sx);
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        const double d = fabs(xn - xe);
        xe = xn;
        if (d <= 4e-16 * fmax(1.0, fabs(xe)) || hi - lo <= 4e-16 * fmax(1.0, fabs(xe))) break;
    }
    double sx, cx;
    sincos(xe, &sx, &cx);
    const double hv = sin(0.5 * xe);
    const double omc = 2.0 * hv * hv;                 // 1 - cos x without cancellation
    const double f = 1.0 - a / r0n * omc;
    const double g = t - (xe - sx) / nm;
    double r1[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) r1[q] = f * r0[q] + g * u0[q];
    const double r1n = sqrt(r1[0] * r1[0] + r1[1] * r1[1] + r1[2] * r1[2]);
    const double fd = -sq * sx / (r0n * r1n);
    const double gd = 1.0 - a / r1n * omc;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double u1 = fd * r0[q] + gd * u0[q];
        const double Rq = R[q] + V[q] * t;
        const size_t oi = (size_t)q * n + i, oj = (size_t)q * n + j;
        x[oi] = Rq - (mj / mu) * r1[q];
        x[oj] = Rq + (mi / mu) * r1[q];
        v[oi] = V[q] - (mj / mu) * u1;
        v[oj] = V[q] + (mi / mu) * u1;
    }
}

// x += w v for the single particles of the set (key < N).
__global__ void drift_singles_kernel(int n, double* __restrict__ x, const double* __restrict__ v,
                                     const int* __restrict__ key, int N, double w) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || key[k] >= N) return;
#pragma unroll
    for (int q = 0; q < 3; ++q) x[(size_t)q * n + k] = fma(w, v[(size_t)q * n + k], x[(size_t)q * n + k]);
}

cudaError_t launch_sub_keys(int n, const int* idx, int N, const int* pairs, int n_pairs,
                            int* where, int* key, int* ppos, int* err, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(where, 0xff, (size_t)N * sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (n > 0) { sub_where_kernel<<<sub_blocks(n), kSubB, 0, s>>>(n, idx, where, key); note_launch(); }
    if (n_pairs > 0) {
        sub_pair_keys_kernel<<<sub_blocks(n_pairs), kSubB, 0, s>>>(n_pairs, pairs, N, where, key, ppos, err);
        note_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_kepler_pairs(int n_pairs, const int* ppos, int n, double* x, double* v,
                                const double* m, double t, int* err, cudaStream_t s) {
    if (n_pairs <= 0) return cudaSuccess;
    { kepler_pairs_kernel<<<sub_blocks(n_pairs), kSubB, 0, s>>>(n_pairs, ppos, n, x, v, m, t, err); note_launch(); }
    return cudaGetLastError();
}

cudaError_t launch_drift_singles(int n, double* x, const double* v, const int* key, int N, double w,
                                 cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    { drift_singles_kernel<<<sub_blocks(n), kSubB, 0, s>>>(n, x, v, key, N, w); note_launch(); }
    return cudaGetLastError();
}

}  // namespace fsi
