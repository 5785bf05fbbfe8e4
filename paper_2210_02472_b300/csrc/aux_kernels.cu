// aux_kernels.cu -- O(n) and small O(n^2) kernels around the pair passes:
// record packing (gather), scatter, kick/drift, PN1.0 pair kicks, time steps, energy,
// set checks.
#include <algorithm>

#include "fsi_internal.cuh"
#include "pair_math.cuh"

namespace fsi {

constexpr int kB = 256;

static inline int blocks_for(long long n, int b = kB) {
    long long g = (n + b - 1) / b;
    return (int)(g < 1 ? 1 : (g > 2147483647LL ? 2147483647LL : g));
}

__device__ __forceinline__ int idx_at(const int* idx, int k) { return idx ? idx[k] : k; }

// ---------------------------------------------------------------------------------
// Packing: global SoA (3 x N) -> compact records of the listed set; optionally also a
// compact FP64 copy xc (3 x n).
template <int P>
__global__ void pack_kernel(int N, const double* __restrict__ pos, const double* __restrict__ mass,
                            const int* __restrict__ idx, int n, void* __restrict__ rec,
                            double* __restrict__ xc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = idx_at(idx, k);
    const double x = pos[i], y = pos[(size_t)N + i], z = pos[2 * (size_t)N + i];
    const double m = mass[i];
    if constexpr (P == FSI_MIXED) {
        reinterpret_cast<RecMix*>(rec)[k] = make_mix_rec(x, y, z, m);
    } else {
        reinterpret_cast<D4*>(rec)[k] = make_d4(x, y, z, m);
    }
    if (xc) {
        xc[k] = x;
        xc[(size_t)n + k] = y;
        xc[2 * (size_t)n + k] = z;
    }
}

cudaError_t launch_pack(int precision, int N, const double* pos, const double* mass,
                        const int* idx, int n, void* rec, double* xc, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (precision == FSI_MIXED)
        { pack_kernel<FSI_MIXED><<<blocks_for(n), kB, 0, s>>>(N, pos, mass, idx, n, rec, xc); note_launch(); }
    else
        { pack_kernel<FSI_FP64><<<blocks_for(n), kB, 0, s>>>(N, pos, mass, idx, n, rec, xc); note_launch(); }
    return cudaGetLastError();
}

// Two packings in one launch (the slow and fast sets of a cross-level kick): CTAs
// [0, ctas_a) pack list A into rec_a, the others list B into rec_b.
template <int P>
__global__ void pack2_kernel(int N, const double* __restrict__ pos, const double* __restrict__ mass,
                             const int* __restrict__ ida, int na, void* __restrict__ rec_a,
                             const int* __restrict__ idb, int nb, void* __restrict__ rec_b,
                             int ctas_a) {
    const bool first = (int)blockIdx.x < ctas_a;
    const int k = (first ? blockIdx.x : blockIdx.x - ctas_a) * blockDim.x + threadIdx.x;
    const int n = first ? na : nb;
    if (k >= n) return;
    const int i = idx_at(first ? ida : idb, k);
    void* rec = first ? rec_a : rec_b;
    const double x = pos[i], y = pos[(size_t)N + i], z = pos[2 * (size_t)N + i];
    if constexpr (P == FSI_MIXED)
        reinterpret_cast<RecMix*>(rec)[k] = make_mix_rec(x, y, z, mass[i]);
    else
        reinterpret_cast<D4*>(rec)[k] = make_d4(x, y, z, mass[i]);
}

cudaError_t launch_pack2(int precision, int N, const double* pos, const double* mass,
                         const int* ida, int na, void* rec_a, const int* idb, int nb, void* rec_b,
                         cudaStream_t s) {
    if (na <= 0 || nb <= 0) {
        cudaError_t e = launch_pack(precision, N, pos, mass, ida, na, rec_a, nullptr, s);
        return e != cudaSuccess ? e : launch_pack(precision, N, pos, mass, idb, nb, rec_b, nullptr, s);
    }
    const int ca = (na + kB - 1) / kB, cb = (nb + kB - 1) / kB;
    if (precision == FSI_MIXED)
        { pack2_kernel<FSI_MIXED><<<ca + cb, kB, 0, s>>>(N, pos, mass, ida, na, rec_a, idb, nb, rec_b, ca); note_launch(); }
    else
        { pack2_kernel<FSI_FP64><<<ca + cb, kB, 0, s>>>(N, pos, mass, ida, na, rec_a, idb, nb, rec_b, ca); note_launch(); }
    return cudaGetLastError();
}

template <int P>
__global__ void pack_acc_kernel(int N, const double* __restrict__ accg,
                                const double* __restrict__ mass, const int* __restrict__ idx,
                                int n, void* __restrict__ accrec, double* __restrict__ ac) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = idx_at(idx, k);
    const double x = accg[i], y = accg[(size_t)N + i], z = accg[2 * (size_t)N + i];
    if constexpr (P == FSI_MIXED)
        reinterpret_cast<float4*>(accrec)[k] = make_float4((float)x, (float)y, (float)z, (float)mass[i]);
    else
        reinterpret_cast<D4*>(accrec)[k] = make_d4(x, y, z, mass[i]);
    if (ac) {
        ac[k] = x;
        ac[(size_t)n + k] = y;
        ac[2 * (size_t)n + k] = z;
    }
}

cudaError_t launch_pack_acc(int precision, int N, const double* accg, const double* mass,
                            const int* idx, int n, void* accrec, double* ac, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (precision == FSI_MIXED)
        { pack_acc_kernel<FSI_MIXED><<<blocks_for(n), kB, 0, s>>>(N, accg, mass, idx, n, accrec, ac); note_launch(); }
    else
        { pack_acc_kernel<FSI_FP64><<<blocks_for(n), kB, 0, s>>>(N, accg, mass, idx, n, accrec, ac); note_launch(); }
    return cudaGetLastError();
}

__global__ void gather3_kernel(int N, const double* __restrict__ src, const int* __restrict__ idx,
                               int n, double* __restrict__ dst) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = idx_at(idx, k);
    dst[k] = src[i];
    dst[(size_t)n + k] = src[(size_t)N + i];
    dst[2 * (size_t)n + k] = src[2 * (size_t)N + i];
}

cudaError_t launch_gather3(int N, const double* src, const int* idx, int n, double* dst,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    { gather3_kernel<<<blocks_for(n), kB, 0, s>>>(N, src, idx, n, dst); note_launch(); }
    return cudaGetLastError();
}

__global__ void scatter3_kernel(int N, const double* __restrict__ src, const int* __restrict__ idx,
                                int n, double* __restrict__ dst) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = idx_at(idx, k);
    dst[i] = src[k];
    dst[(size_t)N + i] = src[(size_t)n + k];
    dst[2 * (size_t)N + i] = src[2 * (size_t)n + k];
}

cudaError_t launch_scatter3(int N, const double* src, const int* idx, int n, double* dst,
                            cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    { scatter3_kernel<<<blocks_for(n), kB, 0, s>>>(N, src, idx, n, dst); note_launch(); }
    return cudaGetLastError();
}

// v[idx[k]] += w * a[:, k]   (scatter-add of a compact 3 x n array into a global 3 x N one)
__global__ void scatter_axpy3_kernel(int N, const double* __restrict__ a, const int* __restrict__ idx,
                                     int n, double w, double* __restrict__ v) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = idx_at(idx, k);
    v[i] = fma(w, a[k], v[i]);
    v[(size_t)N + i] = fma(w, a[(size_t)n + k], v[(size_t)N + i]);
    v[2 * (size_t)N + i] = fma(w, a[2 * (size_t)n + k], v[2 * (size_t)N + i]);
}

cudaError_t launch_scatter_axpy3(int N, const double* a, const int* idx, int n, double w,
                                 double* v, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    { scatter_axpy3_kernel<<<blocks_for(n), kB, 0, s>>>(N, a, idx, n, w, v); note_launch(); }
    return cudaGetLastError();
}

__global__ void gather1_kernel(int N, const double* __restrict__ src, const int* __restrict__ idx,
                               int n, double* __restrict__ dst) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    dst[k] = src[idx_at(idx, k)];
}

cudaError_t launch_gather1(int N, const double* src, const int* idx, int n, double* dst,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    { gather1_kernel<<<blocks_for(n), kB, 0, s>>>(N, src, idx, n, dst); note_launch(); }
    return cudaGetLastError();
}

__global__ void gather_u8_kernel(const unsigned char* __restrict__ src, const int* __restrict__ idx,
                                 int n, unsigned char* __restrict__ dst) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    dst[k] = src[idx_at(idx, k)];
}

cudaError_t launch_gather_u8(const unsigned char* src, const int* idx, int n,
                             unsigned char* dst, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    { gather_u8_kernel<<<blocks_for(n), kB, 0, s>>>(src, idx, n, dst); note_launch(); }
    return cudaGetLastError();
}

// ids[k] = idx[k] (or k) for k < n; -1 up to cap (the padding the bulk copies may read).
__global__ void ids_kernel(const int* __restrict__ idx, int n, int cap, int* __restrict__ ids) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cap) return;
    ids[k] = k < n ? idx_at(idx, k) : -1;
}

cudaError_t launch_ids(const int* idx, int n, int cap, int* ids, cudaStream_t s) {
    if (cap <= 0) return cudaSuccess;
    { ids_kernel<<<blocks_for(cap), kB, 0, s>>>(idx, n, cap, ids); note_launch(); }
    return cudaGetLastError();
}

// accg[:, idx[k]] = ac[:, k]
cudaError_t launch_scatter_acc_global(int n, const double* ac, const int* idx, int N,
                                      double* accg, cudaStream_t s) {
    return launch_scatter3(N, ac, idx, n, accg, s);
}

// ---------------------------------------------------------------------------------
// Disjointness of two id lists: mark B, test A, unmark B.  mark: N zeroed bytes.
__global__ void mark_kernel(const int* __restrict__ B, int nB, unsigned char* mark, unsigned char v) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nB) mark[idx_at(B, k)] = v;
}

__global__ void test_kernel(const int* __restrict__ A, int nA, const unsigned char* mark, int* err) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nA && mark[idx_at(A, k)]) set_error(err, FSI_ERR_ARG);
}

cudaError_t launch_check_disjoint(int N, const int* A, int nA, const int* B, int nB,
                                  unsigned char* mark, int* err, cudaStream_t s) {
    (void)N;
    if (nA <= 0 || nB <= 0) return cudaSuccess;
    { mark_kernel<<<blocks_for(nB), kB, 0, s>>>(B, nB, mark, 1); note_launch(); }
    { test_kernel<<<blocks_for(nA), kB, 0, s>>>(A, nA, mark, err); note_launch(); }
    { mark_kernel<<<blocks_for(nB), kB, 0, s>>>(B, nB, mark, 0); note_launch(); }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Kick + drift on a compact set, rewriting its position records:
//   v += c_kick a;  x += c_drift v;  rec_out <- (x, m from the FP64 masses mc).
template <int P>
__global__ void kick_drift_kernel(int n, double* __restrict__ xc, double* __restrict__ vc,
                                  const double* __restrict__ ac, double c_kick, double c_drift,
                                  const double* __restrict__ mc, void* __restrict__ rec_out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double v[3], x[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        v[c] = vc[(size_t)c * n + k];
        if (ac) v[c] = fma(c_kick, ac[(size_t)c * n + k], v[c]);
        vc[(size_t)c * n + k] = v[c];
        x[c] = xc[(size_t)c * n + k];
        if (c_drift != 0.0) {
            x[c] = fma(c_drift, v[c], x[c]);
            xc[(size_t)c * n + k] = x[c];
        }
    }
    if (rec_out) {
        if constexpr (P == FSI_MIXED)
            reinterpret_cast<RecMix*>(rec_out)[k] = make_mix_rec(x[0], x[1], x[2], mc[k]);
        else
            reinterpret_cast<D4*>(rec_out)[k] = make_d4(x[0], x[1], x[2], mc[k]);
    }
}

cudaError_t launch_kick_drift(int precision, int n, double* xc, double* vc, const double* ac,
                              double c_kick, double c_drift, const double* mc, void* rec_out,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (precision == FSI_MIXED)
        { kick_drift_kernel<FSI_MIXED><<<blocks_for(n), kB, 0, s>>>(n, xc, vc, ac, c_kick, c_drift, mc, rec_out); note_launch(); }
    else
        { kick_drift_kernel<FSI_FP64><<<blocks_for(n), kB, 0, s>>>(n, xc, vc, ac, c_kick, c_drift, mc, rec_out); note_launch(); }
    return cudaGetLastError();
}

// Kick then drift of a listed set in the global SoA state (grid-stride):
//   v[:, i] += c_kick a[:, k];  x[:, i] += c_drift v[:, i];  i = idx[k] (idx null: i = k).
__global__ void kick_drift_ids_kernel(long long N, double* __restrict__ pos,
                                      double* __restrict__ vel, const double* __restrict__ acc,
                                      const int* __restrict__ idx, int n, double c_kick,
                                      double c_drift) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const long long i = idx ? (long long)idx[k] : k;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double v = vel[c * N + i];
            if (acc) v = fma(c_kick, acc[c * (long long)n + k], v);
            vel[c * N + i] = v;
            pos[c * N + i] = fma(c_drift, v, pos[c * N + i]);
        }
    }
}

cudaError_t launch_kick_drift_ids(long long N, double* pos, double* vel, const double* acc,
                                  const int* idx, int n, double c_kick, double c_drift,
                                  int sm_count, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    // 8 CTAs of 256 per SM (full occupancy at <= 32 registers), at most one per 256 ids
    const long long want = (long long)sm_count * 8;
    const int grid = (int)std::min<long long>(want, (n + kB - 1) / kB);
    { kick_drift_ids_kernel<<<grid, kB, 0, s>>>(N, pos, vel, acc, idx, n, c_kick, c_drift); note_launch(); }
    return cudaGetLastError();
}

__global__ void axpy3_kernel(int n, double* __restrict__ v, const double* __restrict__ a, double w) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) v[(size_t)c * n + k] = fma(w, a[(size_t)c * n + k], v[(size_t)c * n + k]);
}

cudaError_t launch_axpy3(int n, double* v, const double* a, double w, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    { axpy3_kernel<<<blocks_for(n), kB, 0, s>>>(n, v, a, w); note_launch(); }
    return cudaGetLastError();
}

// Ordered list of the black holes of a compact set (single CTA, warp-ballot scan).
constexpr int kMaxBH = kMaxBHList;

__global__ void bh_list_kernel(int n, const unsigned char* __restrict__ bhc, int* __restrict__ list,
                               int* __restrict__ count, int* err) {
    __shared__ int warp_tot[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k0 = 0; k0 < n; k0 += blockDim.x) {
        const int k = k0 + threadIdx.x;
        const bool f = k < n && bhc[k];
        const unsigned b = __ballot_sync(0xffffffffu, f);
        if (lane == 0) warp_tot[wid] = __popc(b);
        __syncthreads();
        int off = base;
        for (int w = 0; w < wid; ++w) off += warp_tot[w];
        off += __popc(b & ((1u << lane) - 1u));
        if (f) {
            if (off < kMaxBH) list[off] = k;
            else set_error(err, FSI_ERR_UNSUPPORTED);
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int w = 0; w < nw; ++w) base += warp_tot[w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = min(base, kMaxBH);
}

cudaError_t launch_bh_list(int n, const unsigned char* bhc, int* bh_list, int* n_bh, int* err,
                           cudaStream_t s) {
    { bh_list_kernel<<<1, 1024, 0, s>>>(n, bhc, bh_list, n_bh, err); note_launch(); }
    return cudaGetLastError();
}

// (a) every particle i of the compact set <- every black hole j != i
__global__ void pn_from_bh_kernel(int n, const double* __restrict__ xc, const double* __restrict__ vc,
                                  const double* __restrict__ mc, const int* __restrict__ list,
                                  const int* __restrict__ count, double ic2, double* __restrict__ apn,
                                  int* err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nb = *count;
    const double xi = xc[i], yi = xc[(size_t)n + i], zi = xc[2 * (size_t)n + i];
    const double vxi = vc[i], vyi = vc[(size_t)n + i], vzi = vc[2 * (size_t)n + i];
    double ax = 0, ay = 0, az = 0;
    for (int b = 0; b < nb; ++b) {
        const int j = list[b];
        if (j == i) continue;
        pn_pair(xi, yi, zi, vxi, vyi, vzi, mc[i], xc[j], xc[(size_t)n + j], xc[2 * (size_t)n + j],
                vc[j], vc[(size_t)n + j], vc[2 * (size_t)n + j], mc[j], ic2, ax, ay, az, err);
    }
    apn[i] = ax;
    apn[(size_t)n + i] = ay;
    apn[2 * (size_t)n + i] = az;
}

// (b) black hole b <- every non-black-hole j: per-CTA partial sums, in a fixed order.
constexpr int kPnCtas = kPnPartCtas;

__global__ void pn_bh_from_all_kernel(int n, const double* __restrict__ xc, const double* __restrict__ vc,
                                      const double* __restrict__ mc, const unsigned char* __restrict__ bhc,
                                      const int* __restrict__ list, const int* __restrict__ count,
                                      double ic2, double* __restrict__ part, int* err) {
    for (int b = blockIdx.y; b < *count; b += gridDim.y) {
    const int i = list[b];
    const double xi = xc[i], yi = xc[(size_t)n + i], zi = xc[2 * (size_t)n + i];
    const double vxi = vc[i], vyi = vc[(size_t)n + i], vzi = vc[2 * (size_t)n + i];
    const double mi = mc[i];
    double s[3] = {0, 0, 0};
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        if (bhc[j]) continue;
        pn_pair(xi, yi, zi, vxi, vyi, vzi, mi, xc[j], xc[(size_t)n + j], xc[2 * (size_t)n + j],
                vc[j], vc[(size_t)n + j], vc[2 * (size_t)n + j], mc[j], ic2, s[0], s[1], s[2], err);
    }
    __shared__ double red[3][kB];
#pragma unroll
    for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = s[c];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < 3; ++c) part[((size_t)b * 3 + c) * kPnCtas + blockIdx.x] = red[c][0];
    __syncthreads();
    }
}

__global__ void pn_bh_finish_kernel(int n, const int* __restrict__ list, const int* __restrict__ count,
                                    const double* __restrict__ part, double* __restrict__ apn) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= *count) return;
    const int i = list[b];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double s = 0;
        for (int q = 0; q < kPnCtas; ++q) s += part[((size_t)b * 3 + c) * kPnCtas + q];
        apn[(size_t)c * n + i] += s;
    }
}

// PN1.0 accelerations of the compact set on itself (pairs with a black hole), apn: 3 x n.
cudaError_t launch_pn(int n, const double* xc, const double* vc, const double* mc,
                      const unsigned char* bhc, double c, const int* bh_list, const int* n_bh,
                      int max_bh, double* apn, double* part, int* err, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const double ic2 = 1.0 / (c * c);
    { pn_from_bh_kernel<<<blocks_for(n), kB, 0, s>>>(n, xc, vc, mc, bh_list, n_bh, ic2, apn, err); note_launch(); }
    dim3 g(kPnCtas, max_bh < 32 ? max_bh : 32);
    { pn_bh_from_all_kernel<<<g, kB, 0, s>>>(n, xc, vc, mc, bhc, bh_list, n_bh, ic2, part, err); note_launch(); }
    { pn_bh_finish_kernel<<<blocks_for(max_bh), kB, 0, s>>>(n, bh_list, n_bh, part, apn); note_launch(); }
    return cudaGetLastError();
}

// General (masked) PN pair sum over index lists: thread per i in A, loop over B.
__global__ void pn_pairs_kernel(int N, const double* __restrict__ pos, const double* __restrict__ vel,
                                const double* __restrict__ mass, const unsigned char* __restrict__ is_bh,
                                double ic2, const int* __restrict__ A, int nA,
                                const int* __restrict__ B, int nB, double* __restrict__ out,
                                double wscale, int accumulate, int* err) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nA) return;
    const int i = idx_at(A, k);
    const double xi = pos[i], yi = pos[(size_t)N + i], zi = pos[2 * (size_t)N + i];
    const double vxi = vel[i], vyi = vel[(size_t)N + i], vzi = vel[2 * (size_t)N + i];
    const bool bi = is_bh[i] != 0;
    double ax = 0, ay = 0, az = 0;
    for (int l = 0; l < nB; ++l) {
        const int j = idx_at(B, l);
        if (j == i || (!bi && !is_bh[j])) continue;
        pn_pair(xi, yi, zi, vxi, vyi, vzi, mass[i], pos[j], pos[(size_t)N + j], pos[2 * (size_t)N + j],
                vel[j], vel[(size_t)N + j], vel[2 * (size_t)N + j], mass[j], ic2, ax, ay, az, err);
    }
    if (accumulate) {
        out[k] += wscale * ax;
        out[(size_t)nA + k] += wscale * ay;
        out[2 * (size_t)nA + k] += wscale * az;
    } else {
        out[k] = wscale * ax;
        out[(size_t)nA + k] = wscale * ay;
        out[2 * (size_t)nA + k] = wscale * az;
    }
}

cudaError_t launch_pn_pairs(int N, const double* pos, const double* vel, const double* mass,
                            const unsigned char* is_bh, double c, const int* A, int nA,
                            const int* B, int nB, double* out, int* err, cudaStream_t s) {
    if (nA <= 0) return cudaSuccess;
    { pn_pairs_kernel<<<blocks_for(nA), kB, 0, s>>>(N, pos, vel, mass, is_bh, 1.0 / (c * c), A, nA,
                                                  B, nB, out, 1.0, 0, err); note_launch(); }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// PN1.0 kicks between two disjoint sets of global ids (the slow-fast pairs of an HHS
// level), through the black-hole sublists: for i in A, the terms of the black holes j of
// B (pn_list_from_bh) plus, for a black hole i of A, the terms of every non-black-hole j
// of B (pn_list_bh_from_all + finish).

// Positions k of list L whose particle is a black hole, in list order (single CTA).
__global__ void bh_sublist_kernel(int n, const int* __restrict__ L, const unsigned char* __restrict__ is_bh,
                                  int* __restrict__ out, int* __restrict__ count, int* err) {
    __shared__ int warp_tot[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k0 = 0; k0 < n; k0 += blockDim.x) {
        const int k = k0 + threadIdx.x;
        const bool f = k < n && is_bh[L[k]];
        const unsigned b = __ballot_sync(0xffffffffu, f);
        if (lane == 0) warp_tot[wid] = __popc(b);
        __syncthreads();
        int off = base;
        for (int w = 0; w < wid; ++w) off += warp_tot[w];
        off += __popc(b & ((1u << lane) - 1u));
        if (f) {
            if (off < kMaxBH) out[off] = k;
            else set_error(err, FSI_ERR_UNSUPPORTED);
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int w = 0; w < nw; ++w) base += warp_tot[w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = min(base, kMaxBH);
}

__global__ void pn_list_from_bh_kernel(long long N, const double* __restrict__ pos, const double* __restrict__ vel,
                                       const double* __restrict__ mass, const int* __restrict__ A, int nA,
                                       const int* __restrict__ B, const int* __restrict__ Bbh,
                                       const int* __restrict__ nBbh, double ic2, double* __restrict__ out,
                                       int* err) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nA) return;
    const int i = A[k];
    const double xi = pos[i], yi = pos[N + i], zi = pos[2 * N + i];
    const double ui = vel[i], vi = vel[N + i], wi = vel[2 * N + i];
    double ax = 0, ay = 0, az = 0;
    const int nb = *nBbh;
    for (int q = 0; q < nb; ++q) {
        const int j = B[Bbh[q]];
        if (j == i) continue;
        pn_pair(xi, yi, zi, ui, vi, wi, mass[i], pos[j], pos[N + j], pos[2 * N + j], vel[j], vel[N + j],
                vel[2 * N + j], mass[j], ic2, ax, ay, az, err);
    }
    out[k] = ax;
    out[(size_t)nA + k] = ay;
    out[2 * (size_t)nA + k] = az;
}

__global__ void pn_list_bh_from_all_kernel(long long N, const double* __restrict__ pos, const double* __restrict__ vel,
                                           const double* __restrict__ mass, const unsigned char* __restrict__ is_bh,
                                           const int* __restrict__ A, const int* __restrict__ Abh,
                                           const int* __restrict__ nAbh, const int* __restrict__ B, int nB,
                                           double ic2, double* __restrict__ part, int* err) {
    __shared__ double red[3][kB];
    for (int b = blockIdx.y; b < *nAbh; b += gridDim.y) {
        const int i = A[Abh[b]];
        const double xi = pos[i], yi = pos[N + i], zi = pos[2 * N + i];
        const double ui = vel[i], vi = vel[N + i], wi = vel[2 * N + i];
        double sx = 0, sy = 0, sz = 0;
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nB; q += gridDim.x * blockDim.x) {
            const int j = B[q];
            if (is_bh[j]) continue;
            pn_pair(xi, yi, zi, ui, vi, wi, mass[i], pos[j], pos[N + j], pos[2 * N + j], vel[j],
                    vel[N + j], vel[2 * N + j], mass[j], ic2, sx, sy, sz, err);
        }
        red[0][threadIdx.x] = sx; red[1][threadIdx.x] = sy; red[2][threadIdx.x] = sz;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w)
                for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0)
            for (int c = 0; c < 3; ++c) part[((size_t)b * 3 + c) * kPnCtas + blockIdx.x] = red[c][0];
        __syncthreads();
    }
}

__global__ void pn_list_bh_finish_kernel(const int* __restrict__ Abh, const int* __restrict__ nAbh, int nA,
                                         const double* __restrict__ part, double* __restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= *nAbh) return;
    const int k = Abh[b];
    for (int c = 0; c < 3; ++c) {
        double s = 0;
        for (int q = 0; q < kPnCtas; ++q) s += part[((size_t)b * 3 + c) * kPnCtas + q];
        out[(size_t)c * nA + k] += s;
    }
}

cudaError_t launch_pn_cross(long long N, const double* pos, const double* vel, const double* mass,
                            const unsigned char* is_bh, double c, const int* A, int nA, const int* B,
                            int nB, int* Abh, int* nAbh, int* Bbh, int* nBbh, double* outA,
                            double* outB, double* part, int* err, cudaStream_t s) {
    if (nA <= 0 || nB <= 0) return cudaSuccess;
    const double ic2 = 1.0 / (c * c);
    { bh_sublist_kernel<<<1, 1024, 0, s>>>(nA, A, is_bh, Abh, nAbh, err); note_launch(); }
    { bh_sublist_kernel<<<1, 1024, 0, s>>>(nB, B, is_bh, Bbh, nBbh, err); note_launch(); }
    { pn_list_from_bh_kernel<<<blocks_for(nA), kB, 0, s>>>(N, pos, vel, mass, A, nA, B, Bbh, nBbh, ic2, outA, err); note_launch(); }
    { pn_list_from_bh_kernel<<<blocks_for(nB), kB, 0, s>>>(N, pos, vel, mass, B, nB, A, Abh, nAbh, ic2, outB, err); note_launch(); }
    const dim3 g(kPnCtas, 32);
    { pn_list_bh_from_all_kernel<<<g, kB, 0, s>>>(N, pos, vel, mass, is_bh, A, Abh, nAbh, B, nB, ic2, part, err); note_launch(); }
    { pn_list_bh_finish_kernel<<<blocks_for(kMaxBH), kB, 0, s>>>(Abh, nAbh, nA, part, outA); note_launch(); }
    { pn_list_bh_from_all_kernel<<<g, kB, 0, s>>>(N, pos, vel, mass, is_bh, B, Bbh, nBbh, A, nA, ic2, part, err); note_launch(); }
    { pn_list_bh_finish_kernel<<<blocks_for(kMaxBH), kB, 0, s>>>(Bbh, nBbh, nB, part, outB); note_launch(); }
    return cudaGetLastError();
}

// PN1.0 accelerations of the id list A from the id list B (any overlap; self pairs skipped
// by id) through the black-hole sublists: for i in A the terms of B's black holes j != i,
// plus, for a black hole i of A, the terms of B's other particles.  out (3 x nA)
// overwritten.  A pair with a black hole is counted once per receiver: a black-hole pair
// by the first kernel, a black hole with a star by the first (receiver the star) or the
// second (receiver the black hole).
cudaError_t launch_pn_lists(long long N, const double* pos, const double* vel, const double* mass,
                            const unsigned char* is_bh, double c, const int* A, int nA, const int* B,
                            int nB, int* Abh, int* nAbh, int* Bbh, int* nBbh, double* out,
                            double* part, int* err, cudaStream_t s) {
    if (nA <= 0) return cudaSuccess;
    const double ic2 = 1.0 / (c * c);
    { bh_sublist_kernel<<<1, 1024, 0, s>>>(nA, A, is_bh, Abh, nAbh, err); note_launch(); }
    { bh_sublist_kernel<<<1, 1024, 0, s>>>(nB, B, is_bh, Bbh, nBbh, err); note_launch(); }
    { pn_list_from_bh_kernel<<<blocks_for(nA), kB, 0, s>>>(N, pos, vel, mass, A, nA, B, Bbh, nBbh, ic2, out, err); note_launch(); }
    if (nB > 0) {
        const dim3 g(kPnCtas, 32);
        { pn_list_bh_from_all_kernel<<<g, kB, 0, s>>>(N, pos, vel, mass, is_bh, A, Abh, nAbh, B, nB, ic2, part, err); note_launch(); }
        { pn_list_bh_finish_kernel<<<blocks_for(kMaxBH), kB, 0, s>>>(Abh, nAbh, nA, part, out); note_launch(); }
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Small O(n^2) FP64 loop (energy): thread per i, sources through shared memory in plain
// cooperative tiles.
constexpr int kAuxTile = 128;

// Gradient and velocity-per-acceleration time steps (Sect. 3.4, Eqs. dt-nabla1,
// dt-nabla2, vel-acc-crit) of a compact set from its velocities v, accelerations a and
// force-gradient sums G (3 x n each, G without the eps^2/24 factor):
//   g' = G / 24 (a~ = a + eps^2 g'),  eps = min(eta_va |v|/|a|, eta_grad (|v|/|g'|)^{1/3},
//   eta_grad (|a|/|g'|)^{1/2}), each only when its parameter is > 0 and its denominator
//   is non-zero; step[k] takes the min with it.
__global__ void grad_steps_kernel(int n, const double* __restrict__ v, const double* __restrict__ a,
                                  const double* __restrict__ G, double eta_grad, double eta_va,
                                  double* __restrict__ step) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double vn = 0.0, an = 0.0, gn = 0.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double vq = v[(size_t)q * n + k], aq = a[(size_t)q * n + k];
        const double gq = G[(size_t)q * n + k] * (1.0 / 24.0);
        vn = fma(vq, vq, vn);
        an = fma(aq, aq, an);
        gn = fma(gq, gq, gn);
    }
    vn = sqrt(vn);
    an = sqrt(an);
    gn = sqrt(gn);
    double e = step[k];
    if (eta_va > 0.0 && an > 0.0) e = fmin(e, eta_va * vn / an);
    if (eta_grad > 0.0 && gn > 0.0) {
        e = fmin(e, eta_grad * cbrt(vn / gn));
        e = fmin(e, eta_grad * sqrt(an / gn));
    }
    step[k] = e;
}

cudaError_t launch_grad_steps(int n, const double* vc, const double* a, const double* G,
                              double eta_grad, double eta_va, double* step, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    { grad_steps_kernel<<<blocks_for(n), kB, 0, s>>>(n, vc, a, G, eta_grad, eta_va, step); note_launch(); }
    return cudaGetLastError();
}

// FP32 velocity records (vx, vy, vz, m) of a set: entry k from particle idx[k] of the
// 3 x ld velocity rows (idx null: particle k); with pos, also its mixed position record.
__global__ void pack_vel_kernel(long long ld, const double* __restrict__ v,
                                const double* __restrict__ m, const int* __restrict__ idx, int n,
                                float4* __restrict__ out, const double* __restrict__ pos,
                                RecMix* __restrict__ rec) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long i = idx ? (long long)idx[k] : k;
    out[k] = make_float4((float)v[i], (float)v[ld + i], (float)v[2 * ld + i], (float)m[i]);
    if (pos) rec[k] = make_mix_rec(pos[i], pos[ld + i], pos[2 * ld + i], m[i]);
}

cudaError_t launch_pack_vel(int N, const double* vel, const double* mass, const int* idx, int n,
                            void* vrec, const double* pos, void* rec, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    { pack_vel_kernel<<<blocks_for(n), kB, 0, s>>>(N, vel, mass, idx, n, reinterpret_cast<float4*>(vrec),
                                                   pos, reinterpret_cast<RecMix*>(rec)); note_launch(); }
    return cudaGetLastError();
}

// Energy (Sect. 2.1, the Hamiltonian): per-CTA partial sums of the kinetic energy and of
// the potential -sum_{i<j} m_i m_j / sqrt(r^2 + eps2), every unordered pair once: thread i
// sums m_j / r over the sources j > i, from its block's own tile on, so the blocks of
// small i carry the most sources and, dispatched first, leave the short ones for the
// tail.  The partials are reduced in a fixed order by energy_finish_kernel.  A coincident
// unsoftened pair (r^2 = 0, tested on its bits) is skipped and reported.
__global__ void energy_kernel(int n, const double* __restrict__ xc, const double* __restrict__ vc,
                              const double* __restrict__ mc, double eps2, double* __restrict__ part,
                              int* err) {
    __shared__ double sx[kAuxTile], sy[kAuxTile], sz[kAuxTile], sm[kAuxTile];
    __shared__ double rk[kAuxTile], rw[kAuxTile];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int ii = min(i, n - 1);
    const double xi = xc[ii], yi = xc[(size_t)n + ii], zi = xc[2 * (size_t)n + ii];
    double w = 0.0;
    bool coincident = false;
    const int jstart = blockIdx.x * blockDim.x;
    for (int j0 = jstart; j0 < n; j0 += kAuxTile) {
        __syncthreads();
        for (int t = threadIdx.x; t < kAuxTile; t += blockDim.x) {
            const int j = j0 + t;
            if (j < n) { sx[t] = xc[j]; sy[t] = xc[(size_t)n + j]; sz[t] = xc[2 * (size_t)n + j]; sm[t] = mc[j]; }
        }
        __syncthreads();
        const int cnt = min(kAuxTile, n - j0);
        // the block's own tile: only j > i (a thread past the end, ii = n - 1, has none)
        const int t0 = j0 == jstart ? ii - j0 + 1 : 0;
#pragma unroll 4
        for (int t = t0; t < cnt; ++t) {
            const double dx = sx[t] - xi, dy = sy[t] - yi, dz = sz[t] - zi;
            const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
            if (__double_as_longlong(r2) == 0) { coincident = true; continue; }
            w = fma(sm[t], rsqrt_f64(r2), w);
        }
    }
    if (coincident && i < n) set_error(err, FSI_ERR_COINCIDENT);
    double kin = 0.0;
    if (i < n) {
        const double u = vc[i], v = vc[(size_t)n + i], ww = vc[2 * (size_t)n + i];
        kin = 0.5 * mc[i] * (u * u + v * v + ww * ww);
        w = -mc[i] * w;
    } else {
        w = 0.0;
    }
    rk[threadIdx.x] = kin;
    rw[threadIdx.x] = w;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            rk[threadIdx.x] += rk[threadIdx.x + h];
            rw[threadIdx.x] += rw[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = rk[0];
        part[2 * blockIdx.x + 1] = rw[0];
    }
}

__global__ void energy_finish_kernel(int nb, const double* __restrict__ part, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double k = 0, w = 0, ck = 0, cw = 0;   // Kahan-compensated sums over the CTA partials
    for (int b = 0; b < nb; ++b) {
        double y = part[2 * b] - ck, t = k + y;
        ck = (t - k) - y; k = t;
        y = part[2 * b + 1] - cw; t = w + y;
        cw = (t - w) - y; w = t;
    }
    out[0] = k;
    out[1] = w;
}

int energy_blocks(int n) { return blocks_for(n, kAuxTile); }

cudaError_t launch_energy(int n, const double* xc, const double* vc, const double* mc,
                          double eps2, double* part, double* out, int* err, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int nb = energy_blocks(n);
    { energy_kernel<<<nb, kAuxTile, 0, s>>>(n, xc, vc, mc, eps2, part, err); note_launch(); }
    { energy_finish_kernel<<<1, 32, 0, s>>>(nb, part, out); note_launch(); }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// HHS helpers.
// Stable partition of ids by (step >= tau) into S (slow) and F (fast), single CTA scan.
// counts[0] = |S|, counts[1] = |F|, counts[2] = 1 if some particle wanted a step < tau
// at the deepest level (force_slow).  With step0 the level-step rule is applied first:
// at level 0 the steps are recorded (step0[id] = step), deeper down a step is the min
// with the recorded one.
__global__ void partition_kernel(int n, const int* __restrict__ ids, double* __restrict__ step,
                                 double* __restrict__ step0, int level0, double tau, int force_slow,
                                 int* __restrict__ S, int* __restrict__ F,
                                 int* __restrict__ counts) {
    __shared__ int wS[32], wF[32];
    __shared__ int baseS, baseF, anyfast;
    if (threadIdx.x == 0) { baseS = 0; baseF = 0; anyfast = 0; }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k0 = 0; k0 < n; k0 += blockDim.x) {
        const int k = k0 + threadIdx.x;
        const bool valid = k < n;
        double st = valid ? step[k] : 0.0;
        if (valid && step0) {
            const int i = ids[k];
            if (level0) step0[i] = st;
            else { st = fmin(st, step0[i]); step[k] = st; }
        }
        const bool fastw = valid && st < tau;
        const bool slow = valid && (force_slow || !fastw);
        const bool fast = valid && !slow;
        if (fastw && force_slow) anyfast = 1;
        const unsigned bs = __ballot_sync(0xffffffffu, slow);
        const unsigned bf = __ballot_sync(0xffffffffu, fast);
        if (lane == 0) { wS[wid] = __popc(bs); wF[wid] = __popc(bf); }
        __syncthreads();
        int oS = baseS, oF = baseF;
        for (int w = 0; w < wid; ++w) { oS += wS[w]; oF += wF[w]; }
        const unsigned lm = (1u << lane) - 1u;
        if (slow) S[oS + __popc(bs & lm)] = ids[k];
        if (fast) F[oF + __popc(bf & lm)] = ids[k];
        __syncthreads();
        if (threadIdx.x == 0)
            for (int w = 0; w < nw; ++w) { baseS += wS[w]; baseF += wF[w]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { counts[0] = baseS; counts[1] = baseF; counts[2] = anyfast; }
}

cudaError_t launch_partition(int n, const int* ids, double* step, double* step0, int level0,
                             double tau, int force_slow, int* S, int* F, int* counts, cudaStream_t s) {
    { partition_kernel<<<1, 1024, 0, s>>>(n, ids, step, step0, level0, tau, force_slow, S, F, counts); note_launch(); }
    return cudaGetLastError();
}

__global__ void iota_kernel(int n, int* ids) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) ids[k] = k;
}

cudaError_t launch_iota(int n, int* ids, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    { iota_kernel<<<blocks_for(n), kB, 0, s>>>(n, ids); note_launch(); }
    return cudaGetLastError();
}

}  // namespace fsi
