// order_kernels.cu -- spatial ordering of a set (Morton order) and the far-tile inputs of
// the symmetric mixed kernel.
//
// The pair kernels are exact for any particle order; ordering only decides how many
// (warp, source sub-tile) pairs are far enough apart to take the cheaper separation
// arithmetic.  Steps:
//   1. bounding box of the set (two-stage min/max reduction, FP64);
//   2. 30-bit Morton keys: 10 bits per axis of the position scaled to the box;
//   3. stable LSD radix sort of (key, index) pairs, 4 passes of 8 bits (the last uses 6);
//   4. per position update: for every 32-record sub-tile of the packed records, its
//      centre C (FP32 midpoint of the box of the high parts), the records relative to C
//      rounded once to FP32, and the radius R = max |x_k - C| over the sub-tile.
#include <algorithm>

#include "fsi_internal.cuh"

namespace fsi {

namespace {
constexpr int kOB = 256;            // threads per block for the ordering kernels
constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;

int nblocks(long long n) { return (int)((n + kOB - 1) / kOB); }
}  // namespace

// ---- 1. bounding box ---------------------------------------------------------------
__global__ void bbox_partial_kernel(int n, const double* __restrict__ xc, long long ld,
                                    double* __restrict__ part) {
    __shared__ double lo[3][kOB], hi[3][kOB];
    double l[3] = {INFINITY, INFINITY, INFINITY}, h[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = blockIdx.x * kOB + threadIdx.x; k < n; k += gridDim.x * kOB)
        for (int c = 0; c < 3; ++c) {
            const double v = xc[(size_t)c * ld + k];
            l[c] = fmin(l[c], v);
            h[c] = fmax(h[c], v);
        }
    for (int c = 0; c < 3; ++c) { lo[c][threadIdx.x] = l[c]; hi[c][threadIdx.x] = h[c]; }
    __syncthreads();
    for (int w = kOB / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 3; ++c) {
                lo[c][threadIdx.x] = fmin(lo[c][threadIdx.x], lo[c][threadIdx.x + w]);
                hi[c][threadIdx.x] = fmax(hi[c][threadIdx.x], hi[c][threadIdx.x + w]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) {
            part[blockIdx.x * 6 + c] = lo[c][0];
            part[blockIdx.x * 6 + 3 + c] = hi[c][0];
        }
}

// ---- 2. Morton keys ----------------------------------------------------------------
__device__ __forceinline__ unsigned spread10(unsigned v) {      // 10 bits -> every 3rd bit
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// box[0..5] = (min x, y, z, max x, y, z) from the per-block partials (one warp).
__global__ void bbox_finish_kernel(const double* __restrict__ part, int nparts, double* __restrict__ box) {
    const int lane = threadIdx.x;
    double v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int b = lane; b < nparts; b += 32)
        for (int q = 0; q < 6; ++q) v[q] = q < 3 ? fmin(v[q], part[b * 6 + q]) : fmax(v[q], part[b * 6 + q]);
    for (int o = 16; o > 0; o >>= 1)
        for (int q = 0; q < 6; ++q) {
            const double w = __shfl_xor_sync(0xffffffffu, v[q], o);
            v[q] = q < 3 ? fmin(v[q], w) : fmax(v[q], w);
        }
    if (lane == 0)
        for (int q = 0; q < 6; ++q) box[q] = v[q];
}

__global__ void morton_kernel(int n, const double* __restrict__ xc, long long ld,
                              const double* __restrict__ gbox, unsigned* __restrict__ key,
                              int* __restrict__ idx) {
    __shared__ double lo[3], sc[3];        // box corner, 1024 / extent (0 for a flat axis)
    if (threadIdx.x < 3) {
        const double ext = gbox[3 + threadIdx.x] - gbox[threadIdx.x];
        lo[threadIdx.x] = gbox[threadIdx.x];
        sc[threadIdx.x] = ext > 0.0 ? 1024.0 / ext : 0.0;
    }
    __syncthreads();
    const int k = blockIdx.x * kOB + threadIdx.x;
    if (k >= n) return;
    unsigned code = 0;
    for (int c = 0; c < 3; ++c) {
        const double s = (xc[(size_t)c * ld + k] - lo[c]) * sc[c];
        const unsigned q = (unsigned)fmin(1023.0, fmax(0.0, s));
        code |= spread10(q) << c;
    }
    key[k] = code;
    idx[k] = k;
}

// ---- 3. stable LSD radix sort ------------------------------------------------------
// Pass: per-block digit histograms (digit-major layout hist[d * nb + b]), an exclusive
// scan over that layout (scan_* kernels below), then a stable scatter: the rank of an element among equal
// digits of its block = (equal digits in earlier warps) + (equal digits at lower lanes of
// its warp, from __match_any_sync).
// Exclusive scan of m ints in three launches: scan inside chunks of kScanChunk, scan of
// the chunk totals by one CTA, add the chunk offsets.
constexpr int kScanT = 1024;
constexpr int kScanPer = 4;
constexpr int kScanChunk = kScanT * kScanPer;

// Block-wide exclusive scan of one int per thread (blockDim.x == kScanT); returns the
// thread's exclusive prefix and writes the block total to *total.
__device__ int block_exclusive(int v, int* total) {
    __shared__ int wsum[kScanT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;                      // inclusive over warps
    }
    __syncthreads();
    const int before = (w > 0 ? wsum[w - 1] : 0) + x - v;
    *total = wsum[kScanT / 32 - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(kScanT) scan_chunks_kernel(const int* __restrict__ in, int m,
                                                             int* __restrict__ out, int* __restrict__ sums) {
    const long long base = (long long)blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    int v[kScanPer], t = 0;
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) {
        v[e] = base + e < m ? in[base + e] : 0;
        t += v[e];
    }
    int total;
    int run = block_exclusive(t, &total);
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) {
        if (base + e < m) out[base + e] = run;
        run += v[e];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanT) scan_sums_kernel(int* __restrict__ sums, int nc) {
    const int per = (nc + kScanT - 1) / kScanT;
    const int a = min(nc, (int)threadIdx.x * per), b = min(nc, a + per);
    int t = 0;
    for (int k = a; k < b; ++k) t += sums[k];
    int total;
    int run = block_exclusive(t, &total);
    for (int k = a; k < b; ++k) {
        const int v = sums[k];
        sums[k] = run;
        run += v;
    }
}

__global__ void scan_add_kernel(int* __restrict__ out, int m, const int* __restrict__ sums) {
    const long long k = (long long)blockIdx.x * kOB + threadIdx.x;
    if (k < m) out[k] += sums[k / kScanChunk];
}

__global__ void radix_hist_kernel(int n, const unsigned* __restrict__ key, int shift, int* __restrict__ hist) {
    __shared__ int h[kRadixBins];
    for (int d = threadIdx.x; d < kRadixBins; d += kOB) h[d] = 0;
    __syncthreads();
    const int k = blockIdx.x * kOB + threadIdx.x;
    if (k < n) atomicAdd(&h[(key[k] >> shift) & (kRadixBins - 1)], 1);
    __syncthreads();
    for (int d = threadIdx.x; d < kRadixBins; d += kOB) hist[(size_t)d * gridDim.x + blockIdx.x] = h[d];
}

__global__ void radix_scatter_kernel(int n, const unsigned* __restrict__ kin, const int* __restrict__ iin,
                                     int shift, const int* __restrict__ offs, unsigned* __restrict__ kout,
                                     int* __restrict__ iout) {
    __shared__ int wcount[kOB / 32][kRadixBins];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = threadIdx.x; q < (kOB / 32) * kRadixBins; q += kOB) (&wcount[0][0])[q] = 0;
    __syncthreads();
    const int k = blockIdx.x * kOB + threadIdx.x;
    const bool valid = k < n;
    const unsigned key = valid ? kin[k] : 0u;
    const int d = valid ? (int)((key >> shift) & (kRadixBins - 1)) : kRadixBins;   // invalid: own class
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int lane_rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && lane_rank == 0) wcount[wid][d] = __popc(peers);
    __syncthreads();
    if (!valid) return;
    int before = 0;
    for (int w = 0; w < wid; ++w) before += wcount[w][d];
    const int dst = offs[(size_t)d * gridDim.x + blockIdx.x] + before + lane_rank;
    kout[dst] = key;
    iout[dst] = iin[k];
}

// ---- 4. sub-tiles of the packed records ---------------------------------------------
// One warp per 32 records.  rel[k].w (the FP32 mass) is written once per set order by
// rel_mass_kernel and kept; this kernel rewrites rel[k].xyz and sub[k / 32].
// mass_from_rec: rel.w = m from the record's 2.5 m (within 1.5 ulp of the FP32 mass), for
// sets whose rel.w was not filled from the FP64 masses.
__global__ void subtile_kernel(int n, const RecMix* __restrict__ rec, float4* __restrict__ rel,
                               float4* __restrict__ sub, bool mass_from_rec) {
    const int k = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= (n + 31) >> 5) return;                      // warp-uniform
    const int j = k * 32 + lane;
    const RecMix r = rec[min(j, n - 1)];                 // lanes past n repeat record n-1
    const float xh[3] = {r.hi.x, r.hi.y, r.hi.z};
    const float xl[3] = {r.lo.x, r.lo.y, r.lo.z};
    float C[3], d[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        float lo = xh[q], hi = xh[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        C[q] = 0.5f * lo + 0.5f * hi;
        d[q] = (float)(((double)xh[q] - (double)C[q]) + (double)xl[q]);
    }
    float R = sqrtf(fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) R = fmaxf(R, __shfl_xor_sync(0xffffffffu, R, o));
    if (j < n) {
        float4 v = mass_from_rec ? make_float4(0.f, 0.f, 0.f, (float)(0.4 * (double)r.hi.w)) : rel[j];
        v.x = d[0]; v.y = d[1]; v.z = d[2];
        rel[j] = v;
    }
    if (lane == 0) sub[k] = make_float4(C[0], C[1], C[2], R * (1.0f + 0x1p-20f));
}

__global__ void rel_mass_kernel(const double* __restrict__ mass, const int* __restrict__ idx, int n,
                                float4* __restrict__ rel) {
    const int k = blockIdx.x * kOB + threadIdx.x;
    if (k >= n) return;
    rel[k] = make_float4(0.f, 0.f, 0.f, (float)mass[idx ? idx[k] : k]);
}

// list[k] = idx ? idx[perm[k]] : perm[k]
__global__ void compose_kernel(const int* __restrict__ idx, const int* __restrict__ perm, int n,
                               int* __restrict__ list) {
    const int k = blockIdx.x * kOB + threadIdx.x;
    if (k >= n) return;
    list[k] = idx ? idx[perm[k]] : perm[k];
}

// Workspace (bytes) needed by launch_morton_order for n particles (the same carving).
size_t morton_workspace_bytes(int n) {
    const int nb = nblocks(n);
    const int nparts = std::min(nb, 1024);
    const long long m = (long long)kRadixBins * nb;
    const long long nc = (m + kScanChunk - 1) / kScanChunk;
    auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
    return 3 * r((size_t)n * 4) + 2 * r((size_t)m * 4) + r((size_t)nparts * 6 * 8) + r(6 * 8) +
           r((size_t)nc * 4);
}

// perm[k] = index (into the set) of the particle at sorted position k.  xc: 3 rows of
// leading dimension ld (>= n) holding the set's positions.
cudaError_t launch_morton_order(int n, const double* xc, long long ld, int* perm, void* ws,
                                size_t ws_bytes, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int nb = nblocks(n);
    unsigned char* p = reinterpret_cast<unsigned char*>(ws);
    auto take = [&](size_t bytes) { unsigned char* q = p; p += (bytes + 255) & ~size_t(255); return q; };
    unsigned* k0 = reinterpret_cast<unsigned*>(take((size_t)n * 4));
    unsigned* k1 = reinterpret_cast<unsigned*>(take((size_t)n * 4));
    int* i1 = reinterpret_cast<int*>(take((size_t)n * 4));
    int* hist = reinterpret_cast<int*>(take((size_t)kRadixBins * nb * 4));
    int* offs = reinterpret_cast<int*>(take((size_t)kRadixBins * nb * 4));
    const int nparts = std::min(nb, 1024);
    double* part = reinterpret_cast<double*>(take((size_t)nparts * 6 * 8));
    double* box = reinterpret_cast<double*>(take(6 * 8));
    const int m = kRadixBins * nb;
    const int nc = (m + kScanChunk - 1) / kScanChunk;
    int* sums = reinterpret_cast<int*>(take((size_t)nc * 4));
    if ((size_t)(p - reinterpret_cast<unsigned char*>(ws)) > ws_bytes) return cudaErrorInvalidValue;
    { bbox_partial_kernel<<<nparts, kOB, 0, s>>>(n, xc, ld, part); note_launch(); }
    { bbox_finish_kernel<<<1, 32, 0, s>>>(part, nparts, box); note_launch(); }
    { morton_kernel<<<nb, kOB, 0, s>>>(n, xc, ld, box, k0, perm); note_launch(); }
    unsigned* kin = k0;
    unsigned* kout = k1;
    int* iin = perm;
    int* iout = i1;
    for (int shift = 0; shift < 30; shift += kRadixBits) {
        { radix_hist_kernel<<<nb, kOB, 0, s>>>(n, kin, shift, hist); note_launch(); }
        { scan_chunks_kernel<<<nc, kScanT, 0, s>>>(hist, m, offs, sums); note_launch(); }
        { scan_sums_kernel<<<1, kScanT, 0, s>>>(sums, nc); note_launch(); }
        { scan_add_kernel<<<(m + kOB - 1) / kOB, kOB, 0, s>>>(offs, m, sums); note_launch(); }
        { radix_scatter_kernel<<<nb, kOB, 0, s>>>(n, kin, iin, shift, offs, kout, iout); note_launch(); }
        std::swap(kin, kout);
        std::swap(iin, iout);
    }
    // 4 passes: the result is back in (k0, perm)
    return cudaGetLastError();
}

cudaError_t launch_compose(const int* idx, const int* perm, int n, int* list, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    { compose_kernel<<<nblocks(n), kOB, 0, s>>>(idx, perm, n, list); note_launch(); }
    return cudaGetLastError();
}

cudaError_t launch_rel_mass(const double* mass, const int* idx, int n, void* rel, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    { rel_mass_kernel<<<nblocks(n), kOB, 0, s>>>(mass, idx, n, reinterpret_cast<float4*>(rel)); note_launch(); }
    return cudaGetLastError();
}

cudaError_t launch_subtiles(int n, const void* rec, void* rel, void* sub, cudaStream_t s,
                            bool mass_from_rec) {
    if (n <= 0) return cudaSuccess;
    const long long threads = (long long)((n + 31) / 32) * 32;
    const int blocks = (int)((threads + kOB - 1) / kOB);
    { subtile_kernel<<<blocks, kOB, 0, s>>>(n, reinterpret_cast<const RecMix*>(rec),
                                             reinterpret_cast<float4*>(rel), reinterpret_cast<float4*>(sub),
                                             mass_from_rec);
      note_launch(); }
    return cudaGetLastError();
}

}  // namespace fsi
