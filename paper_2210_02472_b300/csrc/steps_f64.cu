// steps_f64.cu -- time steps of a set against itself (Sect. 3.4) in FP64: the symmetric
// form (every unordered pair of the set evaluated once) and, at the end of the file, the
// one-sided form for receiver slices and small sets with the same pair update.
//
// For receiver i over the other members j of the set (d = x_j - x_i, u = v_j - v_i,
// s^2 = |d|^2 + eps^2):
//   free fall  eps_ff = eta_ff min_j (|d|^3 / (m_i + m_j))^{1/2},
//   fly-by     eps_fb = eta_fb min_j |d| / |u|,
//   jerk       eps_j  = eta_jerk |a_i| / |j_i|,  a_i = sum_j m_j d / s^3,
//              j_i = sum_j m_j (u / s^3 - 3 (d.u) d / s^5),
// eps_i the minimum of the three (no partner: +inf; |u| = 0 and |j| = 0 give no bound).
// |d|^6 / (m_i + m_j)^2, |d|^2 / |u|^2 and d.u are the same for both particles of a pair,
// while the a and j terms change sign with d -> -d, u -> -u: the term of i on j is the
// term of j on i with m_i in place of m_j and the opposite sign.  One evaluation of the
// separation, the reciprocal square root and the tidal factor serves both particles.
//
// The B300 FP64 pipe retires about two lane FMAs per SM and clock (1/64 of the FP32
// rate), so the pair update keeps its FP64 operation count down:
//  - the two minima are running fractions (numerator, denominator), both non-negative: a
//    candidate replaces the running one when n_c d_r < n_r d_c.  The two products are
//    compared through their bit patterns as signed 64-bit integers, which order like the
//    non-negative doubles themselves, so the compare runs on the integer pipe.  A running
//    fraction starts at (DBL_MAX, 1); a zero denominator (equal velocities, two massless
//    particles) then never replaces it;
//  - a coincident pair (|d| = 0) is caught by an integer test of |d|^2's bits;
//  - a fraction becomes a ratio (one correctly rounded division) once per receiver and
//    work item and once per source and warp pass.  Rounding is monotonic, so the minimum
//    of the rounded ratios (64-bit atomicMin on their bits, non-negative doubles again)
//    is the rounded ratio of the smallest fraction, the value the one-sided kernel
//    divides out at its end: both forms give the same steps, up to the summation order
//    of a and j.
//
// Work decomposition (as the symmetric pair kernels): CTAs of 256 threads hold blocks of
// 512 receivers (i0 + tid and i0 + 256 + tid) in registers; sources stream through a
// 3-stage shared-memory ring of 256 records (position (x, y, z, m) and velocity
// (u, v, w, m), 32 B each) filled by cp.async.bulk on mbarriers with bounded waits.  Work
// items (blockIdx.x = b * (1 + nchunk) + c): block b against c = 0, its own two tiles,
// one-sided with the self pair excluded by index; or c >= 1, chunk c - 1 of the tiles
// above it, both sides.  On the two-sided tiles the source side travels through the warp:
// lane l starts with a packet holding source jj + l (its records and its accumulators),
// adds its two receivers' terms to it and hands it to lane l - 1; after 32 steps every
// packet is back in its lane with the terms of all 64 of the warp's receivers, and no
// FP64 work is spent on combining partial sums across lanes.  The packet then goes into
// the set's accumulators (minima by atomicMin on the ratio bits, sums by
// red.global.add.f64), as the receiver side does at the end of the item.  A finalize
// kernel turns the accumulators into steps.
#include <algorithm>
#include <cfloat>

#include "fsi_internal.cuh"
#include "pair_math.cuh"
#include "sym_x2.cuh"

namespace fsi {

namespace {
constexpr int kSfThreads = 256;
constexpr int kSfI = 2;                                  // receivers per thread
constexpr int kSfBlock = kSfThreads * kSfI;              // receivers per block
constexpr int kSfTile = 256;                             // sources per stage
constexpr int kSfBlockTiles = kSfBlock / kSfTile;
constexpr int kSfStage = kSfTile * 64;                   // position + velocity records
constexpr int kSfSmem = kStages * kSfStage;
}  // namespace

struct SfRecv {
    double x, y, z, u, v, w, m;
};

// Running minima (as fractions) and the a and j sums of one particle.
struct SfAcc {
    double ffn, ffd, fbn, fbd;
    double ax, ay, az, jx, jy, jz;
    __device__ __forceinline__ void init() {
        ffn = fbn = DBL_MAX;
        ffd = fbd = 1.0;
        ax = ay = az = jx = jy = jz = 0.0;
    }
};

// n1 / d1 < n2 / d2 for non-negative operands, from the bit patterns of the products.
__device__ __forceinline__ bool frac_lt(double n1, double d1, double n2, double d2) {
    return __double_as_longlong(n1 * d2) < __double_as_longlong(n2 * d1);
}

// The ratio of a running fraction; the starting fraction (no partner) gives +inf.
__device__ __forceinline__ double frac_ratio(double n, double d) {
    return __double_as_longlong(n) == __double_as_longlong(DBL_MAX) ? (double)INFINITY : n / d;
}

// Source (position record pj, velocity record vj) on receiver p: the receiver side into
// r and, with SRC, the source side into q.
template <bool SOFT, bool SRC>
__device__ __forceinline__ void sf_pair(const D4& pj, const D4& vj, const SfRecv& p, double eps2,
                                        SfAcc& r, SfAcc& q, bool& coincident) {
    const double dx = pj.x - p.x, dy = pj.y - p.y, dz = pj.z - p.z;
    const double du = vj.x - p.u, dv = vj.y - p.v, dw = vj.z - p.w;
    const double d2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const double u2 = fma(du, du, fma(dv, dv, dw * dw));
    coincident |= __double_as_longlong(d2) == 0;
    const double y = rsqrt_f64(SOFT ? d2 + eps2 : d2);
    const double ms = p.m + pj.w;
    const double num = (d2 * d2) * d2, den = ms * ms;
    if (frac_lt(num, den, r.ffn, r.ffd)) { r.ffn = num; r.ffd = den; }
    if (frac_lt(d2, u2, r.fbn, r.fbd)) { r.fbn = d2; r.fbd = u2; }
    if constexpr (SRC) {
        if (frac_lt(num, den, q.ffn, q.ffd)) { q.ffn = num; q.ffd = den; }
        if (frac_lt(d2, u2, q.fbn, q.fbd)) { q.fbn = d2; q.fbd = u2; }
    }
    const double y2 = y * y, y3 = y2 * y;
    const double rv = fma(dx, du, fma(dy, dv, dz * dw));
    const double c3 = rv * (-3.0 * y2);
    const double tx = fma(c3, dx, du), ty = fma(c3, dy, dv), tz = fma(c3, dz, dw);
    const double wi = pj.w * y3;
    r.ax = fma(wi, dx, r.ax); r.ay = fma(wi, dy, r.ay); r.az = fma(wi, dz, r.az);
    r.jx = fma(wi, tx, r.jx); r.jy = fma(wi, ty, r.jy); r.jz = fma(wi, tz, r.jz);
    if constexpr (SRC) {
        const double wj = -(p.m * y3);
        q.ax = fma(wj, dx, q.ax); q.ay = fma(wj, dy, q.ay); q.az = fma(wj, dz, q.az);
        q.jx = fma(wj, tx, q.jx); q.jy = fma(wj, ty, q.jy); q.jz = fma(wj, tz, q.jz);
    }
}

// The step from the minima (as ratios) and the a and j sums (Sect. 3.4).
__device__ __forceinline__ double sf_finish(double ff, double fb, double ax, double ay, double az,
                                            double jx, double jy, double jz, double eta_ff,
                                            double eta_fb, double eta_jerk) {
    double e = INFINITY;
    if (ff < INFINITY) e = eta_ff * sqrt(sqrt(ff));
    if (fb < INFINITY) e = fmin(e, eta_fb * sqrt(fb));
    const double jn = sqrt(jx * jx + jy * jy + jz * jz);
    if (jn > 0.0) e = fmin(e, eta_jerk * sqrt(ax * ax + ay * ay + az * az) / jn);
    return e;
}

// One particle's accumulators into the set's: minima as ratio bits, sums by red.add.
__device__ __forceinline__ void sf_put(unsigned long long* mins, double* sums, int n, int i,
                                       const SfAcc& s) {
    atomicMin(mins + i, (unsigned long long)__double_as_longlong(frac_ratio(s.ffn, s.ffd)));
    atomicMin(mins + (size_t)n + i, (unsigned long long)__double_as_longlong(frac_ratio(s.fbn, s.fbd)));
    red_add(sums + i, s.ax);
    red_add(sums + (size_t)n + i, s.ay);
    red_add(sums + 2 * (size_t)n + i, s.az);
    red_add(sums + 3 * (size_t)n + i, s.jx);
    red_add(sums + 4 * (size_t)n + i, s.jy);
    red_add(sums + 5 * (size_t)n + i, s.jz);
}

struct StepF64Args {
    int n;
    const D4* rec;          // position records (x, y, z, m), n entries
    const D4* vrec;         // velocity records (u, v, w, m), n entries
    double eps2;
    int chunk, nchunk;
    unsigned long long* mins;   // 2 x n: bits of the ff and fb ratio minima (+inf to start)
    double* sums;               // 6 x n: a and j sums (0 to start)
    int* err;
    long long timeout_ns;
};

// 32 sources jj .. jj + 31 of a staged tile on the thread's receivers, the source side
// carried around the warp (lane l holds source jj + ((l + k) mod 32) at step k).  FULL:
// all 32 sources exist; otherwise a packet past the tile's cnt sources is carried along
// without terms.
template <bool SOFT, bool FULL>
__device__ __forceinline__ void sf_rotate(const StepF64Args& a, const D4* rec, const D4* vr,
                                          int jj, int cnt, int jt, int lane,
                                          const SfRecv (&pi)[kSfI], SfAcc (&acc)[kSfI],
                                          bool& coincident) {
    const int jh = jj + lane;
    int valid = FULL || jh < cnt;
    const int jl = valid ? jh : jj;
    D4 pj = rec[jl];
    const D4 v0 = vr[jl];
    D4 vj = make_d4(v0.x, v0.y, v0.z, 0.0);
    SfAcc q;
    q.init();
    const int from = (lane + 1) & 31;
#pragma unroll 2
    for (int k = 0; k < 32; ++k) {
        if (FULL || valid) {
#pragma unroll
            for (int u = 0; u < kSfI; ++u) sf_pair<SOFT, true>(pj, vj, pi[u], a.eps2, acc[u], q, coincident);
        }
        pj.x = __shfl_sync(0xffffffffu, pj.x, from);
        pj.y = __shfl_sync(0xffffffffu, pj.y, from);
        pj.z = __shfl_sync(0xffffffffu, pj.z, from);
        pj.w = __shfl_sync(0xffffffffu, pj.w, from);
        vj.x = __shfl_sync(0xffffffffu, vj.x, from);
        vj.y = __shfl_sync(0xffffffffu, vj.y, from);
        vj.z = __shfl_sync(0xffffffffu, vj.z, from);
        q.ffn = __shfl_sync(0xffffffffu, q.ffn, from);
        q.ffd = __shfl_sync(0xffffffffu, q.ffd, from);
        q.fbn = __shfl_sync(0xffffffffu, q.fbn, from);
        q.fbd = __shfl_sync(0xffffffffu, q.fbd, from);
        q.ax = __shfl_sync(0xffffffffu, q.ax, from);
        q.ay = __shfl_sync(0xffffffffu, q.ay, from);
        q.az = __shfl_sync(0xffffffffu, q.az, from);
        q.jx = __shfl_sync(0xffffffffu, q.jx, from);
        q.jy = __shfl_sync(0xffffffffu, q.jy, from);
        q.jz = __shfl_sync(0xffffffffu, q.jz, from);
        if (!FULL) valid = __shfl_sync(0xffffffffu, valid, from);
    }
    // after 32 steps every packet is back in its own lane
    if (FULL || valid) sf_put(a.mins, a.sums, a.n, jt + jh, q);
}

template <bool SOFT>
__global__ void __launch_bounds__(kSfThreads, 1) steps_sym_f64_kernel(const StepF64Args a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[kStages];
    const int b = blockIdx.x / (1 + a.nchunk);
    const int c = blockIdx.x % (1 + a.nchunk);
    const int ntj = (a.n + kSfTile - 1) / kSfTile;
    const bool diag = (c == 0);
    int t0, t1;
    if (diag) { t0 = b * kSfBlockTiles; t1 = min(t0 + kSfBlockTiles, ntj); }
    else { t0 = (b + 1) * kSfBlockTiles + (c - 1) * a.chunk; t1 = min(t0 + a.chunk, ntj); }
    if (t0 >= t1) return;                       // uniform: before any barrier
    const int ntiles = t1 - t0;
    const int tid = threadIdx.x, lane = tid & 31;
    const int i0 = b * kSfBlock;
    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) mbar_init(&bars[st], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int t) {
        const int st = t % kStages;
        const int jt = (t0 + t) * kSfTile;
        const int cnt = min(kSfTile, a.n - jt);
        unsigned char* base = smem + st * kSfStage;
        mbar_arrive_expect_tx(&bars[st], (uint32_t)cnt * 64u);
        bulk_g2s(base, a.rec + jt, (uint32_t)cnt * 32u, &bars[st]);
        bulk_g2s(base + kSfTile * 32, a.vrec + jt, (uint32_t)cnt * 32u, &bars[st]);
    };
    if (tid == 0)
        for (int t = 0; t < min(kStages, ntiles); ++t) issue(t);
    // receivers past the end of the set (last block only) hold a copy of particle n - 1;
    // their self pair is excluded through the clamped index me_c, and they write nothing
    SfRecv pi[kSfI];
    SfAcc acc[kSfI];
    int me[kSfI], me_c[kSfI];
#pragma unroll
    for (int u = 0; u < kSfI; ++u) {
        me[u] = i0 + u * kSfThreads + tid;
        me_c[u] = min(me[u], a.n - 1);
        const D4 r = a.rec[me_c[u]], v = a.vrec[me_c[u]];
        pi[u].x = r.x; pi[u].y = r.y; pi[u].z = r.z; pi[u].m = r.w;
        pi[u].u = v.x; pi[u].v = v.y; pi[u].w = v.z;
        acc[u].init();
    }
    bool coincident = false, aborted = false;
    int t_stop = ntiles;
    for (int t = 0; t < ntiles; ++t) {
        const int st = t % kStages;
        const bool ok = mbar_wait_bounded(&bars[st], (uint32_t)((t / kStages) & 1), a.timeout_ns, a.err);
        const int jt = (t0 + t) * kSfTile;
        const int cnt = min(kSfTile, a.n - jt);
        const D4* rec = reinterpret_cast<const D4*>(smem + st * kSfStage);
        const D4* vr = rec + kSfTile;
        if (diag) {
            for (int jj = 0; jj < cnt; ++jj) {
                const D4 pj = rec[jj], vj = vr[jj];
                const int j = jt + jj;
#pragma unroll
                for (int u = 0; u < kSfI; ++u)
                    if (j != me_c[u]) sf_pair<SOFT, false>(pj, vj, pi[u], a.eps2, acc[u], acc[u], coincident);
            }
        } else {
            // a block with tiles above it is full: every receiver is valid
            for (int jj = 0; jj < cnt; jj += 32) {
                if (jj + 32 <= cnt) sf_rotate<SOFT, true>(a, rec, vr, jj, cnt, jt, lane, pi, acc, coincident);
                else sf_rotate<SOFT, false>(a, rec, vr, jj, cnt, jt, lane, pi, acc, coincident);
            }
        }
        // the barrier also ends every read of stage st before it is refilled
        if (__syncthreads_or(!ok)) { aborted = true; t_stop = t; break; }
        if (tid == 0 && t + kStages < ntiles) issue(t + kStages);
    }
    if (aborted) {
        if (tid == 0) {
            const int issued = min(ntiles, t_stop + kStages);
            for (int t = t_stop; t < issued; ++t)
                mbar_wait_bounded(&bars[t % kStages], (uint32_t)((t / kStages) & 1), a.timeout_ns, nullptr);
        }
        __syncthreads();
        return;
    }
    if (coincident) set_error(a.err, FSI_ERR_COINCIDENT);
#pragma unroll
    for (int u = 0; u < kSfI; ++u)
        if (me[u] < a.n) sf_put(a.mins, a.sums, a.n, me[u], acc[u]);
}

// Records of the set (entry k from particle idx[k] of the 3 x N rows; idx null: particle
// k) and the accumulators' starting values.
__global__ void steps_f64_pack_kernel(long long N, const double* __restrict__ pos,
                                      const double* __restrict__ vel, const double* __restrict__ mass,
                                      const int* __restrict__ idx, int n, D4* __restrict__ rec,
                                      D4* __restrict__ vrec, unsigned long long* __restrict__ mins,
                                      double* __restrict__ sums) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long i = idx ? (long long)idx[k] : k;
    const double m = mass[i];
    rec[k] = make_d4(pos[i], pos[N + i], pos[2 * N + i], m);
    vrec[k] = make_d4(vel[i], vel[N + i], vel[2 * N + i], m);
    mins[k] = mins[(size_t)n + k] = 0x7ff0000000000000ull;      // +inf
#pragma unroll
    for (int q = 0; q < 6; ++q) sums[(size_t)q * n + k] = 0.0;
}

__global__ void steps_f64_finalize_kernel(int n, const unsigned long long* __restrict__ mins,
                                          const double* __restrict__ sums, double eta_ff,
                                          double eta_fb, double eta_jerk, double* __restrict__ step,
                                          int* err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double ff = __longlong_as_double((long long)mins[i]);
    const double fb = __longlong_as_double((long long)mins[(size_t)n + i]);
    const double ax = sums[i], ay = sums[(size_t)n + i], az = sums[2 * (size_t)n + i];
    const double jx = sums[3 * (size_t)n + i], jy = sums[4 * (size_t)n + i], jz = sums[5 * (size_t)n + i];
    if (!(isfinite(ax) && isfinite(ay) && isfinite(az))) set_error(err, FSI_ERR_NONFINITE);
    step[i] = sf_finish(ff, fb, ax, ay, az, jx, jy, jz, eta_ff, eta_fb, eta_jerk);
}

size_t steps_sym_f64_work_bytes(int n) { return (size_t)n * 8 * sizeof(double); }
int steps_sym_f64_min_n() { return 4 * kSfBlock; }

cudaError_t launch_steps_sym_f64(int N, const double* pos, const double* vel, const double* mass,
                                 const int* idx, int n, void* rec, void* vrec, double eps2,
                                 double eta_ff, double eta_fb, double eta_jerk, void* work,
                                 double* step, int* err, long long timeout_ns, int sm_count,
                                 cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    static std::atomic<unsigned long long> attr_dev[2];
    const bool soft = eps2 > 0.0;
    {
        const cudaError_t e = soft ? smem_attr_once(steps_sym_f64_kernel<true>, (int)kSfSmem, attr_dev[1])
                                   : smem_attr_once(steps_sym_f64_kernel<false>, (int)kSfSmem, attr_dev[0]);
        if (e != cudaSuccess) return e;
    }
    StepF64Args a{};
    a.n = n;
    a.rec = reinterpret_cast<const D4*>(rec);
    a.vrec = reinterpret_cast<const D4*>(vrec);
    a.eps2 = eps2;
    a.sums = reinterpret_cast<double*>(work);
    a.mins = reinterpret_cast<unsigned long long*>(a.sums + 6 * (size_t)n);
    a.err = err;
    a.timeout_ns = timeout_ns;
    const long long ntj = (n + kSfTile - 1) / kSfTile;
    const long long nb = (n + kSfBlock - 1) / kSfBlock;
    // about 32 items per SM (one resident CTA each), at most 64 tiles each
    const long long visits = nb * ntj / 2 + 1;
    a.chunk = (int)std::max(1LL, std::min(64LL, visits / (32LL * sm_count)));
    const long long above = ntj > kSfBlockTiles ? ntj - kSfBlockTiles : 0;
    a.nchunk = (int)((above + a.chunk - 1) / a.chunk);
    const long long grid = nb * (1 + a.nchunk);
    if (grid > 2147483647LL) return cudaErrorInvalidValue;
    { steps_f64_pack_kernel<<<(n + 255) / 256, 256, 0, s>>>(N, pos, vel, mass, idx, n,
                                                            reinterpret_cast<D4*>(rec),
                                                            reinterpret_cast<D4*>(vrec), a.mins,
                                                            a.sums); note_launch(); }
    if (soft) { steps_sym_f64_kernel<true><<<(unsigned)grid, kSfThreads, kSfSmem, s>>>(a); note_launch(); }
    else { steps_sym_f64_kernel<false><<<(unsigned)grid, kSfThreads, kSfSmem, s>>>(a); note_launch(); }
    { steps_f64_finalize_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, a.mins, a.sums, eta_ff, eta_fb,
                                                                eta_jerk, step, err); note_launch(); }
    return cudaGetLastError();
}

// =================================================================================
// One-sided form: receivers [i_off, i_off + n_i) of a compact set (3 x n SoA positions and
// velocities, masses) against all n members, every pair evaluated by its receiver: a
// receiver slice of i-sharded time steps, sets below the symmetric form's size, or
// `symmetric` off.  Thread per receiver, sources through shared memory in tiles, the
// receiver side of sf_pair (the same fractions and integer compares), the step finished in
// the thread (step[k] for entry i_off + k).
constexpr int kSfRowTile = 128;

template <bool SOFT>
__global__ void __launch_bounds__(kSfRowTile) steps_f64_rows_kernel(
    int n, const double* __restrict__ xc, const double* __restrict__ vc,
    const double* __restrict__ mc, double eta_ff, double eta_fb, double eta_jerk, double eps2,
    double* __restrict__ step, int* err, int i_off, int n_i) {
    __shared__ D4 sp[kSfRowTile], sv[kSfRowTile];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int ii = i_off + min(k, n_i - 1);            // a thread past n_i repeats the last
    SfRecv p;
    p.x = xc[ii]; p.y = xc[(size_t)n + ii]; p.z = xc[2 * (size_t)n + ii];
    p.u = vc[ii]; p.v = vc[(size_t)n + ii]; p.w = vc[2 * (size_t)n + ii];
    p.m = mc[ii];
    SfAcc acc;
    acc.init();
    bool coincident = false;
    for (int j0 = 0; j0 < n; j0 += kSfRowTile) {
        __syncthreads();
        {
            const int j = j0 + (int)threadIdx.x;
            if (j < n) {
                sp[threadIdx.x] = make_d4(xc[j], xc[(size_t)n + j], xc[2 * (size_t)n + j], mc[j]);
                sv[threadIdx.x] = make_d4(vc[j], vc[(size_t)n + j], vc[2 * (size_t)n + j], 0.0);
            }
        }
        __syncthreads();
        const int cnt = min(kSfRowTile, n - j0);
        if (ii >= j0 && ii < j0 + cnt) {
            for (int t = 0; t < cnt; ++t)
                if (j0 + t != ii) sf_pair<SOFT, false>(sp[t], sv[t], p, eps2, acc, acc, coincident);
        } else {
#pragma unroll 4
            for (int t = 0; t < cnt; ++t) sf_pair<SOFT, false>(sp[t], sv[t], p, eps2, acc, acc, coincident);
        }
    }
    if (k >= n_i) return;
    if (coincident) set_error(err, FSI_ERR_COINCIDENT);
    step[k] = sf_finish(frac_ratio(acc.ffn, acc.ffd), frac_ratio(acc.fbn, acc.fbd), acc.ax, acc.ay,
                        acc.az, acc.jx, acc.jy, acc.jz, eta_ff, eta_fb, eta_jerk);
}

cudaError_t launch_timesteps(int n, const double* xc, const double* vc, const double* mc,
                             double eta_ff, double eta_fb, double eta_jerk, double eps2,
                             double* step, int* err, cudaStream_t s, int i_off, int n_i) {
    if (n_i < 0) n_i = n;
    if (n <= 0 || n_i <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((n_i + kSfRowTile - 1) / kSfRowTile);
    if (eps2 > 0.0) {
        steps_f64_rows_kernel<true><<<grid, kSfRowTile, 0, s>>>(n, xc, vc, mc, eta_ff, eta_fb, eta_jerk,
                                                                 eps2, step, err, i_off, n_i);
    } else {
        steps_f64_rows_kernel<false><<<grid, kSfRowTile, 0, s>>>(n, xc, vc, mc, eta_ff, eta_fb, eta_jerk,
                                                                  eps2, step, err, i_off, n_i);
    }
    note_launch();
    return cudaGetLastError();
}

}  // namespace fsi
