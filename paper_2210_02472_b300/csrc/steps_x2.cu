// steps_x2.cu -- time steps of a set against itself (Sect. 3.4) in the mixed precision,
// with packed FP32 pairs (add/mul/fma.rn.f32x2).
//
// For receiver i over every other member j of the set (d = x_j - x_i, u = v_j - v_i):
//   free fall  eps_ff = eta_ff min_j (r^3 / (m_i + m_j))^{1/2},  r = |d| (unsoftened),
//   fly-by     eps_fb = eta_fb min_j r / |u|,
//   jerk       eps_j  = eta_jerk |a_i| / |j_i|,  a_i and j_i with the softened kernel,
// eps_i the minimum of the three (no partner: +inf; |u| = 0 and |j| = 0 give no bound).
// The minima are tracked as r^3 / (m_i + m_j) and r^2 / |u|^2 with the hardware reciprocal;
// a and j accumulate in FP32 (only the ratio |a| / |j| is needed).
//
// Work decomposition: CTAs of 256 threads hold 4 receivers per thread (two packed pairs);
// sources stream through a 3-stage shared-memory ring of 256 records (position record
// 32 B + velocity record 16 B) filled by cp.async.bulk on mbarriers with bounded waits.
// When the receiver blocks alone cannot fill the GPU, blockIdx.y splits the sources and a
// finalize kernel combines the per-split minima and sums.
#include <algorithm>

#include "fsi_internal.cuh"
#include "pair_math.cuh"
#include "sym_x2.cuh"

namespace fsi {

namespace {
constexpr int kStI = 4;                          // receivers per thread
constexpr int kStNP = kStI / 2;
constexpr int kStThreads = 256;
constexpr int kStTile = 256;                     // sources per stage
constexpr int kStStage = kStTile * (32 + 16);
constexpr int kStSmem = kStages * kStStage;
constexpr int kStPart = 8;                       // ff, fb, ax, ay, az, jx, jy, jz
}  // namespace

__device__ __forceinline__ float rcp_hw(float v) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ float2 rcp2(float2 v) { return make_float2(rcp_hw(v.x), rcp_hw(v.y)); }

struct StepX2I {
    float2 nxh, nyh, nzh, nxl, nyl, nzl;   // -position splits of the two receivers
    float2 nu, nv, nw;                     // -velocities
    float2 m;                              // masses
};

struct StepX2Acc {
    float2 ff, fb, ax, ay, az, jx, jy, jz;
};

// Source j (position record h/l, velocity record vj = (vx, vy, vz, m)) on both receivers
// of a pair.  CHK: the source may be one of them (self_lo / self_hi), which is skipped.
template <bool CHK, bool SOFT>
__device__ __forceinline__ void step_pair_x2(const float4 h, const float4 l, const float4 vj,
                                             const StepX2I& p, float2 eps2, bool self_lo,
                                             bool self_hi, StepX2Acc& s, bool& coincident) {
    const float2 dx = __fadd2_rn(__fadd2_rn(bc2(h.x), p.nxh), __fadd2_rn(bc2(l.x), p.nxl));
    const float2 dy = __fadd2_rn(__fadd2_rn(bc2(h.y), p.nyh), __fadd2_rn(bc2(l.y), p.nyl));
    const float2 dz = __fadd2_rn(__fadd2_rn(bc2(h.z), p.nzh), __fadd2_rn(bc2(l.z), p.nzl));
    float2 d2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
    if (CHK) {
        d2.x = self_lo ? 1.0f : d2.x;
        d2.y = self_hi ? 1.0f : d2.y;
    }
    coincident |= (d2.x == 0.0f) | (d2.y == 0.0f);
    const float2 ux = __fadd2_rn(bc2(vj.x), p.nu), uy = __fadd2_rn(bc2(vj.y), p.nv),
                 uz = __fadd2_rn(bc2(vj.z), p.nw);
    const float2 u2 = __ffma2_rn(ux, ux, __ffma2_rn(uy, uy, __fmul2_rn(uz, uz)));
    const float2 s2 = SOFT ? __fadd2_rn(d2, eps2) : d2;
    float2 y = rsqrt2(s2);
    // one Newton step of the hardware reciprocal square root: y (3 - s2 y^2) / 2
    y = __fmul2_rn(y, __ffma2_rn(__fmul2_rn(s2, bc2(-0.5f)), __fmul2_rn(y, y), bc2(1.5f)));
    const float2 y2 = __fmul2_rn(y, y);
    float2 w = __fmul2_rn(bc2(vj.w), __fmul2_rn(y2, y));                   // m_j / s^3
    const float2 r = __fmul2_rn(d2, SOFT ? rsqrt2(d2) : y);               // |d|
    float2 tff = __fmul2_rn(__fmul2_rn(d2, r), rcp2(__fadd2_rn(bc2(vj.w), p.m)));
    float2 tfb = __fmul2_rn(d2, rcp2(u2));
    if (CHK) {
        tff.x = self_lo ? INFINITY : tff.x; tff.y = self_hi ? INFINITY : tff.y;
        tfb.x = self_lo ? INFINITY : tfb.x; tfb.y = self_hi ? INFINITY : tfb.y;
        w.x = self_lo ? 0.0f : w.x;
        w.y = self_hi ? 0.0f : w.y;
    }
    s.ff.x = fminf(s.ff.x, tff.x); s.ff.y = fminf(s.ff.y, tff.y);
    s.fb.x = fminf(s.fb.x, tfb.x); s.fb.y = fminf(s.fb.y, tfb.y);
    const float2 rv = __ffma2_rn(dx, ux, __ffma2_rn(dy, uy, __fmul2_rn(dz, uz)));
    const float2 c3 = __fmul2_rn(__fmul2_rn(rv, y2), bc2(-3.0f));
    s.ax = __ffma2_rn(w, dx, s.ax); s.ay = __ffma2_rn(w, dy, s.ay); s.az = __ffma2_rn(w, dz, s.az);
    s.jx = __ffma2_rn(w, __ffma2_rn(c3, dx, ux), s.jx);
    s.jy = __ffma2_rn(w, __ffma2_rn(c3, dy, uy), s.jy);
    s.jz = __ffma2_rn(w, __ffma2_rn(c3, dz, uz), s.jz);
}

__device__ __forceinline__ double step_from(float ff, float fb, float ax, float ay, float az,
                                            float jx, float jy, float jz, double eta_ff,
                                            double eta_fb, double eta_jerk) {
    double e = INFINITY;
    if (isfinite(ff)) e = eta_ff * sqrt((double)ff);
    if (isfinite(fb)) e = fmin(e, eta_fb * sqrt((double)fb));
    const double jn = sqrt((double)jx * jx + (double)jy * jy + (double)jz * jz);
    if (jn > 0.0) e = fmin(e, eta_jerk * sqrt((double)ax * ax + (double)ay * ay + (double)az * az) / jn);
    return e;
}

struct StepX2Args {
    int n;                  // sources: records [0, n)
    int i_off, n_i;         // receivers: records [i_off, i_off + n_i), outputs [0, n_i)
    const RecMix* rec;
    const float4* vrec;
    float eps2;
    double eta_ff, eta_fb, eta_jerk;
    int j_per_split;
    float* part;            // split > 1: [split][kStPart][n_i]
    double* step;
    int* err;
    long long timeout_ns;
};

template <bool SOFT>
__global__ void __launch_bounds__(kStThreads, 2) steps_x2_kernel(const StepX2Args a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[kStages];
    const int tid = threadIdx.x;
    const int i0 = blockIdx.x * (kStThreads * kStI);
    const int js = blockIdx.y * a.j_per_split;
    const int je = min(a.n, js + a.j_per_split);
    const int ntiles = max(0, (je - js + kStTile - 1) / kStTile);
    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) mbar_init(&bars[st], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int t) {
        const int st = t % kStages;
        const int jt = js + t * kStTile;
        const int cnt = min(kStTile, je - jt);
        unsigned char* base = smem + st * kStStage;
        mbar_arrive_expect_tx(&bars[st], (uint32_t)cnt * 48u);
        bulk_g2s(base, a.rec + jt, (uint32_t)cnt * 32u, &bars[st]);
        bulk_g2s(base + kStTile * 32, a.vrec + jt, (uint32_t)cnt * 16u, &bars[st]);
    };
    if (tid == 0)
        for (int t = 0; t < min(kStages, ntiles); ++t) issue(t);
    // receivers: i0 + u * 256 + tid, u = 0..3; pair p holds u = 2p (low) and 2p + 1 (high)
    StepX2I pp[kStNP];
    StepX2Acc acc[kStNP];
    // lanes past the end hold a copy of the last receiver and use its index for the self
    // test; receiver k is record i_off + k
    int me[kStI];
#pragma unroll
    for (int u = 0; u < kStI; ++u) {
        const int i = a.i_off + min(i0 + u * kStThreads + tid, a.n_i - 1);
        me[u] = i;
        const RecMix r = a.rec[i];
        const float4 v = a.vrec[i];
        const int h = u & 1;
        StepX2I& q = pp[u >> 1];
        set_half(q.nxh, h, -r.hi.x); set_half(q.nyh, h, -r.hi.y); set_half(q.nzh, h, -r.hi.z);
        set_half(q.nxl, h, -r.lo.x); set_half(q.nyl, h, -r.lo.y); set_half(q.nzl, h, -r.lo.z);
        set_half(q.nu, h, -v.x); set_half(q.nv, h, -v.y); set_half(q.nw, h, -v.z);
        set_half(q.m, h, v.w);
    }
#pragma unroll
    for (int p = 0; p < kStNP; ++p) {
        acc[p].ff = acc[p].fb = bc2(INFINITY);
        acc[p].ax = acc[p].ay = acc[p].az = acc[p].jx = acc[p].jy = acc[p].jz = bc2(0.0f);
    }
    const float2 eps2 = bc2(a.eps2);
    bool coincident = false, aborted = false;
    int t_stop = ntiles;
    for (int t = 0; t < ntiles; ++t) {
        const int st = t % kStages;
        const bool ok = mbar_wait_bounded(&bars[st], (uint32_t)((t / kStages) & 1), a.timeout_ns, a.err);
        const int jt = js + t * kStTile;
        const int cnt = min(kStTile, je - jt);
        const unsigned char* base = smem + st * kStStage;
        const RecMix* rec = reinterpret_cast<const RecMix*>(base);
        const float4* vr = reinterpret_cast<const float4*>(base + kStTile * 32);
        const bool chk = jt < a.i_off + i0 + kStThreads * kStI && jt + cnt > a.i_off + i0;
        if (!chk) {
            for (int jj = 0; jj < cnt; ++jj) {
                const float4 h = rec[jj].hi, l = rec[jj].lo, v = vr[jj];
#pragma unroll
                for (int p = 0; p < kStNP; ++p)
                    step_pair_x2<false, SOFT>(h, l, v, pp[p], eps2, false, false, acc[p], coincident);
            }
        } else {
            for (int jj = 0; jj < cnt; ++jj) {
                const float4 h = rec[jj].hi, l = rec[jj].lo, v = vr[jj];
                const int j = jt + jj;
#pragma unroll
                for (int p = 0; p < kStNP; ++p)
                    step_pair_x2<true, SOFT>(h, l, v, pp[p], eps2, j == me[2 * p], j == me[2 * p + 1],
                                             acc[p], coincident);
            }
        }
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
#pragma unroll
    for (int u = 0; u < kStI; ++u) {
        const int i = i0 + u * kStThreads + tid;
        if (i >= a.n_i) continue;
        if (coincident) set_error(a.err, FSI_ERR_COINCIDENT);
        const StepX2Acc& s = acc[u >> 1];
        const bool hi = (u & 1) != 0;
        const float v[kStPart] = {hi ? s.ff.y : s.ff.x, hi ? s.fb.y : s.fb.x, hi ? s.ax.y : s.ax.x,
                                  hi ? s.ay.y : s.ay.x, hi ? s.az.y : s.az.x, hi ? s.jx.y : s.jx.x,
                                  hi ? s.jy.y : s.jy.x, hi ? s.jz.y : s.jz.x};
        if (gridDim.y > 1) {
#pragma unroll
            for (int k = 0; k < kStPart; ++k) a.part[((size_t)blockIdx.y * kStPart + k) * a.n_i + i] = v[k];
        } else {
            if (!(isfinite(v[2]) && isfinite(v[3]) && isfinite(v[4]))) set_error(a.err, FSI_ERR_NONFINITE);
            a.step[i] = step_from(v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], a.eta_ff, a.eta_fb, a.eta_jerk);
        }
    }
}

// Combine the per-split partials: minima of the ratios, sums of a and j (fixed order).
__global__ void steps_x2_finalize_kernel(const StepX2Args a, int split) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_i) return;
    float v[kStPart];
#pragma unroll
    for (int k = 0; k < kStPart; ++k) v[k] = a.part[(size_t)k * a.n_i + i];
    for (int s = 1; s < split; ++s) {
        const float* q = a.part + (size_t)s * kStPart * a.n_i + i;
        v[0] = fminf(v[0], q[0]);
        v[1] = fminf(v[1], q[(size_t)a.n_i]);
#pragma unroll
        for (int k = 2; k < kStPart; ++k) v[k] += q[(size_t)k * a.n_i];
    }
    if (!(isfinite(v[2]) && isfinite(v[3]) && isfinite(v[4]))) set_error(a.err, FSI_ERR_NONFINITE);
    a.step[i] = step_from(v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], a.eta_ff, a.eta_fb, a.eta_jerk);
}

// Wide form for sets too small for the tiled kernel to fill the GPU: 2^lg lanes per
// receiver stride over the sources (records read through L1), then combine their minima
// and sums by shuffles.  Per pair the arithmetic of step_pair_x2 on one receiver.
template <bool SOFT>
__global__ void __launch_bounds__(kStThreads) steps_wide_kernel(const StepX2Args a, int lg) {
    const int G = 1 << lg;
    const long long gt = (long long)blockIdx.x * kStThreads + threadIdx.x;
    const int slot = (int)(gt >> lg);
    const int g = (int)(gt & (G - 1));
    const bool active = slot < a.n_i;
    const int i = a.i_off + (active ? slot : a.n_i - 1);
    float ff = INFINITY, fb = INFINITY, ax = 0.f, ay = 0.f, az = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
    bool coincident = false;
    if (active) {
        const RecMix ri = a.rec[i];
        const float4 vi = a.vrec[i];
        for (int j = g; j < a.n; j += G) {
            const RecMix rj = a.rec[j];
            const float4 vj = a.vrec[j];
            const bool self = j == i;
            const float dx = (rj.hi.x - ri.hi.x) + (rj.lo.x - ri.lo.x);
            const float dy = (rj.hi.y - ri.hi.y) + (rj.lo.y - ri.lo.y);
            const float dz = (rj.hi.z - ri.hi.z) + (rj.lo.z - ri.lo.z);
            float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            d2 = self ? 1.0f : d2;
            coincident |= d2 == 0.0f;
            const float ux = vj.x - vi.x, uy = vj.y - vi.y, uz = vj.z - vi.z;
            const float u2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
            const float s2 = SOFT ? d2 + a.eps2 : d2;
            float y = rsqrt_hw(s2);
            y = y * fmaf(s2 * -0.5f, y * y, 1.5f);
            const float y2 = y * y;
            float w = vj.w * (y2 * y);
            const float r = d2 * (SOFT ? rsqrt_hw(d2) : y);
            float tff = (d2 * r) * rcp_hw(vj.w + vi.w);
            float tfb = d2 * rcp_hw(u2);
            tff = self ? INFINITY : tff;
            tfb = self ? INFINITY : tfb;
            w = self ? 0.0f : w;
            ff = fminf(ff, tff);
            fb = fminf(fb, tfb);
            const float rv = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
            const float c3 = (rv * y2) * -3.0f;
            ax = fmaf(w, dx, ax); ay = fmaf(w, dy, ay); az = fmaf(w, dz, az);
            jx = fmaf(w, fmaf(c3, dx, ux), jx);
            jy = fmaf(w, fmaf(c3, dy, uy), jy);
            jz = fmaf(w, fmaf(c3, dz, uz), jz);
        }
    }
    if (coincident) set_error(a.err, FSI_ERR_COINCIDENT);
    for (int o = G >> 1; o > 0; o >>= 1) {
        ff = fminf(ff, __shfl_xor_sync(0xffffffffu, ff, o));
        fb = fminf(fb, __shfl_xor_sync(0xffffffffu, fb, o));
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
        jx += __shfl_xor_sync(0xffffffffu, jx, o);
        jy += __shfl_xor_sync(0xffffffffu, jy, o);
        jz += __shfl_xor_sync(0xffffffffu, jz, o);
    }
    if (!active || g != 0) return;
    if (!(isfinite(ax) && isfinite(ay) && isfinite(az))) set_error(a.err, FSI_ERR_NONFINITE);
    a.step[slot] = step_from(ff, fb, ax, ay, az, jx, jy, jz, a.eta_ff, a.eta_fb, a.eta_jerk);
}

// =================================================================================
// Symmetric form: every unordered pair of the set once.  The pair quantities are
// symmetric (r^3 / (m_i + m_j), r^2 / |u|^2, and r.u, hence c3) or flip sign with
// d -> -d, u -> -u (the a and j terms), so the term of i on j is the term of j on i with
// m_i in place of m_j and the opposite sign.  Work items (blockIdx.x = b * (1 + nchunk) +
// c): block b of 1024 receivers (4 per thread) against c = 0: its own 4 tiles, one-sided
// with the self pair excluded by index, or c >= 1: chunk c - 1 of the tiles above it, both
// sides.  The source side of a group of 4 sources is reduced across the warp (lane
// permutation and shuffles: minima by fminf, sums by adds), across the CTA's warps in
// shared memory, then into the set's accumulators: minima as float bits by atomicMin
// (non-negative floats order as unsigned integers), sums by red.global.add.f64.  The
// receiver side goes to the same accumulators at the end of the item; a finalize kernel
// turns them into steps.
namespace {
constexpr int kSsBlock = kStThreads * kStI;                       // receivers per block
constexpr int kSsQ = 8;                                           // ff, fb, ax..az, jx..jz
constexpr int kSsJpart = (kStThreads / 32) * kStTile * kSsQ * 4;   // per-warp source rows
// stage: position records (32 B), velocity records (16 B), far-tile offset records (16 B)
// and the tile's 8 sub-tile (centre, radius) records
constexpr int kSsStage = kStTile * (32 + 16 + 16) + (kStTile / 32) * 16;
constexpr int kSsSmem = kStages * kSsStage + kSsJpart;
}  // namespace

struct StepSymArgs {
    int n;
    const RecMix* rec;
    const float4* vrec;
    float eps2;
    int chunk, nchunk;
    unsigned* mins;         // 2 x n: float bits of the ff and fb minima (+inf to start)
    double* sums;           // 6 x n: a and j sums (0 to start)
    int* err;
    long long timeout_ns;
    // far-tile path (null rel: never taken): the set's records relative to the centres C of
    // their 32-record sub-tiles and the sub-tiles' (C, R), as for the acceleration kernels;
    // a warp takes d = (C - x_i) + (x_j - C) for a sub-tile whose gap to the warp's box is
    // at least sqrt(far_k2) R
    const float4* rel;
    const float4* sub;
    float far_k2;
};

// Source j on both receivers of a packed pair (all receivers valid, j none of them), with
// the separation d = x_j - x_i given: receiver side into s, source side into pj (a_j, j_j
// per half) and the running minima.  The hardware reciprocal square root is used as it is
// (relative error below 2^-22): a time step needs far less.
template <bool SOFT>
__device__ __forceinline__ void step_pair_sym(const float2 dx, const float2 dy, const float2 dz,
                                              const float4 vj, const StepX2I& p, float2 nmi,
                                              float2 eps2, StepX2Acc& s, float2 (&pj)[6],
                                              float& jff, float& jfb, bool& coincident) {
    const float2 d2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
    coincident |= (d2.x == 0.0f) | (d2.y == 0.0f);
    const float2 ux = __fadd2_rn(bc2(vj.x), p.nu), uy = __fadd2_rn(bc2(vj.y), p.nv),
                 uz = __fadd2_rn(bc2(vj.z), p.nw);
    const float2 u2 = __ffma2_rn(ux, ux, __ffma2_rn(uy, uy, __fmul2_rn(uz, uz)));
    const float2 s2 = SOFT ? __fadd2_rn(d2, eps2) : d2;
    const float2 y = rsqrt2(s2);
    const float2 y2 = __fmul2_rn(y, y);
    const float2 y3 = __fmul2_rn(y2, y);
    const float2 wi = __fmul2_rn(bc2(vj.w), y3);                       //  m_j / s^3
    const float2 wj = __fmul2_rn(nmi, y3);                             // -m_i / s^3
    const float2 r = __fmul2_rn(d2, SOFT ? rsqrt2(d2) : y);           // |d|
    const float2 tff = __fmul2_rn(__fmul2_rn(d2, r), rcp2(__fadd2_rn(bc2(vj.w), p.m)));
    const float2 tfb = __fmul2_rn(d2, rcp2(u2));
    s.ff.x = fminf(s.ff.x, tff.x); s.ff.y = fminf(s.ff.y, tff.y);
    s.fb.x = fminf(s.fb.x, tfb.x); s.fb.y = fminf(s.fb.y, tfb.y);
    jff = fminf(jff, fminf(tff.x, tff.y));
    jfb = fminf(jfb, fminf(tfb.x, tfb.y));
    const float2 rv = __ffma2_rn(dx, ux, __ffma2_rn(dy, uy, __fmul2_rn(dz, uz)));
    const float2 c3 = __fmul2_rn(__fmul2_rn(rv, y2), bc2(-3.0f));
    const float2 tx = __ffma2_rn(c3, dx, ux), ty = __ffma2_rn(c3, dy, uy), tz = __ffma2_rn(c3, dz, uz);
    s.ax = __ffma2_rn(wi, dx, s.ax); s.ay = __ffma2_rn(wi, dy, s.ay); s.az = __ffma2_rn(wi, dz, s.az);
    s.jx = __ffma2_rn(wi, tx, s.jx); s.jy = __ffma2_rn(wi, ty, s.jy); s.jz = __ffma2_rn(wi, tz, s.jz);
    pj[0] = __ffma2_rn(wj, dx, pj[0]); pj[1] = __ffma2_rn(wj, dy, pj[1]); pj[2] = __ffma2_rn(wj, dz, pj[2]);
    pj[3] = __ffma2_rn(wj, tx, pj[3]); pj[4] = __ffma2_rn(wj, ty, pj[4]); pj[5] = __ffma2_rn(wj, tz, pj[5]);
}

// A group of 4 sources (lane l takes source jj + (g ^ (l >> 3)) at step g), then the
// warp's source-side totals of the group into jpart (row per warp, 8 values per source).
// FG: far form, the separation from the sub-tile offsets D = (C - xh_i) - xl_i and the
// source's offset record r = x_j - C (3 additions instead of 9).
template <bool SOFT, bool FULL, bool FG>
__device__ __forceinline__ void steps_sym_group(int jj, int cnt, int lane, int warp,
                                                const RecMix* rec, const float4* vr,
                                                const float4* rel_s, const float2 (&D)[kStNP][3],
                                                const StepX2I (&pp)[kStNP], const float2 (&nmi)[kStNP],
                                                float2 eps2, StepX2Acc (&acc)[kStNP], float* jpart,
                                                bool& coincident) {
    const int L = lane >> 3;
    float fj[4][kSsQ];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        fj[g][0] = fj[g][1] = INFINITY;
#pragma unroll
        for (int q = 2; q < kSsQ; ++q) fj[g][q] = 0.f;
        const int jg = jj + (g ^ L);
        if (FULL || jg < cnt) {
            const float4 v = vr[jg];
            float2 pj[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) pj[q] = make_float2(0.f, 0.f);
            float jff = INFINITY, jfb = INFINITY;
            if constexpr (FG) {
                const float4 r = rel_s[jg];
#pragma unroll
                for (int p = 0; p < kStNP; ++p)
                    step_pair_sym<SOFT>(__fadd2_rn(D[p][0], bc2(r.x)), __fadd2_rn(D[p][1], bc2(r.y)),
                                        __fadd2_rn(D[p][2], bc2(r.z)), v, pp[p], nmi[p], eps2, acc[p],
                                        pj, jff, jfb, coincident);
            } else {
                const float4 h = rec[jg].hi, l = rec[jg].lo;
#pragma unroll
                for (int p = 0; p < kStNP; ++p) {
                    const StepX2I& q = pp[p];
                    step_pair_sym<SOFT>(__fadd2_rn(__fadd2_rn(bc2(h.x), q.nxh), __fadd2_rn(bc2(l.x), q.nxl)),
                                        __fadd2_rn(__fadd2_rn(bc2(h.y), q.nyh), __fadd2_rn(bc2(l.y), q.nyl)),
                                        __fadd2_rn(__fadd2_rn(bc2(h.z), q.nzh), __fadd2_rn(bc2(l.z), q.nzl)),
                                        v, q, nmi[p], eps2, acc[p], pj, jff, jfb, coincident);
                }
            }
            fj[g][0] = jff;
            fj[g][1] = jfb;
#pragma unroll
            for (int q = 0; q < 6; ++q) fj[g][2 + q] = pj[q].x + pj[q].y;
        }
    }
#pragma unroll
    for (int q = 0; q < kSsQ; ++q) {
        float r;
        if (q < 2) {
            const float k0 = fminf(fj[0][q], __shfl_xor_sync(0xffffffffu, fj[2][q], 16));
            const float k1 = fminf(fj[1][q], __shfl_xor_sync(0xffffffffu, fj[3][q], 16));
            r = fminf(k0, __shfl_xor_sync(0xffffffffu, k1, 8));
            r = fminf(r, __shfl_xor_sync(0xffffffffu, r, 4));
            r = fminf(r, __shfl_xor_sync(0xffffffffu, r, 2));
            r = fminf(r, __shfl_xor_sync(0xffffffffu, r, 1));
        } else {
            const float k0 = fj[0][q] + __shfl_xor_sync(0xffffffffu, fj[2][q], 16);
            const float k1 = fj[1][q] + __shfl_xor_sync(0xffffffffu, fj[3][q], 16);
            r = k0 + __shfl_xor_sync(0xffffffffu, k1, 8);
            r += __shfl_xor_sync(0xffffffffu, r, 4);
            r += __shfl_xor_sync(0xffffffffu, r, 2);
            r += __shfl_xor_sync(0xffffffffu, r, 1);
        }
        fj[0][q] = r;
    }
    const int jl = jj + L;
    if ((lane & 7) == 0 && (FULL || jl < cnt)) {
        float* dst = jpart + ((size_t)warp * kStTile + jl) * kSsQ;
#pragma unroll
        for (int q = 0; q < kSsQ; ++q) dst[q] = fj[0][q];
    }
}

__device__ __forceinline__ void steps_sym_put(const StepSymArgs& a, int i, float ff, float fb,
                                              const float (&sum)[6]) {
    atomicMin(a.mins + i, __float_as_uint(ff));
    atomicMin(a.mins + (size_t)a.n + i, __float_as_uint(fb));
#pragma unroll
    for (int q = 0; q < 6; ++q) red_add(a.sums + (size_t)q * a.n + i, (double)sum[q]);
}

template <bool SOFT>
__global__ void __launch_bounds__(kStThreads, 1) steps_sym_kernel(const StepSymArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[kStages];
    float* jpart = reinterpret_cast<float*>(smem + kStages * kSsStage);
    const int b = blockIdx.x / (1 + a.nchunk);
    const int c = blockIdx.x % (1 + a.nchunk);
    const int ntj = (a.n + kStTile - 1) / kStTile;
    const bool diag = (c == 0);
    int t0, t1;
    if (diag) { t0 = b * kStI; t1 = min((b + 1) * kStI, ntj); }
    else { t0 = (b + 1) * kStI + (c - 1) * a.chunk; t1 = min(t0 + a.chunk, ntj); }
    if (t0 >= t1) return;                       // uniform: before any barrier
    const int ntiles = t1 - t0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i0 = b * kSsBlock;
    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) mbar_init(&bars[st], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool far_on = a.rel != nullptr && !diag;
    auto issue = [&](int t) {
        const int st = t % kStages;
        const int jt = (t0 + t) * kStTile;
        const int cnt = min(kStTile, a.n - jt);
        const int nsub = (cnt + 31) >> 5;
        unsigned char* base = smem + st * kSsStage;
        mbar_arrive_expect_tx(&bars[st], (uint32_t)cnt * 48u + (far_on ? (uint32_t)(cnt * 16 + nsub * 16) : 0u));
        bulk_g2s(base, a.rec + jt, (uint32_t)cnt * 32u, &bars[st]);
        bulk_g2s(base + kStTile * 32, a.vrec + jt, (uint32_t)cnt * 16u, &bars[st]);
        if (far_on) {
            bulk_g2s(base + kStTile * 48, a.rel + jt, (uint32_t)cnt * 16u, &bars[st]);
            bulk_g2s(base + kStTile * 64, a.sub + jt / 32, (uint32_t)nsub * 16u, &bars[st]);
        }
    };
    if (tid == 0)
        for (int t = 0; t < min(kStages, ntiles); ++t) issue(t);
    // receivers of this thread: ib + 32 u (u = 0..3); packed pair p holds u = 2p, 2p + 1
    const int ib = i0 + warp * (32 * kStI) + lane;
    StepX2I pp[kStNP];
    float2 nmi[kStNP];
    StepX2Acc acc[kStNP];
    int me[kStI];
#pragma unroll
    for (int u = 0; u < kStI; ++u) {
        const int i = min(ib + 32 * u, a.n - 1);
        me[u] = i;
        const RecMix r = a.rec[i];
        const float4 v = a.vrec[i];
        const int h = u & 1;
        StepX2I& q = pp[u >> 1];
        set_half(q.nxh, h, -r.hi.x); set_half(q.nyh, h, -r.hi.y); set_half(q.nzh, h, -r.hi.z);
        set_half(q.nxl, h, -r.lo.x); set_half(q.nyl, h, -r.lo.y); set_half(q.nzl, h, -r.lo.z);
        set_half(q.nu, h, -v.x); set_half(q.nv, h, -v.y); set_half(q.nw, h, -v.z);
        set_half(q.m, h, v.w);
        set_half(nmi[u >> 1], h, -v.w);
    }
#pragma unroll
    for (int p = 0; p < kStNP; ++p) {
        acc[p].ff = acc[p].fb = bc2(INFINITY);
        acc[p].ax = acc[p].ay = acc[p].az = acc[p].jx = acc[p].jy = acc[p].jz = bc2(0.0f);
    }
    // box of the warp's receivers (FP32 high parts), for the far-tile test
    __shared__ float wbox[kStThreads / 32][6];
    if (far_on) {
        float bl[3] = {-pp[0].nxh.x, -pp[0].nyh.x, -pp[0].nzh.x};
        float bh[3] = {bl[0], bl[1], bl[2]};
#pragma unroll
        for (int p = 0; p < kStNP; ++p) {
            bl[0] = fminf(bl[0], -fmaxf(pp[p].nxh.x, pp[p].nxh.y));
            bl[1] = fminf(bl[1], -fmaxf(pp[p].nyh.x, pp[p].nyh.y));
            bl[2] = fminf(bl[2], -fmaxf(pp[p].nzh.x, pp[p].nzh.y));
            bh[0] = fmaxf(bh[0], -fminf(pp[p].nxh.x, pp[p].nxh.y));
            bh[1] = fmaxf(bh[1], -fminf(pp[p].nyh.x, pp[p].nyh.y));
            bh[2] = fmaxf(bh[2], -fminf(pp[p].nzh.x, pp[p].nzh.y));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                bl[q] = fminf(bl[q], __shfl_xor_sync(0xffffffffu, bl[q], o));
                bh[q] = fmaxf(bh[q], __shfl_xor_sync(0xffffffffu, bh[q], o));
            }
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < 3; ++q) { wbox[warp][q] = bl[q]; wbox[warp][3 + q] = bh[q]; }
        __syncwarp();
    }
    const float2 eps2 = bc2(a.eps2);
    bool coincident = false, aborted = false;
    int t_stop = ntiles;
    for (int t = 0; t < ntiles; ++t) {
        const int st = t % kStages;
        const bool ok = mbar_wait_bounded(&bars[st], (uint32_t)((t / kStages) & 1), a.timeout_ns, a.err);
        const int jt = (t0 + t) * kStTile;
        const int cnt = min(kStTile, a.n - jt);
        const unsigned char* base = smem + st * kSsStage;
        const RecMix* rec = reinterpret_cast<const RecMix*>(base);
        const float4* vr = reinterpret_cast<const float4*>(base + kStTile * 32);
        const float4* rel_s = reinterpret_cast<const float4*>(base + kStTile * 48);
        const float4* sub_s = reinterpret_cast<const float4*>(base + kStTile * 64);
        if (diag) {
            for (int jj = 0; jj < cnt; ++jj) {
                const float4 h = rec[jj].hi, l = rec[jj].lo, v = vr[jj];
                const int j = jt + jj;
#pragma unroll
                for (int p = 0; p < kStNP; ++p)
                    step_pair_x2<true, SOFT>(h, l, v, pp[p], eps2, j == me[2 * p], j == me[2 * p + 1],
                                             acc[p], coincident);
            }
        } else {
            // blocks with tiles above them are full: every receiver is valid.  Lanes 0..7
            // test the tile's 8 sub-tiles against the warp's box (gap >= sqrt(far_k2) R)
            unsigned fmask = 0;
            if (far_on) {
                bool fr = false;
                if (lane < ((cnt + 31) >> 5)) {
                    const float4 sb = sub_s[lane];
                    const float* wb = wbox[warp];
                    const float gx = fmaxf(0.f, fmaxf(wb[0] - sb.x, sb.x - wb[3]));
                    const float gy = fmaxf(0.f, fmaxf(wb[1] - sb.y, sb.y - wb[4]));
                    const float gz = fmaxf(0.f, fmaxf(wb[2] - sb.z, sb.z - wb[5]));
                    fr = fmaf(gx, gx, fmaf(gy, gy, gz * gz)) >= a.far_k2 * (sb.w * sb.w);
                }
                fmask = __ballot_sync(0xffffffffu, fr);
            }
            float2 D[kStNP][3];
            for (int k0 = 0; k0 < cnt; k0 += 32) {
                const int jend = min(cnt, k0 + 32);
                if (jend - k0 < 32) {
                    for (int jj = k0; jj < jend; jj += 4)
                        steps_sym_group<SOFT, false, false>(jj, cnt, lane, warp, rec, vr, rel_s, D, pp, nmi, eps2, acc, jpart, coincident);
                } else if ((fmask >> (k0 >> 5)) & 1u) {
                    const float4 C = sub_s[k0 >> 5];
#pragma unroll
                    for (int p = 0; p < kStNP; ++p) {
                        D[p][0] = __fadd2_rn(__fadd2_rn(bc2(C.x), pp[p].nxh), pp[p].nxl);
                        D[p][1] = __fadd2_rn(__fadd2_rn(bc2(C.y), pp[p].nyh), pp[p].nyl);
                        D[p][2] = __fadd2_rn(__fadd2_rn(bc2(C.z), pp[p].nzh), pp[p].nzl);
                    }
                    for (int jj = k0; jj < jend; jj += 4)
                        steps_sym_group<SOFT, true, true>(jj, cnt, lane, warp, rec, vr, rel_s, D, pp, nmi, eps2, acc, jpart, coincident);
                } else {
                    for (int jj = k0; jj < jend; jj += 4)
                        steps_sym_group<SOFT, true, false>(jj, cnt, lane, warp, rec, vr, rel_s, D, pp, nmi, eps2, acc, jpart, coincident);
                }
            }
        }
        if (__syncthreads_or(!ok)) { aborted = true; t_stop = t; break; }
        if (!diag && tid < cnt) {
            float ff = INFINITY, fb = INFINITY, sum[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int w = 0; w < kStThreads / 32; ++w) {
                const float* row = jpart + ((size_t)w * kStTile + tid) * kSsQ;
                ff = fminf(ff, row[0]);
                fb = fminf(fb, row[1]);
#pragma unroll
                for (int q = 0; q < 6; ++q) sum[q] += row[2 + q];
            }
            steps_sym_put(a, jt + tid, ff, fb, sum);
        }
        __syncthreads();
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
    for (int u = 0; u < kStI; ++u) {
        const int i = ib + 32 * u;
        if (i >= a.n) continue;
        const StepX2Acc& sa = acc[u >> 1];
        const bool hi = (u & 1) != 0;
        const float sum[6] = {hi ? sa.ax.y : sa.ax.x, hi ? sa.ay.y : sa.ay.x, hi ? sa.az.y : sa.az.x,
                              hi ? sa.jx.y : sa.jx.x, hi ? sa.jy.y : sa.jy.x, hi ? sa.jz.y : sa.jz.x};
        steps_sym_put(a, i, hi ? sa.ff.y : sa.ff.x, hi ? sa.fb.y : sa.fb.x, sum);
    }
}

__global__ void steps_sym_init_kernel(int n, unsigned* mins, double* sums) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    mins[i] = mins[(size_t)n + i] = 0x7f800000u;      // +inf
#pragma unroll
    for (int q = 0; q < 6; ++q) sums[(size_t)q * n + i] = 0.0;
}

__global__ void steps_sym_finalize_kernel(int n, const unsigned* mins, const double* sums,
                                          double eta_ff, double eta_fb, double eta_jerk,
                                          double* step, int* err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float ff = __uint_as_float(mins[i]), fb = __uint_as_float(mins[(size_t)n + i]);
    float v[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) v[q] = (float)sums[(size_t)q * n + i];
    if (!(isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]))) set_error(err, FSI_ERR_NONFINITE);
    step[i] = step_from(ff, fb, v[0], v[1], v[2], v[3], v[4], v[5], eta_ff, eta_fb, eta_jerk);
}

size_t steps_sym_work_bytes(int n) { return (size_t)n * (2 * sizeof(unsigned) + 6 * sizeof(double)); }
int steps_sym_min_n() { return 4 * kSsBlock; }

// work: steps_sym_work_bytes(n) bytes, 8-byte aligned.
cudaError_t launch_steps_sym(int n, const void* rec, const void* vrec, double eps2, double eta_ff,
                             double eta_fb, double eta_jerk, void* work, double* step, int* err,
                             long long timeout_ns, int sm_count, cudaStream_t s, const void* rel,
                             const void* sub, float far_k2) {
    if (n <= 0) return cudaSuccess;
    static std::atomic<unsigned long long> attr_dev[2];
    const bool soft = eps2 > 0.0;
    {
        const cudaError_t e = soft ? smem_attr_once(steps_sym_kernel<true>, (int)kSsSmem, attr_dev[1])
                                   : smem_attr_once(steps_sym_kernel<false>, (int)kSsSmem, attr_dev[0]);
        if (e != cudaSuccess) return e;
    }
    StepSymArgs a{};
    a.n = n;
    a.rec = reinterpret_cast<const RecMix*>(rec);
    a.vrec = reinterpret_cast<const float4*>(vrec);
    a.eps2 = (float)eps2;
    a.sums = reinterpret_cast<double*>(work);
    a.mins = reinterpret_cast<unsigned*>(a.sums + 6 * (size_t)n);
    a.err = err;
    a.timeout_ns = timeout_ns;
    a.rel = reinterpret_cast<const float4*>(rel);
    a.sub = reinterpret_cast<const float4*>(sub);
    a.far_k2 = far_k2;
    const long long ntj = (n + kStTile - 1) / kStTile;
    const long long nb = (n + kSsBlock - 1) / kSsBlock;
    // about 8 items per resident CTA, at most 64 tiles each
    const long long visits = nb * ntj / 2 + 1;
    a.chunk = (int)std::max(1LL, std::min(64LL, visits / (8LL * sm_count)));
    const long long above = ntj > kStI ? ntj - kStI : 0;
    a.nchunk = (int)((above + a.chunk - 1) / a.chunk);
    const long long grid = nb * (1 + a.nchunk);
    if (grid > 2147483647LL) return cudaErrorInvalidValue;
    { steps_sym_init_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, a.mins, a.sums); note_launch(); }
    if (soft) { steps_sym_kernel<true><<<(unsigned)grid, kStThreads, kSsSmem, s>>>(a); note_launch(); }
    else { steps_sym_kernel<false><<<(unsigned)grid, kStThreads, kSsSmem, s>>>(a); note_launch(); }
    { steps_sym_finalize_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, a.mins, a.sums, eta_ff, eta_fb, eta_jerk, step, err); note_launch(); }
    return cudaGetLastError();
}

size_t steps_x2_part_bytes(int n, int sm_count, int n_i) {
    if (n_i < 0) n_i = n;
    if (n <= 0 || n_i <= 0) return 0;
    const int nb = (n_i + kStThreads * kStI - 1) / (kStThreads * kStI);
    const int want = (2 * sm_count + nb - 1) / nb;
    int split = std::max(1, std::min(want, (n + kStTile - 1) / kStTile));
    int jps = (n + split - 1) / split;
    jps = (jps + kStTile - 1) / kStTile * kStTile;
    split = (n + jps - 1) / jps;
    return split > 1 ? (size_t)split * kStPart * (size_t)n_i * sizeof(float) : 0;
}

// rec, vrec: the set's mixed position records and FP32 velocity records (vx, vy, vz, m),
// 16-byte aligned, n entries each.  part: steps_x2_part_bytes(n, sm_count) bytes.
// wide_ctas: a set whose tiled launch would run fewer CTAs takes steps_wide_kernel.
cudaError_t launch_steps_x2(int n, const void* rec, const void* vrec, double eps2, double eta_ff,
                            double eta_fb, double eta_jerk, float* part, double* step, int* err,
                            long long timeout_ns, int sm_count, int wide_ctas, cudaStream_t s,
                            int i_off, int n_i) {
    if (n_i < 0) n_i = n;
    if (n <= 0 || n_i <= 0) return cudaSuccess;
    const bool soft = eps2 > 0.0;
    {
        // tiled CTAs these receivers would get; below wide_ctas the wide form runs instead
        const long long nb = (n_i + kStThreads * kStI - 1) / (kStThreads * kStI);
        const long long want = (2LL * sm_count + nb - 1) / nb;
        const long long tiled = nb * std::max(1LL, std::min(want, (long long)(n + kStTile - 1) / kStTile));
        if (tiled < wide_ctas) {
            int lg = 5;
            while (lg > 0 && (8 << lg) > n) --lg;
            StepX2Args a{};
            a.n = n;
            a.i_off = i_off;
            a.n_i = n_i;
            a.rec = reinterpret_cast<const RecMix*>(rec);
            a.vrec = reinterpret_cast<const float4*>(vrec);
            a.eps2 = (float)eps2;
            a.eta_ff = eta_ff; a.eta_fb = eta_fb; a.eta_jerk = eta_jerk;
            a.step = step;
            a.err = err;
            const unsigned grid = (unsigned)((((long long)n_i << lg) + kStThreads - 1) / kStThreads);
            if (soft) { steps_wide_kernel<true><<<grid, kStThreads, 0, s>>>(a, lg); note_launch(); }
            else { steps_wide_kernel<false><<<grid, kStThreads, 0, s>>>(a, lg); note_launch(); }
            return cudaGetLastError();
        }
    }
    static std::atomic<unsigned long long> attr_dev[2];
    {
        const cudaError_t e = soft ? smem_attr_once(steps_x2_kernel<true>, (int)kStSmem, attr_dev[1])
                                   : smem_attr_once(steps_x2_kernel<false>, (int)kStSmem, attr_dev[0]);
        if (e != cudaSuccess) return e;
    }
    const int nb = (n_i + kStThreads * kStI - 1) / (kStThreads * kStI);
    const int want = (2 * sm_count + nb - 1) / nb;
    int split = std::max(1, std::min(want, (n + kStTile - 1) / kStTile));
    int jps = (n + split - 1) / split;
    jps = (jps + kStTile - 1) / kStTile * kStTile;
    split = (n + jps - 1) / jps;
    StepX2Args a{};
    a.n = n;
    a.i_off = i_off;
    a.n_i = n_i;
    a.rec = reinterpret_cast<const RecMix*>(rec);
    a.vrec = reinterpret_cast<const float4*>(vrec);
    a.eps2 = (float)eps2;
    a.eta_ff = eta_ff; a.eta_fb = eta_fb; a.eta_jerk = eta_jerk;
    a.j_per_split = jps;
    a.part = part;
    a.step = step;
    a.err = err;
    a.timeout_ns = timeout_ns;
    dim3 grid(nb, split);
    if (soft) { steps_x2_kernel<true><<<grid, kStThreads, kStSmem, s>>>(a); note_launch(); }
    else { steps_x2_kernel<false><<<grid, kStThreads, kStSmem, s>>>(a); note_launch(); }
    if (split > 1) { steps_x2_finalize_kernel<<<(n_i + 255) / 256, 256, 0, s>>>(a, split); note_launch(); }
    return cudaGetLastError();
}

}  // namespace fsi
