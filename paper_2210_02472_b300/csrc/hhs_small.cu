// hhs_small.cu -- the HHS recursion of a small level set inside ONE CTA.
//
// Deep HHS levels (Sect. 2.2) hold few particles but are visited 2^level times; walked
// from the host every visit costs a synchronisation and tens of launches.  Once a fast
// set F has at most kSmallMax particles, HHS(F, tau) -- time steps against F (min with
// the level-0 steps), the split S/F, U_SF(tau/6), FSI(S, tau/2), HHS(F', tau/2),
// U~_SF(2 tau/3), HHS(F', tau/2), FSI(S, tau/2), U_SF(tau/6), recursively -- runs in a
// single CTA with the set's state in shared memory and an explicit frame stack.  Thread t
// owns entry t of whichever index list a phase works on; phases are separated by
// __syncthreads.  The same arithmetic as the large kernels is used (FP64, or FP32 hi/lo
// separations with FP64 state for the mixed precision).  In the mixed precision the pass
// sums are float-float pairs (hi, lo) and reach FP64 only in the per-particle kicks: the
// B300 FP64 unit issues about 1/70 of the FP32 rate, and a pass with G lanes per receiver
// would otherwise spend G FP64 reductions on every receiver.
#include <type_traits>

#include "fsi_internal.cuh"
#include "pair_math.cuh"

namespace fsi {

constexpr int kSmallMax = 512;      // particles per set (one thread each)
constexpr int kSmallDepth = 48;     // recursion frames
constexpr int kSmallLists = kSmallMax * 40;   // index-list stack entries

struct Frame {
    int offS, nS, offF, nF;     // index lists in the list stack
    int offP, nP;               // the frame's own set
    double tau;
    int level;
    int stage;
};

// Pass sums: FP64, or float-float (hi, lo) in the mixed precision (value hi + lo).
template <int P>
using SumT = typename std::conditional<P == FSI_MIXED, float2, double>::type;

__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float2 v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ void from_f64(double& d, double v) { d = v; }
__device__ __forceinline__ void from_f64(float2& d, double v) {
    const float h = (float)v;
    d = make_float2(h, (float)(v - (double)h));
}

template <int P>
struct SmallSmem {
    double x[3][kSmallMax], v[3][kSmallMax], m[kSmallMax], s0[kSmallMax], st[kSmallMax];
    SumT<P> a[3][kSmallMax], g[3][kSmallMax];
    typename std::conditional<P == FSI_MIXED, RecMix, D4>::type rec[kSmallMax];
    typename std::conditional<P == FSI_MIXED, float4, D4>::type arec[kSmallMax];
    float4 vf[kSmallMax];                   // FP32 (vx, vy, vz, m) for the mixed time steps
    unsigned char bh[kSmallMax];            // black-hole flags (PN1.0 pairs)
    unsigned short lists[kSmallLists];      // per frame on the path: its S list then its F list
    Frame fr[kSmallDepth];
    int wsum[32];
    int top, list_top, nS, nF, anyfast;
};

template <int P>
__device__ __forceinline__ void write_rec(SmallSmem<P>& S, int k) {
    if constexpr (P == FSI_MIXED) S.rec[k] = make_mix_rec(S.x[0][k], S.x[1][k], S.x[2][k], S.m[k]);
    else S.rec[k] = make_d4(S.x[0][k], S.x[1][k], S.x[2][k], S.m[k]);
}

// After a drift: new hi/lo position splits, the mass constants kept.
template <int P>
__device__ __forceinline__ void write_rec_pos(SmallSmem<P>& S, int k) {
    if constexpr (P == FSI_MIXED) {
        RecMix r = S.rec[k];
        const float xh = (float)S.x[0][k], yh = (float)S.x[1][k], zh = (float)S.x[2][k];
        r.hi.x = xh; r.hi.y = yh; r.hi.z = zh;
        r.lo.x = (float)(S.x[0][k] - (double)xh);
        r.lo.y = (float)(S.x[1][k] - (double)yh);
        r.lo.z = (float)(S.x[2][k] - (double)zh);
        S.rec[k] = r;
    } else {
        write_rec<P>(S, k);
    }
}

// Source accelerations of a gradient pass (FP32 record in the mixed precision: the
// rounded float-float sum, no FP64 instruction).
template <int P>
__device__ __forceinline__ void write_arec(SmallSmem<P>& S, int k) {
    if constexpr (P == FSI_MIXED)
        S.arec[k] = make_float4(S.a[0][k].x + S.a[0][k].y, S.a[1][k].x + S.a[1][k].y,
                                S.a[2][k].x + S.a[2][k].y, S.vf[k].w);
    else S.arec[k] = make_d4(S.a[0][k], S.a[1][k], S.a[2][k], S.m[k]);
}

// Threads per receiver of a pass with nA receivers: the largest power of two (<= 32) that
// still fits nA groups into the CTA.  Deep levels hold few particles, so their passes are
// latency-bound; a group of G consecutive lanes splits the sources of one receiver and
// reduces its partials with a butterfly of shuffles (a fixed order).
__device__ __forceinline__ int group_size(int nA) {
    int g = 1;
    while (g < 32 && 2 * g * nA <= kSmallMax) g *= 2;
    return g;
}

// out[:, A[t]] = sum over B of the acceleration (kind 0) or gradient (kind 1) pair terms
template <int P, int KIND>
__device__ void small_pass(SmallSmem<P>& S, const unsigned short* A, int nA,
                           const unsigned short* B, int nB, double eps2, SumT<P> (*out)[kSmallMax],
                           unsigned long long* work) {
    const int t = threadIdx.x;
    if (t == 0 && work) atomicAdd(work + KIND, (unsigned long long)nA * (unsigned long long)nB);
    const int G = group_size(nA);
    const int slot = t / G, g = t % G;
    const bool active = slot < nA;
    const int k = active ? A[slot] : 0;
    if constexpr (P == FSI_MIXED) {
        // FP32 partial sums over runs of 256 sources, float-float across runs and lanes
        float sh[3] = {0.f, 0.f, 0.f}, sl[3] = {0.f, 0.f, 0.f};
        if (active) {
            const RecMix ri = S.rec[k];
            MixI p;
            p.xh = ri.hi.x; p.yh = ri.hi.y; p.zh = ri.hi.z;
            p.xl = ri.lo.x; p.yl = ri.lo.y; p.zl = ri.lo.z;
            p.ax = p.ay = p.az = 0.f;
            if (KIND == 1) { p.ax = S.arec[k].x; p.ay = S.arec[k].y; p.az = S.arec[k].z; }
            float f[3] = {0.f, 0.f, 0.f};
            const float eps2f = (float)eps2;
            int cnt = 0;
            for (int q = g; q < nB; q += G) {
                const int j = B[q];
                const RecMix rj = S.rec[j];
                if (KIND == 0) mix_acc_pair<true>(rj.hi, rj.lo, p, eps2f, j == k, f[0], f[1], f[2]);
                else mix_grad_pair<true>(rj.hi, rj.lo, S.arec[j], p, eps2f, j == k, f[0], f[1], f[2]);
                if (++cnt == 256) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) { ff_acc(sh[c], sl[c], f[c]); f[c] = 0.f; }
                    cnt = 0;
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) ff_acc(sh[c], sl[c], f[c]);
        }
        // every lane of the warp takes part in the reduction of its group
        for (int o = G >> 1; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float oh = __shfl_xor_sync(0xffffffffu, sh[c], o);
                const float ol = __shfl_xor_sync(0xffffffffu, sl[c], o);
                ff_acc(sh[c], sl[c], oh);
                sl[c] = __fadd_rn(sl[c], ol);
            }
        if (active && g == 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float h = 0.f, l = 0.f;                  // renormalised: h = fl(hi + lo)
                ff_acc(h, l, sh[c]);
                ff_acc(h, l, sl[c]);
                out[c][k] = make_float2(h, l);
            }
        }
    } else {
        double r[3] = {0.0, 0.0, 0.0};
        if (active) {
            const D4 ri = S.rec[k];
            F64I p;
            p.x = ri.x; p.y = ri.y; p.z = ri.z;
            p.ax = p.ay = p.az = 0.0;
            if (KIND == 1) { p.ax = S.arec[k].x; p.ay = S.arec[k].y; p.az = S.arec[k].z; }
            for (int q = g; q < nB; q += G) {
                const int j = B[q];
                if (KIND == 0) f64_acc_pair<true>(S.rec[j], p, eps2, j == k, r[0], r[1], r[2]);
                else f64_grad_pair<true>(S.rec[j], S.arec[j], p, eps2, j == k, r[0], r[1], r[2]);
            }
        }
        for (int o = G >> 1; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 3; ++q) r[q] += __shfl_xor_sync(0xffffffffu, r[q], o);
        if (active && g == 0) {
            out[0][k] = r[0];
            out[1][k] = r[1];
            out[2][k] = r[2];
        }
    }
}

// Time steps of list L against itself (Sect. 3.4; FP32 pair arithmetic for the mixed
// precision, FP64 otherwise), then the min with the level-0 step.
template <int P>
__device__ void small_timesteps(SmallSmem<P>& S, const unsigned short* L, int n, const SmallArgs& a) {
    using T = typename std::conditional<P == FSI_MIXED, float, double>::type;
    const int t = threadIdx.x;
    const int G = group_size(n);
    const int slot = t / G, g = t % G;
    const bool active = slot < n;
    const int i = active ? L[slot] : 0;
    bool coincident = false;
    StepAcc<T> acc;
    acc.init();
    if (active) {
        if constexpr (P == FSI_MIXED) {
            const RecMix ri = S.rec[i];
            const float4 vi = S.vf[i];
            const float eps2f = (float)a.eps2;
            for (int q = g; q < n; q += G) {
                const int j = L[q];
                if (j == i) continue;
                const RecMix rj = S.rec[j];
                const float4 vj = S.vf[j];
                const float dx = (rj.hi.x - ri.hi.x) + (rj.lo.x - ri.lo.x);
                const float dy = (rj.hi.y - ri.hi.y) + (rj.lo.y - ri.lo.y);
                const float dz = (rj.hi.z - ri.hi.z) + (rj.lo.z - ri.lo.z);
                const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (d2 == 0.f) { coincident = true; continue; }
                step_pair<float>(acc, dx, dy, dz, vj.x - vi.x, vj.y - vi.y, vj.z - vi.z, d2, vj.w,
                                 vi.w + vj.w, rsqrt_f32_refined(d2 + eps2f));
            }
        } else {
            for (int q = g; q < n; q += G) {
                const int j = L[q];
                if (j == i) continue;
                const double dx = S.x[0][j] - S.x[0][i], dy = S.x[1][j] - S.x[1][i], dz = S.x[2][j] - S.x[2][i];
                const double d2 = dx * dx + dy * dy + dz * dz;
                if (d2 == 0.0) { coincident = true; continue; }
                const double y = rsqrt_f64(d2 + a.eps2);
                step_pair<double>(acc, dx, dy, dz, S.v[0][j] - S.v[0][i], S.v[1][j] - S.v[1][i],
                                  S.v[2][j] - S.v[2][i], d2, S.m[j], S.m[i] + S.m[j], y);
            }
        }
    }
    // reduce the group: minima as (numerator, denominator) pairs, sums of a and j
    for (int o = G >> 1; o > 0; o >>= 1) {
        const T ffn = __shfl_xor_sync(0xffffffffu, acc.ffn, o), ffd = __shfl_xor_sync(0xffffffffu, acc.ffd, o);
        const T fbn = __shfl_xor_sync(0xffffffffu, acc.fbn, o), fbd = __shfl_xor_sync(0xffffffffu, acc.fbd, o);
        if (ffn * acc.ffd < acc.ffn * ffd) { acc.ffn = ffn; acc.ffd = ffd; }
        if (fbn * acc.fbd < acc.fbn * fbd) { acc.fbn = fbn; acc.fbd = fbd; }
        acc.ax += __shfl_xor_sync(0xffffffffu, acc.ax, o);
        acc.ay += __shfl_xor_sync(0xffffffffu, acc.ay, o);
        acc.az += __shfl_xor_sync(0xffffffffu, acc.az, o);
        acc.jx += __shfl_xor_sync(0xffffffffu, acc.jx, o);
        acc.jy += __shfl_xor_sync(0xffffffffu, acc.jy, o);
        acc.jz += __shfl_xor_sync(0xffffffffu, acc.jz, o);
    }
    if (coincident) set_error(a.err, FSI_ERR_NONFINITE);
    if (active && g == 0) S.st[i] = fmin(step_finish<T>(acc, a.eta_ff, a.eta_fb, a.eta_jerk), S.s0[i]);
}

// Gradient and velocity-per-acceleration steps (Sect. 3.4) of list L from its own a and
// G (in S.a, S.g): st = min(st, eta_va |v|/|a|, eta_grad (|v|/|g'|)^{1/3},
// eta_grad (|a|/|g'|)^{1/2}), g' = G / 24.
template <int P>
__device__ void small_grad_steps(SmallSmem<P>& S, const unsigned short* L, int n, const SmallArgs& a) {
    const int t = threadIdx.x;
    if (t >= n) return;
    const int k = L[t];
    double vn = 0.0, an = 0.0, gn = 0.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double gq = to_f64(S.g[q][k]) * (1.0 / 24.0);
        const double aq = to_f64(S.a[q][k]);
        vn = fma(S.v[q][k], S.v[q][k], vn);
        an = fma(aq, aq, an);
        gn = fma(gq, gq, gn);
    }
    vn = sqrt(vn);
    an = sqrt(an);
    gn = sqrt(gn);
    double e = S.st[k];
    if (a.eta_va > 0.0 && an > 0.0) e = fmin(e, a.eta_va * vn / an);
    if (a.eta_grad > 0.0 && gn > 0.0) {
        e = fmin(e, a.eta_grad * cbrt(vn / gn));
        e = fmin(e, a.eta_grad * sqrt(an / gn));
    }
    S.st[k] = e;
}

template <int P>
__device__ void small_kick(SmallSmem<P>& S, const unsigned short* L, int n, double w, bool with_grad,
                           double cg) {
    const int t = threadIdx.x;
    if (t >= n) return;
    const int k = L[t];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double ac = to_f64(S.a[c][k]);
        S.v[c][k] = fma(w, with_grad ? fma(cg, to_f64(S.g[c][k]), ac) : ac, S.v[c][k]);
    }
    if constexpr (P == FSI_MIXED) {
        float4 u = S.vf[k];                     // the mass (w) is kept
        u.x = (float)S.v[0][k]; u.y = (float)S.v[1][k]; u.z = (float)S.v[2][k];
        S.vf[k] = u;
    }
}

template <int P>
__device__ void small_drift(SmallSmem<P>& S, const unsigned short* L, int n, double w) {
    const int t = threadIdx.x;
    if (t >= n) return;
    const int k = L[t];
#pragma unroll
    for (int c = 0; c < 3; ++c) S.x[c][k] = fma(w, S.v[c][k], S.x[c][k]);
    write_rec_pos<P>(S, k);
}

// PN1.0 accelerations (into g) of list A from list B, pairs with a black hole, j != i.
template <int P>
__device__ void small_pn(SmallSmem<P>& S, const unsigned short* A, int nA, const unsigned short* B,
                         int nB, const SmallArgs& a) {
    const int t = threadIdx.x;
    if (t >= nA) return;
    const int i = A[t];
    const double ic2 = 1.0 / (a.c * a.c);
    double px = 0, py = 0, pz = 0;
    for (int q = 0; q < nB; ++q) {
        const int j = B[q];
        if (j == i || (!S.bh[i] && !S.bh[j])) continue;
        pn_pair(S.x[0][i], S.x[1][i], S.x[2][i], S.v[0][i], S.v[1][i], S.v[2][i], S.m[i], S.x[0][j],
                S.x[1][j], S.x[2][j], S.v[0][j], S.v[1][j], S.v[2][j], S.m[j], ic2, px, py, pz, a.err);
    }
    from_f64(S.g[0][i], px);
    from_f64(S.g[1][i], py);
    from_f64(S.g[2][i], pz);
}

template <int P>
__device__ void small_kick_g(SmallSmem<P>& S, const unsigned short* L, int n, double w) {
    const int t = threadIdx.x;
    if (t >= n) return;
    const int k = L[t];
#pragma unroll
    for (int c = 0; c < 3; ++c) S.v[c][k] = fma(w, to_f64(S.g[c][k]), S.v[c][k]);
    if constexpr (P == FSI_MIXED) {
        float4 u = S.vf[k];
        u.x = (float)S.v[0][k]; u.y = (float)S.v[1][k]; u.z = (float)S.v[2][k];
        S.vf[k] = u;
    }
}

// PN1.0 kick of weight w: within list L (B == nullptr) or between disjoint L and B; all PN
// accelerations from the velocities at the start of the kick (Sect. 3.9).
template <int P>
__device__ void small_pn_kick(SmallSmem<P>& S, const unsigned short* L, int n, const unsigned short* B,
                              int nB, double w, const SmallArgs& a) {
    if (!(a.c > 0.0)) return;
    if (B == nullptr) {
        small_pn<P>(S, L, n, L, n, a);
        __syncthreads();
        small_kick_g<P>(S, L, n, w);
    } else {
        small_pn<P>(S, L, n, B, nB, a);
        small_pn<P>(S, B, nB, L, n, a);
        __syncthreads();
        small_kick_g<P>(S, L, n, w);
        small_kick_g<P>(S, B, nB, w);
    }
    __syncthreads();
}

// One FSI cycle of list L on itself (Sect. 2.1, Eq. fsi-cycle), wrapped in PN1.0
// half-kicks when c > 0 (Sect. 3.9).
template <int P>
__device__ void small_fsi(SmallSmem<P>& S, const unsigned short* L, int n, double h, const SmallArgs& a) {
    small_pn_kick<P>(S, L, n, nullptr, 0, 0.5 * h, a);
    small_pass<P, 0>(S, L, n, L, n, a.eps2, S.a, a.work); __syncthreads();
    small_kick<P>(S, L, n, h / 6.0, false, 0.0); __syncthreads();
    small_drift<P>(S, L, n, 0.5 * h); __syncthreads();
    small_pass<P, 0>(S, L, n, L, n, a.eps2, S.a, a.work); __syncthreads();
    if (threadIdx.x < n) write_arec<P>(S, L[threadIdx.x]);
    __syncthreads();
    small_pass<P, 1>(S, L, n, L, n, a.eps2, S.g, a.work); __syncthreads();
    small_kick<P>(S, L, n, 2.0 * h / 3.0, true, h * h / 24.0); __syncthreads();
    small_drift<P>(S, L, n, 0.5 * h); __syncthreads();
    small_pass<P, 0>(S, L, n, L, n, a.eps2, S.a, a.work); __syncthreads();
    small_kick<P>(S, L, n, h / 6.0, false, 0.0); __syncthreads();
    small_pn_kick<P>(S, L, n, nullptr, 0, 0.5 * h, a);
}

// Inter-level kick of S and F (Sect. 2.2); gradient: the gradient acceleration of the
// same inter-level term with eps = tau.
template <int P>
__device__ void small_cross(SmallSmem<P>& S, const unsigned short* Ls, int nS,
                            const unsigned short* Lf, int nF, double w, bool gradient, double tau,
                            const SmallArgs& a) {
    small_pass<P, 0>(S, Ls, nS, Lf, nF, a.eps2, S.a, a.work);
    __syncthreads();
    small_pass<P, 0>(S, Lf, nF, Ls, nS, a.eps2, S.a, a.work);
    __syncthreads();
    if (gradient) {
        if (threadIdx.x < nS) write_arec<P>(S, Ls[threadIdx.x]);
        if (threadIdx.x < nF) write_arec<P>(S, Lf[threadIdx.x]);
        __syncthreads();
        small_pass<P, 1>(S, Ls, nS, Lf, nF, a.eps2, S.g, a.work);
        __syncthreads();
        small_pass<P, 1>(S, Lf, nF, Ls, nS, a.eps2, S.g, a.work);
        __syncthreads();
    }
    small_kick<P>(S, Ls, nS, w, gradient, tau * tau / 24.0);
    small_kick<P>(S, Lf, nF, w, gradient, tau * tau / 24.0);
    __syncthreads();
}

// Stable split of list L into S = {st >= tau} and F (all slow at max_level).
template <int P>
__device__ void small_partition(SmallSmem<P>& S, const unsigned short* L, int n, double tau,
                                bool force_slow, unsigned short* outS, unsigned short* outF) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const bool valid = t < n;
    const int k = valid ? L[t] : 0;
    const bool wants_fast = valid && S.st[k] < tau;
    const bool slow = valid && (force_slow || !wants_fast);
    const unsigned bs = __ballot_sync(0xffffffffu, slow);
    const unsigned bv = __ballot_sync(0xffffffffu, valid);
    if (lane == 0) S.wsum[wid] = __popc(bs);
    if (t == 0) S.anyfast = 0;
    __syncthreads();
    if (force_slow && wants_fast) S.anyfast = 1;
    int before = 0, total = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        if (w < wid) before += S.wsum[w];
        total += S.wsum[w];
    }
    const unsigned lm = (1u << lane) - 1u;
    const int rs = before + __popc(bs & lm);
    const int rv = t - rs;                              // valid entries before me that are fast
    (void)bv;
    if (slow) outS[rs] = (unsigned short)k;
    else if (valid) outF[rv] = (unsigned short)k;
    if (t == 0) { S.nS = total; S.nF = n - total; }
    __syncthreads();
}

template <int P>
__global__ void __launch_bounds__(kSmallMax, 1) hhs_small_kernel(const SmallArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmallSmem<P>& S = *reinterpret_cast<SmallSmem<P>*>(smem_raw);
    const int t = threadIdx.x;
    const int n = a.n;
    const long long N = a.N;
    if (t < n) {
        const int i = a.ids[t];
        for (int c = 0; c < 3; ++c) {
            S.x[c][t] = a.pos[c * N + i];
            S.v[c][t] = a.vel[c * N + i];
        }
        S.m[t] = a.mass[i];
        S.s0[t] = a.step0[i];
        write_rec<P>(S, t);
        S.vf[t] = make_float4((float)S.v[0][t], (float)S.v[1][t], (float)S.v[2][t], (float)S.m[t]);
        S.bh[t] = (a.c > 0.0 && a.is_bh) ? a.is_bh[i] : 0;
        S.lists[t] = (unsigned short)t;                 // the root's set
    }
    if (t == 0) {
        S.top = 0;
        S.list_top = n;
        Frame f;
        f.offP = 0; f.nP = n; f.tau = a.tau; f.level = a.level; f.stage = 0;
        f.offS = f.nS = f.offF = f.nF = 0;
        S.fr[0] = f;
    }
    __syncthreads();
    while (true) {
        const int top = S.top;
        if (top < 0) break;
        Frame f = S.fr[top];
        if (f.stage == 0) {
            const unsigned short* L = S.lists + f.offP;
            small_timesteps<P>(S, L, f.nP, a);
            __syncthreads();
            if (a.eta_grad > 0.0 || a.eta_va > 0.0) {
                // a and G of the level set from itself, then the gradient criteria
                small_pass<P, 0>(S, L, f.nP, L, f.nP, a.eps2, S.a, a.work);
                __syncthreads();
                if (t < f.nP) write_arec<P>(S, L[t]);
                __syncthreads();
                small_pass<P, 1>(S, L, f.nP, L, f.nP, a.eps2, S.g, a.work);
                __syncthreads();
                small_grad_steps<P>(S, L, f.nP, a);
                __syncthreads();
            }
            // S goes to [lt, lt + nS), F first to [lt + nP, ...) and is then moved down to
            // [lt + nS, lt + nP): the frame's lists take exactly nP entries.
            const int lt = S.list_top;
            const bool room = lt + 2 * f.nP <= kSmallLists;
            const bool stop = f.level >= a.max_level || !room;
            small_partition<P>(S, L, f.nP, f.tau, stop, S.lists + lt, S.lists + lt + f.nP);
            const int nS = S.nS, nF = S.nF;
            if (t < nF) S.lists[lt + nS + t] = S.lists[lt + f.nP + t];
            if (t == 0) {
                if (stop && S.anyfast) {
                    atomicExch(a.maxlevel_hit, 1);
                    if (!room) set_error(a.err, FSI_ERR_MAXLEVEL);
                }
                atomicAdd(a.level_counts + f.level, (unsigned long long)nS);
            }
            __syncthreads();
            f.offS = lt; f.nS = nS; f.offF = lt + nS; f.nF = nF;
            const unsigned short* Ls = S.lists + f.offS;
            const unsigned short* Lf = S.lists + f.offF;
            if (nS > 0 && nF > 0) {
                small_pn_kick<P>(S, Ls, nS, Lf, nF, 0.5 * f.tau, a);
                small_cross<P>(S, Ls, nS, Lf, nF, f.tau / 6.0, false, 0.0, a);
            }
            if (nS > 0) small_fsi<P>(S, Ls, nS, 0.5 * f.tau, a);
            f.stage = 1;
        } else if (f.stage == 1) {
            const unsigned short* Ls = S.lists + f.offS;
            const unsigned short* Lf = S.lists + f.offF;
            if (f.nS > 0 && f.nF > 0) small_cross<P>(S, Ls, f.nS, Lf, f.nF, 2.0 * f.tau / 3.0, true, f.tau, a);
            f.stage = 2;
        } else {
            const unsigned short* Ls = S.lists + f.offS;
            const unsigned short* Lf = S.lists + f.offF;
            if (f.nS > 0) small_fsi<P>(S, Ls, f.nS, 0.5 * f.tau, a);
            if (f.nS > 0 && f.nF > 0) {
                small_cross<P>(S, Ls, f.nS, Lf, f.nF, f.tau / 6.0, false, 0.0, a);
                small_pn_kick<P>(S, Ls, f.nS, Lf, f.nF, 0.5 * f.tau, a);
            }
            f.stage = 3;
        }
        __syncthreads();
        if (t == 0) {
            if (f.stage == 3) {
                // done: pop, and give the list space back to the parent
                S.top = top - 1;
                S.list_top = f.offS;
            } else {
                // after stage 0 and after stage 1: HHS(F, tau/2)
                S.fr[top] = f;
                S.list_top = f.offS + f.nS + f.nF;
                if (f.nF > 0) {
                    if (top + 1 < kSmallDepth) {
                        Frame c;
                        c.offP = f.offF; c.nP = f.nF; c.tau = 0.5 * f.tau; c.level = f.level + 1;
                        c.stage = 0; c.offS = c.nS = c.offF = c.nF = 0;
                        S.fr[top + 1] = c;
                        S.top = top + 1;
                    } else {
                        set_error(a.err, FSI_ERR_MAXLEVEL);
                    }
                }
            }
        }
        __syncthreads();
    }
    if (t < n) {
        const int i = a.ids[t];
        for (int c = 0; c < 3; ++c) {
            a.pos[c * N + i] = S.x[c][t];
            a.vel[c * N + i] = S.v[c][t];
        }
    }
}

size_t small_smem_bytes(int precision) {
    return precision == FSI_MIXED ? sizeof(SmallSmem<FSI_MIXED>) : sizeof(SmallSmem<FSI_FP64>);
}

int small_max() { return kSmallMax; }

cudaError_t launch_hhs_small(int precision, const SmallArgs& a, cudaStream_t s) {
    const size_t smem = small_smem_bytes(precision);
    static bool attr[2] = {false, false};
    if (!attr[precision]) {
        cudaError_t e = precision == FSI_MIXED
            ? cudaFuncSetAttribute(hhs_small_kernel<FSI_MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
            : cudaFuncSetAttribute(hhs_small_kernel<FSI_FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr[precision] = true;
    }
    if (precision == FSI_MIXED) { hhs_small_kernel<FSI_MIXED><<<1, kSmallMax, smem, s>>>(a); note_launch(); }
    else { hhs_small_kernel<FSI_FP64><<<1, kSmallMax, smem, s>>>(a); note_launch(); }
    return cudaGetLastError();
}

}  // namespace fsi
