// hhs_small.cuh -- the HHS recursion of a small level set inside ONE CTA.
//
// Deep HHS levels (Sect. 2.2) hold few particles but are visited 2^level times; walked
// from the host every visit costs a synchronisation and tens of launches.  Once a fast
// set F has at most kSmallMax particles, HHS(F, tau) -- time steps against F (min with
// the level-0 steps), the split S/F, U_SF(tau/6), FSI(S, tau/2), HHS(F', tau/2),
// U~_SF(2 tau/3), HHS(F', tau/2), FSI(S, tau/2), U_SF(tau/6), recursively -- runs in a
// single CTA with the set's state in shared memory and an explicit frame stack.  Thread t
// owns entry t of whichever index list a phase works on; phases are separated by
// __syncthreads.  The same pair arithmetic as the large kernels is used (FP64, or FP32
// hi/lo separations for the mixed precision).  In the mixed precision the pass sums, and
// the positions and velocities themselves, are float-float pairs (hi, lo) (about 48
// significant bits) updated by FP32 operations, and the kick and drift weights are derived
// from the level's tau in float-float arithmetic: the B300 FP64 unit issues about 1/70 of
// the FP32 rate, so one FP64 warp instruction costs as much as ~70 FP32 ones, and FP64
// partial sums, kicks, drifts and weight divisions made the deep levels FP64-bound.  FP64
// remains for loading and storing the state, the time-step comparisons and PN pairs.
#pragma once
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
    double tau;                 // the level's interval (time-step comparisons)
    float2 tauf;                // the same as a float-float pair (mixed-precision weights)
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

// State (x, v) and kick / drift weights: FP64, or float-float in the mixed precision;
// gradient-kick coefficients eps^2/24: FP64 or FP32 (they scale a correction of relative
// size (eps^2/24) |G| / |a| and are rounded once).
template <int P>
using StT = SumT<P>;
template <int P>
using CgT = typename std::conditional<P == FSI_MIXED, float, double>::type;

// Float-float arithmetic on normalised pairs (|lo| <= ulp(hi) / 2), FP32 operations only:
// TwoSum (Knuth) and the FMA-based exact product, each renormalised by FastTwoSum
// (Dekker).  Relative error of one sum or product ~ 2^-47.
__device__ __forceinline__ float2 ff_norm(float h, float e) {
    const float s = __fadd_rn(h, e);
    return make_float2(s, __fsub_rn(e, __fsub_rn(s, h)));
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    const float s = __fadd_rn(a.x, b.x);
    const float bb = __fsub_rn(s, a.x);
    float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    return ff_norm(s, e);
}
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    return ff_norm(p, e);
}
// a / d for a small integer d (exact in FP32): two quotient digits and the exact remainder
__device__ __forceinline__ float2 ff_div(float2 a, float d) {
    const float q1 = __fdiv_rn(a.x, d);
    const float r = __fadd_rn(fmaf(-q1, d, a.x), a.y);
    return ff_norm(q1, __fdiv_rn(r, d));
}

// v + w a (the kick and drift updates)
__device__ __forceinline__ double axpy(double w, double a, double v) { return fma(w, a, v); }
__device__ __forceinline__ float2 axpy(float2 w, float2 a, float2 v) { return ff_add(v, ff_mul(w, a)); }
// a + c g (the gradient-kick acceleration)
__device__ __forceinline__ double grad_acc(double a, double c, double g) { return fma(c, g, a); }
__device__ __forceinline__ float2 grad_acc(float2 a, float c, float2 g) {
    return ff_add(a, make_float2(__fmul_rn(c, g.x), 0.0f));
}

// Weights from a step h: h/2, h/6, 2h/3 and the gradient coefficient h^2/24.
__device__ __forceinline__ double w_half(double h) { return 0.5 * h; }
__device__ __forceinline__ float2 w_half(float2 h) { return make_float2(0.5f * h.x, 0.5f * h.y); }
__device__ __forceinline__ double w_sixth(double h) { return h / 6.0; }
__device__ __forceinline__ float2 w_sixth(float2 h) { return ff_div(h, 6.0f); }
__device__ __forceinline__ double w_two_thirds(double h) { return 2.0 * h / 3.0; }
__device__ __forceinline__ float2 w_two_thirds(float2 h) {
    return ff_div(make_float2(2.0f * h.x, 2.0f * h.y), 3.0f);
}
__device__ __forceinline__ double w_cg(double h) { return h * h / 24.0; }
__device__ __forceinline__ float w_cg(float2 h) { return __fdiv_rn(__fmul_rn(h.x, h.x), 24.0f); }

template <int P>
__device__ __forceinline__ StT<P> frame_tau(const Frame& f) {
    if constexpr (P == FSI_MIXED) return f.tauf;
    else return f.tau;
}

template <int P>
struct SmallSmem {
    StT<P> x[3][kSmallMax], v[3][kSmallMax];
    double m[kSmallMax], s0[kSmallMax], st[kSmallMax];
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

// Position record of particle k from its state.  Mixed: the record's hi/lo splits are the
// float-float position itself; the mass constants (2.5 m, -1.5 m) are written at the load
// and kept.
template <int P>
__device__ __forceinline__ void write_rec_pos(SmallSmem<P>& S, int k) {
    if constexpr (P == FSI_MIXED) {
        RecMix r = S.rec[k];
        r.hi.x = S.x[0][k].x; r.hi.y = S.x[1][k].x; r.hi.z = S.x[2][k].x;
        r.lo.x = S.x[0][k].y; r.lo.y = S.x[1][k].y; r.lo.z = S.x[2][k].y;
        S.rec[k] = r;
    } else {
        S.rec[k] = make_d4(S.x[0][k], S.x[1][k], S.x[2][k], S.m[k]);
    }
}

// FP32 velocity record (vx, vy, vz, m) of the mixed time steps, mass kept.
template <int P>
__device__ __forceinline__ void write_vf(SmallSmem<P>& S, int k) {
    if constexpr (P == FSI_MIXED) {
        float4 u = S.vf[k];
        u.x = S.v[0][k].x; u.y = S.v[1][k].x; u.z = S.v[2][k].x;
        S.vf[k] = u;
    }
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
// What a pass does with the sum of receiver k, in its group's leader lane: store it in
// out, write k's acceleration record (an acc pass that feeds a gradient pass), and / or
// kick v_k with weight w by the sum (acc) or by a + cg G with a from S.a (gradient).
// No pass reads velocities, so a kick needs no barrier before the next pass.
template <int P>
struct PassOut {
    SumT<P> (*out)[kSmallMax];
    bool arec;
    bool kick;
    StT<P> w;
    CgT<P> cg;
};

template <int P>
__device__ __forceinline__ PassOut<P> pass_store(SumT<P> (*out)[kSmallMax], bool arec) {
    PassOut<P> o{};
    o.out = out;
    o.arec = arec;
    return o;
}

template <int P>
__device__ __forceinline__ PassOut<P> pass_kick(StT<P> w, CgT<P> cg) {
    PassOut<P> o{};
    o.kick = true;
    o.w = w;
    o.cg = cg;
    return o;
}

template <int P, int KIND>
__device__ __forceinline__ void pass_leader(SmallSmem<P>& S, int k, const SumT<P> (&sum)[3],
                                            const PassOut<P>& o) {
    if (o.out)
#pragma unroll
        for (int c = 0; c < 3; ++c) o.out[c][k] = sum[c];
    if (o.arec) {
        if constexpr (P == FSI_MIXED)
            S.arec[k] = make_float4(sum[0].x + sum[0].y, sum[1].x + sum[1].y, sum[2].x + sum[2].y, S.vf[k].w);
        else
            S.arec[k] = make_d4(sum[0], sum[1], sum[2], S.m[k]);
    }
    if (o.kick) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const SumT<P> ac = KIND == 1 ? grad_acc(S.a[c][k], o.cg, sum[c]) : sum[c];
            S.v[c][k] = axpy(o.w, ac, S.v[c][k]);
        }
        write_vf<P>(S, k);
    }
}

template <int P, int KIND>
__device__ void small_pass(SmallSmem<P>& S, const unsigned short* A, int nA,
                           const unsigned short* B, int nB, double eps2, const PassOut<P>& po,
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
            SumT<P> sum[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float h = 0.f, l = 0.f;                  // renormalised: h = fl(hi + lo)
                ff_acc(h, l, sh[c]);
                ff_acc(h, l, sl[c]);
                sum[c] = make_float2(h, l);
            }
            pass_leader<P, KIND>(S, k, sum, po);
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
            const SumT<P> sum[3] = {r[0], r[1], r[2]};
            pass_leader<P, KIND>(S, k, sum, po);
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
    if (coincident) set_error(a.err, FSI_ERR_COINCIDENT);
    if constexpr (P == FSI_MIXED) {
        // the group leaders park their FP32 sums in the pass-sum storage (free until the
        // next pass), then thread t finishes receiver t: the FP64 finish runs on n / 32 full
        // warps instead of one warp per receiver with a single active lane
        StepAcc<T>* sacc = reinterpret_cast<StepAcc<T>*>(&S.a[0][0]);
        static_assert(sizeof(StepAcc<T>) * kSmallMax <= sizeof(S.a) + sizeof(S.g), "step sums");
        if (active && g == 0) sacc[slot] = acc;
        __syncthreads();
        if (t < n) {
            const int k = L[t];
            S.st[k] = fmin(step_finish<T>(sacc[t], a.eta_ff, a.eta_fb, a.eta_jerk), S.s0[k]);
        }
    } else {
        if (active && g == 0) S.st[i] = fmin(step_finish<T>(acc, a.eta_ff, a.eta_fb, a.eta_jerk), S.s0[i]);
    }
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
        const double vq = to_f64(S.v[q][k]);
        vn = fma(vq, vq, vn);
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
__device__ void small_drift(SmallSmem<P>& S, const unsigned short* L, int n, StT<P> w) {
    const int t = threadIdx.x;
    if (t >= n) return;
    const int k = L[t];
#pragma unroll
    for (int c = 0; c < 3; ++c) S.x[c][k] = axpy(w, S.v[c][k], S.x[c][k]);
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
        pn_pair(to_f64(S.x[0][i]), to_f64(S.x[1][i]), to_f64(S.x[2][i]), to_f64(S.v[0][i]),
                to_f64(S.v[1][i]), to_f64(S.v[2][i]), S.m[i], to_f64(S.x[0][j]), to_f64(S.x[1][j]),
                to_f64(S.x[2][j]), to_f64(S.v[0][j]), to_f64(S.v[1][j]), to_f64(S.v[2][j]), S.m[j],
                ic2, px, py, pz, a.err);
    }
    from_f64(S.g[0][i], px);
    from_f64(S.g[1][i], py);
    from_f64(S.g[2][i], pz);
}

template <int P>
__device__ void small_kick_g(SmallSmem<P>& S, const unsigned short* L, int n, StT<P> w) {
    const int t = threadIdx.x;
    if (t >= n) return;
    const int k = L[t];
#pragma unroll
    for (int c = 0; c < 3; ++c) S.v[c][k] = axpy(w, S.g[c][k], S.v[c][k]);
    write_vf<P>(S, k);
}

// PN1.0 kick of weight w: within list L (B == nullptr) or between disjoint L and B; all PN
// accelerations from the velocities at the start of the kick (Sect. 3.9).
template <int P>
__device__ void small_pn_kick(SmallSmem<P>& S, const unsigned short* L, int n, const unsigned short* B,
                              int nB, StT<P> w, const SmallArgs& a) {
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
__device__ void small_fsi(SmallSmem<P>& S, const unsigned short* L, int n, StT<P> h, const SmallArgs& a) {
    const StT<P> h2 = w_half(h), h6 = w_sixth(h), h23 = w_two_thirds(h);
    const CgT<P> cg = w_cg(h);
    small_pn_kick<P>(S, L, n, nullptr, 0, h2, a);
    small_pass<P, 0>(S, L, n, L, n, a.eps2, pass_kick<P>(h6, cg), a.work); __syncthreads();
    small_drift<P>(S, L, n, h2); __syncthreads();
    small_pass<P, 0>(S, L, n, L, n, a.eps2, pass_store<P>(S.a, true), a.work); __syncthreads();
    small_pass<P, 1>(S, L, n, L, n, a.eps2, pass_kick<P>(h23, cg), a.work); __syncthreads();
    small_drift<P>(S, L, n, h2); __syncthreads();
    small_pass<P, 0>(S, L, n, L, n, a.eps2, pass_kick<P>(h6, cg), a.work); __syncthreads();
    small_pn_kick<P>(S, L, n, nullptr, 0, h2, a);
}

// Inter-level kick of S and F (Sect. 2.2); gradient: the gradient acceleration of the
// same inter-level term with eps = tau.
template <int P>
__device__ void small_cross(SmallSmem<P>& S, const unsigned short* Ls, int nS,
                            const unsigned short* Lf, int nF, StT<P> w, bool gradient, CgT<P> cg,
                            const SmallArgs& a) {
    // the two directions touch disjoint velocities and read only records: one phase each
    if (!gradient) {
        small_pass<P, 0>(S, Ls, nS, Lf, nF, a.eps2, pass_kick<P>(w, cg), a.work);
        small_pass<P, 0>(S, Lf, nF, Ls, nS, a.eps2, pass_kick<P>(w, cg), a.work);
        __syncthreads();
        return;
    }
    small_pass<P, 0>(S, Ls, nS, Lf, nF, a.eps2, pass_store<P>(S.a, true), a.work);
    small_pass<P, 0>(S, Lf, nF, Ls, nS, a.eps2, pass_store<P>(S.a, true), a.work);
    __syncthreads();
    small_pass<P, 1>(S, Ls, nS, Lf, nF, a.eps2, pass_kick<P>(w, cg), a.work);
    small_pass<P, 1>(S, Lf, nF, Ls, nS, a.eps2, pass_kick<P>(w, cg), a.work);
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
    if (slow && outS) outS[rs] = (unsigned short)k;
    else if (valid) outF[rv] = (unsigned short)k;
    if (t == 0) { S.nS = total; S.nF = n - total; }
    __syncthreads();
}

// The whole recursion HHS(a.ids, a.tau) of one set, run by all kSmallMax threads of the
// calling CTA on the state in S.  Global inputs written earlier in the same launch by
// other CTAs are read with L1-bypassing loads.
template <int P>
__device__ void small_run(SmallSmem<P>& S, const SmallArgs& a) {
    const int t = threadIdx.x;
    const int n = a.n;
    const long long N = a.N;
    if (t < n) {
        const int i = __ldcg(a.ids + t);
        for (int c = 0; c < 3; ++c) {
            from_f64(S.x[c][t], __ldcg(a.pos + c * N + i));
            from_f64(S.v[c][t], __ldcg(a.vel + c * N + i));
        }
        const double m = a.mass[i];
        S.m[t] = m;
        S.s0[t] = __ldcg(a.step0 + i);
        if constexpr (P == FSI_MIXED) {
            RecMix r;
            r.hi.w = (float)(2.5 * m);
            r.lo.w = (float)(-1.5 * m);
            S.rec[t] = r;
        }
        write_rec_pos<P>(S, t);
        S.vf[t] = make_float4((float)to_f64(S.v[0][t]), (float)to_f64(S.v[1][t]),
                              (float)to_f64(S.v[2][t]), (float)m);
        S.bh[t] = (a.c > 0.0 && a.is_bh) ? a.is_bh[i] : 0;
        S.lists[t] = (unsigned short)t;                 // the root's set
    }
    if (t == 0) {
        S.top = 0;
        S.list_top = n;
        Frame f;
        f.offP = 0; f.nP = n; f.tau = a.tau; f.level = a.level; f.stage = 0;
        from_f64(f.tauf, a.tau);
        f.offS = f.nS = f.offF = f.nF = 0;
        S.fr[0] = f;
    }
    __syncthreads();
    while (true) {
        const int top = S.top;
        if (top < 0) break;
        Frame f = S.fr[top];
        const StT<P> ft = frame_tau<P>(f);
        if (f.stage == 0) {
            const unsigned short* L = S.lists + f.offP;
            small_timesteps<P>(S, L, f.nP, a);
            __syncthreads();
            if (a.eta_grad > 0.0 || a.eta_va > 0.0) {
                // a and G of the level set from itself, then the gradient criteria
                small_pass<P, 0>(S, L, f.nP, L, f.nP, a.eps2, pass_store<P>(S.a, true), a.work);
                __syncthreads();
                small_pass<P, 1>(S, L, f.nP, L, f.nP, a.eps2, pass_store<P>(S.g, false), a.work);
                __syncthreads();
                small_grad_steps<P>(S, L, f.nP, a);
                __syncthreads();
            }
            // S goes to [lt, lt + nS), F first to [lt + nP, ...) and is then moved down to
            // [lt + nS, lt + nP): the frame's lists take exactly nP entries.  When every
            // particle stays slow (max_level, or no room left), S is the frame's own list
            // and nothing is written.
            const int lt = S.list_top;
            const bool room = lt + 2 * f.nP <= kSmallLists;
            const bool stop = f.level >= a.max_level || !room;
            small_partition<P>(S, L, f.nP, f.tau, stop, stop ? nullptr : S.lists + lt, S.lists + lt + f.nP);
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
            f.offS = stop ? f.offP : lt; f.nS = nS; f.offF = f.offS + nS; f.nF = nF;
            const unsigned short* Ls = S.lists + f.offS;
            const unsigned short* Lf = S.lists + f.offF;
            if (nS > 0 && nF > 0) {
                small_pn_kick<P>(S, Ls, nS, Lf, nF, w_half(ft), a);
                small_cross<P>(S, Ls, nS, Lf, nF, w_sixth(ft), false, w_cg(ft), a);
            }
            if (nS > 0) small_fsi<P>(S, Ls, nS, w_half(ft), a);
            f.stage = 1;
        } else if (f.stage == 1) {
            const unsigned short* Ls = S.lists + f.offS;
            const unsigned short* Lf = S.lists + f.offF;
            if (f.nS > 0 && f.nF > 0)
                small_cross<P>(S, Ls, f.nS, Lf, f.nF, w_two_thirds(ft), true, w_cg(ft), a);
            f.stage = 2;
        } else {
            const unsigned short* Ls = S.lists + f.offS;
            const unsigned short* Lf = S.lists + f.offF;
            if (f.nS > 0) small_fsi<P>(S, Ls, f.nS, w_half(ft), a);
            if (f.nS > 0 && f.nF > 0) {
                small_cross<P>(S, Ls, f.nS, Lf, f.nF, w_sixth(ft), false, w_cg(ft), a);
                small_pn_kick<P>(S, Ls, f.nS, Lf, f.nF, w_half(ft), a);
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
                        c.tauf = make_float2(0.5f * f.tauf.x, 0.5f * f.tauf.y);
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
        const int i = __ldcg(a.ids + t);
        for (int c = 0; c < 3; ++c) {
            a.pos[c * N + i] = to_f64(S.x[c][t]);
            a.vel[c * N + i] = to_f64(S.v[c][t]);
        }
    }
}


}  // namespace fsi
