// hhs_grid.cu -- the HHS recursion of a mid-size level set in ONE persistent launch that
// spans the GPU.
//
// Between the one-CTA recursion (sets of <= 256 particles) and the large top levels, a
// fast set of a few hundred to a few thousand particles is visited 2^level times; walked
// from the host, every visit reads the split counts back to the host and launches ~25
// kernels of a few microseconds of work each.  Here HHS(F, tau) (Sect. 2.2, Eq.
// hhsfsi-cycle) -- time steps against F, the split S/F, U_SF(tau/6), FSI(S, tau/2),
// HHS(F', tau/2), U~_SF(2 tau/3), HHS(F', tau/2), FSI(S, tau/2), U_SF(tau/6) -- runs in
// one cooperative launch of one 512-thread CTA per SM:
//   - every CTA runs the same frame stack; its decisions come from counts in global memory
//     read after a barrier, so the control flow is identical in all CTAs;
//   - each phase (time steps, split, pair pass) is spread over the CTAs, and phases are
//     separated by a grid barrier whose waits are bounded (on timeout: FSI_ERR_TIMEOUT,
//     an abort flag every CTA checks, and return);
//   - a fast set of at most small_cap particles recurses in CTA 0 with the one-CTA form
//     while the other CTAs wait at the next barrier;
//   - the state stays in the global FP64 arrays, indexed by particle id; pair passes read
//     position records (FP32 hi/lo splits, or FP64) staged chunk by chunk into shared
//     memory, and a pass whose kick is followed by a drift writes the other record buffer,
//     so the kick and the drift share one phase;
//   - every sum has a fixed order (per-lane runs, a butterfly over the lanes of a
//     receiver), so a launch is deterministic and replays bit for bit.
// A receiver's sources are split over G lanes (a power of two up to 32, the largest that
// still gives every receiver a group within the CTAs of the phase).  The two directions of
// an inter-level kick run in one phase on disjoint CTA ranges.  Data written by other CTAs
// in earlier phases is read with L1-bypassing loads.  PN1.0 kicks (pairs with a black
// hole) take two phases of their own, from black-hole sublists kept per frame.
#include <algorithm>

#include "hhs_small.cuh"

namespace fsi {

constexpr int kGridThreads = kSmallMax;     // the one-CTA recursion runs in CTA 0
constexpr int kGridDepth = 48;              // frames
constexpr int kGridChunk = 1024;            // sources per staged chunk
constexpr int kGridRun = 32;                // mixed: FP32 run length before the float-float carry

template <int P>
using GRec = typename std::conditional<P == FSI_MIXED, RecMix, D4>::type;   // position
template <int P>
using GVec = typename std::conditional<P == FSI_MIXED, float4, D4>::type;   // (a, m), (v, m)

struct GFrame {
    int offP, nP, offS, nS, offF, nF;
    int offB, nBS, nBF;             // black holes of S, then of F, at bhl[offB ...] (PN on)
    double tau;
    int level, stage;
};

// Per-CTA control state (the same in every CTA).
struct GCtl {
    GFrame fr[kGridDepth];
    long long list_top, bh_top;
    long long t_last;               // CTA 0, with a.prof: end of the previous phase
    int top, ok;
};

// Phase kinds of the optional profile (a.prof: [kind] ns, [8 + kind] phases, from CTA 0).
// The split has no barrier of its own (every CTA splits on its own), so kind 1 stays empty
// and the split's time counts toward the phase after it.
enum GPhase { kPhSteps = 0, kPhSplit, kPhCross, kPhFsi, kPhSmall, kPhCrit, kPhInit, kPhPn };

// ---------------------------------------------------------------------------------
// Loads of data other CTAs wrote (L2, not L1) and record packing.
__device__ __forceinline__ RecMix g_ld(const RecMix* p) {
    RecMix r;
    r.hi = __ldcg(&p->hi);
    r.lo = __ldcg(&p->lo);
    return r;
}
__device__ __forceinline__ D4 g_ld(const D4* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 u = __ldcg(q), w = __ldcg(q + 1);
    return make_d4(u.x, u.y, w.x, w.y);
}
__device__ __forceinline__ float4 g_ld(const float4* p) { return __ldcg(p); }

template <int P>
__device__ __forceinline__ void g_put_pos(void* buf, int i, double x, double y, double z, double m) {
    if constexpr (P == FSI_MIXED) reinterpret_cast<RecMix*>(buf)[i] = make_mix_rec(x, y, z, m);
    else reinterpret_cast<D4*>(buf)[i] = make_d4(x, y, z, m);
}
template <int P>
__device__ __forceinline__ void g_put_vec(void* buf, int i, double x, double y, double z, double m) {
    if constexpr (P == FSI_MIXED)
        reinterpret_cast<float4*>(buf)[i] = make_float4((float)x, (float)y, (float)z, (float)m);
    else reinterpret_cast<D4*>(buf)[i] = make_d4(x, y, z, m);
}

// Position and velocity records of particle i from the global state.
template <int P>
__device__ __forceinline__ void g_pack(const GridArgs& a, int i) {
    const long long N = a.s.N;
    const double m = a.s.mass[i];
    g_put_pos<P>(a.rec[0], i, __ldcg(a.s.pos + i), __ldcg(a.s.pos + N + i), __ldcg(a.s.pos + 2 * N + i), m);
    g_put_vec<P>(a.vrec, i, __ldcg(a.s.vel + i), __ldcg(a.s.vel + N + i), __ldcg(a.s.vel + 2 * N + i), m);
}

// ---------------------------------------------------------------------------------
// Grid barrier: one monotonic arrival counter per launch (zeroed before it); barrier k
// completes when the counter reaches (k + 1) * gridDim.x.  Thread 0 of each CTA arrives
// with a release add after the CTA's __syncthreads (the CTA's writes happen before it)
// and waits with acquire loads (the other CTAs' writes happen before the CTA's
// __syncthreads that follows); the wait is bounded, and a CTA that aborts never arrives,
// so the others see the abort flag or run out of time while they spin.
__device__ __forceinline__ unsigned long long ld_acq_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_rel_add_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

__device__ bool grid_sync(const GridArgs& a, unsigned long long& target, GCtl& C, int kind) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        target += gridDim.x;
        red_rel_add_u64(a.bar, 1ull);
        if (ld_acq_u64(a.bar) < target) {
            long long t0 = 0;
            for (int spins = 0;; ++spins) {
                if (ld_acq_u64(a.bar) >= target) break;
                if ((spins & 31) == 31) {
                    // every 32 polls: the abort flag and the clock
                    if (ld_acq_u64(a.bar + 1)) { ok = 0; break; }
                    const long long now = global_ns();
                    if (t0 == 0) t0 = now;
                    else if (now - t0 > a.timeout_ns) {
                        set_error(a.s.err, FSI_ERR_TIMEOUT);
                        atomicExch(a.bar + 1, 1ull);
                        ok = 0;
                        break;
                    }
                    if (spins > 4096) __nanosleep(64);
                }
            }
        }
        C.ok = ok;
        if (a.prof && blockIdx.x == 0) {
            const long long now = global_ns();
            a.prof[kind] += (unsigned long long)(now - C.t_last);
            a.prof[8 + kind] += 1ull;
            C.t_last = now;
        }
    }
    __syncthreads();
    return C.ok != 0;
}

#define GSYNC(kind)                                     \
    do {                                                \
        if (!grid_sync(a, target, C, kind)) return false; \
    } while (0)

// ---------------------------------------------------------------------------------
// Work layout of one phase: direction d of the phase runs on CTAs [cb, cb + nct), with G
// lanes per receiver.
struct GDir {
    const int* A;       // receivers (global ids)
    int nA;
    const int* B;       // sources
    int nB;
    const int* B2;      // a second source range, summed apart (acceleration passes)
    int nB2;
};

struct GLayout {
    GDir d;
    int cb, nct, G, groups, rounds;
    bool mine;          // this CTA works on d
    bool first;         // d is direction 0
};

// CTAs of direction 0 when two directions share a phase: enough for a warp per receiver
// on each side when the grid has room, else in proportion to the pair counts.
__device__ __forceinline__ GLayout g_layout(const GDir& d0, const GDir& d1) {
    const int grid = gridDim.x;
    int c0 = grid;
    if (d1.nA > 0 && d1.nB > 0) {
        if (d0.nA <= 0 || d0.nB <= 0) {
            c0 = 0;
        } else {
            const long long need0 = ((long long)d0.nA * 32 + kGridThreads - 1) / kGridThreads;
            const long long need1 = ((long long)d1.nA * 32 + kGridThreads - 1) / kGridThreads;
            if (need0 + need1 <= grid) {
                c0 = (int)need0;
            } else {
                const double w0 = (double)d0.nA * (d0.nB + d0.nB2), w1 = (double)d1.nA * (d1.nB + d1.nB2);
                c0 = (int)llround(grid * w0 / (w0 + w1));
                c0 = min(max(c0, 1), grid - 1);
            }
        }
    }
    GLayout L;
    const bool first = (int)blockIdx.x < c0;
    L.d = first ? d0 : d1;
    L.first = first;
    L.cb = first ? 0 : c0;
    L.nct = first ? c0 : grid - c0;
    L.mine = L.nct > 0 && L.d.nA > 0 && L.d.nB > 0;
    const long long Td = (long long)L.nct * kGridThreads;
    int G = 32;
    while (G > 1 && (long long)L.d.nA * G > Td) G >>= 1;
    L.G = G;
    L.groups = (int)(Td / G);
    L.rounds = L.mine ? (L.d.nA + L.groups - 1) / L.groups : 0;
    return L;
}

// What the epilogue of receiver i does with its pass sum s:
//   store:  acc[:, i] = s and the acceleration record of i (for a gradient pass);
//   out:    out[:, i] = s;
//   w != 0: kick v_i += w s (acceleration pass) or w (acc[:, i] + cg s) (gradient pass),
//           and, with a second source range, v_i += w2 s2 (before the first kick when
//           other_first, else after it); then, wd != 0, drift x_i += wd v_i and write i's
//           record into rout.
struct GEpi {
    int store;
    double* out;
    double w, cg, wd;
    const void* rin;
    void* rout;
    double w2;          // kick weight of the second source range's sum
    int other_first;    // kick by the second range's sum before the first's
};

// Shared-memory layout of a pass: a staged chunk of source records (and acceleration
// records, ids), then per local receiver of the CTA its id and its sums (up to two
// ranges), which the receiver's leader lane parks there for the epilogue.
template <int P>
struct GSm {
    static constexpr size_t acc = kGridChunk * sizeof(GRec<P>);
    static constexpr size_t id = acc + kGridChunk * sizeof(GVec<P>);
    static constexpr size_t sum = id + kGridChunk * sizeof(int);
    static constexpr size_t idx = sum + kGridThreads * 6 * sizeof(double);
    static constexpr size_t bytes = idx + kGridThreads * sizeof(int);
};

// The epilogue of receiver i, run with one receiver per lane (the B300 FP64 unit issues
// ~1/64 of the FP32 rate, so FP64 work is packed into as few warps as possible).
template <int P, int KIND>
__device__ __forceinline__ void g_epilogue(const GridArgs& a, const GEpi& e, int i, const double (&s)[3],
                                           const double* s2) {
    const long long N = a.s.N;
    const double m = a.s.mass[i];
    if (e.store) {
#pragma unroll
        for (int c = 0; c < 3; ++c) a.acc[c * N + i] = s[c];
        g_put_vec<P>(a.arec, i, s[0], s[1], s[2], m);
    }
    if (e.out) {
#pragma unroll
        for (int c = 0; c < 3; ++c) e.out[c * N + i] = s[c];
    }
    if (e.w != 0.0) {
        double v0[3], x0[3], a0[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            v0[c] = __ldcg(a.s.vel + c * N + i);
            if (e.wd != 0.0) x0[c] = __ldcg(a.s.pos + c * N + i);
            if (KIND == 1) a0[c] = __ldcg(a.acc + c * N + i);
        }
        double v[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double ac = KIND == 1 ? fma(e.cg, s[c], a0[c]) : s[c];
            if (s2 && e.other_first) v[c] = fma(e.w, ac, fma(e.w2, s2[c], v0[c]));
            else if (s2) v[c] = fma(e.w2, s2[c], fma(e.w, ac, v0[c]));
            else v[c] = fma(e.w, ac, v0[c]);
            a.s.vel[c * N + i] = v[c];
        }
        g_put_vec<P>(a.vrec, i, v[0], v[1], v[2], m);
        if (e.wd != 0.0) {
            double x[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                x[c] = fma(e.wd, v[c], x0[c]);
                a.s.pos[c * N + i] = x[c];
            }
            g_put_pos<P>(e.rout, i, x[0], x[1], x[2], m);
        }
    }
}

// One pair pass (KIND 0: acceleration, 1: gradient with the acceleration records) over
// up to two directions (epilogue e0 for direction 0, e1 for direction 1); SELF: the
// receivers are among the sources (the pair i-i is skipped).  An acceleration pass may
// give a direction a second source range, whose sum is kept apart and kicked with its own
// weight.  The leader lane of each receiver parks its sums in shared memory; the
// epilogues then run with one receiver per lane.
template <int P, int KIND, bool SELF>
__device__ void g_pass(const GridArgs& a, unsigned char* smem, const GDir& d0, const GDir& d1,
                       const GEpi& e0, const GEpi& e1) {
    const GLayout L = g_layout(d0, d1);
    if (!L.mine) return;
    const GEpi& e = L.first ? e0 : e1;
    const int t = threadIdx.x;
    if (t == 0 && blockIdx.x == L.cb && a.s.work)
        atomicAdd(a.s.work + KIND, (unsigned long long)L.d.nA * (unsigned long long)(L.d.nB + L.d.nB2));
    GRec<P>* srec = reinterpret_cast<GRec<P>*>(smem);
    GVec<P>* sacc = reinterpret_cast<GVec<P>*>(smem + kGridChunk * sizeof(GRec<P>));
    int* sid = reinterpret_cast<int*>(smem + kGridChunk * (sizeof(GRec<P>) + sizeof(GVec<P>)));
    double* ssum = reinterpret_cast<double*>(smem + GSm<P>::sum);
    int* sidx = reinterpret_cast<int*>(smem + GSm<P>::idx);
    const int G = L.G;
    const int vt = ((int)blockIdx.x - L.cb) * kGridThreads + t;
    const int g = vt & (G - 1);
    const GRec<P>* rin = reinterpret_cast<const GRec<P>*>(e.rin);
    const GVec<P>* arec = reinterpret_cast<const GVec<P>*>(a.arec);
    const int nparts = (KIND == 0 && L.d.nB2 > 0) ? 2 : 1;
    for (int r = 0; r < L.rounds; ++r) {
        const int slot0 = r * L.groups + ((int)blockIdx.x - L.cb) * (kGridThreads / G);
        if (slot0 >= L.d.nA) break;
        const int slot = r * L.groups + vt / G;
        const bool active = slot < L.d.nA;
        const int i = active ? __ldcg(L.d.A + slot) : -1;
        const bool lead = active && g == 0;
        const int lr = t / G;                                  // local receiver
        if (lead) sidx[lr] = i;
        double s[3];
        for (int part = 0; part < nparts; ++part) {
            const int* B = part ? L.d.B2 : L.d.B;
            const int nB = part ? L.d.nB2 : L.d.nB;
            if constexpr (P == FSI_MIXED) {
                MixI p{};
                if (active) {
                    const RecMix ri = g_ld(rin + i);
                    p.xh = ri.hi.x; p.yh = ri.hi.y; p.zh = ri.hi.z;
                    p.xl = ri.lo.x; p.yl = ri.lo.y; p.zl = ri.lo.z;
                    if (KIND == 1) {
                        const float4 ai = g_ld(arec + i);
                        p.ax = ai.x; p.ay = ai.y; p.az = ai.z;
                    }
                }
                const float eps2f = (float)a.s.eps2;
                float f[3] = {0.f, 0.f, 0.f}, sh[3] = {0.f, 0.f, 0.f}, sl[3] = {0.f, 0.f, 0.f};
                int cnt = 0;
                for (int q0 = 0; q0 < nB; q0 += kGridChunk) {
                    const int cn = min(kGridChunk, nB - q0);
                    __syncthreads();
                    for (int u = t; u < cn; u += kGridThreads) {
                        const int j = __ldcg(B + q0 + u);
                        srec[u] = g_ld(rin + j);
                        if (KIND == 1) sacc[u] = g_ld(arec + j);
                        if (SELF) sid[u] = j;
                    }
                    __syncthreads();
                    if (active) {
                        for (int u = g; u < cn; u += G) {
                            const RecMix rj = srec[u];
                            if (KIND == 0) mix_acc_pair<SELF>(rj.hi, rj.lo, p, eps2f, SELF && sid[u] == i, f[0], f[1], f[2]);
                            else mix_grad_pair<SELF>(rj.hi, rj.lo, sacc[u], p, eps2f, SELF && sid[u] == i, f[0], f[1], f[2]);
                            if (++cnt == kGridRun) {
#pragma unroll
                                for (int c = 0; c < 3; ++c) { ff_acc(sh[c], sl[c], f[c]); f[c] = 0.f; }
                                cnt = 0;
                            }
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) ff_acc(sh[c], sl[c], f[c]);
                for (int o = G >> 1; o > 0; o >>= 1)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float oh = __shfl_xor_sync(0xffffffffu, sh[c], o);
                        const float ol = __shfl_xor_sync(0xffffffffu, sl[c], o);
                        ff_acc(sh[c], sl[c], oh);
                        sl[c] = __fadd_rn(sl[c], ol);
                    }
#pragma unroll
                for (int c = 0; c < 3; ++c) s[c] = (double)sh[c] + (double)sl[c];
            } else {
                F64I p{};
                if (active) {
                    const D4 ri = g_ld(rin + i);
                    p.x = ri.x; p.y = ri.y; p.z = ri.z;
                    if (KIND == 1) {
                        const D4 ai = g_ld(arec + i);
                        p.ax = ai.x; p.ay = ai.y; p.az = ai.z;
                    }
                }
                double f[3] = {0.0, 0.0, 0.0};
                for (int q0 = 0; q0 < nB; q0 += kGridChunk) {
                    const int cn = min(kGridChunk, nB - q0);
                    __syncthreads();
                    for (int u = t; u < cn; u += kGridThreads) {
                        const int j = __ldcg(B + q0 + u);
                        srec[u] = g_ld(rin + j);
                        if (KIND == 1) sacc[u] = g_ld(arec + j);
                        if (SELF) sid[u] = j;
                    }
                    __syncthreads();
                    if (active) {
                        for (int u = g; u < cn; u += G) {
                            if (KIND == 0) f64_acc_pair<SELF>(srec[u], p, a.s.eps2, SELF && sid[u] == i, f[0], f[1], f[2]);
                            else f64_grad_pair<SELF>(srec[u], sacc[u], p, a.s.eps2, SELF && sid[u] == i, f[0], f[1], f[2]);
                        }
                    }
                }
                for (int o = G >> 1; o > 0; o >>= 1)
#pragma unroll
                    for (int c = 0; c < 3; ++c) f[c] += __shfl_xor_sync(0xffffffffu, f[c], o);
#pragma unroll
                for (int c = 0; c < 3; ++c) s[c] = f[c];
            }
            if (lead)
#pragma unroll
                for (int c = 0; c < 3; ++c) ssum[6 * lr + 3 * part + c] = s[c];
        }
        // epilogues, one local receiver per lane
        __syncthreads();
        const int nloc = min(kGridThreads / G, L.d.nA - slot0);
        for (int u = t; u < nloc; u += kGridThreads) {
            const double s1[3] = {ssum[6 * u], ssum[6 * u + 1], ssum[6 * u + 2]};
            g_epilogue<P, KIND>(a, e, sidx[u], s1, nparts == 2 ? ssum + 6 * u + 3 : nullptr);
        }
        __syncthreads();
    }
}

// Time steps of list L against itself (Sect. 3.4): free fall, fly-by and jerk criteria
// into st (the level-step rule is applied by the split).
template <int P>
__device__ void g_steps(const GridArgs& a, unsigned char* smem, const int* Lst, int n) {
    using T = typename std::conditional<P == FSI_MIXED, float, double>::type;
    const GDir d{Lst, n, Lst, n};
    const GLayout L = g_layout(d, GDir{nullptr, 0, nullptr, 0});
    if (!L.mine) return;
    const int t = threadIdx.x;
    GRec<P>* srec = reinterpret_cast<GRec<P>*>(smem);
    GVec<P>* svel = reinterpret_cast<GVec<P>*>(smem + kGridChunk * sizeof(GRec<P>));
    int* sid = reinterpret_cast<int*>(smem + kGridChunk * (sizeof(GRec<P>) + sizeof(GVec<P>)));
    StepAcc<T>* sst = reinterpret_cast<StepAcc<T>*>(smem + GSm<P>::sum);
    int* sidx = reinterpret_cast<int*>(smem + GSm<P>::sum + kGridThreads * sizeof(StepAcc<T>));
    const int G = L.G;
    const int vt = ((int)blockIdx.x - L.cb) * kGridThreads + t;
    const int g = vt & (G - 1);
    const GRec<P>* rin = reinterpret_cast<const GRec<P>*>(a.rec[0]);
    const GVec<P>* vin = reinterpret_cast<const GVec<P>*>(a.vrec);
    for (int r = 0; r < L.rounds; ++r) {
        if (r * L.groups + ((int)blockIdx.x - L.cb) * (kGridThreads / G) >= n) break;
        const int slot = r * L.groups + vt / G;
        const bool active = slot < n;
        const int i = active ? __ldcg(Lst + slot) : -1;
        GRec<P> ri{};
        GVec<P> vi{};
        if (active) {
            ri = g_ld(rin + i);
            vi = g_ld(vin + i);
        }
        bool coincident = false;
        StepAcc<T> acc;
        acc.init();
        for (int q0 = 0; q0 < n; q0 += kGridChunk) {
            const int cn = min(kGridChunk, n - q0);
            __syncthreads();
            for (int u = t; u < cn; u += kGridThreads) {
                const int j = __ldcg(Lst + q0 + u);
                srec[u] = g_ld(rin + j);
                svel[u] = g_ld(vin + j);
                sid[u] = j;
            }
            __syncthreads();
            if (!active) continue;
            for (int u = g; u < cn; u += G) {
                if (sid[u] == i) continue;
                const GRec<P> rj = srec[u];
                const GVec<P> vj = svel[u];
                if constexpr (P == FSI_MIXED) {
                    const float dx = (rj.hi.x - ri.hi.x) + (rj.lo.x - ri.lo.x);
                    const float dy = (rj.hi.y - ri.hi.y) + (rj.lo.y - ri.lo.y);
                    const float dz = (rj.hi.z - ri.hi.z) + (rj.lo.z - ri.lo.z);
                    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    if (d2 == 0.f) { coincident = true; continue; }
                    step_pair<float>(acc, dx, dy, dz, vj.x - vi.x, vj.y - vi.y, vj.z - vi.z, d2, vj.w,
                                     vi.w + vj.w, rsqrt_f32_refined(d2 + (float)a.s.eps2));
                } else {
                    const double dx = rj.x - ri.x, dy = rj.y - ri.y, dz = rj.z - ri.z;
                    const double d2 = dx * dx + dy * dy + dz * dz;
                    if (d2 == 0.0) { coincident = true; continue; }
                    step_pair<double>(acc, dx, dy, dz, vj.x - vi.x, vj.y - vi.y, vj.z - vi.z, d2, rj.w,
                                      ri.w + rj.w, rsqrt_f64(d2 + a.s.eps2));
                }
            }
        }
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
        if (coincident) set_error(a.s.err, FSI_ERR_COINCIDENT);
        // the FP64 finish with one receiver per lane
        const int lr = t / G;
        if (active && g == 0) {
            sst[lr] = acc;
            sidx[lr] = i;
        }
        __syncthreads();
        const int slot0 = r * L.groups + ((int)blockIdx.x - L.cb) * (kGridThreads / G);
        const int nloc = min(kGridThreads / G, n - slot0);
        for (int u = t; u < nloc; u += kGridThreads)
            a.st[sidx[u]] = step_finish<T>(sst[u], a.s.eta_ff, a.s.eta_fb, a.s.eta_jerk);
        __syncthreads();
    }
}

// Gradient and velocity-per-acceleration criteria (Sect. 3.4) of list L from its own a
// (acc) and G (aux): st = min(st, eta_va |v|/|a|, eta_grad (|v|/|g'|)^{1/3},
// eta_grad (|a|/|g'|)^{1/2}), g' = G / 24.
__device__ void g_grad_steps(const GridArgs& a, const int* Lst, int n) {
    const long long N = a.s.N;
    for (int k = blockIdx.x * kGridThreads + threadIdx.x; k < n; k += gridDim.x * kGridThreads) {
        const int i = __ldcg(Lst + k);
        double vn = 0.0, an = 0.0, gn = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double gq = __ldcg(a.aux + c * N + i) * (1.0 / 24.0);
            const double aq = __ldcg(a.acc + c * N + i);
            const double vq = __ldcg(a.s.vel + c * N + i);
            vn = fma(vq, vq, vn);
            an = fma(aq, aq, an);
            gn = fma(gq, gq, gn);
        }
        vn = sqrt(vn);
        an = sqrt(an);
        gn = sqrt(gn);
        double e = __ldcg(a.st + i);
        if (a.s.eta_va > 0.0 && an > 0.0) e = fmin(e, a.s.eta_va * vn / an);
        if (a.s.eta_grad > 0.0 && gn > 0.0) {
            e = fmin(e, a.s.eta_grad * cbrt(vn / gn));
            e = fmin(e, a.s.eta_grad * sqrt(an / gn));
        }
        a.st[i] = e;
    }
}

// Stable split of list L into S = {st >= tau} at out[0, nS) and F at out[nS, n), with
// the level-step rule (level 0 records its steps as the level-0 steps, deeper levels take
// the min with them); with PN on, also the black holes of S, then of F, in list order at
// bh[0, nBS + nBF).  Every CTA runs it and writes the same lists (no grid barrier is
// needed before a CTA reads them: the lists it reads are the ones it wrote); CTA 0 alone
// records the level-0 steps and the statistics.  With force_slow every particle stays in
// S, which is then L itself and not written (its black-hole list still is).
struct GSplit {
    int nS, nBS, nBF;
};

__device__ GSplit g_split(const GridArgs& a, const int* Lst, int n, double tau, int level,
                          bool force_slow, bool room, int* out, int* bh) {
    __shared__ int wS[kGridThreads / 32], wBS[kGridThreads / 32], wBF[kGridThreads / 32];
    __shared__ int s_base, s_bs, s_bf, s_total, s_tbs, s_tbf, s_anyfast;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const bool cta0 = blockIdx.x == 0;
    const bool pn = a.s.c > 0.0 && a.s.is_bh;
    auto step_of = [&](int i) {
        const double st = __ldcg(a.st + i);
        return level == 0 ? st : fmin(st, __ldcg(a.s.step0 + i));
    };
    if (t == 0) { s_total = 0; s_tbs = 0; s_tbf = 0; s_anyfast = 0; }
    __syncthreads();
    // pass 1: count S and the black holes of S and F (and record the level-0 steps)
    for (int k0 = 0; k0 < n; k0 += kGridThreads) {
        const int k = k0 + t;
        bool slow = false, bhk = false;
        if (k < n) {
            const int i = __ldcg(Lst + k);
            const double st = step_of(i);
            if (cta0 && level == 0 && a.step0w) a.step0w[i] = st;
            const bool fast = st < tau;
            if (fast && force_slow) s_anyfast = 1;
            slow = force_slow || !fast;
            bhk = pn && a.s.is_bh[i];
        }
        const unsigned b = __ballot_sync(0xffffffffu, slow);
        const unsigned bs = __ballot_sync(0xffffffffu, slow && bhk);
        const unsigned bf = __ballot_sync(0xffffffffu, k < n && !slow && bhk);
        if (lane == 0) {
            if (b) atomicAdd(&s_total, __popc(b));
            if (bs) atomicAdd(&s_tbs, __popc(bs));
            if (bf) atomicAdd(&s_tbf, __popc(bf));
        }
    }
    __syncthreads();
    GSplit r;
    r.nS = s_total;
    r.nBS = s_tbs;
    r.nBF = s_tbf;
    if (!force_slow || r.nBS + r.nBF > 0) {
        if (t == 0) { s_base = 0; s_bs = 0; s_bf = 0; }
        __syncthreads();
        // pass 2: S to out[0, nS) and F to out[nS, n) in list order (not when force_slow),
        // the black holes of S to bh[0, nBS) and of F to bh[nBS, nBS + nBF)
        for (int k0 = 0; k0 < n; k0 += kGridThreads) {
            const int k = k0 + t;
            const bool valid = k < n;
            const int i = valid ? __ldcg(Lst + k) : 0;
            const bool slow = valid && (force_slow || !(step_of(i) < tau));
            const bool bhk = valid && pn && a.s.is_bh[i];
            const unsigned b = __ballot_sync(0xffffffffu, slow);
            const unsigned bs = __ballot_sync(0xffffffffu, slow && bhk);
            const unsigned bf = __ballot_sync(0xffffffffu, valid && !slow && bhk);
            if (lane == 0) { wS[wid] = __popc(b); wBS[wid] = __popc(bs); wBF[wid] = __popc(bf); }
            __syncthreads();
            int before = s_base, bbs = s_bs, bbf = s_bf;
            for (int w = 0; w < wid; ++w) { before += wS[w]; bbs += wBS[w]; bbf += wBF[w]; }
            const unsigned lm = (1u << lane) - 1u;
            const int rs = before + __popc(b & lm);
            if (valid && !force_slow) {
                if (slow) out[rs] = i;
                else out[r.nS + (k - rs)] = i;          // k - rs: fast entries before k
            }
            if (bhk) {
                if (slow) bh[bbs + __popc(bs & lm)] = i;
                else bh[r.nBS + bbf + __popc(bf & lm)] = i;
            }
            __syncthreads();
            if (t == 0)
                for (int w = 0; w < kGridThreads / 32; ++w) { s_base += wS[w]; s_bs += wBS[w]; s_bf += wBF[w]; }
            __syncthreads();
        }
    }
    if (cta0 && t == 0) {
        if (a.s.level_counts) atomicAdd(a.s.level_counts + level, (unsigned long long)r.nS);
        if (force_slow && s_anyfast) {
            atomicExch(a.s.maxlevel_hit, 1);
            if (!room) set_error(a.s.err, FSI_ERR_MAXLEVEL);
        }
    }
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------------
// PN1.0 kicks (Sect. 3.9): pairs with a black hole, accelerations from the velocities at
// the start of the kick.  Phase 1 (g_pn_acc) evaluates, per direction (receivers A,
// sources B, their black-hole sublists bA, bB): a receiver that is not a black hole sums
// over bB (one receiver per lane, into aux); a black-hole receiver (k-th of bA) sums over
// all of B in chunks of kGridPnChunk sources, one warp per (k, chunk) item across the
// grid, each chunk's sum into pnpart.  Phase 2 (g_pn_kick) adds a black hole's chunk sums
// in chunk order and kicks every receiver: v += w pn.  Fixed orders throughout.
struct GPnDir {
    const int* A;
    int nA;
    const int* B;
    int nB;
    const int* bA;
    int nbA;
    const int* bB;
    int nbB;
};

__device__ __forceinline__ void g_pn_pair(const GridArgs& a, int i, const double (&xi)[3],
                                          const double (&vi)[3], double mi, int j, double ic2,
                                          double (&p)[3]) {
    const long long N = a.s.N;
    pn_pair(xi[0], xi[1], xi[2], vi[0], vi[1], vi[2], mi, __ldcg(a.s.pos + j),
            __ldcg(a.s.pos + N + j), __ldcg(a.s.pos + 2 * N + j), __ldcg(a.s.vel + j),
            __ldcg(a.s.vel + N + j), __ldcg(a.s.vel + 2 * N + j), a.s.mass[j], ic2, p[0], p[1],
            p[2], a.s.err);
}

__device__ void g_pn_acc(const GridArgs& a, const GPnDir* d, int ndir) {
    const long long N = a.s.N;
    const double ic2 = 1.0 / (a.s.c * a.s.c);
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (kGridThreads / 32) + (threadIdx.x >> 5);
    const int nw = gridDim.x * (kGridThreads / 32);
    long long part0 = 0;
    for (int q = 0; q < ndir; ++q) {
        // black-hole receivers: one warp per (black hole, chunk of sources)
        const int nch = (d[q].nB + kGridPnChunk - 1) / kGridPnChunk;
        const long long items = (long long)d[q].nbA * nch;
        if (part0 + 3 * items > a.pnpart_cap) {
            if (gw == 0 && lane == 0) set_error(a.s.err, FSI_ERR_UNSUPPORTED);
            return;
        }
        for (long long it = gw; it < items; it += nw) {
            const int k = (int)(it / nch), ch = (int)(it - (long long)k * nch);
            const int i = __ldcg(d[q].bA + k);
            double xi[3], vi[3], p[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xi[c] = __ldcg(a.s.pos + c * N + i);
                vi[c] = __ldcg(a.s.vel + c * N + i);
            }
            const double mi = a.s.mass[i];
            const int q1 = min(d[q].nB, (ch + 1) * kGridPnChunk);
            for (int u = ch * kGridPnChunk + lane; u < q1; u += 32) {
                const int j = __ldcg(d[q].B + u);
                if (j != i) g_pn_pair(a, i, xi, vi, mi, j, ic2, p);
            }
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int c = 0; c < 3; ++c) p[c] += __shfl_xor_sync(0xffffffffu, p[c], o);
            if (lane == 0)
#pragma unroll
                for (int c = 0; c < 3; ++c) a.pnpart[part0 + 3 * it + c] = p[c];
        }
        part0 += 3 * items;
        // the other receivers: one per lane, over the black holes of B
        for (int u = blockIdx.x * kGridThreads + threadIdx.x; u < d[q].nA; u += gridDim.x * kGridThreads) {
            const int i = __ldcg(d[q].A + u);
            if (a.s.is_bh[i]) continue;
            double xi[3], vi[3], p[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xi[c] = __ldcg(a.s.pos + c * N + i);
                vi[c] = __ldcg(a.s.vel + c * N + i);
            }
            const double mi = a.s.mass[i];
            for (int b = 0; b < d[q].nbB; ++b) g_pn_pair(a, i, xi, vi, mi, __ldcg(d[q].bB + b), ic2, p);
#pragma unroll
            for (int c = 0; c < 3; ++c) a.aux[c * N + i] = p[c];
        }
    }
}

template <int P>
__device__ void g_pn_kick(const GridArgs& a, const GPnDir* d, int ndir, double w) {
    const long long N = a.s.N;
    long long part0 = 0;
    for (int q = 0; q < ndir; ++q) {
        const int nch = (d[q].nB + kGridPnChunk - 1) / kGridPnChunk;
        const long long items = (long long)d[q].nbA * nch;
        if (part0 + 3 * items > a.pnpart_cap) return;
        for (int u = blockIdx.x * kGridThreads + threadIdx.x; u < d[q].nA; u += gridDim.x * kGridThreads) {
            const int i = __ldcg(d[q].A + u);
            double p[3];
            if (a.s.is_bh[i]) {
                // the k-th black hole of A: its chunk sums, in chunk order
                int k = 0;
                while (k < d[q].nbA && __ldcg(d[q].bA + k) != i) ++k;
                if (k == d[q].nbA) continue;
                p[0] = p[1] = p[2] = 0.0;
                for (int ch = 0; ch < nch; ++ch)
#pragma unroll
                    for (int c = 0; c < 3; ++c) p[c] += __ldcg(a.pnpart + part0 + 3 * ((long long)k * nch + ch) + c);
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) p[c] = __ldcg(a.aux + c * N + i);
            }
            double v[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                v[c] = fma(w, p[c], __ldcg(a.s.vel + c * N + i));
                a.s.vel[c * N + i] = v[c];
            }
            g_put_vec<P>(a.vrec, i, v[0], v[1], v[2], a.s.mass[i]);
        }
        part0 += 3 * items;
    }
}

// ---------------------------------------------------------------------------------
// Phases of a frame.  Each ends with a grid barrier; false: the launch aborts.
template <int P>
__device__ bool g_cross(const GridArgs& a, unsigned char* smem, GCtl& C, unsigned long long& target,
                        const int* Ls, int nS, const int* Lf, int nF, double w, bool gradient, double cg) {
    const GDir d0{Ls, nS, Lf, nF}, d1{Lf, nF, Ls, nS};
    if (!gradient) {
        const GEpi e{0, nullptr, w, 0.0, 0.0, a.rec[0], nullptr};
        g_pass<P, 0, false>(a, smem, d0, d1, e, e);
        GSYNC(kPhCross);
        return true;
    }
    const GEpi es{1, nullptr, 0.0, 0.0, 0.0, a.rec[0], nullptr};
    g_pass<P, 0, false>(a, smem, d0, d1, es, es);
    GSYNC(kPhCross);
    const GEpi eg{0, nullptr, w, cg, 0.0, a.rec[0], nullptr};
    g_pass<P, 1, false>(a, smem, d0, d1, eg, eg);
    GSYNC(kPhCross);
    return true;
}

// PN1.0 kick of weight w (Sect. 3.9) of the frame's S within itself, or between S and F
// (cross); nothing when no black hole is involved.
template <int P>
__device__ bool g_pn(const GridArgs& a, GCtl& C, unsigned long long& target, const GFrame& f,
                     bool cross, double w) {
    const int* Ls = a.lists + f.offS;
    const int* Lf = a.lists + f.offF;
    const int* bS = a.bhl + f.offB;
    const int* bF = bS + f.nBS;
    if (f.nBS + (cross ? f.nBF : 0) == 0) return true;
    GPnDir d[2];
    int nd = 1;
    if (cross) {
        d[0] = GPnDir{Ls, f.nS, Lf, f.nF, bS, f.nBS, bF, f.nBF};
        d[1] = GPnDir{Lf, f.nF, Ls, f.nS, bF, f.nBF, bS, f.nBS};
        nd = 2;
    } else {
        d[0] = GPnDir{Ls, f.nS, Ls, f.nS, bS, f.nBS, bS, f.nBS};
    }
    g_pn_acc(a, d, nd);
    GSYNC(kPhPn);
    g_pn_kick<P>(a, d, nd, w);
    GSYNC(kPhPn);
    return true;
}

// FSI(S, h) (Sect. 2.1, Eq. fsi-cycle) of the frame's S: kick h/6 + drift h/2, a (stored),
// gradient kick 2h/3 with a + (h^2/24) G + drift h/2, kick h/6, between PN1.0 half-kicks
// h/2 when PN is on (Sect. 3.9).  Records: rec0 -> rec1 -> rec0.  w_open != 0: the
// inter-level kick of S and F with that weight, which comes right before the cycle, shares
// its first pass; w_close != 0: the one right after the cycle shares its last pass (PN
// off only: the PN half-kicks sit between them).  S sums its F sources apart from its S
// sources and F receives from S in the same phase; the kicks are applied in the order of
// the unfused sequence.
template <int P>
__device__ bool g_fsi(const GridArgs& a, unsigned char* smem, GCtl& C, unsigned long long& target,
                      const GFrame& f, double h, double w_open, double w_close) {
    const int* Ls = a.lists + f.offS;
    const int* Lf = a.lists + f.offF;
    const int nS = f.nS, nF = f.nF;
    const bool pn = a.s.c > 0.0;
    const GDir d{Ls, nS, Ls, nS}, none{nullptr, 0, nullptr, 0};
    const GDir dSF{Ls, nS, Ls, nS, Lf, nF}, dF{Lf, nF, Ls, nS};
    const bool open = w_open != 0.0 && nF > 0, close = w_close != 0.0 && nF > 0;
    if (pn && !g_pn<P>(a, C, target, f, false, 0.5 * h)) return false;
    {
        const GEpi e{0, nullptr, h / 6.0, 0.0, 0.5 * h, a.rec[0], a.rec[1], w_open, 1};
        const GEpi ef{0, nullptr, w_open, 0.0, 0.0, a.rec[0], nullptr};
        if (open) g_pass<P, 0, true>(a, smem, dSF, dF, e, ef);
        else g_pass<P, 0, true>(a, smem, d, none, e, e);
        GSYNC(open ? kPhCross : kPhFsi);
    }
    {
        const GEpi e{1, nullptr, 0.0, 0.0, 0.0, a.rec[1], nullptr};
        g_pass<P, 0, true>(a, smem, d, none, e, e);
        GSYNC(kPhFsi);
    }
    {
        const GEpi e{0, nullptr, 2.0 * h / 3.0, h * h / 24.0, 0.5 * h, a.rec[1], a.rec[0]};
        g_pass<P, 1, true>(a, smem, d, none, e, e);
        GSYNC(kPhFsi);
    }
    {
        const GEpi e{0, nullptr, h / 6.0, 0.0, 0.0, a.rec[0], nullptr, w_close, 0};
        const GEpi ef{0, nullptr, w_close, 0.0, 0.0, a.rec[0], nullptr};
        if (close) g_pass<P, 0, true>(a, smem, dSF, dF, e, ef);
        else g_pass<P, 0, true>(a, smem, d, none, e, e);
        GSYNC(close ? kPhCross : kPhFsi);
    }
    if (pn && !g_pn<P>(a, C, target, f, false, 0.5 * h)) return false;
    return true;
}

// Stage 0 of a frame: time steps (and the gradient criteria), the split.
template <int P>
__device__ bool g_assign(const GridArgs& a, unsigned char* smem, GCtl& C, unsigned long long& target,
                         GFrame& f) {
    const int* Lst = a.lists + f.offP;
    g_steps<P>(a, smem, Lst, f.nP);
    GSYNC(kPhSteps);
    if (a.s.eta_grad > 0.0 || a.s.eta_va > 0.0) {
        const GDir d{Lst, f.nP, Lst, f.nP}, none{nullptr, 0, nullptr, 0};
        const GEpi es{1, nullptr, 0.0, 0.0, 0.0, a.rec[0], nullptr};
        g_pass<P, 0, true>(a, smem, d, none, es, es);
        GSYNC(kPhCrit);
        const GEpi eo{0, a.aux, 0.0, 0.0, 0.0, a.rec[0], nullptr};
        g_pass<P, 1, true>(a, smem, d, none, eo, eo);
        GSYNC(kPhCrit);
        g_grad_steps(a, Lst, f.nP);
        GSYNC(kPhCrit);
    }
    const long long lt = C.list_top, bt = C.bh_top;
    const bool room = lt + f.nP <= a.list_cap && bt + f.nP <= a.list_cap;
    const bool stop = f.level >= a.s.max_level || !room;
    const GSplit r = g_split(a, Lst, f.nP, f.tau, f.level, stop, room, a.lists + lt,
                             room ? a.bhl + bt : a.bhl);
    f.offS = stop ? f.offP : (int)lt;
    f.nS = r.nS;
    f.offF = f.offS + r.nS;
    f.nF = f.nP - r.nS;
    f.offB = (int)bt;
    f.nBS = room ? r.nBS : 0;
    f.nBF = room ? r.nBF : 0;
    return true;
}

template <int P>
__global__ void __launch_bounds__(kGridThreads, 1) hhs_grid_kernel(const GridArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ GCtl C;
    unsigned long long target = 0;
    const int t = threadIdx.x;
    const SmallArgs& s = a.s;
    // the root set into the list stack, its records from the state
    for (int k = blockIdx.x * kGridThreads + t; k < s.n; k += gridDim.x * kGridThreads) {
        const int i = s.ids[k];
        a.lists[k] = i;
        g_pack<P>(a, i);
    }
    if (t == 0) {
        GFrame f{};
        f.offP = 0; f.nP = s.n; f.tau = s.tau; f.level = s.level; f.stage = 0;
        C.fr[0] = f;
        C.top = 0;
        C.list_top = s.n;
        C.bh_top = 0;
        C.t_last = global_ns();
    }
    if (!grid_sync(a, target, C, kPhInit)) return;
    auto run = [&]() -> bool {
        while (true) {
            const int top = C.top;
            if (top < 0) return true;
            GFrame f = C.fr[top];
            const double tau = f.tau;
            const bool pn = s.c > 0.0;
            if (f.stage == 0) {
                if (!g_assign<P>(a, smem, C, target, f)) return false;
                const bool cross = f.nS > 0 && f.nF > 0;
                // [PN U_SF(tau/2)] U_SF(tau/6) FSI(S, tau/2): without PN the kick shares the
                // cycle's first pass
                if (cross && pn) {
                    if (!g_pn<P>(a, C, target, f, true, 0.5 * tau)) return false;
                    if (!g_cross<P>(a, smem, C, target, a.lists + f.offS, f.nS, a.lists + f.offF, f.nF,
                                    tau / 6.0, false, 0.0)) return false;
                }
                if (f.nS > 0 && !g_fsi<P>(a, smem, C, target, f, 0.5 * tau, pn ? 0.0 : tau / 6.0, 0.0))
                    return false;
                f.stage = 1;
            } else if (f.stage == 1) {
                if (f.nS > 0 && f.nF > 0 &&
                    !g_cross<P>(a, smem, C, target, a.lists + f.offS, f.nS, a.lists + f.offF, f.nF,
                                2.0 * tau / 3.0, true, tau * tau / 24.0)) return false;
                f.stage = 2;
            } else {
                // FSI(S, tau/2) U_SF(tau/6) [PN U_SF(tau/2)]: without PN the kick shares the
                // cycle's last pass
                const bool cross = f.nS > 0 && f.nF > 0;
                if (f.nS > 0 && !g_fsi<P>(a, smem, C, target, f, 0.5 * tau, 0.0, pn ? 0.0 : tau / 6.0))
                    return false;
                if (cross && pn) {
                    if (!g_cross<P>(a, smem, C, target, a.lists + f.offS, f.nS, a.lists + f.offF, f.nF,
                                    tau / 6.0, false, 0.0)) return false;
                    if (!g_pn<P>(a, C, target, f, true, 0.5 * tau)) return false;
                }
                f.stage = 3;
            }
            __syncthreads();
            if (f.stage == 3) {
                // done: pop, and give the list space back to the parent
                if (t == 0) {
                    C.top = top - 1;
                    C.list_top = f.offS;
                    C.bh_top = f.offB;
                }
                __syncthreads();
                continue;
            }
            // after stages 0 and 1: HHS(F, tau/2)
            if (t == 0) {
                C.fr[top] = f;
                C.list_top = (long long)f.offS + f.nS + f.nF;
                C.bh_top = (long long)f.offB + f.nBS + f.nBF;
            }
            __syncthreads();
            if (f.nF <= 0) continue;
            if (f.nF <= a.small_cap) {
                if (blockIdx.x == 0) {
                    SmallArgs sa = s;
                    sa.ids = a.lists + f.offF;
                    sa.n = f.nF;
                    sa.tau = 0.5 * tau;
                    sa.level = f.level + 1;
                    small_run<P>(*reinterpret_cast<SmallSmem<P>*>(smem), sa);
                    __syncthreads();
                    // the set's records from its new state
                    if (t < f.nF) g_pack<P>(a, __ldcg(a.lists + f.offF + t));
                }
                if (!grid_sync(a, target, C, kPhSmall)) return false;
            } else if (top + 1 < kGridDepth) {
                if (t == 0) {
                    GFrame ch{};
                    ch.offP = f.offF; ch.nP = f.nF; ch.tau = 0.5 * tau; ch.level = f.level + 1;
                    ch.stage = 0;
                    C.fr[top + 1] = ch;
                    C.top = top + 1;
                }
                __syncthreads();
            } else {
                if (blockIdx.x == 0 && t == 0) set_error(s.err, FSI_ERR_MAXLEVEL);
            }
        }
    };
    if (run() && a.latch_maxlevel && blockIdx.x == 0 && t == 0 && __ldcg(s.maxlevel_hit))
        set_error(s.err, FSI_ERR_MAXLEVEL);
}

#undef GSYNC

static size_t grid_smem_bytes(int precision) {
    const size_t stage = precision == FSI_MIXED
        ? std::max(GSm<FSI_MIXED>::bytes, GSm<FSI_MIXED>::sum + kGridThreads * (sizeof(StepAcc<float>) + sizeof(int)))
        : std::max(GSm<FSI_FP64>::bytes, GSm<FSI_FP64>::sum + kGridThreads * (sizeof(StepAcc<double>) + sizeof(int)));
    const size_t small = precision == FSI_MIXED ? sizeof(SmallSmem<FSI_MIXED>) : sizeof(SmallSmem<FSI_FP64>);
    return stage > small ? stage : small;
}

static cudaError_t grid_attr(int precision) {
    static std::atomic<unsigned long long> attr_dev[2];
    const int smem = (int)grid_smem_bytes(precision);
    return precision == FSI_MIXED ? smem_attr_once(hhs_grid_kernel<FSI_MIXED>, smem, attr_dev[1])
                                  : smem_attr_once(hhs_grid_kernel<FSI_FP64>, smem, attr_dev[0]);
}

int grid_ctas(int precision, int sm_count) {
    if (grid_attr(precision) != cudaSuccess) return 0;
    int per_sm = 0;
    const size_t smem = grid_smem_bytes(precision);
    const cudaError_t e = precision == FSI_MIXED
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hhs_grid_kernel<FSI_MIXED>, kGridThreads, smem)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hhs_grid_kernel<FSI_FP64>, kGridThreads, smem);
    if (e != cudaSuccess) return 0;
    return per_sm * sm_count;
}

// Cooperative launch of `ctas` CTAs (at most grid_ctas(), so that all are resident).
cudaError_t launch_hhs_grid(int precision, const GridArgs& a, int ctas, cudaStream_t s) {
    cudaError_t e = grid_attr(precision);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(kGridThreads);
    cfg.dynamicSmemBytes = grid_smem_bytes(precision);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = precision == FSI_MIXED ? cudaLaunchKernelEx(&cfg, hhs_grid_kernel<FSI_MIXED>, a)
                               : cudaLaunchKernelEx(&cfg, hhs_grid_kernel<FSI_FP64>, a);
    note_launch();
    return e;
}

}  // namespace fsi
