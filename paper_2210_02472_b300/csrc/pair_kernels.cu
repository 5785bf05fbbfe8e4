// pair_kernels.cu -- the O(n_i * n_j) direct-summation kernels of libfsi.
//
// One kernel template covers the Newtonian acceleration (Sect. 2.1, Eq. new-newton-acc)
// and the force-gradient sum of the gradient kick (Sect. 2.1, Eq. new-grad-acc), each in
// two precisions:
//
//  FP64  : every pair term in FP64.  The reciprocal square root is seeded by the FP64
//          hardware approximation and refined in FP64 by the second-order series of
//          (1 - e)^{-1/2}:  y = y0 (1 + e/2 + 3 e^2 / 8),  e = 1 - r^2 y0^2
//          (a Householder-type step; error ~ (5/16) e^3 ~ 1e-21, below FP64 rounding).
//  MIXED : pair differences from FP32 hi/lo position splits (FP32-accurate relative to
//          the separation), FP32 pair arithmetic with one first-order residual
//          correction of the hardware rsqrt folded into r^-3 (and r^-5), FP32 partial
//          sums over runs of 32 sources, accumulated as float-float pairs (TwoSum).
//
// Work decomposition (B300: 148 SMs, 227 KB shared memory per CTA):
//  - a CTA of 256 threads owns 256*I consecutive active particles, I per thread held in
//    registers (I = 4 mixed, 2 FP64);
//  - sources stream through shared memory in tiles of 256 records, staged by
//    cp.async.bulk (TMA bulk copies) into a 3-stage ring completed by mbarriers with
//    bounded waits; every thread reads each source record as a broadcast;
//  - blockIdx.y splits the source range when the active set alone cannot fill the GPU;
//    partial sums then go to a scratch buffer and a finalize kernel applies the
//    epilogue;
//  - the epilogue (kick, drift, record rewrite, accel-record write) is fused into the
//    owner thread of particle i once its sum is complete.
//
// Self pairs are excluded by index: the tiles that can contain i (same list: the tiles
// overlapping the CTA's own i-range; general lists: every tile, by global id) run a
// checked loop variant that replaces r^2 by 1 for the self pair (whose separation is
// exactly 0, so its term vanishes).  All other tiles run the unchecked loop.
#include <algorithm>
#include <type_traits>

#include "fsi_internal.cuh"
#include "pair_math.cuh"
#include "sym_x2.cuh"

namespace fsi {

// Mass carried by a position record (mixed records hold 2.5 m in FP32).
template <int P>
__device__ __forceinline__ double record_mass(const void* rec, int i) {
    if constexpr (P == FSI_MIXED) return 0.4 * (double)reinterpret_cast<const RecMix*>(rec)[i].hi.w;
    else return reinterpret_cast<const D4*>(rec)[i].w;
}

// ---------------------------------------------------------------------------------
// Error path of a pass result that is not finite.  Without softening, two distinct
// particles at the same position (a zero separation in the pass's records) make their pair
// term 0 x inf; that case is reported as FSI_ERR_COINCIDENT, every other one (FP32
// overflow of r^-3 in the mixed precision, a non-finite input) as FSI_ERR_NONFINITE.  Only
// the receiver that claims the empty error word scans the pass's sources for a coincident
// partner (the first error of a launch wins), so a launch pays one O(n_j) scan on this
// path and nothing while its results are finite.  Self pairs are recognised as the pass
// excludes them: by index (same list), by global id or key (id lists), never (disjoint).
template <int P>
__device__ __noinline__ void report_nonfinite(const PairArgs& a, int i) {
    if (!a.err || atomicCAS(a.err, 0, FSI_ERR_NONFINITE) != 0) return;
    if (a.eps2 != 0.0 || !a.irec || !a.jrec) return;
    bool hit = false;
    for (int j = 0; j < a.n_j && !hit; ++j) {
        if (a.check == CHECK_DIAG && j == i + a.i_off) continue;
        if (a.check == CHECK_IDS && a.jid[j] == a.iid[i]) continue;
        if constexpr (P == FSI_MIXED) {
            const RecMix ri = reinterpret_cast<const RecMix*>(a.irec)[i];
            const RecMix rj = reinterpret_cast<const RecMix*>(a.jrec)[j];
            hit = rj.hi.x == ri.hi.x && rj.hi.y == ri.hi.y && rj.hi.z == ri.hi.z &&
                  rj.lo.x == ri.lo.x && rj.lo.y == ri.lo.y && rj.lo.z == ri.lo.z;
        } else {
            const D4 ri = reinterpret_cast<const D4*>(a.irec)[i];
            const D4 rj = reinterpret_cast<const D4*>(a.jrec)[j];
            hit = rj.x == ri.x && rj.y == ri.y && rj.z == ri.z;
        }
    }
    if (hit) atomicCAS(a.err, FSI_ERR_NONFINITE, FSI_ERR_COINCIDENT);
}

// Epilogue shared by the pair kernel (split == 1), the wide kernel and the finalize
// kernel, for receiver i of the pass a with pair sums (rx, ry, rz).
template <int P>
__device__ __forceinline__ void epilogue(const PairArgs& a, int i, double rx, double ry, double rz) {
    const Epi& e = a.epi;
    const int n = a.n_i;
    if (!(isfinite(rx) && isfinite(ry) && isfinite(rz))) report_nonfinite<P>(a, i);
    if (e.out) {
        e.out[i] = rx;
        e.out[(size_t)n + i] = ry;
        e.out[2 * (size_t)n + i] = rz;
    }
    // state entry of particle i: compact (row length n) or global through the id list
    const size_t gi = e.ids ? (size_t)e.ids[i] : (size_t)i;
    const size_t L = e.ids ? (size_t)e.ld : (size_t)n;
    if (e.accrec) {   // accel record (ax, ay, az, m): the mass feeds the symmetric gradient
        const double m = e.mc ? e.mc[gi] : record_mass<P>(a.irec, i);
        if (P == FSI_MIXED)
            reinterpret_cast<float4*>(e.accrec)[i] = make_float4((float)rx, (float)ry, (float)rz, (float)m);
        else
            reinterpret_cast<D4*>(e.accrec)[i] = make_d4(rx, ry, rz, m);
    }
    if (e.v) {
        double kx = rx, ky = ry, kz = rz;
        if (e.base) {
            kx = fma(e.c_grad, rx, e.base[i]);
            ky = fma(e.c_grad, ry, e.base[(size_t)n + i]);
            kz = fma(e.c_grad, rz, e.base[2 * (size_t)n + i]);
        }
        const double vx = fma(e.c_kick, kx, e.v[gi]);
        const double vy = fma(e.c_kick, ky, e.v[L + gi]);
        const double vz = fma(e.c_kick, kz, e.v[2 * L + gi]);
        e.v[gi] = vx;
        e.v[L + gi] = vy;
        e.v[2 * L + gi] = vz;
        if (e.x && e.c_drift != 0.0) {
            const double x = fma(e.c_drift, vx, e.x[gi]);
            const double y = fma(e.c_drift, vy, e.x[L + gi]);
            const double z = fma(e.c_drift, vz, e.x[2 * L + gi]);
            e.x[gi] = x;
            e.x[L + gi] = y;
            e.x[2 * L + gi] = z;
            if (e.rec_out) {
                if constexpr (P == FSI_MIXED)
                    reinterpret_cast<RecMix*>(e.rec_out)[i] = make_mix_rec(x, y, z, e.mc[gi]);
                else
                    reinterpret_cast<D4*>(e.rec_out)[i] = make_d4(x, y, z, e.mc[gi]);
            }
        }
    }
}

// ---------------------------------------------------------------------------------
template <int P, int KIND>
struct Cfg {
    static constexpr int ACCREC = KIND == KIND_ACC ? 0 : (P == FSI_MIXED ? 16 : 32);
};

constexpr int kRec = 32;

// The FP32 partial sums of a receiver in the mixed pair kernels (one-sided, wide, packed
// symmetric and bipartite forms) run over at most kSymFlushJ sources before they are added
// into a float-float accumulator (TwoSum).  A linear FP32 sum of k terms carries up to
// ~sqrt(k) roundings of its running value, so runs of 256 sources left the sum, not the
// pair terms, as the largest part of the acceleration error (median 4e-8, 99th percentile
// 3e-7 of |a| at N = 65536); runs of 32 bring it down to about the pair terms' own
// rounding (median 2.2e-8, 99th percentile 1.4e-7).
constexpr int kSymFlushJ = 32;

__host__ __device__ constexpr int stage_bytes(int accrec) { return kTileJ * (kRec + accrec + 4); }

// P: precision; KIND: acc or grad; I: active particles per thread; FF (mixed only): 0 and 1
// = scalar FP32 pair arithmetic (identical since both carry float-float sums over runs of
// kSymFlushJ sources; 1 is kept as a tuning-table entry); 2 = the tiles without the self
// pair run packed FP32x2 arithmetic on pairs of active particles (I even).  No FP64
// instruction in the loop (the B300 FP64 pipe runs at ~1/64 of the FP32 rate).
template <int P, int KIND, int I, int FF>
__global__ void __launch_bounds__(kThreads, (I <= 2 ? 3 : 2)) pair_kernel(const PairArgs a) {
    constexpr int ACCREC = Cfg<P, KIND>::ACCREC;
    constexpr int SB = stage_bytes(ACCREC);
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[kStages];

    const int tid = threadIdx.x;
    const int i0 = blockIdx.x * (kThreads * I);
    const int js = blockIdx.y * a.j_per_split;
    const int je = min(a.n_j, js + a.j_per_split);
    const int nj = max(0, je - js);
    const int ntiles = (nj + kTileJ - 1) / kTileJ;
    const bool use_ids = (a.check == CHECK_IDS);

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int t) {
        const int s = t % kStages;
        const int jt = js + t * kTileJ;
        const int cnt = min(kTileJ, je - jt);
        unsigned char* base = smem + s * SB;
        const uint32_t idb = use_ids ? (uint32_t)((cnt + 3) & ~3) * 4u : 0u;
        mbar_arrive_expect_tx(&bars[s], (uint32_t)cnt * (kRec + ACCREC) + idb);
        bulk_g2s(base, (const unsigned char*)a.jrec + (size_t)jt * kRec, (uint32_t)cnt * kRec, &bars[s]);
        if (ACCREC)
            bulk_g2s(base + kTileJ * kRec, (const unsigned char*)a.jacc + (size_t)jt * ACCREC,
                     (uint32_t)cnt * ACCREC, &bars[s]);
        if (use_ids) bulk_g2s(base + kTileJ * (kRec + ACCREC), a.jid + jt, idb, &bars[s]);
    };
    if (tid == 0)
        for (int t = 0; t < min(kStages, ntiles); ++t) issue(t);

    // ---- i-side registers
    int my_id[I];
    double acc64[I][3];
#pragma unroll
    for (int u = 0; u < I; ++u) {
        acc64[u][0] = acc64[u][1] = acc64[u][2] = 0.0;
        const int i = min(i0 + u * kThreads + tid, max(a.n_i - 1, 0));
        my_id[u] = use_ids ? a.iid[i] : (i0 + a.i_off + u * kThreads + tid);
    }

    bool aborted = false;
    int t_stop = ntiles;       // first tile not consumed (on abort)
    if constexpr (P == FSI_MIXED) {
        MixI pi[I];
        float f[I][3];
        float hi[I][3], lo[I][3];   // float-float running sums (FF variant)
        constexpr int NP = (FF == 2) ? I / 2 : 1;
        X2I pp[NP];                 // packed pairs of active particles (FF == 2)
        float2 f2[NP][3];
#pragma unroll
        for (int u = 0; u < I; ++u) {
            const int i = min(i0 + u * kThreads + tid, max(a.n_i - 1, 0));
            const RecMix r = reinterpret_cast<const RecMix*>(a.irec)[i];
            pi[u].xh = r.hi.x; pi[u].yh = r.hi.y; pi[u].zh = r.hi.z;
            pi[u].xl = r.lo.x; pi[u].yl = r.lo.y; pi[u].zl = r.lo.z;
            if constexpr (KIND == KIND_GRAD) {
                const float4 ai = reinterpret_cast<const float4*>(a.iacc)[i];
                pi[u].ax = ai.x; pi[u].ay = ai.y; pi[u].az = ai.z;
            } else {
                pi[u].ax = pi[u].ay = pi[u].az = 0.f;
            }
            f[u][0] = f[u][1] = f[u][2] = 0.f;
#pragma unroll
            for (int q = 0; q < 3; ++q) hi[u][q] = lo[u][q] = 0.f;
            if constexpr (FF == 2) {
                X2I& q = pp[u >> 1];
                const int h = u & 1;
                set_half(q.nxh, h, -pi[u].xh); set_half(q.nyh, h, -pi[u].yh); set_half(q.nzh, h, -pi[u].zh);
                set_half(q.nxl, h, -pi[u].xl); set_half(q.nyl, h, -pi[u].yl); set_half(q.nzl, h, -pi[u].zl);
                set_half(q.nax, h, -pi[u].ax); set_half(q.nay, h, -pi[u].ay); set_half(q.naz, h, -pi[u].az);
            }
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) f2[p][0] = f2[p][1] = f2[p][2] = make_float2(0.f, 0.f);
        const float2 eps2x = bc2((float)a.eps2);
        const float eps2f = (float)a.eps2;
        // every kSymFlushJ sources: the FP32 partials (packed halves first) go into the
        // float-float running sums by Knuth's TwoSum (hi + f = sum + e exactly)
        auto flush = [&]() {
            if constexpr (FF == 2) {
#pragma unroll
                for (int p = 0; p < NP; ++p)
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        f[2 * p][q] += f2[p][q].x;
                        f[2 * p + 1][q] += f2[p][q].y;
                        f2[p][q] = make_float2(0.f, 0.f);
                    }
            }
#pragma unroll
            for (int u = 0; u < I; ++u)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float sum = hi[u][q] + f[u][q];
                    const float bb = sum - hi[u][q];
                    const float e = (hi[u][q] - (sum - bb)) + (f[u][q] - bb);
                    hi[u][q] = sum;
                    lo[u][q] += e;
                    f[u][q] = 0.f;
                }
        };
        for (int t = 0; t < ntiles; ++t) {
            const int s = t % kStages;
            const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((t / kStages) & 1), a.timeout_ns, a.err);
            const int jt = js + t * kTileJ;
            const int cnt = min(kTileJ, je - jt);
            const unsigned char* base = smem + s * SB;
            const RecMix* rec = reinterpret_cast<const RecMix*>(base);
            const float4* arec = reinterpret_cast<const float4*>(base + kTileJ * kRec);
            const int* jidt = reinterpret_cast<const int*>(base + kTileJ * (kRec + ACCREC));
            const bool chk = use_ids || (a.check == CHECK_DIAG && jt < i0 + a.i_off + kThreads * I && jt + cnt > i0 + a.i_off);
            if (FF == 2 && !chk) {
                for (int jj = 0; jj < cnt; ++jj) {
                    if constexpr (KIND == KIND_ACC) {
#pragma unroll
                        for (int p = 0; p < NP; ++p) x2_acc_one(rec[jj].hi, rec[jj].lo, pp[p], eps2x, f2[p]);
                    } else {
                        const float4 aj = arec[jj];
#pragma unroll
                        for (int p = 0; p < NP; ++p) x2_grad_one(rec[jj].hi, rec[jj].lo, aj, pp[p], eps2x, f2[p]);
                    }
                    if (((jj + 1) & (kSymFlushJ - 1)) == 0 || jj == cnt - 1) flush();
                }
            } else if (!chk) {
#pragma unroll 2
                for (int jj = 0; jj < cnt; ++jj) {
                    const float4 h = rec[jj].hi;
                    const float4 l = rec[jj].lo;
                    if constexpr (KIND == KIND_ACC) {
#pragma unroll
                        for (int u = 0; u < I; ++u)
                            mix_acc_pair<false>(h, l, pi[u], eps2f, false, f[u][0], f[u][1], f[u][2]);
                    } else {
                        const float4 aj = arec[jj];
#pragma unroll
                        for (int u = 0; u < I; ++u)
                            mix_grad_pair<false>(h, l, aj, pi[u], eps2f, false, f[u][0], f[u][1], f[u][2]);
                    }
                    if (((jj + 1) & (kSymFlushJ - 1)) == 0 || jj == cnt - 1) flush();
                }
            } else {
                for (int jj = 0; jj < cnt; ++jj) {
                    const float4 h = rec[jj].hi;
                    const float4 l = rec[jj].lo;
                    const int jid = use_ids ? jidt[jj] : jt + jj;
                    if constexpr (KIND == KIND_ACC) {
#pragma unroll
                        for (int u = 0; u < I; ++u)
                            mix_acc_pair<true>(h, l, pi[u], eps2f, jid == my_id[u], f[u][0], f[u][1], f[u][2]);
                    } else {
                        const float4 aj = arec[jj];
#pragma unroll
                        for (int u = 0; u < I; ++u)
                            mix_grad_pair<true>(h, l, aj, pi[u], eps2f, jid == my_id[u], f[u][0], f[u][1], f[u][2]);
                    }
                    if (((jj + 1) & (kSymFlushJ - 1)) == 0 || jj == cnt - 1) flush();
                }
            }
            if (__syncthreads_or(!ok)) { aborted = true; t_stop = t; break; }
            if (tid == 0 && t + kStages < ntiles) issue(t + kStages);
        }
#pragma unroll
        for (int u = 0; u < I; ++u)
#pragma unroll
            for (int q = 0; q < 3; ++q) acc64[u][q] = (double)hi[u][q] + (double)lo[u][q];
    } else {
        F64I pi[I];
#pragma unroll
        for (int u = 0; u < I; ++u) {
            const int i = min(i0 + u * kThreads + tid, max(a.n_i - 1, 0));
            const D4 r = reinterpret_cast<const D4*>(a.irec)[i];
            pi[u].x = r.x; pi[u].y = r.y; pi[u].z = r.z;
            if constexpr (KIND == KIND_GRAD) {
                const D4 ai = reinterpret_cast<const D4*>(a.iacc)[i];
                pi[u].ax = ai.x; pi[u].ay = ai.y; pi[u].az = ai.z;
            } else {
                pi[u].ax = pi[u].ay = pi[u].az = 0.0;
            }
        }
        for (int t = 0; t < ntiles; ++t) {
            const int s = t % kStages;
            const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((t / kStages) & 1), a.timeout_ns, a.err);
            const int jt = js + t * kTileJ;
            const int cnt = min(kTileJ, je - jt);
            const unsigned char* base = smem + s * SB;
            const D4* rec = reinterpret_cast<const D4*>(base);
            const D4* arec = reinterpret_cast<const D4*>(base + kTileJ * kRec);
            const int* jidt = reinterpret_cast<const int*>(base + kTileJ * (kRec + ACCREC));
            const bool chk = use_ids || (a.check == CHECK_DIAG && jt < i0 + a.i_off + kThreads * I && jt + cnt > i0 + a.i_off);
            if (!chk) {
#pragma unroll 2
                for (int jj = 0; jj < cnt; ++jj) {
                    const D4 r = rec[jj];
                    if constexpr (KIND == KIND_ACC) {
#pragma unroll
                        for (int u = 0; u < I; ++u)
                            f64_acc_pair<false>(r, pi[u], a.eps2, false, acc64[u][0], acc64[u][1], acc64[u][2]);
                    } else {
                        const D4 aj = arec[jj];
#pragma unroll
                        for (int u = 0; u < I; ++u)
                            f64_grad_pair<false>(r, aj, pi[u], a.eps2, false, acc64[u][0], acc64[u][1], acc64[u][2]);
                    }
                }
            } else {
                for (int jj = 0; jj < cnt; ++jj) {
                    const D4 r = rec[jj];
                    const int jid = use_ids ? jidt[jj] : jt + jj;
                    if constexpr (KIND == KIND_ACC) {
#pragma unroll
                        for (int u = 0; u < I; ++u)
                            f64_acc_pair<true>(r, pi[u], a.eps2, jid == my_id[u], acc64[u][0], acc64[u][1], acc64[u][2]);
                    } else {
                        const D4 aj = arec[jj];
#pragma unroll
                        for (int u = 0; u < I; ++u)
                            f64_grad_pair<true>(r, aj, pi[u], a.eps2, jid == my_id[u], acc64[u][0], acc64[u][1], acc64[u][2]);
                    }
                }
            }
            if (__syncthreads_or(!ok)) { aborted = true; t_stop = t; break; }
            if (tid == 0 && t + kStages < ntiles) issue(t + kStages);
        }
    }

    if (aborted) {
        // Tiles [t_stop, issued) were issued but not consumed: let each of those copies
        // land (bounded) before the CTA's shared memory is released.
        if (tid == 0) {
            const int issued = min(ntiles, t_stop + kStages);
            for (int t = t_stop; t < issued; ++t)
                mbar_wait_bounded(&bars[t % kStages], (uint32_t)((t / kStages) & 1),
                                  a.timeout_ns, nullptr);
        }
        __syncthreads();
        if (!a.err) {
            // no error word to latch (allocation-free entry point): the CTA's results
            // become quiet NaN, so the abort shows in the outputs (through the finalize
            // sum when the sources are split)
            const double qnan = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
            for (int u = 0; u < I; ++u) {
                const int i = i0 + u * kThreads + tid;
                if (i >= a.n_i) continue;
                double* o = gridDim.y > 1 ? a.part + (size_t)blockIdx.y * 3 * a.n_i : a.epi.out;
                if (!o) continue;
                o[i] = qnan;
                o[(size_t)a.n_i + i] = qnan;
                o[2 * (size_t)a.n_i + i] = qnan;
            }
        }
        return;
    }

#pragma unroll
    for (int u = 0; u < I; ++u) {
        const int i = i0 + u * kThreads + tid;
        if (i >= a.n_i) continue;
        if (gridDim.y > 1) {
            double* p = a.part + (size_t)blockIdx.y * 3 * a.n_i;
            p[i] = acc64[u][0];
            p[(size_t)a.n_i + i] = acc64[u][1];
            p[2 * (size_t)a.n_i + i] = acc64[u][2];
        } else {
            epilogue<P>(a, i, acc64[u][0], acc64[u][1], acc64[u][2]);
        }
    }
}

// Sums the split partials in a fixed order (deterministic) and applies the epilogue.
template <int P>
__global__ void finalize_kernel(const PairArgs a, int split) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_i) return;
    double r[3] = {0.0, 0.0, 0.0};
    for (int y = 0; y < split; ++y) {
        const double* p = a.part + (size_t)y * 3 * a.n_i;
        r[0] += p[i];
        r[1] += p[(size_t)a.n_i + i];
        r[2] += p[2 * (size_t)a.n_i + i];
    }
    epilogue<P>(a, i, r[0], r[1], r[2]);
}

// =================================================================================
// Wide one-sided kernel: passes too small for the tiled form to fill the GPU (the deep
// HHS levels, the cross-level kicks of small sets).  G = 2^lg consecutive lanes (G <= 32,
// so a group never straddles a warp) share one receiver and stride over its sources;
// blockIdx.y splits the source range as in the tiled form.  The set is small, so source
// records are read through L1 without staging.  Mixed: FP32 partial sums over runs of
// kSymFlushJ sources per lane, float-float (TwoSum) across runs and lanes, no FP64 instruction
// before the epilogue; FP64: FP64 throughout.  DIAG: same list on both sides, the self
// pair excluded by index.
// One CTA of a wide pass: receiver block bx, source slice by of ny.
template <int P, int KIND, bool DIAG>
__device__ __forceinline__ void wide_pair_body(const PairArgs& a, int lg, int bx, int by, int ny) {
    const int G = 1 << lg;
    const long long gt = (long long)bx * kThreads + threadIdx.x;
    const int slot = (int)(gt >> lg);
    const int g = (int)(gt & (G - 1));
    const bool active = slot < a.n_i;
    const int i = active ? slot : a.n_i - 1;
    const int js = by * a.j_per_split;
    const int je = min(a.n_j, js + a.j_per_split);
    double r[3];
    if constexpr (P == FSI_MIXED) {
        const RecMix ri = reinterpret_cast<const RecMix*>(a.irec)[i];
        MixI p;
        p.xh = ri.hi.x; p.yh = ri.hi.y; p.zh = ri.hi.z;
        p.xl = ri.lo.x; p.yl = ri.lo.y; p.zl = ri.lo.z;
        p.ax = p.ay = p.az = 0.f;
        if constexpr (KIND == KIND_GRAD) {
            const float4 ai = reinterpret_cast<const float4*>(a.iacc)[i];
            p.ax = ai.x; p.ay = ai.y; p.az = ai.z;
        }
        const RecMix* J = reinterpret_cast<const RecMix*>(a.jrec);
        const float4* JA = reinterpret_cast<const float4*>(a.jacc);
        const float eps2f = (float)a.eps2;
        float sh[3] = {0.f, 0.f, 0.f}, sl[3] = {0.f, 0.f, 0.f}, f[3] = {0.f, 0.f, 0.f};
        if (active) {
            int cnt = 0;
            for (int j = js + g; j < je; j += G) {
                const RecMix rj = J[j];
                if constexpr (KIND == KIND_ACC)
                    mix_acc_pair<DIAG>(rj.hi, rj.lo, p, eps2f, j == i + a.i_off, f[0], f[1], f[2]);
                else
                    mix_grad_pair<DIAG>(rj.hi, rj.lo, JA[j], p, eps2f, j == i + a.i_off, f[0], f[1], f[2]);
                if (++cnt == kSymFlushJ) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) { ff_acc(sh[c], sl[c], f[c]); f[c] = 0.f; }
                    cnt = 0;
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) ff_acc(sh[c], sl[c], f[c]);
        }
        // every lane of the warp takes part (inactive lanes add zeros)
        for (int o = G >> 1; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float oh = __shfl_xor_sync(0xffffffffu, sh[c], o);
                const float ol = __shfl_xor_sync(0xffffffffu, sl[c], o);
                ff_acc(sh[c], sl[c], oh);
                sl[c] = __fadd_rn(sl[c], ol);
            }
        if (!active || g != 0) return;
#pragma unroll
        for (int c = 0; c < 3; ++c) r[c] = (double)sh[c] + (double)sl[c];
    } else {
        const D4 ri = reinterpret_cast<const D4*>(a.irec)[i];
        F64I p;
        p.x = ri.x; p.y = ri.y; p.z = ri.z;
        p.ax = p.ay = p.az = 0.0;
        if constexpr (KIND == KIND_GRAD) {
            const D4 ai = reinterpret_cast<const D4*>(a.iacc)[i];
            p.ax = ai.x; p.ay = ai.y; p.az = ai.z;
        }
        const D4* J = reinterpret_cast<const D4*>(a.jrec);
        const D4* JA = reinterpret_cast<const D4*>(a.jacc);
        r[0] = r[1] = r[2] = 0.0;
        if (active) {
            for (int j = js + g; j < je; j += G) {
                if constexpr (KIND == KIND_ACC)
                    f64_acc_pair<DIAG>(J[j], p, a.eps2, j == i + a.i_off, r[0], r[1], r[2]);
                else
                    f64_grad_pair<DIAG>(J[j], JA[j], p, a.eps2, j == i + a.i_off, r[0], r[1], r[2]);
            }
        }
        for (int o = G >> 1; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < 3; ++c) r[c] += __shfl_xor_sync(0xffffffffu, r[c], o);
        if (!active || g != 0) return;
    }
    if (ny == 1) {
        epilogue<P>(a, i, r[0], r[1], r[2]);
    } else {
        double* part = a.part + (size_t)by * 3 * a.n_i;
        part[i] = r[0];
        part[(size_t)a.n_i + i] = r[1];
        part[2 * (size_t)a.n_i + i] = r[2];
    }
}

template <int P, int KIND, bool DIAG>
__global__ void __launch_bounds__(kThreads) wide_pair_kernel(const PairArgs a, int lg) {
    wide_pair_body<P, KIND, DIAG>(a, lg, blockIdx.x, blockIdx.y, gridDim.y);
}

// Two independent unmasked passes in one launch (the two directions of a cross-level
// kick, one source slice each): CTAs [0, ctas_a) run a, the others b.
template <int P, int KIND>
__global__ void __launch_bounds__(kThreads) wide_pair2_kernel(const PairArgs a, const PairArgs b,
                                                              int lga, int lgb, int ctas_a) {
    if ((int)blockIdx.x < ctas_a) wide_pair_body<P, KIND, false>(a, lga, blockIdx.x, 0, 1);
    else wide_pair_body<P, KIND, false>(b, lgb, blockIdx.x - ctas_a, 0, 1);
}

// =================================================================================
// Symmetric pair kernel: the self-interaction of one set with every unordered pair
// evaluated once (Newton's third law: the term of j on i and of i on j share the
// separation, the reciprocal square root and the tidal factor).
//
// Work items (blockIdx.x = b * (1 + nchunk) + c): i-block b (256 * I consecutive
// particles held in registers) against
//   c = 0   : the tiles of its own block, one-sided (i-side only, self pair excluded
//             by index) -- every pair inside a block is then evaluated twice, which is
//             only (256 I)/n of the work;
//   c >= 1  : chunk c-1 of `chunk` tiles among the tiles above the block, symmetric.
// Items past the end of the tile range exit at once.  The i-side sums (mixed: FP32 per
// tile, FP64 across tiles; FP64: FP64) and the j-side sums (mixed: FP32 warp
// reduce-scatter; FP64: carried around the warp by f64_rotate32; then a shared-memory sum
// over the CTA's warps, per tile) are added to the FP64 accumulator with red.global.add;
// a finalize kernel then applies the epilogue.
struct SymArgs {
    const void* rec;
    const void* accrec;
    int n;
    int chunk;
    int nchunk;
    double eps2;
    double* accum;      // 3 x n, zeroed before the launch
    int* err;
    long long timeout_ns;
    // far-tile path of the second form (null rel: never taken), see SymFar
    const float4* rel;
    const float4* sub;
    float far_k2;
    unsigned long long* far_stats;
    int skip_diag;      // packed form: the blocks' own pairs are left to sym_diag_ff_kernel
    // share `part` of nparts (0: all): the launch covers the items of a contiguous range of
    // i-blocks (sym_part_blocks), item index = blockIdx.x + item0
    int part, nparts;
    int item0;
};

// i-blocks [b0, b1) of share `part` of nparts of a symmetric pass over nb blocks of bt
// source tiles each (ntj tiles in all): contiguous ranges with about equal tile visits,
// block b costing its own bt tiles plus the ntj - (b + 1) bt tiles above it, each block in
// the share where the midpoint of its visits falls.  Shares may be empty.
static void sym_part_blocks(int nb, int bt, int ntj, int part, int nparts, int& b0, int& b1) {
    if (nparts <= 1) { b0 = 0; b1 = nb; return; }
    auto w = [&](int b) { return (long long)bt + std::max(0, ntj - (b + 1) * bt); };
    long long total = 0;
    for (int b = 0; b < nb; ++b) total += w(b);
    long long cum = 0;
    b0 = b1 = nb;
    bool open = false;
    for (int b = 0; b < nb; ++b) {
        const long long wb = w(b);
        const int owner = (int)std::min<long long>(nparts - 1, (2 * cum + wb) * nparts / (2 * total));
        if (owner == part && !open) { b0 = b; open = true; }
        if (owner > part) { if (!open) b0 = b; b1 = b; return; }
        cum += wb;
    }
    if (!open) b0 = nb;
}


// Reduce-scatter of 4 j-groups x 3 components over a warp: on return every lane holds in
// out[] the warp total of j-group (lane >> 3).
template <class T>
__device__ __forceinline__ void reduce_scatter4(const T (&v)[4][3], int lane, T (&out)[3]) {
    const bool b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1;
    T k1[2][3];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const T send = b4 ? v[k][q] : v[2 + k][q];
            const T keep = b4 ? v[2 + k][q] : v[k][q];
            k1[k][q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const T send = b3 ? k1[0][q] : k1[1][q];
        const T keep = b3 ? k1[1][q] : k1[0][q];
        T r = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        r += __shfl_xor_sync(0xffffffffu, r, 4);
        r += __shfl_xor_sync(0xffffffffu, r, 2);
        r += __shfl_xor_sync(0xffffffffu, r, 1);
        out[q] = r;
    }
}

// i-side state of the symmetric kernel.
struct SymMixI {
    float xh, yh, zh, xl, yl, zl;
    float nA, nB;          // -2.5 m_i, +1.5 m_i  (j-side weight -m_i r^-3, refined)
    float ax, ay, az, nm;  // gradient: a_i and -m_i
};

__device__ __forceinline__ void mix_acc_sym(const float4 h, const float4 l, const SymMixI& p,
                                            float eps2f, float (&fi)[3], float (&fj)[3]) {
    const float dx = (h.x - p.xh) + (l.x - p.xl);
    const float dy = (h.y - p.yh) + (l.y - p.yl);
    const float dz = (h.z - p.zh) + (l.z - p.zl);
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2f)));
    const float y = rsqrt_hw(r2);
    const float y2 = y * y;
    const float sres = r2 * y2;
    const float y3 = y2 * y;
    const float wi = y3 * fmaf(sres, l.w, h.w);     //  m_j r^-3
    const float wj = y3 * fmaf(sres, p.nB, p.nA);   // -m_i r^-3
    fi[0] = fmaf(wi, dx, fi[0]); fi[1] = fmaf(wi, dy, fi[1]); fi[2] = fmaf(wi, dz, fi[2]);
    fj[0] = fmaf(wj, dx, fj[0]); fj[1] = fmaf(wj, dy, fj[1]); fj[2] = fmaf(wj, dz, fj[2]);
}

__device__ __forceinline__ void mix_grad_sym(const float4 h, const float4 l, const float4 aj,
                                             const SymMixI& p, float eps2f,
                                             float (&gi)[3], float (&gj)[3]) {
    const float dx = (h.x - p.xh) + (l.x - p.xl);
    const float dy = (h.y - p.yh) + (l.y - p.yl);
    const float dz = (h.z - p.zh) + (l.z - p.zl);
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2f)));
    const float y = rsqrt_hw(r2);
    const float y2 = y * y;
    const float sres = r2 * y2;
    const float r3 = (y2 * y) * fmaf(sres, -1.5f, 2.5f);           // r^-3 (refined)
    const float bx = aj.x - p.ax, by = aj.y - p.ay, bz = aj.z - p.az;
    const float dot = fmaf(bx, dx, fmaf(by, dy, bz * dz));
    const float q = r3 * (y2 * fmaf(3.0f, sres, -6.0f));           // -3 r^-5 (refined)
    const float s = q * dot;
    // T(d) b = r^-3 b - 3 r^-5 (b.d) d: on i with weight m_j, on j with weight -m_i
    const float tx = fmaf(r3, bx, s * dx), ty = fmaf(r3, by, s * dy), tz = fmaf(r3, bz, s * dz);
    gi[0] = fmaf(aj.w, tx, gi[0]); gi[1] = fmaf(aj.w, ty, gi[1]); gi[2] = fmaf(aj.w, tz, gi[2]);
    gj[0] = fmaf(p.nm, tx, gj[0]); gj[1] = fmaf(p.nm, ty, gj[1]); gj[2] = fmaf(p.nm, tz, gj[2]);
}

// Far-tile forms.  r = (x_j - C, y_j - C, z_j - C, m_j) is the source relative to the
// centre C of its 32-record sub-tile, rounded once to FP32; D = (C - xh_i) - xl_i.  Then
// d = D + r.xyz costs 3 additions instead of 9, with error at most about
// 3 u (|d| + |r.xyz|) (u = 2^-24): the far test keeps |r.xyz| <= |d| / kappa.
__device__ __forceinline__ void mix_acc_sym_far(const float4 r, const float (&D)[3], float nmi,
                                                float eps2f, float (&fi)[3], float (&fj)[3]) {
    const float dx = D[0] + r.x, dy = D[1] + r.y, dz = D[2] + r.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2f)));
    const float y = rsqrt_hw(r2);
    const float y2 = y * y;
    const float sres = r2 * y2;
    const float r3 = (y2 * y) * fmaf(sres, -1.5f, 2.5f);           // r^-3 (refined)
    const float wi = r3 * r.w;                                       //  m_j r^-3
    const float wj = r3 * nmi;                                       // -m_i r^-3
    fi[0] = fmaf(wi, dx, fi[0]); fi[1] = fmaf(wi, dy, fi[1]); fi[2] = fmaf(wi, dz, fi[2]);
    fj[0] = fmaf(wj, dx, fj[0]); fj[1] = fmaf(wj, dy, fj[1]); fj[2] = fmaf(wj, dz, fj[2]);
}

__device__ __forceinline__ void mix_grad_sym_far(const float4 r, const float4 aj, const float (&D)[3],
                                                 const SymMixI& p, float eps2f,
                                                 float (&gi)[3], float (&gj)[3]) {
    const float dx = D[0] + r.x, dy = D[1] + r.y, dz = D[2] + r.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2f)));
    const float y = rsqrt_hw(r2);
    const float y2 = y * y;
    const float sres = r2 * y2;
    const float r3 = (y2 * y) * fmaf(sres, -1.5f, 2.5f);
    const float bx = aj.x - p.ax, by = aj.y - p.ay, bz = aj.z - p.az;
    const float dot = fmaf(bx, dx, fmaf(by, dy, bz * dz));
    const float q = r3 * (y2 * fmaf(3.0f, sres, -6.0f));
    const float s = q * dot;
    const float tx = fmaf(r3, bx, s * dx), ty = fmaf(r3, by, s * dy), tz = fmaf(r3, bz, s * dz);
    gi[0] = fmaf(aj.w, tx, gi[0]); gi[1] = fmaf(aj.w, ty, gi[1]); gi[2] = fmaf(aj.w, tz, gi[2]);
    gj[0] = fmaf(p.nm, tx, gj[0]); gj[1] = fmaf(p.nm, ty, gj[1]); gj[2] = fmaf(p.nm, tz, gj[2]);
}

struct SymF64I {
    double x, y, z, nm;
    double ax, ay, az;
};

__device__ __forceinline__ void f64_acc_sym(const D4 j, const SymF64I& p, double eps2,
                                            double (&fi)[3], double (&fj)[3]) {
    const double dx = j.x - p.x, dy = j.y - p.y, dz = j.z - p.z;
    const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
    const double y = rsqrt_f64(r2);
    const double y3 = (y * y) * y;
    const double wi = j.w * y3, wj = p.nm * y3;
    fi[0] = fma(wi, dx, fi[0]); fi[1] = fma(wi, dy, fi[1]); fi[2] = fma(wi, dz, fi[2]);
    fj[0] = fma(wj, dx, fj[0]); fj[1] = fma(wj, dy, fj[1]); fj[2] = fma(wj, dz, fj[2]);
}

__device__ __forceinline__ void f64_grad_sym(const D4 j, const D4 aj, const SymF64I& p,
                                             double eps2, double (&gi)[3], double (&gj)[3]) {
    const double dx = j.x - p.x, dy = j.y - p.y, dz = j.z - p.z;
    const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
    const double y = rsqrt_f64(r2);
    const double y2 = y * y;
    const double y3 = y2 * y;
    const double bx = aj.x - p.ax, by = aj.y - p.ay, bz = aj.z - p.az;
    const double dot = fma(bx, dx, fma(by, dy, bz * dz));
    const double s = (y3 * y2) * (-3.0 * dot);
    const double tx = fma(y3, bx, s * dx), ty = fma(y3, by, s * dy), tz = fma(y3, bz, s * dz);
    gi[0] = fma(aj.w, tx, gi[0]); gi[1] = fma(aj.w, ty, gi[1]); gi[2] = fma(aj.w, tz, gi[2]);
    gj[0] = fma(p.nm, tx, gj[0]); gj[1] = fma(p.nm, ty, gj[1]); gj[2] = fma(p.nm, tz, gj[2]);
}

// 32 sources jj .. jj + 31 of a staged tile on the thread's I receivers, both sides, with
// the source side carried around the warp: lane l starts with a packet of source jj + l
// (position record, acceleration record for the gradient, partial sums) and hands it to
// lane l - 1 after each step, so that after 32 steps the packet is back in lane l with
// the terms of all the warp's receivers, and the lanes' partial sums need no FP64 adds to
// be combined (the B300 FP64 pipe issues only two lane operations per SM and clock; the
// shuffles run elsewhere).  tot: the warp's sums for source jj + lane (zero past cnt).
// FULL: all 32 sources exist; otherwise a packet past the tile's cnt sources is carried
// along without terms.
template <int KIND, int I, bool FULL>
__device__ __forceinline__ void f64_rotate32(const D4* rec, const D4* arec, int jj, int cnt,
                                             int lane, const SymF64I (&pi)[I], double eps2,
                                             double (&acc)[I][3], double (&tot)[3]) {
    const int jh = jj + lane;
    int valid = FULL || jh < cnt;
    const int jl = valid ? jh : jj;
    D4 r = rec[jl];
    D4 aj = make_d4(0.0, 0.0, 0.0, 0.0);
    if constexpr (KIND == KIND_GRAD) aj = arec[jl];
    double f[3] = {0.0, 0.0, 0.0};
    const int from = (lane + 1) & 31;
#pragma unroll 2
    for (int k = 0; k < 32; ++k) {
        if (FULL || valid) {
            if constexpr (KIND == KIND_ACC) {
#pragma unroll
                for (int u = 0; u < I; ++u) f64_acc_sym(r, pi[u], eps2, acc[u], f);
            } else {
#pragma unroll
                for (int u = 0; u < I; ++u) f64_grad_sym(r, aj, pi[u], eps2, acc[u], f);
            }
        }
        r.x = __shfl_sync(0xffffffffu, r.x, from);
        r.y = __shfl_sync(0xffffffffu, r.y, from);
        r.z = __shfl_sync(0xffffffffu, r.z, from);
        if constexpr (KIND == KIND_ACC) {
            r.w = __shfl_sync(0xffffffffu, r.w, from);
        } else {
            aj.x = __shfl_sync(0xffffffffu, aj.x, from);
            aj.y = __shfl_sync(0xffffffffu, aj.y, from);
            aj.z = __shfl_sync(0xffffffffu, aj.z, from);
            aj.w = __shfl_sync(0xffffffffu, aj.w, from);
        }
        f[0] = __shfl_sync(0xffffffffu, f[0], from);
        f[1] = __shfl_sync(0xffffffffu, f[1], from);
        f[2] = __shfl_sync(0xffffffffu, f[2], from);
        if (!FULL) valid = __shfl_sync(0xffffffffu, valid, from);
    }
    tot[0] = f[0]; tot[1] = f[1]; tot[2] = f[2];
}

template <int P, int KIND>
struct SymCfg {
    static constexpr int ACCREC = Cfg<P, KIND>::ACCREC;
    static constexpr int SB = kTileJ * (kRec + ACCREC);           // one pipeline stage
    using JT = typename std::conditional<P == FSI_MIXED, float, double>::type;
    static constexpr int JPART = (kThreads / 32) * kTileJ * 3 * (int)sizeof(JT);
    static constexpr int SMEM = kStages * SB + JPART;
};

template <int P, int KIND, int I>
__global__ void __launch_bounds__(kThreads, 2) sym_pair_kernel(const SymArgs a) {
    static_assert(kThreads == kTileJ, "an i-block spans I source tiles");
    using JT = typename SymCfg<P, KIND>::JT;
    constexpr int ACCREC = SymCfg<P, KIND>::ACCREC;
    constexpr int SB = SymCfg<P, KIND>::SB;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[kStages];
    JT* jpart = reinterpret_cast<JT*>(smem + kStages * SB);

    const int item = (int)blockIdx.x + a.item0;
    const int b = item / (1 + a.nchunk);
    const int c = item % (1 + a.nchunk);
    const int ntj = (a.n + kTileJ - 1) / kTileJ;
    const bool diag = (c == 0);
    int t0, t1;
    if (diag) { t0 = b * I; t1 = min((b + 1) * I, ntj); }
    else { t0 = (b + 1) * I + (c - 1) * a.chunk; t1 = min(t0 + a.chunk, ntj); }
    if (t0 >= t1) return;                       // uniform: before any barrier
    const int ntiles = t1 - t0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i0 = b * (kThreads * I);

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int t) {
        const int s = t % kStages;
        const int jt = (t0 + t) * kTileJ;
        const int cnt = min(kTileJ, a.n - jt);
        unsigned char* base = smem + s * SB;
        mbar_arrive_expect_tx(&bars[s], (uint32_t)cnt * (kRec + ACCREC));
        bulk_g2s(base, (const unsigned char*)a.rec + (size_t)jt * kRec, (uint32_t)cnt * kRec, &bars[s]);
        if (ACCREC)
            bulk_g2s(base + kTileJ * kRec, (const unsigned char*)a.accrec + (size_t)jt * ACCREC,
                     (uint32_t)cnt * ACCREC, &bars[s]);
    };
    if (tid == 0)
        for (int t = 0; t < min(kStages, ntiles); ++t) issue(t);

    double acc64[I][3];
    bool valid[I];
    int my_i[I];
#pragma unroll
    for (int u = 0; u < I; ++u) {
        acc64[u][0] = acc64[u][1] = acc64[u][2] = 0.0;
        my_i[u] = i0 + u * kThreads + tid;
        valid[u] = my_i[u] < a.n;
    }

    bool aborted = false;
    int t_stop = ntiles;
    if constexpr (P == FSI_MIXED) {
        SymMixI pi[I];
        float f[I][3];
#pragma unroll
        for (int u = 0; u < I; ++u) {
            const int i = min(my_i[u], a.n - 1);
            const RecMix r = reinterpret_cast<const RecMix*>(a.rec)[i];
            pi[u].xh = r.hi.x; pi[u].yh = r.hi.y; pi[u].zh = r.hi.z;
            pi[u].xl = r.lo.x; pi[u].yl = r.lo.y; pi[u].zl = r.lo.z;
            // an i past the end contributes nothing to the j side
            pi[u].nA = valid[u] ? -r.hi.w : 0.f;
            pi[u].nB = valid[u] ? -r.lo.w : 0.f;
            if constexpr (KIND == KIND_GRAD) {
                const float4 ai = reinterpret_cast<const float4*>(a.accrec)[i];
                pi[u].ax = ai.x; pi[u].ay = ai.y; pi[u].az = ai.z;
                pi[u].nm = valid[u] ? -ai.w : 0.f;
            } else {
                pi[u].ax = pi[u].ay = pi[u].az = pi[u].nm = 0.f;
            }
            f[u][0] = f[u][1] = f[u][2] = 0.f;
        }
        const float eps2f = (float)a.eps2;
        for (int t = 0; t < ntiles; ++t) {
            const int s = t % kStages;
            const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((t / kStages) & 1), a.timeout_ns, a.err);
            const int jt = (t0 + t) * kTileJ;
            const int cnt = min(kTileJ, a.n - jt);
            const unsigned char* base = smem + s * SB;
            const RecMix* rec = reinterpret_cast<const RecMix*>(base);
            const float4* arec = reinterpret_cast<const float4*>(base + kTileJ * kRec);
            if (diag) {
                // one-sided, self pair excluded by index (reuses the one-sided pair code)
                MixI q[I];
#pragma unroll
                for (int u = 0; u < I; ++u) {
                    q[u].xh = pi[u].xh; q[u].yh = pi[u].yh; q[u].zh = pi[u].zh;
                    q[u].xl = pi[u].xl; q[u].yl = pi[u].yl; q[u].zl = pi[u].zl;
                    q[u].ax = pi[u].ax; q[u].ay = pi[u].ay; q[u].az = pi[u].az;
                }
                for (int jj = 0; jj < cnt; ++jj) {
                    const float4 h = rec[jj].hi;
                    const float4 l = rec[jj].lo;
                    if constexpr (KIND == KIND_ACC) {
#pragma unroll
                        for (int u = 0; u < I; ++u)
                            mix_acc_pair<true>(h, l, q[u], eps2f, jt + jj == my_i[u], f[u][0], f[u][1], f[u][2]);
                    } else {
                        const float4 aj = arec[jj];
#pragma unroll
                        for (int u = 0; u < I; ++u)
                            mix_grad_pair<true>(h, l, aj, q[u], eps2f, jt + jj == my_i[u], f[u][0], f[u][1], f[u][2]);
                    }
                }
            } else {
                for (int jj = 0; jj < cnt; jj += 4) {
                    float fj[4][3];
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        fj[g][0] = fj[g][1] = fj[g][2] = 0.f;
                        if (jj + g < cnt) {
                            const float4 h = rec[jj + g].hi;
                            const float4 l = rec[jj + g].lo;
                            if constexpr (KIND == KIND_ACC) {
#pragma unroll
                                for (int u = 0; u < I; ++u) mix_acc_sym(h, l, pi[u], eps2f, f[u], fj[g]);
                            } else {
                                const float4 aj = arec[jj + g];
#pragma unroll
                                for (int u = 0; u < I; ++u) mix_grad_sym(h, l, aj, pi[u], eps2f, f[u], fj[g]);
                            }
                        }
                    }
                    float tot[3];
                    reduce_scatter4<float>(fj, lane, tot);
                    const int jl = jj + (lane >> 3);
                    if ((lane & 7) == 0 && jl < cnt) {
                        JT* dst = jpart + ((size_t)warp * kTileJ + jl) * 3;
                        dst[0] = tot[0]; dst[1] = tot[1]; dst[2] = tot[2];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < I; ++u)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    acc64[u][q] += (double)f[u][q];
                    f[u][q] = 0.f;
                }
            if (__syncthreads_or(!ok)) { aborted = true; t_stop = t; break; }
            if (!diag && tid < cnt) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    float sum = 0.f;
#pragma unroll
                    for (int w = 0; w < kThreads / 32; ++w) sum += jpart[((size_t)w * kTileJ + tid) * 3 + q];
                    red_add(a.accum + (size_t)q * a.n + jt + tid, (double)sum);
                }
            }
            __syncthreads();
            if (tid == 0 && t + kStages < ntiles) issue(t + kStages);
        }
    } else {
        SymF64I pi[I];
#pragma unroll
        for (int u = 0; u < I; ++u) {
            const int i = min(my_i[u], a.n - 1);
            const D4 r = reinterpret_cast<const D4*>(a.rec)[i];
            pi[u].x = r.x; pi[u].y = r.y; pi[u].z = r.z;
            pi[u].nm = valid[u] ? -r.w : 0.0;
            if constexpr (KIND == KIND_GRAD) {
                const D4 ai = reinterpret_cast<const D4*>(a.accrec)[i];
                pi[u].ax = ai.x; pi[u].ay = ai.y; pi[u].az = ai.z;
            } else {
                pi[u].ax = pi[u].ay = pi[u].az = 0.0;
            }
        }
        for (int t = 0; t < ntiles; ++t) {
            const int s = t % kStages;
            const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((t / kStages) & 1), a.timeout_ns, a.err);
            const int jt = (t0 + t) * kTileJ;
            const int cnt = min(kTileJ, a.n - jt);
            const unsigned char* base = smem + s * SB;
            const D4* rec = reinterpret_cast<const D4*>(base);
            const D4* arec = reinterpret_cast<const D4*>(base + kTileJ * kRec);
            if (diag) {
                F64I q[I];
#pragma unroll
                for (int u = 0; u < I; ++u) {
                    q[u].x = pi[u].x; q[u].y = pi[u].y; q[u].z = pi[u].z;
                    q[u].ax = pi[u].ax; q[u].ay = pi[u].ay; q[u].az = pi[u].az;
                }
                for (int jj = 0; jj < cnt; ++jj) {
                    const D4 r = rec[jj];
                    if constexpr (KIND == KIND_ACC) {
#pragma unroll
                        for (int u = 0; u < I; ++u)
                            f64_acc_pair<true>(r, q[u], a.eps2, jt + jj == my_i[u], acc64[u][0], acc64[u][1], acc64[u][2]);
                    } else {
                        const D4 aj = arec[jj];
#pragma unroll
                        for (int u = 0; u < I; ++u)
                            f64_grad_pair<true>(r, aj, q[u], a.eps2, jt + jj == my_i[u], acc64[u][0], acc64[u][1], acc64[u][2]);
                    }
                }
            } else {
                for (int jj = 0; jj < cnt; jj += 32) {
                    double tot[3];
                    if (jj + 32 <= cnt) f64_rotate32<KIND, I, true>(rec, arec, jj, cnt, lane, pi, a.eps2, acc64, tot);
                    else f64_rotate32<KIND, I, false>(rec, arec, jj, cnt, lane, pi, a.eps2, acc64, tot);
                    const int jl = jj + lane;
                    if (jl < cnt) {
                        JT* dst = jpart + ((size_t)warp * kTileJ + jl) * 3;
                        dst[0] = tot[0]; dst[1] = tot[1]; dst[2] = tot[2];
                    }
                }
            }
            if (__syncthreads_or(!ok)) { aborted = true; t_stop = t; break; }
            if (!diag && tid < cnt) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    double sum = 0.0;
#pragma unroll
                    for (int w = 0; w < kThreads / 32; ++w) sum += jpart[((size_t)w * kTileJ + tid) * 3 + q];
                    red_add(a.accum + (size_t)q * a.n + jt + tid, sum);
                }
            }
            __syncthreads();
            if (tid == 0 && t + kStages < ntiles) issue(t + kStages);
        }
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
    for (int u = 0; u < I; ++u) {
        if (!valid[u]) continue;
#pragma unroll
        for (int q = 0; q < 3; ++q) red_add(a.accum + (size_t)q * a.n + my_i[u], acc64[u][q]);
    }
}

// ---------------------------------------------------------------------------------
// Symmetric mixed kernel, second form (autotuned against the first):
//  - the FP64 per-particle sums live in shared memory (one slot per thread and particle),
//    so a thread can hold up to 6 active particles in registers;
//  - warp w holds the 32 I consecutive particles i0 + 32 I w + 32 u + lane (u < I), so
//    that a warp's particles are close in space when the set is in spatial order;
//  - inside each group of 4 sources, lane l visits source (g XOR (l >> 3)) at step g, so
//    after the pair loop slot s of lane l holds the partial of source s ^ (l >> 3); the
//    warp reduce-scatter then needs no selects: at the xor-16 level every lane keeps slots
//    0, 1 and sends 2, 3, at the xor-8 level keeps slot 0 and sends 1, and three butterfly
//    levels finish; lane l ends with the total of source l >> 3.  The 4 sources read at one
//    step are 4 consecutive records, so the shared-memory loads stay conflict-free.
//  - FAR: each stage also holds the tile's relative records and its 8 sub-tile centres;
//    a warp whose box of particles is far from a 32-record sub-tile (gap to the centre
//    >= (kappa + 1) R, R the sub-tile radius) takes the 3-addition separation
//    (mix_*_sym_far) for the whole sub-tile.  The test is warp-uniform, so the two loops
//    never diverge inside a warp.
template <int KIND, int I, bool FAR>
__global__ void __launch_bounds__(kThreads, 2) sym_mixed_v2_kernel(const SymArgs a) {
    static_assert(kThreads == kTileJ, "an i-block spans I source tiles");
    constexpr int ACCREC = SymCfg<FSI_MIXED, KIND>::ACCREC;
    constexpr int RELB = FAR ? 16 : 0;
    constexpr int SUBB = FAR ? (kTileJ / 32) * 16 : 0;
    constexpr int SB = kTileJ * (kRec + ACCREC + RELB) + SUBB;
    constexpr int JPART = SymCfg<FSI_MIXED, KIND>::JPART;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[kStages];
    __shared__ float wbox[FAR ? kThreads / 32 : 1][6];
    float* jpart = reinterpret_cast<float*>(smem + kStages * SB);
    double* acc_s = reinterpret_cast<double*>(smem + kStages * SB + JPART);   // [I][3][kThreads]

    const int item = (int)blockIdx.x + a.item0;
    const int b = item / (1 + a.nchunk);
    const int c = item % (1 + a.nchunk);
    const int ntj = (a.n + kTileJ - 1) / kTileJ;
    const bool diag = (c == 0);
    int t0, t1;
    if (diag) { t0 = b * I; t1 = min((b + 1) * I, ntj); }
    else { t0 = (b + 1) * I + (c - 1) * a.chunk; t1 = min(t0 + a.chunk, ntj); }
    if (t0 >= t1) return;
    const int ntiles = t1 - t0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, L = lane >> 3;
    const int i0 = b * (kThreads * I);
    const bool far_on = FAR && a.rel != nullptr && !diag;

    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) mbar_init(&bars[st], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int t) {
        const int st = t % kStages;
        const int jt = (t0 + t) * kTileJ;
        const int cnt = min(kTileJ, a.n - jt);
        const int nsub = (cnt + 31) >> 5;
        unsigned char* base = smem + st * SB;
        mbar_arrive_expect_tx(&bars[st], (uint32_t)cnt * (kRec + ACCREC) +
                                             (far_on ? (uint32_t)(cnt * 16 + nsub * 16) : 0u));
        bulk_g2s(base, (const unsigned char*)a.rec + (size_t)jt * kRec, (uint32_t)cnt * kRec, &bars[st]);
        if (ACCREC)
            bulk_g2s(base + kTileJ * kRec, (const unsigned char*)a.accrec + (size_t)jt * ACCREC,
                     (uint32_t)cnt * ACCREC, &bars[st]);
        if (far_on) {
            bulk_g2s(base + kTileJ * (kRec + ACCREC), (const unsigned char*)(a.rel + jt),
                     (uint32_t)cnt * 16, &bars[st]);
            bulk_g2s(base + kTileJ * (kRec + ACCREC + RELB), (const unsigned char*)(a.sub + jt / 32),
                     (uint32_t)nsub * 16, &bars[st]);
        }
    };
    if (tid == 0)
        for (int t = 0; t < min(kStages, ntiles); ++t) issue(t);

    SymMixI pi[I];
    float f[I][3];
    int my_i[I];
    bool valid[I];
#pragma unroll
    for (int u = 0; u < I; ++u) {
        my_i[u] = i0 + warp * (32 * I) + u * 32 + lane;
        valid[u] = my_i[u] < a.n;
        const int i = min(my_i[u], a.n - 1);
        const RecMix r = reinterpret_cast<const RecMix*>(a.rec)[i];
        pi[u].xh = r.hi.x; pi[u].yh = r.hi.y; pi[u].zh = r.hi.z;
        pi[u].xl = r.lo.x; pi[u].yl = r.lo.y; pi[u].zl = r.lo.z;
        pi[u].nA = valid[u] ? -r.hi.w : 0.f;
        pi[u].nB = valid[u] ? -r.lo.w : 0.f;
        if constexpr (KIND == KIND_GRAD) {
            const float4 ai = reinterpret_cast<const float4*>(a.accrec)[i];
            pi[u].ax = ai.x; pi[u].ay = ai.y; pi[u].az = ai.z;
            pi[u].nm = valid[u] ? -ai.w : 0.f;
        } else {
            pi[u].ax = pi[u].ay = pi[u].az = 0.f;
            pi[u].nm = (far_on && valid[u]) ? -a.rel[i].w : 0.f;    // -m_i for the far form
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            f[u][q] = 0.f;
            acc_s[(u * 3 + q) * kThreads + tid] = 0.0;
        }
    }
    if (far_on) {
        // box of the warp's particles (FP32 high parts)
        float bl[3] = {pi[0].xh, pi[0].yh, pi[0].zh}, bh[3] = {pi[0].xh, pi[0].yh, pi[0].zh};
#pragma unroll
        for (int u = 1; u < I; ++u) {
            bl[0] = fminf(bl[0], pi[u].xh); bl[1] = fminf(bl[1], pi[u].yh); bl[2] = fminf(bl[2], pi[u].zh);
            bh[0] = fmaxf(bh[0], pi[u].xh); bh[1] = fmaxf(bh[1], pi[u].yh); bh[2] = fmaxf(bh[2], pi[u].zh);
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
            for (int q = 0; q < 3; ++q) { wbox[FAR ? warp : 0][q] = bl[q]; wbox[FAR ? warp : 0][3 + q] = bh[q]; }
        __syncwarp();
    }
    const float eps2f = (float)a.eps2;
    unsigned far_visits = 0, near_visits = 0;
    bool aborted = false;
    int t_stop = ntiles;
    for (int t = 0; t < ntiles; ++t) {
        const int st = t % kStages;
        const bool ok = mbar_wait_bounded(&bars[st], (uint32_t)((t / kStages) & 1), a.timeout_ns, a.err);
        const int jt = (t0 + t) * kTileJ;
        const int cnt = min(kTileJ, a.n - jt);
        const unsigned char* base = smem + st * SB;
        const RecMix* rec = reinterpret_cast<const RecMix*>(base);
        const float4* arec = reinterpret_cast<const float4*>(base + kTileJ * kRec);
        const float4* rel_s = reinterpret_cast<const float4*>(base + kTileJ * (kRec + ACCREC));
        const float4* sub_s = reinterpret_cast<const float4*>(base + kTileJ * (kRec + ACCREC + RELB));
        if (diag) {
            MixI q[I];
#pragma unroll
            for (int u = 0; u < I; ++u) {
                q[u].xh = pi[u].xh; q[u].yh = pi[u].yh; q[u].zh = pi[u].zh;
                q[u].xl = pi[u].xl; q[u].yl = pi[u].yl; q[u].zl = pi[u].zl;
                q[u].ax = pi[u].ax; q[u].ay = pi[u].ay; q[u].az = pi[u].az;
            }
            for (int jj = 0; jj < cnt; ++jj) {
                const float4 h = rec[jj].hi;
                const float4 l = rec[jj].lo;
                if constexpr (KIND == KIND_ACC) {
#pragma unroll
                    for (int u = 0; u < I; ++u)
                        mix_acc_pair<true>(h, l, q[u], eps2f, jt + jj == my_i[u], f[u][0], f[u][1], f[u][2]);
                } else {
                    const float4 aj = arec[jj];
#pragma unroll
                    for (int u = 0; u < I; ++u)
                        mix_grad_pair<true>(h, l, aj, q[u], eps2f, jt + jj == my_i[u], f[u][0], f[u][1], f[u][2]);
                }
            }
        } else {
            unsigned fmask = 0;
            if (far_on) {
                bool fr = false;
                if (lane < ((cnt + 31) >> 5)) {
                    const float4 sb = sub_s[lane];
                    const float* wb = wbox[FAR ? warp : 0];
                    const float gx = fmaxf(0.f, fmaxf(wb[0] - sb.x, sb.x - wb[3]));
                    const float gy = fmaxf(0.f, fmaxf(wb[1] - sb.y, sb.y - wb[4]));
                    const float gz = fmaxf(0.f, fmaxf(wb[2] - sb.z, sb.z - wb[5]));
                    fr = fmaf(gx, gx, fmaf(gy, gy, gz * gz)) >= a.far_k2 * (sb.w * sb.w);
                }
                fmask = __ballot_sync(0xffffffffu, fr);
            }
            // one group of 4 sources; FG selects the far form, FULL drops the bounds check
            // (a full 32-record sub-tile)
            auto group = [&](int jj, auto fg, auto full, const float (&D)[I][3]) {
                constexpr bool FG = decltype(fg)::value;
                constexpr bool FULL = decltype(full)::value;
                float fj[4][3];
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    fj[g][0] = fj[g][1] = fj[g][2] = 0.f;
                    const int jg = jj + (g ^ L);
                    if (FULL || jg < cnt) {
                        if constexpr (FG) {
                            const float4 r = rel_s[jg];
                            if constexpr (KIND == KIND_ACC) {
#pragma unroll
                                for (int u = 0; u < I; ++u) mix_acc_sym_far(r, D[u], pi[u].nm, eps2f, f[u], fj[g]);
                            } else {
                                const float4 aj = arec[jg];
#pragma unroll
                                for (int u = 0; u < I; ++u) mix_grad_sym_far(r, aj, D[u], pi[u], eps2f, f[u], fj[g]);
                            }
                        } else {
                            const float4 h = rec[jg].hi;
                            const float4 l = rec[jg].lo;
                            if constexpr (KIND == KIND_ACC) {
#pragma unroll
                                for (int u = 0; u < I; ++u) mix_acc_sym(h, l, pi[u], eps2f, f[u], fj[g]);
                            } else {
                                const float4 aj = arec[jg];
#pragma unroll
                                for (int u = 0; u < I; ++u) mix_grad_sym(h, l, aj, pi[u], eps2f, f[u], fj[g]);
                            }
                        }
                    }
                }
                float tot[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float k0 = fj[0][q] + __shfl_xor_sync(0xffffffffu, fj[2][q], 16);
                    const float k1 = fj[1][q] + __shfl_xor_sync(0xffffffffu, fj[3][q], 16);
                    float r = k0 + __shfl_xor_sync(0xffffffffu, k1, 8);
                    r += __shfl_xor_sync(0xffffffffu, r, 4);
                    r += __shfl_xor_sync(0xffffffffu, r, 2);
                    r += __shfl_xor_sync(0xffffffffu, r, 1);
                    tot[q] = r;
                }
                const int jl = jj + L;
                if ((lane & 7) == 0 && (FULL || jl < cnt)) {
                    float* dst = jpart + ((size_t)warp * kTileJ + jl) * 3;
                    dst[0] = tot[0]; dst[1] = tot[1]; dst[2] = tot[2];
                }
            };
            for (int k0 = 0; k0 < cnt; k0 += 32) {
                const int jend = min(cnt, k0 + 32);
                if (jend - k0 < 32) {
                    // the ragged end of the last tile: checked hi/lo form
                    float D0[I][3];
                    for (int jj = k0; jj < jend; jj += 4)
                        group(jj, std::false_type{}, std::false_type{}, D0);
                    ++near_visits;
                } else if (FAR && ((fmask >> (k0 >> 5)) & 1u)) {
                    const float4 C = sub_s[k0 >> 5];
                    float D[I][3];
#pragma unroll
                    for (int u = 0; u < I; ++u) {
                        D[u][0] = (C.x - pi[u].xh) - pi[u].xl;
                        D[u][1] = (C.y - pi[u].yh) - pi[u].yl;
                        D[u][2] = (C.z - pi[u].zh) - pi[u].zl;
                    }
                    for (int jj = k0; jj < jend; jj += 4) group(jj, std::true_type{}, std::true_type{}, D);
                    ++far_visits;
                } else {
                    float D0[I][3];
                    for (int jj = k0; jj < jend; jj += 4) group(jj, std::false_type{}, std::true_type{}, D0);
                    ++near_visits;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < I; ++u)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                acc_s[(u * 3 + q) * kThreads + tid] += (double)f[u][q];
                f[u][q] = 0.f;
            }
        if (__syncthreads_or(!ok)) { aborted = true; t_stop = t; break; }
        if (!diag && tid < cnt) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                float sum = 0.f;
#pragma unroll
                for (int w = 0; w < kThreads / 32; ++w) sum += jpart[((size_t)w * kTileJ + tid) * 3 + q];
                red_add(a.accum + (size_t)q * a.n + jt + tid, (double)sum);
            }
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
    if (FAR && a.far_stats && lane == 0 && !diag) {
        atomicAdd(a.far_stats, (unsigned long long)far_visits);
        atomicAdd(a.far_stats + 1, (unsigned long long)near_visits);
    }
#pragma unroll
    for (int u = 0; u < I; ++u) {
        if (!valid[u]) continue;
#pragma unroll
        for (int q = 0; q < 3; ++q)
            red_add(a.accum + (size_t)q * a.n + my_i[u], acc_s[(u * 3 + q) * kThreads + tid]);
    }
}

// ---------------------------------------------------------------------------------
// Symmetric mixed kernel, packed form: the second form's work decomposition with the pair
// arithmetic on packed FP32 pairs (add/mul/fma.rn.f32x2, sm_100 and later).  The pair
// kernels are bound by instruction issue (every FP32 instruction, MUFU, shuffle and
// shared-memory load takes an issue slot); one packed instruction does two FP32 lane
// operations, so the FP32 pipe, not issue, becomes the limit.
//  - a thread's I particles (I even) form I/2 packed pairs (particles 2p, 2p+1 in the
//    low / high half); every source value is broadcast into both halves;
//  - per source, the j-side partials of the two halves are added once (one FP32 add per
//    component) before the warp reduce-scatter of the second form;
//  - the per-pair arithmetic is the second form's, operation for operation, so each
//    half rounds exactly as the scalar code does; only the order of the j-side sums
//    differs.

template <int KIND, int I, int MINB, int NT>
__global__ void __launch_bounds__(NT, MINB) sym_mixed_x2_kernel(const SymArgs a) {
    static_assert((NT * I) % kTileJ == 0 && NT >= kTileJ && NT % 32 == 0,
                  "an i-block spans whole source tiles");
    static_assert(I % 2 == 0, "particles are handled in packed pairs");
    constexpr int BT = NT * I / kTileJ;                 // source tiles per i-block
    constexpr int NP = I / 2;
    constexpr int ACCREC = SymCfg<FSI_MIXED, KIND>::ACCREC;
    constexpr int RELB = 16;
    constexpr int SUBB = (kTileJ / 32) * 16;
    constexpr int SB = kTileJ * (kRec + ACCREC + RELB) + SUBB;
    constexpr int JPART = (NT / 32) * kTileJ * 3 * (int)sizeof(float);
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[kStages];
    __shared__ float wbox[NT / 32][6];
    float* jpart = reinterpret_cast<float*>(smem + kStages * SB);
    // i-side sums across tiles as float-float pairs: acc_s[(p * 3 + q) * NT + tid] =
    // (hi of 2p, hi of 2p+1, lo of 2p, lo of 2p+1) for component q
    float4* acc_s = reinterpret_cast<float4*>(smem + kStages * SB + JPART);

    const int item = (int)blockIdx.x + a.item0;
    const int b = item / (1 + a.nchunk);
    const int c = item % (1 + a.nchunk);
    const int ntj = (a.n + kTileJ - 1) / kTileJ;
    const bool diag = (c == 0);
    int t0, t1;
    if (diag) { t0 = b * BT; t1 = min((b + 1) * BT, ntj); }
    else { t0 = (b + 1) * BT + (c - 1) * a.chunk; t1 = min(t0 + a.chunk, ntj); }
    if (t0 >= t1 || (diag && a.skip_diag)) return;
    const int ntiles = t1 - t0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i0 = b * (NT * I);
    const bool far_on = a.rel != nullptr && !diag;

    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) mbar_init(&bars[st], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int t) {
        const int st = t % kStages;
        const int jt = (t0 + t) * kTileJ;
        const int cnt = min(kTileJ, a.n - jt);
        const int nsub = (cnt + 31) >> 5;
        unsigned char* base = smem + st * SB;
        mbar_arrive_expect_tx(&bars[st], (uint32_t)cnt * (kRec + ACCREC) +
                                             (far_on ? (uint32_t)(cnt * 16 + nsub * 16) : 0u));
        bulk_g2s(base, (const unsigned char*)a.rec + (size_t)jt * kRec, (uint32_t)cnt * kRec, &bars[st]);
        if (ACCREC)
            bulk_g2s(base + kTileJ * kRec, (const unsigned char*)a.accrec + (size_t)jt * ACCREC,
                     (uint32_t)cnt * ACCREC, &bars[st]);
        if (far_on) {
            bulk_g2s(base + kTileJ * (kRec + ACCREC), (const unsigned char*)(a.rel + jt),
                     (uint32_t)cnt * 16, &bars[st]);
            bulk_g2s(base + kTileJ * (kRec + ACCREC + RELB), (const unsigned char*)(a.sub + jt / 32),
                     (uint32_t)nsub * 16, &bars[st]);
        }
    };
    if (tid == 0)
        for (int t = 0; t < min(kStages, ntiles); ++t) issue(t);

    X2I pp[NP];
    float2 f[NP][3];
    const int ib = i0 + warp * (32 * I) + lane;     // particle u of this thread: ib + 32 u
#pragma unroll
    for (int u = 0; u < I; ++u) {
        const bool valid = ib + 32 * u < a.n;
        const int i = min(ib + 32 * u, a.n - 1);
        const RecMix r = reinterpret_cast<const RecMix*>(a.rec)[i];
        float nm = 0.f, nax = 0.f, nay = 0.f, naz = 0.f;
        if constexpr (KIND == KIND_GRAD) {
            const float4 ai = reinterpret_cast<const float4*>(a.accrec)[i];
            nax = -ai.x; nay = -ai.y; naz = -ai.z;
            nm = valid ? -ai.w : 0.f;
        } else {
            nm = (far_on && valid) ? -a.rel[i].w : 0.f;    // -m_i for the far form
        }
        const int h = u & 1;
        X2I& q = pp[u >> 1];
        set_half(q.nxh, h, -r.hi.x); set_half(q.nyh, h, -r.hi.y); set_half(q.nzh, h, -r.hi.z);
        set_half(q.nxl, h, -r.lo.x); set_half(q.nyl, h, -r.lo.y); set_half(q.nzl, h, -r.lo.z);
        set_half(q.nA, h, valid ? -r.hi.w : 0.f);
        set_half(q.nB, h, valid ? -r.lo.w : 0.f);
        set_half(q.nm, h, nm);
        set_half(q.nax, h, nax); set_half(q.nay, h, nay); set_half(q.naz, h, naz);
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        f[p][0] = f[p][1] = f[p][2] = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 3; ++q) acc_s[(p * 3 + q) * NT + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (far_on) {
        // box of the warp's particles (FP32 high parts)
        float bl[3] = {-pp[0].nxh.x, -pp[0].nyh.x, -pp[0].nzh.x};
        float bh[3] = {bl[0], bl[1], bl[2]};
#pragma unroll
        for (int p = 0; p < NP; ++p) {
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
    const float eps2f = (float)a.eps2;
    const float2 eps2 = bc2(eps2f);
    unsigned far_visits = 0, near_visits = 0;
    bool aborted = false;
    int t_stop = ntiles;
    for (int t = 0; t < ntiles; ++t) {
        const int st = t % kStages;
        const bool ok = mbar_wait_bounded(&bars[st], (uint32_t)((t / kStages) & 1), a.timeout_ns, a.err);
        const int jt = (t0 + t) * kTileJ;
        const int cnt = min(kTileJ, a.n - jt);
        const unsigned char* base = smem + st * SB;
        const RecMix* rec = reinterpret_cast<const RecMix*>(base);
        const float4* arec = reinterpret_cast<const float4*>(base + kTileJ * kRec);
        const float4* rel_s = reinterpret_cast<const float4*>(base + kTileJ * (kRec + ACCREC));
        const float4* sub_s = reinterpret_cast<const float4*>(base + kTileJ * (kRec + ACCREC + RELB));
        if (diag) {
            // the block's own tiles: one-sided scalar loop with the self pair excluded by index
            MixI q[I];
            float fs[I][3];
#pragma unroll
            for (int u = 0; u < I; ++u) {
                const X2I& s = pp[u >> 1];
                const bool hi = (u & 1) != 0;
                q[u].xh = -(hi ? s.nxh.y : s.nxh.x); q[u].yh = -(hi ? s.nyh.y : s.nyh.x);
                q[u].zh = -(hi ? s.nzh.y : s.nzh.x); q[u].xl = -(hi ? s.nxl.y : s.nxl.x);
                q[u].yl = -(hi ? s.nyl.y : s.nyl.x); q[u].zl = -(hi ? s.nzl.y : s.nzl.x);
                q[u].ax = -(hi ? s.nax.y : s.nax.x); q[u].ay = -(hi ? s.nay.y : s.nay.x);
                q[u].az = -(hi ? s.naz.y : s.naz.x);
                fs[u][0] = fs[u][1] = fs[u][2] = 0.f;
            }
            auto own_pair = [&](int jj) {
                const float4 h = rec[jj].hi;
                const float4 l = rec[jj].lo;
                if constexpr (KIND == KIND_ACC) {
#pragma unroll
                    for (int u = 0; u < I; ++u)
                        mix_acc_pair<true>(h, l, q[u], eps2f, jt + jj == ib + 32 * u, fs[u][0], fs[u][1], fs[u][2]);
                } else {
                    const float4 aj = arec[jj];
#pragma unroll
                    for (int u = 0; u < I; ++u)
                        mix_grad_pair<true>(h, l, aj, q[u], eps2f, jt + jj == ib + 32 * u, fs[u][0], fs[u][1], fs[u][2]);
                }
            };
            auto own_flush = [&]() {
#pragma unroll
                for (int p = 0; p < NP; ++p)
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        ff_add2(acc_s[(p * 3 + q) * NT + tid], make_float2(fs[2 * p][q], fs[2 * p + 1][q]));
                        fs[2 * p][q] = fs[2 * p + 1][q] = 0.f;
                    }
            };
            if constexpr (I <= 4) {
                // few particles per thread: runs of kSymFlushJ sources as an inner loop
                for (int k0 = 0; k0 < cnt; k0 += kSymFlushJ) {
                    const int kend = min(cnt, k0 + kSymFlushJ);
                    for (int jj = k0; jj < kend; ++jj) own_pair(jj);
                    own_flush();
                }
            } else {
                // (the nested form spills at 6 and 8 particles per thread)
                for (int jj = 0; jj < cnt; ++jj) {
                    own_pair(jj);
                    if ((jj & (kSymFlushJ - 1)) == kSymFlushJ - 1 || jj == cnt - 1) own_flush();
                }
            }
        } else {
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
            for (int k0 = 0; k0 < cnt; k0 += 32) {
                const int jend = min(cnt, k0 + 32);
                if (jend - k0 < 32) {
                    // the ragged end of the last tile: checked hi/lo form
                    float2 D0[NP][3];
                    for (int jj = k0; jj < jend; jj += 4)
                        x2_group<KIND, NP, false, false>(jj, cnt, lane, warp, rec, arec, rel_s, pp, D0, eps2, f, jpart);
                    ++near_visits;
                } else if ((fmask >> (k0 >> 5)) & 1u) {
                    const float4 C = sub_s[k0 >> 5];
                    float2 D[NP][3];
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        D[p][0] = __fadd2_rn(__fadd2_rn(bc2(C.x), pp[p].nxh), pp[p].nxl);
                        D[p][1] = __fadd2_rn(__fadd2_rn(bc2(C.y), pp[p].nyh), pp[p].nyl);
                        D[p][2] = __fadd2_rn(__fadd2_rn(bc2(C.z), pp[p].nzh), pp[p].nzl);
                    }
                    for (int jj = k0; jj < jend; jj += 4)
                        x2_group<KIND, NP, true, true>(jj, cnt, lane, warp, rec, arec, rel_s, pp, D, eps2, f, jpart);
                    ++far_visits;
                } else {
                    float2 D0[NP][3];
                    for (int jj = k0; jj < jend; jj += 4)
                        x2_group<KIND, NP, false, true>(jj, cnt, lane, warp, rec, arec, rel_s, pp, D0, eps2, f, jpart);
                    ++near_visits;
                }
                if (jend == cnt || (jend % kSymFlushJ) == 0) {
#pragma unroll
                    for (int p = 0; p < NP; ++p)
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            ff_add2(acc_s[(p * 3 + q) * NT + tid], f[p][q]);
                            f[p][q] = make_float2(0.f, 0.f);
                        }
                }
            }
        }
        if (__syncthreads_or(!ok)) { aborted = true; t_stop = t; break; }
        if (!diag && tid < cnt) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                float sum = 0.f;
#pragma unroll
                for (int w = 0; w < NT / 32; ++w) sum += jpart[((size_t)w * kTileJ + tid) * 3 + q];
                red_add(a.accum + (size_t)q * a.n + jt + tid, (double)sum);
            }
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
    if (a.far_stats && lane == 0 && !diag) {
        atomicAdd(a.far_stats, (unsigned long long)far_visits);
        atomicAdd(a.far_stats + 1, (unsigned long long)near_visits);
    }
#pragma unroll
    for (int u = 0; u < I; ++u) {
        if (ib + 32 * u >= a.n) continue;
#pragma unroll
        for (int q = 0; q < 3; ++q)
        {
            const float4 v = acc_s[((u >> 1) * 3 + q) * NT + tid];
            const double sum = (u & 1) ? (double)v.y + (double)v.w : (double)v.x + (double)v.z;
            red_add(a.accum + (size_t)q * a.n + ib + 32 * u, sum);
        }
    }
}

// =================================================================================
// The pairs inside each i-block of a packed symmetric acceleration pass (the block's own
// tiles: in Morton order, each particle's nearest neighbours), evaluated in float-float
// arithmetic on the FP32 pipe instead of plain FP32.  The nearest terms carry most of the
// mixed path's rounding error: with them accurate the relative acceleration error of the
// whole sum stays within ~1e-7 (the remaining terms' FP32 roundings are independent and
// small).  Each receiver sums its block's other members one-sided; separations, r^2, the
// r^-3 factor and the products are float-float pairs (TwoSum / exact FMA products), the
// reciprocal square root refined from the hardware seed to first order in its residual
// e (e^2 ~ 2^-44 dropped); the source mass is the record's FP32 value (0.4 x 2.5 m).  The
// block's totals are added to the pass's FP64 accumulator.
__device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void ff_two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = fmaf(a, b, -p);
}

// Float-float term m_j d / r^3 of source (h, l) on receiver (xh, xl) into (ah, al).
__device__ __forceinline__ void ff_acc_pair(const float4 h, const float4 l, const float (&xh)[3],
                                            const float (&xl)[3], float eps2,
                                            float (&ah)[3], float (&al)[3]) {
    const float hj[3] = {h.x, h.y, h.z}, lj[3] = {l.x, l.y, l.z};
    float d[3], dt[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        float a, ae;
        ff_two_sum(hj[q], -xh[q], a, ae);
        const float b = __fadd_rn(__fsub_rn(lj[q], xl[q]), ae);
        ff_two_sum(a, b, d[q], dt[q]);
    }
    // r^2 = |d + dt|^2 + eps2 as (r2h, r2l)
    float px, ex, py, ey, pz, ez;
    ff_two_prod(d[0], d[0], px, ex);
    ff_two_prod(d[1], d[1], py, ey);
    ff_two_prod(d[2], d[2], pz, ez);
    float s1, e1, s2, e2, s3, e3;
    ff_two_sum(px, py, s1, e1);
    ff_two_sum(s1, pz, s2, e2);
    ff_two_sum(s2, eps2, s3, e3);
    const float cross = 2.0f * fmaf(d[0], dt[0], fmaf(d[1], dt[1], d[2] * dt[2]));
    const float low = ((e1 + e2) + (e3 + ex)) + ((ey + ez) + cross);
    float r2h, r2l;
    ff_two_sum(s3, low, r2h, r2l);
    // r^-3 = y0^3 (1 - e)^{-3/2} ~ y0^3 (1 + 1.5 e), e = 1 - r^2 y0^2 formed accurately
    const float y0 = rsqrt_hw(r2h);
    float t, te;
    ff_two_prod(y0, y0, t, te);
    float qh, qe;
    ff_two_prod(r2h, t, qh, qe);
    const float ql = fmaf(r2h, te, fmaf(r2l, t, qe));
    const float e = __fsub_rn(__fsub_rn(1.0f, qh), ql);
    float c3, c3e;
    ff_two_prod(t, y0, c3, c3e);
    c3e = fmaf(te, y0, c3e);
    // (c3 + c3e)(1 + 1.5 e) = c3 + (c3e + 1.5 e c3)
    const float r3l = fmaf(1.5f * e, c3, c3e);
    // w = m (c3 + r3l)
    const float m = 0.4f * h.w;
    float wh, we;
    ff_two_prod(m, c3, wh, we);
    we = fmaf(m, r3l, we);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        float th, tl;
        ff_two_prod(wh, d[q], th, tl);
        tl = fmaf(wh, dt[q], fmaf(we, d[q], tl));
        float sh, se;
        ff_two_sum(ah[q], th, sh, se);
        ah[q] = sh;
        al[q] = __fadd_rn(al[q], __fadd_rn(se, tl));
    }
}

// CTA (x, y) of a grid over blocks block0 + x of `bsz` consecutive members of a set of n (records
// `rec`): the members r = block start + y RPT kThreads + tid + kThreads k (k < RPT) each
// sum the other members of their block, added into accum (3 x n); sources staged through
// shared memory in tiles.
constexpr int kDiagFfRpt = 4;                           // receivers per thread
__global__ void __launch_bounds__(kThreads) sym_diag_ff_kernel(const RecMix* __restrict__ rec, int n,
                                                               int bsz, int block0, float eps2,
                                                               double* __restrict__ accum) {
    constexpr int RPT = kDiagFfRpt;
    __shared__ RecMix src[kTileJ];
    const int b0 = ((int)blockIdx.x + block0) * bsz;
    const int b1 = min(n, b0 + bsz);
    {
        const int r0 = b0 + (int)blockIdx.y * RPT * kThreads;
        if (r0 >= b1) return;                           // uniform: before any barrier
        float xh[RPT][3], xl[RPT][3], ah[RPT][3], al[RPT][3];
        int me[RPT];
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            me[u] = r0 + u * kThreads + threadIdx.x;
            const RecMix r = rec[min(me[u], b1 - 1)];
            xh[u][0] = r.hi.x; xh[u][1] = r.hi.y; xh[u][2] = r.hi.z;
            xl[u][0] = r.lo.x; xl[u][1] = r.lo.y; xl[u][2] = r.lo.z;
#pragma unroll
            for (int q = 0; q < 3; ++q) ah[u][q] = al[u][q] = 0.f;
        }
        for (int j0 = b0; j0 < b1; j0 += kTileJ) {
            const int cnt = min(kTileJ, b1 - j0);
            __syncthreads();
            if ((int)threadIdx.x < cnt) src[threadIdx.x] = rec[j0 + threadIdx.x];
            __syncthreads();
            for (int jj = 0; jj < cnt; ++jj) {
                const float4 h = src[jj].hi, l = src[jj].lo;
#pragma unroll
                for (int u = 0; u < RPT; ++u)
                    if (j0 + jj != me[u]) ff_acc_pair(h, l, xh[u], xl[u], eps2, ah[u], al[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            if (me[u] >= b1) continue;
#pragma unroll
            for (int q = 0; q < 3; ++q)
                red_add(accum + (size_t)q * n + me[u], (double)ah[u][q] + (double)al[u][q]);
        }
    }
}

cudaError_t launch_sym_diag_ff(const void* rec, int n, int bsz, double eps2, double* accum,
                               cudaStream_t s, int part, int nparts) {
    if (n <= 0 || bsz <= 0) return cudaSuccess;
    const int nb = (n + bsz - 1) / bsz;
    // the blocks of the same share as the symmetric launch (blocks of bsz = bt tiles)
    int b0, b1;
    sym_part_blocks(nb, bsz / kTileJ, (n + kTileJ - 1) / kTileJ, part, nparts, b0, b1);
    if (b1 <= b0) return cudaSuccess;
    const int sweeps = (bsz + kDiagFfRpt * kThreads - 1) / (kDiagFfRpt * kThreads);
    const dim3 grid((unsigned)(b1 - b0), (unsigned)sweeps);
    { sym_diag_ff_kernel<<<grid, kThreads, 0, s>>>(reinterpret_cast<const RecMix*>(rec), n, bsz, b0,
                                                   (float)eps2, accum); note_launch(); }
    return cudaGetLastError();
}

// =================================================================================
// Bipartite packed symmetric kernel: the two directions of a cross-level pass (Sect. 2.2,
// S <- F and F <- S of disjoint sets) with every S-F pair evaluated once and added to both
// particles (Newton's third law; for the gradient, the inter-level accelerations a_S of
// S <- F and a_F of F <- S make the pair term antisymmetric up to the masses).  Work
// items (blockIdx.x = b * nchunk + c): i-block b of 256 I particles of S in registers
// against chunk c of `chunk` source tiles of F.  Hi/lo (near) form only: the sets are in
// no spatial order.  Both sides are added into FP64 accumulators (red.global.add); two
// finalize launches then apply the epilogues.
struct CrossArgs {
    const void* irec; const void* iacc;   // S: position / accel records, n_i
    const void* jrec; const void* jacc;   // F: position / accel records, n_j
    int n_i, n_j;
    int chunk, nchunk;
    double eps2;
    double* acc_i;      // 3 x n_i, zeroed before the launch
    double* acc_j;      // 3 x n_j, zeroed before the launch
    int* err;
    long long timeout_ns;
    // far-tile path (mixed; null rel: never taken): F's records relative to the centres of
    // their 32-record sub-tiles (w = mass) and the sub-tiles' (centre, radius)
    const float4* rel;
    const float4* sub;
    float far_k2;
};

template <int KIND, int I, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) cross_mixed_x2_kernel(const CrossArgs a) {
    static_assert(I % 2 == 0, "particles are handled in packed pairs");
    constexpr int NP = I / 2;
    constexpr int ACCREC = SymCfg<FSI_MIXED, KIND>::ACCREC;
    constexpr int RELB = 16;
    constexpr int SUBB = (kTileJ / 32) * 16;
    constexpr int SB = kTileJ * (kRec + ACCREC + RELB) + SUBB;
    constexpr int JPART = SymCfg<FSI_MIXED, KIND>::JPART;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[kStages];
    __shared__ float wbox[kThreads / 32][6];
    float* jpart = reinterpret_cast<float*>(smem + kStages * SB);
    float4* acc_s = reinterpret_cast<float4*>(smem + kStages * SB + JPART);

    const int b = blockIdx.x / a.nchunk;
    const int c = blockIdx.x % a.nchunk;
    const int ntj = (a.n_j + kTileJ - 1) / kTileJ;
    const int t0 = c * a.chunk;
    const int t1 = min(t0 + a.chunk, ntj);
    if (t0 >= t1) return;                       // uniform: before any barrier
    const int ntiles = t1 - t0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i0 = b * (kThreads * I);
    const bool far_on = a.rel != nullptr;

    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) mbar_init(&bars[st], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int t) {
        const int st = t % kStages;
        const int jt = (t0 + t) * kTileJ;
        const int cnt = min(kTileJ, a.n_j - jt);
        const int nsub = (cnt + 31) >> 5;
        unsigned char* base = smem + st * SB;
        mbar_arrive_expect_tx(&bars[st], (uint32_t)cnt * (kRec + ACCREC) +
                                             (far_on ? (uint32_t)(cnt * 16 + nsub * 16) : 0u));
        bulk_g2s(base, (const unsigned char*)a.jrec + (size_t)jt * kRec, (uint32_t)cnt * kRec, &bars[st]);
        if (ACCREC)
            bulk_g2s(base + kTileJ * kRec, (const unsigned char*)a.jacc + (size_t)jt * ACCREC,
                     (uint32_t)cnt * ACCREC, &bars[st]);
        if (far_on) {
            bulk_g2s(base + kTileJ * (kRec + ACCREC), (const unsigned char*)(a.rel + jt),
                     (uint32_t)cnt * 16, &bars[st]);
            bulk_g2s(base + kTileJ * (kRec + ACCREC + RELB), (const unsigned char*)(a.sub + jt / 32),
                     (uint32_t)nsub * 16, &bars[st]);
        }
    };
    if (tid == 0)
        for (int t = 0; t < min(kStages, ntiles); ++t) issue(t);

    X2I pp[NP];
    float2 f[NP][3];
    const int ib = i0 + warp * (32 * I) + lane;     // particle u of this thread: ib + 32 u
#pragma unroll
    for (int u = 0; u < I; ++u) {
        const bool valid = ib + 32 * u < a.n_i;
        const int i = min(ib + 32 * u, a.n_i - 1);
        const RecMix r = reinterpret_cast<const RecMix*>(a.irec)[i];
        float nm = 0.f, nax = 0.f, nay = 0.f, naz = 0.f;
        if constexpr (KIND == KIND_GRAD) {
            const float4 ai = reinterpret_cast<const float4*>(a.iacc)[i];
            nax = -ai.x; nay = -ai.y; naz = -ai.z;
            nm = valid ? -ai.w : 0.f;
        } else {
            // -m_i for the far form, from the record's 2.5 m
            nm = (far_on && valid) ? -(float)(0.4 * (double)r.hi.w) : 0.f;
        }
        const int h = u & 1;
        X2I& q = pp[u >> 1];
        set_half(q.nxh, h, -r.hi.x); set_half(q.nyh, h, -r.hi.y); set_half(q.nzh, h, -r.hi.z);
        set_half(q.nxl, h, -r.lo.x); set_half(q.nyl, h, -r.lo.y); set_half(q.nzl, h, -r.lo.z);
        // a receiver past the end contributes nothing to the source side
        set_half(q.nA, h, valid ? -r.hi.w : 0.f);
        set_half(q.nB, h, valid ? -r.lo.w : 0.f);
        set_half(q.nm, h, nm);
        set_half(q.nax, h, nax); set_half(q.nay, h, nay); set_half(q.naz, h, naz);
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        f[p][0] = f[p][1] = f[p][2] = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 3; ++q) acc_s[(p * 3 + q) * kThreads + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (far_on) {
        // box of the warp's particles (FP32 high parts)
        float bl[3] = {-pp[0].nxh.x, -pp[0].nyh.x, -pp[0].nzh.x};
        float bh[3] = {bl[0], bl[1], bl[2]};
#pragma unroll
        for (int p = 0; p < NP; ++p) {
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
    const float2 eps2 = bc2((float)a.eps2);
    float2 D0[NP][3];                           // unused by the near form
    bool aborted = false;
    int t_stop = ntiles;
    for (int t = 0; t < ntiles; ++t) {
        const int st = t % kStages;
        const bool ok = mbar_wait_bounded(&bars[st], (uint32_t)((t / kStages) & 1), a.timeout_ns, a.err);
        const int jt = (t0 + t) * kTileJ;
        const int cnt = min(kTileJ, a.n_j - jt);
        const unsigned char* base = smem + st * SB;
        const RecMix* rec = reinterpret_cast<const RecMix*>(base);
        const float4* arec = reinterpret_cast<const float4*>(base + kTileJ * kRec);
        const float4* rel_s = reinterpret_cast<const float4*>(base + kTileJ * (kRec + ACCREC));
        const float4* sub_s = reinterpret_cast<const float4*>(base + kTileJ * (kRec + ACCREC + RELB));
        unsigned fmask = 0;
        if (far_on) {
            // far test of this warp's box against each full 32-record sub-tile (warp-uniform)
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
        for (int k0 = 0; k0 < cnt; k0 += 32) {
            const int jend = min(cnt, k0 + 32);
            if (jend - k0 < 32) {
                for (int jj = k0; jj < jend; jj += 4)
                    x2_group<KIND, NP, false, false>(jj, cnt, lane, warp, rec, arec, rel_s, pp, D0, eps2, f, jpart);
            } else if ((fmask >> (k0 >> 5)) & 1u) {
                const float4 C = sub_s[k0 >> 5];
                float2 D[NP][3];
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    D[p][0] = __fadd2_rn(__fadd2_rn(bc2(C.x), pp[p].nxh), pp[p].nxl);
                    D[p][1] = __fadd2_rn(__fadd2_rn(bc2(C.y), pp[p].nyh), pp[p].nyl);
                    D[p][2] = __fadd2_rn(__fadd2_rn(bc2(C.z), pp[p].nzh), pp[p].nzl);
                }
                for (int jj = k0; jj < jend; jj += 4)
                    x2_group<KIND, NP, true, true>(jj, cnt, lane, warp, rec, arec, rel_s, pp, D, eps2, f, jpart);
            } else {
                for (int jj = k0; jj < jend; jj += 4)
                    x2_group<KIND, NP, false, true>(jj, cnt, lane, warp, rec, arec, rel_s, pp, D0, eps2, f, jpart);
            }
            if (jend == cnt || (jend % kSymFlushJ) == 0) {
#pragma unroll
                for (int p = 0; p < NP; ++p)
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        ff_add2(acc_s[(p * 3 + q) * kThreads + tid], f[p][q]);
                        f[p][q] = make_float2(0.f, 0.f);
                    }
            }
        }
        if (__syncthreads_or(!ok)) { aborted = true; t_stop = t; break; }
        if (tid < cnt) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                float sum = 0.f;
#pragma unroll
                for (int w = 0; w < kThreads / 32; ++w) sum += jpart[((size_t)w * kTileJ + tid) * 3 + q];
                red_add(a.acc_j + (size_t)q * a.n_j + jt + tid, (double)sum);
            }
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
#pragma unroll
    for (int u = 0; u < I; ++u) {
        if (ib + 32 * u >= a.n_i) continue;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float4 v = acc_s[((u >> 1) * 3 + q) * kThreads + tid];
            const double sum = (u & 1) ? (double)v.y + (double)v.w : (double)v.x + (double)v.z;
            red_add(a.acc_i + (size_t)q * a.n_i + ib + 32 * u, sum);
        }
    }
}

template <int KIND>
static cudaError_t launch_cross_x2_t(const CrossArgs& a, cudaStream_t s) {
    constexpr int I = 4;
    constexpr int SB = kTileJ * (kRec + SymCfg<FSI_MIXED, KIND>::ACCREC + 16) + (kTileJ / 32) * 16;
    constexpr int SMEM = kStages * SB + SymCfg<FSI_MIXED, KIND>::JPART + (I / 2) * 3 * kThreads * 16;
    static std::atomic<unsigned long long> attr_dev{0};
    {
        const cudaError_t e = smem_attr_once(cross_mixed_x2_kernel<KIND, I, 2>, SMEM, attr_dev);
        if (e != cudaSuccess) return e;
    }
    const long long nb = (a.n_i + kThreads * I - 1) / (kThreads * I);
    const long long grid = nb * a.nchunk;
    if (grid <= 0 || grid > 2147483647LL) return cudaErrorInvalidValue;
    { cross_mixed_x2_kernel<KIND, I, 2><<<(unsigned)grid, kThreads, SMEM, s>>>(a); note_launch(); }
    return cudaGetLastError();
}

// FP64 form of the bipartite kernel: the symmetric FP64 pair terms of the single-set
// kernel (I = 2 particles of S per thread), the F side carried around the warp
// (f64_rotate32).
template <int KIND, int I>
__global__ void __launch_bounds__(kThreads, 2) cross_f64_kernel(const CrossArgs a) {
    constexpr int ACCREC = SymCfg<FSI_FP64, KIND>::ACCREC;
    constexpr int SB = SymCfg<FSI_FP64, KIND>::SB;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[kStages];
    double* jpart = reinterpret_cast<double*>(smem + kStages * SB);
    const int b = blockIdx.x / a.nchunk;
    const int c = blockIdx.x % a.nchunk;
    const int ntj = (a.n_j + kTileJ - 1) / kTileJ;
    const int t0 = c * a.chunk;
    const int t1 = min(t0 + a.chunk, ntj);
    if (t0 >= t1) return;                       // uniform: before any barrier
    const int ntiles = t1 - t0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i0 = b * (kThreads * I);
    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) mbar_init(&bars[st], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int t) {
        const int st = t % kStages;
        const int jt = (t0 + t) * kTileJ;
        const int cnt = min(kTileJ, a.n_j - jt);
        unsigned char* base = smem + st * SB;
        mbar_arrive_expect_tx(&bars[st], (uint32_t)cnt * (kRec + ACCREC));
        bulk_g2s(base, (const unsigned char*)a.jrec + (size_t)jt * kRec, (uint32_t)cnt * kRec, &bars[st]);
        if (ACCREC)
            bulk_g2s(base + kTileJ * kRec, (const unsigned char*)a.jacc + (size_t)jt * ACCREC,
                     (uint32_t)cnt * ACCREC, &bars[st]);
    };
    if (tid == 0)
        for (int t = 0; t < min(kStages, ntiles); ++t) issue(t);
    double acc64[I][3];
    bool valid[I];
    int my_i[I];
    SymF64I pi[I];
#pragma unroll
    for (int u = 0; u < I; ++u) {
        acc64[u][0] = acc64[u][1] = acc64[u][2] = 0.0;
        my_i[u] = i0 + u * kThreads + tid;
        valid[u] = my_i[u] < a.n_i;
        const int i = min(my_i[u], a.n_i - 1);
        const D4 r = reinterpret_cast<const D4*>(a.irec)[i];
        pi[u].x = r.x; pi[u].y = r.y; pi[u].z = r.z;
        pi[u].nm = valid[u] ? -r.w : 0.0;       // a receiver past the end adds nothing to F
        if constexpr (KIND == KIND_GRAD) {
            const D4 ai = reinterpret_cast<const D4*>(a.iacc)[i];
            pi[u].ax = ai.x; pi[u].ay = ai.y; pi[u].az = ai.z;
        } else {
            pi[u].ax = pi[u].ay = pi[u].az = 0.0;
        }
    }
    bool aborted = false;
    int t_stop = ntiles;
    for (int t = 0; t < ntiles; ++t) {
        const int st = t % kStages;
        const bool ok = mbar_wait_bounded(&bars[st], (uint32_t)((t / kStages) & 1), a.timeout_ns, a.err);
        const int jt = (t0 + t) * kTileJ;
        const int cnt = min(kTileJ, a.n_j - jt);
        const unsigned char* base = smem + st * SB;
        const D4* rec = reinterpret_cast<const D4*>(base);
        const D4* arec = reinterpret_cast<const D4*>(base + kTileJ * kRec);
        for (int jj = 0; jj < cnt; jj += 32) {
            double tot[3];
            if (jj + 32 <= cnt) f64_rotate32<KIND, I, true>(rec, arec, jj, cnt, lane, pi, a.eps2, acc64, tot);
            else f64_rotate32<KIND, I, false>(rec, arec, jj, cnt, lane, pi, a.eps2, acc64, tot);
            const int jl = jj + lane;
            if (jl < cnt) {
                double* dst = jpart + ((size_t)warp * kTileJ + jl) * 3;
                dst[0] = tot[0]; dst[1] = tot[1]; dst[2] = tot[2];
            }
        }
        if (__syncthreads_or(!ok)) { aborted = true; t_stop = t; break; }
        if (tid < cnt) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                double sum = 0.0;
#pragma unroll
                for (int w = 0; w < kThreads / 32; ++w) sum += jpart[((size_t)w * kTileJ + tid) * 3 + q];
                red_add(a.acc_j + (size_t)q * a.n_j + jt + tid, sum);
            }
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
#pragma unroll
    for (int u = 0; u < I; ++u) {
        if (!valid[u]) continue;
#pragma unroll
        for (int q = 0; q < 3; ++q) red_add(a.acc_i + (size_t)q * a.n_i + my_i[u], acc64[u][q]);
    }
}

template <int KIND>
static cudaError_t launch_cross_f64_t(const CrossArgs& a, cudaStream_t s) {
    constexpr int I = 2;
    constexpr int SMEM = SymCfg<FSI_FP64, KIND>::SMEM;
    static std::atomic<unsigned long long> attr_dev{0};
    {
        const cudaError_t e = smem_attr_once(cross_f64_kernel<KIND, I>, SMEM, attr_dev);
        if (e != cudaSuccess) return e;
    }
    const long long nb = (a.n_i + kThreads * I - 1) / (kThreads * I);
    const long long grid = nb * a.nchunk;
    if (grid <= 0 || grid > 2147483647LL) return cudaErrorInvalidValue;
    { cross_f64_kernel<KIND, I><<<(unsigned)grid, kThreads, SMEM, s>>>(a); note_launch(); }
    return cudaGetLastError();
}

int cross_block_size(int precision) { return kThreads * (precision == FSI_MIXED ? 4 : 2); }

cudaError_t launch_cross_pair(int precision, int kind, const void* irec, const void* iacc,
                              int n_i, const void* jrec, const void* jacc, int n_j, double eps2,
                              int chunk, double* acc_i, double* acc_j, int* err,
                              long long timeout_ns, cudaStream_t s, const SymFar* far) {
    if (n_i <= 0 || n_j <= 0) return cudaErrorInvalidValue;
    CrossArgs a{};
    a.irec = irec; a.iacc = iacc; a.jrec = jrec; a.jacc = jacc;
    a.n_i = n_i; a.n_j = n_j;
    const int ntj = (n_j + kTileJ - 1) / kTileJ;
    a.chunk = std::max(1, std::min(chunk, ntj));
    a.nchunk = (ntj + a.chunk - 1) / a.chunk;
    a.eps2 = eps2; a.acc_i = acc_i; a.acc_j = acc_j; a.err = err; a.timeout_ns = timeout_ns;
    if (far && precision == FSI_MIXED) {
        a.rel = reinterpret_cast<const float4*>(far->rel);
        a.sub = reinterpret_cast<const float4*>(far->sub);
        a.far_k2 = far->k2;
    }
    if (precision == FSI_FP64)
        return kind == KIND_ACC ? launch_cross_f64_t<KIND_ACC>(a, s) : launch_cross_f64_t<KIND_GRAD>(a, s);
    return kind == KIND_ACC ? launch_cross_x2_t<KIND_ACC>(a, s) : launch_cross_x2_t<KIND_GRAD>(a, s);
}

// MINB: resident CTAs per SM the register budget is sized for (2: 128 registers per
// thread, 1: 255).
template <int KIND, int I, int MINB, int NT = kThreads>
static cudaError_t launch_sym_x2(SymArgs a, cudaStream_t s) {
    constexpr int SB = kTileJ * (kRec + SymCfg<FSI_MIXED, KIND>::ACCREC + 16) + (kTileJ / 32) * 16;
    constexpr int JPART = (NT / 32) * kTileJ * 3 * (int)sizeof(float);
    constexpr int SMEM = kStages * SB + JPART + I * 3 * NT * (int)sizeof(double);
    static std::atomic<unsigned long long> attr_dev{0};
    {
        const cudaError_t e = smem_attr_once(sym_mixed_x2_kernel<KIND, I, MINB, NT>, SMEM, attr_dev);
        if (e != cudaSuccess) return e;
    }
    // work items per i-block: its own tiles, then chunks of the tiles above it
    constexpr int BT = NT * I / kTileJ;
    const int ntj = (a.n + kTileJ - 1) / kTileJ;
    const int above = ntj > BT ? ntj - BT : 0;
    a.nchunk = (above + a.chunk - 1) / a.chunk;
    const int nb = (a.n + NT * I - 1) / (NT * I);
    int b0, b1;
    sym_part_blocks(nb, BT, ntj, a.part, a.nparts, b0, b1);
    a.item0 = b0 * (1 + a.nchunk);
    const long long grid = (long long)(b1 - b0) * (1 + a.nchunk);
    if (grid > 2147483647LL) return cudaErrorInvalidValue;
    if (grid == 0) return cudaSuccess;
    { sym_mixed_x2_kernel<KIND, I, MINB, NT><<<(unsigned)grid, NT, SMEM, s>>>(a); note_launch(); }
    return cudaGetLastError();
}

template <int KIND, int I, bool FAR>
static cudaError_t launch_sym_v2(SymArgs a, cudaStream_t s) {
    constexpr int SB = kTileJ * (kRec + SymCfg<FSI_MIXED, KIND>::ACCREC + (FAR ? 16 : 0)) +
                       (FAR ? (kTileJ / 32) * 16 : 0);
    constexpr int SMEM = kStages * SB + SymCfg<FSI_MIXED, KIND>::JPART + I * 3 * kThreads * (int)sizeof(double);
    static std::atomic<unsigned long long> attr_dev{0};
    {
        const cudaError_t e = smem_attr_once(sym_mixed_v2_kernel<KIND, I, FAR>, SMEM, attr_dev);
        if (e != cudaSuccess) return e;
    }
    const int nb = (a.n + kThreads * I - 1) / (kThreads * I);
    int b0, b1;
    sym_part_blocks(nb, I, (a.n + kTileJ - 1) / kTileJ, a.part, a.nparts, b0, b1);
    a.item0 = b0 * (1 + a.nchunk);
    const long long grid = (long long)(b1 - b0) * (1 + a.nchunk);
    if (grid > 2147483647LL) return cudaErrorInvalidValue;
    if (grid == 0) return cudaSuccess;
    { sym_mixed_v2_kernel<KIND, I, FAR><<<(unsigned)grid, kThreads, SMEM, s>>>(a); note_launch(); }
    return cudaGetLastError();
}

template <int P, int KIND, int I>
static cudaError_t launch_sym_one(SymArgs a, cudaStream_t s) {
    constexpr int SMEM = SymCfg<P, KIND>::SMEM;
    static std::atomic<unsigned long long> attr_dev{0};
    {
        const cudaError_t e = smem_attr_once(sym_pair_kernel<P, KIND, I>, SMEM, attr_dev);
        if (e != cudaSuccess) return e;
    }
    const int nb = (a.n + kThreads * I - 1) / (kThreads * I);
    int b0, b1;
    sym_part_blocks(nb, I, (a.n + kTileJ - 1) / kTileJ, a.part, a.nparts, b0, b1);
    a.item0 = b0 * (1 + a.nchunk);
    const long long grid = (long long)(b1 - b0) * (1 + a.nchunk);
    if (grid > 2147483647LL) return cudaErrorInvalidValue;
    if (grid == 0) return cudaSuccess;
    { sym_pair_kernel<P, KIND, I><<<(unsigned)grid, kThreads, SMEM, s>>>(a); note_launch(); }
    return cudaGetLastError();
}

template <int P, int KIND>
static cudaError_t launch_sym_ipt(int ipt, const SymArgs& a, cudaStream_t s) {
    switch (ipt) {
        case 1: return launch_sym_one<P, KIND, 1>(a, s);
        case 2: return launch_sym_one<P, KIND, 2>(a, s);
        case 3: return launch_sym_one<P, KIND, 3>(a, s);
        case 4: return launch_sym_one<P, KIND, 4>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sym_pair(int precision, int kind, int ipt, const void* rec, const void* accrec,
                            int n, double eps2, int chunk, double* accum, int* err,
                            long long timeout_ns, const SymFar* far, cudaStream_t s, bool skip_diag,
                            int part, int nparts) {
    if (n <= 0) return cudaSuccess;
    if (nparts < 1 || part < 0 || part >= nparts) return cudaErrorInvalidValue;
    SymArgs a{};
    a.rec = rec; a.accrec = accrec; a.n = n; a.eps2 = eps2; a.accum = accum; a.err = err;
    a.timeout_ns = timeout_ns;
    a.part = part;
    a.nparts = nparts;
    a.skip_diag = skip_diag && precision == FSI_MIXED && (ipt & 128) ? 1 : 0;
    if (far && (ipt & 64)) {
        a.rel = reinterpret_cast<const float4*>(far->rel);
        a.sub = reinterpret_cast<const float4*>(far->sub);
        a.far_k2 = far->k2;
        a.far_stats = far->stats;
    }
    const int I = ipt & 15;
    const int ntj = (n + kTileJ - 1) / kTileJ;
    a.chunk = chunk > 0 ? chunk : 1;
    const int above = ntj > I ? ntj - I : 0;       // most tiles above any block (block 0)
    a.nchunk = (above + a.chunk - 1) / a.chunk;
    if (precision == FSI_MIXED && (ipt & 128) && (ipt & 512)) {
        // packed form with CTAs of 384 threads (12 warps per SM, ~170 registers)
        switch (I * 2 + kind) {
            case 4 * 2 + KIND_ACC: return launch_sym_x2<KIND_ACC, 4, 1, 384>(a, s);
            case 4 * 2 + KIND_GRAD: return launch_sym_x2<KIND_GRAD, 4, 1, 384>(a, s);
            case 6 * 2 + KIND_ACC: return launch_sym_x2<KIND_ACC, 6, 1, 384>(a, s);
            case 6 * 2 + KIND_GRAD: return launch_sym_x2<KIND_GRAD, 6, 1, 384>(a, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if (precision == FSI_MIXED && (ipt & 128)) {
        // packed form; bit 16 selects the one-CTA-per-SM register budget
        switch ((ipt & 16 ? 64 : 0) + I * 2 + kind) {
            case 2 * 2 + KIND_ACC: return launch_sym_x2<KIND_ACC, 2, 2>(a, s);
            case 2 * 2 + KIND_GRAD: return launch_sym_x2<KIND_GRAD, 2, 2>(a, s);
            case 4 * 2 + KIND_ACC: return launch_sym_x2<KIND_ACC, 4, 2>(a, s);
            case 6 * 2 + KIND_ACC: return launch_sym_x2<KIND_ACC, 6, 2>(a, s);
            case 4 * 2 + KIND_GRAD: return launch_sym_x2<KIND_GRAD, 4, 2>(a, s);
            case 6 * 2 + KIND_GRAD: return launch_sym_x2<KIND_GRAD, 6, 2>(a, s);
            case 64 + 6 * 2 + KIND_ACC: return launch_sym_x2<KIND_ACC, 6, 1>(a, s);
            case 64 + 6 * 2 + KIND_GRAD: return launch_sym_x2<KIND_GRAD, 6, 1>(a, s);
            case 64 + 8 * 2 + KIND_ACC: return launch_sym_x2<KIND_ACC, 8, 1>(a, s);
            case 64 + 8 * 2 + KIND_GRAD: return launch_sym_x2<KIND_GRAD, 8, 1>(a, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if (precision == FSI_MIXED && (ipt & 64)) {
        switch (I * 2 + kind) {
            case 4 * 2 + KIND_ACC: return launch_sym_v2<KIND_ACC, 4, true>(a, s);
            case 5 * 2 + KIND_ACC: return launch_sym_v2<KIND_ACC, 5, true>(a, s);
            case 3 * 2 + KIND_GRAD: return launch_sym_v2<KIND_GRAD, 3, true>(a, s);
            case 4 * 2 + KIND_GRAD: return launch_sym_v2<KIND_GRAD, 4, true>(a, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if (precision == FSI_MIXED && (ipt & 32)) {
        switch (I * 2 + kind) {
            case 4 * 2 + KIND_ACC: return launch_sym_v2<KIND_ACC, 4, false>(a, s);
            case 5 * 2 + KIND_ACC: return launch_sym_v2<KIND_ACC, 5, false>(a, s);
            case 6 * 2 + KIND_ACC: return launch_sym_v2<KIND_ACC, 6, false>(a, s);
            case 4 * 2 + KIND_GRAD: return launch_sym_v2<KIND_GRAD, 4, false>(a, s);
            case 5 * 2 + KIND_GRAD: return launch_sym_v2<KIND_GRAD, 5, false>(a, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if (precision == FSI_MIXED)
        return kind == KIND_ACC ? launch_sym_ipt<FSI_MIXED, KIND_ACC>(I, a, s)
                                : launch_sym_ipt<FSI_MIXED, KIND_GRAD>(I, a, s);
    return kind == KIND_ACC ? launch_sym_ipt<FSI_FP64, KIND_ACC>(I, a, s)
                            : launch_sym_ipt<FSI_FP64, KIND_GRAD>(I, a, s);
}

// ---------------------------------------------------------------------------------
template <int P, int KIND, int I, int FF>
static cudaError_t launch_one(const PairArgs& a, int split, cudaStream_t s) {
    constexpr int SMEM = kStages * stage_bytes(Cfg<P, KIND>::ACCREC);
    static std::atomic<unsigned long long> attr_dev{0};
    {
        const cudaError_t e = smem_attr_once(pair_kernel<P, KIND, I, FF>, SMEM, attr_dev);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((a.n_i + kThreads * I - 1) / (kThreads * I), split);
    { pair_kernel<P, KIND, I, FF><<<grid, kThreads, SMEM, s>>>(a); note_launch(); }
    return cudaGetLastError();
}

// A variant is encoded as ipt + 16 * ff.
template <int P, int KIND>
static cudaError_t launch_variant(int v, const PairArgs& a, int split, cudaStream_t s) {
    switch (v) {
        case 1: return launch_one<P, KIND, 1, 0>(a, split, s);
        case 2: return launch_one<P, KIND, 2, 0>(a, split, s);
        case 3: return launch_one<P, KIND, 3, 0>(a, split, s);
        case 4: return launch_one<P, KIND, 4, 0>(a, split, s);
        case 16 + 2: return launch_one<P, KIND, 2, 1>(a, split, s);
        case 16 + 3: return launch_one<P, KIND, 3, 1>(a, split, s);
        case 16 + 4: return launch_one<P, KIND, 4, 1>(a, split, s);
        case 32 + 4:
            if constexpr (P == FSI_MIXED) return launch_one<P, KIND, 4, 2>(a, split, s);
            else return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

int pair_variants(int precision, int kind, int* out) {
    (void)kind;
    int n = 0;
    if (precision == FSI_MIXED) {
        for (int ipt = 2; ipt <= 4; ++ipt) out[n++] = ipt;
        for (int ipt = 2; ipt <= 4; ++ipt) out[n++] = 16 + ipt;
        out[n++] = 32 + 4;      // packed FP32x2 (two pairs of active particles per thread)
    } else {
        out[n++] = 1; out[n++] = 2; out[n++] = 3;
    }
    return n;
}

int sym_variants(int precision, int kind, int* out) {
    int n = 0;
    if (precision == FSI_MIXED) {
        for (int ipt = 2; ipt <= 4; ++ipt) out[n++] = ipt;
        out[n++] = 32 + 4;
        out[n++] = 32 + 5;
        if (kind == KIND_ACC) out[n++] = 32 + 6;
        // second form with the far-tile path
        if (kind == KIND_ACC) { out[n++] = 96 + 4; out[n++] = 96 + 5; }
        else { out[n++] = 96 + 3; out[n++] = 96 + 4; }
        // packed FP32x2 form (far-tile path included)
        out[n++] = 224 + 2;
        out[n++] = 224 + 4;
        out[n++] = 224 + 6;
        out[n++] = 240 + 6;     // one CTA per SM (255 registers)
        out[n++] = 240 + 8;
        out[n++] = 752 + 4;     // one CTA of 384 threads per SM (~170 registers)
        out[n++] = 752 + 6;
    } else {
        out[n++] = 1; out[n++] = 2; out[n++] = 3;
    }
    return n;
}

int pair_default_ipt(int precision, int kind) {
    return precision == FSI_MIXED ? (kind == KIND_ACC ? 4 : 2) : 2;
}

int variant_ipt(int v) { return v & 15; }

int sym_block_particles(int v) { return ((v & 128) && (v & 512) ? 384 : kThreads) * (v & 15); }

cudaError_t launch_pair(int precision, int kind, int ipt, const PairArgs& a, int split,
                        cudaStream_t s) {
    if (a.n_i <= 0) return cudaSuccess;
    if (precision == FSI_MIXED)
        return kind == KIND_ACC ? launch_variant<FSI_MIXED, KIND_ACC>(ipt, a, split, s)
                                : launch_variant<FSI_MIXED, KIND_GRAD>(ipt, a, split, s);
    if (ipt >= 16) return cudaErrorInvalidValue;
    return kind == KIND_ACC ? launch_variant<FSI_FP64, KIND_ACC>(ipt, a, split, s)
                            : launch_variant<FSI_FP64, KIND_GRAD>(ipt, a, split, s);
}

template <int P, int KIND>
cudaError_t launch_wide_t(bool diag, const PairArgs& a, int lg, int split, cudaStream_t s) {
    const long long threads = (long long)a.n_i << lg;
    const dim3 grid((unsigned)((threads + kThreads - 1) / kThreads), (unsigned)split);
    if (diag) { wide_pair_kernel<P, KIND, true><<<grid, kThreads, 0, s>>>(a, lg); note_launch(); }
    else { wide_pair_kernel<P, KIND, false><<<grid, kThreads, 0, s>>>(a, lg); note_launch(); }
    return cudaGetLastError();
}

template <int P, int KIND>
cudaError_t launch_wide2_t(const PairArgs& a, const PairArgs& b, int lga, int lgb, cudaStream_t s) {
    const long long ca = (((long long)a.n_i << lga) + kThreads - 1) / kThreads;
    const long long cb = (((long long)b.n_i << lgb) + kThreads - 1) / kThreads;
    { wide_pair2_kernel<P, KIND><<<(unsigned)(ca + cb), kThreads, 0, s>>>(a, b, lga, lgb, (int)ca); note_launch(); }
    return cudaGetLastError();
}

cudaError_t launch_wide_pair2(int precision, int kind, const PairArgs& a, const PairArgs& b,
                              int lga, int lgb, cudaStream_t s) {
    if (a.n_i <= 0 || b.n_i <= 0) return cudaErrorInvalidValue;
    if (lga < 0 || lga > 5 || lgb < 0 || lgb > 5) return cudaErrorInvalidValue;
    if (precision == FSI_MIXED)
        return kind == KIND_ACC ? launch_wide2_t<FSI_MIXED, KIND_ACC>(a, b, lga, lgb, s)
                                : launch_wide2_t<FSI_MIXED, KIND_GRAD>(a, b, lga, lgb, s);
    return kind == KIND_ACC ? launch_wide2_t<FSI_FP64, KIND_ACC>(a, b, lga, lgb, s)
                            : launch_wide2_t<FSI_FP64, KIND_GRAD>(a, b, lga, lgb, s);
}

cudaError_t launch_wide_pair(int precision, int kind, bool diag, const PairArgs& a, int lg,
                             int split, cudaStream_t s) {
    if (a.n_i <= 0) return cudaSuccess;
    if (lg < 0 || lg > 5 || split < 1 || split > 65535) return cudaErrorInvalidValue;
    if (precision == FSI_MIXED)
        return kind == KIND_ACC ? launch_wide_t<FSI_MIXED, KIND_ACC>(diag, a, lg, split, s)
                                : launch_wide_t<FSI_MIXED, KIND_GRAD>(diag, a, lg, split, s);
    return kind == KIND_ACC ? launch_wide_t<FSI_FP64, KIND_ACC>(diag, a, lg, split, s)
                            : launch_wide_t<FSI_FP64, KIND_GRAD>(diag, a, lg, split, s);
}

cudaError_t launch_finalize_p(int precision, const PairArgs& a, int split, cudaStream_t s) {
    if (a.n_i <= 0) return cudaSuccess;
    const int b = 256;
    if (precision == FSI_MIXED)
        { finalize_kernel<FSI_MIXED><<<(a.n_i + b - 1) / b, b, 0, s>>>(a, split); note_launch(); }
    else
        { finalize_kernel<FSI_FP64><<<(a.n_i + b - 1) / b, b, 0, s>>>(a, split); note_launch(); }
    return cudaGetLastError();
}

}  // namespace fsi
