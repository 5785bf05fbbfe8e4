// batch_kernels.cu -- FSI cycles of an ensemble of independent clusters of uneven size in
// ONE persistent launch.
//
// Each cluster k (particles [off_k, off_k + n_k) of the concatenated SoA arrays) evolves
// on its own (Sect. 2.1, Eq. fsi-cycle).  The launch runs a sequence of phases:
//   phase 0              pack the records of every cluster from x
//   phase 1              acc pass on rec0 -> kick h/6, drift h/2, records -> rec1
//   per step s (3 phases)
//     1 + 3s + 1         acc pass on rec1 -> a (FP64) and accel records
//     1 + 3s + 2         grad pass on rec1 -> kick 2h/3 (a + h^2/24 G), drift h/2 -> rec0
//     1 + 3s + 3         acc pass on rec0 -> kick h/3 and drift h/2 -> rec1 (between steps)
//                                          or kick h/6 (after the last step)
// A work item is (phase, cluster, i-block of 256*I particles); items are handed out in
// phase-major order by an atomic counter (clusters by decreasing size within a phase),
// and an item of phase p of cluster k first waits until all items of phase p-1 of
// cluster k have signalled.  Every wait is bounded: on timeout the launch latches
// FSI_ERR_TIMEOUT, raises an abort flag that every CTA checks, and returns.  Since an
// item only waits on items handed out before it, and those are held by resident CTAs
// that never wait on later items, the schedule cannot deadlock.
//
// Cross-phase data written by other SMs is read with L1-bypassing loads (ld.global.cg).
#include <algorithm>

#include "fsi_internal.cuh"
#include "pair_math.cuh"
#include "sym_x2.cuh"

namespace fsi {

constexpr int kBatchThreads = 256;
constexpr int kBatchTile = 256;

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <class T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

__device__ __forceinline__ RecMix ldcg_rec(const RecMix* p) {
    RecMix r;
    r.hi = __ldcg(&p->hi);
    r.lo = __ldcg(&p->lo);
    return r;
}

__device__ __forceinline__ D4 ldcg_d4(const D4* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 a = __ldcg(q), b = __ldcg(q + 1);
    return make_d4(a.x, a.y, b.x, b.y);
}

// role of a phase: 0 pack, 1 acc+kick+drift, 2 acc->a, 3 grad+kick+drift, 4 acc+kick(+drift)
__device__ __forceinline__ int phase_role(int p) {
    if (p == 0) return 0;
    if (p == 1) return 1;
    return 2 + (p - 2) % 3;
}

// Idle accounting (fsi_batch_stats): thread 0 of every CTA adds the time it spent waiting
// for other CTAs' phases and its lifetime when it leaves the persistent loop.
__device__ __forceinline__ void batch_stats_exit(const BatchArgs& a, long long t_start,
                                                 long long waited) {
    if (threadIdx.x == 0 && a.stats) {
        atomicAdd(a.stats, (unsigned long long)waited);
        atomicAdd(a.stats + 1, (unsigned long long)(global_ns() - t_start));
    }
}

// Error path of a non-finite pass sum of cluster particle il (global index off + il):
// without softening, a distinct particle of the same cluster at exactly the same position
// in the pass's records rin makes a pair term 0 x inf and is reported as
// FSI_ERR_COINCIDENT, anything else as FSI_ERR_NONFINITE.  Only the thread that claims the
// empty error word scans the cluster (first error wins).
template <int P>
__device__ __noinline__ void batch_report_nonfinite(const BatchArgs& a, const void* rin, long long off,
                                                    int n, int il) {
    if (!a.err || atomicCAS(a.err, 0, FSI_ERR_NONFINITE) != 0) return;
    if (a.eps2 != 0.0) return;
    bool hit = false;
    for (int j = 0; j < n && !hit; ++j) {
        if (j == il) continue;
        if constexpr (P == FSI_MIXED) {
            const RecMix ri = reinterpret_cast<const RecMix*>(rin)[off + il];
            const RecMix rj = reinterpret_cast<const RecMix*>(rin)[off + j];
            hit = rj.hi.x == ri.hi.x && rj.hi.y == ri.hi.y && rj.hi.z == ri.hi.z &&
                  rj.lo.x == ri.lo.x && rj.lo.y == ri.lo.y && rj.lo.z == ri.lo.z;
        } else {
            const D4 ri = reinterpret_cast<const D4*>(rin)[off + il];
            const D4 rj = reinterpret_cast<const D4*>(rin)[off + j];
            hit = rj.x == ri.x && rj.y == ri.y && rj.z == ri.z;
        }
    }
    if (hit) atomicCAS(a.err, FSI_ERR_NONFINITE, FSI_ERR_COINCIDENT);
}

template <int P, int I>
__global__ void __launch_bounds__(kBatchThreads, 2) batch_kernel(const BatchArgs a) {
    constexpr int JREC = 32;
    constexpr int AREC = P == FSI_MIXED ? 16 : 32;
    __shared__ __align__(16) unsigned char sm_rec[kBatchTile * JREC];
    __shared__ __align__(16) unsigned char sm_acc[kBatchTile * AREC];
    __shared__ int s_item, s_flag;
    const int tid = threadIdx.x;
    const long long N = a.ntot;
    const long long t_start = global_ns();
    long long waited = 0;

    while (true) {
        if (tid == 0) {
            int t = atomicAdd(a.next, 1);
            if (t >= a.items_per_phase * a.nphase || ld_acquire(a.abort_flag)) t = -1;
            s_item = t;
        }
        __syncthreads();
        const int t = s_item;
        __syncthreads();
        if (t < 0) { batch_stats_exit(a, t_start, waited); return; }
        const int p = t / a.items_per_phase;
        const BatchItem it = a.items[t % a.items_per_phase];
        const int role = phase_role(p);
        // ---- wait until the previous phase of this cluster is complete
        if (p > 0) {
            if (tid == 0) {
                const int* cnt = a.done + (size_t)it.cluster * a.nphase + (p - 1);
                const int need = a.nblocks[it.cluster];
                int flag = 0;
                if (ld_acquire(cnt) < need) {
                    const long long t0 = global_ns();
                    while (ld_acquire(cnt) < need) {
                        if (ld_acquire(a.abort_flag)) { flag = 1; break; }
                        if (global_ns() - t0 > a.timeout_ns) {
                            set_error(a.err, FSI_ERR_TIMEOUT);
                            atomicExch(a.abort_flag, 1);
                            flag = 1;
                            break;
                        }
                        __nanosleep(64);
                    }
                    waited += global_ns() - t0;
                }
                __threadfence();
                s_flag = flag;
            }
            __syncthreads();
            if (s_flag) { batch_stats_exit(a, t_start, waited); return; }
        }
        const int ib = it.block * (kBatchThreads * I);        // first i of the block (local)
        // ---- phase 0: pack records of the block from x
        if (role == 0) {
#pragma unroll
            for (int u = 0; u < I; ++u) {
                const int il = ib + u * kBatchThreads + tid;
                if (il < it.n) {
                    const long long i = it.off + il;
                    const double x = a.x[i], y = a.x[N + i], z = a.x[2 * N + i];
                    if constexpr (P == FSI_MIXED) {
                        const RecMix r = make_mix_rec(x, y, z, a.m[i]);
                        RecMix* o = reinterpret_cast<RecMix*>(a.rec0) + i;
                        __stcg(&o->hi, r.hi);
                        __stcg(&o->lo, r.lo);
                    } else {
                        double2* o = reinterpret_cast<double2*>(reinterpret_cast<D4*>(a.rec0) + i);
                        __stcg(o, make_double2(x, y));
                        __stcg(o + 1, make_double2(z, a.m[i]));
                    }
                }
            }
        } else {
            const bool grad = (role == 3);
            // role 1 reads rec0, 2 and 3 read rec1, 4 reads rec0
            const void* rin = (role == 1 || role == 4) ? a.rec0 : a.rec1;
            double acc64[I][3];
            int myl[I];
#pragma unroll
            for (int u = 0; u < I; ++u) {
                acc64[u][0] = acc64[u][1] = acc64[u][2] = 0.0;
                myl[u] = ib + u * kBatchThreads + tid;
            }
            if constexpr (P == FSI_MIXED) {
                MixI pi[I];
                float f[I][3];
                // I = 2: the two particles as one packed pair for the tiles without the
                // self pair (fma.rn.f32x2 arithmetic, same rounding per half)
                X2I pp;
                float2 f2[3];
#pragma unroll
                for (int u = 0; u < I; ++u) {
                    const long long i = it.off + min(myl[u], it.n - 1);
                    const RecMix r = ldcg_rec(reinterpret_cast<const RecMix*>(rin) + i);
                    pi[u].xh = r.hi.x; pi[u].yh = r.hi.y; pi[u].zh = r.hi.z;
                    pi[u].xl = r.lo.x; pi[u].yl = r.lo.y; pi[u].zl = r.lo.z;
                    pi[u].ax = pi[u].ay = pi[u].az = 0.f;
                    if (grad) {
                        const float4 ai = __ldcg(reinterpret_cast<const float4*>(a.accrec) + i);
                        pi[u].ax = ai.x; pi[u].ay = ai.y; pi[u].az = ai.z;
                    }
                    f[u][0] = f[u][1] = f[u][2] = 0.f;
                    if constexpr (I == 2) {
                        set_half(pp.nxh, u, -pi[u].xh); set_half(pp.nyh, u, -pi[u].yh);
                        set_half(pp.nzh, u, -pi[u].zh); set_half(pp.nxl, u, -pi[u].xl);
                        set_half(pp.nyl, u, -pi[u].yl); set_half(pp.nzl, u, -pi[u].zl);
                        set_half(pp.nax, u, -pi[u].ax); set_half(pp.nay, u, -pi[u].ay);
                        set_half(pp.naz, u, -pi[u].az);
                    }
                }
                f2[0] = f2[1] = f2[2] = make_float2(0.f, 0.f);
                const float2 eps2x = bc2((float)a.eps2);
                const float eps2f = (float)a.eps2;
                for (int j0 = 0; j0 < it.n; j0 += kBatchTile) {
                    const int cnt = min(kBatchTile, it.n - j0);
                    __syncthreads();
                    if (tid < cnt) {
                        const long long j = it.off + j0 + tid;
                        reinterpret_cast<RecMix*>(sm_rec)[tid] = ldcg_rec(reinterpret_cast<const RecMix*>(rin) + j);
                        if (grad)
                            reinterpret_cast<float4*>(sm_acc)[tid] = __ldcg(reinterpret_cast<const float4*>(a.accrec) + j);
                    }
                    __syncthreads();
                    const RecMix* rec = reinterpret_cast<const RecMix*>(sm_rec);
                    const float4* arec = reinterpret_cast<const float4*>(sm_acc);
                    const bool chk = j0 < ib + kBatchThreads * I && j0 + cnt > ib;
                    if (!chk && I == 2) {
                        if (!grad) {
                            for (int jj = 0; jj < cnt; ++jj) x2_acc_one(rec[jj].hi, rec[jj].lo, pp, eps2x, f2);
                        } else {
                            for (int jj = 0; jj < cnt; ++jj)
                                x2_grad_one(rec[jj].hi, rec[jj].lo, arec[jj], pp, eps2x, f2);
                        }
                    } else if (!chk) {
                        for (int jj = 0; jj < cnt; ++jj) {
                            const float4 hh = rec[jj].hi, ll = rec[jj].lo;
                            if (!grad) {
#pragma unroll
                                for (int u = 0; u < I; ++u) mix_acc_pair<false>(hh, ll, pi[u], eps2f, false, f[u][0], f[u][1], f[u][2]);
                            } else {
                                const float4 aj = arec[jj];
#pragma unroll
                                for (int u = 0; u < I; ++u) mix_grad_pair<false>(hh, ll, aj, pi[u], eps2f, false, f[u][0], f[u][1], f[u][2]);
                            }
                        }
                    } else {
                        for (int jj = 0; jj < cnt; ++jj) {
                            const float4 hh = rec[jj].hi, ll = rec[jj].lo;
                            if (!grad) {
#pragma unroll
                                for (int u = 0; u < I; ++u) mix_acc_pair<true>(hh, ll, pi[u], eps2f, j0 + jj == myl[u], f[u][0], f[u][1], f[u][2]);
                            } else {
                                const float4 aj = arec[jj];
#pragma unroll
                                for (int u = 0; u < I; ++u) mix_grad_pair<true>(hh, ll, aj, pi[u], eps2f, j0 + jj == myl[u], f[u][0], f[u][1], f[u][2]);
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < I; ++u)
#pragma unroll
                        for (int q = 0; q < 3; ++q) { acc64[u][q] += (double)f[u][q]; f[u][q] = 0.f; }
                    if constexpr (I == 2) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            acc64[0][q] += (double)f2[q].x;
                            acc64[1][q] += (double)f2[q].y;
                            f2[q] = make_float2(0.f, 0.f);
                        }
                    }
                }
            } else {
                F64I pi[I];
#pragma unroll
                for (int u = 0; u < I; ++u) {
                    const long long i = it.off + min(myl[u], it.n - 1);
                    const D4 r = ldcg_d4(reinterpret_cast<const D4*>(rin) + i);
                    pi[u].x = r.x; pi[u].y = r.y; pi[u].z = r.z;
                    pi[u].ax = pi[u].ay = pi[u].az = 0.0;
                    if (grad) {
                        const D4 ai = ldcg_d4(reinterpret_cast<const D4*>(a.accrec) + i);
                        pi[u].ax = ai.x; pi[u].ay = ai.y; pi[u].az = ai.z;
                    }
                }
                for (int j0 = 0; j0 < it.n; j0 += kBatchTile) {
                    const int cnt = min(kBatchTile, it.n - j0);
                    __syncthreads();
                    if (tid < cnt) {
                        const long long j = it.off + j0 + tid;
                        reinterpret_cast<D4*>(sm_rec)[tid] = ldcg_d4(reinterpret_cast<const D4*>(rin) + j);
                        if (grad) reinterpret_cast<D4*>(sm_acc)[tid] = ldcg_d4(reinterpret_cast<const D4*>(a.accrec) + j);
                    }
                    __syncthreads();
                    const D4* rec = reinterpret_cast<const D4*>(sm_rec);
                    const D4* arec = reinterpret_cast<const D4*>(sm_acc);
                    for (int jj = 0; jj < cnt; ++jj) {
                        const D4 r = rec[jj];
                        if (!grad) {
#pragma unroll
                            for (int u = 0; u < I; ++u) f64_acc_pair<true>(r, pi[u], a.eps2, j0 + jj == myl[u], acc64[u][0], acc64[u][1], acc64[u][2]);
                        } else {
                            const D4 aj = arec[jj];
#pragma unroll
                            for (int u = 0; u < I; ++u) f64_grad_pair<true>(r, aj, pi[u], a.eps2, j0 + jj == myl[u], acc64[u][0], acc64[u][1], acc64[u][2]);
                        }
                    }
                }
            }
            // ---- epilogue of the block's particles
            const double h = a.h;
            const bool last_acc = (role == 4) && (p == a.nphase - 1);
            double ck = 0.0, cd = 0.0;
            if (role == 1) { ck = h / 6.0; cd = 0.5 * h; }
            if (role == 3) { ck = 2.0 * h / 3.0; cd = 0.5 * h; }
            if (role == 4) { ck = last_acc ? h / 6.0 : h / 3.0; cd = last_acc ? 0.0 : 0.5 * h; }
            void* rout = (role == 3) ? a.rec0 : a.rec1;
#pragma unroll
            for (int u = 0; u < I; ++u) {
                if (myl[u] >= it.n) continue;
                const long long i = it.off + myl[u];
                double r3[3] = {acc64[u][0], acc64[u][1], acc64[u][2]};
                if (!(isfinite(r3[0]) && isfinite(r3[1]) && isfinite(r3[2])))
                    batch_report_nonfinite<P>(a, rin, it.off, it.n, myl[u]);
                if (role == 2) {
                    const double mi = a.m[i];
#pragma unroll
                    for (int q = 0; q < 3; ++q) __stcg(a.ac + q * N + i, r3[q]);
                    if constexpr (P == FSI_MIXED)
                        __stcg(reinterpret_cast<float4*>(a.accrec) + i, make_float4((float)r3[0], (float)r3[1], (float)r3[2], (float)mi));
                    else {
                        double2* q = reinterpret_cast<double2*>(reinterpret_cast<D4*>(a.accrec) + i);
                        __stcg(q, make_double2(r3[0], r3[1]));
                        __stcg(q + 1, make_double2(r3[2], mi));
                    }
                    continue;
                }
                double xv[3], vv[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    double kq = r3[q];
                    if (role == 3) kq = fma(h * h / 24.0, r3[q], __ldcg(a.ac + q * N + i));
                    vv[q] = fma(ck, kq, __ldcg(a.v + q * N + i));
                    __stcg(a.v + q * N + i, vv[q]);
                    xv[q] = __ldcg(a.x + q * N + i);
                    if (cd != 0.0) {
                        xv[q] = fma(cd, vv[q], xv[q]);
                        __stcg(a.x + q * N + i, xv[q]);
                    }
                }
                if (cd != 0.0) {
                    const double mi = a.m[i];
                    if constexpr (P == FSI_MIXED) {
                        const RecMix r = make_mix_rec(xv[0], xv[1], xv[2], mi);
                        RecMix* o = reinterpret_cast<RecMix*>(rout) + i;
                        __stcg(&o->hi, r.hi);
                        __stcg(&o->lo, r.lo);
                    } else {
                        double2* o = reinterpret_cast<double2*>(reinterpret_cast<D4*>(rout) + i);
                        __stcg(o, make_double2(xv[0], xv[1]));
                        __stcg(o + 1, make_double2(xv[2], mi));
                    }
                }
            }
        }
        // ---- signal completion of this item (release)
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(a.done + (size_t)it.cluster * a.nphase + p, 1);
        }
    }
}

// =================================================================================
// Symmetric persistent ensemble kernel (mixed precision).  The same phase machinery as
// batch_kernel, but every pair pass is split into
//   a sum phase:   items (cluster, i-block of 1024 particles, source tiles [t0, t1));
//                  every unordered pair is evaluated once with the packed symmetric
//                  arithmetic (sym_x2.cuh: i-side in registers, source side by the warp
//                  reduce-scatter), except the pairs inside one warp's 128 particles
//                  (one-sided, self pair excluded); both sides are added into the FP64
//                  accumulator accum (red.global.add);
//   an apply phase: items (cluster, block): the pass's epilogue from accum, which it
//                  clears for the next pass.
// A sum item of a cluster waits for the previous apply (or pack) phase of that cluster,
// an apply item for all sum items of its pass.  Source tiles stream through a 3-stage
// shared-memory ring filled by cp.async.bulk on mbarriers whose phase parity follows a
// running per-CTA tile count; every wait is bounded as in batch_kernel.
namespace {
// ring depth of the symmetric form: a block's own tiles (4 with 4 particles per thread) land
// at once, so its diagonal item runs with one barrier instead of one per tile
constexpr int kBSStages = 4;
constexpr int kBSStage = kBatchTile * (32 + 16);                     // record + accel record
constexpr int kBSJpart = (kBatchThreads / 32) * kBatchTile * 3 * 4;
static_assert(kBatchTile == kTileJ && kBatchThreads == kThreads, "tile sizes of sym_x2.cuh");
// I particles per thread: a block of 256 I particles (I source tiles), I / 2 packed pairs
// per thread; warp w holds the I consecutive 32-record sub-tiles of group w of the block.
template <int I>
struct BS {
    static constexpr int NP = I / 2;                                 // packed pairs per thread
    static constexpr int Block = kBatchThreads * I;                  // particles per block
    static constexpr int AccS = NP * 3 * kBatchThreads * 16;
    static constexpr int Smem = kBSStages * kBSStage + kBSJpart + AccS;
};
}  // namespace

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Epilogue of one particle (global index i) of a pass with role 1..4 from its pair sum r3.
template <int P>
__device__ __forceinline__ void batch_apply(const BatchArgs& a, int role, bool last_acc, long long i,
                                            const double (&r3)[3], void* rout) {
    const long long N = a.ntot;
    const double h = a.h;
    if (role == 2) {
        const double mi = a.m[i];
#pragma unroll
        for (int q = 0; q < 3; ++q) __stcg(a.ac + q * N + i, r3[q]);
        if constexpr (P == FSI_MIXED)
            __stcg(reinterpret_cast<float4*>(a.accrec) + i, make_float4((float)r3[0], (float)r3[1], (float)r3[2], (float)mi));
        else {
            double2* q = reinterpret_cast<double2*>(reinterpret_cast<D4*>(a.accrec) + i);
            __stcg(q, make_double2(r3[0], r3[1]));
            __stcg(q + 1, make_double2(r3[2], mi));
        }
        return;
    }
    double ck = 0.0, cd = 0.0;
    if (role == 1) { ck = h / 6.0; cd = 0.5 * h; }
    if (role == 3) { ck = 2.0 * h / 3.0; cd = 0.5 * h; }
    if (role == 4) { ck = last_acc ? h / 6.0 : h / 3.0; cd = last_acc ? 0.0 : 0.5 * h; }
    double xv[3], vv[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        double kq = r3[q];
        if (role == 3) kq = fma(h * h / 24.0, r3[q], __ldcg(a.ac + q * N + i));
        vv[q] = fma(ck, kq, __ldcg(a.v + q * N + i));
        __stcg(a.v + q * N + i, vv[q]);
        xv[q] = __ldcg(a.x + q * N + i);
        if (cd != 0.0) {
            xv[q] = fma(cd, vv[q], xv[q]);
            __stcg(a.x + q * N + i, xv[q]);
        }
    }
    if (cd != 0.0) {
        const double mi = a.m[i];
        if constexpr (P == FSI_MIXED) {
            const RecMix r = make_mix_rec(xv[0], xv[1], xv[2], mi);
            RecMix* o = reinterpret_cast<RecMix*>(rout) + i;
            __stcg(&o->hi, r.hi);
            __stcg(&o->lo, r.lo);
        } else {
            double2* o = reinterpret_cast<double2*>(reinterpret_cast<D4*>(rout) + i);
            __stcg(o, make_double2(xv[0], xv[1]));
            __stcg(o + 1, make_double2(xv[2], mi));
        }
    }
}

// One sum item: block `it.block` of cluster it.cluster against its source tiles [t0, t1).
// g: the CTA's running tile count (advanced by the item's tiles).  Returns false if a wait
// timed out (the caller leaves the kernel).
template <int KIND, int I>
__device__ bool batch_sum_item(const BatchArgs& a, const BatchSymItem& it, const void* rin,
                               double* __restrict__ accum, unsigned char* smem, uint64_t* bars,
                               float* jpart, float4* acc_s, unsigned& g) {
    constexpr int NP = BS<I>::NP;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long N = a.ntot;
    const RecMix* R = reinterpret_cast<const RecMix*>(rin) + it.off;
    const float4* AR = reinterpret_cast<const float4*>(a.accrec) + it.off;
    const bool diag = (it.t0 == it.block * I);
    const int ntiles = it.t1 - it.t0;
    auto issue = [&](int tl) {
        const unsigned gg = g + (unsigned)tl;
        const int st = (int)(gg % kBSStages);
        const int jt = (it.t0 + tl) * kBatchTile;
        const int cnt = min(kBatchTile, it.n - jt);
        unsigned char* base = smem + st * kBSStage;
        mbar_arrive_expect_tx(&bars[st], (uint32_t)cnt * (32u + (KIND == KIND_GRAD ? 16u : 0u)));
        bulk_g2s(base, R + jt, (uint32_t)cnt * 32u, &bars[st]);
        if (KIND == KIND_GRAD) bulk_g2s(base + kBatchTile * 32, AR + jt, (uint32_t)cnt * 16u, &bars[st]);
    };
    if (tid == 0) {
        fence_proxy_async();            // records written by generic stores of earlier phases
        for (int tl = 0; tl < min(kBSStages, ntiles); ++tl) issue(tl);
    }
    // i-side state: warp w holds the 32 I consecutive particles i0 + 32 I w + 32 u + lane
    const int ib = it.block * BS<I>::Block + warp * (32 * I) + lane;
    X2I pp[NP];
    float2 f[NP][3];
#pragma unroll
    for (int u = 0; u < I; ++u) {
        const bool valid = ib + 32 * u < it.n;
        const int ic = min(ib + 32 * u, it.n - 1);
        RecMix r;
        r.hi = __ldcg(&R[ic].hi);
        r.lo = __ldcg(&R[ic].lo);
        float nm = 0.f, nax = 0.f, nay = 0.f, naz = 0.f;
        if constexpr (KIND == KIND_GRAD) {
            const float4 ai = __ldcg(AR + ic);
            nax = -ai.x; nay = -ai.y; naz = -ai.z;
            nm = valid ? -ai.w : 0.f;
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
        for (int q = 0; q < 3; ++q) acc_s[(p * 3 + q) * kBatchThreads + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float eps2f = (float)a.eps2;
    const float2 eps2 = bc2(eps2f);
    bool ok_all = true;
    int t_stop = ntiles;
    // the block's own tiles, each unordered pair once: warp w holds the block's 32-record
    // sub-tiles I w .. I w + I - 1 (group w); the pairs of groups w and v != w are evaluated
    // symmetrically by w when (v - w) mod 8 is 1, 2 or 3, or 4 with w < 4 (by v otherwise),
    // so every warp takes 3 or 4 of the 7 other groups; its own group one-sided (self pair
    // excluded by index).  A warp past the end of the cluster holds copies of its last
    // particle and takes no pairs: that particle's pairs belong to the warp that holds it.
    // DIRECT: the source-side totals go straight into the accumulator (every own tile in
    // shared memory at once, no barrier between tiles); otherwise into jpart per tile.
    auto diag_tile = [&](int tl, const RecMix* rec, const float4* arec, int jt, int cnt, auto direct) {
        constexpr bool DIRECT = decltype(direct)::value;
        const bool wvalid = it.block * BS<I>::Block + warp * (32 * I) < it.n;
        double* jg = accum + it.off + jt;
        float2 D0[NP][3];
        for (int k0 = 0; k0 < cnt; k0 += 32) {
            const int jend = min(cnt, k0 + 32);
            const int sub = 8 * tl + (k0 >> 5);                // sub-tile within the block
            const int dv = ((sub / I) - warp) & 7;
            if (wvalid && dv >= 1 && (dv <= 3 || (dv == 4 && warp < 4))) {
                if (jend - k0 < 32) {
                    for (int jj = k0; jj < jend; jj += 4)
                        x2_group<KIND, NP, false, false, DIRECT>(jj, cnt, lane, warp, rec, arec, nullptr, pp, D0, eps2, f, jpart, jg, N);
                } else {
                    for (int jj = k0; jj < jend; jj += 4)
                        x2_group<KIND, NP, false, true, DIRECT>(jj, cnt, lane, warp, rec, arec, nullptr, pp, D0, eps2, f, jpart, jg, N);
                }
                continue;
            }
            if (!DIRECT && k0 + lane < jend) {
                float* dst = jpart + ((size_t)warp * kBatchTile + k0 + lane) * 3;
                dst[0] = dst[1] = dst[2] = 0.f;
            }
            if (dv != 0) continue;
            for (int jj = k0; jj < jend; ++jj) {
                const float4 h = rec[jj].hi;
                const float4 l = rec[jj].lo;
                const int j = jt + jj;
                if constexpr (KIND == KIND_ACC) {
#pragma unroll
                    for (int p = 0; p < NP; ++p)
                        x2_acc_one_chk(h, l, pp[p], eps2, j == ib + 64 * p, j == ib + 64 * p + 32, f[p]);
                } else {
                    const float4 aj = arec[jj];
#pragma unroll
                    for (int p = 0; p < NP; ++p)
                        x2_grad_one_chk(h, l, aj, pp[p], eps2, j == ib + 64 * p, j == ib + 64 * p + 32, f[p]);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                ff_add2(acc_s[(p * 3 + c) * kBatchThreads + tid], f[p][c]);
                f[p][c] = make_float2(0.f, 0.f);
            }
    };
    if (diag && ntiles <= kBSStages) {
        // every own tile was issued above: wait for all, one pass over them, one barrier
        bool ok = true;
        for (int tl = 0; tl < ntiles; ++tl) {
            const unsigned gg = g + (unsigned)tl;
            ok = mbar_wait_bounded(&bars[gg % kBSStages], (gg / kBSStages) & 1u, a.timeout_ns, a.err) && ok;
        }
        if (!__syncthreads_or(!ok)) {
            for (int tl = 0; tl < ntiles; ++tl) {
                const unsigned char* base = smem + ((g + (unsigned)tl) % kBSStages) * kBSStage;
                const int jt = (it.t0 + tl) * kBatchTile;
                diag_tile(tl, reinterpret_cast<const RecMix*>(base),
                          reinterpret_cast<const float4*>(base + kBatchTile * 32), jt,
                          min(kBatchTile, it.n - jt), std::true_type{});
            }
        } else {
            ok_all = false;
            t_stop = 0;
        }
        __syncthreads();                // shared memory free for the next item's copies
    }
    for (int tl = 0; tl < ntiles && !(diag && ntiles <= kBSStages); ++tl) {
        const unsigned gg = g + (unsigned)tl;
        const int st = (int)(gg % kBSStages);
        const bool ok = mbar_wait_bounded(&bars[st], (gg / kBSStages) & 1u, a.timeout_ns, a.err);
        const int jt = (it.t0 + tl) * kBatchTile;
        const int cnt = min(kBatchTile, it.n - jt);
        const unsigned char* base = smem + st * kBSStage;
        const RecMix* rec = reinterpret_cast<const RecMix*>(base);
        const float4* arec = reinterpret_cast<const float4*>(base + kBatchTile * 32);
        if (diag) {
            diag_tile(tl, rec, arec, jt, cnt, std::false_type{});
        } else {
            float2 D0[NP][3];
            for (int k0 = 0; k0 < cnt; k0 += 32) {
                const int jend = min(cnt, k0 + 32);
                if (jend - k0 < 32) {
                    for (int jj = k0; jj < jend; jj += 4)
                        x2_group<KIND, NP, false, false>(jj, cnt, lane, warp, rec, arec, nullptr, pp, D0, eps2, f, jpart);
                } else {
                    for (int jj = k0; jj < jend; jj += 4)
                        x2_group<KIND, NP, false, true>(jj, cnt, lane, warp, rec, arec, nullptr, pp, D0, eps2, f, jpart);
                }
            }
#pragma unroll
            for (int p = 0; p < NP; ++p)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    ff_add2(acc_s[(p * 3 + c) * kBatchThreads + tid], f[p][c]);
                    f[p][c] = make_float2(0.f, 0.f);
                }
        }
        if (__syncthreads_or(!ok)) { ok_all = false; t_stop = tl; break; }
        if (tid < cnt) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float sum = 0.f;
#pragma unroll
                for (int w = 0; w < kBatchThreads / 32; ++w) sum += jpart[((size_t)w * kBatchTile + tid) * 3 + c];
                red_add(accum + (size_t)c * N + it.off + jt + tid, (double)sum);
            }
        }
        __syncthreads();
        if (tid == 0 && tl + kBSStages < ntiles) issue(tl + kBSStages);
    }
    if (!ok_all) {
        // let every copy still in flight land (bounded) before the CTA leaves
        if (tid == 0) {
            const int issued = min(ntiles, t_stop + kBSStages);
            for (int tl = t_stop; tl < issued; ++tl) {
                const unsigned gg = g + (unsigned)tl;
                mbar_wait_bounded(&bars[gg % kBSStages], (gg / kBSStages) & 1u, a.timeout_ns, nullptr);
            }
        }
        __syncthreads();
        return false;
    }
    g += (unsigned)ntiles;
#pragma unroll
    for (int u = 0; u < I; ++u) {
        if (ib + 32 * u >= it.n) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 s = acc_s[((u >> 1) * 3 + c) * kBatchThreads + tid];
            const double sum = (u & 1) ? (double)s.y + (double)s.w : (double)s.x + (double)s.z;
            red_add(accum + (size_t)c * N + it.off + ib + 32 * u, sum);
        }
    }
    return true;
}

template <int I, int MINB>
__global__ void __launch_bounds__(kBatchThreads, MINB) batch_sym_kernel(
    const BatchArgs a, const BatchSymItem* __restrict__ sitems, int nS, const int* __restrict__ nsum,
    double* __restrict__ accum) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[kBSStages];
    __shared__ int s_item, s_flag;
    float* jpart = reinterpret_cast<float*>(smem + kBSStages * kBSStage);
    float4* acc_s = reinterpret_cast<float4*>(smem + kBSStages * kBSStage + kBSJpart);
    const int tid = threadIdx.x;
    const long long N = a.ntot;
    const long long t_start = global_ns();
    long long waited = 0;
    const int nA = a.items_per_phase;
    const int npass = 1 + 3 * a.nsteps;
    const long long total = (long long)nA + (long long)npass * (long long)(nS + nA);
    if (tid == 0) {
        for (int st = 0; st < kBSStages; ++st) mbar_init(&bars[st], 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned g = 0;
    while (true) {
        if (tid == 0) {
            long long t = atomicAdd(a.next, 1);
            if (t >= total || ld_acquire(a.abort_flag)) t = -1;
            s_item = (int)t;
        }
        __syncthreads();
        const int t = s_item;
        __syncthreads();
        if (t < 0) { batch_stats_exit(a, t_start, waited); return; }
        int phase, pass = -1, r = t;
        bool is_sum = false;
        if (t >= nA) {
            const int tt = t - nA;
            pass = tt / (nS + nA);
            r = tt % (nS + nA);
            is_sum = r < nS;
            if (!is_sum) r -= nS;
            phase = 1 + 2 * pass + (is_sum ? 0 : 1);
        } else {
            phase = 0;
        }
        const int cluster = is_sum ? sitems[r].cluster : a.items[r].cluster;
        if (phase > 0) {
            // wait until the previous phase of this cluster is complete: a sum phase has
            // odd index, the pack and apply phases even
            if (tid == 0) {
                const int* cnt = a.done + (size_t)cluster * a.nphase + (phase - 1);
                const int need = ((phase - 1) & 1) ? nsum[cluster] : a.nblocks[cluster];
                int flag = 0;
                if (ld_acquire(cnt) < need) {
                    const long long t0 = global_ns();
                    while (ld_acquire(cnt) < need) {
                        if (ld_acquire(a.abort_flag)) { flag = 1; break; }
                        if (global_ns() - t0 > a.timeout_ns) {
                            set_error(a.err, FSI_ERR_TIMEOUT);
                            atomicExch(a.abort_flag, 1);
                            flag = 1;
                            break;
                        }
                        __nanosleep(64);
                    }
                    waited += global_ns() - t0;
                }
                __threadfence();
                s_flag = flag;
            }
            __syncthreads();
            if (s_flag) { batch_stats_exit(a, t_start, waited); return; }
        }
        // item time by kind (stats[2 + k] ns, stats[5 + k] items): k = 0 a sum item of a
        // block with itself, 1 a sum item of two blocks, 2 a pack or apply item
        const long long t_item = global_ns();
        const int ikind = is_sum ? (sitems[r].t0 == sitems[r].block * I ? 0 : 1) : 2;
        const int role = phase == 0 ? 0 : (pass == 0 ? 1 : 2 + (pass - 1) % 3);
        if (phase == 0) {
            // pack the block's records from x
            const BatchItem it = a.items[r];
#pragma unroll
            for (int u = 0; u < I; ++u) {
                const int il = it.block * BS<I>::Block + u * kBatchThreads + tid;
                if (il < it.n) {
                    const long long i = it.off + il;
                    const RecMix rr = make_mix_rec(a.x[i], a.x[N + i], a.x[2 * N + i], a.m[i]);
                    RecMix* o = reinterpret_cast<RecMix*>(a.rec0) + i;
                    __stcg(&o->hi, rr.hi);
                    __stcg(&o->lo, rr.lo);
                }
            }
        } else if (is_sum) {
            const BatchSymItem it = sitems[r];
            // roles 1 and 4 read rec0, 2 and 3 read rec1
            const void* rin = (role == 1 || role == 4) ? a.rec0 : a.rec1;
            const bool ok = role == 3
                ? batch_sum_item<KIND_GRAD, I>(a, it, rin, accum, smem, bars, jpart, acc_s, g)
                : batch_sum_item<KIND_ACC, I>(a, it, rin, accum, smem, bars, jpart, acc_s, g);
            if (!ok) {
                if (tid == 0) atomicExch(a.abort_flag, 1);
                batch_stats_exit(a, t_start, waited);
                return;
            }
        } else {
            const BatchItem it = a.items[r];
            const bool last_acc = (role == 4) && (pass == npass - 1);
            void* rout = (role == 3) ? a.rec0 : a.rec1;
#pragma unroll
            for (int u = 0; u < I; ++u) {
                const int il = it.block * BS<I>::Block + u * kBatchThreads + tid;
                if (il >= it.n) continue;
                const long long i = it.off + il;
                double r3[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    r3[c] = __ldcg(accum + c * N + i);
                    __stcg(accum + c * N + i, 0.0);
                }
                if (!(isfinite(r3[0]) && isfinite(r3[1]) && isfinite(r3[2])))
                    batch_report_nonfinite<FSI_MIXED>(a, (role == 1 || role == 4) ? a.rec0 : a.rec1,
                                                      it.off, it.n, il);
                batch_apply<FSI_MIXED>(a, role, last_acc, i, r3, rout);
            }
        }
        // signal completion of this item (release); the proxy fence orders this thread's
        // generic stores before the bulk copies (async proxy) of later items
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(a.done + (size_t)cluster * a.nphase + phase, 1);
            if (a.stats) {
                atomicAdd(a.stats + 2 + ikind, (unsigned long long)(global_ns() - t_item));
                atomicAdd(a.stats + 5 + ikind, 1ull);
            }
        }
    }
}

template <int I, int MINB>
static cudaError_t launch_batch_sym_i(int ctas, const BatchArgs& a, const BatchSymItem* sitems,
                                      int sitems_per_phase, const int* nsum, double* accum,
                                      cudaStream_t s) {
    static std::atomic<unsigned long long> attr_dev{0};
    {
        const cudaError_t e = smem_attr_once(batch_sym_kernel<I, MINB>, (int)BS<I>::Smem, attr_dev);
        if (e != cudaSuccess) return e;
    }
    { batch_sym_kernel<I, MINB><<<ctas, kBatchThreads, BS<I>::Smem, s>>>(a, sitems, sitems_per_phase, nsum, accum); note_launch(); }
    return cudaGetLastError();
}

cudaError_t launch_batch_sym(int ipt, int ctas, const BatchArgs& a, const BatchSymItem* sitems,
                             int sitems_per_phase, const int* nsum, double* accum,
                             cudaStream_t s) {
    if (ipt == kBatchSymI) return launch_batch_sym_i<kBatchSymI, 2>(ctas, a, sitems, sitems_per_phase, nsum, accum, s);
    if (ipt == kBatchSymI15) return launch_batch_sym_i<kBatchSymI15, 2>(ctas, a, sitems, sitems_per_phase, nsum, accum, s);
    if (ipt == kBatchSymI2) return launch_batch_sym_i<kBatchSymI2, 1>(ctas, a, sitems, sitems_per_phase, nsum, accum, s);
    return cudaErrorInvalidValue;
}

template <int I, int MINB>
static int batch_sym_ctas_i() {
    if (cudaFuncSetAttribute(batch_sym_kernel<I, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             BS<I>::Smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_sym_kernel<I, MINB>, kBatchThreads,
                                                      BS<I>::Smem) != cudaSuccess)
        return 0;
    return nb;
}

int batch_sym_max_ctas_per_sm(int ipt) {
    if (ipt == kBatchSymI) return batch_sym_ctas_i<kBatchSymI, 2>();
    if (ipt == kBatchSymI15) return batch_sym_ctas_i<kBatchSymI15, 2>();
    if (ipt == kBatchSymI2) return batch_sym_ctas_i<kBatchSymI2, 1>();
    return 0;
}

cudaError_t launch_batch(int precision, int ipt, int ctas, const BatchArgs& a, cudaStream_t s) {
    switch (precision * 8 + ipt) {
        case FSI_MIXED * 8 + 1: { batch_kernel<FSI_MIXED, 1><<<ctas, kBatchThreads, 0, s>>>(a); note_launch(); break; }
        case FSI_MIXED * 8 + 2: { batch_kernel<FSI_MIXED, 2><<<ctas, kBatchThreads, 0, s>>>(a); note_launch(); break; }
        case FSI_FP64 * 8 + 1: { batch_kernel<FSI_FP64, 1><<<ctas, kBatchThreads, 0, s>>>(a); note_launch(); break; }
        case FSI_FP64 * 8 + 2: { batch_kernel<FSI_FP64, 2><<<ctas, kBatchThreads, 0, s>>>(a); note_launch(); break; }
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int batch_block_size(int ipt) { return kBatchThreads * ipt; }

int batch_max_ctas_per_sm(int precision, int ipt) {
    int nb = 0;
    cudaError_t e = cudaSuccess;
    if (precision == FSI_MIXED)
        e = ipt == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<FSI_MIXED, 1>, kBatchThreads, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<FSI_MIXED, 2>, kBatchThreads, 0);
    else
        e = ipt == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<FSI_FP64, 1>, kBatchThreads, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<FSI_FP64, 2>, kBatchThreads, 0);
    return e == cudaSuccess ? nb : 0;
}

}  // namespace fsi
