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

template <int P, int I>
__global__ void __launch_bounds__(kBatchThreads, 2) batch_kernel(const BatchArgs a) {
    constexpr int JREC = 32;
    constexpr int AREC = P == FSI_MIXED ? 16 : 32;
    __shared__ __align__(16) unsigned char sm_rec[kBatchTile * JREC];
    __shared__ __align__(16) unsigned char sm_acc[kBatchTile * AREC];
    __shared__ int s_item, s_flag;
    const int tid = threadIdx.x;
    const long long N = a.ntot;

    while (true) {
        if (tid == 0) {
            int t = atomicAdd(a.next, 1);
            if (t >= a.items_per_phase * a.nphase || ld_acquire(a.abort_flag)) t = -1;
            s_item = t;
        }
        __syncthreads();
        const int t = s_item;
        __syncthreads();
        if (t < 0) return;
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
                }
                __threadfence();
                s_flag = flag;
            }
            __syncthreads();
            if (s_flag) return;
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
                }
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
                    if (!chk) {
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
                if (!(isfinite(r3[0]) && isfinite(r3[1]) && isfinite(r3[2]))) set_error(a.err, FSI_ERR_NONFINITE);
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
