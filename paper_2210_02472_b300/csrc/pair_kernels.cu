// pair_kernels.cu -- the O(n_i * n_j) direct-summation kernels of libfsi.
//
// One kernel template covers the Newtonian acceleration (Sect. 2.1, Eq. new-newton-acc)
// and the force-gradient sum of the gradient kick (Sect. 2.1, Eq. new-grad-acc), each in
// two precisions:
//
//  FP64  : every pair term in FP64.  The reciprocal square root is seeded by the FP32
//          hardware approximation and refined in FP64 by the second-order series of
//          (1 - e)^{-1/2}:  y = y0 (1 + e/2 + 3 e^2 / 8),  e = 1 - r^2 y0^2
//          (a Householder-type step; error ~ (5/16) e^3 ~ 1e-21, below FP64 rounding).
//  MIXED : pair differences from FP32 hi/lo position splits (FP32-accurate relative to
//          the separation), FP32 pair arithmetic with one first-order residual
//          correction of the hardware rsqrt folded into r^-3 (and r^-5), FP32 partial
//          sums over one source tile, accumulated across tiles in FP64.
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
#include "fsi_internal.cuh"

namespace fsi {

// ---------------------------------------------------------------------------------
// Per-pair arithmetic.
struct MixI {
    float xh, yh, zh, xl, yl, zl;
    float ax, ay, az;
};

template <bool CHK>
__device__ __forceinline__ void mix_acc_pair(const float4 h, const float4 l, const MixI& p,
                                             float eps2f, bool self,
                                             float& fx, float& fy, float& fz) {
    const float dx = (h.x - p.xh) + (l.x - p.xl);
    const float dy = (h.y - p.yh) + (l.y - p.yl);
    const float dz = (h.z - p.zh) + (l.z - p.zl);
    float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2f)));
    if (CHK) r2 = self ? 1.0f : r2;
    const float y = rsqrt_hw(r2);
    const float y2 = y * y;
    const float sres = r2 * y2;                      // 1 - e, e = rsqrt residual
    // m r^-3 = m y^3 (1 - e)^{-3/2} ~ y^3 (2.5 m - 1.5 m (1 - e)); h.w = 2.5 m, l.w = -1.5 m
    const float w = (y2 * y) * fmaf(sres, l.w, h.w);
    fx = fmaf(w, dx, fx);
    fy = fmaf(w, dy, fy);
    fz = fmaf(w, dz, fz);
}

template <bool CHK>
__device__ __forceinline__ void mix_grad_pair(const float4 h, const float4 l, const float4 aj,
                                              const MixI& p, float eps2f, bool self,
                                              float& gx, float& gy, float& gz) {
    const float dx = (h.x - p.xh) + (l.x - p.xl);
    const float dy = (h.y - p.yh) + (l.y - p.yl);
    const float dz = (h.z - p.zh) + (l.z - p.zl);
    float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2f)));
    if (CHK) r2 = self ? 1.0f : r2;
    const float y = rsqrt_hw(r2);
    const float y2 = y * y;
    const float sres = r2 * y2;                      // 1 - e
    const float w = (y2 * y) * fmaf(sres, l.w, h.w); // m r^-3
    const float bx = aj.x - p.ax, by = aj.y - p.ay, bz = aj.z - p.az;   // a_ji
    const float dot = fmaf(bx, dx, fmaf(by, dy, bz * dz));
    // -3 m r^-5 = -3 w y^2 (1 + e) = w y^2 (3 (1 - e) - 6)
    const float q = (w * y2) * fmaf(3.0f, sres, -6.0f);
    const float s = q * dot;
    gx = fmaf(w, bx, fmaf(s, dx, gx));
    gy = fmaf(w, by, fmaf(s, dy, gy));
    gz = fmaf(w, bz, fmaf(s, dz, gz));
}

__device__ __forceinline__ double rsqrt_f64(double r2) {
    const double y0 = (double)rsqrt_hw(__double2float_rn(r2));
    const double t = r2 * y0;
    const double e = fma(-t, y0, 1.0);
    const double p = fma(0.375, e, 0.5);
    return fma(y0 * e, p, y0);
}

struct F64I {
    double x, y, z;
    double ax, ay, az;
};

template <bool CHK>
__device__ __forceinline__ void f64_acc_pair(const D4 j, const F64I& p, double eps2,
                                             bool self, double& fx, double& fy, double& fz) {
    const double dx = j.x - p.x, dy = j.y - p.y, dz = j.z - p.z;
    double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
    if (CHK) r2 = self ? 1.0 : r2;
    const double y = rsqrt_f64(r2);
    const double y2 = y * y;
    const double w = j.w * (y2 * y);
    fx = fma(w, dx, fx);
    fy = fma(w, dy, fy);
    fz = fma(w, dz, fz);
}

template <bool CHK>
__device__ __forceinline__ void f64_grad_pair(const D4 j, const D4 aj, const F64I& p,
                                              double eps2, bool self,
                                              double& gx, double& gy, double& gz) {
    const double dx = j.x - p.x, dy = j.y - p.y, dz = j.z - p.z;
    double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
    if (CHK) r2 = self ? 1.0 : r2;
    const double y = rsqrt_f64(r2);
    const double y2 = y * y;
    const double w = j.w * (y2 * y);
    const double bx = aj.x - p.ax, by = aj.y - p.ay, bz = aj.z - p.az;
    const double dot = fma(bx, dx, fma(by, dy, bz * dz));
    const double s = (w * y2) * (-3.0 * dot);
    gx = fma(w, bx, fma(s, dx, gx));
    gy = fma(w, by, fma(s, dy, gy));
    gz = fma(w, bz, fma(s, dz, gz));
}

// ---------------------------------------------------------------------------------
// Epilogue shared by the pair kernel (split == 1) and the finalize kernel.
template <int P>
__device__ __forceinline__ void epilogue(const Epi& e, int i, int n, double rx, double ry,
                                         double rz, int* err) {
    if (!(isfinite(rx) && isfinite(ry) && isfinite(rz))) set_error(err, FSI_ERR_NONFINITE);
    if (e.out) {
        e.out[i] = rx;
        e.out[(size_t)n + i] = ry;
        e.out[2 * (size_t)n + i] = rz;
    }
    if (e.accrec) {
        if (P == FSI_MIXED)
            reinterpret_cast<float4*>(e.accrec)[i] = make_float4((float)rx, (float)ry, (float)rz, 0.f);
        else
            reinterpret_cast<D4*>(e.accrec)[i] = make_d4(rx, ry, rz, 0.0);
    }
    if (e.v) {
        double kx = rx, ky = ry, kz = rz;
        if (e.base) {
            kx = fma(e.c_grad, rx, e.base[i]);
            ky = fma(e.c_grad, ry, e.base[(size_t)n + i]);
            kz = fma(e.c_grad, rz, e.base[2 * (size_t)n + i]);
        }
        const double vx = fma(e.c_kick, kx, e.v[i]);
        const double vy = fma(e.c_kick, ky, e.v[(size_t)n + i]);
        const double vz = fma(e.c_kick, kz, e.v[2 * (size_t)n + i]);
        e.v[i] = vx;
        e.v[(size_t)n + i] = vy;
        e.v[2 * (size_t)n + i] = vz;
        if (e.x && e.c_drift != 0.0) {
            const double x = fma(e.c_drift, vx, e.x[i]);
            const double y = fma(e.c_drift, vy, e.x[(size_t)n + i]);
            const double z = fma(e.c_drift, vz, e.x[2 * (size_t)n + i]);
            e.x[i] = x;
            e.x[(size_t)n + i] = y;
            e.x[2 * (size_t)n + i] = z;
            if (e.rec_out) {
                if constexpr (P == FSI_MIXED)
                    reinterpret_cast<RecMix*>(e.rec_out)[i] = make_mix_rec(x, y, z, e.mc[i]);
                else
                    reinterpret_cast<D4*>(e.rec_out)[i] = make_d4(x, y, z, e.mc[i]);
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

__host__ __device__ constexpr int stage_bytes(int accrec) { return kTileJ * (kRec + accrec + 4); }

// P: precision; KIND: acc or grad; I: active particles per thread; FF (mixed only): the
// per-tile FP32 partial sums are accumulated as float-float pairs by TwoSum (FP32 pipe)
// instead of FP64 additions (FP64 pipe, 1/64 of the FP32 rate on B300).
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
        my_id[u] = use_ids ? a.iid[i] : (i0 + u * kThreads + tid);
    }

    bool aborted = false;
    int t_stop = ntiles;       // first tile not consumed (on abort)
    if constexpr (P == FSI_MIXED) {
        MixI pi[I];
        float f[I][3];
        float hi[I][3], lo[I][3];   // float-float running sums (FF variant)
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
        }
        const float eps2f = (float)a.eps2;
        for (int t = 0; t < ntiles; ++t) {
            const int s = t % kStages;
            const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((t / kStages) & 1), a.timeout_ns, a.err);
            const int jt = js + t * kTileJ;
            const int cnt = min(kTileJ, je - jt);
            const unsigned char* base = smem + s * SB;
            const RecMix* rec = reinterpret_cast<const RecMix*>(base);
            const float4* arec = reinterpret_cast<const float4*>(base + kTileJ * kRec);
            const int* jidt = reinterpret_cast<const int*>(base + kTileJ * (kRec + ACCREC));
            const bool chk = use_ids || (a.check == CHECK_DIAG && jt < i0 + kThreads * I && jt + cnt > i0);
            if (!chk) {
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
                }
            }
#pragma unroll
            for (int u = 0; u < I; ++u) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if constexpr (FF) {
                        // error-free transformation (Knuth's TwoSum): hi + f = s + e exactly
                        const float sum = hi[u][q] + f[u][q];
                        const float bb = sum - hi[u][q];
                        const float e = (hi[u][q] - (sum - bb)) + (f[u][q] - bb);
                        hi[u][q] = sum;
                        lo[u][q] += e;
                    } else {
                        acc64[u][q] += (double)f[u][q];
                    }
                    f[u][q] = 0.f;
                }
            }
            if (__syncthreads_or(!ok)) { aborted = true; t_stop = t; break; }
            if (tid == 0 && t + kStages < ntiles) issue(t + kStages);
        }
        if constexpr (FF) {
#pragma unroll
            for (int u = 0; u < I; ++u)
#pragma unroll
                for (int q = 0; q < 3; ++q) acc64[u][q] = (double)hi[u][q] + (double)lo[u][q];
        }
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
            const bool chk = use_ids || (a.check == CHECK_DIAG && jt < i0 + kThreads * I && jt + cnt > i0);
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
            epilogue<P>(a.epi, i, a.n_i, acc64[u][0], acc64[u][1], acc64[u][2], a.err);
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
    epilogue<P>(a.epi, i, a.n_i, r[0], r[1], r[2], a.err);
}

// ---------------------------------------------------------------------------------
template <int P, int KIND, int I, int FF>
static cudaError_t launch_one(const PairArgs& a, int split, cudaStream_t s) {
    constexpr int SMEM = kStages * stage_bytes(Cfg<P, KIND>::ACCREC);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(pair_kernel<P, KIND, I, FF>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
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
        default: return cudaErrorInvalidValue;
    }
}

int pair_variants(int precision, int kind, int* out) {
    (void)kind;
    int n = 0;
    if (precision == FSI_MIXED) {
        for (int ipt = 2; ipt <= 4; ++ipt) out[n++] = ipt;
        for (int ipt = 2; ipt <= 4; ++ipt) out[n++] = 16 + ipt;
    } else {
        out[n++] = 1; out[n++] = 2; out[n++] = 3;
    }
    return n;
}

int pair_default_ipt(int precision, int kind) {
    return precision == FSI_MIXED ? (kind == KIND_ACC ? 4 : 2) : 2;
}

int variant_ipt(int v) { return v & 15; }

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
