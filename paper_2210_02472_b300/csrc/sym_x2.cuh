// sym_x2.cuh -- the source-side machinery of the packed symmetric pair kernels, shared by
// the single-set kernels (pair_kernels.cu) and the persistent ensemble kernel
// (batch_kernels.cu): per-pair terms acting on both particles of a pair and on the
// source (Newton's third law), and one group of 4 sources with its warp reduce-scatter.
#pragma once
#include "fsi_internal.cuh"
#include "pair_math.cuh"

namespace fsi {

__device__ __forceinline__ void red_add(double* p, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" :: "l"(p), "d"(v) : "memory");
}

__device__ __forceinline__ void x2_acc_acc(float2 wi, float2 wj, float2 dx, float2 dy, float2 dz,
                                           float2 (&fi)[3], float2 (&fj)[3]) {
    fi[0] = __ffma2_rn(wi, dx, fi[0]); fi[1] = __ffma2_rn(wi, dy, fi[1]); fi[2] = __ffma2_rn(wi, dz, fi[2]);
    fj[0] = __ffma2_rn(wj, dx, fj[0]); fj[1] = __ffma2_rn(wj, dy, fj[1]); fj[2] = __ffma2_rn(wj, dz, fj[2]);
}

__device__ __forceinline__ void x2_acc_near(const float4 h, const float4 l, const X2I& p, float2 eps2,
                                            float2 (&fi)[3], float2 (&fj)[3]) {
    float2 dx, dy, dz, y2, sres, y3;
    x2_sep_near(h, l, p, dx, dy, dz);
    x2_geom(dx, dy, dz, eps2, y2, sres, y3);
    const float2 wi = __fmul2_rn(y3, __ffma2_rn(sres, bc2(l.w), bc2(h.w)));   //  m_j r^-3
    const float2 wj = __fmul2_rn(y3, __ffma2_rn(sres, p.nB, p.nA));           // -m_i r^-3
    x2_acc_acc(wi, wj, dx, dy, dz, fi, fj);
}

__device__ __forceinline__ void x2_acc_far(const float4 r, const float2 (&D)[3], const X2I& p,
                                           float2 eps2, float2 (&fi)[3], float2 (&fj)[3]) {
    const float2 dx = __fadd2_rn(D[0], bc2(r.x)), dy = __fadd2_rn(D[1], bc2(r.y)),
                 dz = __fadd2_rn(D[2], bc2(r.z));
    float2 y2, sres, y3;
    x2_geom(dx, dy, dz, eps2, y2, sres, y3);
    const float2 r3 = __fmul2_rn(y3, __ffma2_rn(sres, bc2(-1.5f), bc2(2.5f)));
    const float2 wi = __fmul2_rn(r3, bc2(r.w));
    const float2 wj = __fmul2_rn(r3, p.nm);
    x2_acc_acc(wi, wj, dx, dy, dz, fi, fj);
}

// T(d) b = r^-3 b - 3 r^-5 (b.d) d with b = a_j - a_i; on i with weight m_j, on j with -m_i.
__device__ __forceinline__ void x2_grad_tail(float2 dx, float2 dy, float2 dz, float2 y2, float2 sres,
                                             float2 y3, const float4 aj, const X2I& p,
                                             float2 (&gi)[3], float2 (&gj)[3]) {
    const float2 r3 = __fmul2_rn(y3, __ffma2_rn(sres, bc2(-1.5f), bc2(2.5f)));   // r^-3 (refined)
    const float2 bx = __fadd2_rn(bc2(aj.x), p.nax), by = __fadd2_rn(bc2(aj.y), p.nay),
                 bz = __fadd2_rn(bc2(aj.z), p.naz);
    const float2 dot = __ffma2_rn(bx, dx, __ffma2_rn(by, dy, __fmul2_rn(bz, dz)));
    const float2 q = __fmul2_rn(r3, __fmul2_rn(y2, __ffma2_rn(bc2(3.0f), sres, bc2(-6.0f))));
    const float2 s = __fmul2_rn(q, dot);
    const float2 tx = __ffma2_rn(r3, bx, __fmul2_rn(s, dx)), ty = __ffma2_rn(r3, by, __fmul2_rn(s, dy)),
                 tz = __ffma2_rn(r3, bz, __fmul2_rn(s, dz));
    const float2 mj = bc2(aj.w);
    gi[0] = __ffma2_rn(mj, tx, gi[0]); gi[1] = __ffma2_rn(mj, ty, gi[1]); gi[2] = __ffma2_rn(mj, tz, gi[2]);
    gj[0] = __ffma2_rn(p.nm, tx, gj[0]); gj[1] = __ffma2_rn(p.nm, ty, gj[1]); gj[2] = __ffma2_rn(p.nm, tz, gj[2]);
}

__device__ __forceinline__ void x2_grad_near(const float4 h, const float4 l, const float4 aj, const X2I& p,
                                             float2 eps2, float2 (&gi)[3], float2 (&gj)[3]) {
    float2 dx, dy, dz, y2, sres, y3;
    x2_sep_near(h, l, p, dx, dy, dz);
    x2_geom(dx, dy, dz, eps2, y2, sres, y3);
    x2_grad_tail(dx, dy, dz, y2, sres, y3, aj, p, gi, gj);
}

__device__ __forceinline__ void x2_grad_far(const float4 r, const float4 aj, const float2 (&D)[3],
                                            const X2I& p, float2 eps2, float2 (&gi)[3], float2 (&gj)[3]) {
    const float2 dx = __fadd2_rn(D[0], bc2(r.x)), dy = __fadd2_rn(D[1], bc2(r.y)),
                 dz = __fadd2_rn(D[2], bc2(r.z));
    float2 y2, sres, y3;
    x2_geom(dx, dy, dz, eps2, y2, sres, y3);
    x2_grad_tail(dx, dy, dz, y2, sres, y3, aj, p, gi, gj);
}

// One group of 4 sources of the packed kernel (lane l visits source jj + (g ^ (l >> 3)) at
// step g); FG selects the far form, FULL drops the bounds check (a full 32-record sub-tile).
// The j-side totals of the group are left in jpart (one row per warp), or, with JG, added
// straight into the FP64 accumulator jg (rows of stride jstride, source jj at jg[jj]).
template <int KIND, int NP, bool FG, bool FULL, bool JG = false>
__device__ __forceinline__ void x2_group(int jj, int cnt, int lane, int warp, const RecMix* rec,
                                         const float4* arec, const float4* rel_s,
                                         const X2I (&pp)[NP], const float2 (&D)[NP][3],
                                         float2 eps2, float2 (&f)[NP][3], float* jpart,
                                         double* jg = nullptr, long long jstride = 0) {
    const int L = lane >> 3;
    float fj[4][3];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        fj[g][0] = fj[g][1] = fj[g][2] = 0.f;
        const int jg = jj + (g ^ L);
        if (FULL || jg < cnt) {
            float2 pj[3];
            pj[0] = make_float2(0.f, 0.f);
            pj[1] = make_float2(0.f, 0.f);
            pj[2] = make_float2(0.f, 0.f);
            if constexpr (FG) {
                const float4 r = rel_s[jg];
                if constexpr (KIND == KIND_ACC) {
#pragma unroll
                    for (int p = 0; p < NP; ++p) x2_acc_far(r, D[p], pp[p], eps2, f[p], pj);
                } else {
                    const float4 aj = arec[jg];
#pragma unroll
                    for (int p = 0; p < NP; ++p) x2_grad_far(r, aj, D[p], pp[p], eps2, f[p], pj);
                }
            } else {
                const float4 h = rec[jg].hi;
                const float4 l = rec[jg].lo;
                if constexpr (KIND == KIND_ACC) {
#pragma unroll
                    for (int p = 0; p < NP; ++p) x2_acc_near(h, l, pp[p], eps2, f[p], pj);
                } else {
                    const float4 aj = arec[jg];
#pragma unroll
                    for (int p = 0; p < NP; ++p) x2_grad_near(h, l, aj, pp[p], eps2, f[p], pj);
                }
            }
            fj[g][0] = pj[0].x + pj[0].y;
            fj[g][1] = pj[1].x + pj[1].y;
            fj[g][2] = pj[2].x + pj[2].y;
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
        if constexpr (JG) {
            red_add(jg + jl, (double)tot[0]);
            red_add(jg + jstride + jl, (double)tot[1]);
            red_add(jg + 2 * jstride + jl, (double)tot[2]);
        } else {
            float* dst = jpart + ((size_t)warp * kTileJ + jl) * 3;
            dst[0] = tot[0]; dst[1] = tot[1]; dst[2] = tot[2];
        }
    }
}

}  // namespace fsi
