// probe_kernels.cu -- FMA-pipe throughput probe (measures the FP32 / FP64 peaks that the
// pair kernels' roofline fractions are quoted against).
#include "fsi_internal.cuh"

namespace fsi {

template <class T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, T* sink) {
    T a0 = (T)threadIdx.x * (T)1e-3, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
    T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
    const T b = (T)0.999999, c = (T)1e-7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a0 = a0 * b + c; a1 = a1 * b + c; a2 = a2 * b + c; a3 = a3 * b + c;
            a4 = a4 * b + c; a5 = a5 * b + c; a6 = a6 * b + c; a7 = a7 * b + c;
        }
    }
    sink[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

// Packed FP32 form: fma.rn.f32x2 (two FP32 FMAs per instruction, sm_100 and later).
__global__ void __launch_bounds__(256) fma2_probe_kernel(int iters, float* sink) {
    const float t = (float)threadIdx.x * 1e-3f;
    float2 a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = make_float2(t + (float)k, t - (float)k);
    const float2 b = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f, 2e-7f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = __ffma2_rn(a[k], b, c);
    }
    float r = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) r += a[k].x + a[k].y;
    sink[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

cudaError_t launch_fma_probe(int fp64, int blocks, int iters, void* sink, cudaStream_t s) {
    if (fp64 == 2)
        { fma2_probe_kernel<<<blocks, 256, 0, s>>>(iters, reinterpret_cast<float*>(sink)); note_launch(); }
    else if (fp64)
        { fma_probe_kernel<double><<<blocks, 256, 0, s>>>(iters, reinterpret_cast<double*>(sink)); note_launch(); }
    else
        { fma_probe_kernel<float><<<blocks, 256, 0, s>>>(iters, reinterpret_cast<float*>(sink)); note_launch(); }
    return cudaGetLastError();
}

}  // namespace fsi
