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

cudaError_t launch_fma_probe(int fp64, int blocks, int iters, void* sink, cudaStream_t s) {
    if (fp64)
        { fma_probe_kernel<double><<<blocks, 256, 0, s>>>(iters, reinterpret_cast<double*>(sink)); note_launch(); }
    else
        { fma_probe_kernel<float><<<blocks, 256, 0, s>>>(iters, reinterpret_cast<float*>(sink)); note_launch(); }
    return cudaGetLastError();
}

}  // namespace fsi
