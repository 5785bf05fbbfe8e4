// hhs_small.cu -- the one-CTA HHS recursion as its own launch (the recursion itself is
// in hhs_small.cuh, shared with the grid-wide form in hhs_grid.cu).
#include "hhs_small.cuh"

namespace fsi {

template <int P>
__global__ void __launch_bounds__(kSmallMax, 1) hhs_small_kernel(const SmallArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    small_run<P>(*reinterpret_cast<SmallSmem<P>*>(smem_raw), a);
}

size_t small_smem_bytes(int precision) {
    return precision == FSI_MIXED ? sizeof(SmallSmem<FSI_MIXED>) : sizeof(SmallSmem<FSI_FP64>);
}

int small_max() { return kSmallMax; }

cudaError_t launch_hhs_small(int precision, const SmallArgs& a, cudaStream_t s) {
    const size_t smem = small_smem_bytes(precision);
    static std::atomic<unsigned long long> attr_dev[2];
    {
        const cudaError_t e = precision == FSI_MIXED
            ? smem_attr_once(hhs_small_kernel<FSI_MIXED>, (int)smem, attr_dev[1])
            : smem_attr_once(hhs_small_kernel<FSI_FP64>, (int)smem, attr_dev[0]);
        if (e != cudaSuccess) return e;
    }
    if (precision == FSI_MIXED) { hhs_small_kernel<FSI_MIXED><<<1, kSmallMax, smem, s>>>(a); note_launch(); }
    else { hhs_small_kernel<FSI_FP64><<<1, kSmallMax, smem, s>>>(a); note_launch(); }
    return cudaGetLastError();
}

}  // namespace fsi
