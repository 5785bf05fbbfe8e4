// noalloc.cu -- an acceleration entry point that allocates nothing.
//
// fsi_accel needs a context, and a context owns a workspace grown with cudaMalloc.  Some
// callers cannot allocate device memory at all: code running under a host framework that
// owns every device allocation (and forbids cudaMalloc outside its allocator), or code
// that must not allocate between the set-up of a stream capture and its end.  For them,
// fsi_accel_noalloc computes the same Newtonian accelerations (FP64 path) using a fixed
// scratch array that lives in this library's device image: a file-scope static __device__
// array, resident on every GPU that loads the library until the process exits.
//
// Scratch layout: packed source records (32 B per particle) followed by the partial sums
// of up to kSplitMax source slices.  Every call shares the array; a call overwrites every
// byte it later reads (records are packed, partial sums are written, not accumulated), so
// nothing needs to start at zero.  Two calls that overlap on the GPU (different streams,
// no ordering between them) race on the array.
//
// There is no error word either: a bounded wait of the pair kernel that runs out (a
// bulk copy that never lands) makes that CTA write quiet NaN into its results, and a
// non-finite result stays in the output, so every device-side failure shows up as a
// non-finite entry of acc_out.
#include <mutex>

#include "fsi_internal.cuh"

namespace fsi {
int set_last_error(int code, const char* msg);   // fsi_api.cu
}

namespace {

constexpr int kNoAllocMaxN = 32768;                                   // particles per call
constexpr int kSplitMax = 4;                                          // source slices
constexpr size_t kRecBytes = (size_t)kNoAllocMaxN * 32;               // 1 MiB
constexpr size_t kPartBytes = (size_t)kSplitMax * 3 * kNoAllocMaxN * sizeof(double);   // 3 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kRecBytes + kPartBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

// Device address of the scratch array on the current device and that device's SM count
// (both looked up once per device, under one lock).
int scratch_address(void** out, int* sms) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return fsi::set_last_error(FSI_ERR_CUDA, "fsi_accel_noalloc: no usable current device");
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fsi::set_last_error(FSI_ERR_CUDA, "fsi_accel_noalloc: cudaGetSymbolAddress failed");
        }
        int n_sm = 0;
        if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            n_sm <= 0) {
            cudaGetLastError();
            return fsi::set_last_error(FSI_ERR_CUDA, "fsi_accel_noalloc: SM count query failed");
        }
        g_sm_count[dev] = n_sm;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    *sms = g_sm_count[dev];
    return FSI_OK;
}

}  // namespace

extern "C" int fsi_accel_noalloc(int N, const double* pos, const double* mass, double eps2,
                                 double* acc_out, void* stream) {
    using namespace fsi;
    if (N <= 0 || !pos || !mass || !acc_out)
        return set_last_error(FSI_ERR_ARG, "fsi_accel_noalloc: bad arguments");
    if (N > kNoAllocMaxN)
        return set_last_error(FSI_ERR_ARG,
                              "fsi_accel_noalloc: N exceeds the fixed scratch capacity of 32768 "
                              "particles; use fsi_accel with a context");
    void* scratch = nullptr;
    int sms = 0;
    const int rc = scratch_address(&scratch, &sms);
    if (rc != FSI_OK) return rc;
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* base = reinterpret_cast<unsigned char*>(scratch);
    if (launch_pack(FSI_FP64, N, pos, mass, nullptr, N, base, nullptr, s) != cudaSuccess)
        return set_last_error(FSI_ERR_CUDA, "fsi_accel_noalloc: record packing failed to launch");
    // source slices: enough CTAs for two per SM when N is small, at least 4 tiles per slice
    const int ipt = 2;
    const int ctas = (N + kThreads * ipt - 1) / (kThreads * ipt);
    int split = 1;
    while (split < kSplitMax && ctas * split < 2 * sms && N / (split + 1) >= 4 * kTileJ) ++split;
    int jps = (N + split - 1) / split;
    jps = (jps + kTileJ - 1) / kTileJ * kTileJ;
    split = (N + jps - 1) / jps;
    PairArgs a{};
    a.irec = a.jrec = base;
    a.n_i = a.n_j = N;
    a.check = CHECK_DIAG;
    a.j_per_split = jps;
    a.eps2 = eps2;
    a.part = reinterpret_cast<double*>(base + kRecBytes);
    a.err = nullptr;
    a.timeout_ns = 2000000000LL;
    a.epi.out = acc_out;
    if (launch_pair(FSI_FP64, KIND_ACC, ipt, a, split, s) != cudaSuccess)
        return set_last_error(FSI_ERR_CUDA, "fsi_accel_noalloc: pair kernel failed to launch");
    if (split > 1 && launch_finalize_p(FSI_FP64, a, split, s) != cudaSuccess)
        return set_last_error(FSI_ERR_CUDA, "fsi_accel_noalloc: finalize kernel failed to launch");
    return FSI_OK;
}
