// fsi_internal.cuh -- internal types and device helpers of libfsi (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include "../../include/fsi.h"

namespace fsi {

// ---------------------------------------------------------------------------------
// Compact particle records.  A "set" of n particles is gathered once into records so
// that the O(n^2) kernels read contiguous, 16-byte-aligned tiles with bulk copies.
//
//  FP64 position record (32 B):  double4 (x, y, z, m)
//  FP64 accel record    (32 B):  double4 (ax, ay, az, m)
//  MIXED position record (32 B): float4 (xh, yh, zh, 2.5 m), float4 (xl, yl, zl, -1.5 m)
//        with xh = fl32(x) and xl = fl32(x - xh): xh + xl carries ~48 bits of x, so a
//        pair difference (xh_j - xh_i) + (xl_j - xl_i) is accurate to FP32 precision
//        relative to the separation even when |x| >> |r_ij|.  The two mass multiples
//        fold the residual correction of the hardware rsqrt into one FMA:
//        m r^-3 = y^3 (2.5 m - 1.5 m r^2 y^2) to first order in e = 1 - r^2 y^2.
//  MIXED accel record   (16 B):  float4 (ax, ay, az, m)
// ---------------------------------------------------------------------------------
struct alignas(32) D4 { double x, y, z, w; };   // 32-byte aligned FP64 quadruple
__host__ __device__ __forceinline__ D4 make_d4(double x, double y, double z, double w) {
    D4 r; r.x = x; r.y = y; r.z = z; r.w = w; return r;
}
struct RecF64 { double x, y, z, m; };
struct RecMix { float4 hi; float4 lo; };
static_assert(sizeof(RecF64) == 32 && sizeof(RecMix) == 32, "record size");

__device__ __forceinline__ RecMix make_mix_rec(double x, double y, double z, double m) {
    const float xh = (float)x, yh = (float)y, zh = (float)z;
    RecMix r;
    r.hi = make_float4(xh, yh, zh, (float)(2.5 * m));
    r.lo = make_float4((float)(x - (double)xh), (float)(y - (double)yh), (float)(z - (double)zh),
                       (float)(-1.5 * m));
    return r;
}

constexpr int kThreads = 256;      // threads per pair-kernel CTA
constexpr int kTileJ = 256;        // sources per shared-memory tile
constexpr int kStages = 3;         // bulk-copy pipeline depth

enum Kind { KIND_ACC = 0, KIND_GRAD = 1 };
enum Check { CHECK_NONE = 0, CHECK_DIAG = 1, CHECK_IDS = 2 };

// Epilogue of a pair pass, applied by the owner of particle i once its sum is complete.
//   out     : if non-null, out[c * n_i + i] = result_c              (3 x n_i FP64)
//   kick    : if x != null:  v += c_kick * (base + c_grad * result)  (base = a_i for
//             the gradient pass, 0 otherwise -> v += c_kick * result for acc)
//             then x += c_drift * v, and the new position record is written to rec_out.
//   accrec  : if non-null, the accel record of i is written there (acc pass feeding grad)
struct Epi {
    double* out;
    double* x;          // FP64 master positions, 3 x n_i compact or global (ids) (may be null)
    double* v;          // velocities, 3 x n_i compact or global (ids)
    const double* base; // compact 3 x n_i (grad pass: a_i), may be null
    double c_kick, c_grad, c_drift;
    void* rec_out;      // position records for the next pass
    const double* mc;   // FP64 masses, compact or global (ids) (needed when rec_out is written)
    void* accrec;       // accel records (FP64: RecF64-like double4; MIXED: float4)
    const int* ids;     // non-null: x, v, mc are global arrays (rows of ld), entry i at ids[i]
    long long ld;
};

struct PairArgs {
    const void* irec; const void* jrec;   // position records
    const void* iacc; const void* jacc;   // accel records (gradient pass)
    const int* iid; const int* jid;       // global ids (CHECK_IDS); jid padded to 4
    int n_i, n_j;
    int check;                            // Check
    int i_off;                            // CHECK_DIAG: receiver k is source k + i_off (the
                                          // receivers a sub-range of the source list)
    int j_per_split;                      // sources per blockIdx.y slice
    double eps2;
    double* part;                         // split > 1: partial sums [split][3][n_i]
    int* err;
    long long timeout_ns;
    Epi epi;
};

// ---------------------------------------------------------------------------------
// Raises the dynamic shared-memory limit of kernel fn to `bytes` once per device: the
// attribute belongs to the function on the current device, so a process with contexts on
// several GPUs sets it on each (bit d of `devices` records device d < 64; others set it on
// every call).
template <class F>
inline cudaError_t smem_attr_once(F* fn, int bytes, std::atomic<unsigned long long>& devices) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
    if (bit && (devices.load(std::memory_order_relaxed) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) devices.fetch_or(bit, std::memory_order_relaxed);
    return e;
}

// ---------------------------------------------------------------------------------
// Error word helpers.
__device__ __forceinline__ void set_error(int* err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// mbar_wait_bounded with err == nullptr only gives up silently.

__device__ __forceinline__ long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

// ---------------------------------------------------------------------------------
// mbarrier + bulk-copy (TMA, non-tensor) helpers, inline PTX.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Global -> shared bulk copy completing on `bar`.  dst, src 16-byte aligned; bytes a
// multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait: spins until the phase with `parity` completes or the wall-clock budget
// runs out; on timeout latches FSI_ERR_TIMEOUT and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long budget_ns, int* err) {
    if (mbar_try_wait(bar, parity)) return true;
    long long t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > budget_ns) {
            set_error(err, FSI_ERR_TIMEOUT);
            return false;
        }
    }
}

// FP32 reciprocal square root from the hardware approximation (MUFU).
__device__ __forceinline__ float rsqrt_hw(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

}  // namespace fsi

// ---------------------------------------------------------------------------------
// Batched ensemble (batch_kernels.cu): one work item = (cluster, i-block) of one phase.
struct BatchItem {
    int cluster, block, off, n;
};

// Symmetric form (mixed precision): a sum item is (cluster, i-block, source tiles
// [t0, t1) of the cluster); t0 == block * I marks the block's own tiles (one-sided).
struct BatchSymItem {
    int cluster, block, off, n, t0, t1;
};

struct BatchArgs {
    const BatchItem* items;      // items_per_phase entries
    int items_per_phase;
    int nphase;
    int nsteps;
    const int* nblocks;          // per cluster (index = cluster id)
    double* x;                   // 3 x Ntot
    double* v;
    const double* m;             // Ntot
    long long ntot;
    void* rec0;
    void* rec1;
    void* accrec;
    double* ac;                  // 3 x Ntot, FP64 accelerations of the gradient pass
    unsigned long long* stats;   // [0] += wait ns, [1] += CTA lifetime ns (may be null)
    int* done;                   // K x nphase, zeroed before the launch
    int* next;                   // work counter, zeroed
    int* abort_flag;             // zeroed
    double h, eps2;
    int* err;
    long long timeout_ns;
};


// Small-set HHS recursion in one CTA (hhs_small.cu).
struct SmallArgs {
    const int* ids;                 // global ids of the set, n entries
    int n;
    double* pos;                    // 3 x N
    double* vel;
    const double* mass;
    const double* step0;            // level-0 steps (global id)
    long long N;
    double tau;
    int level;
    int max_level;
    double eps2, eta_ff, eta_fb, eta_jerk;
    double eta_grad, eta_va;        // gradient / velocity-per-acceleration criteria (0 = off)
    unsigned long long* level_counts;   // per level (device)
    unsigned long long* work;           // [0] acc pairs, [1] grad pairs
    int* maxlevel_hit;
    int* err;
    const unsigned char* is_bh;     // PN1.0 pair flags (global id), used when c > 0
    double c;
};

// HHS recursion of a mid-size set in one cooperative launch over the GPU (hhs_grid.cu).
// Scratch arrays are indexed by global particle id (N entries) unless noted.
struct GridArgs {
    SmallArgs s;                    // root set, state, parameters, statistics (as above)
    double* step0w;                 // level-0 steps, recorded when the root is level 0
    int small_cap;                  // fast sets of <= small_cap recurse in CTA 0 (one-CTA form)
    void* rec[2];                   // position records (RecMix / D4), two buffers
    void* arec;                     // acceleration records (float4 / D4)
    void* vrec;                     // velocity records (float4 / D4) for the time steps
    double* acc;                    // 3 x N: a of the current pass (gradient-kick base)
    double* aux;                    // 3 x N: G of the gradient time-step criteria
    double* st;                     // time steps
    int* lists;                     // list stack (list_cap entries)
    long long list_cap;
    unsigned long long* bar;        // [0] arrivals, [1] abort; zeroed before each launch
    long long timeout_ns;           // budget of every barrier wait
    int latch_maxlevel;             // also latch FSI_ERR_MAXLEVEL in err on a depth-cap hit
    unsigned long long* prof;       // optional phase profile (16 words), or nullptr
    int* bhl;                       // black-hole sublists of the frames' S and F (list_cap)
    double* pnpart;                 // PN partial sums of black-hole receivers
    long long pnpart_cap;           // doubles in pnpart
};

// ---------------------------------------------------------------------------------
// Host-side launchers (defined in pair_kernels.cu / aux_kernels.cu).
namespace fsi {
void note_launch();                 // counts every kernel launch (fsi_launch_count)
cudaError_t launch_fma_probe(int fp64, int blocks, int iters, void* sink, cudaStream_t s);
// variant: active particles per thread (ipt, low 4 bits) + 16 if the mixed kernel
// accumulates its tile partials as float-float pairs (see pair_variants).
cudaError_t launch_pair(int precision, int kind, int ipt, const PairArgs& a, int split,
                        cudaStream_t s);
// fsi_kick_drift's kernel (global SoA state, optional id list).
cudaError_t launch_kick_drift_ids(long long N, double* pos, double* vel, const double* acc,
                                  const int* idx, int n, double c_kick, double c_drift,
                                  int sm_count, cudaStream_t s);
cudaError_t launch_finalize_p(int precision, const PairArgs& a, int split, cudaStream_t s);
// Wide one-sided pass (2^lg lanes per receiver, split source slices); split == 1 applies
// the epilogue itself, split > 1 writes a.part for launch_finalize_p.
cudaError_t launch_wide_pair(int precision, int kind, bool diag, const PairArgs& a, int lg,
                             int split, cudaStream_t s);
// Two unmasked wide passes (one source slice each) in one launch; each applies its epilogue.
cudaError_t launch_wide_pair2(int precision, int kind, const PairArgs& a, const PairArgs& b,
                              int lga, int lgb, cudaStream_t s);
struct SymFar;
// Bipartite symmetric pass (mixed: packed form; FP64: symmetric FP64 pair terms): every
// pair of the disjoint sets S (i: n_i) and F (j: n_j) once, S's sums added into acc_i
// (3 x n_i) and F's into acc_j (3 x n_j), both zeroed by the caller; `chunk` F tiles per
// work item.
cudaError_t launch_cross_pair(int precision, int kind, const void* irec, const void* iacc,
                              int n_i, const void* jrec, const void* jacc, int n_j, double eps2,
                              int chunk, double* acc_i, double* acc_j, int* err,
                              long long timeout_ns, cudaStream_t s, const SymFar* far = nullptr);
int cross_block_size(int precision);
// Symmetric self-interaction pass (every unordered pair once); adds into accum (3 x n,
// zeroed by the caller); `chunk` source tiles per work item.
// Far-tile inputs of the symmetric mixed kernel (second form with bit 64 in its variant):
// rel[k] = (x_k - C, y_k - C, z_k - C, m_k) in FP32 with C the centre of k's 32-record
// sub-tile, sub[k / 32] = (C, R), R >= max |rel.xyz| over the sub-tile (launch_subtiles);
// a warp takes the far form for a sub-tile when the gap between its particles' box and C
// is at least sqrt(k2) R.  stats (nullable): += [far, near] sub-tile visits.
struct SymFar {
    const void* rel;
    const void* sub;
    float k2;
    unsigned long long* stats;
};
// skip_diag (packed form only): the blocks' own pairs are left out, for launch_sym_diag_ff.
// part / nparts: only the work items of share `part` of the pass (a contiguous range of
// i-blocks with about 1/nparts of the tile visits); the shares' sums add up to the pass.
cudaError_t launch_sym_pair(int precision, int kind, int ipt, const void* rec, const void* accrec,
                            int n, double eps2, int chunk, double* accum, int* err,
                            long long timeout_ns, const SymFar* far, cudaStream_t s,
                            bool skip_diag = false, int part = 0, int nparts = 1);
// The pairs inside each block of bsz consecutive members of a mixed-precision set
// (records rec, n members), each member's sum over its block's other members in
// float-float arithmetic, added into accum (3 x n); part / nparts: the blocks of that
// share of the symmetric launch with blocks of bsz.
cudaError_t launch_sym_diag_ff(const void* rec, int n, int bsz, double eps2, double* accum,
                               cudaStream_t s, int part = 0, int nparts = 1);
// Supported ipt values for (precision, kind): writes up to 16 into out, returns the count.
int pair_variants(int precision, int kind, int* out);
int pair_default_ipt(int precision, int kind);
// Variants of the symmetric kernels: active particles per thread (low 4 bits), + 32 for the
// mixed second form (FP64 sums in shared memory, select-free reduce-scatter).
int sym_variants(int precision, int kind, int* out);
int variant_ipt(int variant);
// Particles per i-block of a symmetric variant (threads per CTA x particles per thread).
int sym_block_particles(int variant);

// Spatial ordering and far-tile inputs (order_kernels.cu).
size_t morton_workspace_bytes(int n);
cudaError_t launch_morton_order(int n, const double* xc, long long ld, int* perm, void* ws,
                                size_t ws_bytes, cudaStream_t s);
cudaError_t launch_compose(const int* idx, const int* perm, int n, int* list, cudaStream_t s);
cudaError_t launch_rel_mass(const double* mass, const int* idx, int n, void* rel, cudaStream_t s);
// mass_from_rec: rel.w from the records' 2.5 m instead of a preceding launch_rel_mass.
cudaError_t launch_subtiles(int n, const void* rec, void* rel, void* sub, cudaStream_t s,
                            bool mass_from_rec = false);

// launch_pack of two id lists (no compact copies) in one launch.
cudaError_t launch_pack2(int precision, int N, const double* pos, const double* mass,
                         const int* ida, int na, void* rec_a, const int* idb, int nb, void* rec_b,
                         cudaStream_t s);
cudaError_t launch_pack(int precision, int N, const double* pos, const double* mass,
                        const int* idx, int n, void* rec, double* xc, cudaStream_t s);
cudaError_t launch_pack_acc(int precision, int N, const double* accg, const double* mass,
                            const int* idx, int n, void* accrec, double* ac, cudaStream_t s);
cudaError_t launch_gather3(int N, const double* src, const int* idx, int n, double* dst,
                           cudaStream_t s);
cudaError_t launch_scatter3(int N, const double* src, const int* idx, int n, double* dst,
                            cudaStream_t s);
cudaError_t launch_scatter_axpy3(int N, const double* a, const int* idx, int n, double w,
                                 double* v, cudaStream_t s);
cudaError_t launch_gather1(int N, const double* src, const int* idx, int n, double* dst,
                           cudaStream_t s);
cudaError_t launch_gather_u8(const unsigned char* src, const int* idx, int n,
                             unsigned char* dst, cudaStream_t s);
cudaError_t launch_ids(const int* idx, int n, int cap, int* ids, cudaStream_t s);
cudaError_t launch_check_disjoint(int N, const int* A, int nA, const int* B, int nB,
                                  unsigned char* mark, int* err, cudaStream_t s);
cudaError_t launch_kick_drift(int precision, int n, double* xc, double* vc, const double* ac,
                              double c_kick, double c_drift, const double* mc, void* rec_out,
                              cudaStream_t s);
cudaError_t launch_axpy3(int n, double* v, const double* a, double w, cudaStream_t s);
// FSI with binary subsystems (subsys_kernels.cu): keys of the set (global id for singles,
// N + s for both members of binary s) and the members' set positions; the exact two-body
// flow of every binary over time t; the drift of the single particles.
cudaError_t launch_sub_keys(int n, const int* idx, int N, const int* pairs, int n_pairs,
                            int* where, int* key, int* ppos, int* err, cudaStream_t s);
cudaError_t launch_kepler_pairs(int n_pairs, const int* ppos, int n, double* x, double* v,
                                const double* m, double t, int* err, cudaStream_t s);
cudaError_t launch_drift_singles(int n, double* x, const double* v, const int* key, int N, double w,
                                 cudaStream_t s);
constexpr int kMaxBHList = 1024;   // black holes per set handled by the PN kernels
constexpr int kGridPnChunk = 256;  // cooperative HHS launch: sources per black-hole PN item
constexpr int kPnPartCtas = 64;    // CTAs per black hole in the PN reduction
cudaError_t launch_bh_list(int n, const unsigned char* bhc, int* bh_list, int* n_bh, int* err,
                           cudaStream_t s);
cudaError_t launch_pn(int n, const double* xc, const double* vc, const double* mc,
                      const unsigned char* bhc, double c, const int* bh_list, const int* n_bh,
                      int max_bh, double* apn, double* part, int* err, cudaStream_t s);
// PN1.0 accelerations of the pairs between disjoint id lists A and B (pairs with a black
// hole): outA (3 x nA) and outB (3 x nB) overwritten.  Abh/Bbh: kMaxBHList ints each,
// nAbh/nBbh: one int each (workspace); part: kMaxBHList * 3 * kPnPartCtas doubles.
cudaError_t launch_pn_cross(long long N, const double* pos, const double* vel, const double* mass,
                            const unsigned char* is_bh, double c, const int* A, int nA, const int* B,
                            int nB, int* Abh, int* nAbh, int* Bbh, int* nBbh, double* outA,
                            double* outB, double* part, int* err, cudaStream_t s);
// PN1.0 accelerations of id list A from id list B (any overlap, self pairs skipped by id)
// through black-hole sublists (at most kMaxBHList black holes per list); workspace as
// launch_pn_cross; out (3 x nA) overwritten.
cudaError_t launch_pn_lists(long long N, const double* pos, const double* vel, const double* mass,
                            const unsigned char* is_bh, double c, const int* A, int nA, const int* B,
                            int nB, int* Abh, int* nAbh, int* Bbh, int* nBbh, double* out,
                            double* part, int* err, cudaStream_t s);
cudaError_t launch_pn_pairs(int N, const double* pos, const double* vel, const double* mass,
                            const unsigned char* is_bh, double c, const int* A, int nA,
                            const int* B, int nB, double* out, int* err, cudaStream_t s);
int energy_blocks(int n);
cudaError_t launch_energy(int n, const double* xc, const double* vc, const double* mc,
                          double eps2, double* part, double* out, int* err, cudaStream_t s);
// Time steps of entries [i_off, i_off + n_i) of the compact set (n_i < 0: all n) against
// all n entries, into step[0, n_i).
cudaError_t launch_timesteps(int n, const double* xc, const double* vc, const double* mc,
                             double eta_ff, double eta_fb, double eta_jerk, double eps2,
                             double* step, int* err, cudaStream_t s, int i_off = 0, int n_i = -1);
// rec_ws, vrec_ws: workspace of >= 32 n and 16 n bytes (mixed records, FP32 velocities)
// step[k] = min(step[k], gradient and velocity-per-acceleration steps) from the set's
// velocities vc, accelerations a and force-gradient sums G (all 3 x n).
cudaError_t launch_grad_steps(int n, const double* vc, const double* a, const double* G,
                              double eta_grad, double eta_va, double* step, cudaStream_t s);
// FP32 velocity records (vx, vy, vz, m) of a compact set.
// FP32 velocity records (vx, vy, vz, m) of the set idx (null: the first n) of 3 x N rows;
// with pos non-null also the mixed position records into rec.
cudaError_t launch_pack_vel(int N, const double* vel, const double* mass, const int* idx, int n,
                            void* vrec, const double* pos, void* rec, cudaStream_t s);
// Mixed time steps with packed FP32 pairs (steps_x2.cu); part: steps_x2_part_bytes bytes.
size_t steps_x2_part_bytes(int n, int sm_count, int n_i = -1);   // n_i receivers (-1: n)
// Symmetric mixed time steps (every unordered pair once) for sets of at least
// steps_sym_min_n() particles; work: steps_sym_work_bytes(n) bytes (8-byte aligned).
size_t steps_sym_work_bytes(int n);
int steps_sym_min_n();
// rel, sub (nullable): far-tile offset records and sub-tile (centre, radius) records of the
// set (launch_subtiles); a warp takes the far-tile separation for a sub-tile whose gap to
// its receivers' box is at least sqrt(far_k2) R.
cudaError_t launch_steps_sym(int n, const void* rec, const void* vrec, double eps2, double eta_ff,
                             double eta_fb, double eta_jerk, void* work, double* step, int* err,
                             long long timeout_ns, int sm_count, cudaStream_t s,
                             const void* rel = nullptr, const void* sub = nullptr,
                             float far_k2 = 0.f);
// Symmetric FP64 time steps (steps_f64.cu, every unordered pair once) of the set idx (null:
// the first n) of the 3 x N rows, for sets of at least steps_sym_f64_min_n() particles.
// rec, vrec: workspace of >= 32 n bytes each (16-byte aligned), filled with the set's
// position and velocity records; work: steps_sym_f64_work_bytes(n) bytes (8-byte aligned).
size_t steps_sym_f64_work_bytes(int n);
int steps_sym_f64_min_n();
cudaError_t launch_steps_sym_f64(int N, const double* pos, const double* vel, const double* mass,
                                 const int* idx, int n, void* rec, void* vrec, double eps2,
                                 double eta_ff, double eta_fb, double eta_jerk, void* work,
                                 double* step, int* err, long long timeout_ns, int sm_count,
                                 cudaStream_t s);
// Mixed time steps (one-sided packed kernel, or its wide form) of records [i_off, i_off +
// n_i) (n_i < 0: all n) against all n records, into step[0, n_i); part: split partials of
// at least steps_x2_part_bytes(n, sm_count, n_i) bytes.
cudaError_t launch_steps_x2(int n, const void* rec, const void* vrec, double eps2, double eta_ff,
                            double eta_fb, double eta_jerk, float* part, double* step, int* err,
                            long long timeout_ns, int sm_count, int wide_ctas, cudaStream_t s,
                            int i_off = 0, int n_i = -1);
cudaError_t launch_partition(int n, const int* ids, double* step, double* step0, int level0,
                             double tau, int force_slow, int* S, int* F, int* counts, cudaStream_t s);
cudaError_t launch_iota(int n, int* ids, cudaStream_t s);
cudaError_t launch_hhs_small(int precision, const SmallArgs& a, cudaStream_t s);
int small_max();
cudaError_t launch_hhs_grid(int precision, const GridArgs& a, int ctas, cudaStream_t s);
int grid_ctas(int precision, int sm_count);   // CTAs of one cooperative launch (0: none fit)
cudaError_t launch_batch(int precision, int ipt, int ctas, const BatchArgs& a, cudaStream_t s);
// Symmetric persistent ensemble kernel (mixed precision): phases pack, then per pair pass
// a sum phase (sitems, red.add into accum) and an apply phase (items: epilogue, accum
// cleared).  nsum: sum items per cluster.
// ipt: particles per thread, kBatchSymI or kBatchSymI15 (2 CTAs per SM) or kBatchSymI2
// (1 CTA per SM).
cudaError_t launch_batch_sym(int ipt, int ctas, const BatchArgs& a, const BatchSymItem* sitems,
                             int sitems_per_phase, const int* nsum, double* accum,
                             cudaStream_t s);
constexpr int kBatchSymI = 4;      // particles per thread of the symmetric ensemble kernel
constexpr int kBatchSymI15 = 6;    // its larger-block variants
constexpr int kBatchSymI2 = 8;
inline bool batch_sym_ipt(int ipt) {
    return ipt == kBatchSymI || ipt == kBatchSymI15 || ipt == kBatchSymI2;
}
int batch_sym_max_ctas_per_sm(int ipt);
int batch_block_size(int ipt);
int batch_max_ctas_per_sm(int precision, int ipt);
// Adjoint pair kernels (FP64): kind 0 = acceleration VJP (vec = cotangent u),
// kind 1 = gradient-sum VJP through r and m (vec = cotangent w, acc = accelerations).
// Adds sx * xbar-part into xbar (3 x n) and sm * mbar-part into mbar (n).
cudaError_t launch_vjp_pair(int kind, int n, const void* rec, const void* vec, const void* acc,
                            double eps2, double sx, double sm, double* xbar, double* mbar,
                            int* err, int sm_count, cudaStream_t s);
cudaError_t launch_lincomb3(int n, const double* a, const double* b, double c, double* out,
                            cudaStream_t s);
cudaError_t launch_scatter_add1(int n, const double* src, const int* idx, double* dst,
                                cudaStream_t s);
}  // namespace fsi
