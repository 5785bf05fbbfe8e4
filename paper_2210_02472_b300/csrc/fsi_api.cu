// fsi_api.cu -- host side of libfsi's C ABI (declared in include/fsi.h).
//
// The host code only gathers index lists into compact device records, schedules the
// pair passes and their fused epilogues, and walks the HHS hierarchy; every arithmetic
// step runs in the kernels of pair_kernels.cu and aux_kernels.cu.
#include <algorithm>
#include <climits>
#include <cmath>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fsi_internal.cuh"

using namespace fsi;

namespace {
std::atomic<long long> g_launches{0};
}

void fsi::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace fsi {
// Records a host-side error message for fsi_last_error (used by the context-free entry point).
int set_last_error(int code, const char* msg);
}

namespace {

thread_local std::string g_err = "";

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(FSI_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                            \
    } while (0)

#define CK(expr)                      \
    do {                              \
        int r_ = (expr);              \
        if (r_ != FSI_OK) return r_;  \
    } while (0)

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace

// Set-size classes of the symmetric variant table: the fastest kernel differs between
// small sets (latency-bound, few CTAs: fewest particles per thread wins) and large ones.
// One-sided passes with at least this many receivers (mixed: the packed form) form the
// second class of the one-sided variant table.
constexpr int kOneSidedLarge = 16384;
constexpr int kSymClasses = 3;
constexpr int kSymClassMin[kSymClasses] = {0, 32768, 196608};
inline int sym_class(int n) { return n >= kSymClassMin[2] ? 2 : (n >= kSymClassMin[1] ? 1 : 0); }

struct fsi_ctx {
    fsi_params p;
    int device = 0;
    int sm_count = 148;
    int* err_d = nullptr;
    int* err_h = nullptr;          // pinned
    int* counts_h = nullptr;       // pinned, 3 ints (HHS partition)
    Buf rec[2], accrec[2], xc, vc, ac, ad, tA, tB, mc, bhc, ids[2], part, mark, bhlist,
        nbh, apn, pnpart, epart, iota, steps, step0, counts, accum, eout, snapx, snapv,
        subwhere, subkey, subppos, stpart;
    std::vector<Buf> lvS, lvF;
    Buf vj[24];                     // adjoint work arrays
    Buf dstats;                     // device HHS stats: level counts (64), work (2), flags
    Buf pnids;                      // fsi_pn_accel: the ids 0 .. N-1 for a NULL list
    std::vector<long long> level_counts;
    int max_level_used = 0;
    int max_level_hit = 0;
    // [precision][kind][receivers >= kOneSidedLarge] one-sided kernel variant (pair_variants):
    // mixed sets of many receivers take the packed FP32x2 form
    int ipt[2][2][2] = {{{2, 2}, {2, 2}}, {{4, 36}, {2, 36}}};
    // [precision][kind][size class] symmetric kernel variant (sym_variants)
    int symv[2][2][kSymClasses] = {{{2, 2, 2}, {2, 2, 2}}, {{226, 228, 230}, {226, 228, 246}}};
    long long work_pairs[2] = {0, 0};   // ordered pairs evaluated by acc / grad passes
    // far-tile path of the symmetric mixed kernel: while far_n > 0, the records of the set
    // being stepped (n = far_n) have valid masses in rel[].w (step_core, autotune)
    Buf rel, sub, ordws, ordperm, ordlist, farstats;
    // HHS recursion of mid-size sets in one cooperative launch (hhs_grid.cu): scratch by
    // particle id, list stack, barrier words; CTAs per launch (-1: not yet queried)
    Buf grec[2], garec, gvrec, gacc, gaux, gst, glists, gbar, gprof, gbhl, gpnpart;
    int grid_nctas[2] = {-1, -1};
    bool stats_on_device = false;   // the last interval was captured: its level statistics
                                    // are read from dstats by fsi_level_stats
    int far_n = 0;
    // far-tile path of the bipartite kernel: set while an HHS interval runs on level lists
    // in Morton order; xrel/xsub hold the sub-tiles of the smaller set of a pass
    bool lists_ordered = false;
    Buf xrel, xsub;
    // fsi_accel_part / fsi_grad_part: the share of the same-set pass run_pair evaluates
    int share_part = 0, share_n = 1;
    // instrumentation: event pairs around pair-kernel launches
    struct ProfRec { int kind; cudaEvent_t a, b; };
    bool profiling = false;
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> ev_pool;
};

namespace {

int ensure(Buf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return FSI_OK;
    if (b.p) {
        CU(cudaFree(b.p));
        b.p = nullptr;
        b.bytes = 0;
    }
    size_t want = (bytes + 255) & ~size_t(255);
    if (cudaMalloc(&b.p, want) != cudaSuccess) {
        cudaGetLastError();
        return fail(FSI_ERR_NOMEM, "cudaMalloc of %zu bytes failed", want);
    }
    b.bytes = want;
    return FSI_OK;
}

template <class T>
T* P(Buf& b) { return reinterpret_cast<T*>(b.p); }

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

long long budget(const fsi_ctx* c) { return c->p.timeout_ns > 0 ? c->p.timeout_ns : 2000000000LL; }

size_t pad_tile(int n) { return (size_t)((n + kTileJ - 1) / kTileJ) * kTileJ; }

// Source-split factor: the smallest S whose CTA count (i-blocks x S) fills the resident
// slots of the GPU (2 CTAs/SM) to >= 90 % in the last wave, keeping >= 4 tiles per slice.
// Default size cap of a fast set whose HHS recursion runs inside one CTA (the kernel holds
// up to 512): with the wide pair passes for the host-walked small levels, sets of 257 to
// 512 particles are faster walked from the host (one HHS interval of 65536 particles,
// mixed: 279.6 ms at 512, 269.5 ms at 256 and 128).
constexpr int kSmallCapDefault = 256;
// Default size cap of a fast set whose HHS recursion runs in one cooperative launch over
// the GPU (hhs_grid.cu); larger sets are walked from the host.
constexpr int kGridCapDefault = 4096;

int choose_split(const fsi_ctx* c, int n_i, int n_j, int ipc) {
    const int ctas = (n_i + ipc - 1) / ipc;
    const int max_s = std::max(1, std::min(64, n_j / (4 * kTileJ)));
    if (c->p.split > 0) return std::min(c->p.split, max_s);
    const int slots = c->sm_count * 2;
    int best = 1;
    double best_eff = 0.0;
    for (int s = 1; s <= max_s; ++s) {
        const long long tot = (long long)ctas * s;
        const long long waves = (tot + slots - 1) / slots;
        const double eff = (double)tot / (double)(waves * slots);
        if (eff >= 0.9) return s;
        if (eff > best_eff + 1e-9) { best_eff = eff; best = s; }
    }
    return best;
}

cudaEvent_t get_event(fsi_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Launch f() bracketed by an event pair when profiling is on.
template <class F>
int timed(fsi_ctx* c, int kind, cudaStream_t s, F&& f) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->profiling) {
        e0 = get_event(c);
        e1 = get_event(c);
        if (e0 && e1) CU(cudaEventRecord(e0, s));
    }
    CU(f());
    if (c->profiling && e0 && e1) {
        CU(cudaEventRecord(e1, s));
        c->prof.push_back({kind, e0, e1});
    }
    return FSI_OK;
}

// Far-tile test of the symmetric mixed kernel: the gap between a warp's particles and a
// sub-tile centre must be at least (kFarKappa + 1) R, so that every source of the
// sub-tile is at least kFarKappa times its offset from the centre away from every
// particle of the warp.
constexpr float kFarKappa = 3.0f;
// Sets of at least this many particles are put in Morton order by step_core when the
// symmetric mixed far-tile kernel is selected (order_min = 0).
constexpr int kOrderMinDefault = 32768;
// Bipartite passes take the far-tile path when the level lists are in Morton order and
// the smaller set has at least this many particles (or order_min, if lower).
constexpr int kCrossFarMin = 16384;

int order_threshold(const fsi_ctx* c) {
    if (c->p.order_min < 0) return INT_MAX;
    return c->p.order_min > 0 ? c->p.order_min : kOrderMinDefault;
}

// Does a set of n particles run a far-tile kernel (and so want Morton order)?
bool far_selected(const fsi_ctx* c, int n) {
    const int k = sym_class(n);
    return c->p.precision == FSI_MIXED && c->p.symmetric &&
           ((c->symv[FSI_MIXED][KIND_ACC][k] & 64) || (c->symv[FSI_MIXED][KIND_GRAD][k] & 64));
}

// Morton order of a set: ordlist[k] = member at sorted position k (global index).
// pos rows have leading dimension N; idx (nullable, then n == N) lists the members.
int order_set(fsi_ctx* c, int N, const double* pos, const int* idx, int n, cudaStream_t s) {
    const double* xs = pos;
    long long ld = N;
    if (idx) {
        CK(ensure(c->xc, 3 * (size_t)n * 8));
        CU(launch_gather3(N, pos, idx, n, P<double>(c->xc), s));
        xs = P<double>(c->xc);
        ld = n;
    }
    CK(ensure(c->ordperm, (size_t)n * 4));
    CK(ensure(c->ordlist, (size_t)n * 4));
    const size_t wsb = morton_workspace_bytes(n);
    CK(ensure(c->ordws, wsb));
    CU(launch_morton_order(n, xs, ld, P<int>(c->ordperm), c->ordws.p, c->ordws.bytes, s));
    CU(launch_compose(idx, P<int>(c->ordperm), n, P<int>(c->ordlist), s));
    return FSI_OK;
}

// Far-tile set-up for the set list (nullable) of n members: masses into rel[].w.
int far_setup(fsi_ctx* c, const double* mass, const int* list, int n, cudaStream_t s) {
    CK(ensure(c->rel, pad_tile(n) * 16));
    CK(ensure(c->sub, (pad_tile(n) / 32) * 16));
    CU(launch_rel_mass(mass, list, n, c->rel.p, s));
    c->far_n = n;
    return FSI_OK;
}

struct FarGuard {
    fsi_ctx* c;
    ~FarGuard() { c->far_n = 0; }
};

// Same-set passes of fsi_accel / fsi_grad / fsi_accel_grad with the far-tile kernel: the
// set runs in Morton order (list = ordlist) with outputs in workspace rows, and unsort()
// scatters each output back to the caller's order.
struct SameSetOrder {
    bool on = false;
    const int* list = nullptr;
    int begin(fsi_ctx* c, int N, const double* pos, const double* mass, const int* A, int n,
              cudaStream_t s) {
        list = A;
        on = far_selected(c, n) && n >= order_threshold(c);
        if (!on) return FSI_OK;
        CK(order_set(c, N, pos, A, n, s));
        list = P<int>(c->ordlist);
        CK(far_setup(c, mass, list, n, s));
        return FSI_OK;
    }
    // out[:, perm[k]] = sorted[:, k]  (both 3 x n)
    int unsort(fsi_ctx* c, const double* sorted, int n, double* out, cudaStream_t s) {
        CU(launch_scatter3(n, sorted, P<int>(c->ordperm), n, out, s));
        return FSI_OK;
    }
};

// Source tiles per work item of the symmetric kernel: about 8 items per resident CTA
// slot, at most 64 tiles each.
int choose_chunk(const fsi_ctx* c, int n, int variant) {
    const long long ntj = (n + kTileJ - 1) / kTileJ;
    const long long bp = sym_block_particles(variant);
    const long long nb = (n + bp - 1) / bp;
    const long long visits = nb * ntj / 2 + 1;
    const long long want = 8LL * 2 * c->sm_count;
    long long ch = visits / want;
    return (int)std::max(1LL, std::min(64LL, ch));
}

// Wide form of a pass (lanes per receiver 2^lg, source slices split) when its tiled
// form would run fewer CTAs than wide_ctas (0: kWideCtasDefault): each lane keeps >= 8
// sources, and the slices aim at 16 resident warps per SM with >= 32 sources per lane.
// Measured on one HHS interval of 65536 particles (mixed): the wide form is faster
// below ~32 tiled CTAs and slower for the mid-size passes above (L1 loads of every
// source record per lane, where the tiled form broadcasts a staged tile).
constexpr int kWideCtasDefault = 32;

int wide_limit(const fsi_ctx* c) {
    return c->p.wide_ctas < 0 ? 0 : (c->p.wide_ctas > 0 ? c->p.wide_ctas : kWideCtasDefault);
}

bool wide_plan(const fsi_ctx* c, int n_i, int n_j, int ipc, int& lg, int& split) {
    if (c->p.wide_ctas < 0) return false;
    const long long limit = wide_limit(c);
    const long long tiled = (long long)((n_i + ipc - 1) / ipc) * choose_split(c, n_i, n_j, ipc);
    if (tiled >= limit) return false;
    lg = 5;
    while (lg > 0 && (8LL << lg) > n_j) --lg;
    const long long warps = (((long long)n_i << lg) + 31) / 32;
    const long long want = 16LL * c->sm_count;
    long long sp = (want + warps - 1) / warps;
    sp = std::min(sp, std::max(1LL, (long long)n_j / (32LL << lg)));
    split = (int)std::max(1LL, std::min(64LL, sp));
    return true;
}

int run_wide(fsi_ctx* c, int kind, PairArgs a, int lg, int split, cudaStream_t s) {
    const int prec = c->p.precision;
    const int jps = (a.n_j + split - 1) / split;
    split = std::max(1, (a.n_j + jps - 1) / jps);
    a.j_per_split = std::max(1, jps);
    a.err = c->err_d;
    if (split > 1) {
        CK(ensure(c->part, (size_t)split * 3 * a.n_i * sizeof(double)));
        a.part = P<double>(c->part);
    }
    const bool diag = a.check == CHECK_DIAG;
    CK(timed(c, kind, s, [&] { return launch_wide_pair(prec, kind, diag, a, lg, split, s); }));
    if (split > 1) CK(timed(c, 2, s, [&] { return launch_finalize_p(prec, a, split, s); }));
    return FSI_OK;
}

int run_pair(fsi_ctx* c, int kind, PairArgs a, cudaStream_t s);

// The two directions of a cross-level pass (independent, unmasked): one launch when both
// take the wide form with a single source slice, else one pass after the other.
int run_pair2(fsi_ctx* c, int kind, PairArgs a, PairArgs b, cudaStream_t s) {
    const int prec = c->p.precision;
    if (a.n_i > 0 && b.n_i > 0 && a.check == CHECK_NONE && b.check == CHECK_NONE) {
        const int ipa = kThreads * variant_ipt(c->ipt[prec][kind][a.n_i >= kOneSidedLarge]);
        const int ipb = kThreads * variant_ipt(c->ipt[prec][kind][b.n_i >= kOneSidedLarge]);
        int lga = 0, lgb = 0, spa = 1, spb = 1;
        if (wide_plan(c, a.n_i, a.n_j, ipa, lga, spa) && wide_plan(c, b.n_i, b.n_j, ipb, lgb, spb) &&
            spa == 1 && spb == 1) {
            c->work_pairs[kind] += (long long)a.n_i * a.n_j + (long long)b.n_i * b.n_j;
            a.err = b.err = c->err_d;
            a.j_per_split = std::max(1, a.n_j);
            b.j_per_split = std::max(1, b.n_j);
            CK(timed(c, kind, s, [&] { return launch_wide_pair2(prec, kind, a, b, lga, lgb, s); }));
            return FSI_OK;
        }
    }
    // symmetric: every S-F pair once in the bipartite kernel, the larger set in registers
    // (full receiver blocks), then one finalize launch per side
    if (c->p.symmetric && a.check == CHECK_NONE && b.check == CHECK_NONE &&
        a.irec == b.jrec && a.jrec == b.irec && a.n_i == b.n_j && a.n_j == b.n_i &&
        std::min(a.n_i, b.n_i) >= kTileJ) {
        PairArgs& L = a.n_i >= b.n_i ? a : b;
        PairArgs& M = a.n_i >= b.n_i ? b : a;
        c->work_pairs[kind] += 2LL * L.n_i * M.n_i;
        const size_t nL = (size_t)L.n_i, nM = (size_t)M.n_i;
        CK(ensure(c->accum, 3 * (nL + nM) * sizeof(double)));
        CU(cudaMemsetAsync(c->accum.p, 0, 3 * (nL + nM) * sizeof(double), s));
        double* accL = P<double>(c->accum);
        double* accM = accL + 3 * nL;
        const long long nb = (L.n_i + cross_block_size(prec) - 1) / cross_block_size(prec);
        const long long visits = nb * ((M.n_i + kTileJ - 1) / kTileJ);
        const int chunk = (int)std::max(1LL, std::min(64LL, visits / (8LL * c->sm_count)));
        L.err = M.err = c->err_d;
        SymFar far{};
        const SymFar* farp = nullptr;
        if (prec == FSI_MIXED && c->lists_ordered &&
            M.n_i >= std::min(kCrossFarMin, order_threshold(c))) {
            // F's sub-tiles (the lists inherit Morton order); masses from the records
            CK(ensure(c->xrel, pad_tile(M.n_i) * 16));
            CK(ensure(c->xsub, (pad_tile(M.n_i) / 32) * 16));
            CU(launch_subtiles(M.n_i, M.irec, c->xrel.p, c->xsub.p, s, true));
            far.rel = c->xrel.p;
            far.sub = c->xsub.p;
            far.k2 = (kFarKappa + 1.0f) * (kFarKappa + 1.0f);
            farp = &far;
        }
        CK(timed(c, kind, s, [&] {
            return launch_cross_pair(prec, kind, L.irec, L.iacc, L.n_i, M.irec, M.iacc, M.n_i, L.eps2,
                                     chunk, accL, accM, c->err_d, budget(c), s, farp);
        }));
        L.part = accL;
        M.part = accM;
        CK(timed(c, 2, s, [&] { return launch_finalize_p(prec, L, 1, s); }));
        CK(timed(c, 2, s, [&] { return launch_finalize_p(prec, M, 1, s); }));
        return FSI_OK;
    }
    CK(run_pair(c, kind, a, s));
    return run_pair(c, kind, b, s);
}

int run_pair(fsi_ctx* c, int kind, PairArgs a, cudaStream_t s) {
    if (a.n_i <= 0) return FSI_OK;
    c->work_pairs[kind] += (long long)a.n_i * (long long)a.n_j;
    const int prec = c->p.precision;
    const int ipt = c->ipt[prec][kind][a.n_i >= kOneSidedLarge];
    if (a.check == CHECK_NONE || a.check == CHECK_DIAG) {
        int lg = 0, split = 1;
        if (wide_plan(c, a.n_i, a.n_j, kThreads * variant_ipt(ipt), lg, split))
            return run_wide(c, kind, a, lg, split, s);
    }
    if (c->p.symmetric && a.check == CHECK_DIAG && a.irec == a.jrec && a.n_i == a.n_j &&
        a.iacc == a.jacc) {
        // self-interaction of one set: every unordered pair once, then the epilogue
        const int n = a.n_i;
        const int sv = c->symv[prec][kind][sym_class(n)];
        CK(ensure(c->accum, 3 * (size_t)n * sizeof(double)));
        CU(cudaMemsetAsync(c->accum.p, 0, 3 * (size_t)n * sizeof(double), s));
        const int chunk = choose_chunk(c, n, sv);
        a.err = c->err_d;
        a.timeout_ns = budget(c);
        SymFar far{};
        const SymFar* farp = nullptr;
        if (prec == FSI_MIXED && (sv & 64) && c->far_n == n) {
            if (!c->farstats.p) {
                CK(ensure(c->farstats, 2 * sizeof(unsigned long long)));
                CU(cudaMemsetAsync(c->farstats.p, 0, 2 * sizeof(unsigned long long), s));
            }
            CU(launch_subtiles(n, a.irec, c->rel.p, c->sub.p, s));
            far.rel = c->rel.p;
            far.sub = c->sub.p;
            far.k2 = (kFarKappa + 1.0f) * (kFarKappa + 1.0f);
            far.stats = P<unsigned long long>(c->farstats);
            farp = &far;
        }
        // mixed acceleration passes of the largest size class: the pairs inside each
        // i-block (each particle's nearest neighbours in Morton order) in float-float
        // arithmetic by their own kernel, which keeps the relative acceleration error of
        // every particle within ~1e-7
        const bool ff_diag = prec == FSI_MIXED && kind == KIND_ACC && (sv & 128) &&
                             n >= kSymClassMin[2];
        CK(timed(c, kind, s, [&] {
            cudaError_t e = launch_sym_pair(prec, kind, sv, a.irec, a.iacc, n, a.eps2, chunk,
                                            P<double>(c->accum), a.err, a.timeout_ns, farp, s, ff_diag,
                                            c->share_part, c->share_n);
            if (e == cudaSuccess && ff_diag)
                e = launch_sym_diag_ff(a.irec, n, sym_block_particles(sv), a.eps2, P<double>(c->accum), s,
                                       c->share_part, c->share_n);
            return e;
        }));
        a.part = P<double>(c->accum);
        CK(timed(c, 2, s, [&] { return launch_finalize_p(prec, a, 1, s); }));
        return FSI_OK;
    }
    const int ipc = kThreads * variant_ipt(ipt);
    int split = choose_split(c, a.n_i, a.n_j, ipc);
    int jps = (a.n_j + split - 1) / split;
    jps = std::max(kTileJ, (jps + kTileJ - 1) / kTileJ * kTileJ);
    split = std::max(1, (a.n_j + jps - 1) / jps);
    a.j_per_split = jps;
    a.err = c->err_d;
    a.timeout_ns = budget(c);
    if (split > 1) {
        CK(ensure(c->part, (size_t)split * 3 * a.n_i * sizeof(double)));
        a.part = P<double>(c->part);
    }
    CK(timed(c, kind, s, [&] { return launch_pair(prec, kind, ipt, a, split, s); }));
    if (split > 1) CK(timed(c, 2, s, [&] { return launch_finalize_p(prec, a, split, s); }));
    return FSI_OK;
}

bool valid_prec(int p) { return p == FSI_FP64 || p == FSI_MIXED; }

// Whether the same-set pass of n particles of this kind takes the tiled symmetric branch
// of run_pair: the only form whose work a share of fsi_accel_part / fsi_grad_part divides.
bool sym_same_set(const fsi_ctx* c, int kind, int n) {
    if (!c->p.symmetric || n <= 0) return false;
    const int ipt = c->ipt[c->p.precision][kind][n >= kOneSidedLarge];
    int lg = 0, split = 1;
    return !wide_plan(c, n, n, kThreads * variant_ipt(ipt), lg, split);
}

// Share `part` of nparts of a same-set pass: `run` evaluates the pass with the share set
// (its tiled symmetric form then takes only the share's work items); a pass without that
// form runs whole in share 0 and leaves zeros (3 x n in out) in the others.
template <class Run>
int run_share(fsi_ctx* c, int kind, int n, int part, int nparts, double* out, cudaStream_t s,
              Run run) {
    if (nparts < 1 || part < 0 || part >= nparts)
        return fail(FSI_ERR_ARG, "bad share %d of %d", part, nparts);
    if (nparts == 1) return run();
    if (!sym_same_set(c, kind, n)) {
        if (part == 0) return run();
        CU(cudaMemsetAsync(out, 0, 3 * (size_t)n * sizeof(double), s));
        return FSI_OK;
    }
    c->share_part = part;
    c->share_n = nparts;
    const int r = run();
    c->share_part = 0;
    c->share_n = 1;
    return r;
}

// Offset k of an id list A inside the id list B when A is the sub-range B[k, k + nA) (same
// memory: a slice of B, as a sharded pass hands each rank), else -1.
long long sub_range(const int* A, int nA, const int* B, int nB) {
    if (!A || !B || A == B) return -1;
    const uintptr_t a = reinterpret_cast<uintptr_t>(A), b = reinterpret_cast<uintptr_t>(B);
    if (a < b || (a - b) % sizeof(int)) return -1;
    const long long k = (long long)((a - b) / sizeof(int));
    return k + nA <= nB ? k : -1;
}

int check_common(fsi_ctx* c, int N) {
    if (!c) return fail(FSI_ERR_ARG, "NULL context");
    if (N <= 0) return fail(FSI_ERR_ARG, "N must be positive (got %d)", N);
    return FSI_OK;
}

// ---------------------------------------------------------------------------------
// FSI cycles of a set on itself (compact buffers; see fsi_step in fsi.h).
// Intermediates of one recorded FSI cycle (compact 3 x n, in the order of the set's ids):
// a(x0), a(x1) and G(x1) with x1 the positions after the first drift.
struct StepRecord {
    double* a0;
    double* a1;
    double* g1;
};

int step_core(fsi_ctx* c, int N, double* pos, double* vel, const double* mass,
              const unsigned char* is_bh, const int* idx, int n, double h, int nsteps,
              cudaStream_t s, const StepRecord* record = nullptr) {
    if (n <= 0 || nsteps <= 0) return FSI_OK;
    const int prec = c->p.precision;
    const bool pn = c->p.c > 0.0;
    if (pn && !is_bh) return fail(FSI_ERR_ARG, "PN on (c > 0) needs is_bh");
    if (record && (pn || nsteps != 1)) return fail(FSI_ERR_ARG, "a recorded step is one Newtonian cycle");
    CK(ensure(c->rec[0], pad_tile(n) * 32));
    CK(ensure(c->rec[1], pad_tile(n) * 32));
    CK(ensure(c->accrec[0], pad_tile(n) * 32));
    CK(ensure(c->ac, 3 * (size_t)n * 8));
    FarGuard far_guard{c};
    // a recorded cycle keeps the set's own order (its intermediates are returned in it)
    const bool far = !record && far_selected(c, n) && n >= order_threshold(c);
    if (far) {
        CK(order_set(c, N, pos, idx, n, s));
        idx = P<int>(c->ordlist);
        CK(far_setup(c, mass, idx, n, s));
    }
    double* xc = pos;
    double* vc = vel;
    const double* mc = mass;
    const unsigned char* bhc = is_bh;
    // Without PN every update of x and v happens in a pass epilogue, which reaches the
    // global state through the id list; the PN kernels work on a compact copy.
    const bool compact = idx && pn;
    const int* eids = (idx && !pn) ? idx : nullptr;
    if (compact) {
        CK(ensure(c->xc, 3 * (size_t)n * 8));
        CK(ensure(c->vc, 3 * (size_t)n * 8));
        CK(ensure(c->mc, (size_t)n * 8));
        xc = P<double>(c->xc);
        vc = P<double>(c->vc);
        CU(launch_gather3(N, vel, idx, n, vc, s));
        CU(launch_gather1(N, mass, idx, n, P<double>(c->mc), s));
        mc = P<double>(c->mc);
    }
    CU(launch_pack(prec, N, pos, mass, idx, n, c->rec[0].p, compact ? xc : nullptr, s));
    if (pn) {
        CK(ensure(c->ad, 3 * (size_t)n * 8));
        CK(ensure(c->apn, 3 * (size_t)n * 8));
        CK(ensure(c->bhlist, 2 * kMaxBHList * 4));
        CK(ensure(c->nbh, 16));
        CK(ensure(c->pnpart, (size_t)kMaxBHList * 3 * kPnPartCtas * 8));
        if (idx) {
            CK(ensure(c->bhc, (size_t)n));
            CU(launch_gather_u8(is_bh, idx, n, P<unsigned char>(c->bhc), s));
            bhc = P<unsigned char>(c->bhc);
        }
        CU(launch_bh_list(n, bhc, P<int>(c->bhlist), P<int>(c->nbh), c->err_d, s));
    }
    auto pn_kick = [&](double w) -> int {
        CU(launch_pn(n, xc, vc, mc, bhc, c->p.c, P<int>(c->bhlist), P<int>(c->nbh), kMaxBHList,
                     P<double>(c->apn), P<double>(c->pnpart), c->err_d, s));
        CU(launch_axpy3(n, vc, P<double>(c->apn), w, s));
        return FSI_OK;
    };
    auto acc_pass = [&](void* rin, void* rout, double ck, double cd, double* out, void* accrec) {
        PairArgs a{};
        a.irec = a.jrec = rin;
        a.n_i = a.n_j = n;
        a.check = CHECK_DIAG;
        a.eps2 = c->p.eps2;
        a.epi.out = out;
        a.epi.accrec = accrec;
        if (ck != 0.0 || cd != 0.0) {
            a.epi.v = vc;
            a.epi.x = xc;
            a.epi.c_kick = ck;
            a.epi.c_drift = cd;
            a.epi.rec_out = rout;
            a.epi.mc = mc;
            a.epi.ids = eids;
            a.epi.ld = N;
        }
        return run_pair(c, KIND_ACC, a, s);
    };
    auto grad_pass = [&](void* rin, void* rout, double ck, double cg, double cd) {
        PairArgs a{};
        a.irec = a.jrec = rin;
        a.iacc = a.jacc = c->accrec[0].p;
        a.n_i = a.n_j = n;
        a.check = CHECK_DIAG;
        a.eps2 = c->p.eps2;
        a.epi.v = vc;
        a.epi.x = xc;
        a.epi.base = P<double>(c->ac);
        a.epi.c_kick = ck;
        a.epi.c_grad = cg;
        a.epi.c_drift = cd;
        a.epi.rec_out = rout;
        a.epi.mc = mc;
        a.epi.ids = eids;
        a.epi.ld = N;
        return run_pair(c, KIND_GRAD, a, s);
    };
    void* r0 = c->rec[0].p;
    void* r1 = c->rec[1].p;
    if (pn) CK(pn_kick(0.5 * h));
    CK(acc_pass(r0, r1, h / 6.0, 0.5 * h, record ? record->a0 : nullptr, nullptr));
    for (int k = 0; k < nsteps; ++k) {
        const bool last = (k == nsteps - 1);
        double* a1 = record ? record->a1 : P<double>(c->ac);
        CK(acc_pass(r1, nullptr, 0.0, 0.0, a1, c->accrec[0].p));
        if (record) {
            // the gradient pass adds its kick to a(x1) from the record and returns G(x1)
            PairArgs a{};
            a.irec = a.jrec = r1;
            a.iacc = a.jacc = c->accrec[0].p;
            a.n_i = a.n_j = n;
            a.check = CHECK_DIAG;
            a.eps2 = c->p.eps2;
            a.epi.out = record->g1;
            a.epi.v = vc;
            a.epi.x = xc;
            a.epi.base = a1;
            a.epi.c_kick = 2.0 * h / 3.0;
            a.epi.c_grad = h * h / 24.0;
            a.epi.c_drift = 0.5 * h;
            a.epi.rec_out = r0;
            a.epi.mc = mc;
            a.epi.ids = eids;
            a.epi.ld = N;
            CK(run_pair(c, KIND_GRAD, a, s));
        } else {
            CK(grad_pass(r1, r0, 2.0 * h / 3.0, h * h / 24.0, 0.5 * h));
        }
        if (!pn && !last) {
            CK(acc_pass(r0, r1, h / 3.0, 0.5 * h, nullptr, nullptr));
        } else {
            CK(acc_pass(r0, nullptr, h / 6.0, 0.0, pn ? P<double>(c->ad) : nullptr, nullptr));
            if (pn) CK(pn_kick(0.5 * h));
            if (!last) {
                CK(pn_kick(0.5 * h));
                CU(launch_kick_drift(prec, n, xc, vc, P<double>(c->ad), h / 6.0, 0.5 * h, mc, r1, s));
            }
        }
    }
    if (compact) {
        CU(launch_scatter3(N, xc, idx, n, pos, s));
        CU(launch_scatter3(N, vc, idx, n, vel, s));
    }
    return FSI_OK;
}

// Inter-level kick of the slow set S and fast set F (Sect. 2.2):
//   gradient == 0:  v_S += w acc(S <- F),  v_F += w acc(F <- S)
//   gradient == 1:  the same with a~ = a + (eps^2/24) G of the same inter-level term.
int cross_kick(fsi_ctx* c, int N, const double* pos, double* vel, const double* mass,
               const int* Sids, int nS, const int* Fids, int nF, double w, int gradient,
               double eps, cudaStream_t s) {
    const int prec = c->p.precision;
    CK(ensure(c->rec[0], pad_tile(nS) * 32));
    CK(ensure(c->rec[1], pad_tile(nF) * 32));
    CK(ensure(c->accrec[0], pad_tile(nS) * 32));
    CK(ensure(c->accrec[1], pad_tile(nF) * 32));
    CK(ensure(c->tA, 3 * (size_t)nS * 8));
    CK(ensure(c->tB, 3 * (size_t)nF * 8));
    CU(launch_pack2(prec, N, pos, mass, Sids, nS, c->rec[0].p, Fids, nF, c->rec[1].p, s));
    // the kicks land on the global velocities through the id lists in the pass epilogues:
    // v += w a (acc passes), or v += w (a + (eps^2/24) G) (grad passes, a from tA / tB)
    auto kick = [&](Epi& e, const int* ids, double* base) {
        e.v = vel;
        e.ids = ids;
        e.ld = N;
        e.c_kick = w;
        if (base) {
            e.base = base;
            e.c_grad = eps * eps / 24.0;
        }
    };
    PairArgs a{};
    a.check = CHECK_NONE;
    a.eps2 = c->p.eps2;
    a.irec = c->rec[0].p; a.jrec = c->rec[1].p; a.n_i = nS; a.n_j = nF;
    PairArgs b{};
    b.check = CHECK_NONE;
    b.eps2 = c->p.eps2;
    b.irec = c->rec[1].p; b.jrec = c->rec[0].p; b.n_i = nF; b.n_j = nS;
    if (gradient) {
        a.epi.out = P<double>(c->tA);
        a.epi.accrec = c->accrec[0].p;
        b.epi.out = P<double>(c->tB);
        b.epi.accrec = c->accrec[1].p;
    } else {
        kick(a.epi, Sids, nullptr);
        kick(b.epi, Fids, nullptr);
    }
    CK(run_pair2(c, KIND_ACC, a, b, s));
    if (gradient) {
        a.iacc = c->accrec[0].p; a.jacc = c->accrec[1].p;
        a.epi = Epi{};
        kick(a.epi, Sids, P<double>(c->tA));
        b.iacc = c->accrec[1].p; b.jacc = c->accrec[0].p;
        b.epi = Epi{};
        kick(b.epi, Fids, P<double>(c->tB));
        CK(run_pair2(c, KIND_GRAD, a, b, s));
    }
    return FSI_OK;
}

// PN1.0 kick of the S-F pairs (both directions, velocities from the start of the kick).
int cross_pn_kick(fsi_ctx* c, int N, const double* pos, double* vel, const double* mass,
                  const unsigned char* is_bh, const int* Sids, int nS, const int* Fids, int nF,
                  double w, cudaStream_t s) {
    CK(ensure(c->tA, 3 * (size_t)nS * 8));
    CK(ensure(c->tB, 3 * (size_t)nF * 8));
    CK(ensure(c->bhlist, 2 * kMaxBHList * 4));
    CK(ensure(c->nbh, 16));
    CK(ensure(c->pnpart, (size_t)kMaxBHList * 3 * kPnPartCtas * 8));
    int* bl = P<int>(c->bhlist);
    int* nb = P<int>(c->nbh);
    CU(launch_pn_cross(N, pos, vel, mass, is_bh, c->p.c, Sids, nS, Fids, nF, bl, nb, bl + kMaxBHList,
                       nb + 1, P<double>(c->tA), P<double>(c->tB), P<double>(c->pnpart), c->err_d, s));
    CU(launch_scatter_axpy3(N, P<double>(c->tA), Sids, nS, w, vel, s));
    CU(launch_scatter_axpy3(N, P<double>(c->tB), Fids, nF, w, vel, s));
    return FSI_OK;
}

// Time steps of the set's entries [lo, hi) (hi < 0: all n) against the whole set, into
// step[0, hi - lo).  A proper sub-range takes the one-sided kernels and needs the gradient
// criteria off (the caller checks).
int timesteps_core(fsi_ctx* c, int N, const double* pos, const double* vel, const double* mass,
                   const int* Pids, int n, double* step, cudaStream_t s, int lo = 0, int hi = -1) {
    if (hi < 0) hi = n;
    if (n <= 0 || hi <= lo) return FSI_OK;
    const bool whole = lo == 0 && hi == n;
    const double* xc = pos;
    const double* vc = vel;
    const double* mc = mass;
    const bool mixed = c->p.precision == FSI_MIXED;
    const bool crit = c->p.eta_grad > 0.0 || c->p.eta_va > 0.0;
    const bool sym64 = !mixed && whole && c->p.symmetric && n >= steps_sym_f64_min_n();
    // compact copies for the one-sided FP64 kernel and the gradient criteria; the mixed
    // and the symmetric FP64 kernels pack their records straight from the global arrays
    // through the id list
    if (Pids && ((!mixed && !sym64) || crit)) {
        CK(ensure(c->xc, 3 * (size_t)n * 8));
        CK(ensure(c->vc, 3 * (size_t)n * 8));
        CK(ensure(c->mc, (size_t)n * 8));
        CU(launch_gather3(N, pos, Pids, n, P<double>(c->xc), s));
        CU(launch_gather3(N, vel, Pids, n, P<double>(c->vc), s));
        CU(launch_gather1(N, mass, Pids, n, P<double>(c->mc), s));
        xc = P<double>(c->xc);
        vc = P<double>(c->vc);
        mc = P<double>(c->mc);
    }
    if (mixed) {
        CK(ensure(c->rec[1], pad_tile(n) * 32));
        CK(ensure(c->accrec[1], pad_tile(n) * 32));
        const bool sym = whole && c->p.symmetric && n >= steps_sym_min_n();
        CK(ensure(c->stpart, sym ? steps_sym_work_bytes(n) : steps_x2_part_bytes(n, c->sm_count, hi - lo)));
        CU(launch_pack_vel(N, vel, mass, Pids, n, c->accrec[1].p, pos, c->rec[1].p, s));
        if (sym) {
            // HHS level lists in Morton order: far source sub-tiles take the 3-addition
            // separation relative to their centre, as in the bipartite cross-level kernel
            const void* frel = nullptr;
            const void* fsub = nullptr;
            if (c->lists_ordered && n >= std::min(kCrossFarMin, order_threshold(c))) {
                CK(ensure(c->xrel, pad_tile(n) * 16));
                CK(ensure(c->xsub, (pad_tile(n) / 32) * 16));
                CU(launch_subtiles(n, c->rec[1].p, c->xrel.p, c->xsub.p, s, true));
                frel = c->xrel.p;
                fsub = c->xsub.p;
            }
            CU(launch_steps_sym(n, c->rec[1].p, c->accrec[1].p, c->p.eps2, c->p.eta_ff, c->p.eta_fb,
                                c->p.eta_jerk, c->stpart.p, step, c->err_d, budget(c), c->sm_count, s,
                                frel, fsub, (kFarKappa + 1.0f) * (kFarKappa + 1.0f)));
        } else
            CU(launch_steps_x2(n, c->rec[1].p, c->accrec[1].p, c->p.eps2, c->p.eta_ff, c->p.eta_fb,
                               c->p.eta_jerk, P<float>(c->stpart), step, c->err_d, budget(c),
                               c->sm_count, wide_limit(c), s, lo, hi - lo));
    }
    else if (sym64) {
        CK(ensure(c->rec[1], pad_tile(n) * 32));
        CK(ensure(c->accrec[1], pad_tile(n) * 32));
        CK(ensure(c->stpart, steps_sym_f64_work_bytes(n)));
        CU(launch_steps_sym_f64(N, pos, vel, mass, Pids, n, c->rec[1].p, c->accrec[1].p, c->p.eps2,
                                c->p.eta_ff, c->p.eta_fb, c->p.eta_jerk, c->stpart.p, step, c->err_d,
                                budget(c), c->sm_count, s));
    } else
        CU(launch_timesteps(n, xc, vc, mc, c->p.eta_ff, c->p.eta_fb, c->p.eta_jerk, c->p.eps2, step,
                            c->err_d, s, lo, hi - lo));
    if (!whole) return crit ? fail(FSI_ERR_UNSUPPORTED, "time steps of a sub-range with the gradient criteria") : FSI_OK;
    if (c->p.eta_grad > 0.0 || c->p.eta_va > 0.0) {
        // gradient and velocity-per-acceleration criteria (Sect. 3.4): a and G of the set
        // from itself, G with the set's own accelerations, then the min into step
        const int prec = c->p.precision;
        CK(ensure(c->rec[0], pad_tile(n) * 32));
        CK(ensure(c->accrec[0], pad_tile(n) * 32));
        CK(ensure(c->tA, 3 * (size_t)n * 8));
        CK(ensure(c->tB, 3 * (size_t)n * 8));
        CU(launch_pack(prec, N, pos, mass, Pids, n, c->rec[0].p, nullptr, s));
        PairArgs a{};
        a.irec = a.jrec = c->rec[0].p;
        a.n_i = a.n_j = n;
        a.check = CHECK_DIAG;
        a.eps2 = c->p.eps2;
        a.epi.out = P<double>(c->tA);
        a.epi.accrec = c->accrec[0].p;
        CK(run_pair(c, KIND_ACC, a, s));
        a.iacc = a.jacc = c->accrec[0].p;
        a.epi = Epi{};
        a.epi.out = P<double>(c->tB);
        CK(run_pair(c, KIND_GRAD, a, s));
        CU(launch_grad_steps(n, vc, P<double>(c->tA), P<double>(c->tB), c->p.eta_grad, c->p.eta_va,
                             step, s));
    }
    return FSI_OK;
}

int hhs_small_cap(const fsi_ctx* c) {
    return c->p.hhs_small_max == 0 ? std::min(kSmallCapDefault, small_max())
                                   : std::min(c->p.hhs_small_max, small_max());
}

// Largest fast set whose HHS recursion runs in one cooperative launch over the GPU; 0 when
// that form is off (hhs_grid_max = -1, or no co-resident grid of 2 CTAs on this device).
int hhs_grid_cap(fsi_ctx* c) {
    if (c->p.hhs_grid_max < 0) return 0;
    const int prec = c->p.precision;
    if (c->grid_nctas[prec] < 0) c->grid_nctas[prec] = grid_ctas(prec, c->sm_count);
    if (c->grid_nctas[prec] < 2) return 0;
    return c->p.hhs_grid_max == 0 ? kGridCapDefault : c->p.hhs_grid_max;
}

// HHS(ids, tau) at `level` in one cooperative launch (hhs_grid.cu); at level 0 the split
// records the level-0 steps.  Statistics go to dstats.
// Workspace of a cooperative HHS launch with a root set of n particles at `level`.
int reserve_hhs_grid(fsi_ctx* c, int N, int n, int level) {
    const int prec = c->p.precision;
    const size_t vb = prec == FSI_MIXED ? 16 : 32;
    CK(ensure(c->grec[0], (size_t)N * 32));
    CK(ensure(c->grec[1], (size_t)N * 32));
    CK(ensure(c->garec, (size_t)N * vb));
    CK(ensure(c->gvrec, (size_t)N * vb));
    CK(ensure(c->gacc, 3 * (size_t)N * 8));
    CK(ensure(c->gaux, 3 * (size_t)N * 8));
    CK(ensure(c->gst, (size_t)N * 8));
    // list stack: the root's copy plus one split per level down to max_level
    const long long cap = (long long)n * std::max(2, c->p.max_level - level + 2);
    if (cap > (1LL << 30)) return fail(FSI_ERR_ARG, "HHS list stack of %lld entries", cap);
    CK(ensure(c->glists, (size_t)cap * 4));
    CK(ensure(c->gbhl, (size_t)cap * 4));
    // PN: one chunk sum per (black hole, kGridPnChunk sources) and direction
    const long long pncap = c->p.c > 0.0 ? 6LL * kMaxBHList * ((n + kGridPnChunk - 1) / kGridPnChunk) : 0;
    if (pncap) CK(ensure(c->gpnpart, (size_t)pncap * 8));
    CK(ensure(c->gbar, 64));
    return FSI_OK;
}

int run_hhs_grid(fsi_ctx* c, int N, double* pos, double* vel, const double* mass,
                 const unsigned char* is_bh, const int* ids, int n, double tau, int level,
                 bool latch_maxlevel, cudaStream_t s) {
    const int prec = c->p.precision;
    CK(reserve_hhs_grid(c, N, n, level));
    const long long cap = (long long)n * std::max(2, c->p.max_level - level + 2);
    const long long pncap = c->p.c > 0.0 ? 6LL * kMaxBHList * ((n + kGridPnChunk - 1) / kGridPnChunk) : 0;
    CU(cudaMemsetAsync(c->gbar.p, 0, 64, s));
    GridArgs g{};
    SmallArgs& sa = g.s;
    sa.ids = ids; sa.n = n; sa.pos = pos; sa.vel = vel; sa.mass = mass;
    sa.step0 = P<double>(c->step0); sa.N = N; sa.tau = tau; sa.level = level;
    sa.max_level = c->p.max_level; sa.eps2 = c->p.eps2; sa.eta_ff = c->p.eta_ff;
    sa.eta_fb = c->p.eta_fb; sa.eta_jerk = c->p.eta_jerk;
    sa.eta_grad = c->p.eta_grad; sa.eta_va = c->p.eta_va;
    unsigned long long* st = P<unsigned long long>(c->dstats);
    sa.level_counts = st; sa.work = st + 64;
    sa.maxlevel_hit = reinterpret_cast<int*>(st + 66);
    sa.err = c->err_d;
    sa.is_bh = is_bh;
    sa.c = c->p.c;
    g.step0w = level == 0 ? P<double>(c->step0) : nullptr;
    g.small_cap = std::max(0, hhs_small_cap(c));
    g.rec[0] = c->grec[0].p; g.rec[1] = c->grec[1].p;
    g.arec = c->garec.p; g.vrec = c->gvrec.p;
    g.acc = P<double>(c->gacc); g.aux = P<double>(c->gaux); g.st = P<double>(c->gst);
    g.lists = P<int>(c->glists); g.list_cap = cap;
    g.bar = P<unsigned long long>(c->gbar);
    g.timeout_ns = budget(c);
    g.latch_maxlevel = latch_maxlevel ? 1 : 0;
    g.bhl = P<int>(c->gbhl);
    g.pnpart = pncap ? P<double>(c->gpnpart) : nullptr;
    g.pnpart_cap = pncap;
    if (c->profiling) {
        if (!c->gprof.p) {
            CK(ensure(c->gprof, 16 * sizeof(unsigned long long)));
            CU(cudaMemsetAsync(c->gprof.p, 0, 16 * sizeof(unsigned long long), s));
        }
        g.prof = P<unsigned long long>(c->gprof);
    }
    const int most = c->grid_nctas[prec];
    const int ctas = c->p.hhs_grid_ctas > 0 ? std::min(most, std::max(2, c->p.hhs_grid_ctas)) : most;
    CU(launch_hhs_grid(prec, g, ctas, s));
    return FSI_OK;
}

int hhs_level(fsi_ctx* c, int N, double* pos, double* vel, const double* mass,
              const unsigned char* is_bh, const int* Pids, int n, double tau, int level,
              cudaStream_t s) {
    if (n <= 0) return FSI_OK;
    if ((int)c->lvS.size() <= level) {
        c->lvS.resize(level + 1);
        c->lvF.resize(level + 1);
    }
    c->max_level_used = std::max(c->max_level_used, level);
    CK(ensure(c->steps, (size_t)n * 8));
    CK(ensure(c->lvS[level], (size_t)n * 4));
    CK(ensure(c->lvF[level], (size_t)n * 4));
    CK(timesteps_core(c, N, pos, vel, mass, Pids, n, P<double>(c->steps), s));
    const int force_slow = level >= c->p.max_level;
    int* Sids = P<int>(c->lvS[level]);
    int* Fids = P<int>(c->lvF[level]);
    // level-step rule (record at level 0, min deeper down) fused into the partition
    CU(launch_partition(n, Pids, P<double>(c->steps), P<double>(c->step0), level == 0, tau, force_slow,
                        Sids, Fids, P<int>(c->counts), s));
    CU(cudaMemcpyAsync(c->counts_h, c->counts.p, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const int nS = c->counts_h[0], nF = c->counts_h[1];
    if (c->counts_h[2]) c->max_level_hit = 1;
    if ((int)c->level_counts.size() <= level) c->level_counts.resize(level + 1, 0);
    c->level_counts[level] += nS;
    const bool cross = nS > 0 && nF > 0;
    const bool pn = c->p.c > 0.0;
    if (cross) {
        if (pn) CK(cross_pn_kick(c, N, pos, vel, mass, is_bh, Sids, nS, Fids, nF, 0.5 * tau, s));
        CK(cross_kick(c, N, pos, vel, mass, Sids, nS, Fids, nF, tau / 6.0, 0, 0.0, s));
    }
    // HHS(F, tau/2): small fast sets recurse inside one CTA, mid-size ones in one
    // cooperative launch over the GPU, larger ones level by level here
    const int small_cap = hhs_small_cap(c);
    const int grid_cap = hhs_grid_cap(c);
    auto recurse = [&]() -> int {
        if (nF <= 0) return FSI_OK;
        if (nF <= small_cap) {
            SmallArgs sa{};
            sa.ids = Fids; sa.n = nF; sa.pos = pos; sa.vel = vel; sa.mass = mass;
            sa.step0 = P<double>(c->step0); sa.N = N; sa.tau = 0.5 * tau; sa.level = level + 1;
            sa.max_level = c->p.max_level; sa.eps2 = c->p.eps2; sa.eta_ff = c->p.eta_ff;
            sa.eta_fb = c->p.eta_fb; sa.eta_jerk = c->p.eta_jerk;
            sa.eta_grad = c->p.eta_grad; sa.eta_va = c->p.eta_va;
            unsigned long long* st = P<unsigned long long>(c->dstats);
            sa.level_counts = st; sa.work = st + 64;
            sa.maxlevel_hit = reinterpret_cast<int*>(st + 66);
            sa.err = c->err_d;
            sa.is_bh = is_bh;
            sa.c = c->p.c;
            CU(launch_hhs_small(c->p.precision, sa, s));
            return FSI_OK;
        }
        if (nF <= grid_cap)
            return run_hhs_grid(c, N, pos, vel, mass, is_bh, Fids, nF, 0.5 * tau, level + 1, false, s);
        return hhs_level(c, N, pos, vel, mass, is_bh, Fids, nF, 0.5 * tau, level + 1, s);
    };
    if (nS > 0) CK(step_core(c, N, pos, vel, mass, is_bh, Sids, nS, 0.5 * tau, 1, s));
    CK(recurse());
    if (cross) CK(cross_kick(c, N, pos, vel, mass, Sids, nS, Fids, nF, 2.0 * tau / 3.0, 1, tau, s));
    CK(recurse());
    if (nS > 0) CK(step_core(c, N, pos, vel, mass, is_bh, Sids, nS, 0.5 * tau, 1, s));
    if (cross) {
        CK(cross_kick(c, N, pos, vel, mass, Sids, nS, Fids, nF, tau / 6.0, 0, 0.0, s));
        if (pn) CK(cross_pn_kick(c, N, pos, vel, mass, is_bh, Sids, nS, Fids, nF, 0.5 * tau, s));
    }
    return FSI_OK;
}

}  // namespace

// A batch plan: per-variant work-item tables and the records of the concatenated set.
struct fsi_batch {
    int K = 0;
    long long ntot = 0;
    int max_steps = 0;
    int ipt = 1;
    int ctas_per_sm = 2;
    int stall_cluster = -1;          // test hook (fsi_batch_inject_stall)
    // per particles-per-thread variant (index 1, 2: one-sided; kBatchSymI, kBatchSymI2:
    // symmetric)
    std::vector<int> nblocks_h[kBatchSymI2 + 1];
    Buf items[kBatchSymI2 + 1], nblocks[kBatchSymI2 + 1];
    int items_per_phase[kBatchSymI2 + 1] = {};
    // symmetric form, per variant (index ipt): sum items, sum items per cluster
    Buf sitems[kBatchSymI2 + 1], nsum[kBatchSymI2 + 1];
    int sitems_per_phase[kBatchSymI2 + 1] = {};
    Buf accum;
    Buf rec0, rec1, accrec, ac, done, ctrl;
    Buf stats;                       // idle accounting: wait ns, CTA lifetime ns
    int last_ctas = 0;
    std::vector<long long> off;
};

int fsi::set_last_error(int code, const char* msg) { return fail(code, "%s", msg); }

// =================================================================================
extern "C" {

void fsi_default_params(fsi_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->precision = FSI_FP64;
    p->eps2 = 0.0;
    p->eta_ff = 0.2;
    p->eta_fb = 0.2;
    p->eta_jerk = 0.1;
    p->max_level = 40;
    p->c = 0.0;
    p->split = 0;
    p->timeout_ns = 0;
    p->symmetric = 1;
    p->hhs_small_max = 0;
    p->order_min = 0;
    p->eta_grad = 0.0;
    p->eta_va = 0.0;
    p->wide_ctas = 0;
    p->hhs_grid_max = 0;
    p->hhs_grid_ctas = 0;
}

const char* fsi_last_error(void) { return g_err.c_str(); }

int fsi_create(fsi_ctx** out, const fsi_params* p) {
    if (!out) return fail(FSI_ERR_ARG, "NULL output handle");
    *out = nullptr;
    fsi_params q;
    if (p) q = *p;
    else fsi_default_params(&q);
    if (!valid_prec(q.precision)) return fail(FSI_ERR_ARG, "unknown precision %d", q.precision);
    if (!(q.eta_grad >= 0.0) || !(q.eta_va >= 0.0))
        return fail(FSI_ERR_ARG, "eta_grad and eta_va must be >= 0 (0 = off)");
    fsi_ctx* c = new fsi_ctx();
    c->p = q;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess ||
        cudaMalloc(&c->err_d, sizeof(int)) != cudaSuccess ||
        cudaMemset(c->err_d, 0, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&c->err_h, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&c->counts_h, 4 * sizeof(int)) != cudaSuccess) {
        const char* msg = cudaGetErrorString(cudaGetLastError());
        delete c;
        return fail(FSI_ERR_CUDA, "context creation failed: %s", msg);
    }
    *out = c;
    return FSI_OK;
}

int fsi_destroy(fsi_ctx* c) {
    if (!c) return FSI_OK;
    cudaDeviceSynchronize();
    Buf* bufs[] = {&c->rec[0], &c->rec[1], &c->accrec[0], &c->accrec[1], &c->xc, &c->vc, &c->ac,
                   &c->ad, &c->tA, &c->tB, &c->mc, &c->bhc, &c->ids[0], &c->ids[1],
                   &c->part, &c->mark, &c->bhlist, &c->nbh, &c->apn, &c->pnpart, &c->epart,
                   &c->iota, &c->steps, &c->step0, &c->counts, &c->accum, &c->dstats,
                   &c->rel, &c->sub, &c->ordws, &c->ordperm, &c->ordlist, &c->farstats,
                   &c->eout, &c->snapx, &c->snapv, &c->subwhere, &c->subkey, &c->subppos, &c->stpart,
                   &c->xrel, &c->xsub, &c->pnids, &c->grec[0], &c->grec[1], &c->garec,
                   &c->gvrec, &c->gacc, &c->gaux, &c->gst, &c->glists, &c->gbar, &c->gprof, &c->gbhl,
                   &c->gpnpart};
    for (Buf* b : bufs)
        if (b->p) cudaFree(b->p);
    for (auto& r : c->prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    for (auto& b : c->vj) if (b.p) cudaFree(b.p);
    for (auto& b : c->lvS) if (b.p) cudaFree(b.p);
    for (auto& b : c->lvF) if (b.p) cudaFree(b.p);
    if (c->err_d) cudaFree(c->err_d);
    if (c->err_h) cudaFreeHost(c->err_h);
    if (c->counts_h) cudaFreeHost(c->counts_h);
    delete c;
    return FSI_OK;
}

int fsi_set_params(fsi_ctx* c, const fsi_params* p) {
    if (!c || !p) return fail(FSI_ERR_ARG, "NULL argument");
    if (!valid_prec(p->precision)) return fail(FSI_ERR_ARG, "unknown precision %d", p->precision);
    if (!(p->eta_grad >= 0.0) || !(p->eta_va >= 0.0))
        return fail(FSI_ERR_ARG, "eta_grad and eta_va must be >= 0 (0 = off)");
    c->p = *p;
    return FSI_OK;
}

int fsi_reserve(fsi_ctx* c, int N, int n) {
    CK(check_common(c, N));
    if (n < 0 || n > N) return fail(FSI_ERR_ARG, "bad set size %d", n);
    const size_t pt = pad_tile(n) * 32;
    for (int k = 0; k < 2; ++k) {
        CK(ensure(c->rec[k], pt));
        CK(ensure(c->accrec[k], pt));
        CK(ensure(c->ids[k], pad_tile(n) * 4));
    }
    Buf* b3[] = {&c->xc, &c->vc, &c->ac, &c->ad, &c->tA, &c->tB, &c->apn};
    for (Buf* b : b3) CK(ensure(*b, 3 * (size_t)n * 8));
    CK(ensure(c->mc, (size_t)n * 8));
    CK(ensure(c->bhc, (size_t)n));
    CK(ensure(c->bhlist, 2 * kMaxBHList * 4));
    CK(ensure(c->nbh, 16));
    CK(ensure(c->pnpart, (size_t)kMaxBHList * 3 * kPnPartCtas * 8));
    CK(ensure(c->part, (size_t)64 * 3 * n * 8));
    CK(ensure(c->epart, (size_t)(energy_blocks(n) * 2 + 2) * 8));
    CK(ensure(c->accum, 3 * (size_t)n * 8));      // also both sides of a bipartite pass
    CK(ensure(c->stpart, std::max({steps_x2_part_bytes(n, c->sm_count), steps_sym_work_bytes(n),
                                   steps_sym_f64_work_bytes(n)})));
    // spatial ordering and far-tile inputs of the symmetric mixed kernel
    CK(ensure(c->rel, pad_tile(n) * 16));
    CK(ensure(c->sub, (pad_tile(n) / 32) * 16));
    CK(ensure(c->ordperm, (size_t)n * 4));
    CK(ensure(c->ordlist, (size_t)n * 4));
    CK(ensure(c->ordws, morton_workspace_bytes(n)));
    if (!c->farstats.p) {
        CK(ensure(c->farstats, 2 * sizeof(unsigned long long)));
        CU(cudaMemset(c->farstats.p, 0, 2 * sizeof(unsigned long long)));
    }
    if (n == N) {
        // an HHS interval of all N: its level-0 lists and statistics, and the cooperative
        // launch's workspace for the largest set it may take (the interval itself when
        // N <= hhs_grid_max, else a fast set of at most hhs_grid_max one level down)
        CK(ensure(c->iota, (size_t)N * 4));
        CK(ensure(c->step0, (size_t)N * 8));
        CK(ensure(c->counts, 16));
        CK(ensure(c->dstats, 68 * sizeof(unsigned long long)));
        const int gcap = hhs_grid_cap(c);
        if (gcap > 0) CK(reserve_hhs_grid(c, N, std::min(N, gcap), 0));
    }
    CU(cudaDeviceSynchronize());
    return FSI_OK;
}

int fsi_sync_status(fsi_ctx* c, void* stream) {
    if (!c) return fail(FSI_ERR_ARG, "NULL context");
    CU(cudaStreamSynchronize(S(stream)));
    CU(cudaMemcpy(c->err_h, c->err_d, sizeof(int), cudaMemcpyDeviceToHost));
    CU(cudaMemset(c->err_d, 0, sizeof(int)));
    const int e = *c->err_h;
    if (e != FSI_OK) fail(e, "device reported status %d", e);
    return e;
}

int fsi_accel(fsi_ctx* c, int N, const double* pos, const double* mass, const int* A, int nA,
              const int* B, int nB, double eps2, double* acc_out, void* stream) {
    CK(check_common(c, N));
    if (nA == 0) return FSI_OK;
    if (nA < 0 || nB < 0 || (!A && nA != N) || (!B && nB != N))
        return fail(FSI_ERR_ARG, "bad set sizes nA=%d nB=%d N=%d", nA, nB, N);
    if (!pos || !mass || !acc_out) return fail(FSI_ERR_ARG, "NULL array");
    const cudaStream_t s = S(stream);
    const int prec = c->p.precision;
    const bool same = (A == B) && (nA == nB);
    CK(ensure(c->rec[0], pad_tile(nA) * 32));
    FarGuard far_guard{c};
    SameSetOrder ord;
    if (same) CK(ord.begin(c, N, pos, mass, A, nA, s));
    if (ord.on) CK(ensure(c->tA, 3 * (size_t)nA * 8));
    CU(launch_pack(prec, N, pos, mass, ord.on ? ord.list : A, nA, c->rec[0].p, nullptr, s));
    PairArgs a{};
    a.irec = c->rec[0].p;
    a.n_i = nA;
    a.n_j = nB;
    a.eps2 = eps2;
    a.epi.out = ord.on ? P<double>(c->tA) : acc_out;
    if (same) {
        a.jrec = c->rec[0].p;
        a.check = CHECK_DIAG;
        CK(run_pair(c, KIND_ACC, a, s));
        return ord.on ? ord.unsort(c, P<double>(c->tA), nA, acc_out, s) : FSI_OK;
    } else if (const long long off = sub_range(A, nA, B, nB); off >= 0) {
        // A is the sub-range B[off, off + nA) of the source list (a rank's slice of a
        // sharded pass): one packing of B, self pairs by index offset
        CK(ensure(c->rec[1], pad_tile(nB) * 32));
        CU(launch_pack(prec, N, pos, mass, B, nB, c->rec[1].p, nullptr, s));
        a.jrec = c->rec[1].p;
        a.irec = static_cast<const unsigned char*>(c->rec[1].p) + off * 32;
        a.check = CHECK_DIAG;
        a.i_off = (int)off;
    } else {
        CK(ensure(c->rec[1], pad_tile(nB) * 32));
        CK(ensure(c->ids[0], pad_tile(nA) * 4));
        CK(ensure(c->ids[1], pad_tile(nB) * 4));
        CU(launch_pack(prec, N, pos, mass, B, nB, c->rec[1].p, nullptr, s));
        CU(launch_ids(A, nA, (int)pad_tile(nA), P<int>(c->ids[0]), s));
        CU(launch_ids(B, nB, (int)pad_tile(nB), P<int>(c->ids[1]), s));
        a.jrec = c->rec[1].p;
        a.check = CHECK_IDS;
        a.iid = P<int>(c->ids[0]);
        a.jid = P<int>(c->ids[1]);
    }
    return run_pair(c, KIND_ACC, a, s);
}

int fsi_grad(fsi_ctx* c, int N, const double* pos, const double* mass, const double* accg,
             const int* A, int nA, const int* B, int nB, double eps2, double* grad_out,
             void* stream) {
    CK(check_common(c, N));
    if (nA == 0) return FSI_OK;
    if (nA < 0 || nB < 0 || (!A && nA != N) || (!B && nB != N))
        return fail(FSI_ERR_ARG, "bad set sizes nA=%d nB=%d N=%d", nA, nB, N);
    if (!pos || !mass || !accg || !grad_out) return fail(FSI_ERR_ARG, "NULL array");
    const cudaStream_t s = S(stream);
    const int prec = c->p.precision;
    const bool same = (A == B) && (nA == nB);
    CK(ensure(c->rec[0], pad_tile(nA) * 32));
    CK(ensure(c->accrec[0], pad_tile(nA) * 32));
    FarGuard far_guard{c};
    SameSetOrder ord;
    if (same) CK(ord.begin(c, N, pos, mass, A, nA, s));
    if (ord.on) CK(ensure(c->tA, 3 * (size_t)nA * 8));
    CU(launch_pack(prec, N, pos, mass, ord.on ? ord.list : A, nA, c->rec[0].p, nullptr, s));
    CU(launch_pack_acc(prec, N, accg, mass, ord.on ? ord.list : A, nA, c->accrec[0].p, nullptr, s));
    PairArgs a{};
    a.irec = c->rec[0].p;
    a.iacc = c->accrec[0].p;
    a.n_i = nA;
    a.n_j = nB;
    a.eps2 = eps2;
    a.epi.out = ord.on ? P<double>(c->tA) : grad_out;
    if (same) {
        a.jrec = a.irec;
        a.jacc = a.iacc;
        a.check = CHECK_DIAG;
        CK(run_pair(c, KIND_GRAD, a, s));
        return ord.on ? ord.unsort(c, P<double>(c->tA), nA, grad_out, s) : FSI_OK;
    } else if (const long long off = sub_range(A, nA, B, nB); off >= 0) {
        // A is the sub-range B[off, off + nA) of the source list: one packing of B
        CK(ensure(c->rec[1], pad_tile(nB) * 32));
        CK(ensure(c->accrec[1], pad_tile(nB) * 32));
        CU(launch_pack(prec, N, pos, mass, B, nB, c->rec[1].p, nullptr, s));
        CU(launch_pack_acc(prec, N, accg, mass, B, nB, c->accrec[1].p, nullptr, s));
        const size_t accb = prec == FSI_MIXED ? 16 : 32;
        a.jrec = c->rec[1].p;
        a.jacc = c->accrec[1].p;
        a.irec = static_cast<const unsigned char*>(c->rec[1].p) + off * 32;
        a.iacc = static_cast<const unsigned char*>(c->accrec[1].p) + off * accb;
        a.check = CHECK_DIAG;
        a.i_off = (int)off;
    } else {
        CK(ensure(c->rec[1], pad_tile(nB) * 32));
        CK(ensure(c->accrec[1], pad_tile(nB) * 32));
        CK(ensure(c->ids[0], pad_tile(nA) * 4));
        CK(ensure(c->ids[1], pad_tile(nB) * 4));
        CU(launch_pack(prec, N, pos, mass, B, nB, c->rec[1].p, nullptr, s));
        CU(launch_pack_acc(prec, N, accg, mass, B, nB, c->accrec[1].p, nullptr, s));
        CU(launch_ids(A, nA, (int)pad_tile(nA), P<int>(c->ids[0]), s));
        CU(launch_ids(B, nB, (int)pad_tile(nB), P<int>(c->ids[1]), s));
        a.jrec = c->rec[1].p;
        a.jacc = c->accrec[1].p;
        a.check = CHECK_IDS;
        a.iid = P<int>(c->ids[0]);
        a.jid = P<int>(c->ids[1]);
    }
    return run_pair(c, KIND_GRAD, a, s);
}

int fsi_accel_part(fsi_ctx* c, int N, const double* pos, const double* mass, const int* A,
                   int nA, int part, int nparts, double eps2, double* acc_out, void* stream) {
    CK(check_common(c, N));
    if (nA == 0) return FSI_OK;
    if (nA < 0 || (!A && nA != N)) return fail(FSI_ERR_ARG, "bad set size nA=%d N=%d", nA, N);
    if (!pos || !mass || !acc_out) return fail(FSI_ERR_ARG, "NULL array");
    return run_share(c, KIND_ACC, nA, part, nparts, acc_out, S(stream), [&] {
        return fsi_accel(c, N, pos, mass, A, nA, A, nA, eps2, acc_out, stream);
    });
}

int fsi_grad_part(fsi_ctx* c, int N, const double* pos, const double* mass, const double* accg,
                  const int* A, int nA, int part, int nparts, double eps2, double* grad_out,
                  void* stream) {
    CK(check_common(c, N));
    if (nA == 0) return FSI_OK;
    if (nA < 0 || (!A && nA != N)) return fail(FSI_ERR_ARG, "bad set size nA=%d N=%d", nA, N);
    if (!pos || !mass || !accg || !grad_out) return fail(FSI_ERR_ARG, "NULL array");
    return run_share(c, KIND_GRAD, nA, part, nparts, grad_out, S(stream), [&] {
        return fsi_grad(c, N, pos, mass, accg, A, nA, A, nA, eps2, grad_out, stream);
    });
}

int fsi_accel_grad(fsi_ctx* c, int N, const double* pos, const double* vel, const double* mass,
                   const int* A, int nA, const int* B, int nB, double eps2, double* acc_out,
                   double* grad_out, void* stream) {
    (void)vel;
    CK(check_common(c, N));
    if (nA == 0) return FSI_OK;
    if (nA < 0 || nB < 0 || (!A && nA != N) || (!B && nB != N))
        return fail(FSI_ERR_ARG, "bad set sizes nA=%d nB=%d N=%d", nA, nB, N);
    if (!pos || !mass || !acc_out || !grad_out) return fail(FSI_ERR_ARG, "NULL array");
    const cudaStream_t s = S(stream);
    const int prec = c->p.precision;
    const bool same = (A == B) && (nA == nB);
    CK(ensure(c->rec[0], pad_tile(nA) * 32));
    CK(ensure(c->accrec[0], pad_tile(nA) * 32));
    FarGuard far_guard{c};
    SameSetOrder ord;
    if (same) CK(ord.begin(c, N, pos, mass, A, nA, s));
    CU(launch_pack(prec, N, pos, mass, ord.on ? ord.list : A, nA, c->rec[0].p, nullptr, s));
    if (same) {
        if (ord.on) {
            CK(ensure(c->tA, 3 * (size_t)nA * 8));
            CK(ensure(c->tB, 3 * (size_t)nA * 8));
        }
        PairArgs a{};
        a.irec = a.jrec = c->rec[0].p;
        a.n_i = a.n_j = nA;
        a.check = CHECK_DIAG;
        a.eps2 = eps2;
        a.epi.out = ord.on ? P<double>(c->tA) : acc_out;
        a.epi.accrec = c->accrec[0].p;
        CK(run_pair(c, KIND_ACC, a, s));
        a.iacc = a.jacc = c->accrec[0].p;
        a.epi = Epi{};
        a.epi.out = ord.on ? P<double>(c->tB) : grad_out;
        CK(run_pair(c, KIND_GRAD, a, s));
        if (!ord.on) return FSI_OK;
        CK(ord.unsort(c, P<double>(c->tA), nA, acc_out, s));
        return ord.unsort(c, P<double>(c->tB), nA, grad_out, s);
    }
    if (!A || !B) return fail(FSI_ERR_ARG, "a NULL (all-particle) list overlaps any other list");
    CK(ensure(c->mark, (size_t)N));
    CU(cudaMemsetAsync(c->mark.p, 0, (size_t)N, s));
    CU(launch_check_disjoint(N, A, nA, B, nB, P<unsigned char>(c->mark), c->err_d, s));
    CK(ensure(c->rec[1], pad_tile(nB) * 32));
    CK(ensure(c->accrec[1], pad_tile(nB) * 32));
    CU(launch_pack(prec, N, pos, mass, B, nB, c->rec[1].p, nullptr, s));
    PairArgs a{};
    a.check = CHECK_NONE;
    a.eps2 = eps2;
    a.irec = c->rec[0].p; a.jrec = c->rec[1].p; a.n_i = nA; a.n_j = nB;
    a.epi.out = acc_out;
    a.epi.accrec = c->accrec[0].p;
    CK(run_pair(c, KIND_ACC, a, s));
    PairArgs b{};
    b.check = CHECK_NONE;
    b.eps2 = eps2;
    b.irec = c->rec[1].p; b.jrec = c->rec[0].p; b.n_i = nB; b.n_j = nA;
    b.epi.accrec = c->accrec[1].p;
    CK(run_pair(c, KIND_ACC, b, s));
    a.iacc = c->accrec[0].p;
    a.jacc = c->accrec[1].p;
    a.epi = Epi{};
    a.epi.out = grad_out;
    return run_pair(c, KIND_GRAD, a, s);
}

int fsi_pn_accel(fsi_ctx* c, int N, const double* pos, const double* vel, const double* mass,
                 const unsigned char* is_bh, double cl, const int* A, int nA, const int* B, int nB,
                 double* out, void* stream) {
    CK(check_common(c, N));
    if (nA < 0 || nB < 0 || (!A && nA != N) || (!B && nB != N))
        return fail(FSI_ERR_ARG, "bad set sizes nA=%d nB=%d N=%d", nA, nB, N);
    if (!(cl > 0.0)) return fail(FSI_ERR_ARG, "speed of light must be positive");
    if (nA == 0) return FSI_OK;
    if (!pos || !vel || !mass || !is_bh || !out) return fail(FSI_ERR_ARG, "NULL array");
    // the pairs with a black hole through black-hole sublists of both lists (a NULL list
    // becomes the ids 0 .. N-1): O((nA + nB) x black holes) instead of O(nA nB)
    const cudaStream_t s = S(stream);
    const int* Al = A;
    const int* Bl = B;
    if (!A || !B) {
        CK(ensure(c->pnids, (size_t)N * sizeof(int)));
        CU(launch_iota(N, P<int>(c->pnids), s));
        if (!A) Al = P<int>(c->pnids);
        if (!B) Bl = P<int>(c->pnids);
    }
    CK(ensure(c->bhlist, 2 * kMaxBHList * 4));
    CK(ensure(c->nbh, 16));
    CK(ensure(c->pnpart, (size_t)kMaxBHList * 3 * kPnPartCtas * 8));
    int* bl = P<int>(c->bhlist);
    int* nb = P<int>(c->nbh);
    CU(launch_pn_lists(N, pos, vel, mass, is_bh, cl, Al, nA, Bl, nB, bl, nb, bl + kMaxBHList, nb + 1,
                       out, P<double>(c->pnpart), c->err_d, s));
    return FSI_OK;
}

int fsi_step(fsi_ctx* c, int N, double* pos, double* vel, const double* mass,
             const unsigned char* is_bh, const int* idx, int n, double h, int nsteps,
             void* stream) {
    CK(check_common(c, N));
    if (n < 0 || (!idx && n != N)) return fail(FSI_ERR_ARG, "bad set size n=%d N=%d", n, N);
    if (nsteps < 0) return fail(FSI_ERR_ARG, "nsteps must be >= 0");
    if (n == 0 || nsteps == 0) return FSI_OK;
    if (!pos || !vel || !mass) return fail(FSI_ERR_ARG, "NULL array");
    return step_core(c, N, pos, vel, mass, is_bh, idx, n, h, nsteps, S(stream));
}

int fsi_kick_drift(fsi_ctx* c, int N, double* pos, double* vel, const double* acc,
                   const int* idx, int n, double c_kick, double c_drift, void* stream) {
    CK(check_common(c, N));
    if (n < 0 || (!idx && n > N)) return fail(FSI_ERR_ARG, "bad set size n=%d N=%d", n, N);
    if (n == 0) return FSI_OK;
    if (!pos || !vel) return fail(FSI_ERR_ARG, "NULL array");
    CU(launch_kick_drift_ids(N, pos, vel, acc, idx, n, c_kick, c_drift, c->sm_count, S(stream)));
    return FSI_OK;
}

int fsi_step_record(fsi_ctx* c, int N, double* pos, double* vel, const double* mass,
                    const int* idx, int n, double h, double* a0, double* a1, double* g1,
                    void* stream) {
    CK(check_common(c, N));
    if (n < 0 || (!idx && n != N)) return fail(FSI_ERR_ARG, "bad set size n=%d N=%d", n, N);
    if (c->p.c > 0.0) return fail(FSI_ERR_UNSUPPORTED, "the recorded cycle is Newtonian (PN off)");
    if (n == 0) return FSI_OK;
    if (!pos || !vel || !mass || !a0 || !a1 || !g1) return fail(FSI_ERR_ARG, "NULL array");
    const StepRecord r{a0, a1, g1};
    return step_core(c, N, pos, vel, mass, nullptr, idx, n, h, 1, S(stream), &r);
}

int fsi_step_sub(fsi_ctx* c, int N, double* pos, double* vel, const double* mass,
                 const int* idx, int n, const int* pairs, int n_pairs, double h, int nsteps,
                 void* stream) {
    CK(check_common(c, N));
    if (!pos || !vel || !mass) return fail(FSI_ERR_ARG, "NULL array");
    if (n < 0 || (!idx && n != N)) return fail(FSI_ERR_ARG, "bad set size n=%d N=%d", n, N);
    if (n_pairs < 0 || (n_pairs > 0 && !pairs) || 2LL * n_pairs > n)
        return fail(FSI_ERR_ARG, "bad binary list (%d pairs for %d particles)", n_pairs, n);
    if (nsteps < 0) return fail(FSI_ERR_ARG, "nsteps must be >= 0");
    if (c->p.c > 0.0) return fail(FSI_ERR_UNSUPPORTED, "subsystem steps are Newtonian (PN off)");
    if (n == 0 || nsteps == 0) return FSI_OK;
    if ((long long)N + n_pairs > INT_MAX) return fail(FSI_ERR_ARG, "N + n_pairs overflows the keys");
    const cudaStream_t s = S(stream);
    const int prec = c->p.precision;
    CK(ensure(c->rec[0], pad_tile(n) * 32));
    CK(ensure(c->accrec[0], pad_tile(n) * 32));
    CK(ensure(c->ac, 3 * (size_t)n * 8));
    CK(ensure(c->subwhere, (size_t)N * 4));
    CK(ensure(c->subkey, (size_t)((n + 3) & ~3) * 4));
    CK(ensure(c->subppos, (size_t)std::max(1, 2 * n_pairs) * 4));
    int* key = P<int>(c->subkey);
    int* ppos = P<int>(c->subppos);
    CU(launch_sub_keys(n, idx, N, pairs, n_pairs, P<int>(c->subwhere), key, ppos, c->err_d, s));
    double* xc = pos;
    double* vc = vel;
    const double* mc = mass;
    if (idx) {
        CK(ensure(c->xc, 3 * (size_t)n * 8));
        CK(ensure(c->vc, 3 * (size_t)n * 8));
        CK(ensure(c->mc, (size_t)n * 8));
        xc = P<double>(c->xc);
        vc = P<double>(c->vc);
        CU(launch_gather3(N, pos, idx, n, xc, s));
        CU(launch_gather3(N, vel, idx, n, vc, s));
        CU(launch_gather1(N, mass, idx, n, P<double>(c->mc), s));
        mc = P<double>(c->mc);
    }
    // a masked pass over the set: sources whose key equals the receiver's add nothing
    auto pass = [&](int kind, double ck, double cg) -> int {
        PairArgs a{};
        a.irec = a.jrec = c->rec[0].p;
        a.n_i = a.n_j = n;
        a.check = CHECK_IDS;
        a.iid = a.jid = key;
        a.eps2 = c->p.eps2;
        a.epi.mc = mc;
        if (kind == KIND_ACC) {
            a.epi.out = P<double>(c->ac);
            a.epi.accrec = c->accrec[0].p;
        } else {
            a.iacc = a.jacc = c->accrec[0].p;
            a.epi.base = P<double>(c->ac);
            a.epi.c_grad = cg;
        }
        if (ck != 0.0) {
            a.epi.v = vc;
            a.epi.c_kick = ck;
        }
        return run_pair(c, kind, a, s);
    };
    // subsystems for t, then the single particles drift t; records repacked
    auto flow = [&](double t) -> int {
        CU(launch_kepler_pairs(n_pairs, ppos, n, xc, vc, mc, t, c->err_d, s));
        CU(launch_drift_singles(n, xc, vc, key, N, t, s));
        CU(launch_pack(prec, n, xc, mc, nullptr, n, c->rec[0].p, nullptr, s));
        return FSI_OK;
    };
    CU(launch_pack(prec, n, xc, mc, nullptr, n, c->rec[0].p, nullptr, s));
    for (int k = 0; k < nsteps; ++k) {
        // Algorithm 1: kick eps/6, H_S + drift eps/2, gradient kick 2 eps/3, H_S + drift
        // eps/2, kick eps/6; all accelerations without intra-subsystem pairs
        CK(pass(KIND_ACC, h / 6.0, 0.0));
        CK(flow(0.5 * h));
        CK(pass(KIND_ACC, 0.0, 0.0));
        CK(pass(KIND_GRAD, 2.0 * h / 3.0, h * h / 24.0));
        CK(flow(0.5 * h));
        CK(pass(KIND_ACC, h / 6.0, 0.0));
    }
    if (idx) {
        CU(launch_scatter3(N, xc, idx, n, pos, s));
        CU(launch_scatter3(N, vc, idx, n, vel, s));
    }
    return FSI_OK;
}

int fsi_timesteps(fsi_ctx* c, int N, const double* pos, const double* vel, const double* mass,
                  const int* Pids, int n, double* step_out, void* stream) {
    CK(check_common(c, N));
    if (n < 0 || (!Pids && n != N)) return fail(FSI_ERR_ARG, "bad set size n=%d N=%d", n, N);
    if (n == 0) return FSI_OK;
    if (!pos || !vel || !mass || !step_out) return fail(FSI_ERR_ARG, "NULL array");
    return timesteps_core(c, N, pos, vel, mass, Pids, n, step_out, S(stream));
}

int fsi_timesteps_sub(fsi_ctx* c, int N, const double* pos, const double* vel, const double* mass,
                      const int* Pids, int n, int lo, int hi, double* step_out, void* stream) {
    CK(check_common(c, N));
    if (n < 0 || (!Pids && n != N)) return fail(FSI_ERR_ARG, "bad set size n=%d N=%d", n, N);
    if (lo < 0 || hi < lo || hi > n) return fail(FSI_ERR_ARG, "bad range [%d, %d) of %d", lo, hi, n);
    if (c->p.eta_grad > 0.0 || c->p.eta_va > 0.0)
        return fail(FSI_ERR_UNSUPPORTED, "time steps of a sub-range with the gradient criteria");
    if (hi == lo) return FSI_OK;
    if (!pos || !vel || !mass || !step_out) return fail(FSI_ERR_ARG, "NULL array");
    return timesteps_core(c, N, pos, vel, mass, Pids, n, step_out, S(stream), lo, hi);
}

int fsi_energy(fsi_ctx* c, int N, const double* pos, const double* vel, const double* mass,
               const int* Pids, int n, double* out, void* stream) {
    CK(check_common(c, N));
    if (n < 0 || (!Pids && n != N)) return fail(FSI_ERR_ARG, "bad set size n=%d N=%d", n, N);
    if (!pos || !vel || !mass || !out) return fail(FSI_ERR_ARG, "NULL array");
    const cudaStream_t s = S(stream);
    if (n == 0) {
        CU(cudaMemsetAsync(out, 0, 2 * sizeof(double), s));
        return FSI_OK;
    }
    const double* xc = pos;
    const double* vc = vel;
    const double* mc = mass;
    if (Pids) {
        CK(ensure(c->xc, 3 * (size_t)n * 8));
        CK(ensure(c->vc, 3 * (size_t)n * 8));
        CK(ensure(c->mc, (size_t)n * 8));
        CU(launch_gather3(N, pos, Pids, n, P<double>(c->xc), s));
        CU(launch_gather3(N, vel, Pids, n, P<double>(c->vc), s));
        CU(launch_gather1(N, mass, Pids, n, P<double>(c->mc), s));
        xc = P<double>(c->xc);
        vc = P<double>(c->vc);
        mc = P<double>(c->mc);
    }
    CK(ensure(c->epart, (size_t)(energy_blocks(n) * 2 + 2) * 8));
    CU(launch_energy(n, xc, vc, mc, c->p.eps2, P<double>(c->epart), out, c->err_d, s));
    return FSI_OK;
}

}  // extern "C"

namespace {

// Adds the statistics of the levels run on the device (one-CTA and grid-wide recursions)
// to the host-walked ones (synchronous); FSI_OK or FSI_ERR_MAXLEVEL.
int merge_hhs_stats(fsi_ctx* c, cudaStream_t s) {
    unsigned long long st[68];
    CU(cudaMemcpyAsync(st, c->dstats.p, sizeof st, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    for (int k = 0; k < 64; ++k) {
        c->level_counts[k] += (long long)st[k];
        if (c->level_counts[k]) c->max_level_used = std::max(c->max_level_used, k);
    }
    c->work_pairs[0] += (long long)st[64];
    c->work_pairs[1] += (long long)st[65];
    if (reinterpret_cast<int*>(st + 66)[0]) c->max_level_hit = 1;
    return c->max_level_hit ? FSI_ERR_MAXLEVEL : FSI_OK;
}

// One HHS interval (arguments checked by the caller); FSI_OK or FSI_ERR_MAXLEVEL.  Under
// stream capture (N <= the grid cap only) the statistics stay on the device.
int hhs_interval_core(fsi_ctx* c, int N, double* pos, double* vel, const double* mass,
                      const unsigned char* is_bh, double tau, cudaStream_t s) {
    CK(ensure(c->iota, (size_t)N * 4));
    CK(ensure(c->step0, (size_t)N * 8));
    CK(ensure(c->counts, 16));
    CK(ensure(c->dstats, 68 * sizeof(unsigned long long)));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(s, &cs));
    const bool capturing = cs != cudaStreamCaptureStatusNone;
    c->level_counts.assign(std::max(c->p.max_level + 1, 64), 0);
    c->max_level_used = 0;
    c->max_level_hit = 0;
    c->stats_on_device = false;
    if (N <= hhs_grid_cap(c)) {
        // the whole interval in one cooperative launch: no host synchronisation
        CU(launch_iota(N, P<int>(c->iota), s));
        CU(cudaMemsetAsync(c->dstats.p, 0, 68 * sizeof(unsigned long long), s));
        CK(run_hhs_grid(c, N, pos, vel, mass, is_bh, P<int>(c->iota), N, tau, 0, capturing, s));
        if (capturing) {
            c->stats_on_device = true;
            return FSI_OK;
        }
        return merge_hhs_stats(c, s);
    }
    if (capturing)
        return fail(FSI_ERR_UNSUPPORTED,
                    "an HHS interval walked from the host cannot be captured (N = %d > %d, the "
                    "largest N run in one launch with these parameters)", N, hhs_grid_cap(c));
    struct OrderedGuard {
        fsi_ctx* c;
        ~OrderedGuard() { c->lists_ordered = false; }
    } ordered_guard{c};
    if (c->p.precision == FSI_MIXED && c->p.symmetric && N >= order_threshold(c)) {
        // level 0 in Morton order of the interval's starting positions: the stable
        // partitions hand the order down, so every level's slow and fast lists are in
        // spatial order too (only the summation order changes)
        CK(order_set(c, N, pos, nullptr, N, s));
        CU(cudaMemcpyAsync(c->iota.p, c->ordlist.p, (size_t)N * 4, cudaMemcpyDeviceToDevice, s));
        c->lists_ordered = true;
    } else {
        CU(launch_iota(N, P<int>(c->iota), s));
    }
    CU(cudaMemsetAsync(c->dstats.p, 0, 68 * sizeof(unsigned long long), s));
    CK(hhs_level(c, N, pos, vel, mass, is_bh, P<int>(c->iota), N, tau, 0, s));
    return merge_hhs_stats(c, s);
}

// E = T + W of all N particles, FP64 (synchronous).
int total_energy(fsi_ctx* c, int N, const double* pos, const double* vel, const double* mass,
                 cudaStream_t s, double* E) {
    CK(ensure(c->eout, 2 * sizeof(double)));
    CK(fsi_energy(c, N, pos, vel, mass, nullptr, N, P<double>(c->eout), s));
    double h[2];
    CU(cudaMemcpyAsync(h, c->eout.p, sizeof h, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    *E = h[0] + h[1];
    return FSI_OK;
}

int check_hhs_args(fsi_ctx* c, int N, const double* pos, const double* vel, const double* mass,
                   const unsigned char* is_bh, double tau) {
    CK(check_common(c, N));
    if (!pos || !vel || !mass) return fail(FSI_ERR_ARG, "NULL array");
    if (!(tau > 0.0)) return fail(FSI_ERR_ARG, "tau must be positive");
    if (c->p.c > 0.0 && !is_bh) return fail(FSI_ERR_ARG, "PN on (c > 0) needs is_bh");
    return FSI_OK;
}

}  // namespace

extern "C" {

int fsi_hhs_interval(fsi_ctx* c, int N, double* pos, double* vel, const double* mass,
                     const unsigned char* is_bh, double tau, void* stream) {
    CK(check_hhs_args(c, N, pos, vel, mass, is_bh, tau));
    const int st = hhs_interval_core(c, N, pos, vel, mass, is_bh, tau, S(stream));
    if (st == FSI_ERR_MAXLEVEL)
        return fail(FSI_ERR_MAXLEVEL, "a particle needed a level deeper than %d", c->p.max_level);
    return st;
}

int fsi_hhs_interval_restart(fsi_ctx* c, int N, double* pos, double* vel, const double* mass,
                             const unsigned char* is_bh, double tau, double eta_restart,
                             int max_restarts, int* restarts, double* rel_err, void* stream) {
    CK(check_hhs_args(c, N, pos, vel, mass, is_bh, tau));
    if (!(eta_restart >= 0.0) || max_restarts < 0)
        return fail(FSI_ERR_ARG, "eta_restart must be >= 0 and max_restarts >= 0");
    const cudaStream_t s = S(stream);
    const size_t bytes = 3 * (size_t)N * sizeof(double);
    CK(ensure(c->snapx, bytes));
    CK(ensure(c->snapv, bytes));
    CU(cudaMemcpyAsync(c->snapx.p, pos, bytes, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(c->snapv.p, vel, bytes, cudaMemcpyDeviceToDevice, s));
    double E0 = 0.0;
    CK(total_energy(c, N, pos, vel, mass, s, &E0));
    const fsi_params keep = c->p;
    double prev = INFINITY, e = INFINITY;
    int k = 0, st = FSI_OK;
    for (;; ++k) {
        // attempt k: every time-step accuracy parameter lowered by 50 % per restart
        const double f = std::ldexp(1.0, -k);
        c->p.eta_ff = keep.eta_ff * f;
        c->p.eta_fb = keep.eta_fb * f;
        c->p.eta_jerk = keep.eta_jerk * f;
        c->p.eta_grad = keep.eta_grad * f;
        c->p.eta_va = keep.eta_va * f;
        if (k > 0) {
            CU(cudaMemcpyAsync(pos, c->snapx.p, bytes, cudaMemcpyDeviceToDevice, s));
            CU(cudaMemcpyAsync(vel, c->snapv.p, bytes, cudaMemcpyDeviceToDevice, s));
        }
        st = hhs_interval_core(c, N, pos, vel, mass, is_bh, tau, s);
        if (st != FSI_OK && st != FSI_ERR_MAXLEVEL) break;
        double E1 = 0.0;
        const int re = total_energy(c, N, pos, vel, mass, s, &E1);
        if (re != FSI_OK) { st = re; break; }
        e = std::fabs((E1 - E0) / E0);
        if (e <= eta_restart || (k > 0 && e > prev) || k >= max_restarts) break;
        prev = e;
    }
    c->p = keep;
    if (restarts) *restarts = k;
    if (rel_err) *rel_err = e;
    if (st == FSI_ERR_MAXLEVEL)
        return fail(FSI_ERR_MAXLEVEL, "a particle needed a level deeper than %d", c->p.max_level);
    return st;
}

int fsi_level_stats(fsi_ctx* c, long long* counts, int max) {
    if (!c || (!counts && max > 0)) return fail(FSI_ERR_ARG, "NULL argument");
    if (c->stats_on_device) {
        // a captured interval: the level counts of its last replay
        unsigned long long st[64];
        CU(cudaDeviceSynchronize());
        CU(cudaMemcpy(st, c->dstats.p, sizeof st, cudaMemcpyDeviceToHost));
        c->level_counts.assign(std::max<size_t>(c->level_counts.size(), 64), 0);
        c->max_level_used = 0;
        for (int k = 0; k < 64; ++k) {
            c->level_counts[k] = (long long)st[k];
            if (st[k]) c->max_level_used = k;
        }
    }
    const int used = std::min<int>((int)c->level_counts.size(), c->max_level_used + 1);
    for (int k = 0; k < max; ++k) counts[k] = k < (int)c->level_counts.size() ? c->level_counts[k] : 0;
    return used;
}

// Adjoint of one cycle; rec (nullable) holds the cycle's recorded intermediates a(x0),
// a(x1), G(x1) (compact, set order), which are otherwise recomputed here.
static int step_vjp_core(fsi_ctx* c, int N, const double* pos0, const double* vel0, const double* mass,
                  const int* idx, int n, double h, const double* rec_a0, const double* rec_a1,
                  const double* rec_g1, const double* gx_out, const double* gv_out,
                  double* gx_in, double* gv_in, double* gm, void* stream) {
    CK(check_common(c, N));
    if (n < 0 || (!idx && n != N)) return fail(FSI_ERR_ARG, "bad set size n=%d N=%d", n, N);
    if (!pos0 || !vel0 || !mass || !gx_out || !gv_out || !gx_in || !gv_in || !gm)
        return fail(FSI_ERR_ARG, "NULL array");
    if (c->p.c > 0.0) return fail(FSI_ERR_UNSUPPORTED, "the adjoint covers the Newtonian FSI cycle (PN off)");
    const cudaStream_t s = S(stream);
    const size_t b3 = 3 * (size_t)N * sizeof(double);
    if (gx_in != gx_out) CU(cudaMemcpyAsync(gx_in, gx_out, b3, cudaMemcpyDeviceToDevice, s));
    if (gv_in != gv_out) CU(cudaMemcpyAsync(gv_in, gv_out, b3, cudaMemcpyDeviceToDevice, s));
    if (n == 0) return FSI_OK;
    const int prec = c->p.precision;
    const double eps2 = c->p.eps2;
    const size_t n3 = 3 * (size_t)n * 8;
    enum { X0, V0, MC, A0, X1, V1, A1, G1, X2, V2, TMP, XB, VB, WT, AB, U, MB, RPOS, RVEC, RACC, NBUF };
    for (int k = 0; k < NBUF; ++k) {
        size_t bytes = (k == MC || k == MB) ? (size_t)n * 8 : (k >= RPOS ? (size_t)n * 32 : n3);
        CK(ensure(c->vj[k], bytes));
    }
    auto B = [&](int k) { return P<double>(c->vj[k]); };
    const double* x0 = pos0;
    const double* v0 = vel0;
    const double* mc = mass;
    if (idx) {
        CU(launch_gather3(N, pos0, idx, n, B(X0), s));
        CU(launch_gather3(N, vel0, idx, n, B(V0), s));
        CU(launch_gather1(N, mass, idx, n, B(MC), s));
        x0 = B(X0); v0 = B(V0); mc = B(MC);
    }
    CK(ensure(c->rec[0], pad_tile(n) * 32));
    CK(ensure(c->accrec[0], pad_tile(n) * 32));
    auto acc_at = [&](const double* x, double* out, void* accrec) -> int {
        CU(launch_pack(prec, n, x, mc, nullptr, n, c->rec[0].p, nullptr, s));
        PairArgs a{};
        a.irec = a.jrec = c->rec[0].p;
        a.n_i = a.n_j = n;
        a.check = CHECK_DIAG;
        a.eps2 = eps2;
        a.epi.out = out;
        a.epi.accrec = accrec;
        a.epi.mc = mc;
        return run_pair(c, KIND_ACC, a, s);
    };
    // ---- the cycle's intermediates: recorded by the forward step, or recomputed here
    // (compact, FP64 state)
    const double* A0p = rec_a0 ? rec_a0 : B(A0);
    const double* A1p = rec_a0 ? rec_a1 : B(A1);
    const double* G1p = rec_a0 ? rec_g1 : B(G1);
    if (!rec_a0) CK(acc_at(x0, B(A0), nullptr));
    CU(launch_lincomb3(n, v0, A0p, h / 6.0, B(V1), s));
    CU(launch_lincomb3(n, x0, B(V1), 0.5 * h, B(X1), s));
    if (!rec_a0) {
        CK(acc_at(B(X1), B(A1), c->accrec[0].p));
        PairArgs a{};
        a.irec = a.jrec = c->rec[0].p;
        a.iacc = a.jacc = c->accrec[0].p;
        a.n_i = a.n_j = n;
        a.check = CHECK_DIAG;
        a.eps2 = eps2;
        a.epi.out = B(G1);
        CK(run_pair(c, KIND_GRAD, a, s));
    }
    CU(launch_lincomb3(n, A1p, G1p, h * h / 24.0, B(TMP), s));
    CU(launch_lincomb3(n, B(V1), B(TMP), 2.0 * h / 3.0, B(V2), s));
    CU(launch_lincomb3(n, B(X1), B(V2), 0.5 * h, B(X2), s));
    // ---- reverse (FP64 adjoint kernels on FP64 records)
    CU(launch_gather3(N, gx_out, idx, n, B(XB), s));
    CU(launch_gather3(N, gv_out, idx, n, B(VB), s));
    CU(cudaMemsetAsync(B(MB), 0, (size_t)n * 8, s));
    void* rpos = c->vj[RPOS].p;
    void* rvec = c->vj[RVEC].p;
    void* racc = c->vj[RACC].p;
    auto vjp = [&](int kind, const double* x, const double* vec, double sx, double sm, double* xb,
                   double* mb) -> int {
        CU(launch_pack(FSI_FP64, n, x, mc, nullptr, n, rpos, nullptr, s));
        CU(launch_pack_acc(FSI_FP64, n, vec, mc, nullptr, n, rvec, nullptr, s));
        CU(launch_vjp_pair(kind, n, rpos, rvec, racc, eps2, sx, sm, xb, mb, c->err_d, c->sm_count, s));
        return FSI_OK;
    };
    // v3 = v2 + h/6 a(x2)
    CK(vjp(0, B(X2), B(VB), h / 6.0, h / 6.0, B(XB), B(MB)));
    // x2 = x1 + h/2 v2
    CU(launch_lincomb3(n, B(VB), B(XB), 0.5 * h, B(VB), s));
    // v2 = v1 + 2h/3 (a(x1) + h^2/24 G(x1)): cotangent on the gradient acceleration
    const double cg = h * h / 24.0;
    CU(launch_lincomb3(n, nullptr, B(VB), 2.0 * h / 3.0, B(WT), s));
    CU(cudaMemsetAsync(B(AB), 0, n3, s));
    CK(vjp(0, B(X1), B(WT), cg, 0.0, B(AB), nullptr));               // abar = cg (dG/da)^T w
    CU(launch_lincomb3(n, B(WT), B(AB), 1.0, B(U), s));               // u = w + abar
    CK(vjp(0, B(X1), B(U), 1.0, 1.0, B(XB), B(MB)));
    CU(launch_pack_acc(FSI_FP64, n, A1p, mc, nullptr, n, racc, nullptr, s));
    CK(vjp(1, B(X1), B(WT), cg, cg, B(XB), B(MB)));
    // x1 = x0 + h/2 v1
    CU(launch_lincomb3(n, B(VB), B(XB), 0.5 * h, B(VB), s));
    // v1 = v0 + h/6 a(x0)
    CK(vjp(0, x0, B(VB), h / 6.0, h / 6.0, B(XB), B(MB)));
    CU(launch_scatter3(N, B(XB), idx, n, gx_in, s));
    CU(launch_scatter3(N, B(VB), idx, n, gv_in, s));
    CU(launch_scatter_add1(n, B(MB), idx, gm, s));
    return FSI_OK;
}

int fsi_step_vjp(fsi_ctx* c, int N, const double* pos0, const double* vel0, const double* mass,
                 const int* idx, int n, double h, const double* gx_out, const double* gv_out,
                 double* gx_in, double* gv_in, double* gm, void* stream) {
    return step_vjp_core(c, N, pos0, vel0, mass, idx, n, h, nullptr, nullptr, nullptr, gx_out,
                         gv_out, gx_in, gv_in, gm, stream);
}

int fsi_step_vjp_rec(fsi_ctx* c, int N, const double* pos0, const double* vel0,
                     const double* mass, const int* idx, int n, double h, const double* a0,
                     const double* a1, const double* g1, const double* gx_out,
                     const double* gv_out, double* gx_in, double* gv_in, double* gm,
                     void* stream) {
    if (n > 0 && (!a0 || !a1 || !g1)) return fail(FSI_ERR_ARG, "NULL recorded intermediate");
    return step_vjp_core(c, N, pos0, vel0, mass, idx, n, h, a0, a1, g1, gx_out, gv_out, gx_in,
                         gv_in, gm, stream);
}

int fsi_batch_create(fsi_ctx* c, int K, const long long* offsets, int max_steps, fsi_batch** out) {
    if (!c || !offsets || !out || K <= 0) return fail(FSI_ERR_ARG, "bad batch arguments");
    *out = nullptr;
    if (offsets[0] != 0) return fail(FSI_ERR_ARG, "offsets[0] must be 0");
    for (int k = 0; k < K; ++k)
        if (offsets[k + 1] < offsets[k]) return fail(FSI_ERR_ARG, "offsets must be non-decreasing");
    const long long ntot = offsets[K];
    if (ntot <= 0 || ntot > 2000000000LL) return fail(FSI_ERR_ARG, "bad total size %lld", ntot);
    if (max_steps <= 0) max_steps = 16;
    fsi_batch* b = new fsi_batch();
    b->K = K;
    b->ntot = ntot;
    b->max_steps = max_steps;
    b->off.assign(offsets, offsets + K + 1);
    // clusters by decreasing size: the largest work first within every phase
    std::vector<int> order(K);
    for (int k = 0; k < K; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return offsets[x + 1] - offsets[x] > offsets[y + 1] - offsets[y];
    });
    int rc = FSI_OK;
    for (int ipt : {1, 2, kBatchSymI, kBatchSymI15, kBatchSymI2}) {
        if (rc != FSI_OK) break;
        const int bs = batch_block_size(ipt);
        std::vector<BatchItem> items;
        b->nblocks_h[ipt].assign(K, 0);
        for (int k : order) {
            const int n = (int)(offsets[k + 1] - offsets[k]);
            const int nb = (n + bs - 1) / bs;
            b->nblocks_h[ipt][k] = nb;
            for (int q = 0; q < nb; ++q) items.push_back(BatchItem{k, q, (int)offsets[k], n});
        }
        b->items_per_phase[ipt] = (int)items.size();
        rc = ensure(b->items[ipt], items.size() * sizeof(BatchItem));
        if (rc == FSI_OK) rc = ensure(b->nblocks[ipt], (size_t)K * sizeof(int));
        if (rc == FSI_OK &&
            (cudaMemcpy(b->items[ipt].p, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(b->nblocks[ipt].p, b->nblocks_h[ipt].data(), (size_t)K * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess))
            rc = fail(FSI_ERR_CUDA, "batch plan upload failed");
    }
    for (int si : {kBatchSymI, kBatchSymI15, kBatchSymI2}) {
        if (rc != FSI_OK || c->p.precision != FSI_MIXED) break;
        // symmetric form: per cluster (largest first) and block of 256 si particles, the
        // block's own si tiles, then chunks of kBatchSymChunk source tiles above it
        constexpr int kBatchSymChunk = 8;
        const int bs = batch_block_size(si);
        std::vector<BatchSymItem> sit;
        std::vector<int> nsum(K, 0);
        for (int k : order) {
            const int n = (int)(offsets[k + 1] - offsets[k]);
            const int ntj = (n + 255) / 256;
            const int nb = (n + bs - 1) / bs;
            for (int q = 0; q < nb; ++q) {
                const int own0 = q * si, own1 = std::min((q + 1) * si, ntj);
                sit.push_back(BatchSymItem{k, q, (int)offsets[k], n, own0, own1});
                for (int t0 = own1; t0 < ntj; t0 += kBatchSymChunk)
                    sit.push_back(BatchSymItem{k, q, (int)offsets[k], n, t0, std::min(t0 + kBatchSymChunk, ntj)});
            }
            int cnt = 0;
            for (size_t z = 0; z < sit.size(); ++z) cnt += sit[z].cluster == k;
            nsum[k] = cnt;
        }
        b->sitems_per_phase[si] = (int)sit.size();
        rc = ensure(b->sitems[si], sit.size() * sizeof(BatchSymItem));
        if (rc == FSI_OK) rc = ensure(b->nsum[si], (size_t)K * sizeof(int));
        if (rc == FSI_OK) rc = ensure(b->accum, 3 * (size_t)ntot * sizeof(double));
        if (rc == FSI_OK &&
            (cudaMemcpy(b->sitems[si].p, sit.data(), sit.size() * sizeof(BatchSymItem), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(b->nsum[si].p, nsum.data(), (size_t)K * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess))
            rc = fail(FSI_ERR_CUDA, "batch plan upload failed");
    }
    // phases: one-sided form 2 + 3 S (pack, first pass, 3 per step); symmetric form
    // 1 + 2 (1 + 3 S) (pack, then a sum and an apply phase per pass)
    const int nphase = 3 + 6 * max_steps;
    if (rc == FSI_OK) rc = ensure(b->rec0, (size_t)ntot * 32);
    if (rc == FSI_OK) rc = ensure(b->rec1, (size_t)ntot * 32);
    if (rc == FSI_OK) rc = ensure(b->accrec, (size_t)ntot * 32);
    if (rc == FSI_OK) rc = ensure(b->ac, 3 * (size_t)ntot * 8);
    if (rc == FSI_OK) rc = ensure(b->done, (size_t)K * nphase * sizeof(int));
    if (rc == FSI_OK) rc = ensure(b->ctrl, 64);
    if (rc == FSI_OK) rc = ensure(b->stats, 8 * sizeof(unsigned long long));
    if (rc == FSI_OK && cudaMemset(b->stats.p, 0, 8 * sizeof(unsigned long long)) != cudaSuccess)
        rc = fail(FSI_ERR_CUDA, "batch counters");
    if (rc == FSI_OK) {
        b->ctas_per_sm = std::max(1, batch_max_ctas_per_sm(c->p.precision, b->ipt));
        *out = b;
        return FSI_OK;
    }
    fsi_batch_destroy(b);
    return rc;
}

int fsi_batch_destroy(fsi_batch* b) {
    if (!b) return FSI_OK;
    cudaDeviceSynchronize();
    Buf* bufs[] = {&b->items[1], &b->items[2], &b->items[kBatchSymI], &b->items[kBatchSymI15],
                   &b->items[kBatchSymI2], &b->nblocks[1], &b->nblocks[2], &b->nblocks[kBatchSymI],
                   &b->nblocks[kBatchSymI15], &b->nblocks[kBatchSymI2], &b->sitems[kBatchSymI],
                   &b->sitems[kBatchSymI15], &b->sitems[kBatchSymI2], &b->nsum[kBatchSymI],
                   &b->nsum[kBatchSymI15], &b->nsum[kBatchSymI2], &b->accum, &b->rec0, &b->rec1,
                   &b->accrec, &b->ac, &b->done, &b->ctrl, &b->stats};
    for (Buf* x : bufs)
        if (x->p) cudaFree(x->p);
    delete b;
    return FSI_OK;
}

int fsi_batch_set_tuning(fsi_ctx* c, fsi_batch* b, int ipt, int ctas_per_sm) {
    if (!c || !b) return fail(FSI_ERR_ARG, "NULL argument");
    if (ipt != 1 && ipt != 2 && !batch_sym_ipt(ipt))
        return fail(FSI_ERR_ARG, "batch variant must be 1, 2 (one-sided), %d, %d or %d (symmetric)",
                    kBatchSymI, kBatchSymI15, kBatchSymI2);
    if (batch_sym_ipt(ipt) && c->p.precision != FSI_MIXED)
        return fail(FSI_ERR_ARG, "the symmetric batch form is mixed precision");
    const int mx = std::max(1, batch_sym_ipt(ipt) ? batch_sym_max_ctas_per_sm(ipt)
                                                  : batch_max_ctas_per_sm(c->p.precision, ipt));
    if (ctas_per_sm <= 0 || ctas_per_sm > mx) ctas_per_sm = mx;
    b->ipt = ipt;
    b->ctas_per_sm = ctas_per_sm;
    return FSI_OK;
}

int fsi_batch_get_tuning(fsi_batch* b, int* ipt, int* ctas_per_sm) {
    if (!b) return fail(FSI_ERR_ARG, "NULL batch");
    if (ipt) *ipt = b->ipt;
    if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
    return FSI_OK;
}

int fsi_batch_stats(fsi_batch* b, long long* wait_ns, long long* life_ns, int* ctas, int reset) {
    if (!b) return fail(FSI_ERR_ARG, "NULL batch");
    unsigned long long st[2] = {0, 0};
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(st, b->stats.p, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(FSI_ERR_CUDA, "batch counters read");
    if (reset && cudaMemset(b->stats.p, 0, sizeof st) != cudaSuccess)
        return fail(FSI_ERR_CUDA, "batch counters reset");
    if (wait_ns) *wait_ns = (long long)st[0];
    if (life_ns) *life_ns = (long long)st[1];
    if (ctas) *ctas = b->last_ctas;
    return FSI_OK;
}

int fsi_batch_item_stats(fsi_batch* b, long long* ns, long long* items, int reset) {
    if (!b || !ns || !items) return fail(FSI_ERR_ARG, "NULL argument");
    unsigned long long st[6] = {};
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(st, P<unsigned long long>(b->stats) + 2, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(FSI_ERR_CUDA, "batch counters read");
    if (reset && cudaMemset(P<unsigned long long>(b->stats) + 2, 0, sizeof st) != cudaSuccess)
        return fail(FSI_ERR_CUDA, "batch counters reset");
    for (int k = 0; k < 3; ++k) {
        ns[k] = (long long)st[k];
        items[k] = (long long)st[3 + k];
    }
    return FSI_OK;
}

int fsi_batch_inject_stall(fsi_batch* b, int cluster) {
    if (!b || cluster < 0 || cluster >= b->K) return fail(FSI_ERR_ARG, "bad cluster");
    b->stall_cluster = cluster;
    return FSI_OK;
}

int fsi_batch_step(fsi_ctx* c, fsi_batch* b, double* pos, double* vel, const double* mass,
                   double h, int nsteps, void* stream) {
    if (!c || !b) return fail(FSI_ERR_ARG, "NULL argument");
    if (!pos || !vel || !mass) return fail(FSI_ERR_ARG, "NULL array");
    if (nsteps <= 0) return FSI_OK;
    if (nsteps > b->max_steps) return fail(FSI_ERR_ARG, "nsteps %d exceeds the plan's max_steps %d", nsteps, b->max_steps);
    if (c->p.c > 0.0) return fail(FSI_ERR_UNSUPPORTED, "batched steps are Newtonian (PN off)");
    const cudaStream_t s = S(stream);
    const int ipt = b->ipt;
    const bool sym = batch_sym_ipt(ipt);
    if (sym && c->p.precision != FSI_MIXED) return fail(FSI_ERR_ARG, "the symmetric batch form is mixed precision");
    const int nphase = sym ? 3 + 6 * nsteps : 2 + 3 * nsteps;
    CU(cudaMemsetAsync(b->done.p, 0, (size_t)b->K * nphase * sizeof(int), s));
    CU(cudaMemsetAsync(b->ctrl.p, 0, 64, s));
    int* nblocks = P<int>(b->nblocks[ipt]);
    if (b->stall_cluster >= 0) {
        // test hook: one cluster waits for a phase count that is never reached
        const int k = b->stall_cluster;
        const int bumped = b->nblocks_h[ipt][k] + 1;
        CU(cudaMemcpy(nblocks + k, &bumped, sizeof(int), cudaMemcpyHostToDevice));
    }
    BatchArgs a{};
    a.items = reinterpret_cast<const BatchItem*>(b->items[ipt].p);
    a.items_per_phase = b->items_per_phase[ipt];
    a.nphase = nphase;
    a.nsteps = nsteps;
    a.nblocks = nblocks;
    a.x = pos;
    a.v = vel;
    a.m = mass;
    a.ntot = b->ntot;
    a.rec0 = b->rec0.p;
    a.rec1 = b->rec1.p;
    a.accrec = b->accrec.p;
    a.ac = P<double>(b->ac);
    a.done = P<int>(b->done);
    a.next = P<int>(b->ctrl);
    a.abort_flag = P<int>(b->ctrl) + 4;
    a.stats = P<unsigned long long>(b->stats);
    a.h = h;
    a.eps2 = c->p.eps2;
    a.err = c->err_d;
    a.timeout_ns = budget(c);
    const int ctas = c->sm_count * b->ctas_per_sm;
    b->last_ctas = ctas;
    if (sym) {
        CU(cudaMemsetAsync(b->accum.p, 0, 3 * (size_t)b->ntot * sizeof(double), s));
        CU(launch_batch_sym(ipt, ctas, a, reinterpret_cast<const BatchSymItem*>(b->sitems[ipt].p),
                            b->sitems_per_phase[ipt], P<int>(b->nsum[ipt]), P<double>(b->accum), s));
    } else {
        CU(launch_batch(c->p.precision, ipt, ctas, a, s));
    }
    if (b->stall_cluster >= 0) {
        const int k = b->stall_cluster;
        CU(cudaMemcpyAsync(nblocks + k, &b->nblocks_h[ipt][k], sizeof(int), cudaMemcpyHostToDevice, s));
        CU(cudaStreamSynchronize(s));
        b->stall_cluster = -1;
    }
    return FSI_OK;
}

int fsi_profile(fsi_ctx* c, int enable) {
    if (!c) return fail(FSI_ERR_ARG, "NULL context");
    c->profiling = enable != 0;
    return FSI_OK;
}

int fsi_grid_stats(fsi_ctx* c, long long* ns, long long* phases, int reset, void* stream) {
    if (!c || !ns || !phases) return fail(FSI_ERR_ARG, "NULL argument");
    unsigned long long st[16] = {};
    const cudaStream_t s = S(stream);
    if (c->gprof.p) {
        CU(cudaMemcpyAsync(st, c->gprof.p, sizeof st, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (reset) CU(cudaMemsetAsync(c->gprof.p, 0, sizeof st, s));
    }
    for (int k = 0; k < 8; ++k) {
        ns[k] = (long long)st[k];
        phases[k] = (long long)st[8 + k];
    }
    return FSI_OK;
}

int fsi_profile_read(fsi_ctx* c, long long* launches, double* ms) {
    if (!c || !launches || !ms) return fail(FSI_ERR_ARG, "NULL argument");
    for (int k = 0; k < 3; ++k) { launches[k] = 0; ms[k] = 0.0; }
    for (auto& r : c->prof) {
        float t = 0.f;
        CU(cudaEventSynchronize(r.b));
        CU(cudaEventElapsedTime(&t, r.a, r.b));
        if (r.kind >= 0 && r.kind < 3) { launches[r.kind] += 1; ms[r.kind] += t; }
        c->ev_pool.push_back(r.a);
        c->ev_pool.push_back(r.b);
    }
    c->prof.clear();
    return FSI_OK;
}

long long fsi_launch_count(void) { return g_launches.load(); }

int fsi_work_stats(fsi_ctx* c, long long* acc_pairs, long long* grad_pairs, int reset) {
    if (!c) return fail(FSI_ERR_ARG, "NULL context");
    if (acc_pairs) *acc_pairs = c->work_pairs[KIND_ACC];
    if (grad_pairs) *grad_pairs = c->work_pairs[KIND_GRAD];
    if (reset) c->work_pairs[0] = c->work_pairs[1] = 0;
    return FSI_OK;
}

}  // extern "C"

namespace {

// Time every candidate variant of both kinds on the first n particles as one set and keep
// the fastest in *slot(kind).
template <class Slot>
int tune_set(fsi_ctx* c, int N, const double* pos, const double* mass, int n, int reps,
             cudaStream_t s, Slot slot) {
    const int prec = c->p.precision;
    CK(ensure(c->rec[0], pad_tile(n) * 32));
    CK(ensure(c->accrec[0], pad_tile(n) * 32));
    CK(ensure(c->tA, 3 * (size_t)n * 8));
    FarGuard far_guard{c};
    const int* list = nullptr;
    if (prec == FSI_MIXED && c->p.symmetric && n >= order_threshold(c)) {
        // the far-tile variants are timed as step_core runs them: set in Morton order
        CK(order_set(c, N, pos, nullptr, n, s));
        list = P<int>(c->ordlist);
        CK(far_setup(c, mass, list, n, s));
    }
    CU(launch_pack(prec, N, pos, mass, list, n, c->rec[0].p, nullptr, s));
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    int rc = FSI_OK;
    for (int kind = 0; kind < 2 && rc == FSI_OK; ++kind) {
        int cand[16];
        const int nc = c->p.symmetric ? sym_variants(prec, kind, cand) : pair_variants(prec, kind, cand);
        float best = 3.4e38f;
        int& cur = slot(kind);
        int best_v = cur;
        for (int v = 0; v < nc && rc == FSI_OK; ++v) {
            cur = cand[v];
            PairArgs a{};
            a.irec = a.jrec = c->rec[0].p;
            a.iacc = a.jacc = c->accrec[0].p;
            a.n_i = a.n_j = n;
            a.check = CHECK_DIAG;
            a.eps2 = c->p.eps2;
            a.epi.out = P<double>(c->tA);
            if (kind == KIND_ACC) a.epi.accrec = c->accrec[0].p;
            rc = run_pair(c, kind, a, s);                      // warm-up (and accel records)
            if (rc != FSI_OK) break;
            if (cudaEventRecord(e0, s) != cudaSuccess) { rc = fail(FSI_ERR_CUDA, "event"); break; }
            for (int r = 0; r < reps && rc == FSI_OK; ++r) rc = run_pair(c, kind, a, s);
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                rc = fail(FSI_ERR_CUDA, "event");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; best_v = cand[v]; }
        }
        cur = best_v;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace

extern "C" {

int fsi_autotune(fsi_ctx* c, int N, const double* pos, const double* mass, int n, int reps,
                 void* stream) {
    CK(check_common(c, N));
    if (n <= 0 || n > N || !pos || !mass) return fail(FSI_ERR_ARG, "bad autotune arguments");
    if (reps <= 0) reps = 2;
    const cudaStream_t s = S(stream);
    const int prec = c->p.precision;
    const bool was = c->profiling;
    c->profiling = false;
    int rc = FSI_OK;
    if (!c->p.symmetric) {
        rc = tune_set(c, N, pos, mass, n, reps, s,
                      [&](int kind) -> int& { return c->ipt[prec][kind][n >= kOneSidedLarge]; });
        for (int kind = 0; kind < 2; ++kind)      // the sampled size stands for both classes
            c->ipt[prec][kind][n < kOneSidedLarge] = c->ipt[prec][kind][n >= kOneSidedLarge];
    } else {
        // one sample per size class that n reaches: 8192 (or n), 65536 (or n), n
        for (int k = 0; k < kSymClasses && rc == FSI_OK; ++k) {
            const int hi = k + 1 < kSymClasses ? kSymClassMin[k + 1] : INT_MAX;
            if (n < kSymClassMin[k]) break;
            int m = k == 0 ? std::min(n, 8192) : k == 1 ? std::min(n, 65536) : n;
            m = std::min(std::max(m, kSymClassMin[k]), hi - 1);
            if (m > n) break;
            rc = tune_set(c, N, pos, mass, m, reps, s,
                          [&](int kind) -> int& { return c->symv[prec][kind][k]; });
        }
    }
    c->profiling = was;
    return rc;
}

int fsi_get_tuning(fsi_ctx* c, int* ipt_acc, int* ipt_grad) {
    if (!c) return fail(FSI_ERR_ARG, "NULL context");
    const int prec = c->p.precision;
    const int k = kSymClasses - 1;
    if (ipt_acc) *ipt_acc = c->p.symmetric ? c->symv[prec][KIND_ACC][k] : c->ipt[prec][KIND_ACC][1];
    if (ipt_grad) *ipt_grad = c->p.symmetric ? c->symv[prec][KIND_GRAD][k] : c->ipt[prec][KIND_GRAD][1];
    return FSI_OK;
}

int fsi_get_tuning_for(fsi_ctx* c, int n, int* ipt_acc, int* ipt_grad) {
    if (!c) return fail(FSI_ERR_ARG, "NULL context");
    if (n < 0) return fail(FSI_ERR_ARG, "negative set size");
    const int prec = c->p.precision;
    const int k = sym_class(n);
    const int big = n >= kOneSidedLarge;
    if (ipt_acc) *ipt_acc = c->p.symmetric ? c->symv[prec][KIND_ACC][k] : c->ipt[prec][KIND_ACC][big];
    if (ipt_grad) *ipt_grad = c->p.symmetric ? c->symv[prec][KIND_GRAD][k] : c->ipt[prec][KIND_GRAD][big];
    return FSI_OK;
}

int fsi_set_tuning(fsi_ctx* c, int ipt_acc, int ipt_grad) {
    if (!c) return fail(FSI_ERR_ARG, "NULL context");
    int cand[16];
    const int prec = c->p.precision;
    for (int kind = 0; kind < 2; ++kind) {
        const int want = kind == KIND_ACC ? ipt_acc : ipt_grad;
        const int nc = c->p.symmetric ? sym_variants(prec, kind, cand) : pair_variants(prec, kind, cand);
        bool ok = false;
        for (int v = 0; v < nc; ++v) ok |= cand[v] == want;
        if (!ok) return fail(FSI_ERR_ARG, "unsupported kernel variant %d", want);
    }
    if (c->p.symmetric) {
        for (int k = 0; k < kSymClasses; ++k) {
            c->symv[prec][KIND_ACC][k] = ipt_acc;
            c->symv[prec][KIND_GRAD][k] = ipt_grad;
        }
    } else {
        for (int b = 0; b < 2; ++b) {
            c->ipt[prec][KIND_ACC][b] = ipt_acc;
            c->ipt[prec][KIND_GRAD][b] = ipt_grad;
        }
    }
    return FSI_OK;
}

int fsi_far_stats(fsi_ctx* c, long long* far_visits, long long* near_visits, int reset,
                  void* stream) {
    if (!c) return fail(FSI_ERR_ARG, "NULL context");
    unsigned long long st[2] = {0, 0};
    const cudaStream_t s = S(stream);
    if (c->farstats.p) {
        CU(cudaMemcpyAsync(st, c->farstats.p, sizeof st, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (reset) CU(cudaMemsetAsync(c->farstats.p, 0, sizeof st, s));
    }
    if (far_visits) *far_visits = (long long)st[0];
    if (near_visits) *near_visits = (long long)st[1];
    return FSI_OK;
}

int fsi_fma_probe(int fp64, int blocks, int iters, void* sink, double* flops, void* stream) {
    if (blocks <= 0 || iters <= 0 || !sink || fp64 < 0 || fp64 > 2)
        return fail(FSI_ERR_ARG, "bad probe arguments");
    CU(launch_fma_probe(fp64, blocks, iters, sink, S(stream)));
    if (flops) *flops = (double)blocks * 256.0 * (double)iters * 4.0 * 8.0 * (fp64 == 2 ? 4.0 : 2.0);
    return FSI_OK;
}

}  // extern "C"
