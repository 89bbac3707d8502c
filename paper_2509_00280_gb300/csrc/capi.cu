// capi.cu -- the C ABI declared in include/relate.h: argument validation,
// the device-memory lifetime of an encoding, the encode pipeline, MTTKRP
// dispatch and the CP-ALS driver loop.
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "internal.cuh"

using namespace relate;

namespace {

thread_local char g_err[512] = "";

int fail(int status, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return status;
}

int cuda_fail(cudaError_t e, const char *where) {
    return fail(e == cudaErrorMemoryAllocation ? RELATE_ERR_OOM : RELATE_ERR_CUDA, "%s: %s (%s)", where,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

bool valid_precision(int f, int a) {
    return (f == RELATE_F64 && a == RELATE_F64) || (f == RELATE_F32 && a == RELATE_F32) ||
           (f == RELATE_BF16 && a == RELATE_F32);
}

int dtype_bytes(int d) { return d == RELATE_F64 ? 8 : d == RELATE_F32 ? 4 : 2; }

// Device memory of handles comes from one stream-ordered pool per device,
// owned by the library. Its release threshold is unlimited: freed blocks stay
// mapped for the next encode or CP-ALS instead of going back to the driver
// at every synchronisation (relate_release_cached_memory trims it).
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};

cudaError_t lib_pool(cudaMemPool_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

// Test hook: RELATE_FAULT=alloc makes every library allocation fail (as if
// the device were out of memory); RELATE_FAULT=timeout makes every MTTKRP
// launch skip its first tile copy with a 1e8-cycle wait limit, so that the
// bounded wait runs out and the launch reports a timeout;
// RELATE_FAULT=gram_timeout makes every tensor-core Gram issue no MMA, with
// the same short limit on its waits for their completion. Unset in normal use.
bool fault_is(const char *what) {
    const char *f = getenv("RELATE_FAULT");
    return f && strcmp(f, what) == 0;
}

// launch_gram with the gram_timeout test hook applied; a tensor-core wait
// that runs out sets bit 1 of *err.
cudaError_t gram_checked(const void *A, int64_t I, int R, int dtype, double *scratch, double *G, int *err,
                         cudaStream_t st, bool cpals = false) {
    const bool f = fault_is("gram_timeout");
    return launch_gram(A, I, R, dtype, scratch, G, err, st, f ? 100000000LL : 0, f ? 1 : 0,
                       cpals && !f && dense_f64_small(I, R));
}

template <typename T>
cudaError_t dalloc(T **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (fault_is("alloc")) return cudaErrorMemoryAllocation;
    cudaMemPool_t pool = nullptr;
    const cudaError_t e = lib_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(reinterpret_cast<void **>(p), bytes, pool, st);
}

// Device bytes of each allocation. relate_encode, the CP-ALS workspace and
// relate_footprint all size their buffers from these.
// 64 bytes of tail padding: tile copies round their size up to 16 bytes
size_t words_bytes(int64_t nnz, size_t kb) { return (size_t)nnz * kb + 64; }
size_t vals_bytes(int64_t nnz, int vb) { return (size_t)nnz * vb + 64; }
size_t bounds_bytes(int64_t P, int N) { return (size_t)(P + 1) * N * 4; }
size_t perm_bytes(int64_t nnz) { return (size_t)nnz * 4 + 16; }
size_t tperm_bytes(int64_t nnz) { return (size_t)nnz * 2 + 64; }
constexpr size_t kSmallBytes = 8 * (1 + 3 * kMaxModes) + 1024 * 8;

struct WsSizes {
    size_t M, scratch, G, RR8, RR4, R8;
};
WsSizes ws_sizes(uint64_t maxI, int N, int R) {
    return WsSizes{maxI * R * 8 + 16, dense_scratch_doubles(R) * 8, (size_t)N * R * R * 8, (size_t)R * R * 8,
                   (size_t)R * R * 4, (size_t)R * 8};
}
size_t ws_total(uint64_t maxI, int N, int R) {
    const WsSizes w = ws_sizes(maxI, N, R);
    return w.M + w.scratch + w.G + 2 * w.RR8 + w.RR4 + 2 * w.R8 + 64 + 64;
}

// Pinned host words for the per-iteration fit / status read-back, handed out
// in 64-byte slots from page-locked chunks that live until the process exits
// (freeing page-locked memory synchronises the device, which would stall the
// other streams of a serving process at every handle release).
class PinnedSlots {
  public:
    double *get() {
        std::lock_guard<std::mutex> lock(mu_);
        if (free_.empty()) {
            void *chunk = nullptr;
            if (cudaMallocHost(&chunk, kChunk * kSlot) != cudaSuccess) return nullptr;
            for (int i = kChunk - 1; i >= 0; i--) free_.push_back(static_cast<char *>(chunk) + (size_t)i * kSlot);
        }
        char *p = free_.back();
        free_.pop_back();
        return reinterpret_cast<double *>(p);
    }
    void put(double *p) {
        std::lock_guard<std::mutex> lock(mu_);
        free_.push_back(reinterpret_cast<char *>(p));
    }

  private:
    static constexpr int kChunk = 256, kSlot = 64;
    std::mutex mu_;
    std::vector<char *> free_;
};
PinnedSlots g_pinned;

}  // namespace

namespace relate {
// Records the last-error message of this host thread for entry points in other
// translation units; returns status.
int set_last_error(int status, const char *msg) {
    snprintf(g_err, sizeof(g_err), "%s", msg ? msg : "");
    return status;
}
// The RELATE_FAULT test hook, for entry points in other translation units.
bool fault_injected(const char *what) { return fault_is(what); }
}  // namespace relate

struct relate_handle_s {
    int N = 0;
    int64_t nnz = 0;
    uint64_t dims[kMaxModes] = {};
    int lbits[kMaxModes] = {};
    int lp = 0;
    int KW = 1;
    int8_t order[RELATE_MAX_KEY_BITS] = {};
    BitRuns runs{};
    Fields fields{};
    int64_t S = 4096, P = 0;
    relate_dtype_t val_dtype = RELATE_F32, factor_dtype = RELATE_F32, acc_dtype = RELATE_F32;
    relate_conflict_t conflict[kMaxModes] = {};
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 152, smem_optin = 0, smem_budget = 0;

    void *d_words = nullptr;
    void *d_vals = nullptr;
    uint32_t *d_perm = nullptr;
    uint32_t *d_plo = nullptr, *d_phi = nullptr;
    uint32_t *d_counts[kMaxModes] = {};
    uint32_t *d_hot_rows[kMaxModes] = {};
    void *d_hot_scratch = nullptr;  // per-block copies of hot rows (SEGMENTED MTTKRP)
    uint16_t *d_tperm[kMaxModes] = {};  // per-mode tile order (SEGMENTED MTTKRP), built on first use
    int tperm_depth[kMaxModes] = {};    // the fiber-factoring depth each tile order was sorted for
    // per-mode fiber-factoring plan (relate_set_mode_plan): depth -1 = AUTO,
    // level order valid when level_set, column passes 0 = AUTO
    int plan_depth[kMaxModes] = {-1, -1, -1, -1, -1, -1, -1, -1};
    int8_t plan_level[kMaxModes][kMaxModes] = {};
    bool level_set[kMaxModes] = {};
    int plan_passes[kMaxModes] = {};
    int plan_kr[kMaxModes] = {-1, -1, -1, -1, -1, -1, -1, -1};  // Khatri-Rao pair: -1 AUTO, 0 off, 1 on
    // the Khatri-Rao rows of the last fused pair (grown on demand) and what
    // they hold: modes (kr_a, kr_b) of factors (kr_fa, kr_fb) at rank kr_R;
    // kr_valid is cleared whenever one of those factors may have changed
    void *d_kr = nullptr;
    size_t kr_bytes = 0;
    int kr_a = -1, kr_b = -1, kr_R = 0;
    const void *kr_fa = nullptr, *kr_fb = nullptr;
    bool kr_valid = false;
    double *d_normX2 = nullptr;
    int *d_err = nullptr;  // device error flags of this handle's kernels
    uint64_t runs_n[kMaxModes] = {}, distinct[kMaxModes] = {}, maxcount[kMaxModes] = {};

    // CP-ALS workspace (grown on demand)
    int ws_R = 0;
    void *d_M = nullptr;
    double *d_scratch = nullptr, *d_G = nullptr, *d_Vinv = nullptr, *d_lambda = nullptr, *d_inner = nullptr,
           *d_fit = nullptr, *d_V = nullptr;
    float *d_Vinv32 = nullptr;
    int *d_status = nullptr;
    // the normal equations of mode n run on `aux`, overlapped with mode n's
    // MTTKRP (they depend only on the other modes' Grams)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_g = nullptr, ev_v = nullptr;
    int use_graph = 0;           // relate_cpals replays a captured iteration
    // nonzero sharding: this handle holds slice [shard_lo, shard_lo + nnz) of
    // the globally sorted stream of `nnz_total` nonzeros; relate_cpals sums
    // each mode's MTTKRP and ||X||^2 over the shards with reduce_fn
    int64_t nnz_total = 0, shard_lo = 0;
    relate_reduce_fn reduce_fn = nullptr;
    void *reduce_user = nullptr;
    double *h_pinned = nullptr;  // pinned host words: fit, status[2], err

    // Device memory comes from the stream-ordered allocator and goes back to
    // it on the handle's stream once that stream and `aux` are idle, so the
    // release never waits for other streams' work.
    ~relate_handle_s() {
        if (aux) {
            cudaStreamSynchronize(aux);
            cudaStreamDestroy(aux);
        }
        if (stream) cudaStreamSynchronize(stream);
        else cudaDeviceSynchronize();
        if (ev_g) cudaEventDestroy(ev_g);
        if (ev_v) cudaEventDestroy(ev_v);
        if (h_pinned) g_pinned.put(h_pinned);
        void *ptrs[] = {d_words, d_vals, d_perm, d_plo, d_phi, d_normX2, d_err, d_M, d_scratch, d_G, d_Vinv,
                        d_lambda, d_inner, d_fit, d_Vinv32, d_status, d_V, d_hot_scratch, d_kr};
        for (void *p : ptrs)
            if (p) cudaFreeAsync(p, stream);
        for (auto *p : d_counts)
            if (p) cudaFreeAsync(p, stream);
        for (auto *p : d_hot_rows)
            if (p) cudaFreeAsync(p, stream);
        for (auto *p : d_tperm)
            if (p) cudaFreeAsync(p, stream);
        cudaStreamSynchronize(stream);
    }
};

namespace {

relate_conflict_t resolve_conflict(const relate_handle_s *h, int mode, int R) {
    if (h->conflict[mode] != RELATE_CONFLICT_AUTO) return h->conflict[mode];
    const int accb = mttkrp_acc_bytes(h->factor_dtype);
    const uint64_t priv_bytes = h->dims[mode] * (uint64_t)R * accb;
    // whole-output privatisation when it leaves room for two blocks per SM;
    // except a short, heavily populated mode on the vector path: the
    // SEGMENTED kernel then keeps every one of its rows in its per-block
    // copies, and runs 1.3x faster than privatising the output in shared memory
    if (priv_bytes <= 32u * 1024u) {
        const uint64_t fb = (uint64_t)dtype_bytes(h->factor_dtype);
        // on the vector path a short mode whose output fits the per-block copy
        // (kHotBlockBytes) takes SEGMENTED with every row in that copy: faster
        // than privatising it in shared memory (the 100-row mode of the 5-mode
        // workload: 3.5 against 8.1 ms), and each block adds only its own
        // tiles' runs to its copy, so FP32 roundings stay few per row
        if (h->N <= 5 && priv_bytes <= kHotBlockBytes && ((uint64_t)R * fb) % 16 == 0 &&
            ((uint64_t)R * accb) % 16 == 0)
            return RELATE_CONFLICT_SEGMENTED;
        return RELATE_CONFLICT_PRIVATIZED;
    }
    const double reuse = h->distinct[mode] ? (double)h->nnz / (double)h->distinct[mode] : 0.0;
    const double mean_run = h->runs_n[mode] ? (double)h->nnz / (double)h->runs_n[mode] : 0.0;
    // "minimum fiber reuse 8" (Sec. 4.1.3) for reduction-based synchronisation
    if (reuse >= 8.0 || mean_run >= 8.0) return RELATE_CONFLICT_SEGMENTED;
    return RELATE_CONFLICT_ATOMIC;
}

int build_runs(relate_handle_s *h) {
    struct Run {
        int mode, src, dst, len;
    };
    std::vector<Run> runs;
    int next[kMaxModes] = {};
    for (int t = 0; t < h->lp; t++) {
        const int m = h->order[t];
        const int s = next[m]++;
        if (!runs.empty() && runs.back().mode == m && runs.back().dst + runs.back().len == t &&
            runs.back().src + runs.back().len == s)
            runs.back().len++;
        else
            runs.push_back({m, s, t, 1});
    }
    BitRuns br{};
    int off = 0;
    for (int m = 0; m < kMaxModes; m++) {
        br.mode_begin[m] = br.nruns;
        br.field_off[m] = m < h->N ? off : 0;
        if (m < h->N) {
            for (const Run &r : runs)
                if (r.mode == m) {
                    br.src[br.nruns] = (uint8_t)r.src;
                    br.dst[br.nruns] = (uint8_t)r.dst;
                    br.len[br.nruns] = (uint8_t)r.len;
                    br.nruns++;
                }
            off += h->lbits[m];
        }
    }
    br.mode_begin[kMaxModes] = br.nruns;
    h->runs = br;
    for (int m = 0; m < kMaxModes; m++) {
        h->fields.shift[m] = br.field_off[m];
        const int l = m < h->N ? h->lbits[m] : 0;
        h->fields.mask[m] = l >= 32 ? 0xffffffffu : ((1u << l) - 1u);
    }
    return RELATE_OK;
}

int bits_for(uint64_t I) {
    int b = 0;
    while (b < 64 && ((uint64_t)1 << b) < I) b++;
    return b;
}

struct AsyncBufs {
    cudaStream_t st;
    std::vector<void *> ptrs;
    cudaError_t alloc(void **p, size_t bytes) {
        *p = nullptr;
        cudaError_t e = dalloc(p, bytes ? bytes : 16, st);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    ~AsyncBufs() {
        for (void *p : ptrs) cudaFreeAsync(p, st);
    }
};

// The handle's second stream and its two events. The normal equations (one
// block) run on it at the highest stream priority, so that the block
// scheduler places them before the waiting MTTKRP blocks; relate_encode
// copies host values on it while the keys are built and sorted.
cudaError_t ensure_aux(relate_handle_s *h) {
    if (h->aux) return cudaSuccess;
    int prio_lo = 0, prio_hi = 0;
    cudaError_t e;
    if ((e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi)) != cudaSuccess ||
        (e = cudaStreamCreateWithPriority(&h->aux, cudaStreamNonBlocking, prio_hi)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->ev_g, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->ev_v, cudaEventDisableTiming)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

int ensure_ws(relate_handle_s *h, int R) {
    if (h->ws_R >= R && h->d_M) return RELATE_OK;
    const cudaStream_t st = h->stream;
    void *ptrs[] = {h->d_M, h->d_scratch, h->d_G, h->d_Vinv, h->d_lambda, h->d_inner, h->d_fit, h->d_Vinv32,
                    h->d_status, h->d_V};
    // earlier iterations on aux are joined into `st` before their results are
    // used, so stream order on `st` covers every use of the old buffers
    for (void *p : ptrs)
        if (p) cudaFreeAsync(p, st);
    h->d_M = nullptr;
    h->d_scratch = h->d_G = h->d_Vinv = h->d_lambda = h->d_inner = h->d_fit = h->d_V = nullptr;
    h->d_Vinv32 = nullptr;
    h->d_status = nullptr;
    h->ws_R = 0;
    uint64_t maxI = 0;
    for (int m = 0; m < h->N; m++) maxI = h->dims[m] > maxI ? h->dims[m] : maxI;
    const WsSizes w = ws_sizes(maxI, h->N, R);
    cudaError_t e;
    if ((e = dalloc(&h->d_M, w.M, st)) != cudaSuccess ||
        (e = dalloc((void **)&h->d_scratch, w.scratch, st)) != cudaSuccess ||
        (e = dalloc((void **)&h->d_G, w.G, st)) != cudaSuccess ||
        (e = dalloc((void **)&h->d_Vinv, w.RR8, st)) != cudaSuccess ||
        (e = dalloc((void **)&h->d_V, w.RR8, st)) != cudaSuccess ||
        (e = dalloc((void **)&h->d_Vinv32, w.RR4, st)) != cudaSuccess ||
        (e = dalloc((void **)&h->d_lambda, w.R8, st)) != cudaSuccess ||
        (e = dalloc((void **)&h->d_inner, w.R8, st)) != cudaSuccess ||
        (e = dalloc((void **)&h->d_fit, 64, st)) != cudaSuccess ||
        (e = dalloc((void **)&h->d_status, 64, st)) != cudaSuccess)
        return cuda_fail(e, "relate_cpals workspace");
    if ((e = ensure_aux(h)) != cudaSuccess) return cuda_fail(e, "relate_cpals: auxiliary stream");
    h->ws_R = R;
    return RELATE_OK;
}

void fill_stream_args(const relate_handle_s *h, int mode, MttkrpArgs &a) {
    a.words = h->d_words;
    a.vals = h->d_vals;
    a.nnz = h->nnz;
    a.S = h->S;
    a.P = h->P;
    a.N = h->N;
    a.mode = mode;
    a.fields = h->fields;
    a.In = h->dims[mode];
    a.plo = h->d_plo;
    a.phi = h->d_phi;
    a.hot_rows = h->d_hot_rows[mode];
    a.maxcount = h->maxcount[mode];
}

// Fiber-factoring plan of a mode (mttkrp_fac.cuh): the SEGMENTED strategy of
// a 3- to 5-mode tensor sums fibers of equal (i_n, i_{p1}, ..., i_{pl}) for
// l <= depth before multiplying by A_pl. AUTO: depth N - 2 and the other modes
// ordered longest first, one column pass: the rows of the longest factors,
// the ones that miss in L2, are gathered once per outer fiber, and the
// innermost slot (gathered per nonzero) is the shortest factor, which stays
// in L1 or L2.
//
// Khatri-Rao pair: with FP64 factors (FP64-pipe bound), depth >= 2 and one
// unfactored slot, the deepest level's mode a and the innermost mode b are
// fused into one slot over the rows of A_a (.) A_b (the Khatri-Rao product of
// the MTTKRP's definition, Sec. 2.2), built before the launch: each nonzero
// then costs one FMA at that level instead of one plus one per closed level-a
// fiber. AUTO fuses when the table has at most nnz / 4 rows (each row reused
// 4 times on average): building a row costs about one FMA per element, and
// on the 150M-nonzero 4-mode tensor even the 24M-row table of its 100K-row
// mode cut that mode from 45.9 to 35.9 ms, build included. On or off by
// relate_set_mode_kr.
struct ModePlan {
    int depth;
    int8_t level[kMaxModes];
    int passes;
    int kr;  // 1: fuse slots depth and depth + 1 (modes level[depth - 1], level[depth])
};

// Largest Khatri-Rao table: rows below 2^32 (32-bit record slots) and 16 GiB.
constexpr uint64_t kKrMaxBytes = 16ull << 30;
bool kr_fits(uint64_t rows, int R) { return rows < (1ull << 32) && rows * (uint64_t)R * 8 <= kKrMaxBytes; }
bool kr_auto(uint64_t rows, int64_t nnz) { return rows * 4 <= (uint64_t)nnz; }

ModePlan resolve_plan(const relate_handle_s *h, int mode, int R) {
    ModePlan p{};
    p.passes = h->plan_passes[mode] > 0 ? h->plan_passes[mode] : 1;
    if (h->N < 3 || h->N > 5 || resolve_conflict(h, mode, R) != RELATE_CONFLICT_SEGMENTED) {
        p.depth = 0;
    } else {
        // AUTO: FP64 factors are bound by the FP64 pipe, so every repeated
        // fiber saves work: all N - 2 levels (the 150M-nonzero 4-mode workload:
        // 10.4 against 11.3 ms per mode at 30M nonzeros). FP32 / BF16 factors
        // are bound by gather latency, and the flat loop, which issues every
        // gather of a record up front, is faster (2.5 against 3.1 ms FP32).
        const int autod = h->factor_dtype == RELATE_F64 ? h->N - 2 : 0;
        p.depth = h->plan_depth[mode] >= 0 ? h->plan_depth[mode] : autod;
        if (p.depth > h->N - 2) p.depth = h->N - 2;
    }
    if (h->level_set[mode]) {
        for (int s = 0; s < h->N - 1; s++) p.level[s] = h->plan_level[mode][s];
    } else {
        int n = 0;
        for (int k = 0; k < h->N; k++)
            if (k != mode) p.level[n++] = (int8_t)k;
        for (int x = 0; x < n; x++)  // stable order by decreasing I_k
            for (int y = x + 1; y < n; y++)
                if (h->dims[p.level[y]] > h->dims[p.level[x]]) {
                    const int8_t t = p.level[x];
                    p.level[x] = p.level[y];
                    p.level[y] = t;
                }
    }
    // the sort key (i_n, slots 1..depth, position in the tile) must fit 128 bits
    int bits = h->lbits[mode] + 11;
    for (int s = 0; s < p.depth; s++) bits += h->lbits[p.level[s]];
    while (p.depth > 0 && bits > 128) bits -= h->lbits[p.level[--p.depth]];
    p.kr = 0;
    if (h->factor_dtype == RELATE_F64 && p.depth >= 2 && h->N - 1 - p.depth == 1 && R % 2 == 0) {
        const uint64_t rows = h->dims[p.level[p.depth - 1]] * h->dims[p.level[p.depth]];
        const bool want = h->plan_kr[mode] >= 0 ? h->plan_kr[mode] == 1 : kr_auto(rows, h->nnz);
        p.kr = want && kr_fits(rows, R) ? 1 : 0;
    }
    return p;
}

void apply_plan(const ModePlan &p, MttkrpArgs &a) {
    a.depth = p.depth;
    for (int s = 0; s < kMaxModes; s++) a.level[s] = p.level[s];
    a.col_passes = p.passes;
}

// The tile order of a SEGMENTED mode (N <= 5): built once per handle and
// mode (sorted for the mode's fiber-factoring plan), on `st`, unless `st` is
// being captured (then the kernel sorts). force: also for another strategy
// (the batched MTTKRP reads every mode's tile order).
int ensure_tile_order(relate_handle_s *h, int mode, int R, cudaStream_t st, bool force = false) {
    if (h->d_tperm[mode] || h->nnz == 0 || h->N > 5) return RELATE_OK;
    if (!force && resolve_conflict(h, mode, R) != RELATE_CONFLICT_SEGMENTED) return RELATE_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return cuda_fail(e, "relate_mttkrp: capture status");
    if (cs != cudaStreamCaptureStatusNone) return RELATE_OK;
    MttkrpArgs a{};
    fill_stream_args(h, mode, a);
    const ModePlan plan = resolve_plan(h, mode, R);
    apply_plan(plan, a);
    h->tperm_depth[mode] = plan.depth;
    uint16_t *p = nullptr;
    if ((e = dalloc(&p, tperm_bytes(h->nnz), st)) != cudaSuccess) return cuda_fail(e, "relate_mttkrp: tile order");
    if ((e = launch_tile_order(a, h->KW, h->num_sms, p, st)) != cudaSuccess) {
        cudaFreeAsync(p, st);
        return cuda_fail(e, "relate_mttkrp: tile order");
    }
    h->d_tperm[mode] = p;
    return RELATE_OK;
}

// The launch arguments of one mode's MTTKRP of the handle.
void fill_run_args(relate_handle_s *h, int mode, void *const *factors, int R, void *out, MttkrpArgs &a);

// The Khatri-Rao table of the handle holds at least `bytes` (regrown outside
// a capture only); false: not available now.
bool ensure_kr(relate_handle_s *h, size_t bytes, cudaStream_t st) {
    if (h->kr_bytes >= bytes && h->d_kr) return true;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    if (h->d_kr) cudaFreeAsync(h->d_kr, st);
    h->d_kr = nullptr;
    h->kr_bytes = 0;
    h->kr_valid = false;
    if (dalloc(&h->d_kr, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        h->d_kr = nullptr;
        return false;
    }
    h->kr_bytes = bytes;
    return true;
}

// Bytes of the Khatri-Rao table mode `mode`'s plan fuses at rank R (0: none).
size_t kr_plan_bytes(const relate_handle_s *h, const ModePlan &p, int R) {
    if (!p.kr) return 0;
    return (size_t)(h->dims[p.level[p.depth - 1]] * h->dims[p.level[p.depth]]) * R * 8;
}

// reuse_kr: the handle's Khatri-Rao rows may be kept when they hold the same
// modes' factors (the caller clears kr_valid when one of them changes).
int run_mttkrp(relate_handle_s *h, int mode, void *const *factors, int R, void *out, cudaStream_t st,
               bool reuse_kr = false) {
    int rc0 = ensure_tile_order(h, mode, R, st);
    if (rc0) return rc0;
    MttkrpArgs a{};
    fill_run_args(h, mode, factors, R, out, a);
    const ModePlan plan = resolve_plan(h, mode, R);
    cudaError_t e;
    const int ka = plan.kr ? plan.level[plan.depth - 1] : 0, kb = plan.kr ? plan.level[plan.depth] : 0;
    // the table is built with 16-byte vector loads of both factors' rows
    if (plan.kr && a.depth == plan.depth && reinterpret_cast<uintptr_t>(factors[ka]) % 16 == 0 &&
        reinterpret_cast<uintptr_t>(factors[kb]) % 16 == 0 && ensure_kr(h, kr_plan_bytes(h, plan, R), st)) {
        const bool keep = reuse_kr && h->kr_valid && h->kr_a == ka && h->kr_b == kb && h->kr_R == R &&
                          h->kr_fa == factors[ka] && h->kr_fb == factors[kb];
        if (!keep) {
            if ((e = launch_kr_rows(factors[ka], factors[kb], h->dims[ka], h->dims[kb], R, h->factor_dtype, h->d_kr,
                                    st)) != cudaSuccess)
                return cuda_fail(e, "relate_mttkrp: Khatri-Rao rows");
            h->kr_a = ka;
            h->kr_b = kb;
            h->kr_R = R;
            h->kr_fa = factors[ka];
            h->kr_fb = factors[kb];
            h->kr_valid = true;
        }
        a.kr_table = h->d_kr;
        a.kr_mul = (uint32_t)h->dims[kb];
    }
    const int accb = mttkrp_acc_bytes(h->factor_dtype);
    e = cudaMemsetAsync(out, 0, h->dims[mode] * (size_t)R * accb, st);
    if (e != cudaSuccess) return cuda_fail(e, "relate_mttkrp memset");
    e = launch_mttkrp(a, h->KW, h->factor_dtype, h->val_dtype, h->smem_budget, h->num_sms, st);
    if (e != cudaSuccess) return cuda_fail(e, "relate_mttkrp launch");
    return RELATE_OK;
}

void fill_run_args(relate_handle_s *h, int mode, void *const *factors, int R, void *out, MttkrpArgs &a) {
    a.words = h->d_words;
    a.vals = h->d_vals;
    a.nnz = h->nnz;
    a.S = h->S;
    a.P = h->P;
    a.N = h->N;
    a.mode = mode;
    a.fields = h->fields;
    for (int k = 0; k < h->N; k++) a.factors[k] = factors[k];
    a.R = R;
    a.out = out;
    a.In = h->dims[mode];
    a.plo = h->d_plo;
    a.phi = h->d_phi;
    a.hot_rows = h->d_hot_rows[mode];
    a.maxcount = h->maxcount[mode];
    a.hot_scratch = h->d_hot_scratch;
    a.tperm = h->d_tperm[mode];
    if (fault_is("timeout")) {
        a.fault_skip_copy = 1;
        a.wait_cycles = 100000000LL;  // ~50 ms
    }
    a.err = h->d_err;
    a.strategy = resolve_conflict(h, mode, R);
    apply_plan(resolve_plan(h, mode, R), a);
    // a tile order sorted without factoring keeps the flat kernel
    if (h->tperm_depth[mode] == 0) a.depth = 0;
    a.vals_f64 = h->val_dtype == RELATE_F64;
}

// One mode of several handles (items) in the fewest launches: items that the
// batched kernel takes (its tile order built, vector path, N <= 5) are grouped
// by (N, key width, factor dtype), up to 24 per launch; the others run alone.
// Outputs are zeroed first.
struct BatchItemRef {
    relate_handle_s *h;
    int mode;
    void *const *factors;
    int R;
    void *out;
};

int run_mttkrp_batch(const BatchItemRef *items, int n, cudaStream_t st) {
    struct Group {
        int N, KW, fdt;
        std::vector<MttkrpArgs> args;
    };
    std::vector<Group> groups;
    cudaError_t e;
    int rc;
    int num_sms = 0;
    for (int i = 0; i < n; i++) {
        relate_handle_s *h = items[i].h;
        const int mode = items[i].mode, R = items[i].R;
        if ((rc = ensure_tile_order(h, mode, R, st, true)) != RELATE_OK) return rc;
        MttkrpArgs a{};
        fill_run_args(h, mode, items[i].factors, R, items[i].out, a);
        if (!batch_eligible(a, h->factor_dtype)) {
            if ((rc = run_mttkrp(h, mode, items[i].factors, R, items[i].out, st)) != RELATE_OK) return rc;
            continue;
        }
        const int accb = mttkrp_acc_bytes(h->factor_dtype);
        if ((e = cudaMemsetAsync(items[i].out, 0, h->dims[mode] * (size_t)R * accb, st)) != cudaSuccess)
            return cuda_fail(e, "relate_mttkrp_batch memset");
        num_sms = h->num_sms;
        Group *g = nullptr;
        for (auto &x : groups)
            if (x.N == h->N && x.KW == h->KW && x.fdt == h->factor_dtype) g = &x;
        if (!g) {
            groups.push_back(Group{h->N, h->KW, (int)h->factor_dtype, {}});
            g = &groups.back();
        }
        g->args.push_back(a);
    }
    for (const auto &g : groups)
        for (size_t b = 0; b < g.args.size(); b += kBatchItems) {
            const int cnt = (int)std::min(g.args.size() - b, (size_t)kBatchItems);
            if ((e = launch_mttkrp_batch(g.args.data() + b, cnt, g.KW, g.fdt, num_sms, st)) != cudaSuccess)
                return cuda_fail(e, "relate_mttkrp_batch launch");
        }
    return RELATE_OK;
}

// The steps of one ALS sweep, enqueued on the handle's stream (capturable).
// V of mode m (the other modes' Grams) runs on aux, forked from `st` once the
// Grams it reads are final: for mode 0 at the start of the iteration; for
// the later modes of the FP32/FP64 path right after the previous mode's
// normalised Gram, so that it overlaps that mode's factor store and this
// mode's MTTKRP (the BF16 path forms the Gram from the stored factor, so
// it forks at the start of the mode).
// The row pass A = M V^{-1} of mode update with the gram_timeout test hook
// applied (the FP64 row pass runs on the tensor cores too).
cudaError_t solve_checked(relate_handle_s *h, int64_t In, int R, cudaStream_t st) {
    const bool f = fault_is("gram_timeout");
    return launch_solve_rows(h->d_M, In, R, h->acc_dtype, h->d_Vinv, h->d_Vinv32, h->d_err, st, f ? 100000000LL : 0,
                             f ? 1 : 0, !f && dense_f64_small(In, R));
}

bool tc_path_of(const relate_handle_s *h, int R) { return h->factor_dtype == RELATE_BF16 && gram_tc_supported(R); }

cudaError_t fork_normal_eq(relate_handle_s *h, int R, int m) {
    const cudaStream_t st = h->stream;
    cudaError_t x;
    if ((x = cudaEventRecord(h->ev_g, st)) != cudaSuccess || (x = cudaStreamWaitEvent(h->aux, h->ev_g, 0)) != cudaSuccess ||
        (x = launch_normal_eq(h->d_G, h->N, m, R, h->d_Vinv, h->d_Vinv32, h->d_V, h->acc_dtype == RELATE_F64,
                              h->d_status, h->aux)) != cudaSuccess)
        return x;
    return cudaEventRecord(h->ev_v, h->aux);
}

// Before mode n's MTTKRP.
int mode_pre(relate_handle_s *h, int R, int n) {
    cudaError_t e;
    if ((n == 0 || tc_path_of(h, R)) && (e = fork_normal_eq(h, R, n)) != cudaSuccess)
        return cuda_fail(e, "relate_cpals: normal equations");
    return RELATE_OK;
}

// After mode n's MTTKRP (into h->d_M): A_n = M V^{-1}, lambda, the normalised
// factor and its Gram, the fit's inner products.
int mode_post(relate_handle_s *h, int R, int n, void *const *factors) {
    const cudaStream_t st = h->stream;
    if (n == h->kr_a || n == h->kr_b) h->kr_valid = false;  // A_n is rewritten below
    const int N = h->N;
    const int RR = R * R;
    const int64_t In = (int64_t)h->dims[n];
    const bool tc_path = tc_path_of(h, R);
    cudaError_t e;
    if ((e = cudaStreamWaitEvent(st, h->ev_v, 0)) != cudaSuccess) return cuda_fail(e, "relate_cpals: mode update");
    if (tc_path) {
        // lambda from Ahat's column norms, store the normalised BF16 factor,
        // then its Gram on the tensor cores (of the stored values)
        if ((e = solve_checked(h, In, R, st)) != cudaSuccess ||
            (e = launch_colnorms((const float *)h->d_M, In, R, h->d_scratch, h->d_lambda, st)) != cudaSuccess ||
            (e = launch_scale_store(h->d_M, In, R, h->acc_dtype, h->d_lambda, factors[n], h->factor_dtype, st)) !=
                cudaSuccess ||
            (e = gram_checked(factors[n], In, R, RELATE_BF16, h->d_scratch, h->d_G + n * RR, h->d_err, st)) !=
                cudaSuccess ||
            (e = launch_inner_from_gram(h->d_V, h->d_G + n * RR, h->d_lambda, R, h->d_inner, st)) != cudaSuccess)
            return cuda_fail(e, "relate_cpals: mode update");
        return RELATE_OK;
    }
    // the row pass and the Gram of its result (tensor cores), then finish,
    // have consumed V^{-1} and V: the next mode's normal equations may
    // overwrite them
    if ((e = solve_checked(h, In, R, st)) != cudaSuccess ||
        (e = gram_checked(h->d_M, In, R, h->acc_dtype, h->d_scratch, h->d_G + n * RR, h->d_err, st, true)) != cudaSuccess ||
        (e = launch_finish_mode(h->d_V, R, h->d_lambda, h->d_G + n * RR, h->d_inner, st)) != cudaSuccess)
        return cuda_fail(e, "relate_cpals: mode update");
    if (n + 1 < N && (e = fork_normal_eq(h, R, n + 1)) != cudaSuccess)
        return cuda_fail(e, "relate_cpals: normal equations");
    if ((e = launch_scale_store(h->d_M, In, R, h->acc_dtype, h->d_lambda, factors[n], h->factor_dtype, st)) !=
        cudaSuccess)
        return cuda_fail(e, "relate_cpals: mode update");
    return RELATE_OK;
}

// After the last mode: the fit, recorded on the device (d_trace) and copied
// with the status words to the pinned host words fit / status.
int iteration_fit(relate_handle_s *h, int R, double *p_fit, int *p_stat, double *d_trace, int *d_counter) {
    const cudaStream_t st = h->stream;
    cudaError_t e;
    if ((e = launch_fit(h->d_G, h->N, R, h->d_lambda, h->d_inner, h->d_normX2 + (h->reduce_fn ? 1 : 0), h->d_fit,
                        st)) != cudaSuccess ||
        (d_trace && (e = launch_record_fit(h->d_fit, h->d_status, d_trace, d_counter, st)) != cudaSuccess) ||
        (e = cudaMemcpyAsync(p_fit, h->d_fit, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(p_stat, h->d_status, 2 * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(p_stat + 2, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "relate_cpals: fit");
    return RELATE_OK;
}

// One ALS sweep over all modes plus the fit, enqueued on the handle's stream
// (capturable): results land in the pinned host words fit / status.
int cpals_iteration(relate_handle_s *h, int R, void *const *factors, double *p_fit, int *p_stat,
                    double *d_trace = nullptr, int *d_counter = nullptr) {
    int rc;
    h->kr_valid = false;  // a captured iteration is replayed after other iterations changed every factor
    for (int n = 0; n < h->N; n++) {
        if ((rc = mode_pre(h, R, n)) != RELATE_OK ||
            (rc = run_mttkrp(h, n, factors, R, h->d_M, h->stream, true)) != RELATE_OK)
            return rc;
        // sharded: the shards' partial MTTKRPs are summed before the update
        if (h->reduce_fn && h->reduce_fn(h->d_M, (int64_t)h->dims[n] * R, h->acc_dtype, h->stream, h->reduce_user) != 0)
            return fail(RELATE_ERR_CUDA, "relate_cpals: the reduce hook failed (mode %d)", n);
        if ((rc = mode_post(h, R, n, factors)) != RELATE_OK) return rc;
    }
    return iteration_fit(h, R, p_fit, p_stat, d_trace, d_counter);
}

}  // namespace

extern "C" {

void relate_params_default(relate_params_t *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->bit_order = nullptr;
    p->bit_order_len = 0;
    p->partition_size = 0;
    for (int m = 0; m < RELATE_MAX_MODES; m++) p->conflict[m] = RELATE_CONFLICT_AUTO;
    p->val_dtype = RELATE_F32;
    p->factor_dtype = RELATE_F32;
    p->acc_dtype = RELATE_F32;
    p->coords_on_device = 0;
    p->stream = nullptr;
    p->smem_budget = 0;
}

int relate_encode(const uint32_t *coords, const void *vals, const uint64_t *dims, int nmodes, int64_t nnz,
                  const relate_params_t *params, relate_handle_t *out) {
    g_err[0] = 0;
    if (!out) return fail(RELATE_ERR_INVALID_ARG, "relate_encode: out is NULL");
    *out = nullptr;
    relate_params_t defaults;
    relate_params_default(&defaults);
    const relate_params_t *p = params ? params : &defaults;
    if (nmodes < 2 || nmodes > RELATE_MAX_MODES)
        return fail(RELATE_ERR_INVALID_ARG, "relate_encode: nmodes=%d not in [2, %d]", nmodes, RELATE_MAX_MODES);
    if (!dims) return fail(RELATE_ERR_INVALID_ARG, "relate_encode: dims is NULL");
    if (nnz < 0 || nnz > (int64_t)0xffffffffLL)
        return fail(RELATE_ERR_INVALID_ARG, "relate_encode: nnz=%lld out of range", (long long)nnz);
    if (nnz > 0 && (!coords || !vals)) return fail(RELATE_ERR_INVALID_ARG, "relate_encode: coords/vals NULL");
    if (p->val_dtype != RELATE_F64 && p->val_dtype != RELATE_F32)
        return fail(RELATE_ERR_INVALID_ARG, "relate_encode: val_dtype must be F64 or F32");
    if (!valid_precision(p->factor_dtype, p->acc_dtype))
        return fail(RELATE_ERR_INVALID_ARG, "relate_encode: factor/acc dtype pair not supported");
    if (p->partition_size < 0) return fail(RELATE_ERR_INVALID_ARG, "relate_encode: partition_size < 0");
    for (int m = 0; m < nmodes; m++)
        if (p->conflict[m] < RELATE_CONFLICT_AUTO || p->conflict[m] > RELATE_CONFLICT_PRIVATIZED)
            return fail(RELATE_ERR_INVALID_ARG, "relate_encode: bad conflict strategy for mode %d", m);

    relate_handle_s *h = new (std::nothrow) relate_handle_s();
    if (!h) return fail(RELATE_ERR_OOM, "relate_encode: host allocation");
    h->N = nmodes;
    h->nnz = nnz;
    h->lp = 0;
    for (int m = 0; m < nmodes; m++) {
        if (dims[m] < 1 || dims[m] > ((uint64_t)1 << 32)) {
            delete h;
            return fail(RELATE_ERR_INVALID_ARG, "relate_encode: dims[%d]=%llu not in [1, 2^32]", m,
                        (unsigned long long)dims[m]);
        }
        h->dims[m] = dims[m];
        h->lbits[m] = bits_for(dims[m]);
        h->lp += h->lbits[m];
    }
    if (h->lp > RELATE_MAX_KEY_BITS) {
        delete h;
        return fail(RELATE_ERR_KEY_TOO_WIDE, "relate_encode: l(p)=%d > 128", h->lp);
    }
    // bit order: explicit (validated by the masking rule) or ALTO default
    if (p->bit_order) {
        if (p->bit_order_len != h->lp) {
            delete h;
            return fail(RELATE_ERR_BAD_BIT_ORDER, "relate_encode: bit order length %d != l(p) %d", p->bit_order_len,
                        h->lp);
        }
        int used[kMaxModes] = {};
        for (int t = 0; t < h->lp; t++) {
            const int m = p->bit_order[t];
            if (m < 0 || m >= nmodes) {
                delete h;
                return fail(RELATE_ERR_BAD_BIT_ORDER, "relate_encode: bit order entry %d names mode %d", t, m);
            }
            used[m]++;
            h->order[t] = (int8_t)m;
        }
        for (int m = 0; m < nmodes; m++)
            if (used[m] != h->lbits[m]) {
                delete h;
                return fail(RELATE_ERR_BAD_BIT_ORDER, "relate_encode: mode %d appears %d times, needs l(n)=%d", m,
                            used[m], h->lbits[m]);
            }
    } else {
        int rank[kMaxModes], left[kMaxModes];
        for (int m = 0; m < nmodes; m++) rank[m] = m;
        for (int a = 0; a < nmodes; a++)  // stable order by (l(n), id)
            for (int b = a + 1; b < nmodes; b++)
                if (h->lbits[rank[b]] < h->lbits[rank[a]]) {
                    int t = rank[a];
                    rank[a] = rank[b];
                    rank[b] = t;
                } else if (h->lbits[rank[b]] == h->lbits[rank[a]] && rank[b] < rank[a]) {
                    int t = rank[a];
                    rank[a] = rank[b];
                    rank[b] = t;
                }
        for (int m = 0; m < nmodes; m++) left[m] = h->lbits[m];
        int t = 0;
        while (t < h->lp)
            for (int a = 0; a < nmodes; a++)
                if (left[rank[a]] > 0) {
                    h->order[t++] = (int8_t)rank[a];
                    left[rank[a]]--;
                }
    }
    h->KW = h->lp <= 32 ? 1 : h->lp <= 64 ? 2 : 4;
    build_runs(h);
    h->S = p->partition_size > 0 ? p->partition_size : 4096;
    // the shard of the sorted stream this handle keeps (all of it unsharded)
    int64_t shard_lo = 0, shard_hi = nnz;
    if (p->shard_count > 1) {
        if (p->shard_rank < 0 || p->shard_rank >= p->shard_count) {
            delete h;
            return fail(RELATE_ERR_INVALID_ARG, "relate_encode: shard_rank %d not in [0, %d)", p->shard_rank,
                        p->shard_count);
        }
        relate_shard_range(nnz, p->shard_rank, p->shard_count, &shard_lo, &shard_hi);
    }
    const int64_t ns = shard_hi - shard_lo;  // nonzeros kept
    h->nnz_total = nnz;
    h->shard_lo = shard_lo;
    h->nnz = ns;
    h->P = (ns + h->S - 1) / h->S;
    h->val_dtype = p->val_dtype;
    h->factor_dtype = p->factor_dtype;
    h->acc_dtype = p->acc_dtype;
    for (int m = 0; m < kMaxModes; m++) h->conflict[m] = m < nmodes ? p->conflict[m] : RELATE_CONFLICT_AUTO;
    h->stream = (cudaStream_t)p->stream;

    cudaError_t e;
    if ((e = cudaGetDevice(&h->device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device)) !=
            cudaSuccess) {
        delete h;
        return cuda_fail(e, "relate_encode: device query");
    }
    h->smem_budget = h->smem_optin - 2048;
    if (p->smem_budget > 0 && p->smem_budget < h->smem_budget) h->smem_budget = p->smem_budget;

    const cudaStream_t st = h->stream;
    const int vb = h->val_dtype == RELATE_F64 ? 8 : 4;
    const size_t kb = 4u * h->KW;
    const int N = nmodes;
    int rc = RELATE_OK;
    {
        AsyncBufs tmp{st, {}};
        // joins the value copy into `st` before the temporaries are released,
        // on every path (declared after `tmp`, so it is destroyed first)
        struct ValsJoin {
            relate_handle_s *h;
            cudaStream_t st;
            bool pending = false;
            cudaError_t join() {
                pending = false;
                return cudaStreamWaitEvent(st, h->ev_v, 0);
            }
            ~ValsJoin() {
                if (pending) cudaStreamWaitEvent(st, h->ev_v, 0);
            }
        } vals_join{h, st};
        void *d_coords = nullptr, *d_vin = nullptr, *keys = nullptr, *keys_alt = nullptr, *idx = nullptr,
             *idx_alt = nullptr, *sort_tmp = nullptr, *d_dims = nullptr, *d_small = nullptr;
        const size_t sort_bytes = radix_sort_temp_bytes(nnz);
        // persistent encoding arrays
        // 64 bytes of tail padding: tile copies round their size up to 16 bytes
        if ((e = dalloc(&h->d_words, words_bytes(ns, kb), st)) != cudaSuccess ||
            (e = dalloc(&h->d_vals, vals_bytes(ns, vb), st)) != cudaSuccess ||
            (e = dalloc((void **)&h->d_plo, bounds_bytes(h->P, N), st)) != cudaSuccess ||
            (e = dalloc((void **)&h->d_phi, bounds_bytes(h->P, N), st)) != cudaSuccess ||
            (e = dalloc((void **)&h->d_normX2, 64, st)) != cudaSuccess ||
            (e = dalloc(&h->d_hot_scratch, kHotScratchBytes, st)) != cudaSuccess ||
            (e = dalloc((void **)&h->d_err, 16, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(h->d_err, 0, 16, st)) != cudaSuccess) {
            rc = cuda_fail(e, "relate_encode: allocation");
            goto done;
        }
        for (int m = 0; m < N; m++)
            if ((e = dalloc((void **)&h->d_counts[m], h->dims[m] * 4, st)) != cudaSuccess ||
                (e = dalloc((void **)&h->d_hot_rows[m], kHotMax * 4, st)) != cudaSuccess) {
                rc = cuda_fail(e, "relate_encode: allocation");
                goto done;
            }
        if ((e = tmp.alloc(&keys, nnz * kb)) != cudaSuccess || (e = tmp.alloc(&keys_alt, nnz * kb)) != cudaSuccess ||
            (e = tmp.alloc(&idx, nnz * 4)) != cudaSuccess || (e = tmp.alloc(&idx_alt, nnz * 4)) != cudaSuccess ||
            (e = tmp.alloc(&sort_tmp, sort_bytes)) != cudaSuccess || (e = tmp.alloc(&d_dims, 64)) != cudaSuccess ||
            (e = tmp.alloc(&d_small, kSmallBytes)) != cudaSuccess) {
            rc = cuda_fail(e, "relate_encode: temporary allocation");
            goto done;
        }
        const uint32_t *c_dev = coords;
        const void *v_dev = vals;
        if (!p->coords_on_device && nnz > 0) {
            if ((e = tmp.alloc(&d_coords, (size_t)N * nnz * 4)) != cudaSuccess ||
                (e = tmp.alloc(&d_vin, (size_t)nnz * vb)) != cudaSuccess) {
                rc = cuda_fail(e, "relate_encode: input staging");
                goto done;
            }
            if ((e = cudaMemcpyAsync(d_coords, coords, (size_t)N * nnz * 4, cudaMemcpyHostToDevice, st)) !=
                cudaSuccess) {
                rc = cuda_fail(e, "relate_encode: host-to-device copy");
                goto done;
            }
            c_dev = (const uint32_t *)d_coords;
            v_dev = d_vin;
        }
        // d_small layout: [0] err flag (u32 in a u64 slot) | runs[8] | summary[2*8] | sumsq partials
        uint32_t *d_err = (uint32_t *)d_small;
        unsigned long long *d_runs = (unsigned long long *)d_small + 1;
        unsigned long long *d_summ = d_runs + kMaxModes;
        double *d_part = (double *)(d_summ + 2 * kMaxModes);
        if ((e = cudaMemsetAsync(d_small, 0, 8 * (1 + 3 * kMaxModes), st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(d_dims, h->dims, sizeof(uint64_t) * N, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
            rc = cuda_fail(e, "relate_encode: setup");
            goto done;
        }
        for (int m = 0; m < N; m++)
            if ((e = cudaMemsetAsync(h->d_counts[m], 0, h->dims[m] * 4, st)) != cudaSuccess) {
                rc = cuda_fail(e, "relate_encode: setup");
                goto done;
            }
        // byte tables of the two bit permutations (coordinates -> p, p -> word)
        std::vector<unsigned char> host_luts(2 * kLutMaxBytes, 0);
        ByteLuts key_luts{}, word_luts{};
        build_key_luts(N, h->lbits, h->order, h->lp, h->KW, key_luts, host_luts.data());
        build_word_luts(N, h->runs.field_off, h->order, h->lp, h->KW, word_luts, host_luts.data() + kLutMaxBytes);
        void *d_luts = nullptr;
        if ((e = tmp.alloc(&d_luts, 2 * (size_t)kLutMaxBytes)) != cudaSuccess ||
            (e = cudaMemcpyAsync(d_luts, host_luts.data(), 2 * kLutMaxBytes, cudaMemcpyHostToDevice, st)) !=
                cudaSuccess) {
            rc = cuda_fail(e, "relate_encode: permutation tables");
            goto done;
        }
        if (d_vin) {
            // the values are first needed by the gather after the sort: they
            // cross on the second stream behind the coordinates and the
            // tables (copies share the copy engine and the link), while the
            // keys are built and sorted
            if ((e = ensure_aux(h)) != cudaSuccess || (e = cudaEventRecord(h->ev_g, st)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(h->aux, h->ev_g, 0)) != cudaSuccess) {
                rc = cuda_fail(e, "relate_encode: copy stream");
                goto done;
            }
            if ((e = cudaMemcpyAsync(d_vin, vals, (size_t)nnz * vb, cudaMemcpyHostToDevice, h->aux)) == cudaSuccess)
                vals_join.pending = true;
            if (e != cudaSuccess || (e = cudaEventRecord(h->ev_v, h->aux)) != cudaSuccess) {
                rc = cuda_fail(e, "relate_encode: host-to-device copy");
                goto done;
            }
        }
        bool in_alt = false;
        if ((e = launch_build_keys_lut(h->KW, c_dev, (const uint64_t *)d_dims, nnz, N, key_luts, d_luts, keys,
                                       (uint32_t *)idx, d_err, st)) != cudaSuccess ||
            (e = radix_sort_pairs(h->KW, keys, (uint32_t *)idx, keys_alt, (uint32_t *)idx_alt, nnz, h->lp, sort_tmp,
                                  sort_bytes, st, &in_alt)) != cudaSuccess) {
            rc = cuda_fail(e, "relate_encode: key build / sort");
            goto done;
        }
        // the handle keeps the shard [shard_lo, shard_hi) of the sorted stream
        void *skeys = (unsigned char *)(in_alt ? keys_alt : keys) + (size_t)shard_lo * kb;
        uint32_t *sperm = (uint32_t *)(in_alt ? idx_alt : idx) + shard_lo;
        if ((e = dalloc((void **)&h->d_perm, perm_bytes(ns), st)) != cudaSuccess ||
            (ns && (e = cudaMemcpyAsync(h->d_perm, sperm, ns * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) ||
            (e = launch_make_words_lut(h->KW, skeys, ns, word_luts, (const unsigned char *)d_luts + kLutMaxBytes,
                                       h->d_words, st)) != cudaSuccess ||
            (vals_join.pending && (e = vals_join.join()) != cudaSuccess) ||
            (e = launch_gather(v_dev, sperm, ns, vb, h->d_vals, st)) != cudaSuccess) {
            rc = cuda_fail(e, "relate_encode: words / gather");
            goto done;
        }
        CountPtrs cp{};
        for (int m = 0; m < N; m++) {
            cp.p[m] = h->d_counts[m];
            cp.len[m] = h->dims[m];
        }
        if ((e = launch_partition_stats(h->KW, h->d_words, ns, N, h->fields, h->S, h->d_plo, h->d_phi, d_runs, cp,
                                        st)) != cudaSuccess) {
            rc = cuda_fail(e, "relate_encode: partition statistics");
            goto done;
        }
        for (int m = 0; m < N; m++)
            if ((e = launch_hist_summary(h->d_counts[m], h->dims[m], d_summ + 2 * m, st)) != cudaSuccess) {
                rc = cuda_fail(e, "relate_encode: histogram summary");
                goto done;
            }
        if ((e = launch_sum_squares(h->d_vals, ns, vb, d_part, h->d_normX2, st)) != cudaSuccess) {
            rc = cuda_fail(e, "relate_encode: norm");
            goto done;
        }
        {
            uint64_t maxI = 0;
            for (int m = 0; m < N; m++) maxI = h->dims[m] > maxI ? h->dims[m] : maxI;
            void *hot_tmp = nullptr;
            if ((e = tmp.alloc(&hot_tmp, hot_table_temp_bytes(maxI))) != cudaSuccess) {
                rc = cuda_fail(e, "relate_encode: hot-row table");
                goto done;
            }
            for (int m = 0; m < N; m++)
                if ((e = launch_hot_table(h->d_counts[m], h->dims[m], h->d_hot_rows[m], hot_tmp, st)) !=
                    cudaSuccess) {
                    rc = cuda_fail(e, "relate_encode: hot-row table");
                    goto done;
                }
        }
        unsigned long long host_small[1 + 3 * kMaxModes];
        if ((e = cudaMemcpyAsync(host_small, d_small, sizeof(host_small), cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            rc = cuda_fail(e, "relate_encode: statistics to host");
            goto done;
        }
        if ((uint32_t)host_small[0] != 0) {
            rc = fail(RELATE_ERR_COORD_OUT_OF_RANGE, "relate_encode: a coordinate is >= its mode length");
            goto done;
        }
        for (int m = 0; m < N; m++) {
            h->runs_n[m] = host_small[1 + m];
            h->distinct[m] = host_small[1 + kMaxModes + 2 * m];
            h->maxcount[m] = host_small[1 + kMaxModes + 2 * m + 1];
        }
    }
done:
    if (rc != RELATE_OK) {
        delete h;
        return rc;
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) {
        delete h;
        return cuda_fail(e, "relate_encode: release temporaries");
    }
    *out = h;
    return RELATE_OK;
}

int relate_mttkrp(relate_handle_t h, int mode, void *const *factors, int R, void *out, void *stream) {
    g_err[0] = 0;
    if (!h) return fail(RELATE_ERR_INVALID_ARG, "relate_mttkrp: NULL handle");
    if (mode < 0 || mode >= h->N) return fail(RELATE_ERR_INVALID_ARG, "relate_mttkrp: mode %d out of range", mode);
    if (R < 1 || R > RELATE_MAX_RANK) return fail(RELATE_ERR_INVALID_ARG, "relate_mttkrp: R=%d not in [1, 64]", R);
    if (!factors || !out) return fail(RELATE_ERR_INVALID_ARG, "relate_mttkrp: NULL factors/out");
    for (int k = 0; k < h->N; k++)
        if (k != mode && !factors[k]) return fail(RELATE_ERR_INVALID_ARG, "relate_mttkrp: factors[%d] is NULL", k);
    return run_mttkrp(h, mode, factors, R, out, (cudaStream_t)stream);
}

int relate_cpals(relate_handle_t h, int R, int iters, double tol, void *const *factors, double *lambda,
                 relate_cpals_info_t *info) {
    g_err[0] = 0;
    if (!h) return fail(RELATE_ERR_INVALID_ARG, "relate_cpals: NULL handle");
    if (R < 1 || R > RELATE_MAX_RANK) return fail(RELATE_ERR_INVALID_ARG, "relate_cpals: R=%d not in [1, 64]", R);
    if (iters < 0 || !factors || !lambda) return fail(RELATE_ERR_INVALID_ARG, "relate_cpals: bad iters/factors/lambda");
    for (int k = 0; k < h->N; k++)
        if (!factors[k]) return fail(RELATE_ERR_INVALID_ARG, "relate_cpals: factors[%d] is NULL", k);
    int rc = ensure_ws(h, R);
    if (rc) return rc;
    const cudaStream_t st = h->stream;
    const int N = h->N;
    size_t kr_need = 0;
    for (int n = 0; n < N; n++) {  // before any capture: tile orders are built once
        if ((rc = ensure_tile_order(h, n, R, st)) != RELATE_OK) return rc;
        const size_t b = kr_plan_bytes(h, resolve_plan(h, n, R), R);
        kr_need = b > kr_need ? b : kr_need;
    }
    if (kr_need) ensure_kr(h, kr_need, st);  // else the modes run unfused
    const int RR = R * R;
    cudaError_t e;
    if ((e = cudaMemsetAsync(h->d_status, 0, 64, st)) != cudaSuccess) return cuda_fail(e, "relate_cpals: setup");
    if (h->reduce_fn) {
        // sharded: ||X||^2 summed over the shards into d_normX2[1], which the
        // fit reads
        if ((e = cudaMemcpyAsync(h->d_normX2 + 1, h->d_normX2, sizeof(double), cudaMemcpyDeviceToDevice, st)) !=
            cudaSuccess)
            return cuda_fail(e, "relate_cpals: norm");
        if (h->reduce_fn(h->d_normX2 + 1, 1, RELATE_F64, st, h->reduce_user) != 0)
            return fail(RELATE_ERR_CUDA, "relate_cpals: the reduce hook failed (norm)");
    }
    for (int k = 0; k < N; k++)
        if ((e = gram_checked(factors[k], (int64_t)h->dims[k], R, h->factor_dtype, h->d_scratch, h->d_G + k * RR,
                              h->d_err, st, true)) != cudaSuccess)
            return cuda_fail(e, "relate_cpals: initial Gram");
    double prev = 0.0, fit = 0.0;
    int done = 0;
    int hstatus[3] = {0, 0, 0};
    if (!h->h_pinned && !(h->h_pinned = g_pinned.get()))
        return fail(RELATE_ERR_OOM, "relate_cpals: pinned host words");
    double *p_fit = h->h_pinned;
    int *p_stat = reinterpret_cast<int *>(h->h_pinned + 1);  // status[0], status[1], err
    cudaGraphExec_t gexec = nullptr;
    // the legacy default stream cannot be captured: graph mode needs a stream;
    // a reduce hook runs host code between the modes, so sharded runs take
    // the plain path
    const bool graph = h->use_graph && st != nullptr && iters > 0 && !h->reduce_fn;
    // graph mode with a fixed iteration count (tol <= 0): the iterations are
    // replayed back to back and the host synchronises once, at the end; each
    // replay records its fit on the device
    const bool no_sync = graph && !(tol > 0.0);
    double *d_trace = nullptr;
    int *d_counter = nullptr;
    if (no_sync) {
        if ((e = dalloc(&d_trace, sizeof(double) * (size_t)iters + 16, st)) != cudaSuccess ||
            (e = dalloc(&d_counter, 16, st)) != cudaSuccess || (e = cudaMemsetAsync(d_counter, 0, 16, st)) != cudaSuccess) {
            if (d_trace) cudaFreeAsync(d_trace, st);
            return cuda_fail(e, "relate_cpals: fit trace");
        }
    }
    auto free_trace = [&]() {
        if (d_trace) cudaFreeAsync(d_trace, st);
        if (d_counter) cudaFreeAsync(d_counter, st);
        d_trace = nullptr;
        d_counter = nullptr;
    };
    if (graph) {
        cudaGraph_t g = nullptr;
        if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
            free_trace();
            return cuda_fail(e, "relate_cpals: begin capture");
        }
        rc = cpals_iteration(h, R, factors, p_fit, p_stat, d_trace, d_counter);
        cudaError_t e2 = cudaStreamEndCapture(st, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            free_trace();
            return rc;
        }
        if (e2 != cudaSuccess) {
            free_trace();
            return cuda_fail(e2, "relate_cpals: end capture");
        }
        // keep the captured per-node priorities (the normal equations' stream)
        e = cudaGraphInstantiate(&gexec, g, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            free_trace();
            return cuda_fail(e, "relate_cpals: graph instantiate");
        }
    }
    if (no_sync) {
        for (int it = 1; it <= iters; it++)
            if ((e = cudaGraphLaunch(gexec, st)) != cudaSuccess) {
                cudaGraphExecDestroy(gexec);
                cudaStreamSynchronize(st);
                free_trace();
                return cuda_fail(e, "relate_cpals: graph launch");
            }
        std::vector<double> trace((size_t)iters);
        int counter[4] = {0, 0, 0, 0};
        if ((e = cudaMemcpyAsync(trace.data(), d_trace, sizeof(double) * iters, cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(counter, d_counter, 2 * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            cudaGraphExecDestroy(gexec);
            free_trace();
            return cuda_fail(e, "relate_cpals: fit trace to host");
        }
        cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        free_trace();
        // the last replay copied the status words to the pinned slots
        hstatus[0] = p_stat[0];
        hstatus[1] = p_stat[1];
        hstatus[2] = p_stat[2];
        // after a NOT_PD iteration the later ones ran on zeroed normal
        // equations: report the fit and the count of the failing iteration
        done = counter[1] > 0 ? counter[1] : iters;
        fit = trace[(size_t)done - 1];
        if (info && info->fit_trace)
            for (int k = 0; k < done; k++) info->fit_trace[k] = trace[(size_t)k];
        if (hstatus[2]) {
            cudaMemsetAsync(h->d_err, 0, 16, st);
            if (info) {
                info->fit = fit;
                info->iters = done;
                info->status = RELATE_ERR_TIMEOUT;
            }
            return fail(RELATE_ERR_TIMEOUT, "relate_cpals: a bounded device wait timed out");
        }
    }
    for (int it = 1; it <= iters && !no_sync; it++) {
        if (graph) {
            if ((e = cudaGraphLaunch(gexec, st)) != cudaSuccess) {
                cudaGraphExecDestroy(gexec);
                return cuda_fail(e, "relate_cpals: graph launch");
            }
        } else if ((rc = cpals_iteration(h, R, factors, p_fit, p_stat)) != RELATE_OK) {
            return rc;
        }
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) {
            if (gexec) cudaGraphExecDestroy(gexec);
            return cuda_fail(e, "relate_cpals: fit to host");
        }
        fit = *p_fit;
        hstatus[0] = p_stat[0];
        hstatus[1] = p_stat[1];
        hstatus[2] = p_stat[2];
        done = it;
        if (info && info->fit_trace) info->fit_trace[it - 1] = fit;
        if (hstatus[2]) {
            if (gexec) cudaGraphExecDestroy(gexec);
            cudaMemsetAsync(h->d_err, 0, 16, st);
            if (info) {
                info->fit = fit;
                info->iters = done;
                info->status = RELATE_ERR_TIMEOUT;
            }
            return fail(RELATE_ERR_TIMEOUT, "relate_cpals: a bounded device wait timed out (iteration %d)", it);
        }
        if (hstatus[1]) break;
        if (it > 1 && (fit - prev < tol && prev - fit < tol)) break;
        prev = fit;
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    // lambda may be host or device memory: the copy's direction follows from
    // the unified address space
    if ((e = cudaMemcpyAsync(lambda, h->d_lambda, sizeof(double) * R, cudaMemcpyDefault, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "relate_cpals: lambda to host");
    rc = hstatus[1] ? fail(RELATE_ERR_NOT_PD, "relate_cpals: normal equations not positive definite") : RELATE_OK;
    if (info) {
        info->fit = fit;
        info->iters = done;
        info->status = rc;
        info->ridge_retries = hstatus[0];
    }
    return rc;
}

int relate_mttkrp_batch(const relate_mttkrp_item_t *items, int nitems, void *stream) {
    g_err[0] = 0;
    if (nitems < 0 || (nitems > 0 && !items)) return fail(RELATE_ERR_INVALID_ARG, "relate_mttkrp_batch: bad item list");
    std::vector<BatchItemRef> refs;
    refs.reserve(nitems);
    for (int i = 0; i < nitems; i++) {
        const relate_mttkrp_item_t &it = items[i];
        relate_handle_s *h = it.h;
        if (!h || it.mode < 0 || it.mode >= h->N || it.R < 1 || it.R > RELATE_MAX_RANK || !it.factors || !it.out)
            return fail(RELATE_ERR_INVALID_ARG, "relate_mttkrp_batch: bad item %d", i);
        for (int k = 0; k < h->N; k++)
            if (k != it.mode && !it.factors[k])
                return fail(RELATE_ERR_INVALID_ARG, "relate_mttkrp_batch: item %d: factors[%d] is NULL", i, k);
        refs.push_back(BatchItemRef{h, it.mode, it.factors, it.R, it.out});
    }
    return run_mttkrp_batch(refs.data(), nitems, (cudaStream_t)stream);
}

int relate_cpals_batch(relate_handle_t const *hs, int n, const int *R, int iters, double tol,
                       void *const *const *factors, double *const *lambdas, const double *prev_fit,
                       relate_cpals_info_t *infos, void *stream) {
    g_err[0] = 0;
    if (n < 0 || (n > 0 && (!hs || !R || !factors || !lambdas)) || iters < 0)
        return fail(RELATE_ERR_INVALID_ARG, "relate_cpals_batch: bad argument");
    const cudaStream_t st = (cudaStream_t)stream;
    if (n > 0 && !st) return fail(RELATE_ERR_INVALID_ARG, "relate_cpals_batch: needs a non-default stream");
    for (int p = 0; p < n; p++) {
        if (!hs[p] || R[p] < 1 || R[p] > RELATE_MAX_RANK || !factors[p] || !lambdas[p])
            return fail(RELATE_ERR_INVALID_ARG, "relate_cpals_batch: bad problem %d", p);
        for (int k = 0; k < hs[p]->N; k++)
            if (!factors[p][k]) return fail(RELATE_ERR_INVALID_ARG, "relate_cpals_batch: problem %d factors[%d] NULL", p, k);
        for (int q = 0; q < p; q++)
            if (hs[q] == hs[p]) return fail(RELATE_ERR_INVALID_ARG, "relate_cpals_batch: handle %d repeated", p);
        if (hs[p]->reduce_fn)
            return fail(RELATE_ERR_UNSUPPORTED, "relate_cpals_batch: problem %d is sharded (use relate_cpals)", p);
    }
    // every problem runs on `st` for this call
    std::vector<cudaStream_t> saved(n);
    for (int p = 0; p < n; p++) {
        saved[p] = hs[p]->stream;
        hs[p]->stream = st;
    }
    struct Restore {
        relate_handle_t const *hs;
        std::vector<cudaStream_t> &saved;
        ~Restore() {
            for (size_t p = 0; p < saved.size(); p++) hs[p]->stream = saved[p];
        }
    } restore{hs, saved};
    int rc;
    cudaError_t e;
    int maxN = 0;
    for (int p = 0; p < n; p++) {
        relate_handle_s *h = hs[p];
        if ((rc = ensure_ws(h, R[p])) != RELATE_OK) return rc;
        for (int m = 0; m < h->N; m++)  // before any capture
            if ((rc = ensure_tile_order(h, m, R[p], st, true)) != RELATE_OK) return rc;
        if ((e = cudaMemsetAsync(h->d_status, 0, 64, st)) != cudaSuccess) return cuda_fail(e, "relate_cpals_batch: setup");
        const int RR = R[p] * R[p];
        for (int k = 0; k < h->N; k++)
            if ((e = gram_checked(factors[p][k], (int64_t)h->dims[k], R[p], h->factor_dtype, h->d_scratch,
                                  h->d_G + k * RR, h->d_err, st, true)) != cudaSuccess)
                return cuda_fail(e, "relate_cpals_batch: initial Gram");
        if (!h->h_pinned && !(h->h_pinned = g_pinned.get()))
            return fail(RELATE_ERR_OOM, "relate_cpals_batch: pinned host words");
        maxN = h->N > maxN ? h->N : maxN;
        if (infos) {
            infos[p].fit = 0.0;
            infos[p].iters = 0;
            infos[p].status = RELATE_OK;
            infos[p].ridge_retries = 0;
        }
    }
    std::vector<int> active;
    for (int p = 0; p < n; p++) active.push_back(p);
    std::vector<double> prev(n, 0.0);
    std::vector<int> have_prev(n, 0);
    for (int p = 0; p < n; p++)
        if (prev_fit && prev_fit[p] == prev_fit[p]) {  // not NaN
            prev[p] = prev_fit[p];
            have_prev[p] = 1;
        }
    std::vector<int> status(n, RELATE_OK);
    // Each problem's dense steps (normal equations, row pass, Gram, fit) run
    // on a branch stream of its own, forked from `st` after each batched
    // MTTKRP and joined before the next, so that in the captured graph the
    // problems' small kernels are independent nodes that run side by side.
    struct Branches {
        std::vector<cudaStream_t> s;
        std::vector<cudaEvent_t> ev;
        cudaEvent_t fork = nullptr;
        ~Branches() {
            for (cudaStream_t x : s) cudaStreamDestroy(x);
            for (cudaEvent_t x : ev) cudaEventDestroy(x);
            if (fork) cudaEventDestroy(fork);
        }
    } br;
    if (n > 0 && (e = cudaEventCreateWithFlags(&br.fork, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "relate_cpals_batch: branch streams");
    for (int p = 0; p < n; p++) {
        cudaStream_t x = nullptr;
        cudaEvent_t v = nullptr;
        if ((e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "relate_cpals_batch: branch streams");
        br.s.push_back(x);
        if ((e = cudaEventCreateWithFlags(&v, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "relate_cpals_batch: branch streams");
        br.ev.push_back(v);
    }
    // runs step(p) for every active problem with s < N on its branch, between a fork from and a join into `st`
    auto on_branches = [&](int s, auto step) -> int {
        cudaError_t x;
        if ((x = cudaEventRecord(br.fork, st)) != cudaSuccess) return cuda_fail(x, "relate_cpals_batch: fork");
        for (int p : active) {
            relate_handle_s *h = hs[p];
            if (s >= h->N) continue;
            h->stream = br.s[p];
            if ((x = cudaStreamWaitEvent(br.s[p], br.fork, 0)) != cudaSuccess) return cuda_fail(x, "relate_cpals_batch: fork");
            const int r = step(p);
            h->stream = st;
            if (r != RELATE_OK) return r;
            if ((x = cudaEventRecord(br.ev[p], br.s[p])) != cudaSuccess || (x = cudaStreamWaitEvent(st, br.ev[p], 0)) != cudaSuccess)
                return cuda_fail(x, "relate_cpals_batch: join");
        }
        return RELATE_OK;
    };
    cudaGraphExec_t gexec = nullptr;
    bool dirty = true;
    auto enqueue_iteration = [&]() -> int {
        for (int s = 0; s < maxN; s++) {
            std::vector<BatchItemRef> items;
            int r = on_branches(s, [&](int p) { return mode_pre(hs[p], R[p], s); });
            if (r != RELATE_OK) return r;
            for (int p : active)
                if (s < hs[p]->N) items.push_back(BatchItemRef{hs[p], s, factors[p], R[p], hs[p]->d_M});
            if (!items.empty() && (rc = run_mttkrp_batch(items.data(), (int)items.size(), st)) != RELATE_OK) return rc;
            if ((r = on_branches(s, [&](int p) { return mode_post(hs[p], R[p], s, factors[p]); })) != RELATE_OK)
                return r;
        }
        return on_branches(0, [&](int p) {
            relate_handle_s *h = hs[p];
            return iteration_fit(h, R[p], h->h_pinned, reinterpret_cast<int *>(h->h_pinned + 1), nullptr, nullptr);
        });
    };
    for (int it = 1; it <= iters && !active.empty(); it++) {
        if (dirty) {  // one ALS iteration of the active problems as a CUDA graph
            if (gexec) cudaGraphExecDestroy(gexec);
            gexec = nullptr;
            cudaGraph_t g = nullptr;
            if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                return cuda_fail(e, "relate_cpals_batch: begin capture");
            rc = enqueue_iteration();
            cudaError_t e2 = cudaStreamEndCapture(st, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e2 != cudaSuccess) return cuda_fail(e2, "relate_cpals_batch: end capture");
            e = cudaGraphInstantiate(&gexec, g, cudaGraphInstantiateFlagUseNodePriority);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(e, "relate_cpals_batch: graph instantiate");
            dirty = false;
        }
        if ((e = cudaGraphLaunch(gexec, st)) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            cudaGraphExecDestroy(gexec);
            return cuda_fail(e, "relate_cpals_batch: iteration");
        }
        std::vector<int> still;
        for (int p : active) {
            relate_handle_s *h = hs[p];
            const double fit = h->h_pinned[0];
            const int *st3 = reinterpret_cast<const int *>(h->h_pinned + 1);
            bool stop = false;
            if (infos) {
                infos[p].fit = fit;
                infos[p].iters = it;
                infos[p].ridge_retries = st3[0];
                if (infos[p].fit_trace) infos[p].fit_trace[it - 1] = fit;
            }
            if (st3[2]) {
                status[p] = RELATE_ERR_TIMEOUT;
                stop = true;
            } else if (st3[1]) {
                status[p] = RELATE_ERR_NOT_PD;
                stop = true;
            } else if ((it > 1 || have_prev[p]) && fit - prev[p] < tol && prev[p] - fit < tol) {
                stop = true;
            }
            prev[p] = fit;
            have_prev[p] = 1;
            if (stop) dirty = true;
            else still.push_back(p);
        }
        active.swap(still);
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    int first_bad = RELATE_OK;
    for (int p = 0; p < n; p++) {
        relate_handle_s *h = hs[p];
        if (status[p] == RELATE_ERR_TIMEOUT) cudaMemsetAsync(h->d_err, 0, 16, st);
        if ((e = cudaMemcpyAsync(lambdas[p], h->d_lambda, sizeof(double) * R[p], cudaMemcpyDefault, st)) != cudaSuccess)
            return cuda_fail(e, "relate_cpals_batch: lambda");
        if (infos) infos[p].status = status[p];
        if (status[p] != RELATE_OK && first_bad == RELATE_OK) first_bad = status[p];
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "relate_cpals_batch: lambda");
    if (first_bad != RELATE_OK)
        return fail(first_bad, "relate_cpals_batch: a problem stopped with %s (see infos)", relate_status_string(first_bad));
    return RELATE_OK;
}

int relate_get_stats(relate_handle_t h, relate_stats_t *s) {
    g_err[0] = 0;
    if (!h || !s) return fail(RELATE_ERR_INVALID_ARG, "relate_get_stats: NULL argument");
    memset(s, 0, sizeof(*s));
    s->nmodes = h->N;
    s->lp = h->lp;
    s->key_bytes = 4 * h->KW;
    s->nnz = h->nnz;
    s->partition_size = h->S;
    s->partitions = h->P;
    s->nnz_total = h->nnz_total;
    s->shard_lo = h->shard_lo;
    for (int m = 0; m < h->N; m++) {
        s->dims[m] = h->dims[m];
        s->lbits[m] = h->lbits[m];
        s->field_offset[m] = h->runs.field_off[m];
        s->runs[m] = h->runs_n[m];
        s->distinct[m] = h->distinct[m];
        s->maxcount[m] = h->maxcount[m];
    }
    memcpy(s->bit_order, h->order, RELATE_MAX_KEY_BITS);
    return RELATE_OK;
}

int relate_get_conflict(relate_handle_t h, int mode, int R, relate_conflict_t *out) {
    g_err[0] = 0;
    if (!h || !out || mode < 0 || mode >= h->N || R < 1 || R > RELATE_MAX_RANK)
        return fail(RELATE_ERR_INVALID_ARG, "relate_get_conflict: bad argument");
    *out = resolve_conflict(h, mode, R);
    return RELATE_OK;
}

int relate_set_conflict(relate_handle_t h, int mode, relate_conflict_t c) {
    g_err[0] = 0;
    if (!h || mode < 0 || mode >= h->N || c < RELATE_CONFLICT_AUTO || c > RELATE_CONFLICT_PRIVATIZED)
        return fail(RELATE_ERR_INVALID_ARG, "relate_set_conflict: bad argument");
    h->conflict[mode] = c;
    return RELATE_OK;
}

int relate_set_mode_plan(relate_handle_t h, int mode, int depth, const int8_t *level, int col_passes) {
    g_err[0] = 0;
    if (!h || mode < 0 || mode >= h->N || depth < -1 || depth > RELATE_MAX_MODES || col_passes < 0 ||
        col_passes > RELATE_MAX_RANK)
        return fail(RELATE_ERR_INVALID_ARG, "relate_set_mode_plan: bad argument");
    if (level) {
        unsigned seen = 0;
        for (int s = 0; s < h->N - 1; s++) {
            const int k = level[s];
            if (k < 0 || k >= h->N || k == mode || ((seen >> k) & 1u))
                return fail(RELATE_ERR_INVALID_ARG, "relate_set_mode_plan: level must list the other modes once");
            seen |= 1u << k;
        }
    }
    const ModePlan before = resolve_plan(h, mode, RELATE_MAX_RANK);
    h->plan_depth[mode] = depth;
    h->level_set[mode] = level != nullptr;
    for (int s = 0; s < kMaxModes; s++) h->plan_level[mode][s] = level && s < h->N - 1 ? level[s] : 0;
    h->plan_passes[mode] = col_passes;
    const ModePlan after = resolve_plan(h, mode, RELATE_MAX_RANK);
    bool same = before.depth == after.depth;
    for (int s = 0; s < h->N - 1 && same; s++) same = before.level[s] == after.level[s];
    if (!same && h->d_tperm[mode]) {  // re-sorted on the mode's next MTTKRP
        cudaFreeAsync(h->d_tperm[mode], h->stream);
        h->d_tperm[mode] = nullptr;
    }
    return RELATE_OK;
}

int relate_get_mode_plan(relate_handle_t h, int mode, int R, int *depth, int8_t *level, int *col_passes) {
    g_err[0] = 0;
    if (!h || mode < 0 || mode >= h->N || R < 1 || R > RELATE_MAX_RANK)
        return fail(RELATE_ERR_INVALID_ARG, "relate_get_mode_plan: bad argument");
    const ModePlan p = resolve_plan(h, mode, R);
    if (depth) *depth = p.depth;
    if (level)
        for (int s = 0; s < h->N - 1; s++) level[s] = p.level[s];
    if (col_passes) *col_passes = p.passes;
    return RELATE_OK;
}

int relate_set_mode_kr(relate_handle_t h, int mode, int kr) {
    g_err[0] = 0;
    if (!h || mode < 0 || mode >= h->N || kr < -1 || kr > 1)
        return fail(RELATE_ERR_INVALID_ARG, "relate_set_mode_kr: bad argument");
    h->plan_kr[mode] = kr;
    return RELATE_OK;
}

int relate_get_mode_kr(relate_handle_t h, int mode, int R, int *kr, uint64_t *rows) {
    g_err[0] = 0;
    if (!h || mode < 0 || mode >= h->N || R < 1 || R > RELATE_MAX_RANK || !kr)
        return fail(RELATE_ERR_INVALID_ARG, "relate_get_mode_kr: bad argument");
    const ModePlan p = resolve_plan(h, mode, R);
    *kr = p.kr;
    if (rows) *rows = p.kr ? h->dims[p.level[p.depth - 1]] * h->dims[p.level[p.depth]] : 0;
    return RELATE_OK;
}

int relate_set_precision(relate_handle_t h, relate_dtype_t factor_dtype, relate_dtype_t acc_dtype) {
    g_err[0] = 0;
    if (!h || !valid_precision(factor_dtype, acc_dtype))
        return fail(RELATE_ERR_INVALID_ARG, "relate_set_precision: unsupported dtype pair");
    h->factor_dtype = factor_dtype;
    h->acc_dtype = acc_dtype;
    return RELATE_OK;
}

int relate_footprint(const uint64_t *dims, int nmodes, int64_t nnz, const relate_params_t *params, int R,
                     relate_footprint_t *out) {
    g_err[0] = 0;
    if (!out || !dims) return fail(RELATE_ERR_INVALID_ARG, "relate_footprint: NULL argument");
    memset(out, 0, sizeof(*out));
    relate_params_t defaults;
    relate_params_default(&defaults);
    const relate_params_t *p = params ? params : &defaults;
    if (nmodes < 2 || nmodes > RELATE_MAX_MODES || nnz < 0 || nnz > (int64_t)0xffffffffLL || R < 1 ||
        R > RELATE_MAX_RANK || p->partition_size < 0 || !valid_precision(p->factor_dtype, p->acc_dtype) ||
        (p->val_dtype != RELATE_F64 && p->val_dtype != RELATE_F32))
        return fail(RELATE_ERR_INVALID_ARG, "relate_footprint: bad argument");
    int lp = 0;
    uint64_t maxI = 0, sumI = 0;
    for (int m = 0; m < nmodes; m++) {
        if (dims[m] < 1 || dims[m] > ((uint64_t)1 << 32))
            return fail(RELATE_ERR_INVALID_ARG, "relate_footprint: dims[%d] not in [1, 2^32]", m);
        lp += bits_for(dims[m]);
        maxI = dims[m] > maxI ? dims[m] : maxI;
        sumI += dims[m];
    }
    if (lp > RELATE_MAX_KEY_BITS) return fail(RELATE_ERR_KEY_TOO_WIDE, "relate_footprint: l(p)=%d > 128", lp);
    const size_t kb = lp <= 32 ? 4 : lp <= 64 ? 8 : 16;
    const int vb = p->val_dtype == RELATE_F64 ? 8 : 4;
    const int64_t S = p->partition_size > 0 ? p->partition_size : 4096;
    const int64_t P = (nnz + S - 1) / S;
    const size_t resident = words_bytes(nnz, kb) + vals_bytes(nnz, vb) + 2 * bounds_bytes(P, nmodes) + 64 + 16 +
                            kHotScratchBytes + (size_t)nmodes * tperm_bytes(nnz) +
                            sumI * 4 + (size_t)nmodes * kHotMax * 4 + perm_bytes(nnz);
    size_t temps = 2 * (size_t)nnz * kb + 2 * (size_t)nnz * 4 + radix_sort_temp_bytes(nnz) + 64 + kSmallBytes +
                   2 * (size_t)kLutMaxBytes + hot_table_temp_bytes(maxI);
    if (!p->coords_on_device && nnz > 0) temps += (size_t)nmodes * nnz * 4 + (size_t)nnz * vb;
    out->encode_peak = resident + temps;
    out->resident = resident;
    out->cpals_workspace = ws_total(maxI, nmodes, R);
    if (p->factor_dtype == RELATE_F64 && nmodes >= 4 && nmodes <= 5 && R % 2 == 0) {
        // the AUTO plans' Khatri-Rao table: the two shortest other modes
        uint64_t kr = 0;
        for (int m = 0; m < nmodes; m++) {
            uint64_t s1 = ~0ull, s2 = ~0ull;  // the two smallest I_k, k != m
            for (int k = 0; k < nmodes; k++) {
                if (k == m) continue;
                if (dims[k] < s1) {
                    s2 = s1;
                    s1 = dims[k];
                } else if (dims[k] < s2) {
                    s2 = dims[k];
                }
            }
            const uint64_t rows = s1 * s2;
            if (kr_auto(rows, nnz) && kr_fits(rows, R) && rows * R * 8 > kr) kr = rows * R * 8;
        }
        out->cpals_workspace += kr;
    }
    out->factors = sumI * (uint64_t)R * dtype_bytes(p->factor_dtype);
    return RELATE_OK;
}

int relate_release_cached_memory(void) {
    g_err[0] = 0;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = lib_pool(&pool);
    if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
    return e == cudaSuccess ? RELATE_OK : cuda_fail(e, "relate_release_cached_memory");
}

void relate_shard_range(int64_t nnz, int rank, int count, int64_t *lo, int64_t *hi) {
    if (count < 1) count = 1;
    if (rank < 0) rank = 0;
    if (rank >= count) rank = count - 1;
    if (nnz < 0) nnz = 0;
    if (lo) *lo = (int64_t)(((__int128)nnz * rank) / count);
    if (hi) *hi = (int64_t)(((__int128)nnz * (rank + 1)) / count);
}

int relate_set_reduce_hook(relate_handle_t h, relate_reduce_fn fn, void *user) {
    g_err[0] = 0;
    if (!h) return fail(RELATE_ERR_INVALID_ARG, "relate_set_reduce_hook: NULL handle");
    h->reduce_fn = fn;
    h->reduce_user = user;
    return RELATE_OK;
}

int relate_set_cpals_graph(relate_handle_t h, int enable) {
    g_err[0] = 0;
    if (!h) return fail(RELATE_ERR_INVALID_ARG, "relate_set_cpals_graph: NULL handle");
    h->use_graph = enable ? 1 : 0;
    return RELATE_OK;
}

int relate_set_stream(relate_handle_t h, void *stream) {
    g_err[0] = 0;
    if (!h) return fail(RELATE_ERR_INVALID_ARG, "relate_set_stream: NULL handle");
    h->stream = (cudaStream_t)stream;
    return RELATE_OK;
}

int relate_decode(relate_handle_t h, uint32_t *coords_out, void *vals_out, uint32_t *perm_out, uint64_t *keys_out,
                  void *stream) {
    g_err[0] = 0;
    if (!h) return fail(RELATE_ERR_INVALID_ARG, "relate_decode: NULL handle");
    const cudaStream_t st = (cudaStream_t)stream;
    const int vb = h->val_dtype == RELATE_F64 ? 8 : 4;
    cudaError_t e = cudaSuccess;
    if (coords_out && (e = launch_decode_words(h->KW, h->d_words, h->nnz, h->N, h->fields, coords_out, st)))
        return cuda_fail(e, "relate_decode: coordinates");
    if (vals_out && h->nnz &&
        (e = cudaMemcpyAsync(vals_out, h->d_vals, (size_t)h->nnz * vb, cudaMemcpyDeviceToDevice, st)))
        return cuda_fail(e, "relate_decode: values");
    if (perm_out && h->nnz &&
        (e = cudaMemcpyAsync(perm_out, h->d_perm, (size_t)h->nnz * 4, cudaMemcpyDeviceToDevice, st)))
        return cuda_fail(e, "relate_decode: permutation");
    if (keys_out && (e = launch_words_to_keys(h->KW, h->d_words, h->nnz, h->runs, keys_out, st)))
        return cuda_fail(e, "relate_decode: positions");
    return RELATE_OK;
}

int relate_get_partitions(relate_handle_t h, uint32_t *lo, uint32_t *hi, void *stream) {
    g_err[0] = 0;
    if (!h || !lo || !hi) return fail(RELATE_ERR_INVALID_ARG, "relate_get_partitions: NULL argument");
    const size_t bytes = (size_t)h->P * h->N * 4;
    if (!bytes) return RELATE_OK;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(lo, h->d_plo, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream)) ||
        (e = cudaMemcpyAsync(hi, h->d_phi, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream)))
        return cuda_fail(e, "relate_get_partitions");
    return RELATE_OK;
}

int relate_gram(const void *A, int64_t I, int R, relate_dtype_t dtype, double *G, void *stream) {
    g_err[0] = 0;
    if ((!A && I > 0) || !G || I < 0 || R < 1 || R > RELATE_MAX_RANK ||
        (dtype != RELATE_F64 && dtype != RELATE_F32 && dtype != RELATE_BF16))
        return fail(RELATE_ERR_INVALID_ARG, "relate_gram: bad argument");
    const cudaStream_t st = (cudaStream_t)stream;
    void *scratch = nullptr;
    cudaError_t e = dalloc(&scratch, dense_scratch_doubles(R) * 8, st);
    if (e != cudaSuccess) return cuda_fail(e, "relate_gram: scratch");
    int *err = gram_err_word((double *)scratch);
    const bool tc = I > 0 && gram_uses_tc(A, R, dtype);
    int flag = 0;
    if ((e = cudaMemsetAsync(err, 0, sizeof(int), st)) == cudaSuccess &&
        (e = gram_checked(A, I, R, dtype, (double *)scratch, G, err, st)) == cudaSuccess && tc) {
        // the tensor-core kernel reports a given-up wait in the status word
        if ((e = cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, st)) == cudaSuccess)
            e = cudaStreamSynchronize(st);
    }
    cudaError_t e2 = cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "relate_gram: launch");
    if (e2 != cudaSuccess) return cuda_fail(e2, "relate_gram: free");
    if (flag) return fail(RELATE_ERR_TIMEOUT, "relate_gram: a bounded tensor-core wait timed out (G is NaN)");
    return RELATE_OK;
}

int relate_solve_rows(void *M, int64_t I, int R, relate_dtype_t dtype, const double *W, void *stream) {
    g_err[0] = 0;
    if ((!M && I > 0) || !W || I < 0 || R < 1 || R > RELATE_MAX_RANK || (dtype != RELATE_F64 && dtype != RELATE_F32))
        return fail(RELATE_ERR_INVALID_ARG, "relate_solve_rows: bad argument");
    const cudaStream_t st = (cudaStream_t)stream;
    if (I == 0) return RELATE_OK;
    void *scratch = nullptr;  // status word, then W in FP32
    cudaError_t e = dalloc(&scratch, 16 + (size_t)R * R * 4, st);
    if (e != cudaSuccess) return cuda_fail(e, "relate_solve_rows: scratch");
    int *err = (int *)scratch;
    float *W32 = (float *)((char *)scratch + 16);
    const bool f = fault_is("gram_timeout");
    int flag = 0;
    if ((e = cudaMemsetAsync(err, 0, sizeof(int), st)) == cudaSuccess &&
        (dtype == RELATE_F64 || (e = launch_to_float(W, R * R, W32, st)) == cudaSuccess) &&
        (e = launch_solve_rows(M, I, R, dtype, W, W32, err, st, f ? 100000000LL : 0, f ? 1 : 0)) == cudaSuccess &&
        (e = cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, st)) == cudaSuccess)
        e = cudaStreamSynchronize(st);
    cudaError_t e2 = cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "relate_solve_rows: launch");
    if (e2 != cudaSuccess) return cuda_fail(e2, "relate_solve_rows: free");
    if (flag) return fail(RELATE_ERR_TIMEOUT, "relate_solve_rows: a bounded tensor-core wait timed out");
    return RELATE_OK;
}

int relate_sync_status(relate_handle_t h, void *stream) {
    g_err[0] = 0;
    if (!h) return fail(RELATE_ERR_INVALID_ARG, "relate_sync_status: NULL handle");
    const cudaStream_t st = (cudaStream_t)stream;
    int flag = 0;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "relate_sync_status");
    if (flag) {
        if ((e = cudaMemsetAsync(h->d_err, 0, 16, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_fail(e, "relate_sync_status: clear");
        return fail(RELATE_ERR_TIMEOUT, "relate_sync_status: a bounded device wait timed out");
    }
    return RELATE_OK;
}

void relate_free(relate_handle_t h) { delete h; }

const char *relate_status_string(int status) {
    switch (status) {
    case RELATE_OK: return "ok";
    case RELATE_ERR_INVALID_ARG: return "invalid argument";
    case RELATE_ERR_BAD_BIT_ORDER: return "bit order breaks the masking rule (mode n must appear l(n) times)";
    case RELATE_ERR_KEY_TOO_WIDE: return "linear position wider than 128 bits";
    case RELATE_ERR_COORD_OUT_OF_RANGE: return "coordinate out of range";
    case RELATE_ERR_OOM: return "out of device memory";
    case RELATE_ERR_NOT_PD: return "normal equations not positive definite";
    case RELATE_ERR_TIMEOUT: return "bounded device wait timed out";
    case RELATE_ERR_CUDA: return "CUDA error";
    case RELATE_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
    }
}

const char *relate_last_error(void) { return g_err; }

const char *relate_version(void) { return RELATE_VERSION_STRING; }

}  // extern "C"
