// libko C ABI: handle management, argument validation, staging of host
// buffers, and dispatch to the simulator kernels.  See include/ko.h.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ko_internal.h"
#include "ko_fast.h"

namespace {

thread_local ko_status t_last_error = KO_OK;
std::atomic<long long> g_launches{0};

ko_status fail(ko_status s)
{
    t_last_error = s;
    return s;
}

ko_status ok()
{
    t_last_error = KO_OK;
    return KO_OK;
}

constexpr size_t kSimpleScratchBudget = size_t(1) << 30;  // bytes for the simple simulator slabs
constexpr int64_t kFactorial[21] = {1LL, 1LL, 2LL, 6LL, 24LL, 120LL, 720LL, 5040LL, 40320LL,
                                    362880LL, 3628800LL, 39916800LL, 479001600LL, 6227020800LL,
                                    87178291200LL, 1307674368000LL, 20922789888000LL,
                                    355687428096000LL, 6402373705728000LL, 121645100408832000LL,
                                    2432902008176640000LL};

int log2_exact(int64_t v)
{
    if (v <= 0 || (v & (v - 1))) return -1;
    int s = 0;
    while ((int64_t(1) << s) != v) s++;
    return s;
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Small per-call device records of a handle.
struct Meta {
    KoChunk chunk[2];                 // [0] heuristic order (mode 2), [1] the main work
    long long ref;                    // reference makespan written by the heuristic pass
    long long pad;
    int8_t perm[KO_MAX_KERNELS + 8];  // heuristic / ranked order
};

}  // namespace

void ko_count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

struct ko_gpu {
    KoSet h{};
    bool frozen = false;       // kernels / capacities fixed after the first evaluation
    KoSet *d_set = nullptr;
    KoAccum *d_acc = nullptr;
    void *scratch = nullptr;   // simple-simulator slabs
    size_t scratch_bytes = 0;
    int64_t *d_ms = nullptr;   // makespan buffer
    size_t ms_cap = 0;
    void *d_stage = nullptr;   // staging for host inputs
    size_t stage_cap = 0;
    unsigned long long *d_hist = nullptr;
    int hist_cap = 0;
    long long h2d = 0, d2h = 0;   // bytes copied by this handle
    Meta *d_meta = nullptr;       // chunk lists, heuristic order, reference makespan (device)
    Meta h_meta{};
    KoFastState fast{};        // run-length simulator state (work list, overflow list)
    bool fast_pending = false; // an asynchronous run-length launch has not been inspected yet

    ~ko_gpu()
    {
        cudaFree(d_set); cudaFree(d_acc); cudaFree(scratch); cudaFree(d_ms); cudaFree(d_stage);
        cudaFree(d_hist);
        cudaFree(d_meta);
        ko_fast_release(&fast);
    }
};

namespace {

ko_status grow(void **p, size_t *cap, size_t need)
{
    if (*cap >= need) return KO_OK;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(p, need) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return KO_ERR_NOMEM;
    }
    *cap = need;
    return KO_OK;
}

// Upload the set (with ref_makespan) and make sure the accumulator exists.
ko_status prepare(ko_gpu *g, cudaStream_t st)
{
    g->frozen = true;
    if (!g->d_set && cudaMalloc(&g->d_set, sizeof(KoSet)) != cudaSuccess) {
        cudaGetLastError();
        return KO_ERR_NOMEM;
    }
    if (!g->d_acc && cudaMalloc(&g->d_acc, sizeof(KoAccum) * 2) != cudaSuccess) {
        cudaGetLastError();
        return KO_ERR_NOMEM;
    }
    if (cudaMemcpyAsync(g->d_set, &g->h, sizeof(KoSet), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return KO_ERR_CUDA;
    g->h2d += sizeof(KoSet);
    return KO_OK;
}

ko_status simple_scratch(ko_gpu *g, int64_t count)
{
    const size_t per = ko_simple_scratch_per_thread(g->h);
    size_t slots = std::max<size_t>(128, std::min<size_t>(kSimpleScratchBudget / per, 152 * 8 * 128));
    slots = std::min<size_t>(slots, (size_t)((count + 127) / 128) * 128);
    slots = std::max<size_t>(slots, 128);
    return grow(&g->scratch, &g->scratch_bytes, slots * per);
}

ko_status check_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return KO_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? KO_ERR_NOMEM : KO_ERR_CUDA;
}

bool fast_ok(const ko_gpu *g) { return !g->fast.disabled && ko_fast_applicable(g->h); }

ko_status upload_meta(ko_gpu *g, cudaStream_t st)
{
    if (!g->d_meta && cudaMalloc(&g->d_meta, sizeof(Meta)) != cudaSuccess) {
        cudaGetLastError();
        return KO_ERR_NOMEM;
    }
    if (cudaMemcpyAsync(g->d_meta, &g->h_meta, sizeof(Meta), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return KO_ERR_CUDA;
    g->h2d += sizeof(Meta);
    return KO_OK;
}

KoWork work_for(ko_gpu *g, int chunk)
{
    KoWork w{};
    w.sets = g->d_set;
    w.chunks = &g->d_meta->chunk[chunk];
    w.nchunks = 1;
    w.n_items = g->h_meta.chunk[chunk].count;
    w.levels = 1;
    return w;
}

// Exhaustive chunk (all N! orders as prefix items) into h_meta.chunk[1].
void exhaustive_chunk(ko_gpu *g, KoWork *w_levels)
{
    const int N = g->h.n;
    const int d0 = ko_fast_d0(g->fast, N);
    KoChunk &c = g->h_meta.chunk[1];
    c = KoChunk{};
    c.first = 0;
    c.count = kFactorial[N] / kFactorial[N - d0];
    c.set = 0;
    c.d0 = d0;
    c.mode = 0;
    *w_levels = KoWork{};
    w_levels->levels = N - 1 - d0 > 0 ? N - 1 - d0 : 1;
}

ko_status fast_launch_timed(ko_gpu *g, const KoWork &w, cudaStream_t st)
{
    KoFastState &fs = g->fast;
    if (!fs.ev0 && (cudaEventCreate(&fs.ev0) != cudaSuccess || cudaEventCreate(&fs.ev1) != cudaSuccess))
        return KO_ERR_CUDA;
    cudaEventRecord(fs.ev0, st);
    ko_status s = ko_fast_launch(&fs, w, ko_slab_bytes(g->h.S, g->h.Bk), st);
    cudaEventRecord(fs.ev1, st);
    return s;
}

// After a synchronise: read the event time and the abandoned-item count.
ko_status fast_after_sync(ko_gpu *g)
{
    KoFastState &fs = g->fast;
    float ms = -1.0f;
    if (fs.ev0 && cudaEventElapsedTime(&ms, fs.ev0, fs.ev1) == cudaSuccess) fs.last_ms = ms;
    cudaGetLastError();
    unsigned long long cnt = 0;
    const unsigned long long *dc = ko_fast_overflow_counter(&fs);
    if (dc && cudaMemcpy(&cnt, dc, sizeof(cnt), cudaMemcpyDeviceToHost) != cudaSuccess) return KO_ERR_CUDA;
    fs.d2h += sizeof(cnt);
    fs.last_overflow = cnt;
    return cnt > fs.ov_cap ? KO_ERR_STATE : KO_OK;  // cannot happen: the lists hold every item
}

}  // namespace

extern "C" {

ko_gpu *ko_create_gpu(int32_t n_sm, int32_t n_reg_sm, int32_t n_shm_sm, int32_t n_warp_sm,
                      int32_t n_blk_sm)
{
    if (n_sm < 1 || n_sm > KO_MAX_SM || n_reg_sm < 1 || n_reg_sm > KO_MAX_CYCLES || n_shm_sm < 1 ||
        n_shm_sm > KO_MAX_CYCLES || n_warp_sm < 1 || n_warp_sm > KO_MAX_CYCLES || n_blk_sm < 1 ||
        n_blk_sm > KO_MAX_BLK_SM) {
        fail(KO_ERR_ARG);
        return nullptr;
    }
    ko_gpu *g = new (std::nothrow) ko_gpu();
    if (!g) {
        fail(KO_ERR_NOMEM);
        return nullptr;
    }
    g->h.S = n_sm; g->h.R = n_reg_sm; g->h.Sh = n_shm_sm; g->h.W = n_warp_sm; g->h.Bk = n_blk_sm;
    g->h.ccap = 32768; g->h.mcap = 32768;
    g->h.cshift = 15; g->h.mshift = 15;
    g->h.n = 0;
    ok();
    return g;
}

ko_status ko_set_capacity(ko_gpu *g, int64_t c_cap, int64_t m_cap)
{
    if (!g || c_cap < 1 || m_cap < 1 || c_cap > (int64_t(1) << 30) || m_cap > (int64_t(1) << 30))
        return fail(KO_ERR_ARG);
    if (g->frozen) return fail(KO_ERR_STATE);
    g->h.ccap = c_cap; g->h.mcap = m_cap;
    g->h.cshift = log2_exact(c_cap); g->h.mshift = log2_exact(m_cap);
    return ok();
}

ko_status ko_set_sampling(ko_gpu *g, int32_t mode)
{
    if (!g || (mode != KO_SAMPLE_BURST_END && mode != KO_SAMPLE_AT_PLACEMENT)) return fail(KO_ERR_ARG);
    if (g->frozen) return fail(KO_ERR_STATE);
    g->h.sampling = mode;
    return ok();
}

int32_t ko_add_kernel(ko_gpu *g, int32_t n_reg_i, int32_t n_shm_i, int32_t n_warp_i,
                      int32_t n_tblk_i, int64_t c_i, int64_t m_i)
{
    if (!g || n_reg_i < 1 || n_shm_i < 0 || n_warp_i < 1 || n_tblk_i < 1 || n_tblk_i > (1 << 20) ||
        c_i < 1 || m_i < 1 || c_i > KO_MAX_CYCLES || m_i > KO_MAX_CYCLES)
        return fail(KO_ERR_ARG);
    if (g->frozen) return fail(KO_ERR_STATE);
    if (g->h.n >= KO_MAX_KERNELS) return fail(KO_ERR_ARG);
    if (n_reg_i > g->h.R || n_shm_i > g->h.Sh || n_warp_i > g->h.W) return fail(KO_ERR_NOFIT);
    KoKern &k = g->h.k[g->h.n];
    k.r = n_reg_i; k.s = n_shm_i; k.w = n_warp_i; k.b = n_tblk_i;
    k.c = (int32_t)c_i; k.m = (int32_t)m_i;
    g->h.lk[g->h.n] = KoLaneK{(uint32_t)n_reg_i | (1u << 19) | ((uint32_t)n_warp_i << 25), (uint32_t)n_shm_i,
                              (uint32_t)c_i, (uint32_t)m_i};
    int64_t lb, ub;
    g->h.n++;
    if (!ko_bounds_host(g->h, &lb, &ub)) {
        g->h.n--;
        return fail(KO_ERR_OVERFLOW);
    }
    ok();
    return g->h.n - 1;
}

int32_t ko_num_kernels(const ko_gpu *g)
{
    if (!g) return fail(KO_ERR_ARG);
    ok();
    return g->h.n;
}

ko_status ko_bounds(ko_gpu *g, int64_t *lb, int64_t *ub)
{
    if (!g || !lb || !ub) return fail(KO_ERR_ARG);
    if (!ko_bounds_host(g->h, lb, ub)) return fail(KO_ERR_OVERFLOW);
    return ok();
}

ko_status ko_heuristic_order(ko_gpu *g, int32_t *order_out)
{
    if (!g || (!order_out && g->h.n > 0)) return fail(KO_ERR_ARG);
    if (g->h.n > 0) ko_heuristic_host(g->h, order_out);
    return ok();
}

ko_status ko_eval_orders_ps(ko_gpu *g, const int8_t *orders, int64_t n, double *makespan_out, void *stream)
{
    if (!g || n < 0 || (n > 0 && (!orders || !makespan_out))) return fail(KO_ERR_ARG);
    if (n == 0) return ok();
    const int N = g->h.n;
    cudaStream_t st = (cudaStream_t)stream;
    const bool out_dev = is_device_ptr(makespan_out);
    if (N == 0) {
        if (out_dev) {
            if (cudaMemsetAsync(makespan_out, 0, sizeof(double) * n, st) != cudaSuccess) return fail(KO_ERR_CUDA);
        } else {
            std::memset(makespan_out, 0, sizeof(double) * n);
        }
        return ok();
    }
    ko_status s = prepare(g, st);
    if (s) return fail(s);
    const size_t in_bytes = (size_t)n * N;
    const bool in_dev = is_device_ptr(orders);
    const size_t need = (in_dev ? 0 : (in_bytes + 255) / 256 * 256) + (out_dev ? 0 : sizeof(double) * n);
    if ((s = grow(&g->d_stage, &g->stage_cap, std::max<size_t>(need, 256)))) return fail(s);
    char *stage = (char *)g->d_stage;
    const int8_t *d_in = orders;
    if (!in_dev) {
        if (cudaMemcpyAsync(stage, orders, in_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return fail(KO_ERR_CUDA);
        g->h2d += (long long)in_bytes;
        d_in = (const int8_t *)stage;
        stage += (in_bytes + 255) / 256 * 256;
    }
    double *d_out = out_dev ? makespan_out : (double *)stage;
    const size_t per = ko_ps_scratch_per_thread(g->h);
    size_t slots = std::max<size_t>(128, std::min<size_t>(kSimpleScratchBudget / per, 152 * 8 * 128));
    slots = std::max<size_t>(128, std::min<size_t>(slots, (size_t)((n + 127) / 128) * 128));
    if ((s = grow(&g->scratch, &g->scratch_bytes, slots * per))) return fail(s);
    if ((s = check_cuda(ko_launch_ps(g->d_set, g->h, d_in, n, d_out, g->scratch, g->scratch_bytes, st))))
        return fail(s);
    if (!out_dev) {
        if (cudaMemcpyAsync(makespan_out, d_out, sizeof(double) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return fail(KO_ERR_CUDA);
        g->d2h += (long long)sizeof(double) * n;
    }
    if ((!in_dev || !out_dev) && cudaStreamSynchronize(st) != cudaSuccess) return fail(KO_ERR_CUDA);
    return ok();
}

ko_status ko_heuristic_order_ex(ko_gpu *g, int32_t reading, int32_t *order_out)
{
    if (!g || (!order_out && g->h.n > 0) || (reading != KO_HEUR_PER_SM && reading != KO_HEUR_PER_BLOCK))
        return fail(KO_ERR_ARG);
    if (g->h.n > 0) ko_heuristic_host(g->h, order_out, reading == KO_HEUR_PER_BLOCK);
    return ok();
}

ko_status ko_eval_orders(ko_gpu *g, const uint64_t *idx, const int8_t *orders, int64_t n,
                         int64_t *makespan_out, void *stream)
{
    if (!g || n < 0 || (idx == nullptr) == (orders == nullptr) || (n > 0 && !makespan_out))
        return fail(KO_ERR_ARG);
    const int N = g->h.n;
    if (idx && N > 20) return fail(KO_ERR_ARG);
    if (n == 0) return ok();
    cudaStream_t st = (cudaStream_t)stream;
    const bool out_dev = is_device_ptr(makespan_out);
    if (N == 0) {
        if (out_dev) {
            if (cudaMemsetAsync(makespan_out, 0, sizeof(int64_t) * n, st) != cudaSuccess)
                return fail(KO_ERR_CUDA);
        } else {
            std::memset(makespan_out, 0, sizeof(int64_t) * n);
        }
        return ok();
    }
    ko_status s = prepare(g, st);
    if (s) return fail(s);
    const void *in = idx ? (const void *)idx : (const void *)orders;
    const size_t in_bytes = idx ? sizeof(uint64_t) * n : (size_t)n * N;
    const bool in_dev = is_device_ptr(in);
    size_t need = (in_dev ? 0 : (in_bytes + 255) / 256 * 256) + (out_dev ? 0 : sizeof(int64_t) * n);
    if ((s = grow(&g->d_stage, &g->stage_cap, std::max<size_t>(need, 256)))) return fail(s);
    char *stage = (char *)g->d_stage;
    const void *d_in = in;
    if (!in_dev) {
        if (cudaMemcpyAsync(stage, in, in_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return fail(KO_ERR_CUDA);
        g->h2d += (long long)in_bytes;
        d_in = stage;
        stage += (in_bytes + 255) / 256 * 256;
    }
    int64_t *d_out = out_dev ? makespan_out : (int64_t *)stage;
    bool used_fast = false;
    if (fast_ok(g)) {
        KoChunk &c = g->h_meta.chunk[1];
        c = KoChunk{};
        c.count = n;
        c.d0 = N;
        c.mode = idx ? 1 : 2;
        if ((s = upload_meta(g, st))) return fail(s);
        KoWork w = work_for(g, 1);
        w.idx = idx ? (const uint64_t *)d_in : nullptr;
        w.perms = idx ? nullptr : (const int8_t *)d_in;
        w.out = d_out;
        if ((s = fast_launch_timed(g, w, st))) return fail(s);
        used_fast = true;
        g->fast_pending = true;
    } else {
        if ((s = simple_scratch(g, n))) return fail(s);
        if ((s = check_cuda(ko_launch_simple(g->d_set, g->h, idx ? nullptr : (const int8_t *)d_in,
                                             idx ? (const uint64_t *)d_in : nullptr, 0, n, d_out,
                                             nullptr, g->scratch, g->scratch_bytes, st))))
            return fail(s);
    }
    if (!out_dev) {
        if (cudaMemcpyAsync(makespan_out, d_out, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
            return fail(KO_ERR_CUDA);
        g->d2h += (long long)sizeof(int64_t) * n;
    }
    if (!in_dev || !out_dev) {
        if (cudaStreamSynchronize(st) != cudaSuccess) return fail(KO_ERR_CUDA);
        if (used_fast) {
            g->fast_pending = false;
            if ((s = fast_after_sync(g))) return fail(s);
        }
    }
    return ok();
}

}  // extern "C"

namespace {

// All N! makespans into d_out (device, nullable) and the accumulator, on
// `st`; with `refs` the counts compare against *refs (device).
ko_status exhaustive(ko_gpu *g, int64_t *d_out, KoAccum *d_acc, long long *refs, cudaStream_t st)
{
    const int64_t total = kFactorial[g->h.n];
    ko_status s = check_cuda(ko_launch_accum_reset(d_acc, 1, st));
    if (s) return s;
    if (fast_ok(g)) {
        KoWork lv;
        exhaustive_chunk(g, &lv);
        if ((s = upload_meta(g, st))) return s;
        KoWork w = work_for(g, 1);
        w.levels = lv.levels;
        w.refs = refs;
        w.accs = d_acc;
        w.out = d_out;
        return fast_launch_timed(g, w, st);
    }
    if ((s = simple_scratch(g, total))) return s;
    return check_cuda(ko_launch_simple(g->d_set, g->h, nullptr, nullptr, 0, total, d_out, d_acc,
                                       g->scratch, g->scratch_bytes, st));
}

ko_status makespan_of(ko_gpu *g, const int32_t *order, int64_t *m, cudaStream_t st)
{
    const int N = g->h.n;
    int8_t perm[KO_MAX_KERNELS];
    for (int i = 0; i < N; i++) perm[i] = (int8_t)order[i];
    ko_status s = grow(&g->d_stage, &g->stage_cap, 256 + sizeof(int64_t));
    if (s) return s;
    int8_t *d_perm = (int8_t *)g->d_stage;
    int64_t *d_m = (int64_t *)((char *)g->d_stage + 256);
    if (cudaMemcpyAsync(d_perm, perm, N, cudaMemcpyHostToDevice, st) != cudaSuccess) return KO_ERR_CUDA;
    g->h2d += N;
    if ((s = simple_scratch(g, 1))) return s;
    if ((s = check_cuda(ko_launch_simple(g->d_set, g->h, d_perm, nullptr, 0, 1, d_m, nullptr,
                                         g->scratch, g->scratch_bytes, st))))
        return s;
    if (cudaMemcpyAsync(m, d_m, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return KO_ERR_CUDA;
    g->d2h += sizeof(int64_t);
    if (cudaStreamSynchronize(st) != cudaSuccess) return KO_ERR_CUDA;
    return KO_OK;
}

}  // namespace

extern "C" {

ko_status ko_eval_all(ko_gpu *g, int64_t *makespans_out, void *stream)
{
    if (!g || !makespans_out || g->h.n < 1) return fail(KO_ERR_ARG);
    if (g->h.n > KO_MAX_EXHAUSTIVE) return fail(KO_ERR_TOO_LARGE);
    if (!is_device_ptr(makespans_out)) return fail(KO_ERR_ARG);
    cudaStream_t st = (cudaStream_t)stream;
    g->h.ref_makespan = 0;
    ko_status s = prepare(g, st);
    if (s) return fail(s);
    if ((s = exhaustive(g, makespans_out, g->d_acc, nullptr, st))) return fail(s);
    g->fast_pending = fast_ok(g);
    return ok();
}

ko_status ko_rank_order(ko_gpu *g, const int32_t *order, ko_rank *out, uint64_t *hist,
                        int32_t nbins, void *stream)
{
    if (!g || !out || (hist && (nbins < 1 || nbins > 32768)) || g->h.n < 1) return fail(KO_ERR_ARG);
    const int N = g->h.n;
    if (N > KO_MAX_EXHAUSTIVE) return fail(KO_ERR_TOO_LARGE);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int32_t> ord(N);
    if (order) {
        uint32_t seen = 0;
        for (int i = 0; i < N; i++) {
            if (order[i] < 0 || order[i] >= N || ((seen >> order[i]) & 1u)) return fail(KO_ERR_ARG);
            seen |= 1u << order[i];
            ord[i] = order[i];
        }
    } else {
        ko_heuristic_host(g->h, ord.data());
    }
    const int64_t total = kFactorial[N];
    g->h.ref_makespan = 0;
    ko_status s = prepare(g, st);
    if (s) return fail(s);
    if ((s = grow((void **)&g->d_ms, &g->ms_cap, sizeof(int64_t) * total))) return fail(s);
    int64_t mh = 0;
    const bool fast = fast_ok(g);
    if (fast) {
        // pass 1: makespan of the ranked order into d_meta->ref (device);
        // pass 2: all N! orders, counted against that reference
        KoChunk &c0 = g->h_meta.chunk[0];
        c0 = KoChunk{};
        c0.count = 1;
        c0.d0 = N;
        c0.mode = 2;
        for (int i = 0; i < N; i++) g->h_meta.perm[i] = (int8_t)ord[i];
        KoWork lv;
        exhaustive_chunk(g, &lv);
        if ((s = upload_meta(g, st))) return fail(s);
        KoWork w0 = work_for(g, 0);
        w0.perms = g->d_meta->perm;
        w0.out = (int64_t *)&g->d_meta->ref;
        if ((s = ko_fast_launch(&g->fast, w0, ko_slab_bytes(g->h.S, g->h.Bk), st))) return fail(s);
        if ((s = check_cuda(ko_launch_accum_reset(g->d_acc, 1, st)))) return fail(s);
        KoWork w1 = work_for(g, 1);
        w1.levels = lv.levels;
        w1.refs = &g->d_meta->ref;
        w1.accs = g->d_acc;
        w1.out = g->d_ms;
        if ((s = fast_launch_timed(g, w1, st))) return fail(s);
    } else {
        if ((s = makespan_of(g, ord.data(), &mh, st))) return fail(s);
        if (mh < 0) return fail(KO_ERR_STATE);
        g->h.ref_makespan = mh;
        if ((s = prepare(g, st))) return fail(s);
        if ((s = exhaustive(g, g->d_ms, g->d_acc, nullptr, st))) return fail(s);
    }
    if (hist) {
        if (g->hist_cap < nbins) {
            cudaFree(g->d_hist);
            g->d_hist = nullptr;
            g->hist_cap = 0;
            if (cudaMalloc(&g->d_hist, sizeof(unsigned long long) * nbins) != cudaSuccess) {
                cudaGetLastError();
                return fail(KO_ERR_NOMEM);
            }
            g->hist_cap = nbins;
        }
        const bool hist_dev = is_device_ptr(hist);
        unsigned long long *dh = hist_dev ? (unsigned long long *)hist : g->d_hist;
        if (cudaMemsetAsync(dh, 0, sizeof(unsigned long long) * nbins, st) != cudaSuccess)
            return fail(KO_ERR_CUDA);
        if ((s = check_cuda(ko_launch_histogram(g->d_ms, total, g->d_acc, dh, nbins, st))))
            return fail(s);
        if (!hist_dev) {
            if (cudaMemcpyAsync(hist, dh, sizeof(unsigned long long) * nbins, cudaMemcpyDeviceToHost,
                                st) != cudaSuccess)
                return fail(KO_ERR_CUDA);
            g->d2h += (long long)sizeof(unsigned long long) * nbins;
        }
    }
    KoAccum acc;
    if (cudaMemcpyAsync(&acc, g->d_acc, sizeof(KoAccum), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return fail(KO_ERR_CUDA);
    g->d2h += sizeof(KoAccum);
    if (fast) {
        if (cudaMemcpyAsync(&mh, &g->d_meta->ref, sizeof(mh), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return fail(KO_ERR_CUDA);
        g->d2h += sizeof(mh);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(KO_ERR_CUDA);
    if (fast && (s = fast_after_sync(g))) return fail(s);
    if (acc.failed || mh < 0) return fail(KO_ERR_STATE);
    out->min = (int64_t)acc.min;
    out->max = (int64_t)acc.max;
    out->makespan = mh;
    out->n_total = (uint64_t)total;
    out->n_better = acc.n_better;
    out->n_equal = acc.n_equal;
    out->n_worse = acc.n_worse;
    out->percentile = 100.0 * (double)(acc.n_worse + acc.n_equal) / (double)total;
    out->percentile_strict = 100.0 * (double)acc.n_worse / (double)total;
    out->speedup_over_worst = (double)out->max / (double)mh;
    out->deviation_from_optimal = (double)(mh - out->min) / (double)out->min;
    return ok();
}

ko_status ko_set_option(ko_gpu *g, int32_t key, int64_t value)
{
    if (!g) return fail(KO_ERR_ARG);
    switch (key) {
    case KO_OPT_LANES:
        if (value != 1 && value != 16 && value != 32) return fail(KO_ERR_ARG);
        g->fast.lanes = (int)value;
        break;
    case KO_OPT_LEVELS:
        if (value < 0 || value > 6) return fail(KO_ERR_ARG);
        g->fast.levels = (int)value;
        break;
    case KO_OPT_SIMPLE_ONLY:
        if (value != 0 && value != 1) return fail(KO_ERR_ARG);
        g->fast.disabled = value == 1;
        break;
    case KO_OPT_RUN_LIMIT:
        if (value < 1 || value > 32) return fail(KO_ERR_ARG);
        g->fast.run_limit = (int)value;
        break;
    case KO_OPT_STACK_GLOBAL:
        if (value != 0 && value != 1) return fail(KO_ERR_ARG);
        g->fast.stack_global = (int)value;
        break;
    case KO_OPT_LANE_STATE:
        if (value < 0 || value > 2) return fail(KO_ERR_ARG);
        g->fast.lane_shape = (int)value;
        break;
    default:
        return fail(KO_ERR_ARG);
    }
    return ok();
}

int64_t ko_get_option(const ko_gpu *g, int32_t key)
{
    if (!g) return fail(KO_ERR_ARG);
    switch (key) {
    case KO_OPT_LANES: return g->fast.lanes;
    case KO_OPT_LEVELS: return g->fast.levels;
    case KO_OPT_SIMPLE_ONLY: return g->fast.disabled ? 1 : 0;
    case KO_OPT_RUN_LIMIT: return g->fast.run_limit;
    case KO_OPT_STACK_GLOBAL: return g->fast.stack_global;
    case KO_OPT_LANE_STATE: return g->fast.lane_shape;
    default: return fail(KO_ERR_ARG);
    }
}

ko_status ko_autotune(ko_gpu *g, const char *cache_path, void *stream)
{
    if (!g || g->h.n < 1) return fail(KO_ERR_ARG);
    if (g->h.n > KO_MAX_EXHAUSTIVE) return fail(KO_ERR_TOO_LARGE);
    if (!ko_fast_applicable(g->h)) return ok();  // only the simple simulator applies
    cudaStream_t st = (cudaStream_t)stream;
    g->h.ref_makespan = 0;
    ko_status s = prepare(g, st);
    if (s) return fail(s);
    if ((s = upload_meta(g, st))) return fail(s);
    int lanes = 16, levels = 4, stack = 1, shape = 0;
    double rate = 0.0;
    s = ko_tune_set(&g->fast, g->h, g->d_set, g->d_acc, cache_path, st, &lanes, &levels, &stack, &shape, &rate);
    if (s) return fail(s);
    g->fast.lanes = lanes;
    g->fast.levels = levels;
    g->fast.stack_global = stack;
    g->fast.lane_shape = shape;
    return ok();
}

ko_status ko_batch_autotune(ko_gpu *const *sets, int32_t nsets, const char *cache_path, void *stream)
{
    if (!sets || nsets < 1) return fail(KO_ERR_ARG);
    std::vector<const KoSet *> hs(nsets);
    for (int i = 0; i < nsets; i++) {
        if (!sets[i] || sets[i]->h.n < 1) return fail(KO_ERR_ARG);
        if (sets[i]->h.n > KO_MAX_EXHAUSTIVE) return fail(KO_ERR_TOO_LARGE);
        if (!ko_fast_applicable(sets[i]->h)) return fail(KO_ERR_OVERFLOW);
        hs[i] = &sets[i]->h;
    }
    std::vector<int> lanes(nsets), levels(nsets), stack(nsets), shape(nsets);
    ko_status s = ko_tune_batch(hs.data(), nsets, cache_path, (cudaStream_t)stream, lanes.data(), levels.data(),
                                stack.data(), shape.data());
    if (s) return fail(s);
    for (int i = 0; i < nsets; i++) {
        sets[i]->fast.lanes = lanes[i];
        sets[i]->fast.levels = levels[i];
        sets[i]->fast.stack_global = stack[i];
        sets[i]->fast.lane_shape = shape[i];
    }
    return ok();
}

int64_t ko_last_fallback_items(const ko_gpu *g)
{
    if (!g) return -1;
    ko_gpu *m = const_cast<ko_gpu *>(g);
    if (m->fast_pending) {  // asynchronous launch: wait for it, then read its counters
        cudaDeviceSynchronize();
        fast_after_sync(m);
        m->fast_pending = false;
    }
    return (int64_t)g->fast.last_overflow;
}

ko_batch *ko_batch_create(ko_gpu *const *sets, int32_t nsets, int32_t nbins)
{
    if (!sets || nsets < 1) {
        fail(KO_ERR_ARG);
        return nullptr;
    }
    std::vector<const KoSet *> hs(nsets);
    std::vector<int> levels(nsets), lanes(nsets), stack(nsets), shape(nsets);
    for (int i = 0; i < nsets; i++) {
        if (!sets[i] || sets[i]->h.sampling != KO_SAMPLE_BURST_END) {
            fail(KO_ERR_ARG);
            return nullptr;
        }
        sets[i]->frozen = true;
        hs[i] = &sets[i]->h;
        levels[i] = sets[i]->fast.levels;
        lanes[i] = sets[i]->fast.lanes;
        stack[i] = sets[i]->fast.stack_global;
        shape[i] = sets[i]->fast.lane_shape;
    }
    ko_status err = KO_OK;
    ko_batch *b = ko_batch_build(hs.data(), levels.data(), lanes.data(), stack.data(), shape.data(), nsets, nbins,
                                 sets[0]->fast.run_limit, &err);
    if (!b) fail(err);
    else ok();
    return b;
}

ko_status ko_batch_run(ko_batch *b, ko_rank *out, uint64_t *hist, void *stream)
{
    if (!b || !out) return fail(KO_ERR_ARG);
    ko_status s = ko_batch_exec(b, out, hist, is_device_ptr(hist), (cudaStream_t)stream);
    return s ? fail(s) : ok();
}

int64_t ko_batch_orders(const ko_batch *b) { return b ? (int64_t)ko_batch_orders_impl(b) : -1; }

int64_t ko_batch_fallback_items(const ko_batch *b) { return b ? (int64_t)ko_batch_fallback(b) : -1; }

void ko_batch_destroy(ko_batch *b) { ko_batch_free(b); }

ko_model *ko_model_create(uint64_t seed)
{
    ko_status err = KO_OK;
    ko_model *m = ko_model_new(seed, &err);
    if (!m) fail(err);
    else ok();
    return m;
}

ko_status ko_model_get_params(const ko_model *m, float *params)
{
    if (!m || !params) return fail(KO_ERR_ARG);
    ko_status s = ko_model_store(m, params);
    return s ? fail(s) : ok();
}

ko_status ko_model_set_params(ko_model *m, const float *params)
{
    if (!m || !params) return fail(KO_ERR_ARG);
    ko_status s = ko_model_load(m, params);
    return s ? fail(s) : ok();
}

ko_status ko_model_predict(ko_model *m, const float *x, int64_t B, float *y, void *stream)
{
    if (!m || !x || !y || B < 64 || B % 64 || B > (1 << 24)) return fail(KO_ERR_ARG);
    ko_status s = ko_model_raw(m, x, nullptr, (int)B, y, nullptr, nullptr, 0.0f, (cudaStream_t)stream);
    return s ? fail(s) : ok();
}

ko_status ko_model_grad(ko_model *m, const float *x, const float *t, int64_t B, float *grad, float *loss,
                        void *stream)
{
    if (!m || !x || !t || !grad || B < 64 || B % 64 || B > (1 << 24)) return fail(KO_ERR_ARG);
    ko_status s = ko_model_raw(m, x, t, (int)B, nullptr, grad, loss, 0.0f, (cudaStream_t)stream);
    return s ? fail(s) : ok();
}

ko_status ko_model_train_step(ko_model *m, const float *x, const float *t, int64_t B, float lr, float *loss,
                              void *stream)
{
    if (!m || !x || !t || B < 64 || B % 64 || B > (1 << 24) || !(lr > 0.0f)) return fail(KO_ERR_ARG);
    ko_status s = ko_model_raw(m, x, t, (int)B, nullptr, nullptr, loss, lr, (cudaStream_t)stream);
    return s ? fail(s) : ok();
}

ko_status ko_model_encode(ko_gpu *g, const int8_t *orders, int64_t n, float *x_out, void *stream)
{
    if (!g || !orders || !x_out || n < 1 || g->h.n < 1) return fail(KO_ERR_ARG);
    for (int64_t i = 0; i < n * g->h.n; i++)
        if (orders[i] < 0 || orders[i] >= g->h.n) return fail(KO_ERR_ARG);
    ko_status s = ko_model_features(g->h, orders, n, x_out, (cudaStream_t)stream);
    return s ? fail(s) : ok();
}

ko_status ko_surrogate_train(ko_model *m, ko_gpu *const *sets, int32_t nsets, int64_t pairs_per_set,
                             int32_t steps, int32_t batch, float lr, uint64_t seed, float *loss_curve,
                             void *stream)
{
    if (!m || !sets || nsets < 1) return fail(KO_ERR_ARG);
    std::vector<const KoSet *> hs(nsets);
    for (int i = 0; i < nsets; i++) {
        if (!sets[i] || sets[i]->h.n < 1 || sets[i]->h.sampling != KO_SAMPLE_BURST_END) return fail(KO_ERR_ARG);
        sets[i]->frozen = true;
        hs[i] = &sets[i]->h;
    }
    ko_status s = ko_model_train_sets(m, hs.data(), nsets, pairs_per_set, steps, batch, lr, seed, loss_curve,
                                      (cudaStream_t)stream);
    return s ? fail(s) : ok();
}

ko_status ko_surrogate_propose(ko_model *m, ko_gpu *g, int64_t n_cand, int32_t top_k, uint64_t seed,
                               int32_t *best_order, int64_t *best_makespan, double *gpu_ms, void *stream)
{
    if (g && g->h.sampling != KO_SAMPLE_BURST_END) return fail(KO_ERR_ARG);
    if (!m || !g || !best_order || !best_makespan || g->h.n < 1) return fail(KO_ERR_ARG);
    g->frozen = true;
    ko_status s = ko_model_propose_set(m, g->h, n_cand, top_k, seed, best_order, best_makespan, gpu_ms,
                                       (cudaStream_t)stream);
    return s ? fail(s) : ok();
}

ko_status ko_surrogate_search(ko_model *m, ko_gpu *g, int64_t n_cand, int32_t top_k, int32_t rounds,
                              int32_t beam, uint64_t seed, int32_t *best_order, int64_t *best_makespan,
                              double *gpu_ms, void *stream)
{
    if (g && g->h.sampling != KO_SAMPLE_BURST_END) return fail(KO_ERR_ARG);
    if (!m || !g || !best_order || !best_makespan || g->h.n < 2) return fail(KO_ERR_ARG);
    g->frozen = true;
    ko_status s = ko_model_search_set(m, g->h, n_cand, top_k, rounds, beam, seed, best_order, best_makespan,
                                      gpu_ms, (cudaStream_t)stream);
    return s ? fail(s) : ok();
}

ko_status ko_random_search(ko_gpu *g, int64_t n_orders, uint64_t seed, int32_t *best_order,
                           int64_t *best_makespan, double *gpu_ms, void *stream)
{
    if (g && g->h.sampling != KO_SAMPLE_BURST_END) return fail(KO_ERR_ARG);
    if (!g || !best_order || !best_makespan || g->h.n < 1) return fail(KO_ERR_ARG);
    g->frozen = true;
    ko_status s = ko_random_search_set(&g->fast, g->h, n_orders, seed, best_order, best_makespan, gpu_ms,
                                       (cudaStream_t)stream);
    return s ? fail(s) : ok();
}

ko_status ko_local_search(ko_gpu *g, const int32_t *start, int32_t moves, int32_t max_iters, int32_t *order_out,
                          int64_t *makespan_out, int32_t *steps_out, int64_t *evals_out, double *gpu_ms,
                          void *stream)
{
    if (g && g->h.sampling != KO_SAMPLE_BURST_END) return fail(KO_ERR_ARG);
    if (!g || !order_out || !makespan_out || g->h.n < 1) return fail(KO_ERR_ARG);
    g->frozen = true;
    std::vector<int32_t> st0(g->h.n);
    if (start) std::copy(start, start + g->h.n, st0.begin());
    else ko_heuristic_host(g->h, st0.data());
    ko_status s = ko_local_search_set(&g->fast, g->h, st0.data(), moves != 0, max_iters, order_out, makespan_out,
                                      steps_out, evals_out, gpu_ms, (cudaStream_t)stream);
    return s ? fail(s) : ok();
}

ko_hw *ko_hw_create(const ko_hw_kernel *ks, int32_t n)
{
    ko_status err = KO_OK;
    ko_hw *h = ko_hw_build(ks, n, &err);
    if (!h) fail(err);
    else ok();
    return h;
}

ko_status ko_hw_device_limits(int32_t out[7])
{
    if (!out) return fail(KO_ERR_ARG);
    ko_status s = ko_hw_limits_impl(out);
    return s ? fail(s) : ok();
}

ko_status ko_hw_regs(int32_t kind, int32_t *regs_per_thread)
{
    if (!regs_per_thread || (kind != KO_HW_COMPUTE && kind != KO_HW_MEMORY)) return fail(KO_ERR_ARG);
    int r = 0;
    ko_status s = ko_hw_regs_impl(kind, &r);
    if (s) return fail(s);
    *regs_per_thread = r;
    return ok();
}

ko_status ko_hw_int_peak(int32_t turns, int64_t *lane_ops, float *ms_out)
{
    if (!lane_ops || !ms_out || turns < 1 || turns > (1 << 20)) return fail(KO_ERR_ARG);
    ko_status s = ko_hw_int_peak_impl(turns, lane_ops, ms_out);
    return s ? fail(s) : ok();
}

ko_status ko_hw_time_orders(ko_hw *h, const int8_t *orders, int64_t count, int32_t reps, float *ms_out)
{
    if (!h || count < 0 || (count > 0 && (!orders || !ms_out)) || reps < 1 || reps > 64) return fail(KO_ERR_ARG);
    ko_status s = ko_hw_time_impl(h, orders, count, reps, ms_out);
    return s ? fail(s) : ok();
}

ko_status ko_hw_time_grid(ko_hw *h, int32_t k, int32_t blocks, int32_t reps, float *ms_out)
{
    if (!h || !ms_out || k < 0 || k >= 8 || blocks < 1 || blocks > (1 << 20) || reps < 1 || reps > 64)
        return fail(KO_ERR_ARG);
    ko_status s = ko_hw_time_grid_impl(h, k, blocks, reps, ms_out);
    return s ? fail(s) : ok();
}

ko_status ko_hw_trace_order(ko_hw *h, const int8_t *order, uint64_t *trace_out, float *ms_out)
{
    if (!h || !order || !trace_out || !ms_out) return fail(KO_ERR_ARG);
    ko_status s = ko_hw_trace_impl(h, order, (unsigned long long *)trace_out, ms_out);
    return s ? fail(s) : ok();
}

int64_t ko_hw_trace_len(const ko_hw *h) { return h ? 4 * ko_hw_trace_blocks(h) : 0; }

void ko_hw_destroy(ko_hw *h) { ko_hw_free(h); }

ko_status ko_model_set_option(ko_model *m, int32_t key, int64_t value)
{
    if (!m) return fail(KO_ERR_ARG);
    ko_status s = ko_model_option(m, key, value);
    return s ? fail(s) : ok();
}

void ko_model_destroy(ko_model *m) { ko_model_free(m); }

ko_status ko_eval_orders_noalloc(const ko_gpu *g, const int8_t *orders, int64_t n, int64_t *makespan_out,
                                 void *stream)
{
    if (!g || n < 0 || g->h.n < 1 || (n > 0 && (!orders || !makespan_out))) return fail(KO_ERR_ARG);
    if (n == 0) return ok();
    if (!is_device_ptr(orders) || !is_device_ptr(makespan_out)) return fail(KO_ERR_ARG);
    ko_status s = ko_noalloc_eval(g->h, orders, n, makespan_out, (cudaStream_t)stream);
    return s ? fail(s) : ok();
}

void ko_destroy_gpu(ko_gpu *g) { delete g; }

const char *ko_status_str(ko_status s)
{
    switch (s) {
    case KO_OK: return "KO_OK";
    case KO_ERR_ARG: return "KO_ERR_ARG";
    case KO_ERR_NOFIT: return "KO_ERR_NOFIT";
    case KO_ERR_TOO_LARGE: return "KO_ERR_TOO_LARGE";
    case KO_ERR_OVERFLOW: return "KO_ERR_OVERFLOW";
    case KO_ERR_CUDA: return "KO_ERR_CUDA";
    case KO_ERR_TIMEOUT: return "KO_ERR_TIMEOUT";
    case KO_ERR_STATE: return "KO_ERR_STATE";
    case KO_ERR_NOMEM: return "KO_ERR_NOMEM";
    default: return "KO_ERR_UNKNOWN";
    }
}

ko_status ko_last_error(void) { return t_last_error; }

int64_t ko_kernel_launches(void) { return (int64_t)g_launches.load(); }

double ko_last_sim_ms(const ko_gpu *g)
{
    if (!g) return -1.0;
    ko_last_fallback_items(g);
    return g->fast.last_ms;
}

ko_status ko_transfer_bytes(const ko_gpu *g, int64_t *h2d, int64_t *d2h)
{
    if (!g || !h2d || !d2h) return fail(KO_ERR_ARG);
    *h2d = g->h2d + g->fast.h2d;
    *d2h = g->d2h + g->fast.d2h;
    return ok();
}

}  // extern "C"
