// Batched exhaustive scoring of many kernel sets in one persistent launch,
// replayed as a CUDA graph (ko_batch_create / ko_batch_run / ko_batch_destroy).
//
// The graph holds, in stream order:
//   1. reset of every set's accumulators;
//   2. one run-length pass evaluating each set's ranked order (Algorithm 1 by
//      default) into a per-set reference makespan;
//   3. one exhaustive launch per group of sets that share a simulator choice
//      (threads per simulation and node-state placement, per set from its
//      handle, usually picked per (N_SM class, N) by ko_batch_autotune): each
//      group's work items, chunks in decreasing order of estimated cost
//      (longest processing time first) so the largest sets start first and
//      small sets fill the tail; abandoned items go on to the later passes;
//   4. optionally, per-set histograms of the stored makespans;
//   5. copies of the accumulators and references to pinned host memory.
// No step waits on the host, so one cudaGraphLaunch runs the whole batch.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "ko_fast.h"
#include "ko_internal.h"

struct ko_batch {
    int nsets = 0;
    int nbins = 0;
    std::vector<KoSet> h_sets;
    std::vector<int> order_rows;      // heuristic order per set, KO_MAX_KERNELS bytes each
    std::vector<long long> ms_off;    // per-set offset into the makespan buffer
    long long ms_total = 0;
    KoSet *d_sets = nullptr;
    KoChunk *d_chunks = nullptr;      // [0, nsets): heuristic rows; [nsets, ...): exhaustive
    int n_ref_chunks = 0, n_ex_chunks = 0;
    long long n_ref_items = 0, n_ex_items = 0;
    int8_t *d_rows = nullptr;
    long long *d_refs = nullptr;
    KoAccum *d_accs = nullptr;
    int64_t *d_ms = nullptr;
    unsigned long long *d_hist = nullptr;
    KoAccum *h_accs = nullptr;        // pinned
    long long *h_refs = nullptr;      // pinned
    int levels_max = 1;
    struct Group {
        int lanes, stack, shape;  // shape: the one-thread pass's state size
        int chunk0, nchunks;      // into the exhaustive chunks
        long long n_items;
        int levels;               // deepest saved levels of its sets
    };
    std::vector<Group> groups;
    size_t slab = 0;
    KoFastState fast{};
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;

    ~ko_batch()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        cudaFree(d_sets); cudaFree(d_chunks); cudaFree(d_rows); cudaFree(d_refs); cudaFree(d_accs);
        cudaFree(d_ms); cudaFree(d_hist);
        cudaFreeHost(h_accs); cudaFreeHost(h_refs);
        ko_fast_release(&fast);
    }
};

namespace {

constexpr long long kFact[13] = {1, 1, 2, 6, 24, 120, 720, 5040, 40320, 362880, 3628800,
                                 39916800, 479001600};

// Relative cost of one order (events scale with the number of distinct SM
// runs, which grows with N_SM): used only to order the work.
double order_cost(const KoSet &h) { return h.S >= 64 ? 3.0 : 1.0; }

template <typename T>
bool dev_alloc(T **p, size_t count)
{
    if (cudaMalloc((void **)p, sizeof(T) * (count ? count : 1)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    return true;
}

ko_status enqueue(ko_batch *b, cudaStream_t st)
{
    if (ko_launch_accum_reset(b->d_accs, b->nsets, st) != cudaSuccess) return KO_ERR_CUDA;
    KoWork w{};
    w.sets = b->d_sets;
    w.chunks = b->d_chunks;
    w.nchunks = b->n_ref_chunks;
    w.n_items = b->n_ref_items;
    w.perms = b->d_rows;
    w.out = (int64_t *)b->d_refs;
    w.levels = 1;
    b->fast.lanes = 16;
    b->fast.stack_global = 1;
    ko_status s = ko_fast_launch(&b->fast, w, b->slab, st);
    if (s) return s;
    for (const ko_batch::Group &gr : b->groups) {
        KoWork x{};
        x.sets = b->d_sets;
        x.chunks = b->d_chunks + b->n_ref_chunks + gr.chunk0;
        x.nchunks = gr.nchunks;
        x.n_items = gr.n_items;
        x.refs = b->d_refs;
        x.accs = b->d_accs;
        x.out = b->d_ms;
        x.levels = gr.levels;
        b->fast.lanes = gr.lanes;
        b->fast.stack_global = gr.stack;
        b->fast.lane_shape = gr.shape;
        if ((s = ko_fast_launch(&b->fast, x, b->slab, st))) return s;
    }
    if (b->nbins > 0) {
        if (cudaMemsetAsync(b->d_hist, 0, sizeof(unsigned long long) * b->nbins * b->nsets, st) !=
            cudaSuccess)
            return KO_ERR_CUDA;
        for (int i = 0; i < b->nsets; i++) {
            if (ko_launch_histogram(b->d_ms + b->ms_off[i], kFact[b->h_sets[i].n], b->d_accs + i,
                                    b->d_hist + (size_t)i * b->nbins, b->nbins, st) != cudaSuccess)
                return KO_ERR_CUDA;
        }
    }
    if (cudaMemcpyAsync(b->h_accs, b->d_accs, sizeof(KoAccum) * b->nsets, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(b->h_refs, b->d_refs, sizeof(long long) * b->nsets, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
        return KO_ERR_CUDA;
    return KO_OK;
}

}  // namespace

ko_batch *ko_batch_build(const KoSet *const *sets, const int *levels, const int *lanes, const int *stack,
                         const int *shape, int nsets, int nbins, int run_limit, ko_status *err)
{
    *err = KO_OK;
    if (nsets < 1 || nbins < 0 || nbins > 32768) { *err = KO_ERR_ARG; return nullptr; }
    ko_batch *b = new (std::nothrow) ko_batch();
    if (!b) { *err = KO_ERR_NOMEM; return nullptr; }
    b->nsets = nsets;
    b->nbins = nbins;
    b->fast.run_limit = run_limit;
    b->h_sets.resize(nsets);
    std::vector<int8_t> rows((size_t)nsets * KO_MAX_KERNELS, 0);
    std::vector<KoChunk> chunks;
    for (int i = 0; i < nsets; i++) {
        KoSet h = *sets[i];
        if (h.n < 1 || h.n > KO_MAX_EXHAUSTIVE) { delete b; *err = h.n < 1 ? KO_ERR_ARG : KO_ERR_TOO_LARGE; return nullptr; }
        if (!ko_fast_applicable(h)) { delete b; *err = KO_ERR_OVERFLOW; return nullptr; }
        h.ref_makespan = 0;
        b->h_sets[i] = h;
        int32_t ord[KO_MAX_KERNELS];
        ko_heuristic_host(h, ord);
        for (int j = 0; j < h.n; j++) rows[(size_t)i * KO_MAX_KERNELS + j] = (int8_t)ord[j];
        KoChunk c{};
        c.first = i;
        c.count = 1;
        c.set = i;
        c.d0 = h.n;
        c.mode = 2;
        c.list_off = (long long)i * KO_MAX_KERNELS;
        c.out_off = i;
        chunks.push_back(c);
        b->slab = std::max(b->slab, ko_slab_bytes(h.S, h.Bk));
    }
    b->n_ref_chunks = nsets;
    b->n_ref_items = nsets;
    // exhaustive chunks: grouped by simulator choice, most expensive set first in each group
    std::vector<int> idx(nsets);
    std::iota(idx.begin(), idx.end(), 0);
    auto gkey = [&](int i) { return lanes[i] * 8 + shape[i] * 2 + (stack[i] ? 1 : 0); };
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
        if (gkey(x) != gkey(y)) return gkey(x) < gkey(y);
        return kFact[b->h_sets[x].n] * order_cost(b->h_sets[x]) > kFact[b->h_sets[y].n] * order_cost(b->h_sets[y]);
    });
    b->ms_off.assign(nsets, 0);
    long long off = 0;
    for (int i = 0; i < nsets; i++) {
        b->ms_off[i] = off;
        off += kFact[b->h_sets[i].n];
    }
    b->ms_total = off;
    long long first = 0, total_items = 0;
    for (int k = 0; k < nsets; k++) {
        const int i = idx[k];
        if (k == 0 || gkey(i) != gkey(idx[k - 1])) {
            b->groups.push_back(ko_batch::Group{lanes[i], stack[i] ? 1 : 0, shape[i], k, 0, 0, 1});
            first = 0;  // each group is its own launch, items counted from 0
        }
        ko_batch::Group &gr = b->groups.back();
        const KoSet &h = b->h_sets[i];
        int lv = levels[i];
        int d0 = h.n - 1 - lv;
        if (d0 < 0) d0 = 0;
        KoChunk c{};
        c.first = first;
        c.count = kFact[h.n] / kFact[h.n - d0];
        c.set = i;
        c.d0 = d0;
        c.mode = 0;
        c.out_off = b->ms_off[i];
        chunks.push_back(c);
        first += c.count;
        gr.nchunks++;
        gr.n_items = first;
        gr.levels = std::max(gr.levels, h.n - 1 - d0);
        b->levels_max = std::max(b->levels_max, h.n - 1 - d0);
        total_items += c.count;
    }
    b->n_ex_chunks = nsets;
    b->n_ex_items = total_items;
    bool okm = dev_alloc(&b->d_sets, nsets) && dev_alloc(&b->d_chunks, chunks.size()) &&
               dev_alloc(&b->d_rows, rows.size()) && dev_alloc(&b->d_refs, nsets) &&
               dev_alloc(&b->d_accs, nsets) && (nbins == 0 || dev_alloc(&b->d_ms, b->ms_total)) &&
               (nbins == 0 || dev_alloc(&b->d_hist, (size_t)nbins * nsets));
    if (!okm || cudaMallocHost((void **)&b->h_accs, sizeof(KoAccum) * nsets) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_refs, sizeof(long long) * nsets) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        *err = KO_ERR_NOMEM;
        return nullptr;
    }
    if (cudaMemcpy(b->d_sets, b->h_sets.data(), sizeof(KoSet) * nsets, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_chunks, chunks.data(), sizeof(KoChunk) * chunks.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(b->d_rows, rows.data(), rows.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        *err = KO_ERR_CUDA;
        return nullptr;
    }
    // allocate the simulators' buffers outside capture: one empty launch with
    // the reference-order pass's choice (16 lanes, global slab, 1 level), then
    // one per group, each with its choice, its deepest levels and the longest list
    long long longest = b->n_ref_items;
    for (const ko_batch::Group &gr : b->groups) longest = std::max(longest, gr.n_items);
    std::vector<ko_batch::Group> sizing;
    sizing.push_back(ko_batch::Group{16, 1, 0, 0, 0, 0, 1});
    sizing.insert(sizing.end(), b->groups.begin(), b->groups.end());
    for (const ko_batch::Group &gr : sizing) {
        KoWork none{};
        none.sets = b->d_sets;
        none.chunks = b->d_chunks;
        none.nchunks = 1;
        none.n_items = 0;
        none.levels = gr.levels;
        none.reserve_items = longest;
        b->fast.lanes = gr.lanes;
        b->fast.stack_global = gr.stack;
        b->fast.lane_shape = gr.shape;
        if (ko_fast_launch(&b->fast, none, b->slab, b->cap_stream) != KO_OK ||
            cudaStreamSynchronize(b->cap_stream) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            *err = KO_ERR_CUDA;
            return nullptr;
        }
    }
    // capture the whole batch once
    if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        *err = KO_ERR_CUDA;
        return nullptr;
    }
    ko_status s = enqueue(b, b->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
    if (s != KO_OK || e != cudaSuccess || !graph) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        delete b;
        *err = s ? s : KO_ERR_CUDA;
        return nullptr;
    }
    b->graph = graph;
    if (cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        *err = KO_ERR_CUDA;
        return nullptr;
    }
    return b;
}

ko_status ko_batch_exec(ko_batch *b, ko_rank *out, uint64_t *hist, bool hist_dev, cudaStream_t st)
{
    if (cudaGraphLaunch(b->exec, st) != cudaSuccess) {
        cudaGetLastError();
        return KO_ERR_CUDA;
    }
    // reset, the reference-order passes (three), each group's passes (three, four with the one-thread pass)
    ko_count_launch(b->nsets * (b->nbins > 0 ? 1 : 0) + 4 + 3 * (int)b->groups.size() +
                    (int)std::count_if(b->groups.begin(), b->groups.end(),
                                       [](const ko_batch::Group &g) { return g.lanes == 1; }));
    if (hist && b->nbins > 0) {
        const size_t bytes = sizeof(unsigned long long) * b->nbins * b->nsets;
        if (cudaMemcpyAsync(hist, b->d_hist, bytes, hist_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            st) != cudaSuccess)
            return KO_ERR_CUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return KO_ERR_CUDA;
    unsigned long long cnt[2] = {0, 0};
    const unsigned long long *dc = ko_fast_overflow_counter(&b->fast);
    if (dc && cudaMemcpy(cnt, dc, sizeof(cnt), cudaMemcpyDeviceToHost) == cudaSuccess)
        b->fast.last_overflow = cnt[0];
    if (cnt[0] > b->fast.ov_cap || cnt[1] > b->fast.ov_cap) return KO_ERR_STATE;  // cannot happen
    for (int i = 0; i < b->nsets; i++) {
        const KoAccum &a = b->h_accs[i];
        const long long mh = b->h_refs[i];
        const long long total = kFact[b->h_sets[i].n];
        if (a.failed || mh < 0) return KO_ERR_STATE;
        ko_rank &r = out[i];
        r.min = (int64_t)a.min;
        r.max = (int64_t)a.max;
        r.makespan = mh;
        r.n_total = (uint64_t)total;
        r.n_better = a.n_better;
        r.n_equal = a.n_equal;
        r.n_worse = a.n_worse;
        r.percentile = 100.0 * (double)(a.n_worse + a.n_equal) / (double)total;
        r.percentile_strict = 100.0 * (double)a.n_worse / (double)total;
        r.speedup_over_worst = (double)r.max / (double)mh;
        r.deviation_from_optimal = (double)(mh - r.min) / (double)r.min;
    }
    return KO_OK;
}

int ko_batch_size(const ko_batch *b) { return b->nsets; }
int ko_batch_nbins(const ko_batch *b) { return b->nbins; }
long long ko_batch_orders_impl(const ko_batch *b)
{
    long long t = 0;
    for (const KoSet &h : b->h_sets) t += kFact[h.n];
    return t;
}
unsigned long long ko_batch_fallback(const ko_batch *b) { return b->fast.last_overflow; }

void ko_batch_free(ko_batch *b) { delete b; }
