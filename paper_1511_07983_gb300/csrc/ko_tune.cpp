// Autotuner of the exhaustive simulators: picks the threads per simulation
// (1: one thread per order with its state in shared-memory columns; 16 or 32:
// the run-length simulator with its state packed in registers, one run per
// lane), where the run-length simulator keeps its saved DFS node states (a
// global slab or shared memory), and the prefix-sharing depth (saved DFS
// levels), per (N_SM class, N), by timing the candidates on the same orders,
// and caches the choice in a small JSON file.
//
// Two tuners share the candidates and the cache:
//   ko_tune_set    one handle: a calibration slice of its own exhaustive space;
//   ko_tune_batch  a batch: per class, a sample of the batch's own sets of that
//                  class run together as one launch (enough of them that the
//                  launch fills the GPU), so small sets are timed the way a
//                  batch runs them, not by their launch overhead.
//
// Cache format (one object, one entry per key; batch entries start with "B_"):
//   {"S160_N12": {"lanes": 16, "levels": 4, "stack": 1, "orders_per_s": 8.4e7}, ...}
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "ko_fast.h"
#include "ko_internal.h"

namespace {

struct Choice {
    int lanes = 16, levels = 4, stack = 1, shape = 0;  // shape: the one-thread pass's state size
    double rate = 0.0;
};

constexpr long long kFact[13] = {1, 1, 2, 6, 24, 120, 720, 5040, 40320, 362880, 3628800,
                                 39916800, 479001600};

std::string key_of(const KoSet &h)
{
    const int s_class = h.S <= 16 ? 16 : h.S <= 32 ? 32 : h.S <= 64 ? 64 : h.S <= 128 ? 128 : h.S <= 160 ? 160 : 1024;
    char buf[64];
    std::snprintf(buf, sizeof(buf), "S%d_N%d", s_class, h.n);
    return buf;
}

// Minimal reader for the format above (keys, two ints and one double each).
std::map<std::string, Choice> read_cache(const char *path)
{
    std::map<std::string, Choice> m;
    if (!path) return m;
    FILE *f = std::fopen(path, "r");
    if (!f) return m;
    std::string text;
    char buf[4096];
    size_t r;
    while ((r = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, r);
    std::fclose(f);
    size_t pos = 0;
    for (;;) {
        const size_t q0 = text.find('"', pos);
        if (q0 == std::string::npos) break;
        const size_t q1 = text.find('"', q0 + 1);
        if (q1 == std::string::npos) break;
        const std::string key = text.substr(q0 + 1, q1 - q0 - 1);
        const size_t close = text.find('}', q1);
        if (key.empty() || (key[0] != 'S' && key[0] != 'B') || close == std::string::npos) {
            pos = q1 + 1;
            continue;
        }
        const std::string body = text.substr(q1, close - q1);
        Choice c;
        int lanes = 0, levels = -1, stack = 1, shape = 0;
        double rate = 0.0;
        const size_t pl = body.find("\"lanes\":"), pv = body.find("\"levels\":"),
                     pr = body.find("\"orders_per_s\":"), ps = body.find("\"stack\":"),
                     ph = body.find("\"shape\":");
        if (pl != std::string::npos) lanes = std::atoi(body.c_str() + pl + 8);
        if (pv != std::string::npos) levels = std::atoi(body.c_str() + pv + 9);
        if (pr != std::string::npos) rate = std::atof(body.c_str() + pr + 15);
        if (ps != std::string::npos) stack = std::atoi(body.c_str() + ps + 8);
        if (ph != std::string::npos) shape = std::atoi(body.c_str() + ph + 8);
        if ((lanes == 1 || lanes == 16 || lanes == 32) && levels >= 0 && levels <= 6 && (stack == 0 || stack == 1) &&
            shape >= 0 && shape <= 2) {
            c.lanes = lanes;
            c.levels = levels;
            c.stack = stack;
            c.shape = shape;
            c.rate = rate;
            m[key] = c;
        }
        pos = close + 1;
    }
    return m;
}

void write_cache(const char *path, const std::map<std::string, Choice> &m)
{
    if (!path) return;
    std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "{\n");
    size_t i = 0;
    for (const auto &kv : m) {
        std::fprintf(f,
                     "  \"%s\": {\"lanes\": %d, \"levels\": %d, \"stack\": %d, \"shape\": %d, \"orders_per_s\": %.6g}%s\n",
                     kv.first.c_str(), kv.second.lanes, kv.second.levels, kv.second.stack, kv.second.shape,
                     kv.second.rate, ++i < m.size() ? "," : "");
    }
    std::fprintf(f, "}\n");
    std::fclose(f);
    std::rename(tmp.c_str(), path);
}

}  // namespace

// Calibration slice, the same orders for every candidate so that no depth is
// timed on an easier part of the space: the whole space when N! <= 64M orders,
// else kSliceChunks ranges of equal length spread evenly over the space, each
// starting and ending on a multiple of 720 = 6! orders -- a multiple of the
// span (levels + 1)! of every candidate depth (levels <= 5).
constexpr int kSliceChunks = 16;
constexpr long long kSliceOrders = 64000000;
constexpr long long kSpanAll = 720;

// Chunks of the slice for a candidate with prefix depth d0; returns the items.
long long ko_tune_chunks(int n, int d0, std::vector<KoChunk> &out)
{
    out.clear();
    const long long span = kFact[n - d0];
    const long long total = kFact[n];
    if (total <= kSliceOrders) {
        KoChunk c{};
        c.count = total / span;
        c.d0 = d0;
        out.push_back(c);
        return c.count;
    }
    const long long len = kSliceOrders / kSliceChunks / kSpanAll * kSpanAll;
    long long first = 0;
    for (int k = 0; k < kSliceChunks; k++) {
        const long long start = (long long)((__int128)total * k / kSliceChunks / kSpanAll) * kSpanAll;
        KoChunk c{};
        c.first = first;
        c.count = len / span;
        c.d0 = d0;
        c.list_off = start / span;
        out.push_back(c);
        first += c.count;
    }
    return first;
}

// Times one launch over `w` with the candidate's lanes and node-state
// placement (best of `reps`); returns orders per second (0 on failure).
static double time_candidate(KoFastState *fs, const KoWork &w, KoAccum *d_acc, int nacc, long long orders,
                             int lanes, int stack, int shape, size_t slab, int reps, cudaStream_t st)
{
    const int saved_lanes = fs->lanes, saved_stack = fs->stack_global, saved_shape = fs->lane_shape;
    fs->lanes = lanes;
    fs->stack_global = stack;
    fs->lane_shape = shape;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double rate = 0.0;
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        for (int rep = 0; rep < reps; rep++) {
            if (ko_launch_accum_reset(d_acc, nacc, st) != cudaSuccess) break;
            cudaEventRecord(e0, st);
            if (ko_fast_launch(fs, w, slab, st) != KO_OK) break;
            cudaEventRecord(e1, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) break;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms > 0.0f) rate = std::max(rate, (double)orders / (ms * 1e-3));
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaGetLastError();
    fs->lanes = saved_lanes;
    fs->stack_global = saved_stack;
    fs->lane_shape = saved_shape;
    return rate;
}

// The candidates: one thread per order (node states always in the global
// slab) with each of the three state shapes (14 runs / 56 group slots at 288
// simulations per SM, 12 / 40 at 352, 10 / 32 at 448), or 16 / 32 lanes with
// node states in the global slab or in shared memory; 1 .. min(N - 1, 5)
// saved levels each.
static std::vector<Choice> candidates(int n)
{
    std::vector<Choice> c;
    const int max_levels = n - 1 < 5 ? n - 1 : 5;
    for (int levels = 1; levels <= (max_levels > 1 ? max_levels : 1); levels++) {
        for (int shape : {0, 1, 2}) c.push_back(Choice{1, levels, 1, shape, 0.0});
        for (int lanes : {16, 32})
            for (int stack : {1, 0}) c.push_back(Choice{lanes, levels, stack, 0, 0.0});
    }
    return c;
}

// Times one candidate on the calibration slice of one set.  d_set / d_chunks /
// d_acc are device scratch of the caller (d_chunks holds kSliceChunks entries).
double ko_tune_measure(KoFastState *fs, const KoSet &h, const KoSet *d_set, KoChunk *d_chunks,
                       KoAccum *d_acc, const Choice &cand, int reps, cudaStream_t st)
{
    const int n = h.n;
    int d0 = n - 1 - cand.levels;
    if (d0 < 0) d0 = 0;
    const long long span = kFact[n - d0];
    if (span > kSpanAll) return 0.0;
    std::vector<KoChunk> chunks;
    const long long items = ko_tune_chunks(n, d0, chunks);
    if (items <= 0) return 0.0;
    if (cudaMemcpyAsync(d_chunks, chunks.data(), sizeof(KoChunk) * chunks.size(), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return 0.0;
    KoWork w{};
    w.sets = d_set;
    w.chunks = d_chunks;
    w.nchunks = (int)chunks.size();
    w.n_items = items;
    w.accs = d_acc;
    w.levels = n - 1 - d0 > 0 ? n - 1 - d0 : 1;
    return time_candidate(fs, w, d_acc, 1, items * span, cand.lanes, cand.stack, cand.shape, ko_slab_bytes(h.S, h.Bk),
                          reps, st);
}

// Pick lanes / levels / node-state placement for the handle's set.
ko_status ko_tune_set(KoFastState *fs, const KoSet &h, const KoSet *d_set, KoAccum *d_acc,
                      const char *cache_path, cudaStream_t st, int *lanes_out, int *levels_out,
                      int *stack_out, int *shape_out, double *rate_out)
{
    const std::string key = key_of(h);
    std::map<std::string, Choice> cache = read_cache(cache_path);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *lanes_out = it->second.lanes;
        *levels_out = it->second.levels;
        *stack_out = it->second.stack;
        *shape_out = it->second.shape;
        *rate_out = it->second.rate;
        return KO_OK;
    }
    Choice best;
    best.rate = -1.0;
    KoChunk *d_chunks = nullptr;
    if (cudaMalloc((void **)&d_chunks, sizeof(KoChunk) * kSliceChunks) != cudaSuccess) {
        cudaGetLastError();
        return KO_ERR_NOMEM;
    }
    bool warmed = false;
    for (const Choice &c : candidates(h.n)) {
        const double r = ko_tune_measure(fs, h, d_set, d_chunks, d_acc, c, warmed ? 1 : 2, st);
        warmed = true;
        if (r > best.rate) {
            best = c;
            best.rate = r;
        }
    }
    cudaFree(d_chunks);
    if (best.rate <= 0.0) return KO_ERR_CUDA;
    cache[key] = best;
    write_cache(cache_path, cache);
    *lanes_out = best.lanes;
    *levels_out = best.levels;
    *stack_out = best.stack;
    *shape_out = best.shape;
    *rate_out = best.rate;
    return KO_OK;
}

// Per-class choices for a batch.  For every (N_SM class, N) class of the
// batch with at least kBatchMinOrders orders, up to kBatchSample of its sets
// (the first ones, until kBatchOrders orders) run together as one exhaustive
// launch per candidate; classes below that size keep the default.
constexpr long long kBatchMinOrders = 1ll << 21;
constexpr long long kBatchOrders = 1ll << 22;
constexpr int kBatchSample = 64;

ko_status ko_tune_batch(const KoSet *const *hs, int nsets, const char *cache_path, cudaStream_t st,
                        int *lanes_out, int *levels_out, int *stack_out, int *shape_out)
{
    std::map<std::string, std::vector<int>> classes;
    for (int i = 0; i < nsets; i++) classes["B_" + key_of(*hs[i])].push_back(i);
    std::map<std::string, Choice> cache = read_cache(cache_path);
    bool dirty = false;
    KoSet *d_sets = nullptr;
    KoChunk *d_chunks = nullptr;
    KoAccum *d_accs = nullptr;
    if (cudaMalloc((void **)&d_sets, sizeof(KoSet) * kBatchSample) != cudaSuccess ||
        cudaMalloc((void **)&d_chunks, sizeof(KoChunk) * kBatchSample) != cudaSuccess ||
        cudaMalloc((void **)&d_accs, sizeof(KoAccum) * kBatchSample) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_sets); cudaFree(d_chunks); cudaFree(d_accs);
        return KO_ERR_NOMEM;
    }
    ko_status status = KO_OK;
    KoFastState fs{};
    for (const auto &kv : classes) {
        const std::vector<int> &members = kv.second;
        const KoSet &h0 = *hs[members[0]];
        Choice choice;
        choice.levels = h0.n - 1 < 4 ? h0.n - 1 : 4;
        auto it = cache.find(kv.first);
        const long long class_orders = (long long)members.size() * kFact[h0.n];
        if (it != cache.end()) {
            choice = it->second;
        } else if (class_orders >= kBatchMinOrders) {
            std::vector<KoSet> sample;
            long long orders = 0;
            for (int i : members) {
                if ((int)sample.size() >= kBatchSample || orders >= kBatchOrders) break;
                sample.push_back(*hs[i]);
                orders += kFact[hs[i]->n];
            }
            size_t slab = 0;
            for (const KoSet &x : sample) slab = std::max(slab, ko_slab_bytes(x.S, x.Bk));
            if (cudaMemcpyAsync(d_sets, sample.data(), sizeof(KoSet) * sample.size(), cudaMemcpyHostToDevice,
                                st) != cudaSuccess) {
                status = KO_ERR_CUDA;
                break;
            }
            Choice best;
            best.rate = -1.0;
            bool warmed = false;
            for (const Choice &c : candidates(h0.n)) {
                std::vector<KoChunk> chunks;
                long long first = 0;
                const int d0 = std::max(0, h0.n - 1 - c.levels);
                for (int j = 0; j < (int)sample.size(); j++) {
                    KoChunk ch{};
                    ch.first = first;
                    ch.count = kFact[sample[j].n] / kFact[sample[j].n - d0];
                    ch.set = j;
                    ch.d0 = d0;
                    chunks.push_back(ch);
                    first += ch.count;
                }
                if (cudaMemcpyAsync(d_chunks, chunks.data(), sizeof(KoChunk) * chunks.size(),
                                    cudaMemcpyHostToDevice, st) != cudaSuccess)
                    break;
                KoWork w{};
                w.sets = d_sets;
                w.chunks = d_chunks;
                w.nchunks = (int)chunks.size();
                w.n_items = first;
                w.accs = d_accs;
                w.levels = std::max(1, h0.n - 1 - d0);
                const double r = time_candidate(&fs, w, d_accs, (int)sample.size(), orders, c.lanes, c.stack,
                                                c.shape, slab, warmed ? 1 : 2, st);
                warmed = true;
                if (r > best.rate) {
                    best = c;
                    best.rate = r;
                }
            }
            if (best.rate <= 0.0) {
                status = KO_ERR_CUDA;
                break;
            }
            choice = best;
            cache[kv.first] = best;
            dirty = true;
        }
        for (int i : members) {
            lanes_out[i] = choice.lanes;
            levels_out[i] = choice.levels;
            stack_out[i] = choice.stack;
            shape_out[i] = choice.shape;
        }
    }
    ko_fast_release(&fs);
    cudaFree(d_sets); cudaFree(d_chunks); cudaFree(d_accs);
    if (status == KO_OK && dirty) write_cache(cache_path, cache);
    return status;
}
