// Autotuner for the run-length simulator: picks the lanes per simulation
// (16 or 32) and the prefix-sharing depth (saved DFS levels) per
// (N_SM class, N) by timing a calibration slice of the handle's own
// exhaustive space, and caches the choice in a small JSON file.
//
// Cache format (one object, one entry per key):
//   {"S148_N12": {"lanes": 32, "levels": 4, "orders_per_s": 2.8e7}, ...}
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "ko_fast.h"
#include "ko_internal.h"

namespace {

struct Choice {
    int lanes = 16, levels = 4;
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
        if (key.empty() || key[0] != 'S' || close == std::string::npos) {
            pos = q1 + 1;
            continue;
        }
        const std::string body = text.substr(q1, close - q1);
        Choice c;
        int lanes = 0, levels = -1;
        double rate = 0.0;
        const size_t pl = body.find("\"lanes\":"), pv = body.find("\"levels\":"),
                     pr = body.find("\"orders_per_s\":");
        if (pl != std::string::npos) lanes = std::atoi(body.c_str() + pl + 8);
        if (pv != std::string::npos) levels = std::atoi(body.c_str() + pv + 9);
        if (pr != std::string::npos) rate = std::atof(body.c_str() + pr + 15);
        if ((lanes == 16 || lanes == 32) && levels >= 0 && levels <= 6) {
            c.lanes = lanes;
            c.levels = levels;
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
        std::fprintf(f, "  \"%s\": {\"lanes\": %d, \"levels\": %d, \"orders_per_s\": %.6g}%s\n",
                     kv.first.c_str(), kv.second.lanes, kv.second.levels, kv.second.rate,
                     ++i < m.size() ? "," : "");
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

// Times one candidate on the calibration slice; returns orders per second
// (0 on failure).  d_set / d_chunks / d_acc are device scratch of the caller
// (d_chunks holds kSliceChunks entries).
double ko_tune_measure(KoFastState *fs, const KoSet &h, const KoSet *d_set, KoChunk *d_chunks,
                       KoAccum *d_acc, int lanes, int levels, int reps, cudaStream_t st)
{
    const int n = h.n;
    int d0 = n - 1 - levels;
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
    const int saved_lanes = fs->lanes;
    fs->lanes = lanes;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        fs->lanes = saved_lanes;
        return 0.0;
    }
    double rate = 0.0;
    for (int rep = 0; rep < reps; rep++) {
        if (ko_launch_accum_reset(d_acc, 1, st) != cudaSuccess) break;
        cudaEventRecord(e0, st);
        if (ko_fast_launch(fs, w, ko_slab_bytes(h.S, h.Bk), st) != KO_OK) break;
        cudaEventRecord(e1, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms > 0.0f) rate = (double)(items * span) / (ms * 1e-3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    fs->lanes = saved_lanes;
    return rate;
}

// Pick lanes/levels for the handle's set; returns KO_OK and the choice.
ko_status ko_tune_set(KoFastState *fs, const KoSet &h, const KoSet *d_set, KoAccum *d_acc,
                      const char *cache_path, cudaStream_t st, int *lanes_out, int *levels_out,
                      double *rate_out)
{
    const std::string key = key_of(h);
    std::map<std::string, Choice> cache = read_cache(cache_path);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *lanes_out = it->second.lanes;
        *levels_out = it->second.levels;
        *rate_out = it->second.rate;
        return KO_OK;
    }
    Choice best;
    best.rate = -1.0;
    const int max_levels = h.n - 1 < 5 ? h.n - 1 : 5;
    KoChunk *d_chunks = nullptr;
    if (cudaMalloc((void **)&d_chunks, sizeof(KoChunk) * kSliceChunks) != cudaSuccess) {
        cudaGetLastError();
        return KO_ERR_NOMEM;
    }
    bool warmed = false;
    for (int lanes : {32, 16}) {
        for (int levels = 1; levels <= (max_levels > 1 ? max_levels : 1); levels++) {
            const double r = ko_tune_measure(fs, h, d_set, d_chunks, d_acc, lanes, levels, warmed ? 1 : 2, st);
            warmed = true;
            if (r > best.rate) {
                best.rate = r;
                best.lanes = lanes;
                best.levels = levels;
            }
        }
    }
    cudaFree(d_chunks);
    if (best.rate <= 0.0) return KO_ERR_CUDA;
    cache[key] = best;
    write_cache(cache_path, cache);
    *lanes_out = best.lanes;
    *levels_out = best.levels;
    *rate_out = best.rate;
    return KO_OK;
}
