// Simple exact simulator: one thread simulates one launch order from t = 0,
// block by block, with per-SM state in a per-thread scratch slab.
//
// It is the general path (any N_SM, any number of distinct SM states) used for
// explicit order lists and as the fallback of the run-length simulator.
//
// Model (Sec. 2 dispatch rule; Sec. 4 balance; durations fixed per burst):
//   queue   blocks of order[0], then order[1], ... (strict FIFO)
//   burst   the head block goes to the first SM, cyclically from the
//           round-robin pointer p, that still fits its registers, shared
//           memory, warps and one more block; p moves past that SM; a head
//           that fits nowhere ends the burst (no overtaking)
//   timing  blocks started in a burst on an SM last
//           max(ceil(c*max(SumC,Ccap)/Ccap), ceil(m*max(SumM,Mcap)/Mcap))
//           with SumC/SumM over the SM's residents after the burst
//   events  t jumps to the earliest end; everything ending then is released
//           before the next burst; the makespan is the last end.
// Blocks of one kernel that start together on one SM share their end time and
// are kept as one group (kernel, count, end).
#include <mutex>

#include "ko_internal.h"
#include "ko_fast.h"

namespace {

__constant__ unsigned long long c_fact[21] = {
    1ull, 1ull, 2ull, 6ull, 24ull, 120ull, 720ull, 5040ull, 40320ull, 362880ull, 3628800ull,
    39916800ull, 479001600ull, 6227020800ull, 87178291200ull, 1307674368000ull,
    20922789888000ull, 355687428096000ull, 6402373705728000ull, 121645100408832000ull,
    2432902008176640000ull};

constexpr int kThreads = 128;

__device__ __forceinline__ int64_t div_up_cap(int64_t x, int64_t cap, int shift)
{
    return shift >= 0 ? ((x + cap - 1) >> shift) : (x + cap - 1) / cap;
}

__device__ __forceinline__ int64_t block_duration(const KoSet &d, int32_t c, int32_t m,
                                                  int64_t sum_c, int64_t sum_m)
{
    int64_t a = div_up_cap((int64_t)c * (sum_c > d.ccap ? sum_c : d.ccap), d.ccap, d.cshift);
    int64_t b = div_up_cap((int64_t)m * (sum_m > d.mcap ? sum_m : d.mcap), d.mcap, d.mshift);
    return a > b ? a : b;
}

// Lexicographic Lehmer unrank: digit j = k / (n-1-j)!, pick the digit-th
// smallest unused kernel id.
__device__ void unrank(int n, unsigned long long k, int8_t *perm)
{
    uint32_t unused = (n >= 32) ? 0xffffffffu : ((1u << n) - 1u);
    for (int j = 0; j < n; j++) {
        unsigned long long f = c_fact[n - 1 - j];
        uint32_t dgt = (uint32_t)(k / f);
        k -= (unsigned long long)dgt * f;
        uint32_t u = unused;
        for (uint32_t q = 0; q < dgt; q++) u &= u - 1u;
        int v = __ffs(u) - 1;
        perm[j] = (int8_t)v;
        unused &= ~(1u << v);
    }
}

// Slab layout for one thread (S SMs, G = Bk group slots per SM):
//   int64 sum_c[S], sum_m[S], gend[S*G]; int32 ur[S], us[S], uw[S], ub[S], ng[S], gk[S*G]
struct Slab {
    int64_t *sum_c, *sum_m, *gend;
    int32_t *ur, *us, *uw, *ub, *ng, *gk;
};

__host__ __device__ inline size_t slab_bytes(int S, int G)
{
    size_t b = (size_t)S * (2 + G) * sizeof(int64_t) + (size_t)S * (5 + G) * sizeof(int32_t);
    return (b + 255) & ~(size_t)255;
}

__device__ Slab slab_at(void *base, size_t per_thread, int S, int G, long long slot)
{
    char *p = (char *)base + per_thread * (size_t)slot;
    Slab s;
    s.sum_c = (int64_t *)p; p += sizeof(int64_t) * S;
    s.sum_m = (int64_t *)p; p += sizeof(int64_t) * S;
    s.gend = (int64_t *)p; p += sizeof(int64_t) * S * G;
    s.ur = (int32_t *)p; p += sizeof(int32_t) * S;
    s.us = (int32_t *)p; p += sizeof(int32_t) * S;
    s.uw = (int32_t *)p; p += sizeof(int32_t) * S;
    s.ub = (int32_t *)p; p += sizeof(int32_t) * S;
    s.ng = (int32_t *)p; p += sizeof(int32_t) * S;
    s.gk = (int32_t *)p;
    return s;
}

// group word: kernel id (bits 0-7) | pending flag (bit 8) | block count (bits 16-31)
constexpr int32_t kPending = 1 << 8;

// Makespan of one order, -1 if it cannot finish.
__device__ int64_t simulate(const KoSet &d, const int8_t *perm, Slab st)
{
    const int n = d.n, S = d.S, G = d.Bk;
    for (int s = 0; s < S; s++) {
        st.sum_c[s] = 0; st.sum_m[s] = 0;
        st.ur[s] = 0; st.us[s] = 0; st.uw[s] = 0; st.ub[s] = 0; st.ng[s] = 0;
    }
    long long total_blocks = 0;
    for (int i = 0; i < n; i++) total_blocks += d.k[i].b;
    int64_t t = 0, makespan = 0;
    int p = 0, pos = 0;
    int32_t left = n > 0 ? d.k[perm[0]].b : 0;
    long long events = 0;
    for (;;) {
        // release every group ending at t
        for (int s = 0; s < S; s++) {
            int g = st.ng[s];
            for (int j = 0; j < g;) {
                if (st.gend[s * G + j] == t) {
                    int32_t w = st.gk[s * G + j];
                    const KoKern &K = d.k[w & 0xff];
                    int32_t cnt = w >> 16;
                    st.ur[s] -= cnt * K.r; st.us[s] -= cnt * K.s; st.uw[s] -= cnt * K.w;
                    st.ub[s] -= cnt;
                    st.sum_c[s] -= (int64_t)cnt * K.c; st.sum_m[s] -= (int64_t)cnt * K.m;
                    g--;
                    st.gk[s * G + j] = st.gk[s * G + g];
                    st.gend[s * G + j] = st.gend[s * G + g];
                } else {
                    j++;
                }
            }
            st.ng[s] = g;
        }
        // one dispatch burst
        while (pos < n) {
            const int kid = perm[pos];
            const KoKern &K = d.k[kid];
            int found = -1;
            for (int off = 0, s = p; off < S; off++) {
                if (st.ur[s] + K.r <= d.R && st.us[s] + K.s <= d.Sh && st.uw[s] + K.w <= d.W &&
                    st.ub[s] + 1 <= d.Bk) {
                    found = s;
                    break;
                }
                if (++s == S) s = 0;
            }
            if (found < 0) break;
            const int s = found;
            st.ur[s] += K.r; st.us[s] += K.s; st.uw[s] += K.w; st.ub[s] += 1;
            st.sum_c[s] += K.c; st.sum_m[s] += K.m;
            int g = st.ng[s], j = 0;
            if (d.sampling == KO_SAMPLE_AT_PLACEMENT) {
                // duration fixed now, from the totals with this block and without later ones;
                // blocks of one kernel ending together share a group
                const int64_t e = t + block_duration(d, K.c, K.m, st.sum_c[s], st.sum_m[s]);
                while (j < g && !((st.gk[s * G + j] & 0xffff) == kid && st.gend[s * G + j] == e)) j++;
                if (j == g) {
                    st.gk[s * G + g] = kid;
                    st.gend[s * G + g] = e;
                    st.ng[s] = g + 1;
                }
                if (e > makespan) makespan = e;
            } else {
                while (j < g && (st.gk[s * G + j] & 0xffff) != (kid | kPending)) j++;
                if (j == g) {
                    st.gk[s * G + g] = kid | kPending;
                    st.gend[s * G + g] = 0;
                    st.ng[s] = g + 1;
                }
            }
            st.gk[s * G + j] += 1 << 16;
            p = (s + 1 == S) ? 0 : s + 1;
            if (--left == 0) {
                pos++;
                left = pos < n ? d.k[perm[pos]].b : 0;
            }
        }
        // fix the durations of the groups started in this burst
        int64_t tmin = INT64_MAX;
        for (int s = 0; s < S; s++) {
            const int g = st.ng[s];
            for (int j = 0; j < g; j++) {
                int32_t w = st.gk[s * G + j];
                if (w & kPending) {
                    const KoKern &K = d.k[w & 0xff];
                    int64_t e = t + block_duration(d, K.c, K.m, st.sum_c[s], st.sum_m[s]);
                    st.gend[s * G + j] = e;
                    st.gk[s * G + j] = w & ~kPending;
                    if (e > makespan) makespan = e;
                }
                if (st.gend[s * G + j] < tmin) tmin = st.gend[s * G + j];
            }
        }
        if (tmin == INT64_MAX) return pos < n ? -1 : makespan;
        if (++events > total_blocks + 2) return -1;  // every event releases >= 1 block
        t = tmin;
    }
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long x = __shfl_xor_sync(0xffffffffu, v, o);
        v = x < v ? x : v;
    }
    return v;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long x = __shfl_xor_sync(0xffffffffu, v, o);
        v = x > v ? x : v;
    }
    return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kThreads)
simple_kernel(const KoSet *__restrict__ d_set, const int8_t *__restrict__ perms,
              const uint64_t *__restrict__ idx, const unsigned long long *__restrict__ items,
              unsigned long long span, unsigned long long first, long long count,
              int64_t *__restrict__ out, KoAccum *acc, void *scratch, size_t per_thread)
{
    __shared__ KoSet sd;
    for (int i = threadIdx.x; i < (int)(sizeof(KoSet) / 4); i += blockDim.x)
        ((int32_t *)&sd)[i] = ((const int32_t *)d_set)[i];
    __syncthreads();
    const long long slot = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    Slab st = slab_at(scratch, per_thread, sd.S, sd.Bk, slot);
    const int n = sd.n;
    const int64_t ref = sd.ref_makespan;
    unsigned long long lmin = ~0ull, lmax = 0, nb = 0, ne = 0, nw = 0, nf = 0;
    // every lane runs the same number of iterations so the warp reductions below are uniform
    const long long iters = (count + stride - 1) / stride;
    for (long long it = 0; it < iters; it++) {
        const long long j = it * stride + slot;
        if (j >= count) continue;
        int8_t perm[KO_MAX_KERNELS];
        bool ok = true;
        long long outpos = j;
        if (items) {
            // work-item list: item covers span consecutive indices, or one idx entry
            const unsigned long long it = items[j / (long long)span];
            if (idx) {
                outpos = (long long)it;
                ok = idx[it] < c_fact[n];
                unrank(n, ok ? idx[it] : 0, perm);
            } else {
                const unsigned long long lehmer = it * span + (unsigned long long)(j % (long long)span);
                outpos = (long long)lehmer;
                unrank(n, lehmer, perm);
            }
        } else if (perms) {
            uint32_t seen = 0;
            for (int q = 0; q < n; q++) {
                int v = perms[j * n + q];
                if (v < 0 || v >= n || (seen >> v) & 1u) ok = false;
                else seen |= 1u << v;
                perm[q] = (int8_t)(v < 0 || v >= n ? 0 : v);
            }
        } else {
            const unsigned long long k = idx ? idx[j] : first + (unsigned long long)j;
            ok = k < c_fact[n];
            unrank(n, ok ? k : 0, perm);
        }
        int64_t ms = ok ? simulate(sd, perm, st) : -1;
        if (out) out[outpos] = ms;
        if (ms < 0) { nf++; continue; }
        unsigned long long u = (unsigned long long)ms;
        lmin = u < lmin ? u : lmin;
        lmax = u > lmax ? u : lmax;
        nb += ms < ref; ne += ms == ref; nw += ms > ref;
    }
    if (acc) {
        lmin = warp_min_u64(lmin); lmax = warp_max_u64(lmax);
        nb = warp_sum_u64(nb); ne = warp_sum_u64(ne); nw = warp_sum_u64(nw); nf = warp_sum_u64(nf);
        if ((threadIdx.x & 31) == 0) {
            if (lmin != ~0ull) atomicMin(&acc->min, lmin);
            if (lmax) atomicMax(&acc->max, lmax);
            if (nb) atomicAdd(&acc->n_better, nb);
            if (ne) atomicAdd(&acc->n_equal, ne);
            if (nw) atomicAdd(&acc->n_worse, nw);
            if (nf) atomicAdd(&acc->failed, nf);
        }
    }
}

__device__ __forceinline__ int find_chunk_simple(const KoChunk *chunks, int nchunks, long long item)
{
    int lo = 0, hi = nchunks - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (chunks[mid].first <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Re-runs the work items the run-length simulator abandoned: one warp per
// item, lanes split the item's orders; same outputs and accumulators.
__global__ void __launch_bounds__(kThreads)
fallback_kernel(KoWork w, void *scratch, size_t per_thread)
{
    const int lane = threadIdx.x & 31;
    const long long slot = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long total = *w.ov_count < w.ov_cap ? *w.ov_count : w.ov_cap;
    for (;;) {
        unsigned long long e = 0;
        if (lane == 0) e = atomicAdd(w.fb_counter, 1ull);
        e = __shfl_sync(0xffffffffu, e, 0);
        if (e >= total) break;
        const long long item = (long long)w.ov_list[e];
        const KoChunk ch = w.chunks[find_chunk_simple(w.chunks, w.nchunks, item)];
        const KoSet &d = w.sets[ch.set];
        const Slab st = slab_at(scratch, per_thread, d.S, d.Bk, slot);
        const int n = d.n;
        const long long local = item - ch.first;
        const long long ref = w.refs ? w.refs[ch.set] : d.ref_makespan;
        const unsigned long long span = ch.mode == 0 ? c_fact[n - ch.d0] : 1ull;
        unsigned long long lmin = ~0ull, lmax = 0, nb = 0, ne = 0, nw = 0;
        for (unsigned long long o = lane; o < span; o += 32) {
            int8_t perm[KO_MAX_KERNELS];
            bool ok = true;
            long long outpos;
            if (ch.mode == 0) {
                const unsigned long long k = (unsigned long long)(ch.list_off + local) * span + o;
                outpos = ch.out_off + (long long)k;
                unrank(n, k, perm);
            } else if (ch.mode == 1) {
                const unsigned long long k = w.idx[ch.list_off + local];
                outpos = ch.out_off + local;
                ok = k < c_fact[n];
                unrank(n, ok ? k : 0, perm);
            } else {
                outpos = ch.out_off + local;
                uint32_t seen = 0;
                const int8_t *row = w.perms + ch.list_off + local * (w.perm_stride ? w.perm_stride : n);
                for (int q = 0; q < n; q++) {
                    const int v = row[q];
                    if (v < 0 || v >= n || ((seen >> v) & 1u)) ok = false;
                    else seen |= 1u << v;
                    perm[q] = (int8_t)(v < 0 || v >= n ? 0 : v);
                }
            }
            const int64_t ms = ok ? simulate(d, perm, st) : -1;
            if (w.out) w.out[outpos] = ms;
            if (ms < 0) continue;
            const unsigned long long u = (unsigned long long)ms;
            lmin = u < lmin ? u : lmin;
            lmax = u > lmax ? u : lmax;
            nb += ms < ref; ne += ms == ref; nw += ms > ref;
        }
        if (w.accs) {
            lmin = warp_min_u64(lmin); lmax = warp_max_u64(lmax);
            nb = warp_sum_u64(nb); ne = warp_sum_u64(ne); nw = warp_sum_u64(nw);
            if (lane == 0) {
                KoAccum *acc = w.accs + ch.set;
                if (lmin != ~0ull) atomicMin(&acc->min, lmin);
                if (lmax) atomicMax(&acc->max, lmax);
                if (nb) atomicAdd(&acc->n_better, nb);
                if (ne) atomicAdd(&acc->n_equal, ne);
                if (nw) atomicAdd(&acc->n_worse, nw);
            }
        }
    }
}

// Variant of simple_kernel for the allocation-free entry point: the set comes
// by value as a kernel parameter and the per-thread slabs live in the
// file-scope array below (its device address is passed in).
__global__ void __launch_bounds__(kThreads)
simple_static_kernel(const KoSet set, const int8_t *__restrict__ perms, long long count,
                     int64_t *__restrict__ out, void *scratch, size_t per_thread)
{
    __shared__ KoSet sd;
    if (threadIdx.x == 0) sd = set;
    __syncthreads();
    const long long slot = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const Slab st = slab_at(scratch, per_thread, sd.S, sd.Bk, slot);
    const int n = sd.n;
    for (long long j = slot; j < count; j += (long long)gridDim.x * blockDim.x) {
        int8_t perm[KO_MAX_KERNELS];
        bool ok = true;
        uint32_t seen = 0;
        for (int q = 0; q < n; q++) {
            const int v = perms[j * n + q];
            if (v < 0 || v >= n || ((seen >> v) & 1u)) ok = false;
            else seen |= 1u << v;
            perm[q] = (int8_t)(v < 0 || v >= n ? 0 : v);
        }
        out[j] = ok ? simulate(sd, perm, st) : -1;
    }
}

constexpr int kHistThreads = 256;

__global__ void __launch_bounds__(kHistThreads)
hist_kernel(const int64_t *__restrict__ ms, long long count, const KoAccum *acc,
            unsigned long long *hist, int nbins)
{
    extern __shared__ uint32_t sh[];
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const long long lo = (long long)acc->min;
    const long long width = (long long)acc->max - lo + 1;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < count;
         j += (long long)gridDim.x * blockDim.x) {
        long long m = ms[j];
        if (m < lo) continue;
        unsigned long long off = (unsigned long long)(m - lo), bin;
        if (width < (1ll << 47))  // (M - min) * nbins stays below 2^62
            bin = off * (unsigned)nbins / (unsigned long long)width;
        else
            bin = (unsigned long long)(((unsigned __int128)off * (unsigned)nbins) / (unsigned long long)width);
        atomicAdd(&sh[bin], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nbins; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], (unsigned long long)sh[i]);
}

__global__ void accum_reset_kernel(KoAccum *acc, int count)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        acc[i].min = ~0ull; acc[i].max = 0;
        acc[i].n_better = 0; acc[i].n_equal = 0; acc[i].n_worse = 0; acc[i].failed = 0;
    }
}

}  // namespace

// ------------------------------------------------- allocation-free evaluation
// Scratch of ko_eval_orders_noalloc: per-thread simulator slabs, shared by
// every call in the process and held on every device that loads the library.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[KO_MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the name is only a host-side stand-in for the device symbol).
ko_status noalloc_scratch(void **ptr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= KO_MAX_DEVICES) {
        cudaGetLastError();
        return KO_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return KO_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *ptr = g_noalloc_ptr[dev];
    return KO_OK;
}

}  // namespace

ko_status ko_noalloc_eval(const KoSet &h, const int8_t *d_orders, long long count, int64_t *d_out,
                          cudaStream_t st)
{
    const size_t per = slab_bytes(h.S, h.Bk);
    const long long slots = (long long)(kNoAllocScratchBytes / per);
    if (slots < kThreads) return KO_ERR_TOO_LARGE;  // the set's simulator state exceeds the array
    if (count <= 0) return KO_OK;
    void *scratch = nullptr;
    ko_status s = noalloc_scratch(&scratch);
    if (s) return s;
    long long blocks = slots / kThreads;
    const long long need = (count + kThreads - 1) / kThreads;
    if (blocks > need) blocks = need;
    simple_static_kernel<<<(unsigned)blocks, kThreads, 0, st>>>(h, d_orders, count, d_out, scratch, per);
    ko_count_launch();
    if (cudaGetLastError() != cudaSuccess) return KO_ERR_CUDA;
    return KO_OK;
}

size_t ko_noalloc_scratch_bytes() { return kNoAllocScratchBytes; }

size_t ko_simple_scratch_per_thread(const KoSet &h) { return slab_bytes(h.S, h.Bk); }

size_t ko_slab_bytes(int S, int Bk) { return slab_bytes(S, Bk); }

cudaError_t ko_launch_fallback(const KoWork &w, void *scratch, size_t scratch_bytes,
                               size_t per_thread, cudaStream_t st)
{
    long long threads = (long long)(scratch_bytes / per_thread);
    long long blocks = threads / kThreads;
    if (blocks > 152 * 4) blocks = 152 * 4;
    if (blocks < 1) return cudaErrorMemoryAllocation;
    fallback_kernel<<<(unsigned)blocks, kThreads, 0, st>>>(w, scratch, per_thread);
    ko_count_launch();
    return cudaGetLastError();
}

cudaError_t ko_launch_simple(const KoSet *d_set, const KoSet &h_set, const int8_t *perms,
                             const uint64_t *idx, uint64_t first, int64_t count, int64_t *out,
                             KoAccum *acc, void *scratch, size_t scratch_bytes, cudaStream_t stream)
{
    if (count <= 0) return cudaSuccess;
    const size_t per = slab_bytes(h_set.S, h_set.Bk);
    long long slots = (long long)(scratch_bytes / per);
    long long blocks = slots / kThreads;
    long long need = (count + kThreads - 1) / kThreads;
    if (blocks > need) blocks = need;
    if (blocks < 1) return cudaErrorMemoryAllocation;
    if (blocks > 65535) blocks = 65535;
    simple_kernel<<<(unsigned)blocks, kThreads, 0, stream>>>(d_set, perms, idx, nullptr, 1, first,
                                                             count, out, acc, scratch, per);
    ko_count_launch();
    return cudaGetLastError();
}


cudaError_t ko_launch_histogram(const int64_t *ms, int64_t count, const KoAccum *acc,
                                unsigned long long *hist, int32_t nbins, cudaStream_t stream)
{
    if (count <= 0) return cudaSuccess;
    long long blocks = (count + kHistThreads * 16 - 1) / (kHistThreads * 16);
    if (blocks > 152 * 8) blocks = 152 * 8;
    size_t smem = sizeof(uint32_t) * (size_t)nbins;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    hist_kernel<<<(unsigned)blocks, kHistThreads, smem, stream>>>(ms, count, acc, hist, nbins);
    ko_count_launch();
    return cudaGetLastError();
}

cudaError_t ko_launch_accum_reset(KoAccum *acc, int count, cudaStream_t stream)
{
    accum_reset_kernel<<<(count + 127) / 128, 128, 0, stream>>>(acc, count);
    ko_count_launch();
    return cudaGetLastError();
}
