// One simulation per thread (ko_lane_sim.cuh), persistent kernel over the same
// work lists as the run-length simulator (ko_fast.cu): exhaustive prefix items
// walked as a lexicographic DFS, Lehmer-index lists and explicit rows.
//
// Each thread runs its own work item as a small state machine -- fetch an
// item, choose the next kernel, step its events, record a leaf and back up to
// the next sibling -- so the threads of a warp advance independently.  A warp
// runs the steps in phases: while fewer than kGather of its threads need the
// control step (choose, save, restore, leaf, next item), the others step their
// events and those threads wait; then the waiting threads take their control
// steps together.  Every control step then runs for several threads at once
// instead of stalling the whole warp for one thread at a time.
//
// Node states (the simulation after a DFS prefix, burst still open) are saved
// to a per-thread slab in global memory (L2-resident), kSaveWords per level,
// 16-byte stores.  A work item that needs more runs or group slots than one
// simulation holds is recorded for the run-length simulator, which re-runs it.
#include "ko_fast.h"
#include "ko_lane_sim.cuh"

namespace {

using namespace kolane;

constexpr unsigned kAll = 0xffffffffu;
// One block per SM: as many simulations (columns of SH::kWords words) as fit
// its shared memory, in whole warps.
template <class SH>
constexpr int lane_threads()
{
    return (232448 / (SH::kWords * 4)) / 32 * 32;
}
static_assert(lane_threads<ShapeL>() == 288 && lane_threads<ShapeM>() == 352 && lane_threads<ShapeS>() == 448,
              "simulations per SM of the three shapes");
// Threads of a warp that must wait for the control step before it runs.
#ifndef KO_LANE_GATHER
#define KO_LANE_GATHER 20
#endif
constexpr int kGather = KO_LANE_GATHER;

__constant__ unsigned long long c_lane_fact[21] = {
    1ull, 1ull, 2ull, 6ull, 24ull, 120ull, 720ull, 5040ull, 40320ull, 362880ull, 3628800ull,
    39916800ull, 479001600ull, 6227020800ull, 87178291200ull, 1307674368000ull,
    20922789888000ull, 355687428096000ull, 6402373705728000ull, 121645100408832000ull,
    2432902008176640000ull};

// Kernel constants of one set in global memory (read-only, L1-resident).
struct GKern {
    const KoSet *set;
    __device__ __forceinline__ KParam full(int i) const
    {
        const int2 a = __ldg(reinterpret_cast<const int2 *>(&set->k[i].r));
        const int2 b = __ldg(reinterpret_cast<const int2 *>(&set->k[i].w));
        const int2 c = __ldg(reinterpret_cast<const int2 *>(&set->k[i].c));
        return KParam{a.x, a.y, b.x, b.y, c.x, c.y};
    }
    __device__ __forceinline__ KRel rel(int i) const
    {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(&set->lk[i]));
        return KRel{v.x, v.y, v.z, v.w};
    }
};

__device__ __forceinline__ int lane_find_chunk(const KoChunk *chunks, int nchunks, long long item)
{
    int lo = 0, hi = nchunks - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (chunks[mid].first <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The dgt-th (0-based) kernel not in `used`.
__device__ __forceinline__ int nth_unused(uint32_t used, uint32_t all, unsigned dgt)
{
    uint32_t u = ~used & all;
    for (unsigned q = 0; q < dgt; q++) u &= u - 1u;
    return __ffs((int)u) - 1;
}

enum Phase : int { PH_FETCH = 0, PH_NEXT, PH_START, PH_EVENT, PH_FINAL, PH_PLACED, PH_DONE };

template <int T, class SH>
__global__ void __launch_bounds__(T, 1) lane_kernel(KoWork a)
{
    constexpr int kRuns = SH::kRuns, kWords = SH::kWords, kSaveWords = SH::kSaveWords;
    extern __shared__ uint32_t lane_cols[];
    LaneSim<T, GKern, SH> sim;
    sim.col = lane_cols + threadIdx.x;
    sim.run_limit = a.run_limit < kRuns ? a.run_limit : kRuns;

    const long long gtid = (long long)blockIdx.x * T + threadIdx.x;
    const int levels = a.levels < 1 ? 1 : a.levels;
    uint32_t *slab = reinterpret_cast<uint32_t *>(a.gstack) + gtid * levels * kSaveWords;
    // a thread without slab room takes no work (the host sizes the grid so this never happens)
    int phase = (gtid + 1) * levels * kSaveWords <= a.gstack_words ? PH_FETCH : PH_DONE;

    // current work item
    const KoSet *set = nullptr;
    int n = 0, d0 = 0, mode = 0, depth = 0, left = 0, set_id = -1, total_blocks = 0, events = 0;
    uint32_t used = 0, all = 0;
    unsigned long long perm = 0;   // kernel at each DFS depth >= d0, 4 bits each
    unsigned long long lk = 0;     // Lehmer digits still to take (prefix kernels)
    unsigned long long rec = 0;    // index the item is recorded under if abandoned
    const int8_t *row = nullptr;
    long long outpos = 0, ref = 0;
    unsigned long long mn = ~0ull, mx = 0;
    unsigned nb = 0, ne = 0, nw = 0;

    for (;;) {
        // Control steps run only when kGather threads wait for them or no thread has events.
        const unsigned busy = __ballot_sync(kAll, phase == PH_EVENT);
        const unsigned want = __ballot_sync(kAll, phase != PH_EVENT && phase != PH_DONE);
        const bool control = __popc(want) >= kGather || busy == 0u;
        if (!control) {
            if (phase == PH_EVENT) {
                const bool last = sim.event(left, busy);
                if (!sim.fail && ++events > total_blocks + 64) sim.fail = 1;  // each event frees >= 1 block
                if (sim.fail) {
                    const unsigned long long slot = atomicAdd(a.ov_count, 1ull);
                    if (slot < a.ov_cap) a.ov_list[slot] = rec;
                    phase = PH_FETCH;
                } else if (last) {
                    phase = PH_FINAL;
                } else if (left == 0) {
                    phase = PH_PLACED;
                }
            }
        } else {
            // The control sub-steps run one after another, each ending at a
            // reconvergence point: threads that took different sub-steps do
            // not stay split for the rest of the iteration.
            int cand = -1;
            if (phase == PH_FINAL) {  // the head kernel's last burst, deferred from its event
                sim.place_partial(left);
                if (sim.fail) {
                    const unsigned long long slot = atomicAdd(a.ov_count, 1ull);
                    if (slot < a.ov_cap) a.ov_list[slot] = rec;
                    phase = PH_FETCH;
                } else {
                    phase = PH_PLACED;
                }
            }
            __syncwarp();
            if (phase == PH_PLACED) {
                depth++;
                if (depth == n) {
                    const long long ms = sim.finish();
                    if (a.out) __stcs(reinterpret_cast<long long *>(&a.out[outpos]), ms);
                    outpos++;
                    const unsigned long long u = (unsigned long long)ms;
                    mn = u < mn ? u : mn;
                    mx = u > mx ? u : mx;
                    nb += ms < ref; ne += ms == ref; nw += ms > ref;
                    // back up to the deepest node with an untried child
                    while (depth > d0) {
                        depth--;
                        const int old = (int)((perm >> (4 * depth)) & 15u);
                        used &= ~(1u << old);
                        const uint32_t avail = ~used & all & ~((2u << old) - 1u);
                        if (avail) {
                            cand = __ffs((int)avail) - 1;
                            // cached in L2 only: the slab stays out of L1, where the set's constants live
                            const uint4 *src = reinterpret_cast<const uint4 *>(slab + (depth - d0) * kSaveWords);
#pragma unroll 13
                            for (int f = 0; f < kWords / 4; f++) {
                                const uint4 v = __ldcg(src + f);
                                sim.W(4 * f) = v.x; sim.W(4 * f + 1) = v.y; sim.W(4 * f + 2) = v.z; sim.W(4 * f + 3) = v.w;
                            }
                            uint32_t r[kRegWords];
#pragma unroll
                            for (int f = 0; f < kRegWords / 4; f++) {
                                const uint4 v = __ldcg(src + kWords / 4 + f);
                                r[4 * f] = v.x; r[4 * f + 1] = v.y; r[4 * f + 2] = v.z; r[4 * f + 3] = v.w;
                            }
                            sim.regs_in(r);
                            break;
                        }
                    }
                    if (cand < 0) {
                        // item complete: fold its statistics into the set's accumulators
                        if (a.accs) {
                            KoAccum *acc = a.accs + set_id;
                            atomicMin(&acc->min, mn);
                            atomicMax(&acc->max, mx);
                            if (nb) atomicAdd(&acc->n_better, (unsigned long long)nb);
                            if (ne) atomicAdd(&acc->n_equal, (unsigned long long)ne);
                            if (nw) atomicAdd(&acc->n_worse, (unsigned long long)nw);
                        }
                        phase = PH_FETCH;
                    } else {
                        perm = (perm & ~(15ull << (4 * depth))) | ((unsigned long long)cand << (4 * depth));
                        used |= 1u << cand;
                        phase = PH_START;
                    }
                } else {
                    if (depth >= d0 && n - depth >= 2) {
                        uint4 *dst = reinterpret_cast<uint4 *>(slab + (depth - d0) * kSaveWords);
#pragma unroll 13
                        for (int f = 0; f < kWords / 4; f++)
                            __stcg(dst + f, make_uint4(sim.W(4 * f), sim.W(4 * f + 1), sim.W(4 * f + 2), sim.W(4 * f + 3)));
                        uint32_t r[kRegWords];
                        sim.regs_out(r);
#pragma unroll
                        for (int f = 0; f < kRegWords / 4; f++)
                            __stcg(dst + kWords / 4 + f, make_uint4(r[4 * f], r[4 * f + 1], r[4 * f + 2], r[4 * f + 3]));
                    }
                    phase = PH_NEXT;
                }
            }
            __syncwarp();
            if (phase == PH_FETCH) {
                for (;;) {  // until an item starts or the list is exhausted
                    const unsigned long long base = atomicAdd(a.counter, 1ull);
                    unsigned long long lim = (unsigned long long)a.n_items;
                    if (a.item_list) lim = *a.item_count < a.ov_cap ? *a.item_count : a.ov_cap;
                    if (base >= lim) { phase = PH_DONE; break; }
                    unsigned long long item = a.item_list ? a.item_list[base] : base;
                    if (item >= (unsigned long long)a.n_items) continue;
                    rec = item;
                    const KoChunk ch = a.chunks[lane_find_chunk(a.chunks, a.nchunks, (long long)item)];
                    set_id = ch.set;
                    set = a.sets + ch.set;
                    n = set->n;
                    all = (1u << n) - 1u;
                    sim.kl.set = set;
                    sim.L = Limits{n, set->S, set->R, set->Sh, set->W, set->Bk, (uint32_t)set->ccap,
                                   (uint32_t)set->mcap, set->cshift, set->mshift};
                    total_blocks = 0;
                    for (int i = 0; i < n; i++) total_blocks += __ldg(&set->k[i].b);
                    ref = a.refs ? a.refs[ch.set] : set->ref_makespan;
                    const long long local = (long long)item - ch.first;
                    mode = ch.mode;
                    bool valid = true;
                    if (mode == 1) {
                        d0 = n;
                        outpos = ch.out_off + local;
                        lk = a.idx[ch.list_off + local];
                        valid = lk < c_lane_fact[n];
                    } else if (mode == 2) {
                        d0 = n;
                        outpos = ch.out_off + local;
                        row = a.perms + ch.list_off + local * (a.perm_stride ? a.perm_stride : n);
                        uint32_t seen = 0;
                        for (int j = 0; j < n; j++) {
                            const int v = row[j];
                            if (v < 0 || v >= n || ((seen >> v) & 1u)) { valid = false; break; }
                            seen |= 1u << v;
                        }
                    } else {
                        d0 = ch.d0;
                        const unsigned long long first =
                            (unsigned long long)(ch.list_off + local) * c_lane_fact[n - d0];
                        outpos = ch.out_off + (long long)first;
                        lk = first;
                    }
                    if (!valid) {
                        if (a.out) a.out[outpos] = -1;
                        continue;
                    }
                    if (set->R >= (1 << 19) || set->W > 127) {  // outside the packed usage word
                        const unsigned long long slot = atomicAdd(a.ov_count, 1ull);
                        if (slot < a.ov_cap) a.ov_list[slot] = rec;
                        continue;
                    }
                    mn = ~0ull; mx = 0; nb = ne = nw = 0;
                    used = 0;
                    depth = 0;
                    perm = 0;
                    sim.init();
                    phase = PH_NEXT;
                    break;
                }
            }
            __syncwarp();
            if (phase == PH_NEXT) {
                if (depth < d0) {
                    if (mode == 2) {
                        cand = row[depth];
                    } else {
                        const unsigned long long f = c_lane_fact[n - 1 - depth];
                        const unsigned dgt = (unsigned)(lk / f);
                        lk -= (unsigned long long)dgt * f;
                        cand = nth_unused(used, all, dgt);
                    }
                } else {
                    cand = __ffs((int)(~used & all)) - 1;
                    perm = (perm & ~(15ull << (4 * depth))) | ((unsigned long long)cand << (4 * depth));
                }
                used |= 1u << cand;
                phase = PH_START;
            }
            __syncwarp();
            if (phase == PH_START) {  // one call site for every kernel start
                left = sim.start_kernel(cand);
                // blocks still queued: the start burst has ended, so its durations are fixed
                // here, together, rather than by the first event of each thread
                if (left > 0) sim.close_burst();
                events = 0;
                if (sim.fail) {
                    const unsigned long long slot = atomicAdd(a.ov_count, 1ull);
                    if (slot < a.ov_cap) a.ov_list[slot] = rec;
                    phase = PH_FETCH;
                } else {
                    phase = left > 0 ? PH_EVENT : PH_PLACED;
                }
            }
        }
        if (!__any_sync(kAll, phase != PH_DONE)) break;
    }
}

}  // namespace

namespace {

template <class SH>
size_t slab_bytes(int levels)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (levels < 1) levels = 1;
    return sizeof(uint32_t) * (size_t)sms * lane_threads<SH>() * levels * SH::kSaveWords;
}

// Threads per block when a launch's work items cannot fill every SM with
// full blocks: small blocks spread the items over all SMs, so each warp shares
// its SM's issue slots with fewer warps (the simulation is latency-bound per
// warp).
constexpr int kSmallT = 64;

template <int T, class SH>
cudaError_t launch_lane_blocks(const KoWork &a, long long blocks, cudaStream_t st)
{
    const size_t smem = sizeof(uint32_t) * (size_t)SH::kWords * T;
    cudaError_t e = cudaFuncSetAttribute(lane_kernel<T, SH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    lane_kernel<T, SH><<<(unsigned)blocks, T, smem, st>>>(a);
    ko_count_launch();
    return cudaGetLastError();
}

template <class SH>
cudaError_t launch_lane(const KoWork &a, cudaStream_t st)
{
    constexpr int T = lane_threads<SH>();
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int levels = a.levels < 1 ? 1 : a.levels;
    const long long work = a.item_list ? (long long)a.ov_cap : a.n_items;
    const long long needed = (work + T - 1) / T;
    if (needed < sms && work > 0) {
        // fewer items than SMs x T: blocks of kSmallT threads, one item per thread at most
        long long blocks = (work + kSmallT - 1) / kSmallT;
        const long long fit = a.gstack_words / ((long long)kSmallT * levels * SH::kSaveWords);
        if (blocks > fit) blocks = fit;  // the slab holds sms x T threads' node states, so fit >= needed
        if (blocks < 1) return cudaErrorInvalidValue;
        return launch_lane_blocks<kSmallT, SH>(a, blocks, st);
    }
    long long blocks = sms;
    const long long fit = a.gstack_words / ((long long)T * levels * SH::kSaveWords);
    if (blocks > fit) blocks = fit;
    if (blocks < 1) return cudaErrorInvalidValue;  // the slab holds no thread's node states
    if (blocks > needed) blocks = needed;
    if (blocks < 1) blocks = 1;  // an empty list (a sizing launch): one block finds no work
    return launch_lane_blocks<T, SH>(a, blocks, st);
}

}  // namespace

size_t ko_lane_slab_bytes(int levels, int shape)
{
    return shape == 2 ? slab_bytes<ShapeS>(levels) : shape == 1 ? slab_bytes<ShapeM>(levels)
                                                                : slab_bytes<ShapeL>(levels);
}

cudaError_t ko_launch_lane(const KoWork &a, int shape, cudaStream_t st)
{
    return shape == 2 ? launch_lane<ShapeS>(a, st) : shape == 1 ? launch_lane<ShapeM>(a, st)
                                                                : launch_lane<ShapeL>(a, st);
}
