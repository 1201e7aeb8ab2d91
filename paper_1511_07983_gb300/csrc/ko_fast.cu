// Run-length, prefix-sharing simulator of the block-dispatch model.
//
// Same model as the simple simulator (Sec. 2 dispatch rule; durations fixed at
// burst end from the SM's SumC / SumM), organised for throughput:
//
// * Runs.  SMs with identical state (usage, SumC, SumM and resident groups
//   with identical end times) form a run of consecutive SM indices.  One lane
//   of a LANES-wide segment (16 or 32 lanes of a warp) holds one run in
//   registers.  Runs are split only where SMs of a run receive different
//   numbers of blocks; the number of runs stays small because the round-robin
//   dispatch treats consecutive SMs alike.
// * Two simulations per warp.  The two 16-lane segments of a warp take two
//   work items whose prefixes differ only in the order of their last two
//   kernels and step through their events together, with whole-warp
//   collectives and per-segment predicates, so they share instructions where
//   their paths agree.
// * Bulk round-robin.  Placing the head kernel is a water-fill: each SM of
//   run j takes at most cap_j more blocks (min over the four limits), sweeps go
//   cyclically from the round-robin pointer p and give one block to every SM
//   with capacity left, so after the placement every SM holds min(cap, L-1)
//   blocks plus one for the first `rem` SMs (cyclic from p) with cap >= L.
//   This reproduces block-by-block first-fit exactly.
// * Groups.  Blocks of one kernel started in one burst on one SM end together
//   and are kept as one group (kernel, count per SM, end).
// * Time.  Ends are kept as 32-bit values modulo 2^32 next to a 64-bit clock;
//   every live end lies within (t, t + max duration] and the host only uses
//   this path when every duration is below 2^31, so comparisons are exact.
// * Prefix sharing.  The lexicographic order of Lehmer indices is a DFS over
//   kernel choices; the state after placing a prefix is saved (in a per-segment
//   global slab that stays in L2, or in shared memory) and restored for each
//   sibling, so each order only pays for the kernels in
//   which it differs from its predecessor (about e kernels per order).
//   The state at a DFS node is "prefix placed, current burst still open":
//   the next kernel continues the same burst.
// * Overflow.  A segment that would need more runs than lanes, or more than
//   kG groups in one run, abandons its work item and records it; a second
//   pass with 32 lanes and 16 group slots re-runs the recorded items, and the
//   simple simulator takes whatever that pass abandons, all on the stream.
#include "ko_fast.h"

namespace {

constexpr int kG = 8;                       // group slots per run (first pass)
constexpr int kGWide = 16;                  // group slots per run (pass over abandoned items)
constexpr uint32_t kPend = 1u << 15;        // group started in the open burst
constexpr uint32_t kValid = 1u << 16;       // slot holds a group
// group word: kernel id (bits 0-4) | blocks per SM (bits 8-13) | kPend | kValid

constexpr int kMaxLevels = 6;               // saved DFS levels per segment
// Per-lane words saved per DFS level: range (beg | cnt << 16), registers,
// shared memory, warps | blocks << 25, SumC, SumM, G/2 words of two 13-bit
// group descriptors, G end times.
__host__ __device__ constexpr int state_words(int G) { return 6 + G / 2 + G; }
constexpr int kThreads = 128;

__constant__ unsigned long long c_fact[21] = {
    1ull, 1ull, 2ull, 6ull, 24ull, 120ull, 720ull, 5040ull, 40320ull, 362880ull, 3628800ull,
    39916800ull, 479001600ull, 6227020800ull, 87178291200ull, 1307674368000ull,
    20922789888000ull, 355687428096000ull, 6402373705728000ull, 121645100408832000ull,
    2432902008176640000ull};

struct SetConst {
    int n, S, R, Sh, W, Bk;
    uint32_t ccap, mcap;  // <= 2^30 (the capacity setter rejects more)
    int cshift, mshift;
    int total_blocks;
    int r[KO_MAX_KERNELS], s[KO_MAX_KERNELS], w[KO_MAX_KERNELS], b[KO_MAX_KERNELS];
    int c[KO_MAX_KERNELS], m[KO_MAX_KERNELS];
    float rr[KO_MAX_KERNELS], rs[KO_MAX_KERNELS], rw[KO_MAX_KERNELS];  // 1/r, 1/s, 1/w
};

// floor(x / d) for 0 <= x <= 2^24 and d >= 1, clamped to at most 32: the
// quotient of min(x, 32 d) estimated with a float reciprocal (error far below
// one unit at that size) and corrected once by an exact integer check.
__device__ __forceinline__ int quot32(int x, int d, float rcp)
{
    const int xc = min(x, d << 5);
    int q = __float2int_rz(__int2float_rn(xc) * rcp);
    if ((q + 1) * d <= xc) q++;
    if (q * d > xc) q--;
    return q;
}

constexpr unsigned kAll = 0xffffffffu;

template <int LANES>
struct Seg {
    unsigned mask;   // lanes of this segment
    int lane;        // lane within segment
    unsigned half;   // segment within the warp (0 for 32-lane segments)
};

// Per-lane run state, held in registers (all array indices are compile-time).
template <int G>
struct Run {
    int beg, cnt, ur, us, uw, ub, sc, sm;
    uint32_t gk[G];
    uint32_t ge[G];
};

// Register-array access by a run-time slot index without local memory: a
// chain of selects (read) or predicated moves (write) over the unrolled slots.
template <int G>
__device__ __forceinline__ uint32_t slot_get(const uint32_t (&a)[G], int g)
{
    uint32_t v = a[0];
#pragma unroll
    for (int i = 1; i < G; i++) v = g == i ? a[i] : v;
    return v;
}
template <int G>
__device__ __forceinline__ void slot_set(uint32_t (&a)[G], int g, uint32_t v)
{
#pragma unroll
    for (int i = 0; i < G; i++)
        if (g == i) a[i] = v;
}

// The simulation of one order by one segment.  The event step (burst,
// close_burst, advance, finish, place_kernel) is executed by every lane of the
// warp together: each function takes `act`, false in a segment with nothing to
// do, which then changes no state, and every collective is a whole-warp
// operation from which a 16-lane segment reads its own half.  So the two
// segments of a warp issue one instruction stream and share every instruction
// where their paths agree, instead of running one after the other.
template <int LANES, int G>
struct Sim {
    static constexpr int kG = G;
    static constexpr int kStateWords = state_words(G);
    Seg<LANES> sg;
    Run<G> run;
    long long t;     // clock (segment-uniform)
    int p;           // round-robin pointer
    int nruns;
    int run_limit;
    int fail;

    // ---- segment collectives, reached by the whole warp
    __device__ __forceinline__ int shfl(int v, int src) const { return __shfl_sync(kAll, v, src, LANES); }
    __device__ __forceinline__ unsigned ballot(bool pred) const
    {
        const unsigned b = __ballot_sync(kAll, pred);
        return LANES == 32 ? b : (b >> (sg.half * 16u)) & 0xffffu;
    }
    __device__ __forceinline__ bool any(bool pred) const { return ballot(pred) != 0u; }
    __device__ __forceinline__ unsigned sum(unsigned v) const
    {
        if (LANES == 32) return __reduce_add_sync(kAll, v);
        const unsigned s0 = __reduce_add_sync(kAll, sg.half ? 0u : v);
        const unsigned s1 = __reduce_add_sync(kAll, sg.half ? v : 0u);
        return sg.half ? s1 : s0;
    }
    __device__ __forceinline__ unsigned umax(unsigned v) const
    {
        if (LANES == 32) return __reduce_max_sync(kAll, v);
        const unsigned s0 = __reduce_max_sync(kAll, sg.half ? 0u : v);
        const unsigned s1 = __reduce_max_sync(kAll, sg.half ? v : 0u);
        return sg.half ? s1 : s0;
    }
    __device__ __forceinline__ unsigned umin(unsigned v) const
    {
        if (LANES == 32) return __reduce_min_sync(kAll, v);
        const unsigned s0 = __reduce_min_sync(kAll, sg.half ? ~0u : v);
        const unsigned s1 = __reduce_min_sync(kAll, sg.half ? v : ~0u);
        return sg.half ? s1 : s0;
    }

    __device__ void init(const SetConst &K) { init_sms(sg.lane == 0 ? K.S : 0); }
    __device__ void init_sms(int sms)  // empty GPU, lane 0's run holding `sms` SMs
    {
        run.beg = 0;
        run.cnt = sms;
        run.ur = run.us = run.uw = run.ub = run.sc = run.sm = 0;
#pragma unroll
        for (int g = 0; g < kG; g++) { run.gk[g] = 0; run.ge[g] = 0; }
        t = 0;
        p = 0;
        nruns = 1;
        fail = 0;
    }

    // Split run j at offset x (0 < x < cnt_j) where `act`: lane j keeps the
    // first x SMs, lane j+1 takes the rest; later lanes move up one.  `extra`
    // registers move with the lanes.
    __device__ void split(int j, int x, int &extra0, int &extra1, bool act)
    {
        bool ok = act;
        if (ok && nruns >= run_limit) { fail = 1; ok = false; }
        const bool up = ok && sg.lane > j;
#define KO_SHIFT(v) { auto _u = __shfl_up_sync(kAll, v, 1, LANES); if (up) v = _u; }
        KO_SHIFT(run.beg) KO_SHIFT(run.cnt) KO_SHIFT(run.ur) KO_SHIFT(run.us) KO_SHIFT(run.uw)
        KO_SHIFT(run.ub) KO_SHIFT(run.sc) KO_SHIFT(run.sm) KO_SHIFT(extra0) KO_SHIFT(extra1)
#pragma unroll
        for (int g = 0; g < kG; g++) { KO_SHIFT(run.gk[g]) KO_SHIFT(run.ge[g]) }
#undef KO_SHIFT
        if (ok && sg.lane == j) run.cnt = x;
        if (ok && sg.lane == j + 1) { run.beg += x; run.cnt -= x; }
        if (ok) nruns++;
    }

    // Add `give` blocks per SM of kernel kid to this lane's run as a new
    // pending group (where `act`).
    __device__ void add_blocks(const SetConst &K, int kid, int give, bool act)
    {
        bool need = act && give > 0 && run.cnt > 0;
        if (need) {
            run.ur += give * K.r[kid];
            run.us += give * K.s[kid];
            run.uw += give * K.w[kid];
            run.ub += give;
            run.sc += give * K.c[kid];
            run.sm += give * K.m[kid];
        }
        bool placed = !need;
#pragma unroll
        for (int g = 0; g < kG; g++) {
            if (!placed && run.gk[g] == 0) {
                run.gk[g] = kValid | kPend | ((uint32_t)give << 8) | (uint32_t)kid;
                placed = true;
            }
        }
        if (any(!placed)) fail = 1;
    }

    // One dispatch burst for the head kernel `kid` with `left` blocks queued.
    __device__ void burst(const SetConst &K, int kid, int &left, bool act)
    {
        const int k = act ? kid : 0;  // kernel 0's constants stand in where the segment is idle
        const int r = K.r[k], s = K.s[k], w = K.w[k];
        int cap = 0;
        if (act && run.cnt > 0) {
            cap = K.Bk - run.ub;
            cap = min(cap, quot32(K.R - run.ur, r, K.rr[k]));
            cap = min(cap, quot32(K.W - run.uw, w, K.rw[k]));
            if (s > 0) cap = min(cap, quot32(K.Sh - run.us, s, K.rs[k]));
            cap = max(cap, 0);
        }
        const int total = (int)sum((unsigned)(run.cnt * cap));
        const int maxcap = (int)umax((unsigned)cap);
        const bool full = act && total > 0 && total <= left;
        bool part = act && total > left;
        int give = 0;
        {
            // every SM takes its full capacity; the last block lands on the SM
            // with cap == maxcap that comes last cyclically from p
            int pos = 0;
            if (full && run.cnt > 0 && cap == maxcap) {
                const int pm1 = p == 0 ? K.S - 1 : p - 1;
                if (pm1 >= run.beg && pm1 < run.beg + run.cnt) pos = K.S;
                else { pos = run.beg + run.cnt - p; if (pos <= 0) pos += K.S; }
            }
            const int maxpos = (int)umax((unsigned)pos);  // last SM's cyclic offset from p, plus one
            if (full) {
                p += maxpos;
                if (p >= K.S) p -= K.S;
                left -= total;
                give = cap;
            }
        }
        if (__any_sync(kAll, part)) {
            // partial placement: smallest sweep count L with F(L) >= left
            int lo = 1, hi = part ? maxcap : 1;
            while (__any_sync(kAll, lo < hi)) {
                const int mid = (lo + hi) >> 1;
                const int f = (int)sum((unsigned)(run.cnt * min(cap, mid)));
                if (lo < hi) {
                    if (f >= left) hi = mid; else lo = mid + 1;
                }
            }
            const int L = lo;
            const int filled = (int)sum((unsigned)(run.cnt * min(cap, L - 1)));
            const int rem = left - filled;  // 1 .. number of SMs with cap >= L
            // Two cuts, one split site: phase 0 cuts the run holding p at p when its
            // SMs are eligible (so the cyclic order from p is a rotation of whole
            // runs); phase 1 cuts the run where the last partial sweep ends.
            int jp = __ffs(ballot(run.cnt > 0 && run.beg <= p && p < run.beg + run.cnt)) - 1;
            int plus = 0, star = 0, x = 0, beg_star = 0;
#pragma unroll 1
            for (int phase = 0; phase < 2; phase++) {
                int cut_lane, cut_at;
                bool need;
                if (phase == 0) {
                    const int beg_jp = shfl(run.beg, jp), cap_jp = shfl(cap, jp);
                    need = part && beg_jp < p && cap_jp >= L;
                    cut_lane = jp;
                    cut_at = p - beg_jp;
                } else {
                    const int e = (run.cnt > 0 && cap >= L) ? run.cnt : 0;
                    int incl = e;
#pragma unroll
                    for (int o = 1; o < LANES; o <<= 1) {
                        const int v = __shfl_up_sync(kAll, incl, o, LANES);
                        if (sg.lane >= o) incl += v;
                    }
                    const int excl = incl - e;
                    const int E = shfl(incl, LANES - 1);
                    const int excl_jp = shfl(excl, jp);
                    const int rot = sg.lane >= jp ? excl - excl_jp : E - excl_jp + excl;
                    star = __ffs(ballot(e > 0 && rot < rem && rem <= rot + e)) - 1;
                    x = rem - shfl(rot, star);
                    const int cnt_star = shfl(run.cnt, star);
                    beg_star = shfl(run.beg, star);
                    // rotated position of each lane relative to jp
                    const int rl = sg.lane >= jp ? sg.lane - jp : sg.lane - jp + nruns;
                    const int rs = star >= jp ? star - jp : star - jp + nruns;
                    plus = (e > 0 && rl < rs) ? 1 : 0;
                    if (sg.lane == star) plus = 1;
                    need = part && x < cnt_star;
                    cut_lane = star;
                    cut_at = x;
                }
                if (__any_sync(kAll, need)) {
                    split(cut_lane, cut_at, cap, plus, need);
                    if (need) {
                        if (fail) part = false;
                        else if (phase == 0) jp++;
                        else if (sg.lane == star + 1) plus = 0;
                    }
                }
            }
            if (part) {
                p = beg_star + x;
                if (p >= K.S) p -= K.S;
                left = 0;
                give = min(cap, L - 1) + plus;
            }
        }
        add_blocks(K, k, give, full || part);
    }

    __device__ __forceinline__ uint32_t duration(const SetConst &K, int kid) const
    {
        // every factor fits 32 bits (c, m <= 2^24; SumC, SumM <= 32 * 2^24; caps <= 2^30), so each
        // product is one 32 x 32 -> 64-bit multiply
        const uint32_t c = (uint32_t)K.c[kid], m = (uint32_t)K.m[kid];
        const uint32_t sc = max((uint32_t)run.sc, K.ccap), sm = max((uint32_t)run.sm, K.mcap);
        const unsigned long long pc = (unsigned long long)c * sc + (K.ccap - 1u);
        const unsigned long long pm = (unsigned long long)m * sm + (K.mcap - 1u);
        const unsigned long long dc = K.cshift >= 0 ? pc >> K.cshift : pc / K.ccap;
        const unsigned long long dm = K.mshift >= 0 ? pm >> K.mshift : pm / K.mcap;
        return (uint32_t)(dc > dm ? dc : dm);
    }

    // Fix the durations of the groups started in the open burst (one body,
    // looped over the set bits of each lane's pending mask).
    __device__ void close_burst(const SetConst &K, bool act)
    {
        const uint32_t t32 = (uint32_t)t;
        uint32_t pend = 0;
        if (act) {
#pragma unroll
            for (int g = 0; g < kG; g++) pend |= ((run.gk[g] & kPend) ? 1u : 0u) << g;
        }
        while (__any_sync(kAll, pend != 0)) {
            if (pend) {
                const int g = __ffs(pend) - 1;
                pend &= pend - 1;
                const uint32_t w = slot_get(run.gk, g);
                slot_set(run.ge, g, t32 + duration(K, w & 31u));
                slot_set(run.gk, g, w & ~kPend);
            }
        }
    }

    // Jump to the earliest end and release every group ending then.
    __device__ void advance(const SetConst &K, bool act)
    {
        const uint32_t t32 = (uint32_t)t;
        uint32_t dmin = 0xffffffffu;
        if (act) {
#pragma unroll
            for (int g = 0; g < kG; g++)
                if (run.gk[g]) dmin = min(dmin, run.ge[g] - t32);
        }
        dmin = umin(dmin);
        bool ok = act;
        if (ok && dmin == 0xffffffffu) { fail = 1; ok = false; }
        uint32_t rel = 0;
        if (ok) {
            t += dmin;
            const uint32_t now = t32 + dmin;
#pragma unroll
            for (int g = 0; g < kG; g++) rel |= (run.gk[g] != 0 && run.ge[g] == now ? 1u : 0u) << g;
        }
        while (__any_sync(kAll, rel != 0)) {
            if (rel) {
                const int g = __ffs(rel) - 1;
                rel &= rel - 1;
                const uint32_t w = slot_get(run.gk, g);
                const int kid = w & 31u;
                const int q = (w >> 8) & 63u;
                run.ur -= q * K.r[kid]; run.us -= q * K.s[kid]; run.uw -= q * K.w[kid];
                run.ub -= q; run.sc -= q * K.c[kid]; run.sm -= q * K.m[kid];
                slot_set(run.gk, g, 0u);
            }
        }
    }

    // Queue all blocks of kernel kid behind the current queue and simulate
    // until the last of them is placed (the burst that places it stays open).
    // The whole warp runs the loop until no segment has events left.
    __device__ void place_kernel(const SetConst &K, int kid, bool act)
    {
        int left = act ? K.b[kid] : 0;
        bool go = act && !fail;
        int it = 0;
        while (__any_sync(kAll, go)) {
            burst(K, kid, left, go);
            const bool more = go && !fail && left > 0;
            close_burst(K, more);
            advance(K, more);
            if (more && ++it > K.total_blocks + 64) fail = 1;  // each event frees >= 1 block
            go = more && !fail;
        }
    }

    // Close the final burst; the makespan is the latest end (where `act`).
    __device__ long long finish(const SetConst &K, bool act)
    {
        close_burst(K, act);
        const uint32_t t32 = (uint32_t)t;
        uint32_t dmax = 0;
        if (act) {
#pragma unroll
            for (int g = 0; g < kG; g++)
                if (run.gk[g]) dmax = max(dmax, run.ge[g] - t32);
        }
        dmax = umax(dmax);
        return t + (long long)dmax;
    }

    // Save / restore the node state; only the first SAVE lanes are stored, so
    // a node with more runs than that abandons the work item.
    // 13-bit form of a group word: kernel (5) | blocks per SM (6) | pending | valid
    __device__ __forceinline__ static uint32_t pack13(uint32_t w)
    {
        return (w & 31u) | (((w >> 8) & 63u) << 5) | (((w >> 15) & 1u) << 11) | (((w >> 16) & 1u) << 12);
    }
    __device__ __forceinline__ static uint32_t unpack13(uint32_t v)
    {
        return (v & 31u) | (((v >> 5) & 63u) << 8) | (((v >> 11) & 1u) << 15) | (((v >> 12) & 1u) << 16);
    }

    template <int SAVE>
    __device__ void save(int *slot)
    {
        if (nruns > SAVE) { fail = 1; return; }
        if (sg.lane < SAVE) {
            int *q = slot + sg.lane;
            q[0 * SAVE] = (int)((uint32_t)run.beg | ((uint32_t)run.cnt << 16));
            q[1 * SAVE] = run.ur;
            q[2 * SAVE] = run.us;
            q[3 * SAVE] = (int)((uint32_t)run.uw | ((uint32_t)run.ub << 25));
            q[4 * SAVE] = run.sc;
            q[5 * SAVE] = run.sm;
#pragma unroll
            for (int g = 0; g < kG; g += 2)
                q[(6 + g / 2) * SAVE] = (int)(pack13(run.gk[g]) | (pack13(run.gk[g + 1]) << 16));
#pragma unroll
            for (int g = 0; g < kG; g++) q[(6 + kG / 2 + g) * SAVE] = (int)run.ge[g];
        }
        if (sg.lane == 0) {
            int *u = slot + kStateWords * SAVE;
            u[0] = (int)(t & 0xffffffffll); u[1] = (int)(t >> 32); u[2] = p; u[3] = nruns;
        }
        __syncwarp(sg.mask);
    }

    template <int SAVE>
    __device__ void restore(const int *slot)
    {
        if (sg.lane < SAVE) {
            const int *q = slot + sg.lane;
            const uint32_t r0 = (uint32_t)q[0 * SAVE], r3 = (uint32_t)q[3 * SAVE];
            run.beg = (int)(r0 & 0xffffu);
            run.cnt = (int)(r0 >> 16);
            run.ur = q[1 * SAVE];
            run.us = q[2 * SAVE];
            run.uw = (int)(r3 & 0x1ffffffu);
            run.ub = (int)(r3 >> 25);
            run.sc = q[4 * SAVE];
            run.sm = q[5 * SAVE];
#pragma unroll
            for (int g = 0; g < kG; g += 2) {
                const uint32_t v = (uint32_t)q[(6 + g / 2) * SAVE];
                run.gk[g] = unpack13(v & 0xffffu);
                run.gk[g + 1] = unpack13(v >> 16);
            }
#pragma unroll
            for (int g = 0; g < kG; g++) run.ge[g] = (uint32_t)q[(6 + kG / 2 + g) * SAVE];
        } else {
            run.beg = 0; run.cnt = 0; run.ur = run.us = run.uw = run.ub = run.sc = run.sm = 0;
#pragma unroll
            for (int g = 0; g < kG; g++) { run.gk[g] = 0; run.ge[g] = 0; }
        }
        const int *u = slot + kStateWords * SAVE;
        t = (long long)(uint32_t)u[0] | ((long long)u[1] << 32);
        p = u[2];
        nruns = u[3];
        fail = 0;
    }
};

// Segment-cooperative load of one set's constants into shared memory.
template <int LANES>
__device__ void load_set(SetConst &K, const KoSet *d, const Seg<LANES> &sg)
{
    int nb = 0;
    for (int i = sg.lane; i < KO_MAX_KERNELS; i += LANES) {
        const KoKern kk = d->k[i];
        K.r[i] = kk.r; K.s[i] = kk.s; K.w[i] = kk.w; K.b[i] = kk.b; K.c[i] = kk.c; K.m[i] = kk.m;
        K.rr[i] = kk.r > 0 ? 1.0f / (float)kk.r : 0.0f;
        K.rs[i] = kk.s > 0 ? 1.0f / (float)kk.s : 0.0f;
        K.rw[i] = kk.w > 0 ? 1.0f / (float)kk.w : 0.0f;
        if (i < d->n) nb += kk.b;
    }
    nb = (int)__reduce_add_sync(sg.mask, (unsigned)nb);
    if (sg.lane == 0) {
        K.n = d->n; K.S = d->S; K.R = d->R; K.Sh = d->Sh; K.W = d->W; K.Bk = d->Bk;
        K.ccap = (uint32_t)d->ccap; K.mcap = (uint32_t)d->mcap; K.cshift = d->cshift; K.mshift = d->mshift;
        K.total_blocks = nb;
    }
    __syncwarp(sg.mask);
}

// first `depth` kernels of the lexicographic permutation with Lehmer index k
__device__ void lehmer_prefix(int n, unsigned long long k, int depth, int8_t *perm, uint32_t &used)
{
    used = 0;
    for (int j = 0; j < depth; j++) {
        const unsigned long long f = c_fact[n - 1 - j];
        const uint32_t dgt = (uint32_t)(k / f);
        k -= (unsigned long long)dgt * f;
        uint32_t u = ~used & ((1u << n) - 1u);
        for (uint32_t q = 0; q < dgt; q++) u &= u - 1u;
        const int v = __ffs(u) - 1;
        perm[j] = (int8_t)v;
        used |= 1u << v;
    }
}

// Order in which a warp's two segments take the prefixes of one exhaustive chunk.  Prefixes
// of length d0 in lexicographic order fall into groups of m (m - 1) (m = N - d0 + 2) that share
// all but their last two kernels; inside a group whose items all lie in [lo, hi), item j and
// j ^ 1 are mapped to two prefixes that end in the same two kernels in swapped order, so the
// two segments then walk the same remaining kernels in the same order.  A bijection on
// [lo, hi); items of a group cut by the range keep their place.
__device__ __forceinline__ unsigned long long pair_swap_order(unsigned long long j, int m, unsigned long long lo,
                                                              unsigned long long hi)
{
    const unsigned long long M = (unsigned long long)m * (m - 1);
    const unsigned long long g0 = j - j % M;
    if (g0 < lo || g0 + M > hi) return j;
    const unsigned v = (unsigned)(j - g0);
    unsigned q = v >> 1;  // unordered pair {x < y} of the group's last two kernels (ranks)
    int x = 0;
    while (q >= (unsigned)(m - 1 - x)) {  // at most m - 1 turns
        q -= (unsigned)(m - 1 - x);
        x++;
    }
    const int y = x + 1 + (int)q;
    const int a0 = (v & 1u) ? y : x, a1 = (v & 1u) ? x : y;
    return g0 + (unsigned long long)a0 * (m - 1) + (unsigned long long)(a1 > a0 ? a1 - 1 : a1);
}

__device__ __forceinline__ int find_chunk(const KoChunk *chunks, int nchunks, long long item)
{
    int lo = 0, hi = nchunks - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (chunks[mid].first <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Per-segment running statistics of the set being worked on.
// Min, max and better / equal / worse counts of a run of makespans.  The
// kernel keeps one per segment for the current work item and one for the
// segment's current set in shared memory (only lane 0 touches them), which
// keeps twenty 32-bit registers out of the simulation loop.
struct SegStats {
    unsigned long long mn, mx, nb, ne, nw;
    __device__ void clear() { mn = ~0ull; mx = 0; nb = ne = nw = 0; }
    __device__ void add(const SegStats &o)
    {
        mn = o.mn < mn ? o.mn : mn;
        mx = o.mx > mx ? o.mx : mx;
        nb += o.nb; ne += o.ne; nw += o.nw;
    }
    __device__ void flush(KoAccum *accs, int set)
    {
        if (set >= 0 && accs) {
            KoAccum *a = accs + set;
            if (mn != ~0ull) atomicMin(&a->min, mn);
            if (mx) atomicMax(&a->max, mx);
            if (nb) atomicAdd(&a->n_better, nb);
            if (ne) atomicAdd(&a->n_equal, ne);
            if (nw) atomicAdd(&a->n_worse, nw);
        }
        clear();
    }
};

// Resident blocks per SM the register budget must allow.  8 blocks (64
// registers, a few spills to L1) measured fastest on the N=12 / 148-SM set:
// the kernel is latency-bound and extra warps hide more than the spills cost.
#ifndef KO_FAST_MIN_BLOCKS
#define KO_FAST_MIN_BLOCKS 8
#endif

template <int LANES, int G, int SAVE>
__global__ void __launch_bounds__(kThreads, KO_FAST_MIN_BLOCKS)
fast_kernel(KoWork a)
{
    constexpr int kStateWords = state_words(G);
    constexpr int kSegs = kThreads / LANES;
    __shared__ SetConst Ks[kSegs];
    extern __shared__ int stack_mem[];

    Sim<LANES, G> sim;
    const int seg = threadIdx.x / LANES;
    sim.sg.lane = threadIdx.x % LANES;
    sim.run_limit = a.run_limit < LANES ? a.run_limit : LANES;
    sim.sg.mask = LANES == 32 ? kAll : (((1u << LANES) - 1u) << ((threadIdx.x & 31) / LANES * LANES));
    const int level_words = kStateWords * SAVE + 4;
    const unsigned half = (threadIdx.x & 31) / LANES;  // segment within the warp
    sim.sg.half = half;
    // node states: per segment, in shared memory or in a global slab
    int *stack = stack_mem + seg * a.levels * level_words;
    if (a.gstack) {
        const long long gseg = (long long)blockIdx.x * kSegs + seg;
        const long long off = gseg * a.levels * level_words;
        // slab too small (never taken): checked for the warp's last segment, so a warp leaves whole
        const long long last = (long long)blockIdx.x * kSegs + seg + (32 / LANES - 1 - (int)half);
        if ((last + 1) * a.levels * level_words > a.gstack_words) return;
        stack = a.gstack + off;
    }
    SetConst &K = Ks[seg];
    int loaded = -1;
    __shared__ SegStats seg_stats[kSegs], item_stats[kSegs];
    SegStats &st = seg_stats[seg], &is = item_stats[seg];  // lane 0 only
    // where the current item's makespans go and what they are ranked against (lane 0 only)
    __shared__ long long item_out[kSegs], item_ref[kSegs];
    int st_set = -1;                                      // set that `st` accumulates (lane 0)
    if (sim.sg.lane == 0) st.clear();
    sim.init_sms(0);  // a segment without an item still takes part in the warp's event steps

    // The warp's segments take consecutive items together and walk them in step: every
    // whole-warp operation below (the fetch's shuffles, the walk's vote, the event vote in
    // place_kernel) is reached by all segments of the warp equally often, and the only exit
    // from this loop is the same for the whole warp.
    constexpr int kPerWarp = 32 / LANES;
    for (;;) {
        unsigned long long base = 0, lim = 0;
        if ((threadIdx.x & 31) == 0) {
            base = atomicAdd(a.counter, (unsigned long long)kPerWarp);
            lim = (unsigned long long)a.n_items;
            if (a.item_list)  // pass over items a previous pass abandoned
                lim = *a.item_count < a.ov_cap ? *a.item_count : a.ov_cap;
        }
        base = __shfl_sync(kAll, base, 0);
        lim = __shfl_sync(kAll, lim, 0);
        if (base >= lim) break;
        unsigned long long item = base + half;
        bool have = item < lim;  // an odd tail leaves the last segment without an item
        if (have && a.item_list) item = a.item_list[item];
        have = have && item < (unsigned long long)a.n_items;
        // the index an abandoned item is recorded under: the later passes take items in plain
        // order, so a reordered prefix is recorded as the item that plain order maps to it
        unsigned long long rec = item;

        // perm[0 .. d0) is the item's fixed prefix (the whole order in list modes)
        int8_t perm[KO_MAX_KERNELS];
        int next[KO_MAX_KERNELS + 1];
        int n = 0, d0 = 0, depth = 0;
        uint32_t all = 0, used = 0;
        bool first_child = true;
        if (have) {
            const KoChunk ch = a.chunks[find_chunk(a.chunks, a.nchunks, (long long)item)];
            if (ch.set != loaded) {
                load_set<LANES>(K, a.sets + ch.set, sim.sg);
                loaded = ch.set;
            }
            if (sim.sg.lane == 0 && st_set != ch.set) {
                st.flush(a.accs, st_set);
                st_set = ch.set;
            }
            n = K.n;
            all = (1u << n) - 1u;
            if (sim.sg.lane == 0) item_ref[seg] = a.refs ? a.refs[ch.set] : a.sets[ch.set].ref_makespan;
            const long long local = (long long)item - ch.first;
            long long outpos;
            bool valid = true;
            if (ch.mode == 1) {
                d0 = n;
                outpos = ch.out_off + local;
                const unsigned long long k = a.idx[ch.list_off + local];
                valid = k < c_fact[n];
                if (valid) lehmer_prefix(n, k, n, perm, used);
            } else if (ch.mode == 2) {
                d0 = n;
                outpos = ch.out_off + local;
                const int8_t *row = a.perms + ch.list_off + local * (a.perm_stride ? a.perm_stride : n);
                for (int j = 0; j < n; j++) {
                    const int v = row[j];
                    if (v < 0 || v >= n || ((used >> v) & 1u)) { valid = false; break; }
                    perm[j] = (int8_t)v;
                    used |= 1u << v;
                }
            } else {
                d0 = ch.d0;
                unsigned long long j = (unsigned long long)(ch.list_off + local);
                // swap partners pair up only in a pass over whole chunks; an item taken from a
                // list of abandoned items is run as the item it names
                if (kPerWarp == 2 && d0 >= 2 && !a.item_list) {
                    j = pair_swap_order(j, n - d0 + 2, (unsigned long long)ch.list_off,
                                        (unsigned long long)(ch.list_off + ch.count));
                    rec = (unsigned long long)ch.first + (j - (unsigned long long)ch.list_off);
                }
                const unsigned long long first = j * c_fact[n - d0];
                outpos = ch.out_off + (long long)first;
                lehmer_prefix(n, first, d0, perm, used);
            }
            if (!valid) {
                if (sim.sg.lane == 0 && a.out) a.out[outpos] = -1;
                have = false;
            } else {
                if (sim.sg.lane == 0) {
                    is.clear();
                    item_out[seg] = outpos;
                }
                used = 0;
                sim.init(K);
                if (d0 == 0) {
                    next[0] = 0;
                    if (n >= 2) sim.template save<SAVE>(stack);
                }
            }
        }

        // One walk per item: depths below d0 take the prefix kernel, depths from
        // d0 on enumerate the unused kernels in increasing id (lexicographic DFS),
        // restoring the saved node state for every child after the first.  Each
        // step places one kernel; a segment whose walk has ended still votes.
        bool going = have && !sim.fail;
        while (__any_sync(kAll, going)) {
            int cand = -1;
            if (going) {
                for (;;) {  // next kernel to place, backing up as needed (depth falls each turn)
                    if (depth < d0) { cand = perm[depth]; break; }
                    const uint32_t avail = ~used & all & ~((1u << next[depth]) - 1u);
                    if (avail) {
                        cand = __ffs(avail) - 1;
                        if (!first_child) sim.template restore<SAVE>(stack + (depth - d0) * level_words);
                        break;
                    }
                    if (depth == d0) break;  // the walk is complete
                    depth--;
                    used &= ~(1u << perm[depth]);
                    next[depth] = perm[depth] + 1;
                    first_child = false;
                }
                if (cand < 0) {
                    going = false;
                } else {
                    perm[depth] = (int8_t)cand;
                    used |= 1u << cand;
                }
            }
            sim.place_kernel(K, cand, going);
            if (going && sim.fail) going = false;
            const bool leaf = going && depth + 1 == n;
            long long ms = 0;
            if (__any_sync(kAll, leaf)) ms = sim.finish(K, leaf);
            if (going) {
                if (leaf) {
                    if (sim.sg.lane == 0) {
                        // evict-first: the makespan stream must not push the node-state slab out of L2
                        const long long pos = item_out[seg]++;
                        if (a.out) __stcs((long long *)&a.out[pos], (long long)ms);
                        const unsigned long long u = (unsigned long long)ms;
                        const long long ref = item_ref[seg];
                        is.mn = u < is.mn ? u : is.mn;
                        is.mx = u > is.mx ? u : is.mx;
                        is.nb += ms < ref; is.ne += ms == ref; is.nw += ms > ref;
                    }
                    if (d0 == n) {
                        going = false;
                    } else {
                        used &= ~(1u << cand);
                        next[depth] = cand + 1;
                        first_child = false;
                    }
                } else {
                    depth++;
                    if (depth >= d0) {
                        next[depth] = 0;
                        first_child = true;
                        if (n - depth >= 2) sim.template save<SAVE>(stack + (depth - d0) * level_words);
                    }
                    if (sim.fail) going = false;
                }
            }
        }
        if (have && sim.sg.lane == 0) {
            if (sim.fail) {
                const unsigned long long slot = atomicAdd(a.ov_count, 1ull);
                if (slot < a.ov_cap) a.ov_list[slot] = rec;
            } else {
                st.add(is);
            }
        }
    }
    if (sim.sg.lane == 0) st.flush(a.accs, st_set);
}

// Device buffer layout inside KoFastState::buf.
struct FastBuf {
    unsigned long long counter[3], ov_count[3], fb_counter, pad[1];
    unsigned long long ov_list[1];   // KoFastState::ov_cap entries per pass
};

constexpr size_t kFallbackScratch = size_t(256) << 20;


template <int LANES, int G, int SAVE>
cudaError_t launch(const KoWork &a, cudaStream_t st)
{
    const int level_words = state_words(G) * SAVE + 4;
    const size_t smem = a.gstack ? 0 : sizeof(int) * (size_t)(kThreads / LANES) * a.levels * level_words;
    cudaError_t e = cudaFuncSetAttribute(fast_kernel<LANES, G, SAVE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fast_kernel<LANES, G, SAVE>, kThreads, smem);
    if (e != cudaSuccess) return e;
    long long blocks = (long long)sms * (per_sm > 0 ? per_sm : 1);
    if (a.gstack) {  // as many blocks as the slab holds segments for
        const long long fit = a.gstack_words / ((long long)(kThreads / LANES) * a.levels * level_words);
        if (blocks > fit) blocks = fit;
    }
    const long long work = a.item_list ? (long long)a.ov_cap : a.n_items;
    const long long blocks_needed = (work + kThreads / LANES - 1) / (kThreads / LANES);
    if (blocks > blocks_needed) blocks = blocks_needed;
    if (blocks < 1) blocks = 1;
    fast_kernel<LANES, G, SAVE><<<(unsigned)blocks, kThreads, smem, st>>>(a);
    ko_count_launch();
    return cudaGetLastError();
}

}  // namespace

bool ko_fast_applicable(const KoSet &h)
{
    if (h.n < 1 || h.sampling != KO_SAMPLE_BURST_END) return false;
    int64_t cmax = 0, mmax = 0;
    for (int i = 0; i < h.n; i++) {
        cmax = h.k[i].c > cmax ? h.k[i].c : cmax;
        mmax = h.k[i].m > mmax ? h.k[i].m : mmax;
    }
    const __int128 sc = (__int128)h.Bk * cmax, sm = (__int128)h.Bk * mmax;
    const __int128 dc = ((__int128)cmax * (sc > h.ccap ? sc : h.ccap) + h.ccap - 1) / h.ccap;
    const __int128 dm = ((__int128)mmax * (sm > h.mcap ? sm : h.mcap) + h.mcap - 1) / h.mcap;
    return dc < ((__int128)1 << 31) && dm < ((__int128)1 << 31);
}

int ko_fast_d0(const KoFastState &fs, int n)
{
    int levels = fs.levels < kMaxLevels ? fs.levels : kMaxLevels;
    const int d0 = n - 1 - levels;
    return d0 < 0 ? 0 : d0;
}

size_t ko_fast_smem_levels_cap() { return kMaxLevels; }

ko_status ko_fast_launch(KoFastState *fs, KoWork w, size_t max_slab_bytes, cudaStream_t st)
{
    // a pass abandons an item at most once, so lists as long as the launch's work lose none
    unsigned long long want = (unsigned long long)(w.n_items > w.reserve_items ? w.n_items : w.reserve_items);
    want = ((want < 1024 ? 1024 : want) + 1023) & ~1023ull;
    if (fs->ov_cap < want) {
        // a stream being captured cannot take a free or a malloc: the caller
        // must size the lists with an uncaptured launch first
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            cudaGetLastError();
            return KO_ERR_STATE;
        }
        const size_t need = sizeof(FastBuf) + sizeof(unsigned long long) * 3 * (size_t)want;
        cudaFree(fs->buf);
        fs->buf = nullptr;
        fs->cap = 0;
        fs->ov_cap = 0;
        if (cudaMalloc(&fs->buf, need) != cudaSuccess) {
            cudaGetLastError();
            return KO_ERR_NOMEM;
        }
        fs->cap = need;
        fs->ov_cap = want;
    }
    if (!fs->fb_scratch) {
        if (cudaMalloc(&fs->fb_scratch, kFallbackScratch) != cudaSuccess) {
            cudaGetLastError();
            return KO_ERR_NOMEM;
        }
        fs->fb_bytes = kFallbackScratch;
    }
    const bool lane = fs->lanes == 1;
    if (lane) {
        // one-thread-per-order pass: a node-state slab for every thread it runs
        const size_t need = ko_lane_slab_bytes(w.levels < 1 ? 1 : w.levels, fs->lane_shape);
        if (fs->lslab_bytes < need) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
                cudaGetLastError();
                return KO_ERR_STATE;
            }
            cudaFree(fs->lslab);
            fs->lslab = nullptr;
            fs->lslab_bytes = 0;
            if (cudaMalloc(&fs->lslab, need) != cudaSuccess) {
                cudaGetLastError();
                return KO_ERR_NOMEM;
            }
            fs->lslab_bytes = need;
        }
    }
    if (fs->stack_global) {
        // pass 1: at most 8 blocks of 8 segments per SM, 16 saved lanes per level
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int lv = w.levels < 1 ? 1 : (w.levels > kMaxLevels ? kMaxLevels : w.levels);
        const size_t need = sizeof(int) * (size_t)sms * 8 * 8 * lv * (state_words(kG) * 16 + 4);
        if (fs->gstack_bytes < need) {
            // a stream being captured cannot take a free or a malloc: the
            // caller must size the slab with an uncaptured launch first
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
                cudaGetLastError();
                return KO_ERR_STATE;
            }
            cudaFree(fs->gstack);
            fs->gstack = nullptr;
            fs->gstack_bytes = 0;
            if (cudaMalloc(&fs->gstack, need) != cudaSuccess) {
                cudaGetLastError();
                return KO_ERR_NOMEM;
            }
            fs->gstack_bytes = need;
        }
    }
    FastBuf *fb = (FastBuf *)fs->buf;
    if (cudaMemsetAsync(fb, 0, sizeof(FastBuf), st) != cudaSuccess) return KO_ERR_CUDA;
    w.run_limit = fs->run_limit;
    if (w.levels < 1) w.levels = 1;
    if (w.levels > kMaxLevels) w.levels = kMaxLevels;
    w.ov_cap = fs->ov_cap;
    w.item_list = nullptr;
    w.item_count = nullptr;
    int list = 0;  // abandoned-item list the next pass writes
    cudaError_t e = cudaSuccess;
    if (lane) {
        // pass 0: all items, one simulation per thread
        KoWork w0 = w;
        w0.counter = &fb->counter[2];
        w0.ov_count = &fb->ov_count[0];
        w0.ov_list = fb->ov_list;
        w0.gstack = (int *)fs->lslab;
        w0.gstack_words = (long long)(fs->lslab_bytes / sizeof(int));
        if ((e = ko_launch_lane(w0, fs->lane_shape, st)) != cudaSuccess) {
            cudaGetLastError();
            return KO_ERR_CUDA;
        }
        w.item_list = fb->ov_list;
        w.item_count = &fb->ov_count[0];
        list = 1;
    }
    // pass 1: all items (or those pass 0 abandoned), 16 lanes per run-length simulation, 8 group slots
    w.counter = &fb->counter[0];
    w.ov_count = &fb->ov_count[list];
    w.ov_list = fb->ov_list + list * fs->ov_cap;
    w.gstack = fs->stack_global ? (int *)fs->gstack : nullptr;
    w.gstack_words = fs->stack_global ? (long long)(fs->gstack_bytes / sizeof(int)) : 0;
    e = fs->lanes == 32 ? launch<32, kG, 16>(w, st) : launch<16, kG, 16>(w, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return KO_ERR_CUDA;
    }
    // pass 2: the items pass 1 abandoned, 32 lanes and 16 group slots per run
    KoWork w2 = w;
    w2.gstack = nullptr;  // the wide pass keeps its (32-lane) node states in shared memory
    w2.gstack_words = 0;
    w2.counter = &fb->counter[1];
    w2.item_list = fb->ov_list + list * fs->ov_cap;
    w2.item_count = &fb->ov_count[list];
    w2.ov_count = &fb->ov_count[list + 1];
    w2.ov_list = fb->ov_list + (list + 1) * fs->ov_cap;
    w2.run_limit = fs->run_limit;
    e = launch<32, kGWide, 32>(w2, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return KO_ERR_CUDA;
    }
    // pass 3: whatever is left, simple simulator
    KoWork w3 = w2;
    w3.fb_counter = &fb->fb_counter;
    e = ko_launch_fallback(w3, fs->fb_scratch, fs->fb_bytes, max_slab_bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return KO_ERR_CUDA;
    }
    return KO_OK;
}

const unsigned long long *ko_fast_overflow_counter(const KoFastState *fs)
{
    return fs->buf ? &((const FastBuf *)fs->buf)->ov_count[0] : nullptr;
}

void ko_fast_release(KoFastState *fs)
{
    if (fs->ev0) cudaEventDestroy(fs->ev0);
    if (fs->ev1) cudaEventDestroy(fs->ev1);
    fs->ev0 = fs->ev1 = nullptr;
    cudaFree(fs->buf);
    cudaFree(fs->fb_scratch);
    cudaFree(fs->gstack);
    fs->gstack = nullptr;
    fs->gstack_bytes = 0;
    cudaFree(fs->lslab);
    fs->lslab = nullptr;
    fs->lslab_bytes = 0;
    fs->buf = nullptr;
    fs->fb_scratch = nullptr;
    fs->cap = 0;
    fs->fb_bytes = 0;
}
