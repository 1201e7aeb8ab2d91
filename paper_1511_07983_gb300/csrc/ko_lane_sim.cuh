// One simulation per thread: the block-dispatch model (Sec. 2 dispatch rule,
// durations fixed at burst end from the SM's SumC / SumM) advanced one event at
// a time by a single thread, touching only the SMs an event changes.
//
// State.  SMs with identical state form runs of consecutive SM indices, kept
// in SM order (run j+1 starts where run j ends).  A run holds usage (registers,
// blocks and warps packed in one word, shared memory, SumC, SumM), the earliest
// end of its started groups, and a 64-bit mask of the slots it holds in a pool
// of groups.  A group is the blocks of one kernel started in one burst on every
// SM of a run (kernel, blocks per SM, end).  When a run splits, both halves
// keep the groups already started, which then sit in both masks; a group that
// is still pending (its burst is open) is copied to a new slot for the new
// half, so each pending group has exactly one owner run, whose SumC / SumM
// fixes its duration when the burst closes.
//
// Per event only the runs whose earliest end is the event time are touched:
// their ending groups are released, and the head kernel is offered to exactly
// those runs (every other run was full for it when the last burst ended).
// Measured on the N=12 / 148-SM set: about 11 runs and 34 groups live, 1.3 runs
// released and 1.3 groups started per event, a split every 15 events; the last
// burst of an order can split up to 13 runs.  56 slots hold every group of
// about 99 % of the 120-order work items; the rest move on to the run-length
// passes.
//
// Layout.  The state of one simulation is a column of kWords 32-bit words in
// shared memory, word f of the thread's column at col[f * STRIDE]; with STRIDE
// = the block's thread count (a multiple of 32) every access of a warp is free
// of bank conflicts whatever run or slot each thread touches.  Registers hold
// the clock, the round-robin pointer, the number of runs, the free and pending
// slot masks and the head kernel's constants.
//
// Time.  Ends are 32-bit values modulo 2^32 beside a 64-bit clock; the host
// uses this path only when every possible duration is below 2^31, so every
// comparison of (end - now) is exact.
#pragma once

#include <stdint.h>

#ifndef KO_HD
#define KO_HD __host__ __device__ __forceinline__
#endif

// Reconvergence point of the threads in `mask` (device only).
#ifdef __CUDA_ARCH__
#define KO_RECONVERGE(mask) __syncwarp(mask)
#else
#define KO_RECONVERGE(mask) ((void)(mask))
#endif

namespace kolane {

// State shape of one simulation: RUNS runs and POOL group slots, laid out as
// the column words below.  Smaller shapes let more simulations share an SM's
// shared memory; a work item that needs more is handed on (see LaneSim).
template <int RUNS, int POOL>
struct Shape {
    static_assert(RUNS <= 16 && POOL <= 64 && POOL % 2 == 0, "run and slot masks are 32 and 64 bits");
    static constexpr int kRuns = RUNS;   // runs one simulation may hold
    static constexpr int kPool = POOL;   // group slots of one simulation
    static constexpr unsigned long long kPoolAll = POOL == 64 ? ~0ull : ((1ull << POOL) - 1ull);
    static constexpr int W_RB = 0;                 // run: first SM | SM count << 16
    static constexpr int W_RU = W_RB + RUNS;       // run: registers | blocks << 19 | warps << 25 in use per SM
    static constexpr int W_RS = W_RU + RUNS;       // run: shared memory in use per SM
    static constexpr int W_RC = W_RS + RUNS;       // run: SumC
    static constexpr int W_RM = W_RC + RUNS;       // run: SumM
    static constexpr int W_RE = W_RM + RUNS;       // run: earliest end of its started groups (where valid)
    static constexpr int W_RG0 = W_RE + RUNS;      // run: pool slots 0..31 it holds
    static constexpr int W_RG1 = W_RG0 + RUNS;     // run: pool slots 32..63
    static constexpr int W_GE = W_RG1 + RUNS;      // slot: end (mod 2^32)
    static constexpr int W_GD = W_GE + POOL;       // slots 2w, 2w+1: 16-bit descriptors
    static constexpr int kWords = W_GD + POOL / 2; // 8 words per run, 1.5 per slot
    static constexpr int kSaveWords = kWords + 12; // with the registers of a node state
    static_assert(kWords % 4 == 0, "node states are copied in 16-byte pieces");
};
// The shapes the one-thread simulator is built for: 14 runs / 56 slots (200
// words), 12 / 40 (156 words), 10 / 32 (128 words).
using ShapeL = Shape<14, 56>;
using ShapeM = Shape<12, 40>;
using ShapeS = Shape<10, 32>;

// Descriptor: kernel (bits 0-4) | blocks per SM - 1 (bits 5-10) | owner run (bits 11-14).
constexpr uint32_t kDescKernel = 31u, kDescOwnerShift = 11;
// Packed usage word: registers in bits 0-18, blocks 19-24, warps 25-31.
constexpr uint32_t kRegMask = (1u << 19) - 1u;

// Registers saved with a node state (beside the column words).
constexpr int kRegWords = 12;

// The set's limits, per thread.
struct Limits {
    int n, S, R, Sh, W, Bk;
    uint32_t ccap, mcap;
    int cshift, mshift;
};

// floor(x / d) for 0 <= x <= 2^24, d >= 1, clamped to 63: the quotient of
// min(x, 63 d) estimated with a float reciprocal (error far below one unit at
// that size) and corrected once by an exact integer check.
KO_HD int quot63(int x, int d, float rcp)
{
    const int xc = x < d * 63 ? x : d * 63;
    int q = (int)((float)xc * rcp);
    if ((q + 1) * d <= xc) q++;
    if (q * d > xc) q--;
    return q;
}

KO_HD int ffs64(unsigned long long v)
{
#ifdef __CUDA_ARCH__
    return __ffsll((long long)v) - 1;
#else
    return __builtin_ffsll((long long)v) - 1;
#endif
}
KO_HD int ffs32(uint32_t v)
{
#ifdef __CUDA_ARCH__
    return __ffs((int)v) - 1;
#else
    return __builtin_ffs((int)v) - 1;
#endif
}

// Insert a copy of bit j at position j + 1 (bits above move up one).
KO_HD uint32_t dup_bit(uint32_t x, int j)
{
    const uint32_t lo = x & ((2u << j) - 1u);
    const uint32_t hi = (x >> (j + 1)) << (j + 2);
    return lo | hi | (((x >> j) & 1u) << (j + 1));
}

// Per-run 8-bit values (up to 16 runs) in two 64-bit words.
struct Bytes16 {
    unsigned long long lo, hi;
    KO_HD int get(int j) const { return (int)(((j < 8 ? lo : hi) >> ((j & 7) * 8)) & 0xffu); }
    KO_HD void set(int j, int v)
    {
        const int sh = (j & 7) * 8;
        const unsigned long long m = ~(0xffull << sh), b = (unsigned long long)(v & 0xff) << sh;
        if (j < 8) lo = (lo & m) | b; else hi = (hi & m) | b;
    }
    // insert a copy of byte j at j + 1 (bytes above move up one)
    KO_HD void dup(int j)
    {
        for (int i = 15; i > j + 1; i--) set(i, get(i - 1));
        set(j + 1, get(j));
    }
};

// Kernel constants a simulation looks up by kernel id: all of them, and the
// packed record the release and duration steps read (one 16-byte load).
struct KParam {
    int r, s, w, b, c, m;
};
struct KRel {
    uint32_t pk;   // registers | 1 << 19 | warps << 25: one block's share of the usage word
    uint32_t s, c, m;
};

template <int STRIDE, class KLoad, class SH>
struct LaneSim {
    static constexpr int kRuns = SH::kRuns, kPool = SH::kPool, kWords = SH::kWords;
    static constexpr unsigned long long kPoolAll = SH::kPoolAll;
    static constexpr int W_RB = SH::W_RB, W_RU = SH::W_RU, W_RS = SH::W_RS, W_RC = SH::W_RC, W_RM = SH::W_RM,
                         W_RE = SH::W_RE, W_RG0 = SH::W_RG0, W_RG1 = SH::W_RG1, W_GE = SH::W_GE, W_GD = SH::W_GD;
    uint32_t *col;            // word f at col[f * STRIDE]
    KLoad kl;                 // kernel constants by id
    Limits L;
    unsigned long long t;     // clock
    unsigned long long tmx;   // latest end given to any group so far
    unsigned long long freeg; // free pool slots
    unsigned long long pend;  // slots started in the open burst
    int p;                    // round-robin pointer (an SM index)
    int nr;                   // runs
    int run_limit;
    uint32_t rv;              // runs whose W_RE holds the earliest end of a started group
    int fail;
    // head kernel
    int hk, hr, hs, hw, hc, hm;
    uint32_t hpk;             // registers | 1 << 19 | warps << 25
    float frr, frs, frw;      // reciprocals of registers, shared memory, warps
    // the last offer: per-run caps, SM-weighted total, maximum, offered runs
    Bytes16 caps;
    int ctotal, cmax;
    uint32_t celig;

    KO_HD uint32_t &W(int f) const { return col[f * STRIDE]; }
    KO_HD uint32_t gd(int g) const { return (W(W_GD + (g >> 1)) >> ((g & 1) * 16)) & 0xffffu; }
    KO_HD void set_gd(int g, uint32_t v) const
    {
        uint32_t &x = W(W_GD + (g >> 1));
        const int sh = (g & 1) * 16;
        x = (x & ~(0xffffu << sh)) | (v << sh);
    }
    KO_HD unsigned long long gmask(int j) const
    {
        return (unsigned long long)W(W_RG0 + j) | ((unsigned long long)W(W_RG1 + j) << 32);
    }
    KO_HD void set_gmask(int j, unsigned long long m) const
    {
        W(W_RG0 + j) = (uint32_t)m;
        W(W_RG1 + j) = (uint32_t)(m >> 32);
    }

    KO_HD void init()
    {
        W(W_RB) = (uint32_t)L.S << 16;
        W(W_RU) = 0; W(W_RS) = 0; W(W_RC) = 0; W(W_RM) = 0;
        set_gmask(0, 0);
        nr = 1;
        t = 0;
        tmx = 0;
        p = 0;
        freeg = kPoolAll;
        pend = 0;
        rv = 0;
        fail = 0;
    }

    KO_HD void set_head(int k)
    {
        const KParam q = kl.full(k);
        hk = k; hr = q.r; hs = q.s; hw = q.w; hc = q.c; hm = q.m;
        hpk = (uint32_t)q.r | (1u << 19) | ((uint32_t)q.w << 25);
        // quot63 corrects its estimate exactly, so an approximate reciprocal will do
#ifdef __CUDA_ARCH__
        frr = __fdividef(1.0f, (float)q.r);
        frw = __fdividef(1.0f, (float)q.w);
        frs = q.s > 0 ? __fdividef(1.0f, (float)q.s) : 0.0f;
#else
        frr = 1.0f / (float)q.r;
        frw = 1.0f / (float)q.w;
        frs = q.s > 0 ? 1.0f / (float)q.s : 0.0f;
#endif
    }

    // Blocks of the head kernel one SM of run j still takes.
    KO_HD int cap(int j) const
    {
        const uint32_t u = W(W_RU + j);
        int c = L.Bk - (int)((u >> 19) & 63u);
        const int qr = quot63(L.R - (int)(u & kRegMask), hr, frr);
        const int qw = quot63(L.W - (int)(u >> 25), hw, frw);
        c = qr < c ? qr : c;
        c = qw < c ? qw : c;
        if (hs > 0) {
            const int qs = quot63(L.Sh - (int)W(W_RS + j), hs, frs);
            c = qs < c ? qs : c;
        }
        return c > 0 ? c : 0;
    }

    // Start q blocks per SM of the head kernel on run j as a new pending group.
    KO_HD void add_group(int j, int q)
    {
        if (freeg == 0) { fail = 1; return; }
        const int g = ffs64(freeg);
        freeg &= freeg - 1;
        pend |= 1ull << g;
        set_gd(g, (uint32_t)hk | ((uint32_t)(q - 1) << 5) | ((uint32_t)j << kDescOwnerShift));
        set_gmask(j, gmask(j) | (1ull << g));
        W(W_RU + j) += (uint32_t)q * hpk;
        W(W_RS + j) += (uint32_t)(q * hs);
        W(W_RC + j) += (uint32_t)(q * hc);
        W(W_RM + j) += (uint32_t)(q * hm);
    }

    // Split run j after x SMs (0 < x < its count): run j keeps the first x, a
    // new run j+1 takes the rest; runs above move up one.  The caller's
    // per-run registers (bit masks, caps) are shifted by the caller.
    KO_HD bool split(int j, int x)
    {
        if (nr >= run_limit) { fail = 1; return false; }
        for (int i = nr - 1; i > j; i--) {
            W(W_RB + i + 1) = W(W_RB + i);
            W(W_RU + i + 1) = W(W_RU + i);
            W(W_RS + i + 1) = W(W_RS + i);
            W(W_RC + i + 1) = W(W_RC + i);
            W(W_RM + i + 1) = W(W_RM + i);
            W(W_RE + i + 1) = W(W_RE + i);
            W(W_RG0 + i + 1) = W(W_RG0 + i);
            W(W_RG1 + i + 1) = W(W_RG1 + i);
        }
        const uint32_t rb = W(W_RB + j);
        const uint32_t beg = rb & 0xffffu, cnt = rb >> 16;
        W(W_RB + j) = beg | ((uint32_t)x << 16);
        W(W_RB + j + 1) = (beg + (uint32_t)x) | ((cnt - (uint32_t)x) << 16);
        W(W_RU + j + 1) = W(W_RU + j);
        W(W_RS + j + 1) = W(W_RS + j);
        W(W_RC + j + 1) = W(W_RC + j);
        W(W_RM + j + 1) = W(W_RM + j);
        W(W_RE + j + 1) = W(W_RE + j);
        rv = dup_bit(rv, j);
        nr++;
        // pending groups owned by runs above j move up with their runs
        for (unsigned long long pm = pend; pm; pm &= pm - 1) {
            const int g = ffs64(pm);
            const uint32_t d = gd(g);
            if ((int)(d >> kDescOwnerShift) > j) set_gd(g, d + (1u << kDescOwnerShift));
        }
        // run j's pending groups: the new run gets its own copies
        unsigned long long m1 = gmask(j);
        for (unsigned long long pm = m1 & pend; pm; pm &= pm - 1) {
            const int g = ffs64(pm);
            if (freeg == 0) { fail = 1; return false; }
            const int g2 = ffs64(freeg);
            freeg &= freeg - 1;
            pend |= 1ull << g2;
            set_gd(g2, (gd(g) & ((1u << kDescOwnerShift) - 1u)) | ((uint32_t)(j + 1) << kDescOwnerShift));
            m1 = (m1 & ~(1ull << g)) | (1ull << g2);
        }
        set_gmask(j + 1, m1);
        return true;
    }

    // Capacities of the head kernel on the runs in `elig` (every other run has
    // no room for it): per-run caps, their SM-weighted total and maximum.
    KO_HD void offer(uint32_t elig)
    {
        caps.lo = caps.hi = 0ull;
        ctotal = 0;
        cmax = 0;
        celig = elig;
        // runs with room for one block (four compares) take the exact capacity
        uint32_t room = 0;
        for (uint32_t e = elig; e; e &= e - 1) {
            const int j = ffs32(e);
            const uint32_t u = W(W_RU + j);
            const bool fits = (int)((u >> 19) & 63u) < L.Bk && (int)(u & kRegMask) + hr <= L.R &&
                              (int)(u >> 25) + hw <= L.W && (int)W(W_RS + j) + hs <= L.Sh;
            room |= (fits ? 1u : 0u) << j;
        }
        uint32_t take = 0;
        for (uint32_t e = room; e; e &= e - 1) {
            const int j = ffs32(e);
            const int c = cap(j);
            caps.set(j, c);
            ctotal += (int)(W(W_RB + j) >> 16) * c;
            cmax = c > cmax ? c : cmax;
            take |= (c > 0 ? 1u : 0u) << j;
        }
        celig = take;  // the placement steps visit only runs that take blocks
    }

    // Every SM of the offered runs takes its full capacity (ctotal <= left);
    // the last block lands on the SM with cap == cmax that comes last
    // cyclically from p.
    KO_HD void place_full(int &left)
    {
        const int S = L.S;
        const int pm1 = p == 0 ? S - 1 : p - 1;
        int best = 0;
        for (uint32_t e = celig; e; e &= e - 1) {
            const int j = ffs32(e);
            const int c = caps.get(j);
            if (c == 0) continue;
            add_group(j, c);
            if (c == cmax) {
                const uint32_t rb = W(W_RB + j);
                const int b = (int)(rb & 0xffffu), n = (int)(rb >> 16);
                int pos;
                if (pm1 >= b && pm1 < b + n) pos = S;
                else { pos = b + n - p; if (pos <= 0) pos += S; }
                best = pos > best ? pos : best;
            }
        }
        p += best;
        if (p >= S) p -= S;
        left -= ctotal;
    }

    // The offered runs hold more room than `left` blocks (ctotal > left): the
    // water-fill stops inside a sweep, cutting runs at p and where it stops.
    KO_HD void place_partial(int &left)
    {
        const int S = L.S;
        uint32_t elig = celig;
        // smallest sweep count L with F(L) = sum cnt * min(cap, L) >= left
        int lo = 1, hi = cmax;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            int f = 0;
            for (uint32_t e = elig; e; e &= e - 1) {
                const int j = ffs32(e);
                const int c = caps.get(j);
                f += (int)(W(W_RB + j) >> 16) * (c < mid ? c : mid);
            }
            if (f >= left) hi = mid; else lo = mid + 1;
        }
        const int Lsw = lo;
        int filled = 0;
        for (uint32_t e = elig; e; e &= e - 1) {
            const int j = ffs32(e);
            const int c = caps.get(j);
            filled += (int)(W(W_RB + j) >> 16) * (c < Lsw - 1 ? c : Lsw - 1);
        }
        const int rem = left - filled;  // 1 .. number of SMs with cap >= Lsw
        // the run holding p; cut it at p when its SMs take a block in the last sweep
        int jp = 0;
        for (int j = 0; j < nr; j++) {
            const uint32_t rb = W(W_RB + j);
            const int b = (int)(rb & 0xffffu), n = (int)(rb >> 16);
            if (b <= p && p < b + n) jp = j;
        }
        uint32_t plus = 0;
        {
            const uint32_t rb = W(W_RB + jp);
            const int b = (int)(rb & 0xffffu);
            if (((elig >> jp) & 1u) && caps.get(jp) >= Lsw && b < p) {
                if (!split(jp, p - b)) return;
                elig = dup_bit(elig, jp);
                caps.dup(jp);
                jp++;
            }
        }
        // walk the runs cyclically from jp, one more block to each SM with cap >= Lsw
        int acc = 0, newp = p, j = jp;
        for (int it = 0; it < nr; it++, j = j + 1 == nr ? 0 : j + 1) {
            if (!((elig >> j) & 1u) || caps.get(j) < Lsw) continue;
            const uint32_t rb = W(W_RB + j);
            const int b = (int)(rb & 0xffffu), n = (int)(rb >> 16);
            if (acc + n >= rem) {
                const int x = rem - acc;
                if (x < n) {
                    if (!split(j, x)) return;
                    elig = dup_bit(elig, j);
                    plus = dup_bit(plus, j) & ~(1u << (j + 1));
                    caps.dup(j);
                }
                plus |= 1u << j;
                newp = b + x;
                break;
            }
            acc += n;
            plus |= 1u << j;
        }
        p = newp >= S ? newp - S : newp;
        for (uint32_t e = elig; e; e &= e - 1) {
            const int jj = ffs32(e);
            const int c = caps.get(jj);
            const int q = (c < Lsw - 1 ? c : Lsw - 1) + (int)((plus >> jj) & 1u);
            if (q > 0) add_group(jj, q);
        }
        left = 0;
    }

    // One dispatch burst of the head kernel with `left` blocks queued over the
    // runs in `elig`.
    KO_HD void burst(int &left, uint32_t elig)
    {
        offer(elig);
        if (ctotal == 0) return;
        if (ctotal <= left) place_full(left);
        else place_partial(left);
    }

    KO_HD uint32_t duration(int k, uint32_t sc, uint32_t sm) const
    {
        // every factor fits 32 bits (c, m <= 2^24; SumC, SumM < 2^30; caps <= 2^30), so each
        // product is one 32 x 32 -> 64-bit multiply
        const KRel q = kl.rel(k);
        const uint32_t scc = sc > L.ccap ? sc : L.ccap, smm = sm > L.mcap ? sm : L.mcap;
        const unsigned long long pc = (unsigned long long)(uint32_t)q.c * scc + (L.ccap - 1u);
        const unsigned long long pmm = (unsigned long long)(uint32_t)q.m * smm + (L.mcap - 1u);
        const unsigned long long dc = L.cshift >= 0 ? pc >> L.cshift : pc / L.ccap;
        const unsigned long long dm = L.mshift >= 0 ? pmm >> L.mshift : pmm / L.mcap;
        return (uint32_t)(dc > dm ? dc : dm);
    }

    // Fix the durations of the groups started in the open burst.
    KO_HD void close_burst()
    {
        const uint32_t t32 = (uint32_t)t;
        for (unsigned long long pm = pend; pm; pm &= pm - 1) {
            const int g = ffs64(pm);
            const uint32_t d = gd(g);
            const int j = (int)(d >> kDescOwnerShift);
            const uint32_t dur = duration((int)(d & kDescKernel), W(W_RC + j), W(W_RM + j));
            const uint32_t e = t32 + dur;
            W(W_GE + g) = e;
            tmx = t + dur > tmx ? t + dur : tmx;
            if ((rv >> j) & 1u) {
                const uint32_t re = W(W_RE + j);
                if (e - t32 < re - t32) W(W_RE + j) = e;
            } else {
                W(W_RE + j) = e;
                rv |= 1u << j;
            }
        }
        pend = 0;
    }

    // Jump to the earliest end and release every group ending then; returns
    // the runs that released blocks (the only ones with room for the head).
    KO_HD uint32_t advance()
    {
        const uint32_t t32 = (uint32_t)t;
        uint32_t e[kRuns];
        uint32_t dmin = 0xffffffffu;
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
        for (int j = 0; j < kRuns; j++) {
            e[j] = 0;
            if ((rv >> j) & 1u) {
                e[j] = W(W_RE + j);
                const uint32_t d = e[j] - t32;
                dmin = d < dmin ? d : dmin;
            }
        }
        if (dmin == 0xffffffffu) { fail = 1; return 0; }
        t += dmin;
        const uint32_t now = t32 + dmin;
        uint32_t fresh = 0;
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
        for (int j = 0; j < kRuns; j++)
            if (((rv >> j) & 1u) && e[j] == now) fresh |= 1u << j;
        unsigned long long rel = 0;
        for (uint32_t f = fresh; f; f &= f - 1) {
            const int j = ffs32(f);
            const unsigned long long m = gmask(j);
            // which of the run's groups end now, and the earliest end of the rest
            unsigned long long gone = 0;
            uint32_t nm = 0xffffffffu;
            for (unsigned long long mm = m; mm; mm &= mm - 1) {
                const int g = ffs64(mm);
                const uint32_t dd = W(W_GE + g) - now;
                if (dd == 0) gone |= 1ull << g;
                else nm = dd < nm ? dd : nm;
            }
            uint32_t u = W(W_RU + j), us = W(W_RS + j), sc = W(W_RC + j), sm = W(W_RM + j);
            for (unsigned long long mm = gone; mm; mm &= mm - 1) {
                const uint32_t d = gd(ffs64(mm));
                const KRel q = kl.rel((int)(d & kDescKernel));
                const uint32_t nb = ((d >> 5) & 63u) + 1u;
                u -= nb * q.pk;
                us -= nb * q.s;
                sc -= nb * q.c;
                sm -= nb * q.m;
            }
            set_gmask(j, m & ~gone);
            W(W_RU + j) = u; W(W_RS + j) = us; W(W_RC + j) = sc; W(W_RM + j) = sm;
            if (nm != 0xffffffffu) W(W_RE + j) = now + nm;
            else rv &= ~(1u << j);
            rel |= gone;
        }
        freeg |= rel;
        return fresh;
    }

    // Queue all blocks of kernel k behind the current queue: the first burst
    // offers it every run.  Returns the blocks still queued.
    KO_HD int start_kernel(int k)
    {
        set_head(k);
        int left = kl.full(k).b;
        burst(left, (nr >= 32 ? 0xffffffffu : ((1u << nr) - 1u)));
        return left;
    }

    // One event while the head kernel still has queued blocks: close the open
    // burst, advance to the next end, release, and place the head kernel where
    // every offered SM takes its full capacity.  Returns true when the offered
    // room exceeds the queue instead; the caller then finishes the burst with
    // place_partial (the kernel's last burst).  `mask`: the threads of the warp
    // that run this event step together; they reconverge after each stage.
    KO_HD bool event(int &left, unsigned mask)
    {
        close_burst();
        KO_RECONVERGE(mask);
        const uint32_t fresh = advance();
        KO_RECONVERGE(mask);
        offer(fail ? 0u : fresh);  // a failed simulation still reaches every reconvergence point
        KO_RECONVERGE(mask);
        if (fail || ctotal == 0) return false;
        if (ctotal <= left) {
            place_full(left);
            return false;
        }
        return true;
    }

    // Close the final burst; the makespan is the latest end of any group.
    KO_HD long long finish()
    {
        close_burst();
        return (long long)tmx;
    }

    // Registers of a node state.
    KO_HD void regs_out(uint32_t *r) const
    {
        r[0] = (uint32_t)t; r[1] = (uint32_t)(t >> 32);
        r[2] = (uint32_t)freeg; r[3] = (uint32_t)(freeg >> 32);
        r[4] = (uint32_t)pend; r[5] = (uint32_t)(pend >> 32);
        r[6] = (uint32_t)p; r[7] = (uint32_t)nr; r[8] = rv;
        r[9] = (uint32_t)tmx; r[10] = (uint32_t)(tmx >> 32); r[11] = 0;
    }
    KO_HD void regs_in(const uint32_t *r)
    {
        t = (unsigned long long)r[0] | ((unsigned long long)r[1] << 32);
        freeg = (unsigned long long)r[2] | ((unsigned long long)r[3] << 32);
        pend = (unsigned long long)r[4] | ((unsigned long long)r[5] << 32);
        p = (int)r[6]; nr = (int)r[7]; rv = r[8];
        tmx = (unsigned long long)r[9] | ((unsigned long long)r[10] << 32);
        fail = 0;
    }
};

}  // namespace kolane
