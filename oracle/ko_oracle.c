/*
 * ko_oracle.c -- plain, slow, obviously correct CPU oracle for launch-order
 * scoring (Li, Narayana, El-Ghazawi, "Reordering GPU Kernel Launches to Enable
 * Efficient Concurrent Execution").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or runs
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code, header or constant with the CUDA library.
 *
 * Contents (each function cites the passage it follows):
 *   or_unrank / or_rank      lexicographic Lehmer code over the N! launch
 *                            orders (the "all permutations" space, Sec. 6).
 *   or_makespan              block-by-block dispatch simulation of one order
 *                            (Sec. 2 dispatch rule; duration rule = reading A1).
 *   or_makespan_sampled      the same with durations fixed at placement instead
 *                            of at the end of the burst (model variant).
 *   or_makespan_ps           processor sharing: rates re-evaluated at every
 *                            event (model variant, double precision).
 *   or_makespans_idx         many orders by Lehmer index, pthreads over ranges.
 *   or_heuristic             Algorithm 1 (ScoreGen, ProfileCombine, rounds);
 *   or_heuristic_fp          the same with a choice of footprint reading.
 *   or_local_search          steepest-descent hill climbing from an order,
 *                            every candidate scored by or_makespan.
 *   or_bounds                work/capacity lower bound and serial upper bound.
 *
 * Model (Sec. 2 and the readings recorded in the design notes):
 *   - blocks are queued kernel by kernel in launch order (all blocks of the
 *     earliest-issued kernel before any block of the next); strict FIFO, a
 *     head block that fits nowhere blocks the queue (head-of-line blocking);
 *   - a head block goes to the first SM, scanning cyclically from the
 *     round-robin pointer p, whose registers, shared memory, warps and block
 *     slots all still fit it (Sec. 2, four SM limits); p becomes that SM + 1;
 *   - at time t: release every block ending at t, place blocks (one burst),
 *     then give each block started in this burst the duration
 *        d = max( ceil(c * max(SumC, Ccap) / Ccap), ceil(m * max(SumM, Mcap) / Mcap) )
 *     where SumC/SumM are the totals over all blocks resident on its SM after
 *     the burst (compute/memory balance, Sec. 4; R_B = Ccap / Mcap);
 *   - advance t to the earliest end; the makespan is the last end.
 * All simulation arithmetic is 64-bit integer.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef struct {
    int64_t n_sm, n_reg_sm, n_shm_sm, n_warp_sm, n_blk_sm, c_cap, m_cap;
} or_gpu;

/* per block: registers, shared-memory bytes, warps; block count; cycles */
typedef struct {
    int64_t n_reg, n_shm, n_warp, n_tblk, c, m;
} or_kernel;

/* ---------------------------------------------------------------- Lehmer --- */

static uint64_t fact(int n)
{
    uint64_t f = 1;
    for (int i = 2; i <= n; i++) f *= (uint64_t)i;
    return f;
}

/* Index k in [0, n!) -> the k-th permutation of 0..n-1 in lexicographic order.
 * Digit j (most significant first) is k / (n-1-j)!, and selects the digit-th
 * smallest kernel index not used yet. */
void or_unrank(int n, uint64_t k, int32_t *perm)
{
    int used[64] = {0};
    for (int j = 0; j < n; j++) {
        uint64_t f = fact(n - 1 - j);
        uint64_t d = k / f;
        k = k % f;
        int seen = 0;
        for (int v = 0; v < n; v++) {
            if (used[v]) continue;
            if ((uint64_t)seen == d) { perm[j] = v; used[v] = 1; break; }
            seen++;
        }
    }
}

/* Inverse of or_unrank. */
uint64_t or_rank(int n, const int32_t *perm)
{
    uint64_t k = 0;
    for (int j = 0; j < n; j++) {
        uint64_t smaller_later = 0;
        for (int l = j + 1; l < n; l++)
            if (perm[l] < perm[j]) smaller_later++;
        k += smaller_later * fact(n - 1 - j);
    }
    return k;
}

/* ------------------------------------------------------------- simulator --- */

static int64_t ceil_div(int64_t x, int64_t y) { return (x + y - 1) / y; }
static int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

/* duration of a block with demands (c, m) on an SM whose resident blocks sum to
 * (sum_c, sum_m) after the burst (reading A1). */
static int64_t duration(const or_gpu *g, int64_t c, int64_t m, int64_t sum_c, int64_t sum_m)
{
    int64_t dc = ceil_div(c * max64(sum_c, g->c_cap), g->c_cap);
    int64_t dm = ceil_div(m * max64(sum_m, g->m_cap), g->m_cap);
    return max64(dc, dm);
}

typedef struct {
    int32_t kernel; /* kernel index */
    int32_t is_new; /* started in the current burst, duration not yet fixed */
    int64_t end;
} resident_block;

/* Makespan of launch order `order` (a permutation of 0..n-1).  Returns -1 if a
 * block cannot fit an empty SM (the simulation could never finish).
 *
 * at_placement selects when a block's duration is fixed: 0 = after the burst
 * that started it, with SumC/SumM over everything then resident on its SM
 * (reading A2, or_makespan); 1 = the moment it is placed, with SumC/SumM over
 * the blocks resident at that moment, itself included and blocks placed later
 * in the same burst excluded (the alternative reading of the same passage). */
int64_t or_makespan_sampled(const or_gpu *g, int n, const or_kernel *k, const int32_t *order, int at_placement)
{
    const int64_t S = g->n_sm, Bk = g->n_blk_sm;
    for (int i = 0; i < n; i++) {
        if (k[i].n_reg > g->n_reg_sm || k[i].n_shm > g->n_shm_sm ||
            k[i].n_warp > g->n_warp_sm || 1 > Bk)
            return -1;
    }
    int64_t *used_r = calloc((size_t)S, sizeof(int64_t));
    int64_t *used_s = calloc((size_t)S, sizeof(int64_t));
    int64_t *used_w = calloc((size_t)S, sizeof(int64_t));
    int64_t *used_b = calloc((size_t)S, sizeof(int64_t));
    int64_t *sum_c = calloc((size_t)S, sizeof(int64_t));
    int64_t *sum_m = calloc((size_t)S, sizeof(int64_t));
    resident_block *res = calloc((size_t)(S * Bk), sizeof(resident_block));

    int64_t t = 0, makespan = 0, p = 0;
    int pos = 0;                                  /* queue head: kernel order[pos] */
    int64_t left = n > 0 ? k[order[0]].n_tblk : 0; /* blocks of the head kernel left */
    while (pos < n && left == 0) { pos++; left = pos < n ? k[order[pos]].n_tblk : 0; }

    for (;;) {
        /* release every block that ends at t */
        for (int64_t s = 0; s < S; s++) {
            int64_t j = 0;
            while (j < used_b[s]) {
                resident_block *rb = &res[s * Bk + j];
                if (!rb->is_new && rb->end == t) {
                    const or_kernel *kk = &k[rb->kernel];
                    used_r[s] -= kk->n_reg; used_s[s] -= kk->n_shm; used_w[s] -= kk->n_warp;
                    sum_c[s] -= kk->c; sum_m[s] -= kk->m;
                    res[s * Bk + j] = res[s * Bk + used_b[s] - 1];
                    used_b[s]--;
                } else {
                    j++;
                }
            }
        }
        /* one dispatch burst: FIFO, round-robin first fit from p */
        while (pos < n) {
            const int i = order[pos];
            const or_kernel *kk = &k[i];
            int64_t found = -1;
            for (int64_t off = 0; off < S; off++) {
                int64_t s = (p + off) % S;
                if (used_r[s] + kk->n_reg <= g->n_reg_sm && used_s[s] + kk->n_shm <= g->n_shm_sm &&
                    used_w[s] + kk->n_warp <= g->n_warp_sm && used_b[s] + 1 <= Bk) {
                    found = s;
                    break;
                }
            }
            if (found < 0) break; /* head-of-line blocking */
            int64_t s = found;
            resident_block *rb = &res[s * Bk + used_b[s]];
            rb->kernel = i; rb->is_new = 1; rb->end = 0;
            used_r[s] += kk->n_reg; used_s[s] += kk->n_shm; used_w[s] += kk->n_warp; used_b[s]++;
            sum_c[s] += kk->c; sum_m[s] += kk->m;
            if (at_placement) {
                rb->end = t + duration(g, kk->c, kk->m, sum_c[s], sum_m[s]);
                rb->is_new = 0;
                if (rb->end > makespan) makespan = rb->end;
            }
            p = (s + 1) % S;
            left--;
            while (pos < n && left == 0) { pos++; left = pos < n ? k[order[pos]].n_tblk : 0; }
        }
        /* fix durations of the blocks started in this burst */
        int any_resident = 0;
        for (int64_t s = 0; s < S; s++) {
            for (int64_t j = 0; j < used_b[s]; j++) {
                resident_block *rb = &res[s * Bk + j];
                if (rb->is_new) {
                    const or_kernel *kk = &k[rb->kernel];
                    rb->end = t + duration(g, kk->c, kk->m, sum_c[s], sum_m[s]);
                    rb->is_new = 0;
                    if (rb->end > makespan) makespan = rb->end;
                }
                any_resident = 1;
            }
        }
        if (!any_resident) {
            if (pos < n) { makespan = -1; } /* cannot happen for valid sets */
            break;
        }
        /* advance to the earliest end */
        int64_t tmin = INT64_MAX;
        for (int64_t s = 0; s < S; s++)
            for (int64_t j = 0; j < used_b[s]; j++)
                if (res[s * Bk + j].end < tmin) tmin = res[s * Bk + j].end;
        t = tmin;
    }
    free(used_r); free(used_s); free(used_w); free(used_b);
    free(sum_c); free(sum_m); free(res);
    return makespan;
}

int64_t or_makespan(const or_gpu *g, int n, const or_kernel *k, const int32_t *order)
{
    return or_makespan_sampled(g, n, k, order, 0);
}

/* ------------------------------------------------------ many orders, threads --- */

typedef struct {
    const or_gpu *g;
    int n;
    const or_kernel *k;
    const uint64_t *idx; /* NULL: contiguous indices first + j */
    uint64_t first;
    int64_t begin, end;
    int64_t *out;
} work_range;

static void *range_worker(void *arg)
{
    work_range *w = (work_range *)arg;
    int32_t perm[64];
    for (int64_t j = w->begin; j < w->end; j++) {
        uint64_t index = w->idx ? w->idx[j] : w->first + (uint64_t)j;
        or_unrank(w->n, index, perm);
        w->out[j] = or_makespan(w->g, w->n, w->k, perm);
    }
    return NULL;
}

/* Makespans of `count` orders: Lehmer indices idx[j] (or first + j when idx is
 * NULL).  Work is split into `threads` contiguous ranges. */
void or_makespans_idx(const or_gpu *g, int n, const or_kernel *k, const uint64_t *idx,
                      uint64_t first, int64_t count, int64_t *out, int threads)
{
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    pthread_t tid[256];
    work_range wr[256];
    for (int t = 0; t < threads; t++) {
        wr[t].g = g; wr[t].n = n; wr[t].k = k; wr[t].idx = idx; wr[t].first = first;
        wr[t].begin = count * t / threads;
        wr[t].end = count * (t + 1) / threads;
        wr[t].out = out;
        pthread_create(&tid[t], NULL, range_worker, &wr[t]);
    }
    for (int t = 0; t < threads; t++) pthread_join(tid[t], NULL);
}

/* Makespans of explicit orders (row-major [count, n]). */
void or_makespans_orders(const or_gpu *g, int n, const or_kernel *k, const int32_t *orders,
                         int64_t count, int64_t *out)
{
    for (int64_t j = 0; j < count; j++) out[j] = or_makespan(g, n, k, orders + j * n);
}

void or_makespans_orders_sampled(const or_gpu *g, int n, const or_kernel *k, const int32_t *orders,
                                 int64_t count, int at_placement, int64_t *out)
{
    for (int64_t j = 0; j < count; j++) out[j] = or_makespan_sampled(g, n, k, orders + j * n, at_placement);
}

/* ------------------------------------------------- processor sharing --- */
/*
 * Model variant: processor sharing with rates re-evaluated at every event.
 * Dispatch is the same FIFO round-robin first fit (Sec. 2).  A resident block
 * has remaining compute work Rc (c at start) and memory work Rm (m at start);
 * on an SM whose resident demands sum to SumC and SumM, every block progresses
 * at rate rc = Ccap / max(SumC, Ccap) on Rc and rm = Mcap / max(SumM, Mcap) on
 * Rm, and it ends when both reach zero: at t + max(Rc / rc, Rm / rm) if the
 * rates stay.  When an SM's residents change (a release or a placement at
 * time t), its other blocks are first advanced to t at the old rates, then
 * their ends are recomputed at the new rates.  With residents that never
 * change this is the duration rule of reading A1 without the rounding up.
 * Times are doubles, every operation written out in a fixed order (compiled
 * without contraction) so that another implementation with the same order
 * gets the same bits; groups whose end equals the event time leave together.
 * Returns -1 if a block cannot fit an empty SM.
 */
typedef struct {
    int32_t kernel, fresh;
    int64_t cnt;
    double rc_left, rm_left, t_upd, end;
} ps_group;

static double ps_rate(int64_t sum, int64_t cap)
{
    return sum <= cap ? 1.0 : (double)cap / (double)sum;
}

double or_makespan_ps(const or_gpu *g, int n, const or_kernel *k, const int32_t *order)
{
    const int64_t S = g->n_sm, Bk = g->n_blk_sm;
    for (int i = 0; i < n; i++)
        if (k[i].n_reg > g->n_reg_sm || k[i].n_shm > g->n_shm_sm || k[i].n_warp > g->n_warp_sm)
            return -1.0;
    int64_t *ur = calloc((size_t)S, sizeof(int64_t)), *us = calloc((size_t)S, sizeof(int64_t));
    int64_t *uw = calloc((size_t)S, sizeof(int64_t)), *ub = calloc((size_t)S, sizeof(int64_t));
    int64_t *sc = calloc((size_t)S, sizeof(int64_t)), *sm = calloc((size_t)S, sizeof(int64_t));
    double *rate_c = malloc(sizeof(double) * (size_t)S), *rate_m = malloc(sizeof(double) * (size_t)S);
    int *ng = calloc((size_t)S, sizeof(int)), *changed = calloc((size_t)S, sizeof(int));
    ps_group *gr = calloc((size_t)(S * Bk), sizeof(ps_group));
    for (int64_t s = 0; s < S; s++) { rate_c[s] = 1.0; rate_m[s] = 1.0; }

    double t = 0.0, makespan = 0.0;
    int64_t p = 0;
    int pos = 0;
    int64_t left = n > 0 ? k[order[0]].n_tblk : 0;
    while (pos < n && left == 0) { pos++; left = pos < n ? k[order[pos]].n_tblk : 0; }
    for (;;) {
        /* release every group whose end is t */
        for (int64_t s = 0; s < S; s++) {
            changed[s] = 0;
            for (int j = 0; j < ng[s];) {
                ps_group *q = &gr[s * Bk + j];
                if (q->end == t) {
                    const or_kernel *kk = &k[q->kernel];
                    ur[s] -= q->cnt * kk->n_reg; us[s] -= q->cnt * kk->n_shm; uw[s] -= q->cnt * kk->n_warp;
                    ub[s] -= q->cnt; sc[s] -= q->cnt * kk->c; sm[s] -= q->cnt * kk->m;
                    gr[s * Bk + j] = gr[s * Bk + ng[s] - 1];
                    ng[s]--;
                    changed[s] = 1;
                } else {
                    j++;
                }
            }
        }
        /* one dispatch burst: FIFO, round-robin first fit from p */
        while (pos < n) {
            const int i = order[pos];
            const or_kernel *kk = &k[i];
            int64_t f = -1;
            for (int64_t off = 0; off < S; off++) {
                int64_t s = (p + off) % S;
                if (ur[s] + kk->n_reg <= g->n_reg_sm && us[s] + kk->n_shm <= g->n_shm_sm &&
                    uw[s] + kk->n_warp <= g->n_warp_sm && ub[s] + 1 <= Bk) {
                    f = s;
                    break;
                }
            }
            if (f < 0) break;
            int j = 0;
            while (j < ng[f] && !(gr[f * Bk + j].fresh && gr[f * Bk + j].kernel == i)) j++;
            if (j == ng[f]) {
                ps_group *q = &gr[f * Bk + j];
                q->kernel = i; q->fresh = 1; q->cnt = 0;
                q->rc_left = (double)kk->c; q->rm_left = (double)kk->m; q->t_upd = t; q->end = 0.0;
                ng[f]++;
            }
            gr[f * Bk + j].cnt++;
            ur[f] += kk->n_reg; us[f] += kk->n_shm; uw[f] += kk->n_warp; ub[f]++;
            sc[f] += kk->c; sm[f] += kk->m;
            changed[f] = 1;
            p = (f + 1) % S;
            left--;
            while (pos < n && left == 0) { pos++; left = pos < n ? k[order[pos]].n_tblk : 0; }
        }
        /* advance the changed SMs' blocks to t at the old rates, re-time them at the new */
        for (int64_t s = 0; s < S; s++) {
            if (!changed[s]) continue;
            const double nrc = ps_rate(sc[s], g->c_cap), nrm = ps_rate(sm[s], g->m_cap);
            for (int j = 0; j < ng[s]; j++) {
                ps_group *q = &gr[s * Bk + j];
                if (!q->fresh) {
                    const double dt = t - q->t_upd;
                    double a = rate_c[s] * dt;
                    q->rc_left = q->rc_left - a;
                    if (q->rc_left < 0.0) q->rc_left = 0.0;
                    a = rate_m[s] * dt;
                    q->rm_left = q->rm_left - a;
                    if (q->rm_left < 0.0) q->rm_left = 0.0;
                    q->t_upd = t;
                }
                q->fresh = 0;
                const double tc = q->rc_left / nrc, tm = q->rm_left / nrm;
                q->end = t + (tc > tm ? tc : tm);
            }
            rate_c[s] = nrc;
            rate_m[s] = nrm;
        }
        /* next event */
        double tmin = -1.0;
        for (int64_t s = 0; s < S; s++)
            for (int j = 0; j < ng[s]; j++)
                if (tmin < 0.0 || gr[s * Bk + j].end < tmin) tmin = gr[s * Bk + j].end;
        if (tmin < 0.0) {
            if (pos < n) makespan = -1.0;
            break;
        }
        t = tmin;
        makespan = t;
    }
    free(ur); free(us); free(uw); free(ub); free(sc); free(sm);
    free(rate_c); free(rate_m); free(ng); free(changed); free(gr);
    return makespan;
}

void or_makespans_ps(const or_gpu *g, int n, const or_kernel *k, const int32_t *orders, int64_t count,
                     double *out)
{
    for (int64_t j = 0; j < count; j++) out[j] = or_makespan_ps(g, n, k, orders + j * n);
}

/* ------------------------------------------------------------- Algorithm 1 --- */
/*
 * Readings: a kernel's resource terms use its per-SM footprint
 * F_i = ceil(N_tblk_i / N_SM) * (regs, smem, warps, 1 block); a group of kernels
 * "fits within an execution round" when the summed footprints are within
 * (N_reg_SM, N_shm_SM, N_warp_SM, N_blk_SM).  R_i = c_i / m_i,
 * R_B = Ccap / Mcap, N_inst_i = N_tblk_i * c_i and N_inst_i / R_i = N_tblk_i * m_i,
 * so ProfileCombine's R_comb is (sum of N_tblk*c) / (sum of N_tblk*m).
 */
typedef struct {
    int64_t fr, fs, fw, fb; /* per-SM footprint */
    int64_t inst, mem;      /* sum N_tblk*c, sum N_tblk*m */
} profile;

/* per_block = 1 is the alternative reading of the resource terms: one block's
 * registers, shared memory and warps (footprint multiplier q = 1). */
static profile profile_of_fp(const or_gpu *g, const or_kernel *kk, int per_block)
{
    profile pr;
    int64_t q = per_block ? 1 : (kk->n_tblk + g->n_sm - 1) / g->n_sm;
    pr.fr = q * kk->n_reg;
    pr.fs = q * kk->n_shm;
    pr.fw = q * kk->n_warp;
    pr.fb = q;
    pr.inst = kk->n_tblk * kk->c;
    pr.mem = kk->n_tblk * kk->m;
    return pr;
}

static profile profile_of(const or_gpu *g, const or_kernel *kk) { return profile_of_fp(g, kk, 0); }

/* ProfileCombine(K_a, K_b): summed footprints, summed instruction and memory
 * totals (the weighted-harmonic R_comb follows from them). */
static profile profile_combine(profile a, profile b)
{
    profile c;
    c.fr = a.fr + b.fr; c.fs = a.fs + b.fs; c.fw = a.fw + b.fw; c.fb = a.fb + b.fb;
    c.inst = a.inst + b.inst; c.mem = a.mem + b.mem;
    return c;
}

static int profiles_fit(const or_gpu *g, profile a, profile b)
{
    return a.fr + b.fr <= g->n_reg_sm && a.fs + b.fs <= g->n_shm_sm &&
           a.fw + b.fw <= g->n_warp_sm && a.fb + b.fb <= g->n_blk_sm;
}

static double dmax(double a, double b) { return a > b ? a : b; }

/* ScoreGen for one pair: zero if they do not fit together, otherwise the free
 * fractions of shared memory, registers and warps, plus the balance term when
 * the two ratios lie on opposite sides of R_B. */
static double score_pair(const or_gpu *g, profile a, profile b)
{
    if (!profiles_fit(g, a, b)) return 0.0;
    double s = 0.0;
    s += dmax((double)(g->n_shm_sm - a.fs - b.fs) / (double)g->n_shm_sm, 0.0);
    s += dmax((double)(g->n_reg_sm - a.fr - b.fr) / (double)g->n_reg_sm, 0.0);
    s += dmax((double)(g->n_warp_sm - a.fw - b.fw) / (double)g->n_warp_sm, 0.0);
    double ra = (double)a.inst / (double)a.mem;
    double rb = (double)b.inst / (double)b.mem;
    double rB = (double)g->c_cap / (double)g->m_cap;
    if ((ra <= rB && rB <= rb) || (rb <= rB && rB <= ra)) {
        double rcomb = (double)(a.inst + b.inst) / (double)(a.mem + b.mem);
        double dev = rcomb - rB;
        if (dev < 0) dev = -dev;
        s += dmax(1.0 - dev / rB, 0.0);
    }
    return s;
}

/* Writes the launch order (n kernel indices) to order_out.  Returns the number
 * of execution rounds.  per_block selects the footprint reading (see
 * profile_of_fp); or_heuristic is the per-SM reading. */
int or_heuristic_fp(const or_gpu *g, int n, const or_kernel *k, int per_block, int32_t *order_out)
{
    profile pr[64];
    int remaining[64];
    double score[64][64];
    for (int i = 0; i < n; i++) { pr[i] = profile_of_fp(g, &k[i], per_block); remaining[i] = 1; }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            score[i][j] = (i == j) ? 0.0 : score_pair(g, pr[i], pr[j]);

    int out = 0, rounds = 0, left = n;
    while (left > 0) {
        rounds++;
        int round_members[64];
        int rn = 0;
        if (left == 1) {
            for (int i = 0; i < n; i++)
                if (remaining[i]) { order_out[out++] = i; remaining[i] = 0; }
            left = 0;
            break;
        }
        /* best pair among the remaining kernels; first maximum in (i, j) order */
        int ba = -1, bb = -1;
        double best = -1.0;
        for (int i = 0; i < n; i++) {
            if (!remaining[i]) continue;
            for (int j = i + 1; j < n; j++) {
                if (!remaining[j]) continue;
                if (score[i][j] > best) { best = score[i][j]; ba = i; bb = j; }
            }
        }
        /* pair enters the round by decreasing shared-memory footprint */
        if (pr[bb].fs > pr[ba].fs) { round_members[0] = bb; round_members[1] = ba; }
        else { round_members[0] = ba; round_members[1] = bb; }
        rn = 2;
        remaining[ba] = 0; remaining[bb] = 0; left -= 2;
        profile comb = profile_combine(pr[ba], pr[bb]);
        /* keep adding the best-scoring kernel that still fits with the round */
        for (;;) {
            int bc = -1;
            double bs = -1.0;
            for (int r = 0; r < n; r++) {
                if (!remaining[r]) continue;
                if (!profiles_fit(g, comb, pr[r])) continue;
                double s = score_pair(g, comb, pr[r]);
                if (s > bs) { bs = s; bc = r; }
            }
            if (bc < 0) break;
            if (pr[bc].fs > comb.fs) {
                for (int q = rn; q > 0; q--) round_members[q] = round_members[q - 1];
                round_members[0] = bc;
            } else {
                round_members[rn] = bc;
            }
            rn++;
            comb = profile_combine(comb, pr[bc]);
            remaining[bc] = 0; left--;
        }
        for (int q = 0; q < rn; q++) order_out[out++] = round_members[q];
    }
    return rounds;
}

int or_heuristic(const or_gpu *g, int n, const or_kernel *k, int32_t *order_out)
{
    return or_heuristic_fp(g, n, k, 0, order_out);
}

/* ------------------------------------------------- exact local search --- */
/*
 * Steepest-descent hill climbing over launch orders, every candidate scored
 * exactly by or_makespan (the "reorder, then measure" loop of Sec. 6 run as a
 * search instead of an enumeration).  The neighbours of an order p are, in
 * this order:
 *   swaps  q = 0 .. n(n-1)/2-1:  exchange positions (i, j), i < j, pairs in
 *          lexicographic order;
 *   moves  (hood = 1 only) q = n(n-1)/2 + from*(n-1) + t:  take the kernel at
 *          position `from` out and reinsert it at position `to`, where `to`
 *          runs over 0..n-1 without `from` (to = t if t < from, else t + 1).
 * One step evaluates every neighbour and moves to the lowest makespan, the
 * lowest q among equals, only if it is strictly below the current makespan.
 * Stops at a local optimum or after max_iters steps.  Returns the number of
 * steps taken; *evals_out counts the orders scored (start included).
 */
static void neighbour(int n, const int32_t *p, int q, int32_t *out)
{
    int swaps = n * (n - 1) / 2;
    for (int i = 0; i < n; i++) out[i] = p[i];
    if (q < swaps) {
        int i = 0, rem = q;
        while (rem >= n - 1 - i) { rem -= n - 1 - i; i++; }
        int j = i + 1 + rem;
        int32_t t = out[i]; out[i] = out[j]; out[j] = t;
        return;
    }
    int mv = q - swaps, from = mv / (n - 1), t = mv % (n - 1);
    int to = t < from ? t : t + 1;
    /* remove, then insert */
    int32_t tmp[64];
    int w = 0;
    for (int i = 0; i < n; i++) if (i != from) tmp[w++] = p[i];
    w = 0;
    for (int i = 0; i < n; i++) out[i] = (i == to) ? p[from] : tmp[w++];
}

int or_local_search(const or_gpu *g, int n, const or_kernel *k, const int32_t *start, int hood,
                    int max_iters, int32_t *order_out, int64_t *makespan_out, int64_t *evals_out)
{
    int32_t cur[64], cand[64], best_nb[64];
    int nq = n * (n - 1) / 2 + (hood ? n * (n - 1) : 0);
    for (int i = 0; i < n; i++) cur[i] = start[i];
    int64_t cur_ms = or_makespan(g, n, k, cur), evals = 1;
    int steps = 0;
    while (steps < max_iters && nq > 0) {
        int64_t best = -1;
        for (int q = 0; q < nq; q++) {
            neighbour(n, cur, q, cand);
            int64_t ms = or_makespan(g, n, k, cand);
            evals++;
            if (best < 0 || ms < best) { best = ms; memcpy(best_nb, cand, sizeof(int32_t) * n); }
        }
        if (best >= cur_ms) break;
        cur_ms = best;
        memcpy(cur, best_nb, sizeof(int32_t) * n);
        steps++;
    }
    for (int i = 0; i < n; i++) order_out[i] = cur[i];
    *makespan_out = cur_ms;
    *evals_out = evals;
    return steps;
}

/* Score matrix as Algorithm 1 builds it (for tests); row-major [n, n]. */
void or_score_matrix(const or_gpu *g, int n, const or_kernel *k, double *out)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            out[i * n + j] = (i == j) ? 0.0 : score_pair(g, profile_of(g, &k[i]), profile_of(g, &k[j]));
}

/* ------------------------------------------------------------------ bounds --- */
/*
 * Lower bound: every block lasts at least its alone-duration d0 (SumC >= c), no
 * SM holds more than its limits at once, so each limit gives an area bound, and
 * no order beats the longest single block.  Upper bound: some block is always
 * running until the end (every block fits an empty SM), so the makespan is at
 * most the sum of all block durations, each at most d computed with
 * SumC <= N_blk_SM * max c and SumM <= N_blk_SM * max m.
 */
static int64_t ceil_div128(__int128 x, __int128 y) { return (int64_t)((x + y - 1) / y); }

void or_bounds(const or_gpu *g, int n, const or_kernel *k, int64_t *lb, int64_t *ub)
{
    int64_t maxc = 0, maxm = 0, dmax0 = 0;
    __int128 a_blk = 0, a_warp = 0, a_reg = 0, a_shm = 0, upper = 0;
    int any_shm = 0;
    for (int i = 0; i < n; i++) {
        if (k[i].c > maxc) maxc = k[i].c;
        if (k[i].m > maxm) maxm = k[i].m;
    }
    for (int i = 0; i < n; i++) {
        int64_t d0 = duration(g, k[i].c, k[i].m, k[i].c, k[i].m);
        if (d0 > dmax0) dmax0 = d0;
        __int128 bd = (__int128)k[i].n_tblk * d0;
        a_blk += bd;
        a_warp += bd * k[i].n_warp;
        a_reg += bd * k[i].n_reg;
        a_shm += bd * k[i].n_shm;
        if (k[i].n_shm > 0) any_shm = 1;
        int64_t dm = duration(g, k[i].c, k[i].m, g->n_blk_sm * maxc, g->n_blk_sm * maxm);
        upper += (__int128)k[i].n_tblk * dm;
    }
    int64_t L = dmax0;
    int64_t v;
    v = ceil_div128(a_blk, (__int128)g->n_sm * g->n_blk_sm); if (v > L) L = v;
    v = ceil_div128(a_warp, (__int128)g->n_sm * g->n_warp_sm); if (v > L) L = v;
    v = ceil_div128(a_reg, (__int128)g->n_sm * g->n_reg_sm); if (v > L) L = v;
    if (any_shm) { v = ceil_div128(a_shm, (__int128)g->n_sm * g->n_shm_sm); if (v > L) L = v; }
    *lb = n > 0 ? L : 0;
    *ub = upper > (__int128)INT64_MAX ? INT64_MAX : (int64_t)upper;
}
