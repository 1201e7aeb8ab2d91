// Host-side parts of the method: Algorithm 1 (launch-order heuristic) and the
// makespan bounds used to validate a set and to size integer arithmetic.
//
// Algorithm 1 readings (the paper leaves these open):
//   * resource terms use a kernel's per-SM footprint: q = ceil(N_tblk / N_SM)
//     blocks, i.e. q * (registers, shared memory, warps, 1 block slot); the
//     per-block reading (q = 1) is selectable for comparison;
//   * "fits within an execution round" = summed footprints within the four
//     per-SM limits;
//   * R_i = c_i / m_i; R_B = Ccap / Mcap; a combined profile carries the sums
//     of N_tblk*c (instructions) and N_tblk*m (memory), so
//     R_comb = sum(N_tblk c) / sum(N_tblk m) -- ProfileCombine's weighted form;
//   * a score is the sum, in this order, of the free shared-memory, register
//     and warp fractions (each clamped at 0) and, when the two ratios lie on
//     opposite sides of R_B, max(1 - |R_comb - R_B| / R_B, 0);
//   * ties go to the lowest index pair (strict '>' scan); the first pair is
//     taken even when every score is 0; a lone remaining kernel is a round;
//   * the seed pair enters by decreasing shared-memory footprint (lower index
//     first on ties); a kernel added later goes in front of the round when its
//     footprint exceeds the round's combined one, else at the back.
// Scores are IEEE doubles evaluated in the order written above, compiled
// without floating-point contraction, so every build gives the same order.
#include <algorithm>
#include <vector>

#include "ko_internal.h"

namespace {

struct Footprint {
    int64_t reg, shm, warp, blk;   // per-SM footprint
    int64_t inst, mem;             // sum N_tblk * c, sum N_tblk * m
};

// per_block: the alternative reading, one block's resources (q = 1)
Footprint footprint(const KoSet &h, const KoKern &k, bool per_block)
{
    const int64_t q = per_block ? 1 : ((int64_t)k.b + h.S - 1) / h.S;
    return Footprint{q * k.r, q * k.s, q * k.w, q, (int64_t)k.b * k.c, (int64_t)k.b * k.m};
}

Footprint combine(const Footprint &a, const Footprint &b)
{
    return Footprint{a.reg + b.reg, a.shm + b.shm, a.warp + b.warp, a.blk + b.blk,
                     a.inst + b.inst, a.mem + b.mem};
}

bool fit_together(const KoSet &h, const Footprint &a, const Footprint &b)
{
    return a.reg + b.reg <= h.R && a.shm + b.shm <= h.Sh && a.warp + b.warp <= h.W &&
           a.blk + b.blk <= h.Bk;
}

double clamp0(double v) { return v > 0.0 ? v : 0.0; }

double pair_score(const KoSet &h, const Footprint &x, const Footprint &y)
{
    if (!fit_together(h, x, y)) return 0.0;
    const double shm_free = clamp0((double)(h.Sh - x.shm - y.shm) / (double)h.Sh);
    const double reg_free = clamp0((double)(h.R - x.reg - y.reg) / (double)h.R);
    const double warp_free = clamp0((double)(h.W - x.warp - y.warp) / (double)h.W);
    double score = 0.0;
    score += shm_free;
    score += reg_free;
    score += warp_free;
    const double r_x = (double)x.inst / (double)x.mem;
    const double r_y = (double)y.inst / (double)y.mem;
    const double r_b = (double)h.ccap / (double)h.mcap;
    const bool opposite = (r_x <= r_b && r_b <= r_y) || (r_y <= r_b && r_b <= r_x);
    if (opposite) {
        const double r_comb = (double)(x.inst + y.inst) / (double)(x.mem + y.mem);
        const double dist = r_comb >= r_b ? r_comb - r_b : r_b - r_comb;
        score += clamp0(1.0 - dist / r_b);
    }
    return score;
}

}  // namespace

int ko_heuristic_host(const KoSet &h, int32_t *order_out, bool per_block)
{
    const int n = h.n;
    std::vector<Footprint> fp(n);
    for (int i = 0; i < n; i++) fp[i] = footprint(h, h.k[i], per_block);
    // ScoreMatrix over all pairs, computed once
    std::vector<double> score((size_t)n * n, 0.0);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            if (i != j) score[(size_t)i * n + j] = pair_score(h, fp[i], fp[j]);

    std::vector<char> left(n, 1);
    int remaining = n, written = 0, rounds = 0;
    while (remaining > 0) {
        ++rounds;
        if (remaining == 1) {
            for (int i = 0; i < n; i++)
                if (left[i]) { order_out[written++] = i; left[i] = 0; }
            break;
        }
        int a = -1, b = -1;
        double best = -1.0;
        for (int i = 0; i < n; i++) {
            if (!left[i]) continue;
            for (int j = i + 1; j < n; j++) {
                if (left[j] && score[(size_t)i * n + j] > best) {
                    best = score[(size_t)i * n + j];
                    a = i;
                    b = j;
                }
            }
        }
        std::vector<int> round;
        if (fp[b].shm > fp[a].shm) round = {b, a};
        else round = {a, b};
        left[a] = left[b] = 0;
        remaining -= 2;
        Footprint comb = combine(fp[a], fp[b]);
        for (;;) {
            int pick = -1;
            double pick_score = -1.0;
            for (int r = 0; r < n; r++) {
                if (!left[r] || !fit_together(h, comb, fp[r])) continue;
                const double s = pair_score(h, comb, fp[r]);
                if (s > pick_score) { pick_score = s; pick = r; }
            }
            if (pick < 0) break;
            if (fp[pick].shm > comb.shm) round.insert(round.begin(), pick);
            else round.push_back(pick);
            comb = combine(comb, fp[pick]);
            left[pick] = 0;
            --remaining;
        }
        for (int v : round) order_out[written++] = v;
    }
    return rounds;
}

namespace {

int64_t alone_or_loaded(const KoSet &h, int64_t c, int64_t m, int64_t sum_c, int64_t sum_m)
{
    const int64_t tc = (c * std::max(sum_c, h.ccap) + h.ccap - 1) / h.ccap;
    const int64_t tm = (m * std::max(sum_m, h.mcap) + h.mcap - 1) / h.mcap;
    return std::max(tc, tm);
}

int64_t div_up(__int128 a, __int128 b) { return (int64_t)((a + b - 1) / b); }

}  // namespace

bool ko_bounds_host(const KoSet &h, int64_t *lb, int64_t *ub)
{
    int64_t c_max = 0, m_max = 0;
    for (int i = 0; i < h.n; i++) {
        c_max = std::max<int64_t>(c_max, h.k[i].c);
        m_max = std::max<int64_t>(m_max, h.k[i].m);
    }
    int64_t longest = 0;
    __int128 area_blk = 0, area_warp = 0, area_reg = 0, area_shm = 0, serial = 0;
    bool uses_shm = false;
    for (int i = 0; i < h.n; i++) {
        const KoKern &k = h.k[i];
        const int64_t d0 = alone_or_loaded(h, k.c, k.m, k.c, k.m);
        longest = std::max(longest, d0);
        const __int128 bd = (__int128)k.b * d0;
        area_blk += bd;
        area_warp += bd * k.w;
        area_reg += bd * k.r;
        area_shm += bd * k.s;
        uses_shm = uses_shm || k.s > 0;
        serial += (__int128)k.b * alone_or_loaded(h, k.c, k.m, (int64_t)h.Bk * c_max,
                                                  (int64_t)h.Bk * m_max);
    }
    int64_t low = longest;
    low = std::max(low, div_up(area_blk, (__int128)h.S * h.Bk));
    low = std::max(low, div_up(area_warp, (__int128)h.S * h.W));
    low = std::max(low, div_up(area_reg, (__int128)h.S * h.R));
    if (uses_shm) low = std::max(low, div_up(area_shm, (__int128)h.S * h.Sh));
    *lb = h.n > 0 ? low : 0;
    // the bound itself saturates only where int64 ends; sets whose bound
    // reaches 2^62 are refused, which keeps every simulated clock far from
    // overflow
    const __int128 limit = (__int128)1 << 62;
    *ub = serial > (__int128)INT64_MAX ? INT64_MAX : (int64_t)serial;
    return serial < limit;
}
