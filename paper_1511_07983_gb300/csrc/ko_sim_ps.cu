// Processor-sharing simulator (model variant): the dispatch of Sec. 2 (FIFO
// over blocks in launch order, round-robin first fit under the four SM
// limits, head-of-line blocking) with durations that are not fixed at start.
// Every resident block progresses its remaining compute work at
// rc = Ccap / max(SumC, Ccap) and its remaining memory work at
// rm = Mcap / max(SumM, Mcap), SumC / SumM over its SM's current residents,
// and ends when both are done.  When an SM's residents change at time t (a
// release or a placement) its blocks are advanced to t at the old rates and
// re-timed at the new ones: end = t + max(Rc / rc, Rm / rm).  Groups whose
// end equals the event time leave together.  With residents that never
// change, a block lasts max(c SumC / Ccap, m SumM / Mcap) -- the duration rule
// of the main model without its rounding up.
//
// Times are doubles.  Every operation uses an explicit round-to-nearest
// intrinsic in a fixed order (no contraction into FMAs), so the result is
// bit-for-bit the one any IEEE implementation with the same order computes.
//
// One thread simulates one explicit order; per-SM state and groups live in a
// per-thread scratch slab.
#include "ko_internal.h"

namespace {

constexpr int kThreads = 128;

// Per-thread slab for S SMs and G = N_blk_SM group slots per SM.
struct PsSlab {
    int64_t *ur, *us, *uw, *ub, *sc, *sm;  // [S]
    double *rate_c, *rate_m;               // [S]
    int64_t *gcnt;                         // [S*G]
    double *grc, *grm, *gtu, *gend;        // [S*G] remaining work, last update, end
    int32_t *ng, *changed;                 // [S]
    int32_t *gk, *gfresh;                  // [S*G]
};

__host__ __device__ inline size_t ps_slab_bytes(int S, int G)
{
    const size_t b = (size_t)S * (8 * 8 + 2 * 4) + (size_t)S * G * (5 * 8 + 2 * 4);
    return (b + 255) & ~(size_t)255;
}

__device__ PsSlab ps_slab_at(void *base, size_t per_thread, int S, int G, long long slot)
{
    char *p = (char *)base + per_thread * (size_t)slot;
    PsSlab s;
    int64_t **i64[6] = {&s.ur, &s.us, &s.uw, &s.ub, &s.sc, &s.sm};
    for (int i = 0; i < 6; i++) { *i64[i] = (int64_t *)p; p += sizeof(int64_t) * S; }
    s.rate_c = (double *)p; p += sizeof(double) * S;
    s.rate_m = (double *)p; p += sizeof(double) * S;
    s.gcnt = (int64_t *)p; p += sizeof(int64_t) * S * G;
    double **dg[4] = {&s.grc, &s.grm, &s.gtu, &s.gend};
    for (int i = 0; i < 4; i++) { *dg[i] = (double *)p; p += sizeof(double) * S * G; }
    s.ng = (int32_t *)p; p += sizeof(int32_t) * S;
    s.changed = (int32_t *)p; p += sizeof(int32_t) * S;
    s.gk = (int32_t *)p; p += sizeof(int32_t) * S * G;
    s.gfresh = (int32_t *)p;
    return s;
}

__device__ __forceinline__ double ps_rate(int64_t sum, int64_t cap)
{
    return sum <= cap ? 1.0 : __ddiv_rn((double)cap, (double)sum);
}

// Makespan of one order under processor sharing, -1 if it cannot finish.
__device__ double simulate_ps(const KoSet &d, const int8_t *perm, PsSlab st)
{
    const int n = d.n, S = d.S, G = d.Bk;
    for (int s = 0; s < S; s++) {
        st.ur[s] = st.us[s] = st.uw[s] = st.ub[s] = st.sc[s] = st.sm[s] = 0;
        st.rate_c[s] = 1.0;
        st.rate_m[s] = 1.0;
        st.ng[s] = 0;
    }
    long long total_blocks = 0;
    for (int i = 0; i < n; i++) total_blocks += d.k[i].b;
    double t = 0.0, makespan = 0.0;
    int p = 0, pos = 0;
    int32_t left = n > 0 ? d.k[perm[0]].b : 0;
    long long events = 0;
    for (;;) {
        // release every group whose end is t
        for (int s = 0; s < S; s++) {
            st.changed[s] = 0;
            int g = st.ng[s];
            for (int j = 0; j < g;) {
                const int q = s * G + j;
                if (st.gend[q] == t) {
                    const KoKern &K = d.k[st.gk[q]];
                    const int64_t cnt = st.gcnt[q];
                    st.ur[s] -= cnt * K.r; st.us[s] -= cnt * K.s; st.uw[s] -= cnt * K.w; st.ub[s] -= cnt;
                    st.sc[s] -= cnt * K.c; st.sm[s] -= cnt * K.m;
                    const int last = s * G + g - 1;
                    st.gk[q] = st.gk[last]; st.gfresh[q] = st.gfresh[last]; st.gcnt[q] = st.gcnt[last];
                    st.grc[q] = st.grc[last]; st.grm[q] = st.grm[last];
                    st.gtu[q] = st.gtu[last]; st.gend[q] = st.gend[last];
                    g--;
                    st.changed[s] = 1;
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
            int g = st.ng[s], j = 0;
            while (j < g && !(st.gfresh[s * G + j] && st.gk[s * G + j] == kid)) j++;
            if (j == g) {
                const int q = s * G + g;
                st.gk[q] = kid; st.gfresh[q] = 1; st.gcnt[q] = 0;
                st.grc[q] = (double)K.c; st.grm[q] = (double)K.m; st.gtu[q] = t; st.gend[q] = 0.0;
                st.ng[s] = g + 1;
            }
            st.gcnt[s * G + j] += 1;
            st.ur[s] += K.r; st.us[s] += K.s; st.uw[s] += K.w; st.ub[s] += 1;
            st.sc[s] += K.c; st.sm[s] += K.m;
            st.changed[s] = 1;
            p = (s + 1 == S) ? 0 : s + 1;
            if (--left == 0) {
                pos++;
                left = pos < n ? d.k[perm[pos]].b : 0;
            }
        }
        // advance the changed SMs' blocks to t at the old rates, re-time them at the new
        for (int s = 0; s < S; s++) {
            if (!st.changed[s]) continue;
            const double nrc = ps_rate(st.sc[s], d.ccap), nrm = ps_rate(st.sm[s], d.mcap);
            for (int j = 0; j < st.ng[s]; j++) {
                const int q = s * G + j;
                if (!st.gfresh[q]) {
                    const double dt = __dsub_rn(t, st.gtu[q]);
                    double rc = __dsub_rn(st.grc[q], __dmul_rn(st.rate_c[s], dt));
                    double rm = __dsub_rn(st.grm[q], __dmul_rn(st.rate_m[s], dt));
                    st.grc[q] = rc < 0.0 ? 0.0 : rc;
                    st.grm[q] = rm < 0.0 ? 0.0 : rm;
                    st.gtu[q] = t;
                }
                st.gfresh[q] = 0;
                const double tc = __ddiv_rn(st.grc[q], nrc), tm = __ddiv_rn(st.grm[q], nrm);
                st.gend[q] = __dadd_rn(t, tc > tm ? tc : tm);
            }
            st.rate_c[s] = nrc;
            st.rate_m[s] = nrm;
        }
        // next event
        double tmin = -1.0;
        for (int s = 0; s < S; s++)
            for (int j = 0; j < st.ng[s]; j++) {
                const double e = st.gend[s * G + j];
                if (tmin < 0.0 || e < tmin) tmin = e;
            }
        if (tmin < 0.0) return pos < n ? -1.0 : makespan;
        if (++events > total_blocks + 2) return -1.0;  // every event releases at least one group
        t = tmin;
        makespan = t;
    }
}

__global__ void __launch_bounds__(kThreads)
ps_kernel(const KoSet *__restrict__ d_set, const int8_t *__restrict__ perms, long long count,
          double *__restrict__ out, void *scratch, size_t per_thread)
{
    __shared__ KoSet sd;
    for (int i = threadIdx.x; i < (int)(sizeof(KoSet) / 4); i += blockDim.x)
        ((int32_t *)&sd)[i] = ((const int32_t *)d_set)[i];
    __syncthreads();
    const long long slot = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const PsSlab st = ps_slab_at(scratch, per_thread, sd.S, sd.Bk, slot);
    const int n = sd.n;
    for (long long j = slot; j < count; j += stride) {
        int8_t perm[KO_MAX_KERNELS];
        uint32_t seen = 0;
        bool ok = true;
        for (int q = 0; q < n; q++) {
            const int v = perms[j * n + q];
            if (v < 0 || v >= n || ((seen >> v) & 1u)) ok = false;
            else seen |= 1u << v;
            perm[q] = (int8_t)(v < 0 || v >= n ? 0 : v);
        }
        out[j] = ok ? simulate_ps(sd, perm, st) : -1.0;
    }
}

}  // namespace

size_t ko_ps_scratch_per_thread(const KoSet &h) { return ps_slab_bytes(h.S, h.Bk); }

cudaError_t ko_launch_ps(const KoSet *d_set, const KoSet &h_set, const int8_t *perms, int64_t count, double *out,
                         void *scratch, size_t scratch_bytes, cudaStream_t stream)
{
    if (count <= 0) return cudaSuccess;
    const size_t per = ps_slab_bytes(h_set.S, h_set.Bk);
    long long blocks = (long long)(scratch_bytes / per) / kThreads;
    const long long need = (count + kThreads - 1) / kThreads;
    if (blocks > need) blocks = need;
    if (blocks < 1) return cudaErrorMemoryAllocation;
    if (blocks > 65535) blocks = 65535;
    ps_kernel<<<(unsigned)blocks, kThreads, 0, stream>>>(d_set, perms, count, out, scratch, per);
    ko_count_launch();
    return cudaGetLastError();
}
