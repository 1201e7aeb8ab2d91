// Host build of the one-thread-per-order simulator's state machine
// (paper_1511_07983_gb300/csrc/ko_lane_sim.cuh is __host__ __device__ code),
// driven the way lane_kernel drives it, so that CPU tests can compare the
// device path's simulator steps with the oracle without a GPU.  Test
// infrastructure: the library never includes this file.
//
//   lane_host_orders   every order simulated from an empty GPU: start each
//                      kernel (its first burst), close that burst if blocks
//                      are still queued, step events until the queue is
//                      empty (the last burst placed by place_partial), and
//                      close the final burst at the leaf;
//   lane_host_subtree  all orders below a prefix, in lexicographic order,
//                      walked depth first with the node state saved after
//                      every placed kernel and restored for each sibling
//                      (column words and registers, as the kernel's slab).
// A simulation the state cannot hold (more runs or group slots than the
// shape has) yields -1, as the kernel hands such items on.
#include <cstdint>
#include <cstring>
#include <vector>

#define KO_HD inline
#include "ko_lane_sim.cuh"

using namespace kolane;

namespace {

struct HostKernels {
    const int64_t *k = nullptr;  // N x 6: regs, smem, warps, blocks, c, m (per block)
    KParam full(int i) const
    {
        const int64_t *r = k + 6 * i;
        return KParam{(int)r[0], (int)r[1], (int)r[2], (int)r[3], (int)r[4], (int)r[5]};
    }
    KRel rel(int i) const
    {
        const int64_t *r = k + 6 * i;
        return KRel{(uint32_t)r[0] | (1u << 19) | ((uint32_t)r[2] << 25), (uint32_t)r[1], (uint32_t)r[4],
                    (uint32_t)r[5]};
    }
};

using Sim = LaneSim<1, HostKernels, ShapeL>;

int log2_exact(int64_t v)
{
    for (int s = 0; s < 31; s++)
        if ((int64_t)1 << s == v) return s;
    return -1;
}

void setup(Sim &s, std::vector<uint32_t> &col, const int64_t *gpu7, const int64_t *kernels, int n)
{
    col.assign(ShapeL::kWords, 0u);
    s.col = col.data();
    s.kl.k = kernels;
    s.run_limit = ShapeL::kRuns;
    s.L = Limits{n, (int)gpu7[0], (int)gpu7[1], (int)gpu7[2], (int)gpu7[3], (int)gpu7[4], (uint32_t)gpu7[5],
                 (uint32_t)gpu7[6], log2_exact(gpu7[5]), log2_exact(gpu7[6])};
    s.init();
}

// Place every block of kernel k (the kernel's PH_START, PH_EVENT and PH_FINAL
// steps); false when the state cannot hold the simulation.
bool place_kernel(Sim &s, int k, int total_blocks)
{
    int left = s.start_kernel(k);
    if (s.fail) return false;
    if (left > 0) s.close_burst();
    int events = 0;
    while (left > 0) {
        const bool last = s.event(left, 0u);
        if (s.fail || ++events > total_blocks + 64) return false;
        if (last) {
            s.place_partial(left);
            if (s.fail) return false;
        }
    }
    return true;
}

int total_blocks_of(const int64_t *kernels, int n)
{
    int t = 0;
    for (int i = 0; i < n; i++) t += (int)kernels[6 * i + 3];
    return t;
}

struct Walker {
    Sim s;
    std::vector<uint32_t> col;
    int n = 0, tb = 0;
    int64_t *out = nullptr;
    int64_t pos = 0;

    void leafs_failed(int depth)
    {
        int64_t c = 1;
        for (int i = 2; i <= n - depth; i++) c *= i;
        for (int64_t i = 0; i < c; i++) out[pos++] = -1;
    }

    void walk(uint32_t used, int depth)
    {
        if (depth == n) {
            out[pos++] = s.finish();
            return;
        }
        const std::vector<uint32_t> saved(col);
        uint32_t regs[kRegWords];
        s.regs_out(regs);
        for (int k = 0; k < n; k++) {
            if ((used >> k) & 1u) continue;
            std::memcpy(col.data(), saved.data(), saved.size() * sizeof(uint32_t));
            s.regs_in(regs);
            if (!place_kernel(s, k, tb)) {
                leafs_failed(depth + 1);
                continue;
            }
            walk(used | (1u << k), depth + 1);
        }
    }
};

}  // namespace

extern "C" {

// Makespans of `count` orders (rows of n kernel ids, stride n) of one set.
// gpu7: N_SM, regs, smem, warps, blocks per SM, Ccap, Mcap.
int lane_host_orders(const int64_t *gpu7, const int64_t *kernels, int n, const int8_t *orders, int64_t count,
                     int64_t *out)
{
    if (n < 1 || n > 12) return -1;
    Sim s;
    std::vector<uint32_t> col;
    const int tb = total_blocks_of(kernels, n);
    for (int64_t r = 0; r < count; r++) {
        setup(s, col, gpu7, kernels, n);
        bool ok = true;
        for (int d = 0; d < n && ok; d++) ok = place_kernel(s, orders[r * n + d], tb);
        out[r] = ok ? s.finish() : -1;
    }
    return 0;
}

// Makespans of every order that starts with `prefix` (plen kernel ids), in
// lexicographic order of the remaining kernels: (n - plen)! values.
int lane_host_subtree(const int64_t *gpu7, const int64_t *kernels, int n, const int8_t *prefix, int plen,
                      int64_t *out)
{
    if (n < 1 || n > 12 || plen < 0 || plen > n) return -1;
    Walker w;
    setup(w.s, w.col, gpu7, kernels, n);
    w.n = n;
    w.tb = total_blocks_of(kernels, n);
    w.out = out;
    uint32_t used = 0;
    for (int d = 0; d < plen; d++) {
        if (!place_kernel(w.s, prefix[d], w.tb)) {
            w.leafs_failed(plen);
            return 0;
        }
        used |= 1u << prefix[d];
    }
    w.walk(used, plen);
    return 0;
}

}  // extern "C"
