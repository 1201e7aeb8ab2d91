// Surrogate GEMMs on the 5th-generation tensor cores (tcgen05), all of the
// form C[m][n] = sum_k A[m][k] * Bt[n][k] with BF16 operands, both K-major,
// and an FP32 accumulator in TMEM:
//
//   tc_layer_kernel<MODE>  M rows (a multiple of 128), N = 256, K in {192, 256}:
//                          Bt (256 x K) is loaded once per CTA and 128-row
//                          tiles of A stream through (persistent grid).
//       MODE 0  out   = bf16(relu(C + bias))               (inference, forward)
//       MODE 1  out   = bf16(relu(C + bias)), out_t = its transpose (training
//                       forward: out_t feeds the weight gradients)
//       MODE 2  outf  = C in FP32                           (input gradients)
//   tc_wgrad_kernel        M <= 256, N = 256, K a multiple of 256 (the batch):
//                          split-K, one 256-wide K slice per CTA, FP32 partial
//                          tiles to a workspace; wgrad_reduce_kernel sums the
//                          slices in a fixed order (deterministic).
//   tc_ws_kernel<OUT>      the MODE 0 layer, warp-specialised: TMA producer,
//                          MMA issuer and epilogue warps over a ring of
//                          128-byte-swizzled A stages and two TMEM
//                          accumulators (the default for inference); with
//                          OUT the network's output layer is fused into the
//                          last hidden layer's epilogue.
//
//  * The cp.async kernels keep operands in the no-swizzle core-matrix layout: a
//    core matrix is 8 rows x 16 bytes; core matrices adjacent along K are
//    LBO = 128 bytes apart, adjacent 8-row groups SBO = (K/8) * 128 bytes
//    apart.  Fills map 8 consecutive threads to one core matrix, so a warp
//    writes 512 contiguous bytes (no bank conflicts) and reads 64-byte runs
//    of 8 rows from global memory; rows past the operand's end are zeroed.
//  * One elected thread issues K/16 tcgen05.mma (cta_group::1, kind::f16,
//    M = 128, N = 256, K = 16) and a tcgen05.commit that arrives on an
//    mbarrier; the CTA waits on it with a bounded spin (an error flag is set
//    if it gives up, and the kernel stops).
//  * Epilogue: eight warps; warp w reads TMEM lanes 32 (w % 4) .. +31 (= rows)
//    and columns 128 (w / 4) .. +127, 32 columns at a time with
//    tcgen05.ld.32x32b.x32.  MODE 0 passes each 32 x 64-byte BF16 piece through
//    a per-warp staging area (16-byte slots XOR-rotated by row, conflict-free
//    both ways) so a store writes 8 whole 64-byte row segments.  MODE 1 stages
//    the 32 x 32 piece as one word per value with a row stride of 33 words,
//    which makes both the row-wise and the column-wise reads conflict-free,
//    and writes out and out_t (64 contiguous bytes per lane) from it.
// Shared memory (at most 226 KB) keeps one CTA per SM, so a TMEM allocation
// (256 columns; 512 in tc_ws_kernel) never waits for another CTA.
#include <cstdint>
#include <cstring>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "ko_mlp.h"

namespace {

constexpr int kTileM = 128, kTileN = 256, kSliceK = 256;
constexpr int kThreadsTc = 256;  // 8 warps
constexpr uint32_t kSpinLimit = 1u << 26;
constexpr int kStageRowWords = 16;  // MODE 0: 32 rows x 16 words per warp
constexpr int kStageTWords = 33;    // MODE 1: 32 rows x 33 words per warp

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (no swizzle): start, leading (K) and stride
// (8-row) byte offsets in 16-byte units, descriptor version 1 in bits 46-48.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Descriptor of a K-major operand in the 128-byte swizzled layout that TMA
// writes with CU_TENSOR_MAP_SWIZZLE_128B: rows of 64 BF16 (128 bytes), 8-row
// atoms of 1024 bytes (SBO), layout type 2 in bits 61-63.  A K = 16 step inside
// the atom starts 32 bytes further (the hardware applies the swizzle to the
// computed addresses).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(1024u >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void cp_async16_tc(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr(dst)), "l"(src));
}

// rows x K operand (row stride ld elements) into the core-matrix layout; rows
// at or past `valid` are zero.  Chunk i: core matrix (i / 8 / kc, i / 8 % kc),
// row i % 8.
__device__ __forceinline__ void tc_fill(uint8_t *dst, const uint16_t *src, int rows, int valid, long long ld,
                                        int K)
{
    const int kc = K / 8;
    const uint32_t sbo = (uint32_t)kc * 128u;
    for (int i = threadIdx.x; i < rows * kc; i += blockDim.x) {
        const int rlo = i & 7, rest = i >> 3, c = rest % kc, rhi = rest / kc;
        const int r = rhi * 8 + rlo;
        uint8_t *d = dst + rhi * sbo + c * 128 + rlo * 16;
        if (r < valid) cp_async16_tc(d, src + (size_t)r * ld + c * 8);
        else *(uint4 *)d = make_uint4(0u, 0u, 0u, 0u);
    }
}

// K/16 MMAs of the 128 x K tile in `sa` against the 256 x K operand in `sb`,
// then a commit to `mbar` (called by one thread).
__device__ __forceinline__ void tc_mma(uint32_t tmem, const uint8_t *sa, const uint8_t *sb, int K, uint64_t *mbar)
{
    const uint32_t sbo = (uint32_t)(K / 8) * 128u;
    const uint32_t idesc = instr_desc(kTileM, kTileN);
    for (int k = 0; k < K / 16; k++) {
        // a 16-wide K step covers two core matrices along K
        const uint64_t ad = smem_desc(saddr(sa) + (uint32_t)k * 256u, 128u, sbo);
        const uint64_t bd = smem_desc(saddr(sb) + (uint32_t)k * 256u, 128u, sbo);
        const uint32_t acc = k > 0 ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(saddr(mbar)));
}

// Bounded wait for phase `phase` of `mbar`; false (and *err = 1) if it gave up.
__device__ __forceinline__ bool tc_wait(uint64_t *mbar, uint32_t phase, int *err)
{
    uint32_t done = 0;
    for (uint32_t spin = 0; spin < kSpinLimit && !done; spin++) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(saddr(mbar)), "r"(phase));
    }
    if (!done && (threadIdx.x & 31) == 0) atomicExch(err, 1);
    return done != 0;
}

// 32 accumulator columns c0.. of TMEM lanes 32q.. into v (this warp's rows).
__device__ __forceinline__ void tc_ld32(uint32_t tmem, int q, int c0, uint32_t (&v)[32])
{
    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
          "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
          "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    // round to nearest even (cvt.rn.bf16x2): lo in the low half, hi in the high half
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    uint32_t u;
    std::memcpy(&u, &h, sizeof(u));
    return u;
}

__device__ __forceinline__ void tc_fence_sync()
{
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
}

// Persistent: one CTA per SM loads Bt once, then walks row tiles (tile,
// tile + gridDim.x, ...).  Operand copies use cp.async, made visible to the
// tensor core's async proxy before each MMA batch; the mbarrier phase
// alternates per tile.  The next tile's A operand is requested as soon as the
// current MMAs complete, so its load overlaps the epilogue.
template <int MODE>
__global__ void __launch_bounds__(kThreadsTc, 1)
tc_layer_kernel(const uint16_t *__restrict__ A, const uint16_t *__restrict__ Wt, int K, int tiles,
                const float *__restrict__ bias, uint16_t *__restrict__ out, uint16_t *__restrict__ out_t,
                long long ldt, float *__restrict__ outf, int *err)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, col0 = (warp >> 2) * (kTileN / 2);
    uint8_t *sa = smem;                              // 128 x K
    uint8_t *sb = smem + (size_t)kTileM * K * 2;     // 256 x K
    float *sbias = (float *)(sb + (size_t)kTileN * K * 2);  // 256
    uint32_t *stage = (uint32_t *)(sbias + kTileN) + warp * 32 * (MODE == 1 ? kStageTWords : kStageRowWords);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n" ::"r"(saddr(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(saddr(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    tc_fill(sb, Wt, kTileN, kTileN, K, K);
    asm volatile("cp.async.commit_group;\n" ::);
    if (MODE != 2)
        for (int i = tid; i < kTileN; i += blockDim.x) sbias[i] = bias[i];
    tc_fence_sync();
    const uint32_t tmem = tmem_base;
    auto load_a = [&](int tile) {
        tc_fill(sa, A + (size_t)tile * kTileM * K, kTileM, kTileM, K, K);
        asm volatile("cp.async.commit_group;\n" ::);
    };
    bool ok = true;
    uint32_t phase = 0;
    if (blockIdx.x < tiles) load_a(blockIdx.x);
    for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, phase ^= 1u) {
        const int m0 = tile * kTileM;
        // operands of this tile have landed: make them visible to the tensor core
        asm volatile("cp.async.wait_all;\n" ::);
        asm volatile("fence.proxy.async.shared::cta;\n" ::);
        tc_fence_sync();
        if (tid == 0) tc_mma(tmem, sa, sb, K, &mbar);
        if (!tc_wait(&mbar, phase, err)) {
            ok = false;
        } else {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
            // the MMAs have read the A tile: start loading the next one under the epilogue
            if (tile + (int)gridDim.x < tiles) load_a(tile + gridDim.x);
            const int row0 = m0 + quarter * 32;
            for (int c0 = col0; c0 < col0 + kTileN / 2; c0 += 32) {
                uint32_t v[32];
                tc_ld32(tmem, quarter, c0, v);
                if constexpr (MODE == 2) {
                    float4 *dst = (float4 *)(outf + (size_t)(row0 + lane) * kTileN + c0);
#pragma unroll
                    for (int q = 0; q < 8; q++)
                        dst[q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                             __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
                    continue;
                } else {
                uint32_t packed[16];
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const float x0 = fmaxf(__uint_as_float(v[2 * j]) + sbias[c0 + 2 * j], 0.0f);
                    const float x1 = fmaxf(__uint_as_float(v[2 * j + 1]) + sbias[c0 + 2 * j + 1], 0.0f);
                    packed[j] = pack_bf16(x0, x1);
                }
                if (MODE == 0) {
                    // row `lane`'s 64 bytes: 16-byte slot q goes to position (q + lane / 2) % 4
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        *(uint4 *)(stage + lane * 16 + ((q + (lane >> 1)) & 3) * 4) =
                            make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
                    __syncwarp();
                    // 8 rows per store: lanes 4r..4r+3 write row r's 64 contiguous bytes
#pragma unroll
                    for (int it = 0; it < 4; it++) {
                        const int r = it * 8 + (lane >> 2), q = lane & 3;
                        const uint4 w = *(const uint4 *)(stage + r * 16 + ((q + (r >> 1)) & 3) * 4);
                        *(uint4 *)(out + (size_t)(row0 + r) * kTileN + c0 + q * 8) = w;
                    }
                    __syncwarp();
                } else {
                    // one value per word, row stride 33 words: row r, column c at r * 33 + c
#pragma unroll
                    for (int j = 0; j < 16; j++) {
                        stage[lane * kStageTWords + 2 * j] = packed[j] & 0xFFFFu;
                        stage[lane * kStageTWords + 2 * j + 1] = packed[j] >> 16;
                    }
                    __syncwarp();
                    // rows: lanes 4r'..4r'+3 write 16 bytes each of row r' (8 rows per pass)
#pragma unroll
                    for (int it = 0; it < 4; it++) {
                        const int r = it * 8 + (lane >> 2), q = lane & 3;
                        const uint32_t *src = stage + r * kStageTWords + q * 8;
                        const uint4 w = make_uint4(src[0] | (src[1] << 16), src[2] | (src[3] << 16),
                                                   src[4] | (src[5] << 16), src[6] | (src[7] << 16));
                        *(uint4 *)(out + (size_t)(row0 + r) * kTileN + c0 + q * 8) = w;
                    }
                    // transpose: lane c writes column c0 + c's 32 rows (64 contiguous bytes of out_t)
                    uint32_t col[16];
#pragma unroll
                    for (int j = 0; j < 16; j++)
                        col[j] = stage[(2 * j) * kStageTWords + lane] |
                                 (stage[(2 * j + 1) * kStageTWords + lane] << 16);
                    uint4 *dt = (uint4 *)(out_t + (size_t)(c0 + lane) * ldt + row0);
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        dt[q] = make_uint4(col[4 * q], col[4 * q + 1], col[4 * q + 2], col[4 * q + 3]);
                    __syncwarp();
                }
                }
            }
        }
        // every warp has drained the accumulator before the next tile's MMAs overwrite it
        tc_fence_sync();
    }
    asm volatile("cp.async.wait_all;\n" ::);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tmem));
}

// One 2-D TMA box copy into shared memory, completion counted in bytes on mbar.
__device__ __forceinline__ void tma_box(uint32_t dst, const CUtensorMap *map, int x, int y, uint64_t *mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(saddr(mbar))
        : "memory");
}

__device__ __forceinline__ void expect_bytes(uint64_t *mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(saddr(mbar)), "r"(bytes) : "memory");
}

// Warp-specialised inference layer (MODE 0 arithmetic): the A operand streams
// through a ring of stages, each a 128-row x 64-element K chunk (16 KB, one
// TMA box in the 128-byte swizzled layout; the weights are K/64 such boxes of
// 256 rows), and the accumulator is
// double-buffered in TMEM (two 256-column accumulators), so that loads, MMAs
// and epilogues of consecutive tiles overlap:
//   warp E (one thread)  TMA producer: weights once, then every A chunk as soon
//                        as its stage is empty;
//   warp E+1 (one thread) MMA issuer: per chunk four K = 16 MMAs into the
//                        tile's accumulator, a commit that empties the stage,
//                        and after a tile's last chunk a commit that marks the
//                        accumulator full;
//   warps 0..E-1         epilogue (as tc_layer_kernel<0>; E = kEpiWarps, warp
//                        w reads TMEM lanes 32 (w % 4).. and kEpiCols columns),
//                        then one arrival per warp that frees the accumulator.
// mbarriers: full/empty per stage, full/free per accumulator, one for the
// weights.  Chunk n of this CTA's stream uses stage n % stages for the
// (n / stages)-th time; tile i uses accumulator i % 2 for the (i / 2)-th time;
// a wait for the u-th completion of a barrier tests phase parity u & 1.  Every
// wait is bounded and checks a shared abort flag, so a failed wait stops all
// roles (error flag set) instead of leaving them spinning.
constexpr int kChunkK = 64;                               // K elements per stage
constexpr uint32_t kStageBytes = kTileM * kChunkK * 2;    // 16 KB
constexpr int kMaxStages = 8;
#ifndef KO_TC_EPI_WARPS
#define KO_TC_EPI_WARPS 16
#endif
constexpr int kEpiWarps = KO_TC_EPI_WARPS;                // 4 per TMEM lane quarter at 16
constexpr int kEpiCols = kTileN / (kEpiWarps / 4);        // accumulator columns per epilogue warp
constexpr int kWsThreads = (kEpiWarps + 2) * 32;          // epilogue warps + producer + MMA warps
static_assert(kEpiWarps % 4 == 0 && kEpiCols % 32 == 0, "epilogue warps cover the lane quarters evenly");

// Bounded wait for the completion of parity `phase` of `mbar`; gives up (sets
// *abort and *err) after kSpinLimit polls or when another role has aborted.
__device__ __forceinline__ bool ws_wait(uint64_t *mbar, uint32_t phase, volatile int *abort, int *err)
{
    uint32_t done = 0;
    for (uint32_t spin = 0; spin < kSpinLimit && !done; spin++) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(saddr(mbar)), "r"(phase));
        if (!done && (spin & 255u) == 255u && *abort) break;
    }
    if (!done) {
        *abort = 1;
        atomicExch(err, 1);
    }
    return done != 0;
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(mbar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(saddr(mbar)) : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
        saddr(mbar)));
}

// Barrier 1 across the epilogue warps, counting the threads whose `flag` is set.
__device__ __forceinline__ int epi_barrier_count(bool flag)
{
    int n;
    asm volatile("{\n.reg .pred p;\nsetp.ne.u32 p, %1, 0;\nbar.red.popc.u32 %0, 1, %2, p;\n}\n"
                 : "=r"(n)
                 : "r"((uint32_t)flag), "n"(kEpiWarps * 32)
                 : "memory");
    return n;
}

// OUT = false: out = bf16(relu(A Wt^T + bias)).  OUT = true (the network's
// last hidden layer): the same BF16 activations are not stored but dotted
// with w4 on the fly, y = a . w4 + b4, in a fixed order that
// ko_mlp_out_fwd repeats: per row, eight 32-column partial sums, each a chain
// of fused multiply-adds in column order, combined as
// ((p0 + p1) + (p2 + p3)) + ((p4 + p5) + (p6 + p7)), then + b4.  Warp
// (quarter, g) holds columns 64 g .. 64 g + 63 of 32 rows, i.e. p(2g) + p(2g+1);
// the four such sums of a row meet in shared memory behind a named barrier
// whose count also tells every epilogue warp whether all of them got the tile.
template <bool OUT>
__global__ void __launch_bounds__(kWsThreads, 1)
tc_ws_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW, int K, int tiles,
             int stages, const float *__restrict__ bias, uint16_t *__restrict__ out,
             const uint16_t *__restrict__ w4, const float *__restrict__ b4, float *__restrict__ y, int *err)
{
    static_assert(!OUT || kEpiCols == 64, "the fused output sums assume 64 columns per epilogue warp");
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t bar_full[kMaxStages], bar_empty[kMaxStages];
    __shared__ __align__(8) uint64_t bar_acc[2], bar_free[2], bar_w, bar_drain;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kchunks = K / kChunkK;
    uint8_t *sw = smem;                                   // K/8 chunks x 256 rows x 16 B
    uint8_t *ring = smem + (size_t)kTileN * K * 2;        // stages x (8 chunks x 128 rows x 16 B)
    float *sbias = (float *)(ring + (size_t)stages * kStageBytes);
    const int ntiles = (int)blockIdx.x < tiles ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    // swizzled TMA destinations and the MMA atoms need 1024-byte aligned stages
    if (saddr(smem) & 1023u) {
        if (tid == 0) atomicExch(err, 1);
        return;
    }

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(saddr(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        for (int s = 0; s < stages; s++) {
            mbar_init(&bar_full[s], 1);
            mbar_init(&bar_empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&bar_acc[b], 1);
            mbar_init(&bar_free[b], kEpiWarps);
        }
        mbar_init(&bar_w, 1);
        mbar_init(&bar_drain, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    for (int i = tid; i < kTileN; i += blockDim.x) sbias[i] = bias[i];
    float *sw4 = sbias + kTileN;    // OUT: w4 as floats, then 2 x 4 x 128 partial sums
    if (OUT)
        for (int i = tid; i < kTileN; i += blockDim.x) sw4[i] = __uint_as_float((uint32_t)w4[i] << 16);
    tc_fence_sync();
    const uint32_t tmem = tmem_base;

    if (warp == kEpiWarps) {
        // TMA producer
        if (lane == 0 && ntiles > 0) {
            expect_bytes(&bar_w, (uint32_t)(kTileN * K * 2));
            for (int c = 0; c < kchunks; c++)
                tma_box(saddr(sw) + (uint32_t)(c * kTileN * kChunkK * 2), &tmW, c * kChunkK, 0, &bar_w);
            int n = 0;
            bool ok = true;
            for (int i = 0; i < ntiles && ok; i++) {
                const int row = ((int)blockIdx.x + i * (int)gridDim.x) * kTileM;
                for (int k = 0; k < kchunks; k++, n++) {
                    const int s = n % stages;
                    const uint32_t u = (uint32_t)(n / stages);
                    if (u > 0 && !ws_wait(&bar_empty[s], (u - 1u) & 1u, &abort_flag, err)) {
                        ok = false;
                        break;
                    }
                    const uint32_t dst = saddr(ring) + (uint32_t)s * kStageBytes;
                    expect_bytes(&bar_full[s], kStageBytes);
                    tma_box(dst, &tmA, k * kChunkK, row, &bar_full[s]);
                }
            }
            if (!ok) {
                // copies still in flight land before the CTA exits: the last load of each stage
                int zero = 0;
                for (int s = 0; s < stages && s < n; s++) {
                    const int last = n - 1 - ((n - 1 - s) % stages);
                    ws_wait(&bar_full[s], (uint32_t)(last / stages) & 1u, &zero, err);
                }
                int wz = 0;
                ws_wait(&bar_w, 0u, &wz, err);
            }
        }
    } else if (warp == kEpiWarps + 1) {
        // MMA issuer
        if (lane == 0 && ntiles > 0) {
            const uint32_t idesc = instr_desc(kTileM, kTileN);
            bool ok = ws_wait(&bar_w, 0u, &abort_flag, err);
            int n = 0;
            for (int i = 0; i < ntiles && ok; i++) {
                const int b = i & 1;
                if (i >= 2 && !ws_wait(&bar_free[b], (uint32_t)((i >> 1) - 1) & 1u, &abort_flag, err)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
                const uint32_t acc_t = tmem + (uint32_t)(b * kTileN);
                for (int k = 0; k < kchunks; k++, n++) {
                    const int s = n % stages;
                    if (!ws_wait(&bar_full[s], (uint32_t)(n / stages) & 1u, &abort_flag, err)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
                    const uint32_t a0 = saddr(ring) + (uint32_t)s * kStageBytes;
                    for (int j = 0; j < kChunkK / 16; j++) {
                        // a 16-wide K step covers two 8-element chunks
                        const int kk = k * (kChunkK / 16) + j;
                        const uint64_t ad = smem_desc_sw128(a0 + (uint32_t)(j * 32));
                        const uint64_t bd = smem_desc_sw128(saddr(sw) + (uint32_t)(k * kTileN * kChunkK * 2 + j * 32));
                        const uint32_t accum = kk > 0 ? 1u : 0u;
                        asm volatile(
                            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_t),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                    }
                    mma_commit(&bar_empty[s]);   // the stage is free once these MMAs have read it
                }
                if (ok) mma_commit(&bar_acc[b]);  // the tile's accumulator is complete
            }
            if (!ok) {
                // MMAs in flight retire before the accumulators are freed
                mma_commit(&bar_drain);
                int zero = 0;
                ws_wait(&bar_drain, 0u, &zero, err);
            }
        }
    } else {
        // epilogue: warps w, w + 4, ... share TMEM lanes 32 (w % 4).., kEpiCols columns each
        const int quarter = warp & 3, col0 = (warp >> 2) * kEpiCols;
        uint32_t *stage = (uint32_t *)(sbias + kTileN) + warp * 32 * kStageRowWords;
        float *s_part = sw4 + kTileN;
        const float b4v = OUT ? b4[0] : 0.0f;
        for (int i = 0; i < ntiles; i++) {
            const int b = i & 1;
            const bool got = ws_wait(&bar_acc[b], (uint32_t)(i >> 1) & 1u, &abort_flag, err);
            const bool all = __all_sync(0xffffffffu, got);
            if (!OUT && !all) break;
            const int row0 = ((int)blockIdx.x + i * (int)gridDim.x) * kTileM + quarter * 32;
            const uint32_t acc_t = tmem + (uint32_t)(b * kTileN);
            float part = 0.0f;
            if (all) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
                for (int c0 = col0; c0 < col0 + kEpiCols; c0 += 32) {
                    uint32_t v[32];
                    tc_ld32(acc_t, quarter, c0, v);
                    uint32_t packed[16];
#pragma unroll
                    for (int q = 0; q < 16; q++) {
                        const float x0 = fmaxf(__uint_as_float(v[2 * q]) + sbias[c0 + 2 * q], 0.0f);
                        const float x1 = fmaxf(__uint_as_float(v[2 * q + 1]) + sbias[c0 + 2 * q + 1], 0.0f);
                        packed[q] = pack_bf16(x0, x1);
                    }
                    if constexpr (OUT) {
                        // this row's 32-column partial: fused multiply-adds in column order
                        float sum = 0.0f;
#pragma unroll
                        for (int q = 0; q < 16; q++) {
                            sum = __fmaf_rn(__uint_as_float(packed[q] << 16), sw4[c0 + 2 * q], sum);
                            sum = __fmaf_rn(__uint_as_float(packed[q] & 0xFFFF0000u), sw4[c0 + 2 * q + 1], sum);
                        }
                        part = c0 == col0 ? sum : part + sum;
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; q++)
                            *(uint4 *)(stage + lane * 16 + ((q + (lane >> 1)) & 3) * 4) =
                                make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
                        __syncwarp();
#pragma unroll
                        for (int it = 0; it < 4; it++) {
                            const int r = it * 8 + (lane >> 2), q = lane & 3;
                            const uint4 w = *(const uint4 *)(stage + r * 16 + ((q + (r >> 1)) & 3) * 4);
                            *(uint4 *)(out + (size_t)(row0 + r) * kTileN + c0 + q * 8) = w;
                        }
                        __syncwarp();
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar_free[b]);
            }
            if constexpr (OUT) {
                float *sp = s_part + b * 4 * kTileM + quarter * 32 + lane;
                if (all) sp[(warp >> 2) * kTileM] = part;
                // every epilogue warp arrives; the count says whether all of them got the tile
                if (epi_barrier_count(all) != kEpiWarps * 32) break;
                if ((warp >> 2) == 0) y[row0 + lane] = ((sp[0] + sp[kTileM]) + (sp[2 * kTileM] + sp[3 * kTileM])) + b4v;
            }
        }
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
}

// cuTensorMapEncodeTiled from the driver, looked up once.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
    }
    return fn;
}

// rows x K BF16 matrix (row-major, K contiguous), boxes of 64 x box_rows in
// the 128-byte swizzled layout (K a multiple of 64).
bool encode_operand_sw128(CUtensorMap *map, const uint16_t *base, long long rows, int K, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || ((uintptr_t)base & 15u) || K % 64) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1u, 1u};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Weight gradient slice: CTA (mt, s) multiplies rows 128 mt.. of A (M x Kdim,
// row stride lda) by all 256 rows of Bt (256 x Kdim, row stride ldb) over the
// K slice 256 s .. 256 s + 255 and writes the FP32 128 x 256 partial tile to
// part[s][128 mt ..][0 .. 256).
__global__ void __launch_bounds__(kThreadsTc, 1)
tc_wgrad_kernel(const uint16_t *__restrict__ A, long long lda, const uint16_t *__restrict__ Bt, long long ldb,
                int M, float *__restrict__ part, int mpad, int *err)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, col0 = (warp >> 2) * (kTileN / 2);
    const int mt = blockIdx.x, s = blockIdx.y;
    const int m0 = mt * kTileM;
    const long long k0 = (long long)s * kSliceK;
    uint8_t *sa = smem;                                 // 128 x 256
    uint8_t *sb = smem + (size_t)kTileM * kSliceK * 2;  // 256 x 256
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n" ::"r"(saddr(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(saddr(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    tc_fill(sa, A + (size_t)m0 * lda + k0, kTileM, M - m0, lda, kSliceK);
    tc_fill(sb, Bt + k0, kTileN, kTileN, ldb, kSliceK);
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_all;\n" ::);
    asm volatile("fence.proxy.async.shared::cta;\n" ::);
    tc_fence_sync();
    const uint32_t tmem = tmem_base;
    if (tid == 0) tc_mma(tmem, sa, sb, kSliceK, &mbar);
    if (tc_wait(&mbar, 0, err)) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        float *dst_row = part + ((size_t)s * mpad + m0 + quarter * 32 + lane) * kTileN;
        for (int c0 = col0; c0 < col0 + kTileN / 2; c0 += 32) {
            uint32_t v[32];
            tc_ld32(tmem, quarter, c0, v);
            float4 *dst = (float4 *)(dst_row + c0);
#pragma unroll
            for (int q = 0; q < 8; q++)
                dst[q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                     __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
        }
    }
    tc_fence_sync();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tmem));
}

// out[m][n] = sum over slices s = 0, 1, ... of part[s][m][n], m < M (fixed order).
__global__ void wgrad_reduce_kernel(const float *__restrict__ part, int slices, int mpad, int M,
                                    float *__restrict__ out, int ldo)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)M * kTileN) return;
    const int m = (int)(i / kTileN), n = (int)(i % kTileN);
    float acc = 0.0f;
    for (int s = 0; s < slices; s++) acc += part[((size_t)s * mpad + m) * kTileN + n];
    out[(size_t)m * ldo + n] = acc;
}

int max_dyn_smem()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

template <int MODE>
cudaError_t launch_layer(const uint16_t *A, const uint16_t *Wt, int M, int K, const float *bias, uint16_t *out,
                         uint16_t *out_t, long long ldt, float *outf, int *err, cudaStream_t st)
{
    if (M % kTileM || (K != 192 && K != 256)) return cudaErrorInvalidValue;
    const int stage_words = MODE == 1 ? kStageTWords : kStageRowWords;
    const size_t smem = (size_t)(kTileM + kTileN) * K * 2 + sizeof(float) * kTileN +
                        (kThreadsTc / 32) * 32 * stage_words * sizeof(uint32_t);
    if ((long long)smem > (long long)max_dyn_smem()) return cudaErrorInvalidValue;
    cudaError_t e =
        cudaFuncSetAttribute(tc_layer_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = M / kTileM;
    const int grid = tiles < sms ? tiles : sms;
    tc_layer_kernel<MODE><<<grid, kThreadsTc, smem, st>>>(A, Wt, K, tiles, bias, out, out_t, ldt, outf, err);
    ko_count_launch();
    return cudaGetLastError();
}

// Launch tc_ws_kernel<OUT> with as many 16 KB A stages as fit beside the
// weights (1 KB kept for the static barriers); cudaErrorNotSupported when
// fewer than two fit or no tensor-map encoder is available (the caller then
// takes the cp.async path).
template <bool OUT>
cudaError_t launch_ws(const uint16_t *A, const uint16_t *Wt, int M, int K, const float *bias, uint16_t *out,
                      const uint16_t *w4, const float *b4, float *y, int *err, cudaStream_t st)
{
    CUtensorMap tma, tmw;
    const size_t tail = OUT ? sizeof(float) * (kTileN + 2 * 4 * kTileM)
                            : (size_t)kEpiWarps * 32 * kStageRowWords * sizeof(uint32_t);
    const size_t fixed = (size_t)kTileN * K * 2 + sizeof(float) * kTileN + tail;
    const long long room = (long long)max_dyn_smem() - 1024 - (long long)fixed;
    int stages = room > 0 ? (int)(room / kStageBytes) : 0;
    stages = stages < kMaxStages ? stages : kMaxStages;
    if (stages < 2 || !encode_operand_sw128(&tma, A, M, K, kTileM) ||
        !encode_operand_sw128(&tmw, Wt, kTileN, K, kTileN))
        return cudaErrorNotSupported;
    const size_t smem = fixed + (size_t)stages * kStageBytes;
    cudaError_t e = cudaFuncSetAttribute(tc_ws_kernel<OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = M / kTileM;
    const int grid = tiles < sms ? tiles : sms;
    tc_ws_kernel<OUT><<<grid, kWsThreads, smem, st>>>(tma, tmw, K, tiles, stages, bias, out, w4, b4, y, err);
    ko_count_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t ko_mlp_layer_tc(const uint16_t *A, const uint16_t *Wt, int M, int K, const float *bias, uint16_t *out,
                            int *err, cudaStream_t st)
{
    if (M % kTileM || (K != 192 && K != 256)) return cudaErrorInvalidValue;
    const cudaError_t e = launch_ws<false>(A, Wt, M, K, bias, out, nullptr, nullptr, nullptr, err, st);
    if (e != cudaErrorNotSupported) return e;
    return launch_layer<0>(A, Wt, M, K, bias, out, nullptr, 0, nullptr, err, st);
}

cudaError_t ko_mlp_layer_tc_out(const uint16_t *A, const uint16_t *Wt, int M, int K, const float *bias,
                                const uint16_t *w4, const float *b4, uint16_t *out, float *y, int *err,
                                cudaStream_t st)
{
    if (M % kTileM || (K != 192 && K != 256)) return cudaErrorInvalidValue;
    const cudaError_t e = launch_ws<true>(A, Wt, M, K, bias, nullptr, w4, b4, y, err, st);
    if (e != cudaErrorNotSupported) return e;
    const cudaError_t e2 = launch_layer<0>(A, Wt, M, K, bias, out, nullptr, 0, nullptr, err, st);
    if (e2 != cudaSuccess) return e2;
    return ko_mlp_out_fwd(out, w4, b4, M, y, st);
}

cudaError_t ko_mlp_layer_tc_t(const uint16_t *A, const uint16_t *Wt, int M, int K, const float *bias, uint16_t *out,
                              uint16_t *out_t, long long ldt, int *err, cudaStream_t st)
{
    if (ldt % 8) return cudaErrorInvalidValue;  // 16-byte stores into out_t rows
    return launch_layer<1>(A, Wt, M, K, bias, out, out_t, ldt, nullptr, err, st);
}

cudaError_t ko_mlp_layer_tc_f32(const uint16_t *A, const uint16_t *Wt, int M, int K, float *outf, int *err,
                                cudaStream_t st)
{
    return launch_layer<2>(A, Wt, M, K, nullptr, nullptr, nullptr, 0, outf, err, st);
}

size_t ko_mlp_wgrad_tc_workspace(int M, long long Kdim)
{
    const int mpad = (M + kTileM - 1) / kTileM * kTileM;
    return sizeof(float) * (size_t)(Kdim / kSliceK) * mpad * kTileN;
}

cudaError_t ko_mlp_wgrad_tc(const uint16_t *A, long long lda, const uint16_t *Bt, long long ldb, int M,
                            long long Kdim, float *out, int ldo, float *work, int *err, cudaStream_t st)
{
    if (M < 1 || M > 2 * kTileM || Kdim < kSliceK || Kdim % kSliceK || lda % 8 || ldb % 8)
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)(kTileM + kTileN) * kSliceK * 2;
    if ((long long)smem > (long long)max_dyn_smem()) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tc_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int mt = (M + kTileM - 1) / kTileM, slices = (int)(Kdim / kSliceK);
    const int mpad = mt * kTileM;
    tc_wgrad_kernel<<<dim3(mt, slices), kThreadsTc, smem, st>>>(A, lda, Bt, ldb, M, work, mpad, err);
    ko_count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long long n = (long long)M * kTileN;
    wgrad_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(work, slices, mpad, M, out, ldo);
    ko_count_launch();
    return cudaGetLastError();
}
