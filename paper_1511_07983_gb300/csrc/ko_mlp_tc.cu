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
//   tc_tma_kernel          the MODE 0 layer with both operands loaded by TMA
//                          (cp.async.bulk.tensor), the default for inference.
//
//  * Operands sit in shared memory in the no-swizzle core-matrix layout: a
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
// Shared memory (at most 226 KB) keeps one CTA per SM, so the 256-column TMEM
// allocation never waits for another CTA.
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

// Inference layer (MODE 0 arithmetic) with operands loaded by TMA.  A 2-D box
// of 8 elements (16 bytes) x R rows lands one K chunk of R rows as R x 16
// contiguous bytes: a column of R / 8 core matrices, so the operand layout is
// K-chunk-major (chunk c at c * R * 16 bytes) and the MMA descriptors take
// LBO = R * 16 bytes (adjacent along K) and SBO = 128 bytes (adjacent 8-row
// groups).  One thread issues K/8 box copies per operand, counted in bytes on
// an mbarrier (expect_tx); the weights (R = 256) and the first A tile (R = 128)
// arrive together, each later A tile as soon as the previous tile's MMAs have
// retired.  Epilogue as tc_layer_kernel<0>.
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

__global__ void __launch_bounds__(kThreadsTc, 1)
tc_tma_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW, int K, int tiles,
              const float *__restrict__ bias, uint16_t *__restrict__ out, int *err)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar_mma, mbar_load;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, col0 = (warp >> 2) * (kTileN / 2);
    const int kc = K / 8;
    uint8_t *sa = smem;                              // kc chunks x 128 rows x 16 B
    uint8_t *sb = smem + (size_t)kTileM * K * 2;     // kc chunks x 256 rows x 16 B
    float *sbias = (float *)(sb + (size_t)kTileN * K * 2);
    uint32_t *stage = (uint32_t *)(sbias + kTileN) + warp * 32 * kStageRowWords;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n" ::"r"(saddr(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(saddr(&mbar_mma)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(saddr(&mbar_load)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    __syncthreads();
    if (tid == 0 && blockIdx.x < tiles) {
        expect_bytes(&mbar_load, (uint32_t)((kTileN + kTileM) * K * 2));
        for (int c = 0; c < kc; c++) {
            tma_box(saddr(sb) + (uint32_t)(c * kTileN * 16), &tmW, c * 8, 0, &mbar_load);
            tma_box(saddr(sa) + (uint32_t)(c * kTileM * 16), &tmA, c * 8, blockIdx.x * kTileM, &mbar_load);
        }
    }
    for (int i = tid; i < kTileN; i += blockDim.x) sbias[i] = bias[i];
    tc_fence_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = instr_desc(kTileM, kTileN);
    bool ok = true;
    uint32_t phase = 0;
    for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, phase ^= 1u) {
        const int m0 = tile * kTileM;
        if (!tc_wait(&mbar_load, phase, err)) { ok = false; break; }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
            for (int k = 0; k < K / 16; k++) {
                // a 16-wide K step covers chunks 2k and 2k + 1
                const uint64_t ad = smem_desc(saddr(sa) + (uint32_t)(2 * k * kTileM * 16), kTileM * 16, 128u);
                const uint64_t bd = smem_desc(saddr(sb) + (uint32_t)(2 * k * kTileN * 16), kTileN * 16, 128u);
                const uint32_t acc = k > 0 ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                saddr(&mbar_mma)));
        }
        if (!tc_wait(&mbar_mma, phase, err)) {
            ok = false;
        } else {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
            // the MMAs have read the A tile: fetch the next one under the epilogue
            const int tn = tile + (int)gridDim.x;
            if (tid == 0 && tn < tiles) {
                expect_bytes(&mbar_load, (uint32_t)(kTileM * K * 2));
                for (int c = 0; c < kc; c++)
                    tma_box(saddr(sa) + (uint32_t)(c * kTileM * 16), &tmA, c * 8, tn * kTileM, &mbar_load);
            }
            const int row0 = m0 + quarter * 32;
            for (int c0 = col0; c0 < col0 + kTileN / 2; c0 += 32) {
                uint32_t v[32];
                tc_ld32(tmem, quarter, c0, v);
                uint32_t packed[16];
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    const float x0 = fmaxf(__uint_as_float(v[2 * q]) + sbias[c0 + 2 * q], 0.0f);
                    const float x1 = fmaxf(__uint_as_float(v[2 * q + 1]) + sbias[c0 + 2 * q + 1], 0.0f);
                    packed[q] = pack_bf16(x0, x1);
                }
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
        // every warp has drained the accumulator before the next tile's MMAs overwrite it
        tc_fence_sync();
    }
    // a load still in flight (only after a failed wait) must land before the CTA exits
    if (!ok && tid == 0) tc_wait(&mbar_load, phase, err);
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tmem));
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

// rows x K BF16 matrix (row-major, K contiguous), boxes of 8 x box_rows.
bool encode_operand(CUtensorMap *map, const uint16_t *base, long long rows, int K, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || ((uintptr_t)base & 15u) || (K * 2) % 16) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {8u, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1u, 1u};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
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

}  // namespace

cudaError_t ko_mlp_layer_tc(const uint16_t *A, const uint16_t *Wt, int M, int K, const float *bias, uint16_t *out,
                            int *err, cudaStream_t st)
{
    if (M % kTileM || (K != 192 && K != 256)) return cudaErrorInvalidValue;
    CUtensorMap tma, tmw;
    const size_t smem = (size_t)(kTileM + kTileN) * K * 2 + sizeof(float) * kTileN +
                        (kThreadsTc / 32) * 32 * kStageRowWords * sizeof(uint32_t);
    if ((long long)smem > (long long)max_dyn_smem() || !encode_operand(&tma, A, M, K, kTileM) ||
        !encode_operand(&tmw, Wt, kTileN, K, kTileN))
        return launch_layer<0>(A, Wt, M, K, bias, out, nullptr, 0, nullptr, err, st);
    cudaError_t e = cudaFuncSetAttribute(tc_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = M / kTileM;
    const int grid = tiles < sms ? tiles : sms;
    tc_tma_kernel<<<grid, kThreadsTc, smem, st>>>(tma, tmw, K, tiles, bias, out, err);
    ko_count_launch();
    return cudaGetLastError();
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
