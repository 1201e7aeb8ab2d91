// Surrogate forward layer on the 5th-generation tensor cores (tcgen05):
// out[m][n] = bf16(relu(sum_k A[m][k] * Wt[n][k] + bias[n])) for a 128-row tile
// per CTA and all 256 outputs, K in {192, 256}.
//
//  * Operands: A tile (128 x K) and Wt (256 x K), BF16, K-major, stored in
//    shared memory in the no-swizzle core-matrix layout: a core matrix is
//    8 rows x 16 bytes; core matrices adjacent along K are LBO = 128 bytes
//    apart, adjacent 8-row groups SBO = (K/8) * 128 bytes apart.
//  * One elected thread issues K/16 tcgen05.mma (cta_group::1, kind::f16,
//    M = 128, N = 256, K = 16, FP32 accumulator in 256 TMEM columns) and a
//    tcgen05.commit that arrives on an mbarrier; the CTA waits on it with a
//    bounded spin (an error flag is set if it gives up).
//  * Epilogue: eight warps; warp w reads TMEM lanes 32 (w % 4) .. +31 (= rows)
//    and columns 128 (w / 4) .. +127, 32 columns at a time with
//    tcgen05.ld.32x32b.x32, adds the bias (staged in shared memory),
//    applies ReLU, rounds to BF16 and passes the 32 x 64-byte piece through a
//    per-warp staging area (16-byte slots XOR-rotated by row so that both the
//    row-wise writes and the segment-wise reads are free of bank conflicts);
//    each store instruction then writes 8 whole 64-byte row segments.
//  * Operand fills: thread i copies 16 bytes so that 8 consecutive threads
//    fill one 128-byte core matrix and a warp fills 512 contiguous bytes of
//    shared memory (no bank conflicts); its global reads are 64-byte runs of
//    8 rows.
// Shared memory (209 KB at K = 256) keeps one CTA per SM, so the 256-column
// TMEM allocation never waits for another CTA.  The grid is persistent (one
// CTA per SM): weights are loaded once per CTA, row tiles stream through.
#include <cstdint>
#include <cstring>

#include <cuda_bf16.h>

#include "ko_mlp.h"

namespace {

constexpr int kTileM = 128, kTileN = 256;
constexpr int kThreadsTc = 256;  // 8 warps: warp w drains TMEM lanes 32 (w % 4).. and columns 128 (w / 4)..
constexpr uint32_t kSpinLimit = 1u << 26;

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

// Persistent: one CTA per SM loads the weights once, then walks row tiles
// (tile, tile + gridDim.x, ...).  Operand copies use cp.async, made visible
// to the tensor core's async proxy before each MMA batch; the mbarrier phase
// alternates per tile.  The next tile's A operand is requested as soon as the
// current MMAs complete, so its load overlaps the epilogue.
__global__ void __launch_bounds__(kThreadsTc, 1)
tc_layer_kernel(const uint16_t *__restrict__ A, const uint16_t *__restrict__ Wt, int K, int tiles,
                const float *__restrict__ bias, uint16_t *__restrict__ out, int *err)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, col0 = (warp >> 2) * (kTileN / 2);
    const uint32_t sbo = (uint32_t)(K / 8) * 128u;
    const int kc = K / 8;
    uint8_t *sa = smem;                              // 128 x K
    uint8_t *sb = smem + (size_t)kTileM * K * 2;     // 256 x K
    float *sbias = (float *)(sb + (size_t)kTileN * K * 2);           // 256
    uint32_t *stage = (uint32_t *)(sbias + kTileN) + warp * 32 * 16;  // this warp: 32 rows x 16 words
    // 16-byte chunk i of a rows x K operand: core matrix (r / 8, c), row r % 8
    auto fill = [&](uint8_t *dst, const uint16_t *src, int rows) {
        for (int i = tid; i < rows * kc; i += blockDim.x) {
            const int rlo = i & 7, rest = i >> 3, c = rest % kc, rhi = rest / kc;
            cp_async16_tc(dst + rhi * sbo + c * 128 + rlo * 16, src + (size_t)(rhi * 8 + rlo) * K + c * 8);
        }
    };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n" ::"r"(saddr(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(saddr(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    // weights and bias once
    fill(sb, Wt, kTileN);
    asm volatile("cp.async.commit_group;\n" ::);
    for (int i = tid; i < kTileN; i += blockDim.x) sbias[i] = bias[i];
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = instr_desc(kTileM, kTileN);
    // A tile (row tile `tile`) into shared memory with cp.async
    auto load_a = [&](int tile) {
        fill(sa, A + (size_t)tile * kTileM * K, kTileM);
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
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        if (tid == 0) {
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
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                saddr(&mbar)));
        }
        uint32_t done = 0;
        for (uint32_t spin = 0; spin < kSpinLimit && !done; spin++) {
            asm volatile(
                "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(saddr(&mbar)), "r"(phase));
        }
        if (!done) {
            if (lane == 0) atomicExch(err, 1);
            ok = false;
        } else {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
            // the MMAs have read the A tile: start loading the next one under the epilogue
            if (tile + (int)gridDim.x < tiles) load_a(tile + gridDim.x);
            for (int c0 = col0; c0 < col0 + kTileN / 2; c0 += 32) {
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                      "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                      "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
                uint32_t packed[16];
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const float x0 = fmaxf(__uint_as_float(v[2 * j]) + sbias[c0 + 2 * j], 0.0f);
                    const float x1 = fmaxf(__uint_as_float(v[2 * j + 1]) + sbias[c0 + 2 * j + 1], 0.0f);
                    // round to nearest even (cvt.rn.bf16x2): x0 in the low half, x1 in the high half
                    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
                    std::memcpy(&packed[j], &h, sizeof(uint32_t));
                }
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
                    *(uint4 *)(out + (size_t)(m0 + quarter * 32 + r) * kTileN + c0 + q * 8) = w;
                }
                __syncwarp();
            }
        }
        // every warp has drained the accumulator before the next tile's MMAs overwrite it
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    }
    asm volatile("cp.async.wait_all;\n" ::);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tmem));
}

}  // namespace

cudaError_t ko_mlp_layer_tc(const uint16_t *A, const uint16_t *Wt, int M, int K, const float *bias, uint16_t *out,
                            int *err, cudaStream_t st)
{
    if (M % kTileM || (K != 192 && K != 256)) return cudaErrorInvalidValue;
    const size_t smem = (size_t)(kTileM + kTileN) * K * 2 + sizeof(float) * kTileN +
                        (kThreadsTc / 32) * 32 * 16 * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(tc_layer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = M / kTileM;
    const int grid = tiles < sms ? tiles : sms;
    tc_layer_kernel<<<grid, kThreadsTc, smem, st>>>(A, Wt, K, tiles, bias, out, err);
    ko_count_launch();
    return cudaGetLastError();
}
