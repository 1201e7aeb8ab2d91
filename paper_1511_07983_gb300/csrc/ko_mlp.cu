// Surrogate MLP kernels: BF16 tensor-core GEMMs with FP32 accumulation and
// fused epilogues, plus the small elementwise kernels of training and
// inference.  The network is 192 -> 256 -> 256 -> 256 -> 1 with ReLU; it
// predicts log2(makespan / lower bound) of a launch order from position-
// ordered kernel descriptors (not part of the paper: a proposal generator for
// sets too large to enumerate, whose proposals are rescored exactly).
//
// The GEMMs here are the warp-level mma.sync path; the tcgen05 kernels of
// ko_mlp_tc.cu run every GEMM whose sizes their tiles divide, and these take
// the rest (batches that are not multiples of 128, or 256 for weight
// gradients) and serve as the cross-check in tests.
//
// GEMM form used everywhere ("NT"): C[m][n] = sum_k A[m][k] * B[n][k], both
// operands K-contiguous BF16 in global memory.  Forward layers take
// B = W^T (stored n-major), input gradients take B = W (k-major), weight
// gradients take A = activations^T and B = dZ^T (both stored transposed by
// the producing kernels).  Tiles: 64 x 128 x 32 per block of 4 warps (each
// warp 32 x 64 = 2 x 8 mma.m16n8k16 tiles), three-stage cp.async pipeline,
// ldmatrix fragment loads from padded shared memory.
#include <cuda_bf16.h>

#include "ko_mlp.h"

namespace {

constexpr int BM = 64, BN = 128, BK = 32, STAGES = 3;
constexpr int PAD = 8;                 // bf16 elements of row padding (16 B): conflict-free ldmatrix
constexpr int LDS = BK + PAD;          // shared-memory row length in elements

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3,
                                            const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float *d, const uint32_t *a, const uint32_t *b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// round-to-nearest-even float -> bf16 bits (explicit bit arithmetic)
__device__ __forceinline__ uint16_t bf16_bits(float x)
{
    uint32_t u = __float_as_uint(x);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
__device__ __forceinline__ float bf16_val(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

struct Epi {
    int mode;                  // kEpiReluBf16 or kEpiF32
    const float *bias;         // [N] (relu mode)
    uint16_t *out_bf16;        // [M x ldo]
    uint16_t *out_bf16_t;      // [N x ldt] transposed copy, nullable
    float *out_f32;            // [M x ldo] (f32 mode)
    int ldo, ldt;
};

__global__ void __launch_bounds__(128)
gemm_nt_kernel(const uint16_t *__restrict__ A, int lda, const uint16_t *__restrict__ B, int ldb, int M,
               int N, int K, Epi ep)
{
    __shared__ __align__(16) uint16_t sA[STAGES][BM][LDS];
    __shared__ __align__(16) uint16_t sB[STAGES][BN][LDS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int ktiles = K / BK;

    auto load_stage = [&](int stage, int kt) {
        const int k0 = kt * BK;
#pragma unroll
        for (int i = 0; i < 2; i++) {  // A: 64 rows x 4 chunks of 8 bf16
            const int c = tid + i * 128, row = c >> 2, ch = c & 3;
            cp_async16(&sA[stage][row][ch * 8], A + (size_t)(m0 + row) * lda + k0 + ch * 8);
        }
#pragma unroll
        for (int i = 0; i < 4; i++) {  // B: 128 rows x 4 chunks
            const int c = tid + i * 128, row = c >> 2, ch = c & 3;
            cp_async16(&sB[stage][row][ch * 8], B + (size_t)(n0 + row) * ldb + k0 + ch * 8);
        }
    };

    float acc[2][8][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 8; j++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[i][j][q] = 0.0f;

#pragma unroll
    for (int s = 0; s < STAGES - 1; s++) {
        if (s < ktiles) load_stage(s, s);
        cp_async_commit();
    }
    for (int kt = 0; kt < ktiles; kt++) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        const int nk = kt + STAGES - 1;
        if (nk < ktiles) load_stage(nk % STAGES, nk);
        cp_async_commit();
        const int st = kt % STAGES;
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bfr[8][2];
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int row = wm * 32 + i * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
                const int col = kk + (lane >> 4) * 8;
                ldmatrix_x4(af[i][0], af[i][1], af[i][2], af[i][3], &sA[st][row][col]);
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int row = wn * 64 + j * 16 + (lane & 7) + (lane >> 4) * 8;
                const int col = kk + ((lane >> 3) & 1) * 8;
                ldmatrix_x4(bfr[2 * j][0], bfr[2 * j][1], bfr[2 * j + 1][0], bfr[2 * j + 1][1],
                            &sB[st][row][col]);
            }
#pragma unroll
            for (int i = 0; i < 2; i++)
#pragma unroll
                for (int j = 0; j < 8; j++) mma_bf16(acc[i][j], af[i], bfr[j]);
        }
    }
    cp_async_wait<0>();

    // epilogue
#pragma unroll
    for (int i = 0; i < 2; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int col = n0 + wn * 64 + j * 8 + (lane & 3) * 2;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int row = m0 + wm * 32 + i * 16 + (lane >> 2) + h * 8;
                float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
                if (ep.mode == kEpiReluBf16) {
                    v0 = fmaxf(v0 + ep.bias[col], 0.0f);
                    v1 = fmaxf(v1 + ep.bias[col + 1], 0.0f);
                    const uint16_t b0 = bf16_bits(v0), b1 = bf16_bits(v1);
                    *(uint32_t *)&ep.out_bf16[(size_t)row * ep.ldo + col] = (uint32_t)b0 | ((uint32_t)b1 << 16);
                    if (ep.out_bf16_t) {
                        ep.out_bf16_t[(size_t)col * ep.ldt + row] = b0;
                        ep.out_bf16_t[(size_t)(col + 1) * ep.ldt + row] = b1;
                    }
                } else {
                    *(float2 *)&ep.out_f32[(size_t)row * ep.ldo + col] = make_float2(v0, v1);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- encoding

// x[b] = features of order rows[b] of set sid[b]: kernel at position p goes to
// slot round(23 p / (N-1)); 7 features per slot; 8 global features; zeros
// elsewhere.  Output bf16 row-major [B x 192] and transposed [192 x B].
// Position of an N-kernel order whose slot is `slot`, or -1 (the slots of
// distinct positions are distinct): slot(p) = (2*23*p + (n-1)) / (2(n-1)),
// inverted by testing the positions nearest to slot*(n-1)/23.
__device__ __forceinline__ int slot_position(int n, int slot)
{
    if (n <= 1) return n == 1 && slot == 0 ? 0 : -1;
    const int p0 = (slot * (n - 1)) / (kSlots - 1);
    int pos = -1;
    for (int p = p0 - 1; p <= p0 + 1; p++)
        if (p >= 0 && p < n && (2 * (kSlots - 1) * p + (n - 1)) / (2 * (n - 1)) == slot) pos = p;
    return pos;
}

// One thread per row, a warp per 32 consecutive rows.  Per block: the slot ->
// position map of every N and -- for a single set (no sid) -- the set's
// kernel and global features.  Per warp step: the 32 rows' order bytes are
// copied to shared memory with coalesced loads (contiguous rows, no pick);
// each thread produces its row's 192 features in order (slot by slot: one
// kernel index, its 7 features; then the globals and the zero padding),
// packs them two BF16 to a word (round to nearest even) and writes them to a
// per-warp staging area (row pitch 400 bytes: conflict-free 16-byte stores);
// the warp then stores its 32 rows (12,288 contiguous bytes) 16 bytes per
// lane.  xt (training) gets the transposed copy value by value.
constexpr int kEncWarps = 2, kEncPitch = 100;  // staging row pitch in words
__global__ void __launch_bounds__(kEncWarps * 32) encode_kernel(const int8_t *__restrict__ rows, int row_stride,
                                                                const int *__restrict__ sid,
                                                                const int *__restrict__ pick,
                                                                const int *__restrict__ set_n,
                                                                const float *__restrict__ kfeat,
                                                                const float *__restrict__ gfeat, int B,
                                                                uint16_t *x, uint16_t *xt)
{
    __shared__ int8_t s_pos[kMaxK + 1][kSlots];
    __shared__ float s_kf[kMaxK * kSlotFeat + kGlobals];
    __shared__ __align__(16) int8_t s_rows[kEncWarps][32 * kMaxK];
    __shared__ __align__(16) uint32_t s_out[kEncWarps][32 * kEncPitch];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < (kMaxK + 1) * kSlots; i += blockDim.x)
        s_pos[i / kSlots][i % kSlots] = (int8_t)slot_position(i / kSlots, i % kSlots);
    if (!sid) {
        for (int i = threadIdx.x; i < kMaxK * kSlotFeat; i += blockDim.x) s_kf[i] = kfeat[i];
        for (int i = threadIdx.x; i < kGlobals; i += blockDim.x) s_kf[kMaxK * kSlotFeat + i] = gfeat[i];
    }
    __syncthreads();
    const bool stage = !pick && row_stride <= kMaxK;
    const long long wsteps = ((long long)B + 31) / 32;
    for (long long ws = (long long)blockIdx.x * kEncWarps + warp; ws < wsteps;
         ws += (long long)gridDim.x * kEncWarps) {
        const int base = (int)(ws * 32), nrows = B - base < 32 ? B - base : 32;
        __syncwarp();  // the previous step's staging has been stored
        if (stage) {
            const int8_t *src = rows + (size_t)base * row_stride;
            const int nb = nrows * row_stride;
            if ((((uintptr_t)src) & 15u) == 0 && (nb & 15) == 0) {
                // 16 bytes per lane: all loads in flight together
                const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
                uint4 *d4 = reinterpret_cast<uint4 *>(s_rows[warp]);
                for (int i = lane; i < nb / 16; i += 32) d4[i] = s4[i];
            } else {
                for (int i = lane; i < nb; i += 32) s_rows[warp][i] = src[i];
            }
            __syncwarp();
        }
        if (lane < nrows) {
            const int b = base + lane;
            const int src = pick ? pick[b] : b;
            const int set = sid ? sid[src] : 0;
            const int n = set_n[set];
            const int8_t *row = stage ? &s_rows[warp][lane * row_stride] : rows + (size_t)src * row_stride;
            const float *kf = sid ? kfeat + (size_t)set * kMaxK * kSlotFeat : s_kf;
            const float *gf = sid ? gfeat + (size_t)set * kGlobals : s_kf + kMaxK * kSlotFeat;
            uint32_t *out = &s_out[warp][lane * kEncPitch];
            float v[8];
            auto put = [&](int f, float val) {  // f is a constant after unrolling
                v[f & 7] = val;
                if ((f & 7) == 7) {
                    uint32_t w[4];
#pragma unroll
                    for (int h = 0; h < 4; h++) {
                        const __nv_bfloat162 p2 = __floats2bfloat162_rn(v[2 * h], v[2 * h + 1]);
                        memcpy(&w[h], &p2, sizeof(uint32_t));
                    }
                    *reinterpret_cast<uint4 *>(out + (f >> 3) * 4) = make_uint4(w[0], w[1], w[2], w[3]);
                    if (xt) {
#pragma unroll
                        for (int h = 0; h < 8; h++)
                            xt[(size_t)((f & ~7) + h) * B + b] = (uint16_t)(w[h >> 1] >> ((h & 1) * 16));
                    }
                }
            };
#pragma unroll
            for (int slot = 0; slot < kSlots; slot++) {
                const int pos = s_pos[n][slot];
                const int k = pos >= 0 ? (int)row[pos] : -1;
#pragma unroll
                for (int q = 0; q < kSlotFeat; q++) put(slot * kSlotFeat + q, k >= 0 ? kf[k * kSlotFeat + q] : 0.0f);
            }
#pragma unroll
            for (int g = 0; g < kGlobals; g++) put(kSlots * kSlotFeat + g, gf[g]);
#pragma unroll
            for (int f = kSlots * kSlotFeat + kGlobals; f < kMlpIn; f++) put(f, 0.0f);
        }
        __syncwarp();
        // the warp's rows are contiguous in x: 16 bytes per lane per store
        uint4 *dst = reinterpret_cast<uint4 *>(x + (size_t)base * kMlpIn);
        for (int i = lane; i < nrows * (kMlpIn / 8); i += 32) {
            const int r = i / (kMlpIn / 8), c = i % (kMlpIn / 8);
            dst[i] = *reinterpret_cast<const uint4 *>(&s_out[warp][r * kEncPitch + c * 4]);
        }
    }
}

// y[b] = A3[b] . w4 + b4: eight threads per row, thread c sums columns
// 32c .. 32c + 31 as a chain of fused multiply-adds in column order, and the
// eight partials combine as ((p0 + p1) + (p2 + p3)) + ((p4 + p5) + (p6 + p7))
// before b4 is added (the order the fused tcgen05 last layer uses too).
__global__ void out_fwd_kernel(const uint16_t *__restrict__ a3, const uint16_t *__restrict__ w4,
                               const float *__restrict__ b4, int B, float *y)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = (int)(i >> 3), c = (int)(i & 7);
    float s = 0.0f;
    if (b < B) {
        const uint4 *src = reinterpret_cast<const uint4 *>(a3 + (size_t)b * kHidden + c * 32);
        const uint16_t *w = w4 + c * 32;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint4 v = src[q];
            const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int h = 0; h < 4; h++) {
                s = __fmaf_rn(__uint_as_float(u[h] << 16), bf16_val(w[8 * q + 2 * h]), s);
                s = __fmaf_rn(__uint_as_float(u[h] & 0xFFFF0000u), bf16_val(w[8 * q + 2 * h + 1]), s);
            }
        }
    }
    // eight threads of a row sit in one aligned group of eight lanes
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    if (b < B && c == 0) y[b] = s + b4[0];
}

// Output layer backward: dy = 2 (y - t) / B; loss sum; dw4 = sum dy * A3; db4 = sum dy;
// dZ3 = dy * w4 * [A3 > 0] (fp32 for the bias gradient, bf16 + transposed for GEMMs).
// Each block writes its partial sums (rows r0 .. r0+31) to part[blockIdx.x]:
// dw4 partials, db3 partials, loss, db4; part_sum_kernel adds them up in
// block order, so the gradients do not depend on the order blocks finish in.
constexpr int kPartOut = 2 * kHidden + 2;

__global__ void out_bwd_kernel(const float *__restrict__ y, const float *__restrict__ t,
                               const uint16_t *__restrict__ a3, const uint16_t *__restrict__ w4, int B,
                               float *part, uint16_t *dz, uint16_t *dzt)
{
    __shared__ float s_dw[kHidden], s_db[kHidden];
    for (int k = threadIdx.x; k < kHidden; k += blockDim.x) { s_dw[k] = 0.0f; s_db[k] = 0.0f; }
    __syncthreads();
    const int rows_per_block = 32;
    const int r0 = blockIdx.x * rows_per_block;
    float lsum = 0.0f, dbsum = 0.0f;
    for (int r = r0; r < r0 + rows_per_block && r < B; r++) {
        const float d = y[r] - t[r];
        const float dy = 2.0f * d / (float)B;
        if (threadIdx.x == 0) { lsum += d * d; dbsum += dy; }
        for (int k = threadIdx.x; k < kHidden; k += blockDim.x) {
            const float a = bf16_val(a3[(size_t)r * kHidden + k]);
            s_dw[k] += dy * a;
            const float g = a > 0.0f ? dy * bf16_val(w4[k]) : 0.0f;
            s_db[k] += g;
            const uint16_t bits = bf16_bits(g);
            dz[(size_t)r * kHidden + k] = bits;
            dzt[(size_t)k * B + r] = bits;
        }
    }
    __syncthreads();
    float *mine = part + (size_t)blockIdx.x * kPartOut;
    for (int k = threadIdx.x; k < kHidden; k += blockDim.x) {
        mine[k] = s_dw[k];
        mine[kHidden + k] = s_db[k];
    }
    if (threadIdx.x == 0) {
        mine[2 * kHidden] = lsum;
        mine[2 * kHidden + 1] = dbsum;
    }
}

// Hidden-layer ReLU backward: dZ = dA * [A > 0]; bias-gradient partials per
// block (fp32) into part[blockIdx.x]; dZ as bf16 row-major and transposed.
__global__ void relu_bwd_kernel(const float *__restrict__ da, const uint16_t *__restrict__ a, int B,
                                float *part, uint16_t *dz, uint16_t *dzt)
{
    __shared__ float s_db[kHidden];
    for (int k = threadIdx.x; k < kHidden; k += blockDim.x) s_db[k] = 0.0f;
    __syncthreads();
    const int rows_per_block = 32;
    const int r0 = blockIdx.x * rows_per_block;
    for (int r = r0; r < r0 + rows_per_block && r < B; r++) {
        for (int k = threadIdx.x; k < kHidden; k += blockDim.x) {
            const size_t i = (size_t)r * kHidden + k;
            const float g = bf16_val(a[i]) > 0.0f ? da[i] : 0.0f;
            s_db[k] += g;
            const uint16_t bits = bf16_bits(g);
            dz[i] = bits;
            dzt[(size_t)k * B + r] = bits;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kHidden; k += blockDim.x) part[(size_t)blockIdx.x * kHidden + k] = s_db[k];
}

// Column sums of nblk rows of `width` partials, rows added in order.  Columns
// [0, span) go to lo[c], [span, 2 span) to hi[c - span], column 2 span to *s0
// and 2 span + 1 to *s1.
struct PartDst {
    float *lo, *hi, *s0, *s1;
    int span;
};
__global__ void part_sum_kernel(const float *__restrict__ part, int nblk, int width, PartDst dst)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= width) return;
    float acc = 0.0f;
    for (int b = 0; b < nblk; b++) acc += part[(size_t)b * width + c];
    if (c < dst.span) dst.lo[c] = acc;
    else if (c < 2 * dst.span) dst.hi[c - dst.span] = acc;
    else if (c == 2 * dst.span) *dst.s0 = acc;
    else *dst.s1 = acc;
}

// Adam on the FP32 master weights, then refresh the BF16 copies the GEMMs read.
__global__ void adam_kernel(float *p, float *m, float *v, const float *g, long long count, float lr,
                            float b1, float b2, float eps, float c1, float c2)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / c1, vh = vi / c2;
        p[i] -= lr * mh / (sqrtf(vh) + eps);
    }
}

// BF16 copies of one weight matrix W [K x N] (k-major): W itself and W^T.
__global__ void weights_bf16_kernel(const float *__restrict__ w, int K, int N, uint16_t *wk,
                                    uint16_t *wt)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K * N; i += gridDim.x * blockDim.x) {
        const int k = i / N, n = i % N;
        const uint16_t b = bf16_bits(w[i]);
        if (wk) wk[i] = b;
        if (wt) wt[(size_t)n * K + k] = b;
    }
}

// Order-preserving key of a float (smaller prediction = smaller key).
__device__ __forceinline__ uint32_t float_key(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Radix-select pass: histogram of the next 8-bit digit among keys whose
// higher digits equal the prefix found so far.
__global__ void select_hist_kernel(const float *__restrict__ y, long long n, const uint32_t *state,
                                   int shift, unsigned int *hist)
{
    __shared__ unsigned int h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint32_t prefix = state[0];
    const uint32_t mask = shift == 24 ? 0u : (0xFFFFFFFFu << (shift + 8));
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const uint32_t k = float_key(y[i]);
        if ((k & mask) == (prefix & mask)) atomicAdd(&h[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// Fix the digit: state = {prefix, remaining k}; clears the histogram.
__global__ void select_scan_kernel(uint32_t *state, int shift, unsigned int *hist)
{
    if (threadIdx.x == 0) {
        uint32_t need = state[1];
        uint32_t cum = 0;
        int digit = 255;
        for (int d = 0; d < 256; d++) {
            if (cum + hist[d] >= need) { digit = d; break; }
            cum += hist[d];
        }
        state[0] |= (uint32_t)digit << shift;
        state[1] = need - cum;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
}

// Write the indices of the k smallest keys: all keys below the threshold and
// `remaining` keys equal to it.
__global__ void select_emit_kernel(const float *__restrict__ y, long long n, const uint32_t *state,
                                   unsigned int *counters, int k, int *out)
{
    const uint32_t thr = state[0], eq_quota = state[1];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const uint32_t key = float_key(y[i]);
        if (key < thr) {
            const unsigned int s = atomicAdd(&counters[0], 1u);
            if (s < (unsigned)k) out[s] = (int)i;
        } else if (key == thr) {
            const unsigned int e = atomicAdd(&counters[1], 1u);
            if (e < eq_quota) {
                const unsigned int s = atomicAdd(&counters[0], 1u);
                if (s < (unsigned)k) out[s] = (int)i;
            }
        }
    }
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Uniform random permutations (Fisher-Yates) from a counter-based SplitMix64
// stream per row: row r uses mix64(seed + (r * 2^6 + step) * golden).
__global__ void random_orders_kernel(int8_t *rows, int stride, long long count, int n,
                                     unsigned long long seed)
{
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < count;
         r += (long long)gridDim.x * blockDim.x) {
        int8_t p[kMaxK];
        for (int i = 0; i < n; i++) p[i] = (int8_t)i;
        for (int i = n - 1; i > 0; i--) {
            const unsigned long long x =
                mix64(seed + ((unsigned long long)r * 64ull + (unsigned long long)i) * 0x9E3779B97F4A7C15ull);
            const int j = (int)(x % (unsigned long long)(i + 1));
            const int8_t t = p[i];
            p[i] = p[j];
            p[j] = t;
        }
        for (int i = 0; i < n; i++) rows[r * stride + i] = p[i];
    }
}

// target = log2(makespan / lower bound) as float; invalid makespans give 0.
__global__ void targets_kernel(const int64_t *ms, const int *sid, const double *log2_lb, long long n,
                               float *t)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long m = ms[i];
        t[i] = m > 0 ? (float)(log2((double)m) - log2_lb[sid ? sid[i] : 0]) : 0.0f;
    }
}

// All single-step neighbours of `beam` base orders (rows of stride 24): first
// the n(n-1)/2 swaps of two positions, then the n(n-1) moves of one kernel to
// another position (the rest shift by one).  Row r = b * per + q.
__global__ void neighbours_kernel(const int8_t *__restrict__ base, int beam, int n, int8_t *out)
{
    const int swaps = n * (n - 1) / 2, per = swaps + n * (n - 1);
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= beam * per) return;
    const int b = r / per, q = r % per;
    int8_t p[kMaxK];
    for (int i = 0; i < n; i++) p[i] = base[b * kMaxK + i];
    if (q < swaps) {
        int i = 0, rem = q;
        while (rem >= n - 1 - i) { rem -= n - 1 - i; i++; }
        const int j = i + 1 + rem;
        const int8_t t = p[i]; p[i] = p[j]; p[j] = t;
    } else {
        const int m = q - swaps, from = m / (n - 1), k = m % (n - 1);
        const int to = k < from ? k : k + 1;
        const int8_t v = p[from];
        if (from < to) { for (int i = from; i < to; i++) p[i] = p[i + 1]; }
        else { for (int i = from; i > to; i--) p[i] = p[i - 1]; }
        p[to] = v;
    }
    int8_t *o = out + (size_t)r * kMaxK;
    for (int i = 0; i < kMaxK; i++) o[i] = i < n ? p[i] : (int8_t)0;
}

__global__ void random_pick_kernel(int *pick, int B, long long pool, unsigned long long seed)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) pick[b] = (int)(mix64(seed + (unsigned long long)b * 0x9E3779B97F4A7C15ull) % (unsigned long long)pool);
}

__global__ void gather_f32_kernel(const float *src, const int *pick, int B, float *dst)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) dst[b] = src[pick[b]];
}

__global__ void gather_rows_kernel(const int8_t *src, int stride, const int *pick, int B, int8_t *dst)
{
    const int b = blockIdx.x;
    if (b < B && threadIdx.x < stride) dst[(size_t)b * stride + threadIdx.x] = src[(size_t)pick[b] * stride + threadIdx.x];
}

}  // namespace

cudaError_t ko_mlp_gemm_relu(const uint16_t *A, int lda, const uint16_t *Bt, int ldb, int M, int N, int K,
                             const float *bias, uint16_t *out, int ldo, uint16_t *out_t, int ldt,
                             cudaStream_t st)
{
    if (M % BM || N % BN || K % BK) return cudaErrorInvalidValue;
    Epi ep{kEpiReluBf16, bias, out, out_t, nullptr, ldo, ldt};
    gemm_nt_kernel<<<dim3(N / BN, M / BM), 128, 0, st>>>(A, lda, Bt, ldb, M, N, K, ep);
    ko_count_launch();
    return cudaGetLastError();
}

cudaError_t ko_mlp_gemm_f32(const uint16_t *A, int lda, const uint16_t *Bt, int ldb, int M, int N, int K,
                            float *out, int ldo, cudaStream_t st)
{
    if (M % BM || N % BN || K % BK) return cudaErrorInvalidValue;
    Epi ep{kEpiF32, nullptr, nullptr, nullptr, out, ldo, 0};
    gemm_nt_kernel<<<dim3(N / BN, M / BM), 128, 0, st>>>(A, lda, Bt, ldb, M, N, K, ep);
    ko_count_launch();
    return cudaGetLastError();
}

cudaError_t ko_mlp_encode(const int8_t *rows, int row_stride, const int *sid, const int *pick,
                          const int *set_n, const float *kfeat, const float *gfeat, int B, uint16_t *x,
                          uint16_t *xt, cudaStream_t st)
{
    if (B <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long blocks = ((long long)B + 32 * kEncWarps - 1) / (32 * kEncWarps);
    const int grid = (int)(blocks < (long long)sms * 8 ? blocks : (long long)sms * 8);
    encode_kernel<<<grid, kEncWarps * 32, 0, st>>>(rows, row_stride, sid, pick, set_n, kfeat, gfeat, B, x, xt);
    ko_count_launch();
    return cudaGetLastError();
}

cudaError_t ko_mlp_out_fwd(const uint16_t *a3, const uint16_t *w4, const float *b4, int B, float *y,
                           cudaStream_t st)
{
    out_fwd_kernel<<<(unsigned)(((long long)B * 8 + 255) / 256), 256, 0, st>>>(a3, w4, b4, B, y);
    ko_count_launch();
    return cudaGetLastError();
}

size_t ko_mlp_part_floats(int B) { return (size_t)((B + 31) / 32) * kPartOut; }

cudaError_t ko_mlp_out_bwd(const float *y, const float *t, const uint16_t *a3, const uint16_t *w4, int B,
                           float *loss_sum, float *dw4, float *db4, float *db3, uint16_t *dz,
                           uint16_t *dzt, float *part, cudaStream_t st)
{
    const int nblk = (B + 31) / 32;
    out_bwd_kernel<<<nblk, 256, 0, st>>>(y, t, a3, w4, B, part, dz, dzt);
    // columns: dw4 [0, 256), db3 [256, 512), loss 512, db4 513
    PartDst d{dw4, db3, loss_sum, db4, kHidden};
    part_sum_kernel<<<(2 * kHidden + 2 + 255) / 256, 256, 0, st>>>(part, nblk, kPartOut, d);
    ko_count_launch(2);
    return cudaGetLastError();
}

cudaError_t ko_mlp_relu_bwd(const float *da, const uint16_t *a, int B, float *db, uint16_t *dz,
                            uint16_t *dzt, float *part, cudaStream_t st)
{
    const int nblk = (B + 31) / 32;
    relu_bwd_kernel<<<nblk, 256, 0, st>>>(da, a, B, part, dz, dzt);
    PartDst d{db, nullptr, nullptr, nullptr, kHidden};
    part_sum_kernel<<<(kHidden + 255) / 256, 256, 0, st>>>(part, nblk, kHidden, d);
    ko_count_launch(2);
    return cudaGetLastError();
}

cudaError_t ko_mlp_adam(float *p, float *m, float *v, const float *g, long long count, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t st)
{
    adam_kernel<<<256, 256, 0, st>>>(p, m, v, g, count, lr, b1, b2, eps, c1, c2);
    ko_count_launch();
    return cudaGetLastError();
}

cudaError_t ko_mlp_weights_bf16(const float *w, int K, int N, uint16_t *wk, uint16_t *wt, cudaStream_t st)
{
    weights_bf16_kernel<<<256, 256, 0, st>>>(w, K, N, wk, wt);
    ko_count_launch();
    return cudaGetLastError();
}

cudaError_t ko_mlp_topk(const float *y, long long n, int k, uint32_t *state, unsigned int *hist,
                        unsigned int *counters, int *out, cudaStream_t st)
{
    // state = {prefix 0, remaining k}; hist and counters zeroed here
    uint32_t init[2] = {0u, (uint32_t)k};
    if (cudaMemcpyAsync(state, init, sizeof(init), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned int), st) != cudaSuccess ||
        cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned int), st) != cudaSuccess)
        return cudaGetLastError();
    const int blocks = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    for (int shift = 24; shift >= 0; shift -= 8) {
        select_hist_kernel<<<blocks, 256, 0, st>>>(y, n, state, shift, hist);
        select_scan_kernel<<<1, 256, 0, st>>>(state, shift, hist);
        ko_count_launch(2);
    }
    select_emit_kernel<<<blocks, 256, 0, st>>>(y, n, state, counters, k, out);
    ko_count_launch();
    return cudaGetLastError();
}

cudaError_t ko_mlp_random_orders(int8_t *rows, int stride, long long count, int n, unsigned long long seed,
                                 cudaStream_t st)
{
    long long blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    random_orders_kernel<<<(unsigned)blocks, 256, 0, st>>>(rows, stride, count, n, seed);
    ko_count_launch();
    return cudaGetLastError();
}

cudaError_t ko_mlp_targets(const int64_t *ms, const int *sid, const double *log2_lb, long long n, float *t,
                           cudaStream_t st)
{
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    targets_kernel<<<(unsigned)blocks, 256, 0, st>>>(ms, sid, log2_lb, n, t);
    ko_count_launch();
    return cudaGetLastError();
}

cudaError_t ko_mlp_pick(int *pick, int B, long long pool, unsigned long long seed, const float *t_src,
                        float *t_dst, cudaStream_t st)
{
    random_pick_kernel<<<(B + 255) / 256, 256, 0, st>>>(pick, B, pool, seed);
    gather_f32_kernel<<<(B + 255) / 256, 256, 0, st>>>(t_src, pick, B, t_dst);
    ko_count_launch(2);
    return cudaGetLastError();
}

cudaError_t ko_mlp_neighbours(const int8_t *base, int beam, int n, int8_t *out, cudaStream_t st)
{
    const int per = n * (n - 1) / 2 + n * (n - 1);
    const int rows = beam * per;
    if (rows <= 0) return cudaSuccess;
    neighbours_kernel<<<(rows + 127) / 128, 128, 0, st>>>(base, beam, n, out);
    ko_count_launch();
    return cudaGetLastError();
}

cudaError_t ko_mlp_gather_rows(const int8_t *src, int stride, const int *pick, int B, int8_t *dst,
                               cudaStream_t st)
{
    gather_rows_kernel<<<B, 32, 0, st>>>(src, stride, pick, B, dst);
    ko_count_launch();
    return cudaGetLastError();
}
