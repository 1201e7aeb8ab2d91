// Hardware validation of the dispatch model: the measurement of Sec. 6 (every
// launch order of a kernel set run on the GPU and timed) applied to synthetic
// busy kernels on this GPU, so that simulated makespans can be ranked against
// measured times.
//
// A busy kernel is one of two fixed-work loops with a chosen block size,
// dynamic shared memory (reserved only, to set occupancy), grid and length:
//   compute  each thread runs a dependent FMA chain of `iters` steps;
//   memory   each thread streams `iters` 16-byte loads from a 256 MB buffer
//            (every address masked into the buffer) and sums them.
// Neither kernel waits on anything, so every launch ends.  A launch order is
// timed by putting kernel order[j] on stream j in host order j = 0, 1, ...
// between two events; the streams let the hardware run the kernels
// concurrently, and the host issue order is the launch order whose effect
// the model predicts (Sec. 2: blocks of the earlier-issued kernel first).
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "ko_internal.h"

namespace {

constexpr size_t kBufBytes = 256ull << 20;  // power of two: indexes are masked into it
constexpr int kMaxStreams = 8;

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned sm_id()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

// Per-block trace record (4 words): start ns, end ns, SM id, kernel id.  Thread
// 0 stamps the start on entry and the end after the block's last thread is done.
struct Trace {
    unsigned long long *rec;  // null: no tracing
    int kid;
    __device__ void begin() const
    {
        if (rec && threadIdx.x == 0) {
            rec[4 * blockIdx.x + 0] = global_ns();
            rec[4 * blockIdx.x + 2] = sm_id();
            rec[4 * blockIdx.x + 3] = (unsigned long long)kid;
        }
    }
    __device__ void end() const
    {
        if (rec) {
            __syncthreads();
            if (threadIdx.x == 0) rec[4 * blockIdx.x + 1] = global_ns();
        }
    }
};

__global__ void __launch_bounds__(1024) hw_compute_kernel(int iters, float b, float c, float *sink, Trace tr)
{
    tr.begin();
    float a = 1.0f + (float)threadIdx.x * 1e-3f;
#pragma unroll 4
    for (int i = 0; i < iters; i++) a = fmaf(a, b, c);
    // never true for the values used (|a| stays finite and != -7.5); keeps the chain live
    if (a == -7.5f) sink[blockIdx.x] = a;
    tr.end();
}

__global__ void __launch_bounds__(1024) hw_memory_kernel(const float4 *__restrict__ buf, unsigned long long mask,
                                                         int iters, float *sink, Trace tr)
{
    tr.begin();
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.0f;
    for (int k = 0; k < iters; k++, i += stride) {
        const float4 v = __ldcs(&buf[i & mask]);
        acc += v.x + v.y + v.z + v.w;
    }
    if (acc == -7.5f) sink[blockIdx.x] = acc;
    tr.end();
}

}  // namespace

struct ko_hw {
    std::vector<ko_hw_kernel> ks;
    cudaStream_t streams[kMaxStreams] = {};
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr, ev_done[kMaxStreams] = {};
    float4 *buf = nullptr;
    float *sink = nullptr;
    unsigned long long *trace = nullptr;  // 4 words per block of every kernel, kernel k at trace_off[k]
    std::vector<long long> trace_off;
    long long trace_blocks = 0;
};

namespace {

void hw_free(ko_hw *h)
{
    if (!h) return;
    for (int i = 0; i < kMaxStreams; i++) {
        if (h->streams[i]) cudaStreamDestroy(h->streams[i]);
        if (h->ev_done[i]) cudaEventDestroy(h->ev_done[i]);
    }
    if (h->ev_start) cudaEventDestroy(h->ev_start);
    if (h->ev_stop) cudaEventDestroy(h->ev_stop);
    cudaFree(h->buf);
    cudaFree(h->sink);
    cudaFree(h->trace);
    delete h;
}

// blocks <= the kernel's grid when traced (the trace holds `blocks` records per kernel)
cudaError_t launch_one(ko_hw *h, int k, int blocks, cudaStream_t st, bool traced = false)
{
    const ko_hw_kernel &d = h->ks[k];
    Trace tr{traced ? h->trace + 4 * h->trace_off[k] : nullptr, k};
    if (d.kind == KO_HW_COMPUTE)
        hw_compute_kernel<<<blocks, d.threads, d.smem, st>>>(d.iters, 0.999999f, 1e-6f, h->sink, tr);
    else
        hw_memory_kernel<<<blocks, d.threads, d.smem, st>>>(h->buf, kBufBytes / sizeof(float4) - 1, d.iters,
                                                            h->sink, tr);
    ko_count_launch();
    return cudaGetLastError();
}

}  // namespace

ko_hw *ko_hw_build(const ko_hw_kernel *ks, int n, ko_status *err)
{
    *err = KO_OK;
    if (!ks || n < 1 || n > kMaxStreams) { *err = KO_ERR_ARG; return nullptr; }
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    for (int i = 0; i < n; i++) {
        const ko_hw_kernel &d = ks[i];
        if ((d.kind != KO_HW_COMPUTE && d.kind != KO_HW_MEMORY) || d.threads < 32 || d.threads > 1024 ||
            d.threads % 32 || d.smem < 0 || d.smem > max_smem || d.blocks < 1 || d.blocks > (1 << 20) ||
            d.iters < 0 || d.iters > (1 << 24)) {
            *err = KO_ERR_ARG;
            return nullptr;
        }
    }
    ko_hw *h = new (std::nothrow) ko_hw();
    if (!h) { *err = KO_ERR_NOMEM; return nullptr; }
    h->ks.assign(ks, ks + n);
    for (int i = 0; i < n; i++) {
        h->trace_off.push_back(h->trace_blocks);
        h->trace_blocks += ks[i].blocks;
    }
    bool ok = cudaFuncSetAttribute(hw_compute_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem) ==
                  cudaSuccess &&
              cudaFuncSetAttribute(hw_memory_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem) ==
                  cudaSuccess;
    for (int i = 0; ok && i < n; i++)
        ok = cudaStreamCreateWithFlags(&h->streams[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreate(&h->ev_done[i]) == cudaSuccess;
    ok = ok && cudaEventCreate(&h->ev_start) == cudaSuccess && cudaEventCreate(&h->ev_stop) == cudaSuccess;
    if (!ok) { cudaGetLastError(); hw_free(h); *err = KO_ERR_CUDA; return nullptr; }
    if (cudaMalloc((void **)&h->buf, kBufBytes) != cudaSuccess || cudaMalloc((void **)&h->sink, 1 << 22) != cudaSuccess ||
        cudaMalloc((void **)&h->trace, sizeof(unsigned long long) * 4 * h->trace_blocks) != cudaSuccess) {
        cudaGetLastError();
        hw_free(h);
        *err = KO_ERR_NOMEM;
        return nullptr;
    }
    if (cudaMemset(h->buf, 0, kBufBytes) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        hw_free(h);
        *err = KO_ERR_CUDA;
        return nullptr;
    }
    return h;
}

void ko_hw_free(ko_hw *h) { hw_free(h); }

ko_status ko_hw_limits_impl(int32_t *out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return KO_ERR_CUDA; }
    const cudaDeviceAttr attrs[7] = {cudaDevAttrMultiProcessorCount,       cudaDevAttrMaxRegistersPerMultiprocessor,
                                     cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                                     cudaDevAttrMaxThreadsPerMultiProcessor, cudaDevAttrMaxBlocksPerMultiprocessor,
                                     cudaDevAttrReservedSharedMemoryPerBlock, cudaDevAttrClockRate};
    for (int i = 0; i < 7; i++) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, attrs[i], dev) != cudaSuccess) { cudaGetLastError(); return KO_ERR_CUDA; }
        out[i] = i == 3 ? v / 32 : v;
    }
    return KO_OK;
}

ko_status ko_hw_regs_impl(int kind, int *regs)
{
    cudaFuncAttributes a{};
    const cudaError_t e = kind == KO_HW_COMPUTE ? cudaFuncGetAttributes(&a, hw_compute_kernel)
                                                : cudaFuncGetAttributes(&a, hw_memory_kernel);
    if (e != cudaSuccess) { cudaGetLastError(); return KO_ERR_CUDA; }
    *regs = a.numRegs;
    return KO_OK;
}

// One launch order: kernel order[j] on stream j, in host order, between the
// start event (stream 0) and the stop event (after every stream's last work).
ko_status ko_hw_time_impl(ko_hw *h, const int8_t *orders, long long count, int reps, float *ms_out)
{
    const int n = (int)h->ks.size();
    cudaStream_t s0 = h->streams[0];
    std::vector<float> t(reps);
    for (long long o = 0; o < count; o++) {
        const int8_t *ord = orders + o * n;
        unsigned used = 0;
        for (int j = 0; j < n; j++) {
            if (ord[j] < 0 || ord[j] >= n || ((used >> ord[j]) & 1u)) return KO_ERR_ARG;
            used |= 1u << ord[j];
        }
        for (int r = 0; r < reps; r++) {
            if (cudaEventRecord(h->ev_start, s0) != cudaSuccess) return KO_ERR_CUDA;
            for (int j = 1; j < n; j++)
                if (cudaStreamWaitEvent(h->streams[j], h->ev_start, 0) != cudaSuccess) return KO_ERR_CUDA;
            for (int j = 0; j < n; j++)
                if (launch_one(h, ord[j], h->ks[ord[j]].blocks, h->streams[j]) != cudaSuccess) return KO_ERR_CUDA;
            for (int j = 1; j < n; j++) {
                if (cudaEventRecord(h->ev_done[j], h->streams[j]) != cudaSuccess ||
                    cudaStreamWaitEvent(s0, h->ev_done[j], 0) != cudaSuccess)
                    return KO_ERR_CUDA;
            }
            if (cudaEventRecord(h->ev_stop, s0) != cudaSuccess || cudaEventSynchronize(h->ev_stop) != cudaSuccess)
                return KO_ERR_CUDA;
            if (cudaEventElapsedTime(&t[r], h->ev_start, h->ev_stop) != cudaSuccess) return KO_ERR_CUDA;
        }
        std::sort(t.begin(), t.end());
        ms_out[o] = t[0];
    }
    return KO_OK;
}

// One run of one launch order with every block traced; records (host,
// 4 words per block, kernels in id order, blocks in index order) and the
// event time of the run.
ko_status ko_hw_trace_impl(ko_hw *h, const int8_t *ord, unsigned long long *rec_out, float *ms_out)
{
    const int n = (int)h->ks.size();
    unsigned used = 0;
    for (int j = 0; j < n; j++) {
        if (ord[j] < 0 || ord[j] >= n || ((used >> ord[j]) & 1u)) return KO_ERR_ARG;
        used |= 1u << ord[j];
    }
    cudaStream_t s0 = h->streams[0];
    const size_t bytes = sizeof(unsigned long long) * 4 * h->trace_blocks;
    if (cudaMemsetAsync(h->trace, 0, bytes, s0) != cudaSuccess || cudaStreamSynchronize(s0) != cudaSuccess)
        return KO_ERR_CUDA;
    if (cudaEventRecord(h->ev_start, s0) != cudaSuccess) return KO_ERR_CUDA;
    for (int j = 1; j < n; j++)
        if (cudaStreamWaitEvent(h->streams[j], h->ev_start, 0) != cudaSuccess) return KO_ERR_CUDA;
    for (int j = 0; j < n; j++)
        if (launch_one(h, ord[j], h->ks[ord[j]].blocks, h->streams[j], true) != cudaSuccess) return KO_ERR_CUDA;
    for (int j = 1; j < n; j++) {
        if (cudaEventRecord(h->ev_done[j], h->streams[j]) != cudaSuccess ||
            cudaStreamWaitEvent(s0, h->ev_done[j], 0) != cudaSuccess)
            return KO_ERR_CUDA;
    }
    if (cudaEventRecord(h->ev_stop, s0) != cudaSuccess || cudaEventSynchronize(h->ev_stop) != cudaSuccess ||
        cudaEventElapsedTime(ms_out, h->ev_start, h->ev_stop) != cudaSuccess)
        return KO_ERR_CUDA;
    if (cudaMemcpy(rec_out, h->trace, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return KO_ERR_CUDA;
    return KO_OK;
}

long long ko_hw_trace_blocks(const ko_hw *h) { return h->trace_blocks; }

// One kernel alone with a chosen grid (calibration of per-block durations and
// of the co-residence slowdown); the fastest of `reps` runs.
ko_status ko_hw_time_grid_impl(ko_hw *h, int k, int blocks, int reps, float *ms_out)
{
    if (k < 0 || k >= (int)h->ks.size()) return KO_ERR_ARG;
    cudaStream_t s0 = h->streams[0];
    float best = 0.0f;
    for (int r = 0; r < reps; r++) {
        float t = 0.0f;
        if (cudaEventRecord(h->ev_start, s0) != cudaSuccess || launch_one(h, k, blocks, s0) != cudaSuccess ||
            cudaEventRecord(h->ev_stop, s0) != cudaSuccess || cudaEventSynchronize(h->ev_stop) != cudaSuccess ||
            cudaEventElapsedTime(&t, h->ev_start, h->ev_stop) != cudaSuccess)
            return KO_ERR_CUDA;
        if (r == 0 || t < best) best = t;
    }
    *ms_out = best;
    return KO_OK;
}

// ------------------------------------------------------------ integer peak
// Issue-rate microbenchmark of the plain integer ALU path: every thread runs 8
// independent chains of (add, xor, min) on 32-bit registers, 16 steps per loop
// turn, each step one PTX instruction; the chains keep every scheduler's issue
// slot fed from register operands alone.  The result is the denominator of the
// simulators' integer roofline (lane-operations per second).
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;
constexpr int kPeakUnroll = 16;
constexpr long long kPeakOpsPerTurn = 3ll * kPeakChains * kPeakUnroll;

__global__ void __launch_bounds__(kPeakThreads) int_peak_kernel(uint32_t *sink, uint32_t s0, int turns)
{
    uint32_t a[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; c++) a[c] = s0 * (threadIdx.x + 1u) + (uint32_t)c * 0x9e3779b9u;
    const uint32_t b = s0 | 1u, x = s0 ^ 0xa5a5a5a5u, m = 0xfffffff0u ^ s0;
    for (int i = 0; i < turns; i++) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; u++) {
#pragma unroll
            for (int c = 0; c < kPeakChains; c++) {
                asm volatile("add.u32 %0, %0, %1;" : "+r"(a[c]) : "r"(b));
                asm volatile("xor.b32 %0, %0, %1;" : "+r"(a[c]) : "r"(x));
                asm volatile("min.u32 %0, %0, %1;" : "+r"(a[c]) : "r"(m));
            }
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int c = 0; c < kPeakChains; c++) r ^= a[c];
    if (r == s0) sink[blockIdx.x * kPeakThreads + threadIdx.x] = r;  // keeps the result observable
}

}  // namespace

ko_status ko_hw_int_peak_impl(int32_t turns, int64_t *lane_ops, float *ms_out)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, int_peak_kernel, kPeakThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return KO_ERR_CUDA;
    }
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    uint32_t *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ko_status st = KO_OK;
    if (cudaMalloc(&sink, sizeof(uint32_t) * (size_t)blocks * kPeakThreads) != cudaSuccess) {
        cudaGetLastError();
        return KO_ERR_NOMEM;
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = KO_ERR_CUDA;
    float best = 0.0f;
    for (int rep = 0; st == KO_OK && rep < 4; rep++) {  // the first run warms up; the fastest of the rest counts
        cudaEventRecord(e0, 0);
        int_peak_kernel<<<blocks, kPeakThreads>>>(sink, 0x1234567u + (uint32_t)rep, rep == 0 ? 16 : turns);
        ko_count_launch();
        cudaEventRecord(e1, 0);
        float ms = 0.0f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            st = KO_ERR_CUDA;
        else if (rep > 0 && (best == 0.0f || ms < best))
            best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    cudaGetLastError();
    if (st) return st;
    *lane_ops = (int64_t)blocks * kPeakThreads * turns * kPeakOpsPerTurn;
    *ms_out = best;
    return KO_OK;
}

