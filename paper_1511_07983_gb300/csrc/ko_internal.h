// Internal declarations shared by libko's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "ko.h"

// Per-block kernel descriptor (Table 1, last three rows): registers, shared
// memory bytes, warps of one block, block count, compute and memory cycles of
// one block running alone.
struct KoKern {
    int32_t r, s, w, b, c, m;
};

// Packed per-kernel record of the one-thread-per-order simulator (ko_lane.cu):
// one block's share of its usage word (registers | 1 << 19 | warps << 25;
// meaningful when N_reg_SM < 2^19 and N_warp_SM < 128), shared memory, c, m.
struct KoLaneK {
    uint32_t pk, s, c, m;
};

// Device-side description of one kernel set on one simulated GPU.
struct KoSet {
    int32_t n;                   // kernels in the set
    int32_t S, R, Sh, W, Bk;     // N_SM and the four per-SM limits
    int64_t ccap, mcap;          // compute / memory capacity (R_B = ccap / mcap)
    int32_t cshift, mshift;      // log2(capacity) when a power of two, else -1
    int32_t sampling;            // KO_SAMPLE_BURST_END or KO_SAMPLE_AT_PLACEMENT
    int32_t pad0;
    int64_t ref_makespan;        // makespan the exhaustive counts compare against
    KoKern k[KO_MAX_KERNELS];
    KoLaneK lk[KO_MAX_KERNELS];  // the same kernels, packed (16-byte aligned: KoKern table is 576 bytes)
};

// Exhaustive accumulators of one set (device memory).
struct KoAccum {
    unsigned long long min, max;
    unsigned long long n_better, n_equal, n_worse;
    unsigned long long failed;   // simulations that could not finish
};

// Count of kernels launched by the library (ko_kernel_launches).
void ko_count_launch(int n = 1);

// ------------------------------------------------------------------ launchers
// All launchers are asynchronous on `stream` and return the launch status.

// Processor-sharing simulator (ko_sim_ps.cu): makespans (double) of explicit
// rows (N bytes each), per-thread scratch of ko_ps_scratch_per_thread bytes.
size_t ko_ps_scratch_per_thread(const KoSet &h);
cudaError_t ko_launch_ps(const KoSet *d_set, const KoSet &h_set, const int8_t *perms, int64_t count, double *out,
                         void *scratch, size_t scratch_bytes, cudaStream_t stream);

// Per-thread scratch bytes the simple simulator needs for one set.
size_t ko_simple_scratch_per_thread(const KoSet &h);

// Simple exact simulator, one thread per order.  Orders come from
//   perms  (count x n int8 rows)            if perms != nullptr,
//   idx    (count Lehmer indices)           else if idx != nullptr,
//   first + j (contiguous Lehmer indices)   otherwise.
// Writes makespans (if out != nullptr) and folds them into acc (if non-null).
cudaError_t ko_launch_simple(const KoSet *d_set, const KoSet &h_set, const int8_t *perms,
                             const uint64_t *idx, uint64_t first, int64_t count, int64_t *out,
                             KoAccum *acc, void *scratch, size_t scratch_bytes,
                             cudaStream_t stream);

// Histogram of `count` makespans with bin = (M - min) * nbins / (max - min + 1),
// min / max read from acc on the device; hist (device, nbins u64) is added to.
cudaError_t ko_launch_histogram(const int64_t *ms, int64_t count, const KoAccum *acc,
                                unsigned long long *hist, int32_t nbins, cudaStream_t stream);

// Resets an accumulator to (min = max u64, max = 0, counts = 0).
cudaError_t ko_launch_accum_reset(KoAccum *acc, int count, cudaStream_t stream);

// Batch internals (ko_batch.cpp).
ko_batch *ko_batch_build(const KoSet *const *sets, const int *levels, const int *lanes, const int *stack,
                         const int *shape, int nsets, int nbins, int run_limit, ko_status *err);
ko_status ko_batch_exec(ko_batch *b, ko_rank *out, uint64_t *hist, bool hist_dev, cudaStream_t st);
long long ko_batch_orders_impl(const ko_batch *b);
unsigned long long ko_batch_fallback(const ko_batch *b);
void ko_batch_free(ko_batch *b);

// Autotuner internals (ko_tune.cpp).
struct KoFastState;
struct KoChunk;
ko_status ko_tune_set(KoFastState *fs, const KoSet &h, const KoSet *d_set, KoAccum *d_acc,
                      const char *cache_path, cudaStream_t st, int *lanes_out, int *levels_out,
                      int *stack_out, int *shape_out, double *rate_out);
ko_status ko_tune_batch(const KoSet *const *hs, int nsets, const char *cache_path, cudaStream_t st,
                        int *lanes_out, int *levels_out, int *stack_out, int *shape_out);

// Surrogate model internals (ko_model.cpp).
ko_model *ko_model_new(uint64_t seed, ko_status *err);
ko_status ko_model_load(ko_model *md, const float *params);
ko_status ko_model_store(const ko_model *md, float *params);
void ko_model_free(ko_model *md);
ko_status ko_model_option(ko_model *md, int key, long long value);
ko_status ko_model_raw(ko_model *md, const float *x, const float *t, int B, float *y_out, float *grad_out,
                       float *loss_out, float lr, cudaStream_t st);
ko_status ko_model_train_sets(ko_model *md, const KoSet *const *hs, int nsets, long long pairs_per_set,
                              int steps, int batch, float lr, uint64_t seed, float *loss_curve, cudaStream_t st);
ko_status ko_model_propose_set(ko_model *md, const KoSet &h, long long n_cand, int top_k, uint64_t seed,
                               int32_t *best_order, int64_t *best_makespan, double *gpu_ms, cudaStream_t st);
ko_status ko_model_search_set(ko_model *md, const KoSet &h, long long n_cand, int top_k, int rounds, int beam,
                              uint64_t seed, int32_t *best_order, int64_t *best_makespan, double *gpu_ms,
                              cudaStream_t st);
ko_status ko_random_search_set(KoFastState *fs, const KoSet &h, long long n_orders, uint64_t seed,
                               int32_t *best_order, int64_t *best_makespan, double *gpu_ms, cudaStream_t st);
ko_status ko_model_features(const KoSet &h, const int8_t *orders, long long n, float *x_out, cudaStream_t st);

// Allocation-free evaluation (ko_sim_simple.cu): explicit device rows, scratch
// in a file-scope device array.
constexpr int KO_MAX_DEVICES = 64;
ko_status ko_noalloc_eval(const KoSet &h, const int8_t *d_orders, long long count, int64_t *d_out,
                          cudaStream_t st);
size_t ko_noalloc_scratch_bytes();

// Host-side Algorithm 1; returns the number of execution rounds.
int ko_heuristic_host(const KoSet &h, int32_t *order_out, bool per_block = false);
// Hardware validation (ko_hw.cu).
ko_hw *ko_hw_build(const ko_hw_kernel *ks, int n, ko_status *err);
void ko_hw_free(ko_hw *h);
ko_status ko_hw_regs_impl(int kind, int *regs);
ko_status ko_hw_limits_impl(int32_t *out);
ko_status ko_hw_time_impl(ko_hw *h, const int8_t *orders, long long count, int reps, float *ms_out);
ko_status ko_hw_time_grid_impl(ko_hw *h, int k, int blocks, int reps, float *ms_out);
ko_status ko_hw_trace_impl(ko_hw *h, const int8_t *ord, unsigned long long *rec_out, float *ms_out);
long long ko_hw_trace_blocks(const ko_hw *h);
ko_status ko_hw_int_peak_impl(int32_t turns, int64_t *lane_ops, float *ms_out);
ko_status ko_local_search_set(KoFastState *fs, const KoSet &h, const int32_t *start, bool moves, int max_iters,
                              int32_t *order_out, int64_t *makespan_out, int32_t *steps_out, int64_t *evals_out,
                              double *gpu_ms, cudaStream_t st);

// Host-side bounds; returns false if the upper bound overflows 62 bits.
bool ko_bounds_host(const KoSet &h, int64_t *lb, int64_t *ub);
