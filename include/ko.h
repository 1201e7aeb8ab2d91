/*
 * ko.h -- C ABI of libko, a GB300 (sm_103a) engine that scores kernel launch
 * orders by makespan over the whole permutation space of a set of independent
 * kernels, each launched on its own stream.
 *
 * Method: Li, Narayana, El-Ghazawi, "Reordering GPU Kernel Launches to Enable
 * Efficient Concurrent Execution" (arXiv 1511.07983).
 *   - GPU / kernel parameters: Table 1.
 *   - Dispatch rule: Sec. 2 -- all thread blocks of the earliest-issued kernel
 *     are placed before any block of the next one, round-robin over SMs, until
 *     one of the four SM limits (registers, shared memory, warps, blocks) is
 *     met; blocks that do not fit wait for a later execution round.
 *   - Compute/memory balance R_B: Sec. 4.
 *   - Launch-order heuristic: Algorithm 1 (ScoreGen, ProfileCombine).
 *   - Evaluation over all permutations, percentile rank, speedup over worst,
 *     deviation from optimal: Sec. 6 and Table 3.
 *
 * The paper measures each order on hardware; this library replaces the
 * measurement with an integer discrete-event model.  A block of kernel i that
 * starts in a dispatch burst on an SM whose resident blocks (after the burst)
 * sum to SumC compute and SumM memory cycles runs for
 *     d = max( ceil(c_i * max(SumC, Ccap) / Ccap), ceil(m_i * max(SumM, Mcap) / Mcap) )
 * cycles, so R_B = Ccap / Mcap.  The round-robin pointer persists across
 * bursts; the queue is strict FIFO (no overtaking); all blocks ending at the
 * same time are released before the next burst.
 *
 * Conventions
 *   - Every call returns a ko_status (0 = KO_OK, negative = error) unless
 *     stated otherwise; ko_last_error() returns the last error of the calling
 *     thread and ko_status_str() names it.
 *   - A handle (ko_gpu) owns copies of all its inputs and the device scratch
 *     it allocates; output buffers belong to the caller.  One handle per host
 *     thread; distinct handles are independent.
 *   - Pointer arguments documented "host or device" are classified with
 *     cudaPointerGetAttributes; host buffers are staged through the handle's
 *     device scratch and copied back before the call returns.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls that
 *     return host results synchronise that stream before returning.
 *   - Lehmer indices are lexicographic: index 0 is the order 0,1,...,N-1 and
 *     index N!-1 is N-1,...,0.
 */
#ifndef KO_H
#define KO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ko_status;

#define KO_OK 0
#define KO_ERR_ARG (-1)       /* NULL handle, non-positive or out-of-range field, N > 24 */
#define KO_ERR_NOFIT (-2)     /* a block of some kernel exceeds an empty SM */
#define KO_ERR_TOO_LARGE (-3) /* exhaustive scoring asked for N > 12 */
#define KO_ERR_OVERFLOW (-4)  /* makespan upper bound does not fit 62 bits */
#define KO_ERR_CUDA (-5)      /* a CUDA runtime call failed */
#define KO_ERR_TIMEOUT (-6)   /* a bounded device wait gave up */
#define KO_ERR_STATE (-7)     /* call not valid in the handle's current state */
#define KO_ERR_NOMEM (-8)     /* device or host allocation failed */

/* Limits accepted by ko_create_gpu / ko_add_kernel. */
#define KO_MAX_KERNELS 24
#define KO_MAX_EXHAUSTIVE 12
#define KO_MAX_SM 1024
#define KO_MAX_BLK_SM 32
#define KO_MAX_CYCLES (1 << 24)

typedef struct ko_gpu ko_gpu;

/* Exhaustive statistics of one set (Table 3 columns, Sec. 6).
 *   min / max            best and worst makespan over all N! orders
 *   makespan             makespan of the ranked order
 *   n_better/equal/worse orders strictly faster / equal / strictly slower
 *   percentile           100 * (n_worse + n_equal) / N!   (share of orders that
 *                        are at least as slow as the ranked one)
 *   percentile_strict    100 * n_worse / N!
 *   speedup_over_worst   max / makespan
 *   deviation_from_optimal (makespan - min) / min                          */
typedef struct {
    int64_t min, max, makespan;
    uint64_t n_total, n_better, n_equal, n_worse;
    double percentile, percentile_strict, speedup_over_worst, deviation_from_optimal;
} ko_rank;

/* Create a simulated GPU (Table 1, first three rows): number of SMs and the
 * per-SM register, shared-memory (bytes), warp and block limits.  Ranges:
 * n_sm 1..1024, n_blk_sm 1..32, the others 1..2^24.  Capacities default to
 * Ccap = Mcap = 32768 (R_B = 1).  Returns NULL on a bad argument
 * (ko_last_error() says why).  The handle must be released with
 * ko_destroy_gpu. */
ko_gpu *ko_create_gpu(int32_t n_sm, int32_t n_reg_sm, int32_t n_shm_sm, int32_t n_warp_sm,
                      int32_t n_blk_sm);

/* Per-SM compute and memory capacities (cycles of demand served per cycle);
 * R_B = c_cap / m_cap (Sec. 4).  Both in 1..2^30.  KO_ERR_STATE after the
 * first evaluation. */
ko_status ko_set_capacity(ko_gpu *g, int64_t c_cap, int64_t m_cap);

/* When a started block's duration is fixed (the duration rule's SumC / SumM
 * are sampled):
 *   KO_SAMPLE_BURST_END     after the dispatch burst that started it, over
 *                           everything then resident on its SM (default);
 *   KO_SAMPLE_AT_PLACEMENT  when it is placed, over the blocks resident at
 *                           that moment, itself included and blocks placed
 *                           later in the same burst excluded.
 * Sec. 2 and Sec. 4 do not say which; the second is a model variant for
 * robustness checks of rankings.  It runs on the general simulator only:
 * ko_eval_orders, ko_eval_all, ko_rank_order and ko_eval_orders_noalloc
 * accept it; batches, the autotuner's fast path, local search and the
 * surrogate calls return KO_ERR_ARG for such a handle.  KO_ERR_ARG for another
 * value, KO_ERR_STATE after the first evaluation. */
#define KO_SAMPLE_BURST_END 0
#define KO_SAMPLE_AT_PLACEMENT 1
ko_status ko_set_sampling(ko_gpu *g, int32_t mode);

/* Append kernel i (Table 1, last three rows), all quantities per thread
 * block: n_reg_i = registers of one block (regs/thread x threads), n_shm_i =
 * shared-memory bytes of one block, n_warp_i = warps of one block,
 * n_tblk_i = number of blocks, c_i / m_i = compute / memory cycles one block
 * needs when running alone (R_i = c_i / m_i).  n_reg_i, n_warp_i, n_tblk_i,
 * c_i, m_i must be >= 1 (n_tblk_i <= 2^20, c_i and m_i <= 2^24), n_shm_i >= 0.
 * Returns the kernel id (0, 1, ...) or a negative ko_status; KO_ERR_NOFIT if
 * one block cannot fit an empty SM, KO_ERR_STATE after the first evaluation. */
int32_t ko_add_kernel(ko_gpu *g, int32_t n_reg_i, int32_t n_shm_i, int32_t n_warp_i,
                      int32_t n_tblk_i, int64_t c_i, int64_t m_i);

/* Number of kernels added so far (>= 0), or KO_ERR_ARG for a NULL handle. */
int32_t ko_num_kernels(const ko_gpu *g);

/* Work/capacity lower bound and serial upper bound on the makespan of any
 * order.  lb = max(longest alone-duration, per-limit area bounds); ub = sum of
 * all blocks' durations with SumC, SumM at N_blk_SM times the largest c, m.
 * Host-only; KO_ERR_OVERFLOW if ub needs more than 62 bits. */
ko_status ko_bounds(ko_gpu *g, int64_t *lb, int64_t *ub);

/* Algorithm 1 (ScoreGen / ProfileCombine, execution rounds), run on the host.
 * Writes N kernel ids to order_out (host memory).  Resource terms use each
 * kernel's per-SM footprint ceil(N_tblk / N_SM) x (regs, smem, warps, 1);
 * R_i = c_i / m_i, R_B = Ccap / Mcap, R_comb = sum(N_tblk c) / sum(N_tblk m). */
ko_status ko_heuristic_order(ko_gpu *g, int32_t *order_out);

/* Algorithm 1 under a chosen reading of its resource terms (Sec. 5, the
 * ScoreGen resource fractions and the "fits within an execution round" test):
 *   KO_HEUR_PER_SM     per-SM footprints ceil(N_tblk / N_SM) x (regs, smem,
 *                      warps, 1) -- what ko_heuristic_order uses;
 *   KO_HEUR_PER_BLOCK  one block's (regs, smem, warps, 1).
 * Writes N kernel ids to order_out (host).  KO_ERR_ARG for another value. */
#define KO_HEUR_PER_SM 0
#define KO_HEUR_PER_BLOCK 1
ko_status ko_heuristic_order_ex(ko_gpu *g, int32_t reading, int32_t *order_out);

/* Makespans of n launch orders, written to makespan_out[n] (host or device).
 * Exactly one of idx / orders is non-NULL:
 *   idx     n Lehmer indices in [0, N!)   (N <= 20), host or device;
 *   orders  n x N kernel ids, row-major, each row a permutation, host or device.
 * A row that is not a permutation of 0..N-1 (or an index >= N!) yields
 * makespan -1.  Asynchronous on `stream` when the input and makespan_out are
 * both device pointers; a host buffer on either side makes the call
 * synchronise `stream` before returning. */
ko_status ko_eval_orders(ko_gpu *g, const uint64_t *idx, const int8_t *orders, int64_t n,
                         int64_t *makespan_out, void *stream);

/* Makespans of n explicit orders (n x N kernel ids, host or device) under the
 * processor-sharing model variant: the same dispatch (Sec. 2), but every
 * resident block progresses its remaining compute and memory work at the rates
 * its SM's current totals allow, Ccap / max(SumC, Ccap) and
 * Mcap / max(SumM, Mcap), re-evaluated whenever the SM's residents change; a
 * block ends when both are done.  With residents that never change this is the
 * duration rule without rounding up.  Times are doubles computed in a fixed
 * operation order without contraction.  makespan_out[n] (host or device)
 * receives them, -1 for a row that is not a permutation.  Ignores
 * ko_set_sampling.  Synchronises `stream` when a buffer is on the host. */
ko_status ko_eval_orders_ps(ko_gpu *g, const int8_t *orders, int64_t n, double *makespan_out, void *stream);

/* Exhaustive scoring of all N! orders (N <= 12, else KO_ERR_TOO_LARGE) and the
 * rank of one order among them.  `order` (host, N ids) is ranked; NULL ranks
 * the Algorithm 1 order.  If hist != NULL (host or device, nbins >= 1
 * entries) it receives the histogram with
 *     bin = floor((M - min) * nbins / (max - min + 1)).
 * Synchronises `stream`; `out` is host memory.  The handle keeps the N!
 * makespans on the device (8 bytes per order) for the histogram, and 16 bytes
 * per work item for the lists that carry abandoned items between passes. */
ko_status ko_rank_order(ko_gpu *g, const int32_t *order, ko_rank *out, uint64_t *hist,
                        int32_t nbins, void *stream);

/* Makespans of all N! orders in Lehmer-index order into makespans_out[N!]
 * (device memory), N <= 12.  Asynchronous on `stream`; the handle holds 16
 * bytes of device memory per work item (N! / (levels + 1)! items) for the
 * lists that carry abandoned items between passes. */
ko_status ko_eval_all(ko_gpu *g, int64_t *makespans_out, void *stream);

/* Tuning knobs of the device simulators (set by the tuner; per handle).
 *   KO_OPT_LANES        threads per simulation: 1 = one thread per order,
 *                       its state in shared memory, followed by the
 *                       run-length passes for the work items it cannot hold;
 *                       16 or 32 = lanes sharing one run-length simulation,
 *                       its state packed in registers (default 16)
 *   KO_OPT_LEVELS       prefix-sharing depth: exhaustive work items fix the
 *                       first N-1-levels kernels and walk the rest depth
 *                       first, saving `levels` states; 0..6 (default 4)
 *   KO_OPT_SIMPLE_ONLY  1 = use only the simple one-thread-per-order
 *                       simulator, 0 = run-length simulator where it applies
 *   KO_OPT_STACK_GLOBAL 1 = keep saved DFS node states in a global-memory
 *                       slab (cached in L2/L1) instead of shared memory,
 *                       which frees shared memory for occupancy and L1 for
 *                       register spills (default 1); 0 = shared memory
 *   KO_OPT_RUN_LIMIT    most runs of distinct SM states one simulation may
 *                       hold before its work item moves to the simple
 *                       simulator, 1..32 (default 32; small values exercise
 *                       that hand-over)
 *   KO_OPT_LANE_STATE   state size of the one-thread-per-order simulator
 *                       (KO_OPT_LANES = 1): 0 = 14 runs and 56 group slots
 *                       (288 simulations per SM, default), 1 = 12 runs and
 *                       40 slots (352), 2 = 10 runs and 32 slots (448).
 *                       Smaller states fit more simulations on an SM; work
 *                       items that need more move on to the run-length passes.
 *                       A launch with fewer work items than SMs x those
 *                       simulations runs in 64-thread blocks spread over
 *                       every SM instead (one item per thread)
 * Results never depend on these knobs.  KO_ERR_ARG for an unknown key or
 * value. */
#define KO_OPT_LANES 1
#define KO_OPT_LEVELS 2
#define KO_OPT_SIMPLE_ONLY 3
#define KO_OPT_RUN_LIMIT 4
#define KO_OPT_STACK_GLOBAL 5
#define KO_OPT_LANE_STATE 6
ko_status ko_set_option(ko_gpu *g, int32_t key, int64_t value);

/* Current value of a tuning knob (KO_OPT_*), or KO_ERR_ARG. */
int64_t ko_get_option(const ko_gpu *g, int32_t key);

/* Autotuner: times the exhaustive simulators on a calibration slice of this
 * set's exhaustive space (the whole space up to 64M orders, else 64M orders in
 * 16 evenly spread ranges) for every candidate -- 1, 16 or 32 threads per
 * simulation; for 1, the three state sizes of KO_OPT_LANE_STATE; for 16 and
 * 32, saved DFS node states in a global slab or in shared memory;
 * 1..min(N-1, 5) saved DFS levels -- keeps the fastest and sets
 * KO_OPT_LANES / KO_OPT_LEVELS / KO_OPT_STACK_GLOBAL / KO_OPT_LANE_STATE on
 * the handle.  With
 * cache_path (nullable) the choice is looked up first and stored after, keyed
 * by (N_SM class, N), in a small JSON file.  Synchronises `stream`; results
 * never depend on the choice.  N <= 12. */
ko_status ko_autotune(ko_gpu *g, const char *cache_path, void *stream);

/* Autotuner for a batch of handles (call before ko_batch_create): groups the
 * sets by (N_SM class, N); for every class with at least 2^21 orders in the
 * batch it runs up to 64 of the class's own sets (the first ones, until 2^22
 * orders) together as one exhaustive launch per candidate (the candidates of
 * ko_autotune) and keeps the fastest, so small sets are timed as a batch runs
 * them; smaller classes keep 16 lanes, a global slab and min(N-1, 4) levels.
 * Sets every handle's KO_OPT_LANES / KO_OPT_LEVELS / KO_OPT_STACK_GLOBAL /
 * KO_OPT_LANE_STATE.  With
 * cache_path (nullable) each class's choice is looked up first and stored
 * after (keys "B_S<class>_N<n>").  KO_ERR_TOO_LARGE for N > 12,
 * KO_ERR_OVERFLOW for a set whose durations reach 2^31 cycles.  Synchronises
 * `stream`; results never depend on the choice. */
ko_status ko_batch_autotune(ko_gpu *const *sets, int32_t nsets, const char *cache_path, void *stream);

/* Work items the last exhaustive or index-list call moved from the
 * run-length simulator to its wider second pass (a simulation needed more runs
 * of distinct SM states than lanes, or more than 8 resident groups in a run;
 * what that pass cannot finish goes to the simple simulator); -1 for a NULL
 * handle.  Informational: results are exact either way, because the lists
 * that carry abandoned items between the passes hold every item of the call
 * (device memory: 16 bytes per work item, allocated by the call). */
int64_t ko_last_fallback_items(const ko_gpu *g);

/* Number of CUDA kernels this library has launched in this process (all
 * handles, all threads).  Diagnostic counter for benchmarks. */
int64_t ko_kernel_launches(void);

/* Device time in milliseconds of the last run-length simulator launch on this
 * handle, measured with CUDA events recorded on the launching stream around
 * that launch; -1 if none. */
double ko_last_sim_ms(const ko_gpu *g);

/* Bytes this handle has copied host->device and device->host since it was
 * created (inputs, staged buffers, results).  KO_ERR_ARG on NULL arguments. */
ko_status ko_transfer_bytes(const ko_gpu *g, int64_t *h2d, int64_t *d2h);

/* ---------------------------------------------------------------- batches
 * Many independent sets scored in one persistent launch (the exhaustive
 * evaluation of Sec. 6 repeated over a population of kernel sets).
 *
 * ko_batch_create snapshots nsets handles (kernels, limits, capacities, each
 * handle's KO_OPT_LEVELS, KO_OPT_LANES, KO_OPT_STACK_GLOBAL and
 * KO_OPT_LANE_STATE -- sets that share lanes, node-state placement and state
 * size run in one launch, one launch per such group -- and KO_OPT_RUN_LIMIT
 * of the first handle), computes
 * each set's Algorithm 1 order on the host, lays out one work list over all
 * sets (largest sets first) and captures the whole evaluation -- reset,
 * ranked-order makespans, all N! orders of every set, optional per-set
 * histograms, copy-out -- as one CUDA graph.  Every set needs 1 <= N <= 12
 * (KO_ERR_TOO_LARGE above) and durations below 2^31 cycles (KO_ERR_OVERFLOW).
 * nbins = 0 skips histograms (and the per-set makespan storage, 8 bytes per
 * order); 1..32768 keeps them.  Returns NULL on error (ko_last_error()).
 * The batch owns its device memory; the handles may be destroyed afterwards. */
typedef struct ko_batch ko_batch;
ko_batch *ko_batch_create(ko_gpu *const *sets, int32_t nsets, int32_t nbins);

/* Launch the captured graph on `stream` and wait for it.  out[i] (host,
 * nsets entries) receives set i's statistics and the rank of its Algorithm 1
 * order (ko_rank fields as in ko_rank_order).  hist (host or device,
 * nsets x nbins, row i = set i) may be NULL. */
ko_status ko_batch_run(ko_batch *b, ko_rank *out, uint64_t *hist, void *stream);

/* Total number of orders one ko_batch_run evaluates (sum of N_i!), or -1. */
int64_t ko_batch_orders(const ko_batch *b);

/* Work items of the last run that moved to the wide pass (diagnostic), or -1. */
int64_t ko_batch_fallback_items(const ko_batch *b);

void ko_batch_destroy(ko_batch *b);

/* -------------------------------------------------------------- surrogate
 * Not part of the paper.  For sets too large to enumerate (N = 16..24), a
 * small MLP predicts log2(makespan / lower bound) of an order from
 * position-ordered kernel descriptors; it is trained on orders the exact
 * simulator labels, proposes the best-predicted of many random candidates,
 * and every proposal is rescored exactly, so every reported makespan is the
 * simulator's.
 *
 * Network: 192 inputs -> 256 -> 256 -> 256 -> 1, ReLU, BF16 weights and
 * activations, FP32 accumulation on tensor cores; MSE loss; Adam
 * (beta 0.9 / 0.999, eps 1e-8) on FP32 master weights.
 * Inputs: 24 position slots x 7 features (regs/N_reg_SM, smem/N_shm_SM,
 * warps/N_warp_SM, ceil(N_tblk/N_SM)/N_blk_SM, log2(c)/16, log2(m)/16,
 * present) + 8 globals (N/24, N_SM/148, log2 of the four limits / 24,
 * log2(lower bound)/32, 1) + 16 zeros; the kernel at position p of an N-kernel
 * order goes to slot round(23 p / (N-1)).
 * Parameters (KO_MODEL_PARAMS floats, host order): W1 [192 x 256] (input-
 * major), b1 [256], W2 [256 x 256], b2, W3 [256 x 256], b3, w4 [256], b4. */
#define KO_MODEL_PARAMS 181249
typedef struct ko_model ko_model;

/* He-normal initial weights from a counter-based SplitMix64 stream. */
ko_model *ko_model_create(uint64_t seed);
ko_status ko_model_get_params(const ko_model *m, float *params);   /* host out */
ko_status ko_model_set_params(ko_model *m, const float *params);   /* host in; resets Adam */

/* Raw-feature entry points (B % 64 == 0, B >= 64; x host [B x 192], values
 * rounded to BF16 on upload; t host [B]).  ko_model_predict writes y [B];
 * ko_model_grad also writes the FP32 gradient of the mean squared error
 * (KO_MODEL_PARAMS floats, host) and the loss; ko_model_train_step does the
 * same and then one Adam step with learning rate lr. */
ko_status ko_model_predict(ko_model *m, const float *x, int64_t B, float *y, void *stream);
ko_status ko_model_grad(ko_model *m, const float *x, const float *t, int64_t B, float *grad,
                        float *loss, void *stream);
ko_status ko_model_train_step(ko_model *m, const float *x, const float *t, int64_t B, float lr,
                              float *loss, void *stream);

/* Encoder output for n explicit orders (host, n x N ids) of a set: host
 * x_out [n x 192] (BF16 values as floats). */
ko_status ko_model_encode(ko_gpu *g, const int8_t *orders, int64_t n, float *x_out, void *stream);

/* Train on simulator-labelled pairs: for each of nsets sets, pairs_per_set
 * uniform random orders (device RNG from `seed`) labelled exactly; then
 * `steps` Adam steps on random minibatches of `batch` (multiple of 64) pairs.
 * loss_curve (host, nullable) receives the mean loss of every step. */
ko_status ko_surrogate_train(ko_model *m, ko_gpu *const *sets, int32_t nsets, int64_t pairs_per_set,
                             int32_t steps, int32_t batch, float lr, uint64_t seed,
                             float *loss_curve, void *stream);

/* Propose an order for a set of any N <= 24: draw n_cand uniform random
 * candidates, score them with the network, keep the top_k best predicted,
 * rescore those exactly and return the best (best_order: host, N ids).
 * gpu_ms (nullable) receives the device time of the whole proposal. */
ko_status ko_surrogate_propose(ko_model *m, ko_gpu *g, int64_t n_cand, int32_t top_k, uint64_t seed,
                               int32_t *best_order, int64_t *best_makespan, double *gpu_ms,
                               void *stream);

/* Surrogate-guided local search for a set with 2 <= N <= 24.  Screening as
 * in ko_surrogate_propose (n_cand candidates, top_k rescored exactly) seeds a
 * beam of the `beam` (1..64) best exact orders; each of `rounds` (0..1024)
 * rounds scores every swap of two positions and every move of one kernel to
 * another position of each beam order with the network, rescores the 256
 * best exactly and keeps the `beam` best distinct orders; then an exact
 * steepest descent from the best order found (KO_MODEL_OPT_POLISH steps at
 * most).  Returns the best exact order found (host, N ids); gpu_ms =
 * device-timeline duration of the whole search including the host's
 * per-round and per-step bookkeeping. */
ko_status ko_surrogate_search(ko_model *m, ko_gpu *g, int64_t n_cand, int32_t top_k, int32_t rounds,
                              int32_t beam, uint64_t seed, int32_t *best_order, int64_t *best_makespan,
                              double *gpu_ms, void *stream);

/* Plain random search, the baseline of the surrogate: n_orders uniform random
 * orders simulated exactly; the best one is returned.  Like the exact
 * rescoring of the surrogate calls and ko_local_search, it picks the threads
 * per simulation by list length and N_SM (32 for more than 32 SMs or up to
 * 4096 orders, 16 up to 32768, one thread per order beyond) instead of the
 * handle's KO_OPT_LANES, which ko_eval_orders and the exhaustive calls use. */
ko_status ko_random_search(ko_gpu *g, int64_t n_orders, uint64_t seed, int32_t *best_order,
                           int64_t *best_makespan, double *gpu_ms, void *stream);

/* Exact local search: steepest-descent hill climbing over launch orders, the
 * heuristic-then-improve step that Sec. 6's exhaustive measurement suggests
 * (the paper itself stops at Algorithm 1).  Starts from `start` (host, N ids;
 * NULL = the Algorithm 1 order).  Each step simulates every neighbour of the
 * current order exactly -- the N(N-1)/2 swaps of two positions, pairs (i, j),
 * i < j, in lexicographic order, then, if moves != 0, the N(N-1) moves of the
 * kernel at position `from` to position `to` (from-major, `to` ascending) --
 * and moves to the lowest makespan (lowest neighbour index among equals) only
 * if it is strictly lower.  Stops at a local optimum or after max_iters steps
 * (0..2^20).  Outputs (host): order_out[N], *makespan_out; steps_out,
 * evals_out (orders simulated, start included) and gpu_ms (elapsed time on
 * `stream`) are nullable.  Synchronises `stream`.  KO_ERR_ARG if start is not
 * a permutation; KO_ERR_OVERFLOW if the set exceeds the run-length
 * simulator's limits. */
ko_status ko_local_search(ko_gpu *g, const int32_t *start, int32_t moves, int32_t max_iters, int32_t *order_out,
                          int64_t *makespan_out, int32_t *steps_out, int64_t *evals_out, double *gpu_ms,
                          void *stream);

/* Model options.  KO_MODEL_OPT_TC: tensor-core path of the inference
 * forward (ko_model_predict, ko_surrogate_propose, ko_surrogate_search) --
 * 0 = warp-level mma.sync BF16 GEMMs, 1 = tcgen05 MMAs with TMEM
 * accumulators (default; used for batches that are multiples of 128, the
 * others fall back to mma.sync).  Both give the same bits.  A tcgen05 completion wait that
 * gives up makes the next call return KO_ERR_TIMEOUT.  KO_ERR_ARG for an
 * unknown key or value (below). */
#define KO_MODEL_OPT_TC 1
/* KO_MODEL_OPT_CHUNK: candidate rows per forward pass in ko_surrogate_propose
 * and ko_surrogate_search (a multiple of 1024 in [1024, 2^22], default 262144);
 * larger chunks amortise each layer's weight load over more row tiles and
 * hold chunk x 1 KB of activations.  Results do not depend on it. */
#define KO_MODEL_OPT_CHUNK 2
/* KO_MODEL_OPT_TC_TRAIN: training GEMMs (forward with transposed copies,
 * input and weight gradients) on tcgen05 (1, default; batches that are
 * multiples of 128, weight gradients of multiples of 256, split-K with a
 * fixed-order reduction) or on warp-level mma.sync (0).  The two paths
 * accumulate in different orders, so their gradients agree to rounding. */
#define KO_MODEL_OPT_TC_TRAIN 3
/* KO_MODEL_OPT_POLISH: after its rounds, ko_surrogate_search walks an exact
 * steepest descent (every swap and every single move simulated, as
 * ko_local_search does) from the best exact order it found, for at most this
 * many steps (0..2^20, default 64; 0 = none), inside its timed region.  The
 * network proposes; the simulator alone accepts. */
#define KO_MODEL_OPT_POLISH 4
ko_status ko_model_set_option(ko_model *m, int32_t key, int64_t value);

void ko_model_destroy(ko_model *m);

/* ------------------------------------------------ allocation-free evaluation
 * The paper has no counterpart to this entry point; it exists for callers of
 * this library that cannot allocate device memory: code running under a
 * memory manager that owns the whole device heap (a framework's caching
 * allocator that has reserved the GPU), or latency-critical code that must
 * not call cudaMalloc / cudaFree because those calls can synchronise the
 * device.  ko_eval_orders_noalloc computes what ko_eval_orders computes for
 * explicit rows (same makespans, -1 for a row that is not a permutation),
 * using the simple one-thread-per-order simulator, and allocates nothing: its
 * per-thread simulator state lives in a file-scope device array of 32 MiB
 * that every GPU which loads the library holds until the process exits.
 *   orders        n x N kernel ids (int8, row-major), device memory
 *   makespan_out  n int64, device memory
 * Host pointers are rejected (KO_ERR_ARG): staging them would need device
 * memory.  The array holds at least 128 threads' state, so a set whose
 * per-thread state, N_SM x (36 + 12 N_blk_SM) bytes rounded up to 256, exceeds
 * 262,144 bytes (for example N_SM > 624 at 32 blocks per SM) is rejected with
 * KO_ERR_TOO_LARGE.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The CUDA runtime reserves the array on a device
 * when it loads this library's device code there (by default at the
 * library's first use on that device), so make the library's first call on a
 * device before another allocator reserves that device's memory: if the
 * reservation fails, calls return KO_ERR_CUDA.  The address is kept per
 * device index for the life of the process; after cudaDeviceReset it is
 * stale, so do not call this entry point again on a device that was reset.
 * Every call shares the one array and uses it as
 * scratch only (nothing carries over between calls), so calls that overlap
 * on the GPU -- concurrent streams, or other host threads -- race on it:
 * serialise them.  Asynchronous on `stream`. */
ko_status ko_eval_orders_noalloc(const ko_gpu *g, const int8_t *orders, int64_t n,
                                 int64_t *makespan_out, void *stream);

/* ------------------------------------------------ hardware validation
 * Sec. 6 measures launch orders by running them on the GPU.  These calls do
 * that for synthetic busy kernels on the current device, so a kernel set's
 * measured times can be ranked against its simulated makespans (the
 * simulator's descriptor of this GPU and the kernels' per-block durations
 * are calibrated by the caller from ko_hw_time_grid).
 *
 * A busy kernel (ko_hw_kernel, host memory):
 *   kind     KO_HW_COMPUTE: every thread runs a dependent FMA chain of
 *            `iters` steps; KO_HW_MEMORY: every thread streams `iters` 16-byte
 *            loads from a 256 MB device buffer (addresses masked into it);
 *   threads  block size, a multiple of 32 in [32, 1024];
 *   smem     dynamic shared memory per block in bytes (reserved, not used;
 *            it sets occupancy), up to the device's opt-in limit;
 *   blocks   grid size in [1, 2^20];  iters  loop length in [0, 2^24].
 * Both loops have a fixed length and wait on nothing. */
#define KO_HW_COMPUTE 0
#define KO_HW_MEMORY 1
typedef struct {
    int32_t kind, threads, smem, blocks, iters;
} ko_hw_kernel;
typedef struct ko_hw ko_hw;

/* Copies n (1..8) kernel descriptions and creates n streams, events and the
 * 256 MB buffer on the current device.  NULL on error (ko_last_error():
 * KO_ERR_ARG for an invalid description, KO_ERR_NOMEM, KO_ERR_CUDA). */
ko_hw *ko_hw_create(const ko_hw_kernel *ks, int32_t n);

/* Limits of the current device as the simulator's GPU descriptor reads them:
 * out[0] N_SM, [1] registers per SM, [2] shared memory per SM (bytes), [3]
 * warps per SM, [4] resident blocks per SM, [5] shared memory the runtime
 * reserves per block (bytes), [6] SM clock (kHz). */
ko_status ko_hw_device_limits(int32_t out[7]);

/* Registers per thread of the busy kernel of `kind` (cudaFuncGetAttributes). */
ko_status ko_hw_regs(int32_t kind, int32_t *regs_per_thread);

/* Integer issue-rate microbenchmark (the denominator of the simulators'
 * integer roofline; not part of the paper).  Fills every SM of the current
 * device with 256-thread blocks whose threads each run 8 independent chains of
 * 32-bit add, xor and min (one instruction each, register operands only) for
 * `turns` (1..2^20) loop turns of 16 steps, and times the launch with CUDA
 * events on the legacy default stream (one warm-up launch, then the fastest of
 * three).  *lane_ops receives the thread-level integer operations one launch
 * executes (threads x turns x 384), *ms_out its time in milliseconds; the
 * rate is lane_ops / ms.  Allocates and frees a small device buffer;
 * synchronises the device's default stream. */
ko_status ko_hw_int_peak(int32_t turns, int64_t *lane_ops, float *ms_out);

/* Times `count` launch orders (host, count x n kernel ids, row-major): for
 * each order, `reps` runs (1..64) that launch kernel order[j] on stream j in
 * host order j = 0..n-1 between a start event and a stop event that waits for
 * every stream; ms_out[count] (host) gets the fastest run in milliseconds.
 * KO_ERR_ARG if a row is not a permutation.  Synchronous. */
ko_status ko_hw_time_orders(ko_hw *h, const int8_t *orders, int64_t count, int32_t reps, float *ms_out);

/* Fastest of `reps` runs of kernel k alone with a grid of `blocks` blocks
 * (calibration), in milliseconds.  Synchronous. */
ko_status ko_hw_time_grid(ko_hw *h, int32_t k, int32_t blocks, int32_t reps, float *ms_out);

/* One run of one launch order (host, n ids) with every block traced.
 * trace_out (host) receives 4 uint64 per block -- start and end time in ns of
 * the device's global timer, SM id, kernel id -- kernels in id order, each
 * kernel's blocks in index order: sum of the kernels' grids x 4 entries
 * (ko_hw_trace_len).  The start is stamped by the block's first thread on
 * entry, the end after all its threads are done.  *ms_out gets the run's
 * event time.  Synchronous. */
ko_status ko_hw_trace_order(ko_hw *h, const int8_t *order, uint64_t *trace_out, float *ms_out);
int64_t ko_hw_trace_len(const ko_hw *h);

/* Release streams, events and buffers.  NULL is ignored. */
void ko_hw_destroy(ko_hw *h);

/* Release the handle and its device scratch.  NULL is ignored. */
void ko_destroy_gpu(ko_gpu *g);

/* Name of a status code (static string). */
const char *ko_status_str(ko_status s);

/* Last error recorded on the calling thread (KO_OK if none). */
ko_status ko_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* KO_H */
