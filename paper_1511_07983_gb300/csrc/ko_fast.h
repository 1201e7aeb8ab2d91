// Work lists of the run-length, prefix-sharing simulator (ko_fast.cu) and of
// its device-side fallback (ko_sim_simple.cu).
#pragma once

#include "ko_internal.h"

// A contiguous range of work items that belong to one set.
struct KoChunk {
    long long first;     // global index of the chunk's first item (chunks sorted by first)
    long long count;     // number of items
    int set;             // index into KoWork::sets / refs / accs
    int d0;              // mode 0: kernels fixed by an item's prefix
    int mode;            // 0 = exhaustive prefixes, 1 = Lehmer index list, 2 = explicit rows
    int pad;
    long long list_off;  // mode 0: item offset of the first item in the set's space (its first
                         // order is Lehmer index list_off * (N - d0)!); mode 1: entry of idx for
                         // the first item; mode 2: byte offset of its row
    long long out_off;   // added to the output position (mode 0: Lehmer index; 1/2: item)
};

// Parameters of one simulator launch (passed by value to the kernels).
struct KoWork {
    const KoSet *sets;
    const KoChunk *chunks;
    int nchunks;
    long long n_items;
    long long *refs;                  // per-set reference makespan, or null (use KoSet::ref_makespan)
    KoAccum *accs;                    // per-set accumulators, or null
    const uint64_t *idx;              // mode 1 entries
    const int8_t *perms;              // mode 2 rows
    int perm_stride;                  // bytes between mode-2 rows (0: N of the row's set)
    int64_t *out;                     // makespans, or null
    unsigned long long *counter;      // next work item
    unsigned long long *ov_count;     // items abandoned by the run-length simulator
    unsigned long long *ov_list;      // their global item indices
    unsigned long long ov_cap;
    unsigned long long *fb_counter;   // next abandoned item for the fallback
    const unsigned long long *item_list;   // non-null: work items are item_list[0 .. *item_count)
    const unsigned long long *item_count;
    int levels;                       // saved DFS levels per segment
    int run_limit;                    // runs one simulation may hold
    int *gstack;                      // non-null: DFS node states in this global slab, not shared memory
    long long gstack_words;           // words of gstack (bounds the segments that may use it)
    long long reserve_items;          // sizing only: abandoned-item lists for this many items
};

// Device-side state of the run-length simulator, owned by a handle or batch.
struct KoFastState {
    void *buf = nullptr;        // counters and the two passes' abandoned-item lists
    size_t cap = 0;
    unsigned long long ov_cap = 0;  // entries of each abandoned-item list
    void *fb_scratch = nullptr; // fallback slabs
    size_t fb_bytes = 0;
    unsigned long long last_overflow = 0;
    int lanes = 16;             // lanes per simulation: 1 (one thread per order, then the run-length
                                // passes over what it abandons), 16 or 32
    int levels = 4;             // saved DFS levels (items fix N - 1 - levels kernels)
    bool disabled = false;      // use the simple simulator only
    int run_limit = 32;         // cap on runs per simulation (tests force the hand-over)
    int stack_global = 1;       // DFS node states in global memory (1) or shared memory (0)
    int lane_shape = 0;         // one-thread pass state: 0 = 14 runs / 56 group slots, 1 = 12 / 40, 2 = 10 / 32
    void *gstack = nullptr;     // global slab for node states
    size_t gstack_bytes = 0;
    void *lslab = nullptr;      // node-state slab of the one-thread-per-order pass
    size_t lslab_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the last run-length launch
    double last_ms = -1.0;
    long long h2d = 0, d2h = 0;
};

// True when the run-length simulator applies to the set (every possible block
// duration below 2^31, so 32-bit modular end times are exact).
bool ko_fast_applicable(const KoSet &h);

// Prefix depth for exhaustive work items of an n-kernel set.
int ko_fast_d0(const KoFastState &fs, int n);

// Enqueue one run-length launch over `w` (counters reset here) followed by the
// device-side fallback for abandoned items.  Fills the counter fields of w.
// Asynchronous, graph-capturable (no host synchronisation) once an earlier
// launch outside capture has sized the buffers: each abandoned-item list holds
// max(w.n_items, w.reserve_items) entries, so no abandoned item is ever lost
// (a pass abandons an item at most once).
ko_status ko_fast_launch(KoFastState *fs, KoWork w, size_t max_slab_bytes, cudaStream_t st);

// One-thread-per-order pass (ko_lane.cu) over the items of `w` (counters and
// the abandoned-item list already set; w.gstack = its node-state slab of
// ko_lane_slab_bytes(w.levels, shape) bytes); shape as KoFastState::lane_shape.
cudaError_t ko_launch_lane(const KoWork &w, int shape, cudaStream_t st);
size_t ko_lane_slab_bytes(int levels, int shape);

// Device address of the count of items the first pass of the last launch
// abandoned (followed by the count the wide second pass abandoned).
const unsigned long long *ko_fast_overflow_counter(const KoFastState *fs);

void ko_fast_release(KoFastState *fs);

// Fallback: re-run the abandoned items of `w` with the simple simulator.
cudaError_t ko_launch_fallback(const KoWork &w, void *scratch, size_t scratch_bytes,
                               size_t per_thread, cudaStream_t st);

// Bytes of one simple-simulator slab for a set.
size_t ko_slab_bytes(int S, int Bk);
