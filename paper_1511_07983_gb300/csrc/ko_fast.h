// Run-length, prefix-sharing simulator (see ko_fast.cu).
#pragma once

#include "ko_internal.h"

// Device buffers the run-length simulator keeps between calls.
struct KoFastState {
    void *buf = nullptr;   // work counter, abandoned-item list
    size_t cap = 0;
    unsigned long long last_overflow = 0;  // items the last launch handed to the simple simulator
    int lanes = 32;                        // lanes per simulation (16 or 32)
    int levels = 4;                        // saved DFS levels (items fix N - 1 - levels kernels)
    bool disabled = false;                 // use the simple simulator only
    int run_limit = 32;                    // cap on runs per simulation (tests force overflow)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the last fast-kernel launch
    double last_ms = -1.0;
    long long h2d = 0, d2h = 0;            // bytes copied by the fast path
};

// Makespans of all N! orders into d_out (if non-null) and the accumulators.
// Returns KO_OK, a negative ko_status, or 1 when this simulator does not apply
// to the set (the caller then uses the simple simulator).
ko_status ko_fast_exhaustive(KoFastState *fs, const KoSet &h, const KoSet *d_set, int64_t *d_out,
                             KoAccum *d_acc, cudaStream_t st);

// Makespans of `count` orders given by Lehmer index; same return convention.
ko_status ko_fast_eval_idx(KoFastState *fs, const KoSet &h, const KoSet *d_set,
                           const uint64_t *d_idx, int64_t count, int64_t *d_out, cudaStream_t st);

void ko_fast_release(KoFastState *fs);
