// Run-length, prefix-sharing simulator: not built yet, always defers.
#include "ko_fast.h"

ko_status ko_fast_exhaustive(KoFastState *, const KoSet &, const KoSet *, int64_t *, KoAccum *,
                             cudaStream_t)
{
    return 1;
}

ko_status ko_fast_eval_idx(KoFastState *, const KoSet &, const KoSet *, const uint64_t *, int64_t,
                           int64_t *, cudaStream_t)
{
    return 1;
}

void ko_fast_release(KoFastState *fs)
{
    cudaFree(fs->buf);
    fs->buf = nullptr;
    fs->cap = 0;
}
