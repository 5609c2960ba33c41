// serve.cu -- Read-Until serving entry points (filled in below).
#include "internal.cuh"

extern "C" int rawalign_dtw_submit_chunk(rawalign_dtw_t *, uint64_t, const float *, uint32_t,
                                         const rawalign_candidate_t *, uint32_t, int, uint64_t *)
{
    return RA_EINVAL;
}

extern "C" int rawalign_dtw_flush(rawalign_dtw_t *) { return RA_OK; }
