// stripe_kernel_et.cu -- the early-terminating instantiations of the striped
// DTW kernel (branch and bound, Sec. 2.4.1; GLOBAL end only).  A separate
// translation unit so that they compile in parallel with the others.
#include "stripe_kernel.cuh"

namespace ra {

template <int G, int HR>
static void *stripe_fn_et(bool smem_ring)
{
    return smem_ring ? (void *)dtw_stripe_kernel<G, HR, false, true, true>
                     : (void *)dtw_stripe_kernel<G, HR, false, false, true>;
}

void *pick_stripe_et(int G, int HR, bool smem_ring)
{
#define RA_PICK_ET(g, h)                                                                           \
    if (G == g && HR == h)                                                                         \
        return stripe_fn_et<g, h>(smem_ring);
    RA_PICK_ET(32, 16)
    RA_PICK_ET(16, 16)
    RA_PICK_ET(32, 24)
    RA_PICK_ET(16, 24)
    RA_PICK_ET(8, 24)
    RA_PICK_ET(4, 24)
    RA_PICK_ET(32, 8)
    RA_PICK_ET(16, 8)
    RA_PICK_ET(8, 8)
    RA_PICK_ET(4, 8)
#undef RA_PICK_ET
    return nullptr;
}

}  // namespace ra
