// stripe_kernel.cu -- instantiations of the striped DTW kernel (the template
// is in stripe_kernel.cuh) and its launchers.  The early-terminating
// instantiations live in stripe_kernel_et.cu so that the two sets compile in
// parallel.
#include <map>
#include <mutex>
#include <tuple>

#include "stripe_kernel.cuh"

namespace ra {

int stripe_max_blocks_uncached(int G, int HR, int block, size_t smem);

// ---------------------------------------------------------------------------
// variant table and launchers
// ---------------------------------------------------------------------------
template <int G, int HR, bool F>
static void *stripe_fn(bool smem_ring)
{
    return smem_ring ? (void *)dtw_stripe_kernel<G, HR, F, true, false>
                     : (void *)dtw_stripe_kernel<G, HR, F, false, false>;
}

static void *pick_stripe(int G, int HR, bool freeend, bool smem_ring)
{
#define RA_PICK(g, h)                                                                              \
    if (G == g && HR == h)                                                                         \
        return freeend ? stripe_fn<g, h, true>(smem_ring) : stripe_fn<g, h, false>(smem_ring);
    RA_PICK(32, 16)
    RA_PICK(16, 16)
    RA_PICK(32, 24)
    RA_PICK(16, 24)
    RA_PICK(8, 24)
    RA_PICK(4, 24)
    RA_PICK(32, 8)
    RA_PICK(16, 8)
    RA_PICK(8, 8)
    RA_PICK(4, 8)
#undef RA_PICK
    return nullptr;
}

// Resident blocks per SM of a variant (occupancy query, cached per device
// and shape: serving asks for it on every flush).
int stripe_max_blocks_per_sm(int G, int HR, int block, size_t smem)
{
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, size_t>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, G, HR, block, smem);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end())
            return it->second;
    }
    const int nb = stripe_max_blocks_uncached(G, HR, block, smem);
    if (nb > 0) {
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = nb;
    }
    return nb;
}

int stripe_max_blocks_uncached(int G, int HR, int block, size_t smem)
{
    void *fn = pick_stripe(G, HR, false, smem > 0);
    void *fn2 = pick_stripe(G, HR, true, smem > 0);
    if (!fn || !fn2)
        return 0;
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(fn2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, smem) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_stripe(int G, int HR, const StripeParams &p, int grid, int block, size_t smem,
                          cudaStream_t s, bool dependent)
{
    void *fn = p.early_term ? pick_stripe_et(G, HR, p.ring_in_smem != 0)
                            : pick_stripe(G, HR, p.end_free != 0, p.ring_in_smem != 0);
    if (!fn)
        return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
    }
    void *args[] = {(void *)&p};
    return launch_maybe_dependent(fn, grid, block, smem, s, args, dependent);
}

cudaError_t launch_maybe_dependent(const void *fn, int grid, int block, size_t smem, cudaStream_t s, void **args,
                                   bool dependent)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = dependent ? 1 : 0;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace ra
