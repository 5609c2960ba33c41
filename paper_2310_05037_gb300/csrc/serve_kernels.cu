// serve_kernels.cu -- the device side of a serving flush's planning: the
// records of newly admitted candidates go to their reads' arena blocks, then
// one block per chunk builds the work record of each of the chunk's pieces
// (serve_piece) and advances each candidate's frontier state past the chunk.
#include "serve_expand.cuh"

namespace ra {

__global__ void serve_init_kernel(char *arena, const uint64_t *off, const ServeCandDev *recs, int n)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n)
        *(ServeCandDev *)(arena + off[x]) = recs[x];
}

__global__ void __launch_bounds__(64) serve_expand_kernel(const ServeChunkDev *chunks, char *arena,
                                                          const int *cls_map, const int *cls_base, int *cls_fill,
                                                          WorkDesc *work, int *read_of)
{
    const uint32_t c = blockIdx.x;
    const ServeChunkDev ch = chunks[c];
    ServeCandDev *recs = (ServeCandDev *)(arena + ch.cand_off);
    for (uint32_t k = threadIdx.x; k < ch.n_cands; k += blockDim.x) {
        ServeCandDev s = recs[k];
        WorkDesc wd{};
        serve_piece(ch, c, k, s, wd);
        // the order inside a class follows arrival; each piece's result does
        // not depend on where it sits in the queue
        const int q = cls_map[s.cls];
        const int slot = cls_base[q] + atomicAdd(cls_fill + q, 1);
        work[slot] = wd;
        read_of[ch.first_piece + k] = (int)c;
        recs[k] = s;
    }
}

cudaError_t launch_serve_init(char *arena, const uint64_t *off, const ServeCandDev *recs, int n, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    serve_init_kernel<<<(n + 127) / 128, 128, 0, s>>>(arena, off, recs, n);
    return cudaGetLastError();
}

cudaError_t launch_serve_expand(const ServeChunkDev *chunks, int n_chunks, char *arena, const int *cls_map,
                                const int *cls_base, int *cls_fill, WorkDesc *work, int *read_of, cudaStream_t s)
{
    if (n_chunks <= 0)
        return cudaSuccess;
    serve_expand_kernel<<<n_chunks, 64, 0, s>>>(chunks, arena, cls_map, cls_base, cls_fill, work, read_of);
    return cudaGetLastError();
}

}  // namespace ra
