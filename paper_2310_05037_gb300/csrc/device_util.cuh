// device_util.cuh -- small device helpers shared by the kernels of librawalign_dtw.
#pragma once

#include <cstdint>

namespace ra {

// min of three floats in one instruction (PTX min.f32 with three sources,
// sm_100 and later); exact, so the result is the plain minimum.
static __device__ __forceinline__ float min3f(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Order-preserving key: larger score first, then smaller candidate index.
static __device__ __forceinline__ unsigned long long best_key(float score, int cand)
{
    unsigned u = __float_as_uint(score);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)cand);
}

static __device__ __forceinline__ float key_score(unsigned long long key)
{
    unsigned u = (unsigned)(key >> 32);
    u = (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u;
    return __uint_as_float(u);
}

static __device__ __forceinline__ void floordivmod(long long x, long long d, long long &q, long long &r)
{
    q = x / d;
    r = x - q * d;
    if (r < 0) {
        q -= 1;
        r += d;
    }
}

// Programmatic dependent launch (sm_90 and later).  pdl_allow_next lets the
// next kernel of the stream, when it is launched as a programmatic
// dependent, start its blocks as soon as SM slots free up; every block calls
// it first, so all blocks of this grid are resident by then.  pdl_wait_prev
// waits until the previous kernel of the stream has completed; a grid whose
// block 0 calls it before exiting completes after its predecessor, so the
// completion of the last kernel of a chain implies that of all of them.
// Both do nothing in a kernel that was not launched as a dependent.
static __device__ __forceinline__ void pdl_allow_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
static __device__ __forceinline__ void pdl_wait_prev() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

}  // namespace ra
