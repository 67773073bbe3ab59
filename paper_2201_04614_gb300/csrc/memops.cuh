// memops.cuh -- vector loads/stores used by the streaming kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace vsz {

// Streaming fp32x4 load: read-only path, no L1 allocation (each input byte
// is read once by the main pass).
__device__ __forceinline__ float4 ld_stream_f4(const float* p) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p));
    return v;
}

__device__ __forceinline__ uint2 ld_stream_u2(const void* p) {
    uint2 v;
    asm("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}

__device__ __forceinline__ uint4 ld_stream_u4(const void* p) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

// Load `valid` (0..4) floats starting at p; the rest read as 0.
__device__ __forceinline__ void load4f(const float* p, int valid, bool vec, float (&v)[4]) {
    if (vec) {
        const float4 f = ld_stream_f4(p);
        v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (k < valid) ? p[k] : 0.0f;
    }
}

// Store 4 uint16 codes packed as {c0 | c1<<16, c2 | c3<<16}; `valid` of them.
__device__ __forceinline__ void store4c(uint16_t* p, int valid, bool vec, uint32_t c01, uint32_t c23) {
    if (vec) {
        *reinterpret_cast<uint2*>(p) = make_uint2(c01, c23);
    } else {
        if (valid > 0) p[0] = (uint16_t)(c01 & 0xffffu);
        if (valid > 1) p[1] = (uint16_t)(c01 >> 16);
        if (valid > 2) p[2] = (uint16_t)(c23 & 0xffffu);
        if (valid > 3) p[3] = (uint16_t)(c23 >> 16);
    }
}

// Load 4 uint16 codes (valid of them; the rest read as 0).
__device__ __forceinline__ void load4c(const uint16_t* p, int valid, bool vec, uint32_t (&c)[4]) {
    if (vec) {
        const uint2 u = ld_stream_u2(p);
        c[0] = u.x & 0xffffu; c[1] = u.x >> 16; c[2] = u.y & 0xffffu; c[3] = u.y >> 16;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = (k < valid) ? (uint32_t)p[k] : 0u;
    }
}

// 16-byte store of a streamed output (written once, not read again by the
// kernel): evict-first when VSZ_STORE_CS is set, a plain store otherwise.
#ifndef VSZ_STORE_CS
#define VSZ_STORE_CS 1
#endif
__device__ __forceinline__ void st_out4(int4* p, int4 v) {
#if VSZ_STORE_CS
    __stcs(p, v);
#else
    *p = v;
#endif
}

}  // namespace vsz
