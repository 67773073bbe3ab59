// misc.cuh -- host launchers of the auxiliary kernels (k_misc.cu).
#pragma once
#include "common.cuh"

namespace vsz {

cudaError_t launch_begin(WsHeader* wsh, uint4* chunks, uint64_t nchunks, vsz_header* hdr, double eb, bool rel,
                         cudaStream_t s);
cudaError_t launch_range(const float* x, uint64_t n, WsHeader* wsh, vsz_header* hdr, double eb, bool vec,
                         cudaStream_t s);
cudaError_t launch_compact_scan(const Geom& g, uint4* chunks, vsz_header* hdr, uint32_t* blk_off,
                                uint64_t out_cap, uint64_t fix_cap, cudaStream_t s);
cudaError_t launch_compact_move(const CompressArgs& a, cudaStream_t s);
cudaError_t launch_origin_fix(const CompressArgs& a, cudaStream_t s);
cudaError_t launch_fixups(const vsz_header* hdr, const uint32_t* fix_idx, const uint32_t* fix_bits,
                          uint64_t fix_cap, float* xhat, uint64_t n, cudaStream_t s);
cudaError_t launch_histogram(const uint16_t* codes, uint64_t n, uint32_t* hist, uint32_t nbins, cudaStream_t s);
// cudaMalloc of the library's own tables, with the failure injection of
// vsz_debug_fail_alloc (api.cu)
cudaError_t lib_malloc(void** p, size_t bytes);

}  // namespace vsz
