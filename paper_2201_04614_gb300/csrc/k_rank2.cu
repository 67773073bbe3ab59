// k_rank2.cu -- 2D instantiations of the fused compression and the inverse
// (one field, and batches of fields).
#include "recon_nd.cuh"

namespace vsz {

cudaError_t launch_lorenzo_2d(const CompressArgs& a, cudaStream_t s) {
    switch (a.g.b) {
    case 4: return launch_nd_compress<2, 4>(a, s);
    case 8: return launch_nd_compress<2, 8>(a, s);
    case 16: return launch_nd_compress<2, 16>(a, s);
    case 32: return launch_nd_compress<2, 32>(a, s);
    case 64: return launch_nd_compress<2, 64>(a, s);
    case 128: return launch_nd_compress<2, 128>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_lorenzo_batch_2d(uint32_t b, int pk, const CompressArgs* fields, const uint64_t* tile_prefix,
                                    int nfields, uint64_t total_tiles, unsigned long long* ticket, LaunchShape sh,
                                    cudaStream_t s, int* occ) {
    switch (b) {
    case 4: return launch_nd_compress_batch<2, 4>(pk, fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 8: return launch_nd_compress_batch<2, 8>(pk, fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 16: return launch_nd_compress_batch<2, 16>(pk, fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 32: return launch_nd_compress_batch<2, 32>(pk, fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 64: return launch_nd_compress_batch<2, 64>(pk, fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 128: return launch_nd_compress_batch<2, 128>(pk, fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_recon_2d(const ReconArgs& a, bool q_out, cudaStream_t s) {
    switch (a.g.b) {
    case 4: return launch_nd_recon<2, 4>(a, q_out, s);
    case 8: return launch_nd_recon<2, 8>(a, q_out, s);
    case 16: return launch_nd_recon<2, 16>(a, q_out, s);
    case 32: return launch_nd_recon<2, 32>(a, q_out, s);
    case 64: return launch_nd_recon<2, 64>(a, q_out, s);
    case 128: return launch_nd_recon<2, 128>(a, q_out, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_recon_batch_2d(uint32_t b, const ReconArgs* fields, const uint64_t* tile_prefix, int nfields,
                                  uint64_t total_tiles, unsigned long long* ticket, LaunchShape sh, cudaStream_t s,
                                  int* occ) {
    switch (b) {
    case 4: return launch_nd_recon_batch<2, 4>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 8: return launch_nd_recon_batch<2, 8>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 16: return launch_nd_recon_batch<2, 16>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 32: return launch_nd_recon_batch<2, 32>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 64: return launch_nd_recon_batch<2, 64>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    case 128: return launch_nd_recon_batch<2, 128>(fields, tile_prefix, nfields, total_tiles, ticket, sh, s, occ);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace vsz
