// Launch interface of the multi-volume octree passes (mboit_multi_amr.cu);
// the grid counterpart is declared in mboit_internal.h.  Not part of the
// public ABI.
#pragma once
#include "mboit_internal.h"

namespace mb {

// The multi-volume frame's two passes over several brick octrees (four power
// moments, fixed step): view slot i samples octree vt.s[i].vol.  `sel`
// selects the checked kernels (an octree with holes among them).  Pass 1
// stores the tile cache when cache.vals is set and pass 2 then blends from
// it; results equal each octree's own frame.
struct AmrTable {
    AmrD a[kMaxVolumes];
};
cudaError_t launch_pass1_multi_amr(const AmrTable& at, const float4* tf, const ViewTable& vt, void* moments,
                                   Counters* ctr, cudaStream_t s, bool sel, TileCache cache);
cudaError_t launch_pass2_multi_amr(const AmrTable& at, const float4* tf, const ViewTable& vt, const void* moments,
                                   float* color, Counters* ctr, cudaStream_t s, bool sel, TileCache cache);
cudaError_t prepare_multi_amr_kernels();

}  // namespace mb
