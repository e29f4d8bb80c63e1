// Several brick octrees in one persistent launch per pass: the octree
// counterpart of mboit_grid_multi.cu.  Each view slot names its volume, whose
// descriptor the kernels read from the AmrTable kernel parameter; the
// per-tile code is the single-volume octree passes' (march_unit in lockstep
// rows for pass 1, blend_rows from the tile cache for pass 2), so every image
// equals its volume's own frame bit for bit.  A volume whose tables failed
// their check (its error word is set) has its tiles skipped in both passes.
#include "mboit_multi.h"
#include "mboit_units.cuh"

namespace mb {
namespace {

template <bool kSel, bool kCache>
__global__ void __launch_bounds__(256, 4) k_pass1_multi_amr(const __grid_constant__ AmrTable at,
                                                            const float4* __restrict__ tf,
                                                            const __grid_constant__ ViewTable vt,
                                                            char* __restrict__ moments, Counters* __restrict__ ctr,
                                                            const TileCache cache) {
    __shared__ float2 s_sig[256];
    __shared__ float4 s_z[kFusedWarps][kDepthRows];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float s0 = tf[i].w;
        s_sig[i] = make_float2(s0, i < 255 ? tf[i + 1].w - s0 : 0.0f);
    }
    __syncthreads();
    float4* zrows = s_z[threadIdx.x >> 5];
    int vi, px, py, tile;
    while (next_tile(vt, &ctr->tile_next[0], vi, px, py, tile)) {
        const ViewSlot& S = vt.s[vi];
        const AmrD& a = at.a[S.vol];
        if (tables_bad(a)) continue;
        const GridD& g = a.g;
        const bool valid = px < S.v.width && py < S.v.height;
        float o[3], d[3];
        int k0, k1;
        ray_range(g, S.v, valid, px, py, o, d, k0, k1);
        auto body = make_moment_body<0>(s_sig, g, S.v);
        if constexpr (kCache) {
            RowStore st{tile_rows(cache, ctr, tile, k0, k1)};
            march_unit<kSel>(a, nullptr, o, d, k0, k1, body, st, zrows);
        } else {
            march_unit<kSel>(a, nullptr, o, d, k0, k1, body, NoStore{}, zrows);
        }
        if (valid) body.store(g, moments, S, S.moment_off, py * S.v.width + px);
        warp_add_u64(&ctr->samples[0], body.n);
    }
}

template <bool kSel, bool kCache>
__global__ void __launch_bounds__(256, 4) k_pass2_multi_amr(const __grid_constant__ AmrTable at,
                                                            const float4* __restrict__ tf,
                                                            const __grid_constant__ ViewTable vt,
                                                            const char* __restrict__ moments, float* __restrict__ color,
                                                            Counters* __restrict__ ctr, const TileCache cache) {
    __shared__ float4 s_tf[512];
    __shared__ __align__(16) float s_rows[kCache ? kFusedWarps : 1][kCache ? kUnitRowBuf : 4];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float4 e0 = tf[i], e1 = i < 255 ? tf[i + 1] : tf[i];
        s_tf[2 * i] = e0;
        s_tf[2 * i + 1] = make_float4(e1.x - e0.x, e1.y - e0.y, e1.z - e0.z, e1.w - e0.w);
    }
    __syncthreads();
    int vi, px, py, tile;
    while (next_tile(vt, &ctr->tile_next[1], vi, px, py, tile)) {
        const ViewSlot& S = vt.s[vi];
        const AmrD& a = at.a[S.vol];
        if (tables_bad(a)) continue;
        const GridD& g = a.g;
        const bool valid = px < S.v.width && py < S.v.height;
        const int pix = valid ? py * S.v.width + px : 0;
        auto body = make_blend_body<0>(s_tf, g, S, moments, S.moment_off, pix, valid);
        count_frames(ctr, body, valid);
        float o[3], d[3];
        int k0, k1;
        ray_range(g, S.v, valid, px, py, o, d, k0, k1);
        const long long tb = kCache ? cache.tile_base[tile] : -1;
        if (kCache && tb >= 0) {
            const int kmin = __reduce_min_sync(0xffffffffu, k0), kmax = __reduce_max_sync(0xffffffffu, k1);
            blend_rows<kSel, false, kUnitRowChunk>(g, cache.vals + tb * 32, kmin, kmax, k0, k1,
                                                   s_rows[kCache ? threadIdx.x >> 5 : 0], body);
        } else {
            march_unit<kSel>(a, nullptr, o, d, k0, k1, body);
        }
        if (valid) {
            const bool raw = (g.flags & kFlagRawSum) != 0;
            reinterpret_cast<float4*>(color + S.color_off)[pix] =
                resolve_pixel(body.C, body.b0, make_float4(0.0f, 0.0f, 0.0f, 0.0f), raw);
        }
        warp_add_u64(&ctr->samples[1], body.n);
    }
}

template <bool kCache>
const void* pass1_fn(bool sel) {
    return sel ? (const void*)k_pass1_multi_amr<true, kCache> : (const void*)k_pass1_multi_amr<false, kCache>;
}
template <bool kCache>
const void* pass2_fn(bool sel) {
    return sel ? (const void*)k_pass2_multi_amr<true, kCache> : (const void*)k_pass2_multi_amr<false, kCache>;
}

}  // namespace

cudaError_t prepare_multi_amr_kernels() {
    for (int sel = 0; sel < 2; ++sel) {
        const void* fs[4] = {pass1_fn<false>(sel), pass1_fn<true>(sel), pass2_fn<false>(sel), pass2_fn<true>(sel)};
        for (const void* f : fs) {
            cudaFuncAttributes attr;
            const cudaError_t e = cudaFuncGetAttributes(&attr, f);
            if (e != cudaSuccess) return e;
            persistent_blocks(f, 256, 0);
        }
    }
    return cudaSuccess;
}

cudaError_t launch_pass1_multi_amr(const AmrTable& at, const float4* tf, const ViewTable& vt, void* moments,
                                   Counters* ctr, cudaStream_t s, bool sel, TileCache cache) {
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[0], 0, sizeof(int32_t), s);
    if (e == cudaSuccess && cache.vals) e = cudaMemsetAsync(&ctr->cache_rows, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const void* fn = cache.vals ? pass1_fn<true>(sel) : pass1_fn<false>(sel);
    char* m = static_cast<char*>(moments);
    void* args[] = {(void*)&at, (void*)&tf, (void*)&vt, (void*)&m, (void*)&ctr, (void*)&cache};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

cudaError_t launch_pass2_multi_amr(const AmrTable& at, const float4* tf, const ViewTable& vt, const void* moments,
                                   float* color, Counters* ctr, cudaStream_t s, bool sel, TileCache cache) {
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[1], 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const void* fn = cache.vals ? pass2_fn<true>(sel) : pass2_fn<false>(sel);
    const char* m = static_cast<const char*>(moments);
    void* args[] = {(void*)&at, (void*)&tf, (void*)&vt, (void*)&m, (void*)&color, (void*)&ctr, (void*)&cache};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

}  // namespace mb
