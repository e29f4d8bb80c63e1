// Several regular-grid volumes in one persistent launch per pass.
//
// The batched frame of Sec. 4 (Alg. 1) over the views of several independent
// volumes at once: the work queue holds the ray tiles of every view, each
// view names its volume, and a warp that pops a tile marches that volume
// (pass 1, Sec. 4.1, Alg. 2) or blends it (pass 2, Sec. 4.2, Alg. 3).  The
// volumes share one transfer function (staged once per CTA in shared
// memory); their fields, domains, sampling steps and moment parameters are
// their own, read from the GridTable kernel parameter by the view's index.
// The per-tile code is the single-volume frame's (march_fused, blend_rows,
// blend_fused), so every pixel equals its volume's own frame bit for bit.
#include "mboit_grid.cuh"

namespace mb {
namespace {

template <class Cfg, bool kCache>
__global__ void __launch_bounds__(256, Cfg::kVec ? 5 : 4) k_pass1_multi(const __grid_constant__ GridTable gt, const float4* __restrict__ tf,
                                                        const __grid_constant__ ViewTable vt, char* __restrict__ moments,
                                                        Counters* __restrict__ ctr, const TileCache cache) {
    __shared__ float2 s_sig[256];
    __shared__ __align__(128) float s_win[kFusedWarps][Cfg::Floats];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float s0 = tf[i].w;
        s_sig[i] = make_float2(s0, i < 255 ? tf[i + 1].w - s0 : 0.0f);
    }
    __syncthreads();
    float* win = s_win[threadIdx.x >> 5];
    int vi, px, py, tile;
    while (next_tile(vt, &ctr->tile_next[0], vi, px, py, tile)) {
        const ViewSlot& S = vt.s[vi];
        const GridD& g = gt.g[S.vol];
        const bool valid = px < S.v.width && py < S.v.height;
        float o[3], d[3];
        int k0, k1;
        ray_range(g, S.v, valid, px, py, o, d, k0, k1);
        auto body = make_moment_body<0>(s_sig, g, S.v);
        if constexpr (kCache) {
            RowStore st{tile_rows(cache, ctr, tile, k0, k1)};
            march_fused<Cfg, false>(g, nullptr, win, o, d, k0, k1, body, st);
        } else {
            march_fused<Cfg, false>(g, nullptr, win, o, d, k0, k1, body);
        }
        if (valid) body.store(g, moments, S, S.moment_off, py * S.v.width + px);
        warp_add_u64(&ctr->samples[0], body.n);
    }
}

template <class Cfg, bool kCache>
__global__ void __launch_bounds__(256) k_pass2_multi(const __grid_constant__ GridTable gt, const float4* __restrict__ tf,
                                                     const __grid_constant__ ViewTable vt,
                                                     const char* __restrict__ moments, float* __restrict__ color,
                                                     Counters* __restrict__ ctr, const TileCache cache) {
    static_assert(Cfg::Floats >= kRowBuf && Cfg::Floats % 4 == 0, "the window slot doubles as the row buffer");
    __shared__ float4 s_tf[512];
    __shared__ __align__(16) float s_win[kFusedWarps][Cfg::Floats];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float4 e0 = tf[i], e1 = i < 255 ? tf[i + 1] : tf[i];
        s_tf[2 * i] = e0;
        s_tf[2 * i + 1] = make_float4(e1.x - e0.x, e1.y - e0.y, e1.z - e0.z, e1.w - e0.w);
    }
    __syncthreads();
    float* win = s_win[threadIdx.x >> 5];
    int vi, px, py, tile;
    while (next_tile(vt, &ctr->tile_next[1], vi, px, py, tile)) {
        const ViewSlot& S = vt.s[vi];
        const GridD& g = gt.g[S.vol];
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
            blend_rows<false>(g, cache.vals + tb * 32, kmin, kmax, k0, k1, win, body);
        } else {
            blend_fused<Cfg, false>(g, nullptr, win, o, d, k0, k1, body);
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
const void* pass1_multi_fn(bool vec) {
    return vec ? (const void*)k_pass1_multi<Stage3, kCache> : (const void*)k_pass1_multi<Stage0, kCache>;
}
template <bool kCache>
const void* pass2_multi_fn(bool vec) {
    return vec ? (const void*)k_pass2_multi<Stage3, kCache> : (const void*)k_pass2_multi<Stage0, kCache>;
}

}  // namespace

cudaError_t prepare_multi_kernels() {
    for (int vec = 0; vec < 2; ++vec) {
        const void* fs[4] = {pass1_multi_fn<false>(vec), pass1_multi_fn<true>(vec), pass2_multi_fn<false>(vec),
                             pass2_multi_fn<true>(vec)};
        for (const void* f : fs) {
            cudaFuncAttributes a;
            const cudaError_t e = cudaFuncGetAttributes(&a, f);
            if (e != cudaSuccess) return e;
            persistent_blocks(f, 256, 0);
        }
    }
    return cudaSuccess;
}

cudaError_t launch_pass1_multi(const GridTable& gt, const float4* tf, const ViewTable& vt, void* moments,
                               Counters* ctr, cudaStream_t s, bool vec, TileCache cache) {
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[0], 0, sizeof(int32_t), s);
    if (e == cudaSuccess && cache.vals) e = cudaMemsetAsync(&ctr->cache_rows, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const void* fn = cache.vals ? pass1_multi_fn<true>(vec) : pass1_multi_fn<false>(vec);
    char* m = static_cast<char*>(moments);
    void* args[] = {(void*)&gt, (void*)&tf, (void*)&vt, (void*)&m, (void*)&ctr, (void*)&cache};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

cudaError_t launch_pass2_multi(const GridTable& gt, const float4* tf, const ViewTable& vt, const void* moments,
                               float* color, Counters* ctr, cudaStream_t s, bool vec, TileCache cache) {
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[1], 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const void* fn = cache.vals ? pass2_multi_fn<true>(vec) : pass2_multi_fn<false>(vec);
    const char* m = static_cast<const char*>(moments);
    void* args[] = {(void*)&gt, (void*)&tf, (void*)&vt, (void*)&m, (void*)&color, (void*)&ctr, (void*)&cache};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

}  // namespace mb
