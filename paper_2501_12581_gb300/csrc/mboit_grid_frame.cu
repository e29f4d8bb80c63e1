// One-launch batched frame for regular grids (four power moments).
//
// In the fused form a warp marches every selected piece of its 32 rays, so
// when its pass 1 (Sec. 4.1, Alg. 2) ends, the moments in its registers are
// already the sum over the pieces (the Allreduce add) for those pixels: no
// other tile contributes to them.  The warp can therefore take the same rays
// through pass 2 (Sec. 4.2, Alg. 1 loop 2, Alg. 3) at once, instead of the
// whole frame waiting for a second launch.  Pass 1 stores every lattice
// point's value in the tile's rows of the frame cache, exactly as in the
// two-launch frame, and pass 2 reads them back (cp.async prefetch through the
// warp's shared-memory slot) after a __syncwarp, which orders the lanes'
// global stores before the other lanes' loads.  On one SM, warps in the march
// (bound by the L1 / shared-memory pipe) then run beside warps in the blend
// (bound by instruction issue).  Results are bit-identical to the two-launch
// frame: the frame is built from the same float32 moments, read from
// registers instead of the moment image.
#include <cstring>

#include "mboit_grid.cuh"

namespace mb {
namespace {

template <bool kSel, class Cfg>
__global__ void __launch_bounds__(256) k_frame_fused(const __grid_constant__ GridD g, const float4* __restrict__ tf,
                                                     const uint8_t* __restrict__ sel, const __grid_constant__ ViewTable vt,
                                                     char* __restrict__ moments, float* __restrict__ color, int mode,
                                                     Counters* __restrict__ ctr, const TileCache cache,
                                                     const __grid_constant__ CUtensorMap tmap) {
    static_assert(Cfg::Floats >= kRowBuf && Cfg::Floats % 4 == 0, "the window slot doubles as the row buffer");
    __shared__ float2 s_sig[256];
    __shared__ float4 s_tf[512];
    __shared__ __align__(128) float s_win[kFusedWarps][Cfg::Floats];
    __shared__ __align__(8) uint64_t s_bar[Cfg::kTma ? kFusedWarps : 1];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float4 e0 = tf[i], e1 = i < 255 ? tf[i + 1] : tf[i];
        s_tf[2 * i] = e0;
        s_tf[2 * i + 1] = make_float4(e1.x - e0.x, e1.y - e0.y, e1.z - e0.z, e1.w - e0.w);
        s_sig[i] = make_float2(e0.w, i < 255 ? e1.w - e0.w : 0.0f);
    }
    tma_init<Cfg>(s_bar);
    __syncthreads();
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float* win = s_win[threadIdx.x >> 5];
    TmaWin tw{&tmap, s_bar + (Cfg::kTma ? threadIdx.x >> 5 : 0), 0u, &ctr->error, (g.flags & kFlagDebugNoCopy) != 0};
    const bool raw = (g.flags & 1u) != 0;
    int vi, px, py, tile;
    while (next_tile(vt, &ctr->tile_next[0], vi, px, py, tile)) {
        const ViewSlot& S = vt.s[vi];
        const bool valid = px < S.v.width && py < S.v.height;
        const int pix = valid ? py * S.v.width + px : 0;
        float o[3], d[3];
        int k0, k1;
        ray_range(g, S.v, valid, px, py, o, d, k0, k1);
        // the tile's cache rows (lane 0 takes them; -1: no room, pass 2 marches again)
        const int kmin = __reduce_min_sync(full, k0), kmax = __reduce_max_sync(full, k1);
        long long base = -1;
        if (lane == 0 && kmax >= kmin) {
            const long long rows = (long long)kmax - kmin + 1;
            const long long r = (long long)atomicAdd(&ctr->cache_rows, (unsigned long long)rows);
            if (r + rows <= cache.rows_cap) base = r;
        }
        base = __shfl_sync(full, base, 0);

        // pass 1: moments of every selected piece, summed in registers
        auto m1 = make_moment_body<0>(s_sig, g, S.v);
        RowStore st{base >= 0 ? cache.vals + (base - kmin) * 32 + lane : nullptr};
        if (!march_fused<Cfg, kSel>(g, sel, win, o, d, k0, k1, m1, st, &tw)) return;
        if (valid) m1.store(g, moments, S, S.moment_off, pix);
        warp_add_u64(&ctr->samples[0], m1.n);

        // pass 2 of the same rays
        BlendBody body = blend_body_of(s_tf, g, S, m1, valid);
        count_frames(ctr, body, valid);
        __syncwarp();  // the rows' stores before any lane reads them; the window slot is free
        if (base >= 0)
            blend_rows<kSel>(g, cache.vals + base * 32, kmin, kmax, k0, k1, win, body);
        else
            if (!blend_fused<Cfg, kSel>(g, sel, win, o, d, k0, k1, body, &tw)) return;
        if (valid) {
            float4* out = reinterpret_cast<float4*>(color + S.color_off) + pix;
            if (mode == kColorResolved)
                *out = resolve_pixel(body.C, body.b0, make_float4(0.0f, 0.0f, 0.0f, 0.0f), raw);
            else
                *out = body.C;
        }
        warp_add_u64(&ctr->samples[1], body.n);
        __syncwarp();  // every lane is done with the slot before the next tile's window
    }
}

const void* frame_fn(int cfg, bool sel) {
    if (sel) return (const void*)k_frame_fused<true, Stage0>;
    switch (cfg) {
        case 1: return (const void*)k_frame_fused<false, Stage1>;
        case 2: return (const void*)k_frame_fused<false, Stage2>;
        case 3: return (const void*)k_frame_fused<false, Stage3>;
        case 4: return (const void*)k_frame_fused<false, Stage4>;
        case 5: return (const void*)k_frame_fused<false, Stage5>;
        case 6: return (const void*)k_frame_fused<false, Stage6>;
        default: return (const void*)k_frame_fused<false, Stage0>;
    }
}

}  // namespace

bool stage_config_eligible(const GridD& g, int cfg);

cudaError_t prepare_frame_kernels() {
    for (int cfg = 0; cfg < kNumStageConfigs; ++cfg)
        for (int sel = 0; sel < 2; ++sel) {
            const void* f = frame_fn(cfg, sel);
            cudaFuncAttributes a;
            const cudaError_t e = cudaFuncGetAttributes(&a, f);
            if (e != cudaSuccess) return e;
            persistent_blocks(f, 256, 0);
        }
    return cudaSuccess;
}

cudaError_t launch_frame_fused(const GridD& g, const float4* tf, const uint8_t* brick_sel, const ViewTable& vt,
                               void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s, int cfg,
                               TileCache cache, const CUtensorMap* tmap) {
    if (!stage_config_eligible(g, cfg)) cfg = 0;
    if ((cfg == 5 || cfg == 6) && !tmap) cfg = 3;
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[0], 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&ctr->cache_rows, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const void* fn = frame_fn(cfg, brick_sel != nullptr);
    char* m = static_cast<char*>(moments);
    int md = mode;
    CUtensorMap map;
    if (tmap)
        map = *tmap;
    else
        std::memset(&map, 0, sizeof map);   // not read by configurations without TMA
    void* args[] = {(void*)&g, (void*)&tf, (void*)&brick_sel, (void*)&vt, (void*)&m, (void*)&color, (void*)&md,
                    (void*)&ctr, (void*)&cache, (void*)&map};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

}  // namespace mb
