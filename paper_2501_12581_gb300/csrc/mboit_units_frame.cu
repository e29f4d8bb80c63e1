// One-launch batched frame for brick octrees and tetrahedral meshes (four
// power moments), the counterpart of k_frame_fused on grids: a warp marches
// every selected piece of its 32 rays (pass 1, Sec. 4.1, Alg. 2), so the
// moments in its registers are the pixels' global moments, and it blends the
// same rays at once (pass 2, Sec. 4.2, Alg. 3) from the sample values it has
// just stored in the tile's cache rows.  On one SM, warps waiting on the
// octree's leaf gathers or the mesh walk run beside warps in the issue-bound
// blend.  Results are bit-identical to the two-launch frame.
#include "mboit_units.cuh"

namespace mb {
namespace {

// Resident CTAs the register budget is set for: 4 on octrees (64 registers,
// no spills, as their pass 1), the mesh passes' bound on meshes.
template <class V> struct FrameMinBlocks { static constexpr int value = 4; };
template <bool k> struct FrameMinBlocks<TetT<k>> { static constexpr int value = MB_TET_MIN_BLOCKS; };

template <class V, bool kSel>
__global__ void __launch_bounds__(256, FrameMinBlocks<V>::value) k_frame_unit(
    const __grid_constant__ V a, const float4* __restrict__ tf, const uint8_t* __restrict__ sel,
    const __grid_constant__ ViewTable vt, char* __restrict__ moments, float* __restrict__ color, int mode,
    Counters* __restrict__ ctr, const TileCache cache) {
    if (tables_bad(a)) return;
    __shared__ float2 s_sig[256];
    __shared__ float4 s_tf[512];
    __shared__ __align__(16) float s_rows[kFusedWarps][kUnitRowBuf];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float4 e0 = tf[i], e1 = i < 255 ? tf[i + 1] : tf[i];
        s_tf[2 * i] = e0;
        s_tf[2 * i + 1] = make_float4(e1.x - e0.x, e1.y - e0.y, e1.z - e0.z, e1.w - e0.w);
        s_sig[i] = make_float2(e0.w, i < 255 ? e1.w - e0.w : 0.0f);
    }
    __syncthreads();
    const GridD& g = a.g;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float* buf = s_rows[threadIdx.x >> 5];
    const bool raw = (g.flags & 1u) != 0;
    bool tagged = false;  // octree samples of the adaptive step carry their weight
    int tmask = 0;
    if constexpr (std::is_same<V, AmrD>::value) {
        tagged = (g.flags & kFlagAdaptiveStep) != 0;
        tmask = tag_mask(a.max_level);
    }
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
        if constexpr (std::is_same<V, AmrD>::value)
            march_unit<kSel>(a, sel, o, d, k0, k1, m1, st, reinterpret_cast<float4*>(buf));
        else
            march_unit<kSel>(a, sel, o, d, k0, k1, m1, st);
        if (valid) m1.store(g, moments, S, S.moment_off, pix);
        warp_add_u64(&ctr->samples[0], m1.n);

        // pass 2 of the same rays
        BlendBody body = blend_body_of(s_tf, g, S, m1, valid);
        count_frames(ctr, body, valid);
        __syncwarp();  // the rows' stores before any lane reads them
        if (base >= 0) {
            if (tagged)
                blend_rows<true, true, kRowChunk>(g, cache.vals + base * 32, kmin, kmax, k0, k1, buf, body, tmask);
            else
                blend_rows<RowsChecked<V, kSel>::value, false, kRowChunk>(g, cache.vals + base * 32, kmin, kmax,
                                                                               k0, k1, buf, body);
        } else {
            march_unit<kSel>(a, sel, o, d, k0, k1, body);
        }
        if (valid) {
            float4* out = reinterpret_cast<float4*>(color + S.color_off) + pix;
            *out = mode == kColorResolved ? resolve_pixel(body.C, body.b0, make_float4(0.0f, 0.0f, 0.0f, 0.0f), raw)
                                          : body.C;
        }
        warp_add_u64(&ctr->samples[1], body.n);
    }
}

template <bool kN>
TetT<kN> as_tet(const TetD& m) {
    TetT<kN> t;
    static_cast<TetD&>(t) = m;
    return t;
}

// Octrees with holes take the checked kernels (see RowsChecked).
template <class V> bool complete_units(const V&) { return true; }
template <> bool complete_units<AmrD>(const AmrD& a) { return a.complete != 0; }

template <class V>
const void* frame_unit_fn(bool sel) {
    return sel ? (const void*)k_frame_unit<V, true> : (const void*)k_frame_unit<V, false>;
}

template <class V>
cudaError_t launch_frame_unit(const V& vol, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                              void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s,
                              TileCache cache) {
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[0], 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&ctr->cache_rows, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const void* fn = frame_unit_fn<V>(unit_sel != nullptr || !complete_units(vol));
    char* mo = static_cast<char*>(moments);
    int md = mode;
    void* args[] = {(void*)&vol, (void*)&tf, (void*)&unit_sel, (void*)&vt, (void*)&mo, (void*)&color, (void*)&md,
                    (void*)&ctr, (void*)&cache};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

}  // namespace

cudaError_t prepare_frame_unit_kernels() {
    const void* fns[] = {frame_unit_fn<AmrD>(false),        frame_unit_fn<AmrD>(true),
                         frame_unit_fn<TetT<true>>(false),  frame_unit_fn<TetT<true>>(true),
                         frame_unit_fn<TetT<false>>(false), frame_unit_fn<TetT<false>>(true)};
    for (const void* f : fns) {
        cudaFuncAttributes attr;
        const cudaError_t e = cudaFuncGetAttributes(&attr, f);
        if (e != cudaSuccess) return e;
        persistent_blocks(f, 256, 0);
    }
    return cudaSuccess;
}

cudaError_t launch_frame_amr(const AmrD& a, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                             void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s,
                             TileCache cache) {
    return launch_frame_unit(a, tf, unit_sel, vt, moments, color, mode, ctr, s, cache);
}

cudaError_t launch_frame_tet(const TetD& m, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                             void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s,
                             TileCache cache) {
    return m.narrow ? launch_frame_unit(as_tet<true>(m), tf, unit_sel, vt, moments, color, mode, ctr, s, cache)
                    : launch_frame_unit(as_tet<false>(m), tf, unit_sel, vt, moments, color, mode, ctr, s, cache);
}

}  // namespace mb
