// Octree and tetrahedral-mesh passes, and the plain per-piece and sort-last
// marches of every volume kind, for sm_103a: kernel selection and launchers
// (the kernel templates are in mboit_units.cuh).
#include "mboit_units.cuh"

namespace mb {

// The kernels of the other moment sets, compiled in parallel: trigonometric
// (mboit_units_trig.cu) and 6 / 8 power moments (mboit_units_power.cu).
// vkind: 0 grid, 1 octree, 2 narrow mesh, 3 wide mesh; pass 1 or 2.
const void* unit_trig_fn(int vkind, int pass, int ms, bool sel, bool cache);
const void* piece_trig_fn(int vkind, int pass, int ms);
const void* unit_power_fn(int vkind, int pass, int ms, bool sel, bool cache);
const void* piece_power_fn(int vkind, int pass, int ms);

namespace {

template <class V> constexpr int vkind_of();
template <> constexpr int vkind_of<GridD>() { return 0; }
template <> constexpr int vkind_of<AmrD>() { return 1; }
template <> constexpr int vkind_of<TetT<true>>() { return 2; }
template <> constexpr int vkind_of<TetT<false>>() { return 3; }

// ms: the moment set's kernel variant (TrigTables::sel): 0, 3, 4, 6 or 8.
template <class V, bool kSel, bool kC>
const void* unit1_ms(int ms) {
    switch (ms) {
        case 3:
        case 4: return unit_trig_fn(vkind_of<V>(), 1, ms, kSel, kC);
        case 6:
        case 8: return unit_power_fn(vkind_of<V>(), 1, ms, kSel, kC);
        default: return (const void*)k_pass1_unit<V, kSel, 0, kC>;
    }
}
template <class V, bool kSel, bool kC>
const void* unit2_ms(int ms) {
    switch (ms) {
        case 3:
        case 4: return unit_trig_fn(vkind_of<V>(), 2, ms, kSel, kC);
        case 6:
        case 8: return unit_power_fn(vkind_of<V>(), 2, ms, kSel, kC);
        default: return (const void*)k_pass2_unit<V, kSel, 0, kC>;
    }
}
template <class V, bool kC = false>
const void* unit1_fn(bool sel, int ms) {
    return sel ? unit1_ms<V, true, kC>(ms) : unit1_ms<V, false, kC>(ms);
}
template <class V, bool kC = false>
const void* unit2_fn(bool sel, int ms) {
    return sel ? unit2_ms<V, true, kC>(ms) : unit2_ms<V, false, kC>(ms);
}

// The plain per-piece kernels of a moment set (same parameters for every set).
template <class V>
const void* piece1_kernel(int ms) {
    switch (ms) {
        case 3:
        case 4: return piece_trig_fn(vkind_of<V>(), 1, ms);
        case 6:
        case 8: return piece_power_fn(vkind_of<V>(), 1, ms);
        default: return (const void*)k_pass1_piece<V, 0>;
    }
}
template <class V>
const void* piece2_kernel(int ms) {
    switch (ms) {
        case 3:
        case 4: return piece_trig_fn(vkind_of<V>(), 2, ms);
        case 6:
        case 8: return piece_power_fn(vkind_of<V>(), 2, ms);
        default: return (const void*)k_pass2_piece<V, 0>;
    }
}

// One launch of a per-piece kernel: 128-thread blocks, 4 ray tiles each.
template <class V>
cudaError_t launch_piece_kernel(const void* fn, const V& vol, const float4* tf, const int32_t* pou, int32_t piece,
                                const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                                const void* moments, float* color, Counters* ctr, cudaStream_t s) {
    const int blocks = (vt.total_tiles + 3) / 4;
    int pc = piece, sl = slot, ns = n_slots;
    const void* m = moments;
    void* args1[] = {(void*)&vol, (void*)&tf, (void*)&pou, (void*)&pc, (void*)&box, (void*)&vt,
                     (void*)&sl, (void*)&ns, (void*)&m, (void*)&ctr};
    void* args2[] = {(void*)&vol, (void*)&tf, (void*)&pou, (void*)&pc, (void*)&box, (void*)&vt,
                     (void*)&sl, (void*)&ns, (void*)&m, (void*)&color, (void*)&ctr};
    return cudaLaunchKernel(fn, dim3(blocks > 0 ? blocks : 1), dim3(128), color ? args2 : args1, 0, s);
}

__global__ void k_tet_values(int4* __restrict__ corners, const int4* __restrict__ cells, int64_t n_tets,
                             const float* __restrict__ values) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tets; t += (int64_t)gridDim.x * blockDim.x) {
        const int4 c = cells[t];
        corners[4 * t].w = __float_as_int(values[c.x]);
        corners[4 * t + 1].w = __float_as_int(values[c.y]);
        corners[4 * t + 2].w = __float_as_int(values[c.z]);
        corners[4 * t + 3].w = __float_as_int(values[c.w]);
    }
}


}  // namespace

cudaError_t prepare_unit_kernels() {
    const void* fns[] = {(const void*)k_sortlast_piece<GridD, true>, (const void*)k_sortlast_piece<GridD, false>,
                         (const void*)k_sortlast_piece<AmrD, true>, (const void*)k_sortlast_piece<AmrD, false>,
                         (const void*)k_sortlast_piece<TetT<true>, true>, (const void*)k_sortlast_piece<TetT<true>, false>,
                         (const void*)k_sortlast_piece<TetT<false>, true>, (const void*)k_sortlast_piece<TetT<false>, false>,
                         (const void*)k_tet_values};
    for (const void* f : fns) {
        cudaFuncAttributes a;
        const cudaError_t e = cudaFuncGetAttributes(&a, f);
        if (e != cudaSuccess) return e;
    }
    const int sets[5] = {0, 3, 4, 6, 8};
    for (int ms : sets) {
        const void* pf[] = {piece1_kernel<GridD>(ms),       piece2_kernel<GridD>(ms),
                            piece1_kernel<AmrD>(ms),        piece2_kernel<AmrD>(ms),
                            piece1_kernel<TetT<true>>(ms),  piece2_kernel<TetT<true>>(ms),
                            piece1_kernel<TetT<false>>(ms), piece2_kernel<TetT<false>>(ms)};
        for (const void* f : pf) {
            cudaFuncAttributes a;
            const cudaError_t e = cudaFuncGetAttributes(&a, f);
            if (e != cudaSuccess) return e;
        }
        for (int sel = 0; sel < 2; ++sel) {
            persistent_blocks(unit1_fn<AmrD>(sel, ms), 256, 0);
            persistent_blocks(unit2_fn<AmrD>(sel, ms), 256, 0);
            persistent_blocks(unit1_fn<AmrD, true>(sel, ms), 256, 0);
            persistent_blocks(unit2_fn<AmrD, true>(sel, ms), 256, 0);
            persistent_blocks(unit1_fn<TetT<true>>(sel, ms), 256, 0);
            persistent_blocks(unit2_fn<TetT<true>>(sel, ms), 256, 0);
            persistent_blocks(unit1_fn<TetT<false>>(sel, ms), 256, 0);
            persistent_blocks(unit2_fn<TetT<false>>(sel, ms), 256, 0);
            persistent_blocks(unit1_fn<TetT<true>, true>(sel, ms), 256, 0);
            persistent_blocks(unit2_fn<TetT<true>, true>(sel, ms), 256, 0);
            persistent_blocks(unit1_fn<TetT<false>, true>(sel, ms), 256, 0);
            persistent_blocks(unit2_fn<TetT<false>, true>(sel, ms), 256, 0);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_pass1_piece(const GridD& g, const float4* tf, const int32_t* pob, int32_t piece,
                               const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                               void* moments, Counters* ctr, cudaStream_t s) {
    return launch_piece_kernel(piece1_kernel<GridD>(g.trig.sel), g, tf, pob, piece, box, vt, slot, n_slots, moments,
                               nullptr, ctr, s);
}

cudaError_t launch_pass2_piece(const GridD& g, const float4* tf, const int32_t* pob, int32_t piece,
                               const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                               const void* moments, float* color, Counters* ctr, cudaStream_t s) {
    return launch_piece_kernel(piece2_kernel<GridD>(g.trig.sel), g, tf, pob, piece, box, vt, slot, n_slots, moments,
                               color, ctr, s);
}

cudaError_t launch_sortlast_march(bool fill, const GridD& g, const float4* tf, const int32_t* pob, int32_t piece,
                                  const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                                  int32_t* counts, const int64_t* starts, int32_t* seg_key, float4* seg_col,
                                  cudaStream_t s) {
    const int blocks = (vt.total_tiles + 3) / 4;
    if (fill)
        k_sortlast_piece<GridD, true><<<blocks, 128, 0, s>>>(g, tf, pob, piece, box, vt, slot, n_slots, counts, starts, seg_key,
                                                      seg_col);
    else
        k_sortlast_piece<GridD, false><<<blocks, 128, 0, s>>>(g, tf, pob, piece, box, vt, slot, n_slots, counts, starts,
                                                       seg_key, seg_col);
    return cudaGetLastError();
}

cudaError_t launch_pass1_amr(const AmrD& a, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                             void* moments, Counters* ctr, cudaStream_t s, TileCache cache) {
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[0], 0, sizeof(int32_t), s);
    if (e == cudaSuccess && cache.vals) e = cudaMemsetAsync(&ctr->cache_rows, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const bool sel = unit_sel != nullptr || !a.complete;   // octrees with holes take the checked kernels
    const void* fn = cache.vals ? unit1_fn<AmrD, true>(sel, a.g.trig.sel) : unit1_fn<AmrD>(sel, a.g.trig.sel);
    char* m = static_cast<char*>(moments);
    void* args[] = {(void*)&a, (void*)&tf, (void*)&unit_sel, (void*)&vt, (void*)&m, (void*)&ctr, (void*)&cache};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

cudaError_t launch_pass2_amr(const AmrD& a, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                             const void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s,
                             TileCache cache) {
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[1], 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const bool sel = unit_sel != nullptr || !a.complete;
    const void* fn = cache.vals ? unit2_fn<AmrD, true>(sel, a.g.trig.sel) : unit2_fn<AmrD>(sel, a.g.trig.sel);
    const char* m = static_cast<const char*>(moments);
    int md = mode;
    void* args[] = {(void*)&a, (void*)&tf, (void*)&unit_sel, (void*)&vt, (void*)&m, (void*)&color, (void*)&md,
                    (void*)&ctr, (void*)&cache};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

cudaError_t launch_pass1_piece(const AmrD& a, const float4* tf, const int32_t* pou, int32_t piece, const PieceBox& box,
                               const ViewTable& vt, int32_t slot, int32_t n_slots, void* moments, Counters* ctr,
                               cudaStream_t s) {
    return launch_piece_kernel(piece1_kernel<AmrD>(a.g.trig.sel), a, tf, pou, piece, box, vt, slot, n_slots, moments,
                               nullptr, ctr, s);
}

cudaError_t launch_pass2_piece(const AmrD& a, const float4* tf, const int32_t* pou, int32_t piece, const PieceBox& box,
                               const ViewTable& vt, int32_t slot, int32_t n_slots, const void* moments, float* color,
                               Counters* ctr, cudaStream_t s) {
    return launch_piece_kernel(piece2_kernel<AmrD>(a.g.trig.sel), a, tf, pou, piece, box, vt, slot, n_slots, moments,
                               color, ctr, s);
}

cudaError_t launch_sortlast_march(bool fill, const AmrD& a, const float4* tf, const int32_t* pou, int32_t piece,
                                  const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                                  int32_t* counts, const int64_t* starts, int32_t* seg_key, float4* seg_col,
                                  cudaStream_t s) {
    const int blocks = (vt.total_tiles + 3) / 4;
    if (fill)
        k_sortlast_piece<AmrD, true><<<blocks, 128, 0, s>>>(a, tf, pou, piece, box, vt, slot, n_slots, counts, starts,
                                                            seg_key, seg_col);
    else
        k_sortlast_piece<AmrD, false><<<blocks, 128, 0, s>>>(a, tf, pou, piece, box, vt, slot, n_slots, counts, starts,
                                                             seg_key, seg_col);
    return cudaGetLastError();
}

namespace {

template <bool kN>
TetT<kN> as_tet(const TetD& m) {
    TetT<kN> t;
    static_cast<TetD&>(t) = m;
    return t;
}

template <class V>
cudaError_t launch_unit1(const V& vol, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt, void* moments,
                         Counters* ctr, cudaStream_t s, TileCache cache) {
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[0], 0, sizeof(int32_t), s);
    if (e == cudaSuccess && cache.vals) e = cudaMemsetAsync(&ctr->cache_rows, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const bool sel = unit_sel != nullptr;
    const void* fn = cache.vals ? unit1_fn<V, true>(sel, vol.g.trig.sel) : unit1_fn<V>(sel, vol.g.trig.sel);
    char* mo = static_cast<char*>(moments);
    void* args[] = {(void*)&vol, (void*)&tf, (void*)&unit_sel, (void*)&vt, (void*)&mo, (void*)&ctr, (void*)&cache};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

template <class V>
cudaError_t launch_unit2(const V& vol, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                         const void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s,
                         TileCache cache) {
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[1], 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const bool sel = unit_sel != nullptr;
    const void* fn = cache.vals ? unit2_fn<V, true>(sel, vol.g.trig.sel) : unit2_fn<V>(sel, vol.g.trig.sel);
    const char* mo = static_cast<const char*>(moments);
    int md = mode;
    void* args[] = {(void*)&vol, (void*)&tf, (void*)&unit_sel, (void*)&vt, (void*)&mo, (void*)&color, (void*)&md,
                    (void*)&ctr, (void*)&cache};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

template <class V>
cudaError_t launch_piece1(const V& m, const float4* tf, const int32_t* pou, int32_t piece, const PieceBox& box,
                          const ViewTable& vt, int32_t slot, int32_t n_slots, void* moments, Counters* ctr,
                          cudaStream_t s) {
    return launch_piece_kernel(piece1_kernel<V>(m.g.trig.sel), m, tf, pou, piece, box, vt, slot, n_slots, moments,
                               nullptr, ctr, s);
}

template <class V>
cudaError_t launch_piece2(const V& m, const float4* tf, const int32_t* pou, int32_t piece, const PieceBox& box,
                          const ViewTable& vt, int32_t slot, int32_t n_slots, const void* moments, float* color,
                          Counters* ctr, cudaStream_t s) {
    return launch_piece_kernel(piece2_kernel<V>(m.g.trig.sel), m, tf, pou, piece, box, vt, slot, n_slots, moments,
                               color, ctr, s);
}

template <class V>
cudaError_t launch_sortlast(bool fill, const V& m, const float4* tf, const int32_t* pou, int32_t piece,
                            const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots, int32_t* counts,
                            const int64_t* starts, int32_t* seg_key, float4* seg_col, cudaStream_t s) {
    const int blocks = (vt.total_tiles + 3) / 4;
    if (fill)
        k_sortlast_piece<V, true><<<blocks, 128, 0, s>>>(m, tf, pou, piece, box, vt, slot, n_slots, counts, starts,
                                                         seg_key, seg_col);
    else
        k_sortlast_piece<V, false><<<blocks, 128, 0, s>>>(m, tf, pou, piece, box, vt, slot, n_slots, counts, starts,
                                                          seg_key, seg_col);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pass1_tet(const TetD& m, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                             void* moments, Counters* ctr, cudaStream_t s, TileCache cache) {
    return m.narrow ? launch_unit1(as_tet<true>(m), tf, unit_sel, vt, moments, ctr, s, cache)
                    : launch_unit1(as_tet<false>(m), tf, unit_sel, vt, moments, ctr, s, cache);
}

cudaError_t launch_pass2_tet(const TetD& m, const float4* tf, const uint8_t* unit_sel, const ViewTable& vt,
                             const void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s,
                             TileCache cache) {
    return m.narrow ? launch_unit2(as_tet<true>(m), tf, unit_sel, vt, moments, color, mode, ctr, s, cache)
                    : launch_unit2(as_tet<false>(m), tf, unit_sel, vt, moments, color, mode, ctr, s, cache);
}

cudaError_t launch_pass1_piece(const TetD& m, const float4* tf, const int32_t* pou, int32_t piece, const PieceBox& box,
                               const ViewTable& vt, int32_t slot, int32_t n_slots, void* moments, Counters* ctr,
                               cudaStream_t s) {
    return m.narrow ? launch_piece1(as_tet<true>(m), tf, pou, piece, box, vt, slot, n_slots, moments, ctr, s)
                    : launch_piece1(as_tet<false>(m), tf, pou, piece, box, vt, slot, n_slots, moments, ctr, s);
}

cudaError_t launch_pass2_piece(const TetD& m, const float4* tf, const int32_t* pou, int32_t piece, const PieceBox& box,
                               const ViewTable& vt, int32_t slot, int32_t n_slots, const void* moments, float* color,
                               Counters* ctr, cudaStream_t s) {
    return m.narrow ? launch_piece2(as_tet<true>(m), tf, pou, piece, box, vt, slot, n_slots, moments, color, ctr, s)
                    : launch_piece2(as_tet<false>(m), tf, pou, piece, box, vt, slot, n_slots, moments, color, ctr, s);
}

cudaError_t launch_sortlast_march(bool fill, const TetD& m, const float4* tf, const int32_t* pou, int32_t piece,
                                  const PieceBox& box, const ViewTable& vt, int32_t slot, int32_t n_slots,
                                  int32_t* counts, const int64_t* starts, int32_t* seg_key, float4* seg_col,
                                  cudaStream_t s) {
    return m.narrow ? launch_sortlast(fill, as_tet<true>(m), tf, pou, piece, box, vt, slot, n_slots, counts, starts,
                                      seg_key, seg_col, s)
                    : launch_sortlast(fill, as_tet<false>(m), tf, pou, piece, box, vt, slot, n_slots, counts, starts,
                                      seg_key, seg_col, s);
}

cudaError_t launch_tet_values(int4* corners, const int4* cells, int64_t n_tets, const float* values, cudaStream_t s) {
    const int64_t nb = (n_tets + 255) / 256;
    k_tet_values<<<(unsigned)(nb < 4096 ? (nb > 0 ? nb : 1) : 4096), 256, 0, s>>>(corners, cells, n_tets, values);
    return cudaGetLastError();
}

}  // namespace mb
