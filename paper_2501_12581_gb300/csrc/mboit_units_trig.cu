// The trigonometric-moment instantiations (3 and 4 complex moments) of the
// octree / mesh passes and of the per-piece kernels (templates in
// mboit_units.cuh), in a translation unit of their own so that they compile
// in parallel with the rest.
#include "mboit_units.cuh"

namespace mb {
namespace {

template <class V, int MS>
const void* unit_fn(int pass, bool sel, bool cache) {
    if (pass == 1)
        return sel ? (cache ? (const void*)k_pass1_unit<V, true, MS, true> : (const void*)k_pass1_unit<V, true, MS, false>)
                   : (cache ? (const void*)k_pass1_unit<V, false, MS, true> : (const void*)k_pass1_unit<V, false, MS, false>);
    return sel ? (cache ? (const void*)k_pass2_unit<V, true, MS, true> : (const void*)k_pass2_unit<V, true, MS, false>)
               : (cache ? (const void*)k_pass2_unit<V, false, MS, true> : (const void*)k_pass2_unit<V, false, MS, false>);
}

template <class V>
const void* unit_fn_ms(int pass, int ms, bool sel, bool cache) {
    return ms == 3 ? unit_fn<V, 3>(pass, sel, cache) : unit_fn<V, 4>(pass, sel, cache);
}

template <class V>
const void* piece_fn(int pass, int ms) {
    if (pass == 1) return ms == 3 ? (const void*)k_pass1_piece<V, 3> : (const void*)k_pass1_piece<V, 4>;
    return ms == 3 ? (const void*)k_pass2_piece<V, 3> : (const void*)k_pass2_piece<V, 4>;
}

}  // namespace

// vkind: 0 grid (per-piece kernels only), 1 octree, 2 narrow mesh, 3 wide mesh.
const void* unit_trig_fn(int vkind, int pass, int ms, bool sel, bool cache) {
    switch (vkind) {
        case 1: return unit_fn_ms<AmrD>(pass, ms, sel, cache);
        case 2: return unit_fn_ms<TetT<true>>(pass, ms, sel, cache);
        default: return unit_fn_ms<TetT<false>>(pass, ms, sel, cache);
    }
}

const void* piece_trig_fn(int vkind, int pass, int ms) {
    switch (vkind) {
        case 0: return piece_fn<GridD>(pass, ms);
        case 1: return piece_fn<AmrD>(pass, ms);
        case 2: return piece_fn<TetT<true>>(pass, ms);
        default: return piece_fn<TetT<false>>(pass, ms);
    }
}

}  // namespace mb
