// The 6- and 8-power-moment instantiations of the fused grid passes
// (templates in mboit_grid.cuh), in a translation unit of their own so that
// they compile in parallel with the rest.
#include "mboit_grid.cuh"

namespace mb {

const void* grid_power_fn(int pass, int ms, int cfg, bool sel, bool cache) {
    if (pass == 1) {
        if (ms == 6) return cache ? pass1_fn_ms<6, true>(cfg, sel) : pass1_fn_ms<6, false>(cfg, sel);
        return cache ? pass1_fn_ms<8, true>(cfg, sel) : pass1_fn_ms<8, false>(cfg, sel);
    }
    if (ms == 6) return cache ? pass2_fn_ms<6, true>(cfg, sel) : pass2_fn_ms<6, false>(cfg, sel);
    return cache ? pass2_fn_ms<8, true>(cfg, sel) : pass2_fn_ms<8, false>(cfg, sel);
}

}  // namespace mb
