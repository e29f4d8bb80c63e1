// Fused, persistent grid passes: kernel selection and launchers (the kernel
// templates and their design are in mboit_grid.cuh).
#include "mboit_grid.cuh"

namespace mb {

// The 6- and 8-power-moment kernels (mboit_grid_power.cu); pass 1 or 2.
const void* grid_power_fn(int pass, int ms, int cfg, bool sel, bool cache);

namespace {

// ms: the moment set's kernel variant (TrigTables::sel)
template <bool kC = false>
const void* pass1_fn(int cfg, bool sel, int ms) {
    switch (ms) {
        case 3: return pass1_fn_ms<3, kC>(cfg, sel);
        case 4: return pass1_fn_ms<4, kC>(cfg, sel);
        case 6:
        case 8: return grid_power_fn(1, ms, cfg, sel, kC);
        default: return pass1_fn_ms<0, kC>(cfg, sel);
    }
}
template <bool kC = false>
const void* pass2_fn(int cfg, bool sel, int ms) {
    switch (ms) {
        case 3: return pass2_fn_ms<3, kC>(cfg, sel);
        case 4: return pass2_fn_ms<4, kC>(cfg, sel);
        case 6:
        case 8: return grid_power_fn(2, ms, cfg, sel, kC);
        default: return pass2_fn_ms<0, kC>(cfg, sel);
    }
}


bool vec_config(int cfg) { return cfg == 2 || cfg == 3 || cfg == 4; }

}  // namespace

bool stage_config_eligible(const GridD& g, int cfg) {
    if (cfg < 0 || cfg >= kNumStageConfigs) return false;
    if (g.trig.sel != 0 && cfg != 0 && cfg != 3) return false;
    if (!vec_config(cfg)) return true;
    return g.nx % 4 == 0 && g.nx >= 4 && (reinterpret_cast<uintptr_t>(g.field) & 15u) == 0;
}

cudaError_t prepare_grid_kernels() {
    const int sets[5] = {0, 3, 4, 6, 8};
    for (int ms : sets)
        for (int cfg = 0; cfg < kNumStageConfigs; ++cfg)
            for (int sel = 0; sel < 2; ++sel) {
                const void* fs[4] = {pass1_fn(cfg, sel, ms), pass2_fn(cfg, sel, ms), pass1_fn<true>(cfg, sel, ms),
                                     pass2_fn<true>(cfg, sel, ms)};
                for (const void* f : fs) {
                    cudaFuncAttributes a;
                    const cudaError_t e = cudaFuncGetAttributes(&a, f);
                    if (e != cudaSuccess) return e;
                    persistent_blocks(f, 256, 0);
                }
            }
    return cudaSuccess;
}

cudaError_t launch_pass1_fused(const GridD& g, const float4* tf, const uint8_t* brick_sel, const ViewTable& vt,
                               void* moments, Counters* ctr, cudaStream_t s, int cfg, TileCache cache) {
    if (!stage_config_eligible(g, cfg)) cfg = 0;
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[0], 0, sizeof(int32_t), s);
    if (e == cudaSuccess && cache.vals) e = cudaMemsetAsync(&ctr->cache_rows, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const bool sel = brick_sel != nullptr;
    const void* fn = cache.vals ? pass1_fn<true>(cfg, sel, g.trig.sel) : pass1_fn(cfg, sel, g.trig.sel);
    char* m = static_cast<char*>(moments);
    void* args[] = {(void*)&g, (void*)&tf, (void*)&brick_sel, (void*)&vt, (void*)&m, (void*)&ctr, (void*)&cache};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

cudaError_t launch_pass2_fused(const GridD& g, const float4* tf, const uint8_t* brick_sel, const ViewTable& vt,
                               const void* moments, float* color, int32_t mode, Counters* ctr, cudaStream_t s,
                               int cfg, TileCache cache) {
    if (!stage_config_eligible(g, cfg)) cfg = 0;
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[1], 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const bool sel = brick_sel != nullptr;
    const void* fn = cache.vals ? pass2_fn<true>(cfg, sel, g.trig.sel) : pass2_fn(cfg, sel, g.trig.sel);
    const char* m = static_cast<const char*>(moments);
    int md = mode;
    void* args[] = {(void*)&g, (void*)&tf, (void*)&brick_sel, (void*)&vt, (void*)&m, (void*)&color, (void*)&md,
                    (void*)&ctr, (void*)&cache};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}


}  // namespace mb
