// Fused, persistent grid passes: kernel selection and launchers (the kernel
// templates and their design are in mboit_grid.cuh).
#include <cstring>

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


bool vec_config(int cfg) { return cfg >= 2 && cfg <= 6; }

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
                               void* moments, Counters* ctr, cudaStream_t s, int cfg, TileCache cache,
                               const CUtensorMap* tmap) {
    if (!stage_config_eligible(g, cfg)) cfg = 0;
    if ((cfg == 5 || cfg == 6) && !tmap) cfg = 3;   // no tensor map: a window by plain loads
    cudaError_t e = cudaMemsetAsync(&ctr->tile_next[0], 0, sizeof(int32_t), s);
    if (e == cudaSuccess && cache.vals) e = cudaMemsetAsync(&ctr->cache_rows, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const bool sel = brick_sel != nullptr;
    const void* fn = cache.vals ? pass1_fn<true>(cfg, sel, g.trig.sel) : pass1_fn(cfg, sel, g.trig.sel);
    char* m = static_cast<char*>(moments);
    CUtensorMap map;
    if (tmap)
        map = *tmap;
    else
        std::memset(&map, 0, sizeof map);   // not read by configurations without TMA
    void* args[] = {(void*)&g, (void*)&tf, (void*)&brick_sel, (void*)&vt, (void*)&m, (void*)&ctr, (void*)&cache,
                    (void*)&map};
    return cudaLaunchKernel(fn, dim3(persistent_blocks(fn, 256, 0)), dim3(256), args, 0, s);
}

bool encode_field_maps(const GridD& g, CUtensorMap out[2]) {
    if (!stage_config_eligible(g, 5)) return false;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return false;
    }
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nx * g.ny * 4};   // bytes, dims 1 and 2
    const cuuint32_t boxes[2][3] = {{(cuuint32_t)Stage5::WX, (cuuint32_t)Stage5::WY, (cuuint32_t)Stage5::WZ},
                                    {(cuuint32_t)Stage6::WX, (cuuint32_t)Stage6::WY, (cuuint32_t)Stage6::WZ}};
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int i = 0; i < 2; ++i) {
        const CUresult r = reinterpret_cast<Encode>(fn)(out + i, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                                                        const_cast<float*>(g.field), dims, strides, boxes[i], estr,
                                                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    return true;
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
