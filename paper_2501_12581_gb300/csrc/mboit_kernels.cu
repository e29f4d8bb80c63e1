// Image-space kernels of the MBOIT puzzle-piece render for sm_103a: the two
// compensated image sums (the paper's Allreduce and Reduce adds), the
// resolve, the sort-last baseline's offsets / sort / blend, the frame
// cache's row count, and the kernel set-up.
#include <map>
#include <mutex>
#include <utility>

#include "mboit_common.cuh"
#include "mboit_multi.h"

namespace mb {
namespace {

// Per pixel: total segments over the pieces, and each (piece, pixel) run of
// counts turned into start offsets in place (given the pixel's base offset).
__global__ void k_sortlast_totals(const ViewTable vt, int n_slots, const int32_t* __restrict__ counts,
                                  int32_t* __restrict__ totals, int64_t total_px) {
    for (int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gp < total_px;
         gp += (int64_t)gridDim.x * blockDim.x) {
        int vi = 0;
        while (vi + 1 < vt.n && gp >= vt.s[vi + 1].color_off / 4) ++vi;
        const ViewSlot& S = vt.s[vi];
        const int64_t npix = (int64_t)S.v.width * S.v.height, local = gp - S.color_off / 4;
        const int32_t* c = counts + (S.color_off / 4) * n_slots + local;
        int32_t sum = 0;
        for (int j = 0; j < n_slots; ++j) sum += c[j * npix];
        totals[gp] = sum;
    }
}

__global__ void k_sortlast_starts(const ViewTable vt, int n_slots, const int32_t* __restrict__ counts,
                                  const int64_t* __restrict__ base, int64_t* __restrict__ starts, int64_t total_px) {
    for (int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gp < total_px;
         gp += (int64_t)gridDim.x * blockDim.x) {
        int vi = 0;
        while (vi + 1 < vt.n && gp >= vt.s[vi + 1].color_off / 4) ++vi;
        const ViewSlot& S = vt.s[vi];
        const int64_t npix = (int64_t)S.v.width * S.v.height, local = gp - S.color_off / 4;
        const int64_t off = (S.color_off / 4) * n_slots + local;
        int64_t run = base[gp];
        for (int j = 0; j < n_slots; ++j) {
            starts[off + j * npix] = run;
            run += counts[off + j * npix];
        }
    }
}

// Exclusive scan of int32 counts into int64 offsets, out[n] = total
// (three phases: 1024-element blocks, block sums, block offsets).
__global__ void __launch_bounds__(1024) k_scan_blocks(const int32_t* __restrict__ in, int64_t* __restrict__ out,
                                                      int64_t* __restrict__ bsum, int64_t n) {
    __shared__ int64_t wtot[32];
    const int64_t i = blockIdx.x * 1024ll + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t x = i < n ? in[i] : 0;
    int64_t v = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += y;
    }
    if (lane == 31) wtot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int64_t w = wtot[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        wtot[lane] = w;
    }
    __syncthreads();
    const int64_t incl = v + (warp > 0 ? wtot[warp - 1] : 0);
    if (i < n) out[i] = incl - x;
    if (threadIdx.x == 1023) bsum[blockIdx.x] = incl;
}

__global__ void __launch_bounds__(1024) k_scan_sums(int64_t* __restrict__ bsum, int64_t nb, int64_t* __restrict__ total) {
    __shared__ int64_t wtot[32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const int64_t x = i < nb ? bsum[i] : 0;
        int64_t v = x;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += y;
        }
        if (lane == 31) wtot[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int64_t w = wtot[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += y;
            }
            wtot[lane] = w;
        }
        __syncthreads();
        const int64_t incl = v + (warp > 0 ? wtot[warp - 1] : 0) + carry;
        if (i < nb) bsum[i] = incl - x;
        __syncthreads();
        if (threadIdx.x == 1023) carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int64_t* __restrict__ out, const int64_t* __restrict__ bsum, int64_t n) {
    const int64_t i = blockIdx.x * 1024ll + threadIdx.x;
    if (i < n) out[i] += bsum[blockIdx.x];
}

// Per pixel: sort its segments by first lattice index (insertion sort; up to
// 64 in registers-backed local arrays, longer lists in place in global
// memory) and composite them front to back.
__global__ void k_sortlast_blend(const int64_t* __restrict__ base, int32_t* __restrict__ seg_key,
                                 float4* __restrict__ seg_col, float* __restrict__ rgba, int64_t total_px,
                                 Counters* __restrict__ ctr) {
    constexpr int kLocal = 64;
    for (int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gp < total_px;
         gp += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = base[gp], n = base[gp + 1] - b;
        float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        float tr = 1.0f;
        if (n <= kLocal) {
            int key[kLocal];
            int idx[kLocal];
            for (int j = 0; j < n; ++j) {
                const int kj = seg_key[b + j];
                int m = j;
                while (m > 0 && key[m - 1] > kj) {
                    key[m] = key[m - 1];
                    idx[m] = idx[m - 1];
                    --m;
                }
                key[m] = kj;
                idx[m] = j;
            }
            for (int j = 0; j < n; ++j) {
                const float4 c = seg_col[b + idx[j]];
                acc.x = ffma(tr, c.x, acc.x);
                acc.y = ffma(tr, c.y, acc.y);
                acc.z = ffma(tr, c.z, acc.z);
                tr *= 1.0f - c.w;
            }
        } else {
            for (int64_t j = 1; j < n; ++j) {
                const int kj = seg_key[b + j];
                const float4 cj = seg_col[b + j];
                int64_t m = j;
                while (m > 0 && seg_key[b + m - 1] > kj) {
                    seg_key[b + m] = seg_key[b + m - 1];
                    seg_col[b + m] = seg_col[b + m - 1];
                    --m;
                }
                seg_key[b + m] = kj;
                seg_col[b + m] = cj;
            }
            for (int64_t j = 0; j < n; ++j) {
                const float4 c = seg_col[b + j];
                acc.x = ffma(tr, c.x, acc.x);
                acc.y = ffma(tr, c.y, acc.y);
                acc.z = ffma(tr, c.z, acc.z);
                tr *= 1.0f - c.w;
            }
        }
        reinterpret_cast<float4*>(rgba)[gp] = make_float4(acc.x, acc.y, acc.z, 1.0f - tr);
        if (n > 0) atomicMax(&ctr->max_segments, (int)n);
    }
}

// ------------------------------------------------------------------------
// image-space reductions (compensated, fixed input order)

struct Neumaier {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
        s = t;
    }
    __device__ __forceinline__ float get() const { return s + c; }
};

__global__ void k_moments_sum(const float4* __restrict__ in, float4* __restrict__ out, int64_t n4, int n_inputs) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        Neumaier x, y, z, w;
        for (int j = 0; j < n_inputs; ++j) {
            const float4 v = __ldg(in + (int64_t)j * n4 + i);
            x.add(v.x);
            y.add(v.y);
            z.add(v.z);
            w.add(v.w);
        }
        out[i] = make_float4(x.get(), y.get(), z.get(), w.get());
    }
}

// Trigonometric slabs: per pixel sum b0 and b0 * tau_j over the inputs
// (compensated), then renormalise and round to the storage format again.
template <int N>
__global__ void k_moments_sum_trig(const __grid_constant__ GridD g, const char* __restrict__ in, char* __restrict__ out,
                                   int64_t plane, int64_t npix, int n_inputs) {
    const int64_t slab = (int64_t)(4 + 4 * N) * plane;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x) {
        Neumaier b0;
        Neumaier tr[N], ti[N];
        for (int j = 0; j < n_inputs; ++j) {
            const char* sl = in + j * slab;
            const float m0 = __ldg(reinterpret_cast<const float*>(sl) + i);
            b0.add(m0);
            for (int k = 0; k < N; ++k) {
                const cf t = unpack16(g, __ldg(reinterpret_cast<const uint32_t*>(sl + 4 * plane * (1 + k)) + i));
                tr[k].add(t.x * m0);
                ti[k].add(t.y * m0);
            }
        }
        const float m0 = b0.get();
        const float inv = m0 > 0.0f ? 1.0f / m0 : 0.0f;
        reinterpret_cast<float*>(out)[i] = m0;
        for (int k = 0; k < N; ++k)
            reinterpret_cast<uint32_t*>(out + 4 * plane * (1 + k))[i] = pack16(g, tr[k].get() * inv, ti[k].get() * inv);
    }
}

__global__ void k_color_resolve(const float4* __restrict__ in, float4* __restrict__ out, const float* __restrict__ b0,
                                int64_t npix, int n_inputs, float4 bg, int raw) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x) {
        Neumaier x, y, z, w;
        for (int j = 0; j < n_inputs; ++j) {
            const float4 v = __ldg(in + (int64_t)j * npix + i);
            x.add(v.x);
            y.add(v.y);
            z.add(v.z);
            w.add(v.w);
        }
        const float4 C = make_float4(x.get(), y.get(), z.get(), w.get());
        out[i] = resolve_pixel(C, raw ? 0.0f : __ldg(b0 + i), bg, raw != 0);
    }
}

// One warp per ray tile: adds the tile's cache rows (kmax - kmin + 1 over its
// rays' exact in-domain intervals, as pass 1 will take them) to *rows.
__global__ void __launch_bounds__(256) k_tile_rows(const __grid_constant__ GridD g, const __grid_constant__ ViewTable vt,
                                                   unsigned long long* __restrict__ rows, int32_t* __restrict__ per_tile) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    unsigned long long mine = 0;
    for (int tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile < vt.total_tiles; tile += warps) {
        const int vi = find_view(vt, tile);
        const ViewSlot& S = vt.s[vi];
        const int lt = tile - S.tile_base;
        int px, py;
        tile_pixel(S, lt, lane, px, py);
        const bool valid = px < S.v.width && py < S.v.height;
        float o[3], d[3];
        int k0, k1;
        ray_range(g, S.v, valid, px, py, o, d, k0, k1);
        const int kmin = __reduce_min_sync(0xffffffffu, k0), kmax = __reduce_max_sync(0xffffffffu, k1);
        if (kmax >= kmin) mine += (unsigned long long)(kmax - kmin + 1);
        if (per_tile && lane == 0) per_tile[tile] = kmax >= kmin ? kmax - kmin + 1 : 0;
    }
    if (lane == 0 && mine) atomicAdd(rows, mine);
}

// ------------------------------------------------------------------------
// table checks of octrees and meshes (failure detection): every entry of a
// library-owned index table is tested against its range before a render's
// passes run; a bad one sets a kErr* bit of the volume's error word, and the
// passes then return at entry (tables_bad), so no out-of-range index is used.

// Ors `code` into *err from one lane of each warp that saw a bad entry.
__device__ __forceinline__ void flag_warp(bool bad, int32_t* err, int32_t code) {
    const unsigned m = __ballot_sync(0xffffffffu, bad);
    if (m && (threadIdx.x & 31) == 0) atomicOr(err, code);
}

// Every ids[i] in [lo, hi].
__global__ void __launch_bounds__(256) k_check_ids(const int32_t* __restrict__ ids, int64_t n, int32_t lo, int32_t hi,
                                                   int32_t* err, int32_t code) {
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i - threadIdx.x % 32 < n; i += stride) {
        if (i < n) {
            const int32_t v = __ldg(ids + i);
            bad |= v < lo || v > hi;
        }
    }
    flag_warp(bad, err, code);
}

// Every face neighbour -1 (boundary) or a tet id.
__global__ void __launch_bounds__(256) k_check_nbrs(const int4* __restrict__ nb, int64_t n, int32_t n_tets,
                                                    int32_t* err) {
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i - threadIdx.x % 32 < n; i += stride) {
        if (i < n) {
            const int4 v = __ldg(nb + i);
            bad |= v.x < -1 || v.x >= n_tets || v.y < -1 || v.y >= n_tets || v.z < -1 || v.z >= n_tets || v.w < -1 ||
                   v.w >= n_tets;
        }
    }
    flag_warp(bad, err, kErrTetId);
}

// Bin offsets non-decreasing from >= 0 to <= the list's length.
__global__ void __launch_bounds__(256) k_check_bins(const int32_t* __restrict__ start, int64_t nbins,
                                                    int32_t n_list, int32_t* err) {
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i - threadIdx.x % 32 < nbins; i += stride) {
        if (i < nbins) {
            const int32_t a = __ldg(start + i), b = __ldg(start + i + 1);
            bad |= a < 0 || b < a || b > n_list;
        }
    }
    flag_warp(bad, err, kErrBinRange);
}

int check_blocks(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (int)(b < 1216 ? (b > 0 ? b : 1) : 1216);  // up to 8 blocks per SM, grid-stride beyond
}

}  // namespace

// Resident CTAs per SM x SMs for a persistent kernel, cached per function.
int persistent_blocks(const void* fn, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find({dev, fn});
    if (it != cache.end()) return it->second;
    int sms = 0, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem);
    const int nb = sms * (occ > 0 ? occ : 1);
    cache[{dev, fn}] = nb;
    return nb;
}

cudaError_t prepare_grid_kernels();
cudaError_t prepare_frame_kernels();
cudaError_t prepare_frame_unit_kernels();
cudaError_t prepare_unit_kernels();

cudaError_t prepare_kernels() {
    // Loads every kernel and fills the occupancy cache, so that no module
    // loading happens later inside a stream capture.
    const void* fns[] = {(const void*)k_moments_sum_trig<3>, (const void*)k_moments_sum_trig<4>,
                         (const void*)k_moments_sum,        (const void*)k_color_resolve,
                         (const void*)k_sortlast_totals,    (const void*)k_sortlast_starts,
                         (const void*)k_scan_blocks,        (const void*)k_scan_sums,
                         (const void*)k_scan_add,           (const void*)k_sortlast_blend,
                         (const void*)k_tile_rows};
    for (const void* f : fns) {
        cudaFuncAttributes a;
        const cudaError_t e = cudaFuncGetAttributes(&a, f);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = prepare_grid_kernels();
    if (e == cudaSuccess) e = prepare_frame_kernels();
    if (e == cudaSuccess) e = prepare_frame_unit_kernels();
    if (e == cudaSuccess) e = prepare_multi_kernels();
    if (e == cudaSuccess) e = prepare_multi_amr_kernels();
    if (e == cudaSuccess) e = prepare_unit_kernels();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_tile_rows(const GridD& g, const ViewTable& vt, unsigned long long* rows, cudaStream_t s,
                             int32_t* per_tile) {
    const int blocks = (vt.total_tiles + 7) / 8;
    k_tile_rows<<<blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096, 256, 0, s>>>(g, vt, rows, per_tile);
    return cudaGetLastError();
}

cudaError_t launch_moments_sum(const GridD& g, const ViewTable& vt, int32_t n_inputs, const void* in, void* out,
                               cudaStream_t s) {
    for (int v = 0; v < vt.n; ++v) {
        const ViewSlot& S = vt.s[v];
        if (g.trig.n) {
            const int64_t npix = (int64_t)S.v.width * S.v.height;
            const char* src = static_cast<const char*>(in) + S.moment_off * n_inputs;
            char* dst = static_cast<char*>(out) + S.moment_off;
            const int blocks = (int)((npix + 255) / 256 < 4096 ? (npix + 255) / 256 : 4096);
            if (g.trig.n == 3)
                k_moments_sum_trig<3><<<blocks > 0 ? blocks : 1, 256, 0, s>>>(g, src, dst, S.plane, npix, n_inputs);
            else
                k_moments_sum_trig<4><<<blocks > 0 ? blocks : 1, 256, 0, s>>>(g, src, dst, S.plane, npix, n_inputs);
            continue;
        }
        // power moments: 2n + 1 float planes (plane is a multiple of 4 pixels)
        const int64_t n4 = (int64_t)(1 + (g.trig.sel ? g.trig.sel : 4)) * S.plane / 4;
        const float4* src = reinterpret_cast<const float4*>(static_cast<const char*>(in) + S.moment_off * n_inputs);
        float4* dst = reinterpret_cast<float4*>(static_cast<char*>(out) + S.moment_off);
        const int blocks = (int)((n4 + 255) / 256 < 4096 ? (n4 + 255) / 256 : 4096);
        k_moments_sum<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(src, dst, n4, n_inputs);
    }
    return cudaGetLastError();
}

cudaError_t launch_color_resolve(const ViewTable& vt, int32_t n_inputs, const float* in, float* out,
                                 const void* moments, float4 bg, int32_t raw_sum, cudaStream_t s) {
    for (int v = 0; v < vt.n; ++v) {
        const ViewSlot& S = vt.s[v];
        const int64_t npix = (int64_t)S.v.width * S.v.height;
        const float4* src = reinterpret_cast<const float4*>(in + S.color_off * n_inputs);
        float4* dst = reinterpret_cast<float4*>(out + S.color_off);
        const float* b0 = moments ? reinterpret_cast<const float*>(static_cast<const char*>(moments) + S.moment_off)
                                  : nullptr;
        const int blocks = (int)((npix + 255) / 256 < 4096 ? (npix + 255) / 256 : 4096);
        k_color_resolve<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(src, dst, b0, npix, n_inputs, bg, raw_sum);
    }
    return cudaGetLastError();
}

cudaError_t launch_sortlast_offsets(const ViewTable& vt, int32_t n_slots, const int32_t* counts, int32_t* totals,
                                   int64_t* base, int64_t* bsum, int64_t* starts, int64_t total_px, cudaStream_t s) {
    const int grid = (int)((total_px + 255) / 256 < 8192 ? (total_px + 255) / 256 : 8192);
    k_sortlast_totals<<<grid, 256, 0, s>>>(vt, n_slots, counts, totals, total_px);
    const int64_t nb = (total_px + 1023) / 1024;
    k_scan_blocks<<<(unsigned)nb, 1024, 0, s>>>(totals, base, bsum, total_px);
    k_scan_sums<<<1, 1024, 0, s>>>(bsum, nb, base + total_px);
    k_scan_add<<<(unsigned)nb, 1024, 0, s>>>(base, bsum, total_px);
    k_sortlast_starts<<<grid, 256, 0, s>>>(vt, n_slots, counts, base, starts, total_px);
    return cudaGetLastError();
}

cudaError_t launch_sortlast_blend(const int64_t* base, int32_t* seg_key, float4* seg_col, float* rgba, int64_t total_px,
                                  Counters* ctr, cudaStream_t s) {
    const int grid = (int)((total_px + 127) / 128 < 16384 ? (total_px + 127) / 128 : 16384);
    k_sortlast_blend<<<grid, 128, 0, s>>>(base, seg_key, seg_col, rgba, total_px, ctr);
    return cudaGetLastError();
}

cudaError_t launch_check_tables(const AmrD& a, cudaStream_t s) {
    const int64_t n = (int64_t)a.fdim * a.fdim * a.fdim;
    k_check_ids<<<check_blocks(n), 256, 0, s>>>(a.fmap, n, -1, a.n_leaves - 1, a.err, kErrLeafId);
    return cudaGetLastError();
}

cudaError_t launch_check_tables(const TetD& m, cudaStream_t s) {
    const int64_t nbins = (int64_t)m.bdim[0] * m.bdim[1] * m.bdim[2];
    k_check_nbrs<<<check_blocks(m.n_tets), 256, 0, s>>>(m.nbrs, m.n_tets, m.n_tets, m.err);
    k_check_bins<<<check_blocks(nbins), 256, 0, s>>>(m.bin_start, nbins, m.n_bin_tets, m.err);
    k_check_ids<<<check_blocks(m.n_bin_tets), 256, 0, s>>>(m.bin_tets, m.n_bin_tets, 0, m.n_tets - 1, m.err, kErrTetId);
    return cudaGetLastError();
}

}  // namespace mb
