// Fused, persistent grid passes of the MBOIT puzzle-piece render for sm_103a.
//
// Work decomposition.  One thread marches one ray; a warp owns an 8 x 4
// pixel tile, so the 32 rays of a warp are spatial neighbours and their
// trilinear gathers at the same lattice index hit a few adjacent cache lines.
// The fused passes are persistent: grid = SMs x resident CTAs, each warp pops
// tiles from an atomic work-queue head (no waits, no spins), which balances
// long centre rays against short silhouette rays.  The transfer function
// (256 x float4, 4 KB) is staged once per CTA in shared memory.
//
// Pass 1 (Sec. 4.1, Alg. 2) accumulates b_j += a z^j in registers over all
// selected pieces: summing the pieces' moment images (the Allreduce add) is
// done in registers because addition commutes.  Pass 2 (Sec. 4.2, Alg. 1
// loop 2, Alg. 3) builds the per-pixel reconstruction frame from the global
// moments once per ray (float-float FP32; FP64 for near-singular Hankel
// matrices), then adds T * alpha * (r, g, b, 1) per sample in FP32; the resolved mode also applies the renormalisation (Sec. 4.3) in
// the epilogue, so the frame needs no separate colour reduction.
//
// In a batched frame (mboit_render_frame) pass 1 also stores every lattice
// point's value in the frame's tile-row cache, and pass 2 reads those rows
// (prefetched into the warp's shared-memory slot) instead of marching the
// field again; a tile that found no room is marched again.  The per-piece
// kernels (mboit_units.cu) are the plain form.
//
// This header holds the kernel templates; mboit_grid.cu selects and launches
// them (four power and trigonometric moments), mboit_grid_power.cu holds the
// 6- and 8-power-moment instantiations, compiled in parallel.
#pragma once
#include "mboit_common.cuh"

namespace mb {
namespace {

// ------------------------------------------------------------------------
// fused, persistent passes
//
// Warp-cooperative staging.  The 32 rays of a warp advance in lockstep over
// the lattice index k; at one k their sample points lie a few voxels apart.
// For a window of S consecutive indices the warp takes the bounding box of
// the cells its samples can touch (from the exact float32 positions of each
// lane's first and last sample in the window: positions are monotone in t,
// so every sample in between lies inside), and if the box fits a WX x WY x WZ
// block, the warp copies that block of the field into its own shared-memory
// slot once, then reads all trilinear corners from shared memory.  Each field
// row is fetched once per window instead of eight times per lattice step.  A
// box that does not fit (widely spread rays) falls back to direct loads.

template <int S_, int WX_, int WY_, int WZ_, bool kVec_, bool kTma_ = false>
struct StageCfg {
    static constexpr int S = S_, WX = WX_, WY = WY_, WZ = WZ_;
    static constexpr bool kVec = kVec_;  // 16-byte loads: x origin rounded down to a multiple of 4
    static constexpr bool kTma = kTma_;  // the window arrives by one tensor copy (TMA) of the warp
    // scalar windows pad rows to an odd pitch; vector windows keep 16-byte rows
    // and shift each plane by 4 floats, both to spread shared-memory banks; a
    // TMA window is the box as the copy lays it out, [z][y][x] without padding
    static constexpr int Pitch = kVec_ ? WX_ : WX_ + 1;
    static constexpr int Plane = kTma_ ? WY_ * WX_ : (kVec_ ? WY_ * WX_ + 4 : WY_ * (WX_ + 1));
    static constexpr int Floats = WZ_ * Plane;
    static constexpr int Elems = WX_ * WY_ * WZ_;
    static_assert(!kVec_ || WX_ % 4 == 0, "vector windows need a multiple of 4 in x");
    static_assert(!kTma_ || (kVec_ && Floats % 32 == 0), "TMA windows start on the x-origin rule and 128-byte slots");
};
// The configurations the autotuner chooses from (index = tuning id).
using Stage0 = StageCfg<6, 8, 8, 8, false>;
using Stage1 = StageCfg<8, 8, 8, 8, false>;
using Stage2 = StageCfg<6, 12, 8, 8, true>;
using Stage3 = StageCfg<6, 16, 8, 8, true>;
using Stage4 = StageCfg<8, 16, 8, 10, true>;
using Stage5 = StageCfg<6, 16, 8, 8, true, true>;   // configuration 3's window by TMA
// A TMA window keeps the box's dense layout, so its planes cannot be shifted
// the way configuration 3's are; rows of 12 floats in planes of 11 rows (132
// floats, 4 banks apart) spread the corner gathers' banks about as well.
using Stage6 = StageCfg<6, 12, 11, 8, true, true>;

// ------------------------------------------------------------------------
// TMA window loads.  One lane of the warp arms the warp's mbarrier with the
// window's byte count and issues cp.async.bulk.tensor.3d from the field's
// tensor map (encoded on the host: dims nx, ny, nz, box WX x WY x WZ floats,
// no swizzle, zero fill outside the field, which no sample reads); every lane
// then waits on the barrier's phase.  The x coordinate is a multiple of 4
// floats (16 bytes), as the tiled copy requires.  A wait gives up after
// kTmaSpin polls: the kernel records kErrTmaTimeout, waits once more, bounded,
// for the copy in flight, and returns.

constexpr int kTmaSpin = 1 << 20;      // polls of at most ~1 us each (the suspend-time hint): ~1 s in all

struct TmaWin {
    const CUtensorMap* map;    // the field's tensor map (a __grid_constant__ kernel parameter)
    uint64_t* bar;             // this warp's mbarrier
    unsigned phase;            // parity of its next completion
    int32_t* err;              // the volume's error word
    bool no_copy;              // kFlagDebugNoCopy: arm the barrier, issue no copy
};

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    for (int i = 0; i < kTmaSpin; ++i) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Copies the WX x WY x WZ box at (x, y, z) of the field into `win` (this
// warp's 128-byte aligned slot); all 32 lanes call it.  False when the copy
// did not complete in time.
template <class Cfg>
__device__ __forceinline__ bool tma_window(TmaWin& tw, float* win, int x, int y, int z) {
    const unsigned bar = smem_addr(tw.bar);
    if ((threadIdx.x & 31) == 0) {
        constexpr unsigned bytes = Cfg::Elems * 4;
        // the lanes' earlier reads of the slot (ordered by the caller's
        // __syncwarp) before the copy's writes
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        if (!tw.no_copy)
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4}], [%5];" ::"r"(smem_addr(win)),
                "l"(reinterpret_cast<uint64_t>(tw.map)), "r"(x), "r"(y), "r"(z), "r"(bar)
                : "memory");
    }
    // one outcome for the warp: lanes that saw the phase complete and a lane
    // that gave up must not part (the caller returns on false)
    const bool ok = __all_sync(0xffffffffu, mbar_wait(bar, tw.phase));
    if (!ok) {
        if ((threadIdx.x & 31) == 0) atomicOr(tw.err, kErrTmaTimeout);
        mbar_wait(bar, tw.phase);   // the copy in flight, once more, bounded
    }
    tw.phase ^= 1u;
    return ok;
}

// Initialises the warps' barriers (one arrival per phase); before the
// kernel's first __syncthreads.
template <class Cfg>
__device__ __forceinline__ void tma_init(uint64_t* bars) {
    if constexpr (Cfg::kTma) {
        if ((threadIdx.x & 31) == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bars + (threadIdx.x >> 5))) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
}

// Bounding box of the cells that lane samples in [ka, kz] can touch, reduced
// over the warp; true if it fits the window.
template <class Cfg>
__device__ __forceinline__ bool window_box(const GridD& g, const float o[3], const float d[3], int ka, int kz,
                                           int LO[3]) {
    const unsigned full = 0xffffffffu;
    const int nmax[3] = {g.nx - 1, g.ny - 1, g.nz - 1};
    int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, hi[3] = {-1, -1, -1};
    if (ka <= kz) {
        const float ta = lattice_t(ka, g.step), tz = lattice_t(kz, g.step);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float pa = ffma(ta, d[c], o[c]), pz = ffma(tz, d[c], o[c]);
            lo[c] = max((int)floorf(fmin_(pa, pz)), 0);
            hi[c] = min((int)floorf(fmax_(pa, pz)) + 1, nmax[c]);
        }
    }
    bool fits = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        LO[c] = __reduce_min_sync(full, lo[c]);
        const int HI = __reduce_max_sync(full, hi[c]);
        if (c == 0 && Cfg::kVec) LO[0] &= ~3;
        const int ext = c == 0 ? Cfg::WX : (c == 1 ? Cfg::WY : Cfg::WZ);
        fits = fits && HI >= LO[c] && HI - LO[c] < ext;
    }
    return fits;
}


// Marches the lattice indices [k0, k1] of this lane's ray (exactly the
// in-domain points; k0 > k1: none), calling body(t, xt) with the table
// coordinate xt of every owned sample in depth order (and storing xt, NaN for
// a point not sampled).  All 32 lanes of the warp call it together.
// Returns false when a TMA window did not arrive in time (the kernel must
// stop; kErrTmaTimeout is recorded).
template <class Cfg, bool kSel, class Body, class Store = NoStore>
__device__ __forceinline__ bool march_fused(const GridD& g, const uint8_t* __restrict__ sel, float* __restrict__ win,
                                            const float o[3], const float d[3], int k0, int k1, Body& body,
                                            Store store = Store{}, TmaWin* tma = nullptr) {
    const unsigned full = 0xffffffffu;
    const int kmin = __reduce_min_sync(full, k0);
    const int kmax = __reduce_max_sync(full, k1);
    const int nmax[3] = {g.nx - 1, g.ny - 1, g.nz - 1};
    for (int kb = kmin; kb <= kmax;) {
        // the longest window (2S, then S steps) whose box fits
        int LO[3];
        int ke = min(kb + 2 * Cfg::S - 1, kmax);
        bool fits = window_box<Cfg>(g, o, d, max(kb, k0), min(ke, k1), LO);
        if (!fits && ke > kb + Cfg::S - 1) {
            ke = kb + Cfg::S - 1;
            fits = window_box<Cfg>(g, o, d, max(kb, k0), min(ke, k1), LO);
        }
        const int ka = max(kb, k0), kz = min(ke, k1);
        if (fits) {
            __syncwarp();
            const int lane = threadIdx.x & 31;
            if constexpr (Cfg::kTma) {
                if (!tma_window<Cfg>(*tma, win, LO[0], LO[1], LO[2])) return false;
            } else if (Cfg::kVec) {
                // nx % 4 == 0 and a 16-byte aligned field (checked by the launcher):
                // every chunk start gx is a multiple of 4 and gx + 3 < nx
                constexpr int QX = Cfg::WX / 4;
                if (QX * Cfg::WY == 32) {
                    // one plane per warp-wide step: lane -> fixed (xq, y), z = step
                    const int xq = lane % QX, y = lane / QX;
                    const int gx = min(LO[0] + 4 * xq, g.nx - 4), gy = min(LO[1] + y, nmax[1]);
                    const float* src = g.field + (size_t)gy * g.nx + gx;
                    float* dst = win + y * Cfg::Pitch + 4 * xq;
                    const size_t zs = (size_t)g.nx * g.ny;
#pragma unroll
                    for (int z = 0; z < Cfg::WZ; ++z) {
                        const int gz = min(LO[2] + z, nmax[2]);
                        *reinterpret_cast<float4*>(dst + z * Cfg::Plane) =
                            __ldg(reinterpret_cast<const float4*>(src + gz * zs));
                    }
                } else {
#pragma unroll 2
                    for (int e = lane; e < QX * Cfg::WY * Cfg::WZ; e += 32) {
                        const int xq = e % QX, y = (e / QX) % Cfg::WY, z = e / (QX * Cfg::WY);
                        const int gx = min(LO[0] + 4 * xq, g.nx - 4), gy = min(LO[1] + y, nmax[1]),
                                  gz = min(LO[2] + z, nmax[2]);
                        *reinterpret_cast<float4*>(win + z * Cfg::Plane + y * Cfg::Pitch + 4 * xq) = __ldg(
                            reinterpret_cast<const float4*>(g.field + ((size_t)gz * g.ny + gy) * (size_t)g.nx + gx));
                    }
                }
            } else {
#pragma unroll 4
                for (int e = lane; e < Cfg::Elems; e += 32) {
                    const int x = e % Cfg::WX, y = (e / Cfg::WX) % Cfg::WY, z = e / (Cfg::WX * Cfg::WY);
                    const int gx = min(LO[0] + x, nmax[0]), gy = min(LO[1] + y, nmax[1]), gz = min(LO[2] + z, nmax[2]);
                    win[z * Cfg::Plane + y * Cfg::Pitch + x] =
                        __ldg(g.field + ((size_t)gz * g.ny + gy) * (size_t)g.nx + gx);
                }
            }
            __syncwarp();
            const float* wbase = win - LO[2] * Cfg::Plane - LO[1] * Cfg::Pitch - LO[0];
            // t_{k+1} = t_k + step exactly (odd multiples of step/2 below 2^24), so the
            // loop runs on t itself
            const float tz = lattice_t(kz, g.step);
            store.seek(ka);
            float t0 = lattice_t(ka, g.step);
            if constexpr (!kSel) {
                // two points at a time: both positions, then both points' 16
                // window reads, then the store and the body in order
                auto window_value = [&](float t) {
                    const float p0 = ffma(t, d[0], o[0]), p1 = ffma(t, d[1], o[1]), p2 = ffma(t, d[2], o[2]);
                    const int ix = (int)p0, iy = (int)p1, iz = (int)p2;
                    const float* c = wbase + iz * Cfg::Plane + iy * Cfg::Pitch + ix;
                    return tf_x(g, trilinear8(c[0], c[1], c[Cfg::Pitch], c[Cfg::Pitch + 1], c[Cfg::Plane],
                                              c[Cfg::Plane + 1], c[Cfg::Plane + Cfg::Pitch],
                                              c[Cfg::Plane + Cfg::Pitch + 1], p0 - (float)ix, p1 - (float)iy,
                                              p2 - (float)iz));
                };
                for (; t0 + g.step <= tz; t0 += 2.0f * g.step) {
                    const float tb = t0 + g.step;
                    const float xa = window_value(t0), xb = window_value(tb);
                    store.put(xa);
                    body(t0, xa);
                    store.put(xb);
                    body(tb, xb);
                }
            }
            for (float t = t0; t <= tz; t += g.step) {
                const float p0 = ffma(t, d[0], o[0]), p1 = ffma(t, d[1], o[1]), p2 = ffma(t, d[2], o[2]);
                const int ix = (int)p0, iy = (int)p1, iz = (int)p2;
                if (kSel) {
                    const int b = ((iz >> g.brick_log2) * g.nby + (iy >> g.brick_log2)) * g.nbx + (ix >> g.brick_log2);
                    if (!__ldg(sel + b)) {
                        store.put(__int_as_float(0x7fc00000));
                        continue;
                    }
                }
                const float* c = wbase + iz * Cfg::Plane + iy * Cfg::Pitch + ix;
                const float val = trilinear8(c[0], c[1], c[Cfg::Pitch], c[Cfg::Pitch + 1], c[Cfg::Plane],
                                             c[Cfg::Plane + 1], c[Cfg::Plane + Cfg::Pitch],
                                             c[Cfg::Plane + Cfg::Pitch + 1], p0 - (float)ix, p1 - (float)iy,
                                             p2 - (float)iz);
                const float xt = tf_x(g, val);
                store.put(xt);
                body(t, xt);
            }
        } else {
            const float tz = lattice_t(kz, g.step);
            store.seek(ka);
            for (float t = lattice_t(ka, g.step); t <= tz; t += g.step) {
                float val;
                if (!field_sample<kSel>(g, sel, t, o, d, val)) {
                    store.put(__int_as_float(0x7fc00000));
                    continue;
                }
                const float xt = tf_x(g, val);
                store.put(xt);
                body(t, xt);
            }
        }
        kb = ke + 1;
    }
    return true;
}


// Pass 2 marching the field: with four power moments, a warp whose lanes
// with samples all have a generic frame takes the body without the
// per-sample test of the frame's kind (the same arithmetic and result).
template <class Cfg, bool kSel, class Body>
__device__ __forceinline__ bool blend_fused(const GridD& g, const uint8_t* __restrict__ sel, float* __restrict__ win,
                                            const float o[3], const float d[3], int k0, int k1, Body& body,
                                            TmaWin* tma = nullptr) {
    if constexpr (std::is_same<Body, BlendBody>::value) {
        if (__all_sync(0xffffffffu, k0 > k1 || body.F.kind == kFrameGeneric)) {
            GenericBlend gb{body};
            return march_fused<Cfg, kSel>(g, sel, win, o, d, k0, k1, gb, NoStore{}, tma);
        }
    }
    return march_fused<Cfg, kSel>(g, sel, win, o, d, k0, k1, body, NoStore{}, tma);
}

template <bool kSel, class Cfg, int MS, bool kCache = false>
__global__ void __launch_bounds__(256, MS == 0 ? 5 : 1) k_pass1_fused(const __grid_constant__ GridD g, const float4* __restrict__ tf,
                                                     const uint8_t* __restrict__ sel, const __grid_constant__ ViewTable vt,
                                                     char* __restrict__ moments, Counters* __restrict__ ctr,
                                                     const TileCache cache, const __grid_constant__ CUtensorMap tmap) {
    __shared__ float2 s_sig[256];
    __shared__ __align__(128) float s_win[kFusedWarps][Cfg::Floats];
    __shared__ __align__(8) uint64_t s_bar[Cfg::kTma ? kFusedWarps : 1];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float s0 = tf[i].w;
        s_sig[i] = make_float2(s0, i < 255 ? tf[i + 1].w - s0 : 0.0f);
    }
    tma_init<Cfg>(s_bar);
    __syncthreads();
    float* win = s_win[threadIdx.x >> 5];
    TmaWin tw{&tmap, s_bar + (Cfg::kTma ? threadIdx.x >> 5 : 0), 0u, &ctr->error, (g.flags & kFlagDebugNoCopy) != 0};
    int vi, px, py, tile;
    while (next_tile(vt, &ctr->tile_next[0], vi, px, py, tile)) {
        const ViewSlot& S = vt.s[vi];
        const bool valid = px < S.v.width && py < S.v.height;
        float o[3], d[3];
        int k0, k1;
        ray_range(g, S.v, valid, px, py, o, d, k0, k1);
        auto body = make_moment_body<MS>(s_sig, g, S.v);
        bool ok;
        if constexpr (kCache) {
            RowStore st{tile_rows(cache, ctr, tile, k0, k1)};
            ok = march_fused<Cfg, kSel>(g, sel, win, o, d, k0, k1, body, st, &tw);
        } else {
            ok = march_fused<Cfg, kSel>(g, sel, win, o, d, k0, k1, body, NoStore{}, &tw);
        }
        if (!ok) return;
        if (valid) body.store(g, moments, S, S.moment_off, py * S.v.width + px);
        warp_add_u64(&ctr->samples[0], body.n);
    }
}

template <bool kSel, class Cfg, int MS, bool kCache = false>
__global__ void __launch_bounds__(256) k_pass2_fused(const __grid_constant__ GridD g, const float4* __restrict__ tf,
                                                     const uint8_t* __restrict__ sel, const __grid_constant__ ViewTable vt,
                                                     const char* __restrict__ moments, float* __restrict__ color,
                                                     int mode, Counters* __restrict__ ctr, const TileCache cache) {
    static_assert(Cfg::Floats >= kRowBuf && Cfg::Floats % 4 == 0, "the window slot doubles as the row buffer");
    __shared__ float4 s_tf[512];
    __shared__ __align__(16) float s_win[kFusedWarps][Cfg::Floats];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const float4 e0 = tf[i], e1 = i < 255 ? tf[i + 1] : tf[i];
        s_tf[2 * i] = e0;
        s_tf[2 * i + 1] = make_float4(e1.x - e0.x, e1.y - e0.y, e1.z - e0.z, e1.w - e0.w);
    }
    __syncthreads();
    // a pass 1 that gave up on a window load left some tiles' cache bases
    // unwritten: nothing of this pass is valid then, and no stale base is read
    if (kCache && (*(volatile const int32_t*)&ctr->error & kErrTmaTimeout)) return;
    float* win = s_win[threadIdx.x >> 5];
    const bool raw = (g.flags & 1u) != 0;
    int vi, px, py, tile;
    while (next_tile(vt, &ctr->tile_next[1], vi, px, py, tile)) {
        const ViewSlot& S = vt.s[vi];
        const bool valid = px < S.v.width && py < S.v.height;
        const int pix = valid ? py * S.v.width + px : 0;
        auto body = make_blend_body<MS>(s_tf, g, S, moments, S.moment_off, pix, valid);
        count_frames(ctr, body, valid);
        float o[3], d[3];
        int k0, k1;
        ray_range(g, S.v, valid, px, py, o, d, k0, k1);
        const long long tb = kCache ? cache.tile_base[tile] : -1;
        if (kCache && tb >= 0) {
            const int kmin = __reduce_min_sync(0xffffffffu, k0), kmax = __reduce_max_sync(0xffffffffu, k1);
            blend_rows<kSel>(g, cache.vals + tb * 32, kmin, kmax, k0, k1, win, body);
        } else {
            blend_fused<Cfg, kSel>(g, sel, win, o, d, k0, k1, body);   // pass 2 has no TMA windows
        }
        if (valid) {
            float4* out = reinterpret_cast<float4*>(color + S.color_off) + pix;
            if (mode == kColorResolved)
                *out = resolve_pixel(body.C, body.b0, make_float4(0.0f, 0.0f, 0.0f, 0.0f), raw);
            else
                *out = body.C;
        }
        warp_add_u64(&ctr->samples[1], body.n);
    }
}

template <int MS, bool kC>
const void* pass1_fn_ms(int cfg, bool sel) {
    if (sel) return (const void*)k_pass1_fused<true, Stage0, MS, kC>;
    if constexpr (MS != 0) {
        // other moment sets: configurations 0 and 3 only
        return cfg == 3 || cfg == 5 || cfg == 6 ? (const void*)k_pass1_fused<false, Stage3, MS, kC>
                                                : (const void*)k_pass1_fused<false, Stage0, MS, kC>;
    } else {
        switch (cfg) {
            case 1: return (const void*)k_pass1_fused<false, Stage1, MS, kC>;
            case 2: return (const void*)k_pass1_fused<false, Stage2, MS, kC>;
            case 3: return (const void*)k_pass1_fused<false, Stage3, MS, kC>;
            case 4: return (const void*)k_pass1_fused<false, Stage4, MS, kC>;
            case 5: return (const void*)k_pass1_fused<false, Stage5, MS, kC>;
            case 6: return (const void*)k_pass1_fused<false, Stage6, MS, kC>;
            default: return (const void*)k_pass1_fused<false, Stage0, MS, kC>;
        }
    }
}

template <int MS, bool kC>
const void* pass2_fn_ms(int cfg, bool sel) {
    if (sel) return (const void*)k_pass2_fused<true, Stage0, MS, kC>;
    if constexpr (MS != 0) {
        // other moment sets: configurations 0 and 3 only
        return cfg == 3 || cfg == 5 || cfg == 6 ? (const void*)k_pass2_fused<false, Stage3, MS, kC>
                                                : (const void*)k_pass2_fused<false, Stage0, MS, kC>;
    } else {
        switch (cfg) {
            case 1: return (const void*)k_pass2_fused<false, Stage1, MS, kC>;
            case 2: return (const void*)k_pass2_fused<false, Stage2, MS, kC>;
            case 3:
            case 5:
            case 6: return (const void*)k_pass2_fused<false, Stage3, MS, kC>;   // pass 2 windows without TMA
            case 4: return (const void*)k_pass2_fused<false, Stage4, MS, kC>;
            default: return (const void*)k_pass2_fused<false, Stage0, MS, kC>;
        }
    }
}

}  // namespace
}  // namespace mb
