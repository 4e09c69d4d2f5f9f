// Render kernels.
//
// cull_kernel (K3): group-major frustum and whole-meshlet back-face culling;
//   a warp item is (scene, meshlet group, block of views): the group box is
//   tested in all views of the block at once, then each meshlet in the views
//   that see the group; visible (view, meshlet) pairs go to per-phase lists
//   (distance bands) as self-contained entries (bin.cuh). The kernel also
//   clears the active views' z-buffers. cull_kernel_vg is the (view, group)
//   form for calls with many scene slots.
// hiz_kernel, hiz_pyramid_kernel, occl_kernel: before every phase after the
//   first, the farthest stored key of every 8x8 tile and its pyramid, and the
//   conservative occlusion test that keeps the pairs not proven hidden.
// raster_kernel: one launch per occlusion phase, a persistent grid whose
//   warps claim chunks of pairs from a shared cursor and stage each meshlet's
//   geometry by bulk copies one meshlet ahead; per pair:
//   K1 — transform + snap the meshlet's vertices into a per-warp
//        shared-memory cache (transform.cuh)
//   K2 — per-lane triangle reject / near clip / cull / depth plane (setup.cuh)
//   K4 — small triangles' covered samples spread over the warp, larger ones
//        rasterised by the warp row by row or binned for big_raster_kernel,
//        into the view's 64-bit z-buffer (raster.cuh)
// shade_kernel (K5): one CTA row per view; each thread resolves kShadePx
//   consecutive pixels of a row (shade.cuh) and writes RGB / depth / id with
//   vector stores when the row layout allows it.
// Work items are ordered scene-major, so a scene's geometry stays hot in L2
// while its views are in flight.
#include <algorithm>

#include <cuda_runtime.h>

#include "hsr_internal.h"
#include "kernels/bin.cuh"
#include "kernels/bulk.cuh"
#include "kernels/raster.cuh"
#include "kernels/setup.cuh"
#include "kernels/shade.cuh"
#include "kernels/transform.cuh"

namespace hsr {

constexpr int kRasterWarps = 8;
constexpr int kRasterThreads = kRasterWarps * 32;
constexpr int kBigCap = 2 * kMeshletTris;        // two per lane (guard-band ones in rounds)
// Shading is bound by the latency of its dependent loads (key -> triangle ->
// vertices -> texels): small CTAs, two pixels per thread and a 64-register
// bound (8 CTAs, 32 warps per SM) keep the most of them in flight; measured
// faster than four pixels per thread or one, at 16 to 40 warps per SM.
constexpr int kShadeThreads = 128;
constexpr int kShadePx = 2;                      // consecutive pixels of a row per shading thread
static_assert(kShadePx == 1 || kShadePx == 2 || kShadePx == 4, "shading vector width");
static_assert(sizeof(BigTri) == sizeof(BigTriStorage), "binned triangle storage size");
constexpr uint32_t kNoRecord = 0xFFFFFFFFu;

// Error flags raised by kernels of this device (kErrWaitTimeout, ...).
__device__ uint32_t g_device_err;

// --------------------------------------------------------------------- cull
// Decode a (view, group) work item: views are sorted by scene, slot k holds
// the items of one scene's views.
struct ItemDecoder {
    int s = -1;
    uint32_t lo = 0, hi = 0, G = 1, vbase = 0, scene = 0;
    __device__ __forceinline__ void locate(const Params &p, uint32_t item)
    {
        if (s >= 0 && item >= lo && item < hi) return;
        int k = 0;
        while (p.slot_item_base[k + 1] <= item) k++;
        s = k;
        lo = p.slot_item_base[k];
        hi = p.slot_item_base[k + 1];
        vbase = p.slot_view_base[k];
        scene = p.slot_scene[k];
        G = p.scenes[scene].n_groups;
    }
};

// Slot of entry k of a phase list (see Params::vis). The three lists share
// 2 * vis_cap slots and hold at most vis_cap entries together.
__device__ __forceinline__ size_t vis_index(const Params &p, uint32_t phase, uint32_t k)
{
    return phase == 0 ? (size_t)k : (phase == 2 ? (size_t)p.vis_cap - 1 - k : (size_t)p.vis_cap + k);
}

// A planar meshlet that faces away from the camera by a margin: every one of
// its triangles then snaps to a non-negative area and is culled by the exact
// per-triangle test, so skipping the meshlet changes nothing. Bound: the
// unsnapped doubled screen area of a triangle of world area a whose plane the
// camera is behind by h is 2 fx fy a h / (d0 d1 d2) (sub-pixels: x 256^2);
// snapping and float rounding move each vertex by at most eta sub-pixels per
// coordinate, which changes the doubled area by at most
// 2 sqrt2 eta (|e1| + |e2|) + 8 eta^2 for edges e1, e2. With the meshlet's
// smallest area, longest edge, the depth range and lateral extent of its box
// and the eye-transform error of its coordinates, the meshlet is skipped only
// when the smallest unsnapped area exceeds twice the largest change.
__device__ __forceinline__ int meshlet_backfacing(const Params &p, const SceneDev &S, const float *M,
                                                   const float *cpos, const float *bmin, const float *bmax,
                                                   uint32_t m)
{
    const float4 pl = S.mplane[2 * (size_t)m], bd = S.mplane[2 * (size_t)m + 1];
    const float area = bd.x, lmax = bd.y, eps_p = bd.z, rho = bd.w;
    if (!(lmax > 0.f) || !(area > 0.f)) return 0;
    const float h = pl.x * cpos[0] + pl.y * cpos[1] + pl.z * cpos[2] - pl.w;
    if (!(h < 0.f)) return 0;
    float ctr[3], ext[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        ctr[k] = 0.5f * (bmin[k] + bmax[k]);
        ext[k] = 0.5f * (bmax[k] - bmin[k]);
    }
    float xc, yc, dc;
    eye_transform(M, ctr[0], ctr[1], ctr[2], xc, yc, dc);
    const float rx = fabsf(M[0]) * ext[0] + fabsf(M[1]) * ext[1] + fabsf(M[2]) * ext[2];
    const float ry = fabsf(M[4]) * ext[0] + fabsf(M[5]) * ext[1] + fabsf(M[6]) * ext[2];
    const float rd = fabsf(M[8]) * ext[0] + fabsf(M[9]) * ext[1] + fabsf(M[10]) * ext[2];
    const float dlo = (dc - rd) * (1.f - 1e-5f), dhi = (dc + rd) * (1.f + 1e-5f) + 1e-6f;
    if (!(dlo > 1.5f * p.znear + 1e-3f)) return 1;            // near-clip path: keep
    const float cmax = fmaxf(fmaxf(fabsf(cpos[0]), fabsf(cpos[1])), fabsf(cpos[2]));
    float D = 0.f;
#pragma unroll
    for (int k = 0; k < 3; k++) D += fabsf(cpos[k] - ctr[k]) + ext[k];
    // distance behind every triangle's own plane, after the planarity slack
    const float hneed = -h - (eps_p + rho * D + 2e-6f * (3.f * cmax + fabsf(pl.w) + 1.f));
    if (!(hneed > 0.f)) return 1;
    const float g = fmaxf(fabsf(xc) + rx, fabsf(yc) + ry) / dlo;
    const float f = fmaxf(p.fx, p.fy), c = fmaxf(fabsf(p.cx), fabsf(p.cy));
    // a box that may project beyond 2^20 pixels may hold triangles clipped
    // to the guard band (from 2^22 pixels), whose sub-triangles the bound
    // below does not cover: keep it
    if (!(f * g + c < 1048576.f)) return 1;
    const float eps_e = 6.f * 5.9604645e-8f * (3.f * S.coord_max + 1.7320508f * cmax);
    const float eta = 0.5f + 256.f * (f * (1.f + g) * eps_e / dlo + 4.f * 5.9604645e-8f * (f * g + c));
    const float emax = 256.f * f * (1.f + g) * lmax * 2.f / dlo;
    const float change = 2.8284272f * eta * 2.f * emax + 8.f * eta * eta;
    const float sub_area = 65536.f * p.fx * p.fy * 2.f * area * hneed / (dhi * dhi * dhi);
    return sub_area > 2.f * change ? 2 : 1;
}

// The warps' remaining staged pairs of each phase, appended with one global
// reservation per phase for the whole CTA (each warp's share is taken in
// shared memory), instead of one per warp and phase: at the end of the
// culling every warp flushes at about the same time, and the reservations
// of all of them fall on the same three counters. Every thread of the CTA
// calls it.
__device__ __forceinline__ void flush_rest_cta(const Params &p, uint4 (*s_buf)[3][2 * 32], const uint32_t (&nbuf)[3],
                                               int lane, int warp)
{
    __shared__ uint32_t s_cnt[3], s_base[3];
    if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    uint32_t off[3];
#pragma unroll
    for (int ph = 0; ph < 3; ph++) {
        uint32_t o = 0u;
        if (lane == 0 && nbuf[ph]) o = atomicAdd(&s_cnt[ph], nbuf[ph]);
        off[ph] = __shfl_sync(0xFFFFFFFFu, o, 0);
    }
    __syncthreads();
    if (threadIdx.x < 3 && s_cnt[threadIdx.x])
        s_base[threadIdx.x] = atomicAdd(p.vis_count + threadIdx.x, s_cnt[threadIdx.x]);
    __syncthreads();
#pragma unroll
    for (int ph = 0; ph < 3; ph++)
        if ((uint32_t)lane < nbuf[ph]) p.vis[vis_index(p, ph, s_base[ph] + off[ph] + lane)] = s_buf[warp][ph][lane];
}

__global__ void __launch_bounds__(256) cull_kernel_vg(const Params p)
{
    allow_dependent_launch();
    // the active views' z-buffers set to empty (~0), 16 bytes per store (the
    // z-buffer starts on a 256-byte boundary); done here, before the raster,
    // so the clear overlaps the culling's record loads and the keys are still
    // in L2 for the raster's atomics
    {
        const size_t n = (size_t)p.dyn[0] * p.width * p.height;
        ulonglong2 *z2 = reinterpret_cast<ulonglong2 *>(p.zbuf);
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n / 2; i += (size_t)gridDim.x * blockDim.x)
            z2[i] = make_ulonglong2(~0ull, ~0ull);
        if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) p.zbuf[n - 1] = ~0ull;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t warp_id = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    // per-warp staging of the phase lists: one atomic claim per 32 entries
    __shared__ uint4 s_buf[8][3][2 * 32];
    uint32_t nbuf[3] = {0u, 0u, 0u};
    auto flush = [&](uint32_t ph, uint32_t cnt) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(p.vis_count + ph, cnt);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if ((uint32_t)lane < cnt) p.vis[vis_index(p, ph, base + lane)] = s_buf[warp][ph][lane];
    };
    ItemDecoder dec;
    const uint32_t total_items = p.dyn[1];
    for (uint32_t item = warp_id; item < total_items; item += n_warps) {
        dec.locate(p, item);
        const uint32_t local = item - dec.lo;
        const uint32_t vi = dec.vbase + local / dec.G, g = local % dec.G;
        const SceneDev &S = p.scenes[dec.scene];
        const float *pl = p.views[vi].planes;
        const Group grp = S.groups[g];
        if (!aabb_visible(pl, grp.bmin, grp.bmax)) continue;
        const uint32_t m = grp.m0 + lane;
        const bool valid = m < grp.m1;
        Meshlet ml{};
        if (valid) ml = S.meshlets[m];
        // the next meshlet's first vertex / triangle close this one's ranges:
        // from the neighbouring lane (whole warp, converged), or loaded by the
        // group's last lane
        uint32_t nvb = __shfl_down_sync(0xFFFFFFFFu, ml.vbase, 1);
        uint32_t ntb = __shfl_down_sync(0xFFFFFFFFu, ml.tbase, 1);
        if (valid && (m + 1 == grp.m1 || lane == 31)) {
            const Meshlet nx = S.meshlets[m + 1];
            nvb = nx.vbase;
            ntb = nx.tbase;
        }
        bool vis = false;
        uint32_t phase = 0;
        uint4 entry = make_uint4(0u, 0u, 0u, 0u);
        if (valid) {
            vis = aabb_visible(pl, ml.bmin, ml.bmax);
            if (vis) {
                const int bf = meshlet_backfacing(p, S, p.views[vi].M, p.views[vi].pos, ml.bmin, ml.bmax, m);
                if (p.stats) {
                    atomicAdd(p.stats + 6, 1u);
                    if (bf) atomicAdd(p.stats + (bf == 2 ? 8 : 7), 1u);
                }
                if (bf == 2) vis = false;
            }
            entry = pair_entry(vi, m, ml.vbase, nvb - ml.vbase, ml.tbase, ntb - ml.tbase);
            // distance band of the box from the camera -> occlusion phase
            const float *cp = p.views[vi].pos;
            float d2 = 0.f;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float dk = fmaxf(fmaxf(ml.bmin[k] - cp[k], cp[k] - ml.bmax[k]), 0.f);
                d2 = __fmaf_rn(dk, dk, d2);
            }
            phase = (p.n_phases > 1 && d2 > p.phase_r2[0]) + (p.n_phases > 2 && d2 > p.phase_r2[1]);
        }
        // stage this item's pairs per phase; flush 32 at a time
#pragma unroll
        for (uint32_t ph = 0; ph < 3; ph++) {
            const bool mine = vis && phase == ph;
            const unsigned mask = __ballot_sync(0xFFFFFFFFu, mine);
            if (!mask) continue;
            if (mine) s_buf[warp][ph][nbuf[ph] + __popc(mask & ((1u << lane) - 1u))] = entry;
            nbuf[ph] += (uint32_t)__popc(mask);
            __syncwarp();
            if (nbuf[ph] >= 32) {
                flush(ph, 32);
                __syncwarp();
                const uint32_t rest = nbuf[ph] - 32;
                uint4 moved = make_uint4(0u, 0u, 0u, 0u);
                if ((uint32_t)lane < rest) moved = s_buf[warp][ph][32 + lane];
                __syncwarp();
                if ((uint32_t)lane < rest) s_buf[warp][ph][lane] = moved;
                nbuf[ph] = rest;
                __syncwarp();
            }
        }
    }
    flush_rest_cta(p, s_buf, nbuf, lane, warp);
}

// Most views of one group tested per warp item (the group's and its
// meshlets' records are read once for all of them); fewer when the call is
// small, so that every warp still gets items.
constexpr uint32_t kCullViews = 16;
constexpr uint32_t kCullSlots = 32;
static_assert(kCullViews <= 32, "one lane per view of a culling item");

// Frustum (and back-face) culling of every (view, meshlet) pair, group-major:
// a warp item is (scene slot, group, block of up to kCullViews of the slot's
// views); the group box is tested in all views of the block at once (a view
// per lane), then lane l holds meshlet m0 + l of the group, loaded once, and
// tests it in each view that sees the group. Visible
// pairs are staged per warp and appended 32 at a time. Used when the call has
// at most kCullSlots scene slots (cull_kernel_vg otherwise).
__global__ void __launch_bounds__(256) cull_kernel(const Params p)
{
    allow_dependent_launch();
    {
        const size_t n = (size_t)p.dyn[0] * p.width * p.height;
        ulonglong2 *z2 = reinterpret_cast<ulonglong2 *>(p.zbuf);
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n / 2; i += (size_t)gridDim.x * blockDim.x)
            z2[i] = make_ulonglong2(~0ull, ~0ull);
        if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) p.zbuf[n - 1] = ~0ull;
    }
    __shared__ uint32_t s_ibase[kCullSlots + 1], s_v0[kCullSlots], s_nv[kCullSlots], s_nch[kCullSlots];
    __shared__ uint32_t s_scene[kCullSlots];
    __shared__ uint4 s_buf[8][3][2 * 32];
    const uint32_t n_slots = p.dyn[2];
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (uint32_t k = 0; k < n_slots; k++) {
            const uint32_t v0 = p.slot_view_base[k];
            const uint32_t v1 = k + 1 < n_slots ? p.slot_view_base[k + 1] : p.dyn[0];
            const uint32_t sc = p.slot_scene[k];
            const uint32_t nch = (v1 - v0 + p.cull_views - 1) / p.cull_views;
            s_ibase[k] = acc;
            s_v0[k] = v0;
            s_nv[k] = v1 - v0;
            s_nch[k] = nch;
            s_scene[k] = sc;
            acc += p.scenes[sc].n_groups * nch;
        }
        s_ibase[n_slots] = acc;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t warp_id = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    uint32_t nbuf[3] = {0u, 0u, 0u};
    auto flush = [&](uint32_t ph, uint32_t cnt) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(p.vis_count + ph, cnt);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if ((uint32_t)lane < cnt) p.vis[vis_index(p, ph, base + lane)] = s_buf[warp][ph][lane];
    };
    const uint32_t total_items = s_ibase[n_slots];
    for (uint32_t item = warp_id; item < total_items; item += n_warps) {
        uint32_t k = 0;
        while (s_ibase[k + 1] <= item) k++;
        const uint32_t local = item - s_ibase[k];
        const uint32_t g = local / s_nch[k], ch = local % s_nch[k];
        const uint32_t va = s_v0[k] + ch * p.cull_views;
        const uint32_t vb = min(va + p.cull_views, s_v0[k] + s_nv[k]);
        const SceneDev &S = p.scenes[s_scene[k]];
        // group g is the run of kGroupMeshlets consecutive meshlets from
        // g * kGroupMeshlets, so the meshlet loads need not wait for its
        // record; the back-face test's plane records are requested into L1
        // at the same time (no register held until the test reads them)
        const uint32_t m = g * kGroupMeshlets + lane;
        const bool valid = m < S.n_meshlets;
        Meshlet ml{};
        if (valid) {
            ml = S.meshlets[m];
            asm volatile("prefetch.global.L1 [%0];" ::"l"(S.mplane + 2 * (size_t)m));
        }
        const Group grp = S.groups[g];
        uint32_t nvb = __shfl_down_sync(0xFFFFFFFFu, ml.vbase, 1);
        uint32_t ntb = __shfl_down_sync(0xFFFFFFFFu, ml.tbase, 1);
        if (valid && (m + 1 == grp.m1 || lane == 31)) {
            const Meshlet nx = S.meshlets[m + 1];
            nvb = nx.vbase;
            ntb = nx.tbase;
        }
        // the group box against every view of the block at once, one view
        // per lane; then only the views that see the group
        uint32_t vmask;
        {
            const uint32_t v = va + (uint32_t)lane;
            vmask = __ballot_sync(0xFFFFFFFFu, v < vb && aabb_visible(p.views[v].planes, grp.bmin, grp.bmax));
        }
        while (vmask) {
            const uint32_t vi = va + (uint32_t)(__ffs(vmask) - 1);
            vmask &= vmask - 1u;
            const float *pl = p.views[vi].planes;
            bool vis = false;
            uint32_t phase = 0;
            uint4 entry = make_uint4(0u, 0u, 0u, 0u);
            if (valid) {
                vis = aabb_visible(pl, ml.bmin, ml.bmax);
                if (vis) {
                    const int bf = meshlet_backfacing(p, S, p.views[vi].M, p.views[vi].pos, ml.bmin, ml.bmax, m);
                    if (p.stats) {
                        atomicAdd(p.stats + 6, 1u);
                        if (bf) atomicAdd(p.stats + (bf == 2 ? 8 : 7), 1u);
                    }
                    if (bf == 2) vis = false;
                }
                entry = pair_entry(vi, m, ml.vbase, nvb - ml.vbase, ml.tbase, ntb - ml.tbase);
                const float *cp = p.views[vi].pos;
                float d2 = 0.f;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const float dk = fmaxf(fmaxf(ml.bmin[c] - cp[c], cp[c] - ml.bmax[c]), 0.f);
                    d2 = __fmaf_rn(dk, dk, d2);
                }
                phase = (p.n_phases > 1 && d2 > p.phase_r2[0]) + (p.n_phases > 2 && d2 > p.phase_r2[1]);
            }
#pragma unroll
            for (uint32_t ph = 0; ph < 3; ph++) {
                const bool mine = vis && phase == ph;
                const unsigned mask = __ballot_sync(0xFFFFFFFFu, mine);
                if (!mask) continue;
                if (mine) s_buf[warp][ph][nbuf[ph] + __popc(mask & ((1u << lane) - 1u))] = entry;
                nbuf[ph] += (uint32_t)__popc(mask);
                __syncwarp();
                if (nbuf[ph] >= 32) {
                    flush(ph, 32);
                    __syncwarp();
                    const uint32_t rest = nbuf[ph] - 32;
                    uint4 moved = make_uint4(0u, 0u, 0u, 0u);
                    if ((uint32_t)lane < rest) moved = s_buf[warp][ph][32 + lane];
                    __syncwarp();
                    if ((uint32_t)lane < rest) s_buf[warp][ph][lane] = moved;
                    nbuf[ph] = rest;
                    __syncwarp();
                }
            }
        }
    }
    flush_rest_cta(p, s_buf, nbuf, lane, warp);
}

// --------------------------------------------------------------------- raster
// Per-warp staging buffer of one meshlet: its vertex block and its triangle
// block, the latter widened to start on a 16-byte boundary (the first
// triangle sits at tri[first_tri & 1]). Filled by the bulk-copy engine while
// the warp works on the previous meshlet.
struct alignas(16) MeshletStage {
    float4 vert[kMeshletVerts];
    uint2 tri[kMeshletTris + 2];
};

// Emit one front-facing (sub-)triangle: clip its pixel range to the image,
// raster it here when small, else queue it for the warp.
// With `small` non-null a small triangle is only set up there (the warp
// rasterises the fragments of all lanes together); else this lane rasterises it.
__device__ __forceinline__ void emit_tri(const Tri2D &t, uint32_t id, const Params &p, unsigned long long *zbuf,
                                         BigTri *bigq, uint32_t *bign, uint32_t view, uint32_t phase,
                                         SmallFrag *small = nullptr)
{
    int x0, x1, y0, y1, spanx, spany;
    pixel_range(t, x0, x1, y0, y1, spanx, spany);
    x0 = max(x0, 0);
    y0 = max(y0, 0);
    x1 = min(x1, (int)p.width - 1);
    y1 = min(y1, (int)p.height - 1);
    if (x0 > x1 || y0 > y1) return;            // no sample on screen
    const int npx = (x1 - x0 + 1) * (y1 - y0 + 1);
    if (spanx < 32768 && spany < 32768 && npx <= (int)p.small_px) {
        if (small)
            small_setup(t, id, x0, x1, y0, y1, *small);
        else
            raster_small(t, id, x0, x1, y0, y1, p.q_far, zbuf, (int)p.width);
        return;
    }
    float pa, pb;
    depth_plane(t, pa, pb);
    BigTri r;
    r.X0 = t.X0; r.Y0 = t.Y0; r.X1 = t.X1; r.Y1 = t.Y1; r.X2 = t.X2; r.Y2 = t.Y2;
    r.pa = pa; r.pb = pb; r.q0 = t.q0; r.qlo = tri_qlo(t); r.qhi = tri_qhi(t); r.id = id;
    r.x0 = (unsigned short)x0; r.x1 = (unsigned short)x1;
    r.y0 = (unsigned short)y0; r.y1 = (unsigned short)y1;
    r.view = view;
    r.pad_ = 0;
    if (p.big_rec && npx > (int)p.bin_px) {
        // bin for the large-triangle pass: instances cover runs of
        // big_rows_per_item rows of the triangle's candidate rectangle
        const uint32_t rpi = (uint32_t)big_rows_per_item(x0, x1);
        const uint32_t ninst = ((uint32_t)(y1 - y0) + rpi) / rpi;
        const uint32_t ri = atomicAdd(p.big_rec_count, 1u);
        if (ri < p.big_rec_cap) {
            const uint32_t k0 = atomicAdd(p.big_inst_count + phase, ninst);
            uint2 *inst = p.big_inst + (size_t)phase * p.big_inst_cap;
            if (k0 + ninst <= p.big_inst_cap && k0 + ninst >= k0) {
                p.big_rec[ri] = r;
                for (uint32_t k = 0; k < ninst; k++) inst[k0 + k] = make_uint2(ri, (k * rpi) | (rpi << 16));
                return;
            }
            // reservation straddles the end: mark the in-range slots as empty
            for (uint32_t k = k0; k < p.big_inst_cap && k - k0 < ninst; k++) inst[k] = make_uint2(kNoRecord, 0u);
        }
    }
    const uint32_t slot = atomicAdd(bign, 1u);     // bins full: the warp rasterises it
    bigq[slot] = r;
}

// Raster of the binned large triangles of one phase: one warp per instance
// (a triangle and a run of up to big_rows_per_item rows of its candidate
// rectangle: first row offset in the low 16 bits, run length in the high
// bits; images are at most 4096 rows), grid-stride.
__global__ void __launch_bounds__(256) big_raster_kernel(const Params p, uint32_t phase)
{
    allow_dependent_launch();
    grid_dependency_wait();
    const int lane = threadIdx.x & 31;
    const uint32_t count = min(p.big_inst_count[phase], p.big_inst_cap);
    const uint32_t warp_id = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    const uint2 *inst = p.big_inst + (size_t)phase * p.big_inst_cap;
    for (uint32_t i = warp_id; i < count; i += n_warps) {
        const uint2 in = inst[i];
        if (in.x == kNoRecord) continue;
        const BigTri t = p.big_rec[in.x];
        unsigned long long *zb = p.zbuf + (size_t)t.view * p.width * p.height;
        const int r0 = (int)t.y0 + (int)(in.y & 0xFFFFu);
        const int r1 = min((int)t.y1, r0 + (int)(in.y >> 16) - 1);
        raster_rows_warp(t, r0, r1, lane, p.q_far, zb, (int)p.width);
    }
}

// One staged meshlet (whole warp): K1 transform + snap its vertices into the
// warp's vertex cache, K2 per-lane triangle setup, K4 raster.
__device__ __forceinline__ void process_meshlet(const MeshletStage &st, const Params &p, uint32_t nv, uint32_t nt,
                                                uint32_t toff, unsigned long long *zbuf, EyeHot *vh, BigTri *bigq,
                                                uint32_t *bign, int lane, uint32_t view, uint32_t phase)
{
    const float zn = p.znear, zf = p.zfar;
    // the view matrix from the view record (the same 48 bytes for every
    // lane: one broadcast load each, served by L1 after the first pair)
    float M[12];
#pragma unroll
    for (int i = 0; i < 12; i++) M[i] = __ldg(p.views[view].M + i);

    // K1: transform + snap this meshlet's vertices (q = 0: near-clipped or
    // beyond the fixed-point range, handled by the clipping path)
    for (uint32_t v = lane; v < nv; v += 32) {
        const float4 P = st.vert[v];
        EyeHot h;
        float xe, ye;
        eye_transform(M, P.x, P.y, P.z, xe, ye, h.d);
        if (h.d >= zn) {
            if (!project_snap(xe, ye, h.d, p.fx, p.fy, p.cx, p.cy, h.q, h.X, h.Y)) h.q = 0.f;
        } else {
            h.q = 0.f;
            h.X = h.Y = 0;
        }
        vh[v] = h;
    }
    __syncwarp();

    // K2 + K4: one triangle per lane. A lane queues at most two large
    // (sub-)triangles here, so the warp's queue (kBigCap) holds them all; a
    // guard-band clip can yield up to six, so those are kept and emitted one
    // per lane per round below, the queue drained after each round.
    SmallFrag sf;
    sf.mask = 0u;
    uint32_t id = 0;
    Tri2D gq[kMaxClipVerts - 2];
    int gn = 0;
    if ((uint32_t)lane < nt) {
        const uint2 mt = st.tri[toff + lane];
        const uint32_t ia = mt.x & 255u, ib = (mt.x >> 8) & 255u, ic = (mt.x >> 16) & 255u;
        const EyeHot a = vh[ia], b = vh[ib], cc = vh[ic];
        id = mt.y;
        const bool all_near = a.d < zn && b.d < zn && cc.d < zn;
        const bool all_far = a.d > zf && b.d > zf && cc.d > zf;
        if (!all_near && !all_far) {
            Tri2D t;
            if (a.q > 0.f && b.q > 0.f && cc.q > 0.f) {
                if (orient_cull(a.X, a.Y, a.q, b.X, b.Y, b.q, cc.X, cc.Y, cc.q, t))
                    emit_tri(t, id, p, zbuf, bigq, bign, view, phase, &sf);
            } else {
                // clipping path: eye-space positions again from the staged
                // vertices, near clip, then the guard band if a snap is out of range
                const uint32_t li[3] = {ia, ib, ic};
                CVert<0> v[3];
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const float4 P = st.vert[li[k]];
                    eye_transform(M, P.x, P.y, P.z, v[k].xe, v[k].ye, v[k].d);
                    v[k].gid = __float_as_uint(P.w);
                }
                CVert<0> poly[4];
                const int np = clip_near<0>(v, zn, poly);
                int X[4], Y[4];
                float q[4];
                bool in_range = true;
                for (int k = 0; k < np; k++)
                    in_range &= project_snap(poly[k].xe, poly[k].ye, poly[k].d, p.fx, p.fy, p.cx, p.cy, q[k], X[k],
                                             Y[k]);
                if (in_range) {
                    for (int f = 0; f + 2 < np; f++) {
                        int ix[3];
                        if (clipped_fan_tri(X, Y, q, f, ix, t)) emit_tri(t, id, p, zbuf, bigq, bign, view, phase);
                    }
                } else {
                    // guard band (out of line); a vertex still out of range
                    // after it (not reachable within the documented input
                    // limits) drops the triangle and raises kErrRange
                    ClipPoly<0> cp;
                    for (int k = 0; k < 4; k++) cp.v[k] = poly[k];
                    cp.n = np;
                    const int ng = guard_fan<0>(cp, GuardCam{p.gx, p.gy, p.fx, p.fy, p.cx, p.cy}, gq, nullptr);
                    if (ng < 0) atomicOr(&g_device_err, kErrRange);
                    // this view's shading needs the guard-band path
                    if (ng > 0) atomicOr(const_cast<uint32_t *>(&p.views[view].outputs), kViewGuard);
                    gn = max(ng, 0);
                }
            }
        }
    }
    __syncwarp();
    // small triangles with few covered samples merge them in their own lane;
    // the warp spreads the fragments of the others
    if (sf.mask && __popc(sf.mask) <= kDirectFrags) {
        raster_fragments_lane(sf, p.q_far, zbuf, (int)p.width);
        sf.mask = 0u;
    }
    raster_fragments_warp(sf, lane, p.q_far, zbuf, (int)p.width);
    const uint32_t nb = *bign;
    for (uint32_t r = 0; r < nb; r++) raster_big_warp(bigq[r], lane, p.q_far, zbuf, (int)p.width);
    __syncwarp();
    if (lane == 0) *bign = 0;
    __syncwarp();
    // guard-band sub-triangles, one per lane per round
    if (__any_sync(0xFFFFFFFFu, gn > 0)) {
        for (int gk = 0; __any_sync(0xFFFFFFFFu, gk < gn); gk++) {
            if (gk < gn) emit_tri(gq[gk], id, p, zbuf, bigq, bign, view, phase);
            __syncwarp();
            const uint32_t ng = *bign;
            for (uint32_t r = 0; r < ng; r++) raster_big_warp(bigq[r], lane, p.q_far, zbuf, (int)p.width);
            __syncwarp();
            if (lane == 0) *bign = 0;
            __syncwarp();
        }
    }
}

// Conservative occlusion test of a meshlet box against the tile-z pyramid of
// the phases already rasterised (one thread). Every fragment of the meshlet
// has inverse depth at most 1/d_min of its (inflated) box, because
// interpolated q is clamped to the vertices' range; if every pyramid texel
// over the box's projected rectangle (grown by a pixel) already holds only
// keys strictly nearer than that bound, none of its fragments can win any
// pixel, and skipping it changes nothing. The level is the first at which the
// rectangle spans at most 2 x 2 texels.
__device__ __forceinline__ bool box_occluded(const float *bmin, const float *bmax, const float *M, const Params &p,
                                             const uint32_t *pyr)
{
    float xe[8], ye[8], de[8];
    float dmin = 3.0e38f;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        eye_transform(M, (c & 1) ? bmax[0] : bmin[0], (c & 2) ? bmax[1] : bmin[1], (c & 4) ? bmax[2] : bmin[2],
                      xe[c], ye[c], de[c]);
        dmin = fminf(dmin, de[c]);
    }
    if (!(dmin > p.znear + 1e-3f)) return false;        // box reaches the near plane: keep
    float sx0 = 3.0e38f, sx1 = -3.0e38f, sy0 = 3.0e38f, sy1 = -3.0e38f;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const float r = __frcp_rn(de[c]);
        const float sx = __fmaf_rn(p.fx, __fmul_rn(xe[c], r), p.cx);
        const float sy = __fmaf_rn(-p.fy, __fmul_rn(ye[c], r), p.cy);
        sx0 = fminf(sx0, sx);
        sx1 = fmaxf(sx1, sx);
        sy0 = fminf(sy0, sy);
        sy1 = fmaxf(sy1, sy);
    }
    const float Wf = (float)p.width, Hf = (float)p.height;
    if (sx1 + 1.f < 0.f || sy1 + 1.f < 0.f || sx0 - 1.f > Wf || sy0 - 1.f > Hf) return false;   // culled elsewhere
    const uint32_t x0 = (uint32_t)fminf(fmaxf(floorf(sx0 - 1.f), 0.f), Wf - 1.f);
    const uint32_t x1 = (uint32_t)fminf(fmaxf(ceilf(sx1 + 1.f), 0.f), Wf - 1.f);
    const uint32_t y0 = (uint32_t)fminf(fmaxf(floorf(sy0 - 1.f), 0.f), Hf - 1.f);
    const uint32_t y1 = (uint32_t)fminf(fmaxf(ceilf(sy1 + 1.f), 0.f), Hf - 1.f);
    uint32_t tx0 = x0 / kHizTile, tx1 = x1 / kHizTile, ty0 = y0 / kHizTile, ty1 = y1 / kHizTile;
    uint32_t w = p.hiz_w, h = p.hiz_h, off = 0;
    while (tx1 - tx0 > 1 || ty1 - ty0 > 1) {
        off += w * h;
        w = (w + 1) / 2;
        h = (h + 1) / 2;
        tx0 >>= 1; tx1 >>= 1; ty0 >>= 1; ty1 >>= 1;
    }
    const uint32_t hb = ~__float_as_uint(__frcp_rn(dmin * (1.0f - 1e-5f)));
    for (uint32_t ty = ty0; ty <= ty1; ty++)
        for (uint32_t tx = tx0; tx <= tx1; tx++)
            if (pyr[off + ty * w + tx] >= hb) return false;
    return true;
}

// Tile z, level 0 of the pyramid: per 8x8 tile of each view the largest
// stored key >> 32 (the farthest fragment, or background = 0xFFFFFFFF). Four
// lanes per tile, each a 16-byte column of its eight rows, so a warp's loads
// cover 512 contiguous bytes of a row; the four are combined with shuffles.
__global__ void __launch_bounds__(256) hiz_kernel(const Params p)
{
    allow_dependent_launch();
    grid_dependency_wait();
    const uint32_t per_view = p.hiz_w * p.hiz_h;
    const uint32_t total = p.dyn[0] * per_view * 4u;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ((total + 31) & ~31u);
         g += gridDim.x * blockDim.x) {
        uint32_t mx = 0;
        const uint32_t t = g >> 2, part = g & 3u;
        if (g < total) {
            const uint32_t v = t / per_view, r = t % per_view;
            const uint32_t ty = r / p.hiz_w, tx = r % p.hiz_w;
            const uint32_t x = tx * kHizTile + 2 * part;
            const uint32_t y0 = ty * kHizTile, y1 = min(y0 + kHizTile, p.height);
            const unsigned long long *zv = p.zbuf + (size_t)v * p.width * p.height;
            if (x + 1 < p.width && (p.width & 1u) == 0) {
                for (uint32_t y = y0; y < y1; y++) {
                    const ulonglong2 k = *reinterpret_cast<const ulonglong2 *>(zv + (size_t)y * p.width + x);
                    mx = max(mx, max((uint32_t)(k.x >> 32), (uint32_t)(k.y >> 32)));
                }
            } else {
                for (uint32_t y = y0; y < y1; y++)
                    for (uint32_t xx = x; xx < min(x + 2, p.width); xx++)
                        mx = max(mx, (uint32_t)(zv[(size_t)y * p.width + xx] >> 32));
            }
        }
        mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, 1));
        mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, 2));
        if (g < total && part == 0) p.hiz[(size_t)(t / per_view) * p.hiz_total + t % per_view] = mx;
    }
}

// Coarser pyramid levels of each active view (one block per view).
__global__ void __launch_bounds__(256) hiz_pyramid_kernel(const Params p)
{
    allow_dependent_launch();
    grid_dependency_wait();
    const uint32_t v = blockIdx.x;
    if (v >= p.dyn[0]) return;
    uint32_t *pyr = p.hiz + (size_t)v * p.hiz_total;
    uint32_t w = p.hiz_w, h = p.hiz_h, off = 0;
    while (w > 1 || h > 1) {
        const uint32_t w2 = (w + 1) / 2, h2 = (h + 1) / 2, off2 = off + w * h;
        for (uint32_t i = threadIdx.x; i < w2 * h2; i += blockDim.x) {
            const uint32_t x = i % w2, y = i / w2;
            const uint32_t xa = 2 * x, xb = min(2 * x + 1, w - 1), ya = 2 * y, yb = min(2 * y + 1, h - 1);
            pyr[off2 + i] = max(max(pyr[off + ya * w + xa], pyr[off + ya * w + xb]),
                                max(pyr[off + yb * w + xa], pyr[off + yb * w + xb]));
        }
        __syncthreads();
        off = off2;
        w = w2;
        h = h2;
    }
}

// Occlusion test of the pairs of a phase after the first (one thread per
// pair); the pairs not proven hidden are compacted into the survivor list.
__global__ void __launch_bounds__(256) occl_kernel(const Params p, uint32_t phase)
{
    allow_dependent_launch();
    grid_dependency_wait();
    const uint32_t count = min(p.vis_count[phase], p.vis_cap);
    const int lane = threadIdx.x & 31;
    const uint32_t rounded = (count + 31u) & ~31u;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < rounded; k += gridDim.x * blockDim.x) {
        bool keep = false;
        uint4 pr = make_uint4(0u, 0u, 0u, 0u);
        if (k < count) {
            pr = p.vis[vis_index(p, phase, k)];
            const uint32_t vi = pair_view(pr);
            const View &V = p.views[vi];
            const Meshlet &ml = p.scenes[V.scene].meshlets[pr.y];
            float M[12];
#pragma unroll
            for (int i = 0; i < 12; i++) M[i] = V.M[i];
            keep = !box_occluded(ml.bmin, ml.bmax, M, p, p.hiz + (size_t)vi * p.hiz_total);
        }
        const unsigned mask = __ballot_sync(0xFFFFFFFFu, keep);
        const unsigned tested = __ballot_sync(0xFFFFFFFFu, k < count);
        uint32_t base = 0;
        if (lane == 0) {
            if (mask) base = atomicAdd(p.surv_count + (phase - 1), (uint32_t)__popc(mask));
            if (p.stats) {
                atomicAdd(p.stats + phase, (uint32_t)__popc(tested));
                atomicAdd(p.stats + 3 + phase, (uint32_t)__popc(tested & ~mask));
            }
        }
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (keep) p.surv[base + __popc(mask & ((1u << lane) - 1u))] = pr;
    }
}

// Scene geometry pointers of the first kSlotCache slots, cached per CTA.
constexpr uint32_t kSlotCache = 32;

// The bulk copies that stage a pair's vertex and triangle blocks (issued by
// one lane).
__device__ __forceinline__ void stage_meshlet(MeshletStage &st, uint64_t *bar, const Params &p, const uint4 &e,
                                              const float4 *mvert, const uint2 *mtri)
{
    const uint32_t nv = pair_nv(e), nt = pair_nt(e);
    const uint32_t t0 = e.w & ~1u;                              // 16-byte aligned start
    const uint32_t tn = (e.w + nt - t0 + 1u) & ~1u;             // even count covering the range
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, nv * 16u + tn * 8u + p.fault_tx);
    bulk_g2s(st.vert, mvert + e.z, nv * 16u, bar);
    bulk_g2s(st.tri, mtri + t0, tn * 8u, bar);
}

// Raster of one phase. Warps take chunks of consecutive pairs from a shared
// cursor; within a warp the next meshlet's matrix, vertices and triangles are
// staged by bulk copies (double buffer) while the current one is rasterised,
// and the next chunk is claimed and read one meshlet ahead, so no global load
// latency sits on the warp's path.
__global__ void __launch_bounds__(kRasterThreads, 3) raster_kernel(const Params p, uint32_t phase)
{
    allow_dependent_launch();
    grid_dependency_wait();
    // dynamic shared memory per warp: two meshlet stages, the vertex cache and
    // the big-triangle queue (kRasterSmem)
    extern __shared__ __align__(128) unsigned char smem[];
    MeshletStage(*s_stage)[2] = reinterpret_cast<MeshletStage(*)[2]>(smem);
    EyeHot(*s_vh)[kMeshletVerts] = reinterpret_cast<EyeHot(*)[kMeshletVerts]>(s_stage + kRasterWarps);
    BigTri(*s_big)[kBigCap] = reinterpret_cast<BigTri(*)[kBigCap]>(s_vh + kRasterWarps);
    __shared__ __align__(8) uint64_t s_bar[kRasterWarps][2];
    __shared__ uint32_t s_bign[kRasterWarps];
    __shared__ uint32_t s_slot_view[kSlotCache + 1];
    __shared__ const float4 *s_slot_mvert[kSlotCache];
    __shared__ const uint2 *s_slot_mtri[kSlotCache];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t n_slots = p.dyn[2];
    if (threadIdx.x < kSlotCache && threadIdx.x < n_slots) {
        const SceneDev &S = p.scenes[p.slot_scene[threadIdx.x]];
        s_slot_view[threadIdx.x] = p.slot_view_base[threadIdx.x];
        s_slot_mvert[threadIdx.x] = S.mvert;
        s_slot_mtri[threadIdx.x] = S.mtri;
    }
    if (threadIdx.x == 0) s_slot_view[min(n_slots, kSlotCache)] = 0xFFFFFFFFu;
    if (lane == 0) {
        s_bign[warp] = 0;
        mbar_init(&s_bar[warp][0]);
        mbar_init(&s_bar[warp][1]);
        mbar_init_fence();
    }
    __syncthreads();

    // phase 0 rasterises its list; later phases the survivors of occl_kernel
    const uint4 *list = phase == 0 ? p.vis : p.surv;
    const uint32_t count = min(phase == 0 ? p.vis_count[0] : p.surv_count[phase - 1], p.vis_cap);
    // chunk shrinks when the phase has few pairs, so that every warp gets work
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t CH = max(1u, min(p.chunk, count / (2 * n_warps)));

    // geometry of the scene a view belongs to (slot cache, else the records)
    auto geometry = [&](uint32_t vi, const float4 *&mv, const uint2 *&mt) {
        if (n_slots <= kSlotCache) {
            uint32_t k = 0;
            while (s_slot_view[k + 1] <= vi) k++;
            mv = s_slot_mvert[k];
            mt = s_slot_mtri[k];
        } else {
            const SceneDev &S = p.scenes[p.views[vi].scene];
            mv = S.mvert;
            mt = S.mtri;
        }
    };

    uint32_t c0 = 0;
    if (lane == 0) c0 = atomicAdd(p.work_counter + phase, CH);
    c0 = __shfl_sync(0xFFFFFFFFu, c0, 0);
    uint32_t ne = c0 < count ? min(CH, count - c0) : 0u;
    uint4 ent = make_uint4(0u, 0u, 0u, 0u);
    if ((uint32_t)lane < ne) ent = list[c0 + lane];
    uint32_t nclaim = 0;                     // claim of the chunk after this one (lane 0)
    if (lane == 0 && ne) nclaim = atomicAdd(p.work_counter + phase, CH);
    uint32_t ne_nx = 0;
    uint4 ent_nx = make_uint4(0u, 0u, 0u, 0u);
    bool nx_read = false;

    uint32_t par = 0;                        // bit s: parity of the next phase of stage s
    uint32_t stg = 0;
    bool failed = false;
    bool pending[2] = {false, false};
    if (ne) {
        const uint4 e = make_uint4(__shfl_sync(0xFFFFFFFFu, ent.x, 0), __shfl_sync(0xFFFFFFFFu, ent.y, 0),
                                   __shfl_sync(0xFFFFFFFFu, ent.z, 0), __shfl_sync(0xFFFFFFFFu, ent.w, 0));
        if (lane == 0) {
            const float4 *mv;
            const uint2 *mt;
            geometry(pair_view(e), mv, mt);
            stage_meshlet(s_stage[warp][0], &s_bar[warp][0], p, e, mv, mt);
        }
        pending[0] = true;
    }
    uint32_t j = 0;
    while (ne) {
        // the pair after (chunk, j): read the next chunk first when needed
        if (!nx_read && (j + 1 >= ne || j == 0)) {
            const uint32_t c1 = __shfl_sync(0xFFFFFFFFu, nclaim, 0);
            ne_nx = c1 < count ? min(CH, count - c1) : 0u;
            if ((uint32_t)lane < ne_nx) ent_nx = list[c1 + lane];
            nx_read = true;
        }
        const bool in_chunk = j + 1 < ne;
        const bool has_next = in_chunk || ne_nx > 0;
        if (has_next) {
            const uint32_t src = in_chunk ? j + 1 : 0u;
            const uint4 sel = in_chunk ? ent : ent_nx;
            const uint4 e = make_uint4(__shfl_sync(0xFFFFFFFFu, sel.x, src), __shfl_sync(0xFFFFFFFFu, sel.y, src),
                                       __shfl_sync(0xFFFFFFFFu, sel.z, src), __shfl_sync(0xFFFFFFFFu, sel.w, src));
            if (lane == 0) {
                const float4 *mv;
                const uint2 *mt;
                geometry(pair_view(e), mv, mt);
                stage_meshlet(s_stage[warp][stg ^ 1], &s_bar[warp][stg ^ 1], p, e, mv, mt);
            }
            pending[stg ^ 1] = true;
        }
        // this pair
        const uint4 e = make_uint4(__shfl_sync(0xFFFFFFFFu, ent.x, j), __shfl_sync(0xFFFFFFFFu, ent.y, j),
                                   __shfl_sync(0xFFFFFFFFu, ent.z, j), __shfl_sync(0xFFFFFFFFu, ent.w, j));
        const bool ok = mbar_wait_bounded(&s_bar[warp][stg], (par >> stg) & 1u);
        par ^= 1u << stg;
        pending[stg] = false;
        if (!__all_sync(0xFFFFFFFFu, ok)) {
            failed = true;
            break;
        }
        const uint32_t vi = pair_view(e);
        if (phase == 0 && p.stats && lane == 0) atomicAdd(p.stats, 1u);
        process_meshlet(s_stage[warp][stg], p, pair_nv(e), pair_nt(e), e.w & 1u,
                        p.zbuf + (size_t)vi * p.width * p.height, s_vh[warp], s_big[warp], &s_bign[warp], lane, vi,
                        phase);
        stg ^= 1;
        if (in_chunk) {
            j++;
        } else {
            if (!ne_nx) break;
            ne = ne_nx;
            ent = ent_nx;
            j = 0;
            nx_read = false;
            if (lane == 0) nclaim = atomicAdd(p.work_counter + phase, CH);
        }
    }
    if (failed) {
        if (lane == 0) atomicOr(&g_device_err, kErrWaitTimeout);
        // let copies still in flight land before the CTA's shared memory goes away
        for (int k = 0; k < 2; k++)
            if (pending[k]) mbar_wait_bounded(&s_bar[warp][k], (par >> k) & 1u);
    }
}

// ----------------------------------------------------------------- mip chain
__global__ void mip_down_kernel(const uint32_t *__restrict__ src, uint32_t w, uint32_t h, uint32_t *__restrict__ dst,
                                uint32_t w2, uint32_t h2)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= w2 * h2) return;
    const uint32_t x = i % w2, y = i / w2;
    const uint32_t xa = min(2 * x, w - 1), xb = min(2 * x + 1, w - 1);
    const uint32_t ya = min(2 * y, h - 1), yb = min(2 * y + 1, h - 1);
    const uint32_t t[4] = {src[(size_t)ya * w + xa], src[(size_t)ya * w + xb], src[(size_t)yb * w + xa],
                           src[(size_t)yb * w + xb]};
    uint32_t out = 0;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        uint32_t sum = 2;
#pragma unroll
        for (int k = 0; k < 4; k++) sum += (t[k] >> (8 * c)) & 255u;
        out |= (sum >> 2) << (8 * c);
    }
    dst[i] = out;
}

cudaError_t launch_mip_down(const uint32_t *src, uint32_t w, uint32_t h, uint32_t *dst, uint32_t w2, uint32_t h2,
                            cudaStream_t stream)
{
    const uint32_t n = w2 * h2;
    mip_down_kernel<<<(n + 255) / 256, 256, 0, stream>>>(src, w, h, dst, w2, h2);
    return cudaGetLastError();
}

// --------------------------------------------------------------------- shade
// N: the call adds depth noise (the host launches this variant for every
// noisy call; it applies the precise noise model).
template <int NA, bool G, bool N>
__device__ __forceinline__ void shade_rows(const Params &p, const SceneDev &S, const float *M, uint32_t vi,
                                           uint32_t frame, uint32_t agent, uint32_t outputs)
{
    constexpr int K = kShadePx;
    const uint32_t W = p.width, H = p.height;
    uint8_t *const out_rgb = (outputs & HSR_OUT_RGB) ? p.rgb : nullptr;
    float *const out_depth = (outputs & HSR_OUT_DEPTH) ? p.depth : nullptr;
    uint32_t *const out_ids = (outputs & HSR_OUT_IDS) ? p.ids : nullptr;
    const uint32_t qpr = (W + K - 1) / K, quads = qpr * H;
    unsigned long long *zb = p.zbuf + (size_t)vi * W * H;
    const size_t fbase = (size_t)frame * W * H;
    // vector stores: K pixels of a row are K consecutive outputs when W is a
    // multiple of K (and the frame base then is too)
    const bool vec = (W % K == 0) && (((uintptr_t)p.rgb & (K == 4 ? 3 : 1)) == 0) &&
                     (((uintptr_t)p.depth & (4 * K - 1)) == 0) && (((uintptr_t)p.ids & (4 * K - 1)) == 0);
    const float sigma = __uint_as_float(p.dyn[3]);
    for (uint32_t qi = blockIdx.x * blockDim.x + threadIdx.x; qi < quads; qi += gridDim.x * blockDim.x) {
        ShadeTri<NA> st;           // setup cache over this thread's run of pixels
        const uint32_t y = qi / qpr, x0 = (qi % qpr) * K;
        const uint32_t n = min((uint32_t)K, W - x0);
        const size_t pi = (size_t)y * W + x0;
        unsigned long long key[K];
        bool loaded = false;
        if constexpr (K > 1) {
            if (vec) {
#pragma unroll
                for (int k = 0; k + 1 < K; k += 2) {
                    // the keys are dead after shading: read them evict-first
                    const ulonglong2 kk = __ldcs(reinterpret_cast<const ulonglong2 *>(zb + pi + k));
                    key[k] = kk.x;
                    key[k + 1] = kk.y;
                }
                loaded = true;
            }
        }
        if (!loaded) {
#pragma unroll
            for (int k = 0; k < K; k++) key[k] = k < (int)n ? zb[pi + k] : ~0ull;
        }
        uint32_t rgb[K], id[K];
        float dep[K];
#pragma unroll
        for (int k = 0; k < K; k++)
            shade_pixel<NA, G>(st, S, M, p, (int)(x0 + k), (int)y, key[k], rgb[k], dep[k], id[k], out_rgb != nullptr);
        if (sigma > 0.f && out_depth) {
            const uint32_t k0 = p.dyn[4], k1 = p.dyn[5];
#pragma unroll
            for (int k = 0; k < K; k++)
                if (key[k] != ~0ull)
                    dep[k] = noisy_depth<N>(sigma, k0, k1, p.inv_far, __uint_as_float(~(uint32_t)(key[k] >> 32)),
                                         (uint32_t)(pi + k), agent);
        }
        const size_t o = fbase + pi;
        if (vec && K > 1) {
            if constexpr (K == 4) {
                if (out_rgb) {
                    // four packed 24-bit RGB values -> three little-endian words
                    uint32_t *r32 = reinterpret_cast<uint32_t *>(out_rgb + 3 * o);
                    r32[0] = rgb[0] | (rgb[1] << 24);
                    r32[1] = (rgb[1] >> 8) | (rgb[2] << 16);
                    r32[2] = (rgb[2] >> 16) | (rgb[3] << 8);
                }
                if (out_depth) *reinterpret_cast<float4 *>(out_depth + o) = make_float4(dep[0], dep[1], dep[2], dep[3]);
                if (out_ids) *reinterpret_cast<uint4 *>(out_ids + o) = make_uint4(id[0], id[1], id[2], id[3]);
            } else if constexpr (K == 2) {
                if (out_rgb) {
                    // two packed 24-bit RGB values -> three little-endian halfwords
                    uint16_t *r16 = reinterpret_cast<uint16_t *>(out_rgb + 3 * o);
                    r16[0] = (uint16_t)rgb[0];
                    r16[1] = (uint16_t)((rgb[0] >> 16) | (rgb[1] << 8));
                    r16[2] = (uint16_t)(rgb[1] >> 8);
                }
                if (out_depth) *reinterpret_cast<float2 *>(out_depth + o) = make_float2(dep[0], dep[1]);
                if (out_ids) *reinterpret_cast<uint2 *>(out_ids + o) = make_uint2(id[0], id[1]);
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; k++) {
                if ((uint32_t)k >= n) break;
                if (out_rgb) {
                    out_rgb[3 * (o + k) + 0] = (uint8_t)(rgb[k] & 255u);
                    out_rgb[3 * (o + k) + 1] = (uint8_t)((rgb[k] >> 8) & 255u);
                    out_rgb[3 * (o + k) + 2] = (uint8_t)((rgb[k] >> 16) & 255u);
                }
                if (out_depth) out_depth[o + k] = dep[k];
                if (out_ids) out_ids[o + k] = id[k];
            }
        }
    }
}

// Shading of one render call. G = false when the host's bound proves that no
// view of the call can snap a vertex beyond +-2^30 sub-pixels (no guard-band
// path compiled in: the common case); G = true otherwise. A view the
// rasteriser flagged for the guard band in a G = false launch would mean
// that bound failed: it is reported (kErrRange) and shaded without it.
template <bool G, bool N>
__global__ void __launch_bounds__(kShadeThreads, 8) shade_kernel(const Params p, uint32_t view0)
{
    grid_dependency_wait();
    __shared__ float sM[12];
    __shared__ SceneDev sS;
    __shared__ uint32_t s_frame, s_agent, s_outputs;
    const uint32_t vi = view0 + blockIdx.y;
    if (vi >= p.dyn[0]) return;
    if (threadIdx.x < 12) sM[threadIdx.x] = p.views[vi].M[threadIdx.x];
    if (threadIdx.x == 0) {
        sS = p.scenes[p.views[vi].scene];
        s_frame = p.views[vi].frame;
        s_agent = p.views[vi].agent;
        s_outputs = p.views[vi].outputs;
    }
    __syncthreads();
    const uint32_t outputs = s_outputs;
    if (!G && (outputs & kViewGuard) && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&g_device_err, kErrRange);
    if (!(outputs & HSR_OUT_RGB))
        shade_rows<0, G, N>(p, sS, sM, vi, s_frame, s_agent, outputs);
    else if (sS.color_mode == kColorTexture)
        shade_rows<2, G, N>(p, sS, sM, vi, s_frame, s_agent, outputs);
    else if (sS.color_mode == kColorVertex)
        shade_rows<3, G, N>(p, sS, sM, vi, s_frame, s_agent, outputs);
    else
        shade_rows<0, G, N>(p, sS, sM, vi, s_frame, s_agent, outputs);
}

constexpr size_t kRasterSmem = kRasterWarps * (2 * sizeof(MeshletStage) + kMeshletVerts * sizeof(EyeHot)) +
                               kRasterWarps * kBigCap * sizeof(BigTri);

static cudaError_t set_raster_smem_attr(int dev)
{
    static int attr_dev[64];
    static bool init = false;
    if (!init) {
        for (int &a : attr_dev) a = 0;
        init = true;
    }
    if (dev >= 0 && dev < 64 && attr_dev[dev]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(raster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRasterSmem);
    if (e == cudaSuccess && dev >= 0 && dev < 64) attr_dev[dev] = 1;
    return e;
}

// --------------------------------------------------------------------- stage timing
// Diagnostic: CUDA events recorded around each stage of every launch while
// enabled (one set of events per process; meant for single-threaded use).
namespace {
bool g_timing = false;
int g_timing_dev = -1;
cudaEvent_t g_ev[4] = {nullptr, nullptr, nullptr, nullptr};
bool g_ev_recorded = false;
}  // namespace

cudaError_t stage_timing_enable(bool on)
{
    if (on) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (g_timing_dev != dev) {
            for (auto &ev : g_ev)
                if (ev) {
                    cudaEventDestroy(ev);
                    ev = nullptr;
                }
            for (auto &ev : g_ev) {
                e = cudaEventCreate(&ev);
                if (e != cudaSuccess) return e;
            }
            g_timing_dev = dev;
        }
    }
    g_timing = on;
    g_ev_recorded = false;
    return cudaSuccess;
}

cudaError_t stage_timing_read(float ms[4])
{
    if (!g_ev_recorded) return cudaErrorNotReady;
    cudaError_t e = cudaEventSynchronize(g_ev[3]);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < 3; k++) {
        e = cudaEventElapsedTime(&ms[k], g_ev[k], g_ev[k + 1]);
        if (e != cudaSuccess) return e;
    }
    return cudaEventElapsedTime(&ms[3], g_ev[0], g_ev[3]);
}

namespace {
uint32_t *g_stats = nullptr;      // device counters (9 words), allocated when enabled
bool g_stats_on = false;
}  // namespace

uint32_t *stage_stats_buffer() { return g_stats_on ? g_stats : nullptr; }

cudaError_t stage_stats_enable(bool on)
{
    if (on && !g_stats) {
        cudaError_t e = cudaMalloc(&g_stats, 16 * sizeof(uint32_t));
        if (e != cudaSuccess) return e;
    }
    g_stats_on = on;
    return cudaSuccess;
}

cudaError_t stage_stats_read(uint32_t out[6])
{
    if (!g_stats) return cudaErrorNotReady;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    return cudaMemcpy(out, g_stats, 9 * sizeof(uint32_t), cudaMemcpyDeviceToHost);
}

static inline void mark(int k, cudaStream_t stream)
{
    if (g_timing) cudaEventRecord(g_ev[k], stream);
}

// --------------------------------------------------------------------- launch
static cudaError_t set_raster_smem_attr(int dev);

cudaError_t read_device_errors(uint32_t *flags, bool clear)
{
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(flags, g_device_err, sizeof(uint32_t));
    if (e == cudaSuccess && clear) {
        const uint32_t zero = 0;
        e = cudaMemcpyToSymbol(g_device_err, &zero, sizeof(uint32_t));
    }
    return e;
}

static uint32_t g_fault_tx = 0;
uint32_t debug_fault_tx() { return g_fault_tx; }
void set_debug_fault_tx(uint32_t b) { g_fault_tx = b; }

cudaError_t prepare_kernels()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    return set_raster_smem_attr(dev);
}

// Launch of a kernel that, with `pdl`, may start while the kernel before it
// on the stream is finishing (programmatic dependent launch): its CTAs are
// scheduled once every CTA of that kernel has allowed it, and wait for its
// completion (grid_dependency_wait) before touching memory, so only the
// launch latency and CTA start-up overlap. Without `pdl` it is an ordinary
// launch (the wait then returns at once).
template <typename... KArgs, typename... Args>
static cudaError_t launch_dependent(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                    cudaStream_t stream, Args... args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// SM count of a device, queried once per device.
static cudaError_t device_sms(int dev, int *sms)
{
    static int cache[64] = {};
    if (dev >= 0 && dev < 64 && cache[dev] > 0) {
        *sms = cache[dev];
        return cudaSuccess;
    }
    const cudaError_t e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && dev >= 0 && dev < 64) cache[dev] = *sms;
    return e;
}

cudaError_t launch_render(const Params &p, const LaunchCfg &cfg, cudaStream_t stream, bool guard, bool noise,
                          bool pdl)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = device_sms(dev, &sms);
    if (e != cudaSuccess) return e;
    mark(0, stream);
    if (p.stats) {
        e = cudaMemsetAsync(p.stats, 0, 9 * sizeof(uint32_t), stream);
        if (e != cudaSuccess) return e;
    }
    // culling (and the z-buffer clear it performs) runs for every call
    // grid from the work: the z-buffer clear (16 bytes per thread, 8 stores
    // each) and the (view, group) items (one per warp: an item is a chain of
    // dependent record loads, so small calls want many warps in flight),
    // capped at 8 CTAs per SM
    const uint64_t clear_blocks = ((uint64_t)p.n_views * p.width * p.height / 2 + 2047) / 2048;
    const uint64_t item_blocks = ((uint64_t)p.total_items + 7) / 8;
    const uint32_t cull_blocks = (uint32_t)std::max<uint64_t>(
        1, std::min<uint64_t>(std::max(clear_blocks, item_blocks), (uint64_t)sms * 8));
    Params pc = p;
    pc.cull_views = (uint32_t)std::max<uint64_t>(
        1, std::min<uint64_t>(kCullViews, (uint64_t)p.total_items / ((uint64_t)sms * 48)));
    if (p.n_slots <= kCullSlots)
        cull_kernel<<<cull_blocks, 256, 0, stream>>>(pc);
    else
        cull_kernel_vg<<<cull_blocks, 256, 0, stream>>>(pc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (p.total_items > 0) {
        mark(1, stream);
        e = set_raster_smem_attr(dev);
        if (e != cudaSuccess) return e;
        const uint32_t hiz_threads = p.n_views * p.hiz_w * p.hiz_h * 4u;
        const uint32_t hiz_blocks = std::min<uint32_t>((hiz_threads + 255) / 256, (uint32_t)sms * 16);
        for (uint32_t ph = 0; ph < std::max<uint32_t>(p.n_phases, 1u); ph++) {
            if (ph > 0) {
                e = launch_dependent(pdl, hiz_kernel, dim3(hiz_blocks), dim3(256), 0, stream, p);
                if (e != cudaSuccess) return e;
                e = launch_dependent(pdl, hiz_pyramid_kernel, dim3(p.n_views), dim3(256), 0, stream, p);
                if (e != cudaSuccess) return e;
                const uint32_t occl_blocks = std::min<uint32_t>((p.vis_cap + 255) / 256, (uint32_t)sms * 16);
                e = launch_dependent(pdl, occl_kernel, dim3(std::max(occl_blocks, 1u)), dim3(256), 0, stream, p, ph);
                if (e != cudaSuccess) return e;
            }
            e = launch_dependent(pdl, raster_kernel, dim3((uint32_t)sms * cfg.raster_ctas_per_sm), dim3(kRasterThreads),
                                 kRasterSmem, stream, p, ph);
            if (e != cudaSuccess) return e;
            if (p.big_rec) {
                e = launch_dependent(pdl, big_raster_kernel, dim3((uint32_t)sms * 8), dim3(256), 0, stream, p, ph);
                if (e != cudaSuccess) return e;
            }
        }
    } else {
        mark(1, stream);
    }
    mark(2, stream);
    // runs of kShadePx pixels per view; each thread takes up to eight of them
    // (grid-stride), enough to amortise a CTA's prologue (the view's scene
    // record), while the call keeps about four waves of resident CTAs
    const uint32_t quads = ((p.width + kShadePx - 1) / kShadePx) * p.height;
    const uint64_t resident = (uint64_t)sms * 8u * kShadeThreads;
    const uint32_t per_thread =
        (uint32_t)std::min<uint64_t>(8, std::max<uint64_t>(1, (uint64_t)quads * p.n_views / (4 * resident)));
    const uint32_t bx =
        std::min<uint32_t>((quads + kShadeThreads * per_thread - 1) / (kShadeThreads * per_thread), 1024);
    for (uint32_t v0 = 0; v0 < p.n_views; v0 += 65535) {
        const uint32_t nv = std::min<uint32_t>(65535, p.n_views - v0);
        void (*shade)(Params, uint32_t) = guard ? (noise ? shade_kernel<true, true> : shade_kernel<true, false>)
                                                : (noise ? shade_kernel<false, true> : shade_kernel<false, false>);
        e = launch_dependent(pdl, shade, dim3(bx, nv), dim3(kShadeThreads), 0, stream, p, v0);
        if (e != cudaSuccess) return e;
    }

    mark(3, stream);
    if (g_timing) g_ev_recorded = true;
    return cudaSuccess;
}

}  // namespace hsr
