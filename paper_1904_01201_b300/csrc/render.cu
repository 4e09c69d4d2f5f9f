// Fused render kernel: one CTA per (view, screen region) work item, all five
// stages in one launch so no intermediate ever leaves the SM:
//   K3 bin   — groups / meshlets culled against the region frustum (bin.cuh)
//   K1       — meshlet vertices transformed and snapped into a per-warp
//              shared-memory cache (transform.cuh)
//   K2       — per-triangle reject / near clip / cull / depth plane (setup.cuh)
//   K4       — per-thread or per-warp fixed-point raster into the region's
//              shared-memory z-buffer (raster.cuh)
//   K5       — deferred resolve + shade + store of the region (shade.cuh)
// In persistent mode a grid of (#SM x CTAs/SM) CTAs pulls further work items
// from a global counter; otherwise each CTA renders exactly one item.
#include <cuda_runtime.h>

#include "hsr_internal.h"
#include "kernels/bin.cuh"
#include "kernels/raster.cuh"
#include "kernels/setup.cuh"
#include "kernels/shade.cuh"
#include "kernels/transform.cuh"

namespace hsr {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kGroupChunk = 64;
constexpr int kMlistCap = kGroupChunk * kGroupMeshlets;
constexpr int kBigCap = 2 * kMeshletTris;        // a lane emits at most two sub-triangles

// Shared-memory layout (every section starts on a 128-byte boundary):
//   z-buffer [RW*RH] u64 | vertex caches [warps][64] | big-triangle queues [warps][64] | meshlet queue
__host__ __device__ constexpr size_t align128(size_t b) { return (b + 127) & ~(size_t)127; }
constexpr size_t kVcacheBytes = align128((size_t)kWarps * kMeshletVerts * sizeof(EyeVert));
constexpr size_t kBigqBytes = align128((size_t)kWarps * kBigCap * sizeof(BigTri));
constexpr size_t kMlistBytes = align128((size_t)kMlistCap * sizeof(uint32_t));

__host__ __device__ inline size_t zbuf_bytes(uint32_t rw, uint32_t rh)
{
    return align128((size_t)rw * rh * sizeof(unsigned long long));
}

size_t render_smem_bytes(const LaunchCfg &c)
{
    return zbuf_bytes(c.region_w, c.region_h) + kVcacheBytes + kBigqBytes + kMlistBytes;
}

// Per-lane sub-triangle after setup (at most two per source triangle).
struct SubTri {
    Tri2D t;
    float pa, pb;
    int x0, x1, y0, y1;
    bool small;
};

__device__ __forceinline__ bool finish_setup(SubTri &s, const Params &p, int rx0, int ry0, int rx1, int ry1)
{
    int spanx, spany;
    pixel_range(s.t, s.x0, s.x1, s.y0, s.y1, spanx, spany);
    s.x0 = max(s.x0, rx0);
    s.y0 = max(s.y0, ry0);
    s.x1 = min(s.x1, rx1 - 1);
    s.y1 = min(s.y1, ry1 - 1);
    if (s.x0 > s.x1 || s.y0 > s.y1) return false;      // no sample of this region
    depth_plane(s.t, s.pa, s.pb);
    const int npx = (s.x1 - s.x0 + 1) * (s.y1 - s.y0 + 1);
    s.small = spanx < 32768 && spany < 32768 && npx <= (int)p.small_px;
    return true;
}

__device__ __forceinline__ void process_meshlet(const SceneDev &S, const float *M, const Params &p,
                                                uint32_t m, EyeVert *vc, BigTri *bigq,
                                                unsigned long long *zbuf, int rx0, int ry0, int rx1, int ry1,
                                                int RW, int lane)
{
    const Meshlet ml = S.meshlets[m];
    const uint32_t vend = S.meshlets[m + 1].vbase, tend = S.meshlets[m + 1].tbase;
    const int nv = (int)(vend - ml.vbase), nt = (int)(tend - ml.tbase);
    const float zn = p.znear, zf = p.zfar;

    // K1: transform + snap this meshlet's vertices
    for (int v = lane; v < nv; v += 32) {
        const float4 P = __ldg(S.mvert + ml.vbase + v);
        EyeVert e;
        eye_transform(M, P.x, P.y, P.z, e.xe, e.ye, e.d);
        e.gid = __float_as_uint(P.w);
        if (e.d >= zn) {
            project_snap(e.xe, e.ye, e.d, p.fx, p.fy, p.cx, p.cy, e.q, e.X, e.Y);
        } else {
            e.q = 0.f;
            e.X = e.Y = 0;
        }
        vc[v] = e;
    }
    __syncwarp();

    // K2: one triangle per lane -> up to two front-facing sub-triangles
    SubTri st[2];
    int nst = 0;
    uint32_t id = 0;
    if (lane < nt) {
        const uint2 mt = __ldg(S.mtri + ml.tbase + lane);
        const EyeVert a = vc[mt.x & 255u], b = vc[(mt.x >> 8) & 255u], c = vc[(mt.x >> 16) & 255u];
        id = mt.y;
        const bool all_near = a.d < zn && b.d < zn && c.d < zn;
        const bool all_far = a.d > zf && b.d > zf && c.d > zf;
        if (!all_near && !all_far) {
            if (a.d >= zn && b.d >= zn && c.d >= zn) {
                if (orient_cull(a.X, a.Y, a.q, b.X, b.Y, b.q, c.X, c.Y, c.q, st[0].t) &&
                    finish_setup(st[0], p, rx0, ry0, rx1, ry1))
                    nst = 1;
            } else {
                CVert<0> v[3];
                v[0].xe = a.xe; v[0].ye = a.ye; v[0].d = a.d; v[0].gid = a.gid;
                v[1].xe = b.xe; v[1].ye = b.ye; v[1].d = b.d; v[1].gid = b.gid;
                v[2].xe = c.xe; v[2].ye = c.ye; v[2].d = c.d; v[2].gid = c.gid;
                CVert<0> poly[4];
                const int np = clip_near<0>(v, zn, poly);
                int X[4], Y[4];
                float q[4];
                for (int k = 0; k < np; k++)
                    project_snap(poly[k].xe, poly[k].ye, poly[k].d, p.fx, p.fy, p.cx, p.cy, q[k], X[k], Y[k]);
                for (int f = 0; f + 2 < np; f++) {
                    SubTri &s = st[nst];
                    if (orient_cull(X[0], Y[0], q[0], X[f + 1], Y[f + 1], q[f + 1], X[f + 2], Y[f + 2], q[f + 2], s.t) &&
                        finish_setup(s, p, rx0, ry0, rx1, ry1))
                        nst++;
                }
            }
        }
    }

    // K4: small triangles per thread; the rest through the warp queue
    int qn = 0;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const bool have = k < nst;
        const bool small = have && st[k].small;
        const bool big = have && !st[k].small;
        if (small)
            raster_small(st[k].t, st[k].pa, st[k].pb, id, st[k].x0, st[k].x1, st[k].y0, st[k].y1, p.q_far, zbuf,
                         rx0, ry0, RW);
        const unsigned bm = __ballot_sync(0xFFFFFFFFu, big);
        if (big) {
            BigTri r;
            r.X0 = st[k].t.X0; r.Y0 = st[k].t.Y0;
            r.X1 = st[k].t.X1; r.Y1 = st[k].t.Y1;
            r.X2 = st[k].t.X2; r.Y2 = st[k].t.Y2;
            r.pa = st[k].pa; r.pb = st[k].pb; r.q0 = st[k].t.q0;
            r.id = id;
            r.x0 = (short)st[k].x0; r.x1 = (short)st[k].x1;
            r.y0 = (short)st[k].y0; r.y1 = (short)st[k].y1;
            bigq[qn + __popc(bm & ((1u << lane) - 1u))] = r;
        }
        qn += __popc(bm);
    }
    __syncwarp();
    for (int r = 0; r < qn; r++) raster_big_warp(bigq[r], lane, p.q_far, zbuf, rx0, ry0, RW);
    __syncwarp();
}

__global__ void __launch_bounds__(kThreads, 2) render_kernel(const Params p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int RW = (int)p.region_w, RH = (int)p.region_h;
    unsigned long long *zbuf = reinterpret_cast<unsigned long long *>(smem);
    const size_t zb = zbuf_bytes(p.region_w, p.region_h);
    EyeVert *vcache = reinterpret_cast<EyeVert *>(smem + zb);
    BigTri *bigq = reinterpret_cast<BigTri *>(smem + zb + kVcacheBytes);
    uint32_t *mlist = reinterpret_cast<uint32_t *>(smem + zb + kVcacheBytes + kBigqBytes);

    __shared__ float sM[12];
    __shared__ Plane sPlanes[6];
    __shared__ SceneDev sS;
    __shared__ uint32_t s_item, s_mcount, s_mnext;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    EyeVert *myvc = vcache + warp * kMeshletVerts;
    BigTri *mybig = bigq + warp * kBigCap;
    const uint32_t nreg = p.regions_x * p.regions_y;

    uint32_t item = blockIdx.x;
    while (item < p.n_items) {
        const uint32_t vi = item / nreg, ri = item % nreg;
        const int rx0 = (int)(ri % p.regions_x) * RW, ry0 = (int)(ri / p.regions_x) * RH;
        const int rx1 = min(rx0 + RW, (int)p.width), ry1 = min(ry0 + RH, (int)p.height);
        const View &V = p.views[vi];
        if (threadIdx.x < 12) sM[threadIdx.x] = V.M[threadIdx.x];
        if (threadIdx.x == 0) {
            sS = p.scenes[V.scene];
            s_mcount = 0;
            s_mnext = 0;
        }
        for (int i = threadIdx.x; i < RW * RH; i += kThreads) zbuf[i] = ~0ull;
        __syncthreads();
        if (threadIdx.x < 6) sPlanes[threadIdx.x] = region_plane(threadIdx.x, sM, p, rx0, ry0, rx1, ry1);
        __syncthreads();

        const uint32_t ngroups = sS.n_groups;
        for (uint32_t g0 = 0; g0 < ngroups; g0 += kGroupChunk) {
            // K3: bin groups -> meshlets of this chunk to the region
            for (uint32_t gi = warp; gi < (uint32_t)kGroupChunk && g0 + gi < ngroups; gi += kWarps) {
                const Group g = sS.groups[g0 + gi];
                if (!aabb_visible(sPlanes, g.bmin, g.bmax)) continue;
                const uint32_t m = g.m0 + lane;
                bool vis = false;
                if (m < g.m1) {
                    const Meshlet ml = sS.meshlets[m];
                    vis = aabb_visible(sPlanes, ml.bmin, ml.bmax);
                }
                const unsigned mask = __ballot_sync(0xFFFFFFFFu, vis);
                uint32_t base = 0;
                if (lane == 0 && mask) base = atomicAdd(&s_mcount, (uint32_t)__popc(mask));
                base = __shfl_sync(0xFFFFFFFFu, base, 0);
                if (vis) mlist[base + __popc(mask & ((1u << lane) - 1u))] = m;
            }
            __syncthreads();
            const uint32_t mcount = s_mcount;
            for (;;) {
                uint32_t k = 0;
                if (lane == 0) k = atomicAdd(&s_mnext, 1u);
                k = __shfl_sync(0xFFFFFFFFu, k, 0);
                if (k >= mcount) break;
                process_meshlet(sS, sM, p, mlist[k], myvc, mybig, zbuf, rx0, ry0, rx1, ry1, RW, lane);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                s_mcount = 0;
                s_mnext = 0;
            }
            __syncthreads();
        }

        // K5: resolve, shade, store
        const uint32_t frame = V.frame;
        const size_t fbase = (size_t)frame * p.width * p.height;
        for (int i = threadIdx.x; i < RW * RH; i += kThreads) {
            const int lx = i % RW, ly = i / RW;
            const int px = rx0 + lx, py = ry0 + ly;
            if (px >= rx1 || py >= ry1) continue;
            const ShadeOut o = shade_pixel(sS, sM, p, px, py, zbuf[i]);
            const size_t pi = fbase + (size_t)py * p.width + px;
            p.rgb[3 * pi + 0] = (uint8_t)(o.rgb & 255u);
            p.rgb[3 * pi + 1] = (uint8_t)((o.rgb >> 8) & 255u);
            p.rgb[3 * pi + 2] = (uint8_t)((o.rgb >> 16) & 255u);
            p.depth[pi] = o.depth;
            if (p.ids) p.ids[pi] = o.id;
        }
        if (!p.work_counter) break;
        __syncthreads();
        if (threadIdx.x == 0) s_item = gridDim.x + atomicAdd(p.work_counter, 1u);
        __syncthreads();
        item = s_item;
    }
}

cudaError_t launch_render(const Params &p, const LaunchCfg &cfg, cudaStream_t stream)
{
    const size_t smem = render_smem_bytes(cfg);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(render_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    uint32_t grid = p.n_items;
    if (p.work_counter) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const uint32_t cap = (uint32_t)sms * cfg.ctas_per_sm;
        if (grid > cap) grid = cap;
    }
    if (grid == 0) return cudaSuccess;
    render_kernel<<<grid, kThreads, smem, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace hsr
