// C-ABI of the sensor-rendering library (include/hsr.h): argument checking,
// scene loading (device-resident meshlet layout), per-view camera setup on the
// host, and launch of the fused render kernel.
#include "../../include/hsr.h"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "hsr_internal.h"

using namespace hsr;

struct hsr_scene {
    int device = 0;
    SceneDev dev{};
    SceneDev *dev_desc = nullptr;      // device copy of `dev`
    std::vector<void *> allocs;
    hsr_scene_info info{};
};

namespace {

constexpr double kCoordLimit = 1048576.0;       // |vertex coordinate| <= 2^20
constexpr double kSnapLimit = 1073741824.0;     // |snapped coordinate| < 2^30

bool finite3(const float *v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

template <typename T>
cudaError_t upload(hsr_scene *s, const T *host, size_t count, const T **out)
{
    *out = nullptr;
    if (count == 0) return cudaSuccess;
    void *d = nullptr;
    cudaError_t e = cudaMalloc(&d, count * sizeof(T));
    if (e != cudaSuccess) return e;
    s->allocs.push_back(d);
    s->info.device_bytes += count * sizeof(T);
    e = cudaMemcpy(d, host, count * sizeof(T), cudaMemcpyHostToDevice);
    *out = static_cast<const T *>(d);
    return e;
}

void free_scene(hsr_scene *s)
{
    if (!s) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    cudaDeviceSynchronize();
    for (void *p : s->allocs) cudaFree(p);
    cudaSetDevice(prev);
    delete s;
}

int cuda_status(cudaError_t e) { return e == cudaErrorMemoryAllocation ? HSR_ERR_OOM : HSR_ERR_CUDA; }

// Morton interleave of three 21-bit integers.
uint64_t spread21(uint64_t x)
{
    x &= 0x1FFFFF;
    x = (x | x << 32) & 0x1F00000000FFFFULL;
    x = (x | x << 16) & 0x1F0000FF0000FFULL;
    x = (x | x << 8) & 0x100F00F00F00F00FULL;
    x = (x | x << 4) & 0x10C30C30C30C30C3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}

// Camera matrix (reading of Sec. 4 "Sensory input": a pinhole sensor at the
// agent pose). Double precision, fixed operation order, rounded once to float.
bool camera_matrix(const hsr_pose &pose, float M[12])
{
    for (int i = 0; i < 3; i++)
        if (!std::isfinite(pose.pos[i])) return false;
    for (int i = 0; i < 4; i++)
        if (!std::isfinite(pose.quat[i])) return false;
    double w = pose.quat[0], x = pose.quat[1], y = pose.quat[2], z = pose.quat[3];
    const double n = std::sqrt(((w * w + x * x) + y * y) + z * z);
    if (!(std::fabs(n - 1.0) <= 1e-3)) return false;
    w /= n; x /= n; y /= n; z /= n;
    double R[3][3];
    R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    R[0][1] = 2.0 * (x * y - w * z);
    R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z);
    R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y);
    R[2][1] = 2.0 * (y * z + w * x);
    R[2][2] = 1.0 - 2.0 * (x * x + y * y);
    const double px = pose.pos[0], py = pose.pos[1], pz = pose.pos[2];
    for (int i = 0; i < 3; i++) {
        for (int j = 0; j < 3; j++) M[i * 4 + j] = (float)R[j][i];
        M[i * 4 + 3] = (float)(-((R[0][i] * px + R[1][i] * py) + R[2][i] * pz));
    }
    return true;
}

bool intrinsics_ok(const hsr_intrinsics *in)
{
    if (!in) return false;
    const float v[6] = {in->fx, in->fy, in->cx, in->cy, in->znear, in->zfar};
    for (float f : v)
        if (!std::isfinite(f)) return false;
    return in->fx > 0.f && in->fy > 0.f && in->znear > 0.f && in->zfar > in->znear;
}

// Smallest positive float q with 1/q <= far (both rounded to nearest), so the
// per-fragment test "1/q > far -> discard" becomes "q < q_far -> discard".
float far_threshold(float zfar)
{
    volatile float one = 1.0f;
    float q = one / zfar;
    while (one / q > zfar) q = std::nextafter(q, FLT_MAX);
    for (;;) {
        const float lo = std::nextafter(q, 0.0f);
        if (lo <= 0.0f || one / lo > zfar) break;
        q = lo;
    }
    return q;
}

// Conservative bound on |256 sx| and |256 sy| for a view of this scene: any
// vertex (or near-clipped point) has |x_e|, |y_e| <= distance to the farthest
// box corner and d >= near.
bool snap_in_range(const hsr_scene *s, const hsr_pose &pose, const hsr_intrinsics &in)
{
    double r2 = 0.0;
    for (int c = 0; c < 8; c++) {
        double d2 = 0.0;
        for (int k = 0; k < 3; k++) {
            const double v = (c >> k) & 1 ? s->info.aabb_max[k] : s->info.aabb_min[k];
            const double dd = v - (double)pose.pos[k];
            d2 += dd * dd;
        }
        r2 = std::max(r2, d2);
    }
    const double R = std::sqrt(r2) * (1.0 + 1e-6) + 1e-6;
    const double f = std::max((double)in.fx, (double)in.fy);
    const double c = std::max(std::fabs((double)in.cx), std::fabs((double)in.cy));
    const double bound = 256.0 * (f * R / (double)in.znear + c + 2.0);
    return bound < kSnapLimit;
}

struct Staging {
    void *host = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    bool pending = false;
    ~Staging()
    {
        if (pending && done) cudaEventSynchronize(done);
        if (host) cudaFreeHost(host);
        if (done) cudaEventDestroy(done);
    }
};
thread_local Staging g_staging;

LaunchCfg default_cfg(uint32_t width, uint32_t height)
{
    LaunchCfg c;
    c.region_w = std::min<uint32_t>(64, width);
    c.region_h = std::min<uint32_t>(64, height);
    return c;
}

int sm_count()
{
    static int cached = -1;
    if (cached < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    }
    return cached;
}

// Shared body of hsr_render / hsr_render_batch.
int render_views(const hsr_scene *const *scenes, uint32_t n_scenes, const uint32_t *scene_of_agent,
                 const hsr_pose *poses, uint32_t n, const hsr_intrinsics *intr, uint32_t width, uint32_t height,
                 uint8_t *rgb, float *depth, uint32_t *ids, void *stream_ptr, const LaunchCfg *cfg_in)
{
    if (!scenes || n_scenes == 0 || !poses || n == 0 || !rgb || !depth) return HSR_ERR_INVALID_ARG;
    if (width == 0 || height == 0 || width > 4096 || height > 4096) return HSR_ERR_INVALID_ARG;
    if (!intrinsics_ok(intr)) return HSR_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < n_scenes; i++)
        if (!scenes[i]) return HSR_ERR_INVALID_ARG;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);

    // host: per-view camera setup (a1)
    const size_t scene_bytes = sizeof(SceneDev) * n_scenes;
    const size_t head = 256;
    const size_t views_off = head + ((scene_bytes + 255) / 256) * 256;
    const size_t total = views_off + sizeof(View) * (size_t)n;
    Staging &st = g_staging;
    if (st.pending) {
        if (cudaEventSynchronize(st.done) != cudaSuccess) return HSR_ERR_CUDA;
        st.pending = false;
    }
    if (st.cap < total) {
        if (st.host) cudaFreeHost(st.host);
        st.host = nullptr;
        st.cap = 0;
        const size_t cap = std::max<size_t>(total, 64 * 1024);
        if (cudaHostAlloc(&st.host, cap, cudaHostAllocDefault) != cudaSuccess) return HSR_ERR_OOM;
        st.cap = cap;
    }
    if (!st.done && cudaEventCreateWithFlags(&st.done, cudaEventDisableTiming) != cudaSuccess) return HSR_ERR_CUDA;
    auto *hbuf = static_cast<unsigned char *>(st.host);
    std::memset(hbuf, 0, head);
    SceneDev *hs = reinterpret_cast<SceneDev *>(hbuf + head);
    for (uint32_t i = 0; i < n_scenes; i++) hs[i] = scenes[i]->dev;
    View *hv = reinterpret_cast<View *>(hbuf + views_off);
    for (uint32_t i = 0; i < n; i++) {
        const uint32_t sidx = scene_of_agent ? scene_of_agent[i] : 0u;
        if (sidx >= n_scenes) return HSR_ERR_INVALID_ARG;
        View &v = hv[i];
        std::memset(&v, 0, sizeof(View));
        if (!camera_matrix(poses[i], v.M)) return HSR_ERR_INVALID_ARG;
        if (!snap_in_range(scenes[sidx], poses[i], *intr)) return HSR_ERR_INVALID_ARG;
        v.scene = sidx;
        v.frame = i;
    }

    LaunchCfg cfg = cfg_in ? *cfg_in : default_cfg(width, height);
    cfg.region_w = std::min(cfg.region_w, width);
    cfg.region_h = std::min(cfg.region_h, height);

    void *dbuf = nullptr;
    cudaError_t e = cudaMallocAsync(&dbuf, total, stream);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaMemcpyAsync(dbuf, hbuf, total, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaEventRecord(st.done, stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(dbuf, stream);
        return HSR_ERR_CUDA;
    }
    st.pending = true;

    Params p{};
    auto *dchar = static_cast<unsigned char *>(dbuf);
    p.work_counter = cfg.persistent ? reinterpret_cast<uint32_t *>(dchar) : nullptr;
    p.scenes = reinterpret_cast<const SceneDev *>(dchar + head);
    p.views = reinterpret_cast<const View *>(dchar + views_off);
    p.rgb = rgb;
    p.depth = depth;
    p.ids = ids;
    p.n_views = n;
    p.width = width;
    p.height = height;
    p.fx = intr->fx; p.fy = intr->fy; p.cx = intr->cx; p.cy = intr->cy;
    p.znear = intr->znear; p.zfar = intr->zfar;
    p.q_far = far_threshold(intr->zfar);
    p.region_w = cfg.region_w;
    p.region_h = cfg.region_h;
    p.regions_x = (width + cfg.region_w - 1) / cfg.region_w;
    p.regions_y = (height + cfg.region_h - 1) / cfg.region_h;
    p.n_items = n * p.regions_x * p.regions_y;
    p.small_px = cfg.small_px;
    (void)sm_count;
    e = launch_render(p, cfg, stream);
    cudaError_t ef = cudaFreeAsync(dbuf, stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (ef != cudaSuccess) return HSR_ERR_CUDA;
    return HSR_OK;
}

}  // namespace

extern "C" {

const char *hsr_version(void) { return "0.1.0"; }

const char *hsr_status_string(int s)
{
    switch (s) {
        case HSR_OK: return "ok";
        case HSR_ERR_INVALID_ARG: return "invalid argument";
        case HSR_ERR_OOM: return "out of memory";
        case HSR_ERR_CUDA: return "CUDA runtime error";
        case HSR_ERR_TIMEOUT: return "bounded device wait expired";
        case HSR_ERR_OVERFLOW: return "fixed-capacity buffer overflow";
        case HSR_ERR_NO_DEVICE: return "no CUDA device";
        default: return "unknown status";
    }
}

int hsr_scene_load(const float *xyz, uint32_t n_verts, const uint32_t *idx, uint32_t n_tris, const float *uv,
                   const uint8_t *vert_rgb, const uint8_t *atlas, uint32_t atlas_w, uint32_t atlas_h,
                   const uint32_t *tri_semantic, hsr_scene **out)
{
    if (!out) return HSR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!xyz || !idx || n_verts == 0 || n_tris == 0) return HSR_ERR_INVALID_ARG;
    if (atlas && (atlas_w == 0 || atlas_h == 0 || atlas_w > 65536 || atlas_h > 65536)) return HSR_ERR_INVALID_ARG;
    for (size_t i = 0; i < (size_t)n_verts; i++) {
        const float *v = xyz + 3 * i;
        if (!finite3(v) || std::fabs(v[0]) > kCoordLimit || std::fabs(v[1]) > kCoordLimit ||
            std::fabs(v[2]) > kCoordLimit)
            return HSR_ERR_INVALID_ARG;
    }
    for (size_t i = 0; i < 3 * (size_t)n_tris; i++)
        if (idx[i] >= n_verts) return HSR_ERR_INVALID_ARG;
    if (uv)
        for (size_t i = 0; i < 2 * (size_t)n_verts; i++)
            if (!std::isfinite(uv[i])) return HSR_ERR_INVALID_ARG;
    if (tri_semantic)
        for (size_t i = 0; i < n_tris; i++)
            if (tri_semantic[i] == 0xFFFFFFFFu) return HSR_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return HSR_ERR_NO_DEVICE;

    hsr_scene *s = new (std::nothrow) hsr_scene();
    if (!s) return HSR_ERR_OOM;
    cudaGetDevice(&s->device);
    try {
        // canonical cyclic order of each index triple
        std::vector<uint32_t> canon(3 * (size_t)n_tris);
        for (size_t t = 0; t < n_tris; t++) {
            const uint32_t a = idx[3 * t], b = idx[3 * t + 1], c = idx[3 * t + 2];
            uint32_t r[3][3] = {{a, b, c}, {b, c, a}, {c, a, b}};
            int best = 0;
            for (int k = 1; k < 3; k++)
                if (std::lexicographical_compare(r[k], r[k] + 3, r[best], r[best] + 3)) best = k;
            canon[3 * t] = r[best][0];
            canon[3 * t + 1] = r[best][1];
            canon[3 * t + 2] = r[best][2];
        }
        // scene bounds
        float bmin[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, bmax[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
        for (size_t i = 0; i < n_verts; i++)
            for (int k = 0; k < 3; k++) {
                bmin[k] = std::min(bmin[k], xyz[3 * i + k]);
                bmax[k] = std::max(bmax[k], xyz[3 * i + k]);
            }
        // Morton order of centroids
        std::vector<std::pair<uint64_t, uint32_t>> order(n_tris);
        double ext[3];
        for (int k = 0; k < 3; k++) ext[k] = std::max(1e-12, (double)bmax[k] - (double)bmin[k]);
        for (uint32_t t = 0; t < n_tris; t++) {
            uint64_t code = 0;
            for (int k = 0; k < 3; k++) {
                const double c = ((double)xyz[3 * (size_t)canon[3 * (size_t)t] + k] +
                                  (double)xyz[3 * (size_t)canon[3 * (size_t)t + 1] + k] +
                                  (double)xyz[3 * (size_t)canon[3 * (size_t)t + 2] + k]) / 3.0;
                double f = (c - bmin[k]) / ext[k];
                f = std::min(std::max(f, 0.0), 1.0);
                code |= spread21((uint64_t)(f * 2097151.0)) << k;
            }
            order[t] = {code, t};
        }
        std::sort(order.begin(), order.end());
        // greedy meshlets: <= 32 triangles, <= 64 distinct vertices
        std::vector<Meshlet> meshlets;
        std::vector<float4> mvert;
        std::vector<uint2> mtri;
        std::vector<uint32_t> stamp(n_verts, 0xFFFFFFFFu);
        std::vector<uint8_t> local(n_verts, 0);
        std::vector<uint32_t> cur_v;
        std::vector<uint32_t> cur_t;
        auto flush = [&]() {
            if (cur_t.empty()) return;
            const uint32_t mid = (uint32_t)meshlets.size();
            Meshlet m{};
            m.vbase = (uint32_t)mvert.size();
            m.tbase = (uint32_t)mtri.size();
            float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
            for (uint32_t v : cur_v) {
                float4 p;
                p.x = xyz[3 * (size_t)v];
                p.y = xyz[3 * (size_t)v + 1];
                p.z = xyz[3 * (size_t)v + 2];
                uint32_t g = v;
                std::memcpy(&p.w, &g, 4);
                mvert.push_back(p);
                lo[0] = std::min(lo[0], p.x); lo[1] = std::min(lo[1], p.y); lo[2] = std::min(lo[2], p.z);
                hi[0] = std::max(hi[0], p.x); hi[1] = std::max(hi[1], p.y); hi[2] = std::max(hi[2], p.z);
            }
            for (uint32_t t : cur_t) {
                uint2 e;
                e.x = (uint32_t)local[canon[3 * (size_t)t]] | ((uint32_t)local[canon[3 * (size_t)t + 1]] << 8) |
                      ((uint32_t)local[canon[3 * (size_t)t + 2]] << 16);
                e.y = t;
                mtri.push_back(e);
            }
            // inflate so the float plane tests stay conservative
            for (int k = 0; k < 3; k++) {
                const float pad = 1e-4f + 1e-6f * std::max(std::fabs(lo[k]), std::fabs(hi[k]));
                m.bmin[k] = lo[k] - pad;
                m.bmax[k] = hi[k] + pad;
            }
            meshlets.push_back(m);
            (void)mid;
            cur_v.clear();
            cur_t.clear();
        };
        uint32_t mstamp = 0;
        for (const auto &ot : order) {
            const uint32_t t = ot.second;
            const uint32_t tv[3] = {canon[3 * (size_t)t], canon[3 * (size_t)t + 1], canon[3 * (size_t)t + 2]};
            int fresh = 0;
            for (int k = 0; k < 3; k++) {
                if (stamp[tv[k]] == mstamp) continue;
                bool dup = false;
                for (int j = 0; j < k; j++) dup |= tv[j] == tv[k];
                if (!dup) fresh++;
            }
            if ((int)cur_t.size() == kMeshletTris || (int)cur_v.size() + fresh > kMeshletVerts) {
                flush();
                mstamp++;
            }
            for (int k = 0; k < 3; k++) {
                const uint32_t v = canon[3 * (size_t)t + k];
                if (stamp[v] != mstamp) {
                    stamp[v] = mstamp;
                    local[v] = (uint8_t)cur_v.size();
                    cur_v.push_back(v);
                }
            }
            cur_t.push_back(t);
        }
        flush();
        const uint32_t n_meshlets = (uint32_t)meshlets.size();
        Meshlet sentinel{};
        sentinel.vbase = (uint32_t)mvert.size();
        sentinel.tbase = (uint32_t)mtri.size();
        meshlets.push_back(sentinel);
        // groups of 32 meshlets
        std::vector<Group> groups;
        for (uint32_t m0 = 0; m0 < n_meshlets; m0 += kGroupMeshlets) {
            Group g{};
            g.m0 = m0;
            g.m1 = std::min(n_meshlets, m0 + kGroupMeshlets);
            for (int k = 0; k < 3; k++) {
                g.bmin[k] = FLT_MAX;
                g.bmax[k] = -FLT_MAX;
            }
            for (uint32_t m = g.m0; m < g.m1; m++)
                for (int k = 0; k < 3; k++) {
                    g.bmin[k] = std::min(g.bmin[k], meshlets[m].bmin[k]);
                    g.bmax[k] = std::max(g.bmax[k], meshlets[m].bmax[k]);
                }
            groups.push_back(g);
        }
        // per-triangle canonical indices + output id; per-vertex attributes
        std::vector<uint4> tri(n_tris);
        for (size_t t = 0; t < n_tris; t++) {
            tri[t].x = canon[3 * t];
            tri[t].y = canon[3 * t + 1];
            tri[t].z = canon[3 * t + 2];
            tri[t].w = tri_semantic ? tri_semantic[t] : (uint32_t)t;
        }
        std::vector<float4> vert(n_verts);
        for (size_t i = 0; i < n_verts; i++) vert[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], 0.f);

        cudaError_t e = cudaSuccess;
        SceneDev &d = s->dev;
        const Meshlet *dm;
        const Group *dg;
        const float4 *dmv, *dv;
        const uint2 *dmt;
        const uint4 *dt;
        if ((e = upload(s, meshlets.data(), meshlets.size(), &dm)) != cudaSuccess) throw e;
        if ((e = upload(s, groups.data(), groups.size(), &dg)) != cudaSuccess) throw e;
        if ((e = upload(s, mvert.data(), mvert.size(), &dmv)) != cudaSuccess) throw e;
        if ((e = upload(s, mtri.data(), mtri.size(), &dmt)) != cudaSuccess) throw e;
        if ((e = upload(s, tri.data(), tri.size(), &dt)) != cudaSuccess) throw e;
        if ((e = upload(s, vert.data(), vert.size(), &dv)) != cudaSuccess) throw e;
        d.meshlets = dm;
        d.groups = dg;
        d.mvert = dmv;
        d.mtri = dmt;
        d.tri = dt;
        d.vert = dv;
        d.n_groups = (uint32_t)groups.size();
        d.n_meshlets = n_meshlets;
        d.n_tris = n_tris;
        d.n_verts = n_verts;
        d.color_mode = kColorWhite;
        if (uv && atlas) {
            const float2 *duv;
            const uint32_t *da;
            if ((e = upload(s, reinterpret_cast<const float2 *>(uv), n_verts, &duv)) != cudaSuccess) throw e;
            if ((e = upload(s, reinterpret_cast<const uint32_t *>(atlas), (size_t)atlas_w * atlas_h, &da)) !=
                cudaSuccess)
                throw e;
            d.uv = duv;
            d.atlas = da;
            d.atlas_w = atlas_w;
            d.atlas_h = atlas_h;
            d.color_mode = kColorTexture;
        } else if (vert_rgb) {
            std::vector<uint32_t> c(n_verts);
            for (size_t i = 0; i < n_verts; i++)
                c[i] = (uint32_t)vert_rgb[3 * i] | ((uint32_t)vert_rgb[3 * i + 1] << 8) |
                       ((uint32_t)vert_rgb[3 * i + 2] << 16);
            const uint32_t *dc;
            if ((e = upload(s, c.data(), c.size(), &dc)) != cudaSuccess) throw e;
            d.vrgb = dc;
            d.color_mode = kColorVertex;
        }
        const SceneDev *dd;
        if ((e = upload(s, &d, 1, &dd)) != cudaSuccess) throw e;
        s->dev_desc = const_cast<SceneDev *>(dd);
        s->info.n_tris = n_tris;
        s->info.n_verts = n_verts;
        s->info.n_meshlets = n_meshlets;
        s->info.n_groups = (uint32_t)groups.size();
        for (int k = 0; k < 3; k++) {
            s->info.aabb_min[k] = bmin[k];
            s->info.aabb_max[k] = bmax[k];
        }
    } catch (cudaError_t e) {
        free_scene(s);
        return cuda_status(e);
    } catch (const std::bad_alloc &) {
        free_scene(s);
        return HSR_ERR_OOM;
    }
    *out = s;
    return HSR_OK;
}

int hsr_scene_free(hsr_scene *scene)
{
    free_scene(scene);
    return HSR_OK;
}

int hsr_scene_get_info(const hsr_scene *scene, hsr_scene_info *info)
{
    if (!scene || !info) return HSR_ERR_INVALID_ARG;
    *info = scene->info;
    return HSR_OK;
}

int hsr_render(const hsr_scene *scene, const hsr_pose *poses, uint32_t n, const hsr_intrinsics *intr,
               uint32_t width, uint32_t height, uint8_t *rgb, float *depth, uint32_t *ids, void *cuda_stream)
{
    if (!scene) return HSR_ERR_INVALID_ARG;
    const hsr_scene *scenes[1] = {scene};
    return render_views(scenes, 1, nullptr, poses, n, intr, width, height, rgb, depth, ids, cuda_stream, nullptr);
}

int hsr_render_batch(const hsr_scene *const *scenes, uint32_t n_scenes, const uint32_t *scene_of_agent,
                     const hsr_pose *poses, uint32_t n, const hsr_intrinsics *intr, uint32_t width,
                     uint32_t height, uint8_t *rgb, float *depth, uint32_t *ids, void *cuda_stream)
{
    if (!scene_of_agent) return HSR_ERR_INVALID_ARG;
    return render_views(scenes, n_scenes, scene_of_agent, poses, n, intr, width, height, rgb, depth, ids,
                        cuda_stream, nullptr);
}

}  // extern "C"
