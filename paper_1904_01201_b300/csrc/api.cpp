// C-ABI of the sensor-rendering library (include/hsr.h): argument checking,
// scene loading (device-resident meshlet layout), per-view camera setup on the
// host, and launch of the cull / raster / shade kernels.
#include "../../include/hsr.h"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "camera.h"
#include "hsr_internal.h"
#include "launch_defaults.h"

using namespace hsr;

struct hsr_scene {
    int device = 0;
    SceneDev dev{};
    SceneDev *dev_desc = nullptr;      // device copy of `dev`
    std::vector<void *> allocs;
    cudaArray_t atlas_array = nullptr; // the atlas as a texture (2D-local layout) for bilinear gathers
    cudaTextureObject_t atlas_tex = 0;
    hsr_scene_info info{};
};


namespace {

constexpr double kCoordLimit = 1048576.0;       // |vertex coordinate| <= 2^20

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
    if (s->atlas_tex) cudaDestroyTextureObject(s->atlas_tex);
    if (s->atlas_array) cudaFreeArray(s->atlas_array);
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
bool camera_matrix(const hsr_pose &pose, float M[12]) { return camera_from_pose(pose.pos, pose.quat, M); }

// Finite, positive focal lengths, a principal point within 2^16 pixels of
// the image origin (so that the guard band, 2^21 pixels either side of it,
// stays inside the fixed-point range), 2^-20 m <= near < far.
bool intrinsics_ok(const hsr_intrinsics *in)
{
    if (!in) return false;
    const float v[6] = {in->fx, in->fy, in->cx, in->cy, in->znear, in->zfar};
    for (float f : v)
        if (!std::isfinite(f)) return false;
    return in->fx > 0.f && in->fy > 0.f && std::fabs(in->cx) <= 65536.f && std::fabs(in->cy) <= 65536.f &&
           in->znear >= 0x1p-20f && in->zfar > in->znear;
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

// Guard-plane slope of a focal length: 2^21 / f (one IEEE float division),
// the planes |x_e| <= g d project 2^21 pixels either side of the principal point.
float guard_g(float f)
{
    volatile float num = 2097152.0f;
    return num / f;
}

// Page-locked staging of one-shot calls' descriptors, per host thread: a
// ring of kStagingSlots buffers, so that a thread may run that many calls
// ahead of the device before it waits for the upload of an earlier one.
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
constexpr int kStagingSlots = 4;
struct StagingRing {
    Staging slot[kStagingSlots];
    int next = 0;
};
thread_local StagingRing g_staging;

constexpr uint64_t kMaxScratchBytes = 2ull << 30;

// Device scratch of one-shot calls, kept per host thread and reused by its
// next call instead of being allocated and freed every call (descriptors
// and scratch of a call up to kReuseBytes; larger calls take stream-ordered
// allocations). A call on another stream than the previous one first waits,
// on the device, for the previous call's work (the `done` event), so two
// calls never share the buffer at the same time.
constexpr size_t kReuseBytes = 256ull << 20;
struct CallScratch {
    int device = -1;
    unsigned char *d = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    cudaStream_t last = nullptr;
    bool used = false;
    ~CallScratch()
    {
        if (used && done) cudaEventSynchronize(done);
        if (d) cudaFree(d);
        if (done) cudaEventDestroy(done);
    }
    // A buffer of at least `bytes` on the current device, ordered after the
    // previous call's use on `stream`; nullptr if it cannot be had.
    unsigned char *acquire(size_t bytes, cudaStream_t stream)
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
        if (dev != device || cap < bytes) {
            if (used && done && cudaEventSynchronize(done) != cudaSuccess) return nullptr;
            if (d) cudaFree(d);
            if (done) cudaEventDestroy(done);
            d = nullptr;
            done = nullptr;
            cap = 0;
            used = false;
            device = dev;
            const size_t want = std::max<size_t>(bytes, 64ull << 20);
            if (cudaMalloc(&d, want) != cudaSuccess) {
                d = nullptr;
                return nullptr;
            }
            if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) {
                cudaFree(d);
                d = nullptr;
                return nullptr;
            }
            cap = want;
        }
        if (used && stream != last && cudaStreamWaitEvent(stream, done, 0) != cudaSuccess) return nullptr;
        return d;
    }
    // The call's work is queued on `stream`.
    bool release(cudaStream_t stream)
    {
        last = stream;
        used = true;
        return cudaEventRecord(done, stream) == cudaSuccess;
    }
};
thread_local CallScratch g_call_scratch;

void view_planes(const float M[12], const hsr_intrinsics &in, uint32_t W, uint32_t H, float planes[24])
{
    frustum_planes(M, in.fx, in.fy, in.cx, in.cy, in.znear, in.zfar, W, H, planes);
}

// ------------------------------------------------------------ tuned configs
struct TuneKey {
    std::vector<const hsr_scene *> scenes;
    uint32_t n, width, height;
    int ids;
    bool operator<(const TuneKey &o) const
    {
        if (scenes != o.scenes) return scenes < o.scenes;
        if (n != o.n) return n < o.n;
        if (width != o.width) return width < o.width;
        if (height != o.height) return height < o.height;
        return ids < o.ids;
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, LaunchCfg> g_tuned;

TuneKey make_key(const hsr_scene *const *scenes, uint32_t n_scenes, uint32_t n, uint32_t w, uint32_t h, int ids)
{
    TuneKey k;
    k.scenes.assign(scenes, scenes + n_scenes);
    k.n = n;
    k.width = w;
    k.height = h;
    k.ids = ids ? 1 : 0;
    return k;
}

bool lookup_tuned(const TuneKey &k, LaunchCfg &out)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(k);
    if (it == g_tuned.end()) return false;
    out = it->second;
    return true;
}

LaunchCfg from_config(const hsr_config &c)
{
    LaunchCfg l;
    l.small_px = std::min<uint32_t>(std::max<uint32_t>(c.small_px, 1), 32);
    l.bin_px = std::max<uint32_t>(c.bin_px, l.small_px);
    l.chunk = std::min<uint32_t>(std::max<uint32_t>(c.chunk, 1), 32);
    l.raster_ctas_per_sm = std::min<uint32_t>(std::max<uint32_t>(c.ctas_per_sm, 1), 3);
    l.n_phases = std::min<uint32_t>(std::max<uint32_t>(c.n_phases, 1), 3);
    l.phase_r[0] = std::isfinite(c.phase_r[0]) ? std::max(c.phase_r[0], 0.0f) : 3.0f;
    l.phase_r[1] = std::isfinite(c.phase_r[1]) ? std::max(c.phase_r[1], l.phase_r[0]) : 7.0f;
    return l;
}

hsr_config to_config(const LaunchCfg &l)
{
    hsr_config c;
    c.small_px = l.small_px;
    c.bin_px = l.bin_px;
    c.chunk = l.chunk;
    c.ctas_per_sm = l.raster_ctas_per_sm;
    c.n_phases = l.n_phases;
    c.phase_r[0] = l.phase_r[0];
    c.phase_r[1] = l.phase_r[1];
    return c;
}

// ------------------------------------------------------------ render plan
// Layout of the per-render descriptors (host staging and device copy) and of
// the device scratch, for a capacity of n_cap views of the given scenes.
//   descriptors: header (counters + dyn words) | scene table | slot arrays | views
//   scratch:     z-buffer | visible lists | tile z | binned triangles | bin instances | survivors
struct Plan {
    uint32_t n_cap = 0, width = 0, height = 0, n_scenes = 0;
    LaunchCfg cfg;
    uint64_t list_cap = 1;           // visible pairs per list (worst case over the capacity)
    uint64_t item_cap = 0;           // (view, group) work items (worst case)
    uint32_t hiz_w = 0, hiz_h = 0, hiz_total = 0;
    size_t off_scenes = 0, off_slots = 0, off_views = 0, desc_bytes = 0;
    size_t z_off = 0, l_off = 0, h_off = 0, r_off = 0, i_off = 0, s_off = 0, scratch_bytes = 0, zbytes = 0;
};

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Header words of the descriptor buffer.
constexpr int kHdrVisCount = 0, kHdrWork = 4, kHdrBigRec = 8, kHdrBigInst = 12, kHdrDyn = 16, kHdrSurv = 24;

// max_meshlets / max_groups: per-view worst case (largest scene that may be rendered)
void make_plan(Plan &pl, uint32_t n_scenes, uint32_t n_cap, uint32_t width, uint32_t height,
               uint64_t list_entries, uint64_t items, const LaunchCfg &cfg)
{
    pl.n_cap = n_cap;
    pl.width = width;
    pl.height = height;
    pl.n_scenes = n_scenes;
    pl.cfg = cfg;
    pl.list_cap = std::max<uint64_t>(list_entries, 1);
    pl.item_cap = items;
    pl.hiz_w = (width + kHizTile - 1) / kHizTile;
    pl.hiz_h = (height + kHizTile - 1) / kHizTile;
    pl.hiz_total = hiz_pyramid_texels(pl.hiz_w, pl.hiz_h, nullptr);
    pl.off_scenes = 256;
    pl.off_slots = pl.off_scenes + al256(sizeof(SceneDev) * n_scenes);
    pl.off_views = pl.off_slots + al256(sizeof(uint32_t) * (3 * (size_t)n_scenes + 1));
    pl.desc_bytes = pl.off_views + sizeof(View) * (size_t)n_cap;
    pl.zbytes = al256((size_t)n_cap * width * height * sizeof(unsigned long long));
    pl.z_off = 0;
    pl.l_off = pl.z_off + pl.zbytes;
    pl.h_off = pl.l_off + al256(2 * (size_t)pl.list_cap * sizeof(uint4));
    pl.r_off = pl.h_off + al256((size_t)n_cap * pl.hiz_total * sizeof(uint32_t));
    pl.i_off = pl.r_off + al256((size_t)kBigRecCap * sizeof(BigTriStorage));
    pl.s_off = pl.i_off + al256(3 * (size_t)kBigInstCap * sizeof(uint2));
    pl.scratch_bytes = pl.s_off + al256((size_t)pl.list_cap * sizeof(uint4));
}

// Depth-noise request of one call: the public struct (or none) plus the
// offset of this call's agents within the caller's (a split call renders
// agents [agent_base, agent_base + n)).
struct NoiseReq {
    const hsr_depth_noise *noise = nullptr;
    uint32_t agent_base = 0;
};

// Step batches: each view names an agent-state slot and an action; the
// actuation pass on the device sets up its camera.
struct StepReq {
    const uint32_t *state = nullptr;
    const uint8_t *action = nullptr;
    uint64_t agents_dev = 0;         // device address of the AgentsDev
};

// View lists: explicit output frames and per-view output masks.
struct ViewsReq {
    const uint32_t *frames = nullptr;
    const uint32_t *outputs = nullptr;
};

// Unpacks a view list into per-view arrays (outputs 0 -> every present
// buffer), checking scene and frame ranges, that each requested output has a
// buffer, and that no output of a frame is written by two views.
int unpack_views(const hsr_view *views, uint32_t n, uint32_t n_scenes, uint32_t n_frames, uint32_t present,
                 std::vector<uint32_t> &soa, std::vector<hsr_pose> &poses, std::vector<uint32_t> &frames,
                 std::vector<uint32_t> &outs)
{
    if (!views || n == 0 || present == 0 || n_frames == 0) return HSR_ERR_INVALID_ARG;
    std::vector<uint8_t> used(n_frames, 0);
    soa.resize(n);
    poses.resize(n);
    frames.resize(n);
    outs.resize(n);
    for (uint32_t i = 0; i < n; i++) {
        const hsr_view &v = views[i];
        if (v.scene >= n_scenes || v.frame >= n_frames || (v.outputs & ~present)) return HSR_ERR_INVALID_ARG;
        const uint32_t o = v.outputs ? v.outputs : present;
        if (used[v.frame] & o) return HSR_ERR_INVALID_ARG;
        used[v.frame] |= (uint8_t)o;
        soa[i] = v.scene;
        poses[i] = v.pose;
        frames[i] = v.frame;
        outs[i] = o;
    }
    return HSR_OK;
}

uint32_t present_outputs(const void *rgb, const void *depth, const void *ids)
{
    return (rgb ? HSR_OUT_RGB : 0u) | (depth ? HSR_OUT_DEPTH : 0u) | (ids ? HSR_OUT_IDS : 0u);
}

bool noise_ok(const hsr_depth_noise *nz)
{
    return !nz || (std::isfinite(nz->depth_sigma) && nz->depth_sigma >= 0.f && nz->reserved == 0);
}

// Whether a call adds depth noise (then it shades with the noise variant).
bool noisy(const hsr_depth_noise *nz) { return nz && nz->depth_sigma > 0.f; }

// Camera setup of n views (a1) into the host staging buffer `hbuf`
// (pl.desc_bytes): views sorted by scene (stable), slot arrays, scene table,
// zeroed counters and the dynamic header words. frames[i] (or i) is the
// output frame of agent i; its depth-noise stream is keyed by
// noise.agent_ids[i], else by agent_base + its output frame.
// *guard (if given) is set when some view may snap a vertex beyond +-2^30
// sub-pixels (guard_free fails for its pose, or, for step batches whose poses
// live on the device, for a camera anywhere in its scene's box).
int fill_descriptors(const Plan &pl, const hsr_scene *const *scenes, const uint32_t *scene_of_agent,
                     const hsr_pose *poses, uint32_t n, const uint32_t *frames, const hsr_intrinsics &intr,
                     unsigned char *hbuf, const NoiseReq &nr = NoiseReq{}, const StepReq *step = nullptr,
                     const uint32_t *outputs = nullptr, bool *guard = nullptr)
{
    bool need_guard = false;
    if (n > pl.n_cap) return HSR_ERR_OVERFLOW;
    if (!noise_ok(nr.noise)) return HSR_ERR_INVALID_ARG;
    const uint32_t *agent_ids = nr.noise ? nr.noise->agent_ids : nullptr;
    std::vector<uint32_t> order(n);
    for (uint32_t i = 0; i < n; i++) {
        order[i] = i;
        if ((scene_of_agent ? scene_of_agent[i] : 0u) >= pl.n_scenes) return HSR_ERR_INVALID_ARG;
    }
    if (scene_of_agent)
        std::stable_sort(order.begin(), order.end(),
                         [&](uint32_t a, uint32_t b) { return scene_of_agent[a] < scene_of_agent[b]; });
    std::memset(hbuf, 0, pl.off_scenes);
    SceneDev *hs = reinterpret_cast<SceneDev *>(hbuf + pl.off_scenes);
    for (uint32_t i = 0; i < pl.n_scenes; i++) hs[i] = scenes[i]->dev;
    uint32_t *hslot = reinterpret_cast<uint32_t *>(hbuf + pl.off_slots);
    const uint32_t S = pl.n_scenes;
    std::memset(hslot, 0, sizeof(uint32_t) * (3 * (size_t)S + 1));
    uint32_t n_slots = 0;
    uint64_t items = 0, lists = 0;
    View *hv = reinterpret_cast<View *>(hbuf + pl.off_views);
    for (uint32_t k = 0; k < n; k++) {
        const uint32_t i = order[k];
        const uint32_t sidx = scene_of_agent ? scene_of_agent[i] : 0u;
        if (n_slots == 0 || hslot[2 * S + 1 + n_slots - 1] != sidx) {
            hslot[n_slots] = (uint32_t)items;             // slot_item_base
            hslot[S + 1 + n_slots] = k;                   // slot_view_base
            hslot[2 * S + 1 + n_slots] = sidx;            // slot_scene
            n_slots++;
        }
        items += scenes[sidx]->dev.n_groups;
        lists += scenes[sidx]->dev.n_meshlets;
        View &v = hv[k];
        std::memset(&v, 0, sizeof(View));
        const hsr_scene_info &box = scenes[sidx]->info;
        if (step) {
            v.state = step->state[i];
            v.action = step->action[i];
            // agents stay inside their scene's box: a camera at one corner
            // sees the farthest corner at the largest possible distance
            need_guard |= !guard_free(box.aabb_min, box.aabb_max, box.aabb_min, intr.fx, intr.fy, intr.cx, intr.cy,
                                      intr.znear);
        } else {
            if (!camera_matrix(poses[i], v.M)) return HSR_ERR_INVALID_ARG;
            view_planes(v.M, intr, pl.width, pl.height, v.planes);
            for (int c = 0; c < 3; c++) v.pos[c] = poses[i].pos[c];
            need_guard |= !guard_free(box.aabb_min, box.aabb_max, poses[i].pos, intr.fx, intr.fy, intr.cx, intr.cy,
                                      intr.znear);
        }
        v.scene = sidx;
        v.outputs = outputs ? outputs[i] : (uint32_t)(HSR_OUT_RGB | HSR_OUT_DEPTH | HSR_OUT_IDS);
        v.frame = frames ? frames[i] : i;
        v.agent = agent_ids ? agent_ids[i] : nr.agent_base + v.frame;
    }
    if (items > pl.item_cap || lists > pl.list_cap) return HSR_ERR_OVERFLOW;
    hslot[n_slots] = (uint32_t)items;                      // slot_item_base[n_slots]
    uint32_t *hdr = reinterpret_cast<uint32_t *>(hbuf);
    hdr[kHdrDyn + 0] = n;
    hdr[kHdrDyn + 1] = (uint32_t)items;
    hdr[kHdrDyn + 2] = n_slots;
    if (step) {
        hdr[kHdrDyn + 6] = (uint32_t)step->agents_dev;
        hdr[kHdrDyn + 7] = (uint32_t)(step->agents_dev >> 32);
    }
    if (nr.noise && nr.noise->depth_sigma > 0.f) {
        std::memcpy(&hdr[kHdrDyn + 3], &nr.noise->depth_sigma, sizeof(float));
        hdr[kHdrDyn + 4] = (uint32_t)nr.noise->seed;
        hdr[kHdrDyn + 5] = (uint32_t)(nr.noise->seed >> 32);
    }
    if (guard) *guard = need_guard;
    return HSR_OK;
}

// Kernel parameters for descriptors at `desc` and scratch at `scratch`.
Params make_params(const Plan &pl, unsigned char *desc, unsigned char *scratch, const hsr_intrinsics &intr,
                   uint8_t *rgb, float *depth, uint32_t *ids)
{
    Params p{};
    uint32_t *hdr = reinterpret_cast<uint32_t *>(desc);
    const uint32_t S = pl.n_scenes;
    const uint32_t *dslot = reinterpret_cast<const uint32_t *>(desc + pl.off_slots);
    p.vis_count = hdr + kHdrVisCount;
    p.work_counter = hdr + kHdrWork;
    p.big_rec_count = hdr + kHdrBigRec;
    p.big_inst_count = hdr + kHdrBigInst;
    p.dyn = hdr + kHdrDyn;
    p.scenes = reinterpret_cast<const SceneDev *>(desc + pl.off_scenes);
    p.views = reinterpret_cast<const View *>(desc + pl.off_views);
    p.slot_item_base = dslot;
    p.slot_view_base = dslot + S + 1;
    p.slot_scene = dslot + 2 * S + 1;
    p.n_slots = S;
    p.zbuf = reinterpret_cast<unsigned long long *>(scratch + pl.z_off);
    p.vis = reinterpret_cast<uint4 *>(scratch + pl.l_off);
    p.vis_cap = (uint32_t)pl.list_cap;
    p.hiz = reinterpret_cast<uint32_t *>(scratch + pl.h_off);
    p.hiz_total = pl.hiz_total;
    p.surv = reinterpret_cast<uint4 *>(scratch + pl.s_off);
    p.surv_count = hdr + kHdrSurv;
    p.fault_tx = debug_fault_tx();
    p.hiz_w = pl.hiz_w;
    p.hiz_h = pl.hiz_h;
    p.big_rec = reinterpret_cast<BigTri *>(scratch + pl.r_off);
    p.big_rec_cap = kBigRecCap;
    p.big_inst = reinterpret_cast<uint2 *>(scratch + pl.i_off);
    p.big_inst_cap = kBigInstCap;
    p.rgb = rgb;
    p.depth = depth;
    p.ids = ids;
    p.n_views = pl.n_cap;
    p.width = pl.width;
    p.height = pl.height;
    p.total_items = (uint32_t)std::min<uint64_t>(pl.item_cap, 0xFFFFFFF0ull);
    p.fx = intr.fx; p.fy = intr.fy; p.cx = intr.cx; p.cy = intr.cy;
    p.znear = intr.znear; p.zfar = intr.zfar;
    p.q_far = far_threshold(intr.zfar);
    p.inv_far = (float)(1.0 / (double)intr.zfar);
    p.gx = guard_g(intr.fx);
    p.gy = guard_g(intr.fy);
    const LaunchCfg &cfg = pl.cfg;
    p.small_px = std::min<uint32_t>(std::max<uint32_t>(cfg.small_px, 1), 32);
    p.bin_px = std::max(cfg.bin_px, p.small_px);
    p.chunk = std::min<uint32_t>(std::max<uint32_t>(cfg.chunk, 1), 32);
    p.n_phases = std::min<uint32_t>(std::max<uint32_t>(cfg.n_phases, 1u), 3u);
    p.phase_r2[0] = cfg.phase_r[0] * cfg.phase_r[0];
    p.phase_r2[1] = cfg.phase_r[1] * cfg.phase_r[1];
    p.stats = stage_stats_buffer();
    return p;
}

// Stream work of one render: upload descriptors, the actuation pass of a
// step batch, the kernels (guard: shading with the guard-band path; noise:
// shading with the depth-noise model).
cudaError_t enqueue_render(const Plan &pl, const Params &p, void *d_desc, const void *h_desc, cudaStream_t stream,
                           bool actuate, bool guard, bool noise)
{
    cudaError_t e = cudaMemcpyAsync(d_desc, h_desc, pl.desc_bytes, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return e;
    if (actuate) {
        e = launch_actuate(p, pl.n_cap, stream);
        if (e != cudaSuccess) return e;
    }
    return launch_render(p, pl.cfg, stream, guard, noise, false);
}

// Scenes, poses, intrinsics and size of a render; at least one output buffer
// (any of colour, depth, ids may be absent).
bool validate_common(const hsr_scene *const *scenes, uint32_t n_scenes, const hsr_pose *poses, uint32_t n,
                     const hsr_intrinsics *intr, uint32_t width, uint32_t height, bool has_output)
{
    if (!scenes || n_scenes == 0 || !poses || n == 0 || n >= kMaxViews || !has_output) return false;
    if (width == 0 || height == 0 || width > 4096 || height > 4096) return false;
    if (!intrinsics_ok(intr)) return false;
    for (uint32_t i = 0; i < n_scenes; i++)
        if (!scenes[i]) return false;
    return true;
}

// Shared body of hsr_render / hsr_render_batch: per-call scratch from the
// stream-ordered allocator, descriptors through thread-local pinned staging.
int render_views(const hsr_scene *const *scenes, uint32_t n_scenes, const uint32_t *scene_of_agent,
                 const hsr_pose *poses, uint32_t n, const hsr_intrinsics *intr, uint32_t width, uint32_t height,
                 uint8_t *rgb, float *depth, uint32_t *ids, void *stream_ptr, const LaunchCfg *cfg_in,
                 const NoiseReq &nr = NoiseReq{}, const ViewsReq &vr = ViewsReq{})
{
    if (!validate_common(scenes, n_scenes, poses, n, intr, width, height, rgb || depth || ids))
        return HSR_ERR_INVALID_ARG;
    if (!noise_ok(nr.noise)) return HSR_ERR_INVALID_ARG;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);

    // scratch: z-buffer (8 B / pixel / view) + visible and survivor lists
    // (48 B per meshlet per view) + tile-z pyramid; large calls are split into halves
    uint64_t list_entries = 0, items = 0;
    for (uint32_t i = 0; i < n; i++) {
        const uint32_t s = scene_of_agent ? scene_of_agent[i] : 0u;
        if (s >= n_scenes) return HSR_ERR_INVALID_ARG;
        list_entries += scenes[s]->dev.n_meshlets;
        items += scenes[s]->dev.n_groups;
    }
    const uint64_t hiz_w = (width + kHizTile - 1) / kHizTile, hiz_h = (height + kHizTile - 1) / kHizTile;
    const uint64_t scratch = (uint64_t)n * width * height * 8ull + list_entries * 48ull +
                             (uint64_t)n * hiz_pyramid_texels((uint32_t)hiz_w, (uint32_t)hiz_h, nullptr) * 4ull;
    if (scratch > kMaxScratchBytes && n > 1) {
        const uint32_t h = n / 2;
        const size_t px = (size_t)width * height;
        int st = render_views(scenes, n_scenes, scene_of_agent, poses, h, intr, width, height, rgb, depth, ids,
                              stream_ptr, cfg_in, nr, vr);
        if (st != HSR_OK) return st;
        hsr_depth_noise tail{};
        NoiseReq nr2 = nr;
        if (nr.noise && nr.noise->agent_ids) {
            tail = *nr.noise;
            tail.agent_ids += h;
            nr2.noise = &tail;
        }
        ViewsReq vr2;
        vr2.outputs = vr.outputs ? vr.outputs + h : nullptr;
        if (vr.frames) {
            // explicit frames index the whole output buffers
            vr2.frames = vr.frames + h;
            return render_views(scenes, n_scenes, scene_of_agent ? scene_of_agent + h : nullptr, poses + h, n - h,
                                intr, width, height, rgb, depth, ids, stream_ptr, cfg_in, nr2, vr2);
        }
        nr2.agent_base += h;
        return render_views(scenes, n_scenes, scene_of_agent ? scene_of_agent + h : nullptr, poses + h, n - h, intr,
                            width, height, rgb ? rgb + 3 * px * h : nullptr, depth ? depth + px * h : nullptr,
                            ids ? ids + px * h : nullptr, stream_ptr, cfg_in, nr2, vr2);
    }
    if (items >= 0xFFFFFFF0ull || list_entries >= 0xFFFFFFF0ull) return HSR_ERR_INVALID_ARG;

    LaunchCfg cfg;
    if (cfg_in)
        cfg = *cfg_in;
    else
        if (!lookup_tuned(make_key(scenes, n_scenes, n, width, height, ids != nullptr), cfg))
            cfg = default_launch_cfg(items, (uint64_t)n * width * height);
    Plan pl;
    make_plan(pl, n_scenes, n, width, height, list_entries, items, cfg);

    Staging &st = g_staging.slot[g_staging.next];
    g_staging.next = (g_staging.next + 1) % kStagingSlots;
    if (st.pending) {
        if (cudaEventSynchronize(st.done) != cudaSuccess) return HSR_ERR_CUDA;
        st.pending = false;
    }
    if (st.cap < pl.desc_bytes) {
        if (st.host) cudaFreeHost(st.host);
        st.host = nullptr;
        st.cap = 0;
        const size_t cap = std::max<size_t>(pl.desc_bytes, 64 * 1024);
        if (cudaHostAlloc(&st.host, cap, cudaHostAllocDefault) != cudaSuccess) return HSR_ERR_OOM;
        st.cap = cap;
    }
    if (!st.done && cudaEventCreateWithFlags(&st.done, cudaEventDisableTiming) != cudaSuccess) return HSR_ERR_CUDA;
    auto *hbuf = static_cast<unsigned char *>(st.host);
    bool guard = false;
    int status = fill_descriptors(pl, scenes, scene_of_agent, poses, n, vr.frames, *intr, hbuf, nr, nullptr,
                                  vr.outputs, &guard);
    if (status != HSR_OK) return status;

    // descriptors and scratch: the thread's reusable buffer, or stream-ordered
    // allocations for calls beyond its size
    const size_t desc_al = al256(pl.desc_bytes);
    void *dbuf = nullptr, *sbuf = nullptr;
    CallScratch &cs = g_call_scratch;
    const bool reuse = desc_al + pl.scratch_bytes <= kReuseBytes;
    cudaError_t e = cudaSuccess;
    if (reuse) {
        unsigned char *buf = cs.acquire(desc_al + pl.scratch_bytes, stream);
        if (!buf) return HSR_ERR_OOM;
        dbuf = buf;
        sbuf = buf + desc_al;
    } else {
        e = cudaMallocAsync(&dbuf, pl.desc_bytes, stream);
        if (e != cudaSuccess) return cuda_status(e);
        e = cudaMallocAsync(&sbuf, pl.scratch_bytes, stream);
        if (e != cudaSuccess) {
            cudaFreeAsync(dbuf, stream);
            return cuda_status(e);
        }
    }
    const Params p = make_params(pl, static_cast<unsigned char *>(dbuf), static_cast<unsigned char *>(sbuf), *intr,
                                 rgb, depth, ids);
    e = cudaMemcpyAsync(dbuf, hbuf, pl.desc_bytes, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaEventRecord(st.done, stream);
    if (e == cudaSuccess) st.pending = true;
    if (e == cudaSuccess) e = launch_render(p, pl.cfg, stream, guard, nr.noise && nr.noise->depth_sigma > 0.f, true);
    if (reuse) {
        if (!cs.release(stream) && e == cudaSuccess) e = cudaErrorUnknown;
        return e == cudaSuccess ? HSR_OK : cuda_status(e);
    }
    cudaError_t e1 = cudaFreeAsync(sbuf, stream);
    cudaError_t e2 = cudaFreeAsync(dbuf, stream);
    if (e != cudaSuccess) return cuda_status(e);
    if (e1 != cudaSuccess || e2 != cudaSuccess) return HSR_ERR_CUDA;
    return HSR_OK;
}

}  // namespace

struct hsr_batch {
    int device = 0;
    std::vector<const hsr_scene *> scenes;
    hsr_intrinsics intr{};
    uint8_t *rgb = nullptr;
    float *depth = nullptr;
    uint32_t *ids = nullptr;
    unsigned char *d_desc[2] = {nullptr, nullptr};
    unsigned char *h_desc[2] = {nullptr, nullptr};
    unsigned char *d_scratch = nullptr;
    // captured renders per descriptor buffer k, in eight variants: pose
    // renders (0) or step renders (2: upload, actuation, render), with the
    // guard-band shading (+1) and / or the depth-noise shading (+4); variant
    // 0 is captured at creation, the others on first use
    cudaGraph_t graph[8][2] = {};
    cudaGraphExec_t exec[8][2] = {};
    cudaEvent_t done[2] = {nullptr, nullptr};
    bool launched[2] = {false, false};
    int cur = 0;
    Plan plan;
    uint32_t n_frames = 0;
    std::mutex mu;
};

namespace {

// Release everything a batch holds (after synchronising its device).
void free_batch(hsr_batch *b)
{
    if (!b) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    for (int k = 0; k < 2; k++) {
        for (int v = 0; v < 8; v++) {
            if (b->exec[v][k]) cudaGraphExecDestroy(b->exec[v][k]);
            if (b->graph[v][k]) cudaGraphDestroy(b->graph[v][k]);
        }
        if (b->done[k]) cudaEventDestroy(b->done[k]);
        if (b->d_desc[k]) cudaFree(b->d_desc[k]);
        if (b->h_desc[k]) cudaFreeHost(b->h_desc[k]);
    }
    if (b->d_scratch) cudaFree(b->d_scratch);
    cudaSetDevice(prev);
    delete b;
}

}  // namespace

// Host helpers shared with other translation units of the library.
namespace hsr {
bool host_camera_matrix(const hsr_pose &pose, float M[12]) { return camera_matrix(pose, M); }
bool host_intrinsics_ok(const hsr_intrinsics *in) { return intrinsics_ok(in); }
float host_far_threshold(float zfar) { return far_threshold(zfar); }
void host_view_planes(const float M[12], const hsr_intrinsics &in, uint32_t W, uint32_t H, float planes[24])
{
    view_planes(M, in, W, H, planes);
}
float host_guard_g(float f) { return guard_g(f); }
bool host_guard_free(const hsr_scene *s, const hsr_pose &pose, const hsr_intrinsics &in)
{
    return guard_free(s->info.aabb_min, s->info.aabb_max, pose.pos, in.fx, in.fy, in.cx, in.cy, in.znear);
}
const SceneDev &host_scene_dev(const hsr_scene *s) { return s->dev; }
}  // namespace hsr

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
        // Order: by the class of the face normal (the six axis directions, or
        // one of 64 octahedral bins), then by the Morton code of the centroid,
        // so meshlets are compact and, where the geometry allows, planar (a
        // planar meshlet facing away is culled whole).
        std::vector<std::pair<uint64_t, uint32_t>> order(n_tris);
        double ext[3];
        for (int k = 0; k < 3; k++) ext[k] = std::max(1e-12, (double)bmax[k] - (double)bmin[k]);
        for (uint32_t t = 0; t < n_tris; t++) {
            uint64_t code = 0;
            double v[3][3];
            for (int j = 0; j < 3; j++)
                for (int k = 0; k < 3; k++) v[j][k] = (double)xyz[3 * (size_t)canon[3 * (size_t)t + j] + k];
            for (int k = 0; k < 3; k++) {
                const double c = (v[0][k] + v[1][k] + v[2][k]) / 3.0;
                double f = (c - bmin[k]) / ext[k];
                f = std::min(std::max(f, 0.0), 1.0);
                code |= spread21((uint64_t)(f * 524287.0)) << k;           // 19 bits per axis
            }
            double n[3] = {(v[1][1] - v[0][1]) * (v[2][2] - v[0][2]) - (v[1][2] - v[0][2]) * (v[2][1] - v[0][1]),
                           (v[1][2] - v[0][2]) * (v[2][0] - v[0][0]) - (v[1][0] - v[0][0]) * (v[2][2] - v[0][2]),
                           (v[1][0] - v[0][0]) * (v[2][1] - v[0][1]) - (v[1][1] - v[0][1]) * (v[2][0] - v[0][0])};
            const double nl = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            uint64_t cls = 127;
            if (nl > 0) {
                for (double &x : n) x /= nl;
                int ax = 0;
                for (int k = 1; k < 3; k++)
                    if (std::fabs(n[k]) > std::fabs(n[ax])) ax = k;
                if (std::fabs(n[ax]) > 0.999) {
                    cls = (uint64_t)(2 * ax + (n[ax] < 0 ? 1 : 0));
                } else {
                    const double l1 = std::fabs(n[0]) + std::fabs(n[1]) + std::fabs(n[2]);
                    double ox = n[0] / l1, oy = n[1] / l1;
                    if (n[2] < 0) {
                        const double tx = (1 - std::fabs(oy)) * (ox < 0 ? -1 : 1);
                        const double ty = (1 - std::fabs(ox)) * (oy < 0 ? -1 : 1);
                        ox = tx;
                        oy = ty;
                    }
                    const int ix = std::min(7, std::max(0, (int)((ox + 1) * 4)));
                    const int iy = std::min(7, std::max(0, (int)((oy + 1) * 4)));
                    cls = (uint64_t)(6 + 8 * ix + iy);
                }
            }
            order[t] = {(cls << 57) | code, t};
        }
        std::sort(order.begin(), order.end());
        // greedy meshlets: <= 32 triangles, <= 64 distinct vertices
        std::vector<Meshlet> meshlets;
        std::vector<float4> mvert;
        std::vector<uint2> mtri;
        std::vector<float4> mplane;
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
            // the meshlet's common plane (when its triangles share one), for
            // culling meshlets that face away as a whole
            {
                double nsum[3] = {0, 0, 0}, amin = 1e300, lmax = 0;
                bool ok = true;
                auto P = [&](uint32_t v, int k) { return (double)xyz[3 * (size_t)v + k]; };
                for (uint32_t t : cur_t) {
                    const uint32_t a = canon[3 * (size_t)t], b = canon[3 * (size_t)t + 1], c = canon[3 * (size_t)t + 2];
                    double e1[3], e2[3], e3[3];
                    for (int k = 0; k < 3; k++) {
                        e1[k] = P(b, k) - P(a, k);
                        e2[k] = P(c, k) - P(a, k);
                        e3[k] = P(c, k) - P(b, k);
                    }
                    const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                                         e1[0] * e2[1] - e1[1] * e2[0]};
                    const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
                    if (!(len > 0)) ok = false;
                    for (int k = 0; k < 3; k++) nsum[k] += n[k];
                    amin = std::min(amin, 0.5 * len);
                    lmax = std::max({lmax, std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]),
                                     std::sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]),
                                     std::sqrt(e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2])});
                }
                const double nl = std::sqrt(nsum[0] * nsum[0] + nsum[1] * nsum[1] + nsum[2] * nsum[2]);
                double nh[3] = {0, 0, 0}, w = 0, eps = 0, rho = 0;
                if (ok && nl > 0) {
                    for (int k = 0; k < 3; k++) nh[k] = nsum[k] / nl;
                    const uint32_t a0 = canon[3 * (size_t)cur_t[0]];
                    w = nh[0] * P(a0, 0) + nh[1] * P(a0, 1) + nh[2] * P(a0, 2);
                    for (uint32_t v : cur_v)
                        eps = std::max(eps, std::fabs(nh[0] * P(v, 0) + nh[1] * P(v, 1) + nh[2] * P(v, 2) - w));
                    for (uint32_t t : cur_t) {
                        const uint32_t a = canon[3 * (size_t)t], b = canon[3 * (size_t)t + 1], c = canon[3 * (size_t)t + 2];
                        double e1[3], e2[3];
                        for (int k = 0; k < 3; k++) {
                            e1[k] = P(b, k) - P(a, k);
                            e2[k] = P(c, k) - P(a, k);
                        }
                        const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                                             e1[0] * e2[1] - e1[1] * e2[0]};
                        const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
                        double d2 = 0;
                        for (int k = 0; k < 3; k++) d2 += (n[k] / len - nh[k]) * (n[k] / len - nh[k]);
                        rho = std::max(rho, std::sqrt(d2));
                    }
                } else {
                    ok = false;
                }
                if (!(rho < 0.01)) ok = false;
                // rounded outwards: area down, the slack terms up
                mplane.push_back(make_float4((float)nh[0], (float)nh[1], (float)nh[2], (float)w));
                mplane.push_back(make_float4(ok ? (float)(amin * (1 - 1e-6)) : 0.f,
                                             ok ? (float)(lmax * (1 + 1e-6)) : -1.f, (float)(eps * 1.01 + 1e-9),
                                             (float)(rho * 1.01 + 1e-9)));
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
        if (n_meshlets > kMaxMeshlets) throw std::bad_alloc();
        Meshlet sentinel{};
        sentinel.vbase = (uint32_t)mvert.size();
        sentinel.tbase = (uint32_t)mtri.size();
        meshlets.push_back(sentinel);
        // two spare entries: triangle blocks are copied in 16-byte units that
        // may run one entry past a meshlet's last triangle
        mtri.push_back(make_uint2(0u, 0u));
        mtri.push_back(make_uint2(0u, 0u));
        // groups of 32 meshlets: group g is meshlets [32 g, min(32 g + 32, n)),
        // which the culling kernel computes without reading the group record
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
        // per-triangle shading records (one 64-byte line: the shading pass
        // reaches a pixel's vertices and attributes with one dependent load)
        std::vector<float4> srec(4 * (size_t)n_tris);
        {
            const bool textured = uv && atlas, coloured = !textured && vert_rgb;
            auto bits = [](uint32_t u) {
                float f;
                std::memcpy(&f, &u, 4);
                return f;
            };
            auto rgb = [&](uint32_t i) {
                return bits((uint32_t)vert_rgb[3 * (size_t)i] | ((uint32_t)vert_rgb[3 * (size_t)i + 1] << 8) |
                            ((uint32_t)vert_rgb[3 * (size_t)i + 2] << 16));
            };
            for (size_t t = 0; t < n_tris; t++) {
                const uint32_t a = tri[t].x, b = tri[t].y, c = tri[t].z;
                const float *pa = xyz + 3 * (size_t)a, *pb = xyz + 3 * (size_t)b, *pc = xyz + 3 * (size_t)c;
                float4 *r = &srec[4 * t];
                r[0] = make_float4(pa[0], pa[1], pa[2], pb[0]);
                r[1] = make_float4(pb[1], pb[2], pc[0], pc[1]);
                if (textured) {
                    r[2] = make_float4(pc[2], uv[2 * (size_t)a], uv[2 * (size_t)a + 1], uv[2 * (size_t)b]);
                    r[3] = make_float4(uv[2 * (size_t)b + 1], uv[2 * (size_t)c], uv[2 * (size_t)c + 1], bits(tri[t].w));
                } else if (coloured) {
                    r[2] = make_float4(pc[2], rgb(a), rgb(b), rgb(c));
                    r[3] = make_float4(0.f, 0.f, 0.f, bits(tri[t].w));
                } else {
                    r[2] = make_float4(pc[2], 0.f, 0.f, 0.f);
                    r[3] = make_float4(0.f, 0.f, 0.f, bits(tri[t].w));
                }
            }
        }

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
        const float4 *dmp;
        if ((e = upload(s, mplane.data(), mplane.size(), &dmp)) != cudaSuccess) throw e;
        d.mplane = dmp;
        float cmax = 0.f;
        for (size_t i = 0; i < 3 * (size_t)n_verts; i++) cmax = std::max(cmax, std::fabs(xyz[i]));
        d.coord_max = cmax;
        if ((e = upload(s, tri.data(), tri.size(), &dt)) != cudaSuccess) throw e;
        if ((e = upload(s, vert.data(), vert.size(), &dv)) != cudaSuccess) throw e;
        const float4 *dsr;
        if ((e = upload(s, srec.data(), srec.size(), &dsr)) != cudaSuccess) throw e;
        d.srec = dsr;
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
            // the same texels in a texture (the driver's 2D-local layout), one
            // 32-bit channel per texel: the bilinear footprint's four packed
            // texels come back from one gather; a scene whose atlas does not
            // fit a texture samples the linear copy
            d.atlas_tex = 0;
            const cudaChannelFormatDesc cd = cudaCreateChannelDesc<unsigned int>();
            if (cudaMallocArray(&s->atlas_array, &cd, atlas_w, atlas_h) == cudaSuccess) {
                cudaResourceDesc rd{};
                rd.resType = cudaResourceTypeArray;
                rd.res.array.array = s->atlas_array;
                cudaTextureDesc td{};
                td.addressMode[0] = cudaAddressModeClamp;
                td.addressMode[1] = cudaAddressModeClamp;
                td.filterMode = cudaFilterModePoint;
                td.readMode = cudaReadModeElementType;
                td.normalizedCoords = 0;
                if (cudaMemcpy2DToArray(s->atlas_array, 0, 0, atlas, (size_t)atlas_w * 4, (size_t)atlas_w * 4, atlas_h,
                                        cudaMemcpyHostToDevice) == cudaSuccess &&
                    cudaCreateTextureObject(&s->atlas_tex, &rd, &td, nullptr) == cudaSuccess) {
                    d.atlas_tex = s->atlas_tex;
                    s->info.device_bytes += (uint64_t)atlas_w * atlas_h * 4;
                } else {
                    s->atlas_tex = 0;
                }
            } else {
                s->atlas_array = nullptr;
            }
            (void)cudaGetLastError();   // a failed texture leaves no sticky error: the linear path serves
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

}  // extern "C"

namespace hsr {
// Batch with view capacity n_cap writing into output frames [0, n_frames).
int batch_create(const hsr_scene *const *scenes, uint32_t n_scenes, uint32_t n_cap, uint32_t n_frames,
                 const hsr_intrinsics *intr, uint32_t width, uint32_t height, uint8_t *rgb, float *depth,
                 uint32_t *ids, const hsr_config *cfg, hsr_batch **out)
{
    if (!out) return HSR_ERR_INVALID_ARG;
    if (n_frames < n_cap) return HSR_ERR_INVALID_ARG;
    *out = nullptr;
    hsr_pose dummy{};
    if (!validate_common(scenes, n_scenes, &dummy, n_cap, intr, width, height, rgb || depth || ids))
        return HSR_ERR_INVALID_ARG;
    uint64_t max_m = 0, max_g = 0;
    for (uint32_t i = 0; i < n_scenes; i++) {
        max_m = std::max<uint64_t>(max_m, scenes[i]->dev.n_meshlets);
        max_g = std::max<uint64_t>(max_g, scenes[i]->dev.n_groups);
    }
    const uint64_t list_entries = (uint64_t)n_cap * max_m, items = (uint64_t)n_cap * max_g;
    if (items >= 0xFFFFFFF0ull || list_entries >= 0xFFFFFFF0ull) return HSR_ERR_INVALID_ARG;
    LaunchCfg lc;
    if (cfg)
        lc = from_config(*cfg);
    else
        if (!lookup_tuned(make_key(scenes, n_scenes, n_cap, width, height, ids != nullptr), lc))
            lc = default_launch_cfg(items, (uint64_t)n_cap * width * height);
    hsr_batch *b = new (std::nothrow) hsr_batch();
    if (!b) return HSR_ERR_OOM;
    cudaGetDevice(&b->device);
    b->scenes.assign(scenes, scenes + n_scenes);
    b->intr = *intr;
    b->rgb = rgb;
    b->depth = depth;
    b->ids = ids;
    Plan pl;
    make_plan(pl, n_scenes, n_cap, width, height, list_entries, items, lc);
    cudaError_t e = cudaSuccess;
    cudaStream_t cs = nullptr;
    auto fail = [&](cudaError_t err) {
        if (cs) cudaStreamDestroy(cs);
        free_batch(b);
        return cuda_status(err);
    };
    if ((e = cudaMalloc(&b->d_scratch, pl.scratch_bytes)) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(b->d_scratch + pl.z_off, 0xFF, pl.zbytes)) != cudaSuccess) return fail(e);
    if ((e = prepare_kernels()) != cudaSuccess) return fail(e);
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
    for (int k = 0; k < 2; k++) {
        if ((e = cudaMalloc(&b->d_desc[k], pl.desc_bytes)) != cudaSuccess) return fail(e);
        if ((e = cudaHostAlloc(&b->h_desc[k], pl.desc_bytes, cudaHostAllocDefault)) != cudaSuccess) return fail(e);
        std::memset(b->h_desc[k], 0, pl.desc_bytes);
        if ((e = cudaEventCreateWithFlags(&b->done[k], cudaEventDisableTiming)) != cudaSuccess) return fail(e);
        const Params p = make_params(pl, b->d_desc[k], b->d_scratch, *intr, rgb, depth, ids);
        if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return fail(e);
        cudaError_t er = enqueue_render(pl, p, b->d_desc[k], b->h_desc[k], cs, false, false, false);
        e = cudaStreamEndCapture(cs, &b->graph[0][k]);
        if (er != cudaSuccess) return fail(er);
        if (e != cudaSuccess) return fail(e);
        if ((e = cudaGraphInstantiate(&b->exec[0][k], b->graph[0][k], 0)) != cudaSuccess) return fail(e);
    }
    cudaStreamDestroy(cs);
    cs = nullptr;
    b->plan = pl;
    b->n_frames = n_frames;
    *out = b;
    return HSR_OK;
}

// Graph variant v (0: pose render, 2: step render, +1: guard-band shading,
// +4: depth-noise shading) of descriptor buffer k, captured on first use.
// Called with the batch's lock.
int batch_exec(hsr_batch *b, int v, int k, cudaGraphExec_t *out)
{
    if (!b->exec[v][k]) {
        cudaStream_t cs = nullptr;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return HSR_ERR_CUDA;
        const Plan &pl = b->plan;
        const Params p = make_params(pl, b->d_desc[k], b->d_scratch, b->intr, b->rgb, b->depth, b->ids);
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t er = enqueue_render(pl, p, b->d_desc[k], b->h_desc[k], cs, (v & 2) != 0, (v & 1) != 0,
                                            (v & 4) != 0);
            e = cudaStreamEndCapture(cs, &b->graph[v][k]);
            if (er != cudaSuccess) e = er;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[v][k], b->graph[v][k], 0);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            if (b->graph[v][k]) cudaGraphDestroy(b->graph[v][k]);
            b->graph[v][k] = nullptr;
            b->exec[v][k] = nullptr;
            return cuda_status(e);
        }
    }
    *out = b->exec[v][k];
    return HSR_OK;
}
}  // namespace hsr

extern "C" {

int hsr_batch_create(const hsr_scene *const *scenes, uint32_t n_scenes, uint32_t n_cap,
                     const hsr_intrinsics *intr, uint32_t width, uint32_t height, uint8_t *rgb, float *depth,
                     uint32_t *ids, const hsr_config *cfg, hsr_batch **out)
{
    return batch_create(scenes, n_scenes, n_cap, n_cap, intr, width, height, rgb, depth, ids, cfg, out);
}

int hsr_batch_render(hsr_batch *b, const uint32_t *scene_of_agent, const hsr_pose *poses, uint32_t n,
                     const uint32_t *frames, void *cuda_stream)
{
    return hsr_batch_render_noisy(b, scene_of_agent, poses, n, frames, nullptr, cuda_stream);
}


int hsr_batch_render_noisy(hsr_batch *b, const uint32_t *scene_of_agent, const hsr_pose *poses, uint32_t n,
                           const uint32_t *frames, const hsr_depth_noise *noise, void *cuda_stream)
{
    if (!b || !poses || n == 0 || !noise_ok(noise)) return HSR_ERR_INVALID_ARG;
    const Plan &pl = b->plan;
    if (n > pl.n_cap) return HSR_ERR_OVERFLOW;
    if (frames)
        for (uint32_t i = 0; i < n; i++)
            if (frames[i] >= b->n_frames) return HSR_ERR_INVALID_ARG;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    std::lock_guard<std::mutex> lock(b->mu);
    const int k = b->cur;
    if (b->launched[k] && cudaEventSynchronize(b->done[k]) != cudaSuccess) return HSR_ERR_CUDA;
    NoiseReq nr;
    nr.noise = noise;
    bool guard = false;
    int st = fill_descriptors(pl, b->scenes.data(), scene_of_agent, poses, n, frames, b->intr, b->h_desc[k], nr,
                              nullptr, nullptr, &guard);
    if (st != HSR_OK) return st;
    cudaGraphExec_t ex = nullptr;
    if ((st = batch_exec(b, (guard ? 1 : 0) | (noisy(noise) ? 4 : 0), k, &ex)) != HSR_OK) return st;
    if (cudaGraphLaunch(ex, stream) != cudaSuccess) return HSR_ERR_CUDA;
    if (cudaEventRecord(b->done[k], stream) != cudaSuccess) return HSR_ERR_CUDA;
    b->launched[k] = true;
    b->cur ^= 1;
    return HSR_OK;
}

int hsr_batch_render_host(hsr_batch *b, const uint32_t *scene_of_agent, const hsr_pose *poses, uint32_t n,
                          uint8_t *host_rgb, float *host_depth, uint32_t *host_ids, void *cuda_stream,
                          uint64_t *h2d_bytes)
{
    if (!b || (host_rgb && !b->rgb) || (host_depth && !b->depth) || (host_ids && !b->ids))
        return HSR_ERR_INVALID_ARG;
    const int st = hsr_batch_render_noisy(b, scene_of_agent, poses, n, nullptr, nullptr, cuda_stream);
    if (st != HSR_OK) return st;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    const size_t px = (size_t)n * b->plan.width * b->plan.height;
    if (host_rgb && cudaMemcpyAsync(host_rgb, b->rgb, 3 * px, cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return HSR_ERR_CUDA;
    if (host_depth &&
        cudaMemcpyAsync(host_depth, b->depth, sizeof(float) * px, cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return HSR_ERR_CUDA;
    if (host_ids &&
        cudaMemcpyAsync(host_ids, b->ids, sizeof(uint32_t) * px, cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return HSR_ERR_CUDA;
    if (h2d_bytes) *h2d_bytes = b->plan.desc_bytes;
    return HSR_OK;
}

int hsr_batch_step(hsr_batch *b, hsr_agents *agents, const uint32_t *agent_idx, const uint8_t *actions, uint32_t n,
                   const uint32_t *frames, const hsr_depth_noise *noise, void *cuda_stream)
{
    AgentsView av{};
    if (!b || !agent_idx || !actions || n == 0 || !noise_ok(noise) || !agents_view(agents, av))
        return HSR_ERR_INVALID_ARG;
    const Plan &pl = b->plan;
    if (n > pl.n_cap) return HSR_ERR_OVERFLOW;
    if (av.device != b->device || av.n_scenes != b->scenes.size()) return HSR_ERR_INVALID_ARG;
    for (uint32_t s = 0; s < av.n_scenes; s++)
        if (av.scenes[s] != b->scenes[s]) return HSR_ERR_INVALID_ARG;
    std::vector<uint32_t> soa(n), sorted(agent_idx, agent_idx + n);
    for (uint32_t i = 0; i < n; i++) {
        if (agent_idx[i] >= av.n_agents || actions[i] > HSR_ACTION_TURN_RIGHT) return HSR_ERR_INVALID_ARG;
        if (frames && frames[i] >= b->n_frames) return HSR_ERR_INVALID_ARG;
        soa[i] = av.scene_of_agent[agent_idx[i]];
    }
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return HSR_ERR_INVALID_ARG;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    std::lock_guard<std::mutex> lock(b->mu);
    const int k = b->cur;
    if (b->launched[k] && cudaEventSynchronize(b->done[k]) != cudaSuccess) return HSR_ERR_CUDA;
    NoiseReq nr;
    nr.noise = noise;
    StepReq sr;
    sr.state = agent_idx;
    sr.action = actions;
    sr.agents_dev = (uint64_t)(uintptr_t)av.dev;
    bool guard = false;
    int st = fill_descriptors(pl, b->scenes.data(), soa.data(), nullptr, n, frames, b->intr, b->h_desc[k], nr, &sr,
                              nullptr, &guard);
    if (st != HSR_OK) return st;
    cudaGraphExec_t ex = nullptr;
    if ((st = batch_exec(b, 2 | (guard ? 1 : 0) | (noisy(noise) ? 4 : 0), k, &ex)) != HSR_OK) return st;
    if (cudaGraphLaunch(ex, stream) != cudaSuccess) return HSR_ERR_CUDA;
    if (cudaEventRecord(b->done[k], stream) != cudaSuccess) return HSR_ERR_CUDA;
    b->launched[k] = true;
    b->cur ^= 1;
    return HSR_OK;
}

int hsr_batch_render_views(hsr_batch *b, const hsr_view *views, uint32_t n, const hsr_depth_noise *noise,
                           void *cuda_stream)
{
    if (!b || !noise_ok(noise)) return HSR_ERR_INVALID_ARG;
    const Plan &pl = b->plan;
    if (n > pl.n_cap) return HSR_ERR_OVERFLOW;
    std::vector<uint32_t> soa, frames, outs;
    std::vector<hsr_pose> poses;
    int st = unpack_views(views, n, (uint32_t)b->scenes.size(), b->n_frames, present_outputs(b->rgb, b->depth, b->ids),
                          soa, poses, frames, outs);
    if (st != HSR_OK) return st;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    std::lock_guard<std::mutex> lock(b->mu);
    const int k = b->cur;
    if (b->launched[k] && cudaEventSynchronize(b->done[k]) != cudaSuccess) return HSR_ERR_CUDA;
    NoiseReq nr;
    nr.noise = noise;
    bool guard = false;
    st = fill_descriptors(pl, b->scenes.data(), soa.data(), poses.data(), n, frames.data(), b->intr, b->h_desc[k], nr,
                          nullptr, outs.data(), &guard);
    if (st != HSR_OK) return st;
    cudaGraphExec_t ex = nullptr;
    if ((st = batch_exec(b, (guard ? 1 : 0) | (noisy(noise) ? 4 : 0), k, &ex)) != HSR_OK) return st;
    if (cudaGraphLaunch(ex, stream) != cudaSuccess) return HSR_ERR_CUDA;
    if (cudaEventRecord(b->done[k], stream) != cudaSuccess) return HSR_ERR_CUDA;
    b->launched[k] = true;
    b->cur ^= 1;
    return HSR_OK;
}

int hsr_batch_destroy(hsr_batch *b)
{
    free_batch(b);
    return HSR_OK;
}

int hsr_config_default(hsr_config *cfg)
{
    if (!cfg) return HSR_ERR_INVALID_ARG;
    *cfg = to_config(LaunchCfg{});
    return HSR_OK;
}

int hsr_set_tuned_config(const hsr_scene *const *scenes, uint32_t n_scenes, uint32_t n, uint32_t width,
                         uint32_t height, int with_ids, const hsr_config *cfg)
{
    if (!scenes || n_scenes == 0) return HSR_ERR_INVALID_ARG;
    const TuneKey k = make_key(scenes, n_scenes, n, width, height, with_ids);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (cfg)
        g_tuned[k] = from_config(*cfg);
    else
        g_tuned.erase(k);
    return HSR_OK;
}

int hsr_autotune(const hsr_scene *const *scenes, uint32_t n_scenes, const uint32_t *scene_of_agent,
                 const hsr_pose *poses, uint32_t n, const hsr_intrinsics *intr, uint32_t width, uint32_t height,
                 uint8_t *rgb, float *depth, uint32_t *ids, void *cuda_stream, uint32_t reps, hsr_config *best,
                 float *best_ms)
{
    if (!scenes || n_scenes == 0 || (n_scenes > 1 && !scene_of_agent)) return HSR_ERR_INVALID_ARG;
    reps = std::max<uint32_t>(1, std::min<uint32_t>(reps, 50));
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return HSR_ERR_CUDA;
    }
    int status = HSR_OK;
    // Each candidate is timed as a batch replays it: captured into a graph,
    // launched after a write of more than the L2 size (so that its geometry
    // and texels come from HBM, and the host has enqueued the graph before
    // the device reaches it), device time between events around the launch.
    const size_t flush_bytes = 256ull << 20;
    void *flush = nullptr;
    if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return HSR_ERR_OOM;
    }
    auto measure = [&](const LaunchCfg &c, float &ms) -> int {
        const hsr_config hc = to_config(c);
        hsr_batch *b = nullptr;
        int st = batch_create(scenes, n_scenes, n, n, intr, width, height, rgb, depth, ids, &hc, &b);
        if (st != HSR_OK) return st;
        std::vector<float> t;
        st = hsr_batch_render(b, scene_of_agent, poses, n, nullptr, cuda_stream);
        for (uint32_t r = 0; r < reps && st == HSR_OK; r++) {
            if (cudaMemsetAsync(flush, r & 1, flush_bytes, stream) != cudaSuccess ||
                cudaEventRecord(e0, stream) != cudaSuccess) {
                st = HSR_ERR_CUDA;
                break;
            }
            st = hsr_batch_render(b, scene_of_agent, poses, n, nullptr, cuda_stream);
            if (st != HSR_OK) break;
            if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                st = HSR_ERR_CUDA;
                break;
            }
            float x = 0;
            cudaEventElapsedTime(&x, e0, e1);
            t.push_back(x);
        }
        free_batch(b);
        if (st != HSR_OK) return st;
        std::sort(t.begin(), t.end());
        ms = t[t.size() / 2];
        return HSR_OK;
    };
    // coordinate descent over the launch parameters from the default, two sweeps
    uint64_t max_g = 0;
    for (uint32_t i = 0; i < n_scenes; i++) max_g = std::max<uint64_t>(max_g, scenes[i]->dev.n_groups);
    LaunchCfg cur = default_launch_cfg((uint64_t)n * max_g, (uint64_t)n * width * height);
    float cur_ms = 0;
    status = measure(cur, cur_ms);
    const uint32_t small_v[] = {8, 16, 24, 32};
    const uint32_t bin_v[] = {16, 32, 64, 128, 256, 512, 4096};
    const uint32_t chunk_v[] = {1, 2, 4, 8, 16, 32};
    // occlusion phases and their radii are searched together: one phase, or
    // two or three with each pair of band radii (the best radii depend on
    // the number of phases)
    const float radius_v[][2] = {{2.f, 5.f}, {3.f, 7.f}, {4.f, 10.f}, {6.f, 14.f}};
    const uint32_t cta_v[] = {2, 3};
    for (int sweep = 0; sweep < 2 && status == HSR_OK; sweep++) {
        for (int param = 0; param < 5 && status == HSR_OK; param++) {
            const int nv = param == 0 ? 4 : param == 1 ? 7 : param == 2 ? 6 : param == 3 ? 9 : 2;
            for (int k = 0; k < nv && status == HSR_OK; k++) {
                LaunchCfg c = cur;
                switch (param) {
                    case 0: c.small_px = small_v[k]; break;
                    case 1: c.bin_px = bin_v[k]; break;
                    case 2: c.chunk = chunk_v[k]; break;
                    case 3:
                        c.n_phases = k == 0 ? 1u : (k <= 4 ? 2u : 3u);
                        if (k > 0) {
                            c.phase_r[0] = radius_v[(k - 1) % 4][0];
                            c.phase_r[1] = radius_v[(k - 1) % 4][1];
                        }
                        break;
                    default: c.raster_ctas_per_sm = cta_v[k]; break;
                }
                c.bin_px = std::max(c.bin_px, c.small_px);
                float ms = 0;
                status = measure(c, ms);
                if (status == HSR_OK && ms < cur_ms) {
                    cur = c;
                    cur_ms = ms;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(flush);
    if (status != HSR_OK) return status;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tuned[make_key(scenes, n_scenes, n, width, height, ids != nullptr)] = cur;
    }
    if (best) *best = to_config(cur);
    if (best_ms) *best_ms = cur_ms;
    return HSR_OK;
}

int hsr_set_stage_timing(int enable)
{
    return stage_timing_enable(enable != 0) == cudaSuccess ? HSR_OK : HSR_ERR_CUDA;
}

int hsr_get_stage_timing(float *ms)
{
    if (!ms) return HSR_ERR_INVALID_ARG;
    const cudaError_t e = stage_timing_read(ms);
    if (e == cudaErrorNotReady) return HSR_ERR_INVALID_ARG;
    return e == cudaSuccess ? HSR_OK : HSR_ERR_CUDA;
}

int hsr_set_stage_stats(int enable)
{
    return stage_stats_enable(enable != 0) == cudaSuccess ? HSR_OK : HSR_ERR_CUDA;
}

int hsr_get_stage_stats(uint32_t *counts)
{
    if (!counts) return HSR_ERR_INVALID_ARG;
    const cudaError_t e = stage_stats_read(counts);
    if (e == cudaErrorNotReady) return HSR_ERR_INVALID_ARG;
    return e == cudaSuccess ? HSR_OK : HSR_ERR_CUDA;
}

int hsr_scene_set_sampling(hsr_scene *s, int mode)
{
    if (!s || (mode != HSR_SAMPLE_BILINEAR && mode != HSR_SAMPLE_TRILINEAR)) return HSR_ERR_INVALID_ARG;
    SceneDev &d = s->dev;
    if (mode == HSR_SAMPLE_TRILINEAR && d.color_mode != kColorTexture) return HSR_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    cudaError_t e = cudaSuccess;
    if (mode == HSR_SAMPLE_TRILINEAR && d.n_levels == 0) {
        // level sizes and offsets: halve (at least 1) down to 1 x 1
        uint32_t w = d.atlas_w, h = d.atlas_h, n = 1;
        uint32_t off[16] = {0};
        uint64_t total = 0;
        while ((w > 1 || h > 1) && n < 16) {
            w = w > 1 ? w >> 1 : 1;
            h = h > 1 ? h >> 1 : 1;
            off[n] = (uint32_t)total;
            total += (uint64_t)w * h;
            n++;
        }
        uint32_t *mips = nullptr;
        if (total) {
            e = cudaMalloc(&mips, total * sizeof(uint32_t));
            if (e == cudaSuccess) s->allocs.push_back(mips);
            uint32_t pw = d.atlas_w, ph = d.atlas_h;
            for (uint32_t l = 1; l < n && e == cudaSuccess; l++) {
                const uint32_t lw = pw > 1 ? pw >> 1 : 1, lh = ph > 1 ? ph >> 1 : 1;
                const uint32_t *src = l == 1 ? d.atlas : mips + off[l - 1];
                e = launch_mip_down(src, pw, ph, mips + off[l], lw, lh, nullptr);
                pw = lw;
                ph = lh;
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
        }
        if (e == cudaSuccess) {
            d.mips = mips;
            d.n_levels = n;
            for (int l = 0; l < 16; l++) d.mip_off[l] = off[l];
        }
    }
    if (e == cudaSuccess) {
        d.sample_mode = (uint32_t)mode;
        e = cudaMemcpy(s->dev_desc, &d, sizeof(SceneDev), cudaMemcpyHostToDevice);
    }
    cudaSetDevice(prev);
    return e == cudaSuccess ? HSR_OK : cuda_status(e);
}

int hsr_device_status(int clear)
{
    uint32_t flags = 0;
    if (read_device_errors(&flags, clear != 0) != cudaSuccess) return HSR_ERR_CUDA;
    if (flags & kErrWaitTimeout) return HSR_ERR_TIMEOUT;
    return (flags & kErrRange) ? HSR_ERR_OVERFLOW : HSR_OK;
}

int hsr_debug_inject_wait_fault(uint32_t extra_bytes)
{
    set_debug_fault_tx(extra_bytes);
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

int hsr_render_views(const hsr_scene *const *scenes, uint32_t n_scenes, const hsr_view *views, uint32_t n,
                     uint32_t n_frames, const hsr_intrinsics *intr, uint32_t width, uint32_t height, uint8_t *rgb,
                     float *depth, uint32_t *ids, const hsr_depth_noise *noise, void *cuda_stream)
{
    std::vector<uint32_t> soa, frames, outs;
    std::vector<hsr_pose> poses;
    const int st = unpack_views(views, n, n_scenes, n_frames, present_outputs(rgb, depth, ids), soa, poses, frames,
                                outs);
    if (st != HSR_OK) return st;
    NoiseReq nr;
    nr.noise = noise;
    ViewsReq vr;
    vr.frames = frames.data();
    vr.outputs = outs.data();
    return render_views(scenes, n_scenes, soa.data(), poses.data(), n, intr, width, height, rgb, depth, ids,
                        cuda_stream, nullptr, nr, vr);
}

int hsr_render_noisy(const hsr_scene *const *scenes, uint32_t n_scenes, const uint32_t *scene_of_agent,
                     const hsr_pose *poses, uint32_t n, const hsr_intrinsics *intr, uint32_t width,
                     uint32_t height, uint8_t *rgb, float *depth, uint32_t *ids, const hsr_depth_noise *noise,
                     void *cuda_stream)
{
    if (n_scenes > 1 && !scene_of_agent) return HSR_ERR_INVALID_ARG;
    NoiseReq nr;
    nr.noise = noise;
    return render_views(scenes, n_scenes, scene_of_agent, poses, n, intr, width, height, rgb, depth, ids,
                        cuda_stream, nullptr, nr);
}

}  // extern "C"
