// hsr_render_noalloc: a variant of hsr_render that performs no memory
// allocation of any kind on the call path.
//
// Some callers cannot let a library allocate: a training process whose
// framework has already reserved (nearly) all device memory in its own
// caching pool, where an extra cudaMalloc would fail or fragment that pool;
// latency-critical loops where an allocator call may block or synchronise the
// device; and hosts that require every device allocation to go through their
// own allocator. For them, the scratch this render needs (per-view
// descriptors, the 64-bit z-buffer, the visible-meshlet list and the
// per-tile occlusion buffer) lives in one
// fixed array in device memory, created when the library is loaded, rather
// than in buffers obtained per call.
//
// Limits and rules (also stated in include/hsr.h):
//  * the array holds kNoAllocScratchBytes = 32 MiB; a call needing more
//    (about 8 bytes per output pixel per view plus 48 bytes per meshlet per
//    view, plus 192 bytes per view) is rejected with HSR_ERR_OVERFLOW;
//  * the host-side descriptors are staged in a fixed 1 MiB host buffer
//    (192 bytes per view after a 768-byte header: at most 5,457 views per
//    call; more return HSR_ERR_OVERFLOW). That buffer is ordinary pageable memory,
//    copied to the device with cudaMemcpyAsync under a process-wide lock, so
//    the copy has finished reading it when the call returns and the call may
//    wait for the stream's earlier work;
//  * every GPU that loads the library keeps the 32 MiB array until the
//    process exits;
//  * all calls share the array: two calls whose work overlaps on the GPU
//    (different streams, or different host threads without ordering) race
//    and give wrong images. Serialise them on one stream.
//  * the first call on each device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it.
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/hsr.h"
#include "hsr_internal.h"
#include "launch_defaults.h"

namespace hsr {

bool host_camera_matrix(const hsr_pose &pose, float M[12]);
bool host_intrinsics_ok(const hsr_intrinsics *in);
float host_far_threshold(float zfar);
float host_guard_g(float f);
bool host_guard_free(const hsr_scene *s, const hsr_pose &pose, const hsr_intrinsics &in);
void host_view_planes(const float M[12], const hsr_intrinsics &in, uint32_t W, uint32_t H, float planes[24]);
const SceneDev &host_scene_dev(const hsr_scene *s);

constexpr size_t kNoAllocScratchBytes = 32ull << 20;
constexpr size_t kNoAllocHostBytes = 1ull << 20;
constexpr int kNoAllocMaxDevices = 64;

// The fixed device scratch. In host code this name is only a stand-in for the
// symbol: its device address must come from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_noalloc_mu;
void *g_noalloc_dev_ptr[kNoAllocMaxDevices] = {};
alignas(256) unsigned char g_noalloc_host[kNoAllocHostBytes];

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
}  // namespace

}  // namespace hsr

using namespace hsr;

extern "C" HSR_API int hsr_render_noalloc(const hsr_scene *scene, const hsr_pose *poses, uint32_t n,
                                          const hsr_intrinsics *intr, uint32_t width, uint32_t height, uint8_t *rgb,
                                          float *depth, uint32_t *ids, void *cuda_stream)
{
    if (!scene || !poses || n == 0 || !(rgb || depth || ids)) return HSR_ERR_INVALID_ARG;
    if (width == 0 || height == 0 || width > 4096 || height > 4096) return HSR_ERR_INVALID_ARG;
    if (!host_intrinsics_ok(intr)) return HSR_ERR_INVALID_ARG;
    const SceneDev &sd = host_scene_dev(scene);

    // layout of the scratch array:
    // [counters | scene | slot | views | z-buffer | visible lists | tile-z pyramid | survivor list]
    const size_t off_scene = 256;
    const size_t off_slots = off_scene + align256(sizeof(SceneDev));
    const size_t off_views = off_slots + 256;
    const size_t desc_bytes = off_views + (size_t)n * sizeof(View);
    const size_t off_z = align256(desc_bytes);
    const uint64_t zbytes = align256((size_t)n * width * height * sizeof(unsigned long long));
    const uint64_t list_entries = (uint64_t)n * sd.n_meshlets;
    const uint64_t items = (uint64_t)n * sd.n_groups;
    const uint32_t hiz_w = (width + kHizTile - 1) / kHizTile, hiz_h = (height + kHizTile - 1) / kHizTile;
    const uint32_t hiz_total = hiz_pyramid_texels(hiz_w, hiz_h, nullptr);
    const uint64_t hbytes = align256((uint64_t)n * hiz_total * sizeof(uint32_t));
    const uint64_t lbytes = align256(2 * list_entries * sizeof(uint4));
    const uint64_t sbytes = list_entries * sizeof(uint4);
    const uint64_t need = (uint64_t)off_z + zbytes + lbytes + hbytes + sbytes;
    if (need > kNoAllocScratchBytes || desc_bytes > kNoAllocHostBytes) return HSR_ERR_OVERFLOW;
    if (items >= 0xFFFFFFF0ull) return HSR_ERR_OVERFLOW;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HSR_ERR_CUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return HSR_ERR_INVALID_ARG;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_dev_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return HSR_ERR_CUDA;
        g_noalloc_dev_ptr[dev] = ptr;
    }
    unsigned char *d = static_cast<unsigned char *>(g_noalloc_dev_ptr[dev]);

    // host descriptors (counters start at zero)
    unsigned char *h = g_noalloc_host;
    std::memset(h, 0, off_views);
    std::memcpy(h + off_scene, &sd, sizeof(SceneDev));
    uint32_t *slot = reinterpret_cast<uint32_t *>(h + off_slots);
    slot[0] = 0;                    // slot_item_base[0]
    slot[1] = (uint32_t)items;      // slot_item_base[1]
    slot[2] = 0;                    // slot_view_base[0]
    slot[3] = 0;                    // slot_scene[0]
    uint32_t *hdr = reinterpret_cast<uint32_t *>(h);
    hdr[16] = n;                    // active views
    hdr[17] = (uint32_t)items;      // work items
    hdr[18] = 1;                    // slots in use
    View *hv = reinterpret_cast<View *>(h + off_views);
    const uint32_t outputs = (rgb ? HSR_OUT_RGB : 0u) | (depth ? HSR_OUT_DEPTH : 0u) | (ids ? HSR_OUT_IDS : 0u);
    bool guard = false;
    for (uint32_t i = 0; i < n; i++) {
        View &v = hv[i];
        std::memset(&v, 0, sizeof(View));
        if (!host_camera_matrix(poses[i], v.M)) return HSR_ERR_INVALID_ARG;
        guard |= !host_guard_free(scene, poses[i], *intr);
        host_view_planes(v.M, *intr, width, height, v.planes);
        for (int k = 0; k < 3; k++) v.pos[k] = poses[i].pos[k];
        v.scene = 0;
        v.frame = i;
        v.agent = i;
        v.outputs = outputs;
    }
    // Pageable source: the copy has consumed `h` when this call returns. The
    // z-buffer needs no preset: the culling kernel clears every active view's.
    if (cudaMemcpyAsync(d, h, desc_bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess) return HSR_ERR_CUDA;

    Params p{};
    p.vis_count = reinterpret_cast<uint32_t *>(d);
    p.work_counter = reinterpret_cast<uint32_t *>(d) + 4;
    p.scenes = reinterpret_cast<const SceneDev *>(d + off_scene);
    const uint32_t *dslot = reinterpret_cast<const uint32_t *>(d + off_slots);
    p.slot_item_base = dslot;
    p.slot_view_base = dslot + 2;
    p.slot_scene = dslot + 3;
    p.n_slots = 1;
    p.dyn = reinterpret_cast<const uint32_t *>(d) + 16;
    p.views = reinterpret_cast<const View *>(d + off_views);
    p.zbuf = reinterpret_cast<unsigned long long *>(d + off_z);
    p.vis = reinterpret_cast<uint4 *>(d + off_z + zbytes);
    p.vis_cap = (uint32_t)list_entries;
    p.rgb = rgb;
    p.depth = depth;
    p.ids = ids;
    p.n_views = n;
    p.width = width;
    p.height = height;
    p.total_items = (uint32_t)items;
    p.fx = intr->fx; p.fy = intr->fy; p.cx = intr->cx; p.cy = intr->cy;
    p.znear = intr->znear; p.zfar = intr->zfar;
    p.q_far = host_far_threshold(intr->zfar);
    p.inv_far = (float)(1.0 / (double)intr->zfar);
    p.gx = host_guard_g(intr->fx);
    p.gy = host_guard_g(intr->fy);
    // the bounded-wait test hook and the diagnostic counters, as in
    // hsr_render (neither allocates here); the large-triangle bins stay off
    // (big_rec null: no scratch for them), so every large triangle takes
    // the per-warp queue
    p.fault_tx = debug_fault_tx();
    p.stats = stage_stats_buffer();
    const LaunchCfg cfg = default_launch_cfg(items, (uint64_t)n * width * height);
    p.small_px = cfg.small_px < 32 ? cfg.small_px : 32;
    p.chunk = cfg.chunk > 0 ? (cfg.chunk < 32 ? cfg.chunk : 32) : 1;
    p.hiz = reinterpret_cast<uint32_t *>(d + off_z + zbytes + lbytes);
    p.hiz_total = hiz_total;
    p.surv = reinterpret_cast<uint4 *>(d + off_z + zbytes + lbytes + hbytes);
    p.surv_count = reinterpret_cast<uint32_t *>(d) + 24;
    p.hiz_w = hiz_w;
    p.hiz_h = hiz_h;
    p.n_phases = cfg.n_phases;
    p.phase_r2[0] = cfg.phase_r[0] * cfg.phase_r[0];
    p.phase_r2[1] = cfg.phase_r[1] * cfg.phase_r[1];
    return launch_render(p, cfg, stream, guard, false, true) == cudaSuccess ? HSR_OK : HSR_ERR_CUDA;
}
