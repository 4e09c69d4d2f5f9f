// Device-resident agents (Sec. 4 "Agent embodiment and action space"): the
// pose of every agent, the navigability grid of every scene and the
// actuation amounts live on the device, so a step batch sends only action
// ids; the actuation pass itself is in actuate.cu.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hsr.h"
#include "camera.h"
#include "hsr_internal.h"

struct hsr_agents {
    int device = 0;
    std::vector<const hsr_scene *> scenes;
    std::vector<uint32_t> scene_of_agent;
    std::vector<hsr_navmap> maps;                 // grid pointers into `grids`
    std::vector<std::vector<uint8_t>> grids;
    std::vector<hsr_scene_info> info;
    float *d_pose = nullptr;
    hsr::NavDev *d_nav = nullptr;
    uint8_t *d_grid = nullptr;
    hsr::AgentsDev *d_agents = nullptr;
    uint32_t n_agents = 0;
};

namespace hsr {
namespace {

bool map_ok(const hsr_navmap &m)
{
    if (!m.grid || m.nx == 0 || m.nz == 0 || (uint64_t)m.nx * m.nz > (1ull << 28)) return false;
    return finite_f(m.x0) && finite_f(m.z0) && finite_f(m.cell) && m.cell > 0.f;
}

// The grid test of the actuation rules: the cell holding (x, z), outside the
// grid counts as blocked.
bool navigable_host(const hsr_navmap &m, float x, float z)
{
    const double ci = std::floor(((double)x - (double)m.x0) / (double)m.cell);
    const double ck = std::floor(((double)z - (double)m.z0) / (double)m.cell);
    if (!(ci >= 0.0 && ci < (double)m.nx && ck >= 0.0 && ck < (double)m.nz)) return false;
    return m.grid[(size_t)ck * m.nx + (size_t)ci] != 0;
}

// Every navigable cell lies inside the scene's bounding box (x and z), so an
// agent that only ever stands on navigable cells stays inside it.
bool cells_inside(const hsr_navmap &m, const hsr_scene_info &in)
{
    for (uint32_t k = 0; k < m.nz; k++)
        for (uint32_t i = 0; i < m.nx; i++) {
            if (!m.grid[(size_t)k * m.nx + i]) continue;
            const double xa = (double)m.x0 + (double)i * m.cell, xb = xa + m.cell;
            const double za = (double)m.z0 + (double)k * m.cell, zb = za + m.cell;
            if (xa < in.aabb_min[0] || xb > in.aabb_max[0] || za < in.aabb_min[2] || zb > in.aabb_max[2])
                return false;
        }
    return true;
}

bool pose_ok(const hsr_agents &a, uint32_t scene, const hsr_pose &p)
{
    float M[12];
    if (!camera_from_pose(p.pos, p.quat, M)) return false;
    const hsr_scene_info &in = a.info[scene];
    if (!(p.pos[1] >= in.aabb_min[1] && p.pos[1] <= in.aabb_max[1])) return false;
    return navigable_host(a.maps[scene], p.pos[0], p.pos[2]);
}

void free_agents(hsr_agents *a)
{
    if (!a) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(a->device);
    cudaDeviceSynchronize();
    if (a->d_pose) cudaFree(a->d_pose);
    if (a->d_nav) cudaFree(a->d_nav);
    if (a->d_grid) cudaFree(a->d_grid);
    if (a->d_agents) cudaFree(a->d_agents);
    cudaSetDevice(prev);
    delete a;
}

int cuda_err(cudaError_t e) { return e == cudaErrorMemoryAllocation ? HSR_ERR_OOM : HSR_ERR_CUDA; }

}  // namespace

bool agents_view(const hsr_agents *a, AgentsView &out)
{
    if (!a) return false;
    out.device = a->device;
    out.scenes = a->scenes.data();
    out.n_scenes = (uint32_t)a->scenes.size();
    out.scene_of_agent = a->scene_of_agent.data();
    out.n_agents = a->n_agents;
    out.dev = a->d_agents;
    out.info = a->info.data();
    return true;
}

}  // namespace hsr

using namespace hsr;

extern "C" {

int hsr_agents_create(const hsr_scene *const *scenes, uint32_t n_scenes, const hsr_navmap *navmaps,
                      uint32_t n_agents, const uint32_t *scene_of_agent, const hsr_pose *poses,
                      const hsr_actuation *act, hsr_agents **out)
{
    if (!out) return HSR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!scenes || n_scenes == 0 || !navmaps || n_agents == 0 || !poses) return HSR_ERR_INVALID_ARG;
    hsr_actuation A{0.25f, 10.0f};
    if (act) A = *act;
    if (!finite_f(A.forward_m) || A.forward_m < 0.f || !finite_f(A.turn_deg)) return HSR_ERR_INVALID_ARG;
    hsr_agents *a = new (std::nothrow) hsr_agents();
    if (!a) return HSR_ERR_OOM;
    cudaGetDevice(&a->device);
    a->n_agents = n_agents;
    a->scenes.assign(scenes, scenes + n_scenes);
    a->info.resize(n_scenes);
    a->maps.resize(n_scenes);
    a->grids.resize(n_scenes);
    auto bad = [&](int st) {
        free_agents(a);
        return st;
    };
    size_t grid_bytes = 0;
    for (uint32_t s = 0; s < n_scenes; s++) {
        if (!scenes[s] || hsr_scene_get_info(scenes[s], &a->info[s]) != HSR_OK) return bad(HSR_ERR_INVALID_ARG);
        if (!map_ok(navmaps[s])) return bad(HSR_ERR_INVALID_ARG);
        a->maps[s] = navmaps[s];
        const size_t nb = (size_t)navmaps[s].nx * navmaps[s].nz;
        a->grids[s].assign(navmaps[s].grid, navmaps[s].grid + nb);
        a->maps[s].grid = a->grids[s].data();
        if (!cells_inside(a->maps[s], a->info[s])) return bad(HSR_ERR_INVALID_ARG);
        grid_bytes += (nb + 255) & ~(size_t)255;
    }
    a->scene_of_agent.resize(n_agents);
    std::vector<float> hp(7 * (size_t)n_agents);
    for (uint32_t i = 0; i < n_agents; i++) {
        const uint32_t s = scene_of_agent ? scene_of_agent[i] : 0u;
        if (s >= n_scenes || !pose_ok(*a, s, poses[i])) return bad(HSR_ERR_INVALID_ARG);
        a->scene_of_agent[i] = s;
        std::memcpy(&hp[7 * (size_t)i], poses[i].pos, 3 * sizeof(float));
        std::memcpy(&hp[7 * (size_t)i + 3], poses[i].quat, 4 * sizeof(float));
    }
    cudaError_t e;
    if ((e = cudaMalloc(&a->d_pose, hp.size() * sizeof(float))) != cudaSuccess) return bad(cuda_err(e));
    if ((e = cudaMalloc(&a->d_nav, n_scenes * sizeof(NavDev))) != cudaSuccess) return bad(cuda_err(e));
    if ((e = cudaMalloc(&a->d_grid, grid_bytes)) != cudaSuccess) return bad(cuda_err(e));
    if ((e = cudaMalloc(&a->d_agents, sizeof(AgentsDev))) != cudaSuccess) return bad(cuda_err(e));
    std::vector<NavDev> nav(n_scenes);
    size_t off = 0;
    for (uint32_t s = 0; s < n_scenes; s++) {
        const hsr_navmap &m = a->maps[s];
        const size_t nb = (size_t)m.nx * m.nz;
        if ((e = cudaMemcpy(a->d_grid + off, m.grid, nb, cudaMemcpyHostToDevice)) != cudaSuccess)
            return bad(cuda_err(e));
        NavDev &d = nav[s];
        std::memset(&d, 0, sizeof(d));
        d.x0 = m.x0; d.z0 = m.z0; d.cell = m.cell; d.nx = m.nx; d.nz = m.nz;
        d.grid = a->d_grid + off;
        off += (nb + 255) & ~(size_t)255;
    }
    AgentsDev ad{};
    ad.pose = a->d_pose;
    ad.nav = a->d_nav;
    ad.n_agents = n_agents;
    ad.n_scenes = n_scenes;
    ad.step = (double)A.forward_m;
    for (int r = 0; r < 2; r++) {
        const double t = (r == 0 ? (double)A.turn_deg : -(double)A.turn_deg) * (3.14159265358979323846 / 180.0);
        ad.c_turn[r] = std::cos(0.5 * t);
        ad.s_turn[r] = std::sin(0.5 * t);
    }
    if ((e = cudaMemcpy(a->d_nav, nav.data(), n_scenes * sizeof(NavDev), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(a->d_agents, &ad, sizeof(ad), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(a->d_pose, hp.data(), hp.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
        return bad(cuda_err(e));
    *out = a;
    return HSR_OK;
}

int hsr_agents_get_poses(hsr_agents *a, hsr_pose *poses, void *cuda_stream)
{
    if (!a || !poses) return HSR_ERR_INVALID_ARG;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    std::vector<float> hp(7 * (size_t)a->n_agents);
    cudaError_t e = cudaMemcpyAsync(hp.data(), a->d_pose, hp.size() * sizeof(float), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return HSR_ERR_CUDA;
    for (uint32_t i = 0; i < a->n_agents; i++) {
        std::memcpy(poses[i].pos, &hp[7 * (size_t)i], 3 * sizeof(float));
        std::memcpy(poses[i].quat, &hp[7 * (size_t)i + 3], 4 * sizeof(float));
    }
    return HSR_OK;
}

int hsr_agents_set_poses(hsr_agents *a, const uint32_t *idx, const hsr_pose *poses, uint32_t n, void *cuda_stream)
{
    if (!a || !idx || !poses || n == 0) return HSR_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < n; i++)
        if (idx[i] >= a->n_agents || !pose_ok(*a, a->scene_of_agent[idx[i]], poses[i])) return HSR_ERR_INVALID_ARG;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    float buf[7];
    for (uint32_t i = 0; i < n; i++) {
        std::memcpy(buf, poses[i].pos, 3 * sizeof(float));
        std::memcpy(buf + 3, poses[i].quat, 4 * sizeof(float));
        // pageable source: the copy has consumed `buf` when the call returns
        if (cudaMemcpyAsync(a->d_pose + 7 * (size_t)idx[i], buf, sizeof(buf), cudaMemcpyHostToDevice, stream) !=
            cudaSuccess)
            return HSR_ERR_CUDA;
    }
    return HSR_OK;
}

int hsr_agents_destroy(hsr_agents *a)
{
    free_agents(a);
    return HSR_OK;
}

}  // extern "C"
