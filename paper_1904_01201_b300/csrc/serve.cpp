// Serving core: continuous batching of render requests (include/hsr.h,
// hsr_server_*). The paper's simulator renders an observation each time an
// agent steps (Sec. 4, actions move_forward / turn); here many rollout
// workers submit such requests concurrently and a scheduler thread packs them
// into graph-replayed micro-batches per resolution, admitted against a fixed
// framebuffer budget, with several micro-batches in flight on separate
// streams; a completion thread polls each stream's event and hands finished
// results back.
#include "../../include/hsr.h"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "hsr_internal.h"

namespace hsr {
int batch_create(const hsr_scene *const *scenes, uint32_t n_scenes, uint32_t n_cap, uint32_t n_frames,
                 const hsr_intrinsics *intr, uint32_t width, uint32_t height, uint8_t *rgb, float *depth,
                 uint32_t *ids, const hsr_config *cfg, hsr_batch **out);
}

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Pending {
    hsr_request req;
    double t_submit;
    uint64_t seq;              // action requests: the agent's submission number
};

struct ResPool {
    uint32_t res = 0;
    uint32_t slots = 0;
    uint8_t *rgb = nullptr;
    float *depth = nullptr;
    uint32_t *ids = nullptr;
    hsr_intrinsics intr{};
    std::vector<uint32_t> free_slots;
    std::vector<hsr_batch *> batch;      // one per stream
    std::deque<Pending> pending;         // pose requests
    std::deque<Pending> pending_act;     // action requests
};

struct InFlight;

}  // namespace

struct hsr_server {
    int device = 0;
    std::vector<const hsr_scene *> scenes;
    hsr_server_config cfg{};
    std::vector<ResPool> pools;
    std::vector<cudaStream_t> streams;
    std::vector<bool> busy;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<Pending> incoming;
    std::deque<hsr_result> done;
    std::thread worker;
    // completion: each stream's batch records done_ev[st]; the completion
    // thread polls the streams whose batch is in flight (flight[st])
    std::vector<cudaEvent_t> done_ev;
    std::vector<InFlight *> flight;
    std::condition_variable flight_cv;
    std::thread completer;
    bool stop = false;
    uint64_t submitted = 0, completed = 0, rejected = 0, batches = 0;
    uint32_t in_flight = 0, queued = 0;
    uint64_t fb_used = 0, fb_total = 0;
    // attached agents (action requests)
    hsr_agents *agents = nullptr;
    uint32_t n_agents = 0;
    std::vector<uint64_t> agent_submitted, agent_launched;
    std::vector<uint8_t> agent_busy;
};

namespace {

struct InFlight {
    hsr_server *srv;
    int stream;
    std::vector<hsr_result> results;
    std::vector<uint32_t> agents;        // action batches: the agents to free on completion
};

// How far into an action queue the scheduler looks for requests whose agent
// is free (requests behind a busy agent wait without blocking the others).
constexpr size_t kActScan = 8;

// Action requests of a queue that may launch now, in queue order: the agent's
// oldest unlaunched action, agent not in flight; at most `max` of them.
void eligible_actions(const hsr_server *s, const std::deque<Pending> &q, size_t max, std::vector<size_t> &pos)
{
    pos.clear();
    const size_t scan = std::min(q.size(), kActScan * std::max<size_t>(max, 1));
    for (size_t i = 0; i < scan && pos.size() < max; i++) {
        const Pending &p = q[i];
        const uint32_t a = (uint32_t)p.req.agent;
        if (s->agent_busy[a] || p.seq != s->agent_launched[a]) continue;
        bool dup = false;
        for (size_t j : pos) dup |= q[j].req.agent == p.req.agent;
        if (!dup) pos.push_back(i);
    }
}

uint64_t frame_bytes(uint32_t res, bool ids) { return (uint64_t)res * res * (ids ? 11u : 7u); }

// A batch has finished on its stream (s->mu held): its results become
// available, its stream and agents free; `status` is HSR_OK unless the
// stream reported an error.
void finish_batch(hsr_server *s, InFlight *f, double t, int status)
{
    for (hsr_result &r : f->results) {
        r.t_done = t;
        if (status != HSR_OK) r.status = status;
        s->done.push_back(r);
    }
    s->completed += f->results.size();
    s->in_flight -= (uint32_t)f->results.size();
    s->busy[f->stream] = false;
    for (uint32_t a : f->agents) s->agent_busy[a] = false;
}

// Completion thread: polls the event of every stream with a batch in flight
// (yielding between rounds, so a finished batch is seen within a few
// microseconds), sleeps while none is; after stop, finishes what is in flight.
// The events are queried without the server's lock (a stream's entry changes
// only after its batch is finished here), so the scheduler thread is not
// kept waiting for the lock.
void complete_loop(hsr_server *s)
{
    cudaSetDevice(s->device);
    std::vector<InFlight *> snap;
    std::vector<cudaError_t> state;
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        snap = s->flight;
        bool any = false;
        for (InFlight *f : snap) any |= f != nullptr;
        if (!any) {
            if (s->stop) break;
            s->flight_cv.wait(lock);
            continue;
        }
        lock.unlock();
        state.assign(snap.size(), cudaErrorNotReady);
        bool ready = false;
        for (size_t st = 0; st < snap.size(); st++)
            if (snap[st]) {
                state[st] = cudaEventQuery(s->done_ev[st]);
                ready |= state[st] != cudaErrorNotReady;
            }
        if (!ready) {
            std::this_thread::yield();
            lock.lock();
            continue;
        }
        const double t = now_s();
        lock.lock();
        for (size_t st = 0; st < snap.size(); st++) {
            if (!snap[st] || state[st] == cudaErrorNotReady) continue;
            finish_batch(s, snap[st], t, state[st] == cudaSuccess ? HSR_OK : HSR_ERR_CUDA);
            s->flight[st] = nullptr;
            delete snap[st];
        }
        s->cv.notify_all();
        s->done_cv.notify_all();
    }
}

void fail_request(hsr_server *s, const Pending &p, int status)
{
    hsr_result r{};
    r.tag = p.req.tag;
    r.status = status;
    r.res = p.req.res;
    r.t_submit = p.t_submit;
    r.t_launch = r.t_done = now_s();
    s->done.push_back(r);
    s->completed++;
}

// Scheduler thread: admit, pack, launch.
void run(hsr_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    while (!s->stop) {
        // route new requests to their resolution queues
        while (!s->incoming.empty()) {
            Pending p = s->incoming.front();
            s->incoming.pop_front();
            int r = -1;
            for (size_t k = 0; k < s->pools.size(); k++)
                if (s->pools[k].res == p.req.res) r = (int)k;
            const bool act = p.req.agent >= 0;
            if (r < 0 || (!act && p.req.scene >= s->scenes.size())) {
                // (action requests were checked at submit: they always route)
                s->queued--;
                fail_request(s, p, HSR_ERR_INVALID_ARG);
            }
            else if (act)
                s->pools[r].pending_act.push_back(p);
            else
                s->pools[r].pending.push_back(p);
        }
        // launch on free streams: the (resolution, kind) queue whose oldest
        // launchable request waited longest
        bool launched = false;
        double next_deadline = 1e300;
        std::vector<size_t> elig;
        for (size_t st = 0; st < s->streams.size(); st++) {
            if (s->busy[st]) continue;
            int best = -1, best_kind = 0;
            double oldest = 1e300;
            const double t = now_s();
            for (size_t k = 0; k < s->pools.size(); k++) {
                ResPool &P = s->pools[k];
                if (P.free_slots.empty()) continue;
                for (int kind = 0; kind < 2; kind++) {
                    const std::deque<Pending> &q = kind ? P.pending_act : P.pending;
                    if (q.empty()) continue;
                    const size_t lim = std::min<size_t>(P.free_slots.size(), s->cfg.max_batch);
                    size_t can;
                    double head;
                    if (kind) {
                        eligible_actions(s, q, lim, elig);
                        if (elig.empty()) continue;
                        can = elig.size();
                        head = q[elig[0]].t_submit;
                    } else {
                        can = std::min(q.size(), lim);
                        head = q.front().t_submit;
                    }
                    const double waited = t - head;
                    const bool full = can >= s->cfg.max_batch || can >= P.free_slots.size();
                    if (!full && waited * 1e6 < s->cfg.max_wait_us) {
                        next_deadline = std::min(next_deadline, head + s->cfg.max_wait_us * 1e-6);
                        continue;
                    }
                    if (head < oldest) {
                        oldest = head;
                        best = (int)k;
                        best_kind = kind;
                    }
                }
            }
            if (best < 0) break;
            ResPool &P = s->pools[best];
            std::deque<Pending> &q = best_kind ? P.pending_act : P.pending;
            const size_t lim = std::min<size_t>(P.free_slots.size(), s->cfg.max_batch);
            std::vector<Pending> take;
            if (best_kind) {
                eligible_actions(s, q, lim, elig);
                for (size_t j : elig) take.push_back(q[j]);
                for (size_t j = elig.size(); j-- > 0;) q.erase(q.begin() + (std::ptrdiff_t)elig[j]);
            } else {
                const size_t n0 = std::min(q.size(), lim);
                for (size_t j = 0; j < n0; j++) {
                    take.push_back(q.front());
                    q.pop_front();
                }
            }
            const uint32_t n = (uint32_t)take.size();
            InFlight *f = new (std::nothrow) InFlight();
            if (!f) {
                // out of host memory: put the requests back and retry later
                for (size_t j = take.size(); j-- > 0;) q.push_front(take[j]);
                break;
            }
            f->srv = s;
            f->stream = (int)st;
            std::vector<uint32_t> soa(n), frames(n), agent_idx(n);
            std::vector<uint8_t> actions(n);
            std::vector<hsr_pose> poses(n);
            const double tl = now_s();
            for (uint32_t i = 0; i < n; i++) {
                const Pending &p = take[i];
                const uint32_t slot = P.free_slots.back();
                P.free_slots.pop_back();
                if (best_kind) {
                    const uint32_t a = (uint32_t)p.req.agent;
                    agent_idx[i] = a;
                    actions[i] = (uint8_t)p.req.action;
                    s->agent_launched[a]++;
                    s->agent_busy[a] = 1;
                    f->agents.push_back(a);
                } else {
                    soa[i] = p.req.scene;
                    poses[i] = p.req.pose;
                }
                frames[i] = slot;
                hsr_result r{};
                r.tag = p.req.tag;
                r.status = HSR_OK;
                r.res = P.res;
                r.slot = slot;
                const size_t px = (size_t)P.res * P.res;
                r.rgb = P.rgb + 3 * px * slot;
                r.depth = P.depth + px * slot;
                r.ids = P.ids ? P.ids + px * slot : nullptr;
                r.t_submit = p.t_submit;
                r.t_launch = tl;
                f->results.push_back(r);
            }
            s->queued -= n;
            s->in_flight += n;
            s->fb_used += (uint64_t)n * frame_bytes(P.res, P.ids != nullptr);
            s->busy[st] = true;
            s->batches++;
            hsr_batch *b = P.batch[st];
            cudaStream_t stream = s->streams[st];
            lock.unlock();
            hsr_agents *ag = s->agents;
            int rc = best_kind ? hsr_batch_step(b, ag, agent_idx.data(), actions.data(), n, frames.data(), nullptr,
                                                stream)
                               : hsr_batch_render(b, soa.data(), poses.data(), n, frames.data(), stream);
            if (rc == HSR_OK && cudaEventRecord(s->done_ev[st], stream) != cudaSuccess) rc = HSR_ERR_CUDA;
            lock.lock();
            if (rc == HSR_OK) {
                s->flight[st] = f;
                s->flight_cv.notify_one();
            }
            if (rc != HSR_OK) {
                // the views could not be rendered: report the error, return the slots
                for (hsr_result &r : f->results) {
                    r.status = rc;
                    r.t_done = now_s();
                    P.free_slots.push_back(r.slot);
                    s->fb_used -= frame_bytes(P.res, P.ids != nullptr);
                    s->done.push_back(r);
                }
                s->completed += n;
                s->in_flight -= n;
                s->busy[st] = false;
                for (uint32_t a : f->agents) s->agent_busy[a] = false;
                delete f;
                s->done_cv.notify_all();
            }
            launched = true;
        }
        if (launched) continue;
        if (!s->incoming.empty()) continue;
        const double wait = std::min(1e-3, std::max(0.0, next_deadline - now_s()));
        s->cv.wait_for(lock, std::chrono::duration<double>(wait));
    }
}

void destroy_server(hsr_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    s->flight_cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    if (s->completer.joinable()) s->completer.join();
    cudaSetDevice(s->device);
    for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
    // a batch launched while the server stopped may not have been collected
    for (InFlight *f : s->flight) delete f;
    for (cudaEvent_t e : s->done_ev)
        if (e) cudaEventDestroy(e);
    for (ResPool &P : s->pools) {
        for (hsr_batch *b : P.batch) hsr_batch_destroy(b);
        if (P.rgb) cudaFree(P.rgb);
        if (P.depth) cudaFree(P.depth);
        if (P.ids) cudaFree(P.ids);
    }
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
}

}  // namespace

extern "C" {

double hsr_server_now(void) { return now_s(); }

int hsr_server_create(const hsr_scene *const *scenes, uint32_t n_scenes, const hsr_server_config *cfg,
                      hsr_server **out)
{
    if (!out || !scenes || n_scenes == 0 || !cfg) return HSR_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->n_res == 0 || cfg->n_res > 8 || cfg->max_batch == 0 || cfg->n_streams == 0 || cfg->n_streams > 16)
        return HSR_ERR_INVALID_ARG;
    if (!(cfg->znear > 0) || !(cfg->zfar > cfg->znear)) return HSR_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < n_scenes; i++)
        if (!scenes[i]) return HSR_ERR_INVALID_ARG;
    float wsum = 0;
    for (uint32_t k = 0; k < cfg->n_res; k++) {
        if (cfg->res[k] == 0 || cfg->res[k] > 4096 || !(cfg->res_weight[k] > 0)) return HSR_ERR_INVALID_ARG;
        wsum += cfg->res_weight[k];
    }
    hsr_server *s = new (std::nothrow) hsr_server();
    if (!s) return HSR_ERR_OOM;
    cudaGetDevice(&s->device);
    s->scenes.assign(scenes, scenes + n_scenes);
    s->cfg = *cfg;
    if (s->cfg.max_queue == 0) s->cfg.max_queue = 1u << 20;
    const bool ids = cfg->with_ids != 0;
    int rc = HSR_OK;
    for (uint32_t st = 0; st < cfg->n_streams && rc == HSR_OK; st++) {
        cudaStream_t stream = nullptr;
        if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) rc = HSR_ERR_CUDA;
        s->streams.push_back(stream);
        s->busy.push_back(false);
        cudaEvent_t ev = nullptr;
        if (rc == HSR_OK && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) rc = HSR_ERR_CUDA;
        s->done_ev.push_back(ev);
        s->flight.push_back(nullptr);
    }
    s->pools.resize(cfg->n_res);
    for (uint32_t k = 0; k < cfg->n_res && rc == HSR_OK; k++) {
        ResPool &P = s->pools[k];
        P.res = cfg->res[k];
        const uint64_t fb = frame_bytes(P.res, ids);
        const uint64_t share = (uint64_t)((double)cfg->fb_bytes * (cfg->res_weight[k] / wsum));
        P.slots = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(share / fb, 1u << 20));
        s->fb_total += (uint64_t)P.slots * fb;
        const size_t px = (size_t)P.res * P.res;
        if (cudaMalloc(&P.rgb, 3 * px * P.slots) != cudaSuccess || cudaMalloc(&P.depth, 4 * px * P.slots) != cudaSuccess ||
            (ids && cudaMalloc(&P.ids, 4 * px * P.slots) != cudaSuccess)) {
            rc = HSR_ERR_OOM;
            break;
        }
        for (uint32_t i = 0; i < P.slots; i++) P.free_slots.push_back(P.slots - 1 - i);
        P.intr.fx = P.intr.fy = P.intr.cx = P.intr.cy = P.res * 0.5f;
        P.intr.znear = cfg->znear;
        P.intr.zfar = cfg->zfar;
        const uint32_t cap = std::min(cfg->max_batch, P.slots);
        for (uint32_t st = 0; st < cfg->n_streams && rc == HSR_OK; st++) {
            hsr_batch *b = nullptr;
            rc = hsr::batch_create(scenes, n_scenes, cap, P.slots, &P.intr, P.res, P.res, P.rgb, P.depth, P.ids,
                                   nullptr, &b);
            P.batch.push_back(b);
        }
    }
    if (rc != HSR_OK) {
        destroy_server(s);
        return rc;
    }
    s->completer = std::thread(complete_loop, s);
    s->worker = std::thread(run, s);
    *out = s;
    return HSR_OK;
}

int hsr_server_attach_agents(hsr_server *s, hsr_agents *agents)
{
    if (!s) return HSR_ERR_INVALID_ARG;
    hsr::AgentsView av{};
    if (agents) {
        if (!hsr::agents_view(agents, av) || av.device != s->device || av.n_scenes != s->scenes.size())
            return HSR_ERR_INVALID_ARG;
        for (uint32_t i = 0; i < av.n_scenes; i++)
            if (av.scenes[i] != s->scenes[i]) return HSR_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->queued || s->in_flight || !s->incoming.empty()) return HSR_ERR_INVALID_ARG;
    s->agents = agents;
    s->n_agents = agents ? av.n_agents : 0;
    s->agent_submitted.assign(s->n_agents, 0);
    s->agent_launched.assign(s->n_agents, 0);
    s->agent_busy.assign(s->n_agents, 0);
    return HSR_OK;
}

int hsr_server_submit(hsr_server *s, const hsr_request *reqs, uint32_t n)
{
    if (!s || (!reqs && n)) return HSR_ERR_INVALID_ARG;
    const double t = now_s();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (uint32_t i = 0; i < n; i++) {
            Pending p{reqs[i], t, 0};
            s->submitted++;
            if (p.req.agent >= 0) {
                bool res_ok = false;
                for (const ResPool &P : s->pools) res_ok |= P.res == p.req.res;
                if (!res_ok || (uint32_t)p.req.agent >= s->n_agents || p.req.action > HSR_ACTION_TURN_RIGHT) {
                    fail_request(s, p, HSR_ERR_INVALID_ARG);
                    continue;
                }
            }
            if (s->queued >= s->cfg.max_queue) {
                s->rejected++;
                fail_request(s, p, HSR_ERR_OVERFLOW);
                continue;
            }
            if (p.req.agent >= 0) p.seq = s->agent_submitted[p.req.agent]++;
            s->queued++;
            s->incoming.push_back(p);
        }
    }
    s->cv.notify_all();
    s->done_cv.notify_all();
    return HSR_OK;
}

int hsr_server_poll(hsr_server *s, hsr_result *out, uint32_t max, uint32_t *n_out, uint32_t wait_us)
{
    if (!s || !n_out || (!out && max)) return HSR_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->done.empty() && wait_us)
        s->done_cv.wait_for(lock, std::chrono::microseconds(wait_us), [&] { return !s->done.empty(); });
    uint32_t k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *n_out = k;
    return HSR_OK;
}

int hsr_server_release(hsr_server *s, const hsr_result *results, uint32_t n)
{
    if (!s || (!results && n)) return HSR_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (uint32_t i = 0; i < n; i++) {
            const hsr_result &r = results[i];
            if (r.status != HSR_OK) continue;
            for (ResPool &P : s->pools)
                if (P.res == r.res && r.slot < P.slots) {
                    P.free_slots.push_back(r.slot);
                    s->fb_used -= frame_bytes(P.res, P.ids != nullptr);
                }
        }
    }
    s->cv.notify_all();
    return HSR_OK;
}

int hsr_server_get_stats(hsr_server *s, hsr_server_stats *st)
{
    if (!s || !st) return HSR_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->rejected = s->rejected;
    st->batches = s->batches;
    st->queued = s->queued;
    st->in_flight = s->in_flight;
    st->fb_bytes_used = s->fb_used;
    st->fb_bytes_total = s->fb_total;
    return HSR_OK;
}

int hsr_server_destroy(hsr_server *s)
{
    destroy_server(s);
    return HSR_OK;
}

}  // extern "C"
