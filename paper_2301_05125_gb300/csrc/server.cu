// server.cu -- continuous-batching request loop for many resident volumes.
//
// A worker thread owns the device side.  Clients submit per-frame update
// requests (any thread); each volume keeps a FIFO of its requests.  The
// worker admits volumes while their estimated device memory fits the budget
// (later ones wait until memory is released), and whenever one of its CUDA
// streams ("slots") is free it starts the oldest request of an idle resident
// volume there as a replay of that volume's captured update graph -- so the
// work of different volumes overlaps on the device and a request never waits
// for a batch boundary.  Completion is observed through one event per slot;
// each result records submit, start and completion times (host clock).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/adgi.h"
#include "adgi_internal.cuh"

namespace adgi {
const char* noalloc_fail(const std::string& msg);
}

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
    uint64_t id = 0;
    double t_submit = 0.0;
    adgi_frame frame{};
    std::vector<adgi_light> lights;
    int move_first = 0;
    std::vector<float> move_verts;
};

struct Vol {
    int id = -1;
    adgi_volume_desc desc{};
    std::vector<float> verts, albedo;
    std::vector<int32_t> idx;
    adgi_volume v = nullptr;
    bool resident = false, busy = false, removed = false, failed = false;
    size_t est_bytes = 0;
    std::deque<Req> q;
    uint64_t rays = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int vol = -1;  // volume in flight, -1 if free
    int rc = 0;    // status of the enqueueing calls
    Req req;
    double t_start = 0.0;
};

}  // namespace

struct adgi_server_s {
    std::mutex mu;
    std::condition_variable cv, idle_cv;
    std::thread worker;
    bool stop = false;
    int coalesce = 0, use_graph = 1;
    cudaStream_t adm_stream = nullptr;  // volume creation and scene upload
    size_t budget = 0, used = 0;
    int device = 0;
    std::deque<Vol> vols;  // deque: references stay valid while volumes are added
    std::vector<Slot> slots;
    std::vector<adgi_result> done;
    uint64_t next_id = 1;
    uint64_t superseded = 0;
    std::string error;
};

namespace {

size_t estimate_bytes(const adgi_volume_desc& d, int nv, int nt)
{
    const size_t P = (size_t)d.dims[0] * d.dims[1] * d.dims[2];
    const size_t Ti = (size_t)(d.irr_interior + 2), Td = (size_t)(d.depth_interior + 2);
    const size_t atl = P * (Ti * Ti * (d.atlas_fp16 ? 8 : 16) + Td * Td * ((d.atlas_fp16 ? 4 : 8) + 1));
    const size_t R = P * (size_t)d.rays_avg;
    const size_t rays = R * (8 + 16 + 8 + 4 * 17) + P * 200;  // hits, records, visibility, shadow jobs (4 lights)
    const size_t M = (size_t)(d.rays_max - 8);
    const size_t sf = 16 * M * (M + 1) / 2;
    const size_t scene = (size_t)nv * 13 + (size_t)nt * (12 + 12 + 48 + 8 + 84 + 48 + 64 + 96 + 64);
    return atl + rays + sf + scene + ((size_t)16 << 20);
}

// admission, dispatch and completion; called by the worker with mu held
void worker_step(adgi_server s, std::unique_lock<std::mutex>& lk)
{
    // completions
    for (auto& sl : s->slots) {
        if (sl.vol < 0) continue;
        cudaError_t e = cudaEventQuery(sl.done);
        if (e == cudaErrorNotReady) continue;
        Vol& V = s->vols[sl.vol];
        adgi_result r{};
        r.request_id = sl.req.id;
        r.volume = sl.vol;
        r.status = sl.rc ? sl.rc : e == cudaSuccess ? ADGI_OK : ADGI_ERR_CUDA;
        r.t_submit_s = sl.req.t_submit;
        r.t_start_s = sl.t_start;
        r.t_done_s = now_s();
        r.rays = (uint64_t)V.desc.dims[0] * V.desc.dims[1] * V.desc.dims[2] * (uint64_t)V.desc.rays_avg;
        s->done.push_back(r);
        V.busy = false;
        sl.vol = -1;
        s->idle_cv.notify_all();
    }
    // admission in registration order while the budget allows
    for (size_t i = 0; i < s->vols.size(); ++i) {  // indices: the lock is dropped inside
        Vol& V = s->vols[i];
        if (V.resident || V.removed || V.failed) continue;
        if (s->used + V.est_bytes > s->budget) break;
        lk.unlock();
        adgi_volume v = nullptr;
        int rc = adgi_create_volume(&V.desc, s->adm_stream, &v);
        if (!rc)
            rc = adgi_set_scene(v, V.verts.data(), (int32_t)(V.verts.size() / 3), V.idx.data(),
                                (int32_t)(V.idx.size() / 3), V.albedo.data(), 0);
        adgi_stats st{};
        if (!rc) rc = adgi_get_stats(v, &st);
        lk.lock();
        if (rc) {  // the volume never becomes resident: its requests fail
            const std::string msg = adgi_last_error();
            lk.unlock();
            if (v) adgi_destroy(v);
            lk.lock();
            V.failed = true;
            s->error = msg;
            for (auto& r : V.q) {
                adgi_result x{};
                x.request_id = r.id;
                x.volume = V.id;
                x.status = rc;
                x.t_submit_s = r.t_submit;
                x.t_start_s = x.t_done_s = now_s();
                s->done.push_back(x);
            }
            V.q.clear();
            s->idle_cv.notify_all();
            continue;
        }
        V.v = v;
        V.resident = true;
        V.est_bytes = std::max(V.est_bytes, (size_t)st.device_bytes);  // charge what it really holds
        s->used += V.est_bytes;
        V.verts.clear();  // the scene now lives on the device
        V.verts.shrink_to_fit();
        V.idx.clear();
        V.idx.shrink_to_fit();
        V.albedo.clear();
        V.albedo.shrink_to_fit();
    }
    // dispatch: every free slot takes the oldest request of an idle resident volume
    for (auto& sl : s->slots) {
        if (sl.vol >= 0) continue;
        int best = -1;
        double t_best = 0.0;
        for (auto& V : s->vols) {
            if (!V.resident || V.busy || V.removed || V.q.empty()) continue;
            if (best < 0 || V.q.front().t_submit < t_best) {
                best = V.id;
                t_best = V.q.front().t_submit;
            }
        }
        if (best < 0) break;
        Vol& V = s->vols[best];
        if (s->coalesce)
            while (V.q.size() > 1) {  // a newer frame supersedes the queued one
                adgi_result r{};
                r.request_id = V.q.front().id;
                r.volume = best;
                r.status = 1;  // superseded
                r.t_submit_s = V.q.front().t_submit;
                r.t_start_s = r.t_done_s = now_s();
                s->done.push_back(r);
                s->superseded++;
                V.q.pop_front();
            }
        sl.req = std::move(V.q.front());
        V.q.pop_front();
        V.busy = true;
        sl.vol = best;
        lk.unlock();
        sl.t_start = now_s();
        adgi_set_stream(V.v, sl.stream);
        int rc = ADGI_OK;
        if (!sl.req.move_verts.empty())
            rc = adgi_move_vertices(V.v, sl.req.move_first, (int32_t)(sl.req.move_verts.size() / 3),
                                    sl.req.move_verts.data(), 0);
        sl.req.frame.lights = sl.req.lights.data();
        if (!rc) rc = s->use_graph ? adgi_update_graph(V.v, &sl.req.frame) : adgi_update(V.v, &sl.req.frame);
        cudaError_t e = cudaEventRecord(sl.done, sl.stream);
        sl.rc = rc ? rc : e == cudaSuccess ? ADGI_OK : ADGI_ERR_CUDA;
        lk.lock();
        if (rc || e != cudaSuccess) s->error = rc ? adgi_last_error() : cudaGetErrorString(e);
        V.rays += (uint64_t)V.desc.dims[0] * V.desc.dims[1] * V.desc.dims[2] * (uint64_t)V.desc.rays_avg;
    }
}

void worker_main(adgi_server s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        worker_step(s, lk);
        bool inflight = false;
        for (auto& sl : s->slots) inflight = inflight || sl.vol >= 0;
        if (inflight)
            s->cv.wait_for(lk, std::chrono::microseconds(50));
        else
            s->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
}

int sfail(int code, const std::string& m)
{
    adgi::noalloc_fail(m);
    return code;
}

}  // namespace

extern "C" {

int adgi_server_create(int32_t streams, uint64_t hbm_budget_bytes, int32_t flags, adgi_server* out)
{
    if (!out || streams < 1 || streams > 64 || hbm_budget_bytes == 0 ||
        (flags & ~(ADGI_SERVER_COALESCE | ADGI_SERVER_NO_GRAPH)))
        return sfail(ADGI_ERR_INVALID_ARG, "server: streams in [1,64], budget > 0, known flags");
    *out = nullptr;
    adgi_server s = new adgi_server_s();
    s->budget = (size_t)hbm_budget_bytes;
    s->coalesce = (flags & ADGI_SERVER_COALESCE) ? 1 : 0;
    s->use_graph = (flags & ADGI_SERVER_NO_GRAPH) ? 0 : 1;
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->adm_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return sfail(ADGI_ERR_CUDA, "server: admission stream");
    }
    s->slots.resize((size_t)streams);
    for (auto& sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            for (auto& x : s->slots) {
                if (x.stream) cudaStreamDestroy(x.stream);
                if (x.done) cudaEventDestroy(x.done);
            }
            cudaStreamDestroy(s->adm_stream);
            delete s;
            return sfail(ADGI_ERR_CUDA, "server: stream creation");
        }
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return ADGI_OK;
}

int adgi_server_add_volume(adgi_server s, const adgi_volume_desc* desc, const float* verts, int32_t nv,
                           const int32_t* idx, int32_t nt, const float* albedo, int32_t* id_out)
{
    if (!s || !desc || !id_out || nv < 0 || nt < 0 || (nv && !verts) || (nt && (!idx || !albedo)))
        return sfail(ADGI_ERR_INVALID_ARG, "server: bad volume arguments");
    Vol V;
    V.desc = *desc;
    V.verts.assign(verts, verts + 3 * (size_t)nv);
    V.idx.assign(idx, idx + 3 * (size_t)nt);
    V.albedo.assign(albedo, albedo + 3 * (size_t)nt);
    V.est_bytes = estimate_bytes(*desc, nv, nt);
    std::lock_guard<std::mutex> lk(s->mu);
    if (V.est_bytes > s->budget) return sfail(ADGI_ERR_OVER_BUDGET, "server: volume larger than the whole budget");
    V.id = (int)s->vols.size();
    *id_out = V.id;
    s->vols.push_back(std::move(V));
    s->cv.notify_all();
    return ADGI_OK;
}

int adgi_server_submit(adgi_server s, int32_t vol, const adgi_frame* frame, int32_t move_first, int32_t move_count,
                       const float* move_verts, uint64_t* req_id)
{
    if (!s || !frame || (move_count > 0 && !move_verts) || move_count < 0 || frame->n_lights < 0 ||
        frame->n_lights > 64 || (frame->n_lights > 0 && !frame->lights))
        return sfail(ADGI_ERR_INVALID_ARG, "server: bad request");
    Req r;
    r.frame = *frame;
    r.lights.assign(frame->lights, frame->lights + frame->n_lights);
    r.move_first = move_first;
    if (move_count > 0) r.move_verts.assign(move_verts, move_verts + 3 * (size_t)move_count);
    r.t_submit = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    if (vol < 0 || vol >= (int)s->vols.size() || s->vols[vol].removed || s->vols[vol].failed)
        return sfail(ADGI_ERR_INVALID_ARG, "server: unknown volume");
    r.id = s->next_id++;
    if (req_id) *req_id = r.id;
    s->vols[vol].q.push_back(std::move(r));
    s->cv.notify_all();
    return ADGI_OK;
}

int adgi_server_poll(adgi_server s, adgi_result* out, int32_t max, int32_t* n)
{
    if (!s || !n || (max > 0 && !out)) return sfail(ADGI_ERR_INVALID_ARG, "server: bad poll");
    std::lock_guard<std::mutex> lk(s->mu);
    int k = 0;
    while (k < max && k < (int)s->done.size()) {
        out[k] = s->done[k];
        ++k;
    }
    s->done.erase(s->done.begin(), s->done.begin() + k);
    *n = k;
    return s->error.empty() ? ADGI_OK : sfail(ADGI_ERR_CUDA, "server: " + s->error);
}

int adgi_server_drain(adgi_server s, double timeout_s)
{
    if (!s) return sfail(ADGI_ERR_INVALID_ARG, "server: NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    const double t_end = now_s() + timeout_s;
    for (;;) {
        bool pending = false;
        for (auto& V : s->vols)
            if (!V.removed && !V.failed && (V.busy || (!V.q.empty()))) pending = true;
        if (!pending) return ADGI_OK;
        if (now_s() > t_end) return sfail(ADGI_ERR_TIMEOUT, "server: drain timed out");
        s->cv.notify_all();
        s->idle_cv.wait_for(lk, std::chrono::milliseconds(1));
    }
}

int adgi_server_volume(adgi_server s, int32_t vol, adgi_volume* out)
{
    if (!s || !out) return sfail(ADGI_ERR_INVALID_ARG, "server: NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    if (vol < 0 || vol >= (int)s->vols.size()) return sfail(ADGI_ERR_INVALID_ARG, "server: unknown volume");
    Vol& V = s->vols[vol];
    if (!V.resident || V.busy || !V.q.empty()) return sfail(ADGI_ERR_INVALID_ARG, "server: volume not idle");
    *out = V.v;
    return ADGI_OK;
}

int adgi_server_remove_volume(adgi_server s, int32_t vol)
{
    if (!s) return sfail(ADGI_ERR_INVALID_ARG, "server: NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    if (vol < 0 || vol >= (int)s->vols.size()) return sfail(ADGI_ERR_INVALID_ARG, "server: unknown volume");
    Vol& V = s->vols[vol];
    V.removed = true;
    V.q.clear();
    while (V.busy) s->idle_cv.wait_for(lk, std::chrono::milliseconds(1));
    if (V.resident) {
        adgi_volume v = V.v;
        V.v = nullptr;
        V.resident = false;
        lk.unlock();
        adgi_destroy(v);
        lk.lock();
        s->used -= V.est_bytes;  // the memory is free: waiting volumes may now be admitted
    }
    s->cv.notify_all();
    return ADGI_OK;
}

int adgi_server_info(adgi_server s, uint64_t* used_bytes, uint64_t* superseded, int32_t* resident, int32_t* waiting)
{
    if (!s) return sfail(ADGI_ERR_INVALID_ARG, "server: NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    int r = 0, w = 0;
    for (auto& V : s->vols) {
        if (V.removed || V.failed) continue;
        if (V.resident)
            ++r;
        else
            ++w;
    }
    if (used_bytes) *used_bytes = s->used;
    if (superseded) *superseded = s->superseded;
    if (resident) *resident = r;
    if (waiting) *waiting = w;
    return ADGI_OK;
}

int adgi_server_destroy(adgi_server s)
{
    if (!s) return ADGI_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    s->worker.join();
    for (auto& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
    }
    for (auto& V : s->vols)
        if (V.v) adgi_destroy(V.v);
    for (auto& sl : s->slots) {
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    cudaStreamDestroy(s->adm_stream);
    delete s;
    return ADGI_OK;
}

}  // extern "C"
