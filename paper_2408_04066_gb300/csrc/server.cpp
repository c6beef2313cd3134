// Serving: continuous batching of pose solves over resident meshes.
//
// A worker thread owns the GPU work.  Between Newton steps it admits queued
// requests into free slots (per-mesh slot sets sized by the device-memory
// budget at mfem_server_add), then advances every admitted request of every
// mesh by one Newton step together -- the element and assembly kernels per
// mesh and one sequence of PCG iteration launches for all of them -- and hands finished
// requests back.  A request's arithmetic never depends on the others in the
// step (per-problem deterministic reductions), so its result equals the same
// pose solved alone.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.h"

using namespace mfem;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int mesh = -1;
    std::vector<double> xf;
    double* out = nullptr;
    int status = MFEM_OK;
    mfem_stats st{};
    double t_submit = 0.0, t_done = 0.0;
    bool done = false;
};

struct MeshEntry {
    mfem_ctx* ctx = nullptr;
    int cap = 0;
    std::vector<ProbHost> ph;
    std::vector<uint64_t> slot_req;  // 0 = free
    // WARM meshes: the mesh's most recent solution (x [n][3], its predictor
    // result [n][3] and its pose [H][12]), copied into the slot of each admitted
    // request, so every request continues from the latest frame solved
    double* bank = nullptr;
    int bank_state = 0;   // 0 none, 1 x and pose, 2 also the predictor result
};

}  // namespace

struct mfem_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Request> reqs;
    std::deque<MeshEntry> meshes;   // deque: references stay valid while meshes are added
    size_t budget = 0, used = 0;
    int max_slots = 0, in_use = 0, peak = 0;
    uint64_t next_ticket = 1;
    int64_t completed = 0, steps = 0, pcg_launches = 0;
    bool stop = false;
    bool started = false;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::thread worker;
    std::string err;

    void run();
    void fail_all_busy(int status);
};

void mfem_server::fail_all_busy(int status) {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& me : meshes)
        for (int b = 0; b < me.cap; ++b)
            if (me.slot_req[b]) {
                auto it = reqs.find(me.slot_req[b]);
                if (it != reqs.end()) {
                    it->second.status = status;
                    it->second.done = true;
                    it->second.t_done = now_s();
                }
                me.slot_req[b] = 0;
                me.ph[b] = ProbHost();
                in_use--;
            }
    cv_done.notify_all();
}

void mfem_server::run() {
    cudaSetDevice(device);
    for (;;) {
        std::vector<std::pair<int, int>> admitted;
        // the meshes known at this step, taken under the lock: mfem_server_add
        // may append to the deque meanwhile (element addresses stay valid)
        std::vector<MeshEntry*> ms;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || !queue.empty() || in_use > 0; });
            if (stop && in_use == 0) break;
            for (auto& m : meshes) ms.push_back(&m);
            // admission: FIFO scan, a full mesh does not block other meshes
            for (auto it = queue.begin(); it != queue.end() && in_use < max_slots;) {
                Request& r = reqs[*it];
                MeshEntry& me = meshes[r.mesh];
                int slot = -1;
                for (int b = 0; b < me.cap; ++b)
                    if (!me.slot_req[b]) { slot = b; break; }
                if (slot < 0) { ++it; continue; }
                me.slot_req[slot] = *it;
                me.ph[slot] = ProbHost();
                me.ph[slot].need_init = 1;
                in_use++;
                peak = std::max(peak, in_use);
                admitted.emplace_back(r.mesh, slot);
                const size_t H = me.ctx->plan.H;
                if (me.bank_state > 0) {
                    mfem_ctx* c = me.ctx;
                    const size_t n3 = (size_t)c->plan.n * 3;
                    cudaMemcpyAsync(c->slot.x + slot * n3, me.bank, n3 * sizeof(double), cudaMemcpyDeviceToDevice,
                                    stream);
                    if (me.bank_state == 2)
                        cudaMemcpyAsync(c->slot.xpred + slot * n3, me.bank + n3, n3 * sizeof(double),
                                        cudaMemcpyDeviceToDevice, stream);
                    cudaMemcpyAsync(c->slot.xf_prev + (size_t)slot * H * 12, me.bank + 2 * n3, H * 12 * sizeof(double),
                                    cudaMemcpyDeviceToDevice, stream);
                    c->warm_kind[slot] = 1;
                    c->xpred_valid[slot] = me.bank_state == 2;
                }
                cudaMemcpyAsync(me.ctx->slot.xf + (size_t)slot * H * 12, r.xf.data(), H * 12 * sizeof(double),
                                cudaMemcpyHostToDevice, stream);
                it = queue.erase(it);
            }
        }
        std::vector<Group> gs;
        for (MeshEntry* mp : ms) {
            MeshEntry& me = *mp;
            bool busy = false;
            for (int b = 0; b < me.cap; ++b) busy |= me.slot_req[b] != 0;
            if (busy) {
                me.ctx->prof.reset();
                gs.push_back(Group{me.ctx, me.cap, me.ph.data()});
            }
        }
        if (gs.empty()) continue;
        mfem_status st = advance(gs);
        {
            std::lock_guard<std::mutex> lk(mu);   // counters and err are read by other threads
            steps++;
            for (auto& g : gs) pcg_launches += g.ctx->prof.pcg_launches;
            if (st != MFEM_OK) err = gs[0].ctx->err;
        }
        if (st != MFEM_OK) {
            fail_all_busy(st);
            continue;
        }
        // completion
        for (MeshEntry* mp : ms) {
            MeshEntry& me = *mp;
            for (int b = 0; b < me.cap; ++b) {
                if (!me.slot_req[b] || me.ph[b].active || me.ph[b].need_init) continue;
                mfem_ctx* c = me.ctx;
                ElemArgs a = elem_args(c);
                const size_t n = c->plan.n;
                a.slot.x += (size_t)b * n * 3;
                double* out = nullptr;
                {
                    std::lock_guard<std::mutex> lk(mu);
                    out = reqs[me.slot_req[b]].out;
                }
                launch_unpermute(a, 1, c->slot.outbuf, stream);
                cudaMemcpyAsync(out, c->slot.outbuf, n * 3 * sizeof(double), cudaMemcpyDeviceToHost, stream);
                cudaError_t e = cudaStreamSynchronize(stream);
                std::lock_guard<std::mutex> lk(mu);
                Request& r = reqs[me.slot_req[b]];
                fill_stats(c, me.ph[b], &r.st);
                r.status = e == cudaSuccess ? me.ph[b].status : MFEM_ECUDA;
                c->warm_kind[b] = 1;   // a WARM-start mesh continues from this solution
                const size_t H = c->plan.H;
                cudaMemcpyAsync(c->slot.xf_prev + (size_t)b * H * 12, c->slot.xf + (size_t)b * H * 12,
                                H * 12 * sizeof(double), cudaMemcpyDeviceToDevice, stream);
                if (me.bank && me.ph[b].status == MFEM_OK) {   // the mesh's latest frame
                    cudaMemcpyAsync(me.bank, c->slot.x + b * n * 3, n * 3 * sizeof(double), cudaMemcpyDeviceToDevice,
                                    stream);
                    if (c->xpred_valid[b])
                        cudaMemcpyAsync(me.bank + n * 3, c->slot.xpred + b * n * 3, n * 3 * sizeof(double),
                                        cudaMemcpyDeviceToDevice, stream);
                    cudaMemcpyAsync(me.bank + 2 * n * 3, c->slot.xf + (size_t)b * H * 12, H * 12 * sizeof(double),
                                    cudaMemcpyDeviceToDevice, stream);
                    me.bank_state = c->xpred_valid[b] ? 2 : 1;
                }
                r.done = true;
                r.t_done = now_s();
                me.slot_req[b] = 0;
                in_use--;
                completed++;
                cv_done.notify_all();
            }
        }
    }
}

extern "C" {

mfem_status mfem_server_create(size_t device_mem_budget, int32_t max_slots, mfem_server** out) {
    if (!out || max_slots < 1) return ctx_fail(nullptr, MFEM_EINVAL, "server needs max_slots >= 1");
    *out = nullptr;
    mfem_server* s = new mfem_server();
    s->budget = device_mem_budget;
    s->max_slots = max_slots;
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return ctx_fail(nullptr, MFEM_ECUDA, "server stream");
    }
    s->worker = std::thread([s] { s->run(); });
    s->started = true;
    *out = s;
    return MFEM_OK;
}

mfem_status mfem_server_add(mfem_server* s, mfem_ctx* c, int32_t* mesh_id) {
    if (!s || !c || !mesh_id) return ctx_fail(nullptr, MFEM_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (c->owned_by_server) return ctx_fail(c, MFEM_EINVAL, "context already belongs to a server");
    const size_t per = slot_bytes_for(c, 1);
    int cap = s->max_slots;
    if (s->budget) {
        size_t left = s->budget > s->used ? s->budget - s->used : 0;
        cap = (int)std::min<size_t>((size_t)cap, left / per);
        if (cap < 1) return ctx_fail(c, MFEM_ENOMEM, "one request slot of this mesh exceeds the server budget");
    }
    MeshEntry me;
    me.ctx = c;
    me.cap = cap;
    // everything that can fail comes before the context is changed, so a
    // refused mesh is left as the caller handed it over
    if (c->opt.init == MFEM_INIT_WARM &&
        cudaMalloc((void**)&me.bank, sizeof(double) * ((size_t)c->plan.n * 6 + (size_t)c->plan.H * 12)) != cudaSuccess)
        return ctx_fail(c, MFEM_ENOMEM, "warm-start bank");
    mfem_status st = ensure_slots(c, cap);
    if (st != MFEM_OK) {
        if (me.bank) cudaFree(me.bank);
        return st;
    }
    cudaStreamSynchronize(c->stream);
    c->stream = s->stream;
    if (c->tile_rows == 0) c->tile_rows = 256;   // one tile for every mesh in a shared launch
    if (!s->meshes.empty()) c->tile_rows = s->meshes[0].ctx->tile_rows;
    c->owned_by_server = true;
    me.ph.assign(cap, ProbHost());
    me.slot_req.assign(cap, 0);
    s->used += per * cap;
    s->meshes.push_back(std::move(me));
    *mesh_id = (int32_t)s->meshes.size() - 1;
    return MFEM_OK;
}

mfem_status mfem_server_submit(mfem_server* s, int32_t mesh_id, const double* xf, double* out, uint64_t* ticket) {
    if (!s || !xf || !out || !ticket) return ctx_fail(nullptr, MFEM_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (mesh_id < 0 || mesh_id >= (int)s->meshes.size()) return ctx_fail(nullptr, MFEM_EINVAL, "bad mesh id");
    mfem_ctx* c = s->meshes[mesh_id].ctx;
    const int H = c->plan.H;
    for (int i = 0; i < 12 * H; ++i)
        if (!std::isfinite(xf[i])) return ctx_fail(nullptr, MFEM_EINVAL, "non-finite handle transform");
    for (int h = 0; h < H; ++h) {
        const double* T = xf + 12 * h;
        double e = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double d = T[i] * T[j] + T[4 + i] * T[4 + j] + T[8 + i] * T[8 + j] - (i == j ? 1.0 : 0.0);
                e = std::max(e, std::fabs(d));
            }
        double det = T[0] * (T[5] * T[10] - T[6] * T[9]) - T[1] * (T[4] * T[10] - T[6] * T[8]) +
                     T[2] * (T[4] * T[9] - T[5] * T[8]);
        if (e > 1e-6 || det <= 0.0) return ctx_fail(nullptr, MFEM_EINVAL, "handle transform is not a rotation");
    }
    uint64_t t = s->next_ticket++;
    Request& r = s->reqs[t];
    r.mesh = mesh_id;
    r.xf.assign(xf, xf + 12 * H);
    r.out = out;
    r.t_submit = now_s();
    s->queue.push_back(t);
    *ticket = t;
    s->cv_work.notify_one();
    return MFEM_OK;
}

mfem_status mfem_server_wait(mfem_server* s, uint64_t ticket, int32_t timeout_ms, mfem_stats* stats,
                             double* latency_s) {
    if (!s) return ctx_fail(nullptr, MFEM_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return ctx_fail(nullptr, MFEM_EINVAL, "unknown ticket");
    auto pred = [&] { return s->reqs[ticket].done; };
    if (timeout_ms < 0) s->cv_done.wait(lk, pred);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
        return ctx_fail(nullptr, MFEM_ETIMEOUT, "request still running");
    Request r = s->reqs[ticket];
    s->reqs.erase(ticket);
    if (stats) *stats = r.st;
    if (latency_s) *latency_s = r.t_done - r.t_submit;
    if (r.status != MFEM_OK && !s->err.empty()) ctx_fail(nullptr, (mfem_status)r.status, s->err);
    return (mfem_status)r.status;
}

mfem_status mfem_server_counters(mfem_server* s, int64_t* completed, int64_t* steps, int64_t* pcg_launches,
                                 int32_t* peak_slots) {
    if (!s) return ctx_fail(nullptr, MFEM_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (completed) *completed = s->completed;
    if (steps) *steps = s->steps;
    if (pcg_launches) *pcg_launches = s->pcg_launches;
    if (peak_slots) *peak_slots = s->peak;
    return MFEM_OK;
}

void mfem_server_destroy(mfem_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->queue.clear();
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto& me : s->meshes) {
        if (me.bank) cudaFree(me.bank);
        me.ctx->owned_by_server = false;
        me.ctx->stream = me.ctx->own_stream;
        mfem_destroy(me.ctx);
    }
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
