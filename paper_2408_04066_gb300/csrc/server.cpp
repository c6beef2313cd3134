// Serving: continuous batching of pose solves over resident meshes.
//
// A worker thread owns the GPU work.  Between Newton steps it admits queued
// requests, then advances every admitted request of every mesh by one Newton
// step together -- the element and assembly kernels per slot pool and one
// sequence of PCG iteration launches for all of them -- and hands finished
// requests back.  A request's arithmetic never depends on the others in the
// step (per-problem deterministic reductions), so its result equals the same
// pose solved alone.
//
// Admission by device memory: a mesh's requests run in slot pools -- its own
// context (the first pool, made when the mesh is added) and further contexts
// that share the mesh's device data but own request slots of their own.  A
// request that finds every slot of its mesh busy gets a new pool when the
// device-memory budget has room for it (pools idle for a while are released
// first when it does not), else it waits in the queue; pools that stay idle
// are released, so memory flows to the meshes that have requests.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.h"

using namespace mfem;

namespace {

constexpr int kPoolSlots = 8;           // request slots per pool
constexpr double kPoolIdleRelease = 2.0;   // seconds a pool other than the first stays idle before release
// A WARM request carries the latest solution's nonlinear correction only when
// no handle has turned more than this from that solution's pose (a few frames
// of an animation); further away it takes the co-rotational start alone, which
// under a backlog -- many frames of a mesh admitted at once, all behind the
// latest solution -- measured fewer Newton steps than a stale correction.
constexpr double kWarmMaxTurn = 15.0 * 3.14159265358979323846 / 180.0;

// Largest rotation angle between the handles of two poses ([H][12] each).
double max_turn(const double* a, const double* b, int H) {
    double worst = 0.0;
    for (int h = 0; h < H; ++h) {
        const double* A = a + 12 * h;
        const double* B = b + 12 * h;
        double tr = 0.0;   // trace(Q_a Q_b^T)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) tr += A[4 * i + j] * B[4 * i + j];
        const double c = std::min(1.0, std::max(-1.0, 0.5 * (tr - 1.0)));
        worst = std::max(worst, std::acos(c));
    }
    return worst;
}

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

struct Pool {
    mfem_ctx* ctx = nullptr;   // the mesh's context (first pool) or a slot clone of it
    int cap = 0;
    size_t bytes = 0;          // charged to the budget
    std::vector<ProbHost> ph;
    std::vector<uint64_t> slot_req;  // 0 = free
    int busy = 0;
    double idle_since = 0.0;
};

struct MeshEntry {
    std::vector<std::unique_ptr<Pool>> pools;   // pools[0] is the context handed to mfem_server_add
    // WARM meshes: the mesh's most recent solution (x [n][3], its predictor
    // result [n][3] and its pose [H][12]), copied into the slot of each admitted
    // request, so every request continues from the latest frame solved
    double* bank = nullptr;
    int bank_state = 0;   // 0 none, 1 x and pose, 2 also the predictor result
    std::vector<double> bank_xf;   // host copy of the bank's pose
    mfem_ctx* owner() const { return pools[0]->ctx; }
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
    int64_t completed = 0, steps = 0, pcg_launches = 0, pools_added = 0, pools_released = 0;
    bool stop = false;
    bool started = false;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::thread worker;
    std::string err;

    void run();
    void fail_all_busy(int status);
    bool grow(MeshEntry& me);           // under mu
    bool release_idle(double older_than, const MeshEntry* keep);   // under mu
};

// A new slot pool for `me` if the budget has room (after releasing idle pools
// of other meshes when it has not).  Called under mu by the worker.
bool mfem_server::grow(MeshEntry& me) {
    const int cap = std::min(kPoolSlots, max_slots - in_use);
    if (cap < 1) return false;
    mfem_ctx* owner = me.owner();
    const size_t bytes = slot_bytes_for(owner, cap);
    if (budget && used + bytes > budget && !(release_idle(0.0, &me) && used + bytes <= budget)) return false;
    mfem_status st;
    mfem_ctx* c = ctx_slot_clone(owner, cap, stream, &st);
    if (!c) return false;
    auto p = std::make_unique<Pool>();
    p->ctx = c;
    p->cap = cap;
    p->bytes = bytes;
    p->ph.assign(cap, ProbHost());
    p->slot_req.assign(cap, 0);
    p->idle_since = now_s();
    me.pools.push_back(std::move(p));
    used += bytes;
    pools_added++;
    return true;
}

// Release pools (never a mesh's first) that have been idle at least
// `older_than` seconds; `keep`'s pools are spared.  Returns true if any was.
bool mfem_server::release_idle(double older_than, const MeshEntry* keep) {
    const double t = now_s();
    bool any = false;
    for (auto& me : meshes) {
        if (&me == keep) continue;
        for (size_t i = me.pools.size(); i-- > 1;) {
            Pool& p = *me.pools[i];
            if (p.busy || t - p.idle_since < older_than) continue;
            mfem_destroy(p.ctx);
            used -= p.bytes;
            me.pools.erase(me.pools.begin() + i);
            pools_released++;
            any = true;
        }
    }
    return any;
}

void mfem_server::fail_all_busy(int status) {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& me : meshes)
        for (auto& pp : me.pools) {
            Pool& p = *pp;
            for (int b = 0; b < p.cap; ++b)
                if (p.slot_req[b]) {
                    auto it = reqs.find(p.slot_req[b]);
                    if (it != reqs.end()) {
                        it->second.status = status;
                        it->second.done = true;
                        it->second.t_done = now_s();
                    }
                    p.slot_req[b] = 0;
                    p.ph[b] = ProbHost();
                    in_use--;
                }
            p.busy = 0;
            p.idle_since = now_s();
        }
    cv_done.notify_all();
}

void mfem_server::run() {
    cudaSetDevice(device);
    for (;;) {
        std::vector<Pool*> ps;   // every pool, taken under the lock
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || !queue.empty() || in_use > 0; });
            if (stop && in_use == 0) break;
            // admission: FIFO scan; a mesh that cannot take a request does not block others
            for (auto it = queue.begin(); it != queue.end() && in_use < max_slots;) {
                Request& r = reqs[*it];
                MeshEntry& me = meshes[r.mesh];
                Pool* pool = nullptr;
                int slot = -1;
                for (auto& pp : me.pools) {
                    for (int b = 0; b < pp->cap && slot < 0; ++b)
                        if (!pp->slot_req[b]) slot = b;
                    if (slot >= 0) { pool = pp.get(); break; }
                }
                if (!pool && grow(me)) {
                    pool = me.pools.back().get();
                    slot = 0;
                }
                if (!pool) { ++it; continue; }
                mfem_ctx* c = pool->ctx;
                pool->slot_req[slot] = *it;
                pool->ph[slot] = ProbHost();
                pool->ph[slot].need_init = 1;
                pool->busy++;
                in_use++;
                peak = std::max(peak, in_use);
                const size_t H = c->plan.H;
                if (me.bank_state > 0) {
                    const size_t n3 = (size_t)c->plan.n * 3;
                    cudaMemcpyAsync(c->slot.x + slot * n3, me.bank, n3 * sizeof(double), cudaMemcpyDeviceToDevice,
                                    stream);
                    if (me.bank_state == 2)
                        cudaMemcpyAsync(c->slot.xpred + slot * n3, me.bank + n3, n3 * sizeof(double),
                                        cudaMemcpyDeviceToDevice, stream);
                    cudaMemcpyAsync(c->slot.xf_prev + (size_t)slot * H * 12, me.bank + 2 * n3, H * 12 * sizeof(double),
                                    cudaMemcpyDeviceToDevice, stream);
                    c->warm_kind[slot] = 1;
                    c->xpred_valid[slot] = me.bank_state == 2 &&
                                           max_turn(r.xf.data(), me.bank_xf.data(), (int)H) <= kWarmMaxTurn;
                }
                cudaMemcpyAsync(c->slot.xf + (size_t)slot * H * 12, r.xf.data(), H * 12 * sizeof(double),
                                cudaMemcpyHostToDevice, stream);
                it = queue.erase(it);
            }
            release_idle(kPoolIdleRelease, nullptr);
            for (auto& m : meshes)
                for (auto& pp : m.pools) ps.push_back(pp.get());
        }
        std::vector<Group> gs;
        for (Pool* p : ps)
            if (p->busy) {
                p->ctx->prof.reset();
                gs.push_back(Group{p->ctx, p->cap, p->ph.data()});
            }
        if (gs.empty()) continue;
        mfem_status st = advance(gs, true);
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
        for (Pool* pp : ps) {
            Pool& pool = *pp;
            if (!pool.busy) continue;
            for (int b = 0; b < pool.cap; ++b) {
                if (!pool.slot_req[b] || pool.ph[b].active || pool.ph[b].need_init) continue;
                mfem_ctx* c = pool.ctx;
                ElemArgs a = elem_args(c);
                const size_t n = c->plan.n;
                a.slot.x += (size_t)b * n * 3;
                double* out = nullptr;
                MeshEntry* me = nullptr;
                {
                    std::lock_guard<std::mutex> lk(mu);
                    const Request& r = reqs[pool.slot_req[b]];
                    out = r.out;
                    me = &meshes[r.mesh];
                }
                launch_unpermute(a, 1, c->slot.outbuf, stream);
                cudaMemcpyAsync(out, c->slot.outbuf, n * 3 * sizeof(double), cudaMemcpyDeviceToHost, stream);
                cudaError_t e = cudaStreamSynchronize(stream);
                std::lock_guard<std::mutex> lk(mu);
                Request& r = reqs[pool.slot_req[b]];
                fill_stats(c, pool.ph[b], &r.st);
                r.status = e == cudaSuccess ? pool.ph[b].status : MFEM_ECUDA;
                c->warm_kind[b] = 1;   // a WARM-start mesh continues from this solution
                const size_t H = c->plan.H;
                cudaMemcpyAsync(c->slot.xf_prev + (size_t)b * H * 12, c->slot.xf + (size_t)b * H * 12,
                                H * 12 * sizeof(double), cudaMemcpyDeviceToDevice, stream);
                if (me->bank && pool.ph[b].status == MFEM_OK) {   // the mesh's latest frame
                    cudaMemcpyAsync(me->bank, c->slot.x + b * n * 3, n * 3 * sizeof(double), cudaMemcpyDeviceToDevice,
                                    stream);
                    if (c->xpred_valid[b])
                        cudaMemcpyAsync(me->bank + n * 3, c->slot.xpred + b * n * 3, n * 3 * sizeof(double),
                                        cudaMemcpyDeviceToDevice, stream);
                    cudaMemcpyAsync(me->bank + 2 * n * 3, c->slot.xf + (size_t)b * H * 12, H * 12 * sizeof(double),
                                    cudaMemcpyDeviceToDevice, stream);
                    me->bank_state = c->xpred_valid[b] ? 2 : 1;
                    me->bank_xf = r.xf;
                }
                r.done = true;
                r.t_done = now_s();
                pool.slot_req[b] = 0;
                pool.busy--;
                if (!pool.busy) pool.idle_since = r.t_done;
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
    // the mesh's first slot pool: its own context, kPoolSlots slots or what the budget holds
    const size_t per = slot_bytes_for(c, 1);
    const size_t bank_bytes = c->opt.init == MFEM_INIT_WARM
                                  ? sizeof(double) * ((size_t)c->plan.n * 6 + (size_t)c->plan.H * 12) : 0;
    int cap = std::min(s->max_slots, kPoolSlots);
    if (s->budget) {
        size_t left = s->budget > s->used + bank_bytes ? s->budget - s->used - bank_bytes : 0;
        cap = (int)std::min<size_t>((size_t)cap, left / per);
        if (cap < 1) return ctx_fail(c, MFEM_ENOMEM, "one request slot of this mesh exceeds the server budget");
    }
    MeshEntry me;
    // everything that can fail comes before the context is changed, so a
    // refused mesh is left as the caller handed it over
    if (bank_bytes && cudaMalloc((void**)&me.bank, bank_bytes) != cudaSuccess)
        return ctx_fail(c, MFEM_ENOMEM, "warm-start bank");
    mfem_status st = ensure_slots(c, cap);
    if (st != MFEM_OK) {
        if (me.bank) cudaFree(me.bank);
        return st;
    }
    cudaStreamSynchronize(c->stream);
    c->stream = s->stream;
    if (c->tile_rows == 0) c->tile_rows = 256;   // one SpMV shape for every mesh in a shared launch
    if (c->spmv_split == 0) c->spmv_split = 1;
    if (!s->meshes.empty()) {
        c->tile_rows = s->meshes[0].owner()->tile_rows;
        c->spmv_split = s->meshes[0].owner()->spmv_split;
    }
    c->owned_by_server = true;
    auto p = std::make_unique<Pool>();
    p->ctx = c;
    p->cap = cap;
    p->bytes = per * cap + bank_bytes;
    p->ph.assign(cap, ProbHost());
    p->slot_req.assign(cap, 0);
    p->idle_since = now_s();
    me.pools.push_back(std::move(p));
    s->used += per * cap + bank_bytes;
    s->meshes.push_back(std::move(me));
    *mesh_id = (int32_t)s->meshes.size() - 1;
    return MFEM_OK;
}

mfem_status mfem_server_submit(mfem_server* s, int32_t mesh_id, const double* xf, double* out, uint64_t* ticket) {
    if (!s || !xf || !out || !ticket) return ctx_fail(nullptr, MFEM_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (mesh_id < 0 || mesh_id >= (int)s->meshes.size()) return ctx_fail(nullptr, MFEM_EINVAL, "bad mesh id");
    mfem_ctx* c = s->meshes[mesh_id].owner();
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
                                 int32_t* peak_slots, int64_t* pools_added, int64_t* pools_released,
                                 int64_t* device_bytes) {
    if (!s) return ctx_fail(nullptr, MFEM_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (completed) *completed = s->completed;
    if (steps) *steps = s->steps;
    if (pcg_launches) *pcg_launches = s->pcg_launches;
    if (peak_slots) *peak_slots = s->peak;
    if (pools_added) *pools_added = s->pools_added;
    if (pools_released) *pools_released = s->pools_released;
    if (device_bytes) *device_bytes = (int64_t)s->used;
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
        for (size_t i = me.pools.size(); i-- > 1;) mfem_destroy(me.pools[i]->ctx);   // slot pools first
        mfem_ctx* c = me.owner();
        c->owned_by_server = false;
        c->stream = c->own_stream;
        mfem_destroy(c);
    }
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
