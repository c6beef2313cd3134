// Solver engine: context creation (device upload of the planned mesh), the
// Newton driver (paper Algorithm 1 and the Newton form of Eq. 12), and the C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"

namespace {
thread_local std::string g_thread_err = "no error";

constexpr double kLsC = 1.0e-4;      // Armijo constant
constexpr int kLsMax = 20;           // halvings
constexpr double kLsNoise = 1.0e-10; // predicted decrease below this * |E|: take the step
constexpr int kPcgTiles[3] = {64, 128, 256};   // PCG rows per block the autotuner times
constexpr int kPcgChunk = 16;                   // PCG iterations enqueued between convergence checks (no history)
constexpr int kPcgChunkMin = 16, kPcgChunkMax = 64;   // bounds of a predicted chunk (multiples of 8)
constexpr int kPcgHistSteps = 16;               // Newton steps remembered per slot
constexpr double kPredTol = 3e-3;   // PCG target of the co-rotational predictor step (at most cg_tol)
constexpr double kEwGamma = 0.9;    // forcing rule where the Newton model is trusted (see advance)
constexpr double kEwMin = 1e-4;     // tightest PCG target that rule sets (well above FP32 PCG's floor)
}  // namespace

namespace mfem {

mfem_status ctx_fail(mfem_ctx* c, mfem_status s, const std::string& msg) {
    if (c) c->err = msg;
    g_thread_err = msg;
    return s;
}

mfem_status cuda_check(mfem_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return MFEM_OK;
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    return ctx_fail(c, e == cudaErrorMemoryAllocation ? MFEM_ENOMEM : MFEM_ECUDA, msg);
}

#define CK(expr)                                                       \
    do {                                                               \
        mfem_status _s = cuda_check(c, (expr), #expr);                 \
        if (_s != MFEM_OK) return _s;                                  \
    } while (0)

int Profiler::begin(int k, cudaStream_t s) {
    if (used + 1 >= (int)ev.size() / 2) return -1;
    int idx = used++;
    kind.push_back(k);
    cudaEventRecord(ev[2 * idx], s);
    return idx;
}

void Profiler::end(int idx, cudaStream_t s) {
    if (idx >= 0) cudaEventRecord(ev[2 * idx + 1], s);
}

ElemArgs elem_args(const mfem_ctx* c) {
    ElemArgs a;
    a.mesh = c->mesh;
    a.slot = c->slot;
    a.model = c->model;
    a.constraint = c->opt.constraint;
    a.ks = c->opt.k_s;
    a.fext = c->fext_dev;
    a.fext_stride = c->fext_sets > 1 ? 3 * (int64_t)c->plan.n : 0;
    a.rot_polar = c->opt.rotation == MFEM_ROT_POLAR ? 1 : 0;
    a.f32_forces = c->slot.prec == 1 && c->opt.newton_tol >= kF32ForcesTol ? 1 : 0;
    a.ff_elem = a.f32_forces && !a.rot_polar && c->slot.xff && c->slot.qff && c->mesh.Dminv_lo && c->mesh.mulam_ff
                    ? 1
                    : 0;
    return a;
}

// Newton steps are line-searched on E when E is not quadratic in x: SNH, and
// every model when the rotations follow F (polar-rotation mode).
bool line_search(const mfem_ctx* c) { return c->model == MFEM_SNH || c->opt.rotation == MFEM_ROT_POLAR; }

namespace {

template <typename U>
mfem_status upload(mfem_ctx* c, U** dst, const U* src, size_t count) {
    *dst = nullptr;
    if (count == 0) return MFEM_OK;
    CK(cudaMalloc((void**)dst, count * sizeof(U)));
    c->mesh_bytes += count * sizeof(U);
    CK(cudaMemcpy(*dst, src, count * sizeof(U), cudaMemcpyHostToDevice));
    return MFEM_OK;
}

void free_slots(mfem_ctx* c) {
    SlotDev& S = c->slot;
    void* ptrs[] = {S.xf, S.xf_prev, S.xpred, S.dcorr, S.tol2, S.coarse_on, S.rcp, S.ec, S.rcs, S.aggq, S.bsplit,
                    S.x, S.xff, S.qff, S.xprev, S.xp,
                    S.g, S.ge, S.Ke, S.val, S.dinv, S.vec, S.part, S.sc, S.active, S.alpha, S.outbuf};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    int prec = S.prec;
    S = SlotDev();
    S.prec = prec;
    c->slot_bytes = 0;
}

// slices of the coarse product (ec partials per problem)
size_t coarse_ks(const mfem_ctx* c) { return ((size_t)c->mesh.coarse_n + kCoarseKC - 1) / kCoarseKC; }

int part_tiles_for(const mfem_ctx* c) {
    int a = (c->plan.n + 31) / 32, b = (c->plan.m + kTetTile - 1) / kTetTile;
    return std::max(std::max(a, b), 1);
}

size_t bytes_per_slot(const mfem_ctx* c) {
    const size_t n = c->plan.n, m = c->plan.m, H = c->plan.H;
    const size_t kt = c->slot.prec == 1 ? 4 : 8;
    const size_t slots = (size_t)c->plan.slice_ptr.back();
    return H * 12 * 8 + 4 * n * 3 * 8 + (kt == 4 ? n * 3 * 8 + H * 9 * 8 : 0) + m * 12 * 8 + m * kKe * kt + slots * 9 * kt +
           9 * npad32((int)n) * kt +
           kVecStride * npad32((int)n) * kt + (size_t)part_tiles_for(c) * 4 * 8 + sizeof(ProbScal) + 4 + 8 + 8 +
           H * 12 * 8 + (c->opt.init == MFEM_INIT_WARM ? 2 * n * 3 * 8 : 0) + 4 + (line_search(c) ? n * 3 * 8 : 0) +
           (c->mesh.coarse_n > 0 ? ((n + 255) / 256) * 24 * 4 + (coarse_ks(c) + 1) * c->mesh.coarse_n * 4 + 128 +
                                        (size_t)c->mesh.n_agg * 9 * 4 +
                                        coarse_b_bytes(c->mesh.coarse_n, kCoarseGroupSlots) / kCoarseGroupSlots
                                  : 0);
}

mfem_status alloc_slots(mfem_ctx* c, int B) {
    SlotDev& S = c->slot;
    const size_t n = c->plan.n, m = c->plan.m, H = c->plan.H;
    const size_t kt = S.prec == 1 ? 4 : 8;
    const size_t slots = (size_t)c->plan.slice_ptr.back();
    S.part_tiles = part_tiles_for(c);
    auto al = [&](void** p, size_t bytes) -> mfem_status {
        CK(cudaMalloc(p, std::max<size_t>(bytes, 16)));
        c->slot_bytes += bytes;
        return MFEM_OK;
    };
    mfem_status st;
#define AL(ptr, bytes) \
    if ((st = al((void**)&(ptr), (bytes))) != MFEM_OK) return st;
    AL(S.xf, B * H * 12 * 8);
    AL(S.xf_prev, B * H * 12 * 8);
    if (c->opt.init == MFEM_INIT_WARM) {
        AL(S.xpred, B * n * 3 * 8);
        AL(S.dcorr, B * n * 3 * 8);
    }
    AL(S.x, B * n * 3 * 8);
    if (S.prec == 1) {
        AL(S.xff, B * n * 3 * sizeof(float2));
        AL(S.qff, B * H * 9 * sizeof(float2));
    }
    if (line_search(c)) AL(S.xprev, B * n * 3 * 8);
    AL(S.xp, B * n * 3 * 8);
    AL(S.g, B * n * 3 * 8);
    AL(S.outbuf, B * n * 3 * 8);
    AL(S.ge, B * m * 12 * 8);
    AL(S.Ke, (B * m * kKe + kKePad) * kt);
    AL(S.val, B * slots * 9 * kt);
    AL(S.dinv, B * 9 * npad32((int)n) * kt);
    AL(S.vec, B * kVecStride * npad32((int)n) * kt);
    AL(S.part, B * (size_t)S.part_tiles * 4 * 8);
    AL(S.sc, B * sizeof(ProbScal));
    AL(S.active, B * sizeof(int));
    AL(S.alpha, B * sizeof(double));
    AL(S.tol2, B * sizeof(double));
    AL(S.coarse_on, B * sizeof(int));
    if (c->mesh.coarse_n > 0) {
        S.rcp_stride = (((size_t)n + 255) / 256) * (256 / kCoarseRows) * 6;
        AL(S.rcp, B * S.rcp_stride * sizeof(float));
        AL(S.ec, B * coarse_ks(c) * c->mesh.coarse_n * sizeof(float));
        S.rcs_stride = ((size_t)c->mesh.coarse_n + 31) & ~(size_t)31;
        AL(S.rcs, B * S.rcs_stride * sizeof(float));
        AL(S.aggq, B * (size_t)c->mesh.n_agg * 9 * sizeof(float));
        AL(S.bsplit, coarse_b_bytes(c->mesh.coarse_n, B));
        CK(cudaMemset(S.bsplit, 0, coarse_b_bytes(c->mesh.coarse_n, B)));   // columns past N stay zero
    }
#undef AL
    CK(cudaMemset(S.sc, 0, B * sizeof(ProbScal)));
    CK(cudaMemset(S.val, 0, B * slots * 9 * kt));   // padding slots stay zero
    CK(cudaMemset(S.vec, 0, B * kVecStride * npad32((int)n) * kt));
    S.cap = B;
    // every slot starts at the rest shape (the WARM start without history)
    for (int b = 0; b < B; ++b)
        CK(cudaMemcpy(S.x + (size_t)b * n * 3, c->mesh.X, n * 3 * 8, cudaMemcpyDeviceToDevice));
    c->warm_kind.assign(B, 0);
    c->xpred_valid.assign(B, 0);
    c->pcg_hist.assign((size_t)B * kPcgHistSteps, 0);
    // pinned host staging
    if (c->sc_host) cudaFreeHost(c->sc_host);
    if (c->active_host) cudaFreeHost(c->active_host);
    if (c->alpha_host) cudaFreeHost(c->alpha_host);
    if (c->alpha_ring) cudaFreeHost(c->alpha_ring);
    CK(cudaMallocHost((void**)&c->sc_host, B * sizeof(ProbScal)));
    CK(cudaMallocHost((void**)&c->active_host, (size_t)kStageRing * B * sizeof(int)));
    CK(cudaMallocHost((void**)&c->alpha_host, B * sizeof(double)));
    CK(cudaMallocHost((void**)&c->alpha_ring, (size_t)kStageRing * B * sizeof(double)));
    c->ring_pos = 0;
    size_t dcap = 2 * B * std::max(sizeof(PcgDesc<float>), sizeof(PcgDesc<double>));
    if (dcap > c->descs_cap) {
        if (c->descs_dev) cudaFree(c->descs_dev);
        if (c->descs_host) cudaFreeHost(c->descs_host);
        CK(cudaMalloc(&c->descs_dev, dcap));
        CK(cudaMallocHost(&c->descs_host, dcap));
        c->descs_cap = dcap;
    }
    return MFEM_OK;
}

}  // namespace

size_t slot_bytes_for(const mfem_ctx* c, int B) { return bytes_per_slot(c) * (size_t)B; }

mfem_status ensure_slots(mfem_ctx* c, int B) {
    if (B <= c->slot.cap) return MFEM_OK;
    free_slots(c);
    return alloc_slots(c, B);
}

void begin_profile(mfem_ctx* c) {
    c->prof.reset();
    cudaEventRecord(c->prof.start, c->stream);
}

void end_profile(mfem_ctx* c) {
    cudaEventRecord(c->prof.stop, c->stream);
    cudaEventSynchronize(c->prof.stop);
    mfem_profile& P = c->last_profile;
    P = mfem_profile();
    P.kernel_launches = c->prof.launches;
    P.pcg_launches = c->prof.pcg_launches;
    P.element_launches = c->prof.element_launches;
    P.pcg_bytes = c->prof.pcg_bytes;
    P.element_bytes = c->prof.element_bytes;
    P.element_updates = c->prof.element_updates;
    P.coarse_dof = c->mesh.coarse_n;
    P.coarse_launches = c->prof.coarse_launches;
    P.coarse_tc = c->mesh.coarse_n > 0 && c->mesh.coarse_tc ? 1 : 0;
    P.pcg_iters = c->prof.pcg_iters;
    P.tile_rows = c->tile_rows;
    P.spmv_split = c->spmv_split;
    P.grid_blocks = c->grid_blocks;
    for (int i = 0; i < c->prof.used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->prof.ev[2 * i], c->prof.ev[2 * i + 1]) != cudaSuccess) continue;
        switch (c->prof.kind[i]) {
            case 0: P.element_ms += ms; break;
            case 1: P.assemble_ms += ms; break;
            case 2: P.pcg_ms += ms; break;
            case 3: P.linesearch_ms += ms; break;
            default: break;
        }
    }
    float tot = 0.f;
    cudaEventElapsedTime(&tot, c->prof.start, c->prof.stop);
    P.total_ms = tot;
    cudaGetLastError();
}

namespace {

// Algorithmic bytes of one PCG iteration of one problem (each datum crossing
// HBM once, 3-vectors counted as 3 elements): k_pcg_spmv reads the matrix
// values and column ids and the row's u and r, and writes w (the neighbours' u
// are the same vector); k_pcg_update reads u, w, p, s, dx, r and the 9-element
// D^-1 and writes p, s, dx, r and zb, and u under block Jacobi.  With the
// two-level preconditioner the update reads the aggregate offset (16) for the
// restriction and the correction reads zb and the offset and writes u (per
// row); the coarse product's A_c^{-1} is counted per launch in run_pcg.
double pcg_bytes_per_iter(const mfem_ctx* c, bool coarse) {
    const double kt = c->slot.prec == 1 ? 4.0 : 8.0;
    const double nnzb = (double)c->plan.nnz_blocks, n = c->plan.n;
    double b = nnzb * (9.0 * kt + 4.0) + n * (3.0 * 3.0 * kt) + n * (6.0 * 3.0 * kt + 9.0 * kt + 5.0 * 3.0 * kt);
    b += coarse ? n * (16.0 + 3.0 * kt + 16.0 + 3.0 * kt) : n * 3.0 * kt;
    return b;
}

// Element kernel: static tet data (idx 16, D_m^-1 72, W 8, cluster 4, mu/lam 16),
// vertex positions once (24 n), element forces (96) and blocks (90 kt) written.
double element_bytes(const mfem_ctx* c) {
    const double kt = c->slot.prec == 1 ? 4.0 : 8.0;
    return (double)c->plan.m * (16 + 72 + 8 + 4 + 16 + 96 + kKe * kt) + 24.0 * c->plan.n;
}

template <typename T>
void build_descs(std::vector<Group>& gs, int tile, int prec, std::vector<PcgDesc<T>>& out, int& units, int& units_u,
                 std::vector<CoarseJob>* jobs = nullptr) {
    units = 0;
    units_u = 0;
    for (auto& g : gs) {
        mfem_ctx* c = g.ctx;
        if (c->slot.prec != prec) continue;
        const int first = (int)out.size();
        bool any_coarse = false;
        for (int b = 0; b < g.B; ++b) any_coarse |= g.ph[b].active && g.ph[b].in_pcg && g.ph[b].coarse;
        const bool tc = c->mesh.coarse_tc && c->mesh.Abf && c->slot.bsplit;
        if (jobs && any_coarse && c->mesh.coarse_n > 0)
            jobs->push_back(CoarseJob{c->mesh.Ainv, tc ? c->mesh.Abf : nullptr, c->slot.bsplit, c->mesh.coarse_err, c,
                                      c->mesh.coarse_n, first, 0, c->plan.agg_size / kCoarseRows, c->slot.cap});
        const int n = c->plan.n;
        const size_t slots = (size_t)c->plan.slice_ptr.back();
        for (int b = 0; b < g.B; ++b) {
            if (!g.ph[b].active || !g.ph[b].in_pcg) continue;
            PcgDesc<T> d;
            d.slice_ptr = c->mesh.slice_ptr;
            d.col = c->mesh.col;
            d.val = (const T*)c->slot.val + (size_t)b * slots * 9;
            d.dinv = (const T*)c->slot.dinv + (size_t)b * 9 * npad32(n);
            const size_t np = npad32(n);
            T* v = (T*)c->slot.vec + (size_t)b * kVecStride * np;
            d.nb = v + kOffNB * np;
            d.rec = v + kOffRec * np;
            d.part = c->slot.part + (size_t)b * c->slot.part_tiles * 4;
            d.sc = c->slot.sc + b;
            d.n_rows = n;
            d.n_tiles = (n + tile - 1) / tile;
            d.unit_begin = units;
            d.n_tiles_u = (n + kRowTileU - 1) / kRowTileU;
            d.unit_begin_u = units_u;
            d.coarse = g.ph[b].coarse && c->mesh.coarse_n > 0;
            d.crel = c->mesh.crel;
            d.aggq = c->slot.aggq ? c->slot.aggq + (size_t)b * c->mesh.n_agg * 9 : nullptr;
            d.rcp = c->slot.rcp ? c->slot.rcp + (size_t)b * c->slot.rcp_stride : nullptr;
            d.ec = c->slot.ec ? c->slot.ec + (size_t)b * coarse_ks(c) * c->mesh.coarse_n : nullptr;
            d.rcs = c->slot.rcs ? c->slot.rcs + (size_t)b * c->slot.rcs_stride : nullptr;
            d.rc = c->plan.agg_size == kCoarseRows ? d.rcp : d.rcs;
            d.ctc = d.coarse && tc;
            uint16_t* bg = c->slot.bsplit ? c->slot.bsplit + (size_t)(b / kCoarseGroupSlots) *
                                                                 coarse_chunks(c->mesh.coarse_n) * kCoarseBChunk
                                          : nullptr;
            d.bunit = d.ctc && c->plan.agg_size == kCoarseRows ? bg : nullptr;
            d.bagg = d.ctc && c->plan.agg_size != kCoarseRows ? bg : nullptr;
            d.bslot = b;
            d.agg_shift = c->mesh.agg_shift;
            d.coarse_n = c->mesh.coarse_n;
            units += d.n_tiles;
            units_u += d.n_tiles_u;
            out.push_back(d);
        }
        if (jobs && !jobs->empty() && jobs->back().d0 == first && jobs->back().key == c)
            jobs->back().nd = (int)out.size() - first;
    }
}

// Next free staging region; waits for the stream only when the ring is used up.
mfem_status next_stage(mfem_ctx* c, int& pos) {
    if (c->ring_pos >= kStageRing) {
        CK(cudaStreamSynchronize(c->stream));
        c->ring_pos = 0;
    }
    pos = c->ring_pos++;
    return MFEM_OK;
}

mfem_status upload_active(mfem_ctx* c, int B, const std::vector<int>& flags) {
    int pos = 0;
    mfem_status st = next_stage(c, pos);
    if (st != MFEM_OK) return st;
    int* h = c->active_host + (size_t)pos * c->slot.cap;
    for (int b = 0; b < B; ++b) h[b] = flags[b];
    CK(cudaMemcpyAsync(c->slot.active, h, B * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    return MFEM_OK;
}

// B doubles -> device through a staging region that is not rewritten before
// the copy has run
mfem_status upload_doubles(mfem_ctx* c, int B, const double* v, double* dst) {
    int pos = 0;
    mfem_status st = next_stage(c, pos);
    if (st != MFEM_OK) return st;
    double* h = c->alpha_ring + (size_t)pos * c->slot.cap;
    for (int b = 0; b < B; ++b) h[b] = v[b];
    CK(cudaMemcpyAsync(dst, h, B * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    return MFEM_OK;
}

mfem_status upload_alpha(mfem_ctx* c, int B) { return upload_doubles(c, B, c->alpha_host, c->slot.alpha); }

mfem_status upload_ints(mfem_ctx* c, int B, const int* v, int* dst) {
    int pos = 0;
    mfem_status st = next_stage(c, pos);
    if (st != MFEM_OK) return st;
    int* h = c->active_host + (size_t)pos * c->slot.cap;
    for (int b = 0; b < B; ++b) h[b] = v[b];
    CK(cudaMemcpyAsync(dst, h, B * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    return MFEM_OK;
}

void synced(std::vector<Group>& gs) {
    for (auto& g : gs) g.ctx->ring_pos = 0;
}

mfem_status read_scalars(mfem_ctx* c, int B) {
    CK(cudaMemcpyAsync(c->sc_host, c->slot.sc, B * sizeof(ProbScal), cudaMemcpyDeviceToHost, c->stream));
    if (c->mesh.coarse_err && c->cerr_host)
        CK(cudaMemcpyAsync(c->cerr_host, c->mesh.coarse_err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    return MFEM_OK;
}

// Enqueue PCG for every active problem of precision `prec` in every group: the
// descriptor table is uploaded once, then chunks of kPcgChunk iterations are
// enqueued and the problem states read back after each chunk (max_iters > 0:
// exactly that many iterations, no checks -- used by the autotuner).
// One chunk of PCG iterations: replayed from a CUDA graph captured the first
// time these launch parameters occur (the descriptor table lives at a fixed
// device address; only its contents change), else launched directly.
template <typename T>
mfem_status launch_chunk(mfem_ctx* c, const PcgDesc<T>* dst, int nd, int units, int units_u, int tile, int split,
                         int n_it, const std::vector<CoarseJob>& jobs) {
    const int nj = (int)jobs.size();
    if (c->opt.launch == MFEM_LAUNCH_GRAPH && !c->graphs_off) {
        char buf[96];
        snprintf(buf, sizeof buf, "%d %p %d %d %d %d %d %d", (int)sizeof(T), (const void*)dst, nd, units, units_u, tile,
                 split, n_it);
        std::string key(buf);
        for (const auto& j : jobs) {
            snprintf(buf, sizeof buf, " %p %d %d %d %d %d", j.key, j.Abf ? 1 : 0, j.N, j.d0, j.nd, j.agg_units);
            key += buf;
        }
        auto it = c->graphs.find(key);
        if (it == c->graphs.end()) {
            if (c->graphs.size() >= 256) {   // bounded cache
                for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
                c->graphs.clear();
            }
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ex = nullptr;
            bool ok = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                const cudaError_t e1 = launch_pcg_iters<T>(dst, nd, units, units_u, tile, split, n_it, jobs.data(), nj, c->stream);
                const cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
                ok = e1 == cudaSuccess && e2 == cudaSuccess && g && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
            }
            if (g) cudaGraphDestroy(g);
            if (!ok) {   // keep to direct launches from now on
                cudaGetLastError();
                c->graphs_off = true;
                CK(launch_pcg_iters<T>(dst, nd, units, units_u, tile, split, n_it, jobs.data(), nj, c->stream));
                return MFEM_OK;
            }
            it = c->graphs.emplace(key, ex).first;
        }
        CK(cudaGraphLaunch(it->second, c->stream));
        return MFEM_OK;
    }
    CK(launch_pcg_iters<T>(dst, nd, units, units_u, tile, split, n_it, jobs.data(), nj, c->stream));
    return MFEM_OK;
}

template <typename T>
mfem_status run_pcg(mfem_ctx* c0, std::vector<Group>& gs, int prec, int tile, int split, int max_iters, bool count,
                    bool one_chunk = false, bool slopes = false, bool per_request = false) {
    mfem_ctx* c = c0;
    std::vector<PcgDesc<T>> d;
    std::vector<CoarseJob> jobs;
    int units = 0, units_u = 0;
    build_descs<T>(gs, tile, prec, d, units, units_u, &jobs);
    if (d.empty()) return MFEM_OK;
    const int nj = (int)jobs.size();
    double coarse_bytes = 0.0;   // A_c^{-1} streamed once per iteration per mesh
    for (const auto& j : jobs) coarse_bytes += j.Abf ? 2.0 * j.N * j.N : 4.0 * j.N * coarse_ld(j.N);
    const size_t bytes = d.size() * sizeof(PcgDesc<T>);
    if (2 * bytes > c->descs_cap) {   // grow: wait until no copy reads the old buffers
        CK(cudaStreamSynchronize(c->stream));
        if (c->descs_dev) cudaFree(c->descs_dev);
        if (c->descs_host) cudaFreeHost(c->descs_host);
        CK(cudaMalloc(&c->descs_dev, 2 * bytes));
        CK(cudaMallocHost(&c->descs_host, 2 * bytes));
        c->descs_cap = 2 * bytes;
    }
    // each precision class has its own half, so two tables of one step never
    // share a staging region; a step starts only after the previous one synced
    const size_t off = (size_t)prec * (c->descs_cap / 2);
    char* hst = (char*)c->descs_host + off;
    const PcgDesc<T>* dst = (const PcgDesc<T>*)((char*)c->descs_dev + off);
    std::memcpy(hst, d.data(), bytes);
    CK(cudaMemcpyAsync((void*)dst, hst, bytes, cudaMemcpyHostToDevice, c->stream));
    c->grid_blocks = units;
    if (max_iters > 0) {
        CK(launch_pcg_iters<T>(dst, (int)d.size(), units, units_u, tile, split, max_iters, jobs.data(), nj,
                               c->stream));
        return MFEM_OK;
    }
    int cap = 0;
    for (auto& g : gs)
        if (g.ctx->slot.prec == prec) cap = std::max(cap, g.ctx->opt.cg_max);
    // one chunk per scheduling round, from each slot's last solve of the same
    // Newton step less what this solve has run (kPcgChunk without history):
    // for a batch call, as many iterations as the last problem of the table is
    // expected to need (at most kPcgChunkMax), so that a round usually ends
    // with every solve done -- a round costs a host round trip (~160 us on the
    // 200k figure) and the batch ends with its last problem (fixed chunks of
    // 16 / 24 / 32 / 48 / 64 gave 471 / 480 / 449 / 490 / 463 frames/s, this
    // rule 489); for served requests, which complete one by one, as many as
    // the first problem is expected to need, at least kPcgChunkMin (served
    // mix at 70% load: p50 37 ms against 57 with the batch rule)
    int chunk = kPcgChunk;
    if (one_chunk) {
        int best = per_request ? kPcgChunkMax : 0;
        for (auto& g : gs) {
            if (g.ctx->slot.prec != prec) continue;
            for (int b = 0; b < g.B; ++b) {
                const ProbHost& p = g.ph[b];
                if (!p.active || !p.in_pcg) continue;
                const int h = g.ctx->pcg_hist[(size_t)b * kPcgHistSteps + std::min(p.it, kPcgHistSteps - 1)];
                const int need = h > 0 ? h - p.pcg_launched : kPcgChunk;
                best = per_request ? std::min(best, need) : std::max(best, need);
            }
        }
        chunk = std::min(kPcgChunkMax, std::max(per_request ? kPcgChunkMin : 8, (best + 7) / 8 * 8));
    }
    for (int done = 0; done < cap; done += chunk) {
        const int n_it = std::min(chunk, cap - done);
        if (one_chunk && done > 0) break;
        if (one_chunk)
            for (auto& g : gs)
                if (g.ctx->slot.prec == prec)
                    for (int b = 0; b < g.B; ++b)
                        if (g.ph[b].active && g.ph[b].in_pcg) g.ph[b].pcg_launched += n_it;
        int pe = count ? c->prof.begin(2, c->stream) : -1;
        mfem_status lst = launch_chunk<T>(c, dst, (int)d.size(), units, units_u, tile, split, n_it, jobs);
        if (lst != MFEM_OK) return lst;
        if (count) {
            c->prof.end(pe, c->stream);
            int cl = nj;   // coarse kernels: per job the product (fused with the correction on the tensor cores) ...
            bool cuda_core = false;
            for (const auto& j : jobs) {
                cl += j.agg_units > 1;   // ... the per-aggregate sums of larger aggregates ...
                cuda_core |= j.Abf == nullptr;
            }
            cl += cuda_core ? 1 : 0;   // ... and the correction after CUDA-core products
            c->prof.launches += (2 + cl) * n_it;
            c->prof.pcg_launches += 2 * n_it;
            c->prof.coarse_launches += cl * n_it;
            c->prof.pcg_bytes += coarse_bytes * n_it;
        }
        // slopes g.dx of every problem inside PCG, read back with the PCG
        // states: a problem whose PCG ended in this chunk has its line-search
        // slope without another round trip (the others' are not used)
        if (slopes)
            for (auto& g : gs) {
                mfem_ctx* gc = g.ctx;
                if (gc->slot.prec != prec || !line_search(gc)) continue;
                std::vector<int> m(g.B, 0);
                bool any_ls = false;
                for (int b = 0; b < g.B; ++b) {
                    m[b] = g.ph[b].active && g.ph[b].in_pcg && !g.ph[b].pred;
                    any_ls |= m[b] != 0;
                }
                if (!any_ls) continue;
                mfem_status st = upload_active(gc, g.B, m);
                if (st != MFEM_OK) return st;
                int pl = gc->prof.begin(3, c->stream);
                launch_slope(elem_args(gc), g.B, c->stream);
                gc->prof.end(pl, c->stream);
                gc->prof.launches++;
            }
        bool any = false;
        for (auto& g : gs)
            if (g.ctx->slot.prec == prec) {
                mfem_status st = read_scalars(g.ctx, g.B);
                if (st != MFEM_OK) return st;
            }
        CK(cudaStreamSynchronize(c->stream));
        synced(gs);
        for (auto& g : gs) {
            if (g.ctx->slot.prec != prec) continue;
            if (g.ctx->cerr_host && *g.ctx->cerr_host)
                return ctx_fail(c, MFEM_ECUDA, "coarse product: a bounded wait in the tensor-core kernel ran out");
            for (int b = 0; b < g.B; ++b)
                if (g.ph[b].active && g.ph[b].in_pcg && g.ctx->sc_host[b].state == kActive) any = true;
        }
        if (!any) break;
    }
    return MFEM_OK;
}

// Pick the SpMV's shape -- rows per block (64, 128, 256) and threads per row
// (1, 2) -- by timing a fixed number of PCG iterations of each candidate on the
// first assembled system (results are discarded; PCG is re-initialised
// afterwards).  A shape fixed by the options is not searched.
// MFEM_AUTOTUNE_CACHE names a file of earlier picks ("key tile split" lines).
mfem_status autotune_tile(mfem_ctx* c, std::vector<Group>& gs) {
    const char* cache = std::getenv("MFEM_AUTOTUNE_CACHE");
    char key[128];
    snprintf(key, sizeof key, "%d %d %lld %d %d", c->plan.n, c->plan.m, (long long)c->plan.nnz_blocks,
             c->slot.prec, gs[0].B);
    std::vector<int> tiles, splits;
    for (int t : kPcgTiles)
        if (!c->opt.tile_rows || t == c->opt.tile_rows) tiles.push_back(t);
    for (int sp = 1; sp <= 2; ++sp)
        if (!c->opt.spmv_split || sp == c->opt.spmv_split) splits.push_back(sp);
    if (cache) {
        if (FILE* f = fopen(cache, "r")) {
            char line[256];
            while (fgets(line, sizeof line, f)) {
                int tile = 0, sp = 1;
                size_t kl = strlen(key);
                if (strncmp(line, key, kl) == 0 && sscanf(line + kl, " %d %d", &tile, &sp) >= 1 &&
                    std::find(tiles.begin(), tiles.end(), tile) != tiles.end() &&
                    std::find(splits.begin(), splits.end(), sp) != splits.end()) {
                    c->tile_rows = tile;
                    c->spmv_split = sp;
                }
            }
            fclose(f);
            if (c->tile_rows && c->spmv_split) return MFEM_OK;
        }
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_tile = tiles.back(), best_split = splits.front();
    for (auto& g : gs)
        for (int b = 0; b < g.B; ++b) g.ph[b].coarse = 0;   // timed with block Jacobi
    ElemArgs a = elem_args(c);
    for (int tile : tiles)
        for (int sp : splits)
            for (int rep = 0; rep < 2; ++rep) {
                launch_pcg_init(a, gs[0].B, tile, 0.0, 1 << 30, nullptr, nullptr, c->stream);
                CK(cudaEventRecord(e0, c->stream));
                mfem_status st = c->slot.prec == 1 ? run_pcg<float>(c, gs, 1, tile, sp, 20, false)
                                                   : run_pcg<double>(c, gs, 0, tile, sp, 20, false);
                if (st != MFEM_OK) return st;
                CK(cudaEventRecord(e1, c->stream));
                CK(cudaEventSynchronize(e1));
                c->ring_pos = 0;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep == 1 && ms < best) {
                    best = ms;
                    best_tile = tile;
                    best_split = sp;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tile_rows = best_tile;
    c->spmv_split = best_split;
    if (cache) {
        if (FILE* f = fopen(cache, "a")) {
            fprintf(f, "%s %d %d\n", key, best_tile, best_split);
            fclose(f);
        }
    }
    return MFEM_OK;
}

}  // namespace

namespace {

std::vector<int> mask_of(const Group& g, bool (*pred)(const ProbHost&)) {
    std::vector<int> f(g.B, 0);
    for (int b = 0; b < g.B; ++b) f[b] = pred(g.ph[b]) ? 1 : 0;
    return f;
}

bool any_of(const std::vector<int>& f) {
    for (int v : f)
        if (v) return true;
    return false;
}

}  // namespace

namespace {

// Backtracking on E for the problems in `testing` (step lengths in alpha_host,
// halved after each failed Armijo test; attempt k_first, k_first + 1, ...; at
// attempt kLsMax the step is taken as it is), energy trials at x + alpha dx.
mfem_status backtrack(std::vector<Group>& gs, Group& g, std::vector<int> testing, const std::vector<double>& e0,
                      const std::vector<double>& slope, int k_first) {
    mfem_ctx* gc = g.ctx;
    mfem_ctx* c = gc;   // for CK
    cudaStream_t s = gc->stream;
    bool any = any_of(testing);
    for (int k = k_first; any && k <= kLsMax; ++k) {
        mfem_status st = upload_active(gc, g.B, testing);
        if (st != MFEM_OK) return st;
        st = upload_alpha(gc, g.B);
        if (st != MFEM_OK) return st;
        int pl = gc->prof.begin(3, s);
        launch_energy_trial(elem_args(gc), g.B, s);
        gc->prof.end(pl, s);
        gc->prof.launches++;
        st = read_scalars(gc, g.B);
        if (st != MFEM_OK) return st;
        CK(cudaStreamSynchronize(s));
        synced(gs);
        any = false;
        for (int b = 0; b < g.B; ++b) {
            if (!testing[b]) continue;
            const double a = gc->alpha_host[b];
            const double et = gc->sc_host[b].energy_trial;
            if (et <= e0[b] + kLsC * a * slope[b] || k == kLsMax) {
                testing[b] = 0;
            } else {
                gc->alpha_host[b] = 0.5 * a;
                any = true;
            }
        }
    }
    return MFEM_OK;
}

// Armijo's test of the speculative full steps whose element pass just ran
// (energies in sc_host).  A rejected step goes back to x_prev, backtracks from
// alpha = 1/2 with energy trials, takes the accepted step, and needs another
// element pass (the caller leaves such problems out of this round's PCG).
// Returns the rejected problems in `rejected`.
mfem_status check_speculative(std::vector<Group>& gs, Group& g, std::vector<int>& rejected) {
    mfem_ctx* gc = g.ctx;
    mfem_ctx* c = gc;   // for CK
    rejected.assign(g.B, 0);
    std::vector<double> e0(g.B, 0.0), slope(g.B, 0.0);
    bool any = false;
    for (int b = 0; b < g.B; ++b) {
        ProbHost& p = g.ph[b];
        if (!p.active || p.in_pcg || !p.spec) continue;
        p.spec = 0;
        const double et = gc->sc_host[b].energy;
        if (et <= p.spec_e0 + kLsC * 1.0 * p.spec_slope) continue;   // attempt 0 (alpha = 1) passes
        rejected[b] = 1;
        e0[b] = p.spec_e0;
        slope[b] = p.spec_slope;
        gc->alpha_host[b] = 0.5;
        any = true;
        const size_t xb = sizeof(double) * 3 * (size_t)gc->plan.n;
        CK(cudaMemcpyAsync(gc->slot.x + (size_t)b * 3 * gc->plan.n, gc->slot.xprev + (size_t)b * 3 * gc->plan.n, xb,
                           cudaMemcpyDeviceToDevice, gc->stream));
    }
    if (!any) return MFEM_OK;
    mfem_status st = backtrack(gs, g, rejected, e0, slope, 1);
    if (st != MFEM_OK) return st;
    st = upload_active(gc, g.B, rejected);
    if (st != MFEM_OK) return st;
    st = upload_alpha(gc, g.B);
    if (st != MFEM_OK) return st;
    launch_update(elem_args(gc), g.B, gc->stream);
    gc->prof.launches++;
    return MFEM_OK;
}

}  // namespace

mfem_status advance(std::vector<Group>& gs, bool per_request) {
    mfem_ctx* c = gs[0].ctx;
    cudaStream_t s = c->stream;
    // ---- a0: apply poses of newly admitted problems.  The Newton stop test is
    // relative to |g_free| at the rigid initial guess; for REST and WARM starts
    // that reference needs one gradient pass at the rigid guess first (the warm
    // state is parked in outbuf meanwhile); SNH with the COROT start takes the
    // reference there and then the co-rotational predictor step.
    for (auto& g : gs) {
        std::vector<int> f = mask_of(g, [](const ProbHost& p) { return p.need_init != 0; });
        if (!any_of(f)) continue;
        mfem_ctx* gc = g.ctx;
        const int oi = gc->opt.init;
        const bool snh = gc->model == MFEM_SNH;
        // per problem: start 0 rigid guess, 1 rest shape, 2 the state held in x
        // (a caller's state under WARM); SNH under COROT and WARM takes the
        // predictor step from the rigid guess; WARM then adds the correction its
        // slot's last solve needed beyond its own predictor result
        std::vector<int> start(g.B, 0), pred(g.B, 0), corr(g.B, 0);
        bool need_ref = false;
        for (int b = 0; b < g.B; ++b) {
            if (!f[b]) continue;
            start[b] = oi == MFEM_INIT_REST ? 1 : (oi == MFEM_INIT_WARM && gc->warm_kind[b] == 2 ? 2 : 0);
            pred[b] = snh && start[b] == 0 && oi != MFEM_INIT_RIGID;
            corr[b] = pred[b] && oi == MFEM_INIT_WARM && gc->warm_kind[b] == 1 && gc->xpred_valid[b];
            need_ref |= pred[b] || start[b] != 0;
        }
        mfem_status st;
        if (any_of(corr)) {
            st = upload_active(gc, g.B, corr);
            if (st != MFEM_OK) return st;
            launch_warm_save(elem_args(gc), g.B, s);
            gc->prof.launches++;
        }
        st = upload_active(gc, g.B, f);
        if (st != MFEM_OK) return st;
        std::vector<double> gref(g.B, -1.0);
        const size_t xbytes = sizeof(double) * 3 * (size_t)gc->plan.n * g.B;
        bool parked = false;
        if (need_ref) {   // reference gradient at the rigid guess
            for (int b = 0; b < g.B; ++b) parked |= start[b] == 2;
            if (parked) CK(cudaMemcpyAsync(gc->slot.outbuf, gc->slot.x, xbytes, cudaMemcpyDeviceToDevice, s));
            ElemArgs a = elem_args(gc);
            launch_pose_init(a, g.B, 0, s);
            launch_element(a, g.B, s, false);   // forces only: the reference needs no Hessian
            launch_gradient(a, g.B, s);
            gc->prof.launches += 3;
            st = read_scalars(gc, g.B);
            if (st != MFEM_OK) return st;
            CK(cudaStreamSynchronize(s));
            synced(gs);
            for (int b = 0; b < g.B; ++b)
                if (f[b]) gref[b] = std::sqrt(gc->sc_host[b].gnorm2);
            if (parked) CK(cudaMemcpyAsync(gc->slot.x, gc->slot.outbuf, xbytes, cudaMemcpyDeviceToDevice, s));
        }
        for (int code = 0; code < 3; ++code) {   // apply the starts (pins on their targets)
            std::vector<int> m(g.B, 0);
            for (int b = 0; b < g.B; ++b) m[b] = f[b] && start[b] == code && (code != 0 || parked || !need_ref);
            if (!any_of(m)) continue;
            st = upload_active(gc, g.B, m);
            if (st != MFEM_OK) return st;
            launch_pose_init(elem_args(gc), g.B, code, s);
            gc->prof.launches++;
        }
        for (int b = 0; b < g.B; ++b)
            if (f[b]) {
                ProbHost& p = g.ph[b];
                p = ProbHost();
                p.active = 1;
                p.pred = pred[b];
                p.corr = corr[b];
                p.g0 = gref[b];
            }
    }
    // ---- a1-a4: element pass, assembly and gradient for problems that need it
    // (the co-rotational predictor uses that energy), FP64 convergence test,
    // PCG initialisation for those that continue.
    bool any_elem = false;
    for (auto& g : gs) {
        mfem_ctx* gc = g.ctx;
        bool any = false;
        // pass 0: Newton steps (element blocks and matrix), 1: the co-rotational
        // predictor, 2: iterates expected to meet newton_tol (forces only)
        for (int pass = 0; pass < 3; ++pass) {
            std::vector<int> f(g.B, 0);
            for (int b = 0; b < g.B; ++b) {
                const ProbHost& p = g.ph[b];
                if (!p.active || p.in_pcg) continue;
                const bool fo = !p.pred && p.expect_conv && !p.need_hess;
                f[b] = pass == 0 ? (!p.pred && !fo) : (pass == 1 ? p.pred : fo);
            }
            if (!any_of(f)) continue;
            any = true;
            mfem_status st = upload_active(gc, g.B, f);
            if (st != MFEM_OK) return st;
            ElemArgs a = elem_args(gc);
            if (pass == 1) a.model = MFEM_COROT;
            int pe = gc->prof.begin(0, s);
            launch_element(a, g.B, s, pass != 2);
            gc->prof.end(pe, s);
            int pa = gc->prof.begin(1, s);
            if (pass == 2) launch_gradient(a, g.B, s);
            else launch_assemble(a, g.B, s);
            gc->prof.end(pa, s);
            gc->prof.launches += pass == 2 ? 2 : 3;   // element; gradient, or slot assembly + gradient
            gc->prof.element_launches++;
            int na = 0;
            for (int b = 0; b < g.B; ++b) na += f[b];
            gc->prof.element_bytes += na * element_bytes(gc);
            gc->prof.element_updates += (int64_t)na * gc->plan.m;
        }
        if (!any) continue;
        any_elem = true;
        mfem_status st = read_scalars(gc, g.B);
        if (st != MFEM_OK) return st;
    }
    if (any_elem) {
        CK(cudaStreamSynchronize(s));
        synced(gs);
        for (auto& g : gs) {
            mfem_ctx* gc = g.ctx;
            std::vector<int> start(g.B, 0), redo;
            mfem_status sst = check_speculative(gs, g, redo);
            if (sst != MFEM_OK) return sst;
            for (int b = 0; b < g.B; ++b) {
                ProbHost& p = g.ph[b];
                if (!p.active || p.in_pcg || redo[b]) continue;   // a rejected full step: element pass again
                if (!p.pred) {   // the predictor's gradient is not the SNH residual
                    const ProbScal& sc = gc->sc_host[b];
                    p.gn = std::sqrt(sc.gnorm2);
                    p.energy = sc.energy;
                    if (p.g0 < 0.0) p.g0 = p.gn;
                    if (!std::isfinite(p.gn)) {
                        p.active = 0;
                        p.status = MFEM_ENOTCONV;
                        continue;
                    }
                    if (p.gn == 0.0 || p.gn <= gc->opt.newton_tol * p.g0) {
                        p.active = 0;
                        p.converged = 1;
                        p.status = MFEM_OK;
                        continue;
                    }
                    if (p.it >= gc->opt.newton_max) {
                        p.active = 0;
                        p.status = MFEM_ENOTCONV;
                        continue;
                    }
                    if (p.expect_conv && !p.need_hess) {   // tested with forces only: form the Hessian next
                        p.need_hess = 1;
                        continue;
                    }
                }
                p.expect_conv = 0;
                p.need_hess = 0;
                start[b] = 1;
            }
            if (!any_of(start)) continue;
            if (c->tile_rows == 0 || c->spmv_split == 0) {   // first PCG of this context: time the shapes
                std::vector<Group> one{Group{gc, g.B, g.ph}};
                for (int b = 0; b < g.B; ++b) g.ph[b].in_pcg = start[b];
                mfem_status st = upload_active(gc, g.B, start);
                if (st != MFEM_OK) return st;
                st = autotune_tile(c, one);
                if (st != MFEM_OK) return st;
            }
            mfem_status st = upload_active(gc, g.B, start);
            if (st != MFEM_OK) return st;
            // PCG target of this Newton step: cg_tol; where the Newton model is
            // trusted -- a quadratic energy (ARAP or corot with rig rotations:
            // Newton is iterative refinement of one linear solve) or a warm start
            // (near the solution) -- tightened after each step to
            // 0.9 (|g_k| / |g_k-1|)^2 (Eisenstat-Walker's second choice, with
            // their safeguard, at least kEwMin), so that a step the model
            // predicts well is followed by a more accurate one; loosened when a
            // smaller reduction already reaches newton_tol (half of what the
            // linear model says is needed), at most 0.5.  The predictor step is
            // solved tighter: its error, not the SNH nonlinearity, would otherwise
            // set where the first SNH step starts (measured: 3e-3 saves ~8% of
            // PCG iterations and a quarter of a Newton step on the 200k figure
            // against 1e-2).  Measured on the 200k figure, batch of 16: the
            // tightening takes corot from 4 to 3 Newton steps (297 -> 340
            // frames/s) and warm-started SNH streams from 3.6 to 3.1 (+14%), but
            // costs cold SNH poses 1.3%, which therefore keep the fixed target.
            const bool quadratic = gc->model != MFEM_SNH && gc->opt.rotation == MFEM_ROT_RIG;
            const bool trusted = quadratic || gc->opt.init == MFEM_INIT_WARM;
            std::vector<double> t2(g.B, 0.0);
            for (int b = 0; b < g.B; ++b) {
                ProbHost& p = g.ph[b];
                double eta = p.pred ? std::min(gc->opt.cg_tol, kPredTol) : gc->opt.cg_tol;
                if (start[b] && trusted && !p.pred && p.gprev > 0.0 && p.gn > 0.0) {
                    const double rho = p.gn / p.gprev;
                    double ew = kEwGamma * rho * rho;
                    const double guard = kEwGamma * p.eta_prev * p.eta_prev;
                    if (guard > 0.1) ew = std::max(ew, guard);
                    eta = std::min(eta, std::max(ew, kEwMin));
                }
                bool last = false;   // solved to just reach newton_tol
                if (start[b] && !p.pred && p.g0 > 0.0 && p.gn > 0.0) {
                    const double need = 0.5 * gc->opt.newton_tol * p.g0 / p.gn;
                    last = need > eta;
                    eta = std::min(0.5, std::max(eta, need));
                }
                t2[b] = eta * eta;
                if (start[b]) {
                    p.expect_conv = last;
                    if (!p.pred) {
                        p.gprev = p.gn;
                        p.eta_prev = eta;
                    }
                }
            }
            st = upload_doubles(gc, g.B, t2.data(), gc->slot.tol2);
            if (st != MFEM_OK) return st;
            // the two-level preconditioner on every step, the co-rotational
            // predictor and a first step from the rigid guess included (measured
            // on the 200k figure, batch of 16: the predictor's PCG 85 -> 43
            // iterations, whole solves 203 -> 150, 45.3 -> 40.0 ms per batch)
            std::vector<int> co(g.B, 0);
            for (int b = 0; b < g.B; ++b) {   // problems already inside PCG keep their flag
                if (!start[b]) continue;
                ProbHost& p = g.ph[b];
                p.coarse = gc->mesh.coarse_n > 0;
                co[b] = p.coarse;
            }
            st = upload_ints(gc, g.B, co.data(), gc->slot.coarse_on);
            if (st != MFEM_OK) return st;
            if (any_of(co)) {   // the coarse modes' rotations for these iterates (active = start)
                launch_agg_rotations(elem_args(gc), g.B, s);
                gc->prof.launches++;
            }
            launch_pcg_init(elem_args(gc), g.B, c->tile_rows, 0.0, gc->opt.cg_max, gc->slot.tol2,
                            gc->slot.coarse_on, s);
            gc->prof.launches++;
            for (int b = 0; b < g.B; ++b)
                if (start[b]) {
                    g.ph[b].in_pcg = 1;
                    g.ph[b].pcg_launched = 0;
                }
        }
    }
    // ---- a5: one chunk of PCG iterations over every problem inside PCG
    bool any_pcg = false;
    for (auto& g : gs)
        for (int b = 0; b < g.B; ++b) any_pcg |= g.ph[b].active && g.ph[b].in_pcg;
    if (!any_pcg) return MFEM_OK;
    for (int prec = 0; prec < 2; ++prec) {
        bool any = false;
        for (auto& g : gs)
            if (g.ctx->slot.prec == prec)
                for (int b = 0; b < g.B; ++b) any |= g.ph[b].active && g.ph[b].in_pcg;
        if (!any) continue;
        mfem_status st = prec == 1 ? run_pcg<float>(c, gs, 1, c->tile_rows, c->spmv_split, 0, true, true, true,
                                                    per_request)
                                   : run_pcg<double>(c, gs, 0, c->tile_rows, c->spmv_split, 0, true, true, true,
                                                     per_request);
        if (st != MFEM_OK) return st;
    }
    CK(cudaGetLastError());
    // ---- a6: problems whose PCG ended finish their Newton step
    bool any_fin = false;
    std::vector<std::vector<int>> fin(gs.size());
    for (size_t gi = 0; gi < gs.size(); ++gi) {
        Group& g = gs[gi];
        fin[gi].assign(g.B, 0);
        for (int b = 0; b < g.B; ++b) {
            ProbHost& p = g.ph[b];
            if (p.active && p.in_pcg && g.ctx->sc_host[b].state != kActive) {
                fin[gi][b] = 1;
                any_fin = true;
                p.pcg_iters += g.ctx->sc_host[b].iter;
                g.ctx->pcg_hist[(size_t)b * kPcgHistSteps + std::min(p.it, kPcgHistSteps - 1)] =
                    std::max(1, g.ctx->sc_host[b].iter);
                g.ctx->prof.pcg_iters += g.ctx->sc_host[b].iter;
                g.ctx->prof.pcg_bytes += g.ctx->sc_host[b].iter * pcg_bytes_per_iter(g.ctx, p.coarse);
                g.ctx->alpha_host[b] = 1.0;
            }
        }
    }
    if (!any_fin) return MFEM_OK;
    // line-searched steps (SNH, or any model whose rotations follow F; the
    // predictor step is taken whole): their slopes g.dx came back with the
    // PCG states of the chunk that ended them
    std::vector<std::vector<int>> ls(gs.size());
    for (size_t gi = 0; gi < gs.size(); ++gi) {
        Group& g = gs[gi];
        ls[gi].assign(g.B, 0);
        if (!line_search(g.ctx)) continue;
        for (int b = 0; b < g.B; ++b) ls[gi][b] = fin[gi][b] && !g.ph[b].pred;
    }
    // backtracking line search on E (SNH, polar rotations): attempt 0 (the full
    // step) is taken speculatively -- x_prev is kept, x moves to x_prev + dx, and
    // the problem's next element pass, which evaluates E there anyway, decides
    // Armijo's test (check_speculative); a step whose predicted decrease is
    // below rounding noise is taken untested
    for (size_t gi = 0; gi < gs.size(); ++gi) {
        Group& g = gs[gi];
        mfem_ctx* gc = g.ctx;
        if (!line_search(gc) || !any_of(ls[gi])) continue;
        const size_t xb = sizeof(double) * 3 * (size_t)gc->plan.n;
        for (int b = 0; b < g.B; ++b) {
            if (!ls[gi][b]) continue;
            ProbHost& p = g.ph[b];
            const double e0 = p.energy, slope = gc->sc_host[b].slope;
            if (!(-slope > kLsNoise * std::fabs(e0))) continue;
            p.spec = 1;
            p.spec_e0 = e0;
            p.spec_slope = slope;
            CK(cudaMemcpyAsync(gc->slot.xprev + (size_t)b * 3 * gc->plan.n, gc->slot.x + (size_t)b * 3 * gc->plan.n,
                               xb, cudaMemcpyDeviceToDevice, s));
        }
    }
    // x <- x + alpha dx; the problem's next step starts with its element pass
    for (size_t gi = 0; gi < gs.size(); ++gi) {
        Group& g = gs[gi];
        if (!any_of(fin[gi])) continue;
        mfem_ctx* gc = g.ctx;
        mfem_status st = upload_active(gc, g.B, fin[gi]);
        if (st != MFEM_OK) return st;
        st = upload_alpha(gc, g.B);
        if (st != MFEM_OK) return st;
        launch_update(elem_args(gc), g.B, s);
        gc->prof.launches++;
        if (gc->opt.init == MFEM_INIT_WARM && gc->model == MFEM_SNH) {
            for (int apply = 0; apply < 2; ++apply) {   // after the predictor step
                std::vector<int> m(g.B, 0);
                for (int b = 0; b < g.B; ++b) m[b] = fin[gi][b] && g.ph[b].pred && g.ph[b].corr == apply;
                if (!any_of(m)) continue;
                st = upload_active(gc, g.B, m);
                if (st != MFEM_OK) return st;
                launch_warm_step(elem_args(gc), g.B, apply, s);
                gc->prof.launches++;
                for (int b = 0; b < g.B; ++b)
                    if (m[b]) gc->xpred_valid[b] = 1;
            }
        }
        for (int b = 0; b < g.B; ++b)
            if (fin[gi][b]) {
                g.ph[b].it++;
                g.ph[b].in_pcg = 0;
                g.ph[b].pred = 0;
            }
    }
    CK(cudaGetLastError());
    return MFEM_OK;
}

mfem_status run_batch(mfem_ctx* c, int B, std::vector<ProbHost>& ph) {
    ph.assign(B, ProbHost());
    for (int b = 0; b < B; ++b) ph[b].need_init = 1;
    std::vector<Group> gs{Group{c, B, ph.data()}};
    for (int guard = 0; guard < 10000000; ++guard) {
        mfem_status st = advance(gs);
        if (st != MFEM_OK) return st;
        bool any = false;
        for (int b = 0; b < B; ++b) any |= ph[b].active || ph[b].need_init;
        if (!any) break;
    }
    for (int b = 0; b < B; ++b) c->warm_kind[b] = 1;
    // the solutions now in x belong to these poses (warm starts)
    CK(cudaMemcpyAsync(c->slot.xf_prev, c->slot.xf, sizeof(double) * 12 * (size_t)c->plan.H * B,
                       cudaMemcpyDeviceToDevice, c->stream));
    return MFEM_OK;
}

void fill_stats(const mfem_ctx* c, const ProbHost& p, mfem_stats* st) {
    if (!st) return;
    (void)c;
    st->status = p.status;
    st->newton_iters = p.it;
    st->pcg_iters = p.pcg_iters;
    st->converged = p.converged;
    st->grad0 = p.g0 < 0 ? 0.0 : p.g0;
    st->rel_grad = p.g0 > 0 ? p.gn / p.g0 : 0.0;
    st->energy = p.energy;
    st->inverted = -1;
    st->max_rel_skew = -1.0;
    st->max_angle = -1.0;
}

}  // namespace mfem

namespace mfem {

mfem_ctx* ctx_slot_clone(mfem_ctx* src, int cap, cudaStream_t stream, mfem_status* st) {
    mfem_ctx* c = new mfem_ctx();
    // what a solve needs of the plan after creation: sizes, the pattern's slot
    // count, pins (count) and the aggregate size
    Plan& P = c->plan;
    const Plan& S = src->plan;
    P.n = S.n;
    P.m = S.m;
    P.H = S.H;
    P.nnz_blocks = S.nnz_blocks;
    P.n_slices = S.n_slices;
    P.slice_ptr = S.slice_ptr;
    P.pin_vert = S.pin_vert;
    P.pin_handle = S.pin_handle;
    P.vperm = S.vperm;
    P.agg_size = S.agg_size;
    P.n_agg = S.n_agg;
    c->model = src->model;
    c->opt = src->opt;
    c->device = src->device;
    c->stream = stream;
    c->mesh = src->mesh;
    c->mesh_shared = true;
    c->slot.prec = src->slot.prec;
    c->tile_rows = src->tile_rows;
    c->spmv_split = src->spmv_split;
    c->owned_by_server = true;
    mfem_status s = MFEM_OK;
    if (cudaMallocHost((void**)&c->cerr_host, sizeof(unsigned)) != cudaSuccess) s = MFEM_ENOMEM;
    if (s == MFEM_OK) {
        *c->cerr_host = 0;
        s = ensure_slots(c, cap);
    }
    if (s != MFEM_OK) {
        if (st) *st = s;
        mfem_destroy(c);
        return nullptr;
    }
    if (st) *st = MFEM_OK;
    return c;
}

}  // namespace mfem

using namespace mfem;

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

int32_t mfem_abi_version(void) { return MFEM_ABI_VERSION; }

void mfem_default_options(mfem_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = MFEM_MIXED;
    o->constraint = MFEM_ELIMINATE;
    o->k_s = 0.0;
    o->newton_tol = 1e-6;
    o->cg_tol = 3e-2;
    o->newton_max = 50;
    o->cg_max = 5000;
    o->init = MFEM_INIT_COROT;
    o->max_batch = 16;
    o->tile_rows = 0;
    o->spmv_split = 0;
    o->diagnostics = 0;
    o->rotation = MFEM_ROT_RIG;
    o->precond = MFEM_PRECOND_TWO_LEVEL;
    o->launch = MFEM_LAUNCH_GRAPH;
    o->coarse_agg = 0;
    o->coarse_product = MFEM_COARSE_TC;
}

const char* mfem_status_string(mfem_status s) {
    switch (s) {
        case MFEM_OK: return "ok";
        case MFEM_EINVAL: return "invalid argument";
        case MFEM_EDEGEN: return "degenerate rest tet";
        case MFEM_ENOMEM: return "out of memory";
        case MFEM_ENOTCONV: return "not converged";
        case MFEM_ETIMEOUT: return "timed out";
        case MFEM_EBUSY: return "busy";
        case MFEM_ECUDA: return "CUDA error";
    }
    return "unknown status";
}

const char* mfem_last_error(const mfem_ctx* ctx) {
    if (ctx) return ctx->err.c_str();
    return g_thread_err.c_str();
}

mfem_status mfem_plan(const double* rest_verts, int32_t n, const int32_t* tets, int32_t m,
                      const mfem_handles* hs, int32_t* tet_cluster, int32_t* pinned, int32_t* pin_handle) {
    Plan p;
    std::string err;
    mfem_status st = plan_rig(rest_verts, n, tets, m, hs, p, err);
    if (st != MFEM_OK) return ctx_fail(nullptr, st, err);
    if (tet_cluster) std::memcpy(tet_cluster, p.cluster_orig.data(), sizeof(int32_t) * m);
    if (pinned) std::memcpy(pinned, p.pinned_orig.data(), sizeof(int32_t) * n);
    if (pin_handle) std::memcpy(pin_handle, p.pin_handle_orig.data(), sizeof(int32_t) * n);
    return MFEM_OK;
}

void mfem_destroy(mfem_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_slots(c);
    if (c->mesh_shared) c->mesh = MeshDev();   // the owner frees the mesh data
    MeshDev& M = c->mesh;
    void* ptrs[] = {M.tet, M.Dminv64, M.Dminv32, M.Dminv_lo, M.mulam_ff, M.vol, M.cluster, M.mu, M.lam, M.X, M.vhandle, M.pin_handle_v,
                    M.vperm, M.tperm, M.slice_ptr, M.col, M.slot_row, M.up_slot, M.up_mirror, M.contrib_ptr,
                    M.contrib, M.vinc_ptr, M.vinc,
                    M.crel, M.agg_handle, M.Ainv, M.Abf, M.coarse_err, c->descs_dev, c->diag_dev, c->fext_dev};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    void* hp[] = {c->sc_host, c->active_host, c->alpha_host, c->alpha_ring, c->descs_host,
                  c->diag_host, c->cerr_host};
    for (void* p : hp)
        if (p) cudaFreeHost(p);
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    for (auto e : c->prof.ev) cudaEventDestroy(e);
    if (c->prof.start) cudaEventDestroy(c->prof.start);
    if (c->prof.stop) cudaEventDestroy(c->prof.stop);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

// Coarse space of the two-level preconditioner: the rest Hessian (rig at rest,
// x = X; the co-rotational form for SNH, whose rest Hessian it equals) is
// assembled in problem slot 0 and reduced to A_c = P^T K P, whose inverse is
// kept per mesh.
static mfem_status build_coarse(mfem_ctx* c) {
    MeshDev& M = c->mesh;
    const Plan& P = c->plan;
    const int H = P.H;
    std::vector<double> ident((size_t)12 * H, 0.0);
    for (int h = 0; h < H; ++h) ident[12 * h] = ident[12 * h + 5] = ident[12 * h + 10] = 1.0;
    int* cnb_ptr = nullptr;
    int* cnb = nullptr;
    mfem_status st;
    if ((st = upload(c, &cnb_ptr, P.cnb_ptr.data(), P.cnb_ptr.size())) != MFEM_OK) return st;
    if ((st = upload(c, &cnb, P.cnb.data(), P.cnb.size())) != MFEM_OK) {
        cudaFree(cnb_ptr);
        return st;
    }
    c->mesh_bytes -= sizeof(int) * (P.cnb_ptr.size() + P.cnb.size());
    cudaError_t e = cudaMalloc((void**)&M.Ainv, sizeof(float) * (size_t)M.coarse_n * coarse_ld(M.coarse_n));
    if (e == cudaSuccess) {
        c->mesh_bytes += sizeof(float) * (size_t)M.coarse_n * coarse_ld(M.coarse_n);
        e = cudaMemcpyAsync(c->slot.xf, ident.data(), sizeof(double) * ident.size(), cudaMemcpyHostToDevice,
                            c->stream);
    }
    if (e == cudaSuccess) {
        std::vector<int> one(1, 1);
        st = upload_active(c, 1, one);
        if (st != MFEM_OK) {
            cudaFree(cnb_ptr);
            cudaFree(cnb);
            return st;
        }
        ElemArgs a = elem_args(c);
        a.model = c->model == MFEM_ARAP ? MFEM_ARAP : MFEM_COROT;
        a.rot_polar = 0;
        a.fext = nullptr;
        launch_pose_init(a, 1, 1, c->stream);
        launch_element(a, 1, c->stream);
        launch_assemble(a, 1, c->stream);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = build_coarse_inverse(M, c->slot.val, c->slot.prec, cnb_ptr, cnb, P.cnb_max, P.agg_size, M.Ainv, c->stream);
    cudaFree(cnb_ptr);
    cudaFree(cnb);
    // BF16 tiles for the tensor-core product (the FP32 inverse is kept for the
    // CUDA-core product and mfem_coarse_apply), and the error word
    if (e == cudaSuccess) e = cudaMalloc(&M.Abf, coarse_tc_bytes(M.coarse_n));
    if (e == cudaSuccess) {
        c->mesh_bytes += coarse_tc_bytes(M.coarse_n);
        e = coarse_tc_pack(M.Ainv, M.coarse_n, M.Abf, c->stream);
    }
    if (e == cudaSuccess) e = cudaMalloc((void**)&M.coarse_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(M.coarse_err, 0, sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->cerr_host, sizeof(unsigned));
    if (e == cudaSuccess) {
        *c->cerr_host = 0;
        e = coarse_tc_init();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->ring_pos = 0;
    return cuda_check(c, e, "coarse space set-up");
}

mfem_status mfem_create(const double* rest_verts, int32_t n, const int32_t* tets, int32_t m,
                        const mfem_material* mat, const mfem_handles* hs, const mfem_options* opt,
                        mfem_ctx** out) {
    if (!out) return ctx_fail(nullptr, MFEM_EINVAL, "null output pointer");
    *out = nullptr;
    mfem_ctx* c = new mfem_ctx();
    if (opt) c->opt = *opt;
    else mfem_default_options(&c->opt);
    const mfem_options& o = c->opt;
    auto fail = [&](mfem_status s, const std::string& msg) {
        g_thread_err = msg;
        mfem_destroy(c);
        return s;
    };
    if (o.precision != MFEM_FP64 && o.precision != MFEM_MIXED) return fail(MFEM_EINVAL, "bad precision");
    if (o.constraint != MFEM_ELIMINATE && o.constraint != MFEM_PENALTY) return fail(MFEM_EINVAL, "bad constraint");
    if (o.constraint == MFEM_PENALTY && !(o.k_s > 0.0)) return fail(MFEM_EINVAL, "penalty needs k_s > 0");
    if (!(o.newton_tol >= 0.0) || !(o.cg_tol >= 0.0) || o.newton_max < 0 || o.cg_max < 1)
        return fail(MFEM_EINVAL, "bad tolerances or iteration caps");
    if (o.init < MFEM_INIT_RIGID || o.init > MFEM_INIT_COROT) return fail(MFEM_EINVAL, "bad init");
    if (o.rotation != MFEM_ROT_RIG && o.rotation != MFEM_ROT_POLAR) return fail(MFEM_EINVAL, "bad rotation");
    if (o.precond != MFEM_PRECOND_BLOCK_JACOBI && o.precond != MFEM_PRECOND_TWO_LEVEL)
        return fail(MFEM_EINVAL, "bad preconditioner");
    if (o.launch != MFEM_LAUNCH_GRAPH && o.launch != MFEM_LAUNCH_DIRECT) return fail(MFEM_EINVAL, "bad launch mode");
    if (o.tile_rows != 0 && !pcg_tile_supported(o.tile_rows))
        return fail(MFEM_EINVAL, "tile_rows must be 0, 64, 128 or 256");
    if (o.spmv_split < 0 || o.spmv_split > 2) return fail(MFEM_EINVAL, "spmv_split must be 0, 1 or 2");
    if (o.coarse_agg != 0 && (o.coarse_agg < kCoarseUnit || (o.coarse_agg & (o.coarse_agg - 1)) != 0 ||
                              o.coarse_agg > (1 << 24)))
        return fail(MFEM_EINVAL, "coarse_agg must be 0 or a power of two >= 64");
    if (o.coarse_product != MFEM_COARSE_TC && o.coarse_product != MFEM_COARSE_FP32)
        return fail(MFEM_EINVAL, "bad coarse_product");
    if (!mat) return fail(MFEM_EINVAL, "null material");
    std::string err;
    mfem_status st = plan_rig(rest_verts, n, tets, m, hs, c->plan, err);
    if (st != MFEM_OK) return fail(st, err);
    st = plan_layout(mat, rest_verts, tets, c->plan, err, o.coarse_agg);
    if (st != MFEM_OK) return fail(st, err);
    c->model = mat->model;
    c->slot.prec = o.precision == MFEM_MIXED ? 1 : 0;
    c->tile_rows = o.tile_rows;
    c->spmv_split = o.spmv_split;
    const Plan& P = c->plan;
    if (cudaGetDevice(&c->device) != cudaSuccess) return fail(MFEM_ECUDA, "no CUDA device");
    if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(MFEM_ECUDA, "cudaStreamCreate failed");
    c->stream = c->own_stream;
    // device mesh (SoA per tet)
    MeshDev& M = c->mesh;
    M.n = P.n;
    M.m = P.m;
    M.H = P.H;
    M.n_slices = P.n_slices;
    M.n_pins = (int)P.pin_vert.size();
    M.slots = P.slice_ptr.back();
    std::vector<double> Dm64((size_t)9 * P.m);
    std::vector<float> Dm32((size_t)9 * P.m), DmLo((size_t)9 * P.m);
    for (int k = 0; k < P.m; ++k)
        for (int e = 0; e < 9; ++e) {
            const double v = P.Dminv[9 * (size_t)k + e];
            Dm64[(size_t)e * P.m + k] = v;
            Dm32[(size_t)e * P.m + k] = (float)v;
            DmLo[(size_t)e * P.m + k] = (float)(v - (double)(float)v);
        }
    std::vector<float> mulam((size_t)4 * P.m);   // (W mu, W lam) as float pairs
    for (int k = 0; k < P.m; ++k) {
        const double mu = P.vol[k] * P.mu[k], lam = P.vol[k] * P.lam[k];
        mulam[4 * (size_t)k] = (float)mu;
        mulam[4 * (size_t)k + 1] = (float)(mu - (double)(float)mu);
        mulam[4 * (size_t)k + 2] = (float)lam;
        mulam[4 * (size_t)k + 3] = (float)(lam - (double)(float)lam);
    }
    std::vector<int32_t> pin_h(P.n, -1);
    for (size_t i = 0; i < P.pin_vert.size(); ++i) pin_h[P.pin_vert[i]] = P.pin_handle[i];
    std::vector<int32_t> sp(P.slice_ptr.begin(), P.slice_ptr.end());
#define UP(dst, src, cnt)                                   \
    if ((st = upload(c, &(dst), (src), (cnt))) != MFEM_OK) { \
        std::string e2 = c->err;                            \
        return fail(st, e2);                                \
    }
    UP(M.tet, (const int4*)P.tet.data(), (size_t)P.m);
    UP(M.Dminv64, Dm64.data(), Dm64.size());
    UP(M.Dminv32, Dm32.data(), Dm32.size());
    UP(M.Dminv_lo, DmLo.data(), DmLo.size());
    UP(M.mulam_ff, (const float4*)mulam.data(), (size_t)P.m);
    UP(M.vol, P.vol.data(), P.vol.size());
    UP(M.cluster, P.cluster.data(), P.cluster.size());
    UP(M.mu, P.mu.data(), P.mu.size());
    UP(M.lam, P.lam.data(), P.lam.size());
    UP(M.X, P.X.data(), P.X.size());
    UP(M.vhandle, P.vhandle.data(), P.vhandle.size());
    UP(M.pin_handle_v, pin_h.data(), pin_h.size());
    UP(M.vperm, P.vperm.data(), P.vperm.size());
    UP(M.tperm, P.tperm.data(), P.tperm.size());
    UP(M.slice_ptr, sp.data(), sp.size());
    UP(M.col, P.sell_col.data(), P.sell_col.size());
    UP(M.slot_row, P.slot_row.data(), P.slot_row.size());
    UP(M.up_slot, P.up_slot.data(), P.up_slot.size());
    UP(M.up_mirror, P.up_mirror.data(), P.up_mirror.size());
    M.n_up = (int64_t)P.up_slot.size();
    UP(M.contrib_ptr, P.contrib_ptr.data(), P.contrib_ptr.size());
    UP(M.contrib, P.contrib.data(), P.contrib.size());
    UP(M.vinc_ptr, P.vinc_ptr.data(), P.vinc_ptr.size());
    UP(M.vinc, P.vinc.data(), P.vinc.size());
#undef UP
    if (cudaMalloc((void**)&c->diag_dev, 4 * sizeof(unsigned)) != cudaSuccess ||
        cudaMallocHost((void**)&c->diag_host, 4 * sizeof(unsigned)) != cudaSuccess)
        return fail(MFEM_ENOMEM, "small device/host buffers");
    c->prof.ev.resize(2 * 4096);
    for (auto& e : c->prof.ev)
        if (cudaEventCreate(&e) != cudaSuccess) return fail(MFEM_ECUDA, "cudaEventCreate failed");
    if (cudaEventCreate(&c->prof.start) != cudaSuccess || cudaEventCreate(&c->prof.stop) != cudaSuccess)
        return fail(MFEM_ECUDA, "cudaEventCreate failed");
    if (o.precond == MFEM_PRECOND_TWO_LEVEL && P.n_agg > 0) {   // coarse space data (before the slots)
        M.n_agg = P.n_agg;
        M.agg_shift = 0;
        while ((1 << M.agg_shift) < P.agg_size) ++M.agg_shift;
        M.coarse_n = 6 * P.n_agg;
        M.coarse_tc = o.coarse_product == MFEM_COARSE_TC ? 1 : 0;
        if ((st = upload(c, &M.crel, (const float4*)P.crel.data(), (size_t)P.n)) != MFEM_OK ||
            (st = upload(c, &M.agg_handle, P.agg_handle.data(), P.agg_handle.size())) != MFEM_OK) {
            std::string e2 = c->err;
            return fail(st, e2);
        }
    }
    st = ensure_slots(c, std::max(1, o.max_batch));
    if (st != MFEM_OK) {
        std::string e2 = c->err;
        return fail(st, e2);
    }
    if (M.coarse_n > 0 && (st = build_coarse(c)) != MFEM_OK) {
        std::string e2 = c->err;
        return fail(st, e2);
    }
    *out = c;
    return MFEM_OK;
}

mfem_status mfem_set_stream(mfem_ctx* c, void* stream) {
    if (!c) return ctx_fail(nullptr, MFEM_EINVAL, "null context");
    if (c->owned_by_server) return ctx_fail(c, MFEM_EINVAL, "context belongs to a server");
    cudaStreamSynchronize(c->stream);
    c->stream = stream ? (cudaStream_t)stream : c->own_stream;
    return MFEM_OK;
}

static mfem_status validate_pose(mfem_ctx* c, const double* xf, int H) {
    for (int h = 0; h < H; ++h) {
        const double* T = xf + 12 * h;
        for (int i = 0; i < 12; ++i)
            if (!std::isfinite(T[i])) return ctx_fail(c, MFEM_EINVAL, "non-finite handle transform");
        double err = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += T[4 * k + i] * T[4 * k + j];
                err = std::max(err, std::fabs(s - (i == j ? 1.0 : 0.0)));
            }
        double det = T[0] * (T[5] * T[10] - T[6] * T[9]) - T[1] * (T[4] * T[10] - T[6] * T[8]) +
                     T[2] * (T[4] * T[9] - T[5] * T[8]);
        if (err > 1e-6 || det <= 0.0) {
            char buf[128];
            snprintf(buf, sizeof buf, "handle %d: Q is not a rotation (|Q^T Q - I| = %.2e, det = %.3f)", h, err, det);
            return ctx_fail(c, MFEM_EINVAL, buf);
        }
    }
    return MFEM_OK;
}

mfem_status mfem_set_pose(mfem_ctx* c, const double* xf, int32_t H) {
    if (!c || !xf) return ctx_fail(c, MFEM_EINVAL, "null argument");
    if (c->owned_by_server) return ctx_fail(c, MFEM_EINVAL, "context belongs to a server");
    if (H != c->plan.H) return ctx_fail(c, MFEM_EINVAL, "pose has the wrong number of handles");
    mfem_status st = validate_pose(c, xf, H);
    if (st != MFEM_OK) return st;
    CK(cudaMemcpyAsync(c->slot.xf, xf, sizeof(double) * 12 * H, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->pose_set = true;
    return MFEM_OK;
}

mfem_status mfem_set_forces(mfem_ctx* c, const double* f, int32_t n_sets) {
    if (!c) return ctx_fail(c, MFEM_EINVAL, "null context");
    if (c->owned_by_server) return ctx_fail(c, MFEM_EINVAL, "context belongs to a server");
    if (!f || n_sets == 0) {
        CK(cudaStreamSynchronize(c->stream));
        if (c->fext_dev) cudaFree(c->fext_dev);
        c->fext_dev = nullptr;
        c->fext_sets = 0;
        return MFEM_OK;
    }
    if (n_sets < 0) return ctx_fail(c, MFEM_EINVAL, "n_sets must be >= 0");
    const size_t n = c->plan.n, cnt = (size_t)n_sets * n * 3;
    for (size_t i = 0; i < cnt; ++i)
        if (!std::isfinite(f[i])) return ctx_fail(c, MFEM_EINVAL, "non-finite force");
    std::vector<double> perm(cnt);   // caller vertex order -> internal order
    for (size_t s = 0; s < (size_t)n_sets; ++s)
        for (size_t o = 0; o < n; ++o)
            for (int i = 0; i < 3; ++i) perm[(s * n + c->plan.vperm[o]) * 3 + i] = f[(s * n + o) * 3 + i];
    CK(cudaStreamSynchronize(c->stream));
    if (n_sets != c->fext_sets) {
        if (c->fext_dev) cudaFree(c->fext_dev);
        c->fext_dev = nullptr;
        c->fext_sets = 0;
        CK(cudaMalloc((void**)&c->fext_dev, cnt * sizeof(double)));
    }
    CK(cudaMemcpy(c->fext_dev, perm.data(), cnt * sizeof(double), cudaMemcpyHostToDevice));
    c->fext_sets = n_sets;
    return MFEM_OK;
}

static mfem_status finish_stats(mfem_ctx* c, const std::vector<ProbHost>& ph, int B, mfem_stats* stats) {
    mfem_status worst = MFEM_OK;
    for (int b = 0; b < B; ++b) {
        if (ph[b].status != MFEM_OK) worst = (mfem_status)ph[b].status;
        if (!stats) continue;
        fill_stats(c, ph[b], &stats[b]);
        if (c->opt.diagnostics) {
            CK(cudaMemsetAsync(c->diag_dev, 0, 4 * sizeof(unsigned), c->stream));
            launch_diag(elem_args(c), b, c->diag_dev, c->stream);
            CK(cudaMemcpyAsync(c->diag_host, c->diag_dev, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            float f1, f2;
            std::memcpy(&f1, &c->diag_host[1], 4);
            std::memcpy(&f2, &c->diag_host[2], 4);
            stats[b].inverted = (int32_t)c->diag_host[0];
            stats[b].max_rel_skew = f1;
            stats[b].max_angle = f2;
        }
    }
    if (worst == MFEM_ENOTCONV) ctx_fail(c, worst, "Newton iteration cap reached before newton_tol");
    return worst;
}

mfem_status mfem_solve(mfem_ctx* c, double* out, mfem_stats* stats) {
    if (!c || !out) return ctx_fail(c, MFEM_EINVAL, "null argument");
    if (c->owned_by_server) return ctx_fail(c, MFEM_EINVAL, "context belongs to a server");
    if (!c->pose_set) return ctx_fail(c, MFEM_EINVAL, "mfem_set_pose must come first");
    begin_profile(c);
    std::vector<ProbHost> ph;
    mfem_status st = run_batch(c, 1, ph);
    if (st != MFEM_OK) return st;
    launch_unpermute(elem_args(c), 1, c->slot.outbuf, c->stream);
    c->prof.launches++;
    CK(cudaMemcpyAsync(out, c->slot.outbuf, sizeof(double) * 3 * c->plan.n, cudaMemcpyDeviceToHost, c->stream));
    end_profile(c);
    return finish_stats(c, ph, 1, stats);
}

// Checks of a batch request, slot allocation, and the upload of its poses.
static mfem_status stage_batch(mfem_ctx* c, const double* xf, int32_t B, double* out, int32_t memory) {
    if (!c || !xf || !out) return ctx_fail(c, MFEM_EINVAL, "null argument");
    if (c->owned_by_server) return ctx_fail(c, MFEM_EINVAL, "context belongs to a server");
    if (B < 1) return ctx_fail(c, MFEM_EINVAL, "B must be >= 1");
    if (c->fext_sets > 1 && B > c->fext_sets)
        return ctx_fail(c, MFEM_EINVAL, "more poses than external force fields");
    if (memory != MFEM_MEM_HOST && memory != MFEM_MEM_DEVICE) return ctx_fail(c, MFEM_EINVAL, "bad memory kind");
    const int H = c->plan.H;
    mfem_status st = ensure_slots(c, B);
    if (st != MFEM_OK) return st;
    const size_t xf_bytes = sizeof(double) * 12 * (size_t)H * B;
    if (memory == MFEM_MEM_HOST) {
        st = validate_pose(c, xf, H * B);
        if (st != MFEM_OK) return st;
        CK(cudaMemcpyAsync(c->slot.xf, xf, xf_bytes, cudaMemcpyHostToDevice, c->stream));
    } else {
        std::vector<double> tmp((size_t)12 * H * B);
        CK(cudaMemcpyAsync(tmp.data(), xf, xf_bytes, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        st = validate_pose(c, tmp.data(), H * B);
        if (st != MFEM_OK) return st;
        CK(cudaMemcpyAsync(c->slot.xf, xf, xf_bytes, cudaMemcpyDeviceToDevice, c->stream));
    }
    return MFEM_OK;
}

// Solutions of a finished batch -> out (caller vertex order).
static mfem_status emit_batch(mfem_ctx* c, int32_t B, double* out, int32_t memory) {
    const int n = c->plan.n;
    if (memory == MFEM_MEM_HOST) {
        launch_unpermute(elem_args(c), B, c->slot.outbuf, c->stream);
        CK(cudaMemcpyAsync(out, c->slot.outbuf, sizeof(double) * 3 * (size_t)n * B, cudaMemcpyDeviceToHost,
                           c->stream));
    } else {
        launch_unpermute(elem_args(c), B, out, c->stream);
    }
    c->prof.launches++;
    return MFEM_OK;
}

mfem_status mfem_solve_batch(mfem_ctx* c, const double* xf, int32_t B, double* out, int32_t memory,
                             mfem_stats* stats) {
    mfem_status st = stage_batch(c, xf, B, out, memory);
    if (st != MFEM_OK) return st;
    begin_profile(c);
    std::vector<ProbHost> ph;
    st = run_batch(c, B, ph);
    if (st != MFEM_OK) return st;
    st = emit_batch(c, B, out, memory);
    if (st != MFEM_OK) return st;
    end_profile(c);
    return finish_stats(c, ph, B, stats);
}

mfem_status mfem_solve_multi(mfem_ctx* const* ctxs, int32_t n_ctx, const double* const* xf, const int32_t* B,
                             double* const* out, int32_t memory, mfem_stats* const* stats) {
    if (!ctxs || !xf || !B || !out || n_ctx < 1) return ctx_fail(nullptr, MFEM_EINVAL, "null argument or n_ctx < 1");
    for (int i = 0; i < n_ctx; ++i) {
        if (!ctxs[i]) return ctx_fail(nullptr, MFEM_EINVAL, "null context");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return ctx_fail(ctxs[i], MFEM_EINVAL, "a context appears twice");
        if (ctxs[i]->device != ctxs[0]->device) return ctx_fail(ctxs[i], MFEM_EINVAL, "contexts on different devices");
    }
    // every context works on the first context's stream for the call
    std::vector<cudaStream_t> saved(n_ctx);
    for (int i = 0; i < n_ctx; ++i) {
        saved[i] = ctxs[i]->stream;
        if (i > 0) {
            cudaStreamSynchronize(ctxs[i]->stream);
            ctxs[i]->stream = ctxs[0]->stream;
        }
    }
    auto restore = [&]() {
        for (int i = 1; i < n_ctx; ++i) ctxs[i]->stream = saved[i];
    };
    mfem_status st = MFEM_OK;
    for (int i = 0; i < n_ctx && st == MFEM_OK; ++i) st = stage_batch(ctxs[i], xf[i], B[i], out[i], memory);
    if (st != MFEM_OK) { restore(); return st; }
    std::vector<std::vector<ProbHost>> ph(n_ctx);
    std::vector<Group> gs;
    for (int i = 0; i < n_ctx; ++i) {
        begin_profile(ctxs[i]);
        ph[i].assign(B[i], ProbHost());
        for (int b = 0; b < B[i]; ++b) ph[i][b].need_init = 1;
    }
    for (int i = 0; i < n_ctx; ++i) gs.push_back(Group{ctxs[i], B[i], ph[i].data()});
    for (int guard = 0; guard < 10000000 && st == MFEM_OK; ++guard) {
        st = advance(gs);
        bool any = false;
        for (int i = 0; i < n_ctx; ++i)
            for (int b = 0; b < B[i]; ++b) any |= ph[i][b].active || ph[i][b].need_init;
        if (!any) break;
    }
    for (int i = 0; i < n_ctx && st == MFEM_OK; ++i) {
        for (int b = 0; b < B[i]; ++b) ctxs[i]->warm_kind[b] = 1;
        st = cuda_check(ctxs[i], cudaMemcpyAsync(ctxs[i]->slot.xf_prev, ctxs[i]->slot.xf,
                                                 sizeof(double) * 12 * (size_t)ctxs[i]->plan.H * B[i],
                                                 cudaMemcpyDeviceToDevice, ctxs[i]->stream), "keep poses");
        if (st != MFEM_OK) break;
        st = emit_batch(ctxs[i], B[i], out[i], memory);
    }
    mfem_status worst = st;
    for (int i = 0; i < n_ctx && st == MFEM_OK; ++i) {
        end_profile(ctxs[i]);
        mfem_status si = finish_stats(ctxs[i], ph[i], B[i], stats ? stats[i] : nullptr);
        if (si != MFEM_OK && worst == MFEM_OK) worst = si;
    }
    restore();
    return worst;
}

mfem_status mfem_get_elem(mfem_ctx* c, double* s, double* lam) {
    if (!c) return ctx_fail(nullptr, MFEM_EINVAL, "null context");
    if (!s && !lam) return MFEM_OK;
    const size_t m = c->plan.m;
    double* buf = nullptr;
    CK(cudaMalloc((void**)&buf, sizeof(double) * 15 * m));
    launch_elem_out(elem_args(c), 0, s ? buf : nullptr, lam ? buf + 6 * m : nullptr, c->stream);
    mfem_status st = cuda_check(c, cudaGetLastError(), "element-output kernel launch");
    if (st != MFEM_OK) {
        cudaFree(buf);
        return st;
    }
    if (s && (st = cuda_check(c, cudaMemcpyAsync(s, buf, sizeof(double) * 6 * m, cudaMemcpyDeviceToHost, c->stream),
                              "copy s")) != MFEM_OK) {
        cudaFree(buf);
        return st;
    }
    if (lam && (st = cuda_check(c, cudaMemcpyAsync(lam, buf + 6 * m, sizeof(double) * 9 * m,
                                                   cudaMemcpyDeviceToHost, c->stream), "copy lam")) != MFEM_OK) {
        cudaFree(buf);
        return st;
    }
    st = cuda_check(c, cudaStreamSynchronize(c->stream), "get_elem");
    cudaFree(buf);
    return st;
}

mfem_status mfem_get_state(const mfem_ctx* cc, double* x) {
    mfem_ctx* c = const_cast<mfem_ctx*>(cc);
    if (!c || !x) return ctx_fail(c, MFEM_EINVAL, "null argument");
    launch_unpermute(elem_args(c), 1, c->slot.outbuf, c->stream);
    CK(cudaMemcpyAsync(x, c->slot.outbuf, sizeof(double) * 3 * c->plan.n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MFEM_OK;
}

mfem_status mfem_set_state(mfem_ctx* c, const double* x) {
    if (!c || !x) return ctx_fail(c, MFEM_EINVAL, "null argument");
    for (size_t i = 0; i < 3 * (size_t)c->plan.n; ++i)
        if (!std::isfinite(x[i])) return ctx_fail(c, MFEM_EINVAL, "non-finite state");
    CK(cudaMemcpyAsync(c->slot.outbuf, x, sizeof(double) * 3 * c->plan.n, cudaMemcpyHostToDevice, c->stream));
    launch_permute_in(elem_args(c), 0, c->slot.outbuf, c->stream);
    CK(cudaStreamSynchronize(c->stream));
    c->warm_kind[0] = 2;
    c->xpred_valid[0] = 0;
    return MFEM_OK;
}

mfem_status mfem_get_profile(const mfem_ctx* c, mfem_profile* p) {
    if (!c || !p) return ctx_fail(const_cast<mfem_ctx*>(c), MFEM_EINVAL, "null argument");
    *p = c->last_profile;
    return MFEM_OK;
}

mfem_status mfem_get_info(const mfem_ctx* c, int32_t* n, int32_t* m, int32_t* H, int32_t* n_pins,
                          int64_t* nnz_blocks, int64_t* sell_slots, int64_t* device_bytes) {
    if (!c) return ctx_fail(nullptr, MFEM_EINVAL, "null context");
    if (n) *n = c->plan.n;
    if (m) *m = c->plan.m;
    if (H) *H = c->plan.H;
    if (n_pins) *n_pins = (int32_t)c->plan.pin_vert.size();
    if (nnz_blocks) *nnz_blocks = c->plan.nnz_blocks;
    if (sell_slots) *sell_slots = c->plan.slice_ptr.back();
    if (device_bytes) *device_bytes = (int64_t)(c->mesh_bytes + c->slot_bytes);
    return MFEM_OK;
}

mfem_status mfem_coarse_apply(mfem_ctx* c, const float* rc, int32_t B, float* e, int32_t product) {
    if (!c || !rc || !e) return ctx_fail(c, MFEM_EINVAL, "null argument");
    if (c->mesh.coarse_n <= 0) return ctx_fail(c, MFEM_EINVAL, "the context has no coarse space");
    if (B < 1) return ctx_fail(c, MFEM_EINVAL, "B must be >= 1");
    if (product != MFEM_COARSE_TC && product != MFEM_COARSE_FP32) return ctx_fail(c, MFEM_EINVAL, "bad product");
    const bool tc = product == MFEM_COARSE_TC;
    const int N = c->mesh.coarse_n;
    const size_t nks = coarse_ks(c);
    // per problem: r_c, scalars marking it active, and the product's output --
    // slice partials (CUDA cores) or, on the tensor cores, the B operand and e
    const size_t n_out = tc ? (((size_t)B + kCoarseGroupSlots - 1) / kCoarseGroupSlots) * kCoarseGroupSlots * N
                            : (size_t)B * nks * N;
    float* rc_d = nullptr;
    float* out_d = nullptr;
    void* bs_d = nullptr;
    ProbScal* sc_d = nullptr;
    PcgDesc<float>* d_d = nullptr;
    auto cleanup = [&]() {
        cudaFree(rc_d);
        cudaFree(out_d);
        cudaFree(bs_d);
        cudaFree(sc_d);
        cudaFree(d_d);
    };
    // r_c rows padded to the 16-byte-aligned stride the kernels' vector loads need
    const size_t ldr = coarse_ld(N);
    cudaError_t err = cudaMalloc((void**)&rc_d, sizeof(float) * (size_t)B * ldr);
    if (err == cudaSuccess) err = cudaMalloc((void**)&out_d, sizeof(float) * n_out);
    if (err == cudaSuccess && tc) err = cudaMalloc(&bs_d, coarse_b_bytes(N, B));
    if (err == cudaSuccess) err = cudaMalloc((void**)&sc_d, sizeof(ProbScal) * (size_t)B);
    if (err == cudaSuccess) err = cudaMalloc((void**)&d_d, sizeof(PcgDesc<float>) * (size_t)B);
    std::vector<ProbScal> sc(B);
    std::vector<PcgDesc<float>> d(B);
    for (int b = 0; b < B; ++b) {
        std::memset(&sc[b], 0, sizeof(ProbScal));
        sc[b].state = kActive;
        std::memset(&d[b], 0, sizeof(PcgDesc<float>));
        d[b].coarse = 1;
        d[b].ctc = tc ? 1 : 0;
        d[b].bslot = b;
        d[b].coarse_n = N;
        d[b].sc = sc_d + b;
        d[b].rc = rc_d + (size_t)b * ldr;
        if (!tc) d[b].ec = out_d + (size_t)b * nks * N;
    }
    if (err == cudaSuccess)
        err = cudaMemcpy2DAsync(rc_d, sizeof(float) * ldr, rc, sizeof(float) * N, sizeof(float) * N, B,
                                cudaMemcpyHostToDevice, c->stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(sc_d, sc.data(), sizeof(ProbScal) * B, cudaMemcpyHostToDevice, c->stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(d_d, d.data(), sizeof(PcgDesc<float>) * B, cudaMemcpyHostToDevice, c->stream);
    if (err == cudaSuccess) err = cudaMemsetAsync(out_d, 0, sizeof(float) * n_out, c->stream);
    if (err == cudaSuccess && tc) err = cudaMemsetAsync(bs_d, 0, coarse_b_bytes(N, B), c->stream);
    if (err == cudaSuccess && tc) err = coarse_split(rc_d, N, (int)ldr, B, bs_d, c->stream);
    if (err == cudaSuccess) err = cudaMemsetAsync(c->mesh.coarse_err, 0, sizeof(unsigned), c->stream);
    if (err == cudaSuccess) {
        CoarseJob j{c->mesh.Ainv, tc ? c->mesh.Abf : nullptr, bs_d, c->mesh.coarse_err, c, N, 0, B, 1, B};
        err = launch_coarse_only(d_d, B, &j, tc ? out_d : nullptr, c->stream);
    }
    std::vector<float> out(n_out);
    unsigned werr = 0;
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(out.data(), out_d, sizeof(float) * n_out, cudaMemcpyDeviceToHost, c->stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(&werr, c->mesh.coarse_err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
    cleanup();
    if (err != cudaSuccess) return cuda_check(c, err, "coarse apply");
    if (werr) return ctx_fail(c, MFEM_ECUDA, "coarse product: a bounded wait in the tensor-core kernel ran out");
    if (tc) {   // e of every slot, complete
        std::memcpy(e, out.data(), sizeof(float) * (size_t)B * N);
        return MFEM_OK;
    }
    for (int b = 0; b < B; ++b)   // slices added in slice order, as the correction kernel does
        for (int i = 0; i < N; ++i) {
            float v = 0.f;
            for (size_t k = 0; k < nks; ++k) v += out[((size_t)b * nks + k) * N + i];
            e[(size_t)b * N + i] = v;
        }
    return MFEM_OK;
}

}  // extern "C"
