// Engine internals: the solver context and the Newton driver shared by the
// batch entry points and the serving loop.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/mfem.h"
#include "kernels.h"
#include "plan.h"

namespace mfem {

// Host view of one problem (one pose of one mesh) during a Newton solve.
struct ProbHost {
    int active = 0;      // still iterating
    int need_init = 0;   // pose/initial guess not yet applied
    int in_pcg = 0;      // active and inside its PCG solve (else next is the element pass)
    int it = 0;          // Newton steps taken
    int pcg_iters = 0;
    int ran_pcg = 0;     // PCG ran in the current step
    int status = MFEM_OK;
    int converged = 0;
    int pred = 0;        // co-rotational predictor step pending (SNH, COROT or WARM init)
    int corr = 0;        // after the predictor, add the last solve's rotated correction (WARM)
    int coarse = 0;      // the current PCG solve uses the two-level preconditioner
    int expect_conv = 0; // the current step was solved to just reach newton_tol: test the next
                         // iterate with forces only (no element Hessian, no matrix)
    int need_hess = 0;   // that test failed: the next element pass forms the Hessian
    double g0 = -1.0, gn = 0.0, energy = 0.0;
    double gprev = -1.0;   // |g_free| before the last Newton step (not the predictor), for the forcing rule
    double eta_prev = 0.0; // that step's PCG target
    // speculative full step of a line-searched Newton step: x holds x_prev + dx
    // (x_prev kept in slot.xprev) and the next element pass, which computes
    // E(x_prev + dx) anyway, decides Armijo's test at alpha = 1
    int spec = 0;
    double spec_e0 = 0.0, spec_slope = 0.0;
    int pcg_launched = 0;   // PCG iterations launched in the current solve
};

// Profile accumulator with a pool of CUDA events on the context stream.
struct Profiler {
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;   // per event pair: 0 element, 1 assemble, 2 pcg, 3 line search, 4 other
    int used = 0;
    int launches = 0;
    int pcg_launches = 0, element_launches = 0, coarse_launches = 0;
    double pcg_bytes = 0.0, element_bytes = 0.0;
    int64_t pcg_iters = 0;
    int64_t element_updates = 0;
    cudaEvent_t start = nullptr, stop = nullptr;
    void reset() {
        used = 0;
        launches = pcg_launches = element_launches = coarse_launches = 0;
        pcg_bytes = element_bytes = 0.0;
        pcg_iters = 0;
        element_updates = 0;
        kind.clear();
    }
    int begin(int k, cudaStream_t s);   // returns pair index or -1
    void end(int idx, cudaStream_t s);
};

}  // namespace mfem

struct mfem_ctx {
    mfem::Plan plan;
    int model = MFEM_ARAP;
    mfem_options opt{};
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    mfem::MeshDev mesh;
    mfem::SlotDev slot;
    size_t mesh_bytes = 0, slot_bytes = 0;
    void* descs_dev = nullptr;
    size_t descs_cap = 0;
    // pinned host staging.  Async uploads read from a ring of regions so that a
    // region is never rewritten before its copy has run; the ring restarts after
    // every stream synchronisation.
    mfem::ProbScal* sc_host = nullptr;
    int* active_host = nullptr;      // [kStageRing][cap]
    double* alpha_host = nullptr;    // current step lengths [cap]
    double* alpha_ring = nullptr;    // [kStageRing][cap]
    int ring_pos = 0;
    void* descs_host = nullptr;
    unsigned* diag_dev = nullptr;
    double* fext_dev = nullptr;   // external forces [fext_sets][n][3], internal order
    int fext_sets = 0;
    unsigned* diag_host = nullptr;
    unsigned* cerr_host = nullptr;   // pinned copy of mesh.coarse_err, read with the problem scalars
    int tile_rows = 0;       // SpMV rows per block (0: autotune)
    int spmv_split = 0;      // SpMV threads per row, 1 or 2 (0: autotune)
    int grid_blocks = 0;
    bool pose_set = false;
    // per slot: 0 = x holds no start, 1 = x is the solution of the pose in
    // slot.xf_prev (a warm start follows the handles to the new pose),
    // 2 = x was set by the caller (a warm start uses it as it is)
    std::vector<int> warm_kind;
    std::vector<int> xpred_valid;   // per slot: slot.xpred holds the last solve's predictor result
    // per slot and Newton step: PCG iterations that step's last solve took
    // (0 = none yet), from which the length of the next PCG chunk is predicted
    std::vector<int> pcg_hist;
    mfem::Profiler prof;
    // PCG chunks captured as CUDA graphs, keyed by the launch parameters
    std::map<std::string, cudaGraphExec_t> graphs;
    bool graphs_off = false;   // capture failed once (e.g. a stream that cannot capture)
    mfem_profile last_profile{};
    std::string err;
    bool owned_by_server = false;
    bool mesh_shared = false;   // a server slot pool: the mesh's device data belongs to another context
};

namespace mfem {

constexpr int kStageRing = 64;

// One Newton group: B problems of one context.
struct Group {
    mfem_ctx* ctx;
    int B;
    ProbHost* ph;
};

mfem_status ctx_fail(mfem_ctx* c, mfem_status s, const std::string& msg);
// A context that shares src's device mesh data (and preconditioner) but owns
// `cap` request slots of its own, working on `stream` (server slot pools).
// Returns null and sets *st on failure.  Destroy it before src.
mfem_ctx* ctx_slot_clone(mfem_ctx* src, int cap, cudaStream_t stream, mfem_status* st);
mfem_status cuda_check(mfem_ctx* c, cudaError_t e, const char* what);
mfem_status ensure_slots(mfem_ctx* c, int B);
size_t slot_bytes_for(const mfem_ctx* c, int B);
ElemArgs elem_args(const mfem_ctx* c);

// One scheduling round over every problem of every group (all groups share
// groups[0].ctx->stream): apply newly admitted poses; run the element pass,
// assembly and convergence test of problems that need them and start their PCG;
// run one chunk of PCG iterations over the problems inside PCG; finish the
// Newton step (line search, update) of problems whose PCG ended.  Problems move
// through their Newton steps independently, so none waits for another's PCG.
// The round's PCG chunk runs until the last solve of the table is expected to
// end (a batch call: the batch is done when its last problem is), or, with
// per_request, until the first is (a server: each request completes alone).
mfem_status advance(std::vector<Group>& groups, bool per_request = false);

// Whole solve of B problems of one context (poses already in slot.xf).
mfem_status run_batch(mfem_ctx* c, int B, std::vector<ProbHost>& ph);

void fill_stats(const mfem_ctx* c, const ProbHost& p, mfem_stats* st);
void begin_profile(mfem_ctx* c);
void end_profile(mfem_ctx* c);

}  // namespace mfem
