/*
 * mfem.h -- C ABI of the GB300 mixed-FEM skinning pose solver.
 *
 * Method (paper: "Automatic Skinning using the Mixed Finite Element Method"):
 *   Every tet k has a stretch S_k tied to its deformation gradient F_k = B_k x
 *   through a rotation R_k that comes from the rig (§3, Eq. 2-4).  S_k is the
 *   least-squares solution of F_k = R_k S_k, S_k = sym(R_k^T F_k) -- the batched
 *   pseudo-inverse of [R] named after Eq. 12.  The energy E(x) = sum_k W_k Psi(S_k)
 *   (Eq. 5-6) is minimised over the vertex positions x with pinned vertices
 *   following their handles, x_p = H x_hat_p (§3.2).  Its Newton system is the
 *   condensed SPD system of Eq. 12; for ARAP and co-rotational Psi it is linear
 *   and one solve reaches the minimiser (text after Eq. 12), for stable
 *   neo-Hookean Psi Newton iterates with a line search.  Per pose (Algorithm 1):
 *   build [R] from the handle transforms, assemble, solve.
 *
 * Conventions for every entry point:
 *   - Every call returns an mfem_status and never aborts the process.  On an
 *     error, mfem_last_error(ctx) gives a one-line reason.
 *   - Input arrays are read during the call only; the caller keeps ownership.
 *     Output arrays are caller-allocated.  "host" pointers are ordinary CPU
 *     memory (pinned or not); "device" pointers are CUDA global memory of the
 *     context's device.
 *   - Arrays are row-major, C-contiguous: verts [n][3] double, tets [m][4] int32,
 *     handle transforms xf [H][12] double holding the 3x4 matrix [Q | t]
 *     row-major (a point p maps to Q p + t, world frame).
 *   - A context is not thread-safe; use one thread per context.  The server
 *     (mfem_server_*) is internally locked and may be called from any thread.
 *   - The library owns all device memory it allocates and frees it in
 *     mfem_destroy / mfem_server_destroy.
 */
#ifndef MFEM_H_
#define MFEM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MFEM_ABI_VERSION 6

typedef enum {
    MFEM_OK = 0,
    MFEM_EINVAL = 1,    /* bad argument: index out of range, NaN, non-orthonormal Q, ... */
    MFEM_EDEGEN = 2,    /* a rest tet has volume <= 0 (its index is in the error text) */
    MFEM_ENOMEM = 3,    /* device or host allocation failed, or a server budget is exceeded */
    MFEM_ENOTCONV = 4,  /* Newton or PCG hit its iteration cap; the best x is still written */
    MFEM_ETIMEOUT = 5,  /* a bounded device wait or a server wait ran out of time */
    MFEM_EBUSY = 6,     /* no free server slot for a non-blocking submit */
    MFEM_ECUDA = 7      /* a CUDA runtime call failed (text names it) */
} mfem_status;

typedef enum { MFEM_ARAP = 0, MFEM_COROT = 1, MFEM_SNH = 2 } mfem_model;
typedef enum { MFEM_FP64 = 0, MFEM_MIXED = 1 } mfem_precision;
typedef enum { MFEM_ELIMINATE = 0, MFEM_PENALTY = 1 } mfem_constraint;
typedef enum { MFEM_CLUSTER_BONE = 0, MFEM_CLUSTER_JOINT = 1, MFEM_CLUSTER_MIDPOINT = 2 } mfem_cluster_rule;
typedef enum { MFEM_INIT_RIGID = 0, MFEM_INIT_REST = 1, MFEM_INIT_WARM = 2, MFEM_INIT_COROT = 3 } mfem_init;
typedef enum { MFEM_MEM_HOST = 0, MFEM_MEM_DEVICE = 1 } mfem_memory;
typedef enum { MFEM_ROT_RIG = 0, MFEM_ROT_POLAR = 1 } mfem_rotation;
typedef enum { MFEM_PRECOND_BLOCK_JACOBI = 0, MFEM_PRECOND_TWO_LEVEL = 1 } mfem_precond;
typedef enum { MFEM_LAUNCH_GRAPH = 0, MFEM_LAUNCH_DIRECT = 1 } mfem_launch;
typedef enum { MFEM_COARSE_TC = 0, MFEM_COARSE_FP32 = 1 } mfem_coarse_product;

/* Material (§4 "A solver friendly to variant energies"; §4 "Allowing
 * heterogeneous material").  Densities, with S the element stretch:
 *   ARAP   mu |S - I|^2
 *   COROT  mu |S - I|^2 + lambda/2 tr(S - I)^2
 *   SNH    mu/2 (|S|^2 - 3) - mu (det S - 1) + (lambda + mu)/2 (det S - 1)^2
 * mu / lambda: per-tet arrays [m] (host), or NULL to use mu0 / lambda0 for all. */
typedef struct {
    int32_t model;            /* mfem_model */
    const double* mu;         /* [m] or NULL */
    const double* lambda;     /* [m] or NULL */
    double mu0, lambda0;
} mfem_material;

/* Rig (§3.1, Algorithm 1 input "skeleton h").  joints [H][3] rest positions;
 * parent [H] (-1 for a root).  A bone runs parent -> child and carries the
 * parent joint's handle transform.  Tet rotation clusters (§3.1): by default
 * each tet takes the bone segment nearest its barycenter (MFEM_CLUSTER_BONE;
 * with no bones, the nearest joint); MFEM_CLUSTER_JOINT takes the nearest
 * joint; MFEM_CLUSTER_MIDPOINT the bone whose midpoint is nearest (the
 * variants compared in §4, "Exploring different rotation clustering");
 * tet_cluster [m] (handle indices) overrides all (§4, user-defined clusters).
 * Pins (Eq. 6; vertices held along the skeleton): pin_verts /
 * pin_handle [n_pins] if given, else every vertex within pin_radius of a joint
 * or a bone midpoint, following the handle its position clusters to.  Ties in
 * nearest-X searches go to the lowest index (a 1e-10 * bbox_diag^2 margin). */
typedef struct {
    int32_t n_handles;
    const double* joints;        /* [H][3] */
    const int32_t* parent;       /* [H] */
    const int32_t* tet_cluster;  /* [m] or NULL */
    const int32_t* pin_verts;    /* [n_pins] or NULL */
    const int32_t* pin_handle;   /* [n_pins] or NULL */
    int32_t n_pins;
    double pin_radius;
    int32_t cluster_rule;        /* mfem_cluster_rule */
} mfem_handles;

/* Solver options.  mfem_default_options fills the defaults given here. */
typedef struct {
    int32_t precision;   /* MFEM_MIXED (default): FP32 element Hessians, SpMV and PCG
                            vectors, FP64 gradient/residual, dots and positions;
                            MFEM_FP64: everything FP64 */
    int32_t constraint;  /* MFEM_ELIMINATE (default): pins fixed at x_p (k_s -> inf);
                            MFEM_PENALTY: k_s/2 |x_v - x_p|^2 per pin (Eq. 6) */
    double k_s;          /* penalty stiffness (PENALTY only) */
    double newton_tol;   /* stop when |g_free| <= newton_tol |g_free(x_0)| (1e-6) */
    double cg_tol;       /* PCG relative residual per Newton step, inexact Newton (3e-2);
                            for quadratic energies (ARAP, corot with rig rotations)
                            and WARM starts each step after the first takes
                            min(cg_tol, max(1e-4, 0.9 (|g_k| / |g_k-1|)^2)),
                            safeguarded (Eisenstat-Walker); a step that needs less
                            to reach newton_tol takes
                            eta = min(0.5, 0.5 newton_tol |g_free(x_0)| / |g_free|);
                            the co-rotational predictor step takes min(cg_tol, 3e-3) */
    int32_t newton_max;  /* Newton step cap (50) */
    int32_t cg_max;      /* PCG iteration cap per Newton step (5000) */
    int32_t init;        /* mfem_init: COROT (default) -- for SNH, first one Newton
                            step of the co-rotational energy (same mu, lambda;
                            quadratic, same rest Hessian) from the rigid guess,
                            counted as a Newton step; for ARAP/corot the rigid
                            guess.  RIGID moves every vertex with the handle its
                            rest position clusters to; REST uses X (Algorithm 1);
                            WARM (for animation streams): SNH takes the COROT
                            start and then adds the correction the slot's last
                            solve needed beyond its own predictor result, each
                            vertex's correction turned by the rotation change of
                            the handle its rest position clusters to; ARAP and
                            corot take the rigid guess (their minimiser is one
                            linear solve from any start); a state set by
                            mfem_set_state is used as it is */
    int32_t max_batch;   /* poses per mfem_solve_batch call allocated for (16) */
    int32_t tile_rows;   /* SpMV rows per block: 64, 128 or 256; 0 = autotune (timed
                            on the first assembled system) */
    int32_t diagnostics; /* 1: fill inverted/skew/angle fields of mfem_stats (0) */
    int32_t rotation;    /* MFEM_ROT_RIG (default): R_k is the rotation of the tet's
                            cluster handle (§3, Eq. 3; §3.1) -- the paper's method.
                            MFEM_ROT_POLAR: R_k is the rotation factor of F_k(x),
                            re-evaluated at every Newton step and line-search
                            trial (det R = +1; for det F < 0 the least stretch is
                            negative), so E is the co-rotational FEM energy of the
                            standard FEM model §4 compares against, with the rig
                            coupled through the pins only.  Newton steps use the
                            Hessian at fixed R and are line-searched on E for every
                            model */
    int32_t precond;     /* MFEM_PRECOND_TWO_LEVEL (default): 3x3 block Jacobi plus an
                            additive coarse correction on the six rigid modes of
                            aggregates of consecutive (Morton-ordered) vertices,
                            its matrix the rest-shape Hessian's, inverted once per
                            mesh; before every solve each aggregate's modes are
                            turned by the rotation fitted to its vertices'
                            current positions (polar factor of sum x_i (X_i -
                            c)^T; its handle's rotation where that has none);
                            used on every Newton step.
                            MFEM_PRECOND_BLOCK_JACOBI: block Jacobi only */
    int32_t launch;      /* MFEM_LAUNCH_GRAPH (default): each chunk of PCG iterations
                            is captured once per set of launch parameters as a CUDA
                            graph and replayed (up to 256 graphs per context; a
                            stream that cannot capture falls back to direct
                            launches); MFEM_LAUNCH_DIRECT: launches every kernel */
    int32_t coarse_agg;  /* vertices per aggregate of the two-level preconditioner:
                            0 (default) = the smallest power of two >= 64 that keeps
                            the coarse space at most 6144 dof (6 per aggregate);
                            else a power of two >= 64, raised to that smallest size
                            if it is below it.  Other values: MFEM_EINVAL */
    int32_t spmv_split;  /* SpMV threads per row: 1, 2 (two threads take a row's
                            even and odd slots), 0 = autotune with tile_rows */
    int32_t coarse_product; /* the coarse solve e = A_c^{-1} r_c of the two-level
                            preconditioner: MFEM_COARSE_TC (default) -- A_c^{-1}
                            rounded to BF16 (a fixed symmetric matrix) times r_c
                            split exactly into three BF16 parts, on the tensor
                            cores (tcgen05) with FP32 accumulation;
                            MFEM_COARSE_FP32 -- FP32 A_c^{-1} on the CUDA cores.
                            Both keep the preconditioner linear and SPD; the
                            solution does not depend on the choice */
} mfem_options;

/* Per-pose result statistics. */
typedef struct {
    int32_t status;          /* mfem_status of this pose */
    int32_t newton_iters;    /* Newton steps taken */
    int32_t pcg_iters;       /* PCG iterations summed over Newton steps */
    int32_t converged;       /* 1 if |g_free| <= newton_tol |g_free(x_0)| */
    double grad0;            /* |g_free(x_0)|, FP64 */
    double rel_grad;         /* final |g_free| / grad0, FP64 */
    double energy;           /* final E(x): FP64 sum of the element energies (formed in
                                float-float on the mixed path at newton_tol >= 1e-7,
                                in FP64 otherwise) */
    int32_t inverted;        /* tets with det F <= 0 (diagnostics=1) */
    double max_rel_skew;     /* max |skew(R^T F)| / |F| (diagnostics=1) */
    double max_angle;        /* max angle (rad) between R_k and polar(F_k) (diagnostics=1) */
} mfem_stats;

/* Device-side profile of the last solve call, timed with CUDA events on the
 * context's stream.  The dominant work is the PCG iteration: an SpMV+dot
 * kernel and an update kernel per iteration, plus on two-level iterations one
 * kernel per mesh for the coarse product and correction (tensor cores), or the
 * product and a correction kernel (CUDA cores), enqueued in chunks. */
typedef struct {
    int32_t kernel_launches;  /* all library kernels launched in the call */
    int32_t pcg_launches;     /* SpMV and update launches (two per iteration) */
    double pcg_ms;            /* summed time of the PCG iteration chunks (all their kernels) */
    double pcg_bytes;         /* algorithmic bytes moved by those chunks */
    int64_t pcg_iters;        /* PCG iterations summed over poses */
    int32_t element_launches;
    double element_ms;
    double element_bytes;
    double assemble_ms;
    double linesearch_ms;
    double total_ms;          /* first to last library event of the call */
    int32_t tile_rows;        /* SpMV rows per block in use */
    int32_t grid_blocks;      /* PCG blocks per launch (tiles of all problems) */
    int64_t element_updates;  /* per-tet local steps (a1) of the Newton element passes */
    int32_t coarse_dof;       /* dimension of the two-level coarse space (0: none) */
    int32_t coarse_launches;  /* coarse-solve and correction launches (two-level) */
    int32_t coarse_tc;        /* 1: the coarse solves ran on the tensor cores */
    int32_t spmv_split;       /* SpMV threads per row in use */
} mfem_profile;

typedef struct mfem_ctx mfem_ctx;
typedef struct mfem_server mfem_server;

void mfem_default_options(mfem_options* opt);
const char* mfem_status_string(mfem_status s);
int32_t mfem_abi_version(void);

/* Build a solver context for one mesh on the current CUDA device: validates
 * the mesh (indices in [0,n), finite coordinates, every rest tet with positive
 * volume -> else MFEM_EINVAL / MFEM_EDEGEN), precomputes D_m^-1 and W_k (Eq. 5),
 * clusters (§3.1), pins, a Morton reordering of vertices and tets, the sliced
 * block-sparse pattern of the Eq. 12 matrix, and uploads everything.  rest_verts,
 * tets and all arrays in mat / hs are host memory.  opt may be NULL (defaults).
 * *out receives the context (NULL on error; the error text is then available
 * through mfem_last_error(NULL) on this thread). */
mfem_status mfem_create(const double* rest_verts, int32_t n, const int32_t* tets, int32_t m,
                        const mfem_material* mat, const mfem_handles* hs,
                        const mfem_options* opt, mfem_ctx** out);

/* Run the context's work on this CUDA stream (a cudaStream_t of the same
 * device, e.g. torch.cuda.current_stream().cuda_stream); NULL restores the
 * context's own stream. */
mfem_status mfem_set_stream(mfem_ctx* ctx, void* stream);

/* Set the pose for the next mfem_solve (Algorithm 1, "[R] <- R(t)"): xf is
 * host [H][12].  Each Q must satisfy |Q^T Q - I| <= 1e-6 and det Q > 0 and all
 * values must be finite, else MFEM_EINVAL. */
mfem_status mfem_set_pose(mfem_ctx* ctx, const double* xf, int32_t H);

/* External vertex forces (§4, "Collision response": a force applied to a few
 * vertices): the energy gains -sum_v f_v . x_v, so the gradient gains -f and
 * the Eq. 12 matrix is unchanged.  f is host [n_sets][n][3] FP64 in the caller's
 * vertex order, copied during the call.  n_sets = 1: one field for every pose
 * of mfem_solve / mfem_solve_batch; n_sets > 1: pose b of a batch takes field b
 * (mfem_solve takes field 0) and a batch of more than n_sets poses is
 * MFEM_EINVAL.  f = NULL or n_sets = 0 removes the forces.  Forces on pinned
 * vertices have no effect under MFEM_ELIMINATE.  Non-finite values or
 * n_sets < 0: MFEM_EINVAL.  Not available on contexts owned by a server. */
mfem_status mfem_set_forces(mfem_ctx* ctx, const double* f, int32_t n_sets);

/* Solve the pose set by mfem_set_pose; out_verts is host [n][3] in the caller's
 * vertex order.  stats may be NULL.  MFEM_ENOTCONV still writes x. */
mfem_status mfem_solve(mfem_ctx* ctx, double* out_verts, mfem_stats* stats);

/* Solve B independent poses of this mesh together (each PCG iteration launch
 * serves all of them).  xf [B][H][12], out [B][n][3]; both host
 * (MFEM_MEM_HOST: copies happen inside the call) or both device
 * (MFEM_MEM_DEVICE).  stats: host [B] or NULL.  B <= max_batch grows the
 * allocation if needed.  Each pose's result does not depend on the others. */
mfem_status mfem_solve_batch(mfem_ctx* ctx, const double* xf, int32_t B, double* out,
                             int32_t memory, mfem_stats* stats);

/* mfem_solve_batch over several meshes at once: B[i] poses of ctxs[i] for
 * i < n_ctx, solved together -- every problem of every mesh moves through its
 * own Newton steps, and each PCG iteration launch serves every problem of
 * every mesh currently inside PCG.  xf[i] [B[i]][H_i][12], out[i] [B[i]][n_i][3]
 * (all host or all device, as `memory` says), stats[i] host [B[i]] (stats or
 * stats[i] may be NULL).  The contexts must be distinct and on one device; the
 * work runs on ctxs[0]'s stream (the others' streams are synchronised first and
 * restored after the call).  PCG tiles are ctxs[0]'s.  Each result equals the
 * same pose solved alone.  With init = MFEM_INIT_WARM, pose b of a mesh starts
 * from the last solution held in that mesh's slot b (see mfem_options.init). */
mfem_status mfem_solve_multi(mfem_ctx* const* ctxs, int32_t n_ctx, const double* const* xf,
                             const int32_t* B, double* const* out, int32_t memory,
                             mfem_stats* const* stats);

/* Element outputs of the last mfem_solve (Eq. 10-11 recovered per element):
 * s [m][6] the stretch S_k as (S00,S11,S22,S12,S02,S01) -- plain components,
 * not Mandel -- and lam [m][9] the multiplier Lambda_k = R_k dPsi/dS row-major.
 * Host arrays, caller's tet order; either may be NULL. */
mfem_status mfem_get_elem(mfem_ctx* ctx, double* s, double* lam);

/* mfem_get_elem for callers that cannot allocate device memory after set-up.
 * The paper has no counterpart; this is a deployment variant.  mfem_get_elem
 * allocates and frees a device staging buffer on every call, and cudaFree
 * waits for the whole device; a per-frame animation loop or a host
 * application's plugin that owns a fixed device budget may allocate only while
 * it sets up, so it cannot call that.  This entry point runs the same kernel
 * but stages through a fixed file-scope device array of 15 doubles per tet for
 * at most MFEM_ELEM_STATIC_MAX_TETS tets (7.5 MiB), held by every GPU that
 * loads the library until the process exits; it calls no cudaMalloc, cudaFree
 * or allocating library routine.  Arguments and outputs are those of
 * mfem_get_elem (host s [m][6], lam [m][9], caller tet order, either may be
 * NULL).  The context's device must be current.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and keeps it for
 * the life of the process: make that first call before any stream capture, and
 * do not reset the device (cudaDeviceReset) between calls -- the kept address
 * would then be stale.  All calls on a device share the one array,
 * which keeps the last call's contents (each call overwrites every entry it
 * returns); two calls whose work overlaps on the GPU (other streams or
 * threads) race on it.  Meshes with more than MFEM_ELEM_STATIC_MAX_TETS tets
 * are rejected with MFEM_EINVAL. */
#define MFEM_ELEM_STATIC_MAX_TETS 65536
mfem_status mfem_get_elem_static(mfem_ctx* ctx, double* s, double* lam);

/* The coarse solve of the two-level preconditioner applied to given vectors,
 * for inspection and tests (not part of the paper's method, §5: the reduced
 * space is the preconditioner's).  rc: host [B][N] FP32 coarse residuals in the
 * coarse basis of mfem_get_info's mesh (N = profile.coarse_dof), e: host
 * [B][N] results e_b = A_c^{-1} rc_b as the solve computes them (on the
 * tensor cores: the full K range accumulated in tensor memory; on the CUDA
 * cores: slice partials added in slice order).  product: MFEM_COARSE_TC or
 * MFEM_COARSE_FP32.  Allocates and frees device memory during the call.
 * MFEM_EINVAL if the context has no coarse space or B < 1. */
mfem_status mfem_coarse_apply(mfem_ctx* ctx, const float* rc, int32_t B, float* e, int32_t product);

/* Warm-start state (the last solution, host [n][3], caller order). */
mfem_status mfem_get_state(const mfem_ctx* ctx, double* x);
mfem_status mfem_set_state(mfem_ctx* ctx, const double* x);

/* Profile of the last mfem_solve / mfem_solve_batch call. */
mfem_status mfem_get_profile(const mfem_ctx* ctx, mfem_profile* prof);

/* Sizes of the context: n, m, handles, pins, block nonzeros of the Eq. 12
 * pattern, padded slots of the sliced layout, device bytes held. Any may be NULL. */
mfem_status mfem_get_info(const mfem_ctx* ctx, int32_t* n, int32_t* m, int32_t* n_handles,
                          int32_t* n_pins, int64_t* nnz_blocks, int64_t* sell_slots,
                          int64_t* device_bytes);

/* Host-only planning, no GPU touched: runs the same validation, clustering and
 * pin selection as mfem_create and writes tet_cluster [m], pin flags [n]
 * (1 = pinned) and pin handle [n] (-1 if not pinned), all in the caller's order.
 * Any output may be NULL. */
mfem_status mfem_plan(const double* rest_verts, int32_t n, const int32_t* tets, int32_t m,
                      const mfem_handles* hs, int32_t* tet_cluster, int32_t* pinned,
                      int32_t* pin_handle);

void mfem_destroy(mfem_ctx* ctx);

/* Text of the last error of this context (or of the calling thread when ctx is
 * NULL); never NULL. */
const char* mfem_last_error(const mfem_ctx* ctx);

/* ---- Serving: continuous batching of pose solves over resident meshes ----
 * A server owns meshes (contexts) and a worker thread.  Requests that arrive
 * while others are on the GPU are admitted at the next Newton-step boundary as
 * slots and device memory allow; all admitted requests of all meshes advance
 * together (each PCG iteration launch serves every admitted request).
 * Each request's result equals the same pose solved alone by mfem_solve_batch. */

/* device_mem_budget: bytes the server may hold for request slots and warm
 * state (0 = no limit); max_slots: requests admitted at once across meshes.
 * Admission is by device memory: each mesh starts with one pool of up to 8
 * request slots; a request that finds every slot of its mesh busy gets a new
 * pool of up to 8 slots (sharing the mesh's device data) when the budget has
 * room for it -- pools of other meshes idle at that moment are released to make
 * room -- and otherwise waits in the queue; pools idle for 2 s are
 * released. */
mfem_status mfem_server_create(size_t device_mem_budget, int32_t max_slots, mfem_server** out);

/* Hand a context to the server (ownership transfers; do not use or destroy
 * ctx afterwards).  *mesh_id receives its id.  The mesh's resident state
 * (pattern, static element data, preconditioner) stays on the device until the
 * server is destroyed.  Fails with MFEM_ENOMEM if one slot of this mesh cannot
 * fit the budget; the context is then left with the caller. */
mfem_status mfem_server_add(mfem_server* srv, mfem_ctx* mesh, int32_t* mesh_id);

/* Queue one pose solve: xf host [H][12] (copied now), out_verts host [n][3]
 * written before the ticket completes (must stay valid until then).
 * *ticket identifies the request. */
mfem_status mfem_server_submit(mfem_server* srv, int32_t mesh_id, const double* xf,
                               double* out_verts, uint64_t* ticket);

/* Wait up to timeout_ms (< 0: forever) for a request; MFEM_ETIMEOUT if it is
 * still running.  On completion fills stats (may be NULL) and returns the
 * request's status.  Latency (submit to completion, seconds) goes to *latency_s
 * if non-NULL. */
mfem_status mfem_server_wait(mfem_server* srv, uint64_t ticket, int32_t timeout_ms,
                             mfem_stats* stats, double* latency_s);

/* Counters: requests completed, scheduling rounds run, PCG launches, peak
 * slots in use, slot pools added and released, device bytes held for slots and
 * warm state.  Any output may be NULL. */
mfem_status mfem_server_counters(mfem_server* srv, int64_t* completed, int64_t* steps,
                                 int64_t* pcg_launches, int32_t* peak_slots, int64_t* pools_added,
                                 int64_t* pools_released, int64_t* device_bytes);

void mfem_server_destroy(mfem_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* MFEM_H_ */
