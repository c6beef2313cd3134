// Launch wrappers of the pose-solver kernels (host-callable).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dev.cuh"

namespace mfem {

// Static per-mesh data on the device (internal vertex/tet order).
struct MeshDev {
    int n = 0, m = 0, H = 0, n_slices = 0, n_pins = 0;
    int64_t slots = 0;
    int4* tet = nullptr;          // [m]
    double* Dminv64 = nullptr;    // [9][m]
    float* Dminv32 = nullptr;     // [9][m]
    float* Dminv_lo = nullptr;    // [9][m] D_m^{-1} - Dminv32 (the float pair's low part)
    float4* mulam_ff = nullptr;   // [m] (W mu, W lam) as float pairs: (hi, lo, hi, lo); Psi, sigma and
                                  // the Hessian are linear in (mu, lam), so they come out weighted by W
    double* vol = nullptr;        // [m]
    int* cluster = nullptr;       // [m]
    double* mu = nullptr;         // [m]
    double* lam = nullptr;        // [m]
    double* X = nullptr;          // [n][3]
    int* vhandle = nullptr;       // [n]
    int* pin_handle_v = nullptr;  // [n] handle or -1
    int* vperm = nullptr;         // [n] caller vertex -> internal
    int* tperm = nullptr;         // [m] caller tet -> internal
    int* slice_ptr = nullptr;     // [n_slices+1]
    int* col = nullptr;           // [slots]
    int* slot_row = nullptr;      // [slots] block row of each slot
    int64_t n_up = 0;
    int* up_slot = nullptr;       // [n_up] diagonal and upper slots
    int* up_mirror = nullptr;     // [n_up] slot of each one's transposed block, -1 on the diagonal
    int* contrib_ptr = nullptr;   // [slots+1]
    int* contrib = nullptr;       // [16m]
    int* vinc_ptr = nullptr;      // [n+1]
    int* vinc = nullptr;          // [4m]
    // two-level preconditioner (coarse_n = 0: block Jacobi only)
    int n_agg = 0, agg_shift = 0, coarse_n = 0;
    float4* crel = nullptr;       // [n] rest offset from the aggregate centroid, w = 1 free / 0 pin
    int* agg_handle = nullptr;    // [n_agg]
    float* Ainv = nullptr;        // [coarse_n][coarse_ld] inverse of the rest coarse matrix (rows padded)
    void* Abf = nullptr;          // the same inverse in BF16, tiled for the tensor-core product
    unsigned* coarse_err = nullptr;  // [1] bits set by a coarse-product wait that ran out
    int coarse_tc = 0;            // 1: the coarse product runs on the tensor cores (Abf)
};

// Per-batch problem buffers of one mesh (B problems, strides in elements).
struct SlotDev {
    int cap = 0;
    int prec = 1;            // 1 = mixed (float K and PCG vectors), 0 = FP64
    double* xf = nullptr;    // [B][H][12]
    double* xf_prev = nullptr;  // [B][H][12] pose of the solution held in x (warm starts)
    double* xpred = nullptr;    // [B][n][3] x after the predictor step of the last solve (WARM only)
    double* dcorr = nullptr;    // [B][n][3] last solve's solution minus xpred (WARM only)
    double* x = nullptr;     // [B][n][3]
    float2* xff = nullptr;   // [B][n][3] x as float pairs (hi, lo), refreshed before each mixed element pass
    float2* qff = nullptr;   // [B][H][9] handle rotations as float pairs, refreshed with xff
    double* xprev = nullptr; // [B][n][3] x before a speculative full Newton step (line-searched models)
    double* xp = nullptr;    // [B][n][3] pin targets (pinned rows only)
    double* g = nullptr;     // [B][n][3] masked gradient
    double* ge = nullptr;    // [B][m][12] element forces
    void* Ke = nullptr;      // [B][m][kKe] + kKePad element blocks (float or double)
    void* val = nullptr;     // [B][slots*9]
    void* dinv = nullptr;    // [B][9][npad32(n)] block-Jacobi inverses, entry-major
    void* vec = nullptr;     // [B][kVecStride][npad32(n)]: the neighbour record nb and the six row fields
    double* part = nullptr;  // [B][tiles][4]
    int part_tiles = 0;
    ProbScal* sc = nullptr;  // [B]
    int* active = nullptr;   // [B]
    double* alpha = nullptr; // [B] step length for update / trial
    double* tol2 = nullptr;  // [B] squared relative PCG residual target of the current Newton step
    int* coarse_on = nullptr;  // [B] two-level preconditioner in the current PCG solve
    float* rcp = nullptr;    // [B][rcp_stride] restriction partials (6 floats per 64-row unit)
    float* ec = nullptr;     // [B][ceil(coarse_n / kCoarseKC)][coarse_n] partial coarse corrections
    float* rcs = nullptr;    // [B][rcs_stride] per-aggregate coarse residual (aggregates over 64 rows)
    float* aggq = nullptr;   // [B][n_agg][9] rotation of each aggregate's coarse modes for the current solve
    uint16_t* bsplit = nullptr;  // tensor-core coarse product: B operand, [ceil(B/16)][chunks][48 x 256] BF16
    size_t rcs_stride = 0;
    size_t rcp_stride = 0;
    double* outbuf = nullptr;  // [B][n][3] caller-order staging
};

struct ElemArgs {
    MeshDev mesh;
    SlotDev slot;
    int model;        // mfem_model
    int constraint;   // 0 eliminate, 1 penalty
    double ks;
    const double* fext = nullptr;  // external vertex forces [sets][n][3] (internal order) or null
    int64_t fext_stride = 0;       // doubles between problems' force fields (0: one shared field)
    int rot_polar = 0;             // 1: R_k = rotation factor of F_k (co-rotational FEM), else the rig's
    int f32_forces = 0;            // mixed path: element forces formed in FP32 from the FP64 stress
    int ff_elem = 0;               // mixed path: F, S, stress and energy in float-float arithmetic (xff)
};
// The mixed path forms element forces in FP32 when the Newton stop test is at
// least this loose: the FP32 forces leave a residual floor near 1e-8 of the
// initial gradient (measured: the 10k-tet figure converges to 1e-8 and stalls
// at 6e-9; the 200k figure reaches 1e-9), so tighter tests keep FP64 forces.
constexpr double kF32ForcesTol = 1.0e-7;

#ifdef __CUDACC__
// Vector `off` of problem b in the interleaved PCG vector block of a slot.
template <typename T>
__device__ __forceinline__ T* vecp(const SlotDev& S, int b, int off, int n) {
    const size_t np = npad32(n);
    return (T*)S.vec + (size_t)b * kVecStride * np + (size_t)off * np;
}
#endif

// a0: pose -> pin targets and initial guess (init: 0 rigid, 1 rest, 2 the
// state held in x)
void launch_pose_init(const ElemArgs& a, int B, int init, cudaStream_t s);
// warm starts (SNH): dcorr = x - xpred before the new pose is applied; after
// the predictor step xpred = x and, with apply, x += dQ_h dcorr on free vertices
void launch_warm_save(const ElemArgs& a, int B, cudaStream_t s);
void launch_warm_step(const ElemArgs& a, int B, int apply, cudaStream_t s);
// a1: element step (Ke, element forces, energy) for active problems
// hess = false: energy and forces only (no element blocks)
void launch_element(const ElemArgs& a, int B, cudaStream_t s, bool hess = true);
// a6: energy at x + alpha dx for active problems (line-search trial)
void launch_energy_trial(const ElemArgs& a, int B, cudaStream_t s);
// a2/a3/a4: gather matrix blocks with pin elimination, block-Jacobi inverse
void launch_assemble(const ElemArgs& a, int B, cudaStream_t s);
// gradient gather with pin elimination/penalty and |g|^2 per problem
void launch_gradient(const ElemArgs& a, int B, cudaStream_t s);
// slope g.dx per problem
void launch_slope(const ElemArgs& a, int B, cudaStream_t s);
// x += alpha dx
void launch_update(const ElemArgs& a, int B, cudaStream_t s);
// x (internal order) -> out [B][n][3] caller order
void launch_unpermute(const ElemArgs& a, int B, double* out, cudaStream_t s);
// warm state import: caller-order [n][3] -> slot x
void launch_permute_in(const ElemArgs& a, int b, const double* xin, cudaStream_t s);
// element outputs (s, lambda) in caller tet order for problem b
void launch_elem_out(const ElemArgs& a, int b, double* s_out, double* lam_out, cudaStream_t s);
// two-level preconditioner: the rotation of each aggregate's coarse modes for
// the problems' current iterates (shape matching; the handle's rotation when
// the aggregate's deformation has no rotation factor)
void launch_agg_rotations(const ElemArgs& a, int B, cudaStream_t s);
// diagnostics: inverted count, max rel skew, max angle for problem b
void launch_diag(const ElemArgs& a, int b, unsigned* out3, cudaStream_t s);

// PCG: init (r = -g, z = D^{-1} r, rho, |r0|) and `iters` iterations over
// every problem of a descriptor table (spmv + update; with coarse jobs, the
// coarse product per mesh and the correction first); tiles of tile_rows rows
// (64, 128 or 256), n_units = total tiles.
// tol2_b: per-problem squared tolerances on the device, or null for tol2 for all;
// coarse_b: per-problem flags (device) of the two-level preconditioner, or null.
void launch_pcg_init(const ElemArgs& a, int B, int tile_rows, double tol2, int maxit, const double* tol2_b,
                     const int* coarse_b, cudaStream_t s);
// One mesh's coarse solve inside the PCG iterations: descriptors d0 .. d0+nd-1.
struct CoarseJob {
    const float* Ainv;          // FP32 inverse (CUDA-core product) ...
    const void* Abf;            // ... or its packed BF16 rows (fused tensor-core kernel), when not null
    const void* Bs;             // tensor cores: the context's B operand (groups of 16 slots)
    unsigned* err;              // the mesh's coarse-product error word
    const void* key;            // the mesh (context) the job belongs to
    int N, d0, nd, agg_units;   // agg_units: 64-row units per aggregate
    int slots;                  // tensor cores: request slots of the context (B groups = ceil(slots / 16))
};
// n_units: SpMV tiles (tile_rows rows) over all problems; n_units_u: the
// update and correction kernels' tiles (kRowTileU rows); split: SpMV threads
// per row (1 or 2).
template <typename T>
cudaError_t launch_pcg_iters(const PcgDesc<T>* descs_dev, int n_probs, int n_units, int n_units_u, int tile_rows,
                             int split, int iters, const CoarseJob* jobs, int n_jobs, cudaStream_t s);
bool pcg_tile_supported(int tile_rows);

// Coarse space set-up: A_c = P^T K P of the assembled matrix `val` (problem 0 of
// a slot, precision prec) and its FP32 inverse into Ainv (coarse_n rows of
// coarse_ld(coarse_n) floats, zero padding).
cudaError_t build_coarse_inverse(const MeshDev& M, const void* val, int prec, const int* cnb_ptr, const int* cnb,
                                 int cnb_max, int agg_size, float* Ainv, cudaStream_t s);

// The coarse product alone for one job (mfem_coarse_apply): the CUDA-core
// product writes slice partials to each descriptor's ec; the tensor-core
// product writes e[slot][N] to e_out.
cudaError_t launch_coarse_only(const PcgDesc<float>* descs, int n_probs, const CoarseJob* job, float* e_out,
                               cudaStream_t s);
// Fused tensor-core coarse product and correction (k_coarse_tc.cu): bytes of
// the packed BF16 rows of an N x N inverse and of the B operand for `slots`
// request slots, the packing from the FP32 inverse, the split of FP32 coarse
// residuals (rows of ldr floats) into the B operand, the one-time kernel
// attribute set-up (before any capture), and the launch for one job (e_out
// null: correction of the problems' u; else the product alone into e_out).
size_t coarse_tc_bytes(int N);
size_t coarse_b_bytes(int N, int slots);
cudaError_t coarse_tc_pack(const float* Ainv, int N, void* Abf, cudaStream_t s);
cudaError_t coarse_split(const float* rc, int N, int ldr, int B, void* Bs, cudaStream_t s);
cudaError_t coarse_tc_init();
template <typename T>
cudaError_t launch_coarse_fused(const cudaLaunchConfig_t& base, const CoarseJob& j, const PcgDesc<T>* descs,
                                float* e_out);

}  // namespace mfem
