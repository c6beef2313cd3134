// PCG kernels (a5): initialisation and the stream-ordered kernels of one
// preconditioned CG iteration over a table of problems.  The preconditioner is
// 3x3 block Jacobi, or block Jacobi plus an additive coarse correction on the
// rigid modes of vertex aggregates (two-level; set-up in k_coarse.cu).
//
// Paper §3, Eq. 12 and the linear solve of Algorithm 1: the condensed system
// is SPD, so it is solved by conjugate gradients (inexactly inside each Newton
// step, to a relative residual).  Dots are accumulated as float-float partials
// per row and warp and reduced per problem in FP64 with a ticketed, fixed-order
// tile reduction, so results do not depend on scheduling.
#include <cuda_runtime.h>

#include "kernels.h"

namespace mfem {

namespace {

// Rotations of the aggregates a block of rows from row0 touches (blocks hold
// <= 256 rows, so <= 4 aggregates) into qs; threads 0..35 load, the caller
// synchronises (restrict_units does).
__device__ __forceinline__ void stage_rotations(float (*qs)[9], int row0, const float* __restrict__ aggq,
                                                int agg_shift, int n_agg) {
    const int a0 = row0 >> agg_shift;
    if (threadIdx.x < 36) {
        const int ai = threadIdx.x / 9, e = threadIdx.x % 9, a = a0 + ai;
        qs[ai][e] = a < n_agg ? aggq[9 * a + e] : 0.f;
    }
}

// Coarse residual of the rows of one block: y_i = Q_a^T r_i (the aggregate's
// rotation undone, Q staged by stage_rotations), contribution
// P_i^T y_i = (y_i, (X_i - c_a) x y_i) of a free row, summed per 64-row unit
// (two warps: shuffle sums, then the pair in fixed order) and written to
// rcp_block[6 u + c].  Every thread of the block calls it; rows past the end
// pass valid = false.
__device__ __forceinline__ void restrict_units(const float (&r)[3], bool valid, int row, int row0,
                                               const float4* __restrict__ crel, const float (*qs)[9], int agg_shift,
                                               float* __restrict__ rcp_block, uint16_t* __restrict__ bgrp = nullptr,
                                               int bslot = 0, int coarse_n = 0) {
    __shared__ float ws[8][6];
    const int a0 = row0 >> agg_shift;   // row0: the block's first row
    __syncthreads();
    float y[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
        const float4 v = crel[row];
        if (v.w != 0.f) {   // FP32 throughout (the coarse correction is a preconditioner)
            const float* Qt = qs[(row >> agg_shift) - a0];
            const float q0 = Qt[0] * r[0] + Qt[3] * r[1] + Qt[6] * r[2];
            const float q1 = Qt[1] * r[0] + Qt[4] * r[1] + Qt[7] * r[2];
            const float q2 = Qt[2] * r[0] + Qt[5] * r[1] + Qt[8] * r[2];
            y[0] = q0;
            y[1] = q1;
            y[2] = q2;
            y[3] = v.y * q2 - v.z * q1;
            y[4] = v.z * q0 - v.x * q2;
            y[5] = v.x * q1 - v.y * q0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 6; ++c) y[c] += __shfl_xor_sync(0xffffffffu, y[c], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 6; ++c) ws[warp][c] = y[c];
    __syncthreads();
    const int units = blockDim.x / kCoarseRows;
    if ((int)threadIdx.x < 6 * units) {
        const int u = threadIdx.x / 6, c = threadIdx.x % 6;
        const float v = ws[2 * u][c] + ws[2 * u + 1][c];
        rcp_block[6 * u + c] = v;
        // an aggregate is one unit: this is r_c, also written as the
        // tensor-core product's B operand (all its units lie in this block)
        const int k = 6 * (row0 / kCoarseRows + u) + c;   // units past the last aggregate write nothing
        if (bgrp && k < coarse_n) coarse_b_store(bgrp, bslot % kCoarseGroupSlots, k, v);
    }
}

// ---- vector access ------------------------------------------------------------
// 3-vectors stored as aligned 4-element groups (x, y, z, 0)
__device__ __forceinline__ void ld4(const float* p, float (&v)[3]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
}

__device__ __forceinline__ void ld4(const double* p, double (&v)[3]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
}

__device__ __forceinline__ void st4(float* p, float a, float b, float c) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, 0.f);
}

__device__ __forceinline__ void st4(double* p, double a, double b, double c) {
    reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2*>(p)[1] = make_double2(c, 0.0);
}

// Per-row contribution to an inner product and its warp sum: float-float in
// the FP32 path (no FP64 instructions until one conversion per warp), plain
// FP64 in the FP64 path.
template <typename T>
struct Partial;

template <>
struct Partial<float> {
    FF v;
    static __device__ __forceinline__ Partial zero() { return Partial{FF{0.f, 0.f}}; }
};

template <>
struct Partial<double> {
    double v;
    static __device__ __forceinline__ Partial zero() { return Partial{0.0}; }
};

__device__ __forceinline__ Partial<float> dot3_partial(float a0, float a1, float a2, float b0, float b1, float b2) {
    const float a[3] = {a0, a1, a2}, b[3] = {b0, b1, b2};
    return Partial<float>{ff_dot3(a, b)};
}

__device__ __forceinline__ Partial<double> dot3_partial(double a0, double a1, double a2, double b0, double b1,
                                                        double b2) {
    return Partial<double>{a0 * b0 + a1 * b1 + a2 * b2};
}

__device__ __forceinline__ double warp_sum_partial(Partial<float> p) { return ff_warp_sum(p.v); }

__device__ __forceinline__ double warp_sum_partial(Partial<double> p) {
    double v = p.v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// step coefficients in the kernel's precision
__device__ __forceinline__ void coeffs(const ProbScal* sc, float& a, float& b) {
    a = sc->alpha_f;
    b = sc->beta_f;
}
__device__ __forceinline__ void coeffs(const ProbScal* sc, double& a, double& b) {
    a = sc->alpha;
    b = sc->beta;
}

// z_bj = D^{-1} r for one row: D^{-1} row-major 3x3, its entry e of every row
// stored contiguously (entry e of row `row` at di[e * np + row], np = npad32(n)),
// so a warp's load of one entry is one contiguous 32-row run
template <typename T>
__device__ __forceinline__ void apply_dinv(const T* __restrict__ di, size_t np, int row, const T (&r)[3], T (&z)[3]) {
    T m[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) m[e] = di[e * np + row];
#pragma unroll
    for (int i = 0; i < 3; ++i) z[i] = m[3 * i] * r[0] + m[3 * i + 1] * r[1] + m[3 * i + 2] * r[2];
}

// ---- PCG in single-reduction form --------------------------------------------
// Paper §3 Eq. 12: the Newton system K dx = -g is SPD and solved by
// preconditioned conjugate gradients.  The recurrences are those of the
// single-reduction form of PCG (Chronopoulos and Gear, "s-step iterative
// methods for symmetric linear systems", J. Comput. Appl. Math. 1989): with
// u = M^{-1} r and w = K u,
//   gamma = (r, u), delta = (w, u);  beta = gamma / gamma_old,
//   alpha = gamma / (delta - beta gamma / alpha_old)   (first: beta = 0,
//   alpha = gamma / delta);  p = u + beta p, s = w + beta s,
//   dx += alpha p, r -= alpha s,
// so an iteration needs ONE global reduction (gamma, delta and |r|^2 together,
// in the SpMV) where the textbook form needs two; the update and the coarse
// correction are row-local.  M^{-1} = D^{-1} (3x3 block Jacobi), or
// D^{-1} + P Ahat P^T with the coarse correction (two-level).
//
// Kernels of one iteration, over every problem of the descriptor table (a
// block is one (problem, tile) unit and returns at once for an inactive problem):
//   [coarse product e = Ahat r_c per mesh]
//   k_pcg_correct: u = zb + P e                      (two-level problems only)
//   k_pcg_spmv:    w = K u (neighbour u gathered), partials of (r,u), (w,u),
//                  (r,r); the last tile of a problem tests convergence
//                  (|r| <= tol |r0| or the iteration cap) and sets alpha, beta
//   k_pcg_update:  p, s, dx, r as above; zb = D^{-1} r; u = zb (block Jacobi) or
//                  the restriction partials of r (two-level)
// Kernel boundaries order every write before the next kernel's reads, so no
// block ever waits on another.

// r = -g, dx = p = s = 0, zb = D^{-1} r; u = zb, or (two-level, coarse_b[b])
// the restriction partials of r for the first coarse product; |r0|^2.
template <typename T>
__global__ void k_pcg_init(ElemArgs A, double tol2, int maxit, const double* __restrict__ tol2_b,
                           const int* __restrict__ coarse_b) {
    const int b = blockIdx.y;
    if (!A.slot.active[b]) return;
    const int n = A.mesh.n;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const bool coarse = coarse_b && coarse_b[b];
    double v[1] = {0.0};
    float r32[3] = {0.f, 0.f, 0.f};
    if (row < n) {
        const double* g = A.slot.g + ((size_t)b * n + row) * 3;
        const T* di = (const T*)A.slot.dinv + (size_t)b * 9 * npad32(n);
        T* rec = vecp<T>(A.slot, b, kOffRec, n);
        const size_t np = npad32(n);
        const T r[3] = {(T)(-g[0]), (T)(-g[1]), (T)(-g[2])};
        T z[3];
        apply_dinv(di, np, row, r, z);
        st4(rec_field(rec, np, kRecDX, row), (T)0, (T)0, (T)0);
        st4(rec_field(rec, np, kRecR, row), r[0], r[1], r[2]);
        st4(rec_field(rec, np, kRecP, row), (T)0, (T)0, (T)0);
        st4(rec_field(rec, np, kRecS, row), (T)0, (T)0, (T)0);
        st4(rec_field(rec, np, kRecW, row), (T)0, (T)0, (T)0);
        st4(rec_field(rec, np, kRecZB, row), z[0], z[1], z[2]);
        if (!coarse) st4(vecp<T>(A.slot, b, kOffNB, n) + 4 * (size_t)row, z[0], z[1], z[2]);
        v[0] = (double)r[0] * (double)r[0] + (double)r[1] * (double)r[1] + (double)r[2] * (double)r[2];
        r32[0] = (float)r[0];
        r32[1] = (float)r[1];
        r32[2] = (float)r[2];
    }
    if (coarse) {
        __shared__ float qs[4][9];
        const int row0 = (int)(blockIdx.x * blockDim.x);
        stage_rotations(qs, row0, A.slot.aggq + (size_t)b * A.mesh.n_agg * 9, A.mesh.agg_shift, A.mesh.n_agg);
        uint16_t* bg = nullptr;
        if (A.slot.bsplit && A.mesh.agg_shift == 6)
            bg = A.slot.bsplit + (size_t)(b / kCoarseGroupSlots) * coarse_chunks(A.mesh.coarse_n) * kCoarseBChunk;
        restrict_units(r32, row < n, row, row0, A.mesh.crel, qs, A.mesh.agg_shift,
                       A.slot.rcp + (size_t)b * A.slot.rcp_stride + 6 * ((size_t)row0 / kCoarseRows), bg, b,
                       A.mesh.coarse_n);
    }
    double tot[1];
    double* part = A.slot.part + (size_t)b * A.slot.part_tiles * 4;
    if (tile_commit<1>(v, part, blockIdx.x, gridDim.x, &A.slot.sc[b].tk_init, 1, tot) && threadIdx.x == 0) {
        ProbScal* sc = &A.slot.sc[b];
        sc->rho = 0.0;
        sc->first = 1;
        sc->rr0 = tot[0];
        sc->rr = tot[0];
        sc->beta = 0.0;
        sc->alpha = 0.0;
        sc->alpha_f = 0.f;
        sc->beta_f = 0.f;
        sc->iter = 0;
        sc->tol2 = tol2_b ? tol2_b[b] : tol2;
        sc->maxit = maxit;
        sc->state = (tot[0] > 0.0 && maxit > 0) ? kActive : kConverged;
    }
}

// problem of unit u: last descriptor whose unit_begin (SpMV tiles) or
// unit_begin_u (row-local kernels' tiles, ROWU) is <= u
template <bool ROWU = false, typename T>
__device__ __forceinline__ int unit_problem(const PcgDesc<T>* __restrict__ D, int n_probs, int u) {
    int lo = 0, hi = n_probs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((ROWU ? D[mid].unit_begin_u : D[mid].unit_begin) <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Full occupancy (2048 threads per SM) matters more than registers in the FP32
// kernel: it is latency-bound on its dependent col -> neighbour loads.  The
// FP64 kernel is bound by the FP64 pipe and takes half that occupancy for the
// registers its double accumulators need (no spills).
//
// SPLIT = threads per row.  SPLIT = 1: lane l of a warp takes row l of its
// 32-row slice and walks all the row's slots.  SPLIT = 2: a warp takes 16 rows
// of a slice, lanes l and l + 16 the even and odd slots of row l (each warp
// load still covers whole 32-byte sectors: 16 lanes read 64 consecutive
// bytes), so each thread's dependent chain is half as long; the two halves
// are added with one shuffle.  The autotuner picks the tile and SPLIT.
template <typename T, int TILE, int SPLIT>
__global__ void __launch_bounds__(TILE * SPLIT, (sizeof(T) == 4 ? 2048 : 1024) / (TILE * SPLIT))
    k_pcg_spmv(const PcgDesc<T>* __restrict__ D, int n_probs) {
    // prologue on data no kernel of the iteration writes (the descriptor table
    // and the matrix structure), overlapping the previous kernel's drain
    const int u = blockIdx.x;
    const PcgDesc<T>& d = D[unit_problem(D, n_probs, u)];
    ProbScal* sc = d.sc;
    const int tile = u - d.unit_begin;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // row of this thread and its first slot (parity) within the row
    const int half = SPLIT == 2 ? (lane >> 4) : 0;
    const int rs = SPLIT == 2 ? ((warp & 1) << 4) + (lane & 15) : lane;   // row within the slice
    const int row = tile * TILE + (SPLIT == 2 ? (warp >> 1) * 32 : warp * 32) + rs;
    const bool valid = row < d.n_rows;
    int base = 0, w = 0;
    if (valid) {
        const int s = row >> 5;
        base = __ldg(d.slice_ptr + s);
        w = (__ldg(d.slice_ptr + s + 1) - base) >> 5;
    }
    pdl_wait();
    pdl_trigger();
    if (sc->state != kActive) return;
    T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll 4
    for (int k = half; k < w; k += SPLIT) {
        const int g = base + (k << 5);
        const int c = __ldcs(d.col + g + rs);
        if (c >= 0) {
            const T* vv = d.val + (size_t)g * 9 + rs;
            T q[3];
            ld4(d.nb + 4 * (size_t)c, q);
            a0 += __ldcs(vv) * q[0] + __ldcs(vv + 32) * q[1] + __ldcs(vv + 64) * q[2];
            a1 += __ldcs(vv + 96) * q[0] + __ldcs(vv + 128) * q[1] + __ldcs(vv + 160) * q[2];
            a2 += __ldcs(vv + 192) * q[0] + __ldcs(vv + 224) * q[1] + __ldcs(vv + 256) * q[2];
        }
    }
    if (SPLIT == 2) {   // the odd slots' half (lanes 16-31) into the even half
        a0 += __shfl_xor_sync(0xffffffffu, a0, 16);
        a1 += __shfl_xor_sync(0xffffffffu, a1, 16);
        a2 += __shfl_xor_sync(0xffffffffu, a2, 16);
    }
    // epilogue at uniform control flow with short live ranges (the kernel runs
    // at 32 registers): each partial is reduced over the warp as soon as it is
    // formed; rows past the end and the second half of a split row add zeros
    const bool owner = valid && half == 0;
    if (!owner) a0 = a1 = a2 = 0;
    T ur[3] = {0, 0, 0};
    const size_t np = npad32(d.n_rows);
    if (owner) {
        ld4(d.nb + 4 * (size_t)row, ur);
        st4(rec_field(d.rec, np, kRecW, row), a0, a1, a2);
    }
    double v[3];
    v[1] = warp_sum_partial(dot3_partial(a0, a1, a2, ur[0], ur[1], ur[2]));
    T r[3] = {0, 0, 0};
    if (owner) ld4(rec_field(d.rec, np, kRecR, row), r);
    v[0] = warp_sum_partial(dot3_partial(r[0], r[1], r[2], ur[0], ur[1], ur[2]));
    v[2] = warp_sum_partial(dot3_partial(r[0], r[1], r[2], r[0], r[1], r[2]));
    double tot[3];
    if (tile_commit<3>(v, d.part, tile, d.n_tiles, &sc->tk_a, 0, tot, true) && threadIdx.x == 0) {
        const double gamma = tot[0], delta = tot[1];
        sc->rr = tot[2];
        if (!(tot[2] > sc->tol2 * sc->rr0)) {   // |r| at target: dx is the solve's result
            sc->state = kConverged;
        } else if (sc->iter >= sc->maxit) {
            sc->state = kMaxIter;
        } else {
            double beta = 0.0, den = delta;
            if (!sc->first) {
                beta = gamma / sc->rho;
                den = delta - beta * gamma / sc->alpha;
            }
            if (gamma > 0.0 && den > 0.0 && isfinite(gamma) && isfinite(den)) {
                sc->alpha = gamma / den;
                sc->beta = beta;
                sc->rho = gamma;
                sc->first = 0;
                sc->iter = sc->iter + 1;
            } else {   // breakdown (u orthogonal to r, or K / M lost definiteness along u): keep dx
                sc->alpha = 0.0;
                sc->beta = 0.0;
                sc->state = kConverged;
            }
            sc->alpha_f = (float)sc->alpha;
            sc->beta_f = (float)sc->beta;
        }
    }
}

template <typename T, int TILE>
__global__ void __launch_bounds__(TILE) k_pcg_update(const PcgDesc<T>* __restrict__ D, int n_probs) {
    __shared__ float qs[4][9];
    const int u = blockIdx.x;   // prologue: descriptor and aggregate rotations (fixed during the solve)
    const PcgDesc<T>& d = D[unit_problem<true>(D, n_probs, u)];
    ProbScal* sc = d.sc;
    const int tile = u - d.unit_begin_u;
    const int row = tile * TILE + threadIdx.x;
    const bool coarse = d.coarse != 0;
    if (coarse) stage_rotations(qs, tile * TILE, d.aggq, d.agg_shift, d.coarse_n / 6);
    pdl_wait();
    pdl_trigger();
    if (sc->state != kActive) return;   // block-uniform
    T alpha, beta;
    coeffs(sc, alpha, beta);
    float r32[3] = {0.f, 0.f, 0.f};
    if (row < d.n_rows) {
        const size_t np = npad32(d.n_rows);
        T uu[3], ww[3], pp[3], ss[3], dx[3], r[3], z[3];
        ld4(d.nb + 4 * (size_t)row, uu);
        ld4(rec_field(d.rec, np, kRecW, row), ww);
        ld4(rec_field(d.rec, np, kRecP, row), pp);
        ld4(rec_field(d.rec, np, kRecS, row), ss);
        ld4(rec_field(d.rec, np, kRecDX, row), dx);
        ld4(rec_field(d.rec, np, kRecR, row), r);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            pp[i] = fma(beta, pp[i], uu[i]);
            ss[i] = fma(beta, ss[i], ww[i]);
            dx[i] = fma(alpha, pp[i], dx[i]);
            r[i] = fma(-alpha, ss[i], r[i]);
        }
        apply_dinv(d.dinv, np, row, r, z);
        st4(rec_field(d.rec, np, kRecP, row), pp[0], pp[1], pp[2]);
        st4(rec_field(d.rec, np, kRecS, row), ss[0], ss[1], ss[2]);
        st4(rec_field(d.rec, np, kRecDX, row), dx[0], dx[1], dx[2]);
        st4(rec_field(d.rec, np, kRecR, row), r[0], r[1], r[2]);
        st4(rec_field(d.rec, np, kRecZB, row), z[0], z[1], z[2]);
        if (!coarse) st4(d.nb + 4 * (size_t)row, z[0], z[1], z[2]);   // u = D^{-1} r
        r32[0] = (float)r[0];
        r32[1] = (float)r[1];
        r32[2] = (float)r[2];
    }
    if (coarse)   // u is finished by k_pcg_correct after the coarse product
        restrict_units(r32, row < d.n_rows, row, tile * TILE, d.crel, qs, d.agg_shift,
                       d.rcp + 6 * ((size_t)tile * TILE / kCoarseRows), d.bunit, d.bslot, d.coarse_n);
}

// Coarse solve of the two-level preconditioner: e = A_c^{-1} r_c for the
// problems d0 .. d0+nd-1 of the table (one mesh: one A_c^{-1}), NP (8 or 16,
// the smallest that holds them, 16 per grid.z slice beyond) per block.  r_c is the problem's restriction partials when an aggregate
// is one 64-row unit, else their per-aggregate sums (k_coarse_rc).  Block (grid.x, grid.y): 32 rows of A_c^{-1} over one
// slice of kCoarseKC columns; the slice of r_c sits in shared memory as
// [problem][column], a warp takes four rows in turn with its lanes striding the
// columns (coalesced rows of A_c^{-1}), then shuffles each problem's sum down
// in a fixed order.  Slice products go to ec[slice][row]; k_pcg_correct adds
// the slices in order.
// r_c of aggregates larger than one 64-row unit: the units' partials added in
// unit order, for the problems d0 .. d0+nd-1 (grid.y) of one mesh.
template <typename T>
__global__ void k_coarse_rc(const PcgDesc<T>* __restrict__ D, int d0, int nd) {
    const PcgDesc<T>& q = D[d0 + blockIdx.y];
    const bool coarse = q.coarse != 0;
    ProbScal* sc = q.sc;
    pdl_wait();
    pdl_trigger();
    if (!coarse || sc->state != kActive) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= q.coarse_n) return;
    const int a = k / 6, comp = k - 6 * a;
    const int ush = q.agg_shift - 6;
    const int n_units = (q.n_rows + kCoarseRows - 1) / kCoarseRows;
    const int u1 = min(n_units, (a + 1) << ush);
    float v = 0.f;
    for (int u = a << ush; u < u1; ++u) v += q.rcp[6 * (size_t)u + comp];
    q.rcs[k] = v;
    if (q.bagg) coarse_b_store(q.bagg, q.bslot % kCoarseGroupSlots, k, v);
}

template <typename T, int NP>
__global__ void __launch_bounds__(256) k_coarse_gemm(const float* __restrict__ Ainv, int N, int ld,
                                                     const PcgDesc<T>* __restrict__ D, int d0, int nd) {
    __shared__ __align__(16) float rs[NP * kCoarseKC];
    __shared__ const PcgDesc<T>* dp[NP];
    __shared__ int any;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int ks = blockIdx.y, pg = blockIdx.z;
    const PcgDesc<T>* mine = nullptr;   // prologue: descriptors are fixed during the solve
    ProbScal* msc = nullptr;
    if (t < NP && pg * NP + t < nd && D[d0 + pg * NP + t].coarse) {
        mine = &D[d0 + pg * NP + t];
        msc = mine->sc;
    }
    if (t == 0) any = 0;
    pdl_wait();
    pdl_trigger();
    __syncthreads();
    if (t < NP) {
        const PcgDesc<T>* p = nullptr;
        if (mine && msc->state == kActive) p = mine;
        dp[t] = p;
        if (p) atomicOr(&any, 1);
    }
    __syncthreads();
    if (!any) return;
    const int k0 = ks * kCoarseKC, klen = min(kCoarseKC, N - k0);
    constexpr int kQ = kCoarseKC / 4;
    for (int idx = t; idx < NP * kQ; idx += 256) {   // r_c slice, 16-byte loads
        const int p = idx / kQ, kk = 4 * (idx - p * kQ);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        const PcgDesc<T>* q = dp[p];
        if (q && kk < klen) {
            const float* src = q->rc + k0 + kk;
            if (kk + 3 < klen) {
                v = *reinterpret_cast<const float4*>(src);
            } else {
                v.x = src[0];
                if (kk + 1 < klen) v.y = src[1];
                if (kk + 2 < klen) v.z = src[2];
            }
        }
        *reinterpret_cast<float4*>(&rs[p * kCoarseKC + kk]) = v;
    }
    __syncthreads();
    // four rows per warp at once, four columns per lane (16-byte loads of rows
    // padded to ld floats; the padding is zero): each r_c value read from
    // shared memory feeds four rows
    for (int pass = 0; pass < kCoarseRowPasses; ++pass) {
        const int row0 = (blockIdx.x * kCoarseRowPasses + pass) * 32 + warp * 4;
        if (row0 >= N) break;
        float acc[4][NP];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int p = 0; p < NP; ++p) acc[i][p] = 0.f;
        const float* arow = Ainv + (size_t)row0 * ld + k0;
#pragma unroll 2
        for (int kk = 4 * lane; kk < klen; kk += 128) {
            float4 a4[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                a4[i] = row0 + i < N ? __ldcs(reinterpret_cast<const float4*>(arow + (size_t)i * ld + kk))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const float4 rv = *reinterpret_cast<const float4*>(&rs[p * kCoarseKC + kk]);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float t = acc[i][p];
                    t = fmaf(a4[i].x, rv.x, t);
                    t = fmaf(a4[i].y, rv.y, t);
                    t = fmaf(a4[i].z, rv.z, t);
                    acc[i][p] = fmaf(a4[i].w, rv.w, t);
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int p = 0; p < NP; ++p) acc[i][p] += __shfl_xor_sync(0xffffffffu, acc[i][p], o);
        // lane l writes (row i, problem p) = (l / NP, l % NP) + 32 / NP rows per step
#pragma unroll
        for (int h = 0; h < 4 * NP / 32; ++h) {
            const int e = lane + 32 * h, i = e / NP, p = e % NP;
            float mine = 0.f;
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                for (int pp = 0; pp < NP; ++pp)
                    if (ii == i && pp == p) mine = acc[ii][pp];
            if (row0 + i < N && dp[p]) dp[p]->ec[(size_t)ks * N + row0 + i] = mine;
        }
    }
}

// u_i = zb_i + Q_a P_i e_a (e_a = the six coarse values of row i's aggregate,
// e_t + e_w x (X_i - c_a) turned by the aggregate's rotation), written
// to the neighbour record the next k_pcg_spmv gathers.  The block first gathers
// the slice partials of e of its aggregates (added in slice order) and their
// rotations into shared memory.  Problems without the coarse correction return
// at once (their u was written by the update).
template <typename T, int TILE>
__global__ void __launch_bounds__(TILE) k_pcg_correct(const PcgDesc<T>* __restrict__ D, int n_probs) {
    constexpr int kMaxAgg = TILE / kCoarseRows;   // aggregates a block can touch
    __shared__ float es[kMaxAgg][6];
    __shared__ float qs[kMaxAgg][9];
    __shared__ float part_e[TILE];
    // prologue on data fixed during the solve (descriptor, rest offsets, pose
    // rotations), overlapping the previous kernel's drain
    const int u = blockIdx.x;
    const PcgDesc<T>& d = D[unit_problem<true>(D, n_probs, u)];
    if (!d.coarse || d.ctc) return;   // block Jacobi, or corrected by the fused tensor-core kernel
    ProbScal* sc = d.sc;
    const int tile = u - d.unit_begin_u;
    const int row = tile * TILE + threadIdx.x;
    const int a0 = (tile * TILE) >> d.agg_shift;
    const int n_agg = d.coarse_n / 6;
    const int n_ks = (d.coarse_n + kCoarseKC - 1) / kCoarseKC;
    float4 off = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row < d.n_rows) off = d.crel[row];
    if ((int)threadIdx.x < kMaxAgg * 9) {
        const int ai = threadIdx.x / 9, q = threadIdx.x % 9, a = a0 + ai;
        qs[ai][q] = a < n_agg ? d.aggq[9 * a + q] : 0.f;
    }
    pdl_wait();
    pdl_trigger();
    if (sc->state != kActive) return;   // block-uniform: before any barrier
    // the row's own load goes out first, so its latency overlaps the staging
    T z[3] = {(T)0, (T)0, (T)0};
    if (row < d.n_rows) ld4(rec_field(d.rec, npad32(d.n_rows), kRecZB, row), z);
    // slice partials of e, one load per thread, then added in slice order
    for (int idx = threadIdx.x; idx < kMaxAgg * 6 * n_ks && idx < TILE; idx += TILE) {
        const int ks = idx / (kMaxAgg * 6), r = idx - ks * kMaxAgg * 6, a = a0 + r / 6;
        part_e[idx] = a < n_agg ? d.ec[(size_t)ks * d.coarse_n + 6 * a + r % 6] : 0.f;
    }
    __syncthreads();
    if ((int)threadIdx.x < kMaxAgg * 6) {
        float v = 0.f;
        for (int ks = 0; ks < n_ks; ++ks) {
            const int idx = ks * kMaxAgg * 6 + threadIdx.x;
            const int a = a0 + (int)threadIdx.x / 6;
            v += idx < TILE ? part_e[idx]
                            : (a < n_agg ? d.ec[(size_t)ks * d.coarse_n + 6 * a + threadIdx.x % 6] : 0.f);
        }
        es[threadIdx.x / 6][threadIdx.x % 6] = v;
    }
    __syncthreads();
    if (row < d.n_rows) {
        if (off.w != 0.f) {
            const int ai = (row >> d.agg_shift) - a0;
            const float* e = es[ai];
            const float* Q = qs[ai];
            const float l0 = e[0] + (e[4] * off.z - e[5] * off.y);
            const float l1 = e[1] + (e[5] * off.x - e[3] * off.z);
            const float l2 = e[2] + (e[3] * off.y - e[4] * off.x);
#pragma unroll
            for (int i = 0; i < 3; ++i) z[i] += (T)(Q[3 * i] * l0 + Q[3 * i + 1] * l1 + Q[3 * i + 2] * l2);
        }
        st4(d.nb + 4 * (size_t)row, z[0], z[1], z[2]);
    }
}

// Each launch may start while the previous kernel of the stream drains
// (programmatic stream serialization); the kernels wait on it first thing.
template <typename T, int TILE, int SPLIT>
cudaError_t launch_pcg_iters_t(const PcgDesc<T>* descs, int n_probs, int n_units, int n_units_u, int iters,
                               const CoarseJob* jobs, int n_jobs, cudaStream_t s) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_units);
    cfg.blockDim = dim3(TILE);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchConfig_t cfg_u = cfg;   // row-local kernels: their own fixed tile
    cfg_u.gridDim = dim3(n_units_u);
    cfg_u.blockDim = dim3(kRowTileU);
    cudaLaunchConfig_t cfg_s = cfg;   // the SpMV: SPLIT threads per row
    cfg_s.blockDim = dim3(TILE * SPLIT);
    for (int i = 0; i < iters; ++i) {
        cudaError_t e;
        if (n_jobs > 0) {   // two-level: finish u of the current residual first
            bool any_cuda_core = false;
            for (int j = 0; j < n_jobs; ++j) {
                if (jobs[j].agg_units > 1) {   // per-aggregate sums of the unit partials
                    cudaLaunchConfig_t rc = cfg;
                    rc.gridDim = dim3((jobs[j].N + 255) / 256, jobs[j].nd);
                    rc.blockDim = dim3(256);
                    e = cudaLaunchKernelEx(&rc, k_coarse_rc<T>, descs, jobs[j].d0, jobs[j].nd);
                    if (e != cudaSuccess) return e;
                }
                if (jobs[j].Abf) {   // tensor cores, BF16 A_c^{-1}: product and correction in one kernel
                    e = launch_coarse_fused<T>(cfg, jobs[j], descs, nullptr);
                    if (e != cudaSuccess) return e;
                    continue;
                }
                any_cuda_core = true;
                cudaLaunchConfig_t gc = cfg;
                const int np = jobs[j].nd <= 8 ? 8 : 16;
                gc.gridDim = dim3((jobs[j].N + 32 * kCoarseRowPasses - 1) / (32 * kCoarseRowPasses),
                                  (jobs[j].N + kCoarseKC - 1) / kCoarseKC, (jobs[j].nd + np - 1) / np);
                gc.blockDim = dim3(256);
                if (np == 8)
                    e = cudaLaunchKernelEx(&gc, k_coarse_gemm<T, 8>, jobs[j].Ainv, jobs[j].N, coarse_ld(jobs[j].N),
                                           descs, jobs[j].d0, jobs[j].nd);
                else
                    e = cudaLaunchKernelEx(&gc, k_coarse_gemm<T, 16>, jobs[j].Ainv, jobs[j].N, coarse_ld(jobs[j].N),
                                           descs, jobs[j].d0, jobs[j].nd);
                if (e != cudaSuccess) return e;
            }
            if (any_cuda_core) {
                e = cudaLaunchKernelEx(&cfg_u, k_pcg_correct<T, kRowTileU>, descs, n_probs);
                if (e != cudaSuccess) return e;
            }
        }
        e = cudaLaunchKernelEx(&cfg_s, k_pcg_spmv<T, TILE, SPLIT>, descs, n_probs);
        if (e != cudaSuccess) return e;
        e = cudaLaunchKernelEx(&cfg_u, k_pcg_update<T, kRowTileU>, descs, n_probs);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace

void launch_pcg_init(const ElemArgs& a, int B, int tile_rows, double tol2, int maxit, const double* tol2_b,
                     const int* coarse_b, cudaStream_t s) {
    dim3 grid((a.mesh.n + tile_rows - 1) / tile_rows, B);
    if (a.slot.prec == 1) k_pcg_init<float><<<grid, tile_rows, 0, s>>>(a, tol2, maxit, tol2_b, coarse_b);
    else k_pcg_init<double><<<grid, tile_rows, 0, s>>>(a, tol2, maxit, tol2_b, coarse_b);
}

template <typename T>
cudaError_t launch_pcg_iters(const PcgDesc<T>* descs, int n_probs, int n_units, int n_units_u, int tile_rows,
                             int split, int iters, const CoarseJob* jobs, int n_jobs, cudaStream_t s) {
#define MFEM_PCG_CASE(TR, SP)                                                                                  \
    if (tile_rows == TR && split == SP)                                                                        \
        return launch_pcg_iters_t<T, TR, SP>(descs, n_probs, n_units, n_units_u, iters, jobs, n_jobs, s);
    MFEM_PCG_CASE(64, 1)
    MFEM_PCG_CASE(128, 1)
    MFEM_PCG_CASE(256, 1)
    MFEM_PCG_CASE(64, 2)
    MFEM_PCG_CASE(128, 2)
    MFEM_PCG_CASE(256, 2)
#undef MFEM_PCG_CASE
    return cudaErrorInvalidValue;
}

bool pcg_tile_supported(int tile_rows) { return tile_rows == 64 || tile_rows == 128 || tile_rows == 256; }

cudaError_t launch_coarse_only(const PcgDesc<float>* descs, int n_probs, const CoarseJob* job, float* e_out,
                               cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.stream = s;
    if (job->Abf) return launch_coarse_fused<float>(cfg, *job, descs, e_out);
    const int np = job->nd <= 8 ? 8 : 16;
    cfg.gridDim = dim3((job->N + 32 * kCoarseRowPasses - 1) / (32 * kCoarseRowPasses),
                       (job->N + kCoarseKC - 1) / kCoarseKC, (job->nd + np - 1) / np);
    cfg.blockDim = dim3(256);
    (void)n_probs;
    if (np == 8)
        return cudaLaunchKernelEx(&cfg, k_coarse_gemm<float, 8>, job->Ainv, job->N, coarse_ld(job->N), descs,
                                  job->d0, job->nd);
    return cudaLaunchKernelEx(&cfg, k_coarse_gemm<float, 16>, job->Ainv, job->N, coarse_ld(job->N), descs, job->d0,
                              job->nd);
}

template cudaError_t launch_pcg_iters<float>(const PcgDesc<float>*, int, int, int, int, int, int, const CoarseJob*,
                                             int, cudaStream_t);
template cudaError_t launch_pcg_iters<double>(const PcgDesc<double>*, int, int, int, int, int, int,
                                              const CoarseJob*, int, cudaStream_t);

}  // namespace mfem
