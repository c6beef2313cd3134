// Device-side structures and helpers shared by the kernels of the pose solver.
//
// Reductions are deterministic: every per-problem sum is formed per fixed tile
// of rows (or tets), tile partials are written to global memory, and the last
// tile to finish (a ticket counter) adds the partials in tile order.  The result
// therefore does not depend on the grid, on scheduling, or on which other
// problems share the launch.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace mfem {

constexpr int kWarp = 32;
constexpr int kSliceRows = 32;       // rows per SELL slice (one warp)
constexpr int kTetTile = 128;        // tets per element-kernel block
constexpr int kRowTile = 256;        // rows per block in row kernels other than PCG
constexpr int kRowTileU = 256;       // rows per block of the PCG update and correction kernels
// Element blocks of one tet: the upper 3x3 blocks K_ab (a <= b) of the
// symmetric 12x12 element matrix in the order (0,0) (0,1) (0,2) (0,3) (1,1)
// (1,2) (1,3) (2,2) (2,3) (3,3); a diagonal block is symmetric and keeps its six
// upper entries (xx, yy, zz, yz, xz, xy), an off-diagonal block its nine
// (row-major) and one unused value, so that every block starts on an even
// element (8-byte loads in FP32, 16-byte in FP64): 84 values per tet.  The
// element-block array carries kKePad values past its last record (a reader
// may load ten values from the last diagonal block).
constexpr int kKe = 84;
constexpr int kKePad = 4;
__host__ __device__ __forceinline__ int ke_offset(int a, int b) {   // a <= b
    const int p = a * 4 - (a * (a - 1)) / 2 + (b - a);              // block index
    return 10 * p - 4 * (a + (b > a ? 1 : 0));                       // minus the diagonal blocks' 4 saved
}

// Per-problem PCG vector area, in elements of the PCG type, rows padded to 32
// (np = npad32(n)): the neighbour record nb[np][4] = (u.xyz, 0) -- the
// preconditioned residual, the one vector the SpMV gathers from neighbours (16
// bytes in FP32) -- then six row fields of [np][4] each, field-major (a warp's
// access to one field of 32 consecutive rows is one contiguous run): the Newton
// increment dx, the residual r, the search direction p, s = K p, w = K u, and
// the block-Jacobi part zb of u.  Field f (kRecDX .. kRecZB) of row i is at
// rec + f * np + 4 i (rec_field).
constexpr int kVecStride = 28;                 // times npad32(n)
constexpr int kOffNB = 0, kOffRec = 4;
constexpr int kRecDX = 0, kRecR = 4, kRecP = 8, kRecS = 12, kRecW = 16, kRecZB = 20;
__host__ __device__ __forceinline__ size_t npad32(int n) { return ((size_t)n + 31) & ~(size_t)31; }
template <typename T>
__host__ __device__ __forceinline__ T* rec_field(T* rec, size_t np, int f, size_t row) {
    return rec + (size_t)f * np + 4 * row;
}

// Problem states (PCG)
enum : int { kIdle = 0, kActive = 1, kConverged = 2, kMaxIter = 3 };

// Per-problem scalars.  Tickets are reset to 0 by the tile that completes them.
struct ProbScal {
    double rho, alpha, beta, rr0, rr, tol2;   // rho: the last (r, u); alpha, beta: the next step's
    double gnorm2, energy, slope, energy_trial;
    double alpha_ls, pad0;
    float alpha_f, beta_f;   // FP32 copies of alpha and beta for the FP32 kernels
    int iter, state, maxit, active;
    unsigned tk_a, tk_b, tk_g, tk_e, tk_s, tk_init, tk_c;
    int first;   // the next reduction is the solve's first (beta = 0, alpha = (r,u) / (w,u))
};

// Two-level preconditioner constants: restriction partials are formed per unit
// of 64 rows (aggregates hold a power-of-two multiple of 64 vertices) and the
// coarse product is split into slices of kCoarseKC columns of A_c^{-1}.
constexpr int kCoarseRows = 64;
constexpr int kCoarseKC = 256;
constexpr int kCoarseRowPasses = 1;   // 32-row passes per block of the coarse product (measured: 4 is slower)
// row stride of the stored A_c^{-1} (rows padded with zeros to 32 floats)
__host__ __device__ __forceinline__ int coarse_ld(int N) { return (N + 31) & ~31; }

// B operand of the tensor-core coarse product, per group of kCoarseGroupSlots
// request slots of a context: each slot's coarse residual r_c split exactly
// into three BF16 parts (r = hi + mid + lo, 3 x 8 significand bits) that are
// rows p, 16 + p, 32 + p (p = slot mod 16) of an N = 48 operand, stored per
// chunk of kTcKC columns in the MMA's no-swizzle K-major core-matrix layout
// (K step of 16 columns: 1536 bytes; 8-row group: 256 bytes; K-adjacent core
// matrices 128 bytes apart; row: 16 bytes), so that one 1-D bulk copy lands
// a whole chunk.  Columns past N stay zero.
constexpr int kTcKC = 128;
constexpr int kCoarseGroupSlots = 16;
constexpr int kCoarseBRows = 3 * kCoarseGroupSlots;            // 48
constexpr int kCoarseBChunk = kCoarseBRows * kTcKC;            // elements per chunk
__host__ __device__ __forceinline__ int coarse_chunks(int N) { return (N + kTcKC - 1) / kTcKC; }
__host__ __device__ __forceinline__ size_t coarse_b_offset(int row, int k) {
    const int ch = k / kTcKC, kk = k % kTcKC;
    const int s = kk >> 4, j2 = (kk >> 3) & 1, c = kk & 7, g = row >> 3, r = row & 7;
    return (size_t)ch * kCoarseBChunk + s * (kCoarseBRows * 16) + g * 128 + j2 * 64 + r * 8 + c;
}
// Store component k of slot p's coarse residual into its group's B operand.
__device__ __forceinline__ void coarse_b_store(uint16_t* __restrict__ grp, int p, int k, float v) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
    grp[coarse_b_offset(p, k)] = __bfloat16_as_ushort(h);
    grp[coarse_b_offset(kCoarseGroupSlots + p, k)] = __bfloat16_as_ushort(m);
    grp[coarse_b_offset(2 * kCoarseGroupSlots + p, k)] = __bfloat16_as_ushort(l);
}

// One PCG problem (a pose of a mesh) in a descriptor table.
template <typename T>
struct PcgDesc {
    const int* slice_ptr;  // [n_slices+1] first slot of each slice
    const int* col;        // [slots] column block or -1
    const T* val;          // [slots/32][9][32]
    const T* dinv;         // [9][npad32(n)] inverse diagonal blocks, entry-major
    T* nb;                 // [n][4] neighbour records (u)
    T* rec;                // the six row fields (dx, r, p, s, w, zb), field-major (rec_field)
    double* part;          // [tiles][4] tile partials
    ProbScal* sc;
    int n_rows, n_tiles, unit_begin;   // the SpMV's tiles (autotuned rows per block)
    int n_tiles_u;                     // the row-local kernels' tiles (kRowTileU rows per block)
    // two-level preconditioner (coarse = 0: block Jacobi only for this solve)
    const float4* crel;    // [n] rest offset from the aggregate centroid, w = 1 free / 0 pin
    const float* aggq;     // [n_agg][9] the problem's aggregate rotations (row-major)
    float* rcp;            // [ceil(n/64)][6] restriction partials per 64-row unit
    float* rcs;            // [coarse_n] per-aggregate sums of rcp (aggregates over 64 rows)
    const float* rc;       // the coarse residual read by the coarse product: rcp or rcs
    float* ec;             // [ceil(coarse_n / kCoarseKC)][coarse_n] partial coarse corrections
    // tensor-core path: the slot's group of the B operand (null on the CUDA-core
    // path); the restriction writes it where an aggregate is one 64-row unit
    // (bunit), else the per-aggregate sum does (bagg)
    uint16_t* bunit;
    uint16_t* bagg;
    int bslot;             // the problem's request slot in its context
    int ctc;               // 1: coarse product and correction by the fused tensor-core kernel
    int coarse, agg_shift, coarse_n;
    int unit_begin_u;
};

// Programmatic dependent launch: wait for the preceding grid of the stream to
// complete and its writes to be visible; let the next grid start launching.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *(volatile const int*)p; }

// Sum NV doubles over the block with a fixed shuffle/shared-memory tree.  The
// result is valid in thread 0.  All threads of the block must call it.  With
// warp_done the values are already warp sums, held by lane 0 of each warp.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], bool warp_done = false) {
    __shared__ double sm[32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    if (!warp_done) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int i = 0; i < NV; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) sm[warp][i] = v[i];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] = lane < nwarps ? sm[lane][i] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int i = 0; i < NV; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
    __syncthreads();
}

// ---- float-float inner products -------------------------------------------
// GB300 issues FP64 at a small fraction of its FP32 rate, so the FP32 PCG path
// forms its inner products with error-free transformations in FP32 instead of
// FP64 instructions: two-product by fused multiply-add (Dekker, "A floating-point
// technique for extending the available precision", 1971) and two-sum (Knuth,
// TAOCP vol. 2, 4.2.2).  A (hi, lo) pair carries about 48 significant bits; it
// becomes one double per warp.
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return FF{s, e};
}

__device__ __forceinline__ FF ff_add(FF x, FF y) {
    const FF s = ff_two_sum(x.hi, y.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    const float hi = __fadd_rn(s.hi, e);
    return FF{hi, __fsub_rn(e, __fsub_rn(hi, s.hi))};
}

__device__ __forceinline__ FF ff_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return FF{p, __fmaf_rn(a, b, -p)};
}

// a0*b0 + a1*b1 + a2*b2 as a float-float
__device__ __forceinline__ FF ff_dot3(const float (&a)[3], const float (&b)[3]) {
    return ff_add(ff_add(ff_prod(a[0], b[0]), ff_prod(a[1], b[1])), ff_prod(a[2], b[2]));
}

// warp sum of float-float values (fixed xor tree), as a double in lane 0 (0 elsewhere)
__device__ __forceinline__ double ff_warp_sum(FF v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        FF w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = ff_add(v, w);
    }
    double d = 0.0;
    if ((threadIdx.x & 31) == 0) d = (double)v.hi + (double)v.lo;
    return d;
}

// Commit this block's NV partial sums for `tile` of a problem; the block that
// completes the ticket adds all tiles in order and returns true with the totals
// in `tot` (valid in thread 0 only).  part layout: [n_tiles][4], NV <= 4.
template <int NV>
__device__ __forceinline__ bool tile_commit(double (&v)[NV], double* part, int tile, int n_tiles,
                                            unsigned* ticket, int slot0, double (&tot)[NV],
                                            bool warp_done = false) {
    __shared__ int s_last;
    block_sum<NV>(v, warp_done);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) part[4 * tile + slot0 + i] = v[i];
        __threadfence();
        unsigned prev = atomicAdd(ticket, 1u);
        s_last = (prev == (unsigned)(n_tiles - 1));
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x)
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] += *(volatile double*)&part[4 * t + slot0 + i];
    block_sum<NV>(acc);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) tot[i] = acc[i];
        *ticket = 0u;
    }
    return true;
}

}  // namespace mfem
