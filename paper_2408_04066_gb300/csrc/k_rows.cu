// Row-parallel kernels: assembly of the condensed matrix (a2) with pin
// elimination (a3) and block-Jacobi inverse (a4), gradient gather, slope and
// update (a6) and permutations (a7).
//
// Paper §3, Eq. 12 and the assembly and linear-solve steps of Algorithm 1: the matrix
// sum_k W_k A_k^T H_s A_k is gathered per 3x3 block from the element blocks of
// every tet that contains both vertices, in a fixed order (deterministic, no
// atomics).  Pinned vertices (Eq. 6 C(x), §3.2 targets) are eliminated: their
// rows and columns become identity/zero and their gradient entries zero, so the
// Newton increment keeps them at x_p; the penalty form adds k_s I instead.
// External vertex forces (§4, "Collision response") enter the gradient as -f.
#include <cuda_runtime.h>

#include "kernels.h"

namespace mfem {

namespace {

// Gradient of row `row` of problem b: the element forces of its tets in fixed
// incidence order, the external force, and the pin term (zero under
// elimination, k_s (x - x_p) under the penalty form).  Writes g, returns |g|^2.
__device__ __forceinline__ double row_gradient(const ElemArgs& A, int b, int row, bool pin_r) {
    const MeshDev& M = A.mesh;
    const int n = M.n;
    // gradient of row: sum of element forces in fixed incidence order
    const double* ge = A.slot.ge + (size_t)b * M.m * 12;
    double g0 = 0, g1 = 0, g2 = 0;
    for (int ii = M.vinc_ptr[row]; ii < M.vinc_ptr[row + 1]; ++ii) {
        const int code = M.vinc[ii];
        const double* f = ge + (size_t)(code >> 2) * 12 + 3 * (code & 3);
        g0 += f[0];
        g1 += f[1];
        g2 += f[2];
    }
    if (A.fext) {  // external forces: E gains -f.x
        const double* fv = A.fext + (size_t)b * A.fext_stride + 3 * (size_t)row;
        g0 -= fv[0];
        g1 -= fv[1];
        g2 -= fv[2];
    }
    if (pin_r) {
        if (A.constraint == 0) {
            g0 = g1 = g2 = 0.0;
        } else {
            const double* x = A.slot.x + ((size_t)b * n + row) * 3;
            const double* xp = A.slot.xp + ((size_t)b * n + row) * 3;
            g0 += A.ks * (x[0] - xp[0]);
            g1 += A.ks * (x[1] - xp[1]);
            g2 += A.ks * (x[2] - xp[2]);
        }
    }
    double* gout = A.slot.g + ((size_t)b * n + row) * 3;
    gout[0] = g0;
    gout[1] = g1;
    gout[2] = g2;
    return g0 * g0 + g1 * g1 + g2 * g2;
}

// The ten values from the start of contribution `code`'s stored block (tet
// code >> 4, local vertices ((code >> 2) & 3, code & 3), either order): five
// aligned pairs
__device__ __forceinline__ void load_block(const float* __restrict__ Ke, int code, float (&v)[10]) {
    const int t = code >> 4, ea = (code >> 2) & 3, eb = code & 3;
    const float2* q = reinterpret_cast<const float2*>(Ke + (size_t)t * kKe + ke_offset(min(ea, eb), max(ea, eb)));
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float2 p = __ldg(q + i);
        v[2 * i] = p.x;
        v[2 * i + 1] = p.y;
    }
}
__device__ __forceinline__ void load_block(const double* __restrict__ Ke, int code, double (&v)[10]) {
    const int t = code >> 4, ea = (code >> 2) & 3, eb = code & 3;
    const double2* q = reinterpret_cast<const double2*>(Ke + (size_t)t * kKe + ke_offset(min(ea, eb), max(ea, eb)));
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const double2 p = __ldg(q + i);
        v[2 * i] = p.x;
        v[2 * i + 1] = p.y;
    }
}

// Add the block in the slot's orientation: a diagonal block from its six
// upper entries (xx, yy, zz, yz, xz, xy), an upper block as stored, a lower
// block transposed.
template <typename KT>
__device__ __forceinline__ void add_block(KT (&acc)[9], int code, const KT (&v)[10]) {
    const int ea = (code >> 2) & 3, eb = code & 3;
    if (ea == eb) {
        acc[0] += v[0]; acc[1] += v[5]; acc[2] += v[4];
        acc[3] += v[5]; acc[4] += v[1]; acc[5] += v[3];
        acc[6] += v[4]; acc[7] += v[3]; acc[8] += v[2];
    } else if (ea < eb) {
#pragma unroll
        for (int e = 0; e < 9; ++e) acc[e] += v[e];
    } else {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) acc[3 * i + j] += v[3 * j + i];
    }
}

// One thread per diagonal or upper slot of the sliced pattern: the slot's 3x3
// block summed from the element blocks of every tet holding both vertices (the
// contributions of a slot are sorted by tet, so the order -- and every bit of
// the result -- is the same as a row-by-row gather), pin elimination or the
// penalty term, written to the slot and, transposed, to its mirror slot (the
// lower block sums the transposes of the same blocks in the same order: the
// same bits as gathering it), and, on the diagonal, the row's block-Jacobi
// inverse.  Consecutive threads take consecutive upper slots, so the own
// writes are nearly coalesced; the mirror writes are scattered.  The gradient
// gather runs in k_gradient.
// Block Jacobi: the inverse of a 3x3 diagonal block by its cofactors, entry e
// written at di[e * np] (one run per entry).  The FP64 path forms it in FP64.
// The mixed path forms it in FP32 from the block scaled by a power of two
// (the largest entry into [0.5, 1): no overflow or underflow of the
// determinant, and the scaling is exact).  It is only the preconditioner, and
// its matrix is FP32; GB300's FP64 pipe is narrow.
__device__ __forceinline__ void block_jacobi(const double (&a)[9], double* di, size_t np) {
    const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
    const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    const double id = det != 0.0 ? 1.0 / det : 0.0;
    di[0 * np] = c00 * id;
    di[1 * np] = (a[2] * a[7] - a[1] * a[8]) * id;
    di[2 * np] = (a[1] * a[5] - a[2] * a[4]) * id;
    di[3 * np] = c01 * id;
    di[4 * np] = (a[0] * a[8] - a[2] * a[6]) * id;
    di[5 * np] = (a[2] * a[3] - a[0] * a[5]) * id;
    di[6 * np] = c02 * id;
    di[7 * np] = (a[1] * a[6] - a[0] * a[7]) * id;
    di[8 * np] = (a[0] * a[4] - a[1] * a[3]) * id;
}
__device__ __forceinline__ void block_jacobi(const float (&acc)[9], float* di, size_t np) {
    float mx = 0.f;
#pragma unroll
    for (int e = 0; e < 9; ++e) mx = fmaxf(mx, fabsf(acc[e]));
    int ex = 0;
    frexpf(mx, &ex);                       // mx = f 2^ex, f in [0.5, 1)
    const float sc = ldexpf(1.f, -ex);     // exact power of two
    float a[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) a[e] = acc[e] * sc;
    const float c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
    const float det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    // inv(acc) = sc inv(a)
    const float id = det != 0.f ? sc / det : 0.f;
    di[0 * np] = c00 * id;
    di[1 * np] = (a[2] * a[7] - a[1] * a[8]) * id;
    di[2 * np] = (a[1] * a[5] - a[2] * a[4]) * id;
    di[3 * np] = c01 * id;
    di[4 * np] = (a[0] * a[8] - a[2] * a[6]) * id;
    di[5 * np] = (a[2] * a[3] - a[0] * a[5]) * id;
    di[6 * np] = c02 * id;
    di[7 * np] = (a[1] * a[6] - a[0] * a[7]) * id;
    di[8 * np] = (a[0] * a[4] - a[1] * a[3]) * id;
}

template <typename KT>
__global__ void __launch_bounds__(kRowTile) k_assemble_slots(ElemArgs A) {
    const int b = blockIdx.y;
    if (!A.slot.active[b]) return;
    const MeshDev& M = A.mesh;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M.n_up) return;
    const int64_t gs = __ldg(M.up_slot + t);
    const int ms = __ldg(M.up_mirror + t);
    const int c = __ldg(M.col + gs);
    const int row = __ldg(M.slot_row + gs);
    const int lane = row & 31;
    const KT* Ke = (const KT*)A.slot.Ke + (size_t)b * M.m * kKe;
    KT acc[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) acc[e] = (KT)0;
    const int c0 = __ldg(M.contrib_ptr + gs), c1 = __ldg(M.contrib_ptr + gs + 1);
    // contributions four at a time, every load of the four issued first: ten
    // values (five pairs) from each block's start, whatever its kind
    int ci = c0;
    for (; ci + 3 < c1; ci += 4) {
        int code[4];
        KT v[4][10];
#pragma unroll
        for (int q = 0; q < 4; ++q) code[q] = __ldg(M.contrib + ci + q);
#pragma unroll
        for (int q = 0; q < 4; ++q) load_block(Ke, code[q], v[q]);
#pragma unroll
        for (int q = 0; q < 4; ++q) add_block(acc, code[q], v[q]);
    }
    for (; ci < c1; ++ci) {
        const int code = __ldg(M.contrib + ci);
        KT v[10];
        load_block(Ke, code, v);
        add_block(acc, code, v);
    }
    const bool diag = (c == row);
    const bool pin_r = M.pin_handle_v[row] >= 0;
    if (A.constraint == 0) {
        if (pin_r || M.pin_handle_v[c] >= 0) {
#pragma unroll
            for (int e = 0; e < 9; ++e) acc[e] = (diag && (e % 4 == 0)) ? (KT)1 : (KT)0;
        }
    } else if (diag && pin_r) {
        acc[0] += (KT)A.ks;
        acc[4] += (KT)A.ks;
        acc[8] += (KT)A.ks;
    }
    KT* val = (KT*)A.slot.val + (size_t)b * M.slots * 9;
    KT* out = val + (size_t)(gs - lane) * 9 + lane;
#pragma unroll
    for (int e = 0; e < 9; ++e) out[32 * e] = acc[e];
    if (ms >= 0) {   // the transposed block in the mirror slot (lane = its row's)
        KT* mout = val + (size_t)(ms - (c & 31)) * 9 + (c & 31);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) mout[32 * (3 * i + j)] = acc[3 * j + i];
    }
    if (diag) block_jacobi(acc, (KT*)A.slot.dinv + (size_t)b * 9 * npad32(M.n) + row, npad32(M.n));
}

// Gradient only (a convergence test that needs no matrix): |g_free|^2 per problem.
__global__ void __launch_bounds__(kRowTile) k_gradient(ElemArgs A) {
    const int b = blockIdx.y;
    if (!A.slot.active[b]) return;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    double gn[1] = {0.0};
    if (row < A.mesh.n) gn[0] = row_gradient(A, b, row, A.mesh.pin_handle_v[row] >= 0);
    double tot[1];
    double* part = A.slot.part + (size_t)b * A.slot.part_tiles * 4;
    if (tile_commit<1>(gn, part, blockIdx.x, gridDim.x, &A.slot.sc[b].tk_g, 0, tot) && threadIdx.x == 0)
        A.slot.sc[b].gnorm2 = tot[0];
}

template <typename T>
__global__ void __launch_bounds__(kRowTile) k_slope(ElemArgs A) {
    const int b = blockIdx.y;
    if (!A.slot.active[b]) return;
    const int n = A.mesh.n;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    double v[1] = {0.0};
    if (row < n) {
        const double* g = A.slot.g + ((size_t)b * n + row) * 3;
        const T* dx = rec_field(vecp<T>(A.slot, b, kOffRec, n), npad32(n), kRecDX, row);
        v[0] = g[0] * (double)dx[0] + g[1] * (double)dx[1] + g[2] * (double)dx[2];
    }
    double tot[1];
    double* part = A.slot.part + (size_t)b * A.slot.part_tiles * 4;
    if (tile_commit<1>(v, part, blockIdx.x, gridDim.x, &A.slot.sc[b].tk_s, 0, tot) && threadIdx.x == 0)
        A.slot.sc[b].slope = tot[0];
}

template <typename T>
__global__ void k_update(ElemArgs A) {
    const int b = blockIdx.y;
    if (!A.slot.active[b]) return;
    const int n = A.mesh.n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    const T* rec = vecp<T>(A.slot, b, kOffRec, n);
    double* x = A.slot.x + (size_t)b * n * 3;
    x[i] = fma(A.slot.alpha[b], (double)rec_field(rec, npad32(n), kRecDX, i / 3)[i % 3], x[i]);
}

__global__ void k_unpermute(ElemArgs A, double* __restrict__ out) {
    const int b = blockIdx.y;
    const int n = A.mesh.n;
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int v = A.mesh.vperm[o];
    const double* x = A.slot.x + ((size_t)b * n + v) * 3;
    double* y = out + ((size_t)b * n + o) * 3;
    y[0] = x[0];
    y[1] = x[1];
    y[2] = x[2];
}

__global__ void k_permute_in(ElemArgs A, int b, const double* __restrict__ xin) {
    const int n = A.mesh.n;
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int v = A.mesh.vperm[o];
    double* x = A.slot.x + ((size_t)b * n + v) * 3;
    x[0] = xin[3 * (size_t)o];
    x[1] = xin[3 * (size_t)o + 1];
    x[2] = xin[3 * (size_t)o + 2];
}

}  // namespace

void launch_assemble(const ElemArgs& a, int B, cudaStream_t s) {
    const dim3 grid((unsigned)((a.mesh.n_up + kRowTile - 1) / kRowTile), B);
    if (a.slot.prec == 1) k_assemble_slots<float><<<grid, kRowTile, 0, s>>>(a);
    else k_assemble_slots<double><<<grid, kRowTile, 0, s>>>(a);
    launch_gradient(a, B, s);
}

void launch_gradient(const ElemArgs& a, int B, cudaStream_t s) {
    dim3 grid((a.mesh.n + kRowTile - 1) / kRowTile, B);
    k_gradient<<<grid, kRowTile, 0, s>>>(a);
}

void launch_slope(const ElemArgs& a, int B, cudaStream_t s) {
    dim3 grid((a.mesh.n + kRowTile - 1) / kRowTile, B);
    if (a.slot.prec == 1) k_slope<float><<<grid, kRowTile, 0, s>>>(a);
    else k_slope<double><<<grid, kRowTile, 0, s>>>(a);
}

void launch_update(const ElemArgs& a, int B, cudaStream_t s) {
    dim3 grid((3 * a.mesh.n + 255) / 256, B);
    if (a.slot.prec == 1) k_update<float><<<grid, 256, 0, s>>>(a);
    else k_update<double><<<grid, 256, 0, s>>>(a);
}

void launch_unpermute(const ElemArgs& a, int B, double* out, cudaStream_t s) {
    dim3 grid((a.mesh.n + 255) / 256, B);
    k_unpermute<<<grid, 256, 0, s>>>(a, out);
}

void launch_permute_in(const ElemArgs& a, int b, const double* xin, cudaStream_t s) {
    k_permute_in<<<(a.mesh.n + 255) / 256, 256, 0, s>>>(a, b, xin);
}

}  // namespace mfem
