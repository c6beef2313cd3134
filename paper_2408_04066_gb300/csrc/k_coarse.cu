// Coarse space of the two-level PCG preconditioner: set-up, once per mesh.
//
// Aggregates are runs of agg_size consecutive internal (Morton-ordered)
// vertices.  Free vertex i of aggregate a carries the six rigid modes of the
// rest shape, P_i = [I | -[X_i - c_a]x] (3 x 6: a translation and a small
// rotation about the aggregate's centroid); pins carry none.  The coarse matrix
// A_c = sum_ij P_i^T K_ij P_j of the rest Hessian K (the Eq. 12 matrix at x = X
// with the rig at rest) is formed block by block: one warp per aggregate row,
// each lane owning fixed entries of the 6x6 blocks, contributions added in the
// fixed (row, slot) order, so the result is reproducible.  A_c is inverted in
// FP64 by Gauss-Jordan elimination without pivoting (A_c is SPD); a mode whose
// pivot falls below 1e-10 of its own diagonal (an aggregate with too few free
// vertices to carry it) is dropped, its row and column zero in the inverse.
// The inverse is kept in FP32, symmetrised.  During a solve each aggregate's
// modes are turned with a rotation fitted to the aggregate's current motion
// (k_agg_rotations; the coarse matrix of a rigidly turned region is the rest
// one in turned coordinates), so the rest inverse serves every pose.
#include <cuda_runtime.h>

#include "kernels.h"

namespace mfem {

namespace {

// column c of P_i for a vertex at offset v from its aggregate's centroid
__device__ __forceinline__ void mode_col(const float4 v, int c, double (&u)[3]) {
    if (c < 3) {
        u[0] = c == 0;
        u[1] = c == 1;
        u[2] = c == 2;
        return;
    }
    // -[v]x e_(c-3)
    const double x = v.x, y = v.y, z = v.z;
    switch (c - 3) {
        case 0: u[0] = 0.0; u[1] = -z; u[2] = y; break;
        case 1: u[0] = z; u[1] = 0.0; u[2] = -x; break;
        default: u[0] = -y; u[1] = x; u[2] = 0.0; break;
    }
}

template <typename KT>
__global__ void k_coarse_galerkin(MeshDev M, const KT* __restrict__ val, const int* __restrict__ cnb_ptr,
                                  const int* __restrict__ cnb, int agg_size, double* __restrict__ Ac, int N) {
    extern __shared__ double acc[];   // [cnb_count][36]
    const int I = blockIdx.x, lane = threadIdx.x;
    const int j0 = cnb_ptr[I], nj = cnb_ptr[I + 1] - j0;
    for (int e = lane; e < nj * 36; e += 32) acc[e] = 0.0;
    __syncwarp();
    const int i0 = I * agg_size, i1 = min(M.n, i0 + agg_size);
    for (int i = i0; i < i1; ++i) {
        const float4 vi = M.crel[i];
        if (vi.w == 0.f) continue;
        const int s = i >> 5, l = i & 31;
        const int base = M.slice_ptr[s], w = (M.slice_ptr[s + 1] - base) >> 5;
        for (int k = 0; k < w; ++k) {
            const int g = base + (k << 5);
            const int j = M.col[g + l];
            if (j < 0) continue;
            const float4 vj = M.crel[j];
            if (vj.w == 0.f) continue;
            const int J = j / agg_size;
            int lo = 0, hi = nj - 1;   // position of J in the sorted neighbour list
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (cnb[j0 + mid] < J) lo = mid + 1;
                else hi = mid;
            }
            double K[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) K[a][b] = (double)val[(size_t)g * 9 + 32 * (3 * a + b) + l];
            for (int e = lane; e < 36; e += 32) {
                const int r = e / 6, c = e % 6;
                double u[3], v[3];
                mode_col(vi, r, u);
                mode_col(vj, c, v);
                double t = 0.0;
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    t += u[a] * (K[a][0] * v[0] + K[a][1] * v[1] + K[a][2] * v[2]);
                acc[36 * lo + e] += t;
            }
        }
    }
    __syncwarp();
    for (int e = lane; e < nj * 36; e += 32) {
        const int q = e / 36, r = (e % 36) / 6, c = e % 6;
        const int J = cnb[j0 + q];
        Ac[(size_t)(6 * I + r) * N + 6 * J + c] = acc[e];
    }
}

// Gauss-Jordan step k: keep row k and column k (pre-step values) and decide
// whether the pivot is kept.
__global__ void k_gj_save(const double* __restrict__ A, int N, int k, const double* __restrict__ d0,
                          double* __restrict__ rowk, double* __restrict__ colk, int* __restrict__ keep) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        rowk[i] = A[(size_t)k * N + i];
        colk[i] = A[(size_t)i * N + k];
    }
    if (i == 0) keep[0] = A[(size_t)k * N + k] > 1e-10 * d0[k] ? 1 : 0;
}

__global__ void k_gj_step(double* __restrict__ A, int N, int k, const double* __restrict__ rowk,
                          const double* __restrict__ colk, const int* __restrict__ keep) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= N || j >= N) return;
    double& a = A[(size_t)i * N + j];
    if (!keep[0]) {
        if (i == k || j == k) a = 0.0;
        return;
    }
    const double ip = 1.0 / rowk[k];
    if (i == k && j == k) a = ip;
    else if (i == k) a = rowk[j] * ip;
    else if (j == k) a = -colk[i] * ip;
    else a -= colk[i] * (rowk[j] * ip);
}

__global__ void k_diag_copy(const double* __restrict__ A, int N, double* __restrict__ d0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) d0[i] = A[(size_t)i * N + i];
}

// out has rows of ld >= N floats; the padding columns are zero.
__global__ void k_sym_f32(const double* __restrict__ A, int N, int ld, float* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= N || j >= ld) return;
    out[(size_t)i * ld + j] = j < N ? (float)(0.5 * (A[(size_t)i * N + j] + A[(size_t)j * N + i])) : 0.f;
}

// Orthogonal polar factor of M by Higham's scaled Newton iteration
// X <- (gamma X + X^{-T} / gamma) / 2 (N. J. Higham, "Computing the polar
// decomposition -- with applications", SIAM J. Sci. Stat. Comput. 1986), in
// FP32 (the rotation turns a preconditioner's coarse modes; it needs no more).
// Returns false if M is singular or not of positive determinant (no rotation).
__device__ bool polar_rotation_pos(const float (&M)[3][3], float (&R)[3][3]) {
    float X[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) X[i][j] = M[i][j];
    for (int it = 0; it < 12; ++it) {
        const float c00 = X[1][1] * X[2][2] - X[1][2] * X[2][1], c01 = X[1][2] * X[2][0] - X[1][0] * X[2][2],
                    c02 = X[1][0] * X[2][1] - X[1][1] * X[2][0];
        const float c10 = X[0][2] * X[2][1] - X[0][1] * X[2][2], c11 = X[0][0] * X[2][2] - X[0][2] * X[2][0],
                    c12 = X[0][1] * X[2][0] - X[0][0] * X[2][1];
        const float c20 = X[0][1] * X[1][2] - X[0][2] * X[1][1], c21 = X[0][2] * X[1][0] - X[0][0] * X[1][2],
                    c22 = X[0][0] * X[1][1] - X[0][1] * X[1][0];
        const float det = X[0][0] * c00 + X[0][1] * c01 + X[0][2] * c02;
        if (!(det > 0.f)) return false;
        const float id = 1.f / det;
        const float IT[3][3] = {{c00 * id, c01 * id, c02 * id}, {c10 * id, c11 * id, c12 * id},
                                {c20 * id, c21 * id, c22 * id}};   // X^{-T}
        float nx = 0.f, ni = 0.f;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                nx += X[i][j] * X[i][j];
                ni += IT[i][j] * IT[i][j];
            }
        const float gam = sqrtf(sqrtf(ni / nx));
        float diff = 0.f;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                const float y = 0.5f * (gam * X[i][j] + IT[i][j] / gam);
                diff += (y - X[i][j]) * (y - X[i][j]);
                X[i][j] = y;
            }
        if (diff <= 1e-12f) break;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R[i][j] = X[i][j];
    return true;
}

// One warp per (aggregate, problem): R_a = the rotation of the polar
// decomposition of M = sum_i x_i (X_i - c_a)^T over the aggregate's free
// vertices (shape matching: for x_i = R (X_i - c_a) + t, M = R S with S
// symmetric positive definite, so the fit is R exactly; sum_i (X_i - c_a) = 0
// makes the translation drop out).  M is summed in FP64 (x carries the
// aggregate's absolute position), the polar factor taken in FP32.  When M has
// no rotation factor (an aggregate without enough free vertices, or inverted),
// R_a is the rotation of the aggregate's majority handle.  The coarse modes of
// the two-level preconditioner are turned by R_a, so they follow each
// aggregate's own motion -- also at cluster boundaries, where the handle's
// rotation does not.
__global__ void __launch_bounds__(32) k_agg_rotations(ElemArgs A) {
    const int a = blockIdx.x, b = blockIdx.y, lane = threadIdx.x;
    if (!A.slot.active[b]) return;   // warp-uniform
    const MeshDev& M = A.mesh;
    const int size = 1 << M.agg_shift;
    const int i0 = a * size, i1 = min(M.n, i0 + size);
    const double* x = A.slot.x + (size_t)b * M.n * 3;
    double m[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) m[e] = 0.0;
    for (int i = i0 + lane; i < i1; i += 32) {
        const float4 r = M.crel[i];
        if (r.w == 0.f) continue;
        const double xi[3] = {x[3 * (size_t)i], x[3 * (size_t)i + 1], x[3 * (size_t)i + 2]};
        const double ri[3] = {r.x, r.y, r.z};
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) m[3 * p + q] = fma(xi[p], ri[q], m[3 * p + q]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int e = 0; e < 9; ++e) m[e] += __shfl_xor_sync(0xffffffffu, m[e], o);
    if (lane == 0) {
        const float Mm[3][3] = {{(float)m[0], (float)m[1], (float)m[2]},
                                {(float)m[3], (float)m[4], (float)m[5]},
                                {(float)m[6], (float)m[7], (float)m[8]}};
        float R[3][3];
        float* out = A.slot.aggq + ((size_t)b * M.n_agg + a) * 9;
        if (polar_rotation_pos(Mm, R)) {
            for (int e = 0; e < 9; ++e) out[e] = R[e / 3][e % 3];
        } else {
            const double* T = A.slot.xf + (size_t)b * M.H * 12 + 12 * (size_t)M.agg_handle[a];
            for (int e = 0; e < 9; ++e) out[e] = (float)T[4 * (e / 3) + e % 3];
        }
    }
}

}  // namespace

void launch_agg_rotations(const ElemArgs& a, int B, cudaStream_t s) {
    if (a.mesh.n_agg <= 0) return;
    k_agg_rotations<<<dim3(a.mesh.n_agg, B), 32, 0, s>>>(a);
}

cudaError_t build_coarse_inverse(const MeshDev& M, const void* val, int prec, const int* cnb_ptr, const int* cnb,
                                 int cnb_max, int agg_size, float* Ainv, cudaStream_t s) {
    const int N = M.coarse_n;
    double* A = nullptr;
    double* tmp = nullptr;
    int* keep = nullptr;
    cudaError_t e = cudaMalloc((void**)&A, sizeof(double) * (size_t)N * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&tmp, sizeof(double) * 3 * (size_t)N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&keep, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(A, 0, sizeof(double) * (size_t)N * N, s);
    const size_t smem = sizeof(double) * 36 * (size_t)cnb_max;
    if (e == cudaSuccess && smem > 48 * 1024)
        e = cudaFuncSetAttribute(prec == 1 ? (const void*)k_coarse_galerkin<float> : (const void*)k_coarse_galerkin<double>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        if (prec == 1)
            k_coarse_galerkin<float><<<M.n_agg, 32, smem, s>>>(M, (const float*)val, cnb_ptr, cnb, agg_size, A, N);
        else
            k_coarse_galerkin<double><<<M.n_agg, 32, smem, s>>>(M, (const double*)val, cnb_ptr, cnb, agg_size, A, N);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        double *d0 = tmp, *rowk = tmp + N, *colk = tmp + 2 * N;
        k_diag_copy<<<(N + 255) / 256, 256, 0, s>>>(A, N, d0);
        const dim3 blk(32, 8), grid((N + 31) / 32, (N + 7) / 8);
        for (int k = 0; k < N && e == cudaSuccess; ++k) {
            k_gj_save<<<(N + 255) / 256, 256, 0, s>>>(A, N, k, d0, rowk, colk, keep);
            k_gj_step<<<grid, blk, 0, s>>>(A, N, k, rowk, colk, keep);
            if ((k & 255) == 0) e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            const int ld = coarse_ld(N);
            k_sym_f32<<<dim3((ld + 31) / 32, (N + 7) / 8), blk, 0, s>>>(A, N, ld, Ainv);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (A) cudaFree(A);
    if (tmp) cudaFree(tmp);
    if (keep) cudaFree(keep);
    return e;
}

}  // namespace mfem
