// PCG kernels (a5): initialisation and the two stream-ordered kernels of one
// block-Jacobi preconditioned CG iteration over a table of problems.
//
// Paper §3, Eq. 12 and Algorithm 1 ("x = A^{-1} b"): the condensed system is
// SPD, so it is solved by conjugate gradients (inexactly inside each Newton
// step, to a relative residual).  Dots are accumulated as float-float partials
// per row and warp and reduced per problem in FP64 with a ticketed, fixed-order
// tile reduction, so results do not depend on scheduling.
#include <cuda_runtime.h>

#include "kernels.h"

namespace mfem {

namespace {

// r = -g, z = D^{-1} r, dx = 0, p_old = 0; rho = r.z, rr0 = r.r per problem.
template <typename T>
__global__ void k_pcg_init(ElemArgs A, double tol2, int maxit, const double* __restrict__ tol2_b) {
    const int b = blockIdx.y;
    if (!A.slot.active[b]) return;
    const int n = A.mesh.n;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    double v[2] = {0.0, 0.0};
    if (row < n) {
        const double* g = A.slot.g + ((size_t)b * n + row) * 3;
        const T* di = (const T*)A.slot.dinv + ((size_t)b * n + row) * 9;
        T* rec = vecp<T>(A.slot, b, kOffRec, n) + kRec * (size_t)row;
        T* zp = vecp<T>(A.slot, b, kOffZP0, n) + 8 * (size_t)row;
        T rr[3] = {(T)(-g[0]), (T)(-g[1]), (T)(-g[2])};
#pragma unroll
        for (int i = 0; i < kRec; ++i) rec[i] = (T)0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            T zi = di[3 * i] * rr[0] + di[3 * i + 1] * rr[1] + di[3 * i + 2] * rr[2];
            rec[kRecR + i] = rr[i];
            zp[i] = zi;
            zp[4 + i] = (T)0;
            v[0] += (double)rr[i] * (double)zi;
            v[1] += (double)rr[i] * (double)rr[i];
        }
        zp[3] = (T)0;
        zp[7] = (T)0;
    }
    double tot[2];
    double* part = A.slot.part + (size_t)b * A.slot.part_tiles * 4;
    if (tile_commit<2>(v, part, blockIdx.x, gridDim.x, &A.slot.sc[b].tk_init, 1, tot) && threadIdx.x == 0) {
        ProbScal* sc = &A.slot.sc[b];
        sc->rho = tot[0];
        sc->rr0 = tot[1];
        sc->rr = tot[1];
        sc->beta = 0.0;
        sc->alpha = 0.0;
        sc->alpha_f = 0.f;
        sc->beta_f = 0.f;
        sc->iter = 0;
        sc->tol2 = tol2_b ? tol2_b[b] : tol2;
        sc->maxit = maxit;
        sc->state = (tot[1] > 0.0 && tot[0] > 0.0 && maxit > 0) ? kActive : kConverged;
    }
}

// ---- PCG iteration kernels ----------------------------------------------------
// One PCG iteration is two ordinary launches over every problem of the
// descriptor table; a block is one (problem, tile of TILE rows) unit and returns
// at once when its problem is not active.
//   k_pcg_spmv:   p_new = z + beta p_old (also for neighbours, recomputed on the
//                 fly from their (z, p_old) record), q = K p_new, tile partial of
//                 p.q; the last tile of a problem sets alpha = rho / p.q.
//   k_pcg_update: dx += alpha p, r -= alpha q, z = D^{-1} r, partials of r.z and
//                 r.r; the last tile sets beta, rho, the iteration count and the
//                 convergence state (|r| <= tol |r0| or the iteration cap).
// Kernel boundaries order every write before the next iteration's reads, so no
// block ever waits on another.  z and p of a vertex share one 32-byte record
// (two ping-pong buffers by iteration parity); the matrix streams through with
// evict-first loads.
__device__ __forceinline__ void ld_zp(const float* zp, int c, float (&z)[3], float (&p)[3]) {
    const float4 a = *reinterpret_cast<const float4*>(zp + 8 * (size_t)c);
    const float4 b = *reinterpret_cast<const float4*>(zp + 8 * (size_t)c + 4);
    z[0] = a.x; z[1] = a.y; z[2] = a.z;
    p[0] = b.x; p[1] = b.y; p[2] = b.z;
}

__device__ __forceinline__ void ld_zp(const double* zp, int c, double (&z)[3], double (&p)[3]) {
    const double2* r = reinterpret_cast<const double2*>(zp + 8 * (size_t)c);
    const double2 a = r[0], b = r[1], e = r[2], f = r[3];
    z[0] = a.x; z[1] = a.y; z[2] = b.x;
    p[0] = e.x; p[1] = e.y; p[2] = f.x;
}

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

// problem of unit u: last descriptor whose unit_begin <= u
template <typename T>
__device__ __forceinline__ int unit_problem(const PcgDesc<T>* __restrict__ D, int n_probs, int u) {
    int lo = 0, hi = n_probs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (D[mid].unit_begin <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Full occupancy (2048 threads per SM) matters more than registers here: the
// kernel is latency-bound on its dependent col -> gather loads.
template <typename T, int TILE>
__global__ void __launch_bounds__(TILE, 2048 / TILE) k_pcg_spmv(const PcgDesc<T>* __restrict__ D, int n_probs) {
    pdl_wait();
    pdl_trigger();
    const int u = blockIdx.x;
    const PcgDesc<T>& d = D[unit_problem(D, n_probs, u)];
    ProbScal* sc = d.sc;
    if (sc->state != kActive) return;
    const int tile = u - d.unit_begin;
    const int row = tile * TILE + threadIdx.x;
    const int iter = sc->iter;
    const T* zpo = (iter & 1) ? d.zp1 : d.zp0;
    T* zpn = (iter & 1) ? d.zp0 : d.zp1;
    T alpha_unused, beta;
    coeffs(sc, alpha_unused, beta);
    double v[1] = {0.0};
    Partial<T> pq = Partial<T>::zero();
    if (row < d.n_rows) {
        const int s = row >> 5, lane = row & 31;
        const int base = __ldg(d.slice_ptr + s), w = (__ldg(d.slice_ptr + s + 1) - base) >> 5;
        T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll 4
        for (int k = 0; k < w; ++k) {
            const int g = base + (k << 5);
            const int c = __ldcs(d.col + g + lane);
            if (c >= 0) {
                const T* vv = d.val + (size_t)g * 9 + lane;
                T zc[3], pc[3];
                ld_zp(zpo, c, zc, pc);
                const T q0 = fma(beta, pc[0], zc[0]);
                const T q1 = fma(beta, pc[1], zc[1]);
                const T q2 = fma(beta, pc[2], zc[2]);
                a0 += __ldcs(vv) * q0 + __ldcs(vv + 32) * q1 + __ldcs(vv + 64) * q2;
                a1 += __ldcs(vv + 96) * q0 + __ldcs(vv + 128) * q1 + __ldcs(vv + 160) * q2;
                a2 += __ldcs(vv + 192) * q0 + __ldcs(vv + 224) * q1 + __ldcs(vv + 256) * q2;
            }
        }
        T zr[3], pr[3];
        ld_zp(zpo, row, zr, pr);
        const T pn0 = fma(beta, pr[0], zr[0]);
        const T pn1 = fma(beta, pr[1], zr[1]);
        const T pn2 = fma(beta, pr[2], zr[2]);
        st4(zpn + 8 * (size_t)row + 4, pn0, pn1, pn2);
        st4(d.rec + kRec * (size_t)row + kRecQ, a0, a1, a2);
        pq = dot3_partial(pn0, pn1, pn2, a0, a1, a2);
    }
    v[0] = warp_sum_partial(pq);
    double tot[1];
    if (tile_commit<1>(v, d.part, tile, d.n_tiles, &sc->tk_a, 0, tot, true) && threadIdx.x == 0) {
        const double pq = tot[0];
        if (pq > 0.0 && isfinite(pq)) {
            sc->alpha = sc->rho / pq;
        } else {  // breakdown (p = 0 or K not SPD along p): stop with the current dx
            sc->alpha = 0.0;
            sc->state = kConverged;
        }
        sc->alpha_f = (float)sc->alpha;
    }
}

template <typename T, int TILE>
__global__ void __launch_bounds__(TILE) k_pcg_update(const PcgDesc<T>* __restrict__ D, int n_probs) {
    pdl_wait();
    pdl_trigger();
    const int u = blockIdx.x;
    const PcgDesc<T>& d = D[unit_problem(D, n_probs, u)];
    ProbScal* sc = d.sc;
    if (sc->state != kActive) return;
    const int tile = u - d.unit_begin;
    const int row = tile * TILE + threadIdx.x;
    const int iter = sc->iter;
    T* zpn = (iter & 1) ? d.zp0 : d.zp1;
    T alpha, beta_unused;
    coeffs(sc, alpha, beta_unused);
    double v[2] = {0.0, 0.0};
    Partial<T> rz = Partial<T>::zero(), rr2 = Partial<T>::zero();
    if (row < d.n_rows) {
        T* zrec = zpn + 8 * (size_t)row;
        T* rec = d.rec + kRec * (size_t)row;
        const T* di = d.dinv + 9 * (size_t)row;
        T pp[3], dxv[3], r0[3], qv[3], rr[3], zz[3];
        ld4(zrec + 4, pp);
        ld4(rec + kRecDX, dxv);
        ld4(rec + kRecR, r0);
        ld4(rec + kRecQ, qv);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            dxv[i] = fma(alpha, pp[i], dxv[i]);
            rr[i] = fma(-alpha, qv[i], r0[i]);
        }
        st4(rec + kRecDX, dxv[0], dxv[1], dxv[2]);
        st4(rec + kRecR, rr[0], rr[1], rr[2]);
#pragma unroll
        for (int i = 0; i < 3; ++i) zz[i] = di[3 * i] * rr[0] + di[3 * i + 1] * rr[1] + di[3 * i + 2] * rr[2];
        st4(zrec, zz[0], zz[1], zz[2]);
        rz = dot3_partial(rr[0], rr[1], rr[2], zz[0], zz[1], zz[2]);
        rr2 = dot3_partial(rr[0], rr[1], rr[2], rr[0], rr[1], rr[2]);
    }
    v[0] = warp_sum_partial(rz);
    v[1] = warp_sum_partial(rr2);
    double tot[2];
    if (tile_commit<2>(v, d.part, tile, d.n_tiles, &sc->tk_b, 1, tot, true) && threadIdx.x == 0) {
        const double rho_new = tot[0];
        sc->beta = sc->rho != 0.0 ? rho_new / sc->rho : 0.0;
        sc->beta_f = (float)sc->beta;
        sc->rho = rho_new;
        sc->rr = tot[1];
        const int itn = sc->iter + 1;
        sc->iter = itn;
        if (!(tot[1] > sc->tol2 * sc->rr0)) sc->state = kConverged;
        else if (itn >= sc->maxit) sc->state = kMaxIter;
    }
}

// Each launch may start while the previous kernel of the stream drains
// (programmatic stream serialization); the kernels wait on it first thing.
template <typename T, int TILE>
cudaError_t launch_pcg_iters_t(const PcgDesc<T>* descs, int n_probs, int n_units, int iters, cudaStream_t s) {
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
    for (int i = 0; i < iters; ++i) {
        cudaError_t e = cudaLaunchKernelEx(&cfg, k_pcg_spmv<T, TILE>, descs, n_probs);
        if (e != cudaSuccess) return e;
        e = cudaLaunchKernelEx(&cfg, k_pcg_update<T, TILE>, descs, n_probs);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace

void launch_pcg_init(const ElemArgs& a, int B, int tile_rows, double tol2, int maxit, const double* tol2_b,
                     cudaStream_t s) {
    dim3 grid((a.mesh.n + tile_rows - 1) / tile_rows, B);
    if (a.slot.prec == 1) k_pcg_init<float><<<grid, tile_rows, 0, s>>>(a, tol2, maxit, tol2_b);
    else k_pcg_init<double><<<grid, tile_rows, 0, s>>>(a, tol2, maxit, tol2_b);
}

template <typename T>
cudaError_t launch_pcg_iters(const PcgDesc<T>* descs, int n_probs, int n_units, int tile_rows, int iters,
                             cudaStream_t s) {
    switch (tile_rows) {
        case 64: return launch_pcg_iters_t<T, 64>(descs, n_probs, n_units, iters, s);
        case 128: return launch_pcg_iters_t<T, 128>(descs, n_probs, n_units, iters, s);
        case 256: return launch_pcg_iters_t<T, 256>(descs, n_probs, n_units, iters, s);
        default: return cudaErrorInvalidValue;
    }
}

bool pcg_tile_supported(int tile_rows) { return tile_rows == 64 || tile_rows == 128 || tile_rows == 256; }

template cudaError_t launch_pcg_iters<float>(const PcgDesc<float>*, int, int, int, int, cudaStream_t);
template cudaError_t launch_pcg_iters<double>(const PcgDesc<double>*, int, int, int, int, cudaStream_t);

}  // namespace mfem
