// Per-tetrahedron kernels: pose update (a0), element local step (a1), line-search
// energy (a6), element outputs and diagnostics.
//
// Element step, paper §3: F_k = B_k x (text after Eq. 4), S_k = sym(R_k^T F_k)
// (the pseudo-inverse of [R] named after Eq. 12), Psi(S_k) and its derivatives
// (Eq. 6), the multiplier Lambda_k = R_k dPsi/dS (Eq. 10-11), the element
// forces W_k Lambda_k G_a and the element blocks of the condensed matrix
// W_k A_k^T H_s A_k of Eq. 12, with A_k = R_k^+ B_k.  R_k is the rotation of the
// rig handle of the tet's cluster (§3.1).
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.h"

namespace mfem {

namespace {

constexpr double kSqrt2 = 1.4142135623730951;
constexpr double kInvSqrt2 = 0.7071067811865476;
constexpr double kSpdEps = 1.0e-6;     // Hessian eigenvalue floor, times mu
constexpr double kFallbackJ = 0.25;    // mixed path: det S below this -> FP64 Hessian

constexpr int kMaxStagedHandles = 64;   // pose rotations staged in shared memory up to this many handles

// Gather the four vertex positions of tet k of problem b (optionally x + alpha dx).
// dx, if given, is read with a stride of dx_stride elements per vertex.
template <typename T>
__device__ __forceinline__ void gather_x(const double* __restrict__ x, const T* __restrict__ dx,
                                         double alpha, int4 tv, double (&xa)[4][3], int dx_stride = 3) {
    const int id[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            double v = x[3 * (size_t)id[a] + i];
            if (dx) v = fma(alpha, (double)dx[(size_t)dx_stride * id[a] + i], v);
            xa[a][i] = v;
        }
}

// Shape-function gradients G_a (rows of D_m^{-1}, G_0 = -(G_1+G_2+G_3)).
__device__ __forceinline__ void load_G(const double* __restrict__ Dm, int m, int k, double (&G)[4][3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) G[r + 1][c] = Dm[(size_t)(3 * r + c) * m + k];
#pragma unroll
    for (int c = 0; c < 3; ++c) G[0][c] = -(G[1][c] + G[2][c] + G[3][c]);
}

__device__ __forceinline__ void load_Q(const double* __restrict__ xf, int h, double (&Q)[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Q[i][j] = xf[12 * h + 4 * i + j];
}

// S = sym(Q^T F), F = sum_{a=1..3} (x_a - x_0) G_a^T.  S as (S00,S11,S22,S12,S02,S01).
__device__ __forceinline__ void stretch(const double (&xa)[4][3], const double (&G)[4][3],
                                        const double (&Q)[3][3], double (&F)[3][3], double (&S)[6]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double f = 0.0;
#pragma unroll
            for (int a = 1; a < 4; ++a) f = fma(xa[a][i] - xa[0][i], G[a][j], f);
            F[i][j] = f;
        }
    double A[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) A[i][j] = Q[0][i] * F[0][j] + Q[1][i] * F[1][j] + Q[2][i] * F[2][j];
    S[0] = A[0][0];
    S[1] = A[1][1];
    S[2] = A[2][2];
    S[3] = 0.5 * (A[1][2] + A[2][1]);
    S[4] = 0.5 * (A[0][2] + A[2][0]);
    S[5] = 0.5 * (A[0][1] + A[1][0]);
}

// Energy density and stress sigma = dPsi/dS (plain symmetric components).
template <int MODEL>
__device__ __forceinline__ double psi_sigma(const double (&S)[6], double mu, double lam, double (&sig)[6]) {
    const double d0 = S[0] - 1.0, d1 = S[1] - 1.0, d2 = S[2] - 1.0;
    if (MODEL == 0 || MODEL == 1) {
        double psi = mu * (d0 * d0 + d1 * d1 + d2 * d2 + 2.0 * (S[3] * S[3] + S[4] * S[4] + S[5] * S[5]));
        sig[0] = 2.0 * mu * d0;
        sig[1] = 2.0 * mu * d1;
        sig[2] = 2.0 * mu * d2;
        sig[3] = 2.0 * mu * S[3];
        sig[4] = 2.0 * mu * S[4];
        sig[5] = 2.0 * mu * S[5];
        if (MODEL == 1) {
            double tr = d0 + d1 + d2;
            psi += 0.5 * lam * tr * tr;
            sig[0] += lam * tr;
            sig[1] += lam * tr;
            sig[2] += lam * tr;
        }
        return psi;
    } else {
        // adjugate (cofactor) of symmetric S and J = det S
        const double a = S[0], b = S[1], c = S[2], s12 = S[3], s02 = S[4], s01 = S[5];
        const double c00 = b * c - s12 * s12, c11 = a * c - s02 * s02, c22 = a * b - s01 * s01;
        const double c12 = s01 * s02 - a * s12, c02 = s01 * s12 - b * s02, c01 = s02 * s12 - c * s01;
        const double J = a * c00 + s01 * c01 + s02 * c02;
        const double ls = lam + mu;
        const double nS2 = a * a + b * b + c * c + 2.0 * (s12 * s12 + s02 * s02 + s01 * s01);
        const double psi = 0.5 * mu * (nS2 - 3.0) - mu * (J - 1.0) + 0.5 * ls * (J - 1.0) * (J - 1.0);
        const double k = ls * (J - 1.0) - mu;
        sig[0] = mu * a + k * c00;
        sig[1] = mu * b + k * c11;
        sig[2] = mu * c + k * c22;
        sig[3] = mu * s12 + k * c12;
        sig[4] = mu * s02 + k * c02;
        sig[5] = mu * s01 + k * c01;
        return psi;
    }
}

// ---- float-float element path (mixed precision) -----------------------------
// F, S, the energy density and the stress in float-float arithmetic (value =
// hi + lo, ~48 significant bits: Dekker's product by fused multiply-add,
// Knuth's two-sum) from positions, shape gradients and rotations held as float
// pairs, so that the element pass needs almost no FP64 instructions (GB300
// issues FP64 at a small fraction of its FP32 rate).  Only the energy's
// weighting and sum stay FP64.
__device__ __forceinline__ FF ff_split(double v) {
    const float h = (float)v;
    return FF{h, (float)(v - (double)h)};
}
__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.hi, -a.lo}; }
__device__ __forceinline__ FF ff_sub(FF a, FF b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float h = __fadd_rn(p, e);
    return FF{h, __fsub_rn(e, __fsub_rn(h, p))};
}
__device__ __forceinline__ FF ff_scale2(FF a, float s) { return FF{a.hi * s, a.lo * s}; }   // s a power of two
__device__ __forceinline__ FF ff_addf(FF a, float b) { return ff_add(a, FF{b, 0.f}); }

// float -> double by the IEEE 754 bit layouts (binary32: 1 + 8 + 23 bits,
// binary64: 1 + 11 + 52) in integer instructions only: the conversion
// instruction runs on GB300's narrow FP64 pipe, and a conversion kept for the
// rare cases would be if-converted and paid by every lane.  Normal numbers:
// the exponent bias grows by 1023 - 127 = 896 and the fraction moves up 29
// bits; a subnormal m 2^-149 with its leading bit at position p - 1 becomes
// 1.f 2^(p - 150); zeros keep their sign; infinities and NaN keep their
// fraction bits (a signalling NaN stays signalling).
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    unsigned long long ed, frac;
    if (e == 0xffu) {
        ed = 0x7ffull;
        frac = (unsigned long long)m << 29;
    } else if (e != 0u) {
        ed = e + 896u;
        frac = (unsigned long long)m << 29;
    } else if (m == 0u) {
        ed = 0ull;
        frac = 0ull;
    } else {
        const int p = 32 - __clz((int)m);
        ed = (unsigned long long)(p + 873);
        frac = ((unsigned long long)m << (53 - p)) & 0xfffffffffffffull;
    }
    return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) | (ed << 52) | frac));
}

// S = sym(Q^T F), F = sum_a (x_a - x_0) G_a^T (a = 1..3), all as float pairs;
// G[r] = row r of D_m^{-1} (G_{r+1}).
__device__ __forceinline__ void stretch_ff(const FF (&xa)[4][3], const FF (&G)[3][3], const FF (&Q)[3][3],
                                           FF (&S)[6]) {
    FF d[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) d[a][i] = ff_sub(xa[a + 1][i], xa[0][i]);
    FF F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            F[i][j] = ff_add(ff_add(ff_mul(d[0][i], G[0][j]), ff_mul(d[1][i], G[1][j])), ff_mul(d[2][i], G[2][j]));
    FF Am[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Am[i][j] = ff_add(ff_add(ff_mul(Q[0][i], F[0][j]), ff_mul(Q[1][i], F[1][j])), ff_mul(Q[2][i], F[2][j]));
    S[0] = Am[0][0];
    S[1] = Am[1][1];
    S[2] = Am[2][2];
    S[3] = ff_scale2(ff_add(Am[1][2], Am[2][1]), 0.5f);
    S[4] = ff_scale2(ff_add(Am[0][2], Am[2][0]), 0.5f);
    S[5] = ff_scale2(ff_add(Am[0][1], Am[1][0]), 0.5f);
}

// psi_sigma in float-float: returns Psi, writes sigma rounded to FP32
template <int MODEL>
__device__ __forceinline__ FF psi_sigma_ff(const FF (&S)[6], FF mu, FF lam, float (&sig)[6]) {
    const FF d0 = ff_addf(S[0], -1.f), d1 = ff_addf(S[1], -1.f), d2 = ff_addf(S[2], -1.f);
    if (MODEL == 0 || MODEL == 1) {
        const FF off = ff_add(ff_add(ff_mul(S[3], S[3]), ff_mul(S[4], S[4])), ff_mul(S[5], S[5]));
        const FF sq = ff_add(ff_add(ff_mul(d0, d0), ff_mul(d1, d1)), ff_mul(d2, d2));
        FF psi = ff_mul(mu, ff_add(sq, ff_scale2(off, 2.f)));
        const float m2 = 2.f * mu.hi;
        sig[0] = m2 * d0.hi;
        sig[1] = m2 * d1.hi;
        sig[2] = m2 * d2.hi;
        sig[3] = m2 * S[3].hi;
        sig[4] = m2 * S[4].hi;
        sig[5] = m2 * S[5].hi;
        if (MODEL == 1) {
            const FF tr = ff_add(ff_add(d0, d1), d2);
            psi = ff_add(psi, ff_scale2(ff_mul(lam, ff_mul(tr, tr)), 0.5f));
            const float lt = lam.hi * tr.hi;
            sig[0] += lt;
            sig[1] += lt;
            sig[2] += lt;
        }
        return psi;
    }
    const FF a = S[0], b = S[1], c = S[2], s12 = S[3], s02 = S[4], s01 = S[5];
    const FF c00 = ff_sub(ff_mul(b, c), ff_mul(s12, s12)), c11 = ff_sub(ff_mul(a, c), ff_mul(s02, s02));
    const FF c22 = ff_sub(ff_mul(a, b), ff_mul(s01, s01));
    const FF c12 = ff_sub(ff_mul(s01, s02), ff_mul(a, s12)), c02 = ff_sub(ff_mul(s01, s12), ff_mul(b, s02));
    const FF c01 = ff_sub(ff_mul(s02, s12), ff_mul(c, s01));
    // the energy in D = S - I, where its terms of first order in the strain
    // cancel exactly: |S|^2 - 3 = 2 tr D + |D|^2 and J - 1 = tr D + I2(D) + det D,
    // so Psi = mu/2 |D|^2 - mu (I2(D) + det D) + (lam + mu)/2 (J - 1)^2 is formed
    // to the precision of Psi itself rather than of mu
    const FF off2 = ff_add(ff_add(ff_mul(s12, s12), ff_mul(s02, s02)), ff_mul(s01, s01));
    const FF nD2 = ff_add(ff_add(ff_add(ff_mul(d0, d0), ff_mul(d1, d1)), ff_mul(d2, d2)), ff_scale2(off2, 2.f));
    const FF I2 = ff_sub(ff_add(ff_add(ff_mul(d0, d1), ff_mul(d0, d2)), ff_mul(d1, d2)), off2);
    const FF I3 = ff_add(ff_add(ff_mul(d0, ff_sub(ff_mul(d1, d2), ff_mul(s12, s12))),
                                ff_mul(s01, ff_sub(ff_mul(s12, s02), ff_mul(s01, d2)))),
                         ff_mul(s02, ff_sub(ff_mul(s01, s12), ff_mul(d1, s02))));
    const FF J1 = ff_add(ff_add(ff_add(ff_add(d0, d1), d2), I2), I3);   // J - 1
    const FF ls = ff_add(lam, mu);
    const FF psi = ff_add(ff_sub(ff_scale2(ff_mul(mu, nD2), 0.5f), ff_mul(mu, ff_add(I2, I3))),
                          ff_scale2(ff_mul(ls, ff_mul(J1, J1)), 0.5f));
    const FF kk = ff_sub(ff_mul(ls, J1), mu);
    const FF sg[6] = {ff_add(ff_mul(mu, a), ff_mul(kk, c00)),   ff_add(ff_mul(mu, b), ff_mul(kk, c11)),
                      ff_add(ff_mul(mu, c), ff_mul(kk, c22)),   ff_add(ff_mul(mu, s12), ff_mul(kk, c12)),
                      ff_add(ff_mul(mu, s02), ff_mul(kk, c02)), ff_add(ff_mul(mu, s01), ff_mul(kk, c01))};
#pragma unroll
    for (int i = 0; i < 6; ++i) sig[i] = sg[i].hi + sg[i].lo;
    return psi;
}

// SNH Hessian from an FP32 stretch (the float-float path's; same formulas as
// snh_hessian below with every operand in FP32)
__device__ void snh_hessian_f(const float (&S)[6], float mu, float lam, float (&C)[6][6]) {
    const float a = S[0], b = S[1], c = S[2];
    const float sq2 = (float)1.4142135623730951, is2 = (float)0.7071067811865476;
    const float d = sq2 * S[3], e = sq2 * S[4], f = sq2 * S[5];
    const float ls = lam + mu;
    const float J = a * b * c + d * e * f * is2 - 0.5f * (a * d * d + b * e * e + c * f * f);
    const float j[6] = {b * c - 0.5f * d * d, a * c - 0.5f * e * e, a * b - 0.5f * f * f,
                        e * f * is2 - a * d,   d * f * is2 - b * e,   d * e * is2 - c * f};
    float HJ[6][6];
#pragma unroll
    for (int p = 0; p < 6; ++p)
#pragma unroll
        for (int q = 0; q < 6; ++q) HJ[p][q] = 0.f;
    HJ[0][1] = HJ[1][0] = c;
    HJ[0][2] = HJ[2][0] = b;
    HJ[1][2] = HJ[2][1] = a;
    HJ[0][3] = HJ[3][0] = -d;
    HJ[1][4] = HJ[4][1] = -e;
    HJ[2][5] = HJ[5][2] = -f;
    HJ[3][3] = -a;
    HJ[4][4] = -b;
    HJ[5][5] = -c;
    HJ[3][4] = HJ[4][3] = f * is2;
    HJ[3][5] = HJ[5][3] = e * is2;
    HJ[4][5] = HJ[5][4] = d * is2;
    const float k = ls * (J - 1.f) - mu;
#pragma unroll
    for (int p = 0; p < 6; ++p)
#pragma unroll
        for (int q = 0; q < 6; ++q) C[p][q] = k * HJ[p][q] + ls * j[p] * j[q] + (p == q ? mu : 0.f);
}

// ---- SNH Hessian in Mandel coordinates, SPD filtering ----------------------
// s = (a, b, c, d, e, f) = (S00, S11, S22, sqrt2 S12, sqrt2 S02, sqrt2 S01).
template <typename RT>
__device__ void snh_hessian(const double (&S)[6], double mu_d, double lam_d, RT (&C)[6][6]) {
    const RT a = (RT)S[0], b = (RT)S[1], c = (RT)S[2];
    const RT d = (RT)(kSqrt2 * S[3]), e = (RT)(kSqrt2 * S[4]), f = (RT)(kSqrt2 * S[5]);
    const RT is2 = (RT)kInvSqrt2;
    const RT mu = (RT)mu_d, ls = (RT)(lam_d + mu_d);
    const RT J = a * b * c + d * e * f * is2 - (RT)0.5 * (a * d * d + b * e * e + c * f * f);
    const RT j[6] = {b * c - (RT)0.5 * d * d, a * c - (RT)0.5 * e * e, a * b - (RT)0.5 * f * f,
                     e * f * is2 - a * d,    d * f * is2 - b * e,    d * e * is2 - c * f};
    RT HJ[6][6];
#pragma unroll
    for (int p = 0; p < 6; ++p)
#pragma unroll
        for (int q = 0; q < 6; ++q) HJ[p][q] = (RT)0;
    HJ[0][1] = HJ[1][0] = c;
    HJ[0][2] = HJ[2][0] = b;
    HJ[1][2] = HJ[2][1] = a;
    HJ[0][3] = HJ[3][0] = -d;
    HJ[1][4] = HJ[4][1] = -e;
    HJ[2][5] = HJ[5][2] = -f;
    HJ[3][3] = -a;
    HJ[4][4] = -b;
    HJ[5][5] = -c;
    HJ[3][4] = HJ[4][3] = f * is2;
    HJ[3][5] = HJ[5][3] = e * is2;
    HJ[4][5] = HJ[5][4] = d * is2;
    const RT k = ls * (J - (RT)1) - mu;
#pragma unroll
    for (int p = 0; p < 6; ++p)
#pragma unroll
        for (int q = 0; q < 6; ++q) C[p][q] = k * HJ[p][q] + ls * j[p] * j[q] + (p == q ? mu : (RT)0);
}

// true if every eigenvalue of C exceeds `floor` (Cholesky of C - floor I)
template <typename RT>
__device__ bool chol_shifted_ok(const RT (&C)[6][6], RT floor) {
    RT L[6][6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        RT dsum = C[j][j] - floor;
#pragma unroll
        for (int k = 0; k < j; ++k) dsum -= L[j][k] * L[j][k];
        if (!(dsum > (RT)0)) return false;
        RT ljj = sqrt(dsum);
        L[j][j] = ljj;
        RT inv = (RT)1 / ljj;
#pragma unroll
        for (int i = j + 1; i < 6; ++i) {
            RT s = C[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            L[i][j] = s * inv;
        }
    }
    return true;
}

// Cyclic Jacobi eigen-decomposition of a symmetric 6x6 (Golub & Van Loan,
// "Matrix Computations", symmetric Jacobi method), then every eigenvalue is
// replaced by max(|eigenvalue|, floor) (absolute-value eigenvalue filtering).
template <typename RT>
__device__ __noinline__ void filter_spd(RT (&C)[6][6], RT floor) {
    RT V[6][6];
    for (int p = 0; p < 6; ++p)
        for (int q = 0; q < 6; ++q) V[p][q] = (p == q) ? (RT)1 : (RT)0;
    const RT eps = sizeof(RT) == 8 ? (RT)1e-15 : (RT)1e-7;
    for (int sweep = 0; sweep < 12; ++sweep) {
        RT off = 0, dia = 0;
        for (int p = 0; p < 6; ++p) {
            dia += C[p][p] * C[p][p];
            for (int q = p + 1; q < 6; ++q) off += C[p][q] * C[p][q];
        }
        if (off <= eps * eps * dia) break;
        for (int p = 0; p < 5; ++p)
            for (int q = p + 1; q < 6; ++q) {
                RT apq = C[p][q];
                if (apq == (RT)0) continue;
                RT theta = (C[q][q] - C[p][p]) / ((RT)2 * apq);
                RT t = (theta >= (RT)0 ? (RT)1 : (RT)-1) / (fabs(theta) + sqrt(theta * theta + (RT)1));
                RT cs = (RT)1 / sqrt(t * t + (RT)1);
                RT sn = t * cs;
                for (int r = 0; r < 6; ++r) {  // columns p, q
                    RT crp = C[r][p], crq = C[r][q];
                    C[r][p] = cs * crp - sn * crq;
                    C[r][q] = sn * crp + cs * crq;
                }
                for (int r = 0; r < 6; ++r) {  // rows p, q
                    RT cpr = C[p][r], cqr = C[q][r];
                    C[p][r] = cs * cpr - sn * cqr;
                    C[q][r] = sn * cpr + cs * cqr;
                }
                for (int r = 0; r < 6; ++r) {
                    RT vrp = V[r][p], vrq = V[r][q];
                    V[r][p] = cs * vrp - sn * vrq;
                    V[r][q] = sn * vrp + cs * vrq;
                }
            }
    }
    RT lam[6];
    for (int p = 0; p < 6; ++p) {
        RT l = fabs(C[p][p]);
        lam[p] = l > floor ? l : floor;
    }
    for (int p = 0; p < 6; ++p)
        for (int q = p; q < 6; ++q) {
            RT s = 0;
            for (int r = 0; r < 6; ++r) s += V[p][r] * lam[r] * V[q][r];
            C[p][q] = s;
            C[q][p] = s;
        }
}

// Column j of E_a = M_a(row j of Q): the Mandel stretch from a unit move of
// vertex a along axis j (rotated into the cluster frame).
template <typename KT>
__device__ __forceinline__ void Ecol(const KT (&g)[3], const KT (&u)[3], KT (&e)[6]) {
    const KT is2 = (KT)kInvSqrt2;
    e[0] = u[0] * g[0];
    e[1] = u[1] * g[1];
    e[2] = u[2] * g[2];
    e[3] = (u[1] * g[2] + u[2] * g[1]) * is2;
    e[4] = (u[0] * g[2] + u[2] * g[0]) * is2;
    e[5] = (u[0] * g[1] + u[1] * g[0]) * is2;
}

// Element blocks K_ab = W E_a^T C E_b for a <= b, generic 6x6 C, in the
// element-block layout (diagonal blocks: upper entries only).
template <typename KT>
__device__ __forceinline__ void blocks_generic(const KT (&C)[6][6], const KT (&G)[4][3], const KT (&Q)[3][3],
                                               KT W, KT* __restrict__ out) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        KT CE[3][6];  // (C E_b) columns
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            KT e[6];
            KT u[3] = {Q[j][0], Q[j][1], Q[j][2]};
            Ecol<KT>(G[b], u, e);
#pragma unroll
            for (int p = 0; p < 6; ++p) {
                KT s = 0;
#pragma unroll
                for (int q = 0; q < 6; ++q) s += C[p][q] * e[q];
                CE[j][p] = s * W;
            }
        }
#pragma unroll
        for (int a = 0; a <= b; ++a) {
            KT* o = out + ke_offset(a, b);
            KT blk[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                KT e[6];
                KT u[3] = {Q[i][0], Q[i][1], Q[i][2]};
                Ecol<KT>(G[a], u, e);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    if (a == b && j < i) continue;   // diagonal block: upper entries
                    KT s = 0;
#pragma unroll
                    for (int p = 0; p < 6; ++p) s += e[p] * CE[j][p];
                    blk[i][j] = s;
                }
            }
            if (a == b) {
                o[0] = blk[0][0]; o[1] = blk[1][1]; o[2] = blk[2][2];
                o[3] = blk[1][2]; o[4] = blk[0][2]; o[5] = blk[0][1];
            } else {
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) o[3 * i + j] = blk[i][j];
            }
        }
    }
}

// ARAP / co-rotational blocks in closed form:
// K_ab = W [mu (G_a.G_b) I + mu h_b h_a^T + lam h_a h_b^T], h_a = Q G_a,
// in the element-block layout.
template <typename KT>
__device__ __forceinline__ void blocks_quadratic(const KT (&G)[4][3], const KT (&Q)[3][3], KT wm, KT wl,
                                                 KT* __restrict__ out) {
    KT h[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) h[a][i] = Q[i][0] * G[a][0] + Q[i][1] * G[a][1] + Q[i][2] * G[a][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = a; b < 4; ++b) {
            KT* o = out + ke_offset(a, b);
            const KT gg = wm * (G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2]);
            KT blk[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    blk[i][j] = (i == j ? gg : (KT)0) + wm * h[b][i] * h[a][j] + wl * h[a][i] * h[b][j];
            if (a == b) {
                o[0] = blk[0][0]; o[1] = blk[1][1]; o[2] = blk[2][2];
                o[3] = blk[1][2]; o[4] = blk[0][2]; o[5] = blk[0][1];
            } else {
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) o[3 * i + j] = blk[i][j];
            }
        }
}

// Orthogonal polar factor by Higham's scaled Newton iteration
// X <- (gamma X + X^{-T} / gamma) / 2 (N. J. Higham, "Computing the polar
// decomposition -- with applications", SIAM J. Sci. Stat. Comput. 1986).
template <typename RT>
__device__ bool polar_newton(const double (&F)[3][3], RT (&R)[3][3]) {
    RT X[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) X[i][j] = (RT)F[i][j];
    const RT tol = sizeof(RT) == 8 ? (RT)1e-13 : (RT)1e-6;
    for (int it = 0; it < 30; ++it) {
        RT c00 = X[1][1] * X[2][2] - X[1][2] * X[2][1], c01 = X[1][2] * X[2][0] - X[1][0] * X[2][2],
           c02 = X[1][0] * X[2][1] - X[1][1] * X[2][0];
        RT c10 = X[0][2] * X[2][1] - X[0][1] * X[2][2], c11 = X[0][0] * X[2][2] - X[0][2] * X[2][0],
           c12 = X[0][1] * X[2][0] - X[0][0] * X[2][1];
        RT c20 = X[0][1] * X[1][2] - X[0][2] * X[1][1], c21 = X[0][2] * X[1][0] - X[0][0] * X[1][2],
           c22 = X[0][0] * X[1][1] - X[0][1] * X[1][0];
        RT det = X[0][0] * c00 + X[0][1] * c01 + X[0][2] * c02;
        if (det == (RT)0) return false;
        // X^{-T} = cof(X) / det
        RT IT[3][3] = {{c00 / det, c01 / det, c02 / det}, {c10 / det, c11 / det, c12 / det},
                       {c20 / det, c21 / det, c22 / det}};
        RT nx = 0, ni = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                nx += X[i][j] * X[i][j];
                ni += IT[i][j] * IT[i][j];
            }
        RT gam = sqrt(sqrt(ni / nx));
        RT diff = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                RT y = (RT)0.5 * (gam * X[i][j] + IT[i][j] / gam);
                diff += (y - X[i][j]) * (y - X[i][j]);
                X[i][j] = y;
            }
        if (diff <= tol * tol * (RT)3) break;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R[i][j] = X[i][j];
    return true;
}

// Eigenvectors of a symmetric 3x3 H by cyclic Jacobi rotations (Golub & Van
// Loan, "Matrix Computations", symmetric Jacobi method): on return H is
// (nearly) diagonal and the columns of V are the eigenvectors.
__device__ void jacobi3(double (&H)[3][3], double (&V)[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 12; ++sweep) {
        const double off = H[0][1] * H[0][1] + H[0][2] * H[0][2] + H[1][2] * H[1][2];
        const double dia = H[0][0] * H[0][0] + H[1][1] * H[1][1] + H[2][2] * H[2][2];
        if (off <= 1e-32 * dia) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (H[p][q] == 0.0) continue;
                const double th = (H[q][q] - H[p][p]) / (2.0 * H[p][q]);
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) {   // H <- H J (columns p, q)
                    const double hp = H[k][p], hq = H[k][q];
                    H[k][p] = c * hp - s * hq;
                    H[k][q] = s * hp + c * hq;
                }
                for (int k = 0; k < 3; ++k) {   // H <- J^T H (rows p, q)
                    const double hp = H[p][k], hq = H[q][k];
                    H[p][k] = c * hp - s * hq;
                    H[q][k] = s * hp + c * hq;
                }
                for (int k = 0; k < 3; ++k) {
                    const double vp = V[k][p], vq = V[k][q];
                    V[k][p] = c * vp - s * vq;
                    V[k][q] = s * vp + c * vq;
                }
            }
    }
}

// Rotation factor R (det +1) of F = R P, P symmetric.  For det F < 0 the
// eigenvalue of P of least magnitude is the negative one: the orthogonal polar
// factor U (det -1) is reflected along the eigenvector of U^T F with the
// smallest eigenvalue.  Returns false if F is singular.
__device__ bool polar_rotation(const double (&F)[3][3], double (&R)[3][3]) {
    double U[3][3];
    if (!polar_newton<double>(F, U)) return false;
    const double detU = U[0][0] * (U[1][1] * U[2][2] - U[1][2] * U[2][1]) -
                        U[0][1] * (U[1][0] * U[2][2] - U[1][2] * U[2][0]) +
                        U[0][2] * (U[1][0] * U[2][1] - U[1][1] * U[2][0]);
    if (detU > 0.0) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) R[i][j] = U[i][j];
        return true;
    }
    double H[3][3], V[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double hij = 0.0, hji = 0.0;
            for (int k = 0; k < 3; ++k) {
                hij += U[k][i] * F[k][j];
                hji += U[k][j] * F[k][i];
            }
            H[i][j] = 0.5 * (hij + hji);
        }
    jacobi3(H, V);
    int im = 0;
    for (int i = 1; i < 3; ++i)
        if (H[i][i] < H[im][im]) im = i;
    const double v[3] = {V[0][im], V[1][im], V[2][im]};
    for (int i = 0; i < 3; ++i) {
        const double uv = U[i][0] * v[0] + U[i][1] * v[1] + U[i][2] * v[2];
        for (int j = 0; j < 3; ++j) R[i][j] = U[i][j] - 2.0 * uv * v[j];
    }
    return true;
}

// Rotation of tet k: its rig cluster's handle rotation (§3.1), or, in the
// polar-rotation mode, the rotation factor of its own F (the rotation a
// co-rotational FEM element takes; the cluster rotation if F is singular).
// qs: the problem's handle rotations staged in shared memory, or null.
__device__ __forceinline__ void tet_rotation(const ElemArgs& A, const double* __restrict__ xf,
                                             const double (*qs)[9], int k, const double (&xa)[4][3],
                                             const double (&G)[4][3], double (&Q)[3][3]) {
    if (A.rot_polar) {
        double F[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                double f = 0.0;
#pragma unroll
                for (int a = 1; a < 4; ++a) f = fma(xa[a][i] - xa[0][i], G[a][j], f);
                F[i][j] = f;
            }
        if (polar_rotation(F, Q)) return;
    }
    const int h = A.mesh.cluster[k];
    if (qs) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Q[i][j] = qs[h][3 * i + j];
    } else {
        load_Q(xf, h, Q);
    }
}

// The problem's handle rotations into shared memory (every thread calls it;
// returns qs, or null when the rig has more handles than are staged).
__device__ __forceinline__ const double (*stage_pose(double (*qs)[9], const double* __restrict__ xf,
                                                     int H))[9] {
    if (H > kMaxStagedHandles) return nullptr;
    for (int i = threadIdx.x; i < 9 * H; i += blockDim.x) {
        const int h = i / 9, e = i - 9 * h;
        qs[h][e] = xf[12 * h + 4 * (e / 3) + e % 3];
    }
    __syncthreads();
    return qs;
}

// The float pairs of the rotations (split once per problem by k_x_split), in
// the same shared memory (8 bytes per entry); global memory past the limit.
__device__ __forceinline__ const float2 (*stage_pose_ff(float2 (*qs)[9], const float2* __restrict__ qff, int H))[9] {
    if (H > kMaxStagedHandles) return reinterpret_cast<const float2(*)[9]>(qff);
    for (int i = threadIdx.x; i < 9 * H; i += blockDim.x) qs[i / 9][i % 9] = qff[i];
    __syncthreads();
    return qs;
}

// Energy terms that live on vertex v at position y: -f_v . y for an external
// force (§4, "Collision response") and k_s/2 |y - x_p|^2 for a pin under the
// penalty form of Eq. 6.
__device__ __forceinline__ double vertex_energy(const ElemArgs& A, int b, int v, const double (&y)[3]) {
    double e = 0.0;
    if (A.fext) {
        const double* f = A.fext + (size_t)b * A.fext_stride + 3 * (size_t)v;
        e -= f[0] * y[0] + f[1] * y[1] + f[2] * y[2];
    }
    if (A.constraint == 1 && A.mesh.pin_handle_v[v] >= 0) {
        const double* xp = A.slot.xp + ((size_t)b * A.mesh.n + v) * 3;
        const double d0 = y[0] - xp[0], d1 = y[1] - xp[1], d2 = y[2] - xp[2];
        e += 0.5 * A.ks * (d0 * d0 + d1 * d1 + d2 * d2);
    }
    return e;
}

// ---------------------------------------------------------------------------
// Thread k handles tet k (k < m) and the vertex terms of vertex k (k < n).
// HESS = false: energy and forces only (a gradient test needs no Hessian).
//
// Stores: each warp's 32 tets write contiguous records (12 FP64 forces, 78
// element-block values), so a thread's record is first built in the warp's
// shared-memory area and the warp then copies the area out with consecutive
// lanes on consecutive words; forces first, then the blocks in the same area.
// FP64 Hessians (KT = double) are written directly.
constexpr int kStageWords = 32 * kKe;   // floats per warp: 32 records of blocks (or 32 x 12 doubles of forces)
static_assert(kStageWords >= 32 * 12 * 2, "the force stage fits");

// Positions and handle rotations of the active problems as float pairs (hi =
// the value rounded to FP32, lo = the remainder rounded), read by the
// float-float element path.
__global__ void k_x_split(ElemArgs A) {
    const int b = blockIdx.y;
    if (!A.slot.active[b]) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 3 * A.mesh.n) {
        const FF v = ff_split(A.slot.x[(size_t)b * A.mesh.n * 3 + i]);
        A.slot.xff[(size_t)b * A.mesh.n * 3 + i] = make_float2(v.hi, v.lo);
    }
    const int H = A.mesh.H;
    if (i < 9 * H) {
        const int h = i / 9, e = i - 9 * h;
        const FF v = ff_split(A.slot.xf[((size_t)b * H + h) * 12 + 4 * (e / 3) + e % 3]);
        A.slot.qff[(size_t)b * H * 9 + i] = make_float2(v.hi, v.lo);
    }
}

template <typename KT, int MODEL, bool HESS>
__global__ void __launch_bounds__(kTetTile, 4) k_element(ElemArgs A) {
    __shared__ double qsh[kMaxStagedHandles][9];
    __shared__ __align__(16) float stage[kTetTile / 32][kStageWords];
    const int b = blockIdx.y;
    if (!A.slot.active[b]) return;   // block-uniform
    const MeshDev& M = A.mesh;
    const int m = M.m, n = M.n;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k0 = k - lane;                         // the warp's first tet
    const int nvalid = max(0, min(32, m - k0));      // tets of this warp
    const double* xf = A.slot.xf + (size_t)b * M.H * 12;
    // mixed path at newton_tol >= kF32ForcesTol with rig rotations: F, S,
    // stress and energy in float-float from the positions' float pairs
    const bool ffp = sizeof(KT) == 4 && A.ff_elem;   // uniform
    const double(*qs)[9] = ffp ? nullptr : stage_pose(qsh, xf, M.H);
    const float2(*qsf)[9] =
        ffp ? stage_pose_ff(reinterpret_cast<float2(*)[9]>(qsh), A.slot.qff + (size_t)b * M.H * 9, M.H) : nullptr;
    double en[1] = {0.0};
    FF enf{0.f, 0.f};   // the float-float path's energy
    double xa[4][3], G[4][3], Q[3][3], F[3][3], S[6], sig[6];
    double mu = 0.0, lam = 0.0, w = 0.0;
    FF Sff[6], Qff[3][3], muf{0.f, 0.f}, lamf{0.f, 0.f};
    double* gs = reinterpret_cast<double*>(stage[warp]);   // [32][12] forces
    if (ffp && k < m) {
        const float2* xp = A.slot.xff + (size_t)b * n * 3;
        const int4 tv = M.tet[k];
        const int id[4] = {tv.x, tv.y, tv.z, tv.w};
        FF xa4[4][3], Gff[3][3];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float2 v = xp[3 * (size_t)id[a] + i];
                xa4[a][i] = FF{v.x, v.y};
            }
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                Gff[r][c] = FF{M.Dminv32[(size_t)(3 * r + c) * m + k], M.Dminv_lo[(size_t)(3 * r + c) * m + k]};
        const int h = M.cluster[k];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float2 v = qsf[h][3 * i + j];
                Qff[i][j] = FF{v.x, v.y};
            }
        stretch_ff(xa4, Gff, Qff, Sff);
        // (W mu, W lam): Psi, sigma and the Hessian below come out weighted by W
        const float4 ml = M.mulam_ff[k];
        muf = FF{ml.x, ml.y};
        lamf = FF{ml.z, ml.w};
        float sg[6];
        enf = psi_sigma_ff<MODEL>(Sff, muf, lamf, sg);
        // forces f_a = W Q sigma G_a in FP32 from the stress (as on the FP32-force path)
        const float sw[3][3] = {{sg[0], sg[5], sg[4]}, {sg[5], sg[1], sg[3]}, {sg[4], sg[3], sg[2]}};
        float P[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                P[i][j] = Qff[i][0].hi * sw[0][j] + Qff[i][1].hi * sw[1][j] + Qff[i][2].hi * sw[2][j];
        double* gl = gs + 12 * lane;
        float f0[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float f = P[i][0] * Gff[a][0].hi + P[i][1] * Gff[a][1].hi + P[i][2] * Gff[a][2].hi;
                gl[3 * (a + 1) + i] = f2d_exact(f);
                f0[i] -= f;
            }
#pragma unroll
        for (int i = 0; i < 3; ++i) gl[i] = f2d_exact(f0[i]);
    } else if (k < m) {
        const double* x = A.slot.x + (size_t)b * n * 3;
        const int4 tv = M.tet[k];
        gather_x<float>(x, nullptr, 0.0, tv, xa);
        load_G(M.Dminv64, m, k, G);
        tet_rotation(A, xf, qs, k, xa, G, Q);
        stretch(xa, G, Q, F, S);
        mu = M.mu[k];
        lam = M.lam[k];
        w = M.vol[k];
        double* gl = gs + 12 * lane;
        if (sizeof(KT) == 4 && A.f32_forces) {
            // mixed path: F, S, the energy and the stress in FP64 (positions and
            // rotations cancel in F and S, the stress terms of order mu cancel
            // near the rest state); the stress rounded to FP32 keeps its own
            // relative precision, and the forces W Q sigma G_a are formed from
            // it in FP32
            en[0] = w * psi_sigma<MODEL>(S, mu, lam, sig);
            float sg[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) sg[i] = (float)sig[i];
            const float wf = (float)w;
            const float sw[3][3] = {{wf * sg[0], wf * sg[5], wf * sg[4]},
                                    {wf * sg[5], wf * sg[1], wf * sg[3]},
                                    {wf * sg[4], wf * sg[3], wf * sg[2]}};
            float Qf[3][3], Gf[3][3], P[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    Qf[i][j] = (float)Q[i][j];
                    Gf[i][j] = M.Dminv32[(size_t)(3 * i + j) * m + k];
                }
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    P[i][j] = Qf[i][0] * sw[0][j] + Qf[i][1] * sw[1][j] + Qf[i][2] * sw[2][j];
            float f0[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float f = P[i][0] * Gf[a][0] + P[i][1] * Gf[a][1] + P[i][2] * Gf[a][2];
                    gl[3 * (a + 1) + i] = (double)f;
                    f0[i] -= f;
                }
#pragma unroll
            for (int i = 0; i < 3; ++i) gl[i] = (double)f0[i];
        } else {
            en[0] = w * psi_sigma<MODEL>(S, mu, lam, sig);
            // forces f_a = W Lambda G_a, Lambda = Q sigma (a = 1..3), f_0 = -(f_1 + f_2 + f_3)
            const double sw[3][3] = {{w * sig[0], w * sig[5], w * sig[4]},
                                     {w * sig[5], w * sig[1], w * sig[3]},
                                     {w * sig[4], w * sig[3], w * sig[2]}};
            double P[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) P[i][j] = Q[i][0] * sw[0][j] + Q[i][1] * sw[1][j] + Q[i][2] * sw[2][j];
            double f0[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int a = 1; a < 4; ++a)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const double f = P[i][0] * G[a][0] + P[i][1] * G[a][1] + P[i][2] * G[a][2];
                    gl[3 * a + i] = f;
                    f0[i] -= f;
                }
#pragma unroll
            for (int i = 0; i < 3; ++i) gl[i] = f0[i];
        }
    }
    __syncwarp();
    {   // forces out: the warp's 32 contiguous 96-byte records
        double* ge = A.slot.ge + ((size_t)b * m + k0) * 12;
        for (int i = lane; i < 12 * nvalid; i += 32) ge[i] = gs[i];
    }
    __syncwarp();
    if (HESS && k < m) {
        KT* ke = sizeof(KT) == 4 ? reinterpret_cast<KT*>(stage[warp]) + kKe * lane
                                 : (KT*)A.slot.Ke + ((size_t)b * m + k) * kKe;
        // FP32 copies of the shape gradients and the rotation (the Hessian's precision)
        KT Gk[4][3], Qk[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Gk[r + 1][c] = sizeof(KT) == 4 ? (KT)M.Dminv32[(size_t)(3 * r + c) * m + k] : (KT)G[r + 1][c];
                Qk[r][c] = ffp ? (KT)Qff[r][c].hi : (KT)Q[r][c];
            }
#pragma unroll
        for (int c = 0; c < 3; ++c) Gk[0][c] = -(Gk[1][c] + Gk[2][c] + Gk[3][c]);
        if (MODEL == 2) {
            bool fp64 = sizeof(KT) == 8;
            float sf[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) sf[i] = ffp ? Sff[i].hi : (float)S[i];
            if (!fp64) {  // near-degenerate or inverted stretch: FP64 Hessian
                const float s0 = sf[0], s1 = sf[1], s2 = sf[2], s3 = sf[3], s4 = sf[4], s5 = sf[5];
                const float J = s0 * (s1 * s2 - s3 * s3) + s5 * (s4 * s3 - s2 * s5) + s4 * (s5 * s3 - s1 * s4);
                fp64 = J < (float)kFallbackJ;
            }
            KT C[6][6];
            if (fp64) {
                // the Hessian of a strongly strained tet in FP64 (its terms cancel);
                // the SPD filter of the result in the kernel's precision (GB300 runs
                // FP64 at a small fraction of FP32, and the filter needs no more)
                double Cd[6][6], Sd[6];
#pragma unroll
                for (int i = 0; i < 6; ++i) Sd[i] = ffp ? (double)Sff[i].hi + (double)Sff[i].lo : S[i];
                if (ffp) {   // weighted by W, as the float-float path's Hessian
                    mu = (double)muf.hi + (double)muf.lo;
                    lam = (double)lamf.hi + (double)lamf.lo;
                }
                snh_hessian<double>(Sd, mu, lam, Cd);
#pragma unroll
                for (int p = 0; p < 6; ++p)
#pragma unroll
                    for (int q = 0; q < 6; ++q) C[p][q] = (KT)Cd[p][q];
            } else if (ffp) {
                snh_hessian_f(sf, muf.hi, lamf.hi, reinterpret_cast<float(&)[6][6]>(C));
            } else {
                snh_hessian<KT>(S, mu, lam, C);
            }
            const KT floor = ffp ? (KT)((float)kSpdEps * muf.hi) : (KT)(kSpdEps * mu);
            if (!chol_shifted_ok<KT>(C, floor)) filter_spd<KT>(C, floor);
            blocks_generic<KT>(C, Gk, Qk, ffp ? (KT)1 : (KT)w, ke);
        } else if (ffp) {
            blocks_quadratic<KT>(Gk, Qk, (KT)muf.hi, (KT)(MODEL == 1 ? lamf.hi : 0.f), ke);
        } else {
            blocks_quadratic<KT>(Gk, Qk, (KT)(w * mu), (KT)(w * (MODEL == 1 ? lam : 0.0)), ke);
        }
    }
    if (HESS && sizeof(KT) == 4) {   // element blocks out: 32 contiguous 312-byte records
        __syncwarp();
        const float2* src = reinterpret_cast<const float2*>(stage[warp]);
        float2* dst = reinterpret_cast<float2*>((float*)A.slot.Ke + ((size_t)b * m + k0) * kKe);
        for (int i = lane; i < (kKe / 2) * nvalid; i += 32) dst[i] = src[i];
    }
    const bool vterms = A.fext || A.constraint == 1;   // uniform
    if (k < n && (vterms || !ffp)) {
        const double* xv = A.slot.x + ((size_t)b * n + k) * 3;
        const double y[3] = {xv[0], xv[1], xv[2]};
        const double ev = vertex_energy(A, b, k, y);
        if (ffp) enf = ff_add(enf, ff_split(ev));
        else en[0] += ev;
    }
    // the float-float path sums its warp's energies in float-float and enters
    // the block sum with the warp's total (FP64 from there on)
    if (ffp) en[0] = ff_warp_sum(enf);
    double tot[1];
    double* part = A.slot.part + (size_t)b * A.slot.part_tiles * 4;
    if (tile_commit<1>(en, part, blockIdx.x, gridDim.x, &A.slot.sc[b].tk_e, 0, tot, ffp) && threadIdx.x == 0)
        A.slot.sc[b].energy = tot[0];
}

// Energy at x + alpha_b dx_b (line search trial, a6).
template <typename T, int MODEL>
__global__ void __launch_bounds__(kTetTile) k_energy_trial(ElemArgs A) {
    __shared__ double qsh[kMaxStagedHandles][9];
    const int b = blockIdx.y;
    if (!A.slot.active[b]) return;   // block-uniform
    const MeshDev& M = A.mesh;
    const int m = M.m, n = M.n;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const double* xf = A.slot.xf + (size_t)b * M.H * 12;
    const double(*qs)[9] = stage_pose(qsh, xf, M.H);
    double en[1] = {0.0};
    if (k < m) {
        const double* x = A.slot.x + (size_t)b * n * 3;
        // the dx field: 4 elements per vertex
        const T* dx = rec_field((const T*)A.slot.vec + (size_t)b * kVecStride * npad32(n) + kOffRec * npad32(n),
                                npad32(n), kRecDX, 0);
        double xa[4][3], G[4][3], Q[3][3], F[3][3], S[6], sig[6];
        gather_x<T>(x, dx, A.slot.alpha[b], M.tet[k], xa, 4);
        load_G(M.Dminv64, m, k, G);
        tet_rotation(A, xf, qs, k, xa, G, Q);
        stretch(xa, G, Q, F, S);
        en[0] = M.vol[k] * psi_sigma<MODEL>(S, M.mu[k], M.lam[k], sig);
    }
    if (k < n) {
        const double* xv = A.slot.x + ((size_t)b * n + k) * 3;
        const T* dv = rec_field((const T*)A.slot.vec + (size_t)b * kVecStride * npad32(n) + kOffRec * npad32(n),
                                npad32(n), kRecDX, k);
        const double al = A.slot.alpha[b];
        const double y[3] = {fma(al, (double)dv[0], xv[0]), fma(al, (double)dv[1], xv[1]),
                             fma(al, (double)dv[2], xv[2])};
        en[0] += vertex_energy(A, b, k, y);
    }
    double tot[1];
    double* part = A.slot.part + (size_t)b * A.slot.part_tiles * 4;
    if (tile_commit<1>(en, part, blockIdx.x, gridDim.x, &A.slot.sc[b].tk_e, 0, tot) && threadIdx.x == 0)
        A.slot.sc[b].energy_trial = tot[0];
}

// Pin targets x_p = Q_h X_v + t_h (§3.2) and the initial guess (a0).
__global__ void k_pose_init(ElemArgs A, int init) {
    const int b = blockIdx.y;
    if (!A.slot.active[b]) return;
    const MeshDev& M = A.mesh;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= M.n) return;
    const double* xf = A.slot.xf + (size_t)b * M.H * 12;
    double* x = A.slot.x + ((size_t)b * M.n + v) * 3;
    const double* X = M.X + 3 * (size_t)v;
    const int ph = M.pin_handle_v[v];
    int h = ph >= 0 ? ph : (init == 0 ? M.vhandle[v] : -1);
    if (h >= 0) {
        const double* T = xf + 12 * h;
        double y[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) y[i] = (T[4 * i] * X[0] + T[4 * i + 1] * X[1]) + T[4 * i + 2] * X[2] + T[4 * i + 3];
#pragma unroll
        for (int i = 0; i < 3; ++i) x[i] = y[i];
        if (ph >= 0) {
            double* xp = A.slot.xp + ((size_t)b * M.n + v) * 3;
#pragma unroll
            for (int i = 0; i < 3; ++i) xp[i] = y[i];
        }
    } else if (init == 1) {
#pragma unroll
        for (int i = 0; i < 3; ++i) x[i] = X[i];
    }
}

// Warm starts (SNH): the correction the slot's last solve needed beyond its own
// predictor result, dcorr = x - xpred, taken before the new pose is applied.
__global__ void k_warm_save(ElemArgs A) {
    const int b = blockIdx.y;
    if (!A.slot.active[b]) return;
    const int n = A.mesh.n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    const size_t o = (size_t)b * n * 3 + i;
    A.slot.dcorr[o] = A.slot.x[o] - A.slot.xpred[o];
}

// After the predictor step: keep x as xpred for the next solve and, with
// apply, add the last correction turned by the rotation change of the handle
// each free vertex's rest position clusters to, Q_h Q_h,prev^T dcorr_v.
__global__ void k_warm_step(ElemArgs A, int apply) {
    const int b = blockIdx.y;
    if (!A.slot.active[b]) return;
    const MeshDev& M = A.mesh;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= M.n) return;
    const size_t o = ((size_t)b * M.n + v) * 3;
    double* x = A.slot.x + o;
    double* xp = A.slot.xpred + o;
    xp[0] = x[0];
    xp[1] = x[1];
    xp[2] = x[2];
    if (!apply || M.pin_handle_v[v] >= 0) return;
    const int h = M.vhandle[v];
    const double* Tn = A.slot.xf + (size_t)b * M.H * 12 + 12 * h;
    const double* Tp = A.slot.xf_prev + (size_t)b * M.H * 12 + 12 * h;
    const double* d = A.slot.dcorr + o;
    double y[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) y[i] = Tp[i] * d[0] + Tp[4 + i] * d[1] + Tp[8 + i] * d[2];   // Qp^T d
#pragma unroll
    for (int i = 0; i < 3; ++i) x[i] += (Tn[4 * i] * y[0] + Tn[4 * i + 1] * y[1]) + Tn[4 * i + 2] * y[2];
}

template <int MODEL>
__global__ void k_elem_out(ElemArgs A, int b, double* __restrict__ s_out, double* __restrict__ lam_out) {
    const MeshDev& M = A.mesh;
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= M.m) return;
    const int k = M.tperm[o];
    const double* x = A.slot.x + (size_t)b * M.n * 3;
    const double* xf = A.slot.xf + (size_t)b * M.H * 12;
    double xa[4][3], G[4][3], Q[3][3], F[3][3], S[6], sig[6];
    gather_x<float>(x, nullptr, 0.0, M.tet[k], xa);
    load_G(M.Dminv64, M.m, k, G);
    tet_rotation(A, xf, nullptr, k, xa, G, Q);
    stretch(xa, G, Q, F, S);
    psi_sigma<MODEL>(S, M.mu[k], M.lam[k], sig);
    if (s_out)
        for (int i = 0; i < 6; ++i) s_out[6 * (size_t)o + i] = S[i];
    if (lam_out) {
        const double sm[3][3] = {{sig[0], sig[5], sig[4]}, {sig[5], sig[1], sig[3]}, {sig[4], sig[3], sig[2]}};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                lam_out[9 * (size_t)o + 3 * i + j] = Q[i][0] * sm[0][j] + Q[i][1] * sm[1][j] + Q[i][2] * sm[2][j];
    }
}

// Diagnostics: inverted tets, max |skew(Q^T F)|/|F|, max angle(Q, polar(F)).
// out3: [0] count, [1] float bits of max skew, [2] float bits of max angle.
__global__ void k_diag(ElemArgs A, int b, unsigned* __restrict__ out3) {
    const MeshDev& M = A.mesh;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M.m) return;
    const double* x = A.slot.x + (size_t)b * M.n * 3;
    const double* xf = A.slot.xf + (size_t)b * M.H * 12;
    double xa[4][3], G[4][3], Q[3][3], F[3][3], S[6];
    gather_x<float>(x, nullptr, 0.0, M.tet[k], xa);
    load_G(M.Dminv64, M.m, k, G);
    tet_rotation(A, xf, nullptr, k, xa, G, Q);
    stretch(xa, G, Q, F, S);
    const double detF = F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) -
                        F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
                        F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
    double nF = 0, nK = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            nF += F[i][j] * F[i][j];
            double aij = Q[0][i] * F[0][j] + Q[1][i] * F[1][j] + Q[2][i] * F[2][j];
            double aji = Q[0][j] * F[0][i] + Q[1][j] * F[1][i] + Q[2][j] * F[2][i];
            nK += 0.25 * (aij - aji) * (aij - aji);
        }
    const float skew = (float)(sqrt(nK) / fmax(sqrt(nF), 1e-300));
    atomicMax(&out3[1], __float_as_uint(skew));
    if (detF <= 0.0) {
        atomicAdd(&out3[0], 1u);
        return;
    }
    // polar rotation in FP32; FP64 when the tet is nearly degenerate
    double ang;
    const double cube = pow(sqrt(nF / 3.0), 3.0);
    if (detF < 1e-2 * cube) {
        double R[3][3];
        if (!polar_newton<double>(F, R)) return;
        double tr = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) tr += Q[i][j] * R[i][j];
        ang = acos(fmin(1.0, fmax(-1.0, 0.5 * (tr - 1.0))));
    } else {
        float R[3][3];
        if (!polar_newton<float>(F, R)) return;
        double tr = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) tr += Q[i][j] * (double)R[i][j];
        ang = acos(fmin(1.0, fmax(-1.0, 0.5 * (tr - 1.0))));
    }
    atomicMax(&out3[2], __float_as_uint((float)ang));
}

template <typename KT>
void launch_element_t(const ElemArgs& a, int B, bool hess, cudaStream_t s) {
    dim3 grid((std::max(a.mesh.m, a.mesh.n) + kTetTile - 1) / kTetTile, B);
    if (hess) {
        switch (a.model) {
            case 0: k_element<KT, 0, true><<<grid, kTetTile, 0, s>>>(a); break;
            case 1: k_element<KT, 1, true><<<grid, kTetTile, 0, s>>>(a); break;
            default: k_element<KT, 2, true><<<grid, kTetTile, 0, s>>>(a); break;
        }
    } else {
        switch (a.model) {
            case 0: k_element<KT, 0, false><<<grid, kTetTile, 0, s>>>(a); break;
            case 1: k_element<KT, 1, false><<<grid, kTetTile, 0, s>>>(a); break;
            default: k_element<KT, 2, false><<<grid, kTetTile, 0, s>>>(a); break;
        }
    }
}

template <typename T>
void launch_trial_t(const ElemArgs& a, int B, cudaStream_t s) {
    dim3 grid((std::max(a.mesh.m, a.mesh.n) + kTetTile - 1) / kTetTile, B);
    switch (a.model) {
        case 0: k_energy_trial<T, 0><<<grid, kTetTile, 0, s>>>(a); break;
        case 1: k_energy_trial<T, 1><<<grid, kTetTile, 0, s>>>(a); break;
        default: k_energy_trial<T, 2><<<grid, kTetTile, 0, s>>>(a); break;
    }
}

}  // namespace

void launch_pose_init(const ElemArgs& a, int B, int init, cudaStream_t s) {
    dim3 grid((a.mesh.n + 255) / 256, B);
    k_pose_init<<<grid, 256, 0, s>>>(a, init);
}

void launch_warm_save(const ElemArgs& a, int B, cudaStream_t s) {
    dim3 grid((3 * a.mesh.n + 255) / 256, B);
    k_warm_save<<<grid, 256, 0, s>>>(a);
}

void launch_warm_step(const ElemArgs& a, int B, int apply, cudaStream_t s) {
    dim3 grid((a.mesh.n + 255) / 256, B);
    k_warm_step<<<grid, 256, 0, s>>>(a, apply);
}

void launch_element(const ElemArgs& a, int B, cudaStream_t s, bool hess) {
    if (a.slot.prec == 1) {
        if (a.ff_elem) k_x_split<<<dim3((max(3 * a.mesh.n, 9 * a.mesh.H) + 255) / 256, B), 256, 0, s>>>(a);
        launch_element_t<float>(a, B, hess, s);
    } else {
        launch_element_t<double>(a, B, hess, s);
    }
}

void launch_energy_trial(const ElemArgs& a, int B, cudaStream_t s) {
    if (a.slot.prec == 1) launch_trial_t<float>(a, B, s);
    else launch_trial_t<double>(a, B, s);
}

void launch_elem_out(const ElemArgs& a, int b, double* s_out, double* lam_out, cudaStream_t s) {
    int grid = (a.mesh.m + 127) / 128;
    switch (a.model) {
        case 0: k_elem_out<0><<<grid, 128, 0, s>>>(a, b, s_out, lam_out); break;
        case 1: k_elem_out<1><<<grid, 128, 0, s>>>(a, b, s_out, lam_out); break;
        default: k_elem_out<2><<<grid, 128, 0, s>>>(a, b, s_out, lam_out); break;
    }
}

void launch_diag(const ElemArgs& a, int b, unsigned* out3, cudaStream_t s) {
    k_diag<<<(a.mesh.m + 127) / 128, 128, 0, s>>>(a, b, out3);
}

}  // namespace mfem
