// Coarse solve and correction of the two-level preconditioner on the tensor
// cores, fused into one kernel per mesh and PCG iteration.
//
// u = zb + P e,  e = A_c^{-1} r_c  for every two-level problem of one mesh: the
// product is the one dense contraction of the solve (the preconditioner's
// reduced space; the method itself has none, paper §5) and it is bound by
// streaming A_c^{-1}, stored once per mesh in BF16.
//
//   * A cluster of kFuSplit CTAs owns a row block of kFuAggsBlk aggregates
//     (their 6 kFuAggsBlk rows of A_c^{-1}, padded to the MMA's M = 128); CTA q
//     of the cluster streams the q-th part of the K range: per chunk of kTcKC
//     columns one 32 KB block of A (packed at set-up in the MMA's no-swizzle
//     K-major core-matrix layout) and the matching 12 KB chunk of the B
//     operand, by 1-D bulk copies (the TMA engine) into a ring of kFuStages
//     shared-memory stages; one thread issues the MMAs (M = 128, N = 48,
//     K = 16), FP32 accumulation in tensor memory.
//   * The cluster adds its kFuSplit partial products through distributed
//     shared memory in rank order (deterministic), CTA q keeping the rows of
//     its kFuAggsCta aggregates; then every thread of the CTA applies the
//     correction to those aggregates' vertex rows: u_i = zb_i + Q_a (e_t +
//     e_w x (X_i - c_a)), written to the neighbour record the next SpMV
//     gathers.  No slice partials, no separate correction kernel.
//   * B: each problem's r_c split exactly into three BF16 parts (r = hi + mid +
//     lo: 3 x 8 significand bits hold the FP32 value), N = 48 columns for 16
//     request slots; the restriction writes it in the operand layout (see
//     coarse_b_store).  The epilogue adds the three FP32 partial products, so
//     the preconditioner stays the fixed linear map block-Jacobi + P Ahat P^T
//     with Ahat = bf16(A_c^{-1}) (symmetric: rounding is entrywise), which
//     keeps PCG's theory intact at any tolerance.
//
// Every wait on a copy or an MMA is bounded by the global timer; a wait that
// runs out sets a bit of the mesh's error word (read by the host after the
// solve), waits (bounded) for the copies it issued and frees its tensor memory.
// The cluster barriers are reached by every CTA of a cluster on every path.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace mfem {

namespace {

constexpr int kFuSplit = 4;                       // CTAs per cluster: parts of the K range
constexpr int kFuAggsCta = 5;                     // aggregates each CTA corrects
constexpr int kFuAggsBlk = kFuSplit * kFuAggsCta; // aggregates per cluster (row block)
constexpr int kFuStages = 4;                      // shared-memory ring of A + B chunks
constexpr int kFuThreads = 320;                   // 10 warps: one per 32 vertex rows of 5 x 64
constexpr int kTcM = 128;                         // MMA M: rows of A_c^{-1} per row block (6 x 20, padded)
constexpr int kTcProbs = kCoarseGroupSlots;       // request slots per CTA group
constexpr int kTcN = kCoarseBRows;                // MMA N: three BF16 parts per slot
constexpr int kTcSteps = kTcKC / 16;              // MMAs per chunk (K = 16 each)
constexpr int kFuStepA = kTcM * 16 * 2;           // bytes of A per K step (4 KB)
constexpr int kFuStepB = kTcN * 16 * 2;           // bytes of B per K step (1.5 KB)
constexpr int kFuChunkA = kFuStepA * kTcSteps;    // 32 KB
constexpr int kFuChunkB = kFuStepB * kTcSteps;    // 12 KB
constexpr int kFuStage = kFuChunkA + kFuChunkB;   // 44 KB
constexpr int kFuSmem = kFuStages * kFuStage + 128;
constexpr int kTcTmemCols = 64;                   // >= kTcN, a power of two >= 32
constexpr uint64_t kTcWaitNs = 200ull * 1000ull * 1000ull;   // 0.2 s per bounded wait

static_assert(6 * kFuAggsBlk <= kTcM, "a row block's coarse rows fit the MMA's M");
static_assert(kFuChunkB == kCoarseBChunk * 2, "B chunk layout shared with the restriction");
static_assert(kTcM * kTcN * 4 <= kFuStage, "the partial product fits one stage for the cluster sum");
static_assert(kFuChunkA % 16 == 0 && kFuChunkB % 16 == 0 && kFuStage % 1024 == 0, "bulk copies: 16-byte units");
static_assert(kFuThreads >= 128, "warps 0-3 read the 128 TMEM lanes");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier to complete, at most kTcWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kTcWaitNs) return false;
    return true;
}

// 1-D bulk copy global -> shared through the TMA engine; completes `bytes` of
// transaction count on the barrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a no-swizzle K-major operand: start
// address, byte offset between K-adjacent core matrices (leading) and between
// 8-row groups (stride), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lead, uint32_t stride) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lead >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((stride >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N and M as given.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Element (row, k) of a row block's chunk (bf16 elements): K step s, K-core j2,
// 8-row group g, row r in the group.
__host__ __device__ __forceinline__ size_t a_offset(int row, int kk) {
    const int s = kk >> 4, j2 = (kk >> 3) & 1, c = kk & 7, g = row >> 3, r = row & 7;
    return (size_t)s * (kTcM * 16) + (size_t)(g * 2 + j2) * 64 + r * 8 + c;
}

// Set-up: FP32 A_c^{-1} (rows of ld floats) -> per row block and chunk, BF16.
__global__ void k_coarse_pack_bf16(const float* __restrict__ Ainv, int N, int ld, int nkc,
                                   __nv_bfloat16* __restrict__ out) {
    const int kk = threadIdx.x;                        // column within the chunk
    const int r = blockIdx.y % kTcM, rb = blockIdx.y / kTcM;
    const int ch = blockIdx.z;
    const int row = rb * 6 * kFuAggsBlk + r, k = ch * kTcKC + kk;
    const float v = (r < 6 * kFuAggsBlk && row < N && k < N) ? Ainv[(size_t)row * ld + k] : 0.f;
    out[((size_t)rb * nkc + ch) * (kFuChunkA / 2) + a_offset(r, kk)] = __float2bfloat16_rn(v);
}

// mfem_coarse_apply: r_c of B problems (rows of ldr floats) -> their B operand.
__global__ void k_coarse_split(const float* __restrict__ rc, int N, int ldr, int nkc, uint16_t* __restrict__ bs) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (k >= N) return;
    coarse_b_store(bs + (size_t)(b / kCoarseGroupSlots) * nkc * kCoarseBChunk, b % kCoarseGroupSlots, k,
                   rc[(size_t)b * ldr + k]);
}

__device__ __forceinline__ void ldv(const float* p, float (&v)[3]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
}
__device__ __forceinline__ void ldv(const double* p, double (&v)[3]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
}
__device__ __forceinline__ void stv(float* p, const float (&v)[3]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], 0.f);
}
__device__ __forceinline__ void stv(double* p, const double (&v)[3]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], 0.0);
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// FP32 at the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ float ld_cluster_f32(const float* local, uint32_t rank) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_u32(local)), "r"(rank));
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(remote) : "memory");
    return v;
}

// Cluster (rb, pg): row block rb (aggregates kFuAggsBlk rb ..), request slots
// 16 pg .. 16 pg + 15 of the context; CTA q = cluster rank takes chunks
// [q c_per, (q + 1) c_per) of the K range and corrects aggregates
// kFuAggsBlk rb + kFuAggsCta q ...  The problems are found in the descriptor
// table d0 .. d0+nd-1 by slot; a slot without a two-level problem inside PCG
// contributes nothing (its B columns give outputs never read).
// e_out (mfem_coarse_apply): write e[slot][row] instead of the correction.
template <typename T>
__global__ void __launch_bounds__(kFuThreads, 1)
    k_coarse_fused(const __nv_bfloat16* __restrict__ Abf, int N, int nkc, const uint16_t* __restrict__ Bs,
                   const PcgDesc<T>* __restrict__ D, int d0, int nd, unsigned* __restrict__ err,
                   float* __restrict__ e_out) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kFuStages * kFuStage);   // chunk landed
    uint64_t* empty = full + kFuStages;                                           // its MMAs done
    uint64_t* done = empty + kFuStages;                                           // every MMA done
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    float* red = reinterpret_cast<float*>(smem);   // after the K loop: the partial product [kTcN][kTcM]
    __shared__ const PcgDesc<T>* dp[kTcProbs];
    __shared__ float es[6 * kFuAggsCta][kTcProbs + 1];
    __shared__ float qs[kFuAggsCta][kTcProbs][9];
    __shared__ int any, s_ok;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t q = cluster_rank();
    const int rb = blockIdx.x / kFuSplit, pg = blockIdx.y;
    const int c_per = (nkc + kFuSplit - 1) / kFuSplit;
    const int c_lo = min(nkc, (int)q * c_per), nch = min(nkc, c_lo + c_per) - c_lo;   // this CTA's chunks
    const int nst = nch < kFuStages ? nch : kFuStages;
    const unsigned char* gA =
        reinterpret_cast<const unsigned char*>(Abf) + ((size_t)rb * nkc + c_lo) * kFuChunkA;
    const unsigned char* gB =
        reinterpret_cast<const unsigned char*>(Bs) + ((size_t)pg * nkc + c_lo) * kFuChunkB;
    const int a_cta = kFuAggsBlk * rb + kFuAggsCta * (int)q;   // first aggregate this CTA corrects
    // prologue on data fixed during the solve, overlapping the previous kernel:
    // the slots' descriptors and aggregate rotations, and the first chunks of
    // A_c^{-1} (their barriers also expect the B chunk, copied after the wait)
    if (t < kTcProbs) {
        const int slot = pg * kTcProbs + t;
        const PcgDesc<T>* mine = nullptr;
#pragma unroll 8
        for (int i = 0; i < nd; ++i) {   // independent loads: no early exit
            const bool hit = D[d0 + i].bslot == slot && D[d0 + i].coarse;
            if (hit && !mine) mine = &D[d0 + i];
        }
        dp[t] = mine;
    }
    if (t == 0) {
        any = 0;
        s_ok = 1;
        for (int c = 0; c < 2 * kFuStages + 1; ++c) mbar_init(&full[c], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int c = 0; c < nst; ++c) {
            mbar_expect_tx(&full[c], kFuStage);
            bulk_g2s(smem + c * kFuStage, gA + (size_t)c * kFuChunkA, kFuChunkA, &full[c]);
        }
    }
    __syncthreads();
    for (int i = t; i < kFuAggsCta * kTcProbs * 9; i += kFuThreads) {
        const int ai = i / (kTcProbs * 9), p = (i / 9) % kTcProbs, e = i % 9;
        const PcgDesc<T>* d = dp[p];
        const int a = a_cta + ai;
        qs[ai][p][e] = (d && d->aggq && a < N / 6) ? d->aggq[9 * a + e] : 0.f;
    }
    pdl_wait();
    pdl_trigger();
    if (t == 0)   // B chunks of the first stages: written by the previous kernel
        for (int c = 0; c < nst; ++c)
            bulk_g2s(smem + c * kFuStage + kFuChunkA, gB + (size_t)c * kFuChunkB, kFuChunkB, &full[c]);
    __syncthreads();
    if (t < kTcProbs) {
        const PcgDesc<T>* d = dp[t];
        if (d && d->sc->state != kActive) d = nullptr;
        dp[t] = d;
        if (d) atomicOr(&any, 1);
    }
    __syncthreads();
    // the same for every CTA of the cluster (same slots, states final after the wait)
    if (!any) {   // nothing to compute; let the copies land before the memory is released
        if (t == 0)
            for (int c = 0; c < nst; ++c)
                if (!mbar_wait(&full[c], 0)) atomicOr(err, 4u);
        return;
    }
    if (warp == 0) {   // tensor memory for the 128 x 48 FP32 accumulator
        __syncwarp();
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (t == 0) {   // one thread issues every MMA and keeps the ring full
        constexpr uint32_t idesc = umma_idesc_bf16(kTcM, kTcN);
        const uint32_t base = smem_u32(smem);
        bool ok = true;
        int issued = nst;   // chunks whose copies were issued
        for (int c = 0; c < nch && ok; ++c) {
            const int s = c % kFuStages;
            ok = mbar_wait(&full[s], (uint32_t)(c / kFuStages) & 1u);
            if (!ok) break;
            tc_fence_after();
            const uint32_t a0 = base + s * kFuStage, b0 = a0 + kFuChunkA;
            for (int k = 0; k < kTcSteps; ++k)
                umma_bf16(tmem, umma_desc(a0 + k * kFuStepA, 128, 256), umma_desc(b0 + k * kFuStepB, 128, 256), idesc,
                          (c > 0 || k > 0) ? 1u : 0u);
            umma_commit(&empty[s]);
            // refill the stage of the previous chunk (its MMAs were issued one
            // chunk ago) with the chunk kFuStages after it
            const int cp = c - 1, cn = cp + kFuStages;
            if (cp >= 0 && cn < nch) {
                const int sp = cp % kFuStages;
                ok = mbar_wait(&empty[sp], (uint32_t)(cp / kFuStages) & 1u);
                if (!ok) break;
                mbar_expect_tx(&full[sp], kFuStage);
                bulk_g2s(smem + sp * kFuStage, gA + (size_t)cn * kFuChunkA, kFuChunkA, &full[sp]);
                bulk_g2s(smem + sp * kFuStage + kFuChunkA, gB + (size_t)cn * kFuChunkB, kFuChunkB, &full[sp]);
                issued = cn + 1;
            }
        }
        // arrives once every MMA issued above has completed (at once if none was)
        umma_commit(done);
        if (!ok) {
            s_ok = 0;
            atomicOr(err, 1u);
            // the copies in flight: the last use of each stage that was issued, bounded
            for (int c = issued - nst; c < issued; ++c)
                if (c >= 0) mbar_wait(&full[c % kFuStages], (uint32_t)(c / kFuStages) & 1u);
        }
    }
    const bool fin = mbar_wait(done, 0);
    tc_fence_after();
    const int all_done = __syncthreads_and(fin ? 1 : 0);
    if (!all_done && t == 0) {
        atomicOr(err, 2u);
        mbar_wait(done, 0);   // once more, bounded, before the memory is reused
    }
    // this CTA's partial product -> shared memory, column-major [kTcN][kTcM]
    // (no MMA ran for a CTA without chunks: its part is zero)
    if (warp < kTcM / 32) {
        const int row = warp * 32 + lane;
        if (nch > 0 && all_done && s_ok) {
            const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
            float v[16];
#pragma unroll
            for (int part = 0; part < 3; ++part) {
                tmem_ld16(lane_addr + part * kTcProbs, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int p = 0; p < kTcProbs; ++p) red[(part * kTcProbs + p) * kTcM + row] = v[p];
            }
        } else {
#pragma unroll
            for (int c = 0; c < kTcN; ++c) red[c * kTcM + row] = 0.f;
        }
    }
    tc_fence_before();
    cluster_sync();   // every CTA's part visible to the cluster
    // the rows of this CTA's aggregates: the cluster's parts added in rank order
    for (int i = t; i < 6 * kFuAggsCta * kTcProbs; i += kFuThreads) {
        const int r = i % (6 * kFuAggsCta), p = i / (6 * kFuAggsCta);
        const int row = 6 * kFuAggsCta * (int)q + r;
        float e = 0.f;
#pragma unroll
        for (uint32_t j = 0; j < (uint32_t)kFuSplit; ++j) {
            const float hi = ld_cluster_f32(red + p * kTcM + row, j);
            const float mid = ld_cluster_f32(red + (kTcProbs + p) * kTcM + row, j);
            const float lo = ld_cluster_f32(red + (2 * kTcProbs + p) * kTcM + row, j);
            e += (hi + mid) + lo;
        }
        es[r][p] = e;
    }
    cluster_sync();   // no CTA leaves or reuses its part while another reads it
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols)
                     : "memory");
    if (e_out) {   // the product alone
        for (int i = t; i < 6 * kFuAggsCta * kTcProbs; i += kFuThreads) {
            const int r = i % (6 * kFuAggsCta), p = i / (6 * kFuAggsCta), row = 6 * a_cta + r;
            if (dp[p] && row < N) e_out[(size_t)(pg * kTcProbs + p) * N + row] = es[r][p];
        }
        return;
    }
    // correction of the aggregates' vertex rows for every problem of the group
    const PcgDesc<T>* d0p = nullptr;
    for (int p = 0; p < kTcProbs && !d0p; ++p) d0p = dp[p];
    const int shift = d0p->agg_shift, n = d0p->n_rows, n_agg = N / 6;
    const int row0 = a_cta << shift;
    const int row1 = min(n, min(n_agg, a_cta + kFuAggsCta) << shift);
    const float4* crel = d0p->crel;
    for (int row = row0 + t; row < row1; row += kFuThreads) {
        const float4 off = crel[row];
        const int ai = (row >> shift) - a_cta;
        T z[kTcProbs][3];
#pragma unroll
        for (int p = 0; p < kTcProbs; ++p)
            if (dp[p]) ldv(rec_field(dp[p]->rec, npad32(n), kRecZB, row), z[p]);
#pragma unroll
        for (int p = 0; p < kTcProbs; ++p) {
            const PcgDesc<T>* d = dp[p];
            if (!d) continue;
            if (off.w != 0.f) {
                const float e0 = es[6 * ai][p], e1 = es[6 * ai + 1][p], e2 = es[6 * ai + 2][p];
                const float e3 = es[6 * ai + 3][p], e4 = es[6 * ai + 4][p], e5 = es[6 * ai + 5][p];
                const float l0 = e0 + (e4 * off.z - e5 * off.y);
                const float l1 = e1 + (e5 * off.x - e3 * off.z);
                const float l2 = e2 + (e3 * off.y - e4 * off.x);
                const float* Q = qs[ai][p];
#pragma unroll
                for (int i = 0; i < 3; ++i) z[p][i] += (T)(Q[3 * i] * l0 + Q[3 * i + 1] * l1 + Q[3 * i + 2] * l2);
            }
            stv(d->nb + 4 * (size_t)row, z[p]);
        }
    }
}

// Row blocks of an N x N inverse (clusters along the mesh's aggregates)
__host__ __device__ __forceinline__ int row_blocks(int N) { return (N / 6 + kFuAggsBlk - 1) / kFuAggsBlk; }

}  // namespace

size_t coarse_tc_bytes(int N) { return (size_t)row_blocks(N) * coarse_chunks(N) * (size_t)kFuChunkA; }

size_t coarse_b_bytes(int N, int slots) {
    const size_t groups = ((size_t)slots + kCoarseGroupSlots - 1) / kCoarseGroupSlots;
    return groups * coarse_chunks(N) * (size_t)kFuChunkB;
}

cudaError_t coarse_tc_pack(const float* Ainv, int N, void* Abf, cudaStream_t s) {
    k_coarse_pack_bf16<<<dim3(1, row_blocks(N) * kTcM, coarse_chunks(N)), kTcKC, 0, s>>>(
        Ainv, N, coarse_ld(N), coarse_chunks(N), static_cast<__nv_bfloat16*>(Abf));
    return cudaGetLastError();
}

cudaError_t coarse_split(const float* rc, int N, int ldr, int B, void* Bs, cudaStream_t s) {
    k_coarse_split<<<dim3((N + 255) / 256, B), 256, 0, s>>>(rc, N, ldr, coarse_chunks(N), static_cast<uint16_t*>(Bs));
    return cudaGetLastError();
}

cudaError_t coarse_tc_init() {
    cudaError_t e = cudaFuncSetAttribute(k_coarse_fused<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFuSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_coarse_fused<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFuSmem);
    return e;
}

template <typename T>
cudaError_t launch_coarse_fused(const cudaLaunchConfig_t& base, const CoarseJob& j, const PcgDesc<T>* descs,
                                float* e_out) {
    cudaLaunchConfig_t cfg = base;
    cudaLaunchAttribute attr[2];
    int na = 0;
    for (unsigned i = 0; i < base.numAttrs && na < 1; ++i) attr[na++] = base.attrs[i];   // programmatic launch
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = kFuSplit;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
    cfg.attrs = attr;
    cfg.numAttrs = na;
    cfg.gridDim = dim3(kFuSplit * row_blocks(j.N), (j.slots + kCoarseGroupSlots - 1) / kCoarseGroupSlots);
    cfg.blockDim = dim3(kFuThreads);
    cfg.dynamicSmemBytes = kFuSmem;
    return cudaLaunchKernelEx(&cfg, k_coarse_fused<T>, static_cast<const __nv_bfloat16*>(j.Abf), j.N,
                              coarse_chunks(j.N), static_cast<const uint16_t*>(j.Bs), descs, j.d0, j.nd, j.err, e_out);
}

template cudaError_t launch_coarse_fused<float>(const cudaLaunchConfig_t&, const CoarseJob&, const PcgDesc<float>*,
                                                float*);
template cudaError_t launch_coarse_fused<double>(const cudaLaunchConfig_t&, const CoarseJob&, const PcgDesc<double>*,
                                                 float*);

}  // namespace mfem
