// Coarse solve of the two-level preconditioner on the tensor cores.
//
// e = A_c^{-1} r_c for every problem of one mesh inside a PCG iteration: a dense
// product of the per-mesh inverse coarse matrix (N x N, N = 6 rigid modes per
// aggregate) with up to 16 coarse residuals per CTA group.  It is the one dense
// contraction of the solve (the preconditioner's reduced space; the method
// itself has none, paper §5), and it is bound by streaming A_c^{-1}: the FP32
// CUDA-core version read 4 bytes of A_c^{-1} per 16 FMAs and was limited by
// instruction issue.  Here A_c^{-1} is stored once per mesh in BF16 (half the
// bytes) and multiplied by tcgen05 MMAs with FP32 accumulation in tensor
// memory:
//
//   * A_c^{-1} is pre-tiled at set-up into tiles of 128 rows x kCoarseKC
//     columns, each tile contiguous and already in the MMA's no-swizzle
//     K-major layout (8-row x 16-byte core matrices; per K = 16 step the
//     128 x 16 sub-tile is 4 KB, core matrices K-adjacent 128 B apart and
//     8-row groups 256 B apart).  One CTA takes one tile: four 16 KB 1-D bulk
//     copies (the TMA engine, one mbarrier each) land it in shared memory, so
//     the MMAs on the first quarter start while the rest arrives.
//   * r_c of each problem is split exactly into three BF16 parts
//     (r = hi + mid + lo: 3 x 8 significand bits hold the FP32 value), the B
//     operand has N = 48 columns (16 problems x 3 parts), and the epilogue adds
//     the three FP32 partial products.  The preconditioner therefore stays the
//     fixed linear map block-Jacobi + P Ahat P^T with Ahat = bf16(A_c^{-1})
//     (symmetric: rounding is entrywise), which keeps PCG's theory intact at
//     any tolerance.
//   * One thread issues the 16 MMAs (M = 128, N = 48, K = 16) of the tile and
//     commits them to an mbarrier; each warp then reads its 32 TMEM lanes
//     (rows) with tcgen05.ld and writes the slice partials ec[slice][row] that
//     the correction kernel adds in slice order, so results are deterministic.
//
// Every wait is bounded by the global timer; a wait that runs out sets a bit
// of the mesh's error word (read by the host after the solve), waits (bounded)
// for the copies it issued, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace mfem {

namespace {

constexpr int kTcM = 128;                       // rows of A_c^{-1} per tile (MMA M)
constexpr int kTcKS = kCoarseKC;                // columns per tile (K slice)
constexpr int kTcProbs = 16;                    // problems per CTA group
constexpr int kTcN = 3 * kTcProbs;              // MMA N: three BF16 parts per problem
constexpr int kTcSteps = kTcKS / 16;            // MMAs per tile (K = 16 each)
constexpr int kTcChunks = 4;                    // bulk copies per tile
constexpr int kTcStepA = kTcM * 16 * 2;         // bytes of A per K step (4 KB)
constexpr int kTcStepB = kTcN * 16 * 2;         // bytes of B per K step (1.5 KB)
constexpr int kTcABytes = kTcStepA * kTcSteps;  // 64 KB
constexpr int kTcBBytes = kTcStepB * kTcSteps;  // 24 KB
constexpr int kTcChunkBytes = kTcABytes / kTcChunks;
constexpr int kTcTmemCols = 64;                 // >= kTcN, a power of two >= 32
constexpr int kTcSmem = kTcABytes + kTcBBytes + 64;
constexpr uint64_t kTcWaitNs = 200ull * 1000ull * 1000ull;   // 0.2 s per bounded wait

static_assert(kTcKS % (16 * kTcChunks) == 0, "K slice must split into whole MMA steps per chunk");
static_assert(kTcChunkBytes % 16 == 0, "bulk copies move multiples of 16 bytes");
static_assert((kTcProbs & (kTcProbs - 1)) == 0 && (kTcProbs * kTcKS / 8) % 128 == 0,
              "B build: whole work items per thread, problem index in the low bits");

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

// Element (row, k) of a 128 x kTcKS tile in its K-major core-matrix layout
// (bf16 elements): K step s, K-core j2, 8-row group g, row r in the group.
__host__ __device__ __forceinline__ size_t tile_offset(int row, int kk) {
    const int s = kk >> 4, j2 = (kk >> 3) & 1, c = kk & 7, g = row >> 3, r = row & 7;
    return (size_t)s * (kTcM * 16) + (size_t)(g * 2 + j2) * 64 + r * 8 + c;
}

// Set-up: FP32 A_c^{-1} (rows of ld floats) -> tiles of BF16.
__global__ void k_coarse_pack_bf16(const float* __restrict__ Ainv, int N, int ld, int nks,
                                   __nv_bfloat16* __restrict__ out) {
    const int kk = blockIdx.x * blockDim.x + threadIdx.x;   // column within the slice
    const int row = blockIdx.y;                              // global row
    const int ks = blockIdx.z;
    if (kk >= kTcKS) return;
    const int mt = row / kTcM, r = row % kTcM, k = ks * kTcKS + kk;
    const float v = (row < N && k < N) ? Ainv[(size_t)row * ld + k] : 0.f;
    out[((size_t)mt * nks + ks) * (kTcM * kTcKS) + tile_offset(r, kk)] = __float2bfloat16_rn(v);
}

template <typename T>
__global__ void __launch_bounds__(128) k_coarse_tc(const __nv_bfloat16* __restrict__ Abf, int N, int nks,
                                                   const PcgDesc<T>* __restrict__ D, int d0, int nd,
                                                   unsigned* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;
    unsigned char* sB = smem + kTcABytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kTcABytes + kTcBBytes);   // chunks, then MMA done
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + kTcChunks + 1);
    __shared__ const PcgDesc<T>* dp[kTcProbs];
    __shared__ const float* rcs[kTcProbs];
    __shared__ int any, s_ok;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int mt = blockIdx.x, ks = blockIdx.y, pg = blockIdx.z;
    // prologue on data fixed during the solve, overlapping the previous kernel:
    // the descriptors, and the tile of A_c^{-1} itself (four bulk copies, one
    // barrier each) -- it does not depend on the previous kernel
    const PcgDesc<T>* mine = nullptr;
    if (t < kTcProbs && pg * kTcProbs + t < nd && D[d0 + pg * kTcProbs + t].coarse) mine = &D[d0 + pg * kTcProbs + t];
    if (t == 0) {
        any = 0;
        s_ok = 1;
        for (int c = 0; c <= kTcChunks; ++c) mbar_init(&bars[c], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const unsigned char* gA =
            reinterpret_cast<const unsigned char*>(Abf + ((size_t)mt * nks + ks) * (size_t)(kTcM * kTcKS));
        for (int c = 0; c < kTcChunks; ++c) {
            mbar_expect_tx(&bars[c], kTcChunkBytes);
            bulk_g2s(sA + c * kTcChunkBytes, gA + (size_t)c * kTcChunkBytes, kTcChunkBytes, &bars[c]);
        }
    }
    pdl_wait();
    pdl_trigger();
    __syncthreads();
    if (t < kTcProbs) {
        const PcgDesc<T>* p = (mine && mine->sc->state == kActive) ? mine : nullptr;
        dp[t] = p;
        rcs[t] = p ? p->rc : nullptr;
        if (p) atomicOr(&any, 1);
    }
    __syncthreads();
    if (!any) {   // block-uniform: nothing to compute; let the prefetch land before the memory is released
        if (t == 0)
            for (int c = 0; c < kTcChunks; ++c) mbar_wait(&bars[c], 0);
        return;
    }
    if (warp == 0) {   // tensor memory for the 128 x 48 FP32 accumulator
        __syncwarp();
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // B operand: each problem's r_c slice as three BF16 parts (rows p, 16 + p,
    // 32 + p of the N = 48 operand), zero for absent problems and past N.  A
    // work item is 8 consecutive columns of one problem: two 16-byte loads, and
    // each part is one 16-byte row of a core matrix; the problem index varies
    // fastest over the threads, so a warp's stores fill consecutive rows.
    const int k0 = ks * kTcKS;
#pragma unroll
    for (int it = 0; it < (kTcProbs * kTcKS / 8) / 128; ++it) {
        const int item = t + 128 * it;
        const int p = item & (kTcProbs - 1), kk0 = 8 * (item / kTcProbs), k = k0 + kk0;
        const float* src = rcs[p];
        float v[8];
        if (src && k + 7 < N) {
            const float4 a = *reinterpret_cast<const float4*>(src + k);
            const float4 c = *reinterpret_cast<const float4*>(src + k + 4);
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = c.x; v[5] = c.y; v[6] = c.z; v[7] = c.w;
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = (src && k + e < N) ? src[k + e] : 0.f;
        }
        uint32_t hi[4], mid[4], lo[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            __nv_bfloat16 h[2], m[2], l[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float r = v[e + q];
                h[q] = __float2bfloat16_rn(r);
                const float r1 = r - __bfloat162float(h[q]);
                m[q] = __float2bfloat16_rn(r1);
                l[q] = __float2bfloat16_rn(r1 - __bfloat162float(m[q]));
            }
            hi[e / 2] = (uint32_t)__bfloat16_as_ushort(h[0]) | ((uint32_t)__bfloat16_as_ushort(h[1]) << 16);
            mid[e / 2] = (uint32_t)__bfloat16_as_ushort(m[0]) | ((uint32_t)__bfloat16_as_ushort(m[1]) << 16);
            lo[e / 2] = (uint32_t)__bfloat16_as_ushort(l[0]) | ((uint32_t)__bfloat16_as_ushort(l[1]) << 16);
        }
        unsigned char* step = sB + (kk0 >> 4) * kTcStepB + ((kk0 >> 3) & 1) * 128;
        const int n0 = p, n1 = kTcProbs + p, n2 = 2 * kTcProbs + p;
        *reinterpret_cast<uint4*>(step + (n0 >> 3) * 256 + (n0 & 7) * 16) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(step + (n1 >> 3) * 256 + (n1 & 7) * 16) = make_uint4(mid[0], mid[1], mid[2], mid[3]);
        *reinterpret_cast<uint4*>(step + (n2 >> 3) * 256 + (n2 & 7) * 16) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // B visible to the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (t == 0) {   // one thread issues every MMA of the tile
        constexpr uint32_t idesc = umma_idesc_bf16(kTcM, kTcN);
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
        bool ok = true;
        for (int c = 0; c < kTcChunks && ok; ++c) {
            ok = mbar_wait(&bars[c], 0);
            if (!ok) break;
            tc_fence_after();
            for (int s = c * (kTcSteps / kTcChunks); s < (c + 1) * (kTcSteps / kTcChunks); ++s)
                umma_bf16(tmem, umma_desc(a0 + s * kTcStepA, 128, 256), umma_desc(b0 + s * kTcStepB, 128, 256),
                          idesc, s > 0 ? 1u : 0u);
        }
        // arrives once every MMA issued above has completed (at once if none was)
        umma_commit(&bars[kTcChunks]);
        if (!ok) {
            s_ok = 0;
            atomicOr(err, 1u);
            for (int c = 0; c < kTcChunks; ++c) mbar_wait(&bars[c], 0);   // our copies in flight, bounded
        }
    }
    const bool done = mbar_wait(&bars[kTcChunks], 0);
    tc_fence_after();
    const int all_done = __syncthreads_and(done ? 1 : 0);
    if (all_done && s_ok) {
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        float hi[16], mid[16], lo[16];
        tmem_ld16(lane_addr, hi);
        tmem_ld16(lane_addr + kTcProbs, mid);
        tmem_ld16(lane_addr + 2 * kTcProbs, lo);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int row = mt * kTcM + warp * 32 + lane;
        if (row < N) {
#pragma unroll
            for (int p = 0; p < kTcProbs; ++p)
                if (dp[p]) dp[p]->ec[(size_t)ks * N + row] = (hi[p] + mid[p]) + lo[p];
        }
    } else if (!all_done) {
        if (t == 0) atomicOr(err, 2u);
        mbar_wait(&bars[kTcChunks], 0);   // once more, bounded, before the memory is released
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols)
                     : "memory");
}

}  // namespace

size_t coarse_tc_bytes(int N) {
    const size_t mt = ((size_t)N + kTcM - 1) / kTcM, nks = ((size_t)N + kTcKS - 1) / kTcKS;
    return mt * nks * (size_t)kTcM * kTcKS * sizeof(__nv_bfloat16);
}

cudaError_t coarse_tc_pack(const float* Ainv, int N, void* Abf, cudaStream_t s) {
    const int mt = (N + kTcM - 1) / kTcM, nks = (N + kTcKS - 1) / kTcKS;
    k_coarse_pack_bf16<<<dim3((kTcKS + 127) / 128, mt * kTcM, nks), 128, 0, s>>>(
        Ainv, N, coarse_ld(N), nks, static_cast<__nv_bfloat16*>(Abf));
    return cudaGetLastError();
}

cudaError_t coarse_tc_init() {
    cudaError_t e = cudaFuncSetAttribute(k_coarse_tc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_coarse_tc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    return e;
}

template <typename T>
cudaError_t launch_coarse_tc(const cudaLaunchConfig_t& base, const CoarseJob& j, const PcgDesc<T>* descs) {
    cudaLaunchConfig_t cfg = base;
    const int mt = (j.N + kTcM - 1) / kTcM, nks = (j.N + kTcKS - 1) / kTcKS;
    cfg.gridDim = dim3(mt, nks, (j.nd + kTcProbs - 1) / kTcProbs);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = kTcSmem;
    return cudaLaunchKernelEx(&cfg, k_coarse_tc<T>, static_cast<const __nv_bfloat16*>(j.Abf), j.N, nks, descs,
                              j.d0, j.nd, j.err);
}

template cudaError_t launch_coarse_tc<float>(const cudaLaunchConfig_t&, const CoarseJob&, const PcgDesc<float>*);
template cudaError_t launch_coarse_tc<double>(const cudaLaunchConfig_t&, const CoarseJob&, const PcgDesc<double>*);

}  // namespace mfem
