// Element outputs without any device allocation.
//
// mfem_get_elem stages the per-element results through a device buffer that it
// allocates and frees on every call, and cudaFree waits for the whole device.
// Callers that may allocate device memory only while they set up -- a per-frame
// animation loop or a host application's plugin running inside a fixed device
// budget -- cannot pay that.  mfem_get_elem_static runs the same kernel but
// stages through the fixed array below, so it calls no cudaMalloc, cudaFree or
// allocating library routine.
#include <cuda_runtime.h>

#include <mutex>

#include "engine.h"

namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kStaticElemMax = MFEM_ELEM_STATIC_MAX_TETS;

// 15 doubles per tet: s (6) then lambda (9) blocks.  Held by every GPU that
// loads the library until the process exits (7.5 MiB).
static __device__ __align__(256) double g_elem_scratch[15 * kStaticElemMax];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the array on the current device, looked up once per device
// (the host-side symbol is only a stand-in, not a device address).
mfem_status scratch_for_current_device(mfem_ctx* c, double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return mfem::cuda_check(c, e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return mfem::ctx_fail(c, MFEM_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_elem_scratch);
        if (e != cudaSuccess) return mfem::cuda_check(c, e, "cudaGetSymbolAddress(g_elem_scratch)");
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return MFEM_OK;
}

}  // namespace

extern "C" mfem_status mfem_get_elem_static(mfem_ctx* c, double* s, double* lam) {
    if (!c) return mfem::ctx_fail(nullptr, MFEM_EINVAL, "null context");
    const size_t m = (size_t)c->plan.m;
    if (m > kStaticElemMax) {
        char buf[160];
        snprintf(buf, sizeof buf, "mesh has %zu tets; mfem_get_elem_static handles at most %zu",
                 m, kStaticElemMax);
        return mfem::ctx_fail(c, MFEM_EINVAL, buf);
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device)
        return mfem::ctx_fail(c, MFEM_EINVAL, "the context's device must be current");
    if (!s && !lam) return MFEM_OK;
    double* scratch = nullptr;
    mfem_status st = scratch_for_current_device(c, &scratch);
    if (st != MFEM_OK) return st;
    // every entry the copies below read is written by the kernel: nothing to clear
    mfem::launch_elem_out(mfem::elem_args(c), 0, s ? scratch : nullptr, lam ? scratch + 6 * m : nullptr,
                          c->stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mfem::cuda_check(c, e, "element-output kernel launch");
    if (s) {
        e = cudaMemcpyAsync(s, scratch, sizeof(double) * 6 * m, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return mfem::cuda_check(c, e, "copy s");
    }
    if (lam) {
        e = cudaMemcpyAsync(lam, scratch + 6 * m, sizeof(double) * 9 * m, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return mfem::cuda_check(c, e, "copy lambda");
    }
    return mfem::cuda_check(c, cudaStreamSynchronize(c->stream), "get_elem_static");
}
