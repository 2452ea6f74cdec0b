// quapi_readout_static: the rho readout of quapi_step_device without any
// device allocation.  The readout kernel needs a scratch buffer for its
// per-CTA partial sums; here that buffer is a fixed array in the library's
// own device memory instead of memory obtained from cudaMalloc.
//
// Scratch limit: kStaticCtas partial-sum slots of up to kSlotWidth complex
// doubles each (kStaticCtas * kSlotWidth * 16 bytes = 216 KiB per device that
// loads the library, held until the process exits).  The readout grid is
// capped at kStaticCtas CTAs (the kernel loops over its tiles, so any grid
// size gives the full sum); a context whose M*M exceeds kSlotWidth is
// rejected with QUAPI_ERR_ARG.
#include <mutex>

#include "quapi_internal.h"

namespace {

constexpr int kStaticCtas = 1536;  // >= 152 SMs x 8 resident CTAs of the readout kernel
constexpr int kSlotWidth = 9;      // M*M for M <= 3

__device__ __align__(256) double2 g_readout_scratch[kStaticCtas * kSlotWidth];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double2* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_readout_scratch on the current device.  In host code the
// symbol names a host-side stand-in, so the address has to be looked up once
// per device (with that device current) and then passed to the kernels.
cudaError_t scratch_for_current_device(double2** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_readout_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double2*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" quapi_status quapi_readout_static(const quapi_ctx* c, int64_t n, const void* A_in_dev, void* rho_dev) {
    using namespace quapi;
    if (!c) return record_error(nullptr, QUAPI_ERR_ARG, "NULL context");
    if (n < 1) return record_error(c, QUAPI_ERR_ARG, "n must be >= 1");
    if (!A_in_dev || !rho_dev) return record_error(c, QUAPI_ERR_ARG, "A_in and rho must not be NULL");
    if ((reinterpret_cast<uintptr_t>(A_in_dev) & 15u) || (reinterpret_cast<uintptr_t>(rho_dev) & 15u))
        return record_error(c, QUAPI_ERR_ARG, "device buffers must be 16-byte aligned");
    StepArgs a;
    int M = 0, form = 0;
    cudaStream_t st = nullptr;
    quapi_status s = readout_launch_args(c, n, A_in_dev, &a, &M, &form, &st);
    if (s != QUAPI_OK) return s;
    const int M2 = M * M;
    if (M2 > kSlotWidth)
        return record_error(c, QUAPI_ERR_ARG, "quapi_readout_static: M*M exceeds its 9 partial sums per CTA");
    // the array's address is looked up for the current device, and the kernels run on the context's
    // tables and stream: both must be the device the context was set up on
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record_error(c, QUAPI_ERR_CUDA, cudaGetErrorString(e));
    if (dev != ctx_device(c))
        return record_error(c, QUAPI_ERR_ARG,
                            "quapi_readout_static: the current CUDA device is not the one the context was set up on");
    double2* scratch = nullptr;
    e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return record_error(c, QUAPI_ERR_CUDA, cudaGetErrorString(e));
    // every launched CTA writes its own M2 slots, so nothing has to be cleared
    a.partial = scratch;
    a.grid = kStaticCtas;
    e = (a.half_digits >= 0) ? (M == 3 ? launch_herm3_step(form, a, st) : launch_herm_step(form, a, st))
                             : launch_step(M, form, a, st);
    if (e != cudaSuccess) return record_error(c, QUAPI_ERR_CUDA, cudaGetErrorString(e));
    e = launch_rho_reduce(scratch, a.grid, M2, static_cast<double2*>(rho_dev), st);
    if (e != cudaSuccess) return record_error(c, QUAPI_ERR_CUDA, cudaGetErrorString(e));
    return QUAPI_OK;
}
