// Allocation-free Hough back projection, for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside another framework's
// memory pool that owns the whole device, plugins that are handed only input and output
// buffers, or real-time loops where an allocation would stall or fail.  They cannot
// create a plan (fbp_plan allocates tables) or a workspace, so this entry point needs
// neither.  Its scratch -- the first-pass Hough buffer of one slice -- is a file-scope
// __device__ array of fixed size that every GPU loading the library holds until the
// process exits.
//
// In host code `g_scratch` names only a host-side shadow of the array, not a device
// address; the device address is obtained with cudaGetSymbolAddress once per device and
// handed to the kernels.  That set-up (and the kernels' shared-memory opt-in) happens on
// the first call on each device, with that device current, so the first call on a device
// should come before any stream capture.  With lazy module loading the driver may back the
// array with device memory only at that first lookup, so the first call on a device is the
// one that can fail for lack of memory (reported as FBP_ERR_OOM); later calls cannot.  Calls that overlap on the GPU share the array
// and race; issue them on one stream (or order them with events).
#include <mutex>

#include "fbp_internal.h"

namespace fbp {
cudaError_t prepare_fht_kernels();
}

namespace {

constexpr int kStaticMaxN = FBP_STATIC_MAX_N;
constexpr size_t kScratchFloats = (size_t)4 * kStaticMaxN * 2 * kStaticMaxN;   // one slice
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_scratch[kScratchFloats];

struct DeviceScratch {
    float* ptr = nullptr;
    bool ready = false;
};
DeviceScratch g_dev[kMaxDevices];
std::mutex g_lock;

// Device address of g_scratch on the current device (first call: look it up and opt the
// Hough kernels into their shared-memory sizes).
cudaError_t scratch_for_current_device(float** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> guard(g_lock);
    DeviceScratch& d = g_dev[dev];
    if (!d.ready) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        e = fbp::prepare_fht_kernels();
        if (e != cudaSuccess) return e;
        d.ptr = (float*)p;
        d.ready = true;
    }
    *out = d.ptr;
    return cudaSuccess;
}

}  // namespace

extern "C" fbp_status fbp_fht_backproject_static(int N, int count, const float* d_lin,
                                                 float* d_img, void* stream)
{
    if (N < 2 || N > kStaticMaxN || (N & (N - 1)) != 0) return FBP_ERR_UNSUPPORTED;
    if (count < 1 || !d_lin || !d_img) return FBP_ERR_INVALID_ARG;
    if (((uintptr_t)d_lin & 15u) || ((uintptr_t)d_img & 15u)) return FBP_ERR_MISALIGNED;
    float* scratch = nullptr;
    const cudaError_t se = scratch_for_current_device(&scratch);
    if (se != cudaSuccess) {
        cudaGetLastError();
        return se == cudaErrorMemoryAllocation ? FBP_ERR_OOM : FBP_ERR_CUDA;
    }
    // The launchers read only the sizes and the pass split from the plan record; a
    // zero-initialised record on the stack allocates nothing.
    fbp_plan_s shape{};
    shape.N = N;
    shape.n = 0;
    while ((1 << shape.n) < N) ++shape.n;
    shape.n1 = shape.n <= 6 ? shape.n : (shape.n + 1) / 2;
    shape.n2 = shape.n - shape.n1;
    const size_t lin = fbp::lin_floats(&shape), img = fbp::img_floats(&shape);
    cudaStream_t st = (cudaStream_t)stream;
    // One slice at a time through the shared scratch; the first pass writes every entry
    // that the second pass reads, so nothing has to be cleared between calls.
    for (int s = 0; s < count; ++s) {
        cudaError_t e = fbp::launch_pass1(&shape, d_lin + (size_t)s * lin, true, scratch, 1, st);
        if (e == cudaSuccess) e = fbp::launch_pass2(&shape, scratch, d_img + (size_t)s * img, 1, false, st);
        if (e == cudaSuccess) e = fbp::launch_pass2(&shape, scratch, d_img + (size_t)s * img, 1, true, st);
        if (e != cudaSuccess) return FBP_ERR_CUDA;
    }
    return FBP_OK;
}
