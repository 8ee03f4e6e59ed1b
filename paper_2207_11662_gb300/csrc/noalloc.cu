// homln_accuracy_noalloc: accuracy of an estimated CC-node set against ground truth
// without any device allocation.
//
// Some callers cannot call cudaMalloc: code whose device memory is already
// reserved by another allocator (a framework's caching pool that owns the GPU),
// or a loop that must never enter the allocator. The handle-based entry points
// allocate (a handle owns its CSRs and scratch), so this entry point takes no
// handle and keeps its scratch in the static device array below instead.
//
// The array is sized for up to HOMLN_NOALLOC_MAX_NODES nodes: two membership
// bitmaps of 2^15 words each plus a few counters (about 256 KB). Every GPU that
// loads the library holds it until the process exits.
#include "common.cuh"
#include "devptr.h"

#include <mutex>

namespace homln {
namespace {

constexpr int32_t kWords = HOMLN_NOALLOC_MAX_NODES / 32;  // one bitmap
// layout in 64-bit words: [pred bitmap | truth bitmap | 3 counters + pad | 4 ratios | error word + pad]
constexpr size_t kBitmapU64 = (size_t)kWords / 2;
constexpr size_t kOffTruth = kBitmapU64;
constexpr size_t kOffCounts = 2 * kBitmapU64;
constexpr size_t kOffRatios = kOffCounts + 4;
constexpr size_t kOffErr = kOffRatios + 4;
constexpr size_t kScratchU64 = kOffErr + 4;

// In host code this name is only a host-side stand-in for the device array, not a
// device address: kernels get the address cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchU64];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Address of the array on the current device, looked up once per device with
// that device current.
void *scratch_address() {
    int dev = 0;
    HCUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) fail(HOMLN_ECUDA, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            fail(HOMLN_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        }
        g_addr[dev] = p;
    }
    return g_addr[dev];
}

// True for device memory of the current device, or managed memory.
bool on_current_device(const void *p) {
    int dev = 0;
    HCUDA(cudaGetDevice(&dev));
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return device_pointer_usable(at, dev);
}

}  // namespace
}  // namespace homln

using namespace homln;

extern "C" homln_status homln_accuracy_noalloc(int32_t n_nodes, const int32_t *pred, int32_t n_pred,
                                               const int32_t *truth, int32_t n_truth, void *stream,
                                               homln_accuracy_t *out) {
    try {
        if (!out) fail(HOMLN_EINVAL, "out is NULL");
        if (n_nodes < 1 || n_nodes > HOMLN_NOALLOC_MAX_NODES)
            fail(HOMLN_EINVAL, "n_nodes must be in [1, HOMLN_NOALLOC_MAX_NODES = 2^20]");
        if (n_pred < 0 || n_truth < 0) fail(HOMLN_EINVAL, "negative list length");
        if ((n_pred > 0 && (!pred || !on_current_device(pred))) ||
            (n_truth > 0 && (!truth || !on_current_device(truth))))
            fail(HOMLN_EINVAL, "pred and truth must be device memory of the current device");
        cudaStream_t s = (cudaStream_t)stream;
        unsigned long long *base = static_cast<unsigned long long *>(scratch_address());
        homln_accuracy_t r;
        int32_t err = 0;
        accuracy_counts_prealloc(n_nodes, pred, n_pred, truth, n_truth, reinterpret_cast<uint32_t *>(base),
                                 reinterpret_cast<uint32_t *>(base + kOffTruth), base + kOffCounts,
                                 reinterpret_cast<double *>(base + kOffRatios),
                                 reinterpret_cast<int32_t *>(base + kOffErr), &r, &err, s);
        if (err != DEV_OK) fail(HOMLN_EINVAL, "node id outside [0, n_nodes)");
        *out = r;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected internal error");
        return HOMLN_ECUDA;
    }
    set_error("");
    return HOMLN_OK;
}
