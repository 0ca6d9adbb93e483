// Allocation-free dose evaluation (lgk_fetch_doses_device).
//
// Some callers cannot allocate device memory while they run: their memory
// belongs to another framework's pool or a fixed arena, they run a real-time
// loop that cannot absorb an allocator's latency and implicit synchronisation,
// or they reserved the whole GPU up front.  For them this entry point takes
// device buffers for its input and output and keeps its one intermediate, the
// plans' sector times, in a static device array that exists for the lifetime
// of the process on every GPU that loads the library.
#include <mutex>
#include <string>

#include "lgk_impl.hpp"

struct lgk_result {
    std::unique_ptr<lgk::ResultData> d;
};

namespace lgk {

// Sector times of the plans being evaluated: K x 24N FP64 (row-major), at most
// LGK_NOALLOC_MAX_TIMES doubles (32 MiB).  Shared by every call: calls that
// overlap on the GPU race on it.
static __device__ __align__(256) double g_times_scratch[LGK_NOALLOC_MAX_TIMES];

constexpr int kMaxDevices = 64;
static double* g_scratch_addr[kMaxDevices] = {};
static std::mutex g_scratch_mu;

// Device address of the scratch array on the current device `dev`.  Host
// code only holds a stand-in for the symbol; the device address must come
// from the runtime.  The first call on a device looks it up (this may load
// the library's module on that device, so it must not happen during a stream
// capture).  Later calls look it up again whenever `st` is not capturing, so
// that an address cached before a device reset (which unloads the module and
// may place the array elsewhere when it is reloaded) is never used; during a
// capture they use the cached address.
static int scratch_address(int dev, cudaStream_t st, double** out) {
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal out of range for the static scratch table");
        return LGK_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusNone;
    }
    if (!g_scratch_addr[dev] || cap == cudaStreamCaptureStatusNone) {
        if (cap != cudaStreamCaptureStatusNone) {
            set_error("lgk_fetch_doses_device: the first call on a device must not be made during a "
                      "stream capture");
            return LGK_EINVAL;
        }
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_times_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
            return LGK_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return LGK_OK;
}

// Restores the caller's current device when the entry point returns.
struct DeviceGuard {
    int prev = -1;
    DeviceGuard() {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// True if p is device memory of device `dev` (or managed memory).
static bool on_device(const void* p, int dev) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace lgk

extern "C" int lgk_fetch_doses_device(const lgk_result* res, const double* phi_eval_dev, int n_eval,
                                      double* dose_dev) {
    using namespace lgk;
    if (!res || !phi_eval_dev || !dose_dev || n_eval < 1) {
        set_error("lgk_fetch_doses_device: NULL result/buffer or n_eval < 1");
        return LGK_EINVAL;
    }
    if (int rb = result_ready(*res->d)) return rb;
    const ResultData& r = *res->d;
    CaseData& cs = *r.cs;
    const long long need = (long long)r.K * cs.n_beams;
    if (need > LGK_NOALLOC_MAX_TIMES) {
        set_error("lgk_fetch_doses_device: K x 24N = " + std::to_string(need) +
                  " sector times exceed the static scratch of " +
                  std::to_string(LGK_NOALLOC_MAX_TIMES) + " doubles; split the plans");
        return LGK_EINVAL;
    }
    DeviceGuard keep_device;
    LGK_CUDA_TRY(cudaSetDevice(cs.device));
    if (!on_device(phi_eval_dev, cs.device) || !on_device(dose_dev, cs.device)) {
        set_error("lgk_fetch_doses_device: phi_eval_dev and dose_dev must be device memory of the "
                  "case's device");
        return LGK_EINVAL;
    }
    double* t = nullptr;
    int rc;
    if ((rc = scratch_address(cs.device, cs.stream, &t))) return rc;
    if ((rc = times_into(r, t))) return rc;
    // dose[K][E] = t[K][B] . phi_eval[E][B]^T, the kernel lgk_fetch_doses uses
    if ((rc = dgemm(cs.stream, false, true, r.K, n_eval, cs.n_beams, 1.0, t, cs.n_beams, phi_eval_dev,
                    cs.n_beams, 0.0, dose_dev, n_eval)))
        return rc;
    LGK_CUDA_TRY(cudaStreamSynchronize(cs.stream));
    return LGK_OK;
}
