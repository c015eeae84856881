// Status strings, version, device checks.
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace apgb {

static int g_sms[64];
static int g_cc[64];
static std::once_flag g_once[64];

static int32_t device_info(int* sms, int* cc) {
    int dev = 0;
    AP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return AP_ERR_CUDA;
    std::call_once(g_once[dev], [dev]() {
        cudaDeviceProp p;
        if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) {
            g_sms[dev] = p.multiProcessorCount;
            g_cc[dev] = p.major * 10 + p.minor;
        }
    });
    *sms = g_sms[dev];
    *cc = g_cc[dev];
    return *sms > 0 ? AP_OK : AP_ERR_CUDA;
}

static std::atomic<uint64_t> g_launches{0};
void note_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int32_t device_sm_count(int* sms) {
    int cc = 0;
    return device_info(sms, &cc);
}

int32_t require_sm103() {
    int sms = 0, cc = 0;
    AP_TRY(device_info(&sms, &cc));
    return cc == 103 ? AP_OK : AP_ERR_UNSUPPORTED;
}

}  // namespace apgb

APGB_API const char* ap_status_string(int32_t s) {
    switch (s) {
        case AP_OK: return "ok";
        case AP_NOT_CONVERGED: return "not converged (max_iter reached)";
        case AP_NO_EXEMPLARS: return "no exemplars";
        case AP_ERR_INVALID_ARG: return "invalid argument";
        case AP_ERR_CUDA: return "CUDA error";
        case AP_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case AP_ERR_TIMEOUT: return "device-side wait timed out";
        case AP_ERR_NONFINITE: return "non-finite similarity";
        case AP_ERR_UNSUPPORTED: return "unsupported device or configuration";
        case AP_ERR_TOO_LARGE: return "problem larger than the built-in scratch of a no-allocation entry";
        default: return "unknown status";
    }
}

APGB_API int32_t ap_version(void) { return 100; }

APGB_API uint64_t ap_kernel_launches(void) {
    return apgb::g_launches.load(std::memory_order_relaxed);
}
