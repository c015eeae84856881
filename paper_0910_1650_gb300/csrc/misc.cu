// Status strings, version, device checks.
#include <atomic>
#include <mutex>

#include "common.cuh"
#include "ptx.cuh"

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

// One CTA waits on a shared-memory mbarrier that nothing completes, with the
// same bounded try-wait loop every wait of the library uses; when the bound
// runs out it records the give-up and returns, with nothing in flight.
__global__ void wait_selftest_kernel(uint32_t limit, int32_t* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    const bool ok = ptx::mbar_wait(&bar, 0u, limit);
    if (threadIdx.x == 0) *status = ok ? AP_OK : AP_ERR_TIMEOUT;
}

}  // namespace apgb

using namespace apgb;

APGB_API int32_t ap_wait_selftest(uint32_t spin_limit, void* stream) {
    AP_TRY(require_sm103());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t* d = nullptr;
    AP_CUDA_TRY(cudaMallocAsync(&d, sizeof(int32_t), s));
    wait_selftest_kernel<<<1, 32, 0, s>>>(spin_limit, d);
    note_launches(1);
    int32_t h = AP_ERR_CUDA;
    const cudaError_t e1 = cudaGetLastError();
    const cudaError_t e2 = cudaMemcpyAsync(&h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    const cudaError_t e3 = cudaFreeAsync(d, s);
    const cudaError_t e4 = cudaStreamSynchronize(s);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess) return AP_ERR_CUDA;
    return h;
}

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
        case AP_ERR_CAPACITY: return "a result outgrew the capacity its workspace was sized for";
        default: return "unknown status";
    }
}

APGB_API int32_t ap_version(void) { return 100; }

APGB_API uint64_t ap_kernel_launches(void) {
    return apgb::g_launches.load(std::memory_order_relaxed);
}
