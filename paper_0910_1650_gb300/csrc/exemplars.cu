// ap_exemplars: the outputs of Algorithm 1 (Section 2) from final messages.
//   E      = {k : argmax_j a(k,j)+r(k,j) == k}          (lowest index on ties)
//   idx(i) = i for i in E, else argmax_{k in E} s(i,k)  (lowest index on ties)
//   dpsim  = sum_{i not in E} s(i, idx(i)),  expref = sum_{k in E} s(k,k),
//   netsim = dpsim + expref                             (float64, fixed order)
#include <algorithm>
#include <climits>
#include <mutex>

#include "common.cuh"

namespace apgb {

// One warp per row: flag[i] = (argmax_k a(i,k)+r(i,k) == i).
__global__ void exemplar_flags_kernel(const float* __restrict__ R, const float* __restrict__ A,
                                      int n, int64_t ld, int32_t* flag) {
    const int warps = blockDim.x >> 5;
    const int lid = threadIdx.x & 31;
    for (int i = blockIdx.x * warps + (threadIdx.x >> 5); i < n; i += gridDim.x * warps) {
        const float* r = R + (int64_t)i * ld;
        const float* a = A + (int64_t)i * ld;
        float v = -INFINITY;
        int j = INT_MAX;
        const int n4 = n / 4;
        for (int f = lid; f < n4; f += 32) {
            const float4 r4 = reinterpret_cast<const float4*>(r)[f];
            const float4 a4 = reinterpret_cast<const float4*>(a)[f];
            argmax_merge(v, j, a4.x + r4.x, 4 * f);
            argmax_merge(v, j, a4.y + r4.y, 4 * f + 1);
            argmax_merge(v, j, a4.z + r4.z, 4 * f + 2);
            argmax_merge(v, j, a4.w + r4.w, 4 * f + 3);
        }
        for (int k = 4 * n4 + lid; k < n; k += 32) argmax_merge(v, j, a[k] + r[k], k);
        argmax_warp(v, j);
        if (lid == 0) flag[i] = (j == i) ? 1 : 0;
    }
}

// Single block: ordered list of exemplars (ascending index) and its length.
__global__ void compact_kernel(const int32_t* __restrict__ flag, int n, int32_t* list,
                               int32_t* count) {
    __shared__ int32_t warp_sum[32];
    __shared__ int32_t base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int lid = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    for (int lo = 0; lo < n; lo += blockDim.x) {
        const int i = lo + threadIdx.x;
        const int f = (i < n) ? flag[i] : 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        const int before_in_warp = __popc(bal & ((1u << lid) - 1u));
        if (lid == 0) warp_sum[wid] = __popc(bal);
        __syncthreads();
        int before = 0;
        for (int w = 0; w < wid; ++w) before += warp_sum[w];
        if (f) list[base + before + before_in_warp] = i;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < nw; ++w) tot += warp_sum[w];
            base += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base;
}

// One warp per row: label and the row's float64 contributions.
__global__ void assign_kernel(const float* __restrict__ S, int n, int64_t ld,
                              const int32_t* __restrict__ flag, const int32_t* __restrict__ list,
                              const int32_t* __restrict__ count, int32_t* idx, double* dp,
                              double* ep) {
    const int warps = blockDim.x >> 5;
    const int lid = threadIdx.x & 31;
    const int ne = *count;
    for (int i = blockIdx.x * warps + (threadIdx.x >> 5); i < n; i += gridDim.x * warps) {
        const float* s = S + (int64_t)i * ld;
        if (ne == 0) {
            if (lid == 0) { idx[i] = -1; dp[i] = 0.0; ep[i] = 0.0; }
            continue;
        }
        if (flag[i]) {
            if (lid == 0) { idx[i] = i; dp[i] = 0.0; ep[i] = (double)s[i]; }
            continue;
        }
        float v = -INFINITY;
        int j = INT_MAX;
        for (int e = lid; e < ne; e += 32) {
            const int k = list[e];
            argmax_merge(v, j, s[k], k);
        }
        argmax_warp(v, j);
        if (lid == 0) { idx[i] = j; dp[i] = (double)v; ep[i] = 0.0; }
    }
}

// Single block, fixed order: thread t sums a contiguous stripe, then a tree.
__global__ void sum2_kernel(const double* __restrict__ a, const double* __restrict__ b, int n,
                            double* out) {
    __shared__ double sa[1024], sb[1024];
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(n, lo + per);
    double x = 0.0, y = 0.0;
    for (int i = lo; i < hi; ++i) { x += a[i]; y += b[i]; }
    sa[threadIdx.x] = x;
    sb[threadIdx.x] = y;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sa[threadIdx.x] += sa[threadIdx.x + w];
            sb[threadIdx.x] += sb[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = sa[0]; out[1] = sb[0]; }
}

struct ExWs {
    int32_t* flag;
    int32_t* list;
    int32_t* count;
    double* dp;
    double* ep;
    double* sums;
};

static size_t carve_ex(void* ws, int64_t n, ExWs* w) {
    Carver c(ws);
    w->flag = c.take<int32_t>(n);
    w->list = c.take<int32_t>(n);
    w->count = c.take<int32_t>(1);
    w->dp = c.take<double>(n);
    w->ep = c.take<double>(n);
    w->sums = c.take<double>(2);
    return c.used;
}

// Shared by ap_exemplars and the partition / landmark paths.
int32_t exemplars_impl(const float* S, const float* R, const float* A, int64_t n, int64_t ld,
                       int32_t* idx, ap_result* out, void* ws, size_t ws_bytes,
                       cudaStream_t s) {
    ExWs w;
    const size_t need = carve_ex(nullptr, n, &w);
    AP_TRY(check_ws(ws, ws_bytes, need));
    carve_ex(ws, n, &w);
    const int ni = (int)n;
    const int rows_per_block = 8;
    const int blocks = (int)std::min<int64_t>((n + rows_per_block - 1) / rows_per_block, 65535);
    exemplar_flags_kernel<<<blocks, 32 * rows_per_block, 0, s>>>(R, A, ni, ld, w.flag);
    compact_kernel<<<1, 1024, 0, s>>>(w.flag, ni, w.list, w.count);
    assign_kernel<<<blocks, 32 * rows_per_block, 0, s>>>(S, ni, ld, w.flag, w.list, w.count, idx,
                                                         w.dp, w.ep);
    sum2_kernel<<<1, 1024, 0, s>>>(w.dp, w.ep, ni, w.sums);
    note_launches(4);
    AP_TRY(last_error());
    double h[2];
    int32_t cnt = 0;
    AP_CUDA_TRY(cudaMemcpyAsync(h, w.sums, sizeof(h), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaMemcpyAsync(&cnt, w.count, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    const int32_t status = cnt > 0 ? AP_OK : AP_NO_EXEMPLARS;
    out->n_exemplars = cnt;
    out->status = status;
    if (cnt > 0) {
        out->dpsim = h[0];
        out->expref = h[1];
        out->netsim = h[0] + h[1];
    } else {
        out->dpsim = out->expref = out->netsim = NAN;
    }
    return status;
}

size_t exemplars_ws_bytes(int64_t n) {
    ExWs w;
    return carve_ex(nullptr, n, &w);
}

}  // namespace apgb

using namespace apgb;

APGB_API size_t ap_exemplars_workspace_size(int64_t n) {
    if (n < 1) return 0;
    return exemplars_ws_bytes(n);
}

APGB_API int32_t ap_exemplars(const float* S, const float* R, const float* A, int64_t n,
                              int64_t ld, int32_t* idx, ap_result* out, void* ws,
                              size_t ws_bytes, void* stream) {
    if (!S || !R || !A || !idx || !out) return AP_ERR_INVALID_ARG;
    if (n < 1 || n > INT_MAX / 2 || ld < n || (ld & 3) || !aligned16(R) || !aligned16(A))
        return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    const int32_t iters = out->iters, conv = out->converged;
    *out = ap_result{};
    out->iters = iters;
    out->converged = conv;
    return exemplars_impl(S, R, A, n, ld, idx, out, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------------------
// No-allocation variant: the workspace is a fixed array inside the library.
// ---------------------------------------------------------------------------
namespace apgb {

static __device__ __align__(256) unsigned char g_noalloc_scratch[AP_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64];

// Device address of the scratch array for the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
static int32_t noalloc_scratch(void** ptr) {
    int dev = 0;
    AP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return AP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return AP_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *ptr = g_noalloc_ptr[dev];
    return AP_OK;
}

}  // namespace apgb

APGB_API int32_t ap_exemplars_noalloc(const float* S, const float* R, const float* A,
                                      int64_t n, int64_t ld, int32_t* idx, ap_result* out,
                                      void* stream) {
    if (!S || !R || !A || !idx || !out) return AP_ERR_INVALID_ARG;
    if (n < 1 || ld < n || (ld & 3) || !aligned16(R) || !aligned16(A)) return AP_ERR_INVALID_ARG;
    if (n > AP_NOALLOC_MAX_N || exemplars_ws_bytes(n) > AP_NOALLOC_SCRATCH_BYTES)
        return AP_ERR_TOO_LARGE;
    AP_TRY(require_sm103());
    void* scratch = nullptr;
    AP_TRY(noalloc_scratch(&scratch));
    const int32_t iters = out->iters, conv = out->converged;
    *out = ap_result{};
    out->iters = iters;
    out->converged = conv;
    return exemplars_impl(S, R, A, n, ld, idx, out, scratch, AP_NOALLOC_SCRATCH_BYTES,
                          static_cast<cudaStream_t>(stream));
}
