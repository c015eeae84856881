// Shared helpers of the CUDA library: status plumbing, workspace carving,
// warp reductions.  Nothing here is arithmetic of the method itself.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>
#include <climits>

#include "../../include/apgb.h"

#define APGB_API extern "C" __attribute__((visibility("default")))

#define AP_CUDA_TRY(expr)                                                     \
    do {                                                                      \
        cudaError_t _e = (expr);                                              \
        if (_e != cudaSuccess) return AP_ERR_CUDA;                            \
    } while (0)

#define AP_TRY(expr)                                                          \
    do {                                                                      \
        int32_t _s = (expr);                                                  \
        if (_s < 0) return _s;                                                \
    } while (0)

namespace apgb {

constexpr size_t kAlign = 256;

__host__ __device__ inline size_t align_up(size_t x, size_t a) {
    return (x + a - 1) / a * a;
}

// Bump allocator over the caller's workspace.  Sizing and carving share this
// code, so a *_workspace_size query and the call that uses it always agree.
struct Carver {
    char*  base;
    size_t used = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <class T>
    T* take(size_t count) {
        size_t off = align_up(used, kAlign);
        used = off + align_up(count * sizeof(T), kAlign);
        return base ? reinterpret_cast<T*>(base + off) : nullptr;
    }
};

inline bool aligned16(const void* p) {
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

inline int32_t check_ws(void* ws, size_t ws_bytes, size_t need) {
    if (need == 0) return AP_OK;
    if (ws == nullptr || ws_bytes < need ||
        (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) != 0)
        return AP_ERR_WORKSPACE;
    return AP_OK;
}

inline int32_t last_error() {
    return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

int32_t device_sm_count(int* sms);       // cached per device
void note_launches(uint64_t k);          // feeds ap_kernel_launches()
// Column means of X (n x d, leading dimension ldx) into mean[d]: compensated
// float32 partials over row blocks, combined in float64 in a fixed order;
// part needs column_mean_part_doubles(n, d) doubles.
size_t column_mean_part_doubles(int64_t n, int d);
int32_t column_means(const float* X, int64_t n, int d, int64_t ldx, double* part, float* mean,
                     cudaStream_t s);
int32_t require_sm103();                 // AP_ERR_UNSUPPORTED on other GPUs

// ---- device helpers ------------------------------------------------------

// Counter-based generator: splitmix64 output number ``ctr`` (1-based) of
// ``seed`` (Steele, Lea & Flood 2014; Vigna's constants).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t ctr) {
    uint64_t z = seed + ctr * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double unit_from_u64(uint64_t v) {
    return (double)(v >> 11) * 0x1.0p-53;
}

// (value, index) arg-max with the lowest index winning ties.
__device__ __forceinline__ void argmax_merge(float& v, int& j, float v2, int j2) {
    if (v2 > v || (v2 == v && j2 < j)) { v = v2; j = j2; }
}

// Row top-2 of a sequence: m1 = max, j1 = lowest index attaining it,
// m2 = max over the other indices (== m1 on a tie).
struct Top2 {
    float m1, m2;
    int   j1;
};

__device__ __forceinline__ void top2_push(Top2& t, float v, int j) {
    if (v > t.m1 || (v == t.m1 && j < t.j1)) {
        t.m2 = t.m1;
        t.m1 = v;
        t.j1 = j;
    } else if (v > t.m2) {
        t.m2 = v;
    }
}

__device__ __forceinline__ Top2 top2_merge(Top2 a, Top2 b) {
    Top2 r;
    if (a.m1 > b.m1 || (a.m1 == b.m1 && a.j1 < b.j1)) {
        r.m1 = a.m1; r.j1 = a.j1; r.m2 = fmaxf(a.m2, b.m1);
    } else {
        r.m1 = b.m1; r.j1 = b.j1; r.m2 = fmaxf(b.m2, a.m1);
    }
    return r;
}

__device__ __forceinline__ Top2 top2_warp(Top2 t) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Top2 u;
        u.m1 = __shfl_xor_sync(0xffffffffu, t.m1, o);
        u.m2 = __shfl_xor_sync(0xffffffffu, t.m2, o);
        u.j1 = __shfl_xor_sync(0xffffffffu, t.j1, o);
        t = top2_merge(t, u);
    }
    return t;
}

__device__ __forceinline__ void argmax_warp(float& v, int& j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float v2 = __shfl_xor_sync(0xffffffffu, v, o);
        int   j2 = __shfl_xor_sync(0xffffffffu, j, o);
        argmax_merge(v, j, v2, j2);
    }
}

// The same reductions with one redux.sync per quantity (sm_100 family):
// m1 = warp max; j1 = lowest index among the lanes holding m1; m2 = max over
// lanes of (their m1, or their m2 for the lane holding j1), since the lanes'
// index sets are disjoint.  NaN inputs are ignored, as fmaxf does.
__device__ __forceinline__ float warp_max_f32(float x) {
    float r;
    asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ Top2 top2_warp_redux(Top2 t) {
    Top2 r;
    r.m1 = warp_max_f32(t.m1);
    r.j1 = __reduce_min_sync(0xffffffffu, t.m1 == r.m1 ? t.j1 : INT_MAX);
    r.m2 = warp_max_f32(t.j1 == r.j1 ? t.m2 : t.m1);
    return r;
}

__device__ __forceinline__ void argmax_warp_redux(float& v, int& j) {
    const float m = warp_max_f32(v);
    j = __reduce_min_sync(0xffffffffu, v == m ? j : INT_MAX);
    v = m;
}

}  // namespace apgb
