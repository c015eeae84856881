// ap_similarity: s(i,k) = -||x_i - x_k||^2 (Section 2) with the preferences
// p(k) on the diagonal (Algorithm 1 input) and the optional tie-break noise.
//
// Pipeline (all on the caller's stream, scratch in the caller's workspace):
//   1. column means of X in float64 (fixed-order two-stage reduction);
//   2. centred copy Xc = X - mean (float32, or bf16 for the tensor-core path),
//      zero padded to whole tiles, and squared norms of the centred rows
//      (of the bf16-rounded rows for the tensor-core path);
//   3. S = 2 Xc Xc^T - |x_i|^2 - |x_k|^2 clamped to <= 0 (SIMT float32 GEMM
//      here, tcgen05 GEMM in tc_gemm.cu);
//   4. preference: exact median of the n(n-1) off-diagonal values by a
//      three-pass radix select on order-preserving 32-bit keys (11/11/10
//      bits), both middle order statistics at once;
//   5. diagonal <- p, then s <- s + noise_rel*|s|*u(i,k) on every entry.
#include <algorithm>
#include <climits>
#include <cmath>

#include <cuda_bf16.h>

#include "common.cuh"

namespace apgb {

int32_t tc_similarity_bf16(const __nv_bfloat16* Xb, const float* nrm, int n, int dpad,
                           float* S, int64_t lds, int32_t* err, cudaStream_t s);
size_t tc_similarity_pad_rows();

// ---- 1. column means -----------------------------------------------------------
__global__ void colsum_partial_kernel(const float* __restrict__ X, int n, int d, int64_t ldx,
                                      int rows_per_block, double* part) {
    const int r0 = blockIdx.x * rows_per_block;
    const int r1 = min(n, r0 + rows_per_block);
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double s = 0.0;
        for (int i = r0; i < r1; ++i) s += (double)X[(int64_t)i * ldx + j];
        part[(int64_t)blockIdx.x * d + j] = s;
    }
}

__global__ void colmean_kernel(const double* __restrict__ part, int nb, int d, int n,
                               float* mean) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)b * d + j];
    mean[j] = (float)(s / (double)n);
}

// ---- 2. centring, norms -----------------------------------------------------------
// One warp per (padded) row.  Rows >= n and columns >= d are written as zero.
template <bool BF16>
__global__ void centre_kernel(const float* __restrict__ X, int n, int d, int64_t ldx,
                              const float* __restrict__ mean, int npad, int dpad, void* out,
                              float* nrm) {
    const int warps = blockDim.x >> 5, lid = threadIdx.x & 31;
    for (int i = blockIdx.x * warps + (threadIdx.x >> 5); i < npad; i += gridDim.x * warps) {
        float acc = 0.f;
        for (int j = lid; j < dpad; j += 32) {
            float v = 0.f;
            if (i < n && j < d) v = X[(int64_t)i * ldx + j] - mean[j];
            if (BF16) {
                const __nv_bfloat16 b = __float2bfloat16_rn(v);
                reinterpret_cast<__nv_bfloat16*>(out)[(int64_t)i * dpad + j] = b;
                v = __bfloat162float(b);
            } else {
                reinterpret_cast<float*>(out)[(int64_t)i * dpad + j] = v;
            }
            acc = fmaf(v, v, acc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lid == 0) nrm[i] = acc;
    }
}

// ---- 3. SIMT float32 GEMM with the distance epilogue ---------------------------
constexpr int GT = 128, GK = 8;

__global__ void __launch_bounds__(256) sim_gemm_fp32_kernel(const float* __restrict__ Xc, int n,
                                                            int dpad, const float* __restrict__ nrm,
                                                            float* __restrict__ S, int64_t lds,
                                                            int vec_ok) {
    __shared__ __align__(16) float As[GK][GT];
    __shared__ __align__(16) float Bs[GK][GT];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.y * GT, k0 = blockIdx.x * GT;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

    const int lr = tid >> 1, lc = (tid & 1) * 4;
    for (int kk = 0; kk < dpad; kk += GK) {
        const float4 va = *reinterpret_cast<const float4*>(Xc + (int64_t)(i0 + lr) * dpad + kk + lc);
        const float4 vb = *reinterpret_cast<const float4*>(Xc + (int64_t)(k0 + lr) * dpad + kk + lc);
        __syncthreads();
        As[lc + 0][lr] = va.x; As[lc + 1][lr] = va.y; As[lc + 2][lr] = va.z; As[lc + 3][lr] = va.w;
        Bs[lc + 0][lr] = vb.x; Bs[lc + 1][lr] = vb.y; Bs[lc + 2][lr] = vb.z; Bs[lc + 3][lr] = vb.w;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[k][ty * 8 + 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[k][tx * 8]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[k][tx * 8 + 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
        }
    }
    float nk[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) nk[b] = nrm[k0 + tx * 8 + b];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int i = i0 + ty * 8 + a;
        if (i >= n) continue;
        const float ni = nrm[i];
        float v[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int k = k0 + tx * 8 + b;
            v[b] = (k == i) ? 0.f : fminf(0.f, 2.f * acc[a][b] - ni - nk[b]);
        }
        float* row = S + (int64_t)i * lds + k0 + tx * 8;
        const int kb = k0 + tx * 8;
        if (kb + 8 <= n && vec_ok) {
            reinterpret_cast<float4*>(row)[0] = make_float4(v[0], v[1], v[2], v[3]);
            reinterpret_cast<float4*>(row)[1] = make_float4(v[4], v[5], v[6], v[7]);
        } else {
#pragma unroll
            for (int b = 0; b < 8; ++b)
                if (kb + b < n) row[b] = v[b];
        }
    }
}

// ---- 4. exact median by radix select -------------------------------------------
__device__ __forceinline__ uint32_t float_key(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
    const uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

struct SelectState {
    uint32_t prefix[2];
    uint32_t known_mask;
    int32_t  pad;
    uint64_t rank[2];
};

// Pass: histogram of the digit at `shift` among entries whose known high bits
// match each target's prefix.
__global__ void radix_hist_kernel(const float* __restrict__ S, int n, int64_t lds, int shift,
                                  int bits, const SelectState* __restrict__ st,
                                  unsigned long long* hist) {
    __shared__ unsigned int h[2][2048];
    const int nb = 1 << bits;
    for (int b = threadIdx.x; b < 2 * 2048; b += blockDim.x) (&h[0][0])[b] = 0;
    __syncthreads();
    const uint32_t km = st->known_mask, p0 = st->prefix[0], p1 = st->prefix[1];
    const uint32_t dm = (uint32_t)nb - 1u;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const float* row = S + (int64_t)i * lds;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            if (k == i) continue;
            const uint32_t key = float_key(row[k]);
            const uint32_t dg = (key >> shift) & dm;
            if ((key & km) == p0) atomicAdd(&h[0][dg], 1u);
            if ((key & km) == p1) atomicAdd(&h[1][dg], 1u);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        if (h[0][b]) atomicAdd(&hist[b], (unsigned long long)h[0][b]);
        if (h[1][b]) atomicAdd(&hist[2048 + b], (unsigned long long)h[1][b]);
    }
}

__global__ void radix_scan_kernel(SelectState* st, unsigned long long* hist, int shift, int bits) {
    if (threadIdx.x >= 2) return;
    const int j = threadIdx.x;
    const int nb = 1 << bits;
    unsigned long long* h = hist + 2048 * j;
    uint64_t r = st->rank[j];
    int b = 0;
    for (; b < nb; ++b) {
        if (r < h[b]) break;
        r -= h[b];
    }
    if (b >= nb) b = nb - 1;     // unreachable when the counts are consistent
    st->prefix[j] |= (uint32_t)b << shift;
    st->rank[j] = r;
    __syncwarp(0x3u);
    for (int x = j; x < nb; x += 2) { hist[x] = 0; hist[2048 + x] = 0; }
    __syncwarp(0x3u);
    if (j == 0) st->known_mask |= (uint32_t)(nb - 1) << shift;
}

__global__ void select_init_kernel(SelectState* st, unsigned long long* hist, uint64_t r0,
                                   uint64_t r1) {
    for (int x = threadIdx.x; x < 4096; x += blockDim.x) hist[x] = 0;
    if (threadIdx.x == 0) {
        st->prefix[0] = st->prefix[1] = 0;
        st->known_mask = 0;
        st->rank[0] = r0;
        st->rank[1] = r1;
    }
}

__global__ void select_finish_kernel(const SelectState* st, float* pref) {
    const double a = (double)key_float(st->prefix[0]);
    const double b = (double)key_float(st->prefix[1]);
    *pref = (float)(0.5 * (a + b));
}

// ---- 5. diagonal and tie-break noise -----------------------------------------------
// p(i) from a device vector, a device scalar or a by-value scalar (in that order).
__global__ void diag_kernel(float* S, int n, int64_t lds, const float* __restrict__ pvec,
                            const float* __restrict__ pdev, float pval) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) S[(int64_t)i * lds + i] = pvec ? pvec[i] : pdev ? *pdev : pval;
}

__global__ void noise_kernel(float* S, int n, int64_t lds, double rel, uint64_t seed) {
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        float* row = S + (int64_t)i * lds;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const double v = (double)row[k];
            const double u = unit_from_u64(splitmix64_at(seed, (uint64_t)i * n + k + 1));
            row[k] = (float)(v + rel * fabs(v) * u);
        }
    }
}

// ---- workspace ---------------------------------------------------------------------
struct SimWs {
    double* part;
    float* mean;
    void* xc;
    float* nrm;
    SelectState* sel;
    unsigned long long* hist;
    float* pref;
    int32_t* err;
};

static int pad_rows(int n) {
    const int t = (int)std::max<size_t>(GT, tc_similarity_pad_rows());
    return (n + t - 1) / t * t;
}
static int pad_dim(int d) { return (d + 63) / 64 * 64; }
static int mean_blocks(int n) { return (n + 1023) / 1024; }

static size_t carve_sim(void* ws, int64_t n, int64_t d, SimWs* w) {
    Carver c(ws);
    const int npad = pad_rows((int)n), dpad = pad_dim((int)d);
    w->part = c.take<double>((size_t)mean_blocks((int)n) * d);
    w->mean = c.take<float>(d);
    w->xc = c.take<float>((size_t)npad * dpad);   // large enough for either precision
    w->nrm = c.take<float>(npad);
    w->sel = c.take<SelectState>(1);
    w->hist = c.take<unsigned long long>(4096);
    w->pref = c.take<float>(1);
    w->err = c.take<int32_t>(1);
    return c.used;
}

int32_t median_offdiag(const float* S, int n, int64_t lds, SelectState* sel,
                       unsigned long long* hist, float* pref, cudaStream_t s) {
    const uint64_t m = (uint64_t)n * (uint64_t)(n - 1);
    select_init_kernel<<<1, 256, 0, s>>>(sel, hist, (m - 1) / 2, m / 2);
    const int grid = std::min(n, 4096);
    const int shifts[3] = {21, 10, 0}, bits[3] = {11, 11, 10};
    for (int p = 0; p < 3; ++p) {
        radix_hist_kernel<<<grid, 256, 0, s>>>(S, n, lds, shifts[p], bits[p], sel, hist);
        radix_scan_kernel<<<1, 32, 0, s>>>(sel, hist, shifts[p], bits[p]);
    }
    select_finish_kernel<<<1, 1, 0, s>>>(sel, pref);
    note_launches(8);
    return last_error();
}

}  // namespace apgb

using namespace apgb;

APGB_API size_t ap_similarity_workspace_size(int64_t n, int64_t d) {
    if (n < 2 || d < 1 || n > INT_MAX / 2 || d > 65536) return 0;
    SimWs w;
    return carve_sim(nullptr, n, d, &w);
}

APGB_API int32_t ap_similarity(const float* X, int64_t n, int64_t d, int64_t ldx, float* S,
                               int64_t lds, int32_t precision, int32_t pref_mode,
                               const float* pref, double noise_rel, uint64_t seed,
                               float* pref_out, void* ws, size_t ws_bytes, void* stream) {
    if (!X || !S || n < 2 || d < 1 || ldx < d || lds < n || n > INT_MAX / 2 || d > 65536)
        return AP_ERR_INVALID_ARG;
    if (precision != AP_PREC_FP32 && precision != AP_PREC_BF16) return AP_ERR_INVALID_ARG;
    if (pref_mode != AP_PREF_MEDIAN && pref_mode != AP_PREF_SCALAR && pref_mode != AP_PREF_VECTOR)
        return AP_ERR_INVALID_ARG;
    if (pref_mode != AP_PREF_MEDIAN && !pref) return AP_ERR_INVALID_ARG;
    if (!(noise_rel >= 0.0) || !std::isfinite(noise_rel)) return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SimWs w;
    AP_TRY(check_ws(ws, ws_bytes, carve_sim(nullptr, n, d, &w)));
    carve_sim(ws, n, d, &w);
    const int ni = (int)n, di = (int)d;
    const int npad = pad_rows(ni), dpad = pad_dim(di);

    const int nb = mean_blocks(ni);
    colsum_partial_kernel<<<nb, 256, 0, s>>>(X, ni, di, ldx, 1024, w.part);
    colmean_kernel<<<(di + 255) / 256, 256, 0, s>>>(w.part, nb, di, ni, w.mean);
    const int cgrid = std::min((npad + 7) / 8, 65535);
    if (precision == AP_PREC_FP32) {
        centre_kernel<false><<<cgrid, 256, 0, s>>>(X, ni, di, ldx, w.mean, npad, dpad, w.xc, w.nrm);
        dim3 grid((ni + GT - 1) / GT, (ni + GT - 1) / GT);
        const int vec_ok = aligned16(S) && (lds & 3) == 0;
        sim_gemm_fp32_kernel<<<grid, 256, 0, s>>>(static_cast<const float*>(w.xc), ni, dpad, w.nrm,
                                                  S, lds, vec_ok);
        AP_TRY(last_error());
    } else {
        centre_kernel<true><<<cgrid, 256, 0, s>>>(X, ni, di, ldx, w.mean, npad, dpad, w.xc, w.nrm);
        AP_TRY(last_error());
        AP_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int32_t), s));
        AP_TRY(tc_similarity_bf16(static_cast<const __nv_bfloat16*>(w.xc), w.nrm, ni, dpad, S, lds,
                                  w.err, s));
    }

    float used = NAN;
    if (pref_mode == AP_PREF_MEDIAN) {
        AP_TRY(median_offdiag(S, ni, lds, w.sel, w.hist, w.pref, s));
        diag_kernel<<<(ni + 255) / 256, 256, 0, s>>>(S, ni, lds, nullptr, w.pref, 0.f);
    } else if (pref_mode == AP_PREF_SCALAR) {
        used = pref[0];
        diag_kernel<<<(ni + 255) / 256, 256, 0, s>>>(S, ni, lds, nullptr, nullptr, used);
    } else {
        diag_kernel<<<(ni + 255) / 256, 256, 0, s>>>(S, ni, lds, pref, nullptr, 0.f);
    }
    if (noise_rel > 0.0) {
        noise_kernel<<<std::min(ni, 8192), 256, 0, s>>>(S, ni, lds, noise_rel, seed);
        note_launches(1);
    }
    note_launches(precision == AP_PREC_FP32 ? 5 : 3);   // means(2), centre, GEMM, diagonal
    AP_TRY(last_error());
    float v = used;
    int32_t err = 0;
    if (pref_mode == AP_PREF_MEDIAN)
        AP_CUDA_TRY(cudaMemcpyAsync(&v, w.pref, sizeof(float), cudaMemcpyDeviceToHost, s));
    if (precision == AP_PREC_BF16)
        AP_CUDA_TRY(cudaMemcpyAsync(&err, w.err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    if (err) return AP_ERR_TIMEOUT;
    if (pref_out) *pref_out = v;
    return AP_OK;
}

APGB_API size_t ap_preference_median_workspace_size(int64_t n) {
    if (n < 2) return 0;
    Carver c(nullptr);
    c.take<SelectState>(1);
    c.take<unsigned long long>(4096);
    c.take<float>(1);
    return c.used;
}

APGB_API int32_t ap_preference_median(const float* S, int64_t n, int64_t ld, float* median,
                                      void* ws, size_t ws_bytes, void* stream) {
    if (!S || !median || n < 2 || n > INT_MAX / 2 || ld < n) return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    AP_TRY(check_ws(ws, ws_bytes, ap_preference_median_workspace_size(n)));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c(ws);
    SelectState* sel = c.take<SelectState>(1);
    unsigned long long* hist = c.take<unsigned long long>(4096);
    float* pref = c.take<float>(1);
    AP_TRY(median_offdiag(S, (int)n, ld, sel, hist, pref, s));
    float v = NAN;
    AP_CUDA_TRY(cudaMemcpyAsync(&v, pref, sizeof(float), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    *median = v;
    return AP_OK;
}
