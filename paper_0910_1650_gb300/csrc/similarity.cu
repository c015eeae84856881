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
#include <mutex>
#include <map>
#include <array>
#include <climits>
#include <cmath>

#include <cuda_bf16.h>

#include <vector>

#include "common.cuh"

namespace apgb {

int32_t tc_similarity_bf16(const __nv_bfloat16* Xb, const float* nrm, int n, int dpad,
                           float* S, int64_t lds, int32_t* err, cudaStream_t s);
size_t tc_similarity_pad_rows();

// ---- 1. column means -----------------------------------------------------------
// Column sums of X in float64 over blocks of `rows` rows.  Block: 32
// columns x 8 row lanes; lane y sums rows y, y+8, ... of the row block, and
// the 8 lane sums are added in a fixed tree (deterministic).  Grid:
// (ceil(d/32), ceil(n/rows)).  part[row block][j].
constexpr int kMeanRows = 256;

__global__ void __launch_bounds__(256) colsum_partial_kernel(const float* __restrict__ X, int64_t n, int d,
                                                             int64_t ldx, int64_t rows, double* part) {
    const int cx = threadIdx.x & 31, ry = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + cx;
    const int64_t r0 = (int64_t)blockIdx.y * rows;
    const int64_t r1 = min(n, r0 + rows);
    __shared__ double ps[8][32];
    // Neumaier-compensated float32 sum of the lane's rows (float64 arithmetic is
    // scarce on this part); (s, c) carries the sum to well below float32 rounding
    float sm = 0.f, cm = 0.f;
    if (j < d) {
#pragma unroll 8
        for (int64_t i = r0 + ry; i < r1; i += 8) {
            const float x = X[i * ldx + j];
            const float t = sm + x;
            cm += (fabsf(sm) >= fabsf(x)) ? (sm - t) + x : (x - t) + sm;
            sm = t;
        }
    }
    ps[ry][cx] = (double)sm + (double)cm;
    __syncthreads();
    if (ry == 0 && j < d)
        part[(int64_t)blockIdx.y * d + j] = ((ps[0][cx] + ps[1][cx]) + (ps[2][cx] + ps[3][cx])) +
                                            ((ps[4][cx] + ps[5][cx]) + (ps[6][cx] + ps[7][cx]));
}

__global__ void colmean_kernel(const double* __restrict__ part, int nb, int d, int64_t n,
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
// Histogram of digit (key >> shift) & (2^bits - 1) over the off-diagonal keys
// that match each order statistic's known prefix.  While both statistics
// share their prefix (always in the first pass, usually later), one histogram
// serves both.  VEC: rows read as float4 (S 16-byte aligned, lds % 4 == 0).
template <bool VEC>
__global__ void __launch_bounds__(256) radix_hist_kernel(const float* __restrict__ S, int n,
                                                         int64_t lds, int shift, int bits,
                                                         const SelectState* __restrict__ st,
                                                         unsigned long long* hist) {
    __shared__ unsigned int h[2][2048];
    const int nb = 1 << bits;
    for (int b = threadIdx.x; b < 2 * 2048; b += blockDim.x) (&h[0][0])[b] = 0;
    __syncthreads();
    const uint32_t km = st->known_mask, p0 = st->prefix[0], p1 = st->prefix[1];
    const bool same = p0 == p1;
    const uint32_t dm = (uint32_t)nb - 1u;
    auto count = [&](float v) {
        const uint32_t key = float_key(v);
        const uint32_t dg = (key >> shift) & dm;
        if ((key & km) == p0) atomicAdd(&h[0][dg], 1u);
        if (!same && (key & km) == p1) atomicAdd(&h[1][dg], 1u);
    };
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const float* row = S + (int64_t)i * lds;
        if (VEC) {
            const float4* row4 = reinterpret_cast<const float4*>(row);
            const int n4 = (n + 3) >> 2;
            for (int k4 = threadIdx.x; k4 < n4; k4 += blockDim.x) {
                const float4 v = row4[k4];
                const int k = 4 * k4;
                if (k != i && k < n) count(v.x);
                if (k + 1 != i && k + 1 < n) count(v.y);
                if (k + 2 != i && k + 2 < n) count(v.z);
                if (k + 3 != i && k + 3 < n) count(v.w);
            }
        } else {
            for (int k = threadIdx.x; k < n; k += blockDim.x)
                if (k != i) count(row[k]);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const unsigned int c0 = h[0][b], c1 = same ? c0 : h[1][b];
        if (c0) atomicAdd(&hist[b], (unsigned long long)c0);
        if (c1) atomicAdd(&hist[2048 + b], (unsigned long long)c1);
    }
}

// For each order statistic: the bin holding its remaining rank (a block-wide
// exclusive scan of the counts; each of the 1024 threads owns 2 bins), then
// the prefix, rank and known-digit mask are advanced and the histograms
// cleared for the next pass.
__global__ void __launch_bounds__(1024) radix_scan_kernel(SelectState* st, unsigned long long* hist,
                                                          int shift, int bits) {
    const int nb = 1 << bits;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    __shared__ unsigned long long wsum[32];
    __shared__ int found[2];
    __shared__ unsigned long long rem[2];
    if (t < 2) {
        found[t] = nb - 1;          // kept only if the counts were inconsistent
        rem[t] = st->rank[t];
    }
    __syncthreads();
    for (int j = 0; j < 2; ++j) {
        const unsigned long long* h = hist + 2048 * j;
        const unsigned long long r = st->rank[j];
        const int b0 = 2 * t;
        const unsigned long long c0 = b0 < nb ? h[b0] : 0ull, c1 = b0 + 1 < nb ? h[b0 + 1] : 0ull;
        unsigned long long x = c0 + c1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long v = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            wsum[lane] = v;
        }
        __syncthreads();
        const unsigned long long base = (warp > 0 ? wsum[warp - 1] : 0ull) + x - (c0 + c1);
        if (r >= base && r < base + c0) {
            found[j] = b0;
            rem[j] = r - base;
        } else if (r >= base + c0 && r < base + c0 + c1) {
            found[j] = b0 + 1;
            rem[j] = r - base - c0;
        }
        __syncthreads();
    }
    if (t < 2) {
        st->prefix[t] |= (uint32_t)found[t] << shift;
        st->rank[t] = rem[t];
    }
    if (t == 0) st->known_mask |= (uint32_t)(nb - 1) << shift;
    for (int b = t; b < 2 * 2048; b += blockDim.x) hist[b] = 0;
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
// Row blocks of the column means: 256 rows, or more so that there are at most
// 2048 blocks (the float64 combine of the partials is sequential per column).
static int64_t mean_rows(int64_t n) { return std::max<int64_t>(kMeanRows, (n + 2047) / 2048); }
static int mean_blocks(int64_t n) { return (int)((n + mean_rows(n) - 1) / mean_rows(n)); }

size_t column_mean_part_doubles(int64_t n, int d) { return (size_t)mean_blocks(n) * (size_t)d; }

int32_t column_means(const float* X, int64_t n, int d, int64_t ldx, double* part, float* mean,
                     cudaStream_t s) {
    const int nb = mean_blocks(n);
    colsum_partial_kernel<<<dim3((d + 31) / 32, nb), 256, 0, s>>>(X, n, d, ldx, mean_rows(n), part);
    colmean_kernel<<<(d + 255) / 256, 256, 0, s>>>(part, nb, d, n, mean);
    note_launches(2);
    return last_error();
}

static size_t carve_sim(void* ws, int64_t n, int64_t d, SimWs* w) {
    Carver c(ws);
    const int npad = pad_rows((int)n), dpad = pad_dim((int)d);
    w->part = c.take<double>(column_mean_part_doubles(n, (int)d));
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
        if (aligned16(S) && (lds & 3) == 0)
            radix_hist_kernel<true><<<grid, 256, 0, s>>>(S, n, lds, shifts[p], bits[p], sel, hist);
        else
            radix_hist_kernel<false><<<grid, 256, 0, s>>>(S, n, lds, shifts[p], bits[p], sel, hist);
        radix_scan_kernel<<<1, 1024, 0, s>>>(sel, hist, shifts[p], bits[p]);
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

namespace apgb {

// Enqueues the whole similarity build of one problem on s (no synchronisation):
// means, centring (+ bf16 rounding), the Gram product with the distance
// epilogue, the preference and the optional noise.  pref_dev receives the
// median (AP_PREF_MEDIAN); err the tensor-core kernel's error flag.
static int32_t similarity_enqueue(const float* X, int ni, int di, int64_t ldx, float* S, int64_t lds,
                                  int32_t precision, int32_t pref_mode, const float* pref,
                                  double noise_rel, uint64_t seed, const SimWs& w, float* pref_dev,
                                  int32_t* err, cudaStream_t s) {
    const int npad = pad_rows(ni), dpad = pad_dim(di);
    AP_TRY(column_means(X, ni, di, ldx, w.part, w.mean, s));
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
        AP_TRY(tc_similarity_bf16(static_cast<const __nv_bfloat16*>(w.xc), w.nrm, ni, dpad, S, lds,
                                  err, s));
    }
    if (pref_mode == AP_PREF_MEDIAN) {
        AP_TRY(median_offdiag(S, ni, lds, w.sel, w.hist, pref_dev, s));
        diag_kernel<<<(ni + 255) / 256, 256, 0, s>>>(S, ni, lds, nullptr, pref_dev, 0.f);
    } else if (pref_mode == AP_PREF_SCALAR) {
        diag_kernel<<<(ni + 255) / 256, 256, 0, s>>>(S, ni, lds, nullptr, nullptr, pref[0]);
    } else {
        diag_kernel<<<(ni + 255) / 256, 256, 0, s>>>(S, ni, lds, pref, nullptr, 0.f);
    }
    if (noise_rel > 0.0) {
        noise_kernel<<<std::min(ni, 8192), 256, 0, s>>>(S, ni, lds, noise_rel, seed);
        note_launches(1);
    }
    note_launches(precision == AP_PREC_FP32 ? 3 : 2);   // centre, GEMM, diagonal
    return last_error();
}

static bool sim_args_ok(int32_t precision, int32_t pref_mode, const float* pref, double noise_rel) {
    if (precision != AP_PREC_FP32 && precision != AP_PREC_BF16) return false;
    if (pref_mode != AP_PREF_MEDIAN && pref_mode != AP_PREF_SCALAR && pref_mode != AP_PREF_VECTOR)
        return false;
    if (pref_mode != AP_PREF_MEDIAN && !pref) return false;
    return noise_rel >= 0.0 && std::isfinite(noise_rel);
}

}  // namespace apgb

APGB_API int32_t ap_similarity(const float* X, int64_t n, int64_t d, int64_t ldx, float* S,
                               int64_t lds, int32_t precision, int32_t pref_mode,
                               const float* pref, double noise_rel, uint64_t seed,
                               float* pref_out, void* ws, size_t ws_bytes, void* stream) {
    if (!X || !S || n < 2 || d < 1 || ldx < d || lds < n || n > INT_MAX / 2 || d > 65536)
        return AP_ERR_INVALID_ARG;
    if (!sim_args_ok(precision, pref_mode, pref, noise_rel)) return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SimWs w;
    AP_TRY(check_ws(ws, ws_bytes, carve_sim(nullptr, n, d, &w)));
    carve_sim(ws, n, d, &w);
    AP_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int32_t), s));
    AP_TRY(similarity_enqueue(X, (int)n, (int)d, ldx, S, lds, precision, pref_mode, pref, noise_rel,
                              seed, w, w.pref, w.err, s));
    float v = pref_mode == AP_PREF_SCALAR ? pref[0] : NAN;
    int32_t err = 0;
    if (pref_mode == AP_PREF_MEDIAN)
        AP_CUDA_TRY(cudaMemcpyAsync(&v, w.pref, sizeof(float), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaMemcpyAsync(&err, w.err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    if (err) return AP_ERR_TIMEOUT;
    if (pref_out) *pref_out = v;
    return AP_OK;
}

namespace apgb {

// Problems of a batch are spread round-robin over kSimStreams library-owned
// streams (created once per device), each with its own workspace slice: the
// small problems' latency-bound kernels then overlap.  They fork from and
// join back to the caller's stream through events.
constexpr int kSimStreams = 4;

static std::mutex g_sim_mu;
static std::map<int, std::array<cudaStream_t, kSimStreams>> g_sim_streams;

static int32_t sim_streams(std::array<cudaStream_t, kSimStreams>* out) {
    int dev = 0;
    AP_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_sim_mu);
    auto it = g_sim_streams.find(dev);
    if (it == g_sim_streams.end()) {
        std::array<cudaStream_t, kSimStreams> a{};
        for (auto& x : a) AP_CUDA_TRY(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
        it = g_sim_streams.emplace(dev, a).first;
    }
    *out = it->second;
    return AP_OK;
}

static size_t batched_slice(int64_t nmax, int64_t d) {
    SimWs w;
    return (carve_sim(nullptr, nmax, d, &w) + 255) / 256 * 256;
}

}  // namespace apgb

APGB_API size_t ap_similarity_batched_workspace_size(const int64_t* n, int32_t count, int64_t d) {
    if (!n || count < 1 || d < 1 || d > 65536) return 0;
    int64_t nmax = 0;
    for (int32_t b = 0; b < count; ++b) {
        if (n[b] < 2 || n[b] > INT_MAX / 2) return 0;
        nmax = std::max(nmax, n[b]);
    }
    Carver c(nullptr);
    c.take<unsigned char>(batched_slice(nmax, d) * kSimStreams);
    c.take<float>((size_t)count);
    return c.used;
}

APGB_API int32_t ap_similarity_batched(const float* X, const int64_t* xoff, const int64_t* n,
                                       int32_t count, int64_t d, int64_t ldx, float* S,
                                       const int64_t* soff, const int64_t* lds, int32_t precision,
                                       int32_t pref_mode, const float* pref, float* pref_out,
                                       void* ws, size_t ws_bytes, void* stream) {
    if (!X || !xoff || !n || !S || !soff || !lds || count < 1 || d < 1 || ldx < d || d > 65536)
        return AP_ERR_INVALID_ARG;
    if (pref_mode == AP_PREF_VECTOR || !sim_args_ok(precision, pref_mode, pref, 0.0))
        return AP_ERR_INVALID_ARG;
    int64_t nmax = 0;
    for (int32_t b = 0; b < count; ++b) {
        if (n[b] < 2 || n[b] > INT_MAX / 2 || lds[b] < n[b] || xoff[b] < 0 || soff[b] < 0)
            return AP_ERR_INVALID_ARG;
        nmax = std::max(nmax, n[b]);
    }
    AP_TRY(require_sm103());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    AP_TRY(check_ws(ws, ws_bytes, ap_similarity_batched_workspace_size(n, count, d)));
    std::array<cudaStream_t, kSimStreams> ss;
    AP_TRY(sim_streams(&ss));
    const size_t slice = batched_slice(nmax, d);
    Carver c(ws);
    unsigned char* base = c.take<unsigned char>(slice * kSimStreams);
    float* prefs = c.take<float>((size_t)count);
    SimWs w[kSimStreams];
    for (int k = 0; k < kSimStreams; ++k) {
        carve_sim(base + slice * k, nmax, d, &w[k]);
        AP_CUDA_TRY(cudaMemsetAsync(w[k].err, 0, sizeof(int32_t), s));
    }
    // fork: every worker stream starts after the caller's earlier work
    cudaEvent_t fork, join[kSimStreams];
    AP_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    for (auto& e : join) AP_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    struct Guard {
        cudaEvent_t f;
        cudaEvent_t* j;
        ~Guard() {
            cudaEventDestroy(f);
            for (int k = 0; k < kSimStreams; ++k) cudaEventDestroy(j[k]);
        }
    } guard{fork, join};
    AP_CUDA_TRY(cudaEventRecord(fork, s));
    for (int k = 0; k < kSimStreams; ++k) AP_CUDA_TRY(cudaStreamWaitEvent(ss[k], fork, 0));
    int32_t st = AP_OK;
    for (int32_t b = 0; b < count && st == AP_OK; ++b) {
        const int k = b % kSimStreams;
        st = similarity_enqueue(X + xoff[b], (int)n[b], (int)d, ldx, S + soff[b], lds[b], precision,
                                pref_mode, pref, 0.0, 0, w[k], prefs + b, w[k].err, ss[k]);
    }
    // join: the caller's stream continues after every worker (also on error)
    for (int k = 0; k < kSimStreams; ++k) {
        AP_CUDA_TRY(cudaEventRecord(join[k], ss[k]));
        AP_CUDA_TRY(cudaStreamWaitEvent(s, join[k], 0));
    }
    AP_TRY(st);
    std::vector<float> v(count, pref_mode == AP_PREF_SCALAR ? pref[0] : NAN);
    int32_t err[kSimStreams] = {0};
    if (pref_mode == AP_PREF_MEDIAN)
        AP_CUDA_TRY(cudaMemcpyAsync(v.data(), prefs, sizeof(float) * count, cudaMemcpyDeviceToHost, s));
    for (int k = 0; k < kSimStreams; ++k)
        AP_CUDA_TRY(cudaMemcpyAsync(&err[k], w[k].err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    for (int k = 0; k < kSimStreams; ++k)
        if (err[k]) return AP_ERR_TIMEOUT;
    if (pref_out)
        for (int32_t b = 0; b < count; ++b) pref_out[b] = v[b];
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
