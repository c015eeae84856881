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
size_t tc_grouped_table_bytes(const int64_t* n, int32_t count);
int32_t tc_similarity_bf16_grouped(const __nv_bfloat16* Xb, const float* nrm, int64_t rows, int dpad,
                                   const int64_t* n, const int64_t* roff, float* const* S,
                                   const int64_t* lds, int32_t count, void* tables, int32_t* err,
                                   cudaStream_t s);
size_t tc_similarity_pad_rows();

// ---- 1. column means -----------------------------------------------------------
// Column sums of X in float64 over blocks of `rows` rows.  Block: 32
// columns x 8 row lanes; lane y sums rows y, y+8, ... of the row block, and
// the 8 lane sums are added in a fixed tree (deterministic).  Grid:
// (ceil(d/32), ceil(n/rows)).  part[row block][j].
constexpr int kMeanRows = 256;

// One block of the column sums: columns bx*32 .. bx*32+31, row block by.
__device__ __forceinline__ void colsum_block(const float* __restrict__ X, int64_t n, int d, int64_t ldx,
                                             int64_t rows, double* part, int bx, int by) {
    const int cx = threadIdx.x & 31, ry = threadIdx.x >> 5;
    const int j = bx * 32 + cx;
    const int64_t r0 = (int64_t)by * rows;
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
        part[(int64_t)by * d + j] = ((ps[0][cx] + ps[1][cx]) + (ps[2][cx] + ps[3][cx])) +
                                    ((ps[4][cx] + ps[5][cx]) + (ps[6][cx] + ps[7][cx]));
}

__global__ void __launch_bounds__(256) colsum_partial_kernel(const float* __restrict__ X, int64_t n, int d,
                                                             int64_t ldx, int64_t rows, double* part) {
    colsum_block(X, n, d, ldx, rows, part, blockIdx.x, blockIdx.y);
}

// The means from the row blocks' sums: columns bx*32 .. bx*32+31, in the
// layout of colsum_block (32 columns x 8 lanes; lane y adds blocks y, y+8,
// ... in order, then the 8 lane sums meet in the same fixed tree), so the
// float64 chain per thread is nb/8 long (float64 is scarce on this part).
__device__ __forceinline__ void colmean_block(const double* __restrict__ part, int nb, int d, int64_t n,
                                              float* mean, int bx) {
    const int cx = threadIdx.x & 31, ry = threadIdx.x >> 5;
    const int j = bx * 32 + cx;
    __shared__ double ps[8][32];
    double sm = 0.0;
    if (j < d)
        for (int b = ry; b < nb; b += 8) sm += part[(int64_t)b * d + j];
    ps[ry][cx] = sm;
    __syncthreads();
    if (ry == 0 && j < d)
        mean[j] = (float)((((ps[0][cx] + ps[1][cx]) + (ps[2][cx] + ps[3][cx])) +
                           ((ps[4][cx] + ps[5][cx]) + (ps[6][cx] + ps[7][cx]))) / (double)n);
}

// grid ceil(d/32), 256 threads
__global__ void __launch_bounds__(256) colmean_kernel(const double* __restrict__ part, int nb, int d,
                                                      int64_t n, float* mean) {
    colmean_block(part, nb, d, n, mean, blockIdx.x);
}

// ---- 2. centring, norms -----------------------------------------------------------
// One warp per (padded) row.  Rows >= n and columns >= d are written as zero.
// Block bx of a grid of gx blocks.
template <bool BF16>
__device__ __forceinline__ void centre_rows(const float* __restrict__ X, int n, int d, int64_t ldx,
                                            const float* __restrict__ mean, int npad, int dpad,
                                            void* out, float* nrm, int bx, int gx) {
    const int warps = blockDim.x >> 5, lid = threadIdx.x & 31;
    for (int i = bx * warps + (threadIdx.x >> 5); i < npad; i += gx * warps) {
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

// The same with four columns per lane and step (float4 loads, 8- or 16-byte
// stores); needs X 16-byte aligned with ldx % 4 == 0 (dpad % 64 == 0 holds).
// Each lane sums the squares of its own columns in order, then the warp adds
// the lane sums in a fixed butterfly, so the norms are deterministic.
template <bool BF16>
__device__ __forceinline__ void centre_rows4(const float* __restrict__ X, int n, int d, int64_t ldx,
                                             const float* __restrict__ mean, int npad, int dpad,
                                             void* out, float* nrm, int bx, int gx) {
    const int warps = blockDim.x >> 5, lid = threadIdx.x & 31;
    for (int i = bx * warps + (threadIdx.x >> 5); i < npad; i += gx * warps) {
        float acc = 0.f;
        for (int j = 4 * lid; j < dpad; j += 128) {
            float v[4];
            if (i < n && j + 3 < d) {
                const float4 x = *reinterpret_cast<const float4*>(X + (int64_t)i * ldx + j);
                const float4 m = *reinterpret_cast<const float4*>(mean + j);
                v[0] = x.x - m.x; v[1] = x.y - m.y; v[2] = x.z - m.z; v[3] = x.w - m.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    v[e] = (i < n && j + e < d) ? X[(int64_t)i * ldx + j + e] - mean[j + e] : 0.f;
            }
            if (BF16) {
                __nv_bfloat16 bv[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    bv[e] = __float2bfloat16_rn(v[e]);
                    v[e] = __bfloat162float(bv[e]);
                }
                uint2 pk;
                pk.x = (uint32_t)__bfloat16_as_ushort(bv[0]) | ((uint32_t)__bfloat16_as_ushort(bv[1]) << 16);
                pk.y = (uint32_t)__bfloat16_as_ushort(bv[2]) | ((uint32_t)__bfloat16_as_ushort(bv[3]) << 16);
                *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(out) + (int64_t)i * dpad + j) = pk;
            } else {
                *reinterpret_cast<float4*>(reinterpret_cast<float*>(out) + (int64_t)i * dpad + j) =
                    make_float4(v[0], v[1], v[2], v[3]);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) acc = fmaf(v[e], v[e], acc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lid == 0) nrm[i] = acc;
    }
}

template <bool BF16, bool VEC>
__global__ void centre_kernel(const float* __restrict__ X, int n, int d, int64_t ldx,
                              const float* __restrict__ mean, int npad, int dpad, void* out,
                              float* nrm) {
    if (VEC) centre_rows4<BF16>(X, n, d, ldx, mean, npad, dpad, out, nrm, blockIdx.x, gridDim.x);
    else centre_rows<BF16>(X, n, d, ldx, mean, npad, dpad, out, nrm, blockIdx.x, gridDim.x);
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
// Block bx of gx blocks (rows bx, bx + gx, ...).
template <bool VEC>
__device__ __forceinline__ void radix_hist_rows(const float* __restrict__ S, int n, int64_t lds,
                                                int shift, int bits, const SelectState* __restrict__ st,
                                                unsigned long long* hist, int bx, int gx) {
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
    for (int i = bx; i < n; i += gx) {
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

template <bool VEC>
__global__ void __launch_bounds__(256) radix_hist_kernel(const float* __restrict__ S, int n,
                                                         int64_t lds, int shift, int bits,
                                                         const SelectState* __restrict__ st,
                                                         unsigned long long* hist) {
    radix_hist_rows<VEC>(S, n, lds, shift, bits, st, hist, blockIdx.x, gridDim.x);
}

// For each order statistic: the bin holding its remaining rank (a block-wide
// exclusive scan of the counts; each of the 1024 threads owns 2 bins), then
// the prefix, rank and known-digit mask are advanced and the histograms
// cleared for the next pass.
__device__ __forceinline__ void radix_scan_block(SelectState* st, unsigned long long* hist,
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

__global__ void __launch_bounds__(1024) radix_scan_kernel(SelectState* st, unsigned long long* hist,
                                                          int shift, int bits) {
    radix_scan_block(st, hist, shift, bits);
}

// The two middle order statistics of the n(n-1) off-diagonal entries:
// ranks (m-1)/2 and m/2, m = n(n-1).
__device__ __forceinline__ void select_init_block(SelectState* st, unsigned long long* hist, int n) {
    const uint64_t m = (uint64_t)n * (uint64_t)(n - 1);
    for (int x = threadIdx.x; x < 4096; x += blockDim.x) hist[x] = 0;
    if (threadIdx.x == 0) {
        st->prefix[0] = st->prefix[1] = 0;
        st->known_mask = 0;
        st->rank[0] = (m - 1) / 2;
        st->rank[1] = m / 2;
    }
}

__global__ void select_init_kernel(SelectState* st, unsigned long long* hist, int n) {
    select_init_block(st, hist, n);
}

__device__ __forceinline__ float select_result(const SelectState* st) {
    const double a = (double)key_float(st->prefix[0]);
    const double b = (double)key_float(st->prefix[1]);
    return (float)(0.5 * (a + b));
}

__global__ void select_finish_kernel(const SelectState* st, float* pref) {
    *pref = select_result(st);
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
// Histogram blocks of the median: about 64K entries each (a block clears and
// flushes up to 4096 bins, which one row of a small problem would not repay),
// at most 4096.
static int hist_blocks(int n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(4096, ((int64_t)n * n + 65535) / 65536));
}
static int mean_blocks(int64_t n) { return (int)((n + mean_rows(n) - 1) / mean_rows(n)); }

size_t column_mean_part_doubles(int64_t n, int d) { return (size_t)mean_blocks(n) * (size_t)d; }

int32_t column_means(const float* X, int64_t n, int d, int64_t ldx, double* part, float* mean,
                     cudaStream_t s) {
    const int nb = mean_blocks(n);
    colsum_partial_kernel<<<dim3((d + 31) / 32, nb), 256, 0, s>>>(X, n, d, ldx, mean_rows(n), part);
    colmean_kernel<<<(d + 31) / 32, 256, 0, s>>>(part, nb, d, n, mean);
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
    select_init_kernel<<<1, 256, 0, s>>>(sel, hist, n);
    const int grid = hist_blocks(n);
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

// ---- the batched build ---------------------------------------------------------------
// ap_similarity_batched runs each stage above once for all problems of the
// batch: a launch's blocks are dealt out to problems by prefix counts, each
// block finds its problem by binary search and runs the single-problem code
// with its local block index, so every problem's S and preference are bit
// for bit those of ap_similarity.  Only the Gram products are launched per
// problem.
struct SimProblem {
    const float* X;
    float* S;
    int64_t lds;
    int n, npad;
    int64_t mrows;          // rows per column-sum block
    int nb;                 // column-sum blocks
    int part_b0;            // first column-sum block of the problem in the batched grid
    int centre_b0, centre_nb;
    int hist_b0, hist_nb;
    double* part;
    float* mean;
    void* xc;
    float* nrm;
    SelectState* sel;
    unsigned long long* hist;
    float* pref;
    int64_t roff;           // first row of the problem in the centred-feature arena
};

// The problem whose blocks (first block b0(P[b])) include block `blk`.
template <class F>
__device__ __forceinline__ int sim_problem_of(const SimProblem* P, int count, int blk, F b0) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b0(P[mid]) <= blk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// grid (sum of column-sum blocks, ceil(d/32))
__global__ void __launch_bounds__(256) colsum_batched_kernel(const SimProblem* __restrict__ P, int count,
                                                             int d, int64_t ldx) {
    const int b = sim_problem_of(P, count, blockIdx.x, [](const SimProblem& q) { return q.part_b0; });
    const SimProblem& q = P[b];
    colsum_block(q.X, q.n, d, ldx, q.mrows, q.part, blockIdx.y, blockIdx.x - q.part_b0);
}

// grid (problems, ceil(d/32)), 256 threads
__global__ void __launch_bounds__(256) colmean_batched_kernel(const SimProblem* __restrict__ P, int d) {
    const SimProblem& q = P[blockIdx.x];
    colmean_block(q.part, q.nb, d, q.n, q.mean, blockIdx.y);
}

// grid (sum of centring blocks)
template <bool BF16, bool VEC>
__global__ void centre_batched_kernel(const SimProblem* __restrict__ P, int count, int d, int64_t ldx,
                                      int dpad) {
    const int b = sim_problem_of(P, count, blockIdx.x, [](const SimProblem& q) { return q.centre_b0; });
    const SimProblem& q = P[b];
    if (VEC)
        centre_rows4<BF16>(q.X, q.n, d, ldx, q.mean, q.npad, dpad, q.xc, q.nrm, blockIdx.x - q.centre_b0,
                           q.centre_nb);
    else
        centre_rows<BF16>(q.X, q.n, d, ldx, q.mean, q.npad, dpad, q.xc, q.nrm, blockIdx.x - q.centre_b0,
                          q.centre_nb);
}

// grid (problems)
__global__ void select_init_batched_kernel(const SimProblem* __restrict__ P) {
    const SimProblem& q = P[blockIdx.x];
    select_init_block(q.sel, q.hist, q.n);
}

// grid (sum of histogram blocks)
template <bool VEC>
__global__ void __launch_bounds__(256) radix_hist_batched_kernel(const SimProblem* __restrict__ P, int count,
                                                                 int shift, int bits) {
    const int b = sim_problem_of(P, count, blockIdx.x, [](const SimProblem& q) { return q.hist_b0; });
    const SimProblem& q = P[b];
    radix_hist_rows<VEC>(q.S, q.n, q.lds, shift, bits, q.sel, q.hist, blockIdx.x - q.hist_b0, q.hist_nb);
}

// grid (problems), 1024 threads
__global__ void __launch_bounds__(1024) radix_scan_batched_kernel(const SimProblem* __restrict__ P, int shift,
                                                                  int bits) {
    const SimProblem& q = P[blockIdx.x];
    radix_scan_block(q.sel, q.hist, shift, bits);
}

// grid (problems, y); the median (median = 1) or the scalar p onto the diagonal
__global__ void diag_batched_kernel(const SimProblem* __restrict__ P, int median, float pval) {
    const SimProblem& q = P[blockIdx.x];
    const float p = median ? select_result(q.sel) : pval;
    if (median && blockIdx.y == 0 && threadIdx.x == 0) *q.pref = p;
    for (int i = blockIdx.y * blockDim.x + threadIdx.x; i < q.n; i += gridDim.y * blockDim.x)
        q.S[(int64_t)i * q.lds + i] = p;
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
    const bool vx = aligned16(X) && (ldx & 3) == 0;
    if (precision == AP_PREC_FP32) {
        if (vx) centre_kernel<false, true><<<cgrid, 256, 0, s>>>(X, ni, di, ldx, w.mean, npad, dpad, w.xc, w.nrm);
        else centre_kernel<false, false><<<cgrid, 256, 0, s>>>(X, ni, di, ldx, w.mean, npad, dpad, w.xc, w.nrm);
        dim3 grid((ni + GT - 1) / GT, (ni + GT - 1) / GT);
        const int vec_ok = aligned16(S) && (lds & 3) == 0;
        sim_gemm_fp32_kernel<<<grid, 256, 0, s>>>(static_cast<const float*>(w.xc), ni, dpad, w.nrm,
                                                  S, lds, vec_ok);
        AP_TRY(last_error());
    } else {
        if (vx) centre_kernel<true, true><<<cgrid, 256, 0, s>>>(X, ni, di, ldx, w.mean, npad, dpad, w.xc, w.nrm);
        else centre_kernel<true, false><<<cgrid, 256, 0, s>>>(X, ni, di, ldx, w.mean, npad, dpad, w.xc, w.nrm);
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

// The Gram products of a batch are spread round-robin over kSimStreams
// library-owned streams (created once per device), so that the small
// problems' products overlap; they fork from and join back to the caller's
// stream through events.  Every other stage is one launch for the whole batch
// on the caller's stream.
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

// Workspace of a batch: the problem table, every problem's column-sum
// partials, mean, centred copy, norms, select state and histograms, its
// preference and its Gram product's error flag.  host[b] receives problem b's
// pointers and block counts (problem fields filled by the caller).
static size_t carve_batched(void* ws, const int64_t* n, int32_t count, int64_t d, int32_t precision,
                            SimProblem** table, std::vector<SimProblem>* host, int32_t** err,
                            float** prefs, void** tables) {
    Carver c(ws);
    SimProblem* t = c.take<SimProblem>((size_t)count);
    int32_t* e = c.take<int32_t>((size_t)count);
    float* pv = c.take<float>((size_t)count);
    const int dpad = pad_dim((int)d);
    const size_t esz = precision == AP_PREC_FP32 ? sizeof(float) : sizeof(__nv_bfloat16);
    // every problem's centred rows (and norms) in one arena, problem b from row
    // roff_b (a multiple of the tensor-core tile), so that one grouped launch
    // covers the whole batch
    int64_t rows = 0;
    for (int32_t b = 0; b < count; ++b) rows += pad_rows((int)n[b]);
    unsigned char* xc_arena = c.take<unsigned char>((size_t)rows * dpad * esz);
    float* nrm_arena = c.take<float>((size_t)rows);
    void* tab = c.take<unsigned char>(tc_grouped_table_bytes(n, count));
    int part_b0 = 0, centre_b0 = 0, hist_b0 = 0;
    int64_t roff = 0;
    for (int32_t b = 0; b < count; ++b) {
        SimProblem q{};
        q.n = (int)n[b];
        q.npad = pad_rows(q.n);
        q.mrows = mean_rows(n[b]);
        q.nb = mean_blocks(n[b]);
        q.part_b0 = part_b0;
        part_b0 += q.nb;
        q.centre_nb = std::min((q.npad + 7) / 8, 65535);
        q.centre_b0 = centre_b0;
        centre_b0 += q.centre_nb;
        q.hist_nb = hist_blocks(q.n);
        q.hist_b0 = hist_b0;
        hist_b0 += q.hist_nb;
        q.part = c.take<double>((size_t)q.nb * d);
        q.mean = c.take<float>((size_t)d);
        q.roff = roff;
        q.xc = xc_arena ? xc_arena + (size_t)roff * dpad * esz : nullptr;
        q.nrm = nrm_arena ? nrm_arena + roff : nullptr;
        roff += q.npad;
        q.sel = c.take<SelectState>(1);
        q.hist = c.take<unsigned long long>(4096);
        q.pref = pv ? pv + b : nullptr;
        if (host) (*host)[b] = q;
    }
    if (table) *table = t;
    if (err) *err = e;
    if (prefs) *prefs = pv;
    if (tables) *tables = tab;
    return c.used;
}

static bool batched_args_ok(const int64_t* n, int32_t count, int64_t d) {
    if (!n || count < 1 || d < 1 || d > 65536) return false;
    int64_t blocks = 0;
    for (int32_t b = 0; b < count; ++b) {
        if (n[b] < 2 || n[b] > INT_MAX / 2) return false;
        blocks += std::min<int64_t>(n[b], 4096);
    }
    return blocks <= INT_MAX;
}

}  // namespace apgb

APGB_API size_t ap_similarity_batched_workspace_size(const int64_t* n, int32_t count, int64_t d) {
    if (!batched_args_ok(n, count, d)) return 0;
    // the bf16 centred copy is the smaller; size for float32 so one query serves both
    return carve_batched(nullptr, n, count, d, AP_PREC_FP32, nullptr, nullptr, nullptr, nullptr,
                         nullptr);
}

APGB_API int32_t ap_similarity_batched(const float* X, const int64_t* xoff, const int64_t* n,
                                       int32_t count, int64_t d, int64_t ldx, float* S,
                                       const int64_t* soff, const int64_t* lds, int32_t precision,
                                       int32_t pref_mode, const float* pref, float* pref_out,
                                       void* ws, size_t ws_bytes, void* stream) {
    if (!X || !xoff || !n || !S || !soff || !lds || ldx < d || !batched_args_ok(n, count, d))
        return AP_ERR_INVALID_ARG;
    if (pref_mode == AP_PREF_VECTOR || !sim_args_ok(precision, pref_mode, pref, 0.0))
        return AP_ERR_INVALID_ARG;
    int64_t nmax = 0;
    bool vec = true;
    for (int32_t b = 0; b < count; ++b) {
        if (lds[b] < n[b] || xoff[b] < 0 || soff[b] < 0) return AP_ERR_INVALID_ARG;
        nmax = std::max(nmax, n[b]);
        vec = vec && aligned16(S + soff[b]) && (lds[b] & 3) == 0;
    }
    // the bf16 path's tensor stores need 16-byte aligned rows of S
    if (precision != AP_PREC_FP32 && !vec) return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    AP_TRY(check_ws(ws, ws_bytes, ap_similarity_batched_workspace_size(n, count, d)));
    std::vector<SimProblem> host(count);
    SimProblem* table = nullptr;
    int32_t* err = nullptr;
    float* prefs = nullptr;
    void* tables = nullptr;
    carve_batched(ws, n, count, d, precision, &table, &host, &err, &prefs, &tables);
    int part_blocks = 0, centre_blocks = 0, hist_blocks = 0;
    for (int32_t b = 0; b < count; ++b) {
        host[b].X = X + xoff[b];
        host[b].S = S + soff[b];
        host[b].lds = lds[b];
        part_blocks += host[b].nb;
        centre_blocks += host[b].centre_nb;
        hist_blocks += host[b].hist_nb;
    }
    const int di = (int)d, dpad = pad_dim(di);
    const bool bf16 = precision != AP_PREC_FP32;
    AP_CUDA_TRY(cudaMemcpyAsync(table, host.data(), sizeof(SimProblem) * count, cudaMemcpyHostToDevice, s));
    AP_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t) * count, s));
    // 1-2. column means and the centred copies of every problem
    colsum_batched_kernel<<<dim3(part_blocks, (di + 31) / 32), 256, 0, s>>>(table, count, di, ldx);
    colmean_batched_kernel<<<dim3(count, (di + 31) / 32), 256, 0, s>>>(table, di);
    bool vx = (ldx & 3) == 0;
    for (int32_t b = 0; b < count; ++b) vx = vx && aligned16(X + xoff[b]);
    if (bf16) {
        if (vx) centre_batched_kernel<true, true><<<centre_blocks, 256, 0, s>>>(table, count, di, ldx, dpad);
        else centre_batched_kernel<true, false><<<centre_blocks, 256, 0, s>>>(table, count, di, ldx, dpad);
    } else {
        if (vx) centre_batched_kernel<false, true><<<centre_blocks, 256, 0, s>>>(table, count, di, ldx, dpad);
        else centre_batched_kernel<false, false><<<centre_blocks, 256, 0, s>>>(table, count, di, ldx, dpad);
    }
    note_launches(3);
    AP_TRY(last_error());
    // 3. the Gram products: bf16 as one persistent tensor-core launch over the
    //    tiles of every problem; float32 forked over the library's streams
    if (bf16) {
        std::vector<int64_t> roffs(count), nn(count), ld(count);
        std::vector<float*> Sp(count);
        int64_t rows = 0;
        for (int32_t b = 0; b < count; ++b) {
            roffs[b] = host[b].roff;
            nn[b] = host[b].n;
            ld[b] = host[b].lds;
            Sp[b] = host[b].S;
            rows = host[b].roff + host[b].npad;
        }
        AP_TRY(tc_similarity_bf16_grouped(static_cast<const __nv_bfloat16*>(host[0].xc), host[0].nrm, rows,
                                          dpad, nn.data(), roffs.data(), Sp.data(), ld.data(), count,
                                          tables, err, s));
    } else {
        std::array<cudaStream_t, kSimStreams> ss;
        AP_TRY(sim_streams(&ss));
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
            const SimProblem& q = host[b];
            cudaStream_t sk = ss[b % kSimStreams];
            dim3 grid((q.n + GT - 1) / GT, (q.n + GT - 1) / GT);
            const int vec_ok = aligned16(q.S) && (q.lds & 3) == 0;
            sim_gemm_fp32_kernel<<<grid, 256, 0, sk>>>(static_cast<const float*>(q.xc), q.n, dpad, q.nrm,
                                                       q.S, q.lds, vec_ok);
            note_launches(1);
            st = last_error();
        }
        // join: the caller's stream continues after every worker (also on error)
        for (int k = 0; k < kSimStreams; ++k) {
            AP_CUDA_TRY(cudaEventRecord(join[k], ss[k]));
            AP_CUDA_TRY(cudaStreamWaitEvent(s, join[k], 0));
        }
        AP_TRY(st);
    }
    // 4-5. the preferences and the diagonals
    const int dgy = (int)std::min<int64_t>((nmax + 255) / 256, 65535);
    if (pref_mode == AP_PREF_MEDIAN) {
        select_init_batched_kernel<<<count, 256, 0, s>>>(table);
        const int shifts[3] = {21, 10, 0}, bits[3] = {11, 11, 10};
        for (int p = 0; p < 3; ++p) {
            if (vec)
                radix_hist_batched_kernel<true><<<hist_blocks, 256, 0, s>>>(table, count, shifts[p], bits[p]);
            else
                radix_hist_batched_kernel<false><<<hist_blocks, 256, 0, s>>>(table, count, shifts[p], bits[p]);
            radix_scan_batched_kernel<<<count, 1024, 0, s>>>(table, shifts[p], bits[p]);
        }
        diag_batched_kernel<<<dim3(count, dgy), 256, 0, s>>>(table, 1, 0.f);
        note_launches(8);
    } else {
        diag_batched_kernel<<<dim3(count, dgy), 256, 0, s>>>(table, 0, pref[0]);
        note_launches(1);
    }
    AP_TRY(last_error());
    std::vector<float> v(count, pref_mode == AP_PREF_SCALAR ? pref[0] : NAN);
    std::vector<int32_t> e(count, 0);
    if (pref_mode == AP_PREF_MEDIAN)
        AP_CUDA_TRY(cudaMemcpyAsync(v.data(), prefs, sizeof(float) * count, cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaMemcpyAsync(e.data(), err, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    for (int32_t b = 0; b < count; ++b)
        if (e[b]) return AP_ERR_TIMEOUT;
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
