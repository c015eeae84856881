// The learned warm start (not part of the paper; it plays the role Algorithm
// 2's merged availabilities play, and its exemplar score can choose
// Algorithm 3's landmarks).
//
// Per point k of S with preference scale p > 0, 25 features:
//   0-15  the 16 largest off-diagonal s(k,j), decreasing (ties: lower j first), / p
//   16-17 mean and standard deviation of the off-diagonal s(k,j), / p
//   18    s(k,k) / p
//   19-22 log(1 + #{j != k : s(k,j) >= -q p}) for q = 1/8, 1/4, 1/2, 1 (the
//         thresholds formed in float32): how many points lie within q times
//         the preference scale, i.e. how much support k could collect
//   23    D(k) - max_j D(j) over the 16 nearest j of k (those of features
//         0-15), with D = feature 20: positive where k is denser than all of
//         its neighbours, as exemplars tend to be
//   24    the fraction of those 16 neighbours with D(j) > D(k)
// A 25-256-256-3 network (ReLU) maps them to (c_hat, a_hat, logit): the
// predicted converged column value min(0, r(k,k) + a(k,k))/p that the warm
// start writes into column k, a(k,k)/p and the exemplar log-odds.  Training:
// mean over rows of (c_hat-t_c)^2 + (a_hat-t_a)^2 + softplus(logit) -
// t_e*logit, Adam.
//
// Parameters: one flat fp32 vector (W1 256x25, b1, W2 256x256, b2, W3 3x256,
// b3, mu 25, isd 25); the input is standardised first, x -> (x - mu) * isd,
// with mu and isd fixed (their gradient is zero, so Adam leaves them).  The
// products use a bf16 copy of the weights with fp32 accumulation.  All
// reductions (loss, weight gradients) run in a fixed order.
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace apgb {
namespace mlp {

constexpr int IN = 25, HID = 256, OUT = 3;
constexpr int F_DENS = 20;       // the density D(k) of features 23-24
constexpr int64_t OFF_W1 = 0, OFF_B1 = OFF_W1 + HID * IN, OFF_W2 = OFF_B1 + HID,
                  OFF_B2 = OFF_W2 + HID * HID, OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + OUT * HID,
                  OFF_MU = OFF_B3 + OUT, OFF_ISD = OFF_MU + IN, NP = OFF_ISD + IN;

// ---- features -------------------------------------------------------------------
constexpr int TOPK = 16;

// Rows k0, k0 + kstep, ... of one problem, one row per block at a time: rows
// of S read once; per-thread sorted top-16 (value, index) lists merged by 16
// rounds of block arg-max ordered by (value desc, index asc).  Writes
// features 0-22 and the 16 neighbour indices (problem-local).
__device__ __forceinline__ void features_rows(const float* __restrict__ S, int n, int64_t ld, float scale,
                                              float* F, int32_t* nbr, int k0, int kstep) {
    __shared__ float hv[32];
    __shared__ int hi[32];
    __shared__ double s1w[32], s2w[32];
    __shared__ int cw[32][4];
    const int tid = threadIdx.x, lid = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const float inv_scale = 1.f / scale;
    float thr[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) thr[q] = -(scale * (0.125f * (float)(1 << q)));   // exact: powers of 2
    for (int k = k0; k < n; k += kstep) {
        const float* row = S + (int64_t)k * ld;
        float top[TOPK];
        int topi[TOPK];
#pragma unroll
        for (int q = 0; q < TOPK; ++q) { top[q] = -INFINITY; topi[q] = INT_MAX; }
        double s1 = 0.0, s2 = 0.0;
        int cnt[4] = {0, 0, 0, 0};
        for (int j = tid; j < n; j += blockDim.x) {
            if (j == k) continue;
            const float v = row[j];
            s1 += v;
            s2 += (double)v * v;
#pragma unroll
            for (int q = 0; q < 4; ++q) cnt[q] += v >= thr[q];
            if (v > top[TOPK - 1]) {            // insertion; equal values keep the lower j first
                float x = v;
                int xi = j;
#pragma unroll
                for (int q = 0; q < TOPK; ++q) {
                    if (x > top[q]) {
                        const float t = top[q];
                        const int ti = topi[q];
                        top[q] = x; topi[q] = xi;
                        x = t; xi = ti;
                    }
                }
            }
        }
        // block sums (fixed order: warp tree, then warps in order)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
#pragma unroll
            for (int q = 0; q < 4; ++q) cnt[q] += __shfl_xor_sync(0xffffffffu, cnt[q], o);
        }
        if (lid == 0) {
            s1w[wid] = s1; s2w[wid] = s2;
#pragma unroll
            for (int q = 0; q < 4; ++q) cw[wid][q] = cnt[q];
        }
        // 16 rounds of block arg-max over each thread's next candidate
        int head = 0;
        float outv[TOPK];
        int outi[TOPK];
        for (int r = 0; r < TOPK; ++r) {
            float v = head < TOPK ? top[head] : -INFINITY;
            int vi = head < TOPK ? topi[head] : INT_MAX;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
                const int i2 = __shfl_xor_sync(0xffffffffu, vi, o);
                if (v2 > v || (v2 == v && i2 < vi)) { v = v2; vi = i2; }
            }
            if (lid == 0) { hv[wid] = v; hi[wid] = vi; }
            __syncthreads();
            float bv = hv[0];
            int bi = hi[0];
            for (int w = 1; w < nw; ++w)
                if (hv[w] > bv || (hv[w] == bv && hi[w] < bi)) { bv = hv[w]; bi = hi[w]; }
            if (head < TOPK && bi != INT_MAX && topi[head] == bi) ++head;
            outv[r] = bv;
            outi[r] = bi;
            __syncthreads();
        }
        if (tid == 0) {
            double t1 = 0.0, t2 = 0.0;
            int c[4] = {0, 0, 0, 0};
            for (int w = 0; w < nw; ++w) {
                t1 += s1w[w]; t2 += s2w[w];
                for (int q = 0; q < 4; ++q) c[q] += cw[w][q];
            }
            const double m = t1 / (double)(n - 1);
            const double var = fmax(0.0, t2 / (double)(n - 1) - m * m);
            float* f = F + (int64_t)k * IN;
            float last = outv[0];
            int lasti = outi[0];
            for (int r = 0; r < TOPK; ++r) {
                if (outv[r] == -INFINITY) { outv[r] = last; outi[r] = lasti; }  // n - 1 < 16
                last = outv[r];
                lasti = outi[r];
                f[r] = outv[r] * inv_scale;
                nbr[(int64_t)k * TOPK + r] = outi[r];
            }
            f[16] = (float)(m * (double)inv_scale);
            f[17] = (float)(sqrt(var) * (double)inv_scale);
            f[18] = row[k] * inv_scale;
            for (int q = 0; q < 4; ++q) f[19 + q] = log1pf((float)c[q]);
        }
        __syncthreads();
    }
}

__global__ void features_kernel(const float* __restrict__ S, int n, int64_t ld, float scale,
                                float* F, int32_t* nbr) {
    features_rows(S, n, ld, scale, F, nbr, blockIdx.x, gridDim.x);
}

// Features 23-24 of row k from the densities of its 16 neighbours.
__device__ __forceinline__ void neighbour_row(int k, const int32_t* __restrict__ nbr, float* F) {
    const float d = F[(int64_t)k * IN + F_DENS];
    float mx = -INFINITY;
    int denser = 0;
#pragma unroll
    for (int q = 0; q < TOPK; ++q) {
        const float dj = F[(int64_t)nbr[(int64_t)k * TOPK + q] * IN + F_DENS];
        mx = fmaxf(mx, dj);
        denser += dj > d;
    }
    F[(int64_t)k * IN + 23] = d - mx;
    F[(int64_t)k * IN + 24] = (float)denser * (1.f / TOPK);
}

__global__ void neighbour_density_kernel(int n, const int32_t* __restrict__ nbr, float* F) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) neighbour_row(k, nbr, F);
}

// ---- the same over a batch of problems (feature rows of problem b from frow) ----
struct BatchProblem {
    const float* S;         // the problem's S (row stride ld)
    float *R, *A;           // its messages (row stride ld)
    int64_t ld;
    int64_t frow;           // first row of the problem in the feature / output arenas
    int n;
    float scale;
    int b0, nb;             // feature blocks: [b0, b0 + nb)
    int w0;                 // warm-start blocks: [w0, w0 + n), one per row
    int pad;
};

// Largest b with key(P[b]) <= x (P sorted by key).
template <class F>
__device__ __forceinline__ int batch_problem_of(const BatchProblem* P, int count, int64_t x, F key) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (key(P[mid]) <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void features_batched_kernel(const BatchProblem* __restrict__ P, int count, float* F, int32_t* nbr) {
    const int b = batch_problem_of(P, count, blockIdx.x, [](const BatchProblem& q) { return (int64_t)q.b0; });
    const BatchProblem& q = P[b];
    features_rows(q.S, q.n, q.ld, q.scale, F + q.frow * IN, nbr + q.frow * TOPK, blockIdx.x - q.b0, q.nb);
}

__global__ void neighbour_density_batched_kernel(const BatchProblem* __restrict__ P, int count, int64_t rows,
                                                 const int32_t* __restrict__ nbr, float* F) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= rows) return;
    const int b = batch_problem_of(P, count, t, [](const BatchProblem& q) { return q.frow; });
    const BatchProblem& q = P[b];
    neighbour_row((int)(t - q.frow), nbr + q.frow * TOPK, F + q.frow * IN);
}

// Fn = (F - mu) * isd, row-major [rows x IN].
__global__ void standardise_kernel(const float* __restrict__ F, int rows,
                                   const float* __restrict__ P, float* Fn) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)rows * IN) return;
    const int j = (int)(e % IN);
    Fn[e] = (F[e] - P[OFF_MU + j]) * P[OFF_ISD + j];
}

// Column j of the standardisation from F [rows x IN] (one block per column,
// float64 sums in a fixed order): mu = mean, isd = 1 / max(std, 1e-3) with the
// population standard deviation.
__global__ void standardisation_kernel(const float* __restrict__ F, int64_t rows, float* P) {
    __shared__ double s1[256], s2[256];
    const int j = blockIdx.x;
    double a = 0.0, b = 0.0;
    for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) {
        const double v = (double)F[r * IN + j];
        a += v;
        b += v * v;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] += s2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double m = s1[0] / (double)rows;
        const double var = fmax(0.0, s2[0] / (double)rows - m * m);
        P[OFF_MU + j] = (float)m;
        P[OFF_ISD + j] = (float)(1.0 / fmax(sqrt(var), 1e-3));
    }
}

// ---- dense layers ----------------------------------------------------------------
constexpr int TR = 64, TO = 64, TK = 16;

// Y[r][o] = act(sum_i X[r][i] W[o][i] + b[o]); W bf16 [out x in].
__global__ void __launch_bounds__(256) linear_fwd_kernel(const float* __restrict__ X, int rows,
                                                         int in, const __nv_bfloat16* __restrict__ W,
                                                         const float* __restrict__ b, int out,
                                                         int relu, float* Y) {
    __shared__ float xs[TK][TR + 1], ws[TK][TO + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int r0 = blockIdx.x * TR, o0 = blockIdx.y * TO;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < in; k0 += TK) {
        for (int e = threadIdx.x; e < TK * TR; e += 256) {
            const int kk = e % TK, rr = e / TK;
            const int r = r0 + rr, k = k0 + kk;
            xs[kk][rr] = (r < rows && k < in) ? X[(int64_t)r * in + k] : 0.f;
            const int o = o0 + rr;
            ws[kk][rr] = (o < out && k < in) ? __bfloat162float(W[(int64_t)o * in + k]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk)
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    acc[a][c] = fmaf(xs[kk][ty * 4 + a], ws[kk][tx * 4 + c], acc[a][c]);
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int r = r0 + ty * 4 + a;
        if (r >= rows) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int o = o0 + tx * 4 + c;
            if (o >= out) continue;
            float v = acc[a][c] + b[o];
            if (relu) v = fmaxf(v, 0.f);
            Y[(int64_t)r * out + o] = v;
        }
    }
}

// dX[r][i] = (sum_o G[r][o] W[o][i]) * (H[r][i] > 0); W bf16 [out x in].
__global__ void __launch_bounds__(256) linear_bwd_input_kernel(const float* __restrict__ G,
                                                               int rows, int out,
                                                               const __nv_bfloat16* __restrict__ W,
                                                               int in, const float* __restrict__ H,
                                                               float* dX) {
    __shared__ float gs[TK][TR + 1], ws[TK][TO + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int r0 = blockIdx.x * TR, i0 = blockIdx.y * TO;
    float acc[4][4] = {};
    for (int o0 = 0; o0 < out; o0 += TK) {
        for (int e = threadIdx.x; e < TK * TR; e += 256) {
            const int oo = e % TK, rr = e / TK;
            const int r = r0 + rr, o = o0 + oo;
            gs[oo][rr] = (r < rows && o < out) ? G[(int64_t)r * out + o] : 0.f;
            const int i = i0 + rr;
            ws[oo][rr] = (o < out && i < in) ? __bfloat162float(W[(int64_t)o * in + i]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int oo = 0; oo < TK; ++oo)
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    acc[a][c] = fmaf(gs[oo][ty * 4 + a], ws[oo][tx * 4 + c], acc[a][c]);
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int r = r0 + ty * 4 + a;
        if (r >= rows) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = i0 + tx * 4 + c;
            if (i >= in) continue;
            const int64_t at = (int64_t)r * in + i;
            dX[at] = H[at] > 0.f ? acc[a][c] : 0.f;
        }
    }
}

// gW[o][i] = sum_r G[r][o] X[r][i] (rows in a fixed order); one output tile
// per block, so the sum is deterministic.
__global__ void __launch_bounds__(256) weight_grad_kernel(const float* __restrict__ G, int rows,
                                                          int out, const float* __restrict__ X,
                                                          int in, float* gW) {
    __shared__ float gs[TK][TO + 1], xs[TK][TO + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int o0 = blockIdx.x * TO, i0 = blockIdx.y * TO;
    float acc[4][4] = {};
    for (int rr0 = 0; rr0 < rows; rr0 += TK) {
        for (int e = threadIdx.x; e < TK * TO; e += 256) {
            const int kk = e / TO, c = e % TO;
            const int r = rr0 + kk;
            gs[kk][c] = (r < rows && o0 + c < out) ? G[(int64_t)r * out + o0 + c] : 0.f;
            xs[kk][c] = (r < rows && i0 + c < in) ? X[(int64_t)r * in + i0 + c] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk)
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    acc[a][c] = fmaf(gs[kk][ty * 4 + a], xs[kk][tx * 4 + c], acc[a][c]);
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int o = o0 + ty * 4 + a;
        if (o >= out) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = i0 + tx * 4 + c;
            if (i < in) gW[(int64_t)o * in + i] = acc[a][c];
        }
    }
}

// gb[o] = sum_r G[r][o], one thread per column, rows in order.
__global__ void bias_grad_kernel(const float* __restrict__ G, int rows, int out, float* gb) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= out) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += G[(int64_t)r * out + o];
    gb[o] = s;
}

// Per-row loss terms and dL/dY (already divided by the row count).
__global__ void loss_kernel(const float* __restrict__ Y, const float* __restrict__ T, int rows,
                            float* G, float* lrow) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const float inv = 1.f / (float)rows;
    const float d = Y[r * 3 + 0] - T[r * 3 + 0];
    const float e = Y[r * 3 + 1] - T[r * 3 + 1];
    const float z = Y[r * 3 + 2], t = T[r * 3 + 2];
    const float sp = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));     // softplus(z)
    lrow[r] = d * d + e * e + sp - t * z;
    G[r * 3 + 0] = 2.f * d * inv;
    G[r * 3 + 1] = 2.f * e * inv;
    G[r * 3 + 2] = (1.f / (1.f + expf(-z)) - t) * inv;
}

__global__ void mean_kernel(const float* __restrict__ v, int n, float* out) {
    __shared__ double sh[1024];
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(n, lo + per);
    double x = 0.0;
    for (int i = lo; i < hi; ++i) x += v[i];
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (float)(sh[0] / (double)n);
}

// Adam with bias correction; refreshes the bf16 copy of the weights.
__global__ void adam_kernel(float* P, const float* __restrict__ g, float* m, float* v, int64_t np,
                            float lr, float b1, float b2, float eps, float c1, float c2,
                            __nv_bfloat16* P16) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float mi = b1 * m[i] + (1.f - b1) * g[i];
        const float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
        m[i] = mi;
        v[i] = vi;
        const float p = P[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        P[i] = p;
        P16[i] = __float2bfloat16_rn(p);
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ P, int64_t np, __nv_bfloat16* P16) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
         i += (int64_t)gridDim.x * blockDim.x)
        P16[i] = __float2bfloat16_rn(P[i]);
}

__global__ void targets_kernel(const float* __restrict__ R, const float* __restrict__ A,
                               const int32_t* __restrict__ dec, int n, int64_t ld, float inv_scale,
                               float* T) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    T[k * 3 + 0] = fminf(0.f, R[(int64_t)k * ld + k] + A[(int64_t)k * ld + k]) * inv_scale;
    T[k * 3 + 1] = A[(int64_t)k * ld + k] * inv_scale;
    T[k * 3 + 2] = dec[k] == k ? 1.f : 0.f;
}

// Column-constant availabilities from the per-point predictions (the fixed
// point of Eq. 3-4 up to the i-th term): A(i,k) = min(0, c_hat_k p) for
// i != k, A(k,k) = max(0, a_hat_k p).  One block-row of A per block.
__global__ void warm_columns_kernel(const float* __restrict__ Y, int n, float scale, float* A,
                                    int64_t ld) {
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        float* row = A + (int64_t)i * ld;
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const float ch = Y[k * 3 + 0], ah = Y[k * 3 + 1];
            row[k] = (k == i) ? fmaxf(0.f, ah * scale) : fminf(0.f, ch * scale);
        }
    }
}

// The warm start of every problem of a batch: one block per row i of problem
// b; R(i,:) = 0 and A(i,:) the column-constant availabilities of b's
// predictions (as warm_columns_kernel).
__global__ void warm_batched_kernel(const BatchProblem* __restrict__ P, int count, const float* __restrict__ Y) {
    const int b = batch_problem_of(P, count, blockIdx.x, [](const BatchProblem& q) { return (int64_t)q.w0; });
    const BatchProblem& q = P[b];
    const int i = blockIdx.x - q.w0;
    const float* y = Y + q.frow * OUT;
    float* rr = q.R + (int64_t)i * q.ld;
    float* ar = q.A + (int64_t)i * q.ld;
    for (int k = threadIdx.x; k < q.n; k += blockDim.x) {
        const float ch = y[k * 3 + 0], ah = y[k * 3 + 1];
        rr[k] = 0.f;
        ar[k] = (k == i) ? fmaxf(0.f, ah * q.scale) : fminf(0.f, ch * q.scale);
    }
}

struct MlpWs {
    float *Fn, *H1, *H2, *Y, *G3, *G2, *G1, *lrow, *grad;
};

static size_t carve(void* ws, int64_t rows, MlpWs* w) {
    Carver c(ws);
    w->Fn = c.take<float>((size_t)rows * IN);
    w->H1 = c.take<float>((size_t)rows * HID);
    w->H2 = c.take<float>((size_t)rows * HID);
    w->Y = c.take<float>((size_t)rows * OUT);
    w->G3 = c.take<float>((size_t)rows * OUT);
    w->G2 = c.take<float>((size_t)rows * HID);
    w->G1 = c.take<float>((size_t)rows * HID);
    w->lrow = c.take<float>(rows);
    w->grad = c.take<float>(NP);
    return c.used;
}

static dim3 grid2(int rows, int cols) { return dim3((rows + TR - 1) / TR, (cols + TO - 1) / TO); }

static int32_t forward(const float* P, const __nv_bfloat16* P16, const float* F, int rows,
                       const MlpWs& w, float* Y, cudaStream_t s) {
    standardise_kernel<<<(int)(((int64_t)rows * IN + 255) / 256), 256, 0, s>>>(F, rows, P, w.Fn);
    linear_fwd_kernel<<<grid2(rows, HID), 256, 0, s>>>(w.Fn, rows, IN, P16 + OFF_W1, P + OFF_B1, HID, 1, w.H1);
    linear_fwd_kernel<<<grid2(rows, HID), 256, 0, s>>>(w.H1, rows, HID, P16 + OFF_W2, P + OFF_B2, HID, 1, w.H2);
    linear_fwd_kernel<<<grid2(rows, OUT), 256, 0, s>>>(w.H2, rows, HID, P16 + OFF_W3, P + OFF_B3, OUT, 0, Y);
    note_launches(4);
    return last_error();
}

}  // namespace mlp
}  // namespace apgb

using namespace apgb;
using namespace apgb::mlp;

APGB_API int64_t apl_param_count(void) { return NP; }

APGB_API size_t apl_features_workspace_size(int64_t n) {
    if (n < 2 || n > INT_MAX) return 0;
    Carver c(nullptr);
    c.take<int32_t>((size_t)n * TOPK);
    return c.used;
}

APGB_API int32_t apl_features(const float* S, int64_t n, int64_t ld, float scale, float* F,
                              void* ws, size_t ws_bytes, void* stream) {
    if (!S || !F || n < 2 || ld < n || n > INT_MAX || !(scale > 0.f)) return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    AP_TRY(check_ws(ws, ws_bytes, apl_features_workspace_size(n)));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver c(ws);
    int32_t* nbr = c.take<int32_t>((size_t)n * TOPK);
    features_kernel<<<(int)std::min<int64_t>(n, 65535), 256, 0, s>>>(S, (int)n, ld, scale, F, nbr);
    neighbour_density_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>((int)n, nbr, F);
    note_launches(2);
    return last_error();
}

APGB_API int32_t apl_targets(const float* R, const float* A, const int32_t* dec, int64_t n,
                             int64_t ld, float scale, float* T, void* stream) {
    if (!R || !A || !dec || !T || n < 1 || ld < n || n > INT_MAX || !(scale > 0.f))
        return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    targets_kernel<<<(int)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        R, A, dec, (int)n, ld, 1.f / scale, T);
    note_launches(1);
    return last_error();
}

APGB_API size_t apl_workspace_size(int64_t rows) {
    if (rows < 1 || rows > INT_MAX / HID) return 0;
    MlpWs w;
    return carve(nullptr, rows, &w);
}

APGB_API int32_t apl_sync_bf16(const float* P, void* P16, void* stream) {
    if (!P || !P16) return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    to_bf16_kernel<<<(int)((NP + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        P, NP, static_cast<__nv_bfloat16*>(P16));
    note_launches(1);
    return last_error();
}

APGB_API int32_t apl_forward(const float* P, const void* P16, const float* F, int64_t rows,
                             float* Y, void* ws, size_t ws_bytes, void* stream) {
    if (!P || !P16 || !F || !Y || rows < 1 || rows > INT_MAX / HID) return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    MlpWs w;
    AP_TRY(check_ws(ws, ws_bytes, carve(nullptr, rows, &w)));
    carve(ws, rows, &w);
    return forward(P, static_cast<const __nv_bfloat16*>(P16), F, (int)rows, w, Y,
                   static_cast<cudaStream_t>(stream));
}

APGB_API int32_t apl_train_step(float* P, void* P16, float* M, float* V, int64_t step, float lr,
                                const float* F, const float* T, int64_t rows, float* loss,
                                float* grad_out, void* ws, size_t ws_bytes, void* stream) {
    if (!P || !P16 || !M || !V || !F || !T || rows < 1 || rows > INT_MAX / HID || step < 1 ||
        !(lr >= 0.f))
        return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MlpWs w;
    AP_TRY(check_ws(ws, ws_bytes, carve(nullptr, rows, &w)));
    carve(ws, rows, &w);
    const int r = (int)rows;
    const __nv_bfloat16* W16 = static_cast<const __nv_bfloat16*>(P16);
    AP_TRY(forward(P, W16, F, r, w, w.Y, s));
    loss_kernel<<<(r + 255) / 256, 256, 0, s>>>(w.Y, T, r, w.G3, w.lrow);
    if (loss) mean_kernel<<<1, 1024, 0, s>>>(w.lrow, r, loss);
    float* g = w.grad;
    // layer 3
    weight_grad_kernel<<<dim3(1, (HID + TO - 1) / TO), 256, 0, s>>>(w.G3, r, OUT, w.H2, HID, g + OFF_W3);
    bias_grad_kernel<<<1, 32, 0, s>>>(w.G3, r, OUT, g + OFF_B3);
    linear_bwd_input_kernel<<<grid2(r, HID), 256, 0, s>>>(w.G3, r, OUT, W16 + OFF_W3, HID, w.H2, w.G2);
    // layer 2
    weight_grad_kernel<<<dim3((HID + TO - 1) / TO, (HID + TO - 1) / TO), 256, 0, s>>>(w.G2, r, HID, w.H1, HID, g + OFF_W2);
    bias_grad_kernel<<<(HID + 255) / 256, 256, 0, s>>>(w.G2, r, HID, g + OFF_B2);
    linear_bwd_input_kernel<<<grid2(r, HID), 256, 0, s>>>(w.G2, r, HID, W16 + OFF_W2, HID, w.H1, w.G1);
    // layer 1
    weight_grad_kernel<<<dim3((HID + TO - 1) / TO, 1), 256, 0, s>>>(w.G1, r, HID, w.Fn, IN, g + OFF_W1);
    bias_grad_kernel<<<(HID + 255) / 256, 256, 0, s>>>(w.G1, r, HID, g + OFF_B1);
    AP_CUDA_TRY(cudaMemsetAsync(g + OFF_MU, 0, sizeof(float) * 2 * IN, s));   // fixed standardisation
    if (grad_out) AP_CUDA_TRY(cudaMemcpyAsync(grad_out, g, sizeof(float) * NP, cudaMemcpyDeviceToDevice, s));
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)step));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)step));
    adam_kernel<<<(int)((NP + 255) / 256), 256, 0, s>>>(P, g, M, V, NP, lr, b1, b2, 1e-8f, c1, c2,
                                                        static_cast<__nv_bfloat16*>(P16));
    note_launches(loss ? 12 : 11);
    return last_error();
}

APGB_API int32_t apl_warm_start(const float* Y, int64_t n, float scale, float* R, float* A,
                                int64_t ld, void* stream) {
    if (!Y || !R || !A || n < 1 || ld < n || n > INT_MAX || !(scale > 0.f)) return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    AP_CUDA_TRY(cudaMemset2DAsync(R, ld * sizeof(float), 0, n * sizeof(float), n, s));
    warm_columns_kernel<<<(int)std::min<int64_t>(n, 4096), 256, 0, s>>>(Y, (int)n, scale, A, ld);
    note_launches(1);
    return last_error();
}

// ---- warm-started Algorithm 1, judged by the cold start ---------------------------
namespace apgb {
int32_t exemplars_impl(const float* S, const float* R, const float* A, int64_t n, int64_t ld,
                       int32_t* idx, ap_result* out, void* ws, size_t ws_bytes, cudaStream_t s);
size_t exemplars_ws_bytes(int64_t n);

struct RunWs {
    float *F, *Y, *R2, *A2;
    int32_t* idx2;
    void* mlp_ws;
    size_t mlp_bytes;
    void* sub_ws;
    size_t sub_bytes;
};

static size_t carve_run(void* ws, int64_t n, int64_t ld, RunWs* w) {
    const size_t mb = apl_workspace_size(n);
    const size_t sb = std::max({ap_iterate_workspace_size(n, ld), exemplars_ws_bytes(n),
                                apl_features_workspace_size(n)});
    Carver c(ws);
    w->F = c.take<float>((size_t)n * mlp::IN);
    w->Y = c.take<float>((size_t)n * mlp::OUT);
    w->R2 = c.take<float>((size_t)n * ld);
    w->A2 = c.take<float>((size_t)n * ld);
    w->idx2 = c.take<int32_t>(n);
    w->mlp_ws = c.take<char>(mb);
    w->mlp_bytes = mb;
    w->sub_ws = c.take<char>(sb);
    w->sub_bytes = sb;
    return (mb && sb) ? c.used : 0;
}
}  // namespace apgb

APGB_API size_t apl_ap_run_workspace_size(int64_t n, int64_t ld) {
    if (n < 2 || ld < n || n > INT_MAX / 256) return 0;
    RunWs w;
    return carve_run(nullptr, n, ld, &w);
}

APGB_API int32_t apl_ap_run(const float* S, int64_t n, int64_t ld, const float* P, const void* P16,
                            float scale, const ap_params* params, int32_t judge, float* R, float* A,
                            int32_t* idx, apl_result* out, void* ws, size_t ws_bytes, void* stream) {
    if (!S || !P || !P16 || !params || !R || !A || !idx || !out || n < 2 || ld < n ||
        n > INT_MAX / 256 || !(scale > 0.f))
        return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    RunWs w;
    const size_t need = carve_run(nullptr, n, ld, &w);
    if (need == 0) return AP_ERR_INVALID_ARG;
    AP_TRY(check_ws(ws, ws_bytes, need));
    carve_run(ws, n, ld, &w);
    cudaEvent_t ev[5];
    for (auto& e : ev) AP_CUDA_TRY(cudaEventCreate(&e));
    struct Guard {
        cudaEvent_t* e;
        ~Guard() { for (int i = 0; i < 5; ++i) cudaEventDestroy(e[i]); }
    } guard{ev};

    *out = apl_result{};
    AP_CUDA_TRY(cudaEventRecord(ev[0], s));
    AP_TRY(apl_features(S, n, ld, scale, w.F, w.sub_ws, w.sub_bytes, stream));
    AP_CUDA_TRY(cudaEventRecord(ev[1], s));
    AP_TRY(apl_forward(P, P16, w.F, n, w.Y, w.mlp_ws, w.mlp_bytes, stream));
    AP_TRY(apl_warm_start(w.Y, n, scale, R, A, ld, stream));
    AP_CUDA_TRY(cudaEventRecord(ev[2], s));
    ap_result rw;
    const int32_t sw = ap_iterate(S, R, A, n, ld, params, nullptr, &rw, w.sub_ws, w.sub_bytes, stream);
    if (sw < 0) return sw;
    const int32_t wi = rw.iters, wc = rw.converged;
    const int32_t swe = exemplars_impl(S, R, A, n, ld, idx, &rw, w.sub_ws, w.sub_bytes, s);
    if (swe < 0) return swe;
    rw.iters = wi;
    rw.converged = wc;
    rw.status = std::max(sw, swe);
    AP_CUDA_TRY(cudaEventRecord(ev[3], s));
    out->warm_iters = wi;
    out->warm_netsim = rw.netsim;
    out->result = rw;
    out->used_warm = 1;
    if (judge) {
        AP_CUDA_TRY(cudaMemset2DAsync(w.R2, ld * sizeof(float), 0, n * sizeof(float), n, s));
        AP_CUDA_TRY(cudaMemset2DAsync(w.A2, ld * sizeof(float), 0, n * sizeof(float), n, s));
        ap_result rc;
        const int32_t sc = ap_iterate(S, w.R2, w.A2, n, ld, params, nullptr, &rc, w.sub_ws,
                                      w.sub_bytes, stream);
        if (sc < 0) return sc;
        const int32_t ci = rc.iters, cc = rc.converged;
        const int32_t sce = exemplars_impl(S, w.R2, w.A2, n, ld, w.idx2, &rc, w.sub_ws,
                                           w.sub_bytes, s);
        if (sce < 0) return sce;
        rc.iters = ci;
        rc.converged = cc;
        rc.status = std::max(sc, sce);
        out->cold_iters = ci;
        out->cold_netsim = rc.netsim;
        // the judge: keep the warm result only within 0.5 % of the cold net similarity
        const bool ok = rw.n_exemplars > 0 && rc.n_exemplars > 0 &&
                        std::fabs(rw.netsim - rc.netsim) <= 0.005 * std::fabs(rc.netsim);
        if (!ok || rw.n_exemplars == 0) {
            out->used_warm = 0;
            out->result = rc;
            AP_CUDA_TRY(cudaMemcpy2DAsync(R, ld * sizeof(float), w.R2, ld * sizeof(float),
                                          n * sizeof(float), n, cudaMemcpyDeviceToDevice, s));
            AP_CUDA_TRY(cudaMemcpy2DAsync(A, ld * sizeof(float), w.A2, ld * sizeof(float),
                                          n * sizeof(float), n, cudaMemcpyDeviceToDevice, s));
            AP_CUDA_TRY(cudaMemcpyAsync(idx, w.idx2, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
        }
    }
    AP_CUDA_TRY(cudaEventRecord(ev[4], s));
    AP_CUDA_TRY(cudaEventSynchronize(ev[4]));
    float ms[4];
    for (int i = 0; i < 4; ++i) AP_CUDA_TRY(cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]));
    out->features_ms = ms[0];
    out->forward_ms = ms[1];
    out->warm_ms = ms[2];
    out->cold_ms = ms[3];
    return out->result.status;
}

// ---- the learned warm start over a batch of problems ------------------------------------
namespace apgb {
namespace mlp {

constexpr int64_t kFwdChunk = 65536;     // rows per forward pass (bounds the layer scratch)

static size_t carve_batch(void* ws, const int64_t* n, int32_t count, BatchProblem** table, float** F,
                          int32_t** nbr, float** Y, void** mlp_ws, size_t* mlp_bytes) {
    int64_t rows = 0;
    for (int32_t b = 0; b < count; ++b) rows += n[b];
    MlpWs tmp;
    const size_t mb = carve(nullptr, std::min(rows, kFwdChunk), &tmp);
    Carver c(ws);
    BatchProblem* t = c.take<BatchProblem>((size_t)count);
    float* f = c.take<float>((size_t)rows * IN);
    int32_t* nb = c.take<int32_t>((size_t)rows * TOPK);
    float* y = c.take<float>((size_t)rows * OUT);
    void* m = c.take<char>(mb);
    if (table) *table = t;
    if (F) *F = f;
    if (nbr) *nbr = nb;
    if (Y) *Y = y;
    if (mlp_ws) *mlp_ws = m;
    if (mlp_bytes) *mlp_bytes = mb;
    return c.used;
}

}  // namespace mlp
}  // namespace apgb

APGB_API size_t apl_warm_start_batched_workspace_size(const int64_t* n, int32_t count) {
    if (!n || count < 1) return 0;
    for (int32_t b = 0; b < count; ++b)
        if (n[b] < 2 || n[b] > INT_MAX) return 0;
    return carve_batch(nullptr, n, count, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
}

APGB_API int32_t apl_warm_start_batched(const float* S, float* R, float* A, const int64_t* offsets,
                                        const int64_t* n, const int64_t* ld, int32_t count,
                                        const float* scale, const float* P, const void* P16, float* Y,
                                        void* ws, size_t ws_bytes, void* stream) {
    if (!S || !R || !A || !offsets || !n || !ld || !scale || !P || !P16 || count < 1)
        return AP_ERR_INVALID_ARG;
    const size_t need = apl_warm_start_batched_workspace_size(n, count);
    if (!need) return AP_ERR_INVALID_ARG;
    int64_t rows = 0, blocks = 0;
    std::vector<BatchProblem> host(count);
    for (int32_t b = 0; b < count; ++b) {
        if (ld[b] < n[b] || offsets[b] < 0 || !(scale[b] > 0.f)) return AP_ERR_INVALID_ARG;
        BatchProblem& q = host[b];
        q.S = S + offsets[b];
        q.R = R + offsets[b];
        q.A = A + offsets[b];
        q.ld = ld[b];
        q.frow = rows;
        q.n = (int)n[b];
        q.scale = scale[b];
        q.nb = (int)std::min<int64_t>(n[b], 1024);
        q.b0 = (int)blocks;
        blocks += q.nb;
        rows += n[b];
    }
    if (blocks > INT_MAX || rows > INT_MAX) return AP_ERR_INVALID_ARG;
    int w0 = 0;
    for (int32_t b = 0; b < count; ++b) {
        host[b].w0 = w0;
        w0 += host[b].n;
    }
    AP_TRY(require_sm103());
    AP_TRY(check_ws(ws, ws_bytes, need));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchProblem* table = nullptr;
    float *F = nullptr, *Yw = nullptr;
    int32_t* nbr = nullptr;
    void* mws = nullptr;
    size_t mbytes = 0;
    carve_batch(ws, n, count, &table, &F, &nbr, &Yw, &mws, &mbytes);
    if (!Y) Y = Yw;
    AP_CUDA_TRY(cudaMemcpyAsync(table, host.data(), sizeof(BatchProblem) * count, cudaMemcpyHostToDevice, s));
    features_batched_kernel<<<(int)blocks, 256, 0, s>>>(table, count, F, nbr);
    neighbour_density_batched_kernel<<<(int)((rows + 255) / 256), 256, 0, s>>>(table, count, rows, nbr, F);
    note_launches(2);
    AP_TRY(last_error());
    MlpWs w;
    carve(mws, std::min(rows, kFwdChunk), &w);
    for (int64_t lo = 0; lo < rows; lo += kFwdChunk) {
        const int cnt = (int)std::min(kFwdChunk, rows - lo);
        AP_TRY(forward(P, static_cast<const __nv_bfloat16*>(P16), F + lo * IN, cnt, w, Y + lo * OUT, s));
    }
    warm_batched_kernel<<<w0, 256, 0, s>>>(table, count, Y);
    note_launches(1);
    return last_error();
}

APGB_API int32_t apl_set_standardisation(float* P, const float* F, int64_t rows, void* stream) {
    if (!P || !F || rows < 1) return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    standardisation_kernel<<<IN, 256, 0, static_cast<cudaStream_t>(stream)>>>(F, rows, P);
    note_launches(1);
    return last_error();
}

APGB_API int32_t apl_judge(const double* cold_netsim, const double* warm_netsim, int32_t count,
                           double tol, int32_t* use_warm) {
    if (!cold_netsim || !warm_netsim || !use_warm || count < 0 || !(tol >= 0.0)) return AP_ERR_INVALID_ARG;
    int32_t kept = 0;
    for (int32_t b = 0; b < count; ++b) {
        const double c = cold_netsim[b], w = warm_netsim[b];
        use_warm[b] = (std::isfinite(c) && std::isfinite(w) && std::fabs(w - c) <= tol * std::fabs(c)) ? 1 : 0;
        kept += use_warm[b];
    }
    return kept;
}
