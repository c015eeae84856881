// lap_run: landmark affinity propagation, Algorithm 3 (Section 4), Steps 1-2.
//   Step 1: a sample M of landmarks -- uniform (the L points with the smallest
//           splitmix64 keys), by a caller-supplied score (the L largest), or
//           given -- then Algorithm 1 on S_M (preference: its off-diagonal
//           median) -> c exemplars.
//   Step 2: every point joins its nearest exemplar (squared Euclidean
//           distance), by the tcgen05 GEMM with the row arg-max fused into its
//           epilogue; exemplars keep themselves.  netsim over all N points in
//           float64.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <climits>
#include <vector>

#include "common.cuh"

namespace apgb {

int32_t exemplars_impl(const float* S, const float* R, const float* A, int64_t n, int64_t ld,
                       int32_t* idx, ap_result* out, void* ws, size_t ws_bytes, cudaStream_t s);
size_t exemplars_ws_bytes(int64_t n);
int32_t tc_assign_argmax(const __nv_bfloat16* A, int na, const __nv_bfloat16* B, int nb,
                         const float* bnrm, int dpad, int32_t* arg, float* best, int32_t* err,
                         cudaStream_t s);
int32_t tc_assign_top2(const __nv_bfloat16* A, int na, const __nv_bfloat16* B, int nb,
                       const float* bnrm, int dpad, int32_t* arg, float* best, int32_t* arg2,
                       float* best2, int32_t* err, cudaStream_t s);

// ---- landmark keys and exact selection of the L smallest -------------------------
__global__ void keys_uniform_kernel(uint64_t seed, int64_t n, uint64_t* keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = splitmix64_at(seed, (uint64_t)i + 1);
}

// Larger score first: key = (order-reversed float key) in the high 32 bits.
__global__ void keys_score_kernel(const float* __restrict__ score, int64_t n, uint64_t* keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t u = __float_as_uint(score[i]);
        const uint32_t fk = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
        keys[i] = (uint64_t)(0xFFFFFFFFu - fk) << 32;
    }
}

struct KSelect {
    uint64_t prefix;      // known high digits of the L-th smallest key
    uint64_t rank;        // its rank among keys sharing the prefix
    int32_t shift;
    int32_t pad;
    uint64_t less;        // keys strictly below the threshold (after the last pass)
};

__global__ void kselect_init_kernel(KSelect* st, uint64_t rank, unsigned* hist) {
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
    if (threadIdx.x == 0) {
        st->prefix = 0;
        st->rank = rank;
        st->shift = 56;
        st->less = 0;
    }
}

__global__ void kselect_hist_kernel(const uint64_t* __restrict__ keys, int64_t n,
                                    const KSelect* __restrict__ st, unsigned* hist) {
    __shared__ unsigned h[256];
    for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const int shift = st->shift;
    const uint64_t mask = (shift >= 56) ? 0ull : (~0ull << (shift + 8));
    const uint64_t pre = st->prefix;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        if ((k & mask) == pre) atomicAdd(&h[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        if (h[b]) atomicAdd(&hist[b], h[b]);
}

__global__ void kselect_scan_kernel(KSelect* st, unsigned* hist) {
    if (threadIdx.x != 0) return;
    uint64_t r = st->rank;
    int b = 0;
    for (; b < 256; ++b) {
        if (r < hist[b]) break;
        r -= hist[b];
        st->less += hist[b];
    }
    if (b > 255) b = 255;            // unreachable with consistent counts
    st->prefix |= (uint64_t)b << st->shift;
    st->rank = r;
    st->shift -= 8;
    for (int x = 0; x < 256; ++x) hist[x] = 0;
}

// ---- order-preserving compaction over up to kCompactBlocks blocks -------------
// Block b owns the contiguous range [b * chunk, min(n, (b + 1) * chunk)).  A
// count kernel stores each block's counts; the write kernel adds the counts of
// the blocks before its own (at most kCompactBlocks) and places every selected
// index at its rank among the selected ones, so the output is ascending.
constexpr int kCompactBlocks = 256;

static int compact_blocks(int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(kCompactBlocks, (n + 1023) / 1024));
}

// Sum of a block's thread values (blockDim.x a multiple of 32, at most 1024).
__device__ __forceinline__ int block_sum(int v, int* red) {
    const int lid = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lid == 0) red[wid] = v;
    __syncthreads();
    int t = 0;
    for (int w = 0; w < nw; ++w) t += red[w];
    return t;
}

// Sum of cnt[0 .. b-1] (b <= kCompactBlocks), in every thread.
__device__ __forceinline__ int64_t counts_before(const unsigned* __restrict__ cnt, int b, int* red) {
    int v = 0;
    for (int c = threadIdx.x; c < b; c += blockDim.x) v += (int)cnt[c];
    return block_sum(v, red);
}

// Landmark selection: per block, the keys below the threshold (cnt[b]) and
// equal to it (cnt[kCompactBlocks + b]).
__global__ void kselect_count_kernel(const uint64_t* __restrict__ keys, int64_t n, int64_t chunk,
                                     const KSelect* __restrict__ st, unsigned* cnt) {
    __shared__ int red[32];
    const uint64_t thr = st->prefix;
    const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    int lt = 0, eq = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const uint64_t k = keys[i];
        lt += k < thr;
        eq += k == thr;
    }
    lt = block_sum(lt, red);
    eq = block_sum(eq, red);
    if (threadIdx.x == 0) {
        cnt[blockIdx.x] = (unsigned)lt;
        cnt[kCompactBlocks + blockIdx.x] = (unsigned)eq;
    }
}

// Index order: every key below the threshold, then as many keys equal to it
// as are needed (the lowest indices).  out is ascending.
__global__ void kselect_write_kernel(const uint64_t* __restrict__ keys, int64_t n, int64_t chunk,
                                     const KSelect* __restrict__ st, int64_t L,
                                     const unsigned* __restrict__ cnt, int32_t* out) {
    __shared__ int red[32], wlt[32], weq[32];
    const uint64_t thr = st->prefix;
    const int64_t ties = L - (int64_t)st->less;             // keys equal to thr to take
    int64_t lt_base = counts_before(cnt, blockIdx.x, red);
    int64_t eq_base = counts_before(cnt + kCompactBlocks, blockIdx.x, red);
    const int lid = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    for (int64_t b0 = lo; b0 < hi; b0 += blockDim.x) {
        const int64_t i = b0 + threadIdx.x;
        const uint64_t k = (i < hi) ? keys[i] : ~0ull;
        const bool lt = i < hi && k < thr, eq = i < hi && k == thr;
        const unsigned blt = __ballot_sync(0xffffffffu, lt), beq = __ballot_sync(0xffffffffu, eq);
        __syncthreads();                                    // the previous step read wlt, weq
        if (lid == 0) { wlt[wid] = __popc(blt); weq[wid] = __popc(beq); }
        __syncthreads();
        int64_t lt_before = lt_base, eq_before = eq_base;
        int tl = 0, te = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < wid) { lt_before += wlt[w]; eq_before += weq[w]; }
            tl += wlt[w];
            te += weq[w];
        }
        const unsigned below = (1u << lid) - 1u;
        lt_before += __popc(blt & below);
        eq_before += __popc(beq & below);
        if (lt || (eq && eq_before < ties))
            out[lt_before + (eq_before < ties ? eq_before : ties)] = (int32_t)i;
        lt_base += tl;
        eq_base += te;
    }
}

// out = the indices i < n with flags[i] != 0, ascending; *count their number.
// Per block, the flags set (cnt[b]).
__global__ void flags_count_kernel(const int32_t* __restrict__ flags, int64_t n, int64_t chunk,
                                   unsigned* cnt) {
    __shared__ int red[32];
    const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    int f = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) f += flags[i] != 0;
    f = block_sum(f, red);
    if (threadIdx.x == 0) cnt[blockIdx.x] = (unsigned)f;
}

__global__ void flags_write_kernel(const int32_t* __restrict__ flags, int64_t n, int64_t chunk,
                                   const unsigned* __restrict__ cnt, int32_t* out, int32_t* count) {
    __shared__ int red[32], wsum[32];
    int64_t base = counts_before(cnt, blockIdx.x, red);
    if (blockIdx.x == gridDim.x - 1) {
        const int64_t own = (threadIdx.x == 0) ? (int64_t)cnt[blockIdx.x] : 0;
        if (threadIdx.x == 0) *count = (int32_t)(base + own);
    }
    const int lid = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    for (int64_t b0 = lo; b0 < hi; b0 += blockDim.x) {
        const int64_t i = b0 + threadIdx.x;
        const bool f = i < hi && flags[i] != 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        __syncthreads();                                    // the previous step read wsum
        if (lid == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        int64_t before = base;
        int t = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < wid) before += wsum[w];
            t += wsum[w];
        }
        if (f) out[before + __popc(bal & ((1u << lid) - 1u))] = (int32_t)i;
        base += t;
    }
}

// The order-preserving compaction of the flags set; cnt: kCompactBlocks
// entries of scratch.
static int32_t compact_flags(const int32_t* flags, int64_t n, int32_t* out, int32_t* count,
                             unsigned* cnt, cudaStream_t s) {
    const int nb = compact_blocks(n);
    const int64_t chunk = (n + nb - 1) / nb;
    flags_count_kernel<<<nb, 1024, 0, s>>>(flags, n, chunk, cnt);
    flags_write_kernel<<<nb, 1024, 0, s>>>(flags, n, chunk, cnt, out, count);
    note_launches(2);
    return last_error();
}

// ---- gathers, centring, labels, netsim -------------------------------------------
__global__ void gather_rows_kernel(const float* __restrict__ X, int64_t ldx, int d,
                                   const int32_t* __restrict__ rows, int64_t m, float* out) {
    for (int64_t r = blockIdx.x; r < m; r += gridDim.x) {
        const float* src = X + (int64_t)rows[r] * ldx;
        for (int j = threadIdx.x; j < d; j += blockDim.x) out[r * d + j] = src[j];
    }
}

// bf16 of (x - mean) for the listed rows (or rows 0..m-1), zero padded to
// [mpad x dpad]; optional fp32 squared norms of the rounded rows.
__global__ void centre_bf16_kernel(const float* __restrict__ X, int64_t ldx, int d,
                                   const int32_t* __restrict__ rows, int64_t m, int64_t mpad,
                                   int dpad, const float* __restrict__ mean, __nv_bfloat16* out,
                                   float* nrm) {
    const int warps = blockDim.x >> 5, lid = threadIdx.x & 31;
    for (int64_t r = blockIdx.x * (int64_t)warps + (threadIdx.x >> 5); r < mpad;
         r += (int64_t)gridDim.x * warps) {
        float acc = 0.f;
        const int64_t src_row = (r < m) ? (rows ? rows[r] : r) : -1;
        for (int j = lid; j < dpad; j += 32) {
            float v = 0.f;
            if (src_row >= 0 && j < d) v = X[src_row * ldx + j] - mean[j];
            const __nv_bfloat16 b = __float2bfloat16_rn(v);
            out[r * dpad + j] = b;
            const float bv = __bfloat162float(b);
            acc = fmaf(bv, bv, acc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (nrm && lid == 0) nrm[r] = acc;
    }
}

// Exemplars of the landmark problem: E = {j : idx_L(j) == j}, as landmark
// positions in ascending order, and their point indices.
__global__ void landmark_exemplars_kernel(const int32_t* __restrict__ idxL, int64_t L,
                                          const int32_t* __restrict__ lm, int32_t* epts,
                                          int32_t* count) {
    __shared__ int wsum[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int lid = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t lo = 0; lo < L; lo += blockDim.x) {
        const int64_t j = lo + threadIdx.x;
        const bool f = j < L && idxL[j] == (int32_t)j;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lid == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        int before = 0;
        for (int w = 0; w < wid; ++w) before += wsum[w];
        if (f) epts[base + before + __popc(bal & ((1u << lid) - 1u))] = lm[j];
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < nw; ++w) t += wsum[w];
            base += t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base;
}

__global__ void labels_kernel(const int32_t* __restrict__ arg, int64_t n,
                              const int32_t* __restrict__ epts, int32_t* idx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        idx[i] = epts[arg[i]];
}

__global__ void exemplars_keep_self_kernel(const int32_t* __restrict__ epts, int c, int32_t* idx) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < c) idx[epts[j]] = epts[j];
}

// dp[i] = -|x_i - x_idx(i)|^2 in float64 (0 for exemplars), one warp per row.
__global__ void lap_dpsim_kernel(const float* __restrict__ X, int64_t ldx, int d, int64_t n,
                                 const int32_t* __restrict__ idx, double* dp) {
    const int warps = blockDim.x >> 5, lid = threadIdx.x & 31;
    for (int64_t i = blockIdx.x * (int64_t)warps + (threadIdx.x >> 5); i < n;
         i += (int64_t)gridDim.x * warps) {
        const int64_t c = idx[i];
        double s = 0.0;
        if (c != i)
            for (int j = lid; j < d; j += 32) {
                const double t = (double)X[i * ldx + j] - (double)X[c * ldx + j];
                s += t * t;
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lid == 0) dp[i] = -s;
    }
}

// Fixed-order float64 sum (one block).
__global__ void sum_f64_kernel(const double* __restrict__ v, int64_t n, double* out) {
    __shared__ double sh[1024];
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t lo = threadIdx.x * per, hi = (lo + per < n) ? lo + per : n;
    double x = 0.0;
    for (int64_t i = lo; i < hi; ++i) x += v[i];
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// ---- Steps 2-4 of the full algorithm ------------------------------------------------
// flags[rows[j]] = 1
__global__ void flag_rows_kernel(const int32_t* __restrict__ rows, int64_t m, int32_t* flags) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
         j += (int64_t)gridDim.x * blockDim.x)
        flags[rows[j]] = 1;
}

// slot[j] = rank of landmark position j among the exemplar positions
// (idxL[j] == j), ascending -- the order landmark_exemplars_kernel lists them.
__global__ void exemplar_slots_kernel(const int32_t* __restrict__ idxL, int64_t L, int32_t* slot) {
    __shared__ int wsum[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int lid = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t lo = 0; lo < L; lo += blockDim.x) {
        const int64_t j = lo + threadIdx.x;
        const bool f = j < L && idxL[j] == (int32_t)j;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lid == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        int before = 0;
        for (int w = 0; w < wid; ++w) before += wsum[w];
        if (f) slot[j] = base + before + __popc(bal & ((1u << lid) - 1u));
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < nw; ++w) t += wsum[w];
            base += t;
        }
        __syncthreads();
    }
}

// max_distance of each class (bit pattern of a float >= 0, so unsigned max
// is float max): the largest -s(i, e) over the landmarks i of the class of e.
__global__ void max_distance_kernel(const float* __restrict__ SL, int64_t ldL,
                                    const int32_t* __restrict__ idxL, const int32_t* __restrict__ slot,
                                    int64_t L, unsigned* maxd) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= L) return;
    const int32_t e = idxL[i];
    const float d = (i == e) ? 0.f : fmaxf(0.f, -SL[i * ldL + e]);
    atomicMax(&maxd[slot[e]], __float_as_uint(d));
}

// Step 2's gate: point i stays unassigned unless it is a landmark or its
// squared distance to its nearest exemplar, |x_i|^2 - best_i on the rounded
// centred points, is below that class's max_distance.  Assigned points get
// their level.
__global__ void gate_kernel(int64_t nl, const int32_t* __restrict__ arg,
                            const float* __restrict__ best, const float* __restrict__ xnrm,
                            const unsigned* __restrict__ maxd, const int32_t* __restrict__ is_lm,
                            const int32_t* __restrict__ ids, int32_t level, int32_t* un,
                            int32_t* level_of) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool ok = is_lm[i] || (xnrm[i] - best[i]) < __uint_as_float(maxd[arg[i]]);
        un[i] = ok ? 0 : 1;
        if (ok && level_of) level_of[ids ? ids[i] : i] = level;
    }
}

// out[j] = ids[local[j]] (ids == NULL: the identity); level_of of those set.
__global__ void map_ids_kernel(const int32_t* __restrict__ local, int64_t m,
                               const int32_t* __restrict__ ids, int32_t* out, int32_t level,
                               int32_t* level_of) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = ids ? ids[local[j]] : local[j];
        out[j] = g;
        if (level_of) level_of[g] = level;
    }
}

__global__ void set_level_kernel(const int32_t* __restrict__ ids, int64_t m, int32_t level,
                                 int32_t* level_of) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
         j += (int64_t)gridDim.x * blockDim.x)
        level_of[ids[j]] = level;
}

__global__ void fill_i32_kernel(int32_t* p, int64_t n, int32_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// ---- Step 4's refinement: a local search on net similarity -------------------------------
// Removal costs are summed in fixed point (units of 2^-20), class sums of the
// features in 64-bit fixed point (units of 2^-scale), so every sum is exact
// integer arithmetic whatever order the atomics land in: the refinement is
// bitwise reproducible.
constexpr double kDeltaUnit = 1048576.0;   // 2^20

// Largest |x| over the n x d features (float bits of non-negative values
// order like unsigned integers).
__global__ void absmax_kernel(const float* __restrict__ X, int64_t n, int d, int64_t ldx, unsigned* out) {
    unsigned m = 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * d;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / d;
        const int j = (int)(t - i * d);
        m = max(m, __float_as_uint(fabsf(X[i * ldx + j])));
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// delta[j1(i)] += d(i, j2) - d(i, j1) = score1 - score2 (scores 2x.e - |e|^2
// of the rounded centred points); a class with a point that has no second
// centre (one centre in all) can never be dropped.
__global__ void refine_costs_kernel(int64_t n, const int32_t* __restrict__ j1, const float* __restrict__ s1,
                                    const int32_t* __restrict__ j2, const float* __restrict__ s2,
                                    unsigned long long* delta, int32_t* nosecond) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int a = j1[i];
        if (j2[i] < 0) {
            nosecond[a] = 1;
            continue;
        }
        const double diff = (double)s1[i] - (double)s2[i];
        atomicAdd(&delta[a], (unsigned long long)llrint(diff * kDeltaUnit));
    }
}

// cand[j]: dropping centre j raises netsim (its removal cost is below -p).
__global__ void refine_candidates_kernel(int c, const unsigned long long* __restrict__ delta,
                                         const int32_t* __restrict__ nosecond, double thr, int32_t* cand) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < c) cand[j] = (!nosecond[j] && (double)delta[j] < thr) ? 1 : 0;
}

// Two candidates conflict when a point has one as nearest and the other as
// second-nearest centre; the one of larger (cost, position) is kept.
__global__ void refine_block_kernel(int64_t n, const int32_t* __restrict__ j1, const int32_t* __restrict__ j2,
                                    const int32_t* __restrict__ cand,
                                    const unsigned long long* __restrict__ delta, int32_t* blocked) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int a = j1[i], b = j2[i];
        if (b < 0 || !cand[a] || !cand[b]) continue;
        const bool a_larger = delta[a] > delta[b] || (delta[a] == delta[b] && a > b);
        blocked[a_larger ? a : b] = 1;
    }
}

// Class of every point once the unblocked candidates are dropped: the
// members of a dropped class move to their second-nearest centre (which,
// the dropped set being independent, stays).
__global__ void refine_classes_kernel(int64_t n, const int32_t* __restrict__ j1, const int32_t* __restrict__ j2,
                                      const int32_t* __restrict__ cand, const int32_t* __restrict__ blocked,
                                      int32_t* cls, int32_t* counts) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int a = j1[i];
        const int k = (cand[a] && !blocked[a]) ? j2[i] : a;
        cls[i] = k;
        atomicAdd(&counts[k], 1);
    }
}

// sums[cls(i)] += x_i in fixed point (one warp per point).
__global__ void class_sum_kernel(const float* __restrict__ X, int64_t ldx, int d, int64_t n,
                                 const int32_t* __restrict__ cls, double scale, unsigned long long* sums) {
    const int warps = blockDim.x >> 5, lid = threadIdx.x & 31;
    for (int64_t i = blockIdx.x * (int64_t)warps + (threadIdx.x >> 5); i < n; i += (int64_t)gridDim.x * warps) {
        unsigned long long* row = sums + (int64_t)cls[i] * d;
        for (int j = lid; j < d; j += 32)
            atomicAdd(row + j, (unsigned long long)llrint((double)X[i * ldx + j] * scale));
    }
}

__global__ void class_mean_kernel(int c, int d, const unsigned long long* __restrict__ sums,
                                  const int32_t* __restrict__ counts, double inv_scale, double* mu) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)c * d;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / d);
        mu[t] = counts[j] ? (double)(long long)sums[t] * inv_scale / (double)counts[j] : 0.0;
    }
}

// dist[i] = |x_i - mean of its class|^2 in float64 (one warp per point, a
// fixed butterfly); mind[class] = the smallest, as float64 bits.
__global__ void class_dist_kernel(const float* __restrict__ X, int64_t ldx, int d, int64_t n,
                                  const int32_t* __restrict__ cls, const double* __restrict__ mu, double* dist,
                                  unsigned long long* mind) {
    const int warps = blockDim.x >> 5, lid = threadIdx.x & 31;
    for (int64_t i = blockIdx.x * (int64_t)warps + (threadIdx.x >> 5); i < n; i += (int64_t)gridDim.x * warps) {
        const int k = cls[i];
        const double* m = mu + (int64_t)k * d;
        double s = 0.0;
        for (int j = lid; j < d; j += 32) {
            const double t = (double)X[i * ldx + j] - m[j];
            s += t * t;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lid == 0) {
            dist[i] = s;
            atomicMin(&mind[k], (unsigned long long)__double_as_longlong(s));
        }
    }
}

// medoid[class] = the lowest point index attaining the class's smallest distance.
__global__ void class_argmin_kernel(int64_t n, const int32_t* __restrict__ cls, const double* __restrict__ dist,
                                    const unsigned long long* __restrict__ mind, int32_t* medoid) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int k = cls[i];
        if ((unsigned long long)__double_as_longlong(dist[i]) == mind[k]) atomicMin(&medoid[k], (int32_t)i);
    }
}

// ---- workspace ------------------------------------------------------------------------
struct LapWs {
    uint64_t* keys;
    KSelect* ks;
    unsigned* hist;
    int32_t* lm;
    float* XL;
    float *SL, *RL, *AL;
    int32_t* idxL;
    void* sub_ws;
    size_t sub_bytes;
    int32_t* epts;
    int32_t* ecount;
    double* part;
    float* mean;
    __nv_bfloat16* Xb;
    __nv_bfloat16* Eb;
    float* enrm;
    int32_t* arg;
    double* dp;
    double* sums;
    int32_t* err;
};

static int64_t ld32(int64_t n) { return (n + 31) / 32 * 32; }

static size_t carve_lap(void* ws, int64_t n, int64_t d, int64_t L, LapWs* w) {
    const int dpad = (int)((d + 63) / 64 * 64);
    const int64_t ldL = ld32(L);
    const size_t sub = std::max({ap_similarity_workspace_size(L, d), ap_iterate_workspace_size(L, ldL),
                                 exemplars_ws_bytes(L)});
    const int64_t npad = (n + 127) / 128 * 128;
    const int64_t cpad = (L + 255) / 256 * 256;        // at most L exemplars
    Carver c(ws);
    w->keys = c.take<uint64_t>(n);
    w->ks = c.take<KSelect>(1);
    w->hist = c.take<unsigned>(256 + 2 * kCompactBlocks);   // radix bins, then compaction counts
    w->lm = c.take<int32_t>(L);
    w->XL = c.take<float>((size_t)L * d);
    w->SL = c.take<float>((size_t)L * ldL);
    w->RL = c.take<float>((size_t)L * ldL);
    w->AL = c.take<float>((size_t)L * ldL);
    w->idxL = c.take<int32_t>(L);
    w->sub_ws = c.take<char>(sub);
    w->sub_bytes = sub;
    w->epts = c.take<int32_t>(L);
    w->ecount = c.take<int32_t>(1);
    w->part = c.take<double>(column_mean_part_doubles(n, (int)d));
    w->mean = c.take<float>(d);
    w->Xb = c.take<__nv_bfloat16>((size_t)npad * dpad);
    w->Eb = c.take<__nv_bfloat16>((size_t)cpad * dpad);
    w->enrm = c.take<float>(cpad);
    w->arg = c.take<int32_t>(n);
    w->dp = c.take<double>(n);
    w->sums = c.take<double>(2);
    w->err = c.take<int32_t>(1);
    return c.used;
}

static int32_t select_smallest(const uint64_t* keys, int64_t n, int64_t L, KSelect* ks,
                               unsigned* hist, int32_t* out, cudaStream_t s) {
    kselect_init_kernel<<<1, 256, 0, s>>>(ks, (uint64_t)(L - 1), hist);
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 2048);
    for (int p = 0; p < 8; ++p) {
        kselect_hist_kernel<<<grid, 256, 0, s>>>(keys, n, ks, hist);
        kselect_scan_kernel<<<1, 32, 0, s>>>(ks, hist);
    }
    const int nb = compact_blocks(n);
    const int64_t chunk = (n + nb - 1) / nb;
    kselect_count_kernel<<<nb, 1024, 0, s>>>(keys, n, chunk, ks, hist + 256);
    kselect_write_kernel<<<nb, 1024, 0, s>>>(keys, n, chunk, ks, L, hist + 256, out);
    note_launches(19);
    return last_error();
}

}  // namespace apgb

using namespace apgb;

APGB_API size_t lap_run_workspace_size(int64_t n, int64_t d, int64_t n_landmarks) {
    if (n < 2 || d < 1 || n_landmarks < 2 || n_landmarks > n || n > INT_MAX / 2 || d > 65536)
        return 0;
    LapWs w;
    return carve_lap(nullptr, n, d, n_landmarks, &w);
}

APGB_API int32_t lap_run(const float* X, int64_t n, int64_t d, int64_t ldx, int64_t L,
                         int32_t mode, const float* score, const int32_t* landmarks,
                         uint64_t seed, int32_t precision, const ap_params* params, int32_t* idx,
                         int32_t* landmarks_out, lap_result* out, void* ws, size_t ws_bytes,
                         void* stream) {
    if (!X || !idx || !out || !params || n < 2 || d < 1 || ldx < d || L < 2 || L > n ||
        n > INT_MAX / 2 || d > 65536)
        return AP_ERR_INVALID_ARG;
    if (mode == AP_LANDMARK_SCORE && !score) return AP_ERR_INVALID_ARG;
    if (mode == AP_LANDMARK_GIVEN && !landmarks) return AP_ERR_INVALID_ARG;
    if (mode != AP_LANDMARK_UNIFORM && mode != AP_LANDMARK_SCORE && mode != AP_LANDMARK_GIVEN)
        return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LapWs w;
    AP_TRY(check_ws(ws, ws_bytes, carve_lap(nullptr, n, d, L, &w)));
    carve_lap(ws, n, d, L, &w);
    const int di = (int)d;
    const int dpad = (di + 63) / 64 * 64;
    const int64_t ldL = ld32(L);

    cudaEvent_t ev[5];
    for (auto& e : ev) AP_CUDA_TRY(cudaEventCreate(&e));
    struct Guard {
        cudaEvent_t* e;
        ~Guard() { for (int i = 0; i < 5; ++i) cudaEventDestroy(e[i]); }
    } guard{ev};
    AP_CUDA_TRY(cudaEventRecord(ev[0], s));

    // ---- Step 1: landmarks ----
    const int kgrid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    if (mode == AP_LANDMARK_GIVEN) {
        AP_CUDA_TRY(cudaMemcpyAsync(w.lm, landmarks, sizeof(int32_t) * L, cudaMemcpyDeviceToDevice, s));
    } else {
        if (mode == AP_LANDMARK_UNIFORM) keys_uniform_kernel<<<kgrid, 256, 0, s>>>(seed, n, w.keys);
        else keys_score_kernel<<<kgrid, 256, 0, s>>>(score, n, w.keys);
        note_launches(1);
        AP_TRY(select_smallest(w.keys, n, L, w.ks, w.hist, w.lm, s));
    }
    if (landmarks_out)
        AP_CUDA_TRY(cudaMemcpyAsync(landmarks_out, w.lm, sizeof(int32_t) * L, cudaMemcpyDeviceToDevice, s));
    gather_rows_kernel<<<(int)std::min<int64_t>(L, 65535), 128, 0, s>>>(X, ldx, di, w.lm, L, w.XL);
    note_launches(1);
    AP_TRY(last_error());
    AP_CUDA_TRY(cudaEventRecord(ev[1], s));

    // ---- Step 1: Algorithm 1 on the landmarks ----
    float pref = 0.f;
    AP_TRY(ap_similarity(w.XL, L, d, d, w.SL, ldL, precision, AP_PREF_MEDIAN, nullptr, 0.0, 0,
                         &pref, w.sub_ws, w.sub_bytes, stream));
    AP_CUDA_TRY(cudaMemset2DAsync(w.RL, ldL * sizeof(float), 0, L * sizeof(float), L, s));
    AP_CUDA_TRY(cudaMemset2DAsync(w.AL, ldL * sizeof(float), 0, L * sizeof(float), L, s));
    ap_result lr;
    const int32_t st_it = ap_iterate(w.SL, w.RL, w.AL, L, ldL, params, nullptr, &lr, w.sub_ws,
                                     w.sub_bytes, stream);
    if (st_it < 0) return st_it;
    const int32_t li = lr.iters, lc = lr.converged;
    const int32_t st_ex = exemplars_impl(w.SL, w.RL, w.AL, L, ldL, w.idxL, &lr, w.sub_ws,
                                         w.sub_bytes, s);
    if (st_ex < 0) return st_ex;
    lr.iters = li;
    lr.converged = lc;
    AP_CUDA_TRY(cudaEventRecord(ev[2], s));
    *out = lap_result{};
    out->n_landmarks = (int32_t)L;
    out->landmark = lr;
    out->pref = pref;
    if (st_ex == AP_NO_EXEMPLARS) {
        AP_CUDA_TRY(cudaMemsetAsync(idx, 0xFF, sizeof(int32_t) * n, s));
        AP_CUDA_TRY(cudaStreamSynchronize(s));
        out->n_exemplars = 0;
        out->dpsim = out->expref = out->netsim = NAN;
        return AP_NO_EXEMPLARS;
    }

    // ---- Step 2: nearest exemplar for every point (tensor cores) ----
    landmark_exemplars_kernel<<<1, 1024, 0, s>>>(w.idxL, L, w.lm, w.epts, w.ecount);
    int32_t c = 0;
    AP_CUDA_TRY(cudaMemcpyAsync(&c, w.ecount, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    AP_TRY(column_means(X, n, di, ldx, w.part, w.mean, s));
    const int64_t npad = (n + 127) / 128 * 128;
    const int64_t cpad = ((int64_t)c + 255) / 256 * 256;
    centre_bf16_kernel<<<(int)std::min<int64_t>((npad + 7) / 8, 65535), 256, 0, s>>>(
        X, ldx, di, nullptr, n, npad, dpad, w.mean, w.Xb, nullptr);
    centre_bf16_kernel<<<(int)std::min<int64_t>((cpad + 7) / 8, 65535), 256, 0, s>>>(
        X, ldx, di, w.epts, c, cpad, dpad, w.mean, w.Eb, w.enrm);
    AP_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int32_t), s));
    note_launches(3);
    AP_TRY(last_error());
    AP_TRY(tc_assign_argmax(w.Xb, (int)n, w.Eb, c, w.enrm, dpad, w.arg, nullptr, w.err, s));
    const int lgrid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    labels_kernel<<<lgrid, 256, 0, s>>>(w.arg, n, w.epts, idx);
    exemplars_keep_self_kernel<<<(c + 255) / 256, 256, 0, s>>>(w.epts, c, idx);
    AP_CUDA_TRY(cudaEventRecord(ev[3], s));
    lap_dpsim_kernel<<<(int)std::min<int64_t>((n + 7) / 8, 65535), 256, 0, s>>>(X, ldx, di, n, idx,
                                                                                   w.dp);
    sum_f64_kernel<<<1, 1024, 0, s>>>(w.dp, n, w.sums);
    note_launches(4);
    AP_TRY(last_error());
    AP_CUDA_TRY(cudaEventRecord(ev[4], s));
    double dps = 0.0;
    int32_t err = 0;
    AP_CUDA_TRY(cudaMemcpyAsync(&dps, w.sums, sizeof(double), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaMemcpyAsync(&err, w.err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    if (err) return AP_ERR_TIMEOUT;
    float ms[4];
    for (int i = 0; i < 4; ++i) AP_CUDA_TRY(cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]));
    out->select_ms = ms[0];
    out->landmark_ms = ms[1];
    out->assign_ms = ms[2];
    out->netsim_ms = ms[3];
    out->n_exemplars = c;
    out->dpsim = dps;
    out->expref = (double)pref * c;
    out->netsim = out->dpsim + out->expref;
    return (params->conv_iter > 0 && !lc) ? AP_NOT_CONVERGED : AP_OK;
}

// ---- Algorithm 3 Step 2 alone: nearest centre of every point --------------------------
namespace apgb {

struct AssignWs {
    double* part;
    float* mean;
    __nv_bfloat16* Xb;
    __nv_bfloat16* Eb;
    float* enrm;
    int32_t* arg;
    int32_t* err;
};

static size_t carve_assign(void* ws, int64_t n, int64_t d, int64_t c, AssignWs* w) {
    const int dpad = (int)((d + 63) / 64 * 64);
    const int64_t npad = (n + 127) / 128 * 128;
    const int64_t cpad = (c + 255) / 256 * 256;
    Carver cv(ws);
    w->part = cv.take<double>(column_mean_part_doubles(n, (int)d));
    w->mean = cv.take<float>(d);
    w->Xb = cv.take<__nv_bfloat16>((size_t)npad * dpad);
    w->Eb = cv.take<__nv_bfloat16>((size_t)cpad * dpad);
    w->enrm = cv.take<float>(cpad);
    w->arg = cv.take<int32_t>(n);
    w->err = cv.take<int32_t>(1);
    return cv.used;
}

}  // namespace apgb

APGB_API size_t lap_assign_workspace_size(int64_t n, int64_t d, int64_t c) {
    if (n < 1 || d < 1 || c < 1 || c > n || n > INT_MAX / 2 || d > 65536) return 0;
    AssignWs w;
    return carve_assign(nullptr, n, d, c, &w);
}

APGB_API int32_t lap_assign(const float* X, int64_t n, int64_t d, int64_t ldx, const int32_t* centres,
                            int64_t c, int32_t* idx, float* best, void* ws, size_t ws_bytes,
                            void* stream) {
    if (!X || !centres || !idx || ldx < d || !lap_assign_workspace_size(n, d, c))
        return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    AssignWs w;
    AP_TRY(check_ws(ws, ws_bytes, carve_assign(nullptr, n, d, c, &w)));
    carve_assign(ws, n, d, c, &w);
    const int di = (int)d, dpad = (di + 63) / 64 * 64;
    const int64_t npad = (n + 127) / 128 * 128, cpad = (c + 255) / 256 * 256;
    AP_TRY(column_means(X, n, di, ldx, w.part, w.mean, s));
    centre_bf16_kernel<<<(int)std::min<int64_t>((npad + 7) / 8, 65535), 256, 0, s>>>(
        X, ldx, di, nullptr, n, npad, dpad, w.mean, w.Xb, nullptr);
    centre_bf16_kernel<<<(int)std::min<int64_t>((cpad + 7) / 8, 65535), 256, 0, s>>>(
        X, ldx, di, centres, c, cpad, dpad, w.mean, w.Eb, w.enrm);
    AP_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int32_t), s));
    note_launches(2);
    AP_TRY(last_error());
    AP_TRY(tc_assign_argmax(w.Xb, (int)n, w.Eb, (int)c, w.enrm, dpad, w.arg, best, w.err, s));
    const int lgrid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    labels_kernel<<<lgrid, 256, 0, s>>>(w.arg, n, centres, idx);
    exemplars_keep_self_kernel<<<(int)((c + 255) / 256), 256, 0, s>>>(centres, (int)c, idx);
    note_launches(2);
    AP_TRY(last_error());
    int32_t err = 0;
    AP_CUDA_TRY(cudaMemcpyAsync(&err, w.err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    return err ? AP_ERR_TIMEOUT : AP_OK;
}

// ---- Algorithm 3, Steps 1-4 --------------------------------------------------------------
namespace apgb {

struct LapFullWs {
    LapWs lap;                  // one level's Steps 1-2 (sized for n points)
    float* Xn[2];               // features of the points left, compacted (n x d each)
    int32_t* ids[2];            // their indices in X
    int32_t *is_lm, *un, *list, *cnt, *slot;
    unsigned* maxd;
    float *best, *xnrm;
    int32_t* E;                 // merged exemplar set (indices in X)
    __nv_bfloat16* Eb;
    float* enrm;
    float *Sm, *Rm, *Am;        // Step 3's Algorithm 1 on at most m0 points
    int32_t* idxm;
    void* sub;
    size_t sub_bytes;
    int64_t emax;
    // Step 4's refinement
    int32_t *j2, *cls, *nosecond, *cand, *blocked, *counts, *medoid;
    float *s1, *s2;
    double *dist, *mu;
    unsigned long long *delta, *sums, *mind;
    unsigned* absmax;
};

static size_t carve_lap_full(void* ws, int64_t n, int64_t d, int64_t L, int64_t m0,
                             int32_t max_levels, LapFullWs* w) {
    const int dpad = (int)((d + 63) / 64 * 64);
    const int64_t npad = (n + 127) / 128 * 128;
    const int64_t emax = std::min<int64_t>(n, L * max_levels + m0);
    const int64_t epad = (emax + 255) / 256 * 256;
    const int64_t ldm = ld32(m0);
    const size_t sub = std::max({ap_similarity_workspace_size(m0, d), ap_iterate_workspace_size(m0, ldm),
                                 exemplars_ws_bytes(m0)});
    LapWs tmp;
    const size_t lap_bytes = carve_lap(nullptr, n, d, L, &tmp);
    Carver c(ws);
    char* lap_base = c.take<char>(lap_bytes);
    if (ws) carve_lap(lap_base, n, d, L, &w->lap);
    for (int b = 0; b < 2; ++b) w->Xn[b] = c.take<float>((size_t)n * d);
    for (int b = 0; b < 2; ++b) w->ids[b] = c.take<int32_t>(n);
    w->is_lm = c.take<int32_t>(n);
    w->un = c.take<int32_t>(n);
    w->list = c.take<int32_t>(n);
    w->cnt = c.take<int32_t>(1);
    w->slot = c.take<int32_t>(L);
    w->maxd = c.take<unsigned>(L);
    w->best = c.take<float>(n);
    w->xnrm = c.take<float>(npad);
    w->E = c.take<int32_t>(emax);
    w->Eb = c.take<__nv_bfloat16>((size_t)epad * dpad);
    w->enrm = c.take<float>(epad);
    w->Sm = c.take<float>((size_t)m0 * ldm);
    w->Rm = c.take<float>((size_t)m0 * ldm);
    w->Am = c.take<float>((size_t)m0 * ldm);
    w->idxm = c.take<int32_t>(m0);
    w->sub = c.take<char>(sub);
    w->sub_bytes = sub;
    w->emax = emax;
    w->j2 = c.take<int32_t>(n);
    w->cls = c.take<int32_t>(n);
    w->s1 = c.take<float>(n);
    w->s2 = c.take<float>(n);
    w->dist = c.take<double>(n);
    w->nosecond = c.take<int32_t>(emax);
    w->cand = c.take<int32_t>(emax);
    w->blocked = c.take<int32_t>(emax);
    w->counts = c.take<int32_t>(emax);
    w->medoid = c.take<int32_t>(emax);
    w->delta = c.take<unsigned long long>(emax);
    w->mind = c.take<unsigned long long>(emax);
    w->sums = c.take<unsigned long long>((size_t)emax * d);
    w->mu = c.take<double>((size_t)emax * d);
    w->absmax = c.take<unsigned>(1);
    return (lap_bytes && sub) ? c.used : 0;
}

static int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

// Algorithm 1 on the landmarks of one level: S (median preference the first
// time, then the kept preference), iterations, exemplars.  Returns the
// exemplar count (0: none) or a negative status.
static int32_t landmark_ap(const LapWs& w, int64_t L, int64_t d, int32_t precision,
                           const ap_params* params, bool have_p, float* p, cudaStream_t s) {
    const int64_t ldL = ld32(L);
    AP_TRY(ap_similarity(w.XL, L, d, d, w.SL, ldL, precision, have_p ? AP_PREF_SCALAR : AP_PREF_MEDIAN,
                         have_p ? p : nullptr, 0.0, 0, have_p ? nullptr : p, w.sub_ws, w.sub_bytes, s));
    AP_CUDA_TRY(cudaMemset2DAsync(w.RL, ldL * sizeof(float), 0, L * sizeof(float), L, s));
    AP_CUDA_TRY(cudaMemset2DAsync(w.AL, ldL * sizeof(float), 0, L * sizeof(float), L, s));
    ap_result r;
    const int32_t st = ap_iterate(w.SL, w.RL, w.AL, L, ldL, params, nullptr, &r, w.sub_ws, w.sub_bytes, s);
    if (st < 0) return st;
    const int32_t se = exemplars_impl(w.SL, w.RL, w.AL, L, ldL, w.idxL, &r, w.sub_ws, w.sub_bytes, s);
    if (se < 0) return se;
    return se == AP_NO_EXEMPLARS ? 0 : 1;
}

}  // namespace apgb

namespace apgb {

// The buffers of Step 4's refinement (device; n points, emax centres at most).
struct RefineView {
    const __nv_bfloat16* Xb;    // the points' bf16 centred features [npad x dpad]
    const float* mean;          // the mean they were centred on
    int32_t* E;                 // the centre list
    __nv_bfloat16* Eb;
    float* enrm;
    int32_t *j1, *j2, *cls, *nosecond, *cand, *blocked, *counts, *medoid;
    float *s1, *s2;
    double *dist, *mu;
    unsigned long long *delta, *sums, *mind;
    unsigned* absmax;
    int32_t* err;
};

struct RefineStats {
    int32_t rounds = 0, removed = 0, moved = 0;
};

// Step 4's refinement (Algorithm 3): rounds of a local search on net
// similarity over the centres E (v.E, *nE entries, ascending; *hE its host
// copy).  A round: nearest and second-nearest centre of every point
// (tensor-core GEMM, top-2 epilogue); the cost of dropping each centre
// (what its class loses moving to second choices); dropping the
// candidates (cost below -p) that no cheaper conflicting candidate blocks;
// every class's centre moved to the member nearest the class mean.  Stops
// after a round that changes nothing, or after `rounds` rounds.
static int32_t refine_centres(const float* X, int64_t n, int di, int64_t ldx, int dpad, float p, int rounds,
                              const RefineView& w, int64_t* nE, std::vector<int32_t>* hE,
                              RefineStats* st, cudaStream_t s) {
    // fixed-point scale of the class sums: |sum| <= n max|x| must stay below 2^62
    AP_CUDA_TRY(cudaMemsetAsync(w.absmax, 0, sizeof(unsigned), s));
    absmax_kernel<<<(int)std::min<int64_t>((n * di + 255) / 256, 4096), 256, 0, s>>>(X, n, di, ldx, w.absmax);
    note_launches(1);
    AP_TRY(last_error());
    unsigned abits = 0;
    AP_CUDA_TRY(cudaMemcpyAsync(&abits, w.absmax, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    float amax;
    std::memcpy(&amax, &abits, sizeof(float));
    if (!std::isfinite(amax)) return AP_ERR_INVALID_ARG;
    int sc = 32;
    while (sc > 0 && std::ldexp((double)amax * (double)n + 1.0, sc) > 4.0e18) --sc;
    const double scale = std::ldexp(1.0, sc);
    const int grid_n = grid_for(n);
    const int grid_w = (int)std::min<int64_t>((n + 7) / 8, 65535);
    for (int r = 0; r < rounds; ++r) {
        const int c = (int)*nE;
        const int64_t epad = ((int64_t)c + 255) / 256 * 256;
        centre_bf16_kernel<<<(int)std::min<int64_t>((epad + 7) / 8, 65535), 256, 0, s>>>(
            X, ldx, di, w.E, c, epad, dpad, w.mean, w.Eb, w.enrm);
        AP_CUDA_TRY(cudaMemsetAsync(w.nosecond, 0, sizeof(int32_t) * c, s));
        AP_CUDA_TRY(cudaMemsetAsync(w.blocked, 0, sizeof(int32_t) * c, s));
        AP_CUDA_TRY(cudaMemsetAsync(w.counts, 0, sizeof(int32_t) * c, s));
        AP_CUDA_TRY(cudaMemsetAsync(w.delta, 0, sizeof(unsigned long long) * c, s));
        AP_CUDA_TRY(cudaMemsetAsync(w.mind, 0xFF, sizeof(unsigned long long) * c, s));
        AP_CUDA_TRY(cudaMemsetAsync(w.medoid, 0x7F, sizeof(int32_t) * c, s));
        AP_CUDA_TRY(cudaMemsetAsync(w.sums, 0, sizeof(unsigned long long) * c * di, s));
        note_launches(1);
        AP_TRY(last_error());
        AP_TRY(tc_assign_top2(w.Xb, (int)n, w.Eb, c, w.enrm, dpad, w.j1, w.s1, w.j2, w.s2,
                              w.err, s));
        refine_costs_kernel<<<grid_n, 256, 0, s>>>(n, w.j1, w.s1, w.j2, w.s2, w.delta, w.nosecond);
        refine_candidates_kernel<<<(c + 255) / 256, 256, 0, s>>>(c, w.delta, w.nosecond,
                                                                 -(double)p * kDeltaUnit, w.cand);
        refine_block_kernel<<<grid_n, 256, 0, s>>>(n, w.j1, w.j2, w.cand, w.delta, w.blocked);
        refine_classes_kernel<<<grid_n, 256, 0, s>>>(n, w.j1, w.j2, w.cand, w.blocked, w.cls, w.counts);
        class_sum_kernel<<<grid_w, 256, 0, s>>>(X, ldx, di, n, w.cls, scale, w.sums);
        class_mean_kernel<<<(int)std::min<int64_t>(((int64_t)c * di + 255) / 256, 4096), 256, 0, s>>>(
            c, di, w.sums, w.counts, 1.0 / scale, w.mu);
        class_dist_kernel<<<grid_w, 256, 0, s>>>(X, ldx, di, n, w.cls, w.mu, w.dist, w.mind);
        class_argmin_kernel<<<grid_n, 256, 0, s>>>(n, w.cls, w.dist, w.mind, w.medoid);
        note_launches(8);
        AP_TRY(last_error());
        std::vector<int32_t> cand(c), blocked(c), counts(c), medoid(c);
        AP_CUDA_TRY(cudaMemcpyAsync(cand.data(), w.cand, sizeof(int32_t) * c, cudaMemcpyDeviceToHost, s));
        AP_CUDA_TRY(cudaMemcpyAsync(blocked.data(), w.blocked, sizeof(int32_t) * c, cudaMemcpyDeviceToHost, s));
        AP_CUDA_TRY(cudaMemcpyAsync(counts.data(), w.counts, sizeof(int32_t) * c, cudaMemcpyDeviceToHost, s));
        AP_CUDA_TRY(cudaMemcpyAsync(medoid.data(), w.medoid, sizeof(int32_t) * c, cudaMemcpyDeviceToHost, s));
        int32_t err = 0;
        AP_CUDA_TRY(cudaMemcpyAsync(&err, w.err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        AP_CUDA_TRY(cudaStreamSynchronize(s));
        if (err) return AP_ERR_TIMEOUT;
        std::vector<int32_t> next;
        next.reserve(c);
        int removed = 0, moved = 0;
        for (int j = 0; j < c; ++j) {
            if ((cand[j] && !blocked[j]) || counts[j] == 0) {      // dropped (or left empty)
                ++removed;
                continue;
            }
            moved += medoid[j] != (*hE)[j];
            next.push_back(medoid[j]);
        }
        st->rounds = r + 1;
        st->removed += removed;
        st->moved += moved;
        if (removed == 0 && moved == 0) break;
        std::sort(next.begin(), next.end());
        *hE = next;
        *nE = (int64_t)next.size();
        AP_CUDA_TRY(cudaMemcpyAsync(w.E, hE->data(), sizeof(int32_t) * next.size(), cudaMemcpyHostToDevice, s));
    }
    return AP_OK;
}

}  // namespace apgb

APGB_API size_t lap_run_full_workspace_size(int64_t n, int64_t d, int64_t n_landmarks, int64_t m0,
                                            int32_t max_levels) {
    if (n < 2 || d < 1 || n_landmarks < 2 || n_landmarks > n || m0 < 2 || m0 > n ||
        max_levels < 1 || max_levels > AP_LAP_MAX_LEVELS || n > INT_MAX / 2 || d > 65536)
        return 0;
    LapFullWs w;
    return carve_lap_full(nullptr, n, d, n_landmarks, m0, max_levels, &w);
}

APGB_API int32_t lap_run_full(const float* X, int64_t n, int64_t d, int64_t ldx, int64_t L,
                              int64_t m0, uint64_t seed, int32_t precision, const ap_params* params,
                              int32_t max_levels, int32_t refine_rounds, int32_t* idx, int32_t* level_of,
                              lap_full_result* out, void* ws, size_t ws_bytes, void* stream) {
    if (!X || !idx || !out || !params || ldx < d ||
        !lap_run_full_workspace_size(n, d, L, m0, max_levels))
        return AP_ERR_INVALID_ARG;
    if (precision != AP_PREC_FP32 && precision != AP_PREC_BF16) return AP_ERR_INVALID_ARG;
    if (refine_rounds < 0) return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LapFullWs w;
    AP_TRY(check_ws(ws, ws_bytes, carve_lap_full(nullptr, n, d, L, m0, max_levels, &w)));
    carve_lap_full(ws, n, d, L, m0, max_levels, &w);
    const int di = (int)d;
    const int dpad = (di + 63) / 64 * 64;
    cudaEvent_t ev[2];
    for (auto& e : ev) AP_CUDA_TRY(cudaEventCreate(&e));
    struct Guard {
        cudaEvent_t* e;
        ~Guard() { for (int i = 0; i < 2; ++i) cudaEventDestroy(e[i]); }
    } guard{ev};
    AP_CUDA_TRY(cudaEventRecord(ev[0], s));
    *out = lap_full_result{};
    if (level_of) fill_i32_kernel<<<grid_for(n), 256, 0, s>>>(level_of, n, -1);
    AP_CUDA_TRY(cudaMemsetAsync(w.lap.err, 0, sizeof(int32_t), s));
    note_launches(1);

    const float* Xl = X;
    int64_t ldl = ldx, nl = n;
    const int32_t* ids = nullptr;          // level 0: the identity
    int cur = 1;
    int64_t nE = 0;
    float p = 0.f;
    bool have_p = false;
    for (int level = 0;; ++level) {
        if (level > 0 && nl <= m0) {
            // ---- Step 3: Algorithm 1 on the points left ----
            out->base_case = 1;
            int32_t added = 0;
            if (nl == 1) {
                AP_CUDA_TRY(cudaMemcpyAsync(w.E + nE, ids, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
                added = 1;
            } else {
                const int64_t ldm = ld32(nl);
                AP_TRY(ap_similarity(Xl, nl, d, ldl, w.Sm, ldm, precision, AP_PREF_SCALAR, &p, 0.0, 0,
                                     nullptr, w.sub, w.sub_bytes, s));
                AP_CUDA_TRY(cudaMemset2DAsync(w.Rm, ldm * sizeof(float), 0, nl * sizeof(float), nl, s));
                AP_CUDA_TRY(cudaMemset2DAsync(w.Am, ldm * sizeof(float), 0, nl * sizeof(float), nl, s));
                ap_result r;
                const int32_t st = ap_iterate(w.Sm, w.Rm, w.Am, nl, ldm, params, nullptr, &r, w.sub,
                                              w.sub_bytes, s);
                if (st < 0) return st;
                const int32_t se = exemplars_impl(w.Sm, w.Rm, w.Am, nl, ldm, w.idxm, &r, w.sub,
                                                  w.sub_bytes, s);
                if (se < 0) return se;
                if (se != AP_NO_EXEMPLARS) {
                    landmark_exemplars_kernel<<<1, 1024, 0, s>>>(w.idxm, nl, ids, w.E + nE, w.cnt);
                    AP_CUDA_TRY(cudaMemcpyAsync(&added, w.cnt, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
                    AP_CUDA_TRY(cudaStreamSynchronize(s));
                    note_launches(1);
                }
            }
            if (level_of) {                 // every point of Step 3 is settled at this level
                set_level_kernel<<<grid_for(nl), 256, 0, s>>>(ids, nl, level, level_of);
                note_launches(1);
            }
            if (nE + added > w.emax) return AP_ERR_CAPACITY;
            nE += added;
            out->exemplars_at[level] = added;
            break;
        }
        // ---- Step 1: landmarks of this level and Algorithm 1 on them ----
        const int64_t Ll = std::min(L, nl);
        keys_uniform_kernel<<<grid_for(nl), 256, 0, s>>>(seed + (uint64_t)level, nl, w.lap.keys);
        note_launches(1);
        AP_TRY(select_smallest(w.lap.keys, nl, Ll, w.lap.ks, w.lap.hist, w.lap.lm, s));
        gather_rows_kernel<<<(int)std::min<int64_t>(Ll, 65535), 128, 0, s>>>(Xl, ldl, di, w.lap.lm, Ll,
                                                                              w.lap.XL);
        note_launches(1);
        const int32_t got = landmark_ap(w.lap, Ll, d, precision, params, have_p, &p, s);
        if (got < 0) return got;
        have_p = true;
        if (got == 0) {
            if (level == 0) {
                AP_CUDA_TRY(cudaMemsetAsync(idx, 0xFF, sizeof(int32_t) * n, s));
                AP_CUDA_TRY(cudaStreamSynchronize(s));
                out->pref = p;
                out->dpsim = out->expref = out->netsim = NAN;
                return AP_NO_EXEMPLARS;
            }
            break;                          // the points left join their nearest exemplar in Step 4
        }
        out->levels = level + 1;
        // ---- Step 2: max_distance per class, nearest exemplar, the gate ----
        landmark_exemplars_kernel<<<1, 1024, 0, s>>>(w.lap.idxL, Ll, w.lap.lm, w.lap.epts, w.lap.ecount);
        exemplar_slots_kernel<<<1, 1024, 0, s>>>(w.lap.idxL, Ll, w.slot);
        int32_t c = 0;
        AP_CUDA_TRY(cudaMemcpyAsync(&c, w.lap.ecount, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        AP_CUDA_TRY(cudaStreamSynchronize(s));
        AP_CUDA_TRY(cudaMemsetAsync(w.maxd, 0, sizeof(unsigned) * c, s));
        max_distance_kernel<<<(int)((Ll + 255) / 256), 256, 0, s>>>(w.lap.SL, ld32(Ll), w.lap.idxL, w.slot,
                                                                     Ll, w.maxd);
        AP_TRY(column_means(Xl, nl, di, ldl, w.lap.part, w.lap.mean, s));
        const int64_t npad = (nl + 127) / 128 * 128, cpad = ((int64_t)c + 255) / 256 * 256;
        centre_bf16_kernel<<<(int)std::min<int64_t>((npad + 7) / 8, 65535), 256, 0, s>>>(
            Xl, ldl, di, nullptr, nl, npad, dpad, w.lap.mean, w.lap.Xb, w.xnrm);
        centre_bf16_kernel<<<(int)std::min<int64_t>((cpad + 7) / 8, 65535), 256, 0, s>>>(
            Xl, ldl, di, w.lap.epts, c, cpad, dpad, w.lap.mean, w.lap.Eb, w.lap.enrm);
        note_launches(5);
        AP_TRY(last_error());
        AP_TRY(tc_assign_argmax(w.lap.Xb, (int)nl, w.lap.Eb, c, w.lap.enrm, dpad, w.lap.arg, w.best,
                                w.lap.err, s));
        AP_CUDA_TRY(cudaMemsetAsync(w.is_lm, 0, sizeof(int32_t) * nl, s));
        flag_rows_kernel<<<grid_for(Ll), 256, 0, s>>>(w.lap.lm, Ll, w.is_lm);
        gate_kernel<<<grid_for(nl), 256, 0, s>>>(nl, w.lap.arg, w.best, w.xnrm, w.maxd, w.is_lm, ids,
                                                 level, w.un, level_of);
        if (nE + c > w.emax) return AP_ERR_CAPACITY;
        map_ids_kernel<<<grid_for(c), 256, 0, s>>>(w.lap.epts, c, ids, w.E + nE, level, level_of);
        nE += c;
        out->exemplars_at[level] = c;
        note_launches(4);
        AP_TRY(last_error());
        AP_TRY(compact_flags(w.un, nl, w.list, w.cnt, w.lap.hist + 256, s));
        int32_t m = 0;
        AP_CUDA_TRY(cudaMemcpyAsync(&m, w.cnt, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        AP_CUDA_TRY(cudaStreamSynchronize(s));
        out->unassigned[level] = m;
        if (m == 0 || level + 1 >= max_levels) break;
        // ---- Step 3 (recursive case): the points left become the next level ----
        const int nxt = cur ^ 1;
        gather_rows_kernel<<<(int)std::min<int64_t>(m, 65535), 128, 0, s>>>(Xl, ldl, di, w.list, m,
                                                                             w.Xn[nxt]);
        map_ids_kernel<<<grid_for(m), 256, 0, s>>>(w.list, m, ids, w.ids[nxt], 0, nullptr);
        note_launches(2);
        Xl = w.Xn[nxt];
        ldl = d;
        ids = w.ids[nxt];
        nl = m;
        cur = nxt;
    }

    // ---- Step 4: every point to its nearest exemplar of the merged set ----
    std::vector<int32_t> hE(nE);
    AP_CUDA_TRY(cudaMemcpyAsync(hE.data(), w.E, sizeof(int32_t) * nE, cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    std::sort(hE.begin(), hE.end());
    AP_CUDA_TRY(cudaMemcpyAsync(w.E, hE.data(), sizeof(int32_t) * nE, cudaMemcpyHostToDevice, s));
    AP_TRY(column_means(X, n, di, ldx, w.lap.part, w.lap.mean, s));
    const int64_t npad = (n + 127) / 128 * 128;
    centre_bf16_kernel<<<(int)std::min<int64_t>((npad + 7) / 8, 65535), 256, 0, s>>>(
        X, ldx, di, nullptr, n, npad, dpad, w.lap.mean, w.lap.Xb, nullptr);
    note_launches(1);
    if (refine_rounds > 0) {
        RefineView v{w.lap.Xb, w.lap.mean, w.E, w.Eb, w.enrm, w.lap.arg, w.j2, w.cls, w.nosecond, w.cand,
                     w.blocked, w.counts, w.medoid, w.s1, w.s2, w.dist, w.mu, w.delta, w.sums, w.mind,
                     w.absmax, w.lap.err};
        RefineStats rs;
        AP_TRY(refine_centres(X, n, di, ldx, dpad, p, refine_rounds, v, &nE, &hE, &rs, s));
        out->refine_rounds = rs.rounds;
        out->refine_removed = rs.removed;
        out->refine_moved = rs.moved;
    }
    const int64_t epad = (nE + 255) / 256 * 256;
    centre_bf16_kernel<<<(int)std::min<int64_t>((epad + 7) / 8, 65535), 256, 0, s>>>(
        X, ldx, di, w.E, nE, epad, dpad, w.lap.mean, w.Eb, w.enrm);
    note_launches(1);
    AP_TRY(last_error());
    AP_TRY(tc_assign_argmax(w.lap.Xb, (int)n, w.Eb, (int)nE, w.enrm, dpad, w.lap.arg, nullptr,
                            w.lap.err, s));
    labels_kernel<<<grid_for(n), 256, 0, s>>>(w.lap.arg, n, w.E, idx);
    exemplars_keep_self_kernel<<<(int)((nE + 255) / 256), 256, 0, s>>>(w.E, (int)nE, idx);
    lap_dpsim_kernel<<<(int)std::min<int64_t>((n + 7) / 8, 65535), 256, 0, s>>>(X, ldx, di, n, idx,
                                                                                   w.lap.dp);
    sum_f64_kernel<<<1, 1024, 0, s>>>(w.lap.dp, n, w.lap.sums);
    note_launches(4);
    AP_TRY(last_error());
    AP_CUDA_TRY(cudaEventRecord(ev[1], s));
    double dps = 0.0;
    int32_t err = 0;
    AP_CUDA_TRY(cudaMemcpyAsync(&dps, w.lap.sums, sizeof(double), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaMemcpyAsync(&err, w.lap.err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    if (err) return AP_ERR_TIMEOUT;
    AP_CUDA_TRY(cudaEventElapsedTime(&out->ms, ev[0], ev[1]));
    out->pref = p;
    out->n_exemplars = (int32_t)nE;
    out->dpsim = dps;
    out->expref = (double)p * (double)nE;
    out->netsim = out->dpsim + out->expref;
    return AP_OK;
}

// ---- Algorithm 3 Step 4 alone: refinement of a given centre set ----------------------------
namespace apgb {

struct RefineWs {
    double* part;
    float* mean;
    __nv_bfloat16 *Xb, *Eb;
    float* enrm;
    int32_t *E, *j1, *j2, *cls, *nosecond, *cand, *blocked, *counts, *medoid;
    float *s1, *s2;
    double *dist, *mu, *dp, *tot;
    unsigned long long *delta, *sums, *mind;
    unsigned* absmax;
    int32_t* err;
};

static size_t carve_refine(void* ws, int64_t n, int64_t d, int64_t c, RefineWs* w) {
    const int dpad = (int)((d + 63) / 64 * 64);
    const int64_t npad = (n + 127) / 128 * 128, cpad = (c + 255) / 256 * 256;
    Carver cv(ws);
    w->part = cv.take<double>(column_mean_part_doubles(n, (int)d));
    w->mean = cv.take<float>(d);
    w->Xb = cv.take<__nv_bfloat16>((size_t)npad * dpad);
    w->Eb = cv.take<__nv_bfloat16>((size_t)cpad * dpad);
    w->enrm = cv.take<float>(cpad);
    w->E = cv.take<int32_t>(c);
    for (int32_t** q : {&w->j1, &w->j2, &w->cls}) *q = cv.take<int32_t>(n);
    for (int32_t** q : {&w->nosecond, &w->cand, &w->blocked, &w->counts, &w->medoid}) *q = cv.take<int32_t>(c);
    w->s1 = cv.take<float>(n);
    w->s2 = cv.take<float>(n);
    w->dist = cv.take<double>(n);
    w->dp = cv.take<double>(n);
    w->tot = cv.take<double>(1);
    w->mu = cv.take<double>((size_t)c * d);
    w->delta = cv.take<unsigned long long>(c);
    w->mind = cv.take<unsigned long long>(c);
    w->sums = cv.take<unsigned long long>((size_t)c * d);
    w->absmax = cv.take<unsigned>(1);
    w->err = cv.take<int32_t>(1);
    return cv.used;
}

}  // namespace apgb

APGB_API size_t lap_refine_workspace_size(int64_t n, int64_t d, int64_t c) {
    if (n < 1 || d < 1 || c < 1 || c > n || n > INT_MAX / 2 || d > 65536) return 0;
    RefineWs w;
    return carve_refine(nullptr, n, d, c, &w);
}

APGB_API int32_t lap_refine(const float* X, int64_t n, int64_t d, int64_t ldx, const int32_t* centres,
                            int64_t c, float pref, int32_t rounds, int32_t* centres_out, int32_t* idx,
                            lap_refine_result* out, void* ws, size_t ws_bytes, void* stream) {
    if (!X || !centres || !centres_out || !idx || !out || ldx < d || rounds < 0 || !std::isfinite(pref) ||
        !lap_refine_workspace_size(n, d, c))
        return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    RefineWs w;
    AP_TRY(check_ws(ws, ws_bytes, carve_refine(nullptr, n, d, c, &w)));
    carve_refine(ws, n, d, c, &w);
    const int di = (int)d, dpad = (di + 63) / 64 * 64;
    // the centre list, ascending and distinct
    std::vector<int32_t> hE(c);
    AP_CUDA_TRY(cudaMemcpyAsync(hE.data(), centres, sizeof(int32_t) * c, cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    std::sort(hE.begin(), hE.end());
    for (int64_t j = 0; j < c; ++j)
        if (hE[j] < 0 || hE[j] >= n || (j > 0 && hE[j] == hE[j - 1])) return AP_ERR_INVALID_ARG;
    AP_CUDA_TRY(cudaMemcpyAsync(w.E, hE.data(), sizeof(int32_t) * c, cudaMemcpyHostToDevice, s));
    AP_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int32_t), s));
    AP_TRY(column_means(X, n, di, ldx, w.part, w.mean, s));
    const int64_t npad = (n + 127) / 128 * 128;
    centre_bf16_kernel<<<(int)std::min<int64_t>((npad + 7) / 8, 65535), 256, 0, s>>>(
        X, ldx, di, nullptr, n, npad, dpad, w.mean, w.Xb, nullptr);
    note_launches(1);
    AP_TRY(last_error());
    int64_t nE = c;
    RefineStats rs;
    if (rounds > 0) {
        RefineView v{w.Xb, w.mean, w.E, w.Eb, w.enrm, w.j1, w.j2, w.cls, w.nosecond, w.cand, w.blocked,
                     w.counts, w.medoid, w.s1, w.s2, w.dist, w.mu, w.delta, w.sums, w.mind, w.absmax, w.err};
        AP_TRY(refine_centres(X, n, di, ldx, dpad, pref, rounds, v, &nE, &hE, &rs, s));
    }
    // every point to its nearest centre of the final set; centres keep themselves
    const int64_t epad = (nE + 255) / 256 * 256;
    centre_bf16_kernel<<<(int)std::min<int64_t>((epad + 7) / 8, 65535), 256, 0, s>>>(
        X, ldx, di, w.E, nE, epad, dpad, w.mean, w.Eb, w.enrm);
    note_launches(1);
    AP_TRY(last_error());
    AP_TRY(tc_assign_argmax(w.Xb, (int)n, w.Eb, (int)nE, w.enrm, dpad, w.j1, nullptr, w.err, s));
    labels_kernel<<<grid_for(n), 256, 0, s>>>(w.j1, n, w.E, idx);
    exemplars_keep_self_kernel<<<(int)((nE + 255) / 256), 256, 0, s>>>(w.E, (int)nE, idx);
    lap_dpsim_kernel<<<(int)std::min<int64_t>((n + 7) / 8, 65535), 256, 0, s>>>(X, ldx, di, n, idx, w.dp);
    sum_f64_kernel<<<1, 1024, 0, s>>>(w.dp, n, w.tot);
    AP_CUDA_TRY(cudaMemcpyAsync(centres_out, w.E, sizeof(int32_t) * nE, cudaMemcpyDeviceToDevice, s));
    note_launches(4);
    AP_TRY(last_error());
    double dps = 0.0;
    int32_t err = 0;
    AP_CUDA_TRY(cudaMemcpyAsync(&dps, w.tot, sizeof(double), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaMemcpyAsync(&err, w.err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    if (err) return AP_ERR_TIMEOUT;
    *out = lap_refine_result{};
    out->rounds = rs.rounds;
    out->removed = rs.removed;
    out->moved = rs.moved;
    out->n_exemplars = (int32_t)nE;
    out->dpsim = dps;
    out->expref = (double)pref * (double)nE;
    out->netsim = out->dpsim + out->expref;
    return AP_OK;
}
