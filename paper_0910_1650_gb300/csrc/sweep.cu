// ap_iterate: the damped message-passing sweep of Algorithm 1 (Section 2,
// Eq. 2-4) as one fused, memory-bound pass over S, R and A per iteration.
//
// Launch t (t = 1, 2, ...) of `sweep_kernel` does, for every row i:
//   * the availability half of iteration t-1 (skipped for t = 1):
//       a(i,k) = min(0, c(k) - max(0, r(i,k)))   k != i,  c(k) = r(k,k)+colp(k)
//       a(i,i) = colp(i)                                            (Eq. 3, 4)
//     damped in place, plus the decision argmax_k a(i,k)+r(i,k) of iteration
//     t-1, where colp(k) = sum_{i' != k} max(0, r(i',k)) over R_{t-1};
//   * the responsibility half of iteration t (skipped for t = max_iter+1):
//       r(i,k) = s(i,k) - (k == j1 ? m2 : m1)                           (Eq. 2)
//     with (m1, j1, m2) the top-2 of the row a(i,.)+s(i,.) just formed,
//     damped, written to the other R buffer, and folded into per-column
//     partial sums of max(0, r) (and r(i,i) captured).
// So each launch reads S, R, A once and writes R, A once: 20 bytes per matrix
// element, the least any implementation of the iteration can move.
//
// Work layout: a thread-block cluster of C CTAs spans a row; CTA c owns a
// fixed slice of W4 float4 columns, so the column partial sums for its slice
// stay in registers across every row the cluster processes.  The per-row
// top-2 and decision arg-max are reduced inside each CTA (warp shuffles) and
// across the cluster through distributed shared memory.  Clusters stride over
// rows.  A second small kernel sums the per-cluster column partials in a fixed
// order (bitwise reproducible), and updates the device-side stop state.
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>
#include <vector>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace apgb {

struct SweepState {
    int32_t t;           // index of the next sweep launch (1-based)
    int32_t done;
    int32_t stable;      // iterations the exemplar set has been constant
    int32_t iters;       // iterations whose messages are final
    int32_t converged;
    int32_t changes;     // exemplar-flag changes seen by the current launch
    int32_t n_ex;        // exemplars in the current launch's decisions
    int32_t max_iter;
    int32_t conv_iter;
    int32_t final_buf;   // R buffer (0 = caller's R, 1 = workspace) with R_iters
    int32_t nonfinite;   // count of NaN/Inf entries of S
    int32_t pad[5];
};

struct SweepArgs {
    const float* S;
    float*       R0;       // caller's R (buffer 0)
    float*       R1;       // workspace R (buffer 1)
    float*       A;
    int64_t      ld;
    int          n;
    int          n4;       // float4 columns spanning n
    int          w4;       // float4 columns per CTA
    float        lam;
    const float* cvec;     // r(k,k) + colp(k) of R_{t-1}
    const float* colp;     // colp(k) of R_{t-1}
    float*       pcol;     // [clusters][n] partial column sums of R_t
    float*       rkk;      // r(k,k) of R_t
    int32_t*     eflag;    // exemplar flags of the previous decisions
    int32_t*     dec;      // decisions (may be null)
    SweepState*  st;
};

struct Slot {
    float m1, m2, dv;
    int   j1, dj;
    int   pad[3];
};

__device__ __forceinline__ float lane(const float4& v, int e) {
    return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}
__device__ __forceinline__ void set_lane(float4& v, int e, float x) {
    if (e == 0) v.x = x; else if (e == 1) v.y = x; else if (e == 2) v.z = x; else v.w = x;
}

template <int EPT>
__global__ void __launch_bounds__(512) sweep_kernel(SweepArgs a) {
    cg::cluster_group cluster = cg::this_cluster();
    const int csize = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int g = blockIdx.x / csize;
    const int G = gridDim.x / csize;
    const int T = blockDim.x;
    const int tid = threadIdx.x;

    __shared__ Slot xs[2];          // this CTA's partial result, by row parity
    __shared__ Slot warp_part[16];
    __shared__ Slot fin;
    __shared__ int  cnt_changes, cnt_ex;

    SweepState* st = a.st;
    const int t = st->t;
    if (st->done) return;                       // uniform across the grid
    const bool doA = t >= 2;
    const bool doR = t <= st->max_iter;
    const float lam = a.lam, oml = 1.0f - a.lam;
    const float* Rin = ((t - 1) & 1) ? a.R1 : a.R0;
    float* Rout = (t & 1) ? a.R1 : a.R0;

    if (tid == 0) { cnt_changes = 0; cnt_ex = 0; }

    const int f_begin = crank * a.w4;
    const int f_end = min(f_begin + a.w4, a.n4);

    float4 cv[EPT], acc[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        cv[q] = acc[q];
        const int f = f_begin + tid + q * T;
        if (doA && f < f_end) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = 4 * f + e;
                set_lane(cv[q], e, k < a.n ? a.cvec[k] : 0.f);
            }
        }
    }
    __syncthreads();

    int par = 0;
    for (int i = g; i < a.n; i += G, par ^= 1) {
        const float* Srow = a.S + (int64_t)i * a.ld;
        const float* Rrow = Rin + (int64_t)i * a.ld;
        float* Arow = a.A + (int64_t)i * a.ld;
        float4 s4[EPT], r4[EPT], a4[EPT];
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int f = f_begin + tid + q * T;
            if (f < f_end) {
                s4[q] = __ldcs(reinterpret_cast<const float4*>(Srow) + f);
                r4[q] = __ldcs(reinterpret_cast<const float4*>(Rrow) + f);
                a4[q] = __ldcs(reinterpret_cast<const float4*>(Arow) + f);
            }
        }
        const float colp_i = doA ? a.colp[i] : 0.f;

        Top2 tp{-INFINITY, -INFINITY, INT_MAX};
        float dv = -INFINITY;
        int dj = INT_MAX;
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int f = f_begin + tid + q * T;
            if (f < f_end) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int k = 4 * f + e;
                    if (k < a.n) {
                        const float s = lane(s4[q], e), r = lane(r4[q], e);
                        float av = lane(a4[q], e);
                        if (doA) {
                            const float an = (k == i) ? colp_i
                                                      : fminf(0.f, lane(cv[q], e) - fmaxf(0.f, r));
                            av = fmaf(lam, av, oml * an);
                            set_lane(a4[q], e, av);
                            argmax_merge(dv, dj, av + r, k);
                        }
                        top2_push(tp, av + s, k);
                    }
                }
                if (doA) {
                    float4* dst = reinterpret_cast<float4*>(Arow) + f;
                    if (4 * f + 3 < a.n) {
                        __stcs(dst, a4[q]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (4 * f + e < a.n) Arow[4 * f + e] = lane(a4[q], e);
                    }
                }
            }
        }

        // ---- CTA reduction of (top-2, decision arg-max) -----------------
        tp = top2_warp(tp);
        argmax_warp(dv, dj);
        const int wid = tid >> 5, lid = tid & 31;
        if (lid == 0) warp_part[wid] = Slot{tp.m1, tp.m2, dv, tp.j1, dj, {0, 0, 0}};
        __syncthreads();
        if (wid == 0) {
            const int nw = T >> 5;
            Top2 u{-INFINITY, -INFINITY, INT_MAX};
            float uv = -INFINITY;
            int uj = INT_MAX;
            if (lid < nw) {
                const Slot p = warp_part[lid];
                u = Top2{p.m1, p.m2, p.j1};
                uv = p.dv;
                uj = p.dj;
            }
            u = top2_warp(u);
            argmax_warp(uv, uj);
            if (lid == 0) xs[par] = Slot{u.m1, u.m2, uv, u.j1, uj, {0, 0, 0}};
        }
        // ---- cluster reduction through distributed shared memory --------
        if (csize > 1) cluster.sync(); else __syncthreads();
        if (wid == 0) {
            Top2 u{-INFINITY, -INFINITY, INT_MAX};
            float uv = -INFINITY;
            int uj = INT_MAX;
            if (lid < csize) {
                const Slot* rs = csize > 1 ? cluster.map_shared_rank(&xs[par], lid) : &xs[par];
                const Slot p = *rs;
                u = Top2{p.m1, p.m2, p.j1};
                uv = p.dv;
                uj = p.dj;
            }
            u = top2_warp(u);
            argmax_warp(uv, uj);
            if (lid == 0) fin = Slot{u.m1, u.m2, uv, u.j1, uj, {0, 0, 0}};
        }
        __syncthreads();
        const float m1 = fin.m1, m2 = fin.m2;
        const int j1 = fin.j1;

        if (doA && crank == 0 && tid == 0) {
            const int d = fin.dj;
            if (a.dec) a.dec[i] = d;
            const int e = (d == i) ? 1 : 0;
            if (a.eflag[i] != e) ++cnt_changes;
            a.eflag[i] = e;
            cnt_ex += e;
        }

        if (doR) {
            float* Orow = Rout + (int64_t)i * a.ld;
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                const int f = f_begin + tid + q * T;
                if (f < f_end) {
                    float4 o;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int k = 4 * f + e;
                        const float s = lane(s4[q], e), r = lane(r4[q], e);
                        const float m = (k == j1) ? m2 : m1;
                        const float rn = fmaf(lam, r, oml * (s - m));
                        set_lane(o, e, rn);
                        if (k < a.n) {
                            if (k == i) a.rkk[i] = rn;
                            else set_lane(acc[q], e, lane(acc[q], e) + fmaxf(0.f, rn));
                        }
                    }
                    float4* dst = reinterpret_cast<float4*>(Orow) + f;
                    if (4 * f + 3 < a.n) {
                        __stcs(dst, o);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (4 * f + e < a.n) Orow[4 * f + e] = lane(o, e);
                    }
                }
            }
        }
    }

    if (doR) {
        float* P = a.pcol + (int64_t)g * a.n;
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int f = f_begin + tid + q * T;
            if (f < f_end) {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (4 * f + e < a.n) P[4 * f + e] = lane(acc[q], e);
            }
        }
    }
    __syncthreads();
    if (tid == 0 && crank == 0 && doA) {
        atomicAdd(&st->changes, cnt_changes);
        atomicAdd(&st->n_ex, cnt_ex);
    }
    // keep this CTA's shared memory alive until every peer has read it
    if (csize > 1) cluster.sync();
}

// Column sums in a fixed cluster order, then the stop rule (block 0).
__global__ void finalize_kernel(const float* __restrict__ pcol, int G, int n,
                                const float* __restrict__ rkk, float* colp,
                                float* cvec, SweepState* st) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        float s = 0.f;
        for (int g = 0; g < G; ++g) s += pcol[(int64_t)g * n + k];
        colp[k] = s;
        cvec[k] = rkk[k] + s;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (st->done) return;
        const int t = st->t;
        if (t >= 2) {
            const int it = t - 1;
            st->stable = (it == 1 || st->changes != 0) ? 1 : st->stable + 1;
            if (st->conv_iter > 0 && st->stable >= st->conv_iter && st->n_ex > 0) {
                st->done = 1;
                st->converged = 1;
                st->iters = it;
                st->final_buf = it & 1;
            }
        }
        if (!st->done && t == st->max_iter + 1) {
            st->done = 1;
            st->iters = st->max_iter;
            st->final_buf = st->max_iter & 1;
        }
        st->changes = 0;
        st->n_ex = 0;
        st->t = t + 1;
    }
}

__global__ void sweep_init_kernel(SweepState* st, int32_t* eflag, int n,
                                  int max_iter, int conv_iter) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) eflag[k] = 0;
    if (k == 0) {
        SweepState s{};
        s.t = 1;
        s.max_iter = max_iter;
        s.conv_iter = conv_iter;
        *st = s;
    }
}

__global__ void nonfinite_kernel(const float* __restrict__ S, int n, int64_t ld,
                                 int32_t* count) {
    int local = 0;
    for (int i = blockIdx.x; i < n; i += gridDim.x)
        for (int k = threadIdx.x; k < n; k += blockDim.x)
            if (!isfinite(S[(int64_t)i * ld + k])) ++local;
    local = __reduce_add_sync(0xffffffffu, local);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

// ---------------------------------------------------------------------------
// Launch configuration
// ---------------------------------------------------------------------------
struct SweepConfig {
    int C, T, EPT, W4, G;
};

template <int EPT>
static void* sweep_fn() { return (void*)sweep_kernel<EPT>; }

static void* sweep_ptr(int ept) {
    switch (ept) {
        case 1: return sweep_fn<1>();
        case 2: return sweep_fn<2>();
        case 3: return sweep_fn<3>();
        default: return sweep_fn<4>();
    }
}

static int32_t max_clusters(int ept, int C, int T, int* out) {
    void* fn = sweep_ptr(ept);
    if (C > 8) AP_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(T, 1, 1);
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = C;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int num = 0;
    if (cudaOccupancyMaxActiveClusters(&num, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        num = 0;
    }
    *out = num;
    return AP_OK;
}

// Smallest cluster whose slices need at most 2 float4 per thread (<= 512
// threads), else 4; the thread count is trimmed to balance the slice.
static int32_t choose_config(int n, SweepConfig* c) {
    const int n4 = (n + 3) / 4;
    const int clusters[] = {1, 2, 4, 8, 16};
    for (int ept_cap : {2, 4}) {
        for (int C : clusters) {
            if (C > 1 && n4 < 64 * C) break;
            const int w4 = (n4 + C - 1) / C;
            int ept = (w4 + 511) / 512;
            if (ept < 1) ept = 1;
            if (ept > ept_cap) continue;
            if (ept == 3 && ept_cap == 4) ept = 4;
            int T = ((w4 + ept - 1) / ept + 31) / 32 * 32;
            T = std::max(T, 64);
            int num = 0;
            AP_TRY(max_clusters(ept, C, T, &num));
            if (num <= 0) continue;
            c->C = C;
            c->T = T;
            c->EPT = ept;
            c->W4 = w4;
            c->G = std::max(1, std::min(num, n));
            return AP_OK;
        }
    }
    return AP_ERR_UNSUPPORTED;
}

// CUDA events bracketing each sweep launch of one chunk (host-side timing).
struct EventPairs {
    std::vector<cudaEvent_t> start, stop;
    int32_t reserve(int64_t k) {
        start.resize(k, nullptr);
        stop.resize(k, nullptr);
        for (int64_t j = 0; j < k; ++j) {
            if (cudaEventCreate(&start[j]) != cudaSuccess) return AP_ERR_CUDA;
            if (cudaEventCreate(&stop[j]) != cudaSuccess) return AP_ERR_CUDA;
        }
        return AP_OK;
    }
    ~EventPairs() {
        for (auto e : start) if (e) cudaEventDestroy(e);
        for (auto e : stop) if (e) cudaEventDestroy(e);
    }
};

struct SweepWs {
    float* R1;
    float* pcol;
    float* colp;
    float* cvec;
    float* rkk;
    int32_t* eflag;
    SweepState* st;
};

static size_t carve_sweep(void* ws, int64_t n, int64_t ld, int G, SweepWs* w) {
    Carver cv(ws);
    w->R1 = cv.take<float>((size_t)n * ld);
    w->pcol = cv.take<float>((size_t)G * n);
    w->colp = cv.take<float>(n);
    w->cvec = cv.take<float>(n);
    w->rkk = cv.take<float>(n);
    w->eflag = cv.take<int32_t>(n);
    w->st = cv.take<SweepState>(1);
    return cv.used;
}

static int32_t launch_sweep(const SweepConfig& c, const SweepArgs& args, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c.C * c.G, 1, 1);
    cfg.blockDim = dim3(c.T, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = c.C;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    switch (c.EPT) {
        case 1: e = cudaLaunchKernelEx(&cfg, sweep_kernel<1>, args); break;
        case 2: e = cudaLaunchKernelEx(&cfg, sweep_kernel<2>, args); break;
        case 3: e = cudaLaunchKernelEx(&cfg, sweep_kernel<3>, args); break;
        default: e = cudaLaunchKernelEx(&cfg, sweep_kernel<4>, args); break;
    }
    return e == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

int32_t sweep_workspace(int64_t n, int64_t ld, size_t* bytes, SweepConfig* cfg_out) {
    if (n < 1 || n > INT_MAX / 4 || ld < n) return AP_ERR_INVALID_ARG;
    SweepConfig c;
    AP_TRY(choose_config((int)n, &c));
    SweepWs w;
    *bytes = carve_sweep(nullptr, n, ld, c.G, &w);
    if (cfg_out) *cfg_out = c;
    return AP_OK;
}

}  // namespace apgb

using namespace apgb;

APGB_API size_t ap_iterate_workspace_size(int64_t n, int64_t ld) {
    size_t b = 0;
    if (sweep_workspace(n, ld, &b, nullptr) != AP_OK) return 0;
    return b;
}

APGB_API int32_t ap_iterate(const float* S, float* R, float* A, int64_t n, int64_t ld,
                            const ap_params* p, int32_t* decisions, ap_result* out,
                            void* ws, size_t ws_bytes, void* stream) {
    if (!S || !R || !A || !p) return AP_ERR_INVALID_ARG;
    if (n < 2 || ld < n || (ld & 3) || !aligned16(S) || !aligned16(R) || !aligned16(A))
        return AP_ERR_INVALID_ARG;
    if (!(p->damping >= 0.f && p->damping < 1.f) || p->max_iter < 1 || p->conv_iter < 0)
        return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SweepConfig c;
    size_t need = 0;
    AP_TRY(sweep_workspace(n, ld, &need, &c));
    AP_TRY(check_ws(ws, ws_bytes, need));
    SweepWs w;
    carve_sweep(ws, n, ld, c.G, &w);
    const int ni = (int)n;

    sweep_init_kernel<<<(ni + 255) / 256, 256, 0, s>>>(w.st, w.eflag, ni, p->max_iter, p->conv_iter);
    nonfinite_kernel<<<1024, 256, 0, s>>>(S, ni, ld, &w.st->nonfinite);
    note_launches(2);
    AP_TRY(last_error());
    SweepState hs;
    AP_CUDA_TRY(cudaMemcpyAsync(&hs, w.st, sizeof(hs), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    if (hs.nonfinite) return AP_ERR_NONFINITE;

    SweepArgs args;
    args.S = S;
    args.R0 = R;
    args.R1 = w.R1;
    args.A = A;
    args.ld = ld;
    args.n = ni;
    args.n4 = (ni + 3) / 4;
    args.w4 = c.W4;
    args.lam = p->damping;
    args.cvec = w.cvec;
    args.colp = w.colp;
    args.pcol = w.pcol;
    args.rkk = w.rkk;
    args.eflag = w.eflag;
    args.dec = decisions;
    args.st = w.st;

    // iterations per host check: about 4 ms of sweeping at full bandwidth
    int chunk = p->check_every;
    if (chunk <= 0) {
        const double t_iter = 20.0 * (double)n * (double)n / 6.0e12 + 6e-6;
        chunk = (int)std::min(64.0, std::max(1.0, 4e-3 / t_iter));
    }
    const int64_t total = (int64_t)p->max_iter + 1;
    const bool timed = (p->flags & AP_FLAG_TIME_SWEEP) != 0;
    EventPairs ev;
    if (timed) AP_TRY(ev.reserve(chunk));
    int64_t launched = 0;
    int32_t worked = 0;
    double sweep_ms = 0.0;
    const int fin_blocks = (ni + 255) / 256;
    int32_t t_before = 1;
    while (launched < total) {
        const int64_t m = std::min<int64_t>(chunk, total - launched);
        for (int64_t j = 0; j < m; ++j) {
            if (timed) AP_CUDA_TRY(cudaEventRecord(ev.start[j], s));
            AP_TRY(launch_sweep(c, args, s));
            if (timed) AP_CUDA_TRY(cudaEventRecord(ev.stop[j], s));
            finalize_kernel<<<fin_blocks, 256, 0, s>>>(w.pcol, c.G, ni, w.rkk, w.colp, w.cvec, w.st);
        }
        note_launches(2 * (uint64_t)m);
        AP_TRY(last_error());
        launched += m;
        AP_CUDA_TRY(cudaMemcpyAsync(&hs, w.st, sizeof(hs), cudaMemcpyDeviceToHost, s));
        AP_CUDA_TRY(cudaStreamSynchronize(s));
        const int32_t did = hs.t - t_before;       // launches in this chunk that did work
        t_before = hs.t;
        worked += did;
        if (timed) {
            for (int32_t j = 0; j < did; ++j) {
                float ms = 0.f;
                AP_CUDA_TRY(cudaEventElapsedTime(&ms, ev.start[j], ev.stop[j]));
                sweep_ms += ms;
            }
        }
        if (hs.done) break;
    }
    if (!hs.done) return AP_ERR_CUDA;   // cannot happen: launch max_iter+1 always stops
    if (hs.final_buf == 1)
        AP_CUDA_TRY(cudaMemcpy2DAsync(R, ld * sizeof(float), w.R1, ld * sizeof(float),
                                      n * sizeof(float), n, cudaMemcpyDeviceToDevice, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    const int32_t status = (p->conv_iter > 0 && !hs.converged) ? AP_NOT_CONVERGED : AP_OK;
    if (out) {
        *out = ap_result{};
        out->iters = hs.iters;
        out->converged = hs.converged;
        out->status = status;
        out->sweep_ms = sweep_ms;
        out->sweep_launches = worked;
    }
    return status;
}
