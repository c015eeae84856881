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
// stay in registers across every row of a work unit.  Each warp reduces its
// share of the row's top-2 and decision arg-max (redux.sync) and pushes it to
// every CTA of the cluster through distributed shared memory; rows are
// software-pipelined so that this exchange overlaps the next row's first half.
// Each cluster runs a host-made list of units (rows of one problem, each unit
// with its own column-partial slot), cut so that every cluster gets an equal
// share of the work.  A second small kernel sums each problem's unit partials
// in a fixed order (bitwise reproducible), and updates the device-side stop
// state.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <array>
#include <climits>
#include <cmath>
#include <functional>
#include <map>
#include <mutex>
#include <set>
#include <thread>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "ptx.cuh"

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
    int32_t error;       // a bounded wait gave up
    int32_t pad[4];
};

// One problem of a launch (a launch sweeps a table of independent problems;
// a single matrix is a table of one).
struct SweepArgs {
    const float* S;
    float*       R0;       // caller's R (buffer 0)
    float*       R1;       // workspace R (buffer 1)
    float*       A;
    int64_t      ld;
    int          n;
    int          n4;       // float4 columns spanning n
    int          w4;       // float4 columns per CTA
    int          G;        // units of this problem (unit g owns column-partial slot g)
    int          ns;       // pipeline stages (launch-wide)
    float        lam;      // launch-wide
    uint32_t     spin_limit;      // launch-wide
    const float* cvec;     // r(k,k) + colp(k) of R_{t-1}
    const float* colp;     // colp(k) of R_{t-1}
    float*       pcol;     // [G][pstride] per-unit partial column sums of R_t
    int64_t      pstride;
    float*       rkk;      // r(k,k) of R_t
    int32_t*     eflag;    // exemplar flags of the previous decisions
    int32_t*     dec;      // decisions (may be null)
    SweepState*  st;
    const float* zero;     // cold start: zeros read as R_0 (t = 1) and A_0 (t <= 2); else null
};

// One unit of a launch's work list: rows first, first + stride, ... (count
// rows) of problem b, whose column partials go to the problem's slot g.
struct __align__(16) Unit {
    int b, g, first, count, stride, pad[3];
};

// A launch's work list: cluster c runs units ubeg[c] .. ubeg[c+1]-1 one after
// another.
struct SweepLaunch {
    const SweepArgs* table;   // device
    const Unit* units;        // grouped by cluster
    const int* ubeg;          // clusters + 1 entries
    int count;
    int w4s;                  // stage stride: the widest slice of the launch (float4)
    int ns;                   // pipeline stages
};

// What a unit's CTA needs about its problem and its column slice.
struct UnitView {
    const SweepArgs* a;                 // read in place: fields used once per row or less
    SweepState* st;
    int g, first, stride, t;
    bool doA, doR;
    const float* Rin;
    float* Rout;
    int f_begin, f_end, nslice, f_full_end, nfull, nrows;
};

__device__ __forceinline__ bool unit_view(const SweepLaunch& L, int u, int crank, UnitView& v) {
    const Unit un = L.units[u];
    v.a = &L.table[un.b];
    v.st = v.a->st;
    if (v.st->done) return false;       // fixed during a launch: every CTA of the cluster agrees
    v.g = un.g;
    v.first = un.first;
    v.stride = un.stride;
    v.t = v.st->t;
    v.doA = v.t >= 2;
    v.doR = v.t <= v.st->max_iter;
    v.Rin = ((v.t - 1) & 1) ? v.a->R1 : v.a->R0;
    v.Rout = (v.t & 1) ? v.a->R1 : v.a->R0;
    v.f_begin = crank * v.a->w4;
    v.f_end = min(v.f_begin + v.a->w4, v.a->n4);
    v.nslice = max(0, v.f_end - v.f_begin);
    v.f_full_end = min(v.f_end, v.a->n >> 2);         // float4s entirely inside n
    v.nfull = max(0, v.f_full_end - v.f_begin);
    v.nrows = un.count;
    return true;
}

// A warp's partial row result, exchanged across the cluster: the top-2
// (m1, m2, j1) and the decision maximum dv; the decision index dj travels
// separately, to cluster rank 0 only.
struct __align__(16) Slot {
    float m1, m2, dv;
    int   j1;
};

constexpr int kMaxStages = 4;
constexpr int kMaxCluster = 16;

// Row partials rotate through kXBuf exchange buffers, row by row.  A warp
// sends row r's partial after it has received every warp's partial of row r-2
// (it waited for them while finishing row r-2), and every warp sends its row
// r-2 partial only after it has read its slots of row r-4 (and the receiving
// barrier's phase for row r-4 has completed); so four buffers are never
// overwritten unread.
constexpr int kXBuf = 4;

// Followed in shared memory by the kXBuf exchange barriers, then the row
// partials, kXBuf x C (sender CTA) x T/32 (sender warp) Slots, then as many
// decision indices (int).
struct __align__(16) Ctl {
    uint64_t full[kMaxStages];     // stage filled by TMA
    uint64_t done[kMaxStages];     // every compute warp finished with the stage
    int abort;                     // a compute warp gave up (stops the producer)
};

__device__ __forceinline__ float lane(const float4& v, int e) {
    return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
}
__device__ __forceinline__ void set_lane(float4& v, int e, float x) {
    if (e == 0) v.x = x; else if (e == 1) v.y = x; else if (e == 2) v.z = x; else v.w = x;
}

// Rows are staged through shared memory by a producer warp (the block's last
// warp, one lane): it keeps up to ns rows of this CTA's slices of S, R_{t-1}
// and A in flight as 1-D TMA bulk copies (mbarrier full[s] per stage), and
// once every compute warp has reported a stage finished (mbarrier done[s]) it
// writes the new A and R slices back with bulk asynchronous stores and refills
// the stage.  The compute warps never meet at a block barrier: their only
// synchronisation is the per-row cluster exchange, which pushes every warp's
// partial result into every CTA's shared memory with st.async, completing on
// the receiver's mbarrier.
// Register ceilings keep two CTAs of up to 320 compute threads (EPT 2) on an SM.
template <int EPT>
struct SweepRegs {
    static constexpr int value = EPT == 1 ? 64 : EPT == 2 ? 96 : 128;
    static constexpr int max_block = EPT >= 3 ? 512 : 544;   // compute threads + producer warp
};

template <int EPT>
__global__ void __launch_bounds__(SweepRegs<EPT>::max_block) __maxnreg__(SweepRegs<EPT>::value)
sweep_kernel(SweepLaunch L) {
    extern __shared__ __align__(128) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int csize = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int gc = blockIdx.x / csize;
    const int u_begin = L.ubeg[gc], u_end = L.ubeg[gc + 1];
    const int T = (int)blockDim.x - 32;         // compute threads
    const int tid = threadIdx.x;
    const int wid = tid >> 5, lid = tid & 31;
    const int nw = T >> 5;                      // compute warps
    const int NS = L.ns;
    const int w4s = L.w4s;
    constexpr int XB = kXBuf;
    float4* stage = reinterpret_cast<float4*>(smem);
    Ctl* ctl = reinterpret_cast<Ctl*>(smem + (size_t)NS * 3 * w4s * sizeof(float4));
    uint64_t* xbar = reinterpret_cast<uint64_t*>(ctl + 1);   // every warp's partial of a row arrived
    Slot* xs = reinterpret_cast<Slot*>(xbar + XB);
    int* xdj = reinterpret_cast<int*>(xs + (size_t)XB * csize * nw);

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            ptx::mbar_init(&ctl->full[s], 1);
            ptx::mbar_init(&ctl->done[s], (uint32_t)nw);
        }
        for (int b = 0; b < XB; ++b) ptx::mbar_init(&xbar[b], 1);
        ptx::fence_mbar_init();
        ctl->abort = 0;
    }
    __syncthreads();
    if (csize > 1) cluster.sync();              // peers' barriers exist before any st.async

    auto sS = [&](int s) { return stage + ((size_t)s * 3 + 0) * w4s; };
    auto sR = [&](int s) { return stage + ((size_t)s * 3 + 1) * w4s; };
    auto sA = [&](int s) { return stage + ((size_t)s * 3 + 2) * w4s; };

    int bad = 0;                                // a wait of this thread ran out
    if (wid == nw) {
        // ------------------------------ producer warp ------------------------------
        if (lid == 0) {
            int q0 = 0;                         // rows of this cluster's earlier units
            int sw = 0;                         // stage of the next row to store
            uint32_t wpar = 0;                  // and the parity of its done barrier's phase
            bool first = true;
            for (int u = u_begin; u < u_end; ++u) {
                UnitView v;
                if (!unit_view(L, u, crank, v)) continue;
                const SweepArgs& a = *v.a;
                const uint32_t slice_bytes = (uint32_t)v.nslice * 16u;
                const uint32_t row_bytes = slice_bytes * (v.doR ? 3u : 2u);
                // the previous unit's stores no longer read the stages about to be refilled
                if (!first) ptx::bulk_wait_read<0>();
                first = false;
                int issued = 0;
                auto issue = [&](int r, int s) {
                    ptx::mbar_arrive_expect_tx(&ctl->full[s], row_bytes);
                    if (v.nslice > 0) {
                        const int64_t off = (int64_t)(v.first + r * v.stride) * a.ld + 4 * (int64_t)v.f_begin;
                        // cold start: R_0 and A_0 are zeros, read from a small zeroed
                        // buffer (it stays in L2) instead of the caller's R and A
                        const float* rsrc = (a.zero && v.t == 1) ? a.zero : v.Rin + off;
                        const float* asrc = (a.zero && v.t <= 2) ? a.zero : a.A + off;
                        if (v.doR) ptx::bulk_g2s(sS(s), a.S + off, slice_bytes, &ctl->full[s]);
                        ptx::bulk_g2s(sR(s), rsrc, slice_bytes, &ctl->full[s]);
                        ptx::bulk_g2s(sA(s), asrc, slice_bytes, &ctl->full[s]);
                    }
                    issued = r + 1;
                };
                for (int r = 0, s = sw; r < min(NS, v.nrows); ++r) {
                    issue(r, s);
                    if (++s == NS) s = 0;
                }
                int k = 0;
                for (; k < v.nrows; ++k) {
                    const int s = sw;
                    // every compute warp is done with row k (bounded; gives up at once
                    // when a compute warp has given up)
                    uint32_t spins = 0;
                    while (!ptx::mbar_try_wait(&ctl->done[s], wpar)) {
                        if (*(volatile int*)&ctl->abort || ++spins >= a.spin_limit) {
                            bad = 1;
                            break;
                        }
                    }
                    if (bad) break;
                    if (v.nfull > 0) {
                        const int64_t off = (int64_t)(v.first + k * v.stride) * a.ld + 4 * (int64_t)v.f_begin;
                        if (v.doA) ptx::bulk_s2g(a.A + off, sA(s), (uint32_t)v.nfull * 16u);
                        if (v.doR) ptx::bulk_s2g(v.Rout + off, sR(s), (uint32_t)v.nfull * 16u);
                    }
                    ptx::bulk_commit();
                    if (k + NS < v.nrows) {
                        ptx::bulk_wait_read<0>();   // the stores no longer read stage s
                        issue(k + NS, s);
                    }
                    if (++sw == NS) {
                        sw = 0;
                        wpar ^= 1u;
                    }
                }
                if (bad) {
                    // drain the loads still in flight before shared memory goes away
                    for (int j = k; j < issued; ++j) {
                        const int q = q0 + j;
                        ptx::mbar_wait(&ctl->full[q % NS], (uint32_t)((q / NS) & 1), a.spin_limit);
                    }
                    atomicExch(&v.st->error, 1);
                    break;
                }
                q0 += v.nrows;
            }
            ptx::bulk_wait_all();
        }
    } else {
        // ------------------------------ compute warps ------------------------------
        const uint32_t nslot = (uint32_t)(csize * nw);
        uint32_t xphase = 0;                    // phase bits of xbar[0..XB-1]
        // Software pipeline over rows (three or more stages): iteration r forms
        // row r's partial result (phase 1) and sends it, then finishes row r-1
        // (phase 2), whose partials have been in flight across the cluster
        // meanwhile; the stage of row r-1 is held one iteration longer.  With
        // two stages iteration r finishes row r itself, so that the producer
        // still keeps one row in flight.
        const int pipe = NS >= 3 ? 1 : 0;
        int sg = 0;                             // stage of the next row
        uint32_t spar = 0;                      // and the parity of its full barrier's phase
        int x1 = 0, x2 = 0;                     // exchange buffers of the next phase-1 and phase-2 rows
        for (int u = u_begin; u < u_end && !bad; ++u) {
            UnitView v;
            if (!unit_view(L, u, crank, v)) continue;
            const SweepArgs& a = *v.a;
            SweepState* st = v.st;
            const int g = v.g, first = v.first, stride = v.stride;
            const bool doA = v.doA, doR = v.doR;
            const float lam = a.lam, oml = 1.0f - a.lam;
            const float2 lam2 = make_float2(lam, lam), oml2 = make_float2(oml, oml),
                         nom2 = make_float2(-oml, -oml);
            const int f_begin = v.f_begin, f_end = v.f_end, f_full_end = v.f_full_end;
            const int nrows = v.nrows;
            const int n = a.n;
            const float* colp = a.colp;
            int32_t* eflag = a.eflag;
            const uint32_t spin = a.spin_limit;
            float* Rout = v.Rout;
            int n_changes = 0, n_ex = 0;        // counted by the deciding lane
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
                        set_lane(cv[q], e, k < n ? oml * a.cvec[k] : 0.f);   // (1-lambda) c(k)
                    }
                }
            }
            // Bytes landing in this CTA's slot buffer per row: every warp of the
            // cluster sends (m1, m2, dv, j1); the decision index dj goes to rank 0
            // only, where warp 0 makes the row's decision.
            const bool decide = doA && crank == 0 && wid == 0;
            const uint32_t xbytes = nslot * (16u + ((doA && crank == 0) ? 4u : 0u));
            // Phase 1 of row i, held in stage s: the availability half of the
            // previous iteration (damped in place) with the decision arg-max, and
            // the partial top-2 of a + s, sent to every CTA of the cluster through
            // exchange buffer xb.
            auto phase1 = [&](int i, int s, float colp_i, int xb) {
                const float4* S4 = sS(s);
                const float4* R4 = sR(s);
                float4* A4 = sA(s);
                const int fi = i >> 2;          // the float4 holding column i
                Top2 tp{-INFINITY, -INFINITY, INT_MAX};
                float dv = -INFINITY;
                int dj = INT_MAX;
                // Columns reach a thread in increasing order, so inside a thread a
                // strictly larger value is all an update needs (the first index
                // stays); index tie-breaks matter only when threads are merged.
#pragma unroll
                for (int q = 0; q < EPT; ++q) {
                    const int f = f_begin + tid + q * T;
                    if (f < f_end) {
                        const int x = f - f_begin;
                        const float4 s4 = doR ? S4[x] : make_float4(0.f, 0.f, 0.f, 0.f);
                        const float4 r4 = R4[x];
                        float4 a4 = A4[x];
                        if (f != fi && f < f_full_end) {
                            // fast path: no diagonal, no ragged tail
                            const int k0 = 4 * f;
                            // (1-lambda) min(0, c - max(0,r)) = min(0, (1-lambda)c - (1-lambda)max(0,r)),
                            // in packed f32x2 arithmetic, two columns per instruction
                            float2 alo = make_float2(a4.x, a4.y), ahi = make_float2(a4.z, a4.w);
                            if (doA) {
                                const float2 tlo = __ffma2_rn(nom2, make_float2(fmaxf(0.f, r4.x), fmaxf(0.f, r4.y)),
                                                              make_float2(cv[q].x, cv[q].y));
                                const float2 thi = __ffma2_rn(nom2, make_float2(fmaxf(0.f, r4.z), fmaxf(0.f, r4.w)),
                                                              make_float2(cv[q].z, cv[q].w));
                                alo = __ffma2_rn(lam2, alo, make_float2(fminf(0.f, tlo.x), fminf(0.f, tlo.y)));
                                ahi = __ffma2_rn(lam2, ahi, make_float2(fminf(0.f, thi.x), fminf(0.f, thi.y)));
                                const float2 dlo = __fadd2_rn(alo, make_float2(r4.x, r4.y));
                                const float2 dhi = __fadd2_rn(ahi, make_float2(r4.z, r4.w));
                                if (dlo.x > dv) { dv = dlo.x; dj = k0; }
                                if (dlo.y > dv) { dv = dlo.y; dj = k0 + 1; }
                                if (dhi.x > dv) { dv = dhi.x; dj = k0 + 2; }
                                if (dhi.y > dv) { dv = dhi.y; dj = k0 + 3; }
                                A4[x] = make_float4(alo.x, alo.y, ahi.x, ahi.y);
                            }
                            if (doR) {
                                const float2 vlo = __fadd2_rn(alo, make_float2(s4.x, s4.y));
                                const float2 vhi = __fadd2_rn(ahi, make_float2(s4.z, s4.w));
                                float v;
                                v = vlo.x; tp.m2 = fmaxf(tp.m2, fminf(tp.m1, v)); if (v > tp.m1) { tp.m1 = v; tp.j1 = k0; }
                                v = vlo.y; tp.m2 = fmaxf(tp.m2, fminf(tp.m1, v)); if (v > tp.m1) { tp.m1 = v; tp.j1 = k0 + 1; }
                                v = vhi.x; tp.m2 = fmaxf(tp.m2, fminf(tp.m1, v)); if (v > tp.m1) { tp.m1 = v; tp.j1 = k0 + 2; }
                                v = vhi.y; tp.m2 = fmaxf(tp.m2, fminf(tp.m1, v)); if (v > tp.m1) { tp.m1 = v; tp.j1 = k0 + 3; }
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int k = 4 * f + e;
                                if (k < n) {
                                    const float sv = lane(s4, e), rv = lane(r4, e);
                                    float av = lane(a4, e);
                                    if (doA) {
                                        const float an = (k == i) ? oml * colp_i
                                                                  : fminf(0.f, fmaf(-oml, fmaxf(0.f, rv), lane(cv[q], e)));
                                        av = fmaf(lam, av, an);
                                        set_lane(a4, e, av);
                                        argmax_merge(dv, dj, av + rv, k);
                                    }
                                    if (doR) top2_push(tp, av + sv, k);
                                }
                            }
                            if (doA) {
                                if (f < f_full_end) {
                                    A4[x] = a4;
                                } else {
                                    float* Arow = a.A + (int64_t)i * a.ld;
#pragma unroll
                                    for (int e = 0; e < 4; ++e)
                                        if (4 * f + e < n) Arow[4 * f + e] = lane(a4, e);
                                }
                            }
                        }
                    }
                }
                // Row partials: every warp's reduced (top-2, arg-max) goes straight
                // into slot (this CTA, this warp) of every CTA of the cluster (this
                // one included) by st.async, completing on the receiver's xbar[xb].
                tp = top2_warp_redux(tp);
                argmax_warp_redux(dv, dj);
                if (tid == 0) ptx::mbar_arrive_expect_tx(&xbar[xb], xbytes);
                if (lid < csize) {
                    const uint32_t at = (uint32_t)xb * nslot + crank * nw + wid;
                    const uint32_t ra = ptx::mapa(xs + at, (uint32_t)lid);
                    const uint32_t rb = ptx::mapa(&xbar[xb], (uint32_t)lid);
                    ptx::st_async_v4(ra, __float_as_uint(tp.m1), __float_as_uint(tp.m2),
                                     __float_as_uint(dv), (uint32_t)tp.j1, rb);
                    if (doA && lid == 0)            // lane 0 writes to rank 0
                        ptx::st_async_b32(ptx::mapa(xdj + at, 0u), (uint32_t)dj, rb);
                }
            };
            // Phase 2 of row i: every warp's partials (false when the wait gave
            // up), the row's decision, and the responsibility half.
            auto phase2 = [&](int i, int s, int ef_rp, int xb) -> bool {
                const bool ok = ptx::mbar_wait(&xbar[xb], (uint32_t)((xphase >> xb) & 1u), spin);
                if (__any_sync(0xffffffffu, !ok)) return false;
                xphase ^= 1u << xb;
                Top2 u{-INFINITY, -INFINITY, INT_MAX};
                float uv = -INFINITY;
                int uj = INT_MAX;
                const Slot* xr = xs + (uint32_t)xb * nslot;
                const int* xd = xdj + (uint32_t)xb * nslot;
                for (uint32_t q = (uint32_t)lid; q < nslot; q += 32) {
                    const float4 p = *reinterpret_cast<const float4*>(&xr[q]);
                    u = top2_merge(u, Top2{p.x, p.y, __float_as_int(p.w)});
                    if (decide) argmax_merge(uv, uj, p.z, xd[q]);
                }
                if (decide) {
                    argmax_warp_redux(uv, uj);
                    if (lid == 0) {
                        if (a.dec) a.dec[i] = uj;
                        const int e = (uj == i) ? 1 : 0;
                        if (ef_rp != e) ++n_changes;
                        eflag[i] = e;
                        n_ex += e;
                    }
                }
                if (doR) {
                    u = top2_warp_redux(u);
                    const float om1 = oml * u.m1, om2 = oml * u.m2;     // (1-lambda) m1, m2
                    const int j1 = u.j1;
                    const float2 nm1 = make_float2(-om1, -om1);
                    const float4* S4 = sS(s);
                    float4* R4 = sR(s);
                    const int fi = i >> 2;
                    const int fj = j1 >> 2;     // the float4 holding the row's arg-max
#pragma unroll
                    for (int q = 0; q < EPT; ++q) {
                        const int f = f_begin + tid + q * T;
                        if (f < f_end) {
                            const int x = f - f_begin;
                            const float4 s4 = S4[x], r4 = R4[x];
                            float4 o;
                            if (f != fi && f != fj && f < f_full_end) {
                                // fast path: every column takes m1, none is the diagonal;
                                // lambda r + (1-lambda) s - (1-lambda) m1, packed f32x2
                                const float2 olo = __ffma2_rn(lam2, make_float2(r4.x, r4.y),
                                                              __ffma2_rn(oml2, make_float2(s4.x, s4.y), nm1));
                                const float2 ohi = __ffma2_rn(lam2, make_float2(r4.z, r4.w),
                                                              __ffma2_rn(oml2, make_float2(s4.z, s4.w), nm1));
                                const float2 plo = __fadd2_rn(make_float2(acc[q].x, acc[q].y),
                                                              make_float2(fmaxf(0.f, olo.x), fmaxf(0.f, olo.y)));
                                const float2 phi = __fadd2_rn(make_float2(acc[q].z, acc[q].w),
                                                              make_float2(fmaxf(0.f, ohi.x), fmaxf(0.f, ohi.y)));
                                acc[q] = make_float4(plo.x, plo.y, phi.x, phi.y);
                                o = make_float4(olo.x, olo.y, ohi.x, ohi.y);
                                R4[x] = o;
                            } else {
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    const int k = 4 * f + e;
                                    const float sv = lane(s4, e), rv = lane(r4, e);
                                    const float om = (k == j1) ? om2 : om1;
                                    const float rn = fmaf(lam, rv, fmaf(oml, sv, -om));
                                    set_lane(o, e, rn);
                                    if (k < n) {
                                        if (k == i) a.rkk[i] = rn;
                                        else set_lane(acc[q], e, lane(acc[q], e) + fmaxf(0.f, rn));
                                    }
                                }
                                if (f < f_full_end) {
                                    R4[x] = o;
                                } else {
                                    float* Orow = Rout + (int64_t)i * a.ld;
#pragma unroll
                                    for (int e = 0; e < 4; ++e)
                                        if (4 * f + e < n) Orow[4 * f + e] = lane(o, e);
                                }
                            }
                        }
                    }
                }
                return true;
            };
            // hand stage s back to the producer: this warp's shared-memory writes
            // are made visible to the bulk stores, then one lane arrives
            auto release = [&](int s) {
                ptx::fence_proxy_async_smem();
                __syncwarp();
                if (lid == 0) ptx::mbar_arrive(&ctl->done[s]);
            };
            // per-row scalars are loaded a row ahead, off the critical path
            float colp_next = (doA && nrows > 0) ? colp[first] : 0.f;
            int ef_next = (decide && lid == 0 && nrows > 0) ? eflag[first] : 0;
            int ef_prev = 0, s_prev = 0;
            for (int r = 0; r < nrows + pipe; ++r) {
                int ef_this = 0, s_this = 0;
                if (r < nrows) {
                    const int i = first + r * stride;
                    const float colp_i = colp_next;
                    if (doA && r + 1 < nrows) colp_next = colp[i + stride];
                    ef_this = ef_next;
                    if (decide && lid == 0 && r + 1 < nrows) ef_next = eflag[i + stride];
                    // a give-up is made warp-uniform: the warp's lanes stay
                    // converged for the redux reductions
                    const bool ok = ptx::mbar_wait(&ctl->full[sg], spar, spin);
                    if (__any_sync(0xffffffffu, !ok)) {
                        bad = 1;
                        break;
                    }
                    s_this = sg;
                    if (++sg == NS) {
                        sg = 0;
                        spar ^= 1u;
                    }
                    phase1(i, s_this, colp_i, x1);
                    if (++x1 == XB) x1 = 0;
                }
                if (r - pipe >= 0) {
                    const int rp = r - pipe;
                    const int s = pipe ? s_prev : s_this;
                    if (!phase2(first + rp * stride, s, pipe ? ef_prev : ef_this, x2)) {
                        bad = 1;
                        break;
                    }
                    if (++x2 == XB) x2 = 0;
                    release(s);
                }
                ef_prev = ef_this;
                s_prev = s_this;
            }
            if (bad) {
                atomicExch(&st->error, 1);
                break;
            }
            // the unit's column partials go to its own slot: the sums over
            // slots are taken in a fixed order whichever cluster ran the unit
            if (doR) {
                float* P = a.pcol + (int64_t)g * a.pstride;
#pragma unroll
                for (int q = 0; q < EPT; ++q) {
                    const int f = f_begin + tid + q * T;
                    if (f < f_end) {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (4 * f + e < n) P[4 * f + e] = lane(acc[q], e);
                    }
                }
            }
            if (decide && lid == 0) {
                atomicAdd(&st->changes, n_changes);
                atomicAdd(&st->n_ex, n_ex);
            }
        }
        if (bad) *(volatile int*)&ctl->abort = 1;
    }
    __syncthreads();
    // keep this CTA's shared memory alive until every peer is done with it
    if (csize > 1) cluster.sync();
}

// Column sums in a fixed order, then the stop rule (block 0 of each
// problem).  Block: 32 columns x 16 lanes over the problem's G unit partials;
// each lane sums every 16th partial, then the 16 lane sums are added in a
// fixed tree, so the result does not depend on the schedule.
// Grid: (ceil(n/32), problems).
constexpr int kFinCols = 32, kFinLanes = 32;

// The kFinLanes lane sums of a column added in a fixed pairwise tree.
__device__ __forceinline__ float lane_tree(const float (*part)[kFinCols], int cx) {
    float v[kFinLanes];
#pragma unroll
    for (int l = 0; l < kFinLanes; ++l) v[l] = part[l][cx];
#pragma unroll
    for (int w = kFinLanes / 2; w >= 1; w >>= 1)
#pragma unroll
        for (int e = 0; e < w; ++e) v[e] = v[2 * e] + v[2 * e + 1];
    return v[0];
}

// Step 4 of Algorithm 1 after launch t (one thread): the exemplar set of
// iteration t-1 extends or resets the run of unchanged sets; stop once it
// has been the same, and non-empty, for conv_iter iterations, or after
// max_iter iterations.
__device__ __forceinline__ void apply_stop_rule(SweepState* st) {
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

__global__ void __launch_bounds__(kFinCols * kFinLanes) finalize_kernel(const SweepArgs* __restrict__ table) {
    const SweepArgs& a = table[blockIdx.y];
    const int cx = threadIdx.x % kFinCols, gy = threadIdx.x / kFinCols;
    const int k = blockIdx.x * kFinCols + cx;
    SweepState* st = a.st;
    if (st->done) return;                       // uniform per problem; finished rows are final
    __shared__ float part[kFinLanes][kFinCols];
    float s = 0.f;
    if (k < a.n) {
#pragma unroll 4
        for (int g = gy; g < a.G; g += kFinLanes) s += a.pcol[(int64_t)g * a.pstride + k];
    }
    part[gy][cx] = s;
    __syncthreads();
    if (gy == 0 && k < a.n) {
        const float t = lane_tree(part, cx);
        const_cast<float*>(a.colp)[k] = t;
        const_cast<float*>(a.cvec)[k] = a.rkk[k] + t;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) apply_stop_rule(st);
}

__global__ void sweep_init_kernel(const SweepArgs* __restrict__ table, int max_iter, int conv_iter) {
    const SweepArgs& a = table[blockIdx.y];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < a.n) a.eflag[k] = 0;
    if (k == 0) {
        SweepState s{};
        s.t = 1;
        s.max_iter = max_iter;
        s.conv_iter = conv_iter;
        *a.st = s;
    }
}

// NaN/Inf entries of every problem's S.  Rows start 16-byte aligned (S is
// 16-byte aligned and ld % 4 == 0), so each row is read as float4 up to its
// last whole group of four, then the ragged tail one float at a time.
__global__ void nonfinite_kernel(const SweepArgs* __restrict__ table) {
    const SweepArgs& a = table[blockIdx.y];
    const int n4 = a.n >> 2;
    int local = 0;
    for (int i = blockIdx.x; i < a.n; i += gridDim.x) {
        const float* row = a.S + (int64_t)i * a.ld;
        const float4* row4 = reinterpret_cast<const float4*>(row);
#pragma unroll 4
        for (int k = threadIdx.x; k < n4; k += blockDim.x) {
            const float4 v = __ldg(row4 + k);
            local += !isfinite(v.x) + !isfinite(v.y) + !isfinite(v.z) + !isfinite(v.w);
        }
        for (int k = 4 * n4 + threadIdx.x; k < a.n; k += blockDim.x) local += !isfinite(row[k]);
    }
    local = __reduce_add_sync(0xffffffffu, local);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(&a.st->nonfinite, local);
}

// ---------------------------------------------------------------------------
// Launch configuration
// ---------------------------------------------------------------------------
struct SweepConfig {
    int C, T, EPT, W4, G, NS;
    int R;                        // resident clusters (G = min(R, n): a single problem's clusters)
    size_t smem;
};

static void* sweep_ptr(int ept) {
    switch (ept) {
        case 1: return (void*)sweep_kernel<1>;
        case 2: return (void*)sweep_kernel<2>;
        case 3: return (void*)sweep_kernel<3>;
        default: return (void*)sweep_kernel<4>;
    }
}

static size_t sweep_smem(int w4, int ns, int C, int T) {
    const size_t slots = (size_t)kXBuf * C * (T / 32);
    return (size_t)ns * 3 * w4 * sizeof(float4) + sizeof(Ctl) + kXBuf * sizeof(uint64_t) +
           (slots * (sizeof(Slot) + sizeof(int)) + 15) / 16 * 16;
}

// Every instantiation of the sweep kernel may use dynamic shared memory up to
// the 227 KB opt-in limit and non-portable cluster sizes.  Set once per
// device and instantiation (a launch still asks only for its own bytes), so
// that launches of different configurations, also from several host threads,
// never lower one another's ceiling.
static int32_t prepare_sweep_fn(int ept) {
    static std::mutex mu;
    static std::set<std::pair<int, int>> ready;
    int dev = 0;
    AP_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (ready.count({dev, ept})) return AP_OK;
    void* fn = sweep_ptr(ept);
    AP_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    AP_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    ready.insert({dev, ept});
    return AP_OK;
}

static int32_t max_clusters(int ept, int C, int T, size_t smem, int* out) {
    void* fn = sweep_ptr(ept);
    AP_TRY(prepare_sweep_fn(ept));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(T + 32, 1, 1);
    cfg.dynamicSmemBytes = smem;
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

// Validates (C, ept, ns) for n and fills the derived launch parameters.
static int32_t make_config(int n, int C, int ept, int ns, SweepConfig* c) {
    if (C < 1 || C > kMaxCluster || ept < 1 || ept > 4 || ns < 2 || ns > kMaxStages)
        return AP_ERR_INVALID_ARG;
    const int n4 = (n + 3) / 4;
    if (C > 1 && n4 < 8 * C) return AP_ERR_UNSUPPORTED;
    const int w4 = (n4 + C - 1) / C;
    int T = ((w4 + ept - 1) / ept + 31) / 32 * 32;
    T = std::max(T, 64);
    const int max_block = ept == 1 ? SweepRegs<1>::max_block : ept == 2 ? SweepRegs<2>::max_block
                                                                       : SweepRegs<3>::max_block;
    if (T + 32 > max_block) return AP_ERR_UNSUPPORTED;
    const size_t smem = sweep_smem(w4, ns, C, T);
    if (smem > 227 * 1024) return AP_ERR_UNSUPPORTED;
    int num = 0;
    AP_TRY(max_clusters(ept, C, T, smem, &num));
    if (num <= 0) return AP_ERR_UNSUPPORTED;
    c->C = C;
    c->T = T;
    c->EPT = ept;
    c->W4 = w4;
    c->NS = ns;
    c->smem = smem;
    c->R = num;
    c->G = std::max(1, std::min(num, n));
    return AP_OK;
}

static std::mutex g_pin_mu;
static std::map<int64_t, std::array<int, 3>> g_pinned;   // n -> (C, ept, ns)
static std::map<int64_t, SweepConfig> g_chosen;         // (device, n) -> default configuration

// The default configuration.  Below 16384 points: the smallest power-of-two
// cluster whose slice is at most 640 float4 columns (a stage of at most
// 30 KB), and among its configurations the most resident CTAs, ties to three
// stages, then four, then two, and to 3, 4, 2, 1 float4 per thread.  From
// 16384 points on, every cluster size from 1 to 16 competes and the most
// resident clusters win (each cluster keeps its own rows in flight, so the
// row pipeline's depth grows with the clusters, not with the CTAs), then the
// most resident CTAs, then the same stage and float4 order.  Measured on the
// 20000-point mixture: 46 clusters of 6 CTAs sweep in 1.118 ms where the
// power-of-two rule's 36 clusters of 8 took 1.190 ms; clusters that are not
// powers of two also pack better onto the GPCs at one CTA per SM (9-CTA
// clusters keep 135 SMs busy at 60000 points where 8-CTA ones keep 120).  A
// configuration pinned for n (by ap_sweep_set_config or the autotuner) takes
// precedence.
constexpr int kAnyClusterN = 16384;

static int32_t choose_config(int n, SweepConfig* c) {
    {
        std::lock_guard<std::mutex> lock(g_pin_mu);
        auto it = g_pinned.find(n);
        if (it != g_pinned.end()) return make_config(n, it->second[0], it->second[1], it->second[2], c);
    }
    int dev = 0;
    AP_CUDA_TRY(cudaGetDevice(&dev));
    const int64_t key = ((int64_t)dev << 32) | (uint32_t)n;
    {
        std::lock_guard<std::mutex> lock(g_pin_mu);
        auto it = g_chosen.find(key);
        if (it != g_chosen.end()) {
            *c = it->second;
            return AP_OK;
        }
    }
    const int n4 = (n + 3) / 4;
    int C0 = 1;
    while (C0 < kMaxCluster && (n4 + C0 - 1) / C0 > 640) C0 *= 2;
    const bool any = n >= kAnyClusterN || (n4 + kMaxCluster - 1) / kMaxCluster > 640;
    auto ns_rank = [](int ns) { return ns == 3 ? 2 : ns == 4 ? 1 : 0; };
    auto ept_rank = [](int e) { return e == 3 ? 3 : e == 4 ? 2 : e == 2 ? 1 : 0; };
    bool found = false;
    SweepConfig best{}, cand{};
    for (int C = any ? 1 : C0; C <= (any ? kMaxCluster : C0); C = any ? C + 1 : 2 * C)
        for (int ns = 2; ns <= kMaxStages; ++ns)
            for (int ept = 1; ept <= 4; ++ept) {
                if (make_config(n, C, ept, ns, &cand) != AP_OK) continue;
                const long ctas = (long)cand.G * cand.C, bctas = (long)best.G * best.C;
                const long cl = any ? cand.G : 0, bcl = any ? best.G : 0;
                const bool better =
                    !found || cl > bcl ||
                    (cl == bcl && (ctas > bctas ||
                                   (ctas == bctas && (ns_rank(cand.NS) > ns_rank(best.NS) ||
                                                      (ns_rank(cand.NS) == ns_rank(best.NS) &&
                                                       ept_rank(cand.EPT) > ept_rank(best.EPT))))));
                if (better) best = cand;
                found = true;
            }
    if (!found) return AP_ERR_UNSUPPORTED;
    *c = best;
    std::lock_guard<std::mutex> lock(g_pin_mu);
    g_chosen[key] = best;
    return AP_OK;
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

// One matrix of a batch, as the caller describes it.
struct Problem {
    const float* S;
    float* R;
    float* A;
    int64_t n, ld;
    int32_t* dec;
};

// How a batch is launched: one configuration (chosen for the largest
// problem) and a work list of units spread over the launch's clusters.
struct Plan {
    SweepConfig c;
    std::vector<int> G;           // units of each problem (0: finished)
    std::vector<int> ufirst;      // each problem's first column-partial slot in the pool
    std::vector<Unit> units;      // grouped by cluster
    std::vector<int> ubeg;        // clusters + 1
    int clusters = 0;
    int nmax = 0;
};

// Cost of one row of n elements, in element-equivalents: n when the row is
// bandwidth-bound, and never below the fixed cost of a row's round trip
// through the cluster, in units of one resident cluster's share of the HBM
// bandwidth (20 B per element).
static double row_cost(int64_t n, const SweepConfig& c) {
    const double t_row = 0.6e-6 * std::pow((double)c.C, 0.8);
    const double elems = t_row * 6.5e12 / (20.0 * std::max(c.R, 1));
    return std::max((double)n, elems);
}

// The work list for the active problems.  Laid end to end (problem order,
// each row weighted by row_cost), the work is cut into R equal shares, one
// per resident cluster, and every row goes to the share holding its
// midpoint; a problem's rows in one share form one unit.  Where consecutive
// shares hold nothing but rows of one problem (always, for a single problem)
// their rows are dealt out to them interleaved instead -- share m of M takes
// rows A + m, A + m + M, ... -- so that the problem's clusters move through
// memory side by side (contiguous blocks per cluster measured about 3 %
// slower).  A problem's units are consecutive in the list and number at most
// min(R, n); the list has at most R + count - 1.  Shares that receive no row
// are dropped.  The same active set always yields the same plan.
static void plan_units(const Problem* P, int count, const std::vector<char>& active, Plan* plan) {
    const SweepConfig& c = plan->c;
    const int K = std::max(c.R, 1);
    std::vector<double> rc(count, 0.0);
    double total = 0.0;
    for (int b = 0; b < count; ++b)
        if (active[b]) {
            rc[b] = row_cost(P[b].n, c);
            total += (double)P[b].n * rc[b];
        }
    const double share = std::max(total / K, 1e-30);
    // contiguous pieces (b, first row, end row, share)
    struct Piece { int b, r0, r1, k; };
    std::vector<Piece> pieces;
    double start = 0.0;                   // work before problem b
    for (int b = 0; b < count; ++b) {
        if (!active[b]) continue;
        const int n = (int)P[b].n;
        const double w = rc[b];
        auto share_of = [&](int j) {
            const double k = std::floor((start + (j + 0.5) * w) / share);
            return (int)std::min<double>(std::max(k, 0.0), K - 1);
        };
        for (int j = 0; j < n;) {
            const int k = share_of(j);
            int jend = n;
            if (k < K - 1) {
                // the first row whose midpoint lies beyond share k
                jend = (int)std::ceil(((k + 1) * share - start) / w - 0.5);
                jend = std::min(std::max(jend, j + 1), n);
                while (jend < n && share_of(jend) == k) ++jend;      // rounding guards
                while (jend > j + 1 && share_of(jend - 1) != k) --jend;
            }
            pieces.push_back({b, j, jend, k});
            j = jend;
        }
        start += (double)n * w;
    }
    std::vector<int> in_share(K, 0);
    for (const Piece& q : pieces) ++in_share[q.k];
    plan->G.assign(count, 0);
    plan->ufirst.assign(count, 0);
    plan->units.clear();
    plan->ubeg.assign(1, 0);
    int slots = 0, klast = -1;
    auto emit = [&](const Piece& q, const Unit& u) {
        if (q.k != klast) {
            if (klast >= 0) plan->ubeg.push_back((int)plan->units.size());
            klast = q.k;
        }
        plan->units.push_back(u);
    };
    for (size_t i = 0; i < pieces.size();) {
        const int b = pieces[i].b;
        if (plan->G[b] == 0) plan->ufirst[b] = slots;
        // a run of pieces of problem b alone in their shares
        size_t j = i;
        while (j < pieces.size() && pieces[j].b == b && in_share[pieces[j].k] == 1) ++j;
        if (j - i >= 2) {
            const int M = (int)(j - i), A = pieces[i].r0, len = pieces[j - 1].r1 - A;
            for (int m = 0; m < M; ++m)
                emit(pieces[i + m], Unit{b, plan->G[b]++, A + m, (len - m + M - 1) / M, M, {0, 0, 0}});
            slots += M;
            i = j;
            continue;
        }
        const Piece& q = pieces[i];
        emit(q, Unit{b, plan->G[b]++, q.r0, q.r1 - q.r0, 1, {0, 0, 0}});
        ++slots;
        ++i;
    }
    plan->ubeg.push_back((int)plan->units.size());
    plan->clusters = (int)plan->ubeg.size() - 1;
}

// Work-list capacity: units, clusters and per-unit column partials.
static size_t max_units(int count, const SweepConfig& c) { return (size_t)std::max(c.R, 1) + count; }

static int32_t make_plan(const Problem* P, int count, const SweepConfig* forced, Plan* plan) {
    int64_t nmax = 0;
    for (int b = 0; b < count; ++b) nmax = std::max(nmax, P[b].n);
    plan->nmax = (int)nmax;
    if (forced) plan->c = *forced;
    else AP_TRY(choose_config((int)nmax, &plan->c));
    std::vector<char> active(count, 1);
    plan_units(P, count, active, plan);
    return AP_OK;
}

struct SweepWs {
    SweepArgs* table;
    Unit* units;
    int* ubeg;
    float* pool;                  // per-unit column partials, nmax floats each
    SweepState* states;           // one per problem, contiguous (one read-back per check)
    float* zero;                  // cold start: zeros, the widest problem's slice
    size_t zero_bytes;
    std::vector<SweepArgs> host;
};

// Workspace: the problem table, the work list and the per-unit column
// partials, then per problem the second R buffer, colp, c = r(k,k)+colp,
// r(k,k), exemplar flags and the stop state.
static size_t carve_sweep(void* ws, const Problem* P, int count, const Plan& plan, SweepWs* w) {
    Carver cv(ws);
    SweepArgs* table = cv.take<SweepArgs>(count);
    Unit* units = cv.take<Unit>(max_units(count, plan.c));
    int* ubeg = cv.take<int>((size_t)std::max(plan.c.R, 1) + 1);
    float* pool = cv.take<float>(max_units(count, plan.c) * (size_t)plan.nmax);
    SweepState* states = cv.take<SweepState>((size_t)count);
    int64_t w4max = 1;
    for (int b = 0; b < count; ++b)
        w4max = std::max<int64_t>(w4max, ((P[b].n + 3) / 4 + plan.c.C - 1) / plan.c.C);
    float* zero = cv.take<float>((size_t)w4max * 4);
    if (w) {
        w->table = table;
        w->units = units;
        w->ubeg = ubeg;
        w->pool = pool;
        w->states = states;
        w->zero = zero;
        w->zero_bytes = (size_t)w4max * 16;
        w->host.assign(count, SweepArgs{});
    }
    for (int b = 0; b < count; ++b) {
        const int64_t n = P[b].n, ld = P[b].ld;
        SweepArgs a{};
        a.S = P[b].S;
        a.R0 = P[b].R;
        a.A = P[b].A;
        a.ld = ld;
        a.n = (int)n;
        a.n4 = (int)((n + 3) / 4);
        a.w4 = (a.n4 + plan.c.C - 1) / plan.c.C;
        a.G = plan.G[b];
        a.pstride = plan.nmax;
        a.pcol = pool + (size_t)plan.ufirst[b] * plan.nmax;
        a.ns = plan.c.NS;
        a.spin_limit = 1u << 20;
        a.R1 = cv.take<float>((size_t)n * ld);
        a.colp = cv.take<float>(n);
        a.cvec = cv.take<float>(n);
        a.rkk = cv.take<float>(n);
        a.eflag = cv.take<int32_t>(n);
        a.st = states ? states + b : nullptr;
        a.dec = P[b].dec;
        if (w) w->host[b] = a;
    }
    return cv.used;
}

static int32_t launch_sweep(const SweepConfig& c, int clusters, const SweepLaunch& L, cudaStream_t s,
                            bool set_attr = true) {
    if (set_attr) AP_TRY(prepare_sweep_fn(c.EPT));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c.C * clusters, 1, 1);
    cfg.blockDim = dim3(c.T + 32, 1, 1);       // compute warps + the producer warp
    cfg.dynamicSmemBytes = c.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = c.C;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    void* args[] = {const_cast<SweepLaunch*>(&L)};
    const cudaError_t e = cudaLaunchKernelExC(&cfg, sweep_ptr(c.EPT), args);
    return e == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

static bool valid_problem(const Problem& p) {
    return p.S && p.R && p.A && p.n >= 2 && p.n <= INT_MAX / 4 && p.ld >= p.n && !(p.ld & 3) &&
           aligned16(p.S) && aligned16(p.R) && aligned16(p.A);
}

static bool valid_params(const ap_params* p) {
    return p && p->damping >= 0.f && p->damping < 1.f && p->max_iter >= 1 && p->conv_iter >= 0;
}

// CUDA graphs of a chunk of iterations (m x {sweep, finalize}).  A chunk is
// captured once on a library-owned stream of the current device and the
// executable graph is kept, keyed by everything its launches bake in (the
// problem table's address and the launch shape), so repeated calls with the
// same workspace replay it.  All iteration state lives on the device, so a
// replay continues where the previous one stopped.
struct GraphKey {
    int dev;
    const void* table;
    int count, C, EPT, NS, T, G, clusters, nmax;
    size_t smem;
    int64_t m;
    bool operator<(const GraphKey& o) const {
        return std::tie(dev, table, count, C, EPT, NS, T, G, clusters, nmax, smem, m) <
               std::tie(o.dev, o.table, o.count, o.C, o.EPT, o.NS, o.T, o.G, o.clusters, o.nmax,
                        o.smem, o.m);
    }
};

static std::mutex g_graph_mu;
static std::map<GraphKey, cudaGraphExec_t> g_graphs;
static std::map<int, cudaStream_t> g_capture_stream;
constexpr size_t kMaxGraphs = 32;

static int32_t enqueue_chunk(const SweepConfig& c, const Plan& plan, const SweepLaunch& L,
                             int64_t m, dim3 fin_grid, cudaStream_t s) {
    for (int64_t j = 0; j < m; ++j) {
        AP_TRY(launch_sweep(c, plan.clusters, L, s, false));
        finalize_kernel<<<fin_grid, kFinCols * kFinLanes, 0, s>>>(L.table);
    }
    return last_error();
}

static int32_t launch_chunk_graph(const SweepConfig& c, const Plan& plan, const SweepLaunch& L,
                                  int64_t m, dim3 fin_grid, cudaStream_t s) {
    int dev = 0;
    AP_CUDA_TRY(cudaGetDevice(&dev));
    const GraphKey key{dev, L.table, L.count, c.C, c.EPT, c.NS, c.T, c.G, plan.clusters,
                       plan.nmax, c.smem, m};
    // the shared-memory ceiling is a function attribute, set outside the capture
    AP_TRY(prepare_sweep_fn(c.EPT));
    std::lock_guard<std::mutex> lock(g_graph_mu);
    auto it = g_graphs.find(key);
    if (it == g_graphs.end()) {
        cudaStream_t cs;
        auto sit = g_capture_stream.find(dev);
        if (sit == g_capture_stream.end()) {
            AP_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            g_capture_stream[dev] = cs;
        } else {
            cs = sit->second;
        }
        AP_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        const int32_t st = enqueue_chunk(c, plan, L, m, fin_grid, cs);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (st != AP_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return st != AP_OK ? st : AP_ERR_CUDA;
        }
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return AP_ERR_CUDA;
        if (g_graphs.size() >= kMaxGraphs) {
            cudaGraphExecDestroy(g_graphs.begin()->second);
            g_graphs.erase(g_graphs.begin());
        }
        it = g_graphs.emplace(key, exec).first;
    }
    AP_CUDA_TRY(cudaGraphLaunch(it->second, s));
    return AP_OK;
}

// Runs Algorithm 1 on every problem of the batch until each has stopped.
// out[b] receives problem b's result; sweep timing is per launch (shared).
static int32_t run_batch(const Problem* P, int count, const ap_params* p, ap_result* out,
                         void* ws, size_t ws_bytes, cudaStream_t s, const Plan& plan) {
    SweepWs w;
    AP_TRY(check_ws(ws, ws_bytes, carve_sweep(nullptr, P, count, plan, nullptr)));
    carve_sweep(ws, P, count, plan, &w);
    const SweepConfig& c = plan.c;
    for (auto& a : w.host) a.lam = p->damping;
    if (p->flags & AP_FLAG_COLD) {
        // R and A start at zero whatever the buffers hold: the first launches
        // read this zeroed buffer instead
        AP_CUDA_TRY(cudaMemsetAsync(w.zero, 0, w.zero_bytes, s));
        for (auto& a : w.host) a.zero = w.zero;
    }
    // the problem table and the work list in force (re-planned as problems finish)
    Plan cur = plan;
    auto upload = [&]() -> int32_t {
        AP_CUDA_TRY(cudaMemcpyAsync(w.table, w.host.data(), sizeof(SweepArgs) * count,
                                    cudaMemcpyHostToDevice, s));
        AP_CUDA_TRY(cudaMemcpyAsync(w.units, cur.units.data(), sizeof(Unit) * cur.units.size(),
                                    cudaMemcpyHostToDevice, s));
        AP_CUDA_TRY(cudaMemcpyAsync(w.ubeg, cur.ubeg.data(), sizeof(int) * cur.ubeg.size(),
                                    cudaMemcpyHostToDevice, s));
        // (pageable sources: each copy has taken its bytes when the call returns)
        return AP_OK;
    };
    AP_TRY(upload());
    const int nmax = plan.nmax;
    const dim3 col_grid((nmax + 255) / 256, count);
    const dim3 fin_grid((nmax + kFinCols - 1) / kFinCols, count);
    sweep_init_kernel<<<col_grid, 256, 0, s>>>(w.table, p->max_iter, p->conv_iter);
    note_launches(1);
    if (!(p->flags & AP_FLAG_S_CHECKED)) {
        nonfinite_kernel<<<dim3(std::min(nmax, 1024), count), 256, 0, s>>>(w.table);
        note_launches(1);
    }
    AP_TRY(last_error());
    std::vector<SweepState> hs(count);
    auto read_states = [&]() -> int32_t {
        AP_CUDA_TRY(cudaMemcpyAsync(hs.data(), w.states, sizeof(SweepState) * count,
                                    cudaMemcpyDeviceToHost, s));
        AP_CUDA_TRY(cudaStreamSynchronize(s));
        return AP_OK;
    };
    AP_TRY(read_states());
    for (int b = 0; b < count; ++b)
        if (hs[b].nonfinite) return AP_ERR_NONFINITE;

    // iterations per host check (at most 64): about 25 ms of sweeping at full
    // bandwidth for one problem -- the stop rule runs on the device, so the
    // launches of a chunk after convergence do no work, while every check
    // costs a host round trip and chunks under 4 iterations run without a
    // graph -- and about 4 ms for a batch, whose work list is rebuilt at a
    // check once a problem has stopped
    std::vector<char> active(count, 1);
    auto chunk_for = [&]() {
        if (p->check_every > 0) return (int)p->check_every;
        double elems = 0.0;
        for (int b = 0; b < count; ++b)
            if (active[b]) elems += (double)P[b].n * (double)P[b].n;
        const double t_iter = 20.0 * elems / 6.0e12 + 6e-6;
        const double target = count == 1 ? 25e-3 : 4e-3;
        return (int)std::min(64.0, std::max(1.0, target / t_iter));
    };
    int chunk = chunk_for();
    const int64_t total = (int64_t)p->max_iter + 1;
    const bool timed = (p->flags & AP_FLAG_TIME_SWEEP) != 0;
    EventPairs ev;
    if (timed) AP_TRY(ev.reserve(std::max(chunk, 64)));
    SweepLaunch L{w.table, w.units, w.ubeg, count, c.W4, c.NS};
    int64_t launched = 0;
    int32_t worked = 0;
    double sweep_ms = 0.0;
    int32_t t_before = 1;
    bool all_done = false;
    const bool graph = !timed && !(p->flags & AP_FLAG_NO_GRAPH);
    while (launched < total) {
        const int64_t m = std::min<int64_t>(chunk, total - launched);
        // a graph pays for its capture only over several iterations
        if (graph && m >= 4) {
            AP_TRY(launch_chunk_graph(c, cur, L, m, fin_grid, s));
        } else {
            for (int64_t j = 0; j < m; ++j) {
                if (timed) AP_CUDA_TRY(cudaEventRecord(ev.start[j], s));
                AP_TRY(launch_sweep(c, cur.clusters, L, s));
                if (timed) AP_CUDA_TRY(cudaEventRecord(ev.stop[j], s));
                finalize_kernel<<<fin_grid, kFinCols * kFinLanes, 0, s>>>(w.table);
            }
        }
        note_launches(2 * (uint64_t)m);
        AP_TRY(last_error());
        launched += m;
        AP_TRY(read_states());
        int32_t tmax = 1;
        all_done = true;
        for (int b = 0; b < count; ++b) {
            if (hs[b].error) return AP_ERR_TIMEOUT;
            tmax = std::max(tmax, hs[b].t);
            all_done = all_done && hs[b].done;
        }
        const int32_t did = tmax - t_before;      // launches of this chunk that did work
        t_before = tmax;
        worked += did;
        if (timed) {
            for (int32_t j = 0; j < did; ++j) {
                float ms = 0.f;
                AP_CUDA_TRY(cudaEventElapsedTime(&ms, ev.start[j], ev.stop[j]));
                sweep_ms += ms;
            }
        }
        if (all_done) break;
        if (count > 1) {
            bool changed = false;
            for (int b = 0; b < count; ++b)
                if (active[b] && hs[b].done) {
                    active[b] = 0;
                    changed = true;
                }
            if (changed) {
                // a new work list over the problems still running, so that no
                // cluster idles on a finished one; nothing is in flight (the
                // states were just read back)
                plan_units(P, count, active, &cur);
                for (int b = 0; b < count; ++b) {
                    w.host[b].G = cur.G[b];
                    w.host[b].pcol = w.pool + (size_t)cur.ufirst[b] * cur.nmax;
                }
                AP_TRY(upload());
                chunk = std::min(chunk_for(), timed ? 64 : 1 << 30);
            }
        }
    }
    if (!all_done) return AP_ERR_CUDA;   // cannot happen: launch max_iter+1 always stops
    int32_t worst = AP_OK;
    for (int b = 0; b < count; ++b) {
        const Problem& q = P[b];
        if (hs[b].final_buf == 1)
            AP_CUDA_TRY(cudaMemcpy2DAsync(q.R, q.ld * sizeof(float), w.host[b].R1,
                                          q.ld * sizeof(float), q.n * sizeof(float), q.n,
                                          cudaMemcpyDeviceToDevice, s));
        const int32_t status = (p->conv_iter > 0 && !hs[b].converged) ? AP_NOT_CONVERGED : AP_OK;
        worst = std::max(worst, status);
        if (out) {
            out[b] = ap_result{};
            out[b].iters = hs[b].iters;
            out[b].converged = hs[b].converged;
            out[b].status = status;
            out[b].sweep_ms = sweep_ms;
            out[b].sweep_launches = worked;
        }
    }
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    return worst;
}

static void fill_public(const SweepConfig& c, ap_sweep_config* o) {
    o->cluster = c.C;
    o->ept = c.EPT;
    o->stages = c.NS;
    o->threads = c.T;
    o->clusters = c.G;
    o->smem_bytes = (int32_t)c.smem;
}

int32_t sweep_workspace(int64_t n, int64_t ld, size_t* bytes) {
    Problem q{nullptr, nullptr, nullptr, n, ld, nullptr};
    if (n < 2 || n > INT_MAX / 4 || ld < n) return AP_ERR_INVALID_ARG;
    Plan plan;
    AP_TRY(make_plan(&q, 1, nullptr, &plan));
    *bytes = carve_sweep(nullptr, &q, 1, plan, nullptr);
    return AP_OK;
}

static int32_t gather_problems(const float* S, float* R, float* A, const int64_t* off,
                               const int64_t* n, const int64_t* ld, int32_t count, int32_t* dec,
                               std::vector<Problem>* P) {
    if (!S || !R || !A || !off || !n || !ld || count < 1) return AP_ERR_INVALID_ARG;
    P->resize(count);
    int64_t doff = 0;
    for (int b = 0; b < count; ++b) {
        Problem& q = (*P)[b];
        q.S = S + off[b];
        q.R = R + off[b];
        q.A = A + off[b];
        q.n = n[b];
        q.ld = ld[b];
        q.dec = dec ? dec + doff : nullptr;
        doff += n[b];
        if (off[b] < 0 || !valid_problem(q)) return AP_ERR_INVALID_ARG;
    }
    return AP_OK;
}

}  // namespace apgb

using namespace apgb;

APGB_API size_t ap_iterate_workspace_size(int64_t n, int64_t ld) {
    size_t b = 0;
    if (sweep_workspace(n, ld, &b) != AP_OK) return 0;
    return b;
}

APGB_API int32_t ap_iterate(const float* S, float* R, float* A, int64_t n, int64_t ld,
                            const ap_params* p, int32_t* decisions, ap_result* out,
                            void* ws, size_t ws_bytes, void* stream) {
    Problem q{S, R, A, n, ld, decisions};
    if (!valid_params(p) || !valid_problem(q)) return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    Plan plan;
    AP_TRY(make_plan(&q, 1, nullptr, &plan));
    return run_batch(&q, 1, p, out, ws, ws_bytes, static_cast<cudaStream_t>(stream), plan);
}

// Size classes of a batch.  A launch configuration is sized for its widest
// rows, and a row costs the same number of bulk copies (and about the same
// time) however narrow it is, so narrow rows run far below the bandwidth
// under a wide configuration (measured: 300-point rows under a 4000-point
// configuration reach about 1 TB/s, under their own about 2.3 TB/s).  The
// batch is therefore split by n at 512 x 2^(j/4) (four classes per octave), a
// class with less work than fills the GPU for about 25 us (8e6 elements)
// joins the next larger one, and the classes run one after another, each with
// its own configuration and the whole GPU.  Problem order within a class is
// kept.  On the 256-problem image batch (n from 200 to 4000) whole-octave
// classes swept at 4.4 TB/s and converged in 0.36 s, half-octave ones at
// 5.6 TB/s in 0.29 s, quarter-octave ones at 5.9 TB/s in 0.26 s; eighths
// gained nothing more, their extra per-class tails eating the gain.
constexpr int kClassesPerOctave = 4;

struct SizeClass {
    std::vector<int> idx;         // problems of the batch
    std::vector<Problem> P;
    Plan plan;
    size_t ws_off = 0, ws_bytes = 0;
    double work = 0.0;            // sum of n^2: the class's elements per iteration
};

// Library-owned streams on which ap_iterate_batched runs its size classes side
// by side (created once per device).
constexpr int kClassStreams = 4;
static std::mutex g_cls_mu;
static std::map<int, std::vector<cudaStream_t>> g_cls_streams;

static int32_t class_streams(std::vector<cudaStream_t>* out) {
    int dev = 0;
    AP_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_cls_mu);
    auto it = g_cls_streams.find(dev);
    if (it == g_cls_streams.end()) {
        std::vector<cudaStream_t> v(kClassStreams);
        for (auto& q : v) AP_CUDA_TRY(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
        it = g_cls_streams.emplace(dev, v).first;
    }
    *out = it->second;
    return AP_OK;
}

// The problems of each class, classes in increasing order of size (host only).
static void split_classes(const Problem* P, int count, std::vector<std::vector<int>>* groups) {
    std::map<int, std::vector<int>> by;
    for (int b = 0; b < count; ++b) {
        // class boundaries at n = 512 x 2^(j / kClassesPerOctave)
        const double x = std::log2((double)P[b].n / 512.0) * kClassesPerOctave;
        const int k = P[b].n <= 512 ? 0 : (int)std::ceil(x - 1e-9);
        by[k].push_back(b);
    }
    groups->clear();
    std::vector<int> carry;
    for (auto it = by.begin(); it != by.end(); ++it) {
        std::vector<int> idx = carry;
        idx.insert(idx.end(), it->second.begin(), it->second.end());
        std::sort(idx.begin(), idx.end());
        double work = 0.0;
        for (int b : idx) work += (double)P[b].n * (double)P[b].n;
        if (work < 8e6 && std::next(it) != by.end()) {
            carry = idx;
            continue;
        }
        carry.clear();
        groups->push_back(idx);
    }
}

static int32_t make_classes(const Problem* P, int count, std::vector<SizeClass>* cls, size_t* total) {
    std::vector<std::vector<int>> groups;
    split_classes(P, count, &groups);
    cls->clear();
    for (const auto& idx : groups) {
        SizeClass c;
        c.idx = idx;
        for (int b : idx) {
            c.P.push_back(P[b]);
            c.work += (double)P[b].n * (double)P[b].n;
        }
        cls->push_back(std::move(c));
    }
    size_t at = 0;
    for (SizeClass& c : *cls) {
        AP_TRY(make_plan(c.P.data(), (int)c.P.size(), nullptr, &c.plan));
        c.ws_off = at;
        c.ws_bytes = carve_sweep(nullptr, c.P.data(), (int)c.P.size(), c.plan, nullptr);
        at = align_up(at + c.ws_bytes, kAlign);
    }
    *total = at;
    return AP_OK;
}

APGB_API int32_t ap_sweep_plan(const int64_t* n, int32_t count, int32_t cluster, int32_t resident,
                              int32_t* units, int32_t cap, int32_t* ubeg, int32_t* n_units,
                              int32_t* n_clusters) {
    if (!n || count < 1 || !units || !ubeg || !n_units || !n_clusters || resident < 1 ||
        cluster < 1 || cluster > kMaxCluster || (cluster & (cluster - 1)))
        return AP_ERR_INVALID_ARG;
    std::vector<Problem> P(count);
    int64_t nmax = 0;
    for (int b = 0; b < count; ++b) {
        if (n[b] < 2 || n[b] > INT_MAX / 4) return AP_ERR_INVALID_ARG;
        P[b] = Problem{nullptr, nullptr, nullptr, n[b], n[b], nullptr};
        nmax = std::max(nmax, n[b]);
    }
    Plan plan;
    plan.c = SweepConfig{};
    plan.c.C = cluster;
    plan.c.R = resident;
    plan.c.G = std::max(1, (int)std::min<int64_t>(resident, nmax));
    plan.nmax = (int)nmax;
    plan_units(P.data(), count, std::vector<char>(count, 1), &plan);
    if ((int64_t)plan.units.size() > cap) return AP_ERR_WORKSPACE;
    for (size_t u = 0; u < plan.units.size(); ++u) {
        const Unit& x = plan.units[u];
        int32_t* o = units + 5 * u;
        o[0] = x.b;
        o[1] = x.g;
        o[2] = x.first;
        o[3] = x.count;
        o[4] = x.stride;
    }
    std::copy(plan.ubeg.begin(), plan.ubeg.end(), ubeg);
    *n_units = (int32_t)plan.units.size();
    *n_clusters = plan.clusters;
    return AP_OK;
}

APGB_API int32_t ap_sweep_classes(const int64_t* n, int32_t count, int32_t* class_of) {
    if (!n || count < 1 || !class_of) return AP_ERR_INVALID_ARG;
    std::vector<Problem> P(count);
    for (int b = 0; b < count; ++b) {
        if (n[b] < 2 || n[b] > INT_MAX / 4) return AP_ERR_INVALID_ARG;
        P[b] = Problem{nullptr, nullptr, nullptr, n[b], n[b], nullptr};
    }
    std::vector<std::vector<int>> groups;
    split_classes(P.data(), count, &groups);
    for (size_t k = 0; k < groups.size(); ++k)
        for (int b : groups[k]) class_of[b] = (int32_t)k;
    return (int32_t)groups.size();
}

APGB_API size_t ap_iterate_batched_workspace_size(const int64_t* n, const int64_t* ld,
                                                  int32_t count) {
    if (!n || !ld || count < 1) return 0;
    if (require_sm103() != AP_OK) return 0;
    std::vector<Problem> P(count);
    for (int b = 0; b < count; ++b) {
        P[b] = Problem{nullptr, nullptr, nullptr, n[b], ld[b], nullptr};
        if (n[b] < 2 || n[b] > INT_MAX / 4 || ld[b] < n[b]) return 0;
    }
    std::vector<SizeClass> cls;
    size_t total = 0;
    if (make_classes(P.data(), count, &cls, &total) != AP_OK) return 0;
    return total;
}

APGB_API int32_t ap_iterate_batched(const float* S, float* R, float* A, const int64_t* offsets,
                                    const int64_t* n, const int64_t* ld, int32_t count,
                                    const ap_params* p, int32_t* decisions, ap_result* out,
                                    void* ws, size_t ws_bytes, void* stream) {
    if (!valid_params(p)) return AP_ERR_INVALID_ARG;
    std::vector<Problem> P;
    AP_TRY(gather_problems(S, R, A, offsets, n, ld, count, decisions, &P));
    AP_TRY(require_sm103());
    std::vector<SizeClass> cls;
    size_t total = 0;
    AP_TRY(make_classes(P.data(), count, &cls, &total));
    AP_TRY(check_ws(ws, ws_bytes, total));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<std::vector<ap_result>> r(cls.size());
    std::vector<int32_t> st(cls.size(), AP_OK);
    auto run_class = [&](size_t i, cudaStream_t cs) {
        r[i].assign(cls[i].P.size(), ap_result{});
        st[i] = run_batch(cls[i].P.data(), (int)cls[i].P.size(), p, r[i].data(),
                          static_cast<char*>(ws) + cls[i].ws_off, cls[i].ws_bytes, cs, cls[i].plan);
    };
    if (cls.size() == 1) {
        run_class(0, s);
    } else {
        // classes run side by side, each on its own stream driven by its own
        // host thread, largest work first: a class's tail (few problems
        // left, clusters idle) overlaps the next classes' work.  Each class
        // owns its workspace region, and a problem's results do not depend
        // on what runs beside it.
        std::vector<cudaStream_t> cs;
        AP_TRY(class_streams(&cs));
        const int workers = (int)std::min(cs.size(), cls.size());
        std::vector<size_t> order(cls.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cls[a].work > cls[b].work; });
        int dev = 0;
        AP_CUDA_TRY(cudaGetDevice(&dev));
        cudaEvent_t fork;
        AP_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        AP_CUDA_TRY(cudaEventRecord(fork, s));
        for (int k = 0; k < workers; ++k) AP_CUDA_TRY(cudaStreamWaitEvent(cs[k], fork, 0));
        cudaEventDestroy(fork);
        std::atomic<size_t> next{0};
        std::vector<std::thread> th;
        for (int k = 0; k < workers; ++k)
            th.emplace_back([&, k]() {
                if (cudaSetDevice(dev) != cudaSuccess) return;
                for (size_t j; (j = next.fetch_add(1)) < order.size();) run_class(order[j], cs[k]);
            });
        for (auto& t : th) t.join();
        // join: the caller's stream continues after every class
        for (int k = 0; k < workers; ++k) {
            cudaEvent_t e;
            AP_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            AP_CUDA_TRY(cudaEventRecord(e, cs[k]));
            AP_CUDA_TRY(cudaStreamWaitEvent(s, e, 0));
            cudaEventDestroy(e);
        }
        if (next.load() < order.size()) return AP_ERR_CUDA;    // a worker could not start
    }
    int32_t worst = AP_OK;
    for (size_t i = 0; i < cls.size(); ++i) {
        if (st[i] < 0) return st[i];
        worst = std::max(worst, st[i]);
        if (out)
            for (size_t j = 0; j < cls[i].idx.size(); ++j) out[cls[i].idx[j]] = r[i][j];
    }
    return worst;
}

APGB_API int32_t ap_sweep_get_config(int64_t n, ap_sweep_config* out) {
    if (!out || n < 2 || n > INT_MAX / 4) return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    SweepConfig c;
    AP_TRY(choose_config((int)n, &c));
    *out = ap_sweep_config{};
    fill_public(c, out);
    return AP_OK;
}

APGB_API int32_t ap_sweep_set_config(int64_t n, const ap_sweep_config* cfg) {
    if (n < 2 || n > INT_MAX / 4) return AP_ERR_INVALID_ARG;
    if (!cfg) {
        std::lock_guard<std::mutex> lock(g_pin_mu);
        g_pinned.erase(n);
        return AP_OK;
    }
    AP_TRY(require_sm103());
    SweepConfig c;
    AP_TRY(make_config((int)n, cfg->cluster, cfg->ept, cfg->stages, &c));
    std::lock_guard<std::mutex> lock(g_pin_mu);
    g_pinned[n] = {cfg->cluster, cfg->ept, cfg->stages};
    return AP_OK;
}

static void for_each_candidate(int n, const std::function<void(const SweepConfig&)>& f) {
    for (int C = 1; C <= kMaxCluster; ++C)
        for (int ept = 1; ept <= 4; ++ept)
            for (int ns = 2; ns <= kMaxStages; ++ns) {
                SweepConfig c;
                if (make_config(n, C, ept, ns, &c) == AP_OK) f(c);
            }
}

APGB_API size_t ap_sweep_autotune_workspace_size(int64_t n, int64_t ld) {
    if (n < 2 || n > INT_MAX / 4 || ld < n) return 0;
    if (require_sm103() != AP_OK) return 0;
    Problem q{nullptr, nullptr, nullptr, n, ld, nullptr};
    size_t best = 0;
    for_each_candidate((int)n, [&](const SweepConfig& c) {
        Plan plan;
        if (make_plan(&q, 1, &c, &plan) == AP_OK)
            best = std::max(best, carve_sweep(nullptr, &q, 1, plan, nullptr));
    });
    return best;
}

APGB_API int32_t ap_sweep_autotune(const float* S, float* R, float* A, int64_t n, int64_t ld,
                                   float damping, int32_t iters, ap_sweep_config* best,
                                   void* ws, size_t ws_bytes, void* stream) {
    Problem q{S, R, A, n, ld, nullptr};
    if (!best || !valid_problem(q) || iters < 1 || !(damping >= 0.f && damping < 1.f))
        return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<SweepConfig> cands;
    for_each_candidate((int)n, [&](const SweepConfig& c) { cands.push_back(c); });
    if (cands.empty()) return AP_ERR_UNSUPPORTED;
    ap_params p{damping, iters, 0, iters + 1, AP_FLAG_TIME_SWEEP};
    double best_ms = 1e300;
    SweepConfig best_c = cands[0];
    for (const SweepConfig& c : cands) {
        AP_CUDA_TRY(cudaMemset2DAsync(R, ld * sizeof(float), 0, n * sizeof(float), n, s));
        AP_CUDA_TRY(cudaMemset2DAsync(A, ld * sizeof(float), 0, n * sizeof(float), n, s));
        Plan plan;
        AP_TRY(make_plan(&q, 1, &c, &plan));
        ap_result r;
        const int32_t st = run_batch(&q, 1, &p, &r, ws, ws_bytes, s, plan);
        if (st < 0) return st;
        const double per = r.sweep_ms / std::max(1, r.sweep_launches);
        if (per < best_ms) {
            best_ms = per;
            best_c = c;
        }
    }
    {
        std::lock_guard<std::mutex> lock(g_pin_mu);
        g_pinned[n] = {best_c.C, best_c.EPT, best_c.NS};
    }
    *best = ap_sweep_config{};
    fill_public(best_c, best);
    best->ms_per_iter = (float)best_ms;
    return AP_OK;
}

// ---------------------------------------------------------------------------
// Row shards: Algorithm 1 with the rows of S, R and A split between several
// devices.  The responsibility half of an iteration and the availability
// half are row-local given the column vectors colp and c = r(k,k) + colp; a
// shard sweeps its own rows with the kernel above (its work list names only
// its rows, and its buffers are addressed from where global row 0 would be),
// exports its share of the column sums, its diagonal responsibilities and its
// decision counts, and the caller sums those over the shards (one all-reduce
// of 2n + 2 floats per iteration) before the stop rule is applied to the
// totals, identically on every shard.
// ---------------------------------------------------------------------------
namespace apgb {

// A shard's share of the column sums in the fixed order of finalize_kernel,
// with its r(k,k) (zero off its rows) and its decision counts: red = (colp
// share [n], r(k,k) share [n], exemplar-set changes, exemplars).
__global__ void __launch_bounds__(kFinCols * kFinLanes) shard_reduce_kernel(const SweepArgs* __restrict__ table,
                                                                           float* red) {
    const SweepArgs& a = table[0];
    const int cx = threadIdx.x % kFinCols, gy = threadIdx.x / kFinCols;
    const int k = blockIdx.x * kFinCols + cx;
    __shared__ float part[kFinLanes][kFinCols];
    float s = 0.f;
    if (k < a.n) {
#pragma unroll 4
        for (int g = gy; g < a.G; g += kFinLanes) s += a.pcol[(int64_t)g * a.pstride + k];
    }
    part[gy][cx] = s;
    __syncthreads();
    if (gy == 0 && k < a.n) {
        red[k] = lane_tree(part, cx);
        red[a.n + k] = a.rkk[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        red[2 * a.n] = (float)a.st->changes;
        red[2 * a.n + 1] = (float)a.st->n_ex;
    }
}

// The summed values back into the iteration: colp, c = r(k,k) + colp and the
// stop rule on the total counts.
__global__ void shard_finish_kernel(const SweepArgs* __restrict__ table, const float* __restrict__ red) {
    const SweepArgs& a = table[0];
    SweepState* st = a.st;
    if (st->done) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < a.n) {
        const_cast<float*>(a.colp)[k] = red[k];
        const_cast<float*>(a.cvec)[k] = red[a.n + k] + red[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->changes = (int32_t)red[2 * a.n];
        st->n_ex = (int32_t)red[2 * a.n + 1];
        apply_stop_rule(st);
    }
}

__global__ void shard_nonfinite_kernel(const float* __restrict__ S, int64_t m, int n, int64_t ld,
                                       SweepState* st) {
    int local = 0;
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x)
        for (int k = threadIdx.x; k < n; k += blockDim.x)
            if (!isfinite(S[i * ld + k])) ++local;
    local = __reduce_add_sync(0xffffffffu, local);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(&st->nonfinite, local);
}

struct ShardWs {
    SweepArgs* table;
    Unit* units;
    int* ubeg;
    float* pool;
    SweepState* st;
    float *R1, *colp, *cvec, *rkk;
    int32_t* eflag;
};

// The shard's launch configuration (chosen for rows of n columns) and its
// work list: the interleaved units of its m rows, moved to global rows r0...
static int32_t shard_plan(int64_t n, int64_t r0, int64_t r1, Plan* plan) {
    AP_TRY(choose_config((int)n, &plan->c));
    plan->nmax = (int)n;
    const Problem rows{nullptr, nullptr, nullptr, r1 - r0, r1 - r0, nullptr};
    std::vector<char> active(1, 1);
    plan_units(&rows, 1, active, plan);
    for (Unit& u : plan->units) u.first += (int)r0;
    return AP_OK;
}

static size_t carve_shard(void* ws, int64_t n, int64_t ld, int64_t m, const Plan& plan, ShardWs* w) {
    Carver cv(ws);
    w->table = cv.take<SweepArgs>(1);
    w->units = cv.take<Unit>(max_units(1, plan.c));
    w->ubeg = cv.take<int>((size_t)std::max(plan.c.R, 1) + 1);
    w->pool = cv.take<float>(max_units(1, plan.c) * (size_t)n);
    w->st = cv.take<SweepState>(1);
    w->R1 = cv.take<float>((size_t)m * ld);
    w->colp = cv.take<float>(n);
    w->cvec = cv.take<float>(n);
    w->rkk = cv.take<float>(n);
    w->eflag = cv.take<int32_t>(n);
    return cv.used;
}

// The shard's problem table entry: buffers addressed from global row 0 (only
// rows r0 .. r1-1 are ever touched).
static SweepArgs shard_args(const float* S, float* R, float* A, int64_t n, int64_t ld, int64_t r0,
                            const ap_params* p, int32_t* dec, const Plan& plan, const ShardWs& w) {
    SweepArgs a{};
    const int64_t back = r0 * ld;
    a.S = S - back;
    a.R0 = R - back;
    a.R1 = w.R1 - back;
    a.A = A - back;
    a.ld = ld;
    a.n = (int)n;
    a.n4 = (int)((n + 3) / 4);
    a.w4 = (a.n4 + plan.c.C - 1) / plan.c.C;
    a.G = plan.G[0];
    a.ns = plan.c.NS;
    a.lam = p->damping;
    a.spin_limit = 1u << 20;
    a.cvec = w.cvec;
    a.colp = w.colp;
    a.pcol = w.pool;
    a.pstride = n;
    a.rkk = w.rkk;
    a.eflag = w.eflag;
    a.dec = dec ? dec - r0 : nullptr;
    a.st = w.st;
    return a;
}

static bool shard_args_ok(const float* S, const float* R, const float* A, int64_t n, int64_t ld,
                          int64_t r0, int64_t r1) {
    return S && R && A && n >= 2 && n <= INT_MAX / 4 && ld >= n && !(ld & 3) && r0 >= 0 && r1 > r0 &&
           r1 <= n && aligned16(S) && aligned16(R) && aligned16(A);
}

}  // namespace apgb

APGB_API size_t ap_shard_workspace_size(int64_t n, int64_t ld, int64_t r0, int64_t r1) {
    if (n < 2 || n > INT_MAX / 4 || ld < n || r0 < 0 || r1 <= r0 || r1 > n) return 0;
    Plan plan;
    if (shard_plan(n, r0, r1, &plan) != AP_OK) return 0;
    ShardWs w;
    return carve_shard(nullptr, n, ld, r1 - r0, plan, &w);
}

APGB_API int32_t ap_shard_begin(const float* S, float* R, float* A, int64_t n, int64_t ld, int64_t r0,
                                int64_t r1, const ap_params* params, int32_t* decisions, void* ws,
                                size_t ws_bytes, void* stream) {
    if (!shard_args_ok(S, R, A, n, ld, r0, r1) || !valid_params(params)) return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Plan plan;
    AP_TRY(shard_plan(n, r0, r1, &plan));
    ShardWs w;
    AP_TRY(check_ws(ws, ws_bytes, carve_shard(nullptr, n, ld, r1 - r0, plan, &w)));
    carve_shard(ws, n, ld, r1 - r0, plan, &w);
    const SweepArgs a = shard_args(S, R, A, n, ld, r0, params, decisions, plan, w);
    AP_CUDA_TRY(cudaMemcpyAsync(w.table, &a, sizeof(SweepArgs), cudaMemcpyHostToDevice, s));
    AP_CUDA_TRY(cudaMemcpyAsync(w.units, plan.units.data(), sizeof(Unit) * plan.units.size(),
                                cudaMemcpyHostToDevice, s));
    AP_CUDA_TRY(cudaMemcpyAsync(w.ubeg, plan.ubeg.data(), sizeof(int) * plan.ubeg.size(),
                                cudaMemcpyHostToDevice, s));
    AP_CUDA_TRY(cudaMemsetAsync(w.rkk, 0, sizeof(float) * n, s));
    sweep_init_kernel<<<dim3((unsigned)((n + 255) / 256), 1), 256, 0, s>>>(w.table, params->max_iter,
                                                                           params->conv_iter);
    shard_nonfinite_kernel<<<(int)std::min<int64_t>(r1 - r0, 1024), 256, 0, s>>>(S, r1 - r0, (int)n, ld, w.st);
    note_launches(2);
    AP_TRY(last_error());
    SweepState h;
    AP_CUDA_TRY(cudaMemcpyAsync(&h, w.st, sizeof(SweepState), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    return h.nonfinite ? AP_ERR_NONFINITE : AP_OK;
}

APGB_API int32_t ap_shard_sweep(const float* S, float* R, float* A, int64_t n, int64_t ld, int64_t r0,
                                int64_t r1, const ap_params* params, int32_t* decisions, float* red,
                                void* ws, size_t ws_bytes, void* stream) {
    if (!shard_args_ok(S, R, A, n, ld, r0, r1) || !valid_params(params) || !red) return AP_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Plan plan;
    AP_TRY(shard_plan(n, r0, r1, &plan));
    ShardWs w;
    AP_TRY(check_ws(ws, ws_bytes, carve_shard(nullptr, n, ld, r1 - r0, plan, &w)));
    carve_shard(ws, n, ld, r1 - r0, plan, &w);
    const SweepConfig& c = plan.c;
    const SweepLaunch L{w.table, w.units, w.ubeg, 1, c.W4, c.NS};
    AP_TRY(launch_sweep(c, plan.clusters, L, s));
    shard_reduce_kernel<<<(unsigned)((n + kFinCols - 1) / kFinCols), kFinCols * kFinLanes, 0, s>>>(w.table, red);
    note_launches(2);
    return last_error();
}

APGB_API int32_t ap_shard_finish(const float* S, float* R, float* A, int64_t n, int64_t ld, int64_t r0,
                                 int64_t r1, const ap_params* params, int32_t* decisions, const float* red,
                                 int32_t* done, ap_result* out, void* ws, size_t ws_bytes, void* stream) {
    if (!shard_args_ok(S, R, A, n, ld, r0, r1) || !valid_params(params) || !red || !done)
        return AP_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Plan plan;
    AP_TRY(shard_plan(n, r0, r1, &plan));
    ShardWs w;
    AP_TRY(check_ws(ws, ws_bytes, carve_shard(nullptr, n, ld, r1 - r0, plan, &w)));
    carve_shard(ws, n, ld, r1 - r0, plan, &w);
    shard_finish_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w.table, red);
    note_launches(1);
    AP_TRY(last_error());
    SweepState h;
    AP_CUDA_TRY(cudaMemcpyAsync(&h, w.st, sizeof(SweepState), cudaMemcpyDeviceToHost, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    if (h.error) return AP_ERR_TIMEOUT;
    *done = h.done;
    if (!h.done) return AP_OK;
    const int64_t m = r1 - r0;
    if (h.final_buf == 1)
        AP_CUDA_TRY(cudaMemcpy2DAsync(R, ld * sizeof(float), w.R1, ld * sizeof(float), n * sizeof(float), m,
                                      cudaMemcpyDeviceToDevice, s));
    AP_CUDA_TRY(cudaStreamSynchronize(s));
    const int32_t status = (params->conv_iter > 0 && !h.converged) ? AP_NOT_CONVERGED : AP_OK;
    if (out) {
        *out = ap_result{};
        out->iters = h.iters;
        out->converged = h.converged;
        out->status = status;
    }
    return status;
}
