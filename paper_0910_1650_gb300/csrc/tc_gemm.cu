// Tensor-core (tcgen05) GEMMs with fused epilogues, for the dense
// contractions of the method:
//   * similarity:  s(i,k) = 2 x_i . x_k - |x_i|^2 - |x_k|^2, clamped to <= 0
//                  (Section 2, s(i,k) = -|x_i - x_k|^2), written as float32;
//   * assignment:  c_i = argmax_j (2 x_i . e_j - |e_j|^2) over the exemplars
//                  e_j (Algorithm 3 Step 2: nearest centre), never writing the
//                  N x c score matrix.
// Operands are bf16, K-major, loaded by TMA with 128-byte swizzle; the
// product accumulates in fp32 in tensor memory.
//
// Persistent, warp-specialised kernel (one CTA per SM, 320 threads), launched
// as clusters of two CTAs that compute vertically adjacent tiles (row blocks
// 2p and 2p+1) against the same column block:
//   warp 0      TMA producer: this CTA's A tile (128 x 64) and one half of the
//               shared B tile (128 of its 256 rows), the half multicast into
//               both CTAs' shared memory, into a 3-stage ring (mbarriers
//               full/empty); a stage is refilled once both CTAs' MMAs have
//               released it (their commits are multicast onto both "empty"s);
//   warp 1      allocates 512 TMEM columns and issues tcgen05.mma
//               (M=128, N=256, K=16) from one elected thread into two
//               256-column accumulators (mbarriers tfull/tempty);
//   warps 2..9  epilogue, two warps per TMEM lane quarter (column halves):
//               tcgen05.ld, the fused arithmetic, then either swizzled shared
//               memory -> TMA tensor store (similarity) or a running per-row
//               arg-max (assignment).
// Multicasting the shared operand cuts each CTA's operand stream from 48 KB
// to 32 KB per K step.
// Every mbarrier wait is bounded; on expiry the kernel records an error and
// all roles stop issuing new work.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cooperative_groups.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "common.cuh"
#include "ptx.cuh"

namespace apgb {
namespace tc {

constexpr int BM = 128, BN = 256, BK = 64;
constexpr int STAGES = 3;
constexpr int A_BYTES = BM * BK * 2;            // 16 KB
constexpr int B_BYTES = BN * BK * 2;            // 32 KB
constexpr int OUT_COLS = 32;                    // fp32 columns per store chunk (128 B)
constexpr int OUT_BYTES = BM * OUT_COLS * 4;    // 16 KB
constexpr int EPI_WARPS = 8;                    // two per TMEM lane quarter: column halves
constexpr int THREADS = 64 + 32 * EPI_WARPS;    // producer, MMA issuer, epilogue
constexpr uint32_t TMEM_COLS = 512;

enum Mode : int { SIM = 0, ARGMAX = 1 };

struct Smem {
    uint8_t a[STAGES][A_BYTES];
    uint8_t b[STAGES][B_BYTES];
    uint8_t out[2][2][OUT_BYTES];   // [column half][double buffer]
    float hbest[BM];                // ARGMAX: the second half's row results
    int hidx[BM];
    float bnrm[2][BN];              // |b_k|^2 of the columns of the tile, by accumulator
    uint64_t full[STAGES], empty[STAGES], tfull[2], tempty[2], mma_done;
    uint32_t tmem_base;
    int abort;                      // any role gave up a bounded wait
    int ep_abort;                   // the epilogue's copy, published at its barriers
};

__device__ __forceinline__ bool aborted(const Smem& sm) {
    return *reinterpret_cast<const volatile int*>(&sm.abort) != 0;
}
constexpr size_t SMEM_BYTES = sizeof(Smem) + 1024;     // + alignment slack

struct Params {
    int M, N, K;                    // rows of A, rows of B, padded K (multiple of 64)
    int mode;
    const float* anrm;              // |a_i|^2 (length >= M)
    const float* bnrm;              // |b_k|^2 (length >= N)
    int32_t* arg;                   // ARGMAX: best column per row
    float* best;                    // ARGMAX: best score per row (may be null)
    int diag_zero;                  // SIM: write 0 where row == column
    // SIM: the tensor store covers columns [0, n4), n4 = N rounded down to a
    // multiple of 4 (a TMA store writes whole 16-byte granules at the right
    // edge of the tensor, which would reach into the caller's columns >= N);
    // columns [n4, N) are written by plain stores to out (row stride lds).
    int n4;
    float* out;
    int64_t lds;
    uint32_t spin_limit;
    int32_t* error;
};

// ---- PTX wrappers specific to tcgen05 and tensor TMA ------------------------
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3}], [%4];" ::"r"(ptx::smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(ptx::smem_u32(bar))
        : "memory");
}

// The same load delivered to the same shared-memory offset (and mbarrier) of
// every CTA of the cluster in `mask`.
__device__ __forceinline__ void tma_load_2d_mc(void* dst, const CUtensorMap* map, int x, int y,
                                               uint64_t* bar, uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster "
        "[%0], [%1, {%2, %3}], [%4], %5;" ::"r"(ptx::smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(ptx::smem_u32(bar)), "h"(mask)
        : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     map),
                 "r"(x), "r"(y), "r"(ptx::smem_u32(src))
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     ptx::smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, M=128, N=256, K=16, bf16 -> fp32.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrives on `bar` of every CTA in `mask` once every tcgen05.mma issued so far
// by this thread is done.
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
        "[%0], %1;" ::"r"(ptx::smem_u32(bar)), "h"(mask)
        : "memory");
}

// Arrives on `bar` once every tcgen05.mma issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            ptx::smem_u32(bar))
        : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 lanes (one row each).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void named_barrier(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Shared-memory matrix descriptor of a K-major bf16 tile with 128-byte
// swizzle: rows of 64 elements (128 B), 8-row swizzle atoms 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(const void* base) {
    const uint64_t addr = ptx::smem_u32(base);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;                // start address
    d |= (uint64_t)0 << 16;                      // leading byte offset (unused: swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                      // descriptor version
    d |= (uint64_t)2 << 61;                      // layout: 128-byte swizzle
    return d;
}

// Instruction descriptor: kind::f16 with bf16 A/B, fp32 D, both K-major.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
    return (1u << 4)                  // D format: f32
           | (1u << 7)                // A format: bf16
           | (1u << 10)               // B format: bf16
           | ((uint32_t)(n >> 3) << 17)
           | ((uint32_t)(m >> 4) << 24);
}

__global__ void __launch_bounds__(THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmOut, Params p) {
    extern __shared__ uint8_t smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cooperative_groups::cluster_group cluster = cooperative_groups::this_cluster();
    const int crank = (int)cluster.block_rank();          // 0 or 1: row block 2p + crank
    const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
    constexpr uint16_t kPair = 0x3;                        // both CTAs of the cluster

    const int numM = (p.M + BM - 1) / BM;
    const int numMp = (numM + 1) / 2;                      // row-block pairs
    const int numN = (p.N + BN - 1) / BN;
    const int numK = p.K / BK;
    // work units of a pair: one tile pair (SIM) or one row-block pair with all
    // its column tiles (ARGMAX); a pair's second row block may lie past the end
    // (zero-filled loads, no outputs)
    const int units = (p.mode == SIM) ? numMp * numN : numMp;
    const int tiles_per_unit = (p.mode == SIM) ? 1 : numN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            ptx::mbar_init(&sm.full[s], 1);
            ptx::mbar_init(&sm.empty[s], 2);               // one commit from each CTA's MMAs
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&sm.tfull[b], 1);
            ptx::mbar_init(&sm.tempty[b], EPI_WARPS);
        }
        ptx::mbar_init(&sm.mma_done, 1);
        ptx::fence_mbar_init();
        sm.abort = 0;
        sm.ep_abort = 0;
    }
    if (warp == 1) tmem_alloc(&sm.tmem_base, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    cluster.sync();                                        // the peer's barriers exist
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;

    auto tile_mn = [&](int u, int q, int& m, int& n) {
        if (p.mode == SIM) { m = 2 * (u / numN) + crank; n = u % numN; }
        else { m = 2 * u + crank; n = q; }
    };

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t eph = 0x7u;                    // empty barriers start "released"
            uint32_t armed = 0;                     // loads issued per stage (low bit = parity)
            int nissued = 0;
            for (int u = pair; u < units && !aborted(sm); u += npairs) {
                for (int q = 0; q < tiles_per_unit && !aborted(sm); ++q) {
                    int m, n;
                    tile_mn(u, q, m, n);
                    for (int kb = 0; kb < numK; ++kb) {
                        if (!ptx::mbar_wait(&sm.empty[stage], (eph >> stage) & 1u, p.spin_limit)) {
                            atomicExch(&sm.abort, 1);
                            break;
                        }
                        eph ^= 1u << stage;
                        ptx::mbar_arrive_expect_tx(&sm.full[stage], A_BYTES + B_BYTES);
                        // own A tile; this CTA's half of the shared B tile, into both CTAs
                        tma_load_2d(sm.a[stage], &tmA, kb * BK, m * BM, &sm.full[stage]);
                        tma_load_2d_mc(sm.b[stage] + crank * (B_BYTES / 2), &tmB, kb * BK,
                                       n * BN + crank * (BN / 2), &sm.full[stage], kPair);
                        armed ^= 1u << stage;
                        ++nissued;
                        stage = (stage + 1) % STAGES;
                    }
                }
            }
            // loads still in flight must land before shared memory is released
            for (int s = 0; s < STAGES && s < nissued; ++s)
                ptx::mbar_wait(&sm.full[s], ((armed >> s) & 1u) ^ 1u, p.spin_limit);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = instr_desc(BM, BN);
            int stage = 0, acc = 0;
            uint32_t fph = 0, tph = 3;              // tempty barriers start "released"
            for (int u = pair; u < units && !aborted(sm); u += npairs) {
                for (int q = 0; q < tiles_per_unit && !aborted(sm); ++q) {
                    if (!ptx::mbar_wait(&sm.tempty[acc], (tph >> acc) & 1u, p.spin_limit)) {
                        atomicExch(&sm.abort, 1);
                        break;
                    }
                    tph ^= 1u << acc;
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(acc * BN);
                    for (int kb = 0; kb < numK; ++kb) {
                        if (!ptx::mbar_wait(&sm.full[stage], (fph >> stage) & 1u, p.spin_limit)) {
                            atomicExch(&sm.abort, 1);
                            break;
                        }
                        fph ^= 1u << stage;
                        tc_fence_after();
                        const uint64_t ad = smem_desc(sm.a[stage]);
                        const uint64_t bd = smem_desc(sm.b[stage]);
#pragma unroll
                        for (int k = 0; k < BK / 16; ++k) {
                            // advance 16 bf16 (32 B) along K inside the swizzle atom
                            mma_bf16(d, ad + (uint64_t)(k * 2), bd + (uint64_t)(k * 2), idesc,
                                     (kb > 0 || k > 0) ? 1u : 0u);
                        }
                        // frees the stage (in both CTAs: the peer's B half lands in it too)
                        mma_commit_mc(&sm.empty[stage], kPair);
                        stage = (stage + 1) % STAGES;
                    }
                    mma_commit(&sm.tfull[acc]);        // accumulator ready for the epilogue
                    acc ^= 1;
                }
            }
            // no MMA may still write tensor memory when it is released
            mma_commit(&sm.mma_done);
            ptx::mbar_wait(&sm.mma_done, 0, p.spin_limit);
        }
    } else {
        // ---------------- epilogue (warps 2..9) ----------------
        // Warp w reads TMEM lane quarter w % 4 (its rows) and column half
        // (w - 2) / 4 of each 256-column accumulator: two warps per quarter.
        const int sub = warp & 3;                    // TMEM lane quarter this warp may access
        const int half = (warp - 2) >> 2;            // column half: chunks 4*half .. 4*half+3
        const int et = threadIdx.x - 64;             // 0..255
        const int eth = et & 127;                    // within the half
        const int hbar = 2 + half;                   // named barrier of the half (128 threads)
        const int row_in_tile = sub * 32 + lane;
        int acc = 0;
        uint32_t tph = 0;
        int ob = 0;
        for (int u = pair; u < units; u += npairs) {
            float best = -INFINITY;
            int bidx = INT_MAX;
            int m0 = 0;
            for (int q = 0; q < tiles_per_unit; ++q) {
                int m, n;
                tile_mn(u, q, m, n);
                m0 = m;
                // column norms of this tile, staged once per tile
                for (int c = et; c < BN; c += 32 * EPI_WARPS) {
                    const int k = n * BN + c;
                    sm.bnrm[acc][c] = (k < p.N) ? p.bnrm[k] : 0.f;
                }
                // one thread waits (bounded) and publishes the outcome, so that
                // all epilogue warps leave the loop at the same barrier
                if (et == 0) {
                    const bool ok = ptx::mbar_wait(&sm.tfull[acc], (tph >> acc) & 1u, p.spin_limit);
                    if (!ok || aborted(sm)) {
                        sm.ep_abort = 1;
                        atomicExch(&sm.abort, 1);
                    }
                }
                tph ^= 1u << acc;
                named_barrier(1, 32 * EPI_WARPS);
                if (*reinterpret_cast<volatile int*>(&sm.ep_abort)) break;
                tc_fence_after();
                const int i = m * BM + row_in_tile;
                const float ai = (i < p.M) ? p.anrm[i] : 0.f;
                const uint32_t tbase = tmem + (uint32_t)(acc * BN) + ((uint32_t)(sub * 32) << 16);
                for (int c = 4 * half; c < 4 * half + 4; ++c) {
                    float v[32];
                    tmem_ld32(tbase + (uint32_t)(c * OUT_COLS), v);
                    if (p.mode == SIM) {
                        // output chunk c: wait until this half's store of two chunks
                        // ago has left the buffer
                        if (eth == 0) ptx::bulk_wait_read<1>();
                        named_barrier(hbar, 128);
                        uint8_t* buf = sm.out[half][ob];
#pragma unroll
                        for (int u4 = 0; u4 < 8; ++u4) {
                            float o[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int col = c * OUT_COLS + u4 * 4 + e;
                                const int k = n * BN + col;
                                const float sv = fminf(0.f, 2.f * v[u4 * 4 + e] - ai - sm.bnrm[acc][col]);
                                o[e] = (p.diag_zero && k == i) ? 0.f : sv;
                            }
                            const int phys = u4 ^ (row_in_tile & 7);
                            *reinterpret_cast<float4*>(buf + row_in_tile * 128 + phys * 16) =
                                make_float4(o[0], o[1], o[2], o[3]);
                        }
                        const int c0 = n * BN + c * OUT_COLS;     // first column of the chunk
                        if (c0 + OUT_COLS > p.n4 && c0 < p.N && i < p.M) {
                            // the ragged columns [n4, N) of this row
#pragma unroll
                            for (int e = 0; e < OUT_COLS; ++e) {
                                const int k = c0 + e;
                                if (k >= p.n4 && k < p.N)
                                    p.out[(int64_t)i * p.lds + k] =
                                        (p.diag_zero && k == i)
                                            ? 0.f
                                            : fminf(0.f, 2.f * v[e] - ai - sm.bnrm[acc][c * OUT_COLS + e]);
                            }
                        }
                        ptx::fence_proxy_async_smem();
                        named_barrier(hbar, 128);
                        if (eth == 0) {
                            if (c0 < p.n4) {
                                tma_store_2d(&tmOut, c0, m * BM, buf);
                            }
                            ptx::bulk_commit();
                        }
                        ob ^= 1;
                    } else {
#pragma unroll
                        for (int e = 0; e < 32; ++e) {
                            const int col = c * OUT_COLS + e;
                            const int k = n * BN + col;
                            const float sc = 2.f * v[e] - sm.bnrm[acc][col];
                            if (k < p.N && sc > best) { best = sc; bidx = k; }
                        }
                    }
                }
                // accumulator drained: hand it back to the MMA warp
                tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&sm.tempty[acc]);
                acc ^= 1;
            }
            if (*reinterpret_cast<volatile int*>(&sm.ep_abort)) break;
            if (p.mode == ARGMAX) {
                // merge the two column halves of each row: the larger score,
                // the lower column on a tie
                if (half == 1) {
                    sm.hbest[row_in_tile] = best;
                    sm.hidx[row_in_tile] = bidx;
                }
                named_barrier(1, 32 * EPI_WARPS);
                if (half == 0) {
                    const float b1 = sm.hbest[row_in_tile];
                    const int i1 = sm.hidx[row_in_tile];
                    if (b1 > best || (b1 == best && i1 < bidx)) { best = b1; bidx = i1; }
                    const int i = m0 * BM + row_in_tile;
                    if (i < p.M) {
                        p.arg[i] = bidx;
                        if (p.best) p.best[i] = best;
                    }
                }
                named_barrier(1, 32 * EPI_WARPS);   // the merge area is reused next unit
            }
        }
        if (eth == 0) ptx::bulk_wait_all();
    }

    tc_fence_before();
    __syncthreads();
    // neither CTA leaves while the other may still multicast into it or
    // arrive on its barriers
    cluster.sync();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
    if (threadIdx.x == 0 && aborted(sm) && p.error) atomicExch(p.error, 1);
}

// ---- host side ----------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2-D row-major map: `rows` x `cols` elements, row pitch `pitch_bytes`.
static int32_t make_map(CUtensorMap* map, CUtensorMapDataType dt, void* base, uint64_t cols,
                        uint64_t rows, uint64_t pitch_bytes, uint32_t box_cols, uint32_t box_rows,
                        CUtensorMapSwizzle sw) {
    auto fn = encode_fn();
    if (!fn) return AP_ERR_CUDA;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {pitch_bytes};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? AP_OK : AP_ERR_CUDA;
}

static int32_t launch(const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& o,
                      const Params& p, int units, cudaStream_t s) {
    int sms = 0;
    AP_TRY(device_sm_count(&sms));
    AP_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SMEM_BYTES));
    // clusters of two CTAs over row-block pairs, as many as can be resident
    // at once (persistent: each takes every `pairs`-th unit)
    static std::mutex mu;
    static int resident[64] = {0};
    int dev = 0;
    AP_CUDA_TRY(cudaGetDevice(&dev));
    int cap = sms / 2;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (dev >= 0 && dev < 64) {
            if (resident[dev] == 0) {
                cudaLaunchConfig_t q = {};
                q.gridDim = dim3(2, 1, 1);
                q.blockDim = dim3(THREADS, 1, 1);
                q.dynamicSmemBytes = SMEM_BYTES;
                cudaLaunchAttribute qa;
                qa.id = cudaLaunchAttributeClusterDimension;
                qa.val.clusterDim.x = 2;
                qa.val.clusterDim.y = 1;
                qa.val.clusterDim.z = 1;
                q.attrs = &qa;
                q.numAttrs = 1;
                int num = 0;
                if (cudaOccupancyMaxActiveClusters(&num, tc_gemm_kernel, &q) != cudaSuccess || num < 1) {
                    cudaGetLastError();
                    num = sms / 2;
                }
                resident[dev] = num;
            }
            cap = std::min(cap, resident[dev]);
        }
    }
    const int pairs = std::max(1, std::min(units, cap));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * pairs, 1, 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    AP_CUDA_TRY(cudaLaunchKernelEx(&cfg, tc_gemm_kernel, a, b, o, p));
    note_launches(1);
    return last_error();
}

}  // namespace tc

size_t tc_similarity_pad_rows() { return tc::BN; }

// S = -|xi - xk|^2 from bf16 features Xb [npad x dpad] (dpad % 64 == 0,
// rows >= n zero) and fp32 norms of the bf16 rows; diagonal written as 0.
int32_t tc_similarity_bf16(const __nv_bfloat16* Xb, const float* nrm, int n, int dpad, float* S,
                           int64_t lds, int32_t* err, cudaStream_t s) {
    using namespace tc;
    if (dpad % BK || (lds & 3) || !aligned16(S)) return AP_ERR_INVALID_ARG;
    const int npad = (n + BN - 1) / BN * BN;
    CUtensorMap ma, mb, mo;
    AP_TRY(make_map(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (void*)Xb, dpad, npad, (uint64_t)dpad * 2,
                    BK, BM, CU_TENSOR_MAP_SWIZZLE_128B));
    AP_TRY(make_map(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (void*)Xb, dpad, npad, (uint64_t)dpad * 2,
                    BK, BN / 2, CU_TENSOR_MAP_SWIZZLE_128B));
    const int n4 = n & ~3;
    AP_TRY(make_map(&mo, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, S, (uint64_t)std::max(n4, 4), (uint64_t)n,
                    (uint64_t)lds * 4, OUT_COLS, BM, CU_TENSOR_MAP_SWIZZLE_128B));
    Params p{};
    p.M = n;
    p.N = n;
    p.K = dpad;
    p.mode = SIM;
    p.anrm = nrm;
    p.bnrm = nrm;
    p.diag_zero = 1;
    p.n4 = n4;
    p.out = S;
    p.lds = lds;
    p.spin_limit = 1u << 22;
    p.error = err;
    const int units = (((n + BM - 1) / BM + 1) / 2) * ((n + BN - 1) / BN);   // tile pairs
    return launch(ma, mb, mo, p, units, s);
}

// arg[i] = argmax_j (2 a_i . b_j - bnrm_j), j < nb; A [>= na rows x dpad],
// B [>= ceil(nb/256)*256 rows x dpad] bf16 (padding rows zero).
int32_t tc_assign_argmax(const __nv_bfloat16* A, int na, const __nv_bfloat16* B, int nb,
                         const float* bnrm, int dpad, int32_t* arg, float* best, int32_t* err,
                         cudaStream_t s) {
    using namespace tc;
    if (dpad % BK) return AP_ERR_INVALID_ARG;
    const int arows = (na + BM - 1) / BM * BM;
    const int brows = (nb + BN - 1) / BN * BN;
    CUtensorMap ma, mb;
    AP_TRY(make_map(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (void*)A, dpad, arows, (uint64_t)dpad * 2,
                    BK, BM, CU_TENSOR_MAP_SWIZZLE_128B));
    AP_TRY(make_map(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (void*)B, dpad, brows, (uint64_t)dpad * 2,
                    BK, BN / 2, CU_TENSOR_MAP_SWIZZLE_128B));
    Params p{};
    p.M = na;
    p.N = nb;
    p.K = dpad;
    p.mode = ARGMAX;
    p.anrm = bnrm;           // unused by the arg-max epilogue
    p.bnrm = bnrm;
    p.arg = arg;
    p.best = best;
    p.spin_limit = 1u << 22;
    p.error = err;
    return launch(ma, mb, ma, p, ((na + BM - 1) / BM + 1) / 2, s);         // row-block pairs
}

}  // namespace apgb
