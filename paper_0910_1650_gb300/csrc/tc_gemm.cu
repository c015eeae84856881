// Tensor-core (tcgen05) GEMMs with fused epilogues, for the dense
// contractions of the method:
//   * similarity:  s(i,k) = 2 x_i . x_k - |x_i|^2 - |x_k|^2, clamped to <= 0
//                  (Section 2, s(i,k) = -|x_i - x_k|^2), written as float32,
//                  for one problem or for a table of tiles of many problems
//                  (one persistent launch over a whole batch);
//   * assignment:  c_i = argmax_j (2 x_i . e_j - |e_j|^2) over the exemplars
//                  e_j (Algorithm 3 Step 2: nearest centre), never writing the
//                  N x c score matrix.  Up to 1024 exemplars, -|e_j|^2/2 enters
//                  the product through one extra K = 16 MMA per tile over
//                  augmented operands resident in shared memory; beyond, the
//                  epilogue subtracts it.
// Operands are bf16, K-major, loaded by TMA with 128-byte swizzle; the
// product accumulates in fp32 in tensor memory.
//
// Persistent, warp-specialised kernel (one CTA per SM, 320 threads):
//   warp 0      TMA producer: the A tile (128 x 64) and the B tile (256 x 64)
//               of each K step into a ring of 2-4 stages (mbarriers
//               full/empty);
//   warp 1      allocates 512 TMEM columns and issues tcgen05.mma
//               (M=128, N=256, K=16) from one elected thread into two
//               256-column accumulators (mbarriers tfull/tempty);
//   warps 2..9  epilogue, two warps per TMEM lane quarter (column halves of
//               128).  Each warp works on its own: it waits for the
//               accumulator itself, reads it with pipelined tcgen05.ld, and
//               either stores its 32 x 32 blocks through its own swizzled
//               shared buffers with TMA tensor stores (similarity) or keeps a
//               running per-row arg-max (assignment; the two column halves of
//               a row are merged once per row block through shared memory,
//               handed over on bounded mbarriers).
// The shared-memory split between operand stages and store buffers depends
// on K: deep operand rings where the product is long (tensor-bound), deep
// store buffering where it is short (bound by writing S).
// Every mbarrier wait is bounded; on expiry the kernel records an error and
// all roles stop issuing new work.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "ptx.cuh"

namespace apgb {
namespace tc {

constexpr int BM = 128, BN = 256, BK = 64;
constexpr int MAX_STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;            // 16 KB
constexpr int B_BYTES = BN * BK * 2;            // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;  // 48 KB
constexpr int OUT_COLS = 32;                    // fp32 columns per store block (128 B)
constexpr int WBUF_BYTES = 32 * OUT_COLS * 4;   // one warp's 32 rows x 32 columns: 4 KB
constexpr int EPI_WARPS = 8;                    // two per TMEM lane quarter: column halves
constexpr int THREADS = 64 + 32 * EPI_WARPS;    // producer, MMA issuer, epilogue
constexpr uint32_t TMEM_COLS = 512;
constexpr int SMEM_LIMIT = 227 * 1024;

enum Mode : int { SIM = 0, ARGMAX = 1, TOP2 = 2 };

// Barriers and flags, after the data area.
struct Ctl {
    uint64_t full[MAX_STAGES], empty[MAX_STAGES], tfull[2], tempty[2], mma_done;
    uint64_t mfull[4], mempty[4];   // ARGMAX/TOP2: column-half hand-over per lane quarter
    uint32_t tmem_base;
    int abort;                      // any role gave up a bounded wait
};

// ARGMAX/TOP2: the second column half's per-row results, after Ctl; the
// staged column norms follow (16-byte aligned).
struct Slots {
    float b1[BM], b2[BM];
    int j1[BM], j2[BM];
};
static_assert((sizeof(Ctl) + sizeof(Slots)) % 16 == 0, "norm table alignment");

// Largest of three (sm_100 and later: one instruction).
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// r[e] = take ? v[e] : r[e] for eight values, as predicated selects (no branch).
__device__ __forceinline__ void select8(float* r, const float* v, uint32_t take) {
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %8, 0;\n\t"
        "selp.f32 %0, %9, %0, q;\n\tselp.f32 %1, %10, %1, q;\n\t"
        "selp.f32 %2, %11, %2, q;\n\tselp.f32 %3, %12, %3, q;\n\t"
        "selp.f32 %4, %13, %4, q;\n\tselp.f32 %5, %14, %5, q;\n\t"
        "selp.f32 %6, %15, %6, q;\n\tselp.f32 %7, %16, %7, q;\n\t}"
        : "+f"(r[0]), "+f"(r[1]), "+f"(r[2]), "+f"(r[3]), "+f"(r[4]), "+f"(r[5]), "+f"(r[6]), "+f"(r[7])
        : "r"(take), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]));
}

__device__ __forceinline__ bool aborted(const Ctl& c) {
    return *reinterpret_cast<const volatile int*>(&c.abort) != 0;
}

// One problem of a grouped similarity launch.  Its features occupy rows
// [roff, roff + npad) of the operand arena (npad a multiple of BN, padding
// rows zero) and its norms the same entries of the norm arena.
struct GroupProblem {
    const CUtensorMap* omap;        // output map of S (device memory, 64-B aligned)
    float* out;                     // S (row stride lds)
    int64_t lds;
    int32_t roff, n, n4, pad;
};

struct Params {
    int M, N, K;                    // rows of A, rows of B, padded K (multiple of 64)
    int mode;
    int stages, nob;                // operand stages; store buffers per epilogue warp
    const float* anrm;              // SIM: |a_i|^2 (length >= M)
    const float* bnrm;              // |b_k|^2 (length >= N rounded up to BN)
    int snrm;                       // ARGMAX/TOP2: entries of bnrm staged in shared memory (0: read global)
    int aug;                        // ARGMAX/TOP2: groups of 1024 columns whose -|b|^2/2 the MMA adds
                                    // through the resident augmented operands (0: the epilogue does)
    int32_t* arg;                   // ARGMAX/TOP2: best column per row
    float* best;                    // ARGMAX/TOP2: best score per row (may be null)
    int32_t* arg2;                  // TOP2: second-best column per row (-1: none)
    float* best2;                   // TOP2: second-best score per row (-inf: none)
    int diag_zero;                  // SIM: write 0 where row == column
    // SIM: the tensor store covers columns [0, n4), n4 = N rounded down to a
    // multiple of 4 (a TMA store writes whole 16-byte granules at the right
    // edge of the tensor, which would reach into the caller's columns >= N);
    // columns [n4, N) are written by plain stores to out (row stride lds).
    int n4;
    float* out;
    int64_t lds;
    // SIM grouped: tile u is (problem, row block, column block) = tiles[u]
    const int4* tiles;
    const GroupProblem* probs;
    int ntiles;
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

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     map),
                 "r"(x), "r"(y), "r"(ptx::smem_u32(src))
                 : "memory");
}

// A tensor map that lives in global memory, written before the launch, is
// made visible to the tensor-copy unit.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
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

// Arrives on `bar` once every tcgen05.mma issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            ptx::smem_u32(bar))
        : "memory");
}

// Starts reading 32 consecutive accumulator columns of this warp's 32 lanes
// (one row each).  The registers hold the values only after tmem_wait(r).
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
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
}

// Waits for this thread's outstanding tcgen05.ld; the registers of the load
// are passed through, so no use of them can be scheduled before the wait.
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                   "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                   "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                   "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
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

// The augmented operands that fold -|b|^2/2 into the product, in the layout
// of the operand tiles (K-major, 128-byte rows, 128-byte swizzle: 16-byte
// unit c of row r sits at unit c ^ (r % 8)).  K block k (16 columns: units
// 2k and 2k+1) of
//   A' (BM rows):          1, 1, 1, 0, ..., 0 in every row and every block;
//   B' group g (BN rows):  row r of block k belongs to column g*1024 + k*256 + r
//                          and holds -h, -m, -l, 0, ..., 0, where h + m + l =
//                          |b|^2/2 exactly (three bf16 terms of a normal
//                          float); zero past `ncols`.
// One K = 16 MMA over block q % 4 of A' and of B' group q / 4 adds -|b|^2/2
// to every row of column tile q.
__device__ void build_augmented(uint8_t* aug, const float* bnrm, int ncols, int groups) {
    auto pack = [](__nv_bfloat16 lo, __nv_bfloat16 hi) -> uint32_t {
        return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
    };
    const __nv_bfloat16 one = __float2bfloat16_rn(1.f), zero = __float2bfloat16_rn(0.f);
    for (int i = threadIdx.x; i < BM * 8; i += blockDim.x) {
        const int r = i >> 3, c = i & 7;
        const uint4 v = (c & 1) ? make_uint4(0, 0, 0, 0) : make_uint4(pack(one, one), pack(one, zero), 0, 0);
        *reinterpret_cast<uint4*>(aug + r * 128 + ((c ^ (r & 7)) << 4)) = v;
    }
    uint8_t* bb = aug + A_BYTES;
    for (int i = threadIdx.x; i < groups * BN * 4; i += blockDim.x) {
        const int k = i & 3, r = (i >> 2) % BN, g = (i >> 2) / BN;
        const int col = g * 4 * BN + k * BN + r;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (col < ncols) {
            const float x = 0.5f * __ldg(bnrm + col);
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            const float r1 = x - __bfloat162float(h);                // exact
            const __nv_bfloat16 m = __float2bfloat16_rn(r1);
            const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));   // exact
            v.x = pack(__hneg(h), __hneg(m));
            v.y = pack(__hneg(l), zero);
        }
        uint8_t* row = bb + (size_t)g * B_BYTES + r * 128;
        *reinterpret_cast<uint4*>(row + (((2 * k) ^ (r & 7)) << 4)) = v;
        *reinterpret_cast<uint4*>(row + (((2 * k + 1) ^ (r & 7)) << 4)) = make_uint4(0, 0, 0, 0);
    }
}

// Instruction descriptor: kind::f16 with bf16 A/B, fp32 D, both K-major.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
    return (1u << 4)                  // D format: f32
           | (1u << 7)                // A format: bf16
           | (1u << 10)               // B format: bf16
           | ((uint32_t)(n >> 3) << 17)
           | ((uint32_t)(m >> 4) << 24);
}

// Where tile (u, q) lies: operand rows of its A and B tiles, its row and
// column block inside its problem, and the problem.
struct Tile {
    int arow, brow, m, n, prob;
};

__device__ __forceinline__ Tile tile_of(const Params& p, int numN, int u, int q) {
    Tile t;
    if (p.mode != SIM) {
        t.m = u; t.n = q; t.prob = 0;
        t.arow = u * BM; t.brow = q * BN;
    } else if (p.tiles) {
        const int4 e = p.tiles[u];
        const int roff = p.probs[e.x].roff;
        t.prob = e.x; t.m = e.y; t.n = e.z;
        t.arow = roff + e.y * BM; t.brow = roff + e.z * BN;
    } else {
        t.m = u / numN; t.n = u % numN; t.prob = 0;
        t.arow = t.m * BM; t.brow = t.n * BN;
    }
    return t;
}

// All but the newest nob-1 store groups of this thread have read shared memory.
__device__ __forceinline__ void wait_store_slot(int nob) {
    switch (nob) {
        case 4: ptx::bulk_wait_read<3>(); break;
        case 3: ptx::bulk_wait_read<2>(); break;
        case 2: ptx::bulk_wait_read<1>(); break;
        default: ptx::bulk_wait_read<0>(); break;
    }
}

__global__ void __launch_bounds__(THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmOut, Params p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~uintptr_t(1023));
    uint8_t* out_base = base + (size_t)p.stages * STAGE_BYTES;
    // ARGMAX/TOP2 with folded norms: the augmented operands (A' then the B'
    // groups, 1024-byte aligned) sit between the store buffers and Ctl
    uint8_t* aug_base = out_base + (size_t)EPI_WARPS * p.nob * WBUF_BYTES;
    Ctl& sm = *reinterpret_cast<Ctl*>(aug_base + (p.aug > 0 ? (size_t)A_BYTES + (size_t)p.aug * B_BYTES : 0));
    Slots& sl = *reinterpret_cast<Slots*>(reinterpret_cast<uint8_t*>(&sm) + sizeof(Ctl));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const int numM = (p.M + BM - 1) / BM;
    const int numN = (p.N + BN - 1) / BN;
    const int numK = p.K / BK;
    // work units: one tile (SIM) or one row block with all its column tiles (ARGMAX, TOP2)
    const bool amax = p.mode != SIM;
    const int units = amax ? numM : (p.tiles ? p.ntiles : numM * numN);
    const int tiles_per_unit = amax ? numN : 1;
    const int ns = p.stages;

    if (threadIdx.x == 0) {
        for (int s = 0; s < MAX_STAGES; ++s) {
            ptx::mbar_init(&sm.full[s], 1);
            ptx::mbar_init(&sm.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&sm.tfull[b], 1);
            ptx::mbar_init(&sm.tempty[b], EPI_WARPS);
        }
        for (int q = 0; q < 4; ++q) {
            ptx::mbar_init(&sm.mfull[q], 32);
            ptx::mbar_init(&sm.mempty[q], 32);
        }
        ptx::mbar_init(&sm.mma_done, 1);
        ptx::fence_mbar_init();
        sm.abort = 0;
    }
    if (warp == 1) tmem_alloc(&sm.tmem_base, TMEM_COLS);
    if (p.aug > 0) {
        build_augmented(aug_base, p.bnrm, numN * BN, p.aug);
        ptx::fence_proxy_async_smem();               // generic stores -> the MMA's reads
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t eph = 0xFu;                    // empty barriers start "released"
            uint32_t armed = 0;                     // loads issued per stage (low bit = parity)
            int nissued = 0;
            for (int u = blockIdx.x; u < units && !aborted(sm); u += gridDim.x) {
                for (int q = 0; q < tiles_per_unit && !aborted(sm); ++q) {
                    const Tile t = tile_of(p, numN, u, q);
                    for (int kb = 0; kb < numK; ++kb) {
                        if (!ptx::mbar_wait(&sm.empty[stage], (eph >> stage) & 1u, p.spin_limit)) {
                            atomicExch(&sm.abort, 1);
                            break;
                        }
                        eph ^= 1u << stage;
                        uint8_t* st = base + (size_t)stage * STAGE_BYTES;
                        ptx::mbar_arrive_expect_tx(&sm.full[stage], STAGE_BYTES);
                        tma_load_2d(st, &tmA, kb * BK, t.arow, &sm.full[stage]);
                        tma_load_2d(st + A_BYTES, &tmB, kb * BK, t.brow, &sm.full[stage]);
                        armed ^= 1u << stage;
                        ++nissued;
                        stage = (stage + 1 == ns) ? 0 : stage + 1;
                    }
                }
            }
            // loads still in flight must land before shared memory is released
            for (int s = 0; s < ns && s < nissued; ++s)
                ptx::mbar_wait(&sm.full[s], ((armed >> s) & 1u) ^ 1u, p.spin_limit);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = instr_desc(BM, BN);
            int stage = 0, acc = 0;
            uint32_t fph = 0, tph = 3;              // tempty barriers start "released"
            for (int u = blockIdx.x; u < units && !aborted(sm); u += gridDim.x) {
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
                        const uint8_t* st = base + (size_t)stage * STAGE_BYTES;
                        const uint64_t ad = smem_desc(st);
                        const uint64_t bd = smem_desc(st + A_BYTES);
#pragma unroll
                        for (int k = 0; k < BK / 16; ++k) {
                            // advance 16 bf16 (32 B) along K inside the swizzle atom
                            mma_bf16(d, ad + (uint64_t)(k * 2), bd + (uint64_t)(k * 2), idesc,
                                     (kb > 0 || k > 0) ? 1u : 0u);
                        }
                        mma_commit(&sm.empty[stage]);  // frees the stage once these MMAs are done
                        stage = (stage + 1 == ns) ? 0 : stage + 1;
                    }
                    if (p.aug > 0) {
                        // + 1 . (-h - m - l) = -|b|^2/2 for every row: column tile q is
                        // K block q % 4 of B' group q / 4 (A' holds the ones in every block)
                        const uint64_t ad = smem_desc(aug_base) + (uint64_t)((q & 3) * 2);
                        const uint64_t bd = smem_desc(aug_base + A_BYTES + (size_t)(q >> 2) * B_BYTES) +
                                            (uint64_t)((q & 3) * 2);
                        mma_bf16(d, ad, bd, idesc, 1u);
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
        // Warp w reads TMEM lane quarter w % 4 (its 32 rows) and column half
        // (w - 2) / 4 (128 of each accumulator's 256 columns).
        const int ew = warp - 2;
        const int sub = warp & 3;
        const int half = ew >> 2;
        const int row_in_tile = sub * 32 + lane;
        uint8_t* wbuf = out_base + (size_t)ew * p.nob * WBUF_BYTES;
        int ob = 0;
        int acc = 0;
        uint32_t tph = 0;
        uint32_t uj = 0;                             // units this warp has finished
        bool dead = false;
        const uint32_t lane_off = (uint32_t)(sub * 32) << 16;
        // ARGMAX/TOP2: the column norms, staged once in shared memory when they
        // fit (the epilogue warps copy them and meet on named barrier 1)
        float* snrm = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(&sl) + sizeof(Slots));
        if (amax && p.snrm > 0) {
            for (int k = threadIdx.x - 64; k < p.snrm / 4; k += 32 * EPI_WARPS)
                reinterpret_cast<float4*>(snrm)[k] = __ldg(reinterpret_cast<const float4*>(p.bnrm) + k);
            asm volatile("bar.sync 1, %0;" ::"n"(32 * EPI_WARPS) : "memory");
        }
        const float* nrm = (amax && p.snrm > 0) ? snrm : p.bnrm;
        for (int u = blockIdx.x; u < units && !dead; u += gridDim.x) {
            float best = -INFINITY;                  // ARGMAX/TOP2: max of x.e - |e|^2/2
            int bidx = INT_MAX;
            int bchunk = -1;                         // ARGMAX: first column of the chunk holding best
            float keep[32];                          // ARGMAX: that chunk's scores
#pragma unroll
            for (int e = 0; e < 32; ++e) keep[e] = 0.f;
            float best2 = -INFINITY;                 // TOP2: the runner-up
            int bidx2 = INT_MAX;
            int m0 = 0;
            for (int q = 0; q < tiles_per_unit; ++q) {
                const Tile t = tile_of(p, numN, u, q);
                m0 = t.m;
                uint32_t ok = 1;
                if (lane == 0)
                    ok = (!aborted(sm) &&
                          ptx::mbar_wait(&sm.tfull[acc], (tph >> acc) & 1u, p.spin_limit)) ? 1u : 0u;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                tph ^= 1u << acc;
                if (!ok) {
                    if (lane == 0) atomicExch(&sm.abort, 1);
                    dead = true;
                    break;
                }
                tc_fence_after();
                const uint32_t tbase = tmem + (uint32_t)(acc * BN + half * 128) + lane_off;
                const int col_half = t.n * BN + half * 128;     // first column of this half
                if (p.mode == SIM) {
                    // the problem's geometry (a table entry in grouped mode)
                    int Mloc = p.M, Nloc = p.N, n4 = p.n4, roff = 0;
                    float* out = p.out;
                    int64_t lds = p.lds;
                    const CUtensorMap* omap = &tmOut;
                    if (p.tiles) {
                        const GroupProblem& g = p.probs[t.prob];
                        Mloc = Nloc = g.n;
                        n4 = g.n4;
                        roff = g.roff;
                        out = g.out;
                        lds = g.lds;
                        omap = g.omap;
                        if (lane == 0) tensormap_acquire(omap);
                    }
                    const int i = t.m * BM + row_in_tile;
                    const float ai = (i < Mloc) ? __ldg(p.anrm + roff + i) : 0.f;
                    const float2 nai = make_float2(-ai, -ai), two = make_float2(2.f, 2.f),
                                 mone = make_float2(-1.f, -1.f);
                    const float* bn = p.bnrm + roff + col_half;
                    uint32_t ra[32], rb[32];
                    auto emit = [&](uint32_t (&v)[32], int c) {
                        const int kcol = col_half + c * OUT_COLS;
                        float o[32];
#pragma unroll
                        for (int u4 = 0; u4 < 8; ++u4) {
                            const float4 b4 = __ldg(reinterpret_cast<const float4*>(bn + c * OUT_COLS) + u4);
                            // (2v - a) - b with the rounding of the plain expression
                            float2 lo = __ffma2_rn(two, make_float2(__uint_as_float(v[4 * u4]),
                                                                    __uint_as_float(v[4 * u4 + 1])), nai);
                            float2 hi = __ffma2_rn(two, make_float2(__uint_as_float(v[4 * u4 + 2]),
                                                                    __uint_as_float(v[4 * u4 + 3])), nai);
                            lo = __ffma2_rn(mone, make_float2(b4.x, b4.y), lo);
                            hi = __ffma2_rn(mone, make_float2(b4.z, b4.w), hi);
                            o[4 * u4] = fminf(0.f, lo.x);
                            o[4 * u4 + 1] = fminf(0.f, lo.y);
                            o[4 * u4 + 2] = fminf(0.f, hi.x);
                            o[4 * u4 + 3] = fminf(0.f, hi.y);
                        }
                        if (p.diag_zero && i >= kcol && i < kcol + OUT_COLS) {
#pragma unroll
                            for (int e = 0; e < 32; ++e)
                                if (kcol + e == i) o[e] = 0.f;
                        }
                        // this warp's buffer `ob` must have been read by its store nob stores ago
                        if (lane == 0) wait_store_slot(p.nob);
                        __syncwarp();
                        uint8_t* buf = wbuf + (size_t)ob * WBUF_BYTES;
#pragma unroll
                        for (int u4 = 0; u4 < 8; ++u4) {
                            const int phys = u4 ^ (lane & 7);
                            *reinterpret_cast<float4*>(buf + lane * 128 + phys * 16) =
                                make_float4(o[4 * u4], o[4 * u4 + 1], o[4 * u4 + 2], o[4 * u4 + 3]);
                        }
                        if (kcol + OUT_COLS > n4 && kcol < Nloc && i < Mloc) {
                            // the ragged columns [n4, N) of this row
#pragma unroll
                            for (int e = 0; e < OUT_COLS; ++e) {
                                const int k = kcol + e;
                                if (k >= n4 && k < Nloc) out[(int64_t)i * lds + k] = o[e];
                            }
                        }
                        ptx::fence_proxy_async_smem();
                        __syncwarp();
                        if (lane == 0) {
                            if (kcol < n4) tma_store_2d(omap, kcol, t.m * BM + sub * 32, buf);
                            ptx::bulk_commit();
                        }
                        ob = (ob + 1 == p.nob) ? 0 : ob + 1;
                        __syncwarp();                // converged for the next tcgen05 op
                    };
                    tmem_ld32_async(tbase, ra);
                    tmem_wait(ra);
#pragma unroll
                    for (int c = 0; c < 4; c += 2) {
                        tmem_ld32_async(tbase + (uint32_t)((c + 1) * OUT_COLS), rb);
                        emit(ra, c);
                        tmem_wait(rb);
                        if (c + 2 < 4) tmem_ld32_async(tbase + (uint32_t)((c + 2) * OUT_COLS), ra);
                        emit(rb, c + 1);
                        if (c + 2 < 4) tmem_wait(ra);
                    }
                } else {
                    // running arg-max of x.e - |e|^2 / 2 (half the score: exact scaling)
                    const float2 mhalf = make_float2(-0.5f, -0.5f);
                    const bool full_tile = col_half + 128 <= p.N;
                    uint32_t ra[32], rb[32];
                    // ARGMAX: each 32-column chunk's maximum by a tree of three-input
                    // maxima; where it beats the running best (strictly: chunks
                    // arrive in increasing column order, so a tie keeps the earlier
                    // chunk) the chunk's scores replace the kept ones by predicated
                    // selects.  The column inside the kept chunk is found once per
                    // row block.  TOP2 also keeps the runner-up (the best of the
                    // other columns, lowest column on ties), column by column.
                    // fold: the MMA has added -|e|^2/2 already (augmented operands)
                    auto scan = [&](uint32_t (&v)[32], int c, auto top2, auto fold) {
                        const int kcol = col_half + c * OUT_COLS;
                        const bool ragged = !full_tile && kcol + OUT_COLS > p.N;
                        const float4* bn4 = reinterpret_cast<const float4*>(nrm + kcol);
                        float sc[32];
                        if (decltype(fold)::value) {
#pragma unroll
                            for (int e = 0; e < 32; ++e) sc[e] = __uint_as_float(v[e]);
                        } else {
#pragma unroll
                            for (int u4 = 0; u4 < 8; ++u4) {
                                const float4 b4 = bn4[u4];
                                const float2 lo = __ffma2_rn(mhalf, make_float2(b4.x, b4.y),
                                                             make_float2(__uint_as_float(v[4 * u4]),
                                                                         __uint_as_float(v[4 * u4 + 1])));
                                const float2 hi = __ffma2_rn(mhalf, make_float2(b4.z, b4.w),
                                                             make_float2(__uint_as_float(v[4 * u4 + 2]),
                                                                         __uint_as_float(v[4 * u4 + 3])));
                                sc[4 * u4] = lo.x;
                                sc[4 * u4 + 1] = lo.y;
                                sc[4 * u4 + 2] = hi.x;
                                sc[4 * u4 + 3] = hi.y;
                            }
                        }
                        if (ragged) {
#pragma unroll
                            for (int e = 0; e < 32; ++e)
                                if (kcol + e >= p.N) sc[e] = -INFINITY;
                        }
                        if (decltype(top2)::value) {
#pragma unroll
                            for (int e = 0; e < 32; ++e) {
                                const int k = kcol + e;
                                const bool gt = sc[e] > best, gt2 = sc[e] > best2;
                                bidx2 = gt ? bidx : (gt2 ? k : bidx2);
                                best2 = fmaxf(best2, fminf(sc[e], best));
                                bidx = gt ? k : bidx;
                                best = fmaxf(best, sc[e]);
                            }
                        } else {
                            float t[11];
#pragma unroll
                            for (int e = 0; e < 10; ++e) t[e] = max3f(sc[3 * e], sc[3 * e + 1], sc[3 * e + 2]);
                            t[10] = fmaxf(sc[30], sc[31]);
                            const float m = fmaxf(max3f(max3f(t[0], t[1], t[2]), max3f(t[3], t[4], t[5]),
                                                        max3f(t[6], t[7], t[8])),
                                                  fmaxf(t[9], t[10]));
                            const uint32_t imp = m > best ? 1u : 0u;
#pragma unroll
                            for (int h = 0; h < 4; ++h) select8(keep + 8 * h, sc + 8 * h, imp);
                            best = imp ? m : best;
                            bchunk = imp ? kcol : bchunk;
                        }
                        __syncwarp();                    // converged for the next tcgen05 op
                    };
                    auto chunks = [&](auto top2, auto fold) {
                        tmem_ld32_async(tbase, ra);
                        tmem_wait(ra);
#pragma unroll
                        for (int c = 0; c < 4; c += 2) {
                            tmem_ld32_async(tbase + (uint32_t)((c + 1) * OUT_COLS), rb);
                            scan(ra, c, top2, fold);
                            tmem_wait(rb);
                            if (c + 2 < 4) tmem_ld32_async(tbase + (uint32_t)((c + 2) * OUT_COLS), ra);
                            scan(rb, c + 1, top2, fold);
                            if (c + 2 < 4) tmem_wait(ra);
                        }
                    };
                    if (p.mode == TOP2) {
                        if (p.aug > 0) chunks(std::true_type{}, std::true_type{});
                        else chunks(std::true_type{}, std::false_type{});
                    } else {
                        if (p.aug > 0) chunks(std::false_type{}, std::true_type{});
                        else chunks(std::false_type{}, std::false_type{});
                    }
                }
                // accumulator drained: hand it back to the MMA warp
                tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&sm.tempty[acc]);
                acc ^= 1;
            }
            if (dead) break;
            if (p.mode == ARGMAX && bchunk >= 0) {
                // the first column of the kept chunk attaining the row's best
                int j = 31;
#pragma unroll
                for (int e = 30; e >= 0; --e) j = (keep[e] == best) ? e : j;
                bidx = bchunk + j;
            }
            if (amax) {
                // merge the two column halves of each row: the larger score,
                // the lower column on a tie (TOP2: the runner-up of the union
                // as well).  The second half hands its results over through this
                // quarter's slots (mfull), the first hands the slots back
                // (mempty); both waits are bounded.
                const uint32_t par = uj & 1u;
                bool okm;
                if (half == 1) {
                    okm = ptx::mbar_wait(&sm.mempty[sub], par ^ 1u, p.spin_limit);
                    if (okm) {
                        sl.b1[row_in_tile] = best;
                        sl.j1[row_in_tile] = bidx;
                        sl.b2[row_in_tile] = best2;
                        sl.j2[row_in_tile] = bidx2;
                        ptx::mbar_arrive(&sm.mfull[sub]);
                    }
                } else {
                    okm = ptx::mbar_wait(&sm.mfull[sub], par, p.spin_limit);
                    if (okm) {
                        const float o1 = sl.b1[row_in_tile], o2 = sl.b2[row_in_tile];
                        const int i1 = sl.j1[row_in_tile], i2 = sl.j2[row_in_tile];
                        ptx::mbar_arrive(&sm.mempty[sub]);
                        auto better = [](float a, int ia, float b, int ib) {
                            return a > b || (a == b && ia < ib);
                        };
                        if (better(o1, i1, best, bidx)) {
                            // the other half holds the best; the runner-up is the
                            // better of this half's best and the other's runner-up
                            if (better(o2, i2, best, bidx)) { best2 = o2; bidx2 = i2; }
                            else { best2 = best; bidx2 = bidx; }
                            best = o1; bidx = i1;
                        } else if (better(o1, i1, best2, bidx2)) {
                            best2 = o1; bidx2 = i1;
                        }
                        const int i = m0 * BM + row_in_tile;
                        if (i < p.M) {
                            p.arg[i] = bidx;
                            if (p.best) p.best[i] = 2.f * best;
                            if (p.mode == TOP2) {
                                p.arg2[i] = (bidx2 == INT_MAX) ? -1 : bidx2;
                                p.best2[i] = 2.f * best2;
                            }
                        }
                    }
                }
                if (__any_sync(0xffffffffu, !okm)) {
                    if (lane == 0) atomicExch(&sm.abort, 1);
                    dead = true;
                }
                ++uj;
            }
        }
        if (p.mode == SIM && lane == 0) ptx::bulk_wait_all();
    }

    tc_fence_before();
    __syncthreads();
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

// The output map of S: fp32 columns [0, max(n4, 4)) of n rows, stored in
// 32 x 32 blocks (one epilogue warp's rows and one 128-byte column block).
static int32_t make_out_map(CUtensorMap* map, float* S, int n, int64_t lds) {
    const int n4 = n & ~3;
    return make_map(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, S, (uint64_t)std::max(n4, 4), (uint64_t)n,
                    (uint64_t)lds * 4, OUT_COLS, 32, CU_TENSOR_MAP_SWIZZLE_128B);
}

// Operand stages and store buffers: a long product (K >= 256) wants a deep
// operand ring and writes S slowly; a short one is bound by writing S.
static void layout_for(int mode, int numK, int* stages, int* nob) {
    if (mode != SIM) { *stages = 3; *nob = 0; }   // (measured no slower than 4 at K = 128)
    else if (numK >= 4) { *stages = 4; *nob = 1; }
    else if (numK >= 2) { *stages = 3; *nob = 2; }
    else { *stages = 2; *nob = 4; }
}

static size_t smem_bytes(int mode, int stages, int nob) {
    return 1024 + (size_t)stages * STAGE_BYTES + (size_t)EPI_WARPS * nob * WBUF_BYTES + sizeof(Ctl) +
           (mode != SIM ? sizeof(Slots) : 0);
}

// ARGMAX/TOP2 norm form: 0 automatic (the first that fits of folded, shared
// table, global); the environment variable APGB_ASSIGN_NORMS = folded |
// shared | global asks for one form (taken where it fits, else the next), so
// the three can be compared on the same inputs.
static int assign_norm_form() {
    const char* e = std::getenv("APGB_ASSIGN_NORMS");
    if (!e) return 0;
    if (!std::strcmp(e, "folded")) return 1;
    if (!std::strcmp(e, "shared")) return 2;
    if (!std::strcmp(e, "global")) return 3;
    return 0;
}

static int32_t launch(const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& o, Params p,
                      int units, cudaStream_t s) {
    int sms = 0;
    AP_TRY(device_sm_count(&sms));
    layout_for(p.mode, p.K / BK, &p.stages, &p.nob);
    size_t bytes = smem_bytes(p.mode, p.stages, p.nob);
    if (bytes > (size_t)SMEM_LIMIT) return AP_ERR_UNSUPPORTED;
    // ARGMAX/TOP2: how -|b|^2/2 enters the scores.  Folded into the product
    // by one extra K = 16 MMA per tile where the augmented operands fit
    // (16 KB + 32 KB per 1024 columns: up to 1024 columns); otherwise the
    // epilogue subtracts it, reading the norms from a shared-memory table
    // where that fits (up to about 20000 columns) or from global memory.
    p.snrm = 0;
    p.aug = 0;
    if (p.mode != SIM) {
        const size_t npad = (size_t)(p.N + BN - 1) / BN * BN;
        const int groups = (int)((npad + 4 * BN - 1) / (4 * BN));
        const size_t augb = (size_t)A_BYTES + (size_t)groups * B_BYTES;
        const int want = assign_norm_form();
        if (want <= 1 && bytes + augb <= (size_t)SMEM_LIMIT) {
            p.aug = groups;
            bytes += augb;
        } else if (want <= 2 && bytes + npad * 4 <= (size_t)SMEM_LIMIT) {
            p.snrm = (int)npad;
            bytes += npad * 4;
        }
    }
    AP_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     SMEM_LIMIT));
    // persistent: one CTA per SM, each taking every gridDim-th unit
    const int grid = std::max(1, std::min(units, sms));
    tc_gemm_kernel<<<grid, THREADS, bytes, s>>>(a, b, o, p);
    note_launches(1);
    return last_error();
}

}  // namespace tc

size_t tc_similarity_pad_rows() { return tc::BN; }

// S = -|xi - xk|^2 from bf16 features Xb [npad x dpad] (dpad % 64 == 0,
// rows >= n zero) and fp32 norms of the bf16 rows (npad entries); diagonal
// written as 0.
int32_t tc_similarity_bf16(const __nv_bfloat16* Xb, const float* nrm, int n, int dpad, float* S,
                           int64_t lds, int32_t* err, cudaStream_t s) {
    using namespace tc;
    if (dpad % BK || (lds & 3) || !aligned16(S)) return AP_ERR_INVALID_ARG;
    const int npad = (n + BN - 1) / BN * BN;
    CUtensorMap ma, mb, mo;
    AP_TRY(make_map(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (void*)Xb, dpad, npad, (uint64_t)dpad * 2,
                    BK, BM, CU_TENSOR_MAP_SWIZZLE_128B));
    AP_TRY(make_map(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (void*)Xb, dpad, npad, (uint64_t)dpad * 2,
                    BK, BN, CU_TENSOR_MAP_SWIZZLE_128B));
    AP_TRY(make_out_map(&mo, S, n, lds));
    Params p{};
    p.M = n;
    p.N = n;
    p.K = dpad;
    p.mode = SIM;
    p.anrm = nrm;
    p.bnrm = nrm;
    p.diag_zero = 1;
    p.n4 = n & ~3;
    p.out = S;
    p.lds = lds;
    p.spin_limit = 1u << 22;
    p.error = err;
    const int units = ((n + BM - 1) / BM) * ((n + BN - 1) / BN);
    return launch(ma, mb, mo, p, units, s);
}

// Device bytes of the tables of a grouped similarity over problems of sizes
// n[0..count): output maps, problem table and tile table.
size_t tc_grouped_table_bytes(const int64_t* n, int32_t count) {
    using namespace tc;
    size_t tiles = 0;
    for (int32_t b = 0; b < count; ++b)
        tiles += (size_t)((n[b] + BM - 1) / BM) * (size_t)((n[b] + BN - 1) / BN);
    Carver c(nullptr);
    c.take<CUtensorMap>((size_t)count);
    c.take<GroupProblem>((size_t)count);
    c.take<int4>(tiles);
    return c.used;
}

// The similarity of every problem of a batch in one persistent launch over a
// table of all their tiles.  Problem b's bf16 features are rows
// [roff[b], roff[b] + ceil(n[b]/256)*256) of the arena Xb [rows x dpad]
// (padding rows zero), its norms the same entries of nrm; S_b at S[b] with
// row stride lds[b].  `tables` is device scratch of tc_grouped_table_bytes.
int32_t tc_similarity_bf16_grouped(const __nv_bfloat16* Xb, const float* nrm, int64_t rows, int dpad,
                                   const int64_t* n, const int64_t* roff, float* const* S,
                                   const int64_t* lds, int32_t count, void* tables, int32_t* err,
                                   cudaStream_t s) {
    using namespace tc;
    if (dpad % BK || count < 1 || !tables || rows > INT_MAX) return AP_ERR_INVALID_ARG;
    Carver c(tables);
    CUtensorMap* dmaps = c.take<CUtensorMap>((size_t)count);
    GroupProblem* dprobs = c.take<GroupProblem>((size_t)count);
    std::vector<CUtensorMap> maps(count);
    std::vector<GroupProblem> probs(count);
    std::vector<int4> tiles;
    for (int32_t b = 0; b < count; ++b) {
        const int nb = (int)n[b];
        if ((lds[b] & 3) || !aligned16(S[b]) || roff[b] % BN || roff[b] + (nb + BN - 1) / BN * BN > rows)
            return AP_ERR_INVALID_ARG;
        AP_TRY(make_out_map(&maps[b], S[b], nb, lds[b]));
        probs[b] = GroupProblem{dmaps + b, S[b], lds[b], (int32_t)roff[b], nb, nb & ~3, 0};
        const int mb = (nb + BM - 1) / BM, nbk = (nb + BN - 1) / BN;
        for (int i = 0; i < mb; ++i)
            for (int j = 0; j < nbk; ++j) tiles.push_back(make_int4(b, i, j, 0));
    }
    int4* dtiles = c.take<int4>(tiles.size());
    AP_CUDA_TRY(cudaMemcpyAsync(dmaps, maps.data(), sizeof(CUtensorMap) * count, cudaMemcpyHostToDevice, s));
    AP_CUDA_TRY(cudaMemcpyAsync(dprobs, probs.data(), sizeof(GroupProblem) * count, cudaMemcpyHostToDevice, s));
    AP_CUDA_TRY(cudaMemcpyAsync(dtiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, s));
    CUtensorMap ma, mb;
    AP_TRY(make_map(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (void*)Xb, dpad, rows, (uint64_t)dpad * 2, BK, BM,
                    CU_TENSOR_MAP_SWIZZLE_128B));
    AP_TRY(make_map(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (void*)Xb, dpad, rows, (uint64_t)dpad * 2, BK, BN,
                    CU_TENSOR_MAP_SWIZZLE_128B));
    Params p{};
    p.M = p.N = 0;
    p.K = dpad;
    p.mode = SIM;
    p.anrm = nrm;
    p.bnrm = nrm;
    p.diag_zero = 1;
    p.tiles = dtiles;
    p.probs = dprobs;
    p.ntiles = (int)tiles.size();
    p.spin_limit = 1u << 22;
    p.error = err;
    // the output map argument is unused in grouped mode (each problem has its own)
    return launch(ma, mb, maps[0], p, p.ntiles, s);
}

// arg[i] = argmax_j (2 a_i . b_j - bnrm_j), j < nb; A [>= na rows x dpad],
// B [>= ceil(nb/256)*256 rows x dpad] bf16 (padding rows zero), bnrm with
// ceil(nb/256)*256 entries.  best[i] (optional) = that maximum score.  With
// arg2 (and best2) given, also the runner-up column and score (-1 and -inf
// when nb == 1).
static int32_t assign_launch(const __nv_bfloat16* A, int na, const __nv_bfloat16* B, int nb,
                             const float* bnrm, int dpad, int32_t* arg, float* best, int32_t* arg2,
                             float* best2, int32_t* err, cudaStream_t s) {
    using namespace tc;
    if (dpad % BK || nb < 1 || na < 1 || (arg2 && !best2)) return AP_ERR_INVALID_ARG;
    const int arows = (na + BM - 1) / BM * BM;
    const int brows = (nb + BN - 1) / BN * BN;
    CUtensorMap ma, mb;
    AP_TRY(make_map(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (void*)A, dpad, arows, (uint64_t)dpad * 2,
                    BK, BM, CU_TENSOR_MAP_SWIZZLE_128B));
    AP_TRY(make_map(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (void*)B, dpad, brows, (uint64_t)dpad * 2,
                    BK, BN, CU_TENSOR_MAP_SWIZZLE_128B));
    Params p{};
    p.M = na;
    p.N = nb;
    p.K = dpad;
    p.mode = arg2 ? TOP2 : ARGMAX;
    p.bnrm = bnrm;
    p.arg = arg;
    p.best = best;
    p.arg2 = arg2;
    p.best2 = best2;
    p.spin_limit = 1u << 22;
    p.error = err;
    return launch(ma, mb, ma, p, (na + BM - 1) / BM, s);                  // row blocks
}

int32_t tc_assign_argmax(const __nv_bfloat16* A, int na, const __nv_bfloat16* B, int nb,
                         const float* bnrm, int dpad, int32_t* arg, float* best, int32_t* err,
                         cudaStream_t s) {
    return assign_launch(A, na, B, nb, bnrm, dpad, arg, best, nullptr, nullptr, err, s);
}

int32_t tc_assign_top2(const __nv_bfloat16* A, int na, const __nv_bfloat16* B, int nb,
                       const float* bnrm, int dpad, int32_t* arg, float* best, int32_t* arg2,
                       float* best2, int32_t* err, cudaStream_t s) {
    return assign_launch(A, na, B, nb, bnrm, dpad, arg, best, arg2, best2, err, s);
}

}  // namespace apgb
