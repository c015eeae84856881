// pap_run: partition affinity propagation, Algorithm 2 (Section 3).
// Step 1 partitions the points; Step 2 runs the diagonal blocks S_jj as one
// batched Algorithm-1 run on a packed, 16-byte aligned copy of the blocks;
// Step 3 scatters their availabilities into a zeroed A (block-diagonal A');
// Step 4 runs Algorithm 1 on the whole S from (R = 0, A = A').
#include <algorithm>
#include <climits>
#include <vector>

#include "common.cuh"

namespace apgb {

int32_t exemplars_impl(const float* S, const float* R, const float* A, int64_t n, int64_t ld,
                       int32_t* idx, ap_result* out, void* ws, size_t ws_bytes, cudaStream_t s);
size_t exemplars_ws_bytes(int64_t n);

struct Block {
    int64_t off;      // first point
    int64_t m;        // points
    int64_t arena;    // element offset of the packed block
    int64_t ld;       // packed leading dimension
};

// Copies S_jj (rows/columns [off, off+m)) into its packed slot, one block per
// blockIdx.y, rows strided over blockIdx.x.
__global__ void gather_blocks_kernel(const float* __restrict__ S, int64_t lds,
                                     const Block* __restrict__ blocks, float* arena) {
    const Block b = blocks[blockIdx.y];
    for (int64_t i = blockIdx.x; i < b.m; i += gridDim.x) {
        const float* src = S + (b.off + i) * lds + b.off;
        float* dst = arena + b.arena + i * b.ld;
        for (int64_t k = threadIdx.x; k < b.m; k += blockDim.x) dst[k] = src[k];
    }
}

// A'(off+i, off+k) = A_jj(i, k): the block-diagonal merge of Step 3.
__global__ void scatter_blocks_kernel(const float* __restrict__ arena,
                                      const Block* __restrict__ blocks, float* A, int64_t lda) {
    const Block b = blocks[blockIdx.y];
    for (int64_t i = blockIdx.x; i < b.m; i += gridDim.x) {
        const float* src = arena + b.arena + i * b.ld;
        float* dst = A + (b.off + i) * lda + b.off;
        for (int64_t k = threadIdx.x; k < b.m; k += blockDim.x) dst[k] = src[k];
    }
}

static int32_t make_blocks(int64_t n, int32_t k, const int64_t* part, std::vector<Block>* blocks,
                           int64_t* arena_elems) {
    if (k < 1 || k > n) return AP_ERR_INVALID_ARG;
    std::vector<int64_t> off(k + 1);
    if (part) {
        for (int j = 0; j <= k; ++j) off[j] = part[j];
        if (off[0] != 0 || off[k] != n) return AP_ERR_INVALID_ARG;
    } else {
        const int64_t m = n / k;               // Section 3, Step 1
        for (int j = 0; j < k; ++j) off[j] = j * m;
        off[k] = n;
    }
    blocks->resize(k);
    int64_t at = 0;
    for (int j = 0; j < k; ++j) {
        const int64_t m = off[j + 1] - off[j];
        if (m < 2) return AP_ERR_INVALID_ARG;
        Block b;
        b.off = off[j];
        b.m = m;
        b.ld = (m + 31) / 32 * 32;
        b.arena = at;
        at += b.m * b.ld;
        (*blocks)[j] = b;
    }
    *arena_elems = at;
    return AP_OK;
}

struct PapWs {
    Block* blocks;
    float *Sa, *Ra, *Aa;
    void* sub_ws;
    size_t sub_bytes;
    void* full_ws;
    size_t full_bytes;
};

static int32_t carve_pap(void* ws, int64_t n, int64_t ld, const std::vector<Block>& blocks,
                         int64_t arena, PapWs* w, size_t* total) {
    std::vector<int64_t> ms(blocks.size()), lds(blocks.size());
    for (size_t j = 0; j < blocks.size(); ++j) {
        ms[j] = blocks[j].m;
        lds[j] = blocks[j].ld;
    }
    const size_t sub = ap_iterate_batched_workspace_size(ms.data(), lds.data(), (int32_t)blocks.size());
    const size_t full = std::max(ap_iterate_workspace_size(n, ld), exemplars_ws_bytes(n));
    if (sub == 0 || full == 0) return AP_ERR_UNSUPPORTED;
    Carver c(ws);
    w->blocks = c.take<Block>(blocks.size());
    w->Sa = c.take<float>(arena);
    w->Ra = c.take<float>(arena);
    w->Aa = c.take<float>(arena);
    w->sub_ws = c.take<char>(sub);
    w->sub_bytes = sub;
    w->full_ws = c.take<char>(full);
    w->full_bytes = full;
    *total = c.used;
    return AP_OK;
}

}  // namespace apgb

using namespace apgb;

APGB_API size_t pap_run_workspace_size(int64_t n, int64_t ld, int32_t k, const int64_t* part) {
    if (n < 2 || ld < n || n > INT_MAX / 4) return 0;
    std::vector<Block> blocks;
    int64_t arena = 0;
    if (make_blocks(n, k, part, &blocks, &arena) != AP_OK) return 0;
    PapWs w;
    size_t total = 0;
    if (carve_pap(nullptr, n, ld, blocks, arena, &w, &total) != AP_OK) return 0;
    return total;
}

APGB_API int32_t pap_run(const float* S, int64_t n, int64_t ld, int32_t k, const int64_t* part,
                         const ap_params* params, float* R, float* A, int32_t* idx,
                         pap_result* out, void* ws, size_t ws_bytes, void* stream) {
    if (!S || !R || !A || !idx || !out || !params || n < 2 || ld < n || (ld & 3) ||
        !aligned16(S) || !aligned16(R) || !aligned16(A))
        return AP_ERR_INVALID_ARG;
    AP_TRY(require_sm103());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<Block> blocks;
    int64_t arena = 0;
    AP_TRY(make_blocks(n, k, part, &blocks, &arena));
    PapWs w;
    size_t need = 0;
    AP_TRY(carve_pap(nullptr, n, ld, blocks, arena, &w, &need));
    AP_TRY(check_ws(ws, ws_bytes, need));
    carve_pap(ws, n, ld, blocks, arena, &w, &need);

    cudaEvent_t ev[5];
    for (auto& e : ev) AP_CUDA_TRY(cudaEventCreate(&e));
    struct Guard {
        cudaEvent_t* e;
        ~Guard() { for (int i = 0; i < 5; ++i) cudaEventDestroy(e[i]); }
    } guard{ev};

    // Step 1-2: pack the diagonal blocks and run them together
    AP_CUDA_TRY(cudaEventRecord(ev[0], s));
    AP_CUDA_TRY(cudaMemcpyAsync(w.blocks, blocks.data(), sizeof(Block) * blocks.size(),
                                cudaMemcpyHostToDevice, s));
    const int kk = (int)blocks.size();
    int64_t mmax = 0;
    for (auto& b : blocks) mmax = std::max(mmax, b.m);
    const dim3 grid((unsigned)std::min<int64_t>(mmax, 1024), kk);
    gather_blocks_kernel<<<grid, 256, 0, s>>>(S, ld, w.blocks, w.Sa);
    AP_CUDA_TRY(cudaMemsetAsync(w.Ra, 0, sizeof(float) * arena, s));
    AP_CUDA_TRY(cudaMemsetAsync(w.Aa, 0, sizeof(float) * arena, s));
    note_launches(1);
    AP_TRY(last_error());
    std::vector<int64_t> offs(kk), ms(kk), lds(kk);
    for (int j = 0; j < kk; ++j) {
        offs[j] = blocks[j].arena;
        ms[j] = blocks[j].m;
        lds[j] = blocks[j].ld;
    }
    std::vector<ap_result> sub(kk);
    const int32_t st_sub = ap_iterate_batched(w.Sa, w.Ra, w.Aa, offs.data(), ms.data(), lds.data(),
                                              kk, params, nullptr, sub.data(), w.sub_ws,
                                              w.sub_bytes, stream);
    if (st_sub < 0) return st_sub;
    AP_CUDA_TRY(cudaEventRecord(ev[1], s));

    // Step 3: A' = blockdiag(A_jj), R = 0 (or R' = blockdiag(R_jj) with AP_FLAG_PAP_CARRY_R)
    AP_CUDA_TRY(cudaMemset2DAsync(A, ld * sizeof(float), 0, n * sizeof(float), n, s));
    AP_CUDA_TRY(cudaMemset2DAsync(R, ld * sizeof(float), 0, n * sizeof(float), n, s));
    scatter_blocks_kernel<<<grid, 256, 0, s>>>(w.Aa, w.blocks, A, ld);
    note_launches(1);
    if (params->flags & AP_FLAG_PAP_CARRY_R) {
        scatter_blocks_kernel<<<grid, 256, 0, s>>>(w.Ra, w.blocks, R, ld);
        note_launches(1);
    }
    AP_TRY(last_error());
    AP_CUDA_TRY(cudaEventRecord(ev[2], s));

    // Step 4: Algorithm 1 on S from (0, A')
    ap_result fin;
    const int32_t st_fin = ap_iterate(S, R, A, n, ld, params, nullptr, &fin, w.full_ws,
                                      w.full_bytes, stream);
    if (st_fin < 0) return st_fin;
    AP_CUDA_TRY(cudaEventRecord(ev[3], s));
    const int32_t iters = fin.iters, conv = fin.converged;
    const int32_t st_ex = exemplars_impl(S, R, A, n, ld, idx, &fin, w.full_ws, w.full_bytes, s);
    if (st_ex < 0) return st_ex;
    fin.iters = iters;
    fin.converged = conv;
    AP_CUDA_TRY(cudaEventRecord(ev[4], s));
    AP_CUDA_TRY(cudaEventSynchronize(ev[4]));

    *out = pap_result{};
    out->k = kk;
    for (int j = 0; j < kk; ++j) {
        out->sub_iters_max = std::max(out->sub_iters_max, sub[j].iters);
        out->sub_iters_sum += sub[j].iters;
        out->sub_not_converged += (params->conv_iter > 0 && !sub[j].converged) ? 1 : 0;
    }
    float ms_[4];
    for (int i = 0; i < 4; ++i) AP_CUDA_TRY(cudaEventElapsedTime(&ms_[i], ev[i], ev[i + 1]));
    out->sub_ms = ms_[0];
    out->merge_ms = ms_[1];
    out->final_ms = ms_[2];
    out->exemplars_ms = ms_[3];
    out->final = fin;
    const int32_t status = std::max(st_fin, st_ex);
    out->final.status = status;
    return status;
}
