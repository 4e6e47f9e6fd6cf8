// Host/device interface of the tcgen05 BF16 GEMM used by the sigma sandwich.
#pragma once
#include <cuda.h>

#include "common.cuh"

namespace pprpa {

constexpr int TC_MAX_STAGES = 8;

struct TcParams {
    int mode = 0;      // 0: stage 1 (BF16 T output), 1: stage 2 (FP32 atomic O output)
    int BN = 256;      // N tile (multiple of 16, <= 256)
    int stages = 0;    // set by the launcher
    int slot_bn = 0;   // B-tile width the shared-memory slots and TMEM accumulators are sized for
    int tmem_cols = 0; // set by the launcher
    int total_items = 0;
    int kb_total = 0;  // 64-wide K blocks per work item before splitting
    int* status = nullptr;
    // limit of each pipeline wait (ns); set by the launcher (PPRPA_TC_WAIT_NS, default 4 s).
    // The drains after an expired wait keep the fixed 4 s limit.
    unsigned long long wait_ns = 4000000000ull;
    // stage 1
    int tiles_n = 0;
    int64_t M_rows = 0;  // naux * n_pad
    int a_col_off = 0;   // K offset of the block inside L_pad columns
    int n_per_j = 0;     // columns per vector (block size)
    int n_total = 0;     // k * n_per_j
    int t_col_off = 0;   // column offset of the block in T rows
    int n_pad = 0;
    int k_vec = 0;
    __nv_bfloat16* t_hi = nullptr;
    __nv_bfloat16* t_lo = nullptr;
    // stage 2
    const int4* tile_list = nullptr;  // (m tile, first column, width, 0) of each output tile
    int ntiles = 0, nbatch = 0, nsplit = 1;
    int kq_blocks = 0;   // ceil(n_pad / 64)
    int row_off = 0, col_off = 0;
    int m_valid = 0, n_valid = 0;
    float* O = nullptr;  // [k][n_pad][n_pad]
    // FP8 stage 1: T = row_scale[R / n_pad] * col_scale[j] * (L8 Z8)
    const float* row_scale = nullptr;
    const float* col_scale = nullptr;
    // set by the launcher: shared memory past the pipeline slots holds one 32 x 128-byte
    // staging tile per epilogue warp, used to write stage-1 output rows coalesced
    int epi_stage = 0;
    int t_store = 0;  // set by the launcher: stage-1 T written by bulk tensor stores
};

// Batched form: one job per (molecule, stage block); tensor maps and parameters in global
// memory (aligned as CUtensorMap requires), one work item per output tile (and K slice).
struct TcJob {
    CUtensorMap a_hi, a_lo, b_hi, b_lo;
    TcParams p;
};
struct TcItem {
    int job, m0, n0, batch, kb0, kb1, nw, pad;  // nw: MMA N of the item (<= its job's BN)
};

int make_tmap_bf16(CUtensorMap* map, const void* ptr, int rank, const uint64_t* dims,
                   const uint64_t* strides_bytes, const uint32_t* box);
int make_tmap(CUtensorMap* map, const void* ptr, int rank, const uint64_t* dims,
              const uint64_t* strides_bytes, const uint32_t* box, int elt_bytes);
int tc_stages_for(int BN, int nterms, bool epi_stage = false);
// t_hi / t_lo (stage 1, optional): 3-D maps of T (column in the block, vector, row) with a
// 64 x 1 x 32 box and 128-byte swizzle, for bulk tensor stores of the output.
int tc_gemm_launch(const CUtensorMap& a_hi, const CUtensorMap& a_lo, const CUtensorMap& b_hi,
                   const CUtensorMap& b_lo, TcParams p, int nterms, int num_sms,
                   cudaStream_t st, bool f8 = false, const CUtensorMap* t_hi = nullptr,
                   const CUtensorMap* t_lo = nullptr);
int tc_gemm_launch_cluster(const CUtensorMap& a_hi, const CUtensorMap& a_lo,
                           const CUtensorMap& b_hi_part, const CUtensorMap& b_lo_part, TcParams p,
                           int nterms, int cl, int num_sms, cudaStream_t st, bool f8 = false,
                           bool pair = false, const CUtensorMap* t_hi = nullptr,
                           const CUtensorMap* t_lo = nullptr);
int tc_gemm_launch_batched(const TcJob* jobs, const TcItem* items, int total_items, int max_bn,
                           int nterms, int num_sms, int* status, cudaStream_t st);

}  // namespace pprpa
