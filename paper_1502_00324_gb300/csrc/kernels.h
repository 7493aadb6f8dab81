// kernels.h -- host-side launch interface of the search kernels.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace fic {

// Arguments of one contraction + scoring launch (one quadtree step of one or
// more images).  The problem table lives in device memory.
struct ContractArgs {
    const Problem* probs;  // n_probs entries (device)
    int n_probs;
    int n_items;           // total work items (sum over problems); with
                           // n_items_dev an upper bound (grid size)
    const int* n_items_dev = nullptr;  // device item count of a graph-captured step
    int K;                 // 16, 64 or 256
    StepParams sp;
    int* err;              // device error word
    int grid_ctas;         // persistent grid size (tensor engines)
    int variant;           // isometry kernel: 0 = 8 epilogue warps, 1 = 16
};

cudaError_t launch_contract_plain(const ContractArgs& a, cudaStream_t s);
cudaError_t launch_contract_tc(const ContractArgs& a, cudaStream_t s);
// Isometry-in-accumulator tensor kernel (K = 16 or 64, |S| <= 3); A in the
// iso-major layout (rows k * Rpad + range, Rpad = rows_pad / 8, a multiple
// of 128); partials per range; gbest per range.
cudaError_t launch_contract_tc_iso(const ContractArgs& a, cudaStream_t s);
bool contract_tc_iso_supports(int K, int ns);
int contract_tc_iso_parts_per_chunk(int variant);
int contract_tc_iso_ntile(int K);
// Domain-side isometry tensor kernel (n = B^2 = 4, 16 or 64, |S| <= 3): A in
// the iso-major layout (isometry 0 block: the ranges as they are), the
// pool operand as gathered; the eight isometries of each domain are built in
// shared memory and their maximum comes from tcgen05.ld.red (sm_103a).
cudaError_t launch_contract_tc_red(const ContractArgs& a, cudaStream_t s);
bool contract_tc_red_supports(int n, int ns);
int contract_tc_red_ntile();
int contract_tc_red_parts_per_chunk();
size_t contract_tc_smem_bytes(int K);
int contract_tc_parts_per_chunk();  // partial bests per (range, column chunk)
int contract_tc_ntile();            // pool columns per tensor-core tile
constexpr int kPlainNTile = 128;    // pool columns per CUDA-core tile

// Step kernels (stages.cu).
// Fixed-point table round(q log2 q 2^49), q = 0 .. count - 1 (count <= 1025).
constexpr int kEntTableCount = 1025;
cudaError_t launch_entropy_table(long long* T, int count, cudaStream_t s);
// Entropy of every 2B x 2B position at step L.  keys == NULL: threshold
// flags (H > thr) and the near-threshold count; else the top-DN keys (and
// rounding-ambiguity flags, consumed by launch_top_select).
cudaError_t launch_entropy(const uint8_t* img, int N, int B, int L, int per, double thr,
                           const long long* T, uint32_t* flags, double* H,
                           unsigned long long* keys, unsigned long long* near, cudaStream_t s);
// Admission flags of the k smallest keys (k < n); adds the positions whose
// rounded entropy is ambiguous near the cut to *near.  state: device
// scratch of select_state_bytes().
size_t select_state_bytes();
cudaError_t launch_top_select(const unsigned long long* keys, int64_t n, int64_t k,
                              void* state, uint32_t* flags, unsigned long long* near,
                              cudaStream_t s, int* launches);
cudaError_t launch_fill_u32(uint32_t* a, int64_t n, uint32_t v, cudaStream_t s);
// Exclusive scan of n uint32 values; *total receives the sum.  tmp holds at
// least scan_tmp_words(n) words.  n_dev (optional, device): scan min(n,
// *n_dev) values instead (grids stay sized for n).
int64_t scan_tmp_words(int64_t n);
cudaError_t launch_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp,
                        uint32_t* total, cudaStream_t s, int* launches,
                        const uint32_t* n_dev = nullptr);
cudaError_t launch_pool_scatter(const uint32_t* flags, const uint32_t* pos, int64_t n_pos,
                                int per, int L, uint32_t* pool_xy, cudaStream_t s);
// Top-level ranges (x | y << 16) of a tops x tops grid of B_max blocks.
cudaError_t launch_init_ranges(uint32_t* act, int tops, int B_max, cudaStream_t s);
// 2x2 box sums of the image, pitch N (entries with x or y = N - 1 unused).
cudaError_t launch_box2(const uint8_t* img, int N, uint16_t* s2, cudaStream_t s);
cudaError_t launch_gather(const uint16_t* s2img, int N, int B, int L, int per,
                          const uint32_t* pool_xy, int64_t dn, int64_t cols_pad, int K,
                          const StepParams& sp, __half* D, float* cf, ColExact* ci,
                          unsigned long long* vd_max, unsigned long long* vd_min_key,
                          cudaStream_t s, const uint32_t* dn_dev = nullptr);
// iso_major = 0: row 8 range + k; 1: row k * (rows_pad / 8) + range.
cudaError_t launch_range_prep(const uint8_t* img, int N, int B, const uint32_t* act, int R,
                              int64_t rows_pad, int K, const StepParams& sp,
                              const unsigned long long* vd_max, int iso_major, __half* A,
                              RowConst* rc, cudaStream_t s, const uint32_t* R_dev = nullptr);
cudaError_t launch_split_decide(const Best* part, int n_chunks, const RowConst* rc, int R,
                                int n, const StepParams& sp, int e16, int last, int dn,
                                const unsigned long long* vd_min_key, Best* best,
                                uint32_t* split, cudaStream_t s, const StepCounts& dc = {});
cudaError_t launch_split_scatter(const uint32_t* act, const Best* best, const uint32_t* split,
                                 const uint32_t* split_pos, const RowConst* rc, int R, int B,
                                 int level, const uint32_t* pool_xy, int per, int L, int dn,
                                 uint32_t* next_act, void* codes, int64_t code_base,
                                 cudaStream_t s, const StepCounts& dc = {});
cudaError_t launch_order_mark(const void* codes, int64_t n_codes, int N, int B_max, int B_min,
                              uint32_t* cellmap, uint32_t* cellflag, cudaStream_t s,
                              const uint32_t* n_dev = nullptr);
cudaError_t launch_order_gather(const void* codes, const uint32_t* cellmap,
                                const uint32_t* cellflag, const uint32_t* rank, int64_t n_cells,
                                void* out, cudaStream_t s);

// Field widths of the stored records per quadtree step.
struct PackLevels {
    int has_pool[4];   // the step's pool is not empty
    int addr_bits[4];  // ceil(log2 DN)
    int s_bits[4];     // ceil(log2 |S|)
};
// Bit fields of n records (device fic_code array) into words (n_words,
// zeroed here); *total_bits (device) receives the payload size.  sizes and
// offs: n words each; scan_tmp: scan_tmp_words(n) words.
cudaError_t launch_pack_records(const void* codes, int64_t n, const PackLevels& pl,
                                uint32_t* sizes, uint32_t* offs, uint32_t* scan_tmp,
                                uint32_t* total_bits, uint32_t* words, int64_t n_words,
                                cudaStream_t s);

// S sets by quadtree step for the decoder (S = p[level][s] / q[level]).
struct DecodeS {
    int B_max;
    int q[4];
    int p[4][16];
};
cudaError_t launch_decode_pass(const void* codes, int64_t n_codes, const DecodeS& ds,
                               const uint8_t* src, uint8_t* dst, int N, unsigned* changed,
                               cudaStream_t s);

}  // namespace fic
