// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/fe.h"

#define FE_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t fe_err_ = (expr);                           \
    if (fe_err_ != cudaSuccess) return fe_cuda_fail(fe_err_); \
  } while (0)

#define FE_TRY(expr)               \
  do {                             \
    int fe_rc_ = (expr);           \
    if (fe_rc_ != FE_OK) return fe_rc_; \
  } while (0)

int fe_cuda_fail(cudaError_t e);  // records the message, returns FE_ERR_CUDA or FE_ERR_NOMEM

// Device status word: code (int32) and smallest offending id (int64).
struct fe_status_word {
  int32_t code;
  int32_t pad;
  unsigned long long id;  // ULLONG_MAX = none
};

__device__ __forceinline__ void fe_report(fe_status_word* st, int32_t code, long long id) {
  atomicCAS(&st->code, 0, code);
  atomicMin(&st->id, (unsigned long long)id);
}

// ---------------------------------------------------------------- pattern handle
struct fe_prof_state;
void fe_prof_free(struct fe_pattern_s* h);
struct fe_host_pipe;
void fe_host_pipe_free(struct fe_pattern_s* h);

struct fe_pattern_s {
  int d = 0, m = 1, nv = 0, npair = 0, flags = 0, strategy = FE_REASM_CHUNKED;
  int threads = 256;                // threads per block of the chunked scalar kernel
  int persistent = 1;               // weighted mass + stiffness kernel: resident grid looping over chunks
  int kdim = 0;                     // element dimension: d (volume) or d - 1 (boundary facets)
  int pk = 1;                       // polynomial degree of the element nodes (App. D); nv nodes
  void* pk_tab = nullptr;           // pk > 1: P_k mass table, double[nv + npair] then float[nv + npair]
  int64_t nq = 0, nme = 0, n = 0, nnz_s = 0, nnz = 0;
  int32_t* me_int = nullptr;        // (d+1) x nme, internal element order
  int32_t* order = nullptr;         // internal -> input element id
  int32_t* row_ptr_s = nullptr;     // scalar CSR (nq+1)
  int32_t* col_idx_s = nullptr;     // scalar CSR (nnz_s)
  int32_t* row_ptr = nullptr;       // CSR of the matrix (== scalar when m == 1)
  int32_t* col_idx = nullptr;
  int32_t* slot2nnz = nullptr;      // nme (d+1)^2
  int32_t* nnz_slot_ptr = nullptr;  // nnz_s + 1
  int32_t* nnz2slot = nullptr;      // nme (d+1)^2
  // element-chunk plan (FE_REASM_CHUNKED). The flat arrays from lv_off to le_str exist
  // only while the plan is built: the per-chunk records (rec) hold copies of their
  // slices, and the flat arrays are released once the records are filled.
  int chunk = 0;
  int64_t nchunks = 0, nlv = 0, nle = 0;
  int32_t* ch_v_ptr = nullptr;      // nchunks + 1: local vertices of chunk c
  int32_t* ch_e_ptr = nullptr;      // nchunks + 1: local edges of chunk c
  uint16_t* lv_off = nullptr;       // nlv: first incidence of local vertex (chunk relative)
  uint16_t* le_off = nullptr;       // nle
  uint16_t* inc_v = nullptr;        // nv nme: e_local * nv + a, grouped by local vertex
  uint16_t* inc_e = nullptr;        // npair nme: ((e_local * npair + p) << 1) | swapped
  int32_t* lv_dst = nullptr;        // nlv: diagonal scalar nnz (>= 0) or -1 - partial index
  int32_t* lv_vid = nullptr;        // nlv: vertex id
  int32_t* le_dst = nullptr;        // 2 nle: scalar nnz (i,j), (j,i) with i < j, or -1 - partial
  uint16_t* lv_str = nullptr;       // m > 1: block row stride of each local vertex (dst = block base)
  uint16_t* le_str = nullptr;       // m > 1: 2 nle block row strides
  int64_t nsh_v = 0, nsh_e = 0;     // shared vertices / edges
  int64_t npart_v = 0, npart = 0;   // partial sums of shared vertices / all partial sums
  int32_t* sh_ptr = nullptr;        // nsh_v + nsh_e + 1: partial ranges (vertices first)
  int32_t* sh_dst = nullptr;        // 2 per shared entity: vertex (diag nnz, vid), edge (nnz_ij, nnz_ji)
  int32_t* sh_str = nullptr;        // m > 1: 2 per shared entity, block row strides
  int64_t plan_bytes = 0;
  uint8_t* rec = nullptr;           // per-chunk plan records (plan.cuh)
  uint32_t* rec_off16 = nullptr;    // nchunks: record offset in 16-byte units
  int64_t rec_bytes = 0, rec_max_bytes = 0;
  int32_t max_lv = 0;               // most local vertices of any chunk
  int32_t max_slots = 0;            // FE_PATTERN_INTERLEAVED: most value slots of any chunk
  // scratch owned by the handle
  void* partials = nullptr; size_t partials_bytes = 0;
  void* kg = nullptr; size_t kg_bytes = 0;
  void* qsplit = nullptr; size_t qsplit_bytes = 0;
  int32_t* vmap_ptr = nullptr;      // nq + 1: vertex -> incidences (backward pass, built on first use)
  int32_t* vmap = nullptr;          // nv nme: e * nv + a, ascending e within each vertex
  void* bwd_scratch = nullptr;      // backward: per-corner gradient contributions
  void* bwd_lpart = nullptr;        // backward: per-block partial sums of L
  fe_status_word* status = nullptr;
  fe_prof_state* prof = nullptr;    // per-kernel event timing (fe_profile)
  fe_host_pipe* pipe = nullptr;     // host-buffer calls: streams, events, staging (host.cu)
  std::vector<int64_t> batch_voff, batch_eoff, batch_noff;  // batches: per-mesh offsets
  int64_t bytes = 0;
};

// ---------------------------------------------------------------- sort.cu
// Stable LSD radix sort of (key, value) pairs on the lowest `bits` key bits.
// Buffers are ping-ponged; on return *keys / *vals point at the sorted data
// (one of the two buffers given).
struct fe_sort_buffers {
  uint64_t* k0; uint64_t* k1;
  uint32_t* v0; uint32_t* v1;
  uint32_t* hist;   // 256 * ntiles
  uint32_t* scan_tmp;
};
size_t fe_sort_hist_size(int64_t n);        // entries of hist for n keys
size_t fe_scan_tmp_size(int64_t n);          // entries of scratch for an exclusive scan of n
int fe_radix_sort(int64_t n, int bits, fe_sort_buffers* b, uint64_t** keys, uint32_t** vals,
                  cudaStream_t s);
// out[i] = sum_{j<i} in[j] (uint32), n entries; out may alias in. tmp: fe_scan_tmp_size(n).
int fe_scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t s);

// Device allocation helpers tracked in the handle's byte count.
int fe_malloc(fe_pattern_s* h, void** p, size_t bytes);
void fe_free_all(fe_pattern_s* h);

// ---------------------------------------------------------------- pk.cu
int fe_pk_nodes(int d, int k);                      // (d+k)! / (d! k!)
int fe_pk_upload_table(fe_pattern_s* h, cudaStream_t s);

// ---------------------------------------------------------------- assemble.cu
int fe_ensure_scratch(fe_pattern_s* h, int strategy);
int fe_build_vertex_map(fe_pattern_s* h, cudaStream_t s);

// Raise a kernel's dynamic shared-memory limit on the current device to at least
// `bytes`: once per (kernel, device) and high-water mark, under a lock, so that the
// attribute is not set again inside a stream capture (every kernel's first launch
// happens outside one) and a process that drives several devices sets it on each.
int fe_smem_limit_raw(const void* kernel, size_t bytes);
template <class K>
int fe_smem_limit(K kernel, size_t bytes) {
  return fe_smem_limit_raw((const void*)kernel, bytes);
}

static inline int fe_grid(int64_t work, int per_block, int max_blocks = 1 << 30) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (int)g;
}
