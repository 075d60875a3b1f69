// C ABI entry points: handle queries, strategy selection, status, and the
// argument checks of the assembly calls.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "fe_internal.cuh"
#include "plan.cuh"
#include "tma.cuh"

int fe_launch_scalar_f64(fe_pattern_s* h, int kind, const double* q, const void* w, int w_kind,
                         void* vals, cudaStream_t s);
int fe_launch_scalar_f32(fe_pattern_s* h, int kind, const double* q, const void* w, int w_kind,
                         void* vals, cudaStream_t s);
int fe_launch_pair_f64(fe_pattern_s* h, const double* q, const void* w, int w_kind, void* vals_mass,
                       void* vals_stiff, cudaStream_t s);
int fe_launch_pair_f32(fe_pattern_s* h, const double* q, const void* w, int w_kind, void* vals_mass,
                       void* vals_stiff, cudaStream_t s);
int fe_launch_pair_f64x(fe_pattern_s* h, const double* q, const void* w, int w_kind, void* vals_mass,
                        void* vals_stiff, cudaStream_t s);
int fe_launch_f64x(fe_pattern_s* h, int kind, const double* q, const void* w, int w_kind, void* vals,
                   cudaStream_t s);
int fe_launch_boundary(fe_pattern_s* h, int kind, const double* q, const void* w, int w_kind, int prec,
                       void* vals, cudaStream_t s);
int fe_launch_elas(fe_pattern_s* h, const double* q, const void* lam, int lam_kind, const void* mu,
                   int mu_kind, int prec, void* vals, cudaStream_t s);
int fe_launch_general(fe_pattern_s* h, const double* q, const void* coef, int coef_kind, int prec,
                      void* vals, cudaStream_t s);
int fe_launch_pk_mass(fe_pattern_s* h, const double* q, int prec, void* vals, cudaStream_t s);
int fe_launch_backward(fe_pattern_s* h, const double* q, const void* w, int w_kind, const void* u,
                       const void* v, void* L, void* dLdw, void* dLdq, int prec, cudaStream_t s);
int fe_launch_vjp(fe_pattern_s* h, const double* q, const void* w, int w_kind, const void* grad_vals,
                  void* dLdw, void* dLdq, int prec, cudaStream_t s);

namespace {
thread_local char g_last_cuda_error[256] = "";  // per calling host thread
}

int fe_cuda_fail(cudaError_t e) {
  snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s", cudaGetErrorString(e));
  cudaGetLastError();  // clear a non-sticky error
  return e == cudaErrorMemoryAllocation ? FE_ERR_NOMEM : FE_ERR_CUDA;
}

int fe_malloc(fe_pattern_s* h, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 1);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fe_cuda_fail(e);
  }
  h->bytes += (int64_t)bytes;
  return FE_OK;
}

void fe_free_all(fe_pattern_s* h) {
  fe_host_pipe_free(h);  // first: its streams may still hold work on the pattern's buffers
  void* ptrs[] = {h->me_int,  h->order,    h->row_ptr_s, h->col_idx_s, h->slot2nnz,
                  h->nnz_slot_ptr, h->nnz2slot, h->ch_v_ptr, h->ch_e_ptr, h->lv_off,
                  h->le_off,  h->inc_v,    h->inc_e,     h->lv_dst,    h->lv_vid,
                  h->le_dst,  h->sh_ptr,   h->sh_dst,    h->partials,  h->kg,
                  h->qsplit,  h->status, h->rec, h->rec_off16,
                  h->lv_str,  h->le_str,   h->sh_str,    h->vmap_ptr,  h->vmap,
                  h->bwd_scratch, h->bwd_lpart, h->pk_tab};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->m > 1) {
    if (h->row_ptr) cudaFree(h->row_ptr);
    if (h->col_idx) cudaFree(h->col_idx);
  }
  fe_prof_free(h);
}

int fe_ensure_scratch(fe_pattern_s* h, int strategy) {
  if (!h->qsplit) {
    h->qsplit_bytes = (size_t)h->nq * (h->d == 3 ? 32 : 16);
    FE_TRY(fe_malloc(h, &h->qsplit, h->qsplit_bytes));
  }
  if (strategy == FE_REASM_GATHER && !h->kg) {
    const int nl = h->nv * h->m;
    h->kg_bytes = (size_t)h->nme * nl * nl * sizeof(double);
    FE_TRY(fe_malloc(h, &h->kg, h->kg_bytes));
  }
  return FE_OK;
}

extern "C" {

const char* fe_version(void) {
#ifdef FE_CHECKED
  return "fe_gb300 0.1 (sm_103a, bounds-checked)";
#else
  return "fe_gb300 0.1 (sm_103a)";
#endif
}

const char* fe_last_cuda_error(void) { return g_last_cuda_error; }
}  // extern "C"

int fe_smem_limit_raw(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> raised;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fe_cuda_fail(e);
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = raised[{kernel, dev}];
  if (bytes <= have) return FE_OK;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return fe_cuda_fail(e);
  have = bytes;
  return FE_OK;
}

extern "C" {

int fe_pattern_csr(fe_pattern_h h, int64_t* n, int64_t* nnz, const int32_t** row_ptr,
                   const int32_t** col_idx) {
  if (!h) return FE_ERR_ARG;
  if (n) *n = h->n;
  if (nnz) *nnz = h->nnz;
  if (row_ptr) *row_ptr = h->row_ptr;
  if (col_idx) *col_idx = h->col_idx;
  return FE_OK;
}

int fe_pattern_slot_map(fe_pattern_h h, const int32_t** slot2nnz, const int32_t** nnz_slot_ptr,
                        const int32_t** nnz2slot) {
  if (!h) return FE_ERR_ARG;
  if (slot2nnz) *slot2nnz = h->slot2nnz;
  if (nnz_slot_ptr) *nnz_slot_ptr = h->nnz_slot_ptr;
  if (nnz2slot) *nnz2slot = h->nnz2slot;
  return FE_OK;
}

int fe_pattern_copy_csr(fe_pattern_h h, int32_t* row_ptr, int32_t* col_idx, void* stream) {
  if (!h) return FE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (row_ptr)
    FE_CUDA_TRY(cudaMemcpyAsync(row_ptr, h->row_ptr, sizeof(int32_t) * (h->n + 1),
                                cudaMemcpyDeviceToDevice, s));
  if (col_idx)
    FE_CUDA_TRY(cudaMemcpyAsync(col_idx, h->col_idx, sizeof(int32_t) * h->nnz,
                                cudaMemcpyDeviceToDevice, s));
  return FE_OK;
}

int fe_pattern_copy_slot_map(fe_pattern_h h, int32_t* slot2nnz, int32_t* nnz_slot_ptr,
                             int32_t* nnz2slot, int32_t* order, void* stream) {
  if (!h) return FE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nslots = (size_t)h->nme * h->nv * h->nv;
  if (slot2nnz)
    FE_CUDA_TRY(cudaMemcpyAsync(slot2nnz, h->slot2nnz, sizeof(int32_t) * nslots,
                                cudaMemcpyDeviceToDevice, s));
  if (nnz_slot_ptr)
    FE_CUDA_TRY(cudaMemcpyAsync(nnz_slot_ptr, h->nnz_slot_ptr, sizeof(int32_t) * (h->nnz_s + 1),
                                cudaMemcpyDeviceToDevice, s));
  if (nnz2slot)
    FE_CUDA_TRY(cudaMemcpyAsync(nnz2slot, h->nnz2slot, sizeof(int32_t) * nslots,
                                cudaMemcpyDeviceToDevice, s));
  if (order)
    FE_CUDA_TRY(cudaMemcpyAsync(order, h->order, sizeof(int32_t) * h->nme,
                                cudaMemcpyDeviceToDevice, s));
  return FE_OK;
}

int fe_pattern_dims(fe_pattern_h h, int32_t* d, int32_t* m, int64_t* nq, int64_t* nme, int64_t* n,
                    int64_t* nnz) {
  if (!h) return FE_ERR_ARG;
  if (d) *d = h->d;
  if (m) *m = h->m;
  if (nq) *nq = h->nq;
  if (nme) *nme = h->nme;
  if (n) *n = h->n;
  if (nnz) *nnz = h->nnz;
  return FE_OK;
}

int fe_pattern_element_order(fe_pattern_h h, const int32_t** order) {
  if (!h || !order) return FE_ERR_ARG;
  *order = h->order;
  return FE_OK;
}

int fe_pattern_set_strategy(fe_pattern_h h, int32_t strategy) {
  if (!h) return FE_ERR_ARG;
  if (strategy != FE_REASM_CHUNKED && strategy != FE_REASM_GATHER && strategy != FE_REASM_ATOMIC)
    return FE_ERR_ARG;
  FE_TRY(fe_ensure_scratch(h, strategy));
  h->strategy = strategy;
  return FE_OK;
}

int fe_pattern_set_threads(fe_pattern_h h, int32_t threads) {
  if (!h || (threads != 128 && threads != 256 && threads != 512)) return FE_ERR_ARG;
  h->threads = threads;
  return FE_OK;
}

int fe_pattern_set_persistent(fe_pattern_h h, int32_t persistent) {
  if (!h || (persistent != 0 && persistent != 1)) return FE_ERR_ARG;
  h->persistent = persistent;
  return FE_OK;
}

int fe_pattern_memory(fe_pattern_h h, int64_t* bytes) {
  if (!h || !bytes) return FE_ERR_ARG;
  *bytes = h->bytes;
  return FE_OK;
}

int fe_pattern_plan_info(fe_pattern_h h, int64_t* chunk, int64_t* local_vertices,
                         int64_t* local_edges, int64_t* partial_vertices, int64_t* partial_edges,
                         int64_t* shared_vertices, int64_t* shared_edges, int64_t* plan_bytes) {
  if (!h) return FE_ERR_ARG;
  if (chunk) *chunk = h->chunk;
  if (local_vertices) *local_vertices = h->nlv;
  if (local_edges) *local_edges = h->nle;
  if (partial_vertices) *partial_vertices = h->npart_v;
  if (partial_edges) *partial_edges = h->npart - h->npart_v;
  if (shared_vertices) *shared_vertices = h->nsh_v;
  if (shared_edges) *shared_edges = h->nsh_e;
  if (plan_bytes) *plan_bytes = h->plan_bytes;
  return FE_OK;
}

int fe_pattern_plan_record(fe_pattern_h h, int64_t c, const void** rec, int64_t* bytes) {
  if (!h || !rec || !bytes || !h->rec || c < 0 || c >= h->nchunks) return FE_ERR_ARG;
  int32_t v[2], e[2];
  uint32_t off16;
  FE_CUDA_TRY(cudaDeviceSynchronize());
  FE_CUDA_TRY(cudaMemcpy(v, h->ch_v_ptr + c, sizeof(v), cudaMemcpyDeviceToHost));
  FE_CUDA_TRY(cudaMemcpy(e, h->ch_e_ptr + c, sizeof(e), cudaMemcpyDeviceToHost));
  FE_CUDA_TRY(cudaMemcpy(&off16, h->rec_off16 + c, sizeof(off16), cudaMemcpyDeviceToHost));
  const int64_t ne = std::min<int64_t>(h->chunk, h->nme - c * h->chunk);
  const fe::RecLayout R = fe::rec_layout((uint32_t)ne, (uint32_t)h->nv, (uint32_t)h->npair,
                                         (uint32_t)(v[1] - v[0]), (uint32_t)(e[1] - e[0]), h->m > 1);
  *rec = h->rec + (int64_t)off16 * 16;
  *bytes = R.total;
  return FE_OK;
}

int fe_pattern_destroy(fe_pattern_h h) {
  if (!h) return FE_ERR_ARG;
  cudaDeviceSynchronize();
  fe_free_all(h);
  delete h;
  return FE_OK;
}

int fe_status(fe_pattern_h h, void* stream, int32_t* code, int64_t* id) {
  if (!h) return FE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  fe_status_word st;
  FE_CUDA_TRY(cudaMemcpyAsync(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost, s));
  FE_CUDA_TRY(cudaStreamSynchronize(s));
  fe_status_word init = {0, 0, ~0ull};
  FE_CUDA_TRY(cudaMemcpyAsync(h->status, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  FE_CUDA_TRY(cudaStreamSynchronize(s));
  if (code) *code = st.code;
  if (id) *id = (st.id == ~0ull) ? -1 : (int64_t)st.id;
  return FE_OK;
}

static int check_common(fe_pattern_h h, const double* q, int32_t prec, const void* vals) {
  if (!h || !q || !vals) return FE_ERR_ARG;
  if (prec != FE_F64 && prec != FE_F32) return FE_ERR_ARG;
  return FE_OK;
}

static int scalar_call(fe_pattern_h h, int kind, const double* q, const void* w, int32_t w_kind,
                       int32_t prec, void* vals, void* stream) {
  if (h && h->pk > 1) {  // P_k patterns: the mass matrix only
    FE_TRY(check_common(h, q, prec == FE_F64X ? FE_F64 : prec, vals));  // F64X: double values
    if (kind != 0) return FE_ERR_ARG;
    return fe_launch_pk_mass(h, q, prec, vals, (cudaStream_t)stream);
  }
  if (h && h->kdim != h->d) {  // boundary facets: mass and weighted mass only
    FE_TRY(check_common(h, q, prec == FE_F64X ? FE_F64 : prec, vals));  // F64X: double data
    if (w_kind != FE_COEF_NONE && !w) return FE_ERR_ARG;
    return fe_launch_boundary(h, kind, q, w, w_kind, prec, vals, (cudaStream_t)stream);
  }
  if (prec == FE_F64X) {  // volume patterns, scalar operators
    if (!h || !q || !vals || h->m != 1) return FE_ERR_ARG;
    if ((h->flags & FE_PATTERN_INTERLEAVED) && h->strategy == FE_REASM_CHUNKED) return FE_ERR_ARG;
    if (w_kind != FE_COEF_NONE && !w) return FE_ERR_ARG;
    return fe_launch_f64x(h, kind, q, w, w_kind, vals, (cudaStream_t)stream);
  }
  FE_TRY(check_common(h, q, prec, vals));
  if (h->m != 1) return FE_ERR_ARG;
  if (w_kind != FE_COEF_NONE && !w) return FE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == FE_F64) return fe_launch_scalar_f64(h, kind, q, w, w_kind, vals, s);
  return fe_launch_scalar_f32(h, kind, q, w, w_kind, vals, s);
}

int fe_assemble_mass(fe_pattern_h h, const double* q, int32_t prec, void* vals, void* stream) {
  return scalar_call(h, 0, q, nullptr, FE_COEF_NONE, prec, vals, stream);
}

int fe_assemble_wmass(fe_pattern_h h, const double* q, const void* w, int32_t w_kind, int32_t prec,
                      void* vals, void* stream) {
  int kind;
  if (w_kind == FE_COEF_P1) kind = 1;
  else if (w_kind == FE_COEF_P0 || w_kind == FE_COEF_P0_INTERNAL) kind = 2;
  else return FE_ERR_ARG;
  return scalar_call(h, kind, q, w, w_kind, prec, vals, stream);
}

int fe_assemble_stiff(fe_pattern_h h, const double* q, const void* w, int32_t w_kind, int32_t prec,
                      void* vals, void* stream) {
  if (w_kind != FE_COEF_NONE && w_kind != FE_COEF_P0 && w_kind != FE_COEF_P0_INTERNAL)
    return FE_ERR_ARG;
  return scalar_call(h, 3, q, w, w_kind, prec, vals, stream);
}

int fe_assemble_wmass_stiff(fe_pattern_h h, const double* q, const void* w, int32_t w_kind, int32_t prec,
                            void* vals_mass, void* vals_stiff, void* stream) {
  FE_TRY(check_common(h, q, prec == FE_F64X ? FE_F64 : prec, vals_mass));  // F64X: double values
  if (!vals_stiff || vals_stiff == vals_mass) return FE_ERR_ARG;
  if (h->m != 1 || h->kdim != h->d || h->pk != 1) return FE_ERR_ARG;
  if (h->flags & FE_PATTERN_INTERLEAVED) return FE_ERR_ARG;
  if (w_kind != FE_COEF_NONE && w_kind != FE_COEF_P0 && w_kind != FE_COEF_P0_INTERNAL) return FE_ERR_ARG;
  if (w_kind != FE_COEF_NONE && !w) return FE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == FE_F64) return fe_launch_pair_f64(h, q, w, w_kind, vals_mass, vals_stiff, s);
  if (prec == FE_F64X) return fe_launch_pair_f64x(h, q, w, w_kind, vals_mass, vals_stiff, s);
  return fe_launch_pair_f32(h, q, w, w_kind, vals_mass, vals_stiff, s);
}

int fe_assemble_elas(fe_pattern_h h, const double* q, const void* lam, int32_t lam_kind,
                     const void* mu, int32_t mu_kind, int32_t prec, void* vals, void* stream) {
  if (prec == FE_F64X) FE_TRY(check_common(h, q, FE_F64, vals));  // F64X: FP64 values and coefficients
  else FE_TRY(check_common(h, q, prec, vals));
  if (h->m != h->d || !lam || !mu) return FE_ERR_ARG;
  auto ok = [](int k) {
    return k == FE_COEF_SCALAR || k == FE_COEF_P0 || k == FE_COEF_P0_INTERNAL || k == FE_COEF_P1;
  };
  if (!ok(lam_kind) || !ok(mu_kind)) return FE_ERR_ARG;
  return fe_launch_elas(h, q, lam, lam_kind, mu, mu_kind, prec, vals, (cudaStream_t)stream);
}

int fe_assemble_general(fe_pattern_h h, const double* q, const void* coef, int32_t coef_kind,
                        int32_t prec, void* vals, void* stream) {
  FE_TRY(check_common(h, q, prec == FE_F64X ? FE_F64 : prec, vals));  // F64X: double data
  if (h->m != 1 || h->kdim != h->d || h->pk != 1 || !coef) return FE_ERR_ARG;
  if ((h->flags & FE_PATTERN_INTERLEAVED) && h->strategy == FE_REASM_CHUNKED) return FE_ERR_ARG;
  if (coef_kind != FE_COEF_SCALAR && coef_kind != FE_COEF_P0 && coef_kind != FE_COEF_P0_INTERNAL &&
      coef_kind != FE_COEF_P1)
    return FE_ERR_ARG;
  return fe_launch_general(h, q, coef, coef_kind, prec, vals, (cudaStream_t)stream);
}

int fe_assemble_stiff_backward(fe_pattern_h h, const double* q, const void* w, int32_t w_kind,
                               const void* u, const void* v, void* L, void* dL_dw, void* dL_dq,
                               int32_t prec, void* stream) {
  if (!h || !q || !u || !v) return FE_ERR_ARG;
  if (prec != FE_F64 && prec != FE_F32 && prec != FE_F64X) return FE_ERR_ARG;
  if (h->m != 1 || h->kdim != h->d || h->pk != 1) return FE_ERR_ARG;
  if (w_kind != FE_COEF_NONE && w_kind != FE_COEF_P0 && w_kind != FE_COEF_P0_INTERNAL)
    return FE_ERR_ARG;
  if (w_kind != FE_COEF_NONE && !w) return FE_ERR_ARG;
  return fe_launch_backward(h, q, w, w_kind, u, v, L, dL_dw, dL_dq, prec, (cudaStream_t)stream);
}

int fe_assemble_stiff_vjp(fe_pattern_h h, const double* q, const void* w, int32_t w_kind,
                          const void* grad_vals, void* dL_dw, void* dL_dq, int32_t prec, void* stream) {
  if (!h || !q || !grad_vals) return FE_ERR_ARG;
  if (prec != FE_F64 && prec != FE_F32 && prec != FE_F64X) return FE_ERR_ARG;
  if (h->m != 1 || h->kdim != h->d || h->pk != 1) return FE_ERR_ARG;
  if (w_kind != FE_COEF_NONE && w_kind != FE_COEF_P0 && w_kind != FE_COEF_P0_INTERNAL)
    return FE_ERR_ARG;
  if (w_kind != FE_COEF_NONE && !w) return FE_ERR_ARG;
  return fe_launch_vjp(h, q, w, w_kind, grad_vals, dL_dw, dL_dq, prec, (cudaStream_t)stream);
}

}  // extern "C"

namespace {
// Self-test of the bounded wait: an mbarrier expects 16 bytes that no copy will bring,
// so the bounded wait runs out; the block reports FE_ERR_TIMEOUT and returns. Nothing
// is in flight when it returns (no copy was issued).
__global__ void k_selftest_wait(uint32_t max_iter, fe_status_word* st) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    fe::mbar_init(&bar, 1);
    fe::mbar_arrive_expect_tx(&bar, 16);
  }
  __syncthreads();
  const bool landed = __syncthreads_and(fe::mbar_wait_bounded(&bar, 0, max_iter));
  if (!landed && threadIdx.x == 0) fe_report(st, FE_ERR_TIMEOUT, 0);
}
}  // namespace

extern "C" int fe_selftest_wait_timeout(int32_t* code, void* stream) {
  if (!code) return FE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  fe_status_word* st = nullptr;
  FE_CUDA_TRY(cudaMalloc(&st, sizeof(fe_status_word)));
  fe_status_word init = {0, 0, ~0ull}, out;
  int rc = FE_OK;
  if (cudaMemcpyAsync(st, &init, sizeof(init), cudaMemcpyHostToDevice, s) != cudaSuccess) rc = FE_ERR_CUDA;
  if (!rc) {
    k_selftest_wait<<<1, 32, 0, s>>>(1u << 12, st);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&out, st, sizeof(out), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = FE_ERR_CUDA;
    else
      *code = out.code;
  }
  cudaFree(st);
  return rc;
}
