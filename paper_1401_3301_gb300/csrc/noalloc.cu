// fe_assemble_stiff_noalloc: the two-pass stiffness assembly (element matrices to
// scratch, then each nonzero sums its slots in ascending slot order) with its
// scratch in a fixed array that is part of this library's device image, so the
// call allocates no device memory.
//
// Who needs it: callers that may not call cudaMalloc while they assemble. A plugin
// inside a host application that owns the whole device-memory budget cannot take
// memory behind the host's back; a time-stepping loop with a latency budget
// cannot afford cudaMalloc, which may synchronise the device. Such callers build
// the pattern once, up front, and then call this entry point with their own input
// and output buffers.
#include <mutex>

#include "assemble_impl.cuh"

namespace {

// Scratch of the element values: 16 MiB on every device that loads the library,
// held until the process exits.
constexpr size_t kNoAllocScratchBytes = 16u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device. In host code the
// array's name is a host-side stand-in, not a device address; the runtime gives
// the real address, looked up once per device with that device current.
int scratch_address(void** out) {
  int dev = 0;
  FE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return FE_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    FE_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return FE_OK;
}

template <int D, class T>
int launch(fe_pattern_s* h, const fe::ElemArgs& A, T* vals, void* scratch, cudaStream_t s) {
  fe::k_elem_kg<D, T, fe::K_STIFF><<<fe_grid(h->nme, 256), 256, 0, s>>>(A, (T*)scratch);
  FE_CUDA_TRY(cudaGetLastError());
  fe::k_gather<T><<<fe_grid(h->nnz_s, 256), 256, 0, s>>>(h->nnz_slot_ptr, h->nnz2slot, h->nnz_s,
                                                         (const T*)scratch, vals);
  FE_CUDA_TRY(cudaGetLastError());
  return FE_OK;
}

}  // namespace

extern "C" int fe_assemble_stiff_noalloc(fe_pattern_h h, const double* q, const void* w,
                                         int32_t w_kind, int32_t prec, void* vals, void* stream) {
  if (!h || !q || !vals) return FE_ERR_ARG;
  if (prec != FE_F64 && prec != FE_F32) return FE_ERR_ARG;
  if (h->m != 1 || h->kdim != h->d || h->pk != 1) return FE_ERR_ARG;
  if (w_kind != FE_COEF_NONE && w_kind != FE_COEF_P0 && w_kind != FE_COEF_P0_INTERNAL) return FE_ERR_ARG;
  if (w_kind != FE_COEF_NONE && !w) return FE_ERR_ARG;
  const size_t need = (size_t)h->nme * h->nv * h->nv * (prec == FE_F64 ? sizeof(double) : sizeof(float));
  if (need > kNoAllocScratchBytes) return FE_ERR_SCRATCH_LIMIT;
  void* scratch = nullptr;
  FE_TRY(scratch_address(&scratch));
  cudaStream_t s = (cudaStream_t)stream;
  fe::ElemArgs A{h->me_int, h->nme, h->nq, q, nullptr, w, w_kind, h->order, h->status};
  if (prec == FE_F32) {
    // the handle's split-coordinate buffer was allocated when the pattern was built
    float4* qs = (float4*)h->qsplit;
    if (h->d == 3) fe::k_split_q<3><<<fe_grid(h->nq, 256), 256, 0, s>>>(q, h->nq, qs);
    else fe::k_split_q<2><<<fe_grid(h->nq, 256), 256, 0, s>>>(q, h->nq, qs);
    FE_CUDA_TRY(cudaGetLastError());
    A.qs = qs;
    return h->d == 3 ? launch<3, float>(h, A, (float*)vals, scratch, s)
                     : launch<2, float>(h, A, (float*)vals, scratch, s);
  }
  return h->d == 3 ? launch<3, double>(h, A, (double*)vals, scratch, s)
                   : launch<2, double>(h, A, (double*)vals, scratch, s);
}
