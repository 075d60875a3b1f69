// Assembly from and to host memory: the copies and the assembly of successive calls
// overlap. Each call takes one of two staging slots (device copies of q, w and the
// values) and runs on three streams owned by the pattern:
//   in:   wait until the slot's previous download is done, upload q (and w);
//   work: wait for the upload, assemble into the slot's values;
//   out:  wait for the assembly, download the values to the caller's buffer.
// The caller's stream then waits for the download, so a call is stream-ordered for the
// caller like the device-memory calls, while call k+1's upload and call k-1's download
// run beside call k's assembly. All assemblies of a pattern run on its one work stream,
// in call order (they share the pattern's partial-sum scratch).
#include "fe_internal.cuh"

struct fe_host_pipe {
  cudaStream_t in = nullptr, work = nullptr, out = nullptr;
  cudaEvent_t uploaded[2] = {nullptr, nullptr}, assembled[2] = {nullptr, nullptr},
              downloaded[2] = {nullptr, nullptr};
  void* q[2] = {nullptr, nullptr};
  void* w[2] = {nullptr, nullptr};
  void* vals[2] = {nullptr, nullptr};
  size_t w_bytes = 0;
  int slot = 0;
};

void fe_host_pipe_free(fe_pattern_s* h) {
  fe_host_pipe* P = h->pipe;
  if (!P) return;
  for (cudaStream_t s : {P->in, P->work, P->out})
    if (s) cudaStreamSynchronize(s);
  for (int i = 0; i < 2; ++i) {
    for (void* p : {P->q[i], P->w[i], P->vals[i]})
      if (p) cudaFree(p);
    for (cudaEvent_t e : {P->uploaded[i], P->assembled[i], P->downloaded[i]})
      if (e) cudaEventDestroy(e);
  }
  for (cudaStream_t s : {P->in, P->work, P->out})
    if (s) cudaStreamDestroy(s);
  delete P;
  h->pipe = nullptr;
}

namespace {

int ensure_pipe(fe_pattern_s* h, size_t w_bytes) {
  if (!h->pipe) {
    fe_host_pipe* P = new fe_host_pipe();
    h->pipe = P;
    for (cudaStream_t* s : {&P->in, &P->work, &P->out})
      FE_CUDA_TRY(cudaStreamCreateWithFlags(s, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      for (cudaEvent_t* e : {&P->uploaded[i], &P->assembled[i], &P->downloaded[i]})
        FE_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
      FE_TRY(fe_malloc(h, &P->q[i], sizeof(double) * h->d * h->nq));
      FE_TRY(fe_malloc(h, &P->vals[i], sizeof(double) * h->nnz));
      // the first wait on `downloaded` must not block: record it once on an idle stream
      FE_CUDA_TRY(cudaEventRecord(P->downloaded[i], P->out));
    }
  }
  fe_host_pipe* P = h->pipe;
  if (w_bytes > P->w_bytes) {
    for (int i = 0; i < 2; ++i) {
      if (P->w[i]) {
        for (cudaStream_t st : {P->in, P->work, P->out}) FE_CUDA_TRY(cudaStreamSynchronize(st));
        cudaFree(P->w[i]);
        P->w[i] = nullptr;
      }
      FE_TRY(fe_malloc(h, &P->w[i], w_bytes));
    }
    P->w_bytes = w_bytes;
  }
  return FE_OK;
}

}  // namespace

extern "C" int fe_assemble_stiff_host(fe_pattern_h h, const double* q_host, const void* w_host, int32_t w_kind,
                                      int32_t prec, void* vals_host, void* stream) {
  if (!h || !q_host || !vals_host) return FE_ERR_ARG;
  if (prec != FE_F64 && prec != FE_F32 && prec != FE_F64X) return FE_ERR_ARG;
  if (w_kind != FE_COEF_NONE && (w_kind != FE_COEF_P0 || !w_host)) return FE_ERR_ARG;
  const size_t vsz = prec == FE_F32 ? sizeof(float) : sizeof(double);
  const size_t w_bytes = w_kind == FE_COEF_NONE ? 0 : vsz * h->nme;
  FE_TRY(ensure_pipe(h, w_bytes));
  fe_host_pipe* P = h->pipe;
  const int i = P->slot;
  P->slot ^= 1;
  FE_CUDA_TRY(cudaStreamWaitEvent(P->in, P->downloaded[i], 0));
  FE_CUDA_TRY(cudaMemcpyAsync(P->q[i], q_host, sizeof(double) * h->d * h->nq, cudaMemcpyHostToDevice, P->in));
  if (w_bytes) FE_CUDA_TRY(cudaMemcpyAsync(P->w[i], w_host, w_bytes, cudaMemcpyHostToDevice, P->in));
  FE_CUDA_TRY(cudaEventRecord(P->uploaded[i], P->in));
  FE_CUDA_TRY(cudaStreamWaitEvent(P->work, P->uploaded[i], 0));
  FE_TRY(fe_assemble_stiff(h, (const double*)P->q[i], w_bytes ? P->w[i] : nullptr, w_kind, prec, P->vals[i],
                           P->work));
  FE_CUDA_TRY(cudaEventRecord(P->assembled[i], P->work));
  FE_CUDA_TRY(cudaStreamWaitEvent(P->out, P->assembled[i], 0));
  FE_CUDA_TRY(cudaMemcpyAsync(vals_host, P->vals[i], vsz * h->nnz, cudaMemcpyDeviceToHost, P->out));
  FE_CUDA_TRY(cudaEventRecord(P->downloaded[i], P->out));
  FE_CUDA_TRY(cudaStreamWaitEvent((cudaStream_t)stream, P->downloaded[i], 0));
  return FE_OK;
}
