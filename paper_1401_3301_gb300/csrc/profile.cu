// Per-kernel CUDA-event timing of a pattern handle (see profile.cuh), and an NVTX range
// named after the kernel around every launch (header-only NVTX 3: a no-op unless a
// profiling tool is attached).
#include <nvtx3/nvToolsExt.h>
#include <string.h>

#include <vector>

#include "profile.cuh"

namespace {
const char* kNames[FE_K_NSLOTS] = {"split_q", "chunk",      "fixup",      "elem_kg",
                                   "gather",  "elem_atomic", "memset",    "elas_chunk",
                                   "elas_fixup", "bwd_chunk", "bwd_fixup", "bwd_reduce"};
}

struct fe_prof_state {
  struct slot_events {
    std::vector<cudaEvent_t> ev;  // start/stop pairs
    size_t used = 0;              // events recorded since the last read
  } slots[FE_K_NSLOTS];
  ~fe_prof_state() {
    for (auto& s : slots)
      for (cudaEvent_t e : s.ev) cudaEventDestroy(e);
  }
};

static int next_event(fe_prof_state::slot_events& se, cudaEvent_t* e) {
  if (se.used == se.ev.size()) {
    cudaEvent_t n;
    FE_CUDA_TRY(cudaEventCreate(&n));
    se.ev.push_back(n);
  }
  *e = se.ev[se.used++];
  return FE_OK;
}

static int record(fe_pattern_s* h, int slot, cudaStream_t s) {
  if (!h->prof) return FE_OK;
  cudaEvent_t e;
  FE_TRY(next_event(h->prof->slots[slot], &e));
  FE_CUDA_TRY(cudaEventRecord(e, s));
  return FE_OK;
}

int fe_prof_begin(fe_pattern_s* h, int slot, cudaStream_t s) {
  nvtxRangePushA(kNames[slot]);
  return record(h, slot, s);
}

int fe_prof_end(fe_pattern_s* h, int slot, cudaStream_t s) {
  nvtxRangePop();
  return record(h, slot, s);
}

void fe_prof_free(fe_pattern_s* h) {
  delete h->prof;
  h->prof = nullptr;
}

extern "C" int fe_profile(fe_pattern_h h, int32_t enable) {
  if (!h) return FE_ERR_ARG;
  if (enable && !h->prof) h->prof = new fe_prof_state();
  if (!enable) fe_prof_free(h);
  return FE_OK;
}

extern "C" int fe_profile_read(fe_pattern_h h, int32_t max_kernels, char* names, double* ms,
                               int64_t* launches, int32_t* count) {
  if (!h || !count) return FE_ERR_ARG;
  *count = 0;
  if (!h->prof) return FE_OK;
  int k = 0;
  for (int slot = 0; slot < FE_K_NSLOTS; ++slot) {
    auto& se = h->prof->slots[slot];
    if (se.used == 0) continue;
    double total = 0.0;
    for (size_t i = 0; i + 1 < se.used; i += 2) {
      FE_CUDA_TRY(cudaEventSynchronize(se.ev[i + 1]));
      float t = 0.f;
      FE_CUDA_TRY(cudaEventElapsedTime(&t, se.ev[i], se.ev[i + 1]));
      total += t;
    }
    if (k < max_kernels) {
      if (names) {
        strncpy(names + 32 * k, kNames[slot], 31);
        names[32 * k + 31] = 0;
      }
      if (ms) ms[k] = total;
      if (launches) launches[k] = (int64_t)(se.used / 2);
    }
    ++k;
    se.used = 0;
  }
  *count = k;
  return FE_OK;
}
