// Optional per-kernel timing: when enabled on a pattern handle, every kernel the
// library launches for it is bracketed by a CUDA event pair on its stream.
#pragma once

#include "fe_internal.cuh"

enum fe_kernel_slot {
  FE_K_SPLIT = 0, FE_K_CHUNK, FE_K_FIXUP, FE_K_ELEM_KG, FE_K_GATHER, FE_K_ATOMIC, FE_K_MEMSET,
  FE_K_ELAS_CHUNK, FE_K_ELAS_FIXUP, FE_K_BWD_CHUNK, FE_K_BWD_FIXUP, FE_K_BWD_REDUCE, FE_K_NSLOTS
};

int fe_prof_begin(fe_pattern_s* h, int slot, cudaStream_t s);
int fe_prof_end(fe_pattern_s* h, int slot, cudaStream_t s);

#define FE_PROF_BEGIN(h, slot, s) FE_TRY(fe_prof_begin((h), (slot), (s)))
#define FE_PROF_END(h, slot, s) FE_TRY(fe_prof_end((h), (slot), (s)))
