// Bounds checks of the FE_CHECKED build for the chunked kernels.
//
// fe_record_valid validates a chunk's plan record once it is in shared memory, before
// any index in it is used: offsets ascend from 0 to the incidence counts, every
// incidence code names a corner / element edge of the chunk, every corner's local
// vertex is below nlv and the vertex incidence lists agree with the corner map (each
// corner once in the list of its own local vertex, so the lists are a permutation of
// the corners), every vertex id is below nq, and every destination is a value inside
// the matrix or a partial-sum slot below npart. A failure records FE_ERR_BOUNDS with the
// chunk id and the whole block skips the chunk.
//
// In the normal build FE_RECORD_VALID is the constant true and nothing here is compiled.
#pragma once

#include "fe_internal.cuh"
#include "plan.cuh"

namespace fe {

#ifdef FE_CHECKED
// m: dofs per vertex (m x m blocks at dst + l * stride + n when m > 1)
static __device__ __noinline__ bool fe_record_valid(const unsigned char* rec, const RecLayout& R, int ne, int nv,
                                             int np, int nlv, int nle, int m, int64_t nq, int64_t nnz,
                                             int64_t npart, fe_status_word* st, int64_t c) {
  const uint16_t* lvid = (const uint16_t*)(rec + R.lvid);
  const uint16_t* inc_v = (const uint16_t*)(rec + R.inc_v);
  const uint16_t* inc_e = (const uint16_t*)(rec + R.inc_e);
  const uint16_t* lv_off = (const uint16_t*)(rec + R.lv_off);
  const uint16_t* le_off = (const uint16_t*)(rec + R.le_off);
  const int32_t* lv_vid = (const int32_t*)(rec + R.lv_vid);
  const int32_t* lv_dst = (const int32_t*)(rec + R.lv_dst);
  const int32_t* le_dst = (const int32_t*)(rec + R.le_dst);
  const uint16_t* lv_str = (const uint16_t*)(rec + R.lv_str);
  const uint16_t* le_str = (const uint16_t*)(rec + R.le_str);
  const int nvv = ne * nv, nee = ne * np;
  // a destination: block base (and row stride) of a value, or -1 - partial index
  auto dst_ok = [&](int32_t dst, int stride) {
    if (dst < 0) return -1 - (int64_t)dst < npart;
    return (int64_t)dst + (int64_t)(m - 1) * stride + (m - 1) < nnz;
  };
  bool bad = false;
  if (threadIdx.x == 0)
    bad = lv_off[0] != 0 || lv_off[nlv] != nvv || le_off[0] != 0 || le_off[nle] != nee;
  for (int u = threadIdx.x; u < nlv; u += blockDim.x) {
    bad |= lv_off[u] >= lv_off[u + 1];
    bad |= lv_vid[u] < 0 || lv_vid[u] >= nq;
    bad |= !dst_ok(lv_dst[u], m > 1 ? lv_str[u] : 0);
  }
  for (int u = threadIdx.x; u < nle; u += blockDim.x) {
    bad |= le_off[u] >= le_off[u + 1];
    const int32_t d0 = le_dst[2 * u], d1 = le_dst[2 * u + 1];
    bad |= !dst_ok(d0, m > 1 ? le_str[2 * u] : 0);
    if (d0 >= 0) bad |= d1 < 0 || !dst_ok(d1, m > 1 ? le_str[2 * u + 1] : 0);
  }
  for (int j = threadIdx.x; j < nee; j += blockDim.x) bad |= (inc_e[j] >> 1) >= nee;
  for (int j = threadIdx.x; j < nvv; j += blockDim.x) bad |= inc_v[j] >= nvv || lvid[j] >= nlv;
  // offsets ascend and end at nvv: the lists are ranges of [0, nvv)
  bad = __syncthreads_or(bad);
  if (!bad) {
    for (int k = threadIdx.x; k < nvv; k += blockDim.x) {  // corner k: once in its vertex's list
      const int u = lvid[k];
      int n = 0;
      for (int j = lv_off[u]; j < lv_off[u + 1]; ++j) n += inc_v[j] == k;
      bad |= n != 1;
    }
  }
  bad = __syncthreads_or(bad);
  if (bad && threadIdx.x == 0) fe_report(st, FE_ERR_BOUNDS, c);
  return !bad;
}

// The same for an interleaved record (plan.cuh IlvLayout): counts at least 1 and
// descending within each group of 32 (so a group's slots fit below the next group's
// first slot), group bases ascending and within max_slots, every corner's local vertex
// below nlv, every slot below the slot count, vertex ids below nq, destinations valid.
static __device__ __noinline__ bool fe_record_valid_ilv(const unsigned char* rec, const IlvLayout& R, int ne,
                                                        int nv, int np, int nlv, int nle, int64_t nq,
                                                        int64_t nnz, int64_t npart, uint32_t max_slots,
                                                        fe_status_word* st, int64_t c) {
  const uint16_t* corner = (const uint16_t*)(rec + R.corner);
  const uint16_t* vpos = (const uint16_t*)(rec + R.vpos);
  const uint16_t* epos = (const uint16_t*)(rec + R.epos);
  const uint16_t* grp = (const uint16_t*)(rec + R.grp);
  const uint16_t* lv_cnt = (const uint16_t*)(rec + R.lv_cnt);
  const uint16_t* le_cnt = (const uint16_t*)(rec + R.le_cnt);
  const int32_t* lv_vid = (const int32_t*)(rec + R.lv_vid);
  const int32_t* lv_dst = (const int32_t*)(rec + R.lv_dst);
  const int32_t* le_dst = (const int32_t*)(rec + R.le_dst);
  const int ngv = (int)ilv_groups(nlv), nge = (int)ilv_groups(nle);
  const uint32_t total = grp[ngv + nge];
  auto dst_ok = [&](int32_t dst) { return dst < 0 ? -1 - (int64_t)dst < npart : (int64_t)dst < nnz; };
  bool bad = total > max_slots;
  for (int g = threadIdx.x; g < ngv + nge; g += blockDim.x) bad |= grp[g] > grp[g + 1];
  // the lists of a group end before the next group starts
  for (int u = threadIdx.x; u < nlv + nle; u += blockDim.x) {
    const bool ed = u >= nlv;
    const int e = ed ? u - nlv : u;
    const int cnt = ed ? le_cnt[e] : lv_cnt[e];
    const int g = (ed ? ngv : 0) + (e >> 5);
    bad |= cnt < 1 || (uint32_t)grp[g] + 32u * (uint32_t)(cnt - 1) + (uint32_t)(e & 31) >= grp[g + 1];
    if (!ed) bad |= lv_vid[e] < 0 || lv_vid[e] >= nq || !dst_ok(lv_dst[e]);
    else {
      const int32_t d0 = le_dst[2 * e], d1 = le_dst[2 * e + 1];
      bad |= !dst_ok(d0) || (d0 >= 0 && !dst_ok(d1)) || (d0 >= 0 && d1 < 0);
    }
  }
  for (int j = threadIdx.x; j < nv * ne; j += blockDim.x) bad |= corner[j] >= nlv || vpos[j] >= total;
  for (int j = threadIdx.x; j < np * ne; j += blockDim.x) bad |= epos[j] >= total;
  bad = __syncthreads_or(bad);
  if (bad && threadIdx.x == 0) fe_report(st, FE_ERR_BOUNDS, c);
  return !bad;
}

// a shared entity's partial range [s, t) and its destination(s) in the fixup kernels
__device__ __forceinline__ bool fe_fixup_valid(int32_t s, int32_t t, int64_t npart, int64_t span0, int64_t span1,
                                               bool two, int64_t nnz, fe_status_word* st, int64_t g) {
  const bool ok = s >= 0 && s < t && t <= npart && span0 >= 0 && span0 < nnz &&
                  (!two || (span1 >= 0 && span1 < nnz));
  if (!ok) fe_report(st, FE_ERR_BOUNDS, g);
  return ok;
}
// the chunk's record and local vertices fit the shared-memory regions sized for them
__device__ __forceinline__ bool fe_chunk_fits(bool ok, fe_status_word* st, int64_t c) {
  if (!ok) fe_report(st, FE_ERR_BOUNDS, c);
  return ok;
}
#define FE_CHUNK_FITS(...) fe_chunk_fits(__VA_ARGS__)
#define FE_RECORD_VALID(...) fe_record_valid(__VA_ARGS__)
#define FE_RECORD_VALID_ILV(...) fe_record_valid_ilv(__VA_ARGS__)
#define FE_FIXUP_VALID(...) fe_fixup_valid(__VA_ARGS__)
#else
#define FE_CHUNK_FITS(...) true
#define FE_RECORD_VALID(...) true
#define FE_RECORD_VALID_ILV(...) true
#define FE_FIXUP_VALID(...) true
#endif

}  // namespace fe
