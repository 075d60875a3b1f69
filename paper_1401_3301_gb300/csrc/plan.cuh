// Layout of the per-chunk plan record: one contiguous, 16-byte aligned block per
// element chunk, copied to shared memory with a single bulk copy by the chunked
// reassembly kernels. Byte offsets within the record:
//   lvid   uint16[nv * ne]     local vertex of corner a of element e_local, at e_local * nv + a
//   inc_v  uint16[nv * ne]     (e_local * nv + a), grouped by local vertex
//   inc_e  uint16[np * ne]     ((e_local * np + p) << 1) | swapped, grouped by local edge
//   lv_off uint16[nlv + 1]     first incidence of each local vertex; lv_off[nlv] = nv * ne
//   le_off uint16[nle + 1]     same for local edges; le_off[nle] = np * ne
//   lv_vid int32[nlv]          global vertex id
//   lv_dst int32[nlv]          diagonal nonzero (>= 0) or -1 - partial index
//   le_dst int32[2 * nle]      nonzeros (i,j), (j,i) with i < j, or -1 - partial index
// Vector problems (m > 1) add the row strides of the m x m blocks, whose entry
// (l, n) is at dst + l * stride + n:
//   lv_str uint16[nlv], le_str uint16[2 * nle]
// Each array starts on a 16-byte boundary.
#pragma once

#include <stdint.h>

namespace fe {

struct RecLayout {
  uint32_t lvid, inc_v, inc_e, lv_off, le_off, lv_vid, lv_dst, le_dst, lv_str, le_str, total;
};

__host__ __device__ __forceinline__ uint32_t pad16(uint32_t x) { return (x + 15u) & ~15u; }

// Dynamic shared memory a chunked kernel may take: the 227 KB a block can opt into, less
// 1 KB for the kernels' static shared variables (barrier, counters, the 128-byte
// alignment of the dynamic array), which count against the same limit.
constexpr uint32_t kSmemDynMax = 227u * 1024u - 1024u;

__host__ __device__ __forceinline__ RecLayout rec_layout(uint32_t ne, uint32_t nv, uint32_t np,
                                                         uint32_t nlv, uint32_t nle,
                                                         bool vector = false) {
  RecLayout L;
  uint32_t o = 0;
  L.lvid = o;   o += pad16(2u * nv * ne);
  L.inc_v = o;  o += pad16(2u * nv * ne);
  L.inc_e = o;  o += pad16(2u * np * ne);
  L.lv_off = o; o += pad16(2u * (nlv + 1));
  L.le_off = o; o += pad16(2u * (nle + 1));
  L.lv_vid = o; o += pad16(4u * nlv);
  L.lv_dst = o; o += pad16(4u * nlv);
  L.le_dst = o; o += pad16(8u * nle);
  L.lv_str = o; o += vector ? pad16(2u * nlv) : 0u;
  L.le_str = o; o += vector ? pad16(4u * nle) : 0u;
  L.total = o;
  return L;
}

// Interleaved layout of a scalar chunk record (FE_PATTERN_INTERLEAVED). The chunk's
// distinct vertices and edges are ordered by descending incidence count and taken in
// groups of 32 (one warp); the j-th incidence of entity u (group g = u / 32, lane
// u % 32) has its value at slot grp[g] + 32 j + lane of the chunk's value array, so a
// warp summing its group's lists reads 32 consecutive slots per step. Vertex groups come
// first, then edge groups. Byte offsets within the record:
//   corner uint16[nv * ne]       local vertex of corner a of element el, at [a * ne + el]
//   vpos   uint16[nv * ne]       slot of that corner's diagonal entry, at [a * ne + el]
//   epos   uint16[np * ne]       slot of local pair p's entry, at [p * ne + el]
//   grp    uint16[ngv + nge + 1] first slot of each group; grp[ngv + nge] = slots used
//   lv_cnt uint16[nlv], le_cnt uint16[nle]   incidences of each vertex / edge
//   lv_vid int32[nlv], lv_dst int32[nlv], le_dst int32[2 * nle]   as in the plain layout
// Each array starts on a 16-byte boundary.
struct IlvLayout {
  uint32_t corner, vpos, epos, grp, lv_cnt, le_cnt, lv_vid, lv_dst, le_dst, total;
};

__host__ __device__ __forceinline__ uint32_t ilv_groups(uint32_t n) { return (n + 31u) / 32u; }

__host__ __device__ __forceinline__ IlvLayout ilv_layout(uint32_t ne, uint32_t nv, uint32_t np, uint32_t nlv,
                                                         uint32_t nle) {
  IlvLayout L;
  uint32_t o = 0;
  L.corner = o; o += pad16(2u * nv * ne);
  L.vpos = o;   o += pad16(2u * nv * ne);
  L.epos = o;   o += pad16(2u * np * ne);
  L.grp = o;    o += pad16(2u * (ilv_groups(nlv) + ilv_groups(nle) + 1u));
  L.lv_cnt = o; o += pad16(2u * nlv);
  L.le_cnt = o; o += pad16(2u * nle);
  L.lv_vid = o; o += pad16(4u * nlv);
  L.lv_dst = o; o += pad16(4u * nlv);
  L.le_dst = o; o += pad16(8u * nle);
  L.total = o;
  return L;
}

// Shared memory of the interleaved chunk kernel: record, staged coordinates, P1
// weights and the value slots (max_slots of them).
struct IlvSmem {
  uint32_t q, w, vals, total;
};
__host__ __device__ __forceinline__ IlvSmem ilv_smem(int D, int sizeT, bool p1_weight, uint32_t rec_max,
                                                     uint32_t max_lv, uint32_t max_slots) {
  IlvSmem L;
  uint32_t o = pad16(rec_max);
  L.q = o;    o += pad16((D == 3 ? 32u : 16u) * max_lv);
  L.w = o;    o += p1_weight ? pad16(sizeT * max_lv) : 0u;
  L.vals = o; o += pad16(sizeT * max_slots);
  L.total = o;
  return L;
}

// Shared-memory layout of the staged chunk kernel (byte offsets).
struct StagedSmem {
  uint32_t q, w, kd, ko, sc, total;
};
__host__ __device__ __forceinline__ StagedSmem staged_smem(int D, int sizeT, bool p1_weight,
                                                           uint32_t rec_max, uint32_t max_lv,
                                                           uint32_t chunk, bool scale = false) {
  const uint32_t nv = D + 1, np = D * (D + 1) / 2;
  StagedSmem L;
  uint32_t o = pad16(rec_max);
  L.q = o;    o += pad16((D == 3 ? 32u : 16u) * max_lv);
  L.w = o;    o += p1_weight ? pad16(sizeT * max_lv) : 0u;
  L.kd = o;   o += pad16(sizeT * nv * chunk);
  L.ko = o;   o += pad16(sizeT * np * chunk);
  L.sc = o;   o += scale ? pad16(sizeT * chunk) : 0u;
  L.total = o;
  return L;
}

struct ElasSmem {
  uint32_t q, coef, cg, lm, total;
};
__host__ __device__ __forceinline__ ElasSmem elas_smem(int D, int sizeT, uint32_t rec_max,
                                                       uint32_t max_lv, uint32_t chunk) {
  const uint32_t nv = D + 1;
  ElasSmem L;
  uint32_t o = pad16(rec_max);
  L.q = o;    o += pad16((D == 3 ? 32u : 16u) * max_lv);
  L.coef = o; o += pad16(2u * sizeT * max_lv);
  L.cg = o;   o += pad16(sizeT * nv * D * chunk);
  L.lm = o;   o += pad16(2u * sizeT * chunk);
  L.total = o;
  return L;
}

// Shared-memory layout of the boundary (facet) kernel: D-dimensional coordinates,
// D vertices and D (D-1)/2 edges per facet.
__host__ __device__ __forceinline__ StagedSmem boundary_smem(int D, int sizeT, bool p1_weight,
                                                             uint32_t rec_max, uint32_t max_lv,
                                                             uint32_t chunk) {
  const uint32_t nv = D, np = D * (D - 1) / 2;
  StagedSmem L;
  uint32_t o = pad16(rec_max);
  L.q = o;    o += pad16((D == 3 ? 32u : 16u) * max_lv);
  L.w = o;    o += p1_weight ? pad16(sizeT * max_lv) : 0u;
  L.kd = o;   o += pad16(sizeT * nv * chunk);
  L.ko = o;   o += pad16(sizeT * np * chunk);
  L.sc = o;
  L.total = o;
  return L;
}

// Shared-memory layout of the general (non-symmetric) operator kernel: one diagonal
// value per corner and two values, one per orientation, per element edge (ko).
__host__ __device__ __forceinline__ StagedSmem general_smem(int D, int sizeT, uint32_t rec_max,
                                                            uint32_t max_lv, uint32_t chunk) {
  const uint32_t nv = D + 1, np = D * (D + 1) / 2;
  StagedSmem L;
  uint32_t o = pad16(rec_max);
  L.q = o;    o += pad16((D == 3 ? 32u : 16u) * max_lv);
  L.w = o;
  L.kd = o;   o += pad16(sizeT * nv * chunk);
  L.ko = o;   o += pad16(2u * sizeT * np * chunk);
  L.sc = o;
  L.total = o;
  return L;
}

// Shared-memory layout of the P_k mass kernel: the |det B| of each element (sc) and the
// constant table (diagonal, then pairs).
struct PkSmem {
  uint32_t sc, tab, total;
};
__host__ __device__ __forceinline__ PkSmem pk_smem(uint32_t nv, uint32_t np, int sizeT, uint32_t rec_max,
                                                   uint32_t chunk) {
  PkSmem L;
  uint32_t o = pad16(rec_max);
  L.sc = o;   o += pad16(sizeT * chunk);
  L.tab = o;  o += pad16(sizeT * (nv + np));
  L.total = o;
  return L;
}

// Largest shared-memory footprint of any chunked kernel for a plan (FP64, with a P1
// coefficient, and the general operator): the plan build shrinks the chunk until it
// fits in one block.
__host__ __device__ __forceinline__ uint32_t plan_smem_worst(int D, int m, uint32_t rec_max,
                                                             uint32_t max_lv, uint32_t chunk) {
  if (m > 1) return elas_smem(D, 8, rec_max, max_lv, chunk).total;
  const uint32_t a = staged_smem(D, 8, true, rec_max, max_lv, chunk).total;
  const uint32_t b = staged_smem(D, 8, false, rec_max, max_lv, chunk, true).total;
  const uint32_t g = general_smem(D, 8, rec_max, max_lv, chunk).total;
  const uint32_t ab = a > b ? a : b;
  return ab > g ? ab : g;
}

}  // namespace fe
