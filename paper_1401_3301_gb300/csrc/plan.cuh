// Layout of the per-chunk plan record: one contiguous, 16-byte aligned block per
// element chunk, copied to shared memory with a single bulk copy by the chunked
// reassembly kernels. Byte offsets within the record:
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
  uint32_t inc_v, inc_e, lv_off, le_off, lv_vid, lv_dst, le_dst, lv_str, le_str, total;
};

__host__ __device__ __forceinline__ uint32_t pad16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ __forceinline__ RecLayout rec_layout(uint32_t ne, uint32_t nv, uint32_t np,
                                                         uint32_t nlv, uint32_t nle,
                                                         bool vector = false) {
  RecLayout L;
  uint32_t o = 0;
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

}  // namespace fe
