// Pattern build (once per mesh topology): the index part of the paper's `sparse`
// constructor (Section 3, Algorithms 2-3 and 9), plus the element-chunk plan used
// by the fused deterministic reassembly.
//
// Steps, all on the device:
//   1. check me against [0, nq);
//   2. internal element order: Morton code of each element centroid, radix-sorted
//      (stable, so equal codes keep input order);
//   3. one 64-bit key row * nq + col per element slot (scalar pattern), radix-sorted
//      with the slot id as value, then run-length encoded into CSR (col_idx,
//      row_ptr), slot2nnz and the slot lists of each nonzero;
//   4. vector problems (m = d): the scalar pattern expanded into m x m blocks in
//      the alternate numbering dof = m v + component;
//   5. element-chunk plan: elements are cut into chunks of C consecutive internal
//      elements; per chunk, the distinct vertices and edges it touches, the
//      (element, corner) and (element, edge) incidences of each, in ascending
//      element order, and where each per-chunk sum goes (the CSR value itself if
//      the chunk holds every element of that vertex or edge, else a partial-sum
//      slot that a second pass adds up in chunk order).
#include <stdio.h>
#include <stdlib.h>

#include <vector>

#include "fe_internal.cuh"
#include "plan.cuh"

namespace {

__host__ __device__ __forceinline__ int bitlen(uint64_t x) {
  int b = 0;
  while (x) { ++b; x >>= 1; }
  return b;
}

__global__ void k_check_me(const int32_t* me, int64_t nme, int nv, int64_t nq, fe_status_word* st) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme;
       k += (int64_t)gridDim.x * blockDim.x) {
    for (int a = 0; a < nv; ++a) {
      const int32_t v = me[(int64_t)a * nme + k];
      if (v < 0 || v >= nq) { fe_report(st, FE_ERR_INDEX, k); break; }
    }
  }
}

// per-block min/max of each coordinate; out[blk * 2d + c] = min, out[blk * 2d + d + c] = max
__global__ void k_bbox_partial(const double* q, int64_t nq, int d, double* out) {
  __shared__ double smin[3][256], smax[3][256];
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nq;
       v += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < d; ++c) {
      const double x = q[(int64_t)c * nq + v];
      lo[c] = fmin(lo[c], x);
      hi[c] = fmax(hi[c], x);
    }
  for (int c = 0; c < d; ++c) { smin[c][threadIdx.x] = lo[c]; smax[c][threadIdx.x] = hi[c]; }
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int c = 0; c < d; ++c) {
        smin[c][threadIdx.x] = fmin(smin[c][threadIdx.x], smin[c][threadIdx.x + s]);
        smax[c][threadIdx.x] = fmax(smax[c][threadIdx.x], smax[c][threadIdx.x + s]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < d; ++c) {
      out[blockIdx.x * 2 * d + c] = smin[c][0];
      out[blockIdx.x * 2 * d + d + c] = smax[c][0];
    }
}

__global__ void k_bbox_final(double* part, int nblk, int d) {
  if (threadIdx.x != 0) return;
  for (int c = 0; c < d; ++c) {
    double lo = part[c], hi = part[d + c];
    for (int b = 1; b < nblk; ++b) {
      lo = fmin(lo, part[b * 2 * d + c]);
      hi = fmax(hi, part[b * 2 * d + d + c]);
    }
    part[c] = lo;
    part[d + c] = hi;
  }
}

__device__ __forceinline__ uint64_t spread_bits(uint64_t x, int d) {
  uint64_t r = 0;
  for (int b = 0; b < 21; ++b) r |= ((x >> b) & 1ull) << (b * d);
  return r;
}

__global__ void k_morton_keys(const double* q, int64_t nq, const int32_t* me, int64_t nme, int d,
                              int nv, const double* bbox, int qbits, const int32_t* group,
                              uint64_t* keys, uint32_t* vals) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nme) return;
  const double scale = (double)(1u << qbits);
  uint64_t code = 0;
  for (int c = 0; c < d; ++c) {
    double s = 0.0;
    for (int a = 0; a < nv; ++a) s += q[(int64_t)c * nq + me[(int64_t)a * nme + k]];
    s /= (double)nv;
    const double lo = bbox[c], hi = bbox[d + c];
    double t = (hi > lo) ? (s - lo) / (hi - lo) : 0.0;
    t = fmin(fmax(t, 0.0), 1.0);
    uint64_t iq = (uint64_t)(t * scale);
    if (iq >= (1ull << qbits)) iq = (1ull << qbits) - 1;
    code |= spread_bits(iq, d) << c;
  }
  if (group) code |= (uint64_t)group[k] << (qbits * d);
  keys[k] = code;
  vals[k] = (uint32_t)k;
}

__global__ void k_iota(uint32_t* v, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) v[i] = (uint32_t)i;
}

__global__ void k_permute_me(const int32_t* me, int64_t nme, int nv, const uint32_t* order,
                             int32_t* me_int, int32_t* order_out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nme) return;
  const int64_t k = order[e];
  for (int a = 0; a < nv; ++a) me_int[(int64_t)a * nme + e] = me[(int64_t)a * nme + k];
  order_out[e] = (int32_t)k;
}

// keys of the scalar slots: slot = e * nv^2 + b * nv + a, (row, col) = (me(a,e), me(b,e))
__global__ void k_slot_keys(const int32_t* me_int, int64_t nme, int nv, int64_t nq, uint64_t* keys,
                            uint32_t* vals) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int S = nv * nv;
  if (s >= nme * S) return;
  const int64_t e = s / S;
  const int loc = (int)(s - e * S);
  const int a = loc % nv, b = loc / nv;
  const uint64_t row = (uint64_t)me_int[(int64_t)a * nme + e];
  const uint64_t col = (uint64_t)me_int[(int64_t)b * nme + e];
  keys[s] = row * (uint64_t)nq + col;
  vals[s] = (uint32_t)s;
}

__global__ void k_key_change(const uint64_t* keys, int64_t n, uint32_t* flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

// flag is overwritten by its exclusive scan in pos; recompute the flag from keys
__global__ void k_rle_scalar(const uint64_t* keys, const uint32_t* vals, const uint32_t* pos,
                             int64_t n, int64_t nq, int32_t* col_idx, int32_t* row_ptr,
                             int32_t* nnz_slot_ptr, int32_t* slot2nnz) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t key = keys[i];
  const bool head = (i == 0) || key != keys[i - 1];
  const uint32_t j = pos[i] + (head ? 1u : 0u) - 1u;
  slot2nnz[vals[i]] = (int32_t)j;
  if (!head) return;
  col_idx[j] = (int32_t)(key % (uint64_t)nq);
  nnz_slot_ptr[j] = (int32_t)i;
  const int64_t r = (int64_t)(key / (uint64_t)nq);
  const int64_t rprev = (i == 0) ? -1 : (int64_t)(keys[i - 1] / (uint64_t)nq);
  for (int64_t rr = rprev + 1; rr <= r; ++rr) row_ptr[rr] = (int32_t)j;
}

__global__ void k_rle_tail(const uint64_t* keys, int64_t n, int64_t nq, int64_t nnz,
                           int32_t* row_ptr, int32_t* nnz_slot_ptr) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int64_t rlast = (n > 0) ? (int64_t)(keys[n - 1] / (uint64_t)nq) : -1;
  for (int64_t rr = rlast + 1; rr <= nq; ++rr) row_ptr[rr] = (int32_t)nnz;
  nnz_slot_ptr[nnz] = (int32_t)n;
}

// m x m block expansion of the scalar CSR (alternate numbering dof = m v + l)
__global__ void k_expand_csr(const int32_t* rp, const int32_t* ci, int64_t nq, int m,
                             int32_t* rp_e, int32_t* ci_e) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nq) return;
  const int32_t r0 = rp[i], len = rp[i + 1] - rp[i];
  for (int l = 0; l < m; ++l) {
    const int64_t base = (int64_t)m * m * r0 + (int64_t)l * m * len;
    rp_e[(int64_t)m * i + l] = (int32_t)base;
    for (int jj = 0; jj < len; ++jj)
      for (int n = 0; n < m; ++n) ci_e[base + (int64_t)m * jj + n] = m * ci[r0 + jj] + n;
  }
  if (i == nq - 1) rp_e[(int64_t)m * nq] = (int32_t)((int64_t)m * m * rp[nq]);
}

__device__ __forceinline__ int32_t find_nnz(const int32_t* rp, const int32_t* ci, int32_t r,
                                            int32_t c) {
  int32_t lo = rp[r], hi = rp[r + 1] - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (ci[mid] < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// vertex incidences: entry i = e * nv + a, key (chunk, vertex), value e_local * nv + a
__global__ void k_vinc_keys(const int32_t* me_int, int64_t nme, int nv, int chunk, int vbits,
                            uint64_t* keys, uint32_t* vals) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nme * nv) return;
  const int64_t e = i / nv;
  const int a = (int)(i - e * nv);
  const uint64_t c = (uint64_t)(e / chunk);
  keys[i] = (c << vbits) | (uint64_t)me_int[(int64_t)a * nme + e];
  vals[i] = (uint32_t)((e % chunk) * nv + a);
}

// edge incidences: entry i = e * npair + p, key (chunk, nonzero of the edge oriented
// (vmin, vmax)) taken from the slot map, value ((e_local * npair + p) << 1) |
// (me(a) > me(b)) for pair p = (a, b), a < b
__global__ void k_einc_keys(const int32_t* me_int, const int32_t* slot2nnz, int64_t nme, int nv,
                            int npair, int chunk, int nbits, uint64_t* keys, uint32_t* vals) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nme * npair) return;
  const int64_t e = i / npair;
  const int p = (int)(i - e * npair);
  int a = 0, b = 1, cnt = 0;
  for (int x = 0; x < nv; ++x)
    for (int y = x + 1; y < nv; ++y) {
      if (cnt == p) { a = x; b = y; }
      ++cnt;
    }
  const int32_t va = me_int[(int64_t)a * nme + e];
  const int32_t vb = me_int[(int64_t)b * nme + e];
  // slot (row a, col b) is e*nv^2 + b*nv + a; take the one whose row is the smaller vertex
  const int64_t slot = va < vb ? e * nv * nv + (int64_t)b * nv + a : e * nv * nv + (int64_t)a * nv + b;
  const uint64_t c = (uint64_t)(e / chunk);
  keys[i] = (c << nbits) | (uint64_t)slot2nnz[slot];
  vals[i] = (uint32_t)((((e % chunk) * npair + p) << 1) | (va > vb ? 1 : 0));
}

// row of nonzero j of a CSR matrix (last row r with rp[r] <= j)
__device__ __forceinline__ int32_t row_of(const int32_t* rp, int64_t nrows, int32_t j) {
  int64_t lo = 0, hi = nrows - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (rp[mid] <= j) lo = mid; else hi = mid - 1;
  }
  return (int32_t)lo;
}

// Local entities from sorted incidence keys. For a head at sorted position i with
// entity index u = pos[i]: offset within the chunk's incidences, chunk start, and the
// global destination(s). Shared entities are flagged for the partial-sum pass.
__global__ void k_local_entities(const uint64_t* keys, const uint32_t* pos, int64_t n, int per_elem,
                                 int chunk, int ebits, int vbits, bool edges, const int32_t* rp,
                                 const int32_t* ci, const int32_t* nnz_slot_ptr, int64_t nq, int m,
                                 uint16_t* off,
                                 int32_t* ch_ptr, int32_t* dst, int32_t* vid, uint16_t* str,
                                 uint32_t* shared_flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t key = keys[i];
  if (i > 0 && keys[i - 1] == key) return;
  const uint32_t u = pos[i];
  const uint64_t c = key >> ebits;
  int64_t end = i + 1;
  while (end < n && keys[end] == key) ++end;
  const int32_t local_count = (int32_t)(end - i);
  off[u] = (uint16_t)(i - (int64_t)c * chunk * per_elem);
  if (i == 0 || (keys[i - 1] >> ebits) != c) ch_ptr[c] = (int32_t)u;
  const uint64_t vmask = (1ull << vbits) - 1ull;
  int32_t global_count;
  if (!edges) {
    const int32_t v = (int32_t)(key & vmask);
    const int32_t dnz = find_nnz(rp, ci, v, v);
    dst[u] = dnz;
    vid[u] = v;
    global_count = nnz_slot_ptr[dnz + 1] - nnz_slot_ptr[dnz];
    if (m > 1) {  // m x m block: entry (l, n) at dst + l * str + n
      dst[u] = m * m * rp[v] + m * (dnz - rp[v]);
      str[u] = (uint16_t)(m * (rp[v + 1] - rp[v]));
    }
  } else {
    const int32_t nij = (int32_t)(key & ((1ull << ebits) - 1ull));
    const int32_t lo = row_of(rp, nq, nij), hi = ci[nij];
    const int32_t nji = find_nnz(rp, ci, hi, lo);
    dst[2 * (int64_t)u] = nij;
    dst[2 * (int64_t)u + 1] = nji;
    global_count = nnz_slot_ptr[nij + 1] - nnz_slot_ptr[nij];
    if (m > 1) {
      dst[2 * (int64_t)u] = m * m * rp[lo] + m * (nij - rp[lo]);
      dst[2 * (int64_t)u + 1] = m * m * rp[hi] + m * (nji - rp[hi]);
      str[2 * (int64_t)u] = (uint16_t)(m * (rp[lo + 1] - rp[lo]));
      str[2 * (int64_t)u + 1] = (uint16_t)(m * (rp[hi + 1] - rp[hi]));
    }
  }
  shared_flag[u] = (local_count < global_count) ? 1u : 0u;
}

__global__ void k_to_u16(const uint32_t* v, uint16_t* o, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) o[i] = (uint16_t)v[i];
}

__global__ void k_entity_change(const uint64_t* k, int64_t n, int cb, uint32_t* f) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) f[i] = (i == 0 || (k[i] >> cb) != (k[i - 1] >> cb)) ? 1u : 0u;
}

__global__ void k_set_last(int32_t* p, int64_t idx, int32_t value) {
  if (blockIdx.x == 0 && threadIdx.x == 0) p[idx] = value;
}

// keys (global entity nnz, chunk) of the shared local entities, compacted with spos
__global__ void k_shared_keys(const uint32_t* shared_flag, const uint32_t* spos, int64_t nloc,
                              const int32_t* dst, int dst_stride, const int32_t* ch_ptr,
                              int64_t nchunks, int cbits, uint64_t* keys, uint32_t* vals) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= nloc || !shared_flag[u]) return;
  // chunk of local entity u: last c with ch_ptr[c] <= u
  int64_t lo = 0, hi = nchunks - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (ch_ptr[mid] <= u) lo = mid; else hi = mid - 1;
  }
  const uint32_t s = spos[u];
  keys[s] = ((uint64_t)dst[(int64_t)u * dst_stride] << cbits) | (uint64_t)lo;
  vals[s] = (uint32_t)u;
}

// after sorting shared keys: partial index of each shared local entity and the
// fixup lists (ranges of partials per global entity, destinations)
__global__ void k_shared_finish(const uint64_t* keys, const uint32_t* vals, const uint32_t* gpos,
                                int64_t n, int cbits, int64_t part_base, int64_t ent_base,
                                int32_t* dst, int dst_stride, const int32_t* vid, bool edges,
                                int32_t* sh_ptr, int32_t* sh_dst, const uint16_t* str,
                                int32_t* sh_str) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t u = vals[i];
  const uint64_t ent = keys[i] >> cbits;
  const bool head = (i == 0) || (keys[i - 1] >> cbits) != ent;
  if (head) {
    const int64_t g = ent_base + gpos[i];
    sh_ptr[g] = (int32_t)(part_base + i);
    if (!edges) {
      sh_dst[2 * g] = dst[(int64_t)u * dst_stride];
      sh_dst[2 * g + 1] = vid[u];
      if (sh_str) sh_str[2 * g] = str[u];
    } else {
      sh_dst[2 * g] = dst[(int64_t)u * dst_stride];
      sh_dst[2 * g + 1] = dst[(int64_t)u * dst_stride + 1];
      if (sh_str) {
        sh_str[2 * g] = str[2 * (int64_t)u];
        sh_str[2 * g + 1] = str[2 * (int64_t)u + 1];
      }
    }
  }
  dst[(int64_t)u * dst_stride] = -1 - (int32_t)(part_base + i);
}

__global__ void k_rec_sizes(int64_t nme, int chunk, int nv, int np, int m, int64_t nchunks,
                            const int32_t* ch_v_ptr, const int32_t* ch_e_ptr, bool interleaved,
                            uint32_t* size16) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nchunks) return;
  const int64_t ne = min((int64_t)chunk, nme - c * chunk);
  const uint32_t nlv = ch_v_ptr[c + 1] - ch_v_ptr[c], nle = ch_e_ptr[c + 1] - ch_e_ptr[c];
  size16[c] = (interleaved ? fe::ilv_layout((uint32_t)ne, nv, np, nlv, nle).total
                           : fe::rec_layout((uint32_t)ne, nv, np, nlv, nle, m > 1).total) / 16u;
}

// Block-wide exclusive scan of one value per thread (blockDim.x a multiple of 32);
// *total receives the block sum. ws: 32 words of shared scratch.
__device__ uint32_t block_exscan(uint32_t v, uint32_t* ws, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < nw ? ws[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) ws[lane] = t;
  }
  __syncthreads();
  const uint32_t base = w ? ws[w - 1] : 0u;
  *total = ws[nw - 1];
  __syncthreads();
  return base + x - v;
}

// Order the n local entities of a chunk by descending incidence count, ties in their
// original order (a stable bucket pass per count value): perm[new] = old, and
// noff[new] = the entity's first incidence in the new layout. cnt holds the counts.
__device__ void order_by_count(const uint16_t* cnt, int32_t n, uint16_t* perm, uint16_t* noff, uint32_t* ws) {
  __shared__ uint32_t mx;
  if (threadIdx.x == 0) mx = 0;
  __syncthreads();
  uint32_t m = 0;
  for (int32_t u = threadIdx.x; u < n; u += blockDim.x) m = max(m, (uint32_t)cnt[u]);
  atomicMax(&mx, m);
  __syncthreads();
  const int top = (int)mx;
  uint32_t base = 0;
  for (int c = top; c >= 1; --c)
    for (int32_t t0 = 0; t0 < n; t0 += blockDim.x) {
      const int32_t u = t0 + threadIdx.x;
      const uint32_t f = (u < n && cnt[u] == c) ? 1u : 0u;
      uint32_t tot;
      const uint32_t r = block_exscan(f, ws, &tot);
      if (f) perm[base + r] = (uint16_t)u;
      base += tot;
    }
  __syncthreads();
  uint32_t carry = 0;
  for (int32_t t0 = 0; t0 < n; t0 += blockDim.x) {
    const int32_t u = t0 + threadIdx.x;
    const uint32_t v = u < n ? cnt[perm[u]] : 0u;
    uint32_t tot;
    const uint32_t r = block_exscan(v, ws, &tot);
    if (u < n) noff[u] = (uint16_t)(carry + r);
    carry += tot;
  }
  __syncthreads();
}

// One block per chunk: copy the chunk's slices of the plan arrays into its record. With
// `ordered`, the chunk's local vertices and edges are laid out by descending incidence
// count (so that the threads of a warp, which take consecutive entities, loop over
// similar counts); each entity's incidence list is copied unchanged, so its sum keeps
// ascending element order. Dynamic shared memory: 6 bytes per entity of the largest
// list when ordered.
__global__ void k_rec_fill(int64_t nme, int chunk, int nv, int np, int m, bool ordered,
                           const int32_t* ch_v_ptr, const int32_t* ch_e_ptr, const uint16_t* inc_v,
                           const uint16_t* inc_e, const uint16_t* lv_off, const uint16_t* le_off,
                           const int32_t* lv_vid, const int32_t* lv_dst, const int32_t* le_dst,
                           const uint16_t* lv_str, const uint16_t* le_str, const uint32_t* off16,
                           uint8_t* rec) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ uint32_t ws[32];
  const int64_t c = blockIdx.x;
  const int64_t ne = min((int64_t)chunk, nme - c * chunk);
  const int32_t vb = ch_v_ptr[c], nlv = ch_v_ptr[c + 1] - vb;
  const int32_t eb = ch_e_ptr[c], nle = ch_e_ptr[c + 1] - eb;
  const fe::RecLayout L = fe::rec_layout((uint32_t)ne, nv, np, nlv, nle, m > 1);
  uint8_t* r = rec + (int64_t)off16[c] * 16;
  uint16_t* r_lvid = (uint16_t*)(r + L.lvid);
  uint16_t* r_inc_v = (uint16_t*)(r + L.inc_v);
  uint16_t* r_inc_e = (uint16_t*)(r + L.inc_e);
  uint16_t* r_lv_off = (uint16_t*)(r + L.lv_off);
  uint16_t* r_le_off = (uint16_t*)(r + L.le_off);
  int32_t* r_lv_vid = (int32_t*)(r + L.lv_vid);
  int32_t* r_lv_dst = (int32_t*)(r + L.lv_dst);
  int32_t* r_le_dst = (int32_t*)(r + L.le_dst);
  uint16_t* r_lv_str = (uint16_t*)(r + L.lv_str);
  uint16_t* r_le_str = (uint16_t*)(r + L.le_str);
  const int64_t ibv = c * (int64_t)chunk * nv, ibe = c * (int64_t)chunk * np;
  for (int pass = 0; pass < 2; ++pass) {
    const bool edges = pass == 1;
    const int32_t n = edges ? nle : nlv, b0 = edges ? eb : vb;
    const uint16_t* off = edges ? le_off : lv_off;
    const uint16_t* inc = (edges ? inc_e : inc_v) + (edges ? ibe : ibv);
    uint16_t* r_inc = edges ? r_inc_e : r_inc_v;
    uint16_t* r_off = edges ? r_le_off : r_lv_off;
    const uint32_t end = (uint32_t)(ne * (edges ? np : nv));
    uint16_t* cnt = (uint16_t*)sm;
    uint16_t* perm = cnt + n;
    uint16_t* noff = perm + n;
    if (ordered) {
      for (int32_t u = threadIdx.x; u < n; u += blockDim.x)
        cnt[u] = (uint16_t)((u + 1 < n ? off[b0 + u + 1] : end) - off[b0 + u]);
      __syncthreads();
      order_by_count(cnt, n, perm, noff, ws);
    }
    for (int32_t nu = threadIdx.x; nu < n; nu += blockDim.x) {
      const int32_t u = ordered ? perm[nu] : nu;
      const uint32_t o = off[b0 + u];
      const uint32_t no = ordered ? noff[nu] : o;
      const uint32_t k = (u + 1 < n ? off[b0 + u + 1] : end) - o;
      for (uint32_t j = 0; j < k; ++j) {
        r_inc[no + j] = inc[o + j];
        if (!edges) r_lvid[inc[o + j]] = (uint16_t)nu;  // corner -> its local vertex
      }
      r_off[nu] = (uint16_t)no;
      if (!edges) {
        r_lv_vid[nu] = lv_vid[vb + u];
        r_lv_dst[nu] = lv_dst[vb + u];
        if (m > 1) r_lv_str[nu] = lv_str[vb + u];
      } else {
        r_le_dst[2 * nu] = le_dst[2 * (int64_t)(eb + u)];
        r_le_dst[2 * nu + 1] = le_dst[2 * (int64_t)(eb + u) + 1];
        if (m > 1) {
          r_le_str[2 * nu] = le_str[2 * (int64_t)(eb + u)];
          r_le_str[2 * nu + 1] = le_str[2 * (int64_t)(eb + u) + 1];
        }
      }
    }
    if (threadIdx.x == 0) r_off[n] = (uint16_t)end;
    __syncthreads();
  }
}

// One block per chunk: the interleaved record of a scalar plan (plan.cuh, IlvLayout).
// The chunk's vertices (then edges) are ordered by descending incidence count and cut
// into groups of 32; group g's slots start at the sum of 32 x (largest count) over the
// groups before it, and the j-th incidence of the entity in lane l of group g gets slot
// base_g + 32 j + l. Each element then learns, per corner and per local pair, the slot of
// its value (vpos, epos) and, per corner, its local vertex (corner). Incidence lists keep
// ascending element order, so each sum keeps the order of the plain layout. slots[c]
// receives the chunk's slot count; a count above 65535 (uint16 slots) sets *overflow.
// Dynamic shared memory: 6 bytes per entity of the larger list, plus one word per group.
__global__ void k_rec_fill_ilv(int64_t nme, int chunk, int nv, int np, const int32_t* ch_v_ptr,
                               const int32_t* ch_e_ptr, const uint16_t* inc_v, const uint16_t* inc_e,
                               const uint16_t* lv_off, const uint16_t* le_off, const int32_t* lv_vid,
                               const int32_t* lv_dst, const int32_t* le_dst, const uint32_t* off16,
                               uint8_t* rec, uint32_t* slots, uint32_t* overflow) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ uint32_t ws[32];
  __shared__ uint32_t base_all;
  const int64_t c = blockIdx.x;
  const int64_t ne = min((int64_t)chunk, nme - c * chunk);
  const int32_t vb = ch_v_ptr[c], nlv = ch_v_ptr[c + 1] - vb;
  const int32_t eb = ch_e_ptr[c], nle = ch_e_ptr[c + 1] - eb;
  const fe::IlvLayout L = fe::ilv_layout((uint32_t)ne, nv, np, nlv, nle);
  uint8_t* r = rec + (int64_t)off16[c] * 16;
  uint16_t* r_corner = (uint16_t*)(r + L.corner);
  uint16_t* r_vpos = (uint16_t*)(r + L.vpos);
  uint16_t* r_epos = (uint16_t*)(r + L.epos);
  uint16_t* r_grp = (uint16_t*)(r + L.grp);
  int32_t* r_lv_vid = (int32_t*)(r + L.lv_vid);
  int32_t* r_lv_dst = (int32_t*)(r + L.lv_dst);
  int32_t* r_le_dst = (int32_t*)(r + L.le_dst);
  const int64_t ibv = c * (int64_t)chunk * nv, ibe = c * (int64_t)chunk * np;
  const int ngv = (int)fe::ilv_groups(nlv);
  if (threadIdx.x == 0) base_all = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const bool edges = pass == 1;
    const int32_t n = edges ? nle : nlv, b0 = edges ? eb : vb;
    const uint16_t* off = edges ? le_off : lv_off;
    const uint16_t* inc = (edges ? inc_e : inc_v) + (edges ? ibe : ibv);
    const uint32_t end = (uint32_t)(ne * (edges ? np : nv));
    uint16_t* cnt = (uint16_t*)sm;
    uint16_t* perm = cnt + n;
    uint16_t* noff = perm + n;
    uint32_t* gbase = (uint32_t*)(sm + 16 * ((6 * (size_t)n + 15) / 16));
    uint16_t* r_cnt = (uint16_t*)(r + (edges ? L.le_cnt : L.lv_cnt));
    for (int32_t u = threadIdx.x; u < n; u += blockDim.x)
      cnt[u] = (uint16_t)((u + 1 < n ? off[b0 + u + 1] : end) - off[b0 + u]);
    __syncthreads();
    order_by_count(cnt, n, perm, noff, ws);
    const int ng = (int)fe::ilv_groups(n);
    if (threadIdx.x == 0) {  // group bases: the first entity of a group has its largest count
      uint32_t b = base_all;
      for (int g = 0; g < ng; ++g) {
        gbase[g] = b;
        r_grp[(edges ? ngv : 0) + g] = (uint16_t)b;
        b += 32u * cnt[perm[32 * g]];
      }
      if (b > 65535u) atomicExch(overflow, 1u);
      base_all = b;
      if (edges) {
        r_grp[ngv + ng] = (uint16_t)b;
        slots[c] = b;
      }
    }
    __syncthreads();
    for (int32_t nu = threadIdx.x; nu < n; nu += blockDim.x) {
      const int32_t u = perm[nu];
      const uint32_t o = off[b0 + u], k = cnt[u];
      const uint32_t first = gbase[nu >> 5] + (uint32_t)(nu & 31);
      for (uint32_t j = 0; j < k; ++j) {
        const uint32_t slot = first + 32u * j;
        const uint32_t code = inc[o + j];
        if (!edges) {
          const uint32_t el = code / nv, a = code - el * nv;
          r_vpos[a * ne + el] = (uint16_t)slot;
          r_corner[a * ne + el] = (uint16_t)nu;
        } else {
          const uint32_t x = code >> 1, el = x / np, pp = x - el * np;
          r_epos[pp * ne + el] = (uint16_t)slot;
        }
      }
      r_cnt[nu] = (uint16_t)k;
      if (!edges) {
        r_lv_vid[nu] = lv_vid[vb + u];
        r_lv_dst[nu] = lv_dst[vb + u];
      } else {
        r_le_dst[2 * nu] = le_dst[2 * (int64_t)(eb + u)];
        r_le_dst[2 * nu + 1] = le_dst[2 * (int64_t)(eb + u) + 1];
      }
    }
    __syncthreads();
  }
}

struct dev_tmp {
  std::vector<void*> ptrs;
  ~dev_tmp() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  int get(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, (count > 0 ? count : 1) * sizeof(T));
    if (e != cudaSuccess) return fe_cuda_fail(e);
    ptrs.push_back(q);
    *p = (T*)q;
    return FE_OK;
  }
};

template <class T>
int to_host(T* dst, const T* src, cudaStream_t s) {
  FE_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(T), cudaMemcpyDeviceToHost, s));
  FE_CUDA_TRY(cudaStreamSynchronize(s));
  return FE_OK;
}

int default_chunk(int d, int m, int flags) {
  const int fc = (flags >> 8) & 0xFFFF;
  if (fc >= 32 && fc <= 4096) return fc;
  const char* env = getenv("FE_CHUNK");
  if (env) {
    const int c = atoi(env);
    if (c >= 32 && c <= 4096) return c;
  }
  return d == 3 ? 512 : 1024;  // scalar and vector problems alike
}

// Builds the element-chunk plan. sort buffers sized for max(nv, npair) * nme keys.
int build_chunk_plan(fe_pattern_s* h, fe_sort_buffers* sb, dev_tmp& tmp, cudaStream_t s) {
  const int nv = h->nv, npair = h->npair, C = h->chunk;
  const int64_t nme = h->nme;
  h->nchunks = (nme + C - 1) / C;
  const int cbits = bitlen((uint64_t)(h->nchunks > 1 ? h->nchunks - 1 : 1));
  const int vbits = bitlen((uint64_t)(h->nq > 1 ? h->nq - 1 : 1));
  const int nbits = bitlen((uint64_t)(h->nnz_s > 1 ? h->nnz_s - 1 : 1));
  const int T = 256;
  uint32_t *flag, *pos;
  const int64_t nmax = nme * (nv > npair ? nv : npair);
  FE_TRY(tmp.get(&flag, nmax + 1));
  FE_TRY(tmp.get(&pos, nmax + 1));
  uint32_t* sflag_v; uint32_t* sflag_e;
  uint64_t* keys; uint32_t* vals;
  int64_t nlv = 0, nle = 0;

  for (int pass = 0; pass < 2; ++pass) {
    const bool edges = pass == 1;
    const int per = edges ? npair : nv;
    const int64_t n = nme * per;
    if (!edges)
      k_vinc_keys<<<fe_grid(n, T), T, 0, s>>>(h->me_int, nme, nv, C, vbits, sb->k0, sb->v0);
    else
      k_einc_keys<<<fe_grid(n, T), T, 0, s>>>(h->me_int, h->slot2nnz, nme, nv, npair, C, nbits, sb->k0,
                                              sb->v0);
    FE_CUDA_TRY(cudaGetLastError());
    const int ebits = edges ? nbits : vbits;
    if (ebits + cbits > 64) return FE_ERR_OVERFLOW;
    FE_TRY(fe_radix_sort(n, ebits + cbits, sb, &keys, &vals, s));
    k_key_change<<<fe_grid(n, T), T, 0, s>>>(keys, n, flag);
    FE_CUDA_TRY(cudaGetLastError());
    FE_TRY(fe_scan_exclusive(flag, pos, n, sb->scan_tmp, s));
    uint32_t last_pos = 0, last_flag = 0;
    FE_TRY(to_host(&last_pos, pos + n - 1, s));
    FE_TRY(to_host(&last_flag, flag + n - 1, s));
    const int64_t nloc = (int64_t)last_pos + last_flag;
    uint16_t* inc; uint16_t* off; int32_t* ch_ptr; int32_t* dst; int32_t* vid = nullptr;
    uint16_t* str = nullptr;
    uint32_t* sflag;
    if (h->m > 1) FE_TRY(fe_malloc(h, (void**)&str, sizeof(uint16_t) * nloc * (edges ? 2 : 1)));
    FE_TRY(fe_malloc(h, (void**)&inc, sizeof(uint16_t) * n));
    FE_TRY(fe_malloc(h, (void**)&off, sizeof(uint16_t) * nloc));
    FE_TRY(fe_malloc(h, (void**)&ch_ptr, sizeof(int32_t) * (h->nchunks + 1)));
    FE_TRY(fe_malloc(h, (void**)&dst, sizeof(int32_t) * nloc * (edges ? 2 : 1)));
    if (!edges) FE_TRY(fe_malloc(h, (void**)&vid, sizeof(int32_t) * nloc));
    FE_TRY(tmp.get(&sflag, nloc + 1));
    // inc = sorted values as uint16 (they are < C * per <= 65536)
    k_to_u16<<<fe_grid(n, T), T, 0, s>>>(vals, inc, n);
    FE_CUDA_TRY(cudaGetLastError());
    k_local_entities<<<fe_grid(n, T), T, 0, s>>>(keys, pos, n, per, C, ebits, vbits, edges,
                                                  h->row_ptr_s, h->col_idx_s, h->nnz_slot_ptr, h->nq,
                                                  h->m, off, ch_ptr, dst, vid, str, sflag);
    FE_CUDA_TRY(cudaGetLastError());
    k_set_last<<<1, 1, 0, s>>>(ch_ptr, h->nchunks, (int32_t)nloc);
    FE_CUDA_TRY(cudaGetLastError());
    if (!edges) {
      h->inc_v = inc; h->lv_off = off; h->ch_v_ptr = ch_ptr; h->lv_dst = dst; h->lv_vid = vid;
      h->lv_str = str;
      sflag_v = sflag; nlv = nloc;
    } else {
      h->inc_e = inc; h->le_off = off; h->ch_e_ptr = ch_ptr; h->le_dst = dst;
      h->le_str = str;
      sflag_e = sflag; nle = nloc;
    }
  }
  h->nlv = nlv;
  h->nle = nle;

  // shared entities: compact, sort by (global entity, chunk), assign partial slots
  int64_t nsh_ent[2] = {0, 0}, npart[2] = {0, 0};
  uint32_t* spos[2];
  for (int pass = 0; pass < 2; ++pass) {
    const bool edges = pass == 1;
    const int64_t nloc = edges ? nle : nlv;
    uint32_t* sflag = edges ? sflag_e : sflag_v;
    FE_TRY(tmp.get(&spos[pass], nloc + 1));
    FE_TRY(fe_scan_exclusive(sflag, spos[pass], nloc, sb->scan_tmp, s));
    uint32_t lp = 0, lf = 0;
    FE_TRY(to_host(&lp, spos[pass] + nloc - 1, s));
    FE_TRY(to_host(&lf, sflag + nloc - 1, s));
    npart[pass] = (int64_t)lp + lf;
  }
  // count distinct shared global entities per kind after sorting; allocate fixup arrays
  // with an upper bound (npart) and trim counts later
  FE_TRY(fe_malloc(h, (void**)&h->sh_ptr, sizeof(int32_t) * (npart[0] + npart[1] + 1)));
  FE_TRY(fe_malloc(h, (void**)&h->sh_dst, sizeof(int32_t) * 2 * (npart[0] + npart[1] + 1)));
  if (h->m > 1)
    FE_TRY(fe_malloc(h, (void**)&h->sh_str, sizeof(int32_t) * 2 * (npart[0] + npart[1] + 1)));
  int64_t ent_base = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const bool edges = pass == 1;
    const int64_t nloc = edges ? nle : nlv;
    const int64_t np = npart[pass];
    if (np == 0) continue;
    int32_t* dst = edges ? h->le_dst : h->lv_dst;
    const int stride = edges ? 2 : 1;
    const int32_t* ch_ptr = edges ? h->ch_e_ptr : h->ch_v_ptr;
    k_shared_keys<<<fe_grid(nloc, T), T, 0, s>>>(edges ? sflag_e : sflag_v, spos[pass], nloc, dst,
                                                 stride, ch_ptr, h->nchunks, cbits, sb->k0, sb->v0);
    FE_CUDA_TRY(cudaGetLastError());
    const int kbits = bitlen((uint64_t)(h->nnz > 1 ? h->nnz - 1 : 1)) + cbits;
    FE_TRY(fe_radix_sort(np, kbits, sb, &keys, &vals, s));
    // distinct entities
    k_entity_change<<<fe_grid(np, T), T, 0, s>>>(keys, np, cbits, flag);
    FE_CUDA_TRY(cudaGetLastError());
    FE_TRY(fe_scan_exclusive(flag, pos, np, sb->scan_tmp, s));
    uint32_t lp = 0, lf = 0;
    FE_TRY(to_host(&lp, pos + np - 1, s));
    FE_TRY(to_host(&lf, flag + np - 1, s));
    nsh_ent[pass] = (int64_t)lp + lf;
    const int64_t part_base = edges ? npart[0] : 0;
    k_shared_finish<<<fe_grid(np, T), T, 0, s>>>(keys, vals, pos, np, cbits, part_base, ent_base,
                                                  dst, stride, h->lv_vid, edges, h->sh_ptr,
                                                  h->sh_dst, edges ? h->le_str : h->lv_str, h->sh_str);
    FE_CUDA_TRY(cudaGetLastError());
    ent_base += nsh_ent[pass];
  }
  h->nsh_v = nsh_ent[0];
  h->nsh_e = nsh_ent[1];
  h->npart_v = npart[0];
  h->npart = npart[0] + npart[1];
  k_set_last<<<1, 1, 0, s>>>(h->sh_ptr, h->nsh_v + h->nsh_e, (int32_t)(npart[0] + npart[1]));
  FE_CUDA_TRY(cudaGetLastError());
  // per-chunk records (contiguous copies of each chunk's slice of the plan)
  {
    uint32_t* size16;
    FE_TRY(tmp.get(&size16, h->nchunks + 1));
    const bool ilv = (h->flags & FE_PATTERN_INTERLEAVED) != 0;
    k_rec_sizes<<<fe_grid(h->nchunks, T), T, 0, s>>>(nme, C, nv, npair, h->m, h->nchunks,
                                                     h->ch_v_ptr, h->ch_e_ptr, ilv, size16);
    FE_CUDA_TRY(cudaGetLastError());
    std::vector<uint32_t> sz(h->nchunks);
    FE_CUDA_TRY(cudaMemcpyAsync(sz.data(), size16, sizeof(uint32_t) * h->nchunks,
                                cudaMemcpyDeviceToHost, s));
    FE_CUDA_TRY(cudaStreamSynchronize(s));
    uint64_t total16 = 0;
    uint32_t max16 = 0;
    for (uint32_t v : sz) {
      total16 += v;
      if (v > max16) max16 = v;
    }
    if (total16 > 0xFFFFFFFFull) return FE_ERR_OVERFLOW;
    FE_TRY(fe_malloc(h, (void**)&h->rec_off16, sizeof(uint32_t) * (h->nchunks + 1)));
    FE_TRY(fe_scan_exclusive(size16, h->rec_off16, h->nchunks, sb->scan_tmp, s));
    FE_TRY(fe_malloc(h, (void**)&h->rec, (size_t)total16 * 16));
    h->rec_bytes = (int64_t)total16 * 16;
    h->plan_bytes = h->rec_bytes + (int64_t)sizeof(int32_t) * 2 * (h->nchunks + 1);
    h->rec_max_bytes = (int64_t)max16 * 16;
    // largest local vertex / edge lists of a chunk (shared memory of the kernels)
    std::vector<int32_t> vp(h->nchunks + 1), ep(h->nchunks + 1);
    FE_CUDA_TRY(cudaMemcpyAsync(vp.data(), h->ch_v_ptr, sizeof(int32_t) * (h->nchunks + 1),
                                cudaMemcpyDeviceToHost, s));
    FE_CUDA_TRY(cudaMemcpyAsync(ep.data(), h->ch_e_ptr, sizeof(int32_t) * (h->nchunks + 1),
                                cudaMemcpyDeviceToHost, s));
    FE_CUDA_TRY(cudaStreamSynchronize(s));
    int32_t mlv = 0, mle = 0;
    for (int64_t c = 0; c < h->nchunks; ++c) {
      mlv = vp[c + 1] - vp[c] > mlv ? vp[c + 1] - vp[c] : mlv;
      mle = ep[c + 1] - ep[c] > mle ? ep[c + 1] - ep[c] : mle;
    }
    h->max_lv = mlv;
    const size_t fill_smem = 6u * (size_t)(mlv > mle ? mlv : mle) + 16u;
    if (ilv) {
      // interleaved records: entities always count-ordered, plus one word per group
      const size_t ilv_smem = 16u * ((fill_smem + 15u) / 16u) + 4u * fe::ilv_groups(mlv > mle ? mlv : mle);
      if (ilv_smem > fe::kSmemDynMax) return FE_ERR_OVERFLOW;
      uint32_t *slots, *ovf;
      FE_TRY(tmp.get(&slots, h->nchunks + 1));
      FE_TRY(tmp.get(&ovf, 1));
      FE_CUDA_TRY(cudaMemsetAsync(ovf, 0, sizeof(uint32_t), s));
      FE_TRY(fe_smem_limit(k_rec_fill_ilv, ilv_smem));
      k_rec_fill_ilv<<<(unsigned)h->nchunks, 256, ilv_smem, s>>>(
          nme, C, nv, npair, h->ch_v_ptr, h->ch_e_ptr, h->inc_v, h->inc_e, h->lv_off, h->le_off, h->lv_vid,
          h->lv_dst, h->le_dst, h->rec_off16, h->rec, slots, ovf);
      FE_CUDA_TRY(cudaGetLastError());
      std::vector<uint32_t> sl(h->nchunks);
      uint32_t overflow = 0;
      FE_CUDA_TRY(cudaMemcpyAsync(sl.data(), slots, sizeof(uint32_t) * h->nchunks, cudaMemcpyDeviceToHost, s));
      FE_CUDA_TRY(cudaMemcpyAsync(&overflow, ovf, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
      FE_CUDA_TRY(cudaStreamSynchronize(s));
      uint32_t ms = 0;
      for (uint32_t v : sl) ms = v > ms ? v : ms;
      // more than 65535 slots in a chunk (uint16 slot numbers): the records are unusable,
      // and the shared-memory check of the caller shrinks the chunk and rebuilds
      h->max_slots = overflow ? (1 << 20) : (int32_t)ms;
    } else {
      const bool ordered = fill_smem <= fe::kSmemDynMax && !(h->flags & FE_PATTERN_ENTITY_ORDER);
      if (ordered) FE_TRY(fe_smem_limit(k_rec_fill, fill_smem));
      k_rec_fill<<<(unsigned)h->nchunks, 256, ordered ? fill_smem : 0, s>>>(
          nme, C, nv, npair, h->m, ordered, h->ch_v_ptr, h->ch_e_ptr, h->inc_v, h->inc_e, h->lv_off,
          h->le_off, h->lv_vid, h->lv_dst, h->le_dst, h->lv_str, h->le_str, h->rec_off16, h->rec);
      FE_CUDA_TRY(cudaGetLastError());
      FE_CUDA_TRY(cudaStreamSynchronize(s));
    }
    // the records hold everything the kernels read: release the plan's flat arrays
    h->bytes -= (int64_t)sizeof(uint16_t) * nme * (nv + npair) + (int64_t)(2 + 4 + 4) * h->nlv +
                (int64_t)(2 + 8) * h->nle + (h->m > 1 ? (int64_t)2 * h->nlv + (int64_t)4 * h->nle : 0);
    uint16_t** u16[] = {&h->inc_v, &h->inc_e, &h->lv_off, &h->le_off, &h->lv_str, &h->le_str};
    for (uint16_t** p : u16) {
      if (*p) cudaFree(*p);
      *p = nullptr;
    }
    int32_t** i32[] = {&h->lv_vid, &h->lv_dst, &h->le_dst};
    for (int32_t** p : i32) {
      if (*p) cudaFree(*p);
      *p = nullptr;
    }
  }
  // partial-sum scratch of 8-byte values: 2 per partial for scalar problems (the
  // general operator keeps one per edge orientation), m * m for the vector blocks
  const int vals_per_partial = (h->m == 1) ? 2 : h->m * h->m;
  const size_t pb = (size_t)(npart[0] + npart[1]) * vals_per_partial * 2 * sizeof(float) + 16;
  FE_TRY(fe_malloc(h, &h->partials, pb));
  h->partials_bytes = pb;
  return FE_OK;
}

__global__ void k_vmap_keys(const int32_t* me_int, int64_t nme, int nv, uint64_t* keys, uint32_t* vals) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nme * nv) return;
  const int64_t e = i / nv;
  const int a = (int)(i - e * nv);
  keys[i] = (uint64_t)me_int[(int64_t)a * nme + e];
  vals[i] = (uint32_t)i;  // e * nv + a
}

__global__ void k_vmap_ptr(const uint64_t* keys, int64_t n, int64_t nq, int32_t* ptr) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t v = (int64_t)keys[i];
  const int64_t vprev = (i == 0) ? -1 : (int64_t)keys[i - 1];
  for (int64_t r = vprev + 1; r <= v; ++r) ptr[r] = (int32_t)i;
  if (i == n - 1)
    for (int64_t r = v + 1; r <= nq; ++r) ptr[r] = (int32_t)n;
}

}  // namespace

namespace {
__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__global__ void k_union_me(const int32_t* me, int64_t nme, int nv, int64_t voff, int64_t eoff,
                           int64_t nme_total, int32_t* me_u) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nme) return;
  for (int a = 0; a < nv; ++a)
    me_u[(int64_t)a * nme_total + eoff + k] = me[(int64_t)a * nme + k] + (int32_t)voff;
}
}  // namespace

// Vertex -> (element, corner) incidence lists, ascending element order within each
// vertex (a stable sort of the corners by vertex). Built on first use.
int fe_build_vertex_map(fe_pattern_s* h, cudaStream_t s) {
  if (h->vmap_ptr) return FE_OK;
  const int64_t n = h->nme * h->nv;
  dev_tmp tmp;
  fe_sort_buffers sb;
  FE_TRY(tmp.get(&sb.k0, n));
  FE_TRY(tmp.get(&sb.k1, n));
  FE_TRY(tmp.get(&sb.v0, n));
  FE_TRY(tmp.get(&sb.v1, n));
  FE_TRY(tmp.get(&sb.hist, fe_sort_hist_size(n)));
  FE_TRY(tmp.get(&sb.scan_tmp, fe_scan_tmp_size((int64_t)fe_sort_hist_size(n)) + 1));
  const int T = 256;
  k_vmap_keys<<<fe_grid(n, T), T, 0, s>>>(h->me_int, h->nme, h->nv, sb.k0, sb.v0);
  FE_CUDA_TRY(cudaGetLastError());
  uint64_t* keys; uint32_t* vals;
  FE_TRY(fe_radix_sort(n, bitlen((uint64_t)(h->nq > 1 ? h->nq - 1 : 1)), &sb, &keys, &vals, s));
  FE_TRY(fe_malloc(h, (void**)&h->vmap_ptr, sizeof(int32_t) * (h->nq + 1)));
  FE_TRY(fe_malloc(h, (void**)&h->vmap, sizeof(int32_t) * n));
  k_vmap_ptr<<<fe_grid(n, T), T, 0, s>>>(keys, n, h->nq, h->vmap_ptr);
  FE_CUDA_TRY(cudaGetLastError());
  FE_CUDA_TRY(cudaMemcpyAsync(h->vmap, vals, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
  FE_CUDA_TRY(cudaStreamSynchronize(s));
  return FE_OK;
}

namespace {
int fe_pattern_impl(const fe_mesh* mesh, int32_t m, int32_t flags, void* stream, fe_pattern_h* out,
                    const int32_t* group, int group_bits, int kdim, int pk = 1);
}  // namespace

extern "C" int fe_batch_pattern(const fe_mesh* meshes, int32_t count, int32_t m, int32_t flags,
                                void* stream, fe_pattern_h* out) {
  if (!meshes || !out || count < 1) return FE_ERR_ARG;
  *out = nullptr;
  const int d = meshes[0].d;
  std::vector<int64_t> voff(count + 1, 0), eoff(count + 1, 0);
  for (int b = 0; b < count; ++b) {
    const fe_mesh& mb = meshes[b];
    if (mb.d != d || mb.nq < 1 || mb.nme < 1 || !mb.q || !mb.me) return FE_ERR_ARG;
    voff[b + 1] = voff[b] + mb.nq;
    eoff[b + 1] = eoff[b] + mb.nme;
  }
  if (voff[count] > INT32_MAX) return FE_ERR_OVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  const int nv = d + 1;
  dev_tmp tmp;
  double* qu;
  int32_t* meu;
  FE_TRY(tmp.get(&qu, (size_t)d * voff[count]));
  FE_TRY(tmp.get(&meu, (size_t)nv * eoff[count]));
  for (int b = 0; b < count; ++b) {
    const fe_mesh& mb = meshes[b];
    for (int c = 0; c < d; ++c)
      FE_CUDA_TRY(cudaMemcpyAsync(qu + c * voff[count] + voff[b], mb.q + c * mb.nq,
                                  sizeof(double) * mb.nq, cudaMemcpyDeviceToDevice, s));
    k_union_me<<<fe_grid(mb.nme, 256), 256, 0, s>>>(mb.me, mb.nme, nv, voff[b], eoff[b], eoff[count], meu);
    FE_CUDA_TRY(cudaGetLastError());
  }
  // order elements by (mesh, Morton code) so that chunks stay inside one mesh
  int32_t* grp;
  FE_TRY(tmp.get(&grp, (size_t)eoff[count]));
  for (int b = 0; b < count; ++b) {
    k_fill_i32<<<fe_grid(eoff[b + 1] - eoff[b], 256), 256, 0, s>>>(grp + eoff[b], eoff[b + 1] - eoff[b], b);
    FE_CUDA_TRY(cudaGetLastError());
  }
  fe_mesh u{d, voff[count], eoff[count], qu, meu};
  FE_TRY(fe_pattern_impl(&u, m, flags, stream, out, grp, bitlen((uint64_t)count), d));
  fe_pattern_s* h = *out;
  h->batch_voff = voff;
  h->batch_eoff = eoff;
  // nonzero offsets: row_ptr at the first row of every mesh
  h->batch_noff.assign(count + 1, 0);
  for (int b = 0; b <= count; ++b) {
    int32_t r = 0;
    FE_CUDA_TRY(cudaMemcpyAsync(&r, h->row_ptr + (int64_t)m * voff[b], sizeof(int32_t),
                                cudaMemcpyDeviceToHost, s));
    FE_CUDA_TRY(cudaStreamSynchronize(s));
    h->batch_noff[b] = r;
  }
  return FE_OK;
}

extern "C" int fe_batch_offsets(fe_pattern_h h, int64_t* vert_off, int64_t* elem_off, int64_t* nnz_off) {
  if (!h || h->batch_voff.empty()) return FE_ERR_ARG;
  const size_t n = h->batch_voff.size();
  for (size_t b = 0; b < n; ++b) {
    if (vert_off) vert_off[b] = h->batch_voff[b];
    if (elem_off) elem_off[b] = h->batch_eoff[b];
    if (nnz_off) nnz_off[b] = h->batch_noff[b];
  }
  return FE_OK;
}

extern "C" int fe_batch_count(fe_pattern_h h, int32_t* count) {
  if (!h || !count) return FE_ERR_ARG;
  *count = h->batch_voff.empty() ? 0 : (int32_t)h->batch_voff.size() - 1;
  return FE_OK;
}

extern "C" int fe_batch_gather_q(fe_pattern_h h, const fe_mesh* meshes, double* q_union, void* stream) {
  if (!h || !meshes || !q_union || h->batch_voff.empty()) return FE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int count = (int)h->batch_voff.size() - 1;
  const int64_t nq = h->nq;
  for (int b = 0; b < count; ++b) {
    if (meshes[b].nq != h->batch_voff[b + 1] - h->batch_voff[b] || !meshes[b].q) return FE_ERR_ARG;
    for (int c = 0; c < h->d; ++c)
      FE_CUDA_TRY(cudaMemcpyAsync(q_union + c * nq + h->batch_voff[b], meshes[b].q + c * meshes[b].nq,
                                  sizeof(double) * meshes[b].nq, cudaMemcpyDeviceToDevice, s));
  }
  return FE_OK;
}

namespace {
// Morton code of each vertex: quantised coordinates (qbits per axis, over the bounding
// box), bits interleaved; value = vertex id (the sort is stable, so ties keep id order).
__global__ void k_vertex_morton_keys(const double* q, int64_t nq, int d, const double* bbox, int qbits,
                                     uint64_t* keys, uint32_t* vals) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= nq) return;
  const double scale = (double)(1u << qbits);
  uint64_t code = 0;
  for (int c = 0; c < d; ++c) {
    const double lo = bbox[c], hi = bbox[d + c];
    double t = (hi > lo) ? (q[(int64_t)c * nq + v] - lo) / (hi - lo) : 0.0;
    t = fmin(fmax(t, 0.0), 1.0);
    uint64_t iq = (uint64_t)(t * scale);
    if (iq >= (1ull << qbits)) iq = (1ull << qbits) - 1;
    code |= spread_bits(iq, d) << c;
  }
  keys[v] = code;
  vals[v] = (uint32_t)v;
}

// inverse permutation; flags an entry of `order` outside [0, n)
__global__ void k_invert_order(const int32_t* order, int64_t n, int32_t* inv, int32_t* bad) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t o = order[i];
  if (o < 0 || o >= n) { atomicExch(bad, 1); return; }
  inv[o] = (int32_t)i;
}

__global__ void k_gather_q(const double* q, int64_t nq, int d, const int32_t* order, double* q_out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nq) return;
  const int32_t o = order[i];
  if (o < 0 || o >= nq) return;
  for (int c = 0; c < d; ++c) q_out[(int64_t)c * nq + i] = q[(int64_t)c * nq + o];
}

__global__ void k_renumber_me(const int32_t* me, int64_t n, int64_t nq, const int32_t* inv, int32_t* me_out,
                              int32_t* bad) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t v = me[i];
  if (v < 0 || v >= nq) { atomicExch(bad, 2); me_out[i] = -1; return; }
  me_out[i] = inv[v];
}
}  // namespace

extern "C" int fe_morton_vertex_order(int32_t d, int64_t nq, const double* q, int32_t* order, void* stream) {
  if ((d != 2 && d != 3) || nq < 1 || nq > INT32_MAX || !q || !order) return FE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int T = 256, qbits = 21;
  dev_tmp tmp;
  fe_sort_buffers sb;
  double* bb;
  FE_TRY(tmp.get(&sb.k0, nq));
  FE_TRY(tmp.get(&sb.k1, nq));
  FE_TRY(tmp.get(&sb.v0, nq));
  FE_TRY(tmp.get(&sb.v1, nq));
  FE_TRY(tmp.get(&sb.hist, fe_sort_hist_size(nq)));
  FE_TRY(tmp.get(&sb.scan_tmp, fe_scan_tmp_size((int64_t)fe_sort_hist_size(nq)) + fe_scan_tmp_size(nq)));
  FE_TRY(tmp.get(&bb, (size_t)256 * 2 * d));
  k_bbox_partial<<<256, 256, 0, s>>>(q, nq, d, bb);
  k_bbox_final<<<1, 32, 0, s>>>(bb, 256, d);
  k_vertex_morton_keys<<<fe_grid(nq, T), T, 0, s>>>(q, nq, d, bb, qbits, sb.k0, sb.v0);
  FE_CUDA_TRY(cudaGetLastError());
  uint64_t* keys;
  uint32_t* vals;
  FE_TRY(fe_radix_sort(nq, qbits * d, &sb, &keys, &vals, s));
  FE_CUDA_TRY(cudaMemcpyAsync(order, vals, sizeof(int32_t) * nq, cudaMemcpyDeviceToDevice, s));
  FE_CUDA_TRY(cudaStreamSynchronize(s));  // the scratch is released on return
  return FE_OK;
}

extern "C" int fe_apply_vertex_order(int32_t d, int64_t nq, int64_t nme, int32_t nv, const double* q,
                                     const int32_t* me, const int32_t* order, double* q_out,
                                     int32_t* me_out, void* stream) {
  if ((d != 2 && d != 3) || nq < 1 || nq > INT32_MAX || nme < 0 || nv < 1 || !q || !me || !order ||
      !q_out || !me_out)
    return FE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int T = 256;
  dev_tmp tmp;
  int32_t *inv, *bad;
  FE_TRY(tmp.get(&inv, nq));
  FE_TRY(tmp.get(&bad, 1));
  FE_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int32_t), s));
  FE_CUDA_TRY(cudaMemsetAsync(inv, 0xFF, sizeof(int32_t) * nq, s));
  k_invert_order<<<fe_grid(nq, T), T, 0, s>>>(order, nq, inv, bad);
  k_gather_q<<<fe_grid(nq, T), T, 0, s>>>(q, nq, d, order, q_out);
  const int64_t n = nme * nv;
  if (n > 0) k_renumber_me<<<fe_grid(n, T), T, 0, s>>>(me, n, nq, inv, me_out, bad);
  FE_CUDA_TRY(cudaGetLastError());
  int32_t flag = 0;
  FE_CUDA_TRY(cudaMemcpyAsync(&flag, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FE_CUDA_TRY(cudaStreamSynchronize(s));
  return flag ? FE_ERR_INDEX : FE_OK;
}

namespace {
void free_plan(fe_pattern_s* h) {
  void** ptrs[] = {(void**)&h->ch_v_ptr, (void**)&h->ch_e_ptr, (void**)&h->lv_off, (void**)&h->le_off,
                   (void**)&h->inc_v,    (void**)&h->inc_e,    (void**)&h->lv_dst, (void**)&h->lv_vid,
                   (void**)&h->le_dst,   (void**)&h->lv_str,   (void**)&h->le_str, (void**)&h->sh_ptr,
                   (void**)&h->sh_dst,   (void**)&h->sh_str,   (void**)&h->rec,    (void**)&h->rec_off16,
                   &h->partials};
  for (void** p : ptrs) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
}

int fe_pattern_impl(const fe_mesh* mesh, int32_t m, int32_t flags, void* stream, fe_pattern_h* out,
                    const int32_t* group, int group_bits, int kdim, int pk);
}  // namespace

extern "C" int fe_pattern(const fe_mesh* mesh, int32_t m, int32_t flags, void* stream,
                          fe_pattern_h* out) {
  if (!mesh) return FE_ERR_ARG;
  return fe_pattern_impl(mesh, m, flags, stream, out, nullptr, 0, mesh->d);
}

extern "C" int fe_boundary_pattern(const fe_mesh* facets, int32_t flags, void* stream, fe_pattern_h* out) {
  if (!facets) return FE_ERR_ARG;
  return fe_pattern_impl(facets, 1, flags, stream, out, nullptr, 0, facets->d - 1);
}

extern "C" int fe_pk_pattern(const fe_mesh* mesh, int32_t k, int32_t flags, void* stream, fe_pattern_h* out) {
  if (!mesh || k < 1 || k > FE_PK_MAX) return FE_ERR_ARG;
  return fe_pattern_impl(mesh, 1, flags, stream, out, nullptr, 0, mesh->d, k);
}

namespace {
int fe_pattern_impl(const fe_mesh* mesh, int32_t m, int32_t flags, void* stream, fe_pattern_h* out,
                    const int32_t* group, int group_bits, int kdim, int pk) {
  if (!mesh || !out) return FE_ERR_ARG;
  *out = nullptr;
  const int d = mesh->d;
  if (d != 2 && d != 3) return FE_ERR_ARG;
  if (m != 1 && m != d) return FE_ERR_ARG;
  if (mesh->nq < 1 || mesh->nme < 1 || !mesh->q || !mesh->me) return FE_ERR_ARG;
  if (kdim != d && !(kdim == d - 1 && m == 1)) return FE_ERR_ARG;
  if (pk > 1 && (kdim != d || m != 1)) return FE_ERR_ARG;
  // interleaved records: scalar volume patterns only
  if ((flags & FE_PATTERN_INTERLEAVED) && (m != 1 || kdim != d || pk > 1)) return FE_ERR_ARG;
  const int nv = pk > 1 ? fe_pk_nodes(d, pk) : kdim + 1, S = nv * nv;
  const int64_t nq = mesh->nq, nme = mesh->nme;
  if (nq > INT32_MAX / m || nme > INT32_MAX / S) return FE_ERR_OVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  fe_pattern_s* h = new fe_pattern_s();
  h->d = d; h->m = m; h->nv = nv; h->npair = nv * (nv - 1) / 2; h->flags = flags;
  h->kdim = kdim;
  h->pk = pk;
  h->nq = nq; h->nme = nme; h->n = (int64_t)m * nq;
  h->chunk = kdim == d ? default_chunk(d, m, flags) : default_chunk(2, 1, flags);
  if (pk > 1) {  // the plan's uint16 incidence codes: chunk * npair < 2^15, chunk * nv < 2^16
    const int cmax = 32767 / h->npair < 65535 / nv ? 32767 / h->npair : 65535 / nv;
    if (h->chunk > cmax) h->chunk = cmax < 1 ? 1 : cmax;
  }
  int rc = FE_OK;
  dev_tmp tmp;
  do {
    const int T = 256;
    rc = fe_malloc(h, (void**)&h->status, sizeof(fe_status_word));
    if (rc) break;
    {
      fe_status_word init = {0, 0, ~0ull};
      if (cudaMemcpyAsync(h->status, &init, sizeof(init), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        rc = FE_ERR_CUDA; break;
      }
    }
    k_check_me<<<fe_grid(nme, T, 4096), T, 0, s>>>(mesh->me, nme, nv, nq, h->status);
    fe_status_word st;
    if (cudaMemcpyAsync(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) { rc = FE_ERR_CUDA; break; }
    if (st.code != 0) { rc = st.code; break; }

    const int64_t nslots = nme * S;
    const int64_t nkeys = nslots > nme * (nv > h->npair ? nv : h->npair) ? nslots : nme * nv;
    fe_sort_buffers sb;
    if ((rc = tmp.get(&sb.k0, nkeys)) || (rc = tmp.get(&sb.k1, nkeys)) ||
        (rc = tmp.get(&sb.v0, nkeys)) || (rc = tmp.get(&sb.v1, nkeys)) ||
        (rc = tmp.get(&sb.hist, fe_sort_hist_size(nkeys))) ||
        (rc = tmp.get(&sb.scan_tmp, fe_scan_tmp_size((int64_t)fe_sort_hist_size(nkeys)) +
                                        fe_scan_tmp_size(nkeys))))
      break;
    uint64_t* keys; uint32_t* vals;

    // 2. internal element order
    if ((rc = fe_malloc(h, (void**)&h->me_int, sizeof(int32_t) * nv * nme))) break;
    if ((rc = fe_malloc(h, (void**)&h->order, sizeof(int32_t) * nme))) break;
    if (flags & FE_PATTERN_KEEP_ORDER) {
      k_iota<<<fe_grid(nme, T), T, 0, s>>>(sb.v0, nme);
      vals = sb.v0;
    } else {
      double* bb;
      const int nblk = 256;
      if ((rc = tmp.get(&bb, (size_t)nblk * 2 * d))) break;
      k_bbox_partial<<<nblk, 256, 0, s>>>(mesh->q, nq, d, bb);
      k_bbox_final<<<1, 32, 0, s>>>(bb, nblk, d);
      int qbits = (bitlen((uint64_t)nme) + d - 1) / d + 2;
      if (qbits > 21) qbits = 21;
      const int gbits = group ? group_bits : 0;
      if (qbits * d + gbits > 64) qbits = (64 - gbits) / d;
      k_morton_keys<<<fe_grid(nme, T), T, 0, s>>>(mesh->q, nq, mesh->me, nme, d, nv, bb, qbits, group,
                                                 sb.k0, sb.v0);
      if (cudaGetLastError() != cudaSuccess) { rc = FE_ERR_CUDA; break; }
      if ((rc = fe_radix_sort(nme, qbits * d + (group ? group_bits : 0), &sb, &keys, &vals, s))) break;
    }
    k_permute_me<<<fe_grid(nme, T), T, 0, s>>>(mesh->me, nme, nv, vals, h->me_int, h->order);
    if (cudaGetLastError() != cudaSuccess) { rc = FE_ERR_CUDA; break; }

    // 3. scalar pattern
    k_slot_keys<<<fe_grid(nslots, T), T, 0, s>>>(h->me_int, nme, nv, nq, sb.k0, sb.v0);
    if (cudaGetLastError() != cudaSuccess) { rc = FE_ERR_CUDA; break; }
    const int kbits = bitlen((uint64_t)nq * (uint64_t)nq - 1ull);
    if ((rc = fe_radix_sort(nslots, kbits, &sb, &keys, &vals, s))) break;
    uint32_t *flag, *pos;
    if ((rc = tmp.get(&flag, nslots + 1)) || (rc = tmp.get(&pos, nslots + 1))) break;
    k_key_change<<<fe_grid(nslots, T), T, 0, s>>>(keys, nslots, flag);
    if ((rc = fe_scan_exclusive(flag, pos, nslots, sb.scan_tmp, s))) break;
    uint32_t lp = 0, lf = 0;
    if ((rc = to_host(&lp, pos + nslots - 1, s)) || (rc = to_host(&lf, flag + nslots - 1, s))) break;
    const int64_t nnz_s = (int64_t)lp + lf;
    if ((int64_t)m * m * nnz_s > INT32_MAX) { rc = FE_ERR_OVERFLOW; break; }
    h->nnz_s = nnz_s;
    h->nnz = (int64_t)m * m * nnz_s;
    if ((rc = fe_malloc(h, (void**)&h->row_ptr_s, sizeof(int32_t) * (nq + 1))) ||
        (rc = fe_malloc(h, (void**)&h->col_idx_s, sizeof(int32_t) * nnz_s)) ||
        (rc = fe_malloc(h, (void**)&h->slot2nnz, sizeof(int32_t) * nslots)) ||
        (rc = fe_malloc(h, (void**)&h->nnz_slot_ptr, sizeof(int32_t) * (nnz_s + 1))) ||
        (rc = fe_malloc(h, (void**)&h->nnz2slot, sizeof(int32_t) * nslots)))
      break;
    k_rle_scalar<<<fe_grid(nslots, T), T, 0, s>>>(keys, vals, pos, nslots, nq, h->col_idx_s,
                                                  h->row_ptr_s, h->nnz_slot_ptr, h->slot2nnz);
    k_rle_tail<<<1, 1, 0, s>>>(keys, nslots, nq, nnz_s, h->row_ptr_s, h->nnz_slot_ptr);
    if (cudaMemcpyAsync(h->nnz2slot, vals, sizeof(int32_t) * nslots, cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess) { rc = FE_ERR_CUDA; break; }
    if (cudaGetLastError() != cudaSuccess) { rc = FE_ERR_CUDA; break; }

    // 4. vector pattern
    if (m == 1) {
      h->row_ptr = h->row_ptr_s;
      h->col_idx = h->col_idx_s;
    } else {
      if ((rc = fe_malloc(h, (void**)&h->row_ptr, sizeof(int32_t) * (m * nq + 1))) ||
          (rc = fe_malloc(h, (void**)&h->col_idx, sizeof(int32_t) * h->nnz)))
        break;
      k_expand_csr<<<fe_grid(nq, T), T, 0, s>>>(h->row_ptr_s, h->col_idx_s, nq, m, h->row_ptr,
                                                h->col_idx);
      if (cudaGetLastError() != cudaSuccess) { rc = FE_ERR_CUDA; break; }
    }

    // 5. chunk plan
    // shrink the chunk until the worst-case block's shared memory fits (227 KB)
    for (;;) {
      const int64_t bytes_before = h->bytes;
      if ((rc = build_chunk_plan(h, &sb, tmp, s))) break;
      const uint32_t need =
          pk > 1 ? fe::pk_smem((uint32_t)nv, (uint32_t)h->npair, 8, (uint32_t)h->rec_max_bytes, (uint32_t)h->chunk).total
          : (flags & FE_PATTERN_INTERLEAVED)
              ? fe::ilv_smem(d, 8, true, (uint32_t)h->rec_max_bytes, (uint32_t)h->max_lv, (uint32_t)h->max_slots).total
          : kdim == d
              ? fe::plan_smem_worst(d, m, (uint32_t)h->rec_max_bytes, (uint32_t)h->max_lv, (uint32_t)h->chunk)
              : fe::boundary_smem(d, 8, true, (uint32_t)h->rec_max_bytes, (uint32_t)h->max_lv,
                                  (uint32_t)h->chunk).total;
      if (need <= fe::kSmemDynMax || h->chunk <= (pk > 1 ? 1 : 32)) break;
      if (cudaStreamSynchronize(s) != cudaSuccess) { rc = FE_ERR_CUDA; break; }
      free_plan(h);
      h->bytes = bytes_before;
      h->chunk /= 2;
    }
    if (rc) break;
    if (pk > 1 && (rc = fe_pk_upload_table(h, s))) break;
    if ((rc = fe_ensure_scratch(h, h->strategy))) break;
    if (cudaStreamSynchronize(s) != cudaSuccess) { rc = FE_ERR_CUDA; break; }
  } while (0);
  if (rc != FE_OK) {
    cudaStreamSynchronize(s);
    fe_free_all(h);
    delete h;
    return rc;
  }
  *out = h;
  return FE_OK;
}
}  // namespace
