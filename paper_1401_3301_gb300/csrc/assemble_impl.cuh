// Scalar operators (mass, weighted mass, stiffness): element values and the three
// reassembly strategies. Included by one translation unit per precision form.
#pragma once

#include "check.cuh"
#include "elem.cuh"
#include "fe_internal.cuh"
#include "plan.cuh"
#include "tma.cuh"

namespace fe {

enum Kind : int { K_MASS = 0, K_WMASS_P1 = 1, K_WMASS_P0 = 2, K_STIFF = 3 };

template <int D, class T>
struct ScalarVals {
  T diag[D + 1];
  T off[Pairs<D>::n];
  T scale;  // common factor still to be applied (1 unless the scaling is deferred)
};

// per-element coefficient (P0 kinds); 1 when there is none
template <class T>
__device__ __forceinline__ T elem_coef(const void* w, int w_kind, const int32_t* order, int64_t e) {
  const T* wp = (const T*)w;
  if (w_kind == FE_COEF_P0) return wp[order[e]];
  if (w_kind == FE_COEF_P0_INTERNAL) return wp[e];
  if (w_kind == FE_COEF_SCALAR) return wp[0];
  return T(1);
}

// Local matrix entries from the geometry. wv: vertex values of the weight (P1 kind).
// Stiffness: FP64 forms the Gram matrix of c_1..c_D and the row of vertex 0 from row
// sums (fewer FP64 operations); FP32 takes c_a . c_b for every pair, c_0 included.
// DEFER (stiffness): leave the per-element factor w / (d! |det B|) in out.scale for the
// caller to apply while summing (one FMA per incidence instead of six products here).
template <int D, class T, int KIND, bool DEFER = false>
__device__ __forceinline__ void values_from_geo(const Geo<D, T>& g, bool has_coef, T coef,
                                                const T* wv, ScalarVals<D, T>& out) {
  constexpr int NV = D + 1;
  const T adet = tabs(g.det);
  out.scale = T(1);
  if constexpr (KIND == K_STIFF) {
    T inv = recip<T>(T(factorial(D)) * adet);
    if (has_coef) inv *= coef;
    if constexpr (DEFER) {
      out.scale = inv;
      inv = T(1);
    }
    if constexpr (sizeof(T) == 4) {
      // FP32: every entry from its own cofactors (c_0 from geo_f32): the row sums that
      // the FP64 form uses for vertex 0 would cancel in float where c_0 is short
      {
#pragma unroll
        for (int a = 0; a < NV; ++a) {
          T t = g.c[a][0] * g.c[a][0];
#pragma unroll
          for (int k = 1; k < D; ++k) t += g.c[a][k] * g.c[a][k];
          out.diag[a] = t * inv;
        }
#pragma unroll
        for (int p = 0; p < Pairs<D>::n; ++p) {
          const int a = Pairs<D>::a(p), b = Pairs<D>::b(p);
          T t = g.c[a][0] * g.c[b][0];
#pragma unroll
          for (int k = 1; k < D; ++k) t += g.c[a][k] * g.c[b][k];
          out.off[p] = t * inv;
        }
        return;
      }
    }
    // scaled Gram matrix of c_1..c_D; the row of vertex 0 follows from sum_a c_a = 0
    T G[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = i; j < D; ++j) {
        T s = g.c[i + 1][0] * g.c[j + 1][0];
#pragma unroll
        for (int k = 1; k < D; ++k) s += g.c[i + 1][k] * g.c[j + 1][k];
        G[i][j] = DEFER ? s : s * inv;
        G[j][i] = G[i][j];
      }
    T nr[D];  // nr[i] = S_{0, i+1} = -sum_j G[i][j]
#pragma unroll
    for (int i = 0; i < D; ++i) {
      T s = -G[i][0];
#pragma unroll
      for (int j = 1; j < D; ++j) s -= G[i][j];
      nr[i] = s;
    }
    T d0 = -nr[0];
#pragma unroll
    for (int i = 1; i < D; ++i) d0 -= nr[i];
    out.diag[0] = d0;
#pragma unroll
    for (int i = 0; i < D; ++i) out.diag[i + 1] = G[i][i];
#pragma unroll
    for (int p = 0; p < Pairs<D>::n; ++p) {
      const int a = Pairs<D>::a(p), b = Pairs<D>::b(p);
      out.off[p] = (a == 0) ? nr[b - 1] : G[a - 1][b - 1];
    }
  } else if constexpr (KIND == K_MASS || KIND == K_WMASS_P0) {
    T m = adet * T(1.0 / factorial(D + 2));
    if (has_coef) m *= coef;
#pragma unroll
    for (int a = 0; a < NV; ++a) out.diag[a] = T(2) * m;
#pragma unroll
    for (int p = 0; p < Pairs<D>::n; ++p) out.off[p] = m;
  } else {  // K_WMASS_P1
    T ws = wv[0];
#pragma unroll
    for (int a = 1; a < NV; ++a) ws += wv[a];
    const T base = adet * T(1.0 / factorial(D + 3));
#pragma unroll
    for (int a = 0; a < NV; ++a) out.diag[a] = T(2) * base * (ws + T(2) * wv[a]);
#pragma unroll
    for (int p = 0; p < Pairs<D>::n; ++p)
      out.off[p] = base * (ws + wv[Pairs<D>::a(p)] + wv[Pairs<D>::b(p)]);
  }
}

struct ElemArgs {
  const int32_t* me;   // internal order, (d+1) x nme
  int64_t nme, nq;
  const double* q;     // FP64 form
  const float4* qs;    // FP32 form: split coordinates
  const void* w;       // coefficient (double or float, by form)
  int w_kind;          // FE_COEF_*
  const int32_t* order;
  fe_status_word* st;
};

// geometry of internal element e (vertex ids in v), coordinates gathered from global
// memory; a degenerate element is reported and given det B = 1
template <int D, class T, bool COF = true>
__device__ __forceinline__ void element_geo(const ElemArgs& A, int64_t e, int32_t v[D + 1], Geo<D, T>& g) {
  constexpr int NV = D + 1;
#pragma unroll
  for (int a = 0; a < NV; ++a) v[a] = __ldg(A.me + (int64_t)a * A.nme + e);
  if constexpr (sizeof(T) == 8) {
    double x[NV][D];
    load_x64<D>(A.q, A.nq, v, x);
    geo_f64<D>(x, g);
  } else {
    float xh[NV][D], xl[NV][D];
    load_x32<D>(A.qs, v, xh, xl);
    geo_f32<D, COF>(xh, xl, g);
    guard_geo_f32<D>(g, A.q, A.nq, v);
  }
  if (!det_ok(g.det)) {
    fe_report(A.st, FE_ERR_DEGENERATE, A.order[e]);
    g.det = T(1);
  }
}

// values of internal element e, coordinates gathered from global memory
template <int D, class T, int KIND>
__device__ __forceinline__ void element_values(const ElemArgs& A, int64_t e, ScalarVals<D, T>& out) {
  constexpr int NV = D + 1;
  int32_t v[NV];
  Geo<D, T> g;
  element_geo<D, T, KIND == K_STIFF>(A, e, v, g);
  T wv[NV];
  if constexpr (KIND == K_WMASS_P1) {
#pragma unroll
    for (int a = 0; a < NV; ++a) wv[a] = ((const T*)A.w)[v[a]];
  }
  const bool has_coef = A.w_kind != FE_COEF_NONE && KIND != K_WMASS_P1;
  const T coef = has_coef ? elem_coef<T>(A.w, A.w_kind, A.order, e) : T(1);
  values_from_geo<D, T, KIND>(g, has_coef, coef, wv, out);
}

// accumulators: FP64 plain sum, FP32 compensated sum
template <class T>
struct Acc;
template <>
struct Acc<double> {
  double s;
  Acc() = default;
  __device__ __forceinline__ explicit Acc(double first) : s(first) {}
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ void add_scaled(double x, double f) { s = fma(x, f, s); }
  __device__ __forceinline__ double value() const { return s; }
  __device__ __forceinline__ void store_partial(void* p, int64_t i) const { ((double*)p)[i] = s; }
  __device__ __forceinline__ static Acc from_partial(const void* p, int64_t i) {
    return Acc(((const double*)p)[i]);
  }
  __device__ __forceinline__ void add_partial(const void* p, int64_t i) { s += ((const double*)p)[i]; }
  __device__ __forceinline__ void add_acc(const Acc& o) { s += o.s; }
  __device__ __forceinline__ void scale2() { s *= 2.0; }  // exact
};
template <>
struct Acc<float> {
  csum s;
  Acc() = default;
  __device__ __forceinline__ explicit Acc(float first) { s.s = first; s.c = 0.f; }
  __device__ __forceinline__ void add(float x) { s.add(x); }
  __device__ __forceinline__ void add_scaled(float x, float f) { s.add(x * f); }
  __device__ __forceinline__ float value() const { return s.value(); }
  // a chunk's partial sum is stored rounded to one float (4 bytes of partial traffic
  // instead of 8; the rounding adds at most 2^-24 of the partial's magnitude, and the
  // fixup sums the partials with compensation again)
  __device__ __forceinline__ void store_partial(void* p, int64_t i) const { ((float*)p)[i] = s.value(); }
  __device__ __forceinline__ static Acc from_partial(const void* p, int64_t i) {
    return Acc(((const float*)p)[i]);
  }
  __device__ __forceinline__ void add_partial(const void* p, int64_t i) { s.add(((const float*)p)[i]); }
  __device__ __forceinline__ void add_acc(const Acc& o) { s.add2(o.s.s, o.s.c); }
  __device__ __forceinline__ void scale2() {  // exact: every rounding of the sum scales by 2
    s.s *= 2.f;
    s.c *= 2.f;
  }
};

// ---------------------------------------------------------------- FE_REASM_CHUNKED
// Bulk (TMA) copy of chunk c's plan record into the start of shared memory, on the
// mbarrier bar; true in every thread once it has landed. On a timeout the block
// reports FE_ERR_TIMEOUT (element e0), waits once more for the copy in flight and
// every thread gets false.
__device__ __forceinline__ bool load_plan_record(unsigned char* smem, uint64_t* bar, const uint8_t* rec,
                                                 const uint32_t* rec_off16, int64_t c, uint32_t bytes,
                                                 fe_status_word* st, int64_t e0, uint32_t spin) {
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_arrive_expect_tx(bar, bytes);
    bulk_copy_g2s(smem, rec + (int64_t)rec_off16[c] * 16, bytes, bar);
  }
  __syncthreads();
  const bool landed = __syncthreads_and(mbar_wait_bounded(bar, 0, spin));
  if (!landed && threadIdx.x == 0) {
    fe_report(st, FE_ERR_TIMEOUT, e0);
    mbar_wait_bounded(bar, 0, spin);  // let the copy in flight finish, if it can
  }
  return landed;
}

// Coordinates of global vertex vid into local slot u of the staged coordinate array
// sq: FP64 (x, y[, z]) in 16 (2D) or 32 (3D) bytes; FP32 the (hi, lo) float split of
// x - xr, xr a reference vertex of the chunk (one FP64 subtraction per coordinate), so
// that the split's error (2^-47 of the split value) scales with the chunk's extent, not
// with the distance from the origin; xr = nullptr splits x itself.
template <int D, class T>
__device__ __forceinline__ void stage_vertex(const double* __restrict__ q, int64_t nq, int64_t vid,
                                             unsigned char* sq, int u, const double* xr = nullptr) {
  double x[D];
#pragma unroll
  for (int k = 0; k < D; ++k) x[k] = __ldg(q + k * nq + vid);
  if constexpr (sizeof(T) == 4) {
    if (xr) {
#pragma unroll
      for (int k = 0; k < D; ++k) x[k] -= xr[k];
    }
  }
  if constexpr (sizeof(T) == 8) {
    double* xs = (double*)sq + (D == 3 ? 4 : 2) * u;
    ((double2*)xs)[0] = make_double2(x[0], x[1]);
    if constexpr (D == 3) xs[2] = x[2];
  } else {
    float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < D; ++k) split_f64(x[k], h[k], l[k]);
    float4* xs = (float4*)sq + (D == 3 ? 2 : 1) * u;
    if constexpr (D == 3) {
      xs[0] = make_float4(h[0], h[1], h[2], 0.f);
      xs[1] = make_float4(l[0], l[1], l[2], 0.f);
    } else {
      xs[0] = make_float4(h[0], h[1], l[0], l[1]);
    }
  }
}

// Geometry of an element whose corners are the local vertices lv of the staged array sq.
// FP32 form: a det B that fails its guard is recomputed in FP64 from q and the global
// vertex ids lv_vid of the chunk's local vertices.
template <int D, class T, bool COF = true>
__device__ __forceinline__ void staged_geo(const unsigned char* sq, const int lv[D + 1], Geo<D, T>& g,
                                           const double* __restrict__ q, int64_t nq, const int32_t* lv_vid) {
  constexpr int NV = D + 1;
  if constexpr (sizeof(T) == 8) {
    double x[NV][D];
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      const double* xs = (const double*)sq + (D == 3 ? 4 : 2) * lv[a];
      const double2 xy = ((const double2*)xs)[0];
      x[a][0] = xy.x;
      x[a][1] = xy.y;
      if constexpr (D == 3) x[a][2] = xs[2];
    }
    geo_f64<D>(x, g);
  } else {
    float xh[NV][D], xl[NV][D];
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      const float4* xs = (const float4*)sq + (D == 3 ? 2 : 1) * lv[a];
      const float4 h = xs[0];
      if constexpr (D == 3) {
        const float4 l = xs[1];
        xh[a][0] = h.x; xh[a][1] = h.y; xh[a][2] = h.z;
        xl[a][0] = l.x; xl[a][1] = l.y; xl[a][2] = l.z;
      } else {
        xh[a][0] = h.x; xh[a][1] = h.y;
        xl[a][0] = h.z; xl[a][1] = h.w;
      }
    }
    geo_f32<D, COF>(xh, xl, g);
    if (g.full || fabsf(g.det) < kDetGuardF32 * g.dsc) {
      int32_t v[NV];
#pragma unroll
      for (int a = 0; a < NV; ++a) v[a] = lv_vid[lv[a]];
      guard_geo_f32<D>(g, q, nq, v);
    }
  }
}

struct StagedArgs {
  int64_t nme, nq;
  int chunk;
  uint32_t rec_max, max_lv;
  const double* q;
  const void* w;
  int w_kind;
  const int32_t* order;
  const int32_t* ch_v_ptr;
  const int32_t* ch_e_ptr;
  const uint8_t* rec;
  const uint32_t* rec_off16;
  fe_status_word* st;
  int64_t nnz, npart;  // sizes of vals and of the partial sums (bounds-checked builds)
  const int32_t* me0;  // FP32 form: corner 0 of each internal element (chunk reference vertex)
};

// FP32 form: coordinates of the chunk's reference vertex, corner 0 of its first element
// (independent of the record's vertex order), or none without me0
template <int D>
struct ChunkRef {
  double x[D];
  bool on;
  __device__ __forceinline__ ChunkRef(const double* __restrict__ q, int64_t nq, const int32_t* me0, int64_t e0)
      : on(me0 != nullptr) {
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = on ? __ldg(q + k * nq + me0[e0]) : 0.0;
  }
  __device__ __forceinline__ const double* ptr() const { return on ? x : nullptr; }
};

constexpr uint32_t kBarrierSpin = 1u << 22;

// One block per chunk of internal elements.
//  0. one bulk (TMA) copy brings the chunk's plan record into shared memory; the
//     coordinates of the chunk's distinct vertices are read once from q (split into
//     hi/lo floats for the FP32 form); the record also gives each element corner its
//     local vertex;
//  1. element values into shared memory (diagonal per corner, off-diagonal per edge);
//  2. each distinct vertex / edge sums its incidences in ascending element order and
//     stores the sum in the CSR value (both (i,j) and (j,i) for an edge: the
//     operators are symmetric) or in its partial-sum slot.
// FP32 form: registers capped so that 6 blocks of 256 threads fit on an SM (40 per
// thread): the kernel is bound by the latency of each block's dependent steps, and more
// resident blocks hide more of it (chunk 384: 0.241 -> 0.209 ms at N=100). The FP64 form
// is bound by the FP64 pipe and keeps the compiler's choice.
template <int D, class T, int KIND, int THREADS>
__global__ void __launch_bounds__(THREADS, sizeof(T) == 4 ? 1536 / THREADS : 1) k_chunk_staged(StagedArgs A, T* __restrict__ vals,
                                                          void* __restrict__ partials) {
  constexpr int NV = D + 1, NP = Pairs<D>::n;
  // FP64 stiffness: apply each element's scale while summing (FMA) instead of per entry
  constexpr bool DEFER = (KIND == K_STIFF) && (sizeof(T) == 8);
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  const int64_t c = blockIdx.x;
  const int64_t e0 = c * A.chunk;
  const int ne = (int)min((int64_t)A.chunk, A.nme - e0);
  const int32_t nlv = A.ch_v_ptr[c + 1] - A.ch_v_ptr[c];
  const int32_t nle = A.ch_e_ptr[c + 1] - A.ch_e_ptr[c];
  const RecLayout R = rec_layout((uint32_t)ne, NV, NP, (uint32_t)nlv, (uint32_t)nle);
  const StagedSmem S = staged_smem(D, (int)sizeof(T), KIND == K_WMASS_P1, A.rec_max, A.max_lv, A.chunk, DEFER);
  if (!FE_CHUNK_FITS(R.total <= A.rec_max && nlv <= (int32_t)A.max_lv, A.st, c)) return;
  // reference vertex of the chunk, loaded while the record copy is in flight
  const ChunkRef<D> xr(A.q, A.nq, sizeof(T) == 4 ? A.me0 : nullptr, e0);
  if (!load_plan_record(smem, &bar, A.rec, A.rec_off16, c, R.total, A.st, e0, kBarrierSpin)) return;
  const uint16_t* inc_v = (const uint16_t*)(smem + R.inc_v);
  const uint16_t* inc_e = (const uint16_t*)(smem + R.inc_e);
  const uint16_t* lv_off = (const uint16_t*)(smem + R.lv_off);
  const uint16_t* le_off = (const uint16_t*)(smem + R.le_off);
  const int32_t* lv_vid = (const int32_t*)(smem + R.lv_vid);
  const int32_t* lv_dst = (const int32_t*)(smem + R.lv_dst);
  const int32_t* le_dst = (const int32_t*)(smem + R.le_dst);
  const uint16_t* lvid = (const uint16_t*)(smem + R.lvid);
  T* Kd = (T*)(smem + S.kd);
  T* Ko = (T*)(smem + S.ko);
  T* wl = (T*)(smem + S.w);
  T* Sc = (T*)(smem + S.sc);
  if (!FE_RECORD_VALID(smem, R, ne, NV, NP, nlv, nle, 1, A.nq, A.nnz, A.npart, A.st, c)) return;

  // 0. vertex coordinates of the chunk (the record carries each corner's local vertex)
  for (int u = threadIdx.x; u < nlv; u += THREADS) {
    const int64_t vid = lv_vid[u];
    stage_vertex<D, T>(A.q, A.nq, vid, smem + S.q, u, xr.ptr());
    if constexpr (KIND == K_WMASS_P1) wl[u] = ((const T*)A.w)[vid];
  }
  __syncthreads();

  // 1. element values
  const bool has_coef = A.w_kind != FE_COEF_NONE && KIND != K_WMASS_P1;
  for (int el = threadIdx.x; el < ne; el += THREADS) {
    int lv[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) lv[a] = lvid[el * NV + a];
    Geo<D, T> g;
    staged_geo<D, T, KIND == K_STIFF>(smem + S.q, lv, g, A.q, A.nq, lv_vid);
    if (!det_ok(g.det)) {
      fe_report(A.st, FE_ERR_DEGENERATE, A.order[e0 + el]);
      g.det = T(1);
    }
    T wv[NV];
    if constexpr (KIND == K_WMASS_P1) {
#pragma unroll
      for (int a = 0; a < NV; ++a) wv[a] = wl[lv[a]];
    }
    const T coef = has_coef ? elem_coef<T>(A.w, A.w_kind, A.order, e0 + el) : T(1);
    ScalarVals<D, T> v;
    values_from_geo<D, T, KIND, DEFER>(g, has_coef, coef, wv, v);
#pragma unroll
    for (int a = 0; a < NV; ++a) Kd[el * NV + a] = v.diag[a];
#pragma unroll
    for (int p = 0; p < NP; ++p) Ko[el * NP + p] = v.off[p];
    if constexpr (DEFER) Sc[el] = v.scale;
  }
  __syncthreads();

  // 2. sums over the incidences of each distinct vertex and edge, in element order
  for (int u = threadIdx.x; u < nlv; u += THREADS) {
    const int s = lv_off[u], t = lv_off[u + 1];
    Acc<T> acc = DEFER ? Acc<T>(Kd[inc_v[s]] * Sc[inc_v[s] / NV]) : Acc<T>(Kd[inc_v[s]]);
    if constexpr (DEFER) {
      // FP64: the scaled sums run faster not unrolled (chunk kernel 0.801 -> 0.791 ms at
      // N=100); the FP32 sums need the compiler's unrolling (0.209 against 0.227 ms)
#pragma unroll 1
      for (int j = s + 1; j < t; ++j) acc.add_scaled(Kd[inc_v[j]], Sc[inc_v[j] / NV]);
    } else {
      for (int j = s + 1; j < t; ++j) acc.add(Kd[inc_v[j]]);
    }
    const int32_t dst = lv_dst[u];
    if (dst >= 0) vals[dst] = acc.value();
    else acc.store_partial(partials, -1 - (int64_t)dst);
  }
  for (int u = threadIdx.x; u < nle; u += THREADS) {
    const int s = le_off[u], t = le_off[u + 1];
    const int i0 = inc_e[s] >> 1;
    Acc<T> acc = DEFER ? Acc<T>(Ko[i0] * Sc[i0 / NP]) : Acc<T>(Ko[i0]);
    if constexpr (DEFER) {
#pragma unroll 1
      for (int j = s + 1; j < t; ++j) {
        const int ij = inc_e[j] >> 1;
        acc.add_scaled(Ko[ij], Sc[ij / NP]);
      }
    } else {
      for (int j = s + 1; j < t; ++j) acc.add(Ko[inc_e[j] >> 1]);
    }
    const int32_t dst = le_dst[2 * u];
    if (dst >= 0) {
      const T val = acc.value();
      vals[dst] = val;
      vals[le_dst[2 * u + 1]] = val;
    } else {
      acc.store_partial(partials, -1 - (int64_t)dst);
    }
  }
}

// Interleaved records (FE_PATTERN_INTERLEAVED, plan.cuh IlvLayout). One block per chunk:
//  0. the record by one bulk (TMA) copy; the coordinates of the chunk's distinct
//     vertices (split into hi/lo floats relative to the chunk's reference vertex in the
//     FP32 form) and their P1 weights;
//  1. each element reads its corners' local vertices from the record, forms its local
//     matrix and stores each value in the slot the record names for it;
//  2. warp w sums the lists of the 32 vertices (then edges) of group w: step j reads
//     slot grp[w] + 32 j + lane, 32 consecutive slots, and the sums run in ascending
//     element order as in k_chunk_staged. Values are scaled before they are stored
//     (no per-element scale at summation), so the FP32 results equal the plain layout's
//     bit for bit.
template <int D, class T, int KIND, int THREADS>
__global__ void __launch_bounds__(THREADS) k_chunk_ilv(StagedArgs A, T* __restrict__ vals,
                                                       void* __restrict__ partials, uint32_t max_slots) {
  constexpr int NV = D + 1, NP = Pairs<D>::n;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  const int64_t c = blockIdx.x;
  const int64_t e0 = c * A.chunk;
  const int ne = (int)min((int64_t)A.chunk, A.nme - e0);
  const int32_t nlv = A.ch_v_ptr[c + 1] - A.ch_v_ptr[c];
  const int32_t nle = A.ch_e_ptr[c + 1] - A.ch_e_ptr[c];
  const IlvLayout R = ilv_layout((uint32_t)ne, NV, NP, (uint32_t)nlv, (uint32_t)nle);
  const IlvSmem S = ilv_smem(D, (int)sizeof(T), KIND == K_WMASS_P1, A.rec_max, A.max_lv, max_slots);
  if (!FE_CHUNK_FITS(R.total <= A.rec_max && nlv <= (int32_t)A.max_lv, A.st, c)) return;
  // reference vertex of the chunk, loaded while the record copy is in flight
  const ChunkRef<D> xr(A.q, A.nq, sizeof(T) == 4 ? A.me0 : nullptr, e0);
  if (!load_plan_record(smem, &bar, A.rec, A.rec_off16, c, R.total, A.st, e0, kBarrierSpin)) return;
  const uint16_t* corner = (const uint16_t*)(smem + R.corner);
  const uint16_t* vpos = (const uint16_t*)(smem + R.vpos);
  const uint16_t* epos = (const uint16_t*)(smem + R.epos);
  const uint16_t* grp = (const uint16_t*)(smem + R.grp);
  const uint16_t* lv_cnt = (const uint16_t*)(smem + R.lv_cnt);
  const uint16_t* le_cnt = (const uint16_t*)(smem + R.le_cnt);
  const int32_t* lv_vid = (const int32_t*)(smem + R.lv_vid);
  const int32_t* lv_dst = (const int32_t*)(smem + R.lv_dst);
  const int32_t* le_dst = (const int32_t*)(smem + R.le_dst);
  T* V = (T*)(smem + S.vals);
  T* wl = (T*)(smem + S.w);
  if (!FE_RECORD_VALID_ILV(smem, R, ne, NV, NP, nlv, nle, A.nq, A.nnz, A.npart, max_slots, A.st, c)) return;

  // 0. vertex coordinates (and P1 weights) of the chunk
  for (int u = threadIdx.x; u < nlv; u += THREADS) {
    const int64_t vid = lv_vid[u];
    stage_vertex<D, T>(A.q, A.nq, vid, smem + S.q, u, xr.ptr());
    if constexpr (KIND == K_WMASS_P1) wl[u] = ((const T*)A.w)[vid];
  }
  __syncthreads();

  // 1. element values, each to its slot
  const bool has_coef = A.w_kind != FE_COEF_NONE && KIND != K_WMASS_P1;
  for (int el = threadIdx.x; el < ne; el += THREADS) {
    int lv[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) lv[a] = corner[a * ne + el];
    Geo<D, T> g;
    staged_geo<D, T, KIND == K_STIFF>(smem + S.q, lv, g, A.q, A.nq, lv_vid);
    if (!det_ok(g.det)) {
      fe_report(A.st, FE_ERR_DEGENERATE, A.order[e0 + el]);
      g.det = T(1);
    }
    T wv[NV];
    if constexpr (KIND == K_WMASS_P1) {
#pragma unroll
      for (int a = 0; a < NV; ++a) wv[a] = wl[lv[a]];
    }
    const T coef = has_coef ? elem_coef<T>(A.w, A.w_kind, A.order, e0 + el) : T(1);
    ScalarVals<D, T> v;
    values_from_geo<D, T, KIND, false>(g, has_coef, coef, wv, v);
#pragma unroll
    for (int a = 0; a < NV; ++a) V[vpos[a * ne + el]] = v.diag[a];
#pragma unroll
    for (int p = 0; p < NP; ++p) V[epos[p * ne + el]] = v.off[p];
  }
  __syncthreads();

  // 2. sums: one group of 32 vertices (edges) per warp, 32 consecutive slots per step
  for (int u = threadIdx.x; u < nlv; u += THREADS) {
    const T* x = V + grp[u >> 5] + (u & 31);
    const int n = lv_cnt[u];
    Acc<T> acc(x[0]);
    for (int j = 1; j < n; ++j) acc.add(x[32 * j]);
    const int32_t dst = lv_dst[u];
    if (dst >= 0) vals[dst] = acc.value();
    else acc.store_partial(partials, -1 - (int64_t)dst);
  }
  const int ngv = (int)ilv_groups((uint32_t)nlv);
  for (int u = threadIdx.x; u < nle; u += THREADS) {
    const T* x = V + grp[ngv + (u >> 5)] + (u & 31);
    const int n = le_cnt[u];
    Acc<T> acc(x[0]);
    for (int j = 1; j < n; ++j) acc.add(x[32 * j]);
    const int32_t dst = le_dst[2 * u];
    if (dst >= 0) {
      const T val = acc.value();
      vals[dst] = val;
      vals[le_dst[2 * u + 1]] = val;
    } else {
      acc.store_partial(partials, -1 - (int64_t)dst);
    }
  }
}

// Sum of the chunk partials of each shared vertex / edge, in chunk order. The kernel is
// bound by load latency rather than bandwidth, so each thread takes several shared
// entities (strided by the block size: every load stays coalesced) and issues the loads
// of all of them before summing: list bounds and destinations, then the first four
// partials of each entity; longer lists finish one partial at a time. Four entities per
// thread for 8-byte values, two for the FP32 form's (more threads in flight: 0.044 ->
// 0.042 ms at N=100, where four cost the FP64 form nothing and gained it 3 %).
template <class T>
constexpr int fixup_per() { return sizeof(T) == 4 ? 2 : 4; }
template <class T, class AccT = Acc<T>>
__global__ void __launch_bounds__(256) k_fixup_scalar(const int32_t* __restrict__ sh_ptr,
                                                      const int32_t* __restrict__ sh_dst, int64_t nsh_v,
                                                      int64_t nsh, const void* __restrict__ partials,
                                                      T* __restrict__ vals, int64_t nnz, int64_t npart,
                                                      fe_status_word* st) {
  constexpr int E = fixup_per<T>(), F = 4;
  const int64_t g0 = (int64_t)blockIdx.x * blockDim.x * E + threadIdx.x;
  int32_t s[E], n[E];
  int2 dd[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int64_t g = g0 + (int64_t)e * blockDim.x;
    s[e] = 0;
    n[e] = 0;
    dd[e] = make_int2(0, 0);
    if (g < nsh) {
      const int32_t t = sh_ptr[g + 1];
      s[e] = sh_ptr[g];
      dd[e] = reinterpret_cast<const int2*>(sh_dst)[g];  // (i,j) and (j,i) in one load
      n[e] = FE_FIXUP_VALID(s[e], t, npart, dd[e].x, dd[e].y, g >= nsh_v, nnz, st, g) ? t - s[e] : 0;
    }
  }
  AccT p[E][F];
#pragma unroll
  for (int e = 0; e < E; ++e)
#pragma unroll
    for (int k = 0; k < F; ++k)
      if (k < n[e]) p[e][k] = AccT::from_partial(partials, (int64_t)s[e] + k);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (n[e] == 0) continue;
    AccT acc = p[e][0];
#pragma unroll
    for (int k = 1; k < F; ++k)
      if (k < n[e]) acc.add_acc(p[e][k]);
    for (int32_t i = s[e] + F; i < s[e] + n[e]; ++i) acc.add_partial(partials, i);
    const T val = acc.value();
    vals[dd[e].x] = val;
    if (g0 + (int64_t)e * blockDim.x >= nsh_v) vals[dd[e].y] = val;
  }
}

// grid of the fixup: fixup_per<T>() shared entities per thread, 256 threads per block
template <class T>
static inline int fixup_grid(int64_t nsh) { return fe_grid(nsh, 256 * fixup_per<T>()); }

// ---------------------------------------------------------------- FE_REASM_GATHER
// Pass 1: full local matrix of each element, column-wise, at kg[e*S + b*NV + a].
template <int D, class T, int KIND>
__global__ void __launch_bounds__(256) k_elem_kg(ElemArgs A, T* __restrict__ kg) {
  constexpr int NV = D + 1, S = NV * NV;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= A.nme) return;
  ScalarVals<D, T> v;
  element_values<D, T, KIND>(A, e, v);
  T* o = kg + e * S;
#pragma unroll
  for (int a = 0; a < NV; ++a) o[a * NV + a] = v.diag[a];
#pragma unroll
  for (int p = 0; p < Pairs<D>::n; ++p) {
    o[Pairs<D>::b(p) * NV + Pairs<D>::a(p)] = v.off[p];
    o[Pairs<D>::a(p) * NV + Pairs<D>::b(p)] = v.off[p];
  }
}

// Pass 2: each nonzero sums its slots in ascending slot order.
template <class T>
__global__ void __launch_bounds__(256) k_gather(const int32_t* __restrict__ nsp,
                                                const int32_t* __restrict__ n2s, int64_t nnz,
                                                const T* __restrict__ kg, T* __restrict__ vals) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nnz) return;
  const int32_t s = nsp[j], t = nsp[j + 1];
  Acc<T> acc(kg[n2s[s]]);
  for (int32_t i = s + 1; i < t; ++i) acc.add(kg[n2s[i]]);
  vals[j] = acc.value();
}

// ---------------------------------------------------------------- FE_REASM_ATOMIC
template <int D, class T, int KIND>
__global__ void __launch_bounds__(256) k_elem_atomic(ElemArgs A, const int32_t* __restrict__ slot2nnz,
                                                     T* __restrict__ vals) {
  constexpr int NV = D + 1, S = NV * NV;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= A.nme) return;
  ScalarVals<D, T> v;
  element_values<D, T, KIND>(A, e, v);
  const int32_t* m = slot2nnz + e * S;
#pragma unroll
  for (int a = 0; a < NV; ++a) atomicAdd(vals + m[a * NV + a], v.diag[a]);
#pragma unroll
  for (int p = 0; p < Pairs<D>::n; ++p) {
    atomicAdd(vals + m[Pairs<D>::b(p) * NV + Pairs<D>::a(p)], v.off[p]);
    atomicAdd(vals + m[Pairs<D>::a(p) * NV + Pairs<D>::b(p)], v.off[p]);
  }
}

// FP32 form of the two-pass and atomic strategies: split FP64 coordinates into
// (hi, lo) floats, one vertex per thread
template <int D>
__global__ void k_split_q(const double* __restrict__ q, int64_t nq, float4* __restrict__ qs) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= nq) return;
  float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int c = 0; c < D; ++c) split_f64(q[(int64_t)c * nq + v], h[c], l[c]);
  if constexpr (D == 3) {
    qs[2 * v] = make_float4(h[0], h[1], h[2], 0.f);
    qs[2 * v + 1] = make_float4(l[0], l[1], l[2], 0.f);
  } else {
    qs[v] = make_float4(h[0], h[1], l[0], l[1]);
  }
}

}  // namespace fe
