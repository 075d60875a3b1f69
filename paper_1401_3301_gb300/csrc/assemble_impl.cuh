// Scalar operators (mass, weighted mass, stiffness): element values and the three
// reassembly strategies. Included by one translation unit per precision form.
#pragma once

#include "elem.cuh"
#include "fe_internal.cuh"

namespace fe {

enum Kind : int { K_MASS = 0, K_WMASS_P1 = 1, K_WMASS_P0 = 2, K_STIFF = 3 };

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

struct PlanArgs {
  int chunk;
  const int32_t* ch_v_ptr;
  const int32_t* ch_e_ptr;
  const uint16_t* lv_off;
  const uint16_t* le_off;
  const uint16_t* inc_v;
  const uint16_t* inc_e;
  const int32_t* lv_dst;
  const int32_t* le_dst;
};

template <int D, class T>
struct ScalarVals {
  T diag[D + 1];
  T off[Pairs<D>::n];
};

template <class T>
__device__ __forceinline__ T load_coef(const ElemArgs& A, int64_t e) {
  const T* w = (const T*)A.w;
  if (A.w_kind == FE_COEF_P0) return w[A.order[e]];
  if (A.w_kind == FE_COEF_P0_INTERNAL) return w[e];
  if (A.w_kind == FE_COEF_SCALAR) return w[0];
  return T(1);
}

// values of internal element e; returns false (and reports) for a degenerate element
template <int D, class T, int KIND>
__device__ __forceinline__ void element_values(const ElemArgs& A, int64_t e, ScalarVals<D, T>& out) {
  constexpr int NV = D + 1;
  int32_t v[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) v[a] = __ldg(A.me + (int64_t)a * A.nme + e);
  Geo<D, T> g;
  if constexpr (sizeof(T) == 8) geo_f64<D>(A.q, A.nq, v, g);
  else geo_f32<D>(A.qs, v, g);
  if (!det_ok(g.det)) {
    fe_report(A.st, FE_ERR_DEGENERATE, A.order[e]);
    g.det = T(1);
  }
  const T adet = g.det < T(0) ? -g.det : g.det;
  if constexpr (KIND == K_STIFF) {
    const T inv = load_coef<T>(A, e) * recip<T>(T(factorial(D)) * adet);
    // Gram matrix of c_1..c_D, scaled; row a = 0 from sum_a c_a = 0
    T G[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = i; j < D; ++j) {
        T s = g.c[i + 1][0] * g.c[j + 1][0];
#pragma unroll
        for (int k = 1; k < D; ++k) s += g.c[i + 1][k] * g.c[j + 1][k];
        G[i][j] = s * inv;
        G[j][i] = G[i][j];
      }
    T r[D];
    T r0 = T(0);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      T s = G[i][0];
#pragma unroll
      for (int j = 1; j < D; ++j) s += G[i][j];
      r[i] = s;
      r0 += s;
    }
    out.diag[0] = r0;
#pragma unroll
    for (int i = 0; i < D; ++i) out.diag[i + 1] = G[i][i];
#pragma unroll
    for (int p = 0; p < Pairs<D>::n; ++p) {
      const int a = Pairs<D>::a(p), b = Pairs<D>::b(p);
      out.off[p] = (a == 0) ? -r[b - 1] : G[a - 1][b - 1];
    }
  } else if constexpr (KIND == K_MASS || KIND == K_WMASS_P0) {
    T m = adet * T(1.0 / factorial(D + 2));
    if constexpr (KIND == K_WMASS_P0) m *= load_coef<T>(A, e);
#pragma unroll
    for (int a = 0; a < NV; ++a) out.diag[a] = T(2) * m;
#pragma unroll
    for (int p = 0; p < Pairs<D>::n; ++p) out.off[p] = m;
  } else {  // K_WMASS_P1
    const T* w = (const T*)A.w;
    T wv[NV];
    T ws = T(0);
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      wv[a] = w[v[a]];
      ws += wv[a];
    }
    const T base = adet * T(1.0 / factorial(D + 3));
#pragma unroll
    for (int a = 0; a < NV; ++a) out.diag[a] = T(2) * base * (ws + T(2) * wv[a]);
#pragma unroll
    for (int p = 0; p < Pairs<D>::n; ++p)
      out.off[p] = base * (ws + wv[Pairs<D>::a(p)] + wv[Pairs<D>::b(p)]);
  }
}

// accumulators: FP64 plain sum, FP32 compensated sum
template <class T>
struct Acc;
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ void add_partial(const void* p, int64_t i) { s += ((const double*)p)[i]; }
  __device__ __forceinline__ double value() const { return s; }
  __device__ __forceinline__ void store_partial(void* p, int64_t i) const { ((double*)p)[i] = s; }
};
template <>
struct Acc<float> {
  csum s;
  __device__ __forceinline__ void add(float x) { s.add(x); }
  __device__ __forceinline__ void add_partial(const void* p, int64_t i) {
    const float2 v = ((const float2*)p)[i];
    s.add2(v.x, v.y);
  }
  __device__ __forceinline__ float value() const { return s.value(); }
  __device__ __forceinline__ void store_partial(void* p, int64_t i) const {
    ((float2*)p)[i] = make_float2(s.s, s.c);
  }
};

// ---------------------------------------------------------------- FE_REASM_CHUNKED
// One block per chunk of internal elements. Phase 1: element values into shared
// memory (diagonal entries per corner, off-diagonal entries per local edge).
// Phase 2: each distinct vertex / edge of the chunk sums its incidences in
// ascending element order and stores the sum in the CSR value (both (i,j) and
// (j,i) for an edge: the operators are symmetric) or in its partial-sum slot.
template <int D, class T, int KIND, int THREADS>
__global__ void __launch_bounds__(THREADS) k_chunk_scalar(ElemArgs A, PlanArgs P, T* __restrict__ vals,
                                                          void* __restrict__ partials) {
  constexpr int NV = D + 1, NP = Pairs<D>::n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Kd = reinterpret_cast<T*>(smem_raw);
  T* Ko = Kd + (int64_t)P.chunk * NV;
  const int64_t c = blockIdx.x;
  const int64_t e0 = c * P.chunk;
  const int ne = (int)min((int64_t)P.chunk, A.nme - e0);
  for (int el = threadIdx.x; el < ne; el += THREADS) {
    ScalarVals<D, T> v;
    element_values<D, T, KIND>(A, e0 + el, v);
#pragma unroll
    for (int a = 0; a < NV; ++a) Kd[el * NV + a] = v.diag[a];
#pragma unroll
    for (int p = 0; p < NP; ++p) Ko[el * NP + p] = v.off[p];
  }
  __syncthreads();
  {
    const int32_t ub = P.ch_v_ptr[c], ue = P.ch_v_ptr[c + 1];
    const uint16_t* inc = P.inc_v + c * (int64_t)P.chunk * NV;
    for (int32_t u = ub + threadIdx.x; u < ue; u += THREADS) {
      const int s = P.lv_off[u];
      const int t = (u + 1 < ue) ? (int)P.lv_off[u + 1] : ne * NV;
      Acc<T> acc;
      for (int j = s; j < t; ++j) acc.add(Kd[inc[j]]);
      const int32_t dst = P.lv_dst[u];
      if (dst >= 0) vals[dst] = acc.value();
      else acc.store_partial(partials, -1 - (int64_t)dst);
    }
  }
  {
    const int32_t ub = P.ch_e_ptr[c], ue = P.ch_e_ptr[c + 1];
    const uint16_t* inc = P.inc_e + c * (int64_t)P.chunk * NP;
    for (int32_t u = ub + threadIdx.x; u < ue; u += THREADS) {
      const int s = P.le_off[u];
      const int t = (u + 1 < ue) ? (int)P.le_off[u + 1] : ne * NP;
      Acc<T> acc;
      for (int j = s; j < t; ++j) acc.add(Ko[inc[j] >> 1]);
      const int32_t dst = P.le_dst[2 * (int64_t)u];
      if (dst >= 0) {
        const T val = acc.value();
        vals[dst] = val;
        vals[P.le_dst[2 * (int64_t)u + 1]] = val;
      } else {
        acc.store_partial(partials, -1 - (int64_t)dst);
      }
    }
  }
}

// Sum of the chunk partials of each shared vertex / edge, in chunk order.
template <class T>
__global__ void k_fixup_scalar(const int32_t* __restrict__ sh_ptr, const int32_t* __restrict__ sh_dst,
                               int64_t nsh_v, int64_t nsh, const void* __restrict__ partials,
                               T* __restrict__ vals) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= nsh) return;
  Acc<T> acc;
  const int32_t s = sh_ptr[g], t = sh_ptr[g + 1];
  for (int32_t i = s; i < t; ++i) acc.add_partial(partials, i);
  const T val = acc.value();
  vals[sh_dst[2 * g]] = val;
  if (g >= nsh_v) vals[sh_dst[2 * g + 1]] = val;
}

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
  Acc<T> acc;
  const int32_t s = nsp[j], t = nsp[j + 1];
  for (int32_t i = s; i < t; ++i) acc.add(kg[n2s[i]]);
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

// FP32 form: split FP64 coordinates into (hi, lo) floats, one vertex per thread
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
