// Double-float (pairs of floats, about 48 significant bits) arithmetic and the
// FP64-class geometry of the F64X forms, on top of the primitives of elem.cuh. On
// this part the FP32 pipe issues 64 times as many operations per clock as the FP64
// pipe, so FP64-class results are cheaper in double-float than in native FP64.
#pragma once

#include <stdint.h>

#include "elem.cuh"

namespace fe {

// Sum of two double-float numbers with one two-sum of the high parts: the error is
// about 2^-47 of |a| + |b| (not of |a + b|), which is the accuracy every sum of these
// kernels is judged by (entries are compared against the sum of the magnitudes of
// their contributions), at about half the operations of the fully accurate df_add.
__device__ __forceinline__ df df_add_fast(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

// double-float helpers on top of elem.cuh: products with the low parts, reciprocal
__device__ __forceinline__ df df_mul_full(df a, df b) {  // relative error ~2^-47
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add_fast(a, df_neg(b)); }
__device__ __forceinline__ df df_recip(df a) {  // one Newton step from the float reciprocal
  const float r = __frcp_rn(a.hi);
  // e = 1 - a r in double-float, then r (1 + e)
  const df ar = df_mul_full(a, df{r, 0.f});
  const df e = df_add(df{1.f, 0.f}, df_neg(ar));
  return df_add(df{r, 0.f}, df_mul_full(df{r, 0.f}, e));
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// double-float of a double constant, rounded at compile time
struct DfConst {
  float hi, lo;
};
constexpr DfConst df_const(double x) { return {(float)x, (float)(x - (double)(float)x)}; }
__device__ __forceinline__ df df_of(DfConst c) { return df{c.hi, c.lo}; }
__device__ __forceinline__ df df_twice(df a) { return df{2.f * a.hi, 2.f * a.lo}; }  // exact
__device__ __forceinline__ df df_split(double x) {
  float h, l;
  split_f64(x, h, l);
  return df{h, l};
}

// a*b - c*d for double-float operands: exact double-float of the high parts plus the
// first-order terms of the low parts
__device__ __forceinline__ df df_cross_term(df a, df b, df c, df d) {
  const df h = diff_of_products(a.hi, b.hi, c.hi, d.hi);
  float lo = h.lo;
  lo = __fmaf_rn(a.lo, b.hi, lo);
  lo = __fmaf_rn(a.hi, b.lo, lo);
  lo = __fmaf_rn(-c.lo, d.hi, lo);
  lo = __fmaf_rn(-c.hi, d.lo, lo);
  return fast_two_sum(h.hi, lo);
}

// x . y of double-float vectors: the products of the high parts exactly (FMA
// two-products) and summed by two-sums, every low-order term (the product errors, the
// cross terms with the low parts, the two-sum errors) in one float, one final
// normalisation; the error is about 2^-46 of sum |x_k y_k|.
template <int D>
__device__ __forceinline__ df df_dot(const df* x, const df* y) {
  float p[D], lo = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    p[k] = __fmul_rn(x[k].hi, y[k].hi);
    lo = __fadd_rn(lo, __fmaf_rn(x[k].hi, y[k].hi, -p[k]));
    lo = __fmaf_rn(x[k].hi, y[k].lo, lo);
    lo = __fmaf_rn(x[k].lo, y[k].hi, lo);
  }
  float s = p[0];
#pragma unroll
  for (int k = 1; k < D; ++k) {
    const df t = two_sum(s, p[k]);
    s = t.hi;
    lo = __fadd_rn(lo, t.lo);
  }
  return fast_two_sum(s, lo);
}

// Coordinates of global vertex vid relative to the reference point xr (FP64
// subtraction, so that large coordinate offsets cost no accuracy), split into
// (hi, lo) floats and stored at local slot u of sq: 3D as two float4 (hi, lo), 2D as
// one float4 (hi x, hi y, lo x, lo y).
template <int D>
__device__ __forceinline__ void x64_stage_vertex(const double* __restrict__ q, int64_t nq, int64_t vid,
                                                 const double* xr, unsigned char* sq, int u) {
  float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < D; ++k) split_f64(__ldg(q + k * nq + vid) - xr[k], h[k], l[k]);
  float4* xs = (float4*)sq + (D == 3 ? 2 : 1) * u;
  if constexpr (D == 3) {
    xs[0] = make_float4(h[0], h[1], h[2], 0.f);
    xs[1] = make_float4(l[0], l[1], l[2], 0.f);
  } else {
    xs[0] = make_float4(h[0], h[1], l[0], l[1]);
  }
}

// Cofactor vectors cf[i] = c_{i+1} (i < D) of B from its double-float edge vectors
// e[i] = x^{i+1} - x^0, and the signed det B (returned).
template <int D>
__device__ __forceinline__ df x64_cofactors(const df e[D][D], df cf[D][D]) {
  if constexpr (D == 3) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const df* u1 = e[(i + 1) % 3];
      const df* u2 = e[(i + 2) % 3];
      cf[i][0] = df_cross_term(u1[1], u2[2], u1[2], u2[1]);
      cf[i][1] = df_cross_term(u1[2], u2[0], u1[0], u2[2]);
      cf[i][2] = df_cross_term(u1[0], u2[1], u1[1], u2[0]);
    }
    return df_dot<3>(e[0], cf[0]);
  } else {
    cf[0][0] = e[1][1];
    cf[0][1] = df_neg(e[1][0]);
    cf[1][0] = df_neg(e[0][1]);
    cf[1][1] = e[0][0];
    return df_cross_term(e[0][0], e[1][1], e[0][1], e[1][0]);
  }
}

// Edge vectors e[i] = x^{i+1} - x^0 (i < NE) of the corners lv[0..NE] staged by
// x64_stage_vertex, as exact double-float differences of the split coordinates.
template <int D, int NE>
__device__ __forceinline__ void x64_edges(const unsigned char* sq, const int lv[NE + 1], df e[NE][D],
                                          float* xmax = nullptr) {
  constexpr int NV = NE + 1;
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
#pragma unroll
  for (int i = 0; i < NE; ++i)
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const df s = two_sum(xh[i + 1][k], -xh[0][k]);
      e[i][k] = fast_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(xl[i + 1][k], xl[0][k])));
    }
  if (xmax) {
    float m = 0.f;
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
      for (int k = 0; k < D; ++k) m = fmaxf(m, fabsf(xh[a][k]));
    *xmax = m;
  }
}

// square root of a positive double-float: one Newton step from the float root
__device__ __forceinline__ df df_sqrt(df a) {
  const float s = __fsqrt_rn(a.hi);
  const df r = df_add(a, df_neg(df_mul_full(df{s, 0.f}, df{s, 0.f})));  // a - s^2
  return fast_two_sum(s, __fmul_rn(r.hi, __fdividef(0.5f, s)));
}

// Double-float geometry of the element whose corners are the staged local vertices
// lv: the cofactor vectors cf[i] = c_{i+1} (i < D) of B = [x^1 - x^0, ...] and the
// signed det B (returned). Edge vectors are exact double-float differences.
template <int D>
__device__ __forceinline__ df x64_geometry(const unsigned char* sq, const int lv[D + 1], df cf[D][D]) {
  df e[D][D];
  x64_edges<D, D>(sq, lv, e);
  return x64_cofactors<D>(e, cf);
}

// x64_geometry with the det B guard of the F64X form (elem.cuh, kDetGuardF64X): a det B
// below the guard times Xmax Emax^(d-1) of the chunk-relative coordinates is recomputed in
// FP64 from q and the global ids lv_vid of the chunk's local vertices.
template <int D>
__device__ __forceinline__ df x64_geometry_guarded(const unsigned char* sq, const int lv[D + 1], df cf[D][D],
                                                   const double* __restrict__ q, int64_t nq,
                                                   const int32_t* lv_vid) {
  df e[D][D];
  float xm;
  x64_edges<D, D>(sq, lv, e, &xm);
  df det = x64_cofactors<D>(e, cf);
  float em = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int k = 0; k < D; ++k) em = fmaxf(em, fabsf(e[i][k].hi));
  if (fabsf(det.hi) < kDetGuardF64X * xm * (D == 3 ? em * em : em)) {
    int32_t v[D + 1];
#pragma unroll
    for (int a = 0; a <= D; ++a) v[a] = lv_vid[lv[a]];
    det = df_split(det_from_q<D>(q, nq, vert_ids<D>(v)));
  }
  return det;
}

// x64_geometry and the verdict of the same guard: exact = true where det B must be
// recomputed in FP64 (the caller does it)
template <int D>
__device__ __forceinline__ df x64_geometry_check(const unsigned char* sq, const int lv[D + 1], df cf[D][D],
                                                 bool& exact) {
  df e[D][D];
  float xm;
  x64_edges<D, D>(sq, lv, e, &xm);
  const df det = x64_cofactors<D>(e, cf);
  float em = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int k = 0; k < D; ++k) em = fmaxf(em, fabsf(e[i][k].hi));
  exact = fabsf(det.hi) < kDetGuardF64X * xm * (D == 3 ? em * em : em);
  return det;
}

// det B is zero or not finite (tested on its float rounding)
__device__ __forceinline__ bool df_degenerate(df det) {
  const float dh = __fadd_rn(det.hi, det.lo);
  const unsigned int ex = (__float_as_uint(dh) >> 23) & 0xFFu;
  return ex == 0u || ex == 0xFFu;
}

// Double-float number with the arithmetic operators, so that value code written as a
// template over the number type also runs in double-float. Built from a double only
// for constants (the split is folded at compile time); data arrives through df_split.
struct dfx {
  float hi, lo;
  dfx() = default;
  __host__ __device__ constexpr dfx(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr explicit dfx(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __device__ __forceinline__ dfx(df v) : hi(v.hi), lo(v.lo) {}
  __device__ __forceinline__ operator df() const { return df{hi, lo}; }
};
__device__ __forceinline__ dfx operator+(dfx a, dfx b) { return df_add_fast(a, b); }
__device__ __forceinline__ dfx operator-(dfx a, dfx b) { return df_add_fast(a, df_neg(b)); }
__device__ __forceinline__ dfx operator-(dfx a) { return dfx(-a.hi, -a.lo); }
__device__ __forceinline__ dfx operator*(dfx a, dfx b) { return df_mul_full(a, b); }
__device__ __forceinline__ dfx& operator+=(dfx& a, dfx b) { return a = a + b; }
__device__ __forceinline__ dfx& operator-=(dfx& a, dfx b) { return a = a - b; }
__device__ __forceinline__ dfx& operator*=(dfx& a, dfx b) { return a = a * b; }
__device__ __forceinline__ bool operator<(dfx a, dfx b) {  // normalised pairs
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ dfx tabs(dfx a) { return a.hi < 0.f ? -a : a; }
template <>
__device__ __forceinline__ dfx recip<dfx>(dfx x) { return df_recip(x); }

// value of a number type from a double datum: identity, float rounding, or the split
template <class T>
__device__ __forceinline__ T from_double(double x) { return T(x); }
template <>
__device__ __forceinline__ dfx from_double<dfx>(double x) { return df_split(x); }

// Double-float accumulator with the interface of the other forms' accumulators;
// partial sums are float2 (hi, lo), final values double.
struct AccX {
  df s;
  AccX() = default;
  __device__ __forceinline__ explicit AccX(df first) : s(first) {}
  __device__ __forceinline__ void add(df x) { s = df_add_fast(s, x); }
  __device__ __forceinline__ void add_prod(df x, df y) { s = df_add_fast(s, df_mul_full(x, y)); }
  __device__ __forceinline__ double value() const { return df_to_double(s); }
  __device__ __forceinline__ void store_partial(void* p, int64_t i) const {
    ((float2*)p)[i] = make_float2(s.hi, s.lo);
  }
  __device__ __forceinline__ static AccX from_partial(const void* p, int64_t i) {
    const float2 v = ((const float2*)p)[i];
    return AccX(df{v.x, v.y});
  }
  __device__ __forceinline__ void add_partial(const void* p, int64_t i) {
    const float2 v = ((const float2*)p)[i];
    add(df{v.x, v.y});
  }
  __device__ __forceinline__ void add_acc(const AccX& o) { add(o.s); }
};

}  // namespace fe
