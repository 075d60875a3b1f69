// Per-element geometry and local matrices (device functions).
//
// Geometry (App. C.1 of the paper): B = [q^1 - q^0, ..., q^d - q^0]; the barycentric
// gradients are grad lambda_i = B^{-T} e_i (i >= 1) and grad lambda_0 = -sum_i grad
// lambda_i. Written with the cofactor vectors c_i (rows of adj(B)), grad lambda_i =
// c_i / det B, so every local matrix is a polynomial in c and 1/det:
//   stiffness (Eq. stiffelemmat): |K| g_a . g_b = (c_a . c_b) / (d! |det B|)
//   mass (Section 4.1, w = 1):    |K| d!/(d+2)! (1 + delta) = |det B| (1 + delta) / (d+2)!
//   P1 weighted mass (Eq. MatElemMassWP1): |det B| (1 + delta)(w^s + w_a + w_b) / (d+3)!
//   elasticity (Lemma lem:VecLocalElas): entry ((a,l),(b,n)) =
//       lam' c_a[l] c_b[n] + mu' (delta_ln c_a . c_b + c_b[l] c_a[n]),
//       lam' = lambda^s / (d! (d+1) |det B|), mu' likewise.
// FP64 form: everything in double. FP32 form: coordinates arrive split into
// (hi, lo) float pairs; edge vectors, cofactors and det B are formed in double-float
// arithmetic on the FP32 pipe (cofactors then rounded to float), values in float.
#pragma once

#include <stdint.h>

namespace fe {

// ---------------------------------------------------------------- double-float helpers
struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  s = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// a*b - c*d of floats as an unevaluated double-float sum: the products are exact
// (two-product by FMA), their difference is an exact two-sum plus the product
// errors; relative error about 2^-48 of the terms.
__device__ __forceinline__ df diff_of_products(float a, float b, float c, float d) {
  const float p = __fmul_rn(a, b), q = __fmul_rn(c, d);
  const float ep = __fmaf_rn(a, b, -p), eq = __fmaf_rn(c, d, -q);
  const df s = two_sum(p, -q);
  return {s.hi, __fadd_rn(s.lo, __fsub_rn(ep, eq))};
}

// Exact-ish split of a double into two floats: hi = x truncated to 24 significant
// bits, lo = the next 24 bits, so |x - hi - lo| < 2^-47 |x|. Integer operations
// only (the FP64 and conversion pipes are slow on this part). Inputs with
// |x| < 2^-100 are flushed to zero; |x| >= 2^128 gives an infinite hi.
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const int ex = (int)((b >> 52) & 0x7FF);
  const unsigned long long man = b & 0xFFFFFFFFFFFFFull;
  const int E = ex - 1023;
  if (ex == 0 || E < -100) { hi = 0.f; lo = 0.f; return; }
  if (E > 127) { hi = __int_as_float(sign | 0x7F800000u); lo = 0.f; return; }
  hi = __int_as_float(sign | ((unsigned int)(E + 127) << 23) | (unsigned int)(man >> 29));
  const unsigned int r = (unsigned int)(man & 0x1FFFFFFFull);
  if (r == 0u) { lo = 0.f; return; }
  const int lz = __clz(r);
  const int eo = (31 - lz) + E - 52 + 127;
  if (eo <= 0) { lo = 0.f; return; }
  lo = __int_as_float(sign | ((unsigned int)eo << 23) | ((r << (lz + 1)) >> 9));
}

// Compensated float accumulator (Kahan's summation): the value is s + c, where c
// carries the low-order part lost by each addition.
struct csum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = __fadd_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(y, __fsub_rn(t, s));
    s = t;
  }
  __device__ __forceinline__ void add2(float xs, float xc) {
    add(xs);
    c = __fadd_rn(c, xc);
  }
  __device__ __forceinline__ float value() const { return __fadd_rn(s, c); }
};

// ---------------------------------------------------------------- geometry
// Cofactor vectors c[a][i] for a = 1..D (c[0] = -sum_a c[a] is formed only where
// a kernel needs it) and det B.
template <int D, class T>
struct Geo {
  T c[D + 1][D];
  T det;      // FP64 form: det B; FP32 form: det B (double-float) rounded to float
  float dsc;  // FP32 form: error scale of the double-float det B (guard_geo_f32)
  bool full;  // FP32 form: badly shaped element, to be recomputed in FP64 (geo_exact_f32)
};

// Guard on the double-float det B of the FP32 and F64X forms. Taking each coordinate as
// a pair of floats moves it by less than 2^-47 |x|, so an edge by 2^-46 Xmax (Xmax the
// largest |coordinate| of the element) and det B by at most about 2^-41 Xmax Emax^(d-1)
// (Emax the largest |edge component|); the double-float products and sums of the rounded
// edges add less than that. Where |det B| < guard * Xmax Emax^(d-1) (a badly shaped element:
// a sliver, a needle, or an element far smaller than its distance from the origin) the
// kernels recompute det B in FP64 from the FP64 coordinates (det_from_q), whose edges
// carry an error of u |e| only, so det B and |K| keep FP64 relative accuracy.
// FP32 form: guard 2^-15, so a det B that is kept is within 2^-26 of its value.
constexpr float kDetGuardF32 = 1.0f / 32768.0f;
// F64X form (coordinates relative to the chunk's reference vertex): guard 2^-7, which
// well-shaped elements clear by a wide margin (a Kuhn tetrahedron with its vertices
// jittered by up to 0.15 h: |det B| / (Xmax Emax^2) above 0.01 in a chunk of diameter
// up to about 10 h).
constexpr float kDetGuardF64X = 1.0f / 128.0f;

template <int D>
__device__ __forceinline__ float abs_max(const float x[D + 1][D]) {
  float m = 0.f;
#pragma unroll
  for (int a = 0; a <= D; ++a)
#pragma unroll
    for (int k = 0; k < D; ++k) m = fmaxf(m, fabsf(x[a][k]));
  return m;
}

template <class T>
__device__ __forceinline__ void cofactors3(const T e[3][3], Geo<3, T>& g) {
  // c_1 = e_2 x e_3, c_2 = e_3 x e_1, c_3 = e_1 x e_2 (rows of adj(B), B = [e_1 e_2 e_3])
  const T* e1 = e[0]; const T* e2 = e[1]; const T* e3 = e[2];
  g.c[1][0] = e2[1] * e3[2] - e2[2] * e3[1];
  g.c[1][1] = e2[2] * e3[0] - e2[0] * e3[2];
  g.c[1][2] = e2[0] * e3[1] - e2[1] * e3[0];
  g.c[2][0] = e3[1] * e1[2] - e3[2] * e1[1];
  g.c[2][1] = e3[2] * e1[0] - e3[0] * e1[2];
  g.c[2][2] = e3[0] * e1[1] - e3[1] * e1[0];
  g.c[3][0] = e1[1] * e2[2] - e1[2] * e2[1];
  g.c[3][1] = e1[2] * e2[0] - e1[0] * e2[2];
  g.c[3][2] = e1[0] * e2[1] - e1[1] * e2[0];
}

template <class T>
__device__ __forceinline__ void cofactors2(const T e[2][2], Geo<2, T>& g) {
  // B = [e_1 e_2]; adj(B) rows: c_1 = (e_2y, -e_2x), c_2 = (-e_1y, e_1x)
  g.c[1][0] = e[1][1];
  g.c[1][1] = -e[1][0];
  g.c[2][0] = -e[0][1];
  g.c[2][1] = e[0][0];
}

template <int D, class T>
__device__ __forceinline__ void form_c0(Geo<D, T>& g) {
  if constexpr (sizeof(T) == 4) return;  // FP32: geo_f32 forms c_0 (accurately where it is small)
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T s = -g.c[1][i];
#pragma unroll
    for (int a = 2; a <= D; ++a) s -= g.c[a][i];
    g.c[0][i] = s;
  }
}

// FP32 form: c_0 = -sum_a c_a (set by geo_f32 with the other cofactors)
template <int D>
__device__ __forceinline__ void form_c0_float(Geo<D, float>& g) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
    float s = -g.c[1][i];
#pragma unroll
    for (int a = 2; a <= D; ++a) s -= g.c[a][i];
    g.c[0][i] = s;
  }
}

// smallest of the cofactors' largest |component|
template <int D>
__device__ __forceinline__ float min_cofactor(const Geo<D, float>& g) {
  float m = 3.4e38f;
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    float x = fabsf(g.c[a][0]);
#pragma unroll
    for (int k = 1; k < D; ++k) x = fmaxf(x, fabsf(g.c[a][k]));
    m = fminf(m, x);
  }
  return m;
}

// FP64 geometry from vertex coordinates x[a][c]
template <int D>
__device__ __forceinline__ void geo_f64(const double x[D + 1][D], Geo<D, double>& g) {
  double e[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int c = 0; c < D; ++c) e[i][c] = x[i + 1][c] - x[0][c];
  if constexpr (D == 3) {
    cofactors3(e, g);
    g.det = e[0][0] * g.c[1][0] + e[0][1] * g.c[1][1] + e[0][2] * g.c[1][2];
  } else {
    cofactors2(e, g);
    g.det = e[0][0] * e[1][1] - e[0][1] * e[1][0];
  }
}

// FP32 geometry from split coordinates (x = xh + xl): double-float edge vectors and
// det B (rounded to float in g.det), float cofactors c_0..c_D from the rounded edges
// (c_0 = -sum_a c_a), each component within about 3 2^-24 Emax^2 of its value.
// Where some cofactor is smaller than kShapeGuard Emax^2 in every component (a tiny
// face, a short edge or nearly parallel edges: needles and caps), that error would be
// large against the cofactor itself, and so would the split coordinates' error against
// a short edge: g.full is set, and the caller recomputes the element from the FP64
// coordinates (geo_exact_f32). COF = false (operators without gradients) skips that
// guard.
constexpr float kShapeGuard = 0.25f;

template <int D, bool COF = true>
__device__ __forceinline__ void geo_f32(const float xh[D + 1][D], const float xl[D + 1][D],
                                        Geo<D, float>& g) {
  df e[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const df s = two_sum(xh[i + 1][c], -xh[0][c]);
      e[i][c] = fast_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(xl[i + 1][c], xl[0][c])));
    }
  float eh[D][D];
  float emax = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      eh[i][c] = e[i][c].hi;
      emax = fmaxf(emax, fabsf(eh[i][c]));
    }
  g.dsc = abs_max<D>(xh) * (D == 3 ? emax * emax : emax);
  // det B = det(eh) + sum_i el_i . c_i + O(el^2): det(eh) in double-float from exact
  // products of the rounded edges, the low parts el against the float cofactors.
  if constexpr (D == 3) {
    cofactors3(eh, g);
    df cr[3];
    cr[0] = diff_of_products(eh[1][1], eh[2][2], eh[1][2], eh[2][1]);
    cr[1] = diff_of_products(eh[1][2], eh[2][0], eh[1][0], eh[2][2]);
    cr[2] = diff_of_products(eh[1][0], eh[2][1], eh[1][1], eh[2][0]);
    float p[3], lo = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      p[k] = __fmul_rn(eh[0][k], cr[k].hi);
      lo = __fadd_rn(lo, __fmaf_rn(eh[0][k], cr[k].lo, __fmaf_rn(eh[0][k], cr[k].hi, -p[k])));
    }
    df s = two_sum(p[0], p[1]);
    const df s2 = two_sum(s.hi, p[2]);
    lo = __fadd_rn(lo, __fadd_rn(s.lo, s2.lo));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) lo = __fmaf_rn(e[i][k].lo, g.c[i + 1][k], lo);
    g.det = __fadd_rn(s2.hi, lo);
  } else {
    cofactors2(eh, g);
    const df dh = diff_of_products(eh[0][0], eh[1][1], eh[0][1], eh[1][0]);
    float lo = dh.lo;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int k = 0; k < 2; ++k) lo = __fmaf_rn(e[i][k].lo, g.c[i + 1][k], lo);
    g.det = __fadd_rn(dh.hi, lo);
  }
  form_c0_float<D>(g);
  g.full = COF && min_cofactor<D>(g) < kShapeGuard * (D == 3 ? emax * emax : emax);
}

// Arguments and results of the out-of-line FP64 recomputations below are passed by
// value: an object whose address reaches a call that is not inlined has to live in local
// memory, and the caller's Geo would then be stored and reloaded for every element.
template <int D>
struct VertIds {
  int32_t v[D + 1];
};
template <int D>
struct GeoCof {
  float c[D + 1][D];
  float det;
};
template <int D>
__device__ __forceinline__ VertIds<D> vert_ids(const int32_t* v) {
  VertIds<D> r;
#pragma unroll
  for (int a = 0; a <= D; ++a) r.v[a] = v[a];
  return r;
}

// FP32 form, badly shaped element (g.full): det B and the cofactors recomputed in FP64
// from the FP64 coordinates of the element's vertices v (edges by one FP64 subtraction
// each, c_a = e_{a+1} x e_{a+2}, c_0 = -sum_a c_a, det B = e_1 . c_1), then rounded to
// float. Rare, so kept out of line.
template <int D>
__device__ __noinline__ GeoCof<D> geo_exact_f32(const double* __restrict__ q, int64_t nq, const VertIds<D> vi) {
  const int32_t* v = vi.v;
  double x0[D], e[D][D], c[D + 1][D];
#pragma unroll
  for (int k = 0; k < D; ++k) x0[k] = __ldg(q + (int64_t)k * nq + v[0]);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int k = 0; k < D; ++k) e[i][k] = __ldg(q + (int64_t)k * nq + v[i + 1]) - x0[k];
  double det;
  if constexpr (D == 3) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double* u = e[(i + 1) % 3];
      const double* w = e[(i + 2) % 3];
#pragma unroll
      for (int k = 0; k < 3; ++k) c[i + 1][k] = u[(k + 1) % 3] * w[(k + 2) % 3] - u[(k + 2) % 3] * w[(k + 1) % 3];
    }
    det = e[0][0] * c[1][0] + e[0][1] * c[1][1] + e[0][2] * c[1][2];
  } else {
    c[1][0] = e[1][1];
    c[1][1] = -e[1][0];
    c[2][0] = -e[0][1];
    c[2][1] = e[0][0];
    det = e[0][0] * e[1][1] - e[0][1] * e[1][0];
  }
#pragma unroll
  for (int k = 0; k < D; ++k) {
    double s = -c[1][k];
#pragma unroll
    for (int a = 2; a <= D; ++a) s -= c[a][k];
    c[0][k] = s;
  }
  GeoCof<D> g;
#pragma unroll
  for (int a = 0; a <= D; ++a)
#pragma unroll
    for (int k = 0; k < D; ++k) g.c[a][k] = (float)c[a][k];
  g.det = (float)det;
  return g;
}

// coordinates of the d+1 vertices gathered from global memory
template <int D>
__device__ __forceinline__ void load_x64(const double* __restrict__ q, int64_t nq, const int32_t v[D + 1],
                                         double x[D + 1][D]) {
#pragma unroll
  for (int a = 0; a <= D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) x[a][c] = __ldg(q + (int64_t)c * nq + v[a]);
}

// split coordinates gathered from the per-vertex float4 array of the FP32 form
template <int D>
__device__ __forceinline__ void load_x32(const float4* __restrict__ qs, const int32_t v[D + 1],
                                         float xh[D + 1][D], float xl[D + 1][D]) {
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    if constexpr (D == 3) {
      const float4 h = __ldg(qs + 2 * (int64_t)v[a]);
      const float4 l = __ldg(qs + 2 * (int64_t)v[a] + 1);
      xh[a][0] = h.x; xh[a][1] = h.y; xh[a][2] = h.z;
      xl[a][0] = l.x; xl[a][1] = l.y; xl[a][2] = l.z;
    } else {
      const float4 h = __ldg(qs + (int64_t)v[a]);
      xh[a][0] = h.x; xh[a][1] = h.y;
      xl[a][0] = h.z; xl[a][1] = h.w;
    }
  }
}

// det B in FP64 of the element with vertex ids v, from the FP64 coordinates q (d x nq):
// one FP64 subtraction per edge component, then the cofactor expansion along the first
// edge. Taken only for elements whose double-float det B fails its guard, so it is kept
// out of line.
template <int D>
__device__ __noinline__ double det_from_q(const double* __restrict__ q, int64_t nq, const VertIds<D> vi) {
  const int32_t* v = vi.v;
  double x0[D], e[D][D];
#pragma unroll
  for (int k = 0; k < D; ++k) x0[k] = __ldg(q + (int64_t)k * nq + v[0]);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int k = 0; k < D; ++k) e[i][k] = __ldg(q + (int64_t)k * nq + v[i + 1]) - x0[k];
  if constexpr (D == 3)
    return e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) + e[0][1] * (e[1][2] * e[2][0] - e[1][0] * e[2][2]) +
           e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
  else
    return e[0][0] * e[1][1] - e[0][1] * e[1][0];
}

// FP32 form: recompute a badly shaped element in FP64 (geo_exact_f32), or replace a
// double-float det B that fails its guard by the FP64 one
template <int D>
__device__ __forceinline__ void guard_geo_f32(Geo<D, float>& g, const double* __restrict__ q, int64_t nq,
                                              const int32_t* v) {
  if (g.full) {
    const GeoCof<D> r = geo_exact_f32<D>(q, nq, vert_ids<D>(v));
#pragma unroll
    for (int a = 0; a <= D; ++a)
#pragma unroll
      for (int k = 0; k < D; ++k) g.c[a][k] = r.c[a][k];
    g.det = r.det;
  } else if (fabsf(g.det) < kDetGuardF32 * g.dsc) {
    g.det = (float)det_from_q<D>(q, nq, vert_ids<D>(v));
  }
}

// det B usable: nonzero, normal and finite (checked on the exponent bits)
__device__ __forceinline__ bool det_ok(double det) {
  const unsigned int ex = ((unsigned int)__double2hiint(det) >> 20) & 0x7FFu;
  return ex != 0u && ex != 0x7FFu;
}
__device__ __forceinline__ bool det_ok(float det) {
  const unsigned int ex = ((unsigned int)__float_as_uint(det) >> 23) & 0xFFu;
  return ex != 0u && ex != 0xFFu;
}

__device__ __forceinline__ double tabs(double x) { return fabs(x); }
__device__ __forceinline__ float tabs(float x) { return fabsf(x); }

template <class T>
__device__ __forceinline__ T recip(T x);
// FP64 reciprocal: hardware approximation refined by two Newton-Raphson steps
// (r <- r + r (1 - x r), each step roughly doubling the correct bits); within a
// couple of ulps of 1/x for the normal, finite x the kernels pass (checked by
// the tests against CUDA's division).
template <>
__device__ __forceinline__ double recip<double>(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
template <>
__device__ __forceinline__ float recip<float>(float x) { return __frcp_rn(x); }

__host__ __device__ constexpr int factorial(int n) { return n <= 1 ? 1 : n * factorial(n - 1); }

// local pair numbering p = 0..npair-1 over a < b, lexicographic
template <int D>
struct Pairs;
template <>
struct Pairs<1> {
  static constexpr int n = 1;
  __device__ static constexpr int a(int) { return 0; }
  __device__ static constexpr int b(int) { return 1; }
};
template <>
struct Pairs<2> {
  static constexpr int n = 3;
  __device__ static constexpr int a(int p) { return p == 2 ? 1 : 0; }
  __device__ static constexpr int b(int p) { return p == 0 ? 1 : 2; }
};
template <>
struct Pairs<3> {
  static constexpr int n = 6;
  __device__ static constexpr int a(int p) { return p < 3 ? 0 : (p < 5 ? 1 : 2); }
  __device__ static constexpr int b(int p) { return p < 3 ? p + 1 : (p < 5 ? p - 1 : 3); }
};

}  // namespace fe
