// Backward pass of the stiffness assembly (the paper has no derivatives; the
// formulas follow from Eq. stiffelemmat and the geometry of App. C.1).
//
// For one element with per-element coefficient w, local stiffness
// S_ab = w |K| g_a . g_b and a weight matrix G^ (G^_ab multiplies S_ab in the loss):
//   L_e       = w |K| t,                     t = sum_ab G^_ab g_a . g_b
//   dL/dw_e   = |K| t
//   dL/dq^c   = w |K| [ t g_c - sum_x g_x (G^s Gamma)_xc ],  G^s = G^ + G^T,
//               Gamma_ab = g_a . g_b,
// the derivative of |det B| / d! and of g_a = B^{-T} g^_a with respect to the
// columns q^i - q^0 of B (the vertex-0 column is minus the sum of the others, which
// the same formula gives because sum_a g_a = 0). With cofactor vectors c_a = det B g_a
// everything is a polynomial in c scaled by 1/(d! |det B|) (and a sign for dq). The
// kernel evaluates it through the D x D matrix W = C^T (G^ + G^T) C: t = tr(W) / 2 and
// sum_x g_x (G^s Gamma)_xc = W c_c / det^2, so dL/dq^c = w / (d! det |det|) (t I - W) c_c.
// Two sources of G^:
//   rank one, G^_ab = u(me(a)) v(me(b)):  L = u^T S(w) v without forming any matrix;
//   general, G^_ab = dL/dS at the nonzero of slot (a, b) (a vector-Jacobian product
//   for any loss of the assembled values).
// Pass 1 (one thread per element) writes dL/dw and each corner's contribution to
// dL/dq; pass 2 (one thread per vertex) sums the contributions of its incidences in
// ascending element order, so the result is bit-identical run to run. The FE_F64X form
// evaluates the same formulas in double-float on the FP32 pipe.
#include "assemble_impl.cuh"
#include "dfloat.cuh"
#include "profile.cuh"

namespace fe {
namespace {

constexpr int BWD_THREADS = 256;

struct BwdArgs {
  const int32_t* me;
  int64_t nme, nq;
  const double* q;
  const float4* qs;
  const void* w;
  int w_kind;
  const int32_t* order;
  const void* u;          // rank one
  const void* v;
  const void* grad_vals;  // general
  const int32_t* slot2nnz;
  void* dLdw;             // may be null
  bool dLdw_internal;     // index dLdw by internal element (else input order)
  void* corner;           // nme * (d+1) * d contributions
  void* lpart;            // per-block L partial sums (rank one), may be null
  fe_status_word* st;
};

template <int D, class T, bool RANK1>
__global__ void __launch_bounds__(BWD_THREADS) k_bwd_elem(BwdArgs A) {
  constexpr int NV = D + 1;
  __shared__ T red[BWD_THREADS];
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  T Le = T(0);
  if (e < A.nme) {
    int32_t vv[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) vv[a] = __ldg(A.me + (int64_t)a * A.nme + e);
    Geo<D, T> g;
    if constexpr (sizeof(T) == 8) {
      double x[NV][D];
      load_x64<D>(A.q, A.nq, vv, x);
      geo_f64<D>(x, g);
    } else {
      float xh[NV][D], xl[NV][D];
      load_x32<D>(A.qs, vv, xh, xl);
      geo_f32<D>(xh, xl, g);
      guard_geo_f32<D>(g, A.q, A.nq, vv);
    }
    if (!det_ok(g.det)) {
      fe_report(A.st, FE_ERR_DEGENERATE, A.order[e]);
      g.det = T(1);
    }
    form_c0<D, T>(g);
    // W = C^T (G^ + G^T) C (D x D, C the NV x D matrix of cofactor vectors): then
    // t = sum_ab G^_ab c_a . c_b = tr(W) / 2, and the bracket of dL/dq^c is
    // t c_c - sum_x c_x (G^s Gamma)_xc = (t I - W) c_c.
    T W[D][D];
    if constexpr (RANK1) {
      // G^ = u v^T: W = ub vb^T + vb ub^T with ub = sum_a u_a c_a, vb = sum_a v_a c_a
      const T* u = (const T*)A.u;
      const T* v = (const T*)A.v;
      T ub[D], vb[D];
      {
        const T u0 = u[vv[0]], v0 = v[vv[0]];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          ub[k] = u0 * g.c[0][k];
          vb[k] = v0 * g.c[0][k];
        }
      }
#pragma unroll
      for (int a = 1; a < NV; ++a) {
        const T ua = u[vv[a]], va = v[vv[a]];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          ub[k] += ua * g.c[a][k];
          vb[k] += va * g.c[a][k];
        }
      }
#pragma unroll
      for (int k = 0; k < D; ++k)
#pragma unroll
        for (int j = k; j < D; ++j) {
          W[k][j] = ub[k] * vb[j] + vb[k] * ub[j];
          W[j][k] = W[k][j];
        }
    } else {
      const T* gv = (const T*)A.grad_vals;
      const int32_t* m = A.slot2nnz + e * NV * NV;
      T Gs[NV][NV];  // G^ + G^T, G^_ab = dL/dS at the nonzero of slot (row a, column b)
#pragma unroll
      for (int a = 0; a < NV; ++a)
#pragma unroll
        for (int b = a; b < NV; ++b) {
          Gs[a][b] = gv[m[b * NV + a]] + gv[m[a * NV + b]];
          Gs[b][a] = Gs[a][b];
        }
      T Pc[NV][D];  // (G^ + G^T) C
#pragma unroll
      for (int x = 0; x < NV; ++x)
#pragma unroll
        for (int j = 0; j < D; ++j) {
          T p = Gs[x][0] * g.c[0][j];
#pragma unroll
          for (int y = 1; y < NV; ++y) p += Gs[x][y] * g.c[y][j];
          Pc[x][j] = p;
        }
#pragma unroll
      for (int k = 0; k < D; ++k)
#pragma unroll
        for (int j = k; j < D; ++j) {
          T w = g.c[0][k] * Pc[0][j];
#pragma unroll
          for (int x = 1; x < NV; ++x) w += g.c[x][k] * Pc[x][j];
          W[k][j] = w;
          W[j][k] = w;
        }
    }
    T t = W[0][0];
#pragma unroll
    for (int k = 1; k < D; ++k) t += W[k][k];
    t *= T(0.5);
    const T adet = tabs(g.det);
    const T inv = recip<T>(T(factorial(D)) * adet);   // |K| / det^2 = 1 / (d! |det|)
    const bool has_w = A.w_kind != FE_COEF_NONE;
    const T w = has_w ? elem_coef<T>(A.w, A.w_kind, A.order, e) : T(1);
    const T dw = t * inv;
    if (A.dLdw) ((T*)A.dLdw)[A.dLdw_internal ? e : A.order[e]] = dw;
    Le = w * dw;
    const T s = w * inv * recip<T>(g.det);            // w |K| / det^3 = w / (d! det |det|)
    T Z[D][D];  // s (t I - W)
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
      for (int j = 0; j < D; ++j) Z[k][j] = s * ((k == j ? t : T(0)) - W[k][j]);
    T* out = (T*)A.corner + e * NV * D;
#pragma unroll
    for (int c = 0; c < NV; ++c)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        T o = Z[k][0] * g.c[c][0];
#pragma unroll
        for (int j = 1; j < D; ++j) o += Z[k][j] * g.c[c][j];
        out[c * D + k] = o;
      }
  }
  if (A.lpart) {  // fixed-order block reduction of L
    red[threadIdx.x] = Le;
    __syncthreads();
    for (int o = BWD_THREADS / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) ((T*)A.lpart)[blockIdx.x] = red[0];
  }
}

// dL/dq of each vertex: its corner contributions in ascending element order
template <int D, class T>
__global__ void k_bwd_vertex(const int32_t* __restrict__ ptr, const int32_t* __restrict__ inc,
                             int64_t nq, const T* __restrict__ corner, T* __restrict__ dLdq) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= nq) return;
  const int32_t s = ptr[v], t = ptr[v + 1];
  if (s == t) {  // a vertex no element uses
#pragma unroll
    for (int k = 0; k < D; ++k) dLdq[k * nq + v] = T(0);
    return;
  }
  // one pass over the incidences, all D components of each corner together
  Acc<T> a[D];
  {
    const T* c0 = corner + (int64_t)inc[s] * D;
#pragma unroll
    for (int k = 0; k < D; ++k) a[k] = Acc<T>(c0[k]);
  }
  for (int32_t j = s + 1; j < t; ++j) {
    const T* cj = corner + (int64_t)inc[j] * D;
#pragma unroll
    for (int k = 0; k < D; ++k) a[k].add(cj[k]);
  }
#pragma unroll
  for (int k = 0; k < D; ++k) dLdq[k * nq + v] = a[k].value();
}

// L = sum of the block partials, in block order (one block)
template <class T>
__global__ void k_bwd_lsum(const T* __restrict__ part, int64_t n, T* __restrict__ L) {
  __shared__ T red[256];
  T s = T(0);
  for (int64_t i = threadIdx.x; i < n; i += 256) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *L = red[0];
}

template <int D, class T>
int launch(fe_pattern_s* h, BwdArgs& A, bool rank1, void* L, void* dLdq, cudaStream_t s) {
  const int nblk = fe_grid(h->nme, BWD_THREADS);
  FE_PROF_BEGIN(h, FE_K_BWD_CHUNK, s);
  if (rank1) k_bwd_elem<D, T, true><<<nblk, BWD_THREADS, 0, s>>>(A);
  else k_bwd_elem<D, T, false><<<nblk, BWD_THREADS, 0, s>>>(A);
  FE_CUDA_TRY(cudaGetLastError());
  FE_PROF_END(h, FE_K_BWD_CHUNK, s);
  if (dLdq) {
    FE_PROF_BEGIN(h, FE_K_BWD_REDUCE, s);
    k_bwd_vertex<D, T><<<fe_grid(h->nq, 256), 256, 0, s>>>(h->vmap_ptr, h->vmap, h->nq, (const T*)A.corner,
                                                          (T*)dLdq);
    FE_CUDA_TRY(cudaGetLastError());
    FE_PROF_END(h, FE_K_BWD_REDUCE, s);
  }
  if (L && A.lpart) {
    k_bwd_lsum<T><<<1, 256, 0, s>>>((const T*)A.lpart, nblk, (T*)L);
    FE_CUDA_TRY(cudaGetLastError());
  }
  return FE_OK;
}

// ---------------------------------------------------------------- FE_F64X form
// Pass 1 in double-float: edge vectors from an FP64 subtraction of the corner
// coordinates, split into float pairs; cofactors, W, t and the corner contributions in
// double-float; dL/dw and L in double, the corner contributions as float2 pairs.
template <int D, bool RANK1>
__global__ void __launch_bounds__(BWD_THREADS) k_bwd_elem_x(BwdArgs A) {
  constexpr int NV = D + 1;
  __shared__ double red[BWD_THREADS];
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double Le = 0.0;
  if (e < A.nme) {
    int32_t vv[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) vv[a] = __ldg(A.me + (int64_t)a * A.nme + e);
    double x[NV][D];
    load_x64<D>(A.q, A.nq, vv, x);
    df ed[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int k = 0; k < D; ++k) ed[i][k] = df_split(x[i + 1][k] - x[0][k]);
    df c[NV][D];
    df det = x64_cofactors<D>(ed, &c[1]);
    if (df_degenerate(det)) {
      fe_report(A.st, FE_ERR_DEGENERATE, A.order[e]);
      det = df{1.f, 0.f};
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      df s = c[1][k];
#pragma unroll
      for (int a = 2; a < NV; ++a) s = df_add_fast(s, c[a][k]);
      c[0][k] = df_neg(s);
    }
    df W[D][D];  // C^T (G^ + G^T) C
    if constexpr (RANK1) {
      const double* u = (const double*)A.u;
      const double* v = (const double*)A.v;
      df ub[D], vb[D];
      {
        const df u0 = df_split(u[vv[0]]), v0 = df_split(v[vv[0]]);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          ub[k] = df_mul_full(u0, c[0][k]);
          vb[k] = df_mul_full(v0, c[0][k]);
        }
      }
#pragma unroll
      for (int a = 1; a < NV; ++a) {
        const df ua = df_split(u[vv[a]]), va = df_split(v[vv[a]]);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          ub[k] = df_add_fast(ub[k], df_mul_full(ua, c[a][k]));
          vb[k] = df_add_fast(vb[k], df_mul_full(va, c[a][k]));
        }
      }
#pragma unroll
      for (int k = 0; k < D; ++k)
#pragma unroll
        for (int j = k; j < D; ++j) {
          W[k][j] = df_add_fast(df_mul_full(ub[k], vb[j]), df_mul_full(vb[k], ub[j]));
          W[j][k] = W[k][j];
        }
    } else {
      const double* gv = (const double*)A.grad_vals;
      const int32_t* m = A.slot2nnz + e * NV * NV;
      df Gs[NV][NV];
#pragma unroll
      for (int a = 0; a < NV; ++a)
#pragma unroll
        for (int b = a; b < NV; ++b) {
          Gs[a][b] = df_add_fast(df_split(gv[m[b * NV + a]]), df_split(gv[m[a * NV + b]]));
          Gs[b][a] = Gs[a][b];
        }
      df Pc[NV][D];
#pragma unroll
      for (int xx = 0; xx < NV; ++xx)
#pragma unroll
        for (int j = 0; j < D; ++j) {
          df p = df_mul_full(Gs[xx][0], c[0][j]);
#pragma unroll
          for (int y = 1; y < NV; ++y) p = df_add_fast(p, df_mul_full(Gs[xx][y], c[y][j]));
          Pc[xx][j] = p;
        }
#pragma unroll
      for (int k = 0; k < D; ++k)
#pragma unroll
        for (int j = k; j < D; ++j) {
          df w = df_mul_full(c[0][k], Pc[0][j]);
#pragma unroll
          for (int xx = 1; xx < NV; ++xx) w = df_add_fast(w, df_mul_full(c[xx][k], Pc[xx][j]));
          W[k][j] = w;
          W[j][k] = w;
        }
    }
    df t = W[0][0];
#pragma unroll
    for (int k = 1; k < D; ++k) t = df_add_fast(t, W[k][k]);
    t = df{0.5f * t.hi, 0.5f * t.lo};  // exact
    const df adet = det.hi < 0.f ? df_neg(det) : det;
    const df inv = df_recip(df_mul_full(adet, df{(float)factorial(D), 0.f}));  // 1 / (d! |det|)
    const bool has_w = A.w_kind != FE_COEF_NONE;
    const df w = has_w ? df_split(elem_coef<double>(A.w, A.w_kind, A.order, e)) : df{1.f, 0.f};
    const df dw = df_mul_full(t, inv);
    if (A.dLdw) ((double*)A.dLdw)[A.dLdw_internal ? e : A.order[e]] = df_to_double(dw);
    Le = df_to_double(df_mul_full(w, dw));
    const df s = df_mul_full(df_mul_full(w, inv), df_recip(det));  // w / (d! det |det|)
    df Z[D][D];  // s (t I - W)
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
      for (int j = 0; j < D; ++j) Z[k][j] = df_mul_full(s, k == j ? df_add_fast(t, df_neg(W[k][j])) : df_neg(W[k][j]));
    float2* out = (float2*)A.corner + e * NV * D;
#pragma unroll
    for (int cc = 0; cc < NV; ++cc)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        df o = df_mul_full(Z[k][0], c[cc][0]);
#pragma unroll
        for (int j = 1; j < D; ++j) o = df_add_fast(o, df_mul_full(Z[k][j], c[cc][j]));
        out[cc * D + k] = make_float2(o.hi, o.lo);
      }
  }
  if (A.lpart) {  // fixed-order block reduction of L
    red[threadIdx.x] = Le;
    __syncthreads();
    for (int o = BWD_THREADS / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) ((double*)A.lpart)[blockIdx.x] = red[0];
  }
}

// pass 2 of the F64X form: double-float sums of the float2 corner contributions
template <int D>
__global__ void k_bwd_vertex_x(const int32_t* __restrict__ ptr, const int32_t* __restrict__ inc,
                               int64_t nq, const float2* __restrict__ corner, double* __restrict__ dLdq) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= nq) return;
  const int32_t s = ptr[v], t = ptr[v + 1];
  if (s == t) {
#pragma unroll
    for (int k = 0; k < D; ++k) dLdq[k * nq + v] = 0.0;
    return;
  }
  AccX a[D];
#pragma unroll
  for (int k = 0; k < D; ++k) a[k] = AccX::from_partial(corner, (int64_t)inc[s] * D + k);
  for (int32_t j = s + 1; j < t; ++j)
#pragma unroll
    for (int k = 0; k < D; ++k) a[k].add_partial(corner, (int64_t)inc[j] * D + k);
#pragma unroll
  for (int k = 0; k < D; ++k) dLdq[k * nq + v] = a[k].value();
}

template <int D>
int launch_x(fe_pattern_s* h, BwdArgs& A, bool rank1, void* L, void* dLdq, cudaStream_t s) {
  const int nblk = fe_grid(h->nme, BWD_THREADS);
  FE_PROF_BEGIN(h, FE_K_BWD_CHUNK, s);
  if (rank1) k_bwd_elem_x<D, true><<<nblk, BWD_THREADS, 0, s>>>(A);
  else k_bwd_elem_x<D, false><<<nblk, BWD_THREADS, 0, s>>>(A);
  FE_CUDA_TRY(cudaGetLastError());
  FE_PROF_END(h, FE_K_BWD_CHUNK, s);
  if (dLdq) {
    FE_PROF_BEGIN(h, FE_K_BWD_REDUCE, s);
    k_bwd_vertex_x<D><<<fe_grid(h->nq, 256), 256, 0, s>>>(h->vmap_ptr, h->vmap, h->nq, (const float2*)A.corner,
                                                         (double*)dLdq);
    FE_CUDA_TRY(cudaGetLastError());
    FE_PROF_END(h, FE_K_BWD_REDUCE, s);
  }
  if (L && A.lpart) {
    k_bwd_lsum<double><<<1, 256, 0, s>>>((const double*)A.lpart, nblk, (double*)L);
    FE_CUDA_TRY(cudaGetLastError());
  }
  return FE_OK;
}

int prepare(fe_pattern_s* h, cudaStream_t s) {
  if (!h->vmap_ptr) FE_TRY(fe_build_vertex_map(h, s));
  if (!h->bwd_scratch) {
    FE_TRY(fe_malloc(h, &h->bwd_scratch, sizeof(double) * (size_t)h->nme * h->nv * h->d));
    FE_TRY(fe_malloc(h, &h->bwd_lpart, sizeof(double) * (size_t)fe_grid(h->nme, BWD_THREADS)));
  }
  return FE_OK;
}

int run(fe_pattern_s* h, const double* q, const void* w, int w_kind, const void* u, const void* v,
        const void* grad_vals, void* L, void* dLdw, void* dLdq, int prec, cudaStream_t s) {
  FE_TRY(prepare(h, s));
  BwdArgs A{h->me_int, h->nme, h->nq, q, nullptr, w, w_kind, h->order, u, v, grad_vals, h->slot2nnz,
            dLdw, w_kind == FE_COEF_P0_INTERNAL, h->bwd_scratch, L ? h->bwd_lpart : nullptr, h->status};
  const bool rank1 = grad_vals == nullptr;
  if (prec == FE_F64X) return h->d == 3 ? launch_x<3>(h, A, rank1, L, dLdq, s) : launch_x<2>(h, A, rank1, L, dLdq, s);
  if (prec == FE_F32) {
    float4* qs = (float4*)h->qsplit;
    if (h->d == 3) k_split_q<3><<<fe_grid(h->nq, 256), 256, 0, s>>>(q, h->nq, qs);
    else k_split_q<2><<<fe_grid(h->nq, 256), 256, 0, s>>>(q, h->nq, qs);
    FE_CUDA_TRY(cudaGetLastError());
    A.qs = qs;
    return h->d == 3 ? launch<3, float>(h, A, rank1, L, dLdq, s) : launch<2, float>(h, A, rank1, L, dLdq, s);
  }
  return h->d == 3 ? launch<3, double>(h, A, rank1, L, dLdq, s) : launch<2, double>(h, A, rank1, L, dLdq, s);
}

}  // namespace
}  // namespace fe

int fe_launch_backward(fe_pattern_s* h, const double* q, const void* w, int w_kind, const void* u,
                       const void* v, void* L, void* dLdw, void* dLdq, int prec, cudaStream_t s) {
  return fe::run(h, q, w, w_kind, u, v, nullptr, L, dLdw, dLdq, prec, s);
}

int fe_launch_vjp(fe_pattern_s* h, const double* q, const void* w, int w_kind, const void* grad_vals,
                  void* dLdw, void* dLdq, int prec, cudaStream_t s) {
  return fe::run(h, q, w, w_kind, nullptr, nullptr, grad_vals, nullptr, dLdw, dLdq, prec, s);
}
