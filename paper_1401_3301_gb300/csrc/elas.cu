// Linear elasticity (Section 5.1 of the paper): the m = d vector problem with the
// isotropic Hooke law, reassembled into the m x m block CSR of the pattern.
//
// Local matrix (Lemma lem:VecLocalElas, App. B, with the P1 interpolants of the
// Lame fields): for vertices a, b and components l, n,
//   K_{(a,l),(b,n)} = |K|/(d+1) (lambda^s g_b[n] g_a[l] + mu^s (delta_ln g_a . g_b + g_b[l] g_a[n]))
// With g_a = c_a / det B (cofactor vectors) this is
//   lp c_a[l] c_b[n] + mp (delta_ln c_a . c_b + c_b[l] c_a[n]),
//   lp = lambda^s / (d! (d+1) |det B|), mp = mu^s / (d! (d+1) |det B|).
// The kernel keeps, per element, the cofactor vectors and (lp, mp) in shared
// memory and forms each 3x3 (2x2) block while summing the incidences of a chunk's
// vertices (diagonal blocks) and edges (off-diagonal blocks, written at (i,j) and,
// transposed, at (j,i)), in ascending element order.
#include "assemble_impl.cuh"
#include "dfloat.cuh"
#include "profile.cuh"

namespace fe {
namespace {

struct ElasArgs {
  int64_t nme, nq;
  int chunk;
  uint32_t rec_max, max_lv;
  const double* q;
  const void* lam;
  int lam_kind;
  const void* mu;
  int mu_kind;
  const int32_t* order;
  const int32_t* ch_v_ptr;
  const int32_t* ch_e_ptr;
  const uint8_t* rec;
  const uint32_t* rec_off16;
  fe_status_word* st;
  int64_t nnz, npart;  // sizes of vals and of the partial blocks (bounds-checked builds)
  const int32_t* me0;  // F64X form: corner 0 of each internal element (chunk reference vertex)
};

// sum over the element's vertices of a coefficient's P1 values (lambda^s, mu^s)
template <int D, class T>
__device__ __forceinline__ T coef_sum(const void* c, int kind, const int32_t* order, int64_t e,
                                      const T* local_p1, const int lv[D + 1]) {
  const T* cp = (const T*)c;
  if (kind == FE_COEF_P1) {
    T s = local_p1[lv[0]];
#pragma unroll
    for (int a = 1; a <= D; ++a) s += local_p1[lv[a]];
    return s;
  }
  T v;
  if (kind == FE_COEF_SCALAR) v = cp[0];
  else if (kind == FE_COEF_P0) v = cp[order[e]];
  else v = cp[e];
  return T(D + 1) * v;
}

// block (a, a) of one element from x = c_a: (lp + mp) x x^T + mp |x|^2 I
template <int D, class T>
__device__ __forceinline__ void diag_block(const T* x, T lp, T mp, T* blk) {
  T xx = x[0] * x[0];
#pragma unroll
  for (int i = 1; i < D; ++i) xx += x[i] * x[i];
  const T lm = lp + mp, mxx = mp * xx;
#pragma unroll
  for (int l = 0; l < D; ++l)
#pragma unroll
    for (int n = 0; n < D; ++n) blk[l * D + n] = lm * x[l] * x[n] + (l == n ? mxx : T(0));
}

// block (a, b) of one element from x = c_a, y = c_b: entry (l, n) =
// lp x_l y_n + mp (y_l x_n + delta_ln x . y)
template <int D, class T>
__device__ __forceinline__ void edge_block(const T* x, const T* y, T lp, T mp, T* blk) {
  T xy = x[0] * y[0];
#pragma unroll
  for (int i = 1; i < D; ++i) xy += x[i] * y[i];
  const T mxy = mp * xy;
#pragma unroll
  for (int l = 0; l < D; ++l)
#pragma unroll
    for (int n = 0; n < D; ++n) blk[l * D + n] = lp * x[l] * y[n] + mp * y[l] * x[n] + (l == n ? mxy : T(0));
}

template <int D, class T, int THREADS>
__global__ void __launch_bounds__(THREADS) k_chunk_elas(ElasArgs A, T* __restrict__ vals,
                                                        void* __restrict__ partials) {
  constexpr int NV = D + 1, NP = Pairs<D>::n, MM = D * D;
  // FP64: the block entries go straight into the accumulators by FMA (about half the
  // FP64 operations of forming each 3 x 3 block first); FP32 forms the block and adds it
  // to its compensated sums
  constexpr bool FUSED = sizeof(T) == 8;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  const int64_t c = blockIdx.x;
  const int64_t e0 = c * A.chunk;
  const int ne = (int)min((int64_t)A.chunk, A.nme - e0);
  const int32_t nlv = A.ch_v_ptr[c + 1] - A.ch_v_ptr[c];
  const int32_t nle = A.ch_e_ptr[c + 1] - A.ch_e_ptr[c];
  const RecLayout R = rec_layout((uint32_t)ne, NV, NP, (uint32_t)nlv, (uint32_t)nle, true);
  const ElasSmem S = elas_smem(D, (int)sizeof(T), A.rec_max, A.max_lv, A.chunk);
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
  const uint16_t* lv_str = (const uint16_t*)(smem + R.lv_str);
  const uint16_t* le_str = (const uint16_t*)(smem + R.le_str);
  const uint16_t* lvid = (const uint16_t*)(smem + R.lvid);
  T* lam_l = (T*)(smem + S.coef);
  T* mu_l = lam_l + A.max_lv;
  T* Cg = (T*)(smem + S.cg);   // [e][a][i]
  T* LM = (T*)(smem + S.lm);   // [e][2]
  if (!FE_RECORD_VALID(smem, R, ne, NV, NP, nlv, nle, D, A.nq, A.nnz, A.npart, A.st, c)) return;

  // 0. coordinates (and P1 Lame values) of the chunk's vertices
  for (int u = threadIdx.x; u < nlv; u += THREADS) {
    const int64_t vid = lv_vid[u];
    stage_vertex<D, T>(A.q, A.nq, vid, smem + S.q, u, xr.ptr());
    if (A.lam_kind == FE_COEF_P1) lam_l[u] = ((const T*)A.lam)[vid];
    if (A.mu_kind == FE_COEF_P1) mu_l[u] = ((const T*)A.mu)[vid];
  }
  __syncthreads();

  // 1. cofactor vectors and scaled Lame sums of every element
  for (int el = threadIdx.x; el < ne; el += THREADS) {
    int lv[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) lv[a] = lvid[el * NV + a];
    Geo<D, T> g;
    staged_geo<D, T>(smem + S.q, lv, g, A.q, A.nq, lv_vid);
    if (!det_ok(g.det)) {
      fe_report(A.st, FE_ERR_DEGENERATE, A.order[e0 + el]);
      g.det = T(1);
    }
    form_c0<D, T>(g);
    const T scale = recip<T>(T(factorial(D) * (D + 1)) * tabs(g.det));
    const T ls = coef_sum<D, T>(A.lam, A.lam_kind, A.order, e0 + el, lam_l, lv);
    const T ms = coef_sum<D, T>(A.mu, A.mu_kind, A.order, e0 + el, mu_l, lv);
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
      for (int i = 0; i < D; ++i) Cg[(el * NV + a) * D + i] = g.c[a][i];
    LM[2 * el] = ls * scale;
    LM[2 * el + 1] = ms * scale;
  }
  __syncthreads();

  // 2a. diagonal blocks: sum over (element, corner) incidences of each vertex
  for (int u = threadIdx.x; u < nlv; u += THREADS) {
    const int s = lv_off[u], t = lv_off[u + 1];
    Acc<T> acc[MM];
    for (int j = s; j < t; ++j) {
      const int inc = inc_v[j];
      const int el = inc / NV;
      if constexpr (FUSED) {
        // (lp + mp) x x^T + mp |x|^2 I, FMA'd straight into the accumulators
        const T* x = Cg + inc * D;
        const T lp = LM[2 * el], mp = LM[2 * el + 1], lm = lp + mp;
        T xx = x[0] * x[0];
#pragma unroll
        for (int i = 1; i < D; ++i) xx = fma(x[i], x[i], xx);
        const T mxx = mp * xx;
#pragma unroll
        for (int l = 0; l < D; ++l) {
          const T lx = lm * x[l];
#pragma unroll
          for (int n = 0; n < D; ++n) {
            if (j == s) acc[l * D + n] = Acc<T>(lx * x[n]);
            else acc[l * D + n].add_scaled(lx, x[n]);
          }
          acc[l * D + l].add(mxx);
        }
      } else {
        T blk[MM];
        diag_block<D, T>(Cg + inc * D, LM[2 * el], LM[2 * el + 1], blk);
#pragma unroll
        for (int k = 0; k < MM; ++k) {
          if (j == s) acc[k] = Acc<T>(blk[k]);
          else acc[k].add(blk[k]);
        }
      }
    }
    const int32_t dst = lv_dst[u];
    if (dst >= 0) {
      const int str = lv_str[u];
#pragma unroll
      for (int l = 0; l < D; ++l)
#pragma unroll
        for (int n = 0; n < D; ++n) vals[dst + l * str + n] = acc[l * D + n].value();
    } else {
      const int64_t pi = (-1 - (int64_t)dst) * MM;
#pragma unroll
      for (int k = 0; k < MM; ++k) acc[k].store_partial(partials, pi + k);
    }
  }
  // 2b. off-diagonal blocks: (element, pair) incidences of each edge, oriented (vmin, vmax)
  for (int u = threadIdx.x; u < nle; u += THREADS) {
    const int s = le_off[u], t = le_off[u + 1];
    Acc<T> acc[MM];
    for (int j = s; j < t; ++j) {
      const int code = inc_e[j];
      const int ep = code >> 1;
      const int el = ep / NP, p = ep - el * NP;
      int a = Pairs<D>::a(p), b = Pairs<D>::b(p);
      if (code & 1) {  // me(a) > me(b): the (vmin, vmax) block is block (b, a)
        const int t2 = a; a = b; b = t2;
      }
      if constexpr (FUSED) {
        // lp x_l y_n + mp y_l x_n + delta_ln mp x.y, FMA'd straight into the accumulators
        const T* x = Cg + (el * NV + a) * D;
        const T* y = Cg + (el * NV + b) * D;
        const T lp = LM[2 * el], mp = LM[2 * el + 1];
        T px[D], qy[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          px[i] = lp * x[i];
          qy[i] = mp * y[i];
        }
        T mxy = qy[0] * x[0];
#pragma unroll
        for (int i = 1; i < D; ++i) mxy = fma(qy[i], x[i], mxy);
#pragma unroll
        for (int l = 0; l < D; ++l) {
#pragma unroll
          for (int n = 0; n < D; ++n) {
            if (j == s) acc[l * D + n] = Acc<T>(px[l] * y[n]);
            else acc[l * D + n].add_scaled(px[l], y[n]);
            acc[l * D + n].add_scaled(qy[l], x[n]);
          }
          acc[l * D + l].add(mxy);
        }
      } else {
        T blk[MM];
        edge_block<D, T>(Cg + (el * NV + a) * D, Cg + (el * NV + b) * D, LM[2 * el], LM[2 * el + 1], blk);
#pragma unroll
        for (int k = 0; k < MM; ++k) {
          if (j == s) acc[k] = Acc<T>(blk[k]);
          else acc[k].add(blk[k]);
        }
      }
    }
    const int32_t dst = le_dst[2 * u];
    if (dst >= 0) {
      const int32_t dst_t = le_dst[2 * u + 1];
      const int str = le_str[2 * u], str_t = le_str[2 * u + 1];
#pragma unroll
      for (int l = 0; l < D; ++l)
#pragma unroll
        for (int n = 0; n < D; ++n) {
          const T v = acc[l * D + n].value();
          vals[dst + l * str + n] = v;
          vals[dst_t + n * str_t + l] = v;
        }
    } else {
      const int64_t pi = (-1 - (int64_t)dst) * MM;
#pragma unroll
      for (int k = 0; k < MM; ++k) acc[k].store_partial(partials, pi + k);
    }
  }
}

// Sum, in chunk order, of the partial blocks of each shared vertex / edge: one thread per
// (entity, block entry), so that neighbouring threads read neighbouring words of the
// partial blocks (partial i of the entity holds its m x m block at i * MM).
template <int D, class T, class AccT = Acc<T>>
__global__ void k_fixup_elas(const int32_t* __restrict__ sh_ptr, const int32_t* __restrict__ sh_dst,
                             const int32_t* __restrict__ sh_str, int64_t nsh_v, int64_t nsh,
                             const void* __restrict__ partials, T* __restrict__ vals, int64_t nnz,
                             int64_t npart, fe_status_word* st) {
  constexpr int MM = D * D;
  const int64_t gk = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gk >= nsh * MM) return;
  const int64_t g = gk / MM;
  const int k = (int)(gk - g * MM);
  const int32_t s = sh_ptr[g], t = sh_ptr[g + 1];
  if (!FE_FIXUP_VALID(s, t, npart, (int64_t)sh_dst[2 * g] + (k / D) * sh_str[2 * g] + k % D,
                      (int64_t)sh_dst[2 * g + 1] + (k % D) * sh_str[2 * g + 1] + k / D, g >= nsh_v, nnz, st, g))
    return;
  AccT acc = AccT::from_partial(partials, (int64_t)s * MM + k);
  for (int32_t i = s + 1; i < t; ++i) acc.add_partial(partials, (int64_t)i * MM + k);
  const T v = acc.value();
  const int l = k / D, n = k % D;
  vals[sh_dst[2 * g] + l * sh_str[2 * g] + n] = v;
  if (g >= nsh_v) vals[sh_dst[2 * g + 1] + n * sh_str[2 * g + 1] + l] = v;
}

template <int D, class T>
int launch(fe_pattern_s* h, const ElasArgs& A, T* vals, cudaStream_t s) {
  constexpr int THREADS = 256;
  const ElasSmem L = elas_smem(D, (int)sizeof(T), A.rec_max, A.max_lv, A.chunk);
  if (L.total > kSmemDynMax) return FE_ERR_ARG;
  auto kern = k_chunk_elas<D, T, THREADS>;
  FE_TRY(fe_smem_limit(kern, L.total));
  FE_PROF_BEGIN(h, FE_K_ELAS_CHUNK, s);
  kern<<<(unsigned)h->nchunks, THREADS, L.total, s>>>(A, vals, h->partials);
  FE_CUDA_TRY(cudaGetLastError());
  FE_PROF_END(h, FE_K_ELAS_CHUNK, s);
  const int64_t nsh = h->nsh_v + h->nsh_e;
  if (nsh > 0) {
    FE_PROF_BEGIN(h, FE_K_ELAS_FIXUP, s);
    k_fixup_elas<D, T><<<fe_grid(nsh * D * D, 256), 256, 0, s>>>(h->sh_ptr, h->sh_dst, h->sh_str, h->nsh_v,
                                                                 nsh, h->partials, vals, h->nnz, h->npart,
                                                                 h->status);
    FE_CUDA_TRY(cudaGetLastError());
    FE_PROF_END(h, FE_K_ELAS_FIXUP, s);
  }
  return FE_OK;
}


// ---------------------------------------------------------------- FE_F64X form
// The same element blocks and fixed-order sums in double-float on the FP32 pipe: the
// coordinates relative to the chunk's reference vertex are split into float pairs
// (as for the F64X scalar operators), the cofactor vectors and scaled Lame sums are
// kept as float pairs in shared memory, and every block entry is formed and summed in
// double-float. Coefficient arrays are double.

// lambda^s (or mu^s) of one element in double-float
template <int D>
__device__ __forceinline__ df coef_sum_x(const void* c, int kind, const int32_t* order, int64_t e,
                                         const float2* local_p1, const int lv[D + 1]) {
  if (kind == FE_COEF_P1) {
    float2 v = local_p1[lv[0]];
    df s{v.x, v.y};
#pragma unroll
    for (int a = 1; a <= D; ++a) {
      v = local_p1[lv[a]];
      s = df_add_fast(s, df{v.x, v.y});
    }
    return s;
  }
  const double* cp = (const double*)c;
  const double v = kind == FE_COEF_SCALAR ? cp[0] : (kind == FE_COEF_P0 ? cp[order[e]] : cp[e]);
  return df_mul_full(df_split(v), df{(float)(D + 1), 0.f});
}

__device__ __forceinline__ df ld_df(const float2* p) {
  const float2 v = *p;
  return df{v.x, v.y};
}

template <int D, int THREADS>
__global__ void __launch_bounds__(THREADS) k_chunk_elas_x(ElasArgs A, double* __restrict__ vals,
                                                          float2* __restrict__ partials) {
  constexpr int NV = D + 1, NP = Pairs<D>::n, MM = D * D;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  const int64_t c = blockIdx.x;
  const int64_t e0 = c * A.chunk;
  const int ne = (int)min((int64_t)A.chunk, A.nme - e0);
  const int32_t nlv = A.ch_v_ptr[c + 1] - A.ch_v_ptr[c];
  const int32_t nle = A.ch_e_ptr[c + 1] - A.ch_e_ptr[c];
  const RecLayout R = rec_layout((uint32_t)ne, NV, NP, (uint32_t)nlv, (uint32_t)nle, true);
  const ElasSmem S = elas_smem(D, 8, A.rec_max, A.max_lv, A.chunk);
  if (!FE_CHUNK_FITS(R.total <= A.rec_max && nlv <= (int32_t)A.max_lv, A.st, c)) return;
  // reference vertex of the chunk, loaded while the record copy is in flight
  double xr[D];
  {
    const int64_t v0 = A.me0[e0];
#pragma unroll
    for (int k = 0; k < D; ++k) xr[k] = __ldg(A.q + k * A.nq + v0);
  }
  if (!load_plan_record(smem, &bar, A.rec, A.rec_off16, c, R.total, A.st, e0, kBarrierSpin)) return;
  const uint16_t* inc_v = (const uint16_t*)(smem + R.inc_v);
  const uint16_t* inc_e = (const uint16_t*)(smem + R.inc_e);
  const uint16_t* lv_off = (const uint16_t*)(smem + R.lv_off);
  const uint16_t* le_off = (const uint16_t*)(smem + R.le_off);
  const int32_t* lv_vid = (const int32_t*)(smem + R.lv_vid);
  const int32_t* lv_dst = (const int32_t*)(smem + R.lv_dst);
  const int32_t* le_dst = (const int32_t*)(smem + R.le_dst);
  const uint16_t* lv_str = (const uint16_t*)(smem + R.lv_str);
  const uint16_t* le_str = (const uint16_t*)(smem + R.le_str);
  const uint16_t* lvid = (const uint16_t*)(smem + R.lvid);
  float2* lam_l = (float2*)(smem + S.coef);
  float2* mu_l = lam_l + A.max_lv;
  float2* Cg = (float2*)(smem + S.cg);  // [e][a][i]
  float2* LM = (float2*)(smem + S.lm);  // [e][2]
  if (!FE_RECORD_VALID(smem, R, ne, NV, NP, nlv, nle, D, A.nq, A.nnz, A.npart, A.st, c)) return;

  // 0. coordinates relative to corner 0 of the chunk's first element, split into float
  //    pairs; P1 Lame values; local vertex of each corner
  for (int u = threadIdx.x; u < nlv; u += THREADS) {
    const int64_t vid = lv_vid[u];
    x64_stage_vertex<D>(A.q, A.nq, vid, xr, smem + S.q, u);
    if (A.lam_kind == FE_COEF_P1) {
      const df v = df_split(((const double*)A.lam)[vid]);
      lam_l[u] = make_float2(v.hi, v.lo);
    }
    if (A.mu_kind == FE_COEF_P1) {
      const df v = df_split(((const double*)A.mu)[vid]);
      mu_l[u] = make_float2(v.hi, v.lo);
    }
  }
  __syncthreads();

  // 1. cofactor vectors (c_0 = -sum c_a) and scaled Lame sums of every element
  for (int el = threadIdx.x; el < ne; el += THREADS) {
    int lv[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) lv[a] = lvid[el * NV + a];
    df cf[D][D];
    df det = x64_geometry_guarded<D>(smem + S.q, lv, cf, A.q, A.nq, lv_vid);
    if (df_degenerate(det)) {
      fe_report(A.st, FE_ERR_DEGENERATE, A.order[e0 + el]);
      det = df{1.f, 0.f};
    }
    if (det.hi < 0.f) det = df_neg(det);
    const df scale = df_recip(df_mul_full(det, df{(float)(factorial(D) * (D + 1)), 0.f}));
    const df ls = coef_sum_x<D>(A.lam, A.lam_kind, A.order, e0 + el, lam_l, lv);
    const df ms = coef_sum_x<D>(A.mu, A.mu_kind, A.order, e0 + el, mu_l, lv);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      df s = cf[0][i];
#pragma unroll
      for (int a = 1; a < D; ++a) s = df_add_fast(s, cf[a][i]);
      Cg[(el * NV) * D + i] = make_float2(-s.hi, -s.lo);
#pragma unroll
      for (int a = 1; a < NV; ++a) Cg[(el * NV + a) * D + i] = make_float2(cf[a - 1][i].hi, cf[a - 1][i].lo);
    }
    const df lp = df_mul_full(ls, scale), mp = df_mul_full(ms, scale);
    LM[2 * el] = make_float2(lp.hi, lp.lo);
    LM[2 * el + 1] = make_float2(mp.hi, mp.lo);
  }
  __syncthreads();

  // 2a. diagonal blocks (lp + mp) x x^T + mp |x|^2 I over the (element, corner)
  //     incidences of each vertex, in element order
  for (int u = threadIdx.x; u < nlv; u += THREADS) {
    const int s = lv_off[u], t = lv_off[u + 1];
    AccX acc[MM];
    for (int j = s; j < t; ++j) {
      const int inc = inc_v[j];
      const int el = inc / NV;
      df x[D];
#pragma unroll
      for (int i = 0; i < D; ++i) x[i] = ld_df(Cg + inc * D + i);
      const df lp = ld_df(LM + 2 * el), mp = ld_df(LM + 2 * el + 1);
      const df lm = df_add_fast(lp, mp);
      const df mxx = df_mul_full(mp, df_dot<D>(x, x));
#pragma unroll
      for (int l = 0; l < D; ++l) {
        const df lx = df_mul_full(lm, x[l]);
#pragma unroll
        for (int n = 0; n < D; ++n) {
          const df v = df_mul_full(lx, x[n]);
          if (j == s) acc[l * D + n] = AccX(v);
          else acc[l * D + n].add(v);
        }
        acc[l * D + l].add(mxx);
      }
    }
    const int32_t dst = lv_dst[u];
    if (dst >= 0) {
      const int str = lv_str[u];
#pragma unroll
      for (int l = 0; l < D; ++l)
#pragma unroll
        for (int n = 0; n < D; ++n) vals[dst + l * str + n] = acc[l * D + n].value();
    } else {
      const int64_t pi = (-1 - (int64_t)dst) * MM;
#pragma unroll
      for (int k = 0; k < MM; ++k) acc[k].store_partial(partials, pi + k);
    }
  }
  // 2b. off-diagonal blocks lp x y^T + mp (y x^T + (x . y) I) over the (element, pair)
  //     incidences of each edge, oriented (vmin, vmax), in element order
  for (int u = threadIdx.x; u < nle; u += THREADS) {
    const int s = le_off[u], t = le_off[u + 1];
    AccX acc[MM];
    for (int j = s; j < t; ++j) {
      const int code = inc_e[j];
      const int ep = code >> 1;
      const int el = ep / NP, p = ep - el * NP;
      int a = Pairs<D>::a(p), b = Pairs<D>::b(p);
      if (code & 1) {  // me(a) > me(b): the (vmin, vmax) block is block (b, a)
        const int t2 = a; a = b; b = t2;
      }
      df x[D], y[D], px[D], qy[D];
      const df lp = ld_df(LM + 2 * el), mp = ld_df(LM + 2 * el + 1);
#pragma unroll
      for (int i = 0; i < D; ++i) {
        x[i] = ld_df(Cg + (el * NV + a) * D + i);
        y[i] = ld_df(Cg + (el * NV + b) * D + i);
        px[i] = df_mul_full(lp, x[i]);
        qy[i] = df_mul_full(mp, y[i]);
      }
      const df mxy = df_dot<D>(qy, x);
#pragma unroll
      for (int l = 0; l < D; ++l) {
#pragma unroll
        for (int n = 0; n < D; ++n) {
          const df v = df_mul_full(px[l], y[n]);
          if (j == s) acc[l * D + n] = AccX(v);
          else acc[l * D + n].add(v);
          acc[l * D + n].add(df_mul_full(qy[l], x[n]));
        }
        acc[l * D + l].add(mxy);
      }
    }
    const int32_t dst = le_dst[2 * u];
    if (dst >= 0) {
      const int32_t dst_t = le_dst[2 * u + 1];
      const int str = le_str[2 * u], str_t = le_str[2 * u + 1];
#pragma unroll
      for (int l = 0; l < D; ++l)
#pragma unroll
        for (int n = 0; n < D; ++n) {
          const double v = acc[l * D + n].value();
          vals[dst + l * str + n] = v;
          vals[dst_t + n * str_t + l] = v;
        }
    } else {
      const int64_t pi = (-1 - (int64_t)dst) * MM;
#pragma unroll
      for (int k = 0; k < MM; ++k) acc[k].store_partial(partials, pi + k);
    }
  }
}

template <int D>
int launch_x(fe_pattern_s* h, const ElasArgs& A, double* vals, cudaStream_t s) {
  constexpr int THREADS = 256;
  const ElasSmem L = elas_smem(D, 8, A.rec_max, A.max_lv, A.chunk);
  if (L.total > kSmemDynMax) return FE_ERR_ARG;
  auto kern = k_chunk_elas_x<D, THREADS>;
  FE_TRY(fe_smem_limit(kern, L.total));
  FE_PROF_BEGIN(h, FE_K_ELAS_CHUNK, s);
  kern<<<(unsigned)h->nchunks, THREADS, L.total, s>>>(A, vals, (float2*)h->partials);
  FE_CUDA_TRY(cudaGetLastError());
  FE_PROF_END(h, FE_K_ELAS_CHUNK, s);
  const int64_t nsh = h->nsh_v + h->nsh_e;
  if (nsh > 0) {
    FE_PROF_BEGIN(h, FE_K_ELAS_FIXUP, s);
    k_fixup_elas<D, double, AccX><<<fe_grid(nsh * D * D, 256), 256, 0, s>>>(
        h->sh_ptr, h->sh_dst, h->sh_str, h->nsh_v, nsh, h->partials, vals, h->nnz, h->npart, h->status);
    FE_CUDA_TRY(cudaGetLastError());
    FE_PROF_END(h, FE_K_ELAS_FIXUP, s);
  }
  return FE_OK;
}

}  // namespace
}  // namespace fe

int fe_launch_elas(fe_pattern_s* h, const double* q, const void* lam, int lam_kind, const void* mu,
                   int mu_kind, int prec, void* vals, cudaStream_t s) {
  using namespace fe;
  if (h->strategy != FE_REASM_CHUNKED) return FE_ERR_ARG;  // vector problems: chunked only
  ElasArgs A{h->nme, h->nq, h->chunk, (uint32_t)h->rec_max_bytes, (uint32_t)h->max_lv, q, lam, lam_kind,
             mu, mu_kind, h->order, h->ch_v_ptr, h->ch_e_ptr, h->rec, h->rec_off16, h->status, h->nnz,
             h->npart, h->me_int};
  if (prec == FE_F64X)
    return h->d == 3 ? launch_x<3>(h, A, (double*)vals, s) : launch_x<2>(h, A, (double*)vals, s);
  if (prec == FE_F64)
    return h->d == 3 ? launch<3, double>(h, A, (double*)vals, s) : launch<2, double>(h, A, (double*)vals, s);
  return h->d == 3 ? launch<3, float>(h, A, (float*)vals, s) : launch<2, float>(h, A, (float*)vals, s);
}
