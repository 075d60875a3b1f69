// Boundary (facet) mass and weighted mass: (d-1)-simplices in d-space, for the
// Neumann and Robin terms the paper's remark after Algorithm 6 mentions. The local
// matrices are those of Section 4.1 with the facet's own dimension k = d - 1 in the
// magic formula (Eq. MagicFormula):
//   mass:          |K| k!/(k+2)! (1 + delta_ab)
//   P1 weighted:   |K| k!/(k+3)! (1 + delta_ab)(w^s + w_a + w_b)
//   P0 weighted:   w_K times the mass
// and |K| the facet measure: the length of a segment (2D), half the norm of the
// cross product of two edges of a triangle (3D), i.e. sqrt(det(B^T B)) / k!.
// Same chunk plan and fixed-order sums as the volume kernels; the FE_F64X form evaluates
// the measure and the entries in double-float (k_chunk_boundary_x).
#include "assemble_impl.cuh"
#include "dfloat.cuh"
#include "profile.cuh"

namespace fe {
namespace {

template <int D, class T, int KIND, int THREADS>
__global__ void __launch_bounds__(THREADS) k_chunk_boundary(StagedArgs A, T* __restrict__ vals,
                                                            void* __restrict__ partials) {
  constexpr int KD = D - 1, NV = D, NP = Pairs<KD>::n;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  const int64_t c = blockIdx.x;
  const int64_t e0 = c * A.chunk;
  const int ne = (int)min((int64_t)A.chunk, A.nme - e0);
  const int32_t nlv = A.ch_v_ptr[c + 1] - A.ch_v_ptr[c];
  const int32_t nle = A.ch_e_ptr[c + 1] - A.ch_e_ptr[c];
  const RecLayout R = rec_layout((uint32_t)ne, NV, NP, (uint32_t)nlv, (uint32_t)nle);
  const StagedSmem S = boundary_smem(D, (int)sizeof(T), KIND == K_WMASS_P1, A.rec_max, A.max_lv, A.chunk);
  if (!FE_CHUNK_FITS(R.total <= A.rec_max && nlv <= (int32_t)A.max_lv, A.st, c)) return;
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
  if (!FE_RECORD_VALID(smem, R, ne, NV, NP, nlv, nle, 1, A.nq, A.nnz, A.npart, A.st, c)) return;

  for (int u = threadIdx.x; u < nlv; u += THREADS) {
    const int64_t vid = lv_vid[u];
    stage_vertex<D, T>(A.q, A.nq, vid, smem + S.q, u);
    if constexpr (KIND == K_WMASS_P1) wl[u] = ((const T*)A.w)[vid];
  }
  __syncthreads();

  const bool has_coef = A.w_kind != FE_COEF_NONE && KIND != K_WMASS_P1;
  for (int el = threadIdx.x; el < ne; el += THREADS) {
    int lv[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) lv[a] = lvid[el * NV + a];
    T e[KD][D];  // edge vectors from vertex 0
    if constexpr (sizeof(T) == 8) {
      double x[NV][D];
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        const double* xs = (const double*)(smem + S.q) + (D == 3 ? 4 : 2) * lv[a];
        const double2 xy = ((const double2*)xs)[0];
        x[a][0] = xy.x;
        x[a][1] = xy.y;
        if constexpr (D == 3) x[a][2] = xs[2];
      }
#pragma unroll
      for (int i = 0; i < KD; ++i)
#pragma unroll
        for (int k = 0; k < D; ++k) e[i][k] = x[i + 1][k] - x[0][k];
    } else {
      float xh[NV][D], xl[NV][D];
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        const float4* xs = (const float4*)(smem + S.q) + (D == 3 ? 2 : 1) * lv[a];
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
      // correctly rounded edges from the split coordinates
#pragma unroll
      for (int i = 0; i < KD; ++i)
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const df s = two_sum(xh[i + 1][k], -xh[0][k]);
          e[i][k] = __fadd_rn(s.hi, __fadd_rn(s.lo, __fsub_rn(xl[i + 1][k], xl[0][k])));
        }
    }
    T meas;  // facet measure |K|
    if constexpr (D == 2) {
      meas = sqrt(e[0][0] * e[0][0] + e[0][1] * e[0][1]);
    } else {
      const T nx = e[0][1] * e[1][2] - e[0][2] * e[1][1];
      const T ny = e[0][2] * e[1][0] - e[0][0] * e[1][2];
      const T nz = e[0][0] * e[1][1] - e[0][1] * e[1][0];
      meas = T(0.5) * sqrt(nx * nx + ny * ny + nz * nz);
    }
    if (!det_ok(meas)) {
      fe_report(A.st, FE_ERR_DEGENERATE, A.order[e0 + el]);
      meas = T(1);
    }
    T diag[NV], off[NP];
    if constexpr (KIND == K_WMASS_P1) {
      T wv[NV], ws = T(0);
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        wv[a] = wl[lv[a]];
        ws += wv[a];
      }
      const T base = meas * T((double)factorial(KD) / (double)factorial(KD + 3));
#pragma unroll
      for (int a = 0; a < NV; ++a) diag[a] = T(2) * base * (ws + T(2) * wv[a]);
#pragma unroll
      for (int p = 0; p < NP; ++p) off[p] = base * (ws + wv[Pairs<KD>::a(p)] + wv[Pairs<KD>::b(p)]);
    } else {
      T m = meas * T(1.0 / ((KD + 1) * (KD + 2)));
      if (has_coef) m *= elem_coef<T>(A.w, A.w_kind, A.order, e0 + el);
#pragma unroll
      for (int a = 0; a < NV; ++a) diag[a] = T(2) * m;
#pragma unroll
      for (int p = 0; p < NP; ++p) off[p] = m;
    }
#pragma unroll
    for (int a = 0; a < NV; ++a) Kd[el * NV + a] = diag[a];
#pragma unroll
    for (int p = 0; p < NP; ++p) Ko[el * NP + p] = off[p];
  }
  __syncthreads();

  for (int u = threadIdx.x; u < nlv; u += THREADS) {
    const int s = lv_off[u], t = lv_off[u + 1];
    Acc<T> acc(Kd[inc_v[s]]);
    for (int j = s + 1; j < t; ++j) acc.add(Kd[inc_v[j]]);
    const int32_t dst = lv_dst[u];
    if (dst >= 0) vals[dst] = acc.value();
    else acc.store_partial(partials, -1 - (int64_t)dst);
  }
  for (int u = threadIdx.x; u < nle; u += THREADS) {
    const int s = le_off[u], t = le_off[u + 1];
    Acc<T> acc(Ko[inc_e[s] >> 1]);
    for (int j = s + 1; j < t; ++j) acc.add(Ko[inc_e[j] >> 1]);
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

template <int D, class T, int KIND>
int launch(fe_pattern_s* h, const StagedArgs& A, T* vals, cudaStream_t s) {
  constexpr int THREADS = 256;
  const StagedSmem L = boundary_smem(D, (int)sizeof(T), KIND == K_WMASS_P1, A.rec_max, A.max_lv, A.chunk);
  if (L.total > kSmemDynMax) return FE_ERR_ARG;
  auto kern = k_chunk_boundary<D, T, KIND, THREADS>;
  FE_TRY(fe_smem_limit(kern, L.total));
  FE_PROF_BEGIN(h, FE_K_CHUNK, s);
  kern<<<(unsigned)h->nchunks, THREADS, L.total, s>>>(A, vals, h->partials);
  FE_CUDA_TRY(cudaGetLastError());
  FE_PROF_END(h, FE_K_CHUNK, s);
  const int64_t nsh = h->nsh_v + h->nsh_e;
  if (nsh > 0) {
    FE_PROF_BEGIN(h, FE_K_FIXUP, s);
    k_fixup_scalar<T><<<fixup_grid<T>(nsh), 256, 0, s>>>(h->sh_ptr, h->sh_dst, h->nsh_v, nsh, h->partials, vals, h->nnz_s, h->npart, h->status);
    FE_CUDA_TRY(cudaGetLastError());
    FE_PROF_END(h, FE_K_FIXUP, s);
  }
  return FE_OK;
}

template <class T>
int dispatch(fe_pattern_s* h, int kind, const StagedArgs& A, T* vals, cudaStream_t s) {
  if (h->d == 3) {
    if (kind == K_MASS) return launch<3, T, K_MASS>(h, A, vals, s);
    if (kind == K_WMASS_P1) return launch<3, T, K_WMASS_P1>(h, A, vals, s);
    return launch<3, T, K_WMASS_P0>(h, A, vals, s);
  }
  if (kind == K_MASS) return launch<2, T, K_MASS>(h, A, vals, s);
  if (kind == K_WMASS_P1) return launch<2, T, K_WMASS_P1>(h, A, vals, s);
  return launch<2, T, K_WMASS_P0>(h, A, vals, s);
}

// FE_F64X form: coordinates relative to the chunk's reference vertex split into float
// pairs, edges, measure (double-float square root) and entries in double-float, sums in
// double-float, double values; weights are double.
template <int D, int KIND, int THREADS>
__global__ void __launch_bounds__(THREADS) k_chunk_boundary_x(StagedArgs A, const int32_t* __restrict__ me0,
                                                              double* __restrict__ vals,
                                                              float2* __restrict__ partials) {
  constexpr int KD = D - 1, NV = D, NP = Pairs<KD>::n;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  const int64_t c = blockIdx.x;
  const int64_t e0 = c * A.chunk;
  const int ne = (int)min((int64_t)A.chunk, A.nme - e0);
  const int32_t nlv = A.ch_v_ptr[c + 1] - A.ch_v_ptr[c];
  const int32_t nle = A.ch_e_ptr[c + 1] - A.ch_e_ptr[c];
  const RecLayout R = rec_layout((uint32_t)ne, NV, NP, (uint32_t)nlv, (uint32_t)nle);
  const StagedSmem S = boundary_smem(D, 8, KIND == K_WMASS_P1, A.rec_max, A.max_lv, A.chunk);
  if (!FE_CHUNK_FITS(R.total <= A.rec_max && nlv <= (int32_t)A.max_lv, A.st, c)) return;
  // reference vertex of the chunk, loaded while the record copy is in flight
  double xr[D];
  {
    const int64_t v0 = me0[e0];
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
  const uint16_t* lvid = (const uint16_t*)(smem + R.lvid);
  float2* Kd = (float2*)(smem + S.kd);
  float2* Ko = (float2*)(smem + S.ko);
  float2* wl = (float2*)(smem + S.w);
  if (!FE_RECORD_VALID(smem, R, ne, NV, NP, nlv, nle, 1, A.nq, A.nnz, A.npart, A.st, c)) return;

  for (int u = threadIdx.x; u < nlv; u += THREADS) {
    const int64_t vid = lv_vid[u];
    x64_stage_vertex<D>(A.q, A.nq, vid, xr, smem + S.q, u);
    if constexpr (KIND == K_WMASS_P1) {
      const df wv = df_split(((const double*)A.w)[vid]);
      wl[u] = make_float2(wv.hi, wv.lo);
    }
  }
  __syncthreads();

  const bool has_coef = A.w_kind != FE_COEF_NONE && KIND != K_WMASS_P1;
  for (int el = threadIdx.x; el < ne; el += THREADS) {
    int lv[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) lv[a] = lvid[el * NV + a];
    df e[KD][D];
    x64_edges<D, KD>(smem + S.q, lv, e);
    df m2;  // squared measure (times 4 for a triangle)
    if constexpr (D == 2) {
      m2 = df_dot<2>(e[0], e[0]);
    } else {
      df n[3];
      n[0] = df_cross_term(e[0][1], e[1][2], e[0][2], e[1][1]);
      n[1] = df_cross_term(e[0][2], e[1][0], e[0][0], e[1][2]);
      n[2] = df_cross_term(e[0][0], e[1][1], e[0][1], e[1][0]);
      m2 = df_dot<3>(n, n);
    }
    if (df_degenerate(m2)) {
      fe_report(A.st, FE_ERR_DEGENERATE, A.order[e0 + el]);
      m2 = df{1.f, 0.f};
    }
    df meas = df_sqrt(m2);
    if constexpr (D == 3) meas = df{0.5f * meas.hi, 0.5f * meas.lo};  // exact
    df dv[NV], ov[NP];
    if constexpr (KIND == K_WMASS_P1) {
      constexpr DfConst kC = df_const(1.0 / ((KD + 1) * (KD + 2) * (KD + 3)));
      const df base = df_mul_full(meas, df_of(kC));
      df w[NV];
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        const float2 x = wl[lv[a]];
        w[a] = df{x.x, x.y};
      }
      df ws = w[0];
#pragma unroll
      for (int a = 1; a < NV; ++a) ws = df_add_fast(ws, w[a]);
#pragma unroll
      for (int a = 0; a < NV; ++a) dv[a] = df_twice(df_mul_full(base, df_add_fast(ws, df_twice(w[a]))));
#pragma unroll
      for (int p = 0; p < NP; ++p)
        ov[p] = df_mul_full(base, df_add_fast(ws, df_add_fast(w[Pairs<KD>::a(p)], w[Pairs<KD>::b(p)])));
    } else {
      constexpr DfConst kC = df_const(1.0 / ((KD + 1) * (KD + 2)));
      df m = df_mul_full(meas, df_of(kC));
      if (has_coef) m = df_mul_full(m, df_split(elem_coef<double>(A.w, A.w_kind, A.order, e0 + el)));
#pragma unroll
      for (int a = 0; a < NV; ++a) dv[a] = df_twice(m);
#pragma unroll
      for (int p = 0; p < NP; ++p) ov[p] = m;
    }
#pragma unroll
    for (int a = 0; a < NV; ++a) Kd[el * NV + a] = make_float2(dv[a].hi, dv[a].lo);
#pragma unroll
    for (int p = 0; p < NP; ++p) Ko[el * NP + p] = make_float2(ov[p].hi, ov[p].lo);
  }
  __syncthreads();

  for (int u = threadIdx.x; u < nlv; u += THREADS) {
    const int s = lv_off[u], t = lv_off[u + 1];
    AccX acc = AccX::from_partial(Kd, inc_v[s]);
    for (int j = s + 1; j < t; ++j) acc.add_partial(Kd, inc_v[j]);
    const int32_t dst = lv_dst[u];
    if (dst >= 0) vals[dst] = acc.value();
    else acc.store_partial(partials, -1 - (int64_t)dst);
  }
  for (int u = threadIdx.x; u < nle; u += THREADS) {
    const int s = le_off[u], t = le_off[u + 1];
    AccX acc = AccX::from_partial(Ko, inc_e[s] >> 1);
    for (int j = s + 1; j < t; ++j) acc.add_partial(Ko, inc_e[j] >> 1);
    const int32_t dst = le_dst[2 * u];
    if (dst >= 0) {
      const double val = acc.value();
      vals[dst] = val;
      vals[le_dst[2 * u + 1]] = val;
    } else {
      acc.store_partial(partials, -1 - (int64_t)dst);
    }
  }
}

template <int D, int KIND>
int launch_x(fe_pattern_s* h, const StagedArgs& A, double* vals, cudaStream_t s) {
  constexpr int THREADS = 256;
  const StagedSmem L = boundary_smem(D, 8, KIND == K_WMASS_P1, A.rec_max, A.max_lv, A.chunk);
  if (L.total > kSmemDynMax) return FE_ERR_ARG;
  auto kern = k_chunk_boundary_x<D, KIND, THREADS>;
  FE_TRY(fe_smem_limit(kern, L.total));
  FE_PROF_BEGIN(h, FE_K_CHUNK, s);
  kern<<<(unsigned)h->nchunks, THREADS, L.total, s>>>(A, h->me_int, vals, (float2*)h->partials);
  FE_CUDA_TRY(cudaGetLastError());
  FE_PROF_END(h, FE_K_CHUNK, s);
  const int64_t nsh = h->nsh_v + h->nsh_e;
  if (nsh > 0) {
    FE_PROF_BEGIN(h, FE_K_FIXUP, s);
    k_fixup_scalar<double, AccX><<<fixup_grid<double>(nsh), 256, 0, s>>>(h->sh_ptr, h->sh_dst, h->nsh_v, nsh,
                                                                  h->partials, vals, h->nnz_s, h->npart,
                                                                  h->status);
    FE_CUDA_TRY(cudaGetLastError());
    FE_PROF_END(h, FE_K_FIXUP, s);
  }
  return FE_OK;
}

int dispatch_x(fe_pattern_s* h, int kind, const StagedArgs& A, double* vals, cudaStream_t s) {
  if (h->d == 3) {
    if (kind == K_MASS) return launch_x<3, K_MASS>(h, A, vals, s);
    if (kind == K_WMASS_P1) return launch_x<3, K_WMASS_P1>(h, A, vals, s);
    return launch_x<3, K_WMASS_P0>(h, A, vals, s);
  }
  if (kind == K_MASS) return launch_x<2, K_MASS>(h, A, vals, s);
  if (kind == K_WMASS_P1) return launch_x<2, K_WMASS_P1>(h, A, vals, s);
  return launch_x<2, K_WMASS_P0>(h, A, vals, s);
}

}  // namespace
}  // namespace fe

int fe_launch_boundary(fe_pattern_s* h, int kind, const double* q, const void* w, int w_kind, int prec,
                       void* vals, cudaStream_t s) {
  using namespace fe;
  if (h->strategy != FE_REASM_CHUNKED || kind == K_STIFF) return FE_ERR_ARG;
  StagedArgs A{h->nme, h->nq, h->chunk, (uint32_t)h->rec_max_bytes, (uint32_t)h->max_lv, q, w, w_kind,
               h->order, h->ch_v_ptr, h->ch_e_ptr, h->rec, h->rec_off16, h->status, h->nnz_s, h->npart};
  if (prec == FE_F64X) return dispatch_x(h, kind, A, (double*)vals, s);
  if (prec == FE_F64) return dispatch<double>(h, kind, A, (double*)vals, s);
  return dispatch<float>(h, kind, A, (float*)vals, s);
}
