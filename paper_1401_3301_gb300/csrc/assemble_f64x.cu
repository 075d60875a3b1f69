// FE_F64X form of the scalar volume operators (mass, weighted mass, stiffness): FP64
// inputs and outputs, FP64-class accuracy, arithmetic in double-float (unevaluated
// sums of two floats, about 48 significant bits) on the FP32 pipe, which on this part
// issues 64 times as many operations per clock as the FP64 pipe. Native FP64 is used
// only to take each chunk vertex's coordinates relative to a reference vertex of the
// chunk (so that large coordinate offsets cannot cost accuracy) and to convert each
// final sum to double; coefficients are split into float pairs without FP64 arithmetic.
//
// Local matrices, with the cofactor vectors c_a of B = [q^1 - q^0, ...] (the row of
// vertex 0 follows from sum_a c_a = 0):
//   stiffness (Eq. stiffelemmat): S_ab = w (c_a . c_b) / (d! |det B|);
//   mass (Section 4.1): |det B| / (d+2)! (1 + delta_ab), times w for a P0 weight;
//   P1-weighted mass (Eq. MatElemMassWP1): |det B| / (d+3)! (1 + delta_ab)(w^s + w_a + w_b).
// Sums over the incidences of each chunk vertex / edge run in ascending element
// order, then over chunks in chunk order (as in the other forms).
#include "assemble_impl.cuh"
#include "dfloat.cuh"
#include "profile.cuh"

namespace fe {
namespace {

struct X64Args {
  int64_t nme, nq;
  int chunk;
  uint32_t rec_max, max_lv;
  const double* q;
  const double* w;
  int w_kind;
  const int32_t* order;
  const int32_t* me0;  // first row of the internal connectivity: corner 0 of each element
  const int32_t* ch_v_ptr;
  const int32_t* ch_e_ptr;
  const uint8_t* rec;
  const uint32_t* rec_off16;
  fe_status_word* st;
  int64_t nnz, npart;  // sizes of vals and of the partial sums (bounds-checked builds)
};

// Entries of element el of chunk c (corners lv, cofactor vectors cf, det B) into its
// diagonal (Kd) and off-diagonal (Ko) double-float slots.
template <int D, int KIND>
__device__ __forceinline__ void x64_element_values(const X64Args& A, int64_t e0, int el, const int lv[D + 1],
                                                   const df cf[D][D], df det, const float2* wl, float2* Kd,
                                                   float2* Ko) {
  constexpr int NV = D + 1, NP = Pairs<D>::n;
  if (df_degenerate(det)) {
    fe_report(A.st, FE_ERR_DEGENERATE, A.order[e0 + el]);
    det = df{1.f, 0.f};
  }
  if (det.hi < 0.f) det = df_neg(det);
  if constexpr (KIND != K_STIFF) {
    df dv[NV], ov[NP];
    if constexpr (KIND == K_WMASS_P1) {
      constexpr DfConst kC = df_const(1.0 / factorial(D + 3));
      const df base = df_mul_full(det, df_of(kC));
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
        ov[p] = df_mul_full(base, df_add_fast(ws, df_add_fast(w[Pairs<D>::a(p)], w[Pairs<D>::b(p)])));
    } else {
      constexpr DfConst kC = df_const(1.0 / factorial(D + 2));
      df m = df_mul_full(det, df_of(kC));
      if (A.w_kind != FE_COEF_NONE)
        m = df_mul_full(m, df_split(elem_coef<double>(A.w, A.w_kind, A.order, e0 + el)));
#pragma unroll
      for (int a = 0; a < NV; ++a) dv[a] = df_twice(m);
#pragma unroll
      for (int p = 0; p < NP; ++p) ov[p] = m;
    }
#pragma unroll
    for (int a = 0; a < NV; ++a) Kd[el * NV + a] = make_float2(dv[a].hi, dv[a].lo);
#pragma unroll
    for (int p = 0; p < NP; ++p) Ko[el * NP + p] = make_float2(ov[p].hi, ov[p].lo);
    return;
  }
  df inv = df_recip(df_mul_full(det, df{(float)factorial(D), 0.f}));
  if (A.w_kind != FE_COEF_NONE)
    inv = df_mul_full(inv, df_split(elem_coef<double>(A.w, A.w_kind, A.order, e0 + el)));
  df G[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) {
      G[i][j] = df_mul_full(df_dot<D>(cf[i], cf[j]), inv);
      G[j][i] = G[i][j];
    }
  df nr[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    df s = df_neg(G[i][0]);
#pragma unroll
    for (int j = 1; j < D; ++j) s = df_sub(s, G[i][j]);
    nr[i] = s;
  }
  df d0 = df_neg(nr[0]);
#pragma unroll
  for (int i = 1; i < D; ++i) d0 = df_sub(d0, nr[i]);
  Kd[el * NV] = make_float2(d0.hi, d0.lo);
#pragma unroll
  for (int i = 0; i < D; ++i) Kd[el * NV + i + 1] = make_float2(G[i][i].hi, G[i][i].lo);
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int a = Pairs<D>::a(p), b = Pairs<D>::b(p);
    const df v = (a == 0) ? nr[b - 1] : G[a - 1][b - 1];
    Ko[el * NP + p] = make_float2(v.hi, v.lo);
  }
}

// registers capped so that 6 blocks of 256 threads fit on an SM (40 per thread, a few
// spilled): the kernel is latency-bound like the FP32 form's (chunk 224: 0.339 -> 0.312 ms
// at N=100)
template <int D, int KIND, int THREADS>
__global__ void __launch_bounds__(THREADS, 1536 / THREADS) k_chunk_f64x(X64Args A, double* __restrict__ vals,
                                                        float2* __restrict__ partials) {
  constexpr int NV = D + 1, NP = Pairs<D>::n;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  const int64_t c = blockIdx.x;
  const int64_t e0 = c * A.chunk;
  const int ne = (int)min((int64_t)A.chunk, A.nme - e0);
  const int32_t nlv = A.ch_v_ptr[c + 1] - A.ch_v_ptr[c];
  const int32_t nle = A.ch_e_ptr[c + 1] - A.ch_e_ptr[c];
  const RecLayout R = rec_layout((uint32_t)ne, NV, NP, (uint32_t)nlv, (uint32_t)nle);
  // same footprint as the FP32 form: split coordinates, float2 values
  // (the region after the values holds the list of elements to recompute)
  const StagedSmem S = staged_smem(D, 8, KIND == K_WMASS_P1, A.rec_max, A.max_lv, A.chunk, true);
  __shared__ int nslow;
  uint16_t* slow = (uint16_t*)(smem + S.sc);
  if (threadIdx.x == 0) nslow = 0;
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
  const uint16_t* lvid = (const uint16_t*)(smem + R.lvid);
  float2* Kd = (float2*)(smem + S.kd);
  float2* Ko = (float2*)(smem + S.ko);
  float2* wl = (float2*)(smem + S.w);  // P1 weight of each chunk vertex
  if (!FE_RECORD_VALID(smem, R, ne, NV, NP, nlv, nle, 1, A.nq, A.nnz, A.npart, A.st, c)) return;

  // 0. coordinates relative to corner 0 of the chunk's first element (FP64), split into
  //    float pairs; the reference does not depend on the record's vertex order
  for (int u = threadIdx.x; u < nlv; u += THREADS) {
    const int64_t vid = lv_vid[u];
    x64_stage_vertex<D>(A.q, A.nq, vid, xr, smem + S.q, u);
    if constexpr (KIND == K_WMASS_P1) {
      const df wv = df_split(A.w[vid]);
      wl[u] = make_float2(wv.hi, wv.lo);
    }
  }
  __syncthreads();

  // 1. element entries in double-float. An element whose double-float det B fails its
  //    guard (dfloat.cuh) is listed and, after the loop, recomputed with the FP64 det B,
  //    so that the common path carries no out-of-line call
  for (int el = threadIdx.x; el < ne; el += THREADS) {
    int lv[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) lv[a] = lvid[el * NV + a];
    df cf[D][D];  // cofactor vectors c_1..c_D
    bool exact;
    const df det = x64_geometry_check<D>(smem + S.q, lv, cf, exact);
    if (exact) slow[atomicAdd(&nslow, 1)] = (uint16_t)el;
    x64_element_values<D, KIND>(A, e0, el, lv, cf, det, wl, Kd, Ko);
  }
  __syncthreads();
  if (nslow > 0) {
    for (int i = threadIdx.x; i < nslow; i += THREADS) {
      const int el = slow[i];
      int lv[NV];
      int32_t v[NV];
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        lv[a] = lvid[el * NV + a];
        v[a] = lv_vid[lv[a]];
      }
      df cf[D][D];
      bool exact;
      x64_geometry_check<D>(smem + S.q, lv, cf, exact);
      x64_element_values<D, KIND>(A, e0, el, lv, cf, df_split(det_from_q<D>(A.q, A.nq, vert_ids<D>(v))), wl, Kd, Ko);
    }
    __syncthreads();
  }

  // 2. sums in element order; owned sums become doubles, shared ones stay float pairs
  for (int u = threadIdx.x; u < nlv; u += THREADS) {
    const int s = lv_off[u], t = lv_off[u + 1];
    float2 v = Kd[inc_v[s]];
    df acc{v.x, v.y};
    for (int j = s + 1; j < t; ++j) {
      v = Kd[inc_v[j]];
      acc = df_add_fast(acc, df{v.x, v.y});
    }
    const int32_t dst = lv_dst[u];
    if (dst >= 0) vals[dst] = df_to_double(acc);
    else partials[-1 - (int64_t)dst] = make_float2(acc.hi, acc.lo);
  }
  for (int u = threadIdx.x; u < nle; u += THREADS) {
    const int s = le_off[u], t = le_off[u + 1];
    float2 v = Ko[inc_e[s] >> 1];
    df acc{v.x, v.y};
    for (int j = s + 1; j < t; ++j) {
      v = Ko[inc_e[j] >> 1];
      acc = df_add_fast(acc, df{v.x, v.y});
    }
    const int32_t dst = le_dst[2 * u];
    if (dst >= 0) {
      const double val = df_to_double(acc);
      vals[dst] = val;
      vals[le_dst[2 * u + 1]] = val;
    } else {
      partials[-1 - (int64_t)dst] = make_float2(acc.hi, acc.lo);
    }
  }
}

template <int D, int KIND, int THREADS>
int launch(fe_pattern_s* h, const X64Args& A, double* vals, cudaStream_t s) {
  const StagedSmem L = staged_smem(D, 8, KIND == K_WMASS_P1, A.rec_max, A.max_lv, A.chunk, true);
  if (L.total > kSmemDynMax) return FE_ERR_ARG;
  auto kern = k_chunk_f64x<D, KIND, THREADS>;
  FE_TRY(fe_smem_limit(kern, L.total));
  FE_PROF_BEGIN(h, FE_K_CHUNK, s);
  kern<<<(unsigned)h->nchunks, THREADS, L.total, s>>>(A, vals, (float2*)h->partials);
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

template <int D, int THREADS>
int launch_kind(fe_pattern_s* h, int kind, const X64Args& A, double* vals, cudaStream_t s) {
  switch (kind) {
    case K_MASS: return launch<D, K_MASS, THREADS>(h, A, vals, s);
    case K_WMASS_P1: return launch<D, K_WMASS_P1, THREADS>(h, A, vals, s);
    case K_WMASS_P0: return launch<D, K_WMASS_P0, THREADS>(h, A, vals, s);
    default: return launch<D, K_STIFF, THREADS>(h, A, vals, s);
  }
}

// threads per block of the pattern (fe_pattern_set_threads): 128, 256 (default) or 512
template <int D>
int launch_threads(fe_pattern_s* h, int kind, const X64Args& A, double* vals, cudaStream_t s) {
  if (h->threads == 128) return launch_kind<D, 128>(h, kind, A, vals, s);
  if (h->threads == 512) return launch_kind<D, 512>(h, kind, A, vals, s);
  return launch_kind<D, 256>(h, kind, A, vals, s);
}

#include "assemble_pair_f64x.inc"

}  // namespace
}  // namespace fe

int fe_launch_pair_f64x(fe_pattern_s* h, const double* q, const void* w, int w_kind, void* vals_mass,
                        void* vals_stiff, cudaStream_t s) {
  using namespace fe;
  if (h->strategy != FE_REASM_CHUNKED) return FE_ERR_ARG;
  X64Args A{h->nme, h->nq, h->chunk, (uint32_t)h->rec_max_bytes, (uint32_t)h->max_lv, q, (const double*)w,
            w_kind, h->order, h->me_int, h->ch_v_ptr, h->ch_e_ptr, h->rec, h->rec_off16, h->status,
            h->nnz_s, h->npart};
  if (h->d == 3) return launch_pair_x_threads<3>(h, A, (double*)vals_mass, (double*)vals_stiff, s);
  return launch_pair_x_threads<2>(h, A, (double*)vals_mass, (double*)vals_stiff, s);
}

int fe_launch_f64x(fe_pattern_s* h, int kind, const double* q, const void* w, int w_kind, void* vals,
                   cudaStream_t s) {
  using namespace fe;
  if (h->strategy != FE_REASM_CHUNKED) return FE_ERR_ARG;
  X64Args A{h->nme, h->nq, h->chunk, (uint32_t)h->rec_max_bytes, (uint32_t)h->max_lv, q, (const double*)w,
            w_kind, h->order, h->me_int, h->ch_v_ptr, h->ch_e_ptr, h->rec, h->rec_off16, h->status,
            h->nnz_s, h->npart};
  if (h->d == 3) return launch_threads<3>(h, kind, A, (double*)vals, s);
  return launch_threads<2>(h, kind, A, (double*)vals, s);
}
