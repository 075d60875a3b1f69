// General second-order operator of Eq. EDP (Section 1),
//   -div(A grad u) + div(b u) + c . grad u + a0 u,
// with coefficients constant on each element, in the weak form obtained by moving the
// divergence terms onto the test function (boundary integrals left out):
//   a(u, v) = int (A grad u) . grad v - int u b . grad v + int (c . grad u) v + int a0 u v.
// Matrix entry (i, j) is a(phi_j, phi_i); the matrix is not symmetric. Coefficients come
// as records of d*d + 2d + 1 values (A row-major, b, c, a0), one per element or vertex. With g_a = c_a / det B
// (cofactor vectors), int phi_a = |K| / (d+1) and the magic formula (Eq. MagicFormula) for
// int phi_a phi_b, the local entry of test vertex a and trial vertex b is
//   E_ab = c_a . (A c_b) / (d! |det B|) + sgn(det B) (c . c_b - b . c_a) / (d+1)!
//          + a0 |det B| (1 + delta_ab) / (d+2)!.
// P1 coefficients (vertex values f(v), f = sum_v f(v) lambda_v on K, f^s = sum_v f(v)) give,
// by the magic formula,
//   E_ab = c_a . (A^s c_b) / ((d+1)! |det B|)
//          + sgn(det B) (c_b . (c^s + c(a)) - c_a . (b^s + b(b))) / (d+2)!
//          + |det B| (1 + delta_ab) (a0^s + a0(a) + a0(b)) / (d+3)!.
// Reassembly follows the chunked plan of the symmetric operators; each edge carries two
// sums, one per orientation, picked per incidence by the plan's orientation bit.
#include "assemble_impl.cuh"
#include "dfloat.cuh"
#include "profile.cuh"

namespace fe {
namespace {

template <int D>
struct GenCoef {
  static constexpr int n = D * D + 2 * D + 1;  // A (row-major), b, c, a0
};

template <int D, class T>
struct GeneralVals {
  T diag[D + 1];
  T lo[Pairs<D>::n];  // E_ab of pair p = (a, b), a < b
  T hi[Pairs<D>::n];  // E_ba
};

// One coefficient record (A row-major, b, c, a0). In 3D a record is 128 B (FP64) or 64 B
// (FP32), so a 16-byte aligned array (vec) keeps every record aligned for vector loads.
template <int D, class T>
__device__ __forceinline__ void load_record(const T* __restrict__ rec, bool vec, T cf[GenCoef<D>::n]) {
  if constexpr (D == 3) {
    if (vec) {
      if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const double2 v = __ldg((const double2*)rec + i);
          cf[2 * i] = v.x;
          cf[2 * i + 1] = v.y;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float4 v = __ldg((const float4*)rec + i);
          cf[4 * i] = v.x;
          cf[4 * i + 1] = v.y;
          cf[4 * i + 2] = v.z;
          cf[4 * i + 3] = v.w;
        }
      }
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < GenCoef<D>::n; ++j) cf[j] = __ldg(rec + j);
}

// a coefficient of stored type R as the number type T of the arithmetic (the same type,
// or a double split into a double-float pair)
template <class T, class R>
__device__ __forceinline__ T coef_value(R x) { return T(x); }
template <>
__device__ __forceinline__ dfx coef_value<dfx, double>(double x) { return df_split(x); }

// one record of stored type R as numbers of type T
template <int D, class T, class R>
__device__ __forceinline__ void load_coef(const R* __restrict__ rec, bool vec, T cf[GenCoef<D>::n]) {
  R r[GenCoef<D>::n];
  load_record<D, R>(rec, vec, r);
#pragma unroll
  for (int j = 0; j < GenCoef<D>::n; ++j) cf[j] = coef_value<T, R>(r[j]);
}

// coefficient record of internal element e: the single record (scalar), or one per element
// in input (P0) or internal (P0_INTERNAL) order
template <int D, class T, class R = T>
__device__ __forceinline__ void general_coef(const R* __restrict__ coef, int kind, bool vec,
                                             const int32_t* order, int64_t e, T cf[GenCoef<D>::n]) {
  const int64_t k = kind == FE_COEF_SCALAR ? 0 : (kind == FE_COEF_P0 ? (int64_t)order[e] : e);
  load_coef<D, T, R>(coef + k * GenCoef<D>::n, vec, cf);
}

// P[a][b] = c_a . (A c_b) for all corners; the products are formed for corners 1..D and
// row and column 0 follow from sum_a c_a = 0.
template <int D, class T>
__device__ __forceinline__ void diffusion_block(const Geo<D, T>& g, const T* A, T P[D + 1][D + 1]) {
  constexpr int NV = D + 1;
  T Ac[D][D];  // Ac[j] = A c_{j+1}
#pragma unroll
  for (int j = 0; j < D; ++j)
#pragma unroll
    for (int r = 0; r < D; ++r) {
      T s = A[r * D] * g.c[j + 1][0];
#pragma unroll
      for (int k = 1; k < D; ++k) s += A[r * D + k] * g.c[j + 1][k];
      Ac[j][r] = s;
    }
#pragma unroll
  for (int i = 1; i < NV; ++i)
#pragma unroll
    for (int j = 1; j < NV; ++j) {
      T s = g.c[i][0] * Ac[j - 1][0];
#pragma unroll
      for (int r = 1; r < D; ++r) s += g.c[i][r] * Ac[j - 1][r];
      P[i][j] = s;
    }
#pragma unroll
  for (int j = 1; j < NV; ++j) {
    T s = -P[1][j];
#pragma unroll
    for (int i = 2; i < NV; ++i) s -= P[i][j];
    P[0][j] = s;
  }
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    T s = -P[i][1];
#pragma unroll
    for (int j = 2; j < NV; ++j) s -= P[i][j];
    P[i][0] = s;
  }
}

// Local matrix of one element with constant coefficients. A is scaled by 1/(d! |det B|)
// before the products; the convection dot products of vertex 0 follow from sum_a c_a = 0;
// then E_ab = P_ab + u_b + w_a (+ m on the diagonal) with u_b = cs c.c_b + m, w_a = -cs b.c_a.
template <int D, class T>
__device__ __forceinline__ void general_values(const Geo<D, T>& g, const T cf[GenCoef<D>::n],
                                               GeneralVals<D, T>& out) {
  constexpr int NV = D + 1;
  const T* bv = cf + D * D;
  const T* cv = cf + D * D + D;
  const T adet = tabs(g.det);
  const T inv = recip<T>(T(factorial(D)) * adet);
  const T cs = (g.det < T(0) ? T(-1) : T(1)) * T(1.0 / factorial(D + 1));
  const T m = cf[D * D + 2 * D] * adet * T(1.0 / factorial(D + 2));
  T As[D * D];
#pragma unroll
  for (int j = 0; j < D * D; ++j) As[j] = cf[j] * inv;
  T P[NV][NV];
  diffusion_block<D, T>(g, As, P);
  T be[NV], ga[NV];  // b . c_a and c . c_a
#pragma unroll
  for (int a = 1; a < NV; ++a) {
    T sb = bv[0] * g.c[a][0], sc = cv[0] * g.c[a][0];
#pragma unroll
    for (int r = 1; r < D; ++r) {
      sb += bv[r] * g.c[a][r];
      sc += cv[r] * g.c[a][r];
    }
    be[a] = sb;
    ga[a] = sc;
  }
  be[0] = -be[1];
  ga[0] = -ga[1];
#pragma unroll
  for (int a = 2; a < NV; ++a) {
    be[0] -= be[a];
    ga[0] -= ga[a];
  }
  T u[NV], w[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    u[a] = cs * ga[a] + m;
    w[a] = -cs * be[a];
  }
#pragma unroll
  for (int a = 0; a < NV; ++a) out.diag[a] = P[a][a] + u[a] + w[a] + m;
#pragma unroll
  for (int p = 0; p < Pairs<D>::n; ++p) {
    const int a = Pairs<D>::a(p), b = Pairs<D>::b(p);
    out.lo[p] = P[a][b] + u[b] + w[a];
    out.hi[p] = P[b][a] + u[a] + w[b];
  }
}

// Local matrix with P1 coefficients: record vid[v] of coef belongs to corner v. The
// corners are visited one at a time, keeping only the dot products the entries need:
// Mb[a][v] = c_a . b(v), Nc[a][v] = c_a . c(v) (row 0 from sum_a c_a = 0).
template <int D, class T, class R = T>
__device__ __forceinline__ void general_values_p1(const Geo<D, T>& g, const R* __restrict__ coef, bool vec,
                                                  const int32_t vid[D + 1], GeneralVals<D, T>& out) {
  constexpr int NV = D + 1;
  T As[D * D], a0v[NV], Mb[NV][NV], Nc[NV][NV];
#pragma unroll
  for (int j = 0; j < D * D; ++j) As[j] = T(0);
  T a0s = T(0);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T cf[GenCoef<D>::n];
    load_coef<D, T, R>(coef + (int64_t)vid[v] * GenCoef<D>::n, vec, cf);
#pragma unroll
    for (int j = 0; j < D * D; ++j) As[j] += cf[j];
    const T* bb = cf + D * D;
    const T* cc = cf + D * D + D;
    a0v[v] = cf[D * D + 2 * D];
    a0s += a0v[v];
#pragma unroll
    for (int a = 1; a < NV; ++a) {
      T sb = g.c[a][0] * bb[0], sc = g.c[a][0] * cc[0];
#pragma unroll
      for (int r = 1; r < D; ++r) {
        sb += g.c[a][r] * bb[r];
        sc += g.c[a][r] * cc[r];
      }
      Mb[a][v] = sb;
      Nc[a][v] = sc;
    }
    T m0 = -Mb[1][v], n0 = -Nc[1][v];
#pragma unroll
    for (int a = 2; a < NV; ++a) {
      m0 -= Mb[a][v];
      n0 -= Nc[a][v];
    }
    Mb[0][v] = m0;
    Nc[0][v] = n0;
  }
  const T adet = tabs(g.det);
  const T inv = recip<T>(T(factorial(D + 1)) * adet);
  const T cs = (g.det < T(0) ? T(-1) : T(1)) * T(1.0 / factorial(D + 2));
  const T mr = adet * T(1.0 / factorial(D + 3));
#pragma unroll
  for (int j = 0; j < D * D; ++j) As[j] *= inv;
  T P[NV][NV];
  diffusion_block<D, T>(g, As, P);
  // E_ab = P_ab + cs (c_b.c^s + c_b.c(a) - c_a.b^s - c_a.b(b)) + mr (1 + delta_ab)(a0^s + a0(a) + a0(b))
  //      = P_ab + U_b + W_a + cs (Nc[b][a] - Mb[a][b])  (+ mr (a0^s + 2 a0(a)) on the diagonal)
  const T r0 = mr * a0s;
  T U[NV], W[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    T bs = Mb[a][0], cc = Nc[a][0];
#pragma unroll
    for (int v = 1; v < NV; ++v) {
      bs += Mb[a][v];
      cc += Nc[a][v];
    }
    const T ra = mr * a0v[a];
    U[a] = cs * cc + ra;
    W[a] = -cs * bs + (ra + r0);
  }
#pragma unroll
  for (int a = 0; a < NV; ++a)
    out.diag[a] = cs * (Nc[a][a] - Mb[a][a]) + (P[a][a] + U[a] + W[a]) + (r0 + T(2) * mr * a0v[a]);
#pragma unroll
  for (int p = 0; p < Pairs<D>::n; ++p) {
    const int a = Pairs<D>::a(p), b = Pairs<D>::b(p);
    out.lo[p] = cs * (Nc[b][a] - Mb[a][b]) + (P[a][b] + U[b] + W[a]);
    out.hi[p] = cs * (Nc[a][b] - Mb[b][a]) + (P[b][a] + U[a] + W[b]);
  }
}

template <class T>
struct Vec2;
template <>
struct Vec2<double> { using type = double2; };
template <>
struct Vec2<float> { using type = float2; };

struct GeneralArgs {
  int64_t nme, nq;
  int chunk;
  uint32_t rec_max, max_lv;
  const double* q;
  const void* coef;
  int coef_kind;
  bool vec;  // coef is 16-byte aligned
  const int32_t* order;
  const int32_t* ch_v_ptr;
  const int32_t* ch_e_ptr;
  const uint8_t* rec;
  const uint32_t* rec_off16;
  int64_t npart;  // the second orientation of edge partial i is at npart + i
  fe_status_word* st;
  int64_t nnz;    // size of vals (bounds-checked builds)
  const int32_t* me0;  // F64X form: corner 0 of each internal element (chunk reference vertex)
};

// One block per chunk, as the symmetric staged kernel: plan record by one bulk copy,
// vertex coordinates staged once, element values into shared memory, then fixed-order
// sums per distinct vertex and, for each distinct edge, one sum per orientation.
template <int D, class T, int THREADS, bool P1>
__global__ void __launch_bounds__(THREADS) k_chunk_general(GeneralArgs A, T* __restrict__ vals,
                                                           void* __restrict__ partials) {
  constexpr int NV = D + 1, NP = Pairs<D>::n;
  using T2 = typename Vec2<T>::type;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  const int64_t c = blockIdx.x;
  const int64_t e0 = c * A.chunk;
  const int ne = (int)min((int64_t)A.chunk, A.nme - e0);
  const int32_t nlv = A.ch_v_ptr[c + 1] - A.ch_v_ptr[c];
  const int32_t nle = A.ch_e_ptr[c + 1] - A.ch_e_ptr[c];
  const RecLayout R = rec_layout((uint32_t)ne, NV, NP, (uint32_t)nlv, (uint32_t)nle);
  const StagedSmem S = general_smem(D, (int)sizeof(T), A.rec_max, A.max_lv, A.chunk);
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
  T2* Ko = (T2*)(smem + S.ko);
  if (!FE_RECORD_VALID(smem, R, ne, NV, NP, nlv, nle, 1, A.nq, A.nnz, A.npart, A.st, c)) return;

  for (int u = threadIdx.x; u < nlv; u += THREADS) {
    stage_vertex<D, T>(A.q, A.nq, lv_vid[u], smem + S.q, u, xr.ptr());
  }
  __syncthreads();

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
    GeneralVals<D, T> v;
    if constexpr (P1) {
      int32_t vid[NV];
#pragma unroll
      for (int a = 0; a < NV; ++a) vid[a] = lv_vid[lv[a]];
      general_values_p1<D, T>(g, (const T*)A.coef, A.vec, vid, v);
    } else {
      T cf[GenCoef<D>::n];
      general_coef<D, T>((const T*)A.coef, A.coef_kind, A.vec, A.order, e0 + el, cf);
      general_values<D, T>(g, cf, v);
    }
#pragma unroll
    for (int a = 0; a < NV; ++a) Kd[el * NV + a] = v.diag[a];
#pragma unroll
    for (int p = 0; p < NP; ++p) Ko[el * NP + p] = T2{v.lo[p], v.hi[p]};
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
  // edge u joins global vertices i < j: sum lo goes to (i, j), sum hi to (j, i). An
  // incidence whose pair (a, b) has me(a) > me(b) (orientation bit set) swaps E_ab, E_ba.
  for (int u = threadIdx.x; u < nle; u += THREADS) {
    const int s = le_off[u], t = le_off[u + 1];
    const int x0 = inc_e[s];
    const T2 v0 = Ko[x0 >> 1];
    Acc<T> lo((x0 & 1) ? v0.y : v0.x), hi((x0 & 1) ? v0.x : v0.y);
    for (int j = s + 1; j < t; ++j) {
      const int x = inc_e[j];
      const T2 v = Ko[x >> 1];
      lo.add((x & 1) ? v.y : v.x);
      hi.add((x & 1) ? v.x : v.y);
    }
    const int32_t dst = le_dst[2 * u];
    if (dst >= 0) {
      vals[dst] = lo.value();
      vals[le_dst[2 * u + 1]] = hi.value();
    } else {
      const int64_t pi = -1 - (int64_t)dst;
      lo.store_partial(partials, pi);
      hi.store_partial(partials, A.npart + pi);
    }
  }
}

// Chunk-order sums of the partials of each shared vertex (one destination) and edge
// (two: (i, j) from partials [s, t), (j, i) from [npart + s, npart + t)).
template <class T, class AccT = Acc<T>>
__global__ void k_fixup_general(const int32_t* __restrict__ sh_ptr, const int32_t* __restrict__ sh_dst,
                                int64_t nsh_v, int64_t nsh, int64_t npart,
                                const void* __restrict__ partials, T* __restrict__ vals, int64_t nnz,
                                fe_status_word* st) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= nsh) return;
  const int32_t s = sh_ptr[g], t = sh_ptr[g + 1];
  if (!FE_FIXUP_VALID(s, t, npart, sh_dst[2 * g], sh_dst[2 * g + 1], g >= nsh_v, nnz, st, g)) return;
  AccT acc = AccT::from_partial(partials, s);
  for (int32_t i = s + 1; i < t; ++i) acc.add_partial(partials, i);
  vals[sh_dst[2 * g]] = acc.value();
  if (g >= nsh_v) {
    AccT acc2 = AccT::from_partial(partials, npart + s);
    for (int32_t i = s + 1; i < t; ++i) acc2.add_partial(partials, npart + i);
    vals[sh_dst[2 * g + 1]] = acc2.value();
  }
}

// local matrix of internal element e with coordinates gathered from global memory
template <int D, class T, bool P1>
__device__ __forceinline__ void general_element(const ElemArgs& A, bool vec, int64_t e, GeneralVals<D, T>& v) {
  int32_t vid[D + 1];
  Geo<D, T> g;
  element_geo<D, T>(A, e, vid, g);
  if constexpr (P1) {
    general_values_p1<D, T>(g, (const T*)A.w, vec, vid, v);
  } else {
    T cf[GenCoef<D>::n];
    general_coef<D, T>((const T*)A.w, A.w_kind, vec, A.order, e, cf);
    general_values<D, T>(g, cf, v);
  }
}

// two-pass strategy, pass 1: E_ab at kg[e*S + b*NV + a], the slot of (row a, column b)
template <int D, class T, bool P1>
__global__ void __launch_bounds__(256) k_general_kg(ElemArgs A, bool vec, T* __restrict__ kg) {
  constexpr int NV = D + 1, S = NV * NV;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= A.nme) return;
  GeneralVals<D, T> v;
  general_element<D, T, P1>(A, vec, e, v);
  T* k = kg + e * S;
#pragma unroll
  for (int a = 0; a < NV; ++a) k[a * NV + a] = v.diag[a];
#pragma unroll
  for (int p = 0; p < Pairs<D>::n; ++p) {
    const int a = Pairs<D>::a(p), b = Pairs<D>::b(p);
    k[b * NV + a] = v.lo[p];
    k[a * NV + b] = v.hi[p];
  }
}

template <int D, class T, bool P1>
__global__ void __launch_bounds__(256) k_general_atomic(ElemArgs A, bool vec, const int32_t* __restrict__ slot2nnz,
                                                        T* __restrict__ vals) {
  constexpr int NV = D + 1, S = NV * NV;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= A.nme) return;
  GeneralVals<D, T> v;
  general_element<D, T, P1>(A, vec, e, v);
  const int32_t* m = slot2nnz + e * S;
#pragma unroll
  for (int a = 0; a < NV; ++a) atomicAdd(vals + m[a * NV + a], v.diag[a]);
#pragma unroll
  for (int p = 0; p < Pairs<D>::n; ++p) {
    const int a = Pairs<D>::a(p), b = Pairs<D>::b(p);
    atomicAdd(vals + m[b * NV + a], v.lo[p]);
    atomicAdd(vals + m[a * NV + b], v.hi[p]);
  }
}

template <int D, class T, int THREADS, bool P1>
int launch_general(fe_pattern_s* h, const ElemArgs& E, T* vals, cudaStream_t s) {
  const bool vec = ((uintptr_t)E.w & 15u) == 0;
  if (h->strategy == FE_REASM_CHUNKED) {
    const StagedSmem L = general_smem(D, (int)sizeof(T), (uint32_t)h->rec_max_bytes, (uint32_t)h->max_lv,
                                      (uint32_t)h->chunk);
    if (L.total > kSmemDynMax) return FE_ERR_ARG;
    GeneralArgs G{h->nme, h->nq, h->chunk, (uint32_t)h->rec_max_bytes, (uint32_t)h->max_lv, E.q, E.w,
                  E.w_kind, vec, h->order, h->ch_v_ptr, h->ch_e_ptr, h->rec, h->rec_off16, h->npart, h->status,
                  h->nnz_s, h->me_int};
    auto kern = k_chunk_general<D, T, THREADS, P1>;
    FE_TRY(fe_smem_limit(kern, L.total));
    FE_PROF_BEGIN(h, FE_K_CHUNK, s);
    kern<<<(unsigned)h->nchunks, THREADS, L.total, s>>>(G, vals, h->partials);
    FE_CUDA_TRY(cudaGetLastError());
    FE_PROF_END(h, FE_K_CHUNK, s);
    const int64_t nsh = h->nsh_v + h->nsh_e;
    if (nsh > 0) {
      FE_PROF_BEGIN(h, FE_K_FIXUP, s);
      k_fixup_general<T><<<fe_grid(nsh, 256), 256, 0, s>>>(h->sh_ptr, h->sh_dst, h->nsh_v, nsh, h->npart,
                                                          h->partials, vals, h->nnz_s, h->status);
      FE_CUDA_TRY(cudaGetLastError());
      FE_PROF_END(h, FE_K_FIXUP, s);
    }
  } else if (h->strategy == FE_REASM_GATHER) {
    T* kg = (T*)h->kg;
    FE_PROF_BEGIN(h, FE_K_ELEM_KG, s);
    k_general_kg<D, T, P1><<<fe_grid(h->nme, 256), 256, 0, s>>>(E, vec, kg);
    FE_CUDA_TRY(cudaGetLastError());
    FE_PROF_END(h, FE_K_ELEM_KG, s);
    FE_PROF_BEGIN(h, FE_K_GATHER, s);
    k_gather<T><<<fe_grid(h->nnz_s, 256), 256, 0, s>>>(h->nnz_slot_ptr, h->nnz2slot, h->nnz_s, kg, vals);
    FE_CUDA_TRY(cudaGetLastError());
    FE_PROF_END(h, FE_K_GATHER, s);
  } else {
    FE_PROF_BEGIN(h, FE_K_MEMSET, s);
    FE_CUDA_TRY(cudaMemsetAsync(vals, 0, sizeof(T) * h->nnz_s, s));
    FE_PROF_END(h, FE_K_MEMSET, s);
    FE_PROF_BEGIN(h, FE_K_ATOMIC, s);
    k_general_atomic<D, T, P1><<<fe_grid(h->nme, 256), 256, 0, s>>>(E, vec, h->slot2nnz, vals);
    FE_CUDA_TRY(cudaGetLastError());
    FE_PROF_END(h, FE_K_ATOMIC, s);
  }
  return FE_OK;
}

template <int D, class T, bool P1>
int launch_general_threads(fe_pattern_s* h, const ElemArgs& E, T* vals, cudaStream_t s) {
  if (h->strategy != FE_REASM_CHUNKED || h->threads == 256) return launch_general<D, T, 256, P1>(h, E, vals, s);
  if (h->threads == 128) return launch_general<D, T, 128, P1>(h, E, vals, s);
  return launch_general<D, T, 512, P1>(h, E, vals, s);
}

template <int D, class T>
int launch_general_dim(fe_pattern_s* h, const ElemArgs& E, T* vals, cudaStream_t s) {
  if (E.w_kind == FE_COEF_P1) return launch_general_threads<D, T, true>(h, E, vals, s);
  return launch_general_threads<D, T, false>(h, E, vals, s);
}

template <class T>
int launch_general_prec(fe_pattern_s* h, const double* q, const void* coef, int coef_kind, T* vals,
                        cudaStream_t s) {
  ElemArgs E{h->me_int, h->nme, h->nq, q, nullptr, coef, coef_kind, h->order, h->status};
  if (sizeof(T) == 4 && h->strategy != FE_REASM_CHUNKED) {
    float4* qs = (float4*)h->qsplit;
    FE_PROF_BEGIN(h, FE_K_SPLIT, s);
    if (h->d == 3) k_split_q<3><<<fe_grid(h->nq, 256), 256, 0, s>>>(q, h->nq, qs);
    else k_split_q<2><<<fe_grid(h->nq, 256), 256, 0, s>>>(q, h->nq, qs);
    FE_CUDA_TRY(cudaGetLastError());
    FE_PROF_END(h, FE_K_SPLIT, s);
    E.qs = qs;
  }
  if (h->d == 3) return launch_general_dim<3, T>(h, E, vals, s);
  return launch_general_dim<2, T>(h, E, vals, s);
}

// ---------------------------------------------------------------- FE_F64X form
// The chunked kernel with double-float element values (general_values over dfx) from
// coordinates relative to the chunk's reference vertex, double-float sums, double
// values; coefficient records are double. Chunked strategy only.
template <int D, int THREADS, bool P1>
__global__ void __launch_bounds__(THREADS, P1 ? 2 : 3) k_chunk_general_x(GeneralArgs A, double* __restrict__ vals,
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
  const StagedSmem S = general_smem(D, 8, A.rec_max, A.max_lv, A.chunk);
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
  float4* Ko = (float4*)(smem + S.ko);  // (E_ab, E_ba) of each element pair as two float pairs
  if (!FE_RECORD_VALID(smem, R, ne, NV, NP, nlv, nle, 1, A.nq, A.nnz, A.npart, A.st, c)) return;

  for (int u = threadIdx.x; u < nlv; u += THREADS) {
    x64_stage_vertex<D>(A.q, A.nq, lv_vid[u], xr, smem + S.q, u);
  }
  __syncthreads();

  for (int el = threadIdx.x; el < ne; el += THREADS) {
    int lv[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) lv[a] = lvid[el * NV + a];
    df cfv[D][D];
    df det = x64_geometry_guarded<D>(smem + S.q, lv, cfv, A.q, A.nq, lv_vid);
    if (df_degenerate(det)) {
      fe_report(A.st, FE_ERR_DEGENERATE, A.order[e0 + el]);
      det = df{1.f, 0.f};
    }
    Geo<D, dfx> g;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int i = 0; i < D; ++i) g.c[a + 1][i] = cfv[a][i];
    g.det = det;
    GeneralVals<D, dfx> v;
    if constexpr (P1) {
      int32_t vid[NV];
#pragma unroll
      for (int a = 0; a < NV; ++a) vid[a] = lv_vid[lv[a]];
      general_values_p1<D, dfx, double>(g, (const double*)A.coef, A.vec, vid, v);
    } else {
      dfx cf[GenCoef<D>::n];
      general_coef<D, dfx, double>((const double*)A.coef, A.coef_kind, A.vec, A.order, e0 + el, cf);
      general_values<D, dfx>(g, cf, v);
    }
#pragma unroll
    for (int a = 0; a < NV; ++a) Kd[el * NV + a] = make_float2(v.diag[a].hi, v.diag[a].lo);
#pragma unroll
    for (int p = 0; p < NP; ++p) Ko[el * NP + p] = make_float4(v.lo[p].hi, v.lo[p].lo, v.hi[p].hi, v.hi[p].lo);
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
    const int x0 = inc_e[s];
    const float4 v0 = Ko[x0 >> 1];
    const df a0{v0.x, v0.y}, b0{v0.z, v0.w};
    AccX lo((x0 & 1) ? b0 : a0), hi((x0 & 1) ? a0 : b0);
    for (int j = s + 1; j < t; ++j) {
      const int x = inc_e[j];
      const float4 v = Ko[x >> 1];
      const df a{v.x, v.y}, b{v.z, v.w};
      lo.add((x & 1) ? b : a);
      hi.add((x & 1) ? a : b);
    }
    const int32_t dst = le_dst[2 * u];
    if (dst >= 0) {
      vals[dst] = lo.value();
      vals[le_dst[2 * u + 1]] = hi.value();
    } else {
      const int64_t pi = -1 - (int64_t)dst;
      lo.store_partial(partials, pi);
      hi.store_partial(partials, A.npart + pi);
    }
  }
}

template <int D, bool P1>
int launch_general_x(fe_pattern_s* h, const double* q, const void* coef, int coef_kind, double* vals,
                     cudaStream_t s) {
  constexpr int THREADS = 256;
  if (h->strategy != FE_REASM_CHUNKED) return FE_ERR_ARG;
  const StagedSmem L = general_smem(D, 8, (uint32_t)h->rec_max_bytes, (uint32_t)h->max_lv, (uint32_t)h->chunk);
  if (L.total > kSmemDynMax) return FE_ERR_ARG;
  const bool vec = ((uintptr_t)coef & 15u) == 0;
  GeneralArgs G{h->nme, h->nq, h->chunk, (uint32_t)h->rec_max_bytes, (uint32_t)h->max_lv, q, coef, coef_kind,
                vec, h->order, h->ch_v_ptr, h->ch_e_ptr, h->rec, h->rec_off16, h->npart, h->status, h->nnz_s,
                h->me_int};
  auto kern = k_chunk_general_x<D, THREADS, P1>;
  FE_TRY(fe_smem_limit(kern, L.total));
  FE_PROF_BEGIN(h, FE_K_CHUNK, s);
  kern<<<(unsigned)h->nchunks, THREADS, L.total, s>>>(G, vals, (float2*)h->partials);
  FE_CUDA_TRY(cudaGetLastError());
  FE_PROF_END(h, FE_K_CHUNK, s);
  const int64_t nsh = h->nsh_v + h->nsh_e;
  if (nsh > 0) {
    FE_PROF_BEGIN(h, FE_K_FIXUP, s);
    k_fixup_general<double, AccX><<<fe_grid(nsh, 256), 256, 0, s>>>(h->sh_ptr, h->sh_dst, h->nsh_v, nsh,
                                                                   h->npart, h->partials, vals, h->nnz_s,
                                                                   h->status);
    FE_CUDA_TRY(cudaGetLastError());
    FE_PROF_END(h, FE_K_FIXUP, s);
  }
  return FE_OK;
}

int launch_general_f64x(fe_pattern_s* h, const double* q, const void* coef, int coef_kind, double* vals,
                        cudaStream_t s) {
  const bool p1 = coef_kind == FE_COEF_P1;
  if (h->d == 3)
    return p1 ? launch_general_x<3, true>(h, q, coef, coef_kind, vals, s)
              : launch_general_x<3, false>(h, q, coef, coef_kind, vals, s);
  return p1 ? launch_general_x<2, true>(h, q, coef, coef_kind, vals, s)
            : launch_general_x<2, false>(h, q, coef, coef_kind, vals, s);
}

}  // namespace
}  // namespace fe

int fe_launch_general(fe_pattern_s* h, const double* q, const void* coef, int coef_kind, int prec,
                      void* vals, cudaStream_t s) {
  if (prec == FE_F64X) return fe::launch_general_f64x(h, q, coef, coef_kind, (double*)vals, s);
  if (prec == FE_F64) return fe::launch_general_prec<double>(h, q, coef, coef_kind, (double*)vals, s);
  return fe::launch_general_prec<float>(h, q, coef, coef_kind, (float*)vals, s);
}
