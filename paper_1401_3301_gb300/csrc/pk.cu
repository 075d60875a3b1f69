// P_k Lagrange mass matrix (App. D): the nodes of each element are the points
// sum_i alpha_i q^i / k of its principal lattice, alpha in S_d^k, and by Eq. MatElemMassPk
//   int_K phi_alpha phi_beta = d! |K| C_{alpha,beta} = |det B| C_{alpha,beta}
// with constants C that do not depend on K. The host computes C once per (d, k) in exact
// integer arithmetic; the chunk kernel then needs |det B| per element and sums
// |det B| C_ab over the incidences of each distinct node and node pair (the plan of the
// P1 operators with nv = ndfe nodes per element).
//
// Local node order: the d+1 vertices k e_0, ..., k e_d first, then the other multi-indices
// in lexicographically decreasing order; node pairs (a, b), a < b, lexicographically.
#include <string.h>

#include <array>
#include <vector>

#include "assemble_impl.cuh"
#include "dfloat.cuh"
#include "profile.cuh"

namespace fe {
namespace {

typedef __int128 i128;

constexpr int binom(int n, int r) { return r == 0 ? 1 : binom(n - 1, r - 1) * n / r; }

// multi-indices of S_d^k in the local node order
std::vector<std::array<int, 4>> node_order(int d, int k) {
  std::vector<std::array<int, 4>> all, out;
  std::array<int, 4> a{};
  // lexicographically decreasing: the first entry from k down, then the rest recursively
  auto rec = [&](auto&& self, int pos, int left) -> void {
    if (pos == d) {
      a[pos] = left;
      all.push_back(a);
      return;
    }
    for (int x = left; x >= 0; --x) {
      a[pos] = x;
      self(self, pos + 1, left - x);
    }
  };
  rec(rec, 0, k);
  auto is_vertex = [&](const std::array<int, 4>& v) {
    for (int i = 0; i <= d; ++i)
      if (v[i] == k) return true;
    return false;
  };
  for (int i = 0; i <= d; ++i) {
    std::array<int, 4> v{};
    v[i] = k;
    out.push_back(v);
  }
  for (const auto& v : all)
    if (!is_vertex(v)) out.push_back(v);
  return out;
}

i128 fact(int n) {
  i128 r = 1;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

i128 gcd128(i128 a, i128 b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b != 0) {
    const i128 t = a % b;
    a = b;
    b = t;
  }
  return a;
}

// Expansion of phi_alpha (Eq. Pk:functions) in barycentric monomials, as integer
// numerators over the common denominator prod_l alpha_l!: for each l the integer
// coefficients of prod_{j < alpha_l} (k lambda_l - j), then all products of one term per l.
struct Expansion {
  std::vector<std::array<int, 4>> mu;
  std::vector<int64_t> num;
  int64_t den;
};

Expansion expand(const std::array<int, 4>& alpha, int d, int k) {
  std::vector<std::vector<int64_t>> coef(d + 1);
  int64_t den = 1;
  for (int l = 0; l <= d; ++l) {
    std::vector<int64_t> c{1};
    for (int j = 0; j < alpha[l]; ++j) {  // times (k lambda - j)
      std::vector<int64_t> nxt(c.size() + 1, 0);
      for (size_t t = 0; t < c.size(); ++t) {
        nxt[t + 1] += (int64_t)k * c[t];
        nxt[t] -= (int64_t)j * c[t];
      }
      c.swap(nxt);
      den *= (j + 1);
    }
    coef[l] = c;
  }
  Expansion E;
  E.den = den;
  std::array<int, 4> m{};
  auto rec = [&](auto&& self, int l, int64_t prod) -> void {
    if (l > d) {
      if (prod != 0) {
        E.mu.push_back(m);
        E.num.push_back(prod);
      }
      return;
    }
    for (int t = 0; t <= alpha[l]; ++t) {
      m[l] = t;
      self(self, l + 1, prod * coef[l][t]);
    }
    m[l] = 0;
  };
  rec(rec, 0, 1);
  return E;
}

// C_{alpha,beta} = sum_{mu,nu} a_mu(alpha) a_nu(beta) prod_i (mu_i + nu_i)! / (d + |mu| + |nu|)!,
// summed exactly over the common denominator (d + 2k)! prod alpha! prod beta!, then
// rounded once per numerator and denominator.
void mass_table(int d, int k, std::vector<double>& C) {
  const auto al = node_order(d, k);
  const int n = (int)al.size();
  std::vector<Expansion> ex;
  for (const auto& a : al) ex.push_back(expand(a, d, k));
  const i128 top = fact(d + 2 * k);
  C.assign((size_t)n * n, 0.0);
  for (int a = 0; a < n; ++a)
    for (int b = a; b < n; ++b) {
      i128 s = 0;
      const Expansion& A = ex[a];
      const Expansion& B = ex[b];
      for (size_t i = 0; i < A.mu.size(); ++i)
        for (size_t j = 0; j < B.mu.size(); ++j) {
          i128 t = (i128)A.num[i] * B.num[j];
          int deg = 0;
          for (int l = 0; l <= d; ++l) {
            const int e = A.mu[i][l] + B.mu[j][l];
            t *= fact(e);
            deg += e;
          }
          t *= top / fact(d + deg);
          s += t;
        }
      i128 den = top * A.den * B.den;
      const i128 g = gcd128(s, den);
      if (g > 1) {
        s /= g;
        den /= g;
      }
      const double v = (double)s / (double)den;
      C[(size_t)a * n + b] = v;
      C[(size_t)b * n + a] = v;
    }
}

struct PkArgs {
  int64_t nme, nq;
  int chunk;
  uint32_t rec_max;
  const double* q;
  const void* tab;  // diagonal C_aa (nv), then pairs C_ab (npair)
  const int32_t* order;
  const int32_t* ch_v_ptr;
  const int32_t* ch_e_ptr;
  const uint8_t* rec;
  const uint32_t* rec_off16;
  fe_status_word* st;
  int64_t nnz, npart;  // sizes of vals and of the partial sums (bounds-checked builds)
};

// One block per chunk: the plan record by one bulk copy, the table and the element
// node -> local node map into shared memory, |det B| per element from the FP64
// coordinates of its d+1 vertices (its first d+1 nodes), then the fixed-order sums of
// |det B| C over the incidences of each distinct node (diagonal) and node pair.
// X (FE_F64X form, T = double): |det B| and the table as double-float pairs in shared
// memory, products and sums in double-float, double values, float2 partials.
template <int D, int K, class T, int THREADS, bool X = false>
__global__ void __launch_bounds__(THREADS) k_chunk_pk(PkArgs A, T* __restrict__ vals, void* __restrict__ partials) {
  constexpr int NV = binom(D + K, K), NP = NV * (NV - 1) / 2;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  const int64_t c = blockIdx.x;
  const int64_t e0 = c * A.chunk;
  const int ne = (int)min((int64_t)A.chunk, A.nme - e0);
  const int32_t nlv = A.ch_v_ptr[c + 1] - A.ch_v_ptr[c];
  const int32_t nle = A.ch_e_ptr[c + 1] - A.ch_e_ptr[c];
  const RecLayout R = rec_layout((uint32_t)ne, NV, NP, (uint32_t)nlv, (uint32_t)nle);
  const PkSmem S = pk_smem(NV, NP, (int)sizeof(T), A.rec_max, (uint32_t)A.chunk);
  if (!FE_CHUNK_FITS(R.total <= A.rec_max, A.st, c)) return;
  if (!load_plan_record(smem, &bar, A.rec, A.rec_off16, c, R.total, A.st, e0, kBarrierSpin)) return;
  const uint16_t* inc_v = (const uint16_t*)(smem + R.inc_v);
  const uint16_t* inc_e = (const uint16_t*)(smem + R.inc_e);
  const uint16_t* lv_off = (const uint16_t*)(smem + R.lv_off);
  const uint16_t* le_off = (const uint16_t*)(smem + R.le_off);
  const int32_t* lv_vid = (const int32_t*)(smem + R.lv_vid);
  const int32_t* lv_dst = (const int32_t*)(smem + R.lv_dst);
  const int32_t* le_dst = (const int32_t*)(smem + R.le_dst);
  const uint16_t* lvid = (const uint16_t*)(smem + R.lvid);
  T* Sc = (T*)(smem + S.sc);
  T* tab = (T*)(smem + S.tab);
  float2* Sx = (float2*)(smem + S.sc);   // X: |det B| pairs
  float2* tabx = (float2*)(smem + S.tab);  // X: table pairs
  if (!FE_RECORD_VALID(smem, R, ne, NV, NP, nlv, nle, 1, A.nq, A.nnz, A.npart, A.st, c)) return;

  for (int i = threadIdx.x; i < NV + NP; i += THREADS) {
    if constexpr (X) {
      const df v = df_split(((const double*)A.tab)[i]);
      tabx[i] = make_float2(v.hi, v.lo);
    } else {
      tab[i] = ((const T*)A.tab)[i];
    }
  }
  __syncthreads();

  for (int el = threadIdx.x; el < ne; el += THREADS) {
    double x[D + 1][D];
#pragma unroll
    for (int a = 0; a <= D; ++a) {
      const int64_t vid = lv_vid[lvid[el * NV + a]];
#pragma unroll
      for (int k = 0; k < D; ++k) x[a][k] = __ldg(A.q + k * A.nq + vid);
    }
    double e[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int k = 0; k < D; ++k) e[i][k] = x[i + 1][k] - x[0][k];
    double det;
    if constexpr (D == 3)
      det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) + e[0][1] * (e[1][2] * e[2][0] - e[1][0] * e[2][2]) +
            e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
    else
      det = e[0][0] * e[1][1] - e[0][1] * e[1][0];
    if (!det_ok(det)) {
      fe_report(A.st, FE_ERR_DEGENERATE, A.order[e0 + el]);
      det = 1.0;
    }
    if constexpr (X) {
      const df v = df_split(fabs(det));
      Sx[el] = make_float2(v.hi, v.lo);
    } else {
      Sc[el] = (T)fabs(det);
    }
  }
  __syncthreads();

  if constexpr (X) {
    auto term = [&](int el, int k) {
      const float2 a = Sx[el], b = tabx[k];
      return df_mul_full(df{a.x, a.y}, df{b.x, b.y});
    };
    for (int u = threadIdx.x; u < nlv; u += THREADS) {
      const int s = lv_off[u], t = lv_off[u + 1];
      AccX acc(term(inc_v[s] / NV, inc_v[s] % NV));
      for (int j = s + 1; j < t; ++j) acc.add(term(inc_v[j] / NV, inc_v[j] % NV));
      const int32_t dst = lv_dst[u];
      if (dst >= 0) vals[dst] = acc.value();
      else acc.store_partial(partials, -1 - (int64_t)dst);
    }
    for (int u = threadIdx.x; u < nle; u += THREADS) {
      const int s = le_off[u], t = le_off[u + 1];
      const int i0 = inc_e[s] >> 1;
      AccX acc(term(i0 / NP, NV + i0 % NP));
      for (int j = s + 1; j < t; ++j) {
        const int i = inc_e[j] >> 1;
        acc.add(term(i / NP, NV + i % NP));
      }
      const int32_t dst = le_dst[2 * u];
      if (dst >= 0) {
        const double v = acc.value();
        vals[dst] = v;
        vals[le_dst[2 * u + 1]] = v;
      } else {
        acc.store_partial(partials, -1 - (int64_t)dst);
      }
    }
  } else {
    for (int u = threadIdx.x; u < nlv; u += THREADS) {
      const int s = lv_off[u], t = lv_off[u + 1];
      const int x0 = inc_v[s];
      Acc<T> acc(Sc[x0 / NV] * tab[x0 % NV]);
      for (int j = s + 1; j < t; ++j) {
        const int x = inc_v[j];
        acc.add(Sc[x / NV] * tab[x % NV]);
      }
      const int32_t dst = lv_dst[u];
      if (dst >= 0) vals[dst] = acc.value();
      else acc.store_partial(partials, -1 - (int64_t)dst);
    }
    for (int u = threadIdx.x; u < nle; u += THREADS) {
      const int s = le_off[u], t = le_off[u + 1];
      const int i0 = inc_e[s] >> 1;
      Acc<T> acc(Sc[i0 / NP] * tab[NV + i0 % NP]);
      for (int j = s + 1; j < t; ++j) {
        const int i = inc_e[j] >> 1;
        acc.add(Sc[i / NP] * tab[NV + i % NP]);
      }
      const int32_t dst = le_dst[2 * u];
      if (dst >= 0) {
        const T v = acc.value();
        vals[dst] = v;
        vals[le_dst[2 * u + 1]] = v;
      } else {
        acc.store_partial(partials, -1 - (int64_t)dst);
      }
    }
  }
}

template <int D, int K, class T, bool X = false>
int launch_pk(fe_pattern_s* h, const double* q, T* vals, cudaStream_t s) {
  constexpr int NV = binom(D + K, K), NP = NV * (NV - 1) / 2;
  constexpr int THREADS = 256;
  if (h->nv != NV || h->npair != NP) return FE_ERR_ARG;
  const PkSmem L = pk_smem(NV, NP, (int)sizeof(T), (uint32_t)h->rec_max_bytes, (uint32_t)h->chunk);
  if (L.total > kSmemDynMax) return FE_ERR_ARG;
  const void* tab = sizeof(T) == 8 ? h->pk_tab : (const void*)((const double*)h->pk_tab + NV + NP);
  PkArgs A{h->nme, h->nq, h->chunk, (uint32_t)h->rec_max_bytes, q, tab, h->order, h->ch_v_ptr, h->ch_e_ptr,
           h->rec, h->rec_off16, h->status, h->nnz_s, h->npart};
  auto kern = k_chunk_pk<D, K, T, THREADS, X>;
  FE_TRY(fe_smem_limit(kern, L.total));
  FE_PROF_BEGIN(h, FE_K_CHUNK, s);
  kern<<<(unsigned)h->nchunks, THREADS, L.total, s>>>(A, vals, h->partials);
  FE_CUDA_TRY(cudaGetLastError());
  FE_PROF_END(h, FE_K_CHUNK, s);
  const int64_t nsh = h->nsh_v + h->nsh_e;
  if (nsh > 0) {
    FE_PROF_BEGIN(h, FE_K_FIXUP, s);
    if constexpr (X)
      k_fixup_scalar<double, AccX><<<fixup_grid<double>(nsh), 256, 0, s>>>(h->sh_ptr, h->sh_dst, h->nsh_v, nsh,
                                                                    h->partials, vals, h->nnz_s, h->npart,
                                                                    h->status);
    else
      k_fixup_scalar<T><<<fixup_grid<T>(nsh), 256, 0, s>>>(h->sh_ptr, h->sh_dst, h->nsh_v, nsh, h->partials,
                                                          vals, h->nnz_s, h->npart, h->status);
    FE_CUDA_TRY(cudaGetLastError());
    FE_PROF_END(h, FE_K_FIXUP, s);
  }
  return FE_OK;
}

template <class T, bool X = false>
int launch_pk_prec(fe_pattern_s* h, const double* q, T* vals, cudaStream_t s) {
  const int key = h->d * 10 + h->pk;
  switch (key) {
    case 22: return launch_pk<2, 2, T, X>(h, q, vals, s);
    case 23: return launch_pk<2, 3, T, X>(h, q, vals, s);
    case 24: return launch_pk<2, 4, T, X>(h, q, vals, s);
    case 25: return launch_pk<2, 5, T, X>(h, q, vals, s);
    case 26: return launch_pk<2, 6, T, X>(h, q, vals, s);
    case 32: return launch_pk<3, 2, T, X>(h, q, vals, s);
    case 33: return launch_pk<3, 3, T, X>(h, q, vals, s);
    case 34: return launch_pk<3, 4, T, X>(h, q, vals, s);
    case 35: return launch_pk<3, 5, T, X>(h, q, vals, s);
    case 36: return launch_pk<3, 6, T, X>(h, q, vals, s);
    default: return FE_ERR_ARG;
  }
}

}  // namespace
}  // namespace fe

int fe_pk_nodes(int d, int k) {
  int n = 1;
  for (int i = 1; i <= d; ++i) n = n * (k + i) / i;
  return n;
}

// Device copy of the table in the kernel's layout: diagonal, then pairs (a < b,
// lexicographic), as double, followed by the same values as float.
int fe_pk_upload_table(fe_pattern_s* h, cudaStream_t s) {
  std::vector<double> C;
  fe::mass_table(h->d, h->pk, C);
  const int n = h->nv;
  std::vector<double> d64;
  for (int a = 0; a < n; ++a) d64.push_back(C[(size_t)a * n + a]);
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b) d64.push_back(C[(size_t)a * n + b]);
  const size_t m = d64.size();
  std::vector<unsigned char> buf(m * 12);
  memcpy(buf.data(), d64.data(), m * 8);
  for (size_t i = 0; i < m; ++i) {
    const float f = (float)d64[i];
    memcpy(buf.data() + m * 8 + i * 4, &f, 4);
  }
  FE_TRY(fe_malloc(h, &h->pk_tab, buf.size()));
  FE_CUDA_TRY(cudaMemcpyAsync(h->pk_tab, buf.data(), buf.size(), cudaMemcpyHostToDevice, s));
  FE_CUDA_TRY(cudaStreamSynchronize(s));  // buf is released on return
  return FE_OK;
}

int fe_launch_pk_mass(fe_pattern_s* h, const double* q, int prec, void* vals, cudaStream_t s) {
  if (h->strategy != FE_REASM_CHUNKED) return FE_ERR_ARG;
  if (prec == FE_F64X) return fe::launch_pk_prec<double, true>(h, q, (double*)vals, s);
  if (prec == FE_F64) return fe::launch_pk_prec<double>(h, q, (double*)vals, s);
  return fe::launch_pk_prec<float>(h, q, (float*)vals, s);
}

extern "C" int fe_pk_mass_table(int32_t d, int32_t k, double* C) {
  if (d < 2 || d > 3 || k < 1 || k > FE_PK_MAX || !C) return FE_ERR_ARG;
  std::vector<double> t;
  fe::mass_table(d, k, t);
  memcpy(C, t.data(), t.size() * sizeof(double));
  return FE_OK;
}
