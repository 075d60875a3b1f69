/*
 * fe_oracle.c -- plain FP64 reference ("oracle") for P1 finite element assembly.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file. The library's GPU path never
 * calls, links or includes it, and it shares no code with that path.
 *
 * What it computes, step by step, in the order of the paper
 * (Cuvelier, Japhet, Scarella, "An efficient way to assemble finite element
 * matrices in vector languages"):
 *   1. per element k: B_k with i-th column q^i - q^0 (App. C.1), the barycentric
 *      gradients G_k as the solution of B_k^T G_k = G^ (Eq. gradient:SystemeMat),
 *      solved here by Gaussian elimination with partial pivoting; det B_k from the
 *      pivots and |K| = |det B_k| / d!;
 *   2. the local matrix E(T_k) from its definition:
 *        mass / weighted mass: integrals of products of barycentric coordinates
 *          by the magic formula (Eq. MagicFormula), with w replaced by its P1
 *          interpolant (Section 4.1);
 *        stiffness: |K| <grad lambda_b, grad lambda_a> (Eq. stiffelemmat), times
 *          an optional per-element coefficient;
 *        elasticity: int eps(phi_j)^T C eps(phi_i) (Eq. StiffElasElem) with the
 *          strain vector order and Hooke matrix C of Section 5.1 and the Lame
 *          coefficients replaced by their P1 interpolants;
 *   3. the (Ig, Jg, Kg) triplets of all elements (Algorithm 2, column-wise local
 *      order), sorted by (row, column, element, local slot) and summed, which is
 *      the `sparse` constructor of Section 3. Entries whose sum is zero are kept.
 * Every step is a plain loop over elements; nothing is blocked or fused.
 *
 * Indices are 0-based; vector unknowns use the alternate numbering
 * dof = m * vertex + component (Section 5).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_INDEX 2
#define ORC_ERR_DEGENERATE 3
#define ORC_ERR_NOMEM 4

#define ORC_MASS 0
#define ORC_WMASS 1
#define ORC_STIFF 2
#define ORC_ELAS 3

/* coefficient kinds */
#define ORC_COEF_NONE 0   /* identically 1 */
#define ORC_COEF_SCALAR 1 /* one value */
#define ORC_COEF_P0 2     /* one value per element */
#define ORC_COEF_P1 3     /* one value per vertex, P1-interpolated */

/* Threads of the element loops and sorts (1 unless orc_set_threads is called on a build
 * with OpenMP). Every result is independent of it: each element writes its own
 * triplets, and the sort order is a total order. */
static int g_threads = 1;

int orc_openmp(void) {
#ifdef _OPENMP
  return 1;
#else
  return 0;
#endif
}

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }

/* Sort n records of `size` bytes by cmp: qsort, or with several threads, qsort of one
 * slice per thread and then rounds of pairwise merges of neighbouring sorted runs. */
static int sort_records(void* base, int64_t n, size_t size, int (*cmp)(const void*, const void*)) {
  int T = g_threads;
  if (T <= 1 || n < 2 * (int64_t)T) {
    qsort(base, (size_t)n, size, cmp);
    return ORC_OK;
  }
  char* a = (char*)base;
  char* b = (char*)malloc((size_t)n * size);
  if (!b) return ORC_ERR_NOMEM;
  int64_t* bound = (int64_t*)malloc(sizeof(int64_t) * (size_t)(T + 1));
  if (!bound) { free(b); return ORC_ERR_NOMEM; }
  for (int i = 0; i <= T; ++i) bound[i] = n * i / T;
#pragma omp parallel for num_threads(T) schedule(static, 1)
  for (int i = 0; i < T; ++i) qsort(a + bound[i] * size, (size_t)(bound[i + 1] - bound[i]), size, cmp);
  for (int width = 1; width < T; width *= 2) {
    const int pairs = (T + 2 * width - 1) / (2 * width);
#pragma omp parallel for num_threads(T) schedule(dynamic, 1)
    for (int pi = 0; pi < pairs; ++pi) {
      const int lo = pi * 2 * width, mid = lo + width < T ? lo + width : T;
      const int hi = lo + 2 * width < T ? lo + 2 * width : T;
      int64_t i = bound[lo], j = bound[mid], o = bound[lo];
      const int64_t ie = bound[mid], je = bound[hi];
      while (i < ie && j < je) {
        if (cmp(a + j * size, a + i * size) < 0) { memcpy(b + o * size, a + j * size, size); ++j; }
        else { memcpy(b + o * size, a + i * size, size); ++i; }
        ++o;
      }
      if (i < ie) memcpy(b + o * size, a + i * size, (size_t)(ie - i) * size), o += ie - i;
      if (j < je) memcpy(b + o * size, a + j * size, (size_t)(je - j) * size);
    }
    char* t = a; a = b; b = t;
  }
  if (a != (char*)base) {
    memcpy(base, a, (size_t)n * size);
    b = a;
  }
  free(b);
  free(bound);
  return ORC_OK;
}

static double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= (double)i;
  return f;
}

/* Eq. MagicFormula: int_K prod_i lambda_i^{n_i} = d! |K| prod_i n_i! / (d + sum_i n_i)! */
double orc_magic(int d, const int* n, double vol) {
  double num = 1.0;
  int s = 0;
  for (int i = 0; i < d + 1; ++i) {
    num *= factorial(n[i]);
    s += n[i];
  }
  return factorial(d) * vol * num / factorial(d + s);
}

/*
 * Geometry of one d-simplex (App. C.1). X holds the d+1 vertices, X[a*d + c] is
 * coordinate c of local vertex a. Output: det = det B, vol = |det B| / d!,
 * G[a*d + i] = d lambda_a / d x_i, found by solving B^T G = G^ with
 * G^ = [-1, I_d] by Gaussian elimination with partial pivoting.
 */
int orc_simplex(int d, const double* X, double* det, double* vol, double* G) {
  if (d < 1 || d > 3) return ORC_ERR_ARG;
  double A[3][3], R[3][4];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) A[i][j] = X[(i + 1) * d + j] - X[j]; /* A = B^T: A[i][j] = B[j][i] */
  for (int i = 0; i < d; ++i) {
    R[i][0] = -1.0;
    for (int a = 1; a <= d; ++a) R[i][a] = (a - 1 == i) ? 1.0 : 0.0;
  }
  double dt = 1.0;
  for (int c = 0; c < d; ++c) {
    int p = c;
    for (int r = c + 1; r < d; ++r)
      if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
    if (A[p][c] == 0.0) {
      *det = 0.0;
      *vol = 0.0;
      return ORC_ERR_DEGENERATE;
    }
    if (p != c) {
      for (int j = 0; j < d; ++j) { double t = A[c][j]; A[c][j] = A[p][j]; A[p][j] = t; }
      for (int a = 0; a <= d; ++a) { double t = R[c][a]; R[c][a] = R[p][a]; R[p][a] = t; }
      dt = -dt;
    }
    dt *= A[c][c];
    for (int r = c + 1; r < d; ++r) {
      double f = A[r][c] / A[c][c];
      for (int j = c; j < d; ++j) A[r][j] -= f * A[c][j];
      for (int a = 0; a <= d; ++a) R[r][a] -= f * R[c][a];
    }
  }
  for (int a = 0; a <= d; ++a) {
    double x[3];
    for (int i = d - 1; i >= 0; --i) {
      double s = R[i][a];
      for (int j = i + 1; j < d; ++j) s -= A[i][j] * x[j];
      x[i] = s / A[i][i];
    }
    for (int i = 0; i < d; ++i) G[a * d + i] = x[i];
  }
  *det = dt;
  *vol = fabs(dt) / factorial(d);
  if (!isfinite(dt) || !isfinite(*vol)) return ORC_ERR_DEGENERATE;
  return ORC_OK;
}

/* integral over K of the P1 interpolant of a field with vertex values f[0..d] */
static double p1_integral(int d, const double* f, double vol) {
  double s = 0.0;
  int n[4];
  for (int g = 0; g <= d; ++g) {
    for (int i = 0; i <= d; ++i) n[i] = (i == g);
    s += f[g] * orc_magic(d, n, vol);
  }
  return s;
}

/* strain vector of phi = lambda_a e_l, in the order of Section 5.1:
 * 2D (e11, e22, 2 e12), 3D (e11, e22, e33, 2 e12, 2 e23, 2 e13). */
static void strain_vector(int d, const double* ga, int l, double* eps) {
  double e[3][3];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) e[i][j] = 0.5 * ((i == l) * ga[j] + (j == l) * ga[i]);
  if (d == 2) {
    eps[0] = e[0][0]; eps[1] = e[1][1]; eps[2] = 2.0 * e[0][1];
  } else {
    eps[0] = e[0][0]; eps[1] = e[1][1]; eps[2] = e[2][2];
    eps[3] = 2.0 * e[0][1]; eps[4] = 2.0 * e[1][2]; eps[5] = 2.0 * e[0][2];
  }
}

/* Hooke matrix of Section 5.1 with lambda, mu replaced by their integrals */
static void hooke(int d, double lam, double mu, double C[6][6]) {
  int ns = (d == 2) ? 3 : 6;
  for (int i = 0; i < ns; ++i)
    for (int j = 0; j < ns; ++j) C[i][j] = 0.0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) C[i][j] = lam + ((i == j) ? 2.0 * mu : 0.0);
  for (int i = d; i < ns; ++i) C[i][i] = mu;
}

/*
 * Local matrix of one element, column-wise: E[j*nl + i], nl = m (d+1), local
 * index i = a m + l for vertex a, component l. S receives the normwise scale of
 * every entry, used by the tests to normalise errors of cancelling sums: the
 * entry itself for (weighted) mass (|.| of each term), w |K| |grad lambda_a|
 * |grad lambda_b| for stiffness and (|lambda^| + 2 |mu^|) |grad lambda_a|
 * |grad lambda_b| for elasticity (lambda^, mu^ the integrals of the Lame fields).
 * cv1 / cv2 are the vertex values of the coefficient(s) (P1 interpolation; a
 * scalar or P0 coefficient is passed as d+1 equal values).
 */
int orc_element(int kind, int d, const double* X, const double* cv1, const double* cv2,
                double* E, double* S) {
  double det, vol, G[4 * 3];
  int rc = orc_simplex(d, X, &det, &vol, G);
  if (rc) return rc;
  int nv = d + 1;
  if (kind == ORC_MASS || kind == ORC_WMASS) {
    for (int b = 0; b < nv; ++b)
      for (int a = 0; a < nv; ++a) {
        double s = 0.0, sa = 0.0;
        int n[4];
        if (kind == ORC_MASS) {
          for (int i = 0; i < nv; ++i) n[i] = (i == a) + (i == b);
          s = orc_magic(d, n, vol);
          sa = s;
        } else {
          for (int g = 0; g < nv; ++g) {
            for (int i = 0; i < nv; ++i) n[i] = (i == a) + (i == b) + (i == g);
            double t = cv1[g] * orc_magic(d, n, vol);
            s += t;
            sa += fabs(t);
          }
        }
        E[b * nv + a] = s;
        S[b * nv + a] = sa;
      }
    return ORC_OK;
  }
  if (kind == ORC_STIFF) {
    double w = cv1 ? cv1[0] : 1.0;
    for (int b = 0; b < nv; ++b)
      for (int a = 0; a < nv; ++a) {
        double s = 0.0, na = 0.0, nb = 0.0;
        for (int i = 0; i < d; ++i) {
          s += G[b * d + i] * G[a * d + i];
          na += G[a * d + i] * G[a * d + i];
          nb += G[b * d + i] * G[b * d + i];
        }
        E[b * nv + a] = w * vol * s;
        S[b * nv + a] = fabs(w) * vol * sqrt(na * nb);
      }
    return ORC_OK;
  }
  if (kind == ORC_ELAS) {
    int m = d, nl = m * nv, ns = (d == 2) ? 3 : 6;
    double lam = p1_integral(d, cv1, vol), mu = p1_integral(d, cv2, vol);
    double C[6][6], ga_norm[4];
    hooke(d, lam, mu, C);
    for (int a = 0; a < nv; ++a) {
      double t = 0.0;
      for (int i = 0; i < d; ++i) t += G[a * d + i] * G[a * d + i];
      ga_norm[a] = sqrt(t);
    }
    for (int b = 0; b < nv; ++b)
      for (int n = 0; n < m; ++n) {
        double eb[6];
        strain_vector(d, &G[b * d], n, eb);
        int j = b * m + n;
        for (int a = 0; a < nv; ++a)
          for (int l = 0; l < m; ++l) {
            double ea[6];
            strain_vector(d, &G[a * d], l, ea);
            int i = a * m + l;
            double s = 0.0;
            for (int r = 0; r < ns; ++r)
              for (int c = 0; c < ns; ++c) s += eb[r] * C[r][c] * ea[c];
            E[j * nl + i] = s;
            S[j * nl + i] = (fabs(lam) + 2.0 * fabs(mu)) * ga_norm[a] * ga_norm[b];
          }
      }
    return ORC_OK;
  }
  return ORC_ERR_ARG;
}

/* vertex values of a coefficient on element k */
static void coef_values(int kind, const double* c, int d, int64_t nme, const int32_t* me, int64_t k,
                        double* out) {
  for (int a = 0; a <= d; ++a) {
    switch (kind) {
      case ORC_COEF_NONE: out[a] = 1.0; break;
      case ORC_COEF_SCALAR: out[a] = c[0]; break;
      case ORC_COEF_P0: out[a] = c[k]; break;
      default: out[a] = c[me[(int64_t)a * nme + k]]; break;
    }
  }
}

typedef struct {
  int64_t row, col, k;
  int32_t slot;
  double v, s;
} triplet;

static int cmp_triplet(const void* pa, const void* pb) {
  const triplet* a = (const triplet*)pa;
  const triplet* b = (const triplet*)pb;
  if (a->row != b->row) return a->row < b->row ? -1 : 1;
  if (a->col != b->col) return a->col < b->col ? -1 : 1;
  if (a->k != b->k) return a->k < b->k ? -1 : 1;
  if (a->slot != b->slot) return a->slot < b->slot ? -1 : 1;
  return 0;
}

/* Sort the triplets by (row, column, element, slot) and sum equal (row, column)
 * into a CSR matrix of order n (the `sparse` constructor of Section 3). Beside each
 * sum: the sum of the contributions' condition scales (scale) and the sum of their
 * absolute values (abssum), the scale of a cancelling sum's rounding error. */
static int triplets_to_csr(triplet* t, int64_t nt, int64_t n, int64_t** row_ptr, int32_t** col_idx,
                           double** val, double** scale, double** abssum, int64_t* nnz_out) {
  if (sort_records(t, nt, sizeof(triplet), cmp_triplet)) return ORC_ERR_NOMEM;
  int64_t nnz = 0;
  for (int64_t i = 0; i < nt; ++i)
    if (i == 0 || t[i].row != t[i - 1].row || t[i].col != t[i - 1].col) ++nnz;
  *row_ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  *col_idx = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
  *val = (double*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
  *scale = (double*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
  *abssum = (double*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
  if (!*row_ptr || !*col_idx || !*val || !*scale || !*abssum) return ORC_ERR_NOMEM;
  int64_t j = -1;
  for (int64_t i = 0; i < nt; ++i) {
    if (i == 0 || t[i].row != t[i - 1].row || t[i].col != t[i - 1].col) {
      ++j;
      (*col_idx)[j] = (int32_t)t[i].col;
      (*val)[j] = 0.0;
      (*scale)[j] = 0.0;
      (*abssum)[j] = 0.0;
      (*row_ptr)[t[i].row + 1] += 1;
    }
    (*val)[j] += t[i].v;
    (*scale)[j] += t[i].s;
    (*abssum)[j] += fabs(t[i].v);
  }
  for (int64_t r = 0; r < n; ++r) (*row_ptr)[r + 1] += (*row_ptr)[r];
  *nnz_out = nnz;
  return ORC_OK;
}

/*
 * Full assembly (Algorithm 2 followed by `sparse`). q is d x nq (q[c*nq + v]),
 * me is (d+1) x nme (me[a*nme + k]). The result is a CSR matrix of order
 * n = m nq with sorted column indices, returned in malloc'ed arrays that the
 * caller frees with orc_free. scale receives, per entry, the sum over its
 * contributions of their condition scale (see orc_element), abssum the sum of
 * their absolute values. On error *bad_id is
 * the offending element (or vertex index for ORC_ERR_INDEX).
 */
int orc_assemble(int kind, int d, int64_t nq, int64_t nme, const double* q, const int32_t* me,
                 int c1_kind, const double* c1, int c2_kind, const double* c2,
                 int64_t* n_out, int64_t* nnz_out, int64_t** row_ptr, int32_t** col_idx,
                 double** val, double** scale, double** abssum, int64_t* bad_id) {
  *bad_id = -1;
  if (d < 1 || d > 3 || nq < 0 || nme < 0) return ORC_ERR_ARG;
  int m = (kind == ORC_ELAS) ? d : 1;
  int nv = d + 1, nl = m * nv, ns = nl * nl;
  int64_t n = (int64_t)m * nq;
  int64_t nt = nme * ns;
  triplet* t = (triplet*)malloc((size_t)(nt > 0 ? nt : 1) * sizeof(triplet));
  if (!t) return ORC_ERR_NOMEM;
  int rc = ORC_OK;
  /* elements are independent; an error reports the smallest failing element */
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int64_t k = 0; k < nme; ++k) {
    double X[12], cv1[4], cv2[4], E[144], S[144];
    int erc = ORC_OK;
    for (int a = 0; a < nv && !erc; ++a) {
      int32_t v = me[(int64_t)a * nme + k];
      if (v < 0 || v >= nq) erc = ORC_ERR_INDEX;
      else
        for (int c = 0; c < d; ++c) X[a * d + c] = q[(int64_t)c * nq + v];
    }
    if (!erc) {
      coef_values(c1_kind, c1, d, nme, me, k, cv1);
      coef_values(c2_kind, c2, d, nme, me, k, cv2);
      erc = orc_element(kind, d, X, cv1, cv2, E, S);
    }
    if (erc) {
#pragma omp critical
      if (*bad_id < 0 || k < *bad_id) { *bad_id = k; rc = erc; }
      continue;
    }
    for (int j = 0; j < nl; ++j)
      for (int i = 0; i < nl; ++i) {
        triplet* p = &t[k * ns + j * nl + i];
        int a = i / m, l = i % m, b = j / m, c = j % m;
        p->row = (int64_t)m * me[(int64_t)a * nme + k] + l;
        p->col = (int64_t)m * me[(int64_t)b * nme + k] + c;
        p->k = k;
        p->slot = j * nl + i;
        p->v = E[j * nl + i];
        p->s = S[j * nl + i];
      }
  }
  if (rc) { free(t); return rc; }
  rc = triplets_to_csr(t, nt, n, row_ptr, col_idx, val, scale, abssum, nnz_out);
  free(t);
  if (rc) return rc;
  *n_out = n;
  return ORC_OK;
}

void orc_free(void* p) { free(p); }

typedef struct {
  uint64_t key;  /* row * n + column */
  int64_t slot;  /* k * ns + local slot (column-wise local order) */
} slot_key;

static int cmp_slot_key(const void* pa, const void* pb) {
  const slot_key* a = (const slot_key*)pa;
  const slot_key* b = (const slot_key*)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return a->slot < b->slot ? -1 : (a->slot > b->slot ? 1 : 0);
}

/*
 * The slot map of the `sparse` step for a fixed pattern: the element slots (k, local
 * slot), numbered k ns + slot with ns = (m (d+1))^2 in the column-wise local order of
 * orc_assemble, sorted by (row, column, element, slot) as orc_assemble sorts its
 * triplets. nnz_ptr[j] .. nnz_ptr[j+1] are the slots of the j-th nonzero (CSR order), in
 * the order their contributions are summed; nnz2slot lists them. malloc'ed arrays; the
 * caller frees them with orc_free.
 */
int orc_slot_map(int d, int m, int64_t nq, int64_t nme, const int32_t* me, int64_t* nnz_out,
                 int64_t** nnz_ptr, int64_t** nnz2slot, int64_t* bad_id) {
  *bad_id = -1;
  if (d < 1 || d > 3 || m < 1 || nq < 0 || nme < 0) return ORC_ERR_ARG;
  const int nv = d + 1, nl = m * nv, ns = nl * nl;
  const int64_t n = (int64_t)m * nq, nt = nme * ns;
  slot_key* t = (slot_key*)malloc((size_t)(nt > 0 ? nt : 1) * sizeof(slot_key));
  if (!t) return ORC_ERR_NOMEM;
  for (int64_t k = 0; k < nme; ++k)
    for (int j = 0; j < nl; ++j)
      for (int i = 0; i < nl; ++i) {
        const int32_t va = me[(int64_t)(i / m) * nme + k], vb = me[(int64_t)(j / m) * nme + k];
        if (va < 0 || va >= nq || vb < 0 || vb >= nq) { *bad_id = k; free(t); return ORC_ERR_INDEX; }
        const int64_t row = (int64_t)m * va + i % m, col = (int64_t)m * vb + j % m;
        t[k * ns + j * nl + i].key = (uint64_t)row * (uint64_t)n + (uint64_t)col;
        t[k * ns + j * nl + i].slot = k * ns + j * nl + i;
      }
  if (sort_records(t, nt, sizeof(slot_key), cmp_slot_key)) { free(t); return ORC_ERR_NOMEM; }
  int64_t nnz = 0;
  for (int64_t i = 0; i < nt; ++i)
    if (i == 0 || t[i].key != t[i - 1].key) ++nnz;
  *nnz_ptr = (int64_t*)malloc((size_t)(nnz + 1) * sizeof(int64_t));
  *nnz2slot = (int64_t*)malloc((size_t)(nt > 0 ? nt : 1) * sizeof(int64_t));
  if (!*nnz_ptr || !*nnz2slot) { free(t); return ORC_ERR_NOMEM; }
  int64_t j = 0;
  for (int64_t i = 0; i < nt; ++i) {
    if (i == 0 || t[i].key != t[i - 1].key) (*nnz_ptr)[j++] = i;
    (*nnz2slot)[i] = t[i].slot;
  }
  (*nnz_ptr)[nnz] = nt;
  free(t);
  *nnz_out = nnz;
  return ORC_OK;
}

/*
 * Fixed-pattern reassembly: every element's local matrix (orc_element, into an
 * element-major array of nme ns values), then each nonzero's sum over its slots in the
 * order of the slot map (orc_slot_map), into val (nnz doubles). The sums run in the order
 * of orc_assemble's, so the values equal its values bit for bit, whatever the thread count.
 * On error *bad_id is the smallest failing element.
 */
int orc_reassemble(int kind, int d, int64_t nq, int64_t nme, const double* q, const int32_t* me,
                   int c1_kind, const double* c1, int c2_kind, const double* c2, int64_t nnz,
                   const int64_t* nnz_ptr, const int64_t* nnz2slot, double* val, int64_t* bad_id) {
  *bad_id = -1;
  if (d < 1 || d > 3 || nq < 0 || nme < 0) return ORC_ERR_ARG;
  const int m = (kind == ORC_ELAS) ? d : 1;
  const int nv = d + 1, nl = m * nv, ns = nl * nl;
  double* kg = (double*)malloc((size_t)(nme * ns > 0 ? nme * ns : 1) * sizeof(double));
  if (!kg) return ORC_ERR_NOMEM;
  int rc = ORC_OK;
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int64_t k = 0; k < nme; ++k) {
    double X[12], cv1[4], cv2[4], S[144];
    int erc = ORC_OK;
    for (int a = 0; a < nv && !erc; ++a) {
      const int32_t v = me[(int64_t)a * nme + k];
      if (v < 0 || v >= nq) erc = ORC_ERR_INDEX;
      else
        for (int c = 0; c < d; ++c) X[a * d + c] = q[(int64_t)c * nq + v];
    }
    if (!erc) {
      coef_values(c1_kind, c1, d, nme, me, k, cv1);
      coef_values(c2_kind, c2, d, nme, me, k, cv2);
      erc = orc_element(kind, d, X, cv1, cv2, kg + k * ns, S);
    }
    if (erc) {
#pragma omp critical
      if (*bad_id < 0 || k < *bad_id) { *bad_id = k; rc = erc; }
    }
  }
  if (rc) { free(kg); return rc; }
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int64_t j = 0; j < nnz; ++j) {
    double s = 0.0;
    for (int64_t i = nnz_ptr[j]; i < nnz_ptr[j + 1]; ++i) s += kg[nnz2slot[i]];
    val[j] = s;
  }
  free(kg);
  return ORC_OK;
}

static int cmp_u64(const void* pa, const void* pb) {
  const uint64_t a = *(const uint64_t*)pa, b = *(const uint64_t*)pb;
  return a < b ? -1 : (a > b ? 1 : 0);
}

/*
 * Nonzero pattern alone of the matrix that orc_assemble builds (the `sparse`
 * constructor of Section 3 keeps one entry per distinct (row, column) of the
 * triplets): every element contributes the (d+1)^2 vertex pairs (me(a,k), me(b,k));
 * they are sorted as keys row * nq + column and repeated keys dropped. With m dofs
 * per vertex (m > 1, vector problems of Section 5, dof = m vertex + component) each
 * vertex pair (v, w) stands for the m x m block of entries (m v + l, m w + n).
 * Returns malloc'ed CSR arrays (order m nq, sorted columns) the caller frees with
 * orc_free; *bad_id is the offending element when an index is out of range.
 */
int orc_pattern(int d, int m, int64_t nq, int64_t nme, const int32_t* me, int64_t* nnz_out,
                int64_t** row_ptr, int32_t** col_idx, int64_t* bad_id) {
  *bad_id = -1;
  if (d < 1 || d > 3 || m < 1 || nq < 0 || nme < 0) return ORC_ERR_ARG;
  const int nv = d + 1;
  const int64_t nk = nme * nv * nv;
  uint64_t* key = (uint64_t*)malloc((size_t)(nk > 0 ? nk : 1) * sizeof(uint64_t));
  if (!key) return ORC_ERR_NOMEM;
  for (int64_t k = 0; k < nme; ++k)
    for (int b = 0; b < nv; ++b)
      for (int a = 0; a < nv; ++a) {
        const int32_t r = me[(int64_t)a * nme + k], c = me[(int64_t)b * nme + k];
        if (r < 0 || r >= nq || c < 0 || c >= nq) {
          *bad_id = k;
          free(key);
          return ORC_ERR_INDEX;
        }
        key[(k * nv + b) * nv + a] = (uint64_t)r * (uint64_t)nq + (uint64_t)c;
      }
  qsort(key, (size_t)nk, sizeof(uint64_t), cmp_u64);
  int64_t nu = 0;
  for (int64_t i = 0; i < nk; ++i)
    if (i == 0 || key[i] != key[i - 1]) key[nu++] = key[i];
  /* scalar pattern as CSR: rows are vertices */
  int64_t* vptr = (int64_t*)calloc((size_t)nq + 1, sizeof(int64_t));
  if (!vptr) { free(key); return ORC_ERR_NOMEM; }
  for (int64_t i = 0; i < nu; ++i) vptr[key[i] / (uint64_t)nq + 1] += 1;
  for (int64_t v = 0; v < nq; ++v) vptr[v + 1] += vptr[v];
  const int64_t n = (int64_t)m * nq, nnz = nu * m * m;
  *row_ptr = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
  *col_idx = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
  if (!*row_ptr || !*col_idx) { free(key); free(vptr); return ORC_ERR_NOMEM; }
  int64_t j = 0;
  (*row_ptr)[0] = 0;
  for (int64_t v = 0; v < nq; ++v)
    for (int l = 0; l < m; ++l) {
      for (int64_t i = vptr[v]; i < vptr[v + 1]; ++i) {
        const int64_t w = (int64_t)(key[i] % (uint64_t)nq);
        for (int c = 0; c < m; ++c) (*col_idx)[j++] = (int32_t)(m * w + c);
      }
      (*row_ptr)[m * v + l + 1] = j;
    }
  free(key);
  free(vptr);
  *nnz_out = nnz;
  return ORC_OK;
}

/*
 * General second-order operator of Eq. EDP, -div(A grad u) + div(b u) + c . grad u + a0 u,
 * in weak form (the divergence terms integrated by parts, boundary terms left out):
 *   a(u, v) = int (A grad u) . grad v - int u b . grad v + int (c . grad u) v + int a0 u v.
 * The matrix entry of row i, column j is a(phi_j, phi_i), so the local entry (a, b)
 * (test vertex a, trial vertex b) is
 *   int (A g_b) . g_a - int lambda_b (b . g_a) + int lambda_a (c . g_b) + int a0 lambda_a lambda_b.
 * Each coefficient is written on K as sum_c f(c) lambda_c: f(c) its value at local vertex
 * c (P1, interpolated) or the element's value for every c (scalar, P0; then sum_c lambda_c = 1
 * gives back the constant), and every integral of a product of barycentric coordinates is
 * taken by the magic formula (Eq. MagicFormula).
 * coef holds records of nc = d*d + 2d + 1 values A (row-major), b, c, a0: one record
 * (ORC_COEF_SCALAR: coef[j]), one per element (ORC_COEF_P0: coef[k * nc + j]) or one per
 * vertex (ORC_COEF_P1: coef[v * nc + j]).
 * The condition scale of an entry is the same sum with every term replaced by its absolute
 * bound: |A(c)|_F |g_a| |g_b|, |b(c)| |g_a|, |c(c)| |g_b|, |a0(c)| under the same integrals.
 */
int orc_assemble_general(int d, int64_t nq, int64_t nme, const double* q, const int32_t* me,
                         int coef_kind, const double* coef, int64_t* n_out, int64_t* nnz_out,
                         int64_t** row_ptr, int32_t** col_idx, double** val, double** scale, double** abssum,
                         int64_t* bad_id) {
  *bad_id = -1;
  if (d < 2 || d > 3) return ORC_ERR_ARG;
  if (coef_kind != ORC_COEF_SCALAR && coef_kind != ORC_COEF_P0 && coef_kind != ORC_COEF_P1)
    return ORC_ERR_ARG;
  const int nv = d + 1, ns = nv * nv, nc = d * d + 2 * d + 1;
  triplet* t = (triplet*)malloc((size_t)(nme * ns > 0 ? nme * ns : 1) * sizeof(triplet));
  if (!t) return ORC_ERR_NOMEM;
  double X[12], G[12], det, vol, cf[4][16];
  int rc = ORC_OK;
  for (int64_t k = 0; k < nme && rc == ORC_OK; ++k) {
    int32_t vid[4];
    for (int a = 0; a < nv; ++a) {
      const int32_t v = me[(int64_t)a * nme + k];
      if (v < 0 || v >= nq) { *bad_id = k; rc = ORC_ERR_INDEX; break; }
      vid[a] = v;
      for (int c = 0; c < d; ++c) X[a * d + c] = q[(int64_t)c * nq + v];
    }
    if (rc) break;
    rc = orc_simplex(d, X, &det, &vol, G);
    if (rc) { *bad_id = k; break; }
    /* cf[c][j]: coefficient j at local vertex c */
    for (int c = 0; c < nv; ++c)
      for (int j = 0; j < nc; ++j)
        cf[c][j] = coef_kind == ORC_COEF_SCALAR ? coef[j]
                 : coef_kind == ORC_COEF_P0     ? coef[k * nc + j]
                                                : coef[(int64_t)vid[c] * nc + j];
    double gn[4];
    for (int a = 0; a < nv; ++a) {
      double s = 0.0;
      for (int i = 0; i < d; ++i) s += G[a * d + i] * G[a * d + i];
      gn[a] = sqrt(s);
    }
    for (int b = 0; b < nv; ++b)
      for (int a = 0; a < nv; ++a) {
        double v = 0.0, sc = 0.0;
        for (int c = 0; c < nv; ++c) {
          const double* A = cf[c];
          const double* bv = cf[c] + d * d;
          const double* cv = cf[c] + d * d + d;
          const double a0 = cf[c][d * d + 2 * d];
          int n[4];
          for (int i = 0; i < nv; ++i) n[i] = (i == c);
          const double i_c = orc_magic(d, n, vol);                 /* int lambda_c */
          n[b] += 1;
          const double i_cb = orc_magic(d, n, vol);                /* int lambda_c lambda_b */
          n[a] += 1;
          const double i_cab = orc_magic(d, n, vol);               /* int lambda_c lambda_a lambda_b */
          for (int i = 0; i < nv; ++i) n[i] = (i == c) + (i == a);
          const double i_ca = orc_magic(d, n, vol);                /* int lambda_c lambda_a */
          double diff = 0.0, bga = 0.0, cgb = 0.0, an = 0.0, bn = 0.0, cn = 0.0;
          for (int i = 0; i < d; ++i) {
            double Agb = 0.0;
            for (int j = 0; j < d; ++j) {
              Agb += A[i * d + j] * G[b * d + j];
              an += A[i * d + j] * A[i * d + j];
            }
            diff += G[a * d + i] * Agb;
            bga += bv[i] * G[a * d + i];
            cgb += cv[i] * G[b * d + i];
            bn += bv[i] * bv[i];
            cn += cv[i] * cv[i];
          }
          v += i_c * diff - i_cb * bga + i_ca * cgb + i_cab * a0;
          sc += i_c * sqrt(an) * gn[a] * gn[b] + i_cb * sqrt(bn) * gn[a] + i_ca * sqrt(cn) * gn[b] +
                i_cab * fabs(a0);
        }
        triplet* p = &t[k * ns + b * nv + a];
        p->row = vid[a];
        p->col = vid[b];
        p->k = k;
        p->slot = b * nv + a;
        p->v = v;
        p->s = sc;
      }
  }
  if (rc) { free(t); return rc; }
  rc = triplets_to_csr(t, nme * ns, nq, row_ptr, col_idx, val, scale, abssum, nnz_out);
  free(t);
  *n_out = nq;
  return rc;
}

/*
 * P_k mass (App. D, Eq. MatElemMassPk and Algorithm 15): every element contributes
 * |K| * tab[b * ndfe + a] to entry (me(a), me(b)), where tab = (integral of
 * phi_alpha phi_beta) / |K| is the same for every element. |K| comes from the element's
 * first d + 1 nodes, its vertices. The caller supplies tab (computed exactly from the
 * basis functions of Eq. Pk:functions and the magic formula) and the node order it
 * belongs to. The condition scale of an entry is the sum of |K| |tab|.
 */
int orc_assemble_table(int d, int64_t nq, int64_t nme, int ndfe, const double* q, const int32_t* me,
                       const double* tab, int64_t* n_out, int64_t* nnz_out, int64_t** row_ptr,
                       int32_t** col_idx, double** val, double** scale, double** abssum, int64_t* bad_id) {
  *bad_id = -1;
  if (d < 2 || d > 3 || ndfe < d + 1) return ORC_ERR_ARG;
  const int64_t ns = (int64_t)ndfe * ndfe;
  triplet* t = (triplet*)malloc((size_t)(nme * ns > 0 ? nme * ns : 1) * sizeof(triplet));
  if (!t) return ORC_ERR_NOMEM;
  double X[12], G[12], det, vol;
  int rc = ORC_OK;
  for (int64_t k = 0; k < nme && rc == ORC_OK; ++k) {
    for (int a = 0; a < ndfe; ++a) {
      const int32_t v = me[(int64_t)a * nme + k];
      if (v < 0 || v >= nq) { *bad_id = k; rc = ORC_ERR_INDEX; break; }
      if (a <= d)
        for (int c = 0; c < d; ++c) X[a * d + c] = q[(int64_t)c * nq + v];
    }
    if (rc) break;
    rc = orc_simplex(d, X, &det, &vol, G);
    if (rc) { *bad_id = k; break; }
    for (int b = 0; b < ndfe; ++b)
      for (int a = 0; a < ndfe; ++a) {
        triplet* p = &t[k * ns + (int64_t)b * ndfe + a];
        p->row = me[(int64_t)a * nme + k];
        p->col = me[(int64_t)b * nme + k];
        p->k = k;
        p->slot = b * ndfe + a;
        p->v = vol * tab[(int64_t)b * ndfe + a];
        p->s = fabs(p->v);
      }
  }
  if (rc) { free(t); return rc; }
  rc = triplets_to_csr(t, nme * ns, nq, row_ptr, col_idx, val, scale, abssum, nnz_out);
  free(t);
  *n_out = nq;
  return rc;
}

/*
 * Measure of a (d-1)-simplex in d-space with vertices X (d vertices x d coordinates):
 * sqrt(det(B^T B)) / (d-1)!, B the d x (d-1) matrix of edge vectors q^i - q^0 (the
 * Gram determinant; for a segment its length, for a triangle half the parallelogram).
 */
int orc_facet(int d, const double* X, double* meas) {
  const int k = d - 1;
  if (k < 1 || k > 2) return ORC_ERR_ARG;
  double B[3][2], M[2][2];
  for (int c = 0; c < d; ++c)
    for (int i = 0; i < k; ++i) B[c][i] = X[(i + 1) * d + c] - X[c];
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int c = 0; c < d; ++c) s += B[c][i] * B[c][j];
      M[i][j] = s;
    }
  const double g = (k == 1) ? M[0][0] : M[0][0] * M[1][1] - M[0][1] * M[1][0];
  *meas = sqrt(g) / factorial(k);
  if (!(*meas > 0.0) || !isfinite(*meas)) return ORC_ERR_DEGENERATE;
  return ORC_OK;
}

/*
 * Boundary mass / weighted mass: facets (d rows, 0-based) of dimension k = d - 1;
 * local entries int_K w phi_b phi_a by the magic formula with k in place of d and w
 * P1-interpolated (COEF_P1) or per facet (COEF_P0); kind ORC_MASS or ORC_WMASS.
 */
int orc_assemble_boundary(int kind, int d, int64_t nq, int64_t nf, const double* q, const int32_t* fa,
                          int c1_kind, const double* c1, int64_t* n_out, int64_t* nnz_out,
                          int64_t** row_ptr, int32_t** col_idx, double** val, double** scale, double** abssum,
                          int64_t* bad_id) {
  *bad_id = -1;
  if (d < 2 || d > 3 || (kind != ORC_MASS && kind != ORC_WMASS)) return ORC_ERR_ARG;
  const int k = d - 1, nv = d, ns = nv * nv;
  triplet* t = (triplet*)malloc((size_t)(nf * ns > 0 ? nf * ns : 1) * sizeof(triplet));
  if (!t) return ORC_ERR_NOMEM;
  double X[9], w[3];
  int rc = ORC_OK;
  for (int64_t f = 0; f < nf && rc == ORC_OK; ++f) {
    for (int a = 0; a < nv; ++a) {
      const int32_t v = fa[(int64_t)a * nf + f];
      if (v < 0 || v >= nq) { *bad_id = f; rc = ORC_ERR_INDEX; break; }
      for (int c = 0; c < d; ++c) X[a * d + c] = q[(int64_t)c * nq + v];
      w[a] = (kind == ORC_MASS || c1_kind == ORC_COEF_NONE) ? 1.0
             : (c1_kind == ORC_COEF_SCALAR) ? c1[0]
             : (c1_kind == ORC_COEF_P0) ? c1[f] : c1[v];
    }
    if (rc) break;
    double meas;
    rc = orc_facet(d, X, &meas);
    if (rc) { *bad_id = f; break; }
    for (int b = 0; b < nv; ++b)
      for (int a = 0; a < nv; ++a) {
        double s = 0.0, sa = 0.0;
        int n[4];
        for (int g = 0; g < nv; ++g) {
          for (int i = 0; i < nv; ++i) n[i] = (i == a) + (i == b) + (i == g);
          const double tg = w[g] * orc_magic(k, n, meas);  /* int w_g lambda_g lambda_a lambda_b */
          s += tg;
          sa += fabs(tg);
        }
        triplet* p = &t[f * ns + b * nv + a];
        p->row = fa[(int64_t)a * nf + f];
        p->col = fa[(int64_t)b * nf + f];
        p->k = f;
        p->slot = b * nv + a;
        p->v = s;
        p->s = sa;
      }
  }
  if (rc) { free(t); return rc; }
  rc = triplets_to_csr(t, nf * ns, nq, row_ptr, col_idx, val, scale, abssum, nnz_out);
  free(t);
  *n_out = nq;
  return rc;
}

/*
 * Loss L = u^T K(w) v for the stiffness matrix with per-element coefficient w
 * (NULL: w = 1), and its gradients. Per element, with ubar = sum_a u_a grad
 * lambda_a and vbar likewise, the element part is L_e = w_e |K| ubar . vbar, so
 *   dL/dw_e = |K| ubar . vbar,
 *   dL/dq^c = sum over elements containing vertex c of
 *             w_e |K| [ (ubar . vbar) g_c - ubar (g_c . vbar) - vbar (g_c . ubar) ],
 * where g_c is the gradient of the barycentric coordinate of that vertex. The
 * last formula is the derivative of |det B| / d! and of B^{-T} with respect to
 * the columns of B = [q^1 - q^0, ...] (App. C.1); the paper itself has no
 * derivatives. dLdq is d x nq like q and is accumulated in element order.
 */
int orc_stiff_loss(int d, int64_t nq, int64_t nme, const double* q, const int32_t* me,
                   const double* w, const double* u, const double* v, double* L, double* dLdw,
                   double* dLdq, int64_t* bad_id) {
  *bad_id = -1;
  int nv = d + 1;
  double X[12], G[12], det, vol;
  double total = 0.0;
  if (dLdq) memset(dLdq, 0, sizeof(double) * (size_t)(d * nq));
  for (int64_t k = 0; k < nme; ++k) {
    int32_t vid[4];
    for (int a = 0; a < nv; ++a) {
      vid[a] = me[(int64_t)a * nme + k];
      if (vid[a] < 0 || vid[a] >= nq) { *bad_id = k; return ORC_ERR_INDEX; }
      for (int c = 0; c < d; ++c) X[a * d + c] = q[(int64_t)c * nq + vid[a]];
    }
    int rc = orc_simplex(d, X, &det, &vol, G);
    if (rc) { *bad_id = k; return rc; }
    double ub[3] = {0, 0, 0}, vb[3] = {0, 0, 0};
    for (int a = 0; a < nv; ++a)
      for (int i = 0; i < d; ++i) {
        ub[i] += u[vid[a]] * G[a * d + i];
        vb[i] += v[vid[a]] * G[a * d + i];
      }
    double uv = 0.0;
    for (int i = 0; i < d; ++i) uv += ub[i] * vb[i];
    double we = w ? w[k] : 1.0;
    total += we * vol * uv;
    if (dLdw) dLdw[k] = vol * uv;
    if (dLdq) {
      for (int c = 0; c < nv; ++c) {
        const double* g = &G[c * d];
        double gu = 0.0, gv = 0.0;
        for (int i = 0; i < d; ++i) { gu += g[i] * ub[i]; gv += g[i] * vb[i]; }
        for (int i = 0; i < d; ++i)
          dLdq[(int64_t)i * nq + vid[c]] += we * vol * (uv * g[i] - ub[i] * gv - vb[i] * gu);
      }
    }
  }
  *L = total;
  return ORC_OK;
}
