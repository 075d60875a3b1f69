/*
 * fe.h -- C ABI of the GB300 P1 finite element assembly library (libfe_gb300.so).
 *
 * The library computes the P1 Lagrange finite element matrices of a simplicial
 * mesh (Cuvelier, Japhet, Scarella, "An efficient way to assemble finite element
 * matrices in vector languages"): mass, weighted mass, stiffness and linear
 * elasticity, the general second-order operator of Eq. EDP, boundary (facet) mass
 * and P_k mass (App. D), and assembles them into CSR form with duplicate
 * contributions summed, which is the `sparse(Ig, Jg, Kg, m, n)` constructor of
 * Section 3; also the gradients of L = u^T S(w) v (and general vector-Jacobian
 * products) of the stiffness matrix. Values come in three precision forms (FE_F64,
 * FE_F32 and FE_F64X, defined below).
 *
 * Conventions shared by every call
 *   - Mesh (Section 2, Table 1): q is d x nq (coordinate c of vertex v at
 *     q[c*nq + v], FP64), me is (d+1) x nme (vertex of local corner a of element k
 *     at me[a*nme + k], int32, 0-BASED; the paper's arrays are 1-based).
 *   - Vector problems use the alternate numbering of Section 5:
 *     dof = m * vertex + component (0-based).
 *   - Every pointer argument is a DEVICE pointer unless stated otherwise. The
 *     caller owns q, me, coefficients and output arrays; the library owns the
 *     arrays of a pattern handle until fe_pattern_destroy.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls are stream-ordered and asynchronous except where stated.
 *   - Every call returns an fe status code. Argument errors are detected on the
 *     host before any launch. Data errors found by a kernel (a vertex index out
 *     of range, a degenerate element) are recorded in the handle's device status
 *     word; read it with fe_status(), which synchronises the stream.
 *   - Results are bit-identical from run to run for the deterministic
 *     reassembly strategies (FE_REASM_CHUNKED, FE_REASM_GATHER).
 */
#ifndef FE_GB300_H
#define FE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes */
#define FE_OK 0
#define FE_ERR_ARG 1        /* invalid argument (host-side check) */
#define FE_ERR_INDEX 2      /* me holds a vertex index outside [0, nq) */
#define FE_ERR_DEGENERATE 3 /* an element has det B = 0 or a non-finite det B */
#define FE_ERR_OVERFLOW 4   /* a size does not fit the library's 32-bit indices */
#define FE_ERR_CUDA 5       /* a CUDA runtime call failed */
#define FE_ERR_TIMEOUT 6    /* a bounded device-side wait for a chunk's plan record
                               gave up; that chunk's values are missing, and the
                               block that gave up may have left its record copy in
                               flight into shared memory (it waits once more, also
                               bounded): treat every value of that launch and of any
                               launch overlapping it as undefined */
#define FE_ERR_NOMEM 7      /* device allocation failed */
#define FE_ERR_SCRATCH_LIMIT 8 /* the mesh needs more scratch than fe_assemble_stiff_noalloc has */
#define FE_ERR_BOUNDS 9     /* bounds-checked builds only (FE_CHECKED): an index fell outside its
                               buffer; the access was skipped, *id is the element chunk */

/* ---- precision forms of the element and value kernels */
#define FE_F64 0 /* FP64 arithmetic, FP64 values */
#define FE_F32 1 /* FP32 values; det B and |K| from FP64-accurate coordinates
                    differences in double-float arithmetic; compensated sums */
#define FE_F64X 2 /* every operator (mass, weighted mass, stiffness with its backward
                    and VJP, elasticity, general operator; volume, facet and P_k
                    patterns), chunked strategy only: FP64 values of FP64-class accuracy
                    computed in double-float (pairs of floats, about 48 bits) on the
                    FP32 pipe; native FP64 only for coordinates relative to a vertex of
                    each element chunk and for converting sums to double. Coefficients
                    are double, as for FE_F64. Other operators and patterns: FE_ERR_ARG. */

/* ---- coefficient kinds (coefficient arrays use the precision of the form:
 *      double for FE_F64, float for FE_F32) */
#define FE_COEF_NONE 0        /* identically 1; pointer ignored */
#define FE_COEF_SCALAR 1      /* one value, device pointer to it */
#define FE_COEF_P0 2          /* one value per element, input element order */
#define FE_COEF_P1 3          /* one value per vertex, P1-interpolated */
#define FE_COEF_P0_INTERNAL 4 /* one value per element, in the pattern's internal
                                 order (see fe_pattern_element_order) */

/* ---- reassembly strategies */
#define FE_REASM_CHUNKED 0 /* default: fused element + fixed-order on-chip sums over
                              element chunks, then a fixed-order sum of the chunk
                              partials of shared rows. Deterministic, no atomics. */
#define FE_REASM_GATHER 1  /* two passes: element values to scratch, then each
                              nonzero sums its slots in ascending slot order.
                              Deterministic, no atomics. */
#define FE_REASM_ATOMIC 2  /* fused element + atomicAdd scatter. NOT reproducible. */

/* ---- pattern flags */
#define FE_PATTERN_KEEP_ORDER 1 /* do not reorder elements internally (default:
                                   Morton order of element centroids) */
#define FE_PATTERN_ENTITY_ORDER 2 /* keep each chunk's distinct vertices and edges in
                                     nonzero order (default: by descending number of
                                     incidences, so that the threads of a warp sum
                                     lists of similar length; the nonzero order writes
                                     neighbouring values together). Values are the
                                     same bit for bit either way. */
#define FE_PATTERN_INTERLEAVED 4 /* interleaved chunk records (scalar volume patterns,
                                    m = 1): each element's values go straight to
                                    slots laid out so that the 32 threads of a warp
                                    sum 32 distinct vertices' or edges' lists from
                                    consecutive slots. Only the mass, weighted mass
                                    and stiffness calls (FE_F64, FE_F32) and the
                                    gather and atomic strategies accept such a
                                    pattern; the others return FE_ERR_ARG. Values are
                                    bit-identical to the plain layout's in FE_F32. */
/* elements per chunk of the chunked reassembly, 32..4096 (0: the default, 512 in
   3D and 1024 in 2D) */
#define FE_PATTERN_CHUNK(c) ((int32_t)(c) << 8)

typedef struct fe_mesh {
  int32_t d;          /* 2 or 3 */
  int64_t nq;         /* number of vertices */
  int64_t nme;        /* number of elements */
  const double* q;    /* device, d x nq, FP64 */
  const int32_t* me;  /* device, (d+1) x nme, 0-based */
} fe_mesh;

typedef struct fe_pattern_s* fe_pattern_h;

/*
 * fe_pattern -- build the sparsity pattern of the global matrix once per mesh
 * topology. Index part of `sparse` (Section 3): the (Ig, Jg) pairs of every
 * element slot (Algorithm 3: Ig(l,:) = me(a,:), Jg(l,:) = me(b,:); vector case
 * Algorithm 9: Ig = m me(a,:) + l, Jg = m me(b,:) + n, 0-based) are sorted by
 * a 64-bit key row * n + col with a device radix sort and run-length encoded.
 * The matrix has order n = m nq; every (row, col) pair shared by an element is
 * a structural nonzero, even when its value sums to zero. Column indices are
 * sorted within each row.
 *   m       dofs per vertex: 1 (mass, weighted mass, stiffness) or d (elasticity)
 *   flags   FE_PATTERN_* bits
 *   out     receives the handle. The pattern keeps a copy of me (internal order)
 *           and coordinates are passed again to every assembly call, so q may
 *           change between calls while me may not.
 * Synchronous: returns after the pattern is complete. Errors: FE_ERR_ARG,
 * FE_ERR_INDEX (me out of range), FE_ERR_OVERFLOW (more than 2^31-1 element
 * slots, nonzeros or rows), FE_ERR_NOMEM, FE_ERR_CUDA.
 */
int fe_pattern(const fe_mesh* mesh, int32_t m, int32_t flags, void* stream, fe_pattern_h* out);

/*
 * fe_batch_pattern -- one pattern for `count` meshes at once (host array of
 * descriptors, all of dimension d): the disjoint union of the meshes, with the
 * vertices of mesh b numbered after those of meshes 0..b-1 and its elements after
 * theirs. The global matrix is block diagonal and the CSR rows of mesh b form one
 * contiguous range (fe_batch_offsets), so every assembly call covers all meshes in
 * one launch. Coordinates for the assembly calls are the union array (d x total
 * vertices, SoA), which fe_batch_gather_q fills from the per-mesh arrays;
 * per-element coefficients are in the concatenated element order. Synchronous.
 */
int fe_batch_pattern(const fe_mesh* meshes, int32_t count, int32_t m, int32_t flags, void* stream,
                     fe_pattern_h* out);

/* Host arrays of count+1 offsets of a batch pattern: first vertex, first element and
 * first nonzero of each mesh (the last entry is the total). Any pointer may be NULL. */
int fe_batch_offsets(fe_pattern_h h, int64_t* vert_off, int64_t* elem_off, int64_t* nnz_off);

/* Number of meshes of a batch pattern (0 for a single-mesh pattern). */
int fe_batch_count(fe_pattern_h h, int32_t* count);

/* Copy the coordinates of the batch's meshes into the union array q_union
 * (d x total vertices), stream-ordered (one device copy per mesh and coordinate). */
int fe_batch_gather_q(fe_pattern_h h, const fe_mesh* meshes, double* q_union, void* stream);

/*
 * fe_boundary_pattern -- pattern of a mesh of boundary facets: (d-1)-simplices in
 * d-space (segments in 2D, triangles in 3D), for Neumann / Robin terms (Remark
 * after Algorithm 6: the weighted mass algorithm applies to n-simplices, n <= d).
 * facets->me has d rows (the facet's vertices, 0-based into q); q is d x nq.
 * Only fe_assemble_mass and fe_assemble_wmass accept such a pattern; the facet
 * measure is the Gram determinant sqrt(det(B^T B)) / (d-1)! with B the d x (d-1)
 * matrix of edge vectors. Other conventions as fe_pattern (m = 1).
 */
int fe_boundary_pattern(const fe_mesh* facets, int32_t flags, void* stream, fe_pattern_h* out);

/*
 * Vertex renumbering along a Morton curve (a caller-side utility: the library never
 * renumbers the matrix itself, which keeps the caller's vertex numbering).
 *
 * fe_morton_vertex_order -- order[i] = the vertex placed at position i: vertices sorted by
 * the Morton code of their coordinates (21 bits per axis over the bounding box, bits
 * interleaved x fastest), ties by vertex id. q: d x nq SoA, device; order: nq int32,
 * device. Synchronous (allocates and frees scratch).
 *
 * fe_apply_vertex_order -- the renumbered mesh: q_out[:, i] = q[:, order[i]] and
 * me_out = new ids of me (nv x nme, any number of rows, e.g. a P_k or a facet mesh).
 * All device pointers; q_out and me_out must not alias the inputs. FE_ERR_INDEX if
 * order has an entry outside [0, nq) or me one outside [0, nq) (those entries are left
 * unspecified). Synchronous.
 */
int fe_morton_vertex_order(int32_t d, int64_t nq, const double* q, int32_t* order, void* stream);
int fe_apply_vertex_order(int32_t d, int64_t nq, int64_t nme, int32_t nv, const double* q, const int32_t* me,
                          const int32_t* order, double* q_out, int32_t* me_out, void* stream);

/*
 * fe_pk_pattern -- pattern of a P_k mesh (App. D): q holds the coordinates of all
 * P_k nodes (d x nq) and mesh->me has ndfe = (d+k)!/(d! k!) rows, the nodes of each
 * element in the local order: the d+1 vertices (multi-indices k e_0, ..., k e_d)
 * first, then the other multi-indices alpha (|alpha| = k) in lexicographically
 * decreasing order. The element geometry comes from the first d+1 nodes. d = 2 or 3,
 * 1 <= k <= FE_PK_MAX; k = 1 is fe_pattern. Only fe_assemble_mass accepts a pattern
 * with k >= 2, which then assembles the P_k mass matrix of Eq. MatElemMassPk
 * (Algorithm 15): local entry |det B| C_{alpha,beta} = d! |K| C_{alpha,beta}, chunked
 * reassembly only. The element chunk is bounded by the plan's 16-bit incidence codes
 * (chunk * ndfe (ndfe - 1) / 2 < 32768), so high k uses small chunks. Other
 * conventions as fe_pattern (m = 1).
 */
#define FE_PK_MAX 6
int fe_pk_pattern(const fe_mesh* mesh, int32_t k, int32_t flags, void* stream, fe_pattern_h* out);

/*
 * fe_pk_mass_table -- the constants C_{alpha,beta} of Eq. MatElemMassPk for (d, k),
 * host only: C[a * ndfe + b] for local nodes a, b in the order of fe_pk_pattern.
 * Each is summed exactly in integer arithmetic from the basis functions of Eq.
 * Pk:functions and the magic formula, then rounded once (numerator and denominator
 * to double, then divided). C must hold ndfe * ndfe doubles.
 */
int fe_pk_mass_table(int32_t d, int32_t k, double* C);

/* Borrowed CSR arrays (int32, device): row_ptr[n+1], col_idx[nnz]. */
int fe_pattern_csr(fe_pattern_h h, int64_t* n, int64_t* nnz, const int32_t** row_ptr,
                   const int32_t** col_idx);

/*
 * Borrowed slot maps of the SCALAR pattern (device, int32). A slot is one entry
 * of one element matrix: slot id = e * (d+1)^2 + b (d+1) + a for element e in
 * the internal order and local entry (a, b) (column-wise, Section 3).
 *   slot2nnz[slot]         nonzero the slot is added to
 *   nnz2slot[nnz_slot_ptr[j] .. nnz_slot_ptr[j+1]-1]  slots of nonzero j, ascending
 */
int fe_pattern_slot_map(fe_pattern_h h, const int32_t** slot2nnz, const int32_t** nnz_slot_ptr,
                        const int32_t** nnz2slot);

/* Copies of the CSR arrays into caller-owned device buffers (row_ptr[n+1],
 * col_idx[nnz]); either pointer may be NULL. Stream-ordered. */
int fe_pattern_copy_csr(fe_pattern_h h, int32_t* row_ptr, int32_t* col_idx, void* stream);

/* Copies of the scalar slot maps (sizes as in fe_pattern_slot_map) and of the
 * internal element order (nme) into caller-owned device buffers; any may be NULL. */
int fe_pattern_copy_slot_map(fe_pattern_h h, int32_t* slot2nnz, int32_t* nnz_slot_ptr,
                             int32_t* nnz2slot, int32_t* order, void* stream);

/* Dimensions of a pattern: d, m, nq, nme, n = m nq, nnz. Any pointer may be NULL. */
int fe_pattern_dims(fe_pattern_h h, int32_t* d, int32_t* m, int64_t* nq, int64_t* nme, int64_t* n,
                    int64_t* nnz);

/* Borrowed internal element order (device int32[nme]): internal element e is
 * input element order[e]. Identity under FE_PATTERN_KEEP_ORDER. */
int fe_pattern_element_order(fe_pattern_h h, const int32_t** order);

/* Select the reassembly strategy used by later fe_assemble_* calls. Strategies
 * that need scratch memory allocate it here (synchronously), never inside an
 * assembly call. */
int fe_pattern_set_strategy(fe_pattern_h h, int32_t strategy);

/* Threads per block of the chunked kernel of the scalar operators: 128, 256
 * (default) or 512. Set by the autotuner (paper_1401_3301_gb300/tune.py). */
int fe_pattern_set_threads(fe_pattern_h h, int32_t threads);

/* Launch shape of fe_assemble_wmass_stiff: 1 (default) a persistent grid of as many
 * blocks as fit on the device at once, each looping over element chunks; 0 one block
 * per chunk. Set by the autotuner. FE_ERR_ARG for other values. */
int fe_pattern_set_persistent(fe_pattern_h h, int32_t persistent);

/* Device bytes held by the handle (pattern, plan and scratch). */
int fe_pattern_memory(fe_pattern_h h, int64_t* bytes);

/* Counts of the element-chunk plan used by FE_REASM_CHUNKED (for roofline
 * accounting): elements per chunk, distinct (chunk, vertex) and (chunk, edge)
 * pairs, how many of those are partial sums (the vertex or edge also belongs to
 * another chunk), distinct shared vertices and edges, and the plan's bytes.
 * Any pointer may be NULL. */
int fe_pattern_plan_info(fe_pattern_h h, int64_t* chunk, int64_t* local_vertices,
                         int64_t* local_edges, int64_t* partial_vertices, int64_t* partial_edges,
                         int64_t* shared_vertices, int64_t* shared_edges, int64_t* plan_bytes);

/* Device address and size in bytes of the plan record of element chunk c (the
 * layout is in csrc/plan.cuh; it starts with the uint16 local vertex of each element
 * corner, at e_local * nv + a). Borrowed: owned by the handle, valid until fe_pattern_destroy,
 * read by every chunked assembly. Synchronises the device to read the offsets.
 * FE_ERR_ARG for c outside [0, nchunks) or a handle without a chunk plan. */
int fe_pattern_plan_record(fe_pattern_h h, int64_t c, const void** rec, int64_t* bytes);

/*
 * fe_selftest_wait_timeout -- exercises the failure path of the kernels' bounded
 * waits without any fault: a one-block kernel waits on an mbarrier for 16 bytes that
 * no copy will bring, gives up after a short bound and records FE_ERR_TIMEOUT in a
 * status word, which is returned in *code (FE_ERR_TIMEOUT when the path works). The
 * CUDA context stays usable. Synchronous. The paper has no counterpart.
 */
int fe_selftest_wait_timeout(int32_t* code, void* stream);

/* Release everything the handle owns (synchronises the device first). */
int fe_pattern_destroy(fe_pattern_h h);

/*
 * Read and clear the device status word of h (synchronises `stream`).
 * *code is an FE_ERR_* (FE_OK if none) and *id the smallest offending element
 * (input element order) or -1.
 */
int fe_status(fe_pattern_h h, void* stream, int32_t* code, int64_t* id);

/*
 * Assembly into the fixed pattern of h (the value part of `sparse`). `vals`
 * receives nnz values, double for FE_F64 and float for FE_F32, in CSR order.
 * The pattern must have been built with m = 1.
 *
 * fe_assemble_mass  -- M_ij = int phi_j phi_i: local |K| d!/(d+2)! (1 + delta_ab),
 *                      i.e. |K|/12 (2D) and |K|/20 (3D) (Section 4.1, w = 1).
 * fe_assemble_wmass -- weighted mass int w phi_j phi_i (Eq. massw) with w given
 *                      per vertex and P1-interpolated (Eq. MatElemMassWP1:
 *                      d!/(d+3)! |K| (1 + delta_ab)(w^s + w_a + w_b)), or per
 *                      element (P0: w_K times the mass matrix). w_kind is
 *                      FE_COEF_P1, FE_COEF_P0 or FE_COEF_P0_INTERNAL.
 * fe_assemble_stiff -- S_ij = int w grad phi_j . grad phi_i with local
 *                      w_K |K| <grad lambda_b, grad lambda_a> (Eq. stiffelemmat,
 *                      Algorithm 7); w per element (FE_COEF_P0 or
 *                      FE_COEF_P0_INTERNAL) or FE_COEF_NONE.
 * Asynchronous on `stream`. Degenerate elements set FE_ERR_DEGENERATE in the
 * status word and leave `vals` unspecified.
 */
int fe_assemble_mass(fe_pattern_h h, const double* q, int32_t prec, void* vals, void* stream);
int fe_assemble_wmass(fe_pattern_h h, const double* q, const void* w, int32_t w_kind,
                      int32_t prec, void* vals, void* stream);
int fe_assemble_stiff(fe_pattern_h h, const double* q, const void* w, int32_t w_kind,
                      int32_t prec, void* vals, void* stream);

/*
 * fe_assemble_wmass_stiff -- the weighted mass and the stiffness matrix with the same
 * per-element coefficient in one pass, for repeated reassembly with new coefficients
 * (the motivation of Section 1; the paper assembles each matrix by its own pass,
 * Algorithms 6 and 7). vals_mass receives the matrix of fe_assemble_wmass and
 * vals_stiff that of fe_assemble_stiff for the same w / w_kind (FE_COEF_NONE: the
 * plain mass matrix and the unweighted stiffness), bit for bit: one chunk kernel
 * reads each plan record once, forms each element's geometry once and keeps both
 * matrices' sums in the separate calls' order; one fixup completes the shared
 * entries. w_kind: FE_COEF_NONE, FE_COEF_P0 or FE_COEF_P0_INTERNAL (w NULL only for
 * NONE). prec: FE_F64, FE_F32 or FE_F64X (w and both value arrays then FP64; one block per
 * chunk whatever the launch shape, and one fixup per matrix). Pattern: m = 1 volume pattern
 * from fe_pattern or fe_batch_pattern, chunked strategy (else FE_ERR_ARG). The two
 * value arrays must be distinct, nnz entries each. Asynchronous on `stream`; launch
 * shape as set by fe_pattern_set_persistent.
 */
int fe_assemble_wmass_stiff(fe_pattern_h h, const double* q, const void* w, int32_t w_kind,
                            int32_t prec, void* vals_mass, void* vals_stiff, void* stream);

/*
 * fe_assemble_elas -- elastic stiffness (Eq. StiffElasMat, Section 5.1) for an
 * isotropic Hooke law, pattern built with m = d. Local entry
 *   K_{(a,l),(b,n)} = |K|/(d+1) (lambda^s <g_b, Q^{n,l} g_a> + mu^s <g_b, S^{n,l} g_a>)
 * with Q^{n,l} = e_n e_l^T and S^{n,l} = delta_nl I + e_l e_n^T (Lemma
 * lem:VecLocalElas, App. B), lambda^s and mu^s the sums of the vertex values of
 * the P1 interpolants (a P0 or scalar coefficient counts as d+1 equal values).
 * lam_kind / mu_kind: FE_COEF_SCALAR, FE_COEF_P0, FE_COEF_P0_INTERNAL or FE_COEF_P1.
 * prec: FE_F64, FE_F32 or FE_F64X (double coefficients and values, double-float
 * arithmetic). Chunked strategy only.
 */
int fe_assemble_elas(fe_pattern_h h, const double* q, const void* lam, int32_t lam_kind,
                     const void* mu, int32_t mu_kind, int32_t prec, void* vals, void* stream);

/*
 * fe_assemble_general -- the general second-order operator of Eq. EDP,
 *   -div(A grad u) + div(b u) + c . grad u + a0 u,
 * which the paper states its algorithms extend to (remark after Eq. MagicFormula).
 * Weak form with the divergence terms on the test function and no boundary terms:
 *   a(u, v) = int (A grad u).grad v - int u b.grad v + int (c.grad u) v + int a0 u v,
 * entry (i, j) = a(phi_j, phi_i), NOT symmetric. Local entry of test vertex a and
 * trial vertex b (coefficients constant on K, g_a = grad lambda_a):
 *   |K| g_a^T A g_b - |K|/(d+1) b.g_a + |K|/(d+1) c.g_b + a0 |K| d!/(d+2)! (1 + delta_ab).
 * coef holds records of nc = d*d + 2d + 1 values (A row-major, b, c, a0), in the
 * precision of the form (double for FE_F64, float for FE_F32):
 *   FE_COEF_SCALAR       one record, coef[j];
 *   FE_COEF_P0           one per element in input element order, coef[k * nc + j];
 *   FE_COEF_P0_INTERNAL  the same in the pattern's internal element order;
 *   FE_COEF_P1           one per vertex, coef[v * nc + j], each coefficient
 *                        P1-interpolated on K and the integrals taken by the magic
 *                        formula (Eq. MagicFormula), as for Eq. MatElemMassWP1.
 * Records are read whole; a 16-byte aligned coef lets 3D records load as vectors.
 * Pattern: m = 1, built by fe_pattern or fe_batch_pattern (not a boundary pattern).
 * Every reassembly strategy for FE_F64 and FE_F32; FE_F64X (double coefficient records,
 * double-float arithmetic) with the chunked strategy only (FE_ERR_ARG otherwise).
 * Asynchronous on `stream`; degenerate elements as for the other operators.
 */
int fe_assemble_general(fe_pattern_h h, const double* q, const void* coef, int32_t coef_kind,
                        int32_t prec, void* vals, void* stream);

/*
 * fe_assemble_stiff_host -- fe_assemble_stiff with HOST buffers: q_host (d x nq
 * doubles, SoA), w_host (nme values of the form's precision, input element order, with
 * w_kind FE_COEF_P0; or NULL with FE_COEF_NONE) and vals_host (nnz values of the form's
 * precision) are in host memory, page-locked for the copies to be asynchronous. Forms
 * FE_F64, FE_F32 and FE_F64X.
 * The call returns at once; `stream` waits for the result to reach vals_host, so
 * synchronise it (or an event recorded on it) before reading vals_host. Successive calls
 * overlap: the pattern owns three streams (upload, assembly, download) and two device
 * staging slots, so call k's assembly runs beside call k+1's upload and call k-1's
 * download. The caller must not change q_host / w_host until the call's result is back
 * (or the next-but-one call on the pattern has started), nor read vals_host before.
 * The first call allocates the slots (2 x (q + values) on the device; w on demand).
 * Assemblies on one pattern share its scratch: do not mix this call with device-memory
 * calls on another stream without ordering them.
 */
int fe_assemble_stiff_host(fe_pattern_h h, const double* q_host, const void* w_host, int32_t w_kind,
                           int32_t prec, void* vals_host, void* stream);

/*
 * fe_assemble_stiff_backward -- gradients of L = u^T S(w) v, S the stiffness
 * matrix of fe_assemble_stiff, without forming any matrix (the paper has no
 * derivatives; these follow from Eq. stiffelemmat and App. C.1). Per element,
 * with ubar = sum_a u(me(a)) grad lambda_a and vbar likewise:
 *   L_K = w_K |K| ubar . vbar,     dL/dw_K = |K| ubar . vbar,
 *   dL/dq^c = sum_K w_K |K| [(ubar . vbar) g_c - ubar (g_c . vbar) - vbar (g_c . ubar)],
 * g_c the gradient of the barycentric coordinate of vertex c in K.
 *   w, w_kind   per-element coefficient (FE_COEF_NONE, FE_COEF_P0, FE_COEF_P0_INTERNAL)
 *   u, v        nq values each
 *   L           one value, or NULL
 *   dL_dw       nme values (input element order, or internal for
 *               FE_COEF_P0_INTERNAL), or NULL
 *   dL_dq       d x nq like q, or NULL
 * All of u, v, L, dL_dw, dL_dq (and w) use the precision of the form (double for
 * FE_F64 and FE_F64X, whose gradients are evaluated in double-float). Sums over
 * the elements of a vertex, and the sum of L, are taken in a fixed order
 * (bit-identical run to run). The first backward call on a handle allocates its
 * scratch (d (d+1) values per element) and builds the vertex -> element lists,
 * synchronously; later calls allocate nothing.
 */
int fe_assemble_stiff_backward(fe_pattern_h h, const double* q, const void* w, int32_t w_kind,
                               const void* u, const void* v, void* L, void* dL_dw, void* dL_dq,
                               int32_t prec, void* stream);

/*
 * fe_assemble_stiff_vjp -- vector-Jacobian product of the stiffness assembly: for
 * any loss L of the CSR values S(w, q), given grad_vals = dL/dS (nnz values, CSR
 * order), writes dL/dw (nme values, as in fe_assemble_stiff_backward) and dL/dq
 * (d x nq). Per element the weights G^_ab = grad_vals at the nonzero of slot (a, b)
 * enter dL/dw_K = |K| sum_ab G^_ab g_a . g_b and
 * dL/dq^c = w_K |K| [t g_c - sum_x g_x ((G^ + G^T) Gamma)_xc], t = sum_ab G^_ab
 * Gamma_ab, Gamma_ab = g_a . g_b. Same scratch rules as fe_assemble_stiff_backward.
 */
int fe_assemble_stiff_vjp(fe_pattern_h h, const double* q, const void* w, int32_t w_kind,
                          const void* grad_vals, void* dL_dw, void* dL_dq, int32_t prec,
                          void* stream);

/*
 * Per-kernel timing. fe_profile(h, 1) makes every later kernel launch of h be
 * bracketed by a CUDA event pair on its stream and by an NVTX range named after the
 * kernel (visible to a timeline profiler; a no-op without one). fe_profile(h, 0) stops
 * and frees them. fe_profile_read synchronises on the recorded events and returns, per
 * kernel kind launched since the last read, its name (32-byte slots in `names`),
 * total milliseconds and launch count; *count receives the number of kinds
 * (entries beyond max_kernels are dropped). Host pointers.
 */
int fe_profile(fe_pattern_h h, int32_t enable);
int fe_profile_read(fe_pattern_h h, int32_t max_kernels, char* names, double* ms,
                    int64_t* launches, int32_t* count);

/*
 * fe_assemble_stiff_noalloc -- the stiffness assembly of fe_assemble_stiff (same
 * arguments, with prec FE_F64 or FE_F32 only: FE_F64X gives FE_ERR_ARG; same result up
 * to the summation order), computed by the two-pass scheme of FE_REASM_GATHER, that
 * allocates no device memory. The paper has no
 * counterpart: this exists for callers that may not call cudaMalloc while they
 * assemble, such as a plugin inside an application that owns the whole
 * device-memory budget, or a time-stepping loop that cannot afford the device
 * synchronisation cudaMalloc may cause. Build the pattern first (fe_pattern
 * allocates); this call then reads the handle and writes `vals`, and in FE_F32 also
 * rewrites the handle's split-coordinate buffer (allocated with the pattern).
 *   - Its element values go to a fixed 16 MiB scratch array that is part of the
 *     library's device image (every GPU that loads the library holds it until the
 *     process exits). Meshes that need more, i.e. nme (d+1)^2 times 8 bytes
 *     (FE_F64) or 4 bytes (FE_F32) above 16 MiB, are rejected with
 *     FE_ERR_SCRATCH_LIMIT before anything is launched (3D: up to 131,072 tets
 *     in FP64, 262,144 in FP32).
 *   - The first call on a device looks up the scratch array's device address
 *     (cudaGetSymbolAddress, no allocation) with that device current, and caches
 *     it; make that first call before any stream capture. The cache lives as long as
 *     the process's device contexts: a cudaDeviceReset invalidates it, as it does
 *     every pattern handle's device memory.
 *   - Every call, on any handle, shares the one scratch array, which keeps the last
 *     call's contents: two calls whose kernels overlap on the GPU (different
 *     streams, no ordering between them) race and give wrong results. Every slot
 *     the second pass reads is written by the first, so nothing needs clearing.
 *   - In FE_F32 the call also rewrites the handle's split-coordinate buffer, which the
 *     FE_F32 calls of fe_assemble_stiff (gather and atomic strategies), of
 *     fe_assemble_general and of the backward calls on the same handle use too: order
 *     such calls on one handle (one stream, or events), even where neither of them
 *     uses the scratch array.
 */
int fe_assemble_stiff_noalloc(fe_pattern_h h, const double* q, const void* w, int32_t w_kind,
                              int32_t prec, void* vals, void* stream);

/* Library version string (host pointer, static); the bounds-checked build (compiled
 * with FE_CHECKED) says "bounds-checked" in it. */
const char* fe_version(void);

/* Text of the last CUDA runtime error the library saw on the calling host thread
 * (host pointer to a per-thread buffer, valid until that thread's next failing
 * call; empty if none). */
const char* fe_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FE_GB300_H */
