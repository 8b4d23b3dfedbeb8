/* gfmom: GB300 (sm_103a) method-of-moments impedance-matrix fill with the
 * adaptive interpolation tables of Yang & Su, "Fast Green Function
 * Evaluation for Method of Moment".
 *
 * Operator (Section II.A, Section IV.B: EFIE "L" operator, RWG basis on
 * planar triangles, Galerkin testing), e^{jwt} convention:
 *   Z_mn = jk eta int_{T_m} int_{T_n} [f_m . f_n - (1/k^2) div f_m div' f_n]
 *          e^{-jkR} / (4 pi R) dS' dS.
 * Regular triangle pairs use the m-point rule on both triangles with
 * e^{-jkR}/R from the Lagrange table (Eq. 3, 5) or from sincos/exp; near pairs
 * (sharing a vertex, or centroids closer than near_dist) use singularity
 * cancellation with an angular transformation in FP64, with e^{-jkR} on the
 * source edges from the linear table (Eq. 3, 4) when r_min <= R <= r_max
 * (Section II.C), else directly.
 *
 * Conventions
 *   - RWG unknown n = the n-th interior edge in lexicographic order of its
 *     (lower, higher) vertex-index pair; T+ = the adjacent triangle with the
 *     smaller index. Boundary edges carry no unknown; an edge shared by more
 *     than two triangles is an error.
 *   - Z is row-major on the device: Z[m * ldz + n] = Z_mn (test edge m,
 *     source edge n), ldz >= ne, complex64 (GF_FP32) or complex128 (GF_FP64)
 *     as interleaved (re, im).
 *   - Device pointers, sizes and the stream are the caller's; the caller owns
 *     every buffer it passes. The library owns its handles and the device
 *     memory inside them (geometry, near lists, table images, a mesh's list of
 *     flagged point pairs), released by the matching *_destroy (kept in a
 *     small pool for the next handle of a similar size). Handles are bound to the device that was
 *     current at creation; calls must be made with that device current.
 *   - Calls that launch kernels are asynchronous on `stream` (a cudaStream_t,
 *     NULL = legacy default stream) unless stated otherwise.
 *   - Every call returns GF_OK or a negative status; gf_last_error() gives the
 *     message of the calling thread's last failure. Nothing is thrown across
 *     the ABI.
 */
#ifndef GFMOM_H
#define GFMOM_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef int gf_status;
#define GF_OK 0
#define GF_ERR_ARG (-1)     /* invalid argument (null pointer, bad size, bad option) */
#define GF_ERR_MESH (-2)    /* degenerate / non-manifold mesh, bad vertex index */
#define GF_ERR_RANGE (-3)   /* no regular pair, or a table that would be too large */
#define GF_ERR_CUDA (-4)    /* a CUDA runtime call failed */
#define GF_ERR_ALLOC (-5)   /* device or host allocation failed */
#define GF_ERR_DEVICE (-6)  /* handle used with another device current */

#define GF_FP32 32          /* FP32 quadrature with Kahan outer sums, complex64 Z */
#define GF_FP64 64          /* FP64 throughout, complex128 Z */

#define GF_GREEN 1          /* e^{-jkr}/r, Lagrange table */
#define GF_EXP 0            /* e^{-jkr}, linear table */

typedef struct gf_mesh gf_mesh;
typedef struct gf_table gf_table;

typedef struct {
  int rule;                   /* points per triangle: 1, 3, 4, 6, 7 (Dunavant)          */
  double table_tol;           /* relative tolerance of both tables (default 1e-6)       */
  int green_n_per_lambda;     /* Green table base samples per wavelength, Eq. (2) (1000)*/
  int exp_n_per_lambda;       /* Exp table samples per wavelength; 0 = smallest multiple
                                 of 4 in [1000, 10000] with (k t)^2/8 <= tol, Eq. (10)   */
  int lagrange_degree;        /* degree n of Eq. (5) for the Green table (3)            */
  int refine;                 /* local refinement + forced zeros, Section II.B (1)      */
  double refine_factor;       /* refined spacing / t (0.5)                              */
  double refine_halfwidth_t;  /* refinement window |r - z| <= this * t (2.0 = "4t")     */
  double merge_t;             /* samples closer than this * t to a zero are dropped (0.25) */
  int grade;                  /* bisect intervals whose Eq. (11) bound exceeds tol (1)  */
  int nphi;                   /* angular points per source edge, near pairs (8)         */
  int nl;                     /* line points per source edge, near pairs (8)            */
  double eta;                 /* wave impedance (376.730313668)                         */
  int near_fp64;              /* GF_FP32 fills: 0 = near pairs with FP64 geometry and
                                 static parts, FP32 sampling on the source edges and FP32
                                 assembly of the 3x3 block from the inner integrals;
                                 1 = FP64 throughout (GF_FP64 fills always are) (0)       */
  int green_from_exp;         /* regular pairs of gf_fill / gf_fill_parts with a table:
                                 0 = e^{-jkR}/R from the Lagrange Green table (Section
                                 II.C); 1 = e^{-jkR} from the linear Exp table times 1/R
                                 (one 16-byte record per evaluation in FP32). gf_batch_*
                                 and gf_fill_backward accept 0 only (0)                   */
} gf_params;

/* Fills *p with the defaults listed above. */
void gf_params_default(gf_params* p);

/* Message of the calling thread's last failure ("" if none). */
const char* gf_last_error(void);

/* ---------------------------------------------------------------- mesh ---
 * xyz: host [nv][3] float64, tri: host [nt][3] int32 (copied). Builds the RWG
 * edges and the near-pair lists on the host, uploads the geometry to the
 * current device (synchronous). near_dist > 0 adds every pair of triangles
 * whose centroids are closer than near_dist to the vertex-sharing near pairs.
 * Errors: GF_ERR_ARG (null, nv < 3, nt < 1), GF_ERR_MESH (index out of range,
 * repeated vertex in a triangle, edge shared by more than two triangles),
 * GF_ERR_CUDA / GF_ERR_ALLOC. */
gf_status gf_mesh_create(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt,
                         double near_dist, gf_mesh** out);

/* Sizes: vertices, triangles, RWG edges, ordered near pairs (p, q) (any may be NULL). */
gf_status gf_mesh_info(const gf_mesh* m, int64_t* nv, int64_t* nt, int64_t* ne, int64_t* n_near);

/* Host copies: edge_verts [ne][2] (lower, higher), edge_tris [ne][2] (T+, T-);
 * either may be NULL. */
gf_status gf_mesh_edges(const gf_mesh* m, int32_t* edge_verts, int32_t* edge_tris);

/* Replaces the vertex coordinates (host [nv][3] float64, same topology) and
 * re-uploads the geometry (synchronous). Near lists are kept. */
gf_status gf_mesh_set_vertices(gf_mesh* m, const double* xyz);

gf_status gf_mesh_destroy(gf_mesh* m);

/* ---------------------------------------------------------------- range --
 * Minimum and maximum distance between integration points of the `rule` over
 * all regular (not near) triangle pairs: the table range of Section II.B
 * (abstract: "the maximum and minimum distance between any two integration
 * points"). GF_FP64 reduces FP64 distances; GF_FP32 screens with FP32
 * distances and reports the FP64 distance of the extremal point pairs.
 * Runs on the device on `stream`, then synchronizes it and writes the two
 * host doubles. GF_ERR_RANGE if every pair is near. */
gf_status gf_range(const gf_mesh* m, int rule, int precision, double* r_min, double* r_max,
                   void* stream);

/* ---------------------------------------------------------------- tables -
 * Builds the Green (Lagrange, Eq. 3 + 5) and Exp (linear, Eq. 3 + 4) tables
 * of Section II.B-C over [r_min, r_max] for wavenumber k: sample positions on
 * the host in FP64 (uniform t from r_min, refinement near the zeros of the
 * real and imaginary parts, forced zeros, Eq. (11) grading), then sample
 * values, per-interval polynomial coefficients (FP64 and FP32 images) and the
 * hash array of Eq. (6) by kernels queued on `stream`. The call returns once
 * the uploads and kernels are queued (it does not wait for them): the table is
 * ready for work later on `stream`; other streams must wait for `stream`.
 * The device memory is one allocation owned by the table.
 * Errors: GF_ERR_ARG (k <= 0, r_min <= 0, r_max <= r_min, bad params),
 * GF_ERR_RANGE (more than 2^26 samples or hash cells, samples closer than the
 * FP32 / FP64 images resolve), GF_ERR_CUDA / GF_ERR_ALLOC. */
gf_status gf_table_create(double k, double r_min, double r_max, const gf_params* p, void* stream,
                          gf_table** out);

/* The same tables in u = kR, for frequency sweeps: one table serves every
 * wavenumber k with [k r_min, k r_max] inside [u_min, u_max] (e^{-jkR} =
 * e^{-ju}, e^{-jkR}/R = k e^{-ju}/u; the tables are those of gf_table_create
 * with k = 1 over [u_min, u_max]). The fills (gf_fill, gf_fill_parts,
 * gf_fill_mfie, gf_fill_sparse, gf_batch_create) read it at x = kR for their
 * own k; the caller keeps [k r_min, k r_max] of each mesh inside [u_min,
 * u_max]. gf_fill_backward rejects it (GF_ERR_ARG). Errors as above. This is a
 * variant of the method, not in the paper. */
gf_status gf_table_create_kr(double u_min, double u_max, const gf_params* p, void* stream, gf_table** out);

/* kind = GF_GREEN or GF_EXP: number of samples, hash cells, hash cell width
 * (= smallest sample spacing); any output may be NULL. */
gf_status gf_table_info(const gf_table* t, int kind, int64_t* n_nodes, int64_t* n_hash, double* dr);

/* Host copies of one table: sample positions r [n_nodes], sample values
 * (fre, fim) [n_nodes] and the hash array [n_hash]; any may be NULL. */
gf_status gf_table_nodes(const gf_table* t, int kind, double* r, double* fre, double* fim,
                         int32_t* hash);

/* Device lookup of n distances: r_dev is float (GF_FP32) or double (GF_FP64),
 * out_dev is interleaved complex of the same type: the table's f(r) (Green:
 * e^{-jkr}/r, Exp: e^{-jkr}, without 1/(4 pi)). Points outside [r_min, r_max]
 * are clamped to the first / last interval. Asynchronous on `stream`. */
gf_status gf_table_eval(const gf_table* t, int kind, int precision, const void* r_dev, int64_t n,
                        void* out_dev, void* stream);

/* Host FP64 lookup of n points x (host [n], table units: R, or u = kR for a
 * table of gf_table_create_kr) through the FP64 cell image of the Eq. (6)
 * hash: exact bracketing against the samples, then the interval's FP64
 * polynomial (Eq. 4 for GF_EXP, Eq. 5 for GF_GREEN). out: host [n][2]
 * float64 (re, im) of e^{-jkr}/r or e^{-jkr} (without 1/(4 pi)).
 * Synchronous (copies the FP64 image from the device). GF_ERR_RANGE if some
 * x lies outside [r_min, r_max] (below r_min the fills evaluate directly). */
gf_status gf_table_eval_host(const gf_table* t, int kind, const double* x, int64_t n, double* out);

/* gf_table_create over the range of a mesh: r_min < 0 or r_max < 0 are
 * replaced by gf_range(m, p->rule, precision) (which synchronizes `stream`).
 * The paper builds its tables over "the maximum and minimum distance between
 * any two integration points" (abstract); errors as gf_range and
 * gf_table_create. */
gf_status gf_table_create_for_mesh(const gf_mesh* m, double k, const gf_params* p, int precision, double r_min,
                                   double r_max, void* stream, gf_table** out);

gf_status gf_table_destroy(gf_table* t);

/* ---------------------------------------------------------------- fill ---
 * Fills Z (device, row-major, ld = ldz) for wavenumber k. table == NULL
 * selects direct evaluation (sincos / exp) everywhere; otherwise regular
 * pairs use its Green table and near pairs its Exp table (the table must
 * cover the range of gf_range for this mesh and rule; distances outside it
 * fall back to direct evaluation in the near-pair path). precision GF_FP32
 * (complex64 Z) or GF_FP64 (complex128 Z). Z is overwritten. Asynchronous on
 * `stream`. An FP32 fill with a table (green_from_exp = 0) keeps, in the
 * mesh, a list of the point pairs whose Green lattice cell holds samples
 * (corrected by a second kernel), sized from the table's share of such cells
 * (at most 1 GiB) and allocated by the first fill that needs it (cudaMalloc,
 * which synchronizes the device). So fills of one mesh must not overlap on
 * different streams. The environment variable GF_FIX_ENTRIES, if set,
 * replaces that size (0: no list, each pair corrected in the pair kernel; a
 * list too small for some CTA makes that CTA scan its pairs again): the
 * results are the same either way. */
gf_status gf_fill(const gf_mesh* m, double k, const gf_params* p, const gf_table* table,
                  int precision, void* Z_dev, int64_t ldz, void* stream);

/* The stages of gf_fill, for callers that time or overlap them: GF_PART_ZERO
 * clears the ne x ne block of Z, GF_PART_REGULAR adds the regular-pair terms,
 * GF_PART_NEAR adds the near-pair terms (one kernel). gf_fill is
 * gf_fill_parts with all three, in that order. GF_PART_REGULAR is the two
 * stages GF_PART_PAIRS | GF_PART_MIRROR: in GF_FP32 the pair kernel adds each
 * unordered triangle pair's terms to the rows of its test triangle's edges
 * only, and the mirror kernel then sets Z <- Z + Z^T (one HBM pass); in
 * GF_FP64 the pair kernel writes both halves and the mirror stage does
 * nothing. So the regular stage expects the block cleared (GF_PART_ZERO in
 * the same or an earlier call on the stream) and no near terms yet: the
 * mirror doubles whatever the block held before. parts = 0 or a bit outside
 * the five is GF_ERR_ARG. */
#define GF_PART_ZERO 1u
#define GF_PART_REGULAR 2u
#define GF_PART_NEAR 4u
#define GF_PART_PAIRS 8u
#define GF_PART_MIRROR 16u
gf_status gf_fill_parts(const gf_mesh* m, double k, const gf_params* p, const gf_table* table,
                        int precision, void* Z_dev, int64_t ldz, unsigned parts, void* stream);

/* ---------------------------------------------------------------- adjoint --
 * Backward of the fill (no counterpart in the paper; the gradient of a loss of
 * Z with respect to the geometry and the wavenumber). gZ: device complex64
 * [ne][ldg], the upstream gradient in the convention dL = Re sum conj(gZ) dZ
 * (PyTorch's for a real loss). Writes dxyz (device float64 [nv][3], original
 * vertex ids) = dL/d(vertex coordinates) and *dk (device float64) = dL/dk.
 * Regular pairs: FP32 reverse mode with the Green values recomputed from
 * `table` (direct if NULL), F' = -(jk + 1/R) F, dF/dk = -jR F. Near pairs:
 * reverse mode (all 19 directions of the pair's coordinates and k in one
 * pass) with FP64 geometry and static parts and FP32 edge sampling; with
 * p->near_fp64, forward mode with FP64 dual numbers (one pass per
 * direction). The
 * near / regular classification, the table range and its samples are held
 * fixed. precision must be GF_FP32. Asynchronous on `stream`; uses per-mesh
 * scratch, so backward calls on one mesh must not overlap. */
gf_status gf_fill_backward(const gf_mesh* m, double k, const gf_params* p, const gf_table* table,
                           int precision, const void* gZ, int64_t ldg, double* dxyz, double* dk,
                           void* stream);

/* ---------------------------------------------------------------- near field
 * Z restricted to a sparsity pattern: the near-field matrix a fast solver
 * keeps (the paper's "3mnNC" count, Section II.A, for the regime of large N).
 * The pattern holds the RWG pairs (m, n) with some triangle of m and some
 * triangle of n whose centroids are closer than `radius`; its values are the
 * full Z_mn of gf_fill (all four triangle pairs), so on the pattern they equal
 * the dense fill's entries.
 *
 * gf_sparse_create: builds the pattern (host) and the work list of triangle
 * pairs; `m` must outlive the handle. GF_ERR_ARG for radius <= 0.
 * gf_sparse_info: nnz of the pattern and the number of regular triangle pairs
 * evaluated by a fill. gf_sparse_pattern: the CSR pattern on the host
 * (row_ptr [ne + 1] int64, cols [nnz] int32 sorted per row; either may be NULL).
 * gf_fill_sparse: vals (device complex64 [nnz], pattern order) overwritten
 * with Z_mn; FP32 only (GF_ERR_ARG otherwise), the same kernels and options as
 * gf_fill (Green table for regular pairs, Exp table and p->near_fp64 for near
 * pairs; table == NULL: direct). Asynchronous on `stream`.
 * gf_sparse_destroy: synchronizes the device, frees the handle. */
typedef struct gf_sparse gf_sparse;
gf_status gf_sparse_create(const gf_mesh* m, double radius, gf_sparse** out);
gf_status gf_sparse_info(const gf_sparse* s, int64_t* nnz, int64_t* n_pairs);
gf_status gf_sparse_pattern(const gf_sparse* s, int64_t* row_ptr, int32_t* cols);
gf_status gf_fill_sparse(const gf_sparse* s, double k, const gf_params* p, const gf_table* table, int precision,
                         void* vals_dev, void* stream);
gf_status gf_sparse_destroy(gf_sparse* s);

/* ---------------------------------------------------------------- MFIE -----
 * The magnetic-field integral equation matrix (the paper's second formulation,
 * Section IV.B: its K operator uses the gradient of the same Green function,
 * so the same tables serve it) for a CLOSED PEC surface whose triangles are
 * wound counter-clockwise seen from outside (outward normals), e^{jwt}:
 *   Z_mn = 1/2 <f_m, f_n> - <f_m, n x PV int grad G x f_n dS'>,
 *   grad G = -(r - r') (1 + jkR) e^{-jkR} / (4 pi R^3).
 * Regular pairs: the m-point rule on both triangles, every ordered pair,
 * e^{-jkR}/R from the table's Green (Lagrange) table (or direct sincos with
 * table == NULL), FP32 with Kahan outer sums (GF_FP32) or FP64. Pairs sharing
 * a vertex and the self pair: FP64, the inner integral of grad G x (r' - v)
 * as three edge line integrals (static part in closed form, e^{-jkR} - 1 by
 * p->nl Gauss points) plus a solid-angle term (angles by p->nphi Gauss points),
 * e^{-jkR} from the Exp table when a table is given. Z (device, row-major,
 * ld = ldz, complex64 / complex128) is overwritten. Asynchronous on `stream`.
 * The right side for a plane wave is gf_excitation with GF_OP_MFIE. */
gf_status gf_fill_mfie(const gf_mesh* m, double k, const gf_params* p, const gf_table* table, int precision,
                       void* Z_dev, int64_t ldz, void* stream);

/* ---------------------------------------------------------------- scattering
 * Plane-wave excitation and far field of an RWG current: with a solve of
 * Z I = V (any dense solver) they turn the filled EFIE matrix into the
 * bistatic radar cross section, the quantity the paper compares between the
 * table and the direct fill (Section IV.B). Not part of the fill's hot path;
 * FP64 arithmetic. Both use the rule p->rule on every triangle and the RWG
 * convention of gf_fill (f_n = +-l_n/(2A)(r - v_opp) on T+ / T-).
 *
 * gf_excitation: the right side of Z I = V for the incident plane wave
 * E_inc = p e^{-jk khat.r} (e^{jwt}; it travels along khat): with op =
 * GF_OP_EFIE, V_m = <f_m, E_inc> (the Z of gf_fill); with GF_OP_MFIE,
 * V_m = <f_m, n x H_inc>, H_inc = (khat x p) e^{-jk khat.r} / eta (the Z of
 * gf_fill_mfie; eta = p->eta). khat: host [3], a unit vector (GF_ERR_ARG
 * otherwise); pol: host [3][2] float64, the complex polarisation (re, im per
 * component); V: device [ne] complex64 (GF_FP32) or complex128 (GF_FP64),
 * overwritten. k >= 0. Asynchronous on `stream`.
 *
 * gf_far_field: for each of n_dir directions d (device float64 [n_dir][3],
 * unit vectors), F(d) = -(j k eta / 4 pi)(N - (d.N) d) with
 * N = sum_n I_n int f_n e^{jk d.r'} dS' (the scattered field is
 * F e^{-jkr} / r far away), written to F (device float64 [n_dir][3][2],
 * complex128), and sigma (device float64 [n_dir]) = 4 pi |F|^2, the bistatic
 * radar cross section for a unit incident field. I: device [ne] complex64
 * (GF_FP32) or complex128 (GF_FP64). eta = p->eta. Asynchronous on `stream`. */
#define GF_OP_EFIE 0
#define GF_OP_MFIE 1
gf_status gf_excitation(const gf_mesh* m, double k, const gf_params* p, const double* khat, const double* pol,
                        int op, int precision, void* V, void* stream);
gf_status gf_far_field(const gf_mesh* m, double k, const gf_params* p, int precision, const void* I,
                       int64_t n_dir, const double* dirs, double* F, double* sigma, void* stream);

/* ---------------------------------------------------------------- batched --
 * Many meshes in one launch per kernel: each mesh i has its own wavenumber
 * k[i], tables[i] (built for k[i] over that mesh's gf_range; tables == NULL:
 * direct evaluation for all) and Z[i] (device, row-major, complex64, ld
 * ldz[i]); all share the params (rule, near-pair options). The work of all
 * meshes forms one task list, largest meshes first, pulled by persistent
 * kernels through an atomic counter; the zeroing of every Z and the kernels
 * are captured once into a CUDA graph on a stream owned by the batch
 * (Section II.A fill; the batching is this library's, not the paper's).
 * autotune != 0 times the launch shapes (block size, CTAs per SM, task
 * chunk) on the batch and keeps the fastest; choices are cached in the file
 * named by $GF_AUTOTUNE_CACHE when it is set (unset, empty or "off": no
 * cache file; the library writes no other host file). precision must be GF_FP32. Meshes, tables and Z must
 * outlive the batch; the batch stores their device pointers. gf_batch_create
 * synchronizes `stream`. */
typedef struct gf_batch gf_batch;
gf_status gf_batch_create(int nmesh, const gf_mesh* const* meshes, const double* k, const gf_params* p,
                          const gf_table* const* tables, int precision, void* const* Z, const int64_t* ldz,
                          int autotune, void* stream, gf_batch** out);

/* Replays the captured graph on `stream` (asynchronous): refills every Z. */
gf_status gf_batch_launch(const gf_batch* b, void* stream);

/* The launch shape in use and the tuner's time per launch (0 if not tuned). */
gf_status gf_batch_config(const gf_batch* b, int* block, int* ctas_per_sm, int* chunk, double* tuned_ms);

gf_status gf_batch_destroy(gf_batch* b);

/* One-shot batched fill: gf_batch_create (no tuning) + gf_batch_launch on
 * `stream` + gf_batch_destroy. Returns after the fill has completed (it
 * synchronizes `stream`); keep a gf_batch to refill the same meshes again
 * without the set-up. Arguments and errors as gf_batch_create (GF_FP32). */
gf_status gf_fill_batched(int nmesh, const gf_mesh* const* meshes, const double* k, const gf_params* p,
                          const gf_table* const* tables, void* const* Z, const int64_t* ldz, void* stream);

/* ---------------------------------------------------------------- no-alloc -
 * gf_range for callers that cannot allocate device memory (for example code
 * running while a CUDA graph is captured, or a plug-in whose host application
 * owns every device allocation). The paper has no counterpart: this is a
 * deployment variant of the range reduction above. It allocates nothing: its
 * scratch (the integration points and a min/max accumulator) is a fixed
 * array of (GF_NOALLOC_MAX_POINTS + 1) x 32 bytes (4 MiB) inside the library,
 * present on every GPU that loads the library until the process exits.
 *
 * tri_xyz: device [nt][9] float64, the three vertices of each triangle;
 * tri_vert: device [nt][3] int32 vertex ids (pairs sharing a vertex are near
 * pairs and are skipped; no centroid criterion); minmax: device [2] float64,
 * written with (r_min, r_max) over the FP64 distances between the `rule`
 * points of all other pairs ((+inf, 0) if there is none). Asynchronous on
 * `stream`. GF_ERR_ARG if nt * rule > GF_NOALLOC_MAX_POINTS, a pointer is
 * null, nt < 1 or the rule is not 1, 3, 4, 6 or 7.
 * The first call on a device looks up the scratch array's device address
 * (once per device and driver context, with that device current; after a
 * cudaDeviceReset the next call looks it up again); make that first call
 * before any stream capture. Every call on a device shares the one scratch array:
 * calls whose work overlaps on the GPU (other streams, other threads) race
 * and give wrong results; serialize them. */
#define GF_NOALLOC_MAX_POINTS 131072
gf_status gf_range_noalloc(const double* tri_xyz, const int32_t* tri_vert, int64_t nt, int rule,
                           double* minmax, void* stream);

#ifdef __cplusplus
}
#endif
#endif
