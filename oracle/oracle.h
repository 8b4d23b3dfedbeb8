/* FP64 CPU oracle for the EFIE / RWG impedance-matrix fill with the adaptive
 * interpolation tables of Yang & Su, "Fast Green Function Evaluation for
 * Method of Moment".
 *
 * TEST INFRASTRUCTURE ONLY. This library is the plain, slow, obviously
 * correct definition that the CUDA library is checked against. Only the test
 * suite, the smoke check and the benchmark's CPU-baseline / reference arm
 * may load it. It shares no code, header, constant or table generator with
 * the CUDA library.
 *
 * Conventions (all lengths in the same unit as 2*pi/k):
 *   - e^{jwt} time convention, Green function G(R) = e^{-jkR} / (4 pi R).
 *   - RWG edge n = the n-th interior edge in lexicographic order of its
 *     (lower, higher) vertex-index pair; T+ = the adjacent triangle with the
 *     smaller index, T- the other one. Boundary edges carry no unknown.
 *   - Z[m][n] = test edge m, source edge n (Galerkin, EFIE L operator).
 *
 * Every function returns 0 on success and a negative code on bad input.
 */
#ifndef GF_ORACLE_H
#define GF_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_mesh or_mesh;
typedef struct or_table or_table;

/* Triangle quadrature (Section II.A: m-point rule on each triangle).
 * npts in {1,3,4,6,7}; bary is [npts][3], w is [npts] with sum(w) = 1. */
int or_rule(int npts, double* bary, double* w);

/* Gauss-Legendre nodes/weights on [-1, 1]. */
int or_gauss_legendre(int n, double* x, double* w);

/* Mesh: vertices [nv][3], triangles [nt][3] (int32). near_dist > 0 adds the
 * pairs whose centroid distance is below it to the vertex-sharing near pairs. */
int or_mesh_new(const double* xyz, int nv, const int* tri, int nt, double near_dist, or_mesh** out);
int or_mesh_ne(const or_mesh* m);
/* edges [ne][2] vertex ids, etri [ne][2] = (T+, T-) */
int or_mesh_edges(const or_mesh* m, int* edges, int* etri);
int or_mesh_is_near(const or_mesh* m, int p, int q);
void or_mesh_free(or_mesh* m);

/* Table of f(r) = e^{-jkr} (kind 0) or e^{-jkr}/r (kind 1) on [r_lo, r_hi]
 * (Section II.B-C). degree 1 = linear (Eq. 3-4), degree >= 2 = Lagrange
 * (Eq. 3, 5). t = base spacing (Eq. 2). refine: local refinement near zeros of
 * Re/Im with spacing t*refine_factor over |r - z| <= refine_halfwidth and zero
 * forcing with merge distance `merge`. grade: bisect every interval whose
 * Eq. (11) relative bound exceeds tol. */
typedef struct {
  int kind;
  int degree;
  double k, r_lo, r_hi;
  double t;
  double tol;
  int refine;
  double refine_factor;    /* 0.5 */
  double refine_halfwidth; /* absolute, e.g. 2 t */
  double merge;            /* absolute, e.g. t / 4 */
  int grade;
} or_table_params;

int or_table_new(const or_table_params* p, or_table** out);
/* n_nodes, n_hash, dr (= min node spacing, the hash cell width of Eq. 6) */
int or_table_info(const or_table* t, int* n_nodes, int* n_hash, double* dr);
/* copies nodes r[n_nodes], values fre/fim[n_nodes], hash[n_hash] (any may be NULL) */
int or_table_get(const or_table* t, double* r, double* fre, double* fim, int* hash);
/* interval index j (r_j <= r < r_{j+1}) from the hash of Eq. 6, for n points */
int or_table_locate(const or_table* t, int n, const double* r, int* j);
/* interpolated f at n points (Eq. 3-5) */
int or_table_eval(const or_table* t, int n, const double* r, double* re, double* im);
/* Eq. (11) relative bound of interval j (the grading criterion) */
double or_table_bound(const or_table* t, int j);
void or_table_free(or_table* t);

/* Inner integrals over source triangle (v0,v1,v2) for observation point r,
 * by singularity cancellation with the angular transformation (Section II.A):
 *   I0 = int_T G dS',  I1 = int_T (r' - rho0) G dS'   (G includes 1/(4 pi))
 * rho0 = projection of r on the triangle's plane (returned). texp may be NULL
 * (direct Exp evaluation); otherwise Exp values with r_lo <= R <= r_hi come
 * from it. */
int or_singular(const double* r, const double* v0, const double* v1, const double* v2, double k,
                int nphi, int nl, const or_table* texp, double* i0 /*[2]*/, double* i1 /*[6]*/,
                double* rho0 /*[3]*/);

/* Min / max distance between integration points over all regular (not near)
 * triangle pairs (Section II.B: table range). */
int or_range(const or_mesh* m, int rule, double* r_min, double* r_max, int nthreads);
/* The same result; prune = 1 skips triangle pairs that cannot hold an extreme
 * (centroid-distance bounds), for large meshes. */
int or_range_ex(const or_mesh* m, int rule, int prune, double* r_min, double* r_max, int nthreads);

/* Z entries (m_i, n_i), i < nent. green_mode 0: direct; 1: tables (tgreen for
 * regular pairs, texp for the near-pair line integrals); 2: texp for both, the
 * regular-pair Green value being e^{-jkR} from the Exp table times 1/(4 pi R)
 * (tgreen unused). */
typedef struct {
  double k;
  double eta;
  int rule;
  int nphi;
  int nl;
  int green_mode;
} or_fill_params;

int or_z_entries(const or_mesh* m, const or_fill_params* p, const or_table* tgreen,
                 const or_table* texp, long nent, const int* mi, const int* ni, double* zre,
                 double* zim, int nthreads);

/* Loss L = Re(a^H Z b) and its gradient by forward-mode dual numbers:
 * dxyz[nv][3] += dL/dx, *dk = dL/dk. Direct Green evaluation. */
int or_loss_grad(const or_mesh* m, const or_fill_params* p, const double* are, const double* aim,
                 const double* bre, const double* bim, double* loss, double* dxyz, double* dk,
                 int nthreads);

/* As or_loss_grad, but only triangle pairs with p or q marked in tri_mask
 * [nt] contribute (exact gradient for vertices whose triangles are all
 * marked; dk and the loss partial). */
int or_loss_grad_masked(const or_mesh* m, const or_fill_params* p, const double* are, const double* aim,
                        const double* bre, const double* bim, const int* tri_mask, double* loss, double* dxyz,
                        double* dk, int nthreads);
/* L and dL/dk over all pairs (one dual direction). */
int or_loss_dk(const or_mesh* m, const or_fill_params* p, const double* are, const double* aim, const double* bre,
               const double* bim, double* loss, double* dk, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
