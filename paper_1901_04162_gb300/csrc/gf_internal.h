// Internal declarations of the gfmom library (host side and kernels).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gfmom.h"

namespace gf {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxRule = 7;
// FP32 range scratch after the candidate list of block pairs: one record pair
// (12 bytes each) per pass-2 block, at most kRangeMaxBlocks blocks.
constexpr int kRangeMaxBlocks = 4096;
inline size_t range_list_ints(int64_t nt) {
  const int64_t nb = (nt + 31) / 32, nbp = nb * (nb + 1) / 2;
  return (size_t)((nbp + 3) & ~int64_t(3)) + 6 * (size_t)kRangeMaxBlocks;
}

}  // namespace gf
struct gf_mesh;
struct gf_table;
namespace gf {

// ---------------------------------------------------------------- errors
gf_status fail(gf_status st, const std::string& msg);
gf_status cuda_fail(cudaError_t e, const char* what);
#define GF_CUDA(call)                                   \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return gf::cuda_fail(_e, #call); \
  } while (0)

// ---------------------------------------------------------------- rules
// Barycentric coordinates and weights (sum 1) of the Dunavant rules.
bool rule_points(int npts, double bary[][3], double* w);

// ---------------------------------------------------------------- device views
// Geometry of one triangle set for one quadrature rule (structure of arrays).
struct GeoView {
  int nt, m;
  const float4* pts32;   // [m][nt]: offset of point a from the centroid, weight
  const float4* cen32;   // [nt]: centroid (FP32), area
  const float4* geo32;   // [nt][3]: delta_i = c - v_i (xyz), s_i * l_i
  const double* pts64;   // [m][nt][4]
  const double* cen64;   // [nt][4]
  const double* geo64;   // [nt][3][4]
  const double* v64;     // [nt][9] vertices
  const double* frame64; // [nt][kFrame] near-pair source frames
  const float* frame32;  // [nt][kFrame32]
  const int4* tvert;     // [nt]: vertex ids (x, y, z)
  const int4* tedge;     // [nt]: RWG edge id of local edge i, or -1
  const int64_t* near_ptr;  // [nt + 1]
  const int32_t* near_idx;  // sorted per row
  const int32_t* near_row;  // row (test triangle) of every near_idx entry
  float near_dist32;        // > 0: centroid criterion present (FP32 screen)
  const float* rad32;       // [nt]: largest |point - centroid| of the rule, rounded up
  const float4* bsph;       // [ceil(nt/32)]: bounding sphere of each block of 32 triangles (with points)
  // Block frames of the FP32 regular pairs: the centre of each block of 32
  // triangles on a grid of step bunit = 2^e (bgrid, in grid units; every
  // coordinate below 2^14 units), and offsets from it.
  const int4* bgrid;        // [ceil(nt/32)]
  const float4* rel32;      // [m][nt]: point a minus its block's centre (FP32 of the FP64 difference), weight
  const float4* geob32;     // [nt][3]: block centre minus v_i (the vertex opposite local edge i), s_i l_i
  float bunit, bunit2;      // 2^e, 2^(2e)
  // FP32 Green-table fills: list of the point pairs whose lattice cell holds
  // samples (fix_cap entries with the per-CTA counts first; mesh scratch)
  int2* fix = nullptr;
  int64_t fix_cap = 0;
};

// Entries to reserve for the flagged point pairs of an FP32 Green-table fill:
// the pair evaluations (nt^2 / 2 unordered pairs, m^2 point pairs each) times
// three times the share of lattice cells holding samples, plus a floor, at
// most kFixMaxBytes. A CTA whose share overflows scans its tasks again.
constexpr int64_t kFixMaxBytes = int64_t(1) << 30;
inline int64_t fix_entries(int64_t nt, int m, int64_t n_busy, int64_t n_lat) {
  const double evals = 0.5 * (double)nt * (double)nt * (double)m * (double)m;
  double f = n_lat > 0 ? 3.0 * (double)n_busy / (double)n_lat + 2e-4 : 1.0;
  if (f > 1.0) f = 1.0;
  const double want = evals * f + 65536.0, most = (double)(kFixMaxBytes / 8);
  return (int64_t)(want < most ? want : most);
}

// FP64 cell record: every x in the cell lies in interval j0 if x < split,
// else in j0 + 1 whose left sample is split; anchor = sample j0.
struct __align__(32) Cell64 {
  double split, anchor;
  int j0, pad;
};

// Coefficients of the interpolant on interval j (samples r, values f as
// (re, im) pairs) as a polynomial in u = x - x0:
// linear (Eq. 4) or the Lagrange form (Eq. 5) on the stencil s0..s0+deg,
// expanded by multiplying out prod_{m != i} (u - (r_m - x0)) / (r_i - r_m).
__host__ __device__ inline void interval_poly(int deg, int n, const double* __restrict__ r,
                                              const double* __restrict__ f, int j, double x0, double cre[4],
                                              double cim[4]) {
  for (int p = 0; p < 4; ++p) cre[p] = cim[p] = 0.0;
  if (deg <= 1) {
    double h = r[j + 1] - r[j];
    double sre = (f[2 * j + 2] - f[2 * j]) / h, sim = (f[2 * j + 3] - f[2 * j + 1]) / h;
    double u0 = x0 - r[j];
    cre[0] = f[2 * j] + sre * u0;
    cim[0] = f[2 * j + 1] + sim * u0;
    cre[1] = sre;
    cim[1] = sim;
    return;
  }
  int s0 = j - (deg - 1) / 2;
  if (s0 > n - 1 - deg) s0 = n - 1 - deg;
  if (s0 < 0) s0 = 0;
  for (int i = s0; i <= s0 + deg; ++i) {
    double poly[4] = {1.0, 0.0, 0.0, 0.0};
    double den = 1.0;
    int len = 1;
    for (int mm = s0; mm <= s0 + deg; ++mm) {
      if (mm == i) continue;
      double e = r[mm] - x0;
      for (int p = len; p >= 1; --p) poly[p] = poly[p - 1] - e * poly[p];
      poly[0] = -e * poly[0];
      ++len;
      den *= (r[i] - r[mm]);
    }
    for (int p = 0; p < len; ++p) {
      double b = poly[p] / den;
      cre[p] += f[2 * i] * b;
      cim[p] += f[2 * i + 1] * b;
    }
  }
}

// One interpolation table as the kernels see it.
struct TabView {
  int n_nodes, n_hash;
  double r_lo, r_hi, dr, inv_dr;
  float r_lo32, inv_dr32;
  const int32_t* hash;     // [n_hash]
  const double* node64;    // [n_nodes]
  const double2* c64;      // [n_nodes-1][4]: (re, im) of c0..c3 about node64[j]
  const float* node32;     // [n_nodes]: FP32 anchors
  const float4* c32a;      // [n_nodes-1]: (c0re, c0im, c1re, c1im) about node32[j]
  const float4* c32b;      // [n_nodes-1]: (c2re, c2im, c3re, c3im)
  // FP32 lattice image. Cells of step h (the base spacing t of Eq. 2, or the
  // refined t / 2) from r_min, aligned with the samples r_min + i h: cell i
  // holds the x with rint(fma(x, lat_inv, lat_nc)) = i (lat_nc = -(r_min / h +
  // 1/2)), found without a conversion instruction (kLatMagic). Its left end is
  // L_i = fma(i, lat_h, lat_lo) and its anchor A_i = fma(i, lat_h, lat_amid):
  // the middle of the cell for the Green table, L_i for the Exp table. For
  // every cell, lat_a holds the polynomial (in s = x - A_i) of the interval
  // that contains the cell's middle: (c0, c1) in FP32 for both tables; the
  // Green table's c2 sits in lat_c as two halves scaled by 2^E (c2 =
  // half * lat_c2d, lat_c2d = 2^-E), and its c3 is left out (the cells where
  // |c3| (h/2)^3 could exceed 4e-8 of |f| are treated as cells holding
  // samples). So one lookup is a 16-byte record plus a 4-byte one (Green) or
  // one 16-byte record (Exp). A cell with no sample inside (farther than a
  // rounding margin from its ends) lies in that interval. A cell holding
  // samples (a forced zero, grading, r_max; for the Green table also the c3
  // and c2-range tests) is flagged by the lowest mantissa bit of c1im, and
  // its lat_c word is its place in the blob's busy list; the blob lists those
  // cells (ascending), a header per cell (first sub-cell, 1/w, count - 1),
  // sub-cells trunc((x - L_i) / w) = (compact interval j0, split, node32[j0],
  // 0) -- x lies in j0 if x < split, else in j0 + 1 whose anchor is split --
  // and the full FP32 interval records about node32 (a, b).
  int n_lat, n_busy, n_sub, n_cmp;
  float lat_inv, lat_nc, lat_h, lat_lo;
  float lat_amid = 0.f;    // anchor base (see above)
  float lat_c2d = 0.f;     // 2^-E: c2 = half value * lat_c2d (Green)
  const float4* lat_a;     // [n_lat]: (c0re, c0im, c1re, c1im) about A_i; busy flag in c1im
  const uint32_t* lat_c;   // [n_lat]: c2 as half2 scaled by 2^E (Green), or the busy ordinal
  const float4* lat_blob;  // [blob_vec4()]
  __host__ __device__ size_t blob_vec4() const { return ((size_t)n_busy + 3) / 4 + n_busy + n_sub + 2 * (size_t)n_cmp; }
  // bytes of the lattice planes in shared memory for a lookup of degree deg
  // (lat_c only for deg > 1, padded to 16 bytes), then the blob
  __host__ __device__ size_t smem32_plane_bytes(int deg) const {
    return (size_t)n_lat * 16 + (deg > 1 ? (((size_t)n_lat * 4 + 15) & ~(size_t)15) : 0);
  }
  __host__ __device__ size_t smem32_bytes(int deg) const { return smem32_plane_bytes(deg) + blob_vec4() * 16; }
  int n_cells64;  // FP64 image of the Eq. (6) hash: cells of width 0.99 dr, one sample at most each
  double lo64c, inv64c;
  const Cell64* cells64;
  // lookups at x = xscale * R: 1 for a table in R, k for a table in u = kR
  // (a frequency-sweep table, one for every k; r_lo, r_hi then bound u)
  float xscale32 = 1.f;
  double xscale64 = 1.0;
};

// Marker (a quiet-NaN bit pattern) of a lattice cell that holds samples.
constexpr int32_t kLatticeSubMark = 0x7FC00001;
// 1.5 * 2^23: for |u| < 2^22, u + kLatMagic rounds u to an integer held in
// the low mantissa bits (the lattice index without a conversion instruction).
constexpr float kLatMagic = 12582912.0f;

// Regular work units of a mesh of nt triangles: (p, 32 consecutive q) over the
// 32 x 32 triangle block pairs bp <= bq, 32 units per block pair; each
// unordered regular pair {p, q} is evaluated once, for Z[m][n] and Z[n][m].
__host__ __device__ inline int64_t regular_units(int nt) {
  const int64_t nb = (nt + 31) / 32;
  return 32 * (nb * (nb + 1) / 2);
}

// Per-fill constants of the FP32 regular-pair kernels.
struct RegK {
  float kpi, kpi_lo;  // k / pi and its FP32 residue
  float scale;        // k eta / (4 pi) (times k for tables in u = kR)
  float inv_k2;       // 1 / k^2
};

inline RegK reg_consts(double k, double scale) {
  RegK K;
  K.kpi = (float)(k / kPi);
  K.kpi_lo = (float)(k / kPi - (double)K.kpi);
  K.scale = (float)scale;
  K.inv_k2 = (float)(1.0 / (k * k));
  return K;
}

// One mesh of a batched fill (device-resident descriptor).
struct BatchItem {
  GeoView g;
  TabView green, exp;
  int use_table;
  RegK rk;                        // constants of the FP32 regular kernel
  double k, scale, inv_k2;        // k, k eta, 1/k^2 for the near kernel
  void* Z;
  int64_t ldz;
  int64_t reg_begin, nchunk;      // first global regular work unit, 32-wide triangle blocks
  int64_t near_begin, n_near;     // first global near pair, near pairs
  int64_t mir_begin;              // first global 32 x 32 tile pair of the mirror pass Z += Z^T
  int ne;                         // RWG unknowns (rows and columns of Z)
};

// ---------------------------------------------------------------- kernels (gf_fill.cu, gf_mfie.cu,
// gf_adjoint.cu, gf_sparse_kernels.cu, gf_batch_kernels.cu; shared device code in gf_device.cuh)
// Doubles per triangle of the near-pair source frames: unit normal [0..2],
// edge lengths [3..5], unit edge tangents [6..14], in-plane edge normals [15..23].
constexpr int kFrame = 28;    // FP64 source frame per triangle: n, len, t, m, 1/area, 1/len
constexpr int kFrame32 = 24;  // FP32 copy of len, t, m (the sampled integrals) and n
cudaError_t launch_prep_geometry(const double* v64, int nt, int m, const double* bary, const double* w,
                                 const int4* tedge, const double* edge_len, float4* pts32, float4* cen32,
                                 float4* geo32, double* pts64, double* cen64, double* geo64, float* rad32,
                                 double* frame64, float* frame32, cudaStream_t s);
// Device build of one table (arrays in its arena; view = its TabView, whose
// lattice fields the lattice stage reads).
struct TableBuild {
  int kind, deg, n, n_hash, n_cells64;
  double r_lo, dr, lo64c, inv64c;
  const double* node64;
  const int8_t* zflag;
  double* fval;
  double2* c64;
  float* node32;
  float4* c32a;
  float4* c32b;
  int32_t* hash;
  Cell64* cells64;
  TabView view;
  const int32_t* lat_j;  // interval of each lattice cell's middle, bit 31: the cell holds samples
  const int32_t* cmp;    // interval of each compact record of the blob
  float4* lat_a;
  uint32_t* lat_c;
};
// Values, Eq. (6) hash, FP64 cells, coefficients and lattice images of two
// tables in three launches on s.
cudaError_t launch_tables(const TableBuild& a, const TableBuild& b, double k, cudaStream_t s);
// Block spheres, block centres on the grid of step g.bunit, and the offsets
// from them (rel32, geob32) of the current rule's geometry.
cudaError_t launch_near_rows(const int64_t* near_ptr, int64_t nt, int32_t* near_row, cudaStream_t s);
cudaError_t launch_block_frames(const GeoView& g, float4* bsph, int4* bgrid, float4* rel32, float4* geob32,
                                cudaStream_t s);
cudaError_t launch_table_eval(const TabView& t, int kind, int precision, const void* r, int64_t n,
                              void* out, cudaStream_t s);
// bpb: scratch of nb (nb + 1) / 2 float2 (nb = ceil(nt / 32)) for the FP32 screen.
cudaError_t launch_fill_mfie(const GeoView& g, const TabView* green, const TabView* texp, double green_scale,
                             int precision, bool mixed, double k, int nphi, int nl, const double* gl_phi,
                             const double* gl_l, void* Z, int64_t ldz, cudaStream_t s);
// Near-field sparse fill (FP32): tasks = SparseTask records {int p, int n, int64 off}
// (sparse_task_bytes() each), widx the work list of source triangles, the CSR
// pattern (row_ptr [ne + 1], cols) and its complex64 values.
cudaError_t launch_fill_sparse(const GeoView& g, const TabView* green, const TabView* texp, double green_scale,
                               bool mixed, double k,
                               double eta, int nphi, int nl, const double* gl_phi, const double* gl_l,
                               const void* tasks, int64_t ntask, const int32_t* widx, const int64_t* row_ptr,
                               const int32_t* cols, void* vals, cudaStream_t s);
int sparse_task_bytes();
cudaError_t launch_range_out(const unsigned long long* d_minmax, unsigned long long* h_range, cudaStream_t s);
cudaError_t launch_range(const GeoView& g, int precision, unsigned long long* d_minmax, float2* bpb, int32_t* list,
                         cudaStream_t s);
// table: the Green table view, or with from_exp the Exp table view (e^{-jkR}
// from the linear table times 1/R); NULL = direct evaluation.
cudaError_t launch_fill_regular(const GeoView& g, const TabView* table, bool from_exp, double green_scale,
                                int precision, double k,
                                double eta, void* Z, int64_t ldz, cudaStream_t s);
// Z <- Z + Z^T on the ne x ne FP32 block (the second half of the FP32
// regular part, whose pair kernel writes the test triangle's rows only).
cudaError_t launch_mirror32(void* Z, int64_t ldz, int64_t ne, cudaStream_t s);
cudaError_t launch_fill_near(const GeoView& g, const TabView* texp, int precision, bool mixed, double k,
                             double eta, int nphi, int nl, const double* gl_phi, const double* gl_l,
                             void* Z, int64_t ldz, cudaStream_t s);

cudaError_t launch_batch_regular(const BatchItem* items, int nitems, int64_t total, unsigned long long* counter, int m,
                                 bool table, int block, int grid, int chunk, cudaStream_t s);
// Z <- Z + Z^T of every mesh in one launch (total = all meshes' 32 x 32 tile
// pairs I <= J).
cudaError_t launch_batch_mirror(const BatchItem* items, int nitems, int64_t total, int grid, cudaStream_t s);
// The batched regular kernel with the largest L1 (no shared memory carve-out)
// or the default split.
cudaError_t set_batch_regular_l1(int m, bool table, bool max_l1);
cudaError_t launch_batch_near(const BatchItem* items, int nitems, int64_t total, unsigned long long* counter,
                              bool mixed, int nphi, int nl, const double* gl_phi, const double* gl_l, int grid,
                              cudaStream_t s);
int batch_regular_blocks_per_sm(int m, bool table, int block);
cudaError_t launch_adjoint(const GeoView& g, const TabView* green, const TabView* texp, bool mixed, double k, double eta,
                           const double* bary, int nphi, int nl, const double* gl_phi, const double* gl_l,
                           const void* gZ, int64_t ldg, double* dtri, double* dk, double* dxyz, int64_t nv,
                           cudaStream_t s);
void gauss_legendre_host(int n, double* x, double* w);
// host helpers shared by the single and batched fills (gf_host.cpp)
gf_status prepare_rule(gf_mesh* m, int rule, cudaStream_t s);
GeoView geo_view(const gf_mesh* m);

}  // namespace gf

// ---------------------------------------------------------------- handles
struct gf_mesh {
  int device;
  int64_t nv, nt, ne;
  double near_dist;
  std::vector<double> xyz;        // [nv][3]
  std::vector<int32_t> tri;       // [nt][3]
  std::vector<int32_t> ev, et;    // [ne][2]
  std::vector<int32_t> tedge;     // [nt][3], -1 if boundary
  std::vector<double> elen;       // [ne]
  std::vector<int32_t> perm;      // internal triangle i = original triangle perm[i] (Morton order)
  std::vector<int32_t> inv_perm;  // original -> internal
  std::vector<int64_t> near_ptr;  // [nt + 1], internal ids
  std::vector<int32_t> near_idx;
  // device: one allocation (d_arena) holds every array but the adjoint scratch
  void* d_arena = nullptr;
  size_t arena_bytes = 0;
  double* d_v64 = nullptr;
  int4* d_tvert = nullptr;
  int4* d_tedge = nullptr;
  double* d_elen = nullptr;
  int64_t* d_near_ptr = nullptr;
  int32_t* d_near_idx = nullptr;
  int32_t* d_near_row = nullptr;
  // per-rule geometry cache
  int rule = 0;
  float4* d_pts32 = nullptr;
  float4* d_cen32 = nullptr;
  float4* d_geo32 = nullptr;
  double* d_pts64 = nullptr;
  double* d_cen64 = nullptr;
  double* d_geo64 = nullptr;
  double* d_frame64 = nullptr;
  float* d_frame32 = nullptr;
  float* d_rad32 = nullptr;
  float4* d_bsph = nullptr;
  int4* d_bgrid = nullptr;
  float4* d_rel32 = nullptr;
  float4* d_geob32 = nullptr;
  int bgrid_e = 0;                          // block-centre grid step 2^bgrid_e
  double* d_dtri = nullptr;                 // adjoint scratch [nt][9]
  double* d_dk = nullptr;                   // adjoint scratch [1]
  unsigned long long* d_minmax = nullptr;  // range scratch [8]
  unsigned long long* h_range = nullptr;   // page-locked, device-mapped: r_min, r_max of the last gf_range
  float2* d_range_bpb = nullptr;          // range scratch: bounds per 32 x 32 block pair
  int32_t* d_range_list = nullptr;        // range scratch: block pairs that can hold an extreme, count last
  int2* d_fix = nullptr;                   // FP32 Green-table fill scratch: flagged point pairs (grown on demand)
  int64_t fix_cap = 0;
  size_t fix_bytes = 0;                    // its block of the device pool
};

struct gf_table {
  int device;
  double k, r_lo, r_hi;
  bool kr = false;  // built in u = kR (k = 1): serves every k (frequency sweeps)
  void* d_arena = nullptr;  // one device allocation holding every array of both tables
  size_t arena_bytes = 0;
  struct One {
    int kind, degree;
    std::vector<double> r;        // host sample positions
    std::vector<int8_t> zflag;    // 1: real part is an exact zero, 2: imaginary part
    double dr;
    int64_t n_hash;
    double* d_node64 = nullptr;   // device arrays: views into the table's arena
    int8_t* d_zflag = nullptr;
    double* d_fval = nullptr;     // [n][2] sample values
    double2* d_c64 = nullptr;
    float* d_node32 = nullptr;
    float4* d_c32a = nullptr;
    float4* d_c32b = nullptr;
    int32_t* d_hash = nullptr;
    int n_lat = 0, n_busy = 0, n_sub = 0, n_cmp = 0;
    float lat_inv = 0.f, lat_nc = 0.f, lat_h = 0.f, lat_lo = 0.f, lat_amid = 0.f, lat_c2d = 0.f;
    int32_t* d_lat_j = nullptr;
    float4* d_lat_a = nullptr;
    uint32_t* d_lat_c = nullptr;
    int32_t* d_lat_cmp = nullptr;
    float4* d_lat_blob = nullptr;
    int n_cells64 = 0;
    double lo64c = 0, inv64c = 0;
    gf::Cell64* d_cells64 = nullptr;
    gf::TabView view() const;
  } green, exp;
  const One& get(int kind) const { return kind == GF_GREEN ? green : exp; }
};
namespace gf {
// Views of `t` for a fill at wavenumber k. A table in u = kR is read at
// x = kR, and e^{-jkR}/R = k e^{-ju}/u: its Green values carry the factor
// *green_scale = k (1 for a table built for this k). False if t is an
// R-table for another k.
inline bool table_views(const gf_table* t, double k, TabView* green, TabView* exp, double* green_scale) {
  if (!t->kr && t->k != k) return false;
  *green = t->green.view();
  *exp = t->exp.view();
  const double x = t->kr ? k : 1.0;
  green->xscale32 = exp->xscale32 = (float)x;
  green->xscale64 = exp->xscale64 = x;
  *green_scale = x;
  return true;
}
}  // namespace gf

