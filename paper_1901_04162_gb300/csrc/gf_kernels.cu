// gfmom kernels for sm_103a.
//
// Regular pairs (Section II.A): one warp per (test triangle p, 32 source
// triangles q), one source triangle per lane. For each test point a the lane
// runs over the source points b: R = |(c_p - c_q) + alpha_a - beta_b|, Green
// value from the Lagrange table (hash of Eq. 6 -> interval -> cubic in
// s = R - r_j, Eq. 3 + 5 re-expanded as monomials) or from sincospi, and four
// moments M0 = sum w w G, Ma = sum w w alpha G, Mb = sum w w beta G,
// Mab = sum w w (alpha . beta) G (8 complex numbers; Kahan-compensated over a
// in FP32). The 3 x 3 RWG block of the pair follows from the moments:
//   Z(e_i, e_j) += jk eta/(4 pi) s_i l_i s_j l_j
//                  [ (Mab + eps_j . Ma + delta_i . Mb + (delta_i . eps_j) M0) / 4 - M0 / k^2 ]
// with delta_i = c_p - v_i, eps_j = c_q - v_j (v = vertex opposite the edge).
// The table sits in shared memory when it fits.
//
// Near pairs: FP64, one thread per (p, q) near pair; the inner integrals over
// q for each test point come from singularity cancellation (exact radial
// integral) with the angular variable u = asinh(tan phi) for the scalar part,
// and from the surface-gradient theorem (line integrals over q's edges, static
// part in closed form) for the vector part. e^{-jkR} on those lines is the
// linear Exp table when r_min <= R <= r_max (Section II.C), else sincos.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <type_traits>

#include "gf_internal.h"

namespace gf {
namespace {

constexpr int kWarps = 8;              // warps per block of the pair kernels
constexpr int kThreads = kWarps * 32;

__device__ __forceinline__ int edge_of(int code) { return code >> 1; }
__device__ __forceinline__ bool edge_valid(int code) { return code >= 0; }

// ---------------------------------------------------------------- geometry prep
__global__ void k_prep_geometry(const double* __restrict__ v64, int nt, int m, const double* __restrict__ bary,
                                const double* __restrict__ w, const int4* __restrict__ tedge,
                                const double* __restrict__ elen, float4* pts32, float4* cen32, float4* geo32,
                                double* pts64, double* cen64, double* geo64, float* rad32, double* frame64,
                                float* frame32) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double v[3][3];
  for (int c = 0; c < 3; ++c)
    for (int x = 0; x < 3; ++x) v[c][x] = v64[9 * (size_t)t + 3 * c + x];
  {
    // source-triangle frame of the near-pair integrals: unit normal, edge
    // lengths, unit edge tangents (v_e -> v_{e+1}), in-plane edge normals t x n
    // and 1/area; an FP32 copy of the lengths, tangents and normals
    double* fr = frame64 + kFrame * (size_t)t;
    float* f32 = frame32 + kFrame32 * (size_t)t;
    const double e1[3] = {v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2]};
    const double e2[3] = {v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double inv = 1.0 / sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int x = 0; x < 3; ++x) fr[x] = n[x] = n[x] * inv;
    fr[24] = 2.0 * inv;  // 1 / area
    for (int e = 0; e < 3; ++e) {
      const double* a = v[e];
      const double* b = v[(e + 1) % 3];
      double tt[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
      const double len = sqrt(tt[0] * tt[0] + tt[1] * tt[1] + tt[2] * tt[2]);
      const double il = 1.0 / len;
      for (int x = 0; x < 3; ++x) tt[x] *= il;
      fr[3 + e] = len;
      for (int x = 0; x < 3; ++x) fr[6 + 3 * e + x] = tt[x];
      fr[15 + 3 * e + 0] = tt[1] * n[2] - tt[2] * n[1];
      fr[15 + 3 * e + 1] = tt[2] * n[0] - tt[0] * n[2];
      fr[15 + 3 * e + 2] = tt[0] * n[1] - tt[1] * n[0];
    }
    for (int i = 0; i < 21; ++i) f32[i] = (float)fr[3 + i];
    for (int i = 0; i < 3; ++i) f32[21 + i] = (float)n[i];  // unit normal (MFIE)
  }
  double c0 = (v[0][0] + v[1][0] + v[2][0]) / 3.0;
  double c1 = (v[0][1] + v[1][1] + v[2][1]) / 3.0;
  double c2 = (v[0][2] + v[1][2] + v[2][2]) / 3.0;
  double e1x = v[1][0] - v[0][0], e1y = v[1][1] - v[0][1], e1z = v[1][2] - v[0][2];
  double e2x = v[2][0] - v[0][0], e2y = v[2][1] - v[0][1], e2z = v[2][2] - v[0][2];
  double nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
  double area = 0.5 * sqrt(nx * nx + ny * ny + nz * nz);
  cen64[4 * (size_t)t + 0] = c0;
  cen64[4 * (size_t)t + 1] = c1;
  cen64[4 * (size_t)t + 2] = c2;
  cen64[4 * (size_t)t + 3] = area;
  cen32[t] = make_float4((float)c0, (float)c1, (float)c2, (float)area);
  double rad = 0.0;
  for (int a = 0; a < m; ++a) {
    double px = bary[3 * a] * v[0][0] + bary[3 * a + 1] * v[1][0] + bary[3 * a + 2] * v[2][0];
    double py = bary[3 * a] * v[0][1] + bary[3 * a + 1] * v[1][1] + bary[3 * a + 2] * v[2][1];
    double pz = bary[3 * a] * v[0][2] + bary[3 * a + 1] * v[1][2] + bary[3 * a + 2] * v[2][2];
    size_t o = (size_t)a * nt + t;
    pts64[4 * o + 0] = px - c0;
    pts64[4 * o + 1] = py - c1;
    pts64[4 * o + 2] = pz - c2;
    pts64[4 * o + 3] = w[a];
    pts32[o] = make_float4((float)(px - c0), (float)(py - c1), (float)(pz - c2), (float)w[a]);
    rad = fmax(rad, sqrt((px - c0) * (px - c0) + (py - c1) * (py - c1) + (pz - c2) * (pz - c2)));
  }
  rad32[t] = (float)(rad * (1.0 + 1e-6));
  int codes[3] = {tedge[t].x, tedge[t].y, tedge[t].z};
  for (int i = 0; i < 3; ++i) {
    double sl = 0.0;
    if (codes[i] >= 0) sl = (codes[i] & 1 ? -1.0 : 1.0) * elen[codes[i] >> 1];
    double dx = c0 - v[i][0], dy = c1 - v[i][1], dz = c2 - v[i][2];
    size_t o = 3 * (size_t)t + i;
    geo64[4 * o + 0] = dx;
    geo64[4 * o + 1] = dy;
    geo64[4 * o + 2] = dz;
    geo64[4 * o + 3] = sl;
    geo32[o] = make_float4((float)dx, (float)dy, (float)dz, (float)sl);
  }
}

// ---------------------------------------------------------------- table image
__device__ void dev_table_values(int j, int kind, double k, const double* __restrict__ r,
                                 const int8_t* __restrict__ zflag, double* fval) {
  double s, c;
  sincos(k * r[j], &s, &c);
  double re = c, im = -s;
  if (kind == GF_GREEN) {
    re = c / r[j];
    im = -s / r[j];
  }
  if (zflag[j] == 1) re = 0.0;
  if (zflag[j] == 2) im = 0.0;
  fval[2 * j] = re;
  fval[2 * j + 1] = im;
}

// Coefficients of the interpolant on interval j as a polynomial in u = x - x0:
// linear (Eq. 4) or the Lagrange form (Eq. 5) on the stencil s0..s0+deg,
// expanded by multiplying out prod_{m != i} (u - (r_m - x0)) / (r_i - r_m).
__device__ void interval_poly(int deg, int n, const double* __restrict__ r, const double* __restrict__ f, int j,
                              double x0, double cre[4], double cim[4]) {
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

__device__ void dev_table_coef(int j, int deg, int n, const double* __restrict__ r, const double* __restrict__ f,
                               double2* c64, float* node32, float4* c32a, float4* c32b) {
  float a32 = (float)r[j];
  node32[j] = a32;
  if (j >= n - 1) return;
  double cre[4], cim[4];
  interval_poly(deg, n, r, f, j, r[j], cre, cim);
  for (int p = 0; p < 4; ++p) c64[4 * j + p] = make_double2(cre[p], cim[p]);
  // FP32 image: the same polynomial about the FP32-representable anchor, so
  // that s = R - node32[j] carries no anchor rounding error
  interval_poly(deg, n, r, f, j, (double)a32, cre, cim);
  c32a[j] = make_float4((float)cre[0], (float)cim[0], (float)cre[1], (float)cim[1]);
  c32b[j] = make_float4((float)cre[2], (float)cim[2], (float)cre[3], (float)cim[3]);
}

// Hash of Eq. (6): cell c holds the largest sample index whose cell
// floor((r_j - r_min)/dr) is <= c (the forward-filled array); cell 0 holds 0.
__device__ void dev_table_hash(int c, int n, const double* __restrict__ r, double r_lo, double dr, int32_t* hash) {
  if (c == 0) {
    hash[0] = 0;
    return;
  }
  int lo = 0, hi = n - 1;  // invariant: cell(lo) <= c
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (floor((r[mid] - r_lo) / dr) <= (double)c) lo = mid;
    else hi = mid - 1;
  }
  hash[c] = lo;
}

// ---------------------------------------------------------------- lookups
struct Tab32 {  // FP32 view (shared or global memory; possibly a window of the lattice)
  const float4* la;   // lattice records, indexed by the global cell number
  const float4* lb;
  const int* busy;    // the blob: cells holding samples (ascending), their headers,
  const float4* hdr;  // sub-cells and compact interval records
  const float4* sub;
  const float4* ca;
  const float4* cb;
  int n_busy;
  float vmin, vmax;   // kLatMagic + first / last cell present (the whole lattice, or a window)
  float inv, nc, h, lo;
  float xscale;       // lookups at x = xscale * R (1, or k for a table in u = kR)
};

// Points a view's blob pointers into a copy of the blob (global or shared).
__device__ __forceinline__ void tab32_blob(Tab32& T, const TabView& t, const float4* blob) {
  T.busy = reinterpret_cast<const int*>(blob);
  T.hdr = blob + (t.n_busy + 3) / 4;
  T.sub = T.hdr + t.n_busy;
  T.ca = T.sub + t.n_sub;
  T.cb = T.ca + t.n_cmp;
  T.n_busy = t.n_busy;
}

__device__ __forceinline__ Tab32 tab32(const TabView& t) {
  Tab32 T;
  T.xscale = t.xscale32;
  T.la = t.lat_a;
  T.lb = t.lat_b;
  tab32_blob(T, t, t.lat_blob);
  T.vmin = kLatMagic;
  T.vmax = kLatMagic + (float)(t.n_lat - 1);
  T.inv = t.lat_inv;
  T.nc = t.lat_nc;
  T.h = t.lat_h;
  T.lo = t.lat_lo;
  return T;
}

// Lattice cell of R (without a conversion instruction) and the exact offset
// s = R - A_i from its anchor; the table builder repeats these float
// operations.
struct LatPos {
  int i;
  float s;
};

__device__ __forceinline__ LatPos lat_pos(const Tab32& T, float R) {
  const float u = __fmaf_rn(R, T.inv, T.nc);
  const float v = fminf(fmaxf(__fadd_rn(u, kLatMagic), T.vmin), T.vmax);
  const float fi = __fsub_rn(v, kLatMagic);
  return LatPos{__float_as_int(v) - __float_as_int(kLatMagic), __fsub_rn(R, __fmaf_rn(fi, T.h, T.lo))};
}

// e^{-jkR}/R (Green) or e^{-jkR} (Exp) from the FP32 lattice image: the
// lattice cell of R (the Eq. 6 hash on the uniform samples) gives the
// polynomial directly; a cell that holds samples adds one sub-cell record
// (exact bracketing) and the interval's own record.
template <int DEG>
__device__ __forceinline__ float2 horner32(float s, float4 a, float4 b) {
  if (DEG == 1) return make_float2(fmaf(s, a.z, a.x), fmaf(s, a.w, a.y));
  float re = fmaf(s, b.z, b.x), im = fmaf(s, b.w, b.y);
  re = fmaf(s, re, a.z);
  im = fmaf(s, im, a.w);
  re = fmaf(s, re, a.x);
  im = fmaf(s, im, a.y);
  return make_float2(re, im);
}

// Branch-free part: the cell's record (the polynomial of the interval at the
// cell's middle); *slow is set when the cell holds samples, where this value
// is exact only on the middle interval.
template <int DEG>
__device__ __forceinline__ float2 lookup32_fast(const Tab32& T, float R, bool* slow) {
  const LatPos q = lat_pos(T, R * T.xscale);
  const float4 a = T.la[q.i];
  float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
  if (DEG > 1) b = T.lb[q.i];
  *slow = (__float_as_int(DEG > 1 ? b.w : a.w) & 1) != 0;
  return horner32<DEG>(q.s, a, b);
}

// Cells holding samples: the cell's place in the busy list (kept in the low
// bits of c3re for the Green table, in lat_b.x for the Exp table; a binary
// search for lists longer than kOrdinalMax), its header, the sub-cell, then
// the compact interval record about node32.
constexpr int kOrdinalMax = 0xFFF;

template <int DEG>
__device__ __forceinline__ float2 lookup32_slow(const Tab32& T, float Rr) {
  const float R = Rr * T.xscale;  // table units
  const LatPos q = lat_pos(T, R);
  int lo = DEG > 1 ? (__float_as_int(T.lb[q.i].z) & kOrdinalMax) : __float_as_int(T.lb[q.i].x);
  if (lo >= kOrdinalMax) {
    lo = 0;
    int hi = T.n_busy - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (T.busy[mid] < q.i) lo = mid + 1;
      else hi = mid;
    }
  }
  const float4 h = T.hdr[lo];
  const int c = __float_as_int(h.x) + min(max(__float2int_rz(__fmul_rn(q.s, h.y)), 0), __float_as_int(h.z));
  const float4 rec = T.sub[c];
  const bool up = R >= rec.y;
  const int j = __float_as_int(rec.x) + (up ? 1 : 0);
  const float4 a = T.ca[j];
  float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
  if (DEG > 1) b = T.cb[j];
  return horner32<DEG>(R - (up ? rec.y : rec.z), a, b);
}

template <int DEG>
__device__ __forceinline__ float2 lookup32(const Tab32& T, float R) {
  bool slow;
  const float2 f = lookup32_fast<DEG>(T, R, &slow);
  return slow ? lookup32_slow<DEG>(T, R) : f;
}

// FP64 lookup through the FP64 cell image (same construction as the FP32
// one, in FP64): exact bracketing against the FP64 samples, then the FP64
// polynomial about the interval's left sample.
__device__ __forceinline__ int cell64_of(double x, double lo, double inv) {
  return __double2int_rz(__dmul_rn(__dsub_rn(x, lo), inv));
}

template <int DEG>
__device__ __forceinline__ double2 lookup64(const TabView& T, double Rr) {
  const double R = Rr * T.xscale64;  // table units
  const int c = min(max(cell64_of(R, T.lo64c, T.inv64c), 0), T.n_cells64 - 1);
  const Cell64 rec = T.cells64[c];
  const bool up = R >= rec.split;
  const int j = rec.j0 + (up ? 1 : 0);
  const double s = R - (up ? rec.split : rec.anchor);
  const double2* cf = T.c64 + 4 * j;
  const double2 c0 = cf[0], c1 = cf[1];
  if (DEG == 1) return make_double2(fma(s, c1.x, c0.x), fma(s, c1.y, c0.y));
  const double2 c2 = cf[2], c3 = cf[3];
  double re = fma(s, c3.x, c2.x), im = fma(s, c3.y, c2.y);
  re = fma(s, re, c1.x);
  im = fma(s, im, c1.y);
  re = fma(s, re, c0.x);
  im = fma(s, im, c0.y);
  return make_double2(re, im);
}

__device__ void dev_table_cells64(int c, int n, const double* __restrict__ node64, double lo, double inv,
                                  Cell64* cells) {
  auto first_at_or_after = [&](int cc) {
    int a = 1, b = n - 1;
    while (a < b) {
      const int mid = (a + b) >> 1;
      if (cell64_of(node64[mid], lo, inv) >= cc) b = mid;
      else a = mid + 1;
    }
    return a;
  };
  const int a = first_at_or_after(c);  // cells hold one interior sample at most (checked on the host)
  Cell64 rec;
  rec.j0 = a - 1;
  rec.split = (a < n - 1 && cell64_of(node64[a], lo, inv) == c) ? node64[a] : INFINITY;
  rec.anchor = node64[a - 1];
  rec.pad = 0;
  cells[c] = rec;
}

// Lattice records: the polynomial of the interval at the cell's middle about
// the cell anchor A_i = fma(i, h, lo) (the anchor the lookups recompute),
// with the flag bit of the cells holding samples.
__device__ void dev_table_lattice(int i, const TabView& v, int deg, const double* __restrict__ r,
                                  const double* __restrict__ f, const int32_t* __restrict__ lat_j,
                                  const int32_t* __restrict__ cmp, bool flag_in_b, float4* la, float4* lb) {
  if (i < v.n_cmp) {  // compact interval records of the blob
    float4* ca = const_cast<float4*>(v.lat_blob) + (v.n_busy + 3) / 4 + v.n_busy + v.n_sub;
    ca[i] = v.c32a[cmp[i]];
    ca[v.n_cmp + i] = v.c32b[cmp[i]];
  }
  if (i >= v.n_lat) return;
  const float A = __fmaf_rn((float)i, v.lat_h, v.lat_lo);
  const int jb = lat_j[i];
  double cre[4], cim[4];
  interval_poly(deg, v.n_nodes, r, f, jb & 0x7fffffff, (double)A, cre, cim);
  float4 a = make_float4((float)cre[0], (float)cim[0], (float)cre[1], (float)cim[1]);
  float4 b = make_float4((float)cre[2], (float)cim[2], (float)cre[3], (float)cim[3]);
  // flag bit: the lowest mantissa bit of the last word (changes it by one ulp at most)
  const int busy = (int)(((unsigned)jb) >> 31);
  float& w = flag_in_b ? b.w : a.w;
  w = __int_as_float((__float_as_int(w) & ~1) | busy);
  if (busy) {  // the cell's place in the busy list, for the exact path
    const int* list = reinterpret_cast<const int*>(v.lat_blob);
    int lo = 0, hi = v.n_busy - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (list[mid] < i) lo = mid + 1;
      else hi = mid;
    }
    const int ord = min(lo, kOrdinalMax);
    if (flag_in_b)  // low 12 bits of c3re: a relative change below 2^-11 of the smallest term
      b.z = __int_as_float((__float_as_int(b.z) & ~kOrdinalMax) | ord);
    else  // lat_b is not part of a linear lookup
      b.x = __int_as_float(ord);
  }
  la[i] = a;
  lb[i] = b;
}

// The table builds of both tables (Green and Exp) in three launches: sample
// values, hash and FP64 cells; interval coefficients; lattice records.
__global__ void k_tables_values(TableBuild a, TableBuild b, double k) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const TableBuild* t[2] = {&a, &b};
  for (int w = 0; w < 2; ++w) {
    const TableBuild& T = *t[w];
    if (i < T.n) return dev_table_values(i, T.kind, k, T.node64, T.zflag, T.fval);
    i -= T.n;
    if (i < T.n_hash) return dev_table_hash(i, T.n, T.node64, T.r_lo, T.dr, T.hash);
    i -= T.n_hash;
    if (i < T.n_cells64) return dev_table_cells64(i, T.n, T.node64, T.lo64c, T.inv64c, T.cells64);
    i -= T.n_cells64;
  }
}

__global__ void k_tables_coef(TableBuild a, TableBuild b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const TableBuild* t[2] = {&a, &b};
  for (int w = 0; w < 2; ++w) {
    const TableBuild& T = *t[w];
    if (i < T.n) return dev_table_coef(i, T.deg, T.n, T.node64, T.fval, T.c64, T.node32, T.c32a, T.c32b);
    i -= T.n;
  }
}

__global__ void k_tables_lattice(TableBuild a, TableBuild b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const TableBuild* t[2] = {&a, &b};
  for (int w = 0; w < 2; ++w) {
    const TableBuild& T = *t[w];
    const int n = max(T.view.n_lat, T.view.n_cmp);
    if (i < n)
      return dev_table_lattice(i, T.view, T.deg, T.node64, T.fval, T.lat_j, T.cmp, T.flag_in_b, T.lat_a, T.lat_b);
    i -= n;
  }
}

template <int DEG>
__global__ void k_table_eval32(TabView t, const float* __restrict__ r, int64_t n, float2* out) {
  const Tab32 T = tab32(t);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = lookup32<DEG>(T, r[i]);
}

template <int DEG>
__global__ void k_table_eval64(TabView t, const double* __restrict__ r, int64_t n, double2* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = lookup64<DEG>(t, r[i]);
}

// ---------------------------------------------------------------- near test
// A pair is near when it shares a vertex, or (centroid criterion) when q is in
// p's sorted near list; the FP32 centroid distance only screens out pairs that
// are clearly farther than near_dist.
__device__ __forceinline__ bool pair_is_near(const GeoView& g, int p, int q, int4 vp, int4 vq, float3 dc) {
  if (vp.x == vq.x || vp.x == vq.y || vp.x == vq.z || vp.y == vq.x || vp.y == vq.y || vp.y == vq.z ||
      vp.z == vq.x || vp.z == vq.y || vp.z == vq.z)
    return true;
  if (g.near_dist32 > 0.f) {
    float th = g.near_dist32 * 1.0001f + 1e-6f;
    if (dc.x * dc.x + dc.y * dc.y + dc.z * dc.z < th * th) {
      int64_t lo = g.near_ptr[p], hi = g.near_ptr[p + 1];
      while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        int v = g.near_idx[mid];
        if (v == q) return true;
        if (v < q) lo = mid + 1;
        else hi = mid;
      }
    }
  }
  return false;
}

// Regular pairs are enumerated once per unordered pair {p, q}, p < q: the
// Galerkin block of (q, p) is the transpose of that of (p, q) (the moments
// swap alpha and beta, the bracket is unchanged), so one evaluation serves
// Z[m][n] and Z[n][m]. Work unit = (p, 32 consecutive q) inside a 32 x 32 block
// pair (bp <= bq); block pairs run column by column, u = bq (bq + 1) / 2 + bp,
// 32 units (one per p of block bp) each; regular_units(nt) counts them.

__device__ __forceinline__ bool sym_task(int64_t task, int nt, int* p, int* q0) {
  const int64_t u = task >> 5;
  int64_t bq = (int64_t)((sqrtf(8.f * (float)u + 1.f) - 1.f) * 0.5f);
  while (bq > 0 && bq * (bq + 1) / 2 > u) --bq;
  while ((bq + 1) * (bq + 2) / 2 <= u) ++bq;
  const int64_t bp = u - bq * (bq + 1) / 2;
  *p = (int)(bp * 32 + (task & 31));
  *q0 = (int)(bq * 32);
  return *p < nt;
}

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

// Range scratch: mm[0] r_min, mm[1] r_max (FP64 bits), mm[2] / mm[3] the
// pass-1 thresholds, mm[4] candidate block pairs, mm[5] blocks of pass 2 done.
__global__ void k_range_init(unsigned long long* mm, float2* bpb, int64_t nbp) {
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i0 == 0) {
    mm[0] = dbits(INFINITY);
    mm[1] = 0ull;
    mm[2] = dbits(INFINITY);
    mm[3] = 0ull;
    mm[4] = 0ull;
    mm[5] = 0ull;
  }
  for (int64_t i = i0; i < nbp; i += (int64_t)gridDim.x * blockDim.x) bpb[i] = make_float2(INFINITY, 0.f);
}

// Every point distance of a pair lies in [D - r_p - r_q, D + r_p + r_q]
// (D = centroid distance, r = largest point offset from the centroid).
// Pass 1 finds thresholds mm[2] >= r_min and mm[3] <= r_max; pass 2
// (k_range32) evaluates the point pairs only of triangle pairs whose interval
// reaches below mm[2] or above mm[3]. FP32 bounds are widened by a slack that
// covers their rounding.
__device__ __forceinline__ void pair_bounds(const GeoView& g, int p, int q, float3 dc, float4 cp, float4 cq,
                                            float* lb, float* ub) {
  const float D = sqrtf(fmaf(dc.x, dc.x, fmaf(dc.y, dc.y, dc.z * dc.z)));
  const float r = g.rad32[p] + g.rad32[q];
  const float mag = fmaxf(fmaxf(fabsf(cp.x), fabsf(cp.y)), fmaxf(fabsf(cp.z), fmaxf(fmaxf(fabsf(cq.x), fabsf(cq.y)),
                                                                                      fabsf(cq.z))));
  const float slack = 1e-5f * (D + r + mag);
  *lb = fmaxf(D - r - slack, 0.f);
  *ub = D + r + slack;
}

constexpr int kRangeSplit = 4;          // pass-1 warps per 32 x 32 block pair (8 test triangles each)

// Pass 1, one warp per 8 test triangles of a 32 x 32 block pair: thresholds
// from actual point distances (the first rule point of each triangle of every
// regular pair: their minimum is >= r_min, their maximum <= r_max), widened by
// a relative 1e-5 for the FP32 rounding (mm[2], mm[3]), and, per block pair,
// the smallest lower and largest upper bound of its regular pairs (bpb, merged
// by integer atomics on the bits of these non-negative floats), so that pass 2
// skips block pairs that cannot hold an extreme.
__global__ void __launch_bounds__(kThreads) k_range_bounds(GeoView g, unsigned long long* mm, float2* bpb) {
  const int lane = threadIdx.x & 31;
  const int64_t nb = (g.nt + 31) / 32, ntask = nb * (nb + 1) / 2 * kRangeSplit;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float min_d = INFINITY, max_d = 0.f;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntask; t += nwarp) {
    const int64_t u = t / kRangeSplit;
    int p0, q0;
    sym_task(u * 32, g.nt, &p0, &q0);
    p0 += (int)(t % kRangeSplit) * (32 / kRangeSplit);
    const int q = min(q0 + lane, g.nt - 1);
    const float4 cq = g.cen32[q], yq = g.pts32[q];
    const int4 vq = g.tvert[q];
    float blk_lb = INFINITY, blk_ub = 0.f;
    const int p1 = min(p0 + 32 / kRangeSplit, g.nt);
#pragma unroll 2
    for (int p = p0; p < p1; ++p) {
      const float4 cp = g.cen32[p];
      const float3 dc = make_float3(cp.x - cq.x, cp.y - cq.y, cp.z - cq.z);
      if (!((q0 + lane < g.nt) && q > p && !pair_is_near(g, p, q, g.tvert[p], vq, dc))) continue;
      float lb, ub;
      pair_bounds(g, p, q, dc, cp, cq, &lb, &ub);
      const float4 xp = g.pts32[p];
      const float rx = (dc.x + xp.x) - yq.x, ry = (dc.y + xp.y) - yq.y, rz = (dc.z + xp.z) - yq.z;
      const float d = sqrtf(fmaf(rx, rx, fmaf(ry, ry, rz * rz)));
      min_d = fminf(min_d, d);
      max_d = fmaxf(max_d, d);
      blk_lb = fminf(blk_lb, lb);
      blk_ub = fmaxf(blk_ub, ub);
    }
    for (int off = 16; off > 0; off >>= 1) {
      blk_lb = fminf(blk_lb, __shfl_xor_sync(0xffffffffu, blk_lb, off));
      blk_ub = fmaxf(blk_ub, __shfl_xor_sync(0xffffffffu, blk_ub, off));
    }
    if (lane == 0 && blk_lb < INFINITY) {
      unsigned* b = reinterpret_cast<unsigned*>(bpb + u);
      atomicMin(b, __float_as_uint(blk_lb) & 0x7fffffffu);  // +0 for a -0 bound
      atomicMax(b + 1, __float_as_uint(blk_ub));
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    min_d = fminf(min_d, __shfl_xor_sync(0xffffffffu, min_d, off));
    max_d = fmaxf(max_d, __shfl_xor_sync(0xffffffffu, max_d, off));
  }
  if (lane == 0) {
    if (min_d < INFINITY) atomicMin(&mm[2], dbits((double)min_d * (1.0 + 1e-5)));
    if (max_d > 0.f) atomicMax(&mm[3], dbits((double)max_d * (1.0 - 1e-5)));
  }
}

// The block pairs that can hold an extreme, appended to list (in any order:
// the result of pass 2 does not depend on it); their count into mm[4].
__global__ void k_range_list(unsigned long long* mm, const float2* bpb, int64_t nbp, int32_t* list) {
  const float u_min = (float)__longlong_as_double((long long)mm[2]);
  const float l_max = (float)__longlong_as_double((long long)mm[3]);
  const int lane = threadIdx.x & 31;
  for (int64_t u0 = (int64_t)blockIdx.x * blockDim.x; u0 < nbp; u0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = u0 + threadIdx.x;
    bool cand = false;
    if (u < nbp) {
      const float2 bb = bpb[u];
      cand = bb.x <= u_min || bb.y >= l_max;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, cand);
    if (!bal) continue;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&mm[4], (unsigned long long)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (cand) list[base + __popc(bal & ((1u << lane) - 1u))] = (int32_t)u;
  }
}

// Extremes of pass 2: the FP32 value (squared distance) and the pair holding
// it; ties go to the smaller (p, q), so that the result is the same in any
// order of evaluation.
struct RExt {
  float v;
  int p, q;
};

__device__ __forceinline__ bool rext_before(bool hi, const RExt& x, const RExt& y) {
  if (x.v != y.v) return hi ? x.v > y.v : x.v < y.v;
  return x.p != y.p ? x.p < y.p : x.q < y.q;
}

__device__ __forceinline__ RExt rext_warp(bool hi, RExt x) {
  for (int off = 16; off > 0; off >>= 1) {
    RExt o;
    o.v = __shfl_xor_sync(0xffffffffu, x.v, off);
    o.p = __shfl_xor_sync(0xffffffffu, x.p, off);
    o.q = __shfl_xor_sync(0xffffffffu, x.q, off);
    if (rext_before(hi, o, x)) x = o;
  }
  return x;
}

// The extremal point pair of triangle pair (p, q) (FP32 rescan, first in
// (a, b) order), evaluated in FP64.
template <int M>
__device__ double range_point64(const GeoView& g, int p, int q, bool hi) {
  const float4 cp = g.cen32[p], cq = g.cen32[q];
  const float3 dc = make_float3(cp.x - cq.x, cp.y - cq.y, cp.z - cq.z);
  float best = hi ? -1.f : INFINITY;
  int ia = 0, ib = 0;
  for (int a = 0; a < M; ++a) {
    const float4 pa = g.pts32[(size_t)a * g.nt + p];
    const float ux = dc.x + pa.x, uy = dc.y + pa.y, uz = dc.z + pa.z;
    for (int b = 0; b < M; ++b) {
      const float4 pb = g.pts32[(size_t)b * g.nt + q];
      const float rx = ux - pb.x, ry = uy - pb.y, rz = uz - pb.z;
      const float R2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
      if (hi ? R2 > best : R2 < best) {
        best = R2;
        ia = a;
        ib = b;
      }
    }
  }
  const double* cp64 = g.cen64 + 4 * (size_t)p;
  const double* cq64 = g.cen64 + 4 * (size_t)q;
  const double* pa = g.pts64 + 4 * ((size_t)ia * g.nt + p);
  const double* pb = g.pts64 + 4 * ((size_t)ib * g.nt + q);
  const double rx = (cp64[0] - cq64[0]) + pa[0] - pb[0];
  const double ry = (cp64[1] - cq64[1]) + pa[1] - pb[1];
  const double rz = (cp64[2] - cq64[2]) + pa[2] - pb[2];
  return sqrt(rx * rx + ry * ry + rz * rz);
}

// Pass 2 (FP32 screen), one warp per (test triangle, block of 32 source
// triangles) of a listed block pair: per candidate pair the FP32 minimum and
// maximum over its point pairs. Each block records its extremes; the last
// block to finish reduces the records and re-evaluates the extremal point
// pairs in FP64 (mm[0], mm[1]). The FP32 screen costs a few ulps: the point
// pair it selects is within its rounding of the true extreme.
template <int M>
__global__ void __launch_bounds__(kThreads) k_range32(GeoView g, unsigned long long* mm, const int32_t* list,
                                                      RExt* rec) {
  __shared__ RExt s_ext[2][kWarps];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float u_min = (float)__longlong_as_double((long long)mm[2]);
  const float l_max = (float)__longlong_as_double((long long)mm[3]);
  const int64_t ntask = (int64_t)mm[4] * 32;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  RExt lo = {INFINITY, INT_MAX, INT_MAX}, hi = {-1.f, INT_MAX, INT_MAX};
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntask; t += nwarp) {
    int p, q0;
    if (!sym_task((int64_t)list[t >> 5] * 32 + (t & 31), g.nt, &p, &q0)) continue;
    const int q = min(q0 + lane, g.nt - 1);
    const float4 cp = g.cen32[p], cq = g.cen32[q];
    const float3 dc = make_float3(cp.x - cq.x, cp.y - cq.y, cp.z - cq.z);
    if (!((q0 + lane < g.nt) && q > p && !pair_is_near(g, p, q, g.tvert[p], g.tvert[q], dc))) continue;
    float lb, ub;
    pair_bounds(g, p, q, dc, cp, cq, &lb, &ub);
    if (lb > u_min && ub < l_max) continue;  // cannot hold an extreme
    float4 beta[M];
#pragma unroll
    for (int b = 0; b < M; ++b) beta[b] = g.pts32[(size_t)b * g.nt + q];
    float pmin = INFINITY, pmax = 0.f;
    for (int a = 0; a < M; ++a) {
      const float4 pa = g.pts32[(size_t)a * g.nt + p];
      const float ux = dc.x + pa.x, uy = dc.y + pa.y, uz = dc.z + pa.z;
#pragma unroll
      for (int b = 0; b < M; ++b) {
        const float rx = ux - beta[b].x, ry = uy - beta[b].y, rz = uz - beta[b].z;
        const float R2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
        pmin = fminf(pmin, R2);
        pmax = fmaxf(pmax, R2);
      }
    }
    const RExt xl = {pmin, p, q}, xh = {pmax, p, q};
    if (rext_before(false, xl, lo)) lo = xl;
    if (rext_before(true, xh, hi)) hi = xh;
  }
  lo = rext_warp(false, lo);
  hi = rext_warp(true, hi);
  if (lane == 0) {
    s_ext[0][warp] = lo;
    s_ext[1][warp] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kWarps; ++w) {
      if (rext_before(false, s_ext[0][w], lo)) lo = s_ext[0][w];
      if (rext_before(true, s_ext[1][w], hi)) hi = s_ext[1][w];
    }
    rec[2 * blockIdx.x] = lo;
    rec[2 * blockIdx.x + 1] = hi;
    __threadfence();
    s_last = atomicAdd(&mm[5], 1ull) == (unsigned long long)(gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  // the last block: every record is visible (each was fenced before its count)
  lo = {INFINITY, INT_MAX, INT_MAX};
  hi = {-1.f, INT_MAX, INT_MAX};
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    const RExt a = {__ldcg(&rec[2 * i].v), __ldcg(&rec[2 * i].p), __ldcg(&rec[2 * i].q)};
    const RExt b = {__ldcg(&rec[2 * i + 1].v), __ldcg(&rec[2 * i + 1].p), __ldcg(&rec[2 * i + 1].q)};
    if (rext_before(false, a, lo)) lo = a;
    if (rext_before(true, b, hi)) hi = b;
  }
  lo = rext_warp(false, lo);
  hi = rext_warp(true, hi);
  __syncthreads();
  if (lane == 0) {
    s_ext[0][warp] = lo;
    s_ext[1][warp] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kWarps; ++w) {
      if (rext_before(false, s_ext[0][w], lo)) lo = s_ext[0][w];
      if (rext_before(true, s_ext[1][w], hi)) hi = s_ext[1][w];
    }
    if (lo.v < INFINITY) mm[0] = dbits(range_point64<M>(g, lo.p, lo.q, false));
    if (hi.v >= 0.f) mm[1] = dbits(range_point64<M>(g, hi.p, hi.q, true));
    mm[5] = 0ull;
  }
}

// ---------------------------------------------------------------- range
// FP64: every point pair of every regular pair, one warp per (p, 32
// consecutive q).
__global__ void __launch_bounds__(kThreads) k_range64(GeoView g, unsigned long long* mm) {
  const int lane = threadIdx.x & 31;
  const int64_t ntask = regular_units(g.nt);
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double best_lo = INFINITY, best_hi = 0.0;
  for (int64_t task = warp0; task < ntask; task += nwarp) {
    int p, q0;
    if (!sym_task(task, g.nt, &p, &q0)) continue;
    const int q = min(q0 + lane, g.nt - 1);
    const float4 cp = g.cen32[p], cq = g.cen32[q];
    const float3 dc = make_float3(cp.x - cq.x, cp.y - cq.y, cp.z - cq.z);
    if (!((q0 + lane < g.nt) && q > p && !pair_is_near(g, p, q, g.tvert[p], g.tvert[q], dc))) continue;
    const double* cp64 = g.cen64 + 4 * (size_t)p;
    const double* cq64 = g.cen64 + 4 * (size_t)q;
    const double dx = cp64[0] - cq64[0], dy = cp64[1] - cq64[1], dz = cp64[2] - cq64[2];
    for (int a = 0; a < g.m; ++a) {
      const double* pa = g.pts64 + 4 * ((size_t)a * g.nt + p);
      const double ux = dx + pa[0], uy = dy + pa[1], uz = dz + pa[2];
      for (int b = 0; b < g.m; ++b) {
        const double* pb = g.pts64 + 4 * ((size_t)b * g.nt + q);
        const double rx = ux - pb[0], ry = uy - pb[1], rz = uz - pb[2];
        const double R = sqrt(rx * rx + ry * ry + rz * rz);
        best_lo = fmin(best_lo, R);
        best_hi = fmax(best_hi, R);
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    best_lo = fmin(best_lo, __shfl_xor_sync(0xffffffffu, best_lo, off));
    best_hi = fmax(best_hi, __shfl_xor_sync(0xffffffffu, best_hi, off));
  }
  if (lane == 0) {
    if (best_lo < INFINITY) atomicMin(&mm[0], dbits(best_lo));
    if (best_hi > 0.0) atomicMax(&mm[1], dbits(best_hi));
  }
}

// ---------------------------------------------------------------- regular fill
struct KSum {  // Kahan-compensated FP32 sum
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

// Blocks of 512 threads when the table is staged in shared memory (one CTA
// per SM holds it), 256 otherwise.
// One warp task of the regular-pair fill: test triangle p, source triangles
// q0..q0+31 (one per lane).
// Green value source of the regular-pair kernels.
enum GreenMode : int {
  kDirect = 0,    // sincospi of k R / pi, times 1/R
  kLagrange = 1,  // e^{-jkR}/R from the Green table (Lagrange, Section II.C)
  kExpOverR = 2,  // e^{-jkR} from the Exp table (linear), times 1/R
};

// DEFER: lookups in the hot loop are branch-free and the rare evaluations in
// lattice cells holding samples are corrected after it (tables with few such
// cells); otherwise each lookup branches to the exact path at once.
// Where the regular fill's 3x3 blocks go (one evaluation per unordered
// pair). DenseUpper (dense and batched fills): Z[m][n] only, the rows of the
// test triangle's edges; k_symmetrize32 then adds the transpose (Z <- Z + Z^T
// on a block that held zero), so that a warp's atomics hit three rows
// instead of 3 + 32. CsrSink (near-field sparse fill): Z[m][n] at its
// position in the CSR pattern, dropped where (m, n) is not in it.
struct DenseUpper {
  float2* Z;
  int64_t ldz;
  __device__ __forceinline__ void operator()(int m, int n, float2 v) const { atomicAdd(Z + (int64_t)m * ldz + n, v); }
};

template <class T>
struct CsrSink {
  const int64_t* row_ptr;  // [ne + 1]
  const int32_t* cols;     // sorted per row
  T* vals;
  __device__ __forceinline__ int64_t find(int m, int n) const {
    int64_t lo = row_ptr[m], hi = row_ptr[m + 1];
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (cols[mid] < n) lo = mid + 1;
      else hi = mid;
    }
    return lo < row_ptr[m + 1] && cols[lo] == n ? lo : -1;
  }
  __device__ __forceinline__ void operator()(int m, int n, float2 v) const {
    const int64_t i = find(m, n);
    if (i >= 0) atomicAdd(reinterpret_cast<float2*>(vals + i), v);
  }
  __device__ __forceinline__ void add(int m, int n, double zr, double zi) const {
    const int64_t i = find(m, n);
    if (i < 0) return;
    if constexpr (sizeof(T) == 8) {
      atomicAdd(reinterpret_cast<float2*>(vals + i), make_float2((float)zr, (float)zi));
    } else {
      atomicAdd(reinterpret_cast<double*>(vals + i), zr);
      atomicAdd(reinterpret_cast<double*>(vals + i) + 1, zi);
    }
  }
};

template <int M, int MODE, bool DEFER = true, class Sink = DenseUpper>
__device__ __forceinline__ void regular_pair32(const GeoView& g, const Tab32& T, float kpi, float scale, float inv_k2,
                                               int p, int q, bool ok, const Sink& sink);

template <int M, int MODE, bool DEFER, class Sink>
__device__ __forceinline__ void regular_task32(const GeoView& g, const Tab32& T, float kpi, float scale, float inv_k2,
                                               const Sink& sink, int p, int q0, int lane) {
  const int q = min(q0 + lane, g.nt - 1);
  const float4 cp = g.cen32[p], cq = g.cen32[q];
  const float3 dc = make_float3(cp.x - cq.x, cp.y - cq.y, cp.z - cq.z);
  const bool ok = (q0 + lane < g.nt) && q > p && !pair_is_near(g, p, q, g.tvert[p], g.tvert[q], dc);
  regular_pair32<M, MODE, DEFER>(g, T, kpi, scale, inv_k2, p, q, ok, sink);
}

// The 3x3 block of regular pair (p, q) (q per lane; lanes with ok == false
// take part in the warp's work but write nothing), handed to `sink`.
template <int M, int MODE, bool DEFER, class Sink>
__device__ __forceinline__ void regular_pair32(const GeoView& g, const Tab32& T, float kpi, float scale, float inv_k2,
                                               int p, int q, bool ok, const Sink& sink) {
  const float4 cp = g.cen32[p], cq = g.cen32[q];
  const float3 dc = make_float3(cp.x - cq.x, cp.y - cq.y, cp.z - cq.z);
  if (!__any_sync(0xffffffffu, ok)) return;
  float4 beta[M];
#pragma unroll
  for (int b = 0; b < M; ++b) beta[b] = g.pts32[(size_t)b * g.nt + q];
  KSum M0r, M0i, Mar[3], Mai[3], Mbr[3], Mbi[3], Mabr, Mabi;
  static_assert(M <= 8, "point pairs are flagged in 8 bits per test point");
  unsigned long long emask = 0;  // point pairs (bit 8 a + b) whose lattice cell holds samples
  float4 al_next = g.pts32[p];
#pragma unroll 1
  for (int a = 0; a < M; ++a) {
    const float4 al = al_next;
    if (a + 1 < M) al_next = g.pts32[(size_t)(a + 1) * g.nt + p];  // issued a whole iteration early
    const float ux = dc.x + al.x, uy = dc.y + al.y, uz = dc.z + al.z;
    // Green values of the M source points: branch-free lookups accumulated at
    // once (every load of the row in flight together); a row that met a
    // lattice cell holding samples is corrected after the loop
    float s0r = 0.f, s0i = 0.f, sbr[3] = {0.f, 0.f, 0.f}, sbi[3] = {0.f, 0.f, 0.f};
    unsigned rowbits = 0;
#pragma unroll
    for (int b = 0; b < M; ++b) {
      const float rx = ux - beta[b].x, ry = uy - beta[b].y, rz = uz - beta[b].z;
      const float R2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
      const float rs = rsqrtf(R2);
      float gr, gi;
      if (MODE == kLagrange) {
        bool sl = false;
        const float2 f = DEFER ? lookup32_fast<3>(T, R2 * rs, &sl) : lookup32<3>(T, R2 * rs);  // e^{-jkR}/R
        if (sl) rowbits |= 1u << b;
        gr = f.x * beta[b].w;
        gi = f.y * beta[b].w;
      } else if (MODE == kExpOverR) {
        bool sl = false;
        const float2 f = DEFER ? lookup32_fast<1>(T, R2 * rs, &sl) : lookup32<1>(T, R2 * rs);  // e^{-jkR}
        if (sl) rowbits |= 1u << b;
        const float wr = beta[b].w * rs;
        gr = f.x * wr;
        gi = f.y * wr;
      } else {
        float sn, cs;
        sincospif(R2 * rs * kpi, &sn, &cs);  // kR / pi
        const float wr = beta[b].w * rs;
        gr = cs * wr;
        gi = -sn * wr;
      }
      s0r += gr;
      s0i += gi;
      sbr[0] = fmaf(beta[b].x, gr, sbr[0]);
      sbi[0] = fmaf(beta[b].x, gi, sbi[0]);
      sbr[1] = fmaf(beta[b].y, gr, sbr[1]);
      sbi[1] = fmaf(beta[b].y, gi, sbi[1]);
      sbr[2] = fmaf(beta[b].z, gr, sbr[2]);
      sbi[2] = fmaf(beta[b].z, gi, sbi[2]);
    }
    emask |= (unsigned long long)rowbits << (8 * a);
    const float wa = al.w;
    M0r.add(wa * s0r);
    M0i.add(wa * s0i);
    const float wal[3] = {wa * al.x, wa * al.y, wa * al.z};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Mar[c].add(wal[c] * s0r);
      Mai[c].add(wal[c] * s0i);
      Mbr[c].add(wa * sbr[c]);
      Mbi[c].add(wa * sbi[c]);
    }
    Mabr.add(wal[0] * sbr[0] + wal[1] * sbr[1] + wal[2] * sbr[2]);
    Mabi.add(wal[0] * sbi[0] + wal[1] * sbi[1] + wal[2] * sbi[2]);
  }
  if (DEFER && MODE != kDirect && __any_sync(0xffffffffu, emask != 0ull)) {
    // exact values where the lattice cell holds samples: add (exact - cell
    // polynomial) to the moments of those point pairs only, in row order,
    // with the same float operations for R as the loop above
    while (emask) {
      const int bit = __ffsll((long long)emask) - 1;
      emask &= emask - 1;
      const int a = bit >> 3, b = bit & 7;
      const float4 al = g.pts32[(size_t)a * g.nt + p];
      const float4 be = g.pts32[(size_t)b * g.nt + q];
      const float ux = dc.x + al.x, uy = dc.y + al.y, uz = dc.z + al.z;
      const float rx = ux - be.x, ry = uy - be.y, rz = uz - be.z;
      const float R2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
      const float rs = rsqrtf(R2);
      constexpr int D = MODE == kLagrange ? 3 : 1;
      bool sl;
      const float2 fa = lookup32_fast<D>(T, R2 * rs, &sl);
      const float2 fe = lookup32_slow<D>(T, R2 * rs);
      const float w = al.w * (MODE == kLagrange ? be.w : be.w * rs);
      const float dr = (fe.x - fa.x) * w, di = (fe.y - fa.y) * w;
      const float ab = al.x * be.x + al.y * be.y + al.z * be.z;
      const float alv[3] = {al.x, al.y, al.z}, bev[3] = {be.x, be.y, be.z};
      M0r.add(dr);
      M0i.add(di);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Mar[c].add(alv[c] * dr);
        Mai[c].add(alv[c] * di);
        Mbr[c].add(bev[c] * dr);
        Mbi[c].add(bev[c] * di);
      }
      Mabr.add(ab * dr);
      Mabi.add(ab * di);
    }
  }
  if (!ok) return;
  const int4 ep = g.tedge[p], eq = g.tedge[q];
  const int ecp[3] = {ep.x, ep.y, ep.z}, ecq[3] = {eq.x, eq.y, eq.z};
  const float m0r = M0r.s, m0i = M0i.s;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (!edge_valid(ecp[i])) continue;
    const float4 gp = g.geo32[3 * (size_t)p + i];  // delta_i, s_i l_i
    const float dMbr = gp.x * Mbr[0].s + gp.y * Mbr[1].s + gp.z * Mbr[2].s;
    const float dMbi = gp.x * Mbi[0].s + gp.y * Mbi[1].s + gp.z * Mbi[2].s;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (!edge_valid(ecq[j])) continue;
      const float4 gq = g.geo32[3 * (size_t)q + j];  // eps_j, s_j l_j
      const float eMar = gq.x * Mar[0].s + gq.y * Mar[1].s + gq.z * Mar[2].s;
      const float eMai = gq.x * Mai[0].s + gq.y * Mai[1].s + gq.z * Mai[2].s;
      const float de = gp.x * gq.x + gp.y * gq.y + gp.z * gq.z;
      const float br = 0.25f * (Mabr.s + eMar + dMbr + de * m0r) - m0r * inv_k2;
      const float bi = 0.25f * (Mabi.s + eMai + dMbi + de * m0i) - m0i * inv_k2;
      const float c = scale * gp.w * gq.w;  // k eta/(4 pi) s_i l_i s_j l_j
      // j * c * (br + j bi) = c * (-bi + j br)
      sink(edge_of(ecp[i]), edge_of(ecq[j]), make_float2(-c * bi, c * br));
    }
  }
}

template <int M, int MODE, bool SMEM, bool DEFER = true>
__global__ void __launch_bounds__(SMEM ? 512 : kThreads) k_fill_regular32(GeoView g, TabView tv, float kpi,
                                                                          float scale, float inv_k2, float2* Z,
                                                                          int64_t ldz) {
  extern __shared__ __align__(16) unsigned char smem[];
  Tab32 T = tab32(tv);
  if (MODE != kDirect && SMEM) {  // the lattice image (lat_b only for the cubic Green table)
    const int nl = tv.n_lat, nblob = (int)tv.blob_vec4();
    float4* sa = reinterpret_cast<float4*>(smem);
    float4* sb = sa + nl;
    float4* sblob = MODE == kLagrange ? sb + nl : sb;
    for (int i = threadIdx.x; i < nl; i += blockDim.x) {
      sa[i] = tv.lat_a[i];
      if (MODE == kLagrange) sb[i] = tv.lat_b[i];
    }
    for (int i = threadIdx.x; i < nblob; i += blockDim.x) sblob[i] = tv.lat_blob[i];
    __syncthreads();
    T.la = sa;
    if (MODE == kLagrange) T.lb = sb;  // the Exp table's lat_b (read only on the exact path) stays global
    tab32_blob(T, tv, sblob);
  }
  const int lane = threadIdx.x & 31;
  const int64_t ntask = regular_units(g.nt);
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t task = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < ntask; task += nwarp) {
    int p, q0;
    if (sym_task(task, g.nt, &p, &q0))
      regular_task32<M, MODE, DEFER>(g, T, kpi, scale, inv_k2, DenseUpper{Z, ldz}, p, q0, lane);
  }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_fill_regular64(GeoView g, TabView tv, double k, double scale,
                                                             double inv_k2, double2* Z, int64_t ldz) {
  const int lane = threadIdx.x & 31;
  const int m = g.m;
  const int64_t ntask = regular_units(g.nt);
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t task = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < ntask; task += nwarp) {
    int p, q0;
    if (!sym_task(task, g.nt, &p, &q0)) continue;
    const int q = min(q0 + lane, g.nt - 1);
    const float4 cp32 = g.cen32[p], cq32 = g.cen32[q];
    const float3 dc32 = make_float3(cp32.x - cq32.x, cp32.y - cq32.y, cp32.z - cq32.z);
    const bool ok = (q0 + lane < g.nt) && q > p && !pair_is_near(g, p, q, g.tvert[p], g.tvert[q], dc32);
    if (!ok) continue;
    const double* cp = g.cen64 + 4 * (size_t)p;
    const double* cq = g.cen64 + 4 * (size_t)q;
    const double dx = cp[0] - cq[0], dy = cp[1] - cq[1], dz = cp[2] - cq[2];
    double M0r = 0, M0i = 0, Mar[3] = {0, 0, 0}, Mai[3] = {0, 0, 0}, Mbr[3] = {0, 0, 0}, Mbi[3] = {0, 0, 0};
    double Mabr = 0, Mabi = 0;
    for (int a = 0; a < m; ++a) {
      const double* al = g.pts64 + 4 * ((size_t)a * g.nt + p);
      const double ux = dx + al[0], uy = dy + al[1], uz = dz + al[2];
      double s0r = 0, s0i = 0, sbr[3] = {0, 0, 0}, sbi[3] = {0, 0, 0};
      for (int b = 0; b < m; ++b) {
        const double* be = g.pts64 + 4 * ((size_t)b * g.nt + q);
        const double rx = ux - be[0], ry = uy - be[1], rz = uz - be[2];
        const double R = sqrt(rx * rx + ry * ry + rz * rz);
        double gr, gi;
        if (MODE == kLagrange) {
          double2 f = lookup64<3>(tv, R);
          gr = f.x * be[3];
          gi = f.y * be[3];
        } else if (MODE == kExpOverR) {
          double2 f = lookup64<1>(tv, R);
          const double wr = be[3] / R;
          gr = f.x * wr;
          gi = f.y * wr;
        } else {
          double sn, cs;
          sincos(k * R, &sn, &cs);
          const double wr = be[3] / R;
          gr = cs * wr;
          gi = -sn * wr;
        }
        s0r += gr;
        s0i += gi;
        for (int c = 0; c < 3; ++c) {
          sbr[c] += be[c] * gr;
          sbi[c] += be[c] * gi;
        }
      }
      const double wa = al[3];
      M0r += wa * s0r;
      M0i += wa * s0i;
      for (int c = 0; c < 3; ++c) {
        Mar[c] += wa * al[c] * s0r;
        Mai[c] += wa * al[c] * s0i;
        Mbr[c] += wa * sbr[c];
        Mbi[c] += wa * sbi[c];
      }
      Mabr += wa * (al[0] * sbr[0] + al[1] * sbr[1] + al[2] * sbr[2]);
      Mabi += wa * (al[0] * sbi[0] + al[1] * sbi[1] + al[2] * sbi[2]);
    }
    const int4 ep = g.tedge[p], eq = g.tedge[q];
    const int ecp[3] = {ep.x, ep.y, ep.z}, ecq[3] = {eq.x, eq.y, eq.z};
    for (int i = 0; i < 3; ++i) {
      if (!edge_valid(ecp[i])) continue;
      const double* gp = g.geo64 + 4 * (3 * (size_t)p + i);
      const double dMbr = gp[0] * Mbr[0] + gp[1] * Mbr[1] + gp[2] * Mbr[2];
      const double dMbi = gp[0] * Mbi[0] + gp[1] * Mbi[1] + gp[2] * Mbi[2];
      double* zrow = reinterpret_cast<double*>(Z + (int64_t)edge_of(ecp[i]) * ldz);
      for (int j = 0; j < 3; ++j) {
        if (!edge_valid(ecq[j])) continue;
        const double* gq = g.geo64 + 4 * (3 * (size_t)q + j);
        const double eMar = gq[0] * Mar[0] + gq[1] * Mar[1] + gq[2] * Mar[2];
        const double eMai = gq[0] * Mai[0] + gq[1] * Mai[1] + gq[2] * Mai[2];
        const double de = gp[0] * gq[0] + gp[1] * gq[1] + gp[2] * gq[2];
        const double br = 0.25 * (Mabr + eMar + dMbr + de * M0r) - M0r * inv_k2;
        const double bi = 0.25 * (Mabi + eMai + dMbi + de * M0i) - M0i * inv_k2;
        const double c = scale * gp[3] * gq[3];
        double* z = zrow + 2 * edge_of(ecq[j]);
        atomicAdd(z, -c * bi);
        atomicAdd(z + 1, c * br);
        double* zt = reinterpret_cast<double*>(Z + (int64_t)edge_of(ecq[j]) * ldz + edge_of(ecp[i]));
        atomicAdd(zt, -c * bi);
        atomicAdd(zt + 1, c * br);
      }
    }
  }
}

// ---------------------------------------------------------------- near pairs (FP64)
struct NearArgs {
  double k, scale, inv_k2;
  int nphi, nl;
  double gx_phi[32], gw_phi[32], gx_l[32], gw_l[32];
  float fx_phi[32], fw_phi[32], fx_l[32], fw_l[32];  // the same rules in FP32
};

struct C2 {
  double re, im;
};

struct C2f {  // FP32 complex of the mixed-precision near-block assembly
  float re, im;
};

struct KScal {  // per-wavenumber scalars of the near-pair fill
  double k, scale, inv_k2, inv_k;
};

__device__ __forceinline__ C2 exp_mjkr(double k, double R, const TabView* te, bool use_table) {
  const double x = use_table ? R * te->xscale64 : R;  // table units
  if (use_table && x >= te->r_lo && x <= te->r_hi) {
    double2 f = lookup64<1>(*te, R);
    return C2{f.x, f.y};
  }
  double s, c;
  sincos(k * R, &s, &c);
  return C2{c, -s};
}

// Inner integrals over triangle v for observation point r (1/(4 pi) included).
__device__ void inner_integrals(const double r[3], const double v[3][3], const NearArgs& A, double k,
                                const TabView* te, bool use_table, C2* I0, C2 I1[3], double rho0[3]) {
  double e1[3] = {v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2]};
  double e2[3] = {v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2]};
  double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  double inv = 1.0 / sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  n[0] *= inv;
  n[1] *= inv;
  n[2] *= inv;
  const double h = n[0] * (r[0] - v[0][0]) + n[1] * (r[1] - v[0][1]) + n[2] * (r[2] - v[0][2]);
  const double d = fabs(h);
  for (int x = 0; x < 3; ++x) rho0[x] = r[x] - h * n[x];
  const C2 ed = exp_mjkr(k, d, te, use_table);
  double sre = 0, sim = 0;                       // scalar sector sums
  double vre[3] = {0, 0, 0}, vim[3] = {0, 0, 0};  // vector remainder
  double vst[3] = {0, 0, 0};                     // vector static part
  for (int e = 0; e < 3; ++e) {
    const double* a = v[e];
    const double* b = v[(e + 1) % 3];
    double t[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    const double len = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    t[0] /= len;
    t[1] /= len;
    t[2] /= len;
    const double mh[3] = {t[1] * n[2] - t[2] * n[1], t[2] * n[0] - t[0] * n[2], t[0] * n[1] - t[1] * n[0]};
    const double ar[3] = {a[0] - rho0[0], a[1] - rho0[1], a[2] - rho0[2]};
    const double br[3] = {b[0] - rho0[0], b[1] - rho0[1], b[2] - rho0[2]};
    const double P0 = ar[0] * mh[0] + ar[1] * mh[1] + ar[2] * mh[2];
    const double lm = ar[0] * t[0] + ar[1] * t[1] + ar[2] * t[2];
    const double lp = br[0] * t[0] + br[1] * t[1] + br[2] * t[2];
    if (fabs(P0) > 1e-12 * len) {
      const double aP = fabs(P0);
      const double um = asinh(lm / aP), up = asinh(lp / aP);
      const double half = 0.5 * (up - um), mid = 0.5 * (up + um);
      double cr = 0, ci = 0;
      for (int i = 0; i < A.nphi; ++i) {
        const double u = mid + half * A.gx_phi[i];
        const double ch = cosh(u);
        const double rho = aP * ch;
        const double Re = sqrt(rho * rho + d * d);
        const C2 eR = exp_mjkr(k, Re, te, use_table);
        const double wt = A.gw_phi[i] / ch;
        cr += (ed.re - eR.re) * wt;
        ci += (ed.im - eR.im) * wt;
      }
      const double sg = P0 > 0 ? half : -half;
      sre += cr * sg;
      sim += ci * sg;
    }
    double lr = 0, li = 0;
    for (int i = 0; i < A.nl; ++i) {
      const double s = 0.5 * len * (A.gx_l[i] + 1.0);
      const double x0 = a[0] + t[0] * s - r[0], x1 = a[1] + t[1] * s - r[1], x2 = a[2] + t[2] * s - r[2];
      const double R = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
      const C2 eR = exp_mjkr(k, R, te, use_table);
      lr += (eR.re - 1.0) * A.gw_l[i];
      li += (eR.im + k * R) * A.gw_l[i];
    }
    lr *= 0.5 * len;
    li *= 0.5 * len;
    const double R02 = P0 * P0 + d * d;
    const double Rm = sqrt(lm * lm + R02), Rp = sqrt(lp * lp + R02);
    double st = 0.5 * (lp * Rp - lm * Rm);
    if (R02 > 0) {
      const double fp = lp >= 0 ? lp + Rp : R02 / (Rp - lp);
      const double fm = lm >= 0 ? lm + Rm : R02 / (Rm - lm);
      st += 0.5 * R02 * (log(fp) - log(fm));
    }
    for (int x = 0; x < 3; ++x) {
      vre[x] += mh[x] * lr;
      vim[x] += mh[x] * li;
      vst[x] += mh[x] * st;
    }
  }
  const double c4 = 1.0 / (4.0 * kPi);
  // I0 = (-j/k) s / (4 pi);  I1 = ((j/k) v + v_static) / (4 pi)
  I0->re = sim / k * c4;
  I0->im = -sre / k * c4;
  for (int x = 0; x < 3; ++x) {
    I1[x].re = (-vim[x] / k + vst[x]) * c4;
    I1[x].im = (vre[x] / k) * c4;
  }
}

__device__ __forceinline__ float2 exp32(float kpi, float R, const Tab32& te, bool use_table, float lo, float hi) {
  const float x = R * te.xscale;  // lo, hi in table units
  if (use_table && x >= lo && x <= hi) return lookup32<1>(te, R);
  float sn, cs;
  sincospif(R * kpi, &sn, &cs);
  return make_float2(cs, -sn);
}

// Mixed precision: the geometry (normal, projection, foot distances, edge
// frames) and the closed-form static part in FP64; the sampling of e^{-jkR}
// at the angular and line nodes of each edge and its sums in FP32 (relative
// quantities of the size of a triangle, FP32 Exp table). The caller assembles
// the 3x3 block from I0, I1 in FP32.
// FP64 where the terms cancel (projection, in-plane distances, the static
// closed form, all sums), FP32 sampling of e^{-jkR} on the edges. The source
// frame (normal, edge tangents, lengths, edge normals) is precomputed per
// triangle; |r - v_c| serves as R at the ends of both edges that meet at v_c,
// and the static log term is one log of a ratio per edge.
__device__ void inner_integrals_mixed(const double r[3], const double v[3][3], const double* __restrict__ fr,
                                      const float* __restrict__ fr32, const NearArgs& A, double k, double inv_k,
                                      const Tab32& te, bool use_table, float lo, float hi, C2* I0, C2 I1[3],
                                      double rho0[3]) {
  const float kpi = (float)(k / kPi), k32 = (float)k;
  const double n[3] = {fr[0], fr[1], fr[2]};
  const double h = n[0] * (r[0] - v[0][0]) + n[1] * (r[1] - v[0][1]) + n[2] * (r[2] - v[0][2]);
  const double d = fabs(h);
  for (int x = 0; x < 3; ++x) rho0[x] = r[x] - h * n[x];
  // |r - v_c| (scalars, so that the edge loop picks them without a local array)
  double Rv0, Rv1, Rv2;
  {
    const double* w = v[0];
    Rv0 = sqrt((w[0] - r[0]) * (w[0] - r[0]) + (w[1] - r[1]) * (w[1] - r[1]) + (w[2] - r[2]) * (w[2] - r[2]));
    w = v[1];
    Rv1 = sqrt((w[0] - r[0]) * (w[0] - r[0]) + (w[1] - r[1]) * (w[1] - r[1]) + (w[2] - r[2]) * (w[2] - r[2]));
    w = v[2];
    Rv2 = sqrt((w[0] - r[0]) * (w[0] - r[0]) + (w[1] - r[1]) * (w[1] - r[1]) + (w[2] - r[2]) * (w[2] - r[2]));
  }
  const float d32 = (float)d;
  const float2 ed = exp32(kpi, d32, te, use_table, lo, hi);
  // the sampled (dynamic) sums carry FP32 samples: FP32 accumulation; the
  // static closed form stays in FP64
  float sre = 0.f, sim = 0.f, vre[3] = {0.f, 0.f, 0.f}, vim[3] = {0.f, 0.f, 0.f};
  double vst[3] = {0, 0, 0};
  for (int e = 0; e < 3; ++e) {
    const double* a = v[e];
    const double len = fr[3 + e];
    const double t[3] = {fr[6 + 3 * e], fr[7 + 3 * e], fr[8 + 3 * e]};
    const double mh[3] = {fr[15 + 3 * e], fr[16 + 3 * e], fr[17 + 3 * e]};
    const double ar[3] = {a[0] - rho0[0], a[1] - rho0[1], a[2] - rho0[2]};
    const double P0 = ar[0] * mh[0] + ar[1] * mh[1] + ar[2] * mh[2];
    const double lm = ar[0] * t[0] + ar[1] * t[1] + ar[2] * t[2];
    const double lp = lm + len;
    if (fabs(P0) > 1e-12 * len) {
      const float aP32 = (float)fabs(P0);
      const float um = asinhf((float)lm / aP32), up = asinhf((float)lp / aP32);
      const float half = 0.5f * (up - um), mid = 0.5f * (up + um);
      float cr = 0.f, ci = 0.f;
      for (int i = 0; i < A.nphi; ++i) {
        const float u = fmaf(half, A.fx_phi[i], mid);
        const float E = expf(u);
        const float ch = 0.5f * (E + __frcp_rn(E));
        const float rho = aP32 * ch;
        const float Re = sqrtf(fmaf(rho, rho, d32 * d32));
        const float2 eR = exp32(kpi, Re, te, use_table, lo, hi);
        const float wt = A.fw_phi[i] * __frcp_rn(ch);
        cr = fmaf(ed.x - eR.x, wt, cr);
        ci = fmaf(ed.y - eR.y, wt, ci);
      }
      const float sg = P0 > 0 ? half : -half;
      sre = fmaf(cr, sg, sre);
      sim = fmaf(ci, sg, sim);
    }
    // line integral of e^{-jkR} - 1 + jkR from r's position relative to a
    const float ax = (float)(a[0] - r[0]), ay = (float)(a[1] - r[1]), az = (float)(a[2] - r[2]);
    const float tx = fr32[3 + 3 * e], ty = fr32[4 + 3 * e], tz = fr32[5 + 3 * e];
    const float hl = 0.5f * fr32[e];
    float lr = 0.f, li = 0.f;
    for (int i = 0; i < A.nl; ++i) {
      const float sp = hl * (A.fx_l[i] + 1.0f);
      const float x0 = fmaf(tx, sp, ax), x1 = fmaf(ty, sp, ay), x2 = fmaf(tz, sp, az);
      const float R = sqrtf(fmaf(x0, x0, fmaf(x1, x1, x2 * x2)));
      const float2 eR = exp32(kpi, R, te, use_table, lo, hi);
      lr = fmaf(eR.x - 1.0f, A.fw_l[i], lr);
      li = fmaf(fmaf(k32, R, eR.y), A.fw_l[i], li);
    }
    lr *= hl;
    li *= hl;
    // static part: int R dl along the edge, with Rm = |r - a|, Rp = |r - b|;
    // log(fp / fm) with fp = lp + Rp = R02 / (Rp - lp), fm = lm + Rm =
    // R02 / (Rm - lm), each in its cancellation-free form (lp >= lm), as one
    // quotient
    const double R02 = P0 * P0 + d * d;
    const double Rm = e == 0 ? Rv0 : (e == 1 ? Rv1 : Rv2), Rp = e == 0 ? Rv1 : (e == 1 ? Rv2 : Rv0);
    double st = 0.5 * (lp * Rp - lm * Rm);
    if (R02 > 0) {
      double ratio;
      if (lm >= 0) ratio = (lp + Rp) / (lm + Rm);
      else if (lp >= 0) ratio = (lp + Rp) * (Rm - lm) / R02;
      else ratio = (Rm - lm) / (Rp - lp);
      st += 0.5 * R02 * log(ratio);
    }
    const float mx = fr32[12 + 3 * e], my = fr32[13 + 3 * e], mz = fr32[14 + 3 * e];
    vre[0] = fmaf(mx, lr, vre[0]);
    vre[1] = fmaf(my, lr, vre[1]);
    vre[2] = fmaf(mz, lr, vre[2]);
    vim[0] = fmaf(mx, li, vim[0]);
    vim[1] = fmaf(my, li, vim[1]);
    vim[2] = fmaf(mz, li, vim[2]);
    for (int x = 0; x < 3; ++x) vst[x] += mh[x] * st;
  }
  const double c4 = 1.0 / (4.0 * kPi), ikc4 = inv_k * c4;
  // I0 = (-j/k) s / (4 pi);  I1 = ((j/k) v + v_static) / (4 pi)
  I0->re = (double)sim * ikc4;
  I0->im = -(double)sre * ikc4;
  for (int x = 0; x < 3; ++x) {
    I1[x].re = fma(-(double)vim[x], inv_k, vst[x]) * c4;
    I1[x].im = (double)vre[x] * ikc4;
  }
}

// Reduce-scatter of the nine complex entries of a 3 x 3 block over the G
// lanes of a group (G = 4 or 8): at each halving step a lane keeps one half
// of its entries and adds the partner's copy of that half, so that the group
// sums end spread over the lanes (at most ceil(9 / G) + 1 entries each) with
// no more additions than entries exchanged.
template <int N, class CT>
__device__ __forceinline__ void rs_halve(const CT (&in)[N], CT (&out)[(N + 1) / 2], bool upper, int off,
                                         unsigned gmask) {
  constexpr int H = (N + 1) / 2;
#pragma unroll
  for (int s = 0; s < H; ++s) {
    const CT lo_v = in[s];
    const CT hi_v = (H + s < N) ? in[H + s] : CT{0, 0};
    const CT keep = upper ? hi_v : lo_v, send = upper ? lo_v : hi_v;
    out[s].re = keep.re + __shfl_xor_sync(gmask, send.re, off);
    out[s].im = keep.im + __shfl_xor_sync(gmask, send.im, off);
  }
}

// One near pair per group of G lanes (G >= the rule size; lane = test point;
// lanes >= m idle); every lane of the group must call (valid_pair is uniform
// over the group). The 3 x 3 block is reduce-scattered over the group and
// each lane adds its entries to Z.
template <class Out>
struct DenseOut {  // Z[m][n] += z (row-major, ld = ldz)
  Out* Z;
  int64_t ldz;
  __device__ __forceinline__ void add(int m, int n, double zr, double zi) const {
    Out* z = Z + (int64_t)m * ldz + n;
    if constexpr (sizeof(Out) == 8) {
      atomicAdd(reinterpret_cast<float2*>(z), make_float2((float)zr, (float)zi));
    } else {
      atomicAdd(reinterpret_cast<double*>(z), zr);
      atomicAdd(reinterpret_cast<double*>(z) + 1, zi);
    }
  }
};

template <bool MIXED, int G, class Sink>
__device__ __forceinline__ void near_pair(const GeoView& g, const TabView& te, const Tab32& te32, float lo32,
                                          float hi32, bool use_table, const NearArgs& A, const KScal& ks,
                                          const Sink& sink, int64_t idx, bool valid_pair, int sub, unsigned gmask);

template <class Out, bool MIXED, int G = 8>
__device__ __forceinline__ void near_task(const GeoView& g, const TabView& te, const Tab32& te32, float lo32,
                                          float hi32, bool use_table, const NearArgs& A, const KScal& ks, Out* Z,
                                          int64_t ldz, int64_t n_near, int64_t idx, bool valid_pair, int sub,
                                          unsigned gmask) {
  near_pair<MIXED, G>(g, te, te32, lo32, hi32, use_table, A, ks, DenseOut<Out>{Z, ldz}, idx, valid_pair, sub, gmask);
}

// The 3x3 block of near pair idx (of the mesh's near list) on a group of G
// lanes, handed to `sink` (sink.add(m, n, re, im)).
template <bool MIXED, int G, class Sink>
__device__ __forceinline__ void near_pair(const GeoView& g, const TabView& te, const Tab32& te32, float lo32,
                                          float hi32, bool use_table, const NearArgs& A, const KScal& ks,
                                          const Sink& sink, int64_t idx, bool valid_pair, int sub, unsigned gmask) {
  if (!valid_pair) return;
  const int p = g.near_row[idx], q = g.near_idx[idx];
  // MIXED: the 3x3 block is assembled from the FP64 inner integrals in FP32
  // (products and sums of smooth quantities, added into an FP32 Z); else FP64
  using CT = typename std::conditional<MIXED, C2f, C2>::type;
  using RT = typename std::conditional<MIXED, float, double>::type;
  CT acc[9];
#pragma unroll
  for (int u = 0; u < 9; ++u) acc[u] = CT{0, 0};
  if (sub < g.m) {
    double vq[3][3];
    for (int c = 0; c < 3; ++c)
      for (int x = 0; x < 3; ++x) vq[c][x] = g.v64[9 * (size_t)q + 3 * c + x];
    const double* cp = g.cen64 + 4 * (size_t)p;
    const double* al = g.pts64 + 4 * ((size_t)sub * g.nt + p);
    const double ra[3] = {cp[0] + al[0], cp[1] + al[1], cp[2] + al[2]};
    C2 I0, I1[3];
    double rho0[3];
    if (MIXED)
      inner_integrals_mixed(ra, vq, g.frame64 + kFrame * (size_t)q, g.frame32 + kFrame32 * (size_t)q, A, ks.k,
                            ks.inv_k, te32, use_table, lo32, hi32, &I0, I1, rho0);
    else inner_integrals(ra, vq, A, ks.k, &te, use_table, &I0, I1, rho0);
    // entry (i, j): w_a ((r - v_i) . J_j / 4 - I0 / k^2), J_j = I1 + (rho0 - v_j) I0;
    // w_a / 4 folded into I0, I1
    const RT w4 = (RT)(0.25 * al[3]);
    const CT S = {w4 * (RT)I0.re, w4 * (RT)I0.im};
    const CT T[3] = {{w4 * (RT)I1[0].re, w4 * (RT)I1[0].im},
                     {w4 * (RT)I1[1].re, w4 * (RT)I1[1].im},
                     {w4 * (RT)I1[2].re, w4 * (RT)I1[2].im}};
    const RT q4 = (RT)(4.0 * ks.inv_k2);
    const CT Q = {q4 * S.re, q4 * S.im};  // w_a I0 / k^2
    RT f[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double* vpi = g.v64 + 9 * (size_t)p + 3 * i;
      f[i][0] = (RT)(ra[0] - vpi[0]);
      f[i][1] = (RT)(ra[1] - vpi[1]);
      f[i][2] = (RT)(ra[2] - vpi[2]);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      CT J[3];
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const RT dv = (RT)(rho0[x] - vq[j][x]);
        J[x].re = fma(dv, S.re, T[x].re);
        J[x].im = fma(dv, S.im, T[x].im);
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        acc[3 * i + j].re = fma(f[i][0], J[0].re, fma(f[i][1], J[1].re, fma(f[i][2], J[2].re, -Q.re)));
        acc[3 * i + j].im = fma(f[i][0], J[0].im, fma(f[i][1], J[1].im, fma(f[i][2], J[2].im, -Q.im)));
      }
    }
  }
  // reduce-scatter: 9 -> 5 -> 3 (-> 2 for G = 8) entries per lane
  CT r5[5], r3[3];
  constexpr int L1 = G / 2, L2 = G / 4;
  rs_halve<9>(acc, r5, (sub & L1) != 0, L1, gmask);
  rs_halve<5>(r5, r3, (sub & L2) != 0, L2, gmask);
  int first = ((sub & L1) ? 5 : 0) + ((sub & L2) ? 3 : 0);  // entry of slot 0
  int count = (sub & L1) ? ((sub & L2) ? 1 : 3) : ((sub & L2) ? 2 : 3);  // 9 = 5 + 4; 5 = 3 + 2; 4 = 3 + 1
  constexpr int NS = G == 8 ? 2 : 3;
  CT fin[NS];
  if constexpr (G == 8) {
    rs_halve<3>(r3, fin, (sub & 1) != 0, 1, gmask);
    const bool up = (sub & 1) != 0;
    first += up ? 2 : 0;
    count = up ? max(count - 2, 0) : min(count, 2);
  } else {
#pragma unroll
    for (int u = 0; u < 3; ++u) fin[u] = r3[u];
  }
  const double inv_area_q = g.frame64[kFrame * (size_t)q + 24];
  const int4 ep = g.tedge[p], eq = g.tedge[q];
#pragma unroll
  for (int u = 0; u < NS; ++u) {
    if (u >= count) break;
    const int e = first + u, i = e / 3, j = e - 3 * (e / 3);
    const int ci = i == 0 ? ep.x : (i == 1 ? ep.y : ep.z), cj = j == 0 ? eq.x : (j == 1 ? eq.y : eq.z);
    if (!edge_valid(ci) || !edge_valid(cj)) continue;
    const double slp = g.geo64[4 * (3 * (size_t)p + i) + 3], slq = g.geo64[4 * (3 * (size_t)q + j) + 3];
    const double c = ks.scale * slp * slq * inv_area_q;  // k eta s_i l_i s_j l_j / A_q
    sink.add(edge_of(ci), edge_of(cj), -c * (double)fin[u].im, c * (double)fin[u].re);
  }
}

template <class Out, bool MIXED, int G>
__global__ void __launch_bounds__(128) k_fill_near(GeoView g, TabView te, bool use_table, NearArgs A, Out* Z,
                                                   int64_t ldz) {
  const Tab32 te32 = tab32(te);
  const float lo32 = (float)te.r_lo, hi32 = (float)te.r_hi;
  const int64_t n_near = g.near_ptr[g.nt];
  const int sub = threadIdx.x & (G - 1);
  const unsigned gmask = ((1u << G) - 1u) << (threadIdx.x & (32 - G));
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t iters = (n_near + ngroups - 1) / ngroups;  // same trip count in every group of a warp
  for (int64_t it = 0; it < iters; ++it) {
    const int64_t idx = g0 + it * ngroups;
    near_task<Out, MIXED, G>(g, te, te32, lo32, hi32, use_table, A, KScal{A.k, A.scale, A.inv_k2, 1.0 / A.k}, Z, ldz, n_near,
                             idx, idx < n_near, sub, gmask);
  }
}

// ---------------------------------------------------------------- MFIE
// K operator of the magnetic-field equation (the paper's second formulation,
// Section IV.B): Z_mn = 1/2 <f_m, f_n> - <f_m, n x int grad G x f_n dS'>,
// grad G = -(r - r') Phi(R), Phi = (1 + jkR) e^{-jkR} / (4 pi R^3) = (1 + jkR) G_tab / (4 pi R^2)
// with G_tab = e^{-jkR}/R, the Green table's function. Regular pairs: every
// ordered pair (the K block of (q, p) is not the transpose of that of (p, q)).
// Per test point a the source sums P_a = sum_b w_b Phi R x beta_b and
// Q_a = sum_b w_b Phi R (R = r_a - r_b) give the block
//   (s_i l_i s_j l_j / 4) sum_a w_a (alpha_a + delta_i) . (n x (P_a + Q_a x eps_j)),
// expanded with n x (Q x eps) = Q (n.eps) - eps (n.Q) into the outer sums
//   S1 = sum w alpha.(n x P), S2 = sum w n x P, S3 = sum w alpha.Q, S4 = sum w Q,
//   S5 = sum w (n.Q) alpha, S6 = sum w n.Q  (Kahan over a):
//   block = S1 + delta.S2 + (n.eps)(S3 + delta.S4) - S5.eps - (delta.eps) S6.
struct MfieSums {
  KSum s1[2], s2[3][2], s3[2], s4[3][2], s5[3][2], s6[2];
};

__device__ __forceinline__ void mfie_outer(MfieSums& S, float wa, const float4& al, float nx, float ny, float nz,
                                           const float (&Pr)[3], const float (&Pi)[3], const float (&Qr)[3],
                                           const float (&Qi)[3]) {
  const float NPr[3] = {ny * Pr[2] - nz * Pr[1], nz * Pr[0] - nx * Pr[2], nx * Pr[1] - ny * Pr[0]};
  const float NPi[3] = {ny * Pi[2] - nz * Pi[1], nz * Pi[0] - nx * Pi[2], nx * Pi[1] - ny * Pi[0]};
  const float alv[3] = {al.x, al.y, al.z};
  const float nQr = nx * Qr[0] + ny * Qr[1] + nz * Qr[2], nQi = nx * Qi[0] + ny * Qi[1] + nz * Qi[2];
  S.s1[0].add(wa * (alv[0] * NPr[0] + alv[1] * NPr[1] + alv[2] * NPr[2]));
  S.s1[1].add(wa * (alv[0] * NPi[0] + alv[1] * NPi[1] + alv[2] * NPi[2]));
  S.s3[0].add(wa * (alv[0] * Qr[0] + alv[1] * Qr[1] + alv[2] * Qr[2]));
  S.s3[1].add(wa * (alv[0] * Qi[0] + alv[1] * Qi[1] + alv[2] * Qi[2]));
  S.s6[0].add(wa * nQr);
  S.s6[1].add(wa * nQi);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    S.s2[c][0].add(wa * NPr[c]);
    S.s2[c][1].add(wa * NPi[c]);
    S.s4[c][0].add(wa * Qr[c]);
    S.s4[c][1].add(wa * Qi[c]);
    S.s5[c][0].add(wa * nQr * alv[c]);
    S.s5[c][1].add(wa * nQi * alv[c]);
  }
}

// the contribution of one point pair (weight and Phi folded into fr, fi) to P and Q
__device__ __forceinline__ void mfie_point(float fr, float fi, float rx, float ry, float rz, const float4& be,
                                          float (&Pr)[3], float (&Pi)[3], float (&Qr)[3], float (&Qi)[3]) {
  const float cx = ry * be.z - rz * be.y, cy = rz * be.x - rx * be.z, cz = rx * be.y - ry * be.x;  // R x beta
  Qr[0] = fmaf(fr, rx, Qr[0]);
  Qi[0] = fmaf(fi, rx, Qi[0]);
  Qr[1] = fmaf(fr, ry, Qr[1]);
  Qi[1] = fmaf(fi, ry, Qi[1]);
  Qr[2] = fmaf(fr, rz, Qr[2]);
  Qi[2] = fmaf(fi, rz, Qi[2]);
  Pr[0] = fmaf(fr, cx, Pr[0]);
  Pi[0] = fmaf(fi, cx, Pi[0]);
  Pr[1] = fmaf(fr, cy, Pr[1]);
  Pi[1] = fmaf(fi, cy, Pi[1]);
  Pr[2] = fmaf(fr, cz, Pr[2]);
  Pi[2] = fmaf(fi, cz, Pi[2]);
}

template <int M, int MODE, bool DEFER>
__device__ __forceinline__ void mfie_task32(const GeoView& g, const Tab32& T, float kpi, float k32, float scale,
                                            float2* Z, int64_t ldz, int p, int q0, int lane) {
  const int q = min(q0 + lane, g.nt - 1);
  const float4 cp = g.cen32[p], cq = g.cen32[q];
  const float3 dc = make_float3(cp.x - cq.x, cp.y - cq.y, cp.z - cq.z);
  const bool ok = (q0 + lane < g.nt) && !pair_is_near(g, p, q, g.tvert[p], g.tvert[q], dc);
  if (!__any_sync(0xffffffffu, ok)) return;
  float4 beta[M];
#pragma unroll
  for (int b = 0; b < M; ++b) beta[b] = g.pts32[(size_t)b * g.nt + q];
  const float* fp = g.frame32 + kFrame32 * (size_t)p;
  const float nx = fp[21], ny = fp[22], nz = fp[23];
  MfieSums S;
  static_assert(M <= 8, "point pairs are flagged in 8 bits per test point");
  unsigned long long emask = 0;  // point pairs (bit 8 a + b) whose lattice cell holds samples
#pragma unroll 1
  for (int a = 0; a < M; ++a) {
    const float4 al = g.pts32[(size_t)a * g.nt + p];
    const float ux = dc.x + al.x, uy = dc.y + al.y, uz = dc.z + al.z;
    float Pr[3] = {0.f, 0.f, 0.f}, Pi[3] = {0.f, 0.f, 0.f}, Qr[3] = {0.f, 0.f, 0.f}, Qi[3] = {0.f, 0.f, 0.f};
    unsigned rowbits = 0;
#pragma unroll
    for (int b = 0; b < M; ++b) {
      const float rx = ux - beta[b].x, ry = uy - beta[b].y, rz = uz - beta[b].z;
      const float R2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
      const float rs = rsqrtf(R2);
      const float R = R2 * rs;
      float gr, gi;
      if (MODE == kLagrange) {
        bool sl = false;
        const float2 f = DEFER ? lookup32_fast<3>(T, R, &sl) : lookup32<3>(T, R);
        if (sl) rowbits |= 1u << b;
        gr = f.x;
        gi = f.y;
      } else {
        float sn, cs;
        sincospif(R * kpi, &sn, &cs);
        gr = cs * rs;
        gi = -sn * rs;
      }
      const float kR = k32 * R, w2 = beta[b].w * rs * rs;
      mfie_point(fmaf(-kR, gi, gr) * w2, fmaf(kR, gr, gi) * w2, rx, ry, rz, beta[b], Pr, Pi, Qr, Qi);
    }
    emask |= (unsigned long long)rowbits << (8 * a);
    mfie_outer(S, al.w, al, nx, ny, nz, Pr, Pi, Qr, Qi);
  }
  if (DEFER && MODE == kLagrange && __any_sync(0xffffffffu, emask != 0ull)) {
    // exact values where the lattice cell holds samples: the difference of
    // each such point pair enters P, Q linearly (R from the same float
    // operations as the loop above)
    while (emask) {
      const int bit = __ffsll((long long)emask) - 1;
      emask &= emask - 1;
      const int a = bit >> 3, b = bit & 7;
      const float4 al = g.pts32[(size_t)a * g.nt + p];
      const float4 be = g.pts32[(size_t)b * g.nt + q];
      const float ux = dc.x + al.x, uy = dc.y + al.y, uz = dc.z + al.z;
      const float rx = ux - be.x, ry = uy - be.y, rz = uz - be.z;
      const float R2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
      const float rs = rsqrtf(R2);
      const float R = R2 * rs;
      bool sl;
      const float2 fa = lookup32_fast<3>(T, R, &sl);
      const float2 fe = lookup32_slow<3>(T, R);
      const float gr = fe.x - fa.x, gi = fe.y - fa.y;
      const float kR = k32 * R, w2 = be.w * rs * rs;
      float Pr[3] = {0.f, 0.f, 0.f}, Pi[3] = {0.f, 0.f, 0.f}, Qr[3] = {0.f, 0.f, 0.f}, Qi[3] = {0.f, 0.f, 0.f};
      mfie_point(fmaf(-kR, gi, gr) * w2, fmaf(kR, gr, gi) * w2, rx, ry, rz, be, Pr, Pi, Qr, Qi);
      mfie_outer(S, al.w, al, nx, ny, nz, Pr, Pi, Qr, Qi);
    }
  }
  if (!ok) return;
  const int4 ep = g.tedge[p], eq = g.tedge[q];
  const int ecp[3] = {ep.x, ep.y, ep.z}, ecq[3] = {eq.x, eq.y, eq.z};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (!edge_valid(ecp[i])) continue;
    const float4 dp = g.geo32[3 * (size_t)p + i];  // delta_i, s_i l_i
    const float dS2r = dp.x * S.s2[0][0].s + dp.y * S.s2[1][0].s + dp.z * S.s2[2][0].s;
    const float dS2i = dp.x * S.s2[0][1].s + dp.y * S.s2[1][1].s + dp.z * S.s2[2][1].s;
    const float dS4r = dp.x * S.s4[0][0].s + dp.y * S.s4[1][0].s + dp.z * S.s4[2][0].s;
    const float dS4i = dp.x * S.s4[0][1].s + dp.y * S.s4[1][1].s + dp.z * S.s4[2][1].s;
    float2* zrow = Z + (int64_t)edge_of(ecp[i]) * ldz;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (!edge_valid(ecq[j])) continue;
      const float4 eq4 = g.geo32[3 * (size_t)q + j];  // eps_j, s_j l_j
      const float ne = nx * eq4.x + ny * eq4.y + nz * eq4.z;
      const float de = dp.x * eq4.x + dp.y * eq4.y + dp.z * eq4.z;
      const float S5er = S.s5[0][0].s * eq4.x + S.s5[1][0].s * eq4.y + S.s5[2][0].s * eq4.z;
      const float S5ei = S.s5[0][1].s * eq4.x + S.s5[1][1].s * eq4.y + S.s5[2][1].s * eq4.z;
      const float br = S.s1[0].s + dS2r + ne * (S.s3[0].s + dS4r) - S5er - de * S.s6[0].s;
      const float bi = S.s1[1].s + dS2i + ne * (S.s3[1].s + dS4i) - S5ei - de * S.s6[1].s;
      const float c = scale * dp.w * eq4.w;  // s_i l_i s_j l_j / (16 pi)
      atomicAdd(zrow + edge_of(ecq[j]), make_float2(c * br, c * bi));
    }
  }
}

// Work unit (p, source block): task = p * nb + block.
template <int M, int MODE, bool SMEM, bool DEFER>
__global__ void __launch_bounds__(SMEM ? 512 : kThreads) k_mfie_regular32(GeoView g, TabView tv, float kpi, float k32,
                                                                          float scale, float2* Z, int64_t ldz) {
  extern __shared__ __align__(16) unsigned char smem[];
  Tab32 T = tab32(tv);
  if (MODE == kLagrange && SMEM) {
    const int nl = tv.n_lat, nblob = (int)tv.blob_vec4();
    float4* sa = reinterpret_cast<float4*>(smem);
    float4* sb = sa + nl;
    float4* sblob = sb + nl;
    for (int i = threadIdx.x; i < nl; i += blockDim.x) {
      sa[i] = tv.lat_a[i];
      sb[i] = tv.lat_b[i];
    }
    for (int i = threadIdx.x; i < nblob; i += blockDim.x) sblob[i] = tv.lat_blob[i];
    __syncthreads();
    T.la = sa;
    T.lb = sb;
    tab32_blob(T, tv, sblob);
  }
  const int lane = threadIdx.x & 31;
  const int64_t nb = (g.nt + 31) / 32, ntask = (int64_t)g.nt * nb;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t task = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < ntask; task += nwarp) {
    const int p = (int)(task / nb), q0 = (int)(task % nb) * 32;
    mfie_task32<M, MODE, DEFER>(g, T, kpi, k32, scale, Z, ldz, p, q0, lane);
  }
}

// FP64 regular pairs (FP64 fills), lane = source triangle, same outer sums in FP64.
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_mfie_regular64(GeoView g, TabView tv, double k, double scale,
                                                             double2* Z, int64_t ldz) {
  const int lane = threadIdx.x & 31;
  const int64_t nb = (g.nt + 31) / 32, ntask = (int64_t)g.nt * nb;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t task = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < ntask; task += nwarp) {
    const int p = (int)(task / nb), q0 = (int)(task % nb) * 32;
    const int q = min(q0 + lane, g.nt - 1);
    const float4 cp32 = g.cen32[p], cq32 = g.cen32[q];
    const float3 dc32 = make_float3(cp32.x - cq32.x, cp32.y - cq32.y, cp32.z - cq32.z);
    if (!((q0 + lane < g.nt) && !pair_is_near(g, p, q, g.tvert[p], g.tvert[q], dc32))) continue;
    const double* cp = g.cen64 + 4 * (size_t)p;
    const double* cq = g.cen64 + 4 * (size_t)q;
    const double* np = g.frame64 + kFrame * (size_t)p;
    const double dx = cp[0] - cq[0], dy = cp[1] - cq[1], dz = cp[2] - cq[2];
    double s1[2] = {0, 0}, s2[3][2] = {}, s3[2] = {0, 0}, s4[3][2] = {}, s5[3][2] = {}, s6[2] = {0, 0};
    for (int a = 0; a < g.m; ++a) {
      const double* al = g.pts64 + 4 * ((size_t)a * g.nt + p);
      double P[3][2] = {}, Q[3][2] = {};
      for (int b = 0; b < g.m; ++b) {
        const double* be = g.pts64 + 4 * ((size_t)b * g.nt + q);
        const double r[3] = {dx + al[0] - be[0], dy + al[1] - be[1], dz + al[2] - be[2]};
        const double R = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        double gr, gi;
        if (MODE == kLagrange) {
          const double2 f = lookup64<3>(tv, R);
          gr = f.x;
          gi = f.y;
        } else {
          double sn, cs;
          sincos(k * R, &sn, &cs);
          gr = cs / R;
          gi = -sn / R;
        }
        const double w2 = be[3] / (R * R), kR = k * R;
        const double fr = (gr - kR * gi) * w2, fi = (gi + kR * gr) * w2;
        const double c[3] = {r[1] * be[2] - r[2] * be[1], r[2] * be[0] - r[0] * be[2], r[0] * be[1] - r[1] * be[0]};
        for (int x = 0; x < 3; ++x) {
          Q[x][0] += fr * r[x];
          Q[x][1] += fi * r[x];
          P[x][0] += fr * c[x];
          P[x][1] += fi * c[x];
        }
      }
      const double wa = al[3];
      for (int h = 0; h < 2; ++h) {
        const double NP[3] = {np[1] * P[2][h] - np[2] * P[1][h], np[2] * P[0][h] - np[0] * P[2][h],
                              np[0] * P[1][h] - np[1] * P[0][h]};
        const double nQ = np[0] * Q[0][h] + np[1] * Q[1][h] + np[2] * Q[2][h];
        s1[h] += wa * (al[0] * NP[0] + al[1] * NP[1] + al[2] * NP[2]);
        s3[h] += wa * (al[0] * Q[0][h] + al[1] * Q[1][h] + al[2] * Q[2][h]);
        s6[h] += wa * nQ;
        for (int x = 0; x < 3; ++x) {
          s2[x][h] += wa * NP[x];
          s4[x][h] += wa * Q[x][h];
          s5[x][h] += wa * nQ * al[x];
        }
      }
    }
    const int4 ep = g.tedge[p], eq = g.tedge[q];
    const int ecp[3] = {ep.x, ep.y, ep.z}, ecq[3] = {eq.x, eq.y, eq.z};
    for (int i = 0; i < 3; ++i) {
      if (!edge_valid(ecp[i])) continue;
      const double* dp = g.geo64 + 4 * (3 * (size_t)p + i);
      for (int j = 0; j < 3; ++j) {
        if (!edge_valid(ecq[j])) continue;
        const double* ej = g.geo64 + 4 * (3 * (size_t)q + j);
        const double ne = np[0] * ej[0] + np[1] * ej[1] + np[2] * ej[2];
        const double de = dp[0] * ej[0] + dp[1] * ej[1] + dp[2] * ej[2];
        double b[2];
        for (int h = 0; h < 2; ++h) {
          const double dS2 = dp[0] * s2[0][h] + dp[1] * s2[1][h] + dp[2] * s2[2][h];
          const double dS4 = dp[0] * s4[0][h] + dp[1] * s4[1][h] + dp[2] * s4[2][h];
          const double S5e = s5[0][h] * ej[0] + s5[1][h] * ej[1] + s5[2][h] * ej[2];
          b[h] = s1[h] + dS2 + ne * (s3[h] + dS4) - S5e - de * s6[h];
        }
        const double c = scale * dp[3] * ej[3];
        double* z = reinterpret_cast<double*>(Z + (int64_t)edge_of(ecp[i]) * ldz + edge_of(ecq[j]));
        atomicAdd(z, c * b[0]);
        atomicAdd(z + 1, c * b[1]);
      }
    }
  }
}

// 1/2 <f_m, f_n> on each triangle, closed form:
// int_T (r - v_i).(r - v_j) dS = A [delta_i.delta_j + (1/12) sum_k |delta_k|^2].
template <class Out>
__global__ void k_mfie_identity(GeoView g, Out* Z, int64_t ldz) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.nt) return;
  const int4 e = g.tedge[t];
  const int codes[3] = {e.x, e.y, e.z};
  const double area = g.cen64[4 * (size_t)t + 3];
  const double* d[3] = {g.geo64 + 4 * (3 * (size_t)t), g.geo64 + 4 * (3 * (size_t)t + 1),
                        g.geo64 + 4 * (3 * (size_t)t + 2)};
  double s = 0;
  for (int c = 0; c < 3; ++c) s += d[c][0] * d[c][0] + d[c][1] * d[c][1] + d[c][2] * d[c][2];
  for (int i = 0; i < 3; ++i) {
    if (!edge_valid(codes[i])) continue;
    for (int j = 0; j < 3; ++j) {
      if (!edge_valid(codes[j])) continue;
      const double gram = d[i][0] * d[j][0] + d[i][1] * d[j][1] + d[i][2] * d[j][2] + s / 12.0;
      const double v = d[i][3] * d[j][3] / (8.0 * area) * gram;  // 1/2 (s l / 2A)_i (s l / 2A)_j A gram
      Out* z = Z + (int64_t)edge_of(codes[i]) * ldz + edge_of(codes[j]);
      if constexpr (sizeof(Out) == 8) atomicAdd(reinterpret_cast<float*>(z), (float)v);
      else atomicAdd(reinterpret_cast<double*>(z), v);
    }
  }
}

// Near pairs (sharing a vertex, and the self pair), FP64: the inner integral
// T_j(r) = int_q grad G x (r' - v_j) dS' = -[h n x I_u + h (n x w) I_0 - I_u x w]
// with I_u = -(1/4 pi) sum_e m_e [log((l+ + R+)/(l- + R-)) + int_e (e^{-jkR} - 1)/R dl]
// (the surface-gradient theorem: Phi u = -(1/4 pi) grad'_s (e^{-jkR}/R)) and
// h I_0 = (1/4 pi) sum_e sgn(P0) int dphi (sgn(h) e^{-jkd} - h e^{-jkR_e}/R_e)
// (exact radial integral of Phi rho); h = 0 for the self pair (principal value).
// One near pair per group of G lanes, lane = test point; the 3x3 block is
// reduce-scattered over the group.
// The static part of h I_0 is the solid angle, -Omega / (4 pi), in closed form
// (Van Oosterom & Strackee, IEEE Trans. Biomed. Eng. 30 (1983) 125:
// tan(Omega / 2) = R1.(R2 x R3) / (R1 R2 R3 + (R1.R2) R3 + (R1.R3) R2 +
// (R2.R3) R1), R_i = v_i - r); the angles carry only the smooth remainder.
// MIXED (FP32 fills): the geometry and the closed-form static parts in FP64;
// the remainders e^{-jkR} - 1 on the edge lines and in the angle integrals
// sampled in FP32 (the FP32 Exp table), and the 3x3 block assembled from the
// integrals in FP32, as for the EFIE near pairs.
template <class Out, int G, bool MIXED>
__global__ void __launch_bounds__(128) k_mfie_near(GeoView g, TabView te, bool use_table, NearArgs A, Out* Z,
                                                   int64_t ldz) {
  const Tab32 te32 = tab32(te);
  const float lo32 = (float)te.r_lo, hi32 = (float)te.r_hi, kpi = (float)(A.k / kPi);
  const int64_t n_near = g.near_ptr[g.nt];
  const int sub = threadIdx.x & (G - 1);
  const unsigned gmask = ((1u << G) - 1u) << (threadIdx.x & (32 - G));
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t iters = (n_near + ngroups - 1) / ngroups;
  const double k = A.k, c4 = 1.0 / (4.0 * kPi);
  for (int64_t it = 0; it < iters; ++it) {
    const int64_t idx = g0 + it * ngroups;
    if (idx >= n_near) continue;  // uniform over the group
    const int p = g.near_row[idx], q = g.near_idx[idx];
    // MIXED: the 3x3 block is assembled from the FP64 integrals in FP32
    using CT = typename std::conditional<MIXED, C2f, C2>::type;
    using RT = typename std::conditional<MIXED, float, double>::type;
    CT acc[9];
    for (int u = 0; u < 9; ++u) acc[u] = CT{0, 0};
    if (sub < g.m) {
      const double* fr = g.frame64 + kFrame * (size_t)q;  // n, len, t, m of q
      const double* v = g.v64 + 9 * (size_t)q;
      const double* cp = g.cen64 + 4 * (size_t)p;
      const double* al = g.pts64 + 4 * ((size_t)sub * g.nt + p);
      const double r[3] = {cp[0] + al[0], cp[1] + al[1], cp[2] + al[2]};
      const double n[3] = {fr[0], fr[1], fr[2]};
      const double h = p == q ? 0.0 : n[0] * (r[0] - v[0]) + n[1] * (r[1] - v[1]) + n[2] * (r[2] - v[2]);
      const double d = fabs(h), sgh = h > 0 ? 1.0 : (h < 0 ? -1.0 : 0.0);
      const double rho0[3] = {r[0] - h * n[0], r[1] - h * n[1], r[2] - h * n[2]};
      const C2 ed = exp_mjkr(k, d, &te, use_table);
      double Iu[3][2] = {}, hI0[2] = {0, 0};
      for (int e = 0; e < 3; ++e) {
        const double* a = v + 3 * e;
        const double* b = v + 3 * ((e + 1) % 3);
        const double le = fr[3 + e];
        const double t[3] = {fr[6 + 3 * e], fr[7 + 3 * e], fr[8 + 3 * e]};
        const double m[3] = {fr[15 + 3 * e], fr[16 + 3 * e], fr[17 + 3 * e]};
        const double ar[3] = {a[0] - rho0[0], a[1] - rho0[1], a[2] - rho0[2]};
        const double P0 = ar[0] * m[0] + ar[1] * m[1] + ar[2] * m[2];
        const double lm = ar[0] * t[0] + ar[1] * t[1] + ar[2] * t[2];
        const double lp = lm + le;
        const double Rm = sqrt((r[0] - a[0]) * (r[0] - a[0]) + (r[1] - a[1]) * (r[1] - a[1]) + (r[2] - a[2]) * (r[2] - a[2]));
        const double Rp = sqrt((r[0] - b[0]) * (r[0] - b[0]) + (r[1] - b[1]) * (r[1] - b[1]) + (r[2] - b[2]) * (r[2] - b[2]));
        const double R02 = P0 * P0 + d * d;
        double ratio;
        if (lm >= 0) ratio = (lp + Rp) / (lm + Rm);
        else if (lp >= 0) ratio = (lp + Rp) * (Rm - lm) / R02;
        else ratio = (Rm - lm) / (Rp - lp);
        double lr = log(ratio), li = 0.0;
        if (MIXED) {
          const float* f32 = g.frame32 + kFrame32 * (size_t)q;
          const float ax = (float)(a[0] - r[0]), ay = (float)(a[1] - r[1]), az = (float)(a[2] - r[2]);
          const float tx = f32[3 + 3 * e], ty = f32[4 + 3 * e], tz = f32[5 + 3 * e], hl = 0.5f * f32[e];
          float sr = 0.f, si = 0.f;
          for (int i = 0; i < A.nl; ++i) {
            const float sp = hl * (A.fx_l[i] + 1.0f);
            const float x0 = fmaf(tx, sp, ax), x1 = fmaf(ty, sp, ay), x2 = fmaf(tz, sp, az);
            const float R = sqrtf(fmaf(x0, x0, fmaf(x1, x1, x2 * x2)));
            const float2 eR = exp32(kpi, R, te32, use_table, lo32, hi32);
            const float w = A.fw_l[i] * __frcp_rn(R);
            sr = fmaf(eR.x - 1.0f, w, sr);
            si = fmaf(eR.y, w, si);
          }
          lr += (double)(sr * hl);
          li += (double)(si * hl);
        } else {
          for (int i = 0; i < A.nl; ++i) {
            const double s = 0.5 * le * (A.gx_l[i] + 1.0);
            const double x0 = a[0] + t[0] * s - r[0], x1 = a[1] + t[1] * s - r[1], x2 = a[2] + t[2] * s - r[2];
            const double R = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
            const C2 eR = exp_mjkr(k, R, &te, use_table);
            const double w = 0.5 * le * A.gw_l[i] / R;
            lr += (eR.re - 1.0) * w;
            li += eR.im * w;
          }
        }
        for (int x = 0; x < 3; ++x) {
          Iu[x][0] -= m[x] * lr * c4;
          Iu[x][1] -= m[x] * li * c4;
        }
        if (fabs(P0) > 1e-12 * le && h != 0.0) {
          const double aP = fabs(P0);
          if (MIXED) {  // the remainder sgn(h)(e^{-jkd} - 1) - h (e^{-jkR_e} - 1)/R_e; the static part below
            const float aP32 = (float)aP, d32 = (float)d, h32 = (float)h, sg32 = (float)sgh;
            const float um = asinhf((float)lm / aP32), up = asinhf((float)lp / aP32);
            const float half = 0.5f * (up - um), mid = 0.5f * (up + um);
            const float2 ed32 = exp32(kpi, d32, te32, use_table, lo32, hi32);
            const float er0 = sg32 * (ed32.x - 1.0f), ei0 = sg32 * ed32.y;
            float sr = 0.f, si = 0.f;
            for (int i = 0; i < A.nphi; ++i) {
              const float u = fmaf(half, A.fx_phi[i], mid);
              const float E = expf(u);
              const float ch = 0.5f * (E + __frcp_rn(E));
              const float rho = aP32 * ch;
              const float Re = sqrtf(fmaf(rho, rho, d32 * d32));
              const float2 eR = exp32(kpi, Re, te32, use_table, lo32, hi32);
              const float w = A.fw_phi[i] * __frcp_rn(ch), hr = h32 * __frcp_rn(Re);
              sr = fmaf(fmaf(-hr, eR.x - 1.0f, er0), w, sr);
              si = fmaf(fmaf(-hr, eR.y, ei0), w, si);
            }
            const double sg = P0 > 0 ? (double)half * c4 : -(double)half * c4;
            hI0[0] += (double)sr * sg;
            hI0[1] += (double)si * sg;
          } else {
            const double um = asinh(lm / aP), up = asinh(lp / aP);
            const double half = 0.5 * (up - um), mid = 0.5 * (up + um);
            double sr = 0, si = 0;
            for (int i = 0; i < A.nphi; ++i) {
              const double u = mid + half * A.gx_phi[i];
              const double ch = cosh(u);
              const double Re = sqrt(aP * aP * ch * ch + d * d);
              const C2 eR = exp_mjkr(k, Re, &te, use_table);
              const double w = A.gw_phi[i] / ch;
              sr += (sgh * (ed.re - 1.0) - h * (eR.re - 1.0) / Re) * w;
              si += (sgh * ed.im - h * eR.im / Re) * w;
            }
            const double sg = P0 > 0 ? half * c4 : -half * c4;
            hI0[0] += sr * sg;
            hI0[1] += si * sg;
          }
        }
      }
      if (h != 0.0) {  // static part of h I_0: -Omega / (4 pi)
        double R1[3], R2[3], R3[3];
        for (int x = 0; x < 3; ++x) {
          R1[x] = v[x] - r[x];
          R2[x] = v[3 + x] - r[x];
          R3[x] = v[6 + x] - r[x];
        }
        const double n1 = sqrt(R1[0] * R1[0] + R1[1] * R1[1] + R1[2] * R1[2]);
        const double n2 = sqrt(R2[0] * R2[0] + R2[1] * R2[1] + R2[2] * R2[2]);
        const double n3 = sqrt(R3[0] * R3[0] + R3[1] * R3[1] + R3[2] * R3[2]);
        const double num = R1[0] * (R2[1] * R3[2] - R2[2] * R3[1]) + R1[1] * (R2[2] * R3[0] - R2[0] * R3[2]) +
                           R1[2] * (R2[0] * R3[1] - R2[1] * R3[0]);
        const double den = n1 * n2 * n3 + (R1[0] * R2[0] + R1[1] * R2[1] + R1[2] * R2[2]) * n3 +
                           (R1[0] * R3[0] + R1[1] * R3[1] + R1[2] * R3[2]) * n2 +
                           (R2[0] * R3[0] + R2[1] * R3[1] + R2[2] * R3[2]) * n1;
        hI0[0] -= 2.0 * atan2(num, den) * c4;
      }
      // n x I_u, and the assembly below in RT
      RT nIu[3][2], Iur[3][2], hI0r[2] = {(RT)hI0[0], (RT)hI0[1]};
      const RT nr[3] = {(RT)n[0], (RT)n[1], (RT)n[2]}, hr = (RT)h;
      for (int hh = 0; hh < 2; ++hh) {
        nIu[0][hh] = (RT)(n[1] * Iu[2][hh] - n[2] * Iu[1][hh]);
        nIu[1][hh] = (RT)(n[2] * Iu[0][hh] - n[0] * Iu[2][hh]);
        nIu[2][hh] = (RT)(n[0] * Iu[1][hh] - n[1] * Iu[0][hh]);
        for (int x = 0; x < 3; ++x) Iur[x][hh] = (RT)Iu[x][hh];
      }
      const double* np64 = g.frame64 + kFrame * (size_t)p;  // n_p
      const RT np[3] = {(RT)np64[0], (RT)np64[1], (RT)np64[2]};
      const RT wa = (RT)al[3];
      const double* vp = g.v64 + 9 * (size_t)p;
      for (int j = 0; j < 3; ++j) {
        const RT w[3] = {(RT)(rho0[0] - v[3 * j]), (RT)(rho0[1] - v[3 * j + 1]), (RT)(rho0[2] - v[3 * j + 2])};
        const RT nw[3] = {nr[1] * w[2] - nr[2] * w[1], nr[2] * w[0] - nr[0] * w[2], nr[0] * w[1] - nr[1] * w[0]};
        RT T[3][2];
        for (int hh = 0; hh < 2; ++hh) {
          const RT Iw[3] = {Iur[1][hh] * w[2] - Iur[2][hh] * w[1], Iur[2][hh] * w[0] - Iur[0][hh] * w[2],
                            Iur[0][hh] * w[1] - Iur[1][hh] * w[0]};  // I_u x w
          for (int x = 0; x < 3; ++x) T[x][hh] = -(hr * nIu[x][hh] + nw[x] * hI0r[hh] - Iw[x]);
        }
        // n_p x T_j
        RT NT[3][2];
        for (int hh = 0; hh < 2; ++hh) {
          NT[0][hh] = np[1] * T[2][hh] - np[2] * T[1][hh];
          NT[1][hh] = np[2] * T[0][hh] - np[0] * T[2][hh];
          NT[2][hh] = np[0] * T[1][hh] - np[1] * T[0][hh];
        }
        for (int i = 0; i < 3; ++i) {
          const RT f[3] = {(RT)(r[0] - vp[3 * i]), (RT)(r[1] - vp[3 * i + 1]), (RT)(r[2] - vp[3 * i + 2])};  // r_a - v_i
          acc[3 * i + j].re = -wa * (f[0] * NT[0][0] + f[1] * NT[1][0] + f[2] * NT[2][0]);
          acc[3 * i + j].im = -wa * (f[0] * NT[0][1] + f[1] * NT[1][1] + f[2] * NT[2][1]);
        }
      }
    }
    CT r5[5], r3[3];
    constexpr int L1 = G / 2, L2 = G / 4;
    rs_halve<9>(acc, r5, (sub & L1) != 0, L1, gmask);
    rs_halve<5>(r5, r3, (sub & L2) != 0, L2, gmask);
    int first = ((sub & L1) ? 5 : 0) + ((sub & L2) ? 3 : 0);
    int count = (sub & L1) ? ((sub & L2) ? 1 : 3) : ((sub & L2) ? 2 : 3);
    constexpr int NS = G == 8 ? 2 : 3;
    CT fin[NS];
    if constexpr (G == 8) {
      rs_halve<3>(r3, fin, (sub & 1) != 0, 1, gmask);
      const bool upper = (sub & 1) != 0;
      first += upper ? 2 : 0;
      count = upper ? max(count - 2, 0) : min(count, 2);
    } else {
      for (int u = 0; u < 3; ++u) fin[u] = r3[u];
    }
    const double inv_area_q = g.frame64[kFrame * (size_t)q + 24];
    const int4 ep = g.tedge[p], eq = g.tedge[q];
    for (int u = 0; u < NS; ++u) {
      if (u >= count) break;
      const int e = first + u, i = e / 3, j = e - 3 * (e / 3);
      const int ci = i == 0 ? ep.x : (i == 1 ? ep.y : ep.z), cj = j == 0 ? eq.x : (j == 1 ? eq.y : eq.z);
      if (!edge_valid(ci) || !edge_valid(cj)) continue;
      const double slp = g.geo64[4 * (3 * (size_t)p + i) + 3], slq = g.geo64[4 * (3 * (size_t)q + j) + 3];
      const double c = 0.25 * slp * slq * inv_area_q;  // A_p (s l / 2A)_i (s l / 2A)_j
      Out* z = Z + (int64_t)edge_of(ci) * ldz + edge_of(cj);
      if constexpr (sizeof(Out) == 8) {
        atomicAdd(reinterpret_cast<float2*>(z),
                  make_float2((float)(c * (double)fin[u].re), (float)(c * (double)fin[u].im)));
      } else {
        atomicAdd(reinterpret_cast<double*>(z), c * (double)fin[u].re);
        atomicAdd(reinterpret_cast<double*>(z) + 1, c * (double)fin[u].im);
      }
    }
  }
}

// ---------------------------------------------------------------- near-field sparse fill
// Z restricted to a sparsity pattern (the near field of fast solvers, the
// paper's "3mnNC" regime): the same pair computations, each block handed to a
// CsrSink that keeps the entries of the pattern. Regular pairs come from a
// work list of (test triangle, up to 32 source triangles) tasks; every ordered
// pair is listed (no symmetric second write).
struct SparseTask {
  int p;         // internal test triangle
  int n;         // source triangles in this task (1..32)
  int64_t off;   // first source triangle in the work list
};

template <int M, int MODE, bool SMEM, bool DEFER>
__global__ void __launch_bounds__(SMEM ? 512 : kThreads) k_sparse_regular32(GeoView g, TabView tv, float kpi,
                                                                            float scale, float inv_k2,
                                                                            const SparseTask* __restrict__ tasks,
                                                                            int64_t ntask, const int32_t* __restrict__ widx,
                                                                            CsrSink<float2> sink) {
  extern __shared__ __align__(16) unsigned char smem[];
  Tab32 T = tab32(tv);
  if (MODE != kDirect && SMEM) {
    const int nl = tv.n_lat, nblob = (int)tv.blob_vec4();
    float4* sa = reinterpret_cast<float4*>(smem);
    float4* sb = sa + nl;
    float4* sblob = sb + nl;
    for (int i = threadIdx.x; i < nl; i += blockDim.x) {
      sa[i] = tv.lat_a[i];
      sb[i] = tv.lat_b[i];
    }
    for (int i = threadIdx.x; i < nblob; i += blockDim.x) sblob[i] = tv.lat_blob[i];
    __syncthreads();
    T.la = sa;
    T.lb = sb;
    tab32_blob(T, tv, sblob);
  }
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntask; t += nwarp) {
    const SparseTask tk = tasks[t];
    const bool ok = lane < tk.n;
    const int q = ok ? widx[tk.off + lane] : tk.p;
    regular_pair32<M, MODE, DEFER>(g, T, kpi, scale, inv_k2, tk.p, q, ok, sink);
  }
}

// Near pairs of the mesh's near list into the pattern.
template <bool MIXED, int G>
__global__ void __launch_bounds__(128) k_sparse_near(GeoView g, TabView te, bool use_table, NearArgs A,
                                                     CsrSink<float2> sink) {
  const Tab32 te32 = tab32(te);
  const float lo32 = (float)te.r_lo, hi32 = (float)te.r_hi;
  const int64_t n_near = g.near_ptr[g.nt];
  const int sub = threadIdx.x & (G - 1);
  const unsigned gmask = ((1u << G) - 1u) << (threadIdx.x & (32 - G));
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t iters = (n_near + ngroups - 1) / ngroups;
  for (int64_t it = 0; it < iters; ++it) {
    const int64_t idx = g0 + it * ngroups;
    near_pair<MIXED, G>(g, te, te32, lo32, hi32, use_table, A, KScal{A.k, A.scale, A.inv_k2, 1.0 / A.k}, sink, idx,
                        idx < n_near, sub, gmask);
  }
}

// ---------------------------------------------------------------- windowed table
// Tables larger than shared memory: the fill runs over tiles of 32 test
// triangles x 512 source triangles (consecutive in the Morton order, so
// spatially compact); the bounding spheres of the two sets bound every point
// distance of the tile, and only the lattice records of that distance window
// are staged into shared memory (sub-cells and the interval records of cells
// holding samples stay in global memory). A tile whose window does not fit
// reads the table through L1.
constexpr int kTileQBlocks = 16;
constexpr int kWinBytes = 200 * 1024;

// One warp per block of 32 triangles (lane = triangle): mean of the
// centroids, then the largest centroid distance plus point radius.
__global__ void k_block_spheres(GeoView g, float4* bsph) {
  const int b = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  const int nb = (g.nt + 31) / 32;
  if (b >= nb) return;  // uniform over the warp
  const int t0 = 32 * b, n = min(32, g.nt - t0), t = t0 + min(lane, n - 1);
  const double x = g.cen64[4 * (size_t)t], y = g.cen64[4 * (size_t)t + 1], z = g.cen64[4 * (size_t)t + 2];
  double cx = lane < n ? x : 0.0, cy = lane < n ? y : 0.0, cz = lane < n ? z : 0.0;
  for (int off = 16; off > 0; off >>= 1) {
    cx += __shfl_xor_sync(0xffffffffu, cx, off);
    cy += __shfl_xor_sync(0xffffffffu, cy, off);
    cz += __shfl_xor_sync(0xffffffffu, cz, off);
  }
  cx /= n;
  cy /= n;
  cz /= n;
  const double dx = x - cx, dy = y - cy, dz = z - cz;
  double r = sqrt(dx * dx + dy * dy + dz * dz) + (double)g.rad32[t];
  for (int off = 16; off > 0; off >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, off));
  if (lane == 0) bsph[b] = make_float4((float)cx, (float)cy, (float)cz, (float)(r * (1.0 + 1e-6)));
}

template <int M>
__global__ void __launch_bounds__(512) k_fill_regular32_win(GeoView g, TabView tv, const float4* __restrict__ bsph,
                                                            float kpi, float scale, float inv_k2, float2* Z,
                                                            int64_t ldz) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int win[5];  // c_lo, c_hi, unused, unused, fits
  const int nb = (g.nt + 31) / 32;
  const int nqg = (nb + kTileQBlocks - 1) / kTileQBlocks;
  const int64_t ntiles = (int64_t)nb * nqg;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const Tab32 G = tab32(tv);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int bp = (int)(tile / nqg), bqg = (int)(tile % nqg);
    const int qb1 = min((bqg + 1) * kTileQBlocks, nb);
    if (qb1 <= bp) continue;  // only source blocks bq >= bp (one evaluation per unordered pair)
    const int qb0 = max(bqg * kTileQBlocks, bp);
    if (threadIdx.x == 0) {
      const float4 P = bsph[bp];
      float qx = 0.f, qy = 0.f, qz = 0.f;
      for (int b = qb0; b < qb1; ++b) {
        qx += bsph[b].x;
        qy += bsph[b].y;
        qz += bsph[b].z;
      }
      const float inv_n = 1.f / (float)(qb1 - qb0);
      qx *= inv_n;
      qy *= inv_n;
      qz *= inv_n;
      float rq = 0.f;
      for (int b = qb0; b < qb1; ++b) {
        const float dx = bsph[b].x - qx, dy = bsph[b].y - qy, dz = bsph[b].z - qz;
        rq = fmaxf(rq, sqrtf(dx * dx + dy * dy + dz * dz) + bsph[b].w);
      }
      const float dx = P.x - qx, dy = P.y - qy, dz = P.z - qz;
      const float D = sqrtf(dx * dx + dy * dy + dz * dz);
      const float mag = fmaxf(fmaxf(fabsf(P.x), fabsf(P.y)), fmaxf(fabsf(P.z), fmaxf(fmaxf(fabsf(qx), fabsf(qy)), fabsf(qz))));
      const float slack = 1e-5f * (D + P.w + rq + mag);
      const float lo = D - P.w - rq - slack, hi = D + P.w + rq + slack;
      const int n_lat = tv.n_lat;
      const int c_lo = max(lat_pos(G, lo * G.xscale).i - 2, 0);
      const int c_hi = min(lat_pos(G, hi * G.xscale).i + 2, n_lat - 1);
      win[0] = c_lo;
      win[1] = c_hi;
      win[4] = (int64_t)(c_hi - c_lo + 1) * 32 <= kWinBytes;
    }
    __syncthreads();
    Tab32 T = G;
    if (win[4]) {
      const int c_lo = win[0], c_hi = win[1];
      const int nc = c_hi - c_lo + 1;
      float4* sa = reinterpret_cast<float4*>(smem);
      float4* sb = sa + nc;
      for (int i = threadIdx.x; i < nc; i += blockDim.x) {
        sa[i] = G.la[c_lo + i];
        sb[i] = G.lb[c_lo + i];
      }
      __syncthreads();
      T.la = sa - c_lo;
      T.lb = sb - c_lo;
      T.vmin = kLatMagic + (float)c_lo;
      T.vmax = kLatMagic + (float)c_hi;
    }
    const int ntask = 32 * (qb1 - qb0);
    for (int task = warp; task < ntask; task += nw) {
      const int p = bp * 32 + task / (qb1 - qb0);
      const int q0 = (qb0 + task % (qb1 - qb0)) * 32;
      if (p < g.nt) regular_task32<M, kLagrange, false>(g, T, kpi, scale, inv_k2, DenseUpper{Z, ldz}, p, q0, lane);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- adjoint
// Backward of L with respect to the vertex coordinates and k, given the
// upstream gZ = dL/dconj(Z) (dL = Re sum conj(gZ) dZ). Per regular pair,
//   S = sum_ij h_ij Bt_ij,  h_ij = j kappa s_i l_i s_j l_j conj(gZ_ij),
// Bt_ij the bracket of the forward block, so S = sum_ab w_a w_b F(R_ab) K_ab
// with K_ab = A0 + Aa . alpha_a + Ab . beta_b + Aab alpha_a . beta_b. Green
// values F are recomputed from the table; F' = -(jk + 1/R) F, dF/dk = -jR F.
// Gradients reach the vertices through the points (R and the offsets
// alpha, beta), the edge vectors delta_i = c_p - v_i, eps_j = c_q - v_j, the
// signed edge lengths and k. Classification, range and table samples are held
// fixed. Triangle gradients accumulate in FP64 per triangle (9 values).
struct BaryF {
  float l[kMaxRule][3];
};

__device__ __forceinline__ float re_mul(float ar, float ai, float br, float bi) { return ar * br - ai * bi; }
__device__ __forceinline__ float im_mul(float ar, float ai, float br, float bi) { return ar * bi + ai * br; }

template <int M, bool TABLE>
__device__ __forceinline__ void regular_adjoint_task32(const GeoView& g, const Tab32& T, float k, float kappa,
                                                       float inv_k2, const BaryF& bw, const float2* __restrict__ gZ,
                                                       int64_t ldg, double* dtri, double* dkacc, int p, int q0,
                                                       int lane) {
  const int q = min(q0 + lane, g.nt - 1);
  const float4 cp = g.cen32[p], cq = g.cen32[q];
  const float3 dc = make_float3(cp.x - cq.x, cp.y - cq.y, cp.z - cq.z);
  const bool ok = (q0 + lane < g.nt) && q > p && !pair_is_near(g, p, q, g.tvert[p], g.tvert[q], dc);
  if (!__any_sync(0xffffffffu, ok)) return;
  const int4 ep = g.tedge[p], eq = g.tedge[q];
  const int ecp[3] = {ep.x, ep.y, ep.z}, ecq[3] = {eq.x, eq.y, eq.z};
  float4 gp[3], gq[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    gp[i] = g.geo32[3 * (size_t)p + i];
    gq[i] = g.geo32[3 * (size_t)q + i];
  }
  // The block value B_ij feeds Z[m][n] and Z[n][m], so its cotangent is
  // g = gZ[m][n] + gZ[n][m]; h_ij = j kappa sigma_i sigma_j conj(g) = c (Im g + j Re g)
  auto h_of = [&](int i, int j, float* hr, float* hi) {
    *hr = *hi = 0.f;
    if (ok && edge_valid(ecp[i]) && edge_valid(ecq[j])) {
      const float2 z1 = gZ[(int64_t)edge_of(ecp[i]) * ldg + edge_of(ecq[j])];
      const float2 z2 = gZ[(int64_t)edge_of(ecq[j]) * ldg + edge_of(ecp[i])];
      const float2 z = make_float2(z1.x + z2.x, z1.y + z2.y);
      const float c = kappa * gp[i].w * gq[j].w;
      *hr = c * z.y;
      *hi = c * z.x;
    }
  };
  float Aabr = 0.f, Aabi = 0.f, A0r = 0.f, A0i = 0.f, Aar[3] = {0.f, 0.f, 0.f}, Aai[3] = {0.f, 0.f, 0.f};
  float Abr[3] = {0.f, 0.f, 0.f}, Abi[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float hr, hi;
      h_of(i, j, &hr, &hi);
      Aabr += 0.25f * hr;
      Aabi += 0.25f * hi;
      const float de = gp[i].x * gq[j].x + gp[i].y * gq[j].y + gp[i].z * gq[j].z;
      A0r += hr * (0.25f * de - inv_k2);
      A0i += hi * (0.25f * de - inv_k2);
      const float ej[3] = {gq[j].x, gq[j].y, gq[j].z}, di[3] = {gp[i].x, gp[i].y, gp[i].z};
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        Aar[x] += 0.25f * hr * ej[x];
        Aai[x] += 0.25f * hi * ej[x];
        Abr[x] += 0.25f * hr * di[x];
        Abi[x] += 0.25f * hi * di[x];
      }
    }
  float4 beta[M];
#pragma unroll
  for (int b = 0; b < M; ++b) beta[b] = g.pts32[(size_t)b * g.nt + q];
  float gqb[M][3], gB[M][3];
#pragma unroll
  for (int b = 0; b < M; ++b)
#pragma unroll
    for (int x = 0; x < 3; ++x) gqb[b][x] = gB[b][x] = 0.f;
  float dp[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  float M0r = 0.f, M0i = 0.f, Mar[3] = {0.f, 0.f, 0.f}, Mai[3] = {0.f, 0.f, 0.f}, Mbr[3] = {0.f, 0.f, 0.f},
        Mbi[3] = {0.f, 0.f, 0.f}, Mabr = 0.f, Mabi = 0.f, dkF = 0.f;
#pragma unroll 1
  for (int a = 0; a < M; ++a) {
    const float4 al = g.pts32[(size_t)a * g.nt + p];
    const float alv[3] = {al.x, al.y, al.z};
    const float ux = dc.x + al.x, uy = dc.y + al.y, uz = dc.z + al.z;
    // K_ab = Ka + Kb . beta_b with Ka = A0 + Aa . alpha_a, Kb = Ab + Aab alpha_a
    const float Kar = A0r + Aar[0] * al.x + Aar[1] * al.y + Aar[2] * al.z;
    const float Kai = A0i + Aai[0] * al.x + Aai[1] * al.y + Aai[2] * al.z;
    float Kbr[3], Kbi[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      Kbr[x] = Abr[x] + Aabr * alv[x];
      Kbi[x] = Abi[x] + Aabi * alv[x];
    }
    float ga[3] = {0.f, 0.f, 0.f}, gA[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int b = 0; b < M; ++b) {
      const float rx = ux - beta[b].x, ry = uy - beta[b].y, rz = uz - beta[b].z;
      const float R2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
      const float rs = rsqrtf(R2);
      const float R = R2 * rs;
      float Fr, Fi;
      if (TABLE) {
        const float2 f = lookup32<3>(T, R);
        Fr = f.x;
        Fi = f.y;
      } else {
        float sn, cs;
        sincospif(R * k * 0.318309886183790672f, &sn, &cs);
        Fr = cs * rs;
        Fi = -sn * rs;
      }
      const float ww = al.w * beta[b].w;
      const float bv[3] = {beta[b].x, beta[b].y, beta[b].z};
      const float Kr = Kar + Kbr[0] * bv[0] + Kbr[1] * bv[1] + Kbr[2] * bv[2];
      const float Ki = Kai + Kbi[0] * bv[0] + Kbi[1] * bv[1] + Kbi[2] * bv[2];
      // F' = -(jk + 1/R) F
      const float Fpr = -Fr * rs + k * Fi, Fpi = -Fi * rs - k * Fr;
      const float t1 = ww * re_mul(Kr, Ki, Fpr, Fpi) * rs;  // times r/R below
      const float gR[3] = {t1 * rx, t1 * ry, t1 * rz};
      const float wFr = ww * Fr, wFi = ww * Fi;
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        ga[x] += gR[x];
        gqb[b][x] -= gR[x];
        gA[x] += re_mul(wFr, wFi, Aar[x] + Aabr * bv[x], Aai[x] + Aabi * bv[x]);
        gB[b][x] += re_mul(wFr, wFi, Kbr[x], Kbi[x]);
      }
      dkF += R * im_mul(Kr, Ki, wFr, wFi);
      const float ab = alv[0] * bv[0] + alv[1] * bv[1] + alv[2] * bv[2];
      M0r += wFr;
      M0i += wFi;
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        Mar[x] += alv[x] * wFr;
        Mai[x] += alv[x] * wFi;
        Mbr[x] += bv[x] * wFr;
        Mbi[x] += bv[x] * wFi;
      }
      Mabr += ab * wFr;
      Mabi += ab * wFi;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float lc = bw.l[a][c];
#pragma unroll
      for (int x = 0; x < 3; ++x) dp[c][x] += lc * ga[x] + (lc - (1.f / 3.f)) * gA[x];
    }
  }
  float dq[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
  for (int b = 0; b < M; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float lc = bw.l[b][c];
#pragma unroll
      for (int x = 0; x < 3; ++x) dq[c][x] += lc * gqb[b][x] + (lc - (1.f / 3.f)) * gB[b][x];
    }
  // through delta_i, eps_j, the signed lengths and k explicitly
  float dd[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  float de_[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  float dsp[3] = {0.f, 0.f, 0.f}, dsq[3] = {0.f, 0.f, 0.f}, dkx = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float hr, hi;
      h_of(i, j, &hr, &hi);
      if (hr == 0.f && hi == 0.f) continue;
      const float di[3] = {gp[i].x, gp[i].y, gp[i].z}, ej[3] = {gq[j].x, gq[j].y, gq[j].z};
      const float de = di[0] * ej[0] + di[1] * ej[1] + di[2] * ej[2];
      const float eMar = ej[0] * Mar[0] + ej[1] * Mar[1] + ej[2] * Mar[2];
      const float eMai = ej[0] * Mai[0] + ej[1] * Mai[1] + ej[2] * Mai[2];
      const float dMbr = di[0] * Mbr[0] + di[1] * Mbr[1] + di[2] * Mbr[2];
      const float dMbi = di[0] * Mbi[0] + di[1] * Mbi[1] + di[2] * Mbi[2];
      const float Btr = 0.25f * (Mabr + eMar + dMbr + de * M0r) - M0r * inv_k2;
      const float Bti = 0.25f * (Mabi + eMai + dMbi + de * M0i) - M0i * inv_k2;
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        dd[i][x] += 0.25f * re_mul(hr, hi, Mbr[x] + ej[x] * M0r, Mbi[x] + ej[x] * M0i);
        de_[j][x] += 0.25f * re_mul(hr, hi, Mar[x] + di[x] * M0r, Mai[x] + di[x] * M0i);
      }
      const float hB = re_mul(hr, hi, Btr, Bti);
      dsp[i] += hB / gp[i].w;
      dsq[j] += hB / gq[j].w;
      dkx += hB / k + 2.f * inv_k2 / k * re_mul(hr, hi, M0r, M0i);
    }
  // delta_i = c - v_i; sigma_i = s_i |v_{i+1} - v_{i+2}|, v_{i+1} - v_{i+2} = delta_{i+2} - delta_{i+1}
  auto edge_terms = [&](float dv[3][3], const float4 gv[3], const float dd_[3][3], const float ds[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int x = 0; x < 3; ++x) dv[c][x] += (dd_[0][x] + dd_[1][x] + dd_[2][x]) * (1.f / 3.f) - dd_[c][x];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (gv[i].w == 0.f) continue;
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
      const float s = ds[i] / gv[i].w;
      const float e[3] = {gv[i2].x - gv[i1].x, gv[i2].y - gv[i1].y, gv[i2].z - gv[i1].z};
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        dv[i1][x] += s * e[x];
        dv[i2][x] -= s * e[x];
      }
    }
  };
  edge_terms(dp, gp, dd, dsp);
  edge_terms(dq, gq, de_, dsq);
  float dkl = ok ? dkF + dkx : 0.f;
  if (!ok) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int x = 0; x < 3; ++x) dp[c][x] = dq[c][x] = 0.f;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      float v = dp[c][x];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) atomicAdd(&dtri[9 * (size_t)p + 3 * c + x], (double)v);
      if (ok) atomicAdd(&dtri[9 * (size_t)q + 3 * c + x], (double)dq[c][x]);
    }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) dkl += __shfl_xor_sync(0xffffffffu, dkl, off);
  if (lane == 0) atomicAdd(dkacc, (double)dkl);
}

template <int M, bool TABLE>
__global__ void __launch_bounds__(256) k_adjoint_regular32(GeoView g, TabView tv, float k, float kappa, float inv_k2,
                                                           BaryF bw, const float2* __restrict__ gZ, int64_t ldg,
                                                           double* dtri, double* dkacc) {
  const Tab32 T = tab32(tv);
  const int lane = threadIdx.x & 31;
  const int64_t ntask = regular_units(g.nt);
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t task = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < ntask; task += nwarp) {
    int p, q0;
    if (sym_task(task, g.nt, &p, &q0))
      regular_adjoint_task32<M, TABLE>(g, T, k, kappa, inv_k2, bw, gZ, ldg, dtri, dkacc, p, q0, lane);
  }
}

// ---- near pairs: forward-mode dual numbers (one direction per thread group)
struct D1 {
  double v, d;
};
__device__ __forceinline__ D1 operator+(D1 a, D1 b) { return D1{a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ D1 operator-(D1 a, D1 b) { return D1{a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ D1 operator-(D1 a) { return D1{-a.v, -a.d}; }
__device__ __forceinline__ D1 operator*(D1 a, D1 b) { return D1{a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ D1 operator/(D1 a, D1 b) {
  const double iv = 1.0 / b.v;
  return D1{a.v * iv, (a.d - a.v * iv * b.d) * iv};
}
__device__ __forceinline__ D1 operator*(D1 a, double s) { return D1{a.v * s, a.d * s}; }
__device__ __forceinline__ D1 operator*(double s, D1 a) { return D1{a.v * s, a.d * s}; }
__device__ __forceinline__ D1 operator+(D1 a, double s) { return D1{a.v + s, a.d}; }
__device__ __forceinline__ D1 operator-(D1 a, double s) { return D1{a.v - s, a.d}; }
__device__ __forceinline__ D1 dsqrt(D1 a) {
  const double r = sqrt(a.v);
  return D1{r, a.d / (2.0 * r)};
}
__device__ __forceinline__ D1 dlog(D1 a) { return D1{log(a.v), a.d / a.v}; }
__device__ __forceinline__ D1 dasinh(D1 a) { return D1{asinh(a.v), a.d / sqrt(1.0 + a.v * a.v)}; }
__device__ __forceinline__ D1 dcosh(D1 a) { return D1{cosh(a.v), sinh(a.v) * a.d}; }
__device__ __forceinline__ D1 dabs(D1 a) { return a.v < 0 ? -a : a; }

struct DC {  // complex over D1
  D1 re, im;
};
__device__ __forceinline__ DC operator+(DC a, DC b) { return DC{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ DC operator-(DC a, DC b) { return DC{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ DC operator*(DC a, D1 s) { return DC{a.re * s, a.im * s}; }

// e^{-jkR} with its derivative: from the Exp table when R is in range (the
// derivative then uses -j e^{-jkR} d(kR) with the table value), else direct.
__device__ __forceinline__ DC exp_mjkr_d(D1 k, D1 R, const TabView* te, bool use_table) {
  const D1 ph = k * R;
  double c, s;
  if (use_table && R.v >= te->r_lo && R.v <= te->r_hi) {
    const double2 f = lookup64<1>(*te, R.v);
    c = f.x;
    s = -f.y;
  } else {
    sincos(ph.v, &s, &c);
  }
  // d/dph (c - j s) = -s - j c
  return DC{D1{c, -s * ph.d}, D1{-s, -c * ph.d}};
}

struct V3D {
  D1 x, y, z;
};
__device__ __forceinline__ V3D vsub(V3D a, V3D b) { return V3D{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ D1 vdot(V3D a, V3D b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3D vcross(V3D a, V3D b) {
  return V3D{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ V3D vscale(V3D a, D1 s) { return V3D{a.x * s, a.y * s, a.z * s}; }

// The near-pair inner integrals of inner_integrals() in dual numbers.
__device__ void inner_integrals_d(const V3D& r, const V3D v[3], const NearArgs& A, D1 k, const TabView* te,
                                  bool use_table, DC* I0, DC I1[3], V3D* rho0_out) {
  V3D n = vcross(vsub(v[1], v[0]), vsub(v[2], v[0]));
  const D1 inv = D1{1.0, 0.0} / dsqrt(vdot(n, n));
  n = vscale(n, inv);
  const D1 h = vdot(n, vsub(r, v[0]));
  const D1 d = dabs(h);
  const V3D rho0 = vsub(r, vscale(n, h));
  *rho0_out = rho0;
  const DC ed = exp_mjkr_d(k, d, te, use_table);
  DC sacc{D1{0, 0}, D1{0, 0}};
  DC vacc[3] = {{D1{0, 0}, D1{0, 0}}, {D1{0, 0}, D1{0, 0}}, {D1{0, 0}, D1{0, 0}}};
  D1 vst[3] = {D1{0, 0}, D1{0, 0}, D1{0, 0}};
  for (int e = 0; e < 3; ++e) {
    const V3D a = v[e], b = v[(e + 1) % 3];
    V3D t = vsub(b, a);
    const D1 len = dsqrt(vdot(t, t));
    t = vscale(t, D1{1.0, 0.0} / len);
    const V3D mh = vcross(t, n);
    const V3D ar = vsub(a, rho0), br = vsub(b, rho0);
    const D1 P0 = vdot(ar, mh), lm = vdot(ar, t), lp = vdot(br, t);
    if (fabs(P0.v) > 1e-12 * len.v) {
      const D1 aP = dabs(P0);
      const D1 um = dasinh(lm / aP), up = dasinh(lp / aP);
      const D1 half = (up - um) * 0.5, mid = (up + um) * 0.5;
      DC sec{D1{0, 0}, D1{0, 0}};
      for (int i = 0; i < A.nphi; ++i) {
        const D1 u = mid + half * A.gx_phi[i];
        const D1 ch = dcosh(u);
        const D1 rho = aP * ch;
        const D1 Re = dsqrt(rho * rho + d * d);
        const DC eR = exp_mjkr_d(k, Re, te, use_table);
        sec = sec + (ed - eR) * (D1{A.gw_phi[i], 0.0} / ch);
      }
      sec = sec * (P0.v > 0 ? half : -half);
      sacc = sacc + sec;
    }
    DC li{D1{0, 0}, D1{0, 0}};
    for (int i = 0; i < A.nl; ++i) {
      const D1 sp = len * (0.5 * (A.gx_l[i] + 1.0));
      const V3D x = vsub(V3D{a.x + t.x * sp, a.y + t.y * sp, a.z + t.z * sp}, r);
      const D1 R = dsqrt(vdot(x, x));
      const DC eR = exp_mjkr_d(k, R, te, use_table);
      li = li + DC{eR.re - 1.0, eR.im + k * R} * D1{A.gw_l[i], 0.0};
    }
    li = li * (len * 0.5);
    const D1 R02 = P0 * P0 + d * d;
    const D1 Rm = dsqrt(lm * lm + R02), Rp = dsqrt(lp * lp + R02);
    D1 st = (lp * Rp - lm * Rm) * 0.5;
    if (R02.v > 0) {
      const D1 fp = lp.v >= 0 ? lp + Rp : R02 / (Rp - lp);
      const D1 fm = lm.v >= 0 ? lm + Rm : R02 / (Rm - lm);
      st = st + R02 * (dlog(fp) - dlog(fm)) * 0.5;
    }
    const D1 mhv[3] = {mh.x, mh.y, mh.z};
    for (int x = 0; x < 3; ++x) {
      vacc[x] = vacc[x] + li * mhv[x];
      vst[x] = vst[x] + mhv[x] * st;
    }
  }
  const double c4 = 1.0 / (4.0 * kPi);
  const D1 ik = D1{1.0, 0.0} / k;
  // I0 = (-j/k) s / (4 pi); I1 = ((j/k) v + v_static) / (4 pi)
  I0->re = sacc.im * ik * c4;
  I0->im = -(sacc.re * ik) * c4;
  for (int x = 0; x < 3; ++x) {
    I1[x].re = (vst[x] - vacc[x].im * ik) * c4;
    I1[x].im = vacc[x].re * ik * c4;
  }
}

// FP32 dual numbers for the edge sampling of the mixed-precision near pairs.
struct F1 {
  float v, d;
};
__device__ __forceinline__ F1 operator+(F1 a, F1 b) { return F1{a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ F1 operator-(F1 a, F1 b) { return F1{a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ F1 operator*(F1 a, F1 b) { return F1{a.v * b.v, fmaf(a.d, b.v, a.v * b.d)}; }
__device__ __forceinline__ F1 operator*(F1 a, float s) { return F1{a.v * s, a.d * s}; }
__device__ __forceinline__ F1 f1(D1 a) { return F1{(float)a.v, (float)a.d}; }
__device__ __forceinline__ F1 fsqrt1(F1 a) {
  const float r = sqrtf(a.v);
  return F1{r, a.d * 0.5f * __frcp_rn(r)};
}

// e^{-jk R} and its derivative in FP32 (table value when R is in range).
__device__ __forceinline__ void exp_mjkr_f(F1 k, F1 R, const Tab32& te, bool use_table, float lo, float hi,
                                           F1* re, F1* im) {
  const F1 ph = k * R;
  float c, s;
  if (use_table && R.v >= lo && R.v <= hi) {
    const float2 f = lookup32<1>(te, R.v);
    c = f.x;
    s = -f.y;
  } else {
    sincospif(ph.v * 0.318309886183790672f, &s, &c);
  }
  *re = F1{c, -s * ph.d};
  *im = F1{-s, -c * ph.d};
}

// inner_integrals_d with the sampling of each edge in FP32 duals (geometry,
// closed-form static part and accumulation in FP64 duals).
__device__ void inner_integrals_d_mixed(const V3D& r, const V3D v[3], const NearArgs& A, D1 k, const Tab32& te,
                                        bool use_table, float lo, float hi, DC* I0, DC I1[3], V3D* rho0_out) {
  V3D n = vcross(vsub(v[1], v[0]), vsub(v[2], v[0]));
  const D1 inv = D1{1.0, 0.0} / dsqrt(vdot(n, n));
  n = vscale(n, inv);
  const D1 h = vdot(n, vsub(r, v[0]));
  const D1 d = dabs(h);
  const V3D rho0 = vsub(r, vscale(n, h));
  *rho0_out = rho0;
  const F1 k32 = f1(k), d32 = f1(d);
  F1 edr, edi;
  exp_mjkr_f(k32, d32, te, use_table, lo, hi, &edr, &edi);
  // |r - v_c|: R at the ends of the two edges that meet at v_c (scalars, so
  // that the edge loop can pick them without a local-memory array)
  const V3D dv0 = vsub(v[0], r), dv1 = vsub(v[1], r), dv2 = vsub(v[2], r);
  const D1 Rv0 = dsqrt(vdot(dv0, dv0)), Rv1 = dsqrt(vdot(dv1, dv1)), Rv2 = dsqrt(vdot(dv2, dv2));
  DC sacc{D1{0, 0}, D1{0, 0}};
  DC vacc[3] = {{D1{0, 0}, D1{0, 0}}, {D1{0, 0}, D1{0, 0}}, {D1{0, 0}, D1{0, 0}}};
  D1 vst[3] = {D1{0, 0}, D1{0, 0}, D1{0, 0}};
  for (int e = 0; e < 3; ++e) {
    const V3D a = v[e], b = v[(e + 1) % 3];
    V3D t = vsub(b, a);
    const D1 len = dsqrt(vdot(t, t));
    t = vscale(t, D1{1.0, 0.0} / len);
    const V3D mh = vcross(t, n);
    const V3D ar = vsub(a, rho0);
    const D1 P0 = vdot(ar, mh), lm = vdot(ar, t), lp = lm + len;
    if (fabs(P0.v) > 1e-12 * len.v) {
      const D1 aP = dabs(P0);
      const D1 iaP = D1{1.0, 0.0} / aP;
      const F1 x1 = f1(lm * iaP), x2 = f1(lp * iaP);
      const F1 um = F1{asinhf(x1.v), x1.d * rsqrtf(1.f + x1.v * x1.v)};
      const F1 up = F1{asinhf(x2.v), x2.d * rsqrtf(1.f + x2.v * x2.v)};
      const F1 half = (up - um) * 0.5f, mid = (up + um) * 0.5f;
      const F1 aP32 = f1(aP);
      F1 cr{0.f, 0.f}, ci{0.f, 0.f};
      for (int i = 0; i < A.nphi; ++i) {
        const F1 u = mid + half * A.fx_phi[i];
        const float E = expf(u.v), iE = __frcp_rn(E);
        const F1 ch{0.5f * (E + iE), 0.5f * (E - iE) * u.d};
        const F1 rho = aP32 * ch;
        const F1 Re = fsqrt1(rho * rho + d32 * d32);
        F1 er, ei;
        exp_mjkr_f(k32, Re, te, use_table, lo, hi, &er, &ei);
        const float ich = __frcp_rn(ch.v);
        const F1 wt{A.fw_phi[i] * ich, -A.fw_phi[i] * ich * ich * ch.d};
        cr = cr + (edr - er) * wt;
        ci = ci + (edi - ei) * wt;
      }
      const D1 hd{(double)half.v, (double)half.d};
      const D1 sg = P0.v > 0 ? hd : -hd;
      sacc = DC{sacc.re + D1{(double)cr.v, (double)cr.d} * sg, sacc.im + D1{(double)ci.v, (double)ci.d} * sg};
    }
    const V3D a_r = vsub(a, r);
    const F1 ax = f1(a_r.x), ay = f1(a_r.y), az = f1(a_r.z), tx = f1(t.x), ty = f1(t.y), tz = f1(t.z);
    const F1 hl = f1(len * 0.5);
    F1 lr{0.f, 0.f}, li{0.f, 0.f};
    for (int i = 0; i < A.nl; ++i) {
      const F1 sp = hl * (A.fx_l[i] + 1.0f);
      const F1 x0 = ax + tx * sp, x1v = ay + ty * sp, x2v = az + tz * sp;
      const F1 R = fsqrt1(x0 * x0 + x1v * x1v + x2v * x2v);
      F1 er, ei;
      exp_mjkr_f(k32, R, te, use_table, lo, hi, &er, &ei);
      lr = lr + F1{er.v - 1.f, er.d} * A.fw_l[i];
      li = li + (ei + k32 * R) * A.fw_l[i];
    }
    const D1 lrd = D1{(double)lr.v, (double)lr.d} * (len * 0.5), lid = D1{(double)li.v, (double)li.d} * (len * 0.5);
    const D1 R02 = P0 * P0 + d * d;
    const D1 Rm = e == 0 ? Rv0 : (e == 1 ? Rv1 : Rv2), Rp = e == 0 ? Rv1 : (e == 1 ? Rv2 : Rv0);
    D1 st = (lp * Rp - lm * Rm) * 0.5;
    if (R02.v > 0) {
      const D1 fp = lp.v >= 0 ? lp + Rp : R02 / (Rp - lp);
      const D1 fm = lm.v >= 0 ? lm + Rm : R02 / (Rm - lm);
      st = st + R02 * dlog(fp / fm) * 0.5;
    }
    const D1 mhv[3] = {mh.x, mh.y, mh.z};
    for (int x = 0; x < 3; ++x) {
      vacc[x] = DC{vacc[x].re + lrd * mhv[x], vacc[x].im + lid * mhv[x]};
      vst[x] = vst[x] + mhv[x] * st;
    }
  }
  const double c4 = 1.0 / (4.0 * kPi);
  const D1 ik = D1{1.0, 0.0} / k;
  I0->re = sacc.im * ik * c4;
  I0->im = -(sacc.re * ik) * c4;
  for (int x = 0; x < 3; ++x) {
    I1[x].re = (vst[x] - vacc[x].im * ik) * c4;
    I1[x].im = vacc[x].re * ik * c4;
  }
}

// One (near pair, direction) on 8 lanes, one test point per lane. Direction
// 0..8: p's vertex coordinates, 9..17: q's, 18: k. The derivative of the
// pair's share of L is reduced over the points and added to dtri / dk.
// ---- near pairs, reverse mode (mixed precision): one pass per (near pair,
// test point) gives the derivatives along all 19 directions. The values are
// those of inner_integrals_mixed (FP64 frames, projection, static closed form
// and sums; FP32 samples of e^{-jkR}); the adjoints follow the same split,
// FP32 inside the sampled loops, FP64 elsewhere. Sample derivatives use
// dE/dR = -jk E and dE/dk = -jR E on the interpolated E.
__device__ __forceinline__ void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Adds d(contribution to L)/d(vertices of p), d/d(vertices of q), d/dk of
// one test point a of near pair (p, q): L = sum_ij Re(conj(gZ_ij) dZ_ij).
__device__ void near_point_adjoint(const double vp[3][3], const double vq[3][3], const float lb[3], double wa,
                                   const NearArgs& A, double k, double eta, const Tab32& te, bool use_table, float lo,
                                   float hi, const int ecp[3], const int ecq[3], const float2* __restrict__ gZ,
                                   int64_t ldg, double gp[3][3], double gq[3][3], double* gk) {
  const float kpi = (float)(k / kPi), k32 = (float)k;
  double r[3];
  for (int x = 0; x < 3; ++x) r[x] = (double)lb[0] * vp[0][x] + (double)lb[1] * vp[1][x] + (double)lb[2] * vp[2][x];
  // ---- source frame
  double e1[3], e2[3], nn[3], n[3];
  for (int x = 0; x < 3; ++x) {
    e1[x] = vq[1][x] - vq[0][x];
    e2[x] = vq[2][x] - vq[0][x];
  }
  cross3(e1, e2, nn);
  const double Ln = sqrt(dot3(nn, nn)), iL = 1.0 / Ln;
  for (int x = 0; x < 3; ++x) n[x] = nn[x] * iL;
  double len[3], ilen[3], t[3][3], m[3][3];
  for (int e = 0; e < 3; ++e) {
    const int e2i = e == 2 ? 0 : e + 1;
    double tt[3] = {vq[e2i][0] - vq[e][0], vq[e2i][1] - vq[e][1], vq[e2i][2] - vq[e][2]};
    len[e] = sqrt(dot3(tt, tt));
    ilen[e] = 1.0 / len[e];
    for (int x = 0; x < 3; ++x) t[e][x] = tt[x] * ilen[e];
    cross3(t[e], n, m[e]);
  }
  // ---- projection, vertex distances, e^{-jkd}
  double rv0[3] = {r[0] - vq[0][0], r[1] - vq[0][1], r[2] - vq[0][2]};
  const double h = dot3(n, rv0), d = fabs(h);
  double rho0[3];
  for (int x = 0; x < 3; ++x) rho0[x] = r[x] - h * n[x];
  double Rv[3];
  for (int c = 0; c < 3; ++c) {
    const double dx = vq[c][0] - r[0], dy = vq[c][1] - r[1], dz = vq[c][2] - r[2];
    Rv[c] = sqrt(dx * dx + dy * dy + dz * dz);
  }
  const float d32 = (float)d;
  const float2 ed = exp32(kpi, d32, te, use_table, lo, hi);
  // ---- forward: the per-edge sums
  double sre = 0, sim = 0, vre[3] = {0, 0, 0}, vim[3] = {0, 0, 0}, vst[3] = {0, 0, 0};
  for (int e = 0; e < 3; ++e) {
    const double* a = vq[e];
    const double ar[3] = {a[0] - rho0[0], a[1] - rho0[1], a[2] - rho0[2]};
    const double P0 = dot3(ar, m[e]), lm = dot3(ar, t[e]), lp = lm + len[e];
    if (fabs(P0) > 1e-12 * len[e]) {
      const float aP32 = (float)fabs(P0);
      const float um = asinhf((float)lm / aP32), up = asinhf((float)lp / aP32);
      const float half = 0.5f * (up - um), mid = 0.5f * (up + um);
      float cr = 0.f, ci = 0.f;
      for (int i = 0; i < A.nphi; ++i) {
        const float u = fmaf(half, A.fx_phi[i], mid);
        const float E = expf(u);
        const float ch = 0.5f * (E + __frcp_rn(E));
        const float rho = aP32 * ch;
        const float Re = sqrtf(fmaf(rho, rho, d32 * d32));
        const float2 eR = exp32(kpi, Re, te, use_table, lo, hi);
        const float wt = A.fw_phi[i] * __frcp_rn(ch);
        cr = fmaf(ed.x - eR.x, wt, cr);
        ci = fmaf(ed.y - eR.y, wt, ci);
      }
      const double sg = P0 > 0 ? (double)half : -(double)half;
      sre += (double)cr * sg;
      sim += (double)ci * sg;
    }
    const float ax = (float)(a[0] - r[0]), ay = (float)(a[1] - r[1]), az = (float)(a[2] - r[2]);
    const float tx = (float)t[e][0], ty = (float)t[e][1], tz = (float)t[e][2];
    const float hl = 0.5f * (float)len[e];
    float lr = 0.f, li = 0.f;
    for (int i = 0; i < A.nl; ++i) {
      const float sp = hl * (A.fx_l[i] + 1.0f);
      const float x0 = fmaf(tx, sp, ax), x1 = fmaf(ty, sp, ay), x2 = fmaf(tz, sp, az);
      const float R = sqrtf(fmaf(x0, x0, fmaf(x1, x1, x2 * x2)));
      const float2 eR = exp32(kpi, R, te, use_table, lo, hi);
      lr = fmaf(eR.x - 1.0f, A.fw_l[i], lr);
      li = fmaf(fmaf(k32, R, eR.y), A.fw_l[i], li);
    }
    const double lrd = (double)lr * (0.5 * len[e]), lid = (double)li * (0.5 * len[e]);
    const double R02 = P0 * P0 + d * d;
    const double Rm = Rv[e], Rp = Rv[e == 2 ? 0 : e + 1];
    double st = 0.5 * (lp * Rp - lm * Rm);
    if (R02 > 0) {
      const double fp = lp >= 0 ? lp + Rp : R02 / (Rp - lp);
      const double fm = lm >= 0 ? lm + Rm : R02 / (Rm - lm);
      st += 0.5 * R02 * log(fp / fm);
    }
    for (int x = 0; x < 3; ++x) {
      vre[x] += m[e][x] * lrd;
      vim[x] += m[e][x] * lid;
      vst[x] += m[e][x] * st;
    }
  }
  const double c4 = 1.0 / (4.0 * kPi), ik = 1.0 / k;
  const double I0r = sim * ik * c4, I0i = -sre * ik * c4;
  double I1r[3], I1i[3];
  for (int x = 0; x < 3; ++x) {
    I1r[x] = (vst[x] - vim[x] * ik) * c4;
    I1i[x] = vre[x] * ik * c4;
  }
  // ---- assembly: values and adjoints of I0, I1, rho0, r, p's vertices, L = |nn|, k
  double bI0r = 0, bI0i = 0, bI1r[3] = {0, 0, 0}, bI1i[3] = {0, 0, 0}, brho[3] = {0, 0, 0}, br[3] = {0, 0, 0};
  double bk = 0, bik2 = 0, bA = 0;
  const double Aq = 0.5 * Ln, ik2 = ik * ik, iAq = 1.0 / Aq;
  // per source edge j: s_j l_j, s_j / l_j and rho0 - v_j (reciprocals once: the
  // FP64 divide costs a dozen FP64 operations); the adjoint of s_j l_j is
  // summed over i and applied once
  double slj[3], sjl[3], dvj[3][3], bslj[3] = {0, 0, 0};
  for (int j = 0; j < 3; ++j) {
    const int j1 = j == 2 ? 0 : j + 1, j2 = j1 == 2 ? 0 : j1 + 1;
    const double ej[3] = {vq[j2][0] - vq[j1][0], vq[j2][1] - vq[j1][1], vq[j2][2] - vq[j1][2]};
    const double lj = sqrt(dot3(ej, ej)), sj = (ecq[j] & 1) ? -1.0 : 1.0;
    slj[j] = sj * lj;
    sjl[j] = sj / lj;
    for (int x = 0; x < 3; ++x) dvj[j][x] = rho0[x] - vq[j][x];
  }
  const double kewa = k * eta * wa * iAq;
  for (int i = 0; i < 3; ++i) {
    if (!edge_valid(ecp[i])) continue;
    const int i1 = i == 2 ? 0 : i + 1, i2 = i1 == 2 ? 0 : i1 + 1;
    const double ei[3] = {vp[i2][0] - vp[i1][0], vp[i2][1] - vp[i1][1], vp[i2][2] - vp[i1][2]};
    const double li_ = sqrt(dot3(ei, ei)), si = (ecp[i] & 1) ? -1.0 : 1.0, sli = si * li_;
    const double f[3] = {r[0] - vp[i][0], r[1] - vp[i][1], r[2] - vp[i][2]};
    double bf[3] = {0, 0, 0}, bcsum = 0;
    for (int j = 0; j < 3; ++j) {
      if (!edge_valid(ecq[j])) continue;
      const double* dv = dvj[j];
      double Jr[3], Ji[3];
      for (int x = 0; x < 3; ++x) {
        Jr[x] = I1r[x] + dv[x] * I0r;
        Ji[x] = I1i[x] + dv[x] * I0i;
      }
      const double tr = 0.25 * dot3(f, Jr) - I0r * ik2, ti = 0.25 * dot3(f, Ji) - I0i * ik2;
      const double c = kewa * sli * slj[j];
      const float2 gz = gZ[(int64_t)edge_of(ecp[i]) * ldg + edge_of(ecq[j])];
      // L = gz.x (-c ti) + gz.y (c tr)
      const double btr = (double)gz.y * c, bti = -(double)gz.x * c;
      const double bc = (double)gz.y * tr - (double)gz.x * ti;
      double bdv[3];
      for (int x = 0; x < 3; ++x) {
        bf[x] += 0.25 * (btr * Jr[x] + bti * Ji[x]);
        const double bJr = 0.25 * btr * f[x], bJi = 0.25 * bti * f[x];
        bI1r[x] += bJr;
        bI1i[x] += bJi;
        bdv[x] = bJr * I0r + bJi * I0i;
        bI0r += bJr * dv[x];
        bI0i += bJi * dv[x];
        brho[x] += bdv[x];
        gq[j][x] -= bdv[x];
      }
      bI0r -= btr * ik2;
      bI0i -= bti * ik2;
      bik2 -= btr * I0r + bti * I0i;
      // c = k eta wa sl_i sl_j / A_q: bc c is the adjoint of log c, shared by its factors
      const double bcc = bc * c;
      bcsum += bcc;
      bslj[j] += bcc;  // becomes the adjoint of s_j l_j below
    }
    // log c = log k + log sl_i + log sl_j - log A_q + const
    bk += bcsum * ik;
    bA -= bcsum * iAq;
    const double gsi = bcsum / sli * (si / li_);
    for (int x = 0; x < 3; ++x) {
      br[x] += bf[x];
      gp[i][x] -= bf[x];
      const double g = gsi * ei[x];
      gp[i2][x] += g;
      gp[i1][x] -= g;
    }
  }
  for (int j = 0; j < 3; ++j) {
    if (!edge_valid(ecq[j])) continue;
    const int j1 = j == 2 ? 0 : j + 1, j2 = j1 == 2 ? 0 : j1 + 1;
    // d(s_j l_j)/d v_{j2} = s_j e_j / l_j; the adjoint of s_j l_j is (sum bc c) / (s_j l_j)
    const double g0 = bslj[j] / slj[j] * sjl[j];
    for (int x = 0; x < 3; ++x) {
      const double g = g0 * (vq[j2][x] - vq[j1][x]);
      gq[j2][x] += g;
      gq[j1][x] -= g;
    }
  }
  bk -= 2.0 * bik2 * ik2 * ik;
  // ---- reverse of I0, I1 = f(sre, sim, vre, vim, vst, k)
  const double bsim = bI0r * ik * c4, bsre = -bI0i * ik * c4;
  double bvst[3], bvim[3], bvre[3];
  double bik = c4 * (bI0r * sim - bI0i * sre);
  for (int x = 0; x < 3; ++x) {
    bvst[x] = bI1r[x] * c4;
    bvim[x] = -bI1r[x] * ik * c4;
    bvre[x] = bI1i[x] * ik * c4;
    bik += c4 * (-bI1r[x] * vim[x] + bI1i[x] * vre[x]);
  }
  bk -= bik * ik * ik;
  // ---- reverse of the edges (recomputing their forward values)
  double bd = 0, bRv[3] = {0, 0, 0}, bt[3][3], bm[3][3], blen[3];
  float bedr = 0.f, bedi = 0.f;
  for (int e = 0; e < 3; ++e) {
    const int en = e == 2 ? 0 : e + 1;
    const double* a = vq[e];
    const double ar[3] = {a[0] - rho0[0], a[1] - rho0[1], a[2] - rho0[2]};
    const double P0 = dot3(ar, m[e]), lm = dot3(ar, t[e]), lp = lm + len[e];
    double bP0 = 0, blm = 0, blp = 0, bR02 = 0;
    blen[e] = 0;
    // line integral: values then adjoints
    const float ax = (float)(a[0] - r[0]), ay = (float)(a[1] - r[1]), az = (float)(a[2] - r[2]);
    const float tx = (float)t[e][0], ty = (float)t[e][1], tz = (float)t[e][2];
    const float hl = 0.5f * (float)len[e];
    float lr = 0.f, li = 0.f;
    for (int i = 0; i < A.nl; ++i) {
      const float sp = hl * (A.fx_l[i] + 1.0f);
      const float x0 = fmaf(tx, sp, ax), x1 = fmaf(ty, sp, ay), x2 = fmaf(tz, sp, az);
      const float R = sqrtf(fmaf(x0, x0, fmaf(x1, x1, x2 * x2)));
      const float2 eR = exp32(kpi, R, te, use_table, lo, hi);
      lr = fmaf(eR.x - 1.0f, A.fw_l[i], lr);
      li = fmaf(fmaf(k32, R, eR.y), A.fw_l[i], li);
    }
    const double blrd = dot3(bvre, m[e]), blid = dot3(bvim, m[e]);
    const double lrd = (double)lr * (0.5 * len[e]), lid = (double)li * (0.5 * len[e]);
    const float blr = (float)(blrd * 0.5 * len[e]), bli = (float)(blid * 0.5 * len[e]);
    blen[e] += 0.5 * (blrd * (double)lr + blid * (double)li);
    float bax = 0.f, bay = 0.f, baz = 0.f, btx = 0.f, bty = 0.f, btz = 0.f, bhl = 0.f, bk32 = 0.f;
    for (int i = 0; i < A.nl; ++i) {
      const float sp = hl * (A.fx_l[i] + 1.0f);
      const float x0 = fmaf(tx, sp, ax), x1 = fmaf(ty, sp, ay), x2 = fmaf(tz, sp, az);
      const float R = sqrtf(fmaf(x0, x0, fmaf(x1, x1, x2 * x2)));
      const float2 eR = exp32(kpi, R, te, use_table, lo, hi);
      // lr += w (Er - 1); li += w (Ei + k R); dEr/dph = Ei, dEi/dph = -Er, ph = k R
      const float bEr = blr * A.fw_l[i], bEi = bli * A.fw_l[i];
      const float bph = bEr * eR.y - bEi * eR.x;
      const float bR = bph * k32 + bEi * k32;
      bk32 += bph * R + bEi * R;
      const float iR = __frcp_rn(R);
      const float gx = bR * x0 * iR, gy = bR * x1 * iR, gz_ = bR * x2 * iR;
      bax += gx;
      bay += gy;
      baz += gz_;
      btx += gx * sp;
      bty += gy * sp;
      btz += gz_ * sp;
      bhl += (gx * tx + gy * ty + gz_ * tz) * (A.fx_l[i] + 1.0f);
    }
    bk += (double)bk32;
    blen[e] += 0.5 * (double)bhl;
    // (a - r): a = v_e
    gq[e][0] += bax;
    gq[e][1] += bay;
    gq[e][2] += baz;
    br[0] -= bax;
    br[1] -= bay;
    br[2] -= baz;
    bt[e][0] = btx;
    bt[e][1] = bty;
    bt[e][2] = btz;
    // static part
    const double bst = dot3(bvst, m[e]);
    for (int x = 0; x < 3; ++x) bm[e][x] = bvre[x] * lrd + bvim[x] * lid;
    const double R02 = P0 * P0 + d * d;
    const double Rm = Rv[e], Rp = Rv[en];
    double st = 0.5 * (lp * Rp - lm * Rm);
    blp += 0.5 * Rp * bst;
    blm -= 0.5 * Rm * bst;
    double bRp = 0.5 * lp * bst, bRm = -0.5 * lm * bst;
    if (R02 > 0) {
      const double fp = lp >= 0 ? lp + Rp : R02 / (Rp - lp);
      const double fm = lm >= 0 ? lm + Rm : R02 / (Rm - lm);
      const double Lg = log(fp / fm);
      st += 0.5 * R02 * Lg;
      bR02 += 0.5 * Lg * bst;
      const double bL = 0.5 * R02 * bst;  // adjoint of log fp - log fm
      if (lp >= 0) {
        const double g = bL / fp;
        blp += g;
        bRp += g;
      } else {  // log R02 - log(Rp - lp)
        const double g = bL / (Rp - lp);
        bR02 += bL / R02;
        bRp -= g;
        blp += g;
      }
      if (lm >= 0) {
        const double g = bL / fm;
        blm -= g;
        bRm -= g;
      } else {
        const double g = bL / (Rm - lm);
        bR02 -= bL / R02;
        bRm += g;
        blm -= g;
      }
    }
    for (int x = 0; x < 3; ++x) bm[e][x] += bvst[x] * st;
    bRv[e] += bRm;
    bRv[en] += bRp;
    // angular part
    if (fabs(P0) > 1e-12 * len[e]) {
      const float aP32 = (float)fabs(P0);
      const float zm = (float)lm / aP32, zp = (float)lp / aP32;
      const float um = asinhf(zm), up = asinhf(zp);
      const float half = 0.5f * (up - um), mid = 0.5f * (up + um);
      float cr = 0.f, ci = 0.f;
      for (int i = 0; i < A.nphi; ++i) {
        const float u = fmaf(half, A.fx_phi[i], mid);
        const float E = expf(u);
        const float ch = 0.5f * (E + __frcp_rn(E));
        const float rho = aP32 * ch;
        const float Re = sqrtf(fmaf(rho, rho, d32 * d32));
        const float2 eR = exp32(kpi, Re, te, use_table, lo, hi);
        const float wt = A.fw_phi[i] * __frcp_rn(ch);
        cr = fmaf(ed.x - eR.x, wt, cr);
        ci = fmaf(ed.y - eR.y, wt, ci);
      }
      const double sgn = P0 > 0 ? 1.0 : -1.0, sg = sgn * (double)half;
      const float bcr = (float)(bsre * sg), bci = (float)(bsim * sg);
      float bhalf = (float)(sgn * (bsre * (double)cr + bsim * (double)ci)), bmid = 0.f, baP = 0.f, bd32 = 0.f;
      float bk32a = 0.f;
      for (int i = 0; i < A.nphi; ++i) {
        const float u = fmaf(half, A.fx_phi[i], mid);
        const float E = expf(u), iE = __frcp_rn(E);
        const float ch = 0.5f * (E + iE), sh = 0.5f * (E - iE);
        const float rho = aP32 * ch;
        const float Re = sqrtf(fmaf(rho, rho, d32 * d32));
        const float2 eR = exp32(kpi, Re, te, use_table, lo, hi);
        const float wt = A.fw_phi[i] * __frcp_rn(ch);
        bedr += bcr * wt;
        bedi += bci * wt;
        const float bEr = -bcr * wt, bEi = -bci * wt;
        const float bph = bEr * eR.y - bEi * eR.x;
        const float bRe = bph * k32;
        bk32a += bph * Re;
        const float bwt = bcr * (ed.x - eR.x) + bci * (ed.y - eR.y);
        float bch = -bwt * wt / ch;
        const float iRe = __frcp_rn(Re);
        const float brho = bRe * rho * iRe;
        bd32 += bRe * d32 * iRe;
        baP += brho * ch;
        bch += brho * aP32;
        const float bu = bch * sh;
        bhalf += bu * A.fx_phi[i];
        bmid += bu;
      }
      bk += (double)bk32a;
      bd += (double)bd32;
      const float bup = 0.5f * (bhalf + bmid), bum = 0.5f * (bmid - bhalf);
      const float bzp = bup * rsqrtf(1.f + zp * zp), bzm = bum * rsqrtf(1.f + zm * zm);
      blp += (double)(bzp / aP32);
      blm += (double)(bzm / aP32);
      baP -= (bzp * zp + bzm * zm) / aP32;
      bP0 += sgn * (double)baP;
    }
    bP0 += 2.0 * P0 * bR02;
    bd += 2.0 * d * bR02;
    blm += blp;
    blen[e] += blp;
    for (int x = 0; x < 3; ++x) {
      const double bar = bP0 * m[e][x] + blm * t[e][x];
      bm[e][x] += bP0 * ar[x];
      bt[e][x] += blm * ar[x];
      gq[e][x] += bar;
      brho[x] -= bar;
    }
  }
  // e^{-jkd}
  {
    const float bph = bedr * ed.y - bedi * ed.x;
    bd += (double)(bph * k32);
    bk += (double)(bph * d32);
  }
  // vertex distances
  for (int c = 0; c < 3; ++c) {
    const double gr = bRv[c] / Rv[c];
    for (int x = 0; x < 3; ++x) {
      const double g = gr * (vq[c][x] - r[x]);
      gq[c][x] += g;
      br[x] -= g;
    }
  }
  // d = |h|, rho0 = r - h n, h = n . (r - v0)
  double bh = (h >= 0 ? 1.0 : -1.0) * bd, bn[3];
  for (int x = 0; x < 3; ++x) {
    br[x] += brho[x];
    bh -= brho[x] * n[x];
    bn[x] = -h * brho[x];
  }
  for (int x = 0; x < 3; ++x) {
    bn[x] += bh * rv0[x];
    br[x] += bh * n[x];
    gq[0][x] -= bh * n[x];
  }
  // frame: m_e = t_e x n, t_e = tt / |tt|, n = nn / |nn|, A_q = |nn| / 2
  for (int e = 0; e < 3; ++e) {
    const int en = e == 2 ? 0 : e + 1;
    double c1[3], c2[3];
    cross3(n, bm[e], c1);  // d/dt of (t x n) . bm
    cross3(bm[e], t[e], c2);  // d/dn
    for (int x = 0; x < 3; ++x) {
      bt[e][x] += c1[x];
      bn[x] += c2[x];
    }
    const double tb = dot3(t[e], bt[e]);
    for (int x = 0; x < 3; ++x) {
      const double btt = (bt[e][x] - t[e][x] * tb) * ilen[e] + blen[e] * t[e][x];
      gq[en][x] += btt;
      gq[e][x] -= btt;
    }
  }
  {
    const double nb = dot3(n, bn);
    double bnn[3];
    for (int x = 0; x < 3; ++x) bnn[x] = (bn[x] - n[x] * nb) * iL + 0.5 * bA * n[x];
    double be1[3], be2[3];
    cross3(e2, bnn, be1);
    cross3(bnn, e1, be2);
    for (int x = 0; x < 3; ++x) {
      gq[1][x] += be1[x];
      gq[2][x] += be2[x];
      gq[0][x] -= be1[x] + be2[x];
    }
  }
  // r = sum_c l_c v_c
  for (int c = 0; c < 3; ++c)
    for (int x = 0; x < 3; ++x) gp[c][x] += (double)lb[c] * br[x];
  *gk += bk;
}

// One near pair per group of G lanes, lane = test point; all 19 derivatives
// in one reverse pass, reduced over the group.
template <int G>
__global__ void __launch_bounds__(128) k_adjoint_near_rev(GeoView g, TabView te, bool use_table, NearArgs A, double k,
                                                          double eta, BaryF bw, const float2* __restrict__ gZ,
                                                          int64_t ldg, double* dtri, double* dkacc) {
  const Tab32 te32 = tab32(te);
  const float lo32 = (float)te.r_lo, hi32 = (float)te.r_hi;
  const int64_t n_near = g.near_ptr[g.nt];
  const int sub = threadIdx.x & (G - 1);
  const unsigned gmask = ((1u << G) - 1u) << (threadIdx.x & (32 - G));
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const int64_t iters = (n_near + ngroups - 1) / ngroups;  // same trip count in every group of a warp
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  for (int64_t itn = 0; itn < iters; ++itn) {
    const int64_t idx = g0 + itn * ngroups;
    if (idx >= n_near) continue;  // uniform over the group
    const int p = g.near_row[idx], q = g.near_idx[idx];
    double gp[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, gq[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, gk = 0;
    if (sub < g.m) {
      double vp[3][3], vq[3][3];
      for (int c = 0; c < 3; ++c)
        for (int x = 0; x < 3; ++x) {
          vp[c][x] = g.v64[9 * (size_t)p + 3 * c + x];
          vq[c][x] = g.v64[9 * (size_t)q + 3 * c + x];
        }
      const int4 ep = g.tedge[p], eq = g.tedge[q];
      const int ecp[3] = {ep.x, ep.y, ep.z}, ecq[3] = {eq.x, eq.y, eq.z};
      const double wa = g.pts64[4 * ((size_t)sub * g.nt + p) + 3];
      near_point_adjoint(vp, vq, bw.l[sub], wa, A, k, eta, te32, use_table, lo32, hi32, ecp, ecq, gZ, ldg, gp, gq,
                         &gk);
    }
    for (int off = 1; off < G; off <<= 1) {
      for (int c = 0; c < 3; ++c)
        for (int x = 0; x < 3; ++x) {
          gp[c][x] += __shfl_xor_sync(gmask, gp[c][x], off);
          gq[c][x] += __shfl_xor_sync(gmask, gq[c][x], off);
        }
      gk += __shfl_xor_sync(gmask, gk, off);
    }
    if (sub == 0) {
      for (int c = 0; c < 3; ++c)
        for (int x = 0; x < 3; ++x) {
          atomicAdd(&dtri[9 * (size_t)p + 3 * c + x], gp[c][x]);
          atomicAdd(&dtri[9 * (size_t)q + 3 * c + x], gq[c][x]);
        }
      atomicAdd(dkacc, gk);
    }
  }
}

// One (near pair, derivative direction) per group of G lanes (lane = test
// point): directions 0..8 = p's vertex coordinates, 9..17 = q's, 18 = k.
template <bool MIXED, int G>
__global__ void __launch_bounds__(128) k_adjoint_near(GeoView g, TabView te, bool use_table, NearArgs A, double k,
                                                      double eta, BaryF bw, const float2* __restrict__ gZ, int64_t ldg,
                                                      double* dtri, double* dkacc) {
  const Tab32 te32 = tab32(te);
  const float lo32 = (float)te.r_lo, hi32 = (float)te.r_hi;
  const int64_t n_near = g.near_ptr[g.nt];
  const int64_t njobs = n_near * 19;
  const int sub = threadIdx.x & (G - 1);
  const unsigned gmask = ((1u << G) - 1u) << (threadIdx.x & (32 - G));
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  for (int64_t job = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; job < njobs; job += ngroups) {
    const int64_t idx = job / 19;
    const int dir = (int)(job % 19);
    const int p = g.near_row[idx], q = g.near_idx[idx];
    double dL = 0.0;
    if (sub < g.m) {
      V3D vp[3], vq[3];
      for (int c = 0; c < 3; ++c) {
        const double* xp = g.v64 + 9 * (size_t)p + 3 * c;
        const double* xq = g.v64 + 9 * (size_t)q + 3 * c;
        vp[c] = V3D{D1{xp[0], dir == 3 * c ? 1.0 : 0.0}, D1{xp[1], dir == 3 * c + 1 ? 1.0 : 0.0},
                    D1{xp[2], dir == 3 * c + 2 ? 1.0 : 0.0}};
        vq[c] = V3D{D1{xq[0], dir == 9 + 3 * c ? 1.0 : 0.0}, D1{xq[1], dir == 10 + 3 * c ? 1.0 : 0.0},
                    D1{xq[2], dir == 11 + 3 * c ? 1.0 : 0.0}};
      }
      const D1 kd{k, dir == 18 ? 1.0 : 0.0};
      // test point r_a = sum_c l_ac v_c, weight w_a
      const double* al = g.pts64 + 4 * ((size_t)sub * g.nt + p);
      const double wa = al[3];
      V3D ra{D1{0, 0}, D1{0, 0}, D1{0, 0}};
      for (int c = 0; c < 3; ++c) {
        const double l = (double)bw.l[sub][c];
        ra = V3D{ra.x + vp[c].x * l, ra.y + vp[c].y * l, ra.z + vp[c].z * l};
      }
      DC I0, I1[3];
      V3D rho0;
      if (MIXED) inner_integrals_d_mixed(ra, vq, A, kd, te32, use_table, lo32, hi32, &I0, I1, &rho0);
      else inner_integrals_d(ra, vq, A, kd, &te, use_table, &I0, I1, &rho0);
      const V3D nq = vcross(vsub(vq[1], vq[0]), vsub(vq[2], vq[0]));
      const D1 area_q = dsqrt(vdot(nq, nq)) * 0.5;
      const int4 ep = g.tedge[p], eq = g.tedge[q];
      const int ecp[3] = {ep.x, ep.y, ep.z}, ecq[3] = {eq.x, eq.y, eq.z};
      const D1 inv_k2 = D1{1.0, 0.0} / (kd * kd);
      for (int i = 0; i < 3; ++i) {
        if (!edge_valid(ecp[i])) continue;
        const V3D e_i = vsub(vp[(i + 2) % 3], vp[(i + 1) % 3]);
        const D1 sl_i = dsqrt(vdot(e_i, e_i)) * ((ecp[i] & 1) ? -1.0 : 1.0);
        const V3D f = vsub(ra, vp[i]);
        for (int j = 0; j < 3; ++j) {
          if (!edge_valid(ecq[j])) continue;
          const V3D e_j = vsub(vq[(j + 2) % 3], vq[(j + 1) % 3]);
          const D1 sl_j = dsqrt(vdot(e_j, e_j)) * ((ecq[j] & 1) ? -1.0 : 1.0);
          const V3D dv = vsub(rho0, vq[j]);
          // J = I1 + (rho0 - v_j) I0;  term = w_a (f . J / 4 - I0 / k^2)
          const DC J[3] = {DC{I1[0].re + dv.x * I0.re, I1[0].im + dv.x * I0.im},
                           DC{I1[1].re + dv.y * I0.re, I1[1].im + dv.y * I0.im},
                           DC{I1[2].re + dv.z * I0.re, I1[2].im + dv.z * I0.im}};
          const D1 tr = (f.x * J[0].re + f.y * J[1].re + f.z * J[2].re) * 0.25 - I0.re * inv_k2;
          const D1 ti = (f.x * J[0].im + f.y * J[1].im + f.z * J[2].im) * 0.25 - I0.im * inv_k2;
          // Z share = j k eta sl_i sl_j / A_q * w_a * (tr + j ti) = c (-ti + j tr)
          const D1 c = kd * (eta * wa) * sl_i * sl_j / area_q;
          const D1 zr = -(c * ti), zi = c * tr;
          const float2 gz = gZ[(int64_t)edge_of(ecp[i]) * ldg + edge_of(ecq[j])];
          // dL = Re(conj(gZ) dZ) = gz.x dZr + gz.y dZi
          dL += (double)gz.x * zr.d + (double)gz.y * zi.d;
        }
      }
    }
    for (int off = 1; off < G; off <<= 1) dL += __shfl_xor_sync(gmask, dL, off);
    if (sub == 0) {
      if (dir == 18) atomicAdd(dkacc, dL);
      else if (dir < 9) atomicAdd(&dtri[9 * (size_t)p + dir], dL);
      else atomicAdd(&dtri[9 * (size_t)q + dir - 9], dL);
    }
  }
}

// dxyz[v] += sum over the corners of triangles at v (triangles in internal order)
__global__ void k_adjoint_gather(int nt, const int4* __restrict__ tvert, const double* __restrict__ dtri, double* dxyz) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int4 v = tvert[t];
  const int vs[3] = {v.x, v.y, v.z};
  for (int c = 0; c < 3; ++c)
    for (int x = 0; x < 3; ++x) atomicAdd(&dxyz[3 * (size_t)vs[c] + x], dtri[9 * (size_t)t + 3 * c + x]);
}

// ---------------------------------------------------------------- batched
// Persistent kernels over the regular tasks and near pairs of many meshes:
// warps pull chunks of a global task list (meshes with the most work first)
// from an atomic counter; the mesh of a task is found by binary search in the
// descriptors' prefix offsets. Every mesh has its own k, tables and Z.
__device__ __forceinline__ int batch_item_of(const BatchItem* items, int nitems, int64_t t, bool near) {
  int lo = 0, hi = nitems - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int64_t b = near ? items[mid].near_begin : items[mid].reg_begin;
    if (b <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int M, bool TABLE>
__global__ void __launch_bounds__(512) k_batch_regular32(const BatchItem* __restrict__ items, int nitems, int64_t total,
                                                         unsigned long long* counter, int chunk) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(counter, (unsigned long long)chunk);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((int64_t)base >= total) break;
    const int64_t end = min((int64_t)base + chunk, total);
    for (int64_t t = (int64_t)base; t < end; ++t) {
      const BatchItem& it = items[batch_item_of(items, nitems, t, false)];
      const Tab32 T = tab32(it.green);
      int p, q0;
      if (sym_task(t - it.reg_begin, it.g.nt, &p, &q0))
        regular_task32<M, TABLE ? kLagrange : kDirect, true>(
            it.g, T, it.kpi, it.scale32, it.inv_k2_32, DenseUpper{reinterpret_cast<float2*>(it.Z), it.ldz}, p, q0, lane);
    }
  }
}

template <bool MIXED>
__global__ void __launch_bounds__(128) k_batch_near(const BatchItem* __restrict__ items, int nitems, int64_t total,
                                                    unsigned long long* counter, NearArgs A) {
  const int lane = threadIdx.x & 31;
  const int sub = threadIdx.x & 7;
  const unsigned gmask = 0xFFu << (threadIdx.x & 24);
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(counter, 4ull);  // one near pair per 8-lane group
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((int64_t)base >= total) break;
    const int64_t t = (int64_t)base + (lane >> 3);
    if (t < total) {
      const BatchItem& it = items[batch_item_of(items, nitems, t, true)];
      const Tab32 te32 = tab32(it.exp);
      near_task<float2, MIXED>(it.g, it.exp, te32, (float)it.exp.r_lo, (float)it.exp.r_hi, it.use_table != 0, A,
                               KScal{it.k, it.scale, it.inv_k2, 1.0 / it.k}, reinterpret_cast<float2*>(it.Z), it.ldz, it.n_near,
                               t - it.near_begin, true, sub, gmask);
    }
  }
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

int64_t pair_grid(const GeoView& g, int blocks_per_sm) {
  const int64_t ntask = regular_units(g.nt);
  int64_t blocks = (ntask + kWarps - 1) / kWarps;
  return std::min<int64_t>(blocks, (int64_t)sm_count() * blocks_per_sm);
}

}  // namespace

template <int M>
cudaError_t launch_batch_regular_m(const BatchItem* items, int nitems, int64_t total, unsigned long long* counter,
                                   bool table, int block, int grid, int chunk, cudaStream_t s) {
  if (table)
    k_batch_regular32<M, true><<<grid, block, 0, s>>>(items, nitems, total, counter, chunk);
  else
    k_batch_regular32<M, false><<<grid, block, 0, s>>>(items, nitems, total, counter, chunk);
  return cudaGetLastError();
}

cudaError_t launch_batch_regular(const BatchItem* items, int nitems, int64_t total, unsigned long long* counter, int m,
                                 bool table, int block, int grid, int chunk, cudaStream_t s) {
  switch (m) {
    case 1: return launch_batch_regular_m<1>(items, nitems, total, counter, table, block, grid, chunk, s);
    case 3: return launch_batch_regular_m<3>(items, nitems, total, counter, table, block, grid, chunk, s);
    case 4: return launch_batch_regular_m<4>(items, nitems, total, counter, table, block, grid, chunk, s);
    case 6: return launch_batch_regular_m<6>(items, nitems, total, counter, table, block, grid, chunk, s);
    case 7: return launch_batch_regular_m<7>(items, nitems, total, counter, table, block, grid, chunk, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int M>
int batch_blocks_m(bool table, int block) {
  int n = 0;
  if (table) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_regular32<M, true>, block, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_regular32<M, false>, block, 0);
  return n;
}

int batch_regular_blocks_per_sm(int m, bool table, int block) {
  switch (m) {
    case 1: return batch_blocks_m<1>(table, block);
    case 3: return batch_blocks_m<3>(table, block);
    case 4: return batch_blocks_m<4>(table, block);
    case 6: return batch_blocks_m<6>(table, block);
    case 7: return batch_blocks_m<7>(table, block);
    default: return 0;
  }
}

cudaError_t launch_batch_near(const BatchItem* items, int nitems, int64_t total, unsigned long long* counter,
                              bool mixed, int nphi, int nl, const double* gl_phi, const double* gl_l, int grid,
                              cudaStream_t s) {
  NearArgs A;
  A.k = A.scale = A.inv_k2 = 0.0;  // per mesh, from the descriptors
  A.nphi = nphi;
  A.nl = nl;
  for (int i = 0; i < 32; ++i) {
    A.gx_phi[i] = gl_phi[i];
    A.gw_phi[i] = gl_phi[32 + i];
    A.gx_l[i] = gl_l[i];
    A.gw_l[i] = gl_l[32 + i];
    A.fx_phi[i] = (float)A.gx_phi[i];
    A.fw_phi[i] = (float)A.gw_phi[i];
    A.fx_l[i] = (float)A.gx_l[i];
    A.fw_l[i] = (float)A.gw_l[i];
  }
  if (mixed) k_batch_near<true><<<grid, 128, 0, s>>>(items, nitems, total, counter, A);
  else k_batch_near<false><<<grid, 128, 0, s>>>(items, nitems, total, counter, A);
  return cudaGetLastError();
}

template <int M>
cudaError_t launch_adjoint_regular_m(const GeoView& g, const TabView* green, double k, double eta, const BaryF& bw,
                                     const float2* gZ, int64_t ldg, double* dtri, double* dk, cudaStream_t s) {
  TabView tv{};
  if (green) tv = *green;
  const int64_t blocks = pair_grid(g, 4);
  const float kappa = (float)(k * eta / (4.0 * kPi)), inv_k2 = (float)(1.0 / (k * k));
  if (green)
    k_adjoint_regular32<M, true><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, (float)k, kappa, inv_k2, bw, gZ, ldg,
                                                                       dtri, dk);
  else
    k_adjoint_regular32<M, false><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, (float)k, kappa, inv_k2, bw, gZ, ldg,
                                                                        dtri, dk);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const GeoView& g, const TabView* green, const TabView* texp, bool mixed, double k,
                           double eta, const double* bary, int nphi, int nl, const double* gl_phi, const double* gl_l,
                           const void* gZ, int64_t ldg, double* dtri, double* dk, double* dxyz, int64_t nv,
                           cudaStream_t s) {
  BaryF bw;
  for (int a = 0; a < kMaxRule; ++a)
    for (int c = 0; c < 3; ++c) bw.l[a][c] = a < g.m ? (float)bary[3 * a + c] : 0.f;
  cudaError_t e = cudaMemsetAsync(dtri, 0, 9 * sizeof(double) * (size_t)g.nt, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dk, 0, sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dxyz, 0, 3 * sizeof(double) * (size_t)nv, s);
  if (e != cudaSuccess) return e;
  const float2* gz = (const float2*)gZ;
  switch (g.m) {
    case 1: e = launch_adjoint_regular_m<1>(g, green, k, eta, bw, gz, ldg, dtri, dk, s); break;
    case 3: e = launch_adjoint_regular_m<3>(g, green, k, eta, bw, gz, ldg, dtri, dk, s); break;
    case 4: e = launch_adjoint_regular_m<4>(g, green, k, eta, bw, gz, ldg, dtri, dk, s); break;
    case 6: e = launch_adjoint_regular_m<6>(g, green, k, eta, bw, gz, ldg, dtri, dk, s); break;
    case 7: e = launch_adjoint_regular_m<7>(g, green, k, eta, bw, gz, ldg, dtri, dk, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  NearArgs A;
  A.k = k;
  A.scale = k * eta;
  A.inv_k2 = 1.0 / (k * k);
  A.nphi = nphi;
  A.nl = nl;
  for (int i = 0; i < 32; ++i) {
    A.gx_phi[i] = gl_phi[i];
    A.gw_phi[i] = gl_phi[32 + i];
    A.gx_l[i] = gl_l[i];
    A.gw_l[i] = gl_l[32 + i];
    A.fx_phi[i] = (float)A.gx_phi[i];
    A.fw_phi[i] = (float)A.gw_phi[i];
    A.fx_l[i] = (float)A.gx_l[i];
    A.fw_l[i] = (float)A.gw_l[i];
  }
  TabView te{};
  if (texp) te = *texp;
  const unsigned nblk = (unsigned)(sm_count() * 16);
  const bool t = texp != nullptr;
  // mixed precision: reverse mode, one pass per near pair; FP64 throughout:
  // forward-mode duals, one pass per (near pair, direction)
  if (g.m <= 4) {
    if (mixed) k_adjoint_near_rev<4><<<nblk, 128, 0, s>>>(g, te, t, A, k, eta, bw, gz, ldg, dtri, dk);
    else k_adjoint_near<false, 4><<<nblk, 128, 0, s>>>(g, te, t, A, k, eta, bw, gz, ldg, dtri, dk);
  } else {
    if (mixed) k_adjoint_near_rev<8><<<nblk, 128, 0, s>>>(g, te, t, A, k, eta, bw, gz, ldg, dtri, dk);
    else k_adjoint_near<false, 8><<<nblk, 128, 0, s>>>(g, te, t, A, k, eta, bw, gz, ldg, dtri, dk);
  }
  k_adjoint_gather<<<(g.nt + 127) / 128, 128, 0, s>>>(g.nt, g.tvert, dtri, dxyz);
  return cudaGetLastError();
}

cudaError_t launch_block_spheres(const GeoView& g, float4* bsph, cudaStream_t s) {
  const int nb = (g.nt + 31) / 32;
  k_block_spheres<<<(unsigned)((nb + 3) / 4), 128, 0, s>>>(g, bsph);
  return cudaGetLastError();
}

cudaError_t launch_prep_geometry(const double* v64, int nt, int m, const double* bary, const double* w,
                                 const int4* tedge, const double* edge_len, float4* pts32, float4* cen32,
                                 float4* geo32, double* pts64, double* cen64, double* geo64, float* rad32,
                                 double* frame64, float* frame32, cudaStream_t s) {
  k_prep_geometry<<<(nt + 127) / 128, 128, 0, s>>>(v64, nt, m, bary, w, tedge, edge_len, pts32, cen32, geo32,
                                                   pts64, cen64, geo64, rad32, frame64, frame32);
  return cudaGetLastError();
}

cudaError_t launch_tables(const TableBuild& a, const TableBuild& b, double k, cudaStream_t s) {
  const int n1 = a.n + a.n_hash + a.n_cells64 + b.n + b.n_hash + b.n_cells64;
  const int n2 = a.n + b.n;
  const int n3 = std::max(a.view.n_lat, a.view.n_cmp) + std::max(b.view.n_lat, b.view.n_cmp);
  k_tables_values<<<(n1 + 255) / 256, 256, 0, s>>>(a, b, k);
  k_tables_coef<<<(n2 + 127) / 128, 128, 0, s>>>(a, b);
  k_tables_lattice<<<(n3 + 127) / 128, 128, 0, s>>>(a, b);
  return cudaGetLastError();
}

cudaError_t launch_table_eval(const TabView& t, int kind, int precision, const void* r, int64_t n, void* out,
                              cudaStream_t s) {
  int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16);
  const bool lin = kind == GF_EXP;
  if (precision == GF_FP32) {
    if (lin) k_table_eval32<1><<<(unsigned)blocks, 256, 0, s>>>(t, (const float*)r, n, (float2*)out);
    else k_table_eval32<3><<<(unsigned)blocks, 256, 0, s>>>(t, (const float*)r, n, (float2*)out);
  } else {
    if (lin) k_table_eval64<1><<<(unsigned)blocks, 256, 0, s>>>(t, (const double*)r, n, (double2*)out);
    else k_table_eval64<3><<<(unsigned)blocks, 256, 0, s>>>(t, (const double*)r, n, (double2*)out);
  }
  return cudaGetLastError();
}

cudaError_t launch_range(const GeoView& g, int precision, unsigned long long* d_minmax, float2* bpb, int32_t* list,
                         cudaStream_t s) {
  const int64_t nb = (g.nt + 31) / 32, nbp = nb * (nb + 1) / 2;
  if (precision == GF_FP64) {
    k_range_init<<<1, 32, 0, s>>>(d_minmax, bpb, 0);
    int64_t blocks = pair_grid(g, 8);
    k_range64<<<(unsigned)blocks, kThreads, 0, s>>>(g, d_minmax);
    return cudaGetLastError();
  }
  const unsigned nsm = (unsigned)sm_count();
  const unsigned b0 = (unsigned)std::min<int64_t>((nbp + kThreads - 1) / kThreads, (int64_t)nsm * 4);
  k_range_init<<<b0, kThreads, 0, s>>>(d_minmax, bpb, nbp);
  const int64_t b1 = std::min<int64_t>((nbp * kRangeSplit + kWarps - 1) / kWarps, (int64_t)nsm * 8);
  k_range_bounds<<<(unsigned)b1, kThreads, 0, s>>>(g, d_minmax, bpb);
  k_range_list<<<b0, kThreads, 0, s>>>(d_minmax, bpb, nbp, list);
  // the pass-2 block records follow the list (sized for kRangeMaxBlocks)
  RExt* rec = reinterpret_cast<RExt*>(list + ((nbp + 3) & ~int64_t(3)));
  const unsigned b2 = (unsigned)std::min<int64_t>(std::min<int64_t>((nbp * 32 + kWarps - 1) / kWarps, (int64_t)nsm * 8),
                                                  kRangeMaxBlocks);
  switch (g.m) {
    case 1: k_range32<1><<<b2, kThreads, 0, s>>>(g, d_minmax, list, rec); break;
    case 3: k_range32<3><<<b2, kThreads, 0, s>>>(g, d_minmax, list, rec); break;
    case 4: k_range32<4><<<b2, kThreads, 0, s>>>(g, d_minmax, list, rec); break;
    case 6: k_range32<6><<<b2, kThreads, 0, s>>>(g, d_minmax, list, rec); break;
    case 7: k_range32<7><<<b2, kThreads, 0, s>>>(g, d_minmax, list, rec); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int M, int MODE>
cudaError_t launch_regular32_table(const TabView& tv, const GeoView& g, float kpi, float scale, float inv_k2,
                                   float2* Z, int64_t ldz, cudaStream_t s) {
  const size_t smem = tv.smem32_bytes(MODE == kLagrange ? 3 : 1);
  int dev = 0, max_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem <= (size_t)max_optin) {
    // deferred corrections while at most 0.5 % of the lattice cells hold samples
    auto kern = tv.n_busy * 200 <= tv.n_lat ? k_fill_regular32<M, MODE, true, true> : k_fill_regular32<M, MODE, true, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, smem);
    int64_t blocks = std::min<int64_t>(pair_grid(g, 2 * std::max(per_sm, 1)), (int64_t)sm_count() * std::max(per_sm, 1));
    kern<<<(unsigned)blocks, 512, smem, s>>>(g, tv, kpi, scale, inv_k2, Z, ldz);
  } else if (MODE == kLagrange && g.bsph) {
    cudaError_t e =
        cudaFuncSetAttribute(k_fill_regular32_win<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWinBytes);
    if (e != cudaSuccess) return e;
    k_fill_regular32_win<M><<<(unsigned)sm_count(), 512, kWinBytes, s>>>(g, tv, g.bsph, kpi, scale, inv_k2, Z, ldz);
  } else {
    int64_t blocks = pair_grid(g, 4);
    k_fill_regular32<M, MODE, false><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, kpi, scale, inv_k2, Z, ldz);
  }
  return cudaGetLastError();
}

template <int M>
cudaError_t launch_regular32(const GeoView& g, const TabView* table, bool from_exp, float kpi, float scale,
                             float inv_k2, float2* Z, int64_t ldz, cudaStream_t s) {
  if (!table) {
    TabView tv{};
    int64_t blocks = pair_grid(g, 4);
    k_fill_regular32<M, kDirect, false><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, kpi, scale, inv_k2, Z, ldz);
    return cudaGetLastError();
  }
  if (from_exp) return launch_regular32_table<M, kExpOverR>(*table, g, kpi, scale, inv_k2, Z, ldz, s);
  return launch_regular32_table<M, kLagrange>(*table, g, kpi, scale, inv_k2, Z, ldz, s);
}

// Z <- Z + Z^T on the ne x ne block (row-major, leading dimension ldz): the
// regular fill leaves each unordered pair's block in its test triangle's rows
// only. Per pair of 32 x 32 tiles (I, J), I <= J (a grid-stride walk over all
// (I, J) that skips I > J): both tiles read through shared memory, both
// written; a diagonal tile is its own partner. HBM-bound: 2 x 8 ne^2 bytes.
__global__ void __launch_bounds__(256) k_symmetrize32(float2* __restrict__ Z, int64_t ldz, int ne) {
  __shared__ float2 ta[32][33];
  __shared__ float2 tb[32][33];
  const int nb = (ne + 31) >> 5;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int64_t t = blockIdx.x; t < (int64_t)nb * nb; t += gridDim.x) {
    const int I = (int)(t / nb), J = (int)(t % nb);
    if (I > J) continue;  // uniform over the block
    for (int r = ty; r < 32; r += 8) {
      const int gr = I * 32 + r, gc = J * 32 + tx;
      ta[r][tx] = (gr < ne && gc < ne) ? Z[(int64_t)gr * ldz + gc] : make_float2(0.f, 0.f);
      const int hr = J * 32 + r, hc = I * 32 + tx;
      tb[r][tx] = (hr < ne && hc < ne) ? Z[(int64_t)hr * ldz + hc] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int gr = I * 32 + r, gc = J * 32 + tx;
      const float2 a = ta[r][tx], b = tb[tx][r];
      if (gr < ne && gc < ne) Z[(int64_t)gr * ldz + gc] = make_float2(a.x + b.x, a.y + b.y);
      if (I != J) {
        const int hr = J * 32 + r, hc = I * 32 + tx;
        const float2 c = tb[r][tx], d = ta[tx][r];
        if (hr < ne && hc < ne) Z[(int64_t)hr * ldz + hc] = make_float2(c.x + d.x, c.y + d.y);
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_fill_regular(const GeoView& g, const TabView* table, bool from_exp, double green_scale,
                                int precision, double k, double eta, void* Z, int64_t ldz, cudaStream_t s) {
  const double scale = k * eta / (4.0 * kPi) * (table && !from_exp ? green_scale : 1.0);
  TabView tv{};
  if (table) tv = *table;
  if (precision == GF_FP64) {
    int64_t blocks = pair_grid(g, 4);
    const double ik2 = 1.0 / (k * k);
    if (!table)
      k_fill_regular64<kDirect><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, k, scale, ik2, (double2*)Z, ldz);
    else if (from_exp)
      k_fill_regular64<kExpOverR><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, k, scale, ik2, (double2*)Z, ldz);
    else
      k_fill_regular64<kLagrange><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, k, scale, ik2, (double2*)Z, ldz);
    return cudaGetLastError();
  }
  const float kpi = (float)(k / kPi), sc = (float)scale, ik2 = (float)(1.0 / (k * k));
  float2* Z32 = (float2*)Z;
  // each unordered pair into its test triangle's rows (launch_mirror32 adds
  // the transpose)
  cudaError_t e;
  switch (g.m) {
    case 1: e = launch_regular32<1>(g, table, from_exp, kpi, sc, ik2, Z32, ldz, s); break;
    case 3: e = launch_regular32<3>(g, table, from_exp, kpi, sc, ik2, Z32, ldz, s); break;
    case 4: e = launch_regular32<4>(g, table, from_exp, kpi, sc, ik2, Z32, ldz, s); break;
    case 6: e = launch_regular32<6>(g, table, from_exp, kpi, sc, ik2, Z32, ldz, s); break;
    case 7: e = launch_regular32<7>(g, table, from_exp, kpi, sc, ik2, Z32, ldz, s); break;
    default: return cudaErrorInvalidValue;
  }
  return e;
}

cudaError_t launch_mirror32(void* Z, int64_t ldz, int64_t ne, cudaStream_t s) {
  if (ne == 0) return cudaSuccess;
  const int64_t nb = (ne + 31) / 32;
  const int64_t blocks = std::min<int64_t>(nb * nb, (int64_t)sm_count() * 8);
  k_symmetrize32<<<(unsigned)blocks, 256, 0, s>>>((float2*)Z, ldz, (int)ne);
  return cudaGetLastError();
}

template <int M, bool DEFER>
cudaError_t launch_mfie32_table(const TabView& tv, const GeoView& g, float kpi, float k32, float scale, float2* Z,
                                int64_t ldz, cudaStream_t s) {
  const size_t smem = tv.smem32_bytes(3);
  int dev = 0, max_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int64_t ntask = (int64_t)g.nt * ((g.nt + 31) / 32);
  if (smem <= (size_t)max_optin) {
    auto kern = k_mfie_regular32<M, kLagrange, true, DEFER>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 512, smem);
    const int64_t blocks = std::min<int64_t>((ntask + 15) / 16, (int64_t)sm_count() * std::max(per_sm, 1));
    kern<<<(unsigned)blocks, 512, smem, s>>>(g, tv, kpi, k32, scale, Z, ldz);
  } else {
    const int64_t blocks = std::min<int64_t>((ntask + kWarps - 1) / kWarps, (int64_t)sm_count() * 4);
    k_mfie_regular32<M, kLagrange, false, DEFER><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, kpi, k32, scale, Z, ldz);
  }
  return cudaGetLastError();
}

template <int M>
cudaError_t launch_mfie32(const GeoView& g, const TabView* table, float kpi, float k32, float scale, float2* Z,
                          int64_t ldz, cudaStream_t s) {
  if (!table) {
    TabView tv{};
    const int64_t ntask = (int64_t)g.nt * ((g.nt + 31) / 32);
    const int64_t blocks = std::min<int64_t>((ntask + kWarps - 1) / kWarps, (int64_t)sm_count() * 4);
    k_mfie_regular32<M, kDirect, false, false><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, kpi, k32, scale, Z, ldz);
    return cudaGetLastError();
  }
  if (table->n_busy * 200 <= table->n_lat) return launch_mfie32_table<M, true>(*table, g, kpi, k32, scale, Z, ldz, s);
  return launch_mfie32_table<M, false>(*table, g, kpi, k32, scale, Z, ldz, s);
}

cudaError_t launch_fill_mfie(const GeoView& g, const TabView* green, const TabView* texp, double green_scale,
                             int precision, bool mixed, double k, int nphi, int nl, const double* gl_phi,
                             const double* gl_l, void* Z, int64_t ldz, cudaStream_t s) {
  const unsigned tb = (unsigned)((g.nt + 127) / 128);
  if (precision == GF_FP64) k_mfie_identity<double2><<<tb, 128, 0, s>>>(g, (double2*)Z, ldz);
  else k_mfie_identity<float2><<<tb, 128, 0, s>>>(g, (float2*)Z, ldz);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // (s l / 2)^2 of the two RWG functions and the 1/(4 pi) of Phi (times k for a table in kR)
  const double scale = 1.0 / (16.0 * kPi) * (green ? green_scale : 1.0);
  if (precision == GF_FP64) {
    TabView tv{};
    if (green) tv = *green;
    const int64_t ntask = (int64_t)g.nt * ((g.nt + 31) / 32);
    const int64_t blocks = std::min<int64_t>((ntask + kWarps - 1) / kWarps, (int64_t)sm_count() * 4);
    if (green) k_mfie_regular64<kLagrange><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, k, scale, (double2*)Z, ldz);
    else k_mfie_regular64<kDirect><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, k, scale, (double2*)Z, ldz);
    e = cudaGetLastError();
  } else {
    const float kpi = (float)(k / kPi), k32 = (float)k, sc = (float)scale;
    float2* Z32 = (float2*)Z;
    switch (g.m) {
      case 1: e = launch_mfie32<1>(g, green, kpi, k32, sc, Z32, ldz, s); break;
      case 3: e = launch_mfie32<3>(g, green, kpi, k32, sc, Z32, ldz, s); break;
      case 4: e = launch_mfie32<4>(g, green, kpi, k32, sc, Z32, ldz, s); break;
      case 6: e = launch_mfie32<6>(g, green, kpi, k32, sc, Z32, ldz, s); break;
      case 7: e = launch_mfie32<7>(g, green, kpi, k32, sc, Z32, ldz, s); break;
      default: return cudaErrorInvalidValue;
    }
  }
  if (e != cudaSuccess) return e;
  NearArgs A;
  A.k = k;
  A.scale = 0.0;
  A.inv_k2 = 0.0;
  A.nphi = nphi;
  A.nl = nl;
  for (int i = 0; i < 32; ++i) {
    A.gx_phi[i] = gl_phi[i];
    A.gw_phi[i] = gl_phi[32 + i];
    A.gx_l[i] = gl_l[i];
    A.gw_l[i] = gl_l[32 + i];
    A.fx_phi[i] = (float)A.gx_phi[i];
    A.fw_phi[i] = (float)A.gw_phi[i];
    A.fx_l[i] = (float)A.gx_l[i];
    A.fw_l[i] = (float)A.gw_l[i];
  }
  TabView te{};
  if (texp) te = *texp;
  const bool use_table = texp != nullptr;
  const unsigned nblk = (unsigned)(sm_count() * 16);
  if (g.m <= 4) {
    if (precision == GF_FP64) k_mfie_near<double2, 4, false><<<nblk, 128, 0, s>>>(g, te, use_table, A, (double2*)Z, ldz);
    else if (mixed) k_mfie_near<float2, 4, true><<<nblk, 128, 0, s>>>(g, te, use_table, A, (float2*)Z, ldz);
    else k_mfie_near<float2, 4, false><<<nblk, 128, 0, s>>>(g, te, use_table, A, (float2*)Z, ldz);
  } else {
    if (precision == GF_FP64) k_mfie_near<double2, 8, false><<<nblk, 128, 0, s>>>(g, te, use_table, A, (double2*)Z, ldz);
    else if (mixed) k_mfie_near<float2, 8, true><<<nblk, 128, 0, s>>>(g, te, use_table, A, (float2*)Z, ldz);
    else k_mfie_near<float2, 8, false><<<nblk, 128, 0, s>>>(g, te, use_table, A, (float2*)Z, ldz);
  }
  return cudaGetLastError();
}

template <int M>
cudaError_t launch_sparse32(const GeoView& g, const TabView* table, float kpi, float scale, float inv_k2,
                            const SparseTask* tasks, int64_t ntask, const int32_t* widx, CsrSink<float2> sink,
                            cudaStream_t s) {
  if (ntask == 0) return cudaSuccess;
  if (!table) {
    TabView tv{};
    const int64_t blocks = std::min<int64_t>((ntask + kWarps - 1) / kWarps, (int64_t)sm_count() * 4);
    k_sparse_regular32<M, kDirect, false, false><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, kpi, scale, inv_k2,
                                                                                      tasks, ntask, widx, sink);
    return cudaGetLastError();
  }
  const TabView& tv = *table;
  const size_t smem = tv.smem32_bytes(3);
  int dev = 0, max_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem <= (size_t)max_optin) {
    auto kern = tv.n_busy * 200 <= tv.n_lat ? k_sparse_regular32<M, kLagrange, true, true>
                                            : k_sparse_regular32<M, kLagrange, true, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = std::min<int64_t>((ntask + 15) / 16, (int64_t)sm_count());
    kern<<<(unsigned)blocks, 512, smem, s>>>(g, tv, kpi, scale, inv_k2, tasks, ntask, widx, sink);
  } else {
    const int64_t blocks = std::min<int64_t>((ntask + kWarps - 1) / kWarps, (int64_t)sm_count() * 4);
    k_sparse_regular32<M, kLagrange, false, false><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, kpi, scale, inv_k2,
                                                                                        tasks, ntask, widx, sink);
  }
  return cudaGetLastError();
}

cudaError_t launch_fill_sparse(const GeoView& g, const TabView* green, const TabView* texp, double green_scale,
                               bool mixed, double k, double eta, int nphi, int nl, const double* gl_phi,
                               const double* gl_l, const void* tasks_v, int64_t ntask, const int32_t* widx,
                               const int64_t* row_ptr, const int32_t* cols, void* vals, cudaStream_t s) {
  const SparseTask* tasks = static_cast<const SparseTask*>(tasks_v);
  CsrSink<float2> sink{row_ptr, cols, static_cast<float2*>(vals)};
  const double scale = k * eta / (4.0 * kPi) * (green ? green_scale : 1.0);
  const float kpi = (float)(k / kPi), sc = (float)scale, ik2 = (float)(1.0 / (k * k));
  cudaError_t e;
  switch (g.m) {
    case 1: e = launch_sparse32<1>(g, green, kpi, sc, ik2, tasks, ntask, widx, sink, s); break;
    case 3: e = launch_sparse32<3>(g, green, kpi, sc, ik2, tasks, ntask, widx, sink, s); break;
    case 4: e = launch_sparse32<4>(g, green, kpi, sc, ik2, tasks, ntask, widx, sink, s); break;
    case 6: e = launch_sparse32<6>(g, green, kpi, sc, ik2, tasks, ntask, widx, sink, s); break;
    case 7: e = launch_sparse32<7>(g, green, kpi, sc, ik2, tasks, ntask, widx, sink, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  NearArgs A;
  A.k = k;
  A.scale = k * eta;
  A.inv_k2 = 1.0 / (k * k);
  A.nphi = nphi;
  A.nl = nl;
  for (int i = 0; i < 32; ++i) {
    A.gx_phi[i] = gl_phi[i];
    A.gw_phi[i] = gl_phi[32 + i];
    A.gx_l[i] = gl_l[i];
    A.gw_l[i] = gl_l[32 + i];
    A.fx_phi[i] = (float)A.gx_phi[i];
    A.fw_phi[i] = (float)A.gw_phi[i];
    A.fx_l[i] = (float)A.gx_l[i];
    A.fw_l[i] = (float)A.gw_l[i];
  }
  TabView te{};
  if (texp) te = *texp;
  const bool use_table = texp != nullptr;
  const unsigned nblk = (unsigned)(sm_count() * 16);
  if (g.m <= 4) {
    if (mixed) k_sparse_near<true, 4><<<nblk, 128, 0, s>>>(g, te, use_table, A, sink);
    else k_sparse_near<false, 4><<<nblk, 128, 0, s>>>(g, te, use_table, A, sink);
  } else {
    if (mixed) k_sparse_near<true, 8><<<nblk, 128, 0, s>>>(g, te, use_table, A, sink);
    else k_sparse_near<false, 8><<<nblk, 128, 0, s>>>(g, te, use_table, A, sink);
  }
  return cudaGetLastError();
}

int sparse_task_bytes() { return (int)sizeof(SparseTask); }

cudaError_t launch_fill_near(const GeoView& g, const TabView* texp, int precision, bool mixed, double k, double eta,
                             int nphi, int nl, const double* gl_phi, const double* gl_l, void* Z, int64_t ldz,
                             cudaStream_t s) {
  NearArgs A;
  A.k = k;
  A.scale = k * eta;
  A.inv_k2 = 1.0 / (k * k);
  A.nphi = nphi;
  A.nl = nl;
  for (int i = 0; i < 32; ++i) {
    A.gx_phi[i] = gl_phi[i];
    A.gw_phi[i] = gl_phi[32 + i];
    A.gx_l[i] = gl_l[i];
    A.gw_l[i] = gl_l[32 + i];
    A.fx_phi[i] = (float)A.gx_phi[i];
    A.fw_phi[i] = (float)A.gw_phi[i];
    A.fx_l[i] = (float)A.gx_l[i];
    A.fw_l[i] = (float)A.gw_l[i];
  }
  TabView te{};
  if (texp) te = *texp;
  const int64_t n_near = 0;  // read on the device
  (void)n_near;
  int64_t blocks = (int64_t)sm_count() * 16;
  const bool t = texp != nullptr;
  // groups of 4 lanes for rules of up to 4 points, else 8 (idle lanes still cost FP64 pipe time)
  if (g.m <= 4) {
    if (precision == GF_FP32 && mixed)
      k_fill_near<float2, true, 4><<<(unsigned)blocks, 128, 0, s>>>(g, te, t, A, (float2*)Z, ldz);
    else if (precision == GF_FP32)
      k_fill_near<float2, false, 4><<<(unsigned)blocks, 128, 0, s>>>(g, te, t, A, (float2*)Z, ldz);
    else
      k_fill_near<double2, false, 4><<<(unsigned)blocks, 128, 0, s>>>(g, te, t, A, (double2*)Z, ldz);
  } else {
    if (precision == GF_FP32 && mixed)
      k_fill_near<float2, true, 8><<<(unsigned)blocks, 128, 0, s>>>(g, te, t, A, (float2*)Z, ldz);
    else if (precision == GF_FP32)
      k_fill_near<float2, false, 8><<<(unsigned)blocks, 128, 0, s>>>(g, te, t, A, (float2*)Z, ldz);
    else
      k_fill_near<double2, false, 8><<<(unsigned)blocks, 128, 0, s>>>(g, te, t, A, (double2*)Z, ldz);
  }
  return cudaGetLastError();
}

}  // namespace gf
