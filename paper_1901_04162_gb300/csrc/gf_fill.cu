// gfmom fill kernels for sm_103a: geometry preparation, the device stage of
// the tables (sample values, coefficients, Eq. 6 hash, FP32 lattice image),
// the R_min / R_max reduction, the regular-pair kernels (FP32 with the table
// staged in shared memory or windowed, FP64), the mirror pass Z += Z^T and
// the near-pair kernel, with their launchers.
#include "gf_near.cuh"

namespace gf {
namespace {

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
    // lengths, unit edge tangents (v_e -> v_{e+1}), in-plane edge normals t x n,
    // 1/area and the reciprocal edge lengths; an FP32 copy of the lengths,
    // tangents and normals
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
      fr[25 + e] = il;
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
// the cell anchor A_i = fma(i, h, lat_amid) (the anchor the lookups
// recompute): (c0, c1) in FP32 with the flag bit of the cells holding samples
// in c1im, and for the Green table c2 as a half2 scaled by 2^E; a flagged
// cell's lat_c word is its place in the busy list instead.
__device__ void dev_table_lattice(int i, const TabView& v, int deg, const double* __restrict__ r,
                                  const double* __restrict__ f, const int32_t* __restrict__ lat_j,
                                  const int32_t* __restrict__ cmp, float4* la, uint32_t* lc) {
  if (i < v.n_cmp) {  // full interval records of the blob
    float4* ca = const_cast<float4*>(v.lat_blob) + (v.n_busy + 3) / 4 + v.n_busy + v.n_sub;
    ca[i] = v.c32a[cmp[i]];
    ca[v.n_cmp + i] = v.c32b[cmp[i]];
  }
  if (i >= v.n_lat) return;
  const float A = __fmaf_rn((float)i, v.lat_h, v.lat_amid);
  const int jb = lat_j[i];
  double cre[4], cim[4];
  interval_poly(deg, v.n_nodes, r, f, jb & 0x7fffffff, (double)A, cre, cim);
  float4 a = make_float4((float)cre[0], (float)cim[0], (float)cre[1], (float)cim[1]);
  // flag bit: the lowest mantissa bit of c1im (changes it by one ulp at most)
  const int busy = (int)(((unsigned)jb) >> 31);
  a.w = __int_as_float((__float_as_int(a.w) & ~1) | busy);
  uint32_t c = 0u;
  if (busy) {  // the cell's place in the busy list, for the exact path
    const int* list = reinterpret_cast<const int*>(v.lat_blob);
    int lo = 0, hi = v.n_busy - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (list[mid] < i) lo = mid + 1;
      else hi = mid;
    }
    c = (uint32_t)lo;
  } else if (deg > 1) {
    const double e = 1.0 / (double)v.lat_c2d;  // 2^E
    const __half2 hv = __floats2half2_rn((float)(cre[2] * e), (float)(cim[2] * e));
    const __half2_raw hr = hv;
    c = (uint32_t)hr.x | ((uint32_t)hr.y << 16);
  }
  la[i] = a;
  lc[i] = c;
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
      return dev_table_lattice(i, T.view, T.deg, T.node64, T.fval, T.lat_j, T.cmp, T.lat_a, T.lat_c);
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

// Row (test triangle) of every near-list entry, expanded from the CSR row
// pointers: one warp per row.
__global__ void k_near_rows(const int64_t* __restrict__ near_ptr, int64_t nt, int32_t* near_row) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nt; r += nwarp)
    for (int64_t j = near_ptr[r] + lane; j < near_ptr[r + 1]; j += 32) near_row[j] = (int32_t)r;
}

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

// Every point distance of the triangles of blocks I and J lies in
// [D - r_I - r_J, D + r_I + r_J] (D = distance of the blocks' bounding-sphere
// centres), widened by the slack of pair_bounds.
__device__ __forceinline__ void block_bounds(const float4* __restrict__ bsph, int I, int J, float* lb, float* ub) {
  const float4 a = bsph[I], b = bsph[J];
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  const float D = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
  const float r = a.w + b.w;
  const float mag = fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fmaxf(fmaxf(fabsf(b.x), fabsf(b.y)),
                                                                                  fabsf(b.z))));
  const float slack = 1e-5f * (D + r + mag);
  *lb = fmaxf(D - r - slack, 0.f);
  *ub = D + r + slack;
}

// Pass 0, one warp per 32 x 32 block pair: first thresholds mm[2] >= r_min
// and mm[3] <= r_max from actual distances (the first rule point of the test
// block's first triangle and of each source triangle, regular pairs only),
// so that pass 1 can skip the block pairs whose bounding spheres keep every
// point distance inside (mm[2], mm[3]).
__global__ void __launch_bounds__(kThreads) k_range_witness(GeoView g, unsigned long long* mm) {
  const int lane = threadIdx.x & 31;
  const int64_t nb = (g.nt + 31) / 32, nbp = nb * (nb + 1) / 2;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float min_d = INFINITY, max_d = 0.f;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < nbp; u += nwarp) {
    int p, q0;
    sym_task(u * 32, g.nt, &p, &q0);
    const int q = min(q0 + lane, g.nt - 1);
    const float4 cp = g.cen32[p], cq = g.cen32[q];
    const float3 dc = make_float3(cp.x - cq.x, cp.y - cq.y, cp.z - cq.z);
    if (!((q0 + lane < g.nt) && q > p && !pair_is_near(g, p, q, g.tvert[p], g.tvert[q], dc))) continue;
    const float4 xp = g.pts32[p], yq = g.pts32[q];
    const float rx = (dc.x + xp.x) - yq.x, ry = (dc.y + xp.y) - yq.y, rz = (dc.z + xp.z) - yq.z;
    const float d = sqrtf(fmaf(rx, rx, fmaf(ry, ry, rz * rz)));
    min_d = fminf(min_d, d);
    max_d = fmaxf(max_d, d);
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

// Pass 1, one warp per 8 test triangles of a 32 x 32 block pair whose
// bounding spheres reach below the pass-0 threshold mm[2] or above mm[3]
// (the others hold no extreme and are skipped): thresholds from actual point
// distances (the first rule point of each triangle of every regular pair:
// their minimum is >= r_min, their maximum <= r_max), widened by a relative
// 1e-5 for the FP32 rounding (mm[2], mm[3]), and, per block pair, the
// smallest lower and largest upper bound of its regular pairs (bpb, merged by
// integer atomics on the bits of these non-negative floats), so that pass 2
// skips block pairs that cannot hold an extreme.
__global__ void __launch_bounds__(kThreads) k_range_bounds(GeoView g, unsigned long long* mm, float2* bpb) {
  const int lane = threadIdx.x & 31;
  const int64_t nb = (g.nt + 31) / 32, ntask = nb * (nb + 1) / 2 * kRangeSplit;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // the thresholds of pass 0 (any later, tighter value would serve as well)
  const float u_min = (float)__longlong_as_double((long long)mm[2]);
  const float l_max = (float)__longlong_as_double((long long)mm[3]);
  float min_d = INFINITY, max_d = 0.f;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntask; t += nwarp) {
    const int64_t u = t / kRangeSplit;
    int p0, q0;
    sym_task(u * 32, g.nt, &p0, &q0);
    {
      float lb, ub;
      block_bounds(g.bsph, p0 >> 5, q0 >> 5, &lb, &ub);
      if (lb > u_min && ub < l_max) continue;  // no pair of this block pair can hold an extreme (uniform)
    }
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
  const KScal ks{A.k, A.scale, A.inv_k2, 1.0 / A.k, (float)(4.0 * A.inv_k2), (float)A.scale};
  for (int64_t it = 0; it < iters; ++it) {
    const int64_t idx = g0 + it * ngroups;
    near_task<Out, MIXED, G>(g, te, te32, lo32, hi32, use_table, A, ks, Z, ldz, n_near, idx, idx < n_near, sub, gmask);
  }
}


// One warp per block of 32 triangles (lane = triangle): mean of the
// centroids, then the largest centroid distance plus point radius; the block
// centre for the split distances is the mean rounded to the grid of step
// g.bunit.
__global__ void k_block_spheres(GeoView g, float4* bsph, int4* bgrid) {
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
  // the farthest vertex from the block's centre (the near-pair screen of a task)
  double rv = 0.0;
  for (int i = 0; i < 3; ++i) {
    const double* gi = g.geo64 + 4 * (3 * (size_t)t + i);  // c - v_i
    rv = fmax(rv, sqrt(gi[0] * gi[0] + gi[1] * gi[1] + gi[2] * gi[2]));
  }
  rv += sqrt(dx * dx + dy * dy + dz * dz);
  for (int off = 16; off > 0; off >>= 1) {
    r = fmax(r, __shfl_xor_sync(0xffffffffu, r, off));
    rv = fmax(rv, __shfl_xor_sync(0xffffffffu, rv, off));
  }
  if (lane == 0) {
    bsph[b] = make_float4((float)cx, (float)cy, (float)cz, (float)(r * (1.0 + 1e-6)));
    const double inv = 1.0 / (double)g.bunit;
    // block centre on the grid; w: the vertex radius about it (bits of a float, rounded up)
    bgrid[b] = make_int4((int)llrint(cx * inv), (int)llrint(cy * inv), (int)llrint(cz * inv),
                         __float_as_int((float)((rv + (double)g.bunit) * (1.0 + 1e-6))));
  }
}

// Offsets from the block centres: the rule's points (with their weights) and
// the vertices opposite each local edge (with s_i l_i), FP64 differences
// rounded once to FP32.
__global__ void k_block_offsets(GeoView g, const int4* __restrict__ bgrid, float4* rel32, float4* geob32) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.nt) return;
  const int4 cb = bgrid[t >> 5];
  const double u = (double)g.bunit;
  const double C[3] = {cb.x * u, cb.y * u, cb.z * u};
  const double* c = g.cen64 + 4 * (size_t)t;
  for (int a = 0; a < g.m; ++a) {
    const double* pa = g.pts64 + 4 * ((size_t)a * g.nt + t);
    rel32[(size_t)a * g.nt + t] = make_float4((float)(c[0] + pa[0] - C[0]), (float)(c[1] + pa[1] - C[1]),
                                              (float)(c[2] + pa[2] - C[2]), (float)pa[3]);
  }
  for (int i = 0; i < 3; ++i) {
    const double* gi = g.geo64 + 4 * (3 * (size_t)t + i);  // c - v_i, s_i l_i
    geob32[3 * (size_t)t + i] = make_float4((float)(C[0] - c[0] + gi[0]), (float)(C[1] - c[1] + gi[1]),
                                            (float)(C[2] - c[2] + gi[2]), (float)gi[3]);
  }
}


}  // namespace

cudaError_t launch_block_frames(const GeoView& g, float4* bsph, int4* bgrid, float4* rel32, float4* geob32,
                                cudaStream_t s) {
  const int nb = (g.nt + 31) / 32;
  k_block_spheres<<<(unsigned)((nb + 3) / 4), 128, 0, s>>>(g, bsph, bgrid);
  k_block_offsets<<<(unsigned)((g.nt + 127) / 128), 128, 0, s>>>(g, bgrid, rel32, geob32);
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

// r_min, r_max into page-locked host memory mapped into the device: the host
// reads them after a stream synchronization, with no copy-engine transfer
// (which would queue behind large copies of Z on other streams).
__global__ void k_range_out(const unsigned long long* __restrict__ mm, unsigned long long* h) {
  if (threadIdx.x < 2) h[threadIdx.x] = mm[threadIdx.x];
}

cudaError_t launch_range_out(const unsigned long long* d_minmax, unsigned long long* h_range, cudaStream_t s) {
  k_range_out<<<1, 32, 0, s>>>(d_minmax, h_range);
  return cudaGetLastError();
}

cudaError_t launch_near_rows(const int64_t* near_ptr, int64_t nt, int32_t* near_row, cudaStream_t s) {
  if (nt <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)std::min<int64_t>((nt + kWarps - 1) / kWarps, (int64_t)sm_count() * 8);
  k_near_rows<<<blocks, kThreads, 0, s>>>(near_ptr, nt, near_row);
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
  const int64_t bw = std::min<int64_t>((nbp + kWarps - 1) / kWarps, (int64_t)nsm * 8);
  k_range_witness<<<(unsigned)bw, kThreads, 0, s>>>(g, d_minmax);
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


cudaError_t launch_mirror32(void* Z, int64_t ldz, int64_t ne, cudaStream_t s) {
  if (ne == 0) return cudaSuccess;
  const int64_t nb = (ne + 31) / 32;
  const int64_t blocks = std::min<int64_t>(nb * nb, (int64_t)sm_count() * 8);
  k_symmetrize32<<<(unsigned)blocks, 256, 0, s>>>((float2*)Z, ldz, (int)ne);
  return cudaGetLastError();
}

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
