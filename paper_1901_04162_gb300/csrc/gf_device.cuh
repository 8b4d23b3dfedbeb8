// Device code shared by the gfmom kernel files (sm_103a): the FP32 table
// lookups of Section II.C on the lattice image, the near-pair test and the
// symmetric task map, and the regular-pair computation (moments of a triangle
// pair and its 3x3 RWG block) with its sinks. The near-pair computations are
// in gf_near.cuh.
//
// Regular pairs: one warp per (test triangle p, 32 source triangles q), one
// source triangle per lane. For each test point a the lane runs over the
// source points b: R = |(c_p - c_q) + alpha_a - beta_b| (taken in split form
// from block frames), Green value from the Lagrange table (Eq. 6 hash on the
// lattice -> polynomial in s, Eq. 3 + 5 re-expanded as monomials) or from
// sincospi, and four moments M0 = sum w w G, Ma = sum w w alpha G,
// Mb = sum w w beta G, Mab = sum w w (alpha . beta) G (8 complex numbers;
// Kahan-compensated over a in FP32). The 3 x 3 RWG block:
//   Z(e_i, e_j) += jk eta/(4 pi) s_i l_i s_j l_j
//                  [ (Mab + eps_j . Ma + delta_i . Mb + (delta_i . eps_j) M0) / 4 - M0 / k^2 ]
// with delta_i = c_p - v_i, eps_j = c_q - v_j (v = vertex opposite the edge).
#pragma once
#include <cuda_fp16.h>
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

// ---------------------------------------------------------------- lookups
struct Tab32 {  // FP32 view (shared or global memory; possibly a window of the lattice)
  const float4* la;   // lattice records (c0, c1), indexed by the global cell number
  const uint32_t* lc; // c2 as half2 (Green) or the busy ordinal
  const int* busy;    // the blob: cells holding samples (ascending), their headers,
  const float4* hdr;  // sub-cells and full interval records
  const float4* sub;
  const float4* ca;
  const float4* cb;
  int n_busy;
  float vmin, vmax;   // kLatMagic + first / last cell present (the whole lattice, or a window)
  float inv, nc, h, lo, amid, c2d;
  float xscale;       // lookups at x = xscale * R (1, or k for a table in u = kR)
  // shared-memory copies: address of cell i's record = (bits of kLatMagic + i)
  // * 16 + sa_off, of its lat_c word = (bits) * 4 + sc_off (mod 2^32)
  uint32_t sa_off = 0u, sc_off = 0u;
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
  T.lc = t.lat_c;
  tab32_blob(T, t, t.lat_blob);
  T.vmin = kLatMagic;
  T.vmax = kLatMagic + (float)(t.n_lat - 1);
  T.inv = t.lat_inv;
  T.nc = t.lat_nc;
  T.h = t.lat_h;
  T.lo = t.lat_lo;
  T.amid = t.lat_amid;
  T.c2d = t.lat_c2d;
  return T;
}

// Copies a table's lattice image (records, the c2 plane for deg > 1, the
// blob) into shared memory at `smem` (all threads of the block; the caller
// synchronizes) and points T at the copy.
__device__ __forceinline__ void stage_tab32(Tab32& T, const TabView& tv, int deg, unsigned char* smem) {
  const int nl = tv.n_lat, nblob = (int)tv.blob_vec4();
  float4* sa = reinterpret_cast<float4*>(smem);
  for (int i = threadIdx.x; i < nl; i += blockDim.x) sa[i] = tv.lat_a[i];
  if (deg > 1) {
    uint32_t* sc = reinterpret_cast<uint32_t*>(sa + nl);
    for (int i = threadIdx.x; i < nl; i += blockDim.x) sc[i] = tv.lat_c[i];
    T.lc = sc;
  }
  float4* sblob = reinterpret_cast<float4*>(smem + tv.smem32_plane_bytes(deg));
  for (int i = threadIdx.x; i < nblob; i += blockDim.x) sblob[i] = tv.lat_blob[i];
  T.la = sa;
  tab32_blob(T, tv, sblob);
  const uint32_t mb = (uint32_t)__float_as_int(kLatMagic);
  T.sa_off = (uint32_t)__cvta_generic_to_shared(sa) - mb * 16u;
  T.sc_off = (uint32_t)__cvta_generic_to_shared(sa + nl) - mb * 4u;
}

// Lattice cell of R (without a conversion instruction), its index as a
// float, and the exact offset s = R - A_i from its anchor; the table builder
// repeats these float operations.
struct LatPos {
  int i;
  float s, fi;
};

__device__ __forceinline__ LatPos lat_pos(const Tab32& T, float R) {
  const float u = __fmaf_rn(R, T.inv, T.nc);
  const float v = fminf(fmaxf(__fadd_rn(u, kLatMagic), T.vmin), T.vmax);
  const float fi = __fsub_rn(v, kLatMagic);
  return LatPos{__float_as_int(v) - __float_as_int(kLatMagic), __fsub_rn(R, __fmaf_rn(fi, T.h, T.amid)), fi};
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

// The cell record's value: c0 + s c1 (+ s^2 c2 for the Green table, c2 from
// the half2 word scaled by c2d).
template <int DEG>
__device__ __forceinline__ float2 cell_value32(const Tab32& T, float s, float4 a, uint32_t c) {
  if (DEG == 1) return make_float2(fmaf(s, a.z, a.x), fmaf(s, a.w, a.y));
  __half2_raw hr;
  hr.x = (unsigned short)(c & 0xFFFFu);
  hr.y = (unsigned short)(c >> 16);
  const float2 c2 = __half22float2(__half2(hr));
  const float t = s * T.c2d;
  return make_float2(fmaf(s, fmaf(t, c2.x, a.z), a.x), fmaf(s, fmaf(t, c2.y, a.w), a.y));
}

// Branch-free part: the cell's record (the polynomial of the interval at the
// cell's middle); *slow is set when the cell holds samples, where this value
// is not to be used.
template <int DEG>
__device__ __forceinline__ float2 lookup32_fast(const Tab32& T, float R, bool* slow) {
  const LatPos q = lat_pos(T, R * T.xscale);
  const float4 a = T.la[q.i];
  const uint32_t c = DEG > 1 ? T.lc[q.i] : 0u;
  *slow = (__float_as_int(a.w) & 1) != 0;
  return cell_value32<DEG>(T, q.s, a, c);
}

// Cells holding samples: the cell's place in the busy list (its lat_c
// word), its header, the sub-cell of the offset from the cell's left end,
// then the full interval record about node32. x = x_hi + x_lo in table units
// (x_lo = 0 for an FP32 distance); the bracketing compares x_hi (at a sample
// both neighbouring polynomials take the sample value).
template <int DEG>
__device__ __forceinline__ float2 lookup32_slow_x(const Tab32& T, float xh, float xl) {
  const LatPos q = lat_pos(T, xh);
  const int ord = min(max((int)T.lc[q.i], 0), T.n_busy - 1);  // called for flagged cells only
  const float4 h = T.hdr[ord];
  const float sl = __fadd_rn(__fsub_rn(xh, __fmaf_rn(q.fi, T.h, T.lo)), xl);
  const int c = __float_as_int(h.x) + min(max(__float2int_rz(__fmul_rn(sl, h.y)), 0), __float_as_int(h.z));
  const float4 rec = T.sub[c];
  const bool up = xh >= rec.y;
  const int j = __float_as_int(rec.x) + (up ? 1 : 0);
  const float4 a = T.ca[j];
  float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
  if (DEG > 1) b = T.cb[j];
  return horner32<DEG>(__fadd_rn(xh - (up ? rec.y : rec.z), xl), a, b);
}

template <int DEG>
__device__ __forceinline__ float2 lookup32_slow(const Tab32& T, float Rr) {
  return lookup32_slow_x<DEG>(T, Rr * T.xscale, 0.f);
}

// The same at a split distance already in table units.
template <int DEG>
__device__ __forceinline__ float2 lookup32_slow(const Tab32& T, float xh, float xl) {
  return lookup32_slow_x<DEG>(T, xh, xl);
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
  int64_t bq;
  if (u < (int64_t(1) << 29)) {  // 32-bit integers and conversions (the 64-bit ones take the FP64 pipe)
    const int u32 = (int)u;
    int b = (int)((sqrtf(8.f * (float)u32 + 1.f) - 1.f) * 0.5f);
    while (b > 0 && b * (b + 1) / 2 > u32) --b;
    while ((b + 1) * (b + 2) / 2 <= u32) ++b;
    bq = b;
  } else {
    bq = (int64_t)((sqrtf(8.f * (float)u + 1.f) - 1.f) * 0.5f);
    while (bq > 0 && bq * (bq + 1) / 2 > u) --bq;
    while ((bq + 1) * (bq + 2) / 2 <= u) ++bq;
  }
  const int64_t bp = u - bq * (bq + 1) / 2;
  *p = (int)(bp * 32 + (task & 31));
  *q0 = (int)(bq * 32);
  return *p < nt;
}

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

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
  __device__ __forceinline__ void add32(int m, int n, float zr, float zi) const {  // FP32 values only
    const int64_t i = find(m, n);
    if (i >= 0) atomicAdd(reinterpret_cast<float2*>(vals + i), make_float2(zr, zi));
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

// ---------------------------------------------------------------- packed FP32 pairs
// Two FP32 lanes (re, im) in one 64-bit register for the packed FP32
// instructions of sm_100 and later (add / sub / mul / fma .f32x2, one issue
// slot for both parts, IEEE round-to-nearest in each).
typedef unsigned long long f2x;
__device__ __forceinline__ f2x pk2(float a, float b) {
  f2x r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 up2(f2x r) {
  float a, b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
  return make_float2(a, b);
}
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
  f2x d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
  f2x d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
  f2x d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
  f2x d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

struct KSum2 {  // Kahan-compensated sum of a complex number, both parts at once
  f2x s = 0ull, c = 0ull;
  __device__ __forceinline__ void add(f2x x) {
    const f2x y = sub2(x, c);
    const f2x t = add2(s, y);
    c = sub2(sub2(t, s), y);
    s = t;
  }
};

// ---------------------------------------------------------------- split distances
// The separation of the 32-triangle blocks of p and q. Block centres lie on
// a grid of step u = 2^e (bgrid, in units of u), so B = C_p - C_q is exact in
// FP32 and |B|^2 is an exact unsigned integer in units of u^2 (each
// coordinate below 2^15 units), split into two exact FP32 parts.
struct BlockSep {
  float bx, by, bz, bbh, bbl;
};

__device__ __forceinline__ BlockSep block_sep(const GeoView& g, int p, int q) {
  const int4 cp = g.bgrid[p >> 5], cq = g.bgrid[q >> 5];
  const int dx = cp.x - cq.x, dy = cp.y - cq.y, dz = cp.z - cq.z;
  const unsigned bb = (unsigned)(dx * dx) + (unsigned)(dy * dy) + (unsigned)(dz * dz);
  BlockSep s;
  s.bx = (float)dx * g.bunit;
  s.by = (float)dy * g.bunit;
  s.bz = (float)dz * g.bunit;
  s.bbh = (float)(bb & 0xFFFFFF00u) * g.bunit2;
  s.bbl = (float)(bb & 0xFFu) * g.bunit2;
  return s;
}

// R = |B + r_a - r_b| (r: point offsets from their block centres, FP32) as
// R_hi + R_lo: R^2 = |B|^2 + num with num = 2B.(r_a - r_b) + |r_a - r_b|^2 =
// A_a + B_b - 2 r_a.r_b (A_a = 2B.r_a + |r_a|^2, B_b = |r_b|^2 - 2B.r_b), all
// small terms; R_hi = FP32 sqrt of |B|_hi^2 + num, R_lo = (R^2 - R_hi^2) /
// (2 R_hi) with R_hi^2 taken exactly by an FMA. So R carries about 1e-9 lambda
// of absolute error where one FP32 number would carry ulp(R) / 2 (6e-8 at
// R = 1), and kR keeps its phase across the electrically large workloads.
struct SplitR {
  float hi, lo, rs;  // R_hi, R_lo, 1 / R (FP32)
};

__device__ __forceinline__ SplitR split_r(const BlockSep& bs, float c, float m2x, float m2y, float m2z, float bx,
                                         float by, float bz) {
  const float num = fmaf(m2x, bx, fmaf(m2y, by, fmaf(m2z, bz, c)));
  const float R2 = bs.bbh + num;
  SplitR r;
  r.rs = rsqrtf(R2);
  r.hi = R2 * r.rs;
  float e = fmaf(-r.hi, r.hi, bs.bbh);
  e += num;
  e += bs.bbl;
  r.lo = e * (0.5f * r.rs);
  // 1/R = 1/(R_hi + R_lo): rs is 1/R_hi to FP32 accuracy even where R2 lost
  // digits to the cancellation in |B|^2 + num (R much smaller than |B|)
  r.rs = fmaf(-r.lo * r.rs, r.rs, r.rs);
  return r;
}

// Table units x = xscale R as x_hi + x_lo (xscale = 1 for tables in R).
template <bool KR>
__device__ __forceinline__ void table_x(const Tab32& T, const SplitR& r, float* xh, float* xl) {
  if (!KR) {
    *xh = r.hi;
    *xl = r.lo;
  } else {
    *xh = r.hi * T.xscale;
    *xl = fmaf(r.lo, T.xscale, fmaf(r.hi, T.xscale, -*xh));
  }
}

// Fast lattice lookup at x = x_hi + x_lo: the cell from x_hi, the offset
// s = (x_hi - A_i) + x_lo (the difference exact); SM: the lattice planes in
// shared memory, addressed from the float bits of the cell index (one IMAD
// per plane). *busy: the cell holds samples (the value is then corrected).
template <int DEG, bool SM>
__device__ __forceinline__ float2 lat_fast(const Tab32& T, float xh, float xl, bool* busy) {
  const float u = __fmaf_rn(xh, T.inv, T.nc);
  const float v = fminf(fmaxf(__fadd_rn(u, kLatMagic), T.vmin), T.vmax);
  const float fi = __fsub_rn(v, kLatMagic);
  const float s = __fadd_rn(__fsub_rn(xh, __fmaf_rn(fi, T.h, T.amid)), xl);
  float4 a;
  uint32_t c = 0u;
  if (SM) {
    const uint32_t bits = __float_as_uint(v);
    asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w)
                 : "r"(bits * 16u + T.sa_off));
    if (DEG > 1) asm("ld.shared.b32 %0, [%1];" : "=r"(c) : "r"(bits * 4u + T.sc_off));
  } else {
    const int i = __float_as_int(v) - __float_as_int(kLatMagic);
    a = T.la[i];
    if (DEG > 1) c = T.lc[i];
  }
  *busy = (__float_as_uint(a.w) & 1u) != 0u;
  return cell_value32<DEG>(T, s, a, c);
}

// sincos(pi x) of x = k R / pi from the split R: the product carried exactly
// (x_hi + x_err by an FMA, plus R_lo and the FP32 residue of k / pi), x_hi
// reduced modulo 2 exactly, then CUDA's sincospif of the small argument.
__device__ __forceinline__ void sincos_kr(const SplitR& r, float kpi, float kpi_lo, float* sn, float* cs) {
  const float xh = r.hi * kpi;
  const float xl = fmaf(r.lo, kpi, fmaf(r.hi, kpi_lo, fmaf(r.hi, kpi, -xh)));
  const float n2 = __fsub_rn(__fmaf_rn(xh, 0.5f, kLatMagic), kLatMagic);
  sincospif(fmaf(-2.f, n2, xh) + xl, sn, cs);
}



template <int M, int MODE, bool KR = false, bool SM = false, bool QUEUE = false, class Sink = DenseUpper>
__device__ __forceinline__ unsigned long long regular_pair32(const GeoView& g, const Tab32& T, const RegK& K, int p,
                                                             int q, bool ok, const Sink& sink);

// No pair of the blocks of p and q0 is near when their centres are farther
// apart than the two vertex radii plus the centroid criterion (then no two
// triangles touch and no two centroids are within near_dist).
__device__ __forceinline__ bool blocks_apart(const GeoView& g, int p, int q0) {
  const int4 a = g.bgrid[p >> 5], b = g.bgrid[q0 >> 5];
  const float dx = (float)(a.x - b.x) * g.bunit, dy = (float)(a.y - b.y) * g.bunit, dz = (float)(a.z - b.z) * g.bunit;
  const float lim = __int_as_float(a.w) + __int_as_float(b.w) + g.near_dist32 * 1.0001f + 1e-6f;
  return dx * dx + dy * dy + dz * dz > lim * lim * 1.0001f;
}

// One warp task: test triangle p, source triangles q0 .. q0 + 31 (q0 a
// multiple of 32, one block). QUEUE: returns the lane's flagged point pairs
// (bit a M + b: the lattice cell of that distance holds samples) instead of
// correcting them; the caller lists them for fix_entry32.
template <int M, int MODE, bool KR, bool SM, bool QUEUE = false, class Sink>
__device__ __forceinline__ unsigned long long regular_task32(const GeoView& g, const Tab32& T, const RegK& K,
                                                             const Sink& sink, int p, int q0, int lane) {
  const int q = min(q0 + lane, g.nt - 1);
  bool ok = (q0 + lane < g.nt) && q > p;
  if (!blocks_apart(g, p, q0)) {
    const float4 cp = g.cen32[p], cq = g.cen32[q];
    const float3 dc = make_float3(cp.x - cq.x, cp.y - cq.y, cp.z - cq.z);
    ok = ok && !pair_is_near(g, p, q, g.tvert[p], g.tvert[q], dc);
  }
  return regular_pair32<M, MODE, KR, SM, QUEUE>(g, T, K, p, q, ok, sink);
}

// The 3x3 block of pair (p, q) from its moments (packed complex pairs), handed
// to `sink`: Z(e_i, e_j) += j scale s_i l_i s_j l_j [X_j + delta_i . Y_j / 4]
// with X_j = (Mab + eps'_j . Ma) / 4 - M0 / k^2 and Y_j = Mb + eps'_j M0.
template <class Sink>
__device__ __forceinline__ void pair_block32(const GeoView& g, const RegK& K, int p, int q, f2x M0, const f2x* Ma,
                                             const f2x* Mb, f2x Mab, const Sink& sink) {
  const int4 ep = g.tedge[p], eq = g.tedge[q];
  const int ecp[3] = {ep.x, ep.y, ep.z}, ecq[3] = {eq.x, eq.y, eq.z};
  // (packed pairs: both parts of each complex number in one instruction)
  const f2x m0k = mul2(M0, pk2(-K.inv_k2, -K.inv_k2));
  f2x xj[3], yj[3][3];
  float sl[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float4 gq = g.geob32[3 * (size_t)q + j];  // eps'_j, s_j l_j
    const float e[3] = {gq.x, gq.y, gq.z};
    f2x er = Mab;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const f2x ec = pk2(e[c], e[c]);
      er = fma2(ec, Ma[c], er);
      yj[j][c] = fma2(ec, M0, Mb[c]);
    }
    xj[j] = fma2(pk2(0.25f, 0.25f), er, m0k);
    sl[j] = gq.w;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (!edge_valid(ecp[i])) continue;
    const float4 gp = g.geo32[3 * (size_t)p + i];  // delta_i, s_i l_i
    const f2x d0 = pk2(0.25f * gp.x, 0.25f * gp.x), d1 = pk2(0.25f * gp.y, 0.25f * gp.y),
              d2 = pk2(0.25f * gp.z, 0.25f * gp.z);
    const float ci = K.scale * gp.w;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (!edge_valid(ecq[j])) continue;
      const float2 bz = up2(fma2(d0, yj[j][0], fma2(d1, yj[j][1], fma2(d2, yj[j][2], xj[j]))));
      const float c = ci * sl[j];
      // j * c * (br + j bi) = c * (-bi + j br)
      sink(edge_of(ecp[i]), edge_of(ecq[j]), make_float2(-c * bz.y, c * bz.x));
    }
  }
}

// Point pair (test point a of p, source point b of q) whose lattice cell holds
// samples: the exact table value minus the cell polynomial the loop used (the
// same float operations for R as the loop), times the weights: the increment
// d of M0 (those of Ma, Mb, Mab are d alpha, d beta, d alpha.beta; everything
// is linear in the Green value). al, rb: the two points (offsets, weights).
template <int M, int MODE, bool KR, bool SM>
__device__ __forceinline__ f2x flagged_value32(const GeoView& g, const Tab32& T, const BlockSep& bs, int p, int q,
                                               int a, int b, float4* al_out, float4* rb_out) {
  const float4 ra = g.rel32[(size_t)a * g.nt + p];
  const float4 al = g.pts32[(size_t)a * g.nt + p];
  const float4 rb = g.rel32[(size_t)b * g.nt + q];
  const float Aa = fmaf(2.f * bs.bx, ra.x, fmaf(2.f * bs.by, ra.y, fmaf(2.f * bs.bz, ra.z,
                                                                            fmaf(ra.x, ra.x, fmaf(ra.y, ra.y, ra.z * ra.z)))));
  const float bqb = fmaf(rb.x, rb.x - 2.f * bs.bx, fmaf(rb.y, rb.y - 2.f * bs.by, rb.z * (rb.z - 2.f * bs.bz)));
  const SplitR R = split_r(bs, Aa + bqb, -2.f * ra.x, -2.f * ra.y, -2.f * ra.z, rb.x, rb.y, rb.z);
  float xh, xl;
  table_x<KR>(T, R, &xh, &xl);
  constexpr int D = MODE == kLagrange ? 3 : 1;
  bool busy;
  const float2 fa = lat_fast<D, SM>(T, xh, xl, &busy);
  const float2 fe = busy ? lookup32_slow<D>(T, xh, xl) : fa;
  const float w = al.w * (MODE == kLagrange ? rb.w : rb.w * R.rs);
  *al_out = al;
  *rb_out = rb;
  return pk2((fe.x - fa.x) * w, (fe.y - fa.y) * w);
}

// The 3x3 block of regular pair (p, q) (q per lane; lanes with ok == false
// take part in the warp's work but write nothing), handed to `sink`. Source
// points enter through their offsets r_b from q's block centre (rel32): the
// source moments are taken about that centre, and the block formula uses
// eps'_j = C_b(q) - v_j (geob32) in place of eps_j = c_q - v_j (the same sums:
// r_b + eps'_j = beta_b + eps_j). Point pairs in lattice cells holding
// samples are corrected here after the loop, or (QUEUE) returned as a bit
// mask (bit a M + b) for the caller to list.
template <int M, int MODE, bool KR, bool SM, bool QUEUE, class Sink>
__device__ __forceinline__ unsigned long long regular_pair32(const GeoView& g, const Tab32& T, const RegK& K, int p,
                                                             int q, bool ok, const Sink& sink) {
  if (!__any_sync(0xffffffffu, ok)) return 0ull;
  const BlockSep bs = block_sep(g, p, q);
  // w_b r_b kept in registers for small rules in the kernels of 256-thread
  // CTAs; SM (the lattice in shared memory, or in direct mode one wide CTA per
  // SM) spends those registers on resident warps instead (28 warps at 72
  // registers for the 4-point rule)
  constexpr bool kWQ = M <= 4 && !SM;
  float rx[M], ry[M], rz[M], wb[M], bq[M];
#pragma unroll
  for (int b = 0; b < M; ++b) {
    const float4 r = g.rel32[(size_t)b * g.nt + q];
    rx[b] = r.x;
    ry[b] = r.y;
    rz[b] = r.z;
    wb[b] = r.w;
    bq[b] = fmaf(r.x, r.x - 2.f * bs.bx, fmaf(r.y, r.y - 2.f * bs.by, r.z * (r.z - 2.f * bs.bz)));
  }
  float wqx[kWQ ? M : 1], wqy[kWQ ? M : 1], wqz[kWQ ? M : 1];
  if (kWQ) {
#pragma unroll
    for (int b = 0; b < M; ++b) {
      wqx[b] = wb[b] * rx[b];
      wqy[b] = wb[b] * ry[b];
      wqz[b] = wb[b] * rz[b];
    }
  }
  KSum2 M0, Ma[3], Mb[3], Mab;
  static_assert(M <= 8, "point pairs are flagged in one 64-bit word");
  // point pairs (bit a M + b) whose lattice cell holds samples: 32 bits for
  // rules of up to 5 points; the test-point loop unrolled for up to 4
  using Mask = typename std::conditional<(M * M <= 32), unsigned, unsigned long long>::type;
  constexpr int kUnrollA = M <= 4 ? M : 1;
  Mask emask = 0;
#pragma unroll kUnrollA
  for (int a = 0; a < M; ++a) {
    const float4 ra = g.rel32[(size_t)a * g.nt + p];  // test point: offset from p's block centre
    const float4 al = g.pts32[(size_t)a * g.nt + p];  // offset from p's centroid, weight
    const float Aa = fmaf(2.f * bs.bx, ra.x, fmaf(2.f * bs.by, ra.y, fmaf(2.f * bs.bz, ra.z,
                                                                              fmaf(ra.x, ra.x, fmaf(ra.y, ra.y, ra.z * ra.z)))));
    const float m2x = -2.f * ra.x, m2y = -2.f * ra.y, m2z = -2.f * ra.z;
    float s0r = 0.f, s0i = 0.f, sqr[3] = {0.f, 0.f, 0.f}, sqi[3] = {0.f, 0.f, 0.f};
    unsigned rowbits = 0;
#pragma unroll
    for (int b = 0; b < M; ++b) {
      const SplitR R = split_r(bs, Aa + bq[b], m2x, m2y, m2z, rx[b], ry[b], rz[b]);
      float gr, gi;  // e^{-jkR}/R
      if (MODE == kDirect) {
        float sn, cs;
        sincos_kr(R, K.kpi, K.kpi_lo, &sn, &cs);
        gr = cs * R.rs;
        gi = -sn * R.rs;
      } else {
        float xh, xl;
        table_x<KR>(T, R, &xh, &xl);
        bool busy;
        const float2 f = lat_fast<MODE == kLagrange ? 3 : 1, SM>(T, xh, xl, &busy);
        if (busy) rowbits |= 1u << b;
        if (MODE == kLagrange) {
          gr = f.x;
          gi = f.y;
        } else {  // e^{-jkR} times 1/R
          gr = f.x * R.rs;
          gi = f.y * R.rs;
        }
      }
      if (kWQ) {
        s0r = fmaf(wb[b], gr, s0r);
        s0i = fmaf(wb[b], gi, s0i);
        sqr[0] = fmaf(wqx[b], gr, sqr[0]);
        sqi[0] = fmaf(wqx[b], gi, sqi[0]);
        sqr[1] = fmaf(wqy[b], gr, sqr[1]);
        sqi[1] = fmaf(wqy[b], gi, sqi[1]);
        sqr[2] = fmaf(wqz[b], gr, sqr[2]);
        sqi[2] = fmaf(wqz[b], gi, sqi[2]);
      } else {
        const float wr = wb[b] * gr, wi = wb[b] * gi;
        s0r += wr;
        s0i += wi;
        sqr[0] = fmaf(rx[b], wr, sqr[0]);
        sqi[0] = fmaf(rx[b], wi, sqi[0]);
        sqr[1] = fmaf(ry[b], wr, sqr[1]);
        sqi[1] = fmaf(ry[b], wi, sqi[1]);
        sqr[2] = fmaf(rz[b], wr, sqr[2]);
        sqi[2] = fmaf(rz[b], wi, sqi[2]);
      }
    }
    if (MODE != kDirect) emask |= (Mask)rowbits << (M * a);
    // outer sums over the test points, Kahan-compensated (both parts at once)
    const f2x wa2 = pk2(al.w, al.w);
    const f2x s0 = pk2(s0r, s0i);
    M0.add(mul2(s0, wa2));
    const float wal[3] = {al.w * al.x, al.w * al.y, al.w * al.z};
    f2x xab = 0ull;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const f2x wl = pk2(wal[c], wal[c]);
      const f2x sq = pk2(sqr[c], sqi[c]);
      Ma[c].add(mul2(s0, wl));
      Mb[c].add(mul2(sq, wa2));
      xab = fma2(sq, wl, xab);
    }
    Mab.add(xab);
  }
  if (!QUEUE && MODE != kDirect && __any_sync(0xffffffffu, emask != 0)) {
    // exact values where the lattice cell holds samples: add (exact - cell
    // polynomial) to the moments of those point pairs only
    while (emask) {
      const int bit = sizeof(Mask) == 4 ? __ffs((int)emask) - 1 : __ffsll((long long)emask) - 1;
      emask &= emask - 1;
      const int a = bit / M, b = bit - M * (bit / M);
      float4 al, rb;
      const f2x d = flagged_value32<M, MODE, KR, SM>(g, T, bs, p, q, a, b, &al, &rb);
      M0.add(d);
      const float alv[3] = {al.x, al.y, al.z}, rbv[3] = {rb.x, rb.y, rb.z};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Ma[c].add(mul2(d, pk2(alv[c], alv[c])));
        Mb[c].add(mul2(d, pk2(rbv[c], rbv[c])));
      }
      const float ab = al.x * rb.x + al.y * rb.y + al.z * rb.z;
      Mab.add(mul2(d, pk2(ab, ab)));
    }
  }
  if (!ok) return 0ull;
  const f2x ma[3] = {Ma[0].s, Ma[1].s, Ma[2].s}, mb[3] = {Mb[0].s, Mb[1].s, Mb[2].s};
  pair_block32(g, K, p, q, M0.s, ma, mb, Mab.s, sink);
  return QUEUE ? (unsigned long long)emask : 0ull;
}

// The 3x3 block of one flagged point pair's correction d (exact - cell
// value, times the weights): moments d, d alpha, d beta, d alpha.beta.
template <class Sink>
__device__ __forceinline__ void fix_block32(const GeoView& g, const RegK& K, int p, int q, f2x d, float4 al,
                                            float4 rb, const Sink& sink) {
  const f2x ma[3] = {mul2(d, pk2(al.x, al.x)), mul2(d, pk2(al.y, al.y)), mul2(d, pk2(al.z, al.z))};
  const f2x mb[3] = {mul2(d, pk2(rb.x, rb.x)), mul2(d, pk2(rb.y, rb.y)), mul2(d, pk2(rb.z, rb.z))};
  const float ab = al.x * rb.x + al.y * rb.y + al.z * rb.z;
  pair_block32(g, K, p, q, d, ma, mb, mul2(d, pk2(ab, ab)), sink);
}

// Flagged point pairs of the QUEUE kernels: entries (p, q << 6 | a M + b) in
// per-CTA lists (GeoView::fix), corrected by a second kernel with every
// thread busy, each as a pair block of its own added to Z (the loop's moments
// are left as they are: everything is linear in the Green value).
template <int M, int MODE, bool KR, bool SM, class Sink>
__device__ __forceinline__ void fix_entry32(const GeoView& g, const Tab32& T, const RegK& K, const Sink& sink,
                                            int2 e) {
  const int p = e.x, q = e.y >> 6, bit = e.y & 63;
  const int a = bit / M, b = bit - M * (bit / M);
  const BlockSep bs = block_sep(g, p, q);
  float4 al, rb;
  const f2x d = flagged_value32<M, MODE, KR, SM>(g, T, bs, p, q, a, b, &al, &rb);
  fix_block32(g, K, p, q, d, al, rb, sink);
}

// The tasks of a CTA whose list overflowed are scanned again: every point
// pair's distance and cell as in the loop, the flagged ones corrected at once.
template <int M, int MODE, bool KR, bool SM, class Sink>
__device__ __forceinline__ void fix_rescan32(const GeoView& g, const Tab32& T, const RegK& K, const Sink& sink,
                                             int p, int q0, int lane) {
  const int q = min(q0 + lane, g.nt - 1);
  bool ok = (q0 + lane < g.nt) && q > p;
  if (!blocks_apart(g, p, q0)) {
    const float4 cp = g.cen32[p], cq = g.cen32[q];
    const float3 dc = make_float3(cp.x - cq.x, cp.y - cq.y, cp.z - cq.z);
    ok = ok && !pair_is_near(g, p, q, g.tvert[p], g.tvert[q], dc);
  }
  if (!ok) return;
  const BlockSep bs = block_sep(g, p, q);
  for (int a = 0; a < M; ++a)
    for (int b = 0; b < M; ++b) {
      float4 al, rb;
      const f2x d = flagged_value32<M, MODE, KR, SM>(g, T, bs, p, q, a, b, &al, &rb);
      if (d != 0ull) fix_block32(g, K, p, q, d, al, rb, sink);
    }
}

inline int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

inline int64_t pair_grid(const GeoView& g, int blocks_per_sm) {
  const int64_t ntask = regular_units(g.nt);
  int64_t blocks = (ntask + kWarps - 1) / kWarps;
  return std::min<int64_t>(blocks, (int64_t)sm_count() * blocks_per_sm);
}
}  // namespace
}  // namespace gf
