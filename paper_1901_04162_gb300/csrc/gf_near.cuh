// Device code of the near-pair computations shared by the gfmom kernel files
// (sm_103a): the singular inner integrals over a source triangle (FP64, or
// FP64 geometry and static parts with FP32 sampling of e^{-jkR} on the source
// edges), their near-pair task over groups of lanes, and the 3x3 block.
#pragma once
#include "gf_device.cuh"

namespace gf {
namespace {

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

// Sign tests of FP64 values on their bits (integer compares; a DSETP takes an
// FP64 pipe slot): x > 0 and x >= 0 for finite x (-0 counts as negative in
// nonneg, which the callers' formulas for both signs agree on at zero).
__device__ __forceinline__ bool pos64(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool nonneg64(double x) { return __double_as_longlong(x) >= 0; }

struct KScal {  // per-wavenumber scalars of the near-pair fill
  double k, scale, inv_k2, inv_k;
  float q4f;      // 4 / k^2 in FP32 (the mixed-precision block assembly)
  float scale32;  // k eta in FP32 (the mixed-precision output stage)
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

// Inner integrals over source triangle v (frame fr) for observation point r,
// all in FP64 (1/(4 pi) included); dvq[c] = rho0 - v_c. The steps of the
// mixed-precision version below with FP64 samples: the frame of the source
// triangle precomputed, the vertex offsets and distances formed once and
// shared by the two edges meeting at a vertex, the static part as one log of
// one quotient per edge, the bounds of the angular substitution
// u = asinh(l / |P0|) from the in-plane vertex distances (e^u = (l + rho) / |P0|),
// and e^u at a symmetric pair of angular nodes from e^mid and e^{+-half x}.
__device__ void inner_integrals64(const double r[3], const double v[3][3], const double* __restrict__ fr,
                                  const NearArgs& A, double k, double inv_k, const TabView* te, bool use_table,
                                  C2* I0, C2 I1[3], double dvq[3][3]) {
  const double n[3] = {fr[0], fr[1], fr[2]};
  double w[3][3];  // v_c - r
  for (int c = 0; c < 3; ++c)
    for (int x = 0; x < 3; ++x) w[c][x] = v[c][x] - r[x];
  const double h = -(n[0] * w[0][0] + n[1] * w[0][1] + n[2] * w[0][2]);
  const double d = fabs(h);
  double Rv[3], rv[3];  // |r - v_c| and the in-plane |rho0 - v_c|
  for (int c = 0; c < 3; ++c) {
    Rv[c] = sqrt(w[c][0] * w[c][0] + w[c][1] * w[c][1] + w[c][2] * w[c][2]);
    double u[3];
    for (int x = 0; x < 3; ++x) {
      u[x] = fma(h, n[x], w[c][x]);  // v_c - rho0
      dvq[c][x] = -u[x];
    }
    rv[c] = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  }
  const C2 ed = exp_mjkr(k, d, te, use_table);
  double sre = 0, sim = 0;                        // scalar sector sums
  double vre[3] = {0, 0, 0}, vim[3] = {0, 0, 0};  // vector remainder
  double vst[3] = {0, 0, 0};                      // vector static part
  for (int e = 0; e < 3; ++e) {
    const int en = e == 2 ? 0 : e + 1;
    const double len = fr[3 + e];
    const double t[3] = {fr[6 + 3 * e], fr[7 + 3 * e], fr[8 + 3 * e]};
    const double mh[3] = {fr[15 + 3 * e], fr[16 + 3 * e], fr[17 + 3 * e]};
    const double* ar = w[e];  // its in-plane part differs by h n, normal to t and mh
    const double P0 = ar[0] * mh[0] + ar[1] * mh[1] + ar[2] * mh[2];
    const double lm = ar[0] * t[0] + ar[1] * t[1] + ar[2] * t[2];
    const double lp = lm + len;
    if (fabs(P0) > 1e-12 * len) {
      const double aP = fabs(P0), iaP = 1.0 / aP;
      // e^{asinh(l / aP)} = (l + rho) / aP, for l < 0 as aP / (rho - l)
      const double Em = nonneg64(lm) ? (lm + rv[e]) * iaP : aP / (rv[e] - lm);
      const double Ep = nonneg64(lp) ? (lp + rv[en]) * iaP : aP / (rv[en] - lp);
      const double um = log(Em), up = log(Ep);
      const double half = 0.5 * (up - um);
      const double Emid = sqrt(Em * Ep), iEmid = 1.0 / Emid;  // e^{+-mid}
      double cr = 0, ci = 0;
      // nodes i and nphi - 1 - i sit at mid +- half x_i (x_{n-1-i} = -x_i)
      for (int i = 0; i < (A.nphi + 1) / 2; ++i) {
        const int j = A.nphi - 1 - i;
        const double ex = exp(half * A.gx_phi[i]), iex = 1.0 / ex;
        const double chi = 0.5 * (Emid * ex + iEmid * iex), chj = 0.5 * (Emid * iex + iEmid * ex);  // cosh u
        const double q = 1.0 / (chi * chj);
        {
          const double Re = sqrt(fma(aP * chi, aP * chi, d * d));
          const C2 eR = exp_mjkr(k, Re, te, use_table);
          const double wt = A.gw_phi[i] * (chj * q);
          cr += (ed.re - eR.re) * wt;
          ci += (ed.im - eR.im) * wt;
        }
        if (j != i) {
          const double Re = sqrt(fma(aP * chj, aP * chj, d * d));
          const C2 eR = exp_mjkr(k, Re, te, use_table);
          const double wt = A.gw_phi[j] * (chi * q);
          cr += (ed.re - eR.re) * wt;
          ci += (ed.im - eR.im) * wt;
        }
      }
      const double sg = pos64(P0) ? half : -half;
      sre += cr * sg;
      sim += ci * sg;
    }
    // line integral of e^{-jkR} - 1 + jkR along the edge
    double lr = 0, li = 0;
    const double hl = 0.5 * len;
    for (int i = 0; i < A.nl; ++i) {
      const double s = hl * (A.gx_l[i] + 1.0);
      const double x0 = fma(t[0], s, ar[0]), x1 = fma(t[1], s, ar[1]), x2 = fma(t[2], s, ar[2]);
      const double R = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
      const C2 eR = exp_mjkr(k, R, te, use_table);
      lr += (eR.re - 1.0) * A.gw_l[i];
      li += (eR.im + k * R) * A.gw_l[i];
    }
    lr *= hl;
    li *= hl;
    // static part: int R dl along the edge, with Rm = |r - a|, Rp = |r - b|;
    // log(fp / fm) with fp = lp + Rp = R02 / (Rp - lp), fm = lm + Rm =
    // R02 / (Rm - lm), each in its cancellation-free form (lp >= lm), as one
    // quotient
    const double R02 = P0 * P0 + d * d;
    const double Rm = Rv[e], Rp = Rv[en];
    double st = 0.5 * (lp * Rp - lm * Rm);
    if (pos64(R02)) {
      double ratio;
      if (nonneg64(lm)) ratio = (lp + Rp) / (lm + Rm);
      else if (nonneg64(lp)) ratio = (lp + Rp) * (Rm - lm) / R02;
      else ratio = (Rm - lm) / (Rp - lp);
      st += 0.5 * R02 * log(ratio);
    }
    for (int x = 0; x < 3; ++x) {
      vre[x] += mh[x] * lr;
      vim[x] += mh[x] * li;
      vst[x] += mh[x] * st;
    }
  }
  const double c4 = 1.0 / (4.0 * kPi), ikc4 = inv_k * c4;
  // I0 = (-j/k) s / (4 pi);  I1 = ((j/k) v + v_static) / (4 pi)
  I0->re = sim * ikc4;
  I0->im = -sre * ikc4;
  for (int x = 0; x < 3; ++x) {
    I1[x].re = (vst[x] - vim[x] * inv_k) * c4;
    I1[x].im = vre[x] * ikc4;
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
// The results leave in FP32 (the caller assembles the 3x3 block in FP32):
// I0, I1 and dvq[j] = rho0 - v_j, the latter from the FP32 edge vectors
// v_j - r formed here anyway (each FP64 <-> FP32 conversion costs an FP64
// pipe slot, as much as an FP64 operation).
__device__ __forceinline__ void inner_integrals_mixed(const double r[3], const double v[3][3], const double* __restrict__ fr,
                                      const float* __restrict__ fr32, const NearArgs& A, double k, double inv_k,
                                      const Tab32& te, bool use_table, float lo, float hi, C2f* I0, C2f I1[3],
                                      float dvq[3][3]) {
  const float kpi = (float)(k / kPi), k32 = (float)k;
  const double n[3] = {fr[0], fr[1], fr[2]};
  // v_c - r, once (scalars, so that the edge loop picks them without a local
  // array): the vertex distances, h, and the edge offsets below all use them
  const double w0x = v[0][0] - r[0], w0y = v[0][1] - r[1], w0z = v[0][2] - r[2];
  const double w1x = v[1][0] - r[0], w1y = v[1][1] - r[1], w1z = v[1][2] - r[2];
  const double w2x = v[2][0] - r[0], w2y = v[2][1] - r[1], w2z = v[2][2] - r[2];
  const double h = -(n[0] * w0x + n[1] * w0y + n[2] * w0z);
  const double d = fabs(h);
  const float h32 = (float)h, nx32 = fr32[21], ny32 = fr32[22], nz32 = fr32[23];
  float d0x = 0.f, d0y = 0.f, d0z = 0.f, d1x = 0.f, d1y = 0.f, d1z = 0.f, d2x = 0.f, d2y = 0.f, d2z = 0.f;
  // |r - v_c|
  const double Rv0 = sqrt(w0x * w0x + w0y * w0y + w0z * w0z);
  const double Rv1 = sqrt(w1x * w1x + w1y * w1y + w1z * w1z);
  const double Rv2 = sqrt(w2x * w2x + w2y * w2y + w2z * w2z);
  const float d32 = (float)d;
  const float2 ed = exp32(kpi, d32, te, use_table, lo, hi);
  // the sampled (dynamic) sums carry FP32 samples: FP32 accumulation; the
  // static closed form stays in FP64
  float sre = 0.f, sim = 0.f, vre[3] = {0.f, 0.f, 0.f}, vim[3] = {0.f, 0.f, 0.f};
  double vst[3] = {0, 0, 0};
  for (int e = 0; e < 3; ++e) {
    const double len = fr[3 + e];
    const double t[3] = {fr[6 + 3 * e], fr[7 + 3 * e], fr[8 + 3 * e]};
    const double mh[3] = {fr[15 + 3 * e], fr[16 + 3 * e], fr[17 + 3 * e]};
    // v_e - r; its in-plane part v_e - rho0 differs by h n, normal to t and mh
    const double arx = e == 0 ? w0x : (e == 1 ? w1x : w2x), ary = e == 0 ? w0y : (e == 1 ? w1y : w2y),
                 arz = e == 0 ? w0z : (e == 1 ? w1z : w2z);
    const double P0 = arx * mh[0] + ary * mh[1] + arz * mh[2];
    const double lm = arx * t[0] + ary * t[1] + arz * t[2];
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
      const float sg = pos64(P0) ? half : -half;
      sre = fmaf(cr, sg, sre);
      sim = fmaf(ci, sg, sim);
    }
    // line integral of e^{-jkR} - 1 + jkR from r's position relative to a
    const float ax = (float)arx, ay = (float)ary, az = (float)arz;
    // rho0 - v_e = (r - v_e) - h n (scalars: the edge loop is not unrolled)
    const float ux = fmaf(-h32, nx32, -ax), uy = fmaf(-h32, ny32, -ay), uz = fmaf(-h32, nz32, -az);
    if (e == 0) {
      d0x = ux, d0y = uy, d0z = uz;
    } else if (e == 1) {
      d1x = ux, d1y = uy, d1z = uz;
    } else {
      d2x = ux, d2y = uy, d2z = uz;
    }
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
    if (pos64(R02)) {
      double ratio;
      if (nonneg64(lm)) ratio = (lp + Rp) / (lm + Rm);
      else if (nonneg64(lp)) ratio = (lp + Rp) * (Rm - lm) / R02;
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
  dvq[0][0] = d0x, dvq[0][1] = d0y, dvq[0][2] = d0z;
  dvq[1][0] = d1x, dvq[1][1] = d1y, dvq[1][2] = d1z;
  dvq[2][0] = d2x, dvq[2][1] = d2y, dvq[2][2] = d2z;
  const float c4 = (float)(1.0 / (4.0 * kPi)), ik = (float)inv_k, ikc4 = ik * c4;
  // I0 = (-j/k) s / (4 pi);  I1 = ((j/k) v + v_static) / (4 pi)
  I0->re = sim * ikc4;
  I0->im = -sre * ikc4;
  for (int x = 0; x < 3; ++x) {
    I1[x].re = fmaf(-vim[x], ik, (float)vst[x]) * c4;
    I1[x].im = vre[x] * ikc4;
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
  __device__ __forceinline__ void add32(int m, int n, float zr, float zi) const {  // FP32 Z only
    atomicAdd(reinterpret_cast<float2*>(Z + (int64_t)m * ldz + n), make_float2(zr, zi));
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
    // entry (i, j): w_a ((r - v_i) . J_j / 4 - I0 / k^2), J_j = I1 + (rho0 - v_j) I0;
    // w_a / 4 folded into I0, I1
    CT S, T[3];
    RT f[3][3], dvq[3][3], q4;
    if constexpr (MIXED) {
      C2f I0, I1[3];
      inner_integrals_mixed(ra, vq, g.frame64 + kFrame * (size_t)q, g.frame32 + kFrame32 * (size_t)q, A, ks.k,
                            ks.inv_k, te32, use_table, lo32, hi32, &I0, I1, dvq);
      // r_a - v_i = alpha_a + delta_i from the FP32 offsets (no conversions)
      const float4 alf = g.pts32[(size_t)sub * g.nt + p];
      const float w4 = 0.25f * alf.w;
      S = CT{w4 * I0.re, w4 * I0.im};
#pragma unroll
      for (int x = 0; x < 3; ++x) T[x] = CT{w4 * I1[x].re, w4 * I1[x].im};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float4 dl = g.geo32[3 * (size_t)p + i];  // c_p - v_i
        f[i][0] = alf.x + dl.x;
        f[i][1] = alf.y + dl.y;
        f[i][2] = alf.z + dl.z;
      }
      q4 = ks.q4f;
    } else {
      C2 I0, I1[3];
      double dv64[3][3];
      inner_integrals64(ra, vq, g.frame64 + kFrame * (size_t)q, A, ks.k, ks.inv_k, &te, use_table, &I0, I1, dv64);
      const RT w4 = (RT)(0.25 * al[3]);
      S = CT{w4 * (RT)I0.re, w4 * (RT)I0.im};
#pragma unroll
      for (int x = 0; x < 3; ++x) T[x] = CT{w4 * (RT)I1[x].re, w4 * (RT)I1[x].im};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double* vpi = g.v64 + 9 * (size_t)p + 3 * i;
        for (int x = 0; x < 3; ++x) f[i][x] = (RT)(ra[x] - vpi[x]);
      }
#pragma unroll
      for (int j = 0; j < 3; ++j)
        for (int x = 0; x < 3; ++x) dvq[j][x] = (RT)dv64[j][x];
      q4 = (RT)(4.0 * ks.inv_k2);
    }
    const CT Q = {q4 * S.re, q4 * S.im};  // w_a I0 / k^2
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      CT J[3];
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const RT dv = dvq[j][x];
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
  const double inv_area_q = MIXED ? 0.0 : g.frame64[kFrame * (size_t)q + 24];
  const float inv_area32 = MIXED ? __frcp_rn(g.cen32[q].w) : 0.f;
  const int4 ep = g.tedge[p], eq = g.tedge[q];
#pragma unroll
  for (int u = 0; u < NS; ++u) {
    if (u >= count) break;
    const int e = first + u, i = e / 3, j = e - 3 * (e / 3);
    const int ci = i == 0 ? ep.x : (i == 1 ? ep.y : ep.z), cj = j == 0 ? eq.x : (j == 1 ? eq.y : eq.z);
    if (!edge_valid(ci) || !edge_valid(cj)) continue;
    if constexpr (MIXED) {  // FP32 output: no conversions on the FP64 pipe
      const float c = ks.scale32 * g.geo32[3 * (size_t)p + i].w * g.geo32[3 * (size_t)q + j].w * inv_area32;
      sink.add32(edge_of(ci), edge_of(cj), -c * (float)fin[u].im, c * (float)fin[u].re);
    } else {
      const double slp = g.geo64[4 * (3 * (size_t)p + i) + 3], slq = g.geo64[4 * (3 * (size_t)q + j) + 3];
      const double c = ks.scale * slp * slq * inv_area_q;  // k eta s_i l_i s_j l_j / A_q
      sink.add(edge_of(ci), edge_of(cj), -c * (double)fin[u].im, c * (double)fin[u].re);
    }
  }
}

}  // namespace
}  // namespace gf
