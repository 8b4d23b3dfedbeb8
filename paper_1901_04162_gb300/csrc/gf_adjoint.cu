// gfmom adjoint kernels for sm_103a: dL/d(vertex coordinates) and dL/dk of
// L = Re(sum conj(gZ) Z) for regular pairs (reverse mode, table values
// recomputed) and near pairs (reverse or forward mode through the singular
// scheme), with their launcher.
#include "gf_near.cuh"

namespace gf {
namespace {

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

template <int M, bool TABLE, bool SM>
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
  // (gathered once: 18 scattered loads per pair)
  float hr_[3][3], hi_[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      hr_[i][j] = hi_[i][j] = 0.f;
      if (ok && edge_valid(ecp[i]) && edge_valid(ecq[j])) {
        const float2 z1 = gZ[(int64_t)edge_of(ecp[i]) * ldg + edge_of(ecq[j])];
        const float2 z2 = gZ[(int64_t)edge_of(ecq[j]) * ldg + edge_of(ecp[i])];
        const float c = kappa * gp[i].w * gq[j].w;
        hr_[i][j] = c * (z1.y + z2.y);
        hi_[i][j] = c * (z1.x + z2.x);
      }
    }
  auto h_of = [&](int i, int j, float* hr, float* hi) {
    *hr = hr_[i][j];
    *hi = hi_[i][j];
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
  // point pairs (bit a M + b) whose lattice cell holds samples
  using Mask = typename std::conditional<(M * M <= 32), unsigned, unsigned long long>::type;
  Mask emask = 0;
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
    unsigned rowbits = 0;  // flagged point pairs of this test point
#pragma unroll
    for (int b = 0; b < M; ++b) {
      const float rx = ux - beta[b].x, ry = uy - beta[b].y, rz = uz - beta[b].z;
      const float R2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
      const float rs = rsqrtf(R2);
      const float R = R2 * rs;
      float Fr, Fi;
      if (TABLE) {  // the lattice value; point pairs whose cell holds samples are corrected below
        bool busy;
        const float2 f = SM ? lat_fast<3, true>(T, R * T.xscale, 0.f, &busy) : lookup32_fast<3>(T, R, &busy);
        if (busy) rowbits |= 1u << b;
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
    if (TABLE) emask |= (Mask)rowbits << (M * a);
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
  if (TABLE && __any_sync(0xffffffffu, emask != 0)) {
    // every term above is linear in F (and F' = -(jk + 1/R) F): the flagged
    // point pairs add the same terms for dF = exact - lattice value, with the
    // same float operations for R as the loop above
    while (emask) {
      const int bit = sizeof(Mask) == 4 ? __ffs((int)emask) - 1 : __ffsll((long long)emask) - 1;
      emask &= emask - 1;
      const int a = bit / M, b = bit - M * (bit / M);
      const float4 al = g.pts32[(size_t)a * g.nt + p];
      const float4 bb = g.pts32[(size_t)b * g.nt + q];
      const float alv[3] = {al.x, al.y, al.z}, bv[3] = {bb.x, bb.y, bb.z};
      const float ux = dc.x + al.x, uy = dc.y + al.y, uz = dc.z + al.z;
      const float rx = ux - bb.x, ry = uy - bb.y, rz = uz - bb.z;
      const float R2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
      const float rs = rsqrtf(R2);
      const float R = R2 * rs;
      bool busy;
      const float2 fa = SM ? lat_fast<3, true>(T, R * T.xscale, 0.f, &busy) : lookup32_fast<3>(T, R, &busy);
      const float2 fe = lookup32_slow<3>(T, R * T.xscale, 0.f);
      const float Fr = fe.x - fa.x, Fi = fe.y - fa.y;
      const float Kar = A0r + Aar[0] * al.x + Aar[1] * al.y + Aar[2] * al.z;
      const float Kai = A0i + Aai[0] * al.x + Aai[1] * al.y + Aai[2] * al.z;
      float Kbr[3], Kbi[3];
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        Kbr[x] = Abr[x] + Aabr * alv[x];
        Kbi[x] = Abi[x] + Aabi * alv[x];
      }
      const float ww = al.w * bb.w;
      const float Kr = Kar + Kbr[0] * bv[0] + Kbr[1] * bv[1] + Kbr[2] * bv[2];
      const float Ki = Kai + Kbi[0] * bv[0] + Kbi[1] * bv[1] + Kbi[2] * bv[2];
      const float Fpr = -Fr * rs + k * Fi, Fpi = -Fi * rs - k * Fr;
      const float t1 = ww * re_mul(Kr, Ki, Fpr, Fpi) * rs;
      const float wFr = ww * Fr, wFi = ww * Fi;
      float gA[3], gBb[3];
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        gA[x] = re_mul(wFr, wFi, Aar[x] + Aabr * bv[x], Aai[x] + Aabi * bv[x]);
        gBb[x] = re_mul(wFr, wFi, Kbr[x], Kbi[x]);
      }
      const float gR[3] = {t1 * rx, t1 * ry, t1 * rz};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float la = bw.l[a][c], lb = bw.l[b][c];
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          dp[c][x] += la * gR[x] + (la - (1.f / 3.f)) * gA[x];
          dq[c][x] += -lb * gR[x] + (lb - (1.f / 3.f)) * gBb[x];
        }
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

template <int M, bool TABLE, bool SM>
__global__ void __launch_bounds__(256) k_adjoint_regular32(GeoView g, TabView tv, float k, float kappa, float inv_k2,
                                                           BaryF bw, const float2* __restrict__ gZ, int64_t ldg,
                                                           double* dtri, double* dkacc) {
  extern __shared__ __align__(16) unsigned char smem[];
  Tab32 T = tab32(tv);
  if (SM) {
    stage_tab32(T, tv, 3, smem);
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const int64_t ntask = regular_units(g.nt);
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t task = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < ntask; task += nwarp) {
    int p, q0;
    if (sym_task(task, g.nt, &p, &q0))
      regular_adjoint_task32<M, TABLE, SM>(g, T, k, kappa, inv_k2, bw, gZ, ldg, dtri, dkacc, p, q0, lane);
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
// frp, frq: the triangles' source frames (unit normal, edge lengths, unit
// tangents, in-plane edge normals, 1/area, 1/edge lengths); their values
// enter the forward pass, and the reverse pass maps the frames' adjoints back
// to the vertices. Reciprocals are formed once and shared by the forward
// pass and the reverse one (an FP64 divide costs a dozen FP64 operations).
__device__ void near_point_adjoint(const double vp[3][3], const double vq[3][3], const double* __restrict__ frp,
                                   const double* __restrict__ frq, const float lb[3], double wa, const NearArgs& A,
                                   double k, double ik, float kpi, double eta, const Tab32& te, bool use_table,
                                   float lo, float hi, const int ecp[3], const int ecq[3],
                                   const float2* __restrict__ gZ, int64_t ldg, double gp[3][3], double gq[3][3],
                                   double* gk) {
  const float k32 = (float)k;
  double r[3];
  for (int x = 0; x < 3; ++x) r[x] = (double)lb[0] * vp[0][x] + (double)lb[1] * vp[1][x] + (double)lb[2] * vp[2][x];
  const double n[3] = {frq[0], frq[1], frq[2]};
  // ---- projection, vertex distances (with their reciprocals), e^{-jkd}
  const double rv0[3] = {r[0] - vq[0][0], r[1] - vq[0][1], r[2] - vq[0][2]};
  const double h = dot3(n, rv0), d = fabs(h);
  double rho0[3];
  for (int x = 0; x < 3; ++x) rho0[x] = r[x] - h * n[x];
  double Rv[3], iRv[3];
  for (int c = 0; c < 3; ++c) {
    const double dx = vq[c][0] - r[0], dy = vq[c][1] - r[1], dz = vq[c][2] - r[2];
    const double s2 = dx * dx + dy * dy + dz * dz;  // > 0: r is inside p, off q's vertices
    iRv[c] = rsqrt(s2);
    Rv[c] = s2 * iRv[c];
  }
  const float d32 = (float)d;
  const float2 ed = exp32(kpi, d32, te, use_table, lo, hi);
  // ---- forward: the per-edge sums; the static part's value and its partial
  // derivatives in (l+, l-, R+, R-, R0^2) kept for the reverse pass
  double sre = 0, sim = 0, vre[3] = {0, 0, 0}, vim[3] = {0, 0, 0}, vst[3] = {0, 0, 0};
  double st_[3], s_lp[3], s_lm[3], s_Rp[3], s_Rm[3], s_R02[3];
  float cr_[3], ci_[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int en = e == 2 ? 0 : e + 1;
    const double len = frq[3 + e];
    const double* t = frq + 6 + 3 * e;
    const double* m = frq + 15 + 3 * e;
    const double ar[3] = {vq[e][0] - rho0[0], vq[e][1] - rho0[1], vq[e][2] - rho0[2]};
    const double P0 = dot3(ar, m), lm = dot3(ar, t), lp = lm + len;
    cr_[e] = ci_[e] = 0.f;
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
      cr_[e] = cr;
      ci_[e] = ci;
      const double sg = P0 > 0 ? (double)half : -(double)half;
      sre += (double)cr * sg;
      sim += (double)ci * sg;
    }
    const float ax = (float)(vq[e][0] - r[0]), ay = (float)(vq[e][1] - r[1]), az = (float)(vq[e][2] - r[2]);
    const float tx = (float)t[0], ty = (float)t[1], tz = (float)t[2];
    const float hl = 0.5f * (float)len;
    float lr = 0.f, li = 0.f;
    for (int i = 0; i < A.nl; ++i) {
      const float sp = hl * (A.fx_l[i] + 1.0f);
      const float x0 = fmaf(tx, sp, ax), x1 = fmaf(ty, sp, ay), x2 = fmaf(tz, sp, az);
      const float R = sqrtf(fmaf(x0, x0, fmaf(x1, x1, x2 * x2)));
      const float2 eR = exp32(kpi, R, te, use_table, lo, hi);
      lr = fmaf(eR.x - 1.0f, A.fw_l[i], lr);
      li = fmaf(fmaf(k32, R, eR.y), A.fw_l[i], li);
    }
    const double lrd = (double)lr * (0.5 * len), lid = (double)li * (0.5 * len);
    // static part st = (l+ R+ - l- R-) / 2 + R0^2 / 2 (log F+ - log F-), F = l + R
    // (for l < 0 in its cancellation-free form R0^2 / (R - l)), one log of
    // one quotient; d log F / d l = +-1 / (R +- l), d / dR likewise
    const double R02 = P0 * P0 + d * d;
    const double Rm = Rv[e], Rp = Rv[en];
    double st = 0.5 * (lp * Rp - lm * Rm);
    double slp = 0.5 * Rp, slm = -0.5 * Rm, sRp = 0.5 * lp, sRm = -0.5 * lm, sR02 = 0.0;
    if (R02 > 0) {
      const double Fp = lp >= 0 ? lp + Rp : Rp - lp, Fm = lm >= 0 ? lm + Rm : Rm - lm;
      const double ip = 1.0 / Fp, im = 1.0 / Fm, hR = 0.5 * R02;
      double ratio;
      if (lm >= 0) {
        ratio = Fp * im;
      } else if (lp >= 0) {
        ratio = Fp * Fm / R02;
        sR02 = -0.5;  // R0^2 / 2 times d(-log R0^2)/d R0^2
      } else {
        ratio = Fm * ip;
      }
      const double Lg = log(ratio);
      st += hR * Lg;
      sR02 += 0.5 * Lg;
      slp += hR * ip;
      sRp += lp >= 0 ? hR * ip : -hR * ip;
      slm -= hR * im;
      sRm += lm >= 0 ? -hR * im : hR * im;
    }
    st_[e] = st;
    s_lp[e] = slp;
    s_lm[e] = slm;
    s_Rp[e] = sRp;
    s_Rm[e] = sRm;
    s_R02[e] = sR02;
    for (int x = 0; x < 3; ++x) {
      vre[x] += m[x] * lrd;
      vim[x] += m[x] * lid;
      vst[x] += m[x] * st;
    }
  }
  const double c4 = 1.0 / (4.0 * kPi);
  const double I0r = sim * ik * c4, I0i = -sre * ik * c4;
  double I1r[3], I1i[3];
  for (int x = 0; x < 3; ++x) {
    I1r[x] = (vst[x] - vim[x] * ik) * c4;
    I1i[x] = vre[x] * ik * c4;
  }
  // ---- assembly: values and adjoints of I0, I1, rho0, r, p's vertices, A_q, k.
  // The 3x3 block and its adjoint are products and sums of smooth quantities
  // of the size of a triangle: FP32 (as in the forward fill), with the FP64
  // inputs converted once and the FP32 adjoints added back into the FP64
  // accumulators once (every FP64 <-> FP32 conversion takes an FP64 pipe slot).
  double bI0r = 0, bI0i = 0, bI1r[3] = {0, 0, 0}, bI1i[3] = {0, 0, 0}, brho[3] = {0, 0, 0}, br[3] = {0, 0, 0};
  double bk = 0, bik2 = 0, bA = 0;
  const double ik2 = ik * ik, iAq = frq[24];
  // per source edge j (from v_{j+1} to v_{j+2}: frame edge j + 1): s_j l_j and
  // rho0 - v_j; the adjoint of s_j l_j is summed over i and applied once
  float dvj[3][3], sljf[3], bslj[3] = {0.f, 0.f, 0.f};
  for (int j = 0; j < 3; ++j) {
    const int j1 = j == 2 ? 0 : j + 1;
    sljf[j] = (float)((ecq[j] & 1) ? -frq[3 + j1] : frq[3 + j1]);
    for (int x = 0; x < 3; ++x) dvj[j][x] = (float)(rho0[x] - vq[j][x]);
  }
  const float I0rf = (float)I0r, I0if = (float)I0i, ik2f = (float)ik2;
  const float I1rf[3] = {(float)I1r[0], (float)I1r[1], (float)I1r[2]};
  const float I1if[3] = {(float)I1i[0], (float)I1i[1], (float)I1i[2]};
  const float kewa = (float)(k * eta * wa * iAq);
  float fbI0r = 0.f, fbI0i = 0.f, fbI1r[3] = {0.f, 0.f, 0.f}, fbI1i[3] = {0.f, 0.f, 0.f};
  float fbrho[3] = {0.f, 0.f, 0.f}, fgq[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}}, fbik2 = 0.f;
  for (int i = 0; i < 3; ++i) {
    if (!edge_valid(ecp[i])) continue;
    const int i1 = i == 2 ? 0 : i + 1, i2 = i1 == 2 ? 0 : i1 + 1;
    const double li_ = frp[3 + i1], ili = frp[25 + i1];
    const float f[3] = {(float)(r[0] - vp[i][0]), (float)(r[1] - vp[i][1]), (float)(r[2] - vp[i][2])};
    const float slif = (float)((ecp[i] & 1) ? -li_ : li_);
    float bf[3] = {0.f, 0.f, 0.f}, bcsum = 0.f;
    for (int j = 0; j < 3; ++j) {
      if (!edge_valid(ecq[j])) continue;
      const float* dv = dvj[j];
      float Jr[3], Ji[3];
      for (int x = 0; x < 3; ++x) {
        Jr[x] = fmaf(dv[x], I0rf, I1rf[x]);
        Ji[x] = fmaf(dv[x], I0if, I1if[x]);
      }
      const float tr = 0.25f * (f[0] * Jr[0] + f[1] * Jr[1] + f[2] * Jr[2]) - I0rf * ik2f;
      const float ti = 0.25f * (f[0] * Ji[0] + f[1] * Ji[1] + f[2] * Ji[2]) - I0if * ik2f;
      const float c = kewa * slif * sljf[j];
      const float2 gz = gZ[(int64_t)edge_of(ecp[i]) * ldg + edge_of(ecq[j])];
      // L = gz.x (-c ti) + gz.y (c tr)
      const float btr = gz.y * c, bti = -gz.x * c;
      const float bc = gz.y * tr - gz.x * ti;
      for (int x = 0; x < 3; ++x) {
        bf[x] += 0.25f * (btr * Jr[x] + bti * Ji[x]);
        const float bJr = 0.25f * btr * f[x], bJi = 0.25f * bti * f[x];
        fbI1r[x] += bJr;
        fbI1i[x] += bJi;
        const float bdv = bJr * I0rf + bJi * I0if;
        fbI0r += bJr * dv[x];
        fbI0i += bJi * dv[x];
        fbrho[x] += bdv;
        fgq[j][x] -= bdv;
      }
      fbI0r -= btr * ik2f;
      fbI0i -= bti * ik2f;
      fbik2 -= btr * I0rf + bti * I0if;
      // c = k eta wa sl_i sl_j / A_q: bc c is the adjoint of log c, shared by its factors
      const float bcc = bc * c;
      bcsum += bcc;
      bslj[j] += bcc;  // becomes the adjoint of s_j l_j below
    }
    // log c = log k + log sl_i + log sl_j - log A_q + const; d l_i / d v_{i2} = e_i / l_i
    const double bcs = (double)bcsum;
    bk += bcs * ik;
    bA -= bcs * iAq;
    const double gsi = bcs * ili * ili;
    for (int x = 0; x < 3; ++x) {
      br[x] += (double)bf[x];
      gp[i][x] -= (double)bf[x];
      const double g = gsi * (vp[i2][x] - vp[i1][x]);
      gp[i2][x] += g;
      gp[i1][x] -= g;
    }
  }
  bI0r = (double)fbI0r;
  bI0i = (double)fbI0i;
  bik2 = (double)fbik2;
  for (int x = 0; x < 3; ++x) {
    bI1r[x] = (double)fbI1r[x];
    bI1i[x] = (double)fbI1i[x];
    brho[x] = (double)fbrho[x];
    for (int j = 0; j < 3; ++j) gq[j][x] += (double)fgq[j][x];
  }
  for (int j = 0; j < 3; ++j) {
    if (!edge_valid(ecq[j])) continue;
    const int j1 = j == 2 ? 0 : j + 1, j2 = j1 == 2 ? 0 : j1 + 1;
    // the adjoint of s_j l_j is (sum bc c) / (s_j l_j); d l_j / d v_{j2} = e_j / l_j
    const double ilj = frq[25 + j1];
    const double g0 = (double)bslj[j] * ilj * ilj;
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
  // ---- reverse of the edges (the sampled sums recomputed)
  double bd = 0, bRv[3] = {0, 0, 0}, bt[3][3], bm[3][3], blen[3];
  float bedr = 0.f, bedi = 0.f;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int en = e == 2 ? 0 : e + 1;
    const double len = frq[3 + e];
    const double* t = frq + 6 + 3 * e;
    const double* m = frq + 15 + 3 * e;
    const double ar[3] = {vq[e][0] - rho0[0], vq[e][1] - rho0[1], vq[e][2] - rho0[2]};
    const double P0 = dot3(ar, m), lm = dot3(ar, t), lp = lm + len;
    double bP0 = 0, blm = 0, blp = 0;
    blen[e] = 0;
    // line integral: values then adjoints
    const float ax = (float)(vq[e][0] - r[0]), ay = (float)(vq[e][1] - r[1]), az = (float)(vq[e][2] - r[2]);
    const float tx = (float)t[0], ty = (float)t[1], tz = (float)t[2];
    const float hl = 0.5f * (float)len;
    float lr = 0.f, li = 0.f;
    for (int i = 0; i < A.nl; ++i) {
      const float sp = hl * (A.fx_l[i] + 1.0f);
      const float x0 = fmaf(tx, sp, ax), x1 = fmaf(ty, sp, ay), x2 = fmaf(tz, sp, az);
      const float R = sqrtf(fmaf(x0, x0, fmaf(x1, x1, x2 * x2)));
      const float2 eR = exp32(kpi, R, te, use_table, lo, hi);
      lr = fmaf(eR.x - 1.0f, A.fw_l[i], lr);
      li = fmaf(fmaf(k32, R, eR.y), A.fw_l[i], li);
    }
    const double blrd = dot3(bvre, m), blid = dot3(bvim, m);
    const double lrd = (double)lr * (0.5 * len), lid = (double)li * (0.5 * len);
    const float blr = (float)(blrd * 0.5 * len), bli = (float)(blid * 0.5 * len);
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
    // static part, from its partial derivatives
    const double bst = dot3(bvst, m);
    for (int x = 0; x < 3; ++x) bm[e][x] = bvre[x] * lrd + bvim[x] * lid + bvst[x] * st_[e];
    blp += s_lp[e] * bst;
    blm += s_lm[e] * bst;
    bRv[en] += s_Rp[e] * bst;
    bRv[e] += s_Rm[e] * bst;
    const double bR02 = s_R02[e] * bst;
    // angular part
    if (fabs(P0) > 1e-12 * len) {
      const float aP32 = (float)fabs(P0), iaP = __frcp_rn(aP32);
      const float zm = (float)lm * iaP, zp = (float)lp * iaP;
      const float um = asinhf(zm), up = asinhf(zp);
      const float half = 0.5f * (up - um), mid = 0.5f * (up + um);
      const double sgn = P0 > 0 ? 1.0 : -1.0, sg = sgn * (double)half;
      const float bcr = (float)(bsre * sg), bci = (float)(bsim * sg);
      float bhalf = (float)(sgn * (bsre * (double)cr_[e] + bsim * (double)ci_[e])), bmid = 0.f, baP = 0.f,
            bd32 = 0.f;
      float bk32a = 0.f;
      for (int i = 0; i < A.nphi; ++i) {
        const float u = fmaf(half, A.fx_phi[i], mid);
        const float E = expf(u), iE = __frcp_rn(E);
        const float ch = 0.5f * (E + iE), sh = 0.5f * (E - iE);
        const float rho = aP32 * ch;
        const float Re = sqrtf(fmaf(rho, rho, d32 * d32));
        const float2 eR = exp32(kpi, Re, te, use_table, lo, hi);
        const float ich = __frcp_rn(ch);
        const float wt = A.fw_phi[i] * ich;
        bedr += bcr * wt;
        bedi += bci * wt;
        const float bEr = -bcr * wt, bEi = -bci * wt;
        const float bph = bEr * eR.y - bEi * eR.x;
        const float bRe = bph * k32;
        bk32a += bph * Re;
        const float bwt = bcr * (ed.x - eR.x) + bci * (ed.y - eR.y);
        float bch = -bwt * wt * ich;
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
      blp += (double)(bzp * iaP);
      blm += (double)(bzm * iaP);
      baP -= (bzp * zp + bzm * zm) * iaP;
      bP0 += sgn * (double)baP;
    }
    bP0 += 2.0 * P0 * bR02;
    bd += 2.0 * d * bR02;
    blm += blp;
    blen[e] += blp;
    for (int x = 0; x < 3; ++x) {
      const double bar = bP0 * m[x] + blm * t[x];
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
    const double gr = bRv[c] * iRv[c];
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
    const double t[3] = {frq[6 + 3 * e], frq[7 + 3 * e], frq[8 + 3 * e]};
    const double ilen = frq[25 + e];
    double c1[3], c2[3];
    cross3(n, bm[e], c1);  // d/dt of (t x n) . bm
    cross3(bm[e], t, c2);  // d/dn
    for (int x = 0; x < 3; ++x) {
      bt[e][x] += c1[x];
      bn[x] += c2[x];
    }
    const double tb = dot3(t, bt[e]);
    for (int x = 0; x < 3; ++x) {
      const double btt = (bt[e][x] - t[x] * tb) * ilen + blen[e] * t[x];
      gq[en][x] += btt;
      gq[e][x] -= btt;
    }
  }
  {
    const double iL = 0.5 * frq[24];  // 1 / |nn|, nn = e1 x e2
    const double e1[3] = {vq[1][0] - vq[0][0], vq[1][1] - vq[0][1], vq[1][2] - vq[0][2]};
    const double e2[3] = {vq[2][0] - vq[0][0], vq[2][1] - vq[0][1], vq[2][2] - vq[0][2]};
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

// Near pairs packed P = 32 / M to a warp, lane = (pair slot, test point); all
// 19 derivatives of a pair in one reverse pass, summed over the pair's M
// lanes (32 - P M lanes idle, against 8 - M of every 8 with groups of 8).
template <int M>
__global__ void __launch_bounds__(128) k_adjoint_near_rev(GeoView g, TabView te, bool use_table, NearArgs A, double k,
                                                          double eta, BaryF bw, const float2* __restrict__ gZ,
                                                          int64_t ldg, double* dtri, double* dkacc) {
  constexpr int P = 32 / M;
  const Tab32 te32 = tab32(te);
  const float lo32 = (float)te.r_lo, hi32 = (float)te.r_hi;
  const double ik = 1.0 / k;
  const float kpi = (float)(k / kPi);
  const int64_t n_near = g.near_ptr[g.nt];
  const int lane = threadIdx.x & 31, slot = lane / M, sub = lane - M * (lane / M);
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t iters = (n_near + nwarps * P - 1) / (nwarps * P);  // same trip count in every lane of a warp
  for (int64_t itn = 0; itn < iters; ++itn) {
    const int64_t idx = (w0 + itn * nwarps) * P + slot;
    const bool valid = slot < P && idx < n_near;
    const int p = valid ? g.near_row[idx] : 0, q = valid ? g.near_idx[idx] : 0;
    double gp[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, gq[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, gk = 0;
    if (valid) {
      double vp[3][3], vq[3][3];
      for (int c = 0; c < 3; ++c)
        for (int x = 0; x < 3; ++x) {
          vp[c][x] = g.v64[9 * (size_t)p + 3 * c + x];
          vq[c][x] = g.v64[9 * (size_t)q + 3 * c + x];
        }
      const int4 ep = g.tedge[p], eq = g.tedge[q];
      const int ecp[3] = {ep.x, ep.y, ep.z}, ecq[3] = {eq.x, eq.y, eq.z};
      const double wa = g.pts64[4 * ((size_t)sub * g.nt + p) + 3];
      near_point_adjoint(vp, vq, g.frame64 + kFrame * (size_t)p, g.frame64 + kFrame * (size_t)q, bw.l[sub], wa, A,
                         k, ik, kpi, eta, te32, use_table, lo32, hi32, ecp, ecq, gZ, ldg, gp, gq, &gk);
    }
    // segmented sum over the M lanes of each slot: after the step with offset
    // o, lane sub holds the sum over sub .. sub + 2o - 1 (within the slot)
#pragma unroll
    for (int off = 1; off < M; off <<= 1) {
      const bool take = sub + off < M;
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          const double a = __shfl_down_sync(0xffffffffu, gp[c][x], off);
          const double b = __shfl_down_sync(0xffffffffu, gq[c][x], off);
          if (take) {
            gp[c][x] += a;
            gq[c][x] += b;
          }
        }
      const double a = __shfl_down_sync(0xffffffffu, gk, off);
      if (take) gk += a;
    }
    if (valid && sub == 0) {
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
template <int G>
__global__ void __launch_bounds__(128) k_adjoint_near(GeoView g, TabView te, bool use_table, NearArgs A, double k,
                                                      double eta, BaryF bw, const float2* __restrict__ gZ, int64_t ldg,
                                                      double* dtri, double* dkacc) {
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
      inner_integrals_d(ra, vq, A, kd, &te, use_table, &I0, I1, &rho0);
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

}  // namespace

template <int M>
cudaError_t launch_adjoint_regular_m(const GeoView& g, const TabView* green, double k, double eta, const BaryF& bw,
                                     const float2* gZ, int64_t ldg, double* dtri, double* dk, cudaStream_t s) {
  TabView tv{};
  if (green) tv = *green;
  const int64_t blocks = pair_grid(g, 4);
  const float kappa = (float)(k * eta / (4.0 * kPi)), inv_k2 = (float)(1.0 / (k * k));
  if (!green) {
    k_adjoint_regular32<M, false, false><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, (float)k, kappa, inv_k2, bw, gZ,
                                                                              ldg, dtri, dk);
    return cudaGetLastError();
  }
  // the Green lattice staged in shared memory where it fits (one CTA per SM
  // at this register count: one staging per SM), else read through L1
  const size_t smem = tv.smem32_bytes(3);
  int dev = 0, max_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem <= (size_t)max_optin) {
    auto kern = k_adjoint_regular32<M, true, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    const int64_t b = std::min<int64_t>(blocks, (int64_t)sm_count() * std::max(per_sm, 1));
    kern<<<(unsigned)b, kThreads, smem, s>>>(g, tv, (float)k, kappa, inv_k2, bw, gZ, ldg, dtri, dk);
  } else {
    k_adjoint_regular32<M, true, false><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, (float)k, kappa, inv_k2, bw, gZ,
                                                                             ldg, dtri, dk);
  }
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
  if (mixed) {
    switch (g.m) {
      case 1: k_adjoint_near_rev<1><<<nblk, 128, 0, s>>>(g, te, t, A, k, eta, bw, gz, ldg, dtri, dk); break;
      case 3: k_adjoint_near_rev<3><<<nblk, 128, 0, s>>>(g, te, t, A, k, eta, bw, gz, ldg, dtri, dk); break;
      case 4: k_adjoint_near_rev<4><<<nblk, 128, 0, s>>>(g, te, t, A, k, eta, bw, gz, ldg, dtri, dk); break;
      case 6: k_adjoint_near_rev<6><<<nblk, 128, 0, s>>>(g, te, t, A, k, eta, bw, gz, ldg, dtri, dk); break;
      default: k_adjoint_near_rev<7><<<nblk, 128, 0, s>>>(g, te, t, A, k, eta, bw, gz, ldg, dtri, dk); break;
    }
  } else if (g.m <= 4) {
    k_adjoint_near<4><<<nblk, 128, 0, s>>>(g, te, t, A, k, eta, bw, gz, ldg, dtri, dk);
  } else {
    k_adjoint_near<8><<<nblk, 128, 0, s>>>(g, te, t, A, k, eta, bw, gz, ldg, dtri, dk);
  }
  k_adjoint_gather<<<(g.nt + 127) / 128, 128, 0, s>>>(g.nt, g.tvert, dtri, dxyz);
  return cudaGetLastError();
}

}  // namespace gf
