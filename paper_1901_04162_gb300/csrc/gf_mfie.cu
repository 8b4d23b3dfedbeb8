// gfmom MFIE (K operator) kernels for sm_103a: identity term, regular pairs
// (FP32 with the Green table in shared memory, FP64) and near pairs, with
// their launcher.
#include "gf_near.cuh"

namespace gf {
namespace {

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
    stage_tab32(T, tv, 3, smem);
    __syncthreads();
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
      // v_c - r and |v_c - r|, once (scalars: the edge loop picks them by e)
      const double w0x = v[0] - r[0], w0y = v[1] - r[1], w0z = v[2] - r[2];
      const double w1x = v[3] - r[0], w1y = v[4] - r[1], w1z = v[5] - r[2];
      const double w2x = v[6] - r[0], w2y = v[7] - r[1], w2z = v[8] - r[2];
      const double Rv0 = sqrt(w0x * w0x + w0y * w0y + w0z * w0z), Rv1 = sqrt(w1x * w1x + w1y * w1y + w1z * w1z),
                   Rv2 = sqrt(w2x * w2x + w2y * w2y + w2z * w2z);
      const double h = p == q ? 0.0 : -(n[0] * w0x + n[1] * w0y + n[2] * w0z);
      const double d = fabs(h), sgh = h > 0 ? 1.0 : (h < 0 ? -1.0 : 0.0);
      const double rho0[3] = {r[0] - h * n[0], r[1] - h * n[1], r[2] - h * n[2]};
      const C2 ed = exp_mjkr(k, d, &te, use_table);
      double Iu[3][2] = {}, hI0[2] = {0, 0};
      for (int e = 0; e < 3; ++e) {
        const double* a = v + 3 * e;
        const double le = fr[3 + e];
        const double t[3] = {fr[6 + 3 * e], fr[7 + 3 * e], fr[8 + 3 * e]};
        const double m[3] = {fr[15 + 3 * e], fr[16 + 3 * e], fr[17 + 3 * e]};
        // a - r; its in-plane part a - rho0 differs by h n, normal to t and m
        const double arx = e == 0 ? w0x : (e == 1 ? w1x : w2x), ary = e == 0 ? w0y : (e == 1 ? w1y : w2y),
                     arz = e == 0 ? w0z : (e == 1 ? w1z : w2z);
        const double P0 = arx * m[0] + ary * m[1] + arz * m[2];
        const double lm = arx * t[0] + ary * t[1] + arz * t[2];
        const double lp = lm + le;
        const double Rm = e == 0 ? Rv0 : (e == 1 ? Rv1 : Rv2), Rp = e == 0 ? Rv1 : (e == 1 ? Rv2 : Rv0);
        const double R02 = P0 * P0 + d * d;
        double ratio;
        if (lm >= 0) ratio = (lp + Rp) / (lm + Rm);
        else if (lp >= 0) ratio = (lp + Rp) * (Rm - lm) / R02;
        else ratio = (Rm - lm) / (Rp - lp);
        double lr = log(ratio), li = 0.0;
        if (MIXED) {
          const float* f32 = g.frame32 + kFrame32 * (size_t)q;
          const float ax = (float)arx, ay = (float)ary, az = (float)arz;
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
        const double R1[3] = {w0x, w0y, w0z}, R2[3] = {w1x, w1y, w1z}, R3[3] = {w2x, w2y, w2z};
        const double n1 = Rv0, n2 = Rv1, n3 = Rv2;
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

}  // namespace

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

}  // namespace gf
