// gfmom scattering stage: plane-wave excitation of the RWG functions and the
// far field / bistatic radar cross section of an RWG current. They turn the
// filled EFIE matrix into the quantity the paper compares between the table
// and the direct fill (its RCS results, Section IV.B). FP64 arithmetic (a few
// phase evaluations per quadrature point; not on the fill's hot path).
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <string>

#include "gf_internal.h"

namespace gf {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kRcsThreads = 256;

template <class T>
struct CplxIO;
template <>
struct CplxIO<float2> {
  static __device__ double2 load(const float2* p, int64_t i) {
    const float2 v = p[i];
    return make_double2(v.x, v.y);
  }
  static __device__ void add(float2* p, int64_t i, double2 v) { atomicAdd(p + i, make_float2((float)v.x, (float)v.y)); }
};
template <>
struct CplxIO<double2> {
  static __device__ double2 load(const double2* p, int64_t i) { return p[i]; }
  static __device__ void add(double2* p, int64_t i, double2 v) {
    atomicAdd(reinterpret_cast<double*>(p + i), v.x);
    atomicAdd(reinterpret_cast<double*>(p + i) + 1, v.y);
  }
};

struct PlaneWave {
  double khat[3];
  double pre[3], pim[3];  // complex polarisation (EFIE) or H_inc amplitude khat x p / eta (MFIE)
  int mfie;               // test n x H_inc instead of E_inc
};

// V_m += <f_m, p e^{-jk khat.r}> over triangle t for each of its RWG edges:
// (s l / 2) sum_a w_a ((r_a - v_opp) . p) e^{-jk khat.r_a}, r_a - v_opp =
// alpha_a + delta_j. One thread per triangle; each edge receives exactly two
// additions (T+ and T-), so the sum does not depend on their order.
template <class T>
__global__ void k_excitation(GeoView g, double k, PlaneWave w, T* V) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.nt) return;
  const double* c = g.cen64 + 4 * (size_t)t;
  if (w.mfie) {  // the tested field is n x H_inc: replace the amplitude by n x (khat x p) / eta
    const double* n = g.frame64 + kFrame * (size_t)t;
    const double hr[3] = {w.pre[0], w.pre[1], w.pre[2]}, hi[3] = {w.pim[0], w.pim[1], w.pim[2]};
    w.pre[0] = n[1] * hr[2] - n[2] * hr[1];
    w.pre[1] = n[2] * hr[0] - n[0] * hr[2];
    w.pre[2] = n[0] * hr[1] - n[1] * hr[0];
    w.pim[0] = n[1] * hi[2] - n[2] * hi[1];
    w.pim[1] = n[2] * hi[0] - n[0] * hi[2];
    w.pim[2] = n[0] * hi[1] - n[1] * hi[0];
  }
  double er[8], ei[8], ap[8][2], wa[8];  // per point: phase, alpha . p (complex), weight
  for (int a = 0; a < g.m; ++a) {
    const double* pa = g.pts64 + 4 * ((size_t)a * g.nt + t);
    const double phase = k * (w.khat[0] * (c[0] + pa[0]) + w.khat[1] * (c[1] + pa[1]) + w.khat[2] * (c[2] + pa[2]));
    double s, co;
    sincos(phase, &s, &co);
    er[a] = co;
    ei[a] = -s;
    ap[a][0] = pa[0] * w.pre[0] + pa[1] * w.pre[1] + pa[2] * w.pre[2];
    ap[a][1] = pa[0] * w.pim[0] + pa[1] * w.pim[1] + pa[2] * w.pim[2];
    wa[a] = pa[3];
  }
  const int4 te = g.tedge[t];
  const int codes[3] = {te.x, te.y, te.z};
  for (int j = 0; j < 3; ++j) {
    if (codes[j] < 0) continue;
    const double* gj = g.geo64 + 4 * (3 * (size_t)t + j);  // delta_j = c - v_j, s_j l_j
    const double dre = gj[0] * w.pre[0] + gj[1] * w.pre[1] + gj[2] * w.pre[2];
    const double dim = gj[0] * w.pim[0] + gj[1] * w.pim[1] + gj[2] * w.pim[2];
    double vr = 0, vi = 0;
    for (int a = 0; a < g.m; ++a) {
      const double qr = ap[a][0] + dre, qi = ap[a][1] + dim;  // (r_a - v_j) . p
      vr += wa[a] * (qr * er[a] - qi * ei[a]);
      vi += wa[a] * (qr * ei[a] + qi * er[a]);
    }
    const double h = 0.5 * gj[3];
    CplxIO<T>::add(V, codes[j] >> 1, make_double2(h * vr, h * vi));
  }
}

// One block per direction d: N(d) = sum_t sum_j I_{e_j} (s_j l_j / 2)
// sum_a w_a (alpha_a + delta_j) e^{jk d.r_a}, reduced over the block in a
// fixed order; F = -(j k eta / 4 pi)(N - (d.N) d), sigma = 4 pi |F|^2.
template <class T>
__global__ void __launch_bounds__(kRcsThreads) k_far_field(GeoView g, double k, double eta, const T* __restrict__ I,
                                                           const double* __restrict__ dirs, double* F, double* sigma) {
  __shared__ double red[6][kRcsThreads];
  const int64_t id = blockIdx.x;
  const double d[3] = {dirs[3 * id], dirs[3 * id + 1], dirs[3 * id + 2]};
  double n[6] = {0, 0, 0, 0, 0, 0};  // N: (re, im) per component
  for (int t = threadIdx.x; t < g.nt; t += blockDim.x) {
    const int4 te = g.tedge[t];
    const int codes[3] = {te.x, te.y, te.z};
    // coefficient of (alpha_a + delta_j): c_j = I_{e_j} s_j l_j / 2
    double cr[3], ci[3], dr[3] = {0, 0, 0}, di[3] = {0, 0, 0};  // sum_j c_j delta_j
    double sr = 0, si = 0;                                          // sum_j c_j
    for (int j = 0; j < 3; ++j) {
      cr[j] = ci[j] = 0.0;
      if (codes[j] < 0) continue;
      const double* gj = g.geo64 + 4 * (3 * (size_t)t + j);
      const double2 Ij = CplxIO<T>::load(I, codes[j] >> 1);
      cr[j] = 0.5 * gj[3] * Ij.x;
      ci[j] = 0.5 * gj[3] * Ij.y;
      sr += cr[j];
      si += ci[j];
      for (int x = 0; x < 3; ++x) {
        dr[x] += cr[j] * gj[x];
        di[x] += ci[j] * gj[x];
      }
    }
    if (sr == 0.0 && si == 0.0 && dr[0] == 0.0 && di[0] == 0.0 && dr[1] == 0.0 && dr[2] == 0.0 && di[1] == 0.0 &&
        di[2] == 0.0)
      continue;
    const double* c = g.cen64 + 4 * (size_t)t;
    for (int a = 0; a < g.m; ++a) {
      const double* pa = g.pts64 + 4 * ((size_t)a * g.nt + t);
      double s, co;
      sincos(k * (d[0] * (c[0] + pa[0]) + d[1] * (c[1] + pa[1]) + d[2] * (c[2] + pa[2])), &s, &co);
      const double wr = pa[3] * co, wi = pa[3] * s;  // w_a e^{jk d.r_a}
      for (int x = 0; x < 3; ++x) {
        const double ur = sr * pa[x] + dr[x], ui = si * pa[x] + di[x];  // sum_j c_j (alpha_a + delta_j)
        n[2 * x] += ur * wr - ui * wi;
        n[2 * x + 1] += ur * wi + ui * wr;
      }
    }
  }
  for (int q = 0; q < 6; ++q) red[q][threadIdx.x] = n[q];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int q = 0; q < 6; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  double N[6];
  for (int q = 0; q < 6; ++q) N[q] = red[q][0];
  const double dnr = d[0] * N[0] + d[1] * N[2] + d[2] * N[4], dni = d[0] * N[1] + d[1] * N[3] + d[2] * N[5];
  const double c = k * eta / (4.0 * kPi);
  double s2 = 0;
  for (int x = 0; x < 3; ++x) {
    const double tr = N[2 * x] - dnr * d[x], ti = N[2 * x + 1] - dni * d[x];  // transverse part
    const double fr = c * ti, fi = -c * tr;                                  // -j c (tr + j ti)
    F[6 * id + 2 * x] = fr;
    F[6 * id + 2 * x + 1] = fi;
    s2 += fr * fr + fi * fi;
  }
  sigma[id] = 4.0 * kPi * s2;
}

gf_status mesh_ready(gf_mesh* m, int rule, cudaStream_t s) {
  int cur = -1;
  GF_CUDA(cudaGetDevice(&cur));
  if (cur != m->device) return fail(GF_ERR_DEVICE, "handle belongs to device " + std::to_string(m->device));
  return prepare_rule(m, rule, s);
}

}  // namespace
}  // namespace gf

extern "C" {

gf_status gf_excitation(const gf_mesh* mc, double k, const gf_params* p, const double* khat, const double* pol,
                        int op, int precision, void* V, void* stream) {
  using namespace gf;
  if (!mc || !p || !khat || !pol || !V) return fail(GF_ERR_ARG, "gf_excitation: null argument");
  if (op != GF_OP_EFIE && op != GF_OP_MFIE) return fail(GF_ERR_ARG, "gf_excitation: bad operator");
  if (precision != GF_FP32 && precision != GF_FP64) return fail(GF_ERR_ARG, "gf_excitation: bad precision");
  if (!(k >= 0) || !std::isfinite(k)) return fail(GF_ERR_ARG, "gf_excitation: need k >= 0");
  const double kn = std::sqrt(khat[0] * khat[0] + khat[1] * khat[1] + khat[2] * khat[2]);
  if (!(std::fabs(kn - 1.0) < 1e-9)) return fail(GF_ERR_ARG, "gf_excitation: khat must be a unit vector");
  gf_mesh* m = const_cast<gf_mesh*>(mc);
  cudaStream_t s = (cudaStream_t)stream;
  gf_status st = mesh_ready(m, p->rule, s);
  if (st) return st;
  if (m->ne == 0) return GF_OK;
  PlaneWave w;
  for (int x = 0; x < 3; ++x) {
    w.khat[x] = khat[x];
    w.pre[x] = pol[2 * x];
    w.pim[x] = pol[2 * x + 1];
  }
  w.mfie = op == GF_OP_MFIE;
  if (w.mfie) {  // H_inc amplitude (khat x p) / eta
    if (!(p->eta > 0)) return fail(GF_ERR_ARG, "gf_excitation: need eta > 0");
    const double pr[3] = {w.pre[0], w.pre[1], w.pre[2]}, pi[3] = {w.pim[0], w.pim[1], w.pim[2]};
    for (int x = 0; x < 3; ++x) {
      const int y = (x + 1) % 3, z = (x + 2) % 3;
      w.pre[x] = (khat[y] * pr[z] - khat[z] * pr[y]) / p->eta;
      w.pim[x] = (khat[y] * pi[z] - khat[z] * pi[y]) / p->eta;
    }
  }
  const size_t esz = precision == GF_FP32 ? 8 : 16;
  GF_CUDA(cudaMemsetAsync(V, 0, (size_t)m->ne * esz, s));
  const GeoView g = geo_view(m);
  const unsigned blocks = (unsigned)((m->nt + 127) / 128);
  if (precision == GF_FP32) k_excitation<float2><<<blocks, 128, 0, s>>>(g, k, w, (float2*)V);
  else k_excitation<double2><<<blocks, 128, 0, s>>>(g, k, w, (double2*)V);
  GF_CUDA(cudaGetLastError());
  return GF_OK;
}

gf_status gf_far_field(const gf_mesh* mc, double k, const gf_params* p, int precision, const void* I, int64_t n_dir,
                       const double* dirs, double* F, double* sigma, void* stream) {
  using namespace gf;
  if (!mc || !p || !I || !dirs || !F || !sigma) return fail(GF_ERR_ARG, "gf_far_field: null argument");
  if (precision != GF_FP32 && precision != GF_FP64) return fail(GF_ERR_ARG, "gf_far_field: bad precision");
  if (!(k >= 0) || !std::isfinite(k) || n_dir < 0 || n_dir > (int64_t)INT32_MAX)
    return fail(GF_ERR_ARG, "gf_far_field: need k >= 0 and 0 <= n_dir < 2^31");
  gf_mesh* m = const_cast<gf_mesh*>(mc);
  cudaStream_t s = (cudaStream_t)stream;
  gf_status st = mesh_ready(m, p->rule, s);
  if (st) return st;
  if (n_dir == 0) return GF_OK;
  const GeoView g = geo_view(m);
  if (precision == GF_FP32)
    k_far_field<float2><<<(unsigned)n_dir, kRcsThreads, 0, s>>>(g, k, p->eta, (const float2*)I, dirs, F, sigma);
  else
    k_far_field<double2><<<(unsigned)n_dir, kRcsThreads, 0, s>>>(g, k, p->eta, (const double2*)I, dirs, F, sigma);
  GF_CUDA(cudaGetLastError());
  return GF_OK;
}

}  // extern "C"
