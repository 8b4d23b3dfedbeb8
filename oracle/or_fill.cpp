// Oracle: mesh -> RWG, singular inner integrals, EFIE Z entries, table range
// and the reference gradient. Test infrastructure only (see oracle.h).
//
// Z_mn = jk eta int_{T_m} int_{T_n} [f_m . f_n - (1/k^2) div f_m div' f_n] G dS' dS,
// G = e^{-jkR} / (4 pi R) (EFIE L operator with RWG basis, Galerkin testing,
// planar triangles: Section II.A and Section IV.B of Yang & Su). Each entry is
// the sum over the four (test, source) triangle pairs of edges m and n:
//   * regular pair: the m-point rule on both triangles; G from the direct
//     formula or from the Lagrange table of e^{-jkr}/r;
//   * near pair (sharing a vertex, or centroids closer than near_dist): the
//     m-point rule on the test triangle and, for the inner integral, the
//     singularity cancellation with the angular transformation: the radial
//     integral of e^{-jkR}/R is exact, leaving n_phi-point integrals in the
//     polar angle for each of the three source edges, and the vector part is
//     turned into line integrals over the three edges by the surface-gradient
//     theorem (Section II.A: "n-point numerical integration at each edge of
//     the source triangle ... three lines"). e^{-jkR} on these lines comes from
//     the linear Exp table when r_min <= R <= r_max, else directly (Section
//     II.C: r < r_min falls back to the classical evaluation).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include "oracle.h"
#include "or_types.h"

#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {
void table_value(const or_table* T, double x, double* re, double* im);
double table_lo(const or_table* T);
double table_hi(const or_table* T);
}  // namespace orc

using namespace orc;

namespace {
const double kPi = 3.14159265358979323846;
}

struct or_mesh {
  int nv, nt, ne;
  std::vector<double> xyz;          // [nv][3]
  std::vector<int> tri;             // [nt][3]
  std::vector<int> ev;              // [ne][2] vertex ids (lower, higher)
  std::vector<int> et;              // [ne][2] (T+, T-)
  std::vector<int> eo;              // [ne][2] vertex opposite the edge in T+, T-
  std::vector<int> tedge;           // [nt][3] edge id of the edge opposite local vertex i, or -1
  std::vector<int> tsign;           // [nt][3] +1 if T+ of that edge, -1 if T-
  std::vector<double> cen;          // [nt][3]
  double near_dist;
};

namespace {

V3<double> vtx(const or_mesh* m, int v) {
  return V3<double>(m->xyz[3 * v], m->xyz[3 * v + 1], m->xyz[3 * v + 2]);
}

bool is_near(const or_mesh* m, int p, int q) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (m->tri[3 * p + i] == m->tri[3 * q + j]) return true;
  if (m->near_dist > 0) {
    double dx = m->cen[3 * p] - m->cen[3 * q];
    double dy = m->cen[3 * p + 1] - m->cen[3 * q + 1];
    double dz = m->cen[3 * p + 2] - m->cen[3 * q + 2];
    if (std::sqrt(dx * dx + dy * dy + dz * dz) < m->near_dist) return true;
  }
  return false;
}

// e^{-jkR} (Exp) and e^{-jkR}/R (Green) by formula or by table
template <class T>
Cx<T> exp_mjkr(T k, T R, const or_table* texp) {
  using std::cos;
  using std::sin;
  if (texp) {
    double r = val(R);
    if (r >= table_lo(texp) && r <= table_hi(texp)) {
      double re, im;
      table_value(texp, r, &re, &im);
      return Cx<T>(T(re), T(im));
    }
  }
  T ph = k * R;
  return Cx<T>(cos(ph), -sin(ph));
}

template <class T>
Cx<T> green(T k, T R, const or_table* tgreen) {
  using std::cos;
  using std::sin;
  const double inv4pi = 1.0 / (4.0 * kPi);
  if (tgreen) {
    double r = val(R);
    if (r >= table_lo(tgreen) && r <= table_hi(tgreen)) {
      double re, im;
      table_value(tgreen, r, &re, &im);
      return Cx<T>(T(re * inv4pi), T(im * inv4pi));
    }
  }
  T ph = k * R;
  T s = T(inv4pi) / R;
  return Cx<T>(cos(ph) * s, -(sin(ph) * s));
}

struct Quad {
  int n;
  double bary[7][3];
  double w[7];
  int nphi, nl;
  std::vector<double> gx_phi, gw_phi, gx_l, gw_l;
};

bool make_quad(int rule, int nphi, int nl, Quad* q) {
  q->n = rule;
  if (or_rule(rule, &q->bary[0][0], q->w) != 0) return false;
  q->nphi = nphi;
  q->nl = nl;
  q->gx_phi.resize(nphi);
  q->gw_phi.resize(nphi);
  q->gx_l.resize(nl);
  q->gw_l.resize(nl);
  if (or_gauss_legendre(nphi, q->gx_phi.data(), q->gw_phi.data())) return false;
  if (or_gauss_legendre(nl, q->gx_l.data(), q->gw_l.data())) return false;
  return true;
}

// Inner integrals over source triangle (v[0], v[1], v[2]) for point r:
//   I0 = int G dS',  I1 = int (r' - rho0) G dS'   (1/(4 pi) included)
// Scalar part: polar coordinates about the projection rho0, one sector per
// edge with signed foot distance P0; rho d rho = R dR makes the radial
// integral exact: int_d^{R_e} e^{-jkR} dR = (e^{-jkd} - e^{-jkR_e}) / (jk).
// The angular integral uses u = asinh(tan phi), which keeps the integrand
// smooth when the projection lies close to an edge line.
// Vector part: (r' - rho0) e^{-jkR}/R = (j/k) grad'_s e^{-jkR}, so its
// integral is (j/k) sum_edges m_hat int_edge e^{-jkR} dl. Splitting
// e^{-jkR} = (e^{-jkR} - 1 + jkR) + 1 - jkR and using sum m_hat l = 0 leaves
// sum m_hat int_edge R dl (closed form, = int (r' - rho0)/R dS') plus
// (j/k) sum m_hat int_edge (e^{-jkR} - 1 + jkR) dl, a smooth line integral.
template <class T>
void singular(const V3<T>& r, const V3<T> v[3], T k, const Quad& Q, const or_table* texp, Cx<T>* I0,
              V3<Cx<T>>* I1, V3<T>* rho0_out) {
  using std::atan2;
  using std::fabs;
  using std::sqrt;
  V3<T> nrm = cross(v[1] - v[0], v[2] - v[0]);
  T nn = norm(nrm);
  nrm = nrm * (T(1.0) / nn);
  T h = dot(nrm, r - v[0]);
  T d = fabs(h);
  V3<T> rho0 = r - nrm * h;
  *rho0_out = rho0;
  Cx<T> e_d = exp_mjkr(k, d, texp);
  Cx<T> s_acc;                 // sum of signed sector integrals of (e^{-jkd} - e^{-jkR_e})
  V3<Cx<T>> v_acc;             // sum over edges of m_hat * int (e^{-jkR} - 1 + jkR) dl
  V3<T> v_stat;                // sum over edges of m_hat * int R dl (= int (r' - rho0)/R dS')
  for (int e = 0; e < 3; ++e) {
    const V3<T>& a = v[e];
    const V3<T>& b = v[(e + 1) % 3];
    V3<T> ab = b - a;
    T len = norm(ab);
    V3<T> th = ab * (T(1.0) / len);
    V3<T> mh = cross(th, nrm);  // outward in-plane normal for a counter-clockwise loop
    T P0 = dot(a - rho0, mh);
    T lm = dot(a - rho0, th);
    T lp = dot(b - rho0, th);
    // scalar part: sector angle phi from the foot of the perpendicular, in
    // the variable u = asinh(tan phi) (d phi = du / cosh u, rho_e = |P0| cosh u)
    if (fabs(val(P0)) > 1e-12 * val(len)) {
      using std::asinh;
      using std::cosh;
      T aP = fabs(P0);
      T um = asinh(lm / aP), up = asinh(lp / aP);
      T half = (up - um) * 0.5, mid = (up + um) * 0.5;
      Cx<T> sec;
      for (int i = 0; i < Q.nphi; ++i) {
        T u = mid + half * Q.gx_phi[i];
        T ch = cosh(u);
        T rho_e = aP * ch;
        T Re = sqrt(rho_e * rho_e + d * d);
        Cx<T> eR = exp_mjkr(k, Re, texp);
        sec += (e_d - eR) * (T(Q.gw_phi[i]) / ch);
      }
      sec = sec * half;
      T sg = val(P0) > 0 ? T(1.0) : T(-1.0);
      s_acc += sec * sg;
    }
    // vector part: m_hat int_edge (e^{-jkR} - 1 + jkR) dl numerically; the
    // static part m_hat int_edge R dl is added in closed form below.
    Cx<T> li;
    for (int i = 0; i < Q.nl; ++i) {
      T s = len * (0.5 * (Q.gx_l[i] + 1.0));
      V3<T> x = a + th * s;
      T R = norm(r - x);
      Cx<T> e = exp_mjkr(k, R, texp);
      li += Cx<T>(e.re - 1.0, e.im + k * R) * T(Q.gw_l[i]);
    }
    li = li * (len * 0.5);
    v_acc.x += li * mh.x;
    v_acc.y += li * mh.y;
    v_acc.z += li * mh.z;
    // int_{l-}^{l+} sqrt(l^2 + R0^2) dl = [l R + R0^2 log(l + R)] / 2, with
    // l + R = R0^2 / (R - l) for l < 0
    {
      T R02 = P0 * P0 + d * d;
      T Rm = sqrt(lm * lm + R02), Rp = sqrt(lp * lp + R02);
      T st = (lp * Rp - lm * Rm) * 0.5;
      if (val(R02) > 0) {
        using std::log;
        T fp = val(lp) >= 0 ? lp + Rp : R02 / (Rp - lp);
        T fm = val(lm) >= 0 ? lm + Rm : R02 / (Rm - lm);
        st = st + R02 * (log(fp) - log(fm)) * 0.5;
      }
      v_stat = v_stat + mh * st;
    }
  }
  const T inv4pi = T(1.0 / (4.0 * kPi));
  // (e_d - eR) / (jk) = -j (e_d - eR) / k
  Cx<T> mj_over_k(T(0.0), -(T(1.0) / k));
  *I0 = (s_acc * mj_over_k) * inv4pi;
  Cx<T> j_over_k(T(0.0), T(1.0) / k);
  I1->x = (v_acc.x * j_over_k + Cx<T>(v_stat.x, T(0.0))) * inv4pi;
  I1->y = (v_acc.y * j_over_k + Cx<T>(v_stat.y, T(0.0))) * inv4pi;
  I1->z = (v_acc.z * j_over_k + Cx<T>(v_stat.z, T(0.0))) * inv4pi;
}

// Geometry of one triangle for the RWG functions of its edges.
template <class T>
struct TriGeo {
  V3<T> v[3];
  T area;
};

template <class T>
TriGeo<T> tri_geo(const V3<T> v[3]) {
  TriGeo<T> g;
  for (int i = 0; i < 3; ++i) g.v[i] = v[i];
  g.area = norm(cross(v[1] - v[0], v[2] - v[0])) * 0.5;
  return g;
}

// Contribution of triangle pair (p, q) to Z_mn where m is the edge opposite
// local vertex i of p with sign sp, n the edge opposite local vertex j of q
// with sign sq. Without the jk eta factor.
// texp_regular != NULL: regular-pair Green values are e^{-jkR} from that
// (linear Exp) table times 1/(4 pi R), in place of the Green table.
template <class T>
Cx<T> pair_term(const TriGeo<T>& P, int i, int sp, const TriGeo<T>& Qg, int j, int sq, bool near, T k,
                const Quad& Q, const or_table* tgreen, const or_table* texp,
                const or_table* texp_regular = nullptr) {
  // RWG on p: f = sp * l/(2A) (r - v_i), div f = sp * l / A
  T lm = norm(P.v[(i + 2) % 3] - P.v[(i + 1) % 3]);
  T ln = norm(Qg.v[(j + 2) % 3] - Qg.v[(j + 1) % 3]);
  T cm = T((double)sp) * lm / (P.area * 2.0);
  T cn = T((double)sq) * ln / (Qg.area * 2.0);
  T divm = T((double)sp) * lm / P.area;
  T divn = T((double)sq) * ln / Qg.area;
  T inv_k2 = T(1.0) / (k * k);
  Cx<T> sum;
  for (int a = 0; a < Q.n; ++a) {
    V3<T> ra = P.v[0] * T(Q.bary[a][0]) + P.v[1] * T(Q.bary[a][1]) + P.v[2] * T(Q.bary[a][2]);
    V3<T> fm = (ra - P.v[i]) * cm;
    T wa = P.area * Q.w[a];
    if (!near) {
      for (int b = 0; b < Q.n; ++b) {
        V3<T> rb = Qg.v[0] * T(Q.bary[b][0]) + Qg.v[1] * T(Q.bary[b][1]) + Qg.v[2] * T(Q.bary[b][2]);
        V3<T> fn = (rb - Qg.v[j]) * cn;
        T wb = Qg.area * Q.w[b];
        T R = norm(ra - rb);
        Cx<T> G = texp_regular ? exp_mjkr(k, R, texp_regular) * (T(1.0 / (4.0 * kPi)) / R) : green(k, R, tgreen);
        T kern = dot(fm, fn) - divm * divn * inv_k2;
        sum += G * (wa * wb * kern);
      }
    } else {
      Cx<T> I0;
      V3<Cx<T>> I1;
      V3<T> rho0;
      singular(ra, Qg.v, k, Q, texp, &I0, &I1, &rho0);
      // int_q f_n G = cn [I1 + (rho0 - v_j) I0]
      V3<T> dv = rho0 - Qg.v[j];
      Cx<T> Fx = (I1.x + I0 * dv.x) * cn;
      Cx<T> Fy = (I1.y + I0 * dv.y) * cn;
      Cx<T> Fz = (I1.z + I0 * dv.z) * cn;
      Cx<T> dotF = Fx * fm.x + Fy * fm.y + Fz * fm.z;
      Cx<T> term = dotF - I0 * (divm * divn * inv_k2);
      sum += term * wa;
    }
  }
  return sum;
}

int nthreads_or_default(int n) {
#ifdef _OPENMP
  return n > 0 ? n : omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

}  // namespace

extern "C" {

int or_mesh_new(const double* xyz, int nv, const int* tri, int nt, double near_dist, or_mesh** out) {
  if (!xyz || !tri || nv < 3 || nt < 1 || !out) return -1;
  or_mesh* m = new or_mesh;
  m->nv = nv;
  m->nt = nt;
  m->xyz.assign(xyz, xyz + 3 * (size_t)nv);
  m->tri.assign(tri, tri + 3 * (size_t)nt);
  m->near_dist = near_dist;
  for (int t = 0; t < nt; ++t)
    for (int i = 0; i < 3; ++i)
      if (tri[3 * t + i] < 0 || tri[3 * t + i] >= nv) {
        delete m;
        return -2;
      }
  // edge key (lower, higher) -> list of (triangle, local index of the opposite vertex)
  std::map<std::pair<int, int>, std::vector<std::pair<int, int>>> emap;
  for (int t = 0; t < nt; ++t) {
    for (int i = 0; i < 3; ++i) {
      int a = tri[3 * t + (i + 1) % 3], b = tri[3 * t + (i + 2) % 3];
      if (a == b) {
        delete m;
        return -2;
      }
      emap[std::make_pair(std::min(a, b), std::max(a, b))].push_back(std::make_pair(t, i));
    }
  }
  m->tedge.assign(3 * (size_t)nt, -1);
  m->tsign.assign(3 * (size_t)nt, 0);
  int ne = 0;
  for (auto& kv : emap) {
    if (kv.second.size() > 2) {
      delete m;
      return -2;  // non-manifold
    }
    if (kv.second.size() != 2) continue;  // boundary edge: no unknown
    auto a = kv.second[0], b = kv.second[1];
    if (a.first > b.first) std::swap(a, b);
    if (a.first == b.first) {
      delete m;
      return -2;
    }
    m->ev.push_back(kv.first.first);
    m->ev.push_back(kv.first.second);
    m->et.push_back(a.first);
    m->et.push_back(b.first);
    m->eo.push_back(tri[3 * a.first + a.second]);
    m->eo.push_back(tri[3 * b.first + b.second]);
    m->tedge[3 * a.first + a.second] = ne;
    m->tsign[3 * a.first + a.second] = +1;
    m->tedge[3 * b.first + b.second] = ne;
    m->tsign[3 * b.first + b.second] = -1;
    ++ne;
  }
  m->ne = ne;
  m->cen.resize(3 * (size_t)nt);
  for (int t = 0; t < nt; ++t)
    for (int c = 0; c < 3; ++c)
      m->cen[3 * t + c] =
          (xyz[3 * tri[3 * t] + c] + xyz[3 * tri[3 * t + 1] + c] + xyz[3 * tri[3 * t + 2] + c]) / 3.0;
  *out = m;
  return 0;
}

int or_mesh_ne(const or_mesh* m) { return m ? m->ne : -1; }

int or_mesh_edges(const or_mesh* m, int* edges, int* etri) {
  if (!m) return -1;
  for (int e = 0; e < 2 * m->ne; ++e) {
    if (edges) edges[e] = m->ev[e];
    if (etri) etri[e] = m->et[e];
  }
  return 0;
}

int or_mesh_is_near(const or_mesh* m, int p, int q) { return is_near(m, p, q) ? 1 : 0; }

void or_mesh_free(or_mesh* m) { delete m; }

int or_singular(const double* r, const double* v0, const double* v1, const double* v2, double k, int nphi,
                int nl, const or_table* texp, double* i0, double* i1, double* rho0) {
  Quad Q;
  if (!make_quad(1, nphi, nl, &Q)) return -1;
  V3<double> v[3] = {V3<double>(v0[0], v0[1], v0[2]), V3<double>(v1[0], v1[1], v1[2]),
                     V3<double>(v2[0], v2[1], v2[2])};
  Cx<double> I0;
  V3<Cx<double>> I1;
  V3<double> rh;
  singular(V3<double>(r[0], r[1], r[2]), v, k, Q, texp, &I0, &I1, &rh);
  i0[0] = I0.re;
  i0[1] = I0.im;
  i1[0] = I1.x.re;
  i1[1] = I1.x.im;
  i1[2] = I1.y.re;
  i1[3] = I1.y.im;
  i1[4] = I1.z.re;
  i1[5] = I1.z.im;
  rho0[0] = rh.x;
  rho0[1] = rh.y;
  rho0[2] = rh.z;
  return 0;
}

int or_range(const or_mesh* m, int rule, double* r_min, double* r_max, int nthreads) {
  return or_range_ex(m, rule, 0, r_min, r_max, nthreads);
}

// prune = 1: every point distance of a pair lies in [D - r_p - r_q, D + r_p + r_q]
// (D centroid distance, r largest point-to-centroid distance), so only pairs
// whose interval reaches below min(D + r_p + r_q) or above max(D - r_p - r_q)
// can hold an extreme; those are evaluated point by point (exact result).
int or_range_ex(const or_mesh* m, int rule, int prune, double* r_min, double* r_max, int nthreads) {
  Quad Q;
  if (!m || !make_quad(rule, 1, 1, &Q)) return -1;
  int nt = m->nt;
  std::vector<double> pts(3 * (size_t)nt * Q.n), rad(nt, 0.0);
  for (int t = 0; t < nt; ++t) {
    V3<double> v[3] = {vtx(m, m->tri[3 * t]), vtx(m, m->tri[3 * t + 1]), vtx(m, m->tri[3 * t + 2])};
    V3<double> c(m->cen[3 * t], m->cen[3 * t + 1], m->cen[3 * t + 2]);
    for (int a = 0; a < Q.n; ++a) {
      V3<double> x = v[0] * Q.bary[a][0] + v[1] * Q.bary[a][1] + v[2] * Q.bary[a][2];
      pts[3 * ((size_t)t * Q.n + a)] = x.x;
      pts[3 * ((size_t)t * Q.n + a) + 1] = x.y;
      pts[3 * ((size_t)t * Q.n + a) + 2] = x.z;
      rad[t] = std::max(rad[t], norm(x - c));
    }
  }
  auto cdist = [&](int p, int q) {
    double dx = m->cen[3 * p] - m->cen[3 * q], dy = m->cen[3 * p + 1] - m->cen[3 * q + 1],
           dz = m->cen[3 * p + 2] - m->cen[3 * q + 2];
    return std::sqrt(dx * dx + dy * dy + dz * dz);
  };
  int nth = nthreads_or_default(nthreads);
  double ub_min = 1e300, lb_max = -1.0;
  if (prune) {
#pragma omp parallel for num_threads(nth) reduction(min : ub_min) reduction(max : lb_max) schedule(dynamic, 16)
    for (int p = 0; p < nt; ++p)
      for (int q = 0; q < nt; ++q) {
        if (is_near(m, p, q)) continue;
        double D = cdist(p, q), r = rad[p] + rad[q];
        ub_min = std::min(ub_min, D + r);
        lb_max = std::max(lb_max, D - r);
      }
  }
  double lo = 1e300, hi = -1.0;
#pragma omp parallel for num_threads(nth) reduction(min : lo) reduction(max : hi) schedule(dynamic, 4)
  for (int p = 0; p < nt; ++p) {
    for (int q = 0; q < nt; ++q) {
      if (is_near(m, p, q)) continue;
      if (prune) {
        double D = cdist(p, q), r = rad[p] + rad[q];
        double slack = 1e-12 * (D + r + 1.0);
        if (D - r - slack > ub_min && D + r + slack < lb_max) continue;
      }
      for (int a = 0; a < Q.n; ++a) {
        const double* x = &pts[3 * ((size_t)p * Q.n + a)];
        for (int b = 0; b < Q.n; ++b) {
          const double* y = &pts[3 * ((size_t)q * Q.n + b)];
          double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
          double R = std::sqrt(dx * dx + dy * dy + dz * dz);
          lo = std::min(lo, R);
          hi = std::max(hi, R);
        }
      }
    }
  }
  if (hi < 0) return -4;  // no regular pair
  *r_min = lo;
  *r_max = hi;
  return 0;
}

int or_z_entries(const or_mesh* m, const or_fill_params* fp, const or_table* tgreen, const or_table* texp,
                 long nent, const int* mi, const int* ni, double* zre, double* zim, int nthreads) {
  Quad Q;
  if (!m || !fp || !make_quad(fp->rule, fp->nphi, fp->nl, &Q)) return -1;
  if (fp->green_mode < 0 || fp->green_mode > 2) return -1;
  if (fp->green_mode == 1 && (!tgreen || !texp)) return -1;
  if (fp->green_mode == 2 && !texp) return -1;
  const or_table* tg = fp->green_mode == 1 ? tgreen : nullptr;
  const or_table* te = fp->green_mode >= 1 ? texp : nullptr;
  const or_table* ter = fp->green_mode == 2 ? texp : nullptr;
  for (long e = 0; e < nent; ++e)
    if (mi[e] < 0 || mi[e] >= m->ne || ni[e] < 0 || ni[e] >= m->ne) return -1;
  double k = fp->k;
  int nth = nthreads_or_default(nthreads);
#pragma omp parallel for num_threads(nth) schedule(dynamic, 16)
  for (long e = 0; e < nent; ++e) {
    int em = mi[e], en = ni[e];
    Cx<double> z;
    for (int s = 0; s < 2; ++s) {
      int p = m->et[2 * em + s];
      int sp = s == 0 ? +1 : -1;
      int ip = -1;
      for (int c = 0; c < 3; ++c)
        if (m->tedge[3 * p + c] == em) ip = c;
      V3<double> pv[3] = {vtx(m, m->tri[3 * p]), vtx(m, m->tri[3 * p + 1]), vtx(m, m->tri[3 * p + 2])};
      TriGeo<double> P = tri_geo(pv);
      for (int t = 0; t < 2; ++t) {
        int q = m->et[2 * en + t];
        int sq = t == 0 ? +1 : -1;
        int iq = -1;
        for (int c = 0; c < 3; ++c)
          if (m->tedge[3 * q + c] == en) iq = c;
        V3<double> qv[3] = {vtx(m, m->tri[3 * q]), vtx(m, m->tri[3 * q + 1]), vtx(m, m->tri[3 * q + 2])};
        TriGeo<double> Qg = tri_geo(qv);
        z += pair_term<double>(P, ip, sp, Qg, iq, sq, is_near(m, p, q), k, Q, tg, te, ter);
      }
    }
    // times j k eta
    double s = k * fp->eta;
    zre[e] = -z.im * s;
    zim[e] = z.re * s;
  }
  return 0;
}

// L = Re(a^H Z b) = Re sum_{pairs (p,q)} sum_{i,j} conj(a_m) C_pq(i,j) b_n.
// Each pair term depends only on the 9 coordinates of p, the 9 of q and k, so
// it is evaluated once with 19 dual directions and its derivatives are added
// to the vertices it touches. Near / regular classification is held fixed.
int or_loss_grad(const or_mesh* m, const or_fill_params* fp, const double* are, const double* aim,
                 const double* bre, const double* bim, double* loss, double* dxyz, double* dk, int nthreads) {
  return or_loss_grad_masked(m, fp, are, aim, bre, bim, nullptr, loss, dxyz, dk, nthreads);
}

// tri_mask (may be NULL): only pairs with p or q marked are differentiated;
// the gradient of a vertex whose triangles are all marked is then complete.
int or_loss_grad_masked(const or_mesh* m, const or_fill_params* fp, const double* are, const double* aim,
                        const double* bre, const double* bim, const int* tri_mask, double* loss, double* dxyz,
                        double* dk, int nthreads) {
  typedef Dual<19> D;
  Quad Q;
  if (!m || !fp || !make_quad(fp->rule, fp->nphi, fp->nl, &Q)) return -1;
  int nt = m->nt;
  int nth = nthreads_or_default(nthreads);
  std::vector<double> gacc((size_t)nth * (3 * (size_t)m->nv + 2), 0.0);
#pragma omp parallel num_threads(nth)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* g = &gacc[(size_t)tid * (3 * (size_t)m->nv + 2)];
#pragma omp for schedule(dynamic, 1)
    for (int p = 0; p < nt; ++p) {
      for (int q = 0; q < nt; ++q) {
        if (tri_mask && !tri_mask[p] && !tri_mask[q]) continue;
        bool nr = is_near(m, p, q);
        V3<D> pv[3], qv[3];
        for (int c = 0; c < 3; ++c) {
          V3<double> x = vtx(m, m->tri[3 * p + c]);
          V3<double> y = vtx(m, m->tri[3 * q + c]);
          pv[c] = V3<D>(D::var(x.x, 3 * c), D::var(x.y, 3 * c + 1), D::var(x.z, 3 * c + 2));
          qv[c] = V3<D>(D::var(y.x, 9 + 3 * c), D::var(y.y, 9 + 3 * c + 1), D::var(y.z, 9 + 3 * c + 2));
        }
        D k = D::var(fp->k, 18);
        TriGeo<D> P = tri_geo(pv), Qg = tri_geo(qv);
        Cx<D> acc;
        for (int i = 0; i < 3; ++i) {
          int em = m->tedge[3 * p + i];
          if (em < 0) continue;
          for (int j = 0; j < 3; ++j) {
            int en = m->tedge[3 * q + j];
            if (en < 0) continue;
            Cx<D> c = pair_term<D>(P, i, m->tsign[3 * p + i], Qg, j, m->tsign[3 * q + j], nr, k, Q, nullptr, nullptr);
            // conj(a_m) * c * b_n
            Cx<D> ca(D(are[em]), D(-aim[em]));
            Cx<D> bn(D(bre[en]), D(bim[en]));
            acc += ca * c * bn;
          }
        }
        // times j k eta: Re(j k eta acc) = -k eta Im(acc)
        D Lp = -(k * fp->eta) * acc.im;
        g[3 * (size_t)m->nv] += Lp.v;
        for (int c = 0; c < 3; ++c)
          for (int x = 0; x < 3; ++x) {
            g[3 * (size_t)m->tri[3 * p + c] + x] += Lp.d[3 * c + x];
            g[3 * (size_t)m->tri[3 * q + c] + x] += Lp.d[9 + 3 * c + x];
          }
        g[3 * (size_t)m->nv + 1] += Lp.d[18];
      }
    }
  }
  double L = 0, gk = 0;
  for (int t = 0; t < nth; ++t) {
    const double* g = &gacc[(size_t)t * (3 * (size_t)m->nv + 2)];
    for (size_t i = 0; i < 3 * (size_t)m->nv; ++i) dxyz[i] += g[i];
    L += g[3 * (size_t)m->nv];
    gk += g[3 * (size_t)m->nv + 1];
  }
  *loss = L;
  *dk = gk;
  return 0;
}

// dL/dk alone (one dual direction), all pairs.
int or_loss_dk(const or_mesh* m, const or_fill_params* fp, const double* are, const double* aim, const double* bre,
               const double* bim, double* loss, double* dk, int nthreads) {
  typedef Dual<1> D;
  Quad Q;
  if (!m || !fp || !make_quad(fp->rule, fp->nphi, fp->nl, &Q)) return -1;
  int nt = m->nt;
  int nth = nthreads_or_default(nthreads);
  double L = 0, gk = 0;
#pragma omp parallel for num_threads(nth) reduction(+ : L, gk) schedule(dynamic, 1)
  for (int p = 0; p < nt; ++p) {
    V3<D> pv[3];
    for (int c = 0; c < 3; ++c) {
      V3<double> x = vtx(m, m->tri[3 * p + c]);
      pv[c] = V3<D>(D(x.x), D(x.y), D(x.z));
    }
    TriGeo<D> P = tri_geo(pv);
    for (int q = 0; q < nt; ++q) {
      bool nr = is_near(m, p, q);
      V3<D> qv[3];
      for (int c = 0; c < 3; ++c) {
        V3<double> y = vtx(m, m->tri[3 * q + c]);
        qv[c] = V3<D>(D(y.x), D(y.y), D(y.z));
      }
      D k = D::var(fp->k, 0);
      TriGeo<D> Qg = tri_geo(qv);
      Cx<D> acc;
      for (int i = 0; i < 3; ++i) {
        int em = m->tedge[3 * p + i];
        if (em < 0) continue;
        for (int j = 0; j < 3; ++j) {
          int en = m->tedge[3 * q + j];
          if (en < 0) continue;
          Cx<D> c = pair_term<D>(P, i, m->tsign[3 * p + i], Qg, j, m->tsign[3 * q + j], nr, k, Q, nullptr, nullptr);
          acc += Cx<D>(D(are[em]), D(-aim[em])) * c * Cx<D>(D(bre[en]), D(bim[en]));
        }
      }
      D Lp = -(k * fp->eta) * acc.im;
      L += Lp.v;
      gk += Lp.d[0];
    }
  }
  *loss = L;
  *dk = gk;
  return 0;
}

}  // extern "C"
