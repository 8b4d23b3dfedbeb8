// Oracle: quadrature rules and the adaptive interpolation tables.
// Test infrastructure only (see oracle.h).
//
// Tables follow Section II.B-C and Section III of Yang & Su:
//   * uniform sampling with interval t starting at r_min (Eq. 2),
//   * local refinement with a smaller interval near the zeros of the real and
//     imaginary parts, and forced sampling of the zeros themselves, dropping
//     nearby samples so the minimum interval stays large (Section II.B,
//     items 1 and 2),
//   * interpolation f(r) = sum_j f(r_j) P_{n,j}(r) (Eq. 3) with the linear
//     basis (Eq. 4) or the Lagrange basis (Eq. 5),
//   * the many-to-one hash [(r - r_min) / dr_min] (Eq. 6) into an array
//     filled at the sample positions and forward-filled elsewhere.
// Readings where the paper is silent (all recorded in the design notes):
//   * "range 4t" is the total width of the refinement window: |r - z| <= 2t;
//     every base interval that meets the window is split at spacing
//     refine_factor * t.
//   * "quite near" (item 2) means closer than `merge` (t/4); r_min and r_max
//     are forced samples too.
//   * grading: an interval whose Eq. (11) bound, divided by min |f| on it,
//     exceeds tol is bisected, repeated to a fixed point (the 1/r singularity
//     of e^{-jkr}/r makes uniform t too coarse near r_min at tol 1e-6).
//   * Lagrange stencil of degree n for interval j: nodes s0..s0+n with
//     s0 = clamp(j - (n-1)/2, 0, N-1-n).
#include <algorithm>
#include <cmath>
#include <vector>

#include "oracle.h"

namespace {

const double kPi = 3.14159265358979323846;

struct Table {
  or_table_params p;
  std::vector<double> r, fre, fim;
  std::vector<int> hash;
  double dr;
};

void exact_f(int kind, double k, double r, double* re, double* im) {
  double c = std::cos(k * r), s = std::sin(k * r);
  if (kind == 0) {
    *re = c;
    *im = -s;
  } else {
    *re = c / r;
    *im = -s / r;
  }
}

int stencil_start(int j, int degree, int n_nodes) {
  if (degree <= 1) return j;
  int s0 = j - (degree - 1) / 2;
  if (s0 > n_nodes - 1 - degree) s0 = n_nodes - 1 - degree;
  if (s0 < 0) s0 = 0;
  return s0;
}

double factorial(int n) {
  double f = 1;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

double binom(int n, int i) { return factorial(n) / (factorial(i) * factorial(n - i)); }

// Eq. (11): |f - f_n| <= prod |r - r_s| * |f^{(n+1)}(xi)| / (n+1)!, relative to
// min |f| on the interval. max prod|r - r_s| over [r_j, r_{j+1}] is bounded by
// (h^2/4) for the two interval ends times, for every other stencil node, the
// larger of its distances to the two interval ends. max |f^{(n+1)}| over the
// stencil span: k^{n+1} for e^{-jkr}; for e^{-jkr}/r the Leibniz rule gives
// sum_i C(n+1,i) k^{n+1-i} i! / r^{i+1}, largest at the left end of the span.
double rel_bound(const std::vector<double>& r, int j, int degree, int kind, double k) {
  int n = (int)r.size();
  int s0 = stencil_start(j, degree, n);
  double h = r[j + 1] - r[j];
  double om = h * h / 4.0;
  for (int s = s0; s <= s0 + degree; ++s) {
    if (s == j || s == j + 1) continue;
    om *= std::max(std::fabs(r[j] - r[s]), std::fabs(r[j + 1] - r[s]));
  }
  int q = degree + 1;
  double m;
  if (kind == 0) {
    m = std::pow(k, q);
  } else {
    m = 0;
    double rl = r[s0];
    for (int i = 0; i <= q; ++i) m += binom(q, i) * std::pow(k, q - i) * factorial(i) / std::pow(rl, i + 1);
  }
  double b = om * m / factorial(q);
  if (kind == 1) b *= r[j + 1];  // divide by min |f| = 1 / r_{j+1}
  return b;
}

int build(Table* T) {
  const or_table_params& p = T->p;
  double lo = p.r_lo, hi = p.r_hi, t = p.t;
  // 1) uniform samples starting at r_min (Eq. 2), r_max forced.
  std::vector<double> base;
  for (long i = 0;; ++i) {
    double x = lo + (double)i * t;
    if (x >= hi) break;
    base.push_back(x);
  }
  if (base.size() > 1 && hi - base.back() < p.merge) base.pop_back();
  base.push_back(hi);

  std::vector<double> nodes = base;
  if (p.refine) {
    double lam = 2.0 * kPi / p.k;
    double quarter = lam / 4.0;
    std::vector<double> zeros;
    std::vector<int> zq;
    for (long q = 1;; ++q) {
      double z = (double)q * quarter;
      if (z >= hi) break;
      if (z > lo) {
        zeros.push_back(z);
        zq.push_back((int)q);
      }
    }
    // 2) local refinement: base intervals meeting |r - z| <= halfwidth are
    //    split at spacing refine_factor * t.
    int nsub = (int)std::lround(1.0 / p.refine_factor);
    for (double z : zeros) {
      for (size_t i = 0; i + 1 < base.size(); ++i) {
        double a = base[i], b = base[i + 1];
        if (a < z + p.refine_halfwidth && b > z - p.refine_halfwidth) {
          for (int s = 1; s < nsub; ++s) nodes.push_back(a + (b - a) * s / nsub);
        }
      }
    }
    // 3) forced zero samples; samples closer than `merge` to a zero are dropped.
    for (double z : zeros) {
      if (z - lo < p.merge || hi - z < p.merge) continue;
      std::vector<double> kept;
      for (double x : nodes) {
        if (x != lo && x != hi && std::fabs(x - z) < p.merge) continue;
        kept.push_back(x);
      }
      kept.push_back(z);
      nodes.swap(kept);
    }
  }
  std::sort(nodes.begin(), nodes.end());
  nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());

  // 4) at least degree+1 nodes for the Lagrange stencil
  while ((int)nodes.size() < p.degree + 1) {
    std::vector<double> mids;
    for (size_t i = 0; i + 1 < nodes.size(); ++i) mids.push_back(0.5 * (nodes[i] + nodes[i + 1]));
    nodes.insert(nodes.end(), mids.begin(), mids.end());
    std::sort(nodes.begin(), nodes.end());
  }
  // 5) grading by the Eq. (11) bound
  if (p.grade) {
    for (int pass = 0; pass < 200; ++pass) {
      std::vector<double> mids;
      for (int j = 0; j + 1 < (int)nodes.size(); ++j) {
        if (rel_bound(nodes, j, p.degree, p.kind, p.k) > p.tol)
          mids.push_back(0.5 * (nodes[j] + nodes[j + 1]));
      }
      if (mids.empty()) break;
      nodes.insert(nodes.end(), mids.begin(), mids.end());
      std::sort(nodes.begin(), nodes.end());
      if (nodes.size() > 50000000) return -3;
    }
  }
  T->r = nodes;
  int n = (int)nodes.size();
  T->fre.resize(n);
  T->fim.resize(n);
  double lam = 2.0 * kPi / p.k;
  for (int j = 0; j < n; ++j) {
    exact_f(p.kind, p.k, nodes[j], &T->fre[j], &T->fim[j]);
  }
  // forced zeros carry an exact 0 in the vanishing part: z = q lambda/4 with
  // q odd zeroes the real part (cos), q even the imaginary part (sin).
  if (p.refine) {
    double quarter = lam / 4.0;
    for (int j = 0; j < n; ++j) {
      double q = nodes[j] / quarter;
      long qi = std::lround(q);
      if (qi >= 1 && (double)qi * quarter == nodes[j]) {
        if (qi % 2) T->fre[j] = 0.0;
        else T->fim[j] = 0.0;
      }
    }
  }
  // 6) hash (Eq. 6): cell width dr = min spacing, index placed at
  //    [(r_j - r_min)/dr], then empty cells take the previous cell's index.
  double dr = 1e300;
  for (int j = 0; j + 1 < n; ++j) dr = std::min(dr, nodes[j + 1] - nodes[j]);
  T->dr = dr;
  long L = (long)std::floor((hi - lo) / dr) + 1;
  if (L > 200000000L) return -3;
  T->hash.assign(L, -1);
  for (int j = 0; j < n; ++j) {
    long c = (long)std::floor((nodes[j] - lo) / dr);
    if (c >= 0 && c < L) T->hash[c] = j;
  }
  T->hash[0] = 0;
  for (long c = 1; c < L; ++c)
    if (T->hash[c] < 0) T->hash[c] = T->hash[c - 1];
  return 0;
}

int locate(const Table* T, double x) {
  int n = (int)T->r.size();
  long L = (long)T->hash.size();
  long c = (long)std::floor((x - T->p.r_lo) / T->dr);
  if (c < 0) c = 0;
  if (c > L - 1) c = L - 1;
  int j = T->hash[c];
  while (j > 0 && x < T->r[j]) --j;
  while (j < n - 2 && x >= T->r[j + 1]) ++j;
  if (j > n - 2) j = n - 2;
  return j;
}

void eval(const Table* T, double x, double* re, double* im) {
  int n = (int)T->r.size();
  int j = locate(T, x);
  const std::vector<double>& r = T->r;
  if (T->p.degree == 1) {
    // Eq. (4): P_j = (x - r_{j+1})/(r_j - r_{j+1}), P_{j+1} = (x - r_j)/(r_{j+1} - r_j)
    double pj = (x - r[j + 1]) / (r[j] - r[j + 1]);
    double pj1 = (x - r[j]) / (r[j + 1] - r[j]);
    *re = T->fre[j] * pj + T->fre[j + 1] * pj1;
    *im = T->fim[j] * pj + T->fim[j + 1] * pj1;
    return;
  }
  int deg = T->p.degree;
  int s0 = stencil_start(j, deg, n);
  double sr = 0, si = 0;
  for (int i = s0; i <= s0 + deg; ++i) {
    double P = 1.0;  // Eq. (5)
    for (int m = s0; m <= s0 + deg; ++m) {
      if (m == i) continue;
      P *= (x - r[m]) / (r[i] - r[m]);
    }
    sr += T->fre[i] * P;
    si += T->fim[i] * P;
  }
  *re = sr;
  *im = si;
}

}  // namespace

struct or_table {
  Table t;
};

namespace orc {
// Used by the fill: Exp / Green value from a table (caller checks the range).
void table_value(const or_table* T, double x, double* re, double* im) { eval(&T->t, x, re, im); }
double table_lo(const or_table* T) { return T->t.p.r_lo; }
double table_hi(const or_table* T) { return T->t.p.r_hi; }
}  // namespace orc

extern "C" {

int or_rule(int npts, double* bary, double* w) {
  auto put = [&](int i, double a, double b, double c, double wt) {
    bary[3 * i] = a;
    bary[3 * i + 1] = b;
    bary[3 * i + 2] = c;
    w[i] = wt;
  };
  auto orbit = [&](int i0, double a, double wt) {  // (a, a, 1-2a) and rotations
    double b = 1.0 - 2.0 * a;
    put(i0, b, a, a, wt);
    put(i0 + 1, a, b, a, wt);
    put(i0 + 2, a, a, b, wt);
  };
  switch (npts) {
    case 1:
      put(0, 1.0 / 3, 1.0 / 3, 1.0 / 3, 1.0);
      return 0;
    case 3:  // degree 2
      orbit(0, 1.0 / 6, 1.0 / 3);
      return 0;
    case 4:  // degree 3, negative centroid weight
      put(0, 1.0 / 3, 1.0 / 3, 1.0 / 3, -27.0 / 48);
      orbit(1, 0.2, 25.0 / 48);
      return 0;
    case 6: {
      // degree 4, two (a,a,1-2a) orbits. Exact for all degree-4 polynomials
      // iff exact for the S3 invariants 1, e2, e3, e2^2 of the barycentric
      // coordinates, whose triangle means are 1, 1/4, 1/60, 1/15. Solve those
      // four equations for (a1, a2, w1, w2) by Newton's method.
      double x[4] = {0.445, 0.091, 0.22, 0.11};
      for (int it = 0; it < 60; ++it) {
        double a = x[0], b = x[1], w1 = x[2], w2 = x[3];
        double e2a = 2 * a - 3 * a * a, e2b = 2 * b - 3 * b * b;
        double e3a = a * a - 2 * a * a * a, e3b = b * b - 2 * b * b * b;
        double d2a = 2 - 6 * a, d2b = 2 - 6 * b;
        double d3a = 2 * a - 6 * a * a, d3b = 2 * b - 6 * b * b;
        double F[4] = {3 * w1 + 3 * w2 - 1.0, 3 * w1 * e2a + 3 * w2 * e2b - 0.25,
                       3 * w1 * e3a + 3 * w2 * e3b - 1.0 / 60, 3 * w1 * e2a * e2a + 3 * w2 * e2b * e2b - 1.0 / 15};
        double J[4][4] = {{0, 0, 3, 3},
                          {3 * w1 * d2a, 3 * w2 * d2b, 3 * e2a, 3 * e2b},
                          {3 * w1 * d3a, 3 * w2 * d3b, 3 * e3a, 3 * e3b},
                          {6 * w1 * e2a * d2a, 6 * w2 * e2b * d2b, 3 * e2a * e2a, 3 * e2b * e2b}};
        // Gaussian elimination with partial pivoting: J dx = -F
        double A[4][5];
        for (int i = 0; i < 4; ++i) {
          for (int c = 0; c < 4; ++c) A[i][c] = J[i][c];
          A[i][4] = -F[i];
        }
        for (int c = 0; c < 4; ++c) {
          int piv = c;
          for (int i = c + 1; i < 4; ++i)
            if (std::fabs(A[i][c]) > std::fabs(A[piv][c])) piv = i;
          for (int cc = 0; cc < 5; ++cc) std::swap(A[c][cc], A[piv][cc]);
          for (int i = c + 1; i < 4; ++i) {
            double f = A[i][c] / A[c][c];
            for (int cc = c; cc < 5; ++cc) A[i][cc] -= f * A[c][cc];
          }
        }
        double dx[4];
        for (int i = 3; i >= 0; --i) {
          double s = A[i][4];
          for (int cc = i + 1; cc < 4; ++cc) s -= A[i][cc] * dx[cc];
          dx[i] = s / A[i][i];
        }
        for (int i = 0; i < 4; ++i) x[i] += dx[i];
      }
      orbit(0, x[0], x[2]);
      orbit(3, x[1], x[3]);
      return 0;
    }
    case 7: {  // degree 5 (Radon): centroid plus two orbits, closed form in sqrt(15)
      double s = std::sqrt(15.0);
      put(0, 1.0 / 3, 1.0 / 3, 1.0 / 3, 9.0 / 40);
      orbit(1, (6.0 - s) / 21.0, (155.0 - s) / 1200.0);
      orbit(4, (6.0 + s) / 21.0, (155.0 + s) / 1200.0);
      return 0;
    }
    default:
      return -1;
  }
}

int or_gauss_legendre(int n, double* x, double* w) {
  if (n < 1) return -1;
  // Legendre recurrence k P_k = (2k-1) z P_{k-1} - (k-1) P_{k-2}; Newton on
  // each root from z0 = cos(pi (i + 3/4) / (n + 1/2)).
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double pn = 0, pm = 0;
    for (int it = 0; it < 100; ++it) {
      pn = z;
      pm = 1.0;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * z * pn - (k - 1.0) * pm) / k;
        pm = pn;
        pn = pk;
      }
      if (n == 1) pm = 1.0;
      double dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    pn = z;
    pm = 1.0;
    for (int k = 2; k <= n; ++k) {
      double pk = ((2.0 * k - 1.0) * z * pn - (k - 1.0) * pm) / k;
      pm = pn;
      pn = pk;
    }
    double dp = n * (z * pn - pm) / (z * z - 1.0);
    x[i] = -z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  return 0;
}

int or_table_new(const or_table_params* p, or_table** out) {
  if (!p || !out) return -1;
  if (!(p->k > 0) || !(p->r_lo > 0) || !(p->r_hi > p->r_lo) || !(p->t > 0) || p->degree < 1 ||
      (p->kind != 0 && p->kind != 1) || !(p->tol > 0))
    return -1;
  if (p->refine && !(p->refine_factor > 0 && p->refine_factor <= 1)) return -1;
  or_table* T = new or_table;
  T->t.p = *p;
  int rc = build(&T->t);
  if (rc) {
    delete T;
    return rc;
  }
  *out = T;
  return 0;
}

int or_table_info(const or_table* T, int* n_nodes, int* n_hash, double* dr) {
  if (!T) return -1;
  if (n_nodes) *n_nodes = (int)T->t.r.size();
  if (n_hash) *n_hash = (int)T->t.hash.size();
  if (dr) *dr = T->t.dr;
  return 0;
}

int or_table_get(const or_table* T, double* r, double* fre, double* fim, int* hash) {
  if (!T) return -1;
  size_t n = T->t.r.size();
  for (size_t i = 0; i < n; ++i) {
    if (r) r[i] = T->t.r[i];
    if (fre) fre[i] = T->t.fre[i];
    if (fim) fim[i] = T->t.fim[i];
  }
  if (hash)
    for (size_t i = 0; i < T->t.hash.size(); ++i) hash[i] = T->t.hash[i];
  return 0;
}

int or_table_locate(const or_table* T, int n, const double* r, int* j) {
  if (!T) return -1;
  for (int i = 0; i < n; ++i) j[i] = locate(&T->t, r[i]);
  return 0;
}

int or_table_eval(const or_table* T, int n, const double* r, double* re, double* im) {
  if (!T) return -1;
  for (int i = 0; i < n; ++i) eval(&T->t, r[i], &re[i], &im[i]);
  return 0;
}

double or_table_bound(const or_table* T, int j) {
  return rel_bound(T->t.r, j, T->t.p.degree, T->t.p.kind, T->t.p.k);
}

void or_table_free(or_table* T) { delete T; }

}  // extern "C"
