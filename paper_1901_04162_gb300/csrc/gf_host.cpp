// gfmom host side: errors, quadrature rules, mesh topology (RWG edges, near
// pairs), table sample placement (FP64), and the C-ABI entry points.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "gf_internal.h"

namespace gf {

static thread_local std::string g_err;

gf_status fail(gf_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

gf_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? GF_ERR_ALLOC : GF_ERR_CUDA;
}

// Dunavant rules. Degree 2 (3 points), 3 (4 points, negative centroid
// weight), 4 (6 points), 5 (7 points, Radon's closed form in sqrt 15).
bool rule_points(int npts, double bary[][3], double* w) {
  int n = 0;
  auto one = [&](double a, double b, double c, double wt) {
    bary[n][0] = a;
    bary[n][1] = b;
    bary[n][2] = c;
    w[n] = wt;
    ++n;
  };
  auto s21 = [&](double a, double wt) {  // orbit of (1-2a, a, a)
    one(1.0 - 2.0 * a, a, a, wt);
    one(a, 1.0 - 2.0 * a, a, wt);
    one(a, a, 1.0 - 2.0 * a, wt);
  };
  if (npts == 1) {
    one(1.0 / 3, 1.0 / 3, 1.0 / 3, 1.0);
  } else if (npts == 3) {
    s21(1.0 / 6, 1.0 / 3);
  } else if (npts == 4) {
    one(1.0 / 3, 1.0 / 3, 1.0 / 3, -27.0 / 48);
    s21(0.2, 25.0 / 48);
  } else if (npts == 6) {
    s21(0.44594849091596488632, 0.22338158967801146570);
    s21(0.091576213509770743460, 0.10995174365532186764);
  } else if (npts == 7) {
    const double r15 = std::sqrt(15.0);
    one(1.0 / 3, 1.0 / 3, 1.0 / 3, 0.225);
    s21((6.0 - r15) / 21.0, (155.0 - r15) / 1200.0);
    s21((6.0 + r15) / 21.0, (155.0 + r15) / 1200.0);
  } else {
    return false;
  }
  return true;
}

// Gauss-Legendre nodes on [-1, 1] by Newton's method on the three-term
// recurrence of P_n.
static void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), d = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      d = n * (z * p1 - p2) / (z * z - 1.0);
      double dz = p1 / d;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p1 = 1.0, p2 = 0.0;
    for (int j = 1; j <= n; ++j) {
      double p3 = p2;
      p2 = p1;
      p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
    }
    d = n * (z * p1 - p2) / (z * z - 1.0);
    double wt = 2.0 / ((1.0 - z * z) * d * d);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = wt;
    w[n - 1 - i] = wt;
  }
  if (n % 2) x[n / 2] = 0.0;
}

// ---------------------------------------------------------------- table samples
struct Placement {
  std::vector<double> r;
  std::vector<int8_t> zflag;
  double dr;
  int64_t n_hash;
};

static double fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

// Eq. (11) bound of interval j relative to min |f| on it (see
// gf_table_create). The factors that do not depend on the interval (powers of
// k, factorials, binomials) are formed once, by the same operations in the
// same order as a per-interval evaluation, so the bound is the same number.
struct Eq11 {
  int deg, kind, q;
  double fq, kq, c[8];
  Eq11(int deg_, int kind_, double k) : deg(deg_), kind(kind_), q(deg_ + 1) {
    fq = fact(q);
    kq = std::pow(k, q);
    for (int i = 0; i <= q && i < 8; ++i) c[i] = fact(q) / (fact(i) * fact(q - i)) * std::pow(k, q - i) * fact(i);
  }
  static int stencil(int j, int deg, int n) { return deg <= 1 ? j : std::min(std::max(j - (deg - 1) / 2, 0), n - 1 - deg); }
  double operator()(const std::vector<double>& r, int j) const {
    const int s0 = stencil(j, deg, (int)r.size());
    const double h = r[j + 1] - r[j];
    double om = h * h / 4.0;
    for (int s = s0; s <= s0 + deg; ++s)
      if (s != j && s != j + 1) om *= std::max(std::fabs(r[j] - r[s]), std::fabs(r[j + 1] - r[s]));
    double mq = 0.0;
    if (kind == GF_EXP) {
      mq = kq;
    } else {
      for (int i = 0; i <= q; ++i) mq += c[i] / std::pow(r[s0], i + 1);
    }
    const double b = om * mq / fq;
    return kind == GF_GREEN ? b * r[j + 1] : b;
  }
};

// The same bound with the powers of 1/r formed by products (equal to Eq11 up
// to a few ulps): a screen, so that Eq11 runs only on intervals whose bound is
// within a factor 2 of the tolerance and the grading decisions do not depend
// on the screen.
struct Eq11Screen {
  int deg, kind, q;
  double kq, inv_fq, kp[8], cf[8];
  Eq11Screen(int deg_, int kind_, double k) : deg(deg_), kind(kind_), q(deg_ + 1) {
    kp[0] = 1.0;
    for (int i = 1; i < 8; ++i) kp[i] = kp[i - 1] * k;
    kq = kp[q < 8 ? q : 7];
    inv_fq = 1.0 / fact(q);
    for (int i = 0; i <= q && i < 8; ++i) cf[i] = fact(q) / (fact(i) * fact(q - i)) * fact(i);
  }
  double operator()(const std::vector<double>& r, int j) const {
    const int s0 = Eq11::stencil(j, deg, (int)r.size());
    const double h = r[j + 1] - r[j];
    double om = h * h / 4.0;
    for (int s = s0; s <= s0 + deg; ++s)
      if (s != j && s != j + 1) om *= std::max(std::fabs(r[j] - r[s]), std::fabs(r[j + 1] - r[s]));
    double mq = 0.0;
    if (kind == GF_EXP) {
      mq = kq;
    } else {
      const double inv_r = 1.0 / r[s0];
      double ir = inv_r;
      for (int i = 0; i <= q; ++i, ir *= inv_r) mq += cf[i] * kp[q - i] * ir;
    }
    const double b = om * mq * inv_fq;
    return kind == GF_GREEN ? b * r[j + 1] : b;
  }
};

static gf_status place_samples(int kind, int deg, double k, double lo, double hi, double t,
                               const gf_params& p, Placement* out) {
  const double merge = p.merge_t * t;
  const double hw = p.refine_halfwidth_t * t;
  // uniform samples from r_min with spacing t (Eq. 2); r_max is a sample
  std::vector<double> base;
  if ((hi - lo) / t < (double)(1u << 26)) base.reserve((size_t)((hi - lo) / t) + 2);
  for (int64_t i = 0;; ++i) {
    const double x = lo + (double)i * t;
    if (x >= hi) break;
    base.push_back(x);
    if (base.size() > (1u << 26)) return fail(GF_ERR_RANGE, "table: too many samples");
  }
  if (base.size() > 1 && hi - base.back() < merge) base.pop_back();
  base.push_back(hi);
  std::vector<double> all = base;
  std::vector<double> zeros;
  const double lam = 2.0 * kPi / k;
  const double quarter = lam / 4.0;
  if (p.refine) {
    // zeros of Re / Im of e^{-jkr} (and of e^{-jkr}/r): r = q lambda / 4
    for (int64_t q = 1;; ++q) {
      const double z = (double)q * quarter;
      if (z >= hi) break;
      if (z > lo) zeros.push_back(z);
    }
    const int nsub = (int)std::lround(1.0 / p.refine_factor);
    std::vector<double> extra;
    for (double z : zeros) {
      // base intervals meeting the window [z - hw, z + hw] are subdivided
      auto it = std::lower_bound(base.begin(), base.end(), z - hw);
      size_t i0 = (it == base.begin()) ? 0 : (size_t)(it - base.begin()) - 1;
      for (size_t i = i0; i + 1 < base.size() && base[i] < z + hw; ++i) {
        const double a = base[i], b = base[i + 1];
        if (b > z - hw)
          for (int s = 1; s < nsub; ++s) extra.push_back(a + (b - a) * s / nsub);
      }
    }
    // sorted union of the (sorted) base samples and the refinement samples
    std::sort(extra.begin(), extra.end());
    all.resize(base.size() + extra.size());
    std::merge(base.begin(), base.end(), extra.begin(), extra.end(), all.begin());
    // forced zeros: keep z, drop other samples within `merge` of it
    std::vector<double> kept_zeros;
    for (double z : zeros)
      if (z - lo >= merge && hi - z >= merge) kept_zeros.push_back(z);
    std::vector<double> tmp;
    tmp.reserve(all.size());
    size_t z0 = 0;  // first kept zero >= x - merge (x ascends)
    for (double x : all) {
      bool drop = false;
      if (x != lo && x != hi) {
        while (z0 < kept_zeros.size() && kept_zeros[z0] < x - merge) ++z0;
        for (size_t zi = z0; zi < kept_zeros.size() && kept_zeros[zi] <= x + merge; ++zi)
          if (std::fabs(x - kept_zeros[zi]) < merge) drop = true;
      }
      if (!drop) tmp.push_back(x);
    }
    all.resize(tmp.size() + kept_zeros.size());
    std::merge(tmp.begin(), tmp.end(), kept_zeros.begin(), kept_zeros.end(), all.begin());
  }
  // `all` is sorted here (merges of sorted lists); the sample set is the same
  // as sorting the union
  all.erase(std::unique(all.begin(), all.end()), all.end());
  while ((int)all.size() < deg + 1) {
    const size_t n = all.size();
    for (size_t i = 0; i + 1 < n; ++i) all.push_back(0.5 * (all[i] + all[i + 1]));
    std::sort(all.begin(), all.end());
  }
  if (p.grade) {
    // bisection passes; an interval is examined again only when a new sample
    // lies within its stencil's reach (deg + 1 samples either side): the bound
    // of any other interval is unchanged, so it passes again
    const Eq11Screen screen(deg, kind, k);
    const Eq11 exact(deg, kind, k);
    const bool exact_only = deg + 1 >= 8;
    std::vector<char> dirty(all.size(), 1), fresh;
    std::vector<double> add, merged;
    for (int pass = 0; pass < 200; ++pass) {
      add.clear();
      for (int j = 0; j + 1 < (int)all.size(); ++j)
        if (dirty[j] && (exact_only || kind == GF_EXP || screen(all, j) > 0.5 * p.table_tol) &&
            exact(all, j) > p.table_tol)
          add.push_back(0.5 * (all[j] + all[j + 1]));
      if (add.empty()) break;
      // sorted union (`add` ascends with j), marking the new samples
      merged.resize(all.size() + add.size());
      fresh.assign(merged.size(), 0);
      size_t ia = 0, ib = 0, o = 0;
      while (ia < all.size() || ib < add.size()) {
        if (ib < add.size() && (ia == all.size() || add[ib] < all[ia])) {
          fresh[o] = 1;
          merged[o++] = add[ib++];
        } else {
          merged[o++] = all[ia++];
        }
      }
      all.swap(merged);
      if (all.size() > (1u << 26)) return fail(GF_ERR_RANGE, "table: too many samples");
      const int reach = deg + 2, n = (int)all.size();
      dirty.assign(n, 0);
      for (int i = 0; i < n; ++i)
        if (fresh[i])
          for (int j = std::max(i - reach, 0); j <= std::min(i + reach, n - 1); ++j) dirty[j] = 1;
    }
  }
  out->zflag.assign(all.size(), 0);
  if (p.refine) {
    const double inv_quarter = 1.0 / quarter;  // a multiple of quarter is recognised either way
    for (size_t j = 0; j < all.size(); ++j) {
      const double q = std::nearbyint(all[j] * inv_quarter);
      if (q >= 1 && q * quarter == all[j]) out->zflag[j] = ((int64_t)q % 2) ? 1 : 2;
    }
  }
  double dr = INFINITY;
  for (size_t j = 0; j + 1 < all.size(); ++j) dr = std::min(dr, all[j + 1] - all[j]);
  out->dr = dr;
  out->r = std::move(all);
  const double cells = std::floor((hi - lo) / dr) + 1.0;
  if (!(cells < (double)(1 << 26))) return fail(GF_ERR_RANGE, "table: hash array too large");
  out->n_hash = (int64_t)cells;
  return GF_OK;
}

}  // namespace gf

using namespace gf;

gf::TabView gf_table::One::view() const {
  gf::TabView v;
  v.n_nodes = (int)r.size();
  v.n_hash = (int)n_hash;
  v.r_lo = r.front();
  v.r_hi = r.back();
  v.dr = dr;
  v.inv_dr = 1.0 / dr;
  v.r_lo32 = (float)r.front();
  v.inv_dr32 = (float)(1.0 / dr);
  v.hash = d_hash;
  v.node64 = d_node64;
  v.c64 = d_c64;
  v.node32 = d_node32;
  v.c32a = d_c32a;
  v.c32b = d_c32b;
  v.n_lat = n_lat;
  v.n_sub = n_sub;
  v.lat_inv = lat_inv;
  v.lat_nc = lat_nc;
  v.lat_h = lat_h;
  v.lat_lo = lat_lo;
  v.lat_a = d_lat_a;
  v.lat_blob = d_lat_blob;
  v.n_busy = n_busy;
  v.n_cmp = n_cmp;
  v.lat_c = d_lat_c;
  v.lat_amid = lat_amid;
  v.lat_c2d = lat_c2d;
  v.n_cells64 = n_cells64;
  v.lo64c = lo64c;
  v.inv64c = inv64c;
  v.cells64 = d_cells64;
  return v;
}

namespace {

// Device memory of destroyed tables and meshes (arrays and flagged-pair
// lists) kept for the next one of a similar size on the same device (a table
// is rebuilt for every range / k; cudaMalloc costs as much as building it,
// and a device allocation between stream operations can serialize them). At
// most kPoolBlocks blocks, kPoolBytes bytes.
constexpr int kPoolBlocks = 16;
constexpr size_t kPoolBytes = size_t(2) << 30;

struct ArenaPool {
  std::mutex mu;
  struct Block {
    int device;
    void* ptr;
    size_t bytes;
  };
  std::vector<Block> blocks;
  size_t held = 0;
};

ArenaPool& arena_pool() {
  static ArenaPool* p = new ArenaPool;  // never destroyed: blocks live until the process exits
  return *p;
}

// A pooled block of at least `bytes` (and at most twice that) on `device`, or null.
void* arena_take(int device, size_t bytes, size_t* got) {
  ArenaPool& P = arena_pool();
  std::lock_guard<std::mutex> lock(P.mu);
  int best = -1;
  for (int i = 0; i < (int)P.blocks.size(); ++i) {
    const ArenaPool::Block& b = P.blocks[i];
    if (b.device == device && b.bytes >= bytes && b.bytes <= 2 * bytes + (1 << 20) &&
        (best < 0 || b.bytes < P.blocks[best].bytes))
      best = i;
  }
  if (best < 0) return nullptr;
  void* ptr = P.blocks[best].ptr;
  *got = P.blocks[best].bytes;
  P.held -= *got;
  P.blocks.erase(P.blocks.begin() + best);
  return ptr;
}

// Called with no work in flight on the block (the caller synchronized the device).
void arena_give(int device, void* ptr, size_t bytes) {
  ArenaPool& P = arena_pool();
  {
    std::lock_guard<std::mutex> lock(P.mu);
    if ((int)P.blocks.size() < kPoolBlocks && P.held + bytes <= kPoolBytes) {
      P.blocks.push_back(ArenaPool::Block{device, ptr, bytes});
      P.held += bytes;
      return;
    }
  }
  cudaFree(ptr);
}

template <class T>
gf_status dev_alloc(T** p, size_t n) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  return GF_OK;
}

gf_status check_device(int dev) {
  int cur = -1;
  GF_CUDA(cudaGetDevice(&cur));
  if (cur != dev) return fail(GF_ERR_DEVICE, "handle belongs to device " + std::to_string(dev));
  return GF_OK;
}

void free_mesh_device(gf_mesh* m) {
  if (m->d_arena) {
    cudaDeviceSynchronize();  // no work in flight on the arena when it goes back to the pool
    arena_give(m->device, m->d_arena, m->arena_bytes);
    m->d_arena = nullptr;
  }
  if (m->d_dtri) cudaFree(m->d_dtri);
  if (m->d_dk) cudaFree(m->d_dk);
  if (m->h_range) cudaFreeHost(m->h_range);
  if (m->d_fix) {
    cudaDeviceSynchronize();
    arena_give(m->device, m->d_fix, m->fix_bytes);
  }
  m->d_fix = nullptr;
  m->fix_cap = 0;
  m->fix_bytes = 0;
  m->d_dtri = nullptr;
  m->d_dk = nullptr;
  m->h_range = nullptr;
}

// Triangle corners (internal order) and RWG edge lengths, laid out as on the
// device (elen follows v64 at a 256-byte aligned offset).
void vertex_arrays(const gf_mesh* m, unsigned char* dst) {
  double* v64 = reinterpret_cast<double*>(dst);
  for (int64_t i = 0; i < m->nt; ++i) {
    const int64_t t = m->perm[i];
    for (int c = 0; c < 3; ++c)
      for (int x = 0; x < 3; ++x) v64[9 * i + 3 * c + x] = m->xyz[3 * (size_t)m->tri[3 * t + c] + x];
  }
  double* elen = reinterpret_cast<double*>(dst + (reinterpret_cast<unsigned char*>(m->d_elen) -
                                                  reinterpret_cast<unsigned char*>(m->d_v64)));
  for (int64_t e = 0; e < m->ne; ++e) {
    double s = 0;
    for (int x = 0; x < 3; ++x) {
      double d = m->xyz[3 * (size_t)m->ev[2 * e] + x] - m->xyz[3 * (size_t)m->ev[2 * e + 1] + x];
      s += d * d;
    }
    elen[e] = std::sqrt(s);
  }
}

// Step 2^e of the block-centre grid: every coordinate of the mesh (and so of
// every block centre) below 2^14 - 2 steps, so block separations stay below
// 2^15 steps and |B|^2 fits an unsigned 32-bit integer.
void set_block_grid(gf_mesh* m) {
  double mx = 0.0;
  for (double x : m->xyz) mx = std::max(mx, std::fabs(x));
  int e = -60;
  while (e < 100 && std::ldexp(16382.0, e) <= mx) ++e;
  m->bgrid_e = e;
}

size_t vertex_bytes(const gf_mesh* m) {
  return (size_t)(reinterpret_cast<unsigned char*>(m->d_elen) - reinterpret_cast<unsigned char*>(m->d_v64)) +
         (size_t)std::max<int64_t>(m->ne, 1) * 8;
}

gf_status upload_vertices(gf_mesh* m) {
  std::vector<unsigned char> h(vertex_bytes(m), 0);
  vertex_arrays(m, h.data());
  GF_CUDA(cudaMemcpy(m->d_v64, h.data(), h.size(), cudaMemcpyHostToDevice));
  m->rule = 0;  // geometry cache invalid
  return GF_OK;
}

// Stable LSD radix sort (8-bit digits over the low `bits` bits): the order of
// the keys, equal keys in input order.
std::vector<int32_t> radix_order(const std::vector<uint64_t>& key, int bits) {
  const size_t n = key.size();
  std::vector<int32_t> a(n), b(n);
  std::vector<uint64_t> k(key), kb(n);  // keys carried along with the order
  for (size_t i = 0; i < n; ++i) a[i] = (int32_t)i;
  uint32_t cnt[257];
  for (int sh = 0; sh < bits; sh += 8) {
    std::fill(cnt, cnt + 257, 0u);
    for (size_t i = 0; i < n; ++i) ++cnt[((k[i] >> sh) & 0xFF) + 1];
    if (cnt[1] == n) continue;  // every digit 0
    for (int d = 0; d < 256; ++d) cnt[d + 1] += cnt[d];
    for (size_t i = 0; i < n; ++i) {
      const uint32_t o = cnt[(k[i] >> sh) & 0xFF]++;
      b[o] = a[i];
      kb[o] = k[i];
    }
    a.swap(b);
    k.swap(kb);
  }
  return a;
}

int bit_width(uint64_t v) {
  int b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

// Builds (or reuses) the per-rule geometry on the device.
GeoView geo_view_impl(const gf_mesh* m);

gf_status prepare_rule_impl(gf_mesh* m, int rule, cudaStream_t s) {
  if (m->rule == rule) return GF_OK;
  double bary[kMaxRule][3], w[kMaxRule];
  if (!rule_points(rule, bary, w)) return fail(GF_ERR_ARG, "rule must be 1, 3, 4, 6 or 7");
  double* d_bw = nullptr;
  gf_status st = dev_alloc(&d_bw, 4 * kMaxRule);
  if (st) return st;
  std::vector<double> bw(4 * kMaxRule, 0.0);
  for (int a = 0; a < rule; ++a) {
    for (int c = 0; c < 3; ++c) bw[3 * a + c] = bary[a][c];
    bw[3 * kMaxRule + a] = w[a];
  }
  cudaError_t e = cudaMemcpy(d_bw, bw.data(), bw.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = launch_prep_geometry(m->d_v64, (int)m->nt, rule, d_bw, d_bw + 3 * kMaxRule, m->d_tedge, m->d_elen,
                             m->d_pts32, m->d_cen32, m->d_geo32, m->d_pts64, m->d_cen64, m->d_geo64, m->d_rad32,
                             m->d_frame64, m->d_frame32, s);
  if (e == cudaSuccess) {
    m->rule = rule;  // views below read the new geometry
    e = launch_block_frames(geo_view_impl(m), m->d_bsph, m->d_bgrid, m->d_rel32, m->d_geob32, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_bw);
  if (e != cudaSuccess) {
    m->rule = 0;
    return cuda_fail(e, "prepare geometry");
  }
  m->rule = rule;
  return GF_OK;
}

GeoView geo_view_impl(const gf_mesh* m) {
  GeoView g;
  g.nt = (int)m->nt;
  g.m = m->rule;
  g.pts32 = m->d_pts32;
  g.cen32 = m->d_cen32;
  g.geo32 = m->d_geo32;
  g.pts64 = m->d_pts64;
  g.cen64 = m->d_cen64;
  g.geo64 = m->d_geo64;
  g.v64 = m->d_v64;
  g.frame64 = m->d_frame64;
  g.frame32 = m->d_frame32;
  g.tvert = m->d_tvert;
  g.tedge = m->d_tedge;
  g.near_ptr = m->d_near_ptr;
  g.near_idx = m->d_near_idx;
  g.near_row = m->d_near_row;
  g.near_dist32 = (float)m->near_dist;
  g.rad32 = m->d_rad32;
  g.bsph = m->d_bsph;
  g.bgrid = m->d_bgrid;
  g.rel32 = m->d_rel32;
  g.geob32 = m->d_geob32;
  g.bunit = std::ldexp(1.f, m->bgrid_e);
  g.bunit2 = std::ldexp(1.f, 2 * m->bgrid_e);
  return g;
}

bool params_ok(const gf_params* p) {
  return p && p->table_tol > 0 && p->green_n_per_lambda >= 0 && p->exp_n_per_lambda >= 0 &&
         p->lagrange_degree >= 1 && p->lagrange_degree <= 3 && p->refine_factor > 0 && p->refine_factor <= 1 &&
         p->refine_halfwidth_t >= 0 && p->merge_t >= 0 && p->nphi >= 1 && p->nphi <= 32 && p->nl >= 1 &&
         p->nl <= 32 && p->eta > 0 && (p->near_fp64 == 0 || p->near_fp64 == 1) &&
         (p->green_from_exp == 0 || p->green_from_exp == 1);
}

}  // namespace

namespace gf {
gf_status prepare_rule(gf_mesh* m, int rule, cudaStream_t s) { return ::prepare_rule_impl(m, rule, s); }
GeoView geo_view(const gf_mesh* m) { return ::geo_view_impl(m); }
void gauss_legendre_host(int n, double* x, double* w) { gauss_legendre(n, x, w); }
}  // namespace gf

extern "C" {

void gf_params_default(gf_params* p) {
  if (!p) return;
  p->rule = 3;
  p->table_tol = 1e-6;
  p->green_n_per_lambda = 1000;
  p->exp_n_per_lambda = 0;
  p->lagrange_degree = 3;
  p->refine = 1;
  p->refine_factor = 0.5;
  p->refine_halfwidth_t = 2.0;
  p->merge_t = 0.25;
  p->grade = 1;
  p->nphi = 8;
  p->nl = 8;
  p->eta = 376.730313668;
  p->near_fp64 = 0;
  p->green_from_exp = 0;
}

const char* gf_last_error(void) { return gf::g_err.c_str(); }

gf_status gf_mesh_create(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, double near_dist,
                         gf_mesh** out) {
  if (!xyz || !tri || !out || nv < 3 || nt < 1) return fail(GF_ERR_ARG, "gf_mesh_create: bad arguments");
  if (nt > (1LL << 30) || nv > (1LL << 31) - 1) return fail(GF_ERR_ARG, "gf_mesh_create: mesh too large");
  if (!(near_dist >= 0)) return fail(GF_ERR_ARG, "gf_mesh_create: near_dist must be >= 0");
  for (int64_t i = 0; i < 3 * nv; ++i)
    if (!std::isfinite(xyz[i])) return fail(GF_ERR_MESH, "gf_mesh_create: non-finite vertex coordinate");
  std::unique_ptr<gf_mesh> m(new (std::nothrow) gf_mesh);
  if (!m) return fail(GF_ERR_ALLOC, "gf_mesh_create: out of host memory");
  GF_CUDA(cudaGetDevice(&m->device));
  m->nv = nv;
  m->nt = nt;
  m->near_dist = near_dist;
  m->xyz.assign(xyz, xyz + 3 * nv);
  set_block_grid(m.get());
  m->tri.assign(tri, tri + 3 * nt);
  // ---- RWG edges: records (lower, higher vertex) in (triangle, local index)
  // order, sorted stably by the vertex pair (radix)
  for (int64_t t = 0; t < nt; ++t) {
    const int32_t* v = &tri[3 * t];
    for (int c = 0; c < 3; ++c) {
      if (v[c] < 0 || v[c] >= nv) return fail(GF_ERR_MESH, "gf_mesh_create: vertex index out of range");
    }
    if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2]) return fail(GF_ERR_MESH, "gf_mesh_create: repeated vertex");
  }
  const int vb = std::max(bit_width((uint64_t)(nv - 1)), 1);
  std::vector<uint64_t> ekey(3 * nt);
  for (int64_t t = 0; t < nt; ++t)
    for (int i = 0; i < 3; ++i) {  // local edge i is opposite local vertex i
      const int32_t a = tri[3 * t + (i + 1) % 3], b = tri[3 * t + (i + 2) % 3];
      ekey[3 * t + i] = ((uint64_t)std::min(a, b) << vb) | (uint64_t)std::max(a, b);
    }
  const std::vector<int32_t> eorder = radix_order(ekey, 2 * vb);
  m->tedge.assign(3 * nt, -1);
  m->ev.reserve(3 * nt);
  m->et.reserve(3 * nt);
  for (size_t i = 0; i < eorder.size();) {
    size_t j = i;
    while (j < eorder.size() && ekey[eorder[j]] == ekey[eorder[i]]) ++j;
    if (j - i > 2) return fail(GF_ERR_MESH, "gf_mesh_create: edge shared by more than two triangles");
    if (j - i == 2) {
      const int32_t e = (int32_t)m->ev.size() / 2;
      const int32_t r0 = eorder[i], r1 = eorder[i + 1];  // input order: T+ first
      const int32_t tp = r0 / 3, tm = r1 / 3;
      if (tp == tm) return fail(GF_ERR_MESH, "gf_mesh_create: degenerate triangle");
      m->ev.push_back((int32_t)(ekey[r0] >> vb));
      m->ev.push_back((int32_t)(ekey[r0] & ((uint64_t(1) << vb) - 1)));
      m->et.push_back(tp);
      m->et.push_back(tm);
      m->tedge[r0] = 2 * e;      // even: T+ side
      m->tedge[r1] = 2 * e + 1;  // odd: T- side
    }
    i = j;
  }
  m->ne = (int64_t)m->ev.size() / 2;
  // ---- internal triangle order: Morton order of the centroids (locality of
  // table windows, Z rows and range pruning); outputs use the original ids
  std::vector<double> cen(3 * nt);
  for (int64_t t = 0; t < nt; ++t)
    for (int x = 0; x < 3; ++x)
      cen[3 * t + x] = (xyz[3 * (size_t)tri[3 * t] + x] + xyz[3 * (size_t)tri[3 * t + 1] + x] +
                        xyz[3 * (size_t)tri[3 * t + 2] + x]) / 3.0;
  {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t t = 0; t < nt; ++t)
      for (int x = 0; x < 3; ++x) {
        lo[x] = std::min(lo[x], cen[3 * t + x]);
        hi[x] = std::max(hi[x], cen[3 * t + x]);
      }
    double ext = std::max(std::max(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
    const double scale = ext > 0 ? 2097151.0 / ext : 0.0;
    auto spread = [](uint64_t v) {  // 21 bits -> every third bit
      v &= 0x1FFFFF;
      v = (v | (v << 32)) & 0x1F00000000FFFFULL;
      v = (v | (v << 16)) & 0x1F0000FF0000FFULL;
      v = (v | (v << 8)) & 0x100F00F00F00F00FULL;
      v = (v | (v << 4)) & 0x10C30C30C30C30C3ULL;
      v = (v | (v << 2)) & 0x1249249249249249ULL;
      return v;
    };
    std::vector<uint64_t> code(nt);
    for (int64_t t = 0; t < nt; ++t) {
      uint64_t c = 0;
      for (int x = 0; x < 3; ++x) c |= spread((uint64_t)((cen[3 * t + x] - lo[x]) * scale)) << x;
      code[t] = c;
    }
    m->perm = radix_order(code, 63);  // ties in triangle order
    m->inv_perm.resize(nt);
    for (int64_t i = 0; i < nt; ++i) m->inv_perm[m->perm[i]] = (int32_t)i;
  }
  // ---- near pairs (internal ids): vertex sharing, plus centroids closer
  // than near_dist
  // vertex stars: the triangles (internal ids, ascending) of each vertex
  std::vector<int32_t> vptr(nv + 1, 0), vtri(3 * nt);
  for (int64_t i = 0; i < 3 * nt; ++i) ++vptr[tri[i] + 1];
  for (int64_t v = 0; v < nv; ++v) vptr[v + 1] += vptr[v];
  {
    std::vector<int32_t> fillp(vptr.begin(), vptr.end() - 1);
    for (int64_t pi = 0; pi < nt; ++pi)
      for (int c = 0; c < 3; ++c) vtri[fillp[tri[3 * (size_t)m->perm[pi] + c]]++] = (int32_t)pi;
  }
  // centroid grid of cell near_dist over the internal ids, as sorted cell
  // keys with the ids of each cell (a pair closer than near_dist lies in
  // neighbouring cells)
  const double cell = near_dist;
  auto key = [](int64_t a, int64_t b, int64_t c) {
    return (uint64_t)(((a & 0x1FFFFF) << 42) | ((b & 0x1FFFFF) << 21) | (c & 0x1FFFFF));
  };
  auto cell_of = [&](int64_t t, int x) { return (int64_t)std::floor(cen[3 * t + x] / cell); };
  struct CellPt {  // a centroid and its internal id, stored by cell
    double x, y, z;
    int32_t id;
  };
  std::vector<uint64_t> ckey, cells;  // key of each internal id; distinct keys, ascending
  std::vector<int32_t> cell_ptr;     // offsets of the distinct keys' runs in cpts
  std::vector<CellPt> cpts;
  if (near_dist > 0) {
    ckey.resize(nt);
    for (int64_t pi = 0; pi < nt; ++pi) {
      const int64_t t = m->perm[pi];
      ckey[pi] = key(cell_of(t, 0), cell_of(t, 1), cell_of(t, 2));
    }
    const std::vector<int32_t> by_cell = radix_order(ckey, 63);  // ascending key, ids ascending within a cell
    cpts.resize(nt);
    for (int64_t i = 0; i < nt; ++i) {
      const int32_t qi = by_cell[i];
      const size_t q = (size_t)m->perm[qi];
      cpts[i] = CellPt{cen[3 * q], cen[3 * q + 1], cen[3 * q + 2], qi};
      const uint64_t k = ckey[qi];
      if (cells.empty() || cells.back() != k) {
        cells.push_back(k);
        cell_ptr.push_back((int32_t)i);
      }
    }
    cell_ptr.push_back((int32_t)nt);
  }
  // union of ascending lists, without repeats
  auto merge_into = [](const int32_t* a, int na, const int32_t* b, int nb, std::vector<int32_t>& out) {
    out.clear();
    int i = 0, j = 0;
    while (i < na || j < nb) {
      int32_t x;
      if (j >= nb || (i < na && a[i] < b[j])) x = a[i++];
      else if (i >= na || b[j] < a[i]) x = b[j++];
      else {
        x = a[i++];
        ++j;
      }
      out.push_back(x);
    }
  };
  // rows of the near list (ascending internal ids): the vertex stars of the
  // three vertices, plus the centroids closer than near_dist (the distance
  // compared as sqrt(d2) < near_dist, decided on d2 where it is clear by a
  // margin far above the rounding); built in chunks of rows on several host
  // threads for large meshes, then concatenated in row order
  const double lim_lo = near_dist * near_dist * (1.0 - 1e-9), lim_hi = near_dist * near_dist * (1.0 + 1e-9);
  auto build_rows = [&](int64_t p0, int64_t p1, std::vector<int32_t>& idx, std::vector<int64_t>& cnt) {
    std::vector<int32_t> ab, row, close;
    for (int64_t pi = p0; pi < p1; ++pi) {
      const int64_t p = m->perm[pi];  // original id
      const int32_t* v = &tri[3 * p];
      merge_into(&vtri[vptr[v[0]]], vptr[v[0] + 1] - vptr[v[0]], &vtri[vptr[v[1]]], vptr[v[1] + 1] - vptr[v[1]], ab);
      merge_into(ab.data(), (int)ab.size(), &vtri[vptr[v[2]]], vptr[v[2] + 1] - vptr[v[2]], row);
      if (near_dist > 0) {
        close.clear();
        const int64_t gx = cell_of(p, 0), gy = cell_of(p, 1), gz = cell_of(p, 2);
        for (int dx = -1; dx <= 1; ++dx)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
              const uint64_t k = key(gx + dx, gy + dy, gz + dz);
              const auto it = std::lower_bound(cells.begin(), cells.end(), k);
              if (it == cells.end() || *it != k) continue;
              const size_t c = (size_t)(it - cells.begin());
              for (int32_t i = cell_ptr[c]; i < cell_ptr[c + 1]; ++i) {
                const CellPt& cq = cpts[i];
                const double ax = cen[3 * p] - cq.x, ay = cen[3 * p + 1] - cq.y, az = cen[3 * p + 2] - cq.z;
                const double d2 = ax * ax + ay * ay + az * az;
                if (d2 >= lim_hi) continue;
                if (d2 < lim_lo || std::sqrt(d2) < near_dist) close.push_back(cq.id);
              }
            }
        std::sort(close.begin(), close.end());
        close.erase(std::unique(close.begin(), close.end()), close.end());
        ab.swap(row);
        merge_into(ab.data(), (int)ab.size(), close.data(), (int)close.size(), row);
      }
      idx.insert(idx.end(), row.begin(), row.end());
      cnt.push_back((int64_t)row.size());
    }
  };
  int nthr = 1;
  if (nt >= 8192) nthr = (int)std::min<unsigned>(std::max(std::thread::hardware_concurrency(), 1u), 16u);
  std::vector<std::vector<int32_t>> part_idx(nthr);
  std::vector<std::vector<int64_t>> part_cnt(nthr);
  std::vector<char> part_failed(nthr, 0);
  {
    std::vector<std::thread> pool;
    auto chunk = [&](int w) {
      try {  // (no exception may leave a thread)
        const int64_t p0 = nt * w / nthr, p1 = nt * (w + 1) / nthr;
        part_cnt[w].reserve(p1 - p0);
        part_idx[w].reserve(16 * (size_t)(p1 - p0));
        build_rows(p0, p1, part_idx[w], part_cnt[w]);
      } catch (...) {
        part_failed[w] = 1;
      }
    };
    for (int w = 1; w < nthr; ++w) {
      try {
        pool.emplace_back(chunk, w);
      } catch (...) {  // no thread: this one builds the chunk afterwards
        pool.emplace_back();
      }
    }
    chunk(0);
    for (int w = 1; w < nthr; ++w) {
      if (pool[w - 1].joinable()) pool[w - 1].join();
      else chunk(w);
    }
  }
  for (int w = 0; w < nthr; ++w)
    if (part_failed[w]) return fail(GF_ERR_ALLOC, "gf_mesh_create: out of host memory (near rows)");
  m->near_ptr.assign(nt + 1, 0);
  size_t total = 0;
  for (int w = 0; w < nthr; ++w) total += part_idx[w].size();
  m->near_idx.resize(total);
  {
    int64_t pi = 0;
    size_t at = 0;
    for (int w = 0; w < nthr; ++w) {
      if (!part_idx[w].empty()) std::memcpy(&m->near_idx[at], part_idx[w].data(), part_idx[w].size() * 4);
      at += part_idx[w].size();
      for (int64_t c : part_cnt[w]) {
        m->near_ptr[pi + 1] = m->near_ptr[pi] + c;
        ++pi;
      }
    }
  }
  // ---- device: one pooled allocation; the arrays built here are uploaded
  // with one copy (they lead the arena, in this order)
  const size_t nn = m->near_idx.size();
  const int64_t nb = (nt + 31) / 32;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (std::max<size_t>(bytes, 1) + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_tvert = take(16 * nt), o_tedge = take(16 * nt), o_near_ptr = take(8 * (nt + 1)),
               o_near_idx = take(4 * nn), o_v64 = take(72 * nt), o_elen = take(8 * std::max<int64_t>(m->ne, 1));
  const size_t upload = off;
  const size_t o_near_row = take(4 * nn), o_pts32 = take(16 * kMaxRule * nt), o_cen32 = take(16 * nt), o_geo32 = take(48 * nt),
               o_pts64 = take(32 * kMaxRule * nt), o_cen64 = take(32 * nt), o_geo64 = take(96 * nt),
               o_frame64 = take(8 * kFrame * nt), o_frame32 = take(4 * kFrame32 * nt), o_minmax = take(64),
               o_rad32 = take(4 * nt), o_bsph = take(16 * nb), o_bpb = take(8 * (size_t)(nb * (nb + 1) / 2)),
               o_bgrid = take(16 * nb), o_rel32 = take(16 * kMaxRule * nt), o_geob32 = take(48 * nt),
               o_list = take(4 * range_list_ints(nt));
  size_t got = 0;
  unsigned char* base = static_cast<unsigned char*>(arena_take(m->device, off, &got));
  if (!base) {
    cudaError_t e = cudaMalloc((void**)&base, off);
    if (e != cudaSuccess) return cuda_fail(e, "gf_mesh_create: cudaMalloc");
    got = off;
  }
  m->d_arena = base;
  m->arena_bytes = got;
  m->d_tvert = reinterpret_cast<int4*>(base + o_tvert);
  m->d_tedge = reinterpret_cast<int4*>(base + o_tedge);
  m->d_near_ptr = reinterpret_cast<int64_t*>(base + o_near_ptr);
  m->d_near_idx = reinterpret_cast<int32_t*>(base + o_near_idx);
  m->d_near_row = reinterpret_cast<int32_t*>(base + o_near_row);
  m->d_v64 = reinterpret_cast<double*>(base + o_v64);
  m->d_elen = reinterpret_cast<double*>(base + o_elen);
  m->d_pts32 = reinterpret_cast<float4*>(base + o_pts32);
  m->d_cen32 = reinterpret_cast<float4*>(base + o_cen32);
  m->d_geo32 = reinterpret_cast<float4*>(base + o_geo32);
  m->d_pts64 = reinterpret_cast<double*>(base + o_pts64);
  m->d_cen64 = reinterpret_cast<double*>(base + o_cen64);
  m->d_geo64 = reinterpret_cast<double*>(base + o_geo64);
  m->d_frame64 = reinterpret_cast<double*>(base + o_frame64);
  m->d_frame32 = reinterpret_cast<float*>(base + o_frame32);
  m->d_minmax = reinterpret_cast<unsigned long long*>(base + o_minmax);
  m->d_rad32 = reinterpret_cast<float*>(base + o_rad32);
  m->d_bsph = reinterpret_cast<float4*>(base + o_bsph);
  m->d_bgrid = reinterpret_cast<int4*>(base + o_bgrid);
  m->d_rel32 = reinterpret_cast<float4*>(base + o_rel32);
  m->d_geob32 = reinterpret_cast<float4*>(base + o_geob32);
  m->d_range_bpb = reinterpret_cast<float2*>(base + o_bpb);
  m->d_range_list = reinterpret_cast<int32_t*>(base + o_list);
  std::unique_ptr<unsigned char[]> h(new (std::nothrow) unsigned char[upload]);
  if (!h) {
    free_mesh_device(m.get());
    return fail(GF_ERR_ALLOC, "gf_mesh_create: out of host memory");
  }
  int4* tv = reinterpret_cast<int4*>(&h[o_tvert]);
  int4* te = reinterpret_cast<int4*>(&h[o_tedge]);
  for (int64_t i = 0; i < nt; ++i) {
    const int64_t t = m->perm[i];
    tv[i] = make_int4(tri[3 * t], tri[3 * t + 1], tri[3 * t + 2], 0);
    te[i] = make_int4(m->tedge[3 * t], m->tedge[3 * t + 1], m->tedge[3 * t + 2], 0);
  }
  std::memcpy(&h[o_near_ptr], m->near_ptr.data(), (nt + 1) * 8);
  if (nn) std::memcpy(&h[o_near_idx], m->near_idx.data(), nn * 4);
  vertex_arrays(m.get(), &h[o_v64]);
  cudaError_t e = cudaMemcpy(base, h.get(), upload, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_near_rows(m->d_near_ptr, nt, m->d_near_row, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) {
    free_mesh_device(m.get());
    return cuda_fail(e, "gf_mesh_create upload");
  }
  m->rule = 0;
  *out = m.release();
  return GF_OK;
}

gf_status gf_mesh_info(const gf_mesh* m, int64_t* nv, int64_t* nt, int64_t* ne, int64_t* n_near) {
  if (!m) return fail(GF_ERR_ARG, "gf_mesh_info: null mesh");
  if (nv) *nv = m->nv;
  if (nt) *nt = m->nt;
  if (ne) *ne = m->ne;
  if (n_near) *n_near = (int64_t)m->near_idx.size();
  return GF_OK;
}

gf_status gf_mesh_edges(const gf_mesh* m, int32_t* edge_verts, int32_t* edge_tris) {
  if (!m) return fail(GF_ERR_ARG, "gf_mesh_edges: null mesh");
  if (edge_verts) std::memcpy(edge_verts, m->ev.data(), m->ev.size() * 4);
  if (edge_tris) std::memcpy(edge_tris, m->et.data(), m->et.size() * 4);
  return GF_OK;
}

gf_status gf_mesh_set_vertices(gf_mesh* m, const double* xyz) {
  if (!m || !xyz) return fail(GF_ERR_ARG, "gf_mesh_set_vertices: null argument");
  gf_status st = check_device(m->device);
  if (st) return st;
  for (int64_t i = 0; i < 3 * m->nv; ++i)
    if (!std::isfinite(xyz[i])) return fail(GF_ERR_MESH, "gf_mesh_set_vertices: non-finite coordinate");
  m->xyz.assign(xyz, xyz + 3 * m->nv);
  set_block_grid(m);
  return upload_vertices(m);
}

gf_status gf_mesh_destroy(gf_mesh* m) {
  if (!m) return GF_OK;
  free_mesh_device(m);
  delete m;
  return GF_OK;
}

gf_status gf_range(const gf_mesh* mc, int rule, int precision, double* r_min, double* r_max, void* stream) {
  if (!mc || !r_min || !r_max) return fail(GF_ERR_ARG, "gf_range: null argument");
  if (precision != GF_FP32 && precision != GF_FP64) return fail(GF_ERR_ARG, "gf_range: bad precision");
  gf_mesh* m = const_cast<gf_mesh*>(mc);
  gf_status st = check_device(m->device);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = prepare_rule_impl(m, rule, s))) return st;
  GF_CUDA(launch_range(geo_view_impl(m), precision, m->d_minmax, m->d_range_bpb, m->d_range_list, s));
  // the result through device-mapped page-locked memory, written by a kernel
  if (!m->h_range) GF_CUDA(cudaHostAlloc((void**)&m->h_range, 16, cudaHostAllocMapped));
  unsigned long long* h_dev = nullptr;
  GF_CUDA(cudaHostGetDevicePointer((void**)&h_dev, m->h_range, 0));
  GF_CUDA(launch_range_out(m->d_minmax, h_dev, s));
  GF_CUDA(cudaStreamSynchronize(s));
  unsigned long long mm[2];
  std::memcpy(mm, (const void*)m->h_range, 16);
  double lo, hi;
  std::memcpy(&lo, &mm[0], 8);
  std::memcpy(&hi, &mm[1], 8);
  if (!(hi >= 0) || !(lo < INFINITY)) return fail(GF_ERR_RANGE, "gf_range: every triangle pair is near");
  *r_min = lo;
  *r_max = hi;
  return GF_OK;
}

namespace {

// FP32 lattice image of a table (the device lookups repeat these float
// operations exactly): u = fma(x, inv, nc); v = clamp(u + kLatMagic); the
// cell i is the integer in v, and s = x - fma(i, h, lo) the offset from its
// left end (the sub-cells of a cell holding samples are counted from there).
struct LatPos {
  int i;
  float s;
};

int32_t float_bits(float f) {
  int32_t v;
  std::memcpy(&v, &f, 4);
  return v;
}

float bits_float(int32_t v) {
  float f;
  std::memcpy(&f, &v, 4);
  return f;
}

struct LatMap {
  float inv, nc, h, lo, amid;
};

LatPos lattice_pos(float x, const LatMap& M, float vmin, float vmax) {
  const float u = std::fmaf(x, M.inv, M.nc);
  float v = u + kLatMagic;
  v = std::fmin(std::fmax(v, vmin), vmax);
  const float fi = v - kLatMagic;
  return LatPos{float_bits(v) - float_bits(kLatMagic), x - std::fmaf(fi, M.h, M.lo)};
}

// sub-cell of an offset s inside a cell holding samples
int lattice_sub(float s, float inv_w, int nsub) {
  const float u = s * inv_w;
  const int c = (int)u;
  return c < 0 ? 0 : (c > nsub - 1 ? nsub - 1 : c);
}

struct Lattice {
  int n = 0;
  LatMap map{};
  float c2d = 0.f;            // 2^-E of the Green table's c2 halves
  std::vector<int32_t> j;     // interval containing the middle of each cell; bit 31: the cell holds samples
  std::vector<int32_t> busy;  // cells holding samples, ascending
  std::vector<float4> hdr;    // per busy cell: (first sub-cell, 1/w, count - 1, 0)
  std::vector<float4> sub;    // sub-cell records (compact interval j0, split, node32[j0], 0)
  std::vector<int32_t> cmp;   // interval of each compact interval record
  // the device blob: busy (int32, padded to 16 bytes), hdr, sub, then the
  // compact interval records (a, b), filled on the device from cmp
  size_t blob_vec4() const { return (busy.size() + 3) / 4 + busy.size() + sub.size() + 2 * cmp.size(); }
};

// Shared-memory budget of a lattice image for choosing the finer step.
constexpr int64_t kLatticeSmemBudget = 210 * 1024;

// Bound of |f^(n)| for f = e^{-jkr}/r at r (it decreases with r): the
// Leibniz sum sum_i C(n, i) k^(n-i) i! / r^(i+1).
// (powers by repeated products: it runs for every lattice cell)
double green_deriv_bound(int n, double k, double r) {
  double kp[16];
  kp[0] = 1.0;
  for (int i = 1; i <= n && i < 16; ++i) kp[i] = kp[i - 1] * k;
  const double ir = 1.0 / r;
  double s = 0.0, c = 1.0, fact = 1.0, irp = ir;  // irp = 1 / r^(i+1)
  for (int i = 0; i <= n && i < 16; ++i) {
    if (i > 0) {
      c = c * (n - i + 1) / i;
      fact *= i;
      irp *= ir;
    }
    s += c * kp[n - i] * fact * irp;
  }
  return s;
}

// Relative size (to |f| on the cell) below which the cubic term of the Green
// table's cell polynomial is left out of the lattice record.
constexpr double kDropC3 = 4e-8;
// Largest difference (relative to |f| on the cell) between the Green
// polynomials of the intervals a cell holding samples spans for which the
// cell keeps the plain record of the interval at its middle.
constexpr double kAgree = 1e-8;

// Cells of width `step` (t or t / 2) from r_min (the uniform samples of Eq. 2,
// and the refined ones for t / 2, sit on their ends). A cell is sample-free
// when every interior sample lies within a margin of its ends (FP32 rounding
// of the map and of the samples); R inside such a cell but past a sample at
// its end is evaluated with the neighbour interval's polynomial, an
// extrapolation by at most the margin. Cells holding samples get sub-cells
// narrower than the local spacing, so each holds one sample at most and the
// bracketing against the FP32 samples is exact.
gf_status build_lattice(const std::vector<double>& r, const std::vector<int8_t>& zflag, double step, double t,
                        int degree, double k, Lattice* L) {
  const size_t n = r.size();
  LatMap& M = L->map;
  M.lo = (float)r.front();
  M.h = (float)step;
  M.inv = (float)(1.0 / step);
  M.amid = degree > 1 ? (float)(r.front() + 0.5 * step) : M.lo;
  const float c = (float)((double)M.lo * (double)M.inv + 0.5);
  M.nc = -c;
  const float hi32 = (float)r.back();
  const double span = ((double)hi32 - (double)M.lo) * (double)M.inv;
  if (!(span < (double)(1 << 21))) return fail(GF_ERR_RANGE, "table: FP32 lattice too large");
  const float wide_lo = kLatMagic - (float)(1 << 21), wide_hi = kLatMagic + (float)(1 << 21);
  L->n = std::max(lattice_pos(hi32, M, wide_lo, wide_hi).i, 0) + 1;
  std::vector<float> x32(n);
  for (size_t j = 0; j < n; ++j) x32[j] = (float)r[j];
  std::vector<int> cell(n, 0);
  for (size_t j = 0; j < n; ++j) cell[j] = lattice_pos(x32[j], M, wide_lo, wide_hi).i;
  const double eps = 1e-3 + 8.0 * L->n / 16777216.0;  // margin in cells
  std::vector<char> busy(L->n, 0);
  for (size_t j = 1; j + 1 < n; ++j) {
    const double v = (double)x32[j] * (double)M.inv - (double)c;
    const double ci = std::floor(v + 0.5), d = v - ci;  // d in [-1/2, 1/2)
    const int64_t i = (int64_t)ci;
    if (std::fabs(d) < 0.5 - eps && i >= 0 && i < L->n) busy[i] = 1;
  }
  const double cell_w = 1.0 / (double)M.inv;
  if (degree > 1) {
    // A Green cell holding samples whose intervals' polynomials all agree
    // with that of the interval at its middle within kAgree |f| over the cell
    // (the refinement samples and forced zeros of Section II.B, at spacings
    // where the interpolant is far more accurate than FP32) keeps that one
    // record, as a sample-free cell does: its value then differs from the
    // piecewise interpolant by less than FP32 resolves.
    std::vector<double> f(2 * n);
    for (size_t j = 0; j < n; ++j) {
      const double re = std::cos(k * r[j]) / r[j], im = -std::sin(k * r[j]) / r[j];
      f[2 * j] = zflag[j] == 1 ? 0.0 : re;
      f[2 * j + 1] = zflag[j] == 2 ? 0.0 : im;
    }
    auto interval_at = [&](double x) {  // last sample <= x, as an interval index
      const size_t u = (size_t)(std::upper_bound(r.begin(), r.end(), x) - r.begin());
      return (int)std::min<size_t>(u == 0 ? 0 : u - 1, n - 2);
    };
    for (int i = 0; i < L->n; ++i) {
      if (!busy[i]) continue;
      const double mid = ((double)i + (double)c) * cell_w;
      const double a = mid - 0.5005 * cell_w, b = mid + 0.5005 * cell_w;
      const int jm = interval_at(mid), j0 = interval_at(a), j1 = interval_at(b);
      double pm[2][4], pj[2][4], worst = 0.0;
      interval_poly(degree, (int)n, r.data(), f.data(), jm, mid, pm[0], pm[1]);
      for (int j = j0; j <= j1; ++j) {
        if (j == jm) continue;
        interval_poly(degree, (int)n, r.data(), f.data(), j, mid, pj[0], pj[1]);
        const double xa = std::max(a, j == 0 ? a : r[j]), xb = std::min(b, j == (int)n - 2 ? b : r[j + 1]);
        for (int q = 0; q <= 32 && xb > xa; ++q) {
          const double u = xa + (xb - xa) * q / 32.0 - mid;
          double dre = 0.0, dim = 0.0;
          for (int e = 3; e >= 0; --e) {
            dre = dre * u + (pj[0][e] - pm[0][e]);
            dim = dim * u + (pj[1][e] - pm[1][e]);
          }
          worst = std::max(worst, std::hypot(dre, dim));
        }
      }
      if (worst <= kAgree / b) busy[i] = 0;
    }
  }
  L->c2d = 0.f;
  if (degree > 1) {
    // Green table records hold c0, c1 and c2 (a half2 scaled by 2^E). A cell
    // is treated as one holding samples where the left-out cubic term could
    // exceed kDropC3 |f| (|c3| <= max |f'''| / 3! over the stencil, which
    // starts at most one spacing t below the cell), or where c2 falls out of
    // the half range: |c2| <= max |f''| / 2 + 3 |c3| 1.5 t (the expansion
    // point lies within 1.5 t of the stencil's middle) and |c2| >= 0.9 k / r^2
    // (|f''| >= 2 k / r^2).
    const double hh = 0.51 * step, r0 = r.front();
    double c2max = 0.0;
    std::vector<double> lo_c2(L->n, 0.0);
    for (int i = 0; i < L->n; ++i) {
      const double rl = r0 + i * step, rh = rl + step, rs = std::max(rl - 1.01 * t, r0);
      const double c3 = green_deriv_bound(3, k, rs) / 6.0;
      if (c3 * hh * hh * hh > kDropC3 / rh) busy[i] = 1;
      if (busy[i]) continue;
      c2max = std::max(c2max, green_deriv_bound(2, k, rs) / 2.0 + 4.5 * t * c3);
      lo_c2[i] = 0.9 * k / (rh * rh);
    }
    int E = c2max > 0.0 ? (int)std::floor(std::log2(32768.0 / c2max)) : 0;
    E = std::min(std::max(E, -120), 120);
    L->c2d = (float)std::ldexp(1.0, -E);
    for (int i = 0; i < L->n; ++i)
      if (!busy[i] && std::ldexp(lo_c2[i], E) < std::ldexp(1.0, -13)) busy[i] = 1;
  }
  L->j.assign(L->n, 0);
  L->busy.clear();
  L->hdr.clear();
  L->sub.clear();
  L->cmp.clear();
  size_t jm = 0;  // last sample <= the cell's middle (the middles increase with i)
  for (int i = 0; i < L->n; ++i) {
    const double mid = ((double)i + (double)c) * cell_w;
    while (jm + 1 < n && r[jm + 1] <= mid) ++jm;
    L->j[i] = (int32_t)std::min<size_t>(jm, n - 2);
    if (!busy[i]) continue;
    // interior samples whose FP32 cell is i: [ja, jb)
    size_t ja = 1;
    {
      size_t lo = 1, hi = n - 1;
      while (lo < hi) {
        const size_t mid = (lo + hi) / 2;
        if (cell[mid] >= i) hi = mid;
        else lo = mid + 1;
      }
      ja = lo;
    }
    size_t jb = ja;
    while (jb < n - 1 && cell[jb] == i) ++jb;
    const float vmin = kLatMagic + (float)i, vmax = vmin;
    double w = step;
    for (size_t jj = (ja > 0 ? ja - 1 : 0); jj <= jb && jj + 1 < n; ++jj) w = std::min(w, r[jj + 1] - r[jj]);
    w *= 0.9;
    int nsub = 0;
    float inv_w = 0.f;
    bool ok = false;
    auto sub_of = [&](size_t jj) { return lattice_sub(lattice_pos(x32[jj], M, vmin, vmax).s, inv_w, nsub); };
    for (int attempt = 0; attempt < 30 && !ok; ++attempt, w *= 0.5) {
      inv_w = (float)(1.0 / w);
      nsub = (int)(1.1 * step / w) + 2;
      if (nsub > 65536) break;
      ok = true;
      for (size_t jj = ja; jj + 1 < jb; ++jj)
        if (sub_of(jj) >= sub_of(jj + 1)) ok = false;
    }
    if (!ok) return fail(GF_ERR_RANGE, "table: samples closer than the FP32 resolution");
    // intervals this cell can reach: ja - 1 .. jb - 1, stored as a compact run
    const int first = (int)L->sub.size();
    const int cbase = (int)L->cmp.size() - ((int)ja - 1);
    for (size_t jv = ja - 1; jv < jb; ++jv) L->cmp.push_back((int32_t)jv);
    size_t jj = ja;
    for (int cc = 0; cc < nsub; ++cc) {
      while (jj < jb && sub_of(jj) < cc) ++jj;
      const int j0 = (int)jj - 1;  // interval below every sample of sub-cell cc and later
      const bool has = jj < jb && sub_of(jj) == cc;
      L->sub.push_back(make_float4(bits_float(cbase + j0), has ? x32[jj] : INFINITY, x32[j0], 0.f));
    }
    L->j[i] |= (int32_t)0x80000000u;
    L->busy.push_back(i);
    L->hdr.push_back(make_float4(bits_float(first), inv_w, bits_float(nsub - 1), 0.f));
  }
  return GF_OK;
}

}  // namespace

gf_status gf_table_create(double k, double r_min, double r_max, const gf_params* p, void* stream, gf_table** out) {
  if (!out || !params_ok(p)) return fail(GF_ERR_ARG, "gf_table_create: bad params");
  if (!(k > 0) || !(r_min > 0) || !(r_max > r_min) || !std::isfinite(r_max))
    return fail(GF_ERR_ARG, "gf_table_create: need k > 0 and 0 < r_min < r_max");
  std::unique_ptr<gf_table> T(new (std::nothrow) gf_table);
  if (!T) return fail(GF_ERR_ALLOC, "gf_table_create: out of host memory");
  GF_CUDA(cudaGetDevice(&T->device));
  T->k = k;
  T->r_lo = r_min;
  T->r_hi = r_max;
  const double lam = 2.0 * kPi / k;
  int n_exp = p->exp_n_per_lambda;
  if (n_exp == 0) {
    n_exp = 1000;
    while (n_exp < 10000 && std::pow(2.0 * kPi / n_exp, 2) / 8.0 > p->table_tol) n_exp += 4;
  }
  const int n_green = p->green_n_per_lambda ? p->green_n_per_lambda : 1000;
  cudaStream_t s = (cudaStream_t)stream;
  gf_table::One* ones[2] = {&T->green, &T->exp};
  Lattice lat[2];
  // ---- host: samples (Section II.B) and the FP32 lattice image of both tables
  for (int which = 0; which < 2; ++which) {
    gf_table::One& o = *ones[which];
    o.kind = which == 0 ? GF_GREEN : GF_EXP;
    o.degree = which == 0 ? p->lagrange_degree : 1;
    const double t = lam / (which == 0 ? n_green : n_exp);
    Placement pl;
    gf_status st = place_samples(o.kind, o.degree, k, r_min, r_max, t, *p, &pl);
    if (st) return st;
    o.r = std::move(pl.r);
    o.zflag = std::move(pl.zflag);
    o.dr = pl.dr;
    o.n_hash = pl.n_hash;
    // lattice step: t / 2 (the refined spacing, so refinement windows hold no
    // sample inside a cell) when that image fits the shared-memory budget,
    // else t
    const double rec = o.degree > 1 ? 20.0 : 16.0;
    const double h = p->refine && (r_max - r_min) / (0.5 * t) * rec <= (double)kLatticeSmemBudget &&
                             std::fabs(p->refine_factor - 0.5) < 1e-12
                         ? 0.5 * t
                         : t;
    if ((st = build_lattice(o.r, o.zflag, h, t, o.degree, k, &lat[which]))) return st;
    o.n_lat = lat[which].n;
    o.n_busy = (int)lat[which].busy.size();
    o.n_sub = (int)lat[which].sub.size();
    o.n_cmp = (int)lat[which].cmp.size();
    o.lat_inv = lat[which].map.inv;
    o.lat_nc = lat[which].map.nc;
    o.lat_h = lat[which].map.h;
    o.lat_lo = lat[which].map.lo;
    o.lat_amid = lat[which].map.amid;
    o.lat_c2d = lat[which].c2d;
    o.lo64c = r_min;
    o.inv64c = 1.0 / (0.99 * o.dr);
    o.n_cells64 = (int)std::floor((r_max - r_min) * o.inv64c) + 1;
    // the FP64 cell image holds one interior sample per cell at most (the
    // device cell map, repeated here: no contraction in this file)
    for (size_t j = 1; j + 2 < o.r.size(); ++j)
      if ((int)((o.r[j] - o.lo64c) * o.inv64c) == (int)((o.r[j + 1] - o.lo64c) * o.inv64c))
        return fail(GF_ERR_RANGE, "table: two samples in one FP64 hash cell");
  }
  // ---- one device allocation: the uploaded arrays of both tables first (one
  // host-to-device copy), then the arrays the kernels compute
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (std::max<size_t>(bytes, 1) + 255) & ~(size_t)255;
    return o;
  };
  size_t o_node64[2], o_zflag[2], o_lat_j[2], o_lat_cmp[2], o_lat_blob[2];
  for (int w = 0; w < 2; ++w) {
    const gf_table::One& o = *ones[w];
    o_node64[w] = take(o.r.size() * 8);
    o_zflag[w] = take(o.r.size());
    o_lat_j[w] = take((size_t)o.n_lat * 4);
    o_lat_cmp[w] = take((size_t)o.n_cmp * 4);
    o_lat_blob[w] = take(lat[w].blob_vec4() * 16);
  }
  const size_t upload = off;
  size_t o_fval[2], o_c64[2], o_node32[2], o_c32a[2], o_c32b[2], o_hash[2], o_lat_a[2], o_lat_c[2], o_cells64[2];
  for (int w = 0; w < 2; ++w) {
    const gf_table::One& o = *ones[w];
    const size_t n = o.r.size();
    o_fval[w] = take(2 * n * 8);
    o_c64[w] = take(4 * n * sizeof(double2));
    o_node32[w] = take(n * 4);
    o_c32a[w] = take(n * 16);
    o_c32b[w] = take(n * 16);
    o_hash[w] = take((size_t)o.n_hash * 4);
    o_lat_a[w] = take((size_t)o.n_lat * 16);
    o_lat_c[w] = take((size_t)o.n_lat * 4);
    o_cells64[w] = take((size_t)o.n_cells64 * sizeof(Cell64));
  }
  std::vector<unsigned char> hbuf(upload, 0);
  for (int w = 0; w < 2; ++w) {
    const gf_table::One& o = *ones[w];
    std::memcpy(&hbuf[o_node64[w]], o.r.data(), o.r.size() * 8);
    std::memcpy(&hbuf[o_zflag[w]], o.zflag.data(), o.r.size());
    std::memcpy(&hbuf[o_lat_j[w]], lat[w].j.data(), (size_t)o.n_lat * 4);
    std::memcpy(&hbuf[o_lat_cmp[w]], lat[w].cmp.data(), (size_t)o.n_cmp * 4);
    unsigned char* blob = &hbuf[o_lat_blob[w]];
    std::memcpy(blob, lat[w].busy.data(), (size_t)o.n_busy * 4);
    blob += ((size_t)o.n_busy + 3) / 4 * 16;
    std::memcpy(blob, lat[w].hdr.data(), (size_t)o.n_busy * 16);
    blob += (size_t)o.n_busy * 16;
    std::memcpy(blob, lat[w].sub.data(), (size_t)o.n_sub * 16);  // compact records follow, filled on the device
  }
  size_t got = 0;
  unsigned char* base = static_cast<unsigned char*>(arena_take(T->device, off, &got));
  cudaError_t e = cudaSuccess;
  if (!base) {
    e = cudaMalloc((void**)&base, off);
    if (e != cudaSuccess) return cuda_fail(e, "gf_table_create: cudaMalloc");
    got = off;
  }
  T->d_arena = base;
  T->arena_bytes = got;
  for (int w = 0; w < 2; ++w) {
    gf_table::One& o = *ones[w];
    o.d_node64 = reinterpret_cast<double*>(base + o_node64[w]);
    o.d_zflag = reinterpret_cast<int8_t*>(base + o_zflag[w]);
    o.d_lat_j = reinterpret_cast<int32_t*>(base + o_lat_j[w]);
    o.d_lat_cmp = reinterpret_cast<int32_t*>(base + o_lat_cmp[w]);
    o.d_lat_blob = reinterpret_cast<float4*>(base + o_lat_blob[w]);
    o.d_lat_a = reinterpret_cast<float4*>(base + o_lat_a[w]);
    o.d_fval = reinterpret_cast<double*>(base + o_fval[w]);
    o.d_c64 = reinterpret_cast<double2*>(base + o_c64[w]);
    o.d_node32 = reinterpret_cast<float*>(base + o_node32[w]);
    o.d_c32a = reinterpret_cast<float4*>(base + o_c32a[w]);
    o.d_c32b = reinterpret_cast<float4*>(base + o_c32b[w]);
    o.d_hash = reinterpret_cast<int32_t*>(base + o_hash[w]);
    o.d_lat_c = reinterpret_cast<uint32_t*>(base + o_lat_c[w]);
    o.d_cells64 = reinterpret_cast<Cell64*>(base + o_cells64[w]);
  }
  // ---- device: values, coefficients, hash and images of both tables
  e = cudaMemcpyAsync(base, hbuf.data(), upload, cudaMemcpyHostToDevice, s);
  TableBuild tb[2];
  for (int w = 0; w < 2; ++w) {
    const gf_table::One& o = *ones[w];
    TableBuild& b = tb[w];
    b.kind = o.kind;
    b.deg = o.degree;
    b.n = (int)o.r.size();
    b.n_hash = (int)o.n_hash;
    b.n_cells64 = o.n_cells64;
    b.r_lo = r_min;
    b.dr = o.dr;
    b.lo64c = o.lo64c;
    b.inv64c = o.inv64c;
    b.node64 = o.d_node64;
    b.zflag = o.d_zflag;
    b.fval = o.d_fval;
    b.c64 = o.d_c64;
    b.node32 = o.d_node32;
    b.c32a = o.d_c32a;
    b.c32b = o.d_c32b;
    b.hash = o.d_hash;
    b.cells64 = o.d_cells64;
    b.view = o.view();
    b.lat_j = o.d_lat_j;
    b.cmp = o.d_lat_cmp;
    b.lat_a = o.d_lat_a;
    b.lat_c = o.d_lat_c;
  }
  if (e == cudaSuccess) e = launch_tables(tb[0], tb[1], k, s);
  if (e != cudaSuccess) {
    gf_table_destroy(T.release());
    return cuda_fail(e, "gf_table_create");
  }
  *out = T.release();
  return GF_OK;
}

gf_status gf_table_create_kr(double u_min, double u_max, const gf_params* p, void* stream, gf_table** out) {
  gf_status st = gf_table_create(1.0, u_min, u_max, p, stream, out);
  if (st) return st;
  (*out)->kr = true;
  return GF_OK;
}

gf_status gf_table_info(const gf_table* t, int kind, int64_t* n_nodes, int64_t* n_hash, double* dr) {
  if (!t || (kind != GF_GREEN && kind != GF_EXP)) return fail(GF_ERR_ARG, "gf_table_info: bad argument");
  const gf_table::One& o = t->get(kind);
  if (n_nodes) *n_nodes = (int64_t)o.r.size();
  if (n_hash) *n_hash = o.n_hash;
  if (dr) *dr = o.dr;
  return GF_OK;
}

gf_status gf_table_nodes(const gf_table* t, int kind, double* r, double* fre, double* fim, int32_t* hash) {
  if (!t || (kind != GF_GREEN && kind != GF_EXP)) return fail(GF_ERR_ARG, "gf_table_nodes: bad argument");
  gf_status st = check_device(t->device);
  if (st) return st;
  const gf_table::One& o = t->get(kind);
  const size_t n = o.r.size();
  GF_CUDA(cudaDeviceSynchronize());  // the table's kernels may still run on the creation stream
  if (r) std::memcpy(r, o.r.data(), n * 8);
  if (fre || fim) {
    std::vector<double> f(2 * n);
    GF_CUDA(cudaMemcpy(f.data(), o.d_fval, 2 * n * 8, cudaMemcpyDeviceToHost));
    for (size_t j = 0; j < n; ++j) {
      if (fre) fre[j] = f[2 * j];
      if (fim) fim[j] = f[2 * j + 1];
    }
  }
  if (hash) GF_CUDA(cudaMemcpy(hash, o.d_hash, (size_t)o.n_hash * 4, cudaMemcpyDeviceToHost));
  return GF_OK;
}

gf_status gf_table_eval(const gf_table* t, int kind, int precision, const void* r_dev, int64_t n, void* out_dev,
                        void* stream) {
  if (!t || (kind != GF_GREEN && kind != GF_EXP) || (precision != GF_FP32 && precision != GF_FP64) || n < 0 ||
      (n > 0 && (!r_dev || !out_dev)))
    return fail(GF_ERR_ARG, "gf_table_eval: bad argument");
  gf_status st = check_device(t->device);
  if (st) return st;
  if (n == 0) return GF_OK;
  GF_CUDA(launch_table_eval(t->get(kind).view(), kind, precision, r_dev, n, out_dev, (cudaStream_t)stream));
  return GF_OK;
}

gf_status gf_table_eval_host(const gf_table* t, int kind, const double* x, int64_t n, double* out) {
  if (!t || (kind != GF_GREEN && kind != GF_EXP) || n < 0 || (n > 0 && (!x || !out)))
    return fail(GF_ERR_ARG, "gf_table_eval_host: bad argument");
  if (n == 0) return GF_OK;
  gf_status st = check_device(t->device);
  if (st) return st;
  const gf_table::One& o = t->get(kind);
  const size_t nn = o.r.size();
  for (int64_t i = 0; i < n; ++i)
    if (!(x[i] >= o.r.front() && x[i] <= o.r.back()))
      return fail(GF_ERR_RANGE, "gf_table_eval_host: x outside the table's range");
  // the FP64 interval polynomials and cell records of the device image
  std::vector<double2> c64(4 * nn);
  std::vector<Cell64> cells((size_t)o.n_cells64);
  GF_CUDA(cudaDeviceSynchronize());  // the table's kernels may still run on the creation stream
  GF_CUDA(cudaMemcpy(c64.data(), o.d_c64, c64.size() * sizeof(double2), cudaMemcpyDeviceToHost));
  GF_CUDA(cudaMemcpy(cells.data(), o.d_cells64, cells.size() * sizeof(Cell64), cudaMemcpyDeviceToHost));
  const int deg = o.degree > 1 ? 3 : 1;
  for (int64_t i = 0; i < n; ++i) {
    // the FP64 cell of x brackets it exactly (one sample per cell at most)
    int c = (int)((x[i] - o.lo64c) * o.inv64c);
    c = std::min(std::max(c, 0), o.n_cells64 - 1);
    const Cell64& rec = cells[c];
    const bool up = x[i] >= rec.split;
    const int j = rec.j0 + (up ? 1 : 0);
    const double s = x[i] - (up ? rec.split : rec.anchor);
    const double2* cf = &c64[4 * (size_t)j];
    double re = cf[deg].x, im = cf[deg].y;
    for (int q = deg - 1; q >= 0; --q) {
      re = std::fma(s, re, cf[q].x);
      im = std::fma(s, im, cf[q].y);
    }
    out[2 * i] = re;
    out[2 * i + 1] = im;
  }
  return GF_OK;
}

gf_status gf_table_create_for_mesh(const gf_mesh* m, double k, const gf_params* p, int precision, double r_min,
                                   double r_max, void* stream, gf_table** out) {
  if (!m || !p || !out) return fail(GF_ERR_ARG, "gf_table_create_for_mesh: bad argument");
  if (r_min < 0 || r_max < 0) {
    double lo = 0, hi = 0;
    gf_status st = gf_range(m, p->rule, precision, &lo, &hi, stream);
    if (st) return st;
    if (r_min < 0) r_min = lo;
    if (r_max < 0) r_max = hi;
  }
  return gf_table_create(k, r_min, r_max, p, stream, out);
}

gf_status gf_table_destroy(gf_table* t) {
  if (!t) return GF_OK;
  if (t->d_arena) {
    // like cudaFree, wait for work that may still read the table; then keep
    // the memory for the next table
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != t->device) cudaSetDevice(t->device);
    cudaDeviceSynchronize();
    arena_give(t->device, t->d_arena, t->arena_bytes);
    if (cur >= 0 && cur != t->device) cudaSetDevice(cur);
  }
  delete t;
  return GF_OK;
}

gf_status gf_fill(const gf_mesh* mc, double k, const gf_params* p, const gf_table* table, int precision, void* Z,
                  int64_t ldz, void* stream) {
  return gf_fill_parts(mc, k, p, table, precision, Z, ldz, GF_PART_ZERO | GF_PART_REGULAR | GF_PART_NEAR, stream);
}

gf_status gf_fill_parts(const gf_mesh* mc, double k, const gf_params* p, const gf_table* table, int precision,
                        void* Z, int64_t ldz, unsigned parts, void* stream) {
  if (!mc || !params_ok(p) || !Z) return fail(GF_ERR_ARG, "gf_fill: bad argument");
  if (parts == 0 || (parts & ~(GF_PART_ZERO | GF_PART_REGULAR | GF_PART_NEAR | GF_PART_PAIRS | GF_PART_MIRROR)))
    return fail(GF_ERR_ARG, "gf_fill_parts: bad parts mask");
  if (parts & GF_PART_REGULAR) parts |= GF_PART_PAIRS | GF_PART_MIRROR;
  if (precision != GF_FP32 && precision != GF_FP64) return fail(GF_ERR_ARG, "gf_fill: bad precision");
  if (!(k > 0) || ldz < mc->ne) return fail(GF_ERR_ARG, "gf_fill: need k > 0 and ldz >= ne");
  gf_mesh* m = const_cast<gf_mesh*>(mc);
  gf_status st = check_device(m->device);
  if (st) return st;
  if (table && (table->device != m->device)) return fail(GF_ERR_DEVICE, "gf_fill: table on another device");
  TabView tg, te;
  double gscale = 1.0;
  if (table && !table_views(table, k, &tg, &te, &gscale)) return fail(GF_ERR_ARG, "gf_fill: table built for another k");
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = prepare_rule_impl(m, p->rule, s))) return st;
  if (m->ne == 0) return GF_OK;
  const size_t esz = precision == GF_FP32 ? 8 : 16;
  if (parts & GF_PART_ZERO)
    GF_CUDA(cudaMemset2DAsync(Z, (size_t)ldz * esz, 0, (size_t)m->ne * esz, (size_t)m->ne, s));
  GeoView g = geo_view_impl(m);
  if ((parts & GF_PART_PAIRS) && table && precision == GF_FP32 && !p->green_from_exp) {
    // list of the point pairs in Green lattice cells holding samples (grown
    // on demand); GF_FIX_ENTRIES replaces its size (0: no list, the
    // corrections in the pair kernel's loop; small: lists overflow and their
    // CTAs scan their tasks again)
    int64_t need = fix_entries(m->nt, p->rule, tg.n_busy, tg.n_lat);
    if (const char* ev = std::getenv("GF_FIX_ENTRIES")) need = std::max<int64_t>(0, std::atoll(ev));
    if (m->fix_cap < need) {  // from the library's device pool (no allocation once warm)
      if (m->d_fix) {
        GF_CUDA(cudaDeviceSynchronize());
        arena_give(m->device, m->d_fix, m->fix_bytes);
      }
      m->d_fix = nullptr;
      m->fix_cap = 0;
      m->fix_bytes = 0;
      size_t got = 0;
      void* ptr = arena_take(m->device, (size_t)need * sizeof(int2), &got);
      if (!ptr) {
        got = (size_t)need * sizeof(int2);
        if (cudaMalloc(&ptr, got) != cudaSuccess) {
          (void)cudaGetLastError();
          ptr = nullptr;
          got = 0;
        }
      }
      m->d_fix = static_cast<int2*>(ptr);
      m->fix_bytes = got;
      m->fix_cap = (int64_t)(got / sizeof(int2));
    }
    g.fix = need > 0 ? m->d_fix : nullptr;
    g.fix_cap = std::min(m->fix_cap, need);
  }
  if (parts & GF_PART_PAIRS)
    GF_CUDA(launch_fill_regular(g, table ? (p->green_from_exp ? &te : &tg) : nullptr, p->green_from_exp != 0, gscale,
                                precision, k, p->eta, Z, ldz, s));
  if ((parts & GF_PART_MIRROR) && precision == GF_FP32) GF_CUDA(launch_mirror32(Z, ldz, m->ne, s));
  if (!(parts & GF_PART_NEAR)) return GF_OK;
  double gx_phi[32], gw_phi[32], gx_l[32], gw_l[32];
  gauss_legendre(p->nphi, gx_phi, gw_phi);
  gauss_legendre(p->nl, gx_l, gw_l);
  double glp[64], gll[64];
  for (int i = 0; i < p->nphi; ++i) {
    glp[i] = gx_phi[i];
    glp[32 + i] = gw_phi[i];
  }
  for (int i = 0; i < p->nl; ++i) {
    gll[i] = gx_l[i];
    gll[32 + i] = gw_l[i];
  }
  GF_CUDA(launch_fill_near(g, table ? &te : nullptr, precision, precision == GF_FP32 && !p->near_fp64, k, p->eta,
                           p->nphi, p->nl, glp, gll, Z, ldz, s));
  return GF_OK;
}

gf_status gf_fill_mfie(const gf_mesh* mc, double k, const gf_params* p, const gf_table* table, int precision, void* Z,
                       int64_t ldz, void* stream) {
  if (!mc || !params_ok(p) || !Z) return fail(GF_ERR_ARG, "gf_fill_mfie: bad argument");
  if (precision != GF_FP32 && precision != GF_FP64) return fail(GF_ERR_ARG, "gf_fill_mfie: bad precision");
  if (!(k > 0) || ldz < mc->ne) return fail(GF_ERR_ARG, "gf_fill_mfie: need k > 0 and ldz >= ne");
  gf_mesh* m = const_cast<gf_mesh*>(mc);
  gf_status st = check_device(m->device);
  if (st) return st;
  if (table && (table->device != m->device)) return fail(GF_ERR_DEVICE, "gf_fill_mfie: table on another device");
  TabView tg, te;
  double gscale = 1.0;
  if (table && !table_views(table, k, &tg, &te, &gscale))
    return fail(GF_ERR_ARG, "gf_fill_mfie: table built for another k");
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = prepare_rule_impl(m, p->rule, s))) return st;
  if (m->ne == 0) return GF_OK;
  const size_t esz = precision == GF_FP32 ? 8 : 16;
  GF_CUDA(cudaMemset2DAsync(Z, (size_t)ldz * esz, 0, (size_t)m->ne * esz, (size_t)m->ne, s));
  GeoView g = geo_view_impl(m);
  double gx_phi[32], gw_phi[32], gx_l[32], gw_l[32];
  gauss_legendre(p->nphi, gx_phi, gw_phi);
  gauss_legendre(p->nl, gx_l, gw_l);
  double glp[64], gll[64];
  for (int i = 0; i < p->nphi; ++i) {
    glp[i] = gx_phi[i];
    glp[32 + i] = gw_phi[i];
  }
  for (int i = 0; i < p->nl; ++i) {
    gll[i] = gx_l[i];
    gll[32 + i] = gw_l[i];
  }
  GF_CUDA(launch_fill_mfie(g, table ? &tg : nullptr, table ? &te : nullptr, gscale, precision,
                           precision == GF_FP32 && !p->near_fp64, k, p->nphi, p->nl, glp, gll, Z, ldz, s));
  return GF_OK;
}

gf_status gf_fill_backward(const gf_mesh* mc, double k, const gf_params* p, const gf_table* table, int precision,
                           const void* gZ, int64_t ldg, double* dxyz, double* dk, void* stream) {
  if (!mc || !params_ok(p) || !gZ || !dxyz || !dk) return fail(GF_ERR_ARG, "gf_fill_backward: bad argument");
  if (precision != GF_FP32) return fail(GF_ERR_ARG, "gf_fill_backward: GF_FP32 only");
  if (p->green_from_exp) return fail(GF_ERR_ARG, "gf_fill_backward: green_from_exp must be 0");
  if (!(k > 0) || ldg < mc->ne) return fail(GF_ERR_ARG, "gf_fill_backward: need k > 0 and ldg >= ne");
  gf_mesh* m = const_cast<gf_mesh*>(mc);
  gf_status st = check_device(m->device);
  if (st) return st;
  if (table && (table->device != m->device || table->kr || table->k != k))
    return fail(GF_ERR_ARG, "gf_fill_backward: table on another device, for another k or in kR");
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = prepare_rule_impl(m, p->rule, s))) return st;
  if (!m->d_dtri && ((st = dev_alloc(&m->d_dtri, 9 * (size_t)m->nt)) || (st = dev_alloc(&m->d_dk, 1)))) return st;
  double bary[kMaxRule][3], w[kMaxRule];
  rule_points(p->rule, bary, w);
  double gx[32], gw[32], glp[64] = {0}, gll[64] = {0};
  gauss_legendre(p->nphi, gx, gw);
  for (int i = 0; i < p->nphi; ++i) {
    glp[i] = gx[i];
    glp[32 + i] = gw[i];
  }
  gauss_legendre(p->nl, gx, gw);
  for (int i = 0; i < p->nl; ++i) {
    gll[i] = gx[i];
    gll[32 + i] = gw[i];
  }
  TabView tg, te;
  if (table) {
    tg = table->green.view();
    te = table->exp.view();
  }
  GF_CUDA(launch_adjoint(geo_view_impl(m), table ? &tg : nullptr, table ? &te : nullptr, !p->near_fp64, k, p->eta,
                         &bary[0][0],
                         p->nphi, p->nl, glp, gll, gZ, ldg, m->d_dtri, m->d_dk, dxyz, m->nv, s));
  GF_CUDA(cudaMemcpyAsync(dk, m->d_dk, sizeof(double), cudaMemcpyDeviceToDevice, s));
  return GF_OK;
}

}  // extern "C"
