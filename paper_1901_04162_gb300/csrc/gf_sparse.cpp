// gfmom near-field sparse fill: Z restricted to the RWG pairs whose triangles
// come within a radius of each other (the near field a fast solver keeps; the
// paper's "3mnNC" count, Section II.A), stored as CSR. Host side: the pattern,
// the work list of triangle pairs, the C-ABI entry points.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <unordered_map>
#include <vector>

#include "gf_internal.h"

struct gf_sparse {
  const gf_mesh* mesh = nullptr;
  int device = -1;
  double radius = 0.0, work_radius = 0.0;
  std::vector<int64_t> row_ptr;  // [ne + 1]
  std::vector<int32_t> cols;     // sorted per row
  int64_t n_pairs = 0;           // regular triangle pairs in the work list
  int64_t ntask = 0;
  void* d_arena = nullptr;
  int64_t* d_row_ptr = nullptr;
  int32_t* d_cols = nullptr;
  void* d_tasks = nullptr;
  int32_t* d_widx = nullptr;
};

namespace {

using gf::fail;

// Triangles (indices into cen) whose centroid is within r of centroid i, by a
// uniform grid of cell r; calls f(j) for each (i itself included).
struct Grid {
  double cell;
  std::unordered_map<int64_t, std::vector<int32_t>> cells;
  static int64_t key(int64_t a, int64_t b, int64_t c) {
    return ((a & 0x1FFFFF) << 42) | ((b & 0x1FFFFF) << 21) | (c & 0x1FFFFF);
  }
  Grid(const std::vector<double>& cen, double r) : cell(r) {
    const int64_t n = (int64_t)cen.size() / 3;
    for (int64_t t = 0; t < n; ++t)
      cells[key((int64_t)std::floor(cen[3 * t] / cell), (int64_t)std::floor(cen[3 * t + 1] / cell),
                (int64_t)std::floor(cen[3 * t + 2] / cell))]
          .push_back((int32_t)t);
  }
  template <class F>
  void near(const std::vector<double>& cen, int64_t i, double r, F&& f) const {
    const int64_t gx = (int64_t)std::floor(cen[3 * i] / cell), gy = (int64_t)std::floor(cen[3 * i + 1] / cell),
                  gz = (int64_t)std::floor(cen[3 * i + 2] / cell);
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          auto it = cells.find(key(gx + dx, gy + dy, gz + dz));
          if (it == cells.end()) continue;
          for (int32_t j : it->second) {
            const double ax = cen[3 * i] - cen[3 * (size_t)j], ay = cen[3 * i + 1] - cen[3 * (size_t)j + 1],
                         az = cen[3 * i + 2] - cen[3 * (size_t)j + 2];
            if (std::sqrt(ax * ax + ay * ay + az * az) < r) f(j);
          }
        }
  }
};

}  // namespace

extern "C" {

gf_status gf_sparse_create(const gf_mesh* m, double radius, gf_sparse** out) {
  if (!m || !out) return fail(GF_ERR_ARG, "gf_sparse_create: null argument");
  if (!(radius > 0) || !std::isfinite(radius)) return fail(GF_ERR_ARG, "gf_sparse_create: need radius > 0");
  std::unique_ptr<gf_sparse> S(new (std::nothrow) gf_sparse);
  if (!S) return fail(GF_ERR_ALLOC, "gf_sparse_create: out of host memory");
  int cur = -1;
  GF_CUDA(cudaGetDevice(&cur));
  if (cur != m->device) return fail(GF_ERR_DEVICE, "gf_sparse_create: mesh on another device");
  S->mesh = m;
  S->device = m->device;
  S->radius = radius;
  const int64_t nt = m->nt, ne = m->ne;
  // centroids in the caller's triangle order
  std::vector<double> cen(3 * nt);
  for (int64_t t = 0; t < nt; ++t)
    for (int x = 0; x < 3; ++x)
      cen[3 * t + x] = (m->xyz[3 * (size_t)m->tri[3 * t] + x] + m->xyz[3 * (size_t)m->tri[3 * t + 1] + x] +
                        m->xyz[3 * (size_t)m->tri[3 * t + 2] + x]) / 3.0;
  // ---- pattern: (m, n) with some triangle of m and some triangle of n closer than radius
  std::vector<std::vector<int32_t>> tri_nbr(nt);
  {
    const Grid grid(cen, radius);
    for (int64_t t = 0; t < nt; ++t) grid.near(cen, t, radius, [&](int32_t j) { tri_nbr[t].push_back(j); });
  }
  S->row_ptr.assign(ne + 1, 0);
  std::vector<int32_t> stamp(ne, -1), row;
  for (int64_t e = 0; e < ne; ++e) {
    row.clear();
    for (int s = 0; s < 2; ++s)
      for (int32_t t2 : tri_nbr[m->et[2 * e + s]])
        for (int c = 0; c < 3; ++c) {
          const int32_t code = m->tedge[3 * (size_t)t2 + c];
          if (code < 0) continue;
          const int32_t n = code >> 1;
          if (stamp[n] == (int32_t)e) continue;
          stamp[n] = (int32_t)e;
          row.push_back(n);
        }
    std::sort(row.begin(), row.end());
    S->cols.insert(S->cols.end(), row.begin(), row.end());
    S->row_ptr[e + 1] = (int64_t)S->cols.size();
  }
  tri_nbr.clear();
  tri_nbr.shrink_to_fit();
  // ---- work list: every ordered regular pair (p, q) (internal ids) that can
  // reach the pattern: centroids within radius + 2 d, d the largest centroid
  // distance of an RWG function's two triangles
  double d = 0.0;
  for (int64_t e = 0; e < ne; ++e) {
    const int32_t a = m->et[2 * e], b = m->et[2 * e + 1];
    double s2 = 0;
    for (int x = 0; x < 3; ++x) s2 += (cen[3 * (size_t)a + x] - cen[3 * (size_t)b + x]) * (cen[3 * (size_t)a + x] - cen[3 * (size_t)b + x]);
    d = std::max(d, std::sqrt(s2));
  }
  S->work_radius = radius + 2.0 * d * (1.0 + 1e-9);
  std::vector<int64_t> wptr(nt + 1, 0);
  std::vector<int32_t> widx;
  struct Task {
    int32_t p, n;
    int64_t off;
  };
  static_assert(sizeof(Task) == 16, "task record layout");
  std::vector<Task> tasks;
  {
    const Grid grid(cen, S->work_radius);
    std::vector<int32_t> nrow;
    for (int64_t pi = 0; pi < nt; ++pi) {
      const int64_t p = m->perm[pi];
      nrow.clear();
      grid.near(cen, p, S->work_radius, [&](int32_t j) { nrow.push_back(m->inv_perm[j]); });
      std::sort(nrow.begin(), nrow.end());
      // drop the mesh's near pairs (the near-pair path covers them)
      const int32_t* nb = m->near_idx.data() + m->near_ptr[pi];
      const int32_t* ne_ = m->near_idx.data() + m->near_ptr[pi + 1];
      const int64_t start = (int64_t)widx.size();
      for (int32_t q : nrow)
        if (!std::binary_search(nb, ne_, q)) widx.push_back(q);
      const int64_t len = (int64_t)widx.size() - start;
      for (int64_t o = 0; o < len; o += 32)
        tasks.push_back(Task{(int32_t)pi, (int32_t)std::min<int64_t>(32, len - o), start + o});
      wptr[pi + 1] = (int64_t)widx.size();
    }
  }
  S->n_pairs = (int64_t)widx.size();
  S->ntask = (int64_t)tasks.size();
  if (gf::sparse_task_bytes() != (int)sizeof(Task)) return fail(GF_ERR_ARG, "gf_sparse_create: task layout");
  // ---- device: one allocation, one copy
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (std::max<size_t>(bytes, 1) + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_row = take(8 * (ne + 1)), o_cols = take(4 * S->cols.size()), o_tasks = take(16 * tasks.size()),
               o_widx = take(4 * widx.size());
  std::vector<unsigned char> h(off, 0);
  std::memcpy(&h[o_row], S->row_ptr.data(), 8 * (ne + 1));
  if (!S->cols.empty()) std::memcpy(&h[o_cols], S->cols.data(), 4 * S->cols.size());
  if (!tasks.empty()) std::memcpy(&h[o_tasks], tasks.data(), 16 * tasks.size());
  if (!widx.empty()) std::memcpy(&h[o_widx], widx.data(), 4 * widx.size());
  unsigned char* base = nullptr;
  cudaError_t e = cudaMalloc((void**)&base, off);
  if (e != cudaSuccess) return gf::cuda_fail(e, "gf_sparse_create: cudaMalloc");
  e = cudaMemcpy(base, h.data(), off, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(base);
    return gf::cuda_fail(e, "gf_sparse_create: upload");
  }
  S->d_arena = base;
  S->d_row_ptr = reinterpret_cast<int64_t*>(base + o_row);
  S->d_cols = reinterpret_cast<int32_t*>(base + o_cols);
  S->d_tasks = base + o_tasks;
  S->d_widx = reinterpret_cast<int32_t*>(base + o_widx);
  *out = S.release();
  return GF_OK;
}

gf_status gf_sparse_info(const gf_sparse* s, int64_t* nnz, int64_t* n_pairs) {
  if (!s) return fail(GF_ERR_ARG, "gf_sparse_info: null handle");
  if (nnz) *nnz = (int64_t)s->cols.size();
  if (n_pairs) *n_pairs = s->n_pairs;
  return GF_OK;
}

gf_status gf_sparse_pattern(const gf_sparse* s, int64_t* row_ptr, int32_t* cols) {
  if (!s) return fail(GF_ERR_ARG, "gf_sparse_pattern: null handle");
  if (row_ptr) std::memcpy(row_ptr, s->row_ptr.data(), s->row_ptr.size() * 8);
  if (cols && !s->cols.empty()) std::memcpy(cols, s->cols.data(), s->cols.size() * 4);
  return GF_OK;
}

gf_status gf_fill_sparse(const gf_sparse* s, double k, const gf_params* p, const gf_table* table, int precision,
                         void* vals, void* stream) {
  if (!s || !p || !vals) return fail(GF_ERR_ARG, "gf_fill_sparse: null argument");
  if (precision != GF_FP32) return fail(GF_ERR_ARG, "gf_fill_sparse: FP32 (complex64 values) only");
  if (!(k > 0)) return fail(GF_ERR_ARG, "gf_fill_sparse: need k > 0");
  if (p->nphi < 1 || p->nphi > 32 || p->nl < 1 || p->nl > 32 || p->green_from_exp != 0)
    return fail(GF_ERR_ARG, "gf_fill_sparse: bad params");
  gf_mesh* m = const_cast<gf_mesh*>(s->mesh);
  int cur = -1;
  GF_CUDA(cudaGetDevice(&cur));
  if (cur != s->device) return fail(GF_ERR_DEVICE, "gf_fill_sparse: handle on another device");
  gf::TabView tg, te;
  double gscale = 1.0;
  if (table && !gf::table_views(table, k, &tg, &te, &gscale))
    return fail(GF_ERR_ARG, "gf_fill_sparse: table built for another k");
  cudaStream_t st = (cudaStream_t)stream;
  gf_status r = gf::prepare_rule(m, p->rule, st);
  if (r) return r;
  if (s->cols.empty()) return GF_OK;
  GF_CUDA(cudaMemsetAsync(vals, 0, s->cols.size() * 8, st));
  double gx_phi[32], gw_phi[32], gx_l[32], gw_l[32];
  gf::gauss_legendre_host(p->nphi, gx_phi, gw_phi);
  gf::gauss_legendre_host(p->nl, gx_l, gw_l);
  double glp[64] = {}, gll[64] = {};
  for (int i = 0; i < p->nphi; ++i) {
    glp[i] = gx_phi[i];
    glp[32 + i] = gw_phi[i];
  }
  for (int i = 0; i < p->nl; ++i) {
    gll[i] = gx_l[i];
    gll[32 + i] = gw_l[i];
  }
  const gf::GeoView g = gf::geo_view(m);
  GF_CUDA(gf::launch_fill_sparse(g, table ? &tg : nullptr, table ? &te : nullptr, gscale, !p->near_fp64, k, p->eta, p->nphi,
                                 p->nl, glp, gll, s->d_tasks, s->ntask, s->d_widx, s->d_row_ptr, s->d_cols, vals, st));
  return GF_OK;
}

gf_status gf_sparse_destroy(gf_sparse* s) {
  if (!s) return GF_OK;
  if (s->d_arena) {
    cudaDeviceSynchronize();
    cudaFree(s->d_arena);
  }
  delete s;
  return GF_OK;
}

}  // extern "C"
