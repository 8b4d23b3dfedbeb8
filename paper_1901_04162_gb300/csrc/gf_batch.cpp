// Batched fill: many meshes, each with its own wavenumber, tables and Z, in
// one persistent launch per kernel, captured once in a CUDA graph and
// replayed. The persistent kernels' block size, CTAs per SM and task chunk
// are chosen by a small autotuner whose choices are cached on disk.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include <sys/stat.h>

#include "gf_internal.h"

using namespace gf;

struct gf_batch {
  int device = -1;
  int m = 0;
  bool table = false;
  bool mixed = true;
  int nphi = 8, nl = 8;
  double glp[64], gll[64];
  std::vector<BatchItem> items;  // host copy, sorted by decreasing regular work
  BatchItem* d_items = nullptr;
  unsigned long long* d_counters = nullptr;  // [0] regular, [1] near
  std::vector<void*> z;
  std::vector<int64_t> ldz, ne;
  int64_t total_regular = 0, total_near = 0, total_mirror = 0;
  int block = 256, ctas = 2, chunk = 4;
  int max_l1 = 0;  // 1: the regular kernel with all of the unified memory as L1 (the tables are read through it)
  double tuned_ms = 0.0;
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void release_graph(gf_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Captures zeroing of every Z, the counter reset, the persistent regular
// kernel, one mirror pass over every Z and the persistent near kernel on the
// batch's own stream.
gf_status capture(gf_batch* b, int block, int ctas, int chunk, int max_l1) {
  release_graph(b);
  int sms = 1;
  GF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  GF_CUDA(set_batch_regular_l1(b->m, b->table, max_l1 != 0));
  GF_CUDA(cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < b->z.size() && e == cudaSuccess; ++i)
    e = cudaMemset2DAsync(b->z[i], (size_t)b->ldz[i] * 8, 0, (size_t)b->ne[i] * 8, (size_t)b->ne[i], b->cs);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counters, 0, 2 * sizeof(unsigned long long), b->cs);
  if (e == cudaSuccess && b->total_regular > 0)
    e = launch_batch_regular(b->d_items, (int)b->items.size(), b->total_regular, b->d_counters, b->m, b->table, block,
                             sms * ctas, chunk, b->cs);
  // the regular kernel leaves each pair in its test triangle's rows: Z += Z^T for every mesh
  if (e == cudaSuccess && b->total_regular > 0)
    e = launch_batch_mirror(b->d_items, (int)b->items.size(), b->total_mirror, sms * 8, b->cs);
  if (e == cudaSuccess && b->total_near > 0)
    e = launch_batch_near(b->d_items, (int)b->items.size(), b->total_near, b->d_counters + 1, b->mixed, b->nphi,
                          b->nl, b->glp, b->gll, sms * 16, b->cs);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->cs, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(e, "gf_batch capture");
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  b->graph = g;
  GF_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
  b->block = block;
  b->ctas = ctas;
  b->max_l1 = max_l1;
  b->chunk = chunk;
  return GF_OK;
}

// The tuner's cache file: only where $GF_AUTOTUNE_CACHE names one (the
// library writes nothing else on the host); "" or "off" = no cache.
std::string cache_path() {
  const char* p = std::getenv("GF_AUTOTUNE_CACHE");
  return p ? std::string(p) : std::string();
}

std::string tune_key(const gf_batch* b) {
  cudaDeviceProp prop;
  std::string name = "gpu";
  if (cudaGetDeviceProperties(&prop, b->device) == cudaSuccess) name = prop.name;
  for (char& c : name)
    if (c == ' ' || c == '|') c = '_';
  int lg = 0;
  for (int64_t t = b->total_regular; t > 1; t >>= 1) ++lg;
  char buf[256];
  std::snprintf(buf, sizeof buf, "v2|%s|sm%d|m%d|t%d|n%d|i%zu", name.c_str(),
                prop.multiProcessorCount, b->m, (int)b->table, lg, b->items.size());
  return std::string(buf);
}

bool cache_lookup(const std::string& key, int* block, int* ctas, int* chunk, int* l1, double* ms) {
  std::string path = cache_path();
  if (path.empty() || path == "off") return false;
  FILE* f = std::fopen(path.c_str(), "r");
  if (!f) return false;
  char k[512];
  int bl, ct, ch, li;
  double t;
  bool found = false;
  while (std::fscanf(f, "%511s %d %d %d %d %lf", k, &bl, &ct, &ch, &li, &t) == 6) {
    if (key == k) {  // the last entry for a key wins
      *block = bl;
      *ctas = ct;
      *chunk = ch;
      *l1 = li;
      *ms = t;
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

void cache_store(const std::string& key, int block, int ctas, int chunk, int l1, double ms) {
  std::string path = cache_path();
  if (path.empty() || path == "off") return;
  for (size_t i = 1; i < path.size(); ++i)  // parent directories, errors ignored
    if (path[i] == '/') mkdir(path.substr(0, i).c_str(), 0755);
  FILE* f = std::fopen(path.c_str(), "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %d %d %.6f\n", key.c_str(), block, ctas, chunk, l1, ms);
  std::fclose(f);
}

// Times `reps` graph launches on the batch stream (after one warm-up).
gf_status time_graph(gf_batch* b, int reps, double* ms) {
  cudaEvent_t e0, e1;
  GF_CUDA(cudaEventCreate(&e0));
  GF_CUDA(cudaEventCreate(&e1));
  cudaError_t e = cudaGraphLaunch(b->exec, b->cs);
  if (e == cudaSuccess) e = cudaEventRecord(e0, b->cs);
  for (int i = 0; i < reps && e == cudaSuccess; ++i) e = cudaGraphLaunch(b->exec, b->cs);
  if (e == cudaSuccess) e = cudaEventRecord(e1, b->cs);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "gf_batch timing");
  *ms = t / reps;
  return GF_OK;
}

// Tuning in two stages, each configuration timed over 5 graph replays: the
// launch shape (block size, resident CTAs per SM) at task chunk 4, then at
// the best shape the work granularity and tile order (a warp takes 1, 4 or 32
// consecutive tasks; 32 = the 32 test triangles of one block pair in a row,
// reusing the source block's data) and the table's cache (the regular kernel
// with all of the unified memory as L1, which holds the meshes' lattice
// images, or the driver's split).
gf_status autotune(gf_batch* b) {
  const std::string key = tune_key(b);
  int bl, ct, ch, li;
  double ms;
  if (cache_lookup(key, &bl, &ct, &ch, &li, &ms)) {
    b->tuned_ms = ms;
    return capture(b, bl, ct, ch, li);
  }
  double best = INFINITY;
  int best_bl = 256, best_ct = 2, best_ch = 4, best_l1 = 0;
  const int blocks[] = {128, 256, 512};
  for (int block : blocks) {
    const int occ = batch_regular_blocks_per_sm(b->m, b->table, block);
    for (int ctas = 1; ctas <= std::min(occ, 4); ++ctas) {
      gf_status st = capture(b, block, ctas, 4, 0);
      if (st) return st;
      double t;
      if ((st = time_graph(b, 5, &t))) return st;
      if (t < best) {
        best = t;
        best_bl = block;
        best_ct = ctas;
      }
    }
  }
  const int chunks[] = {1, 4, 32};
  for (int l1 = 0; l1 <= 1; ++l1)
    for (int chunk : chunks) {
      if (chunk == 4 && l1 == 0) continue;  // timed above
      gf_status st = capture(b, best_bl, best_ct, chunk, l1);
      if (st) return st;
      double t;
      if ((st = time_graph(b, 5, &t))) return st;
      if (t < best) {
        best = t;
        best_ch = chunk;
        best_l1 = l1;
      }
    }
  b->tuned_ms = best;
  cache_store(key, best_bl, best_ct, best_ch, best_l1, best);
  return capture(b, best_bl, best_ct, best_ch, best_l1);
}

}  // namespace

extern "C" {

gf_status gf_batch_create(int nmesh, const gf_mesh* const* meshes, const double* k, const gf_params* p,
                          const gf_table* const* tables, int precision, void* const* Z, const int64_t* ldz,
                          int autotune_flag, void* stream, gf_batch** out) {
  if (nmesh < 1 || !meshes || !k || !p || !Z || !ldz || !out)
    return fail(GF_ERR_ARG, "gf_batch_create: bad arguments");
  if (precision != GF_FP32) return fail(GF_ERR_ARG, "gf_batch_create: batched fills are GF_FP32");
  if (p->green_from_exp) return fail(GF_ERR_ARG, "gf_batch_create: green_from_exp must be 0");
  std::unique_ptr<gf_batch> b(new (std::nothrow) gf_batch);
  if (!b) return fail(GF_ERR_ALLOC, "gf_batch_create: out of host memory");
  GF_CUDA(cudaGetDevice(&b->device));
  b->m = p->rule;
  b->table = tables != nullptr;
  b->mixed = !p->near_fp64;
  b->nphi = p->nphi;
  b->nl = p->nl;
  if (p->nphi < 1 || p->nphi > 32 || p->nl < 1 || p->nl > 32 || !(p->eta > 0))
    return fail(GF_ERR_ARG, "gf_batch_create: bad params");
  double x[32], w[32];
  gauss_legendre_host(p->nphi, x, w);
  for (int i = 0; i < 32; ++i) {
    b->glp[i] = i < p->nphi ? x[i] : 0.0;
    b->glp[32 + i] = i < p->nphi ? w[i] : 0.0;
  }
  gauss_legendre_host(p->nl, x, w);
  for (int i = 0; i < 32; ++i) {
    b->gll[i] = i < p->nl ? x[i] : 0.0;
    b->gll[32 + i] = i < p->nl ? w[i] : 0.0;
  }
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> order(nmesh);
  std::vector<BatchItem> items(nmesh);
  for (int i = 0; i < nmesh; ++i) {
    gf_mesh* m = const_cast<gf_mesh*>(meshes[i]);
    if (!m || !Z[i] || !(k[i] > 0) || ldz[i] < m->ne) return fail(GF_ERR_ARG, "gf_batch_create: bad mesh entry");
    if (m->device != b->device) return fail(GF_ERR_DEVICE, "gf_batch_create: mesh on another device");
    if (tables && (!tables[i] || tables[i]->device != b->device))
      return fail(GF_ERR_ARG, "gf_batch_create: table missing or on another device");
    gf_status st = prepare_rule(m, p->rule, s);
    if (st) return st;
    BatchItem& it = items[i];
    std::memset(&it, 0, sizeof it);
    it.g = geo_view(m);
    double gscale = 1.0;
    if (tables && !table_views(tables[i], k[i], &it.green, &it.exp, &gscale))
      return fail(GF_ERR_ARG, "gf_batch_create: table built for another k");
    it.use_table = tables ? 1 : 0;
    it.rk = reg_consts(k[i], k[i] * p->eta / (4.0 * kPi) * gscale);
    it.k = k[i];
    it.scale = k[i] * p->eta;
    it.inv_k2 = 1.0 / (k[i] * k[i]);
    it.Z = Z[i];
    it.ldz = ldz[i];
    it.nchunk = (m->nt + 31) / 32;
    it.n_near = (int64_t)m->near_idx.size();
    order[i] = i;
  }
  // longest first, so the tail of the persistent loop holds the small meshes
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    return items[a].g.nt > items[c].g.nt;
  });
  int64_t reg = 0, nr = 0, mir = 0;
  for (int i : order) {
    BatchItem it = items[i];
    it.reg_begin = reg;
    it.near_begin = nr;
    it.mir_begin = mir;
    it.ne = (int)meshes[i]->ne;
    reg += gf::regular_units(it.g.nt);
    nr += it.n_near;
    const int64_t nb = (it.ne + 31) / 32;
    mir += nb * (nb + 1) / 2;
    b->items.push_back(it);
    b->z.push_back(Z[i]);
    b->ldz.push_back(ldz[i]);
    b->ne.push_back(meshes[i]->ne);
  }
  b->total_regular = reg;
  b->total_near = nr;
  b->total_mirror = mir;
  cudaError_t e = cudaMalloc(&b->d_items, b->items.size() * sizeof(BatchItem));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_items, b->items.data(), b->items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    gf_batch_destroy(b.release());
    return cuda_fail(e, "gf_batch_create");
  }
  gf_status st = autotune_flag ? autotune(b.get()) : capture(b.get(), 256, 2, 4, 0);
  if (st) {
    gf_batch_destroy(b.release());
    return st;
  }
  *out = b.release();
  return GF_OK;
}

gf_status gf_batch_launch(const gf_batch* b, void* stream) {
  if (!b || !b->exec) return fail(GF_ERR_ARG, "gf_batch_launch: bad batch");
  int cur = -1;
  GF_CUDA(cudaGetDevice(&cur));
  if (cur != b->device) return fail(GF_ERR_DEVICE, "gf_batch_launch: batch belongs to another device");
  GF_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  return GF_OK;
}

gf_status gf_batch_config(const gf_batch* b, int* block, int* ctas_per_sm, int* chunk, double* tuned_ms) {
  if (!b) return fail(GF_ERR_ARG, "gf_batch_config: null batch");
  if (block) *block = b->block;
  if (ctas_per_sm) *ctas_per_sm = b->ctas;
  if (chunk) *chunk = b->chunk;
  if (tuned_ms) *tuned_ms = b->tuned_ms;
  return GF_OK;
}

gf_status gf_batch_destroy(gf_batch* b) {
  if (!b) return GF_OK;
  if (b->cs) cudaStreamSynchronize(b->cs);
  release_graph(b);
  if (b->cs) cudaStreamDestroy(b->cs);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_counters) cudaFree(b->d_counters);
  delete b;
  return GF_OK;
}

gf_status gf_fill_batched(int nmesh, const gf_mesh* const* meshes, const double* k, const gf_params* p,
                          const gf_table* const* tables, void* const* Z, const int64_t* ldz, void* stream) {
  gf_batch* b = nullptr;
  gf_status st = gf_batch_create(nmesh, meshes, k, p, tables, GF_FP32, Z, ldz, 0, stream, &b);
  if (st) return st;
  st = gf_batch_launch(b, stream);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  gf_batch_destroy(b);
  if (st) return st;
  if (e != cudaSuccess) return cuda_fail(e, "gf_fill_batched");
  return GF_OK;
}

}  // extern "C"
