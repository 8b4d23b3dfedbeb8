// gfmom near-field sparse fill kernels for sm_103a (regular pairs from a
// work list and near pairs, into a CSR pattern), with their launcher.
#include "gf_near.cuh"

namespace gf {
namespace {

// ---------------------------------------------------------------- near-field sparse fill
// Z restricted to a sparsity pattern (the near field of fast solvers, the
// paper's "3mnNC" regime): the same pair computations, each block handed to a
// CsrSink that keeps the entries of the pattern. Regular pairs come from a
// work list of (test triangle, up to 32 source triangles) tasks; every ordered
// pair is listed (no symmetric second write).
struct SparseTask {
  int p;         // internal test triangle
  int n;         // source triangles in this task (1..32)
  int64_t off;   // first source triangle in the work list
};

template <int M, int MODE, bool SMEM, bool KR>
__global__ void __launch_bounds__(SMEM ? 512 : kThreads) k_sparse_regular32(GeoView g, TabView tv, RegK K,
                                                                            const SparseTask* __restrict__ tasks,
                                                                            int64_t ntask, const int32_t* __restrict__ widx,
                                                                            CsrSink<float2> sink) {
  extern __shared__ __align__(16) unsigned char smem[];
  Tab32 T = tab32(tv);
  if (MODE != kDirect && SMEM) {
    stage_tab32(T, tv, 3, smem);
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntask; t += nwarp) {
    const SparseTask tk = tasks[t];
    const bool ok = lane < tk.n;
    const int q = ok ? widx[tk.off + lane] : tk.p;
    regular_pair32<M, MODE, KR, SMEM && MODE != kDirect>(g, T, K, tk.p, q, ok, sink);
  }
}

// Near pairs of the mesh's near list into the pattern.
template <bool MIXED, int G>
__global__ void __launch_bounds__(128) k_sparse_near(GeoView g, TabView te, bool use_table, NearArgs A,
                                                     CsrSink<float2> sink) {
  const Tab32 te32 = tab32(te);
  const float lo32 = (float)te.r_lo, hi32 = (float)te.r_hi;
  const int64_t n_near = g.near_ptr[g.nt];
  const int sub = threadIdx.x & (G - 1);
  const unsigned gmask = ((1u << G) - 1u) << (threadIdx.x & (32 - G));
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / G;
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t iters = (n_near + ngroups - 1) / ngroups;
  const KScal ks{A.k, A.scale, A.inv_k2, 1.0 / A.k, (float)(4.0 * A.inv_k2), (float)A.scale};
  for (int64_t it = 0; it < iters; ++it) {
    const int64_t idx = g0 + it * ngroups;
    near_pair<MIXED, G>(g, te, te32, lo32, hi32, use_table, A, ks, sink, idx, idx < n_near, sub, gmask);
  }
}

}  // namespace

template <int M, bool KR>
cudaError_t launch_sparse32(const GeoView& g, const TabView* table, const RegK& K, const SparseTask* tasks,
                            int64_t ntask, const int32_t* widx, CsrSink<float2> sink, cudaStream_t s) {
  if (ntask == 0) return cudaSuccess;
  if (!table) {
    TabView tv{};
    const int64_t blocks = std::min<int64_t>((ntask + kWarps - 1) / kWarps, (int64_t)sm_count() * 4);
    k_sparse_regular32<M, kDirect, false, false><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, K, tasks, ntask, widx,
                                                                                      sink);
    return cudaGetLastError();
  }
  const TabView& tv = *table;
  const size_t smem = tv.smem32_bytes(3);
  int dev = 0, max_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem <= (size_t)max_optin) {
    auto kern = k_sparse_regular32<M, kLagrange, true, KR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = std::min<int64_t>((ntask + 15) / 16, (int64_t)sm_count());
    kern<<<(unsigned)blocks, 512, smem, s>>>(g, tv, K, tasks, ntask, widx, sink);
  } else {
    const int64_t blocks = std::min<int64_t>((ntask + kWarps - 1) / kWarps, (int64_t)sm_count() * 4);
    k_sparse_regular32<M, kLagrange, false, KR><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, K, tasks, ntask, widx,
                                                                                     sink);
  }
  return cudaGetLastError();
}

template <int M>
cudaError_t launch_sparse32_any(const GeoView& g, const TabView* table, const RegK& K, const SparseTask* tasks,
                                int64_t ntask, const int32_t* widx, CsrSink<float2> sink, cudaStream_t s) {
  if (table && table->xscale32 != 1.f) return launch_sparse32<M, true>(g, table, K, tasks, ntask, widx, sink, s);
  return launch_sparse32<M, false>(g, table, K, tasks, ntask, widx, sink, s);
}

cudaError_t launch_fill_sparse(const GeoView& g, const TabView* green, const TabView* texp, double green_scale,
                               bool mixed, double k, double eta, int nphi, int nl, const double* gl_phi,
                               const double* gl_l, const void* tasks_v, int64_t ntask, const int32_t* widx,
                               const int64_t* row_ptr, const int32_t* cols, void* vals, cudaStream_t s) {
  const SparseTask* tasks = static_cast<const SparseTask*>(tasks_v);
  CsrSink<float2> sink{row_ptr, cols, static_cast<float2*>(vals)};
  const double scale = k * eta / (4.0 * kPi) * (green ? green_scale : 1.0);
  const RegK K = reg_consts(k, scale);
  cudaError_t e;
  switch (g.m) {
    case 1: e = launch_sparse32_any<1>(g, green, K, tasks, ntask, widx, sink, s); break;
    case 3: e = launch_sparse32_any<3>(g, green, K, tasks, ntask, widx, sink, s); break;
    case 4: e = launch_sparse32_any<4>(g, green, K, tasks, ntask, widx, sink, s); break;
    case 6: e = launch_sparse32_any<6>(g, green, K, tasks, ntask, widx, sink, s); break;
    case 7: e = launch_sparse32_any<7>(g, green, K, tasks, ntask, widx, sink, s); break;
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
  const bool use_table = texp != nullptr;
  const unsigned nblk = (unsigned)(sm_count() * 16);
  if (g.m <= 4) {
    if (mixed) k_sparse_near<true, 4><<<nblk, 128, 0, s>>>(g, te, use_table, A, sink);
    else k_sparse_near<false, 4><<<nblk, 128, 0, s>>>(g, te, use_table, A, sink);
  } else {
    if (mixed) k_sparse_near<true, 8><<<nblk, 128, 0, s>>>(g, te, use_table, A, sink);
    else k_sparse_near<false, 8><<<nblk, 128, 0, s>>>(g, te, use_table, A, sink);
  }
  return cudaGetLastError();
}

int sparse_task_bytes() { return (int)sizeof(SparseTask); }

}  // namespace gf
