// gfmom near-field sparse fill kernels for sm_103a (regular pairs from a
// work list and near pairs, into a CSR pattern), with their launcher.
#include "gf_device.cuh"

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

template <int M, int MODE, bool SMEM, bool DEFER>
__global__ void __launch_bounds__(SMEM ? 512 : kThreads) k_sparse_regular32(GeoView g, TabView tv, float kpi,
                                                                            float scale, float inv_k2,
                                                                            const SparseTask* __restrict__ tasks,
                                                                            int64_t ntask, const int32_t* __restrict__ widx,
                                                                            CsrSink<float2> sink) {
  extern __shared__ __align__(16) unsigned char smem[];
  Tab32 T = tab32(tv);
  if (MODE != kDirect && SMEM) {
    const int nl = tv.n_lat, nblob = (int)tv.blob_vec4();
    float4* sa = reinterpret_cast<float4*>(smem);
    float4* sb = sa + nl;
    float4* sblob = sb + nl;
    for (int i = threadIdx.x; i < nl; i += blockDim.x) {
      sa[i] = tv.lat_a[i];
      sb[i] = tv.lat_b[i];
    }
    for (int i = threadIdx.x; i < nblob; i += blockDim.x) sblob[i] = tv.lat_blob[i];
    __syncthreads();
    T.la = sa;
    T.lb = sb;
    tab32_blob(T, tv, sblob);
  }
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < ntask; t += nwarp) {
    const SparseTask tk = tasks[t];
    const bool ok = lane < tk.n;
    const int q = ok ? widx[tk.off + lane] : tk.p;
    regular_pair32<M, MODE, DEFER>(g, T, kpi, scale, inv_k2, tk.p, q, ok, sink);
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

template <int M>
cudaError_t launch_sparse32(const GeoView& g, const TabView* table, float kpi, float scale, float inv_k2,
                            const SparseTask* tasks, int64_t ntask, const int32_t* widx, CsrSink<float2> sink,
                            cudaStream_t s) {
  if (ntask == 0) return cudaSuccess;
  if (!table) {
    TabView tv{};
    const int64_t blocks = std::min<int64_t>((ntask + kWarps - 1) / kWarps, (int64_t)sm_count() * 4);
    k_sparse_regular32<M, kDirect, false, false><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, kpi, scale, inv_k2,
                                                                                      tasks, ntask, widx, sink);
    return cudaGetLastError();
  }
  const TabView& tv = *table;
  const size_t smem = tv.smem32_bytes(3);
  int dev = 0, max_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem <= (size_t)max_optin) {
    auto kern = tv.n_busy * 200 <= tv.n_lat ? k_sparse_regular32<M, kLagrange, true, true>
                                            : k_sparse_regular32<M, kLagrange, true, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = std::min<int64_t>((ntask + 15) / 16, (int64_t)sm_count());
    kern<<<(unsigned)blocks, 512, smem, s>>>(g, tv, kpi, scale, inv_k2, tasks, ntask, widx, sink);
  } else {
    const int64_t blocks = std::min<int64_t>((ntask + kWarps - 1) / kWarps, (int64_t)sm_count() * 4);
    k_sparse_regular32<M, kLagrange, false, false><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, kpi, scale, inv_k2,
                                                                                        tasks, ntask, widx, sink);
  }
  return cudaGetLastError();
}

cudaError_t launch_fill_sparse(const GeoView& g, const TabView* green, const TabView* texp, double green_scale,
                               bool mixed, double k, double eta, int nphi, int nl, const double* gl_phi,
                               const double* gl_l, const void* tasks_v, int64_t ntask, const int32_t* widx,
                               const int64_t* row_ptr, const int32_t* cols, void* vals, cudaStream_t s) {
  const SparseTask* tasks = static_cast<const SparseTask*>(tasks_v);
  CsrSink<float2> sink{row_ptr, cols, static_cast<float2*>(vals)};
  const double scale = k * eta / (4.0 * kPi) * (green ? green_scale : 1.0);
  const float kpi = (float)(k / kPi), sc = (float)scale, ik2 = (float)(1.0 / (k * k));
  cudaError_t e;
  switch (g.m) {
    case 1: e = launch_sparse32<1>(g, green, kpi, sc, ik2, tasks, ntask, widx, sink, s); break;
    case 3: e = launch_sparse32<3>(g, green, kpi, sc, ik2, tasks, ntask, widx, sink, s); break;
    case 4: e = launch_sparse32<4>(g, green, kpi, sc, ik2, tasks, ntask, widx, sink, s); break;
    case 6: e = launch_sparse32<6>(g, green, kpi, sc, ik2, tasks, ntask, widx, sink, s); break;
    case 7: e = launch_sparse32<7>(g, green, kpi, sc, ik2, tasks, ntask, widx, sink, s); break;
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
