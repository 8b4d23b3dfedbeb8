// gf_range_noalloc: the table-range reduction for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs while a CUDA
// graph is being captured and must not allocate, plug-ins of host
// applications that hand out every device allocation from their own pools,
// or callers with a hard device-memory budget. For them this entry point
// takes device inputs and a device output only, and keeps its scratch (the
// integration points of every triangle and the min/max accumulator) in the
// file-scope array below. The array is part of every GPU that loads the
// library and stays there until the process exits; its size caps the problem
// size.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>
#include <string>
#include <utility>

#include "gf_internal.h"

namespace {

constexpr int64_t kMaxPoints = GF_NOALLOC_MAX_POINTS;
constexpr int kMaxDevices = 64;

struct __align__(32) P4 {
  double x, y, z, w;
};

// [0, kMaxPoints): integration points (x, y, z, unused); slot kMaxPoints
// holds the min / max accumulator as two double bit patterns.
static __device__ __align__(256) P4 g_noalloc_scratch[kMaxPoints + 1];

// The scratch array's device address, per device and per context: a device
// reset (cudaDeviceReset) or a new primary context reloads the module, and
// the array may then sit elsewhere, so the address is looked up again when
// the device's current context is not the one it was taken in (contexts are
// told apart by their driver ID, unique for the life of the process).
struct Slot {
  bool ready = false;
  unsigned long long ctx_id = 0;
  P4* base = nullptr;
};
std::mutex g_mu;
Slot g_slots[kMaxDevices];

// The driver ID of the calling thread's current context (cuCtxGetCurrent and
// cuCtxGetId, fetched through the runtime so the library links no driver
// API); false if the driver does not provide them (then every call looks the
// address up).
bool current_context_id(unsigned long long* id) {
  typedef int (*GetCurrent)(void**);
  typedef int (*GetId)(void*, unsigned long long*);
  static const std::pair<GetCurrent, GetId> fns = [] {
    void* f = nullptr;
    void* g = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      g = nullptr;
    return std::make_pair(reinterpret_cast<GetCurrent>(f), reinterpret_cast<GetId>(g));
  }();
  if (!fns.first || !fns.second) return false;
  void* ctx = nullptr;
  if (fns.first(&ctx) != 0 || !ctx) return false;
  return fns.second(ctx, id) == 0;
}

struct Bary {
  double v[3 * gf::kMaxRule];
};

// Integration points of every triangle; thread 0 also resets the accumulator
// (the scratch keeps the previous call's contents).
__global__ void k_na_points(const double* __restrict__ tri_xyz, int nt, int m, Bary bw, P4* pts,
                            unsigned long long* acc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    acc[0] = (unsigned long long)__double_as_longlong(INFINITY);
    acc[1] = 0ull;
  }
  if (t >= nt) return;
  const double* v = tri_xyz + 9 * (size_t)t;
  for (int a = 0; a < m; ++a) {
    const double b0 = bw.v[3 * a], b1 = bw.v[3 * a + 1], b2 = bw.v[3 * a + 2];
    P4 p;
    p.x = b0 * v[0] + b1 * v[3] + b2 * v[6];
    p.y = b0 * v[1] + b1 * v[4] + b2 * v[7];
    p.z = b0 * v[2] + b1 * v[5] + b2 * v[8];
    p.w = 0.0;
    pts[(size_t)t * m + a] = p;
  }
}

// One warp per (p, 32 consecutive q); pairs sharing a vertex are skipped.
__global__ void __launch_bounds__(256) k_na_range(const int* __restrict__ tri_vert, int nt, int m,
                                                  const P4* __restrict__ pts, unsigned long long* acc) {
  const int lane = threadIdx.x & 31;
  const int64_t nchunk = (nt + 31) / 32;
  const int64_t ntask = (int64_t)nt * nchunk;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double lo = INFINITY, hi = 0.0;
  for (int64_t task = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < ntask; task += nwarp) {
    const int p = (int)(task / nchunk);
    const int q = (int)(task % nchunk) * 32 + lane;
    if (q >= nt) continue;
    const int* vp = tri_vert + 3 * (size_t)p;
    const int* vq = tri_vert + 3 * (size_t)q;
    bool share = false;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) share |= vp[i] == vq[j];
    if (share) continue;
    for (int a = 0; a < m; ++a) {
      const P4 x = pts[(size_t)p * m + a];
      for (int b = 0; b < m; ++b) {
        const P4 y = pts[(size_t)q * m + b];
        const double dx = x.x - y.x, dy = x.y - y.y, dz = x.z - y.z;
        const double R = sqrt(dx * dx + dy * dy + dz * dz);
        lo = fmin(lo, R);
        hi = fmax(hi, R);
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, off));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, off));
  }
  if (lane == 0) {
    if (lo < INFINITY) atomicMin(&acc[0], (unsigned long long)__double_as_longlong(lo));
    if (hi > 0.0) atomicMax(&acc[1], (unsigned long long)__double_as_longlong(hi));
  }
}

__global__ void k_na_out(const unsigned long long* acc, double* out) {
  out[0] = __longlong_as_double((long long)acc[0]);
  out[1] = __longlong_as_double((long long)acc[1]);
}

}  // namespace

extern "C" gf_status gf_range_noalloc(const double* tri_xyz, const int32_t* tri_vert, int64_t nt, int rule,
                                      double* minmax, void* stream) {
  if (!tri_xyz || !tri_vert || !minmax || nt < 1) return gf::fail(GF_ERR_ARG, "gf_range_noalloc: bad arguments");
  double bary[gf::kMaxRule][3], w[gf::kMaxRule];
  if (!gf::rule_points(rule, bary, w))
    return gf::fail(GF_ERR_ARG, "gf_range_noalloc: rule must be 1, 3, 4, 6 or 7");
  if (nt * (int64_t)rule > kMaxPoints)
    return gf::fail(GF_ERR_ARG, "gf_range_noalloc: nt * rule = " + std::to_string(nt * (int64_t)rule) +
                                    " exceeds GF_NOALLOC_MAX_POINTS = " + std::to_string(kMaxPoints));
  int dev = -1;
  GF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return gf::fail(GF_ERR_DEVICE, "gf_range_noalloc: device index too large");
  P4* base = nullptr;
  {
    // set-up, once per device and context, with that device current: the
    // device address of the scratch array (in host code the symbol is only a
    // host-side stand-in, never a device address)
    std::lock_guard<std::mutex> lock(g_mu);
    Slot& slot = g_slots[dev];
    unsigned long long id = 0;
    const bool known = current_context_id(&id);
    if (!slot.ready || !known || slot.ctx_id != id) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return gf::cuda_fail(e, "gf_range_noalloc: cudaGetSymbolAddress");
      slot.base = static_cast<P4*>(ptr);
      slot.ctx_id = id;
      slot.ready = known;
    }
    base = slot.base;
  }
  Bary bw;
  for (int i = 0; i < 3 * gf::kMaxRule; ++i) bw.v[i] = 0.0;
  for (int a = 0; a < rule; ++a)
    for (int c = 0; c < 3; ++c) bw.v[3 * a + c] = bary[a][c];
  (void)w;
  cudaStream_t s = (cudaStream_t)stream;
  const int ntt = (int)nt;
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(base + kMaxPoints);
  k_na_points<<<(ntt + 127) / 128, 128, 0, s>>>(tri_xyz, ntt, rule, bw, base, acc);
  int sms = 1;
  GF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t tasks = (int64_t)ntt * ((ntt + 31) / 32);
  int64_t blocks = (tasks + 7) / 8;
  if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
  k_na_range<<<(unsigned)blocks, 256, 0, s>>>(tri_vert, ntt, rule, base, acc);
  k_na_out<<<1, 1, 0, s>>>(acc, minmax);
  GF_CUDA(cudaGetLastError());
  return GF_OK;
}
