// gfmom batched fill kernels for sm_103a: persistent regular and near
// kernels over the work lists of many meshes, with their launchers.
#include <algorithm>

#include "gf_near.cuh"

namespace gf {
namespace {

// ---------------------------------------------------------------- batched
// Persistent kernels over the regular tasks and near pairs of many meshes:
// warps pull chunks of a global task list (meshes with the most work first)
// from an atomic counter; the mesh of a task is found by binary search in the
// descriptors' prefix offsets. Every mesh has its own k, tables and Z.
__device__ __forceinline__ int batch_item_of(const BatchItem* items, int nitems, int64_t t, bool near) {
  int lo = 0, hi = nitems - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int64_t b = near ? items[mid].near_begin : items[mid].reg_begin;
    if (b <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int M, bool TABLE>
__global__ void __launch_bounds__(512) k_batch_regular32(const BatchItem* __restrict__ items, int nitems, int64_t total,
                                                         unsigned long long* counter, int chunk) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(counter, (unsigned long long)chunk);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((int64_t)base >= total) break;
    const int64_t end = min((int64_t)base + chunk, total);
    for (int64_t t = (int64_t)base; t < end; ++t) {
      const BatchItem& it = items[batch_item_of(items, nitems, t, false)];
      const Tab32 T = tab32(it.green);
      int p, q0;
      if (sym_task(t - it.reg_begin, it.g.nt, &p, &q0))
        regular_task32<M, TABLE ? kLagrange : kDirect, TABLE, false>(
            it.g, T, it.rk, DenseUpper{reinterpret_cast<float2*>(it.Z), it.ldz}, p, q0, lane);
    }
  }
}

// Z <- Z + Z^T per mesh over a global list of 32 x 32 tile pairs (I <= J)
// of all meshes: both tiles through shared memory, both written (a diagonal
// tile is its own partner). HBM-bound.
__device__ __forceinline__ int batch_mirror_item(const BatchItem* items, int nitems, int64_t t) {
  int lo = 0, hi = nitems - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].mir_begin <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(256) k_batch_mirror(const BatchItem* __restrict__ items, int nitems, int64_t total) {
  __shared__ float2 ta[32][33];
  __shared__ float2 tb[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
    const BatchItem& it = items[batch_mirror_item(items, nitems, t)];
    const int64_t u = t - it.mir_begin;
    // tile pair u -> (I, J), I <= J, column by column: u = J (J + 1) / 2 + I
    int64_t J = (int64_t)((sqrtf(8.f * (float)u + 1.f) - 1.f) * 0.5f);
    while (J > 0 && J * (J + 1) / 2 > u) --J;
    while ((J + 1) * (J + 2) / 2 <= u) ++J;
    const int I = (int)(u - J * (J + 1) / 2);
    const int ne = it.ne;
    const int64_t ldz = it.ldz;
    float2* Z = reinterpret_cast<float2*>(it.Z);
    for (int r = ty; r < 32; r += 8) {
      const int gr = I * 32 + r, gc = (int)J * 32 + tx;
      ta[r][tx] = (gr < ne && gc < ne) ? Z[(int64_t)gr * ldz + gc] : make_float2(0.f, 0.f);
      const int hr = (int)J * 32 + r, hc = I * 32 + tx;
      tb[r][tx] = (hr < ne && hc < ne) ? Z[(int64_t)hr * ldz + hc] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int gr = I * 32 + r, gc = (int)J * 32 + tx;
      const float2 a = ta[r][tx], b = tb[tx][r];
      if (gr < ne && gc < ne) Z[(int64_t)gr * ldz + gc] = make_float2(a.x + b.x, a.y + b.y);
      if (I != J) {
        const int hr = (int)J * 32 + r, hc = I * 32 + tx;
        const float2 c = tb[r][tx], d = ta[tx][r];
        if (hr < ne && hc < ne) Z[(int64_t)hr * ldz + hc] = make_float2(c.x + d.x, c.y + d.y);
      }
    }
    __syncthreads();
  }
}

template <bool MIXED>
__global__ void __launch_bounds__(128) k_batch_near(const BatchItem* __restrict__ items, int nitems, int64_t total,
                                                    unsigned long long* counter, NearArgs A) {
  const int lane = threadIdx.x & 31;
  const int sub = threadIdx.x & 7;
  const unsigned gmask = 0xFFu << (threadIdx.x & 24);
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(counter, 4ull);  // one near pair per 8-lane group
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((int64_t)base >= total) break;
    const int64_t t = (int64_t)base + (lane >> 3);
    if (t < total) {
      const BatchItem& it = items[batch_item_of(items, nitems, t, true)];
      const Tab32 te32 = tab32(it.exp);
      near_task<float2, MIXED>(it.g, it.exp, te32, (float)it.exp.r_lo, (float)it.exp.r_hi, it.use_table != 0, A,
                               KScal{it.k, it.scale, it.inv_k2, 1.0 / it.k, (float)(4.0 * it.inv_k2), (float)it.scale}, reinterpret_cast<float2*>(it.Z), it.ldz, it.n_near,
                               t - it.near_begin, true, sub, gmask);
    }
  }
}

}  // namespace

template <int M>
cudaError_t launch_batch_regular_m(const BatchItem* items, int nitems, int64_t total, unsigned long long* counter,
                                   bool table, int block, int grid, int chunk, cudaStream_t s) {
  if (table)
    k_batch_regular32<M, true><<<grid, block, 0, s>>>(items, nitems, total, counter, chunk);
  else
    k_batch_regular32<M, false><<<grid, block, 0, s>>>(items, nitems, total, counter, chunk);
  return cudaGetLastError();
}

cudaError_t launch_batch_regular(const BatchItem* items, int nitems, int64_t total, unsigned long long* counter, int m,
                                 bool table, int block, int grid, int chunk, cudaStream_t s) {
  switch (m) {
    case 1: return launch_batch_regular_m<1>(items, nitems, total, counter, table, block, grid, chunk, s);
    case 3: return launch_batch_regular_m<3>(items, nitems, total, counter, table, block, grid, chunk, s);
    case 4: return launch_batch_regular_m<4>(items, nitems, total, counter, table, block, grid, chunk, s);
    case 6: return launch_batch_regular_m<6>(items, nitems, total, counter, table, block, grid, chunk, s);
    case 7: return launch_batch_regular_m<7>(items, nitems, total, counter, table, block, grid, chunk, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int M>
int batch_blocks_m(bool table, int block) {
  int n = 0;
  if (table) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_regular32<M, true>, block, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_regular32<M, false>, block, 0);
  return n;
}

int batch_regular_blocks_per_sm(int m, bool table, int block) {
  switch (m) {
    case 1: return batch_blocks_m<1>(table, block);
    case 3: return batch_blocks_m<3>(table, block);
    case 4: return batch_blocks_m<4>(table, block);
    case 6: return batch_blocks_m<6>(table, block);
    case 7: return batch_blocks_m<7>(table, block);
    default: return 0;
  }
}

cudaError_t launch_batch_mirror(const BatchItem* items, int nitems, int64_t total, int grid, cudaStream_t s) {
  if (total == 0) return cudaSuccess;
  k_batch_mirror<<<(unsigned)std::min<int64_t>(total, grid), 256, 0, s>>>(items, nitems, total);
  return cudaGetLastError();
}

template <int M>
cudaError_t set_l1_m(bool table, bool max_l1) {
  const int carve = max_l1 ? 0 : -1;  // 0: all of the unified memory as L1; -1: the driver's default
  return table ? cudaFuncSetAttribute(k_batch_regular32<M, true>, cudaFuncAttributePreferredSharedMemoryCarveout, carve)
               : cudaFuncSetAttribute(k_batch_regular32<M, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      carve);
}

cudaError_t set_batch_regular_l1(int m, bool table, bool max_l1) {
  switch (m) {
    case 1: return set_l1_m<1>(table, max_l1);
    case 3: return set_l1_m<3>(table, max_l1);
    case 4: return set_l1_m<4>(table, max_l1);
    case 6: return set_l1_m<6>(table, max_l1);
    case 7: return set_l1_m<7>(table, max_l1);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_batch_near(const BatchItem* items, int nitems, int64_t total, unsigned long long* counter,
                              bool mixed, int nphi, int nl, const double* gl_phi, const double* gl_l, int grid,
                              cudaStream_t s) {
  NearArgs A;
  A.k = A.scale = A.inv_k2 = 0.0;  // per mesh, from the descriptors
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
  if (mixed) k_batch_near<true><<<grid, 128, 0, s>>>(items, nitems, total, counter, A);
  else k_batch_near<false><<<grid, 128, 0, s>>>(items, nitems, total, counter, A);
  return cudaGetLastError();
}

}  // namespace gf
