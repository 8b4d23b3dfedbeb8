// gfmom regular-pair fill kernels for sm_103a: the FP32 kernel over the
// symmetric task list (table in shared memory, through L1, or windowed for
// tables larger than shared memory; Lagrange, Exp x 1/R or direct Green
// values) and the FP64 kernel, with their launchers.
#include "gf_device.cuh"

namespace gf {
namespace {

// Threads of the CTA that holds the table in shared memory (one per SM): 28
// warps for rules of up to 4 points (at most 72 registers a thread; 7 warps per
// scheduler), 16 for the larger rules (128 registers).
template <int M>
constexpr int smem_block() {
  return M <= 4 ? 896 : 512;
}

// One warp per (test triangle p, 32 source triangles) task over the 32 x 32
// triangle block pairs; SMEM: the table's lattice image staged in shared
// memory (one CTA per SM holds it), else read through L1. The direct kernel
// for rules of up to 4 points runs the same CTA shape (one CTA of 896
// threads per SM at 72 registers), which measured faster than three
// 256-thread CTAs per SM. With the Green lattice in shared memory the point
// pairs whose cell holds samples (rare: cells whose polynomials agree count
// as sample-free) are listed (fix_cap entries per CTA after the counts,
// kFixCounts of them, in g.fix) and k_fix_regular32 corrects them; the Exp
// lattice (Exp x 1/R), where such pairs are common, corrects them in the loop.
constexpr int kFixCounts = 4096;  // CTAs of one launch at most (count words, as 2048 int2)

template <int M, int MODE, bool SMEM, bool KR>
__global__ void __launch_bounds__((SMEM || (MODE == kDirect && M <= 4)) ? smem_block<M>() : kThreads, 1)
    k_fill_regular32(GeoView g, TabView tv, RegK K, float2* Z, int64_t ldz, unsigned fix_cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr bool kList = SMEM && MODE == kLagrange;
  __shared__ unsigned fix_n, fix_over;
  Tab32 T = tab32(tv);
  if (SMEM && MODE != kDirect) {
    stage_tab32(T, tv, MODE == kLagrange ? 3 : 1, smem);
    if (threadIdx.x == 0) fix_n = fix_over = 0u;
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const DenseUpper sink{Z, ldz};
  int2* const list = kList ? g.fix + kFixCounts / 2 + (size_t)blockIdx.x * fix_cap : nullptr;
  const int64_t ntask = regular_units(g.nt);
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t task = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < ntask; task += nwarp) {
    int p, q0;
    if (!sym_task(task, g.nt, &p, &q0)) continue;
    unsigned long long emask =
        regular_task32<M, MODE, KR, SMEM || (MODE == kDirect && M <= 4), kList>(g, T, K, sink, p, q0, lane);
    if (kList && emask) {
      const unsigned nb = (unsigned)__popcll(emask);
      unsigned slot = atomicAdd(&fix_n, nb);
      if (slot + nb > fix_cap || slot + nb < slot) fix_over = 1u;
      const int qv = (q0 + lane) << 6;
      while (emask) {
        const int bit = __ffsll((long long)emask) - 1;
        emask &= emask - 1ull;
        if (slot < fix_cap) list[slot] = make_int2(p, qv | bit);
        ++slot;
      }
    }
  }
  if (kList) {
    __syncthreads();
    if (threadIdx.x == 0) reinterpret_cast<unsigned*>(g.fix)[blockIdx.x] = fix_over ? 0xFFFFFFFFu : fix_n;
  }
}

// The corrections of k_fill_regular32's flagged point pairs, launched with
// its grid and CTA shape: CTA b corrects list b (one entry per thread), or,
// where that list overflowed, scans CTA b's tasks again. (As a kernel of its
// own it adds nothing to the pair kernel's registers.)
template <int M, int MODE, bool KR>
__global__ void __launch_bounds__(smem_block<M>(), 1)
    k_fix_regular32(GeoView g, TabView tv, RegK K, float2* Z, int64_t ldz, unsigned fix_cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned n = reinterpret_cast<const unsigned*>(g.fix)[blockIdx.x];
  if (n == 0u) return;
  Tab32 T = tab32(tv);
  stage_tab32(T, tv, MODE == kLagrange ? 3 : 1, smem);
  __syncthreads();
  const DenseUpper sink{Z, ldz};
  if (n != 0xFFFFFFFFu) {
    const int2* list = g.fix + kFixCounts / 2 + (size_t)blockIdx.x * fix_cap;
    for (unsigned i = threadIdx.x; i < n; i += blockDim.x) fix_entry32<M, MODE, KR, true>(g, T, K, sink, list[i]);
    return;
  }
  const int lane = threadIdx.x & 31;
  const int64_t ntask = regular_units(g.nt);
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t task = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < ntask; task += nwarp) {
    int p, q0;
    if (sym_task(task, g.nt, &p, &q0)) fix_rescan32<M, MODE, KR, true>(g, T, K, sink, p, q0, lane);
  }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_fill_regular64(GeoView g, TabView tv, double k, double scale,
                                                             double inv_k2, double2* Z, int64_t ldz) {
  const int lane = threadIdx.x & 31;
  const int m = g.m;
  const int64_t ntask = regular_units(g.nt);
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t task = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < ntask; task += nwarp) {
    int p, q0;
    if (!sym_task(task, g.nt, &p, &q0)) continue;
    const int q = min(q0 + lane, g.nt - 1);
    const float4 cp32 = g.cen32[p], cq32 = g.cen32[q];
    const float3 dc32 = make_float3(cp32.x - cq32.x, cp32.y - cq32.y, cp32.z - cq32.z);
    const bool ok = (q0 + lane < g.nt) && q > p && !pair_is_near(g, p, q, g.tvert[p], g.tvert[q], dc32);
    if (!ok) continue;
    const double* cp = g.cen64 + 4 * (size_t)p;
    const double* cq = g.cen64 + 4 * (size_t)q;
    const double dx = cp[0] - cq[0], dy = cp[1] - cq[1], dz = cp[2] - cq[2];
    double M0r = 0, M0i = 0, Mar[3] = {0, 0, 0}, Mai[3] = {0, 0, 0}, Mbr[3] = {0, 0, 0}, Mbi[3] = {0, 0, 0};
    double Mabr = 0, Mabi = 0;
    for (int a = 0; a < m; ++a) {
      const double* al = g.pts64 + 4 * ((size_t)a * g.nt + p);
      const double ux = dx + al[0], uy = dy + al[1], uz = dz + al[2];
      double s0r = 0, s0i = 0, sbr[3] = {0, 0, 0}, sbi[3] = {0, 0, 0};
      for (int b = 0; b < m; ++b) {
        const double* be = g.pts64 + 4 * ((size_t)b * g.nt + q);
        const double rx = ux - be[0], ry = uy - be[1], rz = uz - be[2];
        const double R = sqrt(rx * rx + ry * ry + rz * rz);
        double gr, gi;
        if (MODE == kLagrange) {
          double2 f = lookup64<3>(tv, R);
          gr = f.x * be[3];
          gi = f.y * be[3];
        } else if (MODE == kExpOverR) {
          double2 f = lookup64<1>(tv, R);
          const double wr = be[3] / R;
          gr = f.x * wr;
          gi = f.y * wr;
        } else {
          double sn, cs;
          sincos(k * R, &sn, &cs);
          const double wr = be[3] / R;
          gr = cs * wr;
          gi = -sn * wr;
        }
        s0r += gr;
        s0i += gi;
        for (int c = 0; c < 3; ++c) {
          sbr[c] += be[c] * gr;
          sbi[c] += be[c] * gi;
        }
      }
      const double wa = al[3];
      M0r += wa * s0r;
      M0i += wa * s0i;
      for (int c = 0; c < 3; ++c) {
        Mar[c] += wa * al[c] * s0r;
        Mai[c] += wa * al[c] * s0i;
        Mbr[c] += wa * sbr[c];
        Mbi[c] += wa * sbi[c];
      }
      Mabr += wa * (al[0] * sbr[0] + al[1] * sbr[1] + al[2] * sbr[2]);
      Mabi += wa * (al[0] * sbi[0] + al[1] * sbi[1] + al[2] * sbi[2]);
    }
    const int4 ep = g.tedge[p], eq = g.tedge[q];
    const int ecp[3] = {ep.x, ep.y, ep.z}, ecq[3] = {eq.x, eq.y, eq.z};
    for (int i = 0; i < 3; ++i) {
      if (!edge_valid(ecp[i])) continue;
      const double* gp = g.geo64 + 4 * (3 * (size_t)p + i);
      const double dMbr = gp[0] * Mbr[0] + gp[1] * Mbr[1] + gp[2] * Mbr[2];
      const double dMbi = gp[0] * Mbi[0] + gp[1] * Mbi[1] + gp[2] * Mbi[2];
      double* zrow = reinterpret_cast<double*>(Z + (int64_t)edge_of(ecp[i]) * ldz);
      for (int j = 0; j < 3; ++j) {
        if (!edge_valid(ecq[j])) continue;
        const double* gq = g.geo64 + 4 * (3 * (size_t)q + j);
        const double eMar = gq[0] * Mar[0] + gq[1] * Mar[1] + gq[2] * Mar[2];
        const double eMai = gq[0] * Mai[0] + gq[1] * Mai[1] + gq[2] * Mai[2];
        const double de = gp[0] * gq[0] + gp[1] * gq[1] + gp[2] * gq[2];
        const double br = 0.25 * (Mabr + eMar + dMbr + de * M0r) - M0r * inv_k2;
        const double bi = 0.25 * (Mabi + eMai + dMbi + de * M0i) - M0i * inv_k2;
        const double c = scale * gp[3] * gq[3];
        double* z = zrow + 2 * edge_of(ecq[j]);
        atomicAdd(z, -c * bi);
        atomicAdd(z + 1, c * br);
        double* zt = reinterpret_cast<double*>(Z + (int64_t)edge_of(ecq[j]) * ldz + edge_of(ecp[i]));
        atomicAdd(zt, -c * bi);
        atomicAdd(zt + 1, c * br);
      }
    }
  }
}

// ---------------------------------------------------------------- windowed table
// Tables larger than shared memory: the fill runs over tiles of 32 test
// triangles x 512 source triangles (consecutive in the Morton order, so
// spatially compact); the bounding spheres of the two sets bound every point
// distance of the tile, and only the lattice records of that distance window
// are staged into shared memory (sub-cells and the interval records of cells
// holding samples stay in global memory). A tile whose window does not fit
// reads the table through L1.
constexpr int kTileQBlocks = 16;
constexpr int kWinBytes = 200 * 1024;

template <int M, bool KR>
__global__ void __launch_bounds__(512) k_fill_regular32_win(GeoView g, TabView tv, const float4* __restrict__ bsph,
                                                            RegK K, float2* Z, int64_t ldz) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int win[5];  // c_lo, c_hi, unused, unused, fits
  const int nb = (g.nt + 31) / 32;
  const int nqg = (nb + kTileQBlocks - 1) / kTileQBlocks;
  const int64_t ntiles = (int64_t)nb * nqg;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const Tab32 G = tab32(tv);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int bp = (int)(tile / nqg), bqg = (int)(tile % nqg);
    const int qb1 = min((bqg + 1) * kTileQBlocks, nb);
    if (qb1 <= bp) continue;  // only source blocks bq >= bp (one evaluation per unordered pair)
    const int qb0 = max(bqg * kTileQBlocks, bp);
    if (threadIdx.x == 0) {
      const float4 P = bsph[bp];
      float qx = 0.f, qy = 0.f, qz = 0.f;
      for (int b = qb0; b < qb1; ++b) {
        qx += bsph[b].x;
        qy += bsph[b].y;
        qz += bsph[b].z;
      }
      const float inv_n = 1.f / (float)(qb1 - qb0);
      qx *= inv_n;
      qy *= inv_n;
      qz *= inv_n;
      float rq = 0.f;
      for (int b = qb0; b < qb1; ++b) {
        const float dx = bsph[b].x - qx, dy = bsph[b].y - qy, dz = bsph[b].z - qz;
        rq = fmaxf(rq, sqrtf(dx * dx + dy * dy + dz * dz) + bsph[b].w);
      }
      const float dx = P.x - qx, dy = P.y - qy, dz = P.z - qz;
      const float D = sqrtf(dx * dx + dy * dy + dz * dz);
      const float mag = fmaxf(fmaxf(fabsf(P.x), fabsf(P.y)), fmaxf(fabsf(P.z), fmaxf(fmaxf(fabsf(qx), fabsf(qy)), fabsf(qz))));
      const float slack = 1e-5f * (D + P.w + rq + mag);
      const float lo = D - P.w - rq - slack, hi = D + P.w + rq + slack;
      const int n_lat = tv.n_lat;
      const int c_lo = max(lat_pos(G, lo * G.xscale).i - 2, 0);
      const int c_hi = min(lat_pos(G, hi * G.xscale).i + 2, n_lat - 1);
      win[0] = c_lo;
      win[1] = c_hi;
      win[4] = (int64_t)(c_hi - c_lo + 1) * 20 + 16 <= kWinBytes;
    }
    __syncthreads();
    Tab32 T = G;
    const bool staged = win[4] != 0;
    if (staged) {  // the window's (c0, c1) records and c2 words
      const int c_lo = win[0], c_hi = win[1];
      const int nc = c_hi - c_lo + 1;
      float4* sa = reinterpret_cast<float4*>(smem);
      uint32_t* sc = reinterpret_cast<uint32_t*>(sa + nc);
      for (int i = threadIdx.x; i < nc; i += blockDim.x) {
        sa[i] = G.la[c_lo + i];
        sc[i] = G.lc[c_lo + i];
      }
      __syncthreads();
      T.la = sa - c_lo;
      T.lc = sc - c_lo;
      T.vmin = kLatMagic + (float)c_lo;
      T.vmax = kLatMagic + (float)c_hi;
      const uint32_t mb = (uint32_t)__float_as_int(kLatMagic) + (uint32_t)c_lo;
      T.sa_off = (uint32_t)__cvta_generic_to_shared(sa) - mb * 16u;
      T.sc_off = (uint32_t)__cvta_generic_to_shared(sc) - mb * 4u;
    }
    const int ntask = 32 * (qb1 - qb0);
    for (int task = warp; task < ntask; task += nw) {
      const int p = bp * 32 + task / (qb1 - qb0);
      const int q0 = (qb0 + task % (qb1 - qb0)) * 32;
      if (p >= g.nt) continue;
      if (staged) regular_task32<M, kLagrange, KR, true>(g, T, K, DenseUpper{Z, ldz}, p, q0, lane);
      else regular_task32<M, kLagrange, KR, false>(g, T, K, DenseUpper{Z, ldz}, p, q0, lane);
    }
    __syncthreads();
  }
}

}  // namespace

template <int M, int MODE, bool KR>
cudaError_t launch_regular32_table(const TabView& tv, const GeoView& g, const RegK& K, float2* Z, int64_t ldz,
                                   cudaStream_t s) {
  const size_t smem = tv.smem32_bytes(MODE == kLagrange ? 3 : 1);
  int dev = 0, max_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // (list entries pack q << 6: fewer than 2^25 triangles)
  if (smem <= (size_t)max_optin && g.nt < (1 << 25)) {
    auto kern = k_fill_regular32<M, MODE, true, KR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, smem_block<M>(), smem);
    int64_t blocks = std::min<int64_t>(pair_grid(g, 2 * std::max(per_sm, 1)), (int64_t)sm_count() * std::max(per_sm, 1));
    // the Green lattice's flagged-pair lists: each CTA's count, then its
    // share of the entries (without the mesh's list, the table is read
    // through L1 with the corrections in the loop)
    blocks = std::min<int64_t>(blocks, kFixCounts);
    if constexpr (MODE != kLagrange) {
      kern<<<(unsigned)blocks, smem_block<M>(), smem, s>>>(g, tv, K, Z, ldz, 0u);
    } else if (g.fix && g.fix_cap > kFixCounts / 2) {
      const int64_t cap = std::min<int64_t>((g.fix_cap - kFixCounts / 2) / blocks, 0xFFFFFFFFll);
      kern<<<(unsigned)blocks, smem_block<M>(), smem, s>>>(g, tv, K, Z, ldz, (unsigned)cap);
      auto fix = k_fix_regular32<M, MODE, KR>;
      e = cudaFuncSetAttribute(fix, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      fix<<<(unsigned)blocks, smem_block<M>(), smem, s>>>(g, tv, K, Z, ldz, (unsigned)cap);
    } else {
      k_fill_regular32<M, MODE, false, KR><<<(unsigned)pair_grid(g, 4), kThreads, 0, s>>>(g, tv, K, Z, ldz, 0u);
    }
  } else if (MODE == kLagrange && g.bsph) {
    cudaError_t e =
        cudaFuncSetAttribute(k_fill_regular32_win<M, KR>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWinBytes);
    if (e != cudaSuccess) return e;
    k_fill_regular32_win<M, KR><<<(unsigned)sm_count(), 512, kWinBytes, s>>>(g, tv, g.bsph, K, Z, ldz);
  } else {
    int64_t blocks = pair_grid(g, 4);
    k_fill_regular32<M, MODE, false, KR><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, K, Z, ldz, 0u);
  }
  return cudaGetLastError();
}

template <int M>
cudaError_t launch_regular32(const GeoView& g, const TabView* table, bool from_exp, const RegK& K, float2* Z,
                             int64_t ldz, cudaStream_t s) {
  if (!table) {
    TabView tv{};
    if (M <= 4) {
      k_fill_regular32<M, kDirect, false, false><<<(unsigned)sm_count(), smem_block<M>(), 0, s>>>(g, tv, K, Z, ldz,
                                                                                                  0u);
    } else {
      int64_t blocks = pair_grid(g, 4);
      k_fill_regular32<M, kDirect, false, false><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, K, Z, ldz, 0u);
    }
    return cudaGetLastError();
  }
  const bool kr = table->xscale32 != 1.f;
  if (from_exp)
    return kr ? launch_regular32_table<M, kExpOverR, true>(*table, g, K, Z, ldz, s)
              : launch_regular32_table<M, kExpOverR, false>(*table, g, K, Z, ldz, s);
  return kr ? launch_regular32_table<M, kLagrange, true>(*table, g, K, Z, ldz, s)
            : launch_regular32_table<M, kLagrange, false>(*table, g, K, Z, ldz, s);
}

cudaError_t launch_fill_regular(const GeoView& g, const TabView* table, bool from_exp, double green_scale,
                                int precision, double k, double eta, void* Z, int64_t ldz, cudaStream_t s) {
  const double scale = k * eta / (4.0 * kPi) * (table && !from_exp ? green_scale : 1.0);
  TabView tv{};
  if (table) tv = *table;
  if (precision == GF_FP64) {
    int64_t blocks = pair_grid(g, 4);
    const double ik2 = 1.0 / (k * k);
    if (!table)
      k_fill_regular64<kDirect><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, k, scale, ik2, (double2*)Z, ldz);
    else if (from_exp)
      k_fill_regular64<kExpOverR><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, k, scale, ik2, (double2*)Z, ldz);
    else
      k_fill_regular64<kLagrange><<<(unsigned)blocks, kThreads, 0, s>>>(g, tv, k, scale, ik2, (double2*)Z, ldz);
    return cudaGetLastError();
  }
  const RegK K = reg_consts(k, scale);
  float2* Z32 = (float2*)Z;
  // each unordered pair into its test triangle's rows (launch_mirror32 adds
  // the transpose)
  cudaError_t e;
  switch (g.m) {
    case 1: e = launch_regular32<1>(g, table, from_exp, K, Z32, ldz, s); break;
    case 3: e = launch_regular32<3>(g, table, from_exp, K, Z32, ldz, s); break;
    case 4: e = launch_regular32<4>(g, table, from_exp, K, Z32, ldz, s); break;
    case 6: e = launch_regular32<6>(g, table, from_exp, K, Z32, ldz, s); break;
    case 7: e = launch_regular32<7>(g, table, from_exp, K, Z32, ldz, s); break;
    default: return cudaErrorInvalidValue;
  }
  return e;
}

}  // namespace gf
