// Staged block products.  The stored values and column indices of a tile of
// consecutive block rows are contiguous in the slab layout, so one bulk
// asynchronous copy each (cp.async.bulk, completion counted in bytes on an
// mbarrier) brings a whole tile into shared memory.  A persistent CTA keeps
// `stages` tiles in flight: while its lanes multiply the tile of one stage
// (values and indices from shared memory, source-vector gathers through
// L1/L2), the copies of the next tiles stream from HBM.
//
// Tiles are whole runs of block rows with at most cap blocks each, cut
// greedily at set-up (cap = what one stage holds).  Every copy starts and
// ends on a 16-byte line (the arrays carry 64 bytes of slack past their
// end, see DeviceArena), and the lanes index the tile from the start's
// offset inside its first line.
//
// Every wait on an mbarrier is bounded: after kWaitLimit polls the CTA
// records a timeout in a device status word, waits (again bounded) for its
// copies still in flight and returns; the host reads the status after the
// solve and reports SCR_DEVICE_TIMEOUT.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "epilogue.cuh"
#include "kernels.h"

namespace scr {
namespace {

constexpr int kStThreads = 256;
constexpr int kMaxStages = 4;
constexpr long long kWaitLimit = 1LL << 22;  // mbarrier polls before a stage counts as lost

__device__ int g_staged_status;  // 0 ok; 1 a stage wait ran out; 2 a tile exceeded its stage

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// global -> shared bulk copy; dst, src and bytes are multiples of 16
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(static_cast<unsigned long long>(__cvta_generic_to_global(src))), "r"(bytes), "r"(bar)
               : "memory");
}

template <typename VT>
struct StagedMatrix {
  const int* rp;
  const int* col;
  const VT* val;
  const int* tiles;
  int ntiles, stage_v, stage_c, nstages;
};

// one scalar row from the staged tile: sc = the row's column indices, sv =
// its k*BC values (slab layout); the G lanes of the group take the blocks in
// turn (the order of the scalar-row kernel), U blocks per lane per pass so
// that U source gathers are in flight
template <int BC, int NRHS, int G, typename VT, typename XT, typename AT>
__device__ __forceinline__ void staged_row(const int* sc, const VT* sv, const XT* __restrict__ x, int k, int lane,
                                           AT (&acc)[NRHS]) {
  constexpr int U = 4;
  for (int t0 = lane; t0 < k; t0 += G * U) {
    int cidx[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = t0 + u * G;
      cidx[u] = t < k ? sc[t] : -1;
    }
    AT xv[U][BC][NRHS];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = cidx[u] >= 0;
      const long long xb = (long long)(ok ? cidx[u] : 0) * BC * NRHS;
#pragma unroll
      for (int c = 0; c < BC; ++c)
#pragma unroll
        for (int h = 0; h < NRHS; ++h) xv[u][c][h] = ok ? (AT)__ldg(x + xb + c * NRHS + h) : (AT)0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (cidx[u] < 0) continue;
      const VT* vt = sv + (t0 + u * G) * BC;
#pragma unroll
      for (int c = 0; c < BC; ++c) {
        const AT a = (AT)vt[c];
#pragma unroll
        for (int h = 0; h < NRHS; ++h) acc[h] = fma(a, xv[u][c][h], acc[h]);
      }
    }
  }
}

template <int BR, int BC, int NRHS, int G, typename VT, typename XT, Epi E>
__global__ void __launch_bounds__(kStThreads) k_spmv_staged(StagedMatrix<VT> M, const XT* __restrict__ x,
                                                           Epilogue<XT, E> epi) {
  using AT = XT;
  constexpr int BS = BR * BC;
  constexpr long long VB = (long long)BS * sizeof(VT);  // bytes per stored block
  constexpr int kGroups = kStThreads / G;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) unsigned long long bars[kMaxStages];
  __shared__ int bad[kMaxStages];
  const int tid = threadIdx.x, lane = tid % G;
  const int nst = M.nstages;
  const int stride = M.stage_v + M.stage_c;
  const int my_tiles = M.ntiles > (int)blockIdx.x ? (M.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  // thread 0: start the copies of this CTA's j-th tile into stage j % nst
  auto issue = [&](int j) {
    const int t = blockIdx.x + j * gridDim.x;
    const int st = j % nst;
    const uint32_t bar = smem_addr(&bars[st]);
    const int lo = __ldg(M.tiles + t), hi = __ldg(M.tiles + t + 1);
    const long long b0 = __ldg(M.rp + lo), b1 = __ldg(M.rp + hi);
    const long long va = (b0 * VB) & ~15LL, vb = (b1 * VB + 15) & ~15LL;
    const long long ca = (b0 * 4) & ~15LL, cb = (b1 * 4 + 15) & ~15LL;
    if (vb - va > M.stage_v || cb - ca > M.stage_c) {
      bad[st] = 1;
      atomicMax(&g_staged_status, 2);
      mbar_arrive(bar);
      return;
    }
    bad[st] = 0;
    const uint32_t nv = (uint32_t)(vb - va), nc = (uint32_t)(cb - ca);
    if (nv + nc == 0) {
      mbar_arrive(bar);
      return;
    }
    mbar_arrive_expect_tx(bar, nv + nc);
    unsigned char* base = smem + (size_t)st * stride;
    if (nv) bulk_load(smem_addr(base), reinterpret_cast<const unsigned char*>(M.val) + va, nv, bar);
    if (nc) bulk_load(smem_addr(base + M.stage_v), reinterpret_cast<const unsigned char*>(M.col) + ca, nc, bar);
  };

  if (tid == 0) {
    for (int st = 0; st < nst; ++st) mbar_init(smem_addr(&bars[st]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int j = 0; j < nst && j < my_tiles; ++j) issue(j);

  int j = 0;
  bool lost = false;
  for (; j < my_tiles; ++j) {
    const int t = blockIdx.x + j * gridDim.x;
    const int st = j % nst;
    const bool ok = mbar_wait_bounded(smem_addr(&bars[st]), (uint32_t)((j / nst) & 1));
    if (__syncthreads_or(!ok)) {
      lost = true;
      break;
    }
    if (!bad[st]) {
      const int lo = __ldg(M.tiles + t), hi = __ldg(M.tiles + t + 1);
      const int b0 = __ldg(M.rp + lo);
      const unsigned char* base = smem + (size_t)st * stride;
      const VT* sv = reinterpret_cast<const VT*>(base + (((long long)b0 * VB) & 15));
      const int* sc = reinterpret_cast<const int*>(base + M.stage_v + (((long long)b0 * 4) & 15));
      const int nrow = (hi - lo) * BR;
      // q0 is uniform over the CTA, so every lane of a warp runs the same
      // passes and the shuffles below see the whole warp
      for (int q0 = 0; q0 < nrow; q0 += kGroups) {
        const int q = q0 + tid / G;
        AT acc[NRHS];
#pragma unroll
        for (int h = 0; h < NRHS; ++h) acc[h] = (AT)0;
        if (q < nrow) {
          const int bi = q / BR, r = q - bi * BR;
          const int s = __ldg(M.rp + lo + bi), k = __ldg(M.rp + lo + bi + 1) - s;
          staged_row<BC, NRHS, G, VT, XT, AT>(sc + (s - b0), sv + (long long)(s - b0) * BS + (long long)r * k * BC,
                                               x, k, lane, acc);
        }
        if constexpr (G > 1) {
#pragma unroll
          for (int h = 0; h < NRHS; ++h)
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) acc[h] += __shfl_xor_sync(0xffffffffu, acc[h], off, G);
        }
        if (q < nrow && lane == 0) {
          const long long o = (long long)lo * BR + q;
#pragma unroll
          for (int h = 0; h < NRHS; ++h) epi(o * NRHS + h, o, acc[h]);
        }
      }
    }
    __syncthreads();  // every lane is done with stage st
    if (tid == 0 && j + nst < my_tiles) issue(j + nst);
  }
  if (lost) {
    // the copies of tiles j .. j + nst - 1 may still be in flight: wait for
    // them (bounded) before the CTA's shared memory is released
    if (tid == 0) {
      atomicMax(&g_staged_status, 1);
      for (int jj = j; jj < j + nst && jj < my_tiles; ++jj)
        mbar_wait_bounded(smem_addr(&bars[jj % nst]), (uint32_t)((jj / nst) & 1));
    }
    __syncthreads();
  }
}

template <int BR, int BC, int NRHS, int G, typename VT, typename XT, Epi E>
void launch_staged(const DBsr<VT>& M, const XT* x, XT* y, const EpiArgs& e, cudaStream_t s) {
  const Epilogue<XT, E> epi = make_epilogue<XT, E>(x, y, e);
  StagedMatrix<VT> S{M.rp, M.col, M.val, M.tiles, M.ntiles, M.stage_v, M.stage_c, M.stages};
  const int smem = M.stages * (M.stage_v + M.stage_c);
  auto kern = k_spmv_staged<BR, BC, NRHS, G, VT, XT, E>;
  // per instantiation and device: the largest dynamic shared-memory size
  // configured so far (the attribute only ever grows, so every size up to it
  // stays launchable) and the resident CTAs per SM at each size
  static std::mutex mu;
  static std::map<int, int> configured;                    // device -> attribute value
  static std::map<std::pair<int, int>, int> per_sm_cache;  // (device, smem) -> CTAs per SM
  int dev = 0;
  SCR_CUDA(cudaGetDevice(&dev));
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    int& cfg = configured[dev];
    if (smem > cfg) {
      SCR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      cfg = smem;
    }
    auto it = per_sm_cache.find({dev, smem});
    if (it == per_sm_cache.end()) {
      SCR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kStThreads, smem));
      per_sm = std::max(1, per_sm);
      per_sm_cache[{dev, smem}] = per_sm;
    } else {
      per_sm = it->second;
    }
  }
  const int grid = std::min<long long>(M.ntiles, (long long)per_sm * sm_count());
  kern<<<grid, kStThreads, smem, s>>>(S, x, epi);
  SCR_LAUNCH();
  counters().staged++;
}

template <int BR, int BC, int NRHS, int G, typename VT, typename XT>
void staged_e(const DBsr<VT>& M, const XT* x, XT* y, const EpiArgs& e, cudaStream_t s) {
  switch (e.kind) {
    case Epi::Set: launch_staged<BR, BC, NRHS, G, VT, XT, Epi::Set>(M, x, y, e, s); break;
    case Epi::Axpby: launch_staged<BR, BC, NRHS, G, VT, XT, Epi::Axpby>(M, x, y, e, s); break;
    case Epi::Resid: launch_staged<BR, BC, NRHS, G, VT, XT, Epi::Resid>(M, x, y, e, s); break;
    case Epi::Jacobi: launch_staged<BR, BC, NRHS, G, VT, XT, Epi::Jacobi>(M, x, y, e, s); break;
    case Epi::ScaledSub: launch_staged<BR, BC, NRHS, G, VT, XT, Epi::ScaledSub>(M, x, y, e, s); break;
    case Epi::ChebFirst: launch_staged<BR, BC, NRHS, G, VT, XT, Epi::ChebFirst>(M, x, y, e, s); break;
    case Epi::ChebStep: launch_staged<BR, BC, NRHS, G, VT, XT, Epi::ChebStep>(M, x, y, e, s); break;
  }
}

template <int BR, int BC, int NRHS, typename VT, typename XT>
void staged_g(int G, const DBsr<VT>& M, const XT* x, XT* y, const EpiArgs& e, cudaStream_t s) {
  switch (G) {
    case 1: staged_e<BR, BC, NRHS, 1, VT, XT>(M, x, y, e, s); break;
    case 2: staged_e<BR, BC, NRHS, 2, VT, XT>(M, x, y, e, s); break;
    case 4: staged_e<BR, BC, NRHS, 4, VT, XT>(M, x, y, e, s); break;
    default: staged_e<BR, BC, NRHS, 8, VT, XT>(M, x, y, e, s); break;
  }
}

}  // namespace

bool staged_shape_supported(int br, int bc, int nrhs) {
  return (br == 3 && bc == 3 && nrhs == 1) || (br == 1 && bc == 1 && (nrhs == 1 || nrhs == 3));
}

template <typename VT, typename XT>
bool spmv_staged(int G, const DBsr<VT>& M, const XT* x, XT* y, int nrhs, const EpiArgs& e, cudaStream_t s) {
  if (!M.tiles || M.ntiles <= 0 || !staged_shape_supported(M.br, M.bc, nrhs)) return false;
  if (M.br == 3) staged_g<3, 3, 1, VT, XT>(G, M, x, y, e, s);
  else if (nrhs == 1) staged_g<1, 1, 1, VT, XT>(G, M, x, y, e, s);
  else staged_g<1, 1, 3, VT, XT>(G, M, x, y, e, s);
  return true;
}
template bool spmv_staged<double, double>(int, const DBsr<double>&, const double*, double*, int, const EpiArgs&,
                                          cudaStream_t);
template bool spmv_staged<float, float>(int, const DBsr<float>&, const float*, float*, int, const EpiArgs&,
                                        cudaStream_t);

template <typename VT>
void build_staged_plan(DBsr<VT>& M, int nrhs, DeviceArena& a, cudaStream_t s, int stage_kb, int stages) {
  M.tiles = nullptr;
  M.ntiles = 0;
  if (M.nbr == 0 || M.nnzb < kStagedMinBlocks || !staged_shape_supported(M.br, M.bc, nrhs)) return;
  if ((reinterpret_cast<uintptr_t>(M.val) & 15) || (reinterpret_cast<uintptr_t>(M.col) & 15)) return;
  stages = std::min(std::max(stages, 2), kMaxStages);
  // all stages of a CTA within 200 KiB of shared memory
  stage_kb = std::min(std::max(stage_kb, 4), std::min(96, 200 / stages - 2));
  const long long vb = (long long)M.br * M.bc * sizeof(VT);
  const long long cap = ((long long)stage_kb * 1024 - 64) / (vb + 4);  // blocks per stage
  // greedy tiles of whole block rows with at most cap blocks each
  std::vector<int> rp(M.nbr + 1);
  SCR_CUDA(cudaMemcpyAsync(rp.data(), M.rp, sizeof(int) * (M.nbr + 1), cudaMemcpyDeviceToHost, s));
  SCR_CUDA(cudaStreamSynchronize(s));
  std::vector<int> tiles{0};
  for (int i = 0; i < M.nbr; ++i) {
    const long long k = rp[i + 1] - rp[i];
    if (k > cap) return;  // a row longer than a stage: plain kernel
    if (rp[i + 1] - rp[tiles.back()] > cap) tiles.push_back(i);
  }
  tiles.push_back(M.nbr);
  const int ntiles = (int)tiles.size() - 1;
  int* dt = a.alloc<int>(tiles.size());
  SCR_CUDA(cudaMemcpyAsync(dt, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice, s));
  SCR_CUDA(cudaStreamSynchronize(s));
  M.tiles = dt;
  M.ntiles = ntiles;
  M.stage_v = (int)(((cap * vb + 32) + 15) & ~15LL);
  M.stage_c = (int)(((cap * 4 + 32) + 15) & ~15LL);
  M.stages = stages;
}
template void build_staged_plan<double>(DBsr<double>&, int, DeviceArena&, cudaStream_t, int, int);
template void build_staged_plan<float>(DBsr<float>&, int, DeviceArena&, cudaStream_t, int, int);

int staged_status_take(cudaStream_t s) {
  int v = 0;
  SCR_CUDA(cudaMemcpyFromSymbolAsync(&v, g_staged_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  SCR_CUDA(cudaStreamSynchronize(s));
  if (v) {
    const int z = 0;
    SCR_CUDA(cudaMemcpyToSymbolAsync(g_staged_status, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    SCR_CUDA(cudaStreamSynchronize(s));
  }
  return v;
}

}  // namespace scr
