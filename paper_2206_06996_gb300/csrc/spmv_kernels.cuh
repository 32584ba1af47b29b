// Product kernels with G lanes per scalar row and their launch dispatch,
// shared by the translation units that instantiate them: spmv.cu (one and
// three right-hand sides) and spmm.cu (eight right-hand sides, the block
// product of the multi-right-hand-side solve).
#pragma once
#include <cuda_bf16.h>

#include "epilogue.cuh"
#include "kernels.h"

#ifndef SCR_SPMV_MINBLOCKS
#define SCR_SPMV_MINBLOCKS 1
#endif
// blocks each lane of a product keeps in flight (FP64 rows use half)
#ifndef SCR_SPMV_BATCH
#define SCR_SPMV_BATCH 4
#endif

namespace scr {

// Programmatic dependent launch (option pdl): a product kernel lets the next
// kernel of the stream start as soon as all of its CTAs are running
// (griddepcontrol.launch_dependents), and, before it reads anything an
// earlier kernel wrote, waits for that kernel to complete with its memory
// visible (griddepcontrol.wait).  Between the two it only prefetches its own
// rows of the stored matrix into L2 (read-only data), so the matrix stream
// of one product overlaps the tail of the previous one.  Launched without
// the attribute, both instructions return at once.
__device__ __forceinline__ void pdl_allow_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait_prev() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ------------------------------------------------------------ SpMV
// accumulate one scalar row r of block row i of M into acc[h]; the lanes of
// a G-group take the row's blocks in turn (BC values each, contiguous in the
// slab layout) so every stored value costs one multiply-add
template <int BC, int NRHS, int G, typename VT, typename XT, typename AT>
__device__ __forceinline__ void scalar_row_accum(const int* __restrict__ rp, const int* __restrict__ col,
                                                 const VT* __restrict__ val, const XT* __restrict__ x, int BR,
                                                 int i, int r, int lane, AT (&acc)[NRHS]) {
  // U blocks per lane in flight: the column indices are loaded first, then
  // every gather and value of the batch, then the multiply-adds, so a lane
  // keeps U independent load chains outstanding instead of one
  // measured on the 616k-node tube: FP64 rows gain from the lower register
  // count of two blocks in flight, FP32 rows from four
  // (with 4 or more right-hand sides a block already brings NRHS gathers per
  // value: one block per lane pass keeps the registers in bounds)
  constexpr int U = NRHS > 3 ? 1 : (sizeof(VT) == 8 ? SCR_SPMV_BATCH / 2 : SCR_SPMV_BATCH);
  const int s = __ldg(rp + i), k = __ldg(rp + i + 1) - s;
  const VT* vr = val + (long long)s * BR * BC + (long long)r * k * BC;
  const int* cr = col + s;
  for (int t0 = lane; t0 < k; t0 += G * U) {
    int cidx[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = t0 + u * G;
      cidx[u] = t < k ? __ldg(cr + t) : -1;
    }
    AT a[U][BC], xv[U][BC][NRHS];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = t0 + u * G;
      const bool ok = cidx[u] >= 0;
      const long long xb = (long long)(ok ? cidx[u] : 0) * BC * NRHS;
#pragma unroll
      for (int c = 0; c < BC; ++c) {
        a[u][c] = ok ? (AT)__ldg(vr + t * BC + c) : (AT)0;
#pragma unroll
        for (int h = 0; h < NRHS; ++h) xv[u][c][h] = ok ? (AT)__ldg(x + xb + c * NRHS + h) : (AT)0;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int c = 0; c < BC; ++c)
#pragma unroll
        for (int h = 0; h < NRHS; ++h)
          if (cidx[u] >= 0) acc[h] = fma(a[u][c], xv[u][c][h], acc[h]);
  }
}

// L2 prefetch (cp.async.bulk.prefetch.L2) of the stored values and column
// indices that the CTA with index cta (256 threads, 256 / G scalar rows)
// will read.  The range is cut to whole 16-byte lines inside it: the first
// line may start up to 15 bytes before the range (the same line as a valid
// byte), the last partial line is left out, so no line outside the arrays
// is named.
template <int BR, int BC, int G, typename VT>
__device__ __forceinline__ void l2_prefetch_rows(const int* __restrict__ rp, const int* __restrict__ col,
                                                 const VT* __restrict__ val, int nbr, long long cta) {
  const long long nrows = (long long)nbr * BR;
  const long long o0 = cta * (256 / G);
  if (o0 >= nrows) return;
  const long long o1 = o0 + 256 / G < nrows ? o0 + 256 / G : nrows;
  const long long b0 = __ldg(rp + o0 / BR), b1 = __ldg(rp + (o1 - 1) / BR + 1);
  const unsigned long long v0 = __cvta_generic_to_global(val + b0 * BR * BC) & ~15ULL;
  const unsigned long long v1 = __cvta_generic_to_global(val + b1 * BR * BC) & ~15ULL;
  const unsigned long long c0 = __cvta_generic_to_global(col + b0) & ~15ULL;
  const unsigned long long c1 = __cvta_generic_to_global(col + b1) & ~15ULL;
  if (v1 > v0)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(v0), "r"((unsigned)(v1 - v0)) : "memory");
  if (c1 > c0)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c0), "r"((unsigned)(c1 - c0)) : "memory");
}

template <int BR, int BC, int NRHS, int G, typename VT, typename XT, typename AT, Epi E>
__global__ void __launch_bounds__(256, SCR_SPMV_MINBLOCKS) k_spmv(int nbr, const int* __restrict__ rp,
                                                                 const int* __restrict__ col,
                                              const VT* __restrict__ val, const XT* __restrict__ x,
                                              Epilogue<XT, E> epi, int pf) {
  const long long o = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / G;  // scalar row
  const int lane = threadIdx.x % G;
  const long long nrows = (long long)nbr * BR;
  const int ahead = pf < 0 ? -pf - 1 : pf;
  pdl_allow_next();
  if (pf < 0 && threadIdx.x == 0) l2_prefetch_rows<BR, BC, G, VT>(rp, col, val, nbr, blockIdx.x);
  pdl_wait_prev();
  if (ahead > 0 && threadIdx.x == 0) l2_prefetch_rows<BR, BC, G, VT>(rp, col, val, nbr, blockIdx.x + (long long)ahead);
  const bool active = o < nrows;  // inactive lanes still join the shuffles
  AT acc[NRHS];
#pragma unroll
  for (int h = 0; h < NRHS; ++h) acc[h] = (AT)0;
  if (active) {
    const int i = (int)(o / BR), r = (int)(o - (long long)i * BR);
    scalar_row_accum<BC, NRHS, G>(rp, col, val, x, BR, i, r, lane, acc);
  }
  if constexpr (G > 1) {
#pragma unroll
    for (int h = 0; h < NRHS; ++h) {
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1) acc[h] += __shfl_xor_sync(0xffffffffu, acc[h], off, G);
    }
  }
  if (active && lane == 0) {
#pragma unroll
    for (int h = 0; h < NRHS; ++h) epi(o * NRHS + h, o, acc[h]);
  }
}

// G lanes per BLOCK row: each lane takes blocks t = lane, lane+G, ... and
// accumulates all BR scalar rows, so the column index and the BC source
// values of a block are loaded once for its BR x BC multiply-adds; the
// BR*NRHS sums are combined over the G lanes and written by distinct lanes.
template <int BR, int BC, int NRHS, int G, typename VT, typename XT, typename AT, Epi E>
__global__ void __launch_bounds__(256) k_spmv_brow(int nbr, const int* __restrict__ rp, const int* __restrict__ col,
                                                   const VT* __restrict__ val, const XT* __restrict__ x,
                                                   Epilogue<XT, E> epi) {
  const long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / G;  // block row
  const int lane = threadIdx.x % G;
  const bool active = i < nbr;
  AT acc[BR][NRHS];
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int h = 0; h < NRHS; ++h) acc[r][h] = (AT)0;
  if (active) {
    const int s = __ldg(rp + i), k = __ldg(rp + i + 1) - s;
    const VT* v0 = val + (long long)s * BR * BC;
    const int* cr = col + s;
#pragma unroll 2
    for (int t = lane; t < k; t += G) {
      const long long xb = (long long)__ldg(cr + t) * BC * NRHS;
      AT xv[BC][NRHS];
#pragma unroll
      for (int c = 0; c < BC; ++c)
#pragma unroll
        for (int h = 0; h < NRHS; ++h) xv[c][h] = (AT)__ldg(x + xb + c * NRHS + h);
#pragma unroll
      for (int r = 0; r < BR; ++r) {
        const VT* vt = v0 + (long long)r * k * BC + t * BC;
#pragma unroll
        for (int c = 0; c < BC; ++c) {
          const AT a = (AT)__ldg(vt + c);
#pragma unroll
          for (int h = 0; h < NRHS; ++h) acc[r][h] = fma(a, xv[c][h], acc[r][h]);
        }
      }
    }
  }
  if constexpr (G > 1) {
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int h = 0; h < NRHS; ++h)
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) acc[r][h] += __shfl_xor_sync(0xffffffffu, acc[r][h], off, G);
  }
  if (active) {
#pragma unroll
    for (int q = 0; q < BR * NRHS; ++q) {
      if (q % G != lane) continue;
      const int r = q / NRHS, h = q - r * NRHS;
      const long long o = i * BR + r;
      epi(o * NRHS + h, o, acc[r][h]);
    }
  }
}

// ------------------------------------------------------------ 16-byte products
// Products on the padded copy of DBsr::vdesc.  Each lane takes a chunk of V
// = 16 / sizeof(VT) blocks (3x3) or entries (1x1) at a time and loads it
// with 16-byte vector loads: for a 3x3 chunk one index vector (V column
// indices) and three value vectors per scalar row, against V column loads
// and 3 V value loads per scalar row in the scalar-row kernel.
// The stored values and indices go through the read-only path with plain
// 16-byte loads (the padded copy starts every chunk on a 16-byte boundary).
// Measured inside the solve on the 616k-node tube (FP32, 4 lanes per block
// row): 115.5 us per level-0 product with plain loads, 127 us with
// L1::no_allocate / L2::256B hints on the value loads: a lane's three value
// vectors of one scalar row share sectors, which L1 then has to keep.
template <typename VT>
__device__ __forceinline__ void ldg16(const VT* p, VT* a) {
  if constexpr (sizeof(VT) == 4) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    a[0] = v.x, a[1] = v.y, a[2] = v.z, a[3] = v.w;
  } else {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    a[0] = v.x, a[1] = v.y;
  }
}
template <int U>
__device__ __forceinline__ void ldg_idx(const int* p, int* c) {
  if constexpr (U == 4) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(p));
    c[0] = v.x, c[1] = v.y, c[2] = v.z, c[3] = v.w;
  } else {
    const int2 v = __ldg(reinterpret_cast<const int2*>(p));
    c[0] = v.x, c[1] = v.y;
  }
}

// L2 prefetch (cp.async.bulk.prefetch.L2) of the padded values and column
// slots of the block rows [i0, i1) of a padded copy (3x3: int4 descriptors;
// 1x1: int2, values and slots sharing their starts).  Whole 16-byte lines
// inside the allocations only.
template <typename VT, bool SQ3>
__device__ __forceinline__ void l2_prefetch_vec(const void* desc, const int* col, const VT* val, long long i0,
                                                long long i1) {
  long long c0, c1, v0, v1;
  if constexpr (SQ3) {
    const int4 a = __ldg(static_cast<const int4*>(desc) + i0), b = __ldg(static_cast<const int4*>(desc) + i1 - 1);
    constexpr int V = 16 / (int)sizeof(VT);
    c0 = a.x, c1 = b.x + (b.y + V - 1) / V * V;
    v0 = a.z, v1 = b.z + 3LL * b.w;
  } else {
    constexpr int V = 16 / (int)sizeof(VT);
    const int2 a = __ldg(static_cast<const int2*>(desc) + i0), b = __ldg(static_cast<const int2*>(desc) + i1 - 1);
    c0 = v0 = a.x;
    c1 = v1 = b.x + (b.y + V - 1) / V * V;
  }
  // runs start on 16-byte boundaries except FP64 column slots (8 bytes): round
  // down the start and up the end (the arrays carry 16 entries of slack)
  const unsigned long long vb = __cvta_generic_to_global(val + v0) & ~15ULL;
  const unsigned long long ve = (__cvta_generic_to_global(val + v1) + 15) & ~15ULL;
  const unsigned long long cb = __cvta_generic_to_global(col + c0) & ~15ULL;
  const unsigned long long ce = (__cvta_generic_to_global(col + c1) + 15) & ~15ULL;
  if (ve > vb)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(vb), "r"((unsigned)(ve - vb)) : "memory");
  if (ce > cb)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(cb), "r"((unsigned)(ce - cb)) : "memory");
}

// 3x3 blocks, one right-hand side: G lanes per block row, each lane takes
// chunks of U = V blocks (3 U values per scalar row, i.e. three 16-byte
// loads) in turn and accumulates all three scalar rows, so a block's column
// index and its three source values are loaded once for its 9 multiply-adds.
// The three row sums are combined over the G lanes and written by lanes 0,
// 1, 2 (mod G).
template <int G, typename VT, typename XT, Epi E>
__global__ void __launch_bounds__(256) k_spmv_vec33(int nbr, const int4* __restrict__ desc, const int* __restrict__ col,
                                                    const VT* __restrict__ val, const XT* __restrict__ x,
                                                    Epilogue<XT, E> epi, int pf) {
  constexpr int V = 16 / (int)sizeof(VT);
  constexpr int U = V;
  const long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / G;
  const int lane = threadIdx.x % G;
  const int ahead = pf < 0 ? -pf - 1 : pf;
  pdl_allow_next();
  if (pf < 0 && threadIdx.x == 0) {
    const long long i0 = blockIdx.x * (long long)(256 / G);
    if (i0 < nbr) l2_prefetch_vec<VT, true>(desc, col, val, i0, i0 + 256 / G < nbr ? i0 + 256 / G : nbr);
  }
  pdl_wait_prev();
  if (ahead > 0 && threadIdx.x == 0) {
    const long long i0 = (blockIdx.x + (long long)ahead) * (256 / G);
    if (i0 < nbr) l2_prefetch_vec<VT, true>(desc, col, val, i0, i0 + 256 / G < nbr ? i0 + 256 / G : nbr);
  }
  const bool active = i < nbr;  // inactive lanes still join the shuffles
  XT acc[3] = {(XT)0, (XT)0, (XT)0};
  if (active) {
    const int4 d = __ldg(desc + i);
    const int k = d.y, rl = d.w;
    const int* __restrict__ cr = col + d.x;
    const VT* __restrict__ v0 = val + d.z;
    for (int j = lane * U; j < k; j += G * U) {
      const int m = k - j < U ? k - j : U;  // blocks of this chunk
      int c[U];
      ldg_idx<U>(cr + j, c);
      VT a[3][3 * U];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (q * V < 3 * m) {
            ldg16<VT>(v0 + (long long)r * rl + 3 * j + q * V, &a[r][q * V]);
          } else {
#pragma unroll
            for (int e = 0; e < V; ++e) a[r][q * V + e] = (VT)0;
          }
        }
      XT xv[U][3];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long xb = 3LL * (u < m ? c[u] : 0);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) xv[u][cc] = u < m ? (XT)__ldg(x + xb + cc) : (XT)0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
#pragma unroll
          for (int r = 0; r < 3; ++r)
            if (u < m) acc[r] = fma((XT)a[r][3 * u + cc], xv[u][cc], acc[r]);
    }
  }
  if constexpr (G > 1) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], off, G);
  }
  if (active) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
      if (r % G == lane) epi(3 * i + r, 3 * i + r, acc[r]);
  }
}

// 1x1 blocks, one right-hand side: G lanes per row, chunks of V entries
// (one 16-byte value load and one index load of V column indices).
template <int G, typename VT, typename XT, Epi E>
__global__ void __launch_bounds__(256) k_spmv_vec11(int nbr, const int2* __restrict__ desc, const int* __restrict__ col,
                                                    const VT* __restrict__ val, const XT* __restrict__ x,
                                                    Epilogue<XT, E> epi, int pf) {
  constexpr int V = 16 / (int)sizeof(VT);
  const long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / G;
  const int lane = threadIdx.x % G;
  const int ahead = pf < 0 ? -pf - 1 : pf;
  pdl_allow_next();
  if (pf < 0 && threadIdx.x == 0) {
    const long long i0 = blockIdx.x * (long long)(256 / G);
    if (i0 < nbr) l2_prefetch_vec<VT, false>(desc, col, val, i0, i0 + 256 / G < nbr ? i0 + 256 / G : nbr);
  }
  pdl_wait_prev();
  if (ahead > 0 && threadIdx.x == 0) {
    const long long i0 = (blockIdx.x + (long long)ahead) * (256 / G);
    if (i0 < nbr) l2_prefetch_vec<VT, false>(desc, col, val, i0, i0 + 256 / G < nbr ? i0 + 256 / G : nbr);
  }
  const bool active = i < nbr;
  XT acc = (XT)0;
  if (active) {
    const int2 d = __ldg(desc + i);
    const int k = d.y;
    const int* __restrict__ cr = col + d.x;
    const VT* __restrict__ vr = val + d.x;
    for (int j = lane * V; j < k; j += G * V) {
      const int m = k - j < V ? k - j : V;
      int c[V];
      VT a[V];
      ldg_idx<V>(cr + j, c);
      ldg16<VT>(vr + j, a);
      XT xv[V];
#pragma unroll
      for (int u = 0; u < V; ++u) xv[u] = u < m ? (XT)__ldg(x + c[u]) : (XT)0;
#pragma unroll
      for (int u = 0; u < V; ++u)
        if (u < m) acc = fma((XT)a[u], xv[u], acc);
    }
  }
  if constexpr (G > 1) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off, G);
  }
  if (active && lane == 0) epi(i, i, acc);
}

// sliced block-ELL product: one lane per block row, no cross-lane sums
template <int BR, int BC, int NRHS, typename VT, typename XT, Epi E>
__global__ void __launch_bounds__(256) k_sell_spmv(DSell<VT> S, const XT* __restrict__ x, Epilogue<XT, E> epi) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int c = (int)(g / kChunk), lane = (int)(g % kChunk);
  if (c >= S.nchunk) return;
  const int q = c * kChunk + lane;
  if (q >= S.nbr) return;
  const int i = __ldg(S.perm + q);
  const int c0 = __ldg(S.cptr + c), L = __ldg(S.cptr + c + 1) - c0;
  const long long base = (long long)c0 * kChunk;
  const int* __restrict__ cl = S.col + base + lane;
  const VT* __restrict__ vl = S.val + base * (BR * BC) + lane;
  using AT = XT;
  AT acc[BR][NRHS];
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int h = 0; h < NRHS; ++h) acc[r][h] = (AT)0;
#pragma unroll 2
  for (int t = 0; t < L; ++t) {
    const long long xb = (long long)__ldg(cl + (long long)t * kChunk) * BC * NRHS;
    AT xv[BC][NRHS];
#pragma unroll
    for (int cc = 0; cc < BC; ++cc)
#pragma unroll
      for (int h = 0; h < NRHS; ++h) xv[cc][h] = (AT)__ldg(x + xb + cc * NRHS + h);
    const VT* vt = vl + (long long)t * kChunk * (BR * BC);
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int cc = 0; cc < BC; ++cc) {
        const AT a = (AT)__ldg(vt + (r * BC + cc) * kChunk);
#pragma unroll
        for (int h = 0; h < NRHS; ++h) acc[r][h] = fma(a, xv[cc][h], acc[r][h]);
      }
  }
#pragma unroll
  for (int r = 0; r < BR; ++r) {
    const long long o = (long long)i * BR + r;
#pragma unroll
    for (int h = 0; h < NRHS; ++h) epi(o * NRHS + h, o, acc[r][h]);
  }
}

// CTAs ahead for the L2 prefetch of the scalar-row kernel (0: off) and the
// forced kernel code of every product (0: per matrix); defined in spmv.cu
extern int g_l2_prefetch;
// launch the product kernels with programmatic stream serialization (option pdl)
extern int g_pdl;

// kern<<<grid, blk, 0, s>>>(args...), with the programmatic-serialization
// attribute when g_pdl is set (the kernel then starts before its
// predecessor completes and waits for it in griddepcontrol.wait); the
// prefetch argument pf is passed negated under PDL, which makes the kernel
// prefetch its own rows before it waits
template <typename... KArgs, typename... Args>
inline void launch_product(void (*kern)(KArgs...), long long grid, int blk, cudaStream_t s, Args... args) {
  if (g_pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)blk);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SCR_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
  } else {
    kern<<<(unsigned)grid, blk, 0, s>>>(args...);
  }
}
// the kernels' prefetch argument: pf >= 0: pf CTAs ahead; pf < 0 (PDL): the
// CTA's own rows before the wait, then -pf - 1 CTAs ahead
inline int pf_arg() { return g_pdl ? -g_l2_prefetch - 1 : g_l2_prefetch; }

template <int BR, int BC, int NRHS, int G, typename VT, typename XT, typename AT, Epi E>
inline void launch_spmv_g(const DBsr<VT>& M, const XT* x, XT* y, const EpiArgs& e, cudaStream_t s) {
  const Epilogue<XT, E> epi = make_epilogue<XT, E>(x, y, e);
  const int blk = 256;
  bool done = false;
  if constexpr (sizeof(VT) >= 4 && NRHS == 1 && ((BR == 3 && BC == 3) || (BR == 1 && BC == 1))) {
    if (M.vdesc && code_of(M) >= 300) {
      if constexpr (BR == 3) {
        const long long threads = (long long)M.nbr * G;
        launch_product(k_spmv_vec33<G, VT, XT, E>, ceil_div(threads, blk), blk, s, M.nbr,
                       static_cast<const int4*>(M.vdesc), (const int*)M.vcol, (const VT*)M.vval, x, epi, pf_arg());
      } else {
        const long long threads = (long long)M.nbr * G;
        launch_product(k_spmv_vec11<G, VT, XT, E>, ceil_div(threads, blk), blk, s, M.nbr,
                       static_cast<const int2*>(M.vdesc), (const int*)M.vcol, (const VT*)M.vval, x, epi, pf_arg());
      }
      done = true;
    }
  }
  if constexpr (sizeof(VT) >= 4 && NRHS <= 3) {  // BF16 values, multi-column products: scalar-row kernel only
    if (done) {
    } else if (M.sell) {
      const DSell<VT>& S = *static_cast<const DSell<VT>*>(M.sell);
      const long long threads = (long long)S.nchunk * kChunk;
      k_sell_spmv<BR, BC, NRHS, VT, XT, E><<<ceil_div(threads, blk), blk, 0, s>>>(S, x, epi);
      done = true;
    } else if (BR > 1 && code_of(M) > 0 && code_of(M) < 100) {
      const long long threads = (long long)M.nbr * G;
      k_spmv_brow<BR, BC, NRHS, G, VT, XT, AT, E><<<ceil_div(threads, blk), blk, 0, s>>>(M.nbr, M.rp, M.col,
                                                                                       M.val, x, epi);
      done = true;
    }
  }
  if (!done) {
    const long long threads = (long long)M.nbr * BR * G;
    launch_product(k_spmv<BR, BC, NRHS, G, VT, XT, AT, E>, ceil_div(threads, blk), blk, s, M.nbr, (const int*)M.rp,
                   (const int*)M.col, (const VT*)M.val, x, epi, pf_arg());
  }
  SCR_LAUNCH();
}

template <int BR, int BC, int NRHS, int G, typename VT, typename XT>
inline void launch_spmv_e(const DBsr<VT>& M, const XT* x, XT* y, const EpiArgs& e, cudaStream_t s) {
  using AT = XT;  // accumulate in the vector precision
  switch (e.kind) {
    case Epi::Set: launch_spmv_g<BR, BC, NRHS, G, VT, XT, AT, Epi::Set>(M, x, y, e, s); break;
    case Epi::Axpby: launch_spmv_g<BR, BC, NRHS, G, VT, XT, AT, Epi::Axpby>(M, x, y, e, s); break;
    case Epi::Resid: launch_spmv_g<BR, BC, NRHS, G, VT, XT, AT, Epi::Resid>(M, x, y, e, s); break;
    case Epi::Jacobi: launch_spmv_g<BR, BC, NRHS, G, VT, XT, AT, Epi::Jacobi>(M, x, y, e, s); break;
    case Epi::ScaledSub: launch_spmv_g<BR, BC, NRHS, G, VT, XT, AT, Epi::ScaledSub>(M, x, y, e, s); break;
    case Epi::ChebFirst:
    case Epi::ChebStep:
      if constexpr (BR == BC) {
        if (e.kind == Epi::ChebFirst) launch_spmv_g<BR, BC, NRHS, G, VT, XT, AT, Epi::ChebFirst>(M, x, y, e, s);
        else launch_spmv_g<BR, BC, NRHS, G, VT, XT, AT, Epi::ChebStep>(M, x, y, e, s);
      } else {
        throw CudaError{cudaErrorInvalidValue, "Chebyshev epilogue on a non-square block shape"};
      }
      break;
  }
}

// lanes per scalar row: FP64 keeps groups narrow (FP64 adds of the
// reduction compete with the products), FP32 widens them for coalescing
// M.g: lanes per block row (1..16, block-row kernel for BR > 1), 100 +
// lanes per scalar row (scalar-row kernel) or 300 + lanes per block row
// (16-byte kernels on the padded copy, when M has one); 0 selects by row
// length
extern int g_forced;

template <typename VT>
inline int code_of(const DBsr<VT>& M) {
  return g_forced > 0 ? g_forced : M.g;
}

template <typename VT>
inline int pick_group(const DBsr<VT>& M) {
  const int g = code_of(M);
  if (g >= 300) return g - 300;
  if (g > 0) return g >= 100 ? g - 100 : g;
  // measured on the 616k-node tube: FP64 3x3 rows are fastest with 2 lanes
  // per scalar row (the FP64 pipe binds), FP32 with 4 (coalescing binds)
  const double per_row = M.nbr ? (double)M.nnzb * M.bc / M.nbr : 0.0;
  int G = sizeof(VT) == 8 ? (per_row >= 24 ? 2 : 1) : (per_row >= 24 ? 4 : 2);
  // small operators (the coarse AMG levels) fill less than a wave of the GPU
  // with one group per row, and their rows are long, so each lane would walk
  // dozens of blocks one dependent L2 round trip at a time: widen the group
  // (up to 16 lanes, at least 4 values per lane) while the grid stays below
  // two waves.  Measured on the coarse tube levels: about 23 us per product
  // with 2 lanes whatever the level's size.
  const long long nrows = (long long)M.nbr * M.br;
  const long long wave = (long long)sm_count() * 2048;
  while (G < 16 && per_row >= 8.0 * G && nrows * G < wave) G *= 2;
  return G;
}

template <int BR, int BC, int NR, typename VT, typename XT>
inline void dispatch_g(int G, const DBsr<VT>& M, const XT* x, XT* y, const EpiArgs& e, cudaStream_t s) {
  switch (G) {
    case 1: launch_spmv_e<BR, BC, NR, 1, VT, XT>(M, x, y, e, s); break;
    case 2: launch_spmv_e<BR, BC, NR, 2, VT, XT>(M, x, y, e, s); break;
    case 4: launch_spmv_e<BR, BC, NR, 4, VT, XT>(M, x, y, e, s); break;
    case 8: launch_spmv_e<BR, BC, NR, 8, VT, XT>(M, x, y, e, s); break;
    default: launch_spmv_e<BR, BC, NR, 16, VT, XT>(M, x, y, e, s); break;
  }
}

}  // namespace scr
