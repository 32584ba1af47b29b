// Sliced block-ELL copies of the hot operators and their products.
//
// A chunk holds 32 block rows, one per lane of the warp that multiplies it.
// Inside a window of W block rows (a multiple of 32) the rows are ordered by decreasing
// length, so the rows of a chunk have nearly the same number of blocks;
// each chunk is padded to its longest row.  Storage of chunk c (cptr[c]
// block slots per lane, starting at slot base = 32 * cptr[c]):
//   col[base + t*32 + lane]                      block column of slot t
//   val[(base + t*32) * BR*BC + e*32 + lane]     entry e = r*BC + c of it
// so every load of a warp is one contiguous segment.  Padding slots carry
// value 0 and repeat the row's last column.  Each lane accumulates all BR
// scalar rows of its block row with one multiply-add per stored value and
// no cross-lane reduction: the FP64 pipe spends its cycles on the product.
#include <algorithm>

#include "kernels.h"

namespace scr {


// sort (length desc, row asc) inside each window of kWindow rows: one block
// of kWindow threads per window, rank by counting
__global__ void __launch_bounds__(1024) k_sell_order(const int* __restrict__ rp, int nbr, int window,
                                                    int* __restrict__ perm) {
  extern __shared__ int len[];
  const int w0 = blockIdx.x * window;
  const int i = w0 + threadIdx.x;
  const int nw = min(window, nbr - w0);
  len[threadIdx.x] = i < nbr ? rp[i + 1] - rp[i] : -1;
  __syncthreads();
  if (threadIdx.x >= nw) return;
  const int my = len[threadIdx.x];
  int rank = 0;
  for (int q = 0; q < nw; ++q) {
    const int l = len[q];
    rank += (l > my) || (l == my && q < (int)threadIdx.x);
  }
  perm[w0 + rank] = i;
}

__global__ void k_sell_chunk_len(const int* __restrict__ rp, const int* __restrict__ perm, int nbr, int nchunk,
                                 int* __restrict__ clen) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchunk) return;
  int m = 0;
  for (int l = 0; l < kChunk; ++l) {
    const int q = c * kChunk + l;
    if (q < nbr) {
      const int i = perm[q];
      m = max(m, rp[i + 1] - rp[i]);
    }
  }
  clen[c] = m;
}

template <typename VT>
__global__ void k_sell_fill(DBsr<double> M, const int* __restrict__ perm, const int* __restrict__ cptr, int nchunk,
                            int* __restrict__ col, VT* __restrict__ val) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int c = (int)(g / kChunk), lane = (int)(g % kChunk);
  if (c >= nchunk) return;
  const int BR = M.br, BC = M.bc, bs = BR * BC;
  const int q = c * kChunk + lane;
  const long long base = (long long)cptr[c] * kChunk;
  const int L = cptr[c + 1] - cptr[c];
  int i = -1, s = 0, k = 0;
  if (q < M.nbr) {
    i = perm[q];
    s = M.rp[i];
    k = M.rp[i + 1] - s;
  }
  int last = k > 0 ? M.col[s + k - 1] : 0;
  for (int t = 0; t < L; ++t) {
    const long long slot = base + (long long)t * kChunk;
    col[slot + lane] = t < k ? M.col[s + t] : last;
    for (int e = 0; e < bs; ++e) {
      const int r = e / BC, cc = e - r * BC;
      const double v = t < k ? M.val[slab_index(s, k, t, r, cc, BR, BC)] : 0.0;
      val[slot * bs + (long long)e * kChunk + lane] = (VT)v;
    }
  }
}

template <typename VT>
void build_sell(const DBsr<double>& M, DSell<VT>& S, DeviceArena& a, cudaStream_t s, int window) {
  if (window < kChunk || window > 1024 || window % kChunk) throw CudaError{cudaErrorInvalidValue, "sell window"};
  S.nbr = M.nbr;
  S.nbc = M.nbc;
  S.br = M.br;
  S.bc = M.bc;
  S.nchunk = ceil_div(M.nbr, kChunk);
  DeviceArena tmp(s);
  S.perm = a.alloc<int>((size_t)S.nchunk * kChunk + 1);
  if (M.nbr == 0) {
    S.cptr = a.alloc<int>(1);
    SCR_CUDA(cudaMemsetAsync(S.cptr, 0, sizeof(int), s));
    S.col = a.alloc<int>(1);
    S.val = a.alloc<VT>(1);
    S.slots = 0;
    return;
  }
  k_sell_order<<<ceil_div(M.nbr, window), window, sizeof(int) * window, s>>>(M.rp, M.nbr, window, S.perm);
  SCR_LAUNCH();
  int* clen = tmp.alloc<int>(S.nchunk + 1);
  k_sell_chunk_len<<<ceil_div(S.nchunk, 256), 256, 0, s>>>(M.rp, S.perm, M.nbr, S.nchunk, clen);
  SCR_LAUNCH();
  S.cptr = a.alloc<int>(S.nchunk + 1);
  const long long slots = exclusive_scan(clen, S.cptr, S.nchunk, tmp, s);
  S.slots = slots;
  S.col = a.alloc<int>(slots * kChunk + 1);
  S.val = a.alloc<VT>(slots * kChunk * M.br * M.bc + 1);
  k_sell_fill<VT><<<ceil_div((long long)S.nchunk * kChunk, 256), 256, 0, s>>>(M, S.perm, S.cptr, S.nchunk, S.col,
                                                                              S.val);
  SCR_LAUNCH();
  counters().launches += 4;
  SCR_CUDA(cudaStreamSynchronize(s));
}
template void build_sell<double>(const DBsr<double>&, DSell<double>&, DeviceArena&, cudaStream_t, int);
template void build_sell<float>(const DBsr<double>&, DSell<float>&, DeviceArena&, cudaStream_t, int);

}  // namespace scr
