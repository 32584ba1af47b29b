// Smoothed-aggregation AMG set-up on the GPU.
//
//  strength graph  ||A_ij||_F >= theta sqrt(||A_ii||_F ||A_jj||_F), made
//                  symmetric (an entry is strong if it or its transpose is);
//  aggregation     distance-2 maximal independent set (parallel, random
//                  priorities from an integer hash, two rounds of max
//                  propagation per sweep), roots seed aggregates, their
//                  strong neighbours join, the remaining nodes join the
//                  aggregate of their strongest aggregated neighbour;
//  prolongator     P = (I - omega D^{-1} A) P_tent, P_tent = I_bs/sqrt(|a|),
//                  omega = 4 / (3 lambda), lambda = max_i sum_j |a_ij|/|a_ii|;
//  coarse operator A_c = R (A P) with R = P^T, by a row-wise hash SpGEMM
//                  whose numeric phase adds the products of each output
//                  entry in a fixed order (results do not depend on
//                  scheduling);
//  coarsest level  dense Gauss-Jordan inverse with partial pivoting.
#include <algorithm>
#include <cmath>

#include "kernels.h"

namespace scr {

// ------------------------------------------------------------ scan
__global__ void k_scan_block(const int* __restrict__ in, int* __restrict__ out, long long* __restrict__ bsum,
                             int n) {
  __shared__ long long wsum[32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long v = i < n ? in[i] : 0;
  long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    long long w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  const long long base = wid > 0 ? wsum[wid - 1] : 0;
  if (i < n) out[i] = (int)(base + x - v);
  if (threadIdx.x == blockDim.x - 1) bsum[blockIdx.x] = base + x;
}

__global__ void k_scan_small(long long* __restrict__ a, int n) {
  // single thread, n <= a few thousand
  long long s = 0;
  for (int i = 0; i < n; ++i) {
    long long v = a[i];
    a[i] = s;
    s += v;
  }
  a[n] = s;
}

__global__ void k_scan_add(int* __restrict__ out, const long long* __restrict__ boff, int n, int* __restrict__ total,
                           int nb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int)(out[i] + boff[blockIdx.x]);
  if (i == 0) *total = (int)boff[nb];
}

long long exclusive_scan(const int* in, int* out, int n, DeviceArena& tmp, cudaStream_t s) {
  // out has n+1 entries; out[n] = total
  const int B = 1024;
  const int nb = std::max(1, ceil_div(n, B));
  long long* bsum = tmp.alloc<long long>(nb + 1);
  if (n > 0) {
    k_scan_block<<<nb, B, 0, s>>>(in, out, bsum, n);
    SCR_LAUNCH();
  } else {
    SCR_CUDA(cudaMemsetAsync(bsum, 0, sizeof(long long), s));
  }
  k_scan_small<<<1, 1, 0, s>>>(bsum, n > 0 ? nb : 0);
  SCR_LAUNCH();
  if (n > 0) {
    k_scan_add<<<nb, B, 0, s>>>(out, bsum, n, out + n, nb);
    SCR_LAUNCH();
  } else {
    SCR_CUDA(cudaMemsetAsync(out, 0, sizeof(int), s));
  }
  counters().launches += 3;
  long long total = 0;
  SCR_CUDA(cudaMemcpyAsync(&total, bsum + (n > 0 ? nb : 0), sizeof(long long), cudaMemcpyDeviceToHost, s));
  SCR_CUDA(cudaStreamSynchronize(s));
  if (total > 2147483647LL) throw CudaError{cudaErrorInvalidValue, "scan total exceeds int32"};
  return total;
}

// ------------------------------------------------------------ row helpers
__device__ __forceinline__ int find_in_row(const int* __restrict__ col, int lo, int hi, int c) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (col[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void k_diag_scalar(DBsr<double> A, double* __restrict__ d, int* __restrict__ bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nbr) return;
  const int s = A.rp[i], e = A.rp[i + 1], k = e - s;
  const int p = find_in_row(A.col, s, e, i);
  const int bs = A.br;
  for (int r = 0; r < bs; ++r) {
    double v = 0.0;
    if (p < e && A.col[p] == i) v = A.val[slab_index(s, k, p - s, r, r, bs, A.bc)];
    d[(long long)i * bs + r] = v;
    if (v == 0.0 || !isfinite(v)) atomicExch(bad, 1);
  }
}

void diag_scalar(const DBsr<double>& A, double* d, int* bad, cudaStream_t s) {
  if (A.nbr == 0) return;
  k_diag_scalar<<<ceil_div(A.nbr, 256), 256, 0, s>>>(A, d, bad);
  SCR_LAUNCH();
  counters().launches++;
}

// per scalar row: 1 / a_ii
__global__ void k_inv_diag(DBsr<double> A, double* __restrict__ dinv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nbr) return;
  const int s = A.rp[i], e = A.rp[i + 1], k = e - s;
  const int p = find_in_row(A.col, s, e, i);
  for (int r = 0; r < A.br; ++r) {
    double v = 0.0;
    if (p < e && A.col[p] == i) v = A.val[slab_index(s, k, p - s, r, r, A.br, A.bc)];
    dinv[(long long)i * A.br + r] = v != 0.0 ? 1.0 / v : 0.0;
  }
}

void inv_diag(const DBsr<double>& A, double* dinv, cudaStream_t s) {
  if (A.nbr == 0) return;
  k_inv_diag<<<ceil_div(A.nbr, 256), 256, 0, s>>>(A, dinv);
  SCR_LAUNCH();
  counters().launches++;
}

// start vector of the power iteration: 1 + ((i * 2654435761) mod 2^32 mod 1000) / 1000
__global__ void k_power_start(double* __restrict__ v, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned h = (unsigned)((unsigned long long)i * 2654435761ULL);
  v[i] = 1.0 + (double)(h % 1000u) / 1000.0;
}

__global__ void k_rsqrt_scalar(const double* __restrict__ in, double* __restrict__ out) {
  const double v = *in;
  *out = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
}

void power_start_unit(double* v, long long n, const Reducer& red, double* nrm, cudaStream_t s) {
  if (n == 0) return;
  k_power_start<<<ceil_div(n, 256), 256, 0, s>>>(v, n);
  SCR_LAUNCH();
  norm2<double>(v, n, nrm, red, s);
  k_rsqrt_scalar<<<1, 1, 0, s>>>(nrm, nrm + 1);
  SCR_LAUNCH();
  scale_by<double>(v, nrm + 1, v, n, s);
  counters().launches += 2;
}

double power_lambda(const DBsr<double>& A, const double* dinv, int iters, cudaStream_t s) {
  const long long n = (long long)A.nbr * A.br;
  if (n == 0) return 0.0;
  DeviceArena tmp(s);
  Reducer red = make_reducer(tmp);
  double* v = tmp.alloc<double>(n);
  double* w = tmp.alloc<double>(n);
  double* nrm = tmp.alloc<double>(2);
  k_power_start<<<ceil_div(n, 256), 256, 0, s>>>(v, n);
  SCR_LAUNCH();
  norm2<double>(v, n, nrm, red, s);
  k_rsqrt_scalar<<<1, 1, 0, s>>>(nrm, nrm + 1);
  scale_by<double>(v, nrm + 1, v, n, s);
  for (int it = 0; it < iters; ++it) {
    spmv<double, double>(A, v, w, 1, EpiArgs(), s);
    diag_scale<double>(w, dinv, w, n, 1, s);
    norm2<double>(w, n, nrm, red, s);
    k_rsqrt_scalar<<<1, 1, 0, s>>>(nrm, nrm + 1);
    scale_by<double>(w, nrm + 1, v, n, s);
  }
  SCR_LAUNCH();
  double h = 0.0;
  SCR_CUDA(cudaMemcpyAsync(&h, nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
  SCR_CUDA(cudaStreamSynchronize(s));
  counters().launches += 2 + 2 * iters;
  return 1.1 * std::sqrt(h);
}

// per scalar row: 1 / sum_j |a_ij|
__global__ void k_l1_inv(DBsr<double> A, double* __restrict__ dinv) {
  const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)A.nbr * A.br;
  if (o >= n) return;
  const int i = (int)(o / A.br), r = (int)(o - (long long)i * A.br);
  const int s = A.rp[i], k = A.rp[i + 1] - s, L = k * A.bc;
  const double* v = A.val + (long long)s * A.br * A.bc + (long long)r * L;
  double acc = 0.0;
  for (int q = 0; q < L; ++q) acc += fabs(v[q]);
  dinv[o] = acc > 0.0 ? 1.0 / acc : 0.0;
}

// per scalar row: sum_j |a_ij| (the lumped diagonal of SIMPLEC)
__global__ void k_abs_rowsum(DBsr<double> A, double* __restrict__ d) {
  const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)A.nbr * A.br;
  if (o >= n) return;
  const int i = (int)(o / A.br), r = (int)(o - (long long)i * A.br);
  const int s = A.rp[i], k = A.rp[i + 1] - s, L = k * A.bc;
  const double* v = A.val + (long long)s * A.br * A.bc + (long long)r * L;
  double acc = 0.0;
  for (int q = 0; q < L; ++q) acc += fabs(v[q]);
  d[o] = acc;
}

void abs_rowsum(const DBsr<double>& A, double* d, cudaStream_t s) {
  const long long n = (long long)A.nbr * A.br;
  if (n == 0) return;
  k_abs_rowsum<<<ceil_div(n, 256), 256, 0, s>>>(A, d);
  SCR_LAUNCH();
  counters().launches++;
}

void l1_inv(const DBsr<double>& A, double* dinv, cudaStream_t s) {
  const long long n = (long long)A.nbr * A.br;
  if (n == 0) return;
  k_l1_inv<<<ceil_div(n, 256), 256, 0, s>>>(A, dinv);
  SCR_LAUNCH();
  counters().launches++;
}

__global__ void k_gershgorin(DBsr<double> A, const double* __restrict__ d, unsigned long long* __restrict__ out) {
  const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)A.nbr * A.br;
  if (o >= n) return;
  const int i = (int)(o / A.br), r = (int)(o - (long long)i * A.br);
  const int s = A.rp[i], k = A.rp[i + 1] - s, L = k * A.bc;
  const double* v = A.val + (long long)s * A.br * A.bc + (long long)r * L;
  double acc = 0.0;
  for (int q = 0; q < L; ++q) acc += fabs(v[q]);
  const double ratio = acc / fabs(d[o]);
  // non-negative doubles order like their bit patterns
  atomicMax(out, (unsigned long long)__double_as_longlong(ratio));
}

void gershgorin(const DBsr<double>& A, const double* d, double* out, cudaStream_t s) {
  const long long n = (long long)A.nbr * A.br;
  SCR_CUDA(cudaMemsetAsync(out, 0, sizeof(double), s));
  if (n == 0) return;
  k_gershgorin<<<ceil_div(n, 256), 256, 0, s>>>(A, d, reinterpret_cast<unsigned long long*>(out));
  SCR_LAUNCH();
  counters().launches++;
}

__global__ void k_prolong_rowscale(const double* __restrict__ d, const double* __restrict__ lambda,
                                   double* __restrict__ rs, int n) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const double omega = 4.0 / (3.0 * (*lambda));
  rs[o] = -omega / d[o];
}

void prolong_rowscale(const double* d, const double* lambda, double* rowscale, int n, cudaStream_t s) {
  if (n == 0) return;
  k_prolong_rowscale<<<ceil_div(n, 256), 256, 0, s>>>(d, lambda, rowscale, n);
  SCR_LAUNCH();
  counters().launches++;
}

// out = diag(d)^{-1} M (scalar rows of M divided by d), same pattern as M
__global__ void k_scale_rows_inv(DBsr<double> M, const double* __restrict__ d, double* __restrict__ out) {
  const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)M.nbr * M.br;
  if (o >= n) return;
  const int i = (int)(o / M.br), r = (int)(o - (long long)i * M.br);
  const int s = M.rp[i], k = M.rp[i + 1] - s, L = k * M.bc;
  const long long base = (long long)s * M.br * M.bc + (long long)r * L;
  const double inv = 1.0 / d[o];
  for (int q = 0; q < L; ++q) out[base + q] = M.val[base + q] * inv;
}

void scale_rows_inv(const DBsr<double>& M, const double* d, DBsr<double>& out, DeviceArena& a, cudaStream_t s) {
  out = M;
  out.val = a.alloc<double>(M.nnzb * M.br * M.bc + 1);
  const long long n = (long long)M.nbr * M.br;
  if (n == 0) return;
  k_scale_rows_inv<<<ceil_div(n, 256), 256, 0, s>>>(M, d, out.val);
  SCR_LAUNCH();
  counters().launches++;
}

// ------------------------------------------------------------ strength
__global__ void k_block_norms(DBsr<double> A, double* __restrict__ bnorm, double* __restrict__ dnorm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nbr) return;
  const int s = A.rp[i], k = A.rp[i + 1] - s;
  double dn = 0.0;
  for (int t = 0; t < k; ++t) {
    double acc = 0.0;
    for (int r = 0; r < A.br; ++r)
      for (int c = 0; c < A.bc; ++c) {
        const double v = A.val[slab_index(s, k, t, r, c, A.br, A.bc)];
        acc += v * v;
      }
    const double nv = sqrt(acc);
    bnorm[s + t] = nv;
    if (A.col[s + t] == i) dn = nv;
  }
  dnorm[i] = dn;
}

__global__ void k_strong(DBsr<double> A, const double* __restrict__ bnorm, const double* __restrict__ dnorm,
                         double theta, unsigned char* __restrict__ strong, int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nbr) return;
  const int s = A.rp[i], e = A.rp[i + 1];
  int c = 0;
  for (int t = s; t < e; ++t) {
    const int j = A.col[t];
    unsigned char f = 0;
    if (j != i) {
      const double thr = theta * sqrt(dnorm[i] * dnorm[j]);
      if (bnorm[t] > 0.0 && bnorm[t] >= thr) f = 1;
      // transpose entry (j, i)
      const int sj = A.rp[j], ej = A.rp[j + 1];
      const int p = find_in_row(A.col, sj, ej, i);
      if (p < ej && A.col[p] == i && bnorm[p] > 0.0 && bnorm[p] >= thr) f = 1;
    }
    strong[t] = f;
    c += f;
  }
  cnt[i] = c;
}

__global__ void k_strong_fill(DBsr<double> A, const unsigned char* __restrict__ strong,
                              const double* __restrict__ bnorm, const int* __restrict__ srp,
                              int* __restrict__ snb, double* __restrict__ sw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nbr) return;
  int o = srp[i];
  for (int t = A.rp[i]; t < A.rp[i + 1]; ++t)
    if (strong[t]) {
      snb[o] = A.col[t];
      sw[o] = bnorm[t];
      ++o;
    }
}

// ------------------------------------------------------------ MIS-2
__device__ __forceinline__ unsigned int hash32(unsigned int x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

enum : unsigned long long { ST_OUT = 0, ST_UNDEC = 1, ST_IN = 2 };

__device__ __forceinline__ unsigned long long make_key(unsigned long long st, int i) {
  const unsigned long long rnd = (hash32((unsigned)i * 2654435761u + 0x9e3779b9u) >> 2) & 0x3fffffffULL;
  return (st << 62) | (rnd << 32) | (unsigned long long)(unsigned)i;
}

__global__ void k_mis_init(const int* __restrict__ srp, int n, unsigned long long* __restrict__ key,
                           unsigned char* __restrict__ isolated) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool iso = srp[i + 1] == srp[i];
  isolated[i] = iso;
  key[i] = make_key(iso ? ST_OUT : ST_UNDEC, i);
}

__global__ void k_mis_max(const int* __restrict__ srp, const int* __restrict__ snb, int n,
                          const unsigned long long* __restrict__ in, unsigned long long* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long m = in[i];
  for (int t = srp[i]; t < srp[i + 1]; ++t) m = max(m, in[snb[t]]);
  out[i] = m;
}

__global__ void k_mis_update(int n, unsigned long long* __restrict__ key, const unsigned long long* __restrict__ t2,
                             int* __restrict__ undecided) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long k = key[i];
  if ((k >> 62) != ST_UNDEC) return;
  const unsigned long long m = t2[i];
  if ((m >> 62) == ST_IN) {
    key[i] = make_key(ST_OUT, i);
  } else if (m == k) {
    key[i] = make_key(ST_IN, i);
  } else {
    atomicAdd(undecided, 1);
  }
}

__global__ void k_root_flags(int n, const unsigned long long* __restrict__ key, int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  flag[i] = (key[i] >> 62) == ST_IN ? 1 : 0;
}

__global__ void k_root_list(int n, const int* __restrict__ flag, const int* __restrict__ rootid,
                            int* __restrict__ roots) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flag[i]) roots[rootid[i]] = i;
}

__global__ void k_agg_pass1(int n, const unsigned long long* __restrict__ key, const int* __restrict__ rootid,
                            const int* __restrict__ srp, const int* __restrict__ snb,
                            const unsigned char* __restrict__ isolated, int* __restrict__ agg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if ((key[i] >> 62) == ST_IN) {
    agg[i] = rootid[i];
    return;
  }
  int a = -1;
  if (!isolated[i]) {
    unsigned long long best = 0;
    for (int t = srp[i]; t < srp[i + 1]; ++t) {
      const int j = snb[t];
      const unsigned long long kj = key[j];
      if ((kj >> 62) == ST_IN && (a < 0 || kj > best)) {
        best = kj;
        a = rootid[j];
      }
    }
  }
  agg[i] = a;
}

__global__ void k_agg_pass2(int n, const int* __restrict__ srp, const int* __restrict__ snb,
                            const double* __restrict__ sw, const unsigned char* __restrict__ isolated,
                            const int* __restrict__ agg1, int* __restrict__ agg2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = agg1[i];
  if (a < 0 && !isolated[i]) {
    double bw = -1.0;
    int bj = 0x7fffffff;
    for (int t = srp[i]; t < srp[i + 1]; ++t) {
      const int j = snb[t];
      const int aj = agg1[j];
      if (aj < 0) continue;
      if (sw[t] > bw || (sw[t] == bw && j < bj)) {
        bw = sw[t];
        bj = j;
        a = aj;
      }
    }
  }
  agg2[i] = a;
}

Aggregation aggregate(const DBsr<double>& A, double theta, DeviceArena& arena, DeviceArena& tmp, cudaStream_t s,
                      int* mis_rounds) {
  const int n = A.nbr;
  Aggregation out;
  out.agg = arena.alloc<int>(n + 1);
  if (n == 0) return out;
  const int T = 256, G = ceil_div(n, T);
  double* bnorm = tmp.alloc<double>(A.nnzb);
  double* dnorm = tmp.alloc<double>(n);
  unsigned char* strong = tmp.alloc<unsigned char>(A.nnzb);
  int* cnt = tmp.alloc<int>(n + 1);
  int* srp = tmp.alloc<int>(n + 1);
  k_block_norms<<<G, T, 0, s>>>(A, bnorm, dnorm);
  SCR_LAUNCH();
  k_strong<<<G, T, 0, s>>>(A, bnorm, dnorm, theta, strong, cnt);
  SCR_LAUNCH();
  const long long ns = exclusive_scan(cnt, srp, n, tmp, s);
  int* snb = tmp.alloc<int>(ns + 1);
  double* sw = tmp.alloc<double>(ns + 1);
  k_strong_fill<<<G, T, 0, s>>>(A, strong, bnorm, srp, snb, sw);
  SCR_LAUNCH();
  unsigned long long* key = tmp.alloc<unsigned long long>(n);
  unsigned long long* t1 = tmp.alloc<unsigned long long>(n);
  unsigned long long* t2 = tmp.alloc<unsigned long long>(n);
  unsigned char* isolated = tmp.alloc<unsigned char>(n);
  int* und = tmp.alloc<int>(1);
  k_mis_init<<<G, T, 0, s>>>(srp, n, key, isolated);
  SCR_LAUNCH();
  counters().launches += 4;
  int rounds = 0;
  for (;;) {
    SCR_CUDA(cudaMemsetAsync(und, 0, sizeof(int), s));
    k_mis_max<<<G, T, 0, s>>>(srp, snb, n, key, t1);
    k_mis_max<<<G, T, 0, s>>>(srp, snb, n, t1, t2);
    k_mis_update<<<G, T, 0, s>>>(n, key, t2, und);
    SCR_LAUNCH();
    counters().launches += 3;
    int h_und = 0;
    SCR_CUDA(cudaMemcpyAsync(&h_und, und, sizeof(int), cudaMemcpyDeviceToHost, s));
    SCR_CUDA(cudaStreamSynchronize(s));
    ++rounds;
    if (h_und == 0) break;
    if (rounds > 200) throw CudaError{cudaErrorUnknown, "MIS-2 did not terminate"};
  }
  if (mis_rounds) *mis_rounds = rounds;
  int* flag = tmp.alloc<int>(n + 1);
  int* rootid = tmp.alloc<int>(n + 1);
  k_root_flags<<<G, T, 0, s>>>(n, key, flag);
  SCR_LAUNCH();
  out.n_agg = (int)exclusive_scan(flag, rootid, n, tmp, s);
  out.roots = arena.alloc<int>(out.n_agg + 1);
  k_root_list<<<G, T, 0, s>>>(n, flag, rootid, out.roots);
  SCR_LAUNCH();
  counters().launches++;
  int* agg1 = tmp.alloc<int>(n);
  k_agg_pass1<<<G, T, 0, s>>>(n, key, rootid, srp, snb, isolated, agg1);
  k_agg_pass2<<<G, T, 0, s>>>(n, srp, snb, sw, isolated, agg1, out.agg);
  SCR_LAUNCH();
  counters().launches += 3;
  return out;
}

// ------------------------------------------------------------ P_tent
__global__ void k_agg_sizes(int n, const int* __restrict__ agg, int* __restrict__ sizes, int* __restrict__ has) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int a = agg[i];
  has[i] = a >= 0 ? 1 : 0;
  if (a >= 0) atomicAdd(sizes + a, 1);
}

__global__ void k_tentative_fill(int n, int bs, const int* __restrict__ agg, const int* __restrict__ sizes,
                                 const int* __restrict__ rp, int* __restrict__ col, double* __restrict__ val) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int a = agg[i];
  if (a < 0) return;
  const int s = rp[i];
  col[s] = a;
  const double v = 1.0 / sqrt((double)sizes[a]);
  for (int r = 0; r < bs; ++r)
    for (int c = 0; c < bs; ++c) val[slab_index(s, 1, 0, r, c, bs, bs)] = r == c ? v : 0.0;
}

void tentative(const int* agg, int nbr, int n_agg, int bs, DBsr<double>& P, DeviceArena& arena, DeviceArena& tmp,
               cudaStream_t s) {
  int* sizes = tmp.alloc<int>(n_agg + 1);
  int* has = tmp.alloc<int>(nbr + 1);
  SCR_CUDA(cudaMemsetAsync(sizes, 0, sizeof(int) * (n_agg + 1), s));
  P.nbr = nbr;
  P.nbc = n_agg;
  P.br = P.bc = bs;
  P.rp = arena.alloc<int>(nbr + 1);
  if (nbr > 0) {
    k_agg_sizes<<<ceil_div(nbr, 256), 256, 0, s>>>(nbr, agg, sizes, has);
    SCR_LAUNCH();
  }
  P.nnzb = exclusive_scan(has, P.rp, nbr, tmp, s);
  P.col = arena.alloc<int>(P.nnzb + 1);
  P.val = arena.alloc<double>(P.nnzb * bs * bs + 1);
  if (nbr > 0) {
    k_tentative_fill<<<ceil_div(nbr, 256), 256, 0, s>>>(nbr, bs, agg, sizes, P.rp, P.col, P.val);
    SCR_LAUNCH();
  }
  counters().launches += 2;
}

// ------------------------------------------------------------ SpGEMM
// Row-wise product C = A * B, one warp per output row.  The symbolic phases
// insert the column indices of the row's partial products into a hash table
// (shared memory for short rows; otherwise the warp's private slice of a
// bounded global scratch, reused row after row by a persistent grid), count
// them, write them out and sort them.  The numeric phase walks A's row in
// order and lets the lanes add the products of one B row at a time into the
// output row (distinct columns per step, so every output entry receives its
// terms in a fixed order).
constexpr int kHashSlots = 1024;          // per warp in shared memory
constexpr int kGlobalSlots = 1 << 16;     // per warp in global scratch
constexpr int kSpgemmWarps = 4;
constexpr int kNumericCols = 512;         // output columns cached per warp in the numeric phase

__device__ __forceinline__ unsigned hash_col(int c) { return (unsigned)c * 2654435761u; }

__global__ void k_spgemm_ub(DBsr<double> A, DBsr<double> B, int* __restrict__ ub) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nbr) return;
  long long u = 0;
  for (int t = A.rp[i]; t < A.rp[i + 1]; ++t) {
    const int j = A.col[t];
    u += B.rp[j + 1] - B.rp[j];
  }
  ub[i] = (int)min(u, (long long)0x3fffffff);
}

// table size for a row with upper bound ub (0: shared-memory table)
__device__ __forceinline__ int global_table_size(int ub) {
  if (ub <= kHashSlots / 2) return 0;
  int g = 1;
  while (g < 2 * ub && g < kGlobalSlots) g <<= 1;
  return g;
}

// insert the columns of row i of A*B into a warp's hash table; returns the
// number of new keys this lane inserted; a table that fills up sets *err.
// When B's rows are short on average (ub < 8 entries per A entry: the
// prolongators and the Galerkin factors), the lanes take the entries of A's
// row in turn and each inserts the whole B row its entry selects, which
// keeps them busy and overlaps the dependent loads of the A entries;
// otherwise the lanes share each B row.  The resulting column set does not
// depend on the order of the inserts.
__device__ __forceinline__ bool spgemm_try_insert(int key, int* table, int hsize, int* err, int& mine) {
  unsigned h = hash_col(key) & (hsize - 1);
  for (int probe = 0;; ++probe) {
    if (probe >= hsize) {
      atomicExch(err, 1);
      return false;
    }
    const int prev = atomicCAS(table + h, -1, key);
    if (prev == -1) {
      ++mine;
      return true;
    }
    if (prev == key) return true;
    h = (h + 1) & (hsize - 1);
  }
}

__device__ int spgemm_insert(const DBsr<double>& A, const DBsr<double>& B, int i, int ub, int* table, int hsize,
                             int lane, int* err) {
  int mine = 0;
  const int as = A.rp[i], ae = A.rp[i + 1];
  if (ub >= 8 * (ae - as)) {
    // long B rows (e.g. C diag(A)^{-1} B): the lanes share each B row
    for (int t = as; t < ae; ++t) {
      const int j = A.col[t];
      for (int u = B.rp[j] + lane; u < B.rp[j + 1]; u += 32)
        if (!spgemm_try_insert(B.col[u], table, hsize, err, mine)) return mine;
    }
    return mine;
  }
  for (int t = as + lane; t < ae; t += 32) {
    const int j = A.col[t];
    for (int u = B.rp[j]; u < B.rp[j + 1]; ++u)
      if (!spgemm_try_insert(B.col[u], table, hsize, err, mine)) return mine;
  }
  return mine;
}

__global__ void __launch_bounds__(32 * kSpgemmWarps) k_spgemm_count(DBsr<double> A, DBsr<double> B,
                                                                   const int* __restrict__ ub, int* __restrict__ gtab,
                                                                   int* __restrict__ cnt, int* __restrict__ err) {
  __shared__ int smem[kSpgemmWarps][kHashSlots];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kSpgemmWarps + w, nw = gridDim.x * kSpgemmWarps;
  int* gtab_w = gtab + (long long)gw * kGlobalSlots;
  for (int i = gw; i < A.nbr; i += nw) {
    const int gs = global_table_size(ub[i]);
    int* table = gs ? gtab_w : smem[w];
    const int hsize = gs ? gs : kHashSlots;
    for (int h = lane; h < hsize; h += 32) table[h] = -1;
    __syncwarp();
    const int mine = spgemm_insert(A, B, i, ub[i], table, hsize, lane, err);
    const int tot = warp_sum(mine);
    if (lane == 0) cnt[i] = tot;
    __syncwarp();
  }
}

__global__ void __launch_bounds__(32 * kSpgemmWarps) k_spgemm_fill(DBsr<double> A, DBsr<double> B,
                                                                  const int* __restrict__ ub, int* __restrict__ gtab,
                                                                  DBsr<double> C, int* __restrict__ err) {
  __shared__ int smem[kSpgemmWarps][kHashSlots];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kSpgemmWarps + w, nw = gridDim.x * kSpgemmWarps;
  int* gtab_w = gtab + (long long)gw * kGlobalSlots;
  for (int i = gw; i < A.nbr; i += nw) {
    const int gs = global_table_size(ub[i]);
    int* table = gs ? gtab_w : smem[w];
    const int hsize = gs ? gs : kHashSlots;
    for (int h = lane; h < hsize; h += 32) table[h] = -1;
    __syncwarp();
    spgemm_insert(A, B, i, ub[i], table, hsize, lane, err);
    __syncwarp();
    // compact the keys into the front of C's row (unsorted) ...
    const int base = C.rp[i], cnt = C.rp[i + 1] - base;
    int o = 0;
    for (int h0 = 0; h0 < hsize; h0 += 32) {
      const int h = h0 + lane;
      const int key = h < hsize ? table[h] : -1;
      const unsigned m = __ballot_sync(0xffffffffu, key >= 0);
      if (key >= 0 && o + __popc(m & ((1u << lane) - 1)) < cnt)
        C.col[base + o + __popc(m & ((1u << lane) - 1))] = key;
      o += __popc(m);
    }
    __syncwarp();
    // ... copy them into the table and rank-sort them back into C's row
    for (int e = lane; e < cnt; e += 32) table[e] = C.col[base + e];
    __syncwarp();
    for (int e = lane; e < cnt; e += 32) {
      const int v = table[e];
      int rank = 0;
      for (int f = 0; f < cnt; ++f) rank += table[f] < v;
      C.col[base + rank] = v;
    }
    __syncwarp();
  }
}

template <int BR, int BK, int BC>
__global__ void __launch_bounds__(32 * kSpgemmWarps) k_spgemm_numeric(DBsr<double> A, DBsr<double> B,
                                                                     DBsr<double> C) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kSpgemmWarps + w;
  if (i >= A.nbr) return;  // uniform over the warp
  const int cs = C.rp[i], ck = C.rp[i + 1] - cs;
  double* cv = C.val + (long long)cs * BR * BC;
  const int as = A.rp[i], ak = A.rp[i + 1] - as;
  if (ck <= 32) {
    // Rows with at most 32 output entries (the prolongator and Galerkin
    // products): A's row is taken in chunks of 32 entries; within a chunk
    // the partial products (t, u) = (entry t of A's row, entry u of the B row
    // it selects) are numbered p in t-major order, lane p % 32 forms product
    // p, and lane e, owner of output entry e, adds the products that land on
    // e in increasing t, i.e. in the order of the general path below.
    constexpr unsigned kFull = 0xffffffffu;
    double acc[BR * BC];
#pragma unroll
    for (int e = 0; e < BR * BC; ++e) acc[e] = 0.0;
    for (int tc = 0; tc < ak; tc += 32) {
      const int nt = min(32, ak - tc);
      int bst = 0, lent = 0;
      if (lane < nt) {
        const int jt = A.col[as + tc + lane];
        bst = B.rp[jt];
        lent = B.rp[jt + 1] - bst;
      }
      int incl = lent;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
      }
      const int off = incl - lent;
      const int np = __shfl_sync(kFull, incl, 31);
      for (int base = 0; base < np; base += 32) {
        const int p = base + lane;
        int tl = 0;  // the last entry of the chunk whose products start at or before p
        for (int q = 1; q < nt; ++q)
          if (__shfl_sync(kFull, off, q) <= p) tl = q;
        const int j_b = __shfl_sync(kFull, bst, tl), j_len = __shfl_sync(kFull, lent, tl);
        const int u = p - __shfl_sync(kFull, off, tl);
        int pos = -1;
        double prod[BR * BC];
#pragma unroll
        for (int e = 0; e < BR * BC; ++e) prod[e] = 0.0;
        if (p < np) {
          const int t = tc + tl;
          pos = find_in_row(C.col, cs, cs + ck, B.col[j_b + u]) - cs;
#pragma unroll
          for (int r = 0; r < BR; ++r)
#pragma unroll
            for (int q = 0; q < BC; ++q) {
              double v = 0.0;
#pragma unroll
              for (int m = 0; m < BK; ++m)
                v = fma(A.val[slab_index(as, ak, t, r, m, BR, BK)], B.val[slab_index(j_b, j_len, u, m, q, BK, BC)],
                        v);
              prod[r * BC + q] = v;
            }
        }
        const int cnt = min(32, np - base);
        for (int q = 0; q < cnt; ++q) {
          const int pq = __shfl_sync(kFull, pos, q);
#pragma unroll
          for (int e = 0; e < BR * BC; ++e) {
            const double v = __shfl_sync(kFull, prod[e], q);
            if (lane == pq) acc[e] += v;
          }
        }
      }
    }
    if (lane < ck) {
#pragma unroll
      for (int r = 0; r < BR; ++r)
#pragma unroll
        for (int q = 0; q < BC; ++q) cv[(long long)r * ck * BC + (long long)lane * BC + q] = acc[r * BC + q];
    }
    return;
  }
  // general path: the output row's columns in shared memory when they fit,
  // for the searches below
  __shared__ int ccol[kSpgemmWarps][kNumericCols];
  const bool cached = ck <= kNumericCols;
  if (cached)
    for (int e = lane; e < ck; e += 32) ccol[w][e] = C.col[cs + e];
  for (int e = lane; e < ck * BR * BC; e += 32) cv[e] = 0.0;
  __syncwarp();
  for (int t = 0; t < ak; ++t) {
    double a[BR][BK];
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int m = 0; m < BK; ++m) a[r][m] = A.val[slab_index(as, ak, t, r, m, BR, BK)];
    const int j = A.col[as + t];
    const int bs = B.rp[j], bk = B.rp[j + 1] - bs;
    for (int u = lane; u < bk; u += 32) {
      const int c = B.col[bs + u];
      const int pos = cached ? find_in_row(ccol[w], 0, ck, c) : find_in_row(C.col, cs, cs + ck, c) - cs;
      if (pos >= ck) continue;  // cannot happen for a consistent symbolic phase
      double b[BK][BC];
#pragma unroll
      for (int m = 0; m < BK; ++m)
#pragma unroll
        for (int q = 0; q < BC; ++q) b[m][q] = B.val[slab_index(bs, bk, u, m, q, BK, BC)];
#pragma unroll
      for (int r = 0; r < BR; ++r)
#pragma unroll
        for (int q = 0; q < BC; ++q) {
          double acc = 0.0;
#pragma unroll
          for (int m = 0; m < BK; ++m) acc = fma(a[r][m], b[m][q], acc);
          cv[(long long)r * ck * BC + (long long)pos * BC + q] += acc;
        }
    }
    __syncwarp();
  }
}

void spgemm(const DBsr<double>& A, const DBsr<double>& B, DBsr<double>& C, DeviceArena& arena, cudaStream_t s) {
  if (A.bc != B.br || A.nbc != B.nbr) throw CudaError{cudaErrorInvalidValue, "spgemm: shape mismatch"};
  DeviceArena tmp(s);
  const int n = A.nbr;
  C.nbr = n;
  C.nbc = B.nbc;
  C.br = A.br;
  C.bc = B.bc;
  C.rp = arena.alloc<int>(n + 1);
  if (n == 0) {
    SCR_CUDA(cudaMemsetAsync(C.rp, 0, sizeof(int), s));
    C.nnzb = 0;
    C.col = arena.alloc<int>(1);
    C.val = arena.alloc<double>(1);
    return;
  }
  int* ub = tmp.alloc<int>(n);
  int* cnt = tmp.alloc<int>(n + 1);
  int* err = tmp.alloc<int>(1);
  SCR_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  k_spgemm_ub<<<ceil_div(n, 256), 256, 0, s>>>(A, B, ub);
  SCR_LAUNCH();
  // persistent grid: 4 blocks of 4 warps per SM, each warp owning a slice
  const int pgrid = std::min(ceil_div(n, kSpgemmWarps), 4 * sm_count());
  int* gtab = tmp.alloc<int>((size_t)pgrid * kSpgemmWarps * kGlobalSlots);
  k_spgemm_count<<<pgrid, 32 * kSpgemmWarps, 0, s>>>(A, B, ub, gtab, cnt, err);
  SCR_LAUNCH();
  C.nnzb = exclusive_scan(cnt, C.rp, n, tmp, s);  // synchronises
  int herr = 0;
  SCR_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  SCR_CUDA(cudaStreamSynchronize(s));
  if (herr) throw CudaError{cudaErrorInvalidValue, "spgemm: a product row exceeds the hash-table capacity"};
  C.col = arena.alloc<int>(C.nnzb + 1);
  C.val = arena.alloc<double>(C.nnzb * C.br * C.bc + 1);
  k_spgemm_fill<<<pgrid, 32 * kSpgemmWarps, 0, s>>>(A, B, ub, gtab, C, err);
  SCR_LAUNCH();
  const int grid = ceil_div(n, kSpgemmWarps);
  const int br = A.br, bk = A.bc, bc = B.bc;
  if (br == 3 && bk == 3 && bc == 3) k_spgemm_numeric<3, 3, 3><<<grid, 32 * kSpgemmWarps, 0, s>>>(A, B, C);
  else if (br == 1 && bk == 3 && bc == 1) k_spgemm_numeric<1, 3, 1><<<grid, 32 * kSpgemmWarps, 0, s>>>(A, B, C);
  else if (br == 1 && bk == 1 && bc == 1) k_spgemm_numeric<1, 1, 1><<<grid, 32 * kSpgemmWarps, 0, s>>>(A, B, C);
  else throw CudaError{cudaErrorInvalidValue, "spgemm: unsupported block shape"};
  SCR_LAUNCH();
  counters().launches += 4;
  SCR_CUDA(cudaStreamSynchronize(s));  // tmp is released on return
}

// ------------------------------------------------------------ sparse add
__global__ void k_spadd_count(DBsr<double> A, DBsr<double> B, int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nbr) return;
  int p = A.rp[i], pe = A.rp[i + 1], q = B.rp[i], qe = B.rp[i + 1], c = 0;
  while (p < pe || q < qe) {
    const int a = p < pe ? A.col[p] : 0x7fffffff, b = q < qe ? B.col[q] : 0x7fffffff;
    if (a <= b) ++p;
    if (b <= a) ++q;
    ++c;
  }
  cnt[i] = c;
}

__global__ void k_spadd_fill(DBsr<double> A, double alpha, DBsr<double> B, double beta,
                             const double* __restrict__ rs, DBsr<double> C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nbr) return;
  const int BR = C.br, BC = C.bc;
  const int as = A.rp[i], ak = A.rp[i + 1] - as, bs = B.rp[i], bk = B.rp[i + 1] - bs;
  const int cs = C.rp[i], ck = C.rp[i + 1] - cs;
  int p = 0, q = 0, o = 0;
  while (p < ak || q < bk) {
    const int a = p < ak ? A.col[as + p] : 0x7fffffff, b = q < bk ? B.col[bs + q] : 0x7fffffff;
    const int c = min(a, b);
    C.col[cs + o] = c;
    for (int r = 0; r < BR; ++r) {
      const double sc = beta * (rs ? rs[(long long)i * BR + r] : 1.0);
      for (int cc = 0; cc < BC; ++cc) {
        double v = 0.0;
        if (a == c) v += alpha * A.val[slab_index(as, ak, p, r, cc, BR, BC)];
        if (b == c) v += sc * B.val[slab_index(bs, bk, q, r, cc, BR, BC)];
        C.val[slab_index(cs, ck, o, r, cc, BR, BC)] = v;
      }
    }
    if (a == c) ++p;
    if (b == c) ++q;
    ++o;
  }
}

void spadd(const DBsr<double>& A, double alpha, const DBsr<double>& B, const double* rowscale, DBsr<double>& C,
           DeviceArena& arena, cudaStream_t s) {
  if (A.nbr != B.nbr || A.br != B.br || A.bc != B.bc) throw CudaError{cudaErrorInvalidValue, "spadd: shape"};
  DeviceArena tmp(s);
  const int n = A.nbr;
  C.nbr = n;
  C.nbc = std::max(A.nbc, B.nbc);
  C.br = A.br;
  C.bc = A.bc;
  C.rp = arena.alloc<int>(n + 1);
  int* cnt = tmp.alloc<int>(n + 1);
  if (n > 0) {
    k_spadd_count<<<ceil_div(n, 256), 256, 0, s>>>(A, B, cnt);
    SCR_LAUNCH();
  }
  C.nnzb = exclusive_scan(cnt, C.rp, n, tmp, s);
  C.col = arena.alloc<int>(C.nnzb + 1);
  C.val = arena.alloc<double>(C.nnzb * C.br * C.bc + 1);
  if (n > 0) {
    // beta = 1 with row scaling, or -1 without (Shat = D - C diag(A)^{-1} B)
    k_spadd_fill<<<ceil_div(n, 256), 256, 0, s>>>(A, alpha, B, rowscale ? 1.0 : -1.0, rowscale, C);
    SCR_LAUNCH();
  }
  counters().launches += 2;
  SCR_CUDA(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------ truncation
// Per block row: the candidates are the blocks with norm >= trunc * row max
// (and > 0); when more than pmax remain, the pmax-th candidate in the order
// (norm descending, column ascending) becomes the cut (cn, cc): a candidate
// is kept iff norm > cn or (norm == cn and col <= cc).
__global__ void k_trunc_select(DBsr<double> P, const double* __restrict__ norms, double trunc, int pmax,
                               double* __restrict__ tmin, double* __restrict__ cn, int* __restrict__ cc,
                               int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.nbr) return;
  const int s = P.rp[i], e = P.rp[i + 1];
  double m = 0.0;
  for (int t = s; t < e; ++t) m = fmax(m, norms[t]);
  const double lo = trunc * m;
  int ncand = 0;
  for (int t = s; t < e; ++t) ncand += (norms[t] > 0.0 && norms[t] >= lo);
  double pn = INFINITY;
  int pc = -1;
  int kept = ncand;
  if (pmax > 0 && ncand > pmax) {
    for (int q = 0; q < pmax; ++q) {
      double bn = -1.0;
      int bc = 0x7fffffff;
      for (int t = s; t < e; ++t) {
        const double v = norms[t];
        const int c = P.col[t];
        if (!(v > 0.0 && v >= lo)) continue;
        const bool after = v < pn || (v == pn && c > pc);
        if (!after) continue;
        if (v > bn || (v == bn && c < bc)) {
          bn = v;
          bc = c;
        }
      }
      pn = bn;
      pc = bc;
    }
    kept = pmax;
  } else {
    pn = -1.0;
    pc = 0x7fffffff;
  }
  tmin[i] = lo;
  cn[i] = pn;
  cc[i] = pc;
  cnt[i] = kept;
}

__device__ __forceinline__ bool trunc_kept(double v, int c, double lo, double cn, int cc) {
  return v > 0.0 && v >= lo && (v > cn || (v == cn && c <= cc));
}

__global__ void k_trunc_fill(DBsr<double> P, const double* __restrict__ norms, const double* __restrict__ tmin,
                             const double* __restrict__ cn, const int* __restrict__ cc, DBsr<double> O) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.nbr) return;
  const int BR = P.br, BC = P.bc;
  const int s = P.rp[i], k = P.rp[i + 1] - s;
  const int os = O.rp[i], ok = O.rp[i + 1] - os;
  for (int r = 0; r < BR; ++r) {
    double sall = 0.0, skept = 0.0;
    for (int t = 0; t < k; ++t) {
      const bool kp = trunc_kept(norms[s + t], P.col[s + t], tmin[i], cn[i], cc[i]);
      for (int c = 0; c < BC; ++c) {
        const double v = P.val[slab_index(s, k, t, r, c, BR, BC)];
        sall += v;
        if (kp) skept += v;
      }
    }
    const double sc = skept != 0.0 ? sall / skept : 1.0;
    int o = 0;
    for (int t = 0; t < k; ++t) {
      if (!trunc_kept(norms[s + t], P.col[s + t], tmin[i], cn[i], cc[i])) continue;
      if (r == 0) O.col[os + o] = P.col[s + t];
      for (int c = 0; c < BC; ++c) O.val[slab_index(os, ok, o, r, c, BR, BC)] = P.val[slab_index(s, k, t, r, c, BR, BC)] * sc;
      ++o;
    }
  }
}

__global__ void k_row_block_norms(DBsr<double> A, double* __restrict__ bnorm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nbr) return;
  const int s = A.rp[i], k = A.rp[i + 1] - s;
  for (int t = 0; t < k; ++t) {
    double acc = 0.0;
    for (int r = 0; r < A.br; ++r)
      for (int c = 0; c < A.bc; ++c) {
        const double v = A.val[slab_index(s, k, t, r, c, A.br, A.bc)];
        acc += v * v;
      }
    bnorm[s + t] = sqrt(acc);
  }
}

void truncate_rows(const DBsr<double>& P, double trunc, int pmax, DBsr<double>& O, DeviceArena& a, cudaStream_t s) {
  DeviceArena tmp(s);
  const int n = P.nbr;
  O.nbr = n;
  O.nbc = P.nbc;
  O.br = P.br;
  O.bc = P.bc;
  O.rp = a.alloc<int>(n + 1);
  double* norms = tmp.alloc<double>(P.nnzb + 1);
  double* tmin = tmp.alloc<double>(n + 1);
  double* cn = tmp.alloc<double>(n + 1);
  int* cc = tmp.alloc<int>(n + 1);
  int* cnt = tmp.alloc<int>(n + 1);
  if (n > 0) {
    k_row_block_norms<<<ceil_div(n, 256), 256, 0, s>>>(P, norms);
    k_trunc_select<<<ceil_div(n, 256), 256, 0, s>>>(P, norms, trunc, pmax, tmin, cn, cc, cnt);
    SCR_LAUNCH();
  }
  O.nnzb = exclusive_scan(cnt, O.rp, n, tmp, s);
  O.col = a.alloc<int>(O.nnzb + 1);
  O.val = a.alloc<double>(O.nnzb * O.br * O.bc + 1);
  if (n > 0) {
    k_trunc_fill<<<ceil_div(n, 256), 256, 0, s>>>(P, norms, tmin, cn, cc, O);
    SCR_LAUNCH();
  }
  counters().launches += 3;
  SCR_CUDA(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------ transpose
__global__ void k_tr_count(DBsr<double> A, int* __restrict__ cnt) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= A.nnzb) return;
  atomicAdd(cnt + A.col[t], 1);
}

__global__ void k_tr_rows(DBsr<double> A, int* __restrict__ cursor, int* __restrict__ ucol, int* __restrict__ usrc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nbr) return;
  for (int t = A.rp[i]; t < A.rp[i + 1]; ++t) {
    const int p = atomicAdd(cursor + A.col[t], 1);
    ucol[p] = i;
    usrc[p] = t;
  }
}

// one warp per row of T: rank-sort the (unordered) source rows, then copy
// the blocks transposed in that order
__global__ void k_tr_sort_fill(DBsr<double> A, DBsr<double> T, const int* __restrict__ ucol,
                               const int* __restrict__ usrc, int* __restrict__ ssrc) {
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= T.nbr) return;
  const int s = T.rp[j], e = T.rp[j + 1], k = e - s;
  for (int q = lane; q < k; q += 32) {
    const int v = ucol[s + q];
    int rank = 0;
    for (int p = 0; p < k; ++p) rank += ucol[s + p] < v;
    T.col[s + rank] = v;
    ssrc[s + rank] = usrc[s + q];
  }
  __syncwarp();
  const int bs = A.br * A.bc;
  for (int q = lane; q < k * bs; q += 32) {
    const int p = q / bs, rem = q - p * bs, r = rem / A.bc, c = rem - r * A.bc;
    const int t = ssrc[s + p];
    const int i = T.col[s + p];
    const int as = A.rp[i], ak = A.rp[i + 1] - as;
    T.val[slab_index(s, k, p, c, r, T.br, T.bc)] = A.val[slab_index(as, ak, t - as, r, c, A.br, A.bc)];
  }
}

void transpose(const DBsr<double>& A, DBsr<double>& T, DeviceArena& arena, cudaStream_t s) {
  DeviceArena tmp(s);
  T.nbr = A.nbc;
  T.nbc = A.nbr;
  T.br = A.bc;
  T.bc = A.br;
  T.nnzb = A.nnzb;
  T.rp = arena.alloc<int>(T.nbr + 1);
  T.col = arena.alloc<int>(A.nnzb + 1);
  T.val = arena.alloc<double>(A.nnzb * A.br * A.bc + 1);
  int* cnt = tmp.alloc<int>(T.nbr + 1);
  int* cursor = tmp.alloc<int>(T.nbr + 1);
  int* ucol = tmp.alloc<int>(A.nnzb + 1);
  int* usrc = tmp.alloc<int>(A.nnzb + 1);
  int* ssrc = tmp.alloc<int>(A.nnzb + 1);
  SCR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (T.nbr + 1), s));
  if (A.nnzb > 0) {
    k_tr_count<<<ceil_div(A.nnzb, 256), 256, 0, s>>>(A, cnt);
    SCR_LAUNCH();
  }
  exclusive_scan(cnt, T.rp, T.nbr, tmp, s);
  SCR_CUDA(cudaMemcpyAsync(cursor, T.rp, sizeof(int) * (T.nbr + 1), cudaMemcpyDeviceToDevice, s));
  if (A.nbr > 0) {
    k_tr_rows<<<ceil_div(A.nbr, 256), 256, 0, s>>>(A, cursor, ucol, usrc);
    SCR_LAUNCH();
  }
  if (T.nbr > 0) {
    k_tr_sort_fill<<<ceil_div((long long)T.nbr * 32, 256), 256, 0, s>>>(A, T, ucol, usrc, ssrc);
    SCR_LAUNCH();
  }
  counters().launches += 3;
  SCR_CUDA(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------ coarsest level
__global__ void k_to_dense(DBsr<double> A, double* __restrict__ M, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nbr) return;
  const int s = A.rp[i], k = A.rp[i + 1] - s;
  for (int t = 0; t < k; ++t) {
    const int j = A.col[s + t];
    for (int r = 0; r < A.br; ++r)
      for (int c = 0; c < A.bc; ++c)
        M[(long long)(i * A.br + r) + (long long)(j * A.bc + c) * n] = A.val[slab_index(s, k, t, r, c, A.br, A.bc)];
  }
}

void to_dense(const DBsr<double>& A, double* dense, cudaStream_t s) {
  const long long n = (long long)A.nbr * A.br;
  SCR_CUDA(cudaMemsetAsync(dense, 0, sizeof(double) * n * n, s));
  if (A.nbr == 0) return;
  k_to_dense<<<ceil_div(A.nbr, 128), 128, 0, s>>>(A, dense, (int)n);
  SCR_LAUNCH();
  counters().launches++;
}

// Gauss-Jordan with partial pivoting by one thread block; M and Inv
// column-major n x n; M is destroyed.
__global__ void __launch_bounds__(1024) k_gauss_jordan(double* __restrict__ M, double* __restrict__ Inv, int n,
                                                       int* __restrict__ singular) {
  extern __shared__ double colk[];
  __shared__ double rv[32];
  __shared__ int ri[32];
  __shared__ int piv;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (long long e = tid; e < (long long)n * n; e += nt) Inv[e] = (e % (n + 1) == 0) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    // pivot: argmax_{r >= k} |M[r, k]|
    double best = -1.0;
    int bi = k;
    for (int r = k + tid; r < n; r += nt) {
      const double v = fabs(M[r + (long long)k * n]);
      if (v > best) {
        best = v;
        bi = r;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if ((tid & 31) == 0) {
      rv[tid >> 5] = best;
      ri[tid >> 5] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      double b = -1.0;
      int p = k;
      for (int w = 0; w < nt / 32; ++w)
        if (rv[w] > b || (rv[w] == b && ri[w] < p)) {
          b = rv[w];
          p = ri[w];
        }
      piv = p;
      if (!(b > 0.0)) *singular = 1;
    }
    __syncthreads();
    const int p = piv;
    if (p != k) {
      for (int c = tid; c < n; c += nt) {
        double t = M[k + (long long)c * n];
        M[k + (long long)c * n] = M[p + (long long)c * n];
        M[p + (long long)c * n] = t;
        t = Inv[k + (long long)c * n];
        Inv[k + (long long)c * n] = Inv[p + (long long)c * n];
        Inv[p + (long long)c * n] = t;
      }
    }
    __syncthreads();
    const double d = M[k + (long long)k * n];
    const double dinv = d != 0.0 ? 1.0 / d : 0.0;
    __syncthreads();
    for (int c = tid; c < n; c += nt) {
      M[k + (long long)c * n] *= dinv;
      Inv[k + (long long)c * n] *= dinv;
    }
    for (int r = tid; r < n; r += nt) colk[r] = M[r + (long long)k * n];
    __syncthreads();
    for (long long e = tid; e < (long long)n * n; e += nt) {
      const int r = (int)(e % n), c = (int)(e / n);
      if (r == k) continue;
      const double f = colk[r];
      if (f != 0.0) {
        M[e] -= f * M[k + (long long)c * n];
        Inv[e] -= f * Inv[k + (long long)c * n];
      }
    }
    __syncthreads();
  }
}

void dense_inverse(double* M, double* inv, int n, int* singular, cudaStream_t s) {
  if (n == 0) return;
  k_gauss_jordan<<<1, 1024, sizeof(double) * n, s>>>(M, inv, n, singular);
  SCR_LAUNCH();
  counters().launches++;
}

template <typename T>
__global__ void k_dense_apply(const T* __restrict__ inv, const T* __restrict__ b, T* __restrict__ x, int n,
                              int nrhs) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n * nrhs) return;
  const int i = o / nrhs, h = o - i * nrhs;
  T acc = 0;
  for (int j = 0; j < n; ++j) acc = fma(inv[i + (long long)j * n], b[(long long)j * nrhs + h], acc);
  x[o] = acc;
}

void dense_apply(const double* inv, const double* b, double* x, int n, int nrhs, cudaStream_t s) {
  if (n == 0) return;
  k_dense_apply<double><<<ceil_div((long long)n * nrhs, 128), 128, 0, s>>>(inv, b, x, n, nrhs);
  SCR_LAUNCH();
  counters().launches++;
}
void dense_apply_f(const float* inv, const float* b, float* x, int n, int nrhs, cudaStream_t s) {
  if (n == 0) return;
  k_dense_apply<float><<<ceil_div((long long)n * nrhs, 128), 128, 0, s>>>(inv, b, x, n, nrhs);
  SCR_LAUNCH();
  counters().launches++;
}

}  // namespace scr

// ------------------------------------------------------------ numeric re-set-up
// The values of a set-up's products for new operator values on unchanged
// patterns (scr_update_values): every output keeps the sparsity pattern of
// the first set-up, only its values are recomputed.
namespace scr {

void spgemm_numeric(const DBsr<double>& A, const DBsr<double>& B, DBsr<double>& C, cudaStream_t s) {
  if (A.nbr == 0 || C.nnzb == 0) return;
  const int grid = ceil_div(A.nbr, kSpgemmWarps);
  const int br = A.br, bk = A.bc, bc = B.bc;
  if (br == 3 && bk == 3 && bc == 3) k_spgemm_numeric<3, 3, 3><<<grid, 32 * kSpgemmWarps, 0, s>>>(A, B, C);
  else if (br == 1 && bk == 3 && bc == 1) k_spgemm_numeric<1, 3, 1><<<grid, 32 * kSpgemmWarps, 0, s>>>(A, B, C);
  else if (br == 1 && bk == 1 && bc == 1) k_spgemm_numeric<1, 1, 1><<<grid, 32 * kSpgemmWarps, 0, s>>>(A, B, C);
  else throw CudaError{cudaErrorInvalidValue, "spgemm_numeric: unsupported block shape"};
  SCR_LAUNCH();
  counters().launches++;
}

void spadd_numeric(const DBsr<double>& A, double alpha, const DBsr<double>& B, const double* rowscale,
                   DBsr<double>& C, cudaStream_t s) {
  if (A.nbr == 0) return;
  // the fill pass of spadd: the union pattern is rewritten with the same columns
  k_spadd_fill<<<ceil_div(A.nbr, 256), 256, 0, s>>>(A, alpha, B, rowscale ? 1.0 : -1.0, rowscale, C);
  SCR_LAUNCH();
  counters().launches++;
}

void scale_rows_inv_values(const DBsr<double>& M, const double* d, double* out, cudaStream_t s) {
  const long long n = (long long)M.nbr * M.br;
  if (n == 0) return;
  k_scale_rows_inv<<<ceil_div(n, 256), 256, 0, s>>>(M, d, out);
  SCR_LAUNCH();
  counters().launches++;
}

// O keeps its kept columns (a subset of P's row, both sorted); per scalar row
// r its values are P's at those columns times sum_all / sum_kept of P's row
// r, the row-sum preserving rescaling of the truncation
__global__ void k_trunc_refill(DBsr<double> P, DBsr<double> O) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.nbr) return;
  const int BR = P.br, BC = P.bc;
  const int s = P.rp[i], k = P.rp[i + 1] - s;
  const int os = O.rp[i], ok = O.rp[i + 1] - os;
  for (int r = 0; r < BR; ++r) {
    double sall = 0.0, skept = 0.0;
    int o = 0;
    for (int t = 0; t < k; ++t) {
      const bool kp = o < ok && O.col[os + o] == P.col[s + t];
      for (int c = 0; c < BC; ++c) {
        const double v = P.val[slab_index(s, k, t, r, c, BR, BC)];
        sall += v;
        if (kp) skept += v;
      }
      if (kp) ++o;
    }
    const double sc = skept != 0.0 ? sall / skept : 1.0;
    o = 0;
    for (int t = 0; t < k && o < ok; ++t) {
      if (O.col[os + o] != P.col[s + t]) continue;
      for (int c = 0; c < BC; ++c)
        O.val[slab_index(os, ok, o, r, c, BR, BC)] = P.val[slab_index(s, k, t, r, c, BR, BC)] * sc;
      ++o;
    }
  }
}

void truncate_refill(const DBsr<double>& P, DBsr<double>& O, cudaStream_t s) {
  if (P.nbr == 0) return;
  k_trunc_refill<<<ceil_div(P.nbr, 256), 256, 0, s>>>(P, O);
  SCR_LAUNCH();
  counters().launches++;
}

// T = A^T on T's existing pattern: every stored block (i, j) of A is found in
// row j of T by binary search and written transposed
__global__ void k_transpose_values(DBsr<double> A, DBsr<double> T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.nbr) return;
  const int BR = A.br, BC = A.bc;
  const int s = A.rp[i], k = A.rp[i + 1] - s;
  for (int t = 0; t < k; ++t) {
    const int j = A.col[s + t];
    int lo = T.rp[j], hi = T.rp[j + 1] - 1;
    const int ts = lo, tk = hi + 1 - lo;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (T.col[mid] < i) lo = mid + 1;
      else hi = mid;
    }
    if (lo > hi || T.col[lo] != i) continue;  // not in the pattern (cannot happen for a transpose)
    for (int r = 0; r < BR; ++r)
      for (int c = 0; c < BC; ++c)
        T.val[slab_index(ts, tk, lo - ts, c, r, BC, BR)] = A.val[slab_index(s, k, t, r, c, BR, BC)];
  }
}

void transpose_numeric(const DBsr<double>& A, DBsr<double>& T, cudaStream_t s) {
  if (A.nbr == 0) return;
  k_transpose_values<<<ceil_div(A.nbr, 256), 256, 0, s>>>(A, T);
  SCR_LAUNCH();
  counters().launches++;
}

}  // namespace scr
