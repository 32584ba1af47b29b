// Vector kernels of the Krylov solvers: deterministic two-stage reductions
// (fixed grid, per-block partial sums reduced in a fixed order), the two
// classical Gram-Schmidt passes of FGMRES/GMRES fused with their dot
// products, Givens rotations of the Hessenberg least-squares problem on the
// device, and the CG recurrences.
#include <algorithm>

#include "kernels.h"

namespace scr {

static constexpr int kRedThreads = 256;

Reducer make_reducer(DeviceArena& a) {
  Reducer r;
  r.nblk = std::min(2 * sm_count(), 1024);
  r.partial = a.alloc<double>((size_t)r.nblk * kMaxBasis);
  return r;
}

// ------------------------------------------------------------ simple ops
template <typename T>
__global__ void k_fill(T* x, T v, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += st) x[i] = v;
}
template <typename T>
__global__ void k_copy(const T* __restrict__ x, T* __restrict__ y, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += st) y[i] = x[i];
}
__global__ void k_f2d(const float* __restrict__ x, double* __restrict__ y, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += st) y[i] = (double)x[i];
}
__global__ void k_d2f_b(const double* __restrict__ x, float* __restrict__ y, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += st) y[i] = (float)x[i];
}
__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += st) y[i] = a * x[i] + b * y[i];
}
template <typename T>
__global__ void k_scale_by(const T* __restrict__ x, const double* __restrict__ sc, T* __restrict__ y, long long n) {
  const T a = (T)*sc;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += st) y[i] = a * x[i];
}
// y = x (times *sc when sc is given), with x and/or y a column of a basis
// whose index is read on the device: column (*xj) of X, column (*yj + yoff)
// of Y (stride ld); a null index pointer names the vector itself
template <typename T>
__global__ void k_col_copy(const T* __restrict__ X, const int* __restrict__ xj, T* __restrict__ Y,
                           const int* __restrict__ yj, int yoff, long long ld, const double* __restrict__ sc,
                           long long n) {
  const T* x = xj ? X + (long long)*xj * ld : X;
  T* y = yj ? Y + (long long)(*yj + yoff) * ld : Y;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  if (sc) {
    const T a = (T)*sc;
    for (; i < n; i += st) y[i] = a * x[i];
  } else {
    for (; i < n; i += st) y[i] = x[i];
  }
}

static int grid_for(long long n) {
  return (int)std::max<long long>(1, std::min<long long>(ceil_div(n, 256), 8LL * sm_count()));
}

template <typename T>
void fill(T* x, T v, long long n, cudaStream_t s) {
  if (n <= 0) return;
  k_fill<T><<<grid_for(n), 256, 0, s>>>(x, v, n);
  SCR_LAUNCH();
  counters().launches++;
}
template void fill<double>(double*, double, long long, cudaStream_t);
template void fill<float>(float*, float, long long, cudaStream_t);
template void fill<int>(int*, int, long long, cudaStream_t);

template <typename T>
void copy(const T* x, T* y, long long n, cudaStream_t s) {
  if (n <= 0) return;
  k_copy<T><<<grid_for(n), 256, 0, s>>>(x, y, n);
  SCR_LAUNCH();
  counters().launches++;
}
template void copy<double>(const double*, double*, long long, cudaStream_t);
template void copy<float>(const float*, float*, long long, cudaStream_t);
template void copy<int>(const int*, int*, long long, cudaStream_t);

// y += (c * dot[0]) a  (dot: a device scalar)
template <typename T>
__global__ void k_axpy_dev(const T* __restrict__ a, const double* __restrict__ dot, double c, T* __restrict__ y,
                           long long n) {
  const double f = c * dot[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += (T)(f * (double)a[i]);
}
template <typename T>
void axpy_dev(const T* a, const double* dot, double c, T* y, long long n, cudaStream_t s) {
  if (n == 0) return;
  k_axpy_dev<T><<<grid_for(n), 256, 0, s>>>(a, dot, c, y, n);
  SCR_LAUNCH();
  counters().launches++;
}
template void axpy_dev<double>(const double*, const double*, double, double*, long long, cudaStream_t);
template void axpy_dev<float>(const float*, const double*, double, float*, long long, cudaStream_t);

// d[i] += c a[i]^2
__global__ void k_add_sq(double* __restrict__ d, const double* __restrict__ a, double c, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) d[i] += c * a[i] * a[i];
}
void add_scaled_squares(double* d, const double* a, double c, long long n, cudaStream_t s) {
  if (n == 0) return;
  k_add_sq<<<ceil_div(n, 256), 256, 0, s>>>(d, a, c, n);
  SCR_LAUNCH();
  counters().launches++;
}

// b = -R on the first n entries with the rows of flagged nodes (3 rows per
// node on the first nv3 entries) set to zero; mask may be null
__global__ void k_neg_masked(const double* __restrict__ R, const unsigned char* __restrict__ mask,
                             double* __restrict__ b, long long nv3, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  b[i] = (mask && i < nv3 && mask[i / 3]) ? 0.0 : -R[i];
}
void negate_masked(const double* R, const unsigned char* mask, double* b, long long nv3, long long n,
                   cudaStream_t s) {
  if (n == 0) return;
  k_neg_masked<<<ceil_div(n, 256), 256, 0, s>>>(R, mask, b, nv3, n);
  SCR_LAUNCH();
  counters().launches++;
}

// Dirichlet data of the mesh-motion problem at t_{n+1}: the interface nodes
// take the solid displacement u_{n+1} = u_n + (u_{n+alpha_f} - u_n) / alpha_f
// of their node, the other Dirichlet nodes zero (the entries of free nodes
// are never read as data: mesh_lift keeps g only on Dirichlet rows)
__global__ void k_mesh_data(const int* __restrict__ node_of_f, const unsigned char* __restrict__ follow,
                            const double* __restrict__ u, const double* __restrict__ un, double af,
                            double* __restrict__ g, long long n3) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const long long f = i / 3, c = i - 3 * f;
  const long long j = 3LL * node_of_f[f] + c;
  g[i] = follow[f] ? un[j] + (u[j] - un[j]) / af : 0.0;
}
void mesh_interface_data(const int* node_of_f, const unsigned char* follow, const double* u, const double* un,
                         double af, double* g, int nf, cudaStream_t s) {
  const long long n3 = 3LL * nf;
  if (n3 == 0) return;
  k_mesh_data<<<ceil_div(n3, 256), 256, 0, s>>>(node_of_f, follow, u, un, af, g, n3);
  SCR_LAUNCH();
  counters().launches++;
}

// right-hand side of the Dirichlet-eliminated mesh system: g on Dirichlet
// rows, -(L_raw g) on the free rows (the lift of the boundary data)
__global__ void k_mesh_lift(const unsigned char* __restrict__ dir_m, const double* __restrict__ g,
                            double* __restrict__ b, long long n3) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n3) return;
  b[i] = dir_m[i / 3] ? g[i] : -b[i];
}
void mesh_lift(const unsigned char* dir_m, const double* g, double* b, int nf, cudaStream_t s) {
  const long long n3 = 3LL * nf;
  if (n3 == 0) return;
  k_mesh_lift<<<ceil_div(n3, 256), 256, 0, s>>>(dir_m, g, b, n3);
  SCR_LAUNCH();
  counters().launches++;
}

// mesh velocity at t_{n+1} from the displacements, then at t_{n+alpha_f}
// (generalized-alpha, Sec. 3.4), written at the fluid nodes
__global__ void k_mesh_velocity(const int* __restrict__ node_of_f, const double* __restrict__ uh,
                                const double* __restrict__ uhn, const double* __restrict__ vn, double af,
                                double gdt, double cv, double* __restrict__ vhat, long long n3) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const long long f = i / 3, c = i - 3 * f;
  const double v0 = vn[i];
  const double v1 = (uh[i] - uhn[i]) / gdt + cv * v0;
  vhat[3LL * node_of_f[f] + c] = v0 + af * (v1 - v0);
}
void mesh_velocity(const int* node_of_f, const double* uh, const double* uhn, const double* vn, double af,
                   double gamma, double dt, double* vhat, int nf, cudaStream_t s) {
  const long long n3 = 3LL * nf;
  if (n3 == 0) return;
  k_mesh_velocity<<<ceil_div(n3, 256), 256, 0, s>>>(node_of_f, uh, uhn, vn, af, gamma * dt,
                                                    (gamma - 1.0) / gamma, vhat, n3);
  SCR_LAUNCH();
  counters().launches++;
}

// y[i] = 1 / x[i]
__global__ void k_recip(const double* __restrict__ x, double* __restrict__ y, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) y[i] = 1.0 / x[i];
}
void reciprocal(const double* x, double* y, long long n, cudaStream_t s) {
  if (n == 0) return;
  k_recip<<<ceil_div(n, 256), 256, 0, s>>>(x, y, n);
  SCR_LAUNCH();
  counters().launches++;
}

// k vectors of length n stored one after another (in[c * n + i]) <->
// interleaved (out[i * k + c])
__global__ void k_interleave(const double* __restrict__ in, double* __restrict__ out, long long n, int k,
                             int to_interleaved) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const long long i = t / k, c = t - i * k;  // t walks the interleaved layout
  if (to_interleaved) out[t] = in[c * n + i];
  else out[c * n + i] = in[t];
}

void interleave(const double* in, double* out, long long n, int k, bool to_interleaved, cudaStream_t s) {
  if (n * k == 0) return;
  k_interleave<<<ceil_div(n * k, 256), 256, 0, s>>>(in, out, n, k, to_interleaved ? 1 : 0);
  SCR_LAUNCH();
  counters().launches++;
}

void cast_d2f(const double* x, float* y, long long n, cudaStream_t s) {
  if (n <= 0) return;
  k_d2f_b<<<grid_for(n), 256, 0, s>>>(x, y, n);
  SCR_LAUNCH();
  counters().launches++;
}
void cast_f2d(const float* x, double* y, long long n, cudaStream_t s) {
  if (n <= 0) return;
  k_f2d<<<grid_for(n), 256, 0, s>>>(x, y, n);
  SCR_LAUNCH();
  counters().launches++;
}
void axpby(double a, const double* x, double b, double* y, long long n, cudaStream_t s) {
  if (n <= 0) return;
  k_axpby<<<grid_for(n), 256, 0, s>>>(a, x, b, y, n);
  SCR_LAUNCH();
  counters().launches++;
}
template <typename T>
void scale_by(const T* x, const double* sc, T* y, long long n, cudaStream_t s) {
  if (n <= 0) return;
  k_scale_by<T><<<grid_for(n), 256, 0, s>>>(x, sc, y, n);
  SCR_LAUNCH();
  counters().launches++;
}

template void scale_by<double>(const double*, const double*, double*, long long, cudaStream_t);

template <typename T>
void col_copy(const T* X, const int* xj, T* Y, const int* yj, int yoff, long long ld, const double* sc, long long n,
              cudaStream_t s) {
  if (n <= 0) return;
  k_col_copy<T><<<grid_for(n), 256, 0, s>>>(X, xj, Y, yj, yoff, ld, sc, n);
  SCR_LAUNCH();
  counters().launches++;
}
template void col_copy<double>(const double*, const int*, double*, const int*, int, long long, const double*,
                               long long, cudaStream_t);
template void col_copy<float>(const float*, const int*, float*, const int*, int, long long, const double*,
                              long long, cudaStream_t);

template <typename T>
__global__ void k_axpby_t(T a, const T* __restrict__ x, T b, T* __restrict__ y, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += st) y[i] = a * x[i] + b * y[i];
}
template <typename T>
void axpby_t(double a, const T* x, double b, T* y, long long n, cudaStream_t s) {
  if (n <= 0) return;
  k_axpby_t<T><<<grid_for(n), 256, 0, s>>>((T)a, x, (T)b, y, n);
  SCR_LAUNCH();
  counters().launches++;
}
template void axpby_t<double>(double, const double*, double, double*, long long, cudaStream_t);
template void axpby_t<float>(double, const float*, double, float*, long long, cudaStream_t);

// x[o*nrhs+h] = b[o*nrhs+h] * d[o]
template <typename T>
__global__ void k_diag_scale(const T* __restrict__ b, const T* __restrict__ d, T* __restrict__ x, long long n,
                             int nrhs) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  for (; i < n * nrhs; i += st) x[i] = b[i] * d[i / nrhs];
}
template <typename T>
void diag_scale(const T* b, const T* d, T* x, long long n, int nrhs, cudaStream_t s) {
  if (n <= 0) return;
  k_diag_scale<T><<<grid_for(n * nrhs), 256, 0, s>>>(b, d, x, n, nrhs);
  SCR_LAUNCH();
  counters().launches++;
}
template void diag_scale<double>(const double*, const double*, double*, long long, int, cudaStream_t);

template <typename T>
__global__ void k_cheb_zero(const T* __restrict__ b, const T* __restrict__ d, T* __restrict__ r, T* __restrict__ dv,
                            T* __restrict__ x, T inv_theta, long long n, int nrhs) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  for (; i < n * nrhs; i += st) {
    const T ri = b[i] * d[i / nrhs];
    const T di = ri * inv_theta;
    r[i] = ri;
    dv[i] = di;
    x[i] = di;
  }
}
template <typename T>
void cheb_zero(const T* b, const T* d, T* r, T* dv, T* x, double inv_theta, long long n, int nrhs, cudaStream_t s) {
  if (n <= 0) return;
  k_cheb_zero<T><<<grid_for(n * nrhs), 256, 0, s>>>(b, d, r, dv, x, (T)inv_theta, n, nrhs);
  SCR_LAUNCH();
  counters().launches++;
}
template void cheb_zero<double>(const double*, const double*, double*, double*, double*, double, long long, int,
                                cudaStream_t);
template void cheb_zero<float>(const float*, const float*, float*, float*, float*, double, long long, int,
                               cudaStream_t);
template void diag_scale<float>(const float*, const float*, float*, long long, int, cudaStream_t);
template void scale_by<float>(const float*, const double*, float*, long long, cudaStream_t);

// ------------------------------------------------------------ reductions
// Reduce KMAX per-thread sums over the block and write them to
// partial[blockIdx.x * kMaxBasis + j].
template <int KMAX>
__device__ __forceinline__ void block_store_partials(double (&acc)[KMAX], int k, double* partial) {
  __shared__ double sm[kRedThreads / 32][KMAX];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    if (j < k) {
      double v = warp_sum(acc[j]);
      if (lane == 0) sm[wid][j] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < kRedThreads / 32; ++w) v += sm[w][threadIdx.x];
    partial[(long long)blockIdx.x * kMaxBasis + threadIdx.x] = v;
  }
}

// partial sums of V_j . w
// per-thread sums in the vector precision T, block and grid sums in FP64
template <int KMAX, typename T>
__device__ __forceinline__ void store_partials_t(T (&acc)[KMAX], int k, double* partial) {
  double d[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) d[j] = (double)acc[j];
  block_store_partials<KMAX>(d, k, partial);
}

// Counts: k, or (*kp + koff) when kp is given (a count kept on the device
// by a loop recorded in a CUDA graph; KMAX bounds it either way).
template <int KMAX, typename T>
__global__ void __launch_bounds__(kRedThreads) k_multidot(const T* __restrict__ V, long long ld, int k,
                                                         const T* __restrict__ w, long long n,
                                                         double* __restrict__ partial, const int* __restrict__ kp,
                                                         int koff) {
  if (kp) k = *kp + koff;
  T acc[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) acc[j] = (T)0;
  const long long st = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += st) {
    const T wi = w[i];
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < k) acc[j] = fma(V[j * ld + i], wi, acc[j]);
  }
  store_partials_t<KMAX, T>(acc, k, partial);
}

// w -= V h; partial sums of V_j . w (new)
template <int KMAX, typename T>
__global__ void __launch_bounds__(kRedThreads) k_cgs_update_dot(const T* __restrict__ V, long long ld, int k,
                                                               const double* __restrict__ h, T* __restrict__ w,
                                                               long long n, double* __restrict__ partial,
                                                               const int* __restrict__ kp, int koff) {
  if (kp) k = *kp + koff;
  T hj[KMAX], acc[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    hj[j] = j < k ? (T)h[j] : (T)0;
    acc[j] = (T)0;
  }
  const long long st = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += st) {
    T wi = w[i];
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < k) wi = fma(-V[j * ld + i], hj[j], wi);
    w[i] = wi;
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < k) acc[j] = fma(V[j * ld + i], wi, acc[j]);
  }
  store_partials_t<KMAX, T>(acc, k, partial);
}

// w -= V h; partial sum of w . w
template <int KMAX, typename T>
__global__ void __launch_bounds__(kRedThreads) k_cgs_update_norm(const T* __restrict__ V, long long ld, int k,
                                                                const double* __restrict__ h, T* __restrict__ w,
                                                                long long n, double* __restrict__ partial,
                                                                const int* __restrict__ kp, int koff) {
  if (kp) k = *kp + koff;
  T hj[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) hj[j] = j < k ? (T)h[j] : (T)0;
  T acc[1] = {(T)0};
  const long long st = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += st) {
    T wi = w[i];
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < k) wi = fma(-V[j * ld + i], hj[j], wi);
    w[i] = wi;
    acc[0] = fma(wi, wi, acc[0]);
  }
  store_partials_t<1, T>(acc, 1, partial);
}

// Device-count variants (loops recorded in a CUDA graph): the count k is
// read on the device, so the dot products are taken kDotTile columns at a time
// with a fixed register tile, one pass over the rows per chunk (a single
// pass for k <= kDotTile, the usual case of the inner solves).  Per column
// they do the same multiply-adds in the same order as the fixed-count
// kernels above and store the same block partial sums, so the results are
// bit-identical; the fixed-count kernels sized for the largest count would
// hold kMaxBasis accumulators per thread instead.
constexpr int kDotTile = 8;

// block partial sums of columns c0 .. c0 + kDotTile - 1 (those < k), as
// block_store_partials stores them
template <typename T>
__device__ __forceinline__ void store_chunk_partials(const T (&acc)[kDotTile], int c0, int k, double* partial) {
  __shared__ double sm[kRedThreads / 32][kDotTile];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kDotTile; ++j) {
    if (c0 + j < k) {
      double v = warp_sum((double)acc[j]);
      if (lane == 0) sm[wid][j] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < kDotTile && c0 + (int)threadIdx.x < k) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < kRedThreads / 32; ++w) v += sm[w][threadIdx.x];
    partial[(long long)blockIdx.x * kMaxBasis + c0 + threadIdx.x] = v;
  }
  __syncthreads();  // sm is reused by the next chunk
}

template <typename T>
__device__ __forceinline__ void chunk_dots(const T* __restrict__ V, long long ld, int c0, int k,
                                           const T* __restrict__ w, long long n, double* __restrict__ partial) {
  T acc[kDotTile];
#pragma unroll
  for (int j = 0; j < kDotTile; ++j) acc[j] = (T)0;
  const long long st = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += st) {
    const T wi = w[i];
#pragma unroll
    for (int j = 0; j < kDotTile; ++j)
      if (c0 + j < k) acc[j] = fma(V[(c0 + j) * ld + i], wi, acc[j]);
  }
  store_chunk_partials<T>(acc, c0, k, partial);
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_multidot_dev(const T* __restrict__ V, long long ld,
                                                             const int* __restrict__ kp, int koff,
                                                             const T* __restrict__ w, long long n,
                                                             double* __restrict__ partial) {
  const int k = *kp + koff;
  for (int c0 = 0; c0 < k; c0 += kDotTile) chunk_dots<T>(V, ld, c0, k, w, n, partial);
}

// w -= V h (columns in increasing order), then the dots of the updated w
// (NORM: its squared norm only)
template <bool NORM, typename T>
__global__ void __launch_bounds__(kRedThreads) k_cgs_update_dev(const T* __restrict__ V, long long ld,
                                                               const int* __restrict__ kp, int koff,
                                                               const double* __restrict__ h, T* __restrict__ w,
                                                               long long n, double* __restrict__ partial) {
  __shared__ T hs[kMaxBasis + 1];
  const int k = *kp + koff;
  for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = (T)h[j];
  __syncthreads();
  T acc[kDotTile];
#pragma unroll
  for (int j = 0; j < kDotTile; ++j) acc[j] = (T)0;
  const long long st = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += st) {
    T wi = w[i];
#pragma unroll 4
    for (int j = 0; j < k; ++j) wi = fma(-V[j * ld + i], hs[j], wi);
    w[i] = wi;
    if constexpr (NORM) {
      acc[0] = fma(wi, wi, acc[0]);
    } else {
#pragma unroll
      for (int j = 0; j < kDotTile; ++j)
        if (j < k) acc[j] = fma(V[j * ld + i], wi, acc[j]);
    }
  }
  if constexpr (NORM) {
    store_chunk_partials<T>(acc, 0, 1, partial);
  } else {
    store_chunk_partials<T>(acc, 0, k, partial);
    for (int c0 = kDotTile; c0 < k; c0 += kDotTile) chunk_dots<T>(V, ld, c0, k, w, n, partial);
  }
}

// out[j] = sum_b partial[b][j], fixed order
__global__ void k_reduce_partials(const double* __restrict__ partial, int nblk, int k, double* __restrict__ out,
                                  const int* __restrict__ kp, int koff) {
  if (kp) k = *kp + koff;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wid; j < k; j += nw) {
    double v = 0.0;
    for (int b = lane; b < nblk; b += 32) v += partial[(long long)b * kMaxBasis + j];
    v = warp_sum(v);
    if (lane == 0) out[j] = v;
  }
}

template <int KMAX, typename T>
static void launch_multidot(const T* V, long long ld, int k, const T* w, long long n, const Reducer& r,
                            cudaStream_t s, const int* kp, int koff) {
  k_multidot<KMAX, T><<<r.nblk, kRedThreads, 0, s>>>(V, ld, k, w, n, r.partial, kp, koff);
}
template <int KMAX, typename T>
static void launch_cgs_dot(const T* V, long long ld, int k, const double* h, T* w, long long n, const Reducer& r,
                           cudaStream_t s, const int* kp, int koff) {
  k_cgs_update_dot<KMAX, T><<<r.nblk, kRedThreads, 0, s>>>(V, ld, k, h, w, n, r.partial, kp, koff);
}
template <int KMAX, typename T>
static void launch_cgs_norm(const T* V, long long ld, int k, const double* h, T* w, long long n, const Reducer& r,
                            cudaStream_t s, const int* kp, int koff) {
  k_cgs_update_norm<KMAX, T><<<r.nblk, kRedThreads, 0, s>>>(V, ld, k, h, w, n, r.partial, kp, koff);
}

#define SCR_KDISPATCH(FN, T, k, ...)                \
  do {                                              \
    if ((k) <= 1) FN<1, T>(__VA_ARGS__);            \
    else if ((k) <= 4) FN<4, T>(__VA_ARGS__);       \
    else if ((k) <= 8) FN<8, T>(__VA_ARGS__);       \
    else if ((k) <= 16) FN<16, T>(__VA_ARGS__);     \
    else if ((k) <= 32) FN<32, T>(__VA_ARGS__);     \
    else FN<kMaxBasis, T>(__VA_ARGS__);             \
  } while (0)

static void reduce(const Reducer& r, int k, double* out, cudaStream_t s, const int* kp = nullptr, int koff = 0) {
  k_reduce_partials<<<1, 256, 0, s>>>(r.partial, r.nblk, k, out, kp, koff);
  SCR_LAUNCH();
  counters().launches += 2;
}

template <typename T>
void norm2(const T* x, long long n, double* out, const Reducer& r, cudaStream_t s) {
  launch_multidot<1, T>(x, 0, 1, x, n, r, s, nullptr, 0);
  SCR_LAUNCH();
  reduce(r, 1, out, s);
}

template <typename T>
void multidot(const T* V, long long ld, int k, const T* w, long long n, double* out, const Reducer& r,
              cudaStream_t s, const int* kp, int koff) {
  if (kp) k_multidot_dev<T><<<r.nblk, kRedThreads, 0, s>>>(V, ld, kp, koff, w, n, r.partial);
  else SCR_KDISPATCH(launch_multidot, T, k, V, ld, k, w, n, r, s, kp, koff);
  SCR_LAUNCH();
  reduce(r, k, out, s, kp, koff);
}

template <typename T>
void cgs_update_dot(const T* V, long long ld, int k, const double* h, T* w, long long n, double* out,
                    const Reducer& r, cudaStream_t s, const int* kp, int koff) {
  if (kp) k_cgs_update_dev<false, T><<<r.nblk, kRedThreads, 0, s>>>(V, ld, kp, koff, h, w, n, r.partial);
  else SCR_KDISPATCH(launch_cgs_dot, T, k, V, ld, k, h, w, n, r, s, kp, koff);
  SCR_LAUNCH();
  reduce(r, k, out, s, kp, koff);
}

template <typename T>
void cgs_update_norm(const T* V, long long ld, int k, const double* h, T* w, long long n, double* out,
                     const Reducer& r, cudaStream_t s, const int* kp, int koff) {
  if (kp) k_cgs_update_dev<true, T><<<r.nblk, kRedThreads, 0, s>>>(V, ld, kp, koff, h, w, n, r.partial);
  else SCR_KDISPATCH(launch_cgs_norm, T, k, V, ld, k, h, w, n, r, s, kp, koff);
  SCR_LAUNCH();
  reduce(r, 1, out, s);
}

#define SCR_INST_BLAS(T)                                                                                      \
  template void norm2<T>(const T*, long long, double*, const Reducer&, cudaStream_t);                         \
  template void multidot<T>(const T*, long long, int, const T*, long long, double*, const Reducer&,           \
                            cudaStream_t, const int*, int);                                                   \
  template void cgs_update_dot<T>(const T*, long long, int, const double*, T*, long long, double*,            \
                                  const Reducer&, cudaStream_t, const int*, int);                             \
  template void cgs_update_norm<T>(const T*, long long, int, const double*, T*, long long, double*,           \
                                   const Reducer&, cudaStream_t, const int*, int);
SCR_INST_BLAS(double)
SCR_INST_BLAS(float)

// ------------------------------------------------------------ Arnoldi scalars
// One warp: the lanes load column j of H (the two Gram-Schmidt passes'
// coefficients) and the previous rotations into shared memory in parallel,
// lane 0 applies the rotations and the new one there (the same operations
// in the same order as a single thread on the state), the lanes write the
// column back.
__global__ void k_arnoldi_finalize(ArnoldiState* st, int j, double* host_rel, const int* __restrict__ jp) {
  if (jp) j = *jp;
  constexpr int ldh = kMaxBasis + 1;
  __shared__ double h[kMaxBasis + 2], rc[kMaxBasis], rs[kMaxBasis];
  const int t = threadIdx.x;
  double* Hj = st->H + (long long)j * ldh;
  for (int i = t; i <= j; i += 32) h[i] = st->h1[i] + st->h2[i];
  for (int i = t; i < j; i += 32) {
    rc[i] = st->cs[i];
    rs[i] = st->sn[i];
  }
  __syncwarp();
  if (t == 0) {
    const double hn = sqrt(fmax(st->nrm2, 0.0));
    h[j + 1] = hn;
    // previous rotations
    for (int i = 0; i < j; ++i) {
      const double v = rc[i] * h[i] + rs[i] * h[i + 1];
      h[i + 1] = -rs[i] * h[i] + rc[i] * h[i + 1];
      h[i] = v;
    }
    const double a = h[j], c = h[j + 1];
    const double d = hypot(a, c);
    double cs = 1.0, sn = 0.0;
    if (d != 0.0) {
      cs = a / d;
      sn = c / d;
    }
    st->cs[j] = cs;
    st->sn[j] = sn;
    h[j] = d;
    h[j + 1] = 0.0;
    const double gj = st->g[j];
    st->g[j + 1] = -sn * gj;
    st->g[j] = cs * gj;
    st->rel = fabs(st->g[j + 1]) / st->bnorm;
    // happy breakdown: the new direction vanished relative to the column
    st->breakdown = (hn <= 1e-300 || d == 0.0) ? 1 : 0;
    st->inv_hnext = hn > 1e-300 ? 1.0 / hn : 0.0;
    if (host_rel) {
      host_rel[0] = st->rel;
      host_rel[1] = (double)st->breakdown;
    }
  }
  __syncwarp();
  for (int i = t; i <= j + 1; i += 32) Hj[i] = h[i];
}

void arnoldi_finalize(ArnoldiState* st, int j, double* host_rel, cudaStream_t s, const int* jp) {
  k_arnoldi_finalize<<<1, 32, 0, s>>>(st, j, host_rel, jp);
  SCR_LAUNCH();
  counters().launches++;
}

__global__ void k_arnoldi_start(ArnoldiState* st, int first, double* host_rel) {
  const double beta = sqrt(fmax(st->nrm2, 0.0));
  st->beta = beta;
  if (first) st->bnorm = beta;
  for (int i = 0; i <= kMaxBasis; ++i) st->g[i] = 0.0;
  st->g[0] = beta;
  st->inv_hnext = beta > 0.0 ? 1.0 / beta : 0.0;
  st->rel = st->bnorm > 0.0 ? beta / st->bnorm : 0.0;
  st->breakdown = 0;
  if (host_rel) {
    host_rel[0] = st->rel;
    host_rel[1] = st->bnorm;
  }
}

void arnoldi_start(ArnoldiState* st, int first, double* host_rel, cudaStream_t s) {
  k_arnoldi_start<<<1, 1, 0, s>>>(st, first, host_rel);
  SCR_LAUNCH();
  counters().launches++;
}

__global__ void k_backsolve(ArnoldiState* st, int k, const int* __restrict__ kp) {
  if (kp) k = *kp;
  constexpr int ldh = kMaxBasis + 1;
  for (int i = k - 1; i >= 0; --i) {
    double v = st->g[i];
    for (int l = i + 1; l < k; ++l) v -= st->H[(long long)l * ldh + i] * st->y[l];
    const double d = st->H[(long long)i * ldh + i];
    st->y[i] = d != 0.0 ? v / d : 0.0;
  }
}

template <int KMAX, typename T>
__global__ void k_update_x(const ArnoldiState* __restrict__ st, int k, const T* __restrict__ Z, long long ld,
                           T* __restrict__ x, long long n, const int* __restrict__ kp) {
  if (kp) k = *kp;
  T y[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) y[j] = j < k ? (T)st->y[j] : (T)0;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x, stp = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += stp) {
    T v = x[i];
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < k) v = fma(y[j], Z[j * ld + i], v);
    x[i] = v;
  }
}
template <int KMAX, typename T>
static void launch_update_x(const ArnoldiState* st, int k, const T* Z, long long ld, T* x, long long n,
                            cudaStream_t s, const int* kp) {
  k_update_x<KMAX, T><<<grid_for(n), 256, 0, s>>>(st, k, Z, ld, x, n, kp);
}

template <typename T>
void gmres_update(ArnoldiState* st, int k, const T* Z, long long ld, T* x, long long n, cudaStream_t s,
                  const int* kp) {
  if (k <= 0) return;
  k_backsolve<<<1, 1, 0, s>>>(st, k, kp);
  SCR_LAUNCH();
  SCR_KDISPATCH(launch_update_x, T, k, st, k, Z, ld, x, n, s, kp);
  SCR_LAUNCH();
  counters().launches += 2;
}
template void gmres_update<double>(ArnoldiState*, int, const double*, long long, double*, long long, cudaStream_t,
                                   const int*);
template void gmres_update<float>(ArnoldiState*, int, const float*, long long, float*, long long, cudaStream_t,
                                  const int*);

// ------------------------------------------------------------ CG
__global__ void k_cg_scalar(CgState* st, int mode, double* host_rel) {
  switch (mode) {
    case 0:  // start: bnorm2 in rr
      st->bnorm2 = st->rr;
      st->rel = st->rr > 0 ? 1.0 : 0.0;
      if (host_rel) host_rel[0] = st->rel, host_rel[1] = st->bnorm2;
      break;
    case 1:  // alpha = rz / pq
      st->alpha = st->pq != 0.0 ? st->rz / st->pq : 0.0;
      break;
    case 2:  // residual estimate
      st->rel = st->bnorm2 > 0 ? sqrt(st->rr / st->bnorm2) : 0.0;
      if (host_rel) host_rel[0] = st->rel;
      break;
    case 3:  // first rz
      st->rz = st->rz_new;
      break;
    case 4:  // beta = rz_new / rz
      st->beta = st->rz != 0.0 ? st->rz_new / st->rz : 0.0;
      st->rz = st->rz_new;
      break;
  }
}

__global__ void k_cg_xr(const CgState* __restrict__ st, const double* __restrict__ p, const double* __restrict__ q,
                        double* __restrict__ x, double* __restrict__ r, long long n, double* __restrict__ partial) {
  const double a = st->alpha;
  double acc[1] = {0.0};
  const long long stp = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stp) {
    x[i] = fma(a, p[i], x[i]);
    const double ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    acc[0] = fma(ri, ri, acc[0]);
  }
  block_store_partials<1>(acc, 1, partial);
}

__global__ void k_cg_p(const CgState* __restrict__ st, const double* __restrict__ z, double* __restrict__ p,
                       long long n) {
  const double b = st->beta;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x, stp = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += stp) p[i] = fma(b, p[i], z[i]);
}

void cg_start(CgState* st, const double* b, long long n, const Reducer& red, double* host_rel, cudaStream_t s) {
  norm2(b, n, &st->rr, red, s);
  k_cg_scalar<<<1, 1, 0, s>>>(st, 0, host_rel);
  SCR_LAUNCH();
  counters().launches++;
}
void cg_dot_rz(CgState* st, const double* r, const double* z, long long n, const Reducer& red, int first,
               cudaStream_t s) {
  multidot(r, 0, 1, z, n, &st->rz_new, red, s);
  k_cg_scalar<<<1, 1, 0, s>>>(st, first ? 3 : 4, nullptr);
  SCR_LAUNCH();
  counters().launches++;
}
void cg_alpha(CgState* st, const double* p, const double* q, long long n, const Reducer& red, cudaStream_t s) {
  multidot(p, 0, 1, q, n, &st->pq, red, s);
  k_cg_scalar<<<1, 1, 0, s>>>(st, 1, nullptr);
  SCR_LAUNCH();
  counters().launches++;
}
void cg_step_x_r(CgState* st, const double* p, const double* q, double* x, double* r, long long n,
                 const Reducer& red, double* host_rel, cudaStream_t s) {
  k_cg_xr<<<red.nblk, kRedThreads, 0, s>>>(st, p, q, x, r, n, red.partial);
  SCR_LAUNCH();
  reduce(red, 1, &st->rr, s);
  k_cg_scalar<<<1, 1, 0, s>>>(st, 2, host_rel);
  SCR_LAUNCH();
  counters().launches += 2;
}
void cg_update_p(CgState* st, const double* z, double* p, long long n, cudaStream_t s) {
  k_cg_p<<<grid_for(n), 256, 0, s>>>(st, z, p, n);
  SCR_LAUNCH();
  counters().launches++;
}

}  // namespace scr
