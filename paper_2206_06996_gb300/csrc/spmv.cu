// Block-sparse matrix-vector products (slab layout), layout conversions and
// the fused 2x2 block operator calA = [[A, B], [C, D]] of Sec. 5.2.1.
//
// Work decomposition: one group of G lanes per SCALAR row.  A scalar row of
// a block row is contiguous in the slab layout (k*BC values), so the G lanes
// stream it with one multiply-add per stored value and combine their partial
// sums with log2(G) shuffles.  G is small (2-8): on GB300 the FP64 pipe
// (about two FP64 FMAs per SM clock) is the binding resource of an FP64
// SpMV, and a wider group would spend more FP64 adds on the cross-lane
// reduction than on the product itself.
#include <cuda_bf16.h>

#include <cstdarg>
#include <cstring>
#include <map>
#include <mutex>
#include <stdexcept>
#include <tuple>
#include <vector>
#include <type_traits>

#include "spmv_kernels.cuh"


namespace scr {

LaunchCounter& counters() {
  static LaunchCounter c;
  return c;
}

KernelProfiler& profiler() {
  static KernelProfiler p;
  return p;
}

int prof_start(int kclass, const void* key, cudaStream_t s) {
  KernelProfiler& p = profiler();
  if (!p.active || p.kclass != kclass || (key && key != p.target)) return -1;
  p.launches++;
  if (p.used >= p.cap) return -1;
  const int i = p.used++;
  SCR_CUDA(cudaEventRecord(p.ev[2 * i], s));
  return i;
}

void prof_stop(int idx, double bytes, double flops, cudaStream_t s) {
  if (idx < 0) return;
  KernelProfiler& p = profiler();
  SCR_CUDA(cudaEventRecord(p.ev[2 * idx + 1], s));
  p.bytes += bytes;
  p.flops += flops;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// ------------------------------------------------------------ layouts
template <typename TO>
__global__ void k_to_slab(const int* __restrict__ rp, const double* __restrict__ in, TO* __restrict__ out,
                          int nbr, int br, int bc) {
  int i = blockIdx.x * blockDim.y + threadIdx.y;
  if (i >= nbr) return;
  int s = rp[i], k = rp[i + 1] - s;
  int bs = br * bc;
  for (int q = threadIdx.x; q < k * bs; q += blockDim.x) {
    int t = q / bs, rem = q - t * bs, r = rem / bc, c = rem - r * bc;
    out[slab_index(s, k, t, r, c, br, bc)] = (TO)in[(long long)(s + t) * bs + rem];
  }
}

template <typename TI>
__global__ void k_from_slab(const int* __restrict__ rp, const TI* __restrict__ in, double* __restrict__ out,
                            int nbr, int br, int bc) {
  int i = blockIdx.x * blockDim.y + threadIdx.y;
  if (i >= nbr) return;
  int s = rp[i], k = rp[i + 1] - s;
  int bs = br * bc;
  for (int q = threadIdx.x; q < k * bs; q += blockDim.x) {
    int t = q / bs, rem = q - t * bs, r = rem / bc, c = rem - r * bc;
    out[(long long)(s + t) * bs + rem] = (double)in[slab_index(s, k, t, r, c, br, bc)];
  }
}

template <typename TO>
void to_slab(const int* rp, const double* std_val, TO* slab_val, int nbr, int br, int bc, long long nnzb,
             cudaStream_t s) {
  if (nbr == 0) return;
  dim3 blk(32, 8);
  k_to_slab<TO><<<ceil_div(nbr, 8), blk, 0, s>>>(rp, std_val, slab_val, nbr, br, bc);
  SCR_LAUNCH();
  counters().launches++;
  (void)nnzb;
}
template void to_slab<double>(const int*, const double*, double*, int, int, int, long long, cudaStream_t);
template void to_slab<float>(const int*, const double*, float*, int, int, int, long long, cudaStream_t);

void from_slab(const int* rp, const double* slab_val, double* std_val, int nbr, int br, int bc, long long,
               cudaStream_t s) {
  if (nbr == 0) return;
  dim3 blk(32, 8);
  k_from_slab<double><<<ceil_div(nbr, 8), blk, 0, s>>>(rp, slab_val, std_val, nbr, br, bc);
  SCR_LAUNCH();
}
void from_slab_f(const int* rp, const float* slab_val, double* std_val, int nbr, int br, int bc, long long,
                 cudaStream_t s) {
  if (nbr == 0) return;
  dim3 blk(32, 8);
  k_from_slab<float><<<ceil_div(nbr, 8), blk, 0, s>>>(rp, slab_val, std_val, nbr, br, bc);
  SCR_LAUNCH();
}

__global__ void k_d2f(const double* __restrict__ x, float* __restrict__ y, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long st = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += st) y[i] = (float)x[i];
}
// FP32 -> BF16, round to nearest even (__float2bfloat16_rn)
__global__ void k_f2bf(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long st = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += st) y[i] = __float2bfloat16_rn(x[i]);
}
void slab_to_bf16(const float* in, void* out, long long n, cudaStream_t s) {
  if (n == 0) return;
  k_f2bf<<<std::min<long long>(ceil_div(n, 256), 4 * 1024), 256, 0, s>>>(in, static_cast<__nv_bfloat16*>(out), n);
  SCR_LAUNCH();
  counters().launches++;
}

void slab_to_float(const double* in, float* out, long long n, cudaStream_t s) {
  if (n == 0) return;
  k_d2f<<<std::min<long long>(ceil_div(n, 256), 4 * 1024), 256, 0, s>>>(in, out, n);
  SCR_LAUNCH();
  counters().launches++;
}

// ------------------------------------------------------------ padded copy
// sizes of the padded copy per block row: column slots (k rounded up to a
// multiple of V) and values (br scalar rows of bc k values each, rounded up
// to a multiple of V)
__global__ void k_vec_sizes(int nbr, const int* __restrict__ rp, int br, int bc, int V, int* __restrict__ csz,
                            int* __restrict__ vsz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbr) return;
  const int k = rp[i + 1] - rp[i];
  csz[i] = (k + V - 1) / V * V;
  vsz[i] = br * ((bc * k + V - 1) / V * V);
}

// one warp per block row: column slots (padding repeats the row's last
// column, or 0 in an empty row) and the padded scalar rows (zeros past bc k)
template <typename T>
__global__ void k_vec_fill(int nbr, const int* __restrict__ rp, const int* __restrict__ col,
                           const T* __restrict__ slab, int br, int bc, int V, const int* __restrict__ cs,
                           const int* __restrict__ vs, void* __restrict__ desc, int* __restrict__ vcol,
                           T* __restrict__ vval) {
  const int i = blockIdx.x * blockDim.y + threadIdx.y;
  if (i >= nbr) return;
  const int s = rp[i], k = rp[i + 1] - s;
  const int c0 = cs[i], cn = cs[i + 1] - c0;
  const int v0 = vs[i], rl = (vs[i + 1] - v0) / br;
  if (threadIdx.x == 0) {
    if (br == 3) static_cast<int4*>(desc)[i] = make_int4(c0, k, v0, rl);
    else static_cast<int2*>(desc)[i] = make_int2(c0, k);
  }
  const int last = k > 0 ? col[s + k - 1] : 0;
  for (int t = threadIdx.x; t < cn; t += blockDim.x) vcol[c0 + t] = t < k ? col[s + t] : last;
  const long long src = (long long)s * br * bc;
  for (int q = threadIdx.x; q < br * rl; q += blockDim.x) {
    const int r = q / rl, e = q - r * rl;
    vval[v0 + q] = e < bc * k ? slab[src + (long long)r * k * bc + e] : (T)0;
  }
}

template <typename VT>
void build_vec(DBsr<VT>& M, DeviceArena& a, cudaStream_t s) {
  const bool sq3 = M.br == 3 && M.bc == 3, sq1 = M.br == 1 && M.bc == 1;
  if (M.nbr == 0 || !(sq3 || sq1)) return;
  constexpr int V = 16 / (int)sizeof(VT);
  DeviceArena tmp(s);
  int* csz = tmp.alloc<int>(M.nbr + 1);
  int* vsz = tmp.alloc<int>(M.nbr + 1);
  int* cs = a.alloc<int>(M.nbr + 1);
  int* vs = tmp.alloc<int>(M.nbr + 1);
  k_vec_sizes<<<ceil_div(M.nbr, 256), 256, 0, s>>>(M.nbr, M.rp, M.br, M.bc, V, csz, vsz);
  SCR_LAUNCH();
  long long nc = 0, nv = 0;
  try {
    nc = exclusive_scan(csz, cs, M.nbr, tmp, s);
    nv = exclusive_scan(vsz, vs, M.nbr, tmp, s);
  } catch (const CudaError&) {
    return;  // padded arrays beyond int32 indexing: keep the slab kernels
  }
  void* desc = sq3 ? static_cast<void*>(a.alloc<int4>(M.nbr)) : static_cast<void*>(a.alloc<int2>(M.nbr));
  // 16 entries of slack: a lane's last vector never leaves the allocation
  int* vcol = a.alloc<int>(nc + 16);
  VT* vval = sq1 ? nullptr : a.alloc<VT>(nv + 16);
  if (sq1) {
    // 1x1: values share the column slots' starts (both padded to V entries)
    vval = a.alloc<VT>(nc + 16);
  }
  dim3 blk(32, 8);
  k_vec_fill<VT><<<ceil_div(M.nbr, 8), blk, 0, s>>>(M.nbr, M.rp, M.col, M.val, M.br, M.bc, V, cs, sq1 ? cs : vs,
                                                    desc, vcol, vval);
  SCR_LAUNCH();
  counters().launches += 2;
  M.vdesc = desc;
  M.vcol = vcol;
  M.vval = vval;
  (void)nv;
}
// the padded values of block row i from its descriptor (the column slots
// are unchanged)
template <typename T>
__global__ void k_vec_refill(int nbr, const int* __restrict__ rp, const T* __restrict__ slab, int br, int bc, int V,
                             const void* __restrict__ desc, T* __restrict__ vval) {
  const int i = blockIdx.x * blockDim.y + threadIdx.y;
  if (i >= nbr) return;
  const int s = rp[i], k = rp[i + 1] - s;
  int v0, rl;
  if (br == 3) {
    const int4 d = static_cast<const int4*>(desc)[i];
    v0 = d.z;
    rl = d.w;
  } else {
    const int2 d = static_cast<const int2*>(desc)[i];
    v0 = d.x;
    rl = (k + V - 1) / V * V;
  }
  const long long src = (long long)s * br * bc;
  for (int q = threadIdx.x; q < br * rl; q += blockDim.x) {
    const int r = q / rl, e = q - r * rl;
    vval[v0 + q] = e < bc * k ? slab[src + (long long)r * k * bc + e] : (T)0;
  }
}

template <typename VT>
void refresh_vec(DBsr<VT>& M, cudaStream_t s) {
  if (!M.vdesc || M.nbr == 0) return;
  constexpr int V = 16 / (int)sizeof(VT);
  dim3 blk(32, 8);
  k_vec_refill<VT><<<ceil_div(M.nbr, 8), blk, 0, s>>>(M.nbr, M.rp, M.val, M.br, M.bc, V, M.vdesc,
                                                      const_cast<VT*>(M.vval));
  SCR_LAUNCH();
  counters().launches++;
}
template void refresh_vec<double>(DBsr<double>&, cudaStream_t);
template void refresh_vec<float>(DBsr<float>&, cudaStream_t);

template void build_vec<double>(DBsr<double>&, DeviceArena&, cudaStream_t);
template void build_vec<float>(DBsr<float>&, DeviceArena&, cudaStream_t);

// ------------------------------------------------------------ SpMV
// CTAs ahead for the L2 prefetch of the scalar-row kernel (0: off); set
// from the options at scr_create.  Measured on the 616k-node tube: 128 to
// 384 CTAs ahead gave the same level-0 product times (FP32 122 -> 110 us,
// FP64 241 -> 229 us); 1536 and more were slower than none.
int g_l2_prefetch = 192;
void set_l2_prefetch(int ctas) { g_l2_prefetch = ctas; }
// programmatic dependent launch of the product kernels (options.pdl)
int g_pdl = 1;
void set_pdl(int on) { g_pdl = on; }
// print every autotune decision with the candidates' times (options.verbose)
static int g_tune_verbose = 0;
void set_tune_verbose(int v) { g_tune_verbose = v; }
// forced kernel code for every product (options.spmv_group)
int g_forced = 0;
void set_forced_group(int code) { g_forced = code; }
int forced_group() { return g_forced; }

template <typename VT, typename XT>
static void spmv_launch(int G, const DBsr<VT>& M, const XT* x, XT* y, int nrhs, const EpiArgs& e, cudaStream_t s) {
  const int br = M.br, bc = M.bc;
  if (br == 3 && bc == 3 && nrhs == 1) dispatch_g<3, 3, 1, VT, XT>(G, M, x, y, e, s);
  else if (br == 3 && bc == 1 && nrhs == 1) dispatch_g<3, 1, 1, VT, XT>(G, M, x, y, e, s);
  else if (br == 1 && bc == 3 && nrhs == 1) dispatch_g<1, 3, 1, VT, XT>(G, M, x, y, e, s);
  else if (br == 1 && bc == 1 && nrhs == 1) dispatch_g<1, 1, 1, VT, XT>(G, M, x, y, e, s);
  else if (br == 1 && bc == 1 && nrhs == 3) dispatch_g<1, 1, 3, VT, XT>(G, M, x, y, e, s);
  else if (nrhs == kSpmmCols) spmm_launch<VT, XT>(G, M, x, y, e, s);
  else throw CudaError{cudaErrorInvalidValue, "spmv: unsupported block shape or number of right-hand sides"};
}

// the product with the values M holds: its BF16 copy when it has one (FP32
// vectors, FP32 sums), else val
template <typename VT, typename XT>
static void product(int G, const DBsr<VT>& M, const XT* x, XT* y, int nrhs, const EpiArgs& e, cudaStream_t s) {
  if constexpr (std::is_same<VT, float>::value) {
    if (M.hval) {
      DBsr<__nv_bfloat16> H;
      H.nbr = M.nbr;
      H.nbc = M.nbc;
      H.br = M.br;
      H.bc = M.bc;
      H.nnzb = M.nnzb;
      H.rp = M.rp;
      H.col = M.col;
      H.val = static_cast<__nv_bfloat16*>(const_cast<void*>(M.hval));
      H.g = M.g;
      spmv_launch<__nv_bfloat16, XT>(G, H, x, y, nrhs, e, s);
      return;
    }
  }
  spmv_launch<VT, XT>(G, M, x, y, nrhs, e, s);
}

template <typename VT, typename XT>
void spmv(const DBsr<VT>& M, const XT* x, XT* y, int nrhs, const EpiArgs& e, cudaStream_t s) {
  if (M.nbr == 0) return;
  const int G = M.sell ? 1 : pick_group(M);
  const int pidx = prof_start(0, M.val, s);
  product<VT, XT>(G, M, x, y, nrhs, e, s);
  counters().launches++;
  {
    // algorithmic bytes: stored values + column indices + row pointers once,
    // the source vector once, the result written once, plus what the
    // epilogue reads (z, the current iterate, the inverse diagonal)
    const double nrow = (double)M.nbr * M.br;
    const double vsz = M.hval ? 2.0 : (double)sizeof(VT);
    double b = (double)M.nnzb * (M.br * M.bc * vsz + sizeof(int)) + (M.nbr + 1.0) * sizeof(int) +
               (double)M.nbc * M.bc * nrhs * sizeof(XT) + nrow * nrhs * sizeof(XT);
    if (e.kind == Epi::Resid || (e.kind == Epi::Axpby && e.z)) b += nrow * nrhs * sizeof(XT);
    if (e.kind == Epi::Jacobi) b += 2.0 * nrow * nrhs * sizeof(XT) + nrow * sizeof(XT);
    if (e.kind == Epi::ScaledSub) b += nrow * nrhs * sizeof(XT) + nrow * sizeof(XT);
    if (e.kind == Epi::ChebFirst) b += 4.0 * nrow * nrhs * sizeof(XT) + nrow * sizeof(XT);
    if (e.kind == Epi::ChebStep) b += 5.0 * nrow * nrhs * sizeof(XT) + nrow * sizeof(XT);
    counters().spmv_bytes += (long long)b;
    prof_stop(pidx, b, 2.0 * (double)M.nnzb * M.br * M.bc * nrhs, s);
  }
}

// Decisions are cached by (shape, size, precision, right-hand sides): a
// Newton step's new Jacobian has the pattern of the previous one, so the
// timing runs once per pattern.
struct TuneKey {
  long long nnzb;
  int nbr, nbc, br, bc, vt, nrhs, dev;
  bool operator<(const TuneKey& o) const {
    return std::tie(nnzb, nbr, nbc, br, bc, vt, nrhs, dev) <
           std::tie(o.nnzb, o.nbr, o.nbc, o.br, o.bc, o.vt, o.nrhs, o.dev);
  }
};
static std::map<TuneKey, int>& tune_cache() {
  static std::map<TuneKey, int> m;
  return m;
}
static std::mutex g_tune_mutex;

template <typename VT>
int autotune_spmv(DBsr<VT>& M, int nrhs, cudaStream_t s) {
  if (M.nbr == 0 || M.sell) return M.g;
  int dev = 0;
  cudaGetDevice(&dev);
  // value bytes, plus 100 when M has the padded 16-byte copy (its candidates differ)
  const TuneKey key{M.nnzb, M.nbr, M.nbc, M.br, M.bc, (int)sizeof(VT) + (M.vdesc ? 100 : 0), nrhs, dev};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = tune_cache().find(key);
    if (it != tune_cache().end()) {
      M.g = it->second;
      return M.g;
    }
  }
  using XT = VT;
  const long long nx = (long long)M.nbc * M.bc * nrhs + 1, ny = (long long)M.nbr * M.br * nrhs + 1;
  XT *x = nullptr, *y = nullptr;
  SCR_CUDA(cudaMallocAsync(&x, nx * sizeof(XT), s));
  SCR_CUDA(cudaMallocAsync(&y, ny * sizeof(XT), s));
  SCR_CUDA(cudaMemsetAsync(x, 0, nx * sizeof(XT), s));
  // square operators are timed with the epilogue they mostly run in a solve
  // (the Chebyshev step of the V-cycle: three more vectors read, three
  // written), the others with the plain product
  EpiArgs ep;
  XT* ev = nullptr;
  if (M.br == M.bc && M.nbr == M.nbc) {
    SCR_CUDA(cudaMallocAsync(&ev, 3 * ny * sizeof(XT), s));
    SCR_CUDA(cudaMemsetAsync(ev, 0, 3 * ny * sizeof(XT), s));
    ep.kind = Epi::ChebStep;
    ep.alpha = 0.5;
    ep.beta = 0.5;
    ep.dinv = ev;
    ep.r = ev + ny;
    ep.xsol = ev + 2 * ny;
    ep.dout = y;
  }
  cudaEvent_t e0, e1;
  SCR_CUDA(cudaEventCreate(&e0));
  SCR_CUDA(cudaEventCreate(&e1));
  // the scalar-row kernel with 1, 2, 4 or 8 lanes (the block-row and
  // sliced-ELL variants measured slower on the tube operators)
  int cands[12] = {101, 102, 104, 108};
  int ncand = 4;
  if (M.nbr && (double)M.nnzb * M.bc / M.nbr >= 64) cands[ncand++] = 116;  // long rows
  // the 16-byte kernels on the padded copy (one right-hand side)
  if (M.vdesc && nrhs == 1) {
    cands[ncand++] = 302;
    cands[ncand++] = 304;
    cands[ncand++] = 308;
    if (M.br == 1) cands[ncand++] = 316;
  }
  float best = 1e30f;
  int bestg = M.g;
  const int saved = M.g;
  float times[12] = {};
  for (int q = 0; q < ncand; ++q) {
    const int code = cands[q];
    M.g = code;
    const int G = pick_group(M);
    auto run = [&] { product<VT, XT>(G, M, x, y, nrhs, ep, s); };
    run();  // warm-up
    SCR_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < 5; ++r) run();
    SCR_CUDA(cudaEventRecord(e1, s));
    SCR_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    SCR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    times[q] = ms;
    if (ms < best) {
      best = ms;
      bestg = code;
    }
  }
  (void)saved;
  counters().launches += 6 * ncand;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  SCR_CUDA(cudaFreeAsync(x, s));
  SCR_CUDA(cudaFreeAsync(y, s));
  if (ev) SCR_CUDA(cudaFreeAsync(ev, s));
  M.g = bestg;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_cache()[key] = bestg;
  }
  if (g_tune_verbose) {
    fprintf(stderr, "[autotune] %dx%d blocks, %d x %d block rows/cols, %lld blocks, %s, nrhs %d -> code %d |",
            M.br, M.bc, M.nbr, M.nbc, M.nnzb, sizeof(VT) == 8 ? "fp64" : "fp32", nrhs, bestg);
    for (int q = 0; q < ncand; ++q) fprintf(stderr, " %d: %.1f us", cands[q], 200.0f * times[q]);
    fprintf(stderr, "\n");
  }
  return bestg;
}
// text form of the cache: "nnzb nbr nbc br bc value_bytes nrhs code" per line
// (value_bytes + 100 for matrices with the padded 16-byte copy)
static bool valid_code(int c) {
  return (c >= 1 && c <= 16) || (c >= 101 && c <= 116) || (c >= 301 && c <= 316);
}

void tune_save(const char* path) {
  FILE* f = fopen(path, "w");
  if (!f) throw std::invalid_argument("scr_tune_save: cannot open the file for writing");
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  fprintf(f, "# scr_gb300 autotune decisions: nnzb nbr nbc br bc value_bytes nrhs code\n");
  for (const auto& kv : tune_cache()) {
    const TuneKey& k = kv.first;
    fprintf(f, "%lld %d %d %d %d %d %d %d\n", k.nnzb, k.nbr, k.nbc, k.br, k.bc, k.vt, k.nrhs, kv.second);
  }
  fclose(f);
}

void tune_load(const char* path) {
  FILE* f = fopen(path, "r");
  if (!f) throw std::invalid_argument("scr_tune_load: cannot open the file");
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<std::pair<TuneKey, int>> got;
  char line[512];
  bool bad = false;
  while (fgets(line, sizeof line, f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    TuneKey k{};
    int code = 0;
    if (sscanf(line, "%lld %d %d %d %d %d %d %d", &k.nnzb, &k.nbr, &k.nbc, &k.br, &k.bc, &k.vt, &k.nrhs, &code) != 8 ||
        !valid_code(code) || k.nnzb < 0 || k.nbr < 0 || k.nbc < 0) {
      bad = true;
      break;
    }
    k.dev = dev;
    got.emplace_back(k, code);
  }
  fclose(f);
  if (bad) throw std::invalid_argument("scr_tune_load: malformed line");
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  for (const auto& kv : got) tune_cache()[kv.first] = kv.second;
}

template int autotune_spmv<double>(DBsr<double>&, int, cudaStream_t);
template int autotune_spmv<float>(DBsr<float>&, int, cudaStream_t);

template void spmv<double, double>(const DBsr<double>&, const double*, double*, int, const EpiArgs&, cudaStream_t);
template void spmv<float, float>(const DBsr<float>&, const float*, float*, int, const EpiArgs&, cudaStream_t);

// ------------------------------------------------------------ calA
// Scalar rows 0..3n_v-1: (A x_v + B x_p); rows 3n_v..3n_v+n_p-1:
// (C x_v + D x_p).  One G-group per scalar row; NRHS interleaved
// right-hand sides (x_p starts at 3 n_v NRHS).
template <int G, int NRHS, bool RESID>
__global__ void __launch_bounds__(256) k_block_op(int nv, int np, DBsr<double> A, DBsr<double> B, DBsr<double> C,
                                                  DBsr<double> D, const double* __restrict__ x,
                                                  double* __restrict__ y, const double* __restrict__ z) {
  const long long o = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / G;
  const int lane = threadIdx.x % G;
  const long long nrow_v = 3LL * nv;
  const bool active = o < nrow_v + np;  // inactive lanes still join the shuffles
  const double* xv = x;
  const double* xp = x + nrow_v * NRHS;
  double acc[NRHS];
#pragma unroll
  for (int h = 0; h < NRHS; ++h) acc[h] = 0.0;
  if (!active) {
  } else if (o < nrow_v) {
    const int i = (int)(o / 3), r = (int)(o - 3LL * i);
    scalar_row_accum<3, NRHS, G>(A.rp, A.col, A.val, xv, 3, i, r, lane, acc);
    scalar_row_accum<1, NRHS, G>(B.rp, B.col, B.val, xp, 3, i, r, lane, acc);
  } else {
    const int i = (int)(o - nrow_v);
    scalar_row_accum<3, NRHS, G>(C.rp, C.col, C.val, xv, 1, i, 0, lane, acc);
    scalar_row_accum<1, NRHS, G>(D.rp, D.col, D.val, xp, 1, i, 0, lane, acc);
  }
#pragma unroll
  for (int h = 0; h < NRHS; ++h)
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) acc[h] += __shfl_xor_sync(0xffffffffu, acc[h], off, G);
  if (active && lane == 0) {
#pragma unroll
    for (int h = 0; h < NRHS; ++h) y[o * NRHS + h] = RESID ? z[o * NRHS + h] - acc[h] : acc[h];
  }
}

// y_p = D x_p - C x_t, the last line of Algorithm 2 (App. B) in one pass:
// one G-group per pressure row accumulates the row of C against x_t and the
// row of D against x_p, so y_p is written once and never read back.
template <int G, int NRHS, typename T>
__global__ void __launch_bounds__(256) k_schur_combine(int np, DBsr<T> C, DBsr<T> D, const T* __restrict__ xt,
                                                       const T* __restrict__ xp, T* __restrict__ yp) {
  const long long o = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / G;
  const int lane = threadIdx.x % G;
  const bool active = o < np;  // inactive lanes still join the shuffles
  T ac[NRHS], ad[NRHS];
#pragma unroll
  for (int h = 0; h < NRHS; ++h) ac[h] = ad[h] = (T)0;
  if (active) {
    scalar_row_accum<3, NRHS, G>(C.rp, C.col, C.val, xt, 1, (int)o, 0, lane, ac);
    scalar_row_accum<1, NRHS, G>(D.rp, D.col, D.val, xp, 1, (int)o, 0, lane, ad);
  }
#pragma unroll
  for (int h = 0; h < NRHS; ++h)
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
      ac[h] += __shfl_xor_sync(0xffffffffu, ac[h], off, G);
      ad[h] += __shfl_xor_sync(0xffffffffu, ad[h], off, G);
    }
  if (active && lane == 0) {
#pragma unroll
    for (int h = 0; h < NRHS; ++h) yp[o * NRHS + h] = ad[h] - ac[h];
  }
}

template <typename T>
void schur_combine(const DBsr<T>& C, const DBsr<T>& D, const T* xt, const T* xp, T* yp, int nrhs,
                   cudaStream_t s) {
  const int np = D.nbr;
  if (np == 0) return;
  constexpr int G = 4;
  const long long threads = (long long)np * G;
  if (nrhs == 1)
    k_schur_combine<G, 1, T><<<ceil_div(threads, 256), 256, 0, s>>>(np, C, D, xt, xp, yp);
  else if (nrhs == kSpmmCols)
    k_schur_combine<G, kSpmmCols, T><<<ceil_div(threads, 256), 256, 0, s>>>(np, C, D, xt, xp, yp);
  else
    throw CudaError{cudaErrorInvalidValue, "schur_combine: unsupported number of right-hand sides"};
  SCR_LAUNCH();
  counters().launches++;
  counters().spmv_bytes += (long long)((double)C.nnzb * (3 * sizeof(T) + 4) + (double)D.nnzb * (sizeof(T) + 4) +
                                       (2.0 * np + 2) * 4 + (double)C.nbc * 3 * nrhs * sizeof(T) +
                                       2.0 * np * nrhs * sizeof(T));
}
template void schur_combine<double>(const DBsr<double>&, const DBsr<double>&, const double*, const double*, double*,
                                    int, cudaStream_t);
template void schur_combine<float>(const DBsr<float>&, const DBsr<float>&, const float*, const float*, float*, int,
                                   cudaStream_t);

template <int NRHS>
static void launch_block_op(int nv, int np, const DBsr<double>& A, const DBsr<double>& B, const DBsr<double>& C,
                            const DBsr<double>& D, const double* x, double* y, const double* z, bool resid,
                            cudaStream_t s) {
  constexpr int G = 4;
  const long long threads = (3LL * nv + np) * G;
  if (resid)
    k_block_op<G, NRHS, true><<<ceil_div(threads, 256), 256, 0, s>>>(nv, np, A, B, C, D, x, y, z);
  else
    k_block_op<G, NRHS, false><<<ceil_div(threads, 256), 256, 0, s>>>(nv, np, A, B, C, D, x, y, z);
  SCR_LAUNCH();
}

void block_op(const DBsr<double>& A, const DBsr<double>& B, const DBsr<double>& C, const DBsr<double>& D,
              const double* x, double* y, const double* z, bool resid, cudaStream_t s, int nrhs) {
  const int nv = A.nbr, np = D.nbr;
  const long long rows = 3LL * nv + np;
  if (rows == 0) return;
  const int pidx = prof_start(1, nullptr, s);
  if (nrhs == 1) launch_block_op<1>(nv, np, A, B, C, D, x, y, z, resid, s);
  else if (nrhs == kSpmmCols) launch_block_op<kSpmmCols>(nv, np, A, B, C, D, x, y, z, resid, s);
  else throw CudaError{cudaErrorInvalidValue, "block_op: unsupported number of right-hand sides"};
  counters().launches++;
  const double b = A.nnzb * 76.0 + B.nnzb * 28.0 + C.nnzb * 28.0 + D.nnzb * 12.0 +
                   (A.nbr + D.nbr + 2.0) * 8.0 + rows * 8.0 * nrhs * (resid ? 3 : 2);
  counters().spmv_bytes += (long long)b;
  prof_stop(pidx, b, 2.0 * nrhs * (9.0 * A.nnzb + 3.0 * B.nnzb + 3.0 * C.nnzb + D.nnzb), s);
}

}  // namespace scr
