// Block products with eight interleaved right-hand sides (the block product
// of the multi-right-hand-side solve): every operator of the solver acts on
// the interleaved vectors as M (x) I_8, so one pass over M's stored blocks
// serves all eight columns.  Instantiated here, apart from spmv.cu, so that
// the two translation units compile in parallel.
#include "spmv_kernels.cuh"

namespace scr {

template <typename VT, typename XT>
void spmm_launch(int G, const DBsr<VT>& M, const XT* x, XT* y, const EpiArgs& e, cudaStream_t s) {
  constexpr int K = kSpmmCols;
  const int br = M.br, bc = M.bc;
  if (br == 3 && bc == 3) dispatch_g<3, 3, K, VT, XT>(G, M, x, y, e, s);
  else if (br == 3 && bc == 1) dispatch_g<3, 1, K, VT, XT>(G, M, x, y, e, s);
  else if (br == 1 && bc == 3) dispatch_g<1, 3, K, VT, XT>(G, M, x, y, e, s);
  else if (br == 1 && bc == 1) dispatch_g<1, 1, K, VT, XT>(G, M, x, y, e, s);
  else throw CudaError{cudaErrorInvalidValue, "spmm: unsupported block shape"};
}
template void spmm_launch<double, double>(int, const DBsr<double>&, const double*, double*, const EpiArgs&,
                                          cudaStream_t);
template void spmm_launch<float, float>(int, const DBsr<float>&, const float*, float*, const EpiArgs&,
                                        cudaStream_t);
template void spmm_launch<__nv_bfloat16, float>(int, const DBsr<__nv_bfloat16>&, const float*, float*,
                                                const EpiArgs&, cudaStream_t);

}  // namespace scr
