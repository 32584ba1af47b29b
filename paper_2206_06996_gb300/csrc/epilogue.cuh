// Fused epilogues of the block products: what a product kernel does with
// the row sum acc of M x for scalar output row o (flat index gi = o * nrhs
// + h for right-hand side h).  Shared by the product kernels.
#pragma once
#include "kernels.h"

namespace scr {

template <typename XT, Epi E>
struct Epilogue {
  XT* y;
  const XT* z;
  const XT* xs;
  const XT* dinv;
  const XT* xin;  // the product's source vector (ChebStep: the direction)
  XT* r;
  XT* dout;
  XT* xsol;
  XT alpha, beta;
  template <typename AT>
  __device__ __forceinline__ void operator()(long long gi, long long o, AT acc) const {
    if constexpr (E == Epi::Set) {
      y[gi] = (XT)acc;
    } else if constexpr (E == Epi::Axpby) {
      XT v = alpha * (XT)acc;
      if (z) v += beta * z[gi];
      y[gi] = v;
    } else if constexpr (E == Epi::Resid) {
      y[gi] = z[gi] - (XT)acc;
    } else if constexpr (E == Epi::Jacobi) {
      y[gi] = xs[gi] + (z[gi] - (XT)acc) * dinv[o];
    } else if constexpr (E == Epi::ScaledSub) {
      y[gi] = z[gi] - (XT)acc * dinv[o];
    } else if constexpr (E == Epi::ChebFirst) {
      const XT ri = (z[gi] - (XT)acc) * dinv[o];
      const XT di = alpha * ri;
      r[gi] = ri;
      dout[gi] = di;
      y[gi] = xs[gi] + di;
    } else {
      const XT ri = r[gi] - (XT)acc * dinv[o];
      const XT di = alpha * xin[gi] + beta * ri;
      r[gi] = ri;
      dout[gi] = di;
      xsol[gi] += di;
    }
  }
};

template <typename XT, Epi E>
Epilogue<XT, E> make_epilogue(const XT* x, XT* y, const EpiArgs& e) {
  Epilogue<XT, E> epi;
  epi.y = y;
  epi.z = static_cast<const XT*>(e.z);
  epi.xs = static_cast<const XT*>(e.xs);
  epi.dinv = static_cast<const XT*>(e.dinv);
  epi.xin = x;
  epi.r = static_cast<XT*>(e.r);
  epi.dout = static_cast<XT*>(e.dout);
  epi.xsol = static_cast<XT*>(e.xsol);
  epi.alpha = (XT)e.alpha;
  epi.beta = (XT)e.beta;
  return epi;
}

}  // namespace scr
