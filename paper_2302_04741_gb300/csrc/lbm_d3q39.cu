// Kernel instantiations for the D3Q39 lattice (seventh-order rule).
#include "lbm_launch.cuh"

namespace lbm {
const LatticeOps& ops_d3q39() {
  static const LatticeOps t = Ops<D3Q39>::table();
  return t;
}
}  // namespace lbm
