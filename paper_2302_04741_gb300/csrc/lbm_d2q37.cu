// Kernel instantiations for the D2Q37 lattice (ninth-order rule, Sec. 3).
#include "lbm_launch.cuh"

namespace lbm {
const LatticeOps& ops_d2q37() {
  static const LatticeOps t = Ops<D2Q37>::table();
  return t;
}
}  // namespace lbm
