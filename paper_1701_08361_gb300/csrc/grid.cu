// One grid of the NLINV kernels: the build compiles this file once per grid
// G = NLINV_G1 x NLINV_G2 with an NLINV_NR x NLINV_NR field of view, tile
// width NLINV_TWU and NLINV_MINBU CTAs per SM (-D flags), each into its own
// object.
#include "grid.cuh"

#if !defined(NLINV_G1) || !defined(NLINV_G2) || !defined(NLINV_NR) || !defined(NLINV_TWU) || !defined(NLINV_MINBU)
#error "NLINV_G1, NLINV_G2, NLINV_NR, NLINV_TWU and NLINV_MINBU select the grid of this unit"
#endif

#define NLINV_OPS_NAME2(a, b, n) grid_ops_##a##_##b##_##n
#define NLINV_OPS_NAME(a, b, n) NLINV_OPS_NAME2(a, b, n)

namespace nlinv {
const GridOps* NLINV_OPS_NAME(NLINV_G1, NLINV_G2, NLINV_NR)() {
  return make_ops<Cfg<NLINV_G1, NLINV_G2, NLINV_NR, NLINV_TWU, NLINV_MINBU>>();
}
}  // namespace nlinv
