// One FFT grid size of the NLINV kernels: the build compiles this file once
// per size G = NLINV_G1 x NLINV_G2 (-D flags), each into its own object.
#include "grid.cuh"

#if !defined(NLINV_G1) || !defined(NLINV_G2)
#error "NLINV_G1 and NLINV_G2 select the grid size of this unit"
#endif

#define NLINV_OPS_NAME2(a, b) grid_ops_##a##_##b
#define NLINV_OPS_NAME(a, b) NLINV_OPS_NAME2(a, b)

namespace nlinv {
const GridOps* NLINV_OPS_NAME(NLINV_G1, NLINV_G2)() { return make_ops<Cfg<NLINV_G1, NLINV_G2>>(); }
}  // namespace nlinv
