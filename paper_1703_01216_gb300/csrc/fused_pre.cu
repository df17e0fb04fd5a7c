// Instantiation of the fused inverse that transforms already solved spectra (the M > 1 path), tile
// variant 1 (xi accumulated in the output array, tall row batches).
#include "fused.cuh"

namespace fr3d {

namespace {
template <int N, int MODE>
int launch_pre(const FusedArgs& a, int nj, cudaStream_t st) {
  using G = FusedGeom<N, 1>;
  constexpr size_t sm = MODE == 1 ? G::smem_xi : G::smem_zeta;
  return launch_clustered<G::CL>(k_inv_fused<N, MODE, 1, true>, nj, G::NT, sm, st, a);
}
}  // namespace

int fused_launch_pre(int n, bool xi, const FusedArgs& a, int nj, cudaStream_t st) {
  switch (n) {
    FR3D_FUSED_CASES(launch_pre, (a, nj, st))
  }
  return FR3D_ERR_UNSUPPORTED_SIZE;
}

}  // namespace fr3d
