// FP32 instantiation of the transform, solve and combination kernels.  Scalar complex adds here: with
// packed FP32x2 adds the row pass with the combination (k_row_c2r, xi output) needs more registers and
// runs 17 % slower at n = 512 (measured at the paper geometry: 0.154 against 0.131 ms).
#define FR3D_SCALAR_COMPLEX_ADDS
#include "ops_impl.cuh"
template struct fr3d::Ops<float>;
