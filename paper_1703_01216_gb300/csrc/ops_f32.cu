// FP32 instantiation of the transform, solve and combination kernels.
#include "ops_impl.cuh"
template struct fr3d::Ops<float>;
