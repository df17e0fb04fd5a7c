// Instantiation of the fused inverse for tile variant 0 (fused.cuh); one file per variant so that
// the variants compile in parallel.
#include "fused.cuh"

namespace fr3d {
FR3D_FUSED_VARIANT(0)
}  // namespace fr3d
