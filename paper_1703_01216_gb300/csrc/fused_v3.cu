// Instantiation of the fused inverse for tile variant 3 (fused.cuh); one file per variant so that
// the variants compile in parallel.
#include "fused.cuh"

namespace fr3d {
FR3D_FUSED_VARIANT(3)
}  // namespace fr3d
