// Instantiation of the fused inverse for tile variant 1 (fused.cuh); one file per variant so that
// the variants compile in parallel.
#include "fused.cuh"

namespace fr3d {
FR3D_FUSED_VARIANT(1)
}  // namespace fr3d
