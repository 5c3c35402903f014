// FP32 instantiation of the step kernels.  Built with fast math: approximate
// division, square root, exp2/log2 on the special-function units, FMA
// contraction and flush-to-zero (the FP32 mode's accuracy target is set
// against the FP64 oracle, not against IEEE FP32).
#include "swe_kernels.cuh"

namespace swe {
SWE_INSTANTIATE(float)
}
