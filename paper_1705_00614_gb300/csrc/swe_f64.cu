// FP64 instantiation of the step kernels.  Built without FMA contraction and
// with IEEE division and square root, so each formula rounds like the FP64
// oracle's plain evaluation of it.
#include "swe_kernels.cuh"

namespace swe {
SWE_INSTANTIATE(double)

__global__ void k_set_tend(Ctl* ctl, double t_end) { ctl->t_end = t_end; }

cudaError_t launch_set_tend(Ctl* ctl, double t_end, cudaStream_t st) {
    k_set_tend<<<1, 1, 0, st>>>(ctl, t_end);
    return cudaGetLastError();
}
}  // namespace swe
