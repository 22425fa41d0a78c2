// Instantiation of the fused FGP pass launcher for TV type 3 (see pass_tv.cuh).
#include "pass_tv.cuh"

namespace ctv {
template cudaError_t launch_pass_tv<3>(int cfg, int cons, const PassParams& p, dim3 grid, cudaStream_t s);
}  // namespace ctv
