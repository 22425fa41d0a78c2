// Instantiation of the fused FGP pass launcher with the duality-gap evaluation
// for TV type 2 (see pass_tv.cuh), in a unit of its own so that it compiles in
// parallel with the plain passes.
#include "pass_tv.cuh"

namespace ctv {
template cudaError_t launch_pass_gap_tv<2>(int cfg, int cons, const PassParams& p, dim3 grid, cudaStream_t s);
}  // namespace ctv
