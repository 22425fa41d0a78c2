// Instantiation of the plan's work-list pass launcher for TV type 2 (see plan_list.cuh).
#include "plan_list.cuh"

namespace ctv {
template cudaError_t launch_plan_list_tv<2>(int cfg, int cons, const ListPassParams& p, int nblocks,
                                             cudaStream_t s, bool set_attr);
}  // namespace ctv
