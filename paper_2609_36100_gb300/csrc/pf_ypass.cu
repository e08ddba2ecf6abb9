// Instantiation of the y-axis column transform (templates in pf_yz.cuh;
// one translation unit each so that they compile in parallel).
#include "pf_yz.cuh"

namespace pf {
template void launch_y_pass<double>(const Geo&, void*, int, int, cudaStream_t);
template void launch_y_pass<float>(const Geo&, void*, int, int, cudaStream_t);
}  // namespace pf
