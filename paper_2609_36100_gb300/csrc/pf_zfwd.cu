// Instantiation of the forward z transform with the k-space scaling of f^E (templates in pf_yz.cuh;
// one translation unit each so that they compile in parallel).
#include "pf_yz.cuh"

namespace pf {
template void launch_z_fwd<double>(const Geo&, const Phys&, const void*, void*, int, cudaStream_t, int);
template void launch_z_fwd<float>(const Geo&, const Phys&, const void*, void*, int, cudaStream_t, int);
template void launch_z_pass<float>(const Geo&, void*, int, int, cudaStream_t);
}  // namespace pf
