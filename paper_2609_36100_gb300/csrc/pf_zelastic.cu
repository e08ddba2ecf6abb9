// Instantiation of the elastic Green's contraction between z transforms (templates in pf_yz.cuh;
// one translation unit each so that they compile in parallel).
#include "pf_yz.cuh"

namespace pf {
template void launch_z_elastic<double>(const Geo&, const Phys&, void*, cudaStream_t);
template void launch_z_elastic<float>(const Geo&, const Phys&, void*, cudaStream_t);
}  // namespace pf
