// Instantiation of the compiled-plan elastic pass without a fused stage
// (templates in pf_yz.cuh; a translation unit of its own so that it compiles
// in parallel with the fused form).
#define PF_ELASTIC_ALT_TU
#include "pf_yz.cuh"

namespace pf {
template bool launch_z_elastic_unfused<double>(const Geo&, const Phys&, void*, int, cudaStream_t);
template bool launch_z_elastic_unfused<float>(const Geo&, const Phys&, void*, int, cudaStream_t);
}  // namespace pf
