// Instantiation of the z stage assembly pass, FP32-bulk form (templates in pf_zstage.cuh;
// one translation unit each so that they compile in parallel).
#include "pf_zstage.cuh"

namespace pf {
template void launch_z_stage<float>(const Geo&, const Phys&, const double2*, const StageTerms&, double2*, void*,
                                    cudaStream_t);
}  // namespace pf
