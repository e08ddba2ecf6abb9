// Instantiation of the z step completion pass, FP64 form (templates in pf_zstage.cuh;
// one translation unit each so that they compile in parallel).
#include "pf_zstage.cuh"

namespace pf {
template void launch_z_final<double>(const Geo&, const Phys&, const double2*, const StageTerms&, const StageTerms&,
                                     int, double2*, void*, cudaStream_t);
}  // namespace pf
