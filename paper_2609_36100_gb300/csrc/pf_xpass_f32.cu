// Instantiation of the x passes (templates in pf_xpass.cuh; one translation
// unit per compute type so that they compile in parallel).
#include "pf_xfused.cuh"

namespace pf {
template int launch_x_pass<float>(const Geo&, const Phys&, int, const void*, void*, void*, const void*, double*,
                                 double, double, const double*, double*, cudaStream_t);
}  // namespace pf
