// dg_adi_f32.cu -- FP32 instantiation of the adiabatic-system launchers.
#include "dg_adi_impl.cuh"

namespace dg {
template cudaError_t launch_adi<float>(const Launch&, double, const AdiLaunch&);
template cudaError_t launch_adi_totals<float>(const Launch&, double, double, const void*, double*, int*);
template cudaError_t launch_adi_shift<float>(const Launch&, void*, double);
}  // namespace dg
