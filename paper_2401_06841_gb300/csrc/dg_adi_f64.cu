// dg_adi_f64.cu -- FP64 instantiation of the adiabatic-system launchers.
#include "dg_adi_impl.cuh"

namespace dg {
template cudaError_t launch_adi<double>(const Launch&, double, const AdiLaunch&);
template cudaError_t launch_adi_totals<double>(const Launch&, double, double, const void*, double*, int*);
template cudaError_t launch_adi_shift<double>(const Launch&, void*, double);
}  // namespace dg
