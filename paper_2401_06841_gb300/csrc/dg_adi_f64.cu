// dg_adi_f64.cu -- FP64 instantiation of the adiabatic-system launchers.
#include "dg_adi_impl.cuh"

namespace dg {
template cudaError_t launch_adi<double>(const Launch&, double, const AdiLaunch&);
template cudaError_t launch_adi_totals<double>(const Launch&, double, const void*, double*, int*);
}  // namespace dg
