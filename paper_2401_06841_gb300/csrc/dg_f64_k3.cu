// FP64 degree-3 tile kernels (all modes).
#include "dg_launch_impl.cuh"
namespace dg {
DG_TILES_INSTANTIATE(double, 3)
}
