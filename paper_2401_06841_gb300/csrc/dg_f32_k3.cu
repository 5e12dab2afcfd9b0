// FP32 degree-3 tile kernels (all modes and back ends).
#include "dg_launch_impl.cuh"
namespace dg {
DG_TILES_INSTANTIATE(float, 3)
}
