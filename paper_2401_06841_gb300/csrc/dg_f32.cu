// FP32 instantiation of the CUDA-core kernels.
#include "dg_launch_impl.cuh"
namespace dg {
DG_INSTANTIATE(float)
}
