// FP64 instantiation of the CUDA-core kernels (parity mode).
#include "dg_launch_impl.cuh"
namespace dg {
DG_INSTANTIATE(double)
}
