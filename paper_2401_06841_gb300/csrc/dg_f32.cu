// FP32 instantiation of the kernels (the degree-3 tile kernels compile in
// dg_f32_k3.cu).
#include "dg_launch_impl.cuh"
namespace dg {
DG_TILES_EXTERN(float, 3)
DG_INSTANTIATE(float)
}
