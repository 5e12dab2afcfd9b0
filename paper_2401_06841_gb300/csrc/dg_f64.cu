// FP64 instantiation of the kernels (the degree-3 tile kernels compile in
// dg_f64_k3.cu).
#include "dg_launch_impl.cuh"
namespace dg {
DG_TILES_EXTERN(double, 3)
DG_INSTANTIATE(double)
}
