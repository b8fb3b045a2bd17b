// 3D instantiation of the kernel templates (Bs 17); the RK stages are
// instantiated in mr_k3s.cu.
#include "mr_launch.cuh"
namespace mr {
MR_EXTERN_STAGE(3, 17)
MR_INSTANTIATE(3)
}
