// 3D instantiation of the kernel templates (Bs 17).
#include "mr_launch.cuh"
namespace mr {
MR_INSTANTIATE(3)
}
