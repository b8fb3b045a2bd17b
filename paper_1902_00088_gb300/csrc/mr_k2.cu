// 2D instantiation of the kernel templates (Bs 17 and 33).
#include "mr_launch.cuh"
namespace mr {
MR_INSTANTIATE(2)
}
