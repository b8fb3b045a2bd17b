// RK stage launchers, 3D, Bs 17.
#include "mr_launch.cuh"
namespace mr {
MR_INSTANTIATE_STAGE(3, 17)
}
