// RK stage launchers, 2D, Bs 33.
#include "mr_launch.cuh"
namespace mr {
MR_INSTANTIATE_STAGE(2, 33)
}
