// RK stage launchers, 2D, Bs 17.
#include "mr_launch.cuh"
namespace mr {
MR_INSTANTIATE_STAGE(2, 17)
}
