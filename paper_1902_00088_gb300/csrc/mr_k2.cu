// 2D instantiation of the kernel templates (Bs 17 and 33); the RK stages are
// instantiated in mr_k2s.cu (Bs 17) and mr_k2t.cu (Bs 33).
#include "mr_launch.cuh"
namespace mr {
MR_EXTERN_STAGE(2, 17)
MR_EXTERN_STAGE(2, 33)
MR_INSTANTIATE(2)
}
