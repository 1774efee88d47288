// FP32 instantiation of the MBO kernels (FP64 accumulation of the energy,
// FP64 re-projection of ill-conditioned points).
#include "mbo_kernels.cuh"
namespace mbo {
MBO_INSTANTIATE(float)
}
