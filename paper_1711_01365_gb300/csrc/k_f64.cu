// FP64 instantiation of the MBO kernels.
#include "mbo_kernels.cuh"
namespace mbo {
MBO_INSTANTIATE(double)
}
