// Instances of the x pass (inverse/forward x transforms, update) for px = 1, px = 4, px = 8, px = 16, px = 32, px = 64, px = 128.
#define FIELD_INSTANTIATE
#include "field_kernels.cuh"

FK_INSTANTIATE_X(0)
FK_INSTANTIATE_X(2)
FK_INSTANTIATE_X(4)
FK_INSTANTIATE_X(8)
FK_INSTANTIATE_X(16)
FK_INSTANTIATE_X(32)
FK_INSTANTIATE_X(64)
