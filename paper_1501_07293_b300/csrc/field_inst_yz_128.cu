// Instances of the y/z pass for py = 128.
#define FIELD_INSTANTIATE
#include "field_kernels.cuh"

FK_INSTANTIATE_YZ(128)
