// Instances of the y/z pass for py = 2048.
#define FIELD_INSTANTIATE
#include "field_kernels.cuh"

FK_INSTANTIATE_YZ(2048)
