// Instances of the y/z pass for py = 1024.
#define FIELD_INSTANTIATE
#include "field_kernels.cuh"

FK_INSTANTIATE_YZ(1024)
