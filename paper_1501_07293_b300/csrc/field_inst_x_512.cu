// Instances of the x pass (inverse/forward x transforms, update) for px = 1024.
#define FIELD_INSTANTIATE
#include "field_kernels.cuh"

FK_INSTANTIATE_X(512)
