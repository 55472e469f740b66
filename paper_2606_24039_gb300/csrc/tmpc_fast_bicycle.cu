// Shared-memory kernels of the kinematic bicycle model.
#define TMPC_FAST_MODEL tmpc::MODEL_BICYCLE
#include "tmpc_fast_model.cuh"
