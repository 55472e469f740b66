// Shared-memory kernels of the planar quadrotor model.
#define TMPC_FAST_MODEL tmpc::MODEL_QUAD
#include "tmpc_fast_model.cuh"
