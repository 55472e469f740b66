// Shared-memory kernels of the double integrator model.
#define TMPC_FAST_MODEL tmpc::MODEL_DI
#include "tmpc_fast_model.cuh"
