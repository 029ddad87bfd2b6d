// Tensor-core (tcgen05) sweep products for the mixed-precision dense model.
#include "wc4d_internal.cuh"

bool tc_sweep_supported(const wc4d_ctx *, int) { return false; }
bool tc_sweep_forward(wc4d_ctx *, int, float *, int64_t) { return false; }
bool tc_sweep_adjoint(wc4d_ctx *, int, float *, int64_t) { return false; }
