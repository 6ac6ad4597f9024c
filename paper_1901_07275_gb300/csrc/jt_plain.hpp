// Plain FP64 comparison path (JT_FP64_PLAIN): the transform as the r^d d-dimensional FFT
// form the paper names in its abstract and conclusion, unfused, with cuFFT Z2Z.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "jt.h"
#include "jt_internal.hpp"

namespace jt {

// Size of the fixed device work area used by plain_apply_static (16 MiB).
#define JT_STATIC_SCRATCH_BYTES (16u << 20)

struct PlainPlan;

jt_status plain_create(PlainPlan** out, const std::vector<const AxisTables*>& axes, cudaStream_t s);
jt_status plain_apply(PlainPlan* p, const double* in, double* out, int64_t nrhs, bool fwd, cudaStream_t s);
// Same apply with the work buffers carved from the library's static device array instead of
// the plan's own: allocates nothing; JT_EINVAL if the plan needs more than the array holds.
jt_status plain_apply_static(PlainPlan* p, const double* in, double* out, int64_t nrhs, bool fwd, cudaStream_t s);
size_t plain_static_bytes(const PlainPlan* p);
void plain_destroy(PlainPlan* p);

}  // namespace jt
