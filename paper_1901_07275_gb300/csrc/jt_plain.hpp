// Plain FP64 comparison path (JT_FP64_PLAIN): the transform as the r^d d-dimensional FFT
// form the paper names in its abstract and conclusion, unfused, with cuFFT Z2Z.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "jt.h"
#include "jt_internal.hpp"

namespace jt {

struct PlainPlan;

jt_status plain_create(PlainPlan** out, const std::vector<const AxisTables*>& axes, cudaStream_t s);
jt_status plain_apply(PlainPlan* p, const double* in, double* out, int64_t nrhs, bool fwd, cudaStream_t s);
void plain_destroy(PlainPlan* p);

}  // namespace jt
