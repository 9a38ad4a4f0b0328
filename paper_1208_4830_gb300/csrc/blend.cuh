// blend.cuh -- the blended model of Section 4.4 (Eq. blend), A_obs = f A + (1 - f), with the
// blending fraction profiled out: with a = A - 1, b = F - 1 and w = 1/sigma^2 the least-squares f
// is sum w a b / sum w a^2 (clamped to [f_min, 1]; 1 when sum w a^2 = 0) and the chi^2 is
// sum w (b - f a)^2. Callers sum the epochs in a fixed order (per thread, then a fixed tree).
#pragma once

#include <cuda_runtime.h>

namespace sblm {

__device__ __forceinline__ double blend_f(double s_ab, double s_aa, double f_min) {
    const double f = s_aa > 0.0 ? s_ab / s_aa : 1.0;
    return fmin(1.0, fmax(f_min, f));
}

}  // namespace sblm
