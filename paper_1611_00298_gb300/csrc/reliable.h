// Reliable-update schedule of the mixed-precision solves (Sec. 5.1 names
// mixed precision; the schedule is this library's reading): the way from
// the residual norm r0 at the start of a CG run to the target is split into
// the fewest equal reductions no larger than dmax, so that a reliable
// update ends every segment but the last.  Plain C++ (no CUDA) so that the
// host tests compile it on their own.
#pragma once
#include <algorithm>
#include <cmath>

// The reduction per segment (0 < dmax < 1); dmax itself when r0 is zero or
// already at or below the target.
inline double equal_segment_reduction(double r0, double target, double dmax) {
    if (!(r0 > 0 && target > 0 && target < r0)) return dmax;
    const double L = std::log(target / r0);
    // (the 1e-9 keeps an exact power of dmax at its own segment count)
    const int k = std::max(1, (int)std::ceil(L / std::log(dmax) - 1e-9));
    return std::exp(L / k);
}
