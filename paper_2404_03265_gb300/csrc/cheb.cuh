// Chebyshev-Jacobi smoother updates (Sec. 3.2), one entry at a time.  The
// element-wise V-cycle kernels and the level sweep's fused store both use these,
// so the two paths round the same expression.
#pragma once

namespace pff {

// the next iterate of the three-term recurrence: x + a (x - x_prev) + b D^-1 (d - A x)
template <typename T>
__device__ __forceinline__ T cheb_next(T xi, T xprev, T dinv, T d, T ax, T a, T b) {
  return xi + a * (xi - xprev) + b * dinv * (d - ax);
}

// the first iterate from a residual r: c0 D^-1 r
template <typename T>
__device__ __forceinline__ T cheb_first_of(T c0, T dinv, T r) {
  return c0 * dinv * r;
}

}  // namespace pff
