// Per-cell fields on the brick layout (per-cell Young's modulus E_K and its gradient).
//
// A cell's value lives at its "cell slot": the slot of the cell's lower-left node
// position in a brick of the cell's own level (leaf layout for leaf cells, the
// level layout of level l for the multigrid level operators of Sec. 3.2).  On a
// level, a leaf cell takes its leaf value and a refined cell the mean of its four
// children, computed from the finest level down.
#include "state.h"

namespace pff {

namespace {

__global__ void k_cells_scatter(int32_t n, const double* __restrict__ v, const int32_t* __restrict__ slot,
                                double* out64, float* out32) {
  const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const double x = v[c];
  out64[slot[c]] = x;
  out32[slot[c]] = float(x);
}

__global__ void k_cells_level(int32_t n, const int32_t* __restrict__ dst, const int32_t* __restrict__ src,
                              const int32_t* __restrict__ child, const double* __restrict__ leaf_v,
                              const double* __restrict__ finer, double* out64, float* out32) {
  const int32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int32_t s = src[q];
  double x;
  if (s >= 0) {
    x = leaf_v[s];
  } else {
    const int32_t* ch = child + 4 * (-1 - s);
    x = 0.25 * (((finer[ch[0]] + finer[ch[1]]) + finer[ch[2]]) + finer[ch[3]]);
  }
  out64[dst[q]] = x;
  out32[dst[q]] = float(x);
}

__global__ void k_cells_gather(int32_t n, const double* __restrict__ in, const int32_t* __restrict__ slot,
                               double* out) {
  const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  out[c] = in[slot[c]];
}

inline unsigned blocks(int32_t n) { return unsigned((int64_t(n) + 255) / 256); }

}  // namespace

cudaError_t cells_scatter(int32_t n, const double* v, const int32_t* slot, double* out64, float* out32,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_cells_scatter<<<blocks(n), 256, 0, s>>>(n, v, slot, out64, out32);
  return cudaGetLastError();
}

cudaError_t cells_level(int32_t n, const int32_t* dst, const int32_t* src, const int32_t* child,
                        const double* leaf_v, const double* finer, double* out64, float* out32, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_cells_level<<<blocks(n), 256, 0, s>>>(n, dst, src, child, leaf_v, finer, out64, out32);
  return cudaGetLastError();
}

cudaError_t cells_gather(int32_t n, const double* in, const int32_t* slot, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_cells_gather<<<blocks(n), 256, 0, s>>>(n, in, slot, out);
  return cudaGetLastError();
}

}  // namespace pff
