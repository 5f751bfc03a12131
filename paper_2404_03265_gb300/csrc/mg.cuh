// Multigrid kernels of libpff (Sec. 3.2 of Kolditz & Wick: Chebyshev-Jacobi
// smoothed geometric multigrid with local smoothing on the diagonal blocks).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace pff {

// Level-mesh device tables (one per refinement level).
struct DevLevel {
  int32_t n_slots = 0;
  int64_t off = 0;                 // slot offset of this level in concatenated level storage
  const uint8_t* flags = nullptr;  // bit0 node, bit1 Dirichlet, bit3 refinement edge, bit4 home of a leaf DoF
  const int32_t* slot_leaf = nullptr;
  const int32_t* P_ptr = nullptr;  // prolongation rows (this level's slots) -> level-1 slots
  const int32_t* P_col = nullptr;
  const float* P_val = nullptr;
  const int32_t* R_ptr = nullptr;  // restriction rows (level-1 slots) -> this level's slots
  const int32_t* R_col = nullptr;
  const float* R_val = nullptr;
  int32_t n_copy = 0;              // leaf nodes whose home level is this one
  const int32_t* copy_leaf = nullptr;
  const int32_t* copy_level = nullptr;
};

// ---- elementwise / sparse kernels (T = float or double for the level vectors)
template <typename T>
cudaError_t mg_chebyshev_first(int64_t n, T* x, T* xprev, const T* dinv, const T* d, T c0, cudaStream_t s);
template <typename T>
cudaError_t mg_chebyshev_step(int64_t n, T* xnew, const T* x, const T* xprev, const T* dinv, const T* d,
                              const T* ax, T a, T b, cudaStream_t s);
template <typename T>
cudaError_t mg_residual(int64_t n, T* r, const T* d, const T* ax, cudaStream_t s);
template <typename T>
cudaError_t mg_axpy(int64_t n, T* y, const T* x, T a, cudaStream_t s);
// d_c[y] += sum_z R[y,z] (d_f[z] - ax_f[z]) over coarse slots; zero on coarse fixed rows
template <typename T>
cudaError_t mg_restrict(int32_t nc, int ncomp, int64_t nc_stride, int64_t nf_stride, const int32_t* ptr,
                        const int32_t* col, const float* val, const T* d_f, const T* ax_f, T* d_c,
                        const uint8_t* cmask_c, int fixbits, cudaStream_t s);
// x_f[z] += sum_y P[z,y] x_c[y]; zero on fine fixed rows
template <typename T>
cudaError_t mg_prolong(int32_t nf, int ncomp, int64_t nf_stride, int64_t nc_stride, const int32_t* ptr,
                       const int32_t* col, const float* val, const T* x_c, T* x_f, const uint8_t* cmask_f,
                       int fixbits, cudaStream_t s);
// level d (ncomp blocks of stride ns_l) <- leaf r (double, ncomp blocks of stride ns_leaf) on free leaf nodes
template <typename T>
cudaError_t mg_copy_in(int32_t n, int ncomp, const int32_t* leaf_slot, const int32_t* lev_slot, const double* r,
                       int64_t ns_leaf, T* d, int64_t ns_l, const uint8_t* leaf_cmask, int fixbits,
                       cudaStream_t s);
template <typename T>
cudaError_t mg_copy_out(int32_t n, int ncomp, const int32_t* leaf_slot, const int32_t* lev_slot, const T* x,
                        int64_t ns_l, double* z, int64_t ns_leaf, const uint8_t* leaf_cmask, int fixbits,
                        cudaStream_t s);
// z = r on fixed leaf DoFs, 0 elsewhere (hanging nodes and holes included)
cudaError_t mg_leaf_init(int64_t ns_leaf, int ncomp, const double* r, double* z, const uint8_t* leaf_cmask,
                         const uint8_t* leaf_flags, int fixbits, cudaStream_t s);
// In-place inverse of a dense SPD matrix (n x n, row-major, FP64) by Gauss-Jordan
// sweeps without pivoting: the pivots are the diagonals of successive Schur
// complements, positive for an SPD matrix.  rc: scratch of 4 n doubles.  *bad is
// set to 1 when a pivot is not positive (the matrix is then not SPD and A holds
// no inverse); it is cleared first.
cudaError_t mg_spd_invert(int32_t n, double* A, double* rc, int32_t* bad, cudaStream_t s);

// coarse solve x[idx] = Ainv (d[idx]) (dense FP64 inverse over the interior entries)
template <typename T>
cudaError_t mg_coarse(int32_t n, const int32_t* idx, const double* Ainv, const T* d, T* x, double* tmp,
                      cudaStream_t s);

// ---- set-up kernels
// level lin (4 blocks of ns_l, double and float) from leaf lin64 (4 blocks of ns_leaf)
cudaError_t mg_inject_lin(int32_t ns_l, const int32_t* slot_leaf, const double* lin64, int64_t ns_leaf,
                          double* lev64, float* lev32, cudaStream_t s);
// level cmask: bits 0,1 Dirichlet, bit 2 active (leaf active at the position, or, below the
// home level, an active child on the next finer level)
cudaError_t mg_level_cmask(int32_t ns_l, const uint8_t* flags, const int32_t* slot_leaf, const uint8_t* leaf_cmask,
                           const int32_t* R_ptr, const int32_t* R_col, const uint8_t* cmask_fine,
                           uint8_t* cmask, cudaStream_t s);
// dinv = 1 / diag on interior entries (node, not fixed, not edge), else 0; both precisions
cudaError_t mg_invert_diag(int32_t ns_l, int ncomp, const double* diag, const uint8_t* flags,
                           const uint8_t* cmask, int fixbits0, double* dinv64, float* dinv32, cudaStream_t s);
// Lanczos start vector on interior entries: 1 + 0.01 * (splitmix64((gx << 32) | gy) mod 1000) / 1000
cudaError_t mg_start_vector(int32_t ns_l, int ncomp, const int32_t* gx, const int32_t* gy, const double* dinv,
                            double* r, cudaStream_t s);
// deterministic dot product: partial sums per block, then one ordered sum -> out[0]
cudaError_t dot64(int64_t n, const double* a, const double* b, double* partial, double* out, cudaStream_t s);
// CG step pieces on device scalars sc[] = {rz, pq, rz_new, alpha, beta, ok}
cudaError_t cg_update_r(int64_t n, double* r, double* z, const double* q, const double* dinv, const double* sc,
                        cudaStream_t s);
cudaError_t cg_update_p(int64_t n, double* p, const double* z, const double* sc, cudaStream_t s);
cudaError_t cg_scalars_alpha(double* sc, cudaStream_t s);
cudaError_t cg_scalars_beta(double* sc, double* hist, int step, cudaStream_t s);
cudaError_t fill64(int64_t n, double* x, double v, cudaStream_t s);
cudaError_t copy64(int64_t n, double* dst, const double* src, cudaStream_t s);

}  // namespace pff
