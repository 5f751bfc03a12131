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
};

// Home level of each leaf slot: a free leaf node's defect enters, and its
// correction leaves, the coarsest level among its leaf cells.  Per leaf slot:
// that level's slot offset in the concatenated level storage, its slot on that
// level (-1: hanging node or hole) and that level's slot count.
struct DevHome {
  const int32_t* off = nullptr;
  const int32_t* slot = nullptr;
  const int32_t* nsl = nullptr;
};

// ---- elementwise / sparse kernels (T = float or double for the level vectors)
// pdl: launch as a programmatic dependent launch (pdl.cuh): the kernel waits for
// the preceding kernel of the stream at its start.
template <typename T>
cudaError_t mg_chebyshev_first(int64_t n, T* x, T* xprev, const T* dinv, const T* d, T c0, cudaStream_t s,
                               bool pdl = false);
template <typename T>
cudaError_t mg_chebyshev_step(int64_t n, T* xnew, const T* x, const T* xprev, const T* dinv, const T* d,
                              const T* ax, T a, T b, cudaStream_t s, bool pdl = false);
// d_c[y] += sum_z R[y,z] (d_f[z] - ax_f[z]) over coarse slots; zero on coarse fixed rows.
// With cur_c set, also the coarse level's first Chebyshev iterate (as
// mg_chebyshev_first): cur_c = c0 dinv_c d_c, prev_c = 0.
template <typename T>
cudaError_t mg_restrict(int32_t nc, int ncomp, int64_t nc_stride, int64_t nf_stride, const int32_t* ptr,
                        const int32_t* col, const float* val, const T* d_f, const T* ax_f, T* d_c,
                        const uint8_t* cmask_c, int fixbits, cudaStream_t s, bool pdl = false,
                        const T* dinv_c = nullptr, T* cur_c = nullptr, T* prev_c = nullptr, T c0 = T(0));
// x_f[z] += sum_y P[z,y] x_c[y]; zero on fine fixed rows
template <typename T>
cudaError_t mg_prolong(int32_t nf, int ncomp, int64_t nf_stride, int64_t nc_stride, const int32_t* ptr,
                       const int32_t* col, const float* val, const T* x_c, T* x_f, const uint8_t* cmask_f,
                       int fixbits, cudaStream_t s, bool pdl = false);
// Level vectors of a block: level l at ncomp * off_l, component c at + c * n_slots_l.
// copy_in: d on each free leaf node's home level <- leaf r (double, ncomp blocks of
// stride ns_leaf).  copy_out: z = r on fixed leaf node DoFs, the home-level value
// of x on free ones, 0 on hanging nodes and holes.
template <typename T>
cudaError_t mg_copy_in(int64_t ns_leaf, int ncomp, DevHome home, const double* r, T* d, const uint8_t* leaf_cmask,
                       int fixbits, cudaStream_t s);
template <typename T>
cudaError_t mg_copy_out(int64_t ns_leaf, int ncomp, DevHome home, const T* x, const double* r, double* z,
                        const uint8_t* leaf_cmask, const uint8_t* leaf_flags, int fixbits, cudaStream_t s,
                        bool pdl = false);
// Post-smoothing pieces.  first_res: r = d - ax, x = c0 D^-1 r, xprev = 0; with
// xadd != NULL (degree 1) instead xadd += c0 D^-1 (d - ax), nothing stored.
// step_add: xadd += the Chebyshev step of mg_chebyshev_step (not stored).
template <typename T>
cudaError_t mg_chebyshev_first_res(int64_t n, T* x, T* xprev, T* r, const T* dinv, const T* d, const T* ax, T c0,
                                   T* xadd, cudaStream_t s, bool pdl = false);
template <typename T>
cudaError_t mg_chebyshev_step_add(int64_t n, T* xadd, const T* x, const T* xprev, const T* dinv, const T* d,
                                  const T* ax, T a, T b, cudaStream_t s, bool pdl = false);
// In-place inverse of a dense SPD matrix (n x n, row-major, FP64) by blocked
// Gauss-Jordan elimination without pivoting (panels of 32 pivots, two launches
// each): the pivots are the diagonals of successive Schur complements, positive
// for an SPD matrix.  scr: device scratch of mg_spd_scratch(cap) doubles for any
// n <= cap.  *bad is set to 1 when a pivot is not positive (the matrix is then
// not SPD and A holds no inverse); it is cleared first.
int64_t mg_spd_scratch(int32_t cap);
cudaError_t mg_spd_invert(int32_t n, double* A, double* scr, int32_t* bad, cudaStream_t s);

// coarse solve x[idx] = Ainv (d[idx]) (dense FP64 inverse over the interior entries)
template <typename T>
cudaError_t mg_coarse(int32_t n, const int32_t* idx, const double* Ainv, const T* d, T* x, double* tmp,
                      cudaStream_t s, bool pdl = false);

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
// Jacobi-preconditioned CG on device scalars sc[] = {rz, pq, rz_new, alpha, beta, ok}.
// dot_partial64: the block partial sums of a.b (the grid and order of dot64);
// cg_dot_final: sc[slot] = their sum, then slot 1 sets alpha, slot 2 beta and
// hist[2 step], hist[2 step + 1]; cg_update_r_dot: r -= alpha q, z = D^-1 r with
// the partial sums of r.z; cg_update_p: p = z + beta p.  partial holds
// mg_dot_partials() doubles.
cudaError_t cg_update_p(int64_t n, double* p, const double* z, const double* sc, cudaStream_t s);
cudaError_t dot_partial64(int64_t n, const double* a, const double* b, double* partial, cudaStream_t s);
cudaError_t cg_dot_final(const double* partial, double* sc, int slot, double* hist, int step, cudaStream_t s);
cudaError_t cg_update_r_dot(int64_t n, double* r, double* z, const double* q, const double* dinv, const double* sc,
                            double* partial, cudaStream_t s);
// CG scalars {rz, pq, rz_new, alpha, beta, ok, -, -} = {0, 0, 0, 0, 0, 1, 0, 0}
cudaError_t cg_init_scalars(double* sc, cudaStream_t s);
// number of per-block partial sums dot64 writes (its partial buffer holds this many doubles)
int mg_dot_partials();
cudaError_t fill64(int64_t n, double* x, double v, cudaStream_t s);
cudaError_t copy64(int64_t n, double* dst, const double* src, cudaStream_t s);

}  // namespace pff
