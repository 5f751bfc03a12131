// Kernels of the Newton / PDAS loop and of GMRES (solve.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"

namespace pff {

// state (4 blocks: u_x, u_y, phi, phi_tilde) with hanging entries from their constraint
cudaError_t make_state(int64_t n, const double* u, const double* phi, const double* phit, const uint8_t* flags,
                       const DevHanging* hang, int32_t nhang, int fe_degree, double* st, cudaStream_t s);
// v[h] = sum_b w_b v[parent_b] on the first nblk blocks of v
cudaError_t distribute_hanging(int64_t n, const DevHanging* hang, int32_t nhang, int fe_degree, int nblk, double* v,
                               cudaStream_t s);
// stats[0] += changes vs prev, stats[1] += active count, stats[2] = min |indicator| (IEEE bits)
cudaError_t active_set(int64_t n, const double* R, const double* B, const double* phi, const double* phi_old,
                       const uint8_t* flags, double c, const uint8_t* prev, uint8_t* act, unsigned long long* stats,
                       cudaStream_t s);
cudaError_t newton_residual(int64_t n, const double* R, const uint8_t* act, const double* phi,
                            const double* phi_old, const uint8_t* flags, double* out, cudaStream_t s);
cudaError_t newton_rhs(int64_t n, const double* R, const double* t, const uint8_t* act, const double* phi,
                       const double* phi_old, const uint8_t* flags, double* rhs, cudaStream_t s);
cudaError_t newton_du0(int64_t n, const uint8_t* act, const double* phi, const double* phi_old, double* du0,
                       cudaStream_t s);
cudaError_t f64_to_f32(int64_t n, const double* a, float* b, cudaStream_t s);
cudaError_t f32_to_f64(int64_t n, const float* a, double* b, cudaStream_t s);
// out = x with fixed components (constraint mask) zeroed, 3 blocks of n
cudaError_t mask_fixed(int64_t n, const uint8_t* cmask, const double* x, double* out, cudaStream_t s);
// out = x on the rows cmask marks fixed; the other rows of out are left as they are
cudaError_t copy_fixed(int64_t n, const uint8_t* cmask, const double* x, double* out, cudaStream_t s);
// g = (0, 0, -t2 + act * (mu_phi - t1_phi)): adjoint right-hand side of the previous load step.
// With p1 = phi^(k-1), p2 = phi^(k-2) (extrapolated phi_tilde of step k): -2 chi t2 in
// place of -t2 (chi: 1 where 2 p1 - p2 lies strictly inside (0, 1)), pend_in (may be
// null) added, and pend_out = chi t2 (may be null; may alias pend_in) for step k - 2.
cudaError_t adj_carry(int64_t n, const uint8_t* act, const double* mu, const double* t1, const double* t2, double* g,
                      cudaStream_t s, const double* p1 = nullptr, const double* p2 = nullptr,
                      const double* pend_in = nullptr, double* pend_out = nullptr);
cudaError_t axpby(int64_t n, double* out, const double* x, double a, const double* y, double b, cudaStream_t s);
int reduction_partials();
// Krylov basis V in row blocks: entry i of basis vector j at
// (i / kBasisBlock) ldb + j kBasisBlock + i % kBasisBlock, ldb = (vectors held) kBasisBlock,
// so the rows of one block of all vectors are adjacent in memory.
constexpr int64_t kBasisBlock = 2048;
inline int64_t basis_blocks(int64_t n) { return (n + kBasisBlock - 1) / kBasisBlock; }
// out[j] = V_j . w, j < k
cudaError_t multidot(int64_t n, int k, const double* V, int64_t ldb, const double* w, double* partial, double* out,
                     cudaStream_t s);
// w[map[i]] += sign * sum_j h[j] V_j[i]  (h on the device; map[i] = i when map is null)
cudaError_t multi_axpy(int64_t n, int k, const double* V, int64_t ldb, const double* h, double sign, double* w,
                       cudaStream_t s, const int32_t* map = nullptr);
// V_j = a x, and vc[map[i]] = a x[i] (map[i] = i when map is null; x may then be vc)
cudaError_t store_basis(int64_t n, double* V, int64_t ldb, int j, const double* x, double a, double* vc,
                        cudaStream_t s, const int32_t* map = nullptr);
// out[i] = x[map[i]], i < n
cudaError_t gather(int64_t n, const int32_t* map, const double* x, double* out, cudaStream_t s);
cudaError_t vsum(int64_t n, const double* a, double* partial, double* out, cudaStream_t s);
// phi_tilde = clip(2 phi^(n-1) - phi^(n-2), 0, 1) per slot
cudaError_t extrapolate_phi(int64_t n, const double* p1, const double* p2, double* out, cudaStream_t s);
cudaError_t all_finite(int64_t n, const double* a, int* bad, cudaStream_t s);

}  // namespace pff
