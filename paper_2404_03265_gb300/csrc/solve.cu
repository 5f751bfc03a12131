// Element-wise kernels of the Newton / primal-dual active set loop (Algorithm 2
// of Kolditz & Wick, arXiv 2404.03265) and the Krylov kernels of GMRES.
//
// A full vector has three blocks of n_slots doubles: u_x, u_y, phi.
// Leaf slot flags: bit0 node, bit1 boundary (Dirichlet u), bit2 hanging.
// All reductions are deterministic (fixed partition, fixed summation order).
#include <cstdint>

#include "kernels.cuh"
#include "solve.cuh"

namespace pff {

namespace {

constexpr int TPB = 256;
constexpr int RED_BLOCKS = 512;

inline unsigned blocks_for(int64_t n) {
  int64_t b = (n + TPB - 1) / TPB;
  if (b > 65535 * 8) b = 65535 * 8;
  return unsigned(b < 1 ? 1 : b);
}

#define GRID_STRIDE(i, n) \
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < (n); i += int64_t(gridDim.x) * blockDim.x)

__global__ void k_make_state(int64_t n, const double* __restrict__ u, const double* __restrict__ phi,
                             const double* __restrict__ phit, const uint8_t* __restrict__ flags, double* st) {
  GRID_STRIDE(s, n) {
    const bool node = flags[s] & 1;
    st[s] = node ? u[s] : 0.0;
    st[n + s] = node ? u[n + s] : 0.0;
    st[2 * n + s] = node ? phi[s] : 0.0;
    st[3 * n + s] = node ? phit[s] : 0.0;
  }
}

__global__ void k_state_hanging(int32_t nh, int64_t n, const DevHanging* __restrict__ hang, int np, int nblk,
                                double* v) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= nh) return;
  const DevHanging e = hang[h];
  for (int k = 0; k < nblk; ++k) {
    double acc = 0.0;
    for (int b = 0; b < np; ++b) acc += e.weight[b] * v[k * n + e.parent[b]];
    v[k * n + e.slot] = acc;
  }
}

// active set: ind = R_phi / B + c (phi - phi_old) > 0 on non-hanging nodes
__global__ void k_active(int64_t n, const double* __restrict__ R, const double* __restrict__ B,
                         const double* __restrict__ phi, const double* __restrict__ phio,
                         const uint8_t* __restrict__ flags, double c, const uint8_t* __restrict__ prev,
                         uint8_t* act, unsigned long long* stats) {
  GRID_STRIDE(s, n) {
    const uint8_t f = flags[s];
    uint8_t a = 0;
    if ((f & 1) && !(f & 4)) {
      // c > 0: constant c; c <= 0: c_i = 2 |lambda_i / (phi_i - phi_old_i)| (Sec. 2), so that
      // c_i (phi_i - phi_old_i) = 2 |lambda_i| sign(phi_i - phi_old_i).  Products and sums are
      // rounded separately (no contraction), as in the reference evaluation of the rule.
      const double lam = __ddiv_rn(R[2 * n + s], B[s]);
      const double d = __dsub_rn(phi[s], phio[s]);
      const double ind = c > 0.0 ? __dadd_rn(lam, __dmul_rn(c, d))
                                 : __dadd_rn(lam, d > 0.0 ? 2.0 * fabs(lam) : (d < 0.0 ? -2.0 * fabs(lam) : 0.0));
      a = ind > 0.0 ? 1 : 0;
      // |ind| as its IEEE bit pattern: ordered like the value for non-negative doubles
      const double ai = fabs(ind);
      atomicMin(stats + 2, (unsigned long long)__double_as_longlong(ai));
      if (a) atomicAdd(stats + 1, 1ull);
    }
    if (a != (prev ? prev[s] : 0)) atomicAdd(stats + 0, 1ull);
    act[s] = a;
  }
}

// Newton residual: R on free rows, phi_old - phi on active phi rows, 0 on Dirichlet / hanging / holes
__global__ void k_newton_res(int64_t n, const double* __restrict__ R, const uint8_t* __restrict__ act,
                             const double* __restrict__ phi, const double* __restrict__ phio,
                             const uint8_t* __restrict__ flags, double* out) {
  GRID_STRIDE(s, n) {
    const uint8_t f = flags[s];
    const bool node = (f & 1) && !(f & 4);
    const bool dir = f & 2;
    out[s] = (node && !dir) ? R[s] : 0.0;
    out[n + s] = (node && !dir) ? R[n + s] : 0.0;
    out[2 * n + s] = node ? (act[s] ? phio[s] - phi[s] : R[2 * n + s]) : 0.0;
  }
}

// rhs = (R - t) on free rows, dU0 = phi_old - phi on active phi rows, 0 elsewhere
__global__ void k_newton_rhs(int64_t n, const double* __restrict__ R, const double* __restrict__ t,
                             const uint8_t* __restrict__ act, const double* __restrict__ phi,
                             const double* __restrict__ phio, const uint8_t* __restrict__ flags, double* rhs) {
  GRID_STRIDE(s, n) {
    const uint8_t f = flags[s];
    const bool node = (f & 1) && !(f & 4);
    const bool dir = f & 2;
    rhs[s] = (node && !dir) ? R[s] - t[s] : 0.0;
    rhs[n + s] = (node && !dir) ? R[n + s] - t[n + s] : 0.0;
    rhs[2 * n + s] = node ? (act[s] ? phio[s] - phi[s] : R[2 * n + s] - t[2 * n + s]) : 0.0;
  }
}

// dU0: phi_old - phi on active phi DoFs, 0 elsewhere
__global__ void k_du0(int64_t n, const uint8_t* __restrict__ act, const double* __restrict__ phi,
                      const double* __restrict__ phio, double* du0) {
  GRID_STRIDE(s, n) {
    du0[s] = 0.0;
    du0[n + s] = 0.0;
    du0[2 * n + s] = act[s] ? phio[s] - phi[s] : 0.0;
  }
}

__global__ void k_f64_to_f32(int64_t n, const double* __restrict__ a, float* b) {
  GRID_STRIDE(s, n) b[s] = float(a[s]);
}
__global__ void k_f32_to_f64(int64_t n, const float* __restrict__ a, double* b) {
  GRID_STRIDE(s, n) b[s] = double(a[s]);
}

// out = x with the fixed components (constraint-mask bits 0, 1, 2) zeroed; 3 blocks
__global__ void k_mask_fixed(int64_t n, const uint8_t* __restrict__ cmask, const double* __restrict__ x,
                             double* out) {
  GRID_STRIDE(s, n) {
    const uint8_t cm = cmask[s];
    out[s] = (cm & 1) ? 0.0 : x[s];
    out[n + s] = (cm & 2) ? 0.0 : x[n + s];
    out[2 * n + s] = (cm & 4) ? 0.0 : x[2 * n + s];
  }
}

// out = x on the fixed rows of cmask (bit 1, 2: u_x, u_y; bit 4: phi), out unchanged elsewhere
__global__ void k_copy_fixed(int64_t n, const uint8_t* __restrict__ cmask, const double* __restrict__ x,
                             double* out) {
  GRID_STRIDE(s, n) {
    const uint8_t cm = cmask[s];
    if (cm & 1) out[s] = x[s];
    if (cm & 2) out[n + s] = x[n + s];
    if (cm & 4) out[2 * n + s] = x[2 * n + s];
  }
}

// Adjoint carry to the previous load step:
// g = (0, 0, -w t2 + act (mu_phi - t1_phi) + pend_in).  phi_tilde = phi^(k-1)
// (p1 null): w = 1.  Extrapolated phi_tilde = clip(2 p1 - p2, 0, 1): w = 2 chi on
// the slots strictly inside the clip (chi = 1, else 0), and pend_out = chi t2 is
// the share that reaches the step before the previous one (weight -1 there, so
// +chi t2 on its right-hand side).  pend_in may alias pend_out.
__global__ void k_adj_carry(int64_t n, const uint8_t* __restrict__ act, const double* __restrict__ mu,
                            const double* __restrict__ t1, const double* __restrict__ t2,
                            const double* __restrict__ p1, const double* __restrict__ p2, const double* pend_in,
                            double* pend_out, double* g) {
  GRID_STRIDE(s, n) {
    const double v = t2[s];
    double w = 1.0, chi = 0.0;
    if (p1) {
      const double raw = 2.0 * p1[s] - p2[s];
      chi = (raw > 0.0 && raw < 1.0) ? 1.0 : 0.0;
      w = 2.0 * chi;
    }
    double gp = -w * v + (act[s] ? mu[2 * n + s] - t1[2 * n + s] : 0.0);
    if (pend_in) gp += pend_in[s];
    g[s] = 0.0;
    g[n + s] = 0.0;
    g[2 * n + s] = gp;
    if (pend_out) pend_out[s] = chi * v;
  }
}

__global__ void k_axpby(int64_t n, double* out, const double* __restrict__ x, double a, const double* __restrict__ y,
                        double b) {
  GRID_STRIDE(i, n) out[i] = a * x[i] + b * y[i];
}

// phi_tilde = clip(2 phi^(n-1) - phi^(n-2), 0, 1)
__global__ void k_extrapolate_phi(int64_t n, const double* __restrict__ p1, const double* __restrict__ p2,
                                  double* out) {
  GRID_STRIDE(i, n) out[i] = fmin(fmax(2.0 * p1[i] - p2[i], 0.0), 1.0);
}


// Krylov basis storage: rows in blocks of kBasisBlock; block r holds the rows
// r kBasisBlock .. of every basis vector j contiguously, at r ldb + j kBasisBlock.
__device__ __forceinline__ int64_t basis_row(int64_t i, int64_t ldb) {
  return (i / kBasisBlock) * ldb + (i % kBasisBlock);
}

// partial[b * k + j] = sum over this block's rows of V_j . w.  The basis vectors
// go in chunks of MD_J (the last one of k mod MD_J, its own instantiation, so no
// multiply is spent on padding); a thread visits its rows i = t, t + S, t + 2 S,
// ... (S = the grid's thread count) in that order, as a plain grid-stride dot
// does, but issues the loads of MD_R consecutive visits (w and the chunk's basis
// entries each) together.  It keeps one sum per vector of the chunk, and the
// block reduces them in one shared-memory tree (fixed order).
constexpr int MD_J = 8;
constexpr int MD_R = 4;
template <int JN>
__device__ __forceinline__ void md_chunk(int64_t n, const double* __restrict__ Vc, int64_t ldb,
                                         const double* __restrict__ w, double (&sh)[MD_J][TPB]) {
  const int64_t S = int64_t(gridDim.x) * TPB;
  double acc[JN];
#pragma unroll
  for (int q = 0; q < JN; ++q) acc[q] = 0.0;
  for (int64_t i0 = int64_t(blockIdx.x) * TPB + threadIdx.x; i0 < n; i0 += MD_R * S) {
    double wv[MD_R], vv[JN][MD_R];
#pragma unroll
    for (int e = 0; e < MD_R; ++e) {
      const int64_t i = i0 + e * S;
      const int64_t bi = basis_row(i, ldb);
      wv[e] = i < n ? w[i] : 0.0;
#pragma unroll
      for (int q = 0; q < JN; ++q) vv[q][e] = i < n ? Vc[bi + q * kBasisBlock] : 0.0;
    }
#pragma unroll
    for (int e = 0; e < MD_R; ++e) {
      if (i0 + e * S < n) {
#pragma unroll
        for (int q = 0; q < JN; ++q) acc[q] += vv[q][e] * wv[e];
      }
    }
  }
#pragma unroll
  for (int q = 0; q < JN; ++q) sh[q][threadIdx.x] = acc[q];
}

__global__ void k_multidot_partial(int64_t n, int k, const double* __restrict__ V, int64_t ldb,
                                   const double* __restrict__ w, double* partial) {
  __shared__ double sh[MD_J][TPB];
  for (int j0 = 0; j0 < k; j0 += MD_J) {
    const int jn = k - j0 < MD_J ? k - j0 : MD_J;
    const double* Vc = V + int64_t(j0) * kBasisBlock;
    switch (jn) {
      case 1: md_chunk<1>(n, Vc, ldb, w, sh); break;
      case 2: md_chunk<2>(n, Vc, ldb, w, sh); break;
      case 3: md_chunk<3>(n, Vc, ldb, w, sh); break;
      case 4: md_chunk<4>(n, Vc, ldb, w, sh); break;
      case 5: md_chunk<5>(n, Vc, ldb, w, sh); break;
      case 6: md_chunk<6>(n, Vc, ldb, w, sh); break;
      case 7: md_chunk<7>(n, Vc, ldb, w, sh); break;
      default: md_chunk<8>(n, Vc, ldb, w, sh); break;
    }
    __syncthreads();
    for (int o = TPB / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        for (int q = 0; q < jn; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
      }
      __syncthreads();
    }
    if (threadIdx.x < jn) partial[int64_t(blockIdx.x) * k + j0 + threadIdx.x] = sh[threadIdx.x][0];
    __syncthreads();
  }
}

__global__ void k_multidot_final(int nb, int k, const double* __restrict__ partial, double* out) {
  __shared__ double sh[TPB];
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += TPB) acc += partial[int64_t(b) * k + j];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = TPB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = sh[0];
}

// w[map(i)] += sign * sum_j h_j V_j[i] (the sum in the order j = 0, 1, ...; loads
// of four basis entries are issued together; h staged in shared memory; map(i) = i
// without a map)
constexpr int MAX_BASIS = 512;
__global__ void k_multi_axpy(int64_t n, int k, const double* __restrict__ V, int64_t ldb, const double* __restrict__ h,
                             double sign, double* w, const int32_t* __restrict__ map) {
  __shared__ double hs[MAX_BASIS];
  for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = h[j];
  __syncthreads();
  GRID_STRIDE(i, n) {
    const double* Vi = V + basis_row(i, ldb);
    double acc = 0.0;
    int j = 0;
    for (; j + 4 <= k; j += 4) {
      const double v0 = Vi[j * kBasisBlock], v1 = Vi[(j + 1) * kBasisBlock], v2 = Vi[(j + 2) * kBasisBlock],
                   v3 = Vi[(j + 3) * kBasisBlock];
      acc += hs[j] * v0;
      acc += hs[j + 1] * v1;
      acc += hs[j + 2] * v2;
      acc += hs[j + 3] * v3;
    }
    for (; j < k; ++j) acc += hs[j] * Vi[j * kBasisBlock];
    const int64_t o = map ? int64_t(map[i]) : i;
    w[o] += sign * acc;
  }
}

// basis vector j = a x, also written to vc[map(i)] (map(i) = i without a map; x may
// be vc when there is no map)
__global__ void k_store_basis(int64_t n, double* V, int64_t ldb, int j, const double* x, double a, double* vc,
                              const int32_t* __restrict__ map) {
  GRID_STRIDE(i, n) {
    const double v = a * x[i];
    V[basis_row(i, ldb) + int64_t(j) * kBasisBlock] = v;
    vc[map ? int64_t(map[i]) : i] = v;
  }
}

__global__ void k_gather(int64_t n, const int32_t* __restrict__ map, const double* __restrict__ x, double* out) {
  GRID_STRIDE(i, n) out[i] = x[map[i]];
}

__global__ void k_sum_partial(int64_t n, const double* __restrict__ a, double* part) {
  __shared__ double sh[TPB];
  double acc = 0.0;
  GRID_STRIDE(i, n) acc += a[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = TPB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_all_finite(int64_t n, const double* __restrict__ a, int* bad) {
  GRID_STRIDE(i, n) if (!isfinite(a[i])) atomicOr(bad, 1);
}

}  // namespace

cudaError_t make_state(int64_t n, const double* u, const double* phi, const double* phit, const uint8_t* flags,
                       const DevHanging* hang, int32_t nhang, int fe_degree, double* st, cudaStream_t s) {
  if (n > 0) k_make_state<<<blocks_for(n), TPB, 0, s>>>(n, u, phi, phit, flags, st);
  if (nhang > 0) k_state_hanging<<<(nhang + 127) / 128, 128, 0, s>>>(nhang, n, hang, fe_degree + 1, 4, st);
  return cudaGetLastError();
}

cudaError_t distribute_hanging(int64_t n, const DevHanging* hang, int32_t nhang, int fe_degree, int nblk, double* v,
                               cudaStream_t s) {
  if (nhang > 0) k_state_hanging<<<(nhang + 127) / 128, 128, 0, s>>>(nhang, n, hang, fe_degree + 1, nblk, v);
  return cudaGetLastError();
}

cudaError_t active_set(int64_t n, const double* R, const double* B, const double* phi, const double* phi_old,
                       const uint8_t* flags, double c, const uint8_t* prev, uint8_t* act, unsigned long long* stats,
                       cudaStream_t s) {
  if (n > 0) k_active<<<blocks_for(n), TPB, 0, s>>>(n, R, B, phi, phi_old, flags, c, prev, act, stats);
  return cudaGetLastError();
}

cudaError_t newton_residual(int64_t n, const double* R, const uint8_t* act, const double* phi,
                            const double* phi_old, const uint8_t* flags, double* out, cudaStream_t s) {
  if (n > 0) k_newton_res<<<blocks_for(n), TPB, 0, s>>>(n, R, act, phi, phi_old, flags, out);
  return cudaGetLastError();
}

cudaError_t newton_rhs(int64_t n, const double* R, const double* t, const uint8_t* act, const double* phi,
                       const double* phi_old, const uint8_t* flags, double* rhs, cudaStream_t s) {
  if (n > 0) k_newton_rhs<<<blocks_for(n), TPB, 0, s>>>(n, R, t, act, phi, phi_old, flags, rhs);
  return cudaGetLastError();
}

cudaError_t newton_du0(int64_t n, const uint8_t* act, const double* phi, const double* phi_old, double* du0,
                       cudaStream_t s) {
  if (n > 0) k_du0<<<blocks_for(n), TPB, 0, s>>>(n, act, phi, phi_old, du0);
  return cudaGetLastError();
}

cudaError_t f64_to_f32(int64_t n, const double* a, float* b, cudaStream_t s) {
  if (n > 0) k_f64_to_f32<<<blocks_for(n), TPB, 0, s>>>(n, a, b);
  return cudaGetLastError();
}
cudaError_t f32_to_f64(int64_t n, const float* a, double* b, cudaStream_t s) {
  if (n > 0) k_f32_to_f64<<<blocks_for(n), TPB, 0, s>>>(n, a, b);
  return cudaGetLastError();
}

cudaError_t mask_fixed(int64_t n, const uint8_t* cmask, const double* x, double* out, cudaStream_t s) {
  if (n > 0) k_mask_fixed<<<blocks_for(n), TPB, 0, s>>>(n, cmask, x, out);
  return cudaGetLastError();
}

cudaError_t copy_fixed(int64_t n, const uint8_t* cmask, const double* x, double* out, cudaStream_t s) {
  if (n > 0) k_copy_fixed<<<blocks_for(n), TPB, 0, s>>>(n, cmask, x, out);
  return cudaGetLastError();
}

cudaError_t adj_carry(int64_t n, const uint8_t* act, const double* mu, const double* t1, const double* t2, double* g,
                      cudaStream_t s, const double* p1, const double* p2, const double* pend_in, double* pend_out) {
  if ((p1 == nullptr) != (p2 == nullptr)) return cudaErrorInvalidValue;
  if (n > 0) k_adj_carry<<<blocks_for(n), TPB, 0, s>>>(n, act, mu, t1, t2, p1, p2, pend_in, pend_out, g);
  return cudaGetLastError();
}

cudaError_t axpby(int64_t n, double* out, const double* x, double a, const double* y, double b, cudaStream_t s) {
  if (n > 0) k_axpby<<<blocks_for(n), TPB, 0, s>>>(n, out, x, a, y, b);
  return cudaGetLastError();
}


int reduction_partials() { return RED_BLOCKS; }

cudaError_t multidot(int64_t n, int k, const double* V, int64_t ldb, const double* w, double* partial, double* out,
                     cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_multidot_partial<<<RED_BLOCKS, TPB, 0, s>>>(n, k, V, ldb, w, partial);
  k_multidot_final<<<k, TPB, 0, s>>>(RED_BLOCKS, k, partial, out);
  return cudaGetLastError();
}

cudaError_t multi_axpy(int64_t n, int k, const double* V, int64_t ldb, const double* h, double sign, double* w,
                       cudaStream_t s, const int32_t* map) {
  if (k > MAX_BASIS) return cudaErrorInvalidValue;
  if (n > 0 && k > 0) k_multi_axpy<<<blocks_for(n), TPB, 0, s>>>(n, k, V, ldb, h, sign, w, map);
  return cudaGetLastError();
}

cudaError_t store_basis(int64_t n, double* V, int64_t ldb, int j, const double* x, double a, double* vc,
                        cudaStream_t s, const int32_t* map) {
  if (n > 0) k_store_basis<<<blocks_for(n), TPB, 0, s>>>(n, V, ldb, j, x, a, vc, map);
  return cudaGetLastError();
}

cudaError_t gather(int64_t n, const int32_t* map, const double* x, double* out, cudaStream_t s) {
  if (n > 0) k_gather<<<blocks_for(n), TPB, 0, s>>>(n, map, x, out);
  return cudaGetLastError();
}

cudaError_t extrapolate_phi(int64_t n, const double* p1, const double* p2, double* out, cudaStream_t s) {
  if (n > 0) k_extrapolate_phi<<<blocks_for(n), TPB, 0, s>>>(n, p1, p2, out);
  return cudaGetLastError();
}

cudaError_t vsum(int64_t n, const double* a, double* partial, double* out, cudaStream_t s) {
  k_sum_partial<<<RED_BLOCKS, TPB, 0, s>>>(n, a, partial);
  k_multidot_final<<<1, TPB, 0, s>>>(RED_BLOCKS, 1, partial, out);
  return cudaGetLastError();
}

cudaError_t all_finite(int64_t n, const double* a, int* bad, cudaStream_t s) {
  if (n > 0) k_all_finite<<<blocks_for(n), TPB, 0, s>>>(n, a, bad);
  return cudaGetLastError();
}

}  // namespace pff
