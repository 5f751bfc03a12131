// Multigrid kernels of libpff (see mg.cuh).  Level vectors of a block are
// stored per level as ncomp consecutive blocks of the level's slot count.
// Fixed rows (Dirichlet u for the u-block, active phi for the phi-block) and
// holes carry zeros; the inverse diagonal is zero off the interior, so the
// Chebyshev updates leave edge and fixed entries untouched.
#include "mg.cuh"

#include <algorithm>

#include "cheb.cuh"
#include "pdl.cuh"

namespace pff {

namespace {

constexpr int TPB = 256;

inline unsigned blocks_for(int64_t n) {
  int64_t b = (n + TPB - 1) / TPB;
  if (b > 65535 * 8) b = 65535 * 8;
  return unsigned(b < 1 ? 1 : b);
}

#define GRID_STRIDE(i, n) for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < (n); i += int64_t(gridDim.x) * blockDim.x)

constexpr int TB = 8;   // transfer-row entries whose loads are issued together

template <typename T>
__global__ void k_cheb_first(int64_t n, T* x, T* xprev, const T* dinv, const T* d, T c0) {
  pdl_trigger();
  pdl_wait();
  GRID_STRIDE(i, n) {
    x[i] = cheb_first_of(c0, dinv[i], d[i]);
    xprev[i] = T(0);
  }
}

template <typename T>
__global__ void k_cheb_step(int64_t n, T* xnew, const T* x, const T* xprev, const T* dinv, const T* d, const T* ax,
                            T a, T b) {
  pdl_trigger();
  pdl_wait();
  GRID_STRIDE(i, n) {
    xnew[i] = cheb_next(x[i], xprev[i], dinv[i], d[i], ax[i], a, b);
  }
}

template <typename T>
__global__ void k_restrict(int32_t nc, int ncomp, int64_t ncs, int64_t nfs, const int32_t* __restrict__ ptr,
                           const int32_t* __restrict__ col, const float* __restrict__ val, const T* __restrict__ df,
                           const T* __restrict__ axf, T* dc, const uint8_t* __restrict__ cmask_c, int fixbits,
                           const T* __restrict__ dinv_c, T* cur_c, T* prev_c, T c0) {
  pdl_trigger();
  pdl_wait();
  GRID_STRIDE(y, nc) {
    const uint8_t cm = cmask_c[y];
    const int e0 = ptr[y], e1 = ptr[y + 1];
    // ncomp is 1 or 2: the second sum is acc1
    T acc0 = dc[y], acc1 = ncomp > 1 ? dc[ncs + y] : T(0);
    // the row in batches of TB entries: indices and weights, then values, then the
    // sums in entry order (as one entry at a time)
    for (int eb = e0; eb < e1; eb += TB) {
      int z[TB];
      T w[TB];
#pragma unroll
      for (int q = 0; q < TB; ++q) {
        z[q] = eb + q < e1 ? col[eb + q] : 0;
        w[q] = eb + q < e1 ? T(val[eb + q]) : T(0);
      }
      for (int c = 0; c < ncomp; ++c) {
        T d[TB];
#pragma unroll
        for (int q = 0; q < TB; ++q) d[q] = eb + q < e1 ? df[c * nfs + z[q]] - axf[c * nfs + z[q]] : T(0);
        T a = c == 0 ? acc0 : acc1;
#pragma unroll
        for (int q = 0; q < TB; ++q)
          if (eb + q < e1) a += w[q] * d[q];
        if (c == 0) acc0 = a; else acc1 = a;
      }
    }
    for (int c = 0; c < ncomp; ++c) {
      const int bit = (fixbits == 4) ? 4 : (1 << c);
      const T v = (cm & bit) ? T(0) : (c == 0 ? acc0 : acc1);
      dc[c * ncs + y] = v;
      if (cur_c != nullptr) {
        cur_c[c * ncs + y] = cheb_first_of(c0, dinv_c[c * ncs + y], v);
        prev_c[c * ncs + y] = T(0);
      }
    }
  }
}

template <typename T>
__global__ void k_prolong(int32_t nf, int ncomp, int64_t nfs, int64_t ncs, const int32_t* __restrict__ ptr,
                          const int32_t* __restrict__ col, const float* __restrict__ val, const T* __restrict__ xc,
                          T* xf, const uint8_t* __restrict__ cmask_f, int fixbits) {
  pdl_trigger();
  pdl_wait();
  GRID_STRIDE(z, nf) {
    const uint8_t cm = cmask_f[z];
    const int e0 = ptr[z], e1 = ptr[z + 1];
    T acc0 = xf[z], acc1 = ncomp > 1 ? xf[nfs + z] : T(0);
    for (int eb = e0; eb < e1; eb += TB) {
      int yy[TB];
      T w[TB];
#pragma unroll
      for (int q = 0; q < TB; ++q) {
        yy[q] = eb + q < e1 ? col[eb + q] : 0;
        w[q] = eb + q < e1 ? T(val[eb + q]) : T(0);
      }
      for (int c = 0; c < ncomp; ++c) {
        T v[TB];
#pragma unroll
        for (int q = 0; q < TB; ++q) v[q] = eb + q < e1 ? xc[c * ncs + yy[q]] : T(0);
        T a = c == 0 ? acc0 : acc1;
#pragma unroll
        for (int q = 0; q < TB; ++q)
          if (eb + q < e1) a += w[q] * v[q];
        if (c == 0) acc0 = a; else acc1 = a;
      }
    }
    for (int c = 0; c < ncomp; ++c) {
      const int bit = (fixbits == 4) ? 4 : (1 << c);
      xf[c * nfs + z] = (cm & bit) ? T(0) : (c == 0 ? acc0 : acc1);
    }
  }
}

template <typename T>
__global__ void k_copy_in(int64_t nsl, int ncomp, DevHome home, const double* __restrict__ r, T* d,
                          const uint8_t* __restrict__ lcm, int fixbits) {
  GRID_STRIDE(s, nsl) {
    const int32_t b = home.slot[s];
    if (b < 0) continue;
    const int64_t base = int64_t(ncomp) * home.off[s] + b, nl = home.nsl[s];
    const uint8_t cm = lcm[s];
    for (int c = 0; c < ncomp; ++c) {
      const int bit = (fixbits == 4) ? 4 : (1 << c);
      if (!(cm & bit)) d[base + c * nl] = T(r[c * nsl + s]);
    }
  }
}

template <typename T>
__global__ void k_copy_out(int64_t nsl, int ncomp, DevHome home, const T* __restrict__ x,
                           const double* __restrict__ r, double* z, const uint8_t* __restrict__ lcm,
                           const uint8_t* __restrict__ lflags, int fixbits) {
  pdl_trigger();
  pdl_wait();
  GRID_STRIDE(s, nsl) {
    const uint8_t cm = lcm[s];
    const bool node = (lflags[s] & 1) && !(lflags[s] & 4);
    const int32_t b = home.slot[s];
    const int64_t base = b >= 0 ? int64_t(ncomp) * home.off[s] + b : 0, nl = b >= 0 ? home.nsl[s] : 0;
    for (int c = 0; c < ncomp; ++c) {
      const int bit = (fixbits == 4) ? 4 : (1 << c);
      double v = 0.0;
      if (cm & bit) v = node ? r[c * nsl + s] : 0.0;
      else if (b >= 0) v = double(x[base + c * nl]);
      z[c * nsl + s] = v;
    }
  }
}

template <typename T>
__global__ void k_cheb_first_res(int64_t n, T* x, T* xprev, T* r, const T* __restrict__ dinv,
                                 const T* __restrict__ d, const T* __restrict__ ax, T c0, T* xadd) {
  pdl_trigger();
  pdl_wait();
  GRID_STRIDE(i, n) {
    const T ri = d[i] - ax[i];
    const T v = cheb_first_of(c0, dinv[i], ri);
    if (xadd != nullptr) {
      xadd[i] += v;
    } else {
      r[i] = ri;
      x[i] = v;
      xprev[i] = T(0);
    }
  }
}

template <typename T>
__global__ void k_cheb_step_add(int64_t n, T* xadd, const T* __restrict__ x, const T* __restrict__ xprev,
                                const T* __restrict__ dinv, const T* __restrict__ d, const T* __restrict__ ax, T a,
                                T b) {
  pdl_trigger();
  pdl_wait();
  GRID_STRIDE(i, n) {
    xadd[i] += cheb_next(x[i], xprev[i], dinv[i], d[i], ax[i], a, b);
  }
}

// Dense FP64 coarse solve: tmp = d[idx] (to FP64), x[idx] = Ainv tmp; one block per row group.
template <typename T>
__global__ void k_coarse_gather(int32_t n, const int32_t* idx, const T* d, double* tmp) {
  pdl_trigger();
  pdl_wait();
  GRID_STRIDE(i, n) tmp[i] = double(d[idx[i]]);
}

// Blocked Gauss-Jordan inversion in place, panels of GJB pivots.  With P the
// panel's rows/columns and R the others, eliminating the pivots of P gives
//   A_PP <- X = A_PP^-1,  A_PR <- X A_PR,  A_RP <- -A_RP X,  A_RR <- A_RR - A_RP X A_PR
// (old A_RP, A_PR on the right), the same as GJB scalar Gauss-Jordan steps.  A_PP
// is then a Schur complement of an SPD matrix, so no pivoting is needed; its
// inversion (one block, scalar steps in shared memory) flags a non-positive pivot.
// Two launches per panel: k_gj_panel inverts A_PP and copies the old A_RP and
// A_PR to scratch; k_gj_update then owns every entry it writes, so no block reads
// an entry another block of the same launch writes.
// Scratch layout (double): X (GJB x GJB, zero beyond b), then Cp ((n - b) x GJB:
// old A_RP by compact row index, zero beyond b), then Rp (GJB x n: old A_PR, zero
// in the panel's columns and beyond b).
constexpr int GJB = 32;
constexpr int GJ_ROWS = 128;   // rows of a k_gj_update tile (its columns: GJB)

__device__ __forceinline__ int gj_row(int ii, int k0, int b) { return ii < k0 ? ii : ii + b; }

// block 0: X = A_PP^-1 (padded with the identity to GJB x GJB); the others copy
// the old pivot columns and rows
__global__ void __launch_bounds__(TPB) k_gj_panel(int32_t n, int32_t k0, int32_t b, double* A, double* scr,
                                                  int32_t* bad) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (blockIdx.x == 0) {
    // one reciprocal per step: the thread that writes the next pivot inverts it
    __shared__ double T[GJB][GJB + 1];
    __shared__ double ipiv[2];
#pragma unroll
    for (int r = 0; r < GJB / 8; ++r) {
      const int i = w + 8 * r;
      T[i][lane] = (i < b && lane < b) ? A[int64_t(k0 + i) * n + k0 + lane] : (i == lane ? 1.0 : 0.0);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (!(T[0][0] > 0.0)) *bad = 1;
      ipiv[0] = 1.0 / T[0][0];
    }
    __syncthreads();
    for (int k = 0; k < GJB; ++k) {
      const double ip = ipiv[k & 1];
      const double sk = T[k][lane] * ip;   // row k scaled by the pivot's reciprocal
      double v[GJB / 8];
#pragma unroll
      for (int r = 0; r < GJB / 8; ++r) {
        const int i = w + 8 * r;
        const double pc = T[i][k];
        if (i == k) v[r] = lane == k ? ip : sk;
        else if (lane == k) v[r] = -pc * ip;
        else v[r] = fma(-pc, sk, T[i][lane]);
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < GJB / 8; ++r) {
        const int i = w + 8 * r;
        T[i][lane] = v[r];
        if (i == k + 1 && lane == k + 1) {
          if (!(v[r] > 0.0)) *bad = 1;
          ipiv[(k + 1) & 1] = 1.0 / v[r];
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < GJB / 8; ++r) {
      const int i = w + 8 * r;
      const bool in = i < b && lane < b;
      scr[i * GJB + lane] = in ? T[i][lane] : 0.0;
      if (in) A[int64_t(k0 + i) * n + k0 + lane] = T[i][lane];
    }
    return;
  }
  double* Cp = scr + GJB * GJB;
  double* Rp = Cp + int64_t(n - b) * GJB;
  const int64_t nc = int64_t(n - b) * GJB, nr = int64_t(GJB) * n;
  const int64_t stride = int64_t(gridDim.x - 1) * blockDim.x;
  for (int64_t e = int64_t(blockIdx.x - 1) * blockDim.x + threadIdx.x; e < nc + nr; e += stride) {
    if (e < nc) {
      const int ii = int(e / GJB), k = int(e % GJB);
      Cp[e] = k < b ? A[int64_t(gj_row(ii, k0, b)) * n + k0 + k] : 0.0;
    } else {
      const int64_t f = e - nc;
      const int k = int(f / n), j = int(f % n);
      Rp[f] = (k < b && (j < k0 || j >= k0 + b)) ? A[int64_t(k0 + k) * n + j] : 0.0;
    }
  }
}

// tile (GJ_ROWS rows outside P) x (GJB columns): the panel's columns get
// -A_RP X; any other column tile forms X A_PR for its columns (written back by
// the first row tile) and subtracts A_RP (X A_PR) from its rows
__global__ void __launch_bounds__(TPB) k_gj_update(int32_t n, int32_t k0, int32_t b, double* A,
                                                   const double* scr) {
  __shared__ double Xs[GJB][GJB];
  __shared__ double Ps[GJB][GJB];       // old A_PR tile, then X A_PR
  __shared__ double Cs[GJ_ROWS][GJB];   // old A_RP rows of the tile
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double* Cp = scr + GJB * GJB;
  const double* Rp = Cp + int64_t(n - b) * GJB;
  const int ii0 = int(blockIdx.y) * GJ_ROWS;
  const int nrow = min(GJ_ROWS, n - b - ii0);
  const int j0 = int(blockIdx.x) * GJB;
  const int j = j0 + lane;
  const bool panel = j0 == k0;
#pragma unroll
  for (int r = 0; r < GJB / 8; ++r) Xs[w + 8 * r][lane] = scr[(w + 8 * r) * GJB + lane];
  for (int r = w; r < GJ_ROWS; r += TPB / 32) Cs[r][lane] = r < nrow ? Cp[int64_t(ii0 + r) * GJB + lane] : 0.0;
  if (!panel) {
#pragma unroll
    for (int r = 0; r < GJB / 8; ++r) Ps[w + 8 * r][lane] = j < n ? Rp[int64_t(w + 8 * r) * n + j] : 0.0;
  }
  __syncthreads();
  if (panel) {
    // A_RP <- -A_RP X
    for (int r = w; r < nrow; r += TPB / 32) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < GJB; ++k) acc = fma(Cs[r][k], Xs[k][lane], acc);
      if (lane < b) A[int64_t(gj_row(ii0 + r, k0, b)) * n + j] = -acc;
    }
    return;
  }
  double pr[GJB / 8];
#pragma unroll
  for (int r = 0; r < GJB / 8; ++r) {
    const int k = w + 8 * r;
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < GJB; ++m) acc = fma(Xs[k][m], Ps[m][lane], acc);
    pr[r] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < GJB / 8; ++r) {
    const int k = w + 8 * r;
    Ps[k][lane] = pr[r];
    if (blockIdx.y == 0 && k < b && j < n) A[int64_t(k0 + k) * n + j] = pr[r];
  }
  __syncthreads();
  if (j >= n) return;
  double pc[GJB];
#pragma unroll
  for (int k = 0; k < GJB; ++k) pc[k] = Ps[k][lane];
  for (int r = w; r < nrow; r += TPB / 32) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < GJB; ++k) acc = fma(Cs[r][k], pc[k], acc);
    double* a = A + int64_t(gj_row(ii0 + r, k0, b)) * n + j;
    *a = *a - acc;
  }
}

template <typename T>
__global__ void k_coarse_matvec(int32_t n, const int32_t* idx, const double* __restrict__ A,
                                const double* __restrict__ tmp, T* x) {
  pdl_trigger();
  pdl_wait();
  // one warp per row, lanes stride the columns, fixed-order warp reduction
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  double acc = 0.0;
  for (int j = lane; j < n; j += 32) acc += A[int64_t(warp) * n + j] * tmp[j];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) x[idx[warp]] = T(acc);
}

__global__ void k_inject_lin(int32_t nsl, const int32_t* __restrict__ sl, const double* __restrict__ lin,
                             int64_t nsleaf, double* l64, float* l32) {
  GRID_STRIDE(s, nsl) {
    const int ls = sl[s];
    for (int f = 0; f < 4; ++f) {
      const double v = ls >= 0 ? lin[f * nsleaf + ls] : 0.0;
      l64[f * int64_t(nsl) + s] = v;
      l32[f * int64_t(nsl) + s] = float(v);
    }
  }
}

__global__ void k_level_cmask(int32_t nsl, const uint8_t* __restrict__ flags, const int32_t* __restrict__ sl,
                              const uint8_t* __restrict__ lcm, const int32_t* __restrict__ Rp,
                              const int32_t* __restrict__ Rc, const uint8_t* __restrict__ cmf, uint8_t* cm) {
  GRID_STRIDE(s, nsl) {
    const uint8_t f = flags[s];
    uint8_t c = 0;
    if ((f & 1) && (f & 2)) c |= 3;
    if (f & 1) {
      const int ls = sl[s];
      bool act = ls >= 0 && (lcm[ls] & 4);
      if (!act && Rp != nullptr && !(f & 16)) {
        for (int e = Rp[s]; e < Rp[s + 1]; ++e)
          if (cmf[Rc[e]] & 4) { act = true; break; }
      }
      if (act) c |= 4;
    }
    cm[s] = c;
  }
}

__global__ void k_invert_diag(int32_t nsl, int ncomp, const double* __restrict__ diag,
                              const uint8_t* __restrict__ flags, const uint8_t* __restrict__ cm, int fixbits,
                              double* d64, float* d32) {
  GRID_STRIDE(s, nsl) {
    const uint8_t f = flags[s];
    for (int c = 0; c < ncomp; ++c) {
      const int bit = (fixbits == 4) ? 4 : (1 << c);
      const int64_t i = c * int64_t(nsl) + s;
      const double dg = diag[i];
      const bool interior = (f & 1) && !(f & 8) && !(cm[s] & bit) && dg != 0.0;
      const double v = interior ? 1.0 / dg : 0.0;
      d64[i] = v;
      d32[i] = float(v);
    }
  }
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_start_vector(int32_t nsl, int ncomp, const int32_t* __restrict__ gx, const int32_t* __restrict__ gy,
                               const double* __restrict__ dinv, double* r) {
  GRID_STRIDE(s, nsl) {
    double v = 0.0;
    if (gx[s] >= 0) {
      const uint64_t h = splitmix64((uint64_t(uint32_t(gx[s])) << 32) | uint64_t(uint32_t(gy[s])));
      v = 1.0 + 0.01 * double(h % 1000ull) / 1000.0;
    }
    for (int c = 0; c < ncomp; ++c) {
      const int64_t i = c * int64_t(nsl) + s;
      r[i] = dinv[i] != 0.0 ? v : 0.0;
    }
  }
}

constexpr int DOT_BLOCKS = 512;

__global__ void k_dot_partial(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* part) {
  __shared__ double sh[TPB];
  double acc = 0.0;
  GRID_STRIDE(i, n) acc += a[i] * b[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = TPB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_dot_final(int nb, const double* __restrict__ part, double* out) {
  __shared__ double sh[TPB];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += TPB) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = TPB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

// sc: 0 rz, 1 pq, 2 rz_new, 3 alpha, 4 beta, 5 ok (1 while the iteration is healthy)
__global__ void k_cg_init(double* sc) {
  if (threadIdx.x < 8) sc[threadIdx.x] = threadIdx.x == 5 ? 1.0 : 0.0;
}

// r -= alpha q, z = D^-1 r and the block partial sums of r.z (the grid and the
// summation order of k_dot_partial, so the dot is the same as a separate one)
__global__ void k_cg_r_dot(int64_t n, double* r, double* z, const double* __restrict__ q,
                           const double* __restrict__ dinv, const double* __restrict__ sc, double* part) {
  __shared__ double sh[TPB];
  const double alpha = sc[3];
  double acc = 0.0;
  GRID_STRIDE(i, n) {
    const double ri = r[i] - alpha * q[i];
    const double zi = dinv[i] * ri;
    r[i] = ri;
    z[i] = zi;
    acc += ri * zi;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = TPB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// sc[slot] = sum of the partials (the order of k_dot_final), then slot 1: alpha =
// rz / pq; slot 2: beta = rz_new / rz, the coefficient history (alpha_j, beta_j;
// alpha_j = 0 marks a stop) and rz = rz_new.  sc[5] drops to 0 on a breakdown.
__global__ void k_dot_final_cg(int nb, const double* __restrict__ part, double* sc, int slot, double* hist,
                               int step) {
  __shared__ double sh[TPB];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += TPB) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = TPB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  sc[slot] = sh[0];
  if (slot == 1) {
    const double pq = sc[1];
    const bool ok = sc[5] > 0.5 && pq > 0.0 && sc[0] > 0.0;
    sc[3] = ok ? sc[0] / pq : 0.0;
    if (!ok) sc[5] = 0.0;
  } else if (slot == 2) {
    const bool ok = sc[5] > 0.5;
    const double beta = ok ? sc[2] / sc[0] : 0.0;
    sc[4] = beta;
    hist[2 * step + 0] = ok ? sc[3] : 0.0;
    hist[2 * step + 1] = beta;
    if (!(ok && sc[2] > 1e-300)) sc[5] = 0.0;
    sc[0] = sc[2];
  }
}

__global__ void k_cg_p(int64_t n, double* p, const double* __restrict__ z, const double* __restrict__ sc) {
  const double beta = sc[4];
  GRID_STRIDE(i, n) p[i] = z[i] + beta * p[i];
}

__global__ void k_fill64(int64_t n, double* x, double v) { GRID_STRIDE(i, n) x[i] = v; }
__global__ void k_copy64(int64_t n, double* d, const double* s) { GRID_STRIDE(i, n) d[i] = s[i]; }

}  // namespace

template <typename T>
cudaError_t mg_chebyshev_first(int64_t n, T* x, T* xprev, const T* dinv, const T* d, T c0, cudaStream_t s, bool pdl) {
  if (n > 0) return launch_ex(pdl, &k_cheb_first<T>, blocks_for(n), TPB, 0, s, n, x, xprev, dinv, d, c0);
  return cudaGetLastError();
}
template <typename T>
cudaError_t mg_chebyshev_step(int64_t n, T* xnew, const T* x, const T* xprev, const T* dinv, const T* d,
                              const T* ax, T a, T b, cudaStream_t s, bool pdl) {
  if (n > 0) return launch_ex(pdl, &k_cheb_step<T>, blocks_for(n), TPB, 0, s, n, xnew, x, xprev, dinv, d, ax, a, b);
  return cudaGetLastError();
}
template <typename T>
cudaError_t mg_restrict(int32_t nc, int ncomp, int64_t ncs, int64_t nfs, const int32_t* ptr, const int32_t* col,
                        const float* val, const T* d_f, const T* ax_f, T* d_c, const uint8_t* cmask_c, int fixbits,
                        cudaStream_t s, bool pdl, const T* dinv_c, T* cur_c, T* prev_c, T c0) {
  if (nc > 0)
    return launch_ex(pdl, &k_restrict<T>, blocks_for(nc), TPB, 0, s, nc, ncomp, ncs, nfs, ptr, col, val, d_f, ax_f,
                     d_c, cmask_c, fixbits, dinv_c, cur_c, prev_c, c0);
  return cudaGetLastError();
}
template <typename T>
cudaError_t mg_prolong(int32_t nf, int ncomp, int64_t nfs, int64_t ncs, const int32_t* ptr, const int32_t* col,
                       const float* val, const T* x_c, T* x_f, const uint8_t* cmask_f, int fixbits, cudaStream_t s,
                       bool pdl) {
  if (nf > 0)
    return launch_ex(pdl, &k_prolong<T>, blocks_for(nf), TPB, 0, s, nf, ncomp, nfs, ncs, ptr, col, val, x_c, x_f,
                     cmask_f, fixbits);
  return cudaGetLastError();
}
template <typename T>
cudaError_t mg_copy_in(int64_t ns_leaf, int ncomp, DevHome home, const double* r, T* d, const uint8_t* leaf_cmask,
                       int fixbits, cudaStream_t s) {
  if (ns_leaf > 0) k_copy_in<T><<<blocks_for(ns_leaf), TPB, 0, s>>>(ns_leaf, ncomp, home, r, d, leaf_cmask, fixbits);
  return cudaGetLastError();
}
template <typename T>
cudaError_t mg_copy_out(int64_t ns_leaf, int ncomp, DevHome home, const T* x, const double* r, double* z,
                        const uint8_t* leaf_cmask, const uint8_t* leaf_flags, int fixbits, cudaStream_t s, bool pdl) {
  if (ns_leaf > 0)
    return launch_ex(pdl, &k_copy_out<T>, blocks_for(ns_leaf), TPB, 0, s, ns_leaf, ncomp, home, x, r, z, leaf_cmask,
                     leaf_flags, fixbits);
  return cudaGetLastError();
}
template <typename T>
cudaError_t mg_chebyshev_first_res(int64_t n, T* x, T* xprev, T* r, const T* dinv, const T* d, const T* ax, T c0,
                                   T* xadd, cudaStream_t s, bool pdl) {
  if (n > 0)
    return launch_ex(pdl, &k_cheb_first_res<T>, blocks_for(n), TPB, 0, s, n, x, xprev, r, dinv, d, ax, c0, xadd);
  return cudaGetLastError();
}
template <typename T>
cudaError_t mg_chebyshev_step_add(int64_t n, T* xadd, const T* x, const T* xprev, const T* dinv, const T* d,
                                  const T* ax, T a, T b, cudaStream_t s, bool pdl) {
  if (n > 0)
    return launch_ex(pdl, &k_cheb_step_add<T>, blocks_for(n), TPB, 0, s, n, xadd, x, xprev, dinv, d, ax, a, b);
  return cudaGetLastError();
}
int64_t mg_spd_scratch(int32_t cap) { return int64_t(GJB) * GJB + 2 * int64_t(GJB) * cap; }

cudaError_t mg_spd_invert(int32_t n, double* A, double* scr, int32_t* bad, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int32_t), s);
  if (e != cudaSuccess || n <= 0) return e;
  for (int32_t k0 = 0; k0 < n; k0 += GJB) {
    const int32_t b = n - k0 < GJB ? n - k0 : GJB;
    const int64_t copies = int64_t(n - b) * GJB + int64_t(GJB) * n;
    const unsigned cb = n > b ? unsigned(std::min<int64_t>((copies + TPB - 1) / TPB, 64)) : 0u;
    k_gj_panel<<<1 + cb, TPB, 0, s>>>(n, k0, b, A, scr, bad);
    if (n > b) {
      const dim3 grid(unsigned((n + GJB - 1) / GJB), unsigned((n - b + GJ_ROWS - 1) / GJ_ROWS));
      k_gj_update<<<grid, TPB, 0, s>>>(n, k0, b, A, scr);
    }
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t mg_coarse(int32_t n, const int32_t* idx, const double* Ainv, const T* d, T* x, double* tmp,
                      cudaStream_t s, bool pdl) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = launch_ex(pdl, &k_coarse_gather<T>, blocks_for(n), TPB, 0, s, n, idx, d, tmp);
  if (e != cudaSuccess) return e;
  const int warps_per_block = TPB / 32;
  return launch_ex(pdl, &k_coarse_matvec<T>, unsigned((n + warps_per_block - 1) / warps_per_block), TPB, 0, s, n, idx,
                   Ainv, static_cast<const double*>(tmp), x);
}

cudaError_t mg_inject_lin(int32_t ns_l, const int32_t* slot_leaf, const double* lin64, int64_t ns_leaf,
                          double* lev64, float* lev32, cudaStream_t s) {
  if (ns_l > 0) k_inject_lin<<<blocks_for(ns_l), TPB, 0, s>>>(ns_l, slot_leaf, lin64, ns_leaf, lev64, lev32);
  return cudaGetLastError();
}
cudaError_t mg_level_cmask(int32_t ns_l, const uint8_t* flags, const int32_t* slot_leaf, const uint8_t* leaf_cmask,
                           const int32_t* R_ptr, const int32_t* R_col, const uint8_t* cmask_fine, uint8_t* cmask,
                           cudaStream_t s) {
  if (ns_l > 0) k_level_cmask<<<blocks_for(ns_l), TPB, 0, s>>>(ns_l, flags, slot_leaf, leaf_cmask, R_ptr, R_col,
                                                                cmask_fine, cmask);
  return cudaGetLastError();
}
cudaError_t mg_invert_diag(int32_t ns_l, int ncomp, const double* diag, const uint8_t* flags, const uint8_t* cmask,
                           int fixbits, double* dinv64, float* dinv32, cudaStream_t s) {
  if (ns_l > 0) k_invert_diag<<<blocks_for(ns_l), TPB, 0, s>>>(ns_l, ncomp, diag, flags, cmask, fixbits, dinv64,
                                                                dinv32);
  return cudaGetLastError();
}
cudaError_t mg_start_vector(int32_t ns_l, int ncomp, const int32_t* gx, const int32_t* gy, const double* dinv,
                            double* r, cudaStream_t s) {
  if (ns_l > 0) k_start_vector<<<blocks_for(ns_l), TPB, 0, s>>>(ns_l, ncomp, gx, gy, dinv, r);
  return cudaGetLastError();
}
cudaError_t dot64(int64_t n, const double* a, const double* b, double* partial, double* out, cudaStream_t s) {
  k_dot_partial<<<DOT_BLOCKS, TPB, 0, s>>>(n, a, b, partial);
  k_dot_final<<<1, TPB, 0, s>>>(DOT_BLOCKS, partial, out);
  return cudaGetLastError();
}
cudaError_t cg_update_p(int64_t n, double* p, const double* z, const double* sc, cudaStream_t s) {
  if (n > 0) k_cg_p<<<blocks_for(n), TPB, 0, s>>>(n, p, z, sc);
  return cudaGetLastError();
}
cudaError_t dot_partial64(int64_t n, const double* a, const double* b, double* partial, cudaStream_t s) {
  k_dot_partial<<<DOT_BLOCKS, TPB, 0, s>>>(n, a, b, partial);
  return cudaGetLastError();
}
cudaError_t cg_dot_final(const double* partial, double* sc, int slot, double* hist, int step, cudaStream_t s) {
  k_dot_final_cg<<<1, TPB, 0, s>>>(DOT_BLOCKS, partial, sc, slot, hist, step);
  return cudaGetLastError();
}
cudaError_t cg_update_r_dot(int64_t n, double* r, double* z, const double* q, const double* dinv, const double* sc,
                            double* partial, cudaStream_t s) {
  k_cg_r_dot<<<DOT_BLOCKS, TPB, 0, s>>>(n, r, z, q, dinv, sc, partial);
  return cudaGetLastError();
}
cudaError_t cg_init_scalars(double* sc, cudaStream_t s) {
  k_cg_init<<<1, 32, 0, s>>>(sc);
  return cudaGetLastError();
}
int mg_dot_partials() { return DOT_BLOCKS; }
cudaError_t fill64(int64_t n, double* x, double v, cudaStream_t s) {
  if (n > 0) k_fill64<<<blocks_for(n), TPB, 0, s>>>(n, x, v);
  return cudaGetLastError();
}
cudaError_t copy64(int64_t n, double* dst, const double* src, cudaStream_t s) {
  if (n > 0) k_copy64<<<blocks_for(n), TPB, 0, s>>>(n, dst, src);
  return cudaGetLastError();
}

#define INST(T)                                                                                                \
  template cudaError_t mg_chebyshev_first<T>(int64_t, T*, T*, const T*, const T*, T, cudaStream_t, bool);     \
  template cudaError_t mg_chebyshev_step<T>(int64_t, T*, const T*, const T*, const T*, const T*, const T*, T,  \
                                            T, cudaStream_t, bool);                                            \
  template cudaError_t mg_restrict<T>(int32_t, int, int64_t, int64_t, const int32_t*, const int32_t*,          \
                                      const float*, const T*, const T*, T*, const uint8_t*, int, cudaStream_t, \
                                      bool, const T*, T*, T*, T);                                              \
  template cudaError_t mg_prolong<T>(int32_t, int, int64_t, int64_t, const int32_t*, const int32_t*,           \
                                     const float*, const T*, T*, const uint8_t*, int, cudaStream_t, bool);     \
  template cudaError_t mg_copy_in<T>(int64_t, int, DevHome, const double*, T*, const uint8_t*, int, cudaStream_t); \
  template cudaError_t mg_copy_out<T>(int64_t, int, DevHome, const T*, const double*, double*, const uint8_t*,     \
                                      const uint8_t*, int, cudaStream_t, bool);                                    \
  template cudaError_t mg_chebyshev_first_res<T>(int64_t, T*, T*, T*, const T*, const T*, const T*, T, T*,        \
                                                 cudaStream_t, bool);                                              \
  template cudaError_t mg_chebyshev_step_add<T>(int64_t, T*, const T*, const T*, const T*, const T*, const T*, T, \
                                                T, cudaStream_t, bool);                                            \
  template cudaError_t mg_coarse<T>(int32_t, const int32_t*, const double*, const T*, T*, double*, cudaStream_t, bool);
INST(float)
INST(double)
#undef INST

}  // namespace pff
