// Matrix-free Jacobian and level-block operators on the brick layout, Q1 elements.
//
// Operator (Kolditz & Wick, arXiv 2404.03265, Sec. 3.1, Jacobian A'(U)):
//   (g(phi~) sigma(du), e(psi_u))
// + (1-kappa)(dphi sigma(u):e(u) + 2 phi sigma(du):e(u), psi_phi)
// + 2 p (dphi div u + phi div du, psi_phi)
// + G_c ((1/l)(dphi, psi_phi) + l (grad dphi, grad psi_phi)),
// g(phi) = (1-kappa) phi^2 + kappa (Problem 1), sigma = 2 mu e + lambda tr(e) I.
// The u-rows do not see dphi (block lower triangular, Sec. 3.2); the diagonal
// blocks are the multigrid level operators (Sec. 3.2).
//
// One CTA of 256 threads per brick of 15x15 owned node slots:
//   1. gather the 17x17 node window (input x with hanging-node constraints
//      resolved on the fly and fixed components masked; linearisation) into
//      shared memory;
//   2. one thread per cell of the 16x16 cell window: sum-factorised 2x2 Gauss
//      evaluation and test, 12 (or fewer) nodal contributions to shared memory;
//   3. one thread per owned node sums its four cells in a fixed order and
//      writes its output once.  Nodes shared with another level, hanging nodes
//      and their parents write partial sums; a small fix-up kernel condenses
//      them (x_full = C x on input, C^T y on output).
// No atomics: every output is produced by exactly one thread in a fixed order.
#include "kernels.cuh"

namespace pff {

namespace {

template <typename T> struct VT;
template <> struct VT<float> { using T2 = float2; using T4 = float4; };
template <> struct VT<double> { using T2 = double2; using T4 = dbl4; };

constexpr int NB = 15;          // owned node slots per brick side
constexpr int WN = 17;          // window nodes per side
constexpr int WC = 16;          // window cells per side
constexpr int NWIN = WN * WN;   // 289
constexpr int NCELL = WC * WC;  // 256
constexpr int NOWN = NB * NB;   // 225
constexpr int NTHREADS = 256;

// 2-point Gauss rule on [0, 1]
constexpr double GA = 0.21132486540518711775;
constexpr double GB = 0.78867513459481288225;

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

__device__ __forceinline__ dbl4 ldg4(const dbl4* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = __ldg(q), b = __ldg(q + 1);
  dbl4 r;
  r.x = a.x; r.y = a.y; r.z = b.x; r.w = b.y;
  return r;
}
__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }

// Reference-cell helpers for one Q1 field with nodal values v0..v3 at
// (0,0), (1,0), (0,1), (1,1): dxi[q2] = dv/dxi at eta = g_q2,
// deta[q1] = dv/deta at xi = g_q1, val[q1][q2].
template <typename T>
struct Q1Field {
  T dxi[2], deta[2];
  __device__ __forceinline__ void grads(T v0, T v1, T v2, T v3) {
    const T dx0 = v1 - v0, dx1 = v3 - v2, dy0 = v2 - v0;
    const T x = dx1 - dx0;
    dxi[0] = dx0 + T(GA) * x;
    dxi[1] = dx0 + T(GB) * x;
    deta[0] = dy0 + T(GA) * x;
    deta[1] = dy0 + T(GB) * x;
  }
};

template <typename T>
__device__ __forceinline__ void q1_values(T v0, T v1, T v2, T v3, T val[2][2]) {
  const T dx0 = v1 - v0, dy0 = v2 - v0;
  const T x = (v3 - v2) - dx0;
  const T de0 = dy0 + T(GA) * x, de1 = dy0 + T(GB) * x;
  const T vb0 = v0 + T(GA) * dx0, vb1 = v0 + T(GB) * dx0;
  val[0][0] = vb0 + T(GA) * de0;
  val[0][1] = vb0 + T(GB) * de0;
  val[1][0] = vb1 + T(GA) * de1;
  val[1][1] = vb1 + T(GB) * de1;
}

// Test of a gradient flux: given per-qp reference fluxes fx (coefficient of
// dN/dxi) and fy (coefficient of dN/deta), accumulate
// sum_q fx dN_A/dxi + fy dN_A/deta into r[0..3] (weights wx, wy).
template <typename T>
__device__ __forceinline__ void q1_test_grad(const T fx[2][2], const T fy[2][2], T wx, T wy, T r[4]) {
  // dN/dxi at eta: N0: -(1-eta), N1: (1-eta), N2: -eta, N3: eta
  const T sx0 = fx[0][0] + fx[1][0], sx1 = fx[0][1] + fx[1][1];   // sums over q1 per q2
  const T px = T(GA) * sx0 + T(GB) * sx1;                         // weight eta
  const T qx = (sx0 + sx1) - px;                                  // weight (1-eta)
  // dN/deta at xi: N0: -(1-xi), N1: -xi, N2: (1-xi), N3: xi
  const T sy0 = fy[0][0] + fy[0][1], sy1 = fy[1][0] + fy[1][1];   // sums over q2 per q1
  const T py = T(GA) * sy0 + T(GB) * sy1;
  const T qy = (sy0 + sy1) - py;
  r[0] += -wx * qx - wy * qy;
  r[1] += wx * qx - wy * py;
  r[2] += -wx * px + wy * qy;
  r[3] += wx * px + wy * py;
}

// Test of a value flux fv[q1][q2] against N_A, weight w.
template <typename T>
__device__ __forceinline__ void q1_test_val(const T fv[2][2], T w, T r[4]) {
  const T s0 = fv[0][0] + fv[0][1], s1 = fv[1][0] + fv[1][1];
  const T t0 = T(GA) * fv[0][0] + T(GB) * fv[0][1];   // eta-weighted, per q1
  const T t1 = T(GA) * fv[1][0] + T(GB) * fv[1][1];
  const T b0 = s0 - t0, b1 = s1 - t1;                 // (1-eta)-weighted
  const T pb = T(GA) * b0 + T(GB) * b1, pt = T(GA) * t0 + T(GB) * t1;
  r[0] += w * ((b0 + b1) - pb);
  r[1] += w * pb;
  r[2] += w * ((t0 + t1) - pt);
  r[3] += w * pt;
}

// One Q1 cell.  Window node indices n0 (0,0), n0+1, n0+WN, n0+WN+1.
// out[3*A + c] (c: 0 u_x, 1 u_y, 2 phi) for OP_FULL/OP_FULL_T; for OP_UU the
// first two components, for OP_PP only component 2 is meaningful.
template <typename T, int OP>
__device__ __forceinline__ void q1_cell(const T* __restrict__ s0, const T* __restrict__ s1,
                                        const T* __restrict__ sp, const typename VT<T>::T4* __restrict__ sl,
                                        int n0, const CellConst<T>& c, T out[12]) {
  const int nd[4] = {n0, n0 + 1, n0 + WN, n0 + WN + 1};
  T rux[4] = {0, 0, 0, 0}, ruy[4] = {0, 0, 0, 0}, rp[4] = {0, 0, 0, 0};
  constexpr bool needU = (OP == OP_FULL || OP == OP_FULL_T || OP == OP_UU || OP == OP_UU_DIAG);
  constexpr bool needP = (OP == OP_FULL || OP == OP_FULL_T || OP == OP_PP || OP == OP_PP_DIAG);
  constexpr bool needLinU = (OP == OP_FULL || OP == OP_FULL_T || OP == OP_PP || OP == OP_PP_DIAG);
  constexpr bool needG = (OP == OP_FULL || OP == OP_FULL_T || OP == OP_UU || OP == OP_UU_DIAG);
  constexpr bool needPhi = (OP == OP_FULL || OP == OP_FULL_T);
  typename VT<T>::T4 L[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) L[a] = sl[nd[a]];
  // ---- linearisation at the Gauss points
  Q1Field<T> fux, fuy;
  T phiq[2][2], phitq[2][2];
  if (needLinU) {
    fux.grads(L[0].x, L[1].x, L[2].x, L[3].x);
    fuy.grads(L[0].y, L[1].y, L[2].y, L[3].y);
  }
  if (needPhi) q1_values(L[0].z, L[1].z, L[2].z, L[3].z, phiq);
  if (needG) q1_values(L[0].w, L[1].w, L[2].w, L[3].w, phitq);
  // ---- input
  Q1Field<T> fxu, fxv, fxp;
  T xpq[2][2];
  if (OP == OP_FULL || OP == OP_FULL_T || OP == OP_UU) {
    fxu.grads(s0[nd[0]], s0[nd[1]], s0[nd[2]], s0[nd[3]]);
    fxv.grads(s1[nd[0]], s1[nd[1]], s1[nd[2]], s1[nd[3]]);
  }
  if (OP == OP_FULL || OP == OP_FULL_T || OP == OP_PP) {
    const T v0 = sp[nd[0]], v1 = sp[nd[1]], v2 = sp[nd[2]], v3 = sp[nd[3]];
    fxp.grads(v0, v1, v2, v3);
    q1_values(v0, v1, v2, v3, xpq);
  }
  T fux_x[2][2], fux_y[2][2], fuy_x[2][2], fuy_y[2][2], fv[2][2];
#pragma unroll
  for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
    for (int q2 = 0; q2 < 2; ++q2) {
      T g = 0, T11 = 0, T22 = 0, T12 = 0, m = 0;
      if (needG) {
        const T pt = phitq[q1][q2];
        g = c.omk * pt * pt + c.kap;
      }
      if (needLinU) {
        const T e11 = fux.dxi[q2] * c.ihx;
        const T e22 = fuy.deta[q1] * c.ihy;
        const T ge12 = fux.deta[q1] * c.ihy + fuy.dxi[q2] * c.ihx;   // 2 e12
        const T s11 = c.c2ml * e11 + c.cl * e22;
        const T s22 = c.cl * e11 + c.c2ml * e22;
        const T s12 = c.cm * ge12;
        const T se = s11 * e11 + s22 * e22 + s12 * ge12;
        m = c.omk * se + T(2) * c.p * (e11 + e22) + c.gcl;
        if (needPhi) {
          const T tp = T(2) * phiq[q1][q2];
          T11 = tp * (c.omk * s11 + c.p);
          T22 = tp * (c.omk * s22 + c.p);
          T12 = tp * (c.omk * s12);
        }
      }
      if (OP == OP_FULL || OP == OP_FULL_T || OP == OP_UU) {
        const T a = fxu.dxi[q2] * c.ihx;                             // d du_x / dx
        const T d = fxv.deta[q1] * c.ihy;                            // d du_y / dy
        const T bc = fxu.deta[q1] * c.ihy + fxv.dxi[q2] * c.ihx;     // d du_x/dy + d du_y/dx
        T S11 = g * (c.c2ml * a + c.cl * d);
        T S22 = g * (c.cl * a + c.c2ml * d);
        T S12 = g * (c.cm * bc);
        if (OP == OP_FULL_T) {
          const T dp = xpq[q1][q2];
          S11 += dp * T11;
          S22 += dp * T22;
          S12 += dp * T12;
        }
        fux_x[q1][q2] = S11;  // u_x test: (S11, S12) . grad psi
        fux_y[q1][q2] = S12;
        fuy_x[q1][q2] = S12;  // u_y test: (S12, S22) . grad psi
        fuy_y[q1][q2] = S22;
        if (OP == OP_FULL) fv[q1][q2] = T11 * a + T22 * d + T12 * bc;
      }
      if (OP == OP_FULL || OP == OP_FULL_T || OP == OP_PP) {
        const T mv = m * xpq[q1][q2];
        if (OP == OP_FULL) fv[q1][q2] += mv; else fv[q1][q2] = mv;
      }
      if (OP == OP_UU_DIAG) {
        // diag of (g sigma(N e_i), e(N e_i)): (2mu+lam)(dN/dx_i)^2 + mu (dN/dx_j)^2
        // qp contributions accumulated directly
        const T xi = q1 ? T(GB) : T(GA), eta = q2 ? T(GB) : T(GA);
        const T dxs[4] = {-(1 - eta), (1 - eta), -eta, eta};
        const T dys[4] = {-(1 - xi), -xi, (1 - xi), xi};
#pragma unroll
        for (int A = 0; A < 4; ++A) {
          const T dx = dxs[A] * c.ihx, dy = dys[A] * c.ihy;
          rux[A] += c.jxw * g * (c.c2ml * dx * dx + c.cm * dy * dy);
          ruy[A] += c.jxw * g * (c.cm * dx * dx + c.c2ml * dy * dy);
        }
      }
      if (OP == OP_PP_DIAG) {
        const T xi = q1 ? T(GB) : T(GA), eta = q2 ? T(GB) : T(GA);
        const T Ns[4] = {(1 - xi) * (1 - eta), xi * (1 - eta), (1 - xi) * eta, xi * eta};
        const T dxs[4] = {-(1 - eta), (1 - eta), -eta, eta};
        const T dys[4] = {-(1 - xi), -xi, (1 - xi), xi};
#pragma unroll
        for (int A = 0; A < 4; ++A) {
          const T dx = dxs[A] * c.ihx, dy = dys[A] * c.ihy;
          rp[A] += c.jxw * (m * Ns[A] * Ns[A] + c.gcL * (dx * dx + dy * dy));
        }
      }
    }
  if (OP == OP_FULL || OP == OP_FULL_T || OP == OP_UU) {
    q1_test_grad(fux_x, fux_y, c.wx, c.wy, rux);
    q1_test_grad(fuy_x, fuy_y, c.wx, c.wy, ruy);
  }
  if (OP == OP_FULL || OP == OP_FULL_T || OP == OP_PP) {
    q1_test_val(fv, c.jxw, rp);
    // G_c l (grad dphi, grad psi): reference fluxes are constant along one direction
    T gx[2][2], gy[2][2];
#pragma unroll
    for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
      for (int q2 = 0; q2 < 2; ++q2) {
        gx[q1][q2] = fxp.dxi[q2];
        gy[q1][q2] = fxp.deta[q1];
      }
    q1_test_grad(gx, gy, c.wpx, c.wpy, rp);
  }
#pragma unroll
  for (int A = 0; A < 4; ++A) {
    out[3 * A + 0] = rux[A];
    out[3 * A + 1] = ruy[A];
    out[3 * A + 2] = rp[A];
  }
  (void)needU; (void)needP;
}

template <typename T>
__device__ __forceinline__ const CellConst<T>& cconst(const ApplyArgs& a, int level);
template <>
__device__ __forceinline__ const CellConst<float>& cconst<float>(const ApplyArgs& a, int level) { return a.cf[level]; }
template <>
__device__ __forceinline__ const CellConst<double>& cconst<double>(const ApplyArgs& a, int level) { return a.cd[level]; }

template <typename T, int OP>
__global__ void __launch_bounds__(NTHREADS) apply_q1_kernel(const __grid_constant__ ApplyArgs a) {
  using T2 = typename VT<T>::T2;
  using T4 = typename VT<T>::T4;
  constexpr bool inU = (OP == OP_FULL || OP == OP_FULL_T || OP == OP_UU);
  constexpr bool inP = (OP == OP_FULL || OP == OP_FULL_T || OP == OP_PP);
  constexpr bool outU = (OP != OP_PP && OP != OP_PP_DIAG);
  constexpr bool outP = (OP == OP_FULL || OP == OP_FULL_T || OP == OP_PP || OP == OP_PP_DIAG);
  constexpr int NOUT = 12;
  __shared__ T s_x0[NWIN], s_x1[NWIN], s_xp[NWIN];
  __shared__ T4 s_lin[NWIN];
  __shared__ T s_out[NOUT][NCELL];
  __shared__ int s_nb[9];
  __shared__ int s_irr, s_level;

  const int tid = threadIdx.x;
  const BrickDesc* bd = a.lay.bricks + blockIdx.x;
  if (tid < 9) s_nb[tid] = bd->nbr_base[tid];
  if (tid == 9) s_irr = bd->irr;
  if (tid == 10) s_level = bd->level;
  __syncthreads();
  const int irr = s_irr;
  const int level = s_level;
  const T2* xu = reinterpret_cast<const T2*>(a.xu);
  const T* xp = reinterpret_cast<const T*>(a.xp);
  const T4* lin = reinterpret_cast<const T4*>(a.lin);
  const bool mask = (a.mode & MODE_MASK_INPUT) != 0;

  // ---- 1. window gather
  for (int s = tid; s < NWIN; s += NTHREADS) {
    int32_t code;
    if (irr < 0) {
      const int oi = s % WN - 1, oj = s / WN - 1;
      const int dx = oi < 0 ? -1 : (oi >= NB ? 1 : 0);
      const int dy = oj < 0 ? -1 : (oj >= NB ? 1 : 0);
      code = s_nb[(dy + 1) * 3 + dx + 1] + (oi - dx * NB) + NB * (oj - dy * NB);
    } else {
      code = a.lay.win[irr * NWIN + s];
    }
    T v0 = 0, v1 = 0, vp = 0;
    T4 L = {0, 0, 0, 0};
    if (code >= 0) {
      if (inU) { const T2 v = ldg(xu + code); v0 = v.x; v1 = v.y; }
      if (inP) vp = ldg(xp + code);
      L = ldg4(lin + code);
      if (mask) {
        const uint8_t cm = ldg(a.cmask + code);
        if (cm & 1) v0 = 0;
        if (cm & 2) v1 = 0;
        if (cm & 4) vp = 0;
      }
    } else if (code <= -2) {
      const DevHanging& h = a.hang[-2 - code];
      L = ldg4(lin + h.slot);
      const int np = a.fe_degree + 1;
      for (int b = 0; b < np; ++b) {
        const int ps = h.parent[b];
        const T w = T(h.weight[b]);
        T p0 = 0, p1 = 0, pp = 0;
        if (inU) { const T2 v = ldg(xu + ps); p0 = v.x; p1 = v.y; }
        if (inP) pp = ldg(xp + ps);
        if (mask) {
          const uint8_t cm = ldg(a.cmask + ps);
          if (cm & 1) p0 = 0;
          if (cm & 2) p1 = 0;
          if (cm & 4) pp = 0;
        }
        v0 += w * p0; v1 += w * p1; vp += w * pp;
      }
    }
    s_x0[s] = v0; s_x1[s] = v1; s_xp[s] = vp;
    s_lin[s] = L;
  }
  __syncthreads();

  // ---- 2. cells
  {
    const int ci = tid % WC, cj = tid / WC;
    bool active = true;
    if (irr >= 0) active = (a.lay.cellmask[irr * 8 + (tid >> 5)] >> (tid & 31)) & 1u;
    T out[12];
    if (active) {
      const CellConst<T>& c = cconst<T>(a, level);
      q1_cell<T, OP>(s_x0, s_x1, s_xp, s_lin, ci + WN * cj, c, out);
    } else {
#pragma unroll
      for (int q = 0; q < 12; ++q) out[q] = 0;
    }
#pragma unroll
    for (int q = 0; q < NOUT; ++q) s_out[q][tid] = out[q];
  }
  __syncthreads();

  // ---- 3. owned nodes
  if (tid < NOWN) {
    const int oi = tid % NB, oj = tid / NB;
    const int c00 = oi + WC * oj;  // this node is local node 3 of c00, 2 of c00+1, 1 of c00+WC, 0 of c00+WC+1
    T y[3];
#pragma unroll
    for (int comp = 0; comp < 3; ++comp)
      y[comp] = s_out[9 + comp][c00] + s_out[6 + comp][c00 + 1] + s_out[3 + comp][c00 + WC] +
                s_out[0 + comp][c00 + WC + 1];
    int act = kActFinal;
    int part = -1;
    if (irr >= 0) {
      act = a.lay.own_act[irr * NOWN + tid];
      part = a.lay.own_part[irr * NOWN + tid];
    }
    const int slot = s_nb[4] + oi + NB * oj;
    T2* yu = reinterpret_cast<T2*>(a.yu);
    T* yp = reinterpret_cast<T*>(a.yp);
    if (part >= 0) {
      T* ib = reinterpret_cast<T*>(a.ibuf) + 3 * int64_t(part);
      ib[0] = y[0]; ib[1] = y[1]; ib[2] = y[2];
    }
    if (act == kActFinal) {
      if (OP == OP_UU_DIAG || OP == OP_PP_DIAG) {
        // diagonal entries; fixed rows get 0 (their inverse is set to 0 too)
        const uint8_t cm = ldg(a.cmask + slot);
        if (outU) {
          T2 o; o.x = (cm & 1) ? T(0) : y[0]; o.y = (cm & 2) ? T(0) : y[1];
          yu[slot] = o;
        }
        if (outP) yp[slot] = (cm & 4) ? T(0) : y[2];
      } else {
        const uint8_t cm = ldg(a.cmask + slot);
        if (cm) {
          const bool ident = (a.mode & MODE_IDENTITY) != 0;
          if (cm & 1) y[0] = ident ? ldg(xu + slot).x : T(0);
          if (cm & 2) y[1] = ident ? ldg(xu + slot).y : T(0);
          if (cm & 4) y[2] = ident ? ldg(xp + slot) : T(0);
        }
        if (outU) { T2 o; o.x = y[0]; o.y = y[1]; yu[slot] = o; }
        if (outP) yp[slot] = y[2];
      }
    } else if (act == kActZero) {
      if (outU) { T2 o; o.x = 0; o.y = 0; yu[slot] = o; }
      if (outP) yp[slot] = 0;
    }
  }
}

template <typename T>
__global__ void fixup_kernel(const FixupArgs a) {
  using T2 = typename VT<T>::T2;
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= a.n) return;
  const int slot = a.slot[f];
  const T* ib = reinterpret_cast<const T*>(a.ibuf);
  T y0 = 0, y1 = 0, y2 = 0;
  for (int e = a.ptr[f]; e < a.ptr[f + 1]; ++e) {
    const int p = a.part[e];
    const T w = T(a.w[e]);
    y0 += w * ib[3 * p + 0];
    y1 += w * ib[3 * p + 1];
    y2 += w * ib[3 * p + 2];
  }
  const uint8_t cm = a.cmask[slot];
  if (cm) {
    const bool ident = (a.mode & MODE_IDENTITY) != 0;
    const T2* xu = reinterpret_cast<const T2*>(a.xu);
    const T* xp = reinterpret_cast<const T*>(a.xp);
    if (cm & 1) y0 = ident ? xu[slot].x : T(0);
    if (cm & 2) y1 = ident ? xu[slot].y : T(0);
    if (cm & 4) y2 = ident ? xp[slot] : T(0);
  }
  T2 o; o.x = y0; o.y = y1;
  reinterpret_cast<T2*>(a.yu)[slot] = o;
  reinterpret_cast<T*>(a.yp)[slot] = y2;
}

__global__ void set_lin_kernel(int64_t n, const double2* __restrict__ u, const double* __restrict__ phi,
                               const double* __restrict__ phit, dbl4* lin64, float4* lin32) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double2 uu = u[s];
  dbl4 v;
  v.x = uu.x; v.y = uu.y; v.z = phi[s]; v.w = phit[s];
  lin64[s] = v;
  lin32[s] = make_float4(float(v.x), float(v.y), float(v.z), float(v.w));
}

__global__ void set_lin_hanging_kernel(int32_t nh, const DevHanging* __restrict__ hang, int np,
                                       dbl4* lin64, float4* lin32) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= nh) return;
  const DevHanging e = hang[h];
  dbl4 v;
  v.x = 0; v.y = 0; v.z = 0; v.w = 0;
  for (int b = 0; b < np; ++b) {
    const dbl4 p = lin64[e.parent[b]];
    v.x += e.weight[b] * p.x; v.y += e.weight[b] * p.y;
    v.z += e.weight[b] * p.z; v.w += e.weight[b] * p.w;
  }
  lin64[e.slot] = v;
  lin32[e.slot] = make_float4(float(v.x), float(v.y), float(v.z), float(v.w));
}

template <typename T>
void fill_cc(CellConst<T>& c, const ApplyArgs& a, double hx, double hy) {
  c.ihx = T(1.0 / hx); c.ihy = T(1.0 / hy);
  c.c2ml = T(2.0 * a.mu + a.lam); c.cl = T(a.lam); c.cm = T(a.mu);
  c.omk = T(1.0 - a.kappa); c.kap = T(a.kappa); c.p = T(a.p);
  c.gcl = T(a.gc_over_l); c.gcL = T(a.gc_times_l);
  c.jxw = T(0.25 * hx * hy);
  c.wx = T(0.25 * hy); c.wy = T(0.25 * hx);
  c.wpx = T(0.25 * a.gc_times_l * hy / hx); c.wpy = T(0.25 * a.gc_times_l * hx / hy);
}

}  // namespace

void fill_cell_constants(ApplyArgs& a, int nlevels) {
  for (int l = 0; l < nlevels && l < kMaxLevels; ++l) {
    fill_cc(a.cf[l], a, a.hx[l], a.hy[l]);
    fill_cc(a.cd[l], a, a.hx[l], a.hy[l]);
  }
}

template <typename T>
cudaError_t launch_apply(const ApplyArgs& a, int op, cudaStream_t s) {
  if (a.lay.nbricks <= 0) return cudaSuccess;
  if (a.fe_degree != 1) return cudaErrorInvalidValue;
  switch (op) {
    case OP_FULL: apply_q1_kernel<T, OP_FULL><<<a.lay.nbricks, NTHREADS, 0, s>>>(a); break;
    case OP_FULL_T: apply_q1_kernel<T, OP_FULL_T><<<a.lay.nbricks, NTHREADS, 0, s>>>(a); break;
    case OP_UU: apply_q1_kernel<T, OP_UU><<<a.lay.nbricks, NTHREADS, 0, s>>>(a); break;
    case OP_PP: apply_q1_kernel<T, OP_PP><<<a.lay.nbricks, NTHREADS, 0, s>>>(a); break;
    case OP_UU_DIAG: apply_q1_kernel<T, OP_UU_DIAG><<<a.lay.nbricks, NTHREADS, 0, s>>>(a); break;
    case OP_PP_DIAG: apply_q1_kernel<T, OP_PP_DIAG><<<a.lay.nbricks, NTHREADS, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fixup(const FixupArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  fixup_kernel<T><<<(a.n + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_set_lin(int64_t n_slots, const double* u, const double* phi, const double* phit,
                           const DevHanging* hang, int32_t nhang, int fe_degree,
                           double* lin64, float* lin32, cudaStream_t s) {
  if (n_slots > 0)
    set_lin_kernel<<<unsigned((n_slots + 255) / 256), 256, 0, s>>>(
        n_slots, reinterpret_cast<const double2*>(u), phi, phit, reinterpret_cast<dbl4*>(lin64),
        reinterpret_cast<float4*>(lin32));
  if (nhang > 0)
    set_lin_hanging_kernel<<<(nhang + 127) / 128, 128, 0, s>>>(nhang, hang, fe_degree + 1,
                                                                reinterpret_cast<dbl4*>(lin64),
                                                                reinterpret_cast<float4*>(lin32));
  return cudaGetLastError();
}

template cudaError_t launch_apply<float>(const ApplyArgs&, int, cudaStream_t);
template cudaError_t launch_apply<double>(const ApplyArgs&, int, cudaStream_t);
template cudaError_t launch_fixup<float>(const FixupArgs&, cudaStream_t);
template cudaError_t launch_fixup<double>(const FixupArgs&, cudaStream_t);

}  // namespace pff

namespace pff {
namespace {
__global__ void leaf_cmask_kernel(int64_t n, const uint8_t* __restrict__ flags, const uint8_t* __restrict__ active,
                                  uint8_t* __restrict__ cmask) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint8_t f = flags[s];
  uint8_t c = 0;
  if ((f & 1) && (f & 2)) c |= 3;                           // Dirichlet u on the boundary
  if (active && (f & 1) && !(f & 4) && active[s]) c |= 4;   // active phi (never on hanging nodes)
  cmask[s] = c;
}
}  // namespace

cudaError_t launch_leaf_cmask(int64_t n, const uint8_t* slot_flags, const uint8_t* active, uint8_t* cmask,
                              cudaStream_t s) {
  if (n > 0) leaf_cmask_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(n, slot_flags, active, cmask);
  return cudaGetLastError();
}
}  // namespace pff
