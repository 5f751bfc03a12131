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
// One warp per strip of RSEG node rows of a brick of 30x30 owned node slots
// (a "row sweep"): lane l owns node column l-1 of the brick window (columns
// -1..30), computes cell (l-1, c) of every cell row c of the strip (sum-factorised
// 2x2 Gauss evaluation and test) and exchanges node values and nodal
// contributions with its neighbour lanes by warp shuffles.  Rows are loaded
// straight from HBM into registers (coalesced: a row of a brick is 30
// consecutive slots) one row ahead of the arithmetic; there is no shared memory
// and no block barrier.  Input x has its hanging-node constraints resolved on
// the fly and fixed components masked.  Each owned node is written once, by
// one lane, in a fixed summation order.  Nodes shared with another level,
// hanging nodes and their parents write partial sums; a small fix-up kernel
// condenses them (x_full = C x on input, C^T y on output).  No atomics.
#include "kernels.cuh"

#include <mutex>
#include <unordered_map>

namespace pff {

namespace {

template <typename T> struct VT;
template <> struct VT<float> { using T2 = float2; using T4 = float4; };
template <> struct VT<double> { using T2 = double2; using T4 = dbl4; };

constexpr int NB = 30;          // owned node slots per brick side
constexpr int WN = 32;          // window nodes per side (columns -1..30)
constexpr int NCW = 31;         // window cells per side (cells -1..29)
#ifndef PFF_RSEG
#define PFF_RSEG 10
#endif
#ifndef PFF_WARPS
#define PFF_WARPS 4
#endif
#ifndef PFF_MINB
#define PFF_MINB 1
#endif
constexpr int RSEG = PFF_RSEG;  // node rows per warp strip (divides NB)
constexpr int NSEG = NB / RSEG;
constexpr int WARPS = PFF_WARPS;  // warps per CTA (independent strips)
static_assert(NB % RSEG == 0, "strip height must divide the brick");

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

// Node data of one window slot held in registers: input x (masked, hanging
// resolved) and the linearisation.
template <typename T>
struct NodeVal {
  T x0, x1, xp;
  typename VT<T>::T4 L;
};

// Which node fields an operator reads.
template <int OP> struct Needs {
  static constexpr bool xu = (OP == OP_FULL || OP == OP_FULL_T || OP == OP_UU);
  static constexpr bool xp = (OP == OP_FULL || OP == OP_FULL_T || OP == OP_PP);
  static constexpr bool linU = (OP == OP_FULL || OP == OP_FULL_T || OP == OP_PP || OP == OP_PP_DIAG);
  static constexpr bool phi = (OP == OP_FULL || OP == OP_FULL_T);
  static constexpr bool phit = (OP == OP_FULL || OP == OP_FULL_T || OP == OP_UU || OP == OP_UU_DIAG);
};

// ---- packed pairs: two Gauss points (eta = GA, GB at one xi) per operation.
// FP32 uses Blackwell's paired FP32 instructions (FFMA2 / FADD2 / FMUL2);
// FP64 falls back to two scalar operations.
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pbc(float s) { return make_float2(s, s); }
__device__ __forceinline__ double2 pfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 pmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 pbc(double s) { return make_double2(s, s); }

// One Q1 cell with nodes v[0] (0,0), v[1] (1,0), v[2] (0,1), v[3] (1,1).
// out[3*A + c] (c: 0 u_x, 1 u_y, 2 phi).  OP_UU fills components 0, 1;
// OP_PP component 2; the *_DIAG operators the diagonal entries.
//
// Reference-cell fields (sum factorisation on 2x2 Gauss points, eta_q = GA, GB):
//   d/dxi at the two eta points is a pair P (same for both xi points),
//   d/deta at xi point q1 is a scalar, values at (xi_q1, eta_*) a pair.
template <typename T, int OP>
__device__ __forceinline__ void q1_cell(const NodeVal<T> v[4], const CellConst<T>& c, T out[12]) {
  using N = Needs<OP>;
  using P = typename VT<T>::T2;
  const P G2 = {T(GA), T(GB)};
  T rux[4] = {0, 0, 0, 0}, ruy[4] = {0, 0, 0, 0}, rp[4] = {0, 0, 0, 0};
  if (OP == OP_UU_DIAG || OP == OP_PP_DIAG) {
    // diagonal entries, once per Newton step: plain scalar quadrature
    Q1Field<T> fux, fuy;
    T phitq[2][2];
    if (N::linU) {
      fux.grads(v[0].L.x, v[1].L.x, v[2].L.x, v[3].L.x);
      fuy.grads(v[0].L.y, v[1].L.y, v[2].L.y, v[3].L.y);
    }
    if (N::phit) q1_values(v[0].L.w, v[1].L.w, v[2].L.w, v[3].L.w, phitq);
#pragma unroll
    for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
      for (int q2 = 0; q2 < 2; ++q2) {
        const T xi = q1 ? T(GB) : T(GA), eta = q2 ? T(GB) : T(GA);
        const T dxs[4] = {-(1 - eta), (1 - eta), -eta, eta};
        const T dys[4] = {-(1 - xi), -xi, (1 - xi), xi};
        if (OP == OP_UU_DIAG) {
          const T pt = phitq[q1][q2];
          const T g = c.omk * pt * pt + c.kap;
#pragma unroll
          for (int A = 0; A < 4; ++A) {
            const T dx = dxs[A] * c.ihx, dy = dys[A] * c.ihy;
            rux[A] += c.jxw * g * (c.c2ml * dx * dx + c.cm * dy * dy);
            ruy[A] += c.jxw * g * (c.cm * dx * dx + c.c2ml * dy * dy);
          }
        } else {
          const T e11 = fux.dxi[q2] * c.ihx, e22 = fuy.deta[q1] * c.ihy;
          const T ge12 = fux.deta[q1] * c.ihy + fuy.dxi[q2] * c.ihx;
          const T s11 = c.c2ml * e11 + c.cl * e22, s22 = c.cl * e11 + c.c2ml * e22, s12 = c.cm * ge12;
          const T m = c.omk * (s11 * e11 + s22 * e22 + s12 * ge12) + T(2) * c.p * (e11 + e22) + c.gcl;
          const T Ns[4] = {(1 - xi) * (1 - eta), xi * (1 - eta), (1 - xi) * eta, xi * eta};
#pragma unroll
          for (int A = 0; A < 4; ++A) {
            const T dx = dxs[A] * c.ihx, dy = dys[A] * c.ihy;
            rp[A] += c.jxw * (m * Ns[A] * Ns[A] + c.gcL * (dx * dx + dy * dy));
          }
        }
      }
  } else {
    // ---- linearisation: d/dxi pairs (eta points), d/deta scalars per xi point
    P e11 = pbc(T(0)), uyxi = pbc(T(0));
    T uxeta[2] = {0, 0}, e22s[2] = {0, 0};
    if (N::linU) {
      const T ax0 = v[1].L.x - v[0].L.x, ay0 = v[2].L.x - v[0].L.x, aX = (v[3].L.x - v[2].L.x) - ax0;
      const T bx0 = v[1].L.y - v[0].L.y, by0 = v[2].L.y - v[0].L.y, bX = (v[3].L.y - v[2].L.y) - bx0;
      e11 = pmul(pfma(G2, pbc(aX), pbc(ax0)), pbc(c.ihx));    // du_x/dx at the eta points
      uyxi = pmul(pfma(G2, pbc(bX), pbc(bx0)), pbc(c.ihx));   // du_y/dx
      uxeta[0] = (ay0 + T(GA) * aX) * c.ihy;                   // du_x/dy at xi points
      uxeta[1] = (ay0 + T(GB) * aX) * c.ihy;
      e22s[0] = (by0 + T(GA) * bX) * c.ihy;                    // du_y/dy
      e22s[1] = (by0 + T(GB) * bX) * c.ihy;
    }
    // values of a field at (xi_q1, eta_*): pair per q1
    auto vals = [&](T v0, T v1, T v2, T v3, P out2[2]) {
      const T dx0 = v1 - v0, dy0 = v2 - v0, X = (v3 - v2) - dx0;
      const T de0 = dy0 + T(GA) * X, de1 = dy0 + T(GB) * X;
      const T vb0 = v0 + T(GA) * dx0, vb1 = v0 + T(GB) * dx0;
      out2[0] = pfma(G2, pbc(de0), pbc(vb0));
      out2[1] = pfma(G2, pbc(de1), pbc(vb1));
    };
    P phiP[2], phitP[2];
    if (N::phi) vals(v[0].L.z, v[1].L.z, v[2].L.z, v[3].L.z, phiP);
    if (N::phit) vals(v[0].L.w, v[1].L.w, v[2].L.w, v[3].L.w, phitP);
    // ---- input
    P axi = pbc(T(0)), cxi = pbc(T(0)), pxi = pbc(T(0));
    T beta[2] = {0, 0}, deta[2] = {0, 0}, peta[2] = {0, 0};
    P xpP[2];
    if (N::xu) {
      const T ax0 = v[1].x0 - v[0].x0, ay0 = v[2].x0 - v[0].x0, aX = (v[3].x0 - v[2].x0) - ax0;
      const T bx0 = v[1].x1 - v[0].x1, by0 = v[2].x1 - v[0].x1, bX = (v[3].x1 - v[2].x1) - bx0;
      axi = pmul(pfma(G2, pbc(aX), pbc(ax0)), pbc(c.ihx));   // d dux/dx (pair over eta)
      cxi = pmul(pfma(G2, pbc(bX), pbc(bx0)), pbc(c.ihx));   // d duy/dx
      beta[0] = (ay0 + T(GA) * aX) * c.ihy;                   // d dux/dy (per xi)
      beta[1] = (ay0 + T(GB) * aX) * c.ihy;
      deta[0] = (by0 + T(GA) * bX) * c.ihy;                   // d duy/dy
      deta[1] = (by0 + T(GB) * bX) * c.ihy;
    }
    if (N::xp) {
      const T px0 = v[1].xp - v[0].xp, py0 = v[2].xp - v[0].xp, pX = (v[3].xp - v[2].xp) - px0;
      pxi = pfma(G2, pbc(pX), pbc(px0));                      // reference d dphi/dxi (pair over eta)
      peta[0] = py0 + T(GA) * pX;                              // reference d dphi/deta (per xi)
      peta[1] = py0 + T(GB) * pX;
      vals(v[0].xp, v[1].xp, v[2].xp, v[3].xp, xpP);
    }
    // per xi point: the pair of eta points
    P Fux_x[2], Fux_y[2], Fuy_y[2], Fv[2];
#pragma unroll
    for (int q1 = 0; q1 < 2; ++q1) {
      P g = pbc(T(0)), T11 = pbc(T(0)), T22 = pbc(T(0)), T12 = pbc(T(0)), m = pbc(T(0));
      if (N::phit) g = pfma(pbc(c.omk), pmul(phitP[q1], phitP[q1]), pbc(c.kap));
      if (N::linU) {
        const P ge12 = padd(pbc(uxeta[q1]), uyxi);   // 2 e12
        const P e22 = pbc(e22s[q1]);
        const P s11 = pfma(pbc(c.c2ml), e11, pbc(c.cl * e22s[q1]));
        const P s22 = pfma(pbc(c.cl), e11, pbc(c.c2ml * e22s[q1]));
        const P s12 = pmul(pbc(c.cm), ge12);
        const P se = pfma(s11, e11, pfma(s22, e22, pmul(s12, ge12)));
        m = pfma(pbc(c.omk), se, pfma(pbc(T(2) * c.p), padd(e11, e22), pbc(c.gcl)));
        if (N::phi) {
          const P tp = padd(phiP[q1], phiP[q1]);
          T11 = pmul(tp, pfma(pbc(c.omk), s11, pbc(c.p)));
          T22 = pmul(tp, pfma(pbc(c.omk), s22, pbc(c.p)));
          T12 = pmul(tp, pmul(pbc(c.omk), s12));
        }
      }
      if (N::xu) {
        const P bcp = padd(pbc(beta[q1]), cxi);          // d dux/dy + d duy/dx
        const P d = pbc(deta[q1]);
        P S11 = pmul(g, pfma(pbc(c.c2ml), axi, pbc(c.cl * deta[q1])));
        P S22 = pmul(g, pfma(pbc(c.cl), axi, pbc(c.c2ml * deta[q1])));
        P S12 = pmul(g, pmul(pbc(c.cm), bcp));
        if (OP == OP_FULL_T) {
          S11 = pfma(xpP[q1], T11, S11);
          S22 = pfma(xpP[q1], T22, S22);
          S12 = pfma(xpP[q1], T12, S12);
        }
        Fux_x[q1] = S11;
        Fux_y[q1] = S12;   // also the d/dxi flux of the u_y test
        Fuy_y[q1] = S22;
        if (OP == OP_FULL) Fv[q1] = pfma(T11, axi, pfma(T22, d, pfma(T12, bcp, pmul(m, xpP[q1]))));
      }
      if (N::xp && OP != OP_FULL) Fv[q1] = pmul(m, xpP[q1]);
    }
    // ---- test.  d/dxi flux pairs (per eta point, summed over xi) and d/deta
    // fluxes (per xi point, summed over eta):
    //   dN/dxi: N0 -(1-eta), N1 (1-eta), N2 -eta, N3 eta
    //   dN/deta: N0 -(1-xi), N1 -xi, N2 (1-xi), N3 xi
    auto test_grad = [&](P fxi0, P fxi1, T fe0, T fe1, T wx, T wy, T r[4]) {
      const P sx = padd(fxi0, fxi1);                  // sum over xi, per eta
      const T px = T(GA) * sx.x + T(GB) * sx.y;       // eta-weighted
      const T qx = (sx.x + sx.y) - px;                // (1-eta)-weighted
      const T py = T(GA) * fe0 + T(GB) * fe1;         // xi-weighted
      const T qy = (fe0 + fe1) - py;
      r[0] += -wx * qx - wy * qy;
      r[1] += wx * qx - wy * py;
      r[2] += -wx * px + wy * qy;
      r[3] += wx * px + wy * py;
    };
    if (N::xu) {
      // u_x test: (S11, S12) . grad psi;  u_y test: (S12, S22) . grad psi
      test_grad(Fux_x[0], Fux_x[1], Fux_y[0].x + Fux_y[0].y, Fux_y[1].x + Fux_y[1].y, c.wx, c.wy, rux);
      test_grad(Fux_y[0], Fux_y[1], Fuy_y[0].x + Fuy_y[0].y, Fuy_y[1].x + Fuy_y[1].y, c.wx, c.wy, ruy);
    }
    if (N::xp) {
      // value test against N_A = L_a(xi) L_b(eta)
      const T s0 = Fv[0].x + Fv[0].y, s1 = Fv[1].x + Fv[1].y;
      const T t0 = T(GA) * Fv[0].x + T(GB) * Fv[0].y, t1 = T(GA) * Fv[1].x + T(GB) * Fv[1].y;
      const T b0 = s0 - t0, b1 = s1 - t1;
      const T pb = T(GA) * b0 + T(GB) * b1, pt = T(GA) * t0 + T(GB) * t1;
      rp[0] += c.jxw * ((b0 + b1) - pb);
      rp[1] += c.jxw * pb;
      rp[2] += c.jxw * ((t0 + t1) - pt);
      rp[3] += c.jxw * pt;
      // G_c l (grad dphi, grad psi): the d/dxi flux is the same at both xi points
      test_grad(pxi, pxi, T(2) * peta[0], T(2) * peta[1], c.wpx, c.wpy, rp);
    }
  }
#pragma unroll
  for (int A = 0; A < 4; ++A) {
    out[3 * A + 0] = rux[A];
    out[3 * A + 1] = ruy[A];
    out[3 * A + 2] = rp[A];
  }
}

template <typename T>
__device__ __forceinline__ const CellConst<T>& cconst(const ApplyArgs& a, int level);
template <>
__device__ __forceinline__ const CellConst<float>& cconst<float>(const ApplyArgs& a, int level) { return a.cf[level]; }
template <>
__device__ __forceinline__ const CellConst<double>& cconst<double>(const ApplyArgs& a, int level) { return a.cd[level]; }

// ---- asynchronous global -> shared copies (Ampere+ cp.async), per lane
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src));
}
template <typename X>
__device__ __forceinline__ void cp_async_x(X* dst, const X* src) {
  if constexpr (sizeof(X) == 4) cp_async4(dst, src);
  else if constexpr (sizeof(X) == 8) cp_async8(dst, src);
  else if constexpr (sizeof(X) == 16) cp_async16(dst, src);
  else { cp_async16(dst, src); cp_async16(reinterpret_cast<char*>(dst) + 16, reinterpret_cast<const char*>(src) + 16); }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

#ifndef PFF_DEPTH
#define PFF_DEPTH 4
#endif
constexpr int DEPTH = PFF_DEPTH;  // ring stages per warp (rows in flight: DEPTH-1)
constexpr int NROWS = RSEG + 2;   // node rows a strip reads

// One ring stage: one node row of the window for the 32 lanes of a warp.
template <typename T>
struct __align__(16) Stage {
  typename VT<T>::T4 lin[32];
  typename VT<T>::T2 xu[32];
  T xp[32];
  uint32_t cm[32];   // the 4-byte word of the constraint mask holding this slot's byte
};

template <typename T>
struct WarpSmem {
  Stage<T> st[DEPTH];
  int32_t code[NROWS][32];
};

// Storage code of window slot (n, r) of a regular brick.
__device__ __forceinline__ int32_t regular_code(int nbase, int n, int r) {
  const int dx = n < 0 ? -1 : (n >= NB ? 1 : 0);
  const int dy = r < 0 ? -1 : (r >= NB ? 1 : 0);
  const int base = __shfl_sync(0xffffffffu, nbase, (dy + 1) * 3 + dx + 1);
  return base + (n - dx * NB) + NB * (r - dy * NB);
}

// Issue the copies of one node row (code per lane) into a ring stage.
template <typename T, int OP>
__device__ __forceinline__ void issue_row(const ApplyArgs& a, int32_t code, Stage<T>& st, int lane) {
  using N = Needs<OP>;
  using T2 = typename VT<T>::T2;
  using T4 = typename VT<T>::T4;
  if (code >= 0) {
    cp_async_x(&st.lin[lane], reinterpret_cast<const T4*>(a.lin) + code);
    if (N::xu) cp_async_x(&st.xu[lane], reinterpret_cast<const T2*>(a.xu) + code);
    if (N::xp) cp_async_x(&st.xp[lane], reinterpret_cast<const T*>(a.xp) + code);
    cp_async4(&st.cm[lane], reinterpret_cast<const uint32_t*>(a.cmask + (code & ~3)));
  }
}

// Node value of window slot with storage code `code` from the ring stage
// (regular slots) or from global memory (hanging nodes: constraint applied).
template <typename T, int OP>
__device__ __forceinline__ void take_node(const ApplyArgs& a, int32_t code, const Stage<T>& st, int lane,
                                          NodeVal<T>& v, uint8_t& cmv) {
  using N = Needs<OP>;
  using T2 = typename VT<T>::T2;
  using T4 = typename VT<T>::T4;
  const bool mask = (a.mode & MODE_MASK_INPUT) != 0;
  v.x0 = 0; v.x1 = 0; v.xp = 0;
  v.L.x = 0; v.L.y = 0; v.L.z = 0; v.L.w = 0;
  cmv = 0;
  if (code >= 0) {
    v.L = st.lin[lane];
    if (N::xu) { const T2 q = st.xu[lane]; v.x0 = q.x; v.x1 = q.y; }
    if (N::xp) v.xp = st.xp[lane];
    cmv = uint8_t(st.cm[lane] >> (8 * (code & 3)));
    if (mask && cmv) {
      if (cmv & 1) v.x0 = 0;
      if (cmv & 2) v.x1 = 0;
      if (cmv & 4) v.xp = 0;
    }
  } else if (code <= -2) {
    const T2* xu = reinterpret_cast<const T2*>(a.xu);
    const T* xp = reinterpret_cast<const T*>(a.xp);
    const DevHanging& h = a.hang[-2 - code];
    v.L = ldg4(reinterpret_cast<const T4*>(a.lin) + h.slot);
    const int np = a.fe_degree + 1;
    for (int b = 0; b < np; ++b) {
      const int ps = h.parent[b];
      const T w = T(h.weight[b]);
      T p0 = 0, p1 = 0, pp = 0;
      if (N::xu) { const T2 q = ldg(xu + ps); p0 = q.x; p1 = q.y; }
      if (N::xp) pp = ldg(xp + ps);
      if (mask) {
        const uint8_t cm = ldg(a.cmask + ps);
        if (cm & 1) p0 = 0;
        if (cm & 2) p1 = 0;
        if (cm & 4) pp = 0;
      }
      v.x0 += w * p0; v.x1 += w * p1; v.xp += w * pp;
    }
  }
}

template <typename T, int OP>
__device__ __forceinline__ NodeVal<T> shfl_down_node(const NodeVal<T>& v) {
  using N = Needs<OP>;
  NodeVal<T> r;
  const unsigned FULL = 0xffffffffu;
  r.x0 = N::xu ? __shfl_down_sync(FULL, v.x0, 1) : T(0);
  r.x1 = N::xu ? __shfl_down_sync(FULL, v.x1, 1) : T(0);
  r.xp = N::xp ? __shfl_down_sync(FULL, v.xp, 1) : T(0);
  r.L.x = N::linU ? __shfl_down_sync(FULL, v.L.x, 1) : T(0);
  r.L.y = N::linU ? __shfl_down_sync(FULL, v.L.y, 1) : T(0);
  r.L.z = N::phi ? __shfl_down_sync(FULL, v.L.z, 1) : T(0);
  r.L.w = N::phit ? __shfl_down_sync(FULL, v.L.w, 1) : T(0);
  return r;
}

template <typename T, int OP>
__global__ void __launch_bounds__(32 * WARPS, PFF_MINB) apply_q1_kernel(const __grid_constant__ ApplyArgs a) {
  using T2 = typename VT<T>::T2;
  constexpr bool outU = (OP != OP_PP && OP != OP_PP_DIAG);
  constexpr bool outP = (OP == OP_FULL || OP == OP_FULL_T || OP == OP_PP || OP == OP_PP_DIAG);
  constexpr bool isDiag = (OP == OP_UU_DIAG || OP == OP_PP_DIAG);
  const unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpSmem<T>& ws = reinterpret_cast<WarpSmem<T>*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int nunits = a.lay.nbricks * NSEG;
  T2* yu = reinterpret_cast<T2*>(a.yu);
  T* yp = reinterpret_cast<T*>(a.yp);
  // persistent warps: grid-stride over strips (unit is uniform per warp)
  for (int unit = blockIdx.x * WARPS + (threadIdx.x >> 5); unit < nunits; unit += gridDim.x * WARPS) {
    const int b = unit / NSEG;
    const int r0 = (unit % NSEG) * RSEG;
    const BrickDesc* bd = a.lay.bricks + b;
    const int nbase = lane < 9 ? __ldg(bd->nbr_base + lane) : 0;
    const int irr = __ldg(&bd->irr);
    const int level = __ldg(&bd->level);
    const CellConst<T>& cc = cconst<T>(a, level);
    const int n = lane - 1;  // node column of this lane (-1..30)
    const int own_base = __shfl_sync(FULL, nbase, 4);
    // storage codes of the strip's window column
    __syncwarp();
#pragma unroll
    for (int i = 0; i < NROWS; ++i) {
      const int r = r0 - 1 + i;
      ws.code[i][lane] = irr < 0 ? regular_code(nbase, n, r) : __ldg(a.lay.win + irr * (WN * WN) + (n + 1) + WN * (r + 1));
    }
    // prologue: rows 0 .. DEPTH-2 in flight
#pragma unroll
    for (int i = 0; i < DEPTH - 1; ++i) {
      issue_row<T, OP>(a, ws.code[i][lane], ws.st[i], lane);
      cp_async_commit();
    }
    NodeVal<T> cur, curR;
    uint8_t cmcur = 0;
    T carry[3] = {0, 0, 0};
#pragma unroll 1
    for (int i = 0; i < NROWS; ++i) {
      if (i + DEPTH - 1 < NROWS) issue_row<T, OP>(a, ws.code[i + DEPTH - 1][lane], ws.st[(i + DEPTH - 1) % DEPTH], lane);
      cp_async_commit();
      cp_async_wait<DEPTH - 1>();
      NodeVal<T> nxt;
      uint8_t cmnxt;
      const int32_t codei = ws.code[i][lane];
      take_node<T, OP>(a, codei, ws.st[i % DEPTH], lane, nxt, cmnxt);
      const NodeVal<T> nxtR = shfl_down_node<T, OP>(nxt);
      if (i == 0) {
        cur = nxt; curR = nxtR; cmcur = cmnxt;
        continue;
      }
      const int c = r0 - 2 + i;  // cell row between node rows c (cur) and c + 1 (nxt)
      bool act = lane < NCW;
      if (irr >= 0 && act) {
        const int ci = (c + 1) * NCW + lane;
        act = (__ldg(a.lay.cellmask + irr * 31 + (ci >> 5)) >> (ci & 31)) & 1u;
      }
      T out[12];
      if (act) {
        NodeVal<T> v[4] = {cur, curR, nxt, nxtR};
        q1_cell<T, OP>(v, cc, out);
      } else {
#pragma unroll
        for (int q = 0; q < 12; ++q) out[q] = 0;
      }
      // the left neighbour's cell (n-1, c) contributes BR to node (n, c) and TR to node (n, c+1)
      T brL[3], trL[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        brL[q] = __shfl_up_sync(FULL, out[3 + q], 1);
        trL[q] = __shfl_up_sync(FULL, out[9 + q], 1);
      }
      if (c >= r0 && lane >= 1 && lane <= NB) {
        // node (n, c) is complete: carry (cells (n-1,c-1) TR, (n,c-1) TL) + (n-1,c) BR + (n,c) BL
        T y[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) y[q] = (carry[q] + brL[q]) + out[q];
        const int o = n + NB * c;  // owned slot
        int act_s = kActFinal, part = -1;
        if (irr >= 0) {
          act_s = __ldg(a.lay.own_act + irr * (NB * NB) + o);
          part = __ldg(a.lay.own_part + irr * (NB * NB) + o);
        }
        const int slot = own_base + o;
        if (part >= 0) {
          T* ib = reinterpret_cast<T*>(a.ibuf) + 3 * int64_t(part);
          ib[0] = y[0]; ib[1] = y[1]; ib[2] = y[2];
        }
        if (act_s == kActFinal) {
          // a home, single-level node: its slot is the window slot (n, c), whose mask is cmcur
          const uint8_t cm = cmcur;
          if (isDiag) {
            if (outU) { T2 o2; o2.x = (cm & 1) ? T(0) : y[0]; o2.y = (cm & 2) ? T(0) : y[1]; yu[slot] = o2; }
            if (outP) yp[slot] = (cm & 4) ? T(0) : y[2];
          } else {
            if (cm) {
              const bool ident = (a.mode & MODE_IDENTITY) != 0;
              const T2* xu = reinterpret_cast<const T2*>(a.xu);
              const T* xp = reinterpret_cast<const T*>(a.xp);
              if (cm & 1) y[0] = ident ? ldg(xu + slot).x : T(0);
              if (cm & 2) y[1] = ident ? ldg(xu + slot).y : T(0);
              if (cm & 4) y[2] = ident ? ldg(xp + slot) : T(0);
            }
            if (outU) { T2 o2; o2.x = y[0]; o2.y = y[1]; yu[slot] = o2; }
            if (outP) yp[slot] = y[2];
          }
        } else if (act_s == kActZero) {
          if (outU) { T2 o2; o2.x = 0; o2.y = 0; yu[slot] = o2; }
          if (outP) yp[slot] = 0;
        }
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) carry[q] = out[6 + q] + trL[q];
      cur = nxt;
      curR = nxtR;
      cmcur = cmnxt;
    }
    cp_async_wait<0>();
  }  // unit
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

// Blocks of `threads` threads of kernel fn that fit on all SMs at once (cached per kernel).
int resident_blocks(const void* fn, int threads, size_t smem) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(fn);
  if (it != cache.end()) return it->second;
  int dev = 0, sms = 1, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess || per_sm < 1) per_sm = 1;
  const int n = sms * per_sm;
  cache[fn] = n;
  return n;
}

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
  const int units = a.lay.nbricks * NSEG;
  const unsigned blk = 32 * WARPS;
  const size_t smem = sizeof(WarpSmem<T>) * WARPS;
  auto grid_of = [&](const void* fn) -> unsigned {
    const int full = resident_blocks(fn, int(blk), smem);
    const int need = (units + WARPS - 1) / WARPS;
    return unsigned(need < full ? need : full);
  };
  switch (op) {
#define PFF_LAUNCH(OPV)                                                                        \
    case OPV: {                                                                                \
      const void* fn = reinterpret_cast<const void*>(&apply_q1_kernel<T, OPV>);               \
      apply_q1_kernel<T, OPV><<<grid_of(fn), blk, smem, s>>>(a);                               \
      break;                                                                                   \
    }
    PFF_LAUNCH(OP_FULL)
    PFF_LAUNCH(OP_FULL_T)
    PFF_LAUNCH(OP_UU)
    PFF_LAUNCH(OP_PP)
    PFF_LAUNCH(OP_UU_DIAG)
    PFF_LAUNCH(OP_PP_DIAG)
#undef PFF_LAUNCH
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
