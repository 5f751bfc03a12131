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
// Execution: a column sweep over the brick layout (see sweep_q1_kernel).  A
// warp takes a strip of a brick of 30x30 owned node slots; lane L holds window
// node column L-1 (-1..30) and evaluates the cell to its right; the strip's
// lower and upper halves advance one cell row per step side by side, so every
// sum-factorised 2x2 Gauss operation of the two cells is one paired FP32
// instruction (FFMA2 / FADD2 / FMUL2) with no per-member index arithmetic.
// Node rows stream into a per-warp cp.async ring in shared memory; a lane reads
// its right neighbour's node values there and receives its left neighbour's
// nodal contributions by shuffle; there is no block barrier.  Fixed input
// components are masked in the ring; the input of hanging nodes (C x) comes from
// a pre-pass kernel.  Each owned node is written once, by one lane, in a fixed
// summation order.
// Nodes shared with another level, hanging nodes and their parents write
// partial sums; a small fix-up kernel condenses them (x_full = C x on input,
// C^T y on output).  No atomics.
#include "kernels.cuh"
#include "cheb.cuh"
#include "pdl.cuh"

#include <cmath>
#include <mutex>
#include <unordered_map>
#include <utility>

namespace pff {

namespace {

template <typename T> struct VT;
template <> struct VT<float> { using T2 = float2; using T4 = float4; };
template <> struct VT<double> { using T2 = double2; using T4 = dbl4; };

constexpr int NB = 30;          // owned node slots per brick side
constexpr int WN = 32;          // window nodes per side (columns -1..30)
constexpr int NCW = 31;         // window cells per side (cells -1..29)

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

// ---- packed pairs (two cells).  FP32: Blackwell paired instructions.
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
template <typename P>
__device__ __forceinline__ P psub(P a, P b) { return pfma(b, pbc(decltype(a.x)(-1)), a); }  // a - b, exact sign flip

// Which node fields an operator reads.
template <int OP> struct Needs {
  static constexpr bool xu = (OP == OP_FULL || OP == OP_FULL_T || OP == OP_UU || OP == OP_VJP || OP == OP_PHIT_VJP);
  static constexpr bool xp = (OP == OP_FULL || OP == OP_FULL_T || OP == OP_PP || OP == OP_VJP);
  static constexpr bool linU = (OP == OP_FULL || OP == OP_FULL_T || OP == OP_PP || OP == OP_PP_DIAG ||
                                OP == OP_RESID || OP == OP_TCV || OP == OP_TCV_GRAD || OP == OP_VJP ||
                                OP == OP_PHIT_VJP);
  static constexpr bool phi = (OP == OP_FULL || OP == OP_FULL_T || OP == OP_RESID || OP == OP_TCV ||
                               OP == OP_TCV_GRAD || OP == OP_VJP);
  static constexpr bool phit = (OP == OP_FULL || OP == OP_FULL_T || OP == OP_UU || OP == OP_UU_DIAG ||
                                OP == OP_RESID || OP == OP_VJP || OP == OP_PHIT_VJP);
};

// Node data of a column pair (A, B) of one window row, in registers.
template <typename T>
struct NodePair {
  typename VT<T>::T2 x0, x1, xp, lx, ly, lz, lw;
};

// Q1 field on a pair of cells: reference derivatives at the Gauss points.
//   dxi[q2] = dv/dxi at eta = g_q2, deta[q1] = dv/deta at xi = g_q1.
template <typename P>
struct PField {
  P dxi[2], deta[2];
  P dx0, dy0, X;
  // b, t: values at the cell's lower-left and upper-left nodes; hb, ht: the
  // right node minus the left node along the lower and upper edge
  __device__ __forceinline__ void init(P b, P hb, P t, P ht) {
    using T = decltype(b.x);
    dx0 = hb;
    dy0 = psub(t, b);
    X = psub(ht, hb);
    dxi[0] = pfma(pbc(T(GA)), X, dx0);
    dxi[1] = pfma(pbc(T(GB)), X, dx0);
    deta[0] = pfma(pbc(T(GA)), X, dy0);
    deta[1] = pfma(pbc(T(GB)), X, dy0);
  }
  // values at (xi_q1, eta_q2) given v0
  __device__ __forceinline__ void values(P v0, P val[2][2]) const {
    using T = decltype(v0.x);
    const P vb0 = pfma(pbc(T(GA)), dx0, v0), vb1 = pfma(pbc(T(GB)), dx0, v0);
    val[0][0] = pfma(pbc(T(GA)), deta[0], vb0);
    val[0][1] = pfma(pbc(T(GB)), deta[0], vb0);
    val[1][0] = pfma(pbc(T(GA)), deta[1], vb1);
    val[1][1] = pfma(pbc(T(GB)), deta[1], vb1);
  }
};

// Test a gradient flux fx (coefficient of dN/dxi), fy (of dN/deta) given per
// Gauss point, with weights wx, wy (nwx = -wx, nwy = -wy), into r[0..3].
//   dN/dxi: N0 -(1-eta), N1 (1-eta), N2 -eta, N3 eta
//   dN/deta: N0 -(1-xi), N1 -xi, N2 (1-xi), N3 xi
template <typename P>
__device__ __forceinline__ void ptest_grad(P sx0, P sx1, P sy0, P sy1, P wx, P wy, P nwx, P nwy, P r[4]) {
  using T = decltype(wx.x);
  const P px = pfma(pbc(T(GA)), sx0, pmul(pbc(T(GB)), sx1));
  const P qx = psub(padd(sx0, sx1), px);
  const P py = pfma(pbc(T(GA)), sy0, pmul(pbc(T(GB)), sy1));
  const P qy = psub(padd(sy0, sy1), py);
  r[0] = pfma(nwx, qx, pfma(nwy, qy, r[0]));
  r[1] = pfma(wx, qx, pfma(nwy, py, r[1]));
  r[2] = pfma(nwx, px, pfma(wy, qy, r[2]));
  r[3] = pfma(wx, px, pfma(wy, py, r[3]));
}

// Test a value f given per Gauss point [q1][q2] against N_A = L_a(xi) L_b(eta), into r[0..3].
template <typename P>
__device__ __forceinline__ void ptest_value(const P fv[2][2], P jxw, P r[4]) {
  using T = decltype(jxw.x);
  const P s0 = padd(fv[0][0], fv[0][1]), s1 = padd(fv[1][0], fv[1][1]);
  const P t0 = pfma(pbc(T(GA)), fv[0][0], pmul(pbc(T(GB)), fv[0][1]));
  const P t1 = pfma(pbc(T(GA)), fv[1][0], pmul(pbc(T(GB)), fv[1][1]));
  const P b0 = psub(s0, t0), b1 = psub(s1, t1);
  const P pb = pfma(pbc(T(GA)), b0, pmul(pbc(T(GB)), b1));
  const P pt = pfma(pbc(T(GA)), t0, pmul(pbc(T(GB)), t1));
  r[0] = pfma(jxw, psub(padd(b0, b1), pb), r[0]);
  r[1] = pfma(jxw, pb, r[1]);
  r[2] = pfma(jxw, psub(padd(t0, t1), pt), r[2]);
  r[3] = pfma(jxw, pt, r[3]);
}

// Two Q1 cells at once (the members of every pair).  b: fields at the cells'
// lower-left nodes (0,0), hb: node (1,0) minus node (0,0); t: fields at the
// upper-left nodes (0,1), ht: node (1,1) minus node (0,1).  out[3*N + c]:
// contribution to node N (0 = (0,0), 1 = (1,0), 2 = (0,1), 3 = (1,1)) of
// component c (0 u_x, 1 u_y, 2 phi), as a pair over the two cells.  ec: the
// cells' moduli E_K (the elastic constants in m are then those of unit E), or 1.
// OP_VJP returns its three per-cell values in out[0..2].
template <typename T, int OP>
__device__ __forceinline__ void q1_cell_pair(const NodePair<T>& b, const NodePair<T>& hb, const NodePair<T>& t,
                                             const NodePair<T>& ht, const MatConst<T>& m, const LevGeom<T>& g,
                                             typename VT<T>::T2 ec, typename VT<T>::T2 out[12]) {
  using N = Needs<OP>;
  using P = typename VT<T>::T2;
  const P zero = pbc(T(0));
  P rux[4] = {zero, zero, zero, zero}, ruy[4] = {zero, zero, zero, zero}, rp[4] = {zero, zero, zero, zero};
  const P ihx = pbc(g.ihx), ihy = pbc(g.ihy);
  const P c2ml = pmul(pbc(m.c2ml), ec), cl = pmul(pbc(m.cl), ec), cm = pmul(pbc(m.cm), ec), omk = pbc(m.omk);
  // ---- linearisation
  PField<P> fux, fuy, fphi, fphit;
  P e11[2], e22[2], uyx[2], uxy[2];
  if (N::linU) {
    fux.init(b.lx, hb.lx, t.lx, ht.lx);
    fuy.init(b.ly, hb.ly, t.ly, ht.ly);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      e11[q] = pmul(fux.dxi[q], ihx);    // du_x/dx at eta_q
      uyx[q] = pmul(fuy.dxi[q], ihx);    // du_y/dx at eta_q
      e22[q] = pmul(fuy.deta[q], ihy);   // du_y/dy at xi_q
      uxy[q] = pmul(fux.deta[q], ihy);   // du_x/dy at xi_q
    }
  }
  P phiq[2][2], phitq[2][2];
  if (N::phi) { fphi.init(b.lz, hb.lz, t.lz, ht.lz); fphi.values(b.lz, phiq); }
  if (N::phit) { fphit.init(b.lw, hb.lw, t.lw, ht.lw); fphit.values(b.lw, phitq); }
  // ---- input
  PField<P> fxu, fxv, fxp;
  P ax[2], dy[2], bxy[2], cyx[2], xpq[2][2];
  if (N::xu) {
    fxu.init(b.x0, hb.x0, t.x0, ht.x0);
    fxv.init(b.x1, hb.x1, t.x1, ht.x1);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      ax[q] = pmul(fxu.dxi[q], ihx);     // d du_x/dx at eta_q
      cyx[q] = pmul(fxv.dxi[q], ihx);    // d du_y/dx at eta_q
      dy[q] = pmul(fxv.deta[q], ihy);    // d du_y/dy at xi_q
      bxy[q] = pmul(fxu.deta[q], ihy);   // d du_x/dy at xi_q
    }
  }
  if (N::xp) { fxp.init(b.xp, hb.xp, t.xp, ht.xp); fxp.values(b.xp, xpq); }
  if (OP == OP_RESID || OP == OP_MASS || OP == OP_TCV) {
    // R = -A(U)(psi), Problem 2 with sigma^+ read as sigma:
    //   A_u(psi)   = (g(phi~) sigma(u), e(psi)) + (phi~^2 p, div psi)
    //   A_phi(psi) = ((1-kappa) phi sigma(u):e(u) + 2 p phi div u - G_c/l (1 - phi), psi)
    //                + G_c l (grad phi, grad psi)
    // MASS: (1, psi);  TCV: (u . grad phi, psi)
    P S11[2][2], S12[2][2], S22[2][2], fv[2][2];
    P uxq[2][2], uyq[2][2];
    if (OP == OP_TCV) { fux.values(b.lx, uxq); fuy.values(b.ly, uyq); }
#pragma unroll
    for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
      for (int q2 = 0; q2 < 2; ++q2) {
        if (OP == OP_MASS) { fv[q1][q2] = pbc(T(1)); continue; }
        if (OP == OP_TCV) {
          // u . grad phi, grad phi from the reference derivatives of phi
          const P gpx = pmul(fphi.dxi[q2], ihx), gpy = pmul(fphi.deta[q1], ihy);
          fv[q1][q2] = pfma(uxq[q1][q2], gpx, pmul(uyq[q1][q2], gpy));
          continue;
        }
        const P gq = pfma(omk, pmul(phitq[q1][q2], phitq[q1][q2]), pbc(m.kap));
        const P ge12 = padd(uxy[q1], uyx[q2]);
        const P s11 = pfma(c2ml, e11[q2], pmul(cl, e22[q1]));
        const P s22 = pfma(cl, e11[q2], pmul(c2ml, e22[q1]));
        const P s12 = pmul(cm, ge12);
        const P pt2 = pmul(pbc(m.p), pmul(phitq[q1][q2], phitq[q1][q2]));
        S11[q1][q2] = pfma(gq, s11, pt2);
        S22[q1][q2] = pfma(gq, s22, pt2);
        S12[q1][q2] = pmul(gq, s12);
        const P se = pfma(s11, e11[q2], pfma(s22, e22[q1], pmul(s12, ge12)));
        const P ph = phiq[q1][q2];
        // (1-kappa) phi se + 2 p phi div u - G_c/l (1 - phi)
        const P a1 = pfma(pmul(omk, ph), se, pmul(pmul(pbc(m.p2), ph), padd(e11[q2], e22[q1])));
        fv[q1][q2] = pfma(pbc(m.gcl), psub(ph, pbc(T(1))), a1);
      }
    const P wx = pbc(g.wx), wy = pbc(g.wy), nwx = pbc(-g.wx), nwy = pbc(-g.wy);
    if (OP == OP_RESID) {
      ptest_grad(padd(S11[0][0], S11[1][0]), padd(S11[0][1], S11[1][1]),
                 padd(S12[0][0], S12[0][1]), padd(S12[1][0], S12[1][1]), wx, wy, nwx, nwy, rux);
      ptest_grad(padd(S12[0][0], S12[1][0]), padd(S12[0][1], S12[1][1]),
                 padd(S22[0][0], S22[0][1]), padd(S22[1][0], S22[1][1]), wx, wy, nwx, nwy, ruy);
      ptest_grad(fphi.dxi[0], fphi.dxi[1], fphi.deta[0], fphi.deta[1], pbc(g.wpx), pbc(g.wpy), pbc(-g.wpx),
                 pbc(-g.wpy), rp);
    }
    {
      const P jxw = pbc(g.jxw);
      const P s0 = padd(fv[0][0], fv[0][1]), s1 = padd(fv[1][0], fv[1][1]);
      const P t0 = pfma(pbc(T(GA)), fv[0][0], pmul(pbc(T(GB)), fv[0][1]));
      const P t1 = pfma(pbc(T(GA)), fv[1][0], pmul(pbc(T(GB)), fv[1][1]));
      const P b0 = psub(s0, t0), b1 = psub(s1, t1);
      const P pb = pfma(pbc(T(GA)), b0, pmul(pbc(T(GB)), b1));
      const P pt = pfma(pbc(T(GA)), t0, pmul(pbc(T(GB)), t1));
      rp[0] = pfma(jxw, psub(padd(b0, b1), pb), rp[0]);
      rp[1] = pfma(jxw, pb, rp[1]);
      rp[2] = pfma(jxw, psub(padd(t0, t1), pt), rp[2]);
      rp[3] = pfma(jxw, pt, rp[3]);
    }
    if (OP == OP_RESID) {
      const P neg = pbc(T(-1));
#pragma unroll
      for (int A = 0; A < 4; ++A) { rux[A] = pmul(rux[A], neg); ruy[A] = pmul(ruy[A], neg); rp[A] = pmul(rp[A], neg); }
    }
  } else if (OP == OP_TCV_GRAD) {
    // J = integral of u . grad phi:  dJ/du_(A,i) = (dphi/dx_i, N_A),  dJ/dphi_A = (u, grad N_A)
    P uxq[2][2], uyq[2][2], gpx[2][2], gpy[2][2];
    fux.values(b.lx, uxq);
    fuy.values(b.ly, uyq);
#pragma unroll
    for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
      for (int q2 = 0; q2 < 2; ++q2) {
        gpx[q1][q2] = pmul(fphi.dxi[q2], ihx);
        gpy[q1][q2] = pmul(fphi.deta[q1], ihy);
      }
    const P jxw = pbc(g.jxw);
    ptest_value(gpx, jxw, rux);
    ptest_value(gpy, jxw, ruy);
    ptest_grad(padd(uxq[0][0], uxq[1][0]), padd(uxq[0][1], uxq[1][1]), padd(uyq[0][0], uyq[0][1]),
               padd(uyq[1][0], uyq[1][1]), pbc(g.wx), pbc(g.wy), pbc(-g.wx), pbc(-g.wy), rp);
  } else if (OP == OP_VJP) {
    // x . dR/dtheta per cell (R = -A, Problem 2; x = (w_u, w_phi) after constraints):
    //   E_K: -[(g(phi~) sigma_1(u), e(w_u)) + (1-kappa)(phi sigma_1(u):e(u), w_phi)]_K
    //   p:   -[(phi~^2, div w_u) + 2 (phi div u, w_phi)]_K
    //   G_c: -[-(1/l)(1 - phi, w_phi) + l (grad phi, grad w_phi)]_K
    // sigma_1: stress of unit modulus (m holds unit-E constants for this operator)
    const P uc2ml = pbc(m.c2ml), ucl = pbc(m.cl), ucm = pbc(m.cm);
    const T ihx2 = g.ihx * g.ihx, ihy2 = g.ihy * g.ihy;
    P sE = zero, sP = zero, sG = zero;
#pragma unroll
    for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
      for (int q2 = 0; q2 < 2; ++q2) {
        const P pt2 = pmul(phitq[q1][q2], phitq[q1][q2]);
        const P gq = pfma(omk, pt2, pbc(m.kap));
        const P ge12 = padd(uxy[q1], uyx[q2]);
        const P s11 = pfma(uc2ml, e11[q2], pmul(ucl, e22[q1]));
        const P s22 = pfma(ucl, e11[q2], pmul(uc2ml, e22[q1]));
        const P s12 = pmul(ucm, ge12);
        const P se = pfma(s11, e11[q2], pfma(s22, e22[q1], pmul(s12, ge12)));
        const P bc = padd(bxy[q1], cyx[q2]);
        const P sw = pfma(s11, ax[q2], pfma(s22, dy[q1], pmul(s12, bc)));
        const P ph = phiq[q1][q2], wp = xpq[q1][q2];
        sE = padd(sE, pfma(gq, sw, pmul(pmul(omk, ph), pmul(se, wp))));
        sP = padd(sP, pfma(pt2, padd(ax[q2], dy[q1]), pmul(padd(ph, ph), pmul(padd(e11[q2], e22[q1]), wp))));
        const P gg = pfma(pmul(fphi.dxi[q2], fxp.dxi[q2]), pbc(ihx2),
                          pmul(pmul(fphi.deta[q1], fxp.deta[q1]), pbc(ihy2)));
        sG = padd(sG, pfma(pbc(m.l), gg, pmul(pbc(-m.il), pmul(psub(pbc(T(1)), ph), wp))));
      }
    const P njxw = pbc(-g.jxw);
    rux[0] = pmul(njxw, sE);
    ruy[0] = pmul(njxw, sP);
    rp[0] = pmul(njxw, sG);
  } else if (OP == OP_PHIT_VJP) {
    // (dA/dphi~)^T x: value test of 2 phi~ [(1-kappa) sigma(u):e(x_u) + p div x_u]
    P fv[2][2];
#pragma unroll
    for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
      for (int q2 = 0; q2 < 2; ++q2) {
        const P ge12 = padd(uxy[q1], uyx[q2]);
        const P s11 = pfma(c2ml, e11[q2], pmul(cl, e22[q1]));
        const P s22 = pfma(cl, e11[q2], pmul(c2ml, e22[q1]));
        const P s12 = pmul(cm, ge12);
        const P sw = pfma(s11, ax[q2], pfma(s22, dy[q1], pmul(s12, padd(bxy[q1], cyx[q2]))));
        const P pt = phitq[q1][q2];
        fv[q1][q2] = pmul(padd(pt, pt), pfma(omk, sw, pmul(pbc(m.p), padd(ax[q2], dy[q1]))));
      }
    ptest_value(fv, pbc(g.jxw), rp);
  } else if (OP == OP_UU_DIAG || OP == OP_PP_DIAG) {
#pragma unroll
    for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
      for (int q2 = 0; q2 < 2; ++q2) {
        const T xi = q1 ? T(GB) : T(GA), eta = q2 ? T(GB) : T(GA);
        const T dxs[4] = {-(1 - eta), (1 - eta), -eta, eta};
        const T dys[4] = {-(1 - xi), -xi, (1 - xi), xi};
        const T Ns[4] = {(1 - xi) * (1 - eta), xi * (1 - eta), (1 - xi) * eta, xi * eta};
        if (OP == OP_UU_DIAG) {
          const P gq = pfma(omk, pmul(phitq[q1][q2], phitq[q1][q2]), pbc(m.kap));
          const P jg = pmul(pmul(pbc(g.jxw), gq), ec);
#pragma unroll
          for (int A = 0; A < 4; ++A) {
            const T dx = dxs[A] * g.ihx, dyy = dys[A] * g.ihy;
            rux[A] = pfma(jg, pbc(m.c2ml * dx * dx + m.cm * dyy * dyy), rux[A]);
            ruy[A] = pfma(jg, pbc(m.cm * dx * dx + m.c2ml * dyy * dyy), ruy[A]);
          }
        } else {
          const P ge12 = padd(uxy[q1], uyx[q2]);
          const P s11 = pfma(c2ml, e11[q2], pmul(cl, e22[q1]));
          const P s22 = pfma(cl, e11[q2], pmul(c2ml, e22[q1]));
          const P s12 = pmul(cm, ge12);
          const P se = pfma(s11, e11[q2], pfma(s22, e22[q1], pmul(s12, ge12)));
          const P mq = pfma(omk, se, pfma(pbc(m.p2), padd(e11[q2], e22[q1]), pbc(m.gcl)));
#pragma unroll
          for (int A = 0; A < 4; ++A) {
            const T dx = dxs[A] * g.ihx, dyy = dys[A] * g.ihy;
            rp[A] = padd(rp[A], pmul(pbc(g.jxw), pfma(mq, pbc(Ns[A] * Ns[A]), pbc(m.gcL * (dx * dx + dyy * dyy)))));
          }
        }
      }
  } else {
    P S11[2][2], S12[2][2], S22[2][2], fv[2][2];
    // q = (1-kappa) sigma(u) + p I, so that the phi rows' coefficients are
    //   (1-kappa) sigma(u):e(u) + 2 p div u + G_c/l = q : e(u) + p div u + G_c/l,
    //   2 phi ((1-kappa) sigma(u) + p I) = 2 phi q
    P oc2ml = zero, ocl = zero, ocm = zero;
    if (N::linU) { oc2ml = pmul(omk, c2ml); ocl = pmul(omk, cl); ocm = pmul(omk, cm); }
#pragma unroll
    for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
      for (int q2 = 0; q2 < 2; ++q2) {
        P gq = zero, T11 = zero, T22 = zero, T12 = zero, mq = zero;
        if (N::phit) gq = pfma(omk, pmul(phitq[q1][q2], phitq[q1][q2]), pbc(m.kap));
        if (N::linU) {
          const P pp = pbc(m.p);
          const P ge12 = padd(uxy[q1], uyx[q2]);   // 2 e12
          const P q11 = pfma(oc2ml, e11[q2], pfma(ocl, e22[q1], pp));
          const P q22 = pfma(ocl, e11[q2], pfma(oc2ml, e22[q1], pp));
          const P q12 = pmul(ocm, ge12);
          mq = pfma(q11, e11[q2], pfma(q22, e22[q1], pfma(q12, ge12, pfma(pp, padd(e11[q2], e22[q1]), pbc(m.gcl)))));
          if (N::phi) {
            const P tp = padd(phiq[q1][q2], phiq[q1][q2]);
            T11 = pmul(tp, q11);
            T22 = pmul(tp, q22);
            T12 = pmul(tp, q12);
          }
        }
        if (N::xu) {
          const P bc = padd(bxy[q1], cyx[q2]);
          P s11 = pmul(gq, pfma(c2ml, ax[q2], pmul(cl, dy[q1])));
          P s22 = pmul(gq, pfma(cl, ax[q2], pmul(c2ml, dy[q1])));
          P s12 = pmul(gq, pmul(cm, bc));
          if (OP == OP_FULL_T) {
            s11 = pfma(xpq[q1][q2], T11, s11);
            s22 = pfma(xpq[q1][q2], T22, s22);
            s12 = pfma(xpq[q1][q2], T12, s12);
          }
          S11[q1][q2] = s11; S12[q1][q2] = s12; S22[q1][q2] = s22;
          if (OP == OP_FULL) fv[q1][q2] = pfma(T11, ax[q2], pfma(T22, dy[q1], pfma(T12, bc, pmul(mq, xpq[q1][q2]))));
        }
        if (N::xp && OP != OP_FULL) fv[q1][q2] = pmul(mq, xpq[q1][q2]);
      }
    const P wx = pbc(g.wx), wy = pbc(g.wy), nwx = pbc(-g.wx), nwy = pbc(-g.wy);
    if (N::xu) {
      // u_x test: (S11, S12) . grad psi;  u_y test: (S12, S22) . grad psi
      ptest_grad(padd(S11[0][0], S11[1][0]), padd(S11[0][1], S11[1][1]),
                 padd(S12[0][0], S12[0][1]), padd(S12[1][0], S12[1][1]), wx, wy, nwx, nwy, rux);
      ptest_grad(padd(S12[0][0], S12[1][0]), padd(S12[0][1], S12[1][1]),
                 padd(S22[0][0], S22[0][1]), padd(S22[1][0], S22[1][1]), wx, wy, nwx, nwy, ruy);
    }
    if (N::xp) {
      // value test against N_A = L_a(xi) L_b(eta)
      const P jxw = pbc(g.jxw);
      const P s0 = padd(fv[0][0], fv[0][1]), s1 = padd(fv[1][0], fv[1][1]);
      const P t0 = pfma(pbc(T(GA)), fv[0][0], pmul(pbc(T(GB)), fv[0][1]));
      const P t1 = pfma(pbc(T(GA)), fv[1][0], pmul(pbc(T(GB)), fv[1][1]));
      const P b0 = psub(s0, t0), b1 = psub(s1, t1);
      const P pb = pfma(pbc(T(GA)), b0, pmul(pbc(T(GB)), b1));
      const P pt = pfma(pbc(T(GA)), t0, pmul(pbc(T(GB)), t1));
      rp[0] = pfma(jxw, psub(padd(b0, b1), pb), rp[0]);
      rp[1] = pfma(jxw, pb, rp[1]);
      rp[2] = pfma(jxw, psub(padd(t0, t1), pt), rp[2]);
      rp[3] = pfma(jxw, pt, rp[3]);
      // G_c l (grad dphi, grad psi): the reference d/dxi flux is the same at both
      // xi points, the d/deta flux at both eta points (factor 2 is in wpx, wpy)
      ptest_grad(fxp.dxi[0], fxp.dxi[1], fxp.deta[0], fxp.deta[1], pbc(g.wpx), pbc(g.wpy), pbc(-g.wpx),
                 pbc(-g.wpy), rp);
    }
  }
#pragma unroll
  for (int A = 0; A < 4; ++A) {
    out[3 * A + 0] = rux[A];
    out[3 * A + 1] = ruy[A];
    out[3 * A + 2] = rp[A];
  }
}

template <typename T> __device__ __forceinline__ const MatConst<T>& matc(const ApplyArgs& a);
template <> __device__ __forceinline__ const MatConst<float>& matc<float>(const ApplyArgs& a) { return a.mf; }
template <> __device__ __forceinline__ const MatConst<double>& matc<double>(const ApplyArgs& a) { return a.md; }
template <typename T> __device__ __forceinline__ LevGeom<T> geom(const ApplyArgs& a, int level);
template <> __device__ __forceinline__ LevGeom<float> geom<float>(const ApplyArgs& a, int level) { return a.gf[level]; }
template <> __device__ __forceinline__ LevGeom<double> geom<double>(const ApplyArgs& a, int level) { return a.gd[level]; }

// Node fields of the cell loops.
enum Field : int { F_XU = 0, F_XV = 1, F_XP = 2, F_LU = 3, F_LV = 4, F_LP = 5, F_LT = 6, NF = 7 };

template <int OP>
__device__ __forceinline__ constexpr bool field_used(int f) {
  using N = Needs<OP>;
  return f == F_XU || f == F_XV ? N::xu : f == F_XP ? N::xp : f == F_LU || f == F_LV ? N::linU
         : f == F_LP ? N::phi : N::phit;
}

template <typename T>
__device__ __forceinline__ const T* field_ptr(const ApplyArgs& a, int f) {
  const T* xu = reinterpret_cast<const T*>(a.xu);
  const T* lin = reinterpret_cast<const T*>(a.lin);
  switch (f) {
    case F_XU: return xu;
    case F_XV: return xu + a.n_slots;
    case F_XP: return reinterpret_cast<const T*>(a.xp);
    default: return lin + (f - F_LU) * a.n_slots;
  }
}

// Final write of owned node (n, c) of an irregular brick: storage action,
// partial sum, constraint rows.
template <typename T, int OP>
__device__ __forceinline__ void write_node(const ApplyArgs& a, int irr, int own_base, int n, int c, uint8_t cm,
                                           T y0, T y1, T y2) {
  constexpr bool outU = (OP != OP_PP && OP != OP_PP_DIAG && OP != OP_MASS && OP != OP_TCV && OP != OP_PHIT_VJP);
  constexpr bool outP = (OP != OP_UU && OP != OP_UU_DIAG);
  constexpr bool isDiag = (OP == OP_UU_DIAG || OP == OP_PP_DIAG);
  T* yu = reinterpret_cast<T*>(a.yu);
  T* yv = yu + a.n_slots;
  T* yp = reinterpret_cast<T*>(a.yp);
  const int o = n + NB * c;
  int act_s = kActFinal, part = -1;
  if (irr >= 0) {
    act_s = __ldg(a.lay.own_act + irr * (NB * NB) + o);
    part = __ldg(a.lay.own_part + irr * (NB * NB) + o);
  }
  const int slot = own_base + o;
  if (part >= 0) {
    T* ib = reinterpret_cast<T*>(a.ibuf) + 3 * int64_t(part);
    ib[0] = y0; ib[1] = y1; ib[2] = y2;
  }
  if (act_s == kActFinal) {
    if (isDiag) {
      if (cm & 1) y0 = T(0);
      if (cm & 2) y1 = T(0);
      if (cm & 4) y2 = T(0);
    } else if (cm) {
      const bool ident = (a.mode & MODE_IDENTITY) != 0;
      const T* xu = reinterpret_cast<const T*>(a.xu);
      if (cm & 1) y0 = ident ? ldg(xu + slot) : T(0);
      if (cm & 2) y1 = ident ? ldg(xu + a.n_slots + slot) : T(0);
      if (cm & 4) y2 = ident ? ldg(reinterpret_cast<const T*>(a.xp) + slot) : T(0);
    }
    if (outU) { yu[slot] = y0; yv[slot] = y1; }
    if (outP) yp[slot] = y2;
  } else if (act_s == kActZero) {
    if (outU) { yu[slot] = T(0); yv[slot] = T(0); }
    if (outP) yp[slot] = T(0);
  }
}

// ---- column sweep (the Q1 cell loop) ---------------------------------------
//
// One warp takes a strip of 2 SH owned node rows r0 .. r0 + 2 SH - 1 of a brick.
// Lane L holds window node column n = L - 1 (-1..30) and evaluates the cell to
// its right.  The strip's two halves (owned rows r0 .. r0+SH-1 and r0+SH ..
// r0+2SH-1) are swept upwards side by side, one cell row each per step: they are
// the two members of every packed operation.  A half needs SH + 1 cell rows (its
// own and the one below), so a step reads one new node row per half.  The right
// neighbour's node values are read from the ring; the contributions of the left
// neighbour's cell come by shuffle, those of the cell row below as a carry in
// registers.  Each owned node is completed once, by its own lane, in the fixed
// order ((carry + left lower-right) + own lower-left); the carry is (own
// upper-left + left upper-right).
// Node rows stream HBM -> shared memory through a per-warp cp.async ring,
// SW_DEPTH - 1 rows ahead of the arithmetic; each lane copies its own column,
// and __syncwarp orders its in-place masking before its left neighbour reads it.

// One warp per block: the block scheduler then fills each SM's free warp slots
// one unit at a time, which evens out the mix of long and short units per SM.
#ifndef PFF_SW_WARPS
#define PFF_SW_WARPS 1
#endif
// Resident one-warp blocks per SM the compiler must allow (the register cap):
// 16 (128 registers) for the FP32 leaf Jacobian, which fits them; 12 for the
// other FP32 operators, which would spill under that cap; 8 in FP64.  A 3-stage ring keeps 16 warps within the
// shared memory of an SM.
#ifndef PFF_SW_MINB_LEAF
#define PFF_SW_MINB_LEAF 16
#endif
#ifndef PFF_SW_MINB
#define PFF_SW_MINB 12
#endif
#ifndef PFF_SW_MINB64
#define PFF_SW_MINB64 8
#endif
#ifndef PFF_SW_DEPTH
#define PFF_SW_DEPTH 3
#endif
#ifndef PFF_SW_UNROLL
#define PFF_SW_UNROLL 2
#endif
constexpr int SW_WARPS = PFF_SW_WARPS;   // warps (strips) per block
constexpr int SW_DEPTH = PFF_SW_DEPTH;   // ring stages per warp
constexpr int SW_UNROLL = PFF_SW_UNROLL; // unrolled steps of the sweep loop
template <typename T, int OP>
constexpr int sw_min_blocks() {
  return sizeof(T) == 8 ? PFF_SW_MINB64 : (OP == OP_FULL || OP == OP_FULL_T) ? PFF_SW_MINB_LEAF : PFF_SW_MINB;
}

// ---- asynchronous global -> shared copies (cp.async), per lane
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src));
}
template <typename T>
__device__ __forceinline__ void cp_one(T* dst, const T* src) {
  if constexpr (sizeof(T) == 4) cp_async4(dst, src); else cp_async8(dst, src);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K)); }

// One node row of both halves in flight.  Every entry is a pair over the two
// halves (lower half in .x, upper half in .y), so that a lane reads the pair of
// its own node, and the pair of its right neighbour, with one shared load each.
// Per lane: node fields (entry 32 pads the right-neighbour read of the last
// lane), storage codes, the aligned constraint-mask words holding each node's
// byte, the modulus of the cell whose lower-left node this is, and (irregular
// bricks) the owned node's word (partial-sum slot + 1) | storage action << 30.
template <typename T>
struct __align__(16) SweepStage {
  typename VT<T>::T2 f[NF][33];
  typename VT<T>::T2 e[32];
  int2 code[32];
  uint2 cm[32];
  int2 own[32];
};

template <typename T>
__device__ __forceinline__ T& half_of(typename VT<T>::T2& p, int h) { return h ? p.y : p.x; }
__device__ __forceinline__ int32_t& half_of_i(int2& p, int h) { return h ? p.y : p.x; }
__device__ __forceinline__ uint32_t& half_of_u(uint2& p, int h) { return h ? p.y : p.x; }

// Issue the copies of the lane's node of half h.  A stored node (code >= 0)
// copies its fields and constraint word from its slot.  A hanging node (code
// <= -2, table entry -2 - code) copies its linearisation from a.hlin and its
// input C x from a.hang_x (written by hang_x_kernel, the launch this one may
// depend on), both indexed by the entry; without a.hlin the linearisation comes
// from the node's own slot (resolved there by set_lin).  Absent nodes are zero.
// Hanging and absent nodes carry no constraint of their own.
template <typename T, int OP>
__device__ __forceinline__ void issue_node(const ApplyArgs& a, int32_t code, SweepStage<T>& st, int h, int lane) {
  using N = Needs<OP>;
  if (code >= 0) {
#pragma unroll
    for (int f = 0; f < NF; ++f)
      if (field_used<OP>(f)) cp_one(&half_of<T>(st.f[f][lane], h), field_ptr<T>(a, f) + code);
    cp_async4(&half_of_u(st.cm[lane], h), reinterpret_cast<const uint32_t*>(a.cmask + (code & ~3)));
    return;
  }
  half_of_u(st.cm[lane], h) = 0u;
  if (code == kAbsent) {
#pragma unroll
    for (int f = 0; f < NF; ++f)
      if (field_used<OP>(f)) half_of<T>(st.f[f][lane], h) = T(0);
    return;
  }
  const int hi = -2 - code;
  if (a.hlin != nullptr) {
    const T* hl = reinterpret_cast<const T*>(a.hlin);
#pragma unroll
    for (int f = F_LU; f < NF; ++f)
      if (field_used<OP>(f)) cp_one(&half_of<T>(st.f[f][lane], h), hl + (f - F_LU) * int64_t(a.nhang) + hi);
  } else {
    const int slot = __ldg(&a.hang[hi].slot);
#pragma unroll
    for (int f = F_LU; f < NF; ++f)
      if (field_used<OP>(f)) cp_one(&half_of<T>(st.f[f][lane], h), field_ptr<T>(a, f) + slot);
  }
  if (N::xu || N::xp) {
    pdl_wait();
    const T* hx = reinterpret_cast<const T*>(a.hang_x);
#pragma unroll
    for (int f = F_XU; f <= F_XP; ++f)
      if (field_used<OP>(f)) cp_one(&half_of<T>(st.f[f][lane], h), hx + f * int64_t(a.nhang) + hi);
  }
}

// Constraint bytes (lower, upper half) of the lane's node in a landed stage.
template <typename T>
__device__ __forceinline__ uint2 node_cm(const SweepStage<T>& st, int lane) {
  const int2 k = st.code[lane];
  const uint2 w = st.cm[lane];
  return make_uint2((w.x >> (8 * (k.x & 3))) & 0xffu, (w.y >> (8 * (k.y & 3))) & 0xffu);
}

// Zero the fixed input components of the lane's node in a landed stage
// (MODE_MASK_INPUT), so that the node and its left neighbour read masked values.
template <typename T, int OP>
__device__ __forceinline__ void mask_node(SweepStage<T>& st, int lane, uint2 cm) {
  using N = Needs<OP>;
  if ((cm.x | cm.y) & 7u) {
    if (N::xu) {
      if (cm.x & 1) st.f[F_XU][lane].x = 0;
      if (cm.y & 1) st.f[F_XU][lane].y = 0;
      if (cm.x & 2) st.f[F_XV][lane].x = 0;
      if (cm.y & 2) st.f[F_XV][lane].y = 0;
    }
    if (N::xp) {
      if (cm.x & 4) st.f[F_XP][lane].x = 0;
      if (cm.y & 4) st.f[F_XP][lane].y = 0;
    }
  }
}

// A node row of both halves as pairs: own values o and (right neighbour - own) h.
template <typename T, int OP>
__device__ __forceinline__ void load_row(const SweepStage<T>& st, int lane, NodePair<T>& o, NodePair<T>& h) {
  using P = typename VT<T>::T2;
  P* po[NF] = {&o.x0, &o.x1, &o.xp, &o.lx, &o.ly, &o.lz, &o.lw};
  P* ph[NF] = {&h.x0, &h.x1, &h.xp, &h.lx, &h.ly, &h.lz, &h.lw};
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    if (field_used<OP>(f)) {
      const P v = st.f[f][lane];
      *po[f] = v;
      *ph[f] = psub(st.f[f][lane + 1], v);
    } else {
      *po[f] = pbc(T(0));
      *ph[f] = pbc(T(0));
    }
  }
}

// Store of an owned node after the cell loop when it is constrained or lies in
// an irregular brick: storage action (final value, zero, or none: another
// level's or the fix-up's), partial sum, constraint rows (identity: y = the
// original x of the node, read back from the input vectors).  Predicated rather
// than branched: the lanes of a row take different actions.
template <typename T, int OP>
__device__ __forceinline__ void store_owned(const ApplyArgs& a, int slot, int act_s, int part, uint8_t cm, T y0, T y1,
                                            T y2) {
  constexpr bool outU = (OP != OP_PP && OP != OP_PP_DIAG && OP != OP_MASS && OP != OP_TCV && OP != OP_PHIT_VJP);
  constexpr bool outP = (OP != OP_UU && OP != OP_UU_DIAG);
  constexpr bool isDiag = (OP == OP_UU_DIAG || OP == OP_PP_DIAG);
  if (part >= 0) {
    T* ib = reinterpret_cast<T*>(a.ibuf) + 3 * int64_t(part);
    ib[0] = y0; ib[1] = y1; ib[2] = y2;
  }
  if (act_s == kActNone) return;
  if (act_s == kActZero) {
    y0 = y1 = y2 = T(0);
  } else if (cm) {
    const bool ident = !isDiag && (a.mode & MODE_IDENTITY) != 0;
    const T* xu = reinterpret_cast<const T*>(a.xu);
    if (cm & 1) y0 = ident ? ldg(xu + slot) : T(0);
    if (cm & 2) y1 = ident ? ldg(xu + a.n_slots + slot) : T(0);
    if (cm & 4) y2 = ident ? ldg(reinterpret_cast<const T*>(a.xp) + slot) : T(0);
  }
  T* yu = reinterpret_cast<T*>(a.yu);
  if (outU) { yu[slot] = y0; yu[a.n_slots + slot] = y1; }
  if (outP) reinterpret_cast<T*>(a.yp)[slot] = y2;
}

// Fused Chebyshev store of a level node (OP_UU: components u_x, u_y; OP_PP: phi):
// the value a plain store would write (zero on absent slots and constrained
// components) enters the smoother update of ChebEpi instead of being stored.
// The operands are loaded at the start of the row step that stores the node, so
// their latency overlaps the step's cell arithmetic.
template <typename T, int OP>
struct ChebOps {
  static constexpr int NC = OP == OP_UU ? 2 : 1;
  T x[NC], prev[NC], dinv[NC], rhs[NC], out[NC];
};

template <typename T, int OP>
__device__ __forceinline__ void cheb_load(const ApplyArgs& a, int slot, ChebOps<T, OP>& o) {
  const ChebEpi& ch = a.ch;
  const T* x = reinterpret_cast<const T*>(OP == OP_UU ? a.xu : a.xp);
#pragma unroll
  for (int c = 0; c < ChebOps<T, OP>::NC; ++c) {
    const int64_t i = c * a.n_slots + slot;
    o.dinv[c] = ldg(reinterpret_cast<const T*>(ch.dinv) + i);
    o.rhs[c] = ldg(reinterpret_cast<const T*>(ch.rhs) + i);
    if (ch.mode != CHEB_FIRST_RES) {
      o.x[c] = ldg(x + i);
      o.prev[c] = ldg(reinterpret_cast<const T*>(ch.prev) + i);
    }
    if (ch.mode == CHEB_STEP_ADD) o.out[c] = reinterpret_cast<const T*>(ch.out)[i];
  }
}

template <typename T, int OP>
__device__ __forceinline__ void cheb_store(const ApplyArgs& a, int slot, int act_s, uint8_t cm, T y0, T y1, T y2,
                                           const ChebOps<T, OP>& o) {
  const ChebEpi& ch = a.ch;
  const T ca = sizeof(T) == 4 ? T(ch.af) : T(ch.ad);
  const T cb = sizeof(T) == 4 ? T(ch.bf) : T(ch.bd);
  T* out = reinterpret_cast<T*>(ch.out);
#pragma unroll
  for (int c = 0; c < ChebOps<T, OP>::NC; ++c) {
    const int bit = OP == OP_UU ? (1 << c) : 4;
    const T y = OP == OP_UU ? (c == 0 ? y0 : y1) : y2;
    const T ye = (act_s == kActZero || (cm & bit)) ? T(0) : y;
    const int64_t i = c * a.n_slots + slot;
    if (ch.mode == CHEB_FIRST_RES) {
      const T ri = o.rhs[c] - ye;
      reinterpret_cast<T*>(ch.r)[i] = ri;
      out[i] = cheb_first_of(ca, o.dinv[c], ri);
      reinterpret_cast<T*>(ch.xprev)[i] = T(0);
    } else {
      const T v = cheb_next(o.x[c], o.prev[c], o.dinv[c], o.rhs[c], ye, ca, cb);
      out[i] = ch.mode == CHEB_STEP_ADD ? o.out[c] + v : v;
    }
  }
}

template <typename T, int OP>
__global__ void __launch_bounds__(32 * SW_WARPS, (sw_min_blocks<T, OP>()))
sweep_q1_kernel(const __grid_constant__ ApplyArgs a, const int32_t* __restrict__ units, int32_t nunits) {
  static_assert(SW_DEPTH >= 3, "the ring holds the lower row, the upper row and at least one row in flight");
  using P = typename VT<T>::T2;
  constexpr bool outU = (OP != OP_PP && OP != OP_PP_DIAG && OP != OP_MASS && OP != OP_TCV && OP != OP_PHIT_VJP);
  constexpr bool outP = (OP != OP_UU && OP != OP_UU_DIAG);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const unsigned FULL = 0xffffffffu;
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  SweepStage<T>* ring = reinterpret_cast<SweepStage<T>*>(smem_raw) + (threadIdx.x >> 5) * SW_DEPTH;
  const int unit = blockIdx.x * SW_WARPS + (threadIdx.x >> 5);
  if (unit >= nunits) { pdl_wait(); return; }   // warp-uniform
  // the warp's strip: owned rows r0 .. r0 + 2 SH - 1 of brick bi
  const int32_t uw = __ldg(units + unit);
  const int bi = uw >> 8;
  const int r0 = (uw >> 3) & 31;
  const int SH = (0x0103050f >> (8 * (uw & 3))) & 0xff;   // 15, 5, 3, 1 for codes 0..3
  const int NROW = SH + 2;                             // node rows per half
  const BrickDesc* bd = a.lay.bricks + bi;
  const int irr = __ldg(&bd->irr);
  const LevGeom<T> g = geom<T>(a, __ldg(&bd->level));
  const MatConst<T>& mc = matc<T>(a);
  const bool mask = (a.mode & MODE_MASK_INPUT) != 0;
  const int n = lane - 1;                              // window node column -1..30
  const int dx = n < 0 ? -1 : (n >= NB ? 1 : 0);
  const int col = n - NB * dx;                         // its column in its brick
  const int base_lo = __ldg(bd->nbr_base + dx + 1);    // the column's bricks below, beside, above
  const int base_mid = __ldg(bd->nbr_base + dx + 4);
  const int base_hi = __ldg(bd->nbr_base + dx + 7);
  const int own_base = __ldg(bd->nbr_base + 4);
  const int32_t* win = a.lay.win + (irr >= 0 ? irr : 0) * (WN * WN) + lane;
  // window cell activity of an irregular brick: 31 words, word i held by lane i
  const uint32_t cmw = (irr >= 0 && lane < 31) ? __ldg(a.lay.cellmask + irr * 31 + lane) : 0u;
  T* yu = reinterpret_cast<T*>(a.yu);
  T* yv = yu + a.n_slots;
  T* yp = reinterpret_cast<T*>(a.yp);
  // the right-neighbour pad of every stage reads as zero
  if (lane < NF)
    for (int j = 0; j < SW_DEPTH; ++j) ring[j].f[lane][32] = pbc(T(0));
  // storage code of window node (n, r) of a regular brick, brick row r = -1..30;
  // also the cell slot of cell (n, r) in any brick (its lower-left node position)
  auto reg_code = [&](int r) -> int32_t {
    return r < 0 ? base_lo + col + NB * (r + NB) : (r >= NB ? base_hi + col + NB * (r - NB) : base_mid + col + NB * r);
  };
  // window cell (n, c) is active (all 32 lanes call it: shuffle).  The last
  // lane's cell lies outside the window: its contributions reach only that
  // lane's own (halo) node, so it is never masked.
  auto cell_active = [&](int c) -> bool {
    if (irr < 0) return true;
    const int i = (c + 1) * NCW + (lane < 31 ? lane : 0);
    const uint32_t w = __shfl_sync(FULL, cmw, (i >> 5) & 31);
    return lane == 31 || ((w >> (i & 31)) & 1u);
  };
  // stream of node rows j = 0 .. NROW-1 per half: brick rows r0 - 1 + j (half 0)
  // and r0 + SH - 1 + j (half 1); the codes of irregular bricks are read one row
  // ahead of their copies
  int32_t kn0 = 0, kn1 = 0;
  if (irr >= 0) { kn0 = __ldg(win + WN * r0); kn1 = __ldg(win + WN * (r0 + SH)); }
  auto issue_extra = [&](SweepStage<T>& st, int h, int r) {
    if (a.ecell != nullptr) {
      // modulus of cell (n, r), r <= 29, whose lower-left node this is (the last
      // lane's cell lies outside the window)
      const bool act = r < NB && cell_active(r) && lane < 31;
      if (act) cp_one(&half_of<T>(st.e[lane], h), reinterpret_cast<const T*>(a.ecell) + reg_code(r));
    }
    if (irr >= 0 && r >= 0 && r < NB && lane >= 1 && lane <= NB)
      cp_async4(&half_of_i(st.own[lane], h), a.lay.own + irr * (NB * NB) + n + NB * r);
  };
  auto issue = [&](int j) {
    if (j < NROW) {
      SweepStage<T>& st = ring[j % SW_DEPTH];
      int32_t k0, k1;
      if (irr >= 0) {
        k0 = kn0;
        k1 = kn1;
        if (j + 1 < NROW) { kn0 = __ldg(win + WN * (r0 + j + 1)); kn1 = __ldg(win + WN * (r0 + SH + j + 1)); }
      } else {
        k0 = reg_code(r0 - 1 + j);
        k1 = reg_code(r0 + SH - 1 + j);
      }
      st.code[lane] = make_int2(k0, k1);
      issue_node<T, OP>(a, k0, st, 0, lane);
      issue_node<T, OP>(a, k1, st, 1, lane);
      if (irr >= 0 || a.ecell != nullptr) {
        issue_extra(st, 0, r0 - 1 + j);
        issue_extra(st, 1, r0 + SH - 1 + j);
      }
    }
    cp_async_commit();
  };
  // Ring: row j lives in stage j % SW_DEPTH from its issue until the step that
  // completes it as the lower row; SW_DEPTH - 2 rows are in flight beyond the
  // one being read.  A landed row is first masked by its owners; __syncwarp
  // orders that before the left neighbours read it.
  // Everything above reads tables that no kernel of a chain writes; the input
  // vector is the preceding kernel's output
  if (a.pdl_in) pdl_wait();
#pragma unroll
  for (int j = 0; j < SW_DEPTH - 1; ++j) issue(j);

  cp_async_wait<SW_DEPTH - 2>();
  uint2 cb = node_cm(ring[0], lane);   // constraint bytes of the lower row's nodes
  if (mask) mask_node<T, OP>(ring[0], lane, cb);
  __syncwarp();
  NodePair<T> ob, hb;                // lower node row of the current cell rows
  load_row<T, OP>(ring[0], lane, ob, hb);
  P carry[3] = {pbc(T(0)), pbc(T(0)), pbc(T(0))};
#pragma unroll SW_UNROLL
  for (int s = 0; s <= SH; ++s) {
    cp_async_wait<SW_DEPTH - 3>();
    SweepStage<T>& sb = ring[s % SW_DEPTH];         // lower row: row s
    SweepStage<T>& st = ring[(s + 1) % SW_DEPTH];   // upper row: row s + 1
    const uint2 ct = node_cm(st, lane);
    if (mask) mask_node<T, OP>(st, lane, ct);
    __syncwarp();
    issue(s + SW_DEPTH - 1);         // into the stage of row s - 1, completed at the previous step
    const int c0 = r0 - 1 + s, c1 = c0 + SH;   // cell rows (and completed node rows) of the halves
    const bool owner = s >= 1 && lane >= 1 && lane <= NB;
    ChebOps<T, OP> ch0, ch1;         // fused Chebyshev store: operands of the two nodes this step stores
    if constexpr (OP == OP_UU || OP == OP_PP) {
      if (a.ch.mode != CHEB_OFF && owner) {
        cheb_load<T, OP>(a, own_base + n + NB * c0, ch0);
        cheb_load<T, OP>(a, own_base + n + NB * c1, ch1);
      }
    }
    NodePair<T> ot, ht;              // upper node row
    load_row<T, OP>(st, lane, ot, ht);
    const bool act0 = cell_active(c0), act1 = cell_active(c1);
    const P ec = a.ecell != nullptr ? sb.e[lane] : pbc(T(1));
    P out[12];
    q1_cell_pair<T, OP>(ob, hb, ot, ht, mc, g, ec, out);
    if (!act0 || !act1) {
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        if (!act0) out[q].x = T(0);
        if (!act1) out[q].y = T(0);
      }
    }
    if constexpr (OP == OP_VJP) {
      // per-cell values of the cells this strip owns (lower-left node owned)
      if (owner) {
        T* co = reinterpret_cast<T*>(a.cell_out);
        const int64_t sA = own_base + n + NB * c0, sB = own_base + n + NB * c1;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (act0) co[q * a.n_slots + sA] = out[q].x;
          if (act1) co[q * a.n_slots + sB] = out[q].y;
        }
      }
    } else {
      P brL[3], trL[3];              // the left neighbour's lower-right and upper-right contributions
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        brL[q].x = __shfl_up_sync(FULL, out[3 + q].x, 1);
        brL[q].y = __shfl_up_sync(FULL, out[3 + q].y, 1);
        trL[q].x = __shfl_up_sync(FULL, out[9 + q].x, 1);
        trL[q].y = __shfl_up_sync(FULL, out[9 + q].y, 1);
      }
      if (owner) {
        P y[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) y[q] = padd(padd(carry[q], brL[q]), out[q]);
        const int s0 = own_base + n + NB * c0, s1 = own_base + n + NB * c1;
        // storage action and partial sum of the two nodes (irregular bricks)
        uint32_t w0 = uint32_t(kActFinal) << 30, w1 = w0;
        if (irr >= 0) {
          const int2 ow = sb.own[lane];
          w0 = uint32_t(ow.x);
          w1 = uint32_t(ow.y);
        }
        const bool plain0 = cb.x == 0 && w0 == (uint32_t(kActFinal) << 30);   // final value, no partial, free
        const bool plain1 = cb.y == 0 && w1 == (uint32_t(kActFinal) << 30);
        bool fused = false;
        if constexpr (OP == OP_UU || OP == OP_PP) fused = a.ch.mode != CHEB_OFF;
        if (fused) {
          cheb_store<T, OP>(a, s0, int(w0 >> 30), uint8_t(cb.x), y[0].x, y[1].x, y[2].x, ch0);
          cheb_store<T, OP>(a, s1, int(w1 >> 30), uint8_t(cb.y), y[0].y, y[1].y, y[2].y, ch1);
        } else if (plain0 && plain1) {
          if (outU) { yu[s0] = y[0].x; yv[s0] = y[1].x; yu[s1] = y[0].y; yv[s1] = y[1].y; }
          if (outP) { yp[s0] = y[2].x; yp[s1] = y[2].y; }
        } else {
          store_owned<T, OP>(a, s0, int(w0 >> 30), int(w0 & 0x3fffffffu) - 1, uint8_t(cb.x), y[0].x, y[1].x, y[2].x);
          store_owned<T, OP>(a, s1, int(w1 >> 30), int(w1 & 0x3fffffffu) - 1, uint8_t(cb.y), y[0].y, y[1].y, y[2].y);
        }
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) carry[q] = padd(out[6 + q], trL[q]);
    }
    ob = ot;
    hb = ht;
    cb = ct;
  }
  cp_async_wait<0>();
  pdl_wait();   // the launch this one depends on (if any) completes before this grid does
}

// C x on the hanging nodes (Q1 leaf): hx[f][h] = sum_b w_b x_f(parent_b), the
// parents' fixed components zeroed under MODE_MASK_INPUT.  Runs before the
// sweep, which may start early (programmatic dependent launch) and waits for
// this grid only where it copies these values.
template <typename T>
__global__ void hang_x_kernel(const DevHanging* __restrict__ hang, int32_t nh, int np, const T* __restrict__ xu,
                              const T* __restrict__ xp, int64_t n_slots, const uint8_t* __restrict__ cmask,
                              int mode, T* __restrict__ hx) {
  pdl_trigger();
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= nh) return;
  const bool mask = (mode & MODE_MASK_INPUT) != 0;
  const DevHanging e = hang[h];
  T v0 = 0, v1 = 0, vp = 0;
  for (int b = 0; b < np; ++b) {
    const int ps = e.parent[b];
    const T w = T(e.weight[b]);
    T p0 = __ldg(xu + ps), p1 = __ldg(xu + n_slots + ps), pp = __ldg(xp + ps);
    if (mask) {
      const uint8_t cm = __ldg(cmask + ps);
      if (cm & 1) p0 = 0;
      if (cm & 2) p1 = 0;
      if (cm & 4) pp = 0;
    }
    v0 += w * p0; v1 += w * p1; vp += w * pp;
  }
  hx[h] = v0;
  hx[int64_t(nh) + h] = v1;
  hx[2 * int64_t(nh) + h] = vp;
}

// C^T on the interface nodes: y = sum of the node's partial sums (weights of
// C), then its constraint rows.  Launched programmatically dependent on the
// apply: everything but the partial sums is read before waiting for it.
template <typename T>
__global__ void fixup_kernel(const FixupArgs a) {
  constexpr int PRE = 4;   // partials whose indices and weights are read before the wait
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const bool ident = (a.mode & MODE_IDENTITY) != 0;
  int slot = 0, e0 = 0, e1 = 0;
  uint8_t cm = 0;
  T xi[3] = {T(0), T(0), T(0)};
  int pp[PRE];
  T ww[PRE];
  if (f < a.n) {
    slot = a.slot[f];
    e0 = a.ptr[f];
    e1 = a.ptr[f + 1];
    cm = a.cmask[slot];
    if (cm && ident) {
      const T* xu = reinterpret_cast<const T*>(a.xu);
      xi[0] = xu[slot];
      xi[1] = xu[a.n_slots + slot];
      xi[2] = reinterpret_cast<const T*>(a.xp)[slot];
    }
#pragma unroll
    for (int q = 0; q < PRE; ++q) {
      pp[q] = e0 + q < e1 ? a.part[e0 + q] : 0;
      ww[q] = e0 + q < e1 ? T(a.w[e0 + q]) : T(0);
    }
  }
  pdl_wait();
  if (f >= a.n) return;
  const T* ib = reinterpret_cast<const T*>(a.ibuf);
  T y0 = 0, y1 = 0, y2 = 0;
#pragma unroll
  for (int q = 0; q < PRE; ++q) {
    if (e0 + q < e1) {
      y0 += ww[q] * ib[3 * pp[q] + 0];
      y1 += ww[q] * ib[3 * pp[q] + 1];
      y2 += ww[q] * ib[3 * pp[q] + 2];
    }
  }
  for (int e = e0 + PRE; e < e1; ++e) {
    const int p = a.part[e];
    const T w = T(a.w[e]);
    y0 += w * ib[3 * p + 0];
    y1 += w * ib[3 * p + 1];
    y2 += w * ib[3 * p + 2];
  }
  if (cm) {
    if (cm & 1) y0 = ident ? xi[0] : T(0);
    if (cm & 2) y1 = ident ? xi[1] : T(0);
    if (cm & 4) y2 = ident ? xi[2] : T(0);
  }
  T* yu = reinterpret_cast<T*>(a.yu);
  yu[slot] = y0;
  yu[a.n_slots + slot] = y1;
  reinterpret_cast<T*>(a.yp)[slot] = y2;
}

// lin blocks (u_x, u_y, phi, phi_tilde) in FP64 and FP32 from the state
__global__ void set_lin_kernel(int64_t n, const double* __restrict__ u, const double* __restrict__ phi,
                               const double* __restrict__ phit, double* lin64, float* lin32) {
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double v[4] = {u[s], u[n + s], phi[s], phit[s]};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    lin64[k * n + s] = v[k];
    lin32[k * n + s] = float(v[k]);
  }
}

__global__ void set_lin_hanging_kernel(int32_t nh, int64_t n, const DevHanging* __restrict__ hang, int np,
                                       double* lin64, float* lin32, double* hlin64, float* hlin32) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= nh) return;
  const DevHanging e = hang[h];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double v = 0;
    for (int b = 0; b < np; ++b) v += e.weight[b] * lin64[k * n + e.parent[b]];
    lin64[k * n + e.slot] = v;
    lin32[k * n + e.slot] = float(v);
    if (hlin64) hlin64[k * int64_t(nh) + h] = v;
    if (hlin32) hlin32[k * int64_t(nh) + h] = float(v);
  }
}

}  // namespace

namespace {
template <typename T>
void fill_mat(MatConst<T>& c, const ApplyArgs& a) {
  c.c2ml = T(2.0 * a.mu + a.lam); c.cl = T(a.lam); c.cm = T(a.mu);
  c.omk = T(1.0 - a.kappa); c.kap = T(a.kappa); c.p = T(a.p); c.p2 = T(2.0 * a.p);
  c.gcl = T(a.gc_over_l); c.gcL = T(a.gc_times_l);
  c.il = T(1.0 / a.ell); c.l = T(a.ell);
}
template <typename T>
void fill_geom(LevGeom<T>& c, const ApplyArgs& a, double hx, double hy) {
  c.ihx = T(1.0 / hx); c.ihy = T(1.0 / hy);
  c.jxw = T(0.25 * hx * hy);
  c.wx = T(0.25 * hy); c.wy = T(0.25 * hx);
  c.wpx = T(0.5 * a.gc_times_l * hy / hx); c.wpy = T(0.5 * a.gc_times_l * hx / hy);
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

namespace {
#include "apply_q2.cuh"
}  // namespace

template <typename T>
void fill_q2(Q2Tab<T>& t) {
  // 3-point Gauss rule on [0, 1]
  const double g[3] = {0.5 - 0.1 * std::sqrt(15.0), 0.5, 0.5 + 0.1 * std::sqrt(15.0)};
  const double w[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  for (int q = 0; q < 3; ++q) {
    const double x = g[q];
    // Lagrange basis on the nodes 0, 1/2, 1 and its derivative
    const double L[3] = {2.0 * (x - 0.5) * (x - 1.0), -4.0 * x * (x - 1.0), 2.0 * x * (x - 0.5)};
    const double D[3] = {4.0 * x - 3.0, 4.0 - 8.0 * x, 4.0 * x - 1.0};
    for (int a = 0; a < 3; ++a) {
      t.L[a][q] = T(L[a]);
      t.D[a][q] = T(D[a]);
    }
    t.w[q] = T(w[q]);
  }
}

void fill_cell_constants(ApplyArgs& a, int nlevels) {
  fill_mat(a.mf, a);
  fill_mat(a.md, a);
  fill_q2(a.q2f);
  fill_q2(a.q2d);
  for (int l = 0; l < nlevels && l < kMaxLevels; ++l) {
    fill_geom(a.gf[l], a, a.hx[l], a.hy[l]);
    fill_geom(a.gd[l], a, a.hx[l], a.hy[l]);
  }
}

// Streaming multiprocessors of the current device (cached per device).
int sm_count() {
  static std::mutex mu;
  static std::unordered_map<int, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int sms = 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
  cache[dev] = sms;
  return sms;
}

// Strip half-height of the column sweep: the Jacobian and the level block
// operators come with SH = 15 (one strip per brick: 32 cell rows evaluated per
// 30 owned rows), 5 and 1 (3 and 15 strips per brick: more, shorter warps for
// small level meshes); the other operators with SH = 15.  a.sweep_sh forces one
// of 15, 5, 1 where it exists; 0 picks the largest whose strips give every SM a
// few warps.
// Work units of the Q1 cell loop (one warp each).  A strip of half-height SH
// evaluates 2 (SH + 1) cell rows for its 2 SH owned rows and pays one pipeline
// start; short strips give small meshes enough warps and even out the slower
// irregular bricks.  Schedules: 0 by mesh size: on meshes with at least four
// bricks per SM, regular bricks SH = 15 (one unit) and then irregular bricks
// SH = 5 (three units), so that the blocks of the shorter irregular units fill
// the slots the regular ones leave; on smaller meshes every brick SH = 5 if that
// gives four warps per SM, else SH = 1; 1, 2, 3: every brick SH = 15, 5, 1.
std::vector<int32_t> sweep_units(const std::vector<BrickDesc>& bricks, int32_t unit_off[5]) {
  std::vector<int32_t> u;
  const int nb = int(bricks.size());
  auto add = [&](int b, int code) {
    const int sh = code == 0 ? 15 : code == 1 ? 5 : code == 2 ? 3 : 1;
    for (int r0 = 0; r0 < NB; r0 += 2 * sh) u.push_back(int32_t(b) << 8 | r0 << 3 | code);
  };
  const int64_t want = int64_t(4) * sm_count();
  unit_off[0] = 0;
  if (nb >= want) {
    for (int b = 0; b < nb; ++b)
      if (bricks[b].irr < 0) add(b, 0);
    for (int b = 0; b < nb; ++b)
      if (bricks[b].irr >= 0) add(b, 1);
  } else {
    const int code = 3 * int64_t(nb) >= want ? 1 : 3;
    for (int b = 0; b < nb; ++b) add(b, code);
  }
  unit_off[1] = int32_t(u.size());
  for (int b = 0; b < nb; ++b) add(b, 0);
  unit_off[2] = int32_t(u.size());
  for (int b = 0; b < nb; ++b) add(b, 1);
  unit_off[3] = int32_t(u.size());
  for (int b = 0; b < nb; ++b) add(b, 3);
  unit_off[4] = int32_t(u.size());
  return u;
}

template <typename T, int OP>
cudaError_t launch_sweep(const ApplyArgs& a, cudaStream_t s) {
  using N = Needs<OP>;
  // FP64 is bound by its arithmetic rate: there the least work (one strip per
  // brick) wins over the balanced schedule, except on small meshes
  int sched = a.sweep_sh == 15 ? 1 : a.sweep_sh == 5 ? 2 : a.sweep_sh == 1 ? 3 : 0;
  if (sched == 0 && sizeof(T) == 8 && a.lay.nbricks >= 4 * sm_count()) sched = 1;
  if (a.lay.units == nullptr) return cudaErrorInvalidValue;
  const int32_t* units = a.lay.units + a.lay.unit_off[sched];
  const int32_t nunits = a.lay.unit_off[sched + 1] - a.lay.unit_off[sched];
  if (nunits <= 0) return cudaSuccess;
  // hanging nodes' input: C x into a.hang_x first; the sweep may start before that
  // grid ends and waits for it only where it copies those values
  bool pdl = a.pdl_in != 0;
  if ((N::xu || N::xp) && a.nhang > 0 && a.hang != nullptr) {
    if (a.hang_x == nullptr) return cudaErrorInvalidValue;
    hang_x_kernel<T><<<(a.nhang + 127) / 128, 128, 0, s>>>(
        a.hang, a.nhang, a.fe_degree + 1, reinterpret_cast<const T*>(a.xu), reinterpret_cast<const T*>(a.xp),
        a.n_slots, a.cmask, a.mode, reinterpret_cast<T*>(a.hang_x));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    pdl = true;
  }
  const unsigned blk = 32 * SW_WARPS;
  const size_t smem = sizeof(SweepStage<T>) * SW_DEPTH * SW_WARPS;
  const auto fn = &sweep_q1_kernel<T, OP>;
  resident_blocks(reinterpret_cast<const void*>(fn), int(blk), smem);   // sets the shared-memory limit once
  return launch_ex(pdl, fn, unsigned((nunits + SW_WARPS - 1) / SW_WARPS), blk, smem, s, a, units, nunits);
}

template <typename T>
cudaError_t launch_apply(const ApplyArgs& a, int op, cudaStream_t s) {
  if (a.lay.nbricks <= 0) return cudaSuccess;
  // the fused Chebyshev store exists in the level block operators only
  if (a.ch.mode != CHEB_OFF && op != OP_UU && op != OP_PP) return cudaErrorInvalidValue;
  if (a.fe_degree == 2) return launch_apply_q2<T>(a, op, s);
  if (a.fe_degree != 1) return cudaErrorInvalidValue;
  switch (op) {
    case OP_FULL: return launch_sweep<T, OP_FULL>(a, s);
    case OP_FULL_T: return launch_sweep<T, OP_FULL_T>(a, s);
    case OP_UU: return launch_sweep<T, OP_UU>(a, s);
    case OP_PP: return launch_sweep<T, OP_PP>(a, s);
    case OP_UU_DIAG: return launch_sweep<T, OP_UU_DIAG>(a, s);
    case OP_PP_DIAG: return launch_sweep<T, OP_PP_DIAG>(a, s);
    case OP_RESID: return launch_sweep<T, OP_RESID>(a, s);
    case OP_MASS: return launch_sweep<T, OP_MASS>(a, s);
    case OP_TCV: return launch_sweep<T, OP_TCV>(a, s);
    case OP_TCV_GRAD: return launch_sweep<T, OP_TCV_GRAD>(a, s);
    case OP_VJP: return launch_sweep<T, OP_VJP>(a, s);
    case OP_PHIT_VJP: return launch_sweep<T, OP_PHIT_VJP>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_fixup(const FixupArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  return launch_ex(true, &fixup_kernel<T>, unsigned((a.n + 127) / 128), 128u, 0, s, a);
}

cudaError_t launch_set_lin(int64_t n_slots, const double* u, const double* phi, const double* phit,
                           const DevHanging* hang, int32_t nhang, int fe_degree,
                           double* lin64, float* lin32, double* hlin64, float* hlin32, cudaStream_t s) {
  if (n_slots > 0)
    set_lin_kernel<<<unsigned((n_slots + 255) / 256), 256, 0, s>>>(n_slots, u, phi, phit, lin64, lin32);
  if (nhang > 0)
    set_lin_hanging_kernel<<<(nhang + 127) / 128, 128, 0, s>>>(nhang, n_slots, hang, fe_degree + 1, lin64, lin32,
                                                               hlin64, hlin32);
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
