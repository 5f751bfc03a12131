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
// Execution: "row sweeps" over strips of RSEG node rows of a brick of 30x30
// owned node slots.  A half-warp (16 lanes) covers the 32 window columns
// -1..30; lane l holds columns 2l-1 and 2l and evaluates the two cells to
// their right as one packed pair: every sum-factorised 2x2 Gauss operation of
// the two cells is one paired FP32 instruction (FFMA2 / FADD2 / FMUL2).
// Node rows stream HBM -> shared memory through a per-half-warp cp.async ring
// several rows ahead of the arithmetic.  Neighbouring lanes exchange node
// values and nodal contributions with shuffles; there is no block barrier.
// Input x has its hanging-node constraints resolved on the fly and fixed
// components masked.  Each owned node is written once, by one lane, in a
// fixed summation order.  Nodes shared with another level, hanging nodes and
// their parents write partial sums; a small fix-up kernel condenses them
// (x_full = C x on input, C^T y on output).  No atomics.
#include "kernels.cuh"

#include <cmath>
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
#define PFF_RSEG 3
#endif
#ifndef PFF_WARPS
#define PFF_WARPS 4
#endif
#ifndef PFF_MINB
#define PFF_MINB 4
#endif
#ifndef PFF_MINB64
#define PFF_MINB64 2
#endif
#ifndef PFF_DEPTH
#define PFF_DEPTH 4
#endif
constexpr int RSEG = PFF_RSEG;    // node rows per half-warp strip
constexpr int NSEG = NB / RSEG;   // strips per brick
constexpr int WARPS = PFF_WARPS;  // warps per CTA; a half-warp sweeps one strip per round
constexpr int DEPTH = PFF_DEPTH;  // ring stages (rows in flight: DEPTH-1)
constexpr int NROWS = RSEG + 2;   // node rows a strip reads
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

// ---- packed pairs (cell A, cell B).  FP32: Blackwell paired instructions.
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
  __device__ __forceinline__ void init(P v0, P v1, P v2, P v3) {
    using T = decltype(v0.x);
    dx0 = psub(v1, v0);
    dy0 = psub(v2, v0);
    X = psub(psub(v3, v2), dx0);
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

// Two Q1 cells at once.  v[0] = nodes (0,0) of cells A and B, v[1] = (1,0),
// v[2] = (0,1), v[3] = (1,1).  out[3*N + c]: contribution to node N of
// component c (0 u_x, 1 u_y, 2 phi), as a pair over the two cells.  ec: the
// cells' moduli E_K (the elastic constants in m are then those of unit E), or 1.
// OP_VJP returns its three per-cell values in out[0..2].
template <typename T, int OP>
__device__ __forceinline__ void q1_cell_pair(const NodePair<T> v[4], const MatConst<T>& m, const LevGeom<T>& g,
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
    fux.init(v[0].lx, v[1].lx, v[2].lx, v[3].lx);
    fuy.init(v[0].ly, v[1].ly, v[2].ly, v[3].ly);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      e11[q] = pmul(fux.dxi[q], ihx);    // du_x/dx at eta_q
      uyx[q] = pmul(fuy.dxi[q], ihx);    // du_y/dx at eta_q
      e22[q] = pmul(fuy.deta[q], ihy);   // du_y/dy at xi_q
      uxy[q] = pmul(fux.deta[q], ihy);   // du_x/dy at xi_q
    }
  }
  P phiq[2][2], phitq[2][2];
  if (N::phi) { fphi.init(v[0].lz, v[1].lz, v[2].lz, v[3].lz); fphi.values(v[0].lz, phiq); }
  if (N::phit) { fphit.init(v[0].lw, v[1].lw, v[2].lw, v[3].lw); fphit.values(v[0].lw, phitq); }
  // ---- input
  PField<P> fxu, fxv, fxp;
  P ax[2], dy[2], bxy[2], cyx[2], xpq[2][2];
  if (N::xu) {
    fxu.init(v[0].x0, v[1].x0, v[2].x0, v[3].x0);
    fxv.init(v[0].x1, v[1].x1, v[2].x1, v[3].x1);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      ax[q] = pmul(fxu.dxi[q], ihx);     // d du_x/dx at eta_q
      cyx[q] = pmul(fxv.dxi[q], ihx);    // d du_y/dx at eta_q
      dy[q] = pmul(fxv.deta[q], ihy);    // d du_y/dy at xi_q
      bxy[q] = pmul(fxu.deta[q], ihy);   // d du_x/dy at xi_q
    }
  }
  if (N::xp) { fxp.init(v[0].xp, v[1].xp, v[2].xp, v[3].xp); fxp.values(v[0].xp, xpq); }
  if (OP == OP_RESID || OP == OP_MASS || OP == OP_TCV) {
    // R = -A(U)(psi), Problem 2 with sigma^+ read as sigma:
    //   A_u(psi)   = (g(phi~) sigma(u), e(psi)) + (phi~^2 p, div psi)
    //   A_phi(psi) = ((1-kappa) phi sigma(u):e(u) + 2 p phi div u - G_c/l (1 - phi), psi)
    //                + G_c l (grad phi, grad psi)
    // MASS: (1, psi);  TCV: (u . grad phi, psi)
    P S11[2][2], S12[2][2], S22[2][2], fv[2][2];
    P uxq[2][2], uyq[2][2];
    if (OP == OP_TCV) { fux.values(v[0].lx, uxq); fuy.values(v[0].ly, uyq); }
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
    fux.values(v[0].lx, uxq);
    fuy.values(v[0].ly, uyq);
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
#pragma unroll
    for (int q1 = 0; q1 < 2; ++q1)
#pragma unroll
      for (int q2 = 0; q2 < 2; ++q2) {
        P gq = zero, T11 = zero, T22 = zero, T12 = zero, mq = zero;
        if (N::phit) gq = pfma(omk, pmul(phitq[q1][q2], phitq[q1][q2]), pbc(m.kap));
        if (N::linU) {
          const P ge12 = padd(uxy[q1], uyx[q2]);   // 2 e12
          const P s11 = pfma(c2ml, e11[q2], pmul(cl, e22[q1]));
          const P s22 = pfma(cl, e11[q2], pmul(c2ml, e22[q1]));
          const P s12 = pmul(cm, ge12);
          const P se = pfma(s11, e11[q2], pfma(s22, e22[q1], pmul(s12, ge12)));
          mq = pfma(omk, se, pfma(pbc(m.p2), padd(e11[q2], e22[q1]), pbc(m.gcl)));
          if (N::phi) {
            const P tp = padd(phiq[q1][q2], phiq[q1][q2]);
            T11 = pmul(tp, pfma(omk, s11, pbc(m.p)));
            T22 = pmul(tp, pfma(omk, s22, pbc(m.p)));
            T12 = pmul(tp, pmul(omk, s12));
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

// ---- asynchronous global -> shared copies (cp.async), per lane
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src));
}
// copies of one value / one adjacent pair of values of type T
template <typename T>
__device__ __forceinline__ void cp_one(T* dst, const T* src) {
  if constexpr (sizeof(T) == 4) cp_async4(dst, src); else cp_async8(dst, src);
}
template <typename T>
__device__ __forceinline__ void cp_pair(T* dst, const T* src) {
  if constexpr (sizeof(T) == 4) cp_async8(dst, src); else cp_async16(dst, src);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K)); }

// Node fields in a ring stage (structure of arrays over the 32 columns of a
// half-warp; lane l holds columns 2l, 2l+1, so its pair is one aligned load).
enum Field : int { F_XU = 0, F_XV = 1, F_XP = 2, F_LU = 3, F_LV = 4, F_LP = 5, F_LT = 6, NF = 7 };

template <int OP>
__device__ __forceinline__ constexpr bool field_used(int f) {
  using N = Needs<OP>;
  return f == F_XU || f == F_XV ? N::xu : f == F_XP ? N::xp : f == F_LU || f == F_LV ? N::linU
         : f == F_LP ? N::phi : N::phit;
}

template <typename T>
struct __align__(16) Stage {
  T f[NF][32];
  uint32_t cm[32];   // constraint-mask words (4 slots per word) of the columns' slots
};

template <typename T, int NR>
struct HalfSmem {
  Stage<T> st[DEPTH];
  int32_t code[2][NR][32];   // storage codes of the lane columns per strip row (two strips)
};

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

// Storage code of node (n, r) (brick-relative, -1..30) of a regular brick; the
// 3x3 neighbour bases are held by lanes 0..8 of each half-warp.  All 32 lanes
// call it (the two half-warps may hold different bricks).
__device__ __forceinline__ int32_t regular_code(int nbase, int n, int r) {
  const int dx = n < 0 ? -1 : (n >= NB ? 1 : 0);
  const int dy = r < 0 ? -1 : (r >= NB ? 1 : 0);
  const int base = __shfl_sync(0xffffffffu, nbase, (dy + 1) * 3 + dx + 1, 16);
  return base + (n - dx * NB) + NB * (r - dy * NB);
}

// Issue the copies of the lane's two columns of one strip row.
template <typename T, int OP>
__device__ __forceinline__ void issue_row(const ApplyArgs& a, bool pairwise, int32_t cA, int32_t cB, Stage<T>& st,
                                          int hl) {
  const int jA = 2 * hl, jB = 2 * hl + 1;
  if (pairwise) {  // both slots present, adjacent and 2-aligned
#pragma unroll
    for (int f = 0; f < NF; ++f)
      if (field_used<OP>(f)) cp_pair(&st.f[f][jA], field_ptr<T>(a, f) + cA);
    cp_async4(&st.cm[jA], reinterpret_cast<const uint32_t*>(a.cmask + (cA & ~3)));
  } else {
    if (cA >= 0) {
#pragma unroll
      for (int f = 0; f < NF; ++f)
        if (field_used<OP>(f)) cp_one(&st.f[f][jA], field_ptr<T>(a, f) + cA);
      cp_async4(&st.cm[jA], reinterpret_cast<const uint32_t*>(a.cmask + (cA & ~3)));
    }
    if (cB >= 0) {
#pragma unroll
      for (int f = 0; f < NF; ++f)
        if (field_used<OP>(f)) cp_one(&st.f[f][jB], field_ptr<T>(a, f) + cB);
      cp_async4(&st.cm[jB], reinterpret_cast<const uint32_t*>(a.cmask + (cB & ~3)));
    }
  }
}

// Make the landed row usable: masked components zeroed, absent slots zeroed,
// hanging slots filled from their constraint x_h = sum w x_parent.  Returns
// the constraint-mask byte of the column.
template <typename T, int OP>
__device__ __forceinline__ uint8_t settle_slot(const ApplyArgs& a, int32_t code, Stage<T>& st, int j, uint32_t cmw,
                                               int byte) {
  using N = Needs<OP>;
  const bool mask = (a.mode & MODE_MASK_INPUT) != 0;
  if (code >= 0) {
    const uint8_t cm = uint8_t(cmw >> (8 * byte));
    if (mask && cm) {
      if (N::xu && (cm & 1)) st.f[F_XU][j] = T(0);
      if (N::xu && (cm & 2)) st.f[F_XV][j] = T(0);
      if (N::xp && (cm & 4)) st.f[F_XP][j] = T(0);
    }
    return cm;
  }
  if (code == kAbsent) {
#pragma unroll
    for (int f = 0; f < NF; ++f)
      if (field_used<OP>(f)) st.f[f][j] = T(0);
    return 0;
  }
  const DevHanging& h = a.hang[-2 - code];
#pragma unroll
  for (int f = F_LU; f < NF; ++f)
    if (field_used<OP>(f)) st.f[f][j] = ldg(field_ptr<T>(a, f) + h.slot);
  T v0 = 0, v1 = 0, vp = 0;
  const int np = a.fe_degree + 1;
  for (int b = 0; b < np; ++b) {
    const int ps = h.parent[b];
    const T w = T(h.weight[b]);
    T p0 = 0, p1 = 0, pp = 0;
    if (N::xu) { p0 = ldg(field_ptr<T>(a, F_XU) + ps); p1 = ldg(field_ptr<T>(a, F_XV) + ps); }
    if (N::xp) pp = ldg(field_ptr<T>(a, F_XP) + ps);
    if (mask) {
      const uint8_t cm = ldg(a.cmask + ps);
      if (cm & 1) p0 = 0;
      if (cm & 2) p1 = 0;
      if (cm & 4) pp = 0;
    }
    v0 += w * p0; v1 += w * p1; vp += w * pp;
  }
  if (N::xu) { st.f[F_XU][j] = v0; st.f[F_XV][j] = v1; }
  if (N::xp) st.f[F_XP][j] = vp;
  return 0;
}

// The lane's node pair of a settled row, and the right-hand pair (own B, next lane's A).
template <typename T, int OP>
__device__ __forceinline__ void read_row(const Stage<T>& st, int hl, int right_lane, NodePair<T>& v, NodePair<T>& r) {
  using P = typename VT<T>::T2;
  const unsigned FULL = 0xffffffffu;
  P* dst[NF] = {&v.x0, &v.x1, &v.xp, &v.lx, &v.ly, &v.lz, &v.lw};
  P* dsr[NF] = {&r.x0, &r.x1, &r.xp, &r.lx, &r.ly, &r.lz, &r.lw};
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    if (field_used<OP>(f)) {
      const P q = *reinterpret_cast<const P*>(&st.f[f][2 * hl]);
      *dst[f] = q;
      P o;
      o.x = q.y;
      o.y = __shfl_sync(FULL, q.x, right_lane);
      *dsr[f] = o;
    } else {
      *dst[f] = pbc(T(0));
      *dsr[f] = pbc(T(0));
    }
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

// RS: node rows per strip (RSEG by default; 1 for latency-bound small level meshes)
template <typename T, int OP, int RS = RSEG>
__global__ void __launch_bounds__(32 * WARPS, sizeof(T) == 4 ? PFF_MINB : PFF_MINB64) apply_q1_kernel(const __grid_constant__ ApplyArgs a) {
  static_assert(NB % RS == 0, "strip height must divide the brick");
  constexpr int SROWS = RS;          // node rows per strip
  constexpr int SSEG = NB / RS;      // strips per brick
  constexpr int SREAD = RS + 2;      // node rows a strip reads
  using P = typename VT<T>::T2;
  constexpr bool outU = (OP != OP_PP && OP != OP_PP_DIAG && OP != OP_MASS && OP != OP_TCV && OP != OP_PHIT_VJP);
  constexpr bool outP = (OP != OP_UU && OP != OP_UU_DIAG);
  constexpr bool isDiag = (OP == OP_UU_DIAG || OP == OP_PP_DIAG);
  const unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int half = lane >> 4, hl = lane & 15;
  HalfSmem<T, SREAD>& sm = reinterpret_cast<HalfSmem<T, SREAD>*>(smem_raw)[(threadIdx.x >> 5) * 2 + half];
  const int right_lane = (half << 4) | ((hl + 1) & 15);
  const int left_lane = (half << 4) | ((hl + 15) & 15);
  const MatConst<T>& mc = matc<T>(a);
  // lane columns: nodes (2hl, 2hl+1) for hl < 15; lane 15 holds the halo nodes (30, -1)
  const int nA = hl < 15 ? 2 * hl : NB, nB = hl < 15 ? 2 * hl + 1 : -1;
  T* yu = reinterpret_cast<T*>(a.yu);
  T* yv = yu + a.n_slots;
  T* yp = reinterpret_cast<T*>(a.yp);
  const int nunits = a.lay.nbricks * SSEG;
  // Persistent warps.  Half-warp h of warp w sweeps the strips (units)
  // 2w + h + k * stride, k = 0, 1, ...; their node rows form one continuous
  // stream j = k * SREAD + i, kept DEPTH-1 rows ahead in the cp.async ring
  // across strip boundaries.
  const int stride = gridDim.x * WARPS * 2;
  const int ubase0 = (blockIdx.x * WARPS + (threadIdx.x >> 5)) * 2;
  if (ubase0 >= nunits) return;  // warp-uniform
  const int nrounds = (nunits - ubase0 + stride - 1) / stride;
  const int nstream = nrounds * SREAD;
  // codes of strip k into table k & 1 (all 32 lanes: shuffles); returns its pairwise flag
  auto build_codes = [&](int k) -> bool {
    const int unit = ubase0 + k * stride + half;
    const bool valid = unit < nunits;
    const int b = valid ? unit / SSEG : 0;
    const int r0 = valid ? (unit % SSEG) * SROWS : 0;
    const BrickDesc* bd = a.lay.bricks + b;
    const int nbase = hl < 9 ? __ldg(bd->nbr_base + hl) : 0;
    const int irr = __ldg(&bd->irr);
#pragma unroll
    for (int i = 0; i < SREAD; ++i) {
      const int r = r0 - 1 + i;
      int32_t cA = regular_code(nbase, nA, r);
      int32_t cB = regular_code(nbase, nB, r);
      if (irr >= 0) {
        const int32_t* w = a.lay.win + irr * (WN * WN) + WN * (r + 1);
        cA = __ldg(w + nA + 1);
        cB = __ldg(w + nB + 1);
      }
      if (!valid) { cA = kAbsent; cB = kAbsent; }
      sm.code[k & 1][i][2 * hl] = cA;
      sm.code[k & 1][i][2 * hl + 1] = cB;
    }
    return valid && irr < 0 && hl < 15;
  };
  bool pw_issue = build_codes(0);   // pairwise flag of the strip being issued
  int k_issue = 0;
  auto issue_stream = [&](int j) {
    if (j < nstream) {
      const int k = j / SREAD, i = j - k * SREAD;
      if (k != k_issue) { pw_issue = build_codes(k); k_issue = k; }
      issue_row<T, OP>(a, pw_issue, sm.code[k & 1][i][2 * hl], sm.code[k & 1][i][2 * hl + 1], sm.st[j % DEPTH], hl);
    }
    cp_async_commit();
  };
#pragma unroll 1
  for (int j = 0; j < DEPTH - 1; ++j) issue_stream(j);

  // per-strip state of the strip being computed
  bool valid = false, pairwise = false;
  int irr = 0, r0 = 0, own_base = 0, cnbase = 0;
  LevGeom<T> gq = geom<T>(a, 0);
  uint8_t cmA = 0, cmB = 0;
  P carry[3] = {pbc(T(0)), pbc(T(0)), pbc(T(0))};
#pragma unroll 1
  for (int j = 0; j < nstream; ++j) {
    const int k = j / SREAD, i = j - k * SREAD;
    if (i == 0) {
      const int unit = ubase0 + k * stride + half;
      valid = unit < nunits;
      const int b = valid ? unit / SSEG : 0;
      r0 = valid ? (unit % SSEG) * SROWS : 0;
      const BrickDesc* bd = a.lay.bricks + b;
      irr = __ldg(&bd->irr);
      own_base = __ldg(bd->nbr_base + 4);
      cnbase = hl < 9 ? __ldg(bd->nbr_base + hl) : 0;
      gq = geom<T>(a, __ldg(&bd->level));
      pairwise = valid && irr < 0 && hl < 15;
    }
    cp_async_wait<DEPTH - 2>();
    Stage<T>& si = sm.st[j % DEPTH];
    const int32_t cA = sm.code[k & 1][i][2 * hl], cB = sm.code[k & 1][i][2 * hl + 1];
    uint8_t nmA, nmB;
    if (pairwise) {
      const uint32_t w = si.cm[2 * hl];
      nmA = settle_slot<T, OP>(a, cA, si, 2 * hl, w, cA & 3);
      nmB = settle_slot<T, OP>(a, cB, si, 2 * hl + 1, w, cB & 3);
    } else {
      nmA = settle_slot<T, OP>(a, cA, si, 2 * hl, si.cm[2 * hl], cA & 3);
      nmB = settle_slot<T, OP>(a, cB, si, 2 * hl + 1, si.cm[2 * hl + 1], cB & 3);
    }
    if (i > 0) {
      const int c = r0 - 2 + i;  // cell row between node rows c and c + 1
      NodePair<T> v[4];
      read_row<T, OP>(sm.st[(j - 1) % DEPTH], hl, right_lane, v[0], v[1]);
      read_row<T, OP>(si, hl, right_lane, v[2], v[3]);
      bool actA = hl < 15, actB = true;
      if (irr >= 0) {
        const uint32_t* cmw = a.lay.cellmask + irr * 31;
        const int ib = (c + 1) * NCW + (nB + 1), ia = ib - 1;  // window cells of cells nA (if hl<15) and nB
        actA = actA && ((__ldg(cmw + (ia >> 5)) >> (ia & 31)) & 1u);
        actB = (__ldg(cmw + (ib >> 5)) >> (ib & 31)) & 1u;
      }
      // cell moduli: the cell slot of a cell is the slot of its lower-left node
      // position in the bricks of this level (neighbour bricks for column/row -1)
      P ec = pbc(T(1));
      if (a.ecell != nullptr) {  // uniform: all 32 lanes take the shuffles in regular_code
        const int32_t sA = regular_code(cnbase, nA, c), sB = regular_code(cnbase, nB, c);
        const T* E = reinterpret_cast<const T*>(a.ecell);
        if (valid && actA) ec.x = ldg(E + sA);
        if (valid && actB) ec.y = ldg(E + sB);
      }
      P out[12];
      q1_cell_pair<T, OP>(v, mc, gq, ec, out);
      if (!actA || !actB) {
#pragma unroll
        for (int q = 0; q < 12; ++q) {
          if (!actA) out[q].x = T(0);
          if (!actB) out[q].y = T(0);
        }
      }
      if constexpr (OP == OP_VJP) {
        // per-cell values of the cells owned by this strip (rows r0.., columns 0..29)
        if (c >= r0 && hl < 15 && valid) {
          T* co = reinterpret_cast<T*>(a.cell_out);
          const int64_t sA = own_base + nA + NB * c;
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            if (actA) co[q * a.n_slots + sA] = out[q].x;
            if (actB) co[q * a.n_slots + sA + 1] = out[q].y;
          }
        }
      } else {
      // the left lane's cell B contributes BR to our node A (row c) and TR to node A (row c+1)
      T brL[3], trL[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        brL[q] = __shfl_sync(FULL, out[3 + q].y, left_lane);
        trL[q] = __shfl_sync(FULL, out[9 + q].y, left_lane);
      }
      if (c >= r0 && hl < 15 && valid) {
        T yA[3], yB[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          yA[q] = (carry[q].x + brL[q]) + out[q].x;
          yB[q] = (carry[q].y + out[3 + q].x) + out[q].y;
        }
        if (irr < 0 && !(cmA | cmB)) {
          // regular brick, unconstrained pair: one aligned pair store per output field
          const int slot = own_base + nA + NB * c;
          if (outU) {
            *reinterpret_cast<P*>(yu + slot) = P{yA[0], yB[0]};
            *reinterpret_cast<P*>(yv + slot) = P{yA[1], yB[1]};
          }
          if (outP) *reinterpret_cast<P*>(yp + slot) = P{yA[2], yB[2]};
        } else {
          write_node<T, OP>(a, irr, own_base, nA, c, cmA, yA[0], yA[1], yA[2]);
          write_node<T, OP>(a, irr, own_base, nB, c, cmB, yB[0], yB[1], yB[2]);
        }
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        carry[q].x = out[6 + q].x + trL[q];
        carry[q].y = out[6 + q].y + out[9 + q].x;
      }
      }
    }
    cmA = nmA;
    cmB = nmB;
    // refill the stage of stream row j-1 (no longer read) with row j+DEPTH-1
    issue_stream(j + DEPTH - 1);
  }
  cp_async_wait<0>();
  (void)isDiag;
}

template <typename T>
__global__ void fixup_kernel(const FixupArgs a) {
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
  const T* xu = reinterpret_cast<const T*>(a.xu);
  const T* xp = reinterpret_cast<const T*>(a.xp);
  if (cm) {
    const bool ident = (a.mode & MODE_IDENTITY) != 0;
    if (cm & 1) y0 = ident ? xu[slot] : T(0);
    if (cm & 2) y1 = ident ? xu[a.n_slots + slot] : T(0);
    if (cm & 4) y2 = ident ? xp[slot] : T(0);
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
                                       double* lin64, float* lin32) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= nh) return;
  const DevHanging e = hang[h];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double v = 0;
    for (int b = 0; b < np; ++b) v += e.weight[b] * lin64[k * n + e.parent[b]];
    lin64[k * n + e.slot] = v;
    lin32[k * n + e.slot] = float(v);
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

template <typename T>
cudaError_t launch_apply(const ApplyArgs& a, int op, cudaStream_t s) {
  if (a.lay.nbricks <= 0) return cudaSuccess;
  if (a.fe_degree == 2) return launch_apply_q2<T>(a, op, s);
  if (a.fe_degree != 1) return cudaErrorInvalidValue;
  const unsigned blk = 32 * WARPS;
  auto grid_of = [&](const void* fn, int strips_per_brick, size_t smem) -> unsigned {
    const int units = (a.lay.nbricks * strips_per_brick + 1) / 2;  // two strips per warp
    const int full = resident_blocks(fn, int(blk), smem);
    const int need = (units + WARPS - 1) / WARPS;
    return unsigned(need < full ? need : full);
  };
  const size_t smem = sizeof(HalfSmem<T, NROWS>) * 2 * WARPS;
  // The level block operators of the V-cycle mostly run on small level meshes,
  // where one wave of single-row strips covers the mesh: there the shorter
  // per-strip chain (3 node rows read, 2 cell rows) gives the lower latency.
  if (op == OP_UU || op == OP_PP) {
    const size_t smem1 = sizeof(HalfSmem<T, 3>) * 2 * WARPS;
    const void* fn = op == OP_UU ? reinterpret_cast<const void*>(&apply_q1_kernel<T, OP_UU, 1>)
                                 : reinterpret_cast<const void*>(&apply_q1_kernel<T, OP_PP, 1>);
    const int need = ((a.lay.nbricks * NB + 1) / 2 + WARPS - 1) / WARPS;
    if (need <= resident_blocks(fn, int(blk), smem1)) {
      const unsigned g = grid_of(fn, NB, smem1);
      if (op == OP_UU) apply_q1_kernel<T, OP_UU, 1><<<g, blk, smem1, s>>>(a);
      else apply_q1_kernel<T, OP_PP, 1><<<g, blk, smem1, s>>>(a);
      return cudaGetLastError();
    }
  }
  switch (op) {
#define PFF_LAUNCH(OPV)                                                                        \
    case OPV: {                                                                                \
      const void* fn = reinterpret_cast<const void*>(&apply_q1_kernel<T, OPV>);               \
      apply_q1_kernel<T, OPV><<<grid_of(fn, NSEG, smem), blk, smem, s>>>(a);                   \
      break;                                                                                   \
    }
    PFF_LAUNCH(OP_FULL)
    PFF_LAUNCH(OP_FULL_T)
    PFF_LAUNCH(OP_UU)
    PFF_LAUNCH(OP_PP)
    PFF_LAUNCH(OP_UU_DIAG)
    PFF_LAUNCH(OP_PP_DIAG)
    PFF_LAUNCH(OP_RESID)
    PFF_LAUNCH(OP_MASS)
    PFF_LAUNCH(OP_TCV)
    PFF_LAUNCH(OP_TCV_GRAD)
    PFF_LAUNCH(OP_VJP)
    PFF_LAUNCH(OP_PHIT_VJP)
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
    set_lin_kernel<<<unsigned((n_slots + 255) / 256), 256, 0, s>>>(n_slots, u, phi, phit, lin64, lin32);
  if (nhang > 0)
    set_lin_hanging_kernel<<<(nhang + 127) / 128, 128, 0, s>>>(nhang, n_slots, hang, fe_degree + 1, lin64, lin32);
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
