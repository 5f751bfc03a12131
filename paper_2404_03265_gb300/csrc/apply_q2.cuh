// Q2 elements (k = 2) on the brick layout: one thread per cell of a brick window.
// Included by apply.cu inside its anonymous namespace (uses its field helpers,
// storage codes and write_node).
//
// Same operators as the Q1 kernel (Sec. 3.1 Jacobian and its transpose, the
// diagonal blocks and their diagonals of Sec. 3.2, the residual of Problem 2,
// lumped mass, TCV and its gradient, the parameter VJP), with the 3x3 Gauss rule.
//
// A brick owns 30 x 30 node slots = 15 x 15 Q2 cells; its window holds the
// 33 x 33 nodes -2..30 and the 16 x 16 cells -1..14 (all cells touching an
// owned node).  A block of 256 threads takes one brick at a time:
//   1. the window's node fields go to shared memory (hanging values from their
//      parents, fixed input components masked, absent nodes zero);
//   2. each thread evaluates one cell, sum-factorised: per Gauss row eta_q2 the
//      3x3 nodal values collapse to three column values, then to the row's
//      three Gauss points; the test runs the same two steps backwards.  Fields
//      that take the same contractions travel as pairs (u_x with u_y of the
//      input and of the linearisation, the input dphi with phi), one paired
//      FP32 instruction for both, and the shared tiles interleave each pair;
//   3. the cells' nodal contributions are added into a shared tile in four
//      colour phases (cells of equal (i, j) parity share no node), so every
//      nodal sum has a fixed order;
//   4. the owned nodes are written (constraint rows, partial sums, holes), or
//      for the level block operators the fused Chebyshev step of ChebEpi.

constexpr int Q2NB = 30;          // owned node slots per side
constexpr int Q2W = 33;           // window nodes per side (-2..30)
constexpr int Q2C = 16;           // window cells per side (-1..14)
constexpr int Q2T = Q2C * Q2C;    // threads per block: one per window cell
constexpr int Q2WW = Q2W * Q2W;

// Field pairs of the window tiles: pair 0 (u_x, u_y of the input), 1 (u_x, u_y
// of the linearisation), 2 (input dphi, phi), 3 (phi_tilde, unused).
constexpr int Q2NP = 4;
__host__ __device__ constexpr int q2_pair(int f) {
  return f == F_XU || f == F_XV ? 0 : f == F_LU || f == F_LV ? 1 : f == F_XP || f == F_LP ? 2 : 3;
}
__host__ __device__ constexpr int q2_half(int f) { return f == F_XV || f == F_LV || f == F_LP ? 1 : 0; }
template <int OP>
__device__ __forceinline__ constexpr bool q2_pair_used(int k) {
  return k == 0 ? field_used<OP>(F_XU) || field_used<OP>(F_XV)
       : k == 1 ? field_used<OP>(F_LU) || field_used<OP>(F_LV)
       : k == 2 ? field_used<OP>(F_XP) || field_used<OP>(F_LP) : field_used<OP>(F_LT);
}

// FP32 keeps two window buffers: while a block computes one brick, the window
// of its next brick, when regular, streams into the other with cp.async.  FP64
// (twice the bytes per field) keeps one and gathers each brick in turn.
template <typename T>
struct Q2Smem {
  using P = typename VT<T>::T2;
  static constexpr int NBUF = sizeof(T) == 4 ? 2 : 1;
  P f[NBUF][Q2NP][Q2WW];    // node fields of the window, as pairs (q2_pair, q2_half)
  P yu[Q2WW];               // nodal sums, u_x and u_y
  T yp[Q2WW];               // nodal sums, phi
  uint32_t cmw[NBUF][Q2WW]; // prefetch: the aligned word holding each node's constraint byte
  int32_t nb[NBUF][9];      // storage bases of the 3x3 neighbour bricks
  uint8_t cmsh[NBUF][Q2WW]; // prefetch: byte position of the constraint byte in its word
  uint8_t cm[Q2WW];         // constraint-mask byte of each window node of the current brick
};

template <typename T>
__device__ __forceinline__ T& q2_field(typename VT<T>::T2 (*fb)[Q2WW], int f, int w) {
  return half_of<T>(fb[q2_pair(f)][w], q2_half(f));
}

// Storage slot of node (n, r) (brick-relative, -2..30) of a brick whose
// neighbour bases are nb; the caller guarantees the neighbour exists.
__device__ __forceinline__ int32_t q2_slot(const int32_t* nb, int n, int r) {
  const int dx = n < 0 ? -1 : (n >= Q2NB ? 1 : 0);
  const int dy = r < 0 ? -1 : (r >= Q2NB ? 1 : 0);
  return nb[(dy + 1) * 3 + dx + 1] + (n - dx * Q2NB) + Q2NB * (r - dy * Q2NB);
}

// Quantities of one Gauss point (only those the operator needs are set).
template <typename T>
struct Q2Point {
  T ux, uy, uxx, uxy, uyx, uyy;   // u and grad u (u_i,j = du_i/dx_j)
  T phi, phix, phiy, phit;        // phi, grad phi, phi_tilde
  T ax, bxy, cyx, dy;             // grad of the input du: du_x,x  du_x,y  du_y,x  du_y,y
  T xp, xpx, xpy;                 // input dphi and its gradient
};

// Test coefficients of one Gauss point: component c gets
//   f0[c] psi + fx[c] dpsi/dx + fy[c] dpsi/dy.
template <typename T>
struct Q2Coef {
  T f0[3], fx[3], fy[3];
};

template <typename T, int OP>
__device__ __forceinline__ void q2_point(const Q2Point<T>& q, const MatConst<T>& m, T c2ml, T cl, T cm,
                                         Q2Coef<T>& c, T cell[3]) {
  using N = Needs<OP>;
#pragma unroll
  for (int k = 0; k < 3; ++k) { c.f0[k] = T(0); c.fx[k] = T(0); c.fy[k] = T(0); }
  T gq = T(0), s11 = T(0), s22 = T(0), s12 = T(0), se = T(0), mq = T(0), ge12 = T(0);
  if (N::phit) gq = m.omk * q.phit * q.phit + m.kap;
  if (N::linU) {
    ge12 = q.uxy + q.uyx;
    s11 = c2ml * q.uxx + cl * q.uyy;
    s22 = cl * q.uxx + c2ml * q.uyy;
    s12 = cm * ge12;
    se = s11 * q.uxx + s22 * q.uyy + s12 * ge12;
    mq = m.omk * se + m.p2 * (q.uxx + q.uyy) + m.gcl;
  }
  if constexpr (OP == OP_FULL || OP == OP_FULL_T || OP == OP_UU) {
    const T bc = q.bxy + q.cyx;
    T S11 = gq * (c2ml * q.ax + cl * q.dy);
    T S22 = gq * (cl * q.ax + c2ml * q.dy);
    T S12 = gq * (cm * bc);
    if constexpr (OP == OP_FULL || OP == OP_FULL_T) {
      const T tp = q.phi + q.phi;
      const T T11 = tp * (m.omk * s11 + m.p), T22 = tp * (m.omk * s22 + m.p), T12 = tp * (m.omk * s12);
      if constexpr (OP == OP_FULL) {
        c.f0[2] = T11 * q.ax + T22 * q.dy + T12 * bc + mq * q.xp;
      } else {
        S11 += q.xp * T11;
        S22 += q.xp * T22;
        S12 += q.xp * T12;
        c.f0[2] = mq * q.xp;
      }
      c.fx[2] = m.gcL * q.xpx;
      c.fy[2] = m.gcL * q.xpy;
    }
    c.fx[0] = S11; c.fy[0] = S12;
    c.fx[1] = S12; c.fy[1] = S22;
  } else if constexpr (OP == OP_PP) {
    c.f0[2] = mq * q.xp;
    c.fx[2] = m.gcL * q.xpx;
    c.fy[2] = m.gcL * q.xpy;
  } else if constexpr (OP == OP_RESID) {
    // R = -A(U)(psi), Problem 2 (sigma^+ read as sigma); the sign is applied by the caller
    const T pt2 = m.p * q.phit * q.phit;
    c.fx[0] = gq * s11 + pt2; c.fy[0] = gq * s12;
    c.fx[1] = gq * s12;       c.fy[1] = gq * s22 + pt2;
    c.f0[2] = m.omk * q.phi * se + m.p2 * q.phi * (q.uxx + q.uyy) + m.gcl * (q.phi - T(1));
    c.fx[2] = m.gcL * q.phix;
    c.fy[2] = m.gcL * q.phiy;
  } else if constexpr (OP == OP_MASS) {
    c.f0[2] = T(1);
  } else if constexpr (OP == OP_TCV) {
    c.f0[2] = q.ux * q.phix + q.uy * q.phiy;
  } else if constexpr (OP == OP_TCV_GRAD) {
    c.f0[0] = q.phix;
    c.f0[1] = q.phiy;
    c.fx[2] = q.ux;
    c.fy[2] = q.uy;
  } else if constexpr (OP == OP_PHIT_VJP) {
    const T sw = s11 * q.ax + s22 * q.dy + s12 * (q.bxy + q.cyx);
    c.f0[2] = T(2) * q.phit * (m.omk * sw + m.p * (q.ax + q.dy));
  } else if constexpr (OP == OP_VJP) {
    // per cell: E_K, p and G_c derivatives of x . R (unit-modulus constants in m)
    const T u11 = m.c2ml * q.uxx + m.cl * q.uyy, u22 = m.cl * q.uxx + m.c2ml * q.uyy, u12 = m.cm * ge12;
    const T use = u11 * q.uxx + u22 * q.uyy + u12 * ge12;
    const T sw = u11 * q.ax + u22 * q.dy + u12 * (q.bxy + q.cyx);
    cell[0] = gq * sw + m.omk * q.phi * use * q.xp;
    cell[1] = q.phit * q.phit * (q.ax + q.dy) + T(2) * q.phi * (q.uxx + q.uyy) * q.xp;
    cell[2] = m.l * (q.phix * q.xpx + q.phiy * q.xpy) - m.il * (T(1) - q.phi) * q.xp;
  }
  (void)se;
}

// One Q2 cell: node (a, b) of the cell (a along x, b along y) is window node
// base + a + Q2W * b.  Contributions to node A = a + 3 b: ru[A] (components u_x,
// u_y) and rp[A] (phi).  cell[]: per-cell values (OP_VJP).
template <typename T, int OP>
__device__ __forceinline__ void q2_cell(const typename VT<T>::T2 (*fb)[Q2WW], int base, const MatConst<T>& m,
                                        const LevGeom<T>& g, const Q2Tab<T>& tb, T ec, typename VT<T>::T2 ru[9],
                                        T rp[9], T cell[3]) {
  using N = Needs<OP>;
  using P = typename VT<T>::T2;
  constexpr bool isDiag = (OP == OP_UU_DIAG || OP == OP_PP_DIAG);
  const T c2ml = m.c2ml * ec, cl = m.cl * ec, cm = m.cm * ec;
  const T area = T(4) * g.jxw;   // hx hy
#pragma unroll
  for (int k = 0; k < 9; ++k) { ru[k] = pbc(T(0)); rp[k] = T(0); }
  cell[0] = cell[1] = cell[2] = T(0);
#pragma unroll
  for (int q2 = 0; q2 < 3; ++q2) {
    // collapse every used pair along eta: V[a] = sum_b l_b(eta) v_ab, E[a] = sum_b l_b'(eta) v_ab
    // (pair 3 holds phi_tilde alone, whose value is all the point needs: no E)
    P V[Q2NP][3], E[Q2NP - 1][3];
#pragma unroll
    for (int k = 0; k < Q2NP; ++k) {
      if (!q2_pair_used<OP>(k)) continue;
      const P* fl = fb[k] + base;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const P v0 = fl[a], v1 = fl[a + Q2W], v2 = fl[a + 2 * Q2W];
        V[k][a] = pfma(pbc(tb.L[2][q2]), v2, pfma(pbc(tb.L[1][q2]), v1, pmul(pbc(tb.L[0][q2]), v0)));
        if (k < Q2NP - 1)
          E[k][a] = pfma(pbc(tb.D[2][q2]), v2, pfma(pbc(tb.D[1][q2]), v1, pmul(pbc(tb.D[0][q2]), v0)));
      }
    }
    // test sums per node column a: value/x-gradient part and y-gradient part
    P RvU[3], ReU[3];
    T Rvp[3], Rep[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) { RvU[a] = pbc(T(0)); ReU[a] = pbc(T(0)); Rvp[a] = T(0); Rep[a] = T(0); }
#pragma unroll
    for (int q1 = 0; q1 < 3; ++q1) {
      auto val = [&](int k) {
        return pfma(pbc(tb.L[2][q1]), V[k][2], pfma(pbc(tb.L[1][q1]), V[k][1], pmul(pbc(tb.L[0][q1]), V[k][0])));
      };
      auto ddx = [&](int k) {
        return pmul(pfma(pbc(tb.D[2][q1]), V[k][2], pfma(pbc(tb.D[1][q1]), V[k][1], pmul(pbc(tb.D[0][q1]), V[k][0]))),
                    pbc(g.ihx));
      };
      auto ddy = [&](int k) {
        return pmul(pfma(pbc(tb.L[2][q1]), E[k][2], pfma(pbc(tb.L[1][q1]), E[k][1], pmul(pbc(tb.L[0][q1]), E[k][0]))),
                    pbc(g.ihy));
      };
      Q2Point<T> q{};
      if (N::xu) {
        const P dx = ddx(0), dy = ddy(0);
        q.ax = dx.x; q.bxy = dy.x; q.cyx = dx.y; q.dy = dy.y;
      }
      if (N::xp || N::phi) {
        const P v = val(2), dx = ddx(2), dy = ddy(2);
        if (N::xp) { q.xp = v.x; q.xpx = dx.x; q.xpy = dy.x; }
        if (N::phi) { q.phi = v.y; q.phix = dx.y; q.phiy = dy.y; }
      }
      if (N::linU) {
        const P dx = ddx(1), dy = ddy(1);
        q.uxx = dx.x; q.uxy = dy.x; q.uyx = dx.y; q.uyy = dy.y;
        if (OP == OP_TCV || OP == OP_TCV_GRAD) {
          const P v = val(1);
          q.ux = v.x; q.uy = v.y;
        }
      }
      if (N::phit) q.phit = val(3).x;
      const T W = area * tb.w[q1] * tb.w[q2];
      if constexpr (isDiag) {
        // diagonal of the element matrix of the block
        T gq = T(0), mq = T(0);
        if (OP == OP_UU_DIAG) gq = m.omk * q.phit * q.phit + m.kap;
        if (OP == OP_PP_DIAG) {
          const T ge12 = q.uxy + q.uyx;
          const T s11 = c2ml * q.uxx + cl * q.uyy, s22 = cl * q.uxx + c2ml * q.uyy, s12 = cm * ge12;
          mq = m.omk * (s11 * q.uxx + s22 * q.uyy + s12 * ge12) + m.p2 * (q.uxx + q.uyy) + m.gcl;
        }
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const T Nv = tb.L[a][q1] * tb.L[b][q2];
            const T dxn = tb.D[a][q1] * tb.L[b][q2] * g.ihx, dyn = tb.L[a][q1] * tb.D[b][q2] * g.ihy;
            const int A = a + 3 * b;
            if (OP == OP_UU_DIAG) {
              ru[A].x += W * gq * (c2ml * dxn * dxn + cm * dyn * dyn);
              ru[A].y += W * gq * (cm * dxn * dxn + c2ml * dyn * dyn);
            } else {
              rp[A] += W * (mq * Nv * Nv + m.gcL * (dxn * dxn + dyn * dyn));
            }
          }
      } else if constexpr (OP == OP_VJP) {
        Q2Coef<T> cf;
        T cv[3];
        q2_point<T, OP>(q, m, c2ml, cl, cm, cf, cv);
        cell[0] += W * cv[0];
        cell[1] += W * cv[1];
        cell[2] += W * cv[2];
      } else {
        Q2Coef<T> cf;
        T cv[3];
        q2_point<T, OP>(q, m, c2ml, cl, cm, cf, cv);
        const T wx = W * g.ihx, wy = W * g.ihy;
        P f0u, fxu, fyu;
        f0u.x = W * cf.f0[0]; f0u.y = W * cf.f0[1];
        fxu.x = wx * cf.fx[0]; fxu.y = wx * cf.fx[1];
        fyu.x = wy * cf.fy[0]; fyu.y = wy * cf.fy[1];
        const T f0p = W * cf.f0[2], fxp = wx * cf.fx[2], fyp = wy * cf.fy[2];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          RvU[a] = pfma(pbc(tb.L[a][q1]), f0u, pfma(pbc(tb.D[a][q1]), fxu, RvU[a]));
          ReU[a] = pfma(pbc(tb.L[a][q1]), fyu, ReU[a]);
          Rvp[a] += tb.L[a][q1] * f0p + tb.D[a][q1] * fxp;
          Rep[a] += tb.L[a][q1] * fyp;
        }
      }
    }
    if constexpr (!isDiag && OP != OP_VJP) {
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int A = a + 3 * b;
          ru[A] = pfma(pbc(tb.L[b][q2]), RvU[a], pfma(pbc(tb.D[b][q2]), ReU[a], ru[A]));
          rp[A] += tb.L[b][q2] * Rvp[a] + tb.D[b][q2] * Rep[a];
        }
    }
  }
  if constexpr (OP == OP_RESID) {
#pragma unroll
    for (int k = 0; k < 9; ++k) { ru[k] = pmul(pbc(T(-1)), ru[k]); rp[k] = -rp[k]; }
  }
  if constexpr (OP == OP_VJP) {
    cell[0] = -cell[0]; cell[1] = -cell[1]; cell[2] = -cell[2];
  }
}

template <typename T> __device__ __forceinline__ const Q2Tab<T>& q2tab(const ApplyArgs& a);
template <> __device__ __forceinline__ const Q2Tab<float>& q2tab<float>(const ApplyArgs& a) { return a.q2f; }
template <> __device__ __forceinline__ const Q2Tab<double>& q2tab<double>(const ApplyArgs& a) { return a.q2d; }

template <typename T, int OP>
__global__ void __launch_bounds__(Q2T, sizeof(T) == 4 ? 2 : 1) apply_q2_kernel(const __grid_constant__ ApplyArgs a) {
  using P = typename VT<T>::T2;
  constexpr bool isVjp = (OP == OP_VJP);
  constexpr int NBUF = Q2Smem<T>::NBUF;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Q2Smem<T>& sm = *reinterpret_cast<Q2Smem<T>*>(smem_raw);
  const int tid = threadIdx.x;
  const bool mask = (a.mode & MODE_MASK_INPUT) != 0;
  const MatConst<T>& mc = matc<T>(a);
  const Q2Tab<T>& tb = q2tab<T>(a);
  const int ci = tid % Q2C, cj = tid / Q2C;          // window cell (cell ci - 1, cj - 1)
  const int cbase = 2 * ci + Q2W * 2 * cj;            // window node (0, 0) of the cell
  const int G = int(gridDim.x);
  // window of regular brick bn into buffer bu: cp.async of every used field and of
  // the word holding each node's constraint byte; committed as one group
  auto prefetch = [&](int bn, int bu) {
    const BrickDesc* bdn = a.lay.bricks + bn;
    int32_t nbv[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) nbv[i] = __ldg(bdn->nbr_base + i);
    if (tid < 9) sm.nb[bu][tid] = nbv[tid];
    for (int w = tid; w < Q2WW; w += Q2T) {
      const int32_t code = q2_slot(nbv, w % Q2W - 2, w / Q2W - 2);
#pragma unroll
      for (int f = 0; f < NF; ++f)
        if (field_used<OP>(f)) cp_one(&q2_field<T>(sm.f[bu], f, w), field_ptr<T>(a, f) + code);
      cp_async4(&sm.cmw[bu][w], a.cmask + (code & ~3));
      sm.cmsh[bu][w] = uint8_t(code & 3);
    }
    cp_async_commit();
  };
  auto regular = [&](int bn) { return __ldg(&a.lay.bricks[bn].irr) < 0; };
  int cur = 0;
  bool pending = false;   // buffer cur holds a prefetch of brick b not yet waited for
  if (NBUF == 2 && int(blockIdx.x) < a.lay.nbricks && regular(blockIdx.x)) {
    prefetch(blockIdx.x, 0);
    pending = true;
  }
#pragma unroll 1
  for (int b = blockIdx.x; b < a.lay.nbricks; b += G) {
    const BrickDesc* bd = a.lay.bricks + b;
    const int irr = __ldg(&bd->irr);
    const int level = __ldg(&bd->level);
    P (*fb)[Q2WW] = sm.f[cur];
    const int32_t* nbc = sm.nb[cur];
    __syncthreads();   // the previous brick's tiles are no longer read
    if (pending) {
      // 1a. the prefetched window: constraint bytes, masked input components, a zero output tile
      cp_async_wait<0>();
      for (int w = tid; w < Q2WW; w += Q2T) {
        const uint8_t cmw = uint8_t((sm.cmw[cur][w] >> (8 * sm.cmsh[cur][w])) & 0xffu);
        sm.cm[w] = cmw;
        if (mask && cmw) {
          if (cmw & 1) q2_field<T>(fb, F_XU, w) = T(0);
          if (cmw & 2) q2_field<T>(fb, F_XV, w) = T(0);
          if (cmw & 4) q2_field<T>(fb, F_XP, w) = T(0);
        }
        if (!isVjp) { sm.yu[w] = pbc(T(0)); sm.yp[w] = T(0); }
      }
    } else {
      if (tid < 9) sm.nb[cur][tid] = __ldg(bd->nbr_base + tid);
      __syncthreads();
      // 1b. window node fields (and a zero output tile)
      for (int w = tid; w < Q2WW; w += Q2T) {
        const int wx = w % Q2W, wy = w / Q2W;
        const int32_t code = irr < 0 ? q2_slot(nbc, wx - 2, wy - 2) : __ldg(a.lay.win + int64_t(irr) * Q2WW + w);
        T v[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) v[f] = T(0);
        uint8_t cmw = 0;
        if (code >= 0) {
          cmw = __ldg(a.cmask + code);
#pragma unroll
          for (int f = 0; f < NF; ++f)
            if (field_used<OP>(f)) v[f] = ldg(field_ptr<T>(a, f) + code);
          if (mask && cmw) {
            if (cmw & 1) v[F_XU] = T(0);
            if (cmw & 2) v[F_XV] = T(0);
            if (cmw & 4) v[F_XP] = T(0);
          }
        } else if (code != kAbsent) {
          const DevHanging& h = a.hang[-2 - code];
#pragma unroll
          for (int f = F_LU; f < NF; ++f)
            if (field_used<OP>(f)) v[f] = ldg(field_ptr<T>(a, f) + h.slot);
          for (int p = 0; p < 3; ++p) {
            const int ps = h.parent[p];
            const T wgt = T(h.weight[p]);
            const uint8_t pc = mask ? __ldg(a.cmask + ps) : uint8_t(0);
#pragma unroll
            for (int f = F_XU; f <= F_XP; ++f)
              if (field_used<OP>(f) && !(pc & (1 << f))) v[f] += wgt * ldg(field_ptr<T>(a, f) + ps);
          }
        }
#pragma unroll
        for (int f = 0; f < NF; ++f)
          if (field_used<OP>(f)) q2_field<T>(fb, f, w) = v[f];
        sm.cm[w] = cmw;
        if (!isVjp) { sm.yu[w] = pbc(T(0)); sm.yp[w] = T(0); }
      }
    }
    __syncthreads();
    // the next brick's window streams in while this one computes
    bool next_pending = false;
    if (NBUF == 2 && b + G < a.lay.nbricks && regular(b + G)) {
      prefetch(b + G, cur ^ 1);
      next_pending = true;
    }
    // 2. one cell per thread
    bool act = true;
    if (irr >= 0) {
      const int c = ci + Q2C * cj;
      act = (__ldg(a.lay.cellmask + irr * ((Q2T + 31) / 32) + (c >> 5)) >> (c & 31)) & 1u;
    }
    T ec = T(1);
    if (a.ecell != nullptr && act) ec = ldg(reinterpret_cast<const T*>(a.ecell) + q2_slot(nbc, 2 * ci - 2, 2 * cj - 2));
    P ru[9];
    T rp[9], cell[3];
    if (act) q2_cell<T, OP>(fb, cbase, mc, geom<T>(a, level), tb, ec, ru, rp, cell);
    if constexpr (isVjp) {
      // the brick owns the cells whose lower-left node it owns (cells 0..14)
      if (act && ci >= 1 && cj >= 1) {
        T* co = reinterpret_cast<T*>(a.cell_out);
        const int64_t s = int64_t(nbc[4]) + 2 * (ci - 1) + Q2NB * 2 * (cj - 1);
#pragma unroll
        for (int q = 0; q < 3; ++q) co[q * a.n_slots + s] = cell[q];
      }
    } else {
      // 3. colour phases: cells of one (i, j) parity add their 9 x 3 contributions
#pragma unroll 1
      for (int ph = 0; ph < 4; ++ph) {
        if (act && (ci & 1) == (ph & 1) && (cj & 1) == (ph >> 1)) {
#pragma unroll
          for (int bb = 0; bb < 3; ++bb)
#pragma unroll
            for (int aa = 0; aa < 3; ++aa) {
              const int w = cbase + aa + Q2W * bb;
              sm.yu[w] = padd(sm.yu[w], ru[aa + 3 * bb]);
              sm.yp[w] += rp[aa + 3 * bb];
            }
        }
        __syncthreads();
      }
      // 4. owned nodes (level block operators: or the fused Chebyshev store)
      const int own_base = nbc[4];
      for (int o = tid; o < Q2NB * Q2NB; o += Q2T) {
        const int oi = o % Q2NB, oj = o / Q2NB;
        const int w = (oi + 2) + Q2W * (oj + 2);
        if constexpr (OP == OP_UU || OP == OP_PP) {
          if (a.ch.mode != CHEB_OFF) {
            const int act_s = irr >= 0 ? int(__ldg(a.lay.own_act + irr * (Q2NB * Q2NB) + o)) : int(kActFinal);
            ChebOps<T, OP> co;
            cheb_load<T, OP>(a, own_base + o, co);
            cheb_store<T, OP>(a, own_base + o, act_s, sm.cm[w], sm.yu[w].x, sm.yu[w].y, sm.yp[w], co);
            continue;
          }
        }
        write_node<T, OP>(a, irr, own_base, oi, oj, sm.cm[w], sm.yu[w].x, sm.yu[w].y, sm.yp[w]);
      }
    }
    if (NBUF == 2) cur ^= 1;
    pending = next_pending;
  }
  cp_async_wait<0>();
}

template <typename T>
cudaError_t launch_apply_q2(const ApplyArgs& a, int op, cudaStream_t s) {
  const size_t smem = sizeof(Q2Smem<T>);
  auto grid_of = [&](const void* fn) -> unsigned {
    const int full = resident_blocks(fn, Q2T, smem);
    return unsigned(a.lay.nbricks < full ? a.lay.nbricks : full);
  };
  switch (op) {
#define PFF_LAUNCH2(OPV)                                                                       \
    case OPV: {                                                                                \
      const void* fn = reinterpret_cast<const void*>(&apply_q2_kernel<T, OPV>);               \
      apply_q2_kernel<T, OPV><<<grid_of(fn), Q2T, smem, s>>>(a);                               \
      break;                                                                                   \
    }
    PFF_LAUNCH2(OP_FULL)
    PFF_LAUNCH2(OP_FULL_T)
    PFF_LAUNCH2(OP_UU)
    PFF_LAUNCH2(OP_PP)
    PFF_LAUNCH2(OP_UU_DIAG)
    PFF_LAUNCH2(OP_PP_DIAG)
    PFF_LAUNCH2(OP_RESID)
    PFF_LAUNCH2(OP_MASS)
    PFF_LAUNCH2(OP_TCV)
    PFF_LAUNCH2(OP_TCV_GRAD)
    PFF_LAUNCH2(OP_VJP)
    PFF_LAUNCH2(OP_PHIT_VJP)
#undef PFF_LAUNCH2
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
