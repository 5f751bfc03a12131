// Host driver of the block-diagonal geometric multigrid preconditioner.
//
// Kolditz & Wick (arXiv 2404.03265), Sec. 3.2: one V-cycle per diagonal block
// (u-u, phi-phi) of the Jacobian; Chebyshev-accelerated Jacobi smoothing with
// the inverse diagonal from cell-local assembly and a CG-based estimate of the
// largest eigenvalue, smoothing range [0.08, 1.2] * lambda_max; local
// smoothing on the level meshes; coarse level solved directly (FP64).
//
// V-cycle of one block (levels L..1, coarse 0):
//   copy the leaf defect to the coarsest level on which each DoF is interior;
//   down: Chebyshev from zero, defect d - A x on interior and edge rows,
//         restriction P^T into the next coarser level;
//   coarse: x_0 = A_0^{-1} d_0 on the interior;
//   up: x += P x_coarse on all level nodes, Chebyshev on d - A x;
//   copy the level solutions back to the leaf DoFs (fixed leaf rows: z = r).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "solve.cuh"
#include "state.h"

namespace pff {

namespace {

constexpr int kMaxLanczos = 64;   // CG coefficient pairs stored per set-up chain

inline int block_op(int b) { return b == 0 ? OP_UU : OP_PP; }
inline int block_diag_op(int b) { return b == 0 ? OP_UU_DIAG : OP_PP_DIAG; }

// Largest eigenvalue of the symmetric tridiagonal matrix (d, e) by bisection on Sturm counts.
double tridiag_max_eig(const std::vector<double>& d, const std::vector<double>& e) {
  const int m = int(d.size());
  if (m == 0) return 0.0;
  double lo = d[0], hi = d[0];
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i < m - 1 ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - r);
    hi = std::max(hi, d[i] + r);
  }
  auto count_below = [&](double x) {  // eigenvalues < x
    int c = 0;
    double q = d[0] - x;
    if (q < 0) ++c;
    for (int i = 1; i < m; ++i) {
      const double qq = (q == 0.0) ? 1e-300 : q;
      q = d[i] - x - e[i - 1] * e[i - 1] / qq;
      if (q < 0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(hi), 1e-300); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(mid) == m) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Smallest eigenvalue of the same symmetric tridiagonal matrix (bisection on the Sturm count).
double tridiag_min_eig(const std::vector<double>& d, const std::vector<double>& e) {
  const int m = int(d.size());
  if (m == 0) return 0.0;
  double lo = d[0], hi = d[0];
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i < m - 1 ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - r);
    hi = std::max(hi, d[i] + r);
  }
  auto count_below = [&](double x) {
    int c = 0;
    double q = d[0] - x;
    if (q < 0) ++c;
    for (int i = 1; i < m; ++i) {
      const double qq = (q == 0.0) ? 1e-300 : q;
      q = d[i] - x - e[i - 1] * e[i - 1] / qq;
      if (q < 0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(hi), 1e-300); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= 1) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Smallest degree m with 1 / T_m((b + a) / (b - a)) <= tol (Chebyshev error bound on [a, b]).
int chebyshev_degree(double a, double b, double tol = 1e-3, int cap = 64) {
  const double sigma = (b + a) / (b - a);
  for (int m = 1; m <= cap; ++m)
    if (1.0 / std::cosh(m * std::acosh(sigma)) <= tol) return m;
  return cap;
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return std::string(#call) + ": " + cudaGetErrorString(e_); \
  } while (0)

}  // namespace

// pdl: launched dependent on the preceding kernel of the stream (the V-cycle chain)
template <typename T>
cudaError_t level_apply(pff_mg& mg, int level, int op, const T* x, T* y, cudaStream_t s, bool pdl,
                        const ChebEpi* ch) {
  pff_problem& pb = *mg.pb;
  const Mesh& M = pb.mesh->m;
  const DevMesh::Level& L = pb.mesh->dev.levels[level];
  ApplyArgs a;
  std::memset(&a, 0, sizeof(a));
  a.lay = L.lay;
  a.hang = nullptr;
  a.cmask = mg.cmask + L.lv.off;
  const int64_t n = L.lv.n_slots;
  if (sizeof(T) == 8) a.lin = mg.lin64 + 4 * L.lv.off; else a.lin = mg.lin32 + 4 * L.lv.off;
  a.xu = x; a.xp = x; a.yu = y; a.yp = y;
  a.ibuf = nullptr;
  a.n_slots = n;
  for (int l = 0; l <= M.Lf && l < kMaxLevels; ++l) { a.hx[l] = M.tree.hx(l); a.hy[l] = M.tree.hy(l); }
  fill_material(pb.prm, a, pb.has_ecell);
  if (pb.has_ecell) {
    if (sizeof(T) == 8) a.ecell = pb.lev_ecell64 + L.lv.off; else a.ecell = pb.lev_ecell32 + L.lv.off;
  }
  fill_cell_constants(a, M.Lf + 1);
  a.fe_degree = M.k;
  a.sweep_sh = pb.sweep_sh;
  a.pdl_in = pdl ? 1 : 0;
  a.mode = MODE_MASK_INPUT;
  if (ch) a.ch = *ch;
  return launch_apply<T>(a, op, s);
}

std::string mg_alloc(pff_mg& mg) {
  const DevMesh& D = mg.pb->mesh->dev;
  const int64_t N = D.lev_total;
  mg.vc_in = mg.mem.alloc<double>(3 * mg.pb->mesh->m.lay.n_slots);
  mg.vc_out = mg.mem.alloc<double>(3 * mg.pb->mesh->m.lay.n_slots);
  mg.lin64 = mg.mem.alloc<double>(4 * N);
  mg.lin32 = mg.mem.alloc<float>(4 * N);
  mg.cmask = mg.mem.alloc<uint8_t>(N);
  const size_t esz = mg.precision == PFF_F64 ? sizeof(double) : sizeof(float);
  for (int b = 0; b < 2; ++b) {
    MGBlock& B = mg.blk[b];
    B.ncomp = b == 0 ? 2 : 1;
    B.fixbits = b == 0 ? 3 : 4;
    const int64_t n = B.ncomp * N;
    B.dinv64 = mg.mem.alloc<double>(n);
    B.dinv32 = mg.mem.alloc<float>(n);
    void** bufs[6] = {&B.d, &B.x, &B.r, &B.y, &B.yp, &B.t};
    for (auto* p : bufs) *p = mg.mem.alloc<unsigned char>(n * esz);
    B.lam.assign(D.levels.size(), 0.0);
  }
  const int nchain = 2 * int(D.levels.size());
  for (int b = 0; b < 2; ++b) mg.su_vec[b] = mg.mem.alloc<double>(5 * mg.blk[b].ncomp * N);
  mg.su_partial = mg.mem.alloc<double>(int64_t(nchain) * mg_dot_partials());
  mg.su_sc = mg.mem.alloc<double>(8 * nchain);
  mg.su_hist = mg.mem.alloc<double>(2 * kMaxLanczos * nchain);
  const int Mc = 2 * mg.pb->mesh->m.k + 1;
  const int64_t n0 = D.levels.empty() ? 0 : D.levels[0].lv.n_slots;
  mg.probe_len = (2 * 2 + 1 * 1) * Mc * Mc * n0;   // sum over blocks of ncomp^2 Mc^2 n_0
  mg.probe_in = mg.mem.alloc<double>(std::max<int64_t>(mg.probe_len, 1));
  mg.probe_out = mg.mem.alloc<double>(std::max<int64_t>(mg.probe_len, 1));
  mg.spd_bad = mg.mem.alloc<int32_t>(2);
  if (!mg.mem.err.empty()) return mg.mem.err;
  return "";
}

// Per Newton step: level linearisation, level constraint masks, inverse
// diagonals, eigenvalue estimates and the coarse inverse of both blocks.
void mg_release_graphs(pff_mg& mg) {
  for (auto& g : mg.vc_exec)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  if (mg.vc_both) { cudaGraphExecDestroy(mg.vc_both); mg.vc_both = nullptr; }
}

void mg_release_setup_graph(pff_mg& mg) {
  if (mg.su_exec) { cudaGraphExecDestroy(mg.su_exec); mg.su_exec = nullptr; }
  mg.su_key.clear();
}

// The CG run of one (block, level) chain on stream t.  Its vectors, dot products
// and coefficients are FP64; the level apply q = A p runs in the V-cycle's
// precision.  In FP32, p is rounded into and q converted out of two FP32
// vectors that take the chain's diagonal slot (free once the inverse diagonal is
// formed): the apply's rounding is relative to its operands, so the small
// residuals of a converging run keep their accuracy.
static cudaError_t setup_cg(pff_mg& mg, int b, int l, bool f32, cudaStream_t t) {
  const DevMesh& D = mg.pb->mesh->dev;
  const int nl = int(D.levels.size());
  const int64_t N = D.lev_total;
  MGBlock& B = mg.blk[b];
  const DevLevel& lv = D.levels[l].lv;
  const int64_t nn = B.ncomp * int64_t(lv.n_slots), o = B.ncomp * lv.off, vs = B.ncomp * N;
  double* r = mg.su_vec[b] + vs + o;
  double* z = mg.su_vec[b] + 2 * vs + o;
  double* p = mg.su_vec[b] + 3 * vs + o;
  double* q = mg.su_vec[b] + 4 * vs + o;
  float* p32 = reinterpret_cast<float*>(mg.su_vec[b] + o);
  float* q32 = p32 + nn;
  const int c = b * nl + l;
  double* part = mg.su_partial + int64_t(c) * mg_dot_partials();
  double* sc = mg.su_sc + 8 * c;
  double* hist = mg.su_hist + 2 * kMaxLanczos * c;
  const double* dinv = B.dinv64 + o;
  cudaError_t e = cudaSuccess;
#define SC(call) do { e = (call); if (e != cudaSuccess) return e; } while (0)
  SC(mg_start_vector(lv.n_slots, B.ncomp, D.levels[l].gx, D.levels[l].gy, dinv, r, t));
  SC(fill64(nn, q, 0.0, t));
  // z = D^-1 r, rz = r.z, p = z
  SC(cg_init_scalars(sc, t));
  SC(cg_update_r_dot(nn, r, z, q, dinv, sc, part, t));
  SC(cg_dot_final(part, sc, 0, hist, 0, t));
  SC(copy64(nn, p, z, t));
  for (int j = 0; j < mg.lanczos_steps; ++j) {
    // q = A p; pq, alpha; r -= alpha q, z = D^-1 r, rz_new, beta; p = z + beta p
    if (f32) {
      SC(f64_to_f32(nn, p, p32, t));
      SC(level_apply<float>(mg, l, block_op(b), p32, q32, t));
      SC(f32_to_f64(nn, q32, q, t));
    } else {
      SC(level_apply<double>(mg, l, block_op(b), p, q, t));
    }
    SC(dot_partial64(nn, p, q, part, t));
    SC(cg_dot_final(part, sc, 1, hist, j, t));
    SC(cg_update_r_dot(nn, r, z, q, dinv, sc, part, t));
    SC(cg_dot_final(part, sc, 2, hist, j, t));
    SC(cg_update_p(nn, p, z, sc, t));
  }
#undef SC
  return e;
}

// Launches of the set-up chains (section 1 of mg_setup) on the first K pool
// streams: one chain per (block, level), finest levels first: the inverse
// diagonal (FP64, cast to both precisions), then the CG run (its applies in the
// V-cycle's precision; level 0: FP64).
static cudaError_t launch_setup_chains(pff_mg& mg) {
  pff_problem& pb = *mg.pb;
  const DevMesh& D = pb.mesh->dev;
  const int nl = int(D.levels.size());
  constexpr int K = pff_mg::kSetupStreams;
  cudaError_t e = cudaSuccess;
  int chain = 0;
  for (int l = nl - 1; l >= 0; --l)
    for (int b = 0; b < 2; ++b, ++chain) {
      cudaStream_t t = mg.su_stream[chain % K];
      MGBlock& B = mg.blk[b];
      const DevLevel& lv = D.levels[l].lv;
      const int64_t o = B.ncomp * lv.off;
      double* diag = mg.su_vec[b] + o;
      e = level_apply<double>(mg, l, block_diag_op(b), diag, diag, t);
      if (e == cudaSuccess)
        e = mg_invert_diag(lv.n_slots, B.ncomp, diag, lv.flags, mg.cmask + lv.off, B.fixbits, B.dinv64 + o,
                           B.dinv32 + o, t);
      if (e != cudaSuccess) return e;
      if (l == 0 && mg.coarse_mode == 0) continue;
      // level 0 (the Chebyshev coarse solver's interval and degree) applies in FP64
      e = setup_cg(mg, b, l, mg.precision == PFF_F32 && l > 0, t);
      if (e != cudaSuccess) return e;
    }
  return e;
}

// What the chains' captured launches depend on besides fixed buffers
static std::vector<unsigned char> setup_key(const pff_mg& mg) {
  const pff_problem& pb = *mg.pb;
  std::vector<unsigned char> k;
  auto put = [&](const void* v, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(v);
    k.insert(k.end(), c, c + n);
  };
  put(&pb.prm, sizeof(pb.prm));
  put(&pb.has_ecell, sizeof(pb.has_ecell));
  put(&pb.lev_ecell64, sizeof(pb.lev_ecell64));
  put(&pb.lev_ecell32, sizeof(pb.lev_ecell32));
  put(&pb.sweep_sh, sizeof(pb.sweep_sh));
  put(&mg.coarse_mode, sizeof(mg.coarse_mode));
  put(&mg.lanczos_steps, sizeof(mg.lanczos_steps));
  put(&mg.precision, sizeof(mg.precision));
  return k;
}

// Capture the chains: a fork from the capture stream to the pool, the chains, a
// join back; false (no graph) if any step fails
static bool capture_setup_chains(pff_mg& mg) {
  constexpr int K = pff_mg::kSetupStreams;
  if (!mg.cap_stream && cudaStreamCreateWithFlags(&mg.cap_stream, cudaStreamNonBlocking) != cudaSuccess) return false;
  if (cudaStreamBeginCapture(mg.cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
  cudaError_t e = cudaEventRecord(mg.su_start, mg.cap_stream);
  for (int i = 0; i < K && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(mg.su_stream[i], mg.su_start, 0);
  if (e == cudaSuccess) e = launch_setup_chains(mg);
  for (int i = 0; i < K && e == cudaSuccess; ++i) {
    e = cudaEventRecord(mg.su_done[i], mg.su_stream[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(mg.cap_stream, mg.su_done[i], 0);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(mg.cap_stream, &g);
  bool ok = e == cudaSuccess && e2 == cudaSuccess && g != nullptr;
  if (ok) ok = cudaGraphInstantiate(&mg.su_exec, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    mg.su_exec = nullptr;
    cudaGetLastError();   // clear a capture error; the chains are launched directly
  }
  return ok;
}

// Lambda_max (and on level 0 the Chebyshev interval) of one (block, level) from
// the CG coefficients alpha_j, beta_j of its chain: the Lanczos tridiagonal
// d_j = 1/alpha_j + beta_{j-1}/alpha_{j-1}, e_j = sqrt(beta_j)/alpha_j.
static void eigen_from_cg(pff_mg& mg, MGBlock& B, int l, const double* hist) {
  std::vector<double> al, be;
  for (int j = 0; j < mg.lanczos_steps; ++j) {
    if (!(hist[2 * j] > 0)) break;
    al.push_back(hist[2 * j]);
    be.push_back(hist[2 * j + 1]);
  }
  const int m = int(al.size());
  std::vector<double> dd(m), ee(m > 0 ? m - 1 : 0);
  for (int j = 0; j < m; ++j) dd[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
  for (int j = 0; j + 1 < m; ++j) ee[j] = std::sqrt(std::max(be[j], 0.0)) / al[j];
  B.lam[l] = tridiag_max_eig(dd, ee);
  if (l == 0 && B.lam[0] > 0.0) {
    // Chebyshev coarse solver: both Ritz extremes of the same CG run
    B.c0_a = 0.9 * tridiag_min_eig(dd, ee);
    B.c0_b = 1.2 * B.lam[0];
    B.c0_deg = B.c0_a > 0.0 ? chebyshev_degree(B.c0_a, B.c0_b) : 0;
  }
}

std::string mg_setup(pff_mg& mg, cudaStream_t s) {
  mg_release_graphs(mg);   // the V-cycle graphs hold this set-up's coefficients
  pff_problem& pb = *mg.pb;
  const Mesh& M = pb.mesh->m;
  const DevMesh& D = pb.mesh->dev;
  const int nl = int(D.levels.size());
  const int64_t nsleaf = M.lay.n_slots;
  const int64_t N = D.lev_total;
  if (mg.lanczos_steps > kMaxLanczos) return "too many Lanczos steps";
  for (int l = 0; l < nl; ++l) {
    const DevLevel& lv = D.levels[l].lv;
    CK(mg_inject_lin(lv.n_slots, lv.slot_leaf, pb.lin64, nsleaf, mg.lin64 + 4 * lv.off, mg.lin32 + 4 * lv.off, s));
  }
  for (int l = nl - 1; l >= 0; --l) {
    const DevLevel& lv = D.levels[l].lv;
    const DevLevel* fine = (l + 1 < nl) ? &D.levels[l + 1].lv : nullptr;
    CK(mg_level_cmask(lv.n_slots, lv.flags, lv.slot_leaf, pb.cmask, fine ? fine->R_ptr : nullptr,
                      fine ? fine->R_col : nullptr, fine ? mg.cmask + fine->off : nullptr, mg.cmask + lv.off, s));
  }
  // 1. One chain per (block, level), finest levels first, spread over the stream
  //    pool: inverse diagonal, then the Jacobi-preconditioned CG run whose
  //    coefficients give lambda_max of D^-1 A on the interior (level 0: only for
  //    the Chebyshev coarse solver).  The chains share no buffer.  From the
  //    second set-up on they replay as one graph on su_side (re-captured when
  //    their arguments change); the extra pool stream K takes the second coarse
  //    inversion below either way.
  constexpr int K = pff_mg::kSetupStreams;
  if (!mg.su_start) CK(cudaEventCreateWithFlags(&mg.su_start, cudaEventDisableTiming));
  if (!mg.su_chains) CK(cudaEventCreateWithFlags(&mg.su_chains, cudaEventDisableTiming));
  if (!mg.su_side) CK(cudaStreamCreateWithFlags(&mg.su_side, cudaStreamNonBlocking));
  for (int i = 0; i <= K; ++i) {
    if (!mg.su_stream[i]) CK(cudaStreamCreateWithFlags(&mg.su_stream[i], cudaStreamNonBlocking));
    if (!mg.su_done[i]) CK(cudaEventCreateWithFlags(&mg.su_done[i], cudaEventDisableTiming));
  }
  for (int b = 0; b < 2; ++b) {
    MGBlock& B = mg.blk[b];
    for (int l = 0; l < nl; ++l) B.lam[l] = 0.0;
    B.c0_a = B.c0_b = 0.0;
    B.c0_deg = 0;
  }
  bool replay = false;
  if (mg.su_graph_ok && mg.su_setups > 0) {
    std::vector<unsigned char> key = setup_key(mg);
    if (mg.su_exec && key != mg.su_key) mg_release_setup_graph(mg);
    if (!mg.su_exec) {
      if (capture_setup_chains(mg)) mg.su_key = key;
      else mg.su_graph_ok = false;
    }
    replay = mg.su_exec != nullptr;
  }
  ++mg.su_setups;
  CK(cudaEventRecord(mg.su_start, s));
  CK(cudaStreamWaitEvent(mg.su_stream[K], mg.su_start, 0));
  if (replay) {
    CK(cudaStreamWaitEvent(mg.su_side, mg.su_start, 0));
    CK(cudaGraphLaunch(mg.su_exec, mg.su_side));
    CK(cudaEventRecord(mg.su_chains, mg.su_side));
  } else {
    for (int i = 0; i < K; ++i) CK(cudaStreamWaitEvent(mg.su_stream[i], mg.su_start, 0));
    CK(launch_setup_chains(mg));
  }
  // 2. Direct coarse solve: the dense level-0 block of each block by probing with
  //    (2k+1)^2 colours per component (all probes applied in one batch on s, beside
  //    the chains), assembled on the host and inverted on the device.
  if (mg.coarse_mode == 0) {
    const DevMesh::Level& L0 = D.levels[0];
    const LevelMesh& lm0 = M.levels[0];
    const int n0 = L0.lv.n_slots;
    std::vector<uint8_t> cm0(n0);
    CK(cudaMemcpyAsync(cm0.data(), mg.cmask + L0.lv.off, n0, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int k = M.k, Mc = 2 * k + 1;
    std::unordered_map<int64_t, int32_t> pos;  // (gx, gy) -> slot
    std::vector<int32_t> gx(n0, -1), gy(n0, -1);
    for (int q = 0; q < n0; ++q)
      if (lm0.slot_X[q] >= 0) {
        gx[q] = lm0.slot_X[q] >> M.Lf;
        gy[q] = lm0.slot_Y[q] >> M.Lf;
        pos[(int64_t(gx[q]) << 32) | gy[q]] = q;
      }
    // probe (b, c, cy, cx) at probe_base[b] + ((c * Mc + cy) * Mc + cx) * ncomp_b * n0
    int64_t probe_base[2];
    probe_base[0] = 0;
    probe_base[1] = int64_t(mg.blk[0].ncomp) * mg.blk[0].ncomp * Mc * Mc * n0;
    if (probe_base[1] + int64_t(mg.blk[1].ncomp) * mg.blk[1].ncomp * Mc * Mc * n0 > mg.probe_len)
      return "coarse probe buffer too small";
    std::vector<double> probes(size_t(mg.probe_len), 0.0), resp(size_t(mg.probe_len));
    for (int b = 0; b < 2; ++b) {
      const int nc = mg.blk[b].ncomp;
      for (int c = 0; c < nc; ++c)
        for (int cy = 0; cy < Mc; ++cy)
          for (int cx = 0; cx < Mc; ++cx) {
            double* pr = probes.data() + probe_base[b] + ((c * Mc + cy) * Mc + cx) * int64_t(nc) * n0;
            for (int q = 0; q < n0; ++q)
              if (gx[q] >= 0 && gx[q] % Mc == cx && gy[q] % Mc == cy) pr[size_t(c) * n0 + q] = 1.0;
          }
    }
    CK(cudaMemcpyAsync(mg.probe_in, probes.data(), probes.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    for (int b = 0; b < 2; ++b) {
      const int nc = mg.blk[b].ncomp;
      for (int pi = 0; pi < nc * Mc * Mc; ++pi) {
        const int64_t off = probe_base[b] + pi * int64_t(nc) * n0;
        CK(level_apply<double>(mg, 0, block_op(b), mg.probe_in + off, mg.probe_out + off, s));
      }
    }
    CK(cudaMemcpyAsync(resp.data(), mg.probe_out, resp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<double> A[2];
    std::vector<int32_t> eidx[2];
    for (int b = 0; b < 2; ++b) {
      MGBlock& B = mg.blk[b];
      const int nc = B.ncomp;
      std::vector<int32_t> ent_of(size_t(nc) * n0, -1);   // interior entries (comp * n0 + slot)
      for (int q = 0; q < n0; ++q)
        for (int c = 0; c < nc; ++c) {
          const int bit = B.fixbits == 4 ? 4 : (1 << c);
          if (gx[q] >= 0 && !(cm0[q] & bit)) {
            ent_of[size_t(c) * n0 + q] = int32_t(eidx[b].size());
            eidx[b].push_back(c * n0 + q);
          }
        }
      const int nI = int(eidx[b].size());
      A[b].assign(size_t(nI) * nI, 0.0);
      for (int c = 0; c < nc; ++c)
        for (int cy = 0; cy < Mc; ++cy)
          for (int cx = 0; cx < Mc; ++cx) {
            const double* yv = resp.data() + probe_base[b] + ((c * Mc + cy) * Mc + cx) * int64_t(nc) * n0;
            for (int q = 0; q < n0; ++q) {
              if (gx[q] < 0) continue;
              // the probed node within distance k of q in each direction
              const int jx = gx[q] - k + ((cx - (gx[q] - k)) % Mc + Mc) % Mc;
              const int jy = gy[q] - k + ((cy - (gy[q] - k)) % Mc + Mc) % Mc;
              auto it = pos.find((int64_t(jx) << 32) | jy);
              if (it == pos.end()) continue;
              const int32_t col = ent_of[size_t(c) * n0 + it->second];
              if (col < 0) continue;
              for (int cr = 0; cr < nc; ++cr) {
                const int32_t row = ent_of[size_t(cr) * n0 + q];
                if (row < 0) continue;
                A[b][size_t(row) * nI + col] = yv[size_t(cr) * n0 + q];
              }
            }
          }
      if (!B.coarse_idx || nI > B.coarse_cap) {
        const int32_t cap = std::max(nI, 1);
        B.coarse_idx = mg.mem.alloc<int32_t>(cap);
        B.coarse_inv = mg.mem.alloc<double>(int64_t(cap) * cap);
        B.coarse_tmp = mg.mem.alloc<double>(cap);
        B.coarse_rc = mg.mem.alloc<double>(mg_spd_scratch(cap));
        if (!mg.mem.err.empty()) return mg.mem.err;
        B.coarse_cap = cap;
      }
      B.n_coarse = nI;
    }
    // the two inversions run side by side (block 1 on the extra pool stream)
    for (int b = 0; b < 2; ++b) {
      MGBlock& B = mg.blk[b];
      cudaStream_t t = b == 0 ? s : mg.su_stream[K];
      CK(cudaMemsetAsync(mg.spd_bad + b, 0, sizeof(int32_t), t));
      if (B.n_coarse == 0) continue;
      CK(cudaMemcpyAsync(B.coarse_idx, eidx[b].data(), B.n_coarse * sizeof(int32_t), cudaMemcpyHostToDevice, t));
      CK(cudaMemcpyAsync(B.coarse_inv, A[b].data(), A[b].size() * sizeof(double), cudaMemcpyHostToDevice, t));
      CK(mg_spd_invert(B.n_coarse, B.coarse_inv, B.coarse_rc, mg.spd_bad + b, t));
    }
  }
  // 3. join the chains and the pool, read the CG coefficients (and coarse status) once
  if (replay) {
    CK(cudaStreamWaitEvent(s, mg.su_chains, 0));
    CK(cudaEventRecord(mg.su_done[K], mg.su_stream[K]));
    CK(cudaStreamWaitEvent(s, mg.su_done[K], 0));
  } else {
    for (int i = 0; i <= K; ++i) {
      CK(cudaEventRecord(mg.su_done[i], mg.su_stream[i]));
      CK(cudaStreamWaitEvent(s, mg.su_done[i], 0));
    }
  }
  std::vector<double> hist(size_t(2) * nl * 2 * kMaxLanczos);
  int32_t bad[2] = {0, 0};
  CK(cudaMemcpyAsync(hist.data(), mg.su_hist, hist.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (mg.coarse_mode == 0) CK(cudaMemcpyAsync(bad, mg.spd_bad, sizeof(bad), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (bad[0] || bad[1]) return "coarse level block is not positive definite";
  for (int b = 0; b < 2; ++b)
    for (int l = 0; l < nl; ++l) {
      if (l == 0 && mg.coarse_mode == 0) continue;
      eigen_from_cg(mg, mg.blk[b], l, hist.data() + size_t(b * nl + l) * 2 * kMaxLanczos);
    }
  mg.ready = true;
  return "";
}

namespace {

template <typename T>
cudaError_t vcycle_t(pff_mg& mg, int b, const double* r, double* z, cudaStream_t s) {
  pff_problem& pb = *mg.pb;
  const Mesh& M = pb.mesh->m;
  const DevMesh& D = pb.mesh->dev;
  MGBlock& B = mg.blk[b];
  const int nc = B.ncomp, nl = int(D.levels.size());
  const int64_t N = D.lev_total;
  const int64_t nsleaf = M.lay.n_slots;
  T* d = static_cast<T*>(B.d);
  T* x = static_cast<T*>(B.x);
  T* rr = static_cast<T*>(B.r);
  T* y = static_cast<T*>(B.y);
  T* yp = static_cast<T*>(B.yp);
  T* t = static_cast<T*>(B.t);
  const T* dinv = sizeof(T) == 8 ? reinterpret_cast<const T*>(B.dinv64) : reinterpret_cast<const T*>(B.dinv32);
  cudaError_t e;
#define VC(call) do { e = (call); if (e != cudaSuccess) return e; } while (0)
  // each Chebyshev step is the store of the level apply that applies A
  const bool fuse = mg.fused != 0;
  auto epi = [&](int mode, const T* prev, const T* dinv_l, const T* rhs, T* out, T* r_out, T* xprev_out, double ca,
                 double cb) {
    ChebEpi c;
    std::memset(&c, 0, sizeof(c));
    c.mode = mode; c.prev = prev; c.dinv = dinv_l; c.rhs = rhs; c.out = out; c.r = r_out; c.xprev = xprev_out;
    c.af = float(T(ca)); c.bf = float(T(cb)); c.ad = double(T(ca)); c.bd = double(T(cb));
    return c;
  };
  VC(cudaMemsetAsync(d, 0, nc * N * sizeof(T), s));
  VC(cudaMemsetAsync(x, 0, nc * N * sizeof(T), s));
  VC(mg_copy_in<T>(nsleaf, nc, D.home, r, d, pb.cmask, B.fixbits, s));
  // Chebyshev on level l over [a, bb], `degree` applications of D^-1: solve A v = rhs
  // from v = 0 into out (buffers yp, y, t).  The three iterates (current,
  // previous, next) rotate roles each step; the start is chosen so that the last
  // step writes `out`.
  auto cheb_bufs = [&](int64_t o, T* out, int degree, T*& cur, T*& prev, T*& nxt) {
    T* w0 = out;
    T* w1 = yp + o;
    T* w2 = y + o;
    switch ((degree - 1) % 3) {   // each step maps (cur, prev, nxt) to (nxt, cur, prev)
      case 0: cur = w0; prev = w1; nxt = w2; break;
      case 1: cur = w1; prev = w2; nxt = w0; break;
      default: cur = w1; prev = w0; nxt = w2; break;
    }
  };
  // first_done: the first iterate was formed with the level's defect (mg_restrict)
  auto cheb_ab = [&](int l, const T* rhs, T* out, double a, double bb, int degree, bool first_done) -> cudaError_t {
    const DevLevel& lv = D.levels[l].lv;
    const int64_t n = nc * int64_t(lv.n_slots), o = nc * lv.off;
    if (!(bb > 0) || degree < 1) return cudaMemsetAsync(out, 0, n * sizeof(T), s);
    const double theta = 0.5 * (bb + a), delta = 0.5 * (bb - a), sigma = theta / delta;
    T *cur, *prev, *nxt;
    cheb_bufs(o, out, degree, cur, prev, nxt);
    cudaError_t ee = first_done ? cudaSuccess
                                : mg_chebyshev_first<T>(n, cur, prev, dinv + o, rhs, T(1.0 / theta), s, true);
    if (ee != cudaSuccess) return ee;
    double rho = 1.0 / sigma;
    for (int j = 1; j < degree; ++j) {
      const double rho_n = 1.0 / (2.0 * sigma - rho);
      // next = cur + rho_n rho (cur - prev) + 2 rho_n / delta D^-1 (rhs - A cur)
      if (fuse) {
        const ChebEpi c = epi(CHEB_STEP, prev, dinv + o, rhs, nxt, nullptr, nullptr, rho_n * rho, 2.0 * rho_n / delta);
        ee = level_apply<T>(mg, l, block_op(b), cur, t + o, s, true, &c);
      } else {
        ee = level_apply<T>(mg, l, block_op(b), cur, t + o, s, true);
        if (ee == cudaSuccess)
          ee = mg_chebyshev_step<T>(n, nxt, cur, prev, dinv + o, rhs, t + o, T(rho_n * rho), T(2.0 * rho_n / delta),
                                    s, true);
      }
      if (ee != cudaSuccess) return ee;
      T* old_prev = prev;
      prev = cur;
      cur = nxt;
      nxt = old_prev;
      rho = rho_n;
    }
    return cudaSuccess;
  };
  // smoothing on level l >= 1: degree mg.degree on [lo, hi] * lambda_max
  auto smooths = [&](int l) { return l >= 1 && B.lam[l] > 0 && mg.degree >= 1; };
  auto cheb = [&](int l, const T* rhs, T* out, bool first_done) -> cudaError_t {
    const double lam = B.lam[l];
    return cheb_ab(l, rhs, out, mg.lo * lam, mg.hi * lam, lam > 0 ? mg.degree : 0, first_done);
  };
  // down sweep; with the fused smoother the restriction also forms the coarser
  // level's first Chebyshev iterate
  bool first_done = false;
  for (int l = nl - 1; l >= 1; --l) {
    const DevLevel& lv = D.levels[l].lv;
    const DevLevel& lc = D.levels[l - 1].lv;
    const int64_t o = nc * lv.off, oc = nc * lc.off;
    VC(cheb(l, d + o, x + o, first_done));
    VC(level_apply<T>(mg, l, block_op(b), x + o, t + o, s, true));
    first_done = fuse && smooths(l - 1);
    if (first_done) {
      const double lam = B.lam[l - 1], theta = 0.5 * (mg.lo * lam + mg.hi * lam);
      T *cur, *prev, *nxt;
      cheb_bufs(oc, x + oc, mg.degree, cur, prev, nxt);
      VC(mg_restrict<T>(lc.n_slots, nc, lc.n_slots, lv.n_slots, lv.R_ptr, lv.R_col, lv.R_val, d + o, t + o, d + oc,
                        mg.cmask + lc.off, B.fixbits, s, true, dinv + oc, cur, prev, T(1.0 / theta)));
    } else {
      VC(mg_restrict<T>(lc.n_slots, nc, lc.n_slots, lv.n_slots, lv.R_ptr, lv.R_col, lv.R_val, d + o, t + o, d + oc,
                        mg.cmask + lc.off, B.fixbits, s, true));
    }
  }
  // coarse
  if (mg.coarse_mode == 1) VC(cheb_ab(0, d, x, B.c0_a, B.c0_b, B.c0_deg, false));
  else VC(mg_coarse<T>(B.n_coarse, B.coarse_idx, B.coarse_inv, d, x, B.coarse_tmp, s, true));
  // Post-smoothing on level l of the defect d - A x, from zero, added to x: the
  // first step applies A to x and forms the defect, the last adds instead of
  // storing.  The level defect d is free once the first step has read it.
  auto cheb_post = [&](int l) -> cudaError_t {
    const DevLevel& lv = D.levels[l].lv;
    const int64_t n = nc * int64_t(lv.n_slots), o = nc * lv.off;
    const double lam = B.lam[l];
    const int degree = mg.degree;
    if (!(lam > 0) || degree < 1) return cudaSuccess;   // a zero correction
    const double a = mg.lo * lam, bb = mg.hi * lam;
    const double theta = 0.5 * (bb + a), delta = 0.5 * (bb - a), sigma = theta / delta;
    cudaError_t ee;
    if (degree == 1) {
      // x += c0 D^-1 (d - A x) reads and writes x: never fused
      ee = level_apply<T>(mg, l, block_op(b), x + o, t + o, s, true);
      if (ee != cudaSuccess) return ee;
      return mg_chebyshev_first_res<T>(n, nullptr, nullptr, nullptr, dinv + o, d + o, t + o, T(1.0 / theta), x + o, s,
                                       true);
    }
    T* cur = yp + o;
    T* prev = y + o;
    T* nxt = d + o;
    if (fuse) {
      const ChebEpi c = epi(CHEB_FIRST_RES, nullptr, dinv + o, d + o, cur, rr + o, prev, 1.0 / theta, 0.0);
      ee = level_apply<T>(mg, l, block_op(b), x + o, t + o, s, true, &c);
    } else {
      ee = level_apply<T>(mg, l, block_op(b), x + o, t + o, s, true);
      if (ee == cudaSuccess)
        ee = mg_chebyshev_first_res<T>(n, cur, prev, rr + o, dinv + o, d + o, t + o, T(1.0 / theta), nullptr, s,
                                       true);
    }
    if (ee != cudaSuccess) return ee;
    double rho = 1.0 / sigma;
    for (int j = 1; j < degree; ++j) {
      const double rho_n = 1.0 / (2.0 * sigma - rho);
      const bool last = j == degree - 1;
      if (fuse) {
        const ChebEpi c = epi(last ? CHEB_STEP_ADD : CHEB_STEP, prev, dinv + o, rr + o, last ? x + o : nxt, nullptr,
                              nullptr, rho_n * rho, 2.0 * rho_n / delta);
        ee = level_apply<T>(mg, l, block_op(b), cur, t + o, s, true, &c);
        if (ee != cudaSuccess || last) return ee;
      } else {
        ee = level_apply<T>(mg, l, block_op(b), cur, t + o, s, true);
        if (ee != cudaSuccess) return ee;
        if (last)
          return mg_chebyshev_step_add<T>(n, x + o, cur, prev, dinv + o, rr + o, t + o, T(rho_n * rho),
                                          T(2.0 * rho_n / delta), s, true);
        ee = mg_chebyshev_step<T>(n, nxt, cur, prev, dinv + o, rr + o, t + o, T(rho_n * rho), T(2.0 * rho_n / delta),
                                  s, true);
        if (ee != cudaSuccess) return ee;
      }
      T* old_prev = prev;
      prev = cur;
      cur = nxt;
      nxt = old_prev;
      rho = rho_n;
    }
    return cudaSuccess;
  };
  // up sweep
  for (int l = 1; l < nl; ++l) {
    const DevLevel& lv = D.levels[l].lv;
    const DevLevel& lc = D.levels[l - 1].lv;
    const int64_t o = nc * lv.off;
    VC(mg_prolong<T>(lv.n_slots, nc, lv.n_slots, lc.n_slots, lv.P_ptr, lv.P_col, lv.P_val, x + nc * lc.off, x + o,
                     mg.cmask + lv.off, B.fixbits, s, true));
    VC(cheb_post(l));
  }
  VC(mg_copy_out<T>(nsleaf, nc, D.home, x, r, z, pb.cmask, pb.mesh->dev.slot_flags, B.fixbits, s, true));
#undef VC
  return cudaSuccess;
}

}  // namespace

static cudaError_t vcycle_direct(pff_mg& mg, int block, const double* r, double* z, cudaStream_t s) {
  if (mg.precision == PFF_F64) return vcycle_t<double>(mg, block, r, z, s);
  return vcycle_t<float>(mg, block, r, z, s);
}

// Capture the V-cycle of one block, reading vc_in and writing vc_out at the
// block's offset; false if the graph could not be made (the direct path is used).
static bool vcycle_capture(pff_mg& mg, int block) {
  const int64_t n = mg.pb->mesh->m.lay.n_slots;
  const int64_t off = block == 0 ? 0 : 2 * n;
  if (!mg.cap_stream && cudaStreamCreateWithFlags(&mg.cap_stream, cudaStreamNonBlocking) != cudaSuccess) return false;
  if (cudaStreamBeginCapture(mg.cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
  const cudaError_t e = vcycle_direct(mg, block, mg.vc_in + off, mg.vc_out + off, mg.cap_stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(mg.cap_stream, &g);
  bool ok = e == cudaSuccess && e2 == cudaSuccess && g != nullptr;
  if (ok) ok = cudaGraphInstantiate(&mg.vc_exec[block], g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    mg.vc_exec[block] = nullptr;
    cudaGetLastError();   // clear a capture error; the direct path follows
  }
  return ok;
}

cudaError_t mg_vcycle(pff_mg& mg, int block, const double* r, double* z, cudaStream_t s) {
  if (mg.graphs_ok && mg.vc_in && mg.vc_out) {
    if (!mg.vc_exec[block] && !vcycle_capture(mg, block)) mg.graphs_ok = false;
    if (mg.vc_exec[block]) {
      const int64_t n = mg.pb->mesh->m.lay.n_slots;
      const int64_t off = block == 0 ? 0 : 2 * n;
      const size_t bytes = size_t(block == 0 ? 2 * n : n) * sizeof(double);
      cudaError_t e = cudaMemcpyAsync(mg.vc_in + off, r, bytes, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = cudaGraphLaunch(mg.vc_exec[block], s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(z, mg.vc_out + off, bytes, cudaMemcpyDeviceToDevice, s);
      return e;
    }
  }
  return vcycle_direct(mg, block, r, z, s);
}

// Capture both blocks' V-cycles as one graph.  They share no buffer (each block
// has its own level vectors, inverse diagonals and coarse data; the staging
// vectors are split at 2 n_slots), so the phi block runs on a second branch
// forked from and joined back into the capture stream.
static bool precond_capture(pff_mg& mg) {
  const int64_t n = mg.pb->mesh->m.lay.n_slots;
  if (!mg.cap_stream && cudaStreamCreateWithFlags(&mg.cap_stream, cudaStreamNonBlocking) != cudaSuccess) return false;
  if (!mg.cap_stream2 && cudaStreamCreateWithFlags(&mg.cap_stream2, cudaStreamNonBlocking) != cudaSuccess) return false;
  if (!mg.ev_fork && cudaEventCreateWithFlags(&mg.ev_fork, cudaEventDisableTiming) != cudaSuccess) return false;
  if (!mg.ev_join && cudaEventCreateWithFlags(&mg.ev_join, cudaEventDisableTiming) != cudaSuccess) return false;
  if (cudaStreamBeginCapture(mg.cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
  cudaError_t e = cudaEventRecord(mg.ev_fork, mg.cap_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(mg.cap_stream2, mg.ev_fork, 0);
  if (e == cudaSuccess) e = vcycle_direct(mg, 1, mg.vc_in + 2 * n, mg.vc_out + 2 * n, mg.cap_stream2);
  if (e == cudaSuccess) e = vcycle_direct(mg, 0, mg.vc_in, mg.vc_out, mg.cap_stream);
  if (e == cudaSuccess) e = cudaEventRecord(mg.ev_join, mg.cap_stream2);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(mg.cap_stream, mg.ev_join, 0);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(mg.cap_stream, &g);
  bool ok = e == cudaSuccess && e2 == cudaSuccess && g != nullptr;
  if (ok) ok = cudaGraphInstantiate(&mg.vc_both, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    mg.vc_both = nullptr;
    cudaGetLastError();
  }
  return ok;
}

cudaError_t mg_precond(pff_mg& mg, const double* v, double* z, cudaStream_t s) {
  const int64_t n = mg.pb->mesh->m.lay.n_slots;
  if (mg.graphs_ok && mg.vc_in && mg.vc_out) {
    if (!mg.vc_both && !precond_capture(mg)) mg.graphs_ok = false;
    if (mg.vc_both) {
      const size_t bytes = size_t(3 * n) * sizeof(double);
      cudaError_t e = cudaMemcpyAsync(mg.vc_in, v, bytes, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = cudaGraphLaunch(mg.vc_both, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(z, mg.vc_out, bytes, cudaMemcpyDeviceToDevice, s);
      return e;
    }
  }
  cudaError_t e = vcycle_direct(mg, 0, v, z, s);
  if (e == cudaSuccess) e = vcycle_direct(mg, 1, v + 2 * n, z + 2 * n, s);
  return e;
}

template cudaError_t level_apply<float>(pff_mg&, int, int, const float*, float*, cudaStream_t, bool, const ChebEpi*);
template cudaError_t level_apply<double>(pff_mg&, int, int, const double*, double*, cudaStream_t, bool,
                                         const ChebEpi*);

}  // namespace pff
