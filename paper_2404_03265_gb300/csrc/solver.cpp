// GMRES and the Newton / primal-dual active set load step (host drivers).
//
// Kolditz & Wick (arXiv 2404.03265):
//  * Sec. 3.2: left-preconditioned GMRES on P^-1 G~ dU = P^-1 R~ with
//    P^-1 = diag(MG(G~uu), MG(G~phiphi)); restart 50, classical Gram-Schmidt with
//    one re-orthogonalisation, Givens rotations, all in FP64.
//  * Algorithm 2 (with Algorithm 1): per Newton iteration the residual, the active
//    set A = { R_i / B_ii + c (phi_i - phi_i^old) > 0 }, the inhomogeneous update
//    constraint dphi = phi_old - phi on A, multigrid set-up, GMRES, hanging values
//    of the update from their constraint, and a line search U + omega^(l-1) dU
//    accepting the first decrease of the Newton residual.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "solve.cuh"
#include "state.h"

namespace pff {

#define RET(call)                                  \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return e_;              \
  } while (0)

cudaError_t leaf_op(pff_problem& pb, int kop, int mode, const double* lin, const uint8_t* cmask, const double* xu,
                    const double* xp, double* yu, double* yp, cudaStream_t s) {
  const Mesh& M = pb.mesh->m;
  const DevMesh& D = pb.mesh->dev;
  ApplyArgs a;
  std::memset(&a, 0, sizeof(a));
  a.lay = D.leaf;
  a.hang = D.hang;
  a.cmask = cmask;
  a.lin = lin;
  a.xu = xu; a.xp = xp; a.yu = yu; a.yp = yp;
  a.ibuf = pb.ibuf64;
  a.hlin = lin == pb.lin64 ? pb.hlin64 : nullptr;   // other states hold their hanging values at the nodes' slots
  a.hang_x = pb.hx64;
  a.nhang = D.nhang;
  a.n_slots = M.lay.n_slots;
  for (int l = 0; l <= M.Lf && l < kMaxLevels; ++l) { a.hx[l] = M.tree.hx(l); a.hy[l] = M.tree.hy(l); }
  leaf_modulus(pb, PFF_F64, a);
  if (kop == OP_VJP) fill_material(pb.prm, a, true);
  fill_cell_constants(a, M.Lf + 1);
  a.fe_degree = M.k;
  a.sweep_sh = pb.sweep_sh;
  a.mode = mode;
  a.cell_out = pb.cell_out;
  FixupArgs f;
  f.n = D.nfix; f.n_slots = M.lay.n_slots; f.slot = D.fix_slot; f.ptr = D.fix_ptr; f.part = D.fix_part;
  f.w = D.fix_w; f.cmask = cmask; f.xu = xu; f.xp = xp; f.yu = yu; f.yp = yp; f.ibuf = a.ibuf; f.mode = mode;
  RET(launch_apply<double>(a, kop, s));
  if (kop == OP_VJP) return cudaSuccess;  // per-cell outputs only
  return launch_fixup<double>(f, s);
}

std::string ensure_workspace(pff_problem& pb, int restart) {
  SolverWS& W = pb.ws;
  const int64_t n = pb.mesh->m.lay.n_slots;
  if (W.ready && W.restart >= restart) return "";
  W.mem.release();
  W = SolverWS();
  W.restart = restart;
  const int64_t n3 = 3 * n;
  {
    // node rows of the three blocks: the other slots are zero in every Krylov vector
    const std::vector<uint8_t>& F = pb.mesh->m.slot_flags;
    std::vector<int32_t> map;
    for (int c = 0; c < 3; ++c)
      for (int64_t i = 0; i < n; ++i)
        if (F[size_t(i)] & 1) map.push_back(int32_t(c * n + i));
    W.nc = int64_t(map.size());
    W.map = W.mem.upload(map);
  }
  W.V = W.mem.alloc<double>(size_t(basis_blocks(W.nc)) * size_t(restart + 1) * kBasisBlock);
  W.wc = W.mem.alloc<double>(W.nc);
  W.vc = W.mem.alloc<double>(n3);
  W.w = W.mem.alloc<double>(n3);
  W.tmp = W.mem.alloc<double>(n3);
  W.rhs = W.mem.alloc<double>(n3);
  W.R = W.mem.alloc<double>(n3);
  W.res = W.mem.alloc<double>(n3);
  W.dU = W.mem.alloc<double>(n3);
  W.du0 = W.mem.alloc<double>(n3);
  W.st = W.mem.alloc<double>(4 * n);
  W.ut = W.mem.alloc<double>(3 * n);
  W.B = W.mem.alloc<double>(n3);
  W.act = W.mem.alloc<uint8_t>(n);
  W.act_prev = W.mem.alloc<uint8_t>(n);
  W.stats = W.mem.alloc<unsigned long long>(4);
  W.partial = W.mem.alloc<double>(size_t(reduction_partials()) * (restart + 2));
  W.h = W.mem.alloc<double>(restart + 2);
  W.hh = W.mem.alloc<double>(2 * (restart + 1) + 1);
  W.scal = W.mem.alloc<double>(8);
  W.bad = W.mem.alloc<int>(1);
  W.x32 = W.mem.alloc<float>(n3);
  W.y32 = W.mem.alloc<float>(n3);
  if (!W.mem.err.empty()) return W.mem.err;
  if (cudaMemset(W.vc, 0, n3 * sizeof(double)) != cudaSuccess) return "workspace: cudaMemset failed";
  W.ready = true;
  return "";
}

static cudaError_t norm2(pff_problem& pb, int64_t n, const double* a, double* out_host, cudaStream_t s) {
  SolverWS& W = pb.ws;
  RET(dot64(n, a, a, W.partial, W.scal, s));
  RET(cudaMemcpyAsync(out_host, W.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  RET(cudaStreamSynchronize(s));
  *out_host = std::sqrt(*out_host);
  return cudaSuccess;
}

// P^-1 v for the full vector (u block, phi block)
static cudaError_t precond(pff_mg& mg, const double* v, double* z, cudaStream_t s) {
  return mg_precond(mg, v, z, s);
}

cudaError_t gmres_solve(pff_problem& pb, pff_mg& mg, int transpose, const double* b, double* x, double rtol,
                        int restart, int maxiter, GmresResult& res, cudaStream_t s, int matvec) {
  SolverWS& W = pb.ws;
  const int64_t n = pb.mesh->m.lay.n_slots, n3 = 3 * n;
  const int op = transpose ? OP_FULL_T : OP_FULL;
  // y = G~ v (or G~^T v); in FP32 the FP64 Krylov vectors are rounded in and out
  auto A = [&](const double* v, double* y) -> cudaError_t {
    if (matvec == PFF_F32) {
      RET(f64_to_f32(n3, v, W.x32, s));
      RET(leaf_apply(pb, PFF_F32, transpose ? PFF_OP_TRANSPOSE : PFF_OP_JACOBIAN, W.x32, W.x32 + 2 * n, W.y32,
                     W.y32 + 2 * n, s));
      return f32_to_f64(n3, W.y32, y, s);
    }
    return leaf_op(pb, op, MODE_MASK_INPUT | MODE_IDENTITY, pb.lin64, pb.cmask, v, v + 2 * n, y, y + 2 * n, s);
  };
  for (auto& e : pb.gm_ev)
    if (!e) RET(cudaEventCreate(&e));
  cudaEvent_t* ev = pb.gm_ev;
  RET(cudaMemsetAsync(x, 0, n3 * sizeof(double), s));
  const int64_t ldb = int64_t(restart + 1) * kBasisBlock;   // row-block stride of the basis
  const int64_t nc = W.nc;
  RET(precond(mg, b, W.w, s));
  RET(gather(nc, W.map, W.w, W.wc, s));
  double beta = 0.0;
  RET(norm2(pb, nc, W.wc, &beta, s));
  res = GmresResult();
  res.initial = beta;
  if (!(beta > 0.0)) {
    res.converged = std::isfinite(beta);
    res.estimate = beta;
    return cudaSuccess;
  }
  const double target = rtol * beta;
  int it = 0;
  std::vector<double> H(size_t(restart + 1) * restart), cs(restart), sn(restart), g(restart + 1),
      hh(2 * (restart + 1) + 1);
  double* h1d = W.hh;                     // first pass coefficients
  double* h2d = W.hh + (restart + 1);     // second pass
  double* nwd = W.hh + 2 * (restart + 1); // |w|^2
  while (it < maxiter) {
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    RET(store_basis(nc, W.V, ldb, 0, W.wc, 1.0 / beta, W.vc, s, W.map));
    int jd = 0;
    bool conv = false;
    for (int j = 0; j < restart; ++j) {
      // W.vc holds V_j in slot layout
      RET(cudaEventRecord(ev[0], s));
      RET(A(W.vc, W.tmp));
      RET(cudaEventRecord(ev[1], s));
      RET(precond(mg, W.tmp, W.w, s));
      RET(cudaEventRecord(ev[2], s));
      // classical Gram-Schmidt, twice, on the node rows; the coefficients stay on
      // the device until one copy brings both passes and |w|^2 to the host
      RET(gather(nc, W.map, W.w, W.wc, s));
      RET(multidot(nc, j + 1, W.V, ldb, W.wc, W.partial, h1d, s));
      RET(multi_axpy(nc, j + 1, W.V, ldb, h1d, -1.0, W.wc, s));
      RET(multidot(nc, j + 1, W.V, ldb, W.wc, W.partial, h2d, s));
      RET(multi_axpy(nc, j + 1, W.V, ldb, h2d, -1.0, W.wc, s));
      RET(dot64(nc, W.wc, W.wc, W.partial, nwd, s));
      RET(cudaEventRecord(ev[3], s));
      RET(cudaMemcpyAsync(hh.data(), W.hh, hh.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      RET(cudaStreamSynchronize(s));
      const double* h = hh.data();
      const double* h2 = hh.data() + (restart + 1);
      const double hn = std::sqrt(hh[2 * (restart + 1)]);
      float ms[3] = {0.f, 0.f, 0.f};
      for (int q = 0; q < 3; ++q) RET(cudaEventElapsedTime(&ms[q], ev[q], ev[q + 1]));
      res.t_apply += 1e-3 * ms[0];
      res.t_vcycle += 1e-3 * ms[1];
      res.t_orth += 1e-3 * ms[2];
      for (int i = 0; i <= j; ++i) H[size_t(i) * restart + j] = h[i] + h2[i];
      H[size_t(j + 1) * restart + j] = hn;
      for (int i = 0; i < j; ++i) {
        const double a0 = H[size_t(i) * restart + j], a1 = H[size_t(i + 1) * restart + j];
        H[size_t(i) * restart + j] = cs[i] * a0 + sn[i] * a1;
        H[size_t(i + 1) * restart + j] = -sn[i] * a0 + cs[i] * a1;
      }
      const double a0 = H[size_t(j) * restart + j], a1 = H[size_t(j + 1) * restart + j];
      const double den = std::hypot(a0, a1);
      if (!(den > 0.0) || !std::isfinite(den)) { res.breakdown = true; jd = j; break; }
      cs[j] = a0 / den;
      sn[j] = a1 / den;
      H[size_t(j) * restart + j] = den;
      H[size_t(j + 1) * restart + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      jd = j + 1;
      if (std::fabs(g[j + 1]) <= target || hn == 0.0 || it >= maxiter) {
        conv = std::fabs(g[j + 1]) <= target || hn == 0.0;
        break;
      }
      RET(store_basis(nc, W.V, ldb, j + 1, W.wc, 1.0 / hn, W.vc, s, W.map));
    }
    // y = H^-1 g (upper triangular), x += V y
    std::vector<double> y(jd, 0.0);
    for (int i = jd - 1; i >= 0; --i) {
      double t = g[i];
      for (int k = i + 1; k < jd; ++k) t -= H[size_t(i) * restart + k] * y[k];
      y[i] = t / H[size_t(i) * restart + i];
    }
    if (jd > 0) {
      RET(cudaMemcpyAsync(W.h, y.data(), jd * sizeof(double), cudaMemcpyHostToDevice, s));
      RET(multi_axpy(nc, jd, W.V, ldb, W.h, 1.0, x, s, W.map));
    }
    res.iterations = it;
    res.estimate = std::fabs(g[jd]);
    if (conv) { res.converged = true; return cudaSuccess; }
    if (res.breakdown) return cudaSuccess;
    // restart from the true preconditioned residual
    RET(A(x, W.tmp));
    RET(axpby(n3, W.tmp, b, 1.0, W.tmp, -1.0, s));
    RET(precond(mg, W.tmp, W.w, s));
    RET(gather(nc, W.map, W.w, W.wc, s));
    RET(norm2(pb, nc, W.wc, &beta, s));
    res.estimate = beta;
    if (beta <= target) { res.converged = true; return cudaSuccess; }
  }
  return cudaSuccess;
}

cudaError_t leaf_residual(pff_problem& pb, const double* u, const double* phi, const double* phit, double* R,
                          cudaStream_t s) {
  const Mesh& M = pb.mesh->m;
  const DevMesh& D = pb.mesh->dev;
  SolverWS& W = pb.ws;
  const int64_t n = M.lay.n_slots;
  RET(make_state(n, u, phi, phit, D.slot_flags, D.hang, D.nhang, M.k, W.st, s));
  return leaf_op(pb, OP_RESID, 0, W.st, pb.cmask_dir, R, R + 2 * n, R, R + 2 * n, s);
}

cudaError_t lumped_mass(pff_problem& pb, double* B, cudaStream_t s) {
  SolverWS& W = pb.ws;
  const int64_t n = pb.mesh->m.lay.n_slots;
  // phi component of OP_MASS is the lumped mass; state and x are not read
  return leaf_op(pb, OP_MASS, 0, W.st, pb.cmask_dir, W.tmp, W.tmp + 2 * n, W.tmp, B, s);
}

cudaError_t total_crack_volume(pff_problem& pb, const double* u, const double* phi, double* out_host, cudaStream_t s) {
  const Mesh& M = pb.mesh->m;
  const DevMesh& D = pb.mesh->dev;
  SolverWS& W = pb.ws;
  const int64_t n = M.lay.n_slots;
  RET(make_state(n, u, phi, phi, D.slot_flags, D.hang, D.nhang, M.k, W.st, s));
  RET(leaf_op(pb, OP_TCV, 0, W.st, pb.cmask_dir, W.tmp, W.tmp + 2 * n, W.tmp, W.w, s));
  RET(vsum(n, W.w, W.partial, W.scal, s));
  RET(cudaMemcpyAsync(out_host, W.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  return cudaStreamSynchronize(s);
}

// One load step of Algorithm 2.  u (2 n), phi (n) are updated in place; active (n) in/out.
cudaError_t newton_pdas_step(pff_problem& pb, pff_mg& mg, double* u, double* phi, const double* phi_old,
                             uint8_t* active, const NewtonOpts& o, NewtonInfo& info, cudaStream_t s) {
  // phi_tilde of the u-equation: the old step unless an extrapolation is given (Sec. 2)
  const double* phit = o.phi_tilde ? o.phi_tilde : phi_old;
  const Mesh& M = pb.mesh->m;
  const DevMesh& D = pb.mesh->dev;
  SolverWS& W = pb.ws;
  const int64_t n = M.lay.n_slots, n3 = 3 * n;
  info = NewtonInfo();
  // lumped mass (phi block of B)
  RET(lumped_mass(pb, W.B + 2 * n, s));
  RET(cudaMemcpyAsync(W.act_prev, active, n, cudaMemcpyDeviceToDevice, s));
  double r0 = -1.0;
  for (int k = 0; k <= o.max_newton; ++k) {
    // residual and active set at U^k
    RET(leaf_residual(pb, u, phi, phit, W.R, s));
    RET(cudaMemsetAsync(W.stats, 0, 2 * sizeof(unsigned long long), s));
    const unsigned long long big = 0x7ff0000000000000ull;
    RET(cudaMemcpyAsync(W.stats + 2, &big, sizeof(big), cudaMemcpyHostToDevice, s));
    RET(active_set(n, W.R, W.B + 2 * n, phi, phi_old, D.slot_flags, pb.prm.c, W.act_prev, W.act, W.stats, s));
    RET(newton_residual(n, W.R, W.act, phi, phi_old, D.slot_flags, W.res, s));
    double nres = 0.0;
    RET(norm2(pb, n3, W.res, &nres, s));
    unsigned long long st[3];
    RET(cudaMemcpyAsync(st, W.stats, sizeof(st), cudaMemcpyDeviceToHost, s));
    RET(cudaStreamSynchronize(s));
    if (!std::isfinite(nres)) { info.nonfinite = true; return cudaSuccess; }
    if (r0 < 0) r0 = nres;
    info.residual.push_back(nres);
    info.active_size.push_back(int64_t(st[1]));
    info.changes.push_back(int64_t(st[0]));
    double margin;
    std::memcpy(&margin, &st[2], sizeof(double));
    info.margin = margin;
    info.residual0 = r0;
    if (st[0] == 0 && nres <= std::max(o.tol * r0, o.atol)) {
      info.converged = true;
      RET(cudaMemcpyAsync(active, W.act, n, cudaMemcpyDeviceToDevice, s));
      return cudaStreamSynchronize(s);
    }
    if (k == o.max_newton) break;
    // linearisation, constraints, right-hand side with the inhomogeneous constraint on A
    RET(launch_set_lin(n, u, phi, phit, D.hang, D.nhang, M.k, pb.lin64, pb.lin32, pb.hlin64, pb.hlin32, s));
    pb.has_state = true;
    RET(launch_leaf_cmask(n, D.slot_flags, W.act, pb.cmask, s));
    RET(newton_du0(n, W.act, phi, phi_old, W.du0, s));
    RET(leaf_op(pb, OP_FULL, 0, pb.lin64, pb.cmask, W.du0, W.du0 + 2 * n, W.tmp, W.tmp + 2 * n, s));
    RET(newton_rhs(n, W.R, W.tmp, W.act, phi, phi_old, D.slot_flags, W.rhs, s));
    const auto t_setup0 = std::chrono::steady_clock::now();
    std::string e = mg_setup(mg, s);
    const auto t_setup1 = std::chrono::steady_clock::now();
    info.t_setup += std::chrono::duration<double>(t_setup1 - t_setup0).count();
    if (!e.empty()) { info.error = e; return cudaErrorUnknown; }
    GmresResult gr;
    RET(gmres_solve(pb, mg, 0, W.rhs, W.dU, o.gmres_rtol, o.restart, o.gmres_maxiter, gr, s, o.matvec));
    info.t_gmres += std::chrono::duration<double>(std::chrono::steady_clock::now() - t_setup1).count();
    info.gmres.push_back(gr.iterations);
    info.t_apply += gr.t_apply;
    info.t_vcycle += gr.t_vcycle;
    info.t_orth += gr.t_orth;
    if (gr.breakdown) info.gmres_breakdown = true;
    // G~ is the identity on the fixed rows and couples them to no free row, so the
    // fixed part of the solution is the right-hand side there, taken exactly
    // (phi_old - phi on the active set: the step lands on phi_old)
    RET(copy_fixed(n, pb.cmask, W.rhs, W.dU, s));
    RET(distribute_hanging(n, D.hang, D.nhang, M.k, 3, W.dU, s));
    // line search on the Newton residual under the current active set
    bool accepted = false;
    double w = 1.0;
    for (int l = 1; l <= o.ls_max; ++l) {
      RET(axpby(2 * n, W.ut, u, 1.0, W.dU, w, s));
      RET(axpby(n, W.ut + 2 * n, phi, 1.0, W.dU + 2 * n, w, s));
      RET(leaf_residual(pb, W.ut, W.ut + 2 * n, phit, W.R, s));
      RET(newton_residual(n, W.R, W.act, W.ut + 2 * n, phi_old, D.slot_flags, W.res, s));
      double nt = 0.0;
      RET(norm2(pb, n3, W.res, &nt, s));
      if (nt < nres) { accepted = true; break; }
      if (l < o.ls_max) w *= o.omega;
    }
    if (!accepted) ++info.linesearch_failures;
    RET(cudaMemcpyAsync(u, W.ut, 2 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RET(cudaMemcpyAsync(phi, W.ut + 2 * n, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RET(cudaMemcpyAsync(W.act_prev, W.act, n, cudaMemcpyDeviceToDevice, s));
    info.newton = k + 1;
  }
  RET(cudaMemcpyAsync(active, W.act_prev, n, cudaMemcpyDeviceToDevice, s));
  return cudaStreamSynchronize(s);
}

}  // namespace pff
