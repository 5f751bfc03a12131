// Crack opening displacement profile (Sec. 4): COD(x) = integral over y of
// u . grad phi along the vertical line at x, by the (k+1)-point Gauss rule in y on
// every leaf cell the line crosses.  A cell [x0, x0 + hx) contains x when
// x0 <= x < x0 + hx (x0 = domain x0 + i hx in FP64).
//
// The host lists, per line, the crossed cells (canonical order) with the local
// coordinate xi of the line and the storage slots of the cell's nodes; one block
// per line sums the contributions in a fixed order (deterministic).
#include <algorithm>
#include <cmath>
#include <unordered_map>
#include <vector>

#include "solve.cuh"
#include "state.h"

namespace pff {

namespace {

constexpr int COD_T = 128;

struct CodEntry {
  double xi, hx, hy;
  int32_t slot[9];   // (k+1)^2 node slots, local index a + (k+1) b
};

__device__ __forceinline__ void lag(int k, double t, double* L, double* dL) {
  if (k == 1) {
    L[0] = 1.0 - t; L[1] = t;
    dL[0] = -1.0; dL[1] = 1.0;
  } else {
    L[0] = 2.0 * (t - 0.5) * (t - 1.0); L[1] = -4.0 * t * (t - 1.0); L[2] = 2.0 * t * (t - 0.5);
    dL[0] = 4.0 * t - 3.0; dL[1] = 4.0 - 8.0 * t; dL[2] = 4.0 * t - 1.0;
  }
}

__global__ void k_cod(int k, const int32_t* __restrict__ ptr, const CodEntry* __restrict__ ent,
                      const double* __restrict__ st, int64_t n, const double* __restrict__ eta,
                      const double* __restrict__ weta, double* out) {
  __shared__ double red[COD_T];
  const int line = blockIdx.x;
  double acc = 0.0;
  for (int e = ptr[line] + threadIdx.x; e < ptr[line + 1]; e += COD_T) {
    const CodEntry E = ent[e];
    double Lx[3], dLx[3];
    lag(k, E.xi, Lx, dLx);
    double tot = 0.0;
    for (int q = 0; q <= k; ++q) {
      double Ly[3], dLy[3];
      lag(k, eta[q], Ly, dLy);
      double ux = 0, uy = 0, px = 0, py = 0;
      for (int b = 0; b <= k; ++b)
        for (int a = 0; a <= k; ++a) {
          const int s = E.slot[a + (k + 1) * b];
          const double N = Lx[a] * Ly[b];
          ux += N * st[s];
          uy += N * st[n + s];
          px += dLx[a] / E.hx * Ly[b] * st[2 * n + s];
          py += Lx[a] * dLy[b] / E.hy * st[2 * n + s];
        }
      tot += weta[q] * (ux * px + uy * py);
    }
    acc += E.hy * tot;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = COD_T / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[line] = red[0];
}

}  // namespace

std::string cod_profile(pff_problem& pb, const double* u, const double* phi, const double* x, int nx, double* out_host,
                        cudaStream_t s) {
  const Mesh& M = pb.mesh->m;
  const DevMesh& D = pb.mesh->dev;
  const Tree& t = M.tree;
  const int k = M.k, nb1 = k + 1;
  // cells per (level, column i)
  std::vector<std::unordered_map<int64_t, std::vector<int32_t>>> col(M.Lf + 1);
  for (size_t c = 0; c < M.leaves.size(); ++c) col[M.leaves[c][0]][M.leaves[c][1]].push_back(int32_t(c));
  std::vector<int32_t> ptr(1, 0);
  std::vector<CodEntry> ent;
  for (int q = 0; q < nx; ++q) {
    std::vector<int32_t> cells;
    for (int l = 0; l <= M.Lf; ++l) {
      const double hx = t.hx(l);
      const int64_t ic = int64_t(std::floor((x[q] - t.x0) / hx));
      for (int64_t i = ic - 1; i <= ic + 1; ++i) {
        auto it = col[l].find(i);
        if (it == col[l].end()) continue;
        const double x0 = t.x0 + double(i) * hx;
        if (!(x0 <= x[q] && x[q] < x0 + hx)) continue;
        cells.insert(cells.end(), it->second.begin(), it->second.end());
      }
    }
    std::sort(cells.begin(), cells.end());
    for (int32_t c : cells) {
      const auto& lc = M.leaves[c];
      const int l = int(lc[0]);
      const double hx = t.hx(l), hy = t.hy(l);
      CodEntry E{};
      E.xi = (x[q] - (t.x0 + double(lc[1]) * hx)) / hx;
      E.hx = hx;
      E.hy = hy;
      const int64_t s = int64_t(1) << (M.Lf - l);
      for (int b = 0; b <= k; ++b)
        for (int a = 0; a <= k; ++a) {
          const int64_t n = M.find_node((lc[1] * k + a) * s, (lc[2] * k + b) * s);
          if (n < 0) return "COD: missing node of a leaf cell";
          E.slot[a + nb1 * b] = M.nslot[n];
        }
      ent.push_back(E);
    }
    ptr.push_back(int32_t(ent.size()));
  }
  // (k+1)-point Gauss rule on [0, 1]
  std::vector<double> eta, weta;
  if (k == 1) {
    eta = {0.5 - 0.5 / std::sqrt(3.0), 0.5 + 0.5 / std::sqrt(3.0)};
    weta = {0.5, 0.5};
  } else {
    eta = {0.5 - 0.1 * std::sqrt(15.0), 0.5, 0.5 + 0.1 * std::sqrt(15.0)};
    weta = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  }
  DevAllocs tmp;
  int32_t* dptr = tmp.upload(ptr);
  CodEntry* dent = tmp.upload(ent);
  double* deta = tmp.upload(eta);
  double* dw = tmp.upload(weta);
  double* dout = tmp.alloc<double>(std::max(nx, 1));
  std::string err = tmp.err;
  SolverWS& W = pb.ws;
  const int64_t n = M.lay.n_slots;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && err.empty()) err = cudaGetErrorString(e);
  };
  if (err.empty()) ck(make_state(n, u, phi, phi, D.slot_flags, D.hang, D.nhang, k, W.st, s));
  if (err.empty() && nx > 0) {
    k_cod<<<nx, COD_T, 0, s>>>(k, dptr, dent, W.st, n, deta, dw, dout);
    ck(cudaGetLastError());
  }
  if (err.empty()) ck(cudaMemcpyAsync(out_host, dout, nx * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (err.empty()) ck(cudaStreamSynchronize(s));
  tmp.release();
  return err;
}

}  // namespace pff
