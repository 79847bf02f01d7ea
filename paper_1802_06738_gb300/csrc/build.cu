// pno_build: device setup of one system (Sec. 2 of arXiv:1802.06738).
//
//  1. T1 dressing of the Hamiltonian (exp(-T1) H exp(T1): B~ = (1-k) B (1+k),
//     h~ likewise) so that every later formula contains T2 only;
//  2. T2 from Eq. T1 when the caller gives none;
//  3. CIS singlet roots, CIS(D) doubles (Eq. cis_d), state-averaged pair
//     densities (Eq. eom:sa_density);
//  4. batched eigendecompositions -> PNOs (T_CutPNO) and OSVs (T_CutOSV),
//     semicanonicalised;
//  5. R-independent intermediates of the closed-shell EOM-CCSD Jacobian and
//     their projections into PNO/OSV spaces: the operator "pool" and the
//     problem lists of the sigma program.
#include "pno.cuh"
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>

namespace pnoeom {
namespace {

using DV = DBuf<double>;
using Dims = std::map<char, int64_t>;

inline unsigned gsz(size_t n) { return (unsigned)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 32)); }
#define GRID_STRIDE(e, n) for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)(n); e += (int64_t)gridDim.x * blockDim.x)

// dst[Q][r][c] = src[Q][r0 + r][c0 + c]
__global__ void k_slice3(double* dst, const double* src, int nq, int nmo, int r0, int nr, int c0, int nc) {
  GRID_STRIDE(e, (int64_t)nq * nr * nc) {
    int64_t q = e / ((int64_t)nr * nc);
    int rc = (int)(e % ((int64_t)nr * nc));
    int r = rc / nc, c = rc % nc;
    dst[e] = src[(q * nmo + r0 + r) * nmo + c0 + c];
  }
}
// gam[Q] = sum_{k<o} B[Q][k][k]
__global__ void k_trace_occ(double* gam, const double* B, int nq, int nmo, int o) {
  GRID_STRIDE(q, nq) {
    double s = 0;
    for (int k = 0; k < o; ++k) s += B[((int64_t)q * nmo + k) * nmo + k];
    gam[q] = s;
  }
}
// x[i,j,a,b] /= (e_i + e_j - e_a - e_b + shift), |denominator| clamped to >= clamp (if clamp > 0)
__global__ void k_pair_div(double* x, const double* eps, int o, int v, double shift, double clamp) {
  GRID_STRIDE(e, (int64_t)o * o * v * v) {
    int b = (int)(e % v); int64_t r = e / v;
    int a = (int)(r % v); r /= v;
    int j = (int)(r % o); int i = (int)(r / o);
    double d = shift + eps[i] + eps[j] - eps[o + a] - eps[o + b];
    if (clamp > 0 && fabs(d) < clamp) d = d < 0 ? -clamp : clamp;
    x[e] /= d;
  }
}
// A[(i,a),(i,a)] += e_a - e_i
__global__ void k_cis_diag(double* A, const double* eps, int o, int v) {
  GRID_STRIDE(e, (int64_t)o * v) {
    int i = (int)(e / v), a = (int)(e % v);
    A[e * (int64_t)o * v + e] += eps[o + a] - eps[i];
  }
}
// U_raw[a][c] = evec[(v - n + c) * v + a] (kept eigenvectors of a column-major v x v matrix)
__global__ void k_extract_kept(double* U, const double* evec, int v, int n) {
  GRID_STRIDE(e, (int64_t)v * n) {
    int a = (int)(e / n), c = (int)(e % n);
    U[e] = evec[(int64_t)(v - n + c) * v + a];
  }
}
// F[c][d] = sum_a U[a][c] f[a] U[a][d], padded into nmax x nmax with diag(1e3 + k)
__global__ void k_fbar_padded(double* Fp, const double* U, const double* f, int v, int n, int nmax) {
  GRID_STRIDE(e, (int64_t)nmax * nmax) {
    int c = (int)(e / nmax), d = (int)(e % nmax);
    double s = 0;
    if (c < n && d < n) {
      for (int a = 0; a < v; ++a) s += U[(int64_t)a * n + c] * f[a] * U[(int64_t)a * n + d];
    } else if (c == d) {
      s = 1.0e3 + c;
    }
    Fp[e] = s;
  }
}
// flip columns of U (v x n) so that the entry of largest magnitude (first on ties) is positive
__global__ void k_sign_fix(double* U, int v, int n) {
  int c = blockIdx.x;
  if (c >= n) return;
  __shared__ double bv[256];
  __shared__ int bi[256];
  double best = -1; int bidx = v;
  for (int a = threadIdx.x; a < v; a += blockDim.x) {
    double x = fabs(U[(int64_t)a * n + c]);
    if (x > best || (x == best && a < bidx)) { best = x; bidx = a; }
  }
  bv[threadIdx.x] = best; bi[threadIdx.x] = bidx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      double x = bv[threadIdx.x + s]; int ix = bi[threadIdx.x + s];
      if (x > bv[threadIdx.x] || (x == bv[threadIdx.x] && ix < bi[threadIdx.x])) { bv[threadIdx.x] = x; bi[threadIdx.x] = ix; }
    }
    __syncthreads();
  }
  bool flip = U[(int64_t)bi[0] * n + c] < 0;
  __syncthreads();
  if (flip)
    for (int a = threadIdx.x; a < v; a += blockDim.x) U[(int64_t)a * n + c] = -U[(int64_t)a * n + c];
}
// diagonal-pair symmetrisation helper for denominators etc. is host side.

// ------------------------------------------------------------------------
struct Builder {
  pnoeom_ctx* ctx;
  const pnoeom_opts* opt;
  cudaStream_t s;
  pnoeom_pno* P;
  int o, v, naux, nmo;
  Dims dm;
  size_t* fp;

  void sync() { PN_CUDA(cudaStreamSynchronize(s)); }

  template <typename F>
  void launch_check(F f) { f(); PN_CUDA(cudaGetLastError()); }

  void con(const char* a, const double* A, const char* b, const double* B, const char* c, double* C,
           double alpha = 1.0, double beta = 0.0, const Dims* d = nullptr) {
    contract<double>(d ? *d : dm, TView<double>{const_cast<double*>(A), a}, TView<double>{const_cast<double*>(B), b},
                     TView<double>{C, c}, alpha, beta, s);
  }
  void perm(const double* in, double* out, std::vector<int64_t> dims, std::vector<int> p, double al, double be) {
    permute<double>(in, out, dims, p, al, be, s);
  }
  DV slice(const DV& B, int r0, int nr, int c0, int nc) {
    DV d((size_t)naux * nr * nc);
    k_slice3<<<gsz(d.n), 256, 0, s>>>(d.get(), B.get(), naux, nmo, r0, nr, c0, nc);
    PN_CUDA(cudaGetLastError());
    return d;
  }
};

void eig_dense_sym(cusolverDnHandle_t h, cudaStream_t s, double* A, double* W, int64_t n, int64_t batch) {
  // column-major symmetric eigendecomposition, eigenvalues ascending, eigenvectors overwrite A
  cusolverDnParams_t params;
  PN_SOLVER(cusolverDnCreateParams(&params));
  PN_SOLVER(cusolverDnSetStream(h, s));
  size_t dws = 0, hws = 0;
  DBuf<int> info(std::max<int64_t>(1, batch));
  if (batch == 1) {
    PN_SOLVER(cusolverDnXsyevd_bufferSize(h, params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, A, n,
                                          CUDA_R_64F, W, CUDA_R_64F, &dws, &hws));
    DBuf<unsigned char> dw(std::max<size_t>(dws, 1));
    std::vector<unsigned char> hw(std::max<size_t>(hws, 1));
    PN_SOLVER(cusolverDnXsyevd(h, params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, A, n,
                               CUDA_R_64F, W, CUDA_R_64F, dw.get(), dws, hw.data(), hws, info.get()));
    PN_CUDA(cudaStreamSynchronize(s));
  } else {
    PN_SOLVER(cusolverDnXsyevBatched_bufferSize(h, params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, A,
                                                n, CUDA_R_64F, W, CUDA_R_64F, &dws, &hws, batch));
    DBuf<unsigned char> dw(std::max<size_t>(dws, 1));
    std::vector<unsigned char> hw(std::max<size_t>(hws, 1));
    PN_SOLVER(cusolverDnXsyevBatched(h, params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, A, n,
                                     CUDA_R_64F, W, CUDA_R_64F, dw.get(), dws, hw.data(), hws, info.get(), batch));
    PN_CUDA(cudaStreamSynchronize(s));
  }
  std::vector<int> hinfo(info.n);
  info.download(hinfo.data(), info.n, s);
  PN_CUDA(cudaStreamSynchronize(s));
  cusolverDnDestroyParams(params);
  for (int x : hinfo) PN_CHECK(x == 0, PNOEOM_ERR_CUDA, "eigensolver info != 0: " + std::to_string(x));
}

// Lowest `nev` eigenpairs of a symmetric n x n matrix (cuSOLVER Xsyevdx, index
// range 1..nev).  Eigenvalues ascending into W, eigenvectors into the first nev
// columns (column-major) of A.
void eig_lowest(cusolverDnHandle_t h, cudaStream_t s, double* A, double* W, int64_t n, int64_t nev) {
  cusolverDnParams_t params;
  PN_SOLVER(cusolverDnCreateParams(&params));
  PN_SOLVER(cusolverDnSetStream(h, s));
  size_t dws = 0, hws = 0;
  int64_t found = 0;
  double vl = 0, vu = 0;
  PN_SOLVER(cusolverDnXsyevdx_bufferSize(h, params, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_LOWER,
                                         n, CUDA_R_64F, A, n, &vl, &vu, 1, nev, &found, CUDA_R_64F, W, CUDA_R_64F, &dws,
                                         &hws));
  DBuf<unsigned char> dw(std::max<size_t>(dws, 1));
  std::vector<unsigned char> hw(std::max<size_t>(hws, 1));
  DBuf<int> info(1);
  PN_SOLVER(cusolverDnXsyevdx(h, params, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_LOWER, n,
                              CUDA_R_64F, A, n, &vl, &vu, 1, nev, &found, CUDA_R_64F, W, CUDA_R_64F, dw.get(), dws,
                              hw.data(), hws, info.get()));
  int hinfo = 0;
  PN_CUDA(cudaMemcpyAsync(&hinfo, info.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  PN_CUDA(cudaStreamSynchronize(s));
  cusolverDnDestroyParams(params);
  PN_CHECK(hinfo == 0 && found >= nev, PNOEOM_ERR_CUDA, "partial eigensolver failed (info " + std::to_string(hinfo) + ")");
}

// Lowest `nev` eigenpairs of a symmetric n x n device matrix A (row-major = column-major)
// by block Davidson in FP64: start from unit vectors at the smallest diagonal entries,
// residuals r = A x - theta x preconditioned by 1 / (theta - A_ii) (|.| >= 1e-4), Gram-Schmidt
// twice, subspace of at most 12 blocks with a restart onto the current Ritz vectors.
// Converged when every ||r|| <= tol.  Eigenvalues ascending into W (host), eigenvectors
// into X (device, nev x n row-major).
void eig_lowest_davidson(cusolverDnHandle_t h, cudaStream_t s, const double* A, int64_t n, int nev, double tol,
                         double* W, double* X) {
  const int nb = std::min<int64_t>(n, nev + 4);
  const int maxsub = (int)std::min<int64_t>(n, 12 * nb);
  std::vector<double> diag(n);
  PN_CUDA(cudaMemcpy2DAsync(diag.data(), 8, A, (n + 1) * 8, 8, n, cudaMemcpyDeviceToHost, s));
  PN_CUDA(cudaStreamSynchronize(s));
  DBuf<double> V((size_t)maxsub * n), AV((size_t)maxsub * n), T((size_t)nb * n), G((size_t)maxsub * maxsub),
      Gw(maxsub), C((size_t)maxsub * nb);
  // V, AV, T store vectors as rows (vector k at k * n)
  std::vector<int64_t> order(n);
  for (int64_t e = 0; e < n; ++e) order[e] = e;
  std::partial_sort(order.begin(), order.begin() + nb, order.end(), [&](int64_t a, int64_t b) { return diag[a] < diag[b]; });
  {
    std::vector<double> t((size_t)nb * n, 0.0);
    for (int k = 0; k < nb; ++k) t[(size_t)k * n + order[k]] = 1.0;
    V.upload(t.data(), t.size(), s);
  }
  auto gemm = [&](const double* a, const double* b, double* c, int M, int N, int K, int lda, int ldb, int ldc, int ta, int tb,
                  double al, double be) {
    grouped_gemm<double>({{a, b, c, M, N, K, lda, ldb, ldc, ta, tb, al, be}}, s);
  };
  int m = nb;                                     // vectors in V
  gemm(V.get(), A, AV.get(), m, (int)n, (int)n, (int)n, (int)n, (int)n, 0, 0, 1.0, 0.0);   // AV = V A (A symmetric)
  std::vector<double> g, ev, res(nb);
  bool done = false;
  for (int it = 0; it < 200 && !done; ++it) {
    gemm(V.get(), AV.get(), G.get(), m, m, (int)n, (int)n, (int)n, m, 0, 1, 1.0, 0.0);       // G = V AV^T
    eig_dense_sym(h, s, G.get(), Gw.get(), m, 1);                                          // column k = eigenvector k
    ev.resize(m);
    Gw.download(ev.data(), m, s);
    // C (nb x m): the lowest nb eigenvectors as rows
    g.resize((size_t)m * m);
    G.download(g.data(), g.size(), s);
    PN_CUDA(cudaStreamSynchronize(s));
    std::vector<double> c((size_t)nb * m);
    for (int k = 0; k < nb; ++k)
      for (int q = 0; q < m; ++q) c[(size_t)k * m + q] = g[(size_t)k * m + q];
    C.upload(c.data(), c.size(), s);
    // Ritz vectors X_k = C V, residuals T_k = C AV - theta_k X_k
    DBuf<double> Xr((size_t)nb * n);
    gemm(C.get(), V.get(), Xr.get(), nb, (int)n, m, m, (int)n, (int)n, 0, 0, 1.0, 0.0);
    gemm(C.get(), AV.get(), T.get(), nb, (int)n, m, m, (int)n, (int)n, 0, 0, 1.0, 0.0);
    std::vector<double> xr((size_t)nb * n), tr((size_t)nb * n);
    Xr.download(xr.data(), xr.size(), s);
    T.download(tr.data(), tr.size(), s);
    PN_CUDA(cudaStreamSynchronize(s));
    double worst = 0;
    for (int k = 0; k < nb; ++k) {
      double r2 = 0;
      for (int64_t e = 0; e < n; ++e) {
        double r = tr[(size_t)k * n + e] - ev[k] * xr[(size_t)k * n + e];
        tr[(size_t)k * n + e] = r;
        r2 += r * r;
      }
      res[k] = std::sqrt(r2);
      if (k < nev) worst = std::max(worst, res[k]);
    }
    if (worst <= tol) {
      for (int k = 0; k < nev; ++k) W[k] = ev[k];
      PN_CUDA(cudaMemcpyAsync(X, Xr.get(), (size_t)nev * n * 8, cudaMemcpyDeviceToDevice, s));
      done = true;
      break;
    }
    // restart when the next block does not fit
    if (m + nb > maxsub) {
      DBuf<double> AX((size_t)nb * n);
      gemm(C.get(), AV.get(), AX.get(), nb, (int)n, m, m, (int)n, (int)n, 0, 0, 1.0, 0.0);
      PN_CUDA(cudaMemcpyAsync(V.get(), Xr.get(), (size_t)nb * n * 8, cudaMemcpyDeviceToDevice, s));
      PN_CUDA(cudaMemcpyAsync(AV.get(), AX.get(), (size_t)nb * n * 8, cudaMemcpyDeviceToDevice, s));
      m = nb;
    }
    // preconditioned residuals, orthogonalised against V (twice) and among themselves
    int added = 0;
    for (int k = 0; k < nb; ++k) {
      if (res[k] <= tol * 1e-3) continue;
      std::vector<double> tk(n);
      double n0 = 0;
      for (int64_t e = 0; e < n; ++e) {
        double den = ev[k] - diag[e];
        if (std::fabs(den) < 1e-4) den = den < 0 ? -1e-4 : 1e-4;
        tk[e] = tr[(size_t)k * n + e] / den;
        n0 += tk[e] * tk[e];
      }
      n0 = std::sqrt(n0);
      if (!(n0 > 0)) continue;
      for (double& x : tk) x /= n0;   // unit length before the projection: what survives it is new
      DBuf<double> tv(n), ov(m + added);
      tv.upload(tk.data(), n, s);
      for (int pass = 0; pass < 2; ++pass) {
        gemm(V.get(), tv.get(), ov.get(), m + added, 1, (int)n, (int)n, 1, 1, 0, 0, 1.0, 0.0);
        gemm(V.get(), ov.get(), tv.get(), (int)n, 1, m + added, (int)n, 1, 1, 1, 0, -1.0, 1.0);
      }
      tv.download(tk.data(), n, s);
      PN_CUDA(cudaStreamSynchronize(s));
      double nrm = 0;
      for (double x : tk) nrm += x * x;
      nrm = std::sqrt(nrm);
      if (nrm < 1e-6) continue;
      for (double& x : tk) x /= nrm;
      PN_CUDA(cudaMemcpyAsync(V.get() + (size_t)(m + added) * n, tk.data(), n * 8, cudaMemcpyHostToDevice, s));
      PN_CUDA(cudaStreamSynchronize(s));
      ++added;
    }
    PN_CHECK(added > 0, PNOEOM_ERR_NOT_CONVERGED, "CIS Davidson: no new direction before convergence");
    gemm(V.get() + (size_t)m * n, A, AV.get() + (size_t)m * n, added, (int)n, (int)n, (int)n, (int)n, (int)n, 0, 0, 1.0, 0.0);
    m += added;
  }
  PN_CHECK(done, PNOEOM_ERR_NOT_CONVERGED, "CIS Davidson did not converge");
}

}  // namespace

// Above this many singles the CIS roots come from the Davidson solver above.
constexpr int64_t CIS_DENSE_MAX = 6000;

// Pool-block bookkeeping on the host.
struct PoolPlan {
  int64_t size = 0;
  int64_t add(int64_t n) { int64_t off = size; size += n; return off; }
};

void build_system(pnoeom_ctx* ctx, const pnoeom_system* sys, const pnoeom_opts* opts, cudaStream_t s, pnoeom_pno* P) {
  auto t_start = std::chrono::steady_clock::now();
  const int o = sys->o, v = sys->v, naux = sys->naux, nmo = o + v;
  PN_CHECK(o >= 1 && v >= 1 && naux >= 1, PNOEOM_ERR_INVALID_ARG, "o, v and naux must be positive");
  PN_CHECK(sys->eps && sys->B, PNOEOM_ERR_INVALID_ARG, "eps and B are required");
  PN_CHECK(opts->nroots_sa >= 1 && opts->nroots_sa <= o * v, PNOEOM_ERR_INVALID_ARG, "nroots_sa out of range");
  PN_CHECK(opts->t_pno_gs >= 0.0, PNOEOM_ERR_INVALID_ARG, "t_pno_gs must be >= 0");
  PN_CHECK(opts->state_specific >= 0 && opts->state_specific <= opts->nroots_sa, PNOEOM_ERR_INVALID_ARG,
           "state_specific must be 0 (state-averaged) or a CIS root in 1..nroots_sa");
  PN_CHECK(opts->t_pno >= 0, PNOEOM_ERR_INVALID_ARG, "t_pno must be >= 0");
  P->o = o; P->v = v; P->naux = naux; P->nroots_sa = opts->nroots_sa;
  P->t_pno = opts->t_pno;
  P->t_osv = opts->t_osv < 0 ? opts->t_pno / 10.0 : opts->t_osv;
  P->has_t1 = sys->t1 != nullptr;
  size_t* fp = &P->footprint;
  Builder bd{ctx, opts, s, P, o, v, naux, nmo, {}, fp};
  bd.dm = Dims{};
  const int64_t O = o, V = v, N = naux;
  // letters: occupied i j k l m ; virtual a b c d ; aux Q ; PNO/OSV indices set per call
  for (char c : std::string("ijklm")) bd.dm[c] = O;
  for (char c : std::string("abcd")) bd.dm[c] = V;
  bd.dm['Q'] = N;
  bd.dm['p'] = nmo; bd.dm['q'] = nmo; bd.dm['r'] = nmo; bd.dm['s'] = nmo;
  const cudaMemcpyKind kind = sys->mem_space == PNOEOM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;

  // ---- inputs ---------------------------------------------------------------
  P->eps.resize(nmo);
  PN_CUDA(cudaMemcpyAsync(P->eps.data(), sys->eps, nmo * sizeof(double),
                          sys->mem_space == PNOEOM_DEVICE ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
  DV deps(nmo);
  PN_CUDA(cudaMemcpyAsync(deps.get(), sys->eps, nmo * sizeof(double), kind, s));
  DV dB((size_t)N * nmo * nmo);
  PN_CUDA(cudaMemcpyAsync(dB.get(), sys->B, dB.n * sizeof(double), kind, s));
  bd.sync();
  StageTimer tm(s);
  tm.mark("inputs");
  const std::vector<double>& eps = P->eps;

  // undressed blocks (CIS, CIS(D), MP1 use the HF Hamiltonian)
  DV Boo = bd.slice(dB, 0, o, 0, o), Bov = bd.slice(dB, 0, o, o, v), Bvo = bd.slice(dB, o, v, 0, o), Bvv = bd.slice(dB, o, v, o, v);

  // ---- T1 dressing (Sec. 2 equations contain T2 only afterwards) --------------
  std::vector<double> Fd((size_t)nmo * nmo, 0.0);
  DV Bd;   // dressed factors (only when T1 given)
  if (sys->t1) {
    std::vector<double> t1((size_t)o * v);
    PN_CUDA(cudaMemcpyAsync(t1.data(), sys->t1, t1.size() * sizeof(double),
                            sys->mem_space == PNOEOM_DEVICE ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
    bd.sync();
    // h = diag(eps) - 2 J + K  (the one-electron operator whose Fock matrix is diag(eps))
    auto fock_parts = [&](const DV& Bx, std::vector<double>& J, std::vector<double>& K) {
      DV gam(N), dJ((size_t)nmo * nmo), dK((size_t)nmo * nmo);
      k_trace_occ<<<gsz(N), 256, 0, s>>>(gam.get(), Bx.get(), naux, nmo, o);
      PN_CUDA(cudaGetLastError());
      bd.con("Qpq", Bx.get(), "Q", gam.get(), "pq", dJ.get());
      DV Bxo = bd.slice(Bx, 0, nmo, 0, o), Box = bd.slice(Bx, 0, o, 0, nmo);
      Dims d2 = bd.dm; d2['k'] = O;
      bd.con("Qpk", Bxo.get(), "Qkq", Box.get(), "pq", dK.get(), 1.0, 0.0, &d2);
      J.resize(dJ.n); K.resize(dK.n);
      dJ.download(J.data(), J.size(), s); dK.download(K.data(), K.size(), s);
      bd.sync();
    };
    std::vector<double> J, K;
    fock_parts(dB, J, K);
    std::vector<double> h((size_t)nmo * nmo);
    for (int p = 0; p < nmo; ++p)
      for (int q = 0; q < nmo; ++q) h[p * nmo + q] = (p == q ? eps[p] : 0.0) - 2 * J[p * nmo + q] + K[p * nmo + q];
    std::vector<double> X((size_t)nmo * nmo, 0.0), Y((size_t)nmo * nmo, 0.0);
    for (int p = 0; p < nmo; ++p) X[p * nmo + p] = Y[p * nmo + p] = 1.0;
    for (int i = 0; i < o; ++i)
      for (int a = 0; a < v; ++a) { X[(o + a) * nmo + i] = -t1[i * v + a]; Y[(o + a) * nmo + i] = t1[i * v + a]; }
    // h~ = X h Y on the host (nmo^2, small)
    std::vector<double> tmp((size_t)nmo * nmo, 0.0), hd((size_t)nmo * nmo, 0.0);
    for (int p = 0; p < nmo; ++p)
      for (int r = 0; r < nmo; ++r) {
        double x = X[p * nmo + r];
        if (x == 0.0) continue;
        for (int q = 0; q < nmo; ++q) tmp[p * nmo + q] += x * h[r * nmo + q];
      }
    for (int p = 0; p < nmo; ++p)
      for (int r = 0; r < nmo; ++r) {
        double x = tmp[p * nmo + r];
        if (x == 0.0) continue;
        for (int q = 0; q < nmo; ++q) hd[p * nmo + q] += x * Y[r * nmo + q];
      }
    DV dX(X.size()), dY(Y.size()), T1b(dB.n);
    dX.upload(X.data(), X.size(), s); dY.upload(Y.data(), Y.size(), s);
    Bd.alloc(dB.n);
    bd.con("pr", dX.get(), "Qrs", dB.get(), "Qps", T1b.get());
    bd.con("Qps", T1b.get(), "sq", dY.get(), "Qpq", Bd.get());
    std::vector<double> Jd, Kd;
    fock_parts(Bd, Jd, Kd);
    for (size_t e = 0; e < Fd.size(); ++e) Fd[e] = hd[e] + 2 * Jd[e] - Kd[e];
  } else {
    for (int p = 0; p < nmo; ++p) Fd[p * nmo + p] = eps[p];
  }
  const DV& Bsrc = sys->t1 ? Bd : dB;
  DV dBoo = bd.slice(Bsrc, 0, o, 0, o), dBov = bd.slice(Bsrc, 0, o, o, v), dBvo = bd.slice(Bsrc, o, v, 0, o),
     dBvv = bd.slice(Bsrc, o, v, o, v);
  dB.release();
  Bd.release();

  tm.mark("dressing");
  // ---- T2 --------------------------------------------------------------------
  DV t2((size_t)O * O * V * V);
  if (sys->t2) {
    PN_CUDA(cudaMemcpyAsync(t2.get(), sys->t2, t2.n * sizeof(double), kind, s));
  } else {  // Eq. T1: t^{ij}_{ab} = (ai|bj) / (f_ii + f_jj - f_aa - f_bb)
    bd.con("Qai", Bvo.get(), "Qbj", Bvo.get(), "ijab", t2.get());
    k_pair_div<<<gsz(t2.n), 256, 0, s>>>(t2.get(), deps.get(), o, v, 0.0, 0.0);
    PN_CUDA(cudaGetLastError());
  }
  if (opts->t_pno_gs > 0.0) {
    // ground-state PNO truncation (Methods): per pair i <= j, D_(0) = 2/(1+d_ij)(T Tt^T + T^T Tt)
    // with Tt = 2T - T^T, eigenvectors of occupation >= t_pno_gs span the pair's space, and
    // T^{ij}, T^{ji} are replaced by P T P with P the projector onto it
    const int npr = o * (o + 1) / 2;
    std::vector<int> pi, pj;
    std::vector<std::vector<int>> pid(o, std::vector<int>(o, 0));
    for (int i = 0; i < o; ++i)
      for (int j = i; j < o; ++j) { pid[i][j] = pid[j][i] = (int)pi.size(); pi.push_back(i); pj.push_back(j); }
    DV D0((size_t)npr * V * V);
    D0.zero(s);
    {
      DV Tt(t2.n);
      bd.perm(t2.get(), Tt.get(), {O, O, V, V}, {0, 1, 3, 2}, -1.0, 0.0);
      axpby<double>(Tt.get(), t2.get(), 2.0, 1.0, Tt.n, s);
      for (int half = 0; half < 2; ++half) {   // two launches: one output tile per launch
        std::vector<GemmProb<double>> pr;
        for (int p = 0; p < npr; ++p) {
          const int i = pi[p], j = pj[p];
          const double c = 2.0 / (1.0 + (i == j));
          const double* T = t2.get() + ((int64_t)i * o + j) * V * V;
          const double* Tx = Tt.get() + ((int64_t)i * o + j) * V * V;
          double* Dp = D0.get() + (int64_t)p * V * V;
          if (half == 0) pr.push_back({T, Tx, Dp, v, v, v, v, v, v, 0, 1, c, 1.0});
          else pr.push_back({T, Tx, Dp, v, v, v, v, v, v, 1, 0, c, 1.0});
        }
        grouped_gemm<double>(pr, s);
      }
    }
    std::vector<double> w0((size_t)npr * v);
    {
      DV W0((size_t)npr * V);
      eig_dense_sym(ctx->solver, s, D0.get(), W0.get(), v, npr);   // ascending; column-major vectors
      W0.download(w0.data(), w0.size(), s);
      bd.sync();
    }
    DV Pj((size_t)npr * V * V), tmp(t2.n);
    Pj.zero(s);
    std::vector<GemmProb<double>> pp, p1, p2;
    for (int p = 0; p < npr; ++p) {
      int n = 0;
      for (int a = 0; a < v; ++a) n += w0[(size_t)p * v + a] >= opts->t_pno_gs;
      if (!n) continue;   // empty space: P = 0
      const double* Uk = D0.get() + (int64_t)p * V * V + (int64_t)(v - n) * v;   // kept eigenvectors (rows)
      pp.push_back({Uk, Uk, Pj.get() + (int64_t)p * V * V, v, v, n, v, v, v, 1, 0, 1.0, 0.0});
    }
    grouped_gemm<double>(pp, s);
    for (int i = 0; i < o; ++i)
      for (int j = 0; j < o; ++j) {
        const double* Pp = Pj.get() + (int64_t)pid[i][j] * V * V;
        double* T = t2.get() + ((int64_t)i * o + j) * V * V;
        double* X = tmp.get() + ((int64_t)i * o + j) * V * V;
        p1.push_back({T, Pp, X, v, v, v, v, v, v, 0, 0, 1.0, 0.0});
        p2.push_back({Pp, X, T, v, v, v, v, v, v, 0, 0, 1.0, 0.0});
      }
    grouped_gemm<double>(p1, s);
    grouped_gemm<double>(p2, s);
  }
  DV u2(t2.n);   // u = 2 t - t^(ab swapped)
  bd.perm(t2.get(), u2.get(), {O, O, V, V}, {0, 1, 3, 2}, -1.0, 0.0);
  axpby<double>(u2.get(), t2.get(), 2.0, 1.0, u2.n, s);

  tm.mark("T2");
  // ---- CIS (singlet; A = delta (e_a - e_i) + 2 (ia|jb) - (ij|ab)) ---------------
  const int nr = opts->nroots_sa;
  const int64_t ov = O * V;
  std::vector<double> bcis((size_t)nr * ov);
  {
    DV A((size_t)ov * ov), W(ov);
    bd.con("Qia", Bov.get(), "Qjb", Bov.get(), "iajb", A.get(), 2.0, 0.0);
    bd.con("Qij", Boo.get(), "Qab", Bvv.get(), "iajb", A.get(), -1.0, 1.0);
    k_cis_diag<<<gsz(ov), 256, 0, s>>>(A.get(), deps.get(), o, v);
    PN_CUDA(cudaGetLastError());
    std::vector<double> w(nr);
    if (ov <= CIS_DENSE_MAX) {   // partial dense eigensolve
      eig_lowest(ctx->solver, s, A.get(), W.get(), ov, nr);
      W.download(w.data(), nr, s);
      PN_CUDA(cudaMemcpyAsync(bcis.data(), A.get(), bcis.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    } else {                     // iterative (the dense reduction of a large matrix is slow)
      DV Xc((size_t)nr * ov);
      eig_lowest_davidson(ctx->solver, s, A.get(), ov, nr, 1e-11, w.data(), Xc.get());
      PN_CUDA(cudaMemcpyAsync(bcis.data(), Xc.get(), bcis.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    bd.sync();
    P->cis_omega = w;
    for (int k = 0; k < nr; ++k) {      // normalise 2 sum b^2 = 1, largest entry positive
      double* x = &bcis[(size_t)k * ov];
      int64_t m = 0;
      for (int64_t e = 1; e < ov; ++e) if (std::fabs(x[e]) > std::fabs(x[m])) m = e;
      double sc = (x[m] < 0 ? -1.0 : 1.0) / std::sqrt(2.0);
      for (int64_t e = 0; e < ov; ++e) x[e] *= sc;
    }
    P->cis_b = bcis;
  }

  tm.mark("CIS");
  // ---- CIS(D) doubles and state-averaged pair densities ------------------------
  // (state_specific = k: the density of CIS root k alone, weight 1)
  const int ss = opts->state_specific;
  const int npairs = o * (o + 1) / 2;
  P->npairs = npairs;
  P->pidx.assign(o, std::vector<int>(o, -1));
  for (int i = 0, p = 0; i < o; ++i)
    for (int j = i; j < o; ++j, ++p) { P->pair_i.push_back(i); P->pair_j.push_back(j); P->pidx[i][j] = P->pidx[j][i] = p; }
  DV Dens((size_t)npairs * V * V);
  Dens.zero(s);
  {
    DV b(ov), Z((size_t)N * ov), K(t2.n), Bt(t2.n);
    for (int k = 0; k < nr; ++k) {
      if (ss > 0 && k != ss - 1) continue;
      b.upload(&bcis[(size_t)k * ov], ov, s);
      // K^{ij}_{ab} = sum_Q Z[Q,i,a] B[Q,b,j] + sum_Q B[Q,a,i] Z[Q,j,b] with
      // Z[Q,i,a] = sum_c b[i,c] B[Q,a,c] - sum_l b[l,a] B[Q,l,i]; the second sum is the
      // first with (i,a) and (j,b) exchanged, so K = M + M^(ij,ab swapped)
      bd.con("ic", b.get(), "Qac", Bvv.get(), "Qia", Z.get());
      bd.con("la", b.get(), "Qli", Boo.get(), "Qia", Z.get(), -1.0, 1.0);
      bd.con("Qia", Z.get(), "Qbj", Bvo.get(), "ijab", Bt.get(), 1.0, 0.0);
      PN_CUDA(cudaMemcpyAsync(K.get(), Bt.get(), K.n * 8, cudaMemcpyDeviceToDevice, s));
      bd.perm(Bt.get(), K.get(), {O, O, V, V}, {1, 0, 3, 2}, 1.0, 1.0);
      k_pair_div<<<gsz(K.n), 256, 0, s>>>(K.get(), deps.get(), o, v, P->cis_omega[k], 1e-4);
      PN_CUDA(cudaGetLastError());
      bd.perm(K.get(), Bt.get(), {O, O, V, V}, {0, 1, 3, 2}, -1.0, 0.0);   // Bt^{ij} = 2 B^{ij} - (B^{ij})^T
      axpby<double>(Bt.get(), K.get(), 2.0, 1.0, Bt.n, s);
      // two launches: problems of one launch must not share an output tile
      for (int half = 0; half < 2; ++half) {
        std::vector<GemmProb<double>> pr;
        for (int p = 0; p < npairs; ++p) {
          int i = P->pair_i[p], j = P->pair_j[p];
          double c = (2.0 / (1.0 + (i == j))) / (ss > 0 ? 1 : nr);
          const double* Bij = K.get() + ((int64_t)i * o + j) * V * V;
          const double* Tij = Bt.get() + ((int64_t)i * o + j) * V * V;
          double* Dp = Dens.get() + (int64_t)p * V * V;
          if (half == 0) pr.push_back({Bij, Tij, Dp, v, v, v, v, v, v, 0, 1, c, 1.0});   // B Bt^T
          else pr.push_back({Bij, Tij, Dp, v, v, v, v, v, v, 1, 0, c, 1.0});            // B^T Bt
        }
        grouped_gemm<double>(pr, s);
      }
    }
  }

  tm.mark("CIS(D) densities");
  // ---- PNOs and OSVs ------------------------------------------------------------
  std::vector<double> occ((size_t)npairs * v);
  {
    DV W((size_t)npairs * V);
    eig_dense_sym(ctx->solver, s, Dens.get(), W.get(), v, npairs);
    W.download(occ.data(), occ.size(), s);
    bd.sync();
  }
  P->occupations = occ;
  auto count_kept = [&](const double* w, double thr) {
    if (thr == 0.0) return v;
    int n = 0;
    for (int a = 0; a < v; ++a) n += w[a] >= thr;
    return n;
  };
  P->nij.resize(npairs); P->ni.resize(o);
  for (int p = 0; p < npairs; ++p) P->nij[p] = count_kept(&occ[(size_t)p * v], P->t_pno);
  for (int i = 0; i < o; ++i) P->ni[i] = count_kept(&occ[(size_t)P->pidx[i][i] * v], P->t_osv);
  // raw kept vectors, semicanonicalisation (padded batched eigensolve), sign fix
  const int nsets = npairs + o;
  std::vector<int> nset(nsets), src(nsets);
  for (int p = 0; p < npairs; ++p) { nset[p] = P->nij[p]; src[p] = p; }
  for (int i = 0; i < o; ++i) { nset[npairs + i] = P->ni[i]; src[npairs + i] = P->pidx[i][i]; }
  std::vector<int64_t> uoff(nsets + 1, 0);
  for (int x = 0; x < nsets; ++x) uoff[x + 1] = uoff[x] + (int64_t)V * nset[x];
  int nmax = 1;
  for (int x : nset) nmax = std::max(nmax, x);
  P->U.alloc(std::max<int64_t>(1, uoff[nsets]), fp);
  DV Uraw(std::max<int64_t>(1, uoff[nsets]));
  for (int x = 0; x < nsets; ++x) {
    if (!nset[x]) continue;
    k_extract_kept<<<gsz((size_t)v * nset[x]), 256, 0, s>>>(Uraw.get() + uoff[x], Dens.get() + (int64_t)src[x] * V * V, v, nset[x]);
  }
  PN_CUDA(cudaGetLastError());
  Dens.release();
  std::vector<double> fb_host((size_t)nsets * nmax);
  {
    DV Fp((size_t)nsets * nmax * nmax), W2((size_t)nsets * nmax);
    for (int x = 0; x < nsets; ++x)
      k_fbar_padded<<<gsz((size_t)nmax * nmax), 256, 0, s>>>(Fp.get() + (int64_t)x * nmax * nmax, Uraw.get() + uoff[x],
                                                             deps.get() + o, v, nset[x], nmax);
    PN_CUDA(cudaGetLastError());
    eig_dense_sym(ctx->solver, s, Fp.get(), W2.get(), nmax, nsets);
    std::vector<GemmProb<double>> pr;
    for (int x = 0; x < nsets; ++x) {
      if (!nset[x]) continue;
      // U = Uraw Z[:n,:n]; Z column-major (column c = eigenvector c) => row-major view transposed
      pr.push_back({Uraw.get() + uoff[x], Fp.get() + (int64_t)x * nmax * nmax, P->U.get() + uoff[x], v, nset[x], nset[x],
                    nset[x], nmax, nset[x], 0, 1, 1.0, 0.0});
    }
    grouped_gemm<double>(pr, s);
    for (int x = 0; x < nsets; ++x)
      if (nset[x]) k_sign_fix<<<nset[x], 256, 0, s>>>(P->U.get() + uoff[x], v, nset[x]);
    PN_CUDA(cudaGetLastError());
    W2.download(fb_host.data(), fb_host.size(), s);
    bd.sync();
  }
  Uraw.release();
  P->Uoff_pair.assign(uoff.begin(), uoff.begin() + npairs);
  P->Uoff_osv.assign(uoff.begin() + npairs, uoff.begin() + nsets);
  {
    std::vector<double> fb;
    std::vector<int64_t> fo(nsets + 1, 0);
    for (int x = 0; x < nsets; ++x) {
      fo[x + 1] = fo[x] + nset[x];
      for (int c = 0; c < nset[x]; ++c) fb.push_back(fb_host[(size_t)x * nmax + c]);
    }
    P->fbar.alloc(std::max<size_t>(1, fb.size()), fp);
    P->fbar.upload(fb.data(), fb.size(), s);
    P->foff_pair.assign(fo.begin(), fo.begin() + npairs);
    P->foff_osv.assign(fo.begin() + npairs, fo.begin() + nsets);
    // packed layout and Davidson denominators (without omega)
    P->off_i.assign(o + 1, 0);
    for (int i = 0; i < o; ++i) P->off_i[i + 1] = P->off_i[i] + P->ni[i];
    P->L1 = P->off_i[o];
    P->off_ij.assign(npairs + 1, P->L1);
    for (int p = 0; p < npairs; ++p) P->off_ij[p + 1] = P->off_ij[p] + (int64_t)P->nij[p] * P->nij[p];
    P->L = P->off_ij[npairs];
    std::vector<double> den(std::max<int64_t>(1, P->L));
    for (int i = 0; i < o; ++i)
      for (int c = 0; c < P->ni[i]; ++c) den[P->off_i[i] + c] = eps[i] - fb[fo[npairs + i] + c];
    for (int p = 0; p < npairs; ++p) {
      int i = P->pair_i[p], j = P->pair_j[p], n = P->nij[p];
      for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
          den[P->off_ij[p] + a * n + b] = eps[i] + eps[j] - fb[fo[p] + a] - fb[fo[p] + b];
    }
    P->denom_base.alloc(den.size(), fp);
    P->denom_base.upload(den.data(), den.size(), s);
    // projected CIS guesses: R1_i = U^i^T b_i, R2 = 0
    std::vector<double> Uh(P->U.n);
    P->U.download(Uh.data(), Uh.size(), s);
    bd.sync();
    std::vector<double> gs((size_t)nr * std::max<int64_t>(1, P->L), 0.0);
    for (int k = 0; k < nr; ++k)
      for (int i = 0; i < o; ++i)
        for (int c = 0; c < P->ni[i]; ++c) {
          double acc = 0;
          for (int a = 0; a < v; ++a) acc += Uh[P->Uoff_osv[i] + (int64_t)a * P->ni[i] + c] * bcis[(size_t)k * ov + i * v + a];
          gs[(size_t)k * P->L + P->off_i[i] + c] = acc;
        }
    P->guesses.alloc(gs.size(), fp);
    P->guesses.upload(gs.data(), gs.size(), s);
  }
  Boo.release(); Bov.release(); Bvo.release(); Bvv.release();
  tm.mark("PNO/OSV eigensolves");

  // The rest (intermediates, pool, problem lists) lives in build_program.cu.
  extern void build_program(pnoeom_pno * P, cudaStream_t s, const double* Fd, DV& dBoo, DV& dBov, DV& dBvo, DV& dBvv,
                            DV& t2, DV& u2);
  build_program(P, s, Fd.data(), dBoo, dBov, dBvo, dBvv, t2, u2);
  bd.sync();
  tm.mark("operator program");
  autotune(P, s);
  tm.mark("autotune");
  PN_CUDA(cudaStreamSynchronize(s));
  pool_trim();   // setup temporaries go back to CUDA
  P->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
}

}  // namespace pnoeom
