// sigma dispatch and the Davidson solver (Sec. 2, PNO-EOM-CCSD Davidson).
#include "pno.cuh"
#include <algorithm>
#include <cmath>
#include <complex>

namespace pnoeom {

// ---------------------------------------------------------------------------
// sigma program execution
template <typename T>
static DBuf<T>& work_of(pnoeom_pno* P);
template <> DBuf<double>& work_of<double>(pnoeom_pno* P) { return P->work64; }
template <> DBuf<float>& work_of<float>(pnoeom_pno* P) { return P->work32; }

template <typename T>
void apply_sigma(pnoeom_pno* P, int nvec, const T* r, T* out, cudaStream_t s) {
  if (nvec <= 0) return;
  DBuf<T>& work = work_of<T>(P);
  const size_t need = (size_t)nvec * P->work_len;
  if (work.n < need) work.alloc(need, &P->footprint);
  PN_CUDA(cudaMemsetAsync(out, 0, (size_t)nvec * P->L * sizeof(T), s));
  work.zero(s);
  Buffers b;
  b.pool = sizeof(T) == 8 ? (const void*)P->pool64.get() : (const void*)P->pool32.get();
  b.rin = r; b.rin_stride = P->L;
  b.work = work.get(); b.work_stride = P->work_len;
  b.sout = out; b.sout_stride = P->L;
  auto timed = [&](int cls, auto&& launch) {
    if (!P->timing) { launch(); return; }
    cudaEvent_t e0, e1;
    PN_CUDA(cudaEventCreate(&e0));
    PN_CUDA(cudaEventCreate(&e1));
    PN_CUDA(cudaEventRecord(e0, s));
    launch();
    PN_CUDA(cudaEventRecord(e1, s));
    P->events.push_back({cls, {e0, e1}});
  };
  timed(0, [&] {
    run_small_sets<T>(P, P->small1, nvec, b, s);
    run_sandwich<T>(P->sp_phase1.get(), P->n_sp1, nvec, b, P->smem_elems, s);
  });
  timed(1, [&] { run_gemv<T>(P->vp_phase1.get(), P->n_vp1, nvec, b, s); });
  timed(2, [&] {
    run_small_sets<T>(P, P->small2, nvec, b, s);
    run_sandwich<T>(P->sp_phase2.get(), P->n_sp2, nvec, b, P->smem_elems, s);
  });
  timed(3, [&] { run_gemv<T>(P->vp_phase2.get(), P->n_vp2, nvec, b, s); });
  if (P->timing) {   // kernel launches per class in this call
    auto nsets = [](const pnoeom_pno::SmallSet* S) { int n = 0; for (int k = 0; k < 3; ++k) n += S[k].nprob > 0; return n; };
    P->prof_launches[0] += nsets(P->small1) + (P->n_sp1 > 0);
    P->prof_launches[1] += P->n_vp1 > 0;
    P->prof_launches[2] += nsets(P->small2) + (P->n_sp2 > 0);
    P->prof_launches[3] += P->n_vp2 > 0;
  }
}
template void apply_sigma<double>(pnoeom_pno*, int, const double*, double*, cudaStream_t);
template void apply_sigma<float>(pnoeom_pno*, int, const float*, float*, cudaStream_t);

// Autotuner: time the FP32 sigma of nroots_sa vectors for every candidate group size of the
// grouped small-sandwich kernel and every roots-per-CTA choice (CUDA events on the build
// stream) and keep the fastest pair.
void autotune(pnoeom_pno* P, cudaStream_t s) {
  const int nv = std::max(1, P->nroots_sa);
  DBuf<float> r((size_t)nv * P->L), o((size_t)nv * P->L);
  r.zero(s);
  cudaEvent_t e0, e1;
  PN_CUDA(cudaEventCreate(&e0));
  PN_CUDA(cudaEventCreate(&e1));
  double best = 1e300;
  int pick = 0, pick_r = 0;
  for (int c = 0; c < NGROUP_CAND; ++c)
    for (int rr = 0; rr < NRPC_CAND; ++rr) {
      P->group_choice = c;
      P->rpc_choice = rr;
      apply_sigma<float>(P, nv, r.get(), o.get(), s);   // warm-up
      PN_CUDA(cudaEventRecord(e0, s));
      for (int k = 0; k < 3; ++k) apply_sigma<float>(P, nv, r.get(), o.get(), s);
      PN_CUDA(cudaEventRecord(e1, s));
      PN_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      PN_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      P->tune_ms[c * NRPC_CAND + rr] = ms / 3;
      if (ms < best) { best = ms; pick = c; pick_r = rr; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  P->group_choice = pick;
  P->rpc_choice = pick_r;
}

// ---------------------------------------------------------------------------
// Small dense non-symmetric eigenproblem on the host: Householder reduction
// to Hessenberg form, then single-shift complex QR iterations with Givens
// rotations (Wilkinson shift, deflation on negligible subdiagonals), giving
// the complex Schur form A = Z T Z^H; eigenvectors by back-substitution on T.
using cd = std::complex<double>;

int small_eig(int n, const double* A, double* wr, double* wi, double* VR) {
  std::vector<cd> H((size_t)n * n), Z((size_t)n * n, 0.0);
  for (int i = 0; i < n * n; ++i) H[i] = A[i];
  for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
  auto h = [&](int i, int j) -> cd& { return H[(size_t)i * n + j]; };
  auto z = [&](int i, int j) -> cd& { return Z[(size_t)i * n + j]; };
  // Householder reduction to upper Hessenberg
  for (int k = 0; k + 2 < n; ++k) {
    double alpha = 0;
    for (int i = k + 1; i < n; ++i) alpha += std::norm(h(i, k));
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    std::vector<cd> u(n, 0.0);
    cd x0 = h(k + 1, k);
    cd phase = std::abs(x0) > 0 ? x0 / std::abs(x0) : cd(1.0);
    for (int i = k + 1; i < n; ++i) u[i] = h(i, k);
    u[k + 1] += phase * alpha;
    double un = 0;
    for (int i = k + 1; i < n; ++i) un += std::norm(u[i]);
    if (un == 0.0) continue;
    // H = (I - 2 u u^H / un) H (I - 2 u u^H / un); Z = Z (I - 2 u u^H / un)
    for (int j = 0; j < n; ++j) {
      cd sdot = 0;
      for (int i = k + 1; i < n; ++i) sdot += std::conj(u[i]) * h(i, j);
      sdot *= 2.0 / un;
      for (int i = k + 1; i < n; ++i) h(i, j) -= u[i] * sdot;
    }
    for (int i = 0; i < n; ++i) {
      cd sdot = 0;
      for (int j = k + 1; j < n; ++j) sdot += h(i, j) * u[j];
      sdot *= 2.0 / un;
      for (int j = k + 1; j < n; ++j) h(i, j) -= sdot * std::conj(u[j]);
      cd zdot = 0;
      for (int j = k + 1; j < n; ++j) zdot += z(i, j) * u[j];
      zdot *= 2.0 / un;
      for (int j = k + 1; j < n; ++j) z(i, j) -= zdot * std::conj(u[j]);
    }
    for (int i = k + 2; i < n; ++i) h(i, k) = 0.0;
  }
  // shifted QR
  const double eps = 1e-15;
  int hi = n - 1, iter = 0, total = 0;
  std::vector<double> cs(n);
  std::vector<cd> sn(n);
  while (hi > 0) {
    int l = hi;
    while (l > 0 && std::abs(h(l, l - 1)) > eps * (std::abs(h(l - 1, l - 1)) + std::abs(h(l, l)))) --l;
    if (l > 0) h(l, l - 1) = 0.0;
    if (l == hi) { --hi; iter = 0; continue; }
    if (++total > 100 * n) return -1;
    cd a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
    cd tr = a + d, det = a * d - b * c;
    cd disc = std::sqrt(tr * tr / 4.0 - det);
    cd m1 = tr / 2.0 + disc, m2 = tr / 2.0 - disc;
    cd mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
    if (iter % 11 == 10) mu = d + std::abs(h(hi, hi - 1));
    ++iter;
    for (int k = l; k <= hi; ++k) h(k, k) -= mu;
    for (int k = l; k < hi; ++k) {
      cd x = h(k, k), y = h(k + 1, k);
      double r = std::sqrt(std::norm(x) + std::norm(y));
      double cc; cd ss;
      if (r == 0.0) { cc = 1.0; ss = 0.0; }
      else if (std::abs(x) == 0.0) { cc = 0.0; ss = std::conj(y) / std::abs(y); }
      else { cc = std::abs(x) / r; ss = (x / std::abs(x)) * std::conj(y) / r; }
      cs[k] = cc; sn[k] = ss;
      for (int j = k; j < n; ++j) {
        cd p = h(k, j), q = h(k + 1, j);
        h(k, j) = cc * p + ss * q;
        h(k + 1, j) = -std::conj(ss) * p + cc * q;
      }
    }
    for (int k = l; k < hi; ++k) {
      double cc = cs[k]; cd ss = sn[k];
      int rmax = std::min(k + 2, hi);
      for (int i = 0; i <= rmax; ++i) {
        cd p = h(i, k), q = h(i, k + 1);
        h(i, k) = cc * p + std::conj(ss) * q;
        h(i, k + 1) = -ss * p + cc * q;
      }
      for (int i = 0; i < n; ++i) {
        cd p = z(i, k), q = z(i, k + 1);
        z(i, k) = cc * p + std::conj(ss) * q;
        z(i, k + 1) = -ss * p + cc * q;
      }
    }
    for (int k = l; k <= hi; ++k) h(k, k) += mu;
  }
  // eigenvectors of T by back-substitution, then V = Z y
  double tnorm = 0;
  for (int i = 0; i < n * n; ++i) tnorm = std::max(tnorm, std::abs(H[i]));
  for (int k = 0; k < n; ++k) {
    std::vector<cd> y(n, 0.0);
    y[k] = 1.0;
    cd lam = h(k, k);
    for (int i = k - 1; i >= 0; --i) {
      cd sacc = 0;
      for (int j = i + 1; j <= k; ++j) sacc += h(i, j) * y[j];
      cd den = h(i, i) - lam;
      if (std::abs(den) < 1e-14 * std::max(1.0, tnorm)) den = 1e-14 * std::max(1.0, tnorm);
      y[i] = -sacc / den;
    }
    std::vector<cd> x(n, 0.0);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j <= k; ++j) x[i] += z(i, j) * y[j];
    // rotate so the largest component is real and positive, then keep the real part
    int im = 0;
    for (int i = 1; i < n; ++i) if (std::abs(x[i]) > std::abs(x[im])) im = i;
    cd ph = std::abs(x[im]) > 0 ? std::conj(x[im]) / std::abs(x[im]) : cd(1.0);
    double nrm = 0;
    for (int i = 0; i < n; ++i) { x[i] *= ph; nrm += std::norm(x[i].real()); }
    nrm = std::sqrt(nrm);
    for (int i = 0; i < n; ++i) VR[(size_t)i * n + k] = nrm > 0 ? x[i].real() / nrm : 0.0;
    wr[k] = lam.real();
    wi[k] = lam.imag();
  }
  return 0;
}

// ---------------------------------------------------------------------------
namespace {
inline unsigned gsz(size_t n) { return (unsigned)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 16)); }

// G[a*mb + b] += sum_k X[a*L + k] Y[b*L + k]; split over k, atomic partial sums
__global__ void k_gram(double* G, const double* X, const double* Y, int ma, int mb, int64_t L) {
  extern __shared__ double red[];
  const int pairs = ma * mb;
  for (int q = 0; q < pairs; ++q) {
    const int a = q / mb, b = q % mb;
    double acc = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L; k += (int64_t)gridDim.x * blockDim.x)
      acc += X[(int64_t)a * L + k] * Y[(int64_t)b * L + k];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&G[q], red[0]);
    __syncthreads();
  }
}
// out[q*L + k] = beta*out[q*L+k] + sum_a C[q*m + a] V[a*L + k]
__global__ void k_combine(double* out, const double* V, const double* C, int m, int nq, int64_t L, double beta) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)nq * L; e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e / L);
    const int64_t k = e % L;
    double acc = 0;
    for (int a = 0; a < m; ++a) acc += C[q * m + a] * V[(int64_t)a * L + k];
    out[e] = (beta == 0.0 ? 0.0 : beta * out[e]) + acc;
  }
}
// t = r / clamp(omega + den), |den| >= 1e-4
__global__ void k_precond(double* t, const double* r, const double* den, double omega, int64_t L) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L; e += (int64_t)gridDim.x * blockDim.x) {
    double d = omega + den[e];
    if (fabs(d) < 1e-4) d = d < 0 ? -1e-4 : 1e-4;
    t[e] = r[e] / d;
  }
}
// symmetrise the diagonal-pair blocks (R^{ii} is symmetric by definition)
__global__ void k_symdiag(double* x, const int64_t* offs, const int* ns, int nd) {
  const int b = blockIdx.x;
  if (b >= nd) return;
  const int n = ns[b];
  double* B = x + offs[b];
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int a = e / n, c = e % n;
    if (a < c) { double s = 0.5 * (B[a * n + c] + B[c * n + a]); B[a * n + c] = s; B[c * n + a] = s; }
  }
}
__global__ void k_f2d_(double* y, const float* x, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) y[e] = x[e];
}
__global__ void k_d2f_(float* y, const double* x, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) y[e] = (float)x[e];
}

struct Dav {
  pnoeom_pno* P;
  cudaStream_t s;
  int64_t L;
  DBuf<double> dG;
  DBuf<int64_t> dOffs; DBuf<int> dNs; int nd = 0;
  DBuf<float> f_in, f_out;

  std::vector<double> gram(const double* X, int ma, const double* Y, int mb) {
    std::vector<double> g((size_t)ma * mb, 0.0);
    if (!ma || !mb) return g;
    if (dG.n < g.size()) dG.alloc(g.size());
    PN_CUDA(cudaMemsetAsync(dG.get(), 0, g.size() * 8, s));
    k_gram<<<gsz(L), 256, 256 * sizeof(double), s>>>(dG.get(), X, Y, ma, mb, L);
    PN_CUDA(cudaGetLastError());
    dG.download(g.data(), g.size(), s);
    PN_CUDA(cudaStreamSynchronize(s));
    return g;
  }
  void combine(double* out, const double* V, const std::vector<double>& C, int m, int nq, double beta) {
    if (!nq) return;
    DBuf<double> dC(std::max<size_t>(1, C.size()));
    dC.upload(C.data(), C.size(), s);
    k_combine<<<gsz((size_t)nq * L), 256, 0, s>>>(out, V, dC.get(), m, nq, L, beta);
    PN_CUDA(cudaGetLastError());
    PN_CUDA(cudaStreamSynchronize(s));
  }
  void symdiag(double* x) {
    if (nd) k_symdiag<<<nd, 256, 0, s>>>(x, dOffs.get(), dNs.get(), nd);
    PN_CUDA(cudaGetLastError());
  }
  void sigma(const double* V, double* S, int nv, int prec) {
    if (!nv) return;
    if (prec == PNOEOM_FP64) { apply_sigma<double>(P, nv, V, S, s); return; }
    size_t n = (size_t)nv * L;
    if (f_in.n < n) { f_in.alloc(n); f_out.alloc(n); }
    k_d2f_<<<gsz(n), 256, 0, s>>>(f_in.get(), V, n);
    apply_sigma<float>(P, nv, f_in.get(), f_out.get(), s);
    k_f2d_<<<gsz(n), 256, 0, s>>>(S, f_out.get(), n);
    PN_CUDA(cudaGetLastError());
  }
  // orthonormalise t against rows 0..m-1 of V (twice); returns the norm before normalisation
  double orth(double* V, int m, double* t) {
    for (int pass = 0; pass < 2; ++pass) {
      if (!m) break;
      std::vector<double> c = gram(t, 1, V, m);
      for (double& x : c) x = -x;
      combine(t, V, c, m, 1, 1.0);
    }
    std::vector<double> nn = gram(t, 1, t, 1);
    double nrm = std::sqrt(std::max(0.0, nn[0]));
    if (nrm > 0) { scale<double>(t, 1.0 / nrm, L, s); }
    return nrm;
  }
};
}  // namespace

void run_davidson(pnoeom_ctx* ctx, pnoeom_pno* P, const pnoeom_opts* opts, cudaStream_t s, double* energies,
                  double* res_norms, int* iters, int* converged) {
  (void)ctx;
  const int nroots = opts->nroots_solve;
  PN_CHECK(nroots >= 1 && nroots <= P->nroots_sa, PNOEOM_ERR_INVALID_ARG, "nroots_solve must be in [1, nroots_sa]");
  const int64_t L = P->L;
  PN_CHECK(L >= nroots, PNOEOM_ERR_INVALID_ARG, "PNO space smaller than the number of roots");
  const int maxsub = std::max(opts->max_subspace > 0 ? opts->max_subspace : 8 * nroots, 2 * nroots + 1);
  const int max_iter = opts->max_iter > 0 ? opts->max_iter : 100;
  const double res_tol = opts->res_tol > 0 ? opts->res_tol : 1e-7;
  const double e_tol = opts->e_tol > 0 ? opts->e_tol : 1e-10;
  Dav D{P, s, L};
  {
    std::vector<int64_t> offs; std::vector<int> ns;
    for (int p = 0; p < P->npairs; ++p)
      if (P->pair_i[p] == P->pair_j[p] && P->nij[p] > 1) { offs.push_back(P->off_ij[p]); ns.push_back(P->nij[p]); }
    D.nd = (int)offs.size();
    D.dOffs.alloc(std::max<size_t>(1, offs.size())); D.dOffs.upload(offs.data(), offs.size(), s);
    D.dNs.alloc(std::max<size_t>(1, ns.size())); D.dNs.upload(ns.data(), ns.size(), s);
  }
  DBuf<double> V((size_t)maxsub * L), S((size_t)maxsub * L), X((size_t)nroots * L), R((size_t)nroots * L), T((size_t)L);
  int m = 0;
  for (int k = 0; k < P->nroots_sa && m < nroots; ++k) {   // projected CIS guesses
    double* t = V.get() + (int64_t)m * L;
    PN_CUDA(cudaMemcpyAsync(t, P->guesses.get() + (int64_t)k * L, L * 8, cudaMemcpyDeviceToDevice, s));
    if (D.orth(V.get(), m, t) > 1e-10) ++m;
  }
  PN_CHECK(m > 0, PNOEOM_ERR_INVALID_ARG, "no guess vector survives the projection");
  int prec = opts->precision == PNOEOM_FP32 ? PNOEOM_FP32 : PNOEOM_FP64;
  const bool refine = prec == PNOEOM_FP32 && opts->refine_fp64;
  // in mixed precision, converge to a looser residual first, then refine in FP64
  const double tol_mixed = refine ? std::max(res_tol, 1e-4) : res_tol;
  D.sigma(V.get(), S.get(), m, prec);
  std::vector<double> w_old;
  int nr = std::min(nroots, m);
  std::vector<double> w(nr), rn(nr);
  *converged = 0;
  int it = 0;
  for (it = 1; it <= max_iter; ++it) {
    std::vector<double> G = D.gram(V.get(), m, S.get(), m);   // G[a][b] = <v_a, sigma(v_b)>
    std::vector<double> wr(m), wi(m), VR((size_t)m * m);
    PN_CHECK(small_eig(m, G.data(), wr.data(), wi.data(), VR.data()) == 0, PNOEOM_ERR_NOT_CONVERGED,
             "subspace eigensolver did not converge");
    std::vector<int> ord(m);
    for (int a = 0; a < m; ++a) ord[a] = a;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return wr[a] < wr[b]; });
    nr = std::min(nroots, m);
    w.assign(nr, 0.0);
    std::vector<double> Cy((size_t)nr * m), Cs((size_t)nr * m);
    for (int q = 0; q < nr; ++q) {
      w[q] = wr[ord[q]];
      for (int a = 0; a < m; ++a) Cy[(size_t)q * m + a] = VR[(size_t)a * m + ord[q]];
    }
    D.combine(X.get(), V.get(), Cy, m, nr, 0.0);                  // Ritz vectors
    D.combine(R.get(), S.get(), Cy, m, nr, 0.0);                  // sigma of Ritz vectors
    for (int q = 0; q < nr; ++q) axpby<double>(R.get() + (int64_t)q * L, X.get() + (int64_t)q * L, -w[q], 1.0, L, s);
    rn.assign(nr, 0.0);
    for (int q = 0; q < nr; ++q) rn[q] = std::sqrt(std::max(0.0, D.gram(R.get() + (int64_t)q * L, 1, R.get() + (int64_t)q * L, 1)[0]));
    double dw = 1e300;
    if ((int)w_old.size() == nr) { dw = 0; for (int q = 0; q < nr; ++q) dw = std::max(dw, std::fabs(w[q] - w_old[q])); }
    w_old = w;
    bool conv = true;
    const double tol_now = prec == PNOEOM_FP32 ? tol_mixed : res_tol;
    for (int q = 0; q < nr; ++q) conv = conv && rn[q] < tol_now;
    conv = conv && (prec == PNOEOM_FP32 && refine ? true : dw < e_tol);
    if (conv) {
      if (prec == PNOEOM_FP32 && refine) {   // FP64 refinement: recompute sigma of the subspace in FP64
        prec = PNOEOM_FP64;
        D.sigma(V.get(), S.get(), m, prec);
        w_old.clear();
        continue;
      }
      *converged = 1;
      break;
    }
    // new directions from the preconditioned residuals
    std::vector<int> add;
    for (int q = 0; q < nr; ++q) if (rn[q] >= tol_now) add.push_back(q);
    if (m + (int)add.size() > maxsub) {      // collapse onto the Ritz vectors
      PN_CUDA(cudaMemcpyAsync(V.get(), X.get(), (size_t)nr * L * 8, cudaMemcpyDeviceToDevice, s));
      int mm = 0;
      for (int q = 0; q < nr; ++q) {
        double* t = V.get() + (int64_t)mm * L;
        if (mm != q) PN_CUDA(cudaMemcpyAsync(t, V.get() + (int64_t)q * L, L * 8, cudaMemcpyDeviceToDevice, s));
        if (D.orth(V.get(), mm, t) > 1e-10) ++mm;
      }
      m = mm;
      D.sigma(V.get(), S.get(), m, prec);
    }
    int m0 = m;
    for (int q : add) {
      if (m >= maxsub) break;
      double* t = V.get() + (int64_t)m * L;
      k_precond<<<gsz(L), 256, 0, s>>>(t, R.get() + (int64_t)q * L, P->denom_base.get(), w[q], L);
      PN_CUDA(cudaGetLastError());
      D.symdiag(t);
      if (D.orth(V.get(), m, t) > 1e-8) ++m;
    }
    if (m == m0) {   // no new direction: converged if every residual is within tolerance
      bool allres = true;
      for (int q = 0; q < nr; ++q) allres = allres && rn[q] < tol_now;
      if (allres && prec == PNOEOM_FP32 && refine) {
        prec = PNOEOM_FP64;
        D.sigma(V.get(), S.get(), m, prec);
        w_old.clear();
        continue;
      }
      *converged = allres ? 1 : 0;
      break;
    }
    D.sigma(V.get() + (int64_t)m0 * L, S.get() + (int64_t)m0 * L, m - m0, prec);
  }
  for (int q = 0; q < nr; ++q) { energies[q] = w[q]; res_norms[q] = rn[q]; }
  for (int q = nr; q < nroots; ++q) { energies[q] = NAN; res_norms[q] = NAN; }
  *iters = std::min(it, max_iter);
  P->last_X.resize((size_t)nr * L);
  X.download(P->last_X.data(), P->last_X.size(), s);
  PN_CUDA(cudaStreamSynchronize(s));
  P->last_nroots = nr;
}

}  // namespace pnoeom
