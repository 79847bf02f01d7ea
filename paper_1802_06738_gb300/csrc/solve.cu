// sigma dispatch and the Davidson solver (Sec. 2, PNO-EOM-CCSD Davidson).
#include "pno.cuh"
#include <algorithm>
#include <cmath>
#include <complex>
#include <memory>
#include <cstdlib>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

namespace pnoeom {

// ---------------------------------------------------------------------------
// sigma program execution
template <typename T>
static DBuf<T>& work_of(pnoeom_pno* P);
template <> DBuf<double>& work_of<double>(pnoeom_pno* P) { return P->work64; }
template <> DBuf<float>& work_of<float>(pnoeom_pno* P) { return P->work32; }

SysBuf sysbuf(const pnoeom_pno* P, int nvec, const void* r, void* out, void* work, bool fp32, bool bf16) {
  SysBuf b{};
  b.pool = fp32 ? (const void*)P->pool32.get() : (const void*)P->pool64.get();
  b.pool16 = fp32 && bf16 ? (const void*)P->pool16.get() : nullptr;
  b.tcimg = fp32 && bf16 && P->prog.n_tcs_jobs > 0 ? (const void*)P->tcimg.get() : nullptr;
  b.rin = r; b.rin_stride = P->L;
  b.work = work; b.work_stride = P->work_len;
  b.sout = out; b.sout_stride = P->L;
  b.nvec = nvec;
  return b;
}

template <typename T>
static void run_small_set(const SmallSet& S, int c, int rr, const SysTable& t, cudaStream_t s) {
  run_sandwich_small<T>(S.probs.get(), S.starts[c].get(), S.ngroups[c], t, S.dims[0], S.dims[1], S.dims[2], S.dims[3],
                        RPC_CAND[rr], S.pb, S.nb, S.shape, s);
}

constexpr int TUNE_REPS = 5;   // separately timed launches per candidate, after one warm-up launch

// Time every small-sandwich set of the program alone for every (group size, vectors
// per CTA) candidate (CUDA events on s) and keep each set's fastest.  sum_ms[c] is the
// summed time of all sets under candidate c; the program's reported choice is the
// candidate with the smallest sum.
template <typename T>
static void tune_sets(Program& prog, const SysTable& t, cudaStream_t s, double* sum_ms) {
  cudaEvent_t e0, e1;
  PN_CUDA(cudaEventCreate(&e0));
  PN_CUDA(cudaEventCreate(&e1));
  for (int c = 0; c < NTUNE; ++c) sum_ms[c] = 0;
  // ms of the fastest of TUNE_REPS timed launches after one warm-up (interference only
  // adds time, so the minimum is the steadiest estimate)
  auto measure = [&](SmallSet& S, int c, int rr) {
    run_small_set<T>(S, c, rr, t, s);
    double best = 1e300;
    for (int q = 0; q < TUNE_REPS; ++q) {
      PN_CUDA(cudaEventRecord(e0, s));
      run_small_set<T>(S, c, rr, t, s);
      PN_CUDA(cudaEventRecord(e1, s));
      PN_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      PN_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      best = std::min(best, (double)ms);
    }
    return best;
  };
  for (SmallSet* sets : {prog.small1, prog.small2})
    for (int k = 0; k < 3; ++k) {
      SmallSet& S = sets[k];
      if (!S.nprob) continue;
      double best = 1e300;
      S.pb = 1;      // candidates are timed unbatched, with buffering by occupancy and the
      S.nb = 0;      // bucket's CTA shape; the shape, the number of stage buffers and the
      S.shape = 0;   // batch size are chosen afterwards
      for (int c = 0; c < NGROUP_CAND; ++c)
        for (int rr = 0; rr < NRPC_CAND; ++rr) {
          const double ms = measure(S, c, rr);
          const int idx = c * NRPC_CAND + rr;
          S.tune_ms[idx] = ms;
          sum_ms[idx] += ms;
          if (ms < best) { best = ms; S.gchoice = c; S.rchoice = rr; }
        }
      int best_shape = 0;
      for (int shc : {1, 2, 3}) {
        S.shape = shc;
        const double ms = measure(S, S.gchoice, S.rchoice);
        if (ms < best) { best = ms; best_shape = shc; }
      }
      S.shape = best_shape;
      int best_nb = 0;
      for (int nbc : {1, 2}) {
        S.nb = nbc;
        const double ms = measure(S, S.gchoice, S.rchoice);
        if (ms < best) { best = ms; best_nb = nbc; }
      }
      S.nb = best_nb;
      int best_pb = 1;
      if (S.ab)
        for (int pbc : {2, 4}) {
          S.pb = pbc;
          const double ms = measure(S, S.gchoice, S.rchoice);
          if (ms < best) { best = ms; best_pb = pbc; }
        }
      S.pb = best_pb;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int pick = 0;
  for (int c = 1; c < NTUNE; ++c)
    if (sum_ms[c] < sum_ms[pick]) pick = c;
  prog.group_choice = pick / NRPC_CAND;
  prog.rpc_choice = pick % NRPC_CAND;
}

template <typename T>
void run_program(const Program& prog, const SysTable& t, const int64_t* out_len, const int64_t* work_len,
                 cudaStream_t s, pnoeom_pno* timing_owner, bool library) {
  for (int k = 0; k < t.nsys; ++k) {
    const SysBuf& b = t.s[k];
    if (b.nvec <= 0) continue;
    PN_CUDA(cudaMemsetAsync(b.sout, 0, (size_t)b.nvec * out_len[k] * sizeof(T), s));
    PN_CUDA(cudaMemsetAsync(b.work, 0, (size_t)b.nvec * work_len[k] * sizeof(T), s));
  }
  pnoeom_pno* P = timing_owner && timing_owner->timing ? timing_owner : nullptr;
  auto timed = [&](int cls, auto&& launch) {
    if (!P) { launch(); return; }
    cudaEvent_t e0, e1;
    PN_CUDA(cudaEventCreate(&e0));
    PN_CUDA(cudaEventCreate(&e1));
    PN_CUDA(cudaEventRecord(e0, s));
    launch();
    PN_CUDA(cudaEventRecord(e1, s));
    P->events.push_back({cls, {e0, e1}});
  };
  auto small = [&](const SmallSet* sets) {
    int n = 0;
    for (int k = 0; k < 3; ++k) {
      const SmallSet& S = sets[k];
      if (!S.nprob) continue;
      run_small_set<T>(S, S.gchoice, S.rchoice, t, s);
      ++n;
    }
    return n;
  };
  // launch order: Y products -> FvR GEMM; FoR; Z GEMM -> E3 products; the sigma classes
  // (all accumulate into sigma, in any order)
  int n0 = 0, n2 = 0;
  timed(0, [&] {
    n0 = small(prog.small1);
    run_sandwich<T>(prog.gen1.get(), prog.n_gen1, t, prog.smem_elems, s);
  });
  // single-precision single-system calls that may use a library (not the no-allocation
  // entry point): the two whole E3 products as strided-batched GEMMs over the vectors (TF32
  // tensor cores for the BF16 sigma, FP32 otherwise)
  const bool whole = library && sizeof(T) == 4 && t.nsys == 1 && prog.h_gfull.size() == 2 && prog.h_gfull[0].tc == 0 &&
                     prog.h_gfull[1].tc == 0;
  auto whole_gemm = [&](const DProb& P) {
    const SysBuf& b = t.s[0];
    auto at = [&](int buf, int64_t off, long long& stride) -> float* {
      switch (buf) {
        case B_POOL: stride = 0; return (float*)b.pool + off;
        case B_RIN: stride = b.rin_stride; return (float*)b.rin + off;
        case B_WORK: stride = b.work_stride; return (float*)b.work + off;
        default: stride = b.sout_stride; return (float*)b.sout + off;
      }
    };
    long long sa, sb, sc;
    const float* A = at(P.a_buf, P.a_off, sa);
    const float* Bm = at(P.b_buf, P.b_off, sb);
    float* C = at(P.c_buf, P.c_off, sc);
    blas_sgemm_strided(b.pool16 != nullptr, P.ta, P.tb, P.M, P.N, P.K, (float)P.alpha, A, P.lda, sa, Bm, P.ldb, sb, 1.0f,
                       C, P.ldc, sc, b.nvec, s);
  };
  timed(4, [&] {
    if (whole) whole_gemm(prog.h_gfull[0]);
    else run_dense<T>(prog.d1.get(), prog.n_d1, t, DENSE_TILE_TC, s);
  });
  timed(1, [&] { run_gemv<T>(prog.v1.get(), prog.n_v1, t, s); });
  timed(5, [&] {
    if (whole) whole_gemm(prog.h_gfull[1]);
    else run_dense<T>(prog.d2.get(), prog.n_d2, t, DENSE_TILE_TC, s);
    run_dense<T>(prog.d3.get(), prog.n_d3, t, 32, s);
  });
  // BF16 single-system calls: the phase-2 sandwiches on the tensor cores (blocks above
  // TCS_MAXN on the generic kernel)
  const bool tcs = sizeof(T) == 4 && t.nsys == 1 && t.s[0].pool16 && t.s[0].tcimg && t.s[0].ximg &&
                   prog.n_tcs_jobs > 0;
  timed(2, [&] {
    if (tcs) {
      run_sandwich_tc(prog.tcs_jobs.get(), prog.n_tcs_jobs, prog.tcs_slots.get(), prog.tcs_recs.get(),
                      prog.tcs_xblk.get(), prog.n_tcs_xblk, t, s);
      run_sandwich<T>(prog.gen2x.get(), prog.n_gen2x, t, prog.smem_elems, s);
    } else {
      n2 = small(prog.small2);
      run_sandwich<T>(prog.gen2.get(), prog.n_gen2, t, prog.smem_elems, s);
    }
  });
  timed(3, [&] { run_gemv<T>(prog.v2.get(), prog.n_v2, t, s); });
  if (P) {   // kernel launches per class in this call
    P->prof_launches[0] += n0 + (prog.n_gen1 > 0);
    P->prof_launches[1] += prog.n_v1 > 0;
    P->prof_launches[2] += tcs ? 2 + (prog.n_gen2x > 0) : n2 + (prog.n_gen2 > 0);
    P->prof_launches[3] += prog.n_v2 > 0;
    P->prof_launches[4] += whole ? 1 : prog.n_d1 > 0;
    P->prof_launches[5] += (whole ? 1 : prog.n_d2 > 0) + (prog.n_d3 > 0);
  }
}
template void run_program<double>(const Program&, const SysTable&, const int64_t*, const int64_t*, cudaStream_t, pnoeom_pno*,
                                   bool);
template void run_program<float>(const Program&, const SysTable&, const int64_t*, const int64_t*, cudaStream_t, pnoeom_pno*,
                                  bool);

template <typename T>
void apply_sigma(pnoeom_pno* P, int nvec, const T* r, T* out, cudaStream_t s, bool bf16) {
  if (nvec <= 0) return;
  DBuf<T>& work = work_of<T>(P);
  const size_t need = (size_t)nvec * P->work_len;
  if (work.n < need) work.alloc(need, &P->footprint);
  SysTable t{};
  t.nsys = 1;
  t.max_nvec = nvec;
  t.s[0] = sysbuf(P, nvec, r, out, work.get(), sizeof(T) == 4, bf16);
  if (t.s[0].tcimg) {   // X images of the tensor-core sandwich path
    const size_t needx = (size_t)nvec * P->prog.tcs_xstride;
    if (P->ximg.n < needx) P->ximg.alloc(needx, &P->footprint);
    t.s[0].ximg = P->ximg.get();
    t.s[0].ximg_stride = P->prog.tcs_xstride;
  }
  const int64_t ol = P->L, wl = P->work_len;
  run_program<T>(P->prog, t, &ol, &wl, s, P, true);
}
template void apply_sigma<double>(pnoeom_pno*, int, const double*, double*, cudaStream_t, bool);
template void apply_sigma<float>(pnoeom_pno*, int, const float*, float*, cudaStream_t, bool);

// Autotuner: time the FP32 sigma of nroots_sa vectors for every candidate group size of the
// grouped small-sandwich kernel and every roots-per-CTA choice (CUDA events on the build
// stream) and keep the fastest pair.
void autotune(pnoeom_pno* P, cudaStream_t s) {
  const int nv = std::max(1, P->nroots_sa);
  DBuf<float> r((size_t)nv * P->L), o((size_t)nv * P->L);
  r.zero(s);
  DBuf<float>& work = work_of<float>(P);
  if (work.n < (size_t)nv * P->work_len) work.alloc((size_t)nv * P->work_len, &P->footprint);
  SysTable t{};
  t.nsys = 1;
  t.max_nvec = nv;
  t.s[0] = sysbuf(P, nv, r.get(), o.get(), work.get(), true, false);
  tune_sets<float>(P->prog, t, s, P->tune_ms);
  // diagnostic overrides of the tuned small-kernel variants (tests force each variant):
  // PNOEOM_SMALL_PB (2 or 4, sets whose problems all have A and B), PNOEOM_SMALL_SHAPE
  // (1..3), PNOEOM_SMALL_NB (1 or 2)
  auto env_int = [](const char* name) {
    const char* e = std::getenv(name);
    return e ? std::atoi(e) : -1;
  };
  const int fpb = env_int("PNOEOM_SMALL_PB"), fsh = env_int("PNOEOM_SMALL_SHAPE"), fnb = env_int("PNOEOM_SMALL_NB");
  for (SmallSet* sets : {P->prog.small1, P->prog.small2})
    for (int k = 0; k < 3; ++k) {
      SmallSet& S = sets[k];
      if (fpb >= 1 && fpb <= 4) S.pb = S.ab ? fpb : 1;
      if (fsh >= 0 && fsh <= 3) S.shape = fsh;
      if (fnb >= 0 && fnb <= 2) S.nb = fnb;
    }
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
  }
  void symdiag(double* x) {
    if (nd) k_symdiag<<<nd, 256, 0, s>>>(x, dOffs.get(), dNs.get(), nd);
    PN_CUDA(cudaGetLastError());
  }
  void sigma(const double* V, double* S, int nv, int prec) {
    if (!nv) return;
    if (prec == PNOEOM_FP64) { apply_sigma<double>(P, nv, V, S, s, false); return; }
    size_t n = (size_t)nv * L;
    if (f_in.n < n) { f_in.alloc(n); f_out.alloc(n); }
    k_d2f_<<<gsz(n), 256, 0, s>>>(f_in.get(), V, n);
    apply_sigma<float>(P, nv, f_in.get(), f_out.get(), s, prec == PNOEOM_BF16);
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
  // orth() of t against rows 0..m-1 of V, applying the same combinations to st (sigma of t)
  // with the rows of S (sigma is linear, so st stays sigma of the orthonormalised t)
  double orth_pair(double* V, double* S, int m, double* t, double* st) {
    for (int pass = 0; pass < 2; ++pass) {
      if (!m) break;
      std::vector<double> c = gram(t, 1, V, m);
      for (double& x : c) x = -x;
      combine(t, V, c, m, 1, 1.0);
      combine(st, S, c, m, 1, 1.0);
    }
    std::vector<double> nn = gram(t, 1, t, 1);
    double nrm = std::sqrt(std::max(0.0, nn[0]));
    if (nrm > 0) {
      scale<double>(t, 1.0 / nrm, L, s);
      scale<double>(st, 1.0 / nrm, L, s);
    }
    return nrm;
  }
};
}  // namespace

// One system's Davidson solve as a state machine.  iterate() needs sigma of
// every vector in the pending slot range [p0, p1) of V in S; drive() or
// drive_round() evaluates those (for many systems at once in a batch) and calls
// iterate() again.  Sec. 2, PNO-EOM-CCSD Davidson; readings in the header of pnoeom.h.
struct DavState {
  pnoeom_pno* P;
  cudaStream_t s;
  int64_t L;
  int nroots, maxsub, max_iter;
  double res_tol, e_tol;
  bool refine;
  int prec;
  bool bf16 = false;        // the current low-precision phase reads the BF16 pool copy for its dense blocks
  double switch_res = 1e-4; // level below which a stalled low-precision phase hands over
  Dav D;
  DBuf<double> V, S, X, R;
  DBuf<float> fin, fout;    // FP32 copies of the pending vectors and their sigma
  int m = 0, nr = 0, it = 0, p0 = 0, p1 = 0;
  int64_t sigma_evals = 0;
  int64_t sigma_evals_prec[2] = {0, 0};   // FP32, FP64 sigma evaluations
  bool done = false, converged = false;
  bool trace = std::getenv("PNOEOM_LOG_DAVIDSON") != nullptr;
  std::vector<double> w, rn, w_old;
  std::vector<double> w_phase[2];  // Ritz values when the BF16 phase [0] and the FP32 phase [1] handed over
  std::vector<double> rhist;   // largest residual norm of every FP32 iteration (mixed solves)

  DavState(pnoeom_pno* P_, const pnoeom_opts* opts, cudaStream_t s_) : P(P_), s(s_), L(P_->L), D{P_, s_, P_->L} {
    nroots = opts->nroots_solve;
    PN_CHECK(nroots >= 1 && nroots <= P->nroots_sa, PNOEOM_ERR_INVALID_ARG, "nroots_solve must be in [1, nroots_sa]");
    PN_CHECK(L >= nroots, PNOEOM_ERR_INVALID_ARG, "PNO space smaller than the number of roots");
    maxsub = std::max(opts->max_subspace > 0 ? opts->max_subspace : 8 * nroots, 2 * nroots + 1);
    max_iter = opts->max_iter > 0 ? opts->max_iter : 100;
    res_tol = opts->res_tol > 0 ? opts->res_tol : 1e-7;
    e_tol = opts->e_tol > 0 ? opts->e_tol : 1e-10;
    prec = (opts->precision == PNOEOM_FP32 || opts->precision == PNOEOM_BF16) ? PNOEOM_FP32 : PNOEOM_FP64;
    bf16 = opts->precision == PNOEOM_BF16;
    // the BF16 blocks carry about 3 significant digits, so that phase stalls far above the
    // FP32 one's floor: it hands over to an FP32 phase as soon as its residuals stop halving
    // below 0.1, and the FP32 phase to FP64 as in a plain FP32 mixed solve
    switch_res = bf16 ? 1e-1 : 1e-4;
    refine = prec == PNOEOM_FP32 && opts->refine_fp64;
    // mixed precision: the FP32 phase aims at the final residual tolerance too and hands
    // over to the FP64 refinement when that holds or, below switch_res, when its largest
    // residual stops halving within three iterations (the error floor of the FP32 sigma)
    std::vector<int64_t> offs;
    std::vector<int> ns;
    for (int p = 0; p < P->npairs; ++p)
      if (P->pair_i[p] == P->pair_j[p] && P->nij[p] > 1) { offs.push_back(P->off_ij[p]); ns.push_back(P->nij[p]); }
    D.nd = (int)offs.size();
    D.dOffs.alloc(std::max<size_t>(1, offs.size())); D.dOffs.upload(offs.data(), offs.size(), s);
    D.dNs.alloc(std::max<size_t>(1, ns.size())); D.dNs.upload(ns.data(), ns.size(), s);
    V.alloc((size_t)maxsub * L); S.alloc((size_t)maxsub * L);
    X.alloc((size_t)nroots * L); R.alloc((size_t)nroots * L);
    for (int k = 0; k < P->nroots_sa && m < nroots; ++k) {   // projected CIS guesses
      double* t = V.get() + (int64_t)m * L;
      PN_CUDA(cudaMemcpyAsync(t, P->guesses.get() + (int64_t)k * L, L * 8, cudaMemcpyDeviceToDevice, s));
      if (D.orth(V.get(), m, t) > 1e-10) ++m;
    }
    PN_CHECK(m > 0, PNOEOM_ERR_INVALID_ARG, "no guess vector survives the projection");
    nr = std::min(nroots, m);
    p0 = 0; p1 = m;
  }

  // one Davidson iteration on the current subspace (all sigma available)
  void iterate() {
    if (++it > max_iter) { it = max_iter; done = true; return; }
    std::vector<double> G = D.gram(V.get(), m, S.get(), m);   // G[a][b] = <v_a, sigma(v_b)>
    std::vector<double> wr(m), wi(m), VR((size_t)m * m);
    PN_CHECK(small_eig(m, G.data(), wr.data(), wi.data(), VR.data()) == 0, PNOEOM_ERR_NOT_CONVERGED,
             "subspace eigensolver did not converge");
    std::vector<int> ord(m);
    for (int a = 0; a < m; ++a) ord[a] = a;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return wr[a] < wr[b]; });
    nr = std::min(nroots, m);
    w.assign(nr, 0.0);
    std::vector<double> Cy((size_t)nr * m);
    for (int q = 0; q < nr; ++q) {
      w[q] = wr[ord[q]];
      for (int a = 0; a < m; ++a) Cy[(size_t)q * m + a] = VR[(size_t)a * m + ord[q]];
    }
    D.combine(X.get(), V.get(), Cy, m, nr, 0.0);                  // Ritz vectors
    D.combine(R.get(), S.get(), Cy, m, nr, 0.0);                  // sigma of Ritz vectors
    for (int q = 0; q < nr; ++q) axpby<double>(R.get() + (int64_t)q * L, X.get() + (int64_t)q * L, -w[q], 1.0, L, s);
    rn.assign(nr, 0.0);
    for (int q = 0; q < nr; ++q)
      rn[q] = std::sqrt(std::max(0.0, D.gram(R.get() + (int64_t)q * L, 1, R.get() + (int64_t)q * L, 1)[0]));
    double dw = 1e300;
    if ((int)w_old.size() == nr) { dw = 0; for (int q = 0; q < nr; ++q) dw = std::max(dw, std::fabs(w[q] - w_old[q])); }
    w_old = w;
    if (trace) {   // PNOEOM_LOG_DAVIDSON: one line per iteration
      double rmax = 0;
      for (double x : rn) rmax = std::max(rmax, x);
      std::fprintf(stderr, "[davidson] L=%lld it=%d m=%d prec=%s max|r|=%.3e dw=%.3e w0=%.10f\n", (long long)L, it, m,
                   prec == PNOEOM_FP32 ? "fp32" : "fp64", rmax, dw, w.empty() ? 0.0 : w[0]);
    }
    bool conv = true;
    for (int q = 0; q < nr; ++q) conv = conv && rn[q] < res_tol;
    conv = conv && (prec == PNOEOM_FP32 && refine ? true : dw < e_tol);
    if (conv) { finish_or_refine(); return; }
    if (prec == PNOEOM_FP32 && refine) {
      double rmax = 0;
      for (double x : rn) rmax = std::max(rmax, x);
      rhist.push_back(rmax);
      const size_t k = rhist.size();
      if (rmax < switch_res && k >= 4 && rmax > 0.5 * rhist[k - 4]) { finish_or_refine(); return; }
    }
    std::vector<int> add;
    for (int q = 0; q < nr; ++q) if (rn[q] >= res_tol) add.push_back(q);
    int first_new = m;
    if (m + (int)add.size() > maxsub) {
      // thick restart: keep the Ritz vectors of the lowest nkeep subspace eigenvalues (at
      // least 2N, half the subspace), with their sigma formed from the stored sigma vectors
      // by the same combinations (no new sigma evaluations)
      const int nkeep = std::max(nr, std::min(m, std::min(std::max(2 * nr, maxsub / 2), maxsub - (int)add.size())));
      std::vector<double> Ck((size_t)nkeep * m);
      for (int q = 0; q < nkeep; ++q)
        for (int a = 0; a < m; ++a) Ck[(size_t)q * m + a] = VR[(size_t)a * m + ord[q]];
      DBuf<double> Xk((size_t)nkeep * L), Sk((size_t)nkeep * L);
      D.combine(Xk.get(), V.get(), Ck, m, nkeep, 0.0);
      D.combine(Sk.get(), S.get(), Ck, m, nkeep, 0.0);
      int mm = 0;
      for (int q = 0; q < nkeep; ++q) {
        double* t = V.get() + (int64_t)mm * L;
        double* st = S.get() + (int64_t)mm * L;
        PN_CUDA(cudaMemcpyAsync(t, Xk.get() + (int64_t)q * L, L * 8, cudaMemcpyDeviceToDevice, s));
        PN_CUDA(cudaMemcpyAsync(st, Sk.get() + (int64_t)q * L, L * 8, cudaMemcpyDeviceToDevice, s));
        if (D.orth_pair(V.get(), S.get(), mm, t, st) > 1e-10) ++mm;
      }
      m = mm;
      first_new = m;
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
    if (m == m0 && first_new == m) {   // no new direction: converged if every residual is within tolerance
      bool allres = true;
      for (int q = 0; q < nr; ++q) allres = allres && rn[q] < res_tol;
      // an FP32 phase whose directions the FP32 sigma can no longer resolve hands over to FP64
      if (allres || (prec == PNOEOM_FP32 && refine)) { finish_or_refine(); return; }
      done = true;
      return;
    }
    p0 = first_new; p1 = m;
  }

  void finish_or_refine() {
    if (prec == PNOEOM_FP32 && refine) {
      // the next phase (BF16 -> FP32 -> FP64) starts from the current Ritz vectors: the
      // subspace collapses onto them (orthonormalised) and only their sigma is evaluated
      // again, in the next precision
      w_phase[bf16 ? 0 : 1] = w;
      rhist.clear();
      if (bf16) { bf16 = false; switch_res = 1e-4; }
      else prec = PNOEOM_FP64;
      w_old.clear();
      int mm = 0;
      for (int q = 0; q < nr; ++q) {
        double* t = V.get() + (int64_t)mm * L;
        PN_CUDA(cudaMemcpyAsync(t, X.get() + (int64_t)q * L, L * 8, cudaMemcpyDeviceToDevice, s));
        if (D.orth(V.get(), mm, t) > 1e-10) ++mm;
      }
      m = mm;
      p0 = 0; p1 = m;
      return;
    }
    converged = true;
    done = true;
  }

  void results(double* energies, double* res_norms, int* iters) {
    for (int q = 0; q < nr; ++q) { energies[q] = w.size() > (size_t)q ? w[q] : NAN; res_norms[q] = rn.size() > (size_t)q ? rn[q] : NAN; }
    for (int q = nr; q < nroots; ++q) { energies[q] = NAN; res_norms[q] = NAN; }
    *iters = it;
    P->last_X.resize((size_t)nr * L);
    X.download(P->last_X.data(), P->last_X.size(), s);
    PN_CUDA(cudaStreamSynchronize(s));
    P->last_nroots = nr;
  }
};

// Drives a set of Davidson states in lockstep: in every round, the pending
// sigma vectors of all states (in chunks of at most `chunk` per state) are
// evaluated by `eval(states, nvec, prec)`, which must fill S[p0 .. p0+nvec)
// of each state with nvec > 0; states whose pending range is empty iterate.
template <typename Eval>
void drive(std::vector<DavState*>& st, int chunk, Eval&& eval) {
  for (;;) {
    bool any = false;
    for (DavState* d : st)
      while (!d->done && d->p0 >= d->p1) d->iterate();
    for (DavState* d : st) any = any || !d->done;
    if (!any) return;
    for (int prec : {PNOEOM_FP32, PNOEOM_FP64}) {
      std::vector<int> nv(st.size(), 0);
      bool need = false;
      for (size_t k = 0; k < st.size(); ++k)
        if (!st[k]->done && st[k]->prec == prec && st[k]->p0 < st[k]->p1) {
          nv[k] = std::min(chunk, st[k]->p1 - st[k]->p0);
          need = true;
        }
      if (!need) continue;
      eval(st, nv, prec);
      for (size_t k = 0; k < st.size(); ++k) {
        st[k]->p0 += nv[k];
        st[k]->sigma_evals += nv[k];
        st[k]->sigma_evals_prec[prec == PNOEOM_FP64] += nv[k];
      }
    }
  }
}

// One round of the lockstep driver (continuous batching): states with an empty
// pending range iterate, then every state's pending chunk is evaluated.
template <typename Eval>
void drive_round(std::vector<DavState*>& st, int chunk, Eval&& eval) {
  for (DavState* d : st)
    while (!d->done && d->p0 >= d->p1) d->iterate();
  for (int prec : {PNOEOM_FP32, PNOEOM_FP64}) {
    std::vector<int> nv(st.size(), 0);
    bool need = false;
    for (size_t k = 0; k < st.size(); ++k)
      if (!st[k]->done && st[k]->prec == prec && st[k]->p0 < st[k]->p1) {
        nv[k] = std::min(chunk, st[k]->p1 - st[k]->p0);
        need = true;
      }
    if (!need) continue;
    eval(st, nv, prec);
    for (size_t k = 0; k < st.size(); ++k) {
      st[k]->p0 += nv[k];
      st[k]->sigma_evals += nv[k];
      st[k]->sigma_evals_prec[prec == PNOEOM_FP64] += nv[k];
    }
  }
}

// sigma of each state's pending chunk through one program launch sequence
void eval_states(const Program& prog, std::vector<DavState*>& st, const std::vector<int>& nv, int prec,
                 std::vector<DBuf<double>>* work64, std::vector<DBuf<float>>* work32, cudaStream_t s,
                 pnoeom_pno* timing_owner) {
  SysTable t{};
  t.nsys = (int)st.size();
  t.max_nvec = 0;
  std::vector<int64_t> ol(st.size()), wl(st.size());
  for (size_t k = 0; k < st.size(); ++k) {
    DavState* d = st[k];
    ol[k] = d->L; wl[k] = d->P->work_len;
    const int n = nv[k];
    t.max_nvec = std::max(t.max_nvec, n);
    if (!n) { t.s[k] = SysBuf{}; continue; }
    const size_t need = (size_t)n * d->P->work_len;
    if (prec == PNOEOM_FP64) {
      DBuf<double>& w = (*work64)[k];
      if (w.n < need) w.alloc(need);
      t.s[k] = sysbuf(d->P, n, d->V.get() + (int64_t)d->p0 * d->L, d->S.get() + (int64_t)d->p0 * d->L, w.get(), false, false);
    } else {
      DBuf<float>& w = (*work32)[k];
      if (w.n < need) w.alloc(need);
      const size_t len = (size_t)n * d->L;
      if (d->fin.n < len) { d->fin.alloc(len); d->fout.alloc(len); }
      d2f(d->fin.get(), d->V.get() + (int64_t)d->p0 * d->L, len, s);
      t.s[k] = sysbuf(d->P, n, d->fin.get(), d->fout.get(), w.get(), true, d->bf16);
    }
  }
  if (prec == PNOEOM_FP64) run_program<double>(prog, t, ol.data(), wl.data(), s, timing_owner);
  else run_program<float>(prog, t, ol.data(), wl.data(), s, timing_owner);
  if (prec == PNOEOM_FP32)
    for (size_t k = 0; k < st.size(); ++k)
      if (nv[k]) f2d(st[k]->S.get() + (int64_t)st[k]->p0 * st[k]->L, st[k]->fout.get(), (size_t)nv[k] * st[k]->L, s);
}

void run_davidson(pnoeom_ctx* ctx, pnoeom_pno* P, const pnoeom_opts* opts, cudaStream_t s, double* energies,
                  double* res_norms, int* iters, int* converged) {
  (void)ctx;
  DavState d(P, opts, s);
  std::vector<DavState*> st{&d};
  std::vector<DBuf<double>> w64(1);
  std::vector<DBuf<float>> w32(1);
  drive(st, d.maxsub, [&](std::vector<DavState*>& ss, const std::vector<int>& nv, int prec) {
    eval_states(P->prog, ss, nv, prec, &w64, &w32, s, nullptr);
  });
  d.results(energies, res_norms, iters);
  P->last_sigma_evals[0] = d.sigma_evals_prec[0];
  P->last_sigma_evals[1] = d.sigma_evals_prec[1];
  P->last_phase_w[0] = d.w_phase[0];
  P->last_phase_w[1] = d.w_phase[1];
  *converged = d.converged ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Batches of systems

// Merge the members' programs: every problem keeps its offsets (relative to its
// own system's buffers) and gets the member index as its system index.
void batch_build(pnoeom_batch* B, cudaStream_t s) { batch_merge(B, s, true); }

void batch_merge(pnoeom_batch* B, cudaStream_t s, bool tune) {
  const int n = (int)B->members.size();
  PN_CHECK(n >= 1 && n <= MAX_SYS, PNOEOM_ERR_INVALID_ARG, "a batch holds 1.." + std::to_string(MAX_SYS) + " systems");
  B->prog = Program();
  Program& G = B->prog;
  for (int k = 0; k < n; ++k) {
    const Program& Pg = B->members[k]->prog;
    auto add = [&](std::vector<SProb>& dst, const std::vector<SProb>& src) {
      for (SProb q : src) { q.sys = k; dst.push_back(q); }
    };
    auto addv = [&](std::vector<VProb>& dst, const std::vector<VProb>& src) {
      for (VProb q : src) { q.sys = k; dst.push_back(q); }
    };
    auto addd = [&](std::vector<DProb>& dst, const std::vector<DProb>& src) {
      for (DProb q : src) { q.sys = k; dst.push_back(q); }
    };
    add(G.h_gen1, Pg.h_gen1); add(G.h_gen2, Pg.h_gen2);
    addv(G.h_v1, Pg.h_v1); addv(G.h_v2, Pg.h_v2);
    addd(G.h_d1, Pg.h_d1); addd(G.h_d2, Pg.h_d2); addd(G.h_d3, Pg.h_d3);
    G.smem_elems = std::max(G.smem_elems, Pg.smem_elems);
    for (int phase = 0; phase < 2; ++phase)
      for (int b = 0; b < 3; ++b) {
        SmallSet& D = phase == 0 ? G.small1[b] : G.small2[b];
        const SmallSet& S = phase == 0 ? Pg.small1[b] : Pg.small2[b];
        const int base = (int)D.h_probs.size();
        for (SProb q : S.h_probs) { q.sys = k; D.h_probs.push_back(q); }
        for (int c = 0; c < NGROUP_CAND; ++c) {
          if (!D.h_starts[c].empty()) D.h_starts[c].pop_back();   // drop the previous end marker
          for (size_t x = 0; x + 1 < S.h_starts[c].size(); ++x) D.h_starts[c].push_back(base + S.h_starts[c][x]);
          D.h_starts[c].push_back((int)D.h_probs.size());
        }
        for (int d = 0; d < 4; ++d) D.dims[d] = std::max(D.dims[d], S.dims[d]);
        if (S.nprob) {   // members with problems in this set
          D.ab = base == 0 ? S.ab : (D.ab && S.ab);
          D.pb = base == 0 ? S.pb : std::min(D.pb, S.pb);
          D.nb = base == 0 ? S.nb : (D.nb == S.nb ? D.nb : 0);
          D.shape = base == 0 ? S.shape : (D.shape == S.shape ? D.shape : 0);
        }
        if (!D.ab) D.pb = 1;
      }
  }
  G.upload(s, &B->footprint);
  B->w64.resize(n);
  B->w32.resize(n);
  G.group_choice = B->members[0]->prog.group_choice;
  G.rpc_choice = B->members[0]->prog.rpc_choice;
  for (int phase = 0; phase < 2; ++phase)   // untuned merge: each set takes the first member's choice
    for (int b = 0; b < 3; ++b) {
      SmallSet& D = phase == 0 ? G.small1[b] : G.small2[b];
      const SmallSet& S0 = phase == 0 ? B->members[0]->prog.small1[b] : B->members[0]->prog.small2[b];
      D.gchoice = S0.gchoice; D.rchoice = S0.rchoice;
    }
  if (!tune) return;
  // autotune the merged program's small sets: FP32, nroots_sa vectors per member
  std::vector<DBuf<float>> r(n), o(n);
  SysTable t{};
  t.nsys = n;
  for (int k = 0; k < n; ++k) {
    pnoeom_pno* P = B->members[k];
    const int nv = std::max(1, P->nroots_sa);
    r[k].alloc((size_t)nv * P->L);
    o[k].alloc((size_t)nv * P->L);
    r[k].zero(s);
    if (B->w32[k].n < (size_t)nv * P->work_len) B->w32[k].alloc((size_t)nv * P->work_len);
    t.max_nvec = std::max(t.max_nvec, nv);
    t.s[k] = sysbuf(P, nv, r[k].get(), o[k].get(), B->w32[k].get(), true, false);
  }
  tune_sets<float>(G, t, s, B->tune_ms);
}

// Capture `body` (stream operations on s) as a CUDA graph and launch it, reusing
// the batch's executable graph through cudaGraphExecUpdate when the topology is
// unchanged (only kernel parameters and pointers differ between calls).
template <typename Body>
void graph_launch(pnoeom_batch* B, cudaStream_t s, Body&& body) {
  if (!B->use_graph || s == nullptr) { body(); return; }
  cudaGraph_t g = nullptr;
  {
    // no allocation, free or trim of another library thread during the capture
    std::lock_guard<std::recursive_mutex> lk(capture_mutex());
    PN_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    try {
      body();
    } catch (...) {
      cudaStreamEndCapture(s, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    PN_CUDA(cudaStreamEndCapture(s, &g));
  }
  bool ok = false;
  if (B->exec) {
    cudaGraphExecUpdateResultInfo info;
    ok = cudaGraphExecUpdate(B->exec, g, &info) == cudaSuccess;
    if (!ok) { cudaGetLastError(); cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
    else ++B->graph_updates;
  }
  if (!ok) {
    PN_CUDA(cudaGraphInstantiate(&B->exec, g, 0));
    ++B->graph_instantiations;
  }
  cudaGraphDestroy(g);
  PN_CUDA(cudaGraphLaunch(B->exec, s));
  ++B->graph_launches;
}

void batch_sigma(pnoeom_batch* B, const int* nvec, const void* const* r, void* const* out, int prec, cudaStream_t s) {
  const int n = (int)B->members.size();
  SysTable t{};
  t.nsys = n;
  std::vector<int64_t> ol(n), wl(n);
  for (int k = 0; k < n; ++k) {
    pnoeom_pno* P = B->members[k];
    ol[k] = P->L; wl[k] = P->work_len;
    const int nv = nvec[k];
    t.max_nvec = std::max(t.max_nvec, nv);
    if (nv <= 0) { t.s[k] = SysBuf{}; continue; }
    PN_CHECK(r[k] && out[k], PNOEOM_ERR_INVALID_ARG, "NULL vector in batch sigma");
    const size_t need = (size_t)nv * P->work_len;
    void* w;
    if (prec == PNOEOM_FP64) { if (B->w64[k].n < need) B->w64[k].alloc(need); w = B->w64[k].get(); }
    else { if (B->w32[k].n < need) B->w32[k].alloc(need); w = B->w32[k].get(); }
    t.s[k] = sysbuf(P, nv, r[k], out[k], w, prec != PNOEOM_FP64, prec == PNOEOM_BF16);
  }
  graph_launch(B, s, [&] {
    if (prec == PNOEOM_FP64) run_program<double>(B->prog, t, ol.data(), wl.data(), s, nullptr);
    else run_program<float>(B->prog, t, ol.data(), wl.data(), s, nullptr);
  });
}

void batch_solve(pnoeom_batch* B, const pnoeom_opts* opts, cudaStream_t s, double* energies, double* res_norms,
                 int* iters, int* converged) {
  const int n = (int)B->members.size();
  std::vector<std::unique_ptr<DavState>> own;
  std::vector<DavState*> st;
  for (int k = 0; k < n; ++k) {
    own.emplace_back(new DavState(B->members[k], opts, s));
    st.push_back(own.back().get());
  }
  std::vector<DBuf<double>>& w64 = B->w64;
  std::vector<DBuf<float>>& w32 = B->w32;
  drive(st, opts->nroots_solve, [&](std::vector<DavState*>& ss, const std::vector<int>& nv, int prec) {
    // work buffers first (no allocation inside the captured region)
    for (size_t k = 0; k < ss.size(); ++k) {
      if (!nv[k]) continue;
      const size_t need = (size_t)nv[k] * ss[k]->P->work_len;
      if (prec == PNOEOM_FP64) { if (w64[k].n < need) w64[k].alloc(need); }
      else {
        if (w32[k].n < need) w32[k].alloc(need);
        const size_t len = (size_t)nv[k] * ss[k]->L;
        if (ss[k]->fin.n < len) { ss[k]->fin.alloc(len); ss[k]->fout.alloc(len); }
      }
    }
    graph_launch(B, s, [&] { eval_states(B->prog, ss, nv, prec, &w64, &w32, s, nullptr); });
  });
  const int nroots = opts->nroots_solve;
  for (int k = 0; k < n; ++k) {
    st[k]->results(energies + (size_t)k * nroots, res_norms + (size_t)k * nroots, iters + k);
    converged[k] = st[k]->converged ? 1 : 0;
  }
}

// ---------------------------------------------------------------------------
// Serving: continuous batching of Davidson solves (a12)

struct Request {
  int64_t id = 0;
  int o = 0, v = 0, naux = 0;
  std::vector<double> eps, B, t1, t2;
  bool has_t1 = false, has_t2 = false;
  pnoeom_opts opts{};
  int status = PNOEOM_REQ_QUEUED;
  int error = 0;
  std::string message;
  size_t est_bytes = 0, resident_bytes = 0;
  double t_submit = 0, t_admit = 0, t_built = 0, t_done = 0;
  pnoeom_pno* pno = nullptr;
  std::unique_ptr<DavState> dav;
  std::vector<double> energies, res_norms;
  int iters = 0;
  int64_t sigma_evals = 0;
};

static double wall_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Upper estimate of the device memory a build of (o, v, naux) needs at its peak:
// the DF factors, the v^3 o integral blocks and their projected copies, and the
// o^2 v^2 amplitude-sized intermediates.
size_t estimate_build_bytes(int o, int v, int naux) {
  const double O = o, Vv = v, nmo = o + v;
  return (size_t)(8.0 * (2.0 * naux * nmo * nmo + 6.0 * O * Vv * Vv * Vv + 16.0 * O * O * Vv * Vv) + 256e6);
}

}  // namespace pnoeom


namespace pnoeom {

static void server_builder(pnoeom_server* S) {
  auto fail = [&](const char* why) {   // the server cannot run: stop it and tell every waiter
    std::lock_guard<std::mutex> lk(S->mu);
    S->fatal = why;
    S->stop = true;
    S->cv.notify_all();
  };
  if (cudaSetDevice(S->device) != cudaSuccess) { fail("builder: cudaSetDevice failed"); return; }
  pnoeom_ctx bctx;
  bctx.device = S->device;
  if (cusolverDnCreate(&bctx.solver) != CUSOLVER_STATUS_SUCCESS) { fail("builder: cusolverDnCreate failed"); return; }
  cudaStream_t bs;
  if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess) {
    cusolverDnDestroy(bctx.solver);
    bctx.solver = nullptr;
    fail("builder: cudaStreamCreateWithFlags failed");
    return;
  }
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] {
        if (S->stop) return true;
        for (auto& q : S->queued)
          if (!S->budget || S->used + q->est_bytes <= S->budget) return true;
        return false;
      });
      if (S->stop) break;
      for (auto it = S->queued.begin(); it != S->queued.end(); ++it)   // oldest request that fits
        if (!S->budget || S->used + (*it)->est_bytes <= S->budget) { r = *it; S->queued.erase(it); break; }
      if (!r) continue;
      S->used += r->est_bytes;
      r->status = PNOEOM_REQ_BUILDING;
      r->t_admit = wall_s() - S->t0;
    }
    pnoeom_system sys{r->o, r->v, r->naux, r->eps.data(), r->B.data(), r->has_t1 ? r->t1.data() : nullptr,
                      r->has_t2 ? r->t2.data() : nullptr, PNOEOM_HOST};
    auto* P = new pnoeom_pno();
    int code = guard_call([&] { build_system(&bctx, &sys, &r->opts, bs, P); });
    const std::string why = code == PNOEOM_OK ? "" : std::string(pnoeom_last_error());
    std::lock_guard<std::mutex> lk(S->mu);
    S->used -= r->est_bytes;
    r->B.clear(); r->B.shrink_to_fit(); r->t2.clear(); r->t2.shrink_to_fit();
    if (code != PNOEOM_OK) {
      delete P;
      r->status = PNOEOM_REQ_FAILED;
      r->error = code;
      r->message = "build failed: " + why;
      r->t_done = wall_s() - S->t0;
    } else {
      r->pno = P;
      r->resident_bytes = P->footprint;
      S->used += r->resident_bytes;
      r->t_built = wall_s() - S->t0;
      S->built.push_back(r);
    }
    S->cv.notify_all();
  }
  cudaStreamDestroy(bs);
  cusolverDnDestroy(bctx.solver);
}

static void server_solver(pnoeom_server* S) {
  cudaStream_t ss;
  if (cudaSetDevice(S->device) != cudaSuccess || cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking) != cudaSuccess) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->fatal = "solver: no stream on the server's device";
    S->stop = true;
    S->cv.notify_all();
    return;
  }
  std::vector<std::shared_ptr<Request>> active;
  pnoeom_batch B;
  bool dirty = true;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] { return S->stop || !active.empty() || !S->built.empty(); });
      if (S->stop) break;
      while (!S->built.empty() && (int)active.size() < S->max_active) {   // join at the round boundary
        auto r = S->built.front();
        S->built.pop_front();
        r->status = PNOEOM_REQ_RUNNING;
        active.push_back(r);
        dirty = true;
      }
    }
    // Davidson states of new members (outside the lock: device work)
    for (auto& r : active) {
      if (r->dav) continue;
      int code = guard_call([&] { r->dav.reset(new DavState(r->pno, &r->opts, ss)); });
      if (code != PNOEOM_OK) {
        std::lock_guard<std::mutex> lk(S->mu);
        r->status = PNOEOM_REQ_FAILED; r->error = code; r->message = "solver setup failed";
      }
    }
    // drop failed ones
    active.erase(std::remove_if(active.begin(), active.end(), [&](auto& r) {
                   if (r->status != PNOEOM_REQ_FAILED) return false;
                   std::lock_guard<std::mutex> lk(S->mu);
                   S->used -= r->resident_bytes;
                   delete r->pno; r->pno = nullptr;
                   r->t_done = wall_s() - S->t0;
                   dirty = true;
                   S->cv.notify_all();
                   return true;
                 }),
                 active.end());
    if (active.empty()) continue;
    int code = guard_call([&] {
      if (dirty) {
        B.members.clear();
        for (auto& r : active) B.members.push_back(r->pno);
        if (B.exec) { cudaGraphExecDestroy(B.exec); B.exec = nullptr; }
        batch_merge(&B, ss, false);
        dirty = false;
        std::lock_guard<std::mutex> lk(S->mu);
        ++S->merges;
      }
      std::vector<DavState*> st;
      for (auto& r : active) st.push_back(r->dav.get());
      int chunk = 1;
      for (auto& r : active) chunk = std::max(chunk, r->opts.nroots_solve);
      drive_round(st, chunk, [&](std::vector<DavState*>& xs, const std::vector<int>& nv, int prec) {
        for (size_t k = 0; k < xs.size(); ++k) {
          if (!nv[k]) continue;
          const size_t need = (size_t)nv[k] * xs[k]->P->work_len;
          if (prec == PNOEOM_FP64) { if (B.w64[k].n < need) B.w64[k].alloc(need); }
          else {
            if (B.w32[k].n < need) B.w32[k].alloc(need);
            const size_t len = (size_t)nv[k] * xs[k]->L;
            if (xs[k]->fin.n < len) { xs[k]->fin.alloc(len); xs[k]->fout.alloc(len); }
          }
        }
        graph_launch(&B, ss, [&] { eval_states(B.prog, xs, nv, prec, &B.w64, &B.w32, ss, nullptr); });
      });
      // retire finished requests
      std::vector<std::shared_ptr<Request>> keep;
      for (auto& r : active) {
        if (!r->dav->done) { keep.push_back(r); continue; }
        const int nr = r->opts.nroots_solve;
        r->energies.assign(nr, NAN); r->res_norms.assign(nr, NAN);
        r->dav->results(r->energies.data(), r->res_norms.data(), &r->iters);
        r->sigma_evals = r->dav->sigma_evals;
        const bool ok = r->dav->converged;
        r->dav.reset();
        delete r->pno; r->pno = nullptr;
        std::lock_guard<std::mutex> lk(S->mu);
        S->used -= r->resident_bytes;
        S->total_sigma_evals += r->sigma_evals;
        r->status = ok ? PNOEOM_REQ_DONE : PNOEOM_REQ_FAILED;
        if (!ok) { r->error = PNOEOM_ERR_NOT_CONVERGED; r->message = "Davidson did not converge"; }
        r->t_done = wall_s() - S->t0;
        dirty = true;
        S->cv.notify_all();
      }
      if (keep.size() != active.size()) pool_trim();   // return retired memory to CUDA
      active.swap(keep);
      std::lock_guard<std::mutex> lk(S->mu);
      ++S->rounds;
    });
    if (code != PNOEOM_OK) {   // a round failed: fail every active request
      std::lock_guard<std::mutex> lk(S->mu);
      for (auto& r : active) {
        r->status = PNOEOM_REQ_FAILED; r->error = code; r->message = "solver round failed";
        r->dav.reset(); delete r->pno; r->pno = nullptr;
        S->used -= r->resident_bytes;
        r->t_done = wall_s() - S->t0;
      }
      active.clear();
      dirty = true;
      S->cv.notify_all();
    }
  }
  for (auto& r : active) { r->dav.reset(); delete r->pno; r->pno = nullptr; }
  if (B.exec) { cudaGraphExecDestroy(B.exec); B.exec = nullptr; }
  cudaStreamDestroy(ss);
}

void server_start(pnoeom_server* S) {
  S->t0 = wall_s();
  int nb = 3;   // builder threads; PNOEOM_SERVER_BUILDERS overrides (1..16)
  if (const char* e = std::getenv("PNOEOM_SERVER_BUILDERS")) nb = std::max(1, std::min(16, std::atoi(e)));
  for (int k = 0; k < nb; ++k) S->builders.emplace_back(server_builder, S);
  S->solver = std::thread(server_solver, S);
}

void server_stop(pnoeom_server* S) {
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto& b : S->builders)
    if (b.joinable()) b.join();
  if (S->solver.joinable()) S->solver.join();
}

int64_t server_submit(pnoeom_server* S, const pnoeom_system* sys, const pnoeom_opts* opts) {
  PN_CHECK(sys && opts && sys->eps && sys->B && sys->mem_space == PNOEOM_HOST, PNOEOM_ERR_INVALID_ARG,
           "server requests take host inputs");
  PN_CHECK(sys->o >= 1 && sys->v >= 1 && sys->naux >= 1, PNOEOM_ERR_INVALID_ARG, "o, v and naux must be positive");
  auto r = std::make_shared<Request>();
  const size_t nmo = sys->o + sys->v;
  r->o = sys->o; r->v = sys->v; r->naux = sys->naux;
  r->eps.assign(sys->eps, sys->eps + nmo);
  r->B.assign(sys->B, sys->B + (size_t)sys->naux * nmo * nmo);
  if (sys->t1) { r->has_t1 = true; r->t1.assign(sys->t1, sys->t1 + (size_t)sys->o * sys->v); }
  if (sys->t2) { r->has_t2 = true; r->t2.assign(sys->t2, sys->t2 + (size_t)sys->o * sys->o * sys->v * sys->v); }
  r->opts = *opts;
  r->est_bytes = estimate_build_bytes(sys->o, sys->v, sys->naux);
  std::lock_guard<std::mutex> lk(S->mu);
  PN_CHECK(S->fatal.empty(), PNOEOM_ERR_CUDA, S->fatal);
  r->id = S->next_id++;
  r->t_submit = wall_s() - S->t0;
  S->reqs[r->id] = r;
  if (S->budget && r->est_bytes > S->budget) {   // can never be admitted
    r->status = PNOEOM_REQ_FAILED;
    r->error = PNOEOM_ERR_NOMEM;
    r->message = "estimated footprint " + std::to_string(r->est_bytes) + " bytes exceeds the server budget";
    r->t_done = r->t_submit;
  } else {
    S->queued.push_back(r);
  }
  S->cv.notify_all();
  return r->id;
}

void server_poll(pnoeom_server* srv, int64_t id, int* status, double* energies, double* res_norms, int* iters,
                 int64_t* sigma_evals, double* times) {
    PN_CHECK(srv, PNOEOM_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    PN_CHECK(it != srv->reqs.end(), PNOEOM_ERR_INVALID_ARG, "unknown request id");
    const auto& r = *it->second;
    if (status) *status = r.status;
    if (r.status == PNOEOM_REQ_DONE) {
      for (size_t q = 0; q < r.energies.size(); ++q) {
        if (energies) energies[q] = r.energies[q];
        if (res_norms) res_norms[q] = r.res_norms[q];
      }
      if (iters) *iters = r.iters;
      if (sigma_evals) *sigma_evals = r.sigma_evals;
    }
    if (times) { times[0] = r.t_submit; times[1] = r.t_admit; times[2] = r.t_built; times[3] = r.t_done; }
    if (r.status == PNOEOM_REQ_FAILED)
      throw Error(r.error ? r.error : PNOEOM_ERR_CUDA, "request failed: " + r.message);
  }

void server_wait(pnoeom_server* srv, int64_t id, double timeout_s) {
    PN_CHECK(srv, PNOEOM_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    PN_CHECK(it != srv->reqs.end(), PNOEOM_ERR_INVALID_ARG, "unknown request id");
    auto r = it->second;
    bool ok = srv->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
      return r->status == PNOEOM_REQ_DONE || r->status == PNOEOM_REQ_FAILED || !srv->fatal.empty();
    });
    PN_CHECK(ok, PNOEOM_ERR_TIMEOUT, "request " + std::to_string(id) + " not finished within the timeout");
    PN_CHECK(r->status == PNOEOM_REQ_DONE || r->status == PNOEOM_REQ_FAILED, PNOEOM_ERR_CUDA,
             "server stopped: " + srv->fatal);
  }

void server_stats(pnoeom_server* srv, size_t* used_bytes, int* queued, int* running, int64_t* rounds,
                  int64_t* merges, int64_t* sigma_evals) {
    PN_CHECK(srv, PNOEOM_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(srv->mu);
    if (used_bytes) *used_bytes = srv->used;
    int q = 0, r = 0;
    for (auto& kv : srv->reqs) {
      q += kv.second->status == PNOEOM_REQ_QUEUED;
      r += kv.second->status == PNOEOM_REQ_BUILDING || kv.second->status == PNOEOM_REQ_RUNNING;
    }
    if (queued) *queued = q;
    if (running) *running = r;
    if (rounds) *rounds = srv->rounds;
    if (merges) *merges = srv->merges;
    if (sigma_evals) *sigma_evals = srv->total_sigma_evals;
  }

}  // namespace pnoeom
