// C entry points: argument checks, error translation, handle lifetime.
#include "pno.cuh"
#include <cmath>
#include <functional>
#include <chrono>
#include <mutex>

namespace pnoeom { int small_eig(int n, const double* A, double* wr, double* wi, double* VR); }

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace pnoeom {
// Runs f, translating exceptions into a return code and the thread-local message.
int guard_call(const std::function<void()>& f);
}

namespace {
int guard(const std::function<void()>& f) { return pnoeom::guard_call(f); }
}  // namespace

int pnoeom::guard_call(const std::function<void()>& f) {
  try {
    f();
    g_last_error.clear();
    return PNOEOM_OK;
  } catch (const pnoeom::Error& e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return PNOEOM_ERR_NOMEM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return PNOEOM_ERR_CUDA;
  } catch (...) {   // nothing may cross the C boundary
    g_last_error = "unknown exception";
    return PNOEOM_ERR_CUDA;
  }
}

namespace {
inline cudaStream_t st(void* p) { return reinterpret_cast<cudaStream_t>(p); }
}  // namespace

extern "C" {

const char* pnoeom_last_error(void) { return g_last_error.c_str(); }

int pnoeom_create(pnoeom_ctx** ctx, int device, size_t hbm_budget_bytes) {
  return guard([&] {
    PN_CHECK(ctx, PNOEOM_ERR_INVALID_ARG, "ctx is NULL");
    int ndev = 0;
    PN_CUDA(cudaGetDeviceCount(&ndev));
    PN_CHECK(device >= 0 && device < ndev, PNOEOM_ERR_INVALID_ARG, "no such CUDA device");
    pnoeom::DeviceScope dev_scope(device);
    auto* c = new pnoeom_ctx();
    c->device = device;
    c->budget = hbm_budget_bytes;
    if (cusolverDnCreate(&c->solver) != CUSOLVER_STATUS_SUCCESS) {
      delete c;
      throw pnoeom::Error(PNOEOM_ERR_CUDA, "cusolverDnCreate failed");
    }
    *ctx = c;
  });
}

void pnoeom_destroy(pnoeom_ctx* ctx) {
  if (!ctx) return;
  if (ctx->solver) cusolverDnDestroy(ctx->solver);
  delete ctx;
}

int pno_build(pnoeom_ctx* ctx, const pnoeom_system* sys, const pnoeom_opts* opts, void* cuda_stream, pnoeom_pno** out) {
  return guard([&] {
    PN_CHECK(ctx && sys && opts && out, PNOEOM_ERR_INVALID_ARG, "NULL argument");
    pnoeom::DeviceScope dev_scope(ctx->device);
    auto* P = new pnoeom_pno();
    try {
      pnoeom::build_system(ctx, sys, opts, st(cuda_stream), P);
      if (ctx->budget && P->footprint > ctx->budget)
        throw pnoeom::Error(PNOEOM_ERR_NOMEM, "device footprint " + std::to_string(P->footprint) +
                                                  " bytes exceeds the context budget");
    } catch (...) {
      // free the partial handle, then return the setup's cached blocks to CUDA (the
      // stream is drained first: blocks may still be in use by queued work)
      delete P;
      cudaStreamSynchronize(st(cuda_stream));
      pnoeom::pool_trim();
      throw;
    }
    *out = P;
  });
}

void pno_destroy(pnoeom_pno* pno) { delete pno; }

double pno_build_seconds(const pnoeom_pno* pno) { return pno ? pno->build_seconds : 0.0; }

int pno_autotune_info(const pnoeom_pno* pno, int ncand, int* group_sizes, int* roots_per_cta, double* ms, int* choice) {
  return guard([&] {
    PN_CHECK(pno, PNOEOM_ERR_INVALID_ARG, "pno is NULL");
    const int total = pnoeom::NTUNE;
    for (int c = 0; c < std::min(ncand, total); ++c) {
      if (group_sizes) group_sizes[c] = pnoeom::GROUP_CAND[c / pnoeom::NRPC_CAND];
      if (roots_per_cta) roots_per_cta[c] = pnoeom::RPC_CAND[c % pnoeom::NRPC_CAND];
      if (ms) ms[c] = pno->tune_ms[c];
    }
    if (choice) *choice = pno->prog.group_choice * pnoeom::NRPC_CAND + pno->prog.rpc_choice;
  });
}

int pno_set_timing(pnoeom_pno* pno, int enable) {
  return guard([&] {
    PN_CHECK(pno, PNOEOM_ERR_INVALID_ARG, "pno is NULL");
    for (auto& e : pno->events) { cudaEventSynchronize(e.second.second); cudaEventDestroy(e.second.first); cudaEventDestroy(e.second.second); }
    pno->events.clear();
    for (int& x : pno->prof_launches) x = 0;
    pno->timing = enable != 0;
  });
}

int pno_sigma_timing(const pnoeom_pno* pno, int k, int nvec, int precision, const char** name, int* launches,
                     double* ms, double* bytes, double* flops) {
  static const char* names[pnoeom_pno::NCLS] = {"sandwich->intermediates", "dense->intermediates", "sandwich->sigma",
                                                "dense->sigma", "gemm->intermediates", "gemm->sigma"};
  return guard([&] {
    PN_CHECK(pno && k >= 0 && k < pnoeom_pno::NCLS, PNOEOM_ERR_INVALID_ARG, "bad arguments");
    int n = 0;
    double t = 0;
    for (const auto& e : pno->events) {
      if (e.first != k) continue;
      PN_CUDA(cudaEventSynchronize(e.second.second));
      float x = 0;
      PN_CUDA(cudaEventElapsedTime(&x, e.second.first, e.second.second));
      t += x; ++n;   // n: sigma calls recorded
    }
    // element sizes: vectors 8 (FP64) or 4 bytes; operator blocks likewise, except in the
    // BF16 sigma the dense GEMV blocks (classes 1 and 3) and the operator images of the
    // tensor-core sandwich terms (class 2), read as 2-byte BF16 (blocks above that path's
    // size limit read the FP32 pool instead; the benchmark workloads have none)
    const double es = precision == PNOEOM_FP64 ? 8.0 : 4.0;
    const double ep = precision == PNOEOM_BF16 && (k == 1 || k == 2 || k == 3) ? 2.0 : es;
    if (name) *name = names[k];
    if (launches) *launches = pno->prof_launches[k];
    if (ms) *ms = t;
    if (bytes) *bytes = ep * pno->prof_pool_elems[k] + es * (double)nvec * pno->prof_vec_elems[k];
    if (flops) *flops = (double)nvec * pno->prof_flops[k];
  });
}

int pno_tc_mma_flops(const pnoeom_pno* pno, double* per_vector) {
  return guard([&] {
    PN_CHECK(pno && per_vector, PNOEOM_ERR_INVALID_ARG, "NULL argument");
    *per_vector = pno->prog.tcs_mma_flops;
  });
}

int pno_query(const pnoeom_pno* pno, int* npairs, const int** n_ij, const int** n_i, size_t* vec_len,
              size_t* footprint_bytes) {
  return guard([&] {
    PN_CHECK(pno, PNOEOM_ERR_INVALID_ARG, "pno is NULL");
    if (npairs) *npairs = pno->npairs;
    if (n_ij) *n_ij = pno->nij.data();
    if (n_i) *n_i = pno->ni.data();
    if (vec_len) *vec_len = (size_t)pno->L;
    if (footprint_bytes) *footprint_bytes = pno->footprint;
  });
}

int pno_get_basis(const pnoeom_pno* pno, int pair, double* U, double* fbar) {
  return guard([&] {
    PN_CHECK(pno && U, PNOEOM_ERR_INVALID_ARG, "NULL argument");
    int64_t uoff, foff;
    int n;
    if (pair >= 0) {
      PN_CHECK(pair < pno->npairs, PNOEOM_ERR_INVALID_ARG, "pair index out of range");
      uoff = pno->Uoff_pair[pair]; foff = pno->foff_pair[pair]; n = pno->nij[pair];
    } else {
      int i = -pair - 1;
      PN_CHECK(i < pno->o, PNOEOM_ERR_INVALID_ARG, "OSV index out of range");
      uoff = pno->Uoff_osv[i]; foff = pno->foff_osv[i]; n = pno->ni[i];
    }
    if (n) {
      PN_CUDA(cudaMemcpy(U, pno->U.get() + uoff, (size_t)pno->v * n * 8, cudaMemcpyDeviceToHost));
      if (fbar) PN_CUDA(cudaMemcpy(fbar, pno->fbar.get() + foff, (size_t)n * 8, cudaMemcpyDeviceToHost));
    }
  });
}

int sigma(pnoeom_ctx* ctx, const pnoeom_pno* pno, int nvec, const void* r_dev, void* s_dev, int precision,
          void* cuda_stream) {
  return guard([&] {
    PN_CHECK(ctx && pno, PNOEOM_ERR_INVALID_ARG, "NULL argument");
    PN_CHECK(nvec >= 0, PNOEOM_ERR_INVALID_ARG, "nvec < 0");
    if (nvec == 0) return;
    PN_CHECK(r_dev && s_dev, PNOEOM_ERR_INVALID_ARG, "NULL vector");
    pnoeom::DeviceScope dev_scope(ctx->device);
    auto* P = const_cast<pnoeom_pno*>(pno);
    if (precision == PNOEOM_FP64)
      pnoeom::apply_sigma<double>(P, nvec, (const double*)r_dev, (double*)s_dev, st(cuda_stream), false);
    else if (precision == PNOEOM_FP32 || precision == PNOEOM_BF16)
      pnoeom::apply_sigma<float>(P, nvec, (const float*)r_dev, (float*)s_dev, st(cuda_stream), precision == PNOEOM_BF16);
    else
      throw pnoeom::Error(PNOEOM_ERR_INVALID_ARG, "unknown precision");
  });
}

int davidson_solve(pnoeom_ctx* ctx, pnoeom_pno* pno, const pnoeom_opts* opts, void* cuda_stream, double* energies,
                   double* res_norms, int* iters) {
  int conv = 0;
  int rc = guard([&] {
    PN_CHECK(ctx && pno && opts && energies && res_norms && iters, PNOEOM_ERR_INVALID_ARG, "NULL argument");
    pnoeom::DeviceScope dev_scope(ctx->device);
    pnoeom::run_davidson(ctx, pno, opts, st(cuda_stream), energies, res_norms, iters, &conv);
    PN_CHECK(pnoeom::device_status(true, st(cuda_stream)) == 0, PNOEOM_ERR_TIMEOUT,
             "a tensor-core kernel's bounded wait ran out during the solve: results are invalid");
  });
  if (rc == PNOEOM_OK && !conv) {
    g_last_error = "Davidson did not converge within max_iter";
    return PNOEOM_ERR_NOT_CONVERGED;
  }
  return rc;
}

int pnoeom_batch_create(pnoeom_ctx* ctx, pnoeom_pno* const* members, int n, void* cuda_stream, pnoeom_batch** out) {
  return guard([&] {
    PN_CHECK(ctx && members && out && n >= 1, PNOEOM_ERR_INVALID_ARG, "bad arguments");
    for (int k = 0; k < n; ++k) PN_CHECK(members[k], PNOEOM_ERR_INVALID_ARG, "NULL member");
    pnoeom::DeviceScope dev_scope(ctx->device);
    auto* B = new pnoeom_batch();
    B->device = ctx->device;
    B->members.assign(members, members + n);
    try {
      pnoeom::batch_build(B, st(cuda_stream));
    } catch (...) {
      delete B;
      throw;
    }
    *out = B;
  });
}

void pnoeom_batch_destroy(pnoeom_batch* batch) { delete batch; }

int pnoeom_batch_sigma(pnoeom_ctx* ctx, pnoeom_batch* batch, const int* nvec, const void* const* r_dev,
                       void* const* s_dev, int precision, void* cuda_stream) {
  return guard([&] {
    PN_CHECK(ctx && batch && nvec && r_dev && s_dev, PNOEOM_ERR_INVALID_ARG, "NULL argument");
    PN_CHECK(precision == PNOEOM_FP64 || precision == PNOEOM_FP32 || precision == PNOEOM_BF16, PNOEOM_ERR_INVALID_ARG,
             "unknown precision");
    pnoeom::DeviceScope dev_scope(ctx->device);
    pnoeom::batch_sigma(batch, nvec, r_dev, s_dev, precision, st(cuda_stream));
  });
}

int pnoeom_batch_solve(pnoeom_ctx* ctx, pnoeom_batch* batch, const pnoeom_opts* opts, void* cuda_stream,
                       double* energies, double* res_norms, int* iters, int* converged) {
  int all = 1;
  int rc = guard([&] {
    PN_CHECK(ctx && batch && opts && energies && res_norms && iters && converged, PNOEOM_ERR_INVALID_ARG, "NULL argument");
    pnoeom::DeviceScope dev_scope(ctx->device);
    pnoeom::batch_solve(batch, opts, st(cuda_stream), energies, res_norms, iters, converged);
    PN_CHECK(pnoeom::device_status(true, st(cuda_stream)) == 0, PNOEOM_ERR_TIMEOUT,
             "a tensor-core kernel's bounded wait ran out during the solve: results are invalid");
    for (size_t k = 0; k < batch->members.size(); ++k) all = all && converged[k];
  });
  if (rc == PNOEOM_OK && !all) {
    g_last_error = "some batch members did not converge within max_iter";
    return PNOEOM_ERR_NOT_CONVERGED;
  }
  return rc;
}

int pnoeom_server_create(pnoeom_ctx* ctx, size_t hbm_budget_bytes, int max_active, pnoeom_server** out) {
  return guard([&] {
    PN_CHECK(ctx && out && max_active >= 1 && max_active <= pnoeom::MAX_SYS, PNOEOM_ERR_INVALID_ARG, "bad arguments");
    auto* S = new pnoeom_server();
    S->device = ctx->device;
    S->budget = hbm_budget_bytes;
    S->max_active = max_active;
    pnoeom::server_start(S);
    *out = S;
  });
}

void pnoeom_server_destroy(pnoeom_server* srv) {
  if (!srv) return;
  pnoeom::server_stop(srv);
  delete srv;
}

int pnoeom_server_submit(pnoeom_server* srv, const pnoeom_system* sys, const pnoeom_opts* opts, int64_t* id) {
  return guard([&] {
    PN_CHECK(srv && id, PNOEOM_ERR_INVALID_ARG, "NULL argument");
    *id = pnoeom::server_submit(srv, sys, opts);
  });
}

int pnoeom_server_poll(pnoeom_server* srv, int64_t id, int* status, double* energies, double* res_norms, int* iters,
                       int64_t* sigma_evals, double* times) {
  return guard([&] { pnoeom::server_poll(srv, id, status, energies, res_norms, iters, sigma_evals, times); });
}

int pnoeom_server_wait(pnoeom_server* srv, int64_t id, double timeout_s) {
  return guard([&] { pnoeom::server_wait(srv, id, timeout_s); });
}

int pnoeom_server_stats(pnoeom_server* srv, size_t* used_bytes, int* queued, int* running, int64_t* rounds,
                        int64_t* merges, int64_t* sigma_evals) {
  return guard([&] { pnoeom::server_stats(srv, used_bytes, queued, running, rounds, merges, sigma_evals); });
}

int pno_get_eigenvectors(const pnoeom_pno* pno, double* X) {
  return guard([&] {
    PN_CHECK(pno && X, PNOEOM_ERR_INVALID_ARG, "NULL argument");
    std::copy(pno->last_X.begin(), pno->last_X.end(), X);
  });
}

int pno_solve_lowprec_energies(const pnoeom_pno* pno, int phase, int n, double* energies, int* count) {
  return guard([&] {
    PN_CHECK(pno && (n <= 0 || energies), PNOEOM_ERR_INVALID_ARG, "NULL argument");
    PN_CHECK(phase == PNOEOM_BF16 || phase == PNOEOM_FP32, PNOEOM_ERR_INVALID_ARG, "phase must be PNOEOM_BF16 or PNOEOM_FP32");
    const std::vector<double>& w = pno->last_phase_w[phase == PNOEOM_BF16 ? 0 : 1];
    const int c = (int)w.size();
    if (count) *count = c;
    for (int k = 0; k < std::min(n, c); ++k) energies[k] = w[k];
  });
}

int pno_solve_stats(const pnoeom_pno* pno, int64_t* sigma_evals_fp32, int64_t* sigma_evals_fp64) {
  return guard([&] {
    PN_CHECK(pno, PNOEOM_ERR_INVALID_ARG, "NULL handle");
    if (sigma_evals_fp32) *sigma_evals_fp32 = pno->last_sigma_evals[0];
    if (sigma_evals_fp64) *sigma_evals_fp64 = pno->last_sigma_evals[1];
  });
}

int pno_get_occupations(const pnoeom_pno* pno, double* occ) {
  return guard([&] {
    PN_CHECK(pno && occ, PNOEOM_ERR_INVALID_ARG, "NULL argument");
    std::copy(pno->occupations.begin(), pno->occupations.end(), occ);
  });
}

int pno_get_cis_vectors(const pnoeom_pno* pno, double* b) {
  return guard([&] {
    PN_CHECK(pno && b, PNOEOM_ERR_INVALID_ARG, "NULL argument");
    std::copy(pno->cis_b.begin(), pno->cis_b.end(), b);
  });
}

int pno_get_cis(const pnoeom_pno* pno, double* omega) {
  return guard([&] {
    PN_CHECK(pno && omega, PNOEOM_ERR_INVALID_ARG, "NULL argument");
    std::copy(pno->cis_omega.begin(), pno->cis_omega.end(), omega);
  });
}

int pnoeom_gemm_tf32x3(pnoeom_ctx* ctx, const float* A, const float* B, float* C, int M, int N, int K, float alpha,
                       void* cuda_stream) {
  return guard([&] {
    PN_CHECK(ctx, PNOEOM_ERR_INVALID_ARG, "NULL context");
    pnoeom::DeviceScope dev_scope(ctx->device);
    pnoeom::gemm_tf32x3(A, B, C, M, N, K, alpha, st(cuda_stream));
  });
}

int pnoeom_device_status(pnoeom_ctx* ctx, int clear, int* status) {
  return guard([&] {
    PN_CHECK(ctx && status, PNOEOM_ERR_INVALID_ARG, "NULL argument");
    pnoeom::DeviceScope dev_scope(ctx->device);
    PN_CUDA(cudaDeviceSynchronize());
    *status = pnoeom::device_status(clear != 0, nullptr);
  });
}

int pnoeom_inject_alloc_failure(long long after) {
  return guard([&] { pnoeom::inject_alloc_failure(after); });
}

int pnoeom_alloc_live_bytes(long long* bytes) {
  return guard([&] {
    PN_CHECK(bytes, PNOEOM_ERR_INVALID_ARG, "NULL argument");
    *bytes = pnoeom::live_alloc_bytes();
  });
}

int pnoeom_selftest_bounded_wait(pnoeom_ctx* ctx, long long budget_cycles, void* cuda_stream, int* timed_out) {
  return guard([&] {
    PN_CHECK(ctx && timed_out, PNOEOM_ERR_INVALID_ARG, "NULL argument");
    PN_CHECK(budget_cycles >= 1 && budget_cycles <= 2000000000LL, PNOEOM_ERR_INVALID_ARG,
             "budget_cycles must be in 1 .. 2e9");
    pnoeom::DeviceScope dev_scope(ctx->device);
    *timed_out = pnoeom::selftest_bounded_wait(budget_cycles, st(cuda_stream));
  });
}

int pnoeom_small_eig(int n, const double* A, double* wr, double* wi, double* VR) {
  return guard([&] {
    PN_CHECK(n >= 1 && A && wr && wi && VR, PNOEOM_ERR_INVALID_ARG, "bad arguments");
    PN_CHECK(pnoeom::small_eig(n, A, wr, wi, VR) == 0, PNOEOM_ERR_NOT_CONVERGED, "QR iteration did not converge");
  });
}

}  // extern "C"
