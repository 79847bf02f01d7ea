/*
 * pnoeom.h -- C ABI of the GB300 state-averaged PNO-EOM-CCSD engine.
 *
 * What the library computes (Peng, Clement, Valeev, arXiv:1802.06738):
 *   * the closed-shell EOM-CCSD eigenproblem  Hbar R|0> = E R|0>,
 *     Hbar = exp(-T) H exp(T), R = R1 + R2 (Sec. 2, the EOM paragraph);
 *   * with R2 stored per occupied pair ij in the pair's state-averaged PNO
 *     space and R1 per occupied i in its OSV space (Sec. 2, Eq. eom:sa_density
 *     and the OSV definition that follows it);
 *   * PNOs are eigenvectors of the CIS(D) pair densities (Eq. cis_d and the
 *     pair-density formula after it) averaged over the N target states,
 *     truncated at T_CutPNO; OSVs are those of the diagonal pairs truncated at
 *     T_CutOSV (default T_CutPNO / 10, Sec. 3);
 *   * eigenvalues are found by a Davidson solver whose residuals are
 *     preconditioned in the semicanonical PNO/OSV bases (Sec. 2, the
 *     PNO-EOM-CCSD Davidson steps 1-4).
 *
 * Conventions
 *   * Orbitals p = 0..o-1 occupied, o..o+v-1 virtual, canonical RHF (Fock
 *     diagonal = eps).  Two-electron integrals enter only through
 *     density-fitting factors B[Q][p][q], (pq|rs) = sum_Q B[Q][p][q] B[Q][r][s]
 *     (Sec. 3: density fitting is used for all calculations).
 *   * Amplitudes: t1[i][a] = t^i_a, t2[i][j][a][b] = t^{ij}_{ab} (row-major,
 *     t2[i][j][a][b] = t2[j][i][b][a]).  T2 = 1/2 t^{ij}_{ab} E^a_i E^b_j.
 *   * Packed PNO vector (one root): [R1: i = 0..o-1, n_i entries each]
 *     [R2: pairs i <= j in lexicographic order, n_ij x n_ij row-major, the row
 *     index in the ij PNO space belonging to orbital i].  Offsets come from
 *     pno_query().  A batch of nvec vectors is nvec such vectors back to back.
 *   * PNO/OSV sign convention: every kept semicanonical vector has its entry
 *     of largest magnitude (the first, on ties) positive.
 *
 * Errors: every int-returning call returns PNOEOM_OK (0) or a negative code;
 * pnoeom_last_error() gives a message for the calling thread.  No call
 * aborts the process.  Ownership: inputs are caller-owned and copied in;
 * handles are library-owned until the matching *_destroy.
 */
#ifndef PNOEOM_H
#define PNOEOM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PNOEOM_OK = 0,
  PNOEOM_ERR_INVALID_ARG = -1,
  PNOEOM_ERR_NOMEM = -2,          /* device allocation failed or footprint over budget */
  PNOEOM_ERR_CUDA = -3,           /* a CUDA / cuSOLVER call failed */
  PNOEOM_ERR_NOT_CONVERGED = -4,  /* Davidson hit max_iter; best values returned */
  PNOEOM_ERR_TIMEOUT = -5,        /* a bounded device wait expired */
  PNOEOM_ERR_UNSUPPORTED = -6
};

enum { PNOEOM_HOST = 0, PNOEOM_DEVICE = 1 };            /* memory space of pointers */
/* sigma precision (BASELINE precision policy of the mixed path, Sec. 2 sigma with the
 * contractions in reduced precision and FP32 accumulation):
 *   PNOEOM_FP64: FP64 vectors, operator blocks and arithmetic;
 *   PNOEOM_FP32: FP32 vectors and operator blocks, FP32 arithmetic (the E3 GEMM tiles on
 *     the tensor cores in 3xTF32);
 *   PNOEOM_BF16: as FP32, but the dense pair blocks (the 4-virtual and T2 ladders with the
 *     virtual Fock term, D_p; the singles couplings A_DS and A_S; the occupied global
 *     blocks) are read from a BF16 copy (rounded to nearest) and multiplied in FP32 with
 *     FP32 accumulation.  Vectors passed to sigma are float, as for PNOEOM_FP32. */
enum { PNOEOM_FP64 = 0, PNOEOM_FP32 = 1, PNOEOM_BF16 = 2 };

typedef struct pnoeom_ctx pnoeom_ctx;
typedef struct pnoeom_pno pnoeom_pno;

/* One closed-shell system.  eps: float64[o+v]; B: float64[naux][o+v][o+v];
 * t1: float64[o][v] or NULL (T1 = 0); t2: float64[o][o][v][v] or NULL, in
 * which case the first-order amplitudes of Eq. T1 are used,
 * t^{ij}_{ab} = (ai|bj) / (eps_i + eps_j - eps_a - eps_b).
 * mem_space says whether the pointers are host or device memory. */
typedef struct {
  int o, v, naux;
  const double* eps;
  const double* B;
  const double* t1;
  const double* t2;
  int mem_space;
} pnoeom_system;

/* t_pno: T_CutPNO (occupations >= t_pno kept; 0 keeps the full virtual space);
 * t_osv: T_CutOSV, < 0 means t_pno / 10 (Sec. 3).  nroots_sa: N of the state
 * average (Eq. eom:sa_density); nroots_solve: roots returned by the solver
 * (<= nroots_sa).  precision: PNOEOM_FP64, PNOEOM_FP32 or PNOEOM_BF16 sigma;
 * refine_fp64: the low-precision phase aims at res_tol and hands over to the next
 * precision (BF16 -> FP32 -> FP64 for PNOEOM_BF16, FP32 -> FP64 for PNOEOM_FP32) when that
 * holds, when its largest residual (below 1e-1 in BF16, 1e-4 in FP32) stops halving
 * within three iterations, or when no new direction survives; each phase restarts from
 * the N Ritz vectors of the last, and the FP64 phase runs until the FP64 tolerances
 * hold.  res_tol: residual 2-norm per root; e_tol: eigenvalue
 * change between iterations; max_subspace <= 0 means 8 * nroots_solve.
 * state_specific: 0 (the default, and the paper's method) builds state-averaged
 * PNOs/OSVs; k in 1..nroots_sa builds them from the CIS(D) pair densities of CIS
 * root k alone (1-based), the state-specific construction the paper compares
 * against (Sec. 2: one PNO space per state); the Davidson solve is unchanged, so
 * root k is energies[k - 1] with nroots_solve >= k.
 * t_pno_gs: 0 (default) leaves the ground-state amplitudes as given; > 0 truncates
 * them to ground-state PNOs: each T^{ij} is projected onto the eigenvectors of its
 * pair density D_(0)^{ij} = 2/(1+delta_ij) (T T~^T + T^T T~), T~ = 2T - T^T, with
 * occupation >= t_pno_gs (Methods, ground-state PNOs from the guess amplitudes).
 * Only T2 is truncated (T1 and a PNO-CCSD re-solution in the truncated spaces are
 * not), which is exact for the MP1 amplitudes used when t2 is NULL. */
typedef struct {
  double t_pno, t_osv;
  int nroots_sa, nroots_solve;
  int precision;
  int refine_fp64;
  int max_iter, max_subspace;
  double res_tol, e_tol;
  int state_specific;
  double t_pno_gs;
} pnoeom_opts;

/* Create a context on CUDA device `device`.  hbm_budget_bytes = 0 means no
 * budget; otherwise pno_build refuses (PNOEOM_ERR_NOMEM) a system whose
 * estimated footprint exceeds it. */
int pnoeom_create(pnoeom_ctx** ctx, int device, size_t hbm_budget_bytes);
/* Frees the context (NULL: no-op).  Handles built on it are destroyed first. */
void pnoeom_destroy(pnoeom_ctx* ctx);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* pnoeom_last_error(void);

/* Setup (Sec. 2): dress the Hamiltonian with T1 (if any), form T2 (Eq. T1 if
 * not supplied), CIS roots, CIS(D) doubles and state-averaged pair densities,
 * PNO/OSV eigendecompositions with truncation and semicanonicalisation, and
 * the R-independent PNO-space operator blocks sigma needs.  Runs on
 * `cuda_stream` (NULL = default stream) and returns when done.  Inputs are
 * copied; *out owns all device state. */
int pno_build(pnoeom_ctx* ctx, const pnoeom_system* sys, const pnoeom_opts* opts,
              void* cuda_stream, pnoeom_pno** out);
/* Frees the handle and its device memory (NULL: no-op).  Work issued on it must
 * have completed, and batches that reference it are destroyed first. */
void pno_destroy(pnoeom_pno* pno);

/* Sizes of the packed PNO vector.  Arrays stay valid until pno_destroy.
 * n_ij has npairs = o(o+1)/2 entries, n_i has o entries. */
int pno_query(const pnoeom_pno* pno, int* npairs, const int** n_ij, const int** n_i,
              size_t* vec_len, size_t* footprint_bytes);

/* PNO bases on the host: U (float64[v][n_ij], row-major) of pair p (i <= j,
 * lexicographic index), or of OSV set i when pair < 0 (index -pair-1).  The
 * caller provides v * n doubles.  fbar (n doubles, may be NULL) receives the
 * semicanonical orbital energies. */
int pno_get_basis(const pnoeom_pno* pno, int pair, double* U, double* fbar);

/* sigma = Hbar R projected into the PNO/OSV spaces (Sec. 2) for nvec packed
 * vectors.  r_dev, s_dev: caller-owned device buffers of nvec * vec_len
 * elements: double for PNOEOM_FP64, float for PNOEOM_FP32 and PNOEOM_BF16.
 * Asynchronous on cuda_stream.  Calls on one handle share its scratch (the
 * R-dependent intermediates, grown when a call needs more vectors than any
 * before it): issue them on one stream, or synchronise between calls on
 * different streams.  Calls on different handles may overlap.  In FP32 some terms run
 * on the tensor cores, whose bounded waits do not raise an error here: the result is
 * valid only if pnoeom_device_status reads 0 once the stream has been synchronised
 * (davidson_solve checks this itself).  The call makes ctx's device current for its
 * duration and restores the caller's current device before returning. */
int sigma(pnoeom_ctx* ctx, const pnoeom_pno* pno, int nvec, const void* r_dev, void* s_dev,
          int precision, void* cuda_stream);

/* sigma without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory
 * while they run, such as a serving loop whose latency budget cannot absorb
 * the device-wide synchronisation cudaMalloc/cudaFree imply, or an
 * application that has handed all device memory to its own pool allocator.
 * It computes exactly what sigma() computes, but its scratch memory (the
 * R-dependent intermediates, nvec * (v*v + o*o + 2*v*sum_ij n_ij) elements:
 * FvR, FoR and the two E3 factors Y and Z) lives in a
 * file-scope device array of PNOEOM_NOALLOC_SCRATCH_BYTES bytes that every
 * GPU which loads the library keeps until the process exits.  Calls needing
 * more scratch than that return PNOEOM_ERR_UNSUPPORTED without launching
 * anything.  The first call on a device looks up the array's device address
 * (once per device, with that device current); make that first call before
 * any stream capture.  The array is shared by all calls and keeps the last
 * call's contents (each call clears what it needs): calls whose executions
 * overlap on the GPU race on it, so issue them on one stream or otherwise
 * serialise them.  No cudaMalloc, cudaFree or allocating library routine is
 * called.  Arguments, layouts and errors are those of sigma(), including the check of
 * pnoeom_device_status that an FP32 result needs before it is trusted. */
#define PNOEOM_NOALLOC_SCRATCH_BYTES (64u << 20)
int sigma_noalloc(pnoeom_ctx* ctx, const pnoeom_pno* pno, int nvec, const void* r_dev, void* s_dev,
                  int precision, void* cuda_stream);

/* Davidson solve (Sec. 2, PNO-EOM-CCSD Davidson): projected CIS guesses,
 * semicanonical preconditioner omega + f_ii (+ f_jj) - fbar_a (- fbar_b),
 * FP64 orthogonalisation and subspace diagonalisation.  energies and
 * res_norms: host arrays of nroots_solve doubles; iters: host int.  Blocking.
 * Returns PNOEOM_ERR_NOT_CONVERGED with the best values after max_iter, and
 * PNOEOM_ERR_TIMEOUT when a tensor-core kernel's bounded wait ran out during the
 * solve (see pnoeom_device_status; the results are then invalid). */
int davidson_solve(pnoeom_ctx* ctx, pnoeom_pno* pno, const pnoeom_opts* opts, void* cuda_stream,
                   double* energies, double* res_norms, int* iters);

/* Batches (many systems in one launch sequence).  A batch references n built
 * systems (1 <= n <= 128, still owned by the caller, who must keep them alive
 * and destroy the batch first).  pnoeom_batch_create merges their sigma
 * programs: every pair block of every system is one problem of the same
 * kernels, so each sigma of the batch is one launch sequence, replayed as a
 * CUDA graph on non-default streams.  The merged program's tile choices are
 * autotuned at creation. */
typedef struct pnoeom_batch pnoeom_batch;
int pnoeom_batch_create(pnoeom_ctx* ctx, pnoeom_pno* const* members, int n, void* cuda_stream, pnoeom_batch** out);
void pnoeom_batch_destroy(pnoeom_batch* batch);

/* sigma for every member at once: nvec[k] packed vectors of member k at
 * r_dev[k] (member k's vec_len each) into s_dev[k]; nvec[k] = 0 skips member k.
 * Precision and layouts as in sigma().  Asynchronous on cuda_stream. */
int pnoeom_batch_sigma(pnoeom_ctx* ctx, pnoeom_batch* batch, const int* nvec, const void* const* r_dev,
                       void* const* s_dev, int precision, void* cuda_stream);

/* Davidson solves of all members in lockstep (each member its own subspace;
 * every round evaluates all members' pending vectors in one sigma launch).
 * Host outputs: energies and res_norms n x nroots_solve, iters and converged n.
 * Returns PNOEOM_ERR_NOT_CONVERGED if any member did not converge, and
 * PNOEOM_ERR_TIMEOUT when a tensor-core kernel's bounded wait ran out (see
 * pnoeom_device_status; the results are then invalid). */
int pnoeom_batch_solve(pnoeom_ctx* ctx, pnoeom_batch* batch, const pnoeom_opts* opts, void* cuda_stream,
                       double* energies, double* res_norms, int* iters, int* converged);

/* Serving (continuous batching of excited-state solves).  A server owns
 * builder threads (3 by default; the environment variable
 * PNOEOM_SERVER_BUILDERS, read at creation, sets 1..16) that admit queued
 * requests in arrival order when their estimated setup footprint fits the
 * HBM budget (0 = no budget) and run pno_build concurrently, each on its own
 * stream and cuSOLVER handle, and a solver thread that keeps every built request's
 * PNOs, operator blocks and Davidson subspace resident and runs lockstep
 * Davidson rounds over all of them through one merged sigma program (a CUDA
 * graph).  Requests that finish building join at the next round boundary;
 * finished ones leave and free their memory, so requests that arrive while
 * others run overlap with them on the device.  At most max_active requests
 * are solved together. */
typedef struct pnoeom_server pnoeom_server;
enum { PNOEOM_REQ_QUEUED = 0, PNOEOM_REQ_BUILDING = 1, PNOEOM_REQ_RUNNING = 2, PNOEOM_REQ_DONE = 3,
       PNOEOM_REQ_FAILED = 4 };
int pnoeom_server_create(pnoeom_ctx* ctx, size_t hbm_budget_bytes, int max_active, pnoeom_server** out);
/* Stops the server's threads (queued requests are not run) and frees all state. */
void pnoeom_server_destroy(pnoeom_server* srv);
/* Queue one solve.  Inputs must be host memory; they are copied.  A request
 * whose estimated footprint exceeds the budget fails at once with
 * PNOEOM_ERR_NOMEM (visible through poll). */
int pnoeom_server_submit(pnoeom_server* srv, const pnoeom_system* sys, const pnoeom_opts* opts, int64_t* id);
/* Non-blocking status of request `id`; when DONE, energies and res_norms
 * (nroots_solve each), iters and sigma_evals are filled (any may be NULL).
 * times (4 doubles, may be NULL): submitted, admitted, built, finished, in
 * seconds since the server started (0 when not reached). */
int pnoeom_server_poll(pnoeom_server* srv, int64_t id, int* status, double* energies, double* res_norms,
                       int* iters, int64_t* sigma_evals, double* times);
/* Block until request `id` is DONE or FAILED, or timeout_s elapses
 * (PNOEOM_ERR_TIMEOUT).  PNOEOM_ERR_CUDA if the server stopped before the
 * request finished (a worker thread could not get its stream or solver handle;
 * submit then fails the same way). */
int pnoeom_server_wait(pnoeom_server* srv, int64_t id, double timeout_s);
/* Counters: device bytes held for admitted requests, queued / building-or-built
 * / running requests, lockstep rounds, program merges, sigma-evals done. */
int pnoeom_server_stats(pnoeom_server* srv, size_t* used_bytes, int* queued, int* running, int64_t* rounds,
                        int64_t* merges, int64_t* sigma_evals);

/* Eigenvectors of the last davidson_solve on this handle, as packed FP64
 * vectors on the host (nroots_solve * vec_len doubles). */
int pno_get_eigenvectors(const pnoeom_pno* pno, double* X);

/* Ritz values of the last davidson_solve on this handle at the moment one of its
 * low-precision phases handed over (refine_fp64 set): phase = PNOEOM_BF16, when the BF16
 * phase of a PNOEOM_BF16 solve handed over to its FP32 phase; PNOEOM_FP32, when the FP32
 * phase (of a PNOEOM_FP32 solve, or the second phase of a PNOEOM_BF16 one) handed over to
 * the FP64 refinement.  These are the unrefined energies of that precision, ascending.
 * Writes min(n, count) doubles and the number available in *count (0 when the last solve
 * had no such phase).  Host-only. */
int pno_solve_lowprec_energies(const pnoeom_pno* pno, int phase, int n, double* energies, int* count);

/* Sigma evaluations (one vector of one root each) of the last davidson_solve on
 * this handle, split by the precision they ran in: FP32 (the mixed phase) and
 * FP64 (a plain FP64 solve, or the refinement that follows the FP32 phase).
 * Both 0 before the first solve.  Host-only; either pointer may be NULL. */
int pno_solve_stats(const pnoeom_pno* pno, int64_t* sigma_evals_fp32, int64_t* sigma_evals_fp64);

/* All eigenvalues (ascending) of every state-averaged pair density D^{ij}
 * (Eq. eom:sa_density): npairs x v doubles on the host, pair-major.  The PNO
 * occupation numbers whose truncation at T_CutPNO defines n_ij. */
int pno_get_occupations(const pnoeom_pno* pno, double* occ);

/* CIS singles amplitudes b^i_a(k) (Sec. 2, CIS(D) paragraph), nroots_sa x o x v
 * doubles on the host, normalised so that R1|0> is a unit vector
 * (2 sum b^2 = 1), largest-magnitude entry positive. */
int pno_get_cis_vectors(const pnoeom_pno* pno, double* b);

/* The nroots_sa lowest singlet CIS excitation energies omega_k (Eh, ascending;
 * Sec. 2, CIS(D) paragraph) whose doubles define the state average, as doubles on
 * the host. */
int pno_get_cis(const pnoeom_pno* pno, double* omega);

/* Dense FP32 product on the tensor cores: C (M x N) += alpha * A (M x K) * B (K x N),
 * row-major device buffers (leading dimensions K, N, N).  It runs the tile kernel the
 * sigma program uses for its dense GEMM tiles (FvR = -U_cat Y and Z = FvR^T U_cat of the
 * E3 term, Sec. 2): tcgen05 kind::tf32 MMAs with each operand split into a tf32 high
 * part and a tf32 remainder, hi*hi + hi*lo + lo*hi accumulated in FP32 in tensor memory,
 * which keeps about 21 bits of every product.  Exported so that kernel can be tested on
 * its own.  Blocks until done on cuda_stream.  Returns PNOEOM_ERR_INVALID_ARG for
 * negative sizes or NULL buffers with nonzero sizes. */
int pnoeom_gemm_tf32x3(pnoeom_ctx* ctx, const float* A, const float* B, float* C, int M, int N, int K, float alpha,
                       void* cuda_stream);

/* Status word of the tensor-core kernels on the context's device: 0 when every bounded
 * wait of those kernels completed; bit 0 set when an mbarrier wait ran past its clock
 * budget (about one second), in which case that tile's contribution was skipped and its
 * result is invalid.  clear != 0 resets the word.  Synchronises the device. */
int pnoeom_device_status(pnoeom_ctx* ctx, int clear, int* status);

/* Failure detection without a GPU fault.  pnoeom_selftest_bounded_wait launches one
 * CTA that waits on an mbarrier nothing ever arrives at, for at most budget_cycles
 * clock cycles (1 .. 2e9, about one second at most), and records the expiry exactly as
 * a tensor-core kernel does: bit 0 of the status word (pnoeom_device_status), so the
 * next davidson_solve or pnoeom_batch_solve returns PNOEOM_ERR_TIMEOUT and clears it.
 * *timed_out receives 1 when the wait ran out (it always should).  Blocking. */
int pnoeom_selftest_bounded_wait(pnoeom_ctx* ctx, long long budget_cycles, void* cuda_stream, int* timed_out);

/* Host-side fault injection in the library's caching device allocator: after `after`
 * further successful allocation requests (0: the very next one) one request fails as
 * if the device were out of memory, so the call making it returns PNOEOM_ERR_NOMEM;
 * a negative value disables the injection.  Process-wide.  pnoeom_alloc_live_bytes
 * reports the bytes of allocator blocks currently held by live objects (handles,
 * batches, scratch), which returns to its earlier value when a failed call has
 * released everything it took. */
int pnoeom_inject_alloc_failure(long long after);
int pnoeom_alloc_live_bytes(long long* bytes);

/* Peak rates of the context's device, measured by the library's own microbenchmarks
 * (the denominators of roofline fractions; no device setting is changed).  Writes up to
 * nout doubles: [0] FP32 FMA TFLOP/s (SIMT), [1] FP64 FMA TFLOP/s (SIMT), [2] tcgen05
 * kind::f16 BF16 MMA TFLOP/s, [3] tcgen05 kind::tf32 MMA TFLOP/s (both 128 x 256 tiles,
 * FP32 accumulation in tensor memory, one CTA per SM), [4] cuBLAS DGEMM TFLOP/s
 * (n = 4096), [5] cuBLAS DGEMM with the fixed-point FP64 emulation math mode (0 when
 * unavailable), [6] the largest |emulated - native| / max |native| of that product,
 * [7] the SM count.  Each rate is the best of a few CUDA-event-timed launches on
 * cuda_stream.  Blocking; takes a few seconds and about 0.5 GB of device memory. */
int pnoeom_measure_peaks(pnoeom_ctx* ctx, void* cuda_stream, double* out, int nout);

/* Eigenpairs of a small dense non-symmetric matrix on the host (the Davidson
 * subspace step, Sec. 2).  A: row-major n x n; wr, wi: real and imaginary
 * parts of the eigenvalues (unsorted); VR[i*n + k]: component i of the right
 * eigenvector of eigenvalue k, rotated so its largest component is real,
 * real part kept, unit 2-norm.  Host memory only, no GPU needed.  Returns 0,
 * PNOEOM_ERR_INVALID_ARG, or PNOEOM_ERR_NOT_CONVERGED. */
int pnoeom_small_eig(int n, const double* A, double* wr, double* wi, double* VR);

/* Tracing of sigma.  pno_set_timing(pno, 1) clears the counters and makes
 * every later sigma call on this handle record CUDA events, on the stream it
 * launches on, around each of its kernels; 0 stops recording.
 * pno_sigma_timing reports, for kernel class `k` (0: sandwich products
 * into the R-dependent intermediates, 1: dense GEMV blocks into those
 * intermediates, 2: sandwich products into sigma, 3: dense GEMV blocks into
 * sigma, 4: GEMM tiles into the intermediates (FvR), 5: GEMM tiles of the
 * E3 term (Z = FvR^T U_cat and its products into sigma)), the number of kernel launches recorded, their summed device time
 * in ms, the algorithmic bytes one sigma call's launches of that class move
 * for nvec vectors (operator blocks
 * read once, vector blocks read and written once per vector, at the element
 * size of `precision`: 8 bytes for PNOEOM_FP64, 4 otherwise, and 2 in PNOEOM_BF16 for
 * the dense GEMV blocks, classes 1 and 3, and the tensor-core operator images of class 2)
 * and their flops.  Any pointer may be NULL.  Blocks
 * until the recorded events complete. */
int pno_set_timing(pnoeom_pno* pno, int enable);
int pno_sigma_timing(const pnoeom_pno* pno, int k, int nvec, int precision, const char** name, int* launches,
                     double* ms, double* bytes, double* flops);

/* Executed tensor-core work of the BF16 sigma's sandwich terms (Sec. 2 ring, Fock and
 * occupied-ladder terms on the tcgen05 path), per vector: 2 M N K summed over every MMA
 * the kernel issues, padding included (bins of 128 rows, K rounded up to 16, both X and
 * X^T in the first product, the whole bin width in the second).  Set by pno_build; 0 when
 * the system has no term on that path.  Compare with the algorithmic flops of class 2 of
 * pno_sigma_timing.  per_vector: host double.  Errors: PNOEOM_ERR_INVALID_ARG for NULL. */
int pno_tc_mma_flops(const pnoeom_pno* pno, double* per_vector);

/* Autotuner record: pno_build times every launch of the output-grouped
 * small-block kernel (one per size bucket and phase) for every candidate
 * (group size x vectors per CTA) on nroots_sa FP32 vectors, and each launch
 * keeps its own fastest candidate.  Writes up to `ncand` candidates (group
 * size, vectors per CTA, summed ms of all those launches under that
 * candidate) and in *choice the index of the candidate with the smallest
 * sum.  Any pointer may be NULL. */
int pno_autotune_info(const pnoeom_pno* pno, int ncand, int* group_sizes, int* roots_per_cta, double* ms, int* choice);

/* Seconds spent in the last pno_build of this handle (setup time). */
double pno_build_seconds(const pnoeom_pno* pno);

#ifdef __cplusplus
}
#endif
#endif
