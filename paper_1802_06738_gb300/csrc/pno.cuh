// Handle state of one built system (pnoeom_pno) and internal entry points.
#pragma once
#include <unordered_map>
#include "common.cuh"
#include "engine.cuh"
#include "sigma_prog.cuh"
#include <cuda_bf16.h>
#include <functional>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

namespace pnoeom {
constexpr int NGROUP_CAND = 5;
constexpr int GROUP_CAND[NGROUP_CAND] = {2, 4, 8, 16, 32};
constexpr int NRPC_CAND = 6;
constexpr int RPC_CAND[NRPC_CAND] = {1, 2, 3, 4, 6, 8};
constexpr int NTUNE = NGROUP_CAND * NRPC_CAND;

// Small sandwich problems of one size bucket: ordered by output block, with one
// group-boundary list per candidate group size.
struct SmallSet {
  DBuf<SProb> probs;
  DBuf<int> starts[NGROUP_CAND];
  int ngroups[NGROUP_CAND] = {0};
  int dims[4] = {1, 1, 1, 1};   // max M, K1, K2, N
  int nprob = 0;
  int gchoice = 2, rchoice = NRPC_CAND - 1;       // tuned (group size, vectors per CTA) of this set
  bool ab = false;                                 // every problem has A and B (batched variant possible)
  int pb = 1;                                      // problems staged together (tuned; 1 unless ab)
  int nb = 0;                                      // stage buffers of the unbatched kernel (tuned; 0 = by occupancy)
  int shape = 0;                                   // CTA shape of the unbatched kernel (tuned; 0 = by bucket)
  double tune_ms[NTUNE] = {0};
  std::vector<SProb> h_probs;                      // host copies (batch merging)
  std::vector<int> h_starts[NGROUP_CAND];
};

// A launchable sigma program: the problem lists of one system, or of a batch
// of systems (problems carry their system index).
struct Program {
  DBuf<SProb> gen1, gen2;          // generic sandwich problems (phase 1: intermediates, phase 2: sigma)
  DBuf<VProb> v1, v2;              // dense GEMV tiles
  DBuf<DProb> d1, d2, d3;          // dense GEMM tiles: FvR (phase 1), Z, E3 products (phase 2)
  int n_gen1 = 0, n_gen2 = 0, n_v1 = 0, n_v2 = 0, n_d1 = 0, n_d2 = 0, n_d3 = 0;
  SmallSet small1[3], small2[3];   // small sandwich problems per size bucket
  int smem_elems = 1;
  int group_choice = 2, rpc_choice = NRPC_CAND - 1;   // fastest single candidate for every set (reported)
  // tensor-core sandwich path of the BF16 sigma (single-system calls): jobs, rounds,
  // sub-terms, copies, X blocks; gen2x: the phase-2 problems it does not cover (dims
  // above TCS_MAXN), run by the generic kernel alongside it
  DBuf<TcsJob> tcs_jobs; DBuf<TcsSlot> tcs_slots; DBuf<TcsRec> tcs_recs;
  DBuf<int64_t> tcs_xblk;
  int n_tcs_jobs = 0, n_tcs_xblk = 0;
  int64_t tcs_xstride = 0;         // elements of one vector's X images
  double tcs_mma_flops = 0;        // flops of every MMA k_sandwich_tc issues for one vector (2 M N K)
  DBuf<SProb> gen2x;
  int n_gen2x = 0;
  std::vector<SProb> h_gen2x;
  std::vector<SProb> h_gen1, h_gen2;
  // the two whole E3 products (FvR = -U_cat Y, Z = FvR^T U_cat) as untiled problems: in the
  // single-precision sigma of a single system they run as strided-batched library GEMMs
  std::vector<DProb> h_gfull;
  std::vector<VProb> h_v1, h_v2;
  std::vector<DProb> h_d1, h_d2, h_d3;
  void upload(cudaStream_t s, size_t* fp);
};
}  // namespace pnoeom

struct pnoeom_pno {
  ~pnoeom_pno() {
    for (auto& e : events) { cudaEventDestroy(e.second.first); cudaEventDestroy(e.second.second); }
  }
  int o = 0, v = 0, naux = 0, nroots_sa = 0;
  double t_pno = 0, t_osv = 0;
  bool has_t1 = false;
  int npairs = 0;
  std::vector<int> nij, ni;                  // PNOs per stored pair (i <= j), OSVs per occupied
  std::vector<int> pair_i, pair_j;
  std::vector<std::vector<int>> pidx;        // pidx[i][j] = stored pair index of {i, j}
  std::vector<int64_t> off_i, off_ij;        // packed-vector offsets
  int64_t L1 = 0, L = 0;
  std::vector<double> eps;                   // host copy
  // bases (FP64 device): pairs then OSVs, each v x n row-major; semicanonical energies
  pnoeom::DBuf<double> U, fbar;
  std::vector<int64_t> Uoff_pair, Uoff_osv, foff_pair, foff_osv;
  // sigma program
  pnoeom::DBuf<double> pool64;
  pnoeom::DBuf<float> pool32;
  pnoeom::DBuf<__nv_bfloat16> pool16;          // BF16 copy (dense GEMV blocks of the BF16 sigma)
  pnoeom::DBuf<__nv_bfloat16> tcimg;           // BF16 operand images of the tensor-core sandwich path
  pnoeom::DBuf<__nv_bfloat16> ximg;            // per-call X images (nvec x prog.tcs_xstride)
  pnoeom::Program prog;
  double tune_ms[pnoeom::NTUNE] = {0};
  static constexpr int NCLS = 6;             // kernel classes of the sigma program (timing)
  int prof_launches[NCLS] = {0};
  int smem_elems = 0;
  int64_t work_len = 0;                      // FvR (v*v) + FoR (o*o) + Y + Z (2 v sum n_p)
  int64_t work_fvr = 0, work_for = 0, work_y = 0, work_z = 0;
  // Davidson data
  pnoeom::DBuf<double> denom_base;           // f_ii (+ f_jj) - fbar_a (- fbar_b), packed
  pnoeom::DBuf<double> guesses;              // projected CIS vectors, nroots_sa x L
  std::vector<double> cis_omega, cis_b;
  std::vector<double> occupations;           // npairs x v eigenvalues of D^{ij}
  std::vector<double> last_X;
  int last_nroots = 0;
  int64_t last_sigma_evals[2] = {0, 0};   // FP32 / FP64 sigma evaluations of the last solve
  std::vector<double> last_phase_w[2];    // Ritz values when the BF16 / FP32 phase of the last mixed solve handed over
  // per-call scratch kept across calls
  pnoeom::DBuf<double> work64; pnoeom::DBuf<float> work32;
  // tracing: per kernel class, operator elements read once per launch,
  // vector elements read+written per vector, flops per vector
  double prof_pool_elems[NCLS] = {0}, prof_vec_elems[NCLS] = {0}, prof_flops[NCLS] = {0};
  bool timing = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> events;
  size_t footprint = 0;
  double build_seconds = 0;
};

// A batch of built systems evaluated together: one merged sigma program whose
// problems carry their member index (a11 of the hot path: all pairs of all
// systems in one launch sequence, replayed as a CUDA graph).
struct pnoeom_batch {
  int device = 0;
  std::vector<pnoeom_pno*> members;
  pnoeom::Program prog;
  std::vector<pnoeom::DBuf<double>> w64;
  std::vector<pnoeom::DBuf<float>> w32;
  cudaGraphExec_t exec = nullptr;
  bool use_graph = true;
  int graph_launches = 0, graph_updates = 0, graph_instantiations = 0;
  double tune_ms[pnoeom::NTUNE] = {0};
  size_t footprint = 0;
  ~pnoeom_batch() { if (exec) cudaGraphExecDestroy(exec); }
};

namespace pnoeom { struct Request; }
struct pnoeom_server {
  int device = 0;
  size_t budget = 0;
  int max_active = 0;
  double t0 = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::map<int64_t, std::shared_ptr<pnoeom::Request>> reqs;
  std::deque<std::shared_ptr<pnoeom::Request>> queued, built;
  size_t used = 0;          // estimated or measured device bytes of admitted requests
  int64_t next_id = 1;
  bool stop = false;
  int64_t rounds = 0, merges = 0, total_sigma_evals = 0;
  std::vector<std::thread> builders;   // concurrent pno_build workers, one stream and solver handle each
  std::thread solver;
  std::string fatal;
};

namespace pnoeom {
void autotune(pnoeom_pno* P, cudaStream_t s);
void batch_build(pnoeom_batch* B, cudaStream_t s);
void batch_merge(pnoeom_batch* B, cudaStream_t s, bool tune);
int guard_call(const std::function<void()>& f);
void server_start(pnoeom_server* S);
void server_stop(pnoeom_server* S);
int64_t server_submit(pnoeom_server* S, const pnoeom_system* sys, const pnoeom_opts* opts);
void server_poll(pnoeom_server* srv, int64_t id, int* status, double* energies, double* res_norms, int* iters,
                 int64_t* sigma_evals, double* times);
void server_wait(pnoeom_server* srv, int64_t id, double timeout_s);
void server_stats(pnoeom_server* srv, size_t* used_bytes, int* queued, int* running, int64_t* rounds,
                  int64_t* merges, int64_t* sigma_evals);
void batch_sigma(pnoeom_batch* B, const int* nvec, const void* const* r, void* const* out, int prec, cudaStream_t s);
void batch_solve(pnoeom_batch* B, const pnoeom_opts* opts, cudaStream_t s, double* energies, double* res_norms,
                 int* iters, int* converged);
// per-system launch entry of a sigma call
SysBuf sysbuf(const pnoeom_pno* P, int nvec, const void* r, void* out, void* work, bool fp32, bool bf16);
// Tensor-core sandwich lists of the BF16 sigma from the phase-2 sandwich problems;
// s_transpose maps the pool offset of an overlap block S(a, b) to (offset of S(b, a), n_a).
void build_tcs(pnoeom_pno* P, const std::vector<SProb>& sp2,
               const std::unordered_map<int64_t, std::pair<int64_t, int>>& s_transpose, cudaStream_t s, size_t* fp);
// zero the outputs and work of every system in the table, then launch the program
// (timing hook: if rec != nullptr, rec(cls, launch) wraps each kernel class)
template <typename T>
void run_program(const Program& prog, const SysTable& t, const int64_t* out_len, const int64_t* work_len,
                 cudaStream_t s, pnoeom_pno* timing_owner = nullptr, bool library = false);
void build_system(pnoeom_ctx* ctx, const pnoeom_system* sys, const pnoeom_opts* opts, cudaStream_t s,
                  pnoeom_pno* P);
template <typename T>
void apply_sigma(pnoeom_pno* P, int nvec, const T* r, T* out, cudaStream_t s, bool bf16);
void run_davidson(pnoeom_ctx* ctx, pnoeom_pno* P, const pnoeom_opts* opts, cudaStream_t s,
                  double* energies, double* res_norms, int* iters, int* converged);
}  // namespace pnoeom
