// Handle state of one built system (pnoeom_pno) and internal entry points.
#pragma once
#include "common.cuh"
#include "engine.cuh"
#include "sigma_prog.cuh"

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
  pnoeom::DBuf<pnoeom::SProb> sp_phase1, sp_phase2;
  pnoeom::DBuf<pnoeom::VProb> vp_phase1, vp_phase2;
  int n_sp1 = 0, n_sp2 = 0, n_vp1 = 0, n_vp2 = 0;
  // small sandwich problems, bucketed by their largest dimension (<= 16, 32, 64) so that each
  // bucket's launch sizes shared memory for its own blocks; within a bucket the problems are
  // ordered by output block, with one group-boundary list per candidate group size
  static constexpr int NGROUP_CAND = 4;
  struct SmallSet {
    pnoeom::DBuf<pnoeom::SProb> probs;
    pnoeom::DBuf<int> starts[NGROUP_CAND];
    int ngroups[NGROUP_CAND] = {0};
    int dims[4] = {1, 1, 1, 1};   // max M, K1, K2, N
    int nprob = 0;
  };
  SmallSet small1[3], small2[3];
  int group_choice = 0;                              // index into GROUP_CAND, set by the autotuner
  int rpc_choice = 0;                                // index into RPC_CAND
  double tune_ms[NGROUP_CAND * 3] = {0};
  int prof_launches[4] = {0, 0, 0, 0};
  int smem_elems = 0;
  int64_t work_len = 0;                      // FvR (v*v) + FoR (o*o)
  int64_t work_fvr = 0, work_for = 0;
  // Davidson data
  pnoeom::DBuf<double> denom_base;           // f_ii (+ f_jj) - fbar_a (- fbar_b), packed
  pnoeom::DBuf<double> guesses;              // projected CIS vectors, nroots_sa x L
  std::vector<double> cis_omega, cis_b;
  std::vector<double> occupations;           // npairs x v eigenvalues of D^{ij}
  std::vector<double> last_X;
  int last_nroots = 0;
  // per-call scratch kept across calls
  pnoeom::DBuf<double> work64; pnoeom::DBuf<float> work32;
  // tracing: per kernel class, operator elements read once per launch,
  // vector elements read+written per vector, flops per vector
  double prof_pool_elems[4] = {0, 0, 0, 0}, prof_vec_elems[4] = {0, 0, 0, 0}, prof_flops[4] = {0, 0, 0, 0};
  bool timing = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> events;
  size_t footprint = 0;
  double build_seconds = 0;
};

namespace pnoeom {
constexpr int NGROUP_CAND = pnoeom_pno::NGROUP_CAND;
constexpr int GROUP_CAND[NGROUP_CAND] = {1, 2, 4, 8};
constexpr int NRPC_CAND = 3;
constexpr int RPC_CAND[NRPC_CAND] = {1, 2, 8};
void autotune(pnoeom_pno* P, cudaStream_t s);
// launch the bucketed small-sandwich problems of one phase with the tuned choices
template <typename T>
inline void run_small_sets(const pnoeom_pno* P, const pnoeom_pno::SmallSet* sets, int nvec, const Buffers& b,
                           cudaStream_t s) {
  for (int k = 0; k < 3; ++k) {
    const auto& S = sets[k];
    if (!S.nprob) continue;
    run_sandwich_small<T>(S.probs.get(), S.starts[P->group_choice].get(), S.ngroups[P->group_choice], nvec, b, S.dims[0],
                          S.dims[1], S.dims[2], S.dims[3], RPC_CAND[P->rpc_choice], s);
  }
}
void build_system(pnoeom_ctx* ctx, const pnoeom_system* sys, const pnoeom_opts* opts, cudaStream_t s,
                  pnoeom_pno* P);
template <typename T>
void apply_sigma(pnoeom_pno* P, int nvec, const T* r, T* out, cudaStream_t s);
void run_davidson(pnoeom_ctx* ctx, pnoeom_pno* P, const pnoeom_opts* opts, cudaStream_t s,
                  double* energies, double* res_norms, int* iters, int* converged);
}  // namespace pnoeom
