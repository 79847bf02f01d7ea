// Dense tensor engine: grouped GEMM, N-d permute, einsum planner.
#include "engine.cuh"
#include <cublas_v2.h>
#include <tuple>
#include <algorithm>
#include <numeric>
#include <map>
#include <chrono>
#include <cstdlib>
#include <atomic>
#include <cuda_bf16.h>

namespace pnoeom {

namespace {
struct ThreadPool {
  std::multimap<size_t, void*> free_blocks;
  ~ThreadPool() {
    if (free_blocks.empty()) return;
    std::lock_guard<std::recursive_mutex> lk(capture_mutex());
    for (auto& b : free_blocks) cudaFree(b.second);
  }
};
thread_local ThreadPool t_pool;

size_t round_size(size_t bytes) {
  if (bytes <= 256) return 256;
  if (bytes >= ((size_t)1 << 20)) return (bytes + ((size_t)1 << 20) - 1) & ~(((size_t)1 << 20) - 1);
  size_t r = 256;
  while (r < bytes) r <<= 1;
  return r;
}
}  // namespace

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
StageTimer::StageTimer(cudaStream_t st) : s(st), on(std::getenv("PNOEOM_LOG_TIMING") != nullptr), t0(now_s()) {}
void StageTimer::mark(const char* what) {
  if (!on) return;
  cudaStreamSynchronize(s);
  double t = now_s();
  std::fprintf(stderr, "[pnoeom] %-28s %8.3f s\n", what, t - t0);
  t0 = t;
}

std::recursive_mutex& capture_mutex() {
  static std::recursive_mutex m;
  return m;
}

// Fault injection and accounting of the caching allocator (host side): the
// countdown makes the allocation request it reaches zero on fail as if the
// device were out of memory; live_bytes counts blocks handed out and not yet
// returned (process-wide, rounded sizes).
static std::atomic<long long> g_fail_countdown{-1};
static std::atomic<long long> g_live_bytes{0};
void inject_alloc_failure(long long after) { g_fail_countdown.store(after < 0 ? -1 : after); }
long long live_alloc_bytes() { return g_live_bytes.load(); }

void* pool_get(size_t bytes) {
  const size_t sz = round_size(bytes);
  long long c = g_fail_countdown.load();
  while (c >= 0 && !g_fail_countdown.compare_exchange_weak(c, c - 1)) {}
  if (c == 0)
    throw Error(PNOEOM_ERR_NOMEM, "device allocation of " + std::to_string(sz) + " bytes failed: injected failure");
  g_live_bytes += (long long)sz;
  auto& fb = t_pool.free_blocks;
  auto it = fb.lower_bound(sz);
  if (it != fb.end() && it->first <= sz + sz / 4) {
    void* p = it->second;
    fb.erase(it);
    return p;
  }
  std::lock_guard<std::recursive_mutex> lk(capture_mutex());
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sz);
  if (e != cudaSuccess) {   // out of memory: return this thread's cache to CUDA and retry once
    cudaGetLastError();
    cudaDeviceSynchronize();
    for (auto& b : fb) cudaFree(b.second);
    fb.clear();
    e = cudaMalloc(&p, sz);
    if (e != cudaSuccess) {
      cudaGetLastError();
      g_live_bytes -= (long long)sz;
      throw Error(e == cudaErrorMemoryAllocation ? PNOEOM_ERR_NOMEM : PNOEOM_ERR_CUDA,
                  "device allocation of " + std::to_string(sz) + " bytes failed: " + cudaGetErrorString(e));
    }
  }
  return p;
}

void pool_put(void* p, size_t bytes) {
  if (!p) return;
  g_live_bytes -= (long long)round_size(bytes);
  t_pool.free_blocks.insert({round_size(bytes), p});
}

void pool_trim() {
  auto& fb = t_pool.free_blocks;
  if (fb.empty()) return;
  std::lock_guard<std::recursive_mutex> lk(capture_mutex());
  for (auto& b : fb) cudaFree(b.second);
  fb.clear();
}

namespace {
constexpr int TM = 64, TN = 64, TK = 16;

struct TileRef { int prob, m0, n0; };

// One 64x64 tile of one problem per CTA; 256 threads as 16x16, each 4x4
// outputs; K staged through shared memory in chunks of 16.
// One BM x BN output tile, 256 threads, each MR x NR outputs; K staged through
// shared memory in chunks of TK.
template <typename T, int BM, int BN, int MR, int NR>
__device__ __forceinline__ void gemm_tile(const GemmProb<T>& P, const TileRef tr, T (*As)[BM + 1], T (*Bs)[BN + 1]) {
  static_assert((BM / MR) * (BN / NR) == 256, "256 threads");
  constexpr int TX = BN / NR;   // threads along N
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  T acc[MR][NR];
#pragma unroll
  for (int i = 0; i < MR; ++i)
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[i][j] = T(0);
  for (int k0 = 0; k0 < P.K; k0 += TK) {
    for (int e = threadIdx.x; e < BM * TK; e += 256) {
      int m, k;
      if (P.ta) { m = e % BM; k = e / BM; } else { k = e % TK; m = e / TK; }
      int gm = tr.m0 + m, gk = k0 + k;
      T val = T(0);
      if (gm < P.M && gk < P.K) val = P.ta ? P.a[(int64_t)gk * P.lda + gm] : P.a[(int64_t)gm * P.lda + gk];
      As[k][m] = val;
    }
    for (int e = threadIdx.x; e < BN * TK; e += 256) {
      int n, k;
      if (P.tb) { k = e % TK; n = e / TK; } else { n = e % BN; k = e / BN; }
      int gn = tr.n0 + n, gk = k0 + k;
      T val = T(0);
      if (gn < P.N && gk < P.K) val = P.tb ? P.b[(int64_t)gn * P.ldb + gk] : P.b[(int64_t)gk * P.ldb + gn];
      Bs[k][n] = val;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TK; ++k) {
      T a[MR], b[NR];
#pragma unroll
      for (int i = 0; i < MR; ++i) a[i] = As[k][ty + (BM / MR) * i];
#pragma unroll
      for (int j = 0; j < NR; ++j) b[j] = Bs[k][tx + TX * j];
#pragma unroll
      for (int i = 0; i < MR; ++i)
#pragma unroll
        for (int j = 0; j < NR; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < MR; ++i) {
    int gm = tr.m0 + ty + (BM / MR) * i;
    if (gm >= P.M) continue;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      int gn = tr.n0 + tx + TX * j;
      if (gn >= P.N) continue;
      T* c = P.c + (int64_t)gm * P.ldc + gn;
      *c = (P.beta == T(0)) ? P.alpha * acc[i][j] : P.alpha * acc[i][j] + P.beta * (*c);
    }
  }
}

// One 64x64 tile of one problem per CTA; 256 threads as 16x16, each 4x4
// outputs; K staged through shared memory in chunks of 16.
template <typename T>
__device__ __forceinline__ void gemm_tile(const GemmProb<T>& P, const TileRef tr, T (*As)[TM + 1], T (*Bs)[TN + 1]) {
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int k0 = 0; k0 < P.K; k0 += TK) {
    for (int e = threadIdx.x; e < TM * TK; e += 256) {
      int m, k;
      if (P.ta) { m = e % TM; k = e / TM; } else { k = e % TK; m = e / TK; }
      int gm = tr.m0 + m, gk = k0 + k;
      T val = T(0);
      if (gm < P.M && gk < P.K) val = P.ta ? P.a[(int64_t)gk * P.lda + gm] : P.a[(int64_t)gm * P.lda + gk];
      As[k][m] = val;
    }
    for (int e = threadIdx.x; e < TN * TK; e += 256) {
      int n, k;
      if (P.tb) { k = e % TK; n = e / TK; } else { n = e % TN; k = e / TN; }
      int gn = tr.n0 + n, gk = k0 + k;
      T val = T(0);
      if (gn < P.N && gk < P.K) val = P.tb ? P.b[(int64_t)gn * P.ldb + gk] : P.b[(int64_t)gk * P.ldb + gn];
      Bs[k][n] = val;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TK; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = tr.m0 + ty + 16 * i;
    if (gm >= P.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = tr.n0 + tx + 16 * j;
      if (gn >= P.N) continue;
      T* c = P.c + (int64_t)gm * P.ldc + gn;
      *c = (P.beta == T(0)) ? P.alpha * acc[i][j] : P.alpha * acc[i][j] + P.beta * (*c);
    }
  }
}

// One 64x64 tile of one problem per CTA; 256 threads as 16x16, each 4x4
// outputs; K staged through shared memory in chunks of 16.
template <typename T>
__global__ void __launch_bounds__(256) k_grouped_gemm(const GemmProb<T>* __restrict__ probs,
                                                      const TileRef* __restrict__ tiles) {
  __shared__ T As[TK][TM + 1];
  __shared__ T Bs[TK][TN + 1];
  const TileRef tr = tiles[blockIdx.x];
  gemm_tile<T, TM, TN, 4, 4>(probs[tr.prob], tr, As, Bs);
}

// Small groups: problems and tile offsets passed by value (no descriptor upload,
// hence no implicit synchronisation of pageable host-to-device copies).
constexpr int NPV = 160;
template <typename T>
struct GemmParams {
  int nprob;
  int tile_start[NPV + 1];
  GemmProb<T> probs[NPV];
};

template <typename T, int BM, int BN, int MR, int NR>
__global__ void __launch_bounds__(256) k_grouped_gemm_v(const __grid_constant__ GemmParams<T> gp) {
  __shared__ T As[TK][BM + 1];
  __shared__ T Bs[TK][BN + 1];
  int lo = 0, hi = gp.nprob - 1;
  const int tile = blockIdx.x;
  while (lo < hi) {   // problem of this tile: last p with tile_start[p] <= tile
    int mid = (lo + hi + 1) / 2;
    if (gp.tile_start[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  const GemmProb<T>& P = gp.probs[lo];
  const int local = tile - gp.tile_start[lo];
  const int ntn = (P.N + BN - 1) / BN;
  TileRef tr{lo, (local / ntn) * BM, (local % ntn) * BN};
  gemm_tile<T, BM, BN, MR, NR>(P, tr, As, Bs);
}

constexpr int PMAX = 8;
struct PermArgs {
  int nd;
  int64_t out_dims[PMAX];
  int64_t in_stride_for_out[PMAX];   // stride in `in` of each output axis
};

template <typename T>
__global__ void k_permute(const T* __restrict__ in, T* __restrict__ out, PermArgs a, int64_t total, T alpha, T beta) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e, off = 0;
    for (int d = a.nd - 1; d >= 0; --d) {
      int64_t c = r % a.out_dims[d];
      r /= a.out_dims[d];
      off += c * a.in_stride_for_out[d];
    }
    T v = alpha * in[off];
    out[e] = (beta == T(0)) ? v : v + beta * out[e];
  }
}

template <typename T>
__global__ void k_axpby(T* y, const T* x, T a, T b, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] = a * x[e] + (b == T(0) ? T(0) : b * y[e]);
}
template <typename T>
__global__ void k_scale(T* y, T a, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) y[e] *= a;
}
__global__ void k_d2f(float* y, const double* x, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) y[e] = (float)x[e];
}
__global__ void k_f2d(double* y, const float* x, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) y[e] = (double)x[e];
}

inline unsigned grid_for(size_t n) {
  size_t g = (n + 255) / 256;
  return (unsigned)std::max<size_t>(1, std::min<size_t>(g, 152 * 32));
}
}  // namespace

namespace {
// One cuBLAS handle per host thread (created on first use, destroyed at thread exit).
struct ThreadBlas {
  cublasHandle_t h = nullptr;
  ~ThreadBlas() {
    if (h) {
      std::lock_guard<std::recursive_mutex> lk(capture_mutex());
      cublasDestroy(h);
    }
  }
  cublasHandle_t get(cudaStream_t s) {
    if (!h) {
      std::lock_guard<std::recursive_mutex> lk(capture_mutex());
      PN_CHECK(cublasCreate(&h) == CUBLAS_STATUS_SUCCESS, PNOEOM_ERR_CUDA, "cublasCreate failed");
    }
    PN_CHECK(cublasSetStream(h, s) == CUBLAS_STATUS_SUCCESS, PNOEOM_ERR_CUDA, "cublasSetStream failed");
    return h;
  }
};
thread_local ThreadBlas t_blas;

// FP64 problems with at least this many multiply-adds go to cuBLAS DGEMM, grouped by
// shape into batched calls; smaller ones stay on the grouped SIMT kernel, where one launch
// covers many of them.
constexpr double BLAS_MIN_MACS = 32768.0;

// C = alpha op(A) op(B) + beta C in row-major storage is, read column-major,
// C^T = alpha op(B)^T op(A)^T + beta C^T: cuBLAS gets B first, m = N, n = M.
void blas_dgemm_groups(const std::vector<GemmProb<double>>& big, cudaStream_t s) {
  if (big.empty()) return;
  using Key = std::tuple<int, int, int, int, int, int, int, int, double, double>;
  std::map<Key, std::vector<const GemmProb<double>*>> groups;
  for (const auto& P : big) groups[Key{P.M, P.N, P.K, P.lda, P.ldb, P.ldc, P.ta, P.tb, P.alpha, P.beta}].push_back(&P);
  cublasHandle_t h = t_blas.get(s);
  for (auto& g : groups) {
    const GemmProb<double>& P = *g.second.front();
    const cublasOperation_t opb = P.tb ? CUBLAS_OP_T : CUBLAS_OP_N, opa = P.ta ? CUBLAS_OP_T : CUBLAS_OP_N;
    const double al = P.alpha, be = P.beta;
    cublasStatus_t st;
    if (g.second.size() == 1) {
      st = cublasDgemm(h, opb, opa, P.N, P.M, P.K, &al, P.b, P.ldb, P.a, P.lda, &be, P.c, P.ldc);
    } else {
      const size_t n = g.second.size();
      std::vector<const double*> hp(3 * n);
      for (size_t k = 0; k < n; ++k) {
        hp[k] = g.second[k]->b;
        hp[n + k] = g.second[k]->a;
        hp[2 * n + k] = g.second[k]->c;
      }
      DBuf<const double*> dp(3 * n);
      dp.upload(hp.data(), 3 * n, s);
      st = cublasDgemmBatched(h, opb, opa, P.N, P.M, P.K, &al, dp.get(), P.ldb, dp.get() + n, P.lda, &be,
                              const_cast<double* const*>(dp.get() + 2 * n), P.ldc, (int)n);
    }
    PN_CHECK(st == CUBLAS_STATUS_SUCCESS, PNOEOM_ERR_CUDA, "cuBLAS DGEMM failed");
  }
}
}  // namespace

// C = alpha op(A) op(B) + beta C (row-major, single precision storage) for `batch`
// independent triples at element strides sA, sB, sC (0: shared operand); tf32 selects
// TF32 tensor-core arithmetic with FP32 accumulation, else plain FP32.
void blas_sgemm_strided(bool tf32, int ta, int tb, int M, int N, int K, float alpha, const float* A, int lda, long long sA,
                        const float* B, int ldb, long long sB, float beta, float* C, int ldc, long long sC, int batch,
                        cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return;
  cublasHandle_t h = t_blas.get(s);
  const cublasOperation_t opb = tb ? CUBLAS_OP_T : CUBLAS_OP_N, opa = ta ? CUBLAS_OP_T : CUBLAS_OP_N;
  const cublasStatus_t st = cublasGemmStridedBatchedEx(
      h, opb, opa, N, M, K, &alpha, B, CUDA_R_32F, ldb, sB, A, CUDA_R_32F, lda, sA, &beta, C, CUDA_R_32F, ldc, sC, batch,
      tf32 ? CUBLAS_COMPUTE_32F_FAST_TF32 : CUBLAS_COMPUTE_32F_PEDANTIC, CUBLAS_GEMM_DEFAULT);
  PN_CHECK(st == CUBLAS_STATUS_SUCCESS, PNOEOM_ERR_CUDA, "cuBLAS strided-batched GEMM failed");
}

template <typename T>
void grouped_gemm(const std::vector<GemmProb<T>>& probs_in, cudaStream_t s) {
  if (probs_in.empty()) return;
  std::vector<GemmProb<T>> rest;
  const std::vector<GemmProb<T>>* pp = &probs_in;
  if (sizeof(T) == 8) {
    std::vector<GemmProb<double>> big;
    for (const auto& P : probs_in) {
      if (P.M <= 0 || P.N <= 0) continue;
      if ((double)P.M * P.N * std::max(P.K, 1) >= BLAS_MIN_MACS && P.K > 0)
        big.push_back(reinterpret_cast<const GemmProb<double>&>(P));
      else
        rest.push_back(P);
    }
    blas_dgemm_groups(big, s);
    pp = &rest;
    if (rest.empty()) return;
  }
  const std::vector<GemmProb<T>>& probs = *pp;
  // by-value path: up to NPV problems per launch
  size_t i0 = 0;
  bool small = true;
  {
    size_t nonempty = 0;
    for (auto& P : probs) nonempty += (P.M > 0 && P.N > 0);
    small = nonempty <= (size_t)4 * NPV;
  }
  if (small) {
    // shape classes: skinny problems (one side <= 16) use 128 x 16 or 16 x 128 tiles,
    // the others 64 x 64
    std::vector<GemmProb<T>> wide, skinny_n, skinny_m;
    for (const auto& P0 : probs) {
      if (P0.M <= 0 || P0.N <= 0) continue;
      if (P0.N <= 16 && P0.M > 16) skinny_n.push_back(P0);
      else if (P0.M <= 16 && P0.N > 16) skinny_m.push_back(P0);
      else wide.push_back(P0);
    }
    auto launch = [&](const std::vector<GemmProb<T>>& L, int bm, int bn) {
      GemmParams<T> gp;
      size_t j = 0;
      while (j < L.size()) {
        gp.nprob = 0;
        int tiles = 0;
        for (; j < L.size() && gp.nprob < NPV; ++j) {
          gp.tile_start[gp.nprob] = tiles;
          gp.probs[gp.nprob++] = L[j];
          tiles += ((L[j].M + bm - 1) / bm) * ((L[j].N + bn - 1) / bn);
        }
        gp.tile_start[gp.nprob] = tiles;
        if (bn == 16) k_grouped_gemm_v<T, 128, 16, 8, 1><<<tiles, 256, 0, s>>>(gp);
        else if (bm == 16) k_grouped_gemm_v<T, 16, 128, 1, 8><<<tiles, 256, 0, s>>>(gp);
        else k_grouped_gemm_v<T, TM, TN, 4, 4><<<tiles, 256, 0, s>>>(gp);
        PN_CUDA(cudaGetLastError());
      }
    };
    launch(wide, TM, TN);
    launch(skinny_n, 128, 16);
    launch(skinny_m, 16, 128);
    return;
  }
  std::vector<TileRef> tiles;
  for (int p = 0; p < (int)probs.size(); ++p) {
    const auto& P = probs[p];
    if (P.M <= 0 || P.N <= 0) continue;
    for (int m0 = 0; m0 < P.M; m0 += TM)
      for (int n0 = 0; n0 < P.N; n0 += TN) tiles.push_back({p, m0, n0});
  }
  if (tiles.empty()) return;
  DBuf<GemmProb<T>> dp(probs.size());
  DBuf<TileRef> dt(tiles.size());
  dp.upload(probs.data(), probs.size(), s);
  dt.upload(tiles.data(), tiles.size(), s);
  k_grouped_gemm<T><<<(unsigned)tiles.size(), 256, 0, s>>>(dp.get(), dt.get());
  PN_CUDA(cudaGetLastError());
  // the descriptor buffers go back to this thread's cache; later reuse is ordered on the same stream
}

template <typename T>
void permute(const T* in, T* out, const std::vector<int64_t>& dims_in, const std::vector<int>& perm,
             T alpha, T beta, cudaStream_t s) {
  int nd = (int)dims_in.size();
  PN_CHECK(nd <= PMAX && (int)perm.size() == nd, PNOEOM_ERR_UNSUPPORTED, "permute rank");
  std::vector<int64_t> stride(nd, 1);
  for (int d = nd - 2; d >= 0; --d) stride[d] = stride[d + 1] * dims_in[d + 1];
  PermArgs a{};
  a.nd = nd;
  int64_t total = 1;
  for (int k = 0; k < nd; ++k) {
    a.out_dims[k] = dims_in[perm[k]];
    a.in_stride_for_out[k] = stride[perm[k]];
    total *= a.out_dims[k];
  }
  if (total == 0) return;
  k_permute<T><<<grid_for(total), 256, 0, s>>>(in, out, a, total, alpha, beta);
  PN_CUDA(cudaGetLastError());
}

template <typename T>
void contract(const std::map<char, int64_t>& dims, TView<T> A, TView<T> B, TView<T> C,
              T alpha, T beta, cudaStream_t s) {
  auto has = [](const std::string& x, char c) { return x.find(c) != std::string::npos; };
  std::string bat, mm, nn, kk;
  for (char c : C.idx) {
    bool a = has(A.idx, c), b = has(B.idx, c);
    PN_CHECK(a || b, PNOEOM_ERR_INVALID_ARG, std::string("contract: output index not in inputs: ") + c);
    if (a && b) bat += c; else if (a) mm += c; else nn += c;
  }
  for (char c : A.idx) if (!has(C.idx, c)) {
    PN_CHECK(has(B.idx, c), PNOEOM_ERR_INVALID_ARG, std::string("contract: dangling index ") + c);
    kk += c;
  }
  for (char c : B.idx) if (!has(C.idx, c) && !has(A.idx, c))
    throw Error(PNOEOM_ERR_INVALID_ARG, std::string("contract: dangling index ") + c);
  auto ext = [&](const std::string& x) { int64_t e = 1; for (char c : x) e *= dims.at(c); return e; };
  const int64_t nb = ext(bat), M = ext(mm), N = ext(nn), K = ext(kk);
  if (nb == 0 || M == 0 || N == 0) return;
  // Bring an operand into the target axis order; returns pointer (maybe the original).
  auto arrange = [&](TView<T> X, const std::string& target, DBuf<T>& tmp) -> const T* {
    if (X.idx == target) return X.p;
    std::vector<int64_t> din;
    for (char c : X.idx) din.push_back(dims.at(c));
    std::vector<int> perm;
    for (char c : target) perm.push_back((int)X.idx.find(c));
    tmp.alloc(ext(target));
    permute<T>(X.p, tmp.get(), din, perm, T(1), T(0), s);
    return tmp.get();
  };
  // A as [bat, mm, kk] or [bat, kk, mm] (transposed) -- pick whichever needs no copy.
  DBuf<T> ta_, tb_, tc_;
  int transA = 0, transB = 0;
  const T* pa;
  if (A.idx == bat + kk + mm) { pa = A.p; transA = 1; }
  else pa = arrange(A, bat + mm + kk, ta_);
  const T* pb;
  if (B.idx == bat + nn + kk) { pb = B.p; transB = 1; }
  else pb = arrange(B, bat + kk + nn, tb_);
  std::string cord = bat + mm + nn;
  T* pc;
  bool direct = (C.idx == cord);
  if (direct) pc = C.p; else { tc_.alloc(nb * M * N); pc = tc_.get(); }
  std::vector<GemmProb<T>> probs;
  probs.reserve(nb);
  for (int64_t b = 0; b < nb; ++b) {
    GemmProb<T> P;
    P.a = pa + b * M * K; P.b = pb + b * K * N; P.c = pc + b * M * N;
    P.M = (int)M; P.N = (int)N; P.K = (int)K;
    P.lda = transA ? (int)M : (int)K;
    P.ldb = transB ? (int)K : (int)N;
    P.ldc = (int)N;
    P.ta = transA; P.tb = transB;
    P.alpha = direct ? alpha : T(1);
    P.beta = direct ? beta : T(0);
    probs.push_back(P);
  }
  PN_CHECK(M < INT32_MAX && N < INT32_MAX && K < INT32_MAX, PNOEOM_ERR_UNSUPPORTED, "contract: extent too large");
  grouped_gemm<T>(probs, s);
  if (!direct) {
    std::vector<int64_t> din;
    for (char c : cord) din.push_back(dims.at(c));
    std::vector<int> perm;
    for (char c : C.idx) perm.push_back((int)cord.find(c));
    permute<T>(pc, C.p, din, perm, alpha, beta, s);
  }
}

template <typename T> void axpby(T* y, const T* x, T a, T b, size_t n, cudaStream_t s) {
  if (!n) return;
  k_axpby<T><<<grid_for(n), 256, 0, s>>>(y, x, a, b, n);
  PN_CUDA(cudaGetLastError());
}
template <typename T> void scale(T* y, T a, size_t n, cudaStream_t s) {
  if (!n) return;
  k_scale<T><<<grid_for(n), 256, 0, s>>>(y, a, n);
  PN_CUDA(cudaGetLastError());
}
void d2f(float* y, const double* x, size_t n, cudaStream_t s) {
  if (!n) return;
  k_d2f<<<grid_for(n), 256, 0, s>>>(y, x, n);
  PN_CUDA(cudaGetLastError());
}
__global__ void k_d2bf(__nv_bfloat16* y, const double* x, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] = __double2bfloat16(x[e]);
}
void d2bf(void* y, const double* x, size_t n, cudaStream_t s) {
  if (!n) return;
  k_d2bf<<<grid_for(n), 256, 0, s>>>((__nv_bfloat16*)y, x, n);
  PN_CUDA(cudaGetLastError());
}
void f2d(double* y, const float* x, size_t n, cudaStream_t s) {
  if (!n) return;
  k_f2d<<<grid_for(n), 256, 0, s>>>(y, x, n);
  PN_CUDA(cudaGetLastError());
}

template void grouped_gemm<double>(const std::vector<GemmProb<double>>&, cudaStream_t);
template void grouped_gemm<float>(const std::vector<GemmProb<float>>&, cudaStream_t);
template void permute<double>(const double*, double*, const std::vector<int64_t>&, const std::vector<int>&, double, double, cudaStream_t);
template void permute<float>(const float*, float*, const std::vector<int64_t>&, const std::vector<int>&, float, float, cudaStream_t);
template void contract<double>(const std::map<char, int64_t>&, TView<double>, TView<double>, TView<double>, double, double, cudaStream_t);
template void axpby<double>(double*, const double*, double, double, size_t, cudaStream_t);
template void axpby<float>(float*, const float*, float, float, size_t, cudaStream_t);
template void scale<double>(double*, double, size_t, cudaStream_t);
template void scale<float>(float*, float, size_t, cudaStream_t);

}  // namespace pnoeom
