// Dense tensor engine: grouped GEMM, N-d permute, einsum planner.
#include "engine.cuh"
#include <algorithm>
#include <numeric>

namespace pnoeom {

namespace {
constexpr int TM = 64, TN = 64, TK = 16;

struct TileRef { int prob, m0, n0; };

// One 64x64 tile of one problem per CTA; 256 threads as 16x16, each 4x4
// outputs; K staged through shared memory in chunks of 16.
template <typename T>
__global__ void __launch_bounds__(256) k_grouped_gemm(const GemmProb<T>* __restrict__ probs,
                                                      const TileRef* __restrict__ tiles) {
  __shared__ T As[TK][TM + 1];
  __shared__ T Bs[TK][TN + 1];
  const TileRef tr = tiles[blockIdx.x];
  const GemmProb<T> P = probs[tr.prob];
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

template <typename T>
void grouped_gemm(const std::vector<GemmProb<T>>& probs, cudaStream_t s) {
  if (probs.empty()) return;
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
  for (size_t t0 = 0; t0 < tiles.size(); t0 += 2147483647u) {
    size_t nt = std::min<size_t>(tiles.size() - t0, 2147483647u);
    k_grouped_gemm<T><<<(unsigned)nt, 256, 0, s>>>(dp.get(), dt.get() + t0);
  }
  PN_CUDA(cudaGetLastError());
  PN_CUDA(cudaStreamSynchronize(s));   // the descriptor buffers are freed on return
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
    PN_CUDA(cudaStreamSynchronize(s));
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
