// Dense tensor engine used by the setup and the sigma program:
//   * grouped GEMM (each problem its own sizes, pointers, transposes,
//     alpha/beta; 64x64 output tiles, one tile per CTA);
//   * N-d permute with scale-and-accumulate;
//   * an einsum-style contraction planner built on the two.
#pragma once
#include "common.cuh"
#include <map>

namespace pnoeom {

template <typename T>
struct GemmProb {
  const T* a; const T* b; T* c;
  int M, N, K;
  int lda, ldb, ldc;
  int ta, tb;          // A is M x K (ta = 0: a[m*lda+k]; 1: a[k*lda+m]); B is K x N likewise
  T alpha, beta;       // C = alpha A B + beta C
};

// Problems of one call run concurrently: their C regions must not overlap.
template <typename T>
void grouped_gemm(const std::vector<GemmProb<T>>& probs, cudaStream_t s);
// C = alpha op(A) op(B) + beta C (row-major FP32 storage) for `batch` triples at element
// strides sA, sB, sC (0: shared operand); tf32: TF32 tensor cores, FP32 accumulation.
void blas_sgemm_strided(bool tf32, int ta, int tb, int M, int N, int K, float alpha, const float* A, int lda, long long sA,
                        const float* B, int ldb, long long sB, float beta, float* C, int ldc, long long sC, int batch,
                        cudaStream_t s);

// out[perm-index] = alpha * in + beta * out, where dims_in are the input's
// dimensions (row-major) and perm[k] = the input axis placed at output axis k.
template <typename T>
void permute(const T* in, T* out, const std::vector<int64_t>& dims_in, const std::vector<int>& perm,
             T alpha, T beta, cudaStream_t s);

// A tensor view for the planner: contiguous row-major array with named axes.
template <typename T>
struct TView {
  T* p;
  std::string idx;     // one letter per axis
};

// C[idxC] = alpha * sum A[idxA] B[idxB] + beta * C.  Every letter appears in
// exactly two of the three operands (batch letters in all three).  `dims`
// gives each letter's extent.  Temporaries are allocated internally.
template <typename T>
void contract(const std::map<char, int64_t>& dims, TView<T> A, TView<T> B, TView<T> C,
              T alpha, T beta, cudaStream_t s);

// Elementwise helpers
template <typename T> void axpby(T* y, const T* x, T a, T b, size_t n, cudaStream_t s);  // y = a x + b y
template <typename T> void scale(T* y, T a, size_t n, cudaStream_t s);
void d2f(float* y, const double* x, size_t n, cudaStream_t s);
void f2d(double* y, const float* x, size_t n, cudaStream_t s);
void d2bf(void* y, const double* x, size_t n, cudaStream_t s);   // y: __nv_bfloat16[n], rounded to nearest

}  // namespace pnoeom
