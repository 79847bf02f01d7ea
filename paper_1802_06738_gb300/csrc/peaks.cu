// Peak-rate microbenchmarks of the device the library runs on, the denominators of
// the roofline fractions the benchmark reports: FP32 and FP64 FMA issue rates of
// the SIMT pipes, tcgen05 MMA rates for kind::f16 (BF16 operands) and kind::tf32
// with FP32 accumulation, and cuBLAS DGEMM, native and with the FP64 emulation
// math mode, for the FP64 setup contractions.  Nothing here changes a device
// setting; each figure is the best of a few CUDA-event-timed launches.
#include "pno.cuh"
#include "tc.cuh"
#include <cublas_v2.h>
#include <algorithm>
#include <cmath>
#include <vector>

namespace pnoeom {
namespace {

constexpr int FMA_CHAINS = 8;     // independent accumulators per thread
constexpr int FMA_UNROLL = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_peak_fma(T* out, int iters, T seed) {
  T a[FMA_CHAINS];
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; ++c) a[c] = seed * (T)(threadIdx.x + c);
  const T b = (T)0.999999, d = (T)1e-7;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < FMA_UNROLL; ++u)
#pragma unroll
      for (int c = 0; c < FMA_CHAINS; ++c) a[c] = fma(a[c], b, d);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < FMA_CHAINS; ++c) s += a[c];
  if (s == (T)-12345.0) out[0] = s;   // keeps the chains alive
}

__device__ int g_peak_status = 0;

// tcgen05 MMA throughput: one CTA per SM, one thread issues `nmma` accumulating MMAs of
// 128 x 256 x K into one TMEM accumulator from fixed shared-memory operand tiles
// (K-major, no swizzle), commits once and waits for completion with a bounded wait.
// kind: 0 = kind::f16 with BF16 operands (K = 16), 1 = kind::tf32 (K = 8).
__global__ void __launch_bounds__(128) k_peak_mma(int nmma, int kind) {
  __shared__ __align__(1024) unsigned char tiles[4096 + 8192];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x;
  for (int e = tid; e < (4096 + 8192) / 4; e += blockDim.x) reinterpret_cast<uint32_t*>(tiles)[e] = 0u;
  if (tid < 32) tc::tmem_alloc(&tslot, 256);
  if (tid == 0) tc::mbar_init(&bar, 1);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  // A: 128 rows x 16 bytes-of-K per core column, B: 256 rows; core matrices 8 rows x 16 B,
  // adjacent along M/N 128 B apart (SBO), adjacent along K rows/8 * 128 B apart (LBO)
  const uint32_t a0 = tc::smem_u32(tiles), b0 = tc::smem_u32(tiles + 4096);
  const uint64_t ad = tc::sdesc(a0, 128 / 8 * 128, 128), bd = tc::sdesc(b0, 256 / 8 * 128, 128);
  if (tid == 0) {
    if (kind == 0) {
      const uint32_t idesc = tc::idesc_bf16(128, 256);
      for (int i = 0; i < nmma; ++i) tc::mma_bf16(tmem, ad, bd, idesc, i > 0 ? 1u : 0u);
    } else {
      const uint32_t idesc = tc::idesc_tf32(128, 256);
      for (int i = 0; i < nmma; ++i) tc::mma_tf32(tmem, ad, bd, idesc, i > 0 ? 1u : 0u);
    }
    tc::mma_commit(&bar);
  }
  const bool ok = __syncthreads_and(tc::mbar_wait_bounded(&bar, 0u, 4000000000LL) ? 1 : 0) != 0;
  if (!ok && tid == 0) atomicOr(&g_peak_status, 1);
  tc::fence_after_sync();
  __syncthreads();
  if (ok && tid < 32) tc::tmem_dealloc(tmem, 256);
}

struct Timer {
  cudaEvent_t a, b;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {
    PN_CUDA(cudaEventCreate(&a));
    PN_CUDA(cudaEventCreate(&b));
  }
  ~Timer() { cudaEventDestroy(a); cudaEventDestroy(b); }
  template <typename F>
  double best_ms(int reps, F&& f) {
    f();   // warm-up
    double best = 1e300;
    for (int r = 0; r < reps; ++r) {
      PN_CUDA(cudaEventRecord(a, s));
      f();
      PN_CUDA(cudaEventRecord(b, s));
      PN_CUDA(cudaEventSynchronize(b));
      float ms = 0;
      PN_CUDA(cudaEventElapsedTime(&ms, a, b));
      best = std::min(best, (double)ms);
    }
    return best;
  }
};

__global__ void k_fill(double* x, size_t n, uint64_t seed) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    uint64_t z = (e + 1) * 0x9E3779B97F4A7C15ull ^ seed;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[e] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
}

}  // namespace

// out (at most nout values): [0] FP32 FMA TFLOP/s, [1] FP64 FMA TFLOP/s, [2] tcgen05 BF16
// TFLOP/s, [3] tcgen05 TF32 TFLOP/s, [4] cuBLAS DGEMM TFLOP/s (n = 4096), [5] cuBLAS DGEMM
// with CUBLAS_FP64_EMULATED_FIXEDPOINT_MATH and the eager emulation strategy, TFLOP/s, [6] max |emulated - native| / max |native|
// of that product, [7] SM count.
void measure_peaks(cudaStream_t s, double* out, int nout) {
  int dev = 0, sms = 0;
  PN_CUDA(cudaGetDevice(&dev));
  PN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  std::vector<double> r(8, 0.0);
  r[7] = sms;
  Timer tm(s);
  {
    DBuf<float> o32(1);
    DBuf<double> o64(1);
    const int blocks = sms * 8, threads = 256, it32 = 4096, it64 = 256;
    const double ms32 = tm.best_ms(3, [&] { k_peak_fma<float><<<blocks, threads, 0, s>>>(o32.get(), it32, 1e-3f); });
    const double ms64 = tm.best_ms(3, [&] { k_peak_fma<double><<<blocks, threads, 0, s>>>(o64.get(), it64, 1e-3); });
    PN_CUDA(cudaGetLastError());
    const double per = 2.0 * blocks * threads * FMA_CHAINS * FMA_UNROLL;
    r[0] = per * it32 / (ms32 * 1e-3) / 1e12;
    r[1] = per * it64 / (ms64 * 1e-3) / 1e12;
  }
  {
    const int nmma = 16384;
    const size_t pad = 160 * 1024;   // unused dynamic shared memory: one CTA per SM
    PN_CUDA(cudaFuncSetAttribute((const void*)k_peak_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pad));
    const double ms16 = tm.best_ms(3, [&] { k_peak_mma<<<sms, 128, pad, s>>>(nmma, 0); });
    const double ms32 = tm.best_ms(3, [&] { k_peak_mma<<<sms, 128, pad, s>>>(nmma, 1); });
    PN_CUDA(cudaGetLastError());
    int st = 0;
    PN_CUDA(cudaMemcpyFromSymbolAsync(&st, g_peak_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    PN_CUDA(cudaStreamSynchronize(s));
    PN_CHECK(st == 0, PNOEOM_ERR_TIMEOUT, "tensor-core peak kernel: a bounded wait ran out");
    r[2] = 2.0 * 128 * 256 * 16 * (double)nmma * sms / (ms16 * 1e-3) / 1e12;
    r[3] = 2.0 * 128 * 256 * 8 * (double)nmma * sms / (ms32 * 1e-3) / 1e12;
  }
  {
    const int n = 4096;
    const size_t nn = (size_t)n * n;
    DBuf<double> A(nn), B(nn), C(nn), C2(nn);
    k_fill<<<sms * 4, 256, 0, s>>>(A.get(), nn, 1);
    k_fill<<<sms * 4, 256, 0, s>>>(B.get(), nn, 2);
    PN_CUDA(cudaGetLastError());
    cublasHandle_t h = nullptr;
    PN_CHECK(cublasCreate(&h) == CUBLAS_STATUS_SUCCESS, PNOEOM_ERR_CUDA, "cublasCreate failed");
    cublasSetStream(h, s);
    const double one = 1.0, zero = 0.0;
    auto gemm = [&](double* Cx) {
      PN_CHECK(cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one, A.get(), n, B.get(), n, &zero, Cx, n) ==
                   CUBLAS_STATUS_SUCCESS, PNOEOM_ERR_CUDA, "cublasDgemm failed");
    };
    const double flops = 2.0 * n * (double)n * n;
    cublasSetMathMode(h, CUBLAS_DEFAULT_MATH);
    r[4] = flops / (tm.best_ms(2, [&] { gemm(C.get()); }) * 1e-3) / 1e12;
    if (cublasSetMathMode(h, CUBLAS_FP64_EMULATED_FIXEDPOINT_MATH) == CUBLAS_STATUS_SUCCESS &&
        cublasSetEmulationStrategy(h, CUBLAS_EMULATION_STRATEGY_EAGER) == CUBLAS_STATUS_SUCCESS) {
      auto gemm_ex = [&](double* Cx) {
        PN_CHECK(cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one, A.get(), CUDA_R_64F, n, B.get(), CUDA_R_64F, n,
                              &zero, Cx, CUDA_R_64F, n, CUBLAS_COMPUTE_64F_EMULATED_FIXEDPOINT,
                              CUBLAS_GEMM_DEFAULT) == CUBLAS_STATUS_SUCCESS, PNOEOM_ERR_CUDA, "cublasGemmEx failed");
      };
      r[5] = flops / (tm.best_ms(2, [&] { gemm_ex(C2.get()); }) * 1e-3) / 1e12;
      std::vector<double> c1(nn), c2(nn);
      C.download(c1.data(), nn, s);
      C2.download(c2.data(), nn, s);
      PN_CUDA(cudaStreamSynchronize(s));
      double mx = 0, md = 0;
      for (size_t e = 0; e < nn; ++e) { mx = std::max(mx, std::fabs(c1[e])); md = std::max(md, std::fabs(c1[e] - c2[e])); }
      r[6] = mx > 0 ? md / mx : 0;
    }
    cublasDestroy(h);
  }
  for (int k = 0; k < std::min(nout, 8); ++k) out[k] = r[k];
}

}  // namespace pnoeom

extern "C" int pnoeom_measure_peaks(pnoeom_ctx* ctx, void* cuda_stream, double* out, int nout) {
  return pnoeom::guard_call([&] {
    PN_CHECK(ctx && out && nout >= 1, PNOEOM_ERR_INVALID_ARG, "bad arguments");
    pnoeom::DeviceScope dev_scope(ctx->device);
    pnoeom::measure_peaks(reinterpret_cast<cudaStream_t>(cuda_stream), out, nout);
  });
}
