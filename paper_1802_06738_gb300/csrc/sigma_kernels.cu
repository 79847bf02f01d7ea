// Kernels of the sigma program (see sigma_prog.cuh).
#include <map>
#include <mutex>
#include "sigma_prog.cuh"

namespace pnoeom {
namespace {

template <typename T>
__device__ __forceinline__ const T* cbuf(const SysTable& t, int sys, int id, int r) {
  const SysBuf& b = t.s[sys];
  switch (id) {
    case B_POOL: return (const T*)b.pool;
    case B_RIN: return (const T*)b.rin + (int64_t)r * b.rin_stride;
    case B_WORK: return (const T*)b.work + (int64_t)r * b.work_stride;
    default: return (const T*)b.sout + (int64_t)r * b.sout_stride;
  }
}
template <typename T>
__device__ __forceinline__ T* mbuf(const SysTable& t, int sys, int id, int r) {
  const SysBuf& b = t.s[sys];
  return id == B_WORK ? (T*)b.work + (int64_t)r * b.work_stride : (T*)b.sout + (int64_t)r * b.sout_stride;
}

// One (problem, root) per CTA.  T_s = opX(X) * opB(B) restricted to the
// output tile's columns is formed in shared memory, then C_tile += alpha *
// opA(A)[tile rows] * T_s.  Accumulation into C is atomic because many
// problems share an output block.
template <typename T>
__global__ void __launch_bounds__(256) k_sandwich(const SProb* __restrict__ probs, const __grid_constant__ SysTable tab) {
  extern __shared__ unsigned char smem_raw[];
  T* Ts = reinterpret_cast<T*>(smem_raw);
  const SProb P = probs[blockIdx.x];
  const int r = blockIdx.y;
  if (r >= tab.s[P.sys].nvec) return;
  const T* X = cbuf<T>(tab, P.sys, P.x_buf, r) + P.x_off;
  const T* A = P.a_buf == B_NONE ? nullptr : cbuf<T>(tab, P.sys, P.a_buf, r) + P.a_off;
  const T* Bm = P.b_buf == B_NONE ? nullptr : cbuf<T>(tab, P.sys, P.b_buf, r) + P.b_off;
  T* C = mbuf<T>(tab, P.sys, P.c_buf, r) + P.c_off;
  const int Mt = min(64, P.M - P.m0), Nt = min(64, P.N - P.n0);
  // rows of T_s: K1 if A is present, else the tile's rows of X (K1 == M)
  const int trow0 = A ? 0 : P.m0;
  const int Tr = A ? P.K1 : Mt;
  for (int e = threadIdx.x; e < Tr * Nt; e += blockDim.x) {
    const int k1 = trow0 + e / Nt, n = P.n0 + e % Nt;
    T acc = T(0);
    if (Bm) {
      for (int k2 = 0; k2 < P.K2; ++k2) {
        T xv = P.tx ? X[(int64_t)k2 * P.ldx + k1] : X[(int64_t)k1 * P.ldx + k2];
        T bv = P.tb ? Bm[(int64_t)n * P.ldb + k2] : Bm[(int64_t)k2 * P.ldb + n];
        acc += xv * bv;
      }
    } else {
      acc = P.tx ? X[(int64_t)n * P.ldx + k1] : X[(int64_t)k1 * P.ldx + n];
    }
    Ts[e] = acc;
  }
  __syncthreads();
  const T alpha = (T)P.alpha;
  for (int e = threadIdx.x; e < Mt * Nt; e += blockDim.x) {
    const int mi = e / Nt, ni = e % Nt;
    const int m = P.m0 + mi, n = P.n0 + ni;
    T acc = T(0);
    if (A) {
      for (int k1 = 0; k1 < P.K1; ++k1) {
        T av = P.ta ? A[(int64_t)k1 * P.lda + m] : A[(int64_t)m * P.lda + k1];
        acc += av * Ts[k1 * Nt + ni];
      }
    } else {
      acc = Ts[mi * Nt + ni];
    }
    T* c = P.tc ? C + (int64_t)n * P.ldc + m : C + (int64_t)m * P.ldc + n;
    atomicAdd(c, alpha * acc);
  }
}

// Small sandwich, grouped by output block: one group of problems sharing the
// same C block per CTA, all roots in the CTA.  Per problem, A (M x K1) and B
// (K2 x N) are staged once in shared memory; per root X is staged, T = X B is
// formed, and alpha A T is accumulated into a shared-memory copy of the C
// block of that root.  After the group, the accumulators are added to C
// (atomic: several groups may share a C block).
template <typename T>
__global__ void __launch_bounds__(256) k_sandwich_small(const SProb* __restrict__ probs, const int* __restrict__ gstart,
                                                        const __grid_constant__ SysTable tab, int nroots, int dm,
                                                        int dk1, int dk2, int dn) {
  extern __shared__ unsigned char smem_raw[];
  T* As = reinterpret_cast<T*>(smem_raw);     // dm x dk1
  T* Bs = As + dm * dk1;                      // dk2 x dn
  T* Xs = Bs + dk2 * dn;                      // dk1 x dk2
  T* Ts = Xs + dk1 * dk2;                     // dk1 x dn
  T* Cs = Ts + dk1 * dn;                      // nroots x dm x dn accumulators
  const int g0 = gstart[blockIdx.x], g1 = gstart[blockIdx.x + 1];
  const SProb P0 = probs[g0];
  // this CTA's roots: [blockIdx.y * nroots, ...) (nroots = roots per CTA), within the system's vectors
  const int rbase = blockIdx.y * nroots;
  nroots = min(nroots, tab.s[P0.sys].nvec - rbase);
  if (nroots <= 0) return;
  const int M = P0.M, N = P0.N;
  for (int e = threadIdx.x; e < nroots * M * N; e += blockDim.x) Cs[e] = T(0);
  for (int g = g0; g < g1; ++g) {
    const SProb P = probs[g];
    const int K1 = P.K1, K2 = P.K2;
    const bool hasA = P.a_buf != B_NONE, hasB = P.b_buf != B_NONE;
    __syncthreads();
    if (hasA) {
      const T* A = cbuf<T>(tab, P.sys, P.a_buf, 0) + P.a_off;
      for (int e = threadIdx.x; e < M * K1; e += blockDim.x) {
        const int m = e / K1, k = e % K1;
        As[m * dk1 + k] = P.ta ? A[(int64_t)k * P.lda + m] : A[(int64_t)m * P.lda + k];
      }
    }
    if (hasB) {
      const T* Bm = cbuf<T>(tab, P.sys, P.b_buf, 0) + P.b_off;
      for (int e = threadIdx.x; e < K2 * N; e += blockDim.x) {
        const int k = e / N, n = e % N;
        Bs[k * dn + n] = P.tb ? Bm[(int64_t)n * P.ldb + k] : Bm[(int64_t)k * P.ldb + n];
      }
    }
    const T alpha = (T)P.alpha;
    for (int r = 0; r < nroots; ++r) {
      const T* X = cbuf<T>(tab, P.sys, P.x_buf, rbase + r) + P.x_off;
      __syncthreads();
      for (int e = threadIdx.x; e < K1 * K2; e += blockDim.x) {
        const int a = e / K2, b = e % K2;
        Xs[a * dk2 + b] = P.tx ? X[(int64_t)b * P.ldx + a] : X[(int64_t)a * P.ldx + b];
      }
      __syncthreads();
      if (hasB) {
        for (int e = threadIdx.x; e < K1 * N; e += blockDim.x) {
          const int a = e / N, n = e % N;
          T acc = T(0);
          for (int k = 0; k < K2; ++k) acc += Xs[a * dk2 + k] * Bs[k * dn + n];
          Ts[a * dn + n] = acc;
        }
        __syncthreads();
      }
      T* Cr = Cs + (size_t)r * M * N;
      for (int e = threadIdx.x; e < M * N; e += blockDim.x) {
        const int m = e / N, n = e % N;
        T acc = T(0);
        if (hasA) {
          if (hasB) for (int k = 0; k < K1; ++k) acc += As[m * dk1 + k] * Ts[k * dn + n];
          else for (int k = 0; k < K1; ++k) acc += As[m * dk1 + k] * Xs[k * dk2 + n];
        } else {
          acc = hasB ? Ts[m * dn + n] : Xs[m * dk2 + n];
        }
        Cr[e] += alpha * acc;
      }
    }
  }
  __syncthreads();
  for (int r = 0; r < nroots; ++r) {
    T* C = mbuf<T>(tab, P0.sys, P0.c_buf, rbase + r) + P0.c_off;
    const T* Cr = Cs + (size_t)r * M * N;
    for (int e = threadIdx.x; e < M * N; e += blockDim.x) {
      const int m = e / N, n = e % N;
      T* c = P0.tc ? C + (int64_t)n * P0.ldc + m : C + (int64_t)m * P0.ldc + n;
      atomicAdd(c, Cr[e]);
    }
  }
}

constexpr int VR = 8;   // roots per pass inside a GEMV CTA

// One (64-row, K-chunk) tile of one dense block per CTA (split-K, atomic
// accumulation).  The K-chunk of every root's input vector is staged in shared
// memory; each warp owns 8 rows and its lanes stride K, so the block rows are
// read from HBM once, coalesced, for all roots.
template <typename T>
__global__ void __launch_bounds__(256) k_gemv(const VProb* __restrict__ probs, const __grid_constant__ SysTable tab) {
  extern __shared__ unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);   // VR x GEMV_KC
  const VProb P = probs[blockIdx.x];
  const int nroots = tab.s[P.sys].nvec;
  const T* A = (const T*)tab.s[P.sys].pool + P.a_off;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const T alpha = (T)P.alpha;
  const int kl = P.klen;
  for (int r0 = 0; r0 < nroots; r0 += VR) {
    const int nr = min(VR, nroots - r0);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * kl; e += blockDim.x) {
      const int q = e / kl, kk = e % kl;
      int xk = P.k0 + kk;
      if (P.xvec_n > 0) xk = (xk % P.xvec_n) * P.xvec_n + xk / P.xvec_n;
      xs[q * GEMV_KC + kk] = cbuf<T>(tab, P.sys, P.x_buf, r0 + q)[P.x_off + (int64_t)xk * P.x_stride];
    }
    __syncthreads();
    for (int ml = warp; ml < 64; ml += 8) {
      const int m = P.m0 + ml;
      if (m >= P.M) break;
      const T* a = A + (int64_t)m * P.lda + P.k0;
      T acc[VR];
#pragma unroll
      for (int q = 0; q < VR; ++q) acc[q] = T(0);
      for (int kk = lane; kk < kl; kk += 32) {
        const T av = a[kk];
#pragma unroll
        for (int q = 0; q < VR; ++q) acc[q] += av * xs[q * GEMV_KC + kk];
      }
#pragma unroll
      for (int q = 0; q < VR; ++q) {
        T v = acc[q];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        acc[q] = v;
      }
      if (lane == 0) {
        int cm = m;
        if (P.cvec_n > 0) cm = (m % P.cvec_n) * P.cvec_n + m / P.cvec_n;
        for (int q = 0; q < nr; ++q)
          atomicAdd(mbuf<T>(tab, P.sys, P.c_buf, r0 + q) + P.c_off + (int64_t)cm * P.c_stride, alpha * acc[q]);
      }
    }
  }
}

}  // namespace

// The dynamic shared-memory limit of a kernel is one attribute per function
// and device for the whole process, so several host threads must agree on it:
// it is only ever raised, under one lock, to the largest size any launch needed.
static void ensure_dynamic_smem(const void* func, size_t smem) {
  if (smem <= 48 * 1024) return;
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> configured;
  int dev = 0;
  PN_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  size_t& conf = configured[{dev, func}];
  if (smem > conf) {
    PN_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    conf = smem;
  }
}

template <typename T>
void run_sandwich(const SProb* d_probs, int nprob, const SysTable& t, int smem_elems, cudaStream_t s) {
  if (nprob <= 0 || t.max_nvec <= 0) return;
  size_t smem = (size_t)smem_elems * sizeof(T);
  ensure_dynamic_smem((const void*)k_sandwich<T>, smem);
  k_sandwich<T><<<dim3(nprob, t.max_nvec), 256, smem, s>>>(d_probs, t);
  PN_CUDA(cudaGetLastError());
}

template <typename T>
void run_gemv(const VProb* d_probs, int nprob, const SysTable& t, cudaStream_t s) {
  if (nprob <= 0 || t.max_nvec <= 0) return;
  const size_t smem = (size_t)VR * GEMV_KC * sizeof(T);
  ensure_dynamic_smem((const void*)k_gemv<T>, smem);
  k_gemv<T><<<nprob, 256, smem, s>>>(d_probs, t);
  PN_CUDA(cudaGetLastError());
}

template <typename T>
void run_sandwich_small(const SProb* d_probs, const int* d_group_start, int ngroups, const SysTable& t, int dm, int dk1,
                        int dk2, int dn, int roots_per_cta, cudaStream_t s) {
  if (ngroups <= 0 || t.max_nvec <= 0) return;
  const size_t base = (size_t)(dm * dk1 + dk2 * dn + dk1 * dk2 + dk1 * dn) * sizeof(T);
  const size_t per_root = (size_t)dm * dn * sizeof(T);
  const size_t limit = 200 * 1024;
  PN_CHECK(base + per_root <= limit, PNOEOM_ERR_UNSUPPORTED, "PNO blocks too large for the grouped sandwich kernel");
  int rpc = std::max(1, std::min(roots_per_cta, t.max_nvec));
  rpc = (int)std::min<size_t>(rpc, (limit - base) / per_root);
  const size_t smem = base + (size_t)rpc * per_root;
  ensure_dynamic_smem((const void*)k_sandwich_small<T>, smem);
  const int ychunks = (t.max_nvec + rpc - 1) / rpc;
  k_sandwich_small<T><<<dim3(ngroups, ychunks), 256, smem, s>>>(d_probs, d_group_start, t, rpc, dm, dk1, dk2, dn);
  PN_CUDA(cudaGetLastError());
}

template void run_sandwich<double>(const SProb*, int, const SysTable&, int, cudaStream_t);
template void run_sandwich<float>(const SProb*, int, const SysTable&, int, cudaStream_t);
template void run_gemv<double>(const VProb*, int, const SysTable&, cudaStream_t);
template void run_gemv<float>(const VProb*, int, const SysTable&, cudaStream_t);
template void run_sandwich_small<double>(const SProb*, const int*, int, const SysTable&, int, int, int, int, int, cudaStream_t);
template void run_sandwich_small<float>(const SProb*, const int*, int, const SysTable&, int, int, int, int, int, cudaStream_t);

}  // namespace pnoeom
