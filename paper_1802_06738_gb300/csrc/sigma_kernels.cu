// Kernels of the sigma program (see sigma_prog.cuh).
#include "sigma_prog.cuh"

namespace pnoeom {
namespace {

template <typename T>
__device__ __forceinline__ const T* cbuf(const Buffers& b, int id, int r) {
  switch (id) {
    case B_POOL: return (const T*)b.pool;
    case B_RIN: return (const T*)b.rin + (int64_t)r * b.rin_stride;
    case B_WORK: return (const T*)b.work + (int64_t)r * b.work_stride;
    default: return (const T*)b.sout + (int64_t)r * b.sout_stride;
  }
}
template <typename T>
__device__ __forceinline__ T* mbuf(const Buffers& b, int id, int r) {
  return id == B_WORK ? (T*)b.work + (int64_t)r * b.work_stride : (T*)b.sout + (int64_t)r * b.sout_stride;
}

// One (problem, root) per CTA.  T_s = opX(X) * opB(B) restricted to the
// output tile's columns is formed in shared memory, then C_tile += alpha *
// opA(A)[tile rows] * T_s.  Accumulation into C is atomic because many
// problems share an output block.
template <typename T>
__global__ void __launch_bounds__(256) k_sandwich(const SProb* __restrict__ probs, Buffers bufs) {
  extern __shared__ unsigned char smem_raw[];
  T* Ts = reinterpret_cast<T*>(smem_raw);
  const SProb P = probs[blockIdx.x];
  const int r = blockIdx.y;
  const T* X = cbuf<T>(bufs, P.x_buf, r) + P.x_off;
  const T* A = P.a_buf == B_NONE ? nullptr : cbuf<T>(bufs, P.a_buf, r) + P.a_off;
  const T* Bm = P.b_buf == B_NONE ? nullptr : cbuf<T>(bufs, P.b_buf, r) + P.b_off;
  T* C = mbuf<T>(bufs, P.c_buf, r) + P.c_off;
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

constexpr int VR = 8;   // roots per pass inside a GEMV CTA

// One 64-row tile of one dense block per CTA; each warp owns 8 rows, lanes
// stride the K dimension (coalesced reads of the row-major block), and all
// roots are handled in the same pass so the block is read from HBM once.
template <typename T>
__global__ void __launch_bounds__(256) k_gemv(const VProb* __restrict__ probs, Buffers bufs, int nroots) {
  const VProb P = probs[blockIdx.x];
  const T* A = (const T*)bufs.pool + P.a_off;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const T alpha = (T)P.alpha;
  for (int r0 = 0; r0 < nroots; r0 += VR) {
    const int nr = min(VR, nroots - r0);
    for (int ml = warp; ml < 64; ml += 8) {
      const int m = P.m0 + ml;
      if (m >= P.M) break;
      const T* a = A + (int64_t)m * P.lda;
      T acc[VR];
#pragma unroll
      for (int q = 0; q < VR; ++q) acc[q] = T(0);
      for (int k = lane; k < P.K; k += 32) {
        const T av = a[k];
        int xk = k;
        if (P.xvec_n > 0) xk = (k % P.xvec_n) * P.xvec_n + k / P.xvec_n;
#pragma unroll
        for (int q = 0; q < VR; ++q)
          if (q < nr) acc[q] += av * cbuf<T>(bufs, P.x_buf, r0 + q)[P.x_off + (int64_t)xk * P.x_stride];
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
          atomicAdd(mbuf<T>(bufs, P.c_buf, r0 + q) + P.c_off + (int64_t)cm * P.c_stride, alpha * acc[q]);
      }
    }
  }
}

}  // namespace

template <typename T>
void run_sandwich(const SProb* d_probs, int nprob, int nroots, const Buffers& b, int smem_elems, cudaStream_t s) {
  if (nprob <= 0 || nroots <= 0) return;
  size_t smem = (size_t)smem_elems * sizeof(T);
  static thread_local size_t configured[2] = {0, 0};
  size_t& conf = configured[sizeof(T) == 8];
  if (smem > 48 * 1024 && smem > conf) {
    PN_CUDA(cudaFuncSetAttribute(k_sandwich<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    conf = smem;
  }
  for (int p0 = 0; p0 < nprob; p0 += 65535 * 16) {
    int n = std::min(nprob - p0, 65535 * 16);
    dim3 grid(n, nroots);
    k_sandwich<T><<<grid, 256, smem, s>>>(d_probs + p0, b);
  }
  PN_CUDA(cudaGetLastError());
}

template <typename T>
void run_gemv(const VProb* d_probs, int nprob, int nroots, const Buffers& b, cudaStream_t s) {
  if (nprob <= 0 || nroots <= 0) return;
  k_gemv<T><<<nprob, 256, 0, s>>>(d_probs, b, nroots);
  PN_CUDA(cudaGetLastError());
}

template void run_sandwich<double>(const SProb*, int, int, const Buffers&, int, cudaStream_t);
template void run_sandwich<float>(const SProb*, int, int, const Buffers&, int, cudaStream_t);
template void run_gemv<double>(const VProb*, int, int, const Buffers&, cudaStream_t);
template void run_gemv<float>(const VProb*, int, int, const Buffers&, cudaStream_t);

}  // namespace pnoeom
