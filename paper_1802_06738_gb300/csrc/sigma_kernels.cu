// Kernels of the sigma program (see sigma_prog.cuh).
#include <map>
#include <mutex>
#include "sigma_prog.cuh"
#include "tc.cuh"
#include <cuda_bf16.h>

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

// Element (a, b) of opX(X) + xb opX(X)^T (opX: X or X^T by tx; the xb term needs square X).
template <typename T>
__device__ __forceinline__ T xeff(const T* X, int ldx, int tx, T xb, int a, int b) {
  T v = tx ? X[(int64_t)b * ldx + a] : X[(int64_t)a * ldx + b];
  if (xb != T(0)) v += xb * (tx ? X[(int64_t)a * ldx + b] : X[(int64_t)b * ldx + a]);
  return v;
}

// One (problem, root) per CTA.  T_s = X_eff * opB(B) restricted to the
// output tile's columns is formed in shared memory, then C_tile += alpha *
// opA(A)[tile rows] * T_s.  Accumulation into C is atomic because many
// problems share an output block.  Used for blocks with a dim above SMALL_DIM.
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
  const T xb = (T)P.xb;
  const int Mt = min(64, P.M - P.m0), Nt = min(64, P.N - P.n0);
  // rows of T_s: K1 if A is present, else the tile's rows of X (K1 == M)
  const int trow0 = A ? 0 : P.m0;
  const int Tr = A ? P.K1 : Mt;
  for (int e = threadIdx.x; e < Tr * Nt; e += blockDim.x) {
    const int k1 = trow0 + e / Nt, n = P.n0 + e % Nt;
    T acc = T(0);
    if (Bm) {
      for (int k2 = 0; k2 < P.K2; ++k2) {
        T bv = P.tb ? Bm[(int64_t)n * P.ldb + k2] : Bm[(int64_t)k2 * P.ldb + n];
        acc += xeff(X, P.ldx, P.tx, xb, k1, k2) * bv;
      }
    } else {
      acc = xeff(X, P.ldx, P.tx, xb, k1, n);
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

// 16-byte shared-memory vectors of four elements
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 q0 = reinterpret_cast<const double2*>(p)[0], q1 = reinterpret_cast<const double2*>(p)[1];
  v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// floor(e / d) for 0 <= e, e + d < 2^22, given rd = 1.0f / d: (e + 1/2) / d lies at
// least 1/(2d) from an integer and the two roundings move it by less than that.
__device__ __forceinline__ int fdiv(int e, float rd) { return __float2int_rz(((float)e + 0.5f) * rd); }

__host__ __device__ constexpr int pad4(int x) { return (x + 3) & ~3; }

// Asynchronous global -> shared copy of one element (cp.async, no register round trip).
template <typename T>
__device__ __forceinline__ void cp_async_el(T* dst, const T* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(sizeof(T)));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Element stride between the per-vector copies of a buffer (0 for the shared pool).
__device__ __forceinline__ int64_t cvstride(const SysTable& t, int sys, int id) {
  const SysBuf& b = t.s[sys];
  switch (id) {
    case B_POOL: return 0;
    case B_RIN: return b.rin_stride;
    case B_WORK: return b.work_stride;
    default: return b.sout_stride;
  }
}

// Staging of nv blocks of R x Cn elements into shared memory with cp.async: element
// (v, r, c) is read at src[v * vs + r * rs + c * cs] and written to dst[v * dvs + r * dld + c].
// Thread t keeps column c = t % Cn and walks rows t / Cn, t / Cn + NT / Cn, ... of the nv
// blocks stacked, so the stores of a warp fall on consecutive words of shared memory (no
// bank conflicts between rows) and, where cs == 1, its loads on consecutive words of the
// source.  Needs 0 < Cn <= NT.
template <typename T, int NT>
__device__ __forceinline__ void stage_block(T* dst, int dvs, int dld, const T* src, int64_t vs, int rs, int cs,
                                            int nv, int R, int Cn, int tid) {
  if (R <= 0 || Cn <= 0) return;
  const int rstep = NT / Cn;
  const int rr = tid / Cn;
  if (rr >= rstep) return;   // the NT % Cn threads left over
  const int c = tid - rr * Cn;
  const int dv = rstep / R, dr = rstep - dv * R;
  int v = rr / R, r = rr - v * R;
  while (v < nv) {
    cp_async_el(dst + v * dvs + r * dld + c, src + v * vs + (r * rs + c * cs));
    r += dr;
    v += dv;
    if (r >= R) {
      r -= R;
      ++v;
    }
  }
}

// X_eff = opX(X) + xb opX(X)^T of nv square K x K blocks (element (a, b) of X_v at
// src[v * vs + a * ldx + b]), merged in registers: dst[v * dvs + b * dld + a] =
// opX(X_v)[a][b] + xb opX(X_v)[b][a], with opX(X)[a][b] = X[b][a] when tx.  Thread mapping
// as in stage_block, a fastest.
template <typename T, int NT>
__device__ __forceinline__ void stage_xeff_block(T* dst, int dvs, int dld, const T* src, int64_t vs, int ldx, bool tx,
                                                 T xb, int nv, int K, int tid) {
  if (K <= 0) return;
  const int rstep = NT / K;
  const int rr = tid / K;
  if (rr >= rstep) return;
  const int a = tid - rr * K;
  const int dv = rstep / K, dr = rstep - dv * K;
  int v = rr / K, b = rr - v * K;
  while (v < nv) {
    const T* X = src + v * vs;
    const T xba = X[b * ldx + a], xab = X[a * ldx + b];   // X[b][a], X[a][b]
    dst[v * dvs + b * dld + a] = tx ? xba + xb * xab : xab + xb * xba;
    b += dr;
    v += dv;
    if (b >= K) {
      b -= K;
      ++v;
    }
  }
}

// Grouped small sandwich (see run_sandwich_small).  Shared memory, with the set's
// bounds dm, dk1 (rows of the staged X block), dk2 (its columns), dn padded to 4,
// and NB copies (NB = 2: problem g and g + 1; NB = 1: one) of the staged operands:
//   As [dk1][Mp]        A^T (tile rows)
//   Bs [dk2][Np]        B (tile columns)
//   Xs [dk2][R * K1p]   opX(X)^T of the R vectors side by side (X_eff after the merge pass)
// and one copy of
//   Ts [K1p][R * Np]    alpha X_eff B of the R vectors side by side.
// With NB = 2 the operands of problem g + 1 are copied with cp.async while problem g
// computes; NB = 1 copies them at the start of each problem and needs half the staging
// memory (more CTAs per SM where the stacked X blocks are large).
// Product 1: Ts = alpha Xs^T Bs, rows (vector, a) x columns n, 4 x 4 register tiles.
// Product 2: C[m][(vector, n)] += As^T Ts, 4 x 4 register tiles that each thread
// keeps for the whole group (MAXT tiles per thread).
template <typename T, int NT, int MAXT, int NB>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? (NT == 128 ? 6 : (MAXT == 2 ? 3 : 2)) : 1) k_sandwich_small(const SProb* __restrict__ probs, const int* __restrict__ gstart,
                                                       const __grid_constant__ SysTable tab, int rpc, int dm, int dk1,
                                                       int dk2, int dn) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Mp = pad4(dm), K1p = pad4(dk1), Np = pad4(dn);
  const int xld = rpc * K1p, tld = rpc * Np;
  const int asz = dk1 * Mp, bsz = dk2 * Np, xsz = dk2 * xld;
  const int stage = asz + bsz + xsz;   // one copy of the staged operands (a multiple of 4)
  T* S0 = reinterpret_cast<T*>(smem_raw);
  T* Ts = S0 + NB * stage;
  const int total = NB * stage + K1p * tld;
  const int tid = threadIdx.x;
  const int g0 = gstart[blockIdx.x], g1 = gstart[blockIdx.x + 1];
  const SProb P0 = probs[g0];
  const int rbase = blockIdx.y * rpc;
  const int nr = min(rpc, tab.s[P0.sys].nvec - rbase);
  if (nr <= 0) return;
  const int Mt = min(64, P0.M - P0.m0), Nt = min(64, P0.N - P0.n0);
  const int nt4 = (Nt + 3) >> 2;
  const int nct = ((Mt + 3) >> 2) * nr * nt4;
  // padding is read (never stored) by the 4-wide tiles: keep it finite
  for (int e = tid; e < total; e += NT) S0[e] = T(0);
  // Product 2 register tiles: when there are fewer C tiles than threads, s2 lanes (a
  // power of two <= 8, adjacent lanes of one warp) share a tile, each summing every s2-th
  // k; their partial tiles are reduced once, after the group.
  int s2 = 1;
  while (s2 < 8 && nct * s2 * 2 <= NT) s2 *= 2;
  const int sl2 = tid & (s2 - 1);
  int cm4[MAXT], cr[MAXT], cn4[MAXT];
  T acc[MAXT][4][4];
#pragma unroll
  for (int j = 0; j < MAXT; ++j) {
    const int t = (tid + j * NT) / s2;
    cn4[j] = t % nt4;
    cr[j] = (t / nt4) % nr;
    cm4[j] = t / (nt4 * nr);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[j][a][b] = T(0);
  }
  // Staging (stage_block): A, B and (when xb == 0) X go through cp.async, every thread
  // taking elements of consecutive destination columns; X with xb != 0 is merged in
  // registers by stage_xeff.
  auto issue = [&](const SProb& P, int buf) {
    T* As = S0 + buf * stage;
    T* Bs = As + asz;
    T* Xs = Bs + bsz;
    const bool hasA = P.a_buf != B_NONE, hasB = P.b_buf != B_NONE;
    const int K1 = P.K1;
    const int kr = hasA ? K1 : Mt, kc = hasB ? P.K2 : Nt;
    const int xr0 = hasA ? 0 : P.m0, xc0 = hasB ? 0 : P.n0;
    if (hasA) {   // As[k][m] = opA(A)[m0 + m][k]; A stored K1 x M (ta) or M x K1
      const T* A = cbuf<T>(tab, P.sys, P.a_buf, 0) + P.a_off;
      if (P.ta)
        stage_block<T, NT>(As, 0, Mp, A + P.m0, 0, P.lda, 1, 1, K1, Mt, tid);
      else
        stage_block<T, NT>(As, 0, Mp, A + (int64_t)P.m0 * P.lda, 0, 1, P.lda, 1, K1, Mt, tid);
    }
    if (hasB) {   // Bs[k][n] = opB(B)[k][n0 + n]; B stored N x K2 (tb) or K2 x N
      const T* Bm = cbuf<T>(tab, P.sys, P.b_buf, 0) + P.b_off;
      if (P.tb)
        stage_block<T, NT>(Bs, 0, Np, Bm + (int64_t)P.n0 * P.ldb, 0, 1, P.ldb, 1, P.K2, Nt, tid);
      else
        stage_block<T, NT>(Bs, 0, Np, Bm + P.n0, 0, P.ldb, 1, 1, P.K2, Nt, tid);
    }
    if (P.xb == 0.0) {   // Xs[b][r K1p + a] = opX(X_r)[xr0 + a][xc0 + b]
      const T* X = cbuf<T>(tab, P.sys, P.x_buf, rbase) + P.x_off;
      const int64_t vs = cvstride(tab, P.sys, P.x_buf);
      if (P.tx)   // opX(X)[a][b] = X[b][a]
        stage_block<T, NT>(Xs, K1p, xld, X + (int64_t)xc0 * P.ldx + xr0, vs, P.ldx, 1, nr, kc, kr, tid);
      else        // opX(X)[a][b] = X[a][b]
        stage_block<T, NT>(Xs, K1p, xld, X + (int64_t)xr0 * P.ldx + xc0, vs, 1, P.ldx, nr, kc, kr, tid);
    }
    cp_async_commit();
  };
  // X_eff = opX(X) + xb opX(X)^T of a square block (xr0 = xc0 = 0, kr = kc).
  auto stage_xeff = [&](const SProb& P, T* Xs, int K) {
    stage_xeff_block<T, NT>(Xs, K1p, xld, cbuf<T>(tab, P.sys, P.x_buf, rbase) + P.x_off, cvstride(tab, P.sys, P.x_buf),
                            P.ldx, P.tx != 0, (T)P.xb, nr, K, tid);
  };
  if (NB == 2) {
    __syncthreads();   // zero fill done before the first copies land
    issue(P0, 0);
  }
  for (int g = g0; g < g1; ++g) {
    int buf = 0;
    if (NB == 2) {   // problem g was copied while g - 1 computed; start copying g + 1
      buf = (g - g0) & 1;
      cp_async_wait_all();
      __syncthreads();   // problem g staged; every thread is done with problem g - 1
      if (g + 1 < g1) issue(probs[g + 1], buf ^ 1);
    } else {         // one stage buffer: copy problem g now
      __syncthreads();   // every thread is done with problem g - 1 (and the zero fill)
      issue(probs[g], 0);
      cp_async_wait_all();
      __syncthreads();
    }
    const SProb P = probs[g];
    T* As = S0 + buf * stage;
    T* Bs = As + asz;
    T* Xs = Bs + bsz;
    const bool hasA = P.a_buf != B_NONE, hasB = P.b_buf != B_NONE;
    const int K1 = P.K1;
    const int kr = hasA ? K1 : Mt, kc = hasB ? P.K2 : Nt;
    const T alpha = (T)P.alpha, xb = (T)P.xb;
    if (xb != T(0)) {   // X_eff staged now, from registers
      stage_xeff(P, Xs, kr);
      __syncthreads();
    }
    {   // product 1: tiles (vector, a4, n4); s1 lanes share a tile over k when tiles are few
      const int ka4 = (kr + 3) >> 2;
      const int n1 = nr * ka4 * nt4;
      int s1 = 1;
      if (hasB)
        while (s1 < 8 && n1 * s1 * 2 <= NT) s1 *= 2;
      const int total1 = n1 * s1;
      const float rd_nt4 = 1.0f / (float)nt4, rd_ka4 = 1.0f / (float)ka4;
      for (int base = 0; base < total1; base += NT) {
        const int tt = base + tid;
        const bool valid = tt < total1;
        const int t = valid ? tt / s1 : 0, sl = tt & (s1 - 1);
        const int rest = fdiv(t, rd_nt4), n4 = t - rest * nt4;
        const int r = fdiv(rest, rd_ka4), a4 = rest - r * ka4;
        T c[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) c[a][b] = T(0);
        const T* xp = Xs + r * K1p + a4 * 4;
        if (hasB) {
          const T* bp = Bs + n4 * 4;
          if (valid)
            for (int b = sl; b < kc; b += s1) {
              T xv[4], bv[4];
              ld4(xp + b * xld, xv);
              ld4(bp + b * Np, bv);
#pragma unroll
              for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int q = 0; q < 4; ++q) c[a][q] += xv[a] * bv[q];
            }
          for (int off = 1; off < s1; off <<= 1)   // every lane of the warp takes part
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int q = 0; q < 4; ++q) c[a][q] += __shfl_xor_sync(0xffffffffu, c[a][q], off);
        } else if (valid) {   // T = X_eff on the tile's columns
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (n4 * 4 + q < kc) {
              T xv[4];
              ld4(xp + (n4 * 4 + q) * xld, xv);
#pragma unroll
              for (int a = 0; a < 4; ++a) c[a][q] = xv[a];
            }
        }
        if (valid && sl == 0) {
          T* tp = Ts + (a4 * 4) * tld + r * Np + n4 * 4;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            T o[4] = {alpha * c[a][0], alpha * c[a][1], alpha * c[a][2], alpha * c[a][3]};
            st4(tp + a * tld, o);
          }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < MAXT; ++j) {   // product 2, into the register tiles
      if (tid + j * NT >= nct * s2) continue;
      const T* tp = Ts + cr[j] * Np + cn4[j] * 4;
      if (hasA) {
        const T* ap = As + cm4[j] * 4;
        for (int k = sl2; k < K1; k += s2) {
          T av[4], tv[4];
          ld4(ap + k * Mp, av);
          ld4(tp + k * tld, tv);
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[j][a][q] += av[a] * tv[q];
        }
      } else if (sl2 == 0) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          T tv[4];
          ld4(tp + (cm4[j] * 4 + a) * tld, tv);
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[j][a][q] += tv[q];
        }
      }
    }
  }
  if (s2 > 1)   // one tile per thread here (nct * s2 <= NT): reduce the s2 partial tiles
    for (int off = 1; off < s2; off <<= 1)
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[0][a][q] += __shfl_xor_sync(0xffffffffu, acc[0][a][q], off);
  // one atomic add per element of the group's C tile (other groups may share it)
#pragma unroll
  for (int j = 0; j < MAXT; ++j) {
    if (tid + j * NT >= nct * s2 || sl2 != 0) continue;
    T* C = mbuf<T>(tab, P0.sys, P0.c_buf, rbase + cr[j]) + P0.c_off;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = cm4[j] * 4 + a, n = cn4[j] * 4 + q;
        if (m < Mt && n < Nt) {
          const int64_t gm = P0.m0 + m, gn = P0.n0 + n;
          atomicAdd(P0.tc ? C + gn * P0.ldc + gm : C + gm * P0.ldc + gn, acc[j][a][q]);
        }
      }
  }
}

// Batched grouped sandwich, for sets whose problems all have A and B: a CTA stages
// pb consecutive problems of its group at once (single stage buffer), forms T for all of
// them in one pass of product 1, and runs product 2 once over the concatenation of their
// K ranges: C[m][(vector, n)] += sum over the batch of A_p T_p = [A_1 .. A_pb][T_1; ..; T_pb].
// Shared memory (floats), K1p = pad4(dk1), with compact K offsets koff_p = sum of pad4(K1):
//   Xs [pb][dk2][R * K1p]   X_eff^T per problem
//   Bs [pb][dk2][Np]        B per problem
//   As [pb * K1p][Mp]       A^T of the batch, rows koff_p .. (pad rows zero)
//   Ts [pb * K1p][R * Np]   alpha_p X_eff B_p of the batch, rows koff_p ..
// Barriers per batch: two (after staging, after product 1), instead of two or three per
// problem.  Register tiles, split-K and staging are those of k_sandwich_small.
constexpr int PB_MAX = 4;
template <typename T, int NT, int MAXT>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? (NT == 128 ? 6 : (MAXT == 2 ? 3 : 2)) : 1)
    k_sandwich_batch(const SProb* __restrict__ probs, const int* __restrict__ gstart, const __grid_constant__ SysTable tab,
                     int rpc, int pb, int dm, int dk1, int dk2, int dn) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Mp = pad4(dm), K1p = pad4(dk1), Np = pad4(dn);
  const int xld = rpc * K1p, tld = rpc * Np;
  const int xsz = dk2 * xld, bsz = dk2 * Np;
  T* Xs0 = reinterpret_cast<T*>(smem_raw);
  T* Bs0 = Xs0 + pb * xsz;
  T* As = Bs0 + pb * bsz;
  T* Ts = As + pb * K1p * Mp;
  const int total = pb * (xsz + bsz + K1p * Mp + K1p * tld);
  const int tid = threadIdx.x;
  const int g0 = gstart[blockIdx.x], g1 = gstart[blockIdx.x + 1];
  const SProb P0 = probs[g0];
  const int rbase = blockIdx.y * rpc;
  const int nr = min(rpc, tab.s[P0.sys].nvec - rbase);
  if (nr <= 0) return;
  const int Mt = min(64, P0.M - P0.m0), Nt = min(64, P0.N - P0.n0);
  const int nt4 = (Nt + 3) >> 2;
  const int nct = ((Mt + 3) >> 2) * nr * nt4;
  for (int e = tid; e < total; e += NT) Xs0[e] = T(0);
  int s2 = 1;
  while (s2 < 8 && nct * s2 * 2 <= NT) s2 *= 2;
  const int sl2 = tid & (s2 - 1);
  int cm4[MAXT], cr[MAXT], cn4[MAXT];
  T acc[MAXT][4][4];
#pragma unroll
  for (int j = 0; j < MAXT; ++j) {
    const int t = (tid + j * NT) / s2;
    cn4[j] = t % nt4;
    cr[j] = (t / nt4) % nr;
    cm4[j] = t / (nt4 * nr);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[j][a][b] = T(0);
  }
  for (int gb = g0; gb < g1; gb += pb) {
    const int nb = min(pb, g1 - gb);
    int koff[PB_MAX + 1], t1off[PB_MAX + 1];
    koff[0] = 0;
    t1off[0] = 0;
#pragma unroll
    for (int q = 0; q < PB_MAX; ++q) {
      const int K1 = q < nb ? probs[gb + q].K1 : 0;
      koff[q + 1] = koff[q] + pad4(K1);
      t1off[q + 1] = t1off[q] + nr * ((K1 + 3) >> 2) * nt4;
    }
    __syncthreads();   // every thread is done with the previous batch
    for (int q = 0; q < nb; ++q) {   // staging
      const SProb& P = probs[gb + q];
      const int K1 = P.K1, K2 = P.K2;
      T* Xs = Xs0 + q * xsz;
      T* Bs = Bs0 + q * bsz;
      T* Aq = As + koff[q] * Mp;
      {   // Aq[k][m] = opA(A)[m0 + m][k]
        const T* A = cbuf<T>(tab, P.sys, P.a_buf, 0) + P.a_off;
        if (P.ta)
          stage_block<T, NT>(Aq, 0, Mp, A + P.m0, 0, P.lda, 1, 1, K1, Mt, tid);
        else
          stage_block<T, NT>(Aq, 0, Mp, A + (int64_t)P.m0 * P.lda, 0, 1, P.lda, 1, K1, Mt, tid);
        for (int e = tid; e < (pad4(K1) - K1) * Mp; e += NT) Aq[K1 * Mp + e] = T(0);   // K padding rows
      }
      {   // Bs[k][n] = opB(B)[k][n0 + n]
        const T* Bm = cbuf<T>(tab, P.sys, P.b_buf, 0) + P.b_off;
        if (P.tb)
          stage_block<T, NT>(Bs, 0, Np, Bm + (int64_t)P.n0 * P.ldb, 0, 1, P.ldb, 1, K2, Nt, tid);
        else
          stage_block<T, NT>(Bs, 0, Np, Bm + P.n0, 0, P.ldb, 1, 1, K2, Nt, tid);
      }
      const T* X = cbuf<T>(tab, P.sys, P.x_buf, rbase) + P.x_off;
      const int64_t vs = cvstride(tab, P.sys, P.x_buf);
      if (P.xb == 0.0) {   // Xs[b][r K1p + a] = opX(X_r)[a][b]
        if (P.tx)
          stage_block<T, NT>(Xs, K1p, xld, X, vs, P.ldx, 1, nr, K2, K1, tid);
        else
          stage_block<T, NT>(Xs, K1p, xld, X, vs, 1, P.ldx, nr, K2, K1, tid);
      } else {   // square X: X_eff = opX(X) + xb opX(X)^T, merged in registers
        stage_xeff_block<T, NT>(Xs, K1p, xld, X, vs, P.ldx, P.tx != 0, (T)P.xb, nr, K1, tid);
      }
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    {   // product 1 over the batch: tiles (problem, vector, a4, n4)
      const int n1 = t1off[nb];
      int s1 = 1;
      while (s1 < 8 && n1 * s1 * 2 <= NT) s1 *= 2;
      const int total1 = n1 * s1;
      const float rd_nt4 = 1.0f / (float)nt4;
      for (int base = 0; base < total1; base += NT) {
        const int tt = base + tid;
        const bool valid = tt < total1;
        const int t = valid ? tt / s1 : 0, sl = tt & (s1 - 1);
        int q = 0;
#pragma unroll
        for (int z = 1; z < PB_MAX; ++z) q += (z < nb && t >= t1off[z]) ? 1 : 0;
        const SProb& P = probs[gb + q];
        const int ka4 = (P.K1 + 3) >> 2;
        const int tl = t - t1off[q];
        const int rest = fdiv(tl, rd_nt4), n4 = tl - rest * nt4;
        const int r = rest / ka4, a4 = rest - r * ka4;
        T c[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) c[a][b] = T(0);
        const T* xp = Xs0 + q * xsz + r * K1p + a4 * 4;
        const T* bp = Bs0 + q * bsz + n4 * 4;
        if (valid)
          for (int b = sl; b < P.K2; b += s1) {
            T xv[4], bv[4];
            ld4(xp + b * xld, xv);
            ld4(bp + b * Np, bv);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int w = 0; w < 4; ++w) c[a][w] += xv[a] * bv[w];
          }
        for (int off = 1; off < s1; off <<= 1)
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int w = 0; w < 4; ++w) c[a][w] += __shfl_xor_sync(0xffffffffu, c[a][w], off);
        if (valid && sl == 0) {
          const T alpha = (T)P.alpha;
          T* tp = Ts + (koff[q] + a4 * 4) * tld + r * Np + n4 * 4;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            T o[4] = {alpha * c[a][0], alpha * c[a][1], alpha * c[a][2], alpha * c[a][3]};
            st4(tp + a * tld, o);
          }
        }
      }
    }
    __syncthreads();
    const int Ktot = koff[nb];
#pragma unroll
    for (int j = 0; j < MAXT; ++j) {   // product 2 over the concatenated K of the batch
      if (tid + j * NT >= nct * s2) continue;
      const T* tp = Ts + cr[j] * Np + cn4[j] * 4;
      const T* ap = As + cm4[j] * 4;
      for (int k = sl2; k < Ktot; k += s2) {
        T av[4], tv[4];
        ld4(ap + k * Mp, av);
        ld4(tp + k * tld, tv);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[j][a][w] += av[a] * tv[w];
      }
    }
  }
  if (s2 > 1)
    for (int off = 1; off < s2; off <<= 1)
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[0][a][w] += __shfl_xor_sync(0xffffffffu, acc[0][a][w], off);
#pragma unroll
  for (int j = 0; j < MAXT; ++j) {
    if (tid + j * NT >= nct * s2 || sl2 != 0) continue;
    T* C = mbuf<T>(tab, P0.sys, P0.c_buf, rbase + cr[j]) + P0.c_off;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int m = cm4[j] * 4 + a, n = cn4[j] * 4 + w;
        if (m < Mt && n < Nt) {
          const int64_t gm = P0.m0 + m, gn = P0.n0 + n;
          atomicAdd(P0.tc ? C + gn * P0.ldc + gm : C + gm * P0.ldc + gn, acc[j][a][w]);
        }
      }
  }
}

// Dense product tile: C[m0.., n0..] += alpha opA(A) opB(B) over K in [k0, k0 + klen).
// The tile is TM rows x BT columns, computed in passes of BT x BT with (BT/4)^2 threads
// and 4 x 4 register tiles, K staged in chunks of 16 (A^T and B in shared memory,
// zero-filled outside the operands).
template <typename T, int BT, int TM>
__global__ void __launch_bounds__((BT / 4) * (BT / 4)) k_dense(const DProb* __restrict__ probs,
                                                              const __grid_constant__ SysTable tab) {
  constexpr int NT = (BT / 4) * (BT / 4), KC = 16, LD = BT + 4;
  __shared__ __align__(16) T As[KC * LD];
  __shared__ __align__(16) T Bs[KC * LD];
  const DProb P = probs[blockIdx.x];
  const int r = blockIdx.y;
  if (r >= tab.s[P.sys].nvec) return;
  const T* A = cbuf<T>(tab, P.sys, P.a_buf, r) + P.a_off;
  const T* Bm = cbuf<T>(tab, P.sys, P.b_buf, r) + P.b_off;
  T* C = mbuf<T>(tab, P.sys, P.c_buf, r) + P.c_off;
  const T alpha = (T)P.alpha;
  const int Nt = min(BT, P.N - P.n0);
  const int tx = threadIdx.x % (BT / 4), ty = threadIdx.x / (BT / 4);
  for (int mh = 0; mh < TM; mh += BT) {
    const int m0 = P.m0 + mh;
    const int Mt = min(BT, P.M - m0);
    if (Mt <= 0) break;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int kk = 0; kk < P.klen; kk += KC) {
      const int kn = min(KC, P.klen - kk), kb = P.k0 + kk;
      __syncthreads();
      for (int e = threadIdx.x; e < KC * BT; e += NT) {
        int k, m;
        if (P.ta) { k = e / BT; m = e % BT; } else { m = e / KC; k = e % KC; }
        T v = T(0);
        if (k < kn && m < Mt)
          v = P.ta ? A[(int64_t)(kb + k) * P.lda + m0 + m] : A[(int64_t)(m0 + m) * P.lda + kb + k];
        As[k * LD + m] = v;
      }
      for (int e = threadIdx.x; e < KC * BT; e += NT) {
        int k, n;
        if (P.tb) { n = e / KC; k = e % KC; } else { k = e / BT; n = e % BT; }
        T v = T(0);
        if (k < kn && n < Nt)
          v = P.tb ? Bm[(int64_t)(P.n0 + n) * P.ldb + kb + k] : Bm[(int64_t)(kb + k) * P.ldb + P.n0 + n];
        Bs[k * LD + n] = v;
      }
      __syncthreads();
      for (int k = 0; k < kn; ++k) {
        T av[4], bv[4];
        ld4(As + k * LD + ty * 4, av);
        ld4(Bs + k * LD + tx * 4, bv);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int m = ty * 4 + a, n = tx * 4 + b;
        if (m < Mt && n < Nt) {
          const int64_t gm = m0 + m, gn = P.n0 + n;
          atomicAdd(P.tc ? C + gn * P.ldc + gm : C + gm * P.ldc + gn, alpha * acc[a][b]);
        }
      }
  }
}

// Dense product with a small output tile (at most 32 x 32) and a long K: one tile per
// CTA of 256 threads.  The 4 x 4 register tiles are fewer than the threads, so s lanes
// (a power of two, adjacent lanes of one warp) share a tile, each taking every s-th k of
// a shared-memory chunk; their partial tiles are reduced with shuffles at the end.
template <typename T>
__global__ void __launch_bounds__(256) k_dense_skinny(const DProb* __restrict__ probs,
                                                     const __grid_constant__ SysTable tab) {
  constexpr int NT = 256, KC = 64, LD = 36;
  __shared__ __align__(16) T As[KC * LD];   // A^T chunk: [k][m]
  __shared__ __align__(16) T Bs[KC * LD];   // B chunk:   [k][n]
  const DProb P = probs[blockIdx.x];
  const int r = blockIdx.y;
  if (r >= tab.s[P.sys].nvec) return;
  const T* A = cbuf<T>(tab, P.sys, P.a_buf, r) + P.a_off;
  const T* Bm = cbuf<T>(tab, P.sys, P.b_buf, r) + P.b_off;
  const int Mt = min(32, P.M - P.m0), Nt = min(32, P.N - P.n0);
  const int mt4 = (Mt + 3) >> 2, nt4 = (Nt + 3) >> 2, tiles = mt4 * nt4;
  int sp = 1;
  while (sp < 32 && tiles * sp * 2 <= NT) sp *= 2;
  const int tid = threadIdx.x, t = tid / sp, sl = tid & (sp - 1);
  const bool valid = t < tiles;
  const int m4 = valid ? t / nt4 : 0, n4 = valid ? t - m4 * nt4 : 0;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int kk = 0; kk < P.klen; kk += KC) {
    const int kn = min(KC, P.klen - kk), kb = P.k0 + kk;
    __syncthreads();
    for (int e = tid; e < KC * 32; e += NT) {
      int k, m;
      if (P.ta) { k = e >> 5; m = e & 31; } else { m = e / KC; k = e % KC; }
      T v = T(0);
      if (k < kn && m < Mt)
        v = P.ta ? A[(int64_t)(kb + k) * P.lda + P.m0 + m] : A[(int64_t)(P.m0 + m) * P.lda + kb + k];
      As[k * LD + m] = v;
    }
    for (int e = tid; e < KC * 32; e += NT) {
      int k, n;
      if (P.tb) { n = e / KC; k = e % KC; } else { k = e >> 5; n = e & 31; }
      T v = T(0);
      if (k < kn && n < Nt)
        v = P.tb ? Bm[(int64_t)(P.n0 + n) * P.ldb + kb + k] : Bm[(int64_t)(kb + k) * P.ldb + P.n0 + n];
      Bs[k * LD + n] = v;
    }
    __syncthreads();
    if (valid)
      for (int k = sl; k < kn; k += sp) {
        T av[4], bv[4];
        ld4(As + k * LD + m4 * 4, av);
        ld4(Bs + k * LD + n4 * 4, bv);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
      }
  }
  for (int off = 1; off < sp; off <<= 1)
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] += __shfl_xor_sync(0xffffffffu, acc[a][b], off);
  if (!valid || sl != 0) return;
  T* C = mbuf<T>(tab, P.sys, P.c_buf, r) + P.c_off;
  const T alpha = (T)P.alpha;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int m = m4 * 4 + a, n = n4 * 4 + b;
      if (m < Mt && n < Nt) {
        const int64_t gm = P.m0 + m, gn = P.n0 + n;
        atomicAdd(P.tc ? C + gn * P.ldc + gm : C + gm * P.ldc + gn, alpha * acc[a][b]);
      }
    }
}

// Device status word shared by the tensor-core kernels: bit 0 is set when an mbarrier
// wait ran out of its clock budget (the kernel then issues no further MMA, waits for the
// ones in flight, frees its TMEM and returns without writing its tile); bit 1 when that
// second wait ran out too and the TMEM columns were left allocated.  Read and cleared by
// pnoeom_device_status.
__device__ int g_tc_status = 0;

constexpr int TC_BM = 128, TC_BN = 64, TC_BK = 32;
constexpr int TC_STAGE = 2 * TC_BM * TC_BK + 2 * TC_BN * TC_BK;   // floats per pipeline stage
constexpr long long TC_WAIT_BUDGET = 2000000000LL;   // clock cycles (about one second)

// Dense product tile on the tensor cores (FP32 data, 3xTF32): C[m0.., n0..] += alpha
// opA(A) opB(B) over K in [k0, k0 + klen), a 128 x 64 tile per CTA of 128 threads.
// Per K chunk of 32 the threads stage A (128 x 32) and B^T (64 x 32) as hi and lo tf32
// parts in the K-major no-swizzle layout, with core matrices adjacent along M/N
// (SBO = 128 B, LBO = rows / 8 * 128 B); one thread issues hi*hi + hi*lo + lo*hi for the
// four K = 8 steps into the FP32 accumulator in TMEM (64 columns) and commits to the
// stage's mbarrier.  Two stages: the next chunk's global loads go to registers while the
// MMAs run.  The epilogue reads TMEM (warp w: lanes 32w..32w+31 = tile rows) and adds
// alpha * D to C.
__global__ void __launch_bounds__(128) k_dense_tc(const DProb* __restrict__ probs, const __grid_constant__ SysTable tab) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // per stage: A hi, A lo (128 x 32 each), B hi, B lo (64 x 32 each); stage b at b * TC_STAGE
  float* sAh = reinterpret_cast<float*>(smem_raw);
  float* sAl = sAh + TC_BM * TC_BK;
  float* sBh = sAl + TC_BM * TC_BK;
  float* sBl = sBh + TC_BN * TC_BK;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(reinterpret_cast<float*>(smem_raw) + 2 * TC_STAGE);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  const DProb P = probs[blockIdx.x];
  const int r = blockIdx.y;
  if (r >= tab.s[P.sys].nvec) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(tslot, TC_BN);
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    tc::mbar_init(mbar + 1, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const float* A = cbuf<float>(tab, P.sys, P.a_buf, r) + P.a_off;
  const float* Bm = cbuf<float>(tab, P.sys, P.b_buf, r) + P.b_off;
  const int Mt = min(TC_BM, P.M - P.m0), Nt = min(TC_BN, P.N - P.n0);
  constexpr uint32_t LBO_A = TC_BM / 8 * 128, LBO_B = TC_BN / 8 * 128, SBO = 128;
  constexpr uint32_t IDESC = tc::idesc_tf32(TC_BM, TC_BN);
  // Software pipeline over K chunks of 32: the global loads of chunk c + 1 are issued into
  // registers while the MMAs of chunk c run; two shared-memory stages, one mbarrier each
  // (the stage of chunk c is reused by chunk c + 2 once its MMAs have completed).
  const int nchunk = (P.klen + TC_BK - 1) / TC_BK;
  float ra[TC_BM * TC_BK / 4 / 128][4], rb[TC_BN * TC_BK / 4 / 128][4];
  auto load = [&](int c) {
    const int kb = P.k0 + c * TC_BK, kn = min(TC_BK, P.klen - c * TC_BK);
#pragma unroll
    for (int q = 0; q < TC_BM * TC_BK / 4 / 128; ++q) {
      const int e = tid + q * 128, m = e % TC_BM, k4 = e / TC_BM;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = k4 * 4 + j;
        ra[q][j] = (m < Mt && k < kn)
                       ? (P.ta ? A[(int64_t)(kb + k) * P.lda + P.m0 + m] : A[(int64_t)(P.m0 + m) * P.lda + kb + k])
                       : 0.f;
      }
    }
#pragma unroll
    for (int q = 0; q < TC_BN * TC_BK / 4 / 128; ++q) {
      const int e = tid + q * 128, n = e % TC_BN, k4 = e / TC_BN;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = k4 * 4 + j;
        rb[q][j] = (n < Nt && k < kn)
                       ? (P.tb ? Bm[(int64_t)(P.n0 + n) * P.ldb + kb + k] : Bm[(int64_t)(kb + k) * P.ldb + P.n0 + n])
                       : 0.f;
      }
    }
  };
  // Every thread polls the stage's mbarrier, and the CTA then agrees on the outcome
  // (__syncthreads_and), so a wait that runs out takes every thread down the same path.
  uint32_t parity[2] = {0u, 0u};
  bool ok = true;
  int issued = 0;   // chunks whose MMAs were issued and committed
  if (nchunk > 0) load(0);
  for (int c = 0; c < nchunk; ++c) {
    const int b = c & 1;
    if (c >= 2) {   // the MMAs of chunk c - 2 read stage b
      ok = __syncthreads_and(tc::mbar_wait_bounded(mbar + b, parity[b], TC_WAIT_BUDGET) ? 1 : 0) != 0;
      if (!ok) break;
      parity[b] ^= 1u;
    }
    float* Ah = sAh + b * TC_STAGE;
    float* Al = sAl + b * TC_STAGE;
    float* Bh = sBh + b * TC_STAGE;
    float* Bl = sBl + b * TC_STAGE;
#pragma unroll
    for (int q = 0; q < TC_BM * TC_BK / 4 / 128; ++q) {
      const int e = tid + q * 128, m = e % TC_BM, k4 = e / TC_BM;
      float h[4], l[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) tc::split_tf32(ra[q][j], h[j], l[j]);
      const uint32_t off = tc::kmajor_off(m, k4 * 4, LBO_A, SBO) / 4;
      st4(Ah + off, h);
      st4(Al + off, l);
    }
#pragma unroll
    for (int q = 0; q < TC_BN * TC_BK / 4 / 128; ++q) {
      const int e = tid + q * 128, n = e % TC_BN, k4 = e / TC_BN;
      float h[4], l[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) tc::split_tf32(rb[q][j], h[j], l[j]);
      const uint32_t off = tc::kmajor_off(n, k4 * 4, LBO_B, SBO) / 4;
      st4(Bh + off, h);
      st4(Bl + off, l);
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t ah = tc::smem_u32(Ah), al = tc::smem_u32(Al), bh = tc::smem_u32(Bh), bl = tc::smem_u32(Bl);
#pragma unroll
      for (int ks = 0; ks < TC_BK / 8; ++ks) {
        const uint32_t da = ks * 2 * LBO_A, db = ks * 2 * LBO_B;
        const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
        tc::mma_tf32(tmem, tc::sdesc(ah + da, LBO_A, SBO), tc::sdesc(bh + db, LBO_B, SBO), IDESC, acc);
        tc::mma_tf32(tmem, tc::sdesc(ah + da, LBO_A, SBO), tc::sdesc(bl + db, LBO_B, SBO), IDESC, 1u);
        tc::mma_tf32(tmem, tc::sdesc(al + da, LBO_A, SBO), tc::sdesc(bh + db, LBO_B, SBO), IDESC, 1u);
      }
      tc::mma_commit(mbar + b);
    }
    issued = c + 1;
    if (c + 1 < nchunk) load(c + 1);
  }
  // the last one or two chunks' MMAs (MMAs complete in issue order: waiting for the last
  // commit covers the earlier ones, but each barrier's phase is consumed to keep them paired)
  for (int c = max(0, issued - 2); c < issued && ok; ++c) {
    const int b = c & 1;
    ok = __syncthreads_and(tc::mbar_wait_bounded(mbar + b, parity[b], TC_WAIT_BUDGET) ? 1 : 0) != 0;
    if (ok) parity[b] ^= 1u;
  }
  bool release = true;
  if (!ok) {
    // A wait ran out: no further MMA was issued.  The MMAs already committed may still
    // write TMEM, so the last commit (which covers every earlier one) is waited for once
    // more before TMEM is released; if that wait runs out as well, the columns are kept
    // (bit 1) rather than released under a running MMA.
    const int last = issued - 1;
    release = last < 0 ||
              __syncthreads_and(tc::mbar_wait_bounded(mbar + (last & 1), parity[last & 1], TC_WAIT_BUDGET) ? 1 : 0) != 0;
    if (tid == 0) atomicOr(&g_tc_status, release ? 1 : 3);
  }
  tc::fence_after_sync();
  if (ok) {
    float* C = mbuf<float>(tab, P.sys, P.c_buf, r) + P.c_off;
    const float alpha = (float)P.alpha;
    const int m = warp * 32 + lane;
#pragma unroll
    for (int c16 = 0; c16 < TC_BN / 16; ++c16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c16 * 16), v);
      if (m < Mt) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = c16 * 16 + j;
          if (n < Nt) {
            const int64_t gm = P.m0 + m, gn = P.n0 + n;
            atomicAdd(P.tc ? C + gn * P.ldc + gm : C + gm * P.ldc + gn, alpha * v[j]);
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0 && release) tc::tmem_dealloc(tmem, TC_BN);
}

// Failure-detection self-test (no MMA, no TMEM): thread 0 initialises an mbarrier that
// expects one arrival, which nothing ever makes, and polls it for at most `budget`
// cycles; the wait therefore runs out, and the kernel records it exactly as a
// tensor-core kernel does (bit 0 of g_tc_status) and reports it in *out.
__global__ void k_wait_selftest(long long budget, int* out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
  __syncthreads();
  const bool ok = __syncthreads_and(tc::mbar_wait_bounded(&bar, 0u, budget) ? 1 : 0) != 0;
  if (threadIdx.x == 0) {
    if (!ok) atomicOr(&g_tc_status, 1);
    *out = ok ? 0 : 1;
  }
}

// Dense block times vectors, one (row range, K-chunk) tile of one block per CTA
// (split-K, atomic accumulation).  The K chunk of up to R vectors is staged in shared
// memory once per tile (zero beyond the block's K; each thread issues eight loads before it
// stores them); the tile's rows are taken in groups of GEMV_ROWS against it (the program
// builder makes one group per tile).  In a group each of the 8 warps owns
// GEMV_ROWS / 8 rows and its lanes read
// 16-byte vectors of consecutive columns, two column steps per iteration (16 loads in
// flight per lane), so each staged x vector is reused for every row of the warp; the partial sums
// stay in registers over the whole chunk and are reduced across the warp once, by a
// reduce-scatter over shuffles (each exchange halves the values a lane holds; lane l ends
// with the sums of flattened (row, vector) indices l * (rows x R / 32) + j).  The pool rows must
// start on 16-byte boundaries (block offsets and leading dimensions are multiples of 8
// elements).  TA is the pool's element type: the arithmetic type T, or bf16 for the BF16 copy.
template <typename TA> struct PoolVec;
template <> struct PoolVec<float> {
  static constexpr int N = 4;
  __device__ static void cvt(const uint4& q, float (&v)[4]) {
    v[0] = __uint_as_float(q.x); v[1] = __uint_as_float(q.y); v[2] = __uint_as_float(q.z); v[3] = __uint_as_float(q.w);
  }
};
template <> struct PoolVec<double> {
  static constexpr int N = 2;
  __device__ static void cvt(const uint4& q, double (&v)[2]) {
    v[0] = __hiloint2double((int)q.y, (int)q.x);
    v[1] = __hiloint2double((int)q.w, (int)q.z);
  }
};
template <> struct PoolVec<__nv_bfloat16> {
  static constexpr int N = 8;
  __device__ static void cvt(const uint4& q, float (&v)[8]) {
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[k]));
      v[2 * k] = f.x;
      v[2 * k + 1] = f.y;
    }
  }
};
constexpr int GEMV_WROWS = GEMV_ROWS / 8;   // rows per warp

// One exchange of the warp reduce-scatter over the first N of the lane's sums (N > 1: the
// lane keeps the upper half when bit sh of its index is set; N == 1: plain pairwise add).
template <typename T, int NV, int N>
__device__ __forceinline__ void gemv_rs_step(T (&acc)[NV], int lane, int sh) {
  if constexpr (N > 1) {
    const bool up = (lane >> sh) & 1;
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const T send = up ? acc[i] : acc[i + N / 2];
      const T keep = up ? acc[i + N / 2] : acc[i];
      acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, 1 << sh);
    }
  } else {
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1 << sh);
  }
}

template <typename T, typename TA, int R>
__device__ __forceinline__ void gemv_tile(const VProb& P, const SysTable& tab, T* xs) {
  constexpr int VEC = PoolVec<TA>::N;
  constexpr int NV = GEMV_WROWS * R;          // partial sums per lane
  constexpr int SL = 8;                       // staged x loads in flight per thread
  static_assert(NV % 32 == 0 || NV == 16, "reduce-scatter of 16 or a multiple of 32 sums");
  const int nroots = tab.s[P.sys].nvec;
  const TA* A = (const TA*)(sizeof(TA) == 2 ? tab.s[P.sys].pool16 : tab.s[P.sys].pool) + P.a_off;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kl = P.klen, klp = (kl + VEC - 1) / VEC * VEC;
  const T alpha = (T)P.alpha;
  for (int r0 = 0; r0 < nroots; r0 += R) {
    const int nr = min(R, nroots - r0);
    __syncthreads();
    // stage the K chunk of nr vectors: each thread issues SL independent loads before
    // it stores any of them
    const int tot = nr * klp;
    for (int base = threadIdx.x; base < tot; base += SL * blockDim.x) {
      T val[SL];
#pragma unroll
      for (int u = 0; u < SL; ++u) {
        const int idx = base + u * blockDim.x;
        val[u] = T(0);
        if (idx < tot) {
          const int q = idx / klp, kk = idx - q * klp;
          if (kk < kl) {
            int xk = P.k0 + kk;
            if (P.xvec_n > 0) xk = (xk % P.xvec_n) * P.xvec_n + xk / P.xvec_n;
            val[u] = cbuf<T>(tab, P.sys, P.x_buf, r0 + q)[P.x_off + (int64_t)xk * P.x_stride];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < SL; ++u) {
        const int idx = base + u * blockDim.x;
        if (idx < tot) {
          const int q = idx / klp;
          xs[q * GEMV_KC + (idx - q * klp)] = val[u];
        }
      }
    }
    __syncthreads();
    auto step = [&](int kk, const uint4 (&raw)[GEMV_WROWS], T (&acc)[NV]) {
      T a[GEMV_WROWS][VEC];
#pragma unroll
      for (int rr = 0; rr < GEMV_WROWS; ++rr) PoolVec<TA>::cvt(raw[rr], a[rr]);
      // each staged x value is read once and applied to every row of the warp
#pragma unroll
      for (int q = 0; q < R; ++q) {
        if (q < nr) {
          const T* xq = xs + q * GEMV_KC + kk;
#pragma unroll
          for (int w = 0; w < VEC; ++w) {
            const T xv = xq[w];
#pragma unroll
            for (int rr = 0; rr < GEMV_WROWS; ++rr) acc[rr * R + q] += a[rr][w] * xv;
          }
        }
      }
    };
    // row groups of the tile, all against the staged chunk; a warp skips a group in
    // which it has no rows (no barrier inside this loop)
    for (int g0 = warp * GEMV_WROWS; g0 < P.mlen; g0 += GEMV_ROWS) {
      const TA* arow[GEMV_WROWS];
      bool rv[GEMV_WROWS];
#pragma unroll
      for (int rr = 0; rr < GEMV_WROWS; ++rr) {
        rv[rr] = g0 + rr < P.mlen;
        arow[rr] = A + (int64_t)(P.m0 + (rv[rr] ? g0 + rr : 0)) * P.lda + P.k0;
      }
      T acc[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] = T(0);
      int kk = lane * VEC;
      for (; kk + 32 * VEC < klp; kk += 64 * VEC) {   // two column steps per iteration
        uint4 ra[GEMV_WROWS], rb[GEMV_WROWS];
#pragma unroll
        for (int rr = 0; rr < GEMV_WROWS; ++rr) {
          ra[rr] = rv[rr] ? *reinterpret_cast<const uint4*>(arow[rr] + kk) : make_uint4(0u, 0u, 0u, 0u);
          rb[rr] = rv[rr] ? *reinterpret_cast<const uint4*>(arow[rr] + kk + 32 * VEC) : make_uint4(0u, 0u, 0u, 0u);
        }
        step(kk, ra, acc);
        step(kk + 32 * VEC, rb, acc);
      }
      if (kk < klp) {
        uint4 ra[GEMV_WROWS];
#pragma unroll
        for (int rr = 0; rr < GEMV_WROWS; ++rr)
          ra[rr] = rv[rr] ? *reinterpret_cast<const uint4*>(arow[rr] + kk) : make_uint4(0u, 0u, 0u, 0u);
        step(kk, ra, acc);
      }
      // reduce-scatter across the warp: after the exchange at bit s a lane keeps the upper
      // half of its values when bit s of its lane index is set (16 sums: four exchanges, then
      // lanes 2l and 2l + 1 add their single values)
      constexpr int PER = NV >= 32 ? NV / 32 : 1;   // sums a lane ends with
      gemv_rs_step<T, NV, NV>(acc, lane, 4);
      gemv_rs_step<T, NV, (NV >= 2 ? NV / 2 : 1)>(acc, lane, 3);
      gemv_rs_step<T, NV, (NV >= 4 ? NV / 4 : 1)>(acc, lane, 2);
      gemv_rs_step<T, NV, (NV >= 8 ? NV / 8 : 1)>(acc, lane, 1);
      gemv_rs_step<T, NV, (NV >= 16 ? NV / 16 : 1)>(acc, lane, 0);
      const bool writer = NV >= 32 || (lane & (32 / NV - 1)) == 0;
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        const int idx = NV >= 32 ? lane * PER + j : lane / (32 / NV), rr = idx / R, q = idx % R;
        if (writer && q < nr && g0 + rr < P.mlen) {
          const int m = P.m0 + g0 + rr;
          int cm = m;
          if (P.cvec_n > 0) cm = (m % P.cvec_n) * P.cvec_n + m / P.cvec_n;
          atomicAdd(mbuf<T>(tab, P.sys, P.c_buf, r0 + q) + P.c_off + (int64_t)cm * P.c_stride, alpha * acc[j]);
        }
      }
    }
  }
}

template <typename T, int R>
__global__ void __launch_bounds__(256) k_gemv(const VProb* __restrict__ probs, const __grid_constant__ SysTable tab) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);   // R x GEMV_KC
  const VProb P = probs[blockIdx.x];
  if constexpr (sizeof(T) == 4) {
    if (tab.s[P.sys].pool16) gemv_tile<float, __nv_bfloat16, R>(P, tab, xs);
    else gemv_tile<float, float, R>(P, tab, xs);
  } else {
    gemv_tile<T, T, R>(P, tab, xs);
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
  constexpr int R = sizeof(T) == 4 ? 8 : 4;
  const size_t smem = (size_t)R * GEMV_KC * sizeof(T);
  ensure_dynamic_smem((const void*)k_gemv<T, R>, smem);
  k_gemv<T, R><<<nprob, 256, smem, s>>>(d_probs, t);
  PN_CUDA(cudaGetLastError());
}

template <typename T, int NT, int MAXT, int NB>
static void launch_small_nb(const SProb* d_probs, const int* d_group_start, int ngroups, const SysTable& t, int dm,
                            int dk1, int dk2, int dn, int rpc, size_t smem, cudaStream_t s) {
  ensure_dynamic_smem((const void*)k_sandwich_small<T, NT, MAXT, NB>, smem);
  const int ychunks = (t.max_nvec + rpc - 1) / rpc;
  k_sandwich_small<T, NT, MAXT, NB>
      <<<dim3(ngroups, ychunks), NT, smem, s>>>(d_probs, d_group_start, t, rpc, dm, dk1, dk2, dn);
  PN_CUDA(cudaGetLastError());
}

template <typename T, int NT, int MAXT>
static void launch_small(const SProb* d_probs, const int* d_group_start, int ngroups, const SysTable& t, int dm, int dk1,
                         int dk2, int dn, int rpc, int nbsel, cudaStream_t s) {
  const int Mp = pad4(dm), K1p = pad4(dk1), Np = pad4(dn);
  // C register tiles per vector: rows/4 x cols/4; at most NT * MAXT per CTA
  const int tiles = (Mp / 4) * (Np / 4);
  rpc = std::max(1, std::min(rpc, std::min(t.max_nvec, NT * MAXT / tiles)));
  auto smem_of = [&](int r, int nb) {
    return (size_t)(nb * (dk1 * Mp + dk2 * Np + dk2 * r * K1p) + K1p * r * Np) * sizeof(T);
  };
  const size_t limit = 200 * 1024, two_per_sm = 113 * 1024;
  // stage buffers: the tuned choice (nbsel 1 or 2) if given, else double buffering unless
  // only single buffering leaves room for two CTAs per SM
  int nb = (smem_of(rpc, 2) > two_per_sm && smem_of(rpc, 1) <= two_per_sm) ? 1 : 2;
  if (nbsel == 1 || nbsel == 2) nb = nbsel;
  while (rpc > 1 && smem_of(rpc, nb) > limit) --rpc;
  if (nb == 2 && smem_of(rpc, 2) > limit) nb = 1;   // the tuned double buffering does not fit (FP64)
  PN_CHECK(smem_of(rpc, nb) <= limit && tiles <= NT * MAXT, PNOEOM_ERR_UNSUPPORTED,
           "PNO blocks too large for the grouped sandwich kernel");
  if (nb == 2)
    launch_small_nb<T, NT, MAXT, 2>(d_probs, d_group_start, ngroups, t, dm, dk1, dk2, dn, rpc, smem_of(rpc, 2), s);
  else
    launch_small_nb<T, NT, MAXT, 1>(d_probs, d_group_start, ngroups, t, dm, dk1, dk2, dn, rpc, smem_of(rpc, 1), s);
}

template <typename T, int NT, int MAXT>
static bool launch_batch(const SProb* d_probs, const int* d_group_start, int ngroups, const SysTable& t, int dm, int dk1,
                         int dk2, int dn, int rpc, int pb, cudaStream_t s) {
  const int Mp = pad4(dm), K1p = pad4(dk1), Np = pad4(dn);
  const int tiles = (Mp / 4) * (Np / 4);
  rpc = std::max(1, std::min(rpc, std::min(t.max_nvec, NT * MAXT / tiles)));
  auto smem_of = [&](int r, int b) {
    return (size_t)b * (size_t)(dk2 * r * K1p + dk2 * Np + K1p * Mp + K1p * r * Np) * sizeof(T);
  };
  const size_t limit = 200 * 1024;
  while (pb > 1 && smem_of(rpc, pb) > limit) --pb;
  while (rpc > 1 && smem_of(rpc, pb) > limit) --rpc;
  if (pb < 2 || smem_of(rpc, pb) > limit || tiles > NT * MAXT) return false;
  const size_t smem = smem_of(rpc, pb);
  ensure_dynamic_smem((const void*)k_sandwich_batch<T, NT, MAXT>, smem);
  const int ychunks = (t.max_nvec + rpc - 1) / rpc;
  k_sandwich_batch<T, NT, MAXT>
      <<<dim3(ngroups, ychunks), NT, smem, s>>>(d_probs, d_group_start, t, rpc, pb, dm, dk1, dk2, dn);
  PN_CUDA(cudaGetLastError());
  return true;
}

template <typename T>
void run_sandwich_small(const SProb* d_probs, const int* d_group_start, int ngroups, const SysTable& t, int dm, int dk1,
                        int dk2, int dn, int roots_per_cta, int pb, int nbsel, int shape, cudaStream_t s) {
  if (ngroups <= 0 || t.max_nvec <= 0) return;
  const int big = std::max(std::max(dm, dn), std::max(dk1, dk2));
  PN_CHECK(big <= SMALL_DIM, PNOEOM_ERR_UNSUPPORTED, "block too large for the grouped sandwich kernel");
  pb = std::min(pb, PB_MAX);
  if (pb > 1) {   // every problem has A and B: batched variant
    bool done;
    if (big <= 16)
      done = launch_batch<T, 128, 2>(d_probs, d_group_start, ngroups, t, dm, dk1, dk2, dn, roots_per_cta, pb, s);
    else if (big <= 32 || sizeof(T) == 8)
      done = launch_batch<T, 256, 2>(d_probs, d_group_start, ngroups, t, dm, dk1, dk2, dn, roots_per_cta, pb, s);
    else
      done = launch_batch<T, 256, 4>(d_probs, d_group_start, ngroups, t, dm, dk1, dk2, dn, roots_per_cta, pb, s);
    if (done) return;
  }
  // CTA shape: 1 = 128 threads x 2 tiles, 2 = 256 x 2, 3 = 256 x 4 (FP32 only); 0 = by bucket
  int sh = shape;
  if (sh == 3 && sizeof(T) == 8) sh = 2;
  if (sh < 1 || sh > 3) sh = big <= 16 ? 1 : (big <= 32 || sizeof(T) == 8) ? 2 : 3;
  const int tiles = (pad4(dm) / 4) * (pad4(dn) / 4);
  if (sh == 1 && tiles > 128 * 2) sh = 2;
  if (sh == 2 && tiles > 256 * 2) sh = sizeof(T) == 8 ? 2 : 3;
  if (sh == 1)
    launch_small<T, 128, 2>(d_probs, d_group_start, ngroups, t, dm, dk1, dk2, dn, roots_per_cta, nbsel, s);
  else if (sh == 2)
    launch_small<T, 256, 2>(d_probs, d_group_start, ngroups, t, dm, dk1, dk2, dn, roots_per_cta, nbsel, s);
  else
    launch_small<T, 256, 4>(d_probs, d_group_start, ngroups, t, dm, dk1, dk2, dn, roots_per_cta, nbsel, s);
}

template <typename T>
void run_dense(const DProb* d_probs, int nprob, const SysTable& t, int tile, cudaStream_t s) {
  if (nprob <= 0 || t.max_nvec <= 0) return;
  if (tile == DENSE_TILE_TC) {   // 128 x 64 tiles: tensor cores in FP32, two 64 x 64 halves in FP64
    if (sizeof(T) == 4) {
      const size_t smem = (size_t)(2 * TC_STAGE) * sizeof(float) + 32;
      ensure_dynamic_smem((const void*)k_dense_tc, smem);
      k_dense_tc<<<dim3(nprob, t.max_nvec), 128, smem, s>>>(d_probs, t);
    } else {
      k_dense<T, 64, 128><<<dim3(nprob, t.max_nvec), 256, 0, s>>>(d_probs, t);
    }
  } else {   // tiles of at most 32 x 32: one per CTA, K split over the spare lanes
    k_dense_skinny<T><<<dim3(nprob, t.max_nvec), 256, 0, s>>>(d_probs, t);
  }
  PN_CUDA(cudaGetLastError());
}

int selftest_bounded_wait(long long budget, cudaStream_t s) {
  DBuf<int> out(1);
  k_wait_selftest<<<1, 32, 0, s>>>(budget, out.get());
  PN_CUDA(cudaGetLastError());
  int v = 0;
  out.download(&v, 1, s);
  PN_CUDA(cudaStreamSynchronize(s));
  return v;
}

int device_status(bool clear, cudaStream_t s) {
  int v = 0;
  PN_CUDA(cudaMemcpyFromSymbolAsync(&v, g_tc_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  PN_CUDA(cudaStreamSynchronize(s));
  if (clear && v) {
    const int z = 0;
    PN_CUDA(cudaMemcpyToSymbolAsync(g_tc_status, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    PN_CUDA(cudaStreamSynchronize(s));
  }
  return v | tcs_status(clear, s);
}

template void run_sandwich<double>(const SProb*, int, const SysTable&, int, cudaStream_t);
template void run_sandwich<float>(const SProb*, int, const SysTable&, int, cudaStream_t);
template void run_gemv<double>(const VProb*, int, const SysTable&, cudaStream_t);
template void run_gemv<float>(const VProb*, int, const SysTable&, cudaStream_t);
template void run_sandwich_small<double>(const SProb*, const int*, int, const SysTable&, int, int, int, int, int, int,
                                        int, int, cudaStream_t);
template void run_sandwich_small<float>(const SProb*, const int*, int, const SysTable&, int, int, int, int, int, int,
                                       int, int, cudaStream_t);
template void run_dense<double>(const DProb*, int, const SysTable&, int, cudaStream_t);
template void run_dense<float>(const DProb*, int, const SysTable&, int, cudaStream_t);

}  // namespace pnoeom

namespace pnoeom {
// C (M x N, row-major, ldc = N) += alpha A (M x K, row-major) B (K x N, row-major), FP32
// device buffers, through the tensor-core dense tile kernel of the sigma program.
void gemm_tf32x3(const float* A, const float* B, float* C, int M, int N, int K, float alpha, cudaStream_t s) {
  PN_CHECK(M >= 0 && N >= 0 && K >= 0 && (M == 0 || N == 0 || K == 0 || (A && B && C)), PNOEOM_ERR_INVALID_ARG,
           "bad GEMM arguments");
  if (M == 0 || N == 0 || K == 0) return;
  std::vector<DProb> h;
  for (int m0 = 0; m0 < M; m0 += TC_BM)
    for (int n0 = 0; n0 < N; n0 += TC_BN) {
      DProb q{};
      q.a_buf = B_POOL; q.b_buf = B_RIN; q.c_buf = B_SOUT;
      q.M = M; q.N = N; q.K = K;
      q.lda = K; q.ldb = N; q.ldc = N;
      q.m0 = m0; q.n0 = n0; q.k0 = 0; q.klen = K;
      q.tile_m = TC_BM; q.tile_n = TC_BN; q.alpha = alpha;
      h.push_back(q);
    }
  DBuf<DProb> d(h.size());
  d.upload(h.data(), h.size(), s);
  SysTable t{};
  t.nsys = 1;
  t.max_nvec = 1;
  t.s[0].pool = A;
  t.s[0].rin = B;
  t.s[0].sout = C;
  t.s[0].nvec = 1;
  run_dense<float>(d.get(), (int)h.size(), t, DENSE_TILE_TC, s);
  PN_CUDA(cudaStreamSynchronize(s));
}
}  // namespace pnoeom
