// Sandwich terms of the sigma vector on the fifth-generation tensor cores (Sec. 2: the
// ring, Fock and occupied-ladder terms of sigma_2, each a product
//     sigma^{ij} += A * (sN X + sT X^T) * B,
// with A and B built from PNO overlaps S(ij,kl) and projected integral blocks, X a pair
// block R^{kl} of the trial vector, all in PNO bases).
//
// Output pair blocks are packed into bins of at most 128 rows (sigma_prog.cuh).  One CTA
// takes one bin and one vector and runs the bin's rounds; a round takes one vector block
// X and at most one term per output block (slot):
//   GEMM1  D1 = [A_t by slot] [X; X^T]^T     (M = 128, N = 2 nk; BF16 operands, FP32 in TMEM)
//   T      = sN D1[:, :nk] + sT D1[:, nk:]   per row, with that row's slot coefficients
//   GEMM2  D2 += T [B_t^T by slot]^T         (M = 128, N = bin rows, K = nk)
// D2 stays in TMEM over the rounds; its diagonal slot blocks are added to the output at
// the end.  Warp 4 streams each round's operand images (built once at setup from the
// FP64 pool; the X images once per call by k_tcs_pack_x) into a shared-memory ring with
// cp.async.bulk, up to TCS_NSLOT rounds ahead; lane 0 of warp 5 issues the MMAs; warps 0-3
// form T (TMEM -> registers -> BF16 -> shared memory).  GEMM1 of round r + 1 and GEMM2 of
// round r - 1 overlap the forming of T for round r (two TMEM column buffers, two T tiles).
// Every wait is bounded; a wait that runs out sets an abort flag, every role stops, the
// CTA drains what it issued and records bit 0 (bit 1 as well when TMEM had to be kept) of
// the status word read by pnoeom_device_status.
#include "pno.cuh"
#include "tc.cuh"
#include <cuda_bf16.h>
#include <algorithm>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <functional>
#include <map>
#include <unordered_map>
#include <vector>

namespace pnoeom {
namespace {

__device__ int g_tcs_status = 0;
// Tracing (PNOEOM_TCS_TRACE): when non-NULL, CTA (0, 0) records clock64() stamps per round:
// [8 r + 0] copy warp armed the stage; [+1] MMA lane saw it land; [+2] GEMM1 issued; [+3] T
// forming starts; [+4] T formed; [+5] GEMM2 issued; [+6] copy warp had the record; [+7]
// copy warp had the ring area.
__device__ long long* g_tcs_trace = nullptr;
constexpr int TCS_TRACE_ROUNDS = 4096;
constexpr long long TCS_WAIT_BUDGET = 2000000000LL;   // clock cycles (about one second)
constexpr int TCS_KMAX = (TCS_MAXN + 15) / 16 * 16;  // largest K of a round
constexpr int TCS_TBUF = TCS_ROWS * TCS_KMAX * 2;    // one T tile
constexpr int TCS_SMEM = 227 * 1024;
constexpr int TCS_DQ = 16;                            // round records prefetched ahead
constexpr int TCS_RING = (TCS_SMEM - 2 * TCS_TBUF - TCS_NSLOT * TCS_HDR - TCS_DQ * (int)sizeof(TcsRec) - 1024) / 1024 * 1024;
constexpr uint32_t TCS_D2_COL = 512 - TCS_ROWS;     // TMEM column of D2 (bin rows <= 128 columns)
constexpr int TCS_MAXD1 = 4;                         // GEMM1 buffers: as many as fit below D2, at most 4
static_assert(TCS_D2_COL >= 2 * 2 * TCS_KMAX, "TMEM budget: two GEMM1 buffers of the largest K");
// largest round area (a single vector block of K = TCS_KMAX with 128-row tiles must fit), and
// the ring holds at least two of them
static_assert((2 * TCS_ROWS + 2 * TCS_KMAX) * TCS_KMAX * 2 <= TCS_MAX_AREA, "round area");
static_assert(2 * TCS_MAX_AREA <= TCS_RING, "ring must hold two rounds");

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(tc::smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tc::smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   tc::smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
               : "memory");
}

// Bounded wait that also gives up when another thread has already set the abort flag.
__device__ __forceinline__ bool tcs_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (tc::mbar_test_wait(bar, parity)) return true;   // the common case: no suspension, no clock read
  const long long t0 = clock64();
  while (!tc::mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > TCS_WAIT_BUDGET) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}
// Bounded wait that ignores the abort flag (drains).
__device__ __forceinline__ bool tcs_drain(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!tc::mbar_try_wait(bar, parity))
    if (clock64() - t0 > TCS_WAIT_BUDGET) return false;
  return true;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// byte offset of element (r, k) in an M-outer image with K16 columns
__host__ __device__ __forceinline__ uint32_t img_off_bytes(int r, int k, int K16) {
  return (uint32_t)(r >> 3) * (uint32_t)(K16 * 16) + (uint32_t)(k >> 3) * 128u + (uint32_t)(r & 7) * 16u +
         (uint32_t)(k & 7) * 2u;
}

// The two-variant X image of every stored vector block, per vector: block q (vector
// offset xblk[3q], n = xblk[3q + 1]) goes to xblk[3q + 2]; rows a < n16 hold X[a, :], rows
// n16 + a hold X[:, a] (K = n16, zero padding).  Grid (blocks, vectors).
__global__ void __launch_bounds__(128) k_tcs_pack_x(const int64_t* __restrict__ xblk, const __grid_constant__ SysTable tab) {
  const int q = blockIdx.x, v = blockIdx.y;
  const SysBuf& SB = tab.s[0];
  if (v >= SB.nvec) return;
  const int n = (int)xblk[3 * q + 1];
  const int n16 = (n + 15) & ~15;
  const float* X = reinterpret_cast<const float*>(SB.rin) + (int64_t)v * SB.rin_stride + xblk[3 * q];
  unsigned char* dst = reinterpret_cast<unsigned char*>(SB.ximg) + ((int64_t)v * SB.ximg_stride + xblk[3 * q + 2]) * 2;
  const int chunks = 2 * n16 * (n16 / 8);
  for (int e = threadIdx.x; e < chunks; e += blockDim.x) {
    const int row = e % (2 * n16), k8 = e / (2 * n16);
    const int a = row < n16 ? row : row - n16;
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = k8 * 8 + j;
      x[j] = (a < n && k < n) ? (row < n16 ? X[(int64_t)a * n + k] : X[(int64_t)k * n + a]) : 0.f;
    }
    uint4 w;
    w.x = pack_bf16x2(x[0], x[1]);
    w.y = pack_bf16x2(x[2], x[3]);
    w.z = pack_bf16x2(x[4], x[5]);
    w.w = pack_bf16x2(x[6], x[7]);
    *reinterpret_cast<uint4*>(dst + img_off_bytes(row, k8 * 8, n16)) = w;
  }
}

// Setup: image i from the FP64 pool, desc[6 i ..] = {src, ld, trans, rows, K, dst};
// element (r, k) = trans ? pool[src + k ld + r] : pool[src + r ld + k].
__global__ void __launch_bounds__(128) k_tcs_make_img(const double* __restrict__ pool, __nv_bfloat16* __restrict__ img,
                                                      const int64_t* __restrict__ desc) {
  const int64_t* d = desc + 6 * (int64_t)blockIdx.x;
  const int64_t src = d[0], dst = d[5];
  const int ld = (int)d[1], trans = (int)d[2], rows = (int)d[3], K = (int)d[4];
  const int R16 = (rows + 15) & ~15, K16 = (K + 15) & ~15;
  unsigned char* out = reinterpret_cast<unsigned char*>(img + dst);
  for (int e = threadIdx.x; e < R16 * (K16 / 8); e += blockDim.x) {
    const int k8 = e % (K16 / 8), r = e / (K16 / 8);
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = k8 * 8 + j;
      x[j] = (r < rows && k < K) ? (float)(trans ? pool[src + (int64_t)k * ld + r] : pool[src + (int64_t)r * ld + k]) : 0.f;
    }
    uint4 w;
    w.x = pack_bf16x2(x[0], x[1]);
    w.y = pack_bf16x2(x[2], x[3]);
    w.z = pack_bf16x2(x[4], x[5]);
    w.w = pack_bf16x2(x[6], x[7]);
    *reinterpret_cast<uint4*>(out + img_off_bytes(r, k8 * 8, K16)) = w;
  }
}

// Round header in shared memory (written by the copy warp): start of the round's area in
// the ring, its sub-blocks (K, GEMM1 columns, T columns, tile offset, mask of slots with a
// term, per-slot coefficients) and the columns of T.
struct SubHdr {
  int nk16, dc, tk;
  uint32_t a_off, b_off, x_off, mask;
  float sN[TCS_MAXSLOTS];
  float sT[TCS_MAXSLOTS];
};
struct RoundHdr {
  uint32_t start;
  int nsub, ktot, pad;
  SubHdr sub[TCS_MAXSUB];
};
static_assert(sizeof(RoundHdr) <= TCS_HDR, "round header");

__global__ void __launch_bounds__(TCS_THREADS, 1)
    k_sandwich_tc(const TcsJob* __restrict__ jobs, const TcsSlot* __restrict__ slots, const TcsRec* __restrict__ recs,
                  const __grid_constant__ SysTable tab) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* ring = sm;
  unsigned char* tbuf = sm + TCS_RING;
  RoundHdr* hdr = reinterpret_cast<RoundHdr*>(tbuf + 2 * TCS_TBUF);
  TcsRec* dq = reinterpret_cast<TcsRec*>(reinterpret_cast<unsigned char*>(hdr) + TCS_NSLOT * TCS_HDR);
  uint64_t* bars = reinterpret_cast<uint64_t*>(dq + TCS_DQ);
  uint64_t* full = bars;                     // [NSLOT] a round's images landed
  uint64_t* empty = bars + TCS_NSLOT;        // [NSLOT] the round's GEMM2 completed (its ring area is free)
  uint64_t* g1 = bars + 2 * TCS_NSLOT;       // [TCS_MAXD1] GEMM1 into D1 buffer b completed
  uint64_t* tready = g1 + TCS_MAXD1;         // [2] T tile b formed (one arrival per T-forming thread)
  uint64_t* d1free = tready + 2;             // [TCS_MAXD1] D1 buffer read out by the T-forming warps
  uint64_t* dqb = d1free + TCS_MAXD1;        // [2] half h of the record queue (TCS_DQ / 2 records) landed
  uint32_t* misc = reinterpret_cast<uint32_t*>(dqb + 2);
  // misc: [0] TMEM base, [1] abort flag, [2] keep-TMEM flag
  volatile int* abort_flag = reinterpret_cast<volatile int*>(misc + 1);
  volatile int* keep_tmem = reinterpret_cast<volatile int*>(misc + 2);

  const TcsJob J = jobs[blockIdx.x];
  const int v = blockIdx.y;
  const SysBuf& SB = tab.s[J.sys];
  if (v >= SB.nvec) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // rows of slots without a term in a round keep older images: finite, never uninitialised
  for (int e = tid; e < TCS_RING / 16; e += TCS_THREADS) reinterpret_cast<uint4*>(ring)[e] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) tc::tmem_alloc(misc, 512);
  if (tid == 0) {
    for (int b = 0; b < 2 * TCS_NSLOT + TCS_MAXD1; ++b) tc::mbar_init(bars + b, 1);
    tc::mbar_init(tready, 32 * TCS_CONV_WARPS);
    tc::mbar_init(tready + 1, 32 * TCS_CONV_WARPS);
    for (int b = 0; b < TCS_MAXD1; ++b) tc::mbar_init(d1free + b, 32 * TCS_CONV_WARPS);
    tc::mbar_init(dqb, 1);
    tc::mbar_init(dqb + 1, 1);
    *abort_flag = 0;
    *keep_tmem = 0;
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = misc[0];
  const int R = J.r1 - J.r0;
  const int rows16 = J.rows16;
  // GEMM1 buffers of d1w columns each below D2: round r uses buffer r % nd1
  const uint32_t d1w = (uint32_t)J.d1w;
  const int nd1 = min(TCS_MAXD1, (int)(TCS_D2_COL / d1w));
  long long* trace = (blockIdx.x == 0 && blockIdx.y == 0) ? g_tcs_trace : nullptr;

  if (warp == TCS_CONV_WARPS) {
    // ---- copy warp: round r goes to ring area [start, start + bytes), header slot r % NSLOT;
    // the records arrive TCS_DQ / 2 at a time, one half of the queue ahead
    const __nv_bfloat16* img = reinterpret_cast<const __nv_bfloat16*>(SB.tcimg);
    const __nv_bfloat16* xim = reinterpret_cast<const __nv_bfloat16*>(SB.ximg) + (int64_t)v * SB.ximg_stride;
    const TcsRec* jrec = recs + J.r0;
    constexpr int HALF = TCS_DQ / 2;
    uint32_t head = 0;
    int tail = 0;                            // rounds before tail are known to be complete
    uint32_t my_rs = 0, my_re = 0;           // lane j < TCS_NSLOT: area of the round in header slot j
    int my_rk = -1;
    int issued = 0, dq_issued = 0, dq_used = 0;
    auto fetch_half = [&](int first) {       // records [first, first + HALF) into half (first / HALF) % 2
      const int n = min(HALF, R - first), h = (first / HALF) & 1;
      if (n <= 0) return;
      const uint32_t by = (uint32_t)n * (uint32_t)sizeof(TcsRec);
      mbar_expect_tx(dqb + h, by);
      bulk_g2s(dq + h * HALF, jrec + first, by, dqb + h);
      dq_issued = first + n;
    };
    if (lane == 0) {
      fetch_half(0);
      fetch_half(HALF);
    }
    dq_issued = __shfl_sync(0xffffffffu, dq_issued, 0);
    for (int r = 0; r < R; ++r) {
      const int qk = r % TCS_DQ;
      if (r % HALF == 0 &&
          !__all_sync(0xffffffffu, tcs_wait(dqb + ((r / HALF) & 1), (uint32_t)(r / TCS_DQ) & 1u, abort_flag)))
        break;
      dq_used = min(R, (r / HALF + 1) * HALF);
      if (trace && lane == 0 && r < TCS_TRACE_ROUNDS) trace[12 * r + 6] = clock64();
      const TcsRec& RD = dq[qk];
      const uint32_t bytes = RD.bytes;
      const uint32_t start = head + bytes <= (uint32_t)TCS_RING ? head : 0u;
      bool ok = true;
      // the newest round in flight that still holds the header slot or part of the area (lane j
      // keeps header slot j's area in registers); GEMM2s complete in issue order, so once it
      // is done every older one is too
      const int need = __reduce_max_sync(
          0xffffffffu, (lane < TCS_NSLOT && my_rk >= tail && start < my_re && my_rs < start + bytes) ? my_rk : r - TCS_NSLOT);
      if (need >= tail) {
        if (lane == 0) {
          ok = tcs_wait(empty + need % TCS_NSLOT, (uint32_t)(need / TCS_NSLOT) & 1u, abort_flag);
        }
        tail = need + 1;
      }
      if (lane == r % TCS_NSLOT) { my_rs = start; my_re = start + bytes; my_rk = r; }
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) break;
      if (trace && lane == 0 && r < TCS_TRACE_ROUNDS) trace[12 * r + 7] = clock64();
      head = start + bytes;
      const int sl = r % TCS_NSLOT;
      RoundHdr* H = hdr + sl;
      static_assert(TCS_MAXSUB * TCS_MAXSLOTS == 32, "one coefficient pair per lane");
      H->sub[lane / TCS_MAXSLOTS].sN[lane % TCS_MAXSLOTS] = 0.f;
      H->sub[lane / TCS_MAXSLOTS].sT[lane % TCS_MAXSLOTS] = 0.f;
      if (lane < RD.nsub) {
        const TcsSub U = RD.subs[lane];
        SubHdr& D = H->sub[lane];
        D.nk16 = U.nk16;
        D.dc = U.dc;
        D.tk = U.tk;
        D.a_off = U.a_off;
        D.b_off = U.b_off;
        D.x_off = U.x_off;
        D.mask = U.mask;
      }
      __syncwarp();
      if (lane < RD.nt) {
        const TcsTerm tm = RD.terms[lane];
        SubHdr& D = H->sub[tm.slot >> 8];
        D.sN[tm.slot & 255] = tm.sN;
        D.sT[tm.slot & 255] = tm.sT;
      }
      if (lane == 0) {
        H->start = start;
        H->nsub = RD.nsub;
        H->ktot = RD.ktot;
      }
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();
        mbar_expect_tx(full + sl, RD.tx);
        if (trace && r < TCS_TRACE_ROUNDS) trace[12 * r] = clock64();
      }
      __syncwarp();
      if (lane < RD.nc) {
        const TcsCopy C = RD.copies[lane];
        bulk_g2s(ring + start + C.dst, (C.kind ? xim : img) + C.src, C.bytes, full + sl);
      }
      issued = r + 1;
      if (r % HALF == HALF - 1) {   // a half of the queue was used up: the records one half ahead into it
        __syncwarp();
        if (lane == 0) {
          tc::fence_async_smem();
          fetch_half(r + 1 + HALF);
        }
        dq_issued = __shfl_sync(0xffffffffu, dq_issued, 0);
      }
    }
    // no copy may still be landing when the CTA exits
    if (lane == 0) {
      for (int r = issued > TCS_NSLOT ? issued - TCS_NSLOT : 0; r < issued; ++r)
        if (!tcs_drain(full + r % TCS_NSLOT, (uint32_t)(r / TCS_NSLOT) & 1u)) *abort_flag = 1;
      for (int r = dq_used; r < dq_issued; r += HALF)
        if (!tcs_drain(dqb + ((r / HALF) & 1), (uint32_t)(r / TCS_DQ) & 1u)) *abort_flag = 1;
    }
    __syncwarp();
  } else if (warp == TCS_CONV_WARPS + 1) {
    // ---- GEMM1 warp: GEMM1 of round r once its images landed and its D1 buffer was read
    // out by the T-forming warps (round r - nd1).  The warp runs converged (warp-uniform
    // descriptors) and one elected lane issues the MMAs and the commit.
    const bool leader = tc::elect_one();
    int last = -1;
    bool ok = true;
    for (int r = 0; r < R; ++r) {
      const int sl = r % TCS_NSLOT;
      bool w = tcs_wait(full + sl, (uint32_t)(r / TCS_NSLOT) & 1u, abort_flag);
      if (w && r >= nd1) w = tcs_wait(d1free + r % nd1, (uint32_t)((r - nd1) / nd1) & 1u, abort_flag);
      ok = __all_sync(0xffffffffu, w);
      if (!ok) break;
      tc::fence_after_sync();
      if (trace && leader && r < TCS_TRACE_ROUNDS) trace[12 * r + 1] = clock64();
      const RoundHdr& H = hdr[sl];
      const uint32_t base = tc::smem_u32(ring + H.start);
      const uint32_t d = tmem + (uint32_t)(r % nd1) * d1w;
      const int nsub = H.nsub;
      for (int i = 0; i < nsub; ++i) {
        const int nk16 = H.sub[i].nk16;
        const uint32_t SBO = (uint32_t)nk16 * 16;
        const uint32_t aS = base + H.sub[i].a_off, xS = base + H.sub[i].x_off;
        const uint32_t idesc1 = tc::idesc_bf16(128, 2 * nk16);
        const uint32_t dd = d + (uint32_t)H.sub[i].dc;
        for (int ks = 0; ks < nk16 / 16; ++ks) {
          const uint64_t ad = tc::sdesc(aS + ks * 256, 128, SBO), xd = tc::sdesc(xS + ks * 256, 128, SBO);
          if (leader) tc::mma_bf16(dd, ad, xd, idesc1, ks > 0 ? 1u : 0u);
        }
      }
      __syncwarp();
      if (leader) tc::mma_commit(g1 + r % nd1);
      last = r;
      if (trace && leader && r < TCS_TRACE_ROUNDS) trace[12 * r + 2] = clock64();
    }
    // the last commit covers every MMA this warp issued: until it lands TMEM stays allocated
    bool drained = true;
    if (leader && last >= 0) drained = tcs_drain(g1 + last % nd1, (uint32_t)(last / nd1) & 1u);
    if (!__all_sync(0xffffffffu, drained || !leader) && leader) *keep_tmem = 1;
    __syncwarp();
  } else if (warp == TCS_CONV_WARPS + 2) {
    // ---- GEMM2 warp: GEMM2 of round r once its T was formed; its commit frees the round's
    // ring area and T tile
    const bool leader = tc::elect_one();
    int last = -1;
    bool ok = true;
    for (int rr = 0; rr < R; ++rr) {
      const int b = rr & 1, sl = rr % TCS_NSLOT;
      ok = __all_sync(0xffffffffu, tcs_wait(tready + b, (uint32_t)(rr / 2) & 1u, abort_flag));
      if (!ok) break;
      if (trace && leader && rr < TCS_TRACE_ROUNDS) trace[12 * rr + 8] = clock64();
      tc::fence_after_sync();
      const RoundHdr& H = hdr[sl];
      const uint32_t base = tc::smem_u32(ring + H.start);
      const uint32_t tS = tc::smem_u32(tbuf + b * TCS_TBUF), SBO_T = (uint32_t)H.ktot * 16;
      const uint32_t idesc2 = tc::idesc_bf16(128, rows16);
      const int nsub = H.nsub;
      if (trace && leader && rr < TCS_TRACE_ROUNDS) trace[12 * rr + 10] = clock64();
      for (int i = 0; i < nsub; ++i) {
        const int nk16 = H.sub[i].nk16;
        const uint32_t bS = base + H.sub[i].b_off;
        const uint32_t t0s = tS + (uint32_t)(H.sub[i].tk >> 3) * 128u;
        for (int ks = 0; ks < nk16 / 16; ++ks) {
          const uint64_t td = tc::sdesc(t0s + ks * 256, 128, SBO_T), bd = tc::sdesc(bS + ks * 256, 128, (uint32_t)nk16 * 16);
          if (leader) tc::mma_bf16(tmem + TCS_D2_COL, td, bd, idesc2, (rr > 0 || i > 0 || ks > 0) ? 1u : 0u);
        }
      }
      __syncwarp();
      if (trace && leader && rr < TCS_TRACE_ROUNDS) trace[12 * rr + 11] = clock64();
      if (leader) tc::mma_commit(empty + sl);   // the round's area and its T tile are free again
      last = rr;
      if (trace && leader && rr < TCS_TRACE_ROUNDS) trace[12 * rr + 5] = clock64();
    }
    bool drained = true;
    if (leader && last >= 0) drained = tcs_drain(empty + last % TCS_NSLOT, (uint32_t)(last / TCS_NSLOT) & 1u);
    if (!__all_sync(0xffffffffu, drained || !leader) && leader) *keep_tmem = 1;
    __syncwarp();
  } else {
    // ---- T-forming warps: T = sN D1[:, :nk] + sT D1[:, nk:] for the rows of this thread's
    // slot; warp w covers TMEM lanes 32 (w % 4) .. + 31 and the 16-column chunks c = w / 4 (mod 2)
    const int quad = warp & 3, half = warp >> 2;
    const int row = quad * 32 + lane;
    int myslot = -1;
    for (int k = 0; k < J.ns; ++k) {
      const TcsSlot S = slots[J.s0 + k];
      if (row >= S.row0 && row < S.row0 + ((S.n_out + 15) & ~15)) myslot = k;
    }
    const bool active = quad * 32 < rows16;   // warp-uniform
    bool ok = true;
    for (int r = 0; r < R; ++r) {
      const int b = r & 1, sl = r % TCS_NSLOT;
      bool w = tcs_wait(g1 + r % nd1, (uint32_t)(r / nd1) & 1u, abort_flag);
      if (w) w = tcs_wait(full + sl, (uint32_t)(r / TCS_NSLOT) & 1u, abort_flag);   // the header
      if (w && r >= 2)   // T tile b: the GEMM2 of round r - 2 completed
        w = tcs_wait(empty + (r - 2) % TCS_NSLOT, (uint32_t)((r - 2) / TCS_NSLOT) & 1u, abort_flag);
      ok = __all_sync(0xffffffffu, w);
      if (!ok) break;
      tc::fence_after_sync();
      if (trace && tid == 0 && r < TCS_TRACE_ROUNDS) trace[12 * r + 3] = clock64();
      const RoundHdr& H = hdr[sl];
      unsigned char* T = tbuf + b * TCS_TBUF;
      if (active) {
        const uint32_t rowoff = (uint32_t)(row >> 3) * (uint32_t)(H.ktot * 16) + (uint32_t)(row & 7) * 16u;
        const uint32_t dbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(r % nd1) * d1w;
        for (int i = 0; i < H.nsub; ++i) {
          const SubHdr& U = H.sub[i];
          const int nk16 = U.nk16, nc = nk16 / 16;
          const bool present = myslot >= 0 && ((U.mask >> myslot) & 1u);
          const float sN = present ? U.sN[myslot] : 0.f, sT = present ? U.sT[myslot] : 0.f;
          const uint32_t db = dbase + (uint32_t)U.dc;
          constexpr int NH = (TCS_KMAX / 16 + 1) / 2;   // chunks per warp and sub-block
          uint32_t xn[NH][16], xt[NH][16];
#pragma unroll
          for (int j = 0; j < NH; ++j) {
            const int c = 2 * j + half;
            if (c < nc) {
              tc::tmem_ld16_nowait(db + (uint32_t)(c * 16), xn[j]);
              tc::tmem_ld16_nowait(db + (uint32_t)(nk16 + c * 16), xt[j]);
            }
          }
          tc::tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < NH; ++j) {
            const int c = 2 * j + half;
            if (c >= nc) break;
            float x[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              asm volatile("" : "+r"(xn[j][e]), "+r"(xt[j][e]));   // keeps every use after the wait
              x[e] = present ? fmaf(sN, __uint_as_float(xn[j][e]), sT * __uint_as_float(xt[j][e])) : 0.f;
            }
            uint4 w0, w1;
            w0.x = pack_bf16x2(x[0], x[1]);
            w0.y = pack_bf16x2(x[2], x[3]);
            w0.z = pack_bf16x2(x[4], x[5]);
            w0.w = pack_bf16x2(x[6], x[7]);
            w1.x = pack_bf16x2(x[8], x[9]);
            w1.y = pack_bf16x2(x[10], x[11]);
            w1.z = pack_bf16x2(x[12], x[13]);
            w1.w = pack_bf16x2(x[14], x[15]);
            const uint32_t k8 = (uint32_t)(U.tk >> 3) + 2u * c;
            *reinterpret_cast<uint4*>(T + rowoff + k8 * 128u) = w0;
            *reinterpret_cast<uint4*>(T + rowoff + (k8 + 1) * 128u) = w1;
          }
        }
      }
      tc::fence_async_smem();
      tc::fence_before_sync();
      if (trace && tid == 0 && r < TCS_TRACE_ROUNDS) trace[12 * r + 4] = clock64();
      mbar_arrive(d1free + r % nd1);   // this round's D1 buffer has been read out
      mbar_arrive(tready + b);
    }
    // the last GEMM2, then the diagonal slot blocks of D2 into the output
    if (ok && R > 0) {
      const int rl = R - 1;
      ok = __all_sync(0xffffffffu, tcs_wait(empty + rl % TCS_NSLOT, (uint32_t)(rl / TCS_NSLOT) & 1u, abort_flag));
    }
    if (ok && R > 0 && active && half == 0) {
      tc::fence_after_sync();
      float* out = reinterpret_cast<float*>(SB.sout) + (int64_t)v * SB.sout_stride;
      for (int k = 0; k < J.ns; ++k) {
        const TcsSlot S = slots[J.s0 + k];
        const int n16 = (S.n_out + 15) & ~15;
        const int rr = row - S.row0;
        for (int c16 = 0; c16 < n16 / 16; ++c16) {
          float x[16];
          tc::tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + TCS_D2_COL + (uint32_t)(S.row0 + c16 * 16), x);
          if (myslot == k && rr < S.n_out) {
            float* C = out + S.c_off + (int64_t)rr * S.n_out;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (c16 * 16 + j < S.n_out) atomicAdd(C + c16 * 16 + j, x[j]);
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0 && (*abort_flag || *keep_tmem)) atomicOr(&g_tcs_status, *keep_tmem ? 3 : 1);
  if (warp == 0 && !*keep_tmem) tc::tmem_dealloc(tmem, 512);
}

}  // namespace

int tcs_status(bool clear, cudaStream_t s) {
  int st = 0;
  PN_CUDA(cudaMemcpyFromSymbolAsync(&st, g_tcs_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  if (clear) {
    const int zero = 0;
    PN_CUDA(cudaMemcpyToSymbolAsync(g_tcs_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
  }
  PN_CUDA(cudaStreamSynchronize(s));
  return st;
}

void make_tc_images(const double* pool, __nv_bfloat16* img, const int64_t* d_desc, int nimg, cudaStream_t s) {
  for (int b = 0; b < nimg; b += 65535) {
    const int n = std::min(65535, nimg - b);
    k_tcs_make_img<<<n, 128, 0, s>>>(pool, img, d_desc + 6 * (int64_t)b);
  }
  PN_CUDA(cudaGetLastError());
}

void run_sandwich_tc(const TcsJob* d_jobs, int njobs, const TcsSlot* d_slots, const TcsRec* d_recs,
                     const int64_t* d_xblk, int nxblk, const SysTable& t, cudaStream_t s) {
  if (njobs <= 0 || t.max_nvec <= 0) return;
  PN_CHECK(t.nsys == 1, PNOEOM_ERR_UNSUPPORTED, "tensor-core sandwich path: one system per launch");
  PN_CUDA(cudaFuncSetAttribute((const void*)k_sandwich_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TCS_SMEM));
  k_tcs_pack_x<<<dim3(nxblk, t.max_nvec), 128, 0, s>>>(d_xblk, t);
  PN_CUDA(cudaGetLastError());
  const char* trace_path = std::getenv("PNOEOM_TCS_TRACE");
  static DBuf<long long>* trace_buf = new DBuf<long long>();   // kept for the process
  if (trace_path) {
    if (!trace_buf->n) trace_buf->alloc(12 * TCS_TRACE_ROUNDS);
    trace_buf->zero(s);
    long long* p = trace_buf->get();
    PN_CUDA(cudaMemcpyToSymbolAsync(g_tcs_trace, &p, sizeof(p), 0, cudaMemcpyHostToDevice, s));
  }
  for (int b = 0; b < njobs; b += 65535) {
    const int n = std::min(65535, njobs - b);
    k_sandwich_tc<<<dim3(n, t.max_nvec), TCS_THREADS, TCS_SMEM, s>>>(d_jobs + b, d_slots, d_recs, t);
  }
  PN_CUDA(cudaGetLastError());
  if (trace_path) {   // the first bin's stamps, appended to the file (synchronises the stream)
    long long* null = nullptr;
    PN_CUDA(cudaMemcpyToSymbolAsync(g_tcs_trace, &null, sizeof(null), 0, cudaMemcpyHostToDevice, s));
    std::vector<long long> h(12 * TCS_TRACE_ROUNDS);
    trace_buf->download(h.data(), h.size(), s);
    PN_CUDA(cudaStreamSynchronize(s));
    if (FILE* f = std::fopen(trace_path, "a")) {
      for (int r = 0; r < TCS_TRACE_ROUNDS && h[12 * r + 1]; ++r) {
        for (int e = 0; e < 12; ++e) std::fprintf(f, "%lld ", h[12 * r + e]);
        std::fprintf(f, "\n");
      }
      std::fprintf(f, "end\n");
      std::fclose(f);
    }
  }
}

}  // namespace pnoeom

// ---------------------------------------------------------------------------
// Setup of the tensor-core sandwich path from the phase-2 sandwich problems.
namespace pnoeom {

namespace {
struct ImgKey {
  int64_t src;
  int ld, trans, rows, K;
  bool operator==(const ImgKey& o) const {
    return src == o.src && ld == o.ld && trans == o.trans && rows == o.rows && K == o.K;
  }
};
struct ImgKeyHash {
  size_t operator()(const ImgKey& k) const {
    uint64_t h = (uint64_t)k.src * 0x9E3779B97F4A7C15ull;
    h ^= ((uint64_t)k.ld << 1) ^ ((uint64_t)k.trans << 33) ^ ((uint64_t)k.rows << 40) ^ ((uint64_t)k.K << 52);
    return (size_t)(h ^ (h >> 29));
  }
};
inline int up16(int x) { return (x + 15) & ~15; }
}  // namespace

void build_tcs(pnoeom_pno* P, const std::vector<SProb>& sp2,
               const std::unordered_map<int64_t, std::pair<int64_t, int>>& s_transpose, cudaStream_t s, size_t* fp) {
  Program& PR = P->prog;
  // X blocks: every stored pair block with PNOs, one two-variant image (2 n16 x n16) each
  std::unordered_map<int64_t, int> xq;          // vector offset -> X block index
  std::vector<int64_t> xblk;
  int64_t xs = 0;
  for (int p = 0; p < P->npairs; ++p) {
    const int n = P->nij[p];
    if (!n) continue;
    xq[P->off_ij[p]] = (int)(xblk.size() / 3);
    xblk.push_back(P->off_ij[p]);
    xblk.push_back(n);
    xblk.push_back(xs);
    xs += 2 * (int64_t)up16(n) * up16(n);
  }
  // terms, normalised to the stored orientation of their output block:
  //   C += A (sN X + sT X^T) B, with GEMM1's two halves A X^T (rows of X) and A X
  struct Term { ImgKey a, b; int q; float sN, sT; };
  std::map<int64_t, std::pair<int, std::vector<Term>>> outs;   // output block offset -> (n_out, terms)
  std::vector<SProb> rest;
  for (const SProb& q : sp2) {
    const bool ok = q.a_buf == B_POOL && q.b_buf == B_POOL && q.x_buf == B_RIN && q.c_buf == B_SOUT && q.M == q.N &&
                    q.K1 == q.K2 && q.M <= TCS_MAXN && q.K1 <= TCS_MAXN && q.ldx == q.K1 && q.ldc == q.M &&
                    xq.count(q.x_off);
    if (!ok) { rest.push_back(q); continue; }
    if (q.m0 != 0 || q.n0 != 0) continue;   // the whole problem is one term
    const ImgKey ka{q.a_off, q.lda, q.ta, q.M, q.K1}, kbt{q.b_off, q.ldb, !q.tb, q.N, q.K2};
    // C = alpha A (Xo + xb Xo^T) B with Xo = opX(X); the stored block gets C (tc = 0) or
    // C^T = alpha B^T (Xo^T + xb Xo) A^T (tc = 1)
    const bool xo_is_x = q.tc ? q.tx != 0 : q.tx == 0;
    const float al = (float)q.alpha, alx = (float)(q.alpha * q.xb);
    Term t{q.tc ? kbt : ka, q.tc ? ka : kbt, xq[q.x_off], xo_is_x ? alx : al, xo_is_x ? al : alx};
    auto& O = outs[q.c_off];
    O.first = q.M;
    O.second.push_back(t);
  }
  // bins: output blocks by decreasing size, first fit into TCS_ROWS rows / TCS_MAXSLOTS slots
  std::vector<std::pair<int, int64_t>> order;
  for (auto& kv : outs) order.push_back({up16(kv.second.first), kv.first});
  std::stable_sort(order.begin(), order.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  std::vector<std::vector<int64_t>> bins;
  std::vector<int> bin_rows;
  for (auto& o : order) {
    size_t b = 0;
    while (b < bins.size() && (bin_rows[b] + o.first > TCS_ROWS || (int)bins[b].size() >= TCS_MAXSLOTS)) ++b;
    if (b == bins.size()) { bins.emplace_back(); bin_rows.push_back(0); }
    bins[b].push_back(o.second);
    bin_rows[b] += o.first;
  }
  // images, deduplicated, allocated in the order rounds first ask for them (so the slots of
  // a round often lie side by side in the pool and share one copy); the transposed image
  // of an overlap block S(a, b) is the image of S(b, a)
  std::unordered_map<ImgKey, int64_t, ImgKeyHash> images;
  std::vector<int64_t> desc;
  int64_t ipool = 0;
  auto canon = [&](ImgKey k) {
    if (k.trans && k.ld == k.rows) {
      auto it = s_transpose.find(k.src);
      if (it != s_transpose.end() && it->second.second == k.K) k = ImgKey{it->second.first, k.K, 0, k.rows, k.K};
    }
    return k;
  };
  auto image = [&](ImgKey k) {
    k = canon(k);
    auto it = images.find(k);
    if (it != images.end()) return it->second;
    const int64_t off = ipool;
    ipool += (int64_t)up16(k.rows) * up16(k.K);
    images.emplace(k, off);
    for (int64_t x : {k.src, (int64_t)k.ld, (int64_t)k.trans, (int64_t)k.rows, (int64_t)k.K, off}) desc.push_back(x);
    return off;
  };
  // units: one vector block and at most one term per slot (the d-th term of every slot)
  struct Unit { int q, nk16; std::vector<std::pair<int, const Term*>> st; };
  std::vector<TcsJob> hj;
  std::vector<TcsSlot> hsl;
  std::vector<std::vector<Unit>> bin_units(bins.size());
  for (size_t bi = 0; bi < bins.size(); ++bi) {
    TcsJob J{};
    J.s0 = (int)hsl.size();
    J.ns = (int)bins[bi].size();
    J.rows16 = bin_rows[bi];
    J.sys = 0;
    std::map<int, std::vector<std::vector<const Term*>>> byq;   // q -> per slot, its terms
    int row0 = 0;
    for (int k = 0; k < J.ns; ++k) {
      auto& O = outs[bins[bi][k]];
      hsl.push_back({bins[bi][k], O.first, row0});
      row0 += up16(O.first);
      for (const Term& t : O.second) {
        auto& v = byq[t.q];
        if (v.empty()) v.resize(J.ns);
        v[k].push_back(&t);
      }
    }
    int kmax16 = 16;
    for (auto& kv : byq) {
      size_t depth = 0;
      for (auto& v : kv.second) depth = std::max(depth, v.size());
      const int nk16 = up16((int)xblk[3 * kv.first + 1]);
      kmax16 = std::max(kmax16, nk16);
      for (size_t d = 0; d < depth; ++d) {
        Unit u{kv.first, nk16, {}};
        for (int k = 0; k < J.ns; ++k)
          if (d < kv.second[k].size()) u.st.push_back({k, kv.second[k][d]});
        bin_units[bi].push_back(u);
      }
    }
    J.d1w = kmax16 <= 64 ? 128 : 2 * kmax16;
    hj.push_back(J);
  }
  // images of the units whose A and B are one image (the occupied ladder: S(ij,kl) on both
  // sides) first, in unit order: the slots of such a unit, and consecutive units of one bin,
  // then lie side by side in the pool and reach the round's area in one copy per tile kind
  for (size_t bi = 0; bi < bins.size(); ++bi)
    for (const Unit& u : bin_units[bi]) {
      bool same = true;
      for (auto& e : u.st) same = same && canon(e.second->a) == canon(e.second->b);
      if (same)
        for (auto& e : u.st) image(e.second->a);
    }
  // rounds: consecutive units share a round while its GEMM1 columns, sub-blocks, terms,
  // area and merged copies fit; the area holds the sub-blocks' A tiles, then their B tiles,
  // then their X tiles, so tiles of consecutive sub-blocks merge into one copy as well
  std::vector<TcsRec> hrec;
  std::vector<double> rcost;                 // per record: MMA issue estimate (for splitting and ordering)
  double mma_flops = 0;                      // executed MMA flops of one vector
  size_t nterms = 0, ncopies = 0;
  auto merge = [](std::vector<TcsCopy> cp) {   // one copy for images adjacent in the source and the area
    std::sort(cp.begin(), cp.end(), [](const TcsCopy& a, const TcsCopy& b) { return a.dst < b.dst; });
    std::vector<TcsCopy> m;
    for (const TcsCopy& c : cp) {
      if (!m.empty()) {
        TcsCopy& l = m.back();
        if (l.kind == c.kind && l.src + l.bytes / 2 == c.src && l.dst + l.bytes == c.dst) { l.bytes += c.bytes; continue; }
      }
      m.push_back(c);
    }
    return m;
  };
  for (size_t bi = 0; bi < bins.size(); ++bi) {
    TcsJob& J = hj[bi];
    J.r0 = (int)hrec.size();
    const std::vector<Unit>& units = bin_units[bi];
    // layout of a round from its units: sub-block records, merged copies, area bytes
    auto layout = [&](const std::vector<const Unit*>& us, TcsRec& R) {
      uint32_t off = 0;
      int cols = 0, ktot = 0;
      R = TcsRec{};
      R.nsub = (int)us.size();
      for (size_t i = 0; i < us.size(); ++i) { R.subs[i].a_off = off; off += (uint32_t)J.rows16 * us[i]->nk16 * 2; }
      for (size_t i = 0; i < us.size(); ++i) { R.subs[i].b_off = off; off += (uint32_t)J.rows16 * us[i]->nk16 * 2; }
      for (size_t i = 0; i < us.size(); ++i) { R.subs[i].x_off = off; off += 2u * us[i]->nk16 * us[i]->nk16 * 2; }
      std::vector<TcsCopy> cp;
      for (size_t i = 0; i < us.size(); ++i) {
        const Unit& u = *us[i];
        TcsSub& U = R.subs[i];
        U.nk16 = (uint16_t)u.nk16;
        U.dc = (uint16_t)cols;
        U.tk = (uint16_t)ktot;
        U.mask = 0;
        for (auto& e : u.st) {
          const TcsSlot& S = hsl[J.s0 + e.first];
          const uint32_t rb = (uint32_t)S.row0 * u.nk16 * 2, sz = (uint32_t)up16(S.n_out) * u.nk16 * 2;
          cp.push_back({image(e.second->a), U.a_off + rb, sz, 0, 0});
          cp.push_back({image(e.second->b), U.b_off + rb, sz, 0, 0});
          if (R.nt < TCS_REC_TERMS) R.terms[R.nt] = {e.first | ((int)i << 8), e.second->sN, e.second->sT};
          ++R.nt;
          U.mask |= 1u << e.first;
        }
        cp.push_back({xblk[3 * u.q + 2], U.x_off, 2u * u.nk16 * u.nk16 * 2, 1, 0});
        cols += 2 * u.nk16;
        ktot += u.nk16;
      }
      const std::vector<TcsCopy> m = merge(cp);
      R.nc = (int)m.size();
      R.tx = 0;
      for (int c = 0; c < R.nc && c < TCS_REC_COPIES; ++c) { R.copies[c] = m[c]; R.tx += m[c].bytes; }
      R.bytes = off;
      R.ktot = ktot;
      return cols;
    };
    auto fits = [&](const TcsRec& R, int cols) {
      return cols <= J.d1w && R.nt <= TCS_REC_TERMS && R.bytes <= (uint32_t)TCS_MAX_AREA && R.nc <= TCS_REC_COPIES;
    };
    size_t ui = 0;
    while (ui < units.size()) {
      std::vector<const Unit*> us{&units[ui]};
      TcsRec R;
      int cols = layout(us, R);
      PN_CHECK(fits(R, cols), PNOEOM_ERR_CUDA, "tensor-core sandwich: a vector block does not fit a round");
      ++ui;
      while (ui < units.size() && (int)us.size() < TCS_MAXSUB) {
        us.push_back(&units[ui]);
        TcsRec R2;
        const int cols2 = layout(us, R2);
        if (!fits(R2, cols2)) { us.pop_back(); break; }
        R = R2;
        ++ui;
      }
      hrec.push_back(R);
      for (int i = 0; i < R.nsub; ++i)   // GEMM1: M = 128, N = 2 nk16, K = nk16; GEMM2: M = 128, N = rows16, K = nk16
        mma_flops += 2.0 * 128.0 * R.subs[i].nk16 * (2.0 * R.subs[i].nk16 + J.rows16);
      double cst = 700.0;
      for (int i = 0; i < R.nsub; ++i) cst += 2.0 * 72.0 * (R.subs[i].nk16 / 16);
      rcost.push_back(cst);
      nterms += R.nt;
      ncopies += R.nc;
    }
    J.r1 = (int)hrec.size();
  }
  {   // drop bins without rounds
    std::vector<TcsJob> keep;
    for (const TcsJob& J : hj)
      if (J.r1 > J.r0) keep.push_back(J);
    hj.swap(keep);
  }
  // enough CTAs for the device (about four per SM with six vectors): a bin's rounds are split
  // into contiguous ranges of similar cost, each a job whose D2 is added to the output
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int want = std::max<int>(1, (4 * sms) / 6);
  const int nsplit = hj.empty() ? 1 : std::min<int>(8, std::max<int>(1, (want + (int)hj.size() - 1) / (int)hj.size()));
  std::vector<std::pair<double, TcsJob>> jobs_c;
  for (const TcsJob& J : hj) {
    double tot = 0;
    for (int r = J.r0; r < J.r1; ++r) tot += rcost[r];
    int r = J.r0;
    for (int k = 0; k < nsplit && r < J.r1; ++k) {
      const double target = tot * (k + 1) / nsplit;
      double acc = 0;
      for (int x = J.r0; x < r; ++x) acc += rcost[x];
      int e = r;
      while (e < J.r1 && (acc + rcost[e] <= target || e == r || k == nsplit - 1)) acc += rcost[e++];
      TcsJob P2 = J;
      P2.r0 = r;
      P2.r1 = e;
      double c = 0;
      for (int x = r; x < e; ++x) c += rcost[x];
      jobs_c.push_back({c, P2});
      r = e;
    }
  }
  // every copy and operand lies inside its source and the round's area, every slot and
  // term inside its bin (the kernels index with these values unchecked)
  for (auto& jc : jobs_c) {
    const TcsJob& J = jc.second;
    PN_CHECK(J.ns >= 1 && J.ns <= TCS_MAXSLOTS && J.rows16 >= 16 && J.rows16 <= TCS_ROWS && J.rows16 % 16 == 0 &&
                 J.r1 > J.r0 && J.d1w >= 32 && J.d1w <= 2 * up16(TCS_MAXN) && J.d1w % 16 == 0 &&
                 2 * J.d1w <= 512 - TCS_ROWS,
             PNOEOM_ERR_CUDA, "tensor-core sandwich: bin shape");
    int rows = 0;
    for (int k = 0; k < J.ns; ++k) {
      const TcsSlot& S = hsl[J.s0 + k];
      PN_CHECK(S.row0 == rows && S.n_out >= 1 && S.n_out <= TCS_MAXN, PNOEOM_ERR_CUDA, "tensor-core sandwich: slot");
      rows += up16(S.n_out);
    }
    PN_CHECK(rows == J.rows16, PNOEOM_ERR_CUDA, "tensor-core sandwich: bin rows");
    for (int r = J.r0; r < J.r1; ++r) {
      const TcsRec& R = hrec[r];
      PN_CHECK(R.nsub >= 1 && R.nsub <= TCS_MAXSUB && R.nt >= 1 && R.nt <= TCS_REC_TERMS && R.nc >= 1 &&
                   R.nc <= TCS_REC_COPIES && R.bytes <= (uint32_t)TCS_MAX_AREA && R.ktot <= up16(TCS_MAXN),
               PNOEOM_ERR_CUDA, "tensor-core sandwich: round");
      uint32_t area = 0;
      int cols = 0, ktot = 0;
      for (int i = 0; i < R.nsub; ++i) {
        const TcsSub& U = R.subs[i];
        PN_CHECK(U.nk16 >= 16 && U.nk16 <= up16(TCS_MAXN) && U.nk16 % 16 == 0 && U.a_off == area && U.dc == cols &&
                     U.tk == ktot,
                 PNOEOM_ERR_CUDA, "tensor-core sandwich: sub-block");
        area += (uint32_t)J.rows16 * U.nk16 * 2;
        cols += 2 * U.nk16;
        ktot += U.nk16;
      }
      for (int i = 0; i < R.nsub; ++i) {
        PN_CHECK(R.subs[i].b_off == area, PNOEOM_ERR_CUDA, "tensor-core sandwich: B tile");
        area += (uint32_t)J.rows16 * R.subs[i].nk16 * 2;
      }
      for (int i = 0; i < R.nsub; ++i) {
        PN_CHECK(R.subs[i].x_off == area, PNOEOM_ERR_CUDA, "tensor-core sandwich: X tile");
        area += 2u * R.subs[i].nk16 * R.subs[i].nk16 * 2;
      }
      PN_CHECK(area == R.bytes && cols <= J.d1w && ktot == R.ktot, PNOEOM_ERR_CUDA, "tensor-core sandwich: round area");
      uint32_t seen[TCS_MAXSUB] = {0, 0, 0, 0}, tx = 0;
      for (int t = 0; t < R.nt; ++t) {
        const int sub = R.terms[t].slot >> 8, slot = R.terms[t].slot & 255;
        PN_CHECK(sub >= 0 && sub < R.nsub && slot >= 0 && slot < J.ns && !(seen[sub] >> slot & 1u) &&
                     (R.subs[sub].mask >> slot & 1u),
                 PNOEOM_ERR_CUDA, "tensor-core sandwich: term slot");
        seen[sub] |= 1u << slot;
      }
      for (int c = 0; c < R.nc; ++c) {
        const TcsCopy& C = R.copies[c];
        const int64_t lim = C.kind ? xs : ipool;
        PN_CHECK(C.src >= 0 && C.src % 8 == 0 && C.src + C.bytes / 2 <= lim && C.bytes % 16 == 0 && C.bytes > 0 &&
                     C.dst % 16 == 0 && C.dst + C.bytes <= R.bytes,
                 PNOEOM_ERR_CUDA, "tensor-core sandwich: copy out of range");
        tx += C.bytes;
      }
      PN_CHECK(tx == R.tx, PNOEOM_ERR_CUDA, "tensor-core sandwich: transaction bytes");
    }
  }
  if (std::getenv("PNOEOM_LOG_TIMING"))
    std::fprintf(stderr,
                 "[pnoeom] tensor-core sandwich: %zu bins (%zu blocks) in %zu jobs, %zu rounds, %zu terms, %zu copies, "
                 "%.1f MB images, %zu problems on the generic kernel, %.3g MMA flops per vector\n",
                 hj.size(), hsl.size(), jobs_c.size(), hrec.size(), nterms, ncopies, ipool * 2e-6, rest.size(), mma_flops);
  // heaviest jobs first
  std::stable_sort(jobs_c.begin(), jobs_c.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  std::vector<TcsJob> hjs;
  for (auto& c : jobs_c) hjs.push_back(c.second);
  PR.h_gen2x = rest;
  PR.n_tcs_jobs = (int)hjs.size();
  PR.n_tcs_xblk = (int)(xblk.size() / 3);
  PR.tcs_xstride = std::max<int64_t>(xs, 256);
  PR.tcs_mma_flops = mma_flops;
  PR.tcs_jobs.alloc(std::max<size_t>(1, hjs.size()), fp); PR.tcs_jobs.upload(hjs.data(), hjs.size(), s);
  PR.tcs_slots.alloc(std::max<size_t>(1, hsl.size()), fp); PR.tcs_slots.upload(hsl.data(), hsl.size(), s);
  PR.tcs_recs.alloc(std::max<size_t>(1, hrec.size()), fp); PR.tcs_recs.upload(hrec.data(), hrec.size(), s);
  PR.tcs_xblk.alloc(std::max<size_t>(1, xblk.size()), fp); PR.tcs_xblk.upload(xblk.data(), xblk.size(), s);
  PR.gen2x.alloc(std::max<size_t>(1, rest.size()), fp); PR.gen2x.upload(rest.data(), rest.size(), s);
  PR.n_gen2x = (int)rest.size();
  P->tcimg.alloc(std::max<int64_t>(ipool, 256), fp);
  const int nimg = (int)(desc.size() / 6);
  if (nimg) {
    DBuf<int64_t> d_desc(desc.size());
    d_desc.upload(desc.data(), desc.size(), s);
    make_tc_images(P->pool64.get(), P->tcimg.get(), d_desc.get(), nimg, s);
    PN_CUDA(cudaStreamSynchronize(s));
  }
  PN_CUDA(cudaStreamSynchronize(s));
}

}  // namespace pnoeom
