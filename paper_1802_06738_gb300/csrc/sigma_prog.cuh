// The sigma program: R-independent PNO-space operator blocks (the "pool")
// plus problem lists applied to a batch of packed vectors.
//   * Sandwich problems  C += alpha * opA(A) * (opX(X) + xb opX(X)^T) * opB(B)   (small blocks)
//   * Dense problems     C += alpha * opA(A) * opB(B)   (GEMM tiles, split K)
//   * GEMV problems      c += alpha * A * x   (dense blocks; all roots per CTA)
// Operands are addressed by (buffer, offset).  Buffers: POOL (shared by all
// roots), RIN (input vector of the root), WORK (per-root intermediates),
// SOUT (output vector of the root).
#pragma once
#include "common.cuh"
#include <cuda_bf16.h>

namespace pnoeom {

enum BufId : int { B_POOL = 0, B_RIN = 1, B_WORK = 2, B_SOUT = 3, B_NONE = 4 };

struct SProb {
  int64_t a_off, x_off, b_off, c_off;
  int sys;                            // system index into the SysTable of the launch
  int a_buf, x_buf, b_buf, c_buf;     // a_buf/b_buf == B_NONE: identity
  int M, K1, K2, N;                   // A: M x K1, X: K1 x K2, B: K2 x N, C: M x N
  int lda, ldx, ldb, ldc;
  int ta, tx, tb, tc;                 // transposed storage flags; tc: C^T is stored
  int m0, n0;                         // output tile origin (tiles of at most 64 x 64)
  double alpha;
  double xb;                          // coefficient of opX(X)^T (square X); 0: opX(X) alone
};

// One output tile (tile x tile) and K chunk of a dense product.
struct DProb {
  int64_t a_off, b_off, c_off;
  int sys;
  int a_buf, b_buf, c_buf;
  int M, N, K;                        // A: M x K, B: K x N, C: M x N
  int lda, ldb, ldc;
  int ta, tb, tc;
  int m0, n0, k0, klen;
  int tile_m, tile_n;                 // tile extents of the list (accounting)
  double alpha;
};

struct VProb {
  int64_t a_off, x_off, c_off;
  int sys;                            // system index into the SysTable of the launch
  int x_buf, c_buf;
  int M, K;                           // A: M x K row-major (lda)
  int lda;
  int x_stride, c_stride;             // element strides of x and c
  int xvec_n, cvec_n;                 // > 0: vectorised n x n block read / written transposed
  int m0, mlen;                       // rows m0 .. m0 + mlen - 1 of this tile (GEMV_ROWS-row groups)
  int k0, klen;                       // K chunk of this tile (split-K; klen <= GEMV_KC)
  double alpha;
};

// Tensor-core sandwich path (BF16 operands, FP32 accumulation in TMEM).  Output pair
// blocks are packed into "bins" of at most 128 rows (each block padded to 16 rows: its
// slot); one CTA evaluates, for one vector, every sandwich term of every block of a bin:
//   C_s += A_t (sN_t X + sT_t X^T) B_t          (slot s of term t, X = stored vector block q)
// in rounds of up to TCS_MAXSUB sub-blocks; a sub-block takes one vector block q and at
// most one term per slot:
//   GEMM1  D1 = [A_t stacked by slot] [X; X^T]^T     (M = 128, N = 2 nk, K = nk)
//   T      = sN D1[:, :nk] + sT D1[:, nk:]           per row (slot), zero for slots without a term
//   GEMM2  D2 += T [B_t^T stacked by slot]^T         (M = 128, N = bin rows, K = nk)
// and adds the diagonal slot blocks of D2 to the output.  Operands are BF16 images in an
// "M-outer" no-swizzle core-matrix layout, element (r, k) of an R x K image at byte
//   (r / 8) * (K16 * 16) + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2     (K16 = K rounded up to 16)
// so images stack along M by concatenation.
constexpr int TCS_MAXN = 80;             // n_out and nk of terms on this path
constexpr int TCS_ROWS = 128;            // rows of a bin
constexpr int TCS_MAXSLOTS = 8;
constexpr int TCS_MAXSUB = 4;            // vector blocks of a round
constexpr int TCS_NSLOT = 8;             // rounds in flight (stage barriers / headers)
constexpr int TCS_HDR = 384;             // bytes of a round header
constexpr int TCS_MAX_AREA = 80 * 1024;  // bytes of one round's tiles
constexpr int TCS_CONV_WARPS = 8;        // warps forming T: two per TMEM lane quarter, alternate 16-column chunks
constexpr int TCS_THREADS = 32 * (TCS_CONV_WARPS + 3);   // + a bulk-copy warp and two MMA-issue warps

struct TcsJob {                          // one bin (CTA x vector)
  int r0, r1;                            // round records [r0, r1) (a bin's rounds may be split over jobs)
  int s0, ns;                            // slots [s0, s0 + ns)
  int rows16;                            // rows of the bin (sum of slot rows)
  int sys;
  int d1w;                               // TMEM columns of one GEMM1 buffer (>= every round's sum of 2 nk)
  int pad;
};
struct TcsSlot {
  int64_t c_off;                         // output block offset (n_out x n_out, row-major)
  int n_out;
  int row0;                              // first row of the slot in the bin
};
struct TcsTerm {
  int slot;                              // slot | (sub-block << 8)
  float sN, sT;
};
struct TcsSub {                          // one vector block of a round
  uint16_t nk16;                         // its K
  uint16_t dc;                           // GEMM1 columns [dc, dc + 2 nk16) of the round's D1 buffer
  uint16_t tk;                           // its columns [tk, tk + nk16) of T
  uint16_t pad;
  uint32_t a_off, b_off, x_off;          // byte offsets of its A, B and X tiles in the round's area
  uint32_t mask;                         // slots with a term
};
struct TcsCopy {                         // bulk copy into the round's stage area
  int64_t src;                           // element offset: image pool (kind 0) or the vector's X images (kind 1)
  uint32_t dst;                          // byte offset from the round's start
  uint32_t bytes;
  int kind;
  int pad;
};
constexpr int TCS_REC_COPIES = 20;
constexpr int TCS_REC_TERMS = TCS_MAXSUB * TCS_MAXSLOTS;
// One round, fixed size (the copy warp prefetches records many rounds ahead with bulk copies).
struct TcsRec {
  uint32_t bytes;                        // area of the round: the A tiles, then the B tiles, then the X tiles
  uint32_t tx;                           // bytes its copies deliver (slots without a term get none)
  int nsub, nt, nc;                      // sub-blocks, terms, copies
  int ktot;                              // sum of the sub-blocks' nk16 (columns of T)
  int pad[2];
  TcsSub subs[TCS_MAXSUB];
  TcsTerm terms[TCS_REC_TERMS];
  TcsCopy copies[TCS_REC_COPIES];
  int pad2[8];
};
static_assert(sizeof(TcsRec) == 1024, "round record");

constexpr int GEMV_KC = 2048;         // K chunk staged in shared memory per GEMV tile
constexpr int GEMV_ROWS = 32;         // rows of one GEMV row group (4 per warp)
constexpr int POOL_ALIGN = 8;         // GEMV blocks: offsets and leading dimensions are multiples of this
constexpr int SMALL_DIM = 64;         // sandwich problems with all dims <= this use the shared-memory kernel

// Per-system buffers of one launch.  nvec = number of vectors of that system
// in this call (0: the system takes no part).
struct SysBuf {
  const void* pool;
  const void* pool16;                 // BF16 copy of the pool, or NULL: in FP32 a non-NULL copy is what the GEMV blocks read
  const void* tcimg;                  // BF16 operand images of the tensor-core sandwich path, or NULL
  void* ximg; int64_t ximg_stride;    // per-vector BF16 images of the vector blocks (X and X^T), or NULL
  const void* rin; int64_t rin_stride;
  void* work; int64_t work_stride;
  void* sout; int64_t sout_stride;
  int nvec;
  int pad;
};
constexpr int MAX_SYS = 128;
// Passed to the kernels by value (__grid_constant__), so no device copy of the
// table is needed and batches of up to MAX_SYS systems share one launch.
struct SysTable {
  int nsys;
  int max_nvec;
  SysBuf s[MAX_SYS];
};

template <typename T>
void run_sandwich(const SProb* d_probs, int nprob, const SysTable& t, int smem_elems, cudaStream_t s);
// Output tiles and operands with every dim <= SMALL_DIM.  Problems are grouped by
// output tile: group g is probs[group_start[g] .. group_start[g+1]), all with the same
// C tile; a CTA takes one group and up to roots_per_cta vectors, stages A and B once
// per problem, stacks the vectors' X blocks so both products of the sandwich are one
// register-tiled GEMM each, keeps the C tile of every vector in registers over the
// group and adds it to C once.  dm, dk1, dk2, dn bound the tile rows, the rows and
// columns of the staged X block, and the tile columns of every problem of the set.
// pb > 1 (every problem of the set has A and B): pb consecutive problems of a group are
// staged together and product 2 runs once over their concatenated K ranges.
// nbsel: stage buffers of the unbatched kernel (1 or 2; 0 = choose by occupancy).
// shape: CTA shape of the unbatched kernel (1 = 128 threads x 2 C tiles each, 2 = 256 x 2,
// 3 = 256 x 4; 0 = by bucket); shapes whose tiles cannot hold the C block are raised.
template <typename T>
void run_sandwich_small(const SProb* d_probs, const int* d_group_start, int ngroups, const SysTable& t, int dm, int dk1,
                        int dk2, int dn, int roots_per_cta, int pb, int nbsel, int shape, cudaStream_t s);
// Tensor-core sandwich path: X images of every vector (one launch), then the bins (one
// launch, grid bins x vectors).  xblk: per stored block (vector offset, n, image offset).
void run_sandwich_tc(const TcsJob* d_jobs, int njobs, const TcsSlot* d_slots, const TcsRec* d_recs,
                     const int64_t* d_xblk, int nxblk, const SysTable& t, cudaStream_t s);
// Builds BF16 images from an FP64 pool: desc = nimg x {src, ld, trans, rows, K, dst}.
// Status word of the tensor-core sandwich kernel (same bits as device_status); clear resets it.
int tcs_status(bool clear, cudaStream_t s);
void make_tc_images(const double* pool, __nv_bfloat16* img, const int64_t* d_desc, int nimg, cudaStream_t s);

template <typename T>
void run_gemv(const VProb* d_probs, int nprob, const SysTable& t, cudaStream_t s);
// Output tiles of a dense list: DENSE_TILE_TC = 128 rows x 64 columns (tensor cores in
// FP32, SIMT in FP64); 32: tiles of at most 32 x 32, one per CTA with K split over lanes.
constexpr int DENSE_TILE_TC = 128;
template <typename T>
void run_dense(const DProb* d_probs, int nprob, const SysTable& t, int tile, cudaStream_t s);
// Reads (and with clear, resets) the tensor-core kernels' device status word, ordered on
// stream s: 0 when every bounded wait completed.
int device_status(bool clear, cudaStream_t s);
// Failure-detection self-test: one CTA waits on an mbarrier that nothing arrives at, for at
// most budget clock cycles, then records bit 0 of the status word like a tensor-core
// kernel whose wait ran out.  Returns 1 when the wait ran out (it always should).
int selftest_bounded_wait(long long budget, cudaStream_t s);
void gemm_tf32x3(const float* A, const float* B, float* C, int M, int N, int K, float alpha, cudaStream_t s);

}  // namespace pnoeom
