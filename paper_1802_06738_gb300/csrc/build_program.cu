// Second half of pno_build: R-independent intermediates of the closed-shell
// EOM-CCSD Jacobian and their projection into PNO/OSV spaces.
//
// sigma = Omega'(T2)[R2] + Omega(T2; [H~, R1]) is the Jacobian of the
// T1-dressed closed-shell CCSD residual (the same residual the oracle pins
// against brute force).  Every term is rewritten with the R-independent
// factors projected into the PNO spaces of the pairs it couples, so the
// sigma program only touches PNO-sized blocks:
//   * pair-diagonal dense block D_p (n^2 x n^2): the 4-virtual ladder
//     sum_cd (ac|bd) r^{cd}_{ij}, the T2-ladder sum_kl t^{kl} <(kc|ld), r^{ij}>
//     and the virtual Fock term;
//   * triple products over one shared occupied index (ring terms, occupied
//     Fock term) and over all pairs (occupied ladder), using overlaps
//     S(ij,kl) = U^ij^T U^kl and mixed-pair blocks U^ij^T W U^kl;
//   * dense singles couplings (OSV rows / columns);
//   * two R-dependent global intermediates (virtual and occupied Fock-like
//     contractions of u(R) with (ld|kc)).
#include "pno.cuh"
#include <algorithm>
#include <cmath>
#include <set>
#include <utility>

namespace pnoeom {
namespace {

using DV = DBuf<double>;
using Dims = std::map<char, int64_t>;

inline unsigned gsz(size_t n) { return (unsigned)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 32)); }
#define GRID_STRIDE(e, n) for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)(n); e += (int64_t)gridDim.x * blockDim.x)

// Acan[i,a,m,d] += delta_im Xv[a,d] - delta_ad Xo[m,i]
__global__ void k_acan_delta(double* A, const double* Xv, const double* Xo, int o, int v) {
  GRID_STRIDE(e, (int64_t)o * v * o * v) {
    int d = (int)(e % v); int64_t r = e / v;
    int m = (int)(r % o); r /= o;
    int a = (int)(r % v); int i = (int)(r / v);
    double val = 0;
    if (i == m) val += Xv[a * v + d];
    if (a == d) val -= Xo[m * o + i];
    A[e] += val;
  }
}
// D[a,b,c,d] += delta_ac F[b,d] + F[a,c] delta_bd
__global__ void k_add_fock_kron(double* D, const double* F, int n) {
  GRID_STRIDE(e, (int64_t)n * n * n * n) {
    int d = (int)(e % n); int64_t r = e / n;
    int c = (int)(r % n); r /= n;
    int b = (int)(r % n); int a = (int)(r / n);
    double val = 0;
    if (a == c) val += F[b * n + d];
    if (b == d) val += F[a * n + c];
    D[e] += val;
  }
}
// Kronecker-type assembly (row-major out with leading dimension ldo):
//  mode 0: out[a*n + b][c] += al S[a][c] w[b]   (a,b < n; c < nc)
//  mode 1: out[a*n + b][c] += al w[a] S[b][c]
//  mode 2: out[a][c*n + d] += al S[a][c] w[d]   (a < nc; c,d < n)
//  mode 3: out[a][c*n + d] += al S[a][d] w[c]
__global__ void k_kron(double* out, int64_t ldo, const double* S, int lds, const double* w, int n, int nc, int mode,
                       double al) {
  GRID_STRIDE(e, (int64_t)n * n * nc) {
    if (mode <= 1) {
      int c = (int)(e % nc); int64_t q = e / nc;
      int b = (int)(q % n), a = (int)(q / n);
      double val = mode == 0 ? S[(int64_t)a * lds + c] * w[b] : w[a] * S[(int64_t)b * lds + c];
      out[((int64_t)a * n + b) * ldo + c] += al * val;
    } else {
      int d = (int)(e % n); int64_t q = e / n;
      int c = (int)(q % n), a = (int)(q / n);
      double val = mode == 2 ? S[(int64_t)a * lds + c] * w[d] : S[(int64_t)a * lds + d] * w[c];
      out[(int64_t)a * ldo + (int64_t)c * n + d] += al * val;
    }
  }
}
// out[r*ldo + c] += al * X[r*ldx + c]  (r < rows, c < cols); transpose_n > 0 maps row r = a*n+b to b*n+a
__global__ void k_add_block(double* out, int64_t ldo, const double* X, int64_t ldx, int rows, int cols, double al,
                            int transpose_n) {
  GRID_STRIDE(e, (int64_t)rows * cols) {
    int r = (int)(e / cols), c = (int)(e % cols);
    int ro = r;
    if (transpose_n > 0) ro = (r % transpose_n) * transpose_n + r / transpose_n;
    out[(int64_t)ro * ldo + c] += al * X[(int64_t)r * ldx + c];
  }
}

// flag = 1 when B[Q][a][b] != B[Q][b][a] for some entry (bitwise comparison)
__global__ void k_asym_flag(int* flag, const double* B, int nq, int v) {
  GRID_STRIDE(e, (int64_t)nq * v * v) {
    const int64_t q = e / ((int64_t)v * v);
    const int r = (int)(e % ((int64_t)v * v));
    const int a = r / v, b = r % v;
    if (a < b && B[e] != B[(q * v + b) * v + a]) *flag = 1;
  }
}

// tb[l,k] = tb[k,l]^T for l > k (blocks of n x n, [k][l][A][B])
__global__ void k_mirror_lower(double* tb, int o, int n) {
  GRID_STRIDE(e, (int64_t)o * o * n * n) {
    const int64_t blk = e / ((int64_t)n * n);
    const int l = (int)(blk / o), k = (int)(blk % o);   // block [l][k]
    if (l <= k) continue;
    const int r = (int)(e % ((int64_t)n * n)), A = r / n, B = r % n;
    tb[e] = tb[((int64_t)k * o + l) * n * n + (int64_t)B * n + A];
  }
}

struct Prog {
  pnoeom_pno* P;
  cudaStream_t s;
  int o, v, naux;
  Dims dm;
  std::vector<SProb> sp1, sp2;
  std::vector<VProb> vp1, vp2;
  std::vector<DProb> dp1, dp2, dp3;
  int smem = 1;

  const double* U(int x, int y) const { return P->U.get() + P->Uoff_pair[P->pidx[x][y]]; }
  int n(int x, int y) const { return P->nij[P->pidx[x][y]]; }
  const double* Uo(int i) const { return P->U.get() + P->Uoff_osv[i]; }
  int no(int i) const { return P->ni[i]; }
  void sync() { PN_CUDA(cudaStreamSynchronize(s)); }

  void con(const Dims& d, const char* a, const double* A, const char* b, const double* B, const char* c, double* C,
           double alpha = 1.0, double beta = 0.0) {
    contract<double>(d, TView<double>{const_cast<double*>(A), a}, TView<double>{const_cast<double*>(B), b},
                     TView<double>{C, c}, alpha, beta, s);
  }
  void con(const char* a, const double* A, const char* b, const double* B, const char* c, double* C,
           double alpha = 1.0, double beta = 0.0) {
    con(dm, a, A, b, B, c, C, alpha, beta);
  }
  void perm(const double* in, double* out, std::vector<int64_t> dims, std::vector<int> p, double al = 1.0,
            double be = 0.0) {
    permute<double>(in, out, dims, p, al, be, s);
  }
  void add_block(double* out, int64_t ldo, const double* X, int64_t ldx, int rows, int cols, double al, int tn = 0) {
    if (rows <= 0 || cols <= 0) return;
    k_add_block<<<gsz((size_t)rows * cols), 256, 0, s>>>(out, ldo, X, ldx, rows, cols, al, tn);
    PN_CUDA(cudaGetLastError());
  }
  void kron(double* out, int64_t ldo, const double* S, int lds, const double* w, int nn, int nc, int mode, double al) {
    if (nn <= 0 || nc <= 0) return;
    k_kron<<<gsz((size_t)nn * nn * nc), 256, 0, s>>>(out, ldo, S, lds, w, nn, nc, mode, al);
    PN_CUDA(cudaGetLastError());
  }

  // out (nL x nR, leading dim ldo) = UL^T op(X) UR for a list of jobs; UL: v x nL, UR: v x nR, X: v x v.
  struct PJ { const double* UL; int nL; const double* X; int ldx; int tx; const double* UR; int nR; double* out; int ldo; double al; double be; };
  void project(const std::vector<PJ>& jobs) {
    const size_t cap = (size_t)64 << 20;   // temp elements per chunk
    size_t i0 = 0;
    while (i0 < jobs.size()) {
      size_t need = 0, i1 = i0;
      while (i1 < jobs.size() && (i1 == i0 || need + (size_t)v * jobs[i1].nR <= cap)) { need += (size_t)v * jobs[i1].nR; ++i1; }
      DV tmp(std::max<size_t>(1, need));
      std::vector<GemmProb<double>> a, b;
      size_t off = 0;
      for (size_t q = i0; q < i1; ++q) {
        const PJ& J = jobs[q];
        if (!J.nL || !J.nR) continue;
        double* T = tmp.get() + off;
        a.push_back({J.X, J.UR, T, v, J.nR, v, J.ldx, J.nR, J.nR, J.tx, 0, 1.0, 0.0});
        b.push_back({J.UL, T, J.out, J.nL, J.nR, v, J.nL, J.nR, J.ldo, 1, 0, J.al, J.be});
        off += (size_t)v * J.nR;
      }
      grouped_gemm<double>(a, s);
      grouped_gemm<double>(b, s);
      i0 = i1;
    }
  }
};

}  // namespace

void build_program(pnoeom_pno* P, cudaStream_t s, const double* Fd, DV& dBoo, DV& dBov, DV& dBvo, DV& dBvv, DV& t2,
                   DV& u2) {
  const int o = P->o, v = P->v, naux = P->naux, nmo = o + v;
  const int64_t O = o, V = v, N = naux;
  Prog G{P, s, o, v, naux, {}, {}, {}, {}, {}, {}, {}, {}, 1};
  for (char c : std::string("ijklmxyz")) G.dm[c] = O;
  for (char c : std::string("abcd")) G.dm[c] = V;
  G.dm['Q'] = N;
  const int npairs = P->npairs;
  const int64_t L1 = P->L1, L = P->L;
  size_t* fp = &P->footprint;

  StageTimer tm(s);
  // ---- dressed Fock blocks ------------------------------------------------------
  std::vector<double> Foo(O * O), Fov(O * V), Fvv(V * V);
  for (int i = 0; i < o; ++i) for (int j = 0; j < o; ++j) Foo[i * o + j] = Fd[i * nmo + j];
  for (int i = 0; i < o; ++i) for (int a = 0; a < v; ++a) Fov[i * v + a] = Fd[i * nmo + o + a];
  for (int a = 0; a < v; ++a) for (int b = 0; b < v; ++b) Fvv[a * v + b] = Fd[(o + a) * nmo + o + b];
  const bool t1 = P->has_t1;

  // ---- integral blocks (dressed), Mulliken (pq|rs) = sum_Q B_pq B_rs ------------
  // Only integrals with at most two virtual indices are formed in full (o^2 v^2 at most);
  // everything with three or four virtual indices enters through the DF factors, already
  // contracted with PNO/OSV bases (the "projected-first" routes below).
  DV g_ovov(O * V * O * V), g_oovv(O * O * V * V), g_voov(V * O * O * V), g_oooo(O * O * O * O), g_ooov(O * O * O * V),
      g_ovoo(O * V * O * O), g_oovo(O * O * V * O), g_vooo(V * O * O * O);
  G.con("Qkc", dBov.get(), "Qld", dBov.get(), "kcld", g_ovov.get());
  G.con("Qki", dBoo.get(), "Qac", dBvv.get(), "kiac", g_oovv.get());
  G.con("Qai", dBvo.get(), "Qkc", dBov.get(), "aikc", g_voov.get());
  G.con("Qki", dBoo.get(), "Qlj", dBoo.get(), "kilj", g_oooo.get());
  G.con("Qki", dBoo.get(), "Qlc", dBov.get(), "kilc", g_ooov.get());
  G.con("Qkc", dBov.get(), "Qlj", dBoo.get(), "kclj", g_ovoo.get());
  G.con("Qki", dBoo.get(), "Qbj", dBvo.get(), "kibj", g_oovo.get());
  G.con("Qai", dBvo.get(), "Qkj", dBoo.get(), "aikj", g_vooo.get());
  // gS[k,c,l,d] = (kd|lc): g_ovov with its two virtual indices exchanged; L = 2 g - gS
  DV gS(g_ovov.n), L_ovov(g_ovov.n);
  G.perm(g_ovov.get(), gS.get(), {O, V, O, V}, {0, 3, 2, 1});
  PN_CUDA(cudaMemcpyAsync(L_ovov.get(), gS.get(), gS.n * 8, cudaMemcpyDeviceToDevice, s));
  axpby<double>(L_ovov.get(), g_ovov.get(), 2.0, -1.0, L_ovov.n, s);
  const double* t = t2.get();
  const double* u = u2.get();
  // uS[x,l,d,a] = u[x,l,a,d]: rows (l,d), columns a, so that sum_a u[x,l,a,d] U[a,A] is one GEMM
  DV uS(u2.n);
  G.perm(u, uS.get(), {O, O, V, V}, {0, 1, 3, 2});
  // the dressed B_vv is symmetric in its two virtual indices unless T1 dressed it
  bool bsym = !t1;
  if (bsym) {
    DBuf<int> flag(1);
    flag.zero(s);
    k_asym_flag<<<gsz(dBvv.n), 256, 0, s>>>(flag.get(), dBvv.get(), naux, v);
    PN_CUDA(cudaGetLastError());
    int h = 0;
    flag.download(&h, 1, s);
    G.sync();
    bsym = h == 0;
  }

  tm.mark("  integral blocks");
  // ---- R-independent intermediates ------------------------------------------------
  DV W(O * O * O * O);       // W[k,i,l,j] = (ki|lj) + sum_cd t^{cd}_{ij} (kc|ld)
  PN_CUDA(cudaMemcpyAsync(W.get(), g_oooo.get(), W.n * 8, cudaMemcpyDeviceToDevice, s));
  G.con("ijcd", t, "kcld", g_ovov.get(), "kilj", W.get(), 1.0, 1.0);
  DV FvvI(V * V), FooI(O * O);
  FvvI.upload(Fvv.data(), Fvv.size(), s);
  FooI.upload(Foo.data(), Foo.size(), s);
  G.con("klbd", u, "ldkc", g_ovov.get(), "bc", FvvI.get(), -1.0, 1.0);
  G.con("ljcd", u, "kdlc", g_ovov.get(), "kj", FooI.get(), 1.0, 1.0);
  std::vector<double> FooI_h(O * O);
  FooI.download(FooI_h.data(), FooI_h.size(), s);
  // singles-singles diagonal parts: Xv = Fvv - sum u (kd|lc), Xo = Foo + sum u (md|kc)
  DV X1(O * O), Y1s(V * V), Xv(V * V);
  G.con("kicd", u, "mdkc", g_ovov.get(), "mi", X1.get());
  G.con("klac", u, "kdlc", g_ovov.get(), "ad", Y1s.get());
  Xv.upload(Fvv.data(), Fvv.size(), s);
  axpby<double>(Xv.get(), Y1s.get(), -1.0, 1.0, Xv.n, s);
  std::vector<double> Xo_h(O * O);
  X1.download(Xo_h.data(), Xo_h.size(), s);
  G.sync();
  for (int e = 0; e < o * o; ++e) Xo_h[e] += Foo[e];
  // small occupied-heavy blocks
  DV govoo_j(O * O * V * O);           // (kc|lj) stored [j][k][c][l]
  G.perm(g_ovoo.get(), govoo_j.get(), {O, V, O, O}, {3, 0, 1, 2});
  DV gooov_i(O * O * O * V);           // (ki|lc) stored [i][k][l][c]
  G.perm(g_ooov.get(), gooov_i.get(), {O, O, O, V}, {1, 0, 2, 3});
  DV wa_can(O * O * O * V), wb_can(O * O * O * V);   // (ki|bj) at [i][j][k][b], (ai|kj) at [i][j][k][a]
  G.perm(g_oovo.get(), wa_can.get(), {O, O, V, O}, {1, 3, 0, 2});
  G.perm(g_vooo.get(), wb_can.get(), {V, O, O, O}, {1, 3, 2, 0});
  DV Gam_can(O * O * O * V);           // [y][k][m][d] = 2 (ky|md) - (kd|my)
  G.perm(g_ooov.get(), Gam_can.get(), {O, O, O, V}, {1, 0, 2, 3}, 2.0);
  G.perm(g_ovoo.get(), Gam_can.get(), {O, V, O, O}, {3, 0, 2, 1}, -1.0, 1.0);
  DV G2q(O * O * O * V), G6q(O * O * O * V);   // G2q[i][m][k][c] = (ki|mc), G6q[x][m][k][c] = (mc|kx)
  G.perm(g_ooov.get(), G2q.get(), {O, O, O, V}, {1, 2, 0, 3});
  G.perm(g_ovoo.get(), G6q.get(), {O, V, O, O}, {3, 0, 2, 1});
  DV BvoT(O * N * V);                  // BvoT[j][Q][b] = B[Q,b,j]
  G.perm(dBvo.get(), BvoT.get(), {N, V, O}, {2, 0, 1});
  // OSV factors: Uocat (v x L1) = all OSV bases side by side; BUo[Q,a,L] = sum_d Bvv[Q,a,d] Uocat[d,L];
  // BoU[Q,k,L] = sum_d Bov[Q,k,d] Uocat[d,L]
  DV Uocat(std::max<int64_t>(1, V * L1)), BUo(std::max<int64_t>(1, N * V * L1)), BoU(std::max<int64_t>(1, N * O * L1));
  if (L1 > 0) {
    for (int m = 0; m < o; ++m)
      if (G.no(m))
        PN_CUDA(cudaMemcpy2DAsync(Uocat.get() + P->off_i[m], L1 * 8, G.Uo(m), G.no(m) * 8, G.no(m) * 8, V,
                                  cudaMemcpyDeviceToDevice, s));
    Dims d = G.dm;
    d['L'] = L1;
    G.con(d, "Qad", dBvv.get(), "dL", Uocat.get(), "QaL", BUo.get());
    G.con(d, "Qkd", dBov.get(), "dL", Uocat.get(), "QkL", BoU.get());
  }
  // columns of OSV m of a [rows][L1] factor, gathered into a contiguous [rows][n_m] buffer
  auto osv_cols = [&](const double* F, int64_t rows, int m, DV& out) {
    out.alloc(std::max<int64_t>(1, rows * G.no(m)));
    if (G.no(m))
      PN_CUDA(cudaMemcpy2DAsync(out.get(), G.no(m) * 8, F + P->off_i[m], L1 * 8, G.no(m) * 8, rows,
                                cudaMemcpyDeviceToDevice, s));
  };

  tm.mark("  o^2v^2 intermediates");
  // ---- projected amplitude and integral factors of the ring terms ---------------------------
  // For every pair {x, y} with PNOs and each of its occupied indices x, four (ov x n) factors
  // with rows (l, d):
  //   TU[x]: sum_a t[l,x,a,d] U[a,A]      UU[x]: sum_a u[x,l,a,d] U[a,A]
  //   GU[x]: sum_c (xd|lc) U[c,C]          LU[x]: sum_c L[l,d,x,c] U[c,C]
  // stored, for each occupied y, side by side over x ("cat" layout of y: column block of
  // pair {x, y} at coff[y][x], clen[y] columns in all).
  std::vector<std::vector<int64_t>> coff(o, std::vector<int64_t>(o, -1));
  std::vector<int64_t> clen(o, 0), cbase(o + 1, 0);
  for (int y = 0; y < o; ++y)
    for (int x = 0; x < o; ++x)
      if (G.n(x, y)) { coff[y][x] = clen[y]; clen[y] += G.n(x, y); }
  const int64_t OV = O * V;
  for (int y = 0; y < o; ++y) cbase[y + 1] = cbase[y] + OV * clen[y];
  DV TUc(std::max<int64_t>(1, cbase[o])), UUc(std::max<int64_t>(1, cbase[o])), GUc(std::max<int64_t>(1, cbase[o])),
      LUc(std::max<int64_t>(1, cbase[o]));
  {
    std::vector<GemmProb<double>> pr;
    for (int y = 0; y < o; ++y)
      for (int x = 0; x < o; ++x) {
        const int nn = G.n(x, y);
        if (!nn) continue;
        const int64_t co = cbase[y] + coff[y][x];
        const int ld = (int)clen[y];
        const double* Uq = G.U(x, y);
        pr.push_back({t + (int64_t)x * OV * V, Uq, TUc.get() + co, (int)OV, nn, v, v, nn, ld, 0, 0, 1.0, 0.0});
        pr.push_back({uS.get() + (int64_t)x * OV * V, Uq, UUc.get() + co, (int)OV, nn, v, v, nn, ld, 0, 0, 1.0, 0.0});
        pr.push_back({gS.get() + (int64_t)x * V * OV, Uq, GUc.get() + co, (int)OV, nn, v, (int)OV, nn, ld, 1, 0, 1.0, 0.0});
        pr.push_back({L_ovov.get() + (int64_t)x * V * OV, Uq, LUc.get() + co, (int)OV, nn, v, (int)OV, nn, ld, 1, 0, 1.0, 0.0});
      }
    grouped_gemm<double>(pr, s);
  }
  // column block of pair {x, y} (x being the amplitude's or integral's own index) as a
  // contiguous (ov x n) buffer
  auto cat_block = [&](const DV& F, int x, int y, DV& out) {
    const int nn = G.n(x, y);
    out.alloc(std::max<int64_t>(1, OV * nn));
    if (nn)
      PN_CUDA(cudaMemcpy2DAsync(out.get(), nn * 8, F.get() + cbase[y] + coff[y][x], clen[y] * 8, nn * 8, OV,
                                cudaMemcpyDeviceToDevice, s));
  };
  gS.release();

  tm.mark("  ring factors");
  // ---- pool layout ------------------------------------------------------------------
  auto nP = [&](int p) { return (int64_t)P->nij[p]; };
  int64_t pool = 0;
  auto take = [&](int64_t n) { int64_t off = pool; pool += n; return off; };
  const int64_t off_U = take(P->U.n);
  // U_cat = [U_p for every stored pair p] (v x sum n_p): one matrix for the global E3 products
  std::vector<int64_t> zc(npairs + 1, 0);
  for (int p = 0; p < npairs; ++p) zc[p + 1] = zc[p] + nP(p);
  const int64_t nsum = zc[npairs];
  const int64_t off_Ucat = take(V * nsum);
  std::vector<int64_t> offS((size_t)npairs * npairs);
  for (int p = 0; p < npairs; ++p) for (int q = 0; q < npairs; ++q) offS[(size_t)p * npairs + q] = take(nP(p) * nP(q));
  // ring blocks, one (clen[y] x clen[y]) matrix per occupied y and family:
  //   MC[i,j,k] = U(i,j)^T Wc[k,i] U(k,j)  at block (i, k) of y = j
  //   MD[i,j,k] = U(i,j)^T Wd[.,i,k,.] U(j,k)  at block (i, k) of y = j
  //   MZ[k,i,j] = U(k,i)^T Zt[k,j] U(i,j)  at block (k, j) of y = i
  //   MZd[k,i,j] = U(i,k)^T Zd[k,j] U(i,j)  at block (k, j) of y = i
  std::vector<int64_t> offMCc(o), offMDc(o), offMZc(o), offMZdc(o);
  for (int y = 0; y < o; ++y) {
    offMCc[y] = take(clen[y] * clen[y]);
    offMDc[y] = take(clen[y] * clen[y]);
    offMZc[y] = take(clen[y] * clen[y]);
    offMZdc[y] = take(clen[y] * clen[y]);
  }
  auto ring_off = [&](const std::vector<int64_t>& base, int y, int r, int c) {
    return base[y] + coff[y][r] * clen[y] + coff[y][c];
  };
  // blocks read by the GEMV kernel start on POOL_ALIGN-element boundaries and have leading
  // dimensions rounded up to POOL_ALIGN (the padding stays zero)
  auto pad = [](int64_t x) { return (x + POOL_ALIGN - 1) / POOL_ALIGN * POOL_ALIGN; };
  auto take_al = [&](int64_t n) { pool = pad(pool); return take(n); };
  const int64_t L1p = pad(L1), Lp = pad(L), Op = pad(O);
  std::vector<int64_t> offGh(O * O), offTh(O * O), offG4(O * O), offT4(O * O);
  for (int x = 0; x < o; ++x) for (int y = 0; y < o; ++y) {
    int64_t nn = G.n(x, y);
    offGh[x * o + y] = take(nn * V);
    offTh[x * o + y] = take(nn * V);
    offG4[x * o + y] = take_al(O * pad(nn * nn));
    offT4[x * o + y] = take_al(nn * nn * Op);
  }
  // Lv1 (v^2 x L1): the R1 part of the virtual global term, applied per call into FvR
  const int64_t off_Lv1 = take_al(V * V * L1p);
  std::vector<int64_t> offD(npairs), offADS(npairs);
  for (int p = 0; p < npairs; ++p) offD[p] = take_al(nP(p) * nP(p) * pad(nP(p) * nP(p)));
  for (int p = 0; p < npairs; ++p) offADS[p] = take_al(nP(p) * nP(p) * L1p);
  const int64_t off_AS = take_al(L1 * Lp);     // singles rows: row off_i[i] + A of OSV i, ld Lp
  P->pool64.alloc(std::max<int64_t>(1, pool), fp);
  P->pool64.zero(s);
  double* pl = P->pool64.get();
  PN_CUDA(cudaMemcpyAsync(pl + off_U, P->U.get(), P->U.n * 8, cudaMemcpyDeviceToDevice, s));
  for (int p = 0; p < npairs; ++p)
    if (nP(p))
      PN_CUDA(cudaMemcpy2DAsync(pl + off_Ucat + zc[p], nsum * 8, P->U.get() + P->Uoff_pair[p], nP(p) * 8, nP(p) * 8, V,
                                cudaMemcpyDeviceToDevice, s));

  // ---- overlaps S(p,q) = U_p^T U_q ----------------------------------------------------
  {
    std::vector<GemmProb<double>> pr;
    for (int p = 0; p < npairs; ++p)
      for (int q = 0; q < npairs; ++q) {
        if (!nP(p) || !nP(q)) continue;
        pr.push_back({P->U.get() + P->Uoff_pair[p], P->U.get() + P->Uoff_pair[q], pl + offS[(size_t)p * npairs + q],
                      (int)nP(p), (int)nP(q), v, (int)nP(p), (int)nP(q), (int)nP(q), 1, 0, 1.0, 0.0});
      }
    grouped_gemm<double>(pr, s);
  }
  auto Sblk = [&](int p, int q) { return offS[(size_t)p * npairs + q]; };

  tm.mark("  overlaps");
  // ---- mixed-pair ring blocks -------------------------------------------------------------
  // rank-(ov) parts, one GEMM per occupied y and family (Wc, Wd, Zt, Zd reassociated:
  //   -1/2 sum_{l,d} t[l,i,a,d] (kd|lc) -> -1/2 TU[i]^T GU[k];  1/2 sum u[i,l,a,d] L[l,d,k,c] -> 1/2 UU[i]^T LU[k];
  //   Zt[k,j][d,b] = sum (md|kc) t[m,j,b,c] -> GU[k]^T TU[j];  Zd[k,j][d,b] = sum L[k,d,m,c] u[j,m,b,c] -> LU[k]^T UU[j])
  {
    std::vector<GemmProb<double>> pr;
    for (int y = 0; y < o; ++y) {
      const int cl = (int)clen[y];
      if (!cl) continue;
      const int64_t b = cbase[y];
      pr.push_back({TUc.get() + b, GUc.get() + b, pl + offMCc[y], cl, cl, (int)OV, cl, cl, cl, 1, 0, -0.5, 0.0});
      pr.push_back({UUc.get() + b, LUc.get() + b, pl + offMDc[y], cl, cl, (int)OV, cl, cl, cl, 1, 0, 0.5, 0.0});
      pr.push_back({GUc.get() + b, TUc.get() + b, pl + offMZc[y], cl, cl, (int)OV, cl, cl, cl, 1, 0, 1.0, 0.0});
      pr.push_back({LUc.get() + b, UUc.get() + b, pl + offMZdc[y], cl, cl, (int)OV, cl, cl, cl, 1, 0, 1.0, 0.0});
    }
    grouped_gemm<double>(pr, s);
    GUc.release();
    LUc.release();
    // one-integral parts: MC += U(i,j)^T (ki|ac) U(k,j); MD += U(i,j)^T (2 (ai|kc) - (ki|ac)) U(j,k)
    // (jobs writing the same block go to separate calls)
    std::vector<Prog::PJ> j1, j2;
    const int64_t vv = V * V;
    for (int j = 0; j < o; ++j)
      for (int i = 0; i < o; ++i) {
        if (!G.n(i, j)) continue;
        for (int k = 0; k < o; ++k) {
          if (!G.n(k, j)) continue;
          j1.push_back({G.U(i, j), G.n(i, j), g_oovv.get() + ((int64_t)k * o + i) * vv, v, 0, G.U(k, j), G.n(k, j),
                        pl + ring_off(offMCc, j, i, k), (int)clen[j], 1.0, 1.0});
          j1.push_back({G.U(i, j), G.n(i, j), g_voov.get() + (int64_t)i * OV + (int64_t)k * V, (int)(O * O * V), 0,
                        G.U(j, k), G.n(j, k), pl + ring_off(offMDc, j, i, k), (int)clen[j], 2.0, 1.0});
          j2.push_back({G.U(i, j), G.n(i, j), g_oovv.get() + ((int64_t)k * o + i) * vv, v, 0, G.U(j, k), G.n(j, k),
                        pl + ring_off(offMDc, j, i, k), (int)clen[j], -1.0, 1.0});
        }
      }
    G.project(j1);
    G.project(j2);
  }
  tm.mark("  ring blocks");
  // ---- E3 / E4 blocks ---------------------------------------------------------------------------
  {
    std::vector<GemmProb<double>> pr;
    for (int k = 0; k < o; ++k) for (int l = 0; l < o; ++l) {
      int nn = G.n(k, l);
      if (!nn) continue;
      // Gh[k,l] = U(k,l)^T G^{lk}, G^{lk}[d,c] = (ld|kc)
      pr.push_back({G.U(k, l), g_ovov.get() + (int64_t)l * V * O * V + (int64_t)k * V, pl + offGh[k * o + l], nn, v, v, nn,
                    o * v, v, 1, 0, 1.0, 0.0});
      // Th[k,l] = U(k,l)^T t[k,l]
      pr.push_back({G.U(k, l), t + ((int64_t)k * o + l) * V * V, pl + offTh[k * o + l], nn, v, v, nn, v, v, 1, 0, 1.0, 0.0});
    }
    grouped_gemm<double>(pr, s);
    std::vector<Prog::PJ> jobs;
    for (int l = 0; l < o; ++l) for (int j = 0; j < o; ++j) {
      int nn = G.n(l, j);
      if (!nn) continue;
      // G4 rows k: U(l,j)^T X_k U(l,j), X_k[c,d] = (kd|lc)
      for (int k = 0; k < o; ++k)
        jobs.push_back({G.U(l, j), nn, g_ovov.get() + (int64_t)k * V * O * V + (int64_t)l * V, o * v, 1, G.U(l, j), nn,
                        pl + offG4[l * o + j] + (int64_t)k * pad(nn * nn), nn, 1.0, 0.0});
    }
    G.project(jobs);
  }
  // T4[(i,j)] = [n^2 x o], column k = vec(U(i,j)^T t[i,k] U(i,j)); keep [k][n^2] copies for e2m
  std::vector<DV> tb3(O * O);
  {
    std::vector<Prog::PJ> jobs;
    for (int i = 0; i < o; ++i) for (int j = 0; j < o; ++j) {
      int nn = G.n(i, j);
      tb3[i * o + j].alloc(std::max<int64_t>(1, O * nn * nn));
      if (!nn) continue;
      for (int k = 0; k < o; ++k)
        jobs.push_back({G.U(i, j), nn, t + ((int64_t)i * o + k) * V * V, v, 0, G.U(i, j), nn,
                        tb3[i * o + j].get() + (int64_t)k * nn * nn, nn, 1.0, 0.0});
    }
    G.project(jobs);
    for (int i = 0; i < o; ++i) for (int j = 0; j < o; ++j) {
      int64_t nn = G.n(i, j);
      if (!nn) continue;
      DV tmp(nn * nn * O);
      G.perm(tb3[i * o + j].get(), tmp.get(), {O, nn * nn}, {1, 0});
      PN_CUDA(cudaMemcpy2DAsync(pl + offT4[i * o + j], Op * 8, tmp.get(), O * 8, O * 8, nn * nn, cudaMemcpyDeviceToDevice, s));
    }
  }

  tm.mark("  global-term blocks");
  // R1 column blocks shared by all pairs: Lv1[b,c,(m,D)] = sum_d (2 (bc|md) - (bd|mc)) U^m[d,D],
  // GamAll[y][k][(m,D)] = sum_d (2 (ky|md) - (kd|my)) U^m[d,D]
  DV Lv1(std::max<int64_t>(1, V * V * L1)), GamAll(std::max<int64_t>(1, O * O * L1));
  // Lv1 is also a pool block (rows b*v + c, padded): sum_L Lv1[b,c,L] r_L is the v x v R1 part
  // of the E3 factor (it adds to FvR; the E3 products then apply t projected on both sides)
  if (L1 > 0) {
    Dims d = G.dm;
    d['L'] = L1;
    {   // 2 (bc|md) U^m: 2 sum_Q B[Q,b,c] BoU[Q,m,(m,D)]
      DV QL(N * L1);
      for (int m = 0; m < o; ++m)
        if (G.no(m))
          PN_CUDA(cudaMemcpy2DAsync(QL.get() + P->off_i[m], L1 * 8, BoU.get() + (int64_t)m * L1 + P->off_i[m], O * L1 * 8,
                                    G.no(m) * 8, N, cudaMemcpyDeviceToDevice, s));
      G.con(d, "Qbc", dBvv.get(), "QL", QL.get(), "bcL", Lv1.get(), 2.0, 0.0);
    }
    for (int m = 0; m < o; ++m) {   // - (bd|mc) U^m: - sum_Q BUo[Q,b,(m,D)] B[Q,m,c]
      const int nm = G.no(m);
      if (!nm) continue;
      Dims dm2 = G.dm;
      dm2['D'] = nm;
      DV BUm, Bm(N * V), tmp(V * V * nm);
      osv_cols(BUo.get(), N * V, m, BUm);
      PN_CUDA(cudaMemcpy2DAsync(Bm.get(), V * 8, dBov.get() + (int64_t)m * V, OV * 8, V * 8, N, cudaMemcpyDeviceToDevice, s));
      G.con(dm2, "QbD", BUm.get(), "Qc", Bm.get(), "bcD", tmp.get());
      G.add_block(Lv1.get() + P->off_i[m], L1, tmp.get(), nm, (int)(V * V), nm, -1.0);
    }
    PN_CUDA(cudaMemcpy2DAsync(pl + off_Lv1, L1p * 8, Lv1.get(), L1 * 8, L1 * 8, V * V, cudaMemcpyDeviceToDevice, s));
    std::vector<GemmProb<double>> pr;
    for (int m = 0; m < o; ++m) {
      if (!G.no(m)) continue;
      for (int y = 0; y < o; ++y)
        pr.push_back({Gam_can.get() + (int64_t)y * O * O * V + (int64_t)m * V, G.Uo(m), GamAll.get() + (int64_t)y * O * L1 + P->off_i[m],
                      o, G.no(m), v, o * v, G.no(m), (int)L1, 0, 0, 1.0, 0.0});
    }
    grouped_gemm<double>(pr, s);
  }

  tm.mark("  singles factors");
  // ---- pair-diagonal dense blocks D_p, singles -> doubles blocks A_DS_p, V_bar rows ------
  double* AS = pl + off_AS;
  for (int p = 0; p < npairs; ++p) {
    const int i = P->pair_i[p], j = P->pair_j[p];
    const int nn = (int)nP(p);
    if (!nn) continue;
    const double* Up = G.U(i, j);
    Dims d = G.dm;
    for (char c : std::string("ABCD")) d[c] = nn;
    d['K'] = OV;
    // DF factors of the pair: BU[Q,a,B] = sum_d Bvv[Q,a,d] U[d,B], BUt[Q,d,B] = sum_b Bvv[Q,b,d] U[b,B]
    DV BU(N * V * nn), BUt_own;
    G.con(d, "Qad", dBvv.get(), "dB", Up, "QaB", BU.get());
    const double* BUt = BU.get();
    if (!bsym) {
      BUt_own.alloc(N * V * nn);
      G.con(d, "Qbd", dBvv.get(), "bB", Up, "QdB", BUt_own.get());
      BUt = BUt_own.get();
    }
    DV Dtmp((int64_t)nn * nn * nn * nn);   // D_p, copied into its padded pool block at the end
    double* Dp = Dtmp.get();
    {   // ladder: Bb[Q,A,C] = U^T B^Q U, D_p = sum_Q Bb[Q,A,C] Bb[Q,B,D]
      DV Bb(N * nn * nn);
      G.con(d, "aA", Up, "QaC", BU.get(), "QAC", Bb.get());
      G.con(d, "QAC", Bb.get(), "QBD", Bb.get(), "ABCD", Dp);
    }
    // T2 ladder: sum_kl tb[kl]_AB gb[kl]_CD, gb[kl]_CD = sum_Q Bh[Q,k,C] Bh[Q,l,D], tb[kl] = U^T t[k,l] U
    DV Bh(N * O * nn), tb(O * O * nn * nn);
    G.con(d, "Qkc", dBov.get(), "cC", Up, "QkC", Bh.get());
    {
      DV gb(O * O * nn * nn), X(O * O * V * nn);
      G.con(d, "QkC", Bh.get(), "QlD", Bh.get(), "klCD", gb.get());
      // tb[kl] = U^T t[k,l] U for k <= l; tb[lk] = tb[kl]^T (t[l,k] = t[k,l]^T)
      {
        std::vector<GemmProb<double>> pr;
        for (int k = 0; k < o; ++k)   // X[k,l,a,B] = sum_b t[k,l,a,b] U[b,B], l >= k
          pr.push_back({t + ((int64_t)k * o + k) * V * V, Up, X.get() + ((int64_t)k * o + k) * V * nn, (o - k) * v, nn, v, v,
                        nn, nn, 0, 0, 1.0, 0.0});
        grouped_gemm<double>(pr, s);
        pr.clear();
        for (int k = 0; k < o; ++k)
          for (int l = k; l < o; ++l)
            pr.push_back({Up, X.get() + ((int64_t)k * o + l) * V * nn, tb.get() + ((int64_t)k * o + l) * nn * nn, nn, nn, v,
                          nn, nn, nn, 1, 0, 1.0, 0.0});
        grouped_gemm<double>(pr, s);
        k_mirror_lower<<<gsz((size_t)o * o * nn * nn), 256, 0, s>>>(tb.get(), o, nn);
        PN_CUDA(cudaGetLastError());
      }
      G.con(d, "klAB", tb.get(), "klCD", gb.get(), "ABCD", Dp, 1.0, 1.0);
    }
    DV Fb(nn * nn);
    G.project({{Up, nn, FvvI.get(), v, 0, Up, nn, Fb.get(), nn, 1.0, 0.0}});
    k_add_fock_kron<<<gsz((size_t)nn * nn * nn * nn), 256, 0, s>>>(Dp, Fb.get(), nn);
    PN_CUDA(cudaGetLastError());
    PN_CUDA(cudaMemcpy2DAsync(pl + offD[p], pad(nn * nn) * 8, Dp, (int64_t)nn * nn * 8, (int64_t)nn * nn * 8, (int64_t)nn * nn,
                              cudaMemcpyDeviceToDevice, s));

    // P_x[Q,A,D] = sum_a U[a,A] (B^Q U^x)[a,D] for the pair's OSVs x = i, j
    const int ni = G.no(i), nj = G.no(j);
    DV Pi, Pj;
    auto make_P = [&](int x, DV& out) {
      const int nx = G.no(x);
      if (!nx) return;
      DV BUx;
      osv_cols(BUo.get(), N * V, x, BUx);
      Dims dx = d;
      dx['D'] = nx;
      out.alloc(N * nn * nx);
      G.con(dx, "aA", Up, "QaD", BUx.get(), "QAD", out.get());
    };
    make_P(i, Pi);
    if (j != i) make_P(j, Pj);
    const DV& Pjr = j != i ? Pj : Pi;

    // ---- V_bar rows of A_S (sigma1 from R2 through (ad|kc)): for the pair's OSV owners x with k
    // the other index, Vb[A,C,D] = sum_{a,c,d} U^x[a,A] (ad|kc) U[c,C] U[d,D]
    //   = sum_Q (U^x^T B^Q U)[A,D] Bh[Q,k,C]; added as 2 Vb - Vb^T (CD) in the orientation of
    //   the stored block
    for (int side = 0; side < (i == j ? 1 : 2); ++side) {
      const int x = side == 0 ? j : i, k = side == 0 ? i : j;
      const int nx = G.no(x);
      if (!nx) continue;
      Dims dx = d;
      dx['X'] = nx;
      DV Px(N * nx * nn), Bk(N * nn), Vb(nx * nn * nn), Vt(nx * nn * nn);
      G.con(dx, "aX", G.Uo(x), "QaD", BU.get(), "QXD", Px.get());
      PN_CUDA(cudaMemcpy2DAsync(Bk.get(), nn * 8, Bh.get() + (int64_t)k * nn, O * nn * 8, nn * 8, N, cudaMemcpyDeviceToDevice, s));
      G.con(dx, "QXD", Px.get(), "QC", Bk.get(), "XCD", Vb.get());
      G.perm(Vb.get(), Vt.get(), {nx, nn, nn}, {0, 2, 1});
      const bool direct = k <= x;
      double* rows = AS + P->off_i[x] * Lp + P->off_ij[p];
      G.add_block(rows, Lp, direct ? Vb.get() : Vt.get(), nn * nn, nx, nn * nn, 2.0);
      G.add_block(rows, Lp, direct ? Vt.get() : Vb.get(), nn * nn, nx, nn * nn, -1.0);
    }

    // ---- singles -> doubles dense block A_DS_p (n^2 x L1) --------------------------------------
    double* Y = pl + offADS[p];
    // (c1)+(c3): columns of OSV i and OSV j
    for (int side = 0; side < 2; ++side) {
      const int x = side == 0 ? i : j;      // OSV whose r1 enters
      const int nx = side == 0 ? ni : nj;
      if (!nx) continue;
      d['C'] = nx;
      DV K3(nn * nn * nx), H(O * O * nx);
      if (side == 0) {  // sum U[a,A] (ac|bj) U^i[c,C] U[b,B] = sum_Q P_i[Q,A,C] (sum_b B[Q,b,j] U[b,B])
        DV bj(N * nn);
        G.con(d, "Qb", BvoT.get() + (int64_t)j * N * V, "bB", Up, "QB", bj.get());
        G.con(d, "QAC", Pi.get(), "QB", bj.get(), "ABC", K3.get());
        G.con(d, "kcl", govoo_j.get() + (int64_t)j * O * V * O, "cC", G.Uo(i), "klC", H.get());
      } else {          // sum U[a,A] (ai|bc) U^j[c,C] U[b,B] = sum_Q (sum_a B[Q,a,i] U[a,A]) P_j[Q,B,C]
        DV ai(N * nn);
        G.con(d, "Qa", BvoT.get() + (int64_t)i * N * V, "aA", Up, "QA", ai.get());
        G.con(d, "QA", ai.get(), "QBC", Pjr.get(), "ABC", K3.get());
        G.con(d, "klc", gooov_i.get() + (int64_t)i * O * O * V, "cC", G.Uo(j), "klC", H.get());
      }
      G.con(d, "klAB", tb.get(), "klC", H.get(), "ABC", K3.get(), 1.0, 1.0);
      G.add_block(Y + P->off_i[x], L1p, K3.get(), nx, nn * nn, nx, 1.0);
    }
    // (c1)+(c2): outer products with S(ij,k) r1_k; wa[k,B] = -sum_b U[b,B] ((ki|bj) + Y1[i,j,k,b]),
    // wb[k,A] = -sum_a U[a,A] ((ai|kj) + Y2[i,j,a,k]) with the T2 parts through the DF factors:
    //   sum_b U[b,B] Y1[i,j,k,b] = sum_{Q,c} B[Q,k,c] sum_d t[i,j,c,d] BUt[Q,d,B]
    //   sum_a U[a,A] Y2[i,j,a,k] = sum_{Q,d} B[Q,k,d] sum_c t[i,j,c,d] BUt[Q,c,A]
    {
      DV Sk(nn * std::max<int64_t>(1, L1)), wa(O * nn), wb(O * nn);
      std::vector<GemmProb<double>> pr;
      for (int k = 0; k < o; ++k)
        if (G.no(k))
          pr.push_back({Up, G.Uo(k), Sk.get() + P->off_i[k], nn, G.no(k), v, nn, G.no(k), (int)L1, 1, 0, 1.0, 0.0});
      pr.push_back({wa_can.get() + ((int64_t)i * o + j) * O * V, Up, wa.get(), o, nn, v, v, nn, nn, 0, 0, -1.0, 0.0});
      pr.push_back({wb_can.get() + ((int64_t)i * o + j) * O * V, Up, wb.get(), o, nn, v, v, nn, nn, 0, 0, -1.0, 0.0});
      grouped_gemm<double>(pr, s);
      const double* tij = t + ((int64_t)i * o + j) * V * V;
      DV Z(N * V * nn);
      G.con(d, "cd", tij, "QdB", BUt, "QcB", Z.get());
      G.con(d, "Qkc", dBov.get(), "QcB", Z.get(), "kB", wa.get(), -1.0, 1.0);
      G.con(d, "cd", tij, "QcA", BUt, "QdA", Z.get());
      G.con(d, "Qkd", dBov.get(), "QdA", Z.get(), "kA", wb.get(), -1.0, 1.0);
      for (int k = 0; k < o; ++k) {
        if (!G.no(k)) continue;
        G.kron(Y + P->off_i[k], L1p, Sk.get() + P->off_i[k], (int)L1, wa.get() + (int64_t)k * nn, nn, G.no(k), 0, 1.0);
        G.kron(Y + P->off_i[k], L1p, Sk.get() + P->off_i[k], (int)L1, wb.get() + (int64_t)k * nn, nn, G.no(k), 1, 1.0);
      }
    }
    // exchange factors of the Qa / Q1 terms: Yx[A,c,k,D] = sum_Q BUt[Q,c,A] BoU[Q,k,(x,D)] for the
    // pair's OSVs x (sum_{a,d} U[a,A] U^x[d,D] (ac|kd) = Yx[A,c,k,D])
    DV Yi, Yj;
    auto make_Y = [&](int x, DV& out) {
      const int nx = G.no(x);
      if (!nx) return;
      DV BoUx;
      osv_cols(BoU.get(), N * O, x, BoUx);
      Dims dx = d;
      dx['D'] = nx;
      out.alloc(nn * V * O * nx);
      G.con(dx, "QcA", BUt, "QkD", BoUx.get(), "AckD", out.get());
    };
    make_Y(i, Yi);
    if (j != i) make_Y(j, Yj);
    auto Yof = [&](int x) -> const DV& { return x == i ? Yi : Yj; };
    auto Pof = [&](int x) -> const DV& { return x == i ? Pi : Pjr; };
    // ordered (x,y) contributions (the P-symmetrised part): (i,j) and, if i < j, (j,i) transposed
    for (int ord = 0; ord < (i == j ? 1 : 2); ++ord) {
      const int x = ord == 0 ? i : j, y = ord == 0 ? j : i;
      DV Yc(nn * nn * std::max<int64_t>(1, L1));
      Yc.zero(s);
      d['L'] = L1;
      // W factors of the pair: ut[k,c,B] = sum_b U[b,B] u[y,k,b,c] = UU[y], ty = sum_b U[b,B] t[k,y,b,c] = TU[y],
      // tx = TU[x]
      DV ut, ty, tx;
      cat_block(UUc, y, x, ut);
      cat_block(TUc, y, x, ty);
      cat_block(TUc, x, y, tx);
      // Qa (OSV x): sum U[a,A] U^x[d,D] [(ad|kc) ut - 1/2 (ac|kd) (ut + ty)][k,c,B];
      // Q1 (OSV y): - sum U[a,A] U^y[d,D] (ac|kd) tx[k,c,B]
      if (G.no(x)) {
        const int nx = G.no(x);
        Dims dx = d;
        dx['D'] = nx;
        DV wq(N * nn), K3(nn * nn * nx), W0(OV * nn);
        G.con(dx, "QK", dBov.get(), "KB", ut.get(), "QB", wq.get());
        G.con(dx, "QAD", Pof(x).get(), "QB", wq.get(), "ABD", K3.get());
        PN_CUDA(cudaMemcpyAsync(W0.get(), ut.get(), W0.n * 8, cudaMemcpyDeviceToDevice, s));
        axpby<double>(W0.get(), ty.get(), 1.0, 1.0, W0.n, s);
        G.con(dx, "AckD", Yof(x).get(), "kcB", W0.get(), "ABD", K3.get(), -0.5, 1.0);
        G.add_block(Yc.get() + P->off_i[x], L1, K3.get(), nx, nn * nn, nx, 1.0);
      }
      if (G.no(y)) {
        const int ny = G.no(y);
        Dims dy = d;
        dy['D'] = ny;
        DV K3(nn * nn * ny);
        G.con(dy, "AckD", Yof(y).get(), "kcB", tx.get(), "ABD", K3.get(), -1.0, 0.0);
        G.add_block(Yc.get() + P->off_i[y], L1, K3.get(), ny, nn * nn, ny, 1.0);
      }
      if (L1 > 0) {
        // (the Lambda term, sum_c t[x,y,a,c] sum_{m,d} (2 (bc|md) - (bd|mc)) r_m,d, is applied per
        // call through FvR: see Lv1 above)
        // e2m: - sum_k tb3[x,k,y] Gam_y[k, L]
        G.con(d, "kAB", tb3[x * o + y].get(), "kL", GamAll.get() + (int64_t)y * O * L1, "ABL", Yc.get(), -1.0, 1.0);
        // qb kron: S(xy,m)[A,C] qb[x,y,m][B], qb = sum_b Qb[m,x,y,b] U[b,B] with
        // Qb[m,x,y,b] = Q2[m,y,x,b] + 1/2 Q2[m,x,y,b] - Q5[m,x,y,b] + 1/2 Q6[m,x,y,b]:
        //   Q2 part: G2q[y] tx + 1/2 G2q[x] ty;  Q5: -g_ooov[m,x,(k,c)] ut;  Q6: 1/2 G6q[x] ut
        DV Sk(nn * L1), qb(O * nn), e2a(O * nn);
        std::vector<GemmProb<double>> pr;
        for (int m = 0; m < o; ++m)
          if (G.no(m))
            pr.push_back({Up, G.Uo(m), Sk.get() + P->off_i[m], nn, G.no(m), v, nn, G.no(m), (int)L1, 1, 0, 1.0, 0.0});
        grouped_gemm<double>(pr, s);
        const int ov = (int)OV;
        grouped_gemm<double>({{G2q.get() + (int64_t)y * O * OV, tx.get(), qb.get(), o, nn, ov, ov, nn, nn, 0, 0, 1.0, 0.0}}, s);
        grouped_gemm<double>({{G2q.get() + (int64_t)x * O * OV, ty.get(), qb.get(), o, nn, ov, ov, nn, nn, 0, 0, 0.5, 1.0}}, s);
        grouped_gemm<double>({{g_ooov.get() + (int64_t)x * OV, ut.get(), qb.get(), o, nn, ov, (int)(O * OV), nn, nn, 0, 0, -1.0, 1.0}}, s);
        grouped_gemm<double>({{G6q.get() + (int64_t)x * O * OV, ut.get(), qb.get(), o, nn, ov, ov, nn, nn, 0, 0, 0.5, 1.0}}, s);
        for (int m = 0; m < o; ++m)
          if (G.no(m))
            G.kron(Yc.get() + P->off_i[m], L1, Sk.get() + P->off_i[m], (int)L1, qb.get() + (int64_t)m * nn, nn, G.no(m), 0, 1.0);
        if (t1) {
          // e2a: - (t[x,y] Fov[m]) projected, b-side S(xy,m)
          DV dFov(O * V), ecan(O * V);
          dFov.upload(Fov.data(), Fov.size(), s);
          grouped_gemm<double>({{dFov.get(), t + ((int64_t)x * o + y) * V * V, ecan.get(), o, v, v, v, v, v, 0, 1, 1.0, 0.0}}, s);
          grouped_gemm<double>({{ecan.get(), Up, e2a.get(), o, nn, v, v, nn, nn, 0, 0, -1.0, 0.0}}, s);
          for (int m = 0; m < o; ++m)
            if (G.no(m))
              G.kron(Yc.get() + P->off_i[m], L1, Sk.get() + P->off_i[m], (int)L1, e2a.get() + (int64_t)m * nn, nn, G.no(m), 1, 1.0);
          // e2j: - sum_m tb3[x,m,y] (Fov[m] . U^y)  (columns of OSV y)
          if (G.no(y)) {
            DV phi(O * G.no(y));
            grouped_gemm<double>({{dFov.get(), G.Uo(y), phi.get(), o, G.no(y), v, v, G.no(y), G.no(y), 0, 0, 1.0, 0.0}}, s);
            Dims d3 = d; d3['C'] = G.no(y);
            DV K3(nn * nn * G.no(y));
            G.con(d3, "kAB", tb3[x * o + y].get(), "kC", phi.get(), "ABC", K3.get());
            G.add_block(Yc.get() + P->off_i[y], L1, K3.get(), G.no(y), nn * nn, G.no(y), -1.0);
          }
        }
      }
      // accumulate into A_DS_p: (i,j) as is, (j,i) with rows transposed; for i == j both
      if (ord == 0) G.add_block(Y, L1p, Yc.get(), L1, nn * nn, (int)L1, 1.0, 0);
      if (ord == 1 || i == j) G.add_block(Y, L1p, Yc.get(), L1, nn * nn, (int)L1, 1.0, nn);
    }
    // no synchronisation per pair: temporaries return to this thread's cache and are
    // reused in stream order, so the host plans the next pair while this one runs
  }
  TUc.release();
  UUc.release();
  BUo.release();

  tm.mark("  pair loop (D, A_DS)");
  // ---- singles rows A_S (L1 x L; the V_bar parts were added in the pair loop) ---------------
  if (L1 > 0) {
    // singles-singles: U^i^T [sum_{k,c} u[i,k,a,c] L[k,c,m,d] + 2 (ai|md) - (mi|ad) + delta_im Xv - delta_ad Xo[m,i]] U^m
    // with the first term as UUo[i]^T LUo[m]: UUo[i][(k,c),A] = sum_a u[i,k,a,c] U^i[a,A],
    // LUo[m][(k,c),D] = sum_d L[m,d,k,c] U^m[d,D]
    DV UUo(OV * L1), LUo(OV * L1);
    std::vector<GemmProb<double>> pr;
    for (int m = 0; m < o; ++m) {
      const int nm = G.no(m);
      if (!nm) continue;
      pr.push_back({uS.get() + (int64_t)m * OV * V, G.Uo(m), UUo.get() + P->off_i[m], (int)OV, nm, v, v, nm, (int)L1, 0, 0, 1.0, 0.0});
      pr.push_back({L_ovov.get() + (int64_t)m * V * OV, G.Uo(m), LUo.get() + P->off_i[m], (int)OV, nm, v, (int)OV, nm, (int)L1, 1, 0, 1.0, 0.0});
    }
    grouped_gemm<double>(pr, s);
    grouped_gemm<double>({{UUo.get(), LUo.get(), AS, (int)L1, (int)L1, (int)OV, (int)L1, (int)L1, (int)Lp, 1, 0, 1.0, 1.0}}, s);
    std::vector<Prog::PJ> ja, jb, jc;
    DV eye(V * V);
    {
      std::vector<double> I((size_t)V * V, 0.0);
      for (int a = 0; a < v; ++a) I[(size_t)a * v + a] = 1.0;
      eye.upload(I.data(), I.size(), s);
    }
    for (int i = 0; i < o; ++i) {
      if (!G.no(i)) continue;
      for (int m = 0; m < o; ++m) {
        if (!G.no(m)) continue;
        double* out = AS + P->off_i[i] * Lp + P->off_i[m];
        ja.push_back({G.Uo(i), G.no(i), g_voov.get() + (int64_t)i * OV + (int64_t)m * V, (int)(O * O * V), 0, G.Uo(m), G.no(m),
                      out, (int)Lp, 2.0, 1.0});
        jb.push_back({G.Uo(i), G.no(i), g_oovv.get() + ((int64_t)m * o + i) * V * V, v, 0, G.Uo(m), G.no(m), out, (int)Lp,
                      -1.0, 1.0});
        if (m == i) jc.push_back({G.Uo(i), G.no(i), Xv.get(), v, 0, G.Uo(i), G.no(i), out, (int)Lp, 1.0, 1.0});
      }
    }
    G.project(ja);
    G.project(jb);
    G.project(jc);
    std::vector<Prog::PJ> jd;   // - Xo[m,i] U^i^T U^m
    for (int i = 0; i < o; ++i)
      for (int m = 0; m < o; ++m)
        if (G.no(i) && G.no(m) && Xo_h[m * o + i] != 0.0)
          jd.push_back({G.Uo(i), G.no(i), eye.get(), v, 0, G.Uo(m), G.no(m), AS + P->off_i[i] * Lp + P->off_i[m], (int)Lp,
                        -Xo_h[m * o + i], 1.0});
    G.project(jd);
  }
  for (int i = 0; i < o; ++i) {
    const int ni = G.no(i);
    if (!ni) continue;
    double* Ai = AS + P->off_i[i] * Lp;
    {   // h_bar term (and F_ov term with T1): -S(i,kl) UR^{kl} h
      DV S(ni * std::max<int64_t>(1, L - L1)), hb((int64_t)O * O * v);
      std::vector<GemmProb<double>> pr;
      for (int q = 0; q < npairs; ++q)
        if (nP(q))
          pr.push_back({G.Uo(i), P->U.get() + P->Uoff_pair[q], S.get() + (P->off_ij[q] - L1), ni, (int)nP(q), v, ni,
                        (int)nP(q), (int)(L - L1), 1, 0, 1.0, 0.0});
      for (int k = 0; k < o; ++k) for (int l = 0; l < o; ++l) {
        int nn = G.n(k, l);
        if (!nn) continue;
        pr.push_back({G.U(k, l), gooov_i.get() + (int64_t)i * O * O * V + ((int64_t)k * o + l) * V, hb.get() + ((int64_t)k * o + l) * V,
                      nn, 1, v, nn, 1, 1, 1, 0, 1.0, 0.0});
      }
      grouped_gemm<double>(pr, s);
      for (int k = 0; k < o; ++k) for (int l = 0; l < o; ++l) {
        const int q = P->pidx[k][l];
        const int nn = (int)nP(q);
        if (!nn) continue;
        const double* Sq = S.get() + (P->off_ij[q] - L1);
        const double* w = hb.get() + ((int64_t)k * o + l) * V;
        double* out = Ai + P->off_ij[q];
        const int lds = (int)(L - L1);
        if (k <= l) { G.kron(out, Lp, Sq, lds, w, nn, ni, 2, -2.0); G.kron(out, Lp, Sq, lds, w, nn, ni, 3, 1.0); }
        else { G.kron(out, Lp, Sq, lds, w, nn, ni, 3, -2.0); G.kron(out, Lp, Sq, lds, w, nn, ni, 2, 1.0); }
      }
      if (t1) {   // + S(i,ik) UR^{ik} fb, fb = U(i,k)^T Fov[k]
        DV dFov(O * V), fb(O * V);
        dFov.upload(Fov.data(), Fov.size(), s);
        std::vector<GemmProb<double>> pf;
        for (int k = 0; k < o; ++k)
          if (G.n(i, k)) pf.push_back({G.U(i, k), dFov.get() + (int64_t)k * V, fb.get() + (int64_t)k * V, G.n(i, k), 1, v, G.n(i, k), 1, 1, 1, 0, 1.0, 0.0});
        grouped_gemm<double>(pf, s);
        for (int k = 0; k < o; ++k) {
          const int q = P->pidx[i][k];
          const int nn = (int)nP(q);
          if (!nn) continue;
          const double* Sq = S.get() + (P->off_ij[q] - L1);
          const double* w = fb.get() + (int64_t)k * V;
          double* out = Ai + P->off_ij[q];
          const int lds = (int)(L - L1);
          if (i <= k) { G.kron(out, Lp, Sq, lds, w, nn, ni, 2, 2.0); G.kron(out, Lp, Sq, lds, w, nn, ni, 3, -1.0); }
          else { G.kron(out, Lp, Sq, lds, w, nn, ni, 3, 2.0); G.kron(out, Lp, Sq, lds, w, nn, ni, 2, -1.0); }
        }
      }
    }
  }
  G.sync();

  tm.mark("  singles rows");
  // ---- problem lists ------------------------------------------------------------------------------
  // per-vector work: FvR (v x v), FoR (o x o), Y (sum n_p x v), Z (v x sum n_p)
  P->work_fvr = 0;
  P->work_for = V * V;
  P->work_y = P->work_for + O * O;
  P->work_z = P->work_y + nsum * V;
  P->work_len = P->work_z + V * nsum;
  auto blk = [&](int x, int y) { return P->pidx[x][y]; };
  // sandwich helper: C(stored out pair, transposed?) += al * A * X(stored q, tx) * B
  auto add_sw = [&](std::vector<SProb>& L_, int cbuf, int64_t coff, int ldc, int tc, int M, int Nn, int abuf, int64_t aoff,
                    int lda, int ta, int K1, int xbuf, int64_t xoff, int ldx, int tx, int K2, int bbuf, int64_t boff,
                    int ldb, int tb, double al, double xb = 0.0) {
    if (M <= 0 || Nn <= 0 || K1 <= 0 || K2 <= 0 || al == 0.0) return;
    for (int m0 = 0; m0 < M; m0 += 64)
      for (int n0 = 0; n0 < Nn; n0 += 64) {
        SProb q{};
        q.a_off = aoff; q.x_off = xoff; q.b_off = boff; q.c_off = coff;
        q.a_buf = abuf; q.x_buf = xbuf; q.b_buf = bbuf; q.c_buf = cbuf;
        q.M = M; q.K1 = K1; q.K2 = K2; q.N = Nn;
        q.lda = lda; q.ldx = ldx; q.ldb = ldb; q.ldc = ldc;
        q.ta = ta; q.tx = tx; q.tb = tb; q.tc = tc;
        q.m0 = m0; q.n0 = n0; q.alpha = al; q.xb = xb;
        L_.push_back(q);
        int tr = abuf == B_NONE ? std::min(64, M - m0) : K1;
        G.smem = std::max(G.smem, tr * std::min(64, Nn - n0));
      }
  };
  auto add_gemv = [&](std::vector<VProb>& L_, int64_t aoff, int M, int K, int lda, int xbuf, int64_t xoff, int xs, int xvn,
                      int cbuf, int64_t coff, int cs, int cvn, double al) {
    if (M <= 0 || K <= 0 || al == 0.0) return;
    // one row group per tile: a warp streams its rows once, so tiles with more groups
    // would serialise their load latencies (measured slower at the medium workload)
    const int groups = 1;
    for (int m0 = 0; m0 < M; m0 += groups * GEMV_ROWS)
      for (int k0 = 0; k0 < K; k0 += GEMV_KC) {
        VProb q{};
        q.a_off = aoff; q.x_off = xoff; q.c_off = coff;
        q.x_buf = xbuf; q.c_buf = cbuf;
        q.M = M; q.K = K; q.lda = lda;
        q.x_stride = xs; q.c_stride = cs; q.xvec_n = xvn; q.cvec_n = cvn;
        q.m0 = m0; q.mlen = std::min(groups * GEMV_ROWS, M - m0);
        q.k0 = k0; q.klen = std::min(GEMV_KC, K - k0); q.alpha = al;
        L_.push_back(q);
      }
  };
  // dense helper: C += al opA(A) opB(B), tiles of `tile`, K split in chunks of kchunk
  auto add_dense = [&](std::vector<DProb>& L_, int tile, int kchunk, int cbuf, int64_t coff, int ldc, int tc, int M,
                       int Nn, int abuf, int64_t aoff, int lda, int ta, int K, int bbuf, int64_t boff, int ldb, int tb,
                       double al) {
    if (M <= 0 || Nn <= 0 || K <= 0 || al == 0.0) return;
    const int tm = tile, tn = tile == DENSE_TILE_TC ? 64 : tile;   // tile rows, tile columns
    for (int m0 = 0; m0 < M; m0 += tm)
      for (int n0 = 0; n0 < Nn; n0 += tn)
        for (int k0 = 0; k0 < K; k0 += kchunk) {
          DProb q{};
          q.a_off = aoff; q.b_off = boff; q.c_off = coff;
          q.a_buf = abuf; q.b_buf = bbuf; q.c_buf = cbuf;
          q.M = M; q.N = Nn; q.K = K;
          q.lda = lda; q.ldb = ldb; q.ldc = ldc;
          q.ta = ta; q.tb = tb; q.tc = tc;
          q.m0 = m0; q.n0 = n0; q.k0 = k0; q.klen = std::min(kchunk, K - k0); q.alpha = al;
          q.tile_m = tm; q.tile_n = tn;
          L_.push_back(q);
        }
  };
  auto Ro = [&](int x, int y) { return P->off_ij[blk(x, y)]; };          // stored block offset
  auto Rt = [&](int x, int y) { return x > y ? 1 : 0; };                  // R^{xy} = stored^T ?
  // Phase 1: E3 virtual intermediate FvR (v x v) and E4 occupied intermediate FoR (o x o).
  // FvR = -sum_kl U^{kl} (2 R^{kl} - R^{kl T}) Gh[k,l] = -U_cat Y, where the rows of Y that
  // belong to stored pair q collect (2 R^{kl} - R^{kl T}) Gh[k,l] over the ordered (k,l) of q.
  for (int k = 0; k < o; ++k) for (int l = 0; l < o; ++l) {
    const int nn = G.n(k, l);
    if (!nn) continue;
    const int q = blk(k, l);
    add_sw(G.sp1, B_WORK, P->work_y + zc[q] * V, v, 0, nn, v, B_NONE, 0, 0, 0, nn, B_RIN, Ro(k, l), nn, Rt(k, l), nn,
           B_POOL, offGh[k * o + l], v, 0, 2.0, -0.5);
    // FoR[:, j] += G4[(l,j)] vec(2 R^{lj} - R^{lj T})   (here (l, j) = (k, l))
    const int lj_l = k, lj_j = l;
    add_gemv(G.vp1, offG4[lj_l * o + lj_j], o, nn * nn, (int)pad(nn * nn), B_RIN, Ro(lj_l, lj_j), 1, Rt(lj_l, lj_j) ? nn : 0, B_WORK,
             P->work_for + lj_j, o, 0, 2.0);
    add_gemv(G.vp1, offG4[lj_l * o + lj_j], o, nn * nn, (int)pad(nn * nn), B_RIN, Ro(lj_l, lj_j), 1, Rt(lj_l, lj_j) ? 0 : nn, B_WORK,
             P->work_for + lj_j, o, 0, -1.0);
  }
  add_dense(G.dp1, DENSE_TILE_TC, 256, B_WORK, P->work_fvr, v, 0, v, v, B_POOL, off_Ucat, (int)nsum, 0, (int)nsum, B_WORK, P->work_y, v,
            0, -1.0);
  // FvR[b,c] += sum_L Lv1[b,c,L] r1_L (the Lambda term of the singles couplings)
  if (L1 > 0)
    add_gemv(G.vp1, off_Lv1, (int)(V * V), (int)L1, (int)L1p, B_RIN, 0, 1, 0, B_WORK, P->work_fvr, 1, 0, 1.0);
  // Phase 2 prologue: Z = FvR^T U_cat (v x sum n_p), read by the E3 products below
  add_dense(G.dp2, DENSE_TILE_TC, 1 << 30, B_WORK, P->work_z, (int)nsum, 0, v, (int)nsum, B_WORK, P->work_fvr, v, 1, v, B_POOL, off_Ucat,
            (int)nsum, 0, 1.0);
  {   // the same two products, whole
    std::vector<DProb> g1, g2;
    add_dense(g1, 1 << 30, 1 << 30, B_WORK, P->work_fvr, v, 0, v, v, B_POOL, off_Ucat, (int)nsum, 0, (int)nsum, B_WORK,
              P->work_y, v, 0, -1.0);
    add_dense(g2, 1 << 30, 1 << 30, B_WORK, P->work_z, (int)nsum, 0, v, (int)nsum, B_WORK, P->work_fvr, v, 1, v, B_POOL,
              off_Ucat, (int)nsum, 0, 1.0);
    P->prog.h_gfull.clear();
    if (g1.size() == 1 && g2.size() == 1) P->prog.h_gfull = {g1[0], g2[0]};
  }
  // Phase 2
  for (int p = 0; p < npairs; ++p) {
    const int nn = (int)nP(p);
    if (!nn) continue;
    add_gemv(G.vp2, offD[p], nn * nn, nn * nn, (int)pad(nn * nn), B_RIN, P->off_ij[p], 1, 0, B_SOUT, P->off_ij[p], 1, 0, 1.0);
    add_gemv(G.vp2, offADS[p], nn * nn, (int)L1, (int)L1p, B_RIN, 0, 1, 0, B_SOUT, P->off_ij[p], 1, 0, 1.0);
  }
  for (int i = 0; i < o; ++i)
    add_gemv(G.vp2, off_AS + P->off_i[i] * Lp, G.no(i), (int)L, (int)Lp, B_RIN, 0, 1, 0, B_SOUT, P->off_i[i], 1, 0, 1.0);
  // ordered (i,j) contributions go to stored {i,j}; transposed when i > j; twice when i == j
  auto targets = [&](int i, int j, std::vector<int>& tcs) {
    tcs.clear();
    if (i < j) tcs.push_back(0); else if (i > j) tcs.push_back(1); else { tcs.push_back(0); tcs.push_back(1); }
  };
  std::vector<int> tcs;
  for (int i = 0; i < o; ++i) for (int j = 0; j < o; ++j) {
    const int nij = G.n(i, j);
    if (!nij) continue;
    const int pij = blk(i, j);
    targets(i, j, tcs);
    for (int tc : tcs) {
      const int64_t co = P->off_ij[pij];
      // E4 phase 2: -sum_k FoR[k,j] vec(tb3[i,k,j])
      add_gemv(G.vp2, offT4[i * o + j], nij * nij, o, (int)Op, B_WORK, P->work_for + j, o, 0, B_SOUT, co, 1, tc ? nij : 0, -1.0);
      // E3 phase 2: Th[i,j] FvR^T U(i,j) = Th[i,j] Z[:, columns of pair {i,j}]
      add_dense(G.dp3, 32, 1 << 30, B_SOUT, co, nij, tc, nij, nij, B_POOL, offTh[i * o + j], v, 0, v, B_WORK,
                P->work_z + zc[pij], (int)nsum, 0, 1.0);
      for (int k = 0; k < o; ++k) {
        const int nkj = G.n(k, j), nki = G.n(k, i), njk = G.n(j, k), nik = G.n(i, k);
        const int pkj = blk(k, j), pki = blk(k, i), pjk = blk(j, k), pik = blk(i, k);
        // C1: -1/2 MC[i,j,k] R^{kj T} S(kj,ij)
        add_sw(G.sp2, B_SOUT, co, nij, tc, nij, nij, B_POOL, ring_off(offMCc, j, i, k), (int)clen[j], 0, nkj, B_RIN, Ro(k, j), nkj,
               1 - Rt(k, j), nkj, B_POOL, Sblk(pkj, pij), nij, 0, -0.5);
        // C2: -MC[j,i,k] R^{ki T} S(ki,ij)
        add_sw(G.sp2, B_SOUT, co, nij, tc, nij, nij, B_POOL, ring_off(offMCc, i, j, k), (int)clen[i], 0, nki, B_RIN, Ro(k, i), nki,
               1 - Rt(k, i), nki, B_POOL, Sblk(pki, pij), nij, 0, -1.0);
        // C3: +1/4 S(ij,ki) R^{ki} MZ[k,i,j]
        add_sw(G.sp2, B_SOUT, co, nij, tc, nij, nij, B_POOL, Sblk(pij, pki), nki, 0, nki, B_RIN, Ro(k, i), nki, Rt(k, i),
               nki, B_POOL, ring_off(offMZc, i, k, j), (int)clen[i], 0, 0.25);
        // C4: +1/2 S(ij,kj) R^{kj} MZ[k,j,i]
        add_sw(G.sp2, B_SOUT, co, nij, tc, nij, nij, B_POOL, Sblk(pij, pkj), nkj, 0, nkj, B_RIN, Ro(k, j), nkj, Rt(k, j),
               nkj, B_POOL, ring_off(offMZc, j, k, i), (int)clen[j], 0, 0.5);
        // D1: MD[i,j,k] (R^{jk T} - 1/2 R^{jk}) S(jk,ij)
        add_sw(G.sp2, B_SOUT, co, nij, tc, nij, nij, B_POOL, ring_off(offMDc, j, i, k), (int)clen[j], 0, njk, B_RIN, Ro(j, k), njk,
               1 - Rt(j, k), njk, B_POOL, Sblk(pjk, pij), nij, 0, 1.0, -0.5);
        // D2: S(ij,ik) (1/2 R^{ik} - 1/4 R^{ik T}) MZd[k,i,j]
        add_sw(G.sp2, B_SOUT, co, nij, tc, nij, nij, B_POOL, Sblk(pij, pik), nik, 0, nik, B_RIN, Ro(i, k), nik, Rt(i, k),
               nik, B_POOL, ring_off(offMZdc, i, k, j), (int)clen[i], 0, 0.5, -0.5);
        // E2: -Foo~[k,j] S(ij,ik) R^{ik} S(ik,ij)
        add_sw(G.sp2, B_SOUT, co, nij, tc, nij, nij, B_POOL, Sblk(pij, pik), nik, 0, nik, B_RIN, Ro(i, k), nik, Rt(i, k),
               nik, B_POOL, Sblk(pik, pij), nij, 0, -FooI_h[k * o + j]);
      }
    }
  }
  // occupied ladder (not symmetrised): stored (i,j) += sum_kl W[k,i,l,j] S(ij,kl) R^{kl} S(kl,ij);
  // (k,l) and (l,k) share the stored block q = {k,l} and its overlaps: one problem with
  // X_eff = W[k,i,l,j] R^q + W[l,i,k,j] R^{q T}
  std::vector<double> W_h(W.n);
  W.download(W_h.data(), W_h.size(), s);
  G.sync();
  for (int p = 0; p < npairs; ++p) {
    const int i = P->pair_i[p], j = P->pair_j[p], nij = (int)nP(p);
    if (!nij) continue;
    for (int k = 0; k < o; ++k) for (int l = k; l < o; ++l) {
      const int q = blk(k, l), nq = (int)nP(q);
      if (!nq) continue;
      const double w1 = W_h[(((size_t)k * o + i) * o + l) * o + j];
      const double w2 = k == l ? 0.0 : W_h[(((size_t)l * o + i) * o + k) * o + j];
      // stored block q is R^{kl} (k <= l); R^{lk} = R^{kl T}
      if (w1 != 0.0)
        add_sw(G.sp2, B_SOUT, P->off_ij[p], nij, 0, nij, nij, B_POOL, Sblk(p, q), nq, 0, nq, B_RIN, P->off_ij[q], nq, 0, nq,
               B_POOL, Sblk(q, p), nij, 0, w1, w2 / w1);
      else
        add_sw(G.sp2, B_SOUT, P->off_ij[p], nij, 0, nij, nij, B_POOL, Sblk(p, q), nq, 0, nq, B_RIN, P->off_ij[q], nq, 1, nq,
               B_POOL, Sblk(q, p), nij, 0, w2);
    }
  }
  // per-problem extents of the small kernel: tile rows, staged X rows and columns, tile columns
  auto extents = [](const SProb& q, int e[4]) {
    const int Mt = std::min(64, q.M - q.m0), Nt = std::min(64, q.N - q.n0);
    e[0] = Mt;
    e[1] = q.a_buf != B_NONE ? q.K1 : Mt;
    e[2] = q.b_buf != B_NONE ? q.K2 : Nt;
    e[3] = Nt;
  };
  // algorithmic traffic and flops of each kernel class (tracing / roofline):
  // operator blocks counted once per launch (distinct blocks), vector blocks
  // once per vector (distinct ranges), flops as issued
  {
    auto acc_sw = [&](const std::vector<SProb>& Lst, int cls) {
      std::set<std::pair<int64_t, int64_t>> pool_blocks, vec_blocks;
      double fl = 0;
      for (const SProb& q : Lst) {
        if (q.a_buf == B_POOL) pool_blocks.insert({q.a_off, (int64_t)q.M * q.K1});
        if (q.b_buf == B_POOL) pool_blocks.insert({q.b_off, (int64_t)q.K2 * q.N});
        if (q.x_buf != B_POOL) vec_blocks.insert({q.x_off + ((int64_t)q.x_buf << 40), (int64_t)q.K1 * q.K2});
        vec_blocks.insert({q.c_off + ((int64_t)q.c_buf << 40), (int64_t)q.M * q.N});
        int e[4];
        extents(q, e);
        if (q.b_buf != B_NONE) fl += 2.0 * e[1] * e[2] * e[3];
        if (q.a_buf != B_NONE) fl += 2.0 * e[0] * e[1] * e[3];
      }
      double pe = 0, ve = 0;
      for (auto& b : pool_blocks) pe += b.second;
      for (auto& b : vec_blocks) ve += b.second;
      P->prof_pool_elems[cls] = pe; P->prof_vec_elems[cls] = ve; P->prof_flops[cls] = fl;
    };
    auto acc_v = [&](const std::vector<VProb>& Lst, int cls) {
      std::set<std::pair<int64_t, int64_t>> vec_blocks;
      double pe = 0, fl = 0;
      for (const VProb& q : Lst) {
        const int rows = q.mlen;
        pe += (double)rows * q.klen;
        fl += 2.0 * rows * q.klen;
        vec_blocks.insert({q.x_off + ((int64_t)q.x_buf << 40), (int64_t)q.K * q.x_stride});
        vec_blocks.insert({q.c_off + ((int64_t)q.c_buf << 40), (int64_t)q.M * q.c_stride});
      }
      double ve = 0;
      for (auto& b : vec_blocks) ve += b.second;
      P->prof_pool_elems[cls] = pe; P->prof_vec_elems[cls] = ve; P->prof_flops[cls] = fl;
    };
    auto acc_d = [&](std::initializer_list<const std::vector<DProb>*> lists, int cls) {
      std::set<std::pair<int64_t, int64_t>> pool_blocks, vec_blocks;
      double fl = 0;
      for (const auto* Lst : lists)
        for (const DProb& q : *Lst) {
          const int64_t asz = (int64_t)q.M * q.K, bsz = (int64_t)q.K * q.N;
          if (q.a_buf == B_POOL) pool_blocks.insert({q.a_off, asz});
          else vec_blocks.insert({q.a_off + ((int64_t)q.a_buf << 40), asz});
          if (q.b_buf == B_POOL) pool_blocks.insert({q.b_off, bsz});
          else vec_blocks.insert({q.b_off + ((int64_t)q.b_buf << 40), bsz});
          vec_blocks.insert({q.c_off + ((int64_t)q.c_buf << 40), (int64_t)q.M * q.N});
          fl += 2.0 * q.klen * std::min(q.tile_m, q.M - q.m0) * std::min(q.tile_n, q.N - q.n0);
        }
      double pe = 0, ve = 0;
      for (auto& b : pool_blocks) pe += b.second;
      for (auto& b : vec_blocks) ve += b.second;
      P->prof_pool_elems[cls] = pe; P->prof_vec_elems[cls] = ve; P->prof_flops[cls] = fl;
    };
    acc_sw(G.sp1, 0); acc_v(G.vp1, 1); acc_sw(G.sp2, 2); acc_v(G.vp2, 3);
    acc_d({&G.dp1}, 4);
    acc_d({&G.dp2, &G.dp3}, 5);
  }
  // split each sandwich list: problems with every dim <= SMALL_DIM (single tile) go to the
  // shared-memory kernel, bucketed by their largest dim
  auto bucket_of = [&](const SProb& q) {
    if (q.a_buf != B_NONE && q.K1 > SMALL_DIM) return -1;
    if (q.b_buf != B_NONE && q.K2 > SMALL_DIM) return -1;
    int e[4];
    extents(q, e);
    // the small kernel forms X + xb X^T in shared memory: the staged block must be all of square X
    const int xr0 = q.a_buf != B_NONE ? 0 : q.m0, xc0 = q.b_buf != B_NONE ? 0 : q.n0;
    if (q.xb != 0.0 && (e[1] != e[2] || xr0 != xc0 || e[1] != q.K1)) return -1;
    const int d = std::max(std::max(e[0], e[1]), std::max(e[2], e[3]));
    return d <= 16 ? 0 : d <= 32 ? 1 : d <= SMALL_DIM ? 2 : -1;
  };
  // order by output block (heaviest blocks first); group boundaries for every candidate size
  auto order_by_output = [&](std::vector<SProb>& Lst) {
    auto key_less = [](const SProb& a, const SProb& b) {
      if (a.c_buf != b.c_buf) return a.c_buf < b.c_buf;
      if (a.c_off != b.c_off) return a.c_off < b.c_off;
      if (a.tc != b.tc) return a.tc < b.tc;
      if (a.M != b.M) return a.M < b.M;
      if (a.N != b.N) return a.N < b.N;
      if (a.m0 != b.m0) return a.m0 < b.m0;
      return a.n0 < b.n0;
    };
    auto same = [](const SProb& a, const SProb& b) {
      return a.c_buf == b.c_buf && a.c_off == b.c_off && a.tc == b.tc && a.M == b.M && a.N == b.N && a.m0 == b.m0 &&
             a.n0 == b.n0;
    };
    std::stable_sort(Lst.begin(), Lst.end(), key_less);
    std::vector<std::pair<double, std::pair<size_t, size_t>>> blocks;
    for (size_t i = 0; i < Lst.size();) {
      size_t j = i;
      double work = 0;
      while (j < Lst.size() && same(Lst[j], Lst[i])) {
        int e[4];
        extents(Lst[j], e);
        work += (double)e[1] * e[2] * e[3] + (double)e[0] * e[1] * e[3];
        ++j;
      }
      blocks.push_back({work, {i, j}});
      i = j;
    }
    std::stable_sort(blocks.begin(), blocks.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    std::vector<SProb> out;
    std::vector<std::pair<int, int>> ranges;
    for (auto& b : blocks) {
      ranges.push_back({(int)out.size(), (int)(out.size() + b.second.second - b.second.first)});
      for (size_t k = b.second.first; k < b.second.second; ++k) out.push_back(Lst[k]);
    }
    Lst.swap(out);
    return ranges;
  };
  auto make_sets = [&](const std::vector<SProb>& Lst, SmallSet* sets, std::vector<SProb>& gen) {
    std::vector<SProb> b[3];
    for (const SProb& q : Lst) {
      int k = bucket_of(q);
      if (k < 0) gen.push_back(q); else b[k].push_back(q);
    }
    for (int k = 0; k < 3; ++k) {
      SmallSet& S = sets[k];
      for (const SProb& q : b[k]) {
        int e[4];
        extents(q, e);
        for (int d = 0; d < 4; ++d) S.dims[d] = std::max(S.dims[d], e[d]);
      }
      auto ranges = order_by_output(b[k]);
      S.nprob = (int)b[k].size();
      bool all_ab = !b[k].empty();
      for (const SProb& q : b[k]) all_ab = all_ab && q.a_buf != B_NONE && q.b_buf != B_NONE;
      S.ab = all_ab;
      S.pb = 1;
      S.h_probs = b[k];
      for (int c = 0; c < NGROUP_CAND; ++c) {
        std::vector<int>& st = S.h_starts[c];
        st.clear();
        for (auto& r : ranges)
          for (int x = r.first; x < r.second; x += GROUP_CAND[c]) st.push_back(x);
        st.push_back(S.nprob);
        S.ngroups[c] = (int)st.size() - 1;
      }
    }
  };
  Program& PR = P->prog;
  {
    std::unordered_map<int64_t, std::pair<int64_t, int>> s_transpose;
    for (int p = 0; p < npairs; ++p)
      for (int q = 0; q < npairs; ++q)
        if (nP(p) && nP(q)) s_transpose[Sblk(p, q)] = {Sblk(q, p), (int)nP(p)};
    build_tcs(P, G.sp2, s_transpose, s, fp);
  }
  make_sets(G.sp1, PR.small1, PR.h_gen1);
  make_sets(G.sp2, PR.small2, PR.h_gen2);
  PR.h_v1 = G.vp1;
  PR.h_v2 = G.vp2;
  PR.h_d1 = G.dp1;
  PR.h_d2 = G.dp2;
  PR.h_d3 = G.dp3;
  PR.smem_elems = G.smem;
  PR.upload(s, fp);
  // FP32 copy of the pool for the mixed-precision sigma
  P->pool32.alloc(P->pool64.n, fp);
  d2f(P->pool32.get(), P->pool64.get(), P->pool64.n, s);
  // BF16 copy for the BF16 sigma (its dense GEMV blocks)
  P->pool16.alloc(P->pool64.n, fp);
  d2bf(P->pool16.get(), P->pool64.get(), P->pool64.n, s);
  G.sync();
}

void Program::upload(cudaStream_t s, size_t* fp) {
  n_gen1 = (int)h_gen1.size(); n_gen2 = (int)h_gen2.size();
  n_v1 = (int)h_v1.size(); n_v2 = (int)h_v2.size();
  gen1.alloc(std::max<size_t>(1, h_gen1.size()), fp); gen1.upload(h_gen1.data(), h_gen1.size(), s);
  gen2.alloc(std::max<size_t>(1, h_gen2.size()), fp); gen2.upload(h_gen2.data(), h_gen2.size(), s);
  v1.alloc(std::max<size_t>(1, h_v1.size()), fp); v1.upload(h_v1.data(), h_v1.size(), s);
  v2.alloc(std::max<size_t>(1, h_v2.size()), fp); v2.upload(h_v2.data(), h_v2.size(), s);
  n_d1 = (int)h_d1.size(); n_d2 = (int)h_d2.size(); n_d3 = (int)h_d3.size();
  d1.alloc(std::max<size_t>(1, h_d1.size()), fp); d1.upload(h_d1.data(), h_d1.size(), s);
  d2.alloc(std::max<size_t>(1, h_d2.size()), fp); d2.upload(h_d2.data(), h_d2.size(), s);
  d3.alloc(std::max<size_t>(1, h_d3.size()), fp); d3.upload(h_d3.data(), h_d3.size(), s);
  for (SmallSet* sets : {small1, small2})
    for (int k = 0; k < 3; ++k) {
      SmallSet& S = sets[k];
      S.nprob = (int)S.h_probs.size();
      S.probs.alloc(std::max<size_t>(1, S.h_probs.size()), fp);
      S.probs.upload(S.h_probs.data(), S.h_probs.size(), s);
      for (int c = 0; c < NGROUP_CAND; ++c) {
        S.ngroups[c] = std::max(0, (int)S.h_starts[c].size() - 1);
        S.starts[c].alloc(std::max<size_t>(1, S.h_starts[c].size()), fp);
        S.starts[c].upload(S.h_starts[c].data(), S.h_starts[c].size(), s);
      }
    }
  PN_CUDA(cudaStreamSynchronize(s));
}

}  // namespace pnoeom
