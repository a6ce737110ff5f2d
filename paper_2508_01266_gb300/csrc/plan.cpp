// Plan builder: the ground-state intermediates and the Jacobian product of
// closed-shell, k-point LR-CCSD as lists of GEMM / layout-permute ops.
//
// Method (Eqs. 7-8 and 13-14 of the paper, read through the supercell picture):
//   Omega(t1, t2) = R(H~(t1), t2), where H~ = exp(-T1) H exp(T1) has DF factors
//   L~ = (1 - tau) L (1 + tau) (tau[a,i] = t1[i,a]) and R is the closed-shell CCD-form
//   residual of a general Hamiltonian:
//     R2 = (ai|bj) + sum_cd t_ij^cd (ac|bd)                                  [A]
//        + sum_kl t_kl^ab [(ki|lj) + sum_cd t_ij^cd (kc|ld)]                  [B]
//        + P_ij^ab { -1/2 sum_kc t_kj^bc [(ki|ac) - 1/2 sum_ld t_li^ad (kd|lc)]
//                    - sum_kc t_ki^bc [(kj|ac) - 1/2 sum_ld t_lj^ad (kd|lc)]  [C]
//                    + 1/2 sum_kc u_jk^bc [L_aikc + 1/2 sum_ld u_il^ad L_ldkc] [D]
//                    + sum_c t_ij^ac [f_bc - sum_kld u_kl^bd (ld|kc)]
//                    - sum_k t_ik^ab [f_kj + sum_lcd u_lj^cd (kd|lc)] }      [E]
//     R1 = f_ai + sum_me u_im^ae f_me + sum_mef u_im^ef (ae|mf) - sum_mne u_mn^ae (ne|mi)
//   with u = 2t - t(a<->b), L_pqrs = 2(pq|rs) - (ps|rq), P_ij^ab Y = Y + Y(i<->j, a<->b).
//   The Jacobian A.X = dOmega(t + hX)/dh is R linearized in t2 (X2 part) plus R
//   evaluated with the dressed-Hamiltonian derivative dH~ = [H~, X1] (X1 part):
//     dL~ = [L~, xi], xi[a,i] = x1[i,a]:  dL~_ai = L~_ae x_i^e - x_m^a L~_mi,
//     dL~_mi = L~_me x_i^e, dL~_ae = -x_m^a L~_me, dL~_me = 0;
//     df~ = [f~, xi] + sum_me x_m^e [2(pq|me) - (pe|mq)].
// Units: the supercell picture uses L / sqrt(Nk) and s2 = t2_paper / Nk; the
// program takes and returns vectors in the paper's normalization (Sec. II.B).
#include "plan.h"

#include <algorithm>
#include <array>
#include <cassert>
#include <map>
#include <stdexcept>

namespace lrcc {

static inline int md(int a, int n) { return ((a % n) + n) % n; }

int64_t layout_offset(const Layout& L, int k1, int k2, int k3, int i1, int i2, int i3, int i4) {
  const int nk = L.nk;
  const int64_t n0 = L.n[0], n1 = L.n[1], n2 = L.n[2], n3 = L.n[3];
  switch (L.kind) {
    case LK_K3:
      return (((int64_t)k1 * nk + k2) * nk + k3) * (n0 * n1 * n2 * n3) +
             ((i1 * n1 + i2) * n2 + i3) * n3 + i4;
    case LK_PP: {
      int P = md(k1 + k2, nk);
      int64_t rows = nk * n0 * n1, cols = nk * n2 * n3;
      int64_t r = ((int64_t)k1 * n0 + i1) * n1 + i2;
      int64_t c = ((int64_t)k3 * n2 + i3) * n3 + i4;
      return (int64_t)P * rows * cols + r * cols + c;
    }
    case LK_PH: {
      int q = md(k3 - k1, nk);
      int k4 = md(k1 + k2 - k3, nk);
      int64_t rows = nk * n0 * n2, cols = nk * n3 * n1;
      int64_t r = ((int64_t)k1 * n0 + i1) * n2 + i3;
      int64_t c = ((int64_t)k4 * n3 + i4) * n1 + i2;
      return (int64_t)q * rows * cols + r * cols + c;
    }
    case LK_CH:
      return (((int64_t)k1 * nk + k3) * nk + k2) * (n0 * n1 * n2 * n3) +
             ((i1 * n2 + i3) * n1 + i2) * n3 + i4;
  }
  throw std::runtime_error("bad layout");
}

int64_t Gemm::flops() const {
  return 8LL * M * N * K * (int64_t)aoff.size();
}

namespace {

struct T4 {
  int ar;
  int64_t off;
  Layout L;
};

struct B {
  Plan& P;
  int nk, o, v, Q;
  bool nonlinear = false;  // programs that are never transposed may multiply two vector-arena operands
  explicit B(Plan& p) : P(p), nk(p.d.nk), o(p.d.o), v(p.d.v), Q(p.d.Q) {}

  int64_t alloc(int ar, int64_t n) {
    int64_t off = P.arena_size[ar];
    const int64_t used = n;
    n = (n + 31) / 32 * 32;  // 512-byte alignment of every buffer
    P.arena_size[ar] += n;
    if (ar == AR_SCR) P.scr_bufs.push_back({off, n, used});
    return off;
  }
  T4 t4(int ar, int kind, int a, int b, int c, int d) {
    T4 t;
    t.ar = ar;
    t.L.kind = kind;
    t.L.nk = nk;
    t.L.n[0] = a; t.L.n[1] = b; t.L.n[2] = c; t.L.n[3] = d;
    t.off = alloc(ar, t.L.size());
    return t;
  }
  T4 relayout(const T4& x, int ar, int kind) {  // same logical tensor, new buffer
    return t4(ar, kind, x.L.n[0], x.L.n[1], x.L.n[2], x.L.n[3]);
  }
  static bool is_var(int ar) { return ar == AR_IN || ar == AR_OUT || ar == AR_SCR; }

  void push(Program& pr, int kind, int idx, int fixed_only = 0) {
    Op op;
    op.kind = kind;
    op.idx = idx;
    op.fixed_only = fixed_only;
    pr.ops.push_back(op);
  }

  // dst += alpha * src o pi (logical permutation)
  void perm(Program& pr, const T4& dst, const T4& src, std::array<int, 4> pi, double ar,
            double ai = 0.0, const char* tag = "") {
    for (int s = 0; s < 4; ++s)
      if (src.L.n[s] != dst.L.n[pi[s]]) throw std::runtime_error(std::string("perm dims ") + tag);
    bool ok = ((pi[0] < 2 && pi[1] < 2 && pi[2] >= 2 && pi[3] >= 2) ||
               (pi[0] >= 2 && pi[1] >= 2 && pi[2] < 2 && pi[3] < 2));
    if (!ok) throw std::runtime_error(std::string("perm breaks momentum rule ") + tag);
    Perm p;
    p.src = src.L;
    p.dst = dst.L;
    for (int s = 0; s < 4; ++s) p.pi[s] = pi[s];
    p.ar = ar;
    p.ai = ai;
    p.arS = src.ar;
    p.arD = dst.ar;
    p.offS = src.off;
    p.offD = dst.off;
    p.tag = tag;
    P.perms.push_back(p);
    push(pr, OP_PERM, (int)P.perms.size() - 1, (!is_var(src.ar) && !is_var(dst.ar)) ? 1 : 0);
  }

  void btr(Program& pr, int nb, int R, int C, int arD, int64_t offD, int arS, int64_t offS,
           double ar, const char* tag = "") {
    BTrans t;
    t.nb = nb; t.R = R; t.C = C;
    t.ar = ar; t.ai = 0.0;
    t.arS = arS; t.arD = arD; t.offS = offS; t.offD = offD;
    t.tag = tag;
    P.btrans.push_back(t);
    push(pr, OP_BTRANS, (int)P.btrans.size() - 1, (!is_var(arS) && !is_var(arD)) ? 1 : 0);
  }

  Gemm& g_new(int M, int N, int K, int ta, int tb, int64_t lda, int64_t ldb, int64_t ldc,
              int arA, int arB, int arC, double ar, double ai, const char* tag) {
    Gemm g;
    g.M = M; g.N = N; g.K = K;
    g.ta = ta; g.tb = tb;
    g.lda = lda; g.ldb = ldb; g.ldc = ldc;
    g.arA = arA; g.arB = arB; g.arC = arC;
    g.ar = ar; g.ai = ai;
    g.tag = tag;
    g.sbeg.push_back(0);
    P.gemms.push_back(g);
    return P.gemms.back();
  }
  static void batch(Gemm& g, int64_t coff) {
    g.coff.push_back(coff);
    g.sbeg.push_back(g.sbeg.back());
  }
  static void seg(Gemm& g, int64_t aoff, int64_t boff) {
    g.aoff.push_back(aoff);
    g.boff.push_back(boff);
    g.sbeg.back() += 1;
  }
  void g_push(Program& pr) {
    Gemm& g = P.gemms.back();
    // drop empty batches
    Gemm h = g;
    h.coff.clear();
    h.sbeg.assign(1, 0);
    h.aoff.clear();
    h.boff.clear();
    for (int b = 0; b < g.nbatch(); ++b) {
      if (g.sbeg[b + 1] == g.sbeg[b]) continue;
      batch(h, g.coff[b]);
      for (int s = g.sbeg[b]; s < g.sbeg[b + 1]; ++s) seg(h, g.aoff[s], g.boff[s]);
    }
    g = h;
    if (g.nbatch() == 0) {
      P.gemms.pop_back();
      return;
    }
    int nvar = (is_var(g.arA) ? 1 : 0) + (is_var(g.arB) ? 1 : 0);
    if (nvar > 1 && !nonlinear) throw std::runtime_error("gemm with two variable operands: " + g.tag);
    bool fixed = !is_var(g.arA) && !is_var(g.arB) && !is_var(g.arC);
    if (!fixed && !is_var(g.arC)) throw std::runtime_error("variable gemm into fixed arena: " + g.tag);
    push(pr, OP_GEMM, (int)P.gemms.size() - 1, fixed ? 1 : 0);
  }

  // pair-matrix geometry
  static void pair_dims(const Layout& L, int64_t& rows, int64_t& cols) {
    if (L.kind == LK_PP) {
      rows = (int64_t)L.nk * L.n[0] * L.n[1];
      cols = (int64_t)L.nk * L.n[2] * L.n[3];
    } else if (L.kind == LK_PH) {
      rows = (int64_t)L.nk * L.n[0] * L.n[2];
      cols = (int64_t)L.nk * L.n[3] * L.n[1];
    } else {
      throw std::runtime_error("pair_dims on non-pair layout");
    }
  }
  // C_g += alpha op(A_g) op(B_g) for every momentum group g
  void pair_gemm(Program& pr, const T4& C, const T4& A, int ta, const T4& Bm, int tb, double ar,
                 double ai, const char* tag) {
    int64_t rA, cA, rB, cB, rC, cC;
    pair_dims(A.L, rA, cA);
    pair_dims(Bm.L, rB, cB);
    pair_dims(C.L, rC, cC);
    int64_t M = ta ? cA : rA, K = ta ? rA : cA;
    int64_t K2 = tb ? cB : rB, N = tb ? rB : cB;
    if (K != K2 || M != rC || N != cC || A.L.kind != C.L.kind || Bm.L.kind != C.L.kind)
      throw std::runtime_error(std::string("pair_gemm shapes ") + tag);
    Gemm& g = g_new((int)M, (int)N, (int)K, ta, tb, cA, cB, cC, A.ar, Bm.ar, C.ar, ar, ai, tag);
    for (int q = 0; q < nk; ++q) {
      batch(g, C.off + q * rC * cC);
      seg(g, A.off + q * rA * cA, Bm.off + q * rB * cB);
    }
    g_push(pr);
  }
};

// scratch buffer containing element offset `off` (buffers sorted by offset)
int scr_find(const std::vector<ScrBuf>& bufs, int64_t off) {
  int lo = 0, hi = (int)bufs.size() - 1, ans = -1;
  while (lo <= hi) {
    int mid = (lo + hi) / 2;
    if (bufs[mid].off <= off) {
      ans = mid;
      lo = mid + 1;
    } else {
      hi = mid - 1;
    }
  }
  if (ans < 0 || off >= bufs[ans].off + bufs[ans].n) throw std::runtime_error("scratch offset outside every buffer");
  return ans;
}

// scratch buffers touched by an op
void scr_touched(const Plan& P, const Op& op, const std::vector<ScrBuf>& bufs, std::vector<int>& out) {
  out.clear();
  if (op.kind == OP_GEMM) {
    const Gemm& g = P.gemms[op.idx];
    if (g.arC == AR_SCR)
      for (int64_t x : g.coff) out.push_back(scr_find(bufs, x));
    if (g.arA == AR_SCR)
      for (int64_t x : g.aoff) out.push_back(scr_find(bufs, x));
    if (g.arB == AR_SCR)
      for (int64_t x : g.boff) out.push_back(scr_find(bufs, x));
  } else if (op.kind == OP_PERM) {
    const Perm& p = P.perms[op.idx];
    if (p.arS == AR_SCR) out.push_back(scr_find(bufs, p.offS));
    if (p.arD == AR_SCR) out.push_back(scr_find(bufs, p.offD));
  } else if (op.kind == OP_BTRANS) {
    const BTrans& t = P.btrans[op.idx];
    if (t.arS == AR_SCR) out.push_back(scr_find(bufs, t.offS));
    if (t.arD == AR_SCR) out.push_back(scr_find(bufs, t.offD));
  }
  std::sort(out.begin(), out.end());
  out.erase(std::unique(out.begin(), out.end()), out.end());
}

// Place scratch buffers so that buffers whose lifetimes overlap (within one program)
// never share memory, rewrite every scratch offset, and insert OP_ZERO ops so that each
// buffer starts at zero: forward programs zero it before its first use; for the
// transposed Jacobian, the op of its last forward use records it in `zl`.
void pack_scratch(Plan& P, const std::vector<Program*>& progs) {
  std::vector<ScrBuf> bufs = P.scr_bufs;
  const int nb = (int)bufs.size();
  if (nb == 0) return;
  std::vector<int> prog_of(nb, -1), first(nb, -1), last(nb, -1);
  std::vector<int> t;
  for (int pi = 0; pi < (int)progs.size(); ++pi) {
    const Program& pr = *progs[pi];
    for (int i = 0; i < (int)pr.ops.size(); ++i) {
      scr_touched(P, pr.ops[i], bufs, t);
      for (int b : t) {
        if (prog_of[b] >= 0 && prog_of[b] != pi) throw std::runtime_error("scratch buffer shared by two programs");
        prog_of[b] = pi;
        if (first[b] < 0) first[b] = i;
        last[b] = i;
      }
    }
  }
  std::vector<int> order(nb);
  for (int i = 0; i < nb; ++i) order[i] = i;
  std::sort(order.begin(), order.end(),
            [&](int a, int b) { return bufs[a].n > bufs[b].n || (bufs[a].n == bufs[b].n && a < b); });
  std::vector<int64_t> place(nb, 0);
  int64_t top = 0;
  std::vector<int> placed;
  for (int b : order) {
    if (prog_of[b] < 0) continue;  // never used
    std::vector<std::pair<int64_t, int64_t>> busy;
    for (int q : placed)
      if (prog_of[q] == prog_of[b] && !(last[q] < first[b] || last[b] < first[q]))
        busy.push_back({place[q], place[q] + bufs[q].n});
    std::sort(busy.begin(), busy.end());
    int64_t off = 0;
    for (auto& iv : busy) {
      if (off + bufs[b].n <= iv.first) break;
      off = std::max(off, iv.second);
    }
    place[b] = off;
    top = std::max(top, off + bufs[b].n);
    placed.push_back(b);
  }
  // zero points (physical regions), by program and op index, before remapping
  std::vector<std::vector<std::vector<int>>> zfirst(progs.size());
  for (size_t pi = 0; pi < progs.size(); ++pi) zfirst[pi].assign(progs[pi]->ops.size(), {});
  std::vector<std::vector<int>> zlast(progs[0]->ops.size());
  for (int b = 0; b < nb; ++b) {
    if (prog_of[b] < 0) continue;
    P.zeros.push_back({AR_SCR, place[b], bufs[b].n, bufs[b].used});
    const int zi = (int)P.zeros.size() - 1;
    zfirst[prog_of[b]][first[b]].push_back(zi);
    if (prog_of[b] == 0) zlast[last[b]].push_back(zi);
  }
  auto remap = [&](int64_t x) {
    const int b = scr_find(bufs, x);
    return place[b] + (x - bufs[b].off);
  };
  for (Program* pr : progs)
    for (const Op& op : pr->ops) {
      if (op.kind == OP_GEMM) {
        Gemm& g = P.gemms[op.idx];
        if (g.arC == AR_SCR)
          for (auto& x : g.coff) x = remap(x);
        if (g.arA == AR_SCR)
          for (auto& x : g.aoff) x = remap(x);
        if (g.arB == AR_SCR)
          for (auto& x : g.boff) x = remap(x);
      } else if (op.kind == OP_PERM) {
        Perm& p = P.perms[op.idx];
        if (p.arS == AR_SCR) p.offS = remap(p.offS);
        if (p.arD == AR_SCR) p.offD = remap(p.offD);
      } else if (op.kind == OP_BTRANS) {
        BTrans& q = P.btrans[op.idx];
        if (q.arS == AR_SCR) q.offS = remap(q.offS);
        if (q.arD == AR_SCR) q.offD = remap(q.offD);
      }
    }
  for (size_t pi = 0; pi < progs.size(); ++pi) {
    Program& pr = *progs[pi];
    std::vector<Op> out;
    for (size_t i = 0; i < pr.ops.size(); ++i) {
      for (int zi : zfirst[pi][i]) {
        Op z;
        z.kind = OP_ZERO;
        z.idx = zi;
        out.push_back(z);
      }
      Op op = pr.ops[i];
      if (pi == 0 && !zlast[i].empty()) {
        P.zlists.push_back(zlast[i]);
        op.zl = (int)P.zlists.size() - 1;
      }
      out.push_back(op);
    }
    pr.ops = out;
  }
  P.arena_size[AR_SCR] = top;
}

}  // namespace

Plan build_plan(const Dims& d, int64_t ws_budget) {
  Plan P;
  P.d = d;
  B b(P);
  const int nk = d.nk, o = d.o, v = d.v, Q = d.Q, n = o + v;
  (void)n;
  const int64_t o2 = (int64_t)o * o, v2 = (int64_t)v * v, ov = (int64_t)o * v;
  auto kb3 = [&](int k1, int k2, int k3) { return md(k1 + k2 - k3, nk); };
  const double sNk = (double)nk;
  // layout extents and GEMM dimensions are 32-bit: the largest single extent is a whole
  // DF factor or pair matrix dimension
  {
    const int64_t n64 = o + (int64_t)v;
    const int64_t big = std::max({(int64_t)nk * nk * Q * n64 * n64, (int64_t)nk * v2 * nk, (int64_t)nk * nk * ov * Q,
                                  (int64_t)nk * o2 * nk});
    if (big > INT32_MAX) throw std::runtime_error("problem too large: an extent exceeds 2^31 elements");
  }

  // ---------------- FIX inputs ----------------
  // DF factor blocks [k1][k2][Q][n1][n2] in supercell units (L / sqrt(Nk))
  auto dfsz = [&](int a, int c) { return (int64_t)nk * nk * Q * a * c; };
  P.off_Loo = b.alloc(AR_FIX, dfsz(o, o));
  P.off_Lov = b.alloc(AR_FIX, dfsz(o, v));
  P.off_Lvo = b.alloc(AR_FIX, dfsz(v, o));
  P.off_Lvv = b.alloc(AR_FIX, dfsz(v, v));
  P.off_f0 = b.alloc(AR_FIX, (int64_t)nk * (o + v) * (o + v));  // diag(eps) per k, n x n
  P.off_t1 = b.alloc(AR_FIX, (int64_t)nk * ov);
  P.off_t2 = b.alloc(AR_FIX, (int64_t)nk * nk * nk * o2 * v2);  // paper units
  P.off_idv = b.alloc(AR_FIX, o2);                               // identity o x o
  P.off_derived = P.arena_size[AR_FIX];
  auto DF = [&](int64_t base, int a, int c, int k1, int k2) {
    return base + ((int64_t)k1 * nk + k2) * Q * a * c;
  };
  const int nn = o + v;
  auto F0 = [&](int k, int p, int q) { return P.off_f0 + ((int64_t)k * nn + p) * nn + q; };
  auto T1 = [&](int k) { return P.off_t1 + (int64_t)k * ov; };

  Program& G = P.ground;
  // dressed factors (ov block unchanged)
  int64_t tLoo = b.alloc(AR_FIX, dfsz(o, o)), tLvo = b.alloc(AR_FIX, dfsz(v, o)),
          tLvv = b.alloc(AR_FIX, dfsz(v, v));
  int64_t Lov = P.off_Lov;
  // Loo~ = Loo + Lov t1[k2]^T  (rows (Q,i), cols j)
  b.perm(G, T4{AR_FIX, tLoo, Layout{LK_K3, 1, {1, 1, 1, (int)dfsz(o, o)}}},
         T4{AR_FIX, P.off_Loo, Layout{LK_K3, 1, {1, 1, 1, (int)dfsz(o, o)}}}, {0, 1, 2, 3}, 1.0, 0.0,
         "copy Loo");
  {
    Gemm& g = b.g_new(Q * o, o, v, 0, 1, v, v, o, AR_FIX, AR_FIX, AR_FIX, 1.0, 0.0, "dress oo");
    for (int k1 = 0; k1 < nk; ++k1)
      for (int k2 = 0; k2 < nk; ++k2) {
        B::batch(g, DF(tLoo, o, o, k1, k2));
        B::seg(g, DF(Lov, o, v, k1, k2), T1(k2));
      }
    b.g_push(G);
  }
  // Lvv~ = Lvv - t1[k1]^T Lov   (per Q)
  b.perm(G, T4{AR_FIX, tLvv, Layout{LK_K3, 1, {1, 1, 1, (int)dfsz(v, v)}}},
         T4{AR_FIX, P.off_Lvv, Layout{LK_K3, 1, {1, 1, 1, (int)dfsz(v, v)}}}, {0, 1, 2, 3}, 1.0, 0.0,
         "copy Lvv");
  {
    Gemm& g = b.g_new(v, v, o, 1, 0, v, v, v, AR_FIX, AR_FIX, AR_FIX, -1.0, 0.0, "dress vv");
    for (int k1 = 0; k1 < nk; ++k1)
      for (int k2 = 0; k2 < nk; ++k2)
        for (int q = 0; q < Q; ++q) {
          B::batch(g, DF(tLvv, v, v, k1, k2) + (int64_t)q * v2);
          B::seg(g, T1(k1), DF(Lov, o, v, k1, k2) + (int64_t)q * ov);
        }
    b.g_push(G);
  }
  // Lvo~ = Lvo + Lvv~ t1[k2]^T - t1[k1]^T Loo
  b.perm(G, T4{AR_FIX, tLvo, Layout{LK_K3, 1, {1, 1, 1, (int)dfsz(v, o)}}},
         T4{AR_FIX, P.off_Lvo, Layout{LK_K3, 1, {1, 1, 1, (int)dfsz(v, o)}}}, {0, 1, 2, 3}, 1.0, 0.0,
         "copy Lvo");
  {
    Gemm& g = b.g_new(Q * v, o, v, 0, 1, v, v, o, AR_FIX, AR_FIX, AR_FIX, 1.0, 0.0, "dress vo a");
    for (int k1 = 0; k1 < nk; ++k1)
      for (int k2 = 0; k2 < nk; ++k2) {
        B::batch(g, DF(tLvo, v, o, k1, k2));
        B::seg(g, DF(tLvv, v, v, k1, k2), T1(k2));
      }
    b.g_push(G);
    Gemm& h = b.g_new(v, o, o, 1, 0, v, o, o, AR_FIX, AR_FIX, AR_FIX, -1.0, 0.0, "dress vo b");
    for (int k1 = 0; k1 < nk; ++k1)
      for (int k2 = 0; k2 < nk; ++k2)
        for (int q = 0; q < Q; ++q) {
          B::batch(h, DF(tLvo, v, o, k1, k2) + (int64_t)q * ov);
          B::seg(h, T1(k1), DF(P.off_Loo, o, o, k1, k2) + (int64_t)q * o2);
        }
    b.g_push(G);
  }

  // ---------------- Fock matrices ----------------
  // G(L)_pq(k) = 2 sum_Q L[k,k]_pq J^Q - sum_k' sum_Qi L[k,k']_pi L[k',k]_iq,  J^Q = sum L[k',k']_ii
  // h = f0 - G(L);  f~ = (1 - tau) h (1 + tau) + G(L~).  Blocks oo, ov, vv are needed.
  int64_t hoo = b.alloc(AR_FIX, nk * o2), hov = b.alloc(AR_FIX, nk * ov), hvv = b.alloc(AR_FIX, nk * v2);
  int64_t foo = b.alloc(AR_FIX, nk * o2), fov = b.alloc(AR_FIX, nk * ov), fvv = b.alloc(AR_FIX, nk * v2);
  int64_t Jq = b.alloc(AR_FIX, Q), Jt = b.alloc(AR_FIX, Q);
  auto fblk = [&](int64_t base, int a, int c, int k) { return base + (int64_t)k * a * c; };
  // f0 blocks into h (h starts as f0)
  for (int k = 0; k < nk; ++k) {
    // oo: rows p<o, cols q<o of the n x n f0 block, copied row by row with a 1-column GEMM-free perm
    for (int p = 0; p < o; ++p) {
      b.perm(G, T4{AR_FIX, fblk(hoo, o, o, k) + (int64_t)p * o, Layout{LK_K3, 1, {1, 1, 1, o}}},
             T4{AR_FIX, F0(k, p, 0), Layout{LK_K3, 1, {1, 1, 1, o}}}, {0, 1, 2, 3}, 1.0, 0.0, "f0 oo");
      b.perm(G, T4{AR_FIX, fblk(hov, o, v, k) + (int64_t)p * v, Layout{LK_K3, 1, {1, 1, 1, v}}},
             T4{AR_FIX, F0(k, p, o), Layout{LK_K3, 1, {1, 1, 1, v}}}, {0, 1, 2, 3}, 1.0, 0.0, "f0 ov");
    }
    for (int p = 0; p < v; ++p)
      b.perm(G, T4{AR_FIX, fblk(hvv, v, v, k) + (int64_t)p * v, Layout{LK_K3, 1, {1, 1, 1, v}}},
             T4{AR_FIX, F0(k, o + p, o), Layout{LK_K3, 1, {1, 1, 1, v}}}, {0, 1, 2, 3}, 1.0, 0.0, "f0 vv");
  }
  // J^Q = sum_k' sum_i L[k',k'][Q]_ii (undressed), Jt with dressed Loo~
  auto coulomb_vec = [&](int64_t J, int64_t Loo_base, const char* tag) {
    Gemm& g = b.g_new(Q, 1, (int)o2, 0, 0, o2, 1, 1, AR_FIX, AR_FIX, AR_FIX, 1.0, 0.0, tag);
    B::batch(g, J);
    for (int k = 0; k < nk; ++k) B::seg(g, DF(Loo_base, o, o, k, k), P.off_idv);
    b.g_push(G);
  };
  coulomb_vec(Jq, P.off_Loo, "J");
  coulomb_vec(Jt, tLoo, "J~");
  // add c * G(L) block (p-range X, q-range Y) into dst
  struct Fac { int64_t base; int a, c; };
  auto addG = [&](int64_t dst, int a, int c, Fac Lpq, Fac Lpi, Fac Liq, int64_t J, double coef,
                  const char* tag) {
    // Coulomb: dst[k](p,q) += 2 coef sum_Q J[Q] L[k,k][Q](p,q)
    Gemm& g = b.g_new(1, a * c, Q, 0, 0, Q, (int64_t)a * c, (int64_t)a * c, AR_FIX, AR_FIX, AR_FIX,
                      2.0 * coef, 0.0, tag);
    for (int k = 0; k < nk; ++k) {
      B::batch(g, dst + (int64_t)k * a * c);
      B::seg(g, J, DF(Lpq.base, Lpq.a, Lpq.c, k, k));
    }
    b.g_push(G);
    // exchange: dst[k](p,q) -= coef sum_{k',Q,i} L[k,k'][Q](p,i) L[k',k][Q](i,q)
    Gemm& h = b.g_new(a, c, o, 0, 0, o, c, c, AR_FIX, AR_FIX, AR_FIX, -coef, 0.0, tag);
    for (int k = 0; k < nk; ++k) {
      B::batch(h, dst + (int64_t)k * a * c);
      for (int kp = 0; kp < nk; ++kp)
        for (int q = 0; q < Q; ++q)
          B::seg(h, DF(Lpi.base, Lpi.a, Lpi.c, k, kp) + (int64_t)q * a * o,
                 DF(Liq.base, Liq.a, Liq.c, kp, k) + (int64_t)q * o * c);
    }
    b.g_push(G);
  };
  // h = f0 - G(L)
  addG(hoo, o, o, {P.off_Loo, o, o}, {P.off_Loo, o, o}, {P.off_Loo, o, o}, Jq, -1.0, "h oo");
  addG(hov, o, v, {P.off_Lov, o, v}, {P.off_Loo, o, o}, {P.off_Lov, o, v}, Jq, -1.0, "h ov");
  addG(hvv, v, v, {P.off_Lvv, v, v}, {P.off_Lvo, v, o}, {P.off_Lov, o, v}, Jq, -1.0, "h vv");
  // f~ = h~ + G(L~):  h~_ij = h_ij + h_ie t_j^e ; h~_ia = h_ia ; h~_ab = h_ab - t_m^a h_mb
  b.perm(G, T4{AR_FIX, foo, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * o2)}}},
         T4{AR_FIX, hoo, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * o2)}}}, {0, 1, 2, 3}, 1.0, 0.0, "h~oo");
  b.perm(G, T4{AR_FIX, fov, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * ov)}}},
         T4{AR_FIX, hov, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * ov)}}}, {0, 1, 2, 3}, 1.0, 0.0, "h~ov");
  b.perm(G, T4{AR_FIX, fvv, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * v2)}}},
         T4{AR_FIX, hvv, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * v2)}}}, {0, 1, 2, 3}, 1.0, 0.0, "h~vv");
  {
    Gemm& g = b.g_new(o, o, v, 0, 1, v, v, o, AR_FIX, AR_FIX, AR_FIX, 1.0, 0.0, "h~oo t");
    for (int k = 0; k < nk; ++k) {
      B::batch(g, fblk(foo, o, o, k));
      B::seg(g, fblk(hov, o, v, k), T1(k));
    }
    b.g_push(G);
    Gemm& h = b.g_new(v, v, o, 1, 0, v, v, v, AR_FIX, AR_FIX, AR_FIX, -1.0, 0.0, "h~vv t");
    for (int k = 0; k < nk; ++k) {
      B::batch(h, fblk(fvv, v, v, k));
      B::seg(h, T1(k), fblk(hov, o, v, k));
    }
    b.g_push(G);
  }
  addG(foo, o, o, {tLoo, o, o}, {tLoo, o, o}, {tLoo, o, o}, Jt, 1.0, "G~ oo");
  addG(fov, o, v, {Lov, o, v}, {tLoo, o, o}, {Lov, o, v}, Jt, 1.0, "G~ ov");
  addG(fvv, v, v, {tLvv, v, v}, {tLvo, v, o}, {Lov, o, v}, Jt, 1.0, "G~ vv");
  int64_t fovT = b.alloc(AR_FIX, nk * ov);
  b.btr(G, nk, o, v, AR_FIX, fovT, AR_FIX, fov, 1.0, "fovT");

  // ---------------- amplitude layouts (supercell units) ----------------
  T4 t2in{AR_FIX, P.off_t2, Layout{LK_K3, nk, {o, o, v, v}}};
  T4 Tk3 = b.t4(AR_FIX, LK_K3, o, o, v, v);
  b.perm(G, Tk3, t2in, {0, 1, 2, 3}, 1.0 / sNk, 0.0, "T sc");
  T4 Tpp = b.relayout(Tk3, AR_FIX, LK_PP);
  b.perm(G, Tpp, Tk3, {0, 1, 2, 3}, 1.0, 0.0, "Tpp");
  T4 Tc = b.relayout(Tk3, AR_FIX, LK_PH);
  b.perm(G, Tc, Tk3, {0, 1, 3, 2}, 1.0, 0.0, "Tc");
  T4 ud = b.relayout(Tk3, AR_FIX, LK_PH);
  b.perm(G, ud, Tk3, {0, 1, 2, 3}, 2.0, 0.0, "ud a");
  b.perm(G, ud, Tk3, {0, 1, 3, 2}, -1.0, 0.0, "ud b");
  T4 uk3 = b.relayout(Tk3, AR_FIX, LK_K3);
  b.perm(G, uk3, Tk3, {0, 1, 2, 3}, 2.0, 0.0, "uk3 a");
  b.perm(G, uk3, Tk3, {0, 1, 3, 2}, -1.0, 0.0, "uk3 b");

  // ---------------- dressed integrals from DF factors ----------------
  // chemist GEMM: CH block (k1,k3,k2) of logical (p, r, q, s): [(p,q)][(r,s)] = sum_Q A[kp,kq](p,q) B[kr,ks](r,s)
  auto chem = [&](Program& pr, const T4& C, int64_t Abase, int na, int nq, int64_t Bbase, int nr, int ns,
                  int arA, int arB, double ar, const char* tag) {
    // logical C(p, r, q, s): n = (na, nr, nq, ns); block index (kp, kq, kr), ks = kp + kr - kq
    Gemm& g = b.g_new(na * nq, nr * ns, Q, 1, 0, (int64_t)na * nq, (int64_t)nr * ns, (int64_t)nr * ns,
                      arA, arB, C.ar, ar, 0.0, tag);
    for (int kp = 0; kp < nk; ++kp)
      for (int kq = 0; kq < nk; ++kq)
        for (int kr = 0; kr < nk; ++kr) {
          int ks = md(kp + kr - kq, nk);
          B::batch(g, C.off + layout_offset(C.L, kp, kr, kq, 0, 0, 0, 0));
          B::seg(g, DF(Abase, na, nq, kp, kq), DF(Bbase, nr, ns, kr, ks));
        }
    b.g_push(pr);
  };
  // V(k,l,c,d) = (kc|ld)
  T4 Vch = b.t4(AR_FIX, LK_CH, o, o, v, v);
  chem(G, Vch, Lov, o, v, Lov, o, v, AR_FIX, AR_FIX, 1.0, "V ovov");
  T4 Vpp = b.relayout(Vch, AR_FIX, LK_PP);
  b.perm(G, Vpp, Vch, {0, 1, 2, 3}, 1.0, 0.0, "Vpp");
  T4 Vk3 = b.relayout(Vch, AR_FIX, LK_K3);
  b.perm(G, Vk3, Vch, {0, 1, 2, 3}, 1.0, 0.0, "Vk3");
  // W(l,k,c,d) = (kd|lc) = V(k,l,d,c)
  T4 Wk3 = b.relayout(Vch, AR_FIX, LK_K3);
  b.perm(G, Wk3, Vch, {1, 0, 3, 2}, 1.0, 0.0, "Wk3");
  // M(d,c,l,k) = (kd|lc) ; ML(d,c,l,k) = 2(ld|kc) - (lc|kd)   (PH)
  T4 Mph = b.t4(AR_FIX, LK_PH, v, v, o, o);
  b.perm(G, Mph, Vch, {3, 2, 0, 1}, 1.0, 0.0, "M");
  T4 MLph = b.t4(AR_FIX, LK_PH, v, v, o, o);
  b.perm(G, MLph, Vch, {2, 3, 0, 1}, 2.0, 0.0, "ML a");
  b.perm(G, MLph, Vch, {2, 3, 1, 0}, -1.0, 0.0, "ML b");

  // hole-hole: Whh(k,l,i,j) = (ki|lj)~ + sum_cd t_ij^cd (kc|ld)   (PP)
  T4 Ioo = b.t4(AR_FIX, LK_CH, o, o, o, o);
  chem(G, Ioo, tLoo, o, o, tLoo, o, o, AR_FIX, AR_FIX, 1.0, "(ki|lj)~");
  T4 Whh = b.relayout(Ioo, AR_FIX, LK_PP);
  b.perm(G, Whh, Ioo, {0, 1, 2, 3}, 1.0, 0.0, "Whh");
  b.pair_gemm(G, Whh, Vpp, 0, Tpp, 1, 1.0, 0.0, "Whh += V T^T");

  // ring C: WC(i,c,a,k) = (ki|ac)~ - 1/2 sum_ld t_li^ad (kd|lc)
  T4 Ikiac = b.t4(AR_FIX, LK_CH, o, v, o, v);  // logical (k,a,i,c)
  chem(G, Ikiac, tLoo, o, o, tLvv, v, v, AR_FIX, AR_FIX, 1.0, "(ki|ac)~");
  T4 WC = b.t4(AR_FIX, LK_PH, o, v, v, o);
  b.perm(G, WC, Ikiac, {3, 2, 0, 1}, 1.0, 0.0, "WC");
  b.pair_gemm(G, WC, Tc, 0, Mph, 0, -0.5, 0.0, "WC -= 1/2 Tc M");
  // ring D: WD(i,c,a,k) = 2(ai|kc)~ - (ac|ki)~ + 1/2 sum_ld u_il^ad L_ldkc
  T4 Iaikc = b.t4(AR_FIX, LK_CH, v, o, o, v);  // logical (a,k,i,c)
  chem(G, Iaikc, tLvo, v, o, Lov, o, v, AR_FIX, AR_FIX, 1.0, "(ai|kc)~");
  T4 Iacki = b.t4(AR_FIX, LK_CH, v, o, v, o);  // logical (a,k,c,i)
  chem(G, Iacki, tLvv, v, v, tLoo, o, o, AR_FIX, AR_FIX, 1.0, "(ac|ki)~");
  T4 WD = b.t4(AR_FIX, LK_PH, o, v, v, o);
  b.perm(G, WD, Iaikc, {2, 3, 0, 1}, 2.0, 0.0, "WD a");
  b.perm(G, WD, Iacki, {2, 3, 1, 0}, -1.0, 0.0, "WD b");
  b.pair_gemm(G, WD, ud, 0, MLph, 0, 0.5, 0.0, "WD += 1/2 ud ML");

  // E intermediates: Fv[kb](b,c) = f~_bc - sum_kld u_kl^bd (ld|kc) ; Fo[kj](k,j) = f~_kj + sum_lcd u_lj^cd (kd|lc)
  int64_t Fv = b.alloc(AR_FIX, nk * v2), Fo = b.alloc(AR_FIX, nk * o2);
  b.perm(G, T4{AR_FIX, Fv, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * v2)}}},
         T4{AR_FIX, fvv, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * v2)}}}, {0, 1, 2, 3}, 1.0, 0.0, "Fv=f");
  b.perm(G, T4{AR_FIX, Fo, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * o2)}}},
         T4{AR_FIX, foo, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * o2)}}}, {0, 1, 2, 3}, 1.0, 0.0, "Fo=f");
  // YEv-type contraction: C[kb](b,c) += alpha sum_{kk,kl,k,l} U[kk,kl,kb](k,l)[b][d] Vk3[kl,kk,kd](l,k)[d][c]
  auto yev = [&](Program& pr, int64_t Cb, int arC, const T4& U, double alpha, const char* tag) {
    Gemm& g = b.g_new(v, v, v, 0, 0, v, v, v, U.ar, AR_FIX, arC, alpha, 0.0, tag);
    for (int kbb = 0; kbb < nk; ++kbb) {
      B::batch(g, Cb + (int64_t)kbb * v2);
      for (int kk = 0; kk < nk; ++kk)
        for (int kl = 0; kl < nk; ++kl) {
          int kd = md(kk + kl - kbb, nk);
          for (int k = 0; k < o; ++k)
            for (int l = 0; l < o; ++l)
              B::seg(g, U.off + layout_offset(U.L, kk, kl, kbb, k, l, 0, 0),
                     Vk3.off + layout_offset(Vk3.L, kl, kk, kd, l, k, 0, 0));
        }
    }
    b.g_push(pr);
  };
  // YEo-type: C[kj](k,j) += alpha sum_{kl,kc,l} Wk3[kl,kj,kc](l)[k][(c,d)] U[kl,kj,kc](l)[j][(c,d)]^T
  auto yeo = [&](Program& pr, int64_t Cb, int arC, const T4& U, double alpha, const char* tag) {
    Gemm& g = b.g_new(o, o, (int)v2, 0, 1, v2, v2, o, AR_FIX, U.ar, arC, alpha, 0.0, tag);
    for (int kj = 0; kj < nk; ++kj) {
      B::batch(g, Cb + (int64_t)kj * o2);
      for (int kl = 0; kl < nk; ++kl)
        for (int kc = 0; kc < nk; ++kc)
          for (int l = 0; l < o; ++l)
            B::seg(g, Wk3.off + layout_offset(Wk3.L, kl, kj, kc, l, 0, 0, 0),
                   U.off + layout_offset(U.L, kl, kj, kc, l, 0, 0, 0));
    }
    b.g_push(pr);
  };
  yev(G, Fv, AR_FIX, uk3, -1.0, "Fv -= u V");
  yeo(G, Fo, AR_FIX, uk3, 1.0, "Fo += W u");
  // G_in = Fo(n,i) - f~(n,i) ; H_af = f~(a,f) - Fv(a,f)
  int64_t Gm = b.alloc(AR_FIX, nk * o2), Hm = b.alloc(AR_FIX, nk * v2);
  b.perm(G, T4{AR_FIX, Gm, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * o2)}}},
         T4{AR_FIX, Fo, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * o2)}}}, {0, 1, 2, 3}, 1.0, 0.0, "G a");
  b.perm(G, T4{AR_FIX, Gm, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * o2)}}},
         T4{AR_FIX, foo, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * o2)}}}, {0, 1, 2, 3}, -1.0, 0.0, "G b");
  b.perm(G, T4{AR_FIX, Hm, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * v2)}}},
         T4{AR_FIX, fvv, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * v2)}}}, {0, 1, 2, 3}, 1.0, 0.0, "H a");
  b.perm(G, T4{AR_FIX, Hm, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * v2)}}},
         T4{AR_FIX, Fv, Layout{LK_K3, 1, {1, 1, 1, (int)(nk * v2)}}}, {0, 1, 2, 3}, -1.0, 0.0, "H b");
  // Lvv~ with the inner matrix transposed: LvvT[k1][k2][Q][e][a]
  int64_t LvvT = b.alloc(AR_FIX, dfsz(v, v));
  b.btr(G, nk * nk * Q, v, v, AR_FIX, LvvT, AR_FIX, tLvv, 1.0, "LvvT");

  // ---------------- W-block workspace and ladder chunks ----------------
  // W(P,ka,kc)[(a,b)][(c,d)] = sum_Q A[ka,kc][Q](a,c) B[kb,kd][Q](b,d)  (kb = P-ka, kd = P-kc)
  struct Tri { int P, ka, kc; };
  std::vector<Tri> tris;
  for (int Pm = 0; Pm < nk; ++Pm)
    for (int ka = 0; ka < nk; ++ka)
      for (int kc = 0; kc < nk; ++kc) tris.push_back({Pm, ka, kc});
  const int64_t wblk_max = std::max<int64_t>(v2 * v2, ov * v2);
  int64_t per_chunk = std::max<int64_t>(1, ws_budget / wblk_max);
  per_chunk = std::min<int64_t>(per_chunk, (int64_t)tris.size());
  P.ws_limit = per_chunk;
  P.arena_size[AR_WS] = per_chunk * wblk_max;
  // ladder over chunks: build (fixed-only) then contract.  Rows: all (ki,i,j) of the PP matrix.
  // half: the caller symmetrises the result over the pair swap (i,j,a,b) -> (j,i,b,a)
  // (momenta swapped too) and the product is pair-symmetric (X and W are), so only the
  // output column blocks ka with ka <= kb = P - ka are computed: ka < kb at twice the
  // weight (the swap supplies block kb), the self-paired block ka = kb at the weight
  // itself.  W blocks are built for those ka only.
  auto ladder = [&](Program& pr, const T4& Cpp, int64_t Afac, int na, const T4& Xpp, double alpha,
                    const char* tag, double* flop_acc, double* build_acc, bool half) {
    // Cpp: logical (i,j,a,b) with a in [0,na); Xpp: logical (i,j,c,d)
    const int64_t rowsX = (int64_t)nk * o2, colsX = (int64_t)nk * v2;
    const int64_t colsC = (int64_t)nk * na * v;
    const int64_t wsz = (int64_t)na * v * v2;
    std::vector<Tri> work;
    for (const Tri& t : tris) {
      const int kbb = md(t.P - t.ka, nk);
      if (!half || t.ka <= kbb) work.push_back(t);
    }
    for (size_t c0 = 0; c0 < work.size(); c0 += per_chunk) {
      size_t c1 = std::min(work.size(), c0 + (size_t)per_chunk);
      Gemm& g = b.g_new(na * v, (int)v2, Q, 1, 0, (int64_t)na * v, v2, 0, AR_FIX, AR_FIX, AR_WS, 1.0, 0.0,
                        "W build");
      g.epi = 1;
      g.ep[0] = na; g.ep[1] = v; g.ep[2] = v; g.ep[3] = v;
      for (size_t t = c0; t < c1; ++t) {
        const Tri& tr = work[t];
        int kbb = md(tr.P - tr.ka, nk), kd = md(tr.P - tr.kc, nk);
        B::batch(g, (int64_t)(t - c0) * wsz);
        B::seg(g, DF(Afac, na, v, tr.ka, tr.kc), DF(tLvv, v, v, kbb, kd));
      }
      if (build_acc) *build_acc += (double)g.flops();
      b.g_push(pr);
      // contraction: C_P[:, ka] += alpha X_P[:, kc] W^T, grouped by (P, ka); with half, the
      // self-paired blocks and the others go to separate ops (different weights)
      std::map<std::pair<int, int>, std::vector<size_t>> grp;
      for (size_t t = c0; t < c1; ++t) grp[{work[t].P, work[t].ka}].push_back(t);
      for (int self = 0; self < (half ? 2 : 1); ++self) {
        bool any = false;
        for (auto& kv : grp) any = any || !half || ((md(kv.first.first - kv.first.second, nk) == kv.first.second) == (self == 1));
        if (!any) continue;
        const double a = half && self == 0 ? 2.0 * alpha : alpha;
        Gemm& h = b.g_new((int)rowsX, na * v, (int)v2, 0, 1, colsX, v2, colsC, Xpp.ar, AR_WS, Cpp.ar, a, 0.0, tag);
        for (auto& kv : grp) {
          int Pm = kv.first.first, ka = kv.first.second;
          if (half && ((md(Pm - ka, nk) == ka) != (self == 1))) continue;
          B::batch(h, Cpp.off + (int64_t)Pm * rowsX * colsC + (int64_t)ka * na * v);
          for (size_t t : kv.second)
            B::seg(h, Xpp.off + (int64_t)Pm * rowsX * colsX + (int64_t)work[t].kc * v2, (int64_t)(t - c0) * wsz);
        }
        if (flop_acc) *flop_acc += (double)h.flops();
        b.g_push(pr);
      }
    }
  };
  // Z(i,j,m,b) = sum_cd t_ij^cd (mc|bd)~   (PP), then K3
  T4 Zpp = b.t4(AR_FIX, LK_PP, o, o, o, v);
  ladder(G, Zpp, Lov, o, Tpp, 1.0, "Z ladder", nullptr, nullptr, false);
  T4 Zk3 = b.relayout(Zpp, AR_FIX, LK_K3);
  b.perm(G, Zk3, Zpp, {0, 1, 2, 3}, 1.0, 0.0, "Zk3");

  // =====================================================================
  // Jacobian program: IN (x1 paper, x2 paper) -> OUT (y1, y2 paper)
  // =====================================================================
  Program& J = P.jac;
  P.off_x1 = b.alloc(AR_IN, nk * ov);
  P.off_x2 = b.alloc(AR_IN, nk * (int64_t)nk * nk * o2 * v2);
  if (b.alloc(AR_OUT, nk * ov) != P.off_x1 || b.alloc(AR_OUT, nk * (int64_t)nk * nk * o2 * v2) != P.off_x2)
    throw std::runtime_error("IN/OUT layouts differ");
  auto X1 = [&](int k) { return P.off_x1 + (int64_t)k * ov; };  // IN
  auto Y1 = [&](int k) { return P.off_x1 + (int64_t)k * ov; };  // OUT
  T4 xin{AR_IN, P.off_x2, Layout{LK_K3, nk, {o, o, v, v}}};
  T4 yout{AR_OUT, P.off_x2, Layout{LK_K3, nk, {o, o, v, v}}};

  // symmetrized input in supercell units: xs = (x + S x) / (2 Nk)
  T4 xs = b.t4(AR_SCR, LK_K3, o, o, v, v);
  b.perm(J, xs, xin, {0, 1, 2, 3}, 0.5 / sNk, 0.0, "xs a");
  b.perm(J, xs, xin, {1, 0, 3, 2}, 0.5 / sNk, 0.0, "xs b");
  T4 xpp = b.relayout(xs, AR_SCR, LK_PP);
  b.perm(J, xpp, xs, {0, 1, 2, 3}, 1.0, 0.0, "xpp");
  T4 xc = b.relayout(xs, AR_SCR, LK_PH);
  b.perm(J, xc, xs, {0, 1, 3, 2}, 1.0, 0.0, "xc");
  T4 Ud = b.relayout(xs, AR_SCR, LK_PH);
  b.perm(J, Ud, xs, {0, 1, 2, 3}, 2.0, 0.0, "Ud a");
  b.perm(J, Ud, xs, {0, 1, 3, 2}, -1.0, 0.0, "Ud b");
  T4 Uk3 = b.relayout(xs, AR_SCR, LK_K3);
  b.perm(J, Uk3, xs, {0, 1, 2, 3}, 2.0, 0.0, "Uk3 a");
  b.perm(J, Uk3, xs, {0, 1, 3, 2}, -1.0, 0.0, "Uk3 b");

  T4 r = b.t4(AR_SCR, LK_K3, o, o, v, v);     // doubles accumulator before (1 + S)
  T4 rpp = b.t4(AR_SCR, LK_PP, o, o, v, v);   // symmetric terms (weight 1/2)
  T4 Zc = b.t4(AR_SCR, LK_PH, o, o, v, v);    // ring C product
  T4 Zd = b.t4(AR_SCR, LK_PH, o, o, v, v);    // ring D product

  // [A] ladder
  ladder(J, rpp, tLvv, v, xpp, 0.5, "ladder", &P.ladder_flops, &P.wbuild_flops, true);
  // [B] hole-hole: rpp += 1/2 Whh^T xpp ; Yhh = V xpp^T ; rpp += 1/2 Yhh^T Tpp.  The last
  //     product shares its right factor with B': Yhh is formed in (13), collects both
  //     left factors, and one GEMM ("hh quad") applies Tpp.
  b.pair_gemm(J, rpp, Whh, 1, xpp, 0, 0.5, 0.0, "hh");
  // [C] ring: Zc = WC xc - 1/2 (xc M) Tc ; the second product is formed in (14) together
  //     with C' (YC = -1/2 xc M + WCx, one Tc product)
  b.pair_gemm(J, Zc, WC, 0, xc, 0, 1.0, 0.0, "ring C");
  // [D] ring: Zd = 1/2 WD Ud + 1/4 (Ud ML) ud ; the second product is formed in (15)
  //     together with D' (YD = 1/2 Ud ML + WDx, one ud product)
  b.pair_gemm(J, Zd, WD, 0, Ud, 0, 0.5, 0.0, "ring D");
  // [E] Fock-like terms in K3 blocks
  auto e_vv = [&](Program& pr, const T4& r, const T4& A, int64_t Bvv, int arB, double alpha, const char* tag) {
    // r[ki,kj,ka](ij a, b) += alpha sum_c A[ki,kj,ka](ij a, c) Bvv[kb](b, c)
    Gemm& g = b.g_new((int)(o2 * v), v, v, 0, 1, v, v, v, A.ar, arB, r.ar, alpha, 0.0, tag);
    for (int ki = 0; ki < nk; ++ki)
      for (int kj = 0; kj < nk; ++kj)
        for (int ka = 0; ka < nk; ++ka) {
          int kbb = kb3(ki, kj, ka);
          B::batch(g, r.off + layout_offset(r.L, ki, kj, ka, 0, 0, 0, 0));
          B::seg(g, A.off + layout_offset(A.L, ki, kj, ka, 0, 0, 0, 0), Bvv + (int64_t)kbb * v2);
        }
    b.g_push(pr);
  };
  auto e_oo = [&](Program& pr, const T4& r, const T4& Bx, int64_t Aoo, int arA, double alpha, const char* tag) {
    // r[ki,kj,ka](i, j, ab) += alpha sum_k Aoo[kj](k, j) Bx[ki,kj,ka](i, k, ab)
    Gemm& g = b.g_new(o, (int)v2, o, 1, 0, o, v2, v2, arA, Bx.ar, r.ar, alpha, 0.0, tag);
    for (int ki = 0; ki < nk; ++ki)
      for (int kj = 0; kj < nk; ++kj)
        for (int ka = 0; ka < nk; ++ka)
          for (int i = 0; i < o; ++i) {
            B::batch(g, r.off + layout_offset(r.L, ki, kj, ka, i, 0, 0, 0));
            B::seg(g, Aoo + (int64_t)kj * o2, Bx.off + layout_offset(Bx.L, ki, kj, ka, i, 0, 0, 0));
          }
    b.g_push(pr);
  };
  e_vv(J, r, xs, Fv, AR_FIX, 1.0, "E vv");
  e_oo(J, r, xs, Fo, AR_FIX, -1.0, "E oo");
  // The quadratic Fock-like terms r -= t YEv^T, r -= YEo^T t share the left factor t with
  // the derivative-Fock terms below (r += t f'vv^T, r -= f'oo^T t): YEv and YEo are
  // accumulated into f'vv (weight -1) and f'oo (weight +1) and applied by those two GEMMs.
  int64_t dfvv = b.alloc(AR_SCR, nk * v2), dfoo = b.alloc(AR_SCR, nk * o2);
  yev(J, dfvv, AR_SCR, Uk3, -1.0, "YEv");
  yeo(J, dfoo, AR_SCR, Uk3, 1.0, "YEo");

  // singles from X2: y1 += Ud_0 fovT + sum_mef U (ae|mf) - sum_mne U (ne|mi)
  {
    Gemm& g = b.g_new((int)(nk * ov), 1, (int)(nk * ov), 0, 0, nk * ov, 1, 1, AR_SCR, AR_FIX, AR_OUT, 1.0,
                      0.0, "S1");
    B::batch(g, Y1(0));
    B::seg(g, Ud.off, fovT);  // q = 0 block of Ud
    b.g_push(J);
  }
  // VQ[k1][k2][i][e][Q] = sum_{k,n} U[k1,k,k2](i,n)[e][f] Lov[k,kf][Q](n,f)^T
  int64_t VQ = b.alloc(AR_SCR, (int64_t)nk * nk * ov * Q);
  {
    Gemm& g = b.g_new(v, Q, v, 0, 1, v, ov, Q, AR_SCR, AR_FIX, AR_SCR, 1.0, 0.0, "VQ");
    for (int k1 = 0; k1 < nk; ++k1)
      for (int k2 = 0; k2 < nk; ++k2)
        for (int i = 0; i < o; ++i) {
          B::batch(g, VQ + (((int64_t)k1 * nk + k2) * o + i) * v * Q);
          for (int k = 0; k < nk; ++k) {
            int kf = md(k1 + k - k2, nk);
            for (int nn2 = 0; nn2 < o; ++nn2)
              B::seg(g, Uk3.off + layout_offset(Uk3.L, k1, k, k2, i, nn2, 0, 0),
                     DF(Lov, o, v, k, kf) + (int64_t)nn2 * v);
          }
        }
    b.g_push(J);
  }
  {
    // y1[ki](i,a) += sum_{ke,e,Q} VQ[ki][ke][i][e][Q] LvvT[ki,ke][Q][e][a]
    Gemm& g = b.g_new(o, v, Q, 0, 0, (int64_t)v * Q, v2, v, AR_SCR, AR_FIX, AR_OUT, 1.0, 0.0, "S2");
    for (int ki = 0; ki < nk; ++ki) {
      B::batch(g, Y1(ki));
      for (int ke = 0; ke < nk; ++ke)
        for (int e = 0; e < v; ++e)
          B::seg(g, VQ + ((int64_t)ki * nk + ke) * o * v * Q + (int64_t)e * Q,
                 DF(LvvT, v, v, ki, ke) + (int64_t)e * v);
    }
    b.g_push(J);
    // y1[ki](i,a) -= sum_{km,m,Q} Loo~[km,ki][Q](m,i) VQ[km][ki][m][a][Q]
    Gemm& h = b.g_new(o, v, Q, 1, 1, o2, Q, v, AR_FIX, AR_SCR, AR_OUT, -1.0, 0.0, "S3");
    for (int ki = 0; ki < nk; ++ki) {
      B::batch(h, Y1(ki));
      for (int km = 0; km < nk; ++km)
        for (int m = 0; m < o; ++m)
          B::seg(h, DF(tLoo, o, o, km, ki) + (int64_t)m * o, VQ + (((int64_t)km * nk + ki) * o + m) * v * Q);
    }
    b.g_push(J);
  }

  // ---------------- X1 part ----------------
  int64_t dLvo = b.alloc(AR_SCR, dfsz(v, o)), dLoo = b.alloc(AR_SCR, dfsz(o, o)),
          dLvv = b.alloc(AR_SCR, dfsz(v, v)), Ey = b.alloc(AR_SCR, dfsz(v, o));
  {
    // dLvo = Lvv~ x[k2]^T - x[k1]^T Loo~
    Gemm& g = b.g_new(Q * v, o, v, 0, 1, v, v, o, AR_FIX, AR_IN, AR_SCR, 1.0, 0.0, "dLvo a");
    for (int k1 = 0; k1 < nk; ++k1)
      for (int k2 = 0; k2 < nk; ++k2) {
        B::batch(g, DF(dLvo, v, o, k1, k2));
        B::seg(g, DF(tLvv, v, v, k1, k2), X1(k2));
      }
    b.g_push(J);
    Gemm& h = b.g_new(v, o, o, 1, 0, v, o, o, AR_IN, AR_FIX, AR_SCR, -1.0, 0.0, "dLvo b");
    for (int k1 = 0; k1 < nk; ++k1)
      for (int k2 = 0; k2 < nk; ++k2)
        for (int q = 0; q < Q; ++q) {
          B::batch(h, DF(dLvo, v, o, k1, k2) + (int64_t)q * ov);
          B::seg(h, X1(k1), DF(tLoo, o, o, k1, k2) + (int64_t)q * o2);
        }
    b.g_push(J);
    // dLoo = Lov x[k2]^T
    Gemm& g2 = b.g_new(Q * o, o, v, 0, 1, v, v, o, AR_FIX, AR_IN, AR_SCR, 1.0, 0.0, "dLoo");
    for (int k1 = 0; k1 < nk; ++k1)
      for (int k2 = 0; k2 < nk; ++k2) {
        B::batch(g2, DF(dLoo, o, o, k1, k2));
        B::seg(g2, DF(Lov, o, v, k1, k2), X1(k2));
      }
    b.g_push(J);
    // dLvv = -x[k1]^T Lov
    Gemm& g3 = b.g_new(v, v, o, 1, 0, v, v, v, AR_IN, AR_FIX, AR_SCR, -1.0, 0.0, "dLvv");
    for (int k1 = 0; k1 < nk; ++k1)
      for (int k2 = 0; k2 < nk; ++k2)
        for (int q = 0; q < Q; ++q) {
          B::batch(g3, DF(dLvv, v, v, k1, k2) + (int64_t)q * v2);
          B::seg(g3, X1(k1), DF(Lov, o, v, k1, k2) + (int64_t)q * ov);
        }
    b.g_push(J);
    // Ey[k1,k2][Q](e,j) = sum_m x[k1](m,e) Loo~[k1,k2][Q](m,j)
    Gemm& g4 = b.g_new(v, o, o, 1, 0, v, o, o, AR_IN, AR_FIX, AR_SCR, 1.0, 0.0, "Ey");
    for (int k1 = 0; k1 < nk; ++k1)
      for (int k2 = 0; k2 < nk; ++k2)
        for (int q = 0; q < Q; ++q) {
          B::batch(g4, DF(Ey, v, o, k1, k2) + (int64_t)q * ov);
          B::seg(g4, X1(k1), DF(tLoo, o, o, k1, k2) + (int64_t)q * o2);
        }
    b.g_push(J);
  }
  // (11) (ai|bj)' : logical (a,b,i,j) in CH, into r with weight 1/2
  {
    T4 Iai = b.t4(AR_SCR, LK_CH, v, v, o, o);
    chem(J, Iai, dLvo, v, o, tLvo, v, o, AR_SCR, AR_FIX, 1.0, "(ai|bj)' a");
    chem(J, Iai, tLvo, v, o, dLvo, v, o, AR_FIX, AR_SCR, 1.0, "(ai|bj)' b");
    b.perm(J, r, Iai, {2, 3, 0, 1}, 0.5, 0.0, "(ai|bj)' -> r");
  }
  // (12) A' : r[ki,kj,ka](ij)[a][b] -= sum_m x[ka](m,a) Z[ki,kj,ka](ij)[m][b]
  {
    Gemm& g = b.g_new(v, v, o, 1, 0, v, v, v, AR_IN, AR_FIX, AR_SCR, -1.0, 0.0, "A'");
    for (int ki = 0; ki < nk; ++ki)
      for (int kj = 0; kj < nk; ++kj)
        for (int ka = 0; ka < nk; ++ka)
          for (int ij = 0; ij < o2; ++ij) {
            B::batch(g, r.off + layout_offset(r.L, ki, kj, ka, 0, 0, 0, 0) + (int64_t)ij * v2);
            B::seg(g, X1(ka), Zk3.off + layout_offset(Zk3.L, ki, kj, ka, 0, 0, 0, 0) + (int64_t)ij * ov);
          }
    b.g_push(J);
  }
  // (13) B' : (ki|lj)' logical (k,l,i,j) -> PP, added to Yhh ; rpp += 1/2 Yhh^T Tpp
  {
    T4 Ioox = b.t4(AR_SCR, LK_CH, o, o, o, o);
    chem(J, Ioox, dLoo, o, o, tLoo, o, o, AR_SCR, AR_FIX, 1.0, "(ki|lj)' a");
    chem(J, Ioox, tLoo, o, o, dLoo, o, o, AR_FIX, AR_SCR, 1.0, "(ki|lj)' b");
    T4 Yhh = b.t4(AR_SCR, LK_PP, o, o, o, o);
    b.pair_gemm(J, Yhh, Vpp, 0, xpp, 1, 1.0, 0.0, "Yhh");
    b.perm(J, Yhh, Ioox, {0, 1, 2, 3}, 1.0, 0.0, "(ki|lj)' pp");
    b.pair_gemm(J, rpp, Yhh, 1, Tpp, 0, 0.5, 0.0, "hh quad");  // hh quad + B'
  }
  // (14) C' : (ki|ac)' logical (k,a,i,c) -> WCx (PH (i,c,a,k)), added to YC ; Zc += YC Tc
  {
    T4 Ix = b.t4(AR_SCR, LK_CH, o, v, o, v);
    chem(J, Ix, dLoo, o, o, tLvv, v, v, AR_SCR, AR_FIX, 1.0, "(ki|ac)' a");
    chem(J, Ix, tLoo, o, o, dLvv, v, v, AR_FIX, AR_SCR, 1.0, "(ki|ac)' b");
    T4 YC = b.t4(AR_SCR, LK_PH, o, v, v, o);
    b.pair_gemm(J, YC, xc, 0, Mph, 0, -0.5, 0.0, "YC");
    b.perm(J, YC, Ix, {3, 2, 0, 1}, 1.0, 0.0, "WCx");
    b.pair_gemm(J, Zc, YC, 0, Tc, 0, 1.0, 0.0, "ring C quad");  // ring C quad + C'
  }
  // (15) D' : 2(ai|kc)' - (ac|ki)' -> WDx, added to YD ; Zd += 1/2 YD ud
  {
    T4 Ia = b.t4(AR_SCR, LK_CH, v, o, o, v);  // (a,k,i,c)
    chem(J, Ia, dLvo, v, o, Lov, o, v, AR_SCR, AR_FIX, 1.0, "(ai|kc)'");
    T4 Ib = b.t4(AR_SCR, LK_CH, v, o, v, o);  // (a,k,c,i)
    chem(J, Ib, dLvv, v, v, tLoo, o, o, AR_SCR, AR_FIX, 1.0, "(ac|ki)' a");
    chem(J, Ib, tLvv, v, v, dLoo, o, o, AR_FIX, AR_SCR, 1.0, "(ac|ki)' b");
    T4 YD = b.t4(AR_SCR, LK_PH, o, v, v, o);
    b.pair_gemm(J, YD, Ud, 0, MLph, 0, 0.5, 0.0, "YD");
    b.perm(J, YD, Ia, {2, 3, 0, 1}, 2.0, 0.0, "WDx a");
    b.perm(J, YD, Ib, {2, 3, 1, 0}, -1.0, 0.0, "WDx b");
    b.pair_gemm(J, Zd, YD, 0, ud, 0, 0.5, 0.0, "ring D quad");  // ring D quad + D'
  }
  // Coulomb vector of x1: Jx[Q] = sum_k sum_(m,e) Lov[k,k][Q](m,e) x1[k](m,e)
  int64_t Jx = b.alloc(AR_SCR, Q);
  {
    Gemm& g = b.g_new(Q, 1, (int)ov, 0, 0, ov, 1, 1, AR_FIX, AR_IN, AR_SCR, 1.0, 0.0, "Jx");
    B::batch(g, Jx);
    for (int k = 0; k < nk; ++k) B::seg(g, DF(Lov, o, v, k, k), X1(k));
    b.g_push(J);
  }
  // derivative Fock blocks f'vv[k](b,c), f'oo[k](k,j), f'vo[k](a,i), f'ov[k](m,e)
  int64_t dfvo = b.alloc(AR_SCR, nk * ov), dfov = b.alloc(AR_SCR, nk * ov), dfovT = b.alloc(AR_SCR, nk * ov);
  auto coul = [&](int64_t dst, int a, int c, int64_t Lbase, int la, int lc, double alpha, const char* tag) {
    Gemm& g = b.g_new(1, a * c, Q, 0, 0, Q, (int64_t)a * c, (int64_t)a * c, AR_SCR, AR_FIX, AR_SCR, alpha, 0.0,
                      tag);
    for (int k = 0; k < nk; ++k) {
      B::batch(g, dst + (int64_t)k * a * c);
      B::seg(g, Jx, DF(Lbase, la, lc, k, k));
    }
    b.g_push(J);
  };
  coul(dfvv, v, v, tLvv, v, v, 2.0, "f'vv J");
  coul(dfoo, o, o, tLoo, o, o, 2.0, "f'oo J");
  coul(dfvo, v, o, tLvo, v, o, 2.0, "f'vo J");
  coul(dfov, o, v, Lov, o, v, 2.0, "f'ov J");
  // exchange parts: C[k](p,q) += alpha sum_{k',Q} A[k,k'][Q](p,e) Bx[k',k][Q](e,q)
  auto exch = [&](int64_t dst, int a, int c, int e, int64_t Abase, int arA, int64_t Bbase, int arB, double alpha,
                  const char* tag) {
    Gemm& g = b.g_new(a, c, e, 0, 0, e, c, c, arA, arB, AR_SCR, alpha, 0.0, tag);
    for (int k = 0; k < nk; ++k) {
      B::batch(g, dst + (int64_t)k * a * c);
      for (int kp = 0; kp < nk; ++kp)
        for (int q = 0; q < Q; ++q)
          B::seg(g, Abase + (((int64_t)k * nk + kp) * Q + q) * a * e, Bbase + (((int64_t)kp * nk + k) * Q + q) * e * c);
    }
    b.g_push(J);
  };
  // f'vv: - sum_me x_m^e (be|mc) = + sum Lvv~[kb,km](b,e) dLvv[km,kb](e,c)
  exch(dfvv, v, v, v, tLvv, AR_FIX, dLvv, AR_SCR, 1.0, "f'vv K");
  // f'oo: - sum_me x_m^e (ke|mj) = - sum Lov[kj,km](k,e) Ey[km,kj](e,j)
  exch(dfoo, o, o, v, Lov, AR_FIX, Ey, AR_SCR, -1.0, "f'oo K");
  // f'vo: - sum_me x_m^e (ae|mi) = - sum Lvv~[k,km](a,e) Ey[km,k](e,i)
  exch(dfvo, v, o, v, tLvv, AR_FIX, Ey, AR_SCR, -1.0, "f'vo K");
  // f'ov: - sum_nf x_n^f (mf|ne) = + sum Lov[km,kn](m,f) dLvv[kn,km](f,e)
  exch(dfov, o, v, v, Lov, AR_FIX, dLvv, AR_SCR, 1.0, "f'ov K");
  // commutator parts: f'vv -= x[kb]^T f~ov ; f'oo += f~ov x^T
  {
    Gemm& g = b.g_new(v, v, o, 1, 0, v, v, v, AR_IN, AR_FIX, AR_SCR, -1.0, 0.0, "f'vv [f,xi]");
    for (int k = 0; k < nk; ++k) {
      B::batch(g, dfvv + (int64_t)k * v2);
      B::seg(g, X1(k), fblk(fov, o, v, k));
    }
    b.g_push(J);
    Gemm& h = b.g_new(o, o, v, 0, 1, v, v, o, AR_FIX, AR_IN, AR_SCR, 1.0, 0.0, "f'oo [f,xi]");
    for (int k = 0; k < nk; ++k) {
      B::batch(h, dfoo + (int64_t)k * o2);
      B::seg(h, fblk(fov, o, v, k), X1(k));
    }
    b.g_push(J);
  }
  // (16) E' : r += sum_c T_ij^ac f'_bc - sum_k T_ik^ab f'_kj
  e_vv(J, r, Tk3, dfvv, AR_SCR, 1.0, "E' vv");   // + E vv quad (through YEv)
  e_oo(J, r, Tk3, dfoo, AR_SCR, -1.0, "E' oo");  // + E oo quad (through YEo)
  // (17) singles from X1
  {
    // sum_e f~vv[k](a,e) x(i,e) -> y1[k](i,a)
    Gemm& g = b.g_new(o, v, v, 0, 1, v, v, v, AR_IN, AR_FIX, AR_OUT, 1.0, 0.0, "y1 f x");
    for (int k = 0; k < nk; ++k) {
      B::batch(g, Y1(k));
      B::seg(g, X1(k), fblk(fvv, v, v, k));
    }
    b.g_push(J);
    // - sum_m f~oo[k](m,i) x(m,a)
    Gemm& h = b.g_new(o, v, o, 1, 0, o, v, v, AR_FIX, AR_IN, AR_OUT, -1.0, 0.0, "y1 x f");
    for (int k = 0; k < nk; ++k) {
      B::batch(h, Y1(k));
      B::seg(h, fblk(foo, o, o, k), X1(k));
    }
    b.g_push(J);
    // - sum_n G[k](n,i) x(n,a)
    Gemm& h2 = b.g_new(o, v, o, 1, 0, o, v, v, AR_FIX, AR_IN, AR_OUT, -1.0, 0.0, "y1 G x");
    for (int k = 0; k < nk; ++k) {
      B::batch(h2, Y1(k));
      B::seg(h2, Gm + (int64_t)k * o2, X1(k));
    }
    b.g_push(J);
    // - sum_f x(i,f) H[k](a,f)
    Gemm& h3 = b.g_new(o, v, v, 0, 1, v, v, v, AR_IN, AR_FIX, AR_OUT, -1.0, 0.0, "y1 x H");
    for (int k = 0; k < nk; ++k) {
      B::batch(h3, Y1(k));
      B::seg(h3, X1(k), Hm + (int64_t)k * v2);
    }
    b.g_push(J);
  }
  b.btr(J, nk, v, o, AR_OUT, Y1(0), AR_SCR, dfvo, 1.0, "f'vo -> y1");
  b.btr(J, nk, o, v, AR_SCR, dfovT, AR_SCR, dfov, 1.0, "f'ov^T");
  {
    // y1 += ud_0 f'ovT   (sum_me u_im^ae f'_me)
    Gemm& g = b.g_new((int)(nk * ov), 1, (int)(nk * ov), 0, 0, nk * ov, 1, 1, AR_FIX, AR_SCR, AR_OUT, 1.0, 0.0,
                      "y1 u f'");
    B::batch(g, Y1(0));
    B::seg(g, ud.off, dfovT);
    b.g_push(J);
  }

  // ---------------- assemble the doubles output ----------------
  b.perm(J, r, rpp, {0, 1, 2, 3}, 1.0, 0.0, "rpp -> r");
  b.perm(J, r, Zc, {0, 1, 2, 3}, -0.5, 0.0, "Zc -> r");
  b.perm(J, r, Zc, {0, 1, 3, 2}, -1.0, 0.0, "Zc sw -> r");
  b.perm(J, r, Zd, {0, 1, 2, 3}, 1.0, 0.0, "Zd -> r");
  b.perm(J, yout, r, {0, 1, 2, 3}, sNk, 0.0, "y2 a");
  b.perm(J, yout, r, {1, 0, 3, 2}, sNk, 0.0, "y2 b");

  // =====================================================================
  // xi program: xi^X(t', mu) = dOmega(t'; h + eps mu)/d eps (paper units), the
  // perturbed-amplitude right-hand side of Eq. 12.  t' is read from IN (x1/x2
  // regions, paper units), the one-body operator mu from FIX (oo/ov/vo/vv blocks and
  // ov transposed).  Omega is linear in the one-body part, so
  //   xi_1 = mu~_ai + sum_me u_im^ae mu~_me,
  //   xi_2 = P_ij^ab [sum_c t_ij^ac mu~_bc - sum_k t_ik^ab mu~_kj],   mu~ = (1-tau) mu (1+tau).
  // Not linear in IN, never transposed.
  // =====================================================================
  {
    P.off_mu = b.alloc(AR_FIX, nk * (o2 + 2 * ov + v2 + ov));
    const int64_t muoo = P.off_mu, muov = muoo + nk * o2, muvo = muov + nk * ov, muvv = muvo + nk * ov,
                  muovT = muvv + nk * v2;
    Program& X = P.xi;
    b.nonlinear = true;
    T4 tin{AR_IN, P.off_x2, Layout{LK_K3, nk, {o, o, v, v}}};
    T4 tk = b.t4(AR_SCR, LK_K3, o, o, v, v);
    b.perm(X, tk, tin, {0, 1, 2, 3}, 1.0 / sNk, 0.0, "xi t");
    T4 ux = b.relayout(tk, AR_SCR, LK_PH);
    b.perm(X, ux, tk, {0, 1, 2, 3}, 2.0, 0.0, "xi u a");
    b.perm(X, ux, tk, {0, 1, 3, 2}, -1.0, 0.0, "xi u b");
    int64_t moo = b.alloc(AR_SCR, nk * o2), mvv = b.alloc(AR_SCR, nk * v2), mvo = b.alloc(AR_SCR, nk * ov);
    auto flat = [&](int ar, int64_t off, int64_t nel) { return T4{ar, off, Layout{LK_K3, 1, {1, 1, 1, (int)nel}}}; };
    b.perm(X, flat(AR_SCR, moo, nk * o2), flat(AR_FIX, muoo, nk * o2), {0, 1, 2, 3}, 1.0, 0.0, "mu~oo");
    b.perm(X, flat(AR_SCR, mvv, nk * v2), flat(AR_FIX, muvv, nk * v2), {0, 1, 2, 3}, 1.0, 0.0, "mu~vv");
    b.perm(X, flat(AR_SCR, mvo, nk * ov), flat(AR_FIX, muvo, nk * ov), {0, 1, 2, 3}, 1.0, 0.0, "mu~vo");
    {
      Gemm& g = b.g_new(o, o, v, 0, 1, v, v, o, AR_FIX, AR_IN, AR_SCR, 1.0, 0.0, "mu~oo t");
      for (int k = 0; k < nk; ++k) {
        B::batch(g, moo + (int64_t)k * o2);
        B::seg(g, muov + (int64_t)k * ov, P.off_x1 + (int64_t)k * ov);
      }
      b.g_push(X);
      Gemm& h = b.g_new(v, v, o, 1, 0, v, v, v, AR_IN, AR_FIX, AR_SCR, -1.0, 0.0, "mu~vv t");
      for (int k = 0; k < nk; ++k) {
        B::batch(h, mvv + (int64_t)k * v2);
        B::seg(h, P.off_x1 + (int64_t)k * ov, muov + (int64_t)k * ov);
      }
      b.g_push(X);
      Gemm& h2 = b.g_new(v, o, v, 0, 1, v, v, o, AR_SCR, AR_IN, AR_SCR, 1.0, 0.0, "mu~vo a");
      for (int k = 0; k < nk; ++k) {
        B::batch(h2, mvo + (int64_t)k * ov);
        B::seg(h2, mvv + (int64_t)k * v2, P.off_x1 + (int64_t)k * ov);
      }
      b.g_push(X);
      Gemm& h3 = b.g_new(v, o, o, 1, 0, v, o, o, AR_IN, AR_FIX, AR_SCR, -1.0, 0.0, "mu~vo b");
      for (int k = 0; k < nk; ++k) {
        B::batch(h3, mvo + (int64_t)k * ov);
        B::seg(h3, P.off_x1 + (int64_t)k * ov, muoo + (int64_t)k * o2);
      }
      b.g_push(X);
    }
    T4 rx = b.t4(AR_SCR, LK_K3, o, o, v, v);
    e_vv(X, rx, tk, mvv, AR_SCR, 1.0, "xi E vv");
    e_oo(X, rx, tk, moo, AR_SCR, -1.0, "xi E oo");
    b.perm(X, yout, rx, {0, 1, 2, 3}, sNk, 0.0, "xi y2 a");
    b.perm(X, yout, rx, {1, 0, 3, 2}, sNk, 0.0, "xi y2 b");
    b.btr(X, nk, v, o, AR_OUT, Y1(0), AR_SCR, mvo, 1.0, "xi mu~vo -> y1");
    Gemm& g = b.g_new((int)(nk * ov), 1, (int)(nk * ov), 0, 0, nk * ov, 1, 1, AR_SCR, AR_FIX, AR_OUT, 1.0, 0.0,
                      "xi u mu");
    B::batch(g, Y1(0));
    B::seg(g, ux.off, muovT);
    b.g_push(X);
    b.nonlinear = false;
  }
  // egrad program: y1 += 2 sum_jb L_iajb x1_jb, L_iajb = 2(ia|jb) - (ib|ja): the singles-singles
  // second derivative of the supercell energy (Eq. 6), needed by the quadratic term of Eq. 15.
  {
    Program& E = P.egrad;
    int64_t tmp = b.alloc(AR_SCR, nk * ov);
    Gemm& g = b.g_new((int)(nk * ov), 1, (int)(nk * ov), 0, 0, nk * ov, 1, 1, AR_FIX, AR_IN, AR_SCR, 2.0, 0.0,
                      "egrad");
    B::batch(g, tmp);
    B::seg(g, MLph.off, P.off_x1);
    b.g_push(E);
    b.btr(E, nk, v, o, AR_OUT, Y1(0), AR_SCR, tmp, 1.0, "egrad -> y1");
  }

  // omega0 program: the residual at t = 0 in paper units.  Doubles: <ab|ij> of the
  // alpha-beta block, (ai|bj) summed over the undressed DF factors (times Nk for paper
  // units; pair-symmetric by construction); singles: f_ai = 0 for the canonical Fock
  // matrix the boundary takes.  With it Omega(t) = Omega(0) + 1/2 [A(s1 t) t + A(s2 t) t],
  // s1,2 = (1 -+ 1/sqrt 3) / 2: two-point Gauss-Legendre of d/ds Omega(s t) = A(s t) t,
  // exact because that is a cubic polynomial in s (Omega has degree 4, Eqs. 7-8).
  {
    Program& O = P.omega0;
    T4 I0 = b.t4(AR_SCR, LK_CH, v, v, o, o);  // logical (a,b,i,j) = (ai|bj)
    chem(O, I0, P.off_Lvo, v, o, P.off_Lvo, v, o, AR_FIX, AR_FIX, 1.0, "(ai|bj)");
    b.perm(O, yout, I0, {2, 3, 0, 1}, sNk, 0.0, "(ai|bj) -> y2");
  }
  // tgrad program: dE/dt for the supercell energy E = sum (2(ia|jb) - (ib|ja)) (t_ij^ab +
  // t_i^a t_j^b) (Eq. 6; f_ia = 0), with respect to the paper-unit amplitudes (t2 = Nk s2):
  // singles 2 sum_jb L_iajb t_jb, doubles L_iajb / Nk.  With it the Lambda equations
  // (Eqs. 10-11) read A^T lam = -dE/dt in the plain pairing.
  {
    Program& E = P.tgrad;
    b.nonlinear = true;
    int64_t tmp = b.alloc(AR_SCR, nk * ov);
    Gemm& g = b.g_new((int)(nk * ov), 1, (int)(nk * ov), 0, 0, nk * ov, 1, 1, AR_FIX, AR_IN, AR_SCR, 2.0, 0.0,
                      "tgrad 1");
    B::batch(g, tmp);
    B::seg(g, MLph.off, P.off_x1);
    b.g_push(E);
    b.btr(E, nk, v, o, AR_OUT, Y1(0), AR_SCR, tmp, 1.0, "tgrad 1 -> y1");
    b.perm(E, yout, Vk3, {0, 1, 2, 3}, 2.0 / sNk, 0.0, "tgrad 2 a");
    b.perm(E, yout, Vk3, {0, 1, 3, 2}, -1.0 / sNk, 0.0, "tgrad 2 b");
    b.nonlinear = false;
  }

  pack_scratch(P, {&P.jac, &P.xi, &P.egrad, &P.omega0, &P.tgrad});
  for (Program* pr : {&P.jac, &P.xi, &P.egrad, &P.omega0, &P.tgrad}) fold_first_writes(P, *pr);

  double tot = 0;
  for (const Op& op : J.ops)
    if (op.kind == OP_GEMM) tot += (double)P.gemms[op.idx].flops();
  P.jac_flops = tot;
  return P;
}

// ---------------------------------------------------------------------------
// bounds validation
// ---------------------------------------------------------------------------
std::string validate_plan(const Plan& P, const Program& pr) {
  auto chk = [&](int ar, int64_t off, int64_t ext, const std::string& what) -> std::string {
    if (ar < 0 || ar >= AR_COUNT) return what + ": bad arena";
    if (off < 0 || ext < 0 || off + ext > P.arena_size[ar])
      return what + ": out of bounds (arena " + std::to_string(ar) + ", off " + std::to_string(off) + ", extent " +
             std::to_string(ext) + ", size " + std::to_string(P.arena_size[ar]) + ")";
    return "";
  };
  for (const Op& op : pr.ops) {
    std::string e;
    if (op.kind == OP_GEMM) {
      const Gemm& g = P.gemms[op.idx];
      if (g.M <= 0 || g.N <= 0 || g.K <= 0) return "gemm " + g.tag + ": empty";
      int64_t rA = g.ta ? g.K : g.M, cA = g.ta ? g.M : g.K;
      int64_t rB = g.tb ? g.N : g.K, cB = g.tb ? g.K : g.N;
      if (cA > g.lda || cB > g.ldb) return "gemm " + g.tag + ": leading dimension";
      int64_t extA = (rA - 1) * g.lda + cA, extB = (rB - 1) * g.ldb + cB;
      int64_t extC = g.epi == 0 ? (int64_t)(g.M - 1) * g.ldc + g.N
                                : (int64_t)(g.M / g.ep[2]) * g.ep[1] * g.ep[2] * g.ep[3];
      if (g.epi == 0 && g.N > g.ldc) return "gemm " + g.tag + ": ldc";
      if ((int)g.sbeg.size() != g.nbatch() + 1) return "gemm " + g.tag + ": segment table";
      for (int b = 0; b < g.nbatch(); ++b) {
        if (!(e = chk(g.arC, g.coff[b], extC, "gemm C " + g.tag)).empty()) return e;
        for (int s = g.sbeg[b]; s < g.sbeg[b + 1]; ++s) {
          if (!(e = chk(g.arA, g.aoff[s], extA, "gemm A " + g.tag)).empty()) return e;
          if (!(e = chk(g.arB, g.boff[s], extB, "gemm B " + g.tag)).empty()) return e;
        }
      }
    } else if (op.kind == OP_PERM) {
      const Perm& p = P.perms[op.idx];
      if (p.src.size() != p.dst.size()) return "perm " + p.tag + ": sizes";
      if (!(e = chk(p.arS, p.offS, p.src.size(), "perm src " + p.tag)).empty()) return e;
      if (!(e = chk(p.arD, p.offD, p.dst.size(), "perm dst " + p.tag)).empty()) return e;
      if (p.arS == p.arD && p.offS < p.offD + p.dst.size() && p.offD < p.offS + p.src.size())
        return "perm " + p.tag + ": source and destination overlap";
    } else if (op.kind == OP_BTRANS) {
      const BTrans& t = P.btrans[op.idx];
      int64_t n = (int64_t)t.nb * t.R * t.C;
      if (!(e = chk(t.arS, t.offS, n, "btrans src " + t.tag)).empty()) return e;
      if (!(e = chk(t.arD, t.offD, n, "btrans dst " + t.tag)).empty()) return e;
    } else if (op.kind == OP_ZERO) {
      if (op.idx < 0 || op.idx >= (int)P.zeros.size()) return "zero: bad index";
      const ZeroSpec& z = P.zeros[op.idx];
      if (!(e = chk(z.arena, z.off, z.n, "zero")).empty()) return e;
    } else {
      return "unknown op kind";
    }
  }
  return "";
}

// True when the C tiles of g (all batch entries) cover [off, off + n) exactly, each element once.
static bool gemm_covers(const Gemm& g, int64_t off, int64_t n) {
  if (g.epi != 0 || (int64_t)g.M * g.N * g.nbatch() != n) return false;
  std::vector<std::pair<int64_t, int64_t>> iv;  // row segments [start, end)
  iv.reserve((size_t)g.M * g.nbatch());
  for (int b = 0; b < g.nbatch(); ++b) {
    if (g.sbeg[b + 1] <= g.sbeg[b]) return false;  // an empty entry: its kernels may skip the tile
    for (int m = 0; m < g.M; ++m) iv.push_back({g.coff[b] + (int64_t)m * g.ldc, g.coff[b] + (int64_t)m * g.ldc + g.N});
  }
  std::sort(iv.begin(), iv.end());
  int64_t at = off;
  for (const auto& x : iv) {
    if (x.first != at) return false;  // a gap or an overlap
    at = x.second;
  }
  return at == off + n;
}

// True when any operand segment of g lies (partly) in arena ar, [off, off + n).
static bool gemm_reads(const Gemm& g, int ar, int64_t off, int64_t n) {
  const int64_t rA = g.ta ? g.K : g.M, cA = g.ta ? g.M : g.K;
  const int64_t rB = g.tb ? g.N : g.K, cB = g.tb ? g.K : g.N;
  const int64_t extA = (rA - 1) * g.lda + cA, extB = (rB - 1) * g.ldb + cB;
  for (size_t s = 0; s < g.aoff.size(); ++s) {
    if (g.arA == ar && g.aoff[s] < off + n && off < g.aoff[s] + extA) return true;
    if (g.arB == ar && g.boff[s] < off + n && off < g.boff[s] + extB) return true;
  }
  return false;
}

void fold_first_writes(Plan& P, Program& pr) {
  std::vector<Op> out;
  out.reserve(pr.ops.size());
  for (const Op& op : pr.ops) {
    bool folded = false;
    if (op.kind == OP_GEMM && !op.fixed_only && !P.gemms[op.idx].store) {
      for (int j = (int)out.size() - 1; j >= 0 && out[j].kind == OP_ZERO; --j) {
        const ZeroSpec& z = P.zeros[out[j].idx];
        const Gemm& g = P.gemms[op.idx];
        if (g.arC == z.arena && gemm_covers(g, z.off, z.used) && !gemm_reads(g, z.arena, z.off, z.n)) {
          Gemm s = g;
          s.store = 1;
          P.gemms.push_back(s);
          Op o2 = op;
          o2.idx = (int)P.gemms.size() - 1;
          out.erase(out.begin() + j);
          out.push_back(o2);
          folded = true;
          break;
        }
      }
    }
    if (op.kind == OP_PERM && !P.perms[op.idx].store) {
      const Perm p = P.perms[op.idx];
      // the zero ops directly ahead of this one (a buffer is zeroed just before its first use)
      for (int j = (int)out.size() - 1; j >= 0 && out[j].kind == OP_ZERO; --j) {
        const ZeroSpec& z = P.zeros[out[j].idx];
        const bool covers = p.arD == z.arena && p.offD == z.off && p.dst.size() == z.used;
        const bool reads = p.arS == z.arena && p.offS < z.off + z.n && z.off < p.offS + p.src.size();
        if (covers && !reads) {
          Perm s = p;
          s.store = 1;
          P.perms.push_back(s);
          Op o2 = op;
          o2.idx = (int)P.perms.size() - 1;
          out.erase(out.begin() + j);
          out.push_back(o2);
          folded = true;
          break;
        }
      }
    }
    if (!folded) out.push_back(op);
  }
  pr.ops = out;
}

// ---------------------------------------------------------------------------
// transposition
// ---------------------------------------------------------------------------
static bool var_arena(int ar) { return ar == AR_IN || ar == AR_OUT || ar == AR_SCR; }

Program transpose_program(Plan& P, const Program& fwd) {
  Program out;
  std::vector<Op> rev;
  // fixed-only ops (W builds) must stay ahead of the contraction that uses them:
  // walk backwards, and when a variable GEMM reads the WS arena, emit the fixed
  // build op(s) that precede it in the forward program first.
  std::vector<int> pending;  // index in fwd of fixed-only ops not yet emitted
  // Only W builds write the WS arena and the contractions only read it, so a build is
  // emitted once for the run of transposed contractions that use it (the forward program
  // builds one W chunk for both ladder contractions of that chunk).
  int last_build = -1;
  for (int i = (int)fwd.ops.size() - 1; i >= 0; --i) {
    const Op& op = fwd.ops[i];
    if (op.fixed_only || op.kind == OP_ZERO) continue;
    if (op.zl >= 0)
      for (int zi : P.zlists[op.zl]) {
        Op z;
        z.kind = OP_ZERO;
        z.idx = zi;
        out.ops.push_back(z);
      }
    if (op.kind == OP_GEMM) {
      const Gemm& g = P.gemms[op.idx];
      if (g.arA == AR_WS || g.arB == AR_WS) {
        // find the nearest preceding fixed-only op (its W build)
        for (int j = i - 1; j >= 0; --j)
          if (fwd.ops[j].fixed_only) {
            if (j != last_build) out.ops.push_back(fwd.ops[j]);
            last_build = j;
            break;
          }
      }
      Gemm g2 = g;  // copy before push_back invalidates
      Gemm t;
      t.ar = g2.ar;
      t.ai = g2.ai;
      t.epi = 0;
      t.tag = g2.tag + "^T";
      bool bvar = var_arena(g2.arB);
      // group segments by the target (variable operand) offset
      std::map<int64_t, std::vector<std::pair<int64_t, int64_t>>> tgt;  // target -> (fixed operand, Cbar)
      for (int b = 0; b < g2.nbatch(); ++b)
        for (int s = g2.sbeg[b]; s < g2.sbeg[b + 1]; ++s) {
          int64_t to = bvar ? g2.boff[s] : g2.aoff[s];
          int64_t fo = bvar ? g2.aoff[s] : g2.boff[s];
          tgt[to].push_back({fo, g2.coff[b]});
        }
      if (bvar) {
        if (g2.tb == 0) {
          // Bbar[k][n] += alpha sum_m opA(m,k) Cbar[m][n]
          t.M = g2.K; t.N = g2.N; t.K = g2.M;
          t.ta = !g2.ta; t.lda = g2.lda; t.arA = g2.arA;
          t.tb = 0; t.ldb = g2.ldc; t.arB = g2.arC;
          t.ldc = g2.ldb; t.arC = g2.arB;
          t.sbeg.push_back(0);
          for (auto& kv : tgt) {
            t.coff.push_back(kv.first);
            t.sbeg.push_back(t.sbeg.back());
            for (auto& fc : kv.second) {
              t.aoff.push_back(fc.first);
              t.boff.push_back(fc.second);
              t.sbeg.back()++;
            }
          }
        } else {
          // B stored [N][K]: Bbar[n][k] += alpha sum_m Cbar[m][n] opA(m,k)
          t.M = g2.N; t.N = g2.K; t.K = g2.M;
          t.ta = 1; t.lda = g2.ldc; t.arA = g2.arC;
          t.tb = g2.ta; t.ldb = g2.lda; t.arB = g2.arA;
          t.ldc = g2.ldb; t.arC = g2.arB;
          t.sbeg.push_back(0);
          for (auto& kv : tgt) {
            t.coff.push_back(kv.first);
            t.sbeg.push_back(t.sbeg.back());
            for (auto& fc : kv.second) {
              t.aoff.push_back(fc.second);
              t.boff.push_back(fc.first);
              t.sbeg.back()++;
            }
          }
        }
      } else {
        if (g2.ta == 0) {
          // Abar[m][k] += alpha sum_n Cbar[m][n] opB(k,n)
          t.M = g2.M; t.N = g2.K; t.K = g2.N;
          t.ta = 0; t.lda = g2.ldc; t.arA = g2.arC;
          t.tb = !g2.tb; t.ldb = g2.ldb; t.arB = g2.arB;
          t.ldc = g2.lda; t.arC = g2.arA;
          t.sbeg.push_back(0);
          for (auto& kv : tgt) {
            t.coff.push_back(kv.first);
            t.sbeg.push_back(t.sbeg.back());
            for (auto& fc : kv.second) {
              t.aoff.push_back(fc.second);
              t.boff.push_back(fc.first);
              t.sbeg.back()++;
            }
          }
        } else {
          // A stored [K][M]: Abar[k][m] += alpha sum_n opB(k,n) Cbar[m][n]
          t.M = g2.K; t.N = g2.M; t.K = g2.N;
          t.ta = g2.tb; t.lda = g2.ldb; t.arA = g2.arB;
          t.tb = 1; t.ldb = g2.ldc; t.arB = g2.arC;
          t.ldc = g2.lda; t.arC = g2.arA;
          t.sbeg.push_back(0);
          for (auto& kv : tgt) {
            t.coff.push_back(kv.first);
            t.sbeg.push_back(t.sbeg.back());
            for (auto& fc : kv.second) {
              t.aoff.push_back(fc.first);
              t.boff.push_back(fc.second);
              t.sbeg.back()++;
            }
          }
        }
      }
      P.gemms.push_back(t);
      Op o2;
      o2.kind = OP_GEMM;
      o2.idx = (int)P.gemms.size() - 1;
      out.ops.push_back(o2);
    } else if (op.kind == OP_PERM) {
      Perm p = P.perms[op.idx];
      Perm t;
      t.src = p.dst; t.dst = p.src;
      for (int s = 0; s < 4; ++s) t.pi[p.pi[s]] = s;
      t.ar = p.ar; t.ai = p.ai;
      t.arS = p.arD; t.arD = p.arS;
      t.offS = p.offD; t.offD = p.offS;
      t.tag = p.tag + "^T";
      P.perms.push_back(t);
      Op o2;
      o2.kind = OP_PERM;
      o2.idx = (int)P.perms.size() - 1;
      out.ops.push_back(o2);
    } else if (op.kind == OP_BTRANS) {
      BTrans p = P.btrans[op.idx];
      BTrans t;
      t.nb = p.nb; t.R = p.C; t.C = p.R;
      t.ar = p.ar; t.ai = p.ai;
      t.arS = p.arD; t.arD = p.arS;
      t.offS = p.offD; t.offD = p.offS;
      t.tag = p.tag + "^T";
      P.btrans.push_back(t);
      Op o2;
      o2.kind = OP_BTRANS;
      o2.idx = (int)P.btrans.size() - 1;
      out.ops.push_back(o2);
    }
  }
  (void)pending;
  fold_first_writes(P, out);
  return out;
}

}  // namespace lrcc
