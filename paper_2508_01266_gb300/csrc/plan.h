// Op-list ("plan") description of the k-blocked LR-CCSD Jacobian products.
//
// A plan is a straight-line list of linear-algebra ops on a handful of device
// arenas.  The ground-state program builds the T-dependent intermediates once per
// (integrals, T); the Jacobian program maps an input vector X (arena IN) to A.X
// (arena OUT) through per-RHS scratch (arena SCR).  Every Jacobian op is linear in
// the vector arenas, so the transpose product is the same list run backwards with
// each op transposed (transpose_op below).  Host code only: nothing here touches
// the GPU.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

struct lrcc_plan;  // introspection handle of include/lrcc.h

namespace lrcc {

enum Arena : int { AR_FIX = 0, AR_IN = 1, AR_OUT = 2, AR_SCR = 3, AR_WS = 4, AR_COUNT = 5 };

// Layouts of a logical 4-index tensor Z(1,2,3,4) with momentum rule k1+k2 = k3+k4
// and orbital extents n[0..3]; the fourth momentum is implied.
//   K3: [k1][k2][k3][i1][i2][i3][i4]
//   PP: [P][k1][i1][i2] x [k3][i3][i4]          P = k1 + k2 (= k3 + k4)
//   PH: [q][k1][i1][i3] x [k4][i4][i2]          q = k3 - k1 (= k2 - k4)
//   CH: [k1][k3][k2][i1][i3][i2][i4]            chemist pairs (1,3) x (2,4)
enum LayoutKind : int { LK_K3 = 0, LK_PP = 1, LK_PH = 2, LK_CH = 3 };

struct Layout {
  int kind = LK_K3;
  int nk = 1;
  int n[4] = {1, 1, 1, 1};
  int64_t size() const {
    return (int64_t)nk * nk * nk * n[0] * n[1] * n[2] * n[3];
  }
};

// Element offset of logical element (k1,k2,k3; i1..i4) in a layout.
int64_t layout_offset(const Layout& L, int k1, int k2, int k3, int i1, int i2, int i3, int i4);

// C (+)= alpha * sum_seg op(A_seg) op(B_seg), row-major, complex, no conjugation.
//   op(A)(m,k) = ta ? A[k*lda + m] : A[m*lda + k]
//   op(B)(k,n) = tb ? B[n*ldb + k] : B[k*ldb + n]
//   epi == 0:  C[m*ldc + n]
//   epi == 1:  m = a*nc + c, n = b*nd + d  ->  C[((a*nb + b)*nc + c)*nd + d] = (stored,
//              not accumulated: W-block workspace slots are reused across chunks)
//   store == 1 (epi == 0 only): C = alpha * sum (C is not read; set by fold_first_writes)
struct Gemm {
  int M = 0, N = 0, K = 0;
  int ta = 0, tb = 0;
  int64_t lda = 0, ldb = 0, ldc = 0;
  double ar = 1.0, ai = 0.0;
  int arA = AR_FIX, arB = AR_FIX, arC = AR_FIX;
  int epi = 0;
  int ep[4] = {0, 0, 0, 0};  // na, nb, nc, nd for epi == 1
  int store = 0;
  std::vector<int64_t> coff;       // per batch
  std::vector<int32_t> sbeg;       // per batch + 1
  std::vector<int64_t> aoff, boff; // per segment
  int nbatch() const { return (int)coff.size(); }
  int64_t flops() const;           // real flops (8 per complex MAC)
  std::string tag;
};

// dst[L_dst(e)] += alpha * src[L_src(e o pi)], e over the destination elements;
// source slot s takes destination slot pi[s].  store == 1: dst[L_dst(e)] = alpha * src[...]
// (the destination is not read; set by fold_first_writes).
struct Perm {
  Layout src, dst;
  int pi[4] = {0, 1, 2, 3};
  double ar = 1.0, ai = 0.0;
  int arS = AR_FIX, arD = AR_FIX;
  int64_t offS = 0, offD = 0;
  int store = 0;
  std::string tag;
};

// Batched 2-D transpose: dst[b][j][i] += alpha * src[b][i][j], i < R, j < C.
struct BTrans {
  int nb = 0, R = 0, C = 0;
  double ar = 1.0, ai = 0.0;
  int arS = AR_FIX, arD = AR_FIX;
  int64_t offS = 0, offD = 0;
  std::string tag;
};

enum OpKind : int { OP_GEMM = 0, OP_PERM = 1, OP_BTRANS = 2, OP_ZERO = 3 };

struct Op {
  int kind = OP_GEMM;
  int idx = 0;        // index into the plan's gemms / perms / btrans / zeros
  int fixed_only = 0; // 1: reads/writes only FIX/WS (e.g. a W-block build); not transposed
  int zl = -1;        // index into Plan::zlists: scratch buffers whose last use is this op
                      // (the transposed program zeroes them before this op's transpose)
};

// zero n elements before the next op; the buffer's tensor holds the first `used` of them (the
// rest is alignment padding that no op reads)
struct ZeroSpec { int arena; int64_t off, n, used; };

struct ScrBuf { int64_t off, n, used; };  // used: elements before rounding to the alignment

struct Program {
  std::vector<Op> ops;
};

struct Dims { int nk, o, v, Q; };

struct Plan {
  Dims d{};
  int64_t arena_size[AR_COUNT] = {0, 0, 0, 0, 0};
  std::vector<Gemm> gemms;
  std::vector<Perm> perms;
  std::vector<BTrans> btrans;
  std::vector<ZeroSpec> zeros;
  std::vector<ScrBuf> scr_bufs;     // scratch buffers (logical, before liveness packing)
  std::vector<std::vector<int>> zlists;  // lists of indices into `zeros`
  Program ground;    // fixed-only ops: ground-state intermediates
  Program jac;       // linear in IN -> OUT (uses SCR, WS)
  Program xi;        // perturbation right-hand side xi^X(t', mu): IN = t' (paper units) -> OUT
  Program egrad;     // IN x1 -> OUT y1 += 2 L x1 (energy second derivative, singles)
  Program omega0;    // OUT = Omega(t = 0) (paper units): doubles (ai|bj), singles f_ai = 0 (canonical)
  Program tgrad;     // IN = t (paper units) -> OUT = dE/dt (paper units, plain pairing)
  // named offsets of the FIX inputs
  int64_t off_Loo = 0, off_Lov = 0, off_Lvo = 0, off_Lvv = 0, off_f0 = 0,
          off_t1 = 0, off_t2 = 0, off_idv = 0, off_derived = 0;
  int64_t off_x1 = 0, off_x2 = 0;    // within IN / OUT
  int64_t off_mu = 0;                // FIX: one-body operator blocks oo, ov, vo, vv, ov^T
  int64_t ws_limit = 0;
  double jac_flops = 0.0, ladder_flops = 0.0, wbuild_flops = 0.0;
};

// Build both programs.  ws_budget: complex elements for the W-block workspace.
Plan build_plan(const Dims& d, int64_t ws_budget);

// The plan of an introspection handle (plan_api.cpp), for host-only queries elsewhere.
const Plan* plan_of(const ::lrcc_plan* h);

// Host-side bounds check of every op against the arena sizes (per-vector sizes for
// the vector arenas).  Returns an empty string when every access is in bounds.
std::string validate_plan(const Plan& P, const Program& pr);

// Transposed op list of the Jacobian program (reverse order, transposed ops).
// New GEMM/PERM/BTRANS entries are appended to the plan's tables.
Program transpose_program(Plan& P, const Program& fwd);

// A scratch buffer is zeroed just before its first use.  Where that use is a permutation or a
// GEMM (epi == 0, every batch entry with at least one segment) that writes every element of
// exactly that buffer once and does not read it, the op stores instead of accumulating (a copy
// of it with store = 1) and the zero op is dropped.
void fold_first_writes(Plan& P, Program& pr);

}  // namespace lrcc
