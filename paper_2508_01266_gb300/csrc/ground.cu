// Ground state on the GPU: CCSD amplitudes T (Eqs. 7-8) and Lambda multipliers
// (Eqs. 10-11), built from the same Jacobian products as the response solver.
//
// Residual.  The CCSD residual Omega(t) is a polynomial of degree 4 in t, so
// d/ds Omega(s t) = A(s t) t is a cubic in s and two-point Gauss-Legendre quadrature is
// exact:  Omega(t) = Omega(0) + 1/2 [A(s1 t) t + A(s2 t) t],  s1,2 = (1 -+ 1/sqrt 3) / 2.
// Omega(0) (the omega0 program: (ai|bj) in the doubles, f_ai = 0) is computed once; each
// residual costs two ground-state rebuilds at s1 t, s2 t and two Jacobian products.
//
// CCSD: Jacobi updates t <- t - Omega(t) / D (D from Eq. 9) with DIIS on e = t_new - t
// (Sec. II.D), until max |Omega| <= conv_tol.  In the mixed-precision modes the amplitudes
// are found by inexact Newton steps instead: the FP64 residual Omega(t) above, then the
// correction A(t) d = -Omega(t) solved by the same Jacobi + DIIS iteration with tensor-core
// products (and tensor-core ground-state intermediates) to a loose relative tolerance,
// t <- t + d.  The FP64 residual decides convergence, so the result meets the same
// max |Omega| <= conv_tol; each step costs one FP64 residual instead of one per Jacobi
// iteration.
// Lambda: the stationarity conditions of E + <lam, Omega> are A^T lam = -dE/dt (plain
// pairing, paper units; dE/dt from the tgrad program), solved with the transpose
// products by the batched Jacobi + DIIS solver (mixed precision: its iterative refinement
// with FP64 residuals).  The result is returned in the paper's
// normalization (alpha-beta block of the spin-orbital multipliers):
//   l1 = lam1 / 2,   l2 = Nk^2 (2 lam2 + lam2(a<->b)) / 3.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kernels.cuh"
#include "runtime.h"
#include "solver_core.h"
#include "solver_kernels.cuh"

using namespace lrcc;

namespace {

struct Ground {
  Runtime& rt;
  const Plan& P;
  cudaStream_t st = 0;
  long long vec;
  size_t n1, n2;
  explicit Ground(Runtime& r) : rt(r), P(r.plan), vec(r.plan.arena_size[AR_IN]) {
    const int nk = rt.dims.nk, o = rt.dims.nocc, v = rt.dims.nvir;
    n1 = (size_t)nk * o * v;
    n2 = (size_t)nk * nk * nk * o * o * v * v;
  }

  lrcc_status rebuild(int prec = 0) {
    if (!rt.ck(cudaMemsetAsync(rt.fix + P.off_derived, 0, (P.arena_size[AR_FIX] - P.off_derived) * sizeof(double2),
                               st),
               "memset derived"))
      return LRCC_ECUDA;
    double2* ar[AR_COUNT] = {rt.fix, nullptr, nullptr, nullptr, rt.ws};
    return rt.run(P.ground, ar, 1, st, prec);
  }
  // ground-state amplitudes in FIX <- s * T (T in the vector layout); intermediates built
  // with the GEMM arithmetic prec
  lrcc_status set_t(const double2* T, double s, int prec = 0) {
    if (!rt.ck(launch_axpby(make_double2(s, 0.0), T + P.off_x1, make_double2(0.0, 0.0), rt.fix + P.off_t1,
                            (long long)n1, st),
               "t1 <- s t") ||
        !rt.ck(launch_axpby(make_double2(s, 0.0), T + P.off_x2, make_double2(0.0, 0.0), rt.fix + P.off_t2,
                            (long long)n2, st),
               "t2 <- s t"))
      return LRCC_ECUDA;
    rt.launches += 2;
    return rebuild(prec);
  }
  // OUT <- program(IN) for one vector
  lrcc_status run_prog(const Program& pr) {
    double2* ar[AR_COUNT] = {rt.fix, rt.in, rt.out, rt.scr, rt.ws};
    if (!rt.ck(cudaMemsetAsync(rt.out, 0, vec * sizeof(double2), st), "memset")) return LRCC_ECUDA;
    return rt.run(pr, ar, 1, st, 0);
  }
  // R <- Omega(T) (paper units); leaves the FIX ground state at s2 T
  lrcc_status residual(const double2* T, const double2* O0, double2* R) {
    lrcc_status s;
    if (!rt.ck(cudaMemcpyAsync(R, O0, vec * sizeof(double2), cudaMemcpyDeviceToDevice, st), "R <- Omega(0)"))
      return LRCC_ECUDA;
    const double q = 0.5 / std::sqrt(3.0);
    for (double sc : {0.5 - q, 0.5 + q}) {
      if ((s = set_t(T, sc)) != LRCC_OK) return s;
      if (!rt.ck(cudaMemcpyAsync(rt.in, T, vec * sizeof(double2), cudaMemcpyDeviceToDevice, st), "T -> in"))
        return LRCC_ECUDA;
      if ((s = rt.apply(0, 1, st, 0)) != LRCC_OK) return s;
      if (!rt.ck(launch_axpby(make_double2(0.5, 0.0), rt.out, make_double2(1.0, 0.0), R, vec, st), "R += A t / 2"))
        return LRCC_ECUDA;
      rt.launches++;
    }
    return LRCC_OK;
  }
};

lrcc_status copy_out(Runtime& rt, void* dst, const double2* src, size_t n, int32_t on_device) {
  if (!dst) return LRCC_OK;
  return rt.ck(cudaMemcpy(dst, src, n * sizeof(double2), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost),
               "copy out")
             ? LRCC_OK
             : LRCC_ECUDA;
}

}  // namespace

extern "C" {

lrcc_status lrcc_residual(lrcc_problem* p, const void* t1, const void* t2, void* r1, void* r2) {
  if (!p) return LRCC_EINVAL;
  Runtime& rt = p->rt;
  if (!p->have_int) {
    rt.err = "residual: integrals not set";
    return LRCC_EINVAL;
  }
  if (!t1 || !t2 || !r1 || !r2) {
    rt.err = "residual: null pointer";
    return LRCC_EINVAL;
  }
  lrcc_status s = rt.ensure_rhs(1);
  if (s != LRCC_OK) return s;
  Ground G(rt);
  const Plan& P = rt.plan;
  Dev dev;
  bool ok = true;
  double2* T = dev.get<double2>(rt, G.vec, ok);
  double2* O0 = dev.get<double2>(rt, G.vec, ok);
  double2* R = dev.get<double2>(rt, G.vec, ok);
  double2* keep1 = dev.get<double2>(rt, G.n1, ok);
  double2* keep2 = dev.get<double2>(rt, G.n2, ok);
  if (!ok) return LRCC_ENOMEM;
  if (!rt.ck(cudaMemset(T, 0, G.vec * sizeof(double2)), "memset") ||
      !rt.ck(cudaMemcpy(T + P.off_x1, t1, G.n1 * sizeof(double2), cudaMemcpyDeviceToDevice), "t1") ||
      !rt.ck(cudaMemcpy(T + P.off_x2, t2, G.n2 * sizeof(double2), cudaMemcpyDeviceToDevice), "t2") ||
      !rt.ck(cudaMemcpy(keep1, rt.fix + P.off_t1, G.n1 * sizeof(double2), cudaMemcpyDeviceToDevice), "keep t1") ||
      !rt.ck(cudaMemcpy(keep2, rt.fix + P.off_t2, G.n2 * sizeof(double2), cudaMemcpyDeviceToDevice), "keep t2"))
    return LRCC_ECUDA;
  if ((s = G.run_prog(P.omega0)) != LRCC_OK) return s;
  if (!rt.ck(cudaMemcpy(O0, rt.out, G.vec * sizeof(double2), cudaMemcpyDeviceToDevice), "Omega(0)")) return LRCC_ECUDA;
  if ((s = G.residual(T, O0, R)) != LRCC_OK) return s;
  // restore the problem's ground state
  if (!rt.ck(cudaMemcpy(rt.fix + P.off_t1, keep1, G.n1 * sizeof(double2), cudaMemcpyDeviceToDevice), "t1") ||
      !rt.ck(cudaMemcpy(rt.fix + P.off_t2, keep2, G.n2 * sizeof(double2), cudaMemcpyDeviceToDevice), "t2"))
    return LRCC_ECUDA;
  if ((s = G.rebuild()) != LRCC_OK) return s;
  if (!rt.ck(cudaMemcpy(r1, R + P.off_x1, G.n1 * sizeof(double2), cudaMemcpyDeviceToDevice), "r1") ||
      !rt.ck(cudaMemcpy(r2, R + P.off_x2, G.n2 * sizeof(double2), cudaMemcpyDeviceToDevice), "r2") ||
      !rt.ck(cudaDeviceSynchronize(), "residual sync"))
    return LRCC_ECUDA;
  return LRCC_OK;
}

lrcc_status lrcc_solve_ground_state(lrcc_problem* p, const lrcc_options* optp, void* t1, void* t2, void* l1,
                                    void* l2, int32_t on_device, double* energy, int32_t* info) {
  if (!p) return LRCC_EINVAL;
  Runtime& rt = p->rt;
  if (!p->have_int) {
    rt.err = "solve_ground_state: integrals not set";
    return LRCC_EINVAL;
  }
  lrcc_options opt;
  lrcc_default_options(&opt);
  if (optp) opt = *optp;
  if (opt.precision < 0 || opt.precision > 2) {
    rt.err = "solve_ground_state: precision must be 0, 1 or 2";
    return LRCC_EINVAL;
  }
  const int prec = opt.precision;
  if (info) std::memset(info, 0, 4 * sizeof(int32_t));
  lrcc_status s = rt.ensure_rhs(1);
  if (s != LRCC_OK) return s;
  Ground G(rt);
  const Plan& P = rt.plan;
  const int nk = rt.dims.nk, o = rt.dims.nocc, v = rt.dims.nvir;
  BatchSolver bs(rt, opt, 1, 4);
  if ((s = bs.init()) != LRCC_OK) return s;
  Dev dev;
  bool ok = true;
  double2* T = dev.get<double2>(rt, G.vec, ok);
  double2* O0 = dev.get<double2>(rt, G.vec, ok);
  double2* Z = dev.get<double2>(rt, G.vec, ok);
  double2* GR = dev.get<double2>(rt, G.vec, ok);
  double2* LV = dev.get<double2>(rt, G.vec, ok);
  double2* L1 = dev.get<double2>(rt, G.n1, ok);
  double2* L2 = dev.get<double2>(rt, G.n2, ok);
  double* W0 = dev.get<double>(rt, 1, ok);
  if (!ok) return LRCC_ENOMEM;
#define CK(x, what) \
  do {              \
    if (!rt.ck((x), what)) return LRCC_ECUDA; \
  } while (0)
  CK(cudaMemset(T, 0, G.vec * sizeof(double2)), "memset");
  CK(cudaMemset(Z, 0, G.vec * sizeof(double2)), "memset");
  CK(cudaMemset(W0, 0, sizeof(double)), "memset");
  if ((s = G.run_prog(P.omega0)) != LRCC_OK) return s;
  CK(cudaMemcpy(O0, rt.out, G.vec * sizeof(double2), cudaMemcpyDeviceToDevice), "Omega(0)");

  // CCSD amplitudes ------------------------------------------------------------------
  const int depth = bs.depth;
  if ((s = bs.diis_reset()) != LRCC_OK) return s;
  CK(launch_inv_den(bs.DEN, W0, bs.INV, G.vec, 1, G.st), "1 / D");
  int nhist = 0, it = 0;
  bool conv = false;
  double err = 0.0;
  for (; it < bs.maxit && prec > 0; ++it) {  // inexact Newton (mixed precision)
    if ((s = G.residual(T, O0, bs.RES)) != LRCC_OK) return s;
    std::vector<double> rmax;
    if ((s = bs.maxabs(bs.RES, 1, rmax)) != LRCC_OK) return s;
    err = rmax[0];
    log_iteration(opt, "ccsd_newton", it, {err});
    if (err <= opt.conv_tol) {
      conv = true;
      break;
    }
    // A(t) d = -Omega(t): tensor-core products at tensor-core intermediates of t
    if ((s = G.set_t(T, 1.0, prec)) != LRCC_OK) return s;
    bool iconv = false;
    const double inner_tol = prec == 1 ? 3e-3 : 1e-4;
    if ((s = bs.jacobi_diis(0, bs.RES, rmax, W0, prec, inner_tol, bs.maxit, iconv)) != LRCC_OK) return s;
    CK(launch_axpby(make_double2(1.0, 0.0), rt.in, make_double2(1.0, 0.0), T, G.vec, G.st), "t += d");
    rt.launches++;
  }
  for (; it < bs.maxit && prec == 0; ++it) {
    if ((s = G.residual(T, O0, bs.RES)) != LRCC_OK) return s;
    const int slot = it % depth;
    CK(cudaMemsetAsync(bs.RMAX, 0, sizeof(unsigned long long), G.st), "memset");
    // e = -Omega / D, t_new = t + e  (update kernel with y = 0, w = 0, rhs = Omega)
    CK(launch_update(T, Z, bs.RES, bs.INV, W0, bs.HE + (size_t)slot * G.vec, bs.HX + (size_t)slot * G.vec, bs.RMAX,
                     G.vec, G.vec, 1, G.st),
       "update");
    rt.launches++;
    unsigned long long hr = 0;
    CK(cudaMemcpy(&hr, bs.RMAX, sizeof(hr), cudaMemcpyDeviceToHost), "rmax");
    err = u64_to_double(hr);
    log_iteration(opt, "ccsd", it, {err});
    if (err <= opt.conv_tol) {
      conv = true;
      break;
    }
    if ((s = bs.diis(it, nhist, T)) != LRCC_OK) return s;
  }
  if (info) {
    info[0] = it;
    info[1] = conv ? 0 : LRCC_ENOCONV;
  }
  if (!conv) {
    rt.err = "solve_ground_state: CCSD amplitudes did not converge (max |Omega| " + std::to_string(err) + ")";
    return LRCC_ENOCONV;
  }
  if ((s = G.set_t(T, 1.0)) != LRCC_OK) return s;

  // energy per cell: E_sc = 1/2 <dE/dt1, t1> + <dE/dt2, t2> (E is quadratic in t1, linear in t2)
  CK(cudaMemcpy(rt.in, T, G.vec * sizeof(double2), cudaMemcpyDeviceToDevice), "T -> in");
  if ((s = G.run_prog(P.tgrad)) != LRCC_OK) return s;
  CK(cudaMemcpy(GR, rt.out, G.vec * sizeof(double2), cudaMemcpyDeviceToDevice), "dE/dt");
  std::vector<cd> d1, d2;
  if ((s = bs.dots({GR + P.off_x1}, {T + P.off_x1}, 0, (long long)G.n1, d1)) != LRCC_OK) return s;
  if ((s = bs.dots({GR + P.off_x2}, {T + P.off_x2}, 0, (long long)G.n2, d2)) != LRCC_OK) return s;
  if (energy) *energy = (0.5 * d1[0] + d2[0]).real() / nk;

  // Lambda: A^T lam = -dE/dt ----------------------------------------------------------
  bool lconv = false;
  if ((s = bs.solve(1, GR, W0, LV, lconv)) != LRCC_OK) return s;
  if (info) {
    info[2] = bs.total_it;
    info[3] = lconv ? 0 : LRCC_ENOCONV;
  }
  if (!lconv) {
    rt.err = "solve_ground_state: Lambda equations did not converge";
    return LRCC_ENOCONV;
  }
  // paper normalization: l1 = lam1 / 2 ; l2 = Nk^2 (2 lam2 + lam2(a<->b)) / 3
  CK(launch_axpby(make_double2(0.5, 0.0), LV + P.off_x1, make_double2(0.0, 0.0), L1, (long long)G.n1, G.st), "l1");
  CK(cudaMemsetAsync(L2, 0, G.n2 * sizeof(double2), G.st), "memset");
  {
    PermArgs pa;
    pa.skind = pa.dkind = LK_K3;
    pa.snk = pa.dnk = nk;
    const int dn[4] = {o, o, v, v};
    for (int i = 0; i < 4; ++i) pa.sn[i] = pa.dn[i] = dn[i];
    pa.total = (long long)G.n2;
    pa.S = LV + P.off_x2;
    pa.D = L2;
    pa.sS = pa.sD = 0;
    pa.ai = 0.0;
    const int id[4] = {0, 1, 2, 3}, sw[4] = {0, 1, 3, 2};
    for (int i = 0; i < 4; ++i) pa.pi[i] = id[i];
    pa.ar = 2.0 * nk * nk / 3.0;
    CK(launch_perm_f64(pa, 1, G.st), "l2 a");
    for (int i = 0; i < 4; ++i) pa.pi[i] = sw[i];
    pa.ar = 1.0 * nk * nk / 3.0;
    CK(launch_perm_f64(pa, 1, G.st), "l2 b");
    rt.launches += 3;
  }
  CK(cudaStreamSynchronize(G.st), "ground sync");
  // the problem's ground state is now the solved one
  s = lrcc_set_ground_state(p, T + P.off_x1, T + P.off_x2, L1, L2, 1);
  if (s != LRCC_OK) return s;
  if ((s = copy_out(rt, t1, T + P.off_x1, G.n1, on_device)) != LRCC_OK ||
      (s = copy_out(rt, t2, T + P.off_x2, G.n2, on_device)) != LRCC_OK ||
      (s = copy_out(rt, l1, L1, G.n1, on_device)) != LRCC_OK || (s = copy_out(rt, l2, L2, G.n2, on_device)) != LRCC_OK)
    return s;
#undef CK
  return LRCC_OK;
}

}  // extern "C"
