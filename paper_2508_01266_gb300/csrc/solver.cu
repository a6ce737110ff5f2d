// Polarizability driver: perturbed-amplitude solves and the linear-response function.
//
//  1. Right-hand sides xi^X = dOmega/d eps_X (Eq. 12) from the xi program.
//  2. All (component, +-w) systems (A - w) t^X(w) = -xi^X (Eqs. 13-14) solved together
//     as one batch: every iteration is one batched Jacobian product, the denominator
//     update t += r / (D - w) (D = e_a - e_i, Eq. 9 with the opposite sign), and DIIS
//     extrapolation with error vectors e = t^n - t^(n-1) and a Hermitian B matrix
//     (Sec. II.D).  Convergence: max|r| / max|xi| <= conv_tol for every system.
//  3. Symmetric linear-response function (Eq. 15 in the form of Christiansen, Jorgensen
//     and Hattig):
//       <<X;Y>>_w = 1/2 C^{+-w} [eta^X t^Y(w) + eta^Y t^X(-w) + F(t^X(-w), t^Y(w))],
//     with eta^X . w = d/ds [E^X + <lam, xi^X>](t + s w) and
//     F . u = d/ds [grad E + A^T lam](t + s u).  Both are exact 4-point stencils (the
//     functions are polynomials of degree <= 3 in s), evaluated with the xi program
//     and with transposed Jacobian products at rebuilt ground-state intermediates.
//     alpha_XY(w) = -<<X;Y>>_w / Nk (per cell).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <complex>
#include <cstring>
#include <vector>

#include "kernels.cuh"
#include "runtime.h"
#include "solver_core.h"
#include "solver_kernels.cuh"

using namespace lrcc;
using cd = std::complex<double>;


namespace lrcc {

double u64_to_double(unsigned long long u) {
  double d;
  std::memcpy(&d, &u, sizeof(d));
  return d;
}

void log_iteration(const lrcc_options& opt, const char* solver, int it, const std::vector<double>& res) {
  if (!opt.log_path) return;
  FILE* f = std::fopen(opt.log_path, "a");
  if (!f) return;
  std::fprintf(f, "{\"solver\": \"%s\", \"iter\": %d, \"residual\": [", solver, it);
  for (size_t i = 0; i < res.size(); ++i) std::fprintf(f, "%s%.6e", i ? ", " : "", res[i]);
  std::fprintf(f, "]}\n");
  std::fclose(f);
}

BatchSolver::BatchSolver(Runtime& r, const lrcc_options& o, int nsys, int min_pairs) : rt(r), opt(o), ns(nsys) {
  depth = std::max(1, std::min(opt.diis_depth, 16));
  maxit = std::max(1, opt.max_iter);
  maxpairs = std::max(min_pairs, depth * ns) + 8;
  vec = rt.plan.arena_size[AR_IN];
  rel.assign(ns, 1.0);
}

lrcc_status BatchSolver::init() {
  bool ok = true;
  const size_t hist = (size_t)depth * ns * vec * sizeof(double2);
  bool host = opt.host_history > 0;
  if (opt.host_history == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) host = 2 * hist > fr / 2;
  }
  if (host) {
    // pinned host memory mapped into the device address space: the update, dot and
    // combination kernels read and write the history over the coherent CPU-GPU link
    HX = (double2*)dev.host(rt, hist, ok);
    HE = (double2*)dev.host(rt, hist, ok);
  } else {
    HX = dev.get<double2>(rt, (size_t)depth * ns * vec, ok);
    HE = dev.get<double2>(rt, (size_t)depth * ns * vec, ok);
  }
  host_history = host;
  RES = dev.get<double2>(rt, (size_t)ns * vec, ok);
  DEN = dev.get<double>(rt, (size_t)vec, ok);
  INV = dev.get<double>(rt, (size_t)ns * vec, ok);
  RMAX = dev.get<unsigned long long>(rt, (size_t)ns, ok);
  PA = dev.get<const double2*>(rt, (size_t)maxpairs, ok);
  PB = dev.get<const double2*>(rt, (size_t)maxpairs, ok);
  PART = dev.get<double2>(rt, dot_partial_elems(maxpairs), ok);
  DOT = dev.get<double2>(rt, (size_t)maxpairs, ok);
  COEF = dev.get<double2>(rt, (size_t)depth * ns, ok);
  BDEV = dev.get<double2>(rt, (size_t)ns * depth * depth, ok);
  PV = dev.get<const double2*>(rt, (size_t)depth, ok);
  if (!ok) return LRCC_ENOMEM;
  const Plan& P = rt.plan;
  const int nk = rt.dims.nk, o = rt.dims.nocc, v = rt.dims.nvir, n = o + v;
  std::vector<double> den(vec, 1.0);
  const std::vector<double>& e = rt.eps;
  for (int k = 0; k < nk; ++k)
    for (int i = 0; i < o; ++i)
      for (int a = 0; a < v; ++a) den[P.off_x1 + ((size_t)k * o + i) * v + a] = e[k * n + o + a] - e[k * n + i];
  size_t q = P.off_x2;
  for (int ki = 0; ki < nk; ++ki)
    for (int kj = 0; kj < nk; ++kj)
      for (int ka = 0; ka < nk; ++ka) {
        const int kb = ((ki + kj - ka) % nk + nk) % nk;
        for (int i = 0; i < o; ++i)
          for (int j = 0; j < o; ++j)
            for (int a = 0; a < v; ++a)
              for (int b = 0; b < v; ++b)
                den[q++] = e[ka * n + o + a] + e[kb * n + o + b] - e[ki * n + i] - e[kj * n + j];
      }
  if (!rt.ck(cudaMemcpy(DEN, den.data(), vec * sizeof(double), cudaMemcpyHostToDevice), "den")) return LRCC_ECUDA;
  return LRCC_OK;
}

lrcc_status BatchSolver::dots(const std::vector<const double2*>& a, const std::vector<const double2*>& b, int conj,
                              long long len, std::vector<cd>& out) {
  const int np = (int)a.size();
  out.assign(np, 0.0);
  for (int c0 = 0; c0 < np; c0 += maxpairs) {
    const int m = std::min(maxpairs, np - c0);
    if (!rt.ck(cudaMemcpy(PA, a.data() + c0, m * sizeof(void*), cudaMemcpyHostToDevice), "dots") ||
        !rt.ck(cudaMemcpy(PB, b.data() + c0, m * sizeof(void*), cudaMemcpyHostToDevice), "dots") ||
        !rt.ck(launch_dots(PA, PB, conj, len, m, PART, DOT, st), "dots kernel"))
      return LRCC_ECUDA;
    rt.launches += 2;
    std::vector<double2> h(m);
    if (!rt.ck(cudaMemcpy(h.data(), DOT, m * sizeof(double2), cudaMemcpyDeviceToHost), "dots")) return LRCC_ECUDA;
    for (int i = 0; i < m; ++i) out[c0 + i] = cd(h[i].x, h[i].y);
  }
  return LRCC_OK;
}

lrcc_status BatchSolver::maxabs(const double2* x, int nrhs, std::vector<double>& out) {
  if (!rt.ck(cudaMemsetAsync(RMAX, 0, nrhs * sizeof(unsigned long long), st), "memset") ||
      !rt.ck(launch_maxabs(x, RMAX, vec, vec, nrhs, st), "maxabs"))
    return LRCC_ECUDA;
  rt.launches++;
  std::vector<unsigned long long> h(nrhs);
  if (!rt.ck(cudaMemcpy(h.data(), RMAX, nrhs * sizeof(unsigned long long), cudaMemcpyDeviceToHost), "maxabs"))
    return LRCC_ECUDA;
  out.resize(nrhs);
  for (int i = 0; i < nrhs; ++i) out[i] = u64_to_double(h[i]);
  return LRCC_OK;
}

// DIIS step on the device: B entries of the newest error vectors, the per-system bordered
// solve and the extrapolated iterates into X (solver_kernels.cu); no host round trip.
lrcc_status BatchSolver::diis(int it, int& nhist, double2* X) {
  nhist = std::min(nhist + 1, depth);
  const int extrapolate = (nhist >= 2 && (opt.diis_period <= 1 || (it + 1) % opt.diis_period == 0)) ? 1 : 0;
  if (!rt.ck(launch_diis_device(HE, HX, BDEV, it, depth, ns, nhist, extrapolate, vec, PART, COEF, X, st), "diis"))
    return LRCC_ECUDA;
  rt.launches += 3;
  return LRCC_OK;
}

lrcc_status BatchSolver::diis_reset() {
  return rt.ck(cudaMemsetAsync(BDEV, 0, (size_t)ns * depth * depth * sizeof(double2), st), "diis reset") ? LRCC_OK
                                                                                                         : LRCC_ECUDA;
}

// Jacobi + DIIS on (A - w) x = -rhs (tr = 0, iterate in rt.in) or (A^T - w) x = -rhs
// (tr = 1, transposed products, iterate in rt.out) for every system; prec selects the
// GEMM arithmetic of the products.  rel receives the relative residual reached.
lrcc_status BatchSolver::jacobi_diis(int tr, const double2* rhs, const std::vector<double>& rhsmax, const double* om,
                                     int prec, double tol, int maxiter, bool& conv) {
  lrcc_status s2;
  double2* X = tr ? rt.out : rt.in;
  double2* Y = tr ? rt.in : rt.out;
  if (!rt.ck(launch_inv_den(DEN, om, INV, vec, ns, st), "1 / (D - w)") ||
      !rt.ck(launch_guess(rhs, INV, X, vec, vec, ns, st), "guess"))
    return LRCC_ECUDA;
  rt.launches++;
  rt.launches++;
  if ((s2 = diis_reset()) != LRCC_OK) return s2;
  int nhist = 0;
  conv = false;
  for (int it = 0; it < maxiter; ++it) {
    ++total_it;
    if ((s2 = rt.apply(tr, ns, st, prec, opt.use_graphs != 0, opt.autotune != 0)) != LRCC_OK) return s2;
    const int slot = it % depth;
    if (!rt.ck(cudaMemsetAsync(RMAX, 0, ns * sizeof(unsigned long long), st), "memset") ||
        !rt.ck(launch_update(X, Y, rhs, INV, om, HE + (size_t)slot * ns * vec, HX + (size_t)slot * ns * vec, RMAX,
                             vec, vec, ns, st),
               "update"))
      return LRCC_ECUDA;
    rt.launches++;
    std::vector<unsigned long long> hr(ns);
    if (!rt.ck(cudaMemcpy(hr.data(), RMAX, ns * sizeof(unsigned long long), cudaMemcpyDeviceToHost), "rmax"))
      return LRCC_ECUDA;
    double worst = 0.0;
    for (int i = 0; i < ns; ++i) {
      rel[i] = u64_to_double(hr[i]) / std::max(rhsmax[i], 1e-300);
      worst = std::max(worst, rel[i]);
    }
    log_iteration(opt, tr ? (prec ? "jacobi_diis_transpose_mixed" : "jacobi_diis_transpose")
                          : (prec ? "jacobi_diis_mixed" : "jacobi_diis"),
                  it, rel);
    if (worst <= tol) {
      conv = true;
      return LRCC_OK;
    }
    if ((s2 = diis(it, nhist, X)) != LRCC_OK) return s2;
  }
  return LRCC_OK;
}

// Solve every system into sol: FP64 Jacobi + DIIS, or (mixed precision) iterative
// refinement: FP64 residual r = -rhs - (A - w) x, tensor-core inner solve of
// (A - w) d = r to a loose tolerance, x += d, until max|r| / max|rhs| <= refine_tol.
lrcc_status BatchSolver::solve(int tr, const double2* rhs, const double* om, double2* sol, bool& converged) {
  lrcc_status s2;
  const int prec = opt.precision;
  double2* X = tr ? rt.out : rt.in;
  double2* Y = tr ? rt.in : rt.out;
  std::vector<double> rhsmax;
  if ((s2 = maxabs(rhs, ns, rhsmax)) != LRCC_OK) return s2;
  converged = false;
  if (prec == 0) {
    if ((s2 = jacobi_diis(tr, rhs, rhsmax, om, 0, opt.conv_tol, maxit, converged)) != LRCC_OK) return s2;
    if (!rt.ck(cudaMemcpy(sol, X, (size_t)ns * vec * sizeof(double2), cudaMemcpyDeviceToDevice), "sol"))
      return LRCC_ECUDA;
    return LRCC_OK;
  }
  // refinement starts from x = 0, whose residual is the right-hand side itself: the first
  // inner solve needs no FP64 product (the inner solver makes its own Jacobi guess)
  if (!rt.ck(cudaMemsetAsync(sol, 0, (size_t)ns * vec * sizeof(double2), st), "sol = 0")) return LRCC_ECUDA;
  const double tol64 = std::min(opt.refine_tol, 1e-3);
  const double inner_tol = prec == 1 ? 3e-3 : 1e-4;
  for (int outer = 0; outer < 40 && !converged; ++outer) {
    std::vector<double> rmx(ns);
    double worst = 0.0;
    if (outer == 0) {
      if (!rt.ck(cudaMemcpyAsync(RES, rhs, (size_t)ns * vec * sizeof(double2), cudaMemcpyDeviceToDevice, st),
                 "R = rhs"))
        return LRCC_ECUDA;
      for (int i = 0; i < ns; ++i) {
        rmx[i] = rhsmax[i];
        rel[i] = rhsmax[i] > 0 ? 1.0 : 0.0;
        worst = std::max(worst, rel[i]);
      }
    } else {
      if (!rt.ck(cudaMemcpy(X, sol, (size_t)ns * vec * sizeof(double2), cudaMemcpyDeviceToDevice), "x -> in"))
        return LRCC_ECUDA;
      if ((s2 = rt.apply(tr, ns, st, 0, opt.use_graphs != 0, opt.autotune != 0)) != LRCC_OK) return s2;
      ++total_it;
      // R = rhs + A x - w x = -r ; its max is the FP64 residual
      if (!rt.ck(cudaMemsetAsync(RMAX, 0, ns * sizeof(unsigned long long), st), "memset") ||
          !rt.ck(launch_residual(X, Y, rhs, om, RES, RMAX, vec, vec, ns, st), "residual"))
        return LRCC_ECUDA;
      rt.launches++;
      std::vector<unsigned long long> hr(ns);
      if (!rt.ck(cudaMemcpy(hr.data(), RMAX, ns * sizeof(unsigned long long), cudaMemcpyDeviceToHost), "rmax"))
        return LRCC_ECUDA;
      for (int i = 0; i < ns; ++i) {
        rmx[i] = u64_to_double(hr[i]);
        rel[i] = rmx[i] / std::max(rhsmax[i], 1e-300);
        worst = std::max(worst, rel[i]);
      }
    }
    log_iteration(opt, tr ? "refinement_transpose" : "refinement", outer, rel);
    if (worst <= tol64) {
      converged = true;
      break;
    }
    bool inner_conv = false;
    if ((s2 = jacobi_diis(tr, RES, rmx, om, prec, inner_tol, maxit, inner_conv)) != LRCC_OK) return s2;
    for (int i = 0; i < ns; ++i) {
      if (!rt.ck(launch_axpby(make_double2(1.0, 0.0), X + (size_t)i * vec, make_double2(1.0, 0.0),
                              sol + (size_t)i * vec, vec, st),
                 "x += d"))
        return LRCC_ECUDA;
      rt.launches++;
    }
  }
  return LRCC_OK;
}

}  // namespace lrcc

lrcc_status lrcc_polarize_impl(Runtime& rt, bool have_t, bool have_l, const int32_t* comps, int32_t ncomp,
                               const double* omegas, int32_t nomega, const lrcc_options* optp, void* alpha_out,
                               int32_t* info, const double2* ops, void* alpha_sym_out) {
  if (!have_t) {
    rt.err = "polarizability: ground state not set";
    return LRCC_EINVAL;
  }
  if (!have_l || !rt.l1 || !rt.l2) {
    rt.err = "polarizability: Lambda multipliers not set";
    return LRCC_EINVAL;
  }
  if ((!ops && (!comps || ncomp > 3)) || ncomp < 1 || ncomp > 16 || !omegas || nomega < 1 || !alpha_out) {
    rt.err = "polarizability: bad arguments";
    return LRCC_EINVAL;
  }
  lrcc_options opt;
  lrcc_default_options(&opt);
  if (optp) opt = *optp;
  if (opt.precision < 0 || opt.precision > 2) {
    rt.err = "polarizability: precision must be 0, 1 or 2";
    return LRCC_EINVAL;
  }
  if (opt.response_form < 0 || opt.response_form > 2) {
    rt.err = "polarizability: response_form must be 0, 1 or 2";
    return LRCC_EINVAL;
  }
  const int form = opt.response_form;
  if (!ops)
    for (int c = 0; c < ncomp; ++c)
      if (comps[c] < 0 || comps[c] > 2) {
        rt.err = "polarizability: component index out of range";
        return LRCC_EINVAL;
      }
  for (int w = 0; w < nomega; ++w)
    if (!std::isfinite(omegas[w])) {
      rt.err = "polarizability: non-finite frequency";
      return LRCC_EINVAL;
    }
  const int nk = rt.dims.nk, o = rt.dims.nocc, v = rt.dims.nvir, n = o + v;
  const Plan& P = rt.plan;
  const long long vec = P.arena_size[AR_IN];
  const cudaStream_t st = 0;
  // the one-body operator of each component: a dipole component, or the caller's matrices
  std::vector<const double2*> opm(ncomp);
  for (int c = 0; c < ncomp; ++c)
    opm[c] = ops ? ops + (size_t)c * nk * n * n : rt.dip_host.data() + (size_t)comps[c] * nk * n * n;

  // components whose integrals vanish are skipped (Sec. II.C)
  std::vector<int> active(ncomp, 1);
  for (int c = 0; c < ncomp; ++c) {
    double m = 0.0;
    const double2* d = opm[c];
    for (size_t i = 0; i < (size_t)nk * n * n; ++i) m = std::max(m, std::hypot(d[i].x, d[i].y));
    if (m < 1e-14) active[c] = 0;
  }
  struct Sys { int c; double w; };
  std::vector<Sys> sys;
  std::vector<std::vector<int>> sidx(ncomp, std::vector<int>(2 * nomega, -1));  // [c][2*iw + (0:+w, 1:-w)]
  for (int c = 0; c < ncomp; ++c) {
    if (!active[c]) continue;
    for (int iw = 0; iw < nomega; ++iw) {
      sidx[c][2 * iw] = (int)sys.size();
      sys.push_back({c, omegas[iw]});
      if (omegas[iw] != 0.0) {
        sidx[c][2 * iw + 1] = (int)sys.size();
        sys.push_back({c, -omegas[iw]});
      } else {
        sidx[c][2 * iw + 1] = sidx[c][2 * iw];
      }
    }
  }
  cd* alpha = (cd*)alpha_out;
  for (int i = 0; i < nomega * ncomp * ncomp; ++i) alpha[i] = 0.0;
  if (info) {
    info[0] = 0;
    info[1] = 0;
    for (int c = 0; c < ncomp; ++c) info[2 + c] = active[c] ? 0 : 1;
  }
  const int ns = (int)sys.size();
  if (ns == 0) return LRCC_OK;

  rt.max_batch = std::max(0, opt.max_batch);
  lrcc_status s = rt.ensure_rhs(ns);
  if (s != LRCC_OK) return s;
  BatchSolver bs(rt, opt, ns, ns * std::max(ns, ncomp));
  if ((s = bs.init()) != LRCC_OK) return s;
  Dev dev;
  bool ok = true;
  double2* XI = dev.get<double2>(rt, (size_t)ns * vec, ok);
  double2* SOL = dev.get<double2>(rt, (size_t)ns * vec, ok);
  double2* FU = dev.get<double2>(rt, (size_t)ns * vec, ok);
  double2* TV = dev.get<double2>(rt, (size_t)vec, ok);
  double2* LAM = dev.get<double2>(rt, (size_t)vec, ok);
  double* OM = dev.get<double>(rt, (size_t)ns, ok);
  // left-response form: eta vectors, left right-hand sides and solutions, shifts -w
  double2* ETA = form ? dev.get<double2>(rt, (size_t)ncomp * vec, ok) : nullptr;
  double2* RHSL = form ? dev.get<double2>(rt, (size_t)ns * vec, ok) : nullptr;
  double2* TBAR = form ? dev.get<double2>(rt, (size_t)ns * vec, ok) : nullptr;
  double* OMN = form ? dev.get<double>(rt, (size_t)ns, ok) : nullptr;
  if (!ok) return LRCC_ENOMEM;
#define CK(x, what) \
  do {              \
    if (!rt.ck((x), what)) return LRCC_ECUDA; \
  } while (0)

  // host helpers ------------------------------------------------------------
  auto dots = [&](const std::vector<const double2*>& a, const std::vector<const double2*>& b, int conj, long long len,
                  std::vector<cd>& out) { return bs.dots(a, b, conj, len, out); };
  auto run_prog = [&](const Program& pr, int nrhs) -> lrcc_status {
    if (!rt.ck(cudaMemsetAsync(rt.out, 0, (size_t)vec * nrhs * sizeof(double2), st), "memset")) return LRCC_ECUDA;
    return rt.run_chunked(pr, nrhs, st, 0);
  };
  auto set_mu = [&](int c) -> lrcc_status {
    const double2* d = opm[c];
    std::vector<double2> blk;
    blk.reserve((size_t)nk * (o * o + 3 * o * v + v * v));
    auto el = [&](int k, int p, int q) { return d[((size_t)k * n + p) * n + q]; };
    for (int k = 0; k < nk; ++k)
      for (int p = 0; p < o; ++p)
        for (int q = 0; q < o; ++q) blk.push_back(el(k, p, q));
    for (int k = 0; k < nk; ++k)
      for (int p = 0; p < o; ++p)
        for (int q = 0; q < v; ++q) blk.push_back(el(k, p, o + q));
    for (int k = 0; k < nk; ++k)
      for (int p = 0; p < v; ++p)
        for (int q = 0; q < o; ++q) blk.push_back(el(k, o + p, q));
    for (int k = 0; k < nk; ++k)
      for (int p = 0; p < v; ++p)
        for (int q = 0; q < v; ++q) blk.push_back(el(k, o + p, o + q));
    for (int k = 0; k < nk; ++k)
      for (int q = 0; q < v; ++q)
        for (int p = 0; p < o; ++p) blk.push_back(el(k, p, o + q));
    CK(cudaMemcpy(rt.fix + P.off_mu, blk.data(), blk.size() * sizeof(double2), cudaMemcpyHostToDevice), "mu");
    return LRCC_OK;
  };
  auto rebuild_ground = [&](int gprec) -> lrcc_status {
    CK(cudaMemsetAsync(rt.fix + P.off_derived, 0, (P.arena_size[AR_FIX] - P.off_derived) * sizeof(double2), st),
       "memset derived");
    double2* ar[AR_COUNT] = {rt.fix, nullptr, nullptr, nullptr, rt.ws};
    return rt.run(P.ground, ar, 1, st, gprec);
  };
  auto maxabs = [&](const double2* x, int nrhs, std::vector<double>& out) { return bs.maxabs(x, nrhs, out); };

  // frequencies, t vector, Lambda in the plain pairing of the paper-unit residual ----
  {
    std::vector<double> om(ns);
    for (int i = 0; i < ns; ++i) om[i] = sys[i].w;
    CK(cudaMemcpy(OM, om.data(), ns * sizeof(double), cudaMemcpyHostToDevice), "omega");
  }
  const size_t n1 = (size_t)nk * o * v, n2 = (size_t)nk * nk * nk * o * o * v * v;
  CK(cudaMemset(TV, 0, vec * sizeof(double2)), "memset");
  CK(cudaMemcpy(TV + P.off_x1, rt.fix + P.off_t1, n1 * sizeof(double2), cudaMemcpyDeviceToDevice), "t1");
  CK(cudaMemcpy(TV + P.off_x2, rt.fix + P.off_t2, n2 * sizeof(double2), cudaMemcpyDeviceToDevice), "t2");
  {
    // lam1 = 2 l1 ; lam2 = (2 l2 - l2(a<->b)) / Nk^2   (paper's spin-orbital Lambda -> plain pairing)
    CK(cudaMemset(LAM, 0, vec * sizeof(double2)), "memset");
    CK(launch_axpby(make_double2(2.0, 0.0), rt.l1, make_double2(0.0, 0.0), LAM + P.off_x1, (long long)n1, st), "lam1");
    PermArgs pa;
    pa.skind = pa.dkind = LK_K3;
    pa.snk = pa.dnk = nk;
    const int dn[4] = {o, o, v, v};
    for (int i = 0; i < 4; ++i) pa.sn[i] = pa.dn[i] = dn[i];
    pa.total = (long long)n2;
    pa.S = rt.l2;
    pa.D = LAM + P.off_x2;
    pa.sS = pa.sD = 0;
    pa.ai = 0.0;
    const int id[4] = {0, 1, 2, 3}, sw[4] = {0, 1, 3, 2};
    for (int i = 0; i < 4; ++i) pa.pi[i] = id[i];
    pa.ar = 2.0 / ((double)nk * nk);
    CK(launch_perm_f64(pa, 1, st), "lam2 a");
    for (int i = 0; i < 4; ++i) pa.pi[i] = sw[i];
    pa.ar = -1.0 / ((double)nk * nk);
    CK(launch_perm_f64(pa, 1, st), "lam2 b");
    rt.launches += 3;
  }

  // 1. right-hand sides -------------------------------------------------------------
  for (int c = 0; c < ncomp; ++c) {
    if (!active[c]) continue;
    if ((s = set_mu(c)) != LRCC_OK) return s;
    CK(cudaMemcpy(rt.in, TV, vec * sizeof(double2), cudaMemcpyDeviceToDevice), "t -> in");
    if ((s = run_prog(P.xi, 1)) != LRCC_OK) return s;
    for (int i = 0; i < ns; ++i)
      if (sys[i].c == c)
        CK(cudaMemcpy(XI + (size_t)i * vec, rt.out, vec * sizeof(double2), cudaMemcpyDeviceToDevice), "xi");
  }
  // 2. batched solves (BatchSolver: FP64 Jacobi + DIIS, or mixed-precision refinement) ----
  auto solve = [&](int tr, const double2* rhs, const double* om, double2* sol, bool& conv) {
    return bs.solve(tr, rhs, om, sol, conv);
  };
  bool converged = false;
  if ((s = solve(0, XI, OM, SOL, converged)) != LRCC_OK) return s;
  if (info) {
    info[0] = bs.total_it;
    info[1] = converged ? 0 : LRCC_ENOCONV;
  }
  if (!converged) {
    rt.err = "polarizability: response equations did not converge";
    return LRCC_ENOCONV;
  }
  std::vector<double> umax;
  if ((s = maxabs(SOL, ns, umax)) != LRCC_OK) return s;
  std::vector<double> hstep(ns);
  for (int i = 0; i < ns; ++i) hstep[i] = (opt.precision ? 1e-1 : 1e-2) / std::max(umax[i], 1e-300);
  const double c4[4] = {-2.0, -1.0, 1.0, 2.0}, w4[4] = {1.0, -8.0, 8.0, -1.0};

  // 3a. eta^X . t_sys for every active component and every solution -----------------
  std::vector<std::vector<cd>> etaw(ncomp, std::vector<cd>(ns, 0.0));
  for (int c = 0; c < ncomp; ++c) {
    if (!active[c]) continue;
    if ((s = set_mu(c)) != LRCC_OK) return s;
    for (int k = 0; k < 4; ++k) {
      for (int i = 0; i < ns; ++i) {
        CK(cudaMemcpy(rt.in + (size_t)i * vec, TV, vec * sizeof(double2), cudaMemcpyDeviceToDevice), "t");
        CK(launch_axpby(make_double2(c4[k] * hstep[i], 0.0), SOL + (size_t)i * vec, make_double2(1.0, 0.0),
                        rt.in + (size_t)i * vec, vec, st),
           "t + s u");
        rt.launches++;
      }
      if ((s = run_prog(P.xi, ns)) != LRCC_OK) return s;
      std::vector<const double2*> pa(ns, LAM), pb(ns);
      for (int i = 0; i < ns; ++i) pb[i] = rt.out + (size_t)i * vec;
      std::vector<cd> g;
      if ((s = dots(pa, pb, 0, vec, g)) != LRCC_OK) return s;
      for (int i = 0; i < ns; ++i) etaw[c][i] += w4[k] * g[i] / (12.0 * hstep[i]);
    }
    // + dE^X/dt . w = 2 sum mu_ia w_ia
    std::vector<const double2*> pa(ns, rt.fix + P.off_mu + (size_t)nk * o * o), pb(ns);
    for (int i = 0; i < ns; ++i) pb[i] = SOL + (size_t)i * vec + P.off_x1;
    std::vector<cd> g;
    if ((s = dots(pa, pb, 0, (long long)n1, g)) != LRCC_OK) return s;
    for (int i = 0; i < ns; ++i) etaw[c][i] += 2.0 * g[i];
  }

  // 3b. F . u for every solution u ---------------------------------------------------
  CK(cudaMemset(FU, 0, (size_t)ns * vec * sizeof(double2)), "memset");
  for (int i = 0; i < ns; ++i) {
    const double2* u = SOL + (size_t)i * vec;
    for (int k = 0; k < 4; ++k) {
      const double sh = c4[k] * hstep[i];
      CK(cudaMemcpy(rt.fix + P.off_t1, TV + P.off_x1, n1 * sizeof(double2), cudaMemcpyDeviceToDevice), "t1");
      CK(cudaMemcpy(rt.fix + P.off_t2, TV + P.off_x2, n2 * sizeof(double2), cudaMemcpyDeviceToDevice), "t2");
      CK(launch_axpby(make_double2(sh, 0.0), u + P.off_x1, make_double2(1.0, 0.0), rt.fix + P.off_t1, (long long)n1,
                      st),
         "t1 + s u1");
      CK(launch_axpby(make_double2(sh, 0.0), u + P.off_x2, make_double2(1.0, 0.0), rt.fix + P.off_t2, (long long)n2,
                      st),
         "t2 + s u2");
      rt.launches += 2;
      // the F stencil divides product differences by the step: the mixed modes take these
      // products in BF16x3 (about 1e-5 relative), which keeps alpha within 1e-6 of FP64
      const int fprec = opt.precision ? 2 : 0;
      if ((s = rebuild_ground(fprec)) != LRCC_OK) return s;
      CK(cudaMemcpy(rt.out, LAM, vec * sizeof(double2), cudaMemcpyDeviceToDevice), "lam -> out");
      if ((s = rt.apply(1, 1, st, fprec)) != LRCC_OK) return s;
      CK(launch_axpby(make_double2(w4[k] / (12.0 * hstep[i]), 0.0), rt.in, make_double2(1.0, 0.0),
                      FU + (size_t)i * vec, vec, st),
         "F u");
      rt.launches++;
    }
    CK(cudaMemcpy(rt.in, u, vec * sizeof(double2), cudaMemcpyDeviceToDevice), "u -> in");
    if ((s = run_prog(P.egrad, 1)) != LRCC_OK) return s;
    CK(launch_axpby(make_double2(1.0, 0.0), rt.out, make_double2(1.0, 0.0), FU + (size_t)i * vec, vec, st), "egrad");
    rt.launches++;
  }
  // restore the ground-state intermediates (FP64)
  CK(cudaMemcpy(rt.fix + P.off_t1, TV + P.off_x1, n1 * sizeof(double2), cudaMemcpyDeviceToDevice), "t1");
  CK(cudaMemcpy(rt.fix + P.off_t2, TV + P.off_x2, n2 * sizeof(double2), cudaMemcpyDeviceToDevice), "t2");
  if ((s = rebuild_ground(0)) != LRCC_OK) return s;
  std::vector<const double2*> pa, pb;
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b < ns; ++b) {
      pa.push_back(FU + (size_t)a * vec);
      pb.push_back(SOL + (size_t)b * vec);
    }
  std::vector<cd> F;
  if ((s = dots(pa, pb, 0, vec, F)) != LRCC_OK) return s;
  CK(cudaDeviceSynchronize(), "solver sync");

  // 3c. response function ------------------------------------------------------------------
  if (form == 0 || alpha_sym_out) {
    cd* alpha_sym = form == 0 ? alpha : (cd*)alpha_sym_out;
    for (int iw = 0; iw < nomega; ++iw)
      for (int x = 0; x < ncomp; ++x)
        for (int y = 0; y < ncomp; ++y) {
          if (!active[x] || !active[y]) continue;
          const int xp = sidx[x][2 * iw], xm = sidx[x][2 * iw + 1];
          const int yp = sidx[y][2 * iw], ym = sidx[y][2 * iw + 1];
          const cd a = etaw[x][yp] + etaw[y][xm] + F[(size_t)xm * ns + yp];
          const cd b = etaw[x][ym] + etaw[y][xp] + F[(size_t)xp * ns + ym];
          const cd lr = 0.5 * (a + std::conj(b));
          alpha_sym[((size_t)iw * ncomp + x) * ncomp + y] = -lr / (double)nk;
        }
    if (form == 0) return LRCC_OK;
  }

  // 4. asymmetric (left-response) form -------------------------------------------------------
  // 4a. eta^X as vectors: the Jacobian is linear in the one-body operator, so
  //     (A^X)^T lam = [A(f + mu)^T lam - A(f - mu)^T lam] / 2 exactly; plus dE^X/dt = 2 mu_ia.
  {
    std::vector<double2> f0h((size_t)nk * n * n);
    CK(cudaMemcpy(f0h.data(), rt.fix + P.off_f0, f0h.size() * sizeof(double2), cudaMemcpyDeviceToHost), "f0");
    std::vector<double2> fm(f0h.size());
    for (int c = 0; c < ncomp; ++c) {
      if (!active[c]) continue;
      const double2* mu = opm[c];
      double2* E = ETA + (size_t)c * vec;
      for (int sg = 1; sg >= -1; sg -= 2) {
        for (size_t i = 0; i < fm.size(); ++i)
          fm[i] = make_double2(f0h[i].x + sg * mu[i].x, f0h[i].y + sg * mu[i].y);
        CK(cudaMemcpy(rt.fix + P.off_f0, fm.data(), fm.size() * sizeof(double2), cudaMemcpyHostToDevice), "f0 +- mu");
        if ((s = rebuild_ground(0)) != LRCC_OK) return s;
        CK(cudaMemcpy(rt.out, LAM, vec * sizeof(double2), cudaMemcpyDeviceToDevice), "lam -> out");
        if ((s = rt.apply(1, 1, st, 0)) != LRCC_OK) return s;
        if (sg > 0) {
          CK(cudaMemcpy(E, rt.in, vec * sizeof(double2), cudaMemcpyDeviceToDevice), "eta +");
        } else {
          CK(launch_axpby(make_double2(-0.5, 0.0), rt.in, make_double2(0.5, 0.0), E, vec, st), "eta -");
          rt.launches++;
        }
      }
      if ((s = set_mu(c)) != LRCC_OK) return s;
      CK(launch_axpby(make_double2(2.0, 0.0), rt.fix + P.off_mu + (size_t)nk * o * o, make_double2(1.0, 0.0),
                      E + P.off_x1, (long long)n1, st),
         "eta 2 mu");
      rt.launches++;
    }
    CK(cudaMemcpy(rt.fix + P.off_f0, f0h.data(), f0h.size() * sizeof(double2), cudaMemcpyHostToDevice), "f0");
    if ((s = rebuild_ground(0)) != LRCC_OK) return s;
  }
  // 4b. left perturbed multipliers: (A^T + w_s) tbar_s = -(eta^X + F t^X(w_s)) for every system
  {
    std::vector<double> omn(ns);
    for (int i = 0; i < ns; ++i) omn[i] = -sys[i].w;
    CK(cudaMemcpy(OMN, omn.data(), ns * sizeof(double), cudaMemcpyHostToDevice), "-omega");
    for (int i = 0; i < ns; ++i) {
      CK(cudaMemcpy(RHSL + (size_t)i * vec, ETA + (size_t)sys[i].c * vec, vec * sizeof(double2),
                    cudaMemcpyDeviceToDevice),
         "eta -> rhs");
      CK(launch_axpby(make_double2(1.0, 0.0), FU + (size_t)i * vec, make_double2(1.0, 0.0), RHSL + (size_t)i * vec,
                      vec, st),
         "rhs += F t");
      rt.launches++;
    }
    bool lconv = false;
    if ((s = solve(1, RHSL, OMN, TBAR, lconv)) != LRCC_OK) return s;
    if (info) {
      info[0] = bs.total_it;
      info[1] = lconv ? 0 : LRCC_ENOCONV;
    }
    if (!lconv) {
      rt.err = "polarizability: left response equations did not converge";
      return LRCC_ENOCONV;
    }
  }
  // 4c. <<X;Y>>_w = 1/2 C^{+-w} [eta^Y t^X(-w) + tbar^X(-w) xi^Y]
  {
    std::vector<int> xi_of(ncomp, -1);
    for (int c = 0; c < ncomp; ++c)
      if (active[c]) xi_of[c] = sidx[c][0];
    std::vector<const double2*> qa, qb;
    for (int i = 0; i < ns; ++i)
      for (int c = 0; c < ncomp; ++c) {
        qa.push_back(TBAR + (size_t)i * vec);
        qb.push_back(XI + (size_t)std::max(xi_of[c], 0) * vec);
      }
    std::vector<cd> TX;
    if ((s = dots(qa, qb, 0, vec, TX)) != LRCC_OK) return s;
    std::vector<cd> asym((size_t)nomega * ncomp * ncomp, 0.0);
    for (int iw = 0; iw < nomega; ++iw)
      for (int x = 0; x < ncomp; ++x)
        for (int y = 0; y < ncomp; ++y) {
          if (!active[x] || !active[y]) continue;
          const int xp = sidx[x][2 * iw], xm = sidx[x][2 * iw + 1];
          const cd a = etaw[y][xm] + TX[(size_t)xm * ncomp + y];
          const cd b = etaw[y][xp] + TX[(size_t)xp * ncomp + y];
          asym[((size_t)iw * ncomp + x) * ncomp + y] = -0.5 * (a + std::conj(b)) / (double)nk;
        }
    for (int iw = 0; iw < nomega; ++iw)
      for (int x = 0; x < ncomp; ++x)
        for (int y = 0; y < ncomp; ++y) {
          const size_t i = ((size_t)iw * ncomp + x) * ncomp + y, j = ((size_t)iw * ncomp + y) * ncomp + x;
          alpha[i] = form == 1 ? 0.5 * (asym[i] + asym[j]) : asym[i];
        }
  }
#undef CK
  return LRCC_OK;
}
