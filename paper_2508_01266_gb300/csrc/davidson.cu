// Linear-response excitation energies: the poles of the response function (Eq. 15) are
// the eigenvalues of the CCSD Jacobian, found here by a non-Hermitian Davidson iteration
// that needs only batched Jacobian products:
//   subspace V (orthonormal in the Hermitian inner product), H = V^H A V, Ritz pairs
//   (theta, y) of H with the smallest real parts, residuals r = A V y - theta V y,
//   corrections t = -r / (D - theta) (orbital-energy denominators of Eq. 9),
//   orthogonalised against V (two Gram-Schmidt passes) and added; when the subspace is
//   full it collapses onto the current Ritz vectors.
// Guesses: singles unit vectors at the smallest denominators e_a - e_i.  Products run in
// the precision the options select (FP64 by default).  The subspace eigenproblem is
// solved on the host (small_eig.cpp).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "kernels.cuh"
#include "runtime.h"
#include "small_eig.h"
#include "solver_core.h"
#include "solver_kernels.cuh"

using namespace lrcc;

extern "C" lrcc_status lrcc_excitation_energies(lrcc_problem* p, int32_t nroots, const lrcc_options* optp,
                                                void* omegas, void* x1, void* x2, int32_t* info) {
  if (!p) return LRCC_EINVAL;
  Runtime& rt = p->rt;
  if (!p->have_t) {
    rt.err = "excitation_energies: ground state not set";
    return LRCC_EINVAL;
  }
  const int nk = rt.dims.nk, o = rt.dims.nocc, v = rt.dims.nvir, n = o + v;
  const long long n1 = (long long)nk * o * v;
  const long long n2 = (long long)nk * nk * nk * o * o * v * v;
  if (nroots < 1 || nroots > n1 || !omegas) {
    rt.err = "excitation_energies: nroots must be in [1, Nk o v] and omegas non-null";
    return LRCC_EINVAL;
  }
  lrcc_options opt;
  lrcc_default_options(&opt);
  if (optp) opt = *optp;
  const double tol = opt.conv_tol;
  const int prec = std::max(0, std::min(2, opt.precision));
  const int mmax = std::min(std::max(6 * nroots, 24), 120);
  const int nguess = (int)std::min<long long>(n1, nroots + 2);
  const Plan& P = rt.plan;
  lrcc_status s = rt.ensure_rhs(std::max(nguess, nroots));
  if (s != LRCC_OK) return s;
  BatchSolver bs(rt, opt, 1, 2 * mmax + 8);
  if ((s = bs.init()) != LRCC_OK) return s;
  const long long vec = bs.vec;
  const cudaStream_t st = 0;
  Dev dev;
  bool ok = true;
  double2* V = dev.get<double2>(rt, (size_t)mmax * vec, ok);
  double2* AV = dev.get<double2>(rt, (size_t)mmax * vec, ok);
  double2* R = dev.get<double2>(rt, (size_t)(nroots + 2) * vec, ok);  // residuals / collapsed vectors
  double2* TMP = dev.get<double2>(rt, (size_t)(nroots + 2) * vec, ok);
  const double2** PV = dev.get<const double2*>(rt, (size_t)(2 * mmax + 2), ok);
  double2* CO = dev.get<double2>(rt, (size_t)(2 * mmax + 2), ok);
  if (!ok) return LRCC_ENOMEM;
#define CK(x, what) \
  do {              \
    if (!rt.ck((x), what)) return LRCC_ECUDA; \
  } while (0)
  auto Vp = [&](int j) { return V + (size_t)j * vec; };
  auto AVp = [&](int j) { return AV + (size_t)j * vec; };
  // out = sum_j c_j x_j (out must not alias any x_j)
  auto combine = [&](const std::vector<const double2*>& xs, const std::vector<cd>& c, double2* out) -> lrcc_status {
    std::vector<double2> h(c.size());
    for (size_t j = 0; j < c.size(); ++j) h[j] = make_double2(c[j].real(), c[j].imag());
    CK(cudaMemcpy(PV, xs.data(), xs.size() * sizeof(void*), cudaMemcpyHostToDevice), "pv");
    CK(cudaMemcpy(CO, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice), "coef");
    CK(launch_lincomb(PV, CO, (int)xs.size(), out, vec, vec, 1, st), "lincomb");
    rt.launches++;
    return LRCC_OK;
  };
  auto norm = [&](const double2* x, double& nv) -> lrcc_status {
    std::vector<cd> d;
    lrcc_status s2 = bs.dots({x}, {x}, 1, vec, d);
    nv = std::sqrt(std::max(d[0].real(), 0.0));
    return s2;
  };
  // orthogonalise x (in place, via TMP slot) against V[0..m) and normalise; returns the
  // norm left after the projections relative to the norm before
  auto orthonormalize = [&](double2* x, double2* tmp, int m, double& kept) -> lrcc_status {
    lrcc_status s2;
    double n0 = 0.0;
    if ((s2 = norm(x, n0)) != LRCC_OK) return s2;
    for (int pass = 0; pass < 2 && m > 0; ++pass) {
      std::vector<const double2*> a, b;
      for (int j = 0; j < m; ++j) {
        a.push_back(Vp(j));
        b.push_back(x);
      }
      std::vector<cd> c;
      if ((s2 = bs.dots(a, b, 1, vec, c)) != LRCC_OK) return s2;
      std::vector<const double2*> xs{x};
      std::vector<cd> co{1.0};
      for (int j = 0; j < m; ++j) {
        xs.push_back(Vp(j));
        co.push_back(-c[j]);
      }
      if ((s2 = combine(xs, co, tmp)) != LRCC_OK) return s2;
      CK(cudaMemcpy(x, tmp, vec * sizeof(double2), cudaMemcpyDeviceToDevice), "copy");
    }
    double n1v = 0.0;
    if ((s2 = norm(x, n1v)) != LRCC_OK) return s2;
    kept = n0 > 0 ? n1v / n0 : 0.0;
    if (n1v > 0) {
      CK(launch_axpby(make_double2(1.0 / n1v, 0.0), x, make_double2(0.0, 0.0), x, vec, st), "scale");
      rt.launches++;
    }
    return LRCC_OK;
  };

  // guesses: singles unit vectors at the smallest denominators
  {
    std::vector<double> d1(n1);
    for (int k = 0; k < nk; ++k)
      for (int i = 0; i < o; ++i)
        for (int a = 0; a < v; ++a) d1[((size_t)k * o + i) * v + a] = rt.eps[k * n + o + a] - rt.eps[k * n + i];
    std::vector<long long> idx(n1);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](long long x, long long y) { return d1[x] < d1[y]; });
    CK(cudaMemset(V, 0, (size_t)nguess * vec * sizeof(double2)), "memset");
    const double2 one = make_double2(1.0, 0.0);
    for (int j = 0; j < nguess; ++j)
      CK(cudaMemcpy(Vp(j) + P.off_x1 + idx[j], &one, sizeof(double2), cudaMemcpyHostToDevice), "guess");
  }

  int m = 0, knew = nguess, it = 0;
  bool conv = false;
  std::vector<cd> H;  // m x m, row-major, H[i][j] = <V_i, A V_j>
  std::vector<cd> theta(nroots), Y;
  std::vector<double> rnorm(nroots, 1.0);
  for (; it < bs.maxit; ++it) {
    // products of the new basis vectors
    CK(cudaMemcpy(rt.in, Vp(m), (size_t)knew * vec * sizeof(double2), cudaMemcpyDeviceToDevice), "V -> in");
    if ((s = rt.apply(0, knew, st, prec, opt.use_graphs != 0, opt.autotune != 0)) != LRCC_OK) return s;
    CK(cudaMemcpy(AVp(m), rt.out, (size_t)knew * vec * sizeof(double2), cudaMemcpyDeviceToDevice), "out -> AV");
    const int m2 = m + knew;
    std::vector<cd> H2((size_t)m2 * m2, 0.0);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) H2[(size_t)i * m2 + j] = H[(size_t)i * m + j];
    {
      std::vector<const double2*> a, b;
      std::vector<std::pair<int, int>> ij;
      for (int i = 0; i < m2; ++i)
        for (int j = 0; j < m2; ++j)
          if (i >= m || j >= m) {
            a.push_back(Vp(i));
            b.push_back(AVp(j));
            ij.push_back({i, j});
          }
      std::vector<cd> d;
      if ((s = bs.dots(a, b, 1, vec, d)) != LRCC_OK) return s;
      for (size_t q = 0; q < ij.size(); ++q) H2[(size_t)ij[q].first * m2 + ij[q].second] = d[q];
    }
    H.swap(H2);
    m = m2;
    std::vector<cd> w, U;
    if (!small_eig(m, H, w, U)) {
      rt.err = "excitation_energies: subspace eigenproblem failed";
      return LRCC_ENOCONV;
    }
    std::vector<int> ord(m);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return w[x].real() < w[y].real(); });
    const int nk_keep = std::min(m, nroots + 2);
    Y.assign((size_t)nk_keep * m, 0.0);  // Ritz coefficient vectors, one per kept root
    for (int r = 0; r < nk_keep; ++r)
      for (int j = 0; j < m; ++j) Y[(size_t)r * m + j] = U[(size_t)j * m + ord[r]];
    for (int r = 0; r < nroots && r < m; ++r) theta[r] = w[ord[r]];
    // residuals of the wanted roots
    double worst = 0.0;
    for (int r = 0; r < nroots && r < m; ++r) {
      std::vector<const double2*> xs;
      std::vector<cd> co;
      for (int j = 0; j < m; ++j) {
        xs.push_back(AVp(j));
        co.push_back(Y[(size_t)r * m + j]);
        xs.push_back(Vp(j));
        co.push_back(-theta[r] * Y[(size_t)r * m + j]);
      }
      if ((s = combine(xs, co, R + (size_t)r * vec)) != LRCC_OK) return s;
      if ((s = norm(R + (size_t)r * vec, rnorm[r])) != LRCC_OK) return s;
      worst = std::max(worst, rnorm[r]);
    }
    log_iteration(opt, "davidson", it, rnorm);
    if (m >= nroots && worst <= tol) {
      conv = true;
      break;
    }
    // collapse when the new corrections would not fit
    int nnew = 0;
    for (int r = 0; r < nroots; ++r)
      if (rnorm[r] > tol) ++nnew;
    if (m + nnew > mmax) {
      // orthonormal basis of the kept Ritz vectors (Gram-Schmidt on their coefficients:
      // V is orthonormal, so <V y_a, V y_b> = y_a^H y_b), then V <- V Y', AV <- AV Y'
      std::vector<std::vector<cd>> Q;
      for (int r = 0; r < nk_keep; ++r) {
        std::vector<cd> y(Y.begin() + (size_t)r * m, Y.begin() + (size_t)(r + 1) * m);
        for (int pass = 0; pass < 2; ++pass)
          for (const auto& qv : Q) {
            cd c = 0.0;
            for (int j = 0; j < m; ++j) c += std::conj(qv[j]) * y[j];
            for (int j = 0; j < m; ++j) y[j] -= c * qv[j];
          }
        double nr = 0.0;
        for (const cd& x : y) nr += std::norm(x);
        nr = std::sqrt(nr);
        if (nr < 1e-10) continue;
        for (cd& x : y) x /= nr;
        Q.push_back(y);
      }
      const int kq = (int)Q.size();
      for (int half = 0; half < 2; ++half) {
        for (int r = 0; r < kq; ++r) {
          std::vector<const double2*> xs;
          for (int j = 0; j < m; ++j) xs.push_back(half ? AVp(j) : Vp(j));
          if ((s = combine(xs, Q[r], TMP + (size_t)r * vec)) != LRCC_OK) return s;
        }
        CK(cudaMemcpy(half ? AV : V, TMP, (size_t)kq * vec * sizeof(double2), cudaMemcpyDeviceToDevice), "collapse");
      }
      std::vector<cd> Hc((size_t)kq * kq, 0.0);
      std::vector<const double2*> a, b;
      for (int i = 0; i < kq; ++i)
        for (int j = 0; j < kq; ++j) {
          a.push_back(Vp(i));
          b.push_back(AVp(j));
        }
      if ((s = bs.dots(a, b, 1, vec, Hc)) != LRCC_OK) return s;
      H.swap(Hc);
      m = kq;
    }
    // corrections for the unconverged roots
    knew = 0;
    for (int r = 0; r < nroots && m + knew < mmax; ++r) {
      if (rnorm[r] <= tol) continue;
      double2* t = Vp(m + knew);
      CK(launch_precond(R + (size_t)r * vec, bs.DEN, make_double2(theta[r].real(), theta[r].imag()), TMP, vec, st),
         "precond");
      rt.launches++;
      // keep the search space pair-symmetric: t2 <- (t2 + S t2) / 2.  The Jacobian
      // symmetrises its input, so rounding residue in the antisymmetric part would
      // otherwise surface as spurious zero eigenvalues.
      CK(cudaMemcpyAsync(t, TMP, vec * sizeof(double2), cudaMemcpyDeviceToDevice, st), "copy");
      CK(cudaMemsetAsync(t + P.off_x2, 0, n2 * sizeof(double2), st), "memset");
      for (int sw = 0; sw < 2; ++sw) {
        PermArgs pa;
        pa.skind = pa.dkind = LK_K3;
        pa.snk = pa.dnk = nk;
        const int dn[4] = {o, o, v, v};
        for (int i = 0; i < 4; ++i) pa.sn[i] = pa.dn[i] = dn[i];
        const int id[4] = {0, 1, 2, 3}, swp[4] = {1, 0, 3, 2};
        for (int i = 0; i < 4; ++i) pa.pi[i] = sw ? swp[i] : id[i];
        pa.total = (long long)n2;
        pa.S = TMP + P.off_x2;
        pa.D = t + P.off_x2;
        pa.sS = pa.sD = 0;
        pa.ar = 0.5;
        pa.ai = 0.0;
        CK(launch_perm_f64(pa, 1, st), "symmetrise");
        rt.launches++;
      }
      double kept = 0.0;
      if ((s = orthonormalize(t, TMP, m + knew, kept)) != LRCC_OK) return s;
      if (kept > 1e-6) ++knew;
    }
    if (knew == 0) {
      rt.err = "excitation_energies: no new search directions (stagnation)";
      break;
    }
  }
  if (info) {
    info[0] = it;
    info[1] = conv ? 0 : LRCC_ENOCONV;
  }
  cd* om = (cd*)omegas;
  for (int r = 0; r < nroots; ++r) om[r] = theta[r];
  // right eigenvectors (paper units), unit Hermitian norm
  if ((x1 || x2) && conv) {
    const size_t b1 = (size_t)n1 * sizeof(double2);
    const size_t b2 = (size_t)n2 * sizeof(double2);
    for (int r = 0; r < nroots; ++r) {
      std::vector<const double2*> xs;
      std::vector<cd> co;
      for (int j = 0; j < m; ++j) {
        xs.push_back(Vp(j));
        co.push_back(Y[(size_t)r * m + j]);
      }
      if ((s = combine(xs, co, TMP)) != LRCC_OK) return s;
      double nv = 1.0;
      if ((s = norm(TMP, nv)) != LRCC_OK) return s;
      CK(launch_axpby(make_double2(1.0 / nv, 0.0), TMP, make_double2(0.0, 0.0), TMP, vec, st), "scale");
      if (x1) CK(cudaMemcpy((char*)x1 + r * b1, TMP + P.off_x1, b1, cudaMemcpyDeviceToDevice), "x1");
      if (x2) CK(cudaMemcpy((char*)x2 + r * b2, TMP + P.off_x2, b2, cudaMemcpyDeviceToDevice), "x2");
    }
  }
  CK(cudaDeviceSynchronize(), "davidson sync");
#undef CK
  if (!conv) {
    if (rt.err.empty()) rt.err = "excitation_energies: Davidson did not converge";
    return LRCC_ENOCONV;
  }
  return LRCC_OK;
}
