// Eigenvalues and right eigenvectors of a small dense complex matrix (the Davidson
// subspace matrix): Householder reduction to upper Hessenberg form, single-shift complex
// QR iterations with Wilkinson shifts and deflation (complex Schur form T = Q^H A Q), then
// eigenvectors of T by back substitution, mapped back with Q.  Textbook algorithms
// (Golub & Van Loan, Matrix Computations, Ch. 7), written for n up to a few hundred.
#include "small_eig.h"

#include <algorithm>
#include <cmath>

namespace lrcc {

using cd = std::complex<double>;

bool small_eig(int n, const std::vector<cd>& Ain, std::vector<cd>& w, std::vector<cd>& V) {
  if (n <= 0 || (int)Ain.size() != n * n) return false;
  std::vector<cd> A = Ain, Q(n * n, 0.0);
  auto a = [&](int i, int j) -> cd& { return A[i * n + j]; };
  auto q = [&](int i, int j) -> cd& { return Q[i * n + j]; };
  for (int i = 0; i < n; ++i) q(i, i) = 1.0;
  double anorm = 0.0;
  for (const cd& x : A) anorm = std::max(anorm, std::abs(x));
  if (!std::isfinite(anorm)) return false;
  if (anorm == 0.0) anorm = 1.0;

  // 1. Hessenberg reduction: A <- H A H, Q <- Q H for Householder H = I - 2 u u^H
  for (int k = 0; k + 2 < n; ++k) {
    double xnorm = 0.0;
    for (int i = k + 1; i < n; ++i) xnorm += std::norm(a(i, k));
    xnorm = std::sqrt(xnorm);
    if (xnorm == 0.0) continue;
    std::vector<cd> u(n, 0.0);
    const cd x0 = a(k + 1, k);
    const cd ph = std::abs(x0) > 0 ? x0 / std::abs(x0) : cd(1.0);
    for (int i = k + 1; i < n; ++i) u[i] = a(i, k);
    u[k + 1] += ph * xnorm;
    double un = 0.0;
    for (int i = k + 1; i < n; ++i) un += std::norm(u[i]);
    un = std::sqrt(un);
    if (un == 0.0) continue;
    for (int i = k + 1; i < n; ++i) u[i] /= un;
    for (int j = 0; j < n; ++j) {  // A <- (I - 2uu^H) A
      cd s = 0.0;
      for (int i = k + 1; i < n; ++i) s += std::conj(u[i]) * a(i, j);
      for (int i = k + 1; i < n; ++i) a(i, j) -= 2.0 * u[i] * s;
    }
    for (int i = 0; i < n; ++i) {  // A <- A (I - 2uu^H), Q <- Q (I - 2uu^H)
      cd s = 0.0, t = 0.0;
      for (int j = k + 1; j < n; ++j) {
        s += a(i, j) * u[j];
        t += q(i, j) * u[j];
      }
      for (int j = k + 1; j < n; ++j) {
        a(i, j) -= 2.0 * s * std::conj(u[j]);
        q(i, j) -= 2.0 * t * std::conj(u[j]);
      }
    }
    for (int i = k + 2; i < n; ++i) a(i, k) = 0.0;
  }

  // 2. shifted QR on the active block [lo, hi]
  const double eps = 1e-15;
  int hi = n - 1, iter = 0, total = 0;
  while (hi > 0) {
    if (++total > 100 * n) return false;
    int l = hi;
    for (; l > 0; --l) {
      const double s = std::abs(a(l - 1, l - 1)) + std::abs(a(l, l));
      if (std::abs(a(l, l - 1)) <= eps * (s > 0 ? s : anorm)) {
        a(l, l - 1) = 0.0;
        break;
      }
    }
    if (l == hi) {
      --hi;
      iter = 0;
      continue;
    }
    // Wilkinson shift: eigenvalue of the trailing 2 x 2 block closer to its last entry
    const cd p = a(hi - 1, hi - 1), b = a(hi - 1, hi), c = a(hi, hi - 1), d = a(hi, hi);
    const cd tr2 = 0.5 * (p + d), disc = std::sqrt(tr2 * tr2 - (p * d - b * c));
    const cd m1 = tr2 + disc, m2 = tr2 - disc;
    cd mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
    if (iter > 0 && iter % 10 == 0) mu = d + std::abs(c);  // exceptional shift
    ++iter;
    // QR step of (A - mu I) on rows/columns l..hi by Givens rotations, A <- R Q + mu I
    std::vector<cd> cs(hi - l), sn(hi - l);
    for (int k = l; k <= hi; ++k) a(k, k) -= mu;
    for (int k = l; k < hi; ++k) {
      const cd x = a(k, k), y = a(k + 1, k);
      const double r = std::sqrt(std::norm(x) + std::norm(y));
      cd cc = 1.0, ss = 0.0;
      if (r > 0) {
        cc = x / r;
        ss = y / r;
      }
      cs[k - l] = cc;
      sn[k - l] = ss;
      // rows k, k+1 <- G^H [row k; row k+1] with G = [[cc, -conj(ss)], [ss, conj(cc)]]
      for (int j = k; j < n; ++j) {
        const cd u0 = a(k, j), u1 = a(k + 1, j);
        a(k, j) = std::conj(cc) * u0 + std::conj(ss) * u1;
        a(k + 1, j) = -ss * u0 + cc * u1;
      }
    }
    for (int k = l; k < hi; ++k) {  // columns k, k+1 <- [col k, col k+1] G
      const cd cc = cs[k - l], ss = sn[k - l];
      for (int i = 0; i <= std::min(hi, k + 1); ++i) {
        const cd u0 = a(i, k), u1 = a(i, k + 1);
        a(i, k) = u0 * cc + u1 * ss;
        a(i, k + 1) = -u0 * std::conj(ss) + u1 * std::conj(cc);
      }
      for (int i = 0; i < n; ++i) {
        const cd u0 = q(i, k), u1 = q(i, k + 1);
        q(i, k) = u0 * cc + u1 * ss;
        q(i, k + 1) = -u0 * std::conj(ss) + u1 * std::conj(cc);
      }
    }
    for (int k = l; k <= hi; ++k) a(k, k) += mu;
  }

  // 3. eigenvalues and eigenvectors of the triangular T, mapped back with Q
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) w[i] = a(i, i);
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    std::vector<cd> x(n, 0.0);
    x[i] = 1.0;
    for (int j = i - 1; j >= 0; --j) {
      cd s = 0.0;
      for (int k = j + 1; k <= i; ++k) s += a(j, k) * x[k];
      cd den = a(j, j) - w[i];
      if (std::abs(den) < eps * anorm) den = eps * anorm;
      x[j] = -s / den;
    }
    double nrm = 0.0;
    std::vector<cd> v(n, 0.0);
    for (int r = 0; r < n; ++r) {
      for (int k = 0; k <= i; ++k) v[r] += q(r, k) * x[k];
      nrm += std::norm(v[r]);
    }
    nrm = std::sqrt(nrm);
    for (int r = 0; r < n; ++r) V[r * n + i] = nrm > 0 ? v[r] / nrm : v[r];
  }
  for (const cd& x : w)
    if (!std::isfinite(x.real()) || !std::isfinite(x.imag())) return false;
  return true;
}

}  // namespace lrcc

extern "C" lrcc_status lrcc_small_eig(int32_t n, const void* a, void* w, void* v) {
  if (n <= 0 || !a || !w) return LRCC_EINVAL;
  const lrcc::cd* A = (const lrcc::cd*)a;
  std::vector<lrcc::cd> M(A, A + (size_t)n * n), ww, VV;
  if (!lrcc::small_eig(n, M, ww, VV)) return LRCC_ENOCONV;
  std::copy(ww.begin(), ww.end(), (lrcc::cd*)w);
  if (v) std::copy(VV.begin(), VV.end(), (lrcc::cd*)v);
  return LRCC_OK;
}
