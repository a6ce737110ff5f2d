// Small dense complex eigensolver (host) used by the Davidson iteration.
#pragma once
#include <complex>
#include <vector>

#include "../../include/lrcc.h"

namespace lrcc {

// Eigenvalues w[n] and unit right eigenvectors (columns of the row-major V[n*n]) of the
// row-major n x n matrix A.  Returns false if the QR iteration does not converge or the
// input is not finite.
bool small_eig(int n, const std::vector<std::complex<double>>& A, std::vector<std::complex<double>>& w,
               std::vector<std::complex<double>>& V);

}  // namespace lrcc
