// Launchers of the FP64 solver vector kernels (solver_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace lrcc {

// inv[r][i] = 1 / (den[i] - omega[r]) for nrhs systems (inv: nrhs x n doubles)
cudaError_t launch_inv_den(const double* den, const double* omega, double* inv, long long n, int nrhs,
                           cudaStream_t st);
// inv as from launch_inv_den (per-system stride n)
cudaError_t launch_update(const double2* x, const double2* y, const double2* xi, const double* inv,
                          const double* omega, double2* e, double2* xnew, unsigned long long* rmax, long long n,
                          long long stride, int nrhs, cudaStream_t st);
cudaError_t launch_residual(const double2* x, const double2* y, const double2* xi, const double* omega, double2* r,
                            unsigned long long* rmax, long long n, long long stride, int nrhs, cudaStream_t st);
cudaError_t launch_guess(const double2* xi, const double* inv, double2* x, long long n, long long stride, int nrhs,
                         cudaStream_t st);
cudaError_t launch_maxabs(const double2* x, unsigned long long* out, long long n, long long stride, int nrhs,
                          cudaStream_t st);
size_t dot_partial_elems(int npairs);
cudaError_t launch_dots(const double2* const* a, const double2* const* b, int conj, long long n, int npairs,
                        double2* part, double2* out, cudaStream_t st);
cudaError_t launch_lincomb(const double2* const* v, const double2* c, int m, double2* out, long long n,
                           long long stride, int nrhs, cudaStream_t st);
// DIIS on the device: B entries of the newest error vector (history ring of `depth` slots of
// ns vectors of n elements), per-system bordered solve, extrapolated iterates into out (RHS
// stride n).  B: ns x depth x depth complex, zeroed before the first iteration; part:
// dot_partial_elems(depth * ns); coef: depth * ns.  depth <= 16.  Three launches.
cudaError_t launch_diis_device(const double2* HE, const double2* HX, double2* B, int it, int depth, int ns, int nhist,
                               int extrapolate, long long n, double2* part, double2* coef, double2* out,
                               cudaStream_t st);
cudaError_t launch_axpby(double2 a, const double2* x, double2 b, double2* y, long long n, cudaStream_t st);
cudaError_t launch_precond(const double2* r, const double* den, double2 theta, double2* out, long long n,
                           cudaStream_t st);

}  // namespace lrcc
