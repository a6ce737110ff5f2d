// Batched linear-solver machinery shared by the polarizability driver (solver.cu) and the
// ground-state solver (ground.cu): orbital-energy denominators, batched dot products,
// DIIS extrapolation (Hermitian B matrix, Sec. II.D), Jacobi + DIIS solves of
// (A - w) x = -rhs or (A^T - w) x = -rhs for a batch of systems, and mixed-precision
// iterative refinement around them.
#pragma once
#include <complex>
#include <vector>

#include "runtime.h"

namespace lrcc {

using cd = std::complex<double>;

// device allocations released together
struct Dev {
  std::vector<void*> ptrs, hptrs;
  ~Dev() {
    for (void* p : ptrs) cudaFree(p);
    for (void* p : hptrs) cudaFreeHost(p);
  }
  // pinned host memory mapped into the device address space; returns the device pointer
  void* host(Runtime& rt, size_t bytes, bool& ok) {
    void* h = nullptr;
    void* d = nullptr;
    if (!ok) return nullptr;
    if (!rt.ck(cudaHostAlloc(&h, std::max<size_t>(bytes, 1), cudaHostAllocMapped), "cudaHostAlloc(history)")) {
      ok = false;
      return nullptr;
    }
    hptrs.push_back(h);
    if (!rt.ck(cudaHostGetDevicePointer(&d, h, 0), "cudaHostGetDevicePointer")) {
      ok = false;
      return nullptr;
    }
    return d;
  }
  template <class T>
  T* get(Runtime& rt, size_t n, bool& ok) {
    void* p = nullptr;
    if (!ok) return nullptr;
    if (!rt.ck(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)), "cudaMalloc(solver)")) {
      ok = false;
      return nullptr;
    }
    ptrs.push_back(p);
    return (T*)p;
  }
};

struct BatchSolver {
  Runtime& rt;
  lrcc_options opt;
  int ns = 1, depth = 8, maxit = 200, maxpairs = 16;
  long long vec = 0;
  cudaStream_t st = 0;
  Dev dev;
  double2 *HX = nullptr, *HE = nullptr, *RES = nullptr, *PART = nullptr, *DOT = nullptr, *COEF = nullptr;
  double2* BDEV = nullptr;  // per-system DIIS B matrices [ns][depth][depth]
  double* DEN = nullptr;
  double* INV = nullptr;  // 1 / (DEN - w) per system of the current solve
  unsigned long long* RMAX = nullptr;
  const double2 **PA = nullptr, **PB = nullptr, **PV = nullptr;
  int total_it = 0;
  bool host_history = false;
  std::vector<double> rel;

  BatchSolver(Runtime& r, const lrcc_options& o, int nsys, int min_pairs);
  // allocations and the denominators e_a - e_i (+ e_b - e_j) of Eq. 9
  lrcc_status init();
  // out[p] = sum_i op(a_p[i]) b_p[i], op = conj when conj != 0
  lrcc_status dots(const std::vector<const double2*>& a, const std::vector<const double2*>& b, int conj,
                   long long len, std::vector<cd>& out);
  lrcc_status maxabs(const double2* x, int nrhs, std::vector<double>& out);
  // DIIS with error vectors HE[slot] and iterates HX[slot] (written by the update kernel):
  // updates the per-system B matrices (device memory) and writes the extrapolated iterates
  // into X, all on the device
  lrcc_status diis(int it, int& nhist, double2* X);
  // zero the B matrices before a new iteration
  lrcc_status diis_reset();
  lrcc_status jacobi_diis(int tr, const double2* rhs, const std::vector<double>& rhsmax, const double* om, int prec,
                          double tol, int maxiter, bool& conv);
  lrcc_status solve(int tr, const double2* rhs, const double* om, double2* sol, bool& converged);
};

double u64_to_double(unsigned long long u);

// One JSON line per solver iteration into opt.log_path (no-op when it is NULL):
// {"solver": name, "iter": it, "residual": [per system]}.
void log_iteration(const lrcc_options& opt, const char* solver, int it, const std::vector<double>& res);

}  // namespace lrcc
