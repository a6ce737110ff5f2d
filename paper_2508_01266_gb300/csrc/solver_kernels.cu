// FP64 vector kernels of the response solver.  All are HBM-bound passes over the
// batched vectors (vector arena layout, RHS-major): the denominator update of the
// perturbed-amplitude equations (Eqs. 13-14, D -+ w), DIIS error inner products and
// extrapolation (Sec. II.D), and the dot products of the response function (Eq. 15).
// Reductions use a fixed partition and a fixed-order second pass, so results are
// bitwise reproducible.
#include "solver_kernels.cuh"

namespace lrcc {

static unsigned grid_for(long long n, int per_block) {
  long long b = (n + per_block - 1) / per_block;
  if (b > 152LL * 16) b = 152LL * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// res = -xi - y + w x ; e = res / (den - w) ; xnew = x + e ; rmax[r] = max |res|
__global__ void update_kernel(const double2* x, const double2* y, const double2* xi, const double* den,
                              const double* omega, double2* e, double2* xnew, unsigned long long* rmax, long long n,
                              long long stride) {
  const long long r = blockIdx.y;
  const double w = omega[r];
  const double2* X = x + r * stride;
  const double2* Y = y + r * stride;
  const double2* XI = xi + r * stride;
  double2* E = e + r * stride;
  double2* XN = xnew + r * stride;
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 xv = X[i], yv = Y[i], s = XI[i];
    const double rr = -s.x - yv.x + w * xv.x;
    const double ri = -s.y - yv.y + w * xv.y;
    const double d = den[i] - w;
    const double2 ev = make_double2(rr / d, ri / d);
    E[i] = ev;
    XN[i] = make_double2(xv.x + ev.x, xv.y + ev.y);
    m = fmax(m, sqrt(rr * rr + ri * ri));
  }
  __shared__ double sm[256];
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(rmax + r, (unsigned long long)__double_as_longlong(sm[0]));
}

cudaError_t launch_update(const double2* x, const double2* y, const double2* xi, const double* den,
                          const double* omega, double2* e, double2* xnew, unsigned long long* rmax, long long n,
                          long long stride, int nrhs, cudaStream_t st) {
  dim3 grid(grid_for(n, 256 * 4), nrhs);
  update_kernel<<<grid, 256, 0, st>>>(x, y, xi, den, omega, e, xnew, rmax, n, stride);
  return cudaGetLastError();
}

// R = xi + y - w x (the negated residual of (A - w) x = -xi); rmax[r] = max |R|
__global__ void residual_kernel(const double2* x, const double2* y, const double2* xi, const double* omega,
                                double2* R, unsigned long long* rmax, long long n, long long stride) {
  const long long r = blockIdx.y;
  const double w = omega[r];
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long q = r * stride + i;
    const double2 xv = x[q], yv = y[q], s = xi[q];
    const double rr = s.x + yv.x - w * xv.x, ri = s.y + yv.y - w * xv.y;
    R[q] = make_double2(rr, ri);
    m = fmax(m, sqrt(rr * rr + ri * ri));
  }
  __shared__ double sm[256];
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(rmax + r, (unsigned long long)__double_as_longlong(sm[0]));
}

cudaError_t launch_residual(const double2* x, const double2* y, const double2* xi, const double* omega, double2* R,
                            unsigned long long* rmax, long long n, long long stride, int nrhs, cudaStream_t st) {
  dim3 grid(grid_for(n, 256 * 4), nrhs);
  residual_kernel<<<grid, 256, 0, st>>>(x, y, xi, omega, R, rmax, n, stride);
  return cudaGetLastError();
}

// x0 = -xi / (den - w)
__global__ void guess_kernel(const double2* xi, const double* den, const double* omega, double2* x, long long n,
                             long long stride) {
  const long long r = blockIdx.y;
  const double w = omega[r];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 s = xi[r * stride + i];
    const double d = den[i] - w;
    x[r * stride + i] = make_double2(-s.x / d, -s.y / d);
  }
}

cudaError_t launch_guess(const double2* xi, const double* den, const double* omega, double2* x, long long n,
                         long long stride, int nrhs, cudaStream_t st) {
  dim3 grid(grid_for(n, 256 * 4), nrhs);
  guess_kernel<<<grid, 256, 0, st>>>(xi, den, omega, x, n, stride);
  return cudaGetLastError();
}

// maxabs over each of nrhs vectors
__global__ void maxabs_kernel(const double2* x, unsigned long long* out, long long n, long long stride) {
  const long long r = blockIdx.y;
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[r * stride + i];
    m = fmax(m, sqrt(v.x * v.x + v.y * v.y));
  }
  __shared__ double sm[256];
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out + r, (unsigned long long)__double_as_longlong(sm[0]));
}

cudaError_t launch_maxabs(const double2* x, unsigned long long* out, long long n, long long stride, int nrhs,
                          cudaStream_t st) {
  dim3 grid(grid_for(n, 256 * 4), nrhs);
  maxabs_kernel<<<grid, 256, 0, st>>>(x, out, n, stride);
  return cudaGetLastError();
}

// batched dot products: out[p] = sum_i op(a_p[i]) b_p[i], op = conj or identity.
// pass 1: fixed partition into DOT_BLOCKS chunks per pair.
constexpr int DOT_BLOCKS = 256;
__global__ void dot_pass1(const double2* const* a, const double2* const* b, int conj, long long n, double2* part) {
  const int p = blockIdx.y;
  const double2* A = a[p];
  const double2* Bv = b[p];
  const long long chunk = (n + DOT_BLOCKS - 1) / DOT_BLOCKS;
  const long long i0 = (long long)blockIdx.x * chunk;
  const long long i1 = (i0 + chunk < n) ? i0 + chunk : n;
  double sr = 0.0, si = 0.0;
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const double2 x = A[i], y = Bv[i];
    const double xi = conj ? -x.y : x.y;
    sr = fma(x.x, y.x, sr);
    sr = fma(-xi, y.y, sr);
    si = fma(x.x, y.y, si);
    si = fma(xi, y.x, si);
  }
  __shared__ double rr[256], ri[256];
  rr[threadIdx.x] = sr;
  ri[threadIdx.x] = si;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      rr[threadIdx.x] += rr[threadIdx.x + s];
      ri[threadIdx.x] += ri[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long long)p * DOT_BLOCKS + blockIdx.x] = make_double2(rr[0], ri[0]);
}

__global__ void dot_pass2(const double2* part, double2* out, int npairs) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  double sr = 0.0, si = 0.0;
  for (int j = 0; j < DOT_BLOCKS; ++j) {
    sr += part[(long long)p * DOT_BLOCKS + j].x;
    si += part[(long long)p * DOT_BLOCKS + j].y;
  }
  out[p] = make_double2(sr, si);
}

size_t dot_partial_elems(int npairs) { return (size_t)npairs * DOT_BLOCKS; }

cudaError_t launch_dots(const double2* const* a, const double2* const* b, int conj, long long n, int npairs,
                        double2* part, double2* out, cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  dim3 grid(DOT_BLOCKS, npairs);
  dot_pass1<<<grid, 256, 0, st>>>(a, b, conj, n, part);
  dot_pass2<<<(npairs + 127) / 128, 128, 0, st>>>(part, out, npairs);
  return cudaGetLastError();
}

// out[r] = sum_j c[j*nrhs + r] * v_j[r]   (v_j given as base pointers with RHS stride)
__global__ void lincomb_kernel(const double2* const* v, const double2* c, int m, double2* out, long long n,
                               long long stride, int nrhs) {
  const long long r = blockIdx.y;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double sr = 0.0, si = 0.0;
    for (int j = 0; j < m; ++j) {
      const double2 cc = c[(long long)j * nrhs + r];
      const double2 x = v[j][r * stride + i];
      sr += cc.x * x.x - cc.y * x.y;
      si += cc.x * x.y + cc.y * x.x;
    }
    out[r * stride + i] = make_double2(sr, si);
  }
}

cudaError_t launch_lincomb(const double2* const* v, const double2* c, int m, double2* out, long long n,
                           long long stride, int nrhs, cudaStream_t st) {
  dim3 grid(grid_for(n, 256 * 4), nrhs);
  lincomb_kernel<<<grid, 256, 0, st>>>(v, c, m, out, n, stride, nrhs);
  return cudaGetLastError();
}

// y = a * x + b * y  (complex a, b), one vector
__global__ void axpby_kernel(double2 a, const double2* x, double2 b, double2* y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 xv = x[i], yv = y[i];
    y[i] = make_double2(a.x * xv.x - a.y * xv.y + b.x * yv.x - b.y * yv.y,
                        a.x * xv.y + a.y * xv.x + b.x * yv.y + b.y * yv.x);
  }
}

cudaError_t launch_axpby(double2 a, const double2* x, double2 b, double2* y, long long n, cudaStream_t st) {
  axpby_kernel<<<grid_for(n, 256 * 4), 256, 0, st>>>(a, x, b, y, n);
  return cudaGetLastError();
}

// Davidson correction: out = -r / (den - theta), theta complex (one vector)
__global__ void precond_kernel(const double2* r, const double* den, double2 theta, double2* out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double dr = den[i] - theta.x, di = -theta.y;
    double q = dr * dr + di * di;
    if (q < 1e-24) q = 1e-24;  // the shift sits on a denominator: keep the correction finite
    const double2 v = r[i];
    // -(v / (dr + i di)) = -(v (dr - i di)) / q
    out[i] = make_double2(-(v.x * dr + v.y * di) / q, -(v.y * dr - v.x * di) / q);
  }
}

cudaError_t launch_precond(const double2* r, const double* den, double2 theta, double2* out, long long n,
                           cudaStream_t st) {
  precond_kernel<<<grid_for(n, 256 * 4), 256, 0, st>>>(r, den, theta, out, n);
  return cudaGetLastError();
}

}  // namespace lrcc
