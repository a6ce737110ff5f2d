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

// Every elementwise pass below takes EU elements per thread per grid-stride step and issues
// all their loads before any result is stored: these passes are bound by HBM latency x
// bandwidth, and one 16-byte load in flight per thread leaves the memory system idle.
constexpr int EU = 4;

// GB300 retires about two FP64 operations per clock per SM, so a division and a square root
// per element would make these passes FP64-pipe bound instead of HBM bound: the solvers keep
// 1 / (den - w) per system (inv_den_kernel, once per solve) and the maxima are taken over
// |res|^2 with one square root per block.

// inv[r][i] = 1 / (den[i] - w_r)
__global__ void inv_den_kernel(const double* __restrict__ den, const double* __restrict__ omega,
                               double* __restrict__ inv, long long n) {
  const long long r = blockIdx.y;
  const double w = omega[r];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    inv[r * n + i] = 1.0 / (den[i] - w);
}

cudaError_t launch_inv_den(const double* den, const double* omega, double* inv, long long n, int nrhs,
                           cudaStream_t st) {
  dim3 grid(grid_for(n, 256 * 4), nrhs);
  inv_den_kernel<<<grid, 256, 0, st>>>(den, omega, inv, n);
  return cudaGetLastError();
}

// res = -xi - y + w x ; e = res * inv ; xnew = x + e ; rmax[r] = max |res|
__global__ void update_kernel(const double2* __restrict__ x, const double2* __restrict__ y,
                              const double2* __restrict__ xi, const double* __restrict__ inv,
                              const double* __restrict__ omega, double2* __restrict__ e, double2* __restrict__ xnew,
                              unsigned long long* rmax, long long n, long long stride) {
  const long long r = blockIdx.y;
  const double w = omega[r];
  const double2* X = x + r * stride;
  const double2* Y = y + r * stride;
  const double2* XI = xi + r * stride;
  const double* IV = inv + r * n;
  double2* E = e + r * stride;
  double2* XN = xnew + r * stride;
  double m = 0.0;
  const long long step = (long long)gridDim.x * blockDim.x;
  for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += EU * step) {
    double2 xv[EU], yv[EU], sv[EU];
    double dv[EU];
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      const long long i = i0 + u * step;
      if (i < n) {
        xv[u] = X[i];
        yv[u] = Y[i];
        sv[u] = XI[i];
        dv[u] = IV[i];
      }
    }
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      const long long i = i0 + u * step;
      if (i < n) {
        const double rr = -sv[u].x - yv[u].x + w * xv[u].x;
        const double ri = -sv[u].y - yv[u].y + w * xv[u].y;
        const double2 ev = make_double2(rr * dv[u], ri * dv[u]);
        E[i] = ev;
        XN[i] = make_double2(xv[u].x + ev.x, xv[u].y + ev.y);
        m = fmax(m, rr * rr + ri * ri);
      }
    }
  }
  __shared__ double sm[256];
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(rmax + r, (unsigned long long)__double_as_longlong(sqrt(sm[0])));
}

cudaError_t launch_update(const double2* x, const double2* y, const double2* xi, const double* inv,
                          const double* omega, double2* e, double2* xnew, unsigned long long* rmax, long long n,
                          long long stride, int nrhs, cudaStream_t st) {
  dim3 grid(grid_for(n, 256 * EU), nrhs);
  update_kernel<<<grid, 256, 0, st>>>(x, y, xi, inv, omega, e, xnew, rmax, n, stride);
  return cudaGetLastError();
}

// R = xi + y - w x (the negated residual of (A - w) x = -xi); rmax[r] = max |R|
__global__ void residual_kernel(const double2* x, const double2* y, const double2* xi, const double* omega,
                                double2* R, unsigned long long* rmax, long long n, long long stride) {
  const long long r = blockIdx.y;
  const double w = omega[r];
  double m = 0.0;
  const long long step = (long long)gridDim.x * blockDim.x;
  for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += EU * step) {
    double2 xv[EU], yv[EU], sv[EU];
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      const long long i = i0 + u * step;
      if (i < n) {
        const long long q = r * stride + i;
        xv[u] = x[q];
        yv[u] = y[q];
        sv[u] = xi[q];
      }
    }
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      const long long i = i0 + u * step;
      if (i < n) {
        const double rr = sv[u].x + yv[u].x - w * xv[u].x, ri = sv[u].y + yv[u].y - w * xv[u].y;
        R[r * stride + i] = make_double2(rr, ri);
        m = fmax(m, rr * rr + ri * ri);
      }
    }
  }
  __shared__ double sm[256];
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(rmax + r, (unsigned long long)__double_as_longlong(sqrt(sm[0])));
}

cudaError_t launch_residual(const double2* x, const double2* y, const double2* xi, const double* omega, double2* R,
                            unsigned long long* rmax, long long n, long long stride, int nrhs, cudaStream_t st) {
  dim3 grid(grid_for(n, 256 * EU), nrhs);
  residual_kernel<<<grid, 256, 0, st>>>(x, y, xi, omega, R, rmax, n, stride);
  return cudaGetLastError();
}

// x0 = -xi * inv   (inv = 1 / (den - w) per system)
__global__ void guess_kernel(const double2* xi, const double* inv, double2* x, long long n, long long stride) {
  const long long r = blockIdx.y;
  const long long step = (long long)gridDim.x * blockDim.x;
  for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += EU * step) {
    double2 sv[EU];
    double dv[EU];
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      const long long i = i0 + u * step;
      if (i < n) {
        sv[u] = xi[r * stride + i];
        dv[u] = inv[r * n + i];
      }
    }
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      const long long i = i0 + u * step;
      if (i < n) {
        x[r * stride + i] = make_double2(-sv[u].x * dv[u], -sv[u].y * dv[u]);
      }
    }
  }
}

cudaError_t launch_guess(const double2* xi, const double* inv, double2* x, long long n, long long stride, int nrhs,
                         cudaStream_t st) {
  dim3 grid(grid_for(n, 256 * EU), nrhs);
  guess_kernel<<<grid, 256, 0, st>>>(xi, inv, x, n, stride);
  return cudaGetLastError();
}

// maxabs over each of nrhs vectors
__global__ void maxabs_kernel(const double2* x, unsigned long long* out, long long n, long long stride) {
  const long long r = blockIdx.y;
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[r * stride + i];
    m = fmax(m, v.x * v.x + v.y * v.y);
  }
  __shared__ double sm[256];
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out + r, (unsigned long long)__double_as_longlong(sqrt(sm[0])));
}

cudaError_t launch_maxabs(const double2* x, unsigned long long* out, long long n, long long stride, int nrhs,
                          cudaStream_t st) {
  dim3 grid(grid_for(n, 256 * 4), nrhs);
  maxabs_kernel<<<grid, 256, 0, st>>>(x, out, n, stride);
  return cudaGetLastError();
}

// batched dot products: out[p] = sum_i op(a_p[i]) b_p[i], op = conj or identity.
// pass 1: fixed partition into DOT_BLOCKS chunks per pair.
constexpr int DOT_BLOCKS = 1024;
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

// ---------------------------------------------------------------------------------
// DIIS on the device (Sec. II.D): the inner products of the newest error vector with the
// history, each system's Hermitian B matrix, the bordered (m+1) x (m+1) solve and the
// extrapolation, all in FP64 without host round trips.  The history is a ring of `depth`
// slots of ns vectors (HE: errors, HX: iterates); iteration `it` wrote slot it % depth and
// the j-th newest entry is slot (it - j) mod depth.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ int ring_slot(int it, int j, int depth) { return ((it - j) % depth + depth) % depth; }

// pass 1 of <HE[newest][i], HE[(it - j)][i]> (first operand conjugated), pair p = j * ns + i
__global__ void diis_dot_pass1(const double2* HE, int it, int depth, int ns, long long n, double2* part) {
  const int p = blockIdx.y;
  const int j = p / ns, i = p - j * ns;
  const double2* A = HE + ((long long)ring_slot(it, 0, depth) * ns + i) * n;
  const double2* Bv = HE + ((long long)ring_slot(it, j, depth) * ns + i) * n;
  const long long chunk = (n + DOT_BLOCKS - 1) / DOT_BLOCKS;
  const long long i0 = (long long)blockIdx.x * chunk;
  const long long i1 = (i0 + chunk < n) ? i0 + chunk : n;
  double sr = 0.0, si = 0.0;
  for (long long k = i0 + threadIdx.x; k < i1; k += blockDim.x) {
    const double2 x = A[k], y = Bv[k];
    sr = fma(x.x, y.x, sr);
    sr = fma(x.y, y.y, sr);
    si = fma(x.x, y.y, si);
    si = fma(-x.y, y.x, si);
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

__device__ __forceinline__ double cabs2(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double q = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / q, (a.y * b.x - a.x * b.y) / q);
}

constexpr int DIIS_MAX = 16;  // history depth limit (the bordered system is at most 17 x 17)

// One thread per system: the second reduction pass (fixed order) of its nhist new B entries,
// the B matrix update (B[slot][sj] and its conjugate), and when `extrapolate` the bordered
// system scaled by 1 / max diag (the coefficients do not depend on the scale), solved by
// Gaussian elimination with partial pivoting.  A singular or non-finite system keeps the
// newest iterate (coefficient 1 on it).
__global__ void diis_solve_kernel(const double2* part, double2* B, int it, int depth, int ns, int nhist,
                                  int extrapolate, double2* coef) {
  // one warp per system: lanes sum the partials k = lane, lane + 32, ... in order, then a fixed
  // shuffle tree; lane 0 goes on alone
  const int i = blockIdx.x;
  const int lane = threadIdx.x;
  double2* Bi = B + (long long)i * depth * depth;
  const int slot = ring_slot(it, 0, depth);
  for (int j = 0; j < nhist; ++j) {
    const long long p = (long long)j * ns + i;
    double sr = 0.0, si = 0.0;
    for (int k = lane; k < DOT_BLOCKS; k += 32) {
      sr += part[p * DOT_BLOCKS + k].x;
      si += part[p * DOT_BLOCKS + k].y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_down_sync(0xffffffffu, sr, o);
      si += __shfl_down_sync(0xffffffffu, si, o);
    }
    if (lane == 0) {
      const int sj = ring_slot(it, j, depth);
      Bi[slot * depth + sj] = make_double2(sr, si);
      Bi[sj * depth + slot] = make_double2(sr, -si);
    }
  }
  if (lane != 0) return;
  double2 x[DIIS_MAX + 1];
  bool good = false;
  if (extrapolate && nhist >= 2) {
    const int m = nhist + 1;
    double2 A[(DIIS_MAX + 1) * (DIIS_MAX + 1)], b[DIIS_MAX + 1];
    double sc = 0.0;
    for (int a = 0; a < nhist; ++a) {
      const int sa = ring_slot(it, a, depth);
      sc = fmax(sc, cabs2(Bi[sa * depth + sa]));
    }
    sc = sc > 0.0 ? 1.0 / sc : 1.0;
    for (int a = 0; a < m; ++a) {
      b[a] = make_double2(a == nhist ? -1.0 : 0.0, 0.0);
      for (int c = 0; c < m; ++c) A[a * m + c] = make_double2(0.0, 0.0);
    }
    for (int a = 0; a < nhist; ++a) {
      const int sa = ring_slot(it, a, depth);
      for (int c = 0; c < nhist; ++c) {
        const double2 v = Bi[sa * depth + ring_slot(it, c, depth)];
        A[a * m + c] = make_double2(sc * v.x, sc * v.y);
      }
      A[a * m + nhist] = make_double2(-1.0, 0.0);
      A[nhist * m + a] = make_double2(-1.0, 0.0);
    }
    good = true;
    for (int c = 0; c < m && good; ++c) {
      int piv = c;
      for (int r = c + 1; r < m; ++r)
        if (cabs2(A[r * m + c]) > cabs2(A[piv * m + c])) piv = r;
      if (cabs2(A[piv * m + c]) < 1e-300) {
        good = false;
        break;
      }
      if (piv != c) {
        for (int k = 0; k < m; ++k) {
          const double2 t = A[c * m + k];
          A[c * m + k] = A[piv * m + k];
          A[piv * m + k] = t;
        }
        const double2 t = b[c];
        b[c] = b[piv];
        b[piv] = t;
      }
      for (int r = c + 1; r < m; ++r) {
        const double2 f = cdiv(A[r * m + c], A[c * m + c]);
        for (int k = c; k < m; ++k) {
          const double2 u = cmul(f, A[c * m + k]);
          A[r * m + k] = make_double2(A[r * m + k].x - u.x, A[r * m + k].y - u.y);
        }
        const double2 u = cmul(f, b[c]);
        b[r] = make_double2(b[r].x - u.x, b[r].y - u.y);
      }
    }
    if (good) {
      for (int r = m - 1; r >= 0; --r) {
        double2 s = b[r];
        for (int k = r + 1; k < m; ++k) {
          const double2 u = cmul(A[r * m + k], x[k]);
          s = make_double2(s.x - u.x, s.y - u.y);
        }
        x[r] = cdiv(s, A[r * m + r]);
        if (!isfinite(x[r].x) || !isfinite(x[r].y)) good = false;
      }
    }
  }
  for (int j = 0; j < nhist; ++j)
    coef[(long long)j * ns + i] = good ? x[j] : make_double2(j == 0 ? 1.0 : 0.0, 0.0);
}

// out[r] = sum_j c[j*nrhs + r] * HX[slot (it - j)][r]
__global__ void diis_lincomb_kernel(const double2* HX, int it, int depth, const double2* c, int m, double2* out,
                                    long long n, long long stride, int nrhs) {
  const long long r = blockIdx.y;
  const long long step = (long long)gridDim.x * blockDim.x;
  for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += EU * step) {
    double sr[EU], si[EU];
#pragma unroll
    for (int u = 0; u < EU; ++u) sr[u] = si[u] = 0.0;
    for (int j = 0; j < m; ++j) {
      const double2 cc = c[(long long)j * nrhs + r];
      const double2* hx = HX + ((long long)ring_slot(it, j, depth) * nrhs + r) * stride;
      double2 x[EU];
#pragma unroll
      for (int u = 0; u < EU; ++u)
        if (i0 + u * step < n) x[u] = hx[i0 + u * step];
#pragma unroll
      for (int u = 0; u < EU; ++u)
        if (i0 + u * step < n) {
          sr[u] += cc.x * x[u].x - cc.y * x[u].y;
          si[u] += cc.x * x[u].y + cc.y * x[u].x;
        }
    }
#pragma unroll
    for (int u = 0; u < EU; ++u)
      if (i0 + u * step < n) out[r * stride + i0 + u * step] = make_double2(sr[u], si[u]);
  }
}

cudaError_t launch_diis_device(const double2* HE, const double2* HX, double2* B, int it, int depth, int ns, int nhist,
                               int extrapolate, long long n, double2* part, double2* coef, double2* out,
                               cudaStream_t st) {
  if (depth > DIIS_MAX || nhist < 1 || nhist > depth || (long long)nhist * ns > 65535) return cudaErrorInvalidValue;
  dim3 g1(DOT_BLOCKS, nhist * ns);
  diis_dot_pass1<<<g1, 256, 0, st>>>(HE, it, depth, ns, n, part);
  diis_solve_kernel<<<ns, 32, 0, st>>>(part, B, it, depth, ns, nhist, extrapolate, coef);
  dim3 g3(grid_for(n, 256 * EU), ns);
  diis_lincomb_kernel<<<g3, 256, 0, st>>>(HX, it, depth, coef, nhist, out, n, n, ns);
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
  const long long step = (long long)gridDim.x * blockDim.x;
  for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += EU * step) {
    double2 xv[EU], yv[EU];
#pragma unroll
    for (int u = 0; u < EU; ++u)
      if (i0 + u * step < n) {
        xv[u] = x[i0 + u * step];
        yv[u] = y[i0 + u * step];
      }
#pragma unroll
    for (int u = 0; u < EU; ++u)
      if (i0 + u * step < n)
        y[i0 + u * step] = make_double2(a.x * xv[u].x - a.y * xv[u].y + b.x * yv[u].x - b.y * yv[u].y,
                                        a.x * xv[u].y + a.y * xv[u].x + b.x * yv[u].y + b.y * yv[u].x);
  }
}

cudaError_t launch_axpby(double2 a, const double2* x, double2 b, double2* y, long long n, cudaStream_t st) {
  axpby_kernel<<<grid_for(n, 256 * EU), 256, 0, st>>>(a, x, b, y, n);
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
