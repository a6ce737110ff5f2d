// FP64 kernels for the two GEMM shapes that tile-based kernels handle poorly, used in
// every precision mode (they are memory-bound, so FP64 costs nothing extra):
//
// skinny_k_kernel — short contraction (K <= 16) with few rows (M <= 64), e.g. the
//   Fock-like hole terms r(i, j, ab) += sum_k F(k, j) x(i, k, ab): one CTA per (batch entry,
//   chunk of 128 columns) stages A (M x K) and the B chunk (K x 128) of each segment in
//   shared memory; every thread owns whole output elements and adds them to C.
//
// reduce_small_kernel — tiny output (M * N <= 64) with a long contraction, both operands
//   K-contiguous (ta = 0, tb = 1), e.g. the o x o intermediates summed over (l, c, d) and
//   three momenta: each warp owns up to 8 output elements, its lanes stride over K and the
//   lane sums meet in a warp shuffle reduction; the (segment, K) iteration space is split
//   over CTAs and the partials go through the fixed-order split reduction.
#include "kernels.cuh"

namespace lrcc {

namespace {

constexpr int SK_NT = 128;       // columns per CTA
constexpr int SK_THREADS = 256;
constexpr int SK_MAXK = 16, SK_MAXM = 64;

__device__ __forceinline__ void cmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

}  // namespace

// PER = outputs per thread = M * SK_NT / SK_THREADS rounded up (the launcher picks the
// smallest instantiation that covers M, keeping the accumulators in registers)
template <int PER>
__global__ void __launch_bounds__(SK_THREADS) skinny_k_kernel(GemmArgs g, int nchunk) {
  __shared__ double2 As[SK_MAXM][SK_MAXK];
  __shared__ double2 Bs[SK_MAXK][SK_NT];
  const int batch = blockIdx.x / nchunk, chunk = blockIdx.x - batch * nchunk;
  const int n0 = chunk * SK_NT;
  const long long rhs = blockIdx.y;
  const double2* Ab = g.A + rhs * g.sA;
  const double2* Bb = g.B + rhs * g.sB;
  const int M = g.M, N = g.N, K = g.K, tid = threadIdx.x;
  const int nout = M * SK_NT;
  double2 acc[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) acc[j] = make_double2(0.0, 0.0);
  for (int s = g.sbeg[batch]; s < g.sbeg[batch + 1]; ++s) {
    const double2* Ap = Ab + g.aoff[s];
    const double2* Bp = Bb + g.boff[s];
    __syncthreads();
    for (int e = tid; e < M * K; e += SK_THREADS) {
      const int m = e / K, k = e - m * K;
      As[m][k] = g.ta ? Ap[(long long)k * g.lda + m] : Ap[(long long)m * g.lda + k];
    }
    for (int e = tid; e < K * SK_NT; e += SK_THREADS) {
      int k, c;
      if (g.tb) {  // B[n][k]: consecutive threads walk k
        c = e / K;
        k = e - c * K;
      } else {     // B[k][n]: consecutive threads walk n
        k = e / SK_NT;
        c = e - k * SK_NT;
      }
      const int n = n0 + c;
      Bs[k][c] = n < N ? (g.tb ? Bp[(long long)n * g.ldb + k] : Bp[(long long)k * g.ldb + n])
                       : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int o = tid + j * SK_THREADS;
      if (o >= nout) break;
      const int m = o / SK_NT, c = o - m * SK_NT;
      for (int k = 0; k < K; ++k) cmac(acc[j], As[m][k], Bs[k][c]);
    }
  }
  double2* Cp = g.C + rhs * g.sC + g.coff[batch];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int o = tid + j * SK_THREADS;
    if (o >= nout) break;
    const int m = o / SK_NT, n = n0 + (o - m * SK_NT);
    if (n >= N) continue;
    const double vr = g.ar * acc[j].x - g.ai * acc[j].y, vi = g.ar * acc[j].y + g.ai * acc[j].x;
    double2* cp = Cp + (long long)m * g.ldc + n;
    double2 cv = *cp;
    cv.x += vr;
    cv.y += vi;
    *cp = cv;
  }
}

bool skinny_k_ok(const GemmArgs& g) { return g.K <= SK_MAXK && g.M <= SK_MAXM && g.epi == 0; }

cudaError_t launch_skinny_k(const GemmArgs& g, int nrhs, cudaStream_t st) {
  if (!skinny_k_ok(g)) return cudaErrorInvalidValue;
  const int nchunk = (g.N + SK_NT - 1) / SK_NT;
  const long long nblk = (long long)g.nbatch * nchunk;
  if (nblk <= 0) return cudaSuccess;
  if (nblk > 2147483647LL || nrhs > 65535) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)nblk, (unsigned)nrhs);
  const int per = (g.M * SK_NT + SK_THREADS - 1) / SK_THREADS;
  if (per <= 4) skinny_k_kernel<4><<<grid, SK_THREADS, 0, st>>>(g, nchunk);
  else if (per <= 8) skinny_k_kernel<8><<<grid, SK_THREADS, 0, st>>>(g, nchunk);
  else if (per <= 16) skinny_k_kernel<16><<<grid, SK_THREADS, 0, st>>>(g, nchunk);
  else skinny_k_kernel<32><<<grid, SK_THREADS, 0, st>>>(g, nchunk);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------------
constexpr int RS_WARPS = 8, RS_OUT = 8;  // outputs per warp

__global__ void __launch_bounds__(RS_WARPS * 32) reduce_small_kernel(GemmArgs g) {
  const int batch = blockIdx.x / g.nsplit, sp = blockIdx.x - batch * g.nsplit;
  const long long rhs = blockIdx.y;
  const double2* Ab = g.A + rhs * g.sA;
  const double2* Bb = g.B + rhs * g.sB;
  const int M = g.M, N = g.N, K = g.K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nout = M * N;
  // this split's share of the (segment, element) iteration space, in whole segments
  const int s0 = g.sbeg[batch], s1 = g.sbeg[batch + 1];
  const long long total = (long long)(s1 - s0);
  const int slo = s0 + (int)(total * sp / g.nsplit), shi = s0 + (int)(total * (sp + 1) / g.nsplit);
  double2 acc[RS_OUT];
  int om[RS_OUT], on[RS_OUT];
#pragma unroll
  for (int j = 0; j < RS_OUT; ++j) {
    acc[j] = make_double2(0.0, 0.0);
    const int o = warp + j * RS_WARPS;
    om[j] = o < nout ? o / N : 0;
    on[j] = o < nout ? o - (o / N) * N : 0;
  }
  for (int s = slo; s < shi; ++s) {
    const double2* Ap = Ab + g.aoff[s];
    const double2* Bp = Bb + g.boff[s];
    for (int k = lane; k < K; k += 32) {
#pragma unroll
      for (int j = 0; j < RS_OUT; ++j) {
        if (warp + j * RS_WARPS >= nout) break;
        cmac(acc[j], Ap[(long long)om[j] * g.lda + k], Bp[(long long)on[j] * g.ldb + k]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < RS_OUT; ++j) {
    for (int off = 16; off > 0; off >>= 1) {
      acc[j].x += __shfl_down_sync(0xffffffffu, acc[j].x, off);
      acc[j].y += __shfl_down_sync(0xffffffffu, acc[j].y, off);
    }
  }
  if (lane != 0) return;
  double2* Pp = g.part + ((rhs * g.nbatch + batch) * g.nsplit + sp) * (long long)M * N;
#pragma unroll
  for (int j = 0; j < RS_OUT; ++j) {
    const int o = warp + j * RS_WARPS;
    if (o >= nout) break;
    Pp[o] = acc[j];  // raw partial of C[om][on], row-major M x N
  }
}

bool reduce_small_ok(const GemmArgs& g) { return g.M * g.N <= RS_WARPS * RS_OUT && g.ta == 0 && g.tb == 1; }

cudaError_t launch_reduce_small(const GemmArgs& g, int nrhs, cudaStream_t st) {
  if (!reduce_small_ok(g) || g.nsplit < 1 || !g.part) return cudaErrorInvalidValue;
  const long long nblk = (long long)g.nbatch * g.nsplit;
  if (nblk <= 0) return cudaSuccess;
  if (nblk > 2147483647LL || nrhs > 65535) return cudaErrorInvalidConfiguration;
  reduce_small_kernel<<<dim3((unsigned)nblk, (unsigned)nrhs), RS_WARPS * 32, 0, st>>>(g);
  return cudaGetLastError();
}

}  // namespace lrcc
