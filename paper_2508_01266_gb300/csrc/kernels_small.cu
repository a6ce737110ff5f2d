// FP64 kernels for the two GEMM shapes that tile-based kernels handle poorly, used in
// every precision mode (they are memory-bound, so FP64 costs nothing extra):
//
// skinny_k_kernel — short contraction (K <= 16) with few rows (M <= 16) and long rows
//   (N >= 64), e.g. the Fock-like hole terms r(i, j, ab) += sum_k F(k, j) x(i, k, ab): one
//   thread per output column, one CTA per (batch entry, 256 columns).
//
// reduce_small_kernel — tiny output (M * N <= 64) with a long contraction, both operands
//   K-contiguous (ta = 0, tb = 1), e.g. the o x o intermediates summed over (l, c, d) and
//   three momenta: each warp owns up to 8 output elements, its lanes stride over K and the
//   lane sums meet in a warp shuffle reduction; the (segment, K) iteration space is split
//   over CTAs and the partials go through the fixed-order split reduction.
#include "kernels.cuh"

namespace lrcc {

namespace {

constexpr int SK_THREADS = 256;  // columns per CTA
constexpr int SK_MAXK = 16, SK_MAXM = 16;

__device__ __forceinline__ void cmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

}  // namespace

// One thread per output column n: it loads the column's K values of B into registers
// (independent loads, all in flight together), keeps M accumulators, and adds the column
// of C at the end; A (M x K) is staged in shared memory per segment.  Memory-bound: every
// element of B and C is touched once.
template <int MM, int KK>  // compile-time bounds of M and K (register arrays)
__global__ void __launch_bounds__(SK_THREADS) skinny_k_kernel(GemmArgs g, int nchunk) {
  __shared__ double2 As[MM][KK];
  const int batch = blockIdx.x / nchunk, chunk = blockIdx.x - batch * nchunk;
  const int n = chunk * SK_THREADS + threadIdx.x;
  const long long rhs = blockIdx.y;
  const double2* Ab = g.A + rhs * g.sA;
  const double2* Bb = g.B + rhs * g.sB;
  const int M = g.M, N = g.N, K = g.K, tid = threadIdx.x;
  double2 acc[MM];
#pragma unroll
  for (int m = 0; m < MM; ++m) acc[m] = make_double2(0.0, 0.0);
  for (int s = g.sbeg[batch]; s < g.sbeg[batch + 1]; ++s) {
    const double2* Ap = Ab + g.aoff[s];
    const double2* Bp = Bb + g.boff[s];
    __syncthreads();
    for (int e = tid; e < M * K; e += SK_THREADS) {
      const int m = e / K, k = e - m * K;
      As[m][k] = g.ta ? Ap[(long long)k * g.lda + m] : Ap[(long long)m * g.lda + k];
    }
    __syncthreads();
    if (n < N) {
      double2 b[KK];
#pragma unroll
      for (int k = 0; k < KK; ++k)
        if (k < K) b[k] = g.tb ? Bp[(long long)n * g.ldb + k] : Bp[(long long)k * g.ldb + n];
#pragma unroll
      for (int m = 0; m < MM; ++m) {
        if (m >= M) break;
#pragma unroll
        for (int k = 0; k < KK; ++k)
          if (k < K) cmac(acc[m], As[m][k], b[k]);
      }
    }
  }
  if (n >= N) return;
  double2* Cp = g.C + rhs * g.sC + g.coff[batch];
  double2 cv[MM];  // all loads first, then the stores (no load waits on a store)
#pragma unroll
  for (int m = 0; m < MM; ++m)
    if (m < M) cv[m] = Cp[(long long)m * g.ldc + n];
#pragma unroll
  for (int m = 0; m < MM; ++m) {
    if (m >= M) break;
    cv[m].x += g.ar * acc[m].x - g.ai * acc[m].y;
    cv[m].y += g.ar * acc[m].y + g.ai * acc[m].x;
    Cp[(long long)m * g.ldc + n] = cv[m];
  }
}

bool skinny_k_ok(const GemmArgs& g) { return g.K <= SK_MAXK && g.M <= SK_MAXM && g.N >= 64 && g.epi == 0; }

cudaError_t launch_skinny_k(const GemmArgs& g, int nrhs, cudaStream_t st) {
  if (!skinny_k_ok(g)) return cudaErrorInvalidValue;
  const int nchunk = (g.N + SK_THREADS - 1) / SK_THREADS;
  const long long nblk = (long long)g.nbatch * nchunk;
  if (nblk <= 0) return cudaSuccess;
  if (nblk > 2147483647LL || nrhs > 65535) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)nblk, (unsigned)nrhs);
  if (g.M <= 8 && g.K <= 8) skinny_k_kernel<8, 8><<<grid, SK_THREADS, 0, st>>>(g, nchunk);
  else skinny_k_kernel<SK_MAXM, SK_MAXK><<<grid, SK_THREADS, 0, st>>>(g, nchunk);
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
