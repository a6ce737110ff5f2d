// Kernels for the two GEMM shapes that tile-based kernels handle poorly.  Both load
// FP64 operands and update the FP64 destination in FP64; the arithmetic is FP64 for the
// FP64 products and FP32 for the mixed-precision ones.  At about 1.3 flops per byte
// (8 complex MACs per loaded element at K = M = 8) these shapes are bound by GB300's
// FP64 pipe (1.25 TFLOP/s against 7.6 TB/s), but by HBM in FP32; the FP32 rounding
// (2^-24 per operand, short chains) is far below the BF16x3 operand split's.
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
__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

template <typename V> struct Arith;  // V: double2 (FP64 arithmetic) or float2 (FP32)
template <> struct Arith<double2> {
  static __device__ __forceinline__ double2 from(double2 v) { return v; }
  static __device__ __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
};
template <> struct Arith<float2> {
  static __device__ __forceinline__ float2 from(double2 v) {
    return make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
  }
  static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
};

}  // namespace

// One thread per output column n: it loads the column's K values of B into registers
// (independent loads, all in flight together), keeps M accumulators, and adds the column
// of C at the end; A (M x K) is staged in shared memory per segment.  Memory-bound: every
// element of B and C is touched once.
template <typename V, int MM, int KK>  // arithmetic type; compile-time bounds of M and K (register arrays)
__global__ void __launch_bounds__(SK_THREADS) skinny_k_kernel(GemmArgs g, int nchunk) {
  using AR = Arith<V>;
  __shared__ V As[MM][KK];
  const int batch = blockIdx.x / nchunk, chunk = blockIdx.x - batch * nchunk;
  const int n = chunk * SK_THREADS + threadIdx.x;
  const long long rhs = blockIdx.y;
  const double2* Ab = g.A + rhs * g.sA;
  const double2* Bb = g.B + rhs * g.sB;
  const int M = g.M, N = g.N, K = g.K, tid = threadIdx.x;
  V acc[MM];
#pragma unroll
  for (int m = 0; m < MM; ++m) acc[m] = AR::zero();
  for (int s = g.sbeg[batch]; s < g.sbeg[batch + 1]; ++s) {
    const double2* Ap = Ab + g.aoff[s];
    const double2* Bp = Bb + g.boff[s];
    __syncthreads();
    for (int e = tid; e < M * K; e += SK_THREADS) {
      const int m = e / K, k = e - m * K;
      As[m][k] = AR::from(g.ta ? Ap[(long long)k * g.lda + m] : Ap[(long long)m * g.lda + k]);
    }
    __syncthreads();
    if (n < N) {
      V b[KK];
#pragma unroll
      for (int k = 0; k < KK; ++k)
        if (k < K) b[k] = AR::from(g.tb ? Bp[(long long)n * g.ldb + k] : Bp[(long long)k * g.ldb + n]);
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
    if (m < M) cv[m] = g.store ? make_double2(0.0, 0.0) : Cp[(long long)m * g.ldc + n];
#pragma unroll
  for (int m = 0; m < MM; ++m) {
    if (m >= M) break;
    const double ur = (double)acc[m].x, ui = (double)acc[m].y;
    cv[m].x += g.ar * ur - g.ai * ui;
    cv[m].y += g.ar * ui + g.ai * ur;
    Cp[(long long)m * g.ldc + n] = cv[m];
  }
}

bool skinny_k_ok(const GemmArgs& g) { return g.K <= SK_MAXK && g.M <= SK_MAXM && g.N >= 64 && g.epi == 0; }

template <typename V>
static void skinny_launch(const GemmArgs& g, dim3 grid, int nchunk, cudaStream_t st) {
  if (g.M <= 8 && g.K <= 8) skinny_k_kernel<V, 8, 8><<<grid, SK_THREADS, 0, st>>>(g, nchunk);
  else skinny_k_kernel<V, SK_MAXM, SK_MAXK><<<grid, SK_THREADS, 0, st>>>(g, nchunk);
}

cudaError_t launch_skinny_k(const GemmArgs& g, int nrhs, cudaStream_t st, bool f32) {
  if (!skinny_k_ok(g)) return cudaErrorInvalidValue;
  const int nchunk = (g.N + SK_THREADS - 1) / SK_THREADS;
  const long long nblk = (long long)g.nbatch * nchunk;
  if (nblk <= 0) return cudaSuccess;
  if (nblk > 2147483647LL || nrhs > 65535) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)nblk, (unsigned)nrhs);
  if (f32) skinny_launch<float2>(g, grid, nchunk, st);
  else skinny_launch<double2>(g, grid, nchunk, st);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------------
constexpr int RS_WARPS = 8, RS_OUT = 8;  // outputs per warp

template <typename V>
__global__ void __launch_bounds__(RS_WARPS * 32) reduce_small_kernel(GemmArgs g) {
  using AR = Arith<V>;
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
  V acc[RS_OUT];
  int om[RS_OUT], on[RS_OUT];
#pragma unroll
  for (int j = 0; j < RS_OUT; ++j) {
    acc[j] = AR::zero();
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
        cmac(acc[j], AR::from(Ap[(long long)om[j] * g.lda + k]), AR::from(Bp[(long long)on[j] * g.ldb + k]));
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
    Pp[o] = make_double2((double)acc[j].x, (double)acc[j].y);  // raw partial of C[om][on], row-major M x N
  }
}

bool reduce_small_ok(const GemmArgs& g) { return g.M * g.N <= RS_WARPS * RS_OUT && g.ta == 0 && g.tb == 1; }

cudaError_t launch_reduce_small(const GemmArgs& g, int nrhs, cudaStream_t st, bool f32) {
  if (!reduce_small_ok(g) || g.nsplit < 1 || !g.part) return cudaErrorInvalidValue;
  const long long nblk = (long long)g.nbatch * g.nsplit;
  if (nblk <= 0) return cudaSuccess;
  if (nblk > 2147483647LL || nrhs > 65535) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)nblk, (unsigned)nrhs);
  if (f32) reduce_small_kernel<float2><<<grid, RS_WARPS * 32, 0, st>>>(g);
  else reduce_small_kernel<double2><<<grid, RS_WARPS * 32, 0, st>>>(g);
  return cudaGetLastError();
}

}  // namespace lrcc
