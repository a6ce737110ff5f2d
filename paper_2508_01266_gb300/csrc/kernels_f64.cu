// FP64 (complex128) kernels of the plan executor: segmented batched GEMM,
// momentum-aware layout permutation, batched 2-D transpose and DF-factor split.
//
// On GB300 the FP64 pipe (measured ~1.2 TFLOP/s for DFMA) is the bound of every
// FP64 contraction in this path, so the GEMM is a shared-memory tiled DFMA kernel:
// each thread owns a TM x TN register tile of complex accumulators (3 DFMA per
// complex MAC: Gauss's three-product form); tiles are picked per op to minimise padded
// work.
//
// The same GEMM with FP32 arithmetic (operands rounded to FP32 when staged in shared
// memory, FP32 accumulators, the FP64 destination updated in FP64) serves the mixed-
// precision products for the small-tile shapes that would leave tensor-core tiles mostly
// padding: at 2 flops per byte they are FP64-pipe bound but HBM bound in FP32, and the
// FP32 rounding (2^-24 per operand, chains capped by the caller) is far below the
// BF16x3 operand split's.
#include <cstdio>

#include "kernels.cuh"

namespace lrcc {

__device__ __forceinline__ int kmod(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

template <typename T> struct Cplx;
template <> struct Cplx<double> {
  using t = double2;
  static __device__ __forceinline__ double2 from(double2 v) { return v; }
  static __device__ __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }
};
template <> struct Cplx<float> {
  using t = float2;
  static __device__ __forceinline__ float2 from(double2 v) {
    return make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
  }
  static __device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }
};

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    zgemm_seg_kernel(GemmArgs g) {
  constexpr int NTX = BN / TN, NTY = BM / TM, NT = NTX * NTY;
  using C2 = Cplx<T>;
  using V2 = typename C2::t;
  // FP64: Gauss's three-product form of the complex MAC.  With P1 = ar br, P2 = ai bi,
  // P3 = (ar + ai)(br + bi) summed over K, C = (P1 - P2) + i (P3 - P1 - P2): 3 DFMA per
  // complex MAC instead of 4 on the FP64 pipe that bounds these GEMMs.  The sums ar + ai and
  // br + bi are formed once per element when the tiles are staged (a third shared-memory
  // plane).  FP32 (mixed precision, HBM-bound shapes) keeps the four-product form.
  constexpr bool G3 = sizeof(T) == 8;
  constexpr int NP = G3 ? 3 : 2;
  __shared__ T As[NP][BK][BM];
  __shared__ T Bs[NP][BK][BN];
  const int tpb = g.tiles_m * g.tiles_n;
  const int bid = blockIdx.x;
  const int per_batch = tpb * g.nsplit;
  const int batch = bid / per_batch;
  const int rem = bid - batch * per_batch;
  const int sp = rem / tpb;
  const int t = rem - sp * tpb;
  const int m0 = (t / g.tiles_n) * BM;
  const int n0 = (t % g.tiles_n) * BN;
  const long long rhs = blockIdx.y;
  const double2* Ab = g.A + rhs * g.sA;
  const double2* Bb = g.B + rhs * g.sB;
  double2* Cb = g.C + rhs * g.sC;
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;
  const int M = g.M, N = g.N, K = g.K;
  // G3: acc[0] = P1, acc[1] = P2, acc[2] = P3; otherwise acc[0] = Re, acc[1] = Im
  T acc[NP][TM][TN];
#pragma unroll
  for (int q = 0; q < NP; ++q)
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[q][i][j] = T(0);
  // iteration space of this batch entry: (segment, K block), segment-major; this CTA
  // takes the split's contiguous range of it
  const int s0 = g.sbeg[batch], s1 = g.sbeg[batch + 1];
  const int nkb = (K + BK - 1) / BK;
  const long long total = (long long)(s1 - s0) * nkb;
  const long long lo = total * sp / g.nsplit, hi = total * (sp + 1) / g.nsplit;
  int s = s0 + (int)(lo / nkb), kb = (int)(lo % nkb);
  for (long long it = lo; it < hi; ++it) {
    const double2* Ap = Ab + g.aoff[s];
    const double2* Bp = Bb + g.boff[s];
    const int k0 = kb * BK;
    {
      for (int idx = tid; idx < BM * BK; idx += NT) {
        int m, k;
        if (!g.ta) {
          k = idx % BK;
          m = idx / BK;
        } else {
          m = idx % BM;
          k = idx / BM;
        }
        const int gm = m0 + m, gk = k0 + k;
        double2 val = make_double2(0.0, 0.0);
        if (gm < M && gk < K) val = g.ta ? Ap[(long long)gk * g.lda + gm] : Ap[(long long)gm * g.lda + gk];
        const V2 cv = C2::from(val);
        As[0][k][m] = cv.x;
        As[1][k][m] = cv.y;
        if constexpr (G3) As[2][k][m] = cv.x + cv.y;
      }
      for (int idx = tid; idx < BK * BN; idx += NT) {
        int k, n;
        if (!g.tb) {
          n = idx % BN;
          k = idx / BN;
        } else {
          k = idx % BK;
          n = idx / BK;
        }
        const int gn = n0 + n, gk = k0 + k;
        double2 val = make_double2(0.0, 0.0);
        if (gn < N && gk < K) val = g.tb ? Bp[(long long)gn * g.ldb + gk] : Bp[(long long)gk * g.ldb + gn];
        const V2 cv = C2::from(val);
        Bs[0][k][n] = cv.x;
        Bs[1][k][n] = cv.y;
        if constexpr (G3) Bs[2][k][n] = cv.x + cv.y;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[NP][TM], b[NP][TN];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
#pragma unroll
          for (int i = 0; i < TM; ++i) a[q][i] = As[q][kk][ty + i * NTY];
#pragma unroll
          for (int j = 0; j < TN; ++j) b[q][j] = Bs[q][kk][tx + j * NTX];
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            if constexpr (G3) {
              acc[0][i][j] = C2::mad(a[0][i], b[0][j], acc[0][i][j]);
              acc[1][i][j] = C2::mad(a[1][i], b[1][j], acc[1][i][j]);
              acc[2][i][j] = C2::mad(a[2][i], b[2][j], acc[2][i][j]);
            } else {
              acc[0][i][j] = C2::mad(a[0][i], b[0][j], acc[0][i][j]);
              acc[0][i][j] = C2::mad(-a[1][i], b[1][j], acc[0][i][j]);
              acc[1][i][j] = C2::mad(a[0][i], b[1][j], acc[1][i][j]);
              acc[1][i][j] = C2::mad(a[1][i], b[0][j], acc[1][i][j]);
            }
          }
      }
      __syncthreads();
    }
    if (++kb == nkb) {
      kb = 0;
      ++s;
    }
  }
  T accr[TM][TN], acci[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      if constexpr (G3) {
        accr[i][j] = acc[0][i][j] - acc[1][i][j];
        acci[i][j] = acc[2][i][j] - acc[0][i][j] - acc[1][i][j];
      } else {
        accr[i][j] = acc[0][i][j];
        acci[i][j] = acc[1][i][j];
      }
    }
  if (g.nsplit > 1) {  // raw partial tile; alpha and the epilogue come in the reduction
    double2* Pp = g.part + ((rhs * g.nbatch + batch) * g.nsplit + sp) * (long long)M * N;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int m = m0 + ty + i * NTY;
      if (m >= M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int n = n0 + tx + j * NTX;
        if (n < N) Pp[(long long)m * N + n] = make_double2((double)accr[i][j], (double)acci[i][j]);
      }
    }
    return;
  }
  double2* Cp = Cb + g.coff[batch];
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + ty + i * NTY;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx + j * NTX;
      if (n >= N) continue;
      long long addr;
      if (g.epi == 0) {
        addr = (long long)m * g.ldc + n;
      } else {
        const int a = m / g.ep2, c = m - a * g.ep2;
        const int b = n / g.ep3, d = n - b * g.ep3;
        addr = (((long long)a * g.ep1 + b) * g.ep2 + c) * g.ep3 + d;
      }
      const double ur = (double)accr[i][j], ui = (double)acci[i][j];
      const double vr = g.ar * ur - g.ai * ui;
      const double vi = g.ar * ui + g.ai * ur;
      if (g.epi == 0) {
        double2 cv = g.store ? make_double2(0.0, 0.0) : Cp[addr];
        cv.x += vr;
        cv.y += vi;
        Cp[addr] = cv;
      } else {  // W-block build: the workspace slot is overwritten
        Cp[addr] = make_double2(vr, vi);
      }
    }
  }
}

// Sum of the split partials in split order, alpha, and the GEMM's epilogue.
__global__ void split_reduce_kernel(GemmArgs g) {
  const long long rhs = blockIdx.y;
  const long long mn = (long long)g.M * g.N;
  const long long total = (long long)g.nbatch * mn;
  double2* Cb = g.C + rhs * g.sC;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int batch = (int)(e / mn);
    const long long r = e - (long long)batch * mn;
    const int m = (int)(r / g.N), n = (int)(r - (long long)m * g.N);
    const double2* p = g.part + (rhs * g.nbatch + batch) * g.nsplit * mn + r;
    double sr = 0.0, si = 0.0;
    for (int k = 0; k < g.nsplit; ++k) {
      const double2 v = p[(long long)k * mn];
      sr += v.x;
      si += v.y;
    }
    const double vr = g.ar * sr - g.ai * si, vi = g.ar * si + g.ai * sr;
    double2* Cp = Cb + g.coff[batch];
    if (g.epi == 0) {
      double2* cp = Cp + (long long)m * g.ldc + n;
      double2 cv = g.store ? make_double2(0.0, 0.0) : *cp;
      cv.x += vr;
      cv.y += vi;
      *cp = cv;
    } else {
      const int a = m / g.ep2, c = m - a * g.ep2;
      const int b = n / g.ep3, d = n - b * g.ep3;
      Cp[(((long long)a * g.ep1 + b) * g.ep2 + c) * g.ep3 + d] = make_double2(vr, vi);
    }
  }
}

cudaError_t launch_split_reduce(const GemmArgs& g, int nrhs, cudaStream_t st) {
  const long long total = (long long)g.nbatch * g.M * g.N;
  if (total <= 0) return cudaSuccess;
  long long blocks = (total + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  dim3 grid((unsigned)blocks, (unsigned)nrhs);
  split_reduce_kernel<<<grid, 256, 0, st>>>(g);
  return cudaGetLastError();
}

void gemm_tile_dims(int tile, int* bm, int* bn) {
  static const int d[GT_COUNT][2] = {{64, 64}, {32, 64}, {64, 32}, {32, 32}, {16, 64}, {64, 16},
                                     {16, 16}, {8, 32},  {1, 256}, {256, 1}, {48, 48}};
  *bm = d[tile][0];
  *bn = d[tile][1];
}

int gemm_pick_tile(int M, int N) {
  int best = 0;
  double bestw = 1e300;
  for (int t = 0; t < GT_COUNT; ++t) {
    int bm, bn;
    gemm_tile_dims(t, &bm, &bn);
    double w = (double)((M + bm - 1) / bm) * bm * (double)((N + bn - 1) / bn) * bn;
    // prefer larger tiles on ties (fewer CTAs, fewer tile reloads)
    w *= 1.0 + 0.02 * (4096.0 / (bm * bn));
    if (w < bestw) {
      bestw = w;
      best = t;
    }
  }
  return best;
}

template <typename T, int BM, int BN, int TM, int TN>
static cudaError_t launch_t(GemmArgs g, int nrhs, cudaStream_t st) {
  g.tiles_m = (g.M + BM - 1) / BM;
  g.tiles_n = (g.N + BN - 1) / BN;
  if (g.nsplit < 1 || (g.nsplit > 1 && !g.part)) return cudaErrorInvalidValue;
  long long nblk = (long long)g.tiles_m * g.tiles_n * g.nbatch * g.nsplit;
  if (nblk <= 0) return cudaSuccess;
  if (nblk > 2147483647LL || nrhs > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)nblk, (unsigned)nrhs);
  zgemm_seg_kernel<T, BM, BN, F64_BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, st>>>(g);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_tile(const GemmArgs& g, int tile, int nrhs, cudaStream_t st) {
  switch (tile) {
    case GT_64x64: return launch_t<T, 64, 64, 4, 4>(g, nrhs, st);
    case GT_32x64: return launch_t<T, 32, 64, 2, 4>(g, nrhs, st);
    case GT_64x32: return launch_t<T, 64, 32, 4, 2>(g, nrhs, st);
    case GT_32x32: return launch_t<T, 32, 32, 2, 2>(g, nrhs, st);
    case GT_16x64: return launch_t<T, 16, 64, 1, 4>(g, nrhs, st);
    case GT_64x16: return launch_t<T, 64, 16, 4, 1>(g, nrhs, st);
    case GT_16x16: return launch_t<T, 16, 16, 1, 1>(g, nrhs, st);
    case GT_8x32: return launch_t<T, 8, 32, 1, 1>(g, nrhs, st);
    case GT_1x256: return launch_t<T, 1, 256, 1, 1>(g, nrhs, st);
    case GT_256x1: return launch_t<T, 256, 1, 1, 1>(g, nrhs, st);
    case GT_48x48: return launch_t<T, 48, 48, 3, 3>(g, nrhs, st);  // 40 x 40 blocks (nvir = 40)
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_gemm_f64(const GemmArgs& g, int tile, int nrhs, cudaStream_t st) {
  return launch_tile<double>(g, tile, nrhs, st);
}

cudaError_t launch_gemm_f32(const GemmArgs& g, int tile, int nrhs, cudaStream_t st) {
  return launch_tile<float>(g, tile, nrhs, st);
}

// --------------------------------------------------------------------------
// layout permutation
// --------------------------------------------------------------------------
__device__ __forceinline__ long long lay_off(int kind, int nk, const int* n, int k1, int k2, int k3, int i1,
                                             int i2, int i3, int i4) {
  const long long n0 = n[0], n1 = n[1], n2 = n[2], n3 = n[3];
  if (kind == 0) {
    return (((long long)k1 * nk + k2) * nk + k3) * (n0 * n1 * n2 * n3) + ((i1 * n1 + i2) * n2 + i3) * n3 + i4;
  } else if (kind == 1) {
    const int P = kmod(k1 + k2, nk);
    const long long rows = nk * n0 * n1, cols = nk * n2 * n3;
    return (long long)P * rows * cols + (((long long)k1 * n0 + i1) * n1 + i2) * cols +
           ((long long)k3 * n2 + i3) * n3 + i4;
  } else if (kind == 2) {
    const int q = kmod(k3 - k1, nk);
    const int k4 = kmod(k1 + k2 - k3, nk);
    const long long rows = nk * n0 * n2, cols = nk * n3 * n1;
    return (long long)q * rows * cols + (((long long)k1 * n0 + i1) * n2 + i3) * cols +
           ((long long)k4 * n3 + i4) * n1 + i2;
  } else {
    return (((long long)k1 * nk + k3) * nk + k2) * (n0 * n1 * n2 * n3) + ((i1 * n2 + i3) * n1 + i2) * n3 + i4;
  }
}

__global__ void perm_kernel(PermArgs p) {
  const long long rhs = blockIdx.y;
  const double2* S = p.S + rhs * p.sS;
  double2* D = p.D + rhs * p.sD;
  const int nk = p.dnk;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < p.total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e;
    int di[4], dk[4];
    di[3] = (int)(r % p.dn[3]); r /= p.dn[3];
    di[2] = (int)(r % p.dn[2]); r /= p.dn[2];
    di[1] = (int)(r % p.dn[1]); r /= p.dn[1];
    di[0] = (int)(r % p.dn[0]); r /= p.dn[0];
    dk[2] = (int)(r % nk); r /= nk;
    dk[1] = (int)(r % nk); r /= nk;
    dk[0] = (int)r;
    dk[3] = kmod(dk[0] + dk[1] - dk[2], nk);
    const long long od = lay_off(p.dkind, nk, p.dn, dk[0], dk[1], dk[2], di[0], di[1], di[2], di[3]);
    const long long os = lay_off(p.skind, p.snk, p.sn, dk[p.pi[0]], dk[p.pi[1]], dk[p.pi[2]], di[p.pi[0]],
                                 di[p.pi[1]], di[p.pi[2]], di[p.pi[3]]);
    const double2 s = S[os];
    double2 d = p.store ? make_double2(0.0, 0.0) : D[od];
    d.x += p.ar * s.x - p.ai * s.y;
    d.y += p.ar * s.y + p.ai * s.x;
    D[od] = d;
  }
}

// Orbital-index strides of a layout at fixed momenta (every layout is affine in its four
// orbital indices once k1, k2, k3 are fixed; see lay_off).
__host__ __device__ inline void lay_strides(int kind, int nk, const int* n, long long* s) {
  const long long n0 = n[0], n1 = n[1], n2 = n[2], n3 = n[3];
  if (kind == 0) {  // K3
    s[0] = n1 * n2 * n3; s[1] = n2 * n3; s[2] = n3; s[3] = 1;
  } else if (kind == 1) {  // PP: cols = nk n2 n3
    const long long cols = (long long)nk * n2 * n3;
    s[0] = n1 * cols; s[1] = cols; s[2] = n3; s[3] = 1;
  } else if (kind == 2) {  // PH: cols = nk n3 n1
    const long long cols = (long long)nk * n3 * n1;
    s[0] = n2 * cols; s[1] = 1; s[2] = cols; s[3] = n1;
  } else {  // CH
    s[0] = n2 * n1 * n3; s[1] = n3; s[2] = n1 * n3; s[3] = 1;
  }
}

constexpr int SLAB_MAX = 64;  // largest orbital extent of a slab dimension

struct SlabArgs {
  PermArgs p;
  int dx, dy;               // destination orbital slots of the slab: dx has stride 1 in the destination
  int o0, o1;               // the other two destination orbital slots (outer)
  long long dsx, dsy;       // destination strides of the slab slots
  long long ssx, ssy;       // source strides of the slab slots
  long long nouter;         // nk^3 * n[o0] * n[o1]
};

// One CTA handles whole slabs: the (dy, dx) plane of the destination at fixed momenta and fixed
// outer orbital indices.  Source elements are read along the source's unit-stride direction
// into shared memory, destination elements written along dx; both global sides coalesce.
__global__ void __launch_bounds__(256) perm_slab_kernel(SlabArgs a) {
  extern __shared__ double2 slab[];  // [ny][nx + 1]
  const PermArgs& p = a.p;
  const long long rhs = blockIdx.y;
  const double2* S = p.S + rhs * p.sS;
  double2* D = p.D + rhs * p.sD;
  const int nk = p.dnk;
  const int nx = p.dn[a.dx], ny = p.dn[a.dy];
  const int pitch = nx + 1;
  const int nel = nx * ny;
  // source slot of each destination slot
  int inv[4];
  for (int s = 0; s < 4; ++s) inv[p.pi[s]] = s;
  const bool src_x_fast = a.ssx <= a.ssy;  // read the source along its faster slab direction
  for (long long ob = blockIdx.x; ob < a.nouter; ob += gridDim.x) {
    long long r = ob;
    int di[4] = {0, 0, 0, 0}, dk[4];
    di[a.o1] = (int)(r % p.dn[a.o1]); r /= p.dn[a.o1];
    di[a.o0] = (int)(r % p.dn[a.o0]); r /= p.dn[a.o0];
    dk[2] = (int)(r % nk); r /= nk;
    dk[1] = (int)(r % nk); r /= nk;
    dk[0] = (int)r;
    dk[3] = kmod(dk[0] + dk[1] - dk[2], nk);
    const long long dbase = lay_off(p.dkind, nk, p.dn, dk[0], dk[1], dk[2], di[0], di[1], di[2], di[3]);
    const long long sbase = lay_off(p.skind, p.snk, p.sn, dk[p.pi[0]], dk[p.pi[1]], dk[p.pi[2]], di[p.pi[0]],
                                    di[p.pi[1]], di[p.pi[2]], di[p.pi[3]]);
    (void)inv;
    __syncthreads();  // the previous slab's writes have read the shared tile
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
      int x, y;
      if (src_x_fast) {
        x = e % nx;
        y = e / nx;
      } else {
        y = e % ny;
        x = e / ny;
      }
      slab[y * pitch + x] = S[sbase + x * a.ssx + y * a.ssy];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
      const int x = e % nx, y = e / nx;
      const double2 s = slab[y * pitch + x];
      double2* dp = D + dbase + x * a.dsx + y * a.dsy;
      double2 d = p.store ? make_double2(0.0, 0.0) : *dp;
      d.x += p.ar * s.x - p.ai * s.y;
      d.y += p.ar * s.y + p.ai * s.x;
      *dp = d;
    }
  }
}

cudaError_t launch_perm_f64(const PermArgs& p, int nrhs, cudaStream_t st) {
  if (p.total <= 0) return cudaSuccess;
  // slab path: destination slot dx with unit stride, dy = the destination slot whose source
  // slot has unit stride (or the next-fastest destination slot when that is dx itself)
  long long ds[4], ss[4];
  lay_strides(p.dkind, p.dnk, p.dn, ds);
  lay_strides(p.skind, p.snk, p.sn, ss);
  int dx = 0;
  for (int s = 0; s < 4; ++s)
    if (ds[s] == 1) dx = s;
  int sfast = 0;
  for (int s = 0; s < 4; ++s)
    if (ss[s] == 1) sfast = s;
  int dy = p.pi[sfast];
  if (dy == dx) {
    dy = -1;
    for (int s = 0; s < 4; ++s)
      if (s != dx && (dy < 0 || ds[s] < ds[dy])) dy = s;
  }
  const bool slab_ok = p.dnk == p.snk && p.dn[dx] <= SLAB_MAX && p.dn[dy] <= SLAB_MAX && p.dn[dx] >= 1 &&
                       p.dn[dy] >= 1;
  if (slab_ok) {
    SlabArgs a;
    a.p = p;
    a.dx = dx;
    a.dy = dy;
    int oth[2], c = 0;
    for (int s = 0; s < 4; ++s)
      if (s != dx && s != dy) oth[c++] = s;
    a.o0 = oth[0];
    a.o1 = oth[1];
    a.dsx = ds[dx];
    a.dsy = ds[dy];
    int inv[4];
    for (int s = 0; s < 4; ++s) inv[p.pi[s]] = s;
    a.ssx = ss[inv[dx]];
    a.ssy = ss[inv[dy]];
    a.nouter = (long long)p.dnk * p.dnk * p.dnk * p.dn[a.o0] * p.dn[a.o1];
    const size_t smem = (size_t)p.dn[dy] * (p.dn[dx] + 1) * sizeof(double2);
    static const cudaError_t attr =  // thread-safe one-time setup: up to 64 x 65 complex
        cudaFuncSetAttribute(perm_slab_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(SLAB_MAX * (SLAB_MAX + 1) * sizeof(double2)));
    if (attr != cudaSuccess) return attr;
    long long blocks = a.nouter;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    dim3 grid((unsigned)blocks, (unsigned)nrhs);
    perm_slab_kernel<<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
  }
  long long blocks = (p.total + 255) / 256;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
  dim3 grid((unsigned)blocks, (unsigned)nrhs);
  perm_kernel<<<grid, 256, 0, st>>>(p);
  return cudaGetLastError();
}

__global__ void btrans_kernel(BTransArgs t) {
  const long long rhs = blockIdx.y;
  const double2* S = t.S + rhs * t.sS;
  double2* D = t.D + rhs * t.sD;
  const long long total = (long long)t.nb * t.R * t.C;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    // e indexes the destination [b][j][i]
    const int i = (int)(e % t.R);
    const long long r = e / t.R;
    const int j = (int)(r % t.C);
    const long long b = r / t.C;
    const double2 s = S[(b * t.R + i) * t.C + j];
    double2 d = D[e];
    d.x += t.ar * s.x - t.ai * s.y;
    d.y += t.ar * s.y + t.ai * s.x;
    D[e] = d;
  }
}

cudaError_t launch_btrans_f64(const BTransArgs& t, int nrhs, cudaStream_t st) {
  long long total = (long long)t.nb * t.R * t.C;
  if (total <= 0) return cudaSuccess;
  long long blocks = (total + 255) / 256;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
  dim3 grid((unsigned)blocks, (unsigned)nrhs);
  btrans_kernel<<<grid, 256, 0, st>>>(t);
  return cudaGetLastError();
}

__global__ void split_df_kernel(const double2* L, int nk, int Q, int o, int v, double scale, double2* Loo,
                                double2* Lov, double2* Lvo, double2* Lvv) {
  const int n = o + v;
  const long long total = (long long)nk * nk * Q * n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(e % n);
    const int p = (int)((e / n) % n);
    const long long kkQ = e / ((long long)n * n);  // (k1*nk + k2)*Q + Q
    double2 x = L[e];
    x.x *= scale;
    x.y *= scale;
    if (p < o && q < o) Loo[kkQ * o * o + p * o + q] = x;
    else if (p < o) Lov[kkQ * o * v + p * v + (q - o)] = x;
    else if (q < o) Lvo[kkQ * v * o + (p - o) * o + q] = x;
    else Lvv[kkQ * v * v + (long long)(p - o) * v + (q - o)] = x;
  }
}

cudaError_t launch_split_df(const double2* L, int nk, int Q, int o, int v, double scale, double2* Loo,
                            double2* Lov, double2* Lvo, double2* Lvv, cudaStream_t st) {
  long long total = (long long)nk * nk * Q * (o + v) * (o + v);
  long long blocks = (total + 255) / 256;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
  split_df_kernel<<<(unsigned)blocks, 256, 0, st>>>(L, nk, Q, o, v, scale, Loo, Lov, Lvo, Lvv);
  return cudaGetLastError();
}

}  // namespace lrcc
