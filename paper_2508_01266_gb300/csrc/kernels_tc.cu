// Tensor-core (tcgen05) version of the segmented batched complex GEMM, for the
// mixed-precision path: operands are read in FP64, rounded on the way into shared
// memory to TF32 (kind::tf32) or split into BF16 hi + lo parts (kind::f16, three
// MMAs hi*hi + hi*lo + lo*hi), accumulated in FP32 in tensor memory, and added to
// the FP64 destination.
//
// Complex arithmetic by real embedding: with A viewed as a real M x 2K matrix
// (re, im interleaved along K) and B expanded to the real 2N x 2K matrix
//   Bt[2n][2k] = Re b, Bt[2n][2k+1] = -Im b, Bt[2n+1][2k] = Im b, Bt[2n+1][2k+1] = Re b,
// the real product C = A Bt^T holds (Re c, Im c) interleaved along N.
//
// Tile: 128 complex rows x 64 complex columns (128 x 128 real accumulator in 128
// TMEM columns), 16 complex K per stage, two shared-memory stages: while the
// tensor core works on one stage all threads load and convert the next.  Shared
// memory operands use the no-swizzle K-major core-matrix layout (8 rows x 16 bytes
// per core matrix; LBO = 128 bytes between K-adjacent core matrices, SBO between
// 8-row groups).  Every mbarrier wait is bounded; on timeout the CTA records an
// error flag, waits (bounded) for its MMAs, releases its tensor memory and exits.
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace lrcc {

namespace {

constexpr int TC_BM = 128;          // complex rows per tile
constexpr int TC_BNC = 64;          // complex columns per tile
constexpr int TC_BKC = TC_BK;       // complex K per stage
constexpr int TC_BKR = 2 * TC_BKC;  // real K per stage
constexpr int TC_NR = 2 * TC_BNC;   // real accumulator columns
constexpr int TC_THREADS = 128;
constexpr long long TC_SPIN = 1LL << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // tcgen05 descriptor version; layout type 0 = no swizzle
  return d;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (long long it = 0; it < TC_SPIN; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// byte offset of element (row, kr) inside a K-major no-swizzle tile with BKR real K
template <int EB>
__device__ __forceinline__ int core_off(int row, int kr) {
  constexpr int T = 16 / EB;
  return ((row >> 3) * (TC_BKR / T) + kr / T) * 128 + (row & 7) * 16 + (kr % T) * EB;
}

}  // namespace

// PREC 1: TF32.  PREC 2: BF16x3.
template <int PREC>
__global__ void __launch_bounds__(TC_THREADS) tc_gemm_kernel(GemmArgs g, int* errflag) {
  constexpr int EB = PREC == 1 ? 4 : 2;
  constexpr int ABYTES = TC_BM * TC_BKR * EB;  // one operand plane
  constexpr int BBYTES = TC_NR * TC_BKR * EB;
  constexpr int NPL = PREC == 1 ? 1 : 2;       // planes per operand (hi, lo)
  constexpr int STAGE = NPL * (ABYTES + BBYTES);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base_sh;

  const int tpb = g.tiles_m * g.tiles_n;
  const int bid = blockIdx.x;
  const int per_batch = tpb * g.nsplit;
  const int batch = bid / per_batch;
  const int rem = bid - batch * per_batch;
  const int sp = rem / tpb;
  const int t = rem - sp * tpb;
  const int m0 = (t / g.tiles_n) * TC_BM;
  const int n0 = (t % g.tiles_n) * TC_BNC;
  const long long rhs = blockIdx.y;
  const double2* Ab = g.A + rhs * g.sA;
  const double2* Bb = g.B + rhs * g.sB;
  double2* Cb = g.C + rhs * g.sC;
  const int tid = threadIdx.x;
  const int M = g.M, N = g.N, K = g.K;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(TC_NR));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_sh;

  constexpr uint32_t LBO = 128;
  constexpr uint32_t SBO = (TC_BKR / (16 / EB)) * 128;
  constexpr int KSTEP = PREC == 1 ? 8 : 16;  // real K per MMA
  const uint32_t fmt = PREC == 1 ? 2u : 1u;  // TF32 : BF16
  const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(TC_NR >> 3) << 17) |
                         ((uint32_t)(TC_BM >> 4) << 24);

  // (segment, K tile) iteration space of the batch entry, segment-major; this CTA takes
  // its split's contiguous range
  const int s0 = g.sbeg[batch], s1 = g.sbeg[batch + 1];
  const int nkt = (K + TC_BKC - 1) / TC_BKC;
  const long long all = (long long)(s1 - s0) * nkt;
  const long long lo = all * sp / g.nsplit, hi = all * (sp + 1) / g.nsplit;
  const int total = (int)(hi - lo);
  bool ok = true;
  int step = 0;
  int s = s0 + (int)(lo / nkt), kt = (int)(lo % nkt);
  for (; step < total && ok; ++step) {
    const double2* Ap = Ab + g.aoff[s];
    const double2* Bp = Bb + g.boff[s];
    {
      const int buf = step & 1;
      unsigned char* st = smem + buf * STAGE;
      if (step >= 2) {
        if (!mbar_wait(smem_u32(&mbar[buf]), ((step - 2) >> 1) & 1)) {
          ok = false;
          break;
        }
      }
      const int k0 = kt * TC_BKC;
      // A tile: 128 rows x 16 complex K
      for (int idx = tid; idx < TC_BM * TC_BKC; idx += TC_THREADS) {
        int m, kc;
        if (!g.ta) {
          kc = idx % TC_BKC;
          m = idx / TC_BKC;
        } else {
          m = idx % TC_BM;
          kc = idx / TC_BM;
        }
        const int gm = m0 + m, gk = k0 + kc;
        double2 val = make_double2(0.0, 0.0);
        if (gm < M && gk < K) val = g.ta ? Ap[(long long)gk * g.lda + gm] : Ap[(long long)gm * g.lda + gk];
        const float vr = (float)val.x, vi = (float)val.y;
        if (PREC == 1) {
          *(float2*)(st + core_off<4>(m, 2 * kc)) = make_float2(vr, vi);
        } else {
          const __nv_bfloat16 hr = __float2bfloat16_rn(vr), hi = __float2bfloat16_rn(vi);
          const __nv_bfloat16 lr = __float2bfloat16_rn(vr - __bfloat162float(hr));
          const __nv_bfloat16 li = __float2bfloat16_rn(vi - __bfloat162float(hi));
          const int off = core_off<2>(m, 2 * kc);
          *(__nv_bfloat162*)(st + off) = __halves2bfloat162(hr, hi);
          *(__nv_bfloat162*)(st + ABYTES + off) = __halves2bfloat162(lr, li);
        }
      }
      // B tile: 64 complex columns x 16 complex K, expanded to 128 x 32 real
      unsigned char* sb = st + NPL * ABYTES;
      for (int idx = tid; idx < TC_BNC * TC_BKC; idx += TC_THREADS) {
        int n, kc;
        if (g.tb) {
          kc = idx % TC_BKC;
          n = idx / TC_BKC;
        } else {
          n = idx % TC_BNC;
          kc = idx / TC_BNC;
        }
        const int gn = n0 + n, gk = k0 + kc;
        double2 val = make_double2(0.0, 0.0);
        if (gn < N && gk < K) val = g.tb ? Bp[(long long)gn * g.ldb + gk] : Bp[(long long)gk * g.ldb + gn];
        const float br = (float)val.x, bi = (float)val.y;
        if (PREC == 1) {
          *(float2*)(sb + core_off<4>(2 * n, 2 * kc)) = make_float2(br, -bi);
          *(float2*)(sb + core_off<4>(2 * n + 1, 2 * kc)) = make_float2(bi, br);
        } else {
          const __nv_bfloat16 hr = __float2bfloat16_rn(br), hi = __float2bfloat16_rn(bi);
          const __nv_bfloat16 lr = __float2bfloat16_rn(br - __bfloat162float(hr));
          const __nv_bfloat16 li = __float2bfloat16_rn(bi - __bfloat162float(hi));
          const int o0 = core_off<2>(2 * n, 2 * kc), o1 = core_off<2>(2 * n + 1, 2 * kc);
          *(__nv_bfloat162*)(sb + o0) = __halves2bfloat162(hr, __hneg(hi));
          *(__nv_bfloat162*)(sb + o1) = __halves2bfloat162(hi, hr);
          *(__nv_bfloat162*)(sb + BBYTES + o0) = __halves2bfloat162(lr, __hneg(li));
          *(__nv_bfloat162*)(sb + BBYTES + o1) = __halves2bfloat162(li, lr);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = smem_u32(st), b0 = smem_u32(sb);
#pragma unroll
        for (int ks = 0; ks < TC_BKR / KSTEP; ++ks) {
          const uint32_t koff = ks * (KSTEP / (16 / EB)) * LBO;
          const uint64_t ahi = sdesc(a0 + koff, LBO, SBO), bhi = sdesc(b0 + koff, LBO, SBO);
          const uint32_t acc0 = (step > 0 || ks > 0) ? 1u : 0u;
          if (PREC == 1) {
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ahi), "l"(bhi), "r"(idesc), "r"(acc0));
          } else {
            const uint64_t alo = sdesc(a0 + ABYTES + koff, LBO, SBO), blo = sdesc(b0 + BBYTES + koff, LBO, SBO);
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ahi), "l"(bhi), "r"(idesc), "r"(acc0));
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, 1, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %4, %5, %3, p;\n}\n" ::"r"(tmem),
                "l"(ahi), "l"(blo), "r"(idesc), "l"(alo), "l"(bhi));
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&mbar[buf]))
                     : "memory");
      }
    }
    if (++kt == nkt) {
      kt = 0;
      ++s;
    }
  }
  // wait for the last commit (it tracks every MMA issued before it)
  if (ok && total > 0) ok = mbar_wait(smem_u32(&mbar[(total - 1) & 1]), ((total - 1) >> 1) & 1);
  if (!ok) {
    if (tid == 0) atomicExch(errflag, 1);
    // drain: wait (bounded) for whatever MMAs were committed before releasing TMEM
    if (step > 0) mbar_wait(smem_u32(&mbar[(step - 1) & 1]), ((step - 1) >> 1) & 1);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  // destination row length of the partials: the original N (= M of a swapped launch)
  const int Nrow = g.swap ? M : N;
  if (ok && g.nsplit > 1 && total == 0) {  // an empty split still owns its partial tile
    const int m = m0 + tid;
    if (m < M) {
      double2* Pp = g.part + ((rhs * g.nbatch + batch) * g.nsplit + sp) * (long long)M * N;
      for (int n = n0; n < n0 + TC_BNC && n < N; ++n)
        Pp[g.swap ? (long long)n * Nrow + m : (long long)m * Nrow + n] = make_double2(0.0, 0.0);
    }
  }
  if (ok && total > 0) {
    const int warp = tid >> 5, lane = tid & 31;
    const int m = m0 + warp * 32 + lane;
    double2* Cp = Cb + g.coff[batch];
    double2* Pp = g.nsplit > 1 ? g.part + ((rhs * g.nbatch + batch) * g.nsplit + sp) * (long long)M * N : nullptr;
#pragma unroll 1
    for (int c0 = 0; c0 < TC_NR; c0 += 16) {
      uint32_t r[16];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (m < M && !Pp && g.epi == 0) {
        // all loads first, then the stores (no load waits on a store)
        const int cnt = min(8, N - (n0 + c0 / 2));
        double2 cv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (j >= cnt) break;
          const int n = n0 + c0 / 2 + j;
          const int mo = g.swap ? n : m, no = g.swap ? m : n;  // element of the original C
          cv[j] = g.store ? make_double2(0.0, 0.0) : Cp[(long long)mo * g.ldc + no];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (j >= cnt) break;
          const int n = n0 + c0 / 2 + j;
          const int mo = g.swap ? n : m, no = g.swap ? m : n;
          const double ar = __uint_as_float(r[2 * j]), ai = __uint_as_float(r[2 * j + 1]);
          cv[j].x += g.ar * ar - g.ai * ai;
          cv[j].y += g.ar * ai + g.ai * ar;
          Cp[(long long)mo * g.ldc + no] = cv[j];
        }
      } else if (m < M) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int n = n0 + c0 / 2 + j;
          if (n >= N) break;
          const double ar = __uint_as_float(r[2 * j]), ai = __uint_as_float(r[2 * j + 1]);
          const int mo = g.swap ? n : m, no = g.swap ? m : n;  // element of the original C
          if (Pp) {  // raw partial; alpha and the epilogue come in the reduction
            Pp[(long long)mo * Nrow + no] = make_double2(ar, ai);
            continue;
          }
          const double vr = g.ar * ar - g.ai * ai, vi = g.ar * ai + g.ai * ar;
          {
            const int a = mo / g.ep2, c = mo - a * g.ep2;
            const int b = no / g.ep3, d = no - b * g.ep3;
            Cp[(((long long)a * g.ep1 + b) * g.ep2 + c) * g.ep3 + d] = make_double2(vr, vi);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_NR));
}

// Bounded-wait self test: one thread waits on an mbarrier that nothing arrives at, gives
// up after `polls` polls and records the timeout in the error flag, exactly as the GEMM
// kernels do when a copy or an MMA never completes (no copies, MMAs or tensor memory
// are involved, so giving up leaves nothing in flight).
__global__ void wait_selftest_kernel(long long polls, int* errflag) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
  asm volatile("fence.mbarrier_init.release.cluster;");
  uint32_t done = 0;
  for (long long it = 0; it < polls && !done; ++it)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(&bar)), "r"(0u)
        : "memory");
  if (!done) atomicExch(errflag, 1);
}

cudaError_t launch_wait_selftest(long long polls, int* errflag, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(polls, errflag);
  return cudaGetLastError();
}

size_t tc_smem_bytes(int prec) {
  const int EB = prec == 1 ? 4 : 2;
  const int NPL = prec == 1 ? 1 : 2;
  return (size_t)2 * NPL * (TC_BM * TC_BKR * EB + TC_NR * TC_BKR * EB) + 1024;
}

cudaError_t launch_gemm_tc(const GemmArgs& g0, int prec, int nrhs, int* errflag, cudaStream_t st) {
  GemmArgs g = g0;
  g.tiles_m = (g.M + TC_BM - 1) / TC_BM;
  g.tiles_n = (g.N + TC_BNC - 1) / TC_BNC;
  if (g.nsplit < 1 || (g.nsplit > 1 && !g.part)) return cudaErrorInvalidValue;
  long long nblk = (long long)g.tiles_m * g.tiles_n * g.nbatch * g.nsplit;
  if (nblk <= 0) return cudaSuccess;
  if (nblk > 2147483647LL || nrhs > 65535) return cudaErrorInvalidConfiguration;
  const size_t sm = tc_smem_bytes(prec);
  dim3 grid((unsigned)nblk, (unsigned)nrhs);
  if (prec == 1) {
    static const cudaError_t attr =  // thread-safe one-time setup
        cudaFuncSetAttribute(tc_gemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (attr != cudaSuccess) return attr;
    tc_gemm_kernel<1><<<grid, TC_THREADS, sm, st>>>(g, errflag);
  } else {
    static const cudaError_t attr =  // thread-safe one-time setup
        cudaFuncSetAttribute(tc_gemm_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (attr != cudaSuccess) return attr;
    tc_gemm_kernel<2><<<grid, TC_THREADS, sm, st>>>(g, errflag);
  }
  return cudaGetLastError();
}

}  // namespace lrcc
