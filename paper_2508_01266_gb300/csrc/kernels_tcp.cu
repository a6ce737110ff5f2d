// Packed-operand tensor-core GEMM (tcgen05, TF32 or BF16x3) for the large GEMMs of
// the mixed-precision path, and the kernel that packs complex FP64 operands.
//
// Packed operand: a complex R x K matrix (any offset / leading dimension / transpose)
// stored as MMA-ready tiles, tile (rt, kt) at byte offset (rt * nkt + kt) * tile bytes,
// each tile in the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core
// matrix, K-adjacent cores 128 bytes apart).  Complex numbers by real embedding:
//   mode A (left operand):  real row r, real K 2k + {0,1} = (Re, Im) of a[r][k];
//   mode B (right operand, stored K-major): real rows 2n, 2n+1 and real K 2k, 2k+1 hold
//   [[Re, -Im], [Im, Re]] of b[k][n], so that C_real = A_real . B_real^T carries
//   (Re c, Im c) interleaved along N.
// TF32 tiles hold fp32 values (4 bytes, 32 real K per 128-byte row); BF16x3 tiles hold
// a bf16 "hi" plane followed by a bf16 "lo" plane (x - hi), 32 real K per 64-byte row.
//
// GEMM: one CTA per 128 x 128 complex output tile (128 x 256 real accumulator in 256
// TMEM columns); warp 0 streams A and B tiles with cp.async.bulk into a 4-stage ring
// (mbarrier transaction counts), warp 1 issues tcgen05.mma (TF32: 4 per stage; BF16x3:
// hi*hi + hi*lo + lo*hi per K=16 step) and releases stages with tcgen05.commit, warps
// 2-5 drain the accumulator (tcgen05.ld) and add alpha * C into the FP64 destination.
// All waits are bounded; on timeout the CTA sets the error flag, drains its own
// outstanding copies (bounded), releases tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "kernels.cuh"

namespace lrcc {

namespace {

constexpr int P_BM = 128;   // real rows of an A tile (= complex rows)
constexpr int P_BNR = 256;  // real rows of a B tile (= 128 complex columns)
constexpr int P_BKR = 32;   // real K per stage
constexpr int P_STAGES = 4;
constexpr int P_ATILE = P_BM * 128;   // bytes (TF32: 128 x 32 x 4; BF16x3: 2 planes x 128 x 32 x 2)
constexpr int P_BTILE = P_BNR * 128;
constexpr int P_THREADS = 192;
constexpr long long P_SPIN = 1LL << 26;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ bool wait_parity(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < P_SPIN; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// byte offset of real element (row, kr) in a tile (PREC 1: fp32; PREC 2: one bf16 plane)
template <int PREC>
__device__ __forceinline__ int tile_off(int row, int kr) {
  constexpr int EB = PREC == 1 ? 4 : 2, T = 16 / EB;
  return ((row >> 3) * (P_BKR / T) + kr / T) * 128 + (row & 7) * 16 + (kr % T) * EB;
}

}  // namespace

// --------------------------------------------------------------------------------
// packing
// --------------------------------------------------------------------------------
// Every work item writes one complex element (or its zero padding) of one packed
// operand: mode A -> 2 reals, mode B -> a 2 x 2 real block.
template <int PREC>
__global__ void pack_kernel(PackArgs p) {
  const int rows_real = p.mode == 0 ? p.R : 2 * p.R;
  const int tr = p.mode == 0 ? P_BM : P_BNR;
  const int nrt = (rows_real + tr - 1) / tr;
  const int nkt = (2 * p.K + P_BKR - 1) / P_BKR;
  const int Rp = p.mode == 0 ? nrt * tr : nrt * tr / 2;  // padded complex rows
  const int Kp = nkt * P_BKR / 2;                         // padded complex K
  const long long per = (long long)Rp * Kp;
  const long long total = per * p.count;
  const long long rhs = blockIdx.y;
  const double2* src = p.src + rhs * p.sS;
  unsigned char* dst = p.dst + rhs * p.sD;
  const long long tile_bytes = (long long)tr * 128;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int li = (int)(e / per);
    const long long w = e - (long long)li * per;
    int r, k;
    if (p.trans) {  // consecutive threads walk rows (contiguous in the source)
      r = (int)(w % Rp);
      k = (int)(w / Rp);
    } else {
      k = (int)(w % Kp);
      r = (int)(w / Kp);
    }
    double2 v = make_double2(0.0, 0.0);
    if (r < p.R && k < p.K) {
      const long long off = p.offs[li] + (p.trans ? (long long)k * p.ld + r : (long long)r * p.ld + k);
      v = src[off];
    }
    unsigned char* base = dst + (long long)li * p.packed_bytes;
    const int kr = 2 * k;
    const int kt = kr / P_BKR, kk = kr % P_BKR;
    if (p.mode == 0) {
      const int rt = r / tr, rr = r % tr;
      unsigned char* tile = base + ((long long)rt * nkt + kt) * tile_bytes;
      const float xr = (float)v.x, xi = (float)v.y;
      if (PREC == 1) {
        *(float2*)(tile + tile_off<1>(rr, kk)) = make_float2(xr, xi);
      } else {
        const __nv_bfloat16 hr = __float2bfloat16_rn(xr), hi = __float2bfloat16_rn(xi);
        const __nv_bfloat16 lr = __float2bfloat16_rn(xr - __bfloat162float(hr));
        const __nv_bfloat16 li2 = __float2bfloat16_rn(xi - __bfloat162float(hi));
        const int o = tile_off<2>(rr, kk);
        *(__nv_bfloat162*)(tile + o) = __halves2bfloat162(hr, hi);
        *(__nv_bfloat162*)(tile + tr * 64 + o) = __halves2bfloat162(lr, li2);
      }
    } else {
      const int r0 = 2 * r;
      const int rt = r0 / tr, rr = r0 % tr;  // rows 2r and 2r+1 share a tile (tr even)
      unsigned char* tile = base + ((long long)rt * nkt + kt) * tile_bytes;
      const float br = (float)v.x, bi = (float)v.y;
      if (PREC == 1) {
        *(float2*)(tile + tile_off<1>(rr, kk)) = make_float2(br, -bi);
        *(float2*)(tile + tile_off<1>(rr + 1, kk)) = make_float2(bi, br);
      } else {
        const __nv_bfloat16 hr = __float2bfloat16_rn(br), hi = __float2bfloat16_rn(bi);
        const __nv_bfloat16 lr = __float2bfloat16_rn(br - __bfloat162float(hr));
        const __nv_bfloat16 li2 = __float2bfloat16_rn(bi - __bfloat162float(hi));
        const int o0 = tile_off<2>(rr, kk), o1 = tile_off<2>(rr + 1, kk);
        *(__nv_bfloat162*)(tile + o0) = __halves2bfloat162(hr, __hneg(hi));
        *(__nv_bfloat162*)(tile + o1) = __halves2bfloat162(hi, hr);
        *(__nv_bfloat162*)(tile + tr * 64 + o0) = __halves2bfloat162(lr, __hneg(li2));
        *(__nv_bfloat162*)(tile + tr * 64 + o1) = __halves2bfloat162(li2, lr);
      }
    }
  }
}

long long packed_bytes(int mode, int R, int K) {
  const int rows_real = mode == 0 ? R : 2 * R;
  const int tr = mode == 0 ? P_BM : P_BNR;
  const long long nrt = (rows_real + tr - 1) / tr;
  const long long nkt = (2LL * K + P_BKR - 1) / P_BKR;
  return nrt * nkt * tr * 128;
}

cudaError_t launch_pack(const PackArgs& p, int prec, int nrhs, cudaStream_t st) {
  const int rows_real = p.mode == 0 ? p.R : 2 * p.R;
  const int tr = p.mode == 0 ? P_BM : P_BNR;
  const long long nrt = (rows_real + tr - 1) / tr;
  const long long nkt = (2LL * p.K + P_BKR - 1) / P_BKR;
  const long long per = (p.mode == 0 ? nrt * tr : nrt * tr / 2) * (nkt * P_BKR / 2);
  const long long total = per * p.count;
  if (total <= 0) return cudaSuccess;
  long long blocks = (total + 255) / 256;
  if (blocks > 152LL * 32) blocks = 152LL * 32;
  dim3 grid((unsigned)blocks, (unsigned)nrhs);
  if (prec == 1) pack_kernel<1><<<grid, 256, 0, st>>>(p);
  else pack_kernel<2><<<grid, 256, 0, st>>>(p);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------------
// packed GEMM
// --------------------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(P_THREADS, 1) tcp_gemm_kernel(PGemmArgs g, int* errflag) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[P_STAGES], empty[P_STAGES], accf;
  __shared__ uint32_t tmem_sh;
  __shared__ int fail_sh;

  const int tpb = g.tiles_m * g.tiles_n;
  const int batch = blockIdx.x / tpb;
  const int t = blockIdx.x - batch * tpb;
  const int mt = t / g.tiles_n, nt = t % g.tiles_n;
  const long long rhs = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s0 = g.sbeg[batch], s1 = g.sbeg[batch + 1];
  const int nkt = g.nkt;
  const int total = (s1 - s0) * nkt;

  if (threadIdx.x == 0) {
    for (int s = 0; s < P_STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&empty[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&accf)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    fail_sh = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_sh)),
                 "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_sh;

  if (warp == 0 && lane == 0 && total > 0) {
    // producer
    const unsigned char* Ab = g.A + rhs * g.sA;
    const unsigned char* Bb = g.B + rhs * g.sB;
    int issued = 0;
    bool ok = true;
    for (int i = 0; i < total && ok; ++i) {
      const int s = i % P_STAGES;
      if (i >= P_STAGES && !wait_parity(su32(&empty[s]), ((i / P_STAGES) - 1) & 1)) {
        ok = false;
        break;
      }
      const int seg = s0 + i / nkt, kt = i % nkt;
      const unsigned char* at = Ab + (long long)g.ia[seg] * g.abytes + ((long long)mt * nkt + kt) * P_ATILE;
      const unsigned char* bt = Bb + (long long)g.ib[seg] * g.bbytes + ((long long)nt * nkt + kt) * P_BTILE;
      unsigned char* sa = smem + s * (P_ATILE + P_BTILE);
      unsigned char* sb = sa + P_ATILE;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&full[s])),
                   "r"(P_ATILE + P_BTILE)
                   : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(sa)),
          "l"(at), "r"(P_ATILE), "r"(su32(&full[s]))
          : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(sb)),
          "l"(bt), "r"(P_BTILE), "r"(su32(&full[s]))
          : "memory");
      ++issued;
    }
    if (!ok) {
      atomicExch(&fail_sh, 1);
      // drain the copies in flight before the CTA releases its shared memory
      for (int i = (issued > P_STAGES ? issued - P_STAGES : 0); i < issued; ++i)
        wait_parity(su32(&full[i % P_STAGES]), (i / P_STAGES) & 1);
    }
  } else if (warp == 1 && lane == 0 && total > 0) {
    // MMA issuer
    constexpr uint32_t LBO = 128;
    constexpr uint32_t SBO_A = (P_BKR / (PREC == 1 ? 4 : 8)) * 128;
    const uint32_t fmt = PREC == 1 ? 2u : 1u;
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(P_BNR >> 3) << 17) |
                           ((uint32_t)(P_BM >> 4) << 24);
    bool ok = true;
    for (int i = 0; i < total; ++i) {
      const int s = i % P_STAGES;
      if (!wait_parity(su32(&full[s]), (i / P_STAGES) & 1)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = su32(smem + s * (P_ATILE + P_BTILE)), b0 = a0 + P_ATILE;
      if (PREC == 1) {
#pragma unroll
        for (int ks = 0; ks < P_BKR / 8; ++ks) {
          const uint32_t ko = ks * 2 * LBO;
          const uint64_t ad = sdesc(a0 + ko, LBO, SBO_A), bd = sdesc(b0 + ko, LBO, SBO_A);
          const uint32_t acc = (i > 0 || ks > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
      } else {
#pragma unroll
        for (int ks = 0; ks < P_BKR / 16; ++ks) {
          const uint32_t ko = ks * 2 * LBO;
          const uint64_t ahi = sdesc(a0 + ko, LBO, SBO_A), bhi = sdesc(b0 + ko, LBO, SBO_A);
          const uint64_t alo = sdesc(a0 + P_BM * 64 + ko, LBO, SBO_A), blo = sdesc(b0 + P_BNR * 64 + ko, LBO, SBO_A);
          const uint32_t acc = (i > 0 || ks > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p, q;\n setp.ne.b32 p, %6, 0;\n setp.ne.b32 q, 1, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %4, %3, q;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %5, %2, %3, q;\n}\n" ::"r"(tmem),
              "l"(ahi), "l"(bhi), "r"(idesc), "l"(blo), "l"(alo), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       su32(&empty[s]))
                   : "memory");
    }
    if (ok) {
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&accf))
                   : "memory");
    } else {
      atomicExch(&fail_sh, 1);
    }
  } else if (warp >= 2 && total > 0) {
    // epilogue: warp w reads TMEM lanes 32*(w%4) .. +31
    const int q = warp & 3;
    const bool ok = wait_parity(su32(&accf), 0);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!ok) {
      atomicExch(&fail_sh, 1);
    } else {
      const int m = mt * P_BM + q * 32 + lane;
      double2* Cp = g.C + rhs * g.sC + g.coff[batch];
#pragma unroll 1
      for (int c0 = 0; c0 < P_BNR; c0 += 16) {
        uint32_t r[16];
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (m < g.M && g.epi == 0) {
          const int nb = nt * (P_BNR / 2) + c0 / 2;
          const int cnt = min(8, g.N - nb);
          double2* cp = Cp + (long long)m * g.ldc + nb;
          double2 cv[8];
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (j < cnt) cv[j] = g.store ? make_double2(0.0, 0.0) : cp[j];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            if (j >= cnt) break;
            const double ar = __uint_as_float(r[2 * j]), ai = __uint_as_float(r[2 * j + 1]);
            cv[j].x += g.ar * ar - g.ai * ai;
            cv[j].y += g.ar * ai + g.ai * ar;
            cp[j] = cv[j];
          }
        } else if (m < g.M) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int n = nt * (P_BNR / 2) + c0 / 2 + j;
            if (n >= g.N) break;
            const double ar = __uint_as_float(r[2 * j]), ai = __uint_as_float(r[2 * j + 1]);
            const double vr = g.ar * ar - g.ai * ai, vi = g.ar * ai + g.ai * ar;
            {
              const int a = m / g.ep2, c = m - a * g.ep2;
              const int b = n / g.ep3, d = n - b * g.ep3;
              Cp[(((long long)a * g.ep1 + b) * g.ep2 + c) * g.ep3 + d] = make_double2(vr, vi);
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (threadIdx.x == 0 && fail_sh) atomicExch(errflag, 1);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

size_t tcp_smem_bytes() { return (size_t)P_STAGES * (P_ATILE + P_BTILE) + 1024; }

cudaError_t launch_gemm_tcp(const PGemmArgs& g0, int prec, int nrhs, int* errflag, cudaStream_t st) {
  PGemmArgs g = g0;
  g.tiles_m = (g.M + P_BM - 1) / P_BM;
  g.tiles_n = (g.N + P_BNR / 2 - 1) / (P_BNR / 2);
  const long long nblk = (long long)g.tiles_m * g.tiles_n * g.nbatch;
  if (nblk <= 0) return cudaSuccess;
  if (nblk > 2147483647LL || nrhs > 65535) return cudaErrorInvalidConfiguration;
  const size_t sm = tcp_smem_bytes();
  dim3 grid((unsigned)nblk, (unsigned)nrhs);
  if (prec == 1) {
    static const cudaError_t attr =  // thread-safe one-time setup
        cudaFuncSetAttribute(tcp_gemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (attr != cudaSuccess) return attr;
    tcp_gemm_kernel<1><<<grid, P_THREADS, sm, st>>>(g, errflag);
  } else {
    static const cudaError_t attr =  // thread-safe one-time setup
        cudaFuncSetAttribute(tcp_gemm_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (attr != cudaSuccess) return attr;
    tcp_gemm_kernel<2><<<grid, P_THREADS, sm, st>>>(g, errflag);
  }
  return cudaGetLastError();
}


// --------------------------------------------------------------------------------
// persistent packed GEMM: one CTA per SM loops over (batch, n tile, m tile, rhs) tiles
// (right-hand sides fastest, so CTAs running together share B tiles in L2); two TMEM
// accumulators (2 x 256 columns) let the epilogue of one tile overlap the MMAs of the
// next.  Barriers: full/empty per smem stage (producer <-> MMA), accf[b] (MMA -> epilogue:
// accumulator b complete), acce[b] (epilogue -> MMA: accumulator b drained), done (all
// MMAs of the CTA complete, before TMEM is released).  Every wait is bounded and also
// gives up when another role has failed; a failing CTA drains its copies and MMAs first.
// --------------------------------------------------------------------------------
namespace {

__device__ __forceinline__ bool wait_or_fail(uint32_t bar, uint32_t parity, volatile int* fail) {
  for (long long it = 0; it < P_SPIN; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255) == 255 && *fail) return false;
  }
  return false;
}

// 16 consecutive 32-bit TMEM columns of this warp's 32 lanes (one row per lane)
__device__ __forceinline__ void tmem_ld16(uint32_t ta, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
}

__device__ __forceinline__ void decode_tile(const PGemmArgs& g, long long tile, int& rhs, int& batch, int& mt,
                                            int& nt) {
  rhs = (int)(tile % g.nrhs);
  long long r = tile / g.nrhs;
  mt = (int)(r % g.tiles_m);
  r /= g.tiles_m;
  nt = (int)(r % g.tiles_n);
  batch = (int)(r / g.tiles_n);
}

}  // namespace

template <int PREC>
__global__ void __launch_bounds__(P_THREADS, 1) tcp_gemm_persistent(PGemmArgs g, int* errflag) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[P_STAGES], empty[P_STAGES], accf[2], acce[2], donebar;
  __shared__ uint32_t tmem_sh;
  __shared__ volatile int fail_sh;

  const long long ntiles = (long long)g.tiles_m * g.tiles_n * g.nbatch * g.nrhs;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkt = g.nkt;

  if (threadIdx.x == 0) {
    for (int s = 0; s < P_STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&empty[s])));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&accf[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(su32(&acce[b])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&donebar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    fail_sh = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_sh)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_sh;

  if (warp == 0 && lane == 0) {
    // producer
    long long it = 0;
    bool ok = true;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      int rhs, batch, mt, nt;
      decode_tile(g, tile, rhs, batch, mt, nt);
      const int s0 = g.sbeg[batch], total = (g.sbeg[batch + 1] - s0) * nkt;
      const unsigned char* Ab = g.A + rhs * g.sA;
      const unsigned char* Bb = g.B + rhs * g.sB;
      // the chunks of a tile are consecutive items of this CTA: the k-steps in order
      for (int i = 0; i < total; ++i) {
        const int s = (int)(it % P_STAGES);
        if (it >= P_STAGES && !wait_or_fail(su32(&empty[s]), (uint32_t)(((it / P_STAGES) - 1) & 1), &fail_sh)) {
          ok = false;
          break;
        }
        const int seg = s0 + i / nkt, kt = i % nkt;
        const unsigned char* at = Ab + (long long)g.ia[seg] * g.abytes + ((long long)mt * nkt + kt) * P_ATILE;
        const unsigned char* bt = Bb + (long long)g.ib[seg] * g.bbytes + ((long long)nt * nkt + kt) * P_BTILE;
        unsigned char* sa = smem + s * (P_ATILE + P_BTILE);
        unsigned char* sb = sa + P_ATILE;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&full[s])),
                     "r"(P_ATILE + P_BTILE)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                su32(sa)),
            "l"(at), "r"(P_ATILE), "r"(su32(&full[s]))
            : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                su32(sb)),
            "l"(bt), "r"(P_BTILE), "r"(su32(&full[s]))
            : "memory");
        ++it;
      }
    }
    if (!ok) {
      fail_sh = 1;
      // drain this CTA's copies still in flight before shared memory is released
      for (long long j = (it > P_STAGES ? it - P_STAGES : 0); j < it; ++j)
        wait_parity(su32(&full[j % P_STAGES]), (uint32_t)((j / P_STAGES) & 1));
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t LBO = 128;
    constexpr uint32_t SBO_A = (P_BKR / (PREC == 1 ? 4 : 8)) * 128;
    const uint32_t fmt = PREC == 1 ? 2u : 1u;
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(P_BNR >> 3) << 17) |
                           ((uint32_t)(P_BM >> 4) << 24);
    long long it = 0;
    int local = 0;
    bool ok = true;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
     int rhs, batch, mt, nt;
     decode_tile(g, tile, rhs, batch, mt, nt);
     const int total = (g.sbeg[batch + 1] - g.sbeg[batch]) * nkt;
     const int nch = total > 0 ? (total + g.kchunk - 1) / g.kchunk : 1;
     for (int ch = 0; ch < nch && ok; ++ch, ++local) {
      const int lo = ch * g.kchunk, hi = min(total, lo + g.kchunk);
      const int b = local & 1;
      if (local >= 2 && !wait_or_fail(su32(&acce[b]), (uint32_t)(((local / 2) - 1) & 1), &fail_sh)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t acc = tmem + (uint32_t)(b * P_BNR);
      for (int i = lo; i < hi; ++i, ++it) {
        const int s = (int)(it % P_STAGES);
        if (!wait_or_fail(su32(&full[s]), (uint32_t)((it / P_STAGES) & 1), &fail_sh)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = su32(smem + s * (P_ATILE + P_BTILE)), b0 = a0 + P_ATILE;
        if (PREC == 1) {
#pragma unroll
          for (int ks = 0; ks < P_BKR / 8; ++ks) {
            const uint32_t ko = ks * 2 * LBO;
            const uint64_t ad = sdesc(a0 + ko, LBO, SBO_A), bd = sdesc(b0 + ko, LBO, SBO_A);
            const uint32_t accum = (i > lo || ks > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc),
                "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
          }
        } else {
#pragma unroll
          for (int ks = 0; ks < P_BKR / 16; ++ks) {
            const uint32_t ko = ks * 2 * LBO;
            const uint64_t ahi = sdesc(a0 + ko, LBO, SBO_A), bhi = sdesc(b0 + ko, LBO, SBO_A);
            const uint64_t alo = sdesc(a0 + P_BM * 64 + ko, LBO, SBO_A),
                           blo = sdesc(b0 + P_BNR * 64 + ko, LBO, SBO_A);
            const uint32_t accum = (i > lo || ks > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p, q;\n setp.ne.b32 p, %6, 0;\n setp.ne.b32 q, 1, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %4, %3, q;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %5, %2, %3, q;\n}\n" ::"r"(acc),
                "l"(ahi), "l"(bhi), "r"(idesc), "l"(blo), "l"(alo), "r"(accum));
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         su32(&empty[s]))
                     : "memory");
      }
      if (!ok) break;
      // accumulator b complete once every MMA above is (immediately when the item is empty)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       su32(&accf[b]))
                   : "memory");
     }
    }
    if (!ok) fail_sh = 1;
    // tracks every MMA this thread issued: TMEM is released only after it completes
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     su32(&donebar))
                 : "memory");
  } else if (warp >= 2) {
    // epilogue: warp w reads TMEM lanes 32*(w%4) .. +31.  The read-modify-write of the
    // FP64 destination dominates short contractions, so the C rows of this CTA's next
    // tile are prefetched into L2 while the current tile drains, and each step keeps 32
    // complex loads of a row in flight.  A storing GEMM does not read C (its first chunk
    // overwrites, later chunks add to what the first wrote).
    const int q = warp & 3;
    auto prefetch_c = [&](long long tl) {
      if (g.epi != 0 || g.store || tl >= ntiles) return;
      int prhs, pbatch, pmt, pnt;
      decode_tile(g, tl, prhs, pbatch, pmt, pnt);
      const int pm = pmt * P_BM + q * 32 + lane;
      const int nb0 = pnt * (P_BNR / 2);
      if (pm >= g.M || nb0 >= g.N) return;
      const int cnt = min(P_BNR / 2, g.N - nb0);
      const double2* row = g.C + prhs * g.sC + g.coff[pbatch] + (long long)pm * g.ldc + nb0;
      for (int j = 0; j < cnt; j += 8) asm volatile("prefetch.global.L2 [%0];" ::"l"(row + j));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(row + cnt - 1));
    };
    int local = 0;
    bool eok = true;
    if (blockIdx.x < ntiles) prefetch_c(blockIdx.x);
    for (long long tile = blockIdx.x; tile < ntiles && eok; tile += gridDim.x) {
     int rhs, batch, mt, nt;
     decode_tile(g, tile, rhs, batch, mt, nt);
     const int tot = (g.sbeg[batch + 1] - g.sbeg[batch]) * nkt;
     const int nch = tot > 0 ? (tot + g.kchunk - 1) / g.kchunk : 1;
     // chunk by chunk, the same thread adds each chunk's sum into the same C elements
     for (int ch = 0; ch < nch; ++ch, ++local) {
      const int total = min(tot - ch * g.kchunk, g.kchunk);
      const int b = local & 1;
      bool ok = wait_or_fail(su32(&accf[b]), (uint32_t)((local / 2) & 1), &fail_sh);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) fail_sh = 1;
        eok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (ch == nch - 1) prefetch_c(tile + gridDim.x);
      const int m = mt * P_BM + q * 32 + lane;
      double2* Cp = g.C + rhs * g.sC + g.coff[batch];
      // 32 complex columns per step: the 32 FP64 loads of the row segment are issued first (in
      // flight together), then the accumulator columns are read from TMEM in two halves
#pragma unroll 1
      const bool st = g.store && ch == 0;
      for (int c0 = 0; c0 < P_BNR; c0 += 64) {
        const bool row = m < g.M && (total > 0 || g.epi == 1 || st);
        const int nb = nt * (P_BNR / 2) + c0 / 2;
        const int cnt = row ? min(32, g.N - nb) : 0;
        double2* cp = Cp + (long long)m * g.ldc + nb;
        double2 cv[32];
        if (g.epi == 0) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < cnt) cv[j] = st ? make_double2(0.0, 0.0) : cp[j];
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t r[32];
          if (total > 0) {
            const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * P_BNR + c0 + 32 * h);
            tmem_ld16(ta, r);
            tmem_ld16(ta + 16u, r + 16);
            asm volatile("tcgen05.wait::ld.sync.aligned;");
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) r[j] = 0u;
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int jj = 16 * h + j;
            if (jj >= cnt) break;
            const double ar = __uint_as_float(r[2 * j]), ai = __uint_as_float(r[2 * j + 1]);
            if (g.epi == 0) {
              cv[jj].x += g.ar * ar - g.ai * ai;
              cv[jj].y += g.ar * ai + g.ai * ar;
              cp[jj] = cv[jj];
            } else {
              const int n = nb + jj;
              const double vr = g.ar * ar - g.ai * ai, vi = g.ar * ai + g.ai * ar;
              const int a = m / g.ep2, c = m - a * g.ep2;
              const int bb = n / g.ep3, d = n - bb * g.ep3;
              Cp[(((long long)a * g.ep1 + bb) * g.ep2 + c) * g.ep3 + d] = make_double2(vr, vi);
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&acce[b])) : "memory");
     }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && !wait_parity(su32(&donebar), 0)) fail_sh = 1;
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (threadIdx.x == 0 && fail_sh) atomicExch(errflag, 1);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

cudaError_t launch_gemm_tcp_persistent(const PGemmArgs& g0, int prec, int nrhs, int* errflag, cudaStream_t st) {
  PGemmArgs g = g0;
  g.tiles_m = (g.M + P_BM - 1) / P_BM;
  g.tiles_n = (g.N + P_BNR / 2 - 1) / (P_BNR / 2);
  g.nrhs = nrhs;
  const long long ntiles = (long long)g.tiles_m * g.tiles_n * g.nbatch * nrhs;
  if (ntiles <= 0) return cudaSuccess;
  static const int nsm = []() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
      return 152;
    return n > 0 ? n : 152;
  }();
  const unsigned grid = (unsigned)std::min<long long>(ntiles, nsm);
  const size_t sm = tcp_smem_bytes();
  if (prec == 1) {
    static const cudaError_t attr =  // thread-safe one-time setup
        cudaFuncSetAttribute(tcp_gemm_persistent<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (attr != cudaSuccess) return attr;
    tcp_gemm_persistent<1><<<grid, P_THREADS, sm, st>>>(g, errflag);
  } else {
    static const cudaError_t attr =
        cudaFuncSetAttribute(tcp_gemm_persistent<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (attr != cudaSuccess) return attr;
    tcp_gemm_persistent<2><<<grid, P_THREADS, sm, st>>>(g, errflag);
  }
  return cudaGetLastError();
}

}  // namespace lrcc
