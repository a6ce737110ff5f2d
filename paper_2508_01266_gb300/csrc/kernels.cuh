// Device-side argument blocks and launchers for the op kinds of a plan.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace lrcc {

// Segmented batched complex GEMM (see plan.h for the exact semantics).
struct GemmArgs {
  int M, N, K, ta, tb, epi, ep1, ep2, ep3;
  long long lda, ldb, ldc;
  double ar, ai;
  const long long* coff;
  const int* sbeg;
  const long long* aoff;
  const long long* boff;
  int tiles_m, tiles_n, nbatch;
  const double2* A;
  const double2* B;
  double2* C;
  long long sA, sB, sC;  // per-vector strides of variable arenas (0 for shared ones)
  // split-K: nsplit > 1 divides each batch entry's (segment, K block) iteration space
  // into nsplit contiguous ranges; every split writes its raw partial tile to
  // part[rhs][batch][split][M][N] and launch_split_reduce sums the splits in a fixed
  // order, applies alpha and the epilogue (bitwise reproducible).
  int nsplit = 1;
  double2* part = nullptr;
  // tensor-core kernel only: the launch computes C^T = B^T A^T (operands and M, N swapped
  // by the caller) and the epilogue writes element (m, n) of the launch to C[n][m]
  int swap = 0;
  // epi == 0: 1 = C is overwritten (C = alpha AB; its old contents are not read), 0 = C += alpha AB
  int store = 0;
};

struct PermArgs {
  int skind, snk, sn[4];
  int dkind, dnk, dn[4];
  int pi[4];
  long long total;
  const double2* S;
  double2* D;
  long long sS, sD;
  double ar, ai;
  int store = 0;  // 1: D = alpha S (D is not read), 0: D += alpha S
};

struct BTransArgs {
  int nb, R, C;
  const double2* S;
  double2* D;
  long long sS, sD;
  double ar, ai;
};

// Tile configurations of the FP64 GEMM kernel.
enum GemmTile : int {
  GT_64x64 = 0, GT_32x64, GT_64x32, GT_32x32, GT_16x64, GT_64x16, GT_16x16, GT_8x32, GT_1x256, GT_256x1,
  GT_48x48,
  GT_COUNT
};
void gemm_tile_dims(int tile, int* bm, int* bn);
int gemm_pick_tile(int M, int N);

cudaError_t launch_gemm_f64(const GemmArgs& g, int tile, int nrhs, cudaStream_t st);
// the same tiled GEMM with FP32 arithmetic (FP64 operands and destination)
cudaError_t launch_gemm_f32(const GemmArgs& g, int tile, int nrhs, cudaStream_t st);
cudaError_t launch_split_reduce(const GemmArgs& g, int nrhs, cudaStream_t st);
// short-contraction and tiny-output GEMM kernels (kernels_small.cu); f32: FP32 arithmetic
bool skinny_k_ok(const GemmArgs& g);
cudaError_t launch_skinny_k(const GemmArgs& g, int nrhs, cudaStream_t st, bool f32);
bool reduce_small_ok(const GemmArgs& g);
cudaError_t launch_reduce_small(const GemmArgs& g, int nrhs, cudaStream_t st, bool f32);
constexpr int F64_BK = 8;  // complex K per iteration of the FP64 GEMM
constexpr int TC_BK = 16;  // complex K per iteration of the unpacked tensor-core GEMM
cudaError_t launch_perm_f64(const PermArgs& p, int nrhs, cudaStream_t st);
cudaError_t launch_btrans_f64(const BTransArgs& t, int nrhs, cudaStream_t st);

// Tensor-core GEMM (kernels_tc.cu): prec 1 = TF32, 2 = BF16x3; same semantics as the
// FP64 kernel, FP32 accumulation.  *errflag is set when a bounded wait gives up.
cudaError_t launch_gemm_tc(const GemmArgs& g, int prec, int nrhs, int* errflag, cudaStream_t st);
size_t tc_smem_bytes(int prec);
cudaError_t launch_wait_selftest(long long polls, int* errflag, cudaStream_t st);

// Packed-operand tensor-core GEMM (kernels_tcp.cu).
struct PackArgs {
  const double2* src;          // arena base (per-vector stride sS)
  unsigned char* dst;          // packed output (per-vector stride sD)
  long long sS, sD;
  const long long* offs;       // element offset of each operand in the arena
  int count;                   // number of operands
  int R, K;                    // complex rows and K of every operand
  long long ld;
  int trans;                   // 0: element (r,k) at r*ld + k; 1: at k*ld + r
  int mode;                    // 0: left operand (A), 1: right operand (B, 2x2 expanded)
  long long packed_bytes;      // bytes per packed operand
};
struct PGemmArgs {
  int M, N, nkt, epi, ep1, ep2, ep3;
  long long ldc;
  double ar, ai;
  const long long* coff;
  const int* sbeg;
  const int* ia;               // packed A operand index of each segment
  const int* ib;               // packed B operand index of each segment
  int tiles_m, tiles_n, nbatch;
  const unsigned char* A;
  const unsigned char* B;
  double2* C;
  long long abytes, bbytes, sA, sB, sC;
  int nrhs = 1;  // persistent kernel: right-hand sides folded into its tile loop
  // persistent kernel: most k-steps (P_BKR real K each) summed in one FP32 accumulator; a
  // tile with more is done in chunks, each added into the FP64 destination by the epilogue
  // (accumulating epilogue only)
  int kchunk = 1 << 30;
  // epi == 0: 1 = the first (or only) chunk overwrites C, later chunks add; 0 = every chunk adds
  int store = 0;
};
long long packed_bytes(int mode, int R, int K);
cudaError_t launch_pack(const PackArgs& p, int prec, int nrhs, cudaStream_t st);
cudaError_t launch_gemm_tcp(const PGemmArgs& g, int prec, int nrhs, int* errflag, cudaStream_t st);
cudaError_t launch_gemm_tcp_persistent(const PGemmArgs& g, int prec, int nrhs, int* errflag, cudaStream_t st);
size_t tcp_smem_bytes();

// DF factor split: L[k1][k2][Q][n][n] (paper units) -> oo/ov/vo/vv blocks * scale.
cudaError_t launch_split_df(const double2* L, int nk, int Q, int o, int v, double scale, double2* Loo,
                            double2* Lov, double2* Lvo, double2* Lvv, cudaStream_t st);

}  // namespace lrcc
