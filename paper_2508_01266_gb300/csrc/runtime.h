// Internal runtime state shared by the ABI implementation and the solvers.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lrcc.h"
#include "kernels.cuh"
#include "plan.h"

namespace lrcc {

struct GemmChoice {
  bool tc = false;  // tensor-core kernel (mixed precision) instead of the FP64 kernel
  int tile = 0;     // FP64 kernel tile (gemm_tile_dims)
  int nsplit = 1;   // split-K factor
  int special = 0;  // 1: short-contraction kernel; 2: tiny-output reduction kernel
  bool packed = false;  // packed-operand tensor-core GEMM (mixed precision)
  bool f32 = false;     // mixed precision: tile / special kernel with FP32 arithmetic
};

struct GemmDesc {
  const long long* coff = nullptr;
  const int* sbeg = nullptr;
  const long long* aoff = nullptr;
  const long long* boff = nullptr;
  int tile = 0;
  int max_seg = 1;  // most segments of any batch entry
};

// Default kernel of a GEMM op for a precision (0 FP64, 1 TF32, 2 BF16x3); host-only, used
// by the executor and by the plan introspection call lrcc_plan_choice.
GemmChoice gemm_default_choice(const Gemm& g, const GemmDesc& d, int prec, bool no_split);

// Packed-operand execution of one GEMM op on the tensor cores (mixed precision).
struct PackPlan {
  bool init = false;
  std::vector<long long> alist, blist;    // distinct operand offsets
  long long *d_aoffs = nullptr, *d_boffs = nullptr;
  int *d_ia = nullptr, *d_ib = nullptr;
  long long abytes = 0, bbytes = 0;       // bytes per packed operand
  unsigned char* fixA[3] = {nullptr, nullptr, nullptr};  // cached packs of fixed operands per precision
  unsigned char* fixB[3] = {nullptr, nullptr, nullptr};
  long long verA[3] = {-1, -1, -1}, verB[3] = {-1, -1, -1};  // fixed-arena version the packs were made from
};

struct Runtime {
  lrcc_dims dims{};
  int device = -1;  // CUDA device current when the problem was created (its buffers live there)
  Plan plan;
  Program jacT;
  std::vector<GemmDesc> gdesc;
  char* desc = nullptr;
  double2 *fix = nullptr, *in = nullptr, *out = nullptr, *scr = nullptr, *ws = nullptr;
  double2 *dip = nullptr, *l1 = nullptr, *l2 = nullptr;
  std::vector<double> eps;
  std::vector<double2> dip_host;  // [3][nk][n][n]
  int cap_rhs = 0;  // vectors held by in/out
  int scr_rhs = 0;  // vectors held by the per-vector scratch (<= cap_rhs)
  int scr_req = 0;  // vectors the scratch was requested for
  int max_batch = 0;  // 0: as many vectors per launch as memory allows
  long long launches = 0;
  std::string err;
  // optional per-op timing with CUDA events on the launching stream
  bool prof = false;
  struct ProfRec { std::string tag; cudaEvent_t a, b; double flops; };
  std::vector<ProfRec> prof_recs;
  std::vector<cudaEvent_t> prof_pool;
  cudaEvent_t prof_event();

  bool ck(cudaError_t e, const char* what);
  lrcc_status init(const lrcc_dims& d, int64_t ws_budget);
  lrcc_status ensure_rhs(int nrhs);
  lrcc_status run_chunked(const Program& pr, int nrhs, cudaStream_t st, int prec);
  int* dflag = nullptr;  // device error flag of the tensor-core kernels (bounded waits)
  std::vector<PackPlan> packs;            // per GEMM op (lazily built)
  long long fix_version = 0;              // bumped whenever the ground-state program rewrites FIX
  unsigned char* packscr = nullptr;       // packed vector-dependent operands (and uncached fixed ones)
  size_t packscr_bytes = 0;
  size_t fixpack_bytes = 0;               // cached packs of fixed operands
  size_t fixpack_budget = (size_t)16 << 30;
  bool use_packed(const Gemm& g, const GemmDesc& d) const;
  // split-K partials (grown on demand; never during a call that must not allocate)
  double2* part = nullptr;
  size_t part_bytes = 0;
  bool no_split = false;
  int pick_split(const Gemm& g, const GemmDesc& d, int nr, bool tc, bool f32 = false) const;
  int pick_split_fill(const Gemm& g, const GemmDesc& d, int nr, bool tc) const;
  lrcc_status run_packed(int gi, const Gemm& g, double2* const ar[AR_COUNT], int nr, bool fixed_only,
                         const long long* stride, cudaStream_t st, int prec);
  // prec: 0 FP64 kernels; 1 TF32 and 2 BF16x3 tensor-core GEMMs (FP32 accumulation)
  lrcc_status run(const Program& pr, double2* const ar[AR_COUNT], int nrhs, cudaStream_t st, int prec = 0);
  lrcc_status apply(int transpose, int nrhs, cudaStream_t st, int prec = 0, bool graphs = false, bool tune = false);
  lrcc_status apply_impl(int transpose, int nrhs, cudaStream_t st, int prec, bool graphs, bool tune);
  // kernel choices of the unpacked GEMMs: default heuristics, or the autotuner's
  // measurements per (transpose, nrhs, prec) when tuning is requested
  GemmChoice default_choice(const Gemm& g, const GemmDesc& d, int prec) const;
  lrcc_status launch_gemm(GemmArgs a, const Gemm& g, const GemmChoice& c, int nr, cudaStream_t st, int prec);
  lrcc_status autotune(const Program& pr, double2* const ar[AR_COUNT], int nrhs, cudaStream_t st, int prec,
                       std::map<int, GemmChoice>& out);
  std::map<std::tuple<int, int, int>, std::map<int, GemmChoice>> tunings;
  const std::map<int, GemmChoice>* tuned = nullptr;  // active during one apply
  // CUDA graphs of whole products, keyed by (transpose, nrhs, prec); a graph is valid
  // while the buffers it was captured with and the fixed-arena version are unchanged
  struct GraphRec {
    cudaGraphExec_t exec = nullptr;
    long long version = -1;
    long long nlaunch = 0;  // kernels in the graph
    const void* bufs[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  };
  std::map<std::tuple<int, int, int>, GraphRec> graphs;
  bool capturing = false;  // inside stream capture: run() skips its host-side flag read
  long long graph_launches = 0;
  void drop_graphs();
  lrcc_status read_flag(cudaStream_t st);
  void release();
  void prof_reset();
};

}  // namespace lrcc

struct lrcc_problem {
  lrcc::Runtime rt;
  bool have_int = false, have_t = false, have_l = false;
};

// Polarizability driver (solver.cu).
// ops (optional): host c128 [ncomp][nk][n][n] one-body operators used instead of the dipole
// components comps (then up to 16 of them).  alpha_sym (optional, asymmetric forms only):
// receives the symmetric form from the same right-hand solutions.
lrcc_status lrcc_polarize_impl(lrcc::Runtime& rt, bool have_t, bool have_l, const int32_t* comps, int32_t ncomp,
                               const double* omegas, int32_t nomega, const lrcc_options* opt, void* alpha,
                               int32_t* info, const double2* ops = nullptr, void* alpha_sym = nullptr);
