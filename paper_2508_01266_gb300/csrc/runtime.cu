// liblrcc runtime: problem handle, device arenas, plan executor and the C-ABI
// entry points of include/lrcc.h (except the host-only plan introspection).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lrcc.h"
#include "kernels.cuh"
#include "plan.h"
#include "runtime.h"

namespace lrcc {

static int64_t align_up(int64_t n) { return (n + 31) / 32 * 32; }

bool Runtime::ck(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  err = std::string(what) + ": " + cudaGetErrorString(e);
  // consume the runtime's last-error state: a recoverable error (for example an
  // allocation that did not fit) must not resurface at the next kernel launch check
  (void)cudaGetLastError();
  return false;
}

cudaEvent_t Runtime::prof_event() {
  if (!prof_pool.empty()) {
    cudaEvent_t e = prof_pool.back();
    prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void Runtime::prof_reset() {
  for (auto& r : prof_recs) {
    prof_pool.push_back(r.a);
    prof_pool.push_back(r.b);
  }
  prof_recs.clear();
}

void Runtime::release() {
  prof_reset();
  for (PackPlan& pp : packs) {
    for (void* p : {(void*)pp.d_aoffs, (void*)pp.d_boffs, (void*)pp.d_ia, (void*)pp.d_ib})
      if (p) cudaFree(p);
    for (int i = 0; i < 3; ++i) {
      if (pp.fixA[i]) cudaFree(pp.fixA[i]);
      if (pp.fixB[i]) cudaFree(pp.fixB[i]);
    }
  }
  packs.clear();
  if (packscr) cudaFree(packscr);
  packscr = nullptr;
  packscr_bytes = 0;
  drop_graphs();
  fixpack_bytes = 0;
  if (part) cudaFree(part);
  part = nullptr;
  part_bytes = 0;
  for (cudaEvent_t e : prof_pool) cudaEventDestroy(e);
  prof_pool.clear();
  for (void* p : {(void*)fix, (void*)in, (void*)out, (void*)scr, (void*)ws, (void*)desc, (void*)dip, (void*)l1,
                  (void*)l2, (void*)dflag})
    if (p) cudaFree(p);
  dflag = nullptr;
  fix = in = out = scr = ws = nullptr;
  desc = nullptr;
  dip = l1 = l2 = nullptr;
  cap_rhs = 0;
}

lrcc_status Runtime::init(const lrcc_dims& d, int64_t ws_budget) {
  dims = d;
  if (cudaGetDevice(&device) != cudaSuccess) device = -1;
  try {
    Dims dd{d.nk, d.nocc, d.nvir, d.naux};
    plan = build_plan(dd, ws_budget);
    jacT = transpose_program(plan, plan.jac);
  } catch (const std::bad_alloc&) {
    err = "host allocation failed while building the plan";
    return LRCC_ENOMEM;
  } catch (const std::exception& e) {
    err = std::string("plan: ") + e.what();
    return LRCC_EINVAL;
  }
  for (const Program* pr : {&plan.ground, &plan.jac, &jacT, &plan.xi, &plan.egrad}) {
    std::string v = validate_plan(plan, *pr);
    if (!v.empty()) {
      err = "plan validation: " + v;
      return LRCC_EINVAL;
    }
  }
  // device descriptor tables of every GEMM
  size_t bytes = 0;
  for (const Gemm& g : plan.gemms)
    bytes += (g.coff.size() + g.aoff.size() + g.boff.size()) * 8 + align_up((int64_t)g.sbeg.size()) * 4 + 64;
  std::vector<char> host(bytes);
  size_t pos = 0;
  std::vector<size_t> base(plan.gemms.size());
  for (size_t i = 0; i < plan.gemms.size(); ++i) {
    const Gemm& g = plan.gemms[i];
    base[i] = pos;
    std::memcpy(&host[pos], g.coff.data(), g.coff.size() * 8);
    pos += g.coff.size() * 8;
    std::memcpy(&host[pos], g.aoff.data(), g.aoff.size() * 8);
    pos += g.aoff.size() * 8;
    std::memcpy(&host[pos], g.boff.data(), g.boff.size() * 8);
    pos += g.boff.size() * 8;
    std::memcpy(&host[pos], g.sbeg.data(), g.sbeg.size() * 4);
    pos += align_up((int64_t)g.sbeg.size()) * 4 + 64;
  }
  if (!ck(cudaMalloc(&desc, bytes > 0 ? bytes : 8), "cudaMalloc(descriptors)")) return LRCC_ENOMEM;
  if (!ck(cudaMemcpy(desc, host.data(), bytes, cudaMemcpyHostToDevice), "cudaMemcpy(descriptors)"))
    return LRCC_ECUDA;
  gdesc.resize(plan.gemms.size());
  for (size_t i = 0; i < plan.gemms.size(); ++i) {
    const Gemm& g = plan.gemms[i];
    char* p = desc + base[i];
    gdesc[i].coff = (const long long*)p;
    gdesc[i].aoff = (const long long*)(p + g.coff.size() * 8);
    gdesc[i].boff = (const long long*)(p + (g.coff.size() + g.aoff.size()) * 8);
    gdesc[i].sbeg = (const int*)(p + (g.coff.size() + g.aoff.size() + g.boff.size()) * 8);
    gdesc[i].tile = gemm_pick_tile(g.M, g.N);
    int ms = 1;
    for (size_t b = 0; b + 1 < g.sbeg.size(); ++b) ms = std::max(ms, g.sbeg[b + 1] - g.sbeg[b]);
    gdesc[i].max_seg = ms;
  }
  const int64_t nk = d.nk, n = d.nocc + d.nvir;
  if (!ck(cudaMalloc(&fix, plan.arena_size[AR_FIX] * sizeof(double2)), "cudaMalloc(fixed arena)")) return LRCC_ENOMEM;
  if (!ck(cudaMalloc(&ws, std::max<int64_t>(plan.arena_size[AR_WS], 1) * sizeof(double2)), "cudaMalloc(workspace)"))
    return LRCC_ENOMEM;
  if (!ck(cudaMalloc(&dip, 3 * nk * n * n * sizeof(double2)), "cudaMalloc(dipoles)")) return LRCC_ENOMEM;
  if (!ck(cudaMemset(fix, 0, plan.arena_size[AR_FIX] * sizeof(double2)), "cudaMemset")) return LRCC_ECUDA;
  if (!ck(cudaMalloc(&dflag, sizeof(int)), "cudaMalloc(flag)")) return LRCC_ENOMEM;
  {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) fixpack_budget = tot / 16;
  }
  if (!ck(cudaMemset(dflag, 0, sizeof(int)), "cudaMemset(flag)")) return LRCC_ECUDA;
  return LRCC_OK;
}

// Longest contraction (complex terms: segments x K) that one FP32 tensor-core
// accumulator may sum.  The FP32 rounding of a chain grows with its length (about
// sqrt(n) u32 typically, n u32 at worst); at 8192 terms the BF16x3 products stay within
// 1e-5 of FP64 on the workloads, while chains of 64000 (the o x o and v x v
// intermediates summed over three momenta) reached 2e-4.  Longer contractions take the
// unpacked kernel with enough K splits, whose partials are summed in FP64.
constexpr long long TC_CHAIN_MAX = 8192;

static long long chain_len(const Gemm& g, const GemmDesc& d) { return (long long)d.max_seg * g.K; }

// Fewest K splits that keep every FP32 accumulator chain of the unpacked tensor-core
// kernel within TC_CHAIN_MAX (its splits take equal shares of the (segment, K tile) range).
static int tc_min_split(const Gemm& g, const GemmDesc& d) {
  const long long iters = (long long)d.max_seg * ((g.K + TC_BK - 1) / TC_BK);
  const long long per = TC_CHAIN_MAX / TC_BK;
  return (int)std::max<long long>(1, (iters + per - 1) / per);
}
// The same bound for the tiled GEMM with FP32 arithmetic (K blocks of F64_BK).
static int f32_min_split(const Gemm& g, const GemmDesc& d) {
  const long long iters = (long long)d.max_seg * ((g.K + F64_BK - 1) / F64_BK);
  const long long per = TC_CHAIN_MAX / F64_BK;
  return (int)std::max<long long>(1, (iters + per - 1) / per);
}
// FP32 tiny-output reduction: a lane sums ceil(K / 32) terms per segment over its split's
// whole segments, then 32 lanes meet in the shuffle tree; keep lanes x chain within
// TC_CHAIN_MAX.  0: not possible (one segment alone is too long).
static int reduce_f32_min_split(const Gemm& g, const GemmDesc& d) {
  const long long lane = (g.K + 31) / 32;
  const long long segs = (TC_CHAIN_MAX / 32) / std::max<long long>(lane, 1);
  if (segs < 1) return 0;
  return (int)std::max<long long>(1, (d.max_seg + segs - 1) / segs);
}

// Complex K terms per k-step of the packed kernel (32 real K = 16 complex).
constexpr long long TCP_KSTEP = 16;
// Output tiles (128 x 128 complex) of one vector of a packed GEMM.
static long long tcp_tiles(const Gemm& g) {
  return (long long)((g.M + 127) / 128) * ((g.N + 127) / 128) * g.nbatch();
}
// Packed-operand tensor-core path for GEMMs with both output dimensions at least
// LRCC_PACKED_MIN (default 32) and K >= 16.  The persistent packed kernel sums at most
// TC_CHAIN_MAX complex terms in one FP32 accumulator: a longer contraction is done in
// chunks whose sums its epilogue adds into the FP64 destination one after the other
// (same thread, same elements).  That serialises a tile's chunks, so long contractions
// take this path only when one vector alone has a few dozen output tiles and the chunks
// are few (the ladder at Nk = 7 and 9: two or three); a storing epilogue (the W-block
// build) cannot be chunked.  The autotuner may also choose it per op, under the same rules.
static bool packed_ok(const Gemm& g, const GemmDesc& d) {
  static const int pmin = []() {
    const char* e = std::getenv("LRCC_PACKED_MIN");
    const int v = e ? std::atoi(e) : 0;
    return v > 0 ? v : 32;
  }();
  if (g.M < pmin || g.N < pmin || g.K < 16) return false;
  const long long chain = chain_len(g, d);
  if (chain <= TC_CHAIN_MAX) return true;
  return g.epi == 0 && chain <= 4 * TC_CHAIN_MAX && tcp_tiles(g) >= 32;
}
bool Runtime::use_packed(const Gemm& g, const GemmDesc& d) const { return packed_ok(g, d); }

// Useful fraction of the unpacked tensor-core tiles (128 x 64 complex, K in steps of 16)
// for an M x N x K GEMM.
static double tc_eff(long long M, long long N, long long K) {
  const double tm = (double)((M + 127) / 128) * 128, tn = (double)((N + 63) / 64) * 64;
  const double tk = (double)((K + 15) / 16) * 16;
  return (double)M * N * K / (tm * tn * tk);
}
// Launch the tensor-core GEMM as C^T = B^T A^T when that fills its tiles better (small M).
static bool tc_swap(const Gemm& g) { return tc_eff(g.N, g.M, g.K) > tc_eff(g.M, g.N, g.K); }
// Mixed precision uses the tensor cores unless even the better orientation leaves under
// 0.4 % of the tile useful (a few sub-tile GEMMs, cheap on the FP64 kernel).
static bool tc_tile_useful(const Gemm& g) {
  return std::max(tc_eff(g.M, g.N, g.K), tc_eff(g.N, g.M, g.K)) >= 0.004;
}

// Split-K factor: enough CTAs to fill the 152 SMs a few times over when the output
// tiles of one vector cannot, keeping at least 8 K iterations per split and the
// partials of one vector under 64 MiB; with FP32 accumulation (tensor cores or FP32
// arithmetic) at least the split that caps the accumulator chains.  The
// choice does not depend on the number of vectors, so a vector's result is bitwise the
// same in any batch.
static int split_fill(const Gemm& g, const GemmDesc& d, bool tc);

static int split_for(const Gemm& g, const GemmDesc& d, bool tc, bool f32, bool no_split) {
  if (no_split) return 1;
  return std::max(split_fill(g, d, tc), tc ? tc_min_split(g, d) : f32 ? f32_min_split(g, d) : 1);
}
int Runtime::pick_split(const Gemm& g, const GemmDesc& d, int nr, bool tc, bool f32) const {
  (void)nr;
  return split_for(g, d, tc, f32, no_split);
}
int Runtime::pick_split_fill(const Gemm& g, const GemmDesc& d, int nr, bool tc) const {
  (void)nr;
  return split_fill(g, d, tc);
}

static int split_fill(const Gemm& g, const GemmDesc& d, bool tc) {
  int bm = 128, bn = 64;
  if (!tc) gemm_tile_dims(d.tile, &bm, &bn);
  const bool sw = tc && tc_swap(g);
  const long long LM = sw ? g.N : g.M, LN = sw ? g.M : g.N;
  const long long tiles = ((LM + bm - 1) / bm) * ((LN + bn - 1) / bn) * g.nbatch();
  const long long target = tc ? 152LL * 3 : 152LL * 6;
  if (tiles >= target) return 1;
  const int bk = tc ? TC_BK : F64_BK;
  const long long iters = (long long)d.max_seg * ((g.K + bk - 1) / bk);
  long long s = (target + tiles - 1) / tiles;
  s = std::min<long long>(s, iters / 8);
  s = std::min<long long>(s, 1024);
  const long long per = (long long)g.nbatch() * g.M * g.N * (long long)sizeof(double2);
  if (per > 0) s = std::min<long long>(s, (64LL << 20) / per);
  return (int)std::max<long long>(s, 1);
}

static bool is_vec_arena(int ar) { return ar == AR_IN || ar == AR_OUT || ar == AR_SCR; }

lrcc_status Runtime::run_packed(int gi, const Gemm& g, double2* const ar[AR_COUNT], int nr, bool fixed_only,
                                const long long* stride, cudaStream_t st, int prec) {
  if (packs.size() < plan.gemms.size()) packs.resize(plan.gemms.size());
  PackPlan& pp = packs[gi];
  if (!pp.init) {
    std::vector<int> ia(g.aoff.size()), ib(g.boff.size());
    std::vector<long long> la, lb;
    for (size_t s = 0; s < g.aoff.size(); ++s) {
      auto it = std::find(la.begin(), la.end(), g.aoff[s]);
      ia[s] = (int)(it - la.begin());
      if (it == la.end()) la.push_back(g.aoff[s]);
      auto jt = std::find(lb.begin(), lb.end(), g.boff[s]);
      ib[s] = (int)(jt - lb.begin());
      if (jt == lb.end()) lb.push_back(g.boff[s]);
    }
    pp.alist = la;
    pp.blist = lb;
    pp.abytes = packed_bytes(0, g.M, g.K);
    pp.bbytes = packed_bytes(1, g.N, g.K);
    if (!ck(cudaMalloc(&pp.d_aoffs, la.size() * 8), "cudaMalloc(pack)") ||
        !ck(cudaMalloc(&pp.d_boffs, lb.size() * 8), "cudaMalloc(pack)") ||
        !ck(cudaMalloc(&pp.d_ia, ia.size() * 4), "cudaMalloc(pack)") ||
        !ck(cudaMalloc(&pp.d_ib, ib.size() * 4), "cudaMalloc(pack)"))
      return LRCC_ENOMEM;
    if (!ck(cudaMemcpy(pp.d_aoffs, la.data(), la.size() * 8, cudaMemcpyHostToDevice), "pack upload") ||
        !ck(cudaMemcpy(pp.d_boffs, lb.data(), lb.size() * 8, cudaMemcpyHostToDevice), "pack upload") ||
        !ck(cudaMemcpy(pp.d_ia, ia.data(), ia.size() * 4, cudaMemcpyHostToDevice), "pack upload") ||
        !ck(cudaMemcpy(pp.d_ib, ib.data(), ib.size() * 4, cudaMemcpyHostToDevice), "pack upload"))
      return LRCC_ECUDA;
    pp.init = true;
  }
  // operands that live in the fixed arena are packed once per precision and cached while
  // the cache stays within its budget (1/16 of device memory); beyond it they are packed
  // into the shared scratch at every use (a memory-bound pass, cheap next to the GEMM).
  // Vector and workspace operands are packed every time.
  const bool varA = g.arA != AR_FIX, varB = g.arB != AR_FIX;
  const int nrA = (!fixed_only && is_vec_arena(g.arA)) ? nr : 1;
  const int nrB = (!fixed_only && is_vec_arena(g.arB)) ? nr : 1;
  const size_t sizeA = (size_t)pp.abytes * pp.alist.size(), sizeB = (size_t)pp.bbytes * pp.blist.size();
  const bool cacheA = !varA && (pp.fixA[prec] || fixpack_bytes + sizeA <= fixpack_budget);
  const bool cacheB = !varB && (pp.fixB[prec] || fixpack_bytes + (cacheA && !pp.fixA[prec] ? sizeA : 0) + sizeB <=
                                                     fixpack_budget);
  const size_t needA = varA ? sizeA * nrA : (cacheA ? 0 : sizeA);
  const size_t needB = varB ? sizeB * nrB : (cacheB ? 0 : sizeB);
  if (needA + needB + 1024 > packscr_bytes) {
    if (!ck(cudaStreamSynchronize(st), "sync")) return LRCC_ECUDA;  // earlier ops may still read it
    if (packscr) cudaFree(packscr);
    packscr = nullptr;
    packscr_bytes = 0;
    if (!ck(cudaMalloc(&packscr, needA + needB + 1024), "cudaMalloc(pack scratch)")) return LRCC_ENOMEM;
    packscr_bytes = needA + needB + 1024;
  }
  auto pack = [&](int mode, int arena, const std::vector<long long>& list, const long long* doffs, int R,
                  long long ld, int trans, long long bytes, unsigned char* dst, int nrr) -> lrcc_status {
    PackArgs pa;
    pa.src = ar[arena];
    pa.dst = dst;
    pa.sS = nrr > 1 ? stride[arena] : 0;
    pa.sD = (long long)bytes * list.size();
    pa.offs = doffs;
    pa.count = (int)list.size();
    pa.R = R;
    pa.K = g.K;
    pa.ld = ld;
    pa.trans = trans;
    pa.mode = mode;
    pa.packed_bytes = bytes;
    if (!ck(launch_pack(pa, prec, nrr, st), "pack")) return LRCC_ECUDA;
    ++launches;
    return LRCC_OK;
  };
  const unsigned char* Ap;
  const unsigned char* Bp;
  lrcc_status s;
  if (!cacheA) {
    if ((s = pack(0, g.arA, pp.alist, pp.d_aoffs, g.M, g.lda, g.ta, pp.abytes, packscr, nrA)) != LRCC_OK) return s;
    Ap = packscr;
  } else {
    if (!pp.fixA[prec]) {
      if (!ck(cudaMalloc(&pp.fixA[prec], sizeA), "cudaMalloc(packed fixed)")) return LRCC_ENOMEM;
      fixpack_bytes += sizeA;
    }
    if (pp.verA[prec] != fix_version) {
      if ((s = pack(0, g.arA, pp.alist, pp.d_aoffs, g.M, g.lda, g.ta, pp.abytes, pp.fixA[prec], 1)) != LRCC_OK)
        return s;
      pp.verA[prec] = fix_version;
    }
    Ap = pp.fixA[prec];
  }
  if (!cacheB) {
    unsigned char* dst = packscr + needA;
    if ((s = pack(1, g.arB, pp.blist, pp.d_boffs, g.N, g.ldb, g.tb ? 0 : 1, pp.bbytes, dst, nrB)) != LRCC_OK)
      return s;
    Bp = dst;
  } else {
    if (!pp.fixB[prec]) {
      if (!ck(cudaMalloc(&pp.fixB[prec], sizeB), "cudaMalloc(packed fixed)")) return LRCC_ENOMEM;
      fixpack_bytes += sizeB;
    }
    if (pp.verB[prec] != fix_version) {
      if ((s = pack(1, g.arB, pp.blist, pp.d_boffs, g.N, g.ldb, g.tb ? 0 : 1, pp.bbytes, pp.fixB[prec], 1)) !=
          LRCC_OK)
        return s;
      pp.verB[prec] = fix_version;
    }
    Bp = pp.fixB[prec];
  }
  const GemmDesc& d = gdesc[gi];
  PGemmArgs a;
  a.M = g.M; a.N = g.N; a.nkt = (int)((2LL * g.K + 31) / 32);
  a.epi = g.epi; a.ep1 = g.ep[1]; a.ep2 = g.ep[2]; a.ep3 = g.ep[3];
  a.ldc = g.ldc; a.ar = g.ar; a.ai = g.ai;
  a.store = g.store;
  a.coff = d.coff; a.sbeg = d.sbeg; a.ia = pp.d_ia; a.ib = pp.d_ib;
  a.nbatch = g.nbatch();
  a.tiles_m = a.tiles_n = 1;
  a.A = Ap; a.B = Bp; a.C = ar[g.arC];
  a.abytes = pp.abytes; a.bbytes = pp.bbytes;
  a.sA = nrA > 1 ? (long long)pp.abytes * pp.alist.size() : 0;
  a.sB = nrB > 1 ? (long long)pp.bbytes * pp.blist.size() : 0;
  a.sC = (!fixed_only && is_vec_arena(g.arC)) ? stride[g.arC] : 0;
  // persistent double-buffered kernel by default; LRCC_PACKED_KERNEL=classic selects the
  // one-tile-per-CTA kernel (same arithmetic, same results)
  static const bool persistent = []() {
    const char* e = std::getenv("LRCC_PACKED_KERNEL");
    return !(e && std::string(e) == "classic");
  }();
  const int nrr = fixed_only ? 1 : nr;
  // FP32 accumulator chains within TC_CHAIN_MAX: longer tiles in chunks (persistent kernel)
  a.kchunk = (int)(TC_CHAIN_MAX / TCP_KSTEP);
  const bool chunked = chain_len(g, d) > TC_CHAIN_MAX;
  if (chunked && g.epi != 0) {
    err = "packed gemm: a storing epilogue cannot take a chunked contraction";
    return LRCC_EINVAL;
  }
  const cudaError_t e = (persistent || chunked) ? launch_gemm_tcp_persistent(a, prec, nrr, dflag, st)
                                                : launch_gemm_tcp(a, prec, nrr, dflag, st);
  if (!ck(e, "packed gemm")) return LRCC_ECUDA;
  ++launches;
  return LRCC_OK;
}

// Input/output vectors for nrhs right-hand sides; per-vector scratch for as many of them
// as fit (max_batch caps it when set): products over larger batches run in chunks of
// scr_rhs vectors (run_chunked), with identical results.
lrcc_status Runtime::ensure_rhs(int nrhs) {
  const int want_scr = max_batch > 0 ? std::min(nrhs, max_batch) : nrhs;
  // keep the buffers when they hold the batch and the scratch was sized for at least this
  // request (a smaller scratch than requested means memory ran out; asking again would not help)
  if (nrhs <= cap_rhs && want_scr <= scr_req && (max_batch <= 0 || scr_rhs <= max_batch)) return LRCC_OK;
  drop_graphs();
  for (double2** p : {&in, &out, &scr})
    if (*p) {
      cudaFree(*p);
      *p = nullptr;
    }
  cap_rhs = 0;
  scr_rhs = 0;
  scr_req = 0;
  const int64_t vin = plan.arena_size[AR_IN], vscr = std::max<int64_t>(plan.arena_size[AR_SCR], 1);
  if (!ck(cudaMalloc(&in, vin * nrhs * sizeof(double2)), "cudaMalloc(input vectors)")) return LRCC_ENOMEM;
  if (!ck(cudaMalloc(&out, vin * nrhs * sizeof(double2)), "cudaMalloc(output vectors)")) return LRCC_ENOMEM;
  for (int k = want_scr; k >= 1; k = k / 2) {
    if (cudaMalloc(&scr, vscr * k * sizeof(double2)) == cudaSuccess) {
      scr_rhs = k;
      break;
    }
    (void)cudaGetLastError();
    scr = nullptr;
    if (k == 1) break;
  }
  if (!scr) {
    err = "cudaMalloc(scratch): out of memory even for one vector";
    return LRCC_ENOMEM;
  }
  cap_rhs = nrhs;
  scr_req = want_scr;
  return LRCC_OK;
}

// A vector program over nrhs vectors held in in/out, in chunks of at most scr_rhs.
lrcc_status Runtime::run_chunked(const Program& pr, int nrhs, cudaStream_t st, int prec) {
  const int64_t vin = plan.arena_size[AR_IN];
  const int step = std::max(1, scr_rhs);
  for (int c0 = 0; c0 < nrhs; c0 += step) {
    const int cnt = std::min(step, nrhs - c0);
    double2* ar[AR_COUNT] = {fix, in + (size_t)c0 * vin, out + (size_t)c0 * vin, scr, ws};
    lrcc_status s = run(pr, ar, cnt, st, prec);
    if (s != LRCC_OK) return s;
  }
  return LRCC_OK;
}

static GemmArgs shape_args(const Gemm& g) {
  GemmArgs a;
  a.M = g.M; a.N = g.N; a.K = g.K; a.ta = g.ta; a.tb = g.tb; a.epi = g.epi;
  return a;
}

// Splits of the tiny-output reduction: whole segments per split, about 8 CTAs per SM.
static int reduce_split(const Gemm& g, const GemmDesc& d) {
  const long long want = (152LL * 8 + g.nbatch() - 1) / g.nbatch();
  long long s = std::min<long long>(want, d.max_seg);
  const long long per = (long long)g.nbatch() * g.M * g.N * (long long)sizeof(double2);
  if (per > 0) s = std::min<long long>(s, (64LL << 20) / per);
  return (int)std::max<long long>(s, 1);
}

// Default kernel of a GEMM op.  FP64 products: the tiny-output reduction kernel where it
// applies, else the FP64 tile kernel.  Mixed precision: the packed tensor-core path for
// large tiles; the reduction and short-contraction kernels in FP32 arithmetic; the FP32
// tile kernel where even the better orientation of the unpacked tensor-core tile would
// be under 20 % useful (small tiles, K <= 40: FP64-pipe bound, HBM bound in FP32); else
// the unpacked tensor-core kernel.  The autotuner may replace any of these per op.
GemmChoice gemm_default_choice(const Gemm& g, const GemmDesc& d, int prec, bool no_split) {
  GemmChoice c;
  if (prec > 0 && packed_ok(g, d)) {
    c.packed = true;
    return c;
  }
  const GemmArgs sa = shape_args(g);
  if (reduce_small_ok(sa) && !no_split) {
    c.special = 2;
    c.nsplit = reduce_split(g, d);
    const int fmin = reduce_f32_min_split(g, d);
    if (prec > 0 && fmin > 0) {
      c.f32 = true;
      c.nsplit = std::max(c.nsplit, fmin);
    }
    return c;
  }
  if (prec > 0 && skinny_k_ok(sa) && chain_len(g, d) <= TC_CHAIN_MAX) {
    c.special = 1;
    c.f32 = true;
    return c;
  }
  c.tile = d.tile;
  if (prec > 0 && std::max(tc_eff(g.M, g.N, g.K), tc_eff(g.N, g.M, g.K)) < 0.2) {
    c.f32 = true;
    c.nsplit = split_for(g, d, false, true, no_split);
    return c;
  }
  c.tc = prec > 0 && tc_tile_useful(g);
  c.nsplit = split_for(g, d, c.tc, false, no_split);
  return c;
}

GemmChoice Runtime::default_choice(const Gemm& g, const GemmDesc& d, int prec) const {
  return gemm_default_choice(g, d, prec, no_split);
}

}  // namespace lrcc

extern "C" lrcc_status lrcc_plan_choice(const lrcc_plan* h, int32_t idx, int32_t precision, int32_t* out) {
  using namespace lrcc;
  const Plan* P = plan_of(h);
  if (!P || !out || idx < 0 || idx >= (int32_t)P->gemms.size() || precision < 0 || precision > 2)
    return LRCC_EINVAL;
  const Gemm& g = P->gemms[idx];
  GemmDesc d;
  d.tile = gemm_pick_tile(g.M, g.N);
  int ms = 1;
  for (size_t b = 0; b + 1 < g.sbeg.size(); ++b) ms = std::max(ms, g.sbeg[b + 1] - g.sbeg[b]);
  d.max_seg = ms;
  const GemmChoice c = gemm_default_choice(g, d, precision, false);
  out[0] = c.packed;
  out[1] = c.special;
  out[2] = c.tc;
  out[3] = c.f32;
  out[4] = c.tile;
  out[5] = c.nsplit;
  out[6] = d.max_seg;
  return LRCC_OK;
}

namespace lrcc {

// One unpacked GEMM op with an explicit kernel choice (tile of the FP64 kernel or the
// tensor-core kernel, split-K factor); grows the split-K partials buffer if needed.
lrcc_status Runtime::launch_gemm(GemmArgs a, const Gemm& g, const GemmChoice& c, int nr, cudaStream_t st, int prec) {
  if (c.special == 1) {
    a.nsplit = 1;
    a.part = nullptr;
    ++launches;
    return ck(launch_skinny_k(a, nr, st, c.f32 && prec > 0), "skinny gemm launch") ? LRCC_OK : LRCC_ECUDA;
  }
  a.nsplit = no_split ? 1 : std::max(1, c.nsplit);
  a.part = nullptr;
  if (a.nsplit > 1) {
    const size_t need = (size_t)nr * g.nbatch() * a.nsplit * g.M * g.N * sizeof(double2);
    if (need > part_bytes) {
      if (part) {
        if (!ck(cudaStreamSynchronize(st), "split-K sync")) return LRCC_ECUDA;
        cudaFree(part);
        part = nullptr;
        part_bytes = 0;
      }
      if (!ck(cudaMalloc(&part, need), "cudaMalloc(split-K partials)")) return LRCC_ENOMEM;
      part_bytes = need;
    }
    a.part = part;
  }
  cudaError_t e;
  if (c.special == 2) {
    if (!a.part) {  // nsplit == 1: one partial buffer still needed
      const size_t need = (size_t)nr * g.nbatch() * g.M * g.N * sizeof(double2);
      if (need > part_bytes) {
        if (part) {
          if (!ck(cudaStreamSynchronize(st), "split-K sync")) return LRCC_ECUDA;
          cudaFree(part);
          part = nullptr;
          part_bytes = 0;
        }
        if (!ck(cudaMalloc(&part, need), "cudaMalloc(split-K partials)")) return LRCC_ENOMEM;
        part_bytes = need;
      }
      a.part = part;
    }
    e = launch_reduce_small(a, nr, st, c.f32 && prec > 0);
    ++launches;
    if (e == cudaSuccess) {
      e = launch_split_reduce(a, nr, st);
      ++launches;
    }
    return ck(e, "reduction gemm launch") ? LRCC_OK : LRCC_ECUDA;
  }
  if (c.tc && prec > 0) {
    GemmArgs b = a;
    if (tc_swap(g)) {  // C^T = B^T A^T: operands, transposes, leading dimensions and M, N swap
      b.swap = 1;
      b.M = a.N;
      b.N = a.M;
      b.A = a.B;
      b.B = a.A;
      b.sA = a.sB;
      b.sB = a.sA;
      b.aoff = a.boff;
      b.boff = a.aoff;
      b.lda = a.ldb;
      b.ldb = a.lda;
      b.ta = !a.tb;
      b.tb = !a.ta;
    }
    e = launch_gemm_tc(b, prec, nr, dflag, st);
  } else {
    e = (c.f32 && prec > 0) ? launch_gemm_f32(a, c.tile, nr, st) : launch_gemm_f64(a, c.tile, nr, st);
  }
  ++launches;
  if (e == cudaSuccess && a.nsplit > 1) {
    e = launch_split_reduce(a, nr, st);
    ++launches;
  }
  return ck(e, "gemm launch") ? LRCC_OK : LRCC_ECUDA;
}

// Autotuner: for every unpacked GEMM op of the program, time the candidate kernel
// choices on the problem's own operands (one untimed launch, one timed launch that
// drops candidates over three times the best so far, then two timed launches; CUDA
// events) and keep the fastest.  Ops whose default already takes over 50 ms are
// compute-saturated large GEMMs and keep their default.  The timing launches
// accumulate into the op's destination, so the caller reruns the product afterwards.
constexpr int kTuneVectors = 4;

lrcc_status Runtime::autotune(const Program& pr, double2* const ar[AR_COUNT], int nrhs, cudaStream_t st, int prec,
                              std::map<int, GemmChoice>& out) {
  long long stride[AR_COUNT] = {0, plan.arena_size[AR_IN], plan.arena_size[AR_OUT], plan.arena_size[AR_SCR], 0};
  cudaEvent_t e0, e1;
  if (!ck(cudaEventCreate(&e0), "autotune event") || !ck(cudaEventCreate(&e1), "autotune event")) return LRCC_ECUDA;
  lrcc_status rs = LRCC_OK;
  for (const Op& op : pr.ops) {
    if (op.kind != OP_GEMM) continue;
    const Gemm& g = plan.gemms[op.idx];
    if (g.arC == AR_FIX) continue;  // never disturb fixed data
    const GemmDesc& d = gdesc[op.idx];
    // candidates are timed on the first few vectors of the batch (per-vector work is the
    // same for every vector; a large batch would multiply the tuning time)
    const int nr = op.fixed_only ? 1 : std::min(nrhs, kTuneVectors);
    GemmArgs a;
    a.M = g.M; a.N = g.N; a.K = g.K; a.ta = g.ta; a.tb = g.tb;
    a.epi = g.epi; a.ep1 = g.ep[1]; a.ep2 = g.ep[2]; a.ep3 = g.ep[3];
    a.lda = g.lda; a.ldb = g.ldb; a.ldc = g.ldc;
    a.ar = g.ar; a.ai = g.ai;
    a.store = g.store;
    a.coff = d.coff; a.sbeg = d.sbeg; a.aoff = d.aoff; a.boff = d.boff;
    a.nbatch = g.nbatch();
    a.tiles_m = a.tiles_n = 1;
    a.A = ar[g.arA]; a.B = ar[g.arB]; a.C = ar[g.arC];
    a.sA = op.fixed_only ? 0 : stride[g.arA];
    a.sB = op.fixed_only ? 0 : stride[g.arB];
    a.sC = op.fixed_only ? 0 : stride[g.arC];
    auto one = [&](const GemmChoice& c) -> lrcc_status {
      return c.packed ? run_packed(op.idx, g, ar, nr, op.fixed_only != 0, stride, st, prec)
                      : launch_gemm(a, g, c, nr, st, prec);
    };
    float best_seen = 1e30f;
    auto time_it = [&](const GemmChoice& c, float& ms) -> lrcc_status {
      // an untimed launch first: a kernel's first launch in the process also loads its
      // code (lazy module loading), which must not count against it
      lrcc_status s2 = one(c);
      if (s2 != LRCC_OK) return s2;
      if (!ck(cudaEventRecord(e0, st), "autotune record")) return LRCC_ECUDA;
      if ((s2 = one(c)) != LRCC_OK) return s2;
      float first = 0.f;
      if (!ck(cudaEventRecord(e1, st), "autotune record") || !ck(cudaEventSynchronize(e1), "autotune sync") ||
          !ck(cudaEventElapsedTime(&first, e0, e1), "autotune elapsed"))
        return LRCC_ECUDA;
      if (first > 3.f * best_seen) {  // far slower than the best so far: not worth timing
        ms = 1e30f;
        return LRCC_OK;
      }
      if (!ck(cudaEventRecord(e0, st), "autotune record")) return LRCC_ECUDA;
      for (int r = 0; r < 2; ++r)
        if ((s2 = one(c)) != LRCC_OK) return s2;
      if (!ck(cudaEventRecord(e1, st), "autotune record") || !ck(cudaEventSynchronize(e1), "autotune sync") ||
          !ck(cudaEventElapsedTime(&ms, e0, e1), "autotune elapsed"))
        return LRCC_ECUDA;
      best_seen = std::min(best_seen, ms / 2.f);
      return LRCC_OK;
    };
    const GemmChoice def = default_choice(g, d, prec);
    float best_ms = 0.f;
    if ((rs = time_it(def, best_ms)) != LRCC_OK) break;
    GemmChoice best = def;
    if (best_ms < 100.f) {
      // candidates: mixed precision tries the tensor-core paths (packed; unpacked with
      // split factors), the short-contraction kernel and the tile shapes of the tiled
      // kernel within 25 % of the least padded one, the last two in FP32 arithmetic
      // (accumulator chains capped by the splits); FP64 tries the short-contraction kernel
      // and the same FP64 tile shapes with split factors.  A candidate whose first timed
      // launch takes over three times the best so far is dropped without further launches.
      std::vector<GemmChoice> cand;
      const bool mixed = prec > 0;
      auto key = [](const GemmChoice& x) {
        const bool tiled = !x.packed && !x.tc && x.special == 0;
        return std::make_tuple(x.packed, x.special, x.tc, x.f32, tiled ? x.tile : -1,
                               (x.packed || x.special == 1) ? 0 : x.nsplit);
      };
      auto add = [&](const GemmChoice& c) {
        if (key(c) == key(def)) return;
        for (const auto& x : cand)
          if (key(x) == key(c)) return;
        cand.push_back(c);
      };
      if (mixed && g.M >= 8 && g.N >= 8 && g.K >= 8 &&
          (chain_len(g, d) <= TC_CHAIN_MAX || packed_ok(g, d))) {
        GemmChoice pk;
        pk.packed = true;
        add(pk);
      }
      if (skinny_k_ok(shape_args(g)) && (!mixed || chain_len(g, d) <= TC_CHAIN_MAX)) {
        GemmChoice sk;
        sk.special = 1;
        sk.f32 = mixed;
        add(sk);
      }
      if (mixed) {
        GemmChoice c;
        c.tc = true;
        c.tile = d.tile;
        const int s0 = pick_split(g, d, 1, true);
        for (int sp : {1, s0, std::max(1, s0 / 2), s0 * 2}) {
          c.nsplit = std::max(sp, tc_min_split(g, d));
          add(c);
        }
      }
      double wmin = 1e300;
      std::vector<double> wt(GT_COUNT);
      for (int t = 0; t < GT_COUNT; ++t) {
        int bm = 1, bn = 1;
        gemm_tile_dims(t, &bm, &bn);
        wt[t] = (double)((g.M + bm - 1) / bm) * bm * (double)((g.N + bn - 1) / bn) * bn;
        wmin = std::min(wmin, wt[t]);
      }
      for (int t = 0; t < GT_COUNT; ++t) {
        if (wt[t] > 1.25 * wmin) continue;
        GemmChoice c;
        c.f32 = mixed;
        c.tile = t;
        GemmDesc dd = d;
        dd.tile = t;
        const int s0 = pick_split(g, dd, 1, false, mixed);
        const int smin = mixed ? f32_min_split(g, dd) : 1;
        for (int sp : {1, s0, std::max(1, s0 / 2), s0 * 2}) {
          c.nsplit = std::max(sp, smin);
          add(c);
        }
      }
      for (const auto& c : cand) {
        float ms = 0.f;
        if ((rs = time_it(c, ms)) != LRCC_OK) break;
        if (ms < best_ms) {
          best_ms = ms;
          best = c;
        }
      }
      if (rs != LRCC_OK) break;
    }
    out[op.idx] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rs == LRCC_OK && prec > 0) rs = read_flag(st);
  return rs;
}

lrcc_status Runtime::run(const Program& pr, double2* const ar[AR_COUNT], int nrhs, cudaStream_t st, int prec) {
  if (&pr == &plan.ground) ++fix_version;  // cached tensor-core packs of fixed operands are stale
  long long stride[AR_COUNT] = {0, plan.arena_size[AR_IN], plan.arena_size[AR_OUT], plan.arena_size[AR_SCR], 0};
  for (const Op& op : pr.ops) {
    cudaError_t e = cudaSuccess;
    const int nr = op.fixed_only ? 1 : nrhs;
    const char* optag = op.kind == OP_GEMM     ? plan.gemms[op.idx].tag.c_str()
                        : op.kind == OP_PERM   ? plan.perms[op.idx].tag.c_str()
                        : op.kind == OP_BTRANS ? plan.btrans[op.idx].tag.c_str()
                                               : "zero";
    nvtxRangePushA(optag);  // per-op range (ncu --nvtx --nvtx-include "<tag>/")
    ProfRec rec{};
    if (prof) {
      rec.a = prof_event();
      rec.b = prof_event();
      rec.flops = 0.0;
      if (op.kind == OP_GEMM) {
        rec.tag = plan.gemms[op.idx].tag;
        rec.flops = (double)plan.gemms[op.idx].flops() * nr;
      } else if (op.kind == OP_PERM) {
        rec.tag = "perm:" + plan.perms[op.idx].tag;
      } else if (op.kind == OP_BTRANS) {
        rec.tag = "btrans:" + plan.btrans[op.idx].tag;
      } else {
        rec.tag = "zero";
      }
      cudaEventRecord(rec.a, st);
    }
    if (op.kind == OP_GEMM) {
      const Gemm& g = plan.gemms[op.idx];
      const GemmDesc& d = gdesc[op.idx];
      GemmArgs a;
      a.M = g.M; a.N = g.N; a.K = g.K; a.ta = g.ta; a.tb = g.tb;
      a.epi = g.epi; a.ep1 = g.ep[1]; a.ep2 = g.ep[2]; a.ep3 = g.ep[3];
      a.lda = g.lda; a.ldb = g.ldb; a.ldc = g.ldc;
      a.ar = g.ar; a.ai = g.ai;
      a.store = g.store;
      a.coff = d.coff; a.sbeg = d.sbeg; a.aoff = d.aoff; a.boff = d.boff;
      a.nbatch = g.nbatch();
      a.tiles_m = a.tiles_n = 1;
      a.A = ar[g.arA]; a.B = ar[g.arB]; a.C = ar[g.arC];
      a.sA = op.fixed_only ? 0 : stride[g.arA];
      a.sB = op.fixed_only ? 0 : stride[g.arB];
      a.sC = op.fixed_only ? 0 : stride[g.arC];
      GemmChoice c = default_choice(g, d, prec);
      if (tuned) {
        auto t = tuned->find(op.idx);
        if (t != tuned->end()) c = t->second;
      }
      if (prec > 0 && c.packed) {
        lrcc_status ps = run_packed(op.idx, g, ar, nr, op.fixed_only != 0, stride, st, prec);
        if (ps != LRCC_OK) return ps;
      } else {
        lrcc_status gs = launch_gemm(a, g, c, nr, st, prec);
        if (gs != LRCC_OK) return gs;
      }
    } else if (op.kind == OP_PERM) {
      const Perm& p = plan.perms[op.idx];
      PermArgs a;
      a.skind = p.src.kind; a.snk = p.src.nk;
      a.dkind = p.dst.kind; a.dnk = p.dst.nk;
      for (int s = 0; s < 4; ++s) {
        a.sn[s] = p.src.n[s];
        a.dn[s] = p.dst.n[s];
        a.pi[s] = p.pi[s];
      }
      a.total = p.dst.size();
      a.S = ar[p.arS] + p.offS;
      a.D = ar[p.arD] + p.offD;
      a.sS = op.fixed_only ? 0 : stride[p.arS];
      a.sD = op.fixed_only ? 0 : stride[p.arD];
      a.ar = p.ar; a.ai = p.ai;
      a.store = p.store;
      e = launch_perm_f64(a, nr, st);
      ++launches;
    } else if (op.kind == OP_BTRANS) {
      const BTrans& t = plan.btrans[op.idx];
      BTransArgs a;
      a.nb = t.nb; a.R = t.R; a.C = t.C;
      a.S = ar[t.arS] + t.offS;
      a.D = ar[t.arD] + t.offD;
      a.sS = op.fixed_only ? 0 : stride[t.arS];
      a.sD = op.fixed_only ? 0 : stride[t.arD];
      a.ar = t.ar; a.ai = t.ai;
      e = launch_btrans_f64(a, nr, st);
      ++launches;
    } else if (op.kind == OP_ZERO) {
      // a scratch buffer starts its lifetime at zero (buffers with disjoint lifetimes share memory)
      const ZeroSpec& z = plan.zeros[op.idx];
      const size_t pitch = (size_t)std::max<long long>(stride[z.arena], z.n) * sizeof(double2);
      if (nr == 1) {
        e = cudaMemsetAsync(ar[z.arena] + z.off, 0, (size_t)z.n * sizeof(double2), st);
      } else if (pitch <= (size_t)INT32_MAX) {
        e = cudaMemset2DAsync(ar[z.arena] + z.off, pitch, 0, (size_t)z.n * sizeof(double2), nr, st);
      } else {  // a 2-D memset's pitch is limited to 2^31 - 1 bytes: one range per vector
        for (int r = 0; r < nr && e == cudaSuccess; ++r)
          e = cudaMemsetAsync(ar[z.arena] + z.off + (long long)r * stride[z.arena], 0,
                              (size_t)z.n * sizeof(double2), st);
      }
    }
    if (prof) {
      cudaEventRecord(rec.b, st);
      prof_recs.push_back(rec);
    }
    nvtxRangePop();
    if (e != cudaSuccess) {
      static const char* kinds[] = {"gemm", "permute", "transpose", "zero"};
      const std::string what = std::string("kernel launch (") + kinds[op.kind] + " op '" + optag + "')";
      if (!ck(e, what.c_str())) return LRCC_ECUDA;
    }
  }
  if (prec > 0 && !capturing) return read_flag(st);
  return LRCC_OK;
}

lrcc_status Runtime::read_flag(cudaStream_t st) {
  int h = 0;
  if (!ck(cudaMemcpyAsync(&h, dflag, sizeof(int), cudaMemcpyDeviceToHost, st), "flag read") ||
      !ck(cudaStreamSynchronize(st), "flag sync"))
    return LRCC_ECUDA;
  if (h) {
    cudaMemsetAsync(dflag, 0, sizeof(int), st);
    err = "tensor-core GEMM: a bounded wait on an mbarrier gave up";
    return LRCC_ETIMEOUT;
  }
  return LRCC_OK;
}

void Runtime::drop_graphs() {
  for (auto& kv : graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  graphs.clear();
}

lrcc_status Runtime::apply(int transpose, int nrhs, cudaStream_t st, int prec, bool use_graphs, bool tune) {
  const lrcc_status s = apply_impl(transpose, nrhs, st, prec, use_graphs, tune);
  tuned = nullptr;
  return s;
}

lrcc_status Runtime::apply_impl(int transpose, int nrhs, cudaStream_t st, int prec, bool use_graphs, bool tune) {
  double2* ar[AR_COUNT] = {fix, in, out, scr, ws};
  tuned = nullptr;
  if (tune) {
    const auto tkey = std::make_tuple(transpose, nrhs, prec);
    auto it = tunings.find(tkey);
    if (it == tunings.end()) {
      // the tuning launches need the product's intermediates in place: one eager
      // product first, then the timing pass (its accumulations are discarded by the
      // product that follows)
      const Program& tp = transpose ? jacT : plan.jac;
      double2* r0 = transpose ? in : out;
      if (!ck(cudaMemsetAsync(r0, 0, plan.arena_size[AR_IN] * nrhs * sizeof(double2), st), "cudaMemsetAsync"))
        return LRCC_ECUDA;
      lrcc_status s0 = run(tp, ar, nrhs, st, prec);
      if (s0 != LRCC_OK) return s0;
      std::map<int, GemmChoice> m;
      if ((s0 = autotune(tp, ar, nrhs, st, prec, m)) != LRCC_OK) return s0;
      it = tunings.emplace(tkey, std::move(m)).first;
      drop_graphs();  // captured with the default choices
    }
    tuned = &it->second;
  }
  const int64_t vin = plan.arena_size[AR_IN];
  // zero the result side (every op accumulates); scratch buffers are zeroed by the
  // program's own zero ops at the start of their lifetimes
  double2* res = transpose ? in : out;
  const Program& pr = transpose ? jacT : plan.jac;
  if (nrhs > scr_rhs) {  // scratch holds fewer vectors than the batch: chunks, no graph
    if (!ck(cudaMemsetAsync(res, 0, vin * nrhs * sizeof(double2), st), "cudaMemsetAsync")) return LRCC_ECUDA;
    return run_chunked(pr, nrhs, st, prec);
  }
  if (!use_graphs || prof) {
    if (!ck(cudaMemsetAsync(res, 0, vin * nrhs * sizeof(double2), st), "cudaMemsetAsync")) return LRCC_ECUDA;
    return run(pr, ar, nrhs, st, prec);
  }
  const auto key = std::make_tuple(transpose, nrhs, prec);
  const void* bufs[5] = {in, out, scr, part, packscr};
  auto it = graphs.find(key);
  bool valid = it != graphs.end() && it->second.version == fix_version;
  if (valid)
    for (int i = 0; i < 5; ++i) valid = valid && it->second.bufs[i] == bufs[i];
  if (!valid) {
    if (it != graphs.end()) {
      if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
      graphs.erase(it);
    }
    // an eager product first: it allocates whatever the product needs (split-K
    // partials, packed operands) and repacks fixed operands, so the capture that
    // follows records kernels only
    if (!ck(cudaMemsetAsync(res, 0, vin * nrhs * sizeof(double2), st), "cudaMemsetAsync")) return LRCC_ECUDA;
    lrcc_status s = run(pr, ar, nrhs, st, prec);
    if (s != LRCC_OK) return s;
    if (!ck(cudaStreamSynchronize(st), "graph: sync before capture")) return LRCC_ECUDA;
    const void* after[5] = {in, out, scr, part, packscr};
    GraphRec rec;
    rec.version = fix_version;
    for (int i = 0; i < 5; ++i) rec.bufs[i] = after[i];
    cudaStream_t cs = nullptr;
    if (!ck(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "graph: capture stream")) return LRCC_ECUDA;
    cudaGraph_t g = nullptr;
    capturing = true;
    const long long l0 = launches;
    bool ok = ck(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "graph: begin capture");
    if (ok) {
      ok = ck(cudaMemsetAsync(res, 0, vin * nrhs * sizeof(double2), cs), "graph: memset");
      lrcc_status rs = ok ? run(pr, ar, nrhs, cs, prec) : LRCC_ECUDA;
      const bool ended = ck(cudaStreamEndCapture(cs, &g), "graph: end capture");
      ok = ok && rs == LRCC_OK && ended;
    }
    capturing = false;
    rec.nlaunch = launches - l0;
    launches = l0;  // the captured kernels run when the graph is launched
    const void* post[5] = {in, out, scr, part, packscr};
    for (int i = 0; i < 5; ++i) ok = ok && post[i] == after[i];
    if (ok) ok = ck(cudaGraphInstantiate(&rec.exec, g, 0), "graph: instantiate");
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (!ok) {
      if (rec.exec) cudaGraphExecDestroy(rec.exec);
      if (err.empty()) err = "graph capture of the product failed";
      return LRCC_ECUDA;
    }
    graphs[key] = rec;
    return prec > 0 ? read_flag(st) : LRCC_OK;  // this call's result is the eager product's
  }
  if (!ck(cudaGraphLaunch(it->second.exec, st), "cudaGraphLaunch")) return LRCC_ECUDA;
  ++graph_launches;
  launches += it->second.nlaunch;
  return prec > 0 ? read_flag(st) : LRCC_OK;
}

}  // namespace lrcc

using namespace lrcc;


static lrcc_status fail(lrcc_problem* p, lrcc_status s, const std::string& m) {
  if (p) p->rt.err = m;
  return s;
}

extern "C" {

void lrcc_default_options(lrcc_options* o) {
  if (!o) return;
  o->conv_tol = 1e-10;
  o->refine_tol = 1e-7;
  o->max_iter = 200;
  o->diis_depth = 8;
  o->diis_period = 1;
  o->precision = 0;
  o->autotune = 0;
  o->use_graphs = 0;
  o->spin_timeout_cycles = 0;
  o->response_form = 0;
  o->log_path = nullptr;
  o->max_batch = 0;
  o->host_history = 0;
}

lrcc_status lrcc_create(const lrcc_dims* dims, lrcc_problem** out) {
  if (!dims || !out) return LRCC_EINVAL;
  *out = nullptr;
  if (dims->nk < 1 || dims->nocc < 1 || dims->nvir < 1 || dims->naux < 1 || dims->kmesh < 0 || dims->kmesh > 2)
    return LRCC_EINVAL;
  lrcc_problem* p = new (std::nothrow) lrcc_problem();
  if (!p) return LRCC_ENOMEM;
  // W-block workspace: up to ~1 GiB of complex128 (at least one block)
  lrcc_status s = p->rt.init(*dims, (int64_t)1 << 26);
  if (s != LRCC_OK) {
    // keep the handle so that lrcc_last_error can report; caller must destroy
    *out = p;
    return s;
  }
  *out = p;
  return LRCC_OK;
}

void lrcc_destroy(lrcc_problem* p) {
  if (!p) return;
  p->rt.release();
  delete p;
}

const char* lrcc_last_error(const lrcc_problem* p) {
  if (!p) return "null problem handle";
  return p->rt.err.c_str();
}

lrcc_status lrcc_set_integrals(lrcc_problem* p, const void* L, const double* eps, const void* dip,
                               int32_t on_device) {
  if (!p || !L || !eps || !dip) return fail(p, LRCC_EINVAL, "set_integrals: null argument");
  Runtime& rt = p->rt;
  if (!rt.fix) return fail(p, LRCC_EINVAL, "set_integrals: problem not initialised");
  const int nk = rt.dims.nk, o = rt.dims.nocc, v = rt.dims.nvir, Q = rt.dims.naux, n = o + v;
  const Plan& P = rt.plan;
  const size_t Lbytes = (size_t)nk * nk * Q * n * n * sizeof(double2);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  // validation before anything is uploaded (a rejected call leaves the problem unchanged):
  // finite values; DF factors Hermitian in (p,k1) <-> (q,k2), which the method's exchange
  // symmetry of the integrals relies on (Sec. II.C); dipoles Hermitian per k; a gapped
  // reference (every virtual above every occupied level), which the denominators of
  // Eq. 9 need.
  {
    std::vector<double2> hl, hd;
    const double2* Lh = (const double2*)L;
    const double2* Dh = (const double2*)dip;
    const double* Eh = eps;
    std::vector<double> he;
    const size_t nL = (size_t)nk * nk * Q * n * n, nD = (size_t)3 * nk * n * n;
    if (on_device) {
      hl.resize(nL);
      hd.resize(nD);
      he.resize((size_t)nk * n);
      if (!rt.ck(cudaMemcpy(hl.data(), L, Lbytes, cudaMemcpyDeviceToHost), "cudaMemcpy(L to host)") ||
          !rt.ck(cudaMemcpy(hd.data(), dip, nD * sizeof(double2), cudaMemcpyDeviceToHost), "cudaMemcpy(dip)") ||
          !rt.ck(cudaMemcpy(he.data(), eps, he.size() * sizeof(double), cudaMemcpyDeviceToHost), "cudaMemcpy(eps)"))
        return LRCC_ECUDA;
      Lh = hl.data();
      Dh = hd.data();
      Eh = he.data();
    }
    double lmax = 0.0, lerr = 0.0;
    for (size_t i = 0; i < nL; ++i) {
      if (!std::isfinite(Lh[i].x) || !std::isfinite(Lh[i].y))
        return fail(p, LRCC_EINVAL, "set_integrals: non-finite DF factor");
      lmax = std::max(lmax, std::hypot(Lh[i].x, Lh[i].y));
    }
    auto li = [&](int k1, int k2, int q, int a, int b) { return (((size_t)k1 * nk + k2) * Q + q) * n * n + (size_t)a * n + b; };
    for (int k1 = 0; k1 < nk; ++k1)
      for (int k2 = 0; k2 < nk; ++k2)
        for (int q = 0; q < Q; ++q)
          for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) {
              const double2 x = Lh[li(k1, k2, q, a, b)], y = Lh[li(k2, k1, q, b, a)];
              lerr = std::max(lerr, std::hypot(x.x - y.x, x.y + y.y));
            }
    if (lerr > 1e-10 * std::max(lmax, 1e-300))
      return fail(p, LRCC_EINVAL, "set_integrals: DF factors are not Hermitian (max |L(k2,k1)^H - L(k1,k2)| = " +
                                      std::to_string(lerr) + ")");
    double dmax = 0.0, derr = 0.0;
    for (size_t i = 0; i < nD; ++i) {
      if (!std::isfinite(Dh[i].x) || !std::isfinite(Dh[i].y))
        return fail(p, LRCC_EINVAL, "set_integrals: non-finite dipole integral");
      dmax = std::max(dmax, std::hypot(Dh[i].x, Dh[i].y));
    }
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < nk; ++k)
        for (int a = 0; a < n; ++a)
          for (int b = 0; b < n; ++b) {
            const double2 x = Dh[(((size_t)c * nk + k) * n + a) * n + b], y = Dh[(((size_t)c * nk + k) * n + b) * n + a];
            derr = std::max(derr, std::hypot(x.x - y.x, x.y + y.y));
          }
    if (derr > 1e-10 * std::max(dmax, 1e-300))
      return fail(p, LRCC_EINVAL, "set_integrals: dipole integrals are not Hermitian");
    double occ_max = -1e300, vir_min = 1e300;
    for (int k = 0; k < nk; ++k)
      for (int q = 0; q < n; ++q) {
        const double x = Eh[(size_t)k * n + q];
        if (!std::isfinite(x)) return fail(p, LRCC_EINVAL, "set_integrals: non-finite orbital energy");
        if (q < o) occ_max = std::max(occ_max, x);
        else vir_min = std::min(vir_min, x);
      }
    if (!(vir_min > occ_max))
      return fail(p, LRCC_EINVAL, "set_integrals: the reference is not gapped (lowest virtual energy not above "
                                  "the highest occupied one)");
  }
  double2* tmp = nullptr;
  if (!rt.ck(cudaMalloc(&tmp, Lbytes), "cudaMalloc(L staging)")) return LRCC_ENOMEM;
  lrcc_status st = LRCC_OK;
  if (!rt.ck(cudaMemcpy(tmp, L, Lbytes, kind), "cudaMemcpy(L)")) st = LRCC_ECUDA;
  if (st == LRCC_OK &&
      !rt.ck(launch_split_df(tmp, nk, Q, o, v, 1.0 / std::sqrt((double)nk), rt.fix + P.off_Loo, rt.fix + P.off_Lov,
                             rt.fix + P.off_Lvo, rt.fix + P.off_Lvv, 0),
             "split_df"))
    st = LRCC_ECUDA;
  if (st == LRCC_OK && !rt.ck(cudaDeviceSynchronize(), "split_df sync")) st = LRCC_ECUDA;
  cudaFree(tmp);
  if (st != LRCC_OK) return st;
  // orbital energies -> f0 = diag(eps) per k ; identity o x o
  std::vector<double> e((size_t)nk * n);
  if (on_device) {
    if (!rt.ck(cudaMemcpy(e.data(), eps, e.size() * sizeof(double), cudaMemcpyDeviceToHost), "cudaMemcpy(eps)"))
      return LRCC_ECUDA;
  } else {
    std::memcpy(e.data(), eps, e.size() * sizeof(double));
  }
  for (double x : e)
    if (!std::isfinite(x)) return fail(p, LRCC_EINVAL, "set_integrals: non-finite orbital energy");
  rt.eps = e;
  std::vector<double2> f0((size_t)nk * n * n, make_double2(0.0, 0.0));
  for (int k = 0; k < nk; ++k)
    for (int q = 0; q < n; ++q) f0[((size_t)k * n + q) * n + q].x = e[(size_t)k * n + q];
  std::vector<double2> idv((size_t)o * o, make_double2(0.0, 0.0));
  for (int i = 0; i < o; ++i) idv[(size_t)i * o + i].x = 1.0;
  if (!rt.ck(cudaMemcpy(rt.fix + P.off_f0, f0.data(), f0.size() * sizeof(double2), cudaMemcpyHostToDevice),
             "cudaMemcpy(f0)") ||
      !rt.ck(cudaMemcpy(rt.fix + P.off_idv, idv.data(), idv.size() * sizeof(double2), cudaMemcpyHostToDevice),
             "cudaMemcpy(identity)") ||
      !rt.ck(cudaMemcpy(rt.dip, dip, (size_t)3 * nk * n * n * sizeof(double2), kind), "cudaMemcpy(dipoles)"))
    return LRCC_ECUDA;
  rt.dip_host.resize((size_t)3 * nk * n * n);
  if (!rt.ck(cudaMemcpy(rt.dip_host.data(), rt.dip, rt.dip_host.size() * sizeof(double2), cudaMemcpyDeviceToHost),
             "cudaMemcpy(dipoles to host)"))
    return LRCC_ECUDA;
  p->have_int = true;
  p->have_t = false;
  return LRCC_OK;
}

lrcc_status lrcc_set_ground_state(lrcc_problem* p, const void* t1, const void* t2, const void* l1, const void* l2,
                                  int32_t on_device) {
  if (!p || !t1 || !t2) return fail(p, LRCC_EINVAL, "set_ground_state: null amplitude pointer");
  if (!p->have_int) return fail(p, LRCC_EINVAL, "set_ground_state: integrals not set");
  Runtime& rt = p->rt;
  const Plan& P = rt.plan;
  const int nk = rt.dims.nk, o = rt.dims.nocc, v = rt.dims.nvir;
  const size_t n1 = (size_t)nk * o * v, n2 = (size_t)nk * nk * nk * o * o * v * v;
  {  // finite amplitudes and multipliers (host data checked in place, device data copied)
    const void* arrs[4] = {t1, t2, l1, l2};
    const size_t cnt[4] = {n1, n2, n1, n2};
    for (int a = 0; a < 4; ++a) {
      if (!arrs[a]) continue;
      std::vector<double2> h;
      const double2* x = (const double2*)arrs[a];
      if (on_device) {
        h.resize(cnt[a]);
        if (!rt.ck(cudaMemcpy(h.data(), arrs[a], cnt[a] * sizeof(double2), cudaMemcpyDeviceToHost), "validate"))
          return LRCC_ECUDA;
        x = h.data();
      }
      for (size_t i = 0; i < cnt[a]; ++i)
        if (!std::isfinite(x[i].x) || !std::isfinite(x[i].y))
          return fail(p, LRCC_EINVAL, "set_ground_state: non-finite amplitude or multiplier");
    }
  }
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (!rt.ck(cudaMemset(rt.fix + P.off_derived, 0, (P.arena_size[AR_FIX] - P.off_derived) * sizeof(double2)),
             "cudaMemset(derived)") ||
      !rt.ck(cudaMemcpy(rt.fix + P.off_t1, t1, n1 * sizeof(double2), kind), "cudaMemcpy(t1)") ||
      !rt.ck(cudaMemcpy(rt.fix + P.off_t2, t2, n2 * sizeof(double2), kind), "cudaMemcpy(t2)"))
    return LRCC_ECUDA;
  if (l1 && l2) {
    if (!rt.l1 && !rt.ck(cudaMalloc(&rt.l1, n1 * sizeof(double2)), "cudaMalloc(l1)")) return LRCC_ENOMEM;
    if (!rt.l2 && !rt.ck(cudaMalloc(&rt.l2, n2 * sizeof(double2)), "cudaMalloc(l2)")) return LRCC_ENOMEM;
    if (!rt.ck(cudaMemcpy(rt.l1, l1, n1 * sizeof(double2), kind), "cudaMemcpy(l1)") ||
        !rt.ck(cudaMemcpy(rt.l2, l2, n2 * sizeof(double2), kind), "cudaMemcpy(l2)"))
      return LRCC_ECUDA;
    p->have_l = true;
  }
  double2* ar[AR_COUNT] = {rt.fix, nullptr, nullptr, nullptr, rt.ws};
  lrcc_status s = rt.run(P.ground, ar, 1, 0);
  if (s != LRCC_OK) return s;
  if (!rt.ck(cudaDeviceSynchronize(), "ground-state program")) return LRCC_ECUDA;
  p->have_t = true;
  return LRCC_OK;
}

// Strided device-to-device copy of `rows` rows of `width` bytes.  A 2-D copy's pitches are
// limited to 2^31 - 1 bytes, and a vector arena of the larger workloads is wider than that
// (6.9 GB per vector at Nk=9, nocc=12, nvir=64): then one copy per row.
static cudaError_t copy_rows(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, int rows,
                             cudaStream_t st) {
  if (rows == 1) return cudaMemcpyAsync(dst, src, width, cudaMemcpyDeviceToDevice, st);
  if (dpitch <= (size_t)INT32_MAX && spitch <= (size_t)INT32_MAX)
    return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows, cudaMemcpyDeviceToDevice, st);
  cudaError_t e = cudaSuccess;
  for (int r = 0; r < rows && e == cudaSuccess; ++r)
    e = cudaMemcpyAsync((char*)dst + r * dpitch, (const char*)src + r * spitch, width, cudaMemcpyDeviceToDevice, st);
  return e;
}

lrcc_status lrcc_jacobian_apply(lrcc_problem* p, int32_t transpose, int32_t nrhs, const void* x1, const void* x2,
                                void* y1, void* y2, const lrcc_options* opt, void* stream) {
  if (!p) return LRCC_EINVAL;
  if (!p->have_t) return fail(p, LRCC_EINVAL, "jacobian_apply: ground state not set");
  if (nrhs < 1 || !x1 || !x2 || !y1 || !y2 || (transpose != 0 && transpose != 1))
    return fail(p, LRCC_EINVAL, "jacobian_apply: bad arguments");
  const int prec = opt ? opt->precision : 0;
  if (prec < 0 || prec > 2) return fail(p, LRCC_EINVAL, "jacobian_apply: precision must be 0, 1 or 2");
  Runtime& rt = p->rt;
  rt.max_batch = opt ? std::max(0, opt->max_batch) : 0;
  lrcc_status s = rt.ensure_rhs(nrhs);
  if (s != LRCC_OK) return s;
  // a null handle is the caller's legacy default stream (this library is built with
  // per-thread default streams, under which 0 would name the calling thread's stream)
  cudaStream_t st = stream ? (cudaStream_t)stream : cudaStreamLegacy;
  const Plan& P = rt.plan;
  const int nk = rt.dims.nk, o = rt.dims.nocc, v = rt.dims.nvir;
  const size_t b1 = (size_t)nk * o * v * sizeof(double2), b2 = (size_t)nk * nk * nk * o * o * v * v * sizeof(double2);
  const size_t pitch = (size_t)P.arena_size[AR_IN] * sizeof(double2);
  double2* src = transpose ? rt.out : rt.in;
  double2* dst = transpose ? rt.in : rt.out;
  if (!rt.ck(copy_rows(src + P.off_x1, pitch, x1, b1, b1, nrhs, st), "copy x1") ||
      !rt.ck(copy_rows(src + P.off_x2, pitch, x2, b2, b2, nrhs, st), "copy x2"))
    return LRCC_ECUDA;
  s = rt.apply(transpose, nrhs, st, prec, opt && opt->use_graphs, opt && opt->autotune);
  if (s != LRCC_OK) return s;
  if (!rt.ck(copy_rows(y1, b1, dst + P.off_x1, pitch, b1, nrhs, st), "copy y1") ||
      !rt.ck(copy_rows(y2, b2, dst + P.off_x2, pitch, b2, nrhs, st), "copy y2"))
    return LRCC_ECUDA;
  return LRCC_OK;
}

lrcc_status lrcc_polarizability(lrcc_problem* p, const int32_t* comps, int32_t ncomp, const double* omegas,
                                int32_t nomega, const lrcc_options* opt, void* alpha, int32_t* info) {
  if (!p) return LRCC_EINVAL;
  return lrcc_polarize_impl(p->rt, p->have_t, p->have_l, comps, ncomp, omegas, nomega, opt, alpha, info);
}

lrcc_status lrcc_polarizability_forms(lrcc_problem* p, const int32_t* comps, int32_t ncomp, const double* omegas,
                                      int32_t nomega, const lrcc_options* opt, void* alpha_sym, void* alpha_asym,
                                      int32_t* info) {
  if (!p) return LRCC_EINVAL;
  if (!alpha_sym || !alpha_asym) return fail(p, LRCC_EINVAL, "polarizability_forms: null output");
  lrcc_options o;
  lrcc_default_options(&o);
  if (opt) o = *opt;
  o.response_form = 2;
  return lrcc_polarize_impl(p->rt, p->have_t, p->have_l, comps, ncomp, omegas, nomega, &o, alpha_asym, info, nullptr,
                            alpha_sym);
}

lrcc_status lrcc_response_function(lrcc_problem* p, int32_t nops, const void* ops, const double* omegas,
                                   int32_t nomega, const lrcc_options* opt, void* out, int32_t* info) {
  if (!p) return LRCC_EINVAL;
  Runtime& rt = p->rt;
  if (!ops || nops < 1 || nops > 16 || !out) return fail(p, LRCC_EINVAL, "response_function: bad arguments");
  const int nk = rt.dims.nk, n = rt.dims.nocc + rt.dims.nvir;
  const double2* X = (const double2*)ops;
  const size_t per = (size_t)nk * n * n;
  for (int c = 0; c < nops; ++c) {
    double xmax = 0.0, herr = 0.0;
    for (size_t i = 0; i < per; ++i) {
      const double2 x = X[c * per + i];
      if (!std::isfinite(x.x) || !std::isfinite(x.y))
        return fail(p, LRCC_EINVAL, "response_function: non-finite operator matrix element");
      xmax = std::max(xmax, std::hypot(x.x, x.y));
    }
    for (int k = 0; k < nk; ++k)
      for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
          const double2 x = X[c * per + ((size_t)k * n + a) * n + b], y = X[c * per + ((size_t)k * n + b) * n + a];
          herr = std::max(herr, std::hypot(x.x - y.x, x.y + y.y));
        }
    if (herr > 1e-10 * std::max(xmax, 1e-300))
      return fail(p, LRCC_EINVAL, "response_function: operator " + std::to_string(c) + " is not Hermitian");
  }
  const lrcc_status s =
      lrcc_polarize_impl(rt, p->have_t, p->have_l, nullptr, nops, omegas, nomega, opt, out, info, X);
  if (s != LRCC_OK) return s;
  // the driver returns alpha = -<<X;Y>>; this call returns the response function itself
  double2* r = (double2*)out;
  for (size_t i = 0; i < (size_t)nomega * nops * nops; ++i) r[i] = make_double2(-r[i].x, -r[i].y);
  return LRCC_OK;
}

lrcc_status lrcc_batch_polarizability(lrcc_problem* const* probs, int32_t nprob, const int32_t* comps,
                                      int32_t ncomp, const double* omegas, int32_t nomega,
                                      const lrcc_options* opt, void* const* alphas, int32_t* const* infos) {
  if (!probs || nprob < 1 || !alphas) return LRCC_EINVAL;
  for (int i = 0; i < nprob; ++i)
    for (int j = 0; j < i; ++j)
      if (probs[i] == probs[j]) return LRCC_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LRCC_ECUDA;
  std::vector<lrcc_status> st(nprob, LRCC_OK);
  std::vector<std::thread> th;
  for (int i = 0; i < nprob; ++i) {
    if (!probs[i] || !alphas[i]) {
      st[i] = LRCC_EINVAL;
      continue;
    }
    th.emplace_back([&, i]() {
      lrcc::Runtime& rt = probs[i]->rt;
      try {
        if (!rt.ck(cudaSetDevice(dev), "batch: cudaSetDevice")) {
          st[i] = LRCC_ECUDA;
          return;
        }
        st[i] = lrcc_polarize_impl(rt, probs[i]->have_t, probs[i]->have_l, comps, ncomp, omegas, nomega, opt,
                                   alphas[i], infos ? infos[i] : nullptr);
        if (!rt.ck(cudaStreamSynchronize(cudaStreamPerThread), "batch: stream sync") && st[i] == LRCC_OK)
          st[i] = LRCC_ECUDA;
      } catch (const std::bad_alloc&) {
        rt.err = "batch: host allocation failed";
        st[i] = LRCC_ENOMEM;
      } catch (...) {
        rt.err = "batch: unexpected host exception";
        st[i] = LRCC_EINVAL;
      }
    });
  }
  for (auto& t : th) t.join();
  for (int i = 0; i < nprob; ++i)
    if (st[i] != LRCC_OK) return st[i];
  return LRCC_OK;
}

lrcc_status lrcc_wait_selftest(lrcc_problem* p, int64_t polls) {
  if (!p || polls < 1) return LRCC_EINVAL;
  Runtime& rt = p->rt;
  if (!rt.ck(launch_wait_selftest(polls, rt.dflag, cudaStreamLegacy), "wait self test")) return LRCC_ECUDA;
  ++rt.launches;
  const lrcc_status s = rt.read_flag(cudaStreamLegacy);
  if (s == LRCC_ETIMEOUT) rt.err = "wait self test: the bounded wait gave up as intended";
  return s;
}

int64_t lrcc_kernel_launches(const lrcc_problem* p) { return p ? p->rt.launches : -1; }

lrcc_status lrcc_profile(lrcc_problem* p, int32_t enable) {
  if (!p) return LRCC_EINVAL;
  p->rt.prof_reset();
  p->rt.prof = enable != 0;
  return LRCC_OK;
}

lrcc_status lrcc_profile_query(lrcc_problem* p, const char* tag, double* ms, int64_t* count, double* flops) {
  if (!p || !tag) return LRCC_EINVAL;
  Runtime& rt = p->rt;
  if (!rt.ck(cudaDeviceSynchronize(), "profile sync")) return LRCC_ECUDA;
  double t = 0.0, f = 0.0;
  int64_t c = 0;
  const std::string want(tag);
  for (auto& r : rt.prof_recs) {
    if (!want.empty() && r.tag != want) continue;
    float x = 0.f;
    if (!rt.ck(cudaEventElapsedTime(&x, r.a, r.b), "cudaEventElapsedTime")) return LRCC_ECUDA;
    t += x;
    f += r.flops;
    ++c;
  }
  if (ms) *ms = t;
  if (count) *count = c;
  if (flops) *flops = f;
  return LRCC_OK;
}

lrcc_status lrcc_profile_report(lrcc_problem* p, char* buf, int64_t len) {
  if (!p || !buf || len < 1) return LRCC_EINVAL;
  Runtime& rt = p->rt;
  if (!rt.ck(cudaDeviceSynchronize(), "profile sync")) return LRCC_ECUDA;
  struct Agg {
    double ms = 0.0, flops = 0.0;
    int64_t n = 0;
  };
  std::map<std::string, Agg> agg;
  for (auto& r : rt.prof_recs) {
    float x = 0.f;
    if (!rt.ck(cudaEventElapsedTime(&x, r.a, r.b), "cudaEventElapsedTime")) return LRCC_ECUDA;
    Agg& a = agg[r.tag];
    a.ms += x;
    a.flops += r.flops;
    ++a.n;
  }
  std::vector<std::pair<std::string, Agg>> v(agg.begin(), agg.end());
  std::sort(v.begin(), v.end(), [](const auto& x, const auto& y) { return x.second.ms > y.second.ms; });
  std::string out;
  char line[256];
  for (auto& e : v) {
    std::snprintf(line, sizeof(line), "%s\t%.6f\t%lld\t%.6e\n", e.first.c_str(), e.second.ms, (long long)e.second.n,
                  e.second.flops);
    out += line;
  }
  const size_t n = std::min<size_t>(out.size(), (size_t)len - 1);
  std::memcpy(buf, out.data(), n);
  buf[n] = 0;
  return out.size() < (size_t)len ? LRCC_OK : LRCC_EINVAL;
}

}  // extern "C"
