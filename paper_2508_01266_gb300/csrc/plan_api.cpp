// Host-only introspection of a Jacobian plan (declared in include/lrcc.h).
// These calls never touch the GPU; they expose the op list so that its index
// arithmetic can be checked on a machine without a GPU.
#include <cstring>
#include <exception>
#include <string>

#include "../../include/lrcc.h"
#include "plan.h"

using namespace lrcc;

struct lrcc_plan {
  Plan P;
  Program jacT;
  std::string err;
};

const Plan* lrcc::plan_of(const lrcc_plan* h) { return h ? &h->P : nullptr; }

static const Program& prog_of(const lrcc_plan* h, int which) {
  switch (which) {
    case 0: return h->P.ground;
    case 1: return h->P.jac;
    case 2: return h->jacT;
    case 3: return h->P.xi;
    case 4: return h->P.egrad;
    case 5: return h->P.omega0;
    default: return h->P.tgrad;
  }
}

extern "C" {

lrcc_status lrcc_plan_create(const lrcc_dims* dims, int64_t ws_budget, lrcc_plan** out) {
  if (!dims || !out) return LRCC_EINVAL;
  *out = nullptr;
  if (dims->nk < 1 || dims->nocc < 1 || dims->nvir < 1 || dims->naux < 1) return LRCC_EINVAL;
  try {
    lrcc_plan* h = new lrcc_plan();
    Dims d{dims->nk, dims->nocc, dims->nvir, dims->naux};
    h->P = build_plan(d, ws_budget > 0 ? ws_budget : (int64_t)1 << 26);
    h->jacT = transpose_program(h->P, h->P.jac);
    *out = h;
    return LRCC_OK;
  } catch (const std::bad_alloc&) {
    return LRCC_ENOMEM;
  } catch (...) {
    return LRCC_EINVAL;
  }
}

void lrcc_plan_destroy(lrcc_plan* h) { delete h; }

lrcc_status lrcc_plan_info(const lrcc_plan* h, int64_t* arena_sizes, int64_t* offsets, double* flops) {
  if (!h) return LRCC_EINVAL;
  const Plan& P = h->P;
  if (arena_sizes)
    for (int a = 0; a < AR_COUNT; ++a) arena_sizes[a] = P.arena_size[a];
  if (offsets) {
    int64_t o[11] = {P.off_Loo, P.off_Lov, P.off_Lvo, P.off_Lvv, P.off_f0, P.off_t1,
                     P.off_t2,  P.off_idv, P.off_x1,  P.off_x2,  P.off_mu};
    std::memcpy(offsets, o, sizeof(o));
  }
  if (flops) {
    flops[0] = P.jac_flops;
    flops[1] = P.ladder_flops;
    flops[2] = P.wbuild_flops;
  }
  return LRCC_OK;
}

int32_t lrcc_plan_num_ops(const lrcc_plan* h, int32_t which) {
  if (!h || which < 0 || which > 6) return -1;
  return (int32_t)prog_of(h, which).ops.size();
}

lrcc_status lrcc_plan_validate(const lrcc_plan* h, char* msg, int32_t len) {
  if (!h || !msg || len < 1) return LRCC_EINVAL;
  std::string e;
  for (int w = 0; w < 7 && e.empty(); ++w) e = validate_plan(h->P, prog_of(h, w));
  std::strncpy(msg, e.c_str(), (size_t)len - 1);
  msg[len - 1] = 0;
  return e.empty() ? LRCC_OK : LRCC_EINVAL;
}

lrcc_status lrcc_plan_op(const lrcc_plan* h, int32_t which, int32_t i, int32_t* kind_idx_fixed) {
  if (!h || which < 0 || which > 6 || !kind_idx_fixed) return LRCC_EINVAL;
  const Program& pr = prog_of(h, which);
  if (i < 0 || i >= (int32_t)pr.ops.size()) return LRCC_EINVAL;
  kind_idx_fixed[0] = pr.ops[i].kind;
  kind_idx_fixed[1] = pr.ops[i].idx;
  kind_idx_fixed[2] = pr.ops[i].fixed_only;
  return LRCC_OK;
}

lrcc_status lrcc_plan_gemm(const lrcc_plan* h, int32_t idx, int32_t* ints, int64_t* lds, double* alpha,
                           int64_t* coff, int32_t* sbeg, int64_t* aoff, int64_t* boff) {
  if (!h || idx < 0 || idx >= (int32_t)h->P.gemms.size()) return LRCC_EINVAL;
  const Gemm& g = h->P.gemms[idx];
  if (ints) {
    int32_t v[16] = {g.M,     g.N,     g.K,     g.ta,    g.tb,    g.arA,       g.arB,
                     g.arC,   g.epi,   g.ep[0], g.ep[1], g.ep[2], g.ep[3], g.nbatch(),
                     (int32_t)g.aoff.size(), g.store};
    std::memcpy(ints, v, sizeof(v));
  }
  if (lds) {
    lds[0] = g.lda;
    lds[1] = g.ldb;
    lds[2] = g.ldc;
  }
  if (alpha) {
    alpha[0] = g.ar;
    alpha[1] = g.ai;
  }
  if (coff) std::memcpy(coff, g.coff.data(), g.coff.size() * sizeof(int64_t));
  if (sbeg) std::memcpy(sbeg, g.sbeg.data(), g.sbeg.size() * sizeof(int32_t));
  if (aoff) std::memcpy(aoff, g.aoff.data(), g.aoff.size() * sizeof(int64_t));
  if (boff) std::memcpy(boff, g.boff.data(), g.boff.size() * sizeof(int64_t));
  return LRCC_OK;
}

lrcc_status lrcc_plan_perm(const lrcc_plan* h, int32_t idx, int32_t* ints, int64_t* offs, double* alpha) {
  if (!h || idx < 0 || idx >= (int32_t)h->P.perms.size()) return LRCC_EINVAL;
  const Perm& p = h->P.perms[idx];
  if (ints) {
    int32_t v[19] = {p.src.kind, p.src.nk, p.src.n[0], p.src.n[1], p.src.n[2], p.src.n[3],
                     p.dst.kind, p.dst.nk, p.dst.n[0], p.dst.n[1], p.dst.n[2], p.dst.n[3],
                     p.pi[0],    p.pi[1],  p.pi[2],    p.pi[3],    p.arS,      p.arD,
                     p.store};
    std::memcpy(ints, v, sizeof(v));
  }
  if (offs) {
    offs[0] = p.offS;
    offs[1] = p.offD;
  }
  if (alpha) {
    alpha[0] = p.ar;
    alpha[1] = p.ai;
  }
  return LRCC_OK;
}

lrcc_status lrcc_plan_btrans(const lrcc_plan* h, int32_t idx, int32_t* ints, int64_t* offs, double* alpha) {
  if (!h || idx < 0 || idx >= (int32_t)h->P.btrans.size()) return LRCC_EINVAL;
  const BTrans& t = h->P.btrans[idx];
  if (ints) {
    int32_t v[5] = {t.nb, t.R, t.C, t.arS, t.arD};
    std::memcpy(ints, v, sizeof(v));
  }
  if (offs) {
    offs[0] = t.offS;
    offs[1] = t.offD;
  }
  if (alpha) {
    alpha[0] = t.ar;
    alpha[1] = t.ai;
  }
  return LRCC_OK;
}

}  // extern "C"

lrcc_status lrcc_plan_zero(const lrcc_plan* h, int32_t idx, int32_t* arena, int64_t* off_n) {
  if (!h || idx < 0 || idx >= (int32_t)h->P.zeros.size()) return LRCC_EINVAL;
  const ZeroSpec& z = h->P.zeros[idx];
  if (arena) *arena = z.arena;
  if (off_n) {
    off_n[0] = z.off;
    off_n[1] = z.n;
  }
  return LRCC_OK;
}
