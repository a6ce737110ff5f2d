// Polarizability driver: placeholder until the response solver lands.
#include "runtime.h"

lrcc_status lrcc_polarize_impl(lrcc::Runtime& rt, bool have_t, bool have_l, const int32_t* comps, int32_t ncomp,
                               const double* omegas, int32_t nomega, const lrcc_options* opt, void* alpha,
                               int32_t* info) {
  (void)have_t; (void)have_l; (void)comps; (void)ncomp; (void)omegas; (void)nomega; (void)opt; (void)alpha;
  (void)info;
  rt.err = "polarizability: not available in this build";
  return LRCC_EUNSUPPORTED;
}
