// CRPQ evaluation (Definition 2).
#include "crpq.h"

namespace rpq {

int crpq_eval(rpq_ctx *ctx, const rpq_graph *, uint32_t, const int32_t *, const crpq_atom *, uint32_t,
              const uint32_t *, uint32_t, uint32_t, rpq_result **) {
  return ctx_error(ctx, RPQ_ERR_INVALID_ARG, "run_crpq is not available yet");
}

}  // namespace rpq
