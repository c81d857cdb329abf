// Batched solves over several contexts (north of Sec. 5.2: the heatbath and
// force need many independent solves of Eq. (8)).
#include "api_util.h"

extern "C" {

int eofa_solve_batched(eofa_ctx* const* ctxs, int n, const eofa_solve_params* params, const double* const* b,
                       double* const* x, eofa_solve_info* info) {
    if (!ctxs || n < 0 || !params || !b || !x) return EOFA_EINVAL;
    int worst = EOFA_OK;
    for (int i = 0; i < n; i++) {
        int rc = eofa_solve(ctxs[i], &params[i], b[i], x[i], info ? &info[i] : nullptr);
        if (rc != EOFA_OK && worst == EOFA_OK) worst = rc;
    }
    return worst;
}

}  // extern "C"
