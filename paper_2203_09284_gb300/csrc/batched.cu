// batched.cu -- personalised PageRank for many teleport vectors (multi
// right-hand-side sweep) and many graphs solved together.
#include "solve_impl.cuh"

using namespace fpr;

extern "C" pr_status pr_solve_batched(pr_graph *, const pr_options *, int32_t, const int32_t *,
                                      float *, pr_result *, void *)
{
    set_error("pr_solve_batched: not built yet");
    return PR_ERR_UNSUPPORTED;
}

extern "C" pr_status pr_solve_multi(pr_graph *const *, int32_t, const pr_options *,
                                    double *const *, pr_result *, void *)
{
    set_error("pr_solve_multi: not built yet");
    return PR_ERR_UNSUPPORTED;
}
