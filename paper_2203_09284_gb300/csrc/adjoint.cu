// adjoint.cu -- reverse mode of the PageRank fixed point.
#include "solve_impl.cuh"

using namespace fpr;

extern "C" pr_status pr_backward(pr_graph *, const pr_options *, const double *, const double *,
                                 double *, double *, pr_result *, void *)
{
    set_error("pr_backward: not built yet");
    return PR_ERR_UNSUPPORTED;
}
