// solve_impl.cuh -- host-side pieces of the solve driver shared by the plain,
// defect-correction, batched, multi-graph and adjoint paths.
#pragma once

#include "common.cuh"
#include "sweep.cuh"

namespace fpr {

pr_status validate_options(const pr_options *o);
pr_status check_device(pr_graph *g);
pr_status ensure_workspace(pr_graph *g, cudaStream_t s);
// validation, work items for the options' thresholds, workspace
pr_status prepare_solve(pr_graph *g, const pr_options *o, pr_tune &tn, cudaStream_t s);
// Sweep parameters over the degree-ordered in-lists; stored vectors of
// `elem` bytes per vertex in ybuf; the staged copy takes the shared memory
// left beside the warp slices of this arithmetic (fp64) and variant (gs).
void fill_params(pr_graph *g, SweepParams &p, bool fp64, size_t elem, bool perf);

// Grid of a persistent sweep kernel over `nitems` warp items with `smem`
// bytes of dynamic shared memory (0 with the error set if it does not fit).
unsigned sweep_grid(const pr_graph *g, int nitems, const void *func, size_t smem);

// The launches of one sweep: one launch over all items, or for the fused
// sweep the hub segments and widest mid groups first, writing their new
// values aside, a copy of those into the stored vector, then the rest (so
// the second launch, its staged copy included, reads the new values).
struct SweepPlan {
    const void *func = nullptr;
    size_t smem = 0;
    int nlaunch = 0;
    unsigned block = SWEEP_BS;
    unsigned grid[2] = {0, 0};
    SweepParams p[2];
    // copy between the two launches (copy_func null: none)
    const void *copy_func = nullptr;
    unsigned copy_grid = 0;
    const SolveState *copy_st = nullptr;
    const void *copy_src = nullptr;
    void *copy_dst = nullptr;
    int32_t copy_n = 0;
};
// kernel launches of one sweep of the plan
inline int plan_launches(const SweepPlan &plan)
{
    return plan.nlaunch + (plan.nlaunch > 1 && plan.copy_func ? 1 : 0);
}
template <typename T, typename A>
pr_status make_plan(pr_graph *g, const SweepParams &p, bool gs, SweepPlan &plan);
// adds the plan's launches as a chain of kernel nodes of `body` (the last
// node in *last, if given)
pr_status add_plan_nodes(cudaGraph_t body, SweepPlan &plan, cudaGraphConditionalHandle h,
                         cudaGraphNode_t *last);
// launches one sweep of the plan (no graph)
pr_status launch_plan(SweepPlan &plan, cudaStream_t s);
// Instantiates (or reuses) a graph: WHILE(cond) { the plan's launches }.
pr_status loop_graph(pr_graph *g, int key, SweepPlan &plan, cudaGraphExec_t *exec_out);
void init_state(pr_graph *g, const pr_options *o, SolveState &h);
pr_status finish_result(pr_graph *g, pr_result *res, cudaStream_t s, int outer);
pr_status solve_dc(pr_graph *g, const pr_options *o, const pr_tune &tn, double *x_out,
                   pr_result *res, cudaStream_t s);
// propagation-blocked Jacobi (blocked.cu)
pr_status solve_blocked(pr_graph *g, const pr_options *o, double *x_out, pr_result *res,
                        cudaStream_t s);

}  // namespace fpr
