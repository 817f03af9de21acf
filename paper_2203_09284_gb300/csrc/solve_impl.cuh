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
void fill_params(pr_graph *g, SweepParams &p, bool fp64, size_t elem);
unsigned sweep_grid(const pr_graph *g, const SweepParams &p, const void *func, size_t smem);
pr_status loop_graph(pr_graph *g, int key, const void *func, unsigned grid, unsigned block,
                     size_t smem, SweepParams &p, cudaGraphExec_t *exec_out);
void init_state(pr_graph *g, const pr_options *o, SolveState &h);
pr_status finish_result(pr_graph *g, pr_result *res, cudaStream_t s, int outer);
pr_status solve_dc(pr_graph *g, const pr_options *o, const pr_tune &tn, double *x_out,
                   pr_result *res, cudaStream_t s);
template <typename T, typename A>
const void *pick_sweep(bool gs, bool weighted);
template <typename T, typename A>
size_t sweep_smem(const SweepParams &p, bool gs);

}  // namespace fpr
