// kernels.cuh -- kernel and shared-memory-size declarations shared by the
// kernel translation units and the host orchestration (api.cu).
#pragma once
#include "plan.cuh"

namespace eclqr {

// shared memory per task, in doubles
__host__ int smem_primal_sweep(int n, int m, int pmax, int qmax);
__host__ int smem_rel_level(int n, int pmax, int qmax);
__host__ int smem_param(int n);
__host__ int smem_elim(int n, int m, int pmax);
__host__ int smem_lqr_up(int n, int m);
__host__ int smem_lqr_level(int n);
__host__ int smem_riccati(int n, int m);
__host__ int smem_riccati_finish(int n, int m);
__host__ int smem_set_costs(int n, int m);
__host__ int smem_primal_stage(int n, int m, int wmax);
__host__ int smem_aff(int n, int m);
__host__ int smem_dual_stage(int n, int m);
__host__ int smem_dual_sweep(int n, int m, int pmax, int qmax);
__host__ int smem_dual_leaf(int n, int m, int wmax);
__host__ int smem_scan_check(int n, int m, int pmax);

// primal scan and elimination (k_primal.cu)
__global__ void k_scan_check(Group g, int per_task);
__global__ void k_skip_flags(Group g, int32_t *flags);
__global__ void k_terminal(Group g, int per_task);
__global__ void k_primal_up(Group g, int per_task);
__global__ void k_rel_level(Group g, int src, int d, int fail_code, int per_task);
__global__ void k_primal_down(Group g, int fin, int per_task, int *queue);
__global__ void k_primal_stage(Group g, int per_task);
__global__ void k_param(Group g, int per_task);
__global__ void __launch_bounds__(256, 4) k_elim(Group g, int per_task);

// reduced LQR, affine chains, recovery (k_lqr.cu)
enum { AFF_ROLL_ = 0, AFF_CROLL_ = 1, AFF_PLIN_ = 2, AFF_NU_ = 3 };
__global__ void k_lqr_up(Group g, int per_task);
__global__ void k_lqr_level(Group g, int src, int d, int per_task);
__global__ void k_riccati_down(Group g, int fin, int per_task, int *queue);
__global__ void k_riccati_finish(Group g, int per_task);
__global__ void k_riccati_down_f32(Group g, int fin, int per_task);  // k_mixed.cu
__global__ void k_aff_up(Group g, int mode, int per_task);
__global__ void k_aff_level(Group g, int src, int d, int fwd, int per_task);
__global__ void k_aff_down(Group g, int mode, int fin, int per_task);
__global__ void k_aff_prep(Group g, int mode, int per_task);
__global__ void k_solve_init(Group g, const double *s0);
__global__ void k_post_roll(Group g, int corr);
__global__ void k_resid(Group g, int per_task);
__global__ void k_pcorr(Group g, int per_task);
__global__ void k_recover(Group g, double *x, double *u);
__global__ void k_dims(Group g, int *nbar, int *mbar);

// multipliers and residual (k_dual.cu)
__global__ void __launch_bounds__(256, 3) k_dual_stage(Group g, const double *x, const double *u, int per_task);
__global__ void k_dual_terminal(Group g, int per_task);
__global__ void k_dual_up(Group g, int per_task);
__global__ void k_dual_down(Group g, int fin, int per_task);
__global__ void k_dual_root(Group g, int per_task);
__global__ void __launch_bounds__(256, 4) k_dual_leaf(Group g, double *lam, double *mu, double *eta, double *alpha, int per_task);
__global__ void k_param_grads(Group g, Sol w, Sol wb, GradOut o);
__global__ void k_set_costs(Group g, int per_task);
__global__ void k_kkt(Group g, const double *s0, const double *x, const double *u, const double *lam,
                      const double *mu, const double *eta, const double *alpha, KktRows rows, double *resid,
                      double *parts);

// refinement on the original KKT residual and non-finite checks (k_refine.cu)
__global__ void k_check_inputs(Group g);
__global__ void k_stage_lists(Group g, RefineMasks mk, int *lists, int *counts);
__global__ void k_refine_prep(Group g, const int32_t *status, const double *resid, const double *parts,
                              RefineMasks mk, int32_t *cstatus, double *tresid, double *tparts, double tol,
                              int first, int *any);
__global__ void k_refine_parts(Group g, const int *active, double *parts, const double *tparts,
                               const double *resid, const double *tresid);
__global__ void k_refine_gate(Group g, const int32_t *cstatus, int *active);
__global__ void k_refine_trial(Group g, Sol w, SolMut t);
__global__ void k_refine_accept(Group g, Sol t, double *x, double *u, double *lam, double *mu, double *eta,
                                double *alpha, const double *resid, const double *tresid);
__global__ void k_refine_post(Group g, double *resid, const double *tresid, int *active);
__global__ void k_rescue_prep(Group g, const int32_t *status, double *resid, double *parts, int *fp64, int *active,
                              double tol, int *any);

}  // namespace eclqr
