// lb_ops.h -- launchers of the precision-dependent kernels, one table per
// population storage type (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include "lb_common.cuh"

namespace lbp {

struct LbOps {
    int id;
    size_t real_size;
    cudaError_t (*setup)();
    // fused kernel: split = 0 k_step (32 x ty tiles), 1 k_step_split (16 x ty, ty 8 or 16);
    // reflect = 1: the fused kernel reflects at solid neighbours itself, 0: k_couple does
    cudaError_t (*step)(int par, int ty, int split, int tau1, int reflect, int ntiles, cudaStream_t st,
                        const BoxDev* boxes, const TileDev* tiles, Shared sh, int rc, int rn, int rz, int mslot);
    cudaError_t (*remap_apply)(int par, cudaStream_t st, const BoxDev* boxes, Shared sh, int rc, int mslot_cur);
    cudaError_t (*remap_finish)(cudaStream_t st, const BoxDev* boxes, Shared sh, int rc);
    cudaError_t (*shell_density)(cudaStream_t st, const BoxDev* boxes, Shared sh, int rc, int NP);
    // impl: some box uses the implicit velocity update (the drag tensor is summed)
    cudaError_t (*couple)(cudaStream_t st, const BoxDev* boxes, Shared sh, int rc, int rn, int mslot, int par,
                          int reflect, int impl, int NP);
    cudaError_t (*couple_correct)(cudaStream_t st, const BoxDev* boxes, Shared sh, int rc, int rn, int mslot, int par,
                                  int reflect, int NP);
    cudaError_t (*wall_shell)(cudaStream_t st, const BoxDev* boxes, int b, int rc);
    cudaError_t (*init_pop)(cudaStream_t st, const BoxDev* boxes, int b, const double* rho_field,
                            const double* u_field, uint64_t s_red, uint64_t s_blue, double noise, int rc,
                            double* mass_out);
    // direction i of both components, canonical order [2][N] doubles
    cudaError_t (*export_dir)(cudaStream_t st, const BoxDev* boxes, int b, int i, int par, int rc, double* out);
    cudaError_t (*import_dir)(cudaStream_t st, const BoxDev* boxes, int b, int i, int par, const double* in);
    cudaError_t (*rho_from_pop)(cudaStream_t st, const BoxDev* boxes, int b, int par, int src, int rc, double* out,
                                double* mass_out);
    cudaError_t (*obs_partial)(cudaStream_t st, const BoxDev* boxes, int b, int par, int rc, double* partials);
    // order parameter of box b (phi[N] may be NULL) and OBS_BLOCKS x {sum phi, sum phi^2}
    cudaError_t (*phi_field)(cudaStream_t st, const BoxDev* boxes, int b, int rc, double* phi, double* partials);
    // interface coverage marks of the particles of box b (marks zeroed by the caller)
    cudaError_t (*coverage_marks)(cudaStream_t st, const BoxDev* boxes, int b, int rc, int* marks);
};

extern const LbOps lb_ops_fp64, lb_ops_fp32, lb_ops_fp16, lb_ops_bf16;

}  // namespace lbp
