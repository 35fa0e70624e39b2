// lb_kern_inst.cu -- instantiates the precision-dependent kernels for one
// population storage type (LB_PREC: 0 FP64, 1 FP32, 2 FP16 deviation,
// 3 BF16 deviation) and exports their launchers as an LbOps table.
#include "lb_aux.cuh"
#include "lb_step_split.cuh"
#include "lb_ops.h"

#ifndef LB_PREC
#error "LB_PREC must be defined"
#endif

namespace lbp {
#if LB_PREC == 0
using PP = P64;
#define OPS_NAME lb_ops_fp64
#elif LB_PREC == 1
using PP = P32;
#define OPS_NAME lb_ops_fp32
#elif LB_PREC == 2
using PP = P16;
#define OPS_NAME lb_ops_fp16
#else
using PP = PB16;
#define OPS_NAME lb_ops_bf16
#endif
using RR = typename PP::real;

namespace {
constexpr int EV_GRID = 304, EV_BLOCK = 256, NODE_GRID = 1216, NODE_BLOCK = 256;

template <int PAR, int TY, bool T1, bool BB>
cudaError_t step_t(int ntiles, cudaStream_t st, const BoxDev* boxes, const TileDev* tiles, Shared sh, int rc, int rn,
                   int rz, int mslot) {
    const size_t smem = StepStage<PP, TY>::smem;
    k_step<PP, PAR, TY, T1, BB><<<ntiles, dim3(32, TY), smem, st>>>(boxes, tiles, sh, rc, rn, rz, mslot);
    return cudaGetLastError();
}

template <int PAR, int TY, bool T1, bool BB>
cudaError_t set_attr() {
    return cudaFuncSetAttribute(k_step<PP, PAR, TY, T1, BB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)StepStage<PP, TY>::smem);
}

template <int PAR, int TY, bool T1, bool BB>
cudaError_t split_t(int ntiles, cudaStream_t st, const BoxDev* boxes, const TileDev* tiles, Shared sh, int rc, int rn,
                    int rz, int mslot) {
    const size_t smem = SplitSmem<RR, TY>::bytes;
    k_step_split<PP, PAR, TY, T1, BB><<<ntiles, dim3(32, TY), smem, st>>>(boxes, tiles, sh, rc, rn, rz, mslot);
    return cudaGetLastError();
}

template <int PAR, int TY, bool T1, bool BB>
cudaError_t set_attr_split() {
    return cudaFuncSetAttribute(k_step_split<PP, PAR, TY, T1, BB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SplitSmem<RR, TY>::bytes);
}

template <bool T1, bool BB>
cudaError_t setup_t() {
    cudaError_t e = cudaSuccess;
    cudaError_t r[10] = {set_attr<0, 4, T1, BB>(),       set_attr<1, 4, T1, BB>(),       set_attr<0, 8, T1, BB>(),
                         set_attr<1, 8, T1, BB>(),       set_attr<0, 16, T1, BB>(),      set_attr<1, 16, T1, BB>(),
                         set_attr_split<0, 8, T1, BB>(), set_attr_split<1, 8, T1, BB>(), set_attr_split<0, 16, T1, BB>(),
                         set_attr_split<1, 16, T1, BB>()};
    for (auto x : r)
        if (x != cudaSuccess) e = x;
    return e;
}

cudaError_t setup() {
    const cudaError_t r[4] = {setup_t<false, false>(), setup_t<false, true>(), setup_t<true, false>(),
                              setup_t<true, true>()};
    for (auto x : r)
        if (x != cudaSuccess) return x;
    return cudaSuccess;
}

template <bool T1, bool BB>
cudaError_t step_tau(int par, int ty, int split, int ntiles, cudaStream_t st, const BoxDev* boxes,
                     const TileDev* tiles, Shared sh, int rc, int rn, int rz, int mslot) {
    if (split) {
        switch (ty * 2 + par) {
            case 16: return split_t<0, 8, T1, BB>(ntiles, st, boxes, tiles, sh, rc, rn, rz, mslot);
            case 17: return split_t<1, 8, T1, BB>(ntiles, st, boxes, tiles, sh, rc, rn, rz, mslot);
            case 32: return split_t<0, 16, T1, BB>(ntiles, st, boxes, tiles, sh, rc, rn, rz, mslot);
            case 33: return split_t<1, 16, T1, BB>(ntiles, st, boxes, tiles, sh, rc, rn, rz, mslot);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (ty * 2 + par) {
        case 8: return step_t<0, 4, T1, BB>(ntiles, st, boxes, tiles, sh, rc, rn, rz, mslot);
        case 9: return step_t<1, 4, T1, BB>(ntiles, st, boxes, tiles, sh, rc, rn, rz, mslot);
        case 16: return step_t<0, 8, T1, BB>(ntiles, st, boxes, tiles, sh, rc, rn, rz, mslot);
        case 17: return step_t<1, 8, T1, BB>(ntiles, st, boxes, tiles, sh, rc, rn, rz, mslot);
        case 32: return step_t<0, 16, T1, BB>(ntiles, st, boxes, tiles, sh, rc, rn, rz, mslot);
        case 33: return step_t<1, 16, T1, BB>(ntiles, st, boxes, tiles, sh, rc, rn, rz, mslot);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t step(int par, int ty, int split, int tau1, int reflect, int ntiles, cudaStream_t st, const BoxDev* boxes,
                 const TileDev* tiles, Shared sh, int rc, int rn, int rz, int mslot) {
    if (ntiles <= 0) return cudaSuccess;
    if (reflect)
        return tau1 ? step_tau<true, true>(par, ty, split, ntiles, st, boxes, tiles, sh, rc, rn, rz, mslot)
                    : step_tau<false, true>(par, ty, split, ntiles, st, boxes, tiles, sh, rc, rn, rz, mslot);
    return tau1 ? step_tau<true, false>(par, ty, split, ntiles, st, boxes, tiles, sh, rc, rn, rz, mslot)
                : step_tau<false, false>(par, ty, split, ntiles, st, boxes, tiles, sh, rc, rn, rz, mslot);
}

cudaError_t remap_apply(int par, cudaStream_t st, const BoxDev* boxes, Shared sh, int rc, int mslot_cur) {
    if (par == 0) k_remap_apply<PP, 0><<<EV_GRID, EV_BLOCK, 0, st>>>(boxes, sh, rc, mslot_cur);
    else k_remap_apply<PP, 1><<<EV_GRID, EV_BLOCK, 0, st>>>(boxes, sh, rc, mslot_cur);
    return cudaGetLastError();
}

cudaError_t remap_finish(cudaStream_t st, const BoxDev* boxes, Shared sh, int rc) {
    k_remap_finish<RR><<<EV_GRID, EV_BLOCK, 0, st>>>(boxes, sh, rc);
    return cudaGetLastError();
}

cudaError_t shell_density(cudaStream_t st, const BoxDev* boxes, Shared sh, int rc, int NP) {
    if (NP <= 0) return cudaSuccess;
    k_shell_density<RR><<<NP, 32 * SHELL_WARPS, 0, st>>>(boxes, sh, rc, NP);
    return cudaGetLastError();
}

cudaError_t couple(cudaStream_t st, const BoxDev* boxes, Shared sh, int rc, int rn, int mslot, int par, int reflect,
                   int impl, int NP) {
    if (NP <= 0) return cudaSuccess;
    if (impl) k_couple<PP, true><<<NP, COUPLE_THREADS, 0, st>>>(boxes, sh, rc, rn, mslot, par, reflect);
    else k_couple<PP, false><<<NP, COUPLE_THREADS, 0, st>>>(boxes, sh, rc, rn, mslot, par, reflect);
    return cudaGetLastError();
}

cudaError_t couple_correct(cudaStream_t st, const BoxDev* boxes, Shared sh, int rc, int rn, int mslot, int par,
                           int reflect, int NP) {
    if (NP <= 0) return cudaSuccess;
    k_couple_correct<PP><<<NP, COUPLE_THREADS, 0, st>>>(boxes, sh, rc, rn, mslot, par, reflect);
    return cudaGetLastError();
}

cudaError_t wall_shell(cudaStream_t st, const BoxDev* boxes, int b, int rc) {
    k_wall_shell<RR><<<NODE_GRID, NODE_BLOCK, 0, st>>>(boxes, b, rc);
    return cudaGetLastError();
}

cudaError_t init_pop(cudaStream_t st, const BoxDev* boxes, int b, const double* rho_field, const double* u_field,
                     uint64_t s_red, uint64_t s_blue, double noise, int rc, double* mass_out) {
    k_init_pop<PP><<<NODE_GRID, NODE_BLOCK, 0, st>>>(boxes, b, rho_field, u_field, s_red, s_blue, noise, rc, mass_out);
    return cudaGetLastError();
}

cudaError_t export_dir(cudaStream_t st, const BoxDev* boxes, int b, int i, int par, int rc, double* out) {
    k_export_dir<PP><<<NODE_GRID, NODE_BLOCK, 0, st>>>(boxes, b, i, par, rc, out);
    return cudaGetLastError();
}

cudaError_t import_dir(cudaStream_t st, const BoxDev* boxes, int b, int i, int par, const double* in) {
    k_import_dir<PP><<<NODE_GRID, NODE_BLOCK, 0, st>>>(boxes, b, i, par, in);
    return cudaGetLastError();
}

cudaError_t rho_from_pop(cudaStream_t st, const BoxDev* boxes, int b, int par, int src, int rc, double* out,
                         double* mass_out) {
    k_rho_from_pop<PP><<<NODE_GRID, NODE_BLOCK, 0, st>>>(boxes, b, par, src, rc, out, mass_out);
    return cudaGetLastError();
}

cudaError_t obs_partial(cudaStream_t st, const BoxDev* boxes, int b, int par, int rc, double* partials) {
    k_obs_partial<PP><<<OBS_BLOCKS, 256, 0, st>>>(boxes, b, par, rc, partials);
    return cudaGetLastError();
}

cudaError_t phi_field(cudaStream_t st, const BoxDev* boxes, int b, int rc, double* phi, double* partials) {
    k_phi<PP><<<OBS_BLOCKS, 256, 0, st>>>(boxes, b, rc, phi, partials);
    return cudaGetLastError();
}

cudaError_t coverage_marks(cudaStream_t st, const BoxDev* boxes, int b, int rc, int* marks) {
    k_coverage_marks<PP><<<NODE_GRID, NODE_BLOCK, 0, st>>>(boxes, b, rc, marks);
    return cudaGetLastError();
}
}  // namespace

const LbOps OPS_NAME = {PP::id,       sizeof(RR),   setup,         step,       remap_apply, remap_finish,
                        shell_density, couple,     couple_correct, wall_shell, init_pop,   export_dir,   import_dir,
                        rho_from_pop,  obs_partial, phi_field,     coverage_marks};

}  // namespace lbp
