// Kernel instantiations for __nv_bfloat16 population storage.
#include "k_adjoint.cuh"
#include "k_fused.cuh"
#include "k_fused2.cuh"
#include "k_twopass.cuh"

// strip width (consumer warps of 30 columns) and staged-row ring depth of the fused kernel
#ifndef LBM_FUSED_NW
#define LBM_FUSED_NW 8
#endif
#ifndef LBM_FUSED_RING
#define LBM_FUSED_RING 8
#endif
// two-nodes-per-lane packed kernel (k_fused2.cuh): 1 selects it; consumer warps of 60
// columns and ring depth
#ifndef LBM_FUSED_PAIRS
#define LBM_FUSED_PAIRS 1
#endif
#ifndef LBM_FUSED2_NW
#define LBM_FUSED2_NW 4
#endif
#ifndef LBM_FUSED2_RING
#define LBM_FUSED2_RING 8  // 16-bit rows are half as large: 8 staged rows fit 4 CTAs per SM
#endif

namespace lbm {

Launchers launchers_bf16()
{
    Launchers L{};
    L.psi_pass = &TwoPass<__nv_bfloat16>::psi_pass;
    L.collide_pass = &TwoPass<__nv_bfloat16>::collide_pass;
#if LBM_FUSED_PAIRS
    L.fused_pass = &Fused2<__nv_bfloat16, LBM_FUSED2_NW, LBM_FUSED2_RING>::launch;
    L.fused_tile_x = FusedLayout2<__nv_bfloat16, LBM_FUSED2_NW, LBM_FUSED2_RING>::TX;
#else
    L.fused_pass = &Fused<__nv_bfloat16, LBM_FUSED_NW, LBM_FUSED_RING>::launch;
    L.fused_tile_x = FusedLayout<__nv_bfloat16, LBM_FUSED_NW, LBM_FUSED_RING>::TX;
#endif
    L.init = &TwoPass<__nv_bfloat16>::init;
    L.moments = &TwoPass<__nv_bfloat16>::moments;
    L.diag = &TwoPass<__nv_bfloat16>::diag;
    L.get_state = &TwoPass<__nv_bfloat16>::get_state;
    L.set_state = &TwoPass<__nv_bfloat16>::set_state;
    L.adj_pass1 = &Adjoint<__nv_bfloat16>::pass1;
    L.adj_pass2 = &Adjoint<__nv_bfloat16>::pass2;
    L.adj_lambda = &Adjoint<__nv_bfloat16>::lambda;
    L.objective = &Adjoint<__nv_bfloat16>::objective;
    L.adj_blocks = &Adjoint<__nv_bfloat16>::blocks;
    L.adj_reduce = &Adjoint<__nv_bfloat16>::reduce;
    L.fused_align = FusedGeom<__nv_bfloat16>::HX;
    L.fused_geometry = LBM_FUSED_PAIRS;
    return L;
}

}  // namespace lbm
