// Kernel instantiations for float population storage.
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
#define LBM_FUSED2_RING 4
#endif

namespace lbm {

Launchers launchers_f32()
{
    Launchers L{};
    L.psi_pass = &TwoPass<float>::psi_pass;
    L.collide_pass = &TwoPass<float>::collide_pass;
#if LBM_FUSED_PAIRS
    L.fused_pass = &Fused2<float, LBM_FUSED2_NW, LBM_FUSED2_RING>::launch;
    L.fused_tile_x = FusedLayout2<float, LBM_FUSED2_NW, LBM_FUSED2_RING>::TX;
#else
    L.fused_pass = &Fused<float, LBM_FUSED_NW, LBM_FUSED_RING>::launch;
    L.fused_tile_x = FusedLayout<float, LBM_FUSED_NW, LBM_FUSED_RING>::TX;
#endif
    L.init = &TwoPass<float>::init;
    L.moments = &TwoPass<float>::moments;
    L.diag = &TwoPass<float>::diag;
    L.get_state = &TwoPass<float>::get_state;
    L.set_state = &TwoPass<float>::set_state;
    L.adj_pass1 = &Adjoint<float>::pass1;
    L.adj_pass2 = &Adjoint<float>::pass2;
    L.adj_lambda = &Adjoint<float>::lambda;
    L.objective = &Adjoint<float>::objective;
    L.adj_blocks = &Adjoint<float>::blocks;
    L.adj_reduce = &Adjoint<float>::reduce;
    L.fused_align = FusedGeom<float>::HX;
    L.fused_geometry = LBM_FUSED_PAIRS;
    return L;
}

}  // namespace lbm
