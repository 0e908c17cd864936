// Kernel instantiations for float population storage.
#include "k_adjoint.cuh"
#include "k_fused.cuh"
#include "k_twopass.cuh"

// strip width (consumer warps of 30 columns) and staged-row ring depth of the fused kernel
#ifndef LBM_FUSED_NW
#define LBM_FUSED_NW 8
#endif
#ifndef LBM_FUSED_RING
#define LBM_FUSED_RING 8
#endif

namespace lbm {

Launchers launchers_f32()
{
    Launchers L{};
    L.psi_pass = &TwoPass<float>::psi_pass;
    L.collide_pass = &TwoPass<float>::collide_pass;
    L.fused_pass = &Fused<float, LBM_FUSED_NW, LBM_FUSED_RING>::launch;
    L.init = &TwoPass<float>::init;
    L.moments = &TwoPass<float>::moments;
    L.diag = &TwoPass<float>::diag;
    L.get_state = &TwoPass<float>::get_state;
    L.set_state = &TwoPass<float>::set_state;
    L.adj_pass1 = &Adjoint<float>::pass1;
    L.adj_pass2 = &Adjoint<float>::pass2;
    L.adj_lambda = &Adjoint<float>::lambda;
    L.objective = &Adjoint<float>::objective;
    L.fused_tile_x = FusedLayout<float, LBM_FUSED_NW, LBM_FUSED_RING>::TX;
    L.fused_align = FusedGeom<float>::HX;
    return L;
}

}  // namespace lbm
