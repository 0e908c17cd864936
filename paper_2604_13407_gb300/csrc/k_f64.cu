// Kernel instantiations for double population storage.
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

Launchers launchers_f64()
{
    Launchers L{};
    L.psi_pass = &TwoPass<double>::psi_pass;
    L.collide_pass = &TwoPass<double>::collide_pass;
    L.fused_pass = &Fused<double, LBM_FUSED_NW, LBM_FUSED_RING>::launch;
    L.init = &TwoPass<double>::init;
    L.moments = &TwoPass<double>::moments;
    L.diag = &TwoPass<double>::diag;
    L.get_state = &TwoPass<double>::get_state;
    L.set_state = &TwoPass<double>::set_state;
    L.adj_pass1 = &Adjoint<double>::pass1;
    L.adj_pass2 = &Adjoint<double>::pass2;
    L.adj_lambda = &Adjoint<double>::lambda;
    L.objective = &Adjoint<double>::objective;
    L.adj_blocks = &Adjoint<double>::blocks;
    L.adj_reduce = &Adjoint<double>::reduce;
    L.fused_tile_x = FusedLayout<double, LBM_FUSED_NW, LBM_FUSED_RING>::TX;
    L.fused_align = FusedGeom<double>::HX;
    return L;
}

}  // namespace lbm
