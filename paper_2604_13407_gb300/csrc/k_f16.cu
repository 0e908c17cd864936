// Kernel instantiations for __half population storage.
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

Launchers launchers_f16()
{
    Launchers L{};
    L.psi_pass = &TwoPass<__half>::psi_pass;
    L.collide_pass = &TwoPass<__half>::collide_pass;
    L.fused_pass = &Fused<__half, LBM_FUSED_NW, LBM_FUSED_RING>::launch;
    L.init = &TwoPass<__half>::init;
    L.moments = &TwoPass<__half>::moments;
    L.diag = &TwoPass<__half>::diag;
    L.get_state = &TwoPass<__half>::get_state;
    L.set_state = &TwoPass<__half>::set_state;
    L.fused_tile_x = FusedLayout<__half, LBM_FUSED_NW, LBM_FUSED_RING>::TX;
    L.fused_align = FusedGeom<__half>::HX;
    return L;
}

}  // namespace lbm
