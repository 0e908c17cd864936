// Kernel instantiations for float population storage.
#include "k_fused.cuh"
#include "k_twopass.cuh"

namespace lbm {

Launchers launchers_f32()
{
    Launchers L{};
    L.psi_pass = &TwoPass<float>::psi_pass;
    L.collide_pass = &TwoPass<float>::collide_pass;
    L.fused_pass = &Fused<float, 4, 8>::launch;
    L.init = &TwoPass<float>::init;
    L.moments = &TwoPass<float>::moments;
    L.diag = &TwoPass<float>::diag;
    L.get_state = &TwoPass<float>::get_state;
    L.set_state = &TwoPass<float>::set_state;
    L.fused_tile_x = FusedLayout<float, 4, 8>::TX;
    L.fused_align = FusedGeom<float>::HX;
    return L;
}

}  // namespace lbm
