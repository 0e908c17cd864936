// Kernel instantiations for double population storage.
#include "k_fused.cuh"
#include "k_twopass.cuh"

namespace lbm {

Launchers launchers_f64()
{
    Launchers L{};
    L.psi_pass = &TwoPass<double>::psi_pass;
    L.collide_pass = &TwoPass<double>::collide_pass;
    L.fused_pass = &Fused<double, 4, 8>::launch;
    L.init = &TwoPass<double>::init;
    L.moments = &TwoPass<double>::moments;
    L.diag = &TwoPass<double>::diag;
    L.get_state = &TwoPass<double>::get_state;
    L.set_state = &TwoPass<double>::set_state;
    L.fused_tile_x = FusedLayout<double, 4, 8>::TX;
    L.fused_align = FusedGeom<double>::HX;
    return L;
}

}  // namespace lbm
