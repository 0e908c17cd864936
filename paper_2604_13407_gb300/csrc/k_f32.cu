// Kernel instantiations for float population storage.
#include "k_twopass.cuh"

namespace lbm {

Launchers launchers_f32()
{
    Launchers L{};
    L.psi_pass = &TwoPass<float>::psi_pass;
    L.collide_pass = &TwoPass<float>::collide_pass;
    L.fused_pass = nullptr;
    L.init = &TwoPass<float>::init;
    L.moments = &TwoPass<float>::moments;
    L.diag = &TwoPass<float>::diag;
    L.get_state = &TwoPass<float>::get_state;
    L.set_state = &TwoPass<float>::set_state;
    L.fused_tile_x = 0;
    L.fused_align = 0;
    return L;
}

}  // namespace lbm
