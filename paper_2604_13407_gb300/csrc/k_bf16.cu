// Kernel instantiations for __nv_bfloat16 population storage.
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

Launchers launchers_bf16()
{
    Launchers L{};
    L.psi_pass = &TwoPass<__nv_bfloat16>::psi_pass;
    L.collide_pass = &TwoPass<__nv_bfloat16>::collide_pass;
    L.fused_pass = &Fused<__nv_bfloat16, LBM_FUSED_NW, LBM_FUSED_RING>::launch;
    L.init = &TwoPass<__nv_bfloat16>::init;
    L.moments = &TwoPass<__nv_bfloat16>::moments;
    L.diag = &TwoPass<__nv_bfloat16>::diag;
    L.get_state = &TwoPass<__nv_bfloat16>::get_state;
    L.set_state = &TwoPass<__nv_bfloat16>::set_state;
    L.fused_tile_x = FusedLayout<__nv_bfloat16, LBM_FUSED_NW, LBM_FUSED_RING>::TX;
    L.fused_align = FusedGeom<__nv_bfloat16>::HX;
    return L;
}

}  // namespace lbm
