// Internal types shared by the host API and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// Derived constants in the arithmetic type R of a kernel, computed on the host, so that
// no kernel converts between double and float per node (GB300's FP64 pipe is narrow).
template <class R>
struct Consts {
    R eos_a, eos_b, eos_RT, eos_R, eos_K, two_over_G, G, kq1, kq7, c1G, c2G, q2fac, sp, sq, nu_l, nu_g, rho_l, rho_g, Lambda, Fx, Fy, psi_s, rho_s, rho_ref, scale, inv_scale;
    R hsp, hsq;  // 1 - s_p/2 and 1 - s_q/2 of the constant relaxation rates
};

// Constant operands of the packed FP32x2 kernel (k_fused2.cuh), each splatted to a pair
// (c, c) on the host, so that the kernel never assembles a constant pair at run time.
struct PairConsts {
    float2 one, m_one, half, m_half, two, m_two, three, m_three, four, m_four, six, m_six;
    float2 third, m_third, twelfth, ninth, w36, sixth, quarter;
    float2 m_G, kq1, q2fac, kq7, c1G, m_c2G, sp, sq, hsp, hsq, six_hsp, m_six_hsp, m_hsq;
    float2 Fx, Fy, rho_g, inv_drho, dnu, nu_g, Lambda;
    float2 m_b, b4, K, RT, a, two_over_G;
    float2 inv_scale, scale, m_scale, psi_s, rho_ref;
    float2 dec[9];  // w_i rho_ref (decode of deviations)
    float2 enc[9];  // -(w_i rho_ref) 2^k (encode of deviations)
    float2 w[9];    // w_i
};

// Everything a kernel needs, passed by value.  Physical constants are kept in double
// (host bookkeeping and the FP64 path) and, for kernels, in cd / cf by arithmetic type.
struct KParams {
    int nx, ny;
    int device;    // CUDA device of the context
    int sm_count;  // its multiprocessor count (queried once, at create)
    int64_t pitch;  // elements per row of a population plane (and of the rho_ref plane)
    int64_t plane;  // elements per population plane = pitch * ny
    int periodic_x, periodic_y;
    int improved;    // 1: improved Q4, Q6 (Eq. qm46.improved)
    int eos;         // 0 van der Waals, 1 Carnahan-Starling
    int force_mode;  // 0 constant, 1 (rho - rho_g) g, 2 field
    int var_tau;     // 1: tau(rho) from the linear nu(rho) interpolation
    int per_node_ref;
    int sr;            // FP16/BF16 storage: 1 stochastic rounding, 0 to nearest
    uint32_t sr_seed;  // random-bit seed of this step (a hash of the step count)
    // EOS: p = K (rho RT g(rho) - a rho^2); psi = sqrt(two_over_G (p - rho/3))
    double eos_a, eos_b, eos_RT, eos_K, two_over_G;
    double eos_R, eos_T;  // raw R and T (FP64 path evaluates (rho R) T like a plain formula)
    double G;
    double k1, k2;        // raw source coefficients (FP64 path)
    // source term with G folded in (|F_int|^2/(G psi^2) = G |S|^2, S = F_int/(-G psi)):
    // Q1 = kq1 |S|^2, Q2 = q2fac Q1, Q7 = kq7 (Sx^2 - Sy^2), Q8 = kq7 Sx Sy,
    // Q4 = (c1G Sx^2 - c2G Sy^2) ux, Q6 = (c1G Sy^2 - c2G Sx^2) uy
    double kq1, kq7, c1G, c2G, q2fac;
    // relaxation: constant rates, or nu(rho) interpolation data
    double sp, sq;
    double nu_l, nu_g, rho_l, rho_g, Lambda;
    double Fx, Fy;
    double psi_s;  // psi(rho_s) of walls
    double rho_s;
    // FP16/BF16 storage codec
    double rho_ref, scale, inv_scale;
    // buffers
    const void *src;       // populations read (post-collision state of the last step)
    void *dst;             // populations written
    const float *ref_src;  // per-node reference density planes (FP16/BF16 with per_node_ref)
    float *ref_dst;
    void *psi;             // psi field [ny*nx] in the kernel's arithmetic type
    float *psi_out;        // one-pass kernel (FP32 arithmetic): also write psi of the state read
                           // here ([ny*nx], as the psi pass does), or null
    const uint8_t *solid;  // [ny*nx] or null
    const double *wall_u;  // [2][ny*nx] or null
    const double *q;       // [8][ny*nx] or null
    const double *fext;    // [2][ny*nx] or null
    const double *wall_rho;  // [ny*nx] virtual density of each solid node, or null (rho_s)
    const double *wall_psi;  // [ny*nx] psi of wall_rho, or null (psi_s)
    // [8][ny][pitch] per fluid node and pulled population i = 1..8 whose source x - e_i is a
    // wall: (q, c) with q the link fraction after the fallback of a missing second node, and
    // c = 6 w_o (e_i . u_w) the moving-wall coefficient (mw = c rho_w); null without
    // interpolated or moving walls.  Read by the one-pass kernel's wall links.
    const float2 *link;
    int *err;              // device error word (0 = fine)
    Consts<double> cd;     // constants for FP64 arithmetic
    Consts<float> cf;      // constants for FP32 arithmetic
    PairConsts c2;         // the same as pairs, for the packed kernel
    unsigned short inv_scale_bits;  // 2^-k in the storage type (FP16 or BF16 bits)
};

// Per-block partial sums of the transposed passes: slots of one row (8 doubles).  Pass 1:
// dJ/dFx, dJ/dFy, dJ/dG (explicit and wall psi), dJ/dT (wall psi), <W, A_t>; pass 2:
// dJ/dG and dJ/dT through psi(rho).
constexpr int kAdjSlots = 8;
enum AdjSlot { SLOT_FX = 0, SLOT_FY = 1, SLOT_G1 = 2, SLOT_T1 = 3, SLOT_J = 4, SLOT_G2 = 5, SLOT_T2 = 6 };

// Buffers and scalars of one transposed step.  Planes use the population row pitch.
struct AdjArgs {
    const void *g_in;   // [9] planes, g of the step after (null: lambda_{t+1} = W_{t+1} only)
    const void *c_in;   // plane, c of the step after (null with g_in)
    void *g_out;        // [9] planes
    void *c_out;        // plane
    void *dS;           // [2] planes, dJ/dS
    void *dpsi;         // plane, local part of dJ/dpsi
    void *rho;          // plane, rho of the pulled populations of A_t
    double w_scale;     // weight of W in lambda_{t+1} (1/n for J = (1/n) sum_t <W, A_t>)
    int objective;      // 0: y momentum handed to the walls by the next streaming; 1: mean j_x
    double inv_nfluid;  // 1 / number of fluid nodes (objective 1)
    double *part;       // per-block FP64 partial sums [blocks][kAdjSlots]
    int sum_J;          // pass 1 also sums <W, A_t> of its state
    float w_scale_f, inv_nfluid_f;  // the two scales rounded to FP32 on the host (FP32 arithmetic
                                    // converts no FP64 value per node)
};

// Storage precisions (match lbm_precision)
enum Prec { P_F64 = 0, P_F32 = 1, P_F16 = 2, P_BF16 = 3 };

// Device error word bits
enum DevErr { DERR_TIMEOUT = 1, DERR_BOUNDS = 2 };

// One-time set-up of a kernel's dynamic shared-memory limit, per kernel and device (an
// attribute set with one device current does not apply to another); lbm_api.cu.
cudaError_t ensure_smem_attribute_ptr(const void *kernel, int device, int bytes);
template <class K>
inline cudaError_t ensure_smem_attribute(K kernel, int device, int bytes)
{
    return ensure_smem_attribute_ptr(reinterpret_cast<const void *>(kernel), device, bytes);
}

// Launchers, defined in the per-precision translation units (k_f64.cu, k_f32.cu,
// k_f16.cu).  All run on `st` and return the launch status.
struct Launchers {
    cudaError_t (*psi_pass)(const KParams &, cudaStream_t);
    cudaError_t (*collide_pass)(const KParams &, cudaStream_t);
    cudaError_t (*fused_pass)(const KParams &, cudaStream_t);  // may be null
    cudaError_t (*init)(const KParams &, const double *rho, const double *ux, const double *uy,
                        cudaStream_t);
    cudaError_t (*moments)(const KParams &, double *rho, double *ux, double *uy, cudaStream_t);
    cudaError_t (*diag)(const KParams &, double *acc, unsigned long long *umax, int *nan_count,
                        cudaStream_t);
    cudaError_t (*get_state)(const KParams &, double *out, cudaStream_t);
    cudaError_t (*set_state)(const KParams &, const double *in, cudaStream_t);
    // transposed step (FP64 arithmetic for FP64 storage, FP32 otherwise); AdjArgs in k_adjoint.cuh
    cudaError_t (*adj_pass1)(const KParams &, const AdjArgs &, cudaStream_t);
    cudaError_t (*adj_pass2)(const KParams &, const AdjArgs &, cudaStream_t);
    cudaError_t (*adj_lambda)(const KParams &, const AdjArgs &, double *out, cudaStream_t);
    cudaError_t (*objective)(const KParams &, int objective, double inv_nfluid, double *acc, cudaStream_t);
    int64_t (*adj_blocks)(const KParams &);  // rows of the per-block partial-sum array (8 doubles each)
    cudaError_t (*adj_reduce)(const KParams &, const double *part, double *out8, cudaStream_t);
    // fused kernel launch constraints
    int fused_tile_x;     // strip width in nodes
    int fused_align;      // nx must be a multiple of this
    int fused_geometry;   // 1: the fused kernel handles solid nodes, moving and interpolated walls
};

Launchers launchers_f64();
Launchers launchers_f32();
Launchers launchers_f16();
Launchers launchers_bf16();

}  // namespace lbm
