// FP64 evaluation of the step in the plain left-to-right order of the formulas of
// Sec. 2 (dense m = M f and f = M^T diag(1/|M_k|^2) m_bar, divisions where the paper
// divides).  Compiled without multiply-add contraction, this makes the FP64 path
// reproducible bit for bit by any plain FP64 evaluation of the same formulas, so FP64
// results can be compared exactly over long, dynamically unstable runs.
#pragma once

namespace lbm {
namespace f64 {

// Orthogonal transformation matrix (Lallemand & Luo, cited in Sec. 2), moment order
// [rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy]; squared row norms.
__host__ __device__ constexpr int M(int k, int i)
{
    constexpr int t[9][9] = {{1, 1, 1, 1, 1, 1, 1, 1, 1},    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
                             {4, -2, -2, -2, -2, 1, 1, 1, 1}, {0, 1, 0, -1, 0, 1, -1, -1, 1},
                             {0, -2, 0, 2, 0, 1, -1, -1, 1},  {0, 0, 1, 0, -1, 1, 1, -1, -1},
                             {0, 0, -2, 0, 2, 1, 1, -1, -1},  {0, 1, -1, 1, -1, 0, 0, 0, 0},
                             {0, 0, 0, 0, 0, 1, -1, 1, -1}};
    return t[k][i];
}
__host__ __device__ constexpr double Mnorm(int k)
{
    constexpr double t[9] = {9, 36, 36, 6, 12, 6, 12, 4, 4};
    return t[k];
}

__device__ __forceinline__ double density(const double (&f)[9])
{
    double r = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) r += f[i];
    return r;
}

__device__ __forceinline__ double p_eos(const KParams &kp, double rho)
{
    if (kp.eos == 0) return kp.eos_K * (rho * kp.eos_R * kp.eos_T / (1.0 - kp.eos_b * rho) - kp.eos_a * rho * rho);
    const double eta = kp.eos_b * rho / 4.0;
    const double num = 1.0 + eta + eta * eta - eta * eta * eta;
    const double den = (1.0 - eta) * (1.0 - eta) * (1.0 - eta);
    return kp.eos_K * (rho * kp.eos_R * kp.eos_T * num / den - kp.eos_a * rho * rho);
}

__device__ __forceinline__ double psi_of(const KParams &kp, double rho)
{
    return sqrt(2.0 * (p_eos(kp, rho) - rho / 3.0) / kp.G);
}

template <class Ps>
__device__ __forceinline__ void stencil_S(const Ps &ps, double &Sx, double &Sy)
{
    double sx = 0.0, sy = 0.0;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const double p = ps(i);
        const double w = (i <= 4) ? 1.0 / 3.0 : 1.0 / 12.0;
        sx += w * p * (double)ex_(i);
        sy += w * p * (double)ey_(i);
    }
    Sx = sx;
    Sy = sy;
}

__device__ __forceinline__ void from_moments(const double (&m)[9], double (&f)[9])
{
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) acc += (double)M(k, i) * (m[k] / Mnorm(k));
        f[i] = acc;
    }
}

__device__ __forceinline__ void equilibrium_moments(double rho, double ux, double uy, double (&meq)[9])
{
    const double u2 = ux * ux + uy * uy;
    meq[0] = rho;
    meq[1] = -2.0 * rho + 3.0 * rho * u2;
    meq[2] = rho - 3.0 * rho * u2;
    meq[3] = rho * ux;
    meq[4] = -rho * ux;
    meq[5] = rho * uy;
    meq[6] = -rho * uy;
    meq[7] = rho * ux * ux - rho * uy * uy;
    meq[8] = rho * ux * uy;
}

__device__ __forceinline__ void equilibrium(double rho, double ux, double uy, double (&fb)[9])
{
    double meq[9];
    equilibrium_moments(rho, ux, uy, meq);
    from_moments(meq, fb);
}

__device__ __forceinline__ void collide(const KParams &kp, const double (&f)[9], double psi, double Sx, double Sy,
                                        double Fex, double Fey, double (&fb)[9], double &uxo, double &uyo)
{
    double rho = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        rho += f[i];
        jx += (double)ex_(i) * f[i];
        jy += (double)ey_(i) * f[i];
    }
    const double Fix = -kp.G * psi * Sx, Fiy = -kp.G * psi * Sy;
    const double Fx = Fix + Fex, Fy = Fiy + Fey;
    const double ux = (jx + 0.5 * Fx) / rho, uy = (jy + 0.5 * Fy) / rho;
    double m[9], meq[9], Fm[9], Q[9], s[9], mb[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) acc += (double)M(k, i) * f[i];
        m[k] = acc;
    }
    equilibrium_moments(rho, ux, uy, meq);
    const double Fu = Fx * ux + Fy * uy;
    Fm[0] = 0.0;
    Fm[1] = 6.0 * Fu;
    Fm[2] = -6.0 * Fu;
    Fm[3] = Fx;
    Fm[4] = -Fx;
    Fm[5] = Fy;
    Fm[6] = -Fy;
    Fm[7] = 2.0 * Fx * ux - 2.0 * Fy * uy;
    Fm[8] = Fx * uy + Fy * ux;
    // Q_m with |F_int|^2 / (G psi^2) as written in the paper
    const double Gpsi2 = kp.G * psi * psi;
    const double X = Fix * Fix / Gpsi2, Y = Fiy * Fiy / Gpsi2;
    const double eps = -8.0 * (kp.k1 + kp.k2);
#pragma unroll
    for (int k = 0; k < 9; ++k) Q[k] = 0.0;
    Q[1] = 3.0 * (kp.k1 + 2.0 * kp.k2) * (X + Y);
    Q[7] = kp.k1 * (Fix * Fix - Fiy * Fiy) / Gpsi2;
    Q[8] = kp.k1 * Fix * Fiy / Gpsi2;
    Q[2] = (kp.q2fac == -1.0) ? -Q[1] : -Q[1] / 2.0;
    if (kp.improved) {
        Q[4] = ((30.0 * eps - 15.0) / 16.0 * X - 3.0 * eps / 8.0 * Y) * ux;
        Q[6] = ((30.0 * eps - 15.0) / 16.0 * Y - 3.0 * eps / 8.0 * X) * uy;
    }
    double sp = kp.sp, sq = kp.sq;
    if (kp.var_tau) {
        double w = (rho - kp.rho_g) / (kp.rho_l - kp.rho_g);
        w = w < 0.0 ? 0.0 : (w > 1.0 ? 1.0 : w);
        const double nu = kp.nu_g + w * (kp.nu_l - kp.nu_g);
        const double tau = 3.0 * nu + 0.5;
        sp = 1.0 / tau;
        sq = 1.0 / (0.5 + kp.Lambda / (tau - 0.5));
    }
    s[0] = 1.0;
    s[1] = sp;
    s[2] = sp;
    s[3] = 1.0;
    s[4] = sq;
    s[5] = 1.0;
    s[6] = sq;
    s[7] = sp;
    s[8] = sp;
#pragma unroll
    for (int k = 0; k < 9; ++k) mb[k] = m[k] + Fm[k] - s[k] * (m[k] - meq[k] + 0.5 * Fm[k]) + s[k] * Q[k];
    from_moments(mb, fb);
    uxo = ux;
    uyo = uy;
}

}  // namespace f64
}  // namespace lbm
