// FP32 arithmetic of the step (FP32, FP16 and BF16 population storage): density, psi,
// psi stencil and collision, written once for a lane type V that is either one node (v1,
// scalar FP32 instructions) or two nodes (v2, packed FP32x2 instructions: FADD2, FMUL2,
// FFMA2 of the sm_100 family).  The two-pass kernels use v1, the packed fused kernel v2;
// both evaluate the same expressions in the same order.  The scalar _rn intrinsics round
// exactly as written (checked bit for bit against a numpy evaluation of the same
// expressions).  The pair intrinsics do not always: measured on this toolchain, a packed
// product that feeds a packed sum is sometimes fused into one multiply-add (a*b + c*d
// with the halves of b and d swapped: 30% of random cases, every mismatch explained by
// the fusion), so the fused kernel agrees with the two-pass kernel to rounding, and keeps
// the x and y mirror symmetries exactly (the same instruction serves a node and its mirror
// image) but the diagonal one only to rounding.
//
// The formulation keeps three properties that plain FP32 evaluation of the step loses:
//
// 1. Exact lattice symmetry (v1).  Every expression is arranged so that reflecting the inputs
//    across the x axis, the y axis or the diagonal (permuting the populations as the
//    reflection permutes e_i, negating the odd quantities) reflects the rounded results
//    exactly: sums of mirror partners are formed pairwise (a + b = b + a exactly),
//    odd quantities as differences of partners (a - b = -(b - a) exactly), every
//    multiply-add has a partner with the same structure, and rounding to nearest even is
//    symmetric under negation.  A mirror-symmetric state therefore stays symmetric bit for
//    bit.  Without this, FP32 rounding breaks the symmetry of a symmetric set-up at the
//    1e-8 level and seeds its unstable modes (the translation mode of a liquid slab
//    between walls grows by 1e11 over 1.4e5 steps).
// 2. Moments relative to the rest state.  The populations enter as
//    delta_i = f_i - (w_i/w_0) f_0 (w_i/w_0 = 1/4 on the axes, 1/16 on the diagonals,
//    powers of two, so delta_i is exact whenever f_i and (w_i/w_0) f_0 are within a factor
//    two, by Sterbenz's lemma).  The non-conserved moments are then formed relative to
//    m_rest(rho) = (rho, -2 rho, rho, 0, ..., 0) as sums of small numbers (m_e + 2 rho =
//    s14 + 4 s58, m_eps - rho = -3 s14), and the post-collision populations as
//    w_i rho + g_i with g_i = (M^-1 (m_bar - m_rest(rho)))_i assembled from small terms
//    first.  Plain evaluation forms m_e ~ -2 rho and m_eq,e - m_e as differences of
//    numbers 10^3..10^5 times larger than the flow signal.
// 3. Unbiased momentum update.  m_bar_j = j + F (s_j = 1) is never rounded as one sum:
//    with |F| << |j| the fraction of F/ulp(j) is the same at every node in a binade, so
//    RN(j + F) carries the same relative force error (up to 1e-3 of a body force of
//    1e-7) at every node, every step.  (j + F)/6 is instead evaluated as
//    j c6_hi + (j c6_lo + F c6_hi), c6_hi + c6_lo = 1/6 to 2^-48, whose rounding varies
//    with the low bits of j c6_hi; the single-term FP32 1/6 would scale the momentum by
//    (1 + 3e-8) every step.
#pragma once

namespace lbm {

// ------------------------------------------------------------ lane types --------
struct v1 {
    float v;
};
struct v2 {
    float2 v;
};
__device__ __forceinline__ v2 V(float a, float b) { return v2{make_float2(a, b)}; }
__device__ __forceinline__ v2 S2(float a) { return v2{make_float2(a, a)}; }

// scalar FP32: the _rn intrinsics are never contracted into multiply-adds, so the
// rounding of every operation is the one written here
__device__ __forceinline__ v1 operator+(v1 a, v1 b) { return v1{__fadd_rn(a.v, b.v)}; }
__device__ __forceinline__ v1 operator-(v1 a, v1 b) { return v1{__fsub_rn(a.v, b.v)}; }
__device__ __forceinline__ v1 operator*(v1 a, v1 b) { return v1{__fmul_rn(a.v, b.v)}; }
__device__ __forceinline__ v1 vfma(v1 a, v1 b, v1 c) { return v1{__fmaf_rn(a.v, b.v, c.v)}; }
// Reciprocal and square root: one hardware instruction each, written as PTX so that
// every kernel uses the same one (rcp.approx.ftz and sqrt.approx.ftz, relative error
// about 2^-23; their arguments here are never subnormal).  LBM_F32_IEEE = 1 selects the
// correctly rounded forms (rcp.rn, sqrt.rn).
#ifndef LBM_F32_IEEE
#define LBM_F32_IEEE 0
#endif
__device__ __forceinline__ float rcp32(float a)
{
    float r;
#if LBM_F32_IEEE
    asm("rcp.rn.f32 %0, %1;" : "=f"(r) : "f"(a));
#else
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
#endif
    return r;
}
__device__ __forceinline__ float sqrt32(float a)
{
    float r;
#if LBM_F32_IEEE
    asm("sqrt.rn.f32 %0, %1;" : "=f"(r) : "f"(a));
#else
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
#endif
    return r;
}
__device__ __forceinline__ v1 vrcp(v1 a) { return v1{rcp32(a.v)}; }
__device__ __forceinline__ v1 vsqrt(v1 a) { return v1{sqrt32(a.v)}; }
__device__ __forceinline__ v1 vclamp01(v1 a) { return v1{fminf(fmaxf(a.v, 0.f), 1.f)}; }

// packed FP32x2: the CUDA pair intrinsics (FADD2 / FMUL2 / FFMA2 of the sm_100 family) with
// round-to-nearest, never contracted; a - b is a + (-b), the same rounding
__device__ __forceinline__ v2 operator+(v2 a, v2 b) { return v2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ v2 operator-(v2 a, v2 b) { return v2{__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y))}; }
__device__ __forceinline__ v2 operator*(v2 a, v2 b) { return v2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ v2 vfma(v2 a, v2 b, v2 c) { return v2{__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ v2 vrcp(v2 a) { return V(rcp32(a.v.x), rcp32(a.v.y)); }
__device__ __forceinline__ v2 vsqrt(v2 a) { return V(sqrt32(a.v.x), sqrt32(a.v.y)); }
__device__ __forceinline__ v2 vclamp01(v2 a) { return V(fminf(fmaxf(a.v.x, 0.f), 1.f), fminf(fmaxf(a.v.y, 0.f), 1.f)); }

// A literal (an immediate operand) and a host-precomputed constant of the pair table.
template <class T> __device__ __forceinline__ T ks(float a);
template <> __device__ __forceinline__ v1 ks<v1>(float a) { return v1{a}; }
template <> __device__ __forceinline__ v2 ks<v2>(float a) { return S2(a); }
template <class T> __device__ __forceinline__ T kc(const float2 &c);
template <> __device__ __forceinline__ v1 kc<v1>(const float2 &c) { return v1{c.x}; }
template <> __device__ __forceinline__ v2 kc<v2>(const float2 &c) { return v2{c}; }

// 1/6 as a sum of two floats (hi = RN(1/6), lo = RN(1/6 - hi))
constexpr float kC6Hi = 1.0f / 6.0f;
constexpr float kC6Lo = (float)(1.0 / 6.0 - (double)(1.0f / 6.0f));

// ------------------------------------------------- rest-state deviations --------
// d[0] = f_0, d[i] = f_i - (w_i/w_0) f_0 (i = 1..8).
template <class T>
__device__ __forceinline__ void to_dev(const T (&f)[9], T (&d)[9])
{
    const T q0 = f[0] * ks<T>(0.25f), o0 = f[0] * ks<T>(0.0625f);
    d[0] = f[0];
    d[1] = f[1] - q0;
    d[2] = f[2] - q0;
    d[3] = f[3] - q0;
    d[4] = f[4] - q0;
    d[5] = f[5] - o0;
    d[6] = f[6] - o0;
    d[7] = f[7] - o0;
    d[8] = f[8] - o0;
}

// rho = sum f_i = (9/4) f_0 + sum_{i>0} delta_i, Eq. (rho.rhou), with one rounding of the
// (9/4) f_0 term (exact inside the multiply-add).
template <class T>
__device__ __forceinline__ T density_dev(const T (&d)[9])
{
    const T s14 = (d[1] + d[3]) + (d[2] + d[4]);
    const T s58 = (d[5] + d[7]) + (d[6] + d[8]);
    return vfma(ks<T>(2.25f), d[0], s14 + s58);
}

// ------------------------------------------------------------------ EOS ---------
// psi = sqrt(2 (p_EOS - rho/3)/G) (Sec. 2), van der Waals or Carnahan-Starling.
template <class T>
__device__ __forceinline__ T psi_v(const KParams &kp, T rho)
{
    const PairConsts &q = kp.c2;
    T p;
    if (kp.eos == 0) {
        const T om = vfma(kc<T>(q.m_b), rho, ks<T>(1.f));
        p = kc<T>(q.K) * vfma(rho * kc<T>(q.RT), vrcp(om), kc<T>(q.a) * rho * rho * ks<T>(-1.f));
    } else {
        const T eta = kc<T>(q.b4) * rho;
        const T om = ks<T>(1.f) - eta;
        const T num = vfma(eta, vfma(eta, om, ks<T>(1.f)), ks<T>(1.f));  // 1 + eta + eta^2 - eta^3
        const T den = om * om * om;
        p = kc<T>(q.K) * vfma(rho * kc<T>(q.RT) * num, vrcp(den), kc<T>(q.a) * rho * rho * ks<T>(-1.f));
    }
    return vsqrt(kc<T>(q.two_over_G) * vfma(rho, ks<T>(-1.0f / 3.0f), p));
}

// --------------------------------------------------------------- stencil --------
// S = sum_i w(|e_i|^2) psi(x + e_i) e_i with w = 1/3 (axes), 1/12 (diagonals), Eq. (fint),
// from the psi of the eight neighbours (east, north, west, south, NE, NW, SW, SE).
template <class T>
__device__ __forceinline__ void stencil_v(T pE, T pN, T pW, T pS, T pNE, T pNW, T pSW, T pSE, T &Sx, T &Sy)
{
    const T dd = pNE - pSW;
    Sx = vfma(ks<T>(1.0f / 3.0f), pE - pW, ks<T>(1.0f / 12.0f) * (dd + (pSE - pNW)));
    Sy = vfma(ks<T>(1.0f / 3.0f), pN - pS, ks<T>(1.0f / 12.0f) * (dd + (pNW - pSE)));
}

// ------------------------------------------------------------- collision --------
// Stages 5-8 of the step for the pulled populations in deviation form d (to_dev), the
// node density rho (density_dev), psi, S and the external force:
// u = (j + F/2)/rho (Eq. rho.rhou); m = M f; m_eq and F_m (Sec. 2); Q_m original or
// improved (Eqs. qm.improved, qm46.improved) with |F_int|^2/(G psi^2) = G |S|^2;
// s_0 = s_j = 1, s_e = s_eps = s_p = 1/tau, (1/s_q - 1/2)(1/s_p - 1/2) = Lambda (Sec. 3);
// m_bar = m + F_m - S (m - m_eq + F_m/2) + S Q_m (Eq. lbe.col); f_bar = M^-1 m_bar.
// Each node's mass is closed through f_bar_0 = rho - sum_{i>0} f_bar_i (rho - S' is exact by
// Sterbenz's lemma, so the closure adds no rounding of its own).
template <class T, class O>
__device__ __forceinline__ void collide_v(const KParams &kp, const T (&d)[9], T rho, T psi, T Sx, T Sy, T Fex,
                                          T Fey, T (&fb)[9], T &ux, T &uy)
{
    const PairConsts &q = kp.c2;
    const T p13 = d[1] + d[3], p24 = d[2] + d[4], a13 = d[1] - d[3], c24 = d[2] - d[4];
    const T p57 = d[5] + d[7], p68 = d[6] + d[8], d57 = d[5] - d[7], d68 = d[6] - d[8];
    const T s14 = p13 + p24, s58 = p57 + p68;
    const T t = d57 - d68, v = d57 + d68;
    const T jx = a13 + t, jy = c24 + v;  // j = sum e_i f_i
    const T nGpsi = kc<T>(q.m_G) * psi;
    const T Fx = vfma(nGpsi, Sx, Fex), Fy = vfma(nGpsi, Sy, Fey);  // F = F_int + F_ext, Eq. (fint)
    const T inv = vrcp(rho);
    ux = vfma(ks<T>(0.5f), Fx, jx) * inv;
    uy = vfma(ks<T>(0.5f), Fy, jy) * inv;

    // non-conserved moments of M f relative to m_rest(rho)
    const T r1 = vfma(ks<T>(4.f), s58, s14);  // m_e + 2 rho
    const T r2 = s14 * ks<T>(-3.f);           // m_eps - rho
    const T r4 = vfma(ks<T>(-2.f), a13, t);   // q_x
    const T r6 = vfma(ks<T>(-2.f), c24, v);   // q_y
    const T r7 = p13 - p24;                   // p_xx
    const T r8 = p57 - p68;                   // p_xy

    // equilibrium moments relative to m_rest(rho) and forcing moments (Sec. 2)
    const T rux = rho * ux, ruy = rho * uy;
    const T uxx = ux * ux, uyy = uy * uy;
    const T ru2 = rho * (uxx + uyy);
    const T e1 = ks<T>(3.f) * ru2;   // m_eq,e + 2 rho
    const T e2 = ks<T>(-3.f) * ru2;  // m_eq,eps - rho
    const T meq7 = rho * (uxx - uyy), meq8 = rho * (ux * uy);
    const T Fxu = Fx * ux, Fyv = Fy * uy;
    const T Fu = Fxu + Fyv;
    const T Fm7 = ks<T>(2.f) * (Fxu - Fyv);
    const T Fm8 = Fx * uy + Fy * ux;

    // third-order source
    const T Sx2 = Sx * Sx, Sy2 = Sy * Sy;
    const T Q1 = kc<T>(q.kq1) * (Sx2 + Sy2);
    const T Q2 = kc<T>(q.q2fac) * Q1;
    const T Q7 = kc<T>(q.kq7) * (Sx2 - Sy2);
    const T Q8 = kc<T>(q.kq7) * (Sx * Sy);
    T Q4 = ks<T>(0.f), Q6 = ks<T>(0.f);
    if (O::improved(kp)) {
        Q4 = vfma(kc<T>(q.c1G), Sx2, kc<T>(q.m_c2G) * Sy2) * ux;
        Q6 = vfma(kc<T>(q.c1G), Sy2, kc<T>(q.m_c2G) * Sx2) * uy;
    }

    // m_bar = m + s (m_eq - m + Q) + (1 - s/2) F_m   (Eq. lbe.col)
    T b1, b2, b4, b6, b7, b8;
    if (O::var_tau(kp)) {
        const T w = vclamp01((rho - kc<T>(q.rho_g)) * kc<T>(q.inv_drho));
        const T tau = vfma(ks<T>(3.f), vfma(w, kc<T>(q.dnu), kc<T>(q.nu_g)), ks<T>(0.5f));
        const T sp = vrcp(tau);
        const T sq = vrcp(vfma(kc<T>(q.Lambda), vrcp(tau - ks<T>(0.5f)), ks<T>(0.5f)));
        const T hsp = vfma(ks<T>(-0.5f), sp, ks<T>(1.f));
        const T mhsq = vfma(ks<T>(0.5f), sq, ks<T>(-1.f));  // -(1 - s_q/2)
        const T h6 = ks<T>(6.f) * hsp;
        b1 = vfma(sp, (e1 - r1) + Q1, vfma(h6, Fu, r1));
        b2 = vfma(sp, (e2 - r2) + Q2, vfma(h6 * ks<T>(-1.f), Fu, r2));
        b4 = vfma(sq, (Q4 - rux) - r4, vfma(mhsq, Fx, r4));
        b6 = vfma(sq, (Q6 - ruy) - r6, vfma(mhsq, Fy, r6));
        b7 = vfma(sp, (meq7 - r7) + Q7, vfma(hsp, Fm7, r7));
        b8 = vfma(sp, (meq8 - r8) + Q8, vfma(hsp, Fm8, r8));
    } else {
        const T sp = kc<T>(q.sp), sq = kc<T>(q.sq), hsp = kc<T>(q.hsp), mhsq = kc<T>(q.m_hsq);
        b1 = vfma(sp, (e1 - r1) + Q1, vfma(kc<T>(q.six_hsp), Fu, r1));
        b2 = vfma(sp, (e2 - r2) + Q2, vfma(kc<T>(q.m_six_hsp), Fu, r2));
        b4 = vfma(sq, (Q4 - rux) - r4, vfma(mhsq, Fx, r4));
        b6 = vfma(sq, (Q6 - ruy) - r6, vfma(mhsq, Fy, r6));
        b7 = vfma(sp, (meq7 - r7) + Q7, vfma(hsp, Fm7, r7));
        b8 = vfma(sp, (meq8 - r8) + Q8, vfma(hsp, Fm8, r8));
    }

    // g = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4) (m_bar - m_rest(rho)),
    // m_bar_j = j + F (s_j = 1) through the two-term 1/6
    const T Bn = b1 * ks<T>(-1.0f / 36.0f), C = b2 * ks<T>(1.0f / 36.0f);
    const T D = vfma(jx, ks<T>(kC6Hi), vfma(jx, ks<T>(kC6Lo), Fx * ks<T>(kC6Hi)));
    const T Gy = vfma(jy, ks<T>(kC6Hi), vfma(jy, ks<T>(kC6Lo), Fy * ks<T>(kC6Hi)));
    const T E = b4 * ks<T>(1.0f / 12.0f), H = b6 * ks<T>(1.0f / 12.0f);
    const T P = b7 * ks<T>(0.25f), Qp = b8 * ks<T>(0.25f);
    const T ax = vfma(ks<T>(-2.f), C, Bn);  // axis directions: -B - 2C
    const T dg = vfma(ks<T>(-2.f), Bn, C);  // diagonal directions: 2B + C
    const T DE = vfma(ks<T>(-2.f), E, D), GH = vfma(ks<T>(-2.f), H, Gy);
    const T DEp = D + E, GHp = Gy + H;
    const T dgp = dg + Qp, dgm = dg - Qp, spp = DEp + GHp, smm = GHp - DEp;
    const T r9 = rho * ks<T>(1.0f / 9.0f), r36 = rho * ks<T>(1.0f / 36.0f);
    fb[1] = r9 + ((ax + DE) + P);
    fb[3] = r9 + ((ax - DE) + P);
    fb[2] = r9 + ((ax + GH) - P);
    fb[4] = r9 + ((ax - GH) - P);
    fb[5] = r36 + (dgp + spp);
    fb[7] = r36 + (dgp - spp);
    fb[6] = r36 + (dgm + smm);
    fb[8] = r36 + (dgm - smm);
    fb[0] = rho - (((fb[1] + fb[3]) + (fb[2] + fb[4])) + ((fb[5] + fb[7]) + (fb[6] + fb[8])));
}

}  // namespace lbm
