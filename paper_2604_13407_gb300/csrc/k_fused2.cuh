// Fused single-pass step with two nodes per lane and packed FP32 arithmetic, for the
// storage types whose arithmetic is FP32 (FP32, FP16 and BF16 deviations).
//
// Same pipeline as k_fused (k_fused.cuh): one producer warp stages every row of the nine
// population planes into a shared-memory ring with bulk async copies (full/empty
// mbarriers, bounded waits); the consumer warps pull, form rho and psi, and one row later
// collide with the 3 x 3 psi neighbourhood from registers and warp shuffles.  What
// changes is the work of a lane: it owns two adjacent columns (an even column and the
// next), so every FP32 addition, multiplication and multiply-add of the step -- moments,
// EOS, stencil, forces, source term, relaxation, back-transform and storage codec -- is
// one packed FP32x2 instruction (FADD2 / FMUL2 / FFMA2 of the sm_100 family) for two
// lattice nodes, the populations of the pair move as 8-byte (FP32) or 4-byte (FP16/BF16)
// shared loads and global stores, and the psi halo costs two shuffles per row for two
// nodes.  Reciprocal and square root stay per node.  A warp covers 64 columns: lanes
// 1..30 update 60 columns, lanes 0 and 31 carry the halo columns.
//
// The collision evaluates the same formulas as `collide` (lbm_device.cuh), in packed form
// and with shared subexpressions, so results agree with the two-pass step to FP32
// rounding (not bit for bit).  The storage codec rounds exactly as `Codec<>`: the
// deviation (f - w_i rho_ref) 2^k is formed as one fused multiply-add of f 2^k and
// -(w_i rho_ref) 2^k, which equals the rounded difference times the power of two.
#pragma once

#include "k_fused.cuh"

namespace lbm {

// ------------------------------------------------------- packed FP32 pairs --
struct v2 {
    float2 v;
};
__device__ __forceinline__ v2 V(float a, float b) { return v2{make_float2(a, b)}; }
__device__ __forceinline__ v2 S2(float a) { return v2{make_float2(a, a)}; }
__device__ __forceinline__ v2 operator+(v2 a, v2 b) { return v2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ v2 operator*(v2 a, v2 b) { return v2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ v2 operator-(v2 a, v2 b)
{
    unsigned long long ra = *reinterpret_cast<unsigned long long *>(&a.v), rb = *reinterpret_cast<unsigned long long *>(&b.v), rd;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    return v2{*reinterpret_cast<float2 *>(&rd)};
}
__device__ __forceinline__ v2 fma2(v2 a, v2 b, v2 c) { return v2{__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ v2 rcp2(v2 a) { return V(1.0f / a.v.x, 1.0f / a.v.y); }
__device__ __forceinline__ v2 sqrt2(v2 a) { return V(sqrtf(a.v.x), sqrtf(a.v.y)); }

// ------------------------------------------------------------ staging --------
template <class S, int NW, int RING>
struct FusedLayout2 {
    static constexpr int TX = 60 * NW;                       // output columns per strip
    static constexpr int HX = FusedGeom<S>::HX;
    static constexpr int W = TX + 2 * HX;                   // staged columns per row
    static constexpr int POP_ROW = 9 * W * (int)sizeof(S);  // bytes of one staged row (9 planes)
    static constexpr int REF_ROW = W * 4;
    // input ring, its reference rows, mbarriers
    static __host__ __device__ size_t in_bytes(bool ref) { return (size_t)RING * POP_ROW + (ref ? (size_t)RING * REF_ROW : 0); }
    static __host__ __device__ size_t bytes(bool ref) { return in_bytes(ref) + 2 * RING * 8 + 16; }
};

// Stored pairs <-> FP32 pairs.  `p` points at the staged element of column c0 (shared
// memory); `load` reads columns (c0 + OFF, c0 + OFF + 1), one aligned load when OFF = 0.
// FP16/BF16 deviations are decoded without a separate conversion: one mixed-precision
// multiply-add per node, f = dev * 2^-k + w_i rho_ref with dev and 2^-k in the storage
// type and the addend and result in FP32 (exact product, one FP32 rounding: the same
// value as converting and then multiply-adding in FP32).
template <class S> struct Pair2;
template <> struct Pair2<float> {
    template <int OFF>
    static __device__ __forceinline__ v2 load(const float *p)
    {
        if (OFF == 0) return v2{*reinterpret_cast<const float2 *>(p)};
        return V(p[OFF], p[OFF + 1]);
    }
    static __device__ __forceinline__ float load1(const float *p) { return *p; }
    static __device__ __forceinline__ void store(float *p, v2 f) { *reinterpret_cast<float2 *>(p) = f.v; }
};
#define LBM_DEC_PAIR(TS, T2, T)                                                                               \
    template <int OFF>                                                                                        \
    static __device__ __forceinline__ v2 dec(const TS *p, v2 wref, unsigned short inv_scale)                 \
    {                                                                                                         \
        unsigned short lo, hi;                                                                                \
        if (OFF == 0) {                                                                                       \
            const T2 h = *reinterpret_cast<const T2 *>(p);                                                    \
            lo = *reinterpret_cast<const unsigned short *>(&h.x);                                             \
            hi = *reinterpret_cast<const unsigned short *>(&h.y);                                             \
        } else {                                                                                              \
            lo = *reinterpret_cast<const unsigned short *>(p + OFF);                                          \
            hi = *reinterpret_cast<const unsigned short *>(p + OFF + 1);                                      \
        }                                                                                                     \
        float x, y;                                                                                           \
        asm("fma.rn.f32." T " %0, %1, %2, %3;" : "=f"(x) : "h"(lo), "h"(inv_scale), "f"(wref.v.x));           \
        asm("fma.rn.f32." T " %0, %1, %2, %3;" : "=f"(y) : "h"(hi), "h"(inv_scale), "f"(wref.v.y));           \
        return V(x, y);                                                                                       \
    }
template <> struct Pair2<__half> {
    LBM_DEC_PAIR(__half, __half2, "f16")
    static __device__ __forceinline__ float load1(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void store(__half *p, v2 f) { *reinterpret_cast<__half2 *>(p) = __float22half2_rn(f.v); }
};
template <> struct Pair2<__nv_bfloat16> {
    LBM_DEC_PAIR(__nv_bfloat16, __nv_bfloat162, "bf16")
    static __device__ __forceinline__ float load1(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void store(__nv_bfloat16 *p, v2 f)
    {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __float22bfloat162_rn(f.v);
    }
};
#undef LBM_DEC_PAIR

__device__ __forceinline__ v2 load_ref_pair(const float *p, int off)
{
    if (off == 0) return v2{*reinterpret_cast<const float2 *>(p)};
    return V(p[off], p[off + 1]);
}

// ------------------------------------------------------------ physics --------
#define LBM_C2(name) v2{q.name}
// Literal constants: immediates (LBM_PAIR_IMM = 1) or pairs from the kernel parameters.
#ifndef LBM_PAIR_IMM
#define LBM_PAIR_IMM 1
#endif
#if LBM_PAIR_IMM
#define LBM_K(name, val) S2(val)
#define LBM_KP(name, val) S2(val)
#else
#define LBM_K(name, val) v2{q.name}
#define LBM_KP(name, val) v2{kp.c2.name}
#endif

// psi = sqrt(2 (p_EOS - rho/3)/G) of two nodes (Sec. 2).
__device__ __forceinline__ v2 psi_pair(const KParams &kp, v2 rho)
{
    const PairConsts &q = kp.c2;
    v2 p;
    if (kp.eos == 0) {
        const v2 om = fma2(LBM_C2(m_b), rho, LBM_K(one, 1.f));
        p = LBM_C2(K) * fma2(rho * LBM_C2(RT), rcp2(om), LBM_C2(a) * rho * rho * LBM_K(m_one, -1.f));
    } else {
        const v2 eta = LBM_C2(b4) * rho;
        const v2 om = LBM_K(one, 1.f) - eta;
        const v2 num = fma2(eta, fma2(eta, om, LBM_K(one, 1.f)), LBM_K(one, 1.f));  // 1 + eta + eta^2 - eta^3
        const v2 den = om * om * om;
        p = LBM_C2(K) * fma2(rho * LBM_C2(RT) * num, rcp2(den), LBM_C2(a) * rho * rho * LBM_K(m_one, -1.f));
    }
    return sqrt2(LBM_C2(two_over_G) * fma2(rho, LBM_K(m_third, -1.0f / 3.0f), p));
}

// Stages 5-8 of two nodes (see `collide`): u, m = M f, m_eq, F_m, Q_m, relaxation,
// f_bar = M^-1 m_bar, with the mass of each node closed through f_bar_0.
template <class O>
__device__ __forceinline__ void collide_pair(const KParams &kp, const v2 (&f)[9], v2 rho, v2 psi, v2 Sx, v2 Sy,
                                             v2 Fex, v2 Fey, v2 (&fb)[9])
{
    const PairConsts &q = kp.c2;
    const v2 a13 = f[1] - f[3], c24 = f[2] - f[4];
    const v2 bx = (f[5] - f[6]) + (f[8] - f[7]);
    const v2 by = (f[5] + f[6]) - (f[7] + f[8]);
    const v2 jx = a13 + bx, jy = c24 + by;
    const v2 nGpsi = LBM_C2(m_G) * psi;
    const v2 Fx = fma2(nGpsi, Sx, Fex), Fy = fma2(nGpsi, Sy, Fey);
    const v2 inv = rcp2(rho);
    const v2 ux = fma2(LBM_K(half, 0.5f), Fx, jx) * inv;
    const v2 uy = fma2(LBM_K(half, 0.5f), Fy, jy) * inv;

    // non-conserved moments of M f
    const v2 p13 = f[1] + f[3], p24 = f[2] + f[4], p57 = f[5] + f[7], p68 = f[6] + f[8];
    const v2 s14 = p13 + p24, s58 = p57 + p68;
    const v2 m1 = fma2(LBM_K(m_four, -4.f), f[0], fma2(LBM_K(two, 2.f), s58, s14 * LBM_K(m_one, -1.f)));
    const v2 m2 = fma2(LBM_K(four, 4.f), f[0], fma2(LBM_K(m_two, -2.f), s14, s58));
    const v2 m4 = fma2(LBM_K(m_two, -2.f), a13, bx);
    const v2 m6 = fma2(LBM_K(m_two, -2.f), c24, by);
    const v2 m7 = p13 - p24;
    const v2 m8 = p57 - p68;

    // equilibrium and forcing moments
    const v2 rux = rho * ux, ruy = rho * uy;
    const v2 u2 = fma2(ux, ux, uy * uy);
    const v2 meq1 = rho * fma2(LBM_K(three, 3.f), u2, LBM_K(m_two, -2.f));
    const v2 meq2 = rho * fma2(LBM_K(m_three, -3.f), u2, LBM_K(one, 1.f));
    const v2 meq7 = fma2(rux, ux, ruy * uy * LBM_K(m_one, -1.f));
    const v2 meq8 = rux * uy;
    const v2 Fu = fma2(Fx, ux, Fy * uy);
    const v2 Fm7 = LBM_K(two, 2.f) * fma2(Fx, ux, Fy * uy * LBM_K(m_one, -1.f));
    const v2 Fm8 = fma2(Fx, uy, Fy * ux);

    // third-order source, |F_int|^2/(G psi^2) = G |S|^2
    const v2 Sx2 = Sx * Sx, Sy2 = Sy * Sy;
    const v2 Q1 = LBM_C2(kq1) * (Sx2 + Sy2);
    const v2 Q2 = LBM_C2(q2fac) * Q1;
    const v2 Q7 = LBM_C2(kq7) * (Sx2 - Sy2);
    const v2 Q8 = LBM_C2(kq7) * Sx * Sy;
    v2 Q4 = S2(0.f), Q6 = S2(0.f);
    if (O::improved(kp)) {
        Q4 = fma2(LBM_C2(c1G), Sx2, LBM_C2(m_c2G) * Sy2) * ux;
        Q6 = fma2(LBM_C2(c1G), Sy2, LBM_C2(m_c2G) * Sx2) * uy;
    }

    v2 b1, b2, b4, b6, b7, b8;
    if (O::var_tau(kp)) {
        v2 w = (rho - LBM_C2(rho_g)) * LBM_C2(inv_drho);
        w = V(fminf(fmaxf(w.v.x, 0.f), 1.f), fminf(fmaxf(w.v.y, 0.f), 1.f));
        const v2 tau = fma2(LBM_K(three, 3.f), fma2(w, LBM_C2(dnu), LBM_C2(nu_g)), LBM_K(half, 0.5f));
        const v2 sp = rcp2(tau);
        const v2 sq = rcp2(fma2(LBM_C2(Lambda), rcp2(tau - LBM_K(half, 0.5f)), LBM_K(half, 0.5f)));
        const v2 hsp = fma2(LBM_K(m_half, -0.5f), sp, LBM_K(one, 1.f));
        const v2 hsq = fma2(LBM_K(m_half, -0.5f), sq, LBM_K(one, 1.f));
        const v2 h6 = LBM_K(six, 6.f) * hsp;
        b1 = fma2(sp, (meq1 - m1) + Q1, fma2(h6, Fu, m1));
        b2 = fma2(sp, (meq2 - m2) + Q2, fma2(h6 * LBM_K(m_one, -1.f), Fu, m2));
        b4 = fma2(sq, (rux * LBM_K(m_one, -1.f) - m4) + Q4, fma2(hsq * LBM_K(m_one, -1.f), Fx, m4));
        b6 = fma2(sq, (ruy * LBM_K(m_one, -1.f) - m6) + Q6, fma2(hsq * LBM_K(m_one, -1.f), Fy, m6));
        b7 = fma2(sp, (meq7 - m7) + Q7, fma2(hsp, Fm7, m7));
        b8 = fma2(sp, (meq8 - m8) + Q8, fma2(hsp, Fm8, m8));
    } else {
        // m_bar = m + s (m_eq - m + Q) + (1 - s/2) F_m   (Eq. lbe.col)
        b1 = fma2(LBM_C2(sp), (meq1 - m1) + Q1, fma2(LBM_C2(six_hsp), Fu, m1));
        b2 = fma2(LBM_C2(sp), (meq2 - m2) + Q2, fma2(LBM_C2(m_six_hsp), Fu, m2));
        b4 = fma2(LBM_C2(sq), fma2(rux, LBM_K(m_one, -1.f), Q4) - m4, fma2(LBM_C2(m_hsq), Fx, m4));
        b6 = fma2(LBM_C2(sq), fma2(ruy, LBM_K(m_one, -1.f), Q6) - m6, fma2(LBM_C2(m_hsq), Fy, m6));
        b7 = fma2(LBM_C2(sp), (meq7 - m7) + Q7, fma2(LBM_C2(hsp), Fm7, m7));
        b8 = fma2(LBM_C2(sp), (meq8 - m8) + Q8, fma2(LBM_C2(hsp), Fm8, m8));
    }
    // s_j = 1: m_bar_j = j + F

    // f_bar = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4) m_bar
    const v2 A0 = rho * LBM_K(ninth, 1.0f / 9.0f), B = b1 * LBM_K(w36, 1.0f / 36.0f), C = b2 * LBM_K(w36, 1.0f / 36.0f);
    const v2 D = (jx + Fx) * LBM_K(sixth, 1.0f / 6.0f), E = b4 * LBM_K(twelfth, 1.0f / 12.0f);
    const v2 Gy = (jy + Fy) * LBM_K(sixth, 1.0f / 6.0f), H = b6 * LBM_K(twelfth, 1.0f / 12.0f);
    const v2 P = b7 * LBM_K(quarter, 0.25f), Qp = b8 * LBM_K(quarter, 0.25f);
    const v2 ax = fma2(LBM_K(m_two, -2.f), C, A0 - B);
    const v2 dg = fma2(LBM_K(two, 2.f), B, A0 + C);
    const v2 DE = fma2(LBM_K(m_two, -2.f), E, D), GH = fma2(LBM_K(m_two, -2.f), H, Gy);
    const v2 DEp = D + E, GHp = Gy + H;
    const v2 GQp = GHp + Qp, GQm = GHp - Qp;
    fb[1] = (ax + DE) + P;
    fb[2] = (ax + GH) - P;
    fb[3] = (ax - DE) + P;
    fb[4] = (ax - GH) - P;
    fb[5] = (dg + DEp) + GQp;
    fb[6] = (dg - DEp) + GQm;
    fb[7] = (dg - DEp) - GQm;
    fb[8] = (dg + DEp) - GQp;
    fb[0] = rho - (((fb[1] + fb[2]) + (fb[3] + fb[4])) + ((fb[5] + fb[6]) + (fb[7] + fb[8])));
}

template <class O>
__device__ __forceinline__ void external_force_pair(const KParams &kp, int64_t node, v2 rho, v2 &Fex, v2 &Fey)
{
    const PairConsts &q = kp.c2;
    const int mode = O::force_mode(kp);
    if (mode == 0) {
        Fex = LBM_C2(Fx);
        Fey = LBM_C2(Fy);
    } else if (mode == 1) {  // Sec. 3.3: (rho - rho_g) g
        const v2 d = rho - LBM_C2(rho_g);
        Fex = d * LBM_C2(Fx);
        Fey = d * LBM_C2(Fy);
    } else {
        const int64_t n = (int64_t)kp.nx * kp.ny;
        Fex = kp.fext ? V(float(kp.fext[node]), float(kp.fext[node + 1])) : S2(0.f);
        Fey = kp.fext ? V(float(kp.fext[n + node]), float(kp.fext[n + node + 1])) : S2(0.f);
    }
}

// ------------------------------------------------------------- kernel --------
// Population I of the pair: staged row 1 - e_Iy, columns c0 - e_Ix and c0 - e_Ix + 1.
#define LBM_PULL_PAIR(I)                                                                                      \
    {                                                                                                         \
        constexpr int d_ = 1 - ey_(I), off_ = -ex_(I), wc_ = I == 0 ? 0 : (I <= 4 ? 1 : 5);                  \
        if constexpr (IsDev<S>::value) {                                                                      \
            const v2 wref = O::per_node_ref(kp) ? v2{kp.c2.w[wc_]} * load_ref_pair(ref[d_], off_) : v2{kp.c2.dec[wc_]}; \
            f_new[I] = Pair2<S>::template dec<off_>(row[d_] + I * W, wref, kp.inv_scale_bits);               \
        } else {                                                                                              \
            f_new[I] = Pair2<S>::template load<off_>(row[d_] + I * W);                                       \
        }                                                                                                     \
    }

#ifndef LBM_FUSED2_MINB
#define LBM_FUSED2_MINB 2  // CTAs per SM the register allocation must allow
#endif
template <class S, int NW, int RING, bool PERIODIC, class O>
__global__ void __launch_bounds__(32 * (NW + 1), LBM_FUSED2_MINB) k_fused2(KParams kp, int seg_rows)
{
    typedef FusedLayout2<S, NW, RING> L;
    constexpr int TX = L::TX, HX = L::HX, W = L::W;
    constexpr uint32_t ES = sizeof(S);
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *pops = smem;
    const bool has_ref = O::per_node_ref(kp);
    float *refs = has_ref ? reinterpret_cast<float *>(smem + (size_t)RING * L::POP_ROW) : nullptr;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L::in_bytes(has_ref));
    uint64_t *empty = full + RING;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nx = kp.nx, ny = kp.ny;
    const int x0 = blockIdx.x * TX;
    const int yb = blockIdx.y * seg_rows;
    const int ye = min(yb + seg_rows, ny);
    const int first = yb - 2, last = ye + 1;  // staged rows
    const int x_lo = x0 - HX;

    // the state this step reads is the one the previous step wrote, and this step writes
    // the buffer the previous step read: nothing global is touched before it has completed
    grid_dependency_wait();
    allow_dependent_launch();
    if (threadIdx.x == 0) {
        for (int s = 0; s < RING; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, NW);
        }
        fence_mbar_init();
        fence_proxy_async();
    }
    __syncthreads();

    if (warp == NW) {
        // ------------------------------------------------------ producer warp
        if (lane != 0) return;
        const S *A = static_cast<const S *>(kp.src);
        // columns [x_lo, x_lo + W) of a row: the part inside the lattice, and the parts
        // that wrap around a periodic x edge (the same for every row)
        const int lo = x_lo, hi = x0 + TX + HX;
        const int m0 = lo < 0 ? 0 : lo, m1 = hi > nx ? nx : hi;
        const int nl = (lo < 0 && kp.periodic_x) ? -lo : 0;
        const int nr = (hi > nx && kp.periodic_x) ? hi - nx : 0;
        const uint32_t cols = (uint32_t)(m1 - m0 + nl + nr);
        int r = first;
        for (; r <= last; ++r) {
            const int slot = (r - first) & (RING - 1);
            const int use = (r - first) / RING;
            if (use > 0 && !mbar_wait_bounded(empty + slot, (uint32_t)((use - 1) & 1))) {
                atomicOr(kp.err, DERR_TIMEOUT);
                break;
            }
            uint64_t *bar = full + slot;
            int gy = r;
            if (gy < 0 || gy >= ny) {
                if (!kp.periodic_y) {
                    mbar_arrive(bar);
                    continue;
                }
                gy = ((gy % ny) + ny) % ny;
            }
            fence_proxy_async();
            mbar_expect_tx(bar, cols * (9u * ES + (refs ? 4u : 0u)));
            S *dst = reinterpret_cast<S *>(pops + (size_t)slot * L::POP_ROW);
            const S *src = A + (int64_t)gy * kp.pitch;
#pragma unroll 1
            for (int i = 0; i < 9; ++i, dst += W, src += kp.plane) {
                bulk_g2s(dst + (m0 - lo), src + m0, (uint32_t)(m1 - m0) * ES, bar);
                if (nl) bulk_g2s(dst, src + (nx + lo), (uint32_t)nl * ES, bar);
                if (nr) bulk_g2s(dst + (nx - lo), src, (uint32_t)nr * ES, bar);
            }
            if (refs) {
                const float *rs = kp.ref_src + (int64_t)gy * kp.pitch;
                float *rd = refs + slot * W;
                bulk_g2s(rd + (m0 - lo), rs + m0, (uint32_t)(m1 - m0) * 4u, bar);
                if (nl) bulk_g2s(rd, rs + (nx + lo), (uint32_t)nl * 4u, bar);
                if (nr) bulk_g2s(rd + (nx - lo), rs, (uint32_t)nr * 4u, bar);
            }
        }
        // drain: every issued row must have landed before the CTA may exit
        for (int q = max(first, r - RING); q < r && q <= last; ++q)
            mbar_wait_bounded(full + ((q - first) & (RING - 1)), (uint32_t)(((q - first) / RING) & 1));
        return;
    }

    // ----------------------------------------------------------- consumer warps
    const int c0 = x0 + 60 * warp - 2 + 2 * lane;  // unwrapped column of this lane's first node (even)
    const int scol = c0 - x_lo;                     // its staged column (even)
    const bool col_out = !PERIODIC && !kp.periodic_x && (c0 < 0 || c0 >= nx);  // both nodes (nx is even)
    const bool collides = lane >= 1 && lane <= 30 && c0 < nx;
    const bool dev = IsDev<S>::value;
    const float inv_scale = kp.cf.inv_scale, rho_ref = kp.cf.rho_ref;
    const v2 psi_s = v2{kp.c2.psi_s};
    v2 f_old[9], rho_old = S2(0.f), psi_m2 = psi_s, psi_m1 = psi_s;
#pragma unroll
    for (int i = 0; i < 9; ++i) f_old[i] = S2(0.f);
    auto wait_full = [&](int r) -> bool {
        const bool got = mbar_wait_bounded(full + ((r - first) & (RING - 1)), (uint32_t)(((r - first) / RING) & 1));
        return __all_sync(0xffffffffu, got);
    };
    bool ok = wait_full(first) && wait_full(first + 1);
    for (int rp = yb - 1; rp <= ye && ok; ++rp) {
        if (!wait_full(rp + 1)) {
            ok = false;
            break;
        }
        const bool row_out = !PERIODIC && !kp.periodic_y && (rp < 0 || rp >= ny);
        v2 f_new[9], rho_new = S2(0.f), psi_new = psi_s;
#pragma unroll
        for (int i = 0; i < 9; ++i) f_new[i] = S2(0.f);
        if (!col_out && !row_out) {
            const S *row[3];
            const float *ref[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int slot = (rp - 1 + d - first) & (RING - 1);
                row[d] = reinterpret_cast<const S *>(pops + (size_t)slot * L::POP_ROW) + scol;
                ref[d] = refs ? refs + slot * W + scol : nullptr;
            }
            // pull, Eq. (lbe.str): population i of the pair comes from columns c0 - e_ix (+1)
            // of row rp - e_iy
            LBM_PULL_PAIR(0) LBM_PULL_PAIR(1) LBM_PULL_PAIR(2) LBM_PULL_PAIR(3) LBM_PULL_PAIR(4)
            LBM_PULL_PAIR(5) LBM_PULL_PAIR(6) LBM_PULL_PAIR(7) LBM_PULL_PAIR(8)
            if (!PERIODIC) {
                // links whose source lies beyond a non-periodic edge: half-way bounce-back
#pragma unroll
                for (int i = 1; i < 9; ++i) {
                    const int ys = rp - ey_(i);
                    const bool yw = !kp.periodic_y && (ys < 0 || ys >= ny);
                    const bool w0 = yw || (!kp.periodic_x && (c0 - ex_(i) < 0 || c0 - ex_(i) >= nx));
                    const bool w1 = yw || (!kp.periodic_x && (c0 + 1 - ex_(i) < 0 || c0 + 1 - ex_(i) >= nx));
                    if (w0 || w1) {
                        const int o = opp_(i);
                        const S *a = row[1] + o * W;
                        float r0 = Pair2<S>::load1(a), r1 = Pair2<S>::load1(a + 1);
                        if (dev) {
                            const float rf0 = has_ref ? ref[1][0] : rho_ref;
                            const float rf1 = has_ref ? ref[1][1] : rho_ref;
                            r0 = r0 * inv_scale + w_<float>(o) * rf0;
                            r1 = r1 * inv_scale + w_<float>(o) * rf1;
                        }
                        if (w0) f_new[i].v.x = r0 + 0.f;
                        if (w1) f_new[i].v.y = r1 + 0.f;
                    }
                }
            }
            rho_new = (((f_new[0] + f_new[1]) + (f_new[2] + f_new[3])) + ((f_new[4] + f_new[5]) + (f_new[6] + f_new[7]))) + f_new[8];
            psi_new = psi_pair(kp, rho_new);
        }
        __syncwarp();
        // row rp - 1 is not needed any more by this warp
        if (lane == 0 && rp - 1 >= first) mbar_arrive(empty + ((rp - 1 - first) & (RING - 1)));
        // psi of the columns left of the pair and right of it, from the adjacent lanes
        const float am = __shfl_up_sync(0xffffffffu, psi_m2.v.y, 1), bm = __shfl_down_sync(0xffffffffu, psi_m2.v.x, 1);
        const float a0 = __shfl_up_sync(0xffffffffu, psi_m1.v.y, 1), b0 = __shfl_down_sync(0xffffffffu, psi_m1.v.x, 1);
        const float ap = __shfl_up_sync(0xffffffffu, psi_new.v.y, 1), bp = __shfl_down_sync(0xffffffffu, psi_new.v.x, 1);
        const int y = rp - 1;
        if (y >= yb && collides) {
            {
                v2 fb[9];
                // rows y-1 (m), y (0), y+1 (p); left (L), centre, right (R) columns of each node
                const v2 Lm = V(am, psi_m2.v.x), Rm = V(psi_m2.v.y, bm);
                const v2 L0 = V(a0, psi_m1.v.x), R0 = V(psi_m1.v.y, b0);
                const v2 Lp = V(ap, psi_new.v.x), Rp = V(psi_new.v.y, bp);
                // S = sum w psi(x + e) e, w = 1/3 (axes), 1/12 (diagonals), Eq. (fint)
                const v2 dd = Rp - Lm;
                const v2 Sx = fma2(LBM_KP(third, 1.0f / 3.0f), R0 - L0, LBM_KP(twelfth, 1.0f / 12.0f) * (dd + (Rm - Lp)));
                const v2 Sy = fma2(LBM_KP(third, 1.0f / 3.0f), psi_new - psi_m2, LBM_KP(twelfth, 1.0f / 12.0f) * (dd + (Lp - Rm)));
                v2 Fex, Fey;
                external_force_pair<O>(kp, (int64_t)y * nx + c0, rho_old, Fex, Fey);
                collide_pair<O>(kp, f_old, rho_old, psi_m1, Sx, Sy, Fex, Fey, fb);
                S *out = static_cast<S *>(kp.dst) + (int64_t)y * kp.pitch + c0;
                if (!dev) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) Pair2<S>::store(out + i * kp.plane, fb[i]);
                } else if (has_ref) {
                    Pair2<float>::store(kp.ref_dst + (int64_t)y * kp.pitch + c0, rho_old);
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        // (f - w_i ref) 2^k as one rounding: f 2^k - (w_i ref) 2^k
                        const v2 nwref = v2{kp.c2.m_scale} * (v2{kp.c2.w[i == 0 ? 0 : (i <= 4 ? 1 : 5)]} * rho_old);
                        Pair2<S>::store(out + i * kp.plane, fma2(fb[i], v2{kp.c2.scale}, nwref));
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 9; ++i)
                        Pair2<S>::store(out + i * kp.plane, fma2(fb[i], v2{kp.c2.scale}, v2{kp.c2.enc[i == 0 ? 0 : (i <= 4 ? 1 : 5)]}));
                }
            }
        }
        psi_m2 = psi_m1;
        psi_m1 = psi_new;
        rho_old = rho_new;
#pragma unroll
        for (int i = 0; i < 9; ++i) f_old[i] = f_new[i];
    }
    if (!ok) atomicOr(kp.err, DERR_TIMEOUT);
    if (!ok && lane == 0)
        for (int s = 0; s < RING; ++s) mbar_arrive(empty + s);
}
#undef LBM_PULL_PAIR

template <class S, int NW, int RING>
struct Fused2 {
    typedef FusedLayout2<S, NW, RING> L;
    template <bool P, class O>
    static cudaError_t launch_one(const KParams &kp, cudaStream_t st)
    {
        static bool configured = false;
        if (!configured) {
            cudaError_t e = cudaFuncSetAttribute(k_fused2<S, NW, RING, P, O>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)L::bytes(true));
            if (e != cudaSuccess) return e;
            configured = true;
        }
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int strips = (kp.nx + L::TX - 1) / L::TX;
        int nseg = (16 * sms + strips - 1) / strips;
        // segments re-read 3 halo rows; a lattice whose two population buffers fit in L2 reads
        // them from L2, so it may be cut into short segments (more CTAs), a larger one not
        const double state_bytes = 2.0 * 9.0 * (double)kp.plane * sizeof(S);
        const int min_rows = state_bytes <= 64.0 * 1024 * 1024 ? 4 : 16;
        const int max_seg = kp.ny / min_rows > 0 ? kp.ny / min_rows : 1;
        if (nseg > max_seg) nseg = max_seg;
        if (nseg < 1) nseg = 1;
        const int seg_rows = (kp.ny + nseg - 1) / nseg;
        nseg = (kp.ny + seg_rows - 1) / seg_rows;
        return launch_dependent(k_fused2<S, NW, RING, P, O>, dim3(strips, nseg), dim3(32 * (NW + 1)),
                                L::bytes(kp.per_node_ref != 0), st, kp, seg_rows);
    }
    // Fully periodic lattices with a constant force and one relaxation time get
    // instantiations with those options (and the reference-density mode) fixed at compile
    // time; everything else reads them at run time.
    static cudaError_t launch(const KParams &kp, cudaStream_t st)
    {
        if (kp.periodic_x && kp.periodic_y && kp.force_mode == 0 && !kp.var_tau) {
            if (IsDev<S>::value && kp.per_node_ref)
                return kp.improved ? launch_one<true, Opts<1, 0, 0, 1>>(kp, st) : launch_one<true, Opts<0, 0, 0, 1>>(kp, st);
            return kp.improved ? launch_one<true, Opts<1, 0, 0, 0>>(kp, st) : launch_one<true, Opts<0, 0, 0, 0>>(kp, st);
        }
        if (kp.periodic_x && kp.periodic_y) return launch_one<true, RuntimeOpts>(kp, st);
        return launch_one<false, RuntimeOpts>(kp, st);
    }
};

}  // namespace lbm
