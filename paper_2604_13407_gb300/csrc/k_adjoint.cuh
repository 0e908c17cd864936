// Transposed (adjoint) step of the D2Q9 pseudopotential MRT update, for one storage type
// S with arithmetic type R (FP64 for FP64 storage, FP32 for FP32 and 16-bit storage).
//
// The step maps the stored populations A_t to A_{t+1} = Step(A_t; Fx, Fy, G, T) (Sec. 2:
// pull streaming, moments, psi(rho) from the EOS, F_int = -G psi S with
// S = sum w psi(x + e) e, velocity, m = M f, m_eq, F_m, Q_m, relaxation, M^-1).  Its
// adjoint maps lambda_{t+1} = dJ/dA_{t+1} to lambda_t = W_t + Step'(A_t)^T lambda_{t+1}
// and accumulates dJ/d(Fx, Fy, G, T).  The local chain rule runs backwards through the
// collision at each node; what couples nodes is (i) the psi stencil, which sends dJ/dS(x)
// to psi of the eight neighbours, and (ii) the pull, whose transpose is again a gather:
//
//   lambda_t[i](y) = W_t[i](y) + ( y + e_i is a wall ? g_o(y) + c(y)
//                                                     : g_i(y + e_i) + c(y + e_i) ),
//   o = opposite of i,
//
// where g_i(x) is the part of dJ/df_i(x) that does not pass through psi(rho(x)) and
// c(x) = psi'(rho(x)) dJ/dpsi(x) is the part that does (the same for all nine f_i since
// d rho/d f_i = 1).  So lambda_t is never stored: it is held as the pair (g, c) of the
// step after it, and the next transposed step assembles lambda at its own node.
//
// Pass 1 (k_adj1): per fluid node, assemble lambda_{t+1}, recompute the forward
// quantities from A_t and the psi field of A_t, and run the chain rule back to g(x),
// dJ/dS(x), the local part of dJ/dpsi(x) (through F_int = -G psi S) and rho(x).
// Pass 2 (k_adj2): dJ/dpsi(x) = local part + sum_i w_i e_i . dJ/dS(x - e_i) over fluid
// x - e_i, then c(x) = psi'(rho) dJ/dpsi.  Parameter derivatives are summed per block
// (warp shuffles) into per-block FP64 slots that one reduction sums at the end of the call.
#pragma once

#include "k_twopass.cuh"

namespace lbm {

__device__ __forceinline__ bool wall_link(const KParams &kp, int x, int y, int i, int64_t &kn)
{
    int xn = x + ex_(i), yn = y + ey_(i);
    if (!wrap_xy(kp, xn, yn)) return true;
    if (kp.solid != nullptr && kp.solid[(int64_t)yn * kp.nx + xn] != 0) return true;
    kn = (int64_t)yn * kp.pitch + xn;
    return false;
}

// Walls among the eight neighbours: bit i set when x + e_i is a solid node or lies beyond a
// non-periodic edge.  One set of global solid-flag reads per node serves the pull
// (population i comes from x - e_i = x + e_opp(i)), lambda_{t+1}, the objective and the wall
// psi terms.
__device__ __forceinline__ unsigned wall_mask(const KParams &kp, const Around &nb)
{
    unsigned wm = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i)
        if (!nb.in(i) || (kp.solid != nullptr && kp.solid[nb.n(i)] != 0)) wm |= 1u << i;
    return wm;
}

// Objective weights W_i(x) at a fluid node (before the 1/n of the time average);
// inv_nf = 1 / number of fluid nodes in the arithmetic type.
template <class R>
__device__ __forceinline__ R objective_weight(int objective, int i, bool wall_ahead, R inv_nf)
{
    if (objective == 0) return wall_ahead ? R(2 * ey_(i)) : R(0);
    return R(ex_(i)) * inv_nf;
}

// lambda_{t+1} of the nine populations of a fluid node: nb its neighbourhood, wm its
// wall_mask.
template <class R>
__device__ __forceinline__ void lambda_at(const KParams &kp, const AdjArgs &aa, const Around &nb, unsigned wm, R wscale,
                                          R inv_nf, R (&lam)[9])
{
    const int64_t k = nb.k(0);
    const R *g = static_cast<const R *>(aa.g_in);
    const R *c = static_cast<const R *>(aa.c_in);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const bool wall = (i != 0) && ((wm >> i) & 1u);
        const int64_t kn = (i == 0 || wall) ? k : nb.k(i);
        R v = wscale * objective_weight<R>(aa.objective, i, wall, inv_nf);
        if (g != nullptr) {
            if (wall) v += g[opp_(i) * kp.plane + k] + c[k];
            else v += g[i * kp.plane + kn] + c[kn];
        }
        lam[i] = v;
    }
}

// dp/drho and dp/dT of the EOS.
template <class R>
__device__ __forceinline__ void p_eos_derivs(const KParams &kp, R rho, R &p_rho, R &p_T)
{
    const Consts<R> &c = cst<R>(kp);
    if (kp.eos == 0) {
        const R om = R(1) - c.eos_b * rho;
        p_rho = c.eos_K * (c.eos_RT / (om * om) - R(2) * c.eos_a * rho);
        p_T = c.eos_K * rho * c.eos_R / om;
        return;
    }
    const R eta = c.eos_b * rho * R(0.25);
    const R om = R(1) - eta;
    const R om2 = om * om;
    const R g = (R(1) + eta + eta * eta - eta * eta * eta) / (om2 * om);
    const R dg = (R(4) + R(4) * eta - R(2) * eta * eta) / (om2 * om2);  // dg/d eta
    p_rho = c.eos_K * (c.eos_RT * (g + eta * dg) - R(2) * c.eos_a * rho);
    p_T = c.eos_K * rho * c.eos_R * g;
}

// Per-block FP64 partial sums of the transposed passes (slots AdjSlot, lbm_internal.h):
// one row of kAdjSlots doubles per block of the row grid, accumulated over all steps of a
// call and reduced once at its end, so no atomic is contended and the summation order is
// fixed.

// Warp sum of one value per lane as a compensated FP32 pair (hi, lo) in lane 0: Knuth's
// TwoSum at every shuffle level, about 2^-48 relative.
__device__ __forceinline__ void warp_sum_pair(float &hi, float &lo)
{
    lo = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ohi = __shfl_down_sync(0xffffffffu, hi, o), olo = __shfl_down_sync(0xffffffffu, lo, o);
        const float sum = hi + ohi, z = sum - hi;
        lo += olo + ((hi - (sum - z)) + (ohi - z));
        hi = sum;
    }
}

// Block sum of N per-thread values added to this block's slots [first, first + N).  FP64
// arithmetic sums in FP64.  FP32 arithmetic keeps each warp's sum as a compensated FP32 pair
// and converts to FP64 only in the block's final step (N threads), which keeps FP64 work
// (a narrow pipe on GB300) out of the per-node path.
template <int N, class R>
__device__ __forceinline__ void block_add(const R (&v)[N], double *part, int first)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double t = 0.0;
    if constexpr (sizeof(R) == 8) {
        __shared__ double red[kRowThreads / 32][N];
        // a quantity that is zero on every lane of the warp (the wall terms away from walls)
        // sums to exactly zero: skip its shuffles
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const double w = __any_sync(0xffffffffu, v[k] != R(0)) ? warp_sum(double(v[k])) : 0.0;
            if (lane == 0) red[wid][k] = w;
        }
        __syncthreads();
        if (threadIdx.x < N)
            for (int q = 0; q < kRowThreads / 32; ++q) t += red[q][threadIdx.x];
    } else {
        __shared__ float2 red[kRowThreads / 32][N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            float hi = float(v[k]), lo = 0.f;
            if (__any_sync(0xffffffffu, v[k] != R(0))) warp_sum_pair(hi, lo);
            if (lane == 0) red[wid][k] = make_float2(hi, lo);
        }
        __syncthreads();
        if (threadIdx.x < N)
            for (int q = 0; q < kRowThreads / 32; ++q) {
                const float2 p = red[q][threadIdx.x];
                t += double(p.x) + double(p.y);
            }
    }
    if (threadIdx.x < N) part[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * kAdjSlots + first + threadIdx.x] += t;
}

// Block sum of one double added to *acc with one FP64 atomic per block.
__device__ __forceinline__ void block_atomic_add(double v, double *acc)
{
    __shared__ double red[kRowThreads / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < kRowThreads / 32; ++q) s += red[q];
        if (s != 0.0) atomicAdd(acc, s);
    }
}

// Pass 1 of the transposed step at A_t (kp.src) with the psi field of A_t (kp.psi).
template <class S>
__global__ void __launch_bounds__(kRowThreads, sizeof(typename Codec<S>::R) == 8 ? 4 : 8) k_adj1(KParams kp, AdjArgs aa)
{
    typedef typename Codec<S>::R R;
    grid_dependency_wait();
    allow_dependent_launch();
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    const int64_t node = (int64_t)y * kp.nx + x, k = (int64_t)y * kp.pitch + x;
    R gFx = R(0), gFy = R(0), gG = R(0), gT = R(0), Jt = R(0);
    const R inv_nf = sizeof(R) == 8 ? R(aa.inv_nfluid) : R(aa.inv_nfluid_f);
    if (x < kp.nx && !node_is_solid(kp, node)) {
        const Consts<R> &cc = cst<R>(kp);
        const Around nb = around(kp, x, y);
        const unsigned wm = wall_mask(kp, nb);
        R lam[9];
        lambda_at<R>(kp, aa, nb, wm, sizeof(R) == 8 ? R(aa.w_scale) : R(aa.w_scale_f), inv_nf, lam);

        // ---- forward quantities at this node: the pull of Eq. (lbe.str) with half-way walls
        // (the only walls the adjoint accepts): f_i = A_o(x) + 0 when x - e_i is a wall, as
        // the forward step's bounce-back rule evaluates it
        R f[9];
        f[0] = load_pop_at<S>(kp, 0, k);
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            if ((wm >> opp_(i)) & 1u) f[i] = load_pop_at<S>(kp, opp_(i), k) + R(0);
            else f[i] = load_pop_at<S>(kp, i, nb.k(opp_(i)));  // x - e_i = x + e_opp(i)
        }
        const R rho = density<R>(f);
        const R jx = ((f[1] - f[3]) + (f[5] - f[6])) + (f[8] - f[7]);
        const R jy = ((f[2] - f[4]) + (f[5] + f[6])) - (f[7] + f[8]);
        if (aa.sum_J) {
            // <W, A_t> at this node from its pulled populations: a population stored at x that
            // the next streaming sends into a wall is pulled back by x itself as f_i with
            // x - e_i a wall; every other one is pulled by exactly one fluid node
            R wall_y = R(0), wall_x = R(0);
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const bool wall = (wm >> opp_(i)) & 1u;
                if (wall) {
                    wall_x += R(ex_(i)) * f[i];
                    wall_y += R(ey_(i)) * f[i];
                }
            }
            Jt = aa.objective == 0 ? R(-2) * wall_y : (jx - R(2) * wall_x) * inv_nf;
        }
        const R *psif = static_cast<const R *>(kp.psi);
        const R psi = psif[node];
        R Sx, Sy, Fex, Fey;
        stencil_S<R>(AroundPsi<R>{kp, psif, nb}, Sx, Sy);
        external_force<R>(kp, node, rho, Fex, Fey);
        const R G = cc.G;
        const R Fx = -G * psi * Sx + Fex, Fy = -G * psi * Sy + Fey;
        const R inv = R(1) / rho;
        const R ux = (jx + R(0.5) * Fx) * inv, uy = (jy + R(0.5) * Fy) * inv;
        const R u2 = ux * ux + uy * uy;
        const R s14 = (f[1] + f[2]) + (f[3] + f[4]);
        const R s58 = (f[5] + f[6]) + (f[7] + f[8]);
        const R m1 = R(-4) * f[0] - s14 + R(2) * s58;
        const R m2 = R(4) * f[0] - R(2) * s14 + s58;
        const R m4 = R(-2) * (f[1] - f[3]) + ((f[5] - f[6]) + (f[8] - f[7]));
        const R m6 = R(-2) * (f[2] - f[4]) + ((f[5] + f[6]) - (f[7] + f[8]));
        const R m7 = (f[1] + f[3]) - (f[2] + f[4]);
        const R m8 = (f[5] + f[7]) - (f[6] + f[8]);
        const R Sx2 = Sx * Sx, Sy2 = Sy * Sy;
        const bool improved = kp.improved != 0;
        const R Q1 = cc.kq1 * (Sx2 + Sy2), Q2 = cc.q2fac * Q1;
        const R Q7 = cc.kq7 * (Sx2 - Sy2), Q8 = cc.kq7 * Sx * Sy;
        const R A4 = cc.c1G * Sx2 - cc.c2G * Sy2, A6 = cc.c1G * Sy2 - cc.c2G * Sx2;
        const R Q4 = improved ? A4 * ux : R(0), Q6 = improved ? A6 * uy : R(0);
        R sp = cc.sp, sq = cc.sq, tau = R(0), wraw = R(0);
        if (kp.var_tau) {
            wraw = (rho - cc.rho_g) / (cc.rho_l - cc.rho_g);
            const R w = wraw < R(0) ? R(0) : (wraw > R(1) ? R(1) : wraw);
            tau = R(3) * (cc.nu_g + w * (cc.nu_l - cc.nu_g)) + R(0.5);
            sp = R(1) / tau;
            sq = R(1) / (R(0.5) + cc.Lambda / (tau - R(0.5)));
        }
        const R hsp = R(1) - R(0.5) * sp, hsq = R(1) - R(0.5) * sq;

        // ---- backward: lambda -> dJ/d m_bar (f_bar = M^T diag(1/|M_k|^2) m_bar)
        const R a14 = (lam[1] + lam[2]) + (lam[3] + lam[4]);
        const R a58 = (lam[5] + lam[6]) + (lam[7] + lam[8]);
        const R b0 = (lam[0] + a14 + a58) * R(1.0 / 9.0);
        const R b1 = (R(-4) * lam[0] - a14 + R(2) * a58) * R(1.0 / 36.0);
        const R b2 = (R(4) * lam[0] - R(2) * a14 + a58) * R(1.0 / 36.0);
        const R b3 = ((lam[1] - lam[3]) + (lam[5] - lam[6]) + (lam[8] - lam[7])) * R(1.0 / 6.0);
        const R b4 = (R(-2) * (lam[1] - lam[3]) + (lam[5] - lam[6]) + (lam[8] - lam[7])) * R(1.0 / 12.0);
        const R b5 = ((lam[2] - lam[4]) + (lam[5] + lam[6]) - (lam[7] + lam[8])) * R(1.0 / 6.0);
        const R b6 = (R(-2) * (lam[2] - lam[4]) + (lam[5] + lam[6]) - (lam[7] + lam[8])) * R(1.0 / 12.0);
        const R b7 = ((lam[1] + lam[3]) - (lam[2] + lam[4])) * R(0.25);
        const R b8 = ((lam[5] + lam[7]) - (lam[6] + lam[8])) * R(0.25);

        // m_bar_k = (1 - s_k) m_k + s_k m_eq_k + (1 - s_k/2) F_m_k + s_k Q_k (Eq. lbe.col);
        // s_0 = s_j = 1 (m_bar_0 = rho, m_bar_j = rho u + F/2)
        const R dm1 = (R(1) - sp) * b1, dm2 = (R(1) - sp) * b2, dm4 = (R(1) - sq) * b4;
        const R dm6 = (R(1) - sq) * b6, dm7 = (R(1) - sp) * b7, dm8 = (R(1) - sp) * b8;
        const R d1 = sp * b1, d2 = sp * b2, d4 = sq * b4, d6 = sq * b6, d7 = sp * b7, d8 = sp * b8;
        const R d0 = b0, d3 = b3, d5 = b5;
        const R g1 = hsp * b1, g2 = hsp * b2, g4 = hsq * b4, g6 = hsq * b6, g7 = hsp * b7, g8 = hsp * b8;
        const R g3 = R(0.5) * b3, g5 = R(0.5) * b5;
        // dQ_k = s_k b_k = d_k

        R drho = R(0), dux = R(0), duy = R(0), dFx = R(0), dFy = R(0), dSx = R(0), dSy = R(0);
        if (kp.var_tau) {
            const R Fu = Fx * ux + Fy * uy;
            const R meq1 = rho * (R(-2) + R(3) * u2), meq2 = rho * (R(1) - R(3) * u2);
            const R meq4 = -rho * ux, meq6 = -rho * uy, meq7 = rho * (ux * ux - uy * uy), meq8 = rho * ux * uy;
            const R Fm1 = R(6) * Fu, Fm2 = R(-6) * Fu, Fm4 = -Fx, Fm6 = -Fy;
            const R Fm7 = R(2) * (Fx * ux - Fy * uy), Fm8 = Fx * uy + Fy * ux;
            const R dsp = b1 * (meq1 - m1 - R(0.5) * Fm1 + Q1) + b2 * (meq2 - m2 - R(0.5) * Fm2 + Q2) +
                          b7 * (meq7 - m7 - R(0.5) * Fm7 + Q7) + b8 * (meq8 - m8 - R(0.5) * Fm8 + Q8);
            const R dsq = b4 * (meq4 - m4 - R(0.5) * Fm4 + Q4) + b6 * (meq6 - m6 - R(0.5) * Fm6 + Q6);
            if (wraw > R(0) && wraw < R(1)) {
                const R tm = tau - R(0.5);
                const R dtau = -dsp * sp * sp + dsq * sq * sq * cc.Lambda / (tm * tm);
                drho += R(3) * dtau * (cc.nu_l - cc.nu_g) / (cc.rho_l - cc.rho_g);
            }
        }
        // m_eq(rho, u)
        drho += d0 + d1 * (R(-2) + R(3) * u2) + d2 * (R(1) - R(3) * u2) + ux * (d3 - d4) + uy * (d5 - d6) +
                (ux * ux - uy * uy) * d7 + ux * uy * d8;
        dux += rho * (R(6) * ux * (d1 - d2) + (d3 - d4) + R(2) * ux * d7 + uy * d8);
        duy += rho * (R(6) * uy * (d1 - d2) + (d5 - d6) - R(2) * uy * d7 + ux * d8);
        // F_m(F, u)
        const R dFu = R(6) * (g1 - g2);
        dFx += dFu * ux + (g3 - g4) + R(2) * ux * g7 + uy * g8;
        dFy += dFu * uy + (g5 - g6) - R(2) * uy * g7 + ux * g8;
        dux += dFu * Fx + R(2) * Fx * g7 + Fy * g8;
        duy += dFu * Fy - R(2) * Fy * g7 + Fx * g8;
        // Q(S, u), with |F_int|^2/(G psi^2) = G |S|^2; the coefficients carry one factor G
        const R dQ1 = d1 + cc.q2fac * d2;
        dSx += R(2) * Sx * (cc.kq1 * dQ1 + cc.kq7 * d7) + cc.kq7 * Sy * d8;
        dSy += R(2) * Sy * (cc.kq1 * dQ1 - cc.kq7 * d7) + cc.kq7 * Sx * d8;
        R dG = (Q1 * dQ1 + Q7 * d7 + Q8 * d8) / G;
        if (improved) {
            dux += A4 * d4;
            duy += A6 * d6;
            dSx += R(2) * Sx * (cc.c1G * ux * d4 - cc.c2G * uy * d6);
            dSy += R(2) * Sy * (cc.c1G * uy * d6 - cc.c2G * ux * d4);
            dG += (Q4 * d4 + Q6 * d6) / G;
        }
        // u = (j + F/2)/rho
        const R djx = dux * inv, djy = duy * inv;
        dFx += R(0.5) * djx;
        dFy += R(0.5) * djy;
        drho -= (ux * dux + uy * duy) * inv;
        // F = -G psi S + F_ext
        if (kp.force_mode == 0) {
            gFx = dFx;
            gFy = dFy;
        } else {
            gFx = (rho - cc.rho_g) * dFx;
            gFy = (rho - cc.rho_g) * dFy;
            drho += cc.Fx * dFx + cc.Fy * dFy;
        }
        const R dpsi_loc = -G * (Sx * dFx + Sy * dFy);
        dG -= psi * (Sx * dFx + Sy * dFy);
        dSx -= G * psi * dFx;
        dSy -= G * psi * dFy;
        // walls in the stencil carry psi(rho_s; T, G)
        R dpsi_s = R(0);
#pragma unroll
        for (int i = 1; i < 9; ++i)
            if ((wm >> i) & 1u) dpsi_s += omega_<R>(i) * (R(ex_(i)) * dSx + R(ey_(i)) * dSy);
        if (dpsi_s != R(0)) {
            R prs, pTs;
            p_eos_derivs<R>(kp, cc.rho_s, prs, pTs);
            dG += -cc.psi_s / (R(2) * G) * dpsi_s;
            gT = pTs / (G * cc.psi_s) * dpsi_s;
        }
        gG = dG;

        // g_i = drho + e_i . dj + (M^T dm)_i
        const R base_ax = -dm1 - R(2) * dm2, base_dg = R(2) * dm1 + dm2;
        R *go = static_cast<R *>(aa.g_out);
        const int64_t P = kp.plane;
        go[0 * P + k] = drho + R(-4) * dm1 + R(4) * dm2;
        go[1 * P + k] = drho + djx + base_ax - R(2) * dm4 + dm7;
        go[2 * P + k] = drho + djy + base_ax - R(2) * dm6 - dm7;
        go[3 * P + k] = drho - djx + base_ax + R(2) * dm4 + dm7;
        go[4 * P + k] = drho - djy + base_ax + R(2) * dm6 - dm7;
        go[5 * P + k] = drho + djx + djy + base_dg + dm4 + dm6 + dm8;
        go[6 * P + k] = drho - djx + djy + base_dg - dm4 + dm6 - dm8;
        go[7 * P + k] = drho - djx - djy + base_dg - dm4 - dm6 + dm8;
        go[8 * P + k] = drho + djx - djy + base_dg + dm4 - dm6 - dm8;
        R *dS = static_cast<R *>(aa.dS);
        dS[k] = dSx;
        dS[P + k] = dSy;
        static_cast<R *>(aa.dpsi)[k] = dpsi_loc;
        static_cast<R *>(aa.rho)[k] = rho;
    }
    const R v[5] = {gFx, gFy, gG, gT, Jt};
    block_add<5>(v, aa.part, SLOT_FX);
}

// Pass 2: dJ/dpsi(x) from the stencils that read psi(x), then c(x) = psi'(rho) dJ/dpsi.
template <class S>
__global__ void __launch_bounds__(kRowThreads) k_adj2(KParams kp, AdjArgs aa)
{
    typedef typename Codec<S>::R R;
    grid_dependency_wait();
    allow_dependent_launch();
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    const int64_t node = (int64_t)y * kp.nx + x, k = (int64_t)y * kp.pitch + x;
    R gG = R(0), gT = R(0);
    if (x < kp.nx && !node_is_solid(kp, node)) {
        const Consts<R> &cc = cst<R>(kp);
        const R *dS = static_cast<const R *>(aa.dS);
        R dpsi = static_cast<const R *>(aa.dpsi)[k];
        const Around nb = around(kp, x, y);
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            // the node z = x - e_i = x + e_opp(i) has x in its stencil along e_i
            const int o = opp_(i);
            if (!nb.in(o)) continue;
            if (kp.solid != nullptr && kp.solid[nb.n(o)] != 0) continue;
            const int64_t kz = nb.k(o);
            dpsi += omega_<R>(i) * (R(ex_(i)) * dS[kz] + R(ey_(i)) * dS[kp.plane + kz]);
        }
        const R rho = static_cast<const R *>(aa.rho)[k];
        const R psi = static_cast<const R *>(kp.psi)[node];
        R p_rho, p_T;
        p_eos_derivs<R>(kp, rho, p_rho, p_T);
        // psi^2 = 2 (p - rho/3)/G
        const R Gpsi = cc.G * psi;
        static_cast<R *>(aa.c_out)[k] = (p_rho - R(1.0 / 3.0)) / Gpsi * dpsi;
        gT = p_T / Gpsi * dpsi;
        gG = -psi / (R(2) * cc.G) * dpsi;
    }
    const R v[2] = {gG, gT};
    block_add<2>(v, aa.part, SLOT_G2);
}

// lambda_0 = dJ/dA at the starting state (no objective weight at t = 0), FP64 [9][ny][nx].
template <class S>
__global__ void __launch_bounds__(kRowThreads) k_adj_lambda(KParams kp, AdjArgs aa, double *out)
{
    typedef typename Codec<S>::R R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= kp.nx) return;
    const int64_t n = (int64_t)kp.nx * kp.ny, node = (int64_t)y * kp.nx + x;
    R lam[9];
    if (node_is_solid(kp, node)) {
#pragma unroll
        for (int i = 0; i < 9; ++i) lam[i] = R(0);
    } else {
        const Around nb = around(kp, x, y);
        lambda_at<R>(kp, aa, nb, wall_mask(kp, nb), R(0), R(aa.inv_nfluid), lam);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) out[i * n + node] = double(lam[i]);
}

// FP64 sum over fluid nodes of sum_i W_i(x) A_i(x) for the state kp.src.
template <class S>
__global__ void __launch_bounds__(kRowThreads) k_objective(KParams kp, int objective, double inv_nfluid, double *acc)
{
    typedef typename Codec<S>::R R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    const int64_t node = (int64_t)y * kp.nx + x;
    double v = 0.0;
    if (x < kp.nx && !node_is_solid(kp, node)) {
        AdjArgs aa{};
        aa.objective = objective;
        aa.inv_nfluid = inv_nfluid;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            int64_t kn;
            const bool wall = (i != 0) && wall_link(kp, x, y, i, kn);
            const double w = double(objective_weight<R>(aa.objective, i, wall, R(aa.inv_nfluid)));
            if (w != 0.0) v += w * double(load_pop<S>(kp, i, x, y));
        }
    }
    block_atomic_add(v, acc);
}

// Sum of the per-block slots: out[k] = sum over blocks of part[b][k], one block per slot,
// in a fixed order (instantiated per storage type S, like the passes it sums).
template <class S>
__global__ void __launch_bounds__(256) k_adj_reduce(const double *part, int64_t blocks, double *out)
{
    __shared__ double red[8];
    const int k = blockIdx.x;
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < blocks; b += blockDim.x) s += part[b * kAdjSlots + k];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += red[q];
        out[k] = t;
    }
}

template <class S>
struct Adjoint {
    static cudaError_t pass1(const KParams &kp, const AdjArgs &aa, cudaStream_t st)
    {
        return launch_dependent(k_adj1<S>, row_grid(kp), dim3(kRowThreads), 0, st, kp, aa);
    }
    static cudaError_t pass2(const KParams &kp, const AdjArgs &aa, cudaStream_t st)
    {
        return launch_dependent(k_adj2<S>, row_grid(kp), dim3(kRowThreads), 0, st, kp, aa);
    }
    static cudaError_t lambda(const KParams &kp, const AdjArgs &aa, double *out, cudaStream_t st)
    {
        k_adj_lambda<S><<<row_grid(kp), kRowThreads, 0, st>>>(kp, aa, out);
        return cudaGetLastError();
    }
    // blocks of the row grid of the transposed passes (rows of the partial-sum array)
    static int64_t blocks(const KParams &kp) { return (int64_t)row_grid(kp).x * row_grid(kp).y; }
    static cudaError_t reduce(const KParams &kp, const double *part, double *out, cudaStream_t st)
    {
        k_adj_reduce<S><<<kAdjSlots, 256, 0, st>>>(part, blocks(kp), out);
        return cudaGetLastError();
    }
    static cudaError_t objective(const KParams &kp, int obj, double inv_nfluid, double *acc, cudaStream_t st)
    {
        k_objective<S><<<row_grid(kp), kRowThreads, 0, st>>>(kp, obj, inv_nfluid, acc);
        return cudaGetLastError();
    }
};

}  // namespace lbm
