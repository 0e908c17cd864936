// Device building blocks of the D2Q9 pseudopotential MRT step: lattice constants,
// storage codecs, EOS pseudopotential, pull streaming with wall links, collision.
// Every kernel variant calls these same functions in the same order, so the two-pass
// and the fused kernels produce bit-identical populations.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "lbm_internal.h"

namespace lbm {

// ---------------------------------------------------------------- lattice --
// D2Q9: e_0 = (0,0); e_1..e_4 = (1,0),(0,1),(-1,0),(0,-1); e_5..e_8 = (1,1),(-1,1),
// (-1,-1),(1,-1) -- the numbering the sums of Eqs. (ali.2) and (obl.3) use.
__host__ __device__ constexpr int ex_(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int ey_(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }
__host__ __device__ constexpr int opp_(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5); }
template <class R>
__host__ __device__ constexpr R w_(int i) { return i == 0 ? R(4.0 / 9.0) : (i <= 4 ? R(1.0 / 9.0) : R(1.0 / 36.0)); }
// Eq. (fint) nearest-neighbour weights: w(1) = 1/3, w(2) = 1/12
template <class R>
__host__ __device__ constexpr R omega_(int i) { return i == 0 ? R(0) : (i <= 4 ? R(1.0 / 3.0) : R(1.0 / 12.0)); }

}  // namespace lbm

#include "lbm_f32.cuh"
#include "lbm_f64.cuh"

namespace lbm {

// ------------------------------------------------ dependent launches ------
// Kernels of the step chain are launched with programmatic stream serialization: the next
// grid may be scheduled while the previous one drains, and waits here until that grid has
// completed and its memory is visible, before touching global memory.  Launched without
// that attribute, both instructions do nothing.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependent_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <class... KArgs, class... Args>
inline cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                    Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <class R>
constexpr bool is_f64() { return std::is_same<R, double>::value; }

// Options a kernel may fix at compile time; -1 means "read from KParams at run time".
template <int IMPROVED = -1, int VAR_TAU = -1, int FORCE_MODE = -1, int NODE_REF = -1>
struct Opts {
    static __device__ __forceinline__ bool improved(const KParams &kp) { return IMPROVED >= 0 ? IMPROVED != 0 : kp.improved != 0; }
    static __device__ __forceinline__ bool var_tau(const KParams &kp) { return VAR_TAU >= 0 ? VAR_TAU != 0 : kp.var_tau != 0; }
    static __device__ __forceinline__ int force_mode(const KParams &kp) { return FORCE_MODE >= 0 ? FORCE_MODE : kp.force_mode; }
    static __device__ __forceinline__ bool per_node_ref(const KParams &kp) { return NODE_REF >= 0 ? NODE_REF != 0 : kp.per_node_ref != 0; }
};
typedef Opts<> RuntimeOpts;

// Kernel constants in arithmetic type R.
template <class R> __device__ __forceinline__ const Consts<R> &cst(const KParams &kp);
template <> __device__ __forceinline__ const Consts<double> &cst<double>(const KParams &kp) { return kp.cd; }
template <> __device__ __forceinline__ const Consts<float> &cst<float>(const KParams &kp) { return kp.cf; }

// ------------------------------------------------------------ codecs -------
// Stored value <-> population.  FP16/BF16 keep (f_i - w_i rho_ref) 2^k, rounded to
// nearest even; decode multiplies back by 2^-k (exact) and adds w_i rho_ref.
template <class S> struct Codec;
template <> struct Codec<double> {
    typedef double R;
    static __device__ __forceinline__ R dec(double v, R, R) { return v; }
    static __device__ __forceinline__ double enc(R f, R, R) { return f; }
};
template <> struct Codec<float> {
    typedef float R;
    static __device__ __forceinline__ R dec(float v, R, R) { return v; }
    static __device__ __forceinline__ float enc(R f, R, R) { return f; }
};
template <> struct Codec<__half> {
    typedef float R;
    static __device__ __forceinline__ R dec(__half v, R wref, R inv_scale) { return __fmaf_rn(__half2float(v), inv_scale, wref); }
    static __device__ __forceinline__ __half enc(R f, R wref, R scale) { return __float2half_rn(__fmul_rn(__fsub_rn(f, wref), scale)); }
};
template <> struct Codec<__nv_bfloat16> {
    typedef float R;
    static __device__ __forceinline__ R dec(__nv_bfloat16 v, R wref, R inv_scale) { return __fmaf_rn(__bfloat162float(v), inv_scale, wref); }
    static __device__ __forceinline__ __nv_bfloat16 enc(R f, R wref, R scale) { return __float2bfloat16_rn(__fmul_rn(__fsub_rn(f, wref), scale)); }
};
template <class S> struct IsDev { static constexpr bool value = false; };
template <> struct IsDev<__half> { static constexpr bool value = true; };
template <> struct IsDev<__nv_bfloat16> { static constexpr bool value = true; };

// ------------------------------------------------------ stochastic rounding ---
// Optional rounding of the 16-bit storage: the scaled deviation is rounded up with a
// probability equal to the fraction of an ulp that rounding down would discard
// (cvt.rs.{f16x2,bf16x2}.f32: random bits are added to the discarded bits, then truncated).
// Nodes come in pairs (2m, 2m + 1) of the padded row-major index k = y pitch + x (pitch is
// even); the pair's random word for population i is sr_bits(sr_hash(m, seed), i), and the
// paired conversion takes the even node's bits from the low half of the word and the odd
// node's from the high half, so the two step kernels (one node or two per thread) round
// every value alike.  sr_hash is MurmurHash3's 32-bit finaliser of the pair index mixed with
// the step's seed.
__device__ __forceinline__ uint32_t sr_hash(uint32_t pair, uint32_t seed)
{
    uint32_t h = pair * 0x9E3779B1u ^ seed;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}
// a different odd multiplier per population (a bijection of every low-bit window)
__device__ __forceinline__ uint32_t sr_bits(uint32_t h, int i) { return h * (0x9E3779B9u + 0x3C6EF372u * (uint32_t)i); }

template <class S> struct SRound;
template <> struct SRound<__half> {
    // low half <- lo, high half <- hi
    static __device__ __forceinline__ uint32_t pack(float lo, float hi, uint32_t r)
    {
        uint32_t d;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
        return d;
    }
    static __device__ __forceinline__ __half from_bits(unsigned short b)
    {
        __half_raw h;
        h.x = b;
        return __half(h);
    }
};
template <> struct SRound<__nv_bfloat16> {
    static __device__ __forceinline__ uint32_t pack(float lo, float hi, uint32_t r)
    {
        uint32_t d;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
        return d;
    }
    static __device__ __forceinline__ __nv_bfloat16 from_bits(unsigned short b)
    {
        __nv_bfloat16_raw h;
        h.x = b;
        return __nv_bfloat16(h);
    }
};
// One already-scaled value rounded stochastically as element `odd` of its node pair.
template <class S>
__device__ __forceinline__ S sr_one(float v, uint32_t r, int odd)
{
    const uint32_t d = odd ? SRound<S>::pack(0.f, v, r) : SRound<S>::pack(v, 0.f, r);
    return SRound<S>::from_bits((unsigned short)(odd ? d >> 16 : d & 0xffffu));
}

// Stored value of population i of node k: the codec's encode, or with stochastic rounding
// the same scaled deviation (f - w_i ref) 2^k rounded with the node pair's random bits h.
template <class S>
__device__ __forceinline__ S enc_pop(const KParams &kp, typename Codec<S>::R f, typename Codec<S>::R wref,
                                     typename Codec<S>::R scale, int64_t k, int i, uint32_t h)
{
    if constexpr (IsDev<S>::value) {
        if (kp.sr) return sr_one<S>(__fmul_rn(__fsub_rn(f, wref), scale), sr_bits(h, i), (int)(k & 1));
    }
    return Codec<S>::enc(f, wref, scale);
}

// ------------------------------------------------------------- EOS ---------
// Sec. 2: psi = sqrt(2 (p_EOS - rho c_s^2)/G); van der Waals (Sec. 3) or Carnahan-Starling.
template <class R>
__device__ __forceinline__ R p_eos(const KParams &kp, R rho)
{
    const R a = cst<R>(kp).eos_a, b = cst<R>(kp).eos_b, RT = cst<R>(kp).eos_RT, K = cst<R>(kp).eos_K;
    if (kp.eos == 0) return K * (rho * RT / (R(1) - b * rho) - a * rho * rho);
    const R eta = b * rho * R(0.25);
    const R om = R(1) - eta;
    const R num = R(1) + eta + eta * eta - eta * eta * eta;
    return K * (rho * RT * num / (om * om * om) - a * rho * rho);
}

template <class R>
__device__ __forceinline__ R psi_of(const KParams &kp, R rho)
{
    if constexpr (is_f64<R>()) return f64::psi_of(kp, rho);
    else return psi_v<v1>(kp, v1{rho}).v;
}

// ------------------------------------------------------------ geometry -----
// Wrap (x, y) along periodic directions; false when the point lies beyond a
// non-periodic edge (a wall).  Only offsets of one node are ever wrapped.
__device__ __forceinline__ bool wrap_xy(const KParams &kp, int &x, int &y)
{
    if (x < 0 || x >= kp.nx) {
        if (!kp.periodic_x) return false;
        x = (x < 0) ? x + kp.nx : x - kp.nx;
    }
    if (y < 0 || y >= kp.ny) {
        if (!kp.periodic_y) return false;
        y = (y < 0) ? y + kp.ny : y - kp.ny;
    }
    return true;
}

__device__ __forceinline__ bool is_wall_at(const KParams &kp, int x, int y)
{
    if (!wrap_xy(kp, x, y)) return true;
    return kp.solid != nullptr && kp.solid[(int64_t)y * kp.nx + x] != 0;
}

// The 3 x 3 neighbourhood of node (x, y), computed once per node so that everything a
// kernel gathers from the eight neighbours (the pull, the psi stencil, the wall mask and the
// gathers of the transposed step) shares one set of index arithmetic: the columns x - 1, x,
// x + 1 and rows y - 1, y, y + 1 wrapped along periodic directions, and bit i set when
// x + e_i lies inside the lattice.  A neighbour beyond a non-periodic edge takes the node's
// own column or row, so no index leaves the lattice even where it is not used.  k(i): the
// pitched plane index of x + e_i; n(i): its psi-field index (nx * ny <= 2^31, so it fits an
// int).
struct Around {
    const KParams &kp;
    int xc[3], yr[3];
    unsigned inside;
    __device__ __forceinline__ int64_t k(int i) const { return (int64_t)yr[ey_(i) + 1] * kp.pitch + xc[ex_(i) + 1]; }
    __device__ __forceinline__ int64_t n(int i) const { return (int64_t)(yr[ey_(i) + 1] * kp.nx + xc[ex_(i) + 1]); }
    __device__ __forceinline__ bool in(int i) const { return (inside >> i) & 1u; }
};

__device__ __forceinline__ Around around(const KParams &kp, int x, int y)
{
    Around a{kp};
    bool okx[3], oky[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int xx = x + d - 1, yy = y + d - 1;
        okx[d] = oky[d] = true;
        if (xx < 0 || xx >= kp.nx) {
            if (kp.periodic_x) xx = xx < 0 ? xx + kp.nx : xx - kp.nx;
            else okx[d] = false, xx = x;
        }
        if (yy < 0 || yy >= kp.ny) {
            if (kp.periodic_y) yy = yy < 0 ? yy + kp.ny : yy - kp.ny;
            else oky[d] = false, yy = y;
        }
        a.xc[d] = xx;
        a.yr[d] = yy;
    }
    a.inside = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i)
        if (okx[ex_(i) + 1] && oky[ey_(i) + 1]) a.inside |= 1u << i;
    return a;
}

// ------------------------------------------------------- global access ------
// Population i of the source state at pitched index k (or at node (x, y)), decoded.
template <class S>
__device__ __forceinline__ typename Codec<S>::R load_pop_at(const KParams &kp, int i, int64_t k)
{
    typedef typename Codec<S>::R R;
    const S *A = static_cast<const S *>(kp.src);
    R wref = R(0);
    if constexpr (IsDev<S>::value) wref = __fmul_rn(w_<R>(i), kp.per_node_ref ? R(kp.ref_src[k]) : cst<R>(kp).rho_ref);
    return Codec<S>::dec(A[i * kp.plane + k], wref, cst<R>(kp).inv_scale);
}

template <class S>
__device__ __forceinline__ typename Codec<S>::R load_pop(const KParams &kp, int i, int x, int y)
{
    return load_pop_at<S>(kp, i, (int64_t)y * kp.pitch + x);
}

// Link closed by a wall (x - e_i is a wall): the population that left (x, y) toward it
// comes back.  `at(k, xx, yy)` reads population k of node (xx, yy) (xx, yy in domain).
// half-way (q = 1/2): f_i = fbar_o(x) + mw
// q <  1/2: f_i = 2q fbar_o(x) + (1 - 2q) fbar_o(x + e_i) + mw          (Bouzidi et al.)
// q >  1/2: f_i = fbar_o(x)/(2q) + (2q - 1)/(2q) fbar_i(x) + mw/(2q)
// mw = 2 w_o rho_w (e_i . u_w)/c_s^2 with rho_w = sum_k fbar_k(x) (Lallemand & Luo).
// mom (may be null) accumulates the momentum handed to the wall, -e_i (fbar_o(x) + f_i).
template <class R, int i, class At>
__device__ __forceinline__ R bounce(const KParams &kp, int x, int y, const At &at, R *mom)
{
    constexpr int o = opp_(i);
    const R fo = at(o, x, y);
    R mw = R(0);
    if (kp.wall_u != nullptr) {
        int wx = x - ex_(i), wy = y - ey_(i);
        if (wrap_xy(kp, wx, wy)) {
            const int64_t wk = (int64_t)wy * kp.nx + wx;
            const R uwx = R(kp.wall_u[wk]);
            const R uwy = R(kp.wall_u[(int64_t)kp.nx * kp.ny + wk]);
            // a wall at rest adds nothing (mw = +-0, which leaves the sum below unchanged)
            if (uwx != R(0) || uwy != R(0)) {
                R rho_w = R(0);
#pragma unroll
                for (int k = 0; k < 9; ++k) rho_w += at(k, x, y);
                mw = R(2) * w_<R>(o) * rho_w * (R(ex_(i)) * uwx + R(ey_(i)) * uwy) * R(3);
            }
        }
    }
    R q = R(0.5);
    if (kp.q != nullptr) q = R(kp.q[(int64_t)(o - 1) * kp.nx * kp.ny + (int64_t)y * kp.nx + x]);
    int xb = x + ex_(i), yb = y + ey_(i);
    if (q < R(0.5) && is_wall_at(kp, xb, yb)) q = R(0.5);
    R f;
    if (q < R(0.5)) {
        wrap_xy(kp, xb, yb);
        f = R(2) * q * fo + (R(1) - R(2) * q) * at(o, xb, yb) + mw;
    } else if (q == R(0.5)) {
        f = fo + mw;
    } else {
        f = fo / (R(2) * q) + (R(2) * q - R(1)) / (R(2) * q) * at(i, x, y) + mw / (R(2) * q);
    }
    if (mom != nullptr) {
        mom[0] += -R(ex_(i)) * (fo + f);
        mom[1] += -R(ey_(i)) * (fo + f);
    }
    return f;
}

// Pull streaming, Eq. (lbe.str): f_i(x) = fbar_i(x - e_i), wall links bounced back.
template <class R, int i, class At>
__device__ __forceinline__ R pull_one(const KParams &kp, int x, int y, const At &at, R *mom)
{
    if (i == 0) return at(0, x, y);
    int xs = x - ex_(i), ys = y - ey_(i);
    const bool inside = wrap_xy(kp, xs, ys);
    if (inside && (kp.solid == nullptr || kp.solid[(int64_t)ys * kp.nx + xs] == 0)) return at(i, xs, ys);
    return bounce<R, i>(kp, x, y, at, mom);
}

template <class R, class At>
__device__ __forceinline__ void pull_node(const KParams &kp, int x, int y, const At &at, R (&f)[9], R *mom)
{
    f[0] = pull_one<R, 0>(kp, x, y, at, mom);
    f[1] = pull_one<R, 1>(kp, x, y, at, mom);
    f[2] = pull_one<R, 2>(kp, x, y, at, mom);
    f[3] = pull_one<R, 3>(kp, x, y, at, mom);
    f[4] = pull_one<R, 4>(kp, x, y, at, mom);
    f[5] = pull_one<R, 5>(kp, x, y, at, mom);
    f[6] = pull_one<R, 6>(kp, x, y, at, mom);
    f[7] = pull_one<R, 7>(kp, x, y, at, mom);
    f[8] = pull_one<R, 8>(kp, x, y, at, mom);
}

// The same pull with the node's neighbourhood nb (x - e_i = x + e_opp(i)); `at.at_k(k, kk)`
// reads population k at pitched index kk.
template <class R, int i, class At>
__device__ __forceinline__ R pull_one_nb(const KParams &kp, const Around &nb, int x, int y, const At &at, R *mom)
{
    if (i == 0) return at.at_k(0, nb.k(0));
    constexpr int o = opp_(i);
    if (nb.in(o) && (kp.solid == nullptr || kp.solid[nb.n(o)] == 0)) return at.at_k(i, nb.k(o));
    return bounce<R, i>(kp, x, y, at, mom);
}

template <class R, class At>
__device__ __forceinline__ void pull_node_nb(const KParams &kp, const Around &nb, int x, int y, const At &at,
                                             R (&f)[9], R *mom)
{
    f[0] = pull_one_nb<R, 0>(kp, nb, x, y, at, mom);
    f[1] = pull_one_nb<R, 1>(kp, nb, x, y, at, mom);
    f[2] = pull_one_nb<R, 2>(kp, nb, x, y, at, mom);
    f[3] = pull_one_nb<R, 3>(kp, nb, x, y, at, mom);
    f[4] = pull_one_nb<R, 4>(kp, nb, x, y, at, mom);
    f[5] = pull_one_nb<R, 5>(kp, nb, x, y, at, mom);
    f[6] = pull_one_nb<R, 6>(kp, nb, x, y, at, mom);
    f[7] = pull_one_nb<R, 7>(kp, nb, x, y, at, mom);
    f[8] = pull_one_nb<R, 8>(kp, nb, x, y, at, mom);
}

// FP32 values as one-node lanes of the FP32 formulation (lbm_f32.cuh)
__device__ __forceinline__ void as_dev1(const float (&f)[9], v1 (&d)[9])
{
    v1 g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = v1{f[i]};
    to_dev(g, d);
}

template <class R>
__device__ __forceinline__ R density(const R (&f)[9])
{
    if constexpr (is_f64<R>()) {
        return f64::density(f);
    } else {
        v1 d[9];
        as_dev1(f, d);
        return density_dev(d).v;
    }
}

// ------------------------------------------------------------ forces -------
template <class R, class O = RuntimeOpts>
__device__ __forceinline__ void external_force(const KParams &kp, int64_t node, R rho, R &Fex, R &Fey)
{
    const int mode = O::force_mode(kp);
    if (mode == 0) {
        Fex = cst<R>(kp).Fx;
        Fey = cst<R>(kp).Fy;
    } else if (mode == 1) {  // Sec. 3.3: (rho - rho_g) g
        Fex = (rho - cst<R>(kp).rho_g) * cst<R>(kp).Fx;
        Fey = (rho - cst<R>(kp).rho_g) * cst<R>(kp).Fy;
    } else {
        Fex = kp.fext ? R(kp.fext[node]) : R(0);
        Fey = kp.fext ? R(kp.fext[(int64_t)kp.nx * kp.ny + node]) : R(0);
    }
}

// S = sum_{i=1..8} w(|e_i|^2) psi(x + e_i) e_i, so F_int = -G psi(x) S (Eq. fint).
// `ps(i)` returns psi of the neighbour along e_i.
template <class R, class Ps>
__device__ __forceinline__ void stencil_S(const Ps &ps, R &Sx, R &Sy)
{
    if constexpr (is_f64<R>()) {
        f64::stencil_S(ps, Sx, Sy);
    } else {
        v1 sx, sy;
        stencil_v<v1>(v1{ps(1)}, v1{ps(2)}, v1{ps(3)}, v1{ps(4)}, v1{ps(5)}, v1{ps(6)}, v1{ps(7)}, v1{ps(8)}, sx, sy);
        Sx = sx.v;
        Sy = sy.v;
    }
}

// --------------------------------------------------------- collision -------
// Stages 5-8 of a node: u = (j + F/2)/rho (Eq. rho.rhou); m = M f; m_eq, F_m (Sec. 2);
// Q_m original or improved (Eqs. qm.improved, qm46.improved); rates s_0 = s_j = 1,
// s_e = s_eps = s_p = 1/tau, (1/s_q - 1/2)(1/s_p - 1/2) = Lambda (Sec. 3);
// m_bar = m + F_m - S (m - m_eq + F_m/2) + S Q_m (Eq. lbe.col); f_bar = M^-1 m_bar.
template <class R, class O = RuntimeOpts>
__device__ __forceinline__ void collide(const KParams &kp, const R (&f)[9], R rho, R psi, R Sx, R Sy,
                                        R Fex, R Fey, R (&fb)[9], R &ux, R &uy)
{
    if constexpr (is_f64<R>()) {
        f64::collide(kp, f, psi, Sx, Sy, Fex, Fey, fb, ux, uy);
    } else {
        v1 d[9], b[9], u, v;
        as_dev1(f, d);
        collide_v<v1, O>(kp, d, v1{rho}, v1{psi}, v1{Sx}, v1{Sy}, v1{Fex}, v1{Fey}, b, u, v);
#pragma unroll
        for (int i = 0; i < 9; ++i) fb[i] = b[i].v;
        ux = u.v;
        uy = v.v;
    }
}

// f_bar = M^-1 m_eq(rho, u): the equilibrium used by lbm_init_fields
template <class R>
__device__ __forceinline__ void equilibrium(R rho, R ux, R uy, R (&fb)[9])
{
    if constexpr (is_f64<R>()) {
        f64::equilibrium(rho, ux, uy, fb);
        return;
    }
    const R u2 = ux * ux + uy * uy;
    const R b1 = rho * (R(-2) + R(3) * u2), b2 = rho * (R(1) - R(3) * u2);
    const R b3 = rho * ux, b4 = -rho * ux, b5 = rho * uy, b6 = -rho * uy;
    const R b7 = rho * (ux * ux - uy * uy), b8 = rho * ux * uy;
    const R A0 = rho * R(1.0 / 9.0), B = b1 * R(1.0 / 36.0), C = b2 * R(1.0 / 36.0);
    const R D = b3 * R(1.0 / 6.0), E = b4 * R(1.0 / 12.0), Gy = b5 * R(1.0 / 6.0), H = b6 * R(1.0 / 12.0);
    const R P = b7 * R(0.25), Qp = b8 * R(0.25);
    const R ax = A0 - B - R(2) * C;
    const R dg = A0 + R(2) * B + C;
    fb[0] = A0 - R(4) * B + R(4) * C;
    fb[1] = ax + (D - R(2) * E) + P;
    fb[2] = ax + (Gy - R(2) * H) - P;
    fb[3] = ax - (D - R(2) * E) + P;
    fb[4] = ax - (Gy - R(2) * H) - P;
    fb[5] = dg + (D + E) + (Gy + H) + Qp;
    fb[6] = dg - (D + E) + (Gy + H) - Qp;
    fb[7] = dg - (D + E) - (Gy + H) + Qp;
    fb[8] = dg + (D + E) - (Gy + H) - Qp;
}

// Encode and store the nine post-collision populations of node (x, y) into dst.
template <class S>
__device__ __forceinline__ void store_node(const KParams &kp, int x, int y, const typename Codec<S>::R (&fb)[9],
                                           typename Codec<S>::R rho)
{
    typedef typename Codec<S>::R R;
    S *Bp = static_cast<S *>(kp.dst);
    const int64_t k = (int64_t)y * kp.pitch + x;
    R ref = cst<R>(kp).rho_ref;
    if (IsDev<S>::value && kp.per_node_ref) {
        ref = rho;
        kp.ref_dst[k] = float(rho);
    }
    const R scale = cst<R>(kp).scale;
    const uint32_t h = IsDev<S>::value && kp.sr ? sr_hash((uint32_t)(k >> 1), kp.sr_seed) : 0u;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        if constexpr (IsDev<S>::value) Bp[i * kp.plane + k] = enc_pop<S>(kp, fb[i], __fmul_rn(w_<R>(i), ref), scale, k, i, h);
        else Bp[i * kp.plane + k] = Codec<S>::enc(fb[i], R(0), scale);
    }
}

}  // namespace lbm
