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
// Density, psi, stencil and collision are the FP32 formulation of lbm_f32.cuh evaluated on
// packed pairs; the two-pass step evaluates the same expressions on single nodes, and the
// two agree to FP32 rounding (the compiler fuses some packed multiply-add chains).  The
// storage codec rounds exactly as
// `Codec<>`: the deviation (f - w_i rho_ref) 2^k is formed as one fused multiply-add of
// f 2^k and -(w_i rho_ref) 2^k, which equals the rounded difference times the power of
// two.
#pragma once

#include "k_fused.cuh"

namespace lbm {

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
    static __device__ __forceinline__ void store_sr(float *p, v2 f, uint32_t) { store(p, f); }  // FP32: exact
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
    // stochastic rounding with the pair's random word r (element 0 from its low half)
    static __device__ __forceinline__ void store_sr(__half *p, v2 f, uint32_t r)
    {
        *reinterpret_cast<uint32_t *>(p) = SRound<__half>::pack(f.v.x, f.v.y, r);
    }
};
template <> struct Pair2<__nv_bfloat16> {
    LBM_DEC_PAIR(__nv_bfloat16, __nv_bfloat162, "bf16")
    static __device__ __forceinline__ float load1(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void store(__nv_bfloat16 *p, v2 f)
    {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __float22bfloat162_rn(f.v);
    }
    static __device__ __forceinline__ void store_sr(__nv_bfloat16 *p, v2 f, uint32_t r)
    {
        *reinterpret_cast<uint32_t *>(p) = SRound<__nv_bfloat16>::pack(f.v.x, f.v.y, r);
    }
};
#undef LBM_DEC_PAIR

// One already-scaled FP32 value rounded to the storage type (as the pair stores round).
template <class S> struct Codec2;
template <> struct Codec2<float> {
    static __device__ __forceinline__ void put(float *p, float v) { *p = v; }
};
template <> struct Codec2<__half> {
    static __device__ __forceinline__ void put(__half *p, float v) { *p = __float2half_rn(v); }
};
template <> struct Codec2<__nv_bfloat16> {
    static __device__ __forceinline__ void put(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

__device__ __forceinline__ v2 load_ref_pair(const float *p, int off)
{
    if (off == 0) return v2{*reinterpret_cast<const float2 *>(p)};
    return V(p[off], p[off + 1]);
}

// ------------------------------------------------------------ physics --------
#define LBM_C2(name) v2{q.name}

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

// ----------------------------------------------------- general geometry ------
// Solid flags of columns c0 - 1 .. c0 + 2 of lattice row y (bit k = column c0 - 1 + k), with
// periodic wrapping; nodes beyond a non-periodic edge read as fluid (those links are walls
// by the edge test).
// The four flags are fetched one row ahead of their use (solid_fetch) and combined when
// the row is reached (solid_bits), so the latency of the global loads overlaps a row of work.
struct SolidRow {
    int v[4];
};
__device__ __forceinline__ SolidRow solid_fetch(const KParams &kp, int y, int c0)
{
    SolidRow w{{0, 0, 0, 0}};
    if (y < 0 || y >= kp.ny) {
        if (!kp.periodic_y) return w;
        y = y < 0 ? y + kp.ny : y - kp.ny;
    }
    const uint8_t *r = kp.solid + (int64_t)y * kp.nx;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int x = c0 - 1 + k;
        if (x < 0 || x >= kp.nx) {
            if (!kp.periodic_x) continue;
            x = x < 0 ? x + kp.nx : x - kp.nx;
        }
        w.v[k] = r[x];
    }
    return w;
}
__device__ __forceinline__ int solid_bits(const SolidRow &w)
{
    return (w.v[0] != 0) | (w.v[1] != 0) << 1 | (w.v[2] != 0) << 2 | (w.v[3] != 0) << 3;
}

// Population k of a node near (xw, yw) read from the staged rows (for `bounce`, which asks
// for the node itself and its neighbour along e_i by lattice coordinates), decoded to FP32
// like the pull: `row`/`ref` point at the staged column of the pair's first node, `e` is
// the element of the pair.
// The three row pointers are separate members and chosen by comparison: an array indexed
// by a run-time row would be placed in local memory, and with it every staged-row access of
// the kernel.
template <class S, int W>
struct StagedAt {
    const KParams &kp;
    const S *rm, *r0, *rp;
    const float *fm, *f0, *fp;
    int e, xw, yw;
    __device__ __forceinline__ float operator()(int k, int xx, int yy) const
    {
        int dx = xx - xw, dy = yy - yw;
        if (dx > 1) dx -= kp.nx;
        else if (dx < -1) dx += kp.nx;
        if (dy > 1) dy -= kp.ny;
        else if (dy < -1) dy += kp.ny;
        const int col = e + dx;
        const S *r = dy < 0 ? rm : (dy > 0 ? rp : r0);
        float v = Pair2<S>::load1(r + k * W + col);
        if constexpr (IsDev<S>::value) {
            const float *f = dy < 0 ? fm : (dy > 0 ? fp : f0);
            const float rf = f0 ? f[col] : kp.cf.rho_ref;
            v = __fmaf_rn(v, kp.cf.inv_scale, __fmul_rn(w_<float>(k), rf));
        }
        return v;
    }
};

// A wall link from its record (KParams::link: link fraction q, moving-wall coefficient c):
// the bounce-back rule of `bounce` (Bouzidi interpolation, moving-wall term c rho_w with
// rho_w the node's own density before the last collision), reading the populations from the
// staged rows.  One 8-byte read per link replaces the separate reads of q, the wall velocity
// and the solid flag of the second node.
template <int I, class At>
__device__ __forceinline__ float bounce_link(const At &at, int x, int y, float2 lk)
{
    constexpr int o = opp_(I);
    const float fo = at(o, x, y);
    const float q = lk.x;
    float mw = 0.f;
    if (lk.y != 0.f) {
        float rho_w = 0.f;
#pragma unroll
        for (int k = 0; k < 9; ++k) rho_w += at(k, x, y);
        mw = lk.y * rho_w;
    }
    if (q < 0.5f) return 2.f * q * fo + (1.f - 2.f * q) * at(o, x + ex_(I), y + ey_(I)) + mw;
    if (q == 0.5f) return fo + mw;
    return fo / (2.f * q) + (2.f * q - 1.f) / (2.f * q) * at(I, x, y) + mw / (2.f * q);
}

// Wall links of the pair (edges beyond a non-periodic side and solid nodes): the bounce-back
// of the two-pass step (half-way, moving wall, interpolated), element by element.
#define LBM_GEOM_LINK(I)                                                                                      \
    {                                                                                                         \
        const int ys_ = rp - ey_(I);                                                                          \
        const bool yw_ = !kp.periodic_y && (ys_ < 0 || ys_ >= ny);                                            \
        const int wsrc_ = I == 0 ? 0 : (ey_(I) > 0 ? win_m : (ey_(I) < 0 ? win_p : win_0));                   \
        _Pragma("unroll") for (int e = 0; e < 2; ++e) {                                                       \
            if ((own >> e) & 1) continue;                                                                     \
            const int xs_ = c0 + e - ex_(I);                                                                  \
            const bool wall_ = yw_ || (!kp.periodic_x && (xs_ < 0 || xs_ >= nx)) || ((wsrc_ >> (e - ex_(I) + 1)) & 1); \
            if (wall_) {                                                                                      \
                float v_;                                                                                     \
                if constexpr (GEOM == 1) {                                                                    \
                    /* half-way: the population that left the node toward the wall returns */                \
                    constexpr int o_ = opp_(I);                                                               \
                    v_ = Pair2<S>::load1(row[1] + o_ * W + e);                                                \
                    if constexpr (IsDev<S>::value)                                                            \
                        v_ = __fmaf_rn(v_, kp.cf.inv_scale, __fmul_rn(w_<float>(o_), ref[1] ? ref[1][e] : kp.cf.rho_ref)); \
                    v_ = v_ + 0.f;                                                                            \
                } else {                                                                                      \
                    /* interpolated or moving walls: the link records exist (set_geometry) */                 \
                    const StagedAt<S, W> at_{kp, row[0], row[1], row[2], ref[0], ref[1], ref[2], e, xw + e, yw}; \
                    v_ = bounce_link<I>(at_, xw + e, yw, e ? make_float2(lrec[I - 1].z, lrec[I - 1].w)         \
                                                         : make_float2(lrec[I - 1].x, lrec[I - 1].y));       \
                }                                                                                             \
                if (e == 0) f_new[I].v.x = v_;                                                                \
                else f_new[I].v.y = v_;                                                                       \
            }                                                                                                 \
        }                                                                                                     \
    }

#ifndef LBM_FUSED2_MINB
#define LBM_FUSED2_MINB 2  // CTAs per SM the register allocation must allow
#endif
// GEOM: 0 no solid nodes; 1 solid nodes with half-way links only; 2 also interpolated or
// moving walls (through the wall-link records).  The half-way-only instantiation keeps the
// link code out of the kernel.
template <class S, int NW, int RING, bool PERIODIC, class O, int GEOM = 0>
__global__ void __launch_bounds__(32 * (NW + 1), GEOM == 2 ? 3 : LBM_FUSED2_MINB) k_fused2(KParams kp, int seg_rows)
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
    // consumer warps whose 60 columns all lie beyond the lattice (the last strip of a lattice
    // whose width is not a multiple of the strip) leave at once and are not counted by the
    // ring's release barriers
    const int nw_act = min(NW, (nx - x0 + 59) / 60);

    // the state this step reads is the one the previous step wrote, and this step writes
    // the buffer the previous step read: nothing global is touched before it has completed
    grid_dependency_wait();
    allow_dependent_launch();
    if (threadIdx.x == 0) {
        for (int s = 0; s < RING; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, nw_act);
        }
        fence_mbar_init();
        fence_proxy_async();
    }
    __syncthreads();

    if (warp < NW && warp >= nw_act) return;
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
        bool drained = true;
        for (int q = max(first, r - RING); q < r && q <= last; ++q)
            drained &= mbar_wait_bounded(full + ((q - first) & (RING - 1)), (uint32_t)(((q - first) / RING) & 1));
        if (!drained) atomicOr(kp.err, DERR_TIMEOUT);
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
    // solid flags of rows rp - 1, rp, rp + 1 around the pair (general geometry only)
    int win_m = 0, win_0 = 0, win_p = 0, own_old = 0;
    SolidRow win_next{{0, 0, 0, 0}};  // raw flags of row rp + 2, fetched one row early
    if constexpr (GEOM) {
        if (kp.solid) {
            win_0 = solid_bits(solid_fetch(kp, yb - 2, c0));
            win_p = solid_bits(solid_fetch(kp, yb - 1, c0));
            win_next = solid_fetch(kp, yb, c0);
        }
    }
    bool ok = wait_full(first) && wait_full(first + 1);
    for (int rp = yb - 1; rp <= ye && ok; ++rp) {
        if (!wait_full(rp + 1)) {
            ok = false;
            break;
        }
        int own = 0;  // solid flags of the pair in row rp
        if constexpr (GEOM) {
            win_m = win_0;
            win_0 = win_p;
            if (kp.solid) {
                win_p = solid_bits(win_next);
                win_next = solid_fetch(kp, rp + 2, c0);
            }
            own = (win_0 >> 1) & 3;
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
            if (!PERIODIC && !GEOM) {
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
                            // as the pull's decode: one rounding of w_o ref, one of the sum
                            r0 = __fmaf_rn(r0, inv_scale, __fmul_rn(w_<float>(o), rf0));
                            r1 = __fmaf_rn(r1, inv_scale, __fmul_rn(w_<float>(o), rf1));
                        }
                        if (w0) f_new[i].v.x = r0 + 0.f;
                        if (w1) f_new[i].v.y = r1 + 0.f;
                    }
                }
            }
            if constexpr (GEOM) {
                // a link can only be a wall link when a solid node lies among columns c0 - 1 ..
                // c0 + 2 of rows rp - 1 .. rp + 1, or those reach beyond a non-periodic edge;
                // most pairs have neither and skip the per-link tests
                const bool edge = (!kp.periodic_y && (rp - 1 < 0 || rp + 1 >= ny)) ||
                                  (!kp.periodic_x && (c0 - 1 < 0 || c0 + 2 >= nx));
                if ((kp.solid || kp.q || kp.wall_u) && (edge || (win_m | win_0 | win_p) != 0)) {
                    const int yw = rp < 0 ? rp + ny : (rp >= ny ? rp - ny : rp);
                    const int xw = c0 < 0 ? c0 + nx : (c0 >= nx ? c0 - nx : c0);
                    // the pair's eight link records, requested together (one 16-byte read per
                    // direction: both nodes), so their latency is paid once
                    float4 lrec[8];
                    if constexpr (GEOM == 2) {
                        const float4 *lk = reinterpret_cast<const float4 *>(kp.link + (int64_t)yw * kp.pitch + xw);
#pragma unroll
                        for (int d = 0; d < 8; ++d) lrec[d] = lk[(int64_t)d * (kp.plane / 2)];
                    }
                    LBM_GEOM_LINK(1) LBM_GEOM_LINK(2) LBM_GEOM_LINK(3) LBM_GEOM_LINK(4)
                    LBM_GEOM_LINK(5) LBM_GEOM_LINK(6) LBM_GEOM_LINK(7) LBM_GEOM_LINK(8)
                }
            }
            // the pulled populations are kept in rest-state deviation form for the collision
            {
                v2 f[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i] = f_new[i];
                to_dev(f, f_new);
            }
            rho_new = density_dev(f_new);
            psi_new = psi_v<v2>(kp, rho_new);
            if constexpr (GEOM) {
                if (own) {
                    // solid nodes: psi of the virtual wall density; rho 1 keeps the unused
                    // arithmetic of the pair finite
                    const int yw = rp < 0 ? rp + ny : (rp >= ny ? rp - ny : rp);
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        if (!((own >> e) & 1)) continue;
                        const int xe = c0 + e < 0 ? c0 + e + nx : (c0 + e >= nx ? c0 + e - nx : c0 + e);
                        const float ps = kp.wall_psi ? float(kp.wall_psi[(int64_t)yw * nx + xe]) : kp.cf.psi_s;
                        if (e == 0) psi_new.v.x = ps, rho_new.v.x = 1.f;
                        else psi_new.v.y = ps, rho_new.v.y = 1.f;
                    }
                }
            }
        }
        __syncwarp();
        // row rp - 1 is not needed any more by this warp
        if (lane == 0 && rp - 1 >= first) mbar_arrive(empty + ((rp - 1 - first) & (RING - 1)));
        // psi of the columns left of the pair and right of it, from the adjacent lanes
        const float am = __shfl_up_sync(0xffffffffu, psi_m2.v.y, 1), bm = __shfl_down_sync(0xffffffffu, psi_m2.v.x, 1);
        const float a0 = __shfl_up_sync(0xffffffffu, psi_m1.v.y, 1), b0 = __shfl_down_sync(0xffffffffu, psi_m1.v.x, 1);
        const float ap = __shfl_up_sync(0xffffffffu, psi_new.v.y, 1), bp = __shfl_down_sync(0xffffffffu, psi_new.v.x, 1);
        const int y = rp - 1;
        // psi of the state read, for a caller that keeps it (the adjoint's recompute): the
        // pair's own row, solid nodes included, as the psi pass writes it
        if (kp.psi_out != nullptr && y >= yb && collides)
            Pair2<float>::store(kp.psi_out + (int64_t)y * nx + c0, psi_m1);
        if (y >= yb && collides && (!GEOM || own_old != 3)) {
            {
                v2 fb[9];
                // rows y-1 (m), y (0), y+1 (p); left (L), centre, right (R) columns of each node
                const v2 Lm = V(am, psi_m2.v.x), Rm = V(psi_m2.v.y, bm);
                const v2 L0 = V(a0, psi_m1.v.x), R0 = V(psi_m1.v.y, b0);
                const v2 Lp = V(ap, psi_new.v.x), Rp = V(psi_new.v.y, bp);
                // S of Eq. (fint): east R0, north psi_new, west L0, south psi_m2, NE Rp, NW Lp,
                // SW Lm, SE Rm
                v2 Sx, Sy, Fex, Fey, ux, uy;
                stencil_v<v2>(R0, psi_new, L0, psi_m2, Rp, Lp, Lm, Rm, Sx, Sy);
                external_force_pair<O>(kp, (int64_t)y * nx + c0, rho_old, Fex, Fey);
                collide_v<v2, O>(kp, f_old, rho_old, psi_m1, Sx, Sy, Fex, Fey, fb, ux, uy);
                S *out = static_cast<S *>(kp.dst) + (int64_t)y * kp.pitch + c0;
                // random word of the pair (stochastic rounding of 16-bit storage only)
                const uint32_t hsr = dev && kp.sr ? sr_hash((uint32_t)(((int64_t)y * kp.pitch + c0) >> 1), kp.sr_seed) : 0u;
                if (GEOM && own_old) {
                    // one node of the pair is solid: store the fluid one alone
                    const int e = own_old == 1 ? 1 : 0;
                    const float rr = e ? rho_old.v.y : rho_old.v.x;
                    if (has_ref) kp.ref_dst[(int64_t)y * kp.pitch + c0 + e] = rr;
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const float fv = e ? fb[i].v.y : fb[i].v.x;
                        if constexpr (IsDev<S>::value) {
                            const int wc = i == 0 ? 0 : (i <= 4 ? 1 : 5);
                            const float nw = has_ref ? -kp.cf.scale * __fmul_rn(kp.c2.w[wc].x, rr) : kp.c2.enc[wc].x;
                            const float sv = __fmaf_rn(fv, kp.cf.scale, nw);
                            if (kp.sr) out[i * kp.plane + e] = sr_one<S>(sv, sr_bits(hsr, i), e);
                            else Codec2<S>::put(out + i * kp.plane + e, sv);
                        } else {
                            out[i * kp.plane + e] = fv;
                        }
                    }
                } else if (!dev) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) Pair2<S>::store(out + i * kp.plane, fb[i]);
                } else if (has_ref) {
                    Pair2<float>::store(kp.ref_dst + (int64_t)y * kp.pitch + c0, rho_old);
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        // (f - w_i ref) 2^k as one rounding: f 2^k - (w_i ref) 2^k
                        const v2 nwref = v2{kp.c2.m_scale} * (v2{kp.c2.w[i == 0 ? 0 : (i <= 4 ? 1 : 5)]} * rho_old);
                        const v2 sv = vfma(fb[i], v2{kp.c2.scale}, nwref);
                        if (kp.sr) Pair2<S>::store_sr(out + i * kp.plane, sv, sr_bits(hsr, i));
                        else Pair2<S>::store(out + i * kp.plane, sv);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const v2 sv = vfma(fb[i], v2{kp.c2.scale}, v2{kp.c2.enc[i == 0 ? 0 : (i <= 4 ? 1 : 5)]});
                        if (kp.sr) Pair2<S>::store_sr(out + i * kp.plane, sv, sr_bits(hsr, i));
                        else Pair2<S>::store(out + i * kp.plane, sv);
                    }
                }
            }
        }
        psi_m2 = psi_m1;
        psi_m1 = psi_new;
        rho_old = rho_new;
        own_old = own;
#pragma unroll
        for (int i = 0; i < 9; ++i) f_old[i] = f_new[i];
    }
    if (!ok) atomicOr(kp.err, DERR_TIMEOUT);
    if (!ok && lane == 0)
        for (int s = 0; s < RING; ++s) mbar_arrive(empty + s);
}
#undef LBM_PULL_PAIR

// Grid shape: about CTAS_PER_SM CTAs per SM, each a strip of rows no shorter than ROWS_L2
// rows when both population buffers together take at most L2_STATE_MB, else ROWS_HBM rows
// (shortened, down to ROWS_L2, where that would leave fewer than MIN_CTAS_PER_SM per SM).
#ifndef LBM_FUSED2_CTAS_PER_SM
#define LBM_FUSED2_CTAS_PER_SM 16
#endif
#ifndef LBM_FUSED2_ROWS_L2
#define LBM_FUSED2_ROWS_L2 4
#endif
#ifndef LBM_FUSED2_ROWS_HBM
#define LBM_FUSED2_ROWS_HBM 16
#endif
#ifndef LBM_FUSED2_L2_STATE_MB
#define LBM_FUSED2_L2_STATE_MB 64
#endif
#ifndef LBM_FUSED2_MIN_CTAS_PER_SM
#define LBM_FUSED2_MIN_CTAS_PER_SM 4
#endif

template <class S, int NW, int RING>
struct Fused2 {
    typedef FusedLayout2<S, NW, RING> L;
    template <bool P, class O, int GEOM = 0>
    static cudaError_t launch_one(const KParams &kp, cudaStream_t st)
    {
        cudaError_t e = ensure_smem_attribute(k_fused2<S, NW, RING, P, O, GEOM>, kp.device, (int)L::bytes(true));
        if (e != cudaSuccess) return e;
        const int sms = kp.sm_count > 0 ? kp.sm_count : 148;
        const int strips = (kp.nx + L::TX - 1) / L::TX;
        int nseg = (LBM_FUSED2_CTAS_PER_SM * sms + strips - 1) / strips;
        // segments re-read 3 halo rows; a lattice whose two population buffers fit in L2 reads
        // them from L2, so it may be cut into short segments (more CTAs), a larger one not
        const double state_bytes = 2.0 * 9.0 * (double)kp.plane * sizeof(S);
        int min_rows = state_bytes <= LBM_FUSED2_L2_STATE_MB * 1048576.0 ? LBM_FUSED2_ROWS_L2 : LBM_FUSED2_ROWS_HBM;
        // but not so long that the grid holds fewer than MIN_CTAS_PER_SM CTAs per SM: a
        // mid-size lattice (1024^2 FP32: 5 strips x 64 segments of 16 rows = 2 CTAs per SM) is
        // then latency bound, one CTA walking its rows with nothing to hide the waits
        const int64_t occ_rows = (int64_t)kp.ny * strips / ((int64_t)LBM_FUSED2_MIN_CTAS_PER_SM * sms);
        if (min_rows > occ_rows) min_rows = occ_rows > LBM_FUSED2_ROWS_L2 ? (int)occ_rows : LBM_FUSED2_ROWS_L2;
        const int max_seg = kp.ny / min_rows > 0 ? kp.ny / min_rows : 1;
        if (nseg > max_seg) nseg = max_seg;
        if (nseg < 1) nseg = 1;
        const int seg_rows = (kp.ny + nseg - 1) / nseg;
        nseg = (kp.ny + seg_rows - 1) / seg_rows;
        return launch_dependent(k_fused2<S, NW, RING, P, O, GEOM>, dim3(strips, nseg), dim3(32 * (NW + 1)),
                                L::bytes(kp.per_node_ref != 0), st, kp, seg_rows);
    }
    // Fully periodic lattices with a constant force and one relaxation time get
    // instantiations with those options (and the reference-density mode) fixed at compile
    // time; everything else reads them at run time.
    static cudaError_t launch(const KParams &kp, cudaStream_t st)
    {
        // solid nodes, moving walls or interpolated links: the general-geometry instantiation
        if (kp.q || kp.wall_u) return launch_one<false, RuntimeOpts, 2>(kp, st);
        if (kp.solid) return launch_one<false, RuntimeOpts, 1>(kp, st);
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
