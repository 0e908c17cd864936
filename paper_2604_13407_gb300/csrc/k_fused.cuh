// Fused single-pass step, warp-specialised.  A CTA owns a strip of 30 NW columns and
// walks down a segment of rows.  One producer warp stages each lattice row of the nine
// population planes (plus the reference-density plane of per-node FP16/BF16 storage)
// into a shared-memory ring with bulk async copies (the TMA engine, cp.async.bulk); each
// ring slot has a "full" mbarrier (completed by the copies' byte count) and an "empty"
// mbarrier (one arrival per consumer warp).  Each of the NW consumer warps owns 32
// consecutive columns: its lanes pull the populations of their node of row r, form rho
// and psi, and keep the pulled populations in registers; one row later, lanes 1..30
// collide their node of row r - 1 with the psi of the 3 x 3 neighbourhood taken from the
// last three psi rows in registers and from neighbouring lanes by warp shuffles (lanes 0
// and 31 supply the halo columns).  There is no block-wide barrier in the loop: warps
// advance independently, limited only by the ring.  Halo psi is recomputed rather than
// written and re-read, so HBM sees each population read once and written once (72 B per
// update in FP32, 36 B in FP16/BF16).
//
// The kernel calls the same pull, density, pseudopotential, stencil and collision
// functions as the two-pass step, so both give bit-identical populations.  Supported
// geometry: periodic directions and half-way walls just outside non-periodic edges (no
// solid mask, no moving or interpolated walls); nx a multiple of the 16-byte column
// group and at least twice the strip width.  Every mbarrier wait is bounded; a wait that
// runs out sets DERR_TIMEOUT in the device error word and the warp leaves its loop; the
// producer drains the copies in flight (again bounded) before the CTA exits.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// ---------------------------------------------------------------- PTX ------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

constexpr uint32_t kWaitLimit = 1u << 22;  // try_wait polls before a wait is declared lost

// Bounded wait for phase `parity` of an mbarrier; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (uint32_t it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

template <class S>
struct FusedGeom {
    static constexpr int HX = (16 / (int)sizeof(S)) < 2 ? 2 : 16 / (int)sizeof(S);  // halo columns, one 16 B group
};

template <class S, int NW, int RING>
struct FusedLayout {
    typedef typename Codec<S>::R R;
    static constexpr int TX = 30 * NW;                          // output columns per strip
    static constexpr int HX = FusedGeom<S>::HX;
    static constexpr int W = TX + 2 * HX;                      // staged columns per row
    static constexpr int POP_ROW = 9 * W * (int)sizeof(S);     // bytes of one staged row (9 planes)
    static constexpr int REF_ROW = W * 4;                      // bytes of one staged reference row
    static size_t bytes(bool ref) { return (size_t)RING * POP_ROW + (ref ? (size_t)RING * REF_ROW : 0) + 2 * RING * 8 + 16; }
};

// Explicit shared-memory loads (32-bit shared-window addresses).
template <class S> struct Lds;
template <> struct Lds<double> {
    static __device__ __forceinline__ double ld(uint32_t a)
    {
        double v;
        asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
        return v;
    }
};
template <> struct Lds<float> {
    static __device__ __forceinline__ float ld(uint32_t a)
    {
        float v;
        asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
        return v;
    }
};
template <> struct Lds<__half> {
    static __device__ __forceinline__ __half ld(uint32_t a)
    {
        unsigned short v;
        asm volatile("ld.shared.b16 %0, [%1];" : "=h"(v) : "r"(a));
        return __ushort_as_half(v);
    }
};
template <> struct Lds<__nv_bfloat16> {
    static __device__ __forceinline__ __nv_bfloat16 ld(uint32_t a)
    {
        unsigned short v;
        asm volatile("ld.shared.b16 %0, [%1];" : "=h"(v) : "r"(a));
        return __ushort_as_bfloat16(v);
    }
};

// Reads staged populations around one node.  The shared-window addresses of the three
// staged rows (y - 1, y, y + 1) at the node's column are formed once per row, so every
// read is one shared load at a compile-time offset from one of three registers.
template <class S, int NW, int RING>
struct RingAt {
    typedef typename Codec<S>::R R;
    typedef FusedLayout<S, NW, RING> L;
    const KParams &kp;
    uint32_t row[3];  // staged rows y-1, y, y+1 at column cx (bytes, shared window)
    uint32_t ref[3];  // same for the reference-density rows
    int cx, cy;
    // (x, y): unwrapped coordinates within one node of (cx, cy)
    __device__ __forceinline__ R operator()(int k, int x, int y) const
    {
        const int dy = y - cy + 1, dx = x - cx;
        const S v = Lds<S>::ld(row[dy] + (uint32_t)((k * L::W + dx) * (int)sizeof(S)));
        R wref = R(0);
        if (IsDev<S>::value)
            wref = w_<R>(k) * (kp.per_node_ref ? R(Lds<float>::ld(ref[dy] + (uint32_t)(dx * 4))) : cst<R>(kp).rho_ref);
        return Codec<S>::dec(v, wref, cst<R>(kp).inv_scale);
    }
};

// Pull of node (cx, cy) (unwrapped column, row) from the ring: plain copies, or half-way
// bounce-back when the source lies beyond a non-periodic edge.
template <bool PERIODIC, class R, class At>
__device__ __forceinline__ void pull_ring(const KParams &kp, int cx, int cy, const At &at, R (&f)[9])
{
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int xs = cx - ex_(i), ys = cy - ey_(i);
        bool wall = false;
        if (!PERIODIC)
            wall = (!kp.periodic_x && (xs < 0 || xs >= kp.nx)) || (!kp.periodic_y && (ys < 0 || ys >= kp.ny));
        if (i == 0 || !wall) f[i] = at(i, xs, ys);
        else f[i] = at(opp_(i), cx, cy) + R(0);  // same arithmetic as bounce() with q = 1/2, u_w = 0
    }
}

template <class S, int NW, int RING, bool PERIODIC, class O>
__global__ void __launch_bounds__(32 * (NW + 1)) k_fused(KParams kp, int seg_rows)
{
    typedef typename Codec<S>::R R;
    typedef FusedLayout<S, NW, RING> L;
    constexpr int TX = L::TX, HX = L::HX, W = L::W;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *pops = smem;
    float *refs = kp.per_node_ref ? reinterpret_cast<float *>(smem + (size_t)RING * L::POP_ROW) : nullptr;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)RING * L::POP_ROW +
                                                  (kp.per_node_ref ? (size_t)RING * L::REF_ROW : 0));
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
            int sx[3], dx[3], cnt[3], nseg = 0;
            const int lo = x_lo, hi = x0 + TX + HX;
            const int m0 = lo < 0 ? 0 : lo, m1 = hi > nx ? nx : hi;
            sx[nseg] = m0, dx[nseg] = m0 - lo, cnt[nseg] = m1 - m0, ++nseg;
            if (lo < 0 && kp.periodic_x) sx[nseg] = nx + lo, dx[nseg] = 0, cnt[nseg] = -lo, ++nseg;
            if (hi > nx && kp.periodic_x) sx[nseg] = 0, dx[nseg] = nx - lo, cnt[nseg] = hi - nx, ++nseg;
            uint32_t cols = 0;
            for (int q = 0; q < nseg; ++q) cols += cnt[q];
            fence_proxy_async();
            mbar_expect_tx(bar, cols * (9u * (uint32_t)sizeof(S) + (refs ? 4u : 0u)));
            unsigned char *prow = pops + (size_t)slot * L::POP_ROW;
            for (int i = 0; i < 9; ++i) {
                const S *src = A + i * kp.plane + (int64_t)gy * kp.pitch;
                S *dst = reinterpret_cast<S *>(prow) + i * W;
                for (int q = 0; q < nseg; ++q) bulk_g2s(dst + dx[q], src + sx[q], cnt[q] * (uint32_t)sizeof(S), bar);
            }
            if (refs) {
                const float *src = kp.ref_src + (int64_t)gy * kp.pitch;
                float *dst = refs + slot * W;
                for (int q = 0; q < nseg; ++q) bulk_g2s(dst + dx[q], src + sx[q], cnt[q] * 4u, bar);
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
    const int col = x0 + 30 * warp - 1 + lane;  // unwrapped column of this lane's node
    const int scol = col - x_lo;                 // its staged column
    const uint32_t pops_s = smem_u32(pops);
    const uint32_t refs_s = refs ? smem_u32(refs) : 0u;
    const bool col_out = !PERIODIC && !kp.periodic_x && (col < 0 || col >= nx);
    const bool collides = lane >= 1 && lane <= 30 && col < nx;
    const R psi_s = cst<R>(kp).psi_s;
    R f_old[9], rho_old = R(0), psi_m2 = psi_s, psi_m1 = psi_s;
#pragma unroll
    for (int i = 0; i < 9; ++i) f_old[i] = R(0);
    // every lane polls; the outcome is made warp-uniform so that the shuffles below never
    // run in a partially exited warp
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
        // pull, rho, psi of node (col, rp)
        const bool row_out = !PERIODIC && !kp.periodic_y && (rp < 0 || rp >= ny);
        R f_new[9], rho_new = R(0), psi_new = psi_s;
#pragma unroll
        for (int i = 0; i < 9; ++i) f_new[i] = R(0);
        if (!col_out && !row_out) {
            RingAt<S, NW, RING> at{kp, {0u, 0u, 0u}, {0u, 0u, 0u}, col, rp};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const uint32_t slot = (uint32_t)((rp - 1 + d - first) & (RING - 1));
                at.row[d] = pops_s + slot * (uint32_t)L::POP_ROW + (uint32_t)(scol * (int)sizeof(S));
                at.ref[d] = refs_s + slot * (uint32_t)L::REF_ROW + (uint32_t)(scol * 4);
            }
            pull_ring<PERIODIC, R>(kp, col, rp, at, f_new);
            rho_new = density<R>(f_new);
            psi_new = psi_of<R>(kp, rho_new);
        }
        __syncwarp();
        // row rp - 1 is not needed any more by this warp
        if (lane == 0 && rp - 1 >= first) mbar_arrive(empty + ((rp - 1 - first) & (RING - 1)));
        // psi of the neighbour columns from the adjacent lanes
        const R a_m2 = __shfl_up_sync(0xffffffffu, psi_m2, 1), b_m2 = __shfl_down_sync(0xffffffffu, psi_m2, 1);
        const R a_m1 = __shfl_up_sync(0xffffffffu, psi_m1, 1), b_m1 = __shfl_down_sync(0xffffffffu, psi_m1, 1);
        const R a_p0 = __shfl_up_sync(0xffffffffu, psi_new, 1), b_p0 = __shfl_down_sync(0xffffffffu, psi_new, 1);
        const int y = rp - 1;
        if (collides && y >= yb) {
            // neighbour psi along e_i: rows y-1 (m2), y (m1), y+1 (new); columns -1 (a), +1 (b)
            auto ps = [&](int i) -> R {
                const int dxn = ex_(i), dyn = ey_(i);
                if (dyn < 0) return dxn < 0 ? a_m2 : (dxn > 0 ? b_m2 : psi_m2);
                if (dyn > 0) return dxn < 0 ? a_p0 : (dxn > 0 ? b_p0 : psi_new);
                return dxn < 0 ? a_m1 : b_m1;
            };
            R fb[9], Sx, Sy, Fex, Fey, ux, uy;
            stencil_S<R>(ps, Sx, Sy);
            external_force<R, O>(kp, (int64_t)y * nx + col, rho_old, Fex, Fey);
            collide<R, O>(kp, f_old, rho_old, psi_m1, Sx, Sy, Fex, Fey, fb, ux, uy);
            // store: one row pointer, planes at a fixed stride
            S *out = static_cast<S *>(kp.dst) + (int64_t)y * kp.pitch + col;
            R ref = cst<R>(kp).rho_ref;
            if (IsDev<S>::value && kp.per_node_ref) {
                ref = rho_old;
                kp.ref_dst[(int64_t)y * kp.pitch + col] = float(rho_old);
            }
            const int64_t kn = (int64_t)y * kp.pitch + col;
            const uint32_t h = IsDev<S>::value && kp.sr ? sr_hash((uint32_t)(kn >> 1), kp.sr_seed) : 0u;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                out[0] = enc_pop<S>(kp, fb[i], w_<R>(i) * ref, cst<R>(kp).scale, kn, i, h);
                out += kp.plane;
            }
        }
        psi_m2 = psi_m1;
        psi_m1 = psi_new;
        rho_old = rho_new;
#pragma unroll
        for (int i = 0; i < 9; ++i) f_old[i] = f_new[i];
    }
    if (!ok) atomicOr(kp.err, DERR_TIMEOUT);
    // release every slot this warp still holds so the producer's bounded waits end early
    if (!ok && lane == 0)
        for (int s = 0; s < RING; ++s) mbar_arrive(empty + s);
}

template <class S, int NW, int RING>
struct Fused {
    typedef FusedLayout<S, NW, RING> L;
    template <bool P, class O>
    static cudaError_t launch_one(const KParams &kp, cudaStream_t st)
    {
        cudaError_t e = ensure_smem_attribute(k_fused<S, NW, RING, P, O>, kp.device, (int)L::bytes(true));
        if (e != cudaSuccess) return e;
        const int sms = kp.sm_count > 0 ? kp.sm_count : 148;
        const int strips = (kp.nx + L::TX - 1) / L::TX;
        int nseg = (16 * sms + strips - 1) / strips;
        // a CTA walks its segment row by row, so short segments cut the latency of small
        // lattices; each segment re-reads 3 halo rows, which come from L2 while the two
        // population buffers fit in it
        const double state_bytes = 2.0 * 9.0 * (double)kp.plane * sizeof(S);
        const int min_rows = state_bytes <= 64.0 * 1024 * 1024 ? 4 : 16;
        const int max_seg = kp.ny / min_rows > 0 ? kp.ny / min_rows : 1;
        if (nseg > max_seg) nseg = max_seg;
        if (nseg < 1) nseg = 1;
        const int seg_rows = (kp.ny + nseg - 1) / nseg;
        nseg = (kp.ny + seg_rows - 1) / seg_rows;
        return launch_dependent(k_fused<S, NW, RING, P, O>, dim3(strips, nseg), dim3(32 * (NW + 1)),
                                L::bytes(kp.per_node_ref != 0), st, kp, seg_rows);
    }
    // Fully periodic lattices with a constant force and one relaxation time get
    // instantiations with those options fixed at compile time; everything else reads them
    // at run time.
    static cudaError_t launch(const KParams &kp, cudaStream_t st)
    {
        if (kp.periodic_x && kp.periodic_y) {
            if (kp.force_mode == 0 && !kp.var_tau)
                return kp.improved ? launch_one<true, Opts<1, 0, 0>>(kp, st) : launch_one<true, Opts<0, 0, 0>>(kp, st);
            return launch_one<true, RuntimeOpts>(kp, st);
        }
        return launch_one<false, RuntimeOpts>(kp, st);
    }
};

}  // namespace lbm
