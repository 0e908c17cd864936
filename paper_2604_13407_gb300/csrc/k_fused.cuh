// Fused single-pass step: one CTA owns a strip of TX columns and walks down a segment of
// rows.  Each lattice row of the nine population planes (plus the reference-density plane
// of per-node FP16/BF16 storage) is brought into a shared-memory ring by bulk async
// copies (the TMA engine, cp.async.bulk) that complete on one mbarrier per ring slot,
// several rows ahead of use.  For every row the CTA computes rho and psi on the strip
// plus a one-node halo from the staged populations, then pulls, collides and stores the
// strip row with coalesced stores.  Halo psi is recomputed instead of being written and
// re-read, so HBM sees each population read once and written once (72 B per update in
// FP32, 36 B in FP16/BF16).
//
// The kernel calls the same pull, density, pseudopotential, stencil and collision
// functions as the two-pass step, so both give bit-identical populations.  Supported
// geometry: periodic directions and half-way walls just outside non-periodic edges (no
// solid mask, no moving or interpolated walls); nx a multiple of the 16-byte column
// group and at least 2 TX.  Every mbarrier wait is bounded; a wait that runs out sets
// DERR_TIMEOUT in the device error word and the CTA returns after a bounded drain.
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

template <class S, int TX, int RING>
struct FusedLayout {
    typedef typename Codec<S>::R R;
    static constexpr int HX = FusedGeom<S>::HX;
    static constexpr int W = TX + 2 * HX;                      // staged columns per row
    static constexpr int POP_ROW = 9 * W * (int)sizeof(S);     // bytes of one staged row (9 planes)
    static constexpr int REF_ROW = W * 4;                      // bytes of one staged reference row
    static constexpr int PSI_ROW = ((TX + 2) * (int)sizeof(R) + 15) / 16 * 16;
    static size_t bytes(bool ref)
    {
        return (size_t)RING * POP_ROW + (ref ? (size_t)RING * REF_ROW : 0) + 4 * (size_t)PSI_ROW + RING * 8 + 16;
    }
};

// Reads population k of node (x, y) from the staged ring.  (x, y) are wrapped domain
// coordinates within one node of the node being processed (cx, cy).
template <class S, int TX, int RING>
struct RingAt {
    typedef typename Codec<S>::R R;
    typedef FusedLayout<S, TX, RING> L;
    const KParams &kp;
    const unsigned char *pops;  // ring base
    const float *refs;          // reference ring base (per-node ref) or null
    int x_lo;                   // global column of staged column 0 (unwrapped)
    int first;                  // first staged row
    int cx, cy;                 // unwrapped coordinates of the node being processed
    __device__ __forceinline__ R operator()(int k, int x, int y) const
    {
        int dx = x - cx, dy = y - cy;
        if (dx > 1) dx -= kp.nx;
        if (dx < -1) dx += kp.nx;
        if (dy > 1) dy -= kp.ny;
        if (dy < -1) dy += kp.ny;
        const int col = cx + dx - x_lo;
        const int slot = (cy + dy - first) & (RING - 1);
        const S *row = reinterpret_cast<const S *>(pops + (size_t)slot * L::POP_ROW) + k * L::W;
        R wref = R(0);
        if (IsDev<S>::value) wref = w_<R>(k) * (kp.per_node_ref ? R(refs[slot * L::W + col]) : R(kp.rho_ref));
        return Codec<S>::dec(row[col], wref, R(kp.inv_scale));
    }
};

// Pull of node (cx, cy) (unwrapped column, row) from the ring: plain copies, or half-way
// bounce-back when the source lies beyond a non-periodic edge.
template <class R, class At>
__device__ __forceinline__ void pull_ring(const KParams &kp, int cx, int cy, const At &at, R (&f)[9])
{
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int xs = cx - ex_(i), ys = cy - ey_(i);
        const bool wall = (!kp.periodic_x && (xs < 0 || xs >= kp.nx)) || (!kp.periodic_y && (ys < 0 || ys >= kp.ny));
        if (i == 0 || !wall) f[i] = at(i, xs, ys);
        else f[i] = at(opp_(i), cx, cy) + R(0);  // same arithmetic as bounce() with q = 1/2, u_w = 0
    }
}

template <class S, int TX, int RING>
__global__ void __launch_bounds__(TX) k_fused(KParams kp, int seg_rows)
{
    typedef typename Codec<S>::R R;
    typedef FusedLayout<S, TX, RING> L;
    constexpr int HX = L::HX, W = L::W;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *pops = smem;
    float *refs = kp.per_node_ref ? reinterpret_cast<float *>(smem + (size_t)RING * L::POP_ROW) : nullptr;
    unsigned char *psi_base = smem + (size_t)RING * L::POP_ROW + (kp.per_node_ref ? (size_t)RING * L::REF_ROW : 0);
    uint64_t *bars = reinterpret_cast<uint64_t *>(psi_base + 4 * L::PSI_ROW);
    int *abort_flag = reinterpret_cast<int *>(bars + RING);

    const int t = threadIdx.x;
    const int nx = kp.nx, ny = kp.ny;
    const int x0 = blockIdx.x * TX;
    const int yb = blockIdx.y * seg_rows;
    const int ye = min(yb + seg_rows, ny);
    const int first = yb - 2, last = ye + 1;  // staged rows
    const int x_lo = x0 - HX;
    const S *A = static_cast<const S *>(kp.src);

    if (t == 0) {
        for (int s = 0; s < RING; ++s) mbar_init(bars + s, 1);
        *abort_flag = 0;
        fence_mbar_init();
        fence_proxy_async();
    }
    __syncthreads();

    // Stage row r (all planes) into its ring slot; rows beyond a non-periodic edge are
    // not loaded, their slot barrier just completes.
    auto issue = [&](int r) {
        const int slot = (r - first) & (RING - 1);
        uint64_t *bar = bars + slot;
        int gy = r;
        if (gy < 0 || gy >= ny) {
            if (!kp.periodic_y) {
                mbar_arrive(bar);
                return;
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
        for (int s = 0; s < nseg; ++s) cols += cnt[s];
        const uint32_t bytes = cols * (9u * (uint32_t)sizeof(S) + (refs ? 4u : 0u));
        mbar_expect_tx(bar, bytes);
        unsigned char *prow = pops + (size_t)slot * L::POP_ROW;
        for (int i = 0; i < 9; ++i) {
            const S *src = A + i * kp.plane + (int64_t)gy * kp.pitch;
            S *dst = reinterpret_cast<S *>(prow) + i * W;
            for (int s = 0; s < nseg; ++s) bulk_g2s(dst + dx[s], src + sx[s], cnt[s] * (uint32_t)sizeof(S), bar);
        }
        if (refs) {
            const float *src = kp.ref_src + (int64_t)gy * kp.pitch;
            float *dst = refs + slot * W;
            for (int s = 0; s < nseg; ++s) bulk_g2s(dst + dx[s], src + sx[s], cnt[s] * 4u, bar);
        }
    };
    auto parity_of = [&](int r) -> uint32_t { return (uint32_t)(((r - first) / RING) & 1); };
    auto wait_row = [&](int r) -> bool { return mbar_wait_bounded(bars + ((r - first) & (RING - 1)), parity_of(r)); };

    if (t == 0)
        for (int r = first; r <= last && r < first + RING; ++r) issue(r);

    const R psi_s = R(kp.psi_s);
    bool ok = true;
    for (int rp = yb - 1; rp <= ye && ok; ++rp) {
        // rows rp - 1 .. rp + 1 must be staged (earlier ones were waited for already)
        bool good = true;
        if (rp == yb - 1) good = wait_row(rp - 1) && wait_row(rp);
        good = good && wait_row(rp + 1);
        if (!good) *abort_flag = 1;

        // psi of row rp over columns x0 - 1 .. x0 + TX
        R *psi_row = reinterpret_cast<R *>(psi_base + ((rp - first) & 3) * L::PSI_ROW);
        for (int c = t; c < TX + 2; c += TX) {
            const int gx = x0 - 1 + c;
            const bool outside = (!kp.periodic_x && (gx < 0 || gx >= nx)) || (!kp.periodic_y && (rp < 0 || rp >= ny));
            R v = psi_s;
            if (!outside && good) {
                R f[9];
                pull_ring<R>(kp, gx, rp, RingAt<S, TX, RING>{kp, pops, refs, x_lo, first, gx, rp}, f);
                v = psi_of<R>(kp, density<R>(f));
            }
            psi_row[c] = v;
        }
        __syncthreads();
        if (*abort_flag) {
            ok = false;
            break;
        }
        // collide row y = rp - 1
        const int y = rp - 1;
        const int x = x0 + t;
        if (y >= yb && x < nx) {
            const R *p0 = reinterpret_cast<const R *>(psi_base + ((y - 1 - first) & 3) * L::PSI_ROW);
            const R *p1 = reinterpret_cast<const R *>(psi_base + ((y - first) & 3) * L::PSI_ROW);
            const R *p2 = reinterpret_cast<const R *>(psi_base + ((y + 1 - first) & 3) * L::PSI_ROW);
            const int c = t + 1;
            auto ps = [&](int i) -> R {
                const int dxn = ex_(i), dyn = ey_(i);
                const R *row = dyn < 0 ? p0 : (dyn > 0 ? p2 : p1);
                return row[c + dxn];
            };
            R f[9], fb[9], Sx, Sy, Fex, Fey, ux, uy;
            pull_ring<R>(kp, x, y, RingAt<S, TX, RING>{kp, pops, refs, x_lo, first, x, y}, f);
            const R rho = density<R>(f);
            stencil_S<R>(ps, Sx, Sy);
            external_force<R>(kp, (int64_t)y * nx + x, rho, Fex, Fey);
            collide<R>(kp, f, rho, p1[c], Sx, Sy, Fex, Fey, fb, ux, uy);
            store_node<S>(kp, x, y, fb, rho);
        }
        __syncthreads();
        // the slot of row rp - 2 is free: stage row rp - 2 + RING into it
        if (t == 0) {
            const int rn = rp - 2 + RING;
            if (rp - 2 >= first && rn <= last) {
                fence_proxy_async();
                issue(rn);
            }
        }
    }
    if (!ok) {
        // drain: wait (bounded) for every row still in flight before the CTA exits
        if (t == 0) {
            atomicOr(kp.err, DERR_TIMEOUT);
            for (int r = last - RING + 1; r <= last; ++r)
                if (r >= first) wait_row(r);
        }
        __syncthreads();
    }
}

template <class S, int TX, int RING>
struct Fused {
    typedef FusedLayout<S, TX, RING> L;
    static cudaError_t launch(const KParams &kp, cudaStream_t st)
    {
        static bool configured = false;
        const size_t smem = L::bytes(true);
        if (!configured) {
            cudaError_t e = cudaFuncSetAttribute(k_fused<S, TX, RING>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            configured = true;
        }
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int strips = (kp.nx + TX - 1) / TX;
        int nseg = (16 * sms + strips - 1) / strips;
        const int max_seg = kp.ny / 16 > 0 ? kp.ny / 16 : 1;
        if (nseg > max_seg) nseg = max_seg;
        if (nseg < 1) nseg = 1;
        const int seg_rows = (kp.ny + nseg - 1) / nseg;
        nseg = (kp.ny + seg_rows - 1) / seg_rows;
        k_fused<S, TX, RING><<<dim3(strips, nseg), TX, L::bytes(kp.per_node_ref != 0), st>>>(kp, seg_rows);
        return cudaGetLastError();
    }
};

}  // namespace lbm
