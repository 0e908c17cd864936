// Two-pass step (psi pass + fused collide-and-pull-stream pass) and the per-node
// service kernels (init, moments, diagnostics, state copy), for one storage type S.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr int kRowThreads = 128;

// Reads population k of node (x, y) of kp.src from global memory.
template <class S>
struct GlobalAt {
    const KParams &kp;
    __device__ __forceinline__ typename Codec<S>::R operator()(int k, int x, int y) const { return load_pop<S>(kp, k, x, y); }
    __device__ __forceinline__ typename Codec<S>::R at_k(int k, int64_t kk) const { return load_pop_at<S>(kp, k, kk); }
};

// psi of the neighbour along e_i of (x, y), read from the psi field written by the psi
// pass (walls beyond a non-periodic edge: psi(rho_s); solid nodes hold the psi of their
// virtual density, rho_s or the per-node wall density).
template <class R>
struct FieldPsi {
    const KParams &kp;
    const R *psi;
    int x, y;
    __device__ __forceinline__ R operator()(int i) const
    {
        int xx = x + ex_(i), yy = y + ey_(i);
        if (!wrap_xy(kp, xx, yy)) return cst<R>(kp).psi_s;
        return psi[(int64_t)yy * kp.nx + xx];
    }
};

// FieldPsi from the node's neighbourhood nb: the psi field inside the lattice (solid
// nodes hold psi of their virtual density there), psi(rho_s) beyond a non-periodic edge.
template <class R>
struct AroundPsi {
    const KParams &kp;
    const R *psi;
    const Around &nb;
    __device__ __forceinline__ R operator()(int i) const { return nb.in(i) ? psi[nb.n(i)] : cst<R>(kp).psi_s; }
};

__device__ __forceinline__ bool node_is_solid(const KParams &kp, int64_t node)
{
    return kp.solid != nullptr && kp.solid[node] != 0;
}

// Pass 1: rho(x) = sum_i f_i(x) of the pulled populations, psi(rho) (Sec. 2).
template <class S>
__global__ void __launch_bounds__(kRowThreads) k_psi(KParams kp)
{
    typedef typename Codec<S>::R R;
    grid_dependency_wait();
    allow_dependent_launch();
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= kp.nx) return;
    const int64_t node = (int64_t)y * kp.nx + x;
    R *psi = static_cast<R *>(kp.psi);
    if (node_is_solid(kp, node)) {
        psi[node] = kp.wall_psi ? R(kp.wall_psi[node]) : cst<R>(kp).psi_s;
        return;
    }
    R f[9];
    pull_node_nb<R>(kp, around(kp, x, y), x, y, GlobalAt<S>{kp}, f, (R *)nullptr);
    psi[node] = psi_of<R>(kp, density<R>(f));
}

// Pass 2: pull, force from the psi stencil, collision, store.
template <class S>
__global__ void __launch_bounds__(kRowThreads) k_collide(KParams kp)
{
    typedef typename Codec<S>::R R;
    grid_dependency_wait();
    allow_dependent_launch();
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= kp.nx) return;
    const int64_t node = (int64_t)y * kp.nx + x;
    if (node_is_solid(kp, node)) return;
    const R *psi = static_cast<const R *>(kp.psi);
    R f[9], fb[9], Sx, Sy, Fex, Fey, ux, uy;
    const Around nb = around(kp, x, y);
    pull_node_nb<R>(kp, nb, x, y, GlobalAt<S>{kp}, f, (R *)nullptr);
    const R rho = density<R>(f);
    stencil_S<R>(AroundPsi<R>{kp, psi, nb}, Sx, Sy);
    external_force<R>(kp, node, rho, Fex, Fey);
    collide<R>(kp, f, rho, psi[node], Sx, Sy, Fex, Fey, fb, ux, uy);
    store_node<S>(kp, x, y, fb, rho);
}

// f_bar = M^-1 m_eq(rho, u) at every node (solid nodes too; they are never read).
template <class S>
__global__ void __launch_bounds__(kRowThreads) k_init(KParams kp, const double *rho0, const double *ux0, const double *uy0)
{
    typedef typename Codec<S>::R R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= kp.nx) return;
    const int64_t node = (int64_t)y * kp.nx + x;
    const R rho = R(rho0[node]);
    const R ux = ux0 ? R(ux0[node]) : R(0), uy = uy0 ? R(uy0[node]) : R(0);
    R fb[9];
    equilibrium<R>(rho, ux, uy, fb);
    store_node<S>(kp, x, y, fb, rho);
}

// rho and u = (j + F/2)/rho of the current state, as the step computes them.
template <class S>
__global__ void __launch_bounds__(kRowThreads) k_moments(KParams kp, double *rho_out, double *ux_out, double *uy_out)
{
    typedef typename Codec<S>::R R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= kp.nx) return;
    const int64_t node = (int64_t)y * kp.nx + x;
    double r = kp.wall_rho ? kp.wall_rho[node] : kp.rho_s, u = 0.0, v = 0.0;
    if (!node_is_solid(kp, node)) {
        const R *psi = static_cast<const R *>(kp.psi);
        R f[9], fb[9], Sx, Sy, Fex, Fey, ux, uy;
        pull_node<R>(kp, x, y, GlobalAt<S>{kp}, f, (R *)nullptr);
        const R rho = density<R>(f);
        stencil_S<R>(FieldPsi<R>{kp, psi, x, y}, Sx, Sy);
        external_force<R>(kp, node, rho, Fex, Fey);
        collide<R>(kp, f, rho, psi[node], Sx, Sy, Fex, Fey, fb, ux, uy);
        r = double(rho);
        u = double(ux);
        v = double(uy);
    }
    if (rho_out) rho_out[node] = r;
    if (ux_out) ux_out[node] = u;
    if (uy_out) uy_out[node] = v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

constexpr int kDiagSums = 9;

// Per-thread sum of FP32-arithmetic kernels: compensated (Knuth's TwoSum), so that the
// pair (s, c) carries the sum of the added floats to about 2^-48 relative, and converted
// to FP64 once; FP64 arithmetic kernels sum in FP64 directly.  (GB300 runs FP32 adds at
// many times the FP64 rate.)
template <class R>
struct DiagAcc {
    double s = 0.0;
    __device__ __forceinline__ void add(R x) { s += double(x); }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DiagAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float t = s + x, z = t - s;
        c += (s - (t - z)) + (x - z);
        s = t;
    }
    __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

// FP64 diagnostics (see lbm_get_diagnostics): a grid-stride pass over all nodes, each
// thread accumulating its nodes (DiagAcc), then FP64 warp-shuffle and block sums and one
// FP64 atomic per block and quantity.  max |u| uses the ordering of non-negative doubles'
// bits.
template <class S>
__global__ void __launch_bounds__(kRowThreads) k_diag(KParams kp, double *acc, unsigned long long *umax, int *nan_count)
{
    typedef typename Codec<S>::R R;
    __shared__ double red[kRowThreads / 32][kDiagSums + 1];
    DiagAcc<R> a[kDiagSums];
    R umax_t = R(0);
    const int64_t n = (int64_t)kp.nx * kp.ny;
    const R half_lg = R(0.5 * (kp.rho_l + kp.rho_g));
    int bad = 0;
    for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < n; node += (int64_t)gridDim.x * blockDim.x) {
        if (node_is_solid(kp, node)) continue;
        const int y = (int)(node / kp.nx), x = (int)(node - (int64_t)y * kp.nx);
        const R *psi = static_cast<const R *>(kp.psi);
        R f[9], fb[9], Sx, Sy, Fex, Fey, ux, uy;
        R mom[2] = {R(0), R(0)};
        pull_node<R>(kp, x, y, GlobalAt<S>{kp}, f, mom);
        const R rho = density<R>(f);
        stencil_S<R>(FieldPsi<R>{kp, psi, x, y}, Sx, Sy);
        external_force<R>(kp, node, rho, Fex, Fey);
        collide<R>(kp, f, rho, psi[node], Sx, Sy, Fex, Fey, fb, ux, uy);
        const R G = cst<R>(kp).G;
        a[0].add(rho);
        a[1].add(((f[1] - f[3]) + (f[5] - f[6])) + (f[8] - f[7]));
        a[2].add(((f[2] - f[4]) + (f[5] + f[6])) - (f[7] + f[8]));
        a[3].add(-G * psi[node] * Sx + Fex);
        a[4].add(-G * psi[node] * Sy + Fey);
        a[5].add(mom[0]);
        a[6].add(mom[1]);
        if (rho > half_lg) {
            a[7].add(rho * uy);
            a[8].add(rho);
        }
        const R um = sqrt(ux * ux + uy * uy);
        umax_t = um > umax_t ? um : umax_t;
        if (!isfinite(double(rho)) || !isfinite(double(um))) bad = 1;
    }
    double v[kDiagSums + 1];
#pragma unroll
    for (int k = 0; k < kDiagSums; ++k) v[k] = a[k].value();
    v[kDiagSums] = double(umax_t);
    if (bad) atomicAdd(nan_count, 1);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kDiagSums; ++k) v[k] = warp_sum(v[k]);
    v[kDiagSums] = warp_max(v[kDiagSums]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k <= kDiagSums; ++k) red[wid][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kRowThreads / 32; ++w) {
            for (int k = 0; k < kDiagSums; ++k) red[0][k] += red[w][k];
            red[0][kDiagSums] = fmax(red[0][kDiagSums], red[w][kDiagSums]);
        }
        for (int k = 0; k < kDiagSums; ++k) atomicAdd(acc + k, red[0][k]);
        atomicMax(umax, (unsigned long long)__double_as_longlong(red[0][kDiagSums]));
    }
}

template <class S>
__global__ void __launch_bounds__(kRowThreads) k_get_state(KParams kp, double *out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= kp.nx) return;
    const int64_t n = (int64_t)kp.nx * kp.ny, node = (int64_t)y * kp.nx + x;
#pragma unroll
    for (int i = 0; i < 9; ++i) out[i * n + node] = double(load_pop<S>(kp, i, x, y));
}

template <class S>
__global__ void __launch_bounds__(kRowThreads) k_set_state(KParams kp, const double *in)
{
    typedef typename Codec<S>::R R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= kp.nx) return;
    const int64_t n = (int64_t)kp.nx * kp.ny, node = (int64_t)y * kp.nx + x;
    R fb[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) fb[i] = R(in[i * n + node]);
    // the reference density of a node is the sum of its stored populations
    store_node<S>(kp, x, y, fb, density<R>(fb));
}

inline dim3 row_grid(const KParams &kp) { return dim3((kp.nx + kRowThreads - 1) / kRowThreads, kp.ny); }

template <class S>
struct TwoPass {
    static cudaError_t psi_pass(const KParams &kp, cudaStream_t st)
    {
        return launch_dependent(k_psi<S>, row_grid(kp), dim3(kRowThreads), 0, st, kp);
    }
    static cudaError_t collide_pass(const KParams &kp, cudaStream_t st)
    {
        return launch_dependent(k_collide<S>, row_grid(kp), dim3(kRowThreads), 0, st, kp);
    }
    static cudaError_t init(const KParams &kp, const double *r, const double *u, const double *v, cudaStream_t st)
    {
        k_init<S><<<row_grid(kp), kRowThreads, 0, st>>>(kp, r, u, v);
        return cudaGetLastError();
    }
    static cudaError_t moments(const KParams &kp, double *r, double *u, double *v, cudaStream_t st)
    {
        k_moments<S><<<row_grid(kp), kRowThreads, 0, st>>>(kp, r, u, v);
        return cudaGetLastError();
    }
    static cudaError_t diag(const KParams &kp, double *acc, unsigned long long *umax, int *nanc, cudaStream_t st)
    {
        const int sms = kp.sm_count > 0 ? kp.sm_count : 148;
        const int64_t n = (int64_t)kp.nx * kp.ny;
        int64_t blocks = (n + kRowThreads - 1) / kRowThreads;
        if (blocks > 32 * (int64_t)sms) blocks = 32 * (int64_t)sms;
        k_diag<S><<<(unsigned)blocks, kRowThreads, 0, st>>>(kp, acc, umax, nanc);
        return cudaGetLastError();
    }
    static cudaError_t get_state(const KParams &kp, double *out, cudaStream_t st)
    {
        k_get_state<S><<<row_grid(kp), kRowThreads, 0, st>>>(kp, out);
        return cudaGetLastError();
    }
    static cudaError_t set_state(const KParams &kp, const double *in, cudaStream_t st)
    {
        k_set_state<S><<<row_grid(kp), kRowThreads, 0, st>>>(kp, in);
        return cudaGetLastError();
    }
};

}  // namespace lbm
