// Host side of the C ABI declared in include/lbm.h: parameter validation, device
// buffers, kernel dispatch, checkpoint/resume and the adjoint driver.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_adjoint.h"
#include "lbm_internal.h"

using namespace lbm;

struct lbm_ctx {
    lbm_params p{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int sm_count = 0;
    size_t elem = 0;        // bytes per stored population
    size_t real = 0;        // bytes of the arithmetic type (psi field)
    int64_t pitch = 0;      // elements per row of a population plane
    int64_t plane = 0;      // elements per plane
    void *pops[2] = {nullptr, nullptr};
    float *refp[2] = {nullptr, nullptr};
    int cur = 0;
    void *psi = nullptr;
    uint8_t *solid = nullptr;
    double *wall_u = nullptr, *q = nullptr, *fext = nullptr;
    double *wall_rho = nullptr, *wall_psi = nullptr;  // per solid node virtual density, its psi
    float2 *link = nullptr;             // wall-link records of the one-pass kernel (KParams::link)
    double *dacc = nullptr;             // diagnostics accumulators (9 doubles, 1 u64, 1 int)
    double *scratch = nullptr;          // host<->device staging for FP64 field copies
    size_t scratch_bytes = 0;
    int *derr = nullptr;
    bool initialised = false;
    bool fused_ok = false;
    int64_t steps = 0;
    int64_t n_fluid = 0;                // nodes that are not solid
    Launchers L{};
    KParams kp{};
    std::string err;
    AdjointState *adj = nullptr;
};

static thread_local std::string g_create_error;

static lbm_status fail(lbm_ctx *c, lbm_status s, const std::string &msg)
{
    if (c) c->err = msg;
    else g_create_error = msg;
    return s;
}

static lbm_status cuda_fail(lbm_ctx *c, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, m);
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

// ------------------------------------------------------------- params ------

static double host_p_eos(const lbm_params &p, double rho)
{
    if (p.eos == LBM_EOS_VDW) return p.K_eos * (rho * p.R * p.T / (1.0 - p.b * rho) - p.a * rho * rho);
    double eta = p.b * rho / 4.0;
    double num = 1.0 + eta + eta * eta - eta * eta * eta;
    double om = 1.0 - eta;
    return p.K_eos * (rho * p.R * p.T * num / (om * om * om) - p.a * rho * rho);
}

static double host_psi(const lbm_params &p, double rho) { return std::sqrt(2.0 * (host_p_eos(p, rho) - rho / 3.0) / p.G); }

extern "C" lbm_status lbm_params_default(lbm_params *p)
{
    if (!p) return LBM_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->struct_size = (int32_t)sizeof(lbm_params);
    p->nx = 4;
    p->ny = 128;
    p->periodic_x = 1;
    p->periodic_y = 0;
    p->precision = LBM_F64;
    p->scheme = LBM_SCHEME_IMPROVED;
    p->eos = LBM_EOS_CS;
    p->force_mode = LBM_FORCE_CONST;
    p->kernel = LBM_KERNEL_AUTO;
    p->storage_rounding = 1;
    p->a = 1.0;
    p->b = 4.0;
    p->R = 1.0;
    p->T = 0.7 * 0.3773 * 1.0 / (4.0 * 1.0);
    p->K_eos = 1.0;
    p->G = -1.0;
    p->k1 = p->k2 = -1.895 / 16.0;
    p->tau_l = p->tau_g = 0.8;
    p->rho_l = 0.3581443962580134;   // Maxwell densities of this EOS at 0.7 T_c
    p->rho_g = 0.009291723294794338;
    p->Lambda = 1.0 / 12.0;
    p->rho_s = p->rho_g;
    p->rho_ref = p->rho_g;
    p->rho_max = 0.0;
    return LBM_OK;
}

static lbm_status validate(lbm_ctx *c, const lbm_params &p)
{
    if (p.struct_size != (int32_t)sizeof(lbm_params)) return fail(c, LBM_EINVAL, "lbm_params.struct_size does not match this library");
    if (p.nx < 1 || p.ny < 1) return fail(c, LBM_EINVAL, "nx and ny must be >= 1");
    if ((int64_t)p.nx * p.ny > (int64_t)1 << 31) return fail(c, LBM_EINVAL, "lattice larger than 2^31 nodes");
    if (p.ny > 65535) return fail(c, LBM_EINVAL, "ny must be <= 65535 (one grid row of blocks per lattice row)");
    if (p.precision < LBM_F64 || p.precision > LBM_BF16DEV) return fail(c, LBM_EINVAL, "unknown precision");
    if (p.scheme != LBM_SCHEME_ORIGINAL && p.scheme != LBM_SCHEME_IMPROVED) return fail(c, LBM_EINVAL, "unknown scheme");
    if (p.eos != LBM_EOS_VDW && p.eos != LBM_EOS_CS) return fail(c, LBM_EINVAL, "unknown eos");
    if (p.force_mode < LBM_FORCE_CONST || p.force_mode > LBM_FORCE_FIELD) return fail(c, LBM_EINVAL, "unknown force_mode");
    if (p.kernel < LBM_KERNEL_AUTO || p.kernel > LBM_KERNEL_FUSED) return fail(c, LBM_EINVAL, "unknown kernel");
    if (!(p.tau_l > 0.5) || !(p.tau_g > 0.5)) return fail(c, LBM_EINVAL, "tau must be > 1/2");
    if (!(p.G < 0.0)) return fail(c, LBM_EINVAL, "G must be < 0");
    if (!(p.Lambda > 0.0)) return fail(c, LBM_EINVAL, "Lambda must be > 0");
    if (p.tau_l != p.tau_g && !(p.rho_l > p.rho_g)) return fail(c, LBM_EINVAL, "rho_l must exceed rho_g when tau_l != tau_g");
    if (p.storage_scale_log2 < -30 || p.storage_scale_log2 > 30) return fail(c, LBM_EINVAL, "storage_scale_log2 out of range");
    if (p.storage_rounding != 0 && p.storage_rounding != 1) return fail(c, LBM_EINVAL, "storage_rounding must be 0 or 1");
    if (p.diag_every < 0) return fail(c, LBM_EINVAL, "diag_every must be >= 0");
    if (p.precision == LBM_F16DEV && (p.storage_scale_log2 < -15 || p.storage_scale_log2 > 24))
        return fail(c, LBM_EINVAL, "FP16 storage needs storage_scale_log2 in [-15, 24] (2^-k must be an FP16 value)");
    double rmax = p.rho_max > 0 ? p.rho_max : 1.25 * std::fmax(std::fmax(p.rho_l, p.rho_g), p.rho_s);
    if (!(rmax > 0)) return fail(c, LBM_EINVAL, "rho_max must be > 0");
    for (int k = 1; k <= 4096; ++k) {
        double rho = rmax * k / 4096.0;
        double d = host_p_eos(p, rho) - rho / 3.0;
        if (!(d < 0.0)) {
            char buf[160];
            std::snprintf(buf, sizeof buf, "p_EOS - rho/3 >= 0 at rho = %.6g: psi is not real on (0, rho_max]", rho);
            return fail(c, LBM_EINVAL, buf);
        }
    }
    if (!(host_psi(p, p.rho_s) > 0)) return fail(c, LBM_EINVAL, "psi(rho_s) is not real");
    return LBM_OK;
}

// Derived kernel constants of the current parameters (Secs. 2-3).
static void fill_constants(lbm_ctx *c)
{
    const lbm_params &p = c->p;
    KParams &k = c->kp;
    k.nx = p.nx;
    k.ny = p.ny;
    k.device = c->device;
    k.sm_count = c->sm_count;
    k.pitch = c->pitch;
    k.plane = c->plane;
    k.periodic_x = p.periodic_x != 0;
    k.periodic_y = p.periodic_y != 0;
    k.improved = p.scheme == LBM_SCHEME_IMPROVED;
    k.eos = p.eos;
    k.force_mode = p.force_mode;
    k.var_tau = p.tau_l != p.tau_g;
    k.per_node_ref = (p.precision >= LBM_F16DEV) && p.per_node_ref;
    k.sr = (p.precision >= LBM_F16DEV) && p.storage_rounding;
    k.eos_a = p.a;
    k.eos_b = p.b;
    k.eos_RT = p.R * p.T;
    k.eos_K = p.K_eos;
    k.two_over_G = 2.0 / p.G;
    k.eos_R = p.R;
    k.eos_T = p.T;
    k.k1 = p.k1;
    k.k2 = p.k2;
    k.G = p.G;
    const double eps = -8.0 * (p.k1 + p.k2);
    k.kq1 = 3.0 * (p.k1 + 2.0 * p.k2) * p.G;
    k.kq7 = p.k1 * p.G;
    k.c1G = (30.0 * eps - 15.0) / 16.0 * p.G;
    k.c2G = 3.0 * eps / 8.0 * p.G;
    k.q2fac = (p.scheme == LBM_SCHEME_ORIGINAL || p.q2_original) ? -1.0 : -0.5;
    const double tau = p.tau_l;
    k.sp = 1.0 / tau;
    k.sq = 1.0 / (0.5 + p.Lambda / (tau - 0.5));
    k.nu_l = (p.tau_l - 0.5) / 3.0;
    k.nu_g = (p.tau_g - 0.5) / 3.0;
    k.rho_l = p.rho_l;
    k.rho_g = p.rho_g;
    k.Lambda = p.Lambda;
    k.Fx = p.Fx;
    k.Fy = p.Fy;
    k.psi_s = host_psi(p, p.rho_s);
    k.rho_s = p.rho_s;
    k.rho_ref = p.rho_ref;
    k.scale = std::ldexp(1.0, p.storage_scale_log2);
    k.inv_scale = std::ldexp(1.0, -p.storage_scale_log2);
    // the same constants in each kernel arithmetic type
#define LBM_FILL(f) k.cd.f = k.f; k.cf.f = (float)k.f;
    LBM_FILL(eos_a) LBM_FILL(eos_b) LBM_FILL(eos_RT) LBM_FILL(eos_R) LBM_FILL(eos_K) LBM_FILL(two_over_G) LBM_FILL(G)
    LBM_FILL(kq1) LBM_FILL(kq7) LBM_FILL(c1G) LBM_FILL(c2G) LBM_FILL(q2fac) LBM_FILL(sp) LBM_FILL(sq)
    LBM_FILL(nu_l) LBM_FILL(nu_g) LBM_FILL(rho_l) LBM_FILL(rho_g) LBM_FILL(Lambda) LBM_FILL(Fx) LBM_FILL(Fy)
    LBM_FILL(psi_s) LBM_FILL(rho_s) LBM_FILL(rho_ref) LBM_FILL(scale) LBM_FILL(inv_scale)
#undef LBM_FILL
    k.cd.hsp = 1.0 - 0.5 * k.sp;
    k.cd.hsq = 1.0 - 0.5 * k.sq;
    k.cf.hsp = 1.0f - 0.5f * (float)k.sp;
    k.cf.hsq = 1.0f - 0.5f * (float)k.sq;
    {
        auto P = [](float v) { return make_float2(v, v); };
        PairConsts &q = k.c2;
        const Consts<float> &f = k.cf;
        q.one = P(1.f), q.m_one = P(-1.f), q.half = P(0.5f), q.m_half = P(-0.5f), q.two = P(2.f), q.m_two = P(-2.f);
        q.three = P(3.f), q.m_three = P(-3.f), q.four = P(4.f), q.m_four = P(-4.f), q.six = P(6.f), q.m_six = P(-6.f);
        q.third = P(1.0f / 3.0f), q.m_third = P(-1.0f / 3.0f), q.twelfth = P(1.0f / 12.0f), q.ninth = P(1.0f / 9.0f);
        q.w36 = P(1.0f / 36.0f), q.sixth = P(1.0f / 6.0f), q.quarter = P(0.25f);
        q.m_G = P(-f.G), q.kq1 = P(f.kq1), q.q2fac = P(f.q2fac), q.kq7 = P(f.kq7), q.c1G = P(f.c1G), q.m_c2G = P(-f.c2G);
        q.sp = P(f.sp), q.sq = P(f.sq), q.hsp = P(f.hsp), q.hsq = P(f.hsq), q.six_hsp = P(6.f * f.hsp);
        q.m_six_hsp = P(-6.f * f.hsp), q.m_hsq = P(-f.hsq);
        q.Fx = P(f.Fx), q.Fy = P(f.Fy), q.rho_g = P(f.rho_g), q.inv_drho = P(1.0f / (f.rho_l - f.rho_g));
        q.dnu = P(f.nu_l - f.nu_g), q.nu_g = P(f.nu_g), q.Lambda = P(f.Lambda);
        q.m_b = P(-f.eos_b), q.b4 = P(f.eos_b * 0.25f), q.K = P(f.eos_K), q.RT = P(f.eos_RT), q.a = P(f.eos_a);
        q.two_over_G = P(f.two_over_G);
        q.inv_scale = P(f.inv_scale), q.scale = P(f.scale), q.m_scale = P(-f.scale), q.psi_s = P(f.psi_s);
        q.rho_ref = P(f.rho_ref);
        // 2^-k as FP16 (normal for k <= 14, subnormal down to 2^-24) or BF16 bits
        const int kk = p.storage_scale_log2;
        if (p.precision == LBM_BF16DEV) k.inv_scale_bits = (unsigned short)((127 - kk) << 7);
        else k.inv_scale_bits = kk <= 14 ? (unsigned short)((15 - kk) << 10) : (unsigned short)(1u << (24 - kk));
        for (int i = 0; i < 9; ++i) {
            const float w = i == 0 ? 4.0f / 9.0f : (i <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f);
            const float wr = w * f.rho_ref;  // rounded like the kernels' w_i rho_ref
            q.w[i] = P(w);
            q.dec[i] = P(wr);
            q.enc[i] = P(-(wr * f.scale));
        }
    }
    k.psi = c->psi;
    k.solid = c->solid;
    k.wall_u = c->wall_u;
    k.q = c->q;
    k.fext = c->fext;
    k.wall_rho = c->wall_rho;
    k.wall_psi = c->wall_psi;
    k.link = c->link;
    k.err = c->derr;
}

static void bind_buffers(lbm_ctx *c, int src)
{
    c->kp.src = c->pops[src];
    c->kp.dst = c->pops[src ^ 1];
    c->kp.ref_src = c->refp[src];
    c->kp.ref_dst = c->refp[src ^ 1];
}

static bool fused_possible(const lbm_ctx *c)
{
    if (!c->L.fused_pass) return false;
    const lbm_params &p = c->p;
    if ((c->solid || c->q || c->wall_u) && !c->L.fused_geometry) return false;
    if (c->L.fused_align <= 0 || p.nx % c->L.fused_align != 0) return false;
    // the wrapped halo segment of the last strip must fit inside the lattice
    if (p.nx < c->L.fused_tile_x + 16 || p.ny < 4) return false;
    return true;
}

// LBM_KERNEL_AUTO: the one-pass kernel where it was measured faster than the two-pass one
// (FP32 on a GB300 unless stated; the two are close at each threshold).  On small lattices a
// CTA's serial walk down its rows dominates the one-pass kernel's time and the two-pass
// kernels, one thread per node, hide latency better: periodic 256^2 7.1 us against 8.8,
// 512^2 12.4 against 10.1; a 256-wide channel with x walls 23.5 against 29.5 (two strips,
// the second 16 columns wide); 512 x 4096 84 against 57.  Solid bands: 256^2 below, 512^2
// 17.8 against 19.2 in FP32 but 25.1 against 22.5 in FP16, 1024^2 55 against 41 (before the
// two-pass kernels shared one neighbourhood computation per node), 2048^2 251 against 100.
// Interpolated and moving walls, whose per-link work sits on the one-pass kernel's serial
// path: annulus 1024^2 44 against 58, 2048^2 207 against 195 (FP16 258 against 211).
static bool auto_prefers_fused(const lbm_ctx *c)
{
    const int64_t n = (int64_t)c->p.nx * c->p.ny;
    if (c->q || c->wall_u) return n >= (int64_t(1) << 22);
    if (c->solid) return n >= (int64_t(1) << (c->p.precision == LBM_F32 ? 19 : 18));
    return (n >= (int64_t(1) << 18) && c->p.nx >= 512) || n >= (int64_t(1) << 21);
}

static void choose_kernel(lbm_ctx *c)
{
    const int want = c->p.kernel;
    c->fused_ok = (want != LBM_KERNEL_TWO_PASS) && fused_possible(c) &&
                  (want == LBM_KERNEL_FUSED || c->p.precision == LBM_F64 || auto_prefers_fused(c));
}

// ------------------------------------------------------------- lifetime ----

static void free_all(lbm_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    void *bufs[] = {c->pops[0], c->pops[1], c->refp[0], c->refp[1], c->psi, c->solid,
                    c->wall_u, c->q, c->fext, c->wall_rho, c->wall_psi, c->link, c->dacc, c->scratch, c->derr};
    for (void *b : bufs)
        if (b) cudaFree(b);
    adjoint_free(c->adj);
    c->adj = nullptr;
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

extern "C" lbm_status lbm_create(const lbm_params *p, void *cuda_stream, lbm_ctx **out)
{
    if (!p || !out) return fail(nullptr, LBM_EINVAL, "null argument");
    *out = nullptr;
    lbm_status s = validate(nullptr, *p);
    if (s != LBM_OK) return s;
    lbm_ctx *c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
    c->p = *p;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        delete c;
        return fail(nullptr, LBM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    }
    e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        delete c;
        return fail(nullptr, LBM_ECUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
    }
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return fail(nullptr, LBM_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
        }
        c->own_stream = true;
    }
    switch (p->precision) {
    case LBM_F64: c->L = launchers_f64(); c->elem = 8; c->real = 8; break;
    case LBM_F32: c->L = launchers_f32(); c->elem = 4; c->real = 4; break;
    case LBM_F16DEV: c->L = launchers_f16(); c->elem = 2; c->real = 4; break;
    default: c->L = launchers_bf16(); c->elem = 2; c->real = 4; break;
    }
    const int64_t per_line = 128 / (int64_t)c->elem;
    c->pitch = ((int64_t)p->nx + per_line - 1) / per_line * per_line;
    c->plane = c->pitch * p->ny;
    const int64_t n = (int64_t)p->nx * p->ny;
    const size_t pop_bytes = (size_t)9 * c->plane * c->elem;
    auto alloc = [&](void **ptr, size_t bytes) -> bool {
        cudaError_t ee = cudaMalloc(ptr, bytes);
        if (ee != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return true;
    };
    bool ok = alloc(&c->pops[0], pop_bytes) && alloc(&c->pops[1], pop_bytes) &&
              alloc(&c->psi, (size_t)n * c->real) && alloc((void **)&c->dacc, 16 * sizeof(double)) &&
              alloc((void **)&c->derr, sizeof(int));
    if (ok && p->precision >= LBM_F16DEV && p->per_node_ref)
        ok = alloc((void **)&c->refp[0], (size_t)c->plane * 4) && alloc((void **)&c->refp[1], (size_t)c->plane * 4);
    if (!ok) {
        free_all(c);
        delete c;
        return fail(nullptr, LBM_ENOMEM, "device allocation failed");
    }
    cudaMemsetAsync(c->pops[0], 0, pop_bytes, c->stream);
    cudaMemsetAsync(c->pops[1], 0, pop_bytes, c->stream);
    cudaMemsetAsync(c->derr, 0, sizeof(int), c->stream);
    c->n_fluid = n;
    fill_constants(c);
    choose_kernel(c);
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        free_all(c);
        delete c;
        return fail(nullptr, LBM_ECUDA, std::string("create: ") + cudaGetErrorString(e));
    }
    *out = c;
    return LBM_OK;
}

extern "C" lbm_status lbm_destroy(lbm_ctx *c)
{
    if (!c) return LBM_OK;
    free_all(c);
    delete c;
    return LBM_OK;
}

// scratch device buffer of at least `bytes`
static lbm_status need_scratch(lbm_ctx *c, size_t bytes)
{
    if (c->scratch_bytes >= bytes) return LBM_OK;
    if (c->scratch) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->scratch);
        c->scratch = nullptr;
        c->scratch_bytes = 0;
    }
    CK(cudaMalloc((void **)&c->scratch, bytes), "cudaMalloc(scratch)");
    c->scratch_bytes = bytes;
    return LBM_OK;
}

template <class T>
static lbm_status upload(lbm_ctx *c, T **dst, const T *src, size_t count, const char *what)
{
    if (*dst) {
        cudaStreamSynchronize(c->stream);
        cudaFree(*dst);
        *dst = nullptr;
    }
    if (!src) return LBM_OK;
    CK(cudaMalloc((void **)dst, count * sizeof(T)), what);
    CK(cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice, c->stream), what);
    return LBM_OK;
}

// Wall-link records of the one-pass kernel (KParams::link), built on the host from the
// geometry as given: for each fluid node x and pulled population i whose source x - e_i is a
// wall (a solid node or beyond a non-periodic edge), the link fraction q of the outgoing
// population o = opp(i) (1/2 without link fractions, and 1/2 where q < 1/2 but the second
// node x + e_i is a wall too -- the same fallback as the two-pass step's bounce-back) and
// the moving-wall coefficient 2 w_o (e_i . u_w) 3 of the wall node (0 beyond an edge).
static lbm_status build_link_records(lbm_ctx *c, const uint8_t *solid, const double *wall_u, const double *q)
{
    static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    static const double W[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    if (c->link) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->link);
        c->link = nullptr;
    }
    if (!q && !wall_u) return LBM_OK;
    const int nx = c->p.nx, ny = c->p.ny;
    const int64_t n = (int64_t)nx * ny, pitch = c->pitch, plane = c->plane;
    auto wall_at = [&](int x, int y, int64_t *node) -> bool {
        if (x < 0 || x >= nx) {
            if (!c->p.periodic_x) return true;
            x = x < 0 ? x + nx : x - nx;
        }
        if (y < 0 || y >= ny) {
            if (!c->p.periodic_y) return true;
            y = y < 0 ? y + ny : y - ny;
        }
        *node = (int64_t)y * nx + x;
        return solid && solid[*node] != 0;
    };
    std::vector<float2> h((size_t)(8 * plane), make_float2(0.5f, 0.0f));
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const int64_t node = (int64_t)y * nx + x, k = (int64_t)y * pitch + x;
            if (solid && solid[node]) continue;
            for (int i = 1; i < 9; ++i) {
                int64_t wn = -1;
                if (!wall_at(x - EX[i], y - EY[i], &wn)) continue;
                const int o = OPP[i];
                double qq = q ? q[(int64_t)(o - 1) * n + node] : 0.5;
                int64_t bn;
                if (qq < 0.5 && wall_at(x + EX[i], y + EY[i], &bn)) qq = 0.5;
                double cw = 0.0;
                if (wall_u && wn >= 0) cw = 2.0 * W[o] * (EX[i] * wall_u[wn] + EY[i] * wall_u[n + wn]) * 3.0;
                h[(size_t)((i - 1) * plane + k)] = make_float2((float)qq, (float)cw);
            }
        }
    CK(cudaMalloc((void **)&c->link, h.size() * sizeof(float2)), "link records");
    CK(cudaMemcpyAsync(c->link, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice, c->stream),
       "link records");
    CK(cudaStreamSynchronize(c->stream), "link records");
    return LBM_OK;
}

extern "C" lbm_status lbm_set_geometry(lbm_ctx *c, const uint8_t *solid, const double *wall_u, const double *q,
                                       const double *force_field)
{
    if (!c) return LBM_EINVAL;
    const size_t n = (size_t)c->p.nx * c->p.ny;
    if (q) {
        for (size_t k = 0; k < 8 * n; ++k)
            if (!(q[k] > 0.0 && q[k] <= 1.0)) return fail(c, LBM_EINVAL, "q must lie in (0, 1]");
    }
    lbm_status s;
    if ((s = upload(c, &c->solid, solid, n, "solid")) != LBM_OK) return s;
    c->n_fluid = (int64_t)n;
    if (solid)
        for (size_t k = 0; k < n; ++k) c->n_fluid -= solid[k] != 0;
    if ((s = upload(c, &c->wall_u, wall_u, 2 * n, "wall_u")) != LBM_OK) return s;
    if ((s = upload(c, &c->q, q, 8 * n, "q")) != LBM_OK) return s;
    if ((s = upload(c, &c->fext, force_field, 2 * n, "force_field")) != LBM_OK) return s;
    if (c->p.precision != LBM_F64 && (s = build_link_records(c, solid, wall_u, q)) != LBM_OK) return s;
    CK(cudaStreamSynchronize(c->stream), "set_geometry");
    fill_constants(c);
    choose_kernel(c);
    return LBM_OK;
}

extern "C" lbm_status lbm_set_wall_density(lbm_ctx *c, const double *wall_rho)
{
    if (!c) return LBM_EINVAL;
    const size_t n = (size_t)c->p.nx * c->p.ny;
    std::vector<double> psi;
    if (wall_rho) {
        psi.resize(n);
        for (size_t k = 0; k < n; ++k) {
            // the same host evaluation as psi(rho_s), so a uniform field equals the scalar
            psi[k] = host_psi(c->p, wall_rho[k]);
            if (!(wall_rho[k] > 0.0) || !(psi[k] > 0.0) || !std::isfinite(psi[k]))
                return fail(c, LBM_EINVAL, "psi of a wall density is not real and positive");
        }
    }
    lbm_status s;
    if ((s = upload(c, &c->wall_rho, wall_rho, n, "wall_rho")) != LBM_OK) return s;
    if ((s = upload(c, &c->wall_psi, wall_rho ? psi.data() : (const double *)nullptr, n, "wall_psi")) != LBM_OK)
        return s;
    CK(cudaStreamSynchronize(c->stream), "set_wall_density");
    fill_constants(c);
    choose_kernel(c);
    return LBM_OK;
}

// Bring `count` doubles from host or device into a device pointer (scratch slot `slot`).
static lbm_status device_input(lbm_ctx *c, const double *src, int on_device, size_t count, size_t slot,
                               const double **out)
{
    if (!src) {
        *out = nullptr;
        return LBM_OK;
    }
    if (on_device) {
        *out = src;
        return LBM_OK;
    }
    double *d = c->scratch + slot * count;
    CK(cudaMemcpyAsync(d, src, count * sizeof(double), cudaMemcpyHostToDevice, c->stream), "H2D");
    *out = d;
    return LBM_OK;
}

extern "C" lbm_status lbm_init_fields(lbm_ctx *c, const double *rho, const double *ux, const double *uy,
                                      int on_device)
{
    if (!c || !rho) return c ? fail(c, LBM_EINVAL, "rho is required") : LBM_EINVAL;
    const size_t n = (size_t)c->p.nx * c->p.ny;
    lbm_status s;
    if (!on_device && (s = need_scratch(c, 3 * n * sizeof(double))) != LBM_OK) return s;
    const double *dr, *du, *dv;
    if ((s = device_input(c, rho, on_device, n, 0, &dr)) != LBM_OK) return s;
    if ((s = device_input(c, ux, on_device, n, 1, &du)) != LBM_OK) return s;
    if ((s = device_input(c, uy, on_device, n, 2, &dv)) != LBM_OK) return s;
    c->cur = 0;
    bind_buffers(c, 1);  // init writes kp.dst = pops[0]
    CK(c->L.init(c->kp, dr, du, dv, c->stream), "init kernel");
    if (!on_device) CK(cudaStreamSynchronize(c->stream), "init");
    c->steps = 0;
    c->initialised = true;
    return LBM_OK;
}

// Seed of the stochastic-rounding bits of step t (MurmurHash3's 32-bit finaliser of the
// step count's two halves; any well-mixed function of t would do).
static uint32_t sr_seed_of(int64_t t)
{
    uint32_t h = (uint32_t)t * 0x9E3779B1u ^ (uint32_t)((uint64_t)t >> 32) * 0x85EBCA77u;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

static lbm_status run_steps(lbm_ctx *c, int64_t nsteps)
{
    for (int64_t t = 0; t < nsteps; ++t) {
        bind_buffers(c, c->cur);
        c->kp.sr_seed = sr_seed_of(c->steps);
        if (c->fused_ok) {
            CK(c->L.fused_pass(c->kp, c->stream), "fused step kernel");
        } else {
            CK(c->L.psi_pass(c->kp, c->stream), "psi kernel");
            CK(c->L.collide_pass(c->kp, c->stream), "collide kernel");
        }
        c->cur ^= 1;
        c->steps += 1;
    }
    return LBM_OK;
}

// Wait for the context stream and read the device error word (set by a bounded device-side
// wait that ran out, or a failed bounds check, in any step launched so far).  Every call
// that synchronises anyway reads it: lbm_sync, the host-side getters and lbm_save_state.
static lbm_status sync_and_check(lbm_ctx *c, const char *what)
{
    int h = 0;
    CK(cudaMemcpyAsync(&h, c->derr, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "error word");
    CK(cudaStreamSynchronize(c->stream), what);
    if (h & DERR_TIMEOUT) return fail(c, LBM_ETIMEOUT, "a device-side wait ran out of iterations");
    if (h & DERR_BOUNDS) return fail(c, LBM_EBOUNDS, "a device-side bounds check failed");
    return LBM_OK;
}

extern "C" lbm_status lbm_step(lbm_ctx *c, int64_t nsteps)
{
    if (!c) return LBM_EINVAL;
    if (!c->initialised) return fail(c, LBM_ESTATE, "fields not initialised");
    if (nsteps < 0) return fail(c, LBM_EINVAL, "nsteps < 0");
    const int64_t D = c->p.diag_every;
    if (D <= 0) return run_steps(c, nsteps);
    // launch up to the next multiple of D, then wait and check the state there
    while (nsteps > 0) {
        const int64_t n = std::min<int64_t>(nsteps, D - c->steps % D);
        lbm_status s = run_steps(c, n);
        if (s != LBM_OK) return s;
        nsteps -= n;
        if (c->steps % D == 0) {
            double d[LBM_NDIAG];
            if ((s = lbm_get_diagnostics(c, d)) != LBM_OK) return s;
        }
    }
    return LBM_OK;
}

// psi field of the current state (needed by the moments and diagnostics kernels)
static lbm_status psi_of_current(lbm_ctx *c)
{
    bind_buffers(c, c->cur);
    CK(c->L.psi_pass(c->kp, c->stream), "psi kernel");
    return LBM_OK;
}

extern "C" lbm_status lbm_get_moments(lbm_ctx *c, double *rho, double *ux, double *uy, int on_device)
{
    if (!c) return LBM_EINVAL;
    if (!c->initialised) return fail(c, LBM_ESTATE, "fields not initialised");
    const size_t n = (size_t)c->p.nx * c->p.ny;
    lbm_status s;
    if ((s = psi_of_current(c)) != LBM_OK) return s;
    if (on_device) {
        CK(c->L.moments(c->kp, rho, ux, uy, c->stream), "moments kernel");
        return LBM_OK;
    }
    if ((s = need_scratch(c, 3 * n * sizeof(double))) != LBM_OK) return s;
    double *d = c->scratch;
    CK(c->L.moments(c->kp, rho ? d : nullptr, ux ? d + n : nullptr, uy ? d + 2 * n : nullptr, c->stream), "moments kernel");
    if (rho) CK(cudaMemcpyAsync(rho, d, n * 8, cudaMemcpyDeviceToHost, c->stream), "D2H");
    if (ux) CK(cudaMemcpyAsync(ux, d + n, n * 8, cudaMemcpyDeviceToHost, c->stream), "D2H");
    if (uy) CK(cudaMemcpyAsync(uy, d + 2 * n, n * 8, cudaMemcpyDeviceToHost, c->stream), "D2H");
    return sync_and_check(c, "get_moments");
}

extern "C" lbm_status lbm_get_diagnostics(lbm_ctx *c, double out[LBM_NDIAG])
{
    if (!c || !out) return LBM_EINVAL;
    if (!c->initialised) return fail(c, LBM_ESTATE, "fields not initialised");
    lbm_status s;
    if ((s = psi_of_current(c)) != LBM_OK) return s;
    CK(cudaMemsetAsync(c->dacc, 0, 16 * sizeof(double), c->stream), "memset");
    unsigned long long *umax = reinterpret_cast<unsigned long long *>(c->dacc + 9);
    int *nanc = reinterpret_cast<int *>(c->dacc + 10);
    CK(c->L.diag(c->kp, c->dacc, umax, nanc, c->stream), "diagnostics kernel");
    double h[16];
    CK(cudaMemcpyAsync(h, c->dacc, sizeof h, cudaMemcpyDeviceToHost, c->stream), "D2H");
    if ((s = sync_and_check(c, "diagnostics")) != LBM_OK) return s;
    for (int k = 0; k < 9; ++k) out[k] = h[k];
    unsigned long long ub;
    std::memcpy(&ub, &h[9], 8);
    double um;
    std::memcpy(&um, &ub, 8);
    out[9] = um;
    int nanc_h;
    std::memcpy(&nanc_h, &h[10], sizeof(int));
    if (nanc_h > 0 || !std::isfinite(out[0])) return fail(c, LBM_ENAN, "non-finite density or velocity");
    return LBM_OK;
}

extern "C" lbm_status lbm_get_state(lbm_ctx *c, double *pops, int on_device)
{
    if (!c || !pops) return LBM_EINVAL;
    const size_t n = (size_t)c->p.nx * c->p.ny;
    bind_buffers(c, c->cur);
    if (on_device) {
        CK(c->L.get_state(c->kp, pops, c->stream), "get_state kernel");
        return LBM_OK;
    }
    lbm_status s;
    if ((s = need_scratch(c, 9 * n * sizeof(double))) != LBM_OK) return s;
    CK(c->L.get_state(c->kp, c->scratch, c->stream), "get_state kernel");
    CK(cudaMemcpyAsync(pops, c->scratch, 9 * n * 8, cudaMemcpyDeviceToHost, c->stream), "D2H");
    return sync_and_check(c, "get_state");
}

extern "C" lbm_status lbm_set_state(lbm_ctx *c, const double *pops, int on_device)
{
    if (!c || !pops) return LBM_EINVAL;
    const size_t n = (size_t)c->p.nx * c->p.ny;
    const double *src = pops;
    if (!on_device) {
        lbm_status s;
        if ((s = need_scratch(c, 9 * n * sizeof(double))) != LBM_OK) return s;
        CK(cudaMemcpyAsync(c->scratch, pops, 9 * n * 8, cudaMemcpyHostToDevice, c->stream), "H2D");
        src = c->scratch;
    }
    c->cur = 0;
    bind_buffers(c, 1);
    CK(c->L.set_state(c->kp, src, c->stream), "set_state kernel");
    if (!on_device) CK(cudaStreamSynchronize(c->stream), "set_state");
    c->steps = 0;
    c->initialised = true;
    return LBM_OK;
}

// --------------------------------------------------- checkpoint / resume ---

struct SnapHeader {
    char magic[8];
    int32_t precision, per_node_ref, nx, ny;
    int64_t pitch, steps;
};

extern "C" lbm_status lbm_save_state(lbm_ctx *c, void *host_buf, size_t *nbytes)
{
    if (!c || !nbytes) return LBM_EINVAL;
    const size_t pop_bytes = (size_t)9 * c->plane * c->elem;
    const size_t ref_bytes = c->refp[0] ? (size_t)c->plane * 4 : 0;
    const size_t need = sizeof(SnapHeader) + pop_bytes + ref_bytes;
    if (!host_buf) {
        *nbytes = need;
        return LBM_OK;
    }
    if (*nbytes < need) return fail(c, LBM_EINVAL, "buffer too small");
    SnapHeader h{};
    std::memcpy(h.magic, "LBMSNAP1", 8);
    h.precision = c->p.precision;
    h.per_node_ref = ref_bytes != 0;
    h.nx = c->p.nx;
    h.ny = c->p.ny;
    h.pitch = c->pitch;
    h.steps = c->steps;
    std::memcpy(host_buf, &h, sizeof h);
    char *dst = static_cast<char *>(host_buf) + sizeof h;
    CK(cudaMemcpyAsync(dst, c->pops[c->cur], pop_bytes, cudaMemcpyDeviceToHost, c->stream), "save");
    if (ref_bytes) CK(cudaMemcpyAsync(dst + pop_bytes, c->refp[c->cur], ref_bytes, cudaMemcpyDeviceToHost, c->stream), "save");
    lbm_status s = sync_and_check(c, "save");
    if (s != LBM_OK) return s;
    *nbytes = need;
    return LBM_OK;
}

extern "C" lbm_status lbm_load_state(lbm_ctx *c, const void *host_buf, size_t nbytes)
{
    if (!c || !host_buf) return LBM_EINVAL;
    const size_t pop_bytes = (size_t)9 * c->plane * c->elem;
    const size_t ref_bytes = c->refp[0] ? (size_t)c->plane * 4 : 0;
    SnapHeader h;
    if (nbytes < sizeof h) return fail(c, LBM_EINVAL, "snapshot too small");
    std::memcpy(&h, host_buf, sizeof h);
    if (std::memcmp(h.magic, "LBMSNAP1", 8) != 0 || h.precision != c->p.precision || h.nx != c->p.nx ||
        h.ny != c->p.ny || h.pitch != c->pitch || (h.per_node_ref != 0) != (ref_bytes != 0) ||
        nbytes != sizeof h + pop_bytes + ref_bytes)
        return fail(c, LBM_EINVAL, "snapshot does not match this context");
    const char *src = static_cast<const char *>(host_buf) + sizeof h;
    c->cur = 0;
    CK(cudaMemcpyAsync(c->pops[0], src, pop_bytes, cudaMemcpyHostToDevice, c->stream), "load");
    if (ref_bytes) CK(cudaMemcpyAsync(c->refp[0], src + pop_bytes, ref_bytes, cudaMemcpyHostToDevice, c->stream), "load");
    CK(cudaStreamSynchronize(c->stream), "load");
    c->steps = h.steps;
    c->initialised = true;
    return LBM_OK;
}

extern "C" lbm_status lbm_set_param(lbm_ctx *c, int32_t which, double value)
{
    if (!c) return LBM_EINVAL;
    lbm_params np = c->p;
    switch (which) {
    case LBM_PARAM_FX: np.Fx = value; break;
    case LBM_PARAM_FY: np.Fy = value; break;
    case LBM_PARAM_G: np.G = value; break;
    case LBM_PARAM_T: np.T = value; break;
    default: return fail(c, LBM_EINVAL, "unknown parameter id");
    }
    lbm_status s = validate(c, np);
    if (s != LBM_OK) return s;
    c->p = np;
    fill_constants(c);
    return LBM_OK;
}

extern "C" lbm_status lbm_adjoint_step(lbm_ctx *c, int64_t nsteps, int32_t checkpoint_every, int32_t objective,
                                       double *J, double grad[4], double *lambda0)
{
    if (!c || !J) return LBM_EINVAL;
    if (!c->initialised) return fail(c, LBM_ESTATE, "fields not initialised");
    std::string msg;
    lbm_status s = adjoint_run(c, nsteps, checkpoint_every, objective, J, grad, lambda0, msg);
    if (s != LBM_OK) return fail(c, s, msg);
    return LBM_OK;
}

extern "C" lbm_status lbm_sync(lbm_ctx *c)
{
    if (!c) return LBM_EINVAL;
    return sync_and_check(c, "sync");
}

extern "C" int64_t lbm_step_count(const lbm_ctx *c) { return c ? c->steps : -1; }

extern "C" int32_t lbm_kernel_in_use(const lbm_ctx *c)
{
    if (!c) return -1;
    return c->fused_ok ? LBM_KERNEL_FUSED : LBM_KERNEL_TWO_PASS;
}

extern "C" const char *lbm_last_error(const lbm_ctx *c)
{
    if (!c) return g_create_error.c_str();
    return c->err.c_str();
}

// ---------------------------------------------- accessors for the adjoint ---

namespace lbm {
ContextView view_of(lbm_ctx *c)
{
    ContextView v;
    v.p = &c->p;
    v.kp = &c->kp;
    v.stream = c->stream;
    v.pops = c->pops;
    v.refp = c->refp;
    v.cur = &c->cur;
    v.steps = &c->steps;
    v.elem = c->elem;
    v.plane = c->plane;
    v.adj = &c->adj;
    v.run_steps = [](lbm_ctx *cc, int64_t n) { return run_steps(cc, n); };
    v.sr_seed = [](int64_t t) { return sr_seed_of(t); };
    v.bind = [](lbm_ctx *cc, int src) { bind_buffers(cc, src); };
    v.psi_pass = c->L.psi_pass;
    v.collide_pass = c->L.collide_pass;
    v.fused_pass = (c->fused_ok && c->p.precision != LBM_F64) ? c->L.fused_pass : nullptr;
    v.L = &c->L;
    v.check_error = [](lbm_ctx *cc, std::string &m) {
        lbm_status s = sync_and_check(cc, "adjoint");
        if (s != LBM_OK) m = cc->err;
        return s;
    };
    v.n_fluid = c->n_fluid;
    v.ctx = c;
    return v;
}
}  // namespace lbm

// ------------------------------------------- helpers for lbm_noalloc.cu ----

namespace lbm {
// Kernel parameters for a lattice described by *p whose population planes have the given
// row pitch (elements); no geometry arrays.  Validates *p like lbm_create.
lbm_status kparams_for(const lbm_params *p, int64_t pitch, KParams *out)
{
    lbm_status s = validate(nullptr, *p);
    if (s != LBM_OK) return s;
    lbm_ctx tmp;
    tmp.p = *p;
    if (cudaGetDevice(&tmp.device) != cudaSuccess ||
        cudaDeviceGetAttribute(&tmp.sm_count, cudaDevAttrMultiProcessorCount, tmp.device) != cudaSuccess)
        return fail(nullptr, LBM_ECUDA, "cannot query the current device");
    tmp.pitch = pitch;
    tmp.plane = pitch * p->ny;
    fill_constants(&tmp);
    *out = tmp.kp;
    return LBM_OK;
}

cudaError_t ensure_smem_attribute_ptr(const void *kernel, int device, int bytes)
{
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto &d : done)
        if (d.first == kernel && d.second == device) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.emplace_back(kernel, device);
    return e;
}

// psi of the EOS of *p at rho (the host evaluation create uses), for lbm_lbana.cu.
double eos_psi(const lbm_params &p, double rho) { return host_psi(p, rho); }

// Record a message for lbm_last_error(NULL).
lbm_status set_global_error(lbm_status s, const std::string &msg) { return fail(nullptr, s, msg); }
}  // namespace lbm
