// Checkpointed adjoint of n steps (host driver of the transposed-step kernels).
//
// J = (1/n) sum_{t=1..n} <W, A_t>, with A_t the stored populations after step t and W
// the weights of the objective.  Reverse-mode differentiation of the time loop:
//
//   lambda_n = W/n,  lambda_t = W/n + Step'(A_t)^T lambda_{t+1}  (t = n-1 .. 1),
//   lambda_0 = Step'(A_0)^T lambda_1,  dJ/dtheta = sum_t (dStep(A_t)/dtheta)^T lambda_{t+1}.
//
// Forward sweep: the context advances n steps with its normal kernels, storing A_t every
// K steps (a checkpoint); <W, A_n> is summed in FP64 there, <W, A_t> of the other states by
// the transposed passes (objective alone: every state in the forward sweep).  Backward sweep, one segment of K
// steps at a time from the last: the states of the segment are recomputed from its
// checkpoint with the step kernels the context uses, each leaving the psi field of the
// state it reads in a buffer of its own (the two-pass step's psi pass writes it anyway; the
// one-pass step writes it on request), then the transposed step runs from the last state
// of the segment to the first.  The recompute of a segment runs on a second stream, overlapping the
// transposed steps of the segment after it, so segment states and psi fields come in two
// sets.  Device memory: ceil(n/K) checkpoints, 2 (K - 1) segment states, 2 K psi fields
// and the adjoint planes; it is kept for the next call with the same sizes.
//
// 16-bit storage: a stored state is its nine planes of deviations plus, with a per-node
// reference density, that plane; the recompute repeats the forward steps' stochastic
// rounding (same step seeds).  The transposed step runs in FP32 on the decoded states and
// differentiates the FP32 step through the storage, whose rounding it takes as the
// identity: the gradient of the unrounded step along the trajectory the 16-bit run takes.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "lbm_adjoint.h"

namespace lbm {

struct AdjointState {
    void *base = nullptr;
    size_t bytes = 0;
    cudaStream_t side = nullptr;  // recomputes the next segment while the transposed steps run
    cudaEvent_t fork = nullptr, recomputed[2] = {nullptr, nullptr}, reversed[2] = {nullptr, nullptr};
};

void adjoint_free(AdjointState *a)
{
    if (!a) return;
    if (a->side) cudaStreamSynchronize(a->side);
    if (a->base) cudaFree(a->base);
    cudaEvent_t evs[] = {a->fork, a->recomputed[0], a->recomputed[1], a->reversed[0], a->reversed[1]};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    if (a->side) cudaStreamDestroy(a->side);
    delete a;
}

namespace {

struct Carver {
    char *p;
    size_t used = 0;
    void *take(size_t bytes)
    {
        void *r = p ? p + used : nullptr;
        used += (bytes + 255) / 256 * 256;
        return r;
    }
};

struct Layout {
    std::vector<void *> ckpt, seg[2], psi[2];  // two sets of segment states and psi fields
    void *g[2], *c[2], *dS, *dpsi, *rho;
    double *part;  // per-block partial sums of the transposed passes [blocks][kAdjSlots]
    double *red;   // their column sums (kAdjSlots)
    double *acc;
};

size_t carve(Carver &cv, Layout &L, int64_t nseg, int64_t K, size_t state_bytes, size_t plane_r, size_t psi_bytes,
             size_t part_bytes)
{
    L.ckpt.resize(nseg);
    for (auto &b : L.ckpt) b = cv.take(state_bytes);
    for (int q = 0; q < 2; ++q) {
        L.seg[q].resize(std::max<int64_t>(K - 1, 1));
        L.psi[q].resize(K);
        for (auto &b : L.seg[q]) b = cv.take(state_bytes);
        for (auto &b : L.psi[q]) b = cv.take(psi_bytes);
    }
    for (int s = 0; s < 2; ++s) {
        L.g[s] = cv.take(9 * plane_r);
        L.c[s] = cv.take(plane_r);
    }
    L.dS = cv.take(2 * plane_r);
    L.dpsi = cv.take(plane_r);
    L.rho = cv.take(plane_r);
    L.part = static_cast<double *>(cv.take(part_bytes));
    L.red = static_cast<double *>(cv.take(kAdjSlots * sizeof(double)));
    L.acc = static_cast<double *>(cv.take(8 * sizeof(double)));
    return cv.used;
}

}  // namespace

#define ACK(call, what)                                                      \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) {                                             \
            msg = std::string(what) + ": " + cudaGetErrorString(e_);         \
            return e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA; \
        }                                                                    \
    } while (0)

lbm_status adjoint_run(lbm_ctx *ctx, int64_t nsteps, int32_t K, int32_t objective, double *J, double *grad,
                       double *lambda0, std::string &msg)
{
    ContextView v = view_of(ctx);
    const lbm_params &p = *v.p;
    if (!v.L->adj_pass1) {
        msg = "no transposed step for this storage type";
        return LBM_ENOTSUP;
    }
    if (v.kp->wall_u || v.kp->q || v.kp->wall_rho) {
        msg = "the adjoint supports resting half-way walls with one virtual density only";
        return LBM_ENOTSUP;
    }
    if (p.force_mode == LBM_FORCE_FIELD) {
        msg = "the adjoint supports CONST and BUOYANT forces only";
        return LBM_ENOTSUP;
    }
    if (nsteps < 1 || K < 1 || (objective != LBM_OBJ_WALL_FORCE_Y && objective != LBM_OBJ_MEAN_JX)) {
        msg = "nsteps and checkpoint_every must be >= 1 and objective one of lbm_objective";
        return LBM_EINVAL;
    }
    if (v.n_fluid < 1) {
        msg = "no fluid node";
        return LBM_EINVAL;
    }
    cudaStream_t st = v.stream;
    const int64_t nseg = (nsteps + K - 1) / K;
    const int64_t Kseg = std::min<int64_t>(K, nsteps);
    // a stored state: the nine planes, then the per-node reference plane of 16-bit storage
    const size_t pop_bytes = (size_t)9 * v.plane * v.elem;
    const size_t ref_bytes = v.refp[0] ? (size_t)v.plane * sizeof(float) : 0;
    const size_t ref_at = (pop_bytes + 255) / 256 * 256;
    const size_t state_bytes = ref_bytes ? ref_at + ref_bytes : pop_bytes;
    auto ref_of = [&](const void *state) -> float * {
        return ref_bytes ? reinterpret_cast<float *>(const_cast<char *>(static_cast<const char *>(state)) + ref_at)
                         : nullptr;
    };
    const size_t real = v.elem == 8 ? 8 : 4;  // arithmetic type: FP64 for FP64 storage, FP32 otherwise
    const size_t plane_r = (size_t)v.plane * real;
    const size_t psi_bytes = (size_t)p.nx * p.ny * real;
    const size_t part_bytes = (size_t)v.L->adj_blocks(*v.kp) * kAdjSlots * sizeof(double);

    // grad == NULL and lambda0 == NULL: the objective alone (forward sweep only)
    const bool backward = grad != nullptr || lambda0 != nullptr;

    // device memory, kept across calls
    Layout L;
    Carver probe{nullptr};
    const size_t need = backward ? carve(probe, L, nseg, Kseg, state_bytes, plane_r, psi_bytes, part_bytes)
                                 : carve(probe, L, 0, 1, 0, 0, 0, 0);
    AdjointState *&as = *v.adj;
    if (!as) as = new AdjointState();
    if (as->bytes < need) {
        if (as->base) {
            cudaStreamSynchronize(st);
            cudaFree(as->base);
            as->base = nullptr;
            as->bytes = 0;
        }
        cudaError_t e = cudaMalloc(&as->base, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            msg = "adjoint: cudaMalloc of " + std::to_string(need >> 20) +
                  " MiB for checkpoints and segment states failed (lower checkpoint_every)";
            return LBM_ENOMEM;
        }
        as->bytes = need;
    }
    Carver cv{static_cast<char *>(as->base)};
    if (backward) carve(cv, L, nseg, Kseg, state_bytes, plane_r, psi_bytes, part_bytes);
    else carve(cv, L, 0, 1, 0, 0, 0, 0);
    if (backward && !as->side) {
        ACK(cudaStreamCreateWithFlags(&as->side, cudaStreamNonBlocking), "cudaStreamCreate");
        cudaEvent_t *evs[] = {&as->fork, &as->recomputed[0], &as->recomputed[1], &as->reversed[0], &as->reversed[1]};
        for (cudaEvent_t *e : evs) ACK(cudaEventCreateWithFlags(e, cudaEventDisableTiming), "cudaEventCreate");
    }

    const double inv_nfluid = 1.0 / double(v.n_fluid);
    const double w = 1.0 / double(nsteps);
    ACK(cudaMemsetAsync(L.acc, 0, 8 * sizeof(double), st), "memset");
    if (backward) ACK(cudaMemsetAsync(L.part, 0, part_bytes, st), "memset");

    // ---- forward sweep: checkpoints and the objective
    KParams kq = *v.kp;
    const int64_t step0 = *v.steps;  // the forward sweep's step t runs as the context's step step0 + t
    for (int64_t t = 0; t < nsteps; ++t) {
        if (backward && t % K == 0) {
            ACK(cudaMemcpyAsync(L.ckpt[t / K], v.pops[*v.cur], pop_bytes, cudaMemcpyDeviceToDevice, st),
                "checkpoint copy");
            if (ref_bytes)
                ACK(cudaMemcpyAsync(ref_of(L.ckpt[t / K]), v.refp[*v.cur], ref_bytes, cudaMemcpyDeviceToDevice, st),
                    "checkpoint copy");
        }
        lbm_status s = v.run_steps(ctx, 1);
        if (s != LBM_OK) {
            msg = "forward step failed";
            return s;
        }
        // with a backward sweep, <W, A_t> of t = 1 .. n-1 is summed by the transposed passes,
        // which read those states anyway; only the last state is summed here
        if (!backward || t == nsteps - 1) {
            kq.src = v.pops[*v.cur];
            kq.ref_src = v.refp[*v.cur];
            ACK(v.L->objective(kq, objective, inv_nfluid, L.acc, st), "objective kernel");
        }
    }

    if (!backward) {
        double h0;
        ACK(cudaMemcpyAsync(&h0, L.acc, sizeof h0, cudaMemcpyDeviceToHost, st), "D2H");
        ACK(cudaStreamSynchronize(st), "objective");
        *J = h0 * w;
        return v.check_error(ctx, msg);
    }

    // ---- backward sweep
    AdjArgs aa{};
    aa.w_scale = w;
    aa.w_scale_f = float(w);
    aa.objective = objective;
    aa.inv_nfluid = inv_nfluid;
    aa.inv_nfluid_f = float(inv_nfluid);
    aa.part = L.part;
    aa.dS = L.dS;
    aa.dpsi = L.dpsi;
    aa.rho = L.rho;
    int gi = 0;  // buffer holding (g, c) of the step after; none before the first reversal
    bool have_next = false;
    // Segment s is recomputed on the side stream into buffer set s & 1 while the transposed
    // steps of segment s + 1 run on the context stream from set (s + 1) & 1; events order a
    // set's reuse after the transposed steps that read it.
    auto recompute = [&](int64_t s) -> lbm_status {
        const int q = (int)(s & 1);
        const int64_t t0 = s * K, t1 = std::min<int64_t>((s + 1) * K, nsteps);
        if (s + 2 < nseg) ACK(cudaStreamWaitEvent(as->side, as->reversed[q], 0), "event wait");
        KParams kp = *v.kp;
        for (int64_t t = t0; t < t1; ++t) {
            kp.src = t == t0 ? L.ckpt[s] : L.seg[q][t - t0 - 1];
            kp.ref_src = ref_of(kp.src);
            kp.psi = L.psi[q][t - t0];
            if (t + 1 < t1) {
                kp.dst = L.seg[q][t - t0];
                kp.ref_dst = ref_of(kp.dst);
                kp.sr_seed = v.sr_seed(step0 + t);
                if (v.fused_pass) {
                    kp.psi_out = static_cast<float *>(kp.psi);
                    ACK(v.fused_pass(kp, as->side), "fused step kernel");
                    kp.psi_out = nullptr;
                } else {
                    ACK(v.psi_pass(kp, as->side), "psi kernel");
                    ACK(v.collide_pass(kp, as->side), "collide kernel");
                }
            } else {
                ACK(v.psi_pass(kp, as->side), "psi kernel");
            }
        }
        ACK(cudaEventRecord(as->recomputed[q], as->side), "event record");
        return LBM_OK;
    };
    ACK(cudaEventRecord(as->fork, st), "event record");
    ACK(cudaStreamWaitEvent(as->side, as->fork, 0), "event wait");
    lbm_status rs = recompute(nseg - 1);
    if (rs != LBM_OK) return rs;
    for (int64_t s = nseg - 1; s >= 0; --s) {
        const int q = (int)(s & 1);
        const int64_t t0 = s * K, t1 = std::min<int64_t>((s + 1) * K, nsteps);
        if (s > 0 && (rs = recompute(s - 1)) != LBM_OK) return rs;
        ACK(cudaStreamWaitEvent(st, as->recomputed[q], 0), "event wait");
        KParams kp = *v.kp;
        for (int64_t t = t1 - 1; t >= t0; --t) {
            kp.src = t == t0 ? L.ckpt[s] : L.seg[q][t - t0 - 1];
            kp.ref_src = ref_of(kp.src);
            kp.psi = L.psi[q][t - t0];
            aa.g_in = have_next ? L.g[gi] : nullptr;
            aa.c_in = have_next ? L.c[gi] : nullptr;
            aa.g_out = L.g[gi ^ 1];
            aa.c_out = L.c[gi ^ 1];
            aa.sum_J = t >= 1;  // <W, A_0> is not part of J
            ACK(v.L->adj_pass1(kp, aa, st), "adjoint pass 1");
            ACK(v.L->adj_pass2(kp, aa, st), "adjoint pass 2");
            gi ^= 1;
            have_next = true;
        }
        ACK(cudaEventRecord(as->reversed[q], st), "event record");
    }

    if (lambda0) {
        const size_t n = (size_t)p.nx * p.ny;
        double *dl = nullptr;
        ACK(cudaMalloc((void **)&dl, 9 * n * sizeof(double)), "cudaMalloc(lambda0)");
        aa.g_in = L.g[gi];
        aa.c_in = L.c[gi];
        KParams kp = *v.kp;
        cudaError_t e = v.L->adj_lambda(kp, aa, dl, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(lambda0, dl, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(dl);
        ACK(e, "lambda0");
    }
    ACK(v.L->adj_reduce(*v.kp, L.part, L.red, st), "adjoint reduction");
    double h[8], r[kAdjSlots];
    ACK(cudaMemcpyAsync(h, L.acc, sizeof h, cudaMemcpyDeviceToHost, st), "D2H");
    ACK(cudaMemcpyAsync(r, L.red, sizeof r, cudaMemcpyDeviceToHost, st), "D2H");
    ACK(cudaStreamSynchronize(st), "adjoint");
    *J = (h[0] + r[SLOT_J]) * w;
    if (grad) {
        grad[0] = r[SLOT_FX];
        grad[1] = r[SLOT_FY];
        grad[2] = r[SLOT_G1] + r[SLOT_G2];
        grad[3] = r[SLOT_T1] + r[SLOT_T2];
    }
    return v.check_error(ctx, msg);
}

}  // namespace lbm
