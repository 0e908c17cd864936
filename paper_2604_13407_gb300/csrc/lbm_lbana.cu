// "LB-ana" of Sec. 3.1 as a library routine: the steady velocity profile of two-phase
// Poiseuille flow that the lattice Boltzmann step itself predicts for a given density
// profile, from the finite-difference velocity equation the paper derives from the step,
// Eq. (fde.ali) for a channel aligned with the lattice and Eq. (fde.obl) for the 45-degree
// channel.  Host code only; no device is touched.
#include <cmath>
#include <string>
#include <vector>

#include "../../include/lbm.h"

namespace lbm {
double eos_psi(const lbm_params &p, double rho);  // lbm_api.cu
lbm_status set_global_error(lbm_status s, const std::string &msg);
}  // namespace lbm

using namespace lbm;

namespace {

// Solve the tridiagonal system sub[i] x[i-1] + diag[i] x[i] + sup[i] x[i+1] = b[i]
// (sub[0], sup[n-1] unused) by Gaussian elimination with partial pivoting; a pivot swap
// between rows i and i+1 creates one extra super-diagonal.  Returns false on a zero pivot.
bool tridiagonal_solve(std::vector<double> sub, std::vector<double> diag, std::vector<double> sup,
                       std::vector<double> b, std::vector<double> &x)
{
    const size_t n = diag.size();
    std::vector<double> sup2(n, 0.0);  // second super-diagonal after pivoting
    for (size_t i = 0; i + 1 < n; ++i) {
        // rows i and i+1 hold the candidates for the pivot of column i
        if (std::fabs(sub[i + 1]) > std::fabs(diag[i])) {
            std::swap(diag[i], sub[i + 1]);
            std::swap(sup[i], diag[i + 1]);
            std::swap(sup2[i], sup[i + 1]);
            std::swap(b[i], b[i + 1]);
        }
        if (diag[i] == 0.0) return false;
        const double m = sub[i + 1] / diag[i];
        diag[i + 1] -= m * sup[i];
        sup[i + 1] -= m * sup2[i];
        b[i + 1] -= m * b[i];
        sub[i + 1] = 0.0;
    }
    if (diag[n - 1] == 0.0) return false;
    x.assign(n, 0.0);
    for (size_t k = n; k-- > 0;) {
        double r = b[k];
        if (k + 1 < n) r -= sup[k] * x[k + 1];
        if (k + 2 < n) r -= sup2[k] * x[k + 2];
        x[k] = r / diag[k];
    }
    return true;
}

}  // namespace

extern "C" lbm_status lbm_lb_ana(const lbm_params *p, int32_t oblique, int32_t n, const double *rho,
                                 const double *f_int, double F_drive, double *u)
{
    if (!p || !rho || !u) return set_global_error(LBM_EINVAL, "null argument");
    if (p->struct_size != (int32_t)sizeof(lbm_params))
        return set_global_error(LBM_EINVAL, "lbm_params.struct_size does not match this library");
    if (n < 3) return set_global_error(LBM_EINVAL, "the profile needs at least 3 nodes");
    if (p->tau_l != p->tau_g || !(p->tau_l > 0.5))
        return set_global_error(LBM_EINVAL, "LB-ana takes one relaxation time tau > 1/2 (tau_l == tau_g)");
    if (!(p->G < 0.0)) return set_global_error(LBM_EINVAL, "G must be < 0");
    const double nu = (p->tau_l - 0.5) / 3.0;
    const double sG = std::sqrt(-p->G);
    // rescaled pseudopotential psi_hat = sqrt(-G) psi of every node, and of the walls
    std::vector<double> ph(n);
    for (int i = 0; i < n; ++i) {
        const double ps = sG * eos_psi(*p, rho[i]);
        if (!(rho[i] > 0.0) || !std::isfinite(ps) || !(ps > 0.0))
            return set_global_error(LBM_EINVAL, "density out of the range where psi is real and positive");
        ph[i] = ps;
    }
    const double pw = sG * eos_psi(*p, p->rho_s);
    if (!std::isfinite(pw)) return set_global_error(LBM_EINVAL, "psi(rho_s) is not real");
    auto psi_at = [&](int i) { return (i < 0 || i >= n) ? pw : ph[i]; };
    // pairwise force along the profile, Eq. (obl.10) (x component at 45 degrees)
    std::vector<double> F(n), X(n);
    for (int i = 0; i < n; ++i) {
        if (f_int) {
            F[i] = f_int[i];
        } else if (!oblique) {
            F[i] = ph[i] * (psi_at(i + 1) - psi_at(i - 1)) / 2.0;
        } else {
            F[i] = ph[i] * (psi_at(i + 2) + 4.0 * psi_at(i + 1) - 4.0 * psi_at(i - 1) - psi_at(i - 2)) / 12.0;
        }
        X[i] = F[i] * F[i] / (ph[i] * ph[i]);  // dt^2 F_hat^2 / psi_hat^2
    }
    // coefficient c of X u in the second difference of the source term:
    //   aligned, Eq. (qm6.ali): Q_m,6 = (3 eps/8) X u   -> c = 3 eps / 8
    //   45 degrees, Eq. (obl.11): -sqrt2/4 times the second difference of Q_m,4+6 =
    //   -2 sqrt2 K X u_beta is + K times that of X u_beta, K = (24 eps - 15)/32
    // and 0 for the original scheme (its Q_m,4 and Q_m,6 vanish)
    const double eps = -8.0 * (p->k1 + p->k2);
    double c = 0.0;
    if (p->scheme == LBM_SCHEME_IMPROVED) c = oblique ? (24.0 * eps - 15.0) / 32.0 : 3.0 * eps / 8.0;
    const double rhs = oblique ? -F_drive / (2.0 * nu) : -F_drive / nu;  // dx^2/2 at 45 degrees
    std::vector<double> sub(n, 0.0), diag(n), sup(n, 0.0), b(n, rhs);
    for (int i = 0; i < n; ++i) {
        diag[i] = -2.0 * (rho[i] + c * X[i]);
        if (i > 0) sub[i] = rho[i - 1] + 1.5 * F[i - 1] + c * X[i - 1];
        if (i + 1 < n) sup[i] = rho[i + 1] - 1.5 * F[i + 1] + c * X[i + 1];
    }
    // half-way no-slip walls: each end row sees a mirror ghost node (u = -u of the end node,
    // its density and X, the normal force reversed)
    diag[0] -= rho[0] - 1.5 * F[0] + c * X[0];
    diag[n - 1] -= rho[n - 1] + 1.5 * F[n - 1] + c * X[n - 1];
    std::vector<double> x;
    if (!tridiagonal_solve(sub, diag, sup, b, x)) return set_global_error(LBM_EINVAL, "singular velocity equation");
    for (int i = 0; i < n; ++i) u[i] = x[i];
    return LBM_OK;
}
