"""FP64 reference adjoint of the pseudopotential MRT-LB step (test infrastructure only).

TEST INFRASTRUCTURE ONLY.  A plain PyTorch (CPU, float64) restatement of the step of
Sec. 2 in the same stage order as the C oracle (lbm_oracle.c), differentiated by
autograd.  It supports what the adjoint covers: periodic directions, half-way resting
walls (non-periodic edges and solid nodes), constant or buoyant external force, one or
two relaxation times.  Its forward pass is pinned to the C oracle; its gradients to
central finite differences of the C oracle.

Objective (the time average used by the library's adjoint):
    J = (1/n) sum_{t=1..n} <W, A_t>
with A_t the stored post-collision populations after step t and W the weights of
    'mean_jx'       W_i(x) = e_ix / N_fluid at fluid nodes
    'wall_force_y'  W_o(x) = 2 e_oy when x + e_o is a wall (the y momentum that the
                    half-way walls receive from A_t in the next streaming).
"""
import numpy as np
import torch

EX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
EY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]
M = [[1, 1, 1, 1, 1, 1, 1, 1, 1], [-4, -1, -1, -1, -1, 2, 2, 2, 2], [4, -2, -2, -2, -2, 1, 1, 1, 1],
     [0, 1, 0, -1, 0, 1, -1, -1, 1], [0, -2, 0, 2, 0, 1, -1, -1, 1], [0, 0, 1, 0, -1, 1, 1, -1, -1],
     [0, 0, -2, 0, 2, 1, 1, -1, -1], [0, 1, -1, 1, -1, 0, 0, 0, 0], [0, 0, 0, 0, 0, 1, -1, 1, -1]]
MNORM = [9, 36, 36, 6, 12, 6, 12, 4, 4]


class Geometry:
    """Index maps of the pull: for node x and direction i, the flat index of x - e_i, and
    whether x - e_i is a wall (beyond a non-periodic edge, or solid)."""

    def __init__(self, nx, ny, periodic_x, periodic_y, solid=None):
        self.nx, self.ny = nx, ny
        self.solid = np.zeros((ny, nx), bool) if solid is None else np.asarray(solid, bool)
        self.fluid = torch.tensor(~self.solid.reshape(-1))
        y, x = np.mgrid[0:ny, 0:nx]

        def wall_and_index(dx, dy):
            xs, ys = x + dx, y + dy
            out = np.zeros((ny, nx), bool)
            if not periodic_x:
                out |= (xs < 0) | (xs >= nx)
            if not periodic_y:
                out |= (ys < 0) | (ys >= ny)
            xs, ys = np.mod(xs, nx), np.mod(ys, ny)
            idx = ys * nx + xs
            out |= self.solid[ys, xs]
            return torch.tensor(out.reshape(-1)), torch.tensor(idx.reshape(-1), dtype=torch.long)

        self.src = [wall_and_index(-EX[i], -EY[i]) for i in range(9)]  # pull source x - e_i
        self.nb = [wall_and_index(EX[i], EY[i]) for i in range(9)]     # neighbour x + e_i


def p_eos(rho, eos, a, b, R, T, K):
    if eos == 0:
        return K * (rho * R * T / (1.0 - b * rho) - a * rho * rho)
    eta = b * rho / 4.0
    return K * (rho * R * T * (1.0 + eta + eta * eta - eta * eta * eta) / ((1.0 - eta) ** 3) - a * rho * rho)


def psi_of(rho, p, G, T):
    return torch.sqrt(2.0 * (p_eos(rho, p.eos, p.a, p.b, p.R, T, p.K_eos) - rho / 3.0) / G)


def step(A, geo, p, theta):
    """One step of the method (Sec. 2) on A [9, n]; theta = (Fx, Fy, G, T) tensors."""
    Fx0, Fy0, G, T = theta
    n = A.shape[1]
    # 1. pull with half-way resting walls
    f = []
    for i in range(9):
        wall, idx = geo.src[i]
        f.append(torch.where(wall, A[OPP[i]], A[i][idx]))
    f = torch.stack(f)
    # 2. moments
    rho = f.sum(0)
    jx = sum(EX[i] * f[i] for i in range(9))
    jy = sum(EY[i] * f[i] for i in range(9))
    # 3. pseudopotential, walls psi(rho_s)
    psi = psi_of(rho, p, G, T)
    psi_s = psi_of(torch.tensor(p.rho_s, dtype=torch.float64), p, G, T)
    # 4. force
    Sx = torch.zeros(n, dtype=torch.float64)
    Sy = torch.zeros(n, dtype=torch.float64)
    for i in range(1, 9):
        wall, idx = geo.nb[i]
        ps = torch.where(wall, psi_s, psi[idx])
        w = 1.0 / 3.0 if i <= 4 else 1.0 / 12.0
        Sx = Sx + w * ps * EX[i]
        Sy = Sy + w * ps * EY[i]
    Fix = -G * psi * Sx
    Fiy = -G * psi * Sy
    if p.force_mode == 0:
        Fex, Fey = Fx0 * torch.ones_like(rho), Fy0 * torch.ones_like(rho)
    else:
        Fex, Fey = (rho - p.rho_g) * Fx0, (rho - p.rho_g) * Fy0
    Fx, Fy = Fix + Fex, Fiy + Fey
    # 5. velocity
    ux = (jx + 0.5 * Fx) / rho
    uy = (jy + 0.5 * Fy) / rho
    # 6. moments, equilibrium, forcing, source
    m = [sum(M[k][i] * f[i] for i in range(9)) for k in range(9)]
    u2 = ux * ux + uy * uy
    meq = [rho, -2.0 * rho + 3.0 * rho * u2, rho - 3.0 * rho * u2, rho * ux, -rho * ux, rho * uy, -rho * uy,
           rho * ux * ux - rho * uy * uy, rho * ux * uy]
    Fu = Fx * ux + Fy * uy
    Fm = [torch.zeros_like(rho), 6.0 * Fu, -6.0 * Fu, Fx, -Fx, Fy, -Fy, 2.0 * Fx * ux - 2.0 * Fy * uy,
          Fx * uy + Fy * ux]
    Gpsi2 = G * psi * psi
    X = Fix * Fix / Gpsi2
    Y = Fiy * Fiy / Gpsi2
    eps = -8.0 * (p.k1 + p.k2)
    zero = torch.zeros_like(rho)
    Q = [zero] * 9
    Q[1] = 3.0 * (p.k1 + 2.0 * p.k2) * (X + Y)
    Q[7] = p.k1 * (Fix * Fix - Fiy * Fiy) / Gpsi2
    Q[8] = p.k1 * Fix * Fiy / Gpsi2
    if p.scheme == 0:
        Q[2] = -Q[1]
    else:
        Q[2] = -Q[1] if p.q2_original else -Q[1] / 2.0
        Q[4] = ((30.0 * eps - 15.0) / 16.0 * X - 3.0 * eps / 8.0 * Y) * ux
        Q[6] = ((30.0 * eps - 15.0) / 16.0 * Y - 3.0 * eps / 8.0 * X) * uy
    # 7. relaxation rates
    if p.tau_l == p.tau_g:
        tau = p.tau_l * torch.ones_like(rho)
    else:
        nu_l, nu_g = (p.tau_l - 0.5) / 3.0, (p.tau_g - 0.5) / 3.0
        w = torch.clamp((rho - p.rho_g) / (p.rho_l - p.rho_g), 0.0, 1.0)
        tau = 3.0 * (nu_g + w * (nu_l - nu_g)) + 0.5
    sp = 1.0 / tau
    sq = 1.0 / (0.5 + p.Lambda / (tau - 0.5))
    one = torch.ones_like(rho)
    s = [one, sp, sp, one, sq, one, sq, sp, sp]
    # 8. collision and back-transform
    mb = [m[k] + Fm[k] - s[k] * (m[k] - meq[k] + 0.5 * Fm[k]) + s[k] * Q[k] for k in range(9)]
    fb = torch.stack([sum(M[k][i] * (mb[k] / MNORM[k]) for k in range(9)) for i in range(9)])
    return torch.where(geo.fluid[None, :], fb, A)


def weights(geo, objective):
    n = geo.nx * geo.ny
    W = torch.zeros((9, n), dtype=torch.float64)
    fluid = geo.fluid
    if objective == "mean_jx":
        nf = float(fluid.sum())
        for i in range(9):
            W[i] = torch.where(fluid, torch.tensor(EX[i] / nf, dtype=torch.float64), torch.tensor(0.0, dtype=torch.float64))
    elif objective == "wall_force_y":
        for o in range(1, 9):
            wall, _ = geo.nb[o]
            W[o] = torch.where(fluid & wall, torch.tensor(2.0 * EY[o], dtype=torch.float64), torch.tensor(0.0, dtype=torch.float64))
    else:
        raise ValueError(objective)
    return W


def objective_and_grad(p, A0, nsteps, objective, solid=None):
    """(J, dJ/d(Fx, Fy, G, T), dJ/dA0 [9, ny, nx]) by autograd through nsteps steps."""
    geo = Geometry(p.nx, p.ny, bool(p.periodic_x), bool(p.periodic_y), solid)
    theta = [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in (p.Fx, p.Fy, p.G, p.T)]
    A = torch.tensor(np.asarray(A0, dtype=np.float64).reshape(9, -1), requires_grad=True)
    W = weights(geo, objective)
    J = torch.zeros((), dtype=torch.float64)
    X = A
    for _ in range(nsteps):
        X = step(X, geo, p, theta)
        J = J + (W * X).sum()
    J = J / nsteps
    J.backward()
    g = np.array([float(t.grad) if t.grad is not None else 0.0 for t in theta])
    return float(J), g, A.grad.numpy().reshape(9, p.ny, p.nx)


def forward_states(p, A0, nsteps, solid=None):
    """States A_1..A_n as a numpy array [n, 9, ny, nx] (for pinning against the C oracle)."""
    geo = Geometry(p.nx, p.ny, bool(p.periodic_x), bool(p.periodic_y), solid)
    theta = [torch.tensor(v, dtype=torch.float64) for v in (p.Fx, p.Fy, p.G, p.T)]
    X = torch.tensor(np.asarray(A0, dtype=np.float64).reshape(9, -1))
    out = []
    with torch.no_grad():
        for _ in range(nsteps):
            X = step(X, geo, p, theta)
            out.append(X.numpy().reshape(9, p.ny, p.nx).copy())
    return np.array(out)


def objective_value(p, states, objective, solid=None):
    """J of a sequence of states (numpy), same weights as above."""
    geo = Geometry(p.nx, p.ny, bool(p.periodic_x), bool(p.periodic_y), solid)
    W = weights(geo, objective).numpy().reshape(9, p.ny, p.nx)
    return float(np.mean([(W * s).sum() for s in states]))
