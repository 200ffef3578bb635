"""Algorithm 2 (HOT) of arXiv 2408.00598 with the relative KKT stopping rule.

Test infrastructure only (see ``oracle/__init__``).

The iteration keeps w = (y, z, x) exactly as Algorithm 2 prints it:

* Step 1  y-bar = argmin_y L_sigma(y, z^k; x^k), i.e. the normal equation
          AA^T y-bar = b/sigma - A(x^k/sigma + z^k - c)   (eq. update:y),
          solved by Prop. 3 (``linsolve.solve_aat``);
* Step 2  x-bar = x^k + sigma (A^T y-bar + z^k - c);
* Step 3  z-bar = Pi_+(c - A^T y-bar - x-bar/sigma)       (Sec. III-B);
* Step 4  w^{k+1} = w^0/(k+2) + (k+1)/(k+2) (2 w-bar - w^k).

The stopping rule is the relative KKT residual eq. (kkt_res) evaluated at
w-bar = (y-bar, z-bar, x-bar), the iterate whose convergence Prop. 2/3 state.

Readings where the paper is silent (Sec. IV-A gives only the stopping rule):

* w^0 = 0.
* The cost is scaled: c <- c / 2^ceil(log2 max c) (a power of two, so the
  scaled costs are exact binary fractions); the KKT residual is measured on the
  scaled problem and the OT value is reported unscaled, <c, x-bar>.
* sigma_0 = ||b|| / ||c|| (scaled c).
* Restarts (the iteration as printed never moves its anchor; the paper cites
  the restarted Halpern scheme of its reference [sun2024accelerating] / HPR):
  every K = 10 iterations, with r = ||w^k - w-bar^k||_M, the seminorm of the
  operator M of eq. (def:M), and r0 its value at the first check of the
  current cycle, restart when r <= 0.2 r0, or r <= 0.8 r0 and r grew since the
  previous check, or the cycle is at least 0.2 times the total iteration count.
  A restart sets the anchor and the iterate to w-bar, the cycle counter k to 0,
  and sigma <- sqrt(sigma * ||x-bar - x_r|| / ||z-bar - z_r||), the geometric
  mean of the old sigma and the primal/dual movement ratio since the previous
  restart point (x_r, z_r) (0 before the first).  The ratio alone balances the
  two parts of the M-norm (App. A) but swings over many orders of magnitude
  on degenerate inputs; the geometric mean damps it.  The new sigma is then
  rounded to the geometric grid 2^(j/16): sigma is a free parameter, so a
  4 % grid leaves the iteration counts unchanged on the synthetic classes,
  while two runs whose norms differ only by rounding (an FP32 and an FP64
  implementation) pick the same sigma instead of drifting apart by the
  rounding error at every restart.
* The iteration cap is tested at check iterations: the solve stops at the first
  check iteration whose total count reaches max_iter.

Variants (Sec. IV-A and App. D):

* method="gadmm": the generalized ADMM the paper compares against, Algorithm 2
  with Step 4 replaced by w^{k+1} = (1 - rho) w^k + rho w-bar^k (rho = 1.7;
  rho = 1 is plain ADMM, w^{k+1} = w-bar^k).  Reading: the restart rule and
  the sigma update above apply unchanged (a restart sets the iterate to w-bar).
* stop="absolute": the absolute KKT residual of Table VI, the three terms of
  eq. (kkt_res) without their normalisers, max{||A^T y + z - c||,
  ||min(x, z)||, ||Ax - b||}.  Reading: measured, like the relative one, on the
  scaled problem that is solved.
"""
from dataclasses import dataclass, field
import math
import numpy as np

from .reduced_model import build_A, build_b, build_c, split_x
from .linsolve import solve_aat


@dataclass
class HotParams:
    """Free parameters of Algorithm 2 plus the restart reading (module docstring)."""
    sigma0: float = 0.0            # <= 0: ||b|| / ||c|| of the scaled problem
    check_every: int = 10          # K
    restart: bool = True           # False: Algorithm 2 exactly as printed
    restart_sufficient: float = 0.2
    restart_necessary: float = 0.8
    restart_long: float = 0.2
    scale_cost: bool = True
    sigma_steps: int = 16          # sigma rounded to 2^(j / sigma_steps) at restarts (0: not rounded)
    method: str = "hot"            # "hot" (Halpern Step 4) or "gadmm" (generalized ADMM)
    relax: float = 1.7             # rho of the generalized ADMM
    stop: str = "relative"         # "relative" (eq. kkt_res) or "absolute" (Table VI)


@dataclass
class HotResult:
    ot_value: float                # <c, x-bar> (unscaled)
    dual_value: float              # <b, y-bar> (unscaled)
    rel_kkt: float
    parts: tuple                   # (dual, complementarity, primal) terms of eq. (kkt_res)
    abs_kkt: float                 # max of the same three terms without normalisers
    iters: int
    restarts: int
    converged: bool
    sigma: float
    cost_scale: float
    x: np.ndarray = field(repr=False)
    y: np.ndarray = field(repr=False)
    z: np.ndarray = field(repr=False)
    trace: list = field(default_factory=list, repr=False)   # (iteration, rel_kkt, restart?, sigma)


def kkt_residual(A, b, c, x, y, z):
    """Relative KKT residual eq. (kkt_res): max of
    ||A^T y + z - c|| / (1 + ||c||), ||min(x, z)|| / (1 + ||x|| + ||z||),
    ||Ax - b|| / (1 + ||b||)."""
    dual = np.linalg.norm(A.T @ y + z - c) / (1.0 + np.linalg.norm(c))
    comp = np.linalg.norm(np.minimum(x, z)) / (1.0 + np.linalg.norm(x) + np.linalg.norm(z))
    primal = np.linalg.norm(A @ x - b) / (1.0 + np.linalg.norm(b))
    return max(dual, comp, primal), (dual, comp, primal)


def kkt_absolute(A, b, c, x, y, z):
    """Absolute KKT residual (Table VI): max{||A^T y + z - c||, ||min(x, z)||, ||Ax - b||}."""
    return max(np.linalg.norm(A.T @ y + z - c), np.linalg.norm(np.minimum(x, z)), np.linalg.norm(A @ x - b))


def kkt_mapping(A, b, c, x, y, z):
    """The residual mapping R(w) of Sec. III-A: (b - Ax, z - Pi_+(z - x), c - A^T y - z)."""
    return (b - A @ x, z - np.maximum(z - x, 0.0), c - A.T @ y - z)


def cost_scale(c, scale_cost=True):
    """Power-of-two cost scale: the smallest 2^e >= max c (reading; 1 if disabled)."""
    cmax = float(np.max(c))
    if not scale_cost or cmax <= 0.0:
        return 1.0
    return 2.0 ** math.ceil(math.log2(cmax))


def hot_step(A, b, c, sigma, x, z, m, n):
    """Steps 1-3 of Algorithm 2 from (x^k, z^k): returns (y-bar, x-bar, z-bar)."""
    # Step 1 (eq. update:y, solved by Prop. 3)
    rhs = b / sigma - A @ (x / sigma + z - c)
    y_bar = solve_aat(rhs, m, n)
    Aty = A.T @ y_bar
    # Step 2
    x_bar = x + sigma * (Aty + z - c)
    # Step 3
    z_bar = np.maximum(c - Aty - x_bar / sigma, 0.0)
    return y_bar, x_bar, z_bar


def hot_solve(mu1, mu2, tol=1e-6, max_iter=100000, params=None, xs=None, ys=None, on_iterate=None):
    """Run Algorithm 2 on the reduced model of (mu1, mu2) until rel-KKT <= tol.

    ``on_iterate(total, sigma, x, z, x_bar, y_bar, z_bar)`` (optional) sees every
    iteration's state on the scaled problem."""
    p = params or HotParams()
    mu1 = np.asarray(mu1, dtype=np.float64)
    mu2 = np.asarray(mu2, dtype=np.float64)
    m, n = mu1.shape
    A = build_A(m, n)
    b = build_b(mu1, mu2)
    c_full = build_c(m, n, xs, ys)
    scale = cost_scale(c_full, p.scale_cost)
    c = c_full / scale
    nb, nc = np.linalg.norm(b), np.linalg.norm(c)
    sigma = float(p.sigma0 if p.sigma0 > 0 else nb / nc)
    N = c.size
    K = p.check_every

    x0 = np.zeros(N)
    z0 = np.zeros(N)
    y0 = np.zeros(A.shape[0])
    x, z, y = x0.copy(), z0.copy(), y0.copy()
    x_r, z_r = np.zeros(N), np.zeros(N)
    k = 0                       # Halpern counter since the last restart
    total = 0
    restarts = 0
    r0 = None
    r_prev = None
    trace = []
    while True:
        y_bar, x_bar, z_bar = hot_step(A, b, c, sigma, x, z, m, n)
        total += 1
        if on_iterate is not None:
            on_iterate(total, sigma, x, z, x_bar, y_bar, z_bar)

        if total % K == 0:
            err, parts = kkt_residual(A, b, c, x_bar, y_bar, z_bar)
            err = float(err)
            parts = tuple(float(q) for q in parts)
            aerr = float(kkt_absolute(A, b, c, x_bar, y_bar, z_bar))
            done = bool((aerr if p.stop == "absolute" else err) <= tol)
            capped = total >= max_iter
            restart = False
            if not done and not capped and p.restart:
                r = float(np.linalg.norm((x - x_bar) + sigma * (z - z_bar))) / math.sqrt(sigma)
                if r0 is None:
                    r0 = r
                restart = (r <= p.restart_sufficient * r0
                           or (r_prev is not None and r <= p.restart_necessary * r0 and r > r_prev)
                           or k >= p.restart_long * total)
                r_prev = r
            trace.append((total, err, restart, sigma))
            if done or capped:
                return HotResult(ot_value=scale * float(c @ x_bar), dual_value=scale * float(b @ y_bar),
                                 rel_kkt=err, parts=parts, abs_kkt=aerr, iters=total, restarts=restarts,
                                 converged=done,
                                 sigma=sigma, cost_scale=scale, x=x_bar, y=scale * y_bar, z=scale * z_bar,
                                 trace=trace)
            if restart:
                dx = float(np.linalg.norm(x_bar - x_r))
                dz = float(np.linalg.norm(z_bar - z_r))
                if dx > 0.0 and dz > 0.0 and math.isfinite(dx / dz):
                    sigma = math.sqrt(sigma * (dx / dz))
                    if p.sigma_steps > 0:
                        q = p.sigma_steps
                        sigma = 2.0 ** (round(math.log2(sigma) * q) / q)
                x_r, z_r = x_bar.copy(), z_bar.copy()
                x0, z0, y0 = x_bar.copy(), z_bar.copy(), y_bar.copy()
                x, z, y = x0.copy(), z0.copy(), y0.copy()
                k = 0
                r0 = None
                r_prev = None
                restarts += 1
                continue

        if p.method == "gadmm":
            # Step 4 of the generalized ADMM: w^{k+1} = (1 - rho) w^k + rho w-bar^k
            rho = p.relax
            x = (1.0 - rho) * x + rho * x_bar
            z = (1.0 - rho) * z + rho * z_bar
            y = (1.0 - rho) * y + rho * y_bar
        else:
            # Step 4 (Halpern, step size 1/(k+2))
            x = x0 / (k + 2) + (k + 1) / (k + 2) * (2.0 * x_bar - x)
            z = z0 / (k + 2) + (k + 1) / (k + 2) * (2.0 * z_bar - z)
            y = y0 / (k + 2) + (k + 1) / (k + 2) * (2.0 * y_bar - y)
        k += 1


def gap(x, x_b, c):
    """Relative objective gap of Sec. IV-A: |<c,x> - <c,x_b>| / (|<c,x_b>| + 1)."""
    return abs(float(c @ x) - float(c @ x_b)) / (abs(float(c @ x_b)) + 1.0)


def feaserr(A, b, x):
    """Relative primal feasibility error of Sec. IV-A:
    max{ ||min(x,0)|| / (1 + ||x||), ||Ax - b|| / (1 + ||b||) }."""
    return max(np.linalg.norm(np.minimum(x, 0.0)) / (1.0 + np.linalg.norm(x)),
               np.linalg.norm(A @ x - b) / (1.0 + np.linalg.norm(b)))


def flows(result, m, n):
    """f1[i,k,j], f2[k,j,l] of the returned x-bar."""
    return split_x(result.x, m, n)
