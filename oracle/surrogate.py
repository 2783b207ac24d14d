"""Oracle of the surrogate stage: training samples from DSMC moment sums, Bayesian ridge
regression with evidence maximisation, model selection and the corrected 1D
macroscopic solve with Monte Carlo uncertainty bands.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct reference
the library's surrogate path is checked against.  Only the tests, the smoke check and
the CPU baseline of the benchmark may import it; the library never does.

Everything is binary64 numpy, written from the paper's text:

* units of Eq. 6, corrected Newton's law Eq. 7, macroscopic equation Eq. 8, no-slip
  and slip boundary conditions Eqs. 9-10 (Sec. 2.2);
* boundary models Eqs. 11-12, constitutive models Eq. 13 with the stress correction
  Eq. 14 and the exponents of Table 1, linear models Eqs. 15-16 with the design
  matrices of Appendix A, model probabilities Eq. 17 (Sec. 2.3);
* Bayesian ridge regression as the paper describes it (Sec. 2.3): an isotropic
  Gaussian prior of precision alpha on the weights, Gaussian noise of precision beta,
  alpha and beta chosen to maximise the evidence with the re-estimation equations of
  MacKay as given by Bishop (Pattern Recognition and Machine Learning, Sec. 3.5) and
  Tipping (2001, App. A): gamma = sum lambda_i / (alpha + lambda_i) over the
  eigenvalues lambda_i of beta Phi^T Phi, alpha = gamma / m^T m,
  beta = (N - gamma) / |t - Phi m|^2, posterior S = (alpha I + beta Phi^T Phi)^-1,
  m = beta S Phi^T t, log evidence (Bishop Eq. 3.86);
* Monte Carlo propagation of the weight posteriors (Sec. 2.3), with the standard
  normal draws passed in.

Readings where the paper is silent (each listed in the design notes):
* a training sample is one window of sampled steps: per cell u = sum vx / N and
  P_xy = 2 n (<vx vy> - <vx><vy>) with n = N / (steps ppc) (Eq. 6 units);
* du/dy at cell i is the central difference of the cell velocities; training points are
  the cells that have both neighbours (N_P = n_cells - 2), or in a sub-domain of the MMS
  hybrid the cells of the training region that have both neighbours;
* the DSMC velocity at a wall is the linear extrapolation from the two nearest cell
  centres, u(wall) = 1.5 u_0 - 0.5 u_1;
* P^CFD at the walls is the exact shear stress of the 1D problem, P(y) = F (2y - 1)
  (Eq. 1 integrated with the symmetry P(1/2) = 0; the paper notes the macroscopic model
  always returns it);
* Table 1 exponents at the tabulated Kn nearest in log Kn, used as printed;
* no intercept and flat hyperpriors in the regression; the weight precision is capped
  at 1e30 when the evidence keeps increasing with it (weights not supported);
* the CFD is cell-centred finite volume on n equal cells with the wall values imposed
  through ghost cells, S evaluated at the cell faces.
"""
from __future__ import annotations

import math

import numpy as np

SQRT_PI = math.sqrt(math.pi)

# Table 1: exponents b_1, b_2, b_3 of the stress-correction basis at the tabulated Kn.
TABLE1_KN = (0.01, 0.05, 0.1, 0.2, 0.5, 1.0, 5.0)
TABLE1_B = ((130.0, 150.0, 200.0), (30.0, 40.0, 70.0), (20.0, 40.0, 10.0), (20.0, 12.0, 8.0),
            (10.0, 7.0, 6.0), (8.0, 6.0, 20.0), (7.0, 6.0, 5.0))

# Largest weight precision: above it the weights are switched off (see brr).
ALPHA_MAX = 1e30

V_MODELS = ("no-slip", "slip")
C_MODELS = ("C0", "C1", "C2", "C3")


def exponents(Kn: float):
    """Table 1 row at the tabulated Kn nearest to Kn in log Kn."""
    k = int(np.argmin([abs(math.log(Kn) - math.log(x)) for x in TABLE1_KN]))
    return TABLE1_B[k]


def cell_fields(acc, n_steps: int, ppc: int):
    """(u, P) per cell from the raw sums of one window (Eq. 6 units)."""
    a = np.asarray(acc, np.float64)
    N = a[:, 0]
    ux = a[:, 1] / N
    uy = a[:, 2] / N
    cxy = a[:, 7] / N - ux * uy
    n = N / (n_steps * ppc)
    return ux, 2.0 * n * cxy


def basis(y, Kn: float, b):
    """Appendix A constitutive basis: (2 Kn / sqrt(pi)) (exp(-b_l y) - exp(-b_l (1 - y)))
    for each exponent (walls at y = 0 and 1), one column per exponent."""
    y = np.asarray(y, np.float64)
    cols = [(2.0 * Kn / SQRT_PI) * (np.exp(-bl * y) - np.exp(-bl * (1.0 - y))) for bl in b]
    return np.stack(cols, axis=1)


def training_sample(acc, n_steps: int, ppc: int, Kn: float, F: float, b, length: float = 1.0,
                    n_train=None):
    """One training sample (Appendix A): the slip-model data and targets
    (x = -P(0) = F at the bottom wall and P(1) = F at the top, t = DSMC wall velocities)
    and the constitutive-model design rows and targets E_i = P_i + (2 Kn / sqrt(pi))
    du/dy_i (Eq. 13).

    The run covers y in [0, length] (channel units) with its cells of equal width.
    length = 1: the whole channel, both walls, training cells 1..n-2.  length < 1: a
    DSMC sub-domain of the MMS hybrid above the bottom wall (Sec. 2, Sec. 3.2), the
    bottom wall only, training cells 1..n_train-1 (the cells within the training
    region; the rest is the buffer next to the interface)."""
    u, P = cell_fields(acc, n_steps, ppc)
    n = u.size
    h = length / n
    y = (np.arange(n) + 0.5) * h
    last = n - 2 if length == 1.0 else int(n_train) - 1
    i = np.arange(1, last + 1)
    dudy = (u[i + 1] - u[i - 1]) / (2.0 * h)
    E = P[i] + (2.0 * Kn / SQRT_PI) * dudy
    u_bot = 1.5 * u[0] - 0.5 * u[1]
    if length == 1.0:
        u_top = 1.5 * u[n - 1] - 0.5 * u[n - 2]
        x_v, t_v = np.array([F, F]), np.array([u_bot, u_top])
    else:
        x_v, t_v = np.array([F]), np.array([u_bot])
    return {"x_v": x_v, "t_v": t_v, "phi_c": basis(y[i], Kn, b), "t_c": E}


def log_evidence_zero(t):
    """Evidence of a model without weights (no-slip, C0): t ~ N(0, beta^-1 I) with beta
    at its maximum N / t^T t."""
    t = np.asarray(t, np.float64)
    N = t.size
    tt = float(t @ t)
    beta = N / tt
    return 0.5 * N * math.log(beta) - 0.5 * N * math.log(2.0 * math.pi) - 0.5 * beta * tt, beta


def brr(Phi, t, max_iter: int = 1000, tol: float = 1e-12):
    """Bayesian ridge regression: evidence maximisation over (alpha, beta) by the
    re-estimation equations, then the posterior (m, S) and the log evidence."""
    Phi = np.asarray(Phi, np.float64)
    t = np.asarray(t, np.float64)
    N, M = Phi.shape
    G = Phi.T @ Phi
    Pt = Phi.T @ t
    eig = np.linalg.eigvalsh(G)
    alpha, beta = 1.0, 1.0 / max(float(np.var(t)), 1e-300)
    for it in range(max_iter):
        A = alpha * np.eye(M) + beta * G
        S = np.linalg.inv(A)
        m = beta * S @ Pt
        lam = beta * eig
        gamma = float(np.sum(lam / (alpha + lam)))
        r = t - Phi @ m
        mm = float(m @ m)
        # When the data do not support the weights, alpha grows without bound (the
        # model tends to its zero-weight limit); it is held at ALPHA_MAX.
        alpha_new = ALPHA_MAX if mm <= gamma / ALPHA_MAX else gamma / mm
        beta_new = (N - gamma) / float(r @ r)
        done = (abs(alpha_new - alpha) <= tol * alpha and abs(beta_new - beta) <= tol * beta)
        alpha, beta = alpha_new, beta_new
        if done:
            break
    A = alpha * np.eye(M) + beta * G
    S = np.linalg.inv(A)
    m = beta * S @ Pt
    r = t - Phi @ m
    E = 0.5 * beta * float(r @ r) + 0.5 * alpha * float(m @ m)
    sign, logdet = np.linalg.slogdet(A)
    logev = (0.5 * M * math.log(alpha) + 0.5 * N * math.log(beta) - E - 0.5 * logdet
             - 0.5 * N * math.log(2.0 * math.pi))
    return {"m": m, "S": S, "alpha": alpha, "beta": beta, "log_evidence": logev,
            "iterations": it + 1}


def probabilities(log_evidences):
    """Eq. 17 with equal priors."""
    le = np.asarray(log_evidences, np.float64)
    w = np.exp(le - le.max())
    return w / w.sum()


# Two models whose log evidences agree to this relative tolerance are tied (rounding
# noise, e.g. every extra weight shrunk to zero on data with no signal for it); Eq. 17
# then ranks them equally and the simpler model, the lower index, is selected.
TIE_REL = 1e-9


def select(log_evidences) -> int:
    """Eq. 17's most probable model (equal priors), the simplest among ties."""
    le = np.asarray(log_evidences, np.float64)
    top = le.max()
    return int(np.flatnonzero(le >= top - TIE_REL * max(1.0, abs(top)))[0])


def train(samples, Kn: float):
    """Fits every boundary and constitutive model to the stacked samples and selects the
    most probable of each kind (Sec. 2.3)."""
    x_v = np.concatenate([s["x_v"] for s in samples])
    t_v = np.concatenate([s["t_v"] for s in samples])
    phi = np.concatenate([s["phi_c"] for s in samples])
    t_c = np.concatenate([s["t_c"] for s in samples])
    v = [dict(zip(("log_evidence", "beta"), log_evidence_zero(t_v)), m=np.zeros(0),
              S=np.zeros((0, 0)))]
    v.append(brr(x_v[:, None], t_v))
    c = [dict(zip(("log_evidence", "beta"), log_evidence_zero(t_c)), m=np.zeros(0),
              S=np.zeros((0, 0)))]
    for k in (1, 2, 3):
        c.append(brr(phi[:, :k], t_c))
    pv = probabilities([f["log_evidence"] for f in v])
    pc = probabilities([f["log_evidence"] for f in c])
    return {"v": v, "c": c, "p_v": pv, "p_c": pc,
            "sel_v": select([f["log_evidence"] for f in v]),
            "sel_c": select([f["log_evidence"] for f in c])}


def stress_correction(y, a, b):
    """Eq. 14 with walls at 0 and 1."""
    y = np.asarray(y, np.float64)
    s = np.zeros_like(y)
    for al, bl in zip(a, b):
        s += al * (np.exp(-bl * y) - np.exp(-bl * (1.0 - y)))
    return s


def cfd(Kn: float, F: float, n: int, sigma_p=None, a=(), b=()):
    """Cell-centred finite-volume solve of Eq. 8 on n cells: for each cell,
    (flux at the upper face - flux at the lower face) = h (-sqrt(pi) F / Kn) with the
    flux du/dy - S at the face; wall values by Eqs. 9-10 with P(0) = -F, P(1) = F
    through ghost cells.  Dense solve (small n)."""
    h = 1.0 / n
    yf = np.arange(n + 1) * h
    S = stress_correction(yf, a, b)
    uw = 0.0 if sigma_p is None else sigma_p * F  # -sigma_P P(0) = sigma_P P(1) = sigma_P F
    A = np.zeros((n, n))
    r = np.full(n, -h * SQRT_PI * F / Kn)
    for i in range(n):
        # upper face
        if i < n - 1:
            A[i, i + 1] += 1.0 / h
            A[i, i] -= 1.0 / h
        else:  # wall at distance h/2
            A[i, i] -= 2.0 / h
            r[i] -= 2.0 * uw / h
        r[i] += S[i + 1]
        # lower face
        if i > 0:
            A[i, i] -= 1.0 / h
            A[i, i - 1] += 1.0 / h
        else:
            A[i, i] -= 2.0 / h
            r[i] -= 2.0 * uw / h
        r[i] -= S[i]
    return np.linalg.solve(A, r)


def exact_profile(Kn: float, F: float, y, sigma_p=None, a=(), b=()):
    """Closed form of Eq. 8 with Eqs. 9-10: u = u_w + sqrt(pi) F y (1 - y) / (2 Kn)
    + integral_0^y S (S is odd about y = 1/2, so du/dy - S vanishes at the centre)."""
    y = np.asarray(y, np.float64)
    uw = 0.0 if sigma_p is None else sigma_p * F
    u = uw + SQRT_PI * F * y * (1.0 - y) / (2.0 * Kn)
    for al, bl in zip(a, b):
        u += al * ((1.0 - np.exp(-bl * y)) / bl - (np.exp(-bl * (1.0 - y)) - np.exp(-bl)) / bl)
    return u


def mc_profiles(fit, Kn: float, F: float, n: int, b, z):
    """Monte Carlo trials (Sec. 2.3): weights of the selected models drawn from their
    posteriors, w = m + L z with S = L L^T (Cholesky), one CFD solve per trial.  z has
    one row of four standard normals per trial (slip coefficient, a_1..a_3); returns the
    mean profile, the per-cell standard deviation and the profiles."""
    z = np.asarray(z, np.float64)
    sel_v, sel_c = fit["sel_v"], fit["sel_c"]
    out = []
    for row in z:
        sp = None
        if sel_v == 1:
            fv = fit["v"][1]
            sp = float(fv["m"][0] + math.sqrt(fv["S"][0, 0]) * row[0])
        a = ()
        if sel_c >= 1:
            fc = fit["c"][sel_c]
            L = np.linalg.cholesky(fc["S"])
            a = tuple(fc["m"] + L @ row[1:1 + sel_c])
        out.append(cfd(Kn, F, n, sp, a, b[:len(a)]))
    out = np.array(out)
    return out.mean(axis=0), out.std(axis=0, ddof=1) if len(out) > 1 else np.zeros(n), out


def selected_profile(fit, Kn: float, F: float, n: int, b):
    """The CFD profile with the posterior means of the selected models."""
    sp = float(fit["v"][1]["m"][0]) if fit["sel_v"] == 1 else None
    a = tuple(fit["c"][fit["sel_c"]]["m"]) if fit["sel_c"] >= 1 else ()
    return cfd(Kn, F, n, sp, a, b[:len(a)])
