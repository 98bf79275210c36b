"""Thermal observables from one batch of samples (Sec. II Eq. 11, Sec. III.A Eq. 13).

TEST INFRASTRUCTURE (oracle): see oracle/__init__.py.

After a total imaginary time t = sum of the SR steps tau, the PEPS approximates
e^{-t calH}|I> = |rho_beta> with beta = 2t (Eq. 3), and Eq. 11 gives the internal energy
of the thermal state at inverse temperature 2 beta = 4t, which is beta_obs here.  That
state is (rho rho^T + rho^T rho) / (2 Tr rho rho^T); with w_i the sample weights:
  <H>   = 1/2 sum_i w_i (E_sys,i + E_anc,i)                (Eq. 11)
  <H^2> = 1/2 sum_i w_i (E_sys,i^2 + E_anc,i^2)             (||H rho||^2 = sum |rho|^2 E_sys^2)
  C/N   = beta_obs^2 (<H^2> - <H>^2) / N
  <Mz^2>= 1/2 sum_i w_i (M(s_i)^2 + M(s'_i)^2),  chi = beta_obs <Mz^2> / N, <Mz>^2 := 0 (Eq. 13)

The paper's own C_v (Sec. III.A) is the derivative of a B-spline fitted to E(beta):
cv_from_energy_curve, a post-processing cross-check of the fluctuation estimate above.
"""
import numpy as np

from .lattice import spin_anc, spin_sys, sz_of


def observables(lat, t, w, e_sys, e_anc, S_batch):
    beta_obs = 4.0 * t
    w = np.asarray(w, dtype=np.float64)
    es, ea = np.asarray(e_sys), np.asarray(e_anc)
    H1 = 0.5 * float(w @ (es + ea))
    H2 = 0.5 * float(w @ (es * es + ea * ea))
    S_batch = np.asarray(S_batch)
    Ms = np.sum(sz_of(spin_sys(S_batch)), axis=1)
    Ma = np.sum(sz_of(spin_anc(S_batch)), axis=1)
    M2 = 0.5 * float(w @ (Ms * Ms + Ma * Ma))
    N = lat.N
    diag = np.all(spin_sys(S_batch) == spin_anc(S_batch), axis=1)
    return dict(t=t, beta_obs=beta_obs, E_site=H1 / N, C_site=beta_obs ** 2 * (H2 - H1 * H1) / N,
                chi=beta_obs * M2 / N, Mz2=M2, diag_frac=float(np.mean(diag)))


def cv_from_energy_curve(betas, E_site, smoothing=0.0, k=3):
    """Specific heat per site from a curve of E/N against beta_obs (Sec. III.A, Fig. 2b):
    a B-spline of degree k fitted to the points (smoothing factor `smoothing`, 0 for
    interpolation), then C/N = dE/dT = -beta^2 dE/dbeta from the spline's derivative.
    Returns a function of beta."""
    from scipy.interpolate import UnivariateSpline
    betas = np.asarray(betas, dtype=np.float64)
    order = np.argsort(betas)
    spl = UnivariateSpline(betas[order], np.asarray(E_site, dtype=np.float64)[order], k=k,
                           s=smoothing)
    dE = spl.derivative()
    return lambda b: -np.asarray(b, dtype=np.float64) ** 2 * dE(b)


def cv_from_energy_gpr(betas, E_site, noise=1e-8, length=None):
    """Specific heat per site from E/N against beta by Gaussian-process regression (the
    scheme named for the Hubbard data, Sec. III.B): a GP with the squared-exponential kernel
    k(b, b') = s^2 exp(-(b - b')^2 / (2 l^2)) around the data mean, noise variance `noise`
    (the variance of the E/N errors), s^2 the data variance, and the length scale l given or
    chosen on a grid by the largest log marginal likelihood; the posterior mean's derivative
    is analytic, and C/N = -beta^2 dE/dbeta.  Returns a function of beta."""
    b = np.asarray(betas, dtype=np.float64)
    y = np.asarray(E_site, dtype=np.float64)
    m = y.mean()
    s2 = max(float(np.var(y)), 1e-12)
    r = y - m

    def fit(l):
        K = s2 * np.exp(-(b[:, None] - b[None, :]) ** 2 / (2 * l * l)) + noise * np.eye(len(b))
        L = np.linalg.cholesky(K)
        a = np.linalg.solve(L.T, np.linalg.solve(L, r))
        return a, -0.5 * r @ a - np.sum(np.log(np.diag(L)))

    if length is None:
        span = b.max() - b.min()
        best = None
        for l in span * np.logspace(-2, 0, 25):
            try:
                a, lml = fit(l)
            except np.linalg.LinAlgError:
                continue
            if best is None or lml > best[2]:
                best = (l, a, lml)
        length, alpha = best[0], best[1]
    else:
        alpha = fit(length)[0]

    def cv(q):
        q = np.atleast_1d(np.asarray(q, dtype=np.float64))
        d = q[:, None] - b[None, :]
        dk = -d / length ** 2 * s2 * np.exp(-d ** 2 / (2 * length ** 2))
        return -q ** 2 * (dk @ alpha)
    return cv
