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

Standard error of <H> (the paper states none; this is the reading used): with
h_i = (E_sys,i + E_anc,i)/2 the per-sample energy of Eq. 11, the estimate <H> = sum_i w_i h_i
is a self-normalised weighted mean, and for independent samples its first-order (delta
method) variance is sum_i w_i^2 (h_i - <H>)^2.  For p = 2 (w_i = 1/n) that is the plain
sigma/sqrt(n) with the population variance; for p = 1 (w_i = |rho_i| / sum |rho|, Eq. A1)
it is the standard error of a ratio estimate.  Correlations between successive samples of
a chain are not included: every chain contributes one sample per step.

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
    E_err = standard_error(w, 0.5 * (es + ea))
    return dict(t=t, beta_obs=beta_obs, E_site=H1 / N, E_err=E_err / N,
                C_site=beta_obs ** 2 * (H2 - H1 * H1) / N,
                chi=beta_obs * M2 / N, Mz2=M2, diag_frac=float(np.mean(diag)))


def standard_error(w, h):
    """Standard error of the weighted mean sum_i w_i h_i (weights summing to one) from
    independent samples: sqrt(sum_i w_i^2 (h_i - mean)^2), the first-order variance of a
    self-normalised estimate (reading stated in the module docstring)."""
    w = np.asarray(w, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    mean = float(w @ h)
    return float(np.sqrt(np.sum(w * w * (h - mean) ** 2)))


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
