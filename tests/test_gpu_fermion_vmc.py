"""Fermionic sampling and SR on the GPU (peps_famp_sweep, peps_famp_sr_step; Sec. II MCMC and
Eqs. 5-10 on the fermionic PEPS of Fig. 1b, Hubbard model of Sec. III.B) through the C ABI
against the oracle: Metropolis sweeps with the same Philox uniforms (configurations and
acceptance counts bit for bit), the SR update of theta and the observables (FP64 to rounding,
FP32 within a bound), argument and configuration errors, and a short cooling run of 2x2 against
exact imaginary-time evolution."""
import functools

import numpy as np
import pytest

from oracle import fermion as fm
from oracle import fermion_vmc as fv
from paper_2409_05285_gb300 import binding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2409_05285_gb300.build import build
    build()


def _flat(T):
    return np.concatenate([t.ravel() for t in T])


def _oracle_amp(nr, nc, T):
    # the oracle's amplitude (configuration sign times the plain contraction of the signed
    # slices), remembered per configuration
    return functools.lru_cache(maxsize=None)(fm.fpeps_amplitude_function(nr, nc, T))


def _near_identity(nr, nc, D, rng, noise):
    T = fm.random_even_fpeps(nr, nc, D, rng, scale=noise)
    for i, A in enumerate(fm.identity_fpeps(nr, nc)):
        T[i][(slice(None), 0, 0, 0, 0)] += A[:, 0, 0, 0, 0]
    return T


def _support_configs(nb, N, rng):
    # configurations of the |I> support: system and ancilla occupations equal per site
    a = rng.integers(0, 4, (nb, N))
    return (a | (a << 2)).astype(np.uint8)


def _oracle_sweeps(nr, nc, T, S, p, n_sweeps, seed, sweep0, u=None):
    amp = _oracle_amp(nr, nc, T)
    M = len(fv.moves(nr, nc))
    out, acc, margin = [], [], np.inf
    for c in range(len(S)):
        x = S[c]
        a = 0
        for k in range(n_sweeps):
            uk = fv.uniforms(seed, c, sweep0 + k, M) if u is None else u[k, c]
            x, ak, mg = fv.sweep(nr, nc, T, x, p, uk, amplitude=lambda X: amp(tuple(int(v) for v in X)))
            a += ak
            margin = min(margin, mg)
        out.append(x)
        acc.append(a)
    return np.array(out), np.array(acc), margin


@pytest.mark.parametrize("shape,p", [((2, 2, 2, 8), 2), ((3, 3, 2, 8), 2), ((3, 3, 2, 8), 1)])
def test_sweeps_match_oracle_with_philox(shape, p):
    nr, nc, D, chi = shape
    rng = np.random.default_rng(nr * 10 + p)
    T = _near_identity(nr, nc, D, rng, 0.4)
    S0 = _support_configs(12, nr * nc, rng)
    f = binding.FermionAmplitudes(nr, nc, D, chi, 12, precision=binding.PEPS_FP64)
    assert f.n_moves == len(fv.moves(nr, nc))
    S, acc, la, sg = f.sweep(_flat(T), S0, p=p, n_sweeps=2, seed=77, sweep0=5)
    S_ref, acc_ref, margin = _oracle_sweeps(nr, nc, T, S0, p, 2, 77, 5)
    assert margin > 1e-8                 # no decision within rounding of its threshold
    assert np.array_equal(S, S_ref)
    assert np.array_equal(acc, acc_ref)
    assert acc.sum() > 0 and not np.array_equal(S, S0)
    for k in range(len(S)):
        ref = fm.fpeps_amplitude_bosonic(nr, nc, T, S[k])
        assert sg[k] == np.sign(ref) and abs(la[k] - np.log(abs(ref))) < 1e-10
    f.close()


def test_sweeps_with_given_uniforms_and_sector():
    nr, nc, D, chi = 2, 3, 2, 8
    rng = np.random.default_rng(8)
    T = _near_identity(nr, nc, D, rng, 0.5)
    S0 = _support_configs(10, nr * nc, rng)
    f = binding.FermionAmplitudes(nr, nc, D, chi, 10, precision=binding.PEPS_FP64)
    u = rng.random((3, 10, f.n_moves))
    S, acc, _, _ = f.sweep(_flat(T), S0, p=2, n_sweeps=3, u=u)
    S_ref, acc_ref, margin = _oracle_sweeps(nr, nc, T, S0, 2, 3, 0, 0, u=u)
    assert margin > 1e-8
    assert np.array_equal(S, S_ref) and np.array_equal(acc, acc_ref)
    # N_s(c) = N_s(d) for both spins (the moves keep the difference)
    for x in S:
        n = [sum((int(v) >> k) & 1 for v in x) for k in range(4)]
        assert n[0] == n[2] and n[1] == n[3]
    f.close()


def test_sweep_and_sr_errors():
    nr, nc, D, chi = 2, 2, 2, 8
    rng = np.random.default_rng(1)
    T = _near_identity(nr, nc, D, rng, 0.3)
    f = binding.FermionAmplitudes(nr, nc, D, chi, 4, precision=binding.PEPS_FP64)
    S = _support_configs(4, 4, rng)
    with pytest.raises(binding.PepsError) as e:
        f.sweep(_flat(T), S, p=3)
    assert e.value.code == binding.PEPS_EINVAL
    bad = S.copy()
    bad[1, 2] = 16
    with pytest.raises(binding.PepsError) as e:
        f.sweep(_flat(T), bad)
    assert e.value.code == binding.PEPS_EINVAL
    odd = S.copy()
    odd[0, 0] ^= 1                       # odd total parity: psi = 0
    with pytest.raises(binding.PepsError) as e:
        f.sr_step(_flat(T), odd, 1.0, 8.0, 4.0)
    assert e.value.code == binding.PEPS_EINVAL
    with pytest.raises(binding.PepsError):
        f.sr_step(_flat(T), S, 1.0, 8.0, 4.0, p=0)
    # n_sweeps = 0 leaves the chains and reports their amplitudes
    S2, acc, la, sg = f.sweep(_flat(T), S, n_sweeps=0)
    assert np.array_equal(S2, S) and not acc.any() and np.all(sg != 0)
    f.close()


def _sr_case(nr, nc, D, nb, seed):
    rng = np.random.default_rng(seed)
    T = _near_identity(nr, nc, D, rng, 0.4)
    S0 = _support_configs(nb, nr * nc, rng)
    return T, S0


@pytest.mark.parametrize("shape,p", [((2, 2, 2, 8, 24), 2), ((2, 2, 2, 8, 24), 1), ((3, 3, 2, 8, 12), 2)])
def test_sr_step_matches_oracle_fp64(shape, p):
    nr, nc, D, chi, nb = shape
    T, S0 = _sr_case(nr, nc, D, nb, 40 + p)
    t_hop, U, mu, tau, eps = 1.0, 8.0, 4.0, 0.02, 1e-3
    f = binding.FermionAmplitudes(nr, nc, D, chi, nb, precision=binding.PEPS_FP64)
    S, _, _, _ = f.sweep(_flat(T), S0, p=p, n_sweeps=2, seed=3)
    th, st = f.sr_step(_flat(T), S, t_hop, U, mu, p=p, tau=tau, eps=eps, max_cg=400, cg_tol=1e-12)
    T_ref, x_ref, g_ref, it, res, obs = fv.sr_step(nr, nc, T, S, t_hop, U, mu, p, tau, eps, 1e-12, 400)
    x = (_flat(T) - th) / tau
    assert np.max(np.abs(x - x_ref)) <= 1e-6 * np.max(np.abs(x_ref))
    assert np.max(np.abs(th - _flat(T_ref))) <= 1e-8
    for k in ("E_site", "E_err", "docc", "density"):
        assert st[k] == pytest.approx(obs[k], rel=1e-10, abs=1e-12), k
    assert abs(st["cg_iters"] - it) <= 2 and st["cg_resid"] <= 1e-12
    f.close()


def test_sr_step_fp32_within_bound():
    nr, nc, D, chi, nb = 2, 2, 2, 8, 24
    T, S0 = _sr_case(nr, nc, D, nb, 52)
    f64 = binding.FermionAmplitudes(nr, nc, D, chi, nb, precision=binding.PEPS_FP64)
    S, _, _, _ = f64.sweep(_flat(T), S0, n_sweeps=2, seed=9)
    f32 = binding.FermionAmplitudes(nr, nc, D, chi, nb, precision=binding.PEPS_FP32)
    th, st = f32.sr_step(_flat(T), S, 1.0, 8.0, 4.0, tau=0.02, eps=1e-3, max_cg=400, cg_tol=1e-10)
    _, x_ref, _, _, _, obs = fv.sr_step(nr, nc, T, S, 1.0, 8.0, 4.0, 2, 0.02, 1e-3, 1e-12, 400)
    x = (_flat(T) - th) / 0.02
    # float32 amplitudes and O rows (relative rounding ~1e-6) through a CG of condition
    # number up to |G|/eps
    assert np.max(np.abs(x - x_ref)) <= 1e-2 * np.max(np.abs(x_ref))
    assert st["E_site"] == pytest.approx(obs["E_site"], abs=1e-4)
    f64.close()
    f32.close()


def test_short_cooling_run_tracks_exact_evolution():
    # 2x2 Hubbard (t = 1, U = 8, mu = 4) from |I> (D = 4, small even noise), 512 chains on
    # the GPU: sweeps and SR steps of tau = 0.01 to t = 0.04 (beta_obs = 0.16).  The energy
    # leaves its infinite-temperature value U/4 - mu = -2 and stays within statistical and
    # first-order-in-tau errors of exp(-t calH)|I>'s
    nr, nc, D, chi, nb = 2, 2, 4, 16, 512
    rng = np.random.default_rng(5)
    T = _near_identity(nr, nc, D, rng, 1e-3)
    th = _flat(T)
    S = _support_configs(nb, 4, rng)
    f = binding.FermionAmplitudes(nr, nc, D, chi, nb, precision=binding.PEPS_FP64)
    S, _, _, _ = f.sweep(th, S, n_sweeps=4, seed=1, sweep0=0)
    first = None
    for step in range(4):
        S, _, _, _ = f.sweep(th, S, n_sweeps=2, seed=1, sweep0=4 + 2 * step)
        th, st = f.sr_step(th, S, 1.0, 8.0, 4.0, tau=0.01, eps=1e-4, max_cg=200, cg_tol=1e-8)
        if first is None:
            first = st
    S, _, _, _ = f.sweep(th, S, n_sweeps=2, seed=1, sweep0=20)
    _, st = f.sr_step(th, S, 1.0, 8.0, 4.0, tau=0.0, eps=1e-4, max_cg=0)
    E_ref, docc_ref = fm.observables(nr, nc, 1.0, 8.0, 4.0, fm.evolve(nr, nc, 1.0, 8.0, 4.0, 0.04))
    assert abs(first["E_site"] + 2.0) < 5 * first["E_err"] + 1e-3
    assert abs(st["E_site"] - E_ref) < 5 * st["E_err"] + 0.05
    assert st["E_site"] < -2.0 and E_ref < -2.0
    assert abs(st["docc"] - docc_ref) < 0.05
    f.close()
