"""Reweighted direct sampling on the GPU (App. A, Eqs. A2-A7) through the C ABI against the
FP64 oracle: the same samples and log q for the same uniforms (exact and truncating chi,
odd double-layer bonds, ragged chain counts), the p = 0 SR step and observables against the
oracle's on the same draws, the histogram of Philox-driven draws against q, and the Eq. A7
energy estimate against the exact average on a lattice small enough to enumerate."""
import numpy as np
import pytest
from scipy import stats

from oracle import direct, ed, peps, sr, observables as obs_mod
from oracle.lattice import Lattice
from paper_2409_05285_gb300 import binding
from paper_2409_05285_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2409_05285_gb300.build import build
    build()


def _ctx(L1, L2, D, chi, n, prec=binding.PEPS_FP64, seed=0, J2=0.0):
    return binding.Context(L1, L2, D, chi, n, J1=1.0, J2=J2, precision=prec, seed=seed,
                           block_mode=binding.PEPS_BLOCKS_BATCHED)


def _all_configs(N):
    return np.array([ed.config_of_index(k, N) for k in range(4 ** N)])


CASES = [  # (L1, L2, D, chi, b_d, exponent, n): exact chi, truncating chi, D^2 = 9, ragged n
    (2, 3, 2, 16, 1.0, 1.0, 9),
    (3, 3, 2, 16, 0.4, 0.5, 24),
    (3, 3, 2, 4, 0.6, 0.5, 13),
    (3, 4, 2, 6, 1.0, 0.5, 11),
    (4, 4, 2, 8, 0.5, 0.5, 37),
    (3, 3, 3, 9, 0.7, 0.5, 6),
]


@pytest.mark.parametrize("case", CASES)
def test_fp64_draws_match_oracle(case):
    # FP64 engine: the drawn states are integer decisions taken from float64 candidate sums
    # on both sides; they agree exactly unless a uniform falls within rounding of a CDF edge
    # (none does for these seeds), and log q agrees to 1e-9 relative
    L1, L2, D, chi, b_d, expo, n = case
    lat = Lattice(L1, L2, D)
    th = wl.random_theta(L1, L2, D, seed=L1 * 7 + L2 + D, scale=0.4, diag_bias=1.0)
    u = np.random.default_rng(L1 + 10 * L2 + chi).random((n, lat.N))
    ctx = _ctx(L1, L2, D, chi, n)
    ctx.set_theta(th)
    lq = ctx.direct_draw(u, b_d, expo)
    S = ctx.get_configs()
    down = direct.summed_down_envs(lat, th, chi)
    for k in range(n):
        So, lqo = direct.draw_bmps(lat, th, u[k], chi, b_d, expo, down=down)
        assert np.array_equal(S[k], So), k
        assert lq[k] == pytest.approx(lqo, rel=1e-9, abs=1e-11), k
    ctx.close()


def test_draws_at_the_bench_size():
    # the bench's geometry and launch configuration (6x6, D=2, chi=16, 30000 chains, TF32,
    # host uniforms): sampled chains against the oracle's boundary-MPS draws for the same
    # uniforms, and the FP64 engine on the first 256 of those chains.  Here chi = 16 cuts the
    # double layer's boundary bonds (exact: 64) through close singular values, so log q is
    # ill-conditioned for any implementation: the oracle's own log q moves by up to 2e-3 when
    # theta is perturbed by 1e-13 relative.  The bound on |d log q| is 5e-3 for FP64 and 3e-2
    # for TF32 (36 sites, each a ratio of candidate sums carrying ~1e-3 TF32 rounding); a
    # draw may differ where a uniform sits that close to a CDF edge.
    L, D, chi, n = 6, 2, 16, 30000
    lat = Lattice(L, L, D)
    th = wl.random_theta(L, L, D, seed=61, scale=0.4, diag_bias=1.0)
    u = np.random.default_rng(62).random((n, lat.N))
    ctx = _ctx(L, L, D, chi, n, prec=binding.PEPS_TF32)
    ctx.set_theta(th)
    lq = ctx.direct_draw(u, 0.6, 0.5)
    S = ctx.get_configs()
    ctx.close()
    ref = _ctx(L, L, D, chi, 256)
    ref.set_theta(th)
    lq64 = ref.direct_draw(u[:256], 0.6, 0.5)
    S64 = ref.get_configs()
    ref.close()
    down = direct.summed_down_envs(lat, th, chi)
    picks = [0, 1, 2, 3, 255, 4097, 17000, n - 1]
    agree, agree64 = 0, 0
    for k in picks:
        So, lqo = direct.draw_bmps(lat, th, u[k], chi, 0.6, 0.5, down=down)
        if k < 256 and np.array_equal(S64[k], So):
            agree64 += 1
            assert abs(lq64[k] - lqo) <= 5e-3, k
        if np.array_equal(S[k], So):
            agree += 1
            assert abs(lq[k] - lqo) <= 3e-2, k
    assert agree64 >= 4 and agree >= len(picks) - 1
    assert np.mean(np.all(S[:256] == S64, axis=1)) >= 0.9
    counts = np.bincount(S.ravel(), minlength=4)
    assert np.all(counts > 0)   # every local state, s = s' and s != s', is drawn


@pytest.mark.parametrize("prec", [binding.PEPS_FP32, binding.PEPS_TF32])
def test_float_draws_follow_their_own_q(prec):
    # float engines: each draw is a valid state whose log q matches the oracle's exact q of
    # that state (chi exact here) to float accuracy, and most draws equal the FP64 ones
    L1, L2, D, chi, b_d, expo, n = 3, 3, 2, 16, 0.5, 0.5, 64
    lat = Lattice(L1, L2, D)
    th = wl.random_theta(L1, L2, D, seed=5, scale=0.4, diag_bias=1.0)
    u = np.random.default_rng(6).random((n, lat.N))
    ref = _ctx(L1, L2, D, chi, n)
    ref.set_theta(th)
    ref.direct_draw(u, b_d, expo)
    S64 = ref.get_configs()
    ctx = _ctx(L1, L2, D, chi, n, prec=prec)
    ctx.set_theta(th)
    lq = ctx.direct_draw(u, b_d, expo)
    S = ctx.get_configs()
    assert S.max() <= 3
    same = np.all(S == S64, axis=1)
    assert same.mean() >= 0.9
    for k in range(n):
        q = direct.sample_prob(lat, th, S[k], b_d, expo)
        assert q > 0
        assert abs(lq[k] - np.log(q)) <= 5e-3 * max(1.0, abs(np.log(q))), k
    ref.close()
    ctx.close()


def test_sr_step_and_observables_on_direct_draws_match_oracle():
    # p = 0 weights r_4 = rho^2 / q (Eq. A7) in the SR step: the update, E, C, chi and the
    # standard error against the oracle's SR step and observables on the same draws
    L1, L2, D, chi, n = 3, 3, 2, 16, 48
    lat = Lattice(L1, L2, D, J1=1.0)
    th = wl.random_theta(L1, L2, D, seed=41, scale=0.3, diag_bias=1.0)
    u = np.random.default_rng(42).random((n, lat.N))
    ctx = _ctx(L1, L2, D, chi, n)
    tau0 = 0.25
    ctx.eval_chains()
    ctx.sr_step(tau0, eps=1e-2, max_cg=5, cg_tol=1e-6, p=2)   # beta_obs = 4 tau0 below
    ctx.set_theta(th)
    lq = ctx.direct_draw(u, b_d=0.5, exponent=0.5)
    S = ctx.get_configs()
    ctx.eval_chains()
    o_gpu = ctx.observables(p=0)
    tau, eps, tol = 0.05, 1e-3, 1e-12
    st = ctx.sr_step(tau, eps=eps, max_cg=500, cg_tol=tol, p=0)
    th_gpu = ctx.get_theta()
    res = [peps.eval_sample(lat, th, S[k], chi) for k in range(n)]
    la = np.array([r['log_abs'] for r in res])
    es = np.array([r['e_sys'] for r in res])
    ea = np.array([r['e_anc'] for r in res])
    O = np.array([r['O'] for r in res])
    _, x, g, it, _ = sr.sr_step(lat, th, S, la, es, ea, O, 0, tau, eps, tol, 500, log_q=lq)
    w = sr.weights(la, 0, lq)
    assert not np.allclose(w, w[0])
    Of = sr.expand_O(lat, S, O)
    obar, _, _ = sr.sr_quantities(Of, w, es + ea)
    xd = np.linalg.solve(sr.dense_G(Of, w, obar, eps), g)
    x_gpu = (th - th_gpu) / tau
    assert np.max(np.abs(x_gpu - xd)) <= 1e-8 * np.max(np.abs(xd))
    assert np.max(np.abs(x_gpu - x)) <= 1e-8 * np.max(np.abs(xd))
    assert st['cg_resid'] <= tol and abs(st['cg_iters'] - it) <= 2
    o = obs_mod.observables(lat, tau0, w, es, ea, S)
    for d in (o_gpu, st):
        assert d['p'] == 0
        assert d['E_site'] == pytest.approx(o['E_site'], rel=1e-10, abs=1e-12)
        assert d['C_site'] == pytest.approx(o['C_site'], rel=1e-10)
        assert d['chi_sus'] == pytest.approx(o['chi'], rel=1e-10)
        assert d['E_err'] == pytest.approx(o['E_err'], rel=1e-10)
        assert d['diag_frac'] == pytest.approx(o['diag_frac'])
    ctx.close()


def test_philox_draws_follow_q_and_estimate_the_exact_energy():
    # 2x2, D=2, chi exact: the histogram of draws with the library's own uniforms follows q
    # (chi^2), and the Eq. A7 estimate of <H> equals the exact p_0 average within 5 standard
    # errors; the same seed repeats the draws, the next call draws new ones
    L1, L2, D, chi, n, b_d = 2, 2, 2, 4, 20000, 0.4
    lat = Lattice(L1, L2, D, J1=1.0)
    th = wl.random_theta(L1, L2, D, seed=51, scale=0.5, diag_bias=1.0)
    cfgs = _all_configs(lat.N)
    res = [peps.eval_sample(lat, th, S, chi) for S in cfgs]
    p0 = np.array([np.exp(2 * r['log_abs']) if r['sign'] != 0 else 0.0 for r in res])
    h = np.array([0.5 * (r['e_sys'] + r['e_anc']) for r in res])
    exact = np.sum(p0 * h) / p0.sum() / lat.N
    q = np.array([direct.sample_prob(lat, th, S, b_d, 0.5) for S in cfgs])
    ctx = _ctx(L1, L2, D, chi, n, seed=7)
    ctx.set_theta(th)
    lq = ctx.direct_draw(None, b_d, 0.5)
    S = ctx.get_configs()
    idx = (S.astype(np.int64) * (4 ** np.arange(lat.N - 1, -1, -1))).sum(axis=1)
    assert np.allclose(lq, np.log(q[idx]), rtol=1e-9, atol=1e-12)
    counts = np.bincount(idx, minlength=len(cfgs))
    keep = q * n >= 5
    obs = np.append(counts[keep], counts[~keep].sum())
    exp = np.append(q[keep] * n, q[~keep].sum() * n)
    exp *= obs.sum() / exp.sum()
    assert stats.chisquare(obs, exp).pvalue > 1e-3
    ctx.eval_chains()
    o = ctx.observables(p=0)
    assert abs(o['E_site'] - exact) <= 5 * o['E_err'] + 1e-12
    again = _ctx(L1, L2, D, chi, n, seed=7)
    again.set_theta(th)
    assert np.array_equal(again.direct_draw(None, b_d, 0.5), lq)
    assert np.array_equal(again.get_configs(), S)
    again.direct_draw(None, b_d, 0.5)
    assert not np.array_equal(again.get_configs(), S)
    ctx.close()
    again.close()


def test_direct_step_cools_and_adapts_b_d():
    # whole steps on direct draws: theta moves, t advances, E stays finite, and b_d follows
    # the rule of peps_direct_next_bd (never above 1, lowered while diagonal terms dominate)
    L1, L2, D, chi, n = 3, 3, 2, 8, 512
    ctx = _ctx(L1, L2, D, chi, n, seed=3)
    b_d = 1.0
    th0 = ctx.get_theta()
    for k in range(3):
        st, b_next = ctx.direct_step(b_d, exponent=0.5, tau=0.02, eps=1e-3, max_cg=50,
                                     cg_tol=1e-8)
        assert st['p'] == 0 and np.isfinite(st['E_site'])
        assert b_next == pytest.approx(binding.direct_next_bd(b_d, st['diag_frac'], L1 * L2))
        assert 0 < b_next <= 1.0
        b_d = b_next
    assert st['t'] == pytest.approx(0.04)   # the samples of the third step, before its update
    assert ctx.t == pytest.approx(0.06)
    assert not np.array_equal(ctx.get_theta(), th0)
    ctx.close()


def test_direct_errors():
    ctx = _ctx(3, 3, 2, 4, 8)
    with pytest.raises(binding.PepsError) as e:
        ctx.direct_draw(None, b_d=0.0)
    assert e.value.code == binding.PEPS_EINVAL
    with pytest.raises(binding.PepsError) as e:
        ctx.direct_draw(None, b_d=1.5)
    assert e.value.code == binding.PEPS_EINVAL
    with pytest.raises(binding.PepsError) as e:
        ctx.direct_draw(None, exponent=-1.0)
    assert e.value.code == binding.PEPS_EINVAL
    ctx.eval_chains()
    with pytest.raises(binding.PepsError) as e:   # chains not from a direct draw
        ctx.sr_step(0.01, p=0)
    assert e.value.code == binding.PEPS_ESTATE
    ctx.direct_draw(None)
    ctx.mc_sweep(1, p=2)
    ctx.eval_chains()
    with pytest.raises(binding.PepsError) as e:   # a sweep moved the chains since
        ctx.observables(p=0)
    assert e.value.code == binding.PEPS_ESTATE
    ctx.direct_draw(None)
    ctx.eval_chains()
    ctx.sr_step(0.01, p=0)
    ctx.eval_chains()
    with pytest.raises(binding.PepsError) as e:   # theta changed since the draw
        ctx.sr_step(0.01, p=0)
    assert e.value.code == binding.PEPS_ESTATE
    ctx.close()
    narrow = binding.Context(3, 3, 2, 4, 8, block_mode=binding.PEPS_BLOCKS_NARROW)
    with pytest.raises(binding.PepsError) as e:
        narrow.direct_draw(None)
    assert e.value.code == binding.PEPS_ESTATE
    narrow.close()
