"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on the same seeded
inputs.  Tolerances: FP64 path, amplitudes 1e-10 relative (|d log rho| <= 1e-10), local
energies and O entries 1e-9 relative to their scale; FP32 path, 2e-4 relative."""
import numpy as np
import pytest

from oracle import peps, sampler, sr, observables as obs_mod
from oracle.lattice import Lattice
from paper_2409_05285_gb300 import binding
from paper_2409_05285_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2409_05285_gb300.build import build
    build()


def _ctx(L1, L2, D, chi, n, J2=0.0, prec=binding.PEPS_FP64, seed=0, noise=1e-3, n_blocks=0,
         mode=binding.PEPS_BLOCKS_AUTO):
    return binding.Context(L1, L2, D, chi, n, J1=1.0, J2=J2, precision=prec, init_noise=noise,
                           seed=seed, n_blocks=n_blocks, block_mode=mode)


def _compare_eval(lat, th, S, chi, got, tol_la, tol_e, tol_o):
    la, sg, es, ea, O = got
    for k in range(S.shape[0]):
        r = peps.eval_sample(lat, th, S[k], chi)
        assert sg[k] == r['sign'], k
        assert abs(la[k] - r['log_abs']) <= tol_la, (k, la[k], r['log_abs'])
        scale = max(1.0, abs(r['e_sys']), abs(r['e_anc']))
        assert abs(es[k] - r['e_sys']) <= tol_e * scale, (k, es[k], r['e_sys'])
        assert abs(ea[k] - r['e_anc']) <= tol_e * scale, (k, ea[k], r['e_anc'])
        oscale = max(1.0, np.max(np.abs(r['O'])))
        assert np.max(np.abs(O[k].astype(np.float64) - r['O'])) <= tol_o * oscale, k


CASES = [  # (L1, L2, D, chi, J2, n): exact chi, truncated chi, ragged tails, NNN bonds
    (2, 2, 2, 4, 0.0, 6),
    (4, 4, 2, 4, 0.0, 12),
    (3, 5, 2, 3, 0.5, 7),
    (4, 4, 3, 4, 0.5, 5),
    (5, 3, 3, 5, 0.2, 5),
]


MODES = [binding.PEPS_BLOCKS_NARROW, binding.PEPS_BLOCKS_WIDE, binding.PEPS_BLOCKS_BATCHED]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("case", CASES)
def test_eval_fp64_matches_oracle(case, mode):
    L1, L2, D, chi, J2, n = case
    lat = Lattice(L1, L2, D, J1=1.0, J2=J2)
    th = wl.random_theta(L1, L2, D, seed=L1 * 10 + L2, scale=0.3, diag_bias=1.0)
    S = wl.random_configs(L1, L2, n, seed=D)
    ctx = _ctx(L1, L2, D, chi, n, J2=J2, n_blocks=3, mode=mode)
    ctx.set_theta(th)
    _compare_eval(lat, th, S, chi, ctx.eval_batch(S), 1e-10, 1e-9, 1e-9)


@pytest.mark.parametrize("mode", [binding.PEPS_BLOCKS_NARROW, binding.PEPS_BLOCKS_BATCHED])
def test_eval_fp64_heis8_shape(mode):
    # 8x8, D=4, chi=16: the bench workload's contraction sizes (truncating chi), sampled rows.
    L, D, chi = 8, 4, 16
    lat = Lattice(L, L, D)
    th = wl.random_theta(L, L, D, seed=81, scale=0.2, diag_bias=1.0)
    S = wl.random_configs(L, L, 3, seed=82)
    ctx = _ctx(L, L, D, chi, 3, mode=mode)
    ctx.set_theta(th)
    _compare_eval(lat, th, S, chi, ctx.eval_batch(S), 1e-10, 1e-9, 1e-8)


@pytest.mark.parametrize("mode", MODES)
def test_eval_fp32_matches_oracle(mode):
    L1, L2, D, chi, J2 = 4, 4, 3, 4, 0.5
    lat = Lattice(L1, L2, D, J1=1.0, J2=J2)
    th = wl.random_theta(L1, L2, D, seed=5, scale=0.3, diag_bias=1.0)
    S = wl.random_configs(L1, L2, 6, seed=6)
    ctx = _ctx(L1, L2, D, chi, 6, J2=J2, prec=binding.PEPS_FP32, mode=mode)
    ctx.set_theta(th)
    _compare_eval(lat, th, S, chi, ctx.eval_batch(S), 2e-4, 2e-4, 2e-3)


@pytest.mark.parametrize("mode", MODES)
def test_eval_fp32_heis8_near_product_state(mode):
    # The bench workload's sizes in both block layouts, on a state near the beta=0 product
    # state (most singular values of the truncation below the float32 rounding floor).
    L, D, chi = 8, 4, 16
    lat = Lattice(L, L, D)
    th = wl.random_theta(L, L, D, seed=83, scale=0.05, diag_bias=1.0)
    S = wl.random_configs(L, L, 4, seed=84)
    ctx = _ctx(L, L, D, chi, 4, prec=binding.PEPS_FP32, mode=mode)
    ctx.set_theta(th)
    _compare_eval(lat, th, S, chi, ctx.eval_batch(S), 1e-3, 1e-3, 5e-3)


def test_eval_config_10x10_d6_chi36_spot_check():
    # The 10x10 J1-J2 workload's sizes (D=6, chi=36: absorbed bond 216, truncated to 36; the
    # batched engine's Jacobi matrices then live in global memory): two sampled
    # configurations against the oracle in FP64 on both engines (about 15 s of oracle time
    # each), then FP32 and TF32 against FP64 on eight.
    L, D, chi, J2 = 10, 6, 36, 0.5
    lat = Lattice(L, L, D, J1=1.0, J2=J2)
    th = wl.random_theta(L, L, D, seed=101, scale=0.1, diag_bias=1.0)
    S = wl.random_configs(L, L, 8, seed=102)
    ref = [peps.eval_sample(lat, th, S[k], chi) for k in range(2)]
    res = {}
    for name, prec, mode in (("narrow", binding.PEPS_FP64, binding.PEPS_BLOCKS_NARROW),
                             ("batched", binding.PEPS_FP64, binding.PEPS_BLOCKS_BATCHED),
                             ("fp32", binding.PEPS_FP32, binding.PEPS_BLOCKS_BATCHED),
                             ("tf32", binding.PEPS_TF32, binding.PEPS_BLOCKS_BATCHED)):
        ctx = _ctx(L, L, D, chi, 8, J2=J2, prec=prec, mode=mode)
        ctx.set_theta(th)
        res[name] = ctx.eval_batch(S, with_O=prec == binding.PEPS_FP64)
        ctx.close()
    for name in ("narrow", "batched"):
        la, sg, es, ea, O = res[name]
        for k in range(2):
            r = ref[k]
            assert sg[k] == r['sign'] and abs(la[k] - r['log_abs']) <= 1e-10, (name, k)
            scale = max(1.0, abs(r['e_sys']), abs(r['e_anc']))
            assert abs(es[k] - r['e_sys']) <= 1e-9 * scale and abs(ea[k] - r['e_anc']) <= 1e-9 * scale
            assert np.max(np.abs(O[k] - r['O'])) <= 1e-8 * max(1.0, np.max(np.abs(r['O'])))
    # Configurations with amplitudes e^-60 below the largest (the uniformly drawn half) are
    # beyond float32's resolution of the truncated environments and are never sampled; the
    # mixed-precision comparison takes the ones within e^-10 of the largest.
    la, sg, es, ea, _ = res["batched"]
    keep = la >= la.max() - 10.0
    assert keep.sum() >= 4
    scale = max(1.0, float(np.max(np.abs(es[keep]))), float(np.max(np.abs(ea[keep]))))
    for name, tol in (("fp32", 2e-3), ("tf32", 5e-2)):
        la2, sg2, es2, ea2, _ = res[name]
        assert np.all(sg2[keep] == sg[keep]), name
        assert np.max(np.abs(la2 - la)[keep]) <= tol, name
        assert np.max(np.abs(es2 - es)[keep]) <= tol * scale, name
        assert np.max(np.abs(ea2 - ea)[keep]) <= tol * scale, name


TF32_CASES = [  # sizes at which the transfer contractions reach the tensor-core path
    (6, 6, 4, 16, 0.0, 8),
    (4, 5, 4, 12, 0.5, 6),
]


@pytest.mark.parametrize("case", TF32_CASES)
def test_eval_tf32_matches_oracle(case):
    # TF32 operands carry 11 significant bits (unit roundoff u = 2^-11 after round-to-
    # nearest); an amplitude is a chain of ~2 L1 L2 contractions, each adding up to
    # u sqrt(K) relative error: ~0.16 in log abs(rho) if every error added up (4x5, K <= 64),
    # ~2e-2 as a random walk, which is what is seen (max 2.03e-2).  Tolerance 5e-2 for
    # log abs(rho), E_loc and O.  Random parameters of scale 0.2 give amplitudes that are
    # sums of cancelling terms, which amplify these errors (E_anc off by 3.8 % seen), so the
    # states here are of scale 0.1.
    L1, L2, D, chi, J2, n = case
    lat = Lattice(L1, L2, D, J1=1.0, J2=J2)
    th = wl.random_theta(L1, L2, D, seed=L1 * 7 + L2, scale=0.1, diag_bias=1.0)
    S = wl.random_configs(L1, L2, n, seed=D + 11)
    ctx = _ctx(L1, L2, D, chi, n, J2=J2, prec=binding.PEPS_TF32)
    ctx.set_theta(th)
    _compare_eval(lat, th, S, chi, ctx.eval_batch(S), 5e-2, 5e-2, 5e-2)


def test_tf32_energy_per_site_within_1e3_of_fp64():
    # The mixed-precision bound at the bench workload's sizes, on a cooled state (four SR
    # steps of tau = 0.1 from beta = 0 in FP64): local energy per site of the TF32 path
    # against the FP64 path on the same parameters and configurations.
    L, D, chi, n = 8, 4, 16, 64
    ref = _ctx(L, L, D, chi, n, prec=binding.PEPS_FP64, seed=3, mode=binding.PEPS_BLOCKS_BATCHED)
    ref.mc_sweep(2, p=1)
    for _ in range(4):
        ref.step(n_sweeps=1, p=2, tau=0.1, eps=1e-4, max_cg=100, cg_tol=1e-10)
    th, S = ref.get_theta(), ref.get_configs()
    la64, sg64, es, ea, _ = ref.eval_batch(S, with_O=False)
    e64 = es + ea
    tf = _ctx(L, L, D, chi, n, prec=binding.PEPS_TF32, seed=3)
    tf.set_theta(th)
    la32, sg32, es, ea, _ = tf.eval_batch(S, with_O=False)
    e32 = es + ea
    N = L * L
    assert np.all(sg64 == sg32)
    assert np.max(np.abs(la64 - la32)) <= 1e-1
    assert abs(np.mean(e64) - np.mean(e32)) / (2 * N) <= 1e-3
    assert np.max(np.abs(e64 - e32)) / (2 * N) <= 1e-3


def _sampled_configs(th, L, D, chi, n, seed, sweeps):
    """Configurations typical of |rho|^2: FP64 Metropolis chains after `sweeps` sweeps."""
    ref = _ctx(L, L, D, chi, n, prec=binding.PEPS_FP64, seed=seed, mode=binding.PEPS_BLOCKS_BATCHED)
    ref.set_theta(th)
    ref.mc_sweep(sweeps, p=2)
    return ref


def _tf32_vs_fp64(th, L, D, chi, n, seed):
    """TF32 against FP64 on configurations drawn from |rho|^2 by FP64 chains; also the FP64
    amplitudes at 2 chi (how far chi resolves each amplitude)."""
    N = L * L
    ref = _sampled_configs(th, L, D, chi, n, seed=seed, sweeps=3)
    S = ref.get_configs()
    la64, sg64, es64, ea64, _ = ref.eval_batch(S, with_O=False)
    wide = _ctx(L, L, D, 2 * chi, n, prec=binding.PEPS_FP64, seed=seed, mode=binding.PEPS_BLOCKS_BATCHED)
    wide.set_theta(th)
    lachi = wide.eval_batch(S, with_O=False)[0]
    tf = _ctx(L, L, D, chi, n, prec=binding.PEPS_TF32, seed=seed)
    tf.set_theta(th)
    la32, sg32, es32, ea32, _ = tf.eval_batch(S, with_O=False)
    dla = np.abs(la32 - la64)
    de = ((es32 + ea32) - (es64 + ea64)) / (2 * N)
    sens = np.abs(lachi - la64)
    print(f"\n8x8 D={D} chi={chi} TF32 vs FP64: chi-sensitivity median {np.median(sens):.2e}; "
          f"sign mismatches {int(np.sum(sg32 != sg64))}; |dlog rho| median {np.median(dla):.2e} "
          f"p90 {np.quantile(dla, 0.9):.2e} max {dla.max():.2e}; |dE_loc|/2N median "
          f"{np.median(np.abs(de)):.2e} max {np.abs(de).max():.2e}; dE/site {abs(de.mean()):.2e}")
    return sg32, sg64, dla, de, sens


def test_tf32_generic_state_8x8():
    # A generic state at the 8x8 D=4 chi=16 shape: entries of scale 0.3 and no diagonal bias.
    # chi = 16 does not resolve it: the FP64 amplitudes at chi = 16 and 32 differ by a median
    # of ~0.7 in log|rho|.  Where a truncation cuts through a nearly flat spectrum any
    # perturbation of the kept subspace moves the amplitude by a comparable amount (FP32 mode,
    # float32 without TF32 operands, shows outliers of the same kind), so per-sample bounds
    # there would test the truncation's conditioning, not the arithmetic.  Tolerances: TF32's
    # unit roundoff u = 2^-11 amplified by ~2 L^2 chained contractions gives ~1e-2 in
    # log|rho| (median bound 2e-2); signs agree on the samples that chi = 16 resolves (within
    # 0.1 of chi = 32) and on 99 % of all; every sample off by more than 0.1 is one that
    # chi = 16 leaves unresolved, its amplitude moving by more than 0.5 in log|rho| (five
    # times the resolution bound above) between chi = 16 and 32.
    L, D, chi, n = 8, 4, 16, 256
    th = wl.random_theta(L, L, D, seed=85, scale=0.3, diag_bias=0.0)
    sg32, sg64, dla, de, sens = _tf32_vs_fp64(th, L, D, chi, n, seed=86)
    assert np.median(dla) <= 2e-2
    assert np.all(sg32[sens <= 0.1] == sg64[sens <= 0.1])
    assert np.mean(sg32 != sg64) <= 0.01
    assert np.all(sens[dla > 0.1] > 0.5)


def test_tf32_resolved_state_8x8():
    # A random state that chi = 16 resolves: entries of scale 0.2 (twice the scale of the older
    # TF32 tests) on top of the beta = 0 product state (diagonal bias 1); the chi = 16 and
    # chi = 32 amplitudes differ by a median of ~1e-2.  Bounds: 5e-2 in log|rho| and in
    # E_loc/(2N) per sample, and the mean energy per site within 1e-3 of FP64 (the
    # mixed-precision bound).
    L, D, chi, n = 8, 4, 16, 256
    th = wl.random_theta(L, L, D, seed=85, scale=0.2, diag_bias=1.0)
    sg32, sg64, dla, de, sens = _tf32_vs_fp64(th, L, D, chi, n, seed=86)
    assert np.all(sg32 == sg64)
    assert dla.max() <= 5e-2
    assert np.abs(de).max() <= 5e-2
    assert abs(de.mean()) <= 1e-3


def test_tf32_metropolis_decisions_on_a_cooled_state():
    # Metropolis decisions on the same Philox stream: one sweep of every chain in TF32 and in
    # FP64 from the same configurations of a cooled 8x8 D=4 chi=16 state (six SR steps of
    # tau = 0.05 in FP64).  A chain's sweep differs as soon as one of its M decisions differs,
    # so the fraction F of differing chains gives the per-decision disagreement rate
    # f = -ln(1 - F) / M.  A decision flips when u falls between the two precisions'
    # acceptance probabilities, |q32 - q64| ~ 2 q |d log ratio| with |d log ratio| ~ 1e-3 on
    # such states: f <= 2e-3.
    L, D, chi, n = 8, 4, 16, 256
    N = L * L
    ref = _ctx(L, L, D, chi, n, prec=binding.PEPS_FP64, seed=87, mode=binding.PEPS_BLOCKS_BATCHED)
    ref.mc_sweep(2, p=1)
    for k in range(6):
        ref.step(n_sweeps=1, p=1 if k < 2 else 2, tau=0.05, eps=1e-4, max_cg=100, cg_tol=1e-10)
    S = ref.get_configs()
    tf = _ctx(L, L, D, chi, n, prec=binding.PEPS_TF32, seed=87)
    tf.set_theta(ref.get_theta())
    tf.set_configs(S)
    tf.sweeps_done = ref.sweeps_done
    ref.mc_sweep(1, p=2)
    tf.mc_sweep(1, p=2)
    diff = np.any(ref.get_configs() != tf.get_configs(), axis=1)
    # decisions per sweep: N both-flips, and of the 4 L (L - 1) exchanges (two layers on every
    # horizontal and vertical bond) the ones between unequal spins, about half
    M = N + 2 * L * (L - 1)
    F = float(np.mean(diff))
    f = -np.log(max(1e-12, 1.0 - min(F, 1.0 - 1.0 / n))) / M
    print(f"\nMetropolis: {int(diff.sum())} of {n} chains differ after one sweep (~{M} decisions "
          f"each): per-decision disagreement rate {f:.2e}")
    assert f <= 2e-3


def test_tf32_needs_batched_blocks():
    with pytest.raises(RuntimeError):
        _ctx(3, 3, 2, 4, 2, prec=binding.PEPS_TF32, mode=binding.PEPS_BLOCKS_NARROW)


def test_init_matches_oracle_bit_exact():
    L1, L2, D, n, seed = 4, 5, 3, 9, 1234
    lat = Lattice(L1, L2, D)
    ctx = _ctx(L1, L2, D, 9, n, seed=seed, noise=1e-3)
    assert np.array_equal(ctx.get_theta(), peps.init_theta(lat, seed, 1e-3))
    assert np.array_equal(ctx.get_configs(), peps.init_configs(lat, seed, n))
    assert ctx.Np == lat.Np and ctx.No == lat.No


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("p", [2, 1])
def test_mc_sweep_matches_oracle(p, mode):
    L1, L2, D, chi, J2, n = 4, 4, 2, 4, 0.3, 16
    lat = Lattice(L1, L2, D, J1=1.0, J2=J2)
    th = wl.random_theta(L1, L2, D, seed=7, scale=0.4, diag_bias=1.0)
    S0 = wl.random_configs(L1, L2, n, seed=8, diagonal_fraction=0.7)
    seed = 99
    ctx = _ctx(L1, L2, D, chi, n, J2=J2, seed=seed, n_blocks=5, mode=mode)
    ctx.set_theta(th)
    ctx.set_configs(S0)
    ctx.sweeps_done = 3
    ctx.mc_sweep(2, p)
    got = ctx.get_configs()
    mismatch = 0
    for k in range(n):
        Sk = S0[k]
        for sw in (3, 4):
            Sk, _, _ = sampler.mc_sweep(lat, th, Sk, chi, p, seed, k, sw)
        mismatch += int(not np.array_equal(Sk, got[k]))
    assert mismatch == 0
    assert ctx.sweeps_done == 5


@pytest.mark.parametrize("mode", [binding.PEPS_BLOCKS_NARROW, binding.PEPS_BLOCKS_BATCHED])
def test_mc_sweep_truncated_chi_matches_oracle(mode):
    L1, L2, D, chi, n = 4, 4, 3, 4, 6
    lat = Lattice(L1, L2, D)
    th = wl.random_theta(L1, L2, D, seed=17, scale=0.4, diag_bias=1.0)
    S0 = wl.random_configs(L1, L2, n, seed=18)
    ctx = _ctx(L1, L2, D, chi, n, seed=5, mode=mode)
    ctx.set_theta(th)
    ctx.set_configs(S0)
    ctx.mc_sweep(1, 2)
    got = ctx.get_configs()
    for k in range(n):
        Sk, _, _ = sampler.mc_sweep(lat, th, S0[k], chi, 2, 5, k, 0)
        assert np.array_equal(Sk, got[k]), k


@pytest.mark.parametrize("p", [2, 1])
def test_sr_step_matches_oracle(p):
    L1, L2, D, chi, J2, n = 3, 3, 2, 4, 0.5, 40
    lat = Lattice(L1, L2, D, J1=1.0, J2=J2)
    th = wl.random_theta(L1, L2, D, seed=21, scale=0.3, diag_bias=1.0)
    S = wl.random_configs(L1, L2, n, seed=22)
    ctx = _ctx(L1, L2, D, chi, n, J2=J2)
    # one step of tau0 first, so that the compared step reports at beta_obs = 4 tau0 != 0
    # (C and chi carry beta_obs factors), then back to the test state
    tau0 = 0.3
    ctx.eval_chains()
    ctx.sr_step(tau0, eps=1e-2, max_cg=5, cg_tol=1e-6, p=p)
    ctx.set_theta(th)
    ctx.set_configs(S)
    ctx.eval_chains()
    tau, eps, tol = 0.05, 1e-3, 1e-12
    st = ctx.sr_step(tau, eps=eps, max_cg=500, cg_tol=tol, p=p)
    th_gpu = ctx.get_theta()
    res = [peps.eval_sample(lat, th, S[k], chi) for k in range(n)]
    la = np.array([r['log_abs'] for r in res])
    es = np.array([r['e_sys'] for r in res])
    ea = np.array([r['e_anc'] for r in res])
    O = np.array([r['O'] for r in res])
    th_or, x, g, it, resid = sr.sr_step(lat, th, S, la, es, ea, O, p, tau, eps, tol, 500)
    w = sr.weights(la, p)
    Of = sr.expand_O(lat, S, O)
    obar, _, _ = sr.sr_quantities(Of, w, es + ea)
    xd = np.linalg.solve(sr.dense_G(Of, w, obar, eps), g)
    x_gpu = (th - th_gpu) / tau
    assert np.max(np.abs(x_gpu - xd)) <= 1e-8 * np.max(np.abs(xd))
    assert np.max(np.abs(x_gpu - x)) <= 1e-8 * np.max(np.abs(xd))
    assert st['cg_resid'] <= tol and not st['cg_maxit']
    assert abs(st['cg_iters'] - it) <= 2
    o = obs_mod.observables(lat, tau0, w, es, ea, S)
    assert st['beta_obs'] == pytest.approx(4 * tau0, rel=1e-15)
    assert st['E_site'] == pytest.approx(o['E_site'], rel=1e-10, abs=1e-12)
    # specific heat, susceptibility and the standard error of E (Eqs. 11, 13; weighted for
    # p = 1, Eq. A1), all float64 reductions: 1e-10 relative
    assert o['C_site'] > 0 and o['chi'] > 0 and o['E_err'] > 0
    assert st['C_site'] == pytest.approx(o['C_site'], rel=1e-10)
    assert st['chi_sus'] == pytest.approx(o['chi'], rel=1e-10)
    assert st['E_err'] == pytest.approx(o['E_err'], rel=1e-10)
    assert st['diag_frac'] == pytest.approx(o['diag_frac'])


@pytest.mark.parametrize("prec", [binding.PEPS_FP32, binding.PEPS_TF32])
@pytest.mark.parametrize("shape", [(4, 2, 4, 256), (3, 3, 4, 300)])
def test_sr_step_float_o_rows_match_oracle(prec, shape):
    # Float32 O rows (16-byte vector passes when every site slice holds a multiple of four
    # entries, as at D=2 on 4x4; element passes at D=3): the SR update from the GPU's own
    # evaluation against the oracle's SR step on those same float values.  The O passes widen
    # every float32 entry and multiply and sum in float64, so both sides solve the same
    # float64 system: CG to 1e-12 on both.  A CG iterate with relative residual tol lies
    # within cond(G + eps) * tol of the solution, so both are compared with the dense solve
    # at 4 cond * tol relative (cond ~ 1e3-1e4 here, so ~1e-8).
    L, D, chi, n = shape
    lat = Lattice(L, L, D, J1=1.0)
    th = wl.random_theta(L, L, D, seed=31, scale=0.3, diag_bias=1.0)
    S = wl.random_configs(L, L, n, seed=32)
    ctx = _ctx(L, L, D, chi, n, prec=prec, mode=binding.PEPS_BLOCKS_BATCHED)
    ctx.set_theta(th)
    ctx.set_configs(S)
    la, sg, es, ea, O = ctx.eval_batch(S)
    ctx.eval_chains()
    tau, eps, tol = 0.05, 1e-1, 1e-12
    st = ctx.sr_step(tau, eps=eps, max_cg=500, cg_tol=tol, p=2)
    assert st['cg_resid'] <= tol and not st['cg_maxit']
    x_gpu = (th - ctx.get_theta()) / tau
    O = O.astype(np.float64)
    _, x, g, it, resid = sr.sr_step(lat, th, S, la, es, ea, O, 2, tau, eps, tol, 500)
    assert resid <= tol
    w = sr.weights(la, 2)
    Of = sr.expand_O(lat, S, O)
    obar, _, _ = sr.sr_quantities(Of, w, es + ea)
    Gm = sr.dense_G(Of, w, obar, eps)
    xd = np.linalg.solve(Gm, g)
    bound = 4 * np.linalg.cond(Gm) * tol * np.max(np.abs(xd))
    assert np.max(np.abs(x_gpu - xd)) <= bound
    assert np.max(np.abs(x - xd)) <= bound
    # at 1e-12 on a system of condition ~1e6 the two sides may need a few more or fewer steps
    assert abs(st['cg_iters'] - it) <= max(2, 0.05 * it)


@pytest.mark.parametrize("prec", [binding.PEPS_FP64, binding.PEPS_FP32])
def test_cg_product_forms_agree(prec):
    # the fused single-read product and the two streaming passes solve the same float64
    # system with different summation orders: after CG to 1e-12, x equal to 1e-10 relative;
    # the passes over a float64 copy of float32 rows (mode 3, the automatic choice there)
    # widen each entry exactly as the passes over the rows do, in the same order: same bits
    L, D, chi, n = 4, 2, 4, 700
    th = wl.random_theta(L, L, D, seed=51, scale=0.3, diag_bias=1.0)
    S = wl.random_configs(L, L, n, seed=52)
    xs = []
    for mode in (1, 2, 3, 0):
        ctx = _ctx(L, L, D, chi, n, prec=prec, mode=binding.PEPS_BLOCKS_BATCHED)
        ctx.set_cg_product(mode)
        ctx.set_theta(th)
        ctx.set_configs(S)
        ctx.eval_chains()
        st = ctx.sr_step(0.05, eps=1e-2, max_cg=500, cg_tol=1e-12, p=1)
        assert st['cg_resid'] <= 1e-12
        xs.append((th - ctx.get_theta()) / 0.05)
        ctx.close()
    assert np.max(np.abs(xs[0] - xs[1])) <= 1e-10 * max(1.0, np.max(np.abs(xs[1])))
    assert np.array_equal(xs[2], xs[3])
    if prec != binding.PEPS_FP64:
        assert np.array_equal(xs[1], xs[2])
    with pytest.raises(binding.PepsError):
        _ctx(3, 3, 2, 4, 4).set_cg_product(4)


def test_sr_step_cg_maxit_warning_and_observables():
    L1, L2, D, chi, n = 3, 3, 2, 4, 24
    lat = Lattice(L1, L2, D)
    th = wl.random_theta(L1, L2, D, seed=31, scale=0.3, diag_bias=1.0)
    S = wl.random_configs(L1, L2, n, seed=32)
    ctx = _ctx(L1, L2, D, chi, n)
    ctx.set_theta(th)
    ctx.set_configs(S)
    ctx.eval_chains()
    ob = ctx.observables(p=2)
    res = [peps.eval_sample(lat, th, S[k], chi, with_O=False) for k in range(n)]
    es = np.array([r['e_sys'] for r in res])
    ea = np.array([r['e_anc'] for r in res])
    o = obs_mod.observables(lat, 0.0, np.full(n, 1.0 / n), es, ea, S)
    assert ob['E_site'] == pytest.approx(o['E_site'], rel=1e-10, abs=1e-12)
    st = ctx.sr_step(0.01, eps=1e-4, max_cg=2, cg_tol=1e-14, p=2)
    assert st['cg_maxit'] and st['cg_iters'] == 2


def test_errors_and_edge_cases():
    ctx = _ctx(3, 3, 2, 4, 4)
    with pytest.raises(binding.PepsError) as e:
        ctx.sr_step(0.01)
    assert e.value.code == binding.PEPS_ESTATE
    bad = np.full((4, 9), 5, np.uint8)
    with pytest.raises(binding.PepsError) as e:
        ctx.set_configs(bad)
    assert e.value.code == binding.PEPS_EINVAL
    with pytest.raises(binding.PepsError):
        ctx.mc_sweep(1, p=3)
    la, sg, es, ea, O = ctx.eval_batch(np.zeros((0, 9), np.uint8))
    assert la.size == 0
    # configuration entries above 3 are rejected before any evaluation, for host batches
    # (checked on the host) and device batches (checked by a kernel), in both engines
    import torch
    for mode in (binding.PEPS_BLOCKS_NARROW, binding.PEPS_BLOCKS_BATCHED):
        cm = _ctx(3, 3, 2, 4, 4, mode=mode)
        bad = np.zeros((2, 9), np.uint8)
        bad[1, 4] = 4
        with pytest.raises(binding.PepsError) as e:
            cm.eval_batch(bad)
        assert e.value.code == binding.PEPS_EINVAL
        dev = torch.device("cuda:0")
        outs = [torch.empty(2, dtype=torch.float64, device=dev), torch.empty(2, dtype=torch.int8, device=dev),
                torch.empty(2, dtype=torch.float64, device=dev), torch.empty(2, dtype=torch.float64, device=dev)]
        with pytest.raises(binding.PepsError) as e:
            cm.eval_batch_device(torch.from_numpy(bad).to(dev), *outs)
        assert e.value.code == binding.PEPS_EINVAL
        cm.eval_batch_device(torch.from_numpy(np.zeros((2, 9), np.uint8)).to(dev), *outs)
        assert np.all(np.isfinite(outs[0].cpu().numpy()))
        cm.close()
    # beta = 0 state with no noise: rho = 1 on diagonal configurations, 0 elsewhere
    ctx0 = _ctx(3, 3, 2, 4, 4, noise=0.0)
    S = np.array([[0] * 9, [3] * 9, [0, 3, 0, 3, 3, 0, 0, 0, 3], [1] + [0] * 8], np.uint8)
    la, sg, es, ea, _ = ctx0.eval_batch(S, with_O=False)
    assert np.allclose(la[:3], 0.0, atol=1e-14) and list(sg) == [1, 1, 1, 0]


def test_checkpoint_resume_is_bit_exact(tmp_path):
    L1, L2, D, chi, n = 3, 3, 2, 4, 16
    a = _ctx(L1, L2, D, chi, n, J2=0.5, seed=11, noise=1e-2)
    a.mc_sweep(2, p=1)
    a.step(n_sweeps=1, p=1, tau=0.02)
    ck = tmp_path / "state.ckpt"
    a.checkpoint(ck)
    for _ in range(2):
        a.step(n_sweeps=1, p=2, tau=0.02)
    b = _ctx(L1, L2, D, chi, n, J2=0.5, seed=11, noise=1e-2)
    b.restore(ck)
    assert b.t == pytest.approx(0.02) and b.sweeps_done == 3
    for _ in range(2):
        b.step(n_sweeps=1, p=2, tau=0.02)
    assert np.array_equal(a.get_theta(), b.get_theta())
    assert np.array_equal(a.get_configs(), b.get_configs())
    # a corrupted or foreign checkpoint is rejected and leaves the context as it was
    raw = bytearray(ck.read_bytes())
    raw[200] ^= 0x40
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(bytes(raw))
    th = b.get_theta()
    with pytest.raises(binding.PepsError) as e:
        b.restore(bad)
    assert e.value.code == binding.PEPS_ECORRUPT
    assert np.array_equal(th, b.get_theta())
    other = _ctx(L1, L2, D, chi + 1, n, J2=0.5)
    with pytest.raises(binding.PepsError) as e:
        other.restore(ck)
    assert e.value.code == binding.PEPS_ECORRUPT


@pytest.mark.parametrize("mode", [binding.PEPS_BLOCKS_NARROW, binding.PEPS_BLOCKS_BATCHED])
@pytest.mark.parametrize("prec", [binding.PEPS_FP64, binding.PEPS_FP32])
def test_eval_with_cached_up_environments_is_identical(prec, mode):
    # eval_chains after a sweep reuses the sweep's up environments; the values must be the
    # same bits as an evaluation of the same configurations from scratch.
    L1, L2, D, chi, n = 5, 4, 3, 4, 12
    ctx = _ctx(L1, L2, D, chi, n, J2=0.5, prec=prec, seed=3, noise=0.05, mode=mode)
    ctx.mc_sweep(2, p=2)
    S = ctx.get_configs()
    la0, sg0, es0, ea0, O0 = ctx.eval_batch(None)
    la1, sg1, es1, ea1, O1 = ctx.eval_batch(S)
    assert np.array_equal(la0, la1) and np.array_equal(sg0, sg1)
    assert np.array_equal(es0, es1) and np.array_equal(ea0, ea1) and np.array_equal(O0, O1)
