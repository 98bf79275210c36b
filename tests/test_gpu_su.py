"""The device simple-update warm start (peps_su_warm_start, App. A) against the oracle's
simple update (pinned to ED in tests/test_oracle_simple_update.py) and against the host
version (peps_su_theta), through gauge-invariant amplitudes, wherever the truncation cuts
between distinct singular values (D = 4: the bond spectra are a singlet and a triplet)."""
import numpy as np
import pytest

from oracle import ed, peps, simple_update as su
from oracle.lattice import Lattice
from paper_2409_05285_gb300 import binding
from paper_2409_05285_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2409_05285_gb300.build import build
    build()


def _oracle_theta(lat, tau, n):
    st = su.SUState(lat)
    for _ in range(n):
        su.su_step(st, tau, lat.D)
    return su.to_theta(st)


def _unit(v):
    return v / np.linalg.norm(v)


def _device_theta(L1, L2, D, J1, tau, n):
    ctx = binding.Context(L1, L2, D, max(1, D * D), 4, J1=J1, precision=binding.PEPS_FP64, seed=1)
    ctx.su_warm_start(tau, n)
    th, t = ctx.get_theta(), ctx.t
    ctx.close()
    assert t == pytest.approx(n * tau, rel=1e-15)
    return th


@pytest.mark.parametrize("shape,n", [((2, 2), 10), ((2, 3), 12), ((3, 2), 7)])
def test_device_su_matches_oracle_on_every_configuration(shape, n):
    lat = Lattice(*shape, 4)
    th = _device_theta(lat.nrow, lat.ncol, 4, 1.0, 0.02, n)
    tho = _oracle_theta(lat, 0.02, n)
    cfgs = [ed.config_of_index(k, lat.N) for k in range(4 ** lat.N)]
    v = np.array([peps.amplitude_exact(lat, th, S) for S in cfgs])
    w = np.array([peps.amplitude_exact(lat, tho, S) for S in cfgs])
    assert np.allclose(_unit(v), _unit(w), atol=1e-12)


def test_device_su_matches_host_su_8x8():
    # the bench workload's lattice: every amplitude of 64 sampled configurations, evaluated
    # exactly enough by the FP64 boundary MPS at chi = 16 on both parameter vectors
    L, D = 8, 4
    th_d = _device_theta(L, L, D, 1.0, 0.01, 15)
    th_h = binding.su_theta(L, L, D, 1.0, 0.01, 15)
    S = wl.random_configs(L, L, 64, seed=41, diagonal_fraction=0.8)
    ctx = binding.Context(L, L, D, 16, 64, precision=binding.PEPS_FP64, seed=1,
                          block_mode=binding.PEPS_BLOCKS_BATCHED)
    out = []
    for th in (th_d, th_h):
        ctx.set_theta(th)
        out.append(ctx.eval_batch(S, with_O=False))
    la_d, sg_d = out[0][:2]
    la_h, sg_h = out[1][:2]
    keep = la_h > la_h.max() - 30.0
    assert keep.sum() >= 40
    assert np.array_equal(sg_d[keep], sg_h[keep])
    assert np.max(np.abs(la_d - la_h)[keep]) <= 1e-9
    ctx.close()


def test_device_su_zero_steps_and_arguments():
    lat = Lattice(3, 4, 3)
    th = _device_theta(3, 4, 3, 1.0, 0.05, 0)
    assert np.array_equal(th, peps.init_theta(lat, 0, 0.0))
    ctx = binding.Context(3, 3, 2, 4, 4, J1=1.0, J2=0.5, precision=binding.PEPS_FP64)
    with pytest.raises(binding.PepsError) as e:
        ctx.su_warm_start(0.01, 2)
    assert e.value.code == binding.PEPS_EINVAL
    ctx.close()
